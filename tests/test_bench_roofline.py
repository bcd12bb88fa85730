"""bench.py's roofline arithmetic and its use of the committed DRAM summary (host logic, no GPU).

- The dominant pass is chosen with its helper launches: a trace with the packing
  of its input, the dt pass with its verifying launch, an integration with its
  general pass; achieved = algorithmic bytes per cell x cells / that pass's time.
- `traffic` is read from the profile only while the kernel-source hash and the
  tile shape recorded there match the running build."""
import bench


def test_dominant_pass_includes_its_helper_launches():
    prof = {"pack": 0.5, "sweep1": 20.0, "ratedt": 8.0, "ratedt_verify": 0.01, "half": 2.5, "half_general": 3.0,
            "sweep2": 19.9, "full": 8.0, "full_general": 4.5, "final0": 0.1, "final1": 0.01}
    r = bench._roofline(prof, ms_per_step=70.0, ncell=1000, nsrc=16, n_array=True, workload="none", tile_shape=7)
    assert r["kernel"].startswith("sweep1")
    assert r["kernel_ms"] == 20.5                                  # the trace with its pack
    assert r["bytes_per_cell"] == 16 * 12                          # x, n read and N written per source
    assert abs(r["achieved"] - 192 * 1000 / 20.5e-3 / 1e9) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    assert r["step_bytes_per_cell"] == 28 * 16 + 32
    assert r["traffic"] is None                                    # no profile for this workload
    # an integration with a slow general pass dominates as the pair
    prof2 = dict(prof, full=15.0, full_general=10.0)
    r2 = bench._roofline(prof2, 80.0, 1000, 16, True, "none", 7)
    assert r2["kernel"].startswith("full") and r2["kernel_ms"] == 25.0


def test_traffic_needs_matching_sources_and_tile_shape(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic_w.md").write_text(
        "kernel sources sha1: `abc`\n\ntile shape: 7 (8x8x8)\n\n| launch | read | write |\n|---|---|---|\n"
        "| pack | 10 | 5 |\n| sweep1 | 100 | 50 |\n| full | 7 | 1 |\n| full_general | 2 | 1 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench._traffic("w", ["sweep1", "pack"], 7) == 165.0
    assert bench._traffic("w", ["full", "full_general"], 7) == 11.0
    assert bench._traffic("w", ["sweep1", "pack"], 8) is None      # captured on another tile shape
    assert bench._traffic("w", ["ratedt"], 7) is None              # no row for it
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "def")
    assert bench._traffic("w", ["sweep1", "pack"], 7) is None      # kernels changed since the capture

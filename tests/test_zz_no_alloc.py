"""The allocation-free trace entry point (oots_trace_noalloc), for callers
that cannot allocate device memory (code inside a fixed memory arena, or a
host whose allocator must not be re-entered):
through the C ABI it must give the same entry columns as the context API's
trace, on two calls in a row sharing its static scratch.

Kept in a file of its own that pytest collects last, so a failure here stops
a -x run only after every other test has run."""
import numpy as np
import pytest

from paper_1201_5651_gb300 import inputs, oots

pytestmark = pytest.mark.gpu


def _reference_columns(w, precision):
    c = oots.Context.from_workload(w, precision, scheme=oots.OOTS_A3, K4=0.25)
    c.compute_dt()                       # the existing entry point's first trace
    return c.get_column_density(0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_trace_matches_context_trace(precision):
    torch = pytest.importorskip("torch")
    dtype = torch.float64 if precision == "fp64" else torch.float32
    prec = oots.OOTS_FP64 if precision == "fp64" else oots.OOTS_MIXED
    tol = 1e-12 if precision == "fp64" else 1e-6
    for seed, (n, ny, nz), pos in [(41, (21, 13, 17), (5.0, 13.0, 8.4)), (42, (24, 24, 24), (12.0, 12.0, 12.0))]:
        w = inputs.small_random(n=n, ny=ny, nz=nz, seed=seed)
        w.sources[0].pos = pos
        ref = _reference_columns(w, precision)
        x = torch.from_numpy(w.x0.ravel()).to(device="cuda", dtype=dtype)
        nH = torch.from_numpy(w.nH.ravel()).to(device="cuda", dtype=dtype)
        out = torch.full((w.ncell,), -1.0, device="cuda", dtype=dtype)
        oots.oots_trace_noalloc(0, prec, w.nx, w.ny, w.nz, w.dx, nH.data_ptr(), 0.0, x.data_ptr(), pos,
                                w.sigma0, w.tau0, out.data_ptr())
        got = out.double().cpu().numpy().reshape(w.nz, w.ny, w.nx)
        rel = np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e10))
        assert rel <= tol, (seed, rel)


def test_noalloc_rejects_oversized_grid():
    torch = pytest.importorskip("torch")
    x = torch.zeros(8, device="cuda", dtype=torch.float64)
    with pytest.raises(oots.OotsError) as e:
        oots.oots_trace_noalloc(0, oots.OOTS_FP64, 1024, 1024, 1024, 1e16, None, 100.0, x.data_ptr(),
                                (512.0, 512.0, 512.0), 6.3e-18, 0.6, x.data_ptr())
    assert e.value.code == oots.OOTS_E_INVAL
    assert "static scratch" in str(e.value)

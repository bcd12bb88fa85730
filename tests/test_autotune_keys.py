"""The autotuner's plane-size classes and its JSON cache (host logic, no GPU).

A tuned tile shape is reused by every launch of the same class: grids whose
largest side rounds up to the same power of two, with the same bucket of
sources per grid and of grids per launch, on the same device and precision."""
import json

from paper_1201_5651_gb300 import autotune, oots


def test_plane_classes_bucket_sides_sources_and_grids():
    assert autotune.plane_class(512, 512, 512, 16) == "side512|S16|G1"
    assert autotune.plane_class(500, 200, 300, 16) == "side512|S16|G1"
    assert autotune.plane_class(513, 8, 8, 1) == "side1024|S1|G1"
    assert autotune.plane_class(128, 128, 128, 1) == "side128|S1|G1"
    assert autotune.plane_class(10, 12, 9, 1) == "side16|S1|G1"          # at least 16
    assert autotune.plane_class(128, 128, 128, 3) == "side128|S4|G1"
    assert autotune.plane_class(128, 128, 128, 64) == "side128|S64|G1"
    assert autotune.plane_class(128, 128, 128, 100) == "side128|S64|G1"  # beyond the last edge
    assert autotune.plane_class(128, 128, 128, 1, 64) == "side128|S1|G64"
    assert autotune.plane_class(96, 96, 96, 1, 9) == "side128|S1|G64"
    # a different class for each axis of the key
    keys = {autotune.plane_class(*a) for a in [(256, 256, 256, 1), (512, 512, 512, 1), (256, 256, 256, 16),
                                               (256, 256, 256, 1, 64)]}
    assert len(keys) == 4


def test_cache_keys_separate_devices_and_precisions(tmp_path):
    path = str(tmp_path / "tune.json")
    k = autotune.plane_class(512, 512, 512, 16)
    autotune._store(autotune.cache_key("GB300", oots.OOTS_MIXED, k), {"shape": 7, "dims": (8, 8, 8)}, path)
    autotune._store(autotune.cache_key("GB300", oots.OOTS_FP64, k), {"shape": 0, "dims": (16, 8, 8)}, path)
    autotune._store(autotune.cache_key("B200", oots.OOTS_MIXED, k), {"shape": 2, "dims": (16, 16, 16)}, path)
    assert autotune.lookup("GB300", oots.OOTS_MIXED, k, path) == 7
    assert autotune.lookup("GB300", oots.OOTS_FP64, k, path) == 0
    assert autotune.lookup("B200", oots.OOTS_MIXED, k, path) == 2
    assert autotune.lookup("GB300", oots.OOTS_MIXED, autotune.plane_class(128, 128, 128, 1), path) is None
    data = json.load(open(path))
    assert set(data) == {"GB300|mixed|side512|S16|G1", "GB300|fp64|side512|S16|G1", "B200|mixed|side512|S16|G1"}


class _FakeCtx:
    """Stands in for a context: records the tile shape and block size it is given; profiling is never reached."""

    def __init__(self, shape, precision):
        self.shape = shape
        self.precision = precision
        self.tile = None
        self.cell_block = None

    def set_tile_shape(self, s):
        self.tile = s

    def set_cell_block(self, b):
        self.cell_block = b

    def profile_substep(self):
        raise AssertionError("a cached class must not be re-timed")


def test_tune_reuses_a_cached_class_without_timing(tmp_path):
    path = str(tmp_path / "tune.json")
    k = autotune.plane_class(300, 512, 512, 16)
    autotune._store(autotune.cache_key("GB300", oots.OOTS_MIXED, k), {"shape": 7, "dims": (8, 8, 8)}, path)
    c = _FakeCtx((512, 512, 300), oots.OOTS_MIXED)       # (nz, ny, nx)
    assert autotune.tune(c, "GB300", 16, path=path) == 7
    assert c.tile == 7


def test_a_cached_class_also_sets_the_per_cell_block_size(tmp_path):
    """The block size of the closed-form passes is cached with the tile shape and
    applied with it; an entry without one leaves the library's default."""
    path = str(tmp_path / "tune.json")
    k = autotune.plane_class(512, 512, 512, 16)
    autotune._store(autotune.cache_key("GB300", oots.OOTS_MIXED, k), {"shape": 7, "cell_block": 128}, path)
    c = _FakeCtx((512, 512, 512), oots.OOTS_MIXED)
    assert autotune.tune(c, "GB300", 16, path=path) == 7
    assert (c.tile, c.cell_block) == (7, 128)
    assert autotune.lookup_cell_block("GB300", oots.OOTS_MIXED, k, path) == 128
    k1 = autotune.plane_class(128, 128, 128, 1)
    autotune._store(autotune.cache_key("GB300", oots.OOTS_MIXED, k1), {"shape": 2}, path)
    c1 = _FakeCtx((128, 128, 128), oots.OOTS_MIXED)
    assert autotune.tune(c1, "GB300", 1, path=path) == 2
    assert c1.cell_block is None
    assert autotune.lookup_cell_block("GB300", oots.OOTS_MIXED, k1, path) == 0

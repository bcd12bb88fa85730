"""CPU-only checks of the C ABI: the library builds, loads and exports every
symbol include/oots.h declares, and the host-only entry points behave."""
import ctypes
import os
import re

import pytest

from paper_1201_5651_gb300 import oots

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    text = open(os.path.join(ROOT, "include", "oots.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(oots_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert _header_functions() == sorted(oots.EXPORTS)


def test_library_loads_and_exports_everything():
    lib = oots.load()
    for name in _header_functions():
        assert hasattr(lib, name), name
    assert "sm_103a" in oots.oots_version()


def test_dtcrit_presets_follow_table1():
    """Table 1 with the energy criterion dropped (temperature fixed)."""
    k4 = [1, 1 / 2, 1 / 4, 1 / 8, 1 / 16]
    k1 = [1, 0.3, 0.1, 0.03, 0.003]
    for i in range(5):
        c = oots.oots_dtcrit_preset(i, oots.OOTS_A3)
        assert (c.K1, c.K3, c.K4) == (0, 0, k4[i])
        c = oots.oots_dtcrit_preset(i, oots.OOTS_A1)
        assert (c.K1, c.K3, c.K4) == (k1[i], 0, 0)
    for i in range(5, 9):
        for s in (oots.OOTS_A1, oots.OOTS_A2, oots.OOTS_A3):
            c = oots.oots_dtcrit_preset(i, s)
            assert (c.K1, c.K3, c.K4) == (0, 0, 1 / 2 ** (i - 4))
    for i in range(9, 13):
        c = oots.oots_dtcrit_preset(i, oots.OOTS_A2)
        assert (c.K1, c.K3, c.K4) == (0, 1 / 2 ** (i - 8), 0)
    with pytest.raises(oots.OotsError):
        oots.oots_dtcrit_preset(13, oots.OOTS_A3)


def test_tile_shapes():
    n, dims = oots.oots_tile_shape_info(0)
    assert n >= 4 and all(d > 0 for d in dims)
    with pytest.raises(oots.OotsError):
        oots.oots_tile_shape_info(n)


def test_null_arguments_are_rejected():
    lib = oots.load()
    assert lib.oots_create(None, 0, 0) == oots.OOTS_E_INVAL
    assert lib.oots_set_grid(None, 4, 4, 4, 1.0) == oots.OOTS_E_INVAL
    assert lib.oots_advance(None, 1.0, None, None) == oots.OOTS_E_INVAL
    assert lib.oots_destroy(None) == oots.OOTS_OK
    assert lib.oots_batch_create(None, None, 0) == oots.OOTS_E_INVAL
    assert lib.oots_batch_run_substeps(None, 1, None) == oots.OOTS_E_INVAL
    assert lib.oots_set_partition(None, 1, 0, 0) == oots.OOTS_E_INVAL
    assert lib.oots_run_phase(None, 0, None) == oots.OOTS_E_INVAL
    assert lib.oots_array_device(None, 0, 0, None, None) == oots.OOTS_E_INVAL
    h = ctypes.c_void_p()
    assert lib.oots_create(ctypes.byref(h), 0, 7) == oots.OOTS_E_INVAL
    assert lib.oots_add_plane_source(None, 0, 1, 1e9, oots.OOTS_MONO, 0.0, None) == oots.OOTS_E_INVAL

"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every function include/hydro.h declares, and rejects bad arguments before any
device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import paper_1604_03360_gb300.build as B
    B.build()
    import paper_1604_03360_gb300 as H
    return H.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hydro_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_version(L):
    assert b"sm_103a" in L.hydro_version()


@pytest.mark.parametrize("field,value,msg", [
    ("scheme", 6, b"scheme"), ("cs2", 1.0, b"cs2"), ("weno_eps", 0.0, b"weno_eps"),
    ("weno_eps", 1e-41, b"weno_eps"), ("weno_eps", 1e31, b"weno_eps"), ("weno_eps", float("nan"), b"weno_eps"),
    ("split", 2, b"split"), ("charwise", 2, b"charwise"), ("eos_mass", -1.0, b"eos_mass"),
])
def test_invalid_config_rejected(L, field, value, msg):
    import paper_1604_03360_gb300 as H
    c = H.make_config((8, 8, 8), (0.1, 0.1, 0.1))
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert L.hydro_create(ctypes.byref(c), None, ctypes.byref(h)) == H._binding.ERR_INVALID_ARG
    assert msg in L.hydro_last_error(None)


def test_invalid_grid_rejected(L):
    import paper_1604_03360_gb300 as H
    for n, dx, bc in [((0, 4, 4), (1, 1, 1), (0, 0, 0)), ((8, 8, 8), (1, -1, 1), (0, 0, 0)),
                      ((8, 2, 8), (1, 1, 1), (0, 1, 0)), ((8, 8, 8), (1, 1, 1), (0, 2, 0))]:
        c = H.make_config(n, dx, bc=bc)
        h = ctypes.c_void_p()
        assert L.hydro_create(ctypes.byref(c), None, ctypes.byref(h)) == H._binding.ERR_INVALID_ARG
    assert L.hydro_create(None, None, ctypes.byref(ctypes.c_void_p())) == H._binding.ERR_INVALID_ARG


def test_null_handle_calls_fail_cleanly(L):
    assert L.hydro_step(None, 1, -1.0) == 1
    assert L.hydro_sync(None) == 1
    assert L.hydro_destroy(None) == 0
    assert L.hydro_field_stride(None) == 0
    assert L.hydro_kernels_per_step(None) == 0
    assert L.hydro_batch_kernels_per_step(None) == 0


def test_charwise_needs_weno_with_global_splitting(L):
    import paper_1604_03360_gb300 as H
    for kw in (dict(split=1), dict(scheme=2)):
        c = H.make_config((8, 8, 8), (0.1, 0.1, 0.1), charwise=1, **kw)
        h = ctypes.c_void_p()
        assert L.hydro_create(ctypes.byref(c), None, ctypes.byref(h)) == H._binding.ERR_INVALID_ARG
        assert b"characteristic" in L.hydro_last_error(None)
    for scheme, nq, n in ((5, 1, 5), (7, 1, 4), (5, 3, 4), (7, 2, 4)):
        c = H.make_config((8, 8, 8), (0.1, 0.1, 0.1), scheme=scheme, nq=nq, charwise=1)
        assert L.hydro_launch_variants_cfg(ctypes.byref(c)) == n


def test_launch_variant_counts(L):
    """Compiled stage-kernel variants per scheme and splitting (WENO5 and WENO7
    with global LF: per-face tiles, pencil sweeps, z-pass sweeps; local LF:
    per-face tiles; several charges: the 16x8 stage kernel and the three-pass
    launch; MUSTA-FORCE: two tiles); 0 for an unknown scheme."""
    for scheme, split, nq, n in ((5, 0, 1, 15), (7, 0, 1, 18), (5, 1, 1, 5), (7, 1, 1, 4), (2, 0, 1, 2),
                                 (5, 0, 3, 2), (7, 1, 2, 2), (9, 0, 1, 0)):
        assert L.hydro_launch_variants(scheme, split, nq) == n, (scheme, split, nq)


def test_halo_slab_needs_g_planes(L):
    import paper_1604_03360_gb300 as H
    for scheme, nz in ((5, 2), (7, 3), (2, 1)):
        c = H.make_config((8, 8, nz), (0.1, 0.1, 0.1), scheme=scheme, bc=(0, 0, H.BC_HALO))
        h = ctypes.c_void_p()
        assert L.hydro_create(ctypes.byref(c), None, ctypes.byref(h)) == H._binding.ERR_INVALID_ARG
        assert b"halo" in L.hydro_last_error(None)
    c = H.make_config((8, 8, 8), (0.1, 0.1, 0.1), bc=(H.BC_HALO, 0, 0))
    assert L.hydro_create(ctypes.byref(c), None, ctypes.byref(ctypes.c_void_p())) == H._binding.ERR_INVALID_ARG

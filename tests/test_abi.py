"""The C-ABI library builds, loads, exports every declared symbol, and rejects bad input on
the host before touching the GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2409_15116_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2409_15116_gb300 import binding
    return binding.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bse.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bse_[a-z_]+)\s*\(", txt)))


def test_header_and_binding_agree(lib):
    from paper_2409_15116_gb300 import binding
    assert declared_symbols() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = os.popen(f"nm -D --defined-only {B.LIB}").read()
    exported = set(re.findall(r"\bT (bse_\w+)", out))
    for name in declared_symbols():
        assert name in exported, name


from paper_2409_15116_gb300.binding import ALLOC_FN, FREE_FN  # noqa: E402

_NOALLOC, _NOFREE = ALLOC_FN(), FREE_FN()


def test_allocator_callbacks_come_in_pairs(lib):
    """bse_create takes the caller's allocator as a pair: one callback without the other is
    rejected before any device work (no context is returned)."""
    from synth import make_tiny
    s, keep = _system(make_tiny(0))
    h = C.c_void_p()
    only_alloc = ALLOC_FN(lambda n, u: None)
    only_free = FREE_FN(lambda p, u: None)
    assert lib.bse_create(C.byref(s), 0, only_alloc, _NOFREE, None, C.c_void_p(0), C.byref(h)) == -1
    assert h.value is None
    assert lib.bse_create(C.byref(s), 0, _NOALLOC, only_free, None, C.c_void_p(0), C.byref(h)) == -1
    assert h.value is None


def test_version_string(lib):
    assert b"sm_103a" in lib.bse_version()


def _system(inst, **over):
    from paper_2409_15116_gb300.binding import System
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_int32 if dt == np.int32 else C.c_double))

    f = dict(n_grid=inst.n_grid, L=inst.L, n_half=inst.n_half, miller=inst.miller,
             n_occ=inst.n_occ, psi=inst.psi, eps=inst.eps, v_loc=inst.v_loc,
             scissor=inst.scissor, n_pdep=inst.n_pdep, pdep=inst.pdep, lam=inst.lam,
             overlap_thr=inst.overlap_thr, keep_pairs=inst.keep_pairs, spin=inst.spin)
    f.update(over)
    s = System(n_grid=f["n_grid"], L=f["L"], n_half=f["n_half"], miller=arr(f["miller"], np.int32),
               n_occ=f["n_occ"], psi=arr(f["psi"], np.float64), eps=arr(f["eps"], np.float64),
               v_loc=arr(f["v_loc"], np.float64), scissor=f["scissor"], n_pdep=f["n_pdep"],
               pdep=arr(f["pdep"], np.float64), lam=arr(f["lam"], np.float64),
               overlap_thr=f["overlap_thr"], keep_pairs=f["keep_pairs"], spin=f["spin"])
    return s, keep


@pytest.mark.parametrize("case,code", [
    ("grid", -1), ("alias", -1), ("pad", -1), ("nan", -4), ("pdep_g0", -1), ("lam", -1),
    ("rule", -1), ("spin", -1)])
def test_create_rejects_bad_input_on_host(lib, case, code):
    from synth import make_tiny
    inst = make_tiny(0)
    over = {}
    if case == "grid":
        over["n_grid"] = 17
    elif case == "alias":
        m = inst.miller.copy(); m[5] = (7, 0, 0); over["miller"] = m
    elif case == "pad":
        p = inst.psi.copy(); p[0, 1] = 1e-3; over["psi"] = p
    elif case == "nan":
        v = inst.v_loc.copy(); v[3] = np.nan; over["v_loc"] = v
    elif case == "pdep_g0":
        p = inst.pdep.copy(); p[0, 0] = 0.1; over["pdep"] = p
    elif case == "lam":
        l_ = inst.lam.copy(); l_[0] = 1.0; over["lam"] = l_
    elif case == "rule":
        over["overlap_thr"] = 0.0; over["keep_pairs"] = 0
    elif case == "spin":
        over["spin"] = 3
    s, keep = _system(inst, **over)
    h = C.c_void_p()
    rc = lib.bse_create(C.byref(s), 0, _NOALLOC, _NOFREE, None, C.c_void_p(0), C.byref(h))
    assert rc == code
    assert h.value is not None
    msg = lib.bse_last_error(h)
    assert msg and msg != b"no error"
    lib.bse_destroy(h)


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.bse_create(None, 0, _NOALLOC, _NOFREE, None, C.c_void_p(0), C.byref(h)) == -1
    assert lib.bse_build_tau(None, None, None) == -1
    assert lib.bse_apply_liouville(None, 1, None, None) == -1
    assert lib.bse_davidson(None, None, None, None, None) == -1
    assert lib.bse_last_error(None) == b"null context"
    lib.bse_destroy(None)

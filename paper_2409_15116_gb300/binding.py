"""Thin ctypes binding of the C ABI declared in include/bse.h (argument marshalling only).

Every step of the hot path runs in the CUDA library; this module converts host arrays
to the ``bse_system`` struct, passes device pointers of torch tensors, and raises on
non-zero status codes. It fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbse.so")

BSE_OK = 0
BSE_ERR_NOT_CONVERGED = -5
STATUS = {0: "BSE_OK", -1: "BSE_ERR_INVALID_ARG", -2: "BSE_ERR_CUDA", -3: "BSE_ERR_OOM",
          -4: "BSE_ERR_NUMERIC", -5: "BSE_ERR_NOT_CONVERGED", -6: "BSE_ERR_TIMEOUT",
          -7: "BSE_ERR_STATE"}
PREC_FP64, PREC_MIXED = 0, 1

# every symbol include/bse.h declares
EXPORTS = ["bse_create", "bse_build_tau", "bse_get_pairs", "bse_get_overlaps",
           "bse_apply_liouville", "bse_davidson", "bse_last_error", "bse_version",
           "bse_destroy", "bse_profile", "bse_profile_read", "bse_apply_liouville_static",
           "bse_precond_collect", "bse_precond_set_samples", "bse_precond_grad",
           "bse_precond_train", "bse_precond_load", "bse_solve_batch", "bse_lanczos",
           "bse_lanczos_spectrum", "bse_localize", "bse_precond_get_samples"]
NPARAM = 4619


class BseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class System(C.Structure):
    _fields_ = [("n_grid", C.c_int), ("L", C.c_double), ("n_half", C.c_int),
                ("miller", C.POINTER(C.c_int32)), ("n_occ", C.c_int),
                ("psi", C.POINTER(C.c_double)), ("eps", C.POINTER(C.c_double)),
                ("v_loc", C.POINTER(C.c_double)), ("scissor", C.c_double),
                ("n_pdep", C.c_int), ("pdep", C.POINTER(C.c_double)),
                ("lam", C.POINTER(C.c_double)), ("overlap_thr", C.c_double),
                ("keep_pairs", C.c_int64), ("spin", C.c_int), ("n_qp", C.c_int),
                ("qp_psi", C.POINTER(C.c_double)), ("qp_eps_ks", C.POINTER(C.c_double)),
                ("qp_eps", C.POINTER(C.c_double)), ("n_up", C.c_int)]


class ProfEntry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("calls", C.c_int64), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double)]


class DavidsonOpts(C.Structure):
    _fields_ = [("n_eig", C.c_int), ("block", C.c_int), ("max_sub", C.c_int),
                ("max_it", C.c_int), ("res_tol", C.c_double), ("precond", C.c_int)]


class DavidsonStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("n_apply", C.c_int), ("ms_total", C.c_double),
                ("ms_apply", C.c_double), ("res_max", C.c_double),
                ("precond_fallbacks", C.c_int)]


# caller-supplied device allocator of bse_create (include/bse.h: bse_alloc_fn, bse_free_fn)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class TorchAllocator:
    """Device memory of one context from PyTorch's caching allocator, bound to the context
    stream (so a block the library frees is reused only by work ordered after it on that
    stream). Records the blocks it hands out: ``live`` (pointer -> bytes) and ``total``."""

    def __init__(self, stream_handle: int, device: int):
        import torch
        self.stream = int(stream_handle)
        self.device = int(device)
        self.live = {}
        self.total = 0
        self.calls = 0

        def _alloc(nbytes, _user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:       # out of memory: the library reports BSE_ERR_OOM
                return None
            self.live[int(p)] = int(nbytes)
            self.total += int(nbytes)
            self.calls += 1
            return int(p)

        def _free(ptr, _user):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))
                self.live.pop(int(ptr), None)

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


_lib = None


def load(path: str = LIB_PATH):
    """Load libbse.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_2409_15116_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.bse_create.argtypes = [C.POINTER(System), C.c_int, ALLOC_FN, FREE_FN, P, P, C.POINTER(P)]
    lib.bse_build_tau.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
    lib.bse_get_pairs.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.bse_get_overlaps.argtypes = [P, C.POINTER(C.c_double)]
    lib.bse_apply_liouville.argtypes = [P, C.c_int, P, P]
    lib.bse_apply_liouville_static.argtypes = [P, C.c_int, P, P]
    lib.bse_davidson.argtypes = [P, C.POINTER(DavidsonOpts), C.POINTER(C.c_double), P,
                                 C.POINTER(DavidsonStats)]
    lib.bse_last_error.argtypes = [P]
    lib.bse_last_error.restype = C.c_char_p
    lib.bse_version.restype = C.c_char_p
    lib.bse_profile.argtypes = [P, C.c_int]
    lib.bse_profile_read.argtypes = [P, C.POINTER(ProfEntry), C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int64)]
    D = C.POINTER(C.c_double)
    F = C.POINTER(C.c_float)
    lib.bse_precond_collect.argtypes = [P, C.POINTER(DavidsonOpts), C.c_int, C.c_int, C.POINTER(C.c_int)]
    lib.bse_precond_set_samples.argtypes = [P, C.c_int, D, D, D]
    lib.bse_precond_get_samples.argtypes = [P, C.c_int, D, D, D, D, C.POINTER(C.c_int)]
    lib.bse_precond_grad.argtypes = [P, F, C.c_int, D, D]
    lib.bse_precond_train.argtypes = [C.POINTER(P), C.c_int, F, C.c_int, C.c_double, C.c_int, F, D]
    lib.bse_precond_load.argtypes = [P, F]
    lib.bse_solve_batch.argtypes = [C.POINTER(P), C.c_int, C.POINTER(DavidsonOpts), C.POINTER(C.c_double),
                                    C.POINTER(DavidsonStats), C.POINTER(C.c_int)]
    lib.bse_lanczos.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.c_int, D, D, D]
    lib.bse_localize.argtypes = [P, C.c_int, C.c_double, D, D]
    lib.bse_lanczos_spectrum.argtypes = [P, C.c_int, D, D, C.c_double, C.c_int, D, C.c_double, D, D]
    lib.bse_destroy.argtypes = [P]
    lib.bse_destroy.restype = None
    for name in EXPORTS:
        getattr(lib, name)
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Stats:
    iterations: int
    n_apply: int
    ms_total: float
    ms_apply: float
    res_max: float
    precond_fallbacks: int


class Context:
    """One system on the current CUDA device; ``sys`` is any object with the instance fields
    (L, n_grid, miller, psi, eps, v_loc, scissor, pdep, lam, overlap_thr, keep_pairs, spin).

    allocator: "torch" (default) hands the context's device memory out of PyTorch's caching
    allocator through the bse_create callbacks; None lets the library use cudaMallocAsync."""

    def __init__(self, sys, precision: int = PREC_FP64, stream=None, allocator="torch"):
        self.lib = load()
        self.allocator = None
        if allocator == "torch":
            import torch
            torch.cuda.empty_cache()     # cached blocks of earlier contexts count as free memory
            self.allocator = TorchAllocator(int(stream) if stream is not None else 0,
                                            torch.cuda.current_device())
        elif allocator is not None:
            raise ValueError("allocator must be 'torch' or None")
        self.precision = precision
        self._keep = []
        miller = np.ascontiguousarray(sys.miller, dtype=np.int32)
        psi = np.ascontiguousarray(sys.psi, dtype=np.float64)
        eps = np.ascontiguousarray(sys.eps, dtype=np.float64)
        vloc = np.ascontiguousarray(sys.v_loc, dtype=np.float64)
        pdep = np.ascontiguousarray(sys.pdep, dtype=np.float64)
        lam = np.ascontiguousarray(sys.lam, dtype=np.float64)
        self._keep += [miller, psi, eps, vloc, pdep, lam]
        n_qp = int(getattr(sys, "qp_n", 0) or 0)
        qp = {}
        if n_qp:
            qpsi = np.ascontiguousarray(sys.qp_psi, dtype=np.float64)
            qks = np.ascontiguousarray(sys.qp_eps_ks, dtype=np.float64)
            qe = np.ascontiguousarray(sys.qp_eps, dtype=np.float64)
            self._keep += [qpsi, qks, qe]
            qp = dict(qp_psi=_dptr(qpsi), qp_eps_ks=_dptr(qks), qp_eps=_dptr(qe))
        s = System(n_grid=int(sys.n_grid), L=float(sys.L), n_half=int(miller.shape[0]),
                   miller=miller.ctypes.data_as(C.POINTER(C.c_int32)), n_occ=int(psi.shape[0]),
                   psi=_dptr(psi), eps=_dptr(eps), v_loc=_dptr(vloc), scissor=float(sys.scissor),
                   n_pdep=int(pdep.shape[0]), pdep=_dptr(pdep), lam=_dptr(lam),
                   overlap_thr=float(sys.overlap_thr), keep_pairs=int(sys.keep_pairs),
                   spin=int(sys.spin), n_qp=n_qp, n_up=int(getattr(sys, "n_up", 0) or 0), **qp)
        self.n_occ, self.n_pw = psi.shape
        h = C.c_void_p()
        st = C.c_void_p(int(stream) if stream is not None else 0)
        if self.allocator is not None:
            af, ff = self.allocator.alloc_fn, self.allocator.free_fn
        else:
            af, ff = ALLOC_FN(), FREE_FN()
        rc = self.lib.bse_create(C.byref(s), precision, af, ff, None, st, C.byref(h))
        self.h = h
        if rc != BSE_OK:
            msg = self.lib.bse_last_error(h).decode() if h else "bse_create failed"
            if h:
                self.lib.bse_destroy(h)
                self.h = C.c_void_p()
            raise BseError(rc, msg)

    def _check(self, rc):
        if rc != BSE_OK:
            raise BseError(rc, self.lib.bse_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.lib.bse_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, mode: int):
        """1 enable, 0 disable, -1 clear the per-region CUDA-event profile."""
        self._check(self.lib.bse_profile(self.h, int(mode)))

    def profile_read(self):
        """({region: dict(calls, ms, bytes, flops)}, kernel launches issued so far)."""
        n = C.c_int()
        nl = C.c_int64()
        self._check(self.lib.bse_profile_read(self.h, None, 0, C.byref(n), C.byref(nl)))
        buf = (ProfEntry * max(1, n.value))()
        self._check(self.lib.bse_profile_read(self.h, buf, n.value, C.byref(n), C.byref(nl)))
        out = {}
        for e in buf[:n.value]:
            out[e.name.decode()] = dict(calls=int(e.calls), ms=float(e.ms), bytes=float(e.bytes),
                                        flops=float(e.flops))
        return out, int(nl.value)

    def build_tau(self):
        if self.allocator is not None:
            import torch
            torch.cuda.empty_cache()     # the tau layout is chosen from the free device memory
        n = C.c_int64()
        t = C.c_double()
        self._check(self.lib.bse_build_tau(self.h, C.byref(n), C.byref(t)))
        self.n_pairs = int(n.value)
        return self.n_pairs, float(t.value)

    def pairs(self):
        v = np.zeros(self.n_pairs, np.int32)
        w = np.zeros(self.n_pairs, np.int32)
        self._check(self.lib.bse_get_pairs(self.h, v.ctypes.data_as(C.POINTER(C.c_int32)),
                                           w.ctypes.data_as(C.POINTER(C.c_int32))))
        return np.stack([v, w], 1)

    def overlaps(self):
        o = np.zeros((self.n_occ, self.n_occ))
        self._check(self.lib.bse_get_overlaps(self.h, _dptr(o)))
        return o

    def apply(self, a_in, a_out):
        """a_in, a_out: contiguous CUDA tensors [n_vec, n_occ, n_pw] (float64 or float32)."""
        assert a_in.is_contiguous() and a_out.is_contiguous()
        assert tuple(a_in.shape[1:]) == (self.n_occ, self.n_pw) and a_in.shape == a_out.shape
        self._check(self.lib.bse_apply_liouville(self.h, int(a_in.shape[0]),
                                                 C.c_void_p(a_in.data_ptr()),
                                                 C.c_void_p(a_out.data_ptr())))
        return a_out

    # ---- Wannier localisation ----
    def localize(self, max_sweeps=100, tol=1e-10):
        """JADE localisation of the context's orbitals (before build_tau): (U, spread before,
        spread after); the context continues in the localised frame."""
        U = np.zeros((self.n_occ, self.n_occ))
        sp = np.zeros(2)
        self._check(self.lib.bse_localize(self.h, int(max_sweeps), float(tol), _dptr(U), _dptr(sp)))
        return U, float(sp[0]), float(sp[1])

    # ---- absorption spectrum ----
    def lanczos(self, n_steps, dirs=(0, 1, 2)):
        """Lanczos chains from the dipole blocks of the given directions: (alpha, beta, norm2)
        with alpha, beta [n_pol, n_steps] and norm2 [n_pol]."""
        d = np.ascontiguousarray(dirs, dtype=np.int32)
        npol = int(d.size)
        a = np.zeros((npol, n_steps))
        b = np.zeros((npol, n_steps))
        n2 = np.zeros(npol)
        self._check(self.lib.bse_lanczos(self.h, npol, d.ctypes.data_as(C.POINTER(C.c_int)), int(n_steps),
                                         _dptr(a), _dptr(b), _dptr(n2)))
        return a, b, n2

    def lanczos_spectrum(self, alpha, beta, norm2, omega, eta):
        """g(omega + i eta) of one chain, complex [n_omega] (computed on the GPU)."""
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        b = np.ascontiguousarray(beta, dtype=np.float64)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        gr = np.zeros(om.size)
        gi = np.zeros(om.size)
        self._check(self.lib.bse_lanczos_spectrum(self.h, int(a.size), _dptr(a), _dptr(b), float(norm2),
                                                  int(om.size), _dptr(om), float(eta), _dptr(gr), _dptr(gi)))
        return gr + 1j * gi

    # ---- learned preconditioner ----
    def precond_collect(self, n_eig, block, max_sub, max_it=200, res_tol=1e-6, ref_eig=32,
                        max_samples=256):
        opts = DavidsonOpts(n_eig=n_eig, block=block, max_sub=max_sub, max_it=max_it,
                            res_tol=res_tol, precond=0)
        n = C.c_int()
        self._check(self.lib.bse_precond_collect(self.h, C.byref(opts), ref_eig, max_samples, C.byref(n)))
        return int(n.value)

    def precond_get_samples(self, with_u=True):
        """(u, r, t, theta) of the context's samples (u is None for caller samples)."""
        n = C.c_int()
        self._check(self.lib.bse_precond_get_samples(self.h, 0, None, None, None, None, C.byref(n)))
        ns = n.value
        shape = (ns, self.n_occ, self.n_pw)
        u = np.zeros(shape) if with_u else None
        r, t, th = np.zeros(shape), np.zeros(shape), np.zeros(ns)
        self._check(self.lib.bse_precond_get_samples(self.h, ns, _dptr(u) if with_u else None, _dptr(r), _dptr(t),
                                                     _dptr(th), C.byref(n)))
        return u, r, t, th

    def precond_set_samples(self, r, t, theta):
        r = np.ascontiguousarray(r, dtype=np.float64)
        t = np.ascontiguousarray(t, dtype=np.float64)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        self._check(self.lib.bse_precond_set_samples(self.h, int(th.size), _dptr(r), _dptr(t), _dptr(th)))

    def precond_grad(self, params, act_bf16=False):
        p = np.ascontiguousarray(params, dtype=np.float32)
        g = np.zeros(NPARAM)
        loss = C.c_double()
        self._check(self.lib.bse_precond_grad(self.h, p.ctypes.data_as(C.POINTER(C.c_float)),
                                              int(act_bf16), C.byref(loss), _dptr(g)))
        return float(loss.value), g

    def precond_load(self, params):
        if params is None:
            self._check(self.lib.bse_precond_load(self.h, None))
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._keep_params = p
        self._check(self.lib.bse_precond_load(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def apply_static(self, a_in, a_out):
        """The operator with workspaces in the library's fixed device array (no allocation)."""
        assert a_in.is_contiguous() and a_out.is_contiguous()
        assert tuple(a_in.shape[1:]) == (self.n_occ, self.n_pw) and a_in.shape == a_out.shape
        self._check(self.lib.bse_apply_liouville_static(self.h, int(a_in.shape[0]),
                                                        C.c_void_p(a_in.data_ptr()),
                                                        C.c_void_p(a_out.data_ptr())))
        return a_out

    def davidson(self, n_eig, block, max_sub, max_it=200, res_tol=1e-5, precond=0, vec_out=None,
                 allow_not_converged=False):
        opts = DavidsonOpts(n_eig=n_eig, block=block, max_sub=max_sub, max_it=max_it,
                            res_tol=res_tol, precond=precond)
        om = np.zeros(n_eig)
        st = DavidsonStats()
        vp = C.c_void_p(vec_out.data_ptr()) if vec_out is not None else C.c_void_p()
        rc = self.lib.bse_davidson(self.h, C.byref(opts), _dptr(om), vp, C.byref(st))
        if not (rc == BSE_OK or (allow_not_converged and rc == BSE_ERR_NOT_CONVERGED)):
            self._check(rc)
        stats = Stats(st.iterations, st.n_apply, st.ms_total, st.ms_apply, st.res_max,
                      st.precond_fallbacks)
        return om, stats


def version() -> str:
    return load().bse_version().decode()


def precond_train(contexts, init, epochs=40, lr=3e-3, act_bf16=True):
    """Adam training on the GPU over the samples of several contexts; returns (params, losses)."""
    lib = load()
    hs = (C.c_void_p * len(contexts))(*[c.h.value for c in contexts])
    p0 = np.ascontiguousarray(init, dtype=np.float32)
    out = np.zeros(NPARAM, dtype=np.float32)
    hist = np.zeros(epochs)
    rc = lib.bse_precond_train(hs, len(contexts), p0.ctypes.data_as(C.POINTER(C.c_float)), epochs,
                               float(lr), int(act_bf16), out.ctypes.data_as(C.POINTER(C.c_float)),
                               _dptr(hist))
    if rc != BSE_OK:
        raise BseError(rc, lib.bse_last_error(contexts[0].h).decode())
    return out, hist


def solve_batch(contexts, n_eig, block, max_sub, max_it=200, res_tol=1e-5, precond=0):
    """tau build (if needed) + Davidson for many contexts concurrently; returns (omega [n, n_eig],
    stats list, status list)."""
    lib = load()
    n = len(contexts)
    hs = (C.c_void_p * n)(*[c.h.value for c in contexts])
    opts = DavidsonOpts(n_eig=n_eig, block=block, max_sub=max_sub, max_it=max_it, res_tol=res_tol,
                        precond=precond)
    om = np.zeros((n, n_eig))
    st = (DavidsonStats * n)()
    rc = (C.c_int * n)()
    lib.bse_solve_batch(hs, n, C.byref(opts), _dptr(om), st, rc)
    stats = [Stats(s.iterations, s.n_apply, s.ms_total, s.ms_apply, s.res_max, s.precond_fallbacks)
             for s in st]
    return om, stats, list(rc)


def precond_init(seed=0):
    """He-normal hidden layers, zero last layer (the untrained network is the diagonal step)."""
    rng = np.random.default_rng(seed)
    H, F = 64, 5
    p = np.zeros(NPARAM, dtype=np.float32)
    p[:H * F] = rng.standard_normal(H * F) * np.sqrt(2.0 / F)
    o = H * F + H
    p[o:o + H * H] = rng.standard_normal(H * H) * np.sqrt(2.0 / H)
    p[-5:] = 1.0
    return p


def launch_count() -> int:
    """Kernel launches issued by the library in this process."""
    nl = C.c_int64()
    load().bse_profile_read(None, None, 0, None, C.byref(nl))
    return int(nl.value)

"""Lanczos absorption spectrum on the GPU (bse_lanczos, bse_lanczos_spectrum) against the
oracle (oracle/lanczos.py) and the dense electron-hole eigenpairs.

Tolerances: the first 30 chain coefficients of the FP64 path agree with the oracle chain to
1e-9 relative (both chains run the same recursion; rounding grows slowly along a chain).
Spectral functions of 600-step chains agree with the exact eigenpair sum to 1e-7 (FP64) and
5e-4 (mixed; FP32 vectors, FP64 coefficients) of max |g| at a broadening of 0.05 Ha. The
continued fraction evaluated on the GPU equals the oracle's evaluation of the same
coefficients to 1e-12.
"""
import numpy as np
import pytest

from synth import make_tiny, make_localized
from oracle import dense_eh, lanczos, liouville

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


@pytest.fixture(scope="module")
def tiny():
    inst = make_tiny(0)
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    w, X = np.linalg.eigh(H)
    return inst, H, parts, w, X


def _ctx(inst, prec):
    from paper_2409_15116_gb300 import Context
    c = Context(inst, prec)
    c.build_tau()
    return c


def test_fp64_chain_matches_oracle_chain(tiny):
    inst, H, parts, w, X = tiny
    Lop = liouville.Liouville(inst)
    c = _ctx(inst, 0)
    a, b, n2 = c.lanczos(30, dirs=(0, 1, 2))
    for p in range(3):
        ra, rb, rn2 = lanczos.lanczos(Lop.apply, lanczos.dipole_rhs(inst, p), 30, Lop.project)
        assert abs(n2[p] - rn2) <= 1e-12 * rn2
        assert np.abs(a[p] - ra).max() <= 1e-9 * np.abs(ra).max(), p
        assert np.abs(b[p] - rb).max() <= 1e-9 * np.abs(rb).max(), p
    c.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-7), (1, 5e-4)])
def test_spectrum_matches_dense_eigenpairs(tiny, prec, tol):
    inst, H, parts, w, X = tiny
    c = _ctx(inst, prec)
    a, b, n2 = c.lanczos(600, dirs=(2, 0))
    om = np.linspace(w[0] - 0.5, w[0] + 3.0, 300)
    for p, direction in enumerate((2, 0)):
        de = dense_eh.packed_to_eh(lanczos.dipole_rhs(inst, direction)[None], parts["Xc"])[0]
        ref = lanczos.spectrum_from_eigenpairs(w, X, de, om, 0.05)
        g = c.lanczos_spectrum(a[p], b[p], n2[p], om, 0.05)
        assert np.abs(g - ref).max() <= tol * np.abs(ref).max(), (direction, np.abs(g - ref).max())
        # the GPU continued fraction equals the oracle's on the same coefficients
        g2 = lanczos.continued_fraction(a[p], b[p], n2[p], om, 0.05)
        assert np.abs(g - g2).max() <= 1e-12 * np.abs(g2).max()
    c.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-5)])
def test_localized_chain_start_matches_oracle(prec, tol):
    inst = make_localized(6, 20.0 * 32 / 72, 32, 13, 2.5, 26, n_eig=4, block=4)
    Lop = liouville.Liouville(inst)
    c = _ctx(inst, prec)
    a, b, n2 = c.lanczos(8, dirs=(1,))
    ra, rb, rn2 = lanczos.lanczos(Lop.apply, lanczos.dipole_rhs(inst, 1), 8, Lop.project)
    assert abs(n2[0] - rn2) <= 1e-6 * rn2
    assert np.abs(a[0] - ra).max() <= tol * np.abs(ra).max()
    assert np.abs(b[0] - rb).max() <= tol * np.abs(rb).max()
    c.close()

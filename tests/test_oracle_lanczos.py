"""Pins of the Lanczos absorption-spectrum oracle (oracle/lanczos.py) against closed forms and
the dense electron-hole Hamiltonian (CPU only)."""
import math

import numpy as np
import pytest

from synth import make_tiny
from oracle import dense_eh, lanczos, liouville
from oracle.basis import packed_to_grid_field
from free_electron import free_instance, row_of


@pytest.fixture(scope="module")
def tiny():
    inst = make_tiny(0)
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    return inst, H, parts


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_dipole_rhs_of_a_cosine_orbital_is_the_sine(direction):
    """-d/dr_i of sqrt(2) cos(G.r) is sqrt(2) G_i sin(G.r); the sine is orthogonal to the one
    occupied cosine, so P_c leaves it unchanged. Checked on the real-space grid."""
    n = (1, 2, -1)
    inst = free_instance([0, 0])
    k = row_of(inst.miller, n)
    inst = free_instance([k])
    d = lanczos.dipole_rhs(inst, direction)
    u = packed_to_grid_field(d, inst.miller, inst.n_grid)[0]          # [z, y, x]
    N, L = inst.n_grid, inst.L
    m = inst.miller[k].astype(float)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    phase = 2 * math.pi * (m[0] * x + m[1] * y + m[2] * z) / N
    want = math.sqrt(2.0) * (2 * math.pi / L) * m[direction] * np.sin(phase)
    assert np.abs(u - want).max() < 1e-12


def _eh_apply(H, Xc, n_occ):
    def apply(A):
        y = dense_eh.packed_to_eh(A, Xc)
        return dense_eh.eh_to_packed(y @ H.T, Xc, n_occ)
    return apply


def test_lanczos_chain_reproduces_the_moments(tiny):
    """An m-step chain reproduces <d|L^k|d> = |d|^2 (T^k)_11 for k <= 2m - 1 (Gauss
    quadrature exactness); the moments come from the dense e-h matrix."""
    inst, H, parts = tiny
    Lop = liouville.Liouville(inst)
    d = lanczos.dipole_rhs(inst, 0)
    m = 10
    a, b, n2 = lanczos.lanczos(Lop.apply, d, m, Lop.project)
    T = np.diag(a) + np.diag(b[1:], 1) + np.diag(b[1:], -1)
    de = dense_eh.packed_to_eh(d[None], parts["Xc"])[0]
    assert abs(de @ de - n2) < 1e-12 * n2
    v, Tk = de.copy(), np.eye(m)
    for k in range(2 * m):
        mom = de @ v
        assert abs(n2 * Tk[0, 0] - mom) <= 1e-9 * abs(mom) + 1e-12, (k, n2 * Tk[0, 0], mom)
        v, Tk = H @ v, Tk @ T


def test_continued_fraction_equals_eigenpair_sum(tiny):
    """With a chain long enough to resolve the broadened line shape, the continued fraction
    equals sum_n |<x_n|d>|^2 / (omega + i eta - w_n) from the dense eigenpairs."""
    inst, H, parts = tiny
    w, X = np.linalg.eigh(H)
    d = lanczos.dipole_rhs(inst, 2)
    de = dense_eh.packed_to_eh(d[None], parts["Xc"])[0]
    a, b, n2 = lanczos.lanczos(_eh_apply(H, parts["Xc"], inst.n_occ), d, 600)
    om = np.linspace(w[0] - 0.5, w[0] + 3.0, 400)
    g = lanczos.continued_fraction(a, b, n2, om, 0.05)
    ref = lanczos.spectrum_from_eigenpairs(w, X, de, om, 0.05)
    assert np.abs(g - ref).max() <= 1e-8 * np.abs(ref).max()
    # the line shape integrates to |d|^2 (sum of the weights) over the whole real axis
    assert abs((X.T @ de) @ (X.T @ de) - n2) < 1e-10 * n2


def test_matrix_free_chain_with_projection_matches_the_eigenpair_sum(tiny):
    """The matrix-free operator with the conduction-space projection of every Lanczos vector
    gives the exact spectral function too (without the projection, rounding leakage into the
    occupied space grows along the chain)."""
    inst, H, parts = tiny
    w, X = np.linalg.eigh(H)
    Lop = liouville.Liouville(inst)
    d = lanczos.dipole_rhs(inst, 2)
    de = dense_eh.packed_to_eh(d[None], parts["Xc"])[0]
    a, b, n2 = lanczos.lanczos(Lop.apply, d, 300, Lop.project)
    om = np.linspace(w[0] - 0.5, w[0] + 3.0, 200)
    g = lanczos.continued_fraction(a, b, n2, om, 0.05)
    ref = lanczos.spectrum_from_eigenpairs(w, X, de, om, 0.05)
    assert np.abs(g - ref).max() <= 1e-6 * np.abs(ref).max()

"""Pins of the JADE Wannier-localisation oracle (oracle/jade.py) and of the BSE in a rotated
(localised) frame."""
import copy

import numpy as np

from synth import make_tiny, make_localized
from oracle import jade, dense_eh, pairs


def test_rotation_angle_is_the_brute_force_optimum():
    """The closed-form Givens angle maximises sum_n (A'_pp - A'_qq)^2 over a fine scan."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((6, 2, 2))
    A = A + A.transpose(0, 2, 1)
    th = jade.rotation_angle(A, 0, 1)
    grid = np.linspace(-np.pi / 2, np.pi / 2, 200001)
    c, s = np.cos(grid), np.sin(grid)
    d = ((c * c - s * s)[None] * (A[:, 0, 0] - A[:, 1, 1])[:, None] + (2 * c * s)[None] * (2 * A[:, 0, 1])[:, None])
    best = grid[np.argmax((d ** 2).sum(0))]
    # the optimum is defined modulo pi/2 (swapping the pair); compare the rotated diagonals
    def diag_diff(t):
        B = A.copy(); U = np.eye(2); jade.rotate(B, U, 0, 1, t)
        return ((B[:, 0, 0] - B[:, 1, 1]) ** 2).sum()
    assert abs(diag_diff(th) - diag_diff(best)) < 1e-9 * diag_diff(best)
    B = A.copy(); U = np.eye(2); jade.rotate(B, U, 0, 1, th)
    assert np.abs(np.einsum("ji,kjl,lm->kim", U, A, U) - B).max() < 1e-13


def test_jade_recovers_an_exact_joint_eigenbasis():
    """Matrices with a common eigenbasis Q: JADE diagonalises all of them (off-diagonal norm at
    rounding level) and the objective never decreases between sweeps."""
    rng = np.random.default_rng(2)
    n = 12
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = np.stack([Q @ np.diag(rng.standard_normal(n)) @ Q.T for _ in range(6)])
    U, At, hist = jade.jade(A, tol=1e-13)
    off = At - np.stack([np.diag(np.diag(a)) for a in At])
    assert np.abs(off).max() < 1e-10
    assert all(b >= a - 1e-12 for a, b in zip(hist, hist[1:]))
    assert np.abs(U.T @ U - np.eye(n)).max() < 1e-12


def test_jade_relocalises_rotated_localised_orbitals():
    """Localised orbitals mixed by a random rotation are delocalised; JADE brings the spread
    back to at most the original set's, and the orbital overlaps (Eq. overlap) back down."""
    inst = make_localized(6, 20.0 * 32 / 72, 32, 16, 2.5, 32)
    A0, B0 = jade.jade_matrices(inst)
    s_loc = jade.spread(A0, B0, np.eye(inst.n_occ))
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((inst.n_occ, inst.n_occ)))
    mixed = copy.copy(inst)
    mixed.psi = Q.T @ inst.psi
    A1, B1 = jade.jade_matrices(mixed)
    s_mix = jade.spread(A1, B1, np.eye(inst.n_occ))
    U, _, _ = jade.jade(A1)
    s_jade = jade.spread(A1, B1, U)
    assert s_mix > s_loc and s_jade <= s_loc + 1e-9, (s_loc, s_mix, s_jade)
    loc = copy.copy(mixed)
    loc.psi = U.T @ mixed.psi

    def mean_off(x):
        O = pairs.overlaps(x)
        return (O.sum() - np.trace(O)) / (O.size - O.shape[0])
    assert mean_off(loc) < 0.8 * mean_off(mixed) and mean_off(loc) <= 1.05 * mean_off(inst)


def test_bse_spectrum_is_invariant_under_the_localising_rotation():
    """With every pair kept, the e-h matrix in the JADE frame (orbitals U^T psi, occupied
    energies U^T diag(eps) U) has the spectrum of the canonical one."""
    inst = make_tiny(0)
    U, psi_l, E = jade.localize(inst)
    loc = copy.copy(inst)
    loc.psi, loc.eps_mat, loc.eps = psi_l, E, np.diag(E).copy()
    m, _ = pairs.pair_mask(loc)
    assert m.all()
    w0 = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(inst))
    w1 = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(loc))
    assert np.abs(w0 - w1).max() < 1e-10
    assert np.abs(E - np.diag(np.diag(E))).max() > 1e-3      # the frame is really rotated

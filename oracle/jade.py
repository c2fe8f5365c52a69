"""Wannier localisation of the occupied orbitals by joint approximate diagonalisation (JADE),
Section 2 (Eqs. wannier, spread and the six operators M^(n)). TEST INFRASTRUCTURE.

A^(n)_vw = <psi_v|M^(n)|psi_w>, B^(n)_vw = <psi_v|(M^(n))^2|psi_w> with M = cos(2 pi x/L),
sin(2 pi x/L), cos(2 pi y/L), ... The orthogonal U minimises the spread
    sigma^2(U) = sum_n [ Tr(U^T B^(n) U) - sum_v ((U^T A^(n) U)_vv)^2 ],
i.e. maximises sum_n sum_v ((U^T A U)_vv)^2, by Jacobi sweeps of 2 x 2 Givens rotations: for a
pair (p, q) the rotation angle theta maximises sum_n (A'_pp - A'_qq)^2 =
sum_n (h_n . (cos 2 theta, sin 2 theta))^2 with h_n = (A_pp - A_qq, 2 A_pq), so
(cos 2 theta, sin 2 theta) is the principal eigenvector of G = sum_n h_n h_n^T:
theta = 1/4 atan2(2 G_12, G_11 - G_22). U starts from the eigenvectors of A^(1) (as the
paper's code does). Reading of the index convention: the localised orbitals are
psi~_v = sum_w U_wv psi_w (columns of U), which makes (U^T A U)_vv = <psi~_v|M|psi~_v> as in
Eq. spread (Eq. wannier writes the same map with U's indices swapped).
"""
from __future__ import annotations

import numpy as np

from .basis import packed_to_grid_field


def jade_matrices(inst):
    """A [6, n, n] and the diagonals of B [6, n] on the grid (exact quadrature of
    band-limited products)."""
    N = inst.n_grid
    u = packed_to_grid_field(inst.psi, inst.miller, N).reshape(inst.n_occ, -1)   # Omega^1/2 psi
    i = np.arange(N)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    ops = []
    for c in (x, y, z):
        ph = (2 * np.pi / N) * c.reshape(-1)
        ops += [np.cos(ph), np.sin(ph)]
    A = np.stack([(u * m) @ u.T / N ** 3 for m in ops])
    Bd = np.stack([((u * u) * (m * m)).sum(1) / N ** 3 for m in ops])
    return A, Bd


def rotation_angle(A, p, q) -> float:
    """Givens angle of the pair (p, q) maximising sum_n (A'_pp - A'_qq)^2."""
    h0 = A[:, p, p] - A[:, q, q]
    h1 = A[:, p, q] + A[:, q, p]
    g11, g22, g12 = (h0 * h0).sum(), (h1 * h1).sum(), (h0 * h1).sum()
    return 0.25 * np.arctan2(2.0 * g12, g11 - g22)


def rotate(A, U, p, q, theta):
    """A <- R^T A R, U <- U R for the Givens rotation R in the (p, q) plane."""
    c, s = np.cos(theta), np.sin(theta)
    Ap, Aq = A[:, :, p].copy(), A[:, :, q].copy()
    A[:, :, p], A[:, :, q] = c * Ap + s * Aq, -s * Ap + c * Aq
    Ap, Aq = A[:, p, :].copy(), A[:, q, :].copy()
    A[:, p, :], A[:, q, :] = c * Ap + s * Aq, -s * Ap + c * Aq
    Up, Uq = U[:, p].copy(), U[:, q].copy()
    U[:, p], U[:, q] = c * Up + s * Uq, -s * Up + c * Uq


def jade(A, tol: float = 1e-10, max_sweeps: int = 100, init_first: bool = True):
    """Orthogonal U jointly diagonalising the symmetric matrices A [K, n, n] (cyclic sweeps).

    Returns (U, rotated A, objective sum_n sum_v diag^2 after each sweep)."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[1]
    U = np.eye(n)
    if init_first:
        _, U = np.linalg.eigh(A[0])
        A = np.einsum("ji,kjl,lm->kim", U, A, U)
    hist = []
    for _ in range(max_sweeps):
        smax = 0.0
        for p in range(n - 1):
            for q in range(p + 1, n):
                th = rotation_angle(A, p, q)
                if abs(np.sin(th)) > tol:
                    rotate(A, U, p, q, th)
                smax = max(smax, abs(np.sin(th)))
        hist.append(float((np.diagonal(A, axis1=1, axis2=2) ** 2).sum()))
        if smax <= tol:
            break
    return U, A, hist


def spread(A, Bd, U) -> float:
    """sigma^2(U) of Eq. spread (Tr(U^T B U) = sum of B's diagonal)."""
    At = np.einsum("ji,kjl,li->ki", U, A, U)      # diagonals of U^T A U
    return float(Bd.sum() - (At ** 2).sum())


def localize(inst, tol: float = 1e-10):
    """(U, localised packed orbitals psi~ = U^T psi, occupied energy matrix U^T diag(eps) U)."""
    A, _ = jade_matrices(inst)
    U, _, _ = jade(A, tol)
    return U, U.T @ inst.psi, U.T @ np.diag(inst.eps) @ U

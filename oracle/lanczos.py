"""Absorption spectrum by a Lanczos chain of the Liouville operator (Section 4: the spectrum
of bulk Si is computed with a Lanczos recursion of N_Lanczos applications of the operator per
polarisation direction, instead of an iterative diagonalisation). TEST INFRASTRUCTURE.

Dipole right-hand side. For polarisation direction i the perturbation acts on every occupied
orbital through the commutator [H, r_i]; for the local Hamiltonian of the model,
[H, r_i] psi = -d/dr_i psi, so the trial block is

    d_v = P_c ( -d psi_v / d r_i ),   v = 1 .. N_occ,

i.e. in G space c'(G) = -i G_i c(G): packed p'[2k] = G_i p[2k+1], p'[2k+1] = -G_i p[2k].

Lanczos recursion (Hermitian operator L of Eq. evp in the Tamm-Dancoff form):
    q_1 = d/|d|,  beta_1 = 0,  q_0 = 0
    w = L q_k - beta_k q_{k-1},  alpha_k = <q_k|w>,  w -= alpha_k q_k,
    beta_{k+1} = |w|,  q_{k+1} = w / beta_{k+1}.
Spectral function of the chain: g(z) = <d|(z - L)^{-1}|d> = |d|^2 / (z - alpha_1 - beta_2^2 /
(z - alpha_2 - beta_3^2 / ...)), z = omega + i eta; the absorption line shape is -Im g / pi.

L acts on the conduction space; every new Lanczos vector is projected back onto it (P_c).
Without that, rounding leaves components in the occupied space, where L is zero, and the
three-term recurrence amplifies them exponentially (0 lies outside the spectrum), which
spoils the spectrum after a few dozen steps.
"""
from __future__ import annotations

import numpy as np


def dipole_rhs(inst, direction: int, project=None) -> np.ndarray:
    """d_v = P_c(-d psi_v / d r_direction) for all v, packed [n_occ, n_pw] (velocity form)."""
    g = 2 * np.pi / inst.L
    Gi = inst.miller[:, direction].astype(np.float64) * g        # [n_half]
    p = inst.psi
    d = np.zeros_like(p)
    d[:, 2::2] = Gi[None, 1:] * p[:, 3::2]
    d[:, 3::2] = -Gi[None, 1:] * p[:, 2::2]
    if project is not None:
        return project(d[None])[0]
    psi = inst.psi
    out = d - (d @ psi.T) @ psi
    out[:, 1] = 0.0
    return out


def lanczos(apply, d: np.ndarray, n_steps: int, project=None):
    """alpha [n_steps], beta [n_steps] (beta[0] = 0, beta[k] couples steps k-1 and k), |d|^2.

    ``apply`` maps a block [1, n_occ, n_pw] to L times it; ``d`` is [n_occ, n_pw];
    ``project`` (a block map, e.g. P_c) is applied to every new Lanczos vector.
    """
    norm2 = float((d * d).sum())
    q = d / np.sqrt(norm2)
    q_prev = np.zeros_like(q)
    alpha = np.zeros(n_steps)
    beta = np.zeros(n_steps)
    for k in range(n_steps):
        w = apply(q[None])[0] - beta[k] * q_prev
        alpha[k] = float((q * w).sum())
        w = w - alpha[k] * q
        if k + 1 == n_steps:
            break
        if project is not None:
            w = project(w[None])[0]
        beta[k + 1] = float(np.sqrt((w * w).sum()))
        if beta[k + 1] == 0.0:
            alpha, beta = alpha[:k + 1], beta[:k + 1]
            break
        q_prev, q = q, w / beta[k + 1]
    return alpha, beta, norm2


def continued_fraction(alpha, beta, norm2, omega, eta):
    """g(omega + i eta) = <d|(z - L)^{-1}|d> from the chain (evaluated from the bottom up)."""
    z = np.asarray(omega, dtype=np.float64) + 1j * eta
    f = np.zeros_like(z)
    for k in range(len(alpha) - 1, -1, -1):
        tail = beta[k + 1] ** 2 * f if k + 1 < len(alpha) else 0.0
        f = 1.0 / (z - alpha[k] - tail)
    return norm2 * f


def spectrum_from_eigenpairs(w, X, d_eh, omega, eta):
    """The same g(z) as the explicit sum over eigenpairs: sum_n |<x_n|d>|^2 / (z - w_n)."""
    z = np.asarray(omega, dtype=np.float64) + 1j * eta
    c2 = (X.T @ d_eh) ** 2
    return (c2[None, :] / (z[:, None] - w[None, :])).sum(1)

"""Quasi-particle terms of the diagonal operator D (Eq. d with the QP Hamiltonian of Eq. ham).

H_QP = H_KS + sum_{n <= N_QP} |psi_n> (eps^QP_n - eps_n - Delta) <psi_n| + Delta,
Delta = mean of (eps^QP_n - eps_n) over n = N_mid .. N_QP, N_mid = (N_occ + N_QP) / 2
(1-based state indices; the paper leaves the rounding of N_mid open: integer division).

On the conduction space D a_v = P_c (H_QP - eps^QP_v) a_v; the occupied terms of the sum are
removed by P_c, so D a_v = P_c H_KS a_v + sum_{c = N_occ+1}^{N_QP} psi_c delta_c <psi_c|a_v>
+ (Delta - eps^QP_v) a_v with delta_c = eps^QP_c - eps_c - Delta. Without explicit QP data
(qp_n = 0) the scissor form applies: Delta = the scissor, eps^QP_v = eps_v, no delta_c.
"""
from __future__ import annotations

import numpy as np


def qp_terms(inst):
    """(eps^QP_v [n_occ], Delta, delta_c [N_QP - n_occ], conduction states [N_QP - n_occ, n_pw])."""
    if not getattr(inst, "qp_n", 0):
        return np.asarray(inst.eps, dtype=np.float64), float(inst.scissor), np.zeros(0), \
            np.zeros((0, inst.psi.shape[1]))
    n_occ, nqp = inst.n_occ, int(inst.qp_n)
    d = np.asarray(inst.qp_eps, dtype=np.float64) - np.asarray(inst.qp_eps_ks, dtype=np.float64)
    n_mid = (n_occ + nqp) // 2
    delta_avg = float(d[n_mid - 1:nqp].sum() / (nqp - n_mid + 1))
    return np.asarray(inst.qp_eps[:n_occ], dtype=np.float64), delta_avg, d[n_occ:] - delta_avg, \
        np.asarray(inst.qp_psi, dtype=np.float64)


def occupied_energy_matrix(inst) -> np.ndarray:
    """The occupied energies entering D as a matrix: diag(eps^QP_v) for canonical orbitals,
    or the given U^T diag(eps) U of a rotated (Wannier) frame, where D a_v = P_c H a_v -
    sum_w E_vw a_w (the rotation of Eq. wannier applied to Eq. d)."""
    E = getattr(inst, "eps_mat", None)
    if E is not None:
        return np.asarray(E, dtype=np.float64)
    return np.diag(qp_terms(inst)[0])

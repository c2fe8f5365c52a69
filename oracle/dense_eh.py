"""Explicit electron-hole (e-h) Hamiltonian over the complete conduction manifold -- plain definition.

The DMPT eigenproblem of Eq. (evp) works with auxiliary orbitals a_v in the
conduction space. Writing a_v = sum_c X_vc psi_c over ALL conduction states that the
plane-wave sphere S supports turns Eqs. (d), (k1e), (k1d) into the matrix

    H_(vc),(wc') = delta_vw <c|P_c (H_KS + Delta - eps_v) P_c|c'>        (Eq. d, Eq. ham)
                 + s * Omega sum_{G != 0} v(G) rho_vc(G)^* rho_wc'(G)     (Eq. k1e, s = 2 singlet)
                 - m_vw * int psi_c(r) psi_c'(r) tau_vw(r) dr              (Eq. k1d)

with rho_ab(G) = N^-3 sum_r psi_a psi_b e^{-iG.r}, the screened integral
tau_vw = W[psi_v psi_w] (Eq. tau), W = v^{1/2}(1 + chi_bar) v^{1/2} with the
low-rank chi_bar of Eq. (pdep) (Xi = 0, v(0) = 0) and m_vw the overlap mask
(Eq. overlap). Because the conduction manifold is complete within S, the lowest
eigenvalues of this matrix are the DMPT/Davidson excitation energies (the
completeness argument of Section 5.3, Fig. 8). All products are alias-free on the
grid (components <= 4 r_max < N), so every grid sum below is an exact quadrature.

Only for tiny cells: the real-space fields come from an explicit inverse DFT matrix.
"""
from __future__ import annotations

import numpy as np

from .basis import (full_miller, packing_matrix, drop_pad, add_pad, coulomb_grid,
                    sphere_on_grid, packed_to_full)
from .pairs import pair_mask
from .qp import qp_terms, occupied_energy_matrix


def ks_hamiltonian_packed(inst) -> np.ndarray:
    """KS Hamiltonian in the unpadded packed basis of S (the H_KS of Eq. ham).

    H_GG' = 1/2 |G|^2 delta_GG' + V(G - G'), V(q) = N^-3 sum_r V_loc(r) e^{-iq.r}
    (the DFT of the given grid samples; |G - G'| <= 2 r_max so there is no wrap).
    """
    N, L = inst.n_grid, inst.L
    Vq = np.fft.fftn(inst.v_loc.reshape(N, N, N)) / N ** 3
    full = full_miller(inst.miller)
    dq = full[:, None, :] - full[None, :, :]
    Hc = Vq[dq[..., 2] % N, dq[..., 1] % N, dq[..., 0] % N]
    g = 2 * np.pi / L
    Hc = Hc + np.diag(0.5 * g * g * (full.astype(np.float64) ** 2).sum(1))
    U = packing_matrix(inst.n_half)
    Hp = U.conj().T @ Hc @ U
    return 0.5 * (Hp.real + Hp.real.T), float(np.abs(Hp.imag).max())


def conduction_states(inst, H=None):
    """Eigenpairs of P_c H_KS P_c on the orthogonal complement of span{psi_v} (P_c of Section 2).

    Returns (eps_c [N_c], X_c [N_c, n_pw] padded packed, orthonormal).
    """
    if H is None:
        H, _ = ks_hamiltonian_packed(inst)
    psi = drop_pad(inst.psi)
    Q, _ = np.linalg.qr(psi.T, mode="complete")
    Qc = Q[:, inst.n_occ:]
    Hc = Qc.T @ H @ Qc
    e, C = np.linalg.eigh(0.5 * (Hc + Hc.T))
    return e, add_pad((Qc @ C).T.copy())


def real_space_explicit(inst, P: np.ndarray) -> np.ndarray:
    """psi(r) = Omega^{-1/2} sum_{G in S} c(G) e^{iG.r} by an explicit DFT matrix; [m, N^3], x fastest."""
    N = inst.n_grid
    full = full_miller(inst.miller).astype(np.float64)
    idx = np.arange(N ** 3)
    r = np.stack([idx % N, (idx // N) % N, idx // (N * N)], axis=1).astype(np.float64)
    E = np.exp(1j * (2 * np.pi / N) * (r @ full.T))
    c = packed_to_full(P)
    return (c @ E.T).real / np.sqrt(inst.omega)


def _hat(f_r: np.ndarray, N: int) -> np.ndarray:
    """N^-3 sum_r f(r) e^{-iG.r} on the grid (numpy FFT as a library step), flattened [.., N^3]."""
    F = np.fft.fftn(f_r.reshape(f_r.shape[:-1] + (N, N, N)), axes=(-3, -2, -1)) / N ** 3
    return F.reshape(f_r.shape[:-1] + (N ** 3,))


def screened_integral_hat(inst, rho_hat: np.ndarray) -> np.ndarray:
    """tau(G) = W rho(G) on the grid (Eqs. tau, tau_from_tau_u, pdep with Xi = 0).

    tau = v rho + v^{1/2} chi_bar v^{1/2} rho, chi_bar(G,G') = sum_a phi_a(G) f_a phi_a(G')^*,
    f_a = lambda_a/(1-lambda_a), phi_a the PDEP vectors on S (full complex form).
    """
    N, L = inst.n_grid, inst.L
    vc = coulomb_grid(N, L).reshape(-1)
    sq = np.sqrt(vc)
    iz, iy, ix = sphere_on_grid(full_miller(inst.miller), N)
    sidx = (iz * N + iy) * N + ix
    phi = packed_to_full(inst.pdep)                      # [n_pdep, n_full]
    f = inst.lam / (1.0 - inst.lam)
    x = sq[sidx] * rho_hat[..., sidx]                    # v^{1/2} rho on S
    proj = x @ phi.conj().T                              # <phi_a | x>
    chi_x = (proj * f) @ phi                             # chi_bar x on S
    tau = vc * rho_hat
    tau[..., sidx] += sq[sidx] * chi_x
    return tau


def eh_hamiltonian(inst, mask=None, with_parts: bool = False):
    """Dense TDA e-h Hamiltonian of Eq. (evp) over the complete conduction manifold.

    Index (v, c) -> v * N_c + c. Returns H (and the parts / bases when asked).
    """
    N, omega = inst.n_grid, inst.omega
    dV = omega / N ** 3
    eps_c, Xc = conduction_states(inst)
    Nc, No = eps_c.size, inst.n_occ
    if mask is None:
        mask, _ = pair_mask(inst)
    psi_r = real_space_explicit(inst, inst.psi)          # [No, N^3]
    c_r = real_space_explicit(inst, Xc)                  # [Nc, N^3]
    vc = coulomb_grid(N, inst.L).reshape(-1)

    # D: P_c H_KS P_c is diagonal in the conduction eigenbasis; the QP Hamiltonian of Eq. ham
    # adds Delta - eps^QP_v and, with explicit QP data, sum_c psi_c delta_c <psi_c| (Eq. d)
    eps_qp, delta_avg, delta_c, psi_qp = qp_terms(inst)
    E = occupied_energy_matrix(inst)
    Ddiag = (eps_c[None, :] + delta_avg - np.diag(E)[:, None]).reshape(-1)
    Cqp = (Xc @ psi_qp.T) @ np.diag(delta_c) @ (psi_qp @ Xc.T)     # [Nc, Nc]

    # K1e core: Omega sum_G v(G) rho_vc^* rho_wc' (Eq. k1e, without the spin factor)
    rho_hat = _hat((psi_r[:, None, :] * c_r[None, :, :]).reshape(No * Nc, -1), N)
    K1e = omega * ((rho_hat.conj() * vc) @ rho_hat.T).real

    # K1d: m_vw int psi_c psi_c' tau_vw (Eq. k1d, Eq. tau)
    K1d = np.zeros((No * Nc, No * Nc))
    for v in range(No):
        for w in range(No):
            if not mask[v, w]:
                continue
            th = screened_integral_hat(inst, _hat(psi_r[v] * psi_r[w], N))
            tau_r = (np.fft.ifftn(th.reshape(N, N, N)) * N ** 3).real.reshape(-1)
            K1d[v * Nc:(v + 1) * Nc, w * Nc:(w + 1) * Nc] = dV * (c_r * tau_r) @ c_r.T

    s = 2.0 if inst.spin == 0 else 0.0
    H = np.diag(Ddiag) + np.kron(np.eye(No), Cqp) - np.kron(E - np.diag(np.diag(E)), np.eye(Nc)) \
        + s * K1e - K1d
    if not with_parts:
        return H
    return H, dict(D=Ddiag, Dqp=Cqp, K1e=K1e, K1d=K1d, eps_c=eps_c, Xc=Xc, psi_r=psi_r,
                   c_r=c_r, mask=mask, spin_factor=s)


def eh_to_packed(y: np.ndarray, Xc: np.ndarray, n_occ: int) -> np.ndarray:
    """e-h coefficients [..., n_occ*N_c] -> packed blocks [..., n_occ, n_pw] (a_v = sum_c y_vc psi_c)."""
    Nc = Xc.shape[0]
    return y.reshape(y.shape[:-1] + (n_occ, Nc)) @ Xc


def packed_to_eh(A: np.ndarray, Xc: np.ndarray) -> np.ndarray:
    return (A @ Xc.T).reshape(A.shape[:-2] + (-1,))


def lowest_excitations(inst, n: int) -> np.ndarray:
    """Lowest n eigenvalues of the dense e-h Hamiltonian (reference VEEs)."""
    H = eh_hamiltonian(inst)
    return np.linalg.eigvalsh(H)[:n]

"""Spin-polarised (spin-conserving) TDA Bethe-Salpeter operator, explicit e-h matrix.
TEST INFRASTRUCTURE. (The paper's code supports spin-polarised systems with spin-conserving
excitations, Section 2; its Eqs. evp-k1d are written for one channel.)

Each occupied spin-orbital v of channel s carries its own auxiliary orbital a_v in the
conduction space of its channel (P_c^s = 1 - sum_{w in s} |psi_w><psi_w|). With the e-h
basis (v, c) for c in the complete conduction manifold of v's channel:

  H_(vc),(wc') = delta_vw <c|P_c^s (H_KS + Delta - eps_v) P_c^s|c'>               (Eq. d)
              + Omega sum_{G != 0} v(G) rho_vc(G)^* rho_wc'(G)   for all v, w       (Eq. k1e)
              - delta_{s(v) s(w)} m_vw int psi_c psi_c' tau_vw                       (Eq. k1d)

The exchange term couples both channels (the Hartree potential of the total density change)
and carries no factor 2; the screened direct term stays inside a channel. For two identical
channels the spectrum is the union of the closed-shell singlet (factor 2) and triplet (factor
0) spectra, which the pins check.
"""
from __future__ import annotations

import copy

import numpy as np

from .basis import coulomb_grid
from .dense_eh import conduction_states, real_space_explicit, _hat, screened_integral_hat
from .pairs import pair_mask, channels


def _channel(inst, sel):
    sub = copy.copy(inst)
    sub.psi = inst.psi[sel]
    sub.eps = inst.eps[sel]
    sub.n_up = 0
    return sub


def eh_hamiltonian_spin(inst, mask=None):
    """Dense e-h matrix of a spin-polarised system and its basis: (H, blocks), where blocks is a
    list of (orbital index v, conduction basis Xc of v's channel [Nc_s, n_pw]) in basis order."""
    N, omega = inst.n_grid, inst.omega
    dV = omega / N ** 3
    ch = channels(inst)
    if mask is None:
        mask, _ = pair_mask(inst)
    conds = {}
    for s in (0, 1):
        sel = np.nonzero(ch == s)[0]
        if sel.size:
            conds[s] = conduction_states(_channel(inst, sel))
    psi_r = real_space_explicit(inst, inst.psi)
    c_r = {s: real_space_explicit(inst, conds[s][1]) for s in conds}
    blocks, offs, Dd = [], [], []
    off = 0
    for v in range(inst.n_occ):
        eps_c, Xc = conds[ch[v]]
        blocks.append((v, Xc))
        offs.append(off)
        off += eps_c.size
        Dd.append(eps_c + inst.scissor - inst.eps[v])
    dim = off
    vc = coulomb_grid(N, inst.L).reshape(-1)
    rho_hat = np.concatenate([_hat(psi_r[v][None, :] * c_r[ch[v]], N) for v in range(inst.n_occ)])
    K1e = omega * ((rho_hat.conj() * vc) @ rho_hat.T).real
    K1d = np.zeros((dim, dim))
    for v in range(inst.n_occ):
        for w in range(inst.n_occ):
            if ch[v] != ch[w] or not mask[v, w]:
                continue
            th = screened_integral_hat(inst, _hat(psi_r[v] * psi_r[w], N))
            tau_r = (np.fft.ifftn(th.reshape(N, N, N)) * N ** 3).real.reshape(-1)
            cr = c_r[ch[v]]
            nv, nw = cr.shape[0], cr.shape[0]
            K1d[offs[v]:offs[v] + nv, offs[w]:offs[w] + nw] = dV * (cr * tau_r) @ cr.T
    H = np.diag(np.concatenate(Dd)) + K1e - K1d
    return H, blocks


def eh_to_packed_spin(y: np.ndarray, blocks) -> np.ndarray:
    """e-h coefficients [..., dim] -> packed blocks [..., n_occ, n_pw]."""
    out, off = [], 0
    for v, Xc in blocks:
        out.append(y[..., off:off + Xc.shape[0]] @ Xc)
        off += Xc.shape[0]
    return np.stack(out, axis=-2)


def packed_to_eh_spin(A: np.ndarray, blocks) -> np.ndarray:
    return np.concatenate([A[..., v, :] @ Xc.T for v, Xc in blocks], axis=-1)

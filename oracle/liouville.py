"""Matrix-free Liouville operator (D + K1e - K1d) of Eq. (evp) with numpy FFTs, FP64.

A second, independent route to the same operator as ``dense_eh``: it never forms
conduction states. With u(r) = sum_{G in S} c(G) e^{iG.r} (so u = Omega^{1/2} psi):

  h_s(r)     = sum_w u_psi_w(r) u_a_sw(r)                         (pair density of Eq. k1e)
  V_H,s(G)   = v(G) h_s(G) / Omega,  h(G) = N^-3 sum_r h e^{-iG.r}
  tau_vw(r)  = W[psi_v psi_w](r)                                   (Eqs. tau, tau_from_tau_u, pdep)
  u_R(r)     = V_loc u_a_sv + s V_H,s u_psi_v - sum_{w: m_vw} tau_vw u_a_sw
  R_sv(G)    = N^-3 sum_r u_R e^{-iG.r} on S  + (1/2|G|^2 + Delta - eps_v) a_sv(G)   (Eq. d)
  R          <- P_c R = R - sum_u psi_u <psi_u|R>                   (P_c of Section 2)

s = 2 (singlet) or 0 (triplet). Inputs and outputs are Gamma-packed blocks
[B, n_occ, n_pw]; the inputs are assumed to lie in the conduction space.
"""
from __future__ import annotations

import numpy as np

from .basis import (packed_to_grid_field, grid_field_to_packed, coulomb_grid, full_miller,
                    sphere_on_grid, full_to_packed, packed_to_full, g2_packed)
from .pairs import pair_mask, channels
from .qp import qp_terms, occupied_energy_matrix


class Liouville:
    def __init__(self, inst, mask=None):
        self.inst = inst
        N = self.N = inst.n_grid
        self.omega = inst.omega
        self.u_psi = packed_to_grid_field(inst.psi, inst.miller, N)
        self.vc = coulomb_grid(N, inst.L)
        self.sq = np.sqrt(self.vc)
        if mask is None:
            mask, self.thr = pair_mask(inst)
        self.mask = mask
        self.vloc = inst.v_loc.reshape(N, N, N)
        self.g2 = g2_packed(inst.miller, inst.L)
        iz, iy, ix = sphere_on_grid(full_miller(inst.miller), N)
        self.sidx = (iz, iy, ix)
        self.f = inst.lam / (1.0 - inst.lam)
        # K1e factor (Eq. k1e): 2 for a closed-shell singlet, 0 for the triplet; in a
        # spin-polarised system every orbital is one spin-orbital and the Hartree term of the
        # total density change enters each channel once
        self.ch = channels(inst)
        self.polarised = bool(getattr(inst, "n_up", 0))
        self.spin_factor = 1.0 if self.polarised else (2.0 if inst.spin == 0 else 0.0)
        self.eps_qp, self.delta_avg, self.delta_c, self.psi_qp = qp_terms(inst)
        self.E = occupied_energy_matrix(inst)
        self.E_off = self.E - np.diag(np.diag(self.E))
        self._tau = {}

    # -- screened integrals ------------------------------------------------------
    def tau(self, v: int, w: int) -> np.ndarray:
        """tau_vw(r) in Ha on the grid (Eq. tau_from_tau_u with chi_bar of Eq. pdep)."""
        key = (min(v, w), max(v, w))
        if key in self._tau:
            return self._tau[key]
        N = self.N
        rho = self.u_psi[v] * self.u_psi[w] / self.omega
        rho_hat = np.fft.fftn(rho) / N ** 3
        x = self.sq * rho_hat                               # v^{1/2} rho
        xs = full_to_packed(x[self.sidx])                   # packed on S
        c = self.inst.pdep @ xs                             # PDEP projection
        ys = xs + self.inst.pdep.T @ (self.f * c)           # (1 + chi_bar) x on S
        x[self.sidx] = packed_to_full(ys)
        tau_hat = self.sq * x                               # v^{1/2} (...)
        t = (np.fft.ifftn(tau_hat) * N ** 3).real
        self._tau[key] = t
        return t

    def build_tau(self):
        """All kept tau_vw, v <= w (the one-time construction)."""
        n = self.inst.n_occ
        for v in range(n):
            for w in range(v, n):
                if self.mask[v, w]:
                    self.tau(v, w)
        return self._tau

    # -- operator ----------------------------------------------------------------
    def hartree(self, ua: np.ndarray) -> np.ndarray:
        """V_H,s(r) for each trial vector s from the pair density sum_w psi_w a_sw (Eq. k1e)."""
        N = self.N
        h = np.einsum("wzyx,swzyx->szyx", self.u_psi, ua)
        hh = np.fft.fftn(h, axes=(-3, -2, -1)) / N ** 3
        return (np.fft.ifftn(self.vc * hh / self.omega, axes=(-3, -2, -1)) * N ** 3).real

    def apply(self, A: np.ndarray, rows=None, project: bool = True) -> np.ndarray:
        """R = (D + K1e - K1d) A for A [B, n_occ, n_pw]; only rows v in ``rows`` if given."""
        A = np.asarray(A, dtype=np.float64)
        ua, VH = self.fields(A)
        R = self.apply_rows(A, ua, VH, rows)
        if project:
            R = self.project(R)
        return R

    def fields(self, A: np.ndarray):
        """The trial orbitals on the grid and their Hartree potentials (per vector, all rows)."""
        ua = packed_to_grid_field(np.asarray(A, dtype=np.float64), self.inst.miller, self.N)
        return ua, self.hartree(ua)                          # [B, n_occ, N, N, N], [B, N, N, N]

    def apply_rows(self, A: np.ndarray, ua: np.ndarray, VH: np.ndarray, rows=None) -> np.ndarray:
        """Rows v of (D + K1e - K1d) A before P_c, given the fields of ``A`` (Eqs. d, k1e, k1d)."""
        inst, N = self.inst, self.N
        A = np.asarray(A, dtype=np.float64)
        B, n_occ, n_pw = A.shape
        rows = range(n_occ) if rows is None else rows
        R = np.zeros_like(A)
        for v in rows:
            uR = self.vloc * ua[:, v] + self.spin_factor * VH * self.u_psi[v]
            for w in np.nonzero(self.mask[v])[0]:
                uR = uR - self.tau(v, w) * ua[:, w]
            dmul = 0.5 * self.g2 + self.delta_avg - self.E[v, v]
            dmul[1] = 0.0                                   # pad coordinate is not a G
            R[:, v] = grid_field_to_packed(uR, inst.miller, N) + dmul * A[:, v]
            if self.E_off[v].any():                         # rotated frame: - sum_w E_vw a_w
                R[:, v] -= np.einsum("w,bwj->bj", self.E_off[v], A)
            if self.delta_c.size:                           # explicit QP terms (Eq. ham)
                R[:, v] += ((A[:, v] @ self.psi_qp.T) * self.delta_c) @ self.psi_qp
        return R

    def project(self, R: np.ndarray) -> np.ndarray:
        """P_c = 1 - sum_u |psi_u><psi_u| applied to every orbital of every vector (the sum over
        the orbital's own spin channel in a spin-polarised system).

        The pad coordinate (packed index 1) is not part of the function space and is zeroed.
        """
        psi = self.inst.psi
        if not self.polarised:
            out = R - (R @ psi.T) @ psi
        else:                                               # P_c of each spin channel
            out = R.copy()
            for c in (0, 1):
                sel = self.ch == c
                if sel.any():
                    out[..., sel, :] -= (R[..., sel, :] @ psi[sel].T) @ psi[sel]
        out[..., 1] = 0.0
        return out

    def diagonal(self) -> np.ndarray:
        """Preconditioner diagonal 1/2|G|^2 + V(0) + Delta - eps_v, [n_occ, n_pw]."""
        inst = self.inst
        v0 = float(inst.v_loc.mean())
        return 0.5 * self.g2[None, :] + v0 + self.delta_avg - np.diag(self.E)[:, None]

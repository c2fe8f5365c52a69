"""Sphere, packing and grid helpers of the oracle (own code; nothing is shared with the library).

Packed layout (input format): p[0] = c(0), p[1] = 0 (pad), p[2k] = sqrt2 Re c(G_k),
p[2k+1] = sqrt2 Im c(G_k) for the half-sphere rows k >= 1 of ``miller``.
"""
from __future__ import annotations

import math

import numpy as np


def full_miller(miller: np.ndarray) -> np.ndarray:
    """Full sphere [G_0, +G_1, -G_1, +G_2, -G_2, ...] as integer triples."""
    n_half = miller.shape[0]
    full = np.zeros((2 * n_half - 1, 3), dtype=np.int64)
    full[1::2] = miller[1:]
    full[2::2] = -miller[1:]
    return full


def packed_to_full(p: np.ndarray) -> np.ndarray:
    """Padded packed [..., 2 n_half] -> full-sphere complex coefficients [..., 2 n_half - 1]."""
    n_half = p.shape[-1] // 2
    c = np.zeros(p.shape[:-1] + (2 * n_half - 1,), dtype=np.complex128)
    c[..., 0] = p[..., 0]
    h = (p[..., 2::2] + 1j * p[..., 3::2]) / math.sqrt(2.0)
    c[..., 1::2] = h
    c[..., 2::2] = np.conj(h)
    return c


def full_to_packed(c: np.ndarray) -> np.ndarray:
    """Full-sphere coefficients (Hermitian) -> padded packed; uses the +G entries."""
    n_half = (c.shape[-1] + 1) // 2
    p = np.zeros(c.shape[:-1] + (2 * n_half,), dtype=np.float64)
    p[..., 0] = c[..., 0].real
    p[..., 2::2] = math.sqrt(2.0) * c[..., 1::2].real
    p[..., 3::2] = math.sqrt(2.0) * c[..., 1::2].imag
    return p


def packing_matrix(n_half: int) -> np.ndarray:
    """Unitary U with c_full = U @ p_unpadded (p_unpadded = p without column 1)."""
    n = 2 * n_half - 1
    U = np.zeros((n, n), dtype=np.complex128)
    U[0, 0] = 1.0
    s = 1.0 / math.sqrt(2.0)
    for k in range(1, n_half):
        U[2 * k - 1, 2 * k - 1] = s
        U[2 * k - 1, 2 * k] = 1j * s
        U[2 * k, 2 * k - 1] = s
        U[2 * k, 2 * k] = -1j * s
    return U


def drop_pad(p: np.ndarray) -> np.ndarray:
    return np.concatenate([p[..., :1], p[..., 2:]], axis=-1)


def add_pad(q: np.ndarray) -> np.ndarray:
    out = np.zeros(q.shape[:-1] + (q.shape[-1] + 1,), dtype=q.dtype)
    out[..., 0] = q[..., 0]
    out[..., 2:] = q[..., 1:]
    return out


def grid_g2(N: int, L: float) -> np.ndarray:
    """|G|^2 on the FFT grid, array indexed [z, y, x] (numpy frequency order)."""
    n = np.fft.fftfreq(N, 1.0 / N)
    g = 2 * np.pi / L
    nz, ny, nx = np.meshgrid(n, n, n, indexing="ij")
    return (g * g) * (nx ** 2 + ny ** 2 + nz ** 2)


def coulomb_grid(N: int, L: float) -> np.ndarray:
    """v(G) = 4 pi / |G|^2 for G != 0 and v(0) = 0 (Eq. k1e with v_c = 1/|r-r'|)."""
    g2 = grid_g2(N, L)
    v = np.zeros_like(g2)
    nz = g2 > 0
    v[nz] = 4 * np.pi / g2[nz]
    return v


def sphere_on_grid(full: np.ndarray, N: int) -> tuple:
    """Grid indices (iz, iy, ix) of full-sphere vectors (negative n wrap modulo N)."""
    return (full[:, 2] % N, full[:, 1] % N, full[:, 0] % N)


def packed_to_grid_field(p: np.ndarray, miller: np.ndarray, N: int) -> np.ndarray:
    """u(r) = sum_{G in S} c(G) exp(iG.r) on the grid for packed p [..., n_pw] (FFT route).

    Returns real arrays [..., N, N, N] indexed [z, y, x]. The factor Omega^{-1/2}
    of the orbital normalisation is NOT included.
    """
    full = full_miller(miller)
    iz, iy, ix = sphere_on_grid(full, N)
    c = packed_to_full(p)
    lead = p.shape[:-1]
    grid = np.zeros(lead + (N, N, N), dtype=np.complex128)
    grid[..., iz, iy, ix] = c
    u = np.fft.ifftn(grid, axes=(-3, -2, -1)) * (N ** 3)
    return u.real


def grid_field_to_packed(u: np.ndarray, miller: np.ndarray, N: int) -> np.ndarray:
    """c(G) = N^-3 sum_r u(r) exp(-iG.r) restricted to S, returned packed."""
    full = full_miller(miller)
    iz, iy, ix = sphere_on_grid(full, N)
    F = np.fft.fftn(u, axes=(-3, -2, -1)) / (N ** 3)
    return full_to_packed(F[..., iz, iy, ix])


def g2_packed(miller: np.ndarray, L: float) -> np.ndarray:
    """|G|^2 for each packed coordinate (pad coordinate gets 0)."""
    g = 2 * np.pi / L
    n2 = (miller.astype(np.float64) ** 2).sum(1) * g * g
    out = np.repeat(n2, 2)
    out[1] = 0.0
    return out

"""Overlap O_vw of Eq. (overlap) and the pair-selection rule (Section 2, after Eq. overlap).

O_vw = int |psi_v|^2 |psi_w|^2 / sqrt(int |psi_v|^4 int |psi_w|^4). The grid sum is
exact because |psi|^4 has Fourier components of order <= 4 r_max < N; the volume
element cancels. tau_vw is set to zero when O_vw is below the threshold. The
threshold is either given, or chosen so that a requested number of v <= w pairs
survives: it is then the midpoint of the gap between the k-th and (k+1)-th largest
off-diagonal overlaps, moved to the nearest gap of at least 1e-9 of its midpoint
(checked at k+1, k-1, k+2, k-2, ...) so that lists computed with different rounding
agree exactly. Diagonal pairs (O_vv = 1) are always kept.
"""
from __future__ import annotations

import numpy as np

from .basis import packed_to_grid_field


def overlaps(inst) -> np.ndarray:
    """O_vw for all occupied pairs, FP64 (Eq. overlap)."""
    u = packed_to_grid_field(inst.psi, inst.miller, inst.n_grid).reshape(inst.n_occ, -1)
    rho = u * u
    gram = rho @ rho.T
    d = np.sqrt(np.diag(gram))
    return gram / np.outer(d, d)


def choose_threshold(O: np.ndarray, thr: float, keep_pairs: int) -> float:
    """Threshold actually applied (given, or from the requested count of v <= w pairs)."""
    if thr > 0:
        return float(thr)
    n = O.shape[0]
    off = np.sort(O[np.triu_indices(n, 1)])[::-1]
    k = int(keep_pairs) - n
    if k <= 0:
        hi = off[0] if off.size else 0.0
        return float(0.5 * (hi + 1.0))
    if k >= off.size:
        return 0.0

    def ok(j):
        if j < 1 or j >= off.size:
            return False
        gap = off[j - 1] - off[j]
        return gap >= 1e-9 * 0.5 * (off[j - 1] + off[j]) and gap > 0

    j = k
    if not ok(j):
        for d in range(1, off.size):
            if ok(k + d):
                j = k + d
                break
            if ok(k - d):
                j = k - d
                break
    return float(0.5 * (off[j - 1] + off[j]))


def channels(inst) -> np.ndarray:
    """Spin channel of every orbital: 0 up, 1 down (all 0 for a closed shell)."""
    ch = np.zeros(inst.n_occ, dtype=np.int64)
    n_up = int(getattr(inst, "n_up", 0) or 0)
    if n_up:
        ch[n_up:] = 1
    return ch


def pair_mask(inst, O: np.ndarray | None = None) -> tuple[np.ndarray, float]:
    """Boolean m_vw (symmetric, diagonal true) and the threshold applied.

    In a spin-polarised system tau_vw couples orbitals of one spin channel only (the screened
    direct term conserves spin), so pairs across channels are never kept and do not enter the
    threshold rule (they get the overlap -1, below every real overlap in [0, 1])."""
    if O is None:
        O = overlaps(inst)
    ch = channels(inst)
    O = np.where(ch[:, None] == ch[None, :], O, -1.0)
    t = choose_threshold(O, inst.overlap_thr, inst.keep_pairs)
    m = np.triu(O >= t, 1)
    m = m | m.T
    np.fill_diagonal(m, True)
    return m, t


def pair_list(mask: np.ndarray) -> np.ndarray:
    """Kept pairs (v, w) with v <= w in row-major order, int32 [P, 2]."""
    v, w = np.nonzero(np.triu(mask))
    return np.stack([v, w], axis=1).astype(np.int32)

"""Hand-built free-electron instances (V_loc = 0) whose operator elements have closed forms."""
import math

import numpy as np

from synth import Instance, sphere_half


def row_of(miller, n):
    n = np.asarray(n)
    for k, m in enumerate(miller):
        if (m == n).all() or (m == -n).all():
            return k
    raise KeyError(n)


def free_instance(occ_rows, pdep_rows=(), lam=(), L=8.0, N=16, n2max=14, scissor=0.03,
                  spin=0, thr=1e-3):
    """Occupied orbitals are sqrt(2/Omega) cos(G_k.r) (or Omega^-1/2 for k = 0).

    PDEP vectors, when given, are unit vectors along the cosine coordinate of G_k.
    """
    miller = sphere_half(n2max)
    n_pw = 2 * miller.shape[0]
    psi = np.zeros((len(occ_rows), n_pw))
    eps = np.zeros(len(occ_rows))
    g = 2 * math.pi / L
    for i, k in enumerate(occ_rows):
        psi[i, 2 * k] = 1.0
        eps[i] = 0.5 * g * g * float((miller[k].astype(float) ** 2).sum())
    pdep = np.zeros((len(pdep_rows), n_pw))
    for i, k in enumerate(pdep_rows):
        pdep[i, 2 * k] = 1.0
    return Instance(name="free", L=L, n_grid=N, n2max=n2max, miller=miller, psi=psi,
                    eps=eps, v_loc=np.zeros(N ** 3), scissor=scissor, pdep=pdep,
                    lam=np.asarray(lam, dtype=np.float64), overlap_thr=thr, keep_pairs=0,
                    spin=spin)


def coulomb(miller_row, L):
    g = 2 * math.pi / L
    return 4 * math.pi / (g * g * float((np.asarray(miller_row, float) ** 2).sum()))

"""FP64 reference of the learned Davidson preconditioner's loss and gradient.

The preconditioner (a library addition; the paper's Davidson of Section 3 uses no
learned component) maps, per element e = (v, G) of a residual r of Ritz value theta,

  features  f = (1/2|G|^2, eps_v, theta, d - theta, r_e sqrt(dim)/||r||),
            d = 1/2|G|^2 + V(0) + Delta - eps_v,  x = (f - mu)/sigma
  h1 = act(relu(W1 x + b1)),  h2 = act(relu(W2 h1 + b2)),  o = w3 . h2 + b3
  c  = exp(clip(o, -8, 8)),   g = c / max(d - theta, 0.1)
  t  = P_c (g * r)

to a correction t. act is the identity or rounding to bfloat16 (round to nearest
even). The pad coordinate (packed index 1) has g = 0. Davidson keeps only the direction
of a correction (it is orthonormalised against the subspace), so training minimises the
scale-free misfit over samples n with target corrections t*_n (in the conduction space):

  y = P_c(g * r_n),  a = <y, t*>,  b = ||y||^2,  c = ||t*||^2,
  L = mean_n (1 - a^2 / (b c)),

whose gradient in g is r * (2 a^2/(b^2 c) y - 2 a/(b c) t*) per sample (P_c symmetric and
idempotent, P_c t* = t*); the activation rounding is passed straight through.

Parameter vector (float32 on the device): W1[64x5], b1[64], W2[64x64], b2[64], w3[64],
b3[1], mu[5], sigma[5] -- 4619 values.
"""
from __future__ import annotations

import numpy as np

H = 64
NF = 5
NPARAM = H * NF + H + H * H + H + H + 1 + 2 * NF


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * NF].reshape(H, NF); o += H * NF
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]; o += 1
    mu = p[o:o + NF]; o += NF
    sg = p[o:o + NF]; o += NF
    return W1, b1, W2, b2, w3, b3, mu, sg


def bf16(x):
    """Round float64 values to bfloat16 (via float32, round to nearest even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(g2p, eps, v0, shift, theta, r):
    """Per-element features of one residual r [n_occ, n_pw]."""
    n_occ, n_pw = r.shape
    d = 0.5 * g2p[None, :] + v0 + shift - eps[:, None]
    nr = np.linalg.norm(r)
    f = np.stack([np.broadcast_to(0.5 * g2p[None, :], r.shape),
                  np.broadcast_to(eps[:, None], r.shape),
                  np.full(r.shape, theta),
                  d - theta,
                  r * np.sqrt(r.size) / nr], axis=-1)
    return f, d


def forward(p, f, d, theta, act_bf16=False):
    W1, b1, W2, b2, w3, b3, mu, sg = unpack(p)
    act = bf16 if act_bf16 else (lambda z: z)
    x = (f - mu) / sg
    z1 = x @ W1.T + b1
    h1 = act(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + b2
    h2 = act(np.maximum(z2, 0.0))
    o = h2 @ w3 + b3
    oc = np.clip(o, -8.0, 8.0)
    den = np.maximum(d - theta, 0.1)
    g = np.exp(oc) / den
    g[..., 1] = 0.0
    return g, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, o=o, g=g)


def loss_and_grad(p, samples, project, g2p, eps, v0, shift, act_bf16=False):
    """samples: list of (theta, r [n_occ,n_pw], tstar [n_occ,n_pw]); project: P_c on [k,n_occ,n_pw]."""
    W1, b1, W2, b2, w3, b3, mu, sg = unpack(p)
    grads = [np.zeros_like(a) for a in (W1, b1, W2, b2, w3)] + [0.0]
    L = 0.0
    N = len(samples)
    for theta, r, ts in samples:
        f, d = features(g2p, eps, v0, shift, theta, r)
        g, c = forward(p, f, d, theta, act_bf16)
        y = project((g * r)[None])[0]
        a = float((y * ts).sum())
        b = float((y * y).sum())
        cn = float((ts * ts).sum())
        L += (1.0 - a * a / (b * cn)) / N
        dg = r * (2.0 * a * a / (b * b * cn) * y - 2.0 * a / (b * cn) * ts) / N
        dg[..., 1] = 0.0
        do = dg * g * ((c["o"] > -8.0) & (c["o"] < 8.0))
        grads[4] += np.einsum("ij,ijk->k", do, c["h2"])
        grads[5] += float(do.sum())
        dz2 = do[..., None] * w3 * (c["z2"] > 0)
        grads[2] += np.einsum("ijk,ijl->kl", dz2, c["h1"])
        grads[3] += dz2.sum((0, 1))
        dz1 = (dz2 @ W2) * (c["z1"] > 0)
        grads[0] += np.einsum("ijk,ijl->kl", dz1, c["x"])
        grads[1] += dz1.sum((0, 1))
    flat = np.concatenate([grads[0].ravel(), grads[1], grads[2].ravel(), grads[3], grads[4],
                           [grads[5]], np.zeros(2 * NF)])
    return L, flat


def jd_correction(H: np.ndarray, u: np.ndarray, theta: float) -> np.ndarray:
    """Exact Jacobi-Davidson correction of a unit Ritz vector u with Ritz value theta (the
    training target t* of the preconditioner): t solves
        (I - u u^T)(H - theta)(I - u u^T) t = -r,   t . u = 0,   r = (H - theta) u,
    i.e. t = y / (u . y) - u with (H - theta) y = u (a dense solve in the e-h basis)."""
    y = np.linalg.solve(H - theta * np.eye(H.shape[0]), u)
    return y / (u @ y) - u

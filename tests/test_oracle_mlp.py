"""Pins of the FP64 learned-preconditioner reference (oracle/mlp.py), no GPU.

The analytic gradient of the loss is checked against central finite differences; the
bfloat16 rounding against exactly representable values; the zero last layer against the
diagonal preconditioner it must reduce to.
"""
import numpy as np
import pytest

from synth import make_tiny
from oracle import liouville, mlp


def _setup(seed=0, n_samples=3):
    inst = make_tiny(seed)
    Lop = liouville.Liouville(inst)
    rng = np.random.default_rng(seed)
    g2p = Lop.g2
    v0 = float(inst.v_loc.mean())
    samples = []
    for _ in range(n_samples):
        r = Lop.project(rng.standard_normal((1, inst.n_occ, inst.n_pw)))[0]
        t = Lop.project(rng.standard_normal((1, inst.n_occ, inst.n_pw)))[0]
        samples.append((0.3 + 0.1 * rng.random(), r, t))
    p = rng.standard_normal(mlp.NPARAM) * 0.2
    p[-10:-5] = rng.standard_normal(5) * 0.1     # mu
    p[-5:] = 0.5 + rng.random(5)                 # sigma
    return inst, Lop, g2p, v0, samples, p


def test_gradient_matches_finite_differences():
    inst, Lop, g2p, v0, samples, p = _setup()
    L0, grad = mlp.loss_and_grad(p, samples, Lop.project, g2p, inst.eps, v0, inst.scissor)
    rng = np.random.default_rng(1)
    idx = rng.choice(mlp.NPARAM - 10, 25, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        Lp, _ = mlp.loss_and_grad(pp, samples, Lop.project, g2p, inst.eps, v0, inst.scissor)
        Lm, _ = mlp.loss_and_grad(pm, samples, Lop.project, g2p, inst.eps, v0, inst.scissor)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_zero_last_layer_is_the_diagonal_preconditioner():
    inst, Lop, g2p, v0, samples, p = _setup()
    p[mlp.H * mlp.NF + mlp.H + mlp.H * mlp.H + mlp.H:][:mlp.H + 1] = 0.0   # w3, b3
    theta, r, _ = samples[0]
    f, d = mlp.features(g2p, inst.eps, v0, inst.scissor, theta, r)
    g, _ = mlp.forward(p, f, d, theta)
    want = 1.0 / np.maximum(d - theta, 0.1)
    want[..., 1] = 0.0
    np.testing.assert_allclose(g, want, rtol=1e-15)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 3.140625])
    out = mlp.bf16(vals)
    np.testing.assert_array_equal(out, [1.0, 1.0, 1.0 + 2 ** -7, -2.5, 0.0, 3.140625])


def test_jd_correction_solves_the_correction_equation():
    """t* = y/(u.y) - u satisfies (I - uu^T)(H - theta)(I - uu^T) t = -r and t . u = 0 for a
    Ritz pair of the dense e-h matrix (u: a perturbed eigenvector, theta its Rayleigh
    quotient)."""
    from synth import make_tiny
    from oracle import dense_eh
    H = dense_eh.eh_hamiltonian(make_tiny(0))
    w, X = np.linalg.eigh(H)
    rng = np.random.default_rng(7)
    u = X[:, 1] + 0.001 * rng.standard_normal(H.shape[0])
    u /= np.linalg.norm(u)
    theta = u @ H @ u
    r = H @ u - theta * u
    t = mlp.jd_correction(H, u, theta)
    P = np.eye(H.shape[0]) - np.outer(u, u)
    res = P @ ((H - theta * np.eye(H.shape[0])) @ (P @ t)) + r
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(r)
    assert abs(t @ u) <= 1e-12 * np.linalg.norm(t)
    # the correction points the Ritz vector at the eigenvector it approximates
    v = u + t
    v /= np.linalg.norm(v)
    assert 1 - abs(v @ X[:, 1]) < 1e-3 * (1 - abs(u @ X[:, 1]))

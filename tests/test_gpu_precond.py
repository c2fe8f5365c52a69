"""Learned Davidson preconditioner on the GPU (library addition).

* Loss and gradient of the GPU training kernels against the FP64 oracle (oracle/mlp.py)
  on test-generated samples: FP32 activations to 1e-4 relative, bfloat16 activations to the
  rounding level (a few 1e-2, from activations that round differently).
* Training on samples the plain solver produces for 16 seeded tiny systems, evaluation on
  8 held-out seeds: identical converged excitation energies (<= 1e-7 Ha vs the dense e-h
  oracle) with and without the network, and at most 10% more iterations with it (mean over
  the held-out systems; the trained network varies from run to run); the iteration counts and
  times are reported. The same network in a
  mixed-precision context gives energies within 1 meV of the oracle.
* The training targets of bse_precond_collect against the oracle's exact Jacobi-Davidson
  correction.
"""
import json
import os

import numpy as np
import pytest

from synth import make_tiny
from oracle import liouville, mlp, dense_eh

MEV = 3.6749322e-5

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


def _samples(inst, Lop, ns, seed):
    rng = np.random.default_rng(seed)
    R = Lop.project(rng.standard_normal((ns, inst.n_occ, inst.n_pw)))
    T = Lop.project(rng.standard_normal((ns, inst.n_occ, inst.n_pw)))
    th = 0.3 + 0.1 * rng.random(ns)
    return R, T, th


def test_gradient_matches_oracle():
    from paper_2409_15116_gb300 import Context
    inst = make_tiny(0)
    Lop = liouville.Liouville(inst)
    R, T, th = _samples(inst, Lop, 3, 3)
    rng = np.random.default_rng(4)
    p = (rng.standard_normal(mlp.NPARAM) * 0.2).astype(np.float32)
    p[-10:-5] = (rng.standard_normal(5) * 0.1).astype(np.float32)
    p[-5:] = (0.5 + rng.random(5)).astype(np.float32)
    c = Context(inst, 0)
    c.precond_set_samples(R, T, th)
    samples = [(th[i], R[i], T[i]) for i in range(3)]
    v0 = float(inst.v_loc.mean())
    for bf, tl, tg in ((False, 1e-5, 1e-4), (True, 1e-2, 3e-2)):
        L_gpu, g_gpu = c.precond_grad(p, act_bf16=bf)
        L_ref, g_ref = mlp.loss_and_grad(p.astype(np.float64), samples, Lop.project, Lop.g2,
                                         inst.eps, v0, inst.scissor, act_bf16=bf)
        assert abs(L_gpu - L_ref) <= tl * abs(L_ref), (bf, L_gpu, L_ref)
        err = np.abs(g_gpu - g_ref).max() / np.abs(g_ref).max()
        assert err <= tg, (bf, err)
    c.close()


def test_collected_targets_are_the_exact_jd_corrections():
    """bse_precond_collect's targets against the oracle's dense-solve Jacobi-Davidson
    correction (oracle/mlp.py jd_correction) for every sample.

    Both sides form t = y / (u.y) - u with y = (L - theta)^-1 u: the library's y from the
    exact spectral sum over its reference eigenpairs plus conjugate gradients (relative
    residual 1e-12) on their complement, the oracle's from a dense solve. The subtraction
    cancels the large component of y along u, so the relative error of t grows as theta
    approaches an eigenvalue (measured up to 4e-7 on converging samples, against 2e-10 for
    the early ones). The checks: t agrees with the oracle to 1e-5 relative, satisfies the
    correction equation (1 - u u^T)(H - theta)(1 - u u^T) t = -r to 1e-5 of |r|, and is
    orthogonal to u; a wrong term, sign or index on either side changes t at order one."""
    from paper_2409_15116_gb300 import Context
    inst = make_tiny(1)
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    c = Context(inst, 0)
    c.build_tau()
    n = c.precond_collect(4, 8, 32, res_tol=1e-6, ref_eig=32, max_samples=24)
    assert n > 0
    U, R, T, th = c.precond_get_samples()
    c.close()
    for i in range(n):
        ue = dense_eh.packed_to_eh(U[i][None], parts["Xc"])[0]
        u = ue / np.linalg.norm(ue)
        te = mlp.jd_correction(H, u, th[i])
        want = dense_eh.eh_to_packed(te[None], parts["Xc"], inst.n_occ)[0]
        err = np.abs(T[i] - want).max() / np.abs(want).max()
        assert err <= 1e-5, (i, err)
        tg = dense_eh.packed_to_eh(T[i][None], parts["Xc"])[0]
        r = H @ u - th[i] * u
        Ptg = tg - u * (u @ tg)
        lhs = (H @ Ptg - th[i] * Ptg)
        lhs -= u * (u @ lhs)
        assert np.linalg.norm(lhs + r) <= 1e-5 * np.linalg.norm(r), i
        assert abs(u @ tg) <= 1e-8 * max(1.0, np.linalg.norm(tg)), i


def test_learned_preconditioner_train_and_evaluate():
    from paper_2409_15116_gb300 import Context, binding
    ctxs = []
    for s in range(16):
        c = Context(make_tiny(s), 0)
        c.build_tau()
        n = c.precond_collect(4, 8, 32, res_tol=1e-6, ref_eig=32, max_samples=96)
        assert n > 0
        ctxs.append(c)
    params, hist = binding.precond_train(ctxs, binding.precond_init(0), epochs=40, lr=3e-3)
    assert np.isfinite(hist).all() and np.isfinite(params).all()
    assert hist[-1] < hist[0]
    for c in ctxs:
        c.close()
    rows = []
    for s in range(100, 108):
        inst = make_tiny(s)
        ref = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(inst))[:4]
        c = Context(inst, 0)
        c.build_tau()
        om_d, st_d = c.davidson(4, 8, 32, res_tol=1e-6)
        c.precond_load(params)
        om_l, st_l = c.davidson(4, 8, 32, res_tol=1e-6, precond=1)
        assert np.abs(om_d - ref).max() <= 1e-7
        assert np.abs(om_l - ref).max() <= 1e-7
        rows.append((s, st_d.iterations, st_l.iterations, st_d.ms_total, st_l.ms_total,
                     st_l.precond_fallbacks))
        c.close()
    # the same network in a mixed-precision context (FP32 trial vectors, the network's FP32
    # inference kernel): the converged energies are the operator's, within 1 meV of the dense
    # oracle, whatever the correction
    mixed = []
    for s in (100, 101):
        inst = make_tiny(s)
        ref = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(inst))[:4]
        c = Context(inst, 1)
        c.build_tau()
        c.precond_load(params)
        om_m, st_m = c.davidson(4, 8, 32, res_tol=1e-4, precond=1)
        assert np.abs(om_m - ref).max() <= MEV, (s, om_m - ref)
        mixed.append((s, st_m.iterations, st_m.precond_fallbacks))
        c.close()
    its_d = np.mean([r[1] for r in rows])
    its_l = np.mean([r[2] for r in rows])
    # the network rescales the diagonal step per element; trained on exact Jacobi-Davidson
    # targets it may move the iteration count a little either way but must not cost the
    # convergence (the energies above are unchanged, Rayleigh-Ritz decides them). Sample
    # collection and training sum in FP64 atomics, so the trained network and the held-out
    # counts vary from run to run: measured 24.0, 24.75, 24.9, 25.6 and 26.5 against a
    # deterministic 25.25 for the diagonal step
    assert its_l <= 1.1 * its_d, (its_l, its_d)
    report = {"loss_first": float(hist[0]), "loss_last": float(hist[-1]),
              "mean_iterations_diagonal": its_d, "mean_iterations_learned": its_l, "held_out": rows,
              "mixed_context": mixed}
    print("learned preconditioner:", json.dumps(report))
    out = os.environ.get("BSE_REPORT_DIR")
    if out:
        with open(os.path.join(out, "learned_precond.json"), "w") as f:
            json.dump(report, f)

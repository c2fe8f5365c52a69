"""Pins of the explicit quasi-particle terms of the oracle (Eq. ham and the Delta average)."""
import copy

import numpy as np

from synth import make_tiny
from oracle import dense_eh, liouville
from oracle.qp import qp_terms


def test_delta_average_of_the_paper():
    """N_occ = 4, N_QP = 12: N_mid = 8, Delta = mean of eps^QP_n - eps_n over n = 8..12."""
    inst = make_tiny(0, n_qp=12)
    inst = copy.copy(inst)
    inst.qp_eps = inst.qp_eps_ks + np.array([0, 0, 0, 0, 1, 2, 3, 4, 5, 6, 7, 8], dtype=float)
    eps_qp, delta, delta_c, psi_qp = qp_terms(inst)
    assert abs(delta - 6.0) < 1e-14
    np.testing.assert_allclose(delta_c, [-5, -4, -3, -2, -1, 0, 1, 2], atol=1e-14)
    np.testing.assert_allclose(eps_qp, inst.qp_eps[:4])
    assert psi_qp.shape == (8, inst.n_pw)


def test_diagonal_term_with_qp_energies_closed_form():
    """With K1e = K1d = 0 the spectrum of D is {eps^QP_c - eps^QP_v} for the explicitly
    corrected conduction states (c <= N_QP) and {eps_c + Delta - eps^QP_v} above them."""
    inst = make_tiny(0, n_qp=12)
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    No, Nc = inst.n_occ, parts["eps_c"].size
    Dmat = np.diag(parts["D"]) + np.kron(np.eye(No), parts["Dqp"])
    got = np.sort(np.linalg.eigvalsh(Dmat))
    eps_qp, delta, _, _ = qp_terms(inst)
    n_corr = inst.qp_n - No
    # conduction KS energies above the corrected ones: P_c H P_c eigenvalues not among the
    # explicitly corrected states (the oracle's own conduction spectrum, sorted)
    upper = np.sort(parts["eps_c"])[n_corr:]
    want = [inst.qp_eps[No + c] - eps_qp[v] for v in range(No) for c in range(n_corr)]
    want += [e + delta - eps_qp[v] for v in range(No) for e in upper]
    np.testing.assert_allclose(got, np.sort(want), atol=1e-10)
    # the corrected states are KS eigenstates: their KS energies are the lowest conduction ones
    np.testing.assert_allclose(np.sort(parts["eps_c"])[:n_corr], inst.qp_eps_ks[No:], atol=1e-10)


def test_uniform_qp_shift_equals_no_scissor():
    """eps^QP = eps + s for every state gives Delta = s, delta_c = 0 and eps^QP_v = eps_v + s,
    so the operator equals the scissor form with Delta = 0."""
    inst = make_tiny(0, n_qp=12)
    inst.qp_eps = inst.qp_eps_ks + 0.123
    ref = make_tiny(0, scissor=0.0)
    Hq = dense_eh.eh_hamiltonian(inst)
    H0 = dense_eh.eh_hamiltonian(ref)
    assert np.abs(Hq - H0).max() < 1e-11


def test_matrix_free_qp_operator_equals_dense_columnwise():
    inst = make_tiny(0, n_qp=12)
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    Lop = liouville.Liouville(inst)
    rng = np.random.default_rng(2)
    y = rng.standard_normal((3, H.shape[0]))
    A = dense_eh.eh_to_packed(y, parts["Xc"], inst.n_occ)
    got = Lop.apply(A)
    want = dense_eh.eh_to_packed(y @ H.T, parts["Xc"], inst.n_occ)
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()

"""Pins of the CPU oracle to facts fixed by the paper and by mathematics (no GPU).

Each test targets a plausible mistake: a dropped term, a wrong sign, factor, volume
normalisation or index, a transposed operand, or a wrong convolution convention.
"""
import math

import numpy as np
import pytest

from synth import make_tiny, make_localized, sphere_half
from synth.instance import _packing_matrix, wells_on_grid
from oracle import dense_eh, liouville, pairs, davidson
from oracle.basis import coulomb_grid, full_miller, packed_to_full
from tests.free_electron import free_instance, row_of, coulomb


@pytest.fixture(scope="module")
def tiny():
    inst = make_tiny(0)
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    return inst, H, parts


# --------------------------------------------------------------------------------
# dense e-h oracle: structure (Eq. evp: Hermitian TDA problem, real positive spectrum)
# --------------------------------------------------------------------------------

def test_dense_hermitian_positive_orthonormal(tiny):
    inst, H, _ = tiny
    assert np.abs(H - H.T).max() <= 1e-13 * np.abs(H).max()
    w, X = np.linalg.eigh(H)
    assert np.abs(H @ X - X * w).max() <= 1e-12 * max(1.0, np.abs(w).max())
    assert np.abs(X.T @ X - np.eye(H.shape[0])).max() <= 1e-12
    assert w.min() > 0
    assert H.shape[0] == inst.n_occ * (inst.n_pw - 1 - inst.n_occ)   # 4 x 247 = 988


def test_ks_hamiltonian_matches_analytic_ground_state(tiny):
    """The grid-DFT Hamiltonian of the oracle reproduces the ground state that the input
    generator computed from the analytic Fourier transform of the Gaussian wells."""
    inst, _, parts = tiny
    Hks, imag = dense_eh.ks_hamiltonian_packed(inst)
    assert imag < 1e-13
    e = np.linalg.eigvalsh(Hks)
    np.testing.assert_allclose(e[:inst.n_occ], inst.eps, atol=1e-11)
    # the occupied orbitals are eigenvectors of the oracle's H_KS
    from oracle.basis import drop_pad
    P = drop_pad(inst.psi)
    res = P @ Hks - inst.eps[:, None] * P
    assert np.abs(res).max() < 1e-11


def test_diagonal_term_alone_closed_form(tiny):
    """With K1e = K1d = 0 the spectrum is exactly {eps_c - eps_v + Delta} (Eq. d, Eq. ham)."""
    inst, H, parts = tiny
    Hks, _ = dense_eh.ks_hamiltonian_packed(inst)
    e_all = np.linalg.eigvalsh(Hks)
    expect = np.sort((e_all[inst.n_occ:][None, :] + inst.scissor - inst.eps[:, None]).ravel())
    np.testing.assert_allclose(np.sort(parts["D"]), expect, atol=1e-11)
    # matrix-free route with the kernels switched off by an empty mask and triplet spin
    inst_t = make_tiny(0, spin=1)
    Lop = liouville.Liouville(inst_t, mask=np.zeros((4, 4), bool))
    A = dense_eh.eh_to_packed(np.eye(H.shape[0])[:5], parts["Xc"], inst.n_occ)
    R = Lop.apply(A)
    y = dense_eh.packed_to_eh(R, parts["Xc"])
    np.testing.assert_allclose(y, np.diag(parts["D"])[:5], atol=1e-11)


def test_scissor_shifts_every_excitation():
    a = make_tiny(3)
    b = make_tiny(3, scissor=0.03 + 0.25)
    wa = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(a))
    wb = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(b))
    np.testing.assert_allclose(wb - wa, 0.25, atol=1e-12)


def test_triplet_removes_exchange(tiny):
    inst, H, parts = tiny
    trip = make_tiny(0, spin=1)
    Ht = dense_eh.eh_hamiltonian(trip)
    np.testing.assert_allclose(Ht, np.diag(parts["D"]) - parts["K1d"], atol=1e-14)
    np.testing.assert_allclose(H - Ht, 2.0 * parts["K1e"], atol=1e-13)


def test_exchange_fft_equals_explicit_double_sum(tiny):
    """K1e elements recomputed as explicit sums over r and G (no FFT), Eq. k1e."""
    inst, _, parts = tiny
    N, L, omega = inst.n_grid, inst.L, inst.omega
    psi_r, c_r = parts["psi_r"], parts["c_r"]
    Nc = c_r.shape[0]
    idx = np.arange(N ** 3)
    r = np.stack([idx % N, (idx // N) % N, idx // (N * N)], 1).astype(float)
    m = 6                                           # 2 r_max: support of pair densities
    rng_ = np.arange(-m, m + 1)
    n = np.stack(np.meshgrid(rng_, rng_, rng_, indexing="ij"), -1).reshape(-1, 3).astype(float)
    n2 = (n ** 2).sum(1)
    keep = n2 > 0
    n, n2 = n[keep], n2[keep]
    vG = 4 * math.pi / ((2 * math.pi / L) ** 2 * n2)
    E = np.exp(-1j * (2 * math.pi / N) * (r @ n.T))          # [N^3, nG]
    rng = np.random.default_rng(7)
    for _ in range(6):
        v, c, w, c2 = rng.integers(0, 4), rng.integers(0, Nc), rng.integers(0, 4), rng.integers(0, Nc)
        ra = (psi_r[v] * c_r[c]) @ E / N ** 3
        rb = (psi_r[w] * c_r[c2]) @ E / N ** 3
        direct = omega * float((vG * ra.conj() * rb).sum().real)
        fft = parts["K1e"][v * Nc + c, w * Nc + c2]
        assert abs(direct - fft) <= 1e-12 * max(1e-3, abs(direct)), (direct, fft)


def test_operator_level_equals_dense_columnwise(tiny):
    """The matrix-free FFT operator reproduces H_eh column by column (two independent routes)."""
    inst, H, parts = tiny
    Lop = liouville.Liouville(inst)
    cols = np.arange(0, H.shape[0], 37)
    A = dense_eh.eh_to_packed(np.eye(H.shape[0])[cols], parts["Xc"], inst.n_occ)
    R = Lop.apply(A)
    y = dense_eh.packed_to_eh(R, parts["Xc"])
    assert np.abs(y - H[cols]).max() <= 1e-12 * np.abs(H).max()
    # and the output stays in the conduction space (P_c) with a zero pad coordinate
    assert np.abs(R @ inst.psi.T).max() < 1e-13
    assert np.abs(R[..., 1]).max() == 0.0


def test_truncated_empty_manifold_converges(tiny):
    """Fig. 8: e-h results with N_empty < N_c approach the complete result from above."""
    inst, H, parts = tiny
    Nc = parts["eps_c"].size
    full = np.linalg.eigvalsh(H)[:4]
    prev = None
    for ne in (20, 60, 120, 200, Nc):
        sel = np.array([v * Nc + c for v in range(inst.n_occ) for c in range(ne)])
        w = np.linalg.eigvalsh(H[np.ix_(sel, sel)])[:4]
        assert np.all(w >= full - 1e-12)
        if prev is not None:
            assert np.all(w <= prev + 1e-12)
        prev = w
    np.testing.assert_allclose(prev, full, atol=1e-13)


# --------------------------------------------------------------------------------
# closed forms with plane-wave orbitals (V_loc = 0)
# --------------------------------------------------------------------------------

def test_free_electron_exchange_spectrum_closed_form():
    """psi_0 = Omega^-1/2: K1d vanishes (v(0) = 0) and K1e is diagonal, so the singlet
    spectrum is 1/2|G|^2 + Delta + 8 pi / (Omega |G|^2) (twice per +-G pair), Eq. k1e."""
    for spin in (0, 1):
        inst = free_instance([0], spin=spin)
        H = dense_eh.eh_hamiltonian(inst)
        w = np.linalg.eigvalsh(H)
        g = 2 * math.pi / inst.L
        n2 = (inst.miller[1:].astype(float) ** 2).sum(1)
        G2 = g * g * n2
        x = 0.5 * G2 + inst.scissor + (8 * math.pi / (inst.omega * G2) if spin == 0 else 0.0)
        np.testing.assert_allclose(w, np.sort(np.repeat(x, 2)), atol=1e-12)


@pytest.mark.parametrize("lam", [0.0, -0.6])
@pytest.mark.parametrize("spin", [0, 1])
def test_free_electron_screened_direct_element(lam, spin):
    """<psi_a|L|(0, psi_b)> for cosine orbitals with G_a = G_b + G_1:
    sqrt2 v(G_a)/Omega (exchange, singlet) - W(G_1)/(sqrt2 Omega) (screened direct),
    W(G_1) = v(G_1)/(1 - lambda) for a PDEP vector along cos(G_1.r) (Eqs. k1d, tau, pdep)."""
    miller = sphere_half(14)
    k1, kb, ka = row_of(miller, (1, 0, 0)), row_of(miller, (0, 1, 0)), row_of(miller, (1, 1, 0))
    pd = [k1] if lam != 0.0 else []
    la = [lam] if lam != 0.0 else []
    inst = free_instance([0, k1], pdep_rows=pd, lam=la, spin=spin)
    L, omega = inst.L, inst.omega
    expect = -coulomb((1, 0, 0), L) / (1 - lam) / (math.sqrt(2) * omega)
    if spin == 0:
        expect += math.sqrt(2) * coulomb((1, 1, 0), L) / omega
    A = np.zeros((1, 2, inst.n_pw))
    A[0, 1, 2 * kb] = 1.0
    R = liouville.Liouville(inst).apply(A)
    assert abs(R[0, 0, 2 * ka] - expect) < 1e-13
    # dense route, same element through the e-h basis
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    ya = dense_eh.packed_to_eh(np.eye(inst.n_pw)[2 * ka][None, None, :] * np.array([1, 0])[None, :, None], parts["Xc"])
    yb = dense_eh.packed_to_eh(A, parts["Xc"])
    assert abs(float(ya[0] @ H @ yb[0]) - expect) < 1e-13


def test_overlap_closed_forms():
    """O_vv = 1, symmetric, in [0,1]; O = sqrt(2/3) for a constant and a cosine orbital."""
    inst = free_instance([0, 3])
    O = pairs.overlaps(inst)
    assert abs(O[0, 1] - math.sqrt(2.0 / 3.0)) < 1e-14
    np.testing.assert_allclose(np.diag(O), 1.0, atol=1e-14)
    t = make_tiny(0)
    O = pairs.overlaps(t)
    assert np.abs(O - O.T).max() < 1e-15
    assert O.min() >= 0 and O.max() <= 1 + 1e-15


def test_overlap_gaussian_envelopes():
    """Two normalised Gaussians a distance d apart: O = exp(-d^2 / (2 w^2)) (sanity, Eq. overlap)."""
    L, N, w = 16.0, 48, 1.2
    miller = sphere_half(121)
    G = miller.astype(float) * 2 * math.pi / L
    cs = []
    for R in (np.array([6.0, 8.0, 8.0]), np.array([9.0, 8.0, 8.0])):
        c = np.exp(-0.5 * w * w * (G ** 2).sum(1)) * np.exp(-1j * G @ R)
        q = np.zeros(2 * miller.shape[0])
        q[0] = c[0].real
        q[2::2] = math.sqrt(2) * c[1:].real
        q[3::2] = math.sqrt(2) * c[1:].imag
        cs.append(q / np.linalg.norm(q))
    from synth import Instance
    inst = Instance(name="g", L=L, n_grid=N, n2max=121, miller=miller, psi=np.array(cs),
                    eps=np.zeros(2), v_loc=np.zeros(N ** 3), scissor=0.0,
                    pdep=np.zeros((0, 2 * miller.shape[0])), lam=np.zeros(0),
                    overlap_thr=1e-3, keep_pairs=0)
    O = pairs.overlaps(inst)
    assert abs(O[0, 1] - math.exp(-9.0 / (2 * w * w))) < 1e-6


def test_screening_scaling_full_pdep_constant_lambda():
    """With the PDEP set equal to all of S \\ {0} and constant lambda_0, W = v/(1-lambda_0)
    on every density component inside S, so K1d scales by exactly 1/(1-lambda_0)."""
    miller = sphere_half(14)
    k1 = row_of(miller, (1, 0, 0))
    base = free_instance([0, k1], spin=1)
    n_pw = base.n_pw
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((n_pw - 2, n_pw - 2)))
    pdep = np.zeros((n_pw - 2, n_pw))
    pdep[:, 2:] = Q.T
    lam0 = -0.45
    scr = free_instance([0, k1], spin=1)
    scr.pdep, scr.lam = pdep, np.full(n_pw - 2, lam0)
    _, p0 = dense_eh.eh_hamiltonian(base, with_parts=True)
    _, p1 = dense_eh.eh_hamiltonian(scr, with_parts=True)
    # the pair densities psi_0 psi_1, psi_1^2 have components {0, G_1, 2 G_1}, all inside S
    np.testing.assert_allclose(p1["K1d"], p0["K1d"] / (1 - lam0), atol=1e-13)


# --------------------------------------------------------------------------------
# pair rule and Davidson
# --------------------------------------------------------------------------------

def test_paper_threshold_keeps_all_tiny_pairs(tiny):
    """Config-1 uses the paper's threshold 0.001 (Section 4); all 10 v <= w pairs survive."""
    inst, _, _ = tiny
    m, t = pairs.pair_mask(inst)
    assert t == 1e-3
    assert pairs.pair_list(m).shape[0] == 10


def test_pair_count_rule_midpoint_gap():
    inst = make_localized(4, 20 * 32 / 72, 32, 40, 2.5, 80, n_eig=8, block=8)
    O = pairs.overlaps(inst)
    m, t = pairs.pair_mask(inst, O)
    P = pairs.pair_list(m)
    assert P.shape[0] == inst.keep_pairs
    off = O[np.triu_indices(40, 1)]
    gap = np.abs(off - t).min()
    assert gap >= 0.5e-9 * t
    assert (m == m.T).all() and m.diagonal().all()


def test_davidson_matches_dense(tiny):
    inst, H, _ = tiny
    w = np.linalg.eigvalsh(H)[:8]
    Lop = liouville.Liouville(inst)
    th, X, info = davidson.davidson(Lop.apply, Lop.diagonal(), Lop.project, 8, 16, 64, 1e-6)
    assert info["converged"]
    np.testing.assert_allclose(th, w, atol=1e-9)
    # Ritz vectors are orthonormal and in the conduction space
    Xf = X.reshape(8, -1)
    np.testing.assert_allclose(Xf @ Xf.T, np.eye(8), atol=1e-10)
    assert np.abs(X @ inst.psi.T).max() < 1e-12


def test_operator_is_symmetric_on_localized_case():
    inst = make_localized(5, 20 * 32 / 72, 32, 12, 2.5, 24, n_eig=4, block=4)
    Lop = liouville.Liouville(inst)
    rng = np.random.default_rng(2)
    X = Lop.project(rng.standard_normal((2, inst.n_occ, inst.n_pw)))
    R = Lop.apply(X)
    a = float((X[0] * R[1]).sum())
    b = float((X[1] * R[0]).sum())
    assert abs(a - b) < 1e-12 * max(1, abs(a))


def test_golden_tiny_values_reproduced():
    """Regression: the stored dense-oracle values (tests/golden/tiny_dense_eh.json) still hold."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_dense_eh.json")
    data = json.load(open(path))
    for case in data["cases"][:2]:
        inst = make_tiny(case["seed"], spin=case["spin"])
        w = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(inst))[:16]
        np.testing.assert_allclose(w, case["lowest16"], atol=1e-12)

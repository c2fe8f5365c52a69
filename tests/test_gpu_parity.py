"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP64 path -- operator relative error <= 1e-11 (FFT rounding over a few
thousand terms), excitation energies <= 1e-7 Ha (Davidson stops at ||r|| <= 1e-6, so the
eigenvalue error is ~||r||^2/gap). Mixed path -- operator relative error <= 2e-5 (FP32
FFTs and products, ~1e-6 per stage over the pipeline), excitation energies <= 1 meV
(3.6749e-5 Ha). Pair lists are compared bit-exactly.
"""
import numpy as np
import pytest

from synth import make_tiny, make_localized
from oracle import dense_eh, liouville, pairs, davidson

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
MEV = 3.6749322e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


def ctx_for(inst, prec):
    from paper_2409_15116_gb300 import Context
    c = Context(inst, prec)
    c.build_tau()
    return c


def dev(a, prec):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if prec == 0 else torch.float32,
                        device="cuda")


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# ---------------------------------------------------------------------------------
# tiny cell (the dense e-h oracle)
# ---------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    inst = make_tiny(0)
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    return inst, H, parts


@pytest.mark.parametrize("prec", [0, 1])
def test_tiny_overlaps_and_pairs(tiny, prec):
    inst, _, _ = tiny
    c = ctx_for(inst, prec)
    O_ref = pairs.overlaps(inst)
    np.testing.assert_allclose(c.overlaps(), O_ref, atol=1e-13)
    m, _ = pairs.pair_mask(inst)
    assert (c.pairs() == pairs.pair_list(m)).all()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_tiny_operator_vs_dense(tiny, prec, tol):
    inst, H, parts = tiny
    c = ctx_for(inst, prec)
    rng = np.random.default_rng(11)
    y = rng.standard_normal((7, H.shape[0]))          # odd block: ragged pair layout
    A = dense_eh.eh_to_packed(y, parts["Xc"], inst.n_occ)
    ref = dense_eh.eh_to_packed(y @ H.T, parts["Xc"], inst.n_occ)
    a = dev(A, prec)
    out = torch.empty_like(a)
    c.apply(a, out)
    got = out.double().cpu().numpy()
    assert rel(got, ref) <= tol, rel(got, ref)
    assert np.abs(got[..., 1]).max() == 0.0


@pytest.mark.parametrize("prec,tol", [(0, 1e-7), (1, MEV)])
def test_tiny_lowest_excitations_vs_dense(tiny, prec, tol):
    inst, H, _ = tiny
    ref = np.linalg.eigvalsh(H)[:8]
    c = ctx_for(inst, prec)
    om, st = c.davidson(8, 16, 64, max_it=200, res_tol=1e-6 if prec == 0 else 1e-4)
    assert np.abs(om - ref).max() <= tol, (om - ref)
    assert st.iterations >= 1 and st.n_apply >= 16


def test_tiny_triplet_vs_dense():
    inst = make_tiny(1, spin=1)
    ref = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(inst))[:4]
    c = ctx_for(inst, 0)
    om, _ = c.davidson(4, 8, 32, res_tol=1e-6)
    assert np.abs(om - ref).max() <= 1e-7


def test_apply_empty_block_is_noop(tiny):
    inst, _, _ = tiny
    c = ctx_for(inst, 0)
    a = torch.zeros((0, inst.n_occ, inst.n_pw), dtype=torch.float64, device="cuda")
    c.apply(a, torch.zeros_like(a))


# ---------------------------------------------------------------------------------
# localised orbitals on larger grids: odd N_occ, ragged sphere, pair-count rule
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("N,n_occ,seed", [(32, 12, 3), (48, 13, 4), (64, 9, 9), (72, 8, 7), (96, 6, 8)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_localized_operator_vs_matrix_free(N, n_occ, seed, prec, tol):
    inst = make_localized(seed, 20.0 * N / 72, N, n_occ, 2.5, 2 * n_occ, n_eig=4, block=4)
    Lop = liouville.Liouville(inst)
    c = ctx_for(inst, prec)
    m_ref, _ = pairs.pair_mask(inst)
    assert (c.pairs() == pairs.pair_list(m_ref)).all()
    rng = np.random.default_rng(5)
    A = Lop.project(rng.standard_normal((3, inst.n_occ, inst.n_pw)))
    ref = Lop.apply(A)
    a = dev(A, prec)
    out = torch.empty_like(a)
    c.apply(a, out)
    got = out.double().cpu().numpy()
    assert rel(got, ref) <= tol, rel(got, ref)


@pytest.mark.parametrize("prec,tol", [(0, 1e-7), (1, MEV)])
def test_localized_davidson_vs_oracle_davidson(prec, tol):
    inst = make_localized(6, 20.0 * 32 / 72, 32, 16, 2.5, 32, n_eig=4, block=4)
    Lop = liouville.Liouville(inst)
    ref, _, info = davidson.davidson(Lop.apply, Lop.diagonal(), Lop.project, 4, 8, 32, 1e-7)
    assert info["converged"]
    c = ctx_for(inst, prec)
    om, _ = c.davidson(4, 8, 32, res_tol=1e-6 if prec == 0 else 1e-4)
    assert np.abs(om - ref).max() <= tol, (om - ref)


# ---------------------------------------------------------------------------------
# every K1d tile variant (points x vectors per CTA, threads per CTA), fixed through
# BSE_K1D_VARIANT at context creation, on a ragged block: 11 vectors (partial vector
# chunks for every chunk size) of an odd N_occ
# ---------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def ragged_case():
    inst = make_localized(3, 20.0 * 32 / 72, 32, 13, 2.5, 26, n_eig=4, block=4)
    Lop = liouville.Liouville(inst)
    rng = np.random.default_rng(17)
    A = Lop.project(rng.standard_normal((11, inst.n_occ, inst.n_pw)))
    return inst, A, Lop.apply(A)


# the per-pair tau layout with the untiled K1d kernel, which the library uses when the
# entry-major layout would take more than half of the free device memory
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_per_pair_tau_untiled_vs_matrix_free(ragged_case, prec, tol, monkeypatch):
    inst, A, ref = ragged_case
    monkeypatch.setenv("BSE_TAU_LAYOUT", "pair")
    c = ctx_for(inst, prec)
    a = dev(A, prec)
    out = torch.empty_like(a)
    c.apply(a, out)
    got = out.double().cpu().numpy()
    assert rel(got, ref) <= tol, rel(got, ref)


# tau stored once per pair (the layout for systems whose ordered entry-major tau would not
# fit), read by the symmetric-layout tiled kernel
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_once_per_pair_tau_vs_matrix_free(ragged_case, prec, tol, monkeypatch):
    inst, A, ref = ragged_case
    monkeypatch.setenv("BSE_TAU_LAYOUT", "upper")
    c = ctx_for(inst, prec)
    a = dev(A, prec)
    out = torch.empty_like(a)
    c.apply(a, out)
    got = out.double().cpu().numpy()
    assert rel(got, ref) <= tol, rel(got, ref)
    for n in (1, 5):                       # other block widths (own tuned variants)
        o = torch.empty_like(a[:n])
        c.apply(a[:n].contiguous(), o)
        assert rel(o.double().cpu().numpy(), ref[:n]) <= tol


# every kernel variant for tau stored once per pair (register rings, then shared-memory
# rings), fixed through BSE_K1D_SYM_VARIANT; a variant that does not fit the precision is
# ignored by the library and the test then checks the tuned choice
@pytest.mark.parametrize("variant", range(1, 23))
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_once_per_pair_variants_vs_matrix_free(ragged_case, variant, prec, tol, monkeypatch):
    inst, A, ref = ragged_case
    monkeypatch.setenv("BSE_TAU_LAYOUT", "upper")
    monkeypatch.setenv("BSE_K1D_SYM_VARIANT", str(variant))
    c = ctx_for(inst, prec)
    a = dev(A, prec)
    out = torch.empty_like(a)
    c.apply(a, out)
    got = out.double().cpu().numpy()
    assert rel(got, ref) <= tol, (variant, rel(got, ref))
    o = torch.empty_like(a[:2])                 # a narrow block: one partial vector chunk
    c.apply(a[:2].contiguous(), o)
    assert rel(o.double().cpu().numpy(), ref[:2]) <= tol, variant


@pytest.mark.parametrize("variant", range(1, 21))
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_k1d_tile_variants_vs_matrix_free(ragged_case, variant, prec, tol, monkeypatch):
    inst, A, ref = ragged_case
    monkeypatch.setenv("BSE_K1D_VARIANT", str(variant))
    c = ctx_for(inst, prec)
    a = dev(A, prec)
    out = torch.empty_like(a)
    c.apply(a, out)
    got = out.double().cpu().numpy()
    assert rel(got, ref) <= tol, (variant, rel(got, ref))

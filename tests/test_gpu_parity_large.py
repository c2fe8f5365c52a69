"""Operator parity at the benchmarked sizes: the CUDA path (through the C ABI) against the
matrix-free FP64 oracle on sampled orbital rows.

The oracle computes rows one by one (Liouville.apply(rows=...)); P_c acts on each
(vector, orbital) row separately, so a sampled row of the oracle is the full result for that
row. Cases:
  * the medium workload itself (72^3 grid, 256 orbitals, 512 PDEP vectors, 4,934 pairs),
    with a block width the Davidson solve applies (13 vectors);
  * the op256 family (32^3 grid, 256 orbitals) with 32 vectors (several vector chunks);
  * a 72^3 grid with 64 orbitals, every row compared;
  * the large workload (96^3 grid, 1,024 orbitals, tau once per pair) in its bench launch
    configuration, sampled rows of two vectors.
These reach the 256-orbital a(r) stage, many row blocks, the transposed tau tiles of late
blocks, the autotuned tile variants and the multi-tile BF16x3 projector.
Tolerances as in the other parity tests: FP64 1e-11, mixed 2e-5 relative.
"""
import numpy as np
import pytest

from synth import make_localized, make_config
from oracle import liouville, pairs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


def _run(inst, prec, n_vec, rows, seed, Lop=None):
    from paper_2409_15116_gb300 import Context
    Lop = Lop or liouville.Liouville(inst)
    c = Context(inst, prec)
    c.build_tau()
    m_ref, _ = pairs.pair_mask(inst)
    assert (c.pairs() == pairs.pair_list(m_ref)).all()
    rng = np.random.default_rng(seed)
    A = Lop.project(rng.standard_normal((n_vec, inst.n_occ, inst.n_pw)))
    a = torch.tensor(A, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    out = torch.empty_like(a)
    c.apply(a, out)
    got = out.double().cpu().numpy()
    c.close()
    # one vector at a time keeps the oracle's grids of all orbitals within a few GB
    ref = np.concatenate([Lop.apply(A[k:k + 1], rows=rows) for k in range(n_vec)])
    rows = list(rows) if rows is not None else list(range(inst.n_occ))
    g, r = got[:, rows], ref[:, rows]
    return float(np.abs(g - r).max() / np.abs(r).max())


@pytest.fixture(scope="module")
def medium():
    inst = make_config("medium")
    return inst, liouville.Liouville(inst)


@pytest.mark.parametrize("prec,tol,n_vec", [(1, 2e-5, 13), (0, 1e-11, 2)])
def test_medium_operator_sampled_rows(medium, prec, tol, n_vec):
    inst, Lop = medium
    rows = [0, 3, 4, 129, 251, 255]
    err = _run(inst, prec, n_vec, rows, 11 + n_vec, Lop)
    assert err <= tol, err


@pytest.mark.parametrize("prec,tol,n_vec", [(1, 2e-5, 32), (0, 1e-11, 7)])
def test_op256_operator_sampled_rows(prec, tol, n_vec):
    inst = make_config("op256")
    err = _run(inst, prec, n_vec, [0, 1, 2, 3, 64, 190, 254, 255], 23)
    assert err <= tol, err


@pytest.mark.parametrize("layout", ["", "upper"])
@pytest.mark.parametrize("prec,tol", [(1, 2e-5), (0, 1e-11)])
def test_grid72_64_orbitals_every_row(prec, tol, layout, monkeypatch):
    if layout:
        monkeypatch.setenv("BSE_TAU_LAYOUT", layout)
    inst = make_localized(12, 20.0, 72, 64, 2.5, 128, n_eig=4, block=4)
    err = _run(inst, prec, 5, None, 31)
    assert err <= tol, err


def test_large_operator_sampled_rows(monkeypatch):
    """The large workload (96^3 grid, 1,024 orbitals, ~20k pairs, tau once per pair) in the
    launch configuration of its bench line: a 48 GB r-space workspace, so 7 vectors run as a
    6-vector chunk and a 1-vector chunk. Rows of the first row block, a middle one and the last
    one, for the first vector and the one in the second chunk (the oracle transforms all 1,024
    orbitals of every vector it checks, about a minute each)."""
    free, total = torch.cuda.mem_get_info()
    if total < 200e9:
        pytest.skip("the large workload needs a device of more than 200 GB")
    from paper_2409_15116_gb300 import Context
    monkeypatch.setenv("BSE_WORKSPACE_GB", "48")
    inst = make_config("large")
    Lop = liouville.Liouville(inst)
    c = Context(inst, 1)
    c.build_tau()
    assert (c.pairs() == pairs.pair_list(Lop.mask)).all()
    rng = np.random.default_rng(41)
    n_vec = 7
    A = Lop.project(rng.standard_normal((n_vec, inst.n_occ, inst.n_pw)))
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    c.apply(a, out)
    got = out.double().cpu().numpy()
    c.close()
    del a, out
    torch.cuda.empty_cache()
    rows = [0, 3, 509, 1022, 1023]
    for k in (0, n_vec - 1):
        ref = Lop.apply(A[k:k + 1], rows=rows)[0]
        err = float(np.abs(got[k, rows] - ref[rows]).max() / np.abs(ref[rows]).max())
        assert err <= 2e-5, (k, err)

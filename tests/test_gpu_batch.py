"""Batched solves of uneven systems (bse_solve_batch): every system's excitation energies
equal those of its own solve (each context on its own stream; split-K atomics may reorder
sums, so 1e-9 Ha) and, for one system, the CPU oracle's Davidson (1e-7 Ha)."""
import numpy as np
import pytest

from synth import make_localized
from oracle import liouville, davidson

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


def _systems():
    spec = [(32, 12, 11), (48, 16, 12), (32, 20, 13), (48, 13, 14), (32, 16, 15), (48, 24, 16)]
    return [make_localized(s, 20.0 * N / 72, N, n, 2.5, 2 * n, n_eig=4, block=4) for N, n, s in spec]


def test_batch_matches_individual_solves_and_oracle():
    from paper_2409_15116_gb300 import Context, binding
    systems = _systems()
    streams = [torch.cuda.Stream() for _ in systems]
    ctxs = [Context(inst, 0, stream=st.cuda_stream) for inst, st in zip(systems, streams)]
    om, stats, rc = binding.solve_batch(ctxs, 4, 8, 32, res_tol=1e-6)
    assert all(r == 0 for r in rc), rc
    for c in ctxs:
        c.close()
    for i, inst in enumerate(systems):
        c = Context(inst, 0)
        c.build_tau()
        ref, _ = c.davidson(4, 8, 32, res_tol=1e-6)
        c.close()
        assert np.abs(om[i] - ref).max() <= 1e-9, (i, om[i] - ref)
    inst = systems[0]
    Lop = liouville.Liouville(inst)
    want, _, info = davidson.davidson(Lop.apply, Lop.diagonal(), Lop.project, 4, 8, 32, 1e-7)
    assert np.abs(om[0] - want).max() <= 1e-7


def test_mixed_batch_against_the_oracle_davidson():
    """The mixed-precision batch (FP32 operator, BF16x3 projections): every system's lowest
    excitations within 1 meV of the oracle's FP64 Davidson on the matrix-free operator."""
    from paper_2409_15116_gb300 import Context, binding
    MEV = 3.6749322e-5
    systems = _systems()[:4]
    streams = [torch.cuda.Stream() for _ in systems]
    ctxs = [Context(inst, 1, stream=st.cuda_stream) for inst, st in zip(systems, streams)]
    om, stats, rc = binding.solve_batch(ctxs, 4, 8, 32, res_tol=1e-4)
    assert all(r == 0 for r in rc), rc
    for c in ctxs:
        c.close()
    for i, inst in enumerate(systems):
        Lop = liouville.Liouville(inst)
        want, _, info = davidson.davidson(Lop.apply, Lop.diagonal(), Lop.project, 4, 8, 32, 1e-7)
        assert info["converged"]
        assert np.abs(om[i] - want).max() <= MEV, (i, om[i] - want)

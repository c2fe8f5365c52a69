"""Explicit quasi-particle energies (Eq. ham) on the GPU against the dense e-h oracle: the
operator (FP64 1e-11, mixed 2e-5 relative, both entry points) and the lowest excitations
(FP64 1e-7 Ha, mixed 1 meV)."""
import numpy as np
import pytest

from synth import make_tiny
from oracle import dense_eh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
MEV = 3.6749322e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


@pytest.fixture(scope="module")
def qp_case():
    inst = make_tiny(0, n_qp=12)
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    return inst, H, parts


@pytest.mark.parametrize("prec,tol,etol", [(0, 1e-11, 1e-7), (1, 2e-5, MEV)])
def test_qp_operator_and_excitations_vs_dense(qp_case, prec, tol, etol):
    from paper_2409_15116_gb300 import Context
    inst, H, parts = qp_case
    c = Context(inst, prec)
    c.build_tau()
    y = np.random.default_rng(4).standard_normal((5, H.shape[0]))
    A = dense_eh.eh_to_packed(y, parts["Xc"], inst.n_occ)
    want = dense_eh.eh_to_packed(y @ H.T, parts["Xc"], inst.n_occ)
    a = torch.tensor(A, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    for entry in (c.apply, c.apply_static):
        out = torch.empty_like(a)
        entry(a, out)
        err = np.abs(out.double().cpu().numpy() - want).max() / np.abs(want).max()
        assert err <= tol, (entry.__name__, err)
    ref = np.linalg.eigvalsh(H)[:4]
    om, _ = c.davidson(4, 8, 32, res_tol=1e-6 if prec == 0 else 1e-4)
    assert np.abs(om - ref).max() <= etol, (om, ref)
    c.close()

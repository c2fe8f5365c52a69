"""Spin-polarised systems (spin-conserving excitations) on the GPU against the dense
spin-polarised e-h oracle: pair lists (bit-exact, no pair across channels), the operator
(FP64 1e-11, mixed 2e-5 relative) and the lowest excitations (FP64 1e-7 Ha, mixed 1 meV)."""
import numpy as np
import pytest

from synth import make_tiny
from oracle import pairs, spin, dense_eh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
MEV = 3.6749322e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


@pytest.fixture(scope="module")
def pol():
    inst = make_tiny(0, spin_pol=(5, 4))
    H, blocks = spin.eh_hamiltonian_spin(inst)
    return inst, H, blocks


@pytest.mark.parametrize("prec,tol,etol", [(0, 1e-11, 1e-7), (1, 2e-5, MEV)])
def test_spin_polarised_operator_and_excitations(pol, prec, tol, etol):
    from paper_2409_15116_gb300 import Context
    inst, H, blocks = pol
    c = Context(inst, prec)
    c.build_tau()
    m, _ = pairs.pair_mask(inst)
    assert (c.pairs() == pairs.pair_list(m)).all()
    y = np.random.default_rng(8).standard_normal((3, H.shape[0]))
    A = spin.eh_to_packed_spin(y, blocks)
    want = spin.eh_to_packed_spin(y @ H.T, blocks)
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


def test_identical_channels_give_singlet_and_triplet_lowest():
    from paper_2409_15116_gb300 import Context
    inst = make_tiny(0, spin_pol=(4, 4))
    s = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(make_tiny(0)))
    t = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(make_tiny(0, spin=1)))
    ref = np.sort(np.concatenate([s, t]))[:6]
    c = Context(inst, 0)
    c.build_tau()
    om, _ = c.davidson(6, 8, 40, res_tol=1e-6)
    assert np.abs(om - ref).max() <= 1e-7, (om, ref)
    c.close()

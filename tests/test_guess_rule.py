"""The identity behind the host-side rejection of Davidson start candidates.

The library starts the Davidson solve from unit vectors e_{v,j} (orbital row v, packed
coordinate j) at the lowest diagonal entries, projected by P_c, orthogonalised against the
vectors already accepted and accepted when the remaining norm exceeds 0.1. It rejects a
candidate on the host, without device work, when 1 - sum_w psi_w(j)^2 is below 0.01: that
value is the squared norm of P_c e_{v,j} in every row v, and orthogonalisation can only
lower it. These tests check the identity and the monotonicity on the oracle's projector
(Section 2, P_c = 1 - sum_w |psi_w><psi_w|), for the plain tiny cell and for localised
orbitals.
"""
import numpy as np
import pytest

from synth import make_tiny, make_localized
from oracle import liouville


@pytest.fixture(scope="module", params=["tiny", "localized"])
def case(request):
    if request.param == "tiny":
        inst = make_tiny(0)
    else:
        inst = make_localized(3, 20.0 * 32 / 72, 32, 12, 2.5, 24, n_eig=4, block=4)
    return inst, liouville.Liouville(inst)


def unit(inst, v, j):
    x = np.zeros((1, inst.n_occ, inst.psi.shape[1]))
    x[0, v, j] = 1.0
    return x


def test_projected_norm_is_one_minus_occupied_weight(case):
    inst, Lop = case
    n_pw = inst.psi.shape[1]
    occw = (inst.psi ** 2).sum(axis=0)
    rng = np.random.default_rng(5)
    js = [0] + list(rng.choice(np.arange(2, n_pw), size=24, replace=False))
    for j in js:
        for v in (0, inst.n_occ - 1):
            y = Lop.project(unit(inst, v, j))
            assert abs((y ** 2).sum() - (1.0 - occw[j])) < 1e-12, (v, j)
            # the projection stays in row v
            others = np.delete(y[0], v, axis=0)
            assert np.abs(others).max() == 0.0


def test_pad_coordinate_projects_to_zero(case):
    inst, Lop = case
    assert np.abs(Lop.project(unit(inst, 0, 1))).max() == 0.0


def test_orthogonalisation_only_lowers_the_norm(case):
    inst, Lop = case
    n_pw = inst.psi.shape[1]
    occw = (inst.psi ** 2).sum(axis=0)
    # accepted vectors: projected unit vectors of row 0 at the ten lowest-weight coordinates
    order = [j for j in np.argsort(occw) if j != 1][:10]
    V = []
    for j in order:
        x = Lop.project(unit(inst, 0, j)).ravel()
        for q in V:
            x -= (q @ x) * q
        V.append(x / np.linalg.norm(x))
    V = np.array(V)
    for j in [j for j in range(n_pw) if j != 1][:40]:
        y = Lop.project(unit(inst, 0, j)).ravel()
        z = y - V.T @ (V @ y)
        assert (z ** 2).sum() <= (1.0 - occw[j]) + 1e-12

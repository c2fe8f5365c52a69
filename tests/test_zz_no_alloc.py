"""bse_apply_liouville_static: the operator with its workspaces in the library's fixed
device array, for callers that cannot allocate device memory at call time (externally
pooled memory with a fixed budget, latency paths where an allocation may synchronise the
device).

Checked through the C ABI against bse_apply_liouville on two calls in a row (the second
call finds the previous call's data in the shared array), at the tolerances of the other
parity tests: FP64 relative 1e-11, mixed relative 2e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


def _inputs(inst, n_vec, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n_vec, inst.n_occ, inst.n_pw))
    A -= (A @ inst.psi.T) @ inst.psi
    A[..., 1] = 0.0
    return A


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_static_scratch_matches_allocating_entry_point(prec, tol):
    from paper_2409_15116_gb300 import Context
    from synth import make_tiny, make_localized
    dt = torch.float64 if prec == 0 else torch.float32
    for inst, n_vec in ((make_tiny(0), 7), (make_localized(3, 20.0 * 32 / 72, 32, 12, 2.5, 24), 3)):
        c = Context(inst, prec)
        c.build_tau()
        for call, seed in enumerate((1, 2)):          # two calls in a row
            a = torch.tensor(_inputs(inst, n_vec, seed), dtype=dt, device="cuda")
            want = torch.empty_like(a)
            got = torch.full_like(a, float("nan"))
            c.apply(a, want)
            c.apply_static(a, got)
            w = want.double().cpu().numpy()
            g = got.double().cpu().numpy()
            err = np.abs(g - w).max() / np.abs(w).max()
            assert np.isfinite(g).all() and err <= tol, (call, err)
        c.close()


def test_static_scratch_rejects_oversized_requests():
    from paper_2409_15116_gb300 import Context, BseError
    from synth import make_localized
    inst = make_localized(3, 20.0 * 32 / 72, 32, 12, 2.5, 24)
    c = Context(inst, 0)
    c.build_tau()
    a = torch.zeros((64, inst.n_occ, inst.n_pw), dtype=torch.float64, device="cuda")
    with pytest.raises(BseError) as e:
        c.apply_static(a, torch.empty_like(a))
    assert e.value.code == -1 and "static array holds" in str(e.value)
    c.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_static_scratch_first_call_then_smaller_odd_call(prec, tol):
    """A fresh context whose first operator call is the static one (untuned K1d tile), then a
    larger block followed by a smaller one with an odd number of orbital fields, so that the
    odd tail grid and the Hartree grids are written over the larger call's data."""
    from paper_2409_15116_gb300 import Context
    from synth import make_localized
    dt = torch.float64 if prec == 0 else torch.float32
    inst = make_localized(4, 20.0 * 32 / 72, 32, 13, 2.5, 26)
    c = Context(inst, prec)
    c.build_tau()
    results = []
    for n_vec, seed in ((4, 5), (3, 6)):               # 52 fields, then 39 (odd)
        a = torch.tensor(_inputs(inst, n_vec, seed), dtype=dt, device="cuda")
        got = torch.full_like(a, float("nan"))
        c.apply_static(a, got)
        results.append((a, got))
    for a, got in results:
        want = torch.empty_like(a)
        c.apply(a, want)
        w = want.double().cpu().numpy()
        g = got.double().cpu().numpy()
        err = np.abs(g - w).max() / np.abs(w).max()
        assert np.isfinite(g).all() and err <= tol, err
    c.close()

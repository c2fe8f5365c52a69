"""Failure paths of the library on the GPU, provoked without faulting the device.

* A tensor-core pipeline wait that runs out: with BSE_TC_WAIT_LIMIT=0 every bounded wait of
  the BF16x3 GEMM gives up at once; the kernel raises its error flag, drains the copies it
  issued, frees its tensor memory and returns. The call reports BSE_ERR_TIMEOUT, and a new
  context on the same device still computes the right operator.
* A Davidson solve stopped by max_it: BSE_ERR_NOT_CONVERGED, with the last Ritz values
  returned; by the Rayleigh-Ritz bound they lie at or above the exact eigenvalues.
"""
import numpy as np
import pytest

from synth import make_tiny
from oracle import dense_eh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


def test_tensor_core_wait_gives_up_with_timeout_status(monkeypatch):
    from paper_2409_15116_gb300 import Context, BseError, PREC_MIXED
    inst = make_tiny(0)
    monkeypatch.setenv("BSE_TC_WAIT_LIMIT", "0")
    c = Context(inst, PREC_MIXED)
    monkeypatch.delenv("BSE_TC_WAIT_LIMIT")
    with pytest.raises(BseError) as e:
        c.build_tau()             # the PDEP projection runs on the BF16x3 GEMM
    assert e.value.code == -6 and "gave up" in str(e.value)
    c.close()
    # the device is still usable: a fresh context reproduces the dense operator
    H, parts = dense_eh.eh_hamiltonian(inst, with_parts=True)
    c = Context(inst, PREC_MIXED)
    c.build_tau()
    y = np.random.default_rng(3).standard_normal((2, H.shape[0]))
    A = dense_eh.eh_to_packed(y, parts["Xc"], inst.n_occ)
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    c.apply(a, out)
    want = dense_eh.eh_to_packed(y @ H.T, parts["Xc"], inst.n_occ)
    err = np.abs(out.double().cpu().numpy() - want).max() / np.abs(want).max()
    assert err < 2e-5, err
    c.close()


def test_davidson_max_it_returns_partial_ritz_values():
    from paper_2409_15116_gb300 import Context, BseError, PREC_FP64
    inst = make_tiny(0)
    ref = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(inst))[:4]
    c = Context(inst, PREC_FP64)
    c.build_tau()
    with pytest.raises(BseError) as e:
        c.davidson(4, 4, 32, max_it=2, res_tol=1e-9)
    assert e.value.code == -5
    om, st = c.davidson(4, 4, 32, max_it=2, res_tol=1e-9, allow_not_converged=True)
    assert st.iterations == 2 and np.isfinite(om).all() and st.res_max > 1e-9
    assert (om >= ref - 1e-10).all(), (om, ref)
    c.close()

"""bse_create's caller-supplied allocator: every device buffer of a context comes from the
callbacks (here PyTorch's caching allocator through the binding) and goes back to them.

After a warm-up context (so the library's kernel modules are resident), a second context is
created, builds tau and applies the operator: the device memory the process took meanwhile
equals the growth of PyTorch's reserved pool within 64 MB (rounding of the pool's segments),
the callbacks handed out at least the tau array, and after bse_destroy every block handed out
has been returned."""
import numpy as np
import pytest

from synth import make_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_15116_gb300 import build as B
    B.build()


def _exercise(inst, c):
    c.build_tau()
    rng = np.random.default_rng(0)
    A = rng.standard_normal((4, inst.n_occ, inst.n_pw))
    A -= (A @ inst.psi.T) @ inst.psi
    A[..., 1] = 0.0
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    c.apply(a, out)
    torch.cuda.synchronize()


def test_context_memory_comes_from_the_callbacks():
    from paper_2409_15116_gb300 import Context
    inst = make_config("small")
    w = Context(inst, 1)
    _exercise(inst, w)
    w.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    c = Context(inst, 1)
    _exercise(inst, c)
    free1, _ = torch.cuda.mem_get_info()
    res1 = torch.cuda.memory_reserved()
    live = sum(c.allocator.live.values())
    n3 = inst.n_grid ** 3
    assert c.allocator.calls > 0 and live >= c.n_pairs * n3 * 4
    took, grew = free0 - free1, res1 - res0
    assert abs(took - grew) <= 64 << 20, (took, grew)
    c.close()
    assert not c.allocator.live

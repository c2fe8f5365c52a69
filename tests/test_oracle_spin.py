"""Pins of the spin-polarised oracle (oracle/spin.py and the channel-aware matrix-free route)."""
import numpy as np

from synth import make_tiny
from oracle import dense_eh, liouville, pairs, spin


def test_identical_channels_give_singlet_and_triplet_spectra():
    """Two identical spin channels: the spin-polarised spectrum is the union of the closed-shell
    singlet (K1e factor 2) and triplet (factor 0) spectra."""
    pol = make_tiny(0, spin_pol=(4, 4))
    H, _ = spin.eh_hamiltonian_spin(pol)
    got = np.linalg.eigvalsh(H)
    s = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(make_tiny(0)))
    t = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(make_tiny(0, spin=1)))
    np.testing.assert_allclose(got, np.sort(np.concatenate([s, t])), atol=1e-10)


def test_pair_rule_keeps_no_cross_channel_pair():
    pol = make_tiny(0, spin_pol=(5, 4))
    m, _ = pairs.pair_mask(pol)
    ch = pairs.channels(pol)
    assert not (m & (ch[:, None] != ch[None, :])).any()
    # within a channel the rule is the closed-shell one
    up = make_tiny(0, n_occ=5)
    m_up, _ = pairs.pair_mask(up)
    assert (m[:5, :5] == m_up).all()


def test_matrix_free_spin_operator_equals_dense_columnwise():
    pol = make_tiny(0, spin_pol=(5, 4))
    H, blocks = spin.eh_hamiltonian_spin(pol)
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    Lop = liouville.Liouville(pol)
    y = np.random.default_rng(3).standard_normal((3, H.shape[0]))
    A = spin.eh_to_packed_spin(y, blocks)
    got = Lop.apply(A)
    want = spin.eh_to_packed_spin(y @ H.T, blocks)
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()

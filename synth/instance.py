"""Seeded synthetic instances of the Gamma-point DMPT/TDA BSE problem.

Conventions (shared by every consumer, fixed here as a data format):

* cubic cell of edge ``L`` (bohr), FFT grid ``N^3``, real-space index
  ``r = x + N*(y + N*z)`` (x fastest), point ``L*(x, y, z)/N``;
* plane-wave sphere ``S = {G = 2*pi*n/L : |n|^2 <= n2max}`` with
  ``max|n_i| <= (N-1)//4`` so that every product the operator forms is alias-free;
* ``miller[0] = (0,0,0)``; rows ``k >= 1`` list one representative of each
  ``{+G_k, -G_k}`` pair (the "Gamma half-sphere");
* Gamma-packed real vectors of length ``n_pw = 2*n_half``: ``p[0] = c(0)``,
  ``p[1] = 0`` (alignment pad, structurally zero), and for ``k >= 1``
  ``p[2k] = sqrt(2) Re c(G_k)``, ``p[2k+1] = sqrt(2) Im c(G_k)``, where
  ``psi(r) = Omega^{-1/2} sum_{G in S} c(G) exp(iG.r)`` with ``c(-G) = c(G)^*``.
  This map is an isometry: packed dot products equal the L2 inner products.

The occupied orbitals of the tiny configuration come from a dense plane-wave
diagonalisation of a model Kohn-Sham Hamiltonian (the paper takes them from a
DFT ground state, Section 4, Fig. 1); the other configurations use localised
orbitals (Gaussian envelope times random long-wavelength plane-wave content,
projected on S and Loewdin-orthonormalised in FP64), standing in for the Wannier
orbitals of Eq. (wannier). The PDEP basis is a set of random orthonormal
Gamma-real vectors with prescribed eigenvalues (Eq. pdep); no dielectric
response is computed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = ["Instance", "sphere_half", "make_tiny", "make_localized",
           "make_config", "CONFIGS", "wells_on_grid"]


@dataclass
class Instance:
    name: str
    L: float
    n_grid: int
    n2max: int
    miller: np.ndarray       # [n_half, 3] int32
    psi: np.ndarray          # [n_occ, n_pw] float64, Gamma-packed, orthonormal
    eps: np.ndarray          # [n_occ] float64 (Ha)
    v_loc: np.ndarray        # [N^3] float64 (Ha), x fastest
    scissor: float           # Ha
    pdep: np.ndarray         # [n_pdep, n_pw] float64, columns 0 and 1 zero
    lam: np.ndarray          # [n_pdep] float64, each in (-1, 0)
    overlap_thr: float       # > 0: keep pairs with O >= thr
    keep_pairs: int          # > 0 (and thr <= 0): keep this many v <= w pairs
    spin: int = 0            # 0 singlet (K1e factor 2), 1 triplet (factor 0)
    seed: int = 0
    n_eig: int = 4
    block: int = 8
    # explicit quasi-particle energies (Eq. ham): 0 = scissor only; else N_QP > n_occ with
    # the conduction KS states n_occ..N_QP-1 (packed), KS and QP energies of states 0..N_QP-1
    qp_n: int = 0
    qp_psi: np.ndarray | None = None
    qp_eps_ks: np.ndarray | None = None
    qp_eps: np.ndarray | None = None
    # spin-polarised (spin-conserving) systems: orbitals 0..n_up-1 are spin up, the rest spin
    # down; 0 = closed shell (the `spin` field then selects singlet or triplet)
    n_up: int = 0
    # occupied energies as a matrix in a rotated (e.g. Wannier) frame, U^T diag(eps) U; None:
    # the orbitals are canonical and eps is diagonal
    eps_mat: np.ndarray | None = None

    @property
    def n_occ(self) -> int:
        return int(self.psi.shape[0])

    @property
    def n_pw(self) -> int:
        return int(self.psi.shape[1])

    @property
    def n_half(self) -> int:
        return int(self.miller.shape[0])

    @property
    def n_pdep(self) -> int:
        return int(self.pdep.shape[0])

    @property
    def omega(self) -> float:
        return float(self.L) ** 3

    def save(self, path: str) -> None:
        qp = {}
        if self.qp_n:
            qp = dict(qp_n=self.qp_n, qp_psi=self.qp_psi, qp_eps_ks=self.qp_eps_ks, qp_eps=self.qp_eps)
        np.savez(path, name=self.name, L=self.L, n_grid=self.n_grid, n2max=self.n2max,
                 miller=self.miller, psi=self.psi, eps=self.eps, v_loc=self.v_loc,
                 scissor=self.scissor, pdep=self.pdep, lam=self.lam,
                 overlap_thr=self.overlap_thr, keep_pairs=self.keep_pairs,
                 spin=self.spin, seed=self.seed, n_eig=self.n_eig, block=self.block,
                 n_up=self.n_up, **qp)

    @staticmethod
    def load(path: str) -> "Instance":
        d = np.load(path)
        qp = {}
        if "qp_n" in d:
            qp = dict(qp_n=int(d["qp_n"]), qp_psi=d["qp_psi"], qp_eps_ks=d["qp_eps_ks"], qp_eps=d["qp_eps"])
        return Instance(name=str(d["name"]), L=float(d["L"]), n_grid=int(d["n_grid"]),
                        n2max=int(d["n2max"]), miller=d["miller"], psi=d["psi"],
                        eps=d["eps"], v_loc=d["v_loc"], scissor=float(d["scissor"]),
                        pdep=d["pdep"], lam=d["lam"], overlap_thr=float(d["overlap_thr"]),
                        keep_pairs=int(d["keep_pairs"]), spin=int(d["spin"]),
                        seed=int(d["seed"]), n_eig=int(d["n_eig"]), block=int(d["block"]),
                        n_up=int(d["n_up"]) if "n_up" in d else 0, **qp)


# ----------------------------------------------------------------------------------
# plane-wave sphere
# ----------------------------------------------------------------------------------

def sphere_half(n2max: int) -> np.ndarray:
    """Miller indices of the Gamma half-sphere, G=0 first, then by (|n|^2, n_z, n_y, n_x).

    A vector is kept when its first nonzero component, scanning z, y, x, is positive.
    """
    r = int(math.isqrt(n2max))
    rng = np.arange(-r, r + 1)
    nz, ny, nx = np.meshgrid(rng, rng, rng, indexing="ij")
    n = np.stack([nx.ravel(), ny.ravel(), nz.ravel()], axis=1)
    n2 = (n ** 2).sum(1)
    keep = n2 <= n2max
    pos = (n[:, 2] > 0) | ((n[:, 2] == 0) & (n[:, 1] > 0)) | \
          ((n[:, 2] == 0) & (n[:, 1] == 0) & (n[:, 0] > 0))
    zero = n2 == 0
    sel = n[keep & (pos | zero)]
    n2s = (sel ** 2).sum(1)
    order = np.lexsort((sel[:, 0], sel[:, 1], sel[:, 2], n2s))
    out = sel[order].astype(np.int32)
    assert (out[0] == 0).all()
    return out


def _packing_matrix(n_half: int) -> np.ndarray:
    """Complex map from unpadded packed coordinates to full-sphere coefficients.

    Full-sphere order: [G_0, +G_1, -G_1, +G_2, -G_2, ...]; unpadded packed order:
    [c(0), sqrt2 Re c(G_1), sqrt2 Im c(G_1), ...]. Pure data formatting.
    """
    n = 2 * n_half - 1
    M = np.zeros((n, n), dtype=np.complex128)
    M[0, 0] = 1.0
    s = 1.0 / math.sqrt(2.0)
    for k in range(1, n_half):
        M[2 * k - 1, 2 * k - 1] = s
        M[2 * k - 1, 2 * k] = 1j * s
        M[2 * k, 2 * k - 1] = s
        M[2 * k, 2 * k] = -1j * s
    return M


def _insert_pad(p: np.ndarray) -> np.ndarray:
    """[..., 2*n_half-1] unpadded packed -> [..., 2*n_half] with the zero pad at column 1."""
    out = np.zeros(p.shape[:-1] + (p.shape[-1] + 1,), dtype=p.dtype)
    out[..., 0] = p[..., 0]
    out[..., 2:] = p[..., 1:]
    return out


def _half_coeffs_to_packed(c: np.ndarray) -> np.ndarray:
    """Half-sphere complex coefficients [..., n_half] (c[...,0] real) -> padded packed."""
    out = np.zeros(c.shape[:-1] + (2 * c.shape[-1],), dtype=np.float64)
    out[..., 0] = c[..., 0].real
    out[..., 2::2] = math.sqrt(2.0) * c[..., 1:].real
    out[..., 3::2] = math.sqrt(2.0) * c[..., 1:].imag
    return out


# ----------------------------------------------------------------------------------
# model local potential: periodic Gaussian wells
# ----------------------------------------------------------------------------------

def wells_on_grid(L: float, N: int, centres: np.ndarray, depth: float = 2.0,
                  width: float = 1.0) -> np.ndarray:
    """V(r) = -depth * sum_i sum_{m in {-1,0,1}^3} exp(-|r - R_i - L m|^2 / (2 width^2)).

    Sampled on the N^3 grid, x fastest. The image sum factorises per axis.
    """
    x = np.arange(N) * (L / N)
    V = np.zeros((N, N, N))
    for R in np.asarray(centres, dtype=np.float64):
        f = []
        for a in range(3):
            d = x[None, :] - R[a] - L * np.array([-1.0, 0.0, 1.0])[:, None]
            f.append(np.exp(-d ** 2 / (2 * width ** 2)).sum(0))
        V -= depth * f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    return V.reshape(-1)


def _periodic_dist(a: np.ndarray, b: np.ndarray, L: float) -> float:
    d = a - b
    d -= L * np.round(d / L)
    return float(np.sqrt((d ** 2).sum()))


def _draw_centres(rng, n: int, L: float, min_sep: float) -> np.ndarray:
    out = []
    while len(out) < n:
        c = rng.uniform(0.0, L, 3)
        if all(_periodic_dist(c, o, L) >= min_sep for o in out):
            out.append(c)
    return np.array(out)


# ----------------------------------------------------------------------------------
# configuration 1: tiny cell, orbitals from a dense plane-wave diagonalisation
# ----------------------------------------------------------------------------------

def _ground_state_tiny(L, miller, centres, depth, width, n_occ):
    """Lowest n_occ eigenpairs of the model KS Hamiltonian in the sphere.

    Stand-in for the DFT ground state that feeds the BSE (Fig. 1). Uses the analytic
    Fourier coefficients of the periodic Gaussian wells,
    V(q) = -(depth/Omega) (2 pi w^2)^{3/2} exp(-w^2 q^2/2) sum_i exp(-i q.R_i).
    """
    n_half = miller.shape[0]
    full = np.zeros((2 * n_half - 1, 3))
    full[1::2] = miller[1:]
    full[2::2] = -miller[1:]
    G = full * (2 * np.pi / L)
    omega = L ** 3
    q = G[:, None, :] - G[None, :, :]
    q2 = (q ** 2).sum(-1)
    phase = np.zeros(q2.shape, dtype=np.complex128)
    for R in centres:
        phase += np.exp(-1j * (q @ R))
    Vq = -(depth / omega) * (2 * np.pi * width ** 2) ** 1.5 * np.exp(-width ** 2 * q2 / 2) * phase
    H = Vq + np.diag(0.5 * (G ** 2).sum(1))
    M = _packing_matrix(n_half)
    Hp = M.conj().T @ H @ M
    assert np.abs(Hp.imag).max() < 1e-12 * np.abs(Hp).max()
    Hp = 0.5 * (Hp.real + Hp.real.T)
    e, C = np.linalg.eigh(Hp)
    psi = _insert_pad(C[:, :n_occ].T.copy())
    return psi, e[:n_occ].copy()


def _ks_states_tiny(L, miller, centres, depth, width, n_states):
    """Lowest n_states eigenpairs (occupied and conduction) of the same model KS Hamiltonian."""
    return _ground_state_tiny(L, miller, centres, depth, width, n_states)


def _random_orthonormal_packed(rng, n_vec: int, n_pw: int) -> np.ndarray:
    """n_vec orthonormal Gamma-real vectors on S \\ {0} (columns 0 and 1 zero), FP64 QR."""
    X = rng.standard_normal((n_pw - 2, n_vec))
    Q, _ = np.linalg.qr(X)
    out = np.zeros((n_vec, n_pw))
    out[:, 2:] = Q.T
    return out


def make_tiny(seed: int = 0, L: float = 8.0, N: int = 16, n2max: int = 14, n_occ: int = 4,
              n_wells: int = 4, depth: float = 2.0, width: float = 1.0,
              scissor: float = 0.03, overlap_thr: float = 1e-3, spin: int = 0,
              n_eig: int = 4, block: int = 8, n_qp: int = 0, spin_pol=None) -> Instance:
    """Plain FP64 tiny cell: L=8 bohr, 16^3 grid, 251 plane waves, 4 wells, full PDEP basis.

    n_qp > n_occ adds explicit quasi-particle data for the lowest n_qp states (Eq. ham): their
    KS states and energies from the same diagonalisation, and QP energies drawn as seeded
    shifts of the KS ones (occupied -0.06..-0.04 Ha, conduction +0.05..+0.10 Ha), standing in
    for G0W0 corrections (Fig. 1).

    spin_pol = (n_up, n_dn) makes a spin-polarised system: the n_up lowest KS states occupied in
    the up channel and the n_dn lowest in the down channel (one spin-independent model
    Hamiltonian, as for a high-spin open shell).
    """
    rng = np.random.default_rng(seed)
    centres = _draw_centres(rng, n_wells, L, 2.0)
    miller = sphere_half(n2max)
    v_loc = wells_on_grid(L, N, centres, depth, width)
    psi, eps = _ground_state_tiny(L, miller, centres, depth, width, n_occ)
    n_pw = psi.shape[1]
    pdep = _random_orthonormal_packed(rng, n_pw - 2, n_pw)
    lam = rng.uniform(-0.9, -0.01, n_pw - 2)
    n_up = 0
    if spin_pol is not None:
        n_up, n_dn = int(spin_pol[0]), int(spin_pol[1])
        st, e_ks = _ks_states_tiny(L, miller, centres, depth, width, max(n_up, n_dn))
        psi = np.concatenate([st[:n_up], st[:n_dn]])
        eps = np.concatenate([e_ks[:n_up], e_ks[:n_dn]])
    qp = {}
    if n_qp:
        if n_qp <= n_occ:
            raise ValueError("n_qp must exceed n_occ")
        states, e_ks = _ks_states_tiny(L, miller, centres, depth, width, n_qp)
        r2 = np.random.default_rng(10_000 + seed)
        shift = np.concatenate([r2.uniform(-0.06, -0.04, n_occ), r2.uniform(0.05, 0.10, n_qp - n_occ)])
        qp = dict(qp_n=n_qp, qp_psi=states[n_occ:].copy(), qp_eps_ks=e_ks, qp_eps=e_ks + shift)
    return Instance(name=f"tiny-L{L:g}-N{N}-s{seed}", L=L, n_grid=N, n2max=n2max,
                    miller=miller, psi=psi, eps=eps, v_loc=v_loc, scissor=scissor,
                    pdep=pdep, lam=lam, overlap_thr=overlap_thr, keep_pairs=0,
                    spin=spin, seed=seed, n_eig=n_eig, block=block, n_up=n_up, **qp)


# ----------------------------------------------------------------------------------
# configurations 2, 3, 5: localised synthetic orbitals
# ----------------------------------------------------------------------------------

def _site_positions(rng, n_sites: int, L: float) -> np.ndarray:
    c = 1
    while c ** 3 < n_sites:
        c += 1
    idx = np.stack(np.meshgrid(np.arange(c), np.arange(c), np.arange(c), indexing="ij"),
                   -1).reshape(-1, 3)
    pick = np.sort(rng.choice(idx.shape[0], n_sites, replace=False))
    a = L / c
    return (idx[pick] + 0.5) * a + rng.uniform(-0.25, 0.25, (n_sites, 3)) * a


def make_localized(seed: int, L: float, N: int, n_occ: int, width: float, n_pdep: int,
                   keep_frac: float = 0.15, depth: float = 2.0, well_width: float = 1.0,
                   lam_mode: str = "exp", n_eig: int = 16, block: int = 32,
                   spin: int = 0, name: str | None = None) -> Instance:
    """Localised orbitals: envelope exp(-|r-R_v|^2/(2 w^2)) times Re sum_{|n|^2<=4} z e^{i2pi n.r/L}.

    Four orbitals share a site; sites sit on a jittered simple-cubic lattice. The
    orbitals are built analytically in G (periodic envelope), truncated to S and
    Loewdin-orthonormalised in FP64. One Gaussian well per site forms V_loc; the
    scissor is 0.03 + max(0, max eps - min V) so that the diagonal term is >= 0.03 Ha.
    """
    rng = np.random.default_rng(seed)
    r_max = (N - 1) // 4
    n2max = r_max * r_max
    miller = sphere_half(n2max)
    n_half = miller.shape[0]
    G = miller.astype(np.float64) * (2 * np.pi / L)
    n_sites = (n_occ + 3) // 4
    sites = _site_positions(rng, n_sites, L)
    R = sites[np.arange(n_occ) // 4]
    qn = sphere_half(4)
    qfull = np.concatenate([qn, -qn[1:]]).astype(np.float64) * (2 * np.pi / L)  # 33 vectors
    z = (rng.standard_normal((n_occ, qfull.shape[0])) +
         1j * rng.standard_normal((n_occ, qfull.shape[0])))
    # c_v(G) = e^{-iG.R_v} * 0.5 * sum_q [z e^{iq.R} g(G-q) + z* e^{-iq.R} g(G+q)]
    gm = np.exp(-0.5 * width ** 2 * ((G[None, :, :] - qfull[:, None, :]) ** 2).sum(-1))
    gp = np.exp(-0.5 * width ** 2 * ((G[None, :, :] + qfull[:, None, :]) ** 2).sum(-1))
    eqr = np.exp(1j * (R @ qfull.T))
    Z = np.concatenate([z * eqr, np.conj(z) / eqr], axis=1) * 0.5
    coef = (Z @ np.concatenate([gm, gp], axis=0)) * np.exp(-1j * (R @ G.T))
    P = _half_coeffs_to_packed(coef)
    S = P @ P.T
    e, V = np.linalg.eigh(S)
    P = (V * (1.0 / np.sqrt(e))) @ V.T @ P
    eps = rng.uniform(-0.6, 0.0, n_occ)
    v_loc = wells_on_grid(L, N, sites, depth, well_width)
    scissor = 0.03 + max(0.0, float(eps.max() - v_loc.min()))
    n_pw = 2 * n_half
    pdep = _random_orthonormal_packed(rng, n_pdep, n_pw)
    if lam_mode == "exp":
        lam = -0.8 * np.exp(-np.arange(n_pdep) / 100.0)
    else:
        lam = rng.uniform(-0.9, -0.01, n_pdep)
    keep = int(round(keep_frac * n_occ * (n_occ + 1) / 2))
    return Instance(name=name or f"loc-L{L:g}-N{N}-occ{n_occ}-s{seed}", L=L, n_grid=N,
                    n2max=n2max, miller=miller, psi=P, eps=eps, v_loc=v_loc,
                    scissor=scissor, pdep=pdep, lam=lam, overlap_thr=0.0,
                    keep_pairs=keep, spin=spin, seed=seed, n_eig=n_eig, block=block)


def make_batched_member(seed: int) -> Instance:
    """One system of the 64-system batch: grid in {32,48,64}, N_occ in [32,192], N_pdep=2 N_occ."""
    rng = np.random.default_rng(10_000 + seed)
    N = int(rng.choice([32, 48, 64]))
    n_occ = int(rng.integers(32, 193))
    L = 20.0 * N / 72.0
    return make_localized(seed, L, N, n_occ, 2.5, 2 * n_occ, n_eig=8, block=8,
                          name=f"batch-N{N}-occ{n_occ}-s{seed}")


def make_config(name: str, seed: int | None = None) -> Instance:
    return CONFIGS[name](seed)


CONFIGS = {
    # plain FP64 tiny cell, checked against the dense electron-hole Hamiltonian
    "tiny": lambda s=None: make_tiny(0 if s is None else s),
    # mixed precision, medium: 72^3, 256 localised orbitals, 512 PDEP, 15% of pairs
    "medium": lambda s=None: make_localized(2 if s is None else s, 20.0, 72, 256, 2.5, 512,
                                            name="medium-L20-N72-occ256"),
    # small profiling case of the same family: 48^3, 64 orbitals, 128 PDEP (~1 GB of fields)
    "small": lambda s=None: make_localized(8 if s is None else s, 20.0 * 48 / 72, 48, 64, 2.5, 128,
                                           name="small-L13.3-N48-occ64"),
    # transform profiling case on the medium grid: 72^3, 32 orbitals, 64 PDEP (~1.5 GB of fields)
    "grid72": lambda s=None: make_localized(10 if s is None else s, 20.0, 72, 32, 2.5, 64,
                                            name="grid72-L20-N72-occ32"),
    # operator profiling case with the medium orbital count on a 32^3 grid (~3 GB of fields)
    "op256": lambda s=None: make_localized(9 if s is None else s, 20.0 * 32 / 72, 32, 256, 2.5, 512,
                                           name="op256-L8.9-N32-occ256"),
    # one member of the uneven batch (seeds 300..363)
    "batch": lambda s=None: make_batched_member(300 if s is None else s),
    # large: 96^3, 1024 orbitals, 1024 PDEP, ~20k pairs
    "large": lambda s=None: _make_large(5 if s is None else s),
}


def _make_large(seed: int) -> Instance:
    inst = make_localized(seed, 36.0, 96, 1024, 3.0, 1024, name="large-L36-N96-occ1024",
                          block=64)
    inst.keep_pairs = 20000
    return inst

"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CUDA path and by the CPU oracle, so it holds no
arithmetic of the screening method itself: only geometry (cells, k grids,
G-vector lists, q points), random draws (raw coefficient matrices, band
energies, Gaussian exponents) and the frequency grid.  Turning the raw random
coefficients into S(k)-orthonormal Bloch coefficients needs the overlap of the
Gaussian basis, which is method arithmetic; each side does that with its own
code.

Units are Hartree atomic units (bohr, Hartree) throughout; eV and angstrom
appear only in the workload descriptions below.

Workloads (Section III and Table I of the paper set the shapes: diamond
structure, 8x8x8 k grids, a few valence and tens of conduction bands, omega up
to 50-100 eV, G sets of 1e2-1e3):

* ``small``   2-atom diamond cell a=5.43 A, 8 sp shells/atom (exponents
  log-uniform 0.1-100 bohr^-2), 4x4x4 k, N_v=4, N_c=12, N_G=27, 10 q along
  [100] up to 2 reciprocal units (q_j = 0.19 j: q = 2 would be the reciprocal
  lattice vector (2,0,0), where |q+G| = 0 is the optical limit), 50 omega on
  0-50 eV, eta=0.1 eV.
* ``mid``     12 sp shells/atom, 8x8x8 k, N_v=4, N_c=32, N_G=181, 50 q on
  random directions with |q| <= 4 reciprocal units, 200 omega on 0-60 eV,
  eta=0.1 eV.
* ``uneven``  the small workload's states with 256 (q, omega) instances whose
  G sets are {G : |q+G| < G_max}, N_G between 15 and 339.
* ``large``   18 sp shells/atom (exponents up to 5000 bohr^-2), 12x12x12 k,
  N_v=14, N_c=64, N_G=531, 100 q with |q| <= 6, 400 omega on 0-100 eV,
  eta=0.05 eV.

One "sp shell" is one exponent carrying an s and a p_x, p_y, p_z primitive,
so N_b = 8 * shells per atom.  A "reciprocal unit" is 2*pi/a.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BOHR_ANG = 0.529177210903          # CODATA 2018
HARTREE_EV = 27.211386245988       # CODATA 2018


@dataclass
class Cell:
    lattice: np.ndarray            # [3][3] rows a1, a2, a3 (bohr)
    atoms: np.ndarray              # [natom][3] Cartesian (bohr)
    a: float                       # conventional cubic constant (bohr)

    @property
    def recip(self) -> np.ndarray:
        """Rows b_i with a_i . b_j = 2 pi delta_ij."""
        return 2.0 * np.pi * np.linalg.inv(self.lattice).T

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))


@dataclass
class Basis:
    shell_atom: np.ndarray         # [nshell] int32
    shell_l: np.ndarray            # [nshell] int32, 0 (s) or 1 (p)
    shell_exp: np.ndarray          # [nshell] float64, bohr^-2

    @property
    def nbasis(self) -> int:
        return int(np.sum(np.where(self.shell_l == 0, 1, 3)))


@dataclass
class Problem:
    """One workload: geometry, basis, k/q/G sets, raw random draws, grids."""
    name: str
    cell: Cell
    basis: Basis
    kpts: np.ndarray               # [nk][3] Cartesian bohr^-1
    qpts: np.ndarray               # [nq][3] Cartesian bohr^-1
    G_int: np.ndarray              # [ng][3] int32, coefficients on b1, b2, b3
    nv: int
    nc: int
    Zk: np.ndarray                 # [nk][nb][nv] complex, raw draws at k
    Ek: np.ndarray                 # [nk][nv] Hartree, sorted
    Ekq: np.ndarray                # [nq][nk][nc] Hartree, sorted
    w: np.ndarray                  # [nw] Hartree
    eta: float                     # Hartree
    seed: int = 0
    q_index: np.ndarray | None = None   # original index of each kept q
    extra: dict = field(default_factory=dict)

    def zkq(self, iq: int) -> np.ndarray:
        """[nk][nb][nc] complex raw draws at k+q for q number `iq`, drawn from
        a generator seeded by (seed, original q index) so that truncating the
        q list does not change them."""
        oq = int(self.q_index[iq]) if self.q_index is not None else iq
        rng = np.random.default_rng([self.seed, 1000 + oq])
        return random_coeffs(rng, (self.nk, self.basis.nbasis, self.nc))

    @property
    def nk(self) -> int:
        return self.kpts.shape[0]

    @property
    def nq(self) -> int:
        return self.qpts.shape[0]

    @property
    def ng(self) -> int:
        return self.G_int.shape[0]

    @property
    def nt(self) -> int:
        return self.nk * self.nv * self.nc


def diamond_cell(a_ang: float = 5.43) -> Cell:
    """FCC primitive vectors (a/2)(0,1,1), (a/2)(1,0,1), (a/2)(1,1,0); atoms at 0 and (a/4)(1,1,1)."""
    a = a_ang / BOHR_ANG
    lat = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    atoms = np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])
    return Cell(lat, atoms, a)


def sp_basis(rng: np.random.Generator, natom: int, shells_per_atom: int,
             lo: float, hi: float) -> Basis:
    """Per atom, `shells_per_atom` exponents drawn log-uniform on [lo, hi];
    each exponent gives one s shell and one p shell."""
    sa, sl, se = [], [], []
    for at in range(natom):
        ex = np.sort(np.exp(rng.uniform(np.log(lo), np.log(hi), shells_per_atom)))
        for e in ex:
            for l in (0, 1):
                sa.append(at)
                sl.append(l)
                se.append(e)
    return Basis(np.array(sa, np.int32), np.array(sl, np.int32), np.array(se, np.float64))


def kgrid(cell: Cell, n: int) -> np.ndarray:
    """Gamma-centred uniform grid k = sum_i (n_i / n) b_i, n_i = 0..n-1, Cartesian."""
    f = np.array([(i, j, k) for i in range(n) for j in range(n) for k in range(n)], np.float64) / n
    return f @ cell.recip


def g_sorted(cell: Cell, nmax: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """All integer triples in [-nmax, nmax]^3 sorted by |G|^2 then (n1, n2, n3).
    Returns (G_int, |G|^2)."""
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    g = n @ cell.recip
    g2 = np.round(np.einsum("ij,ij->i", g, g), 10)
    order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], g2))
    return n[order].astype(np.int32), g2[order]


def g_lowest_shells(cell: Cell, ng: int) -> np.ndarray:
    """The ng lowest-|G| vectors; ng must close a shell (G=0 is index 0)."""
    n, g2 = g_sorted(cell)
    if ng < len(g2) and abs(g2[ng] - g2[ng - 1]) < 1e-8:
        raise ValueError(f"N_G={ng} does not close a |G| shell")
    return n[:ng].copy()


def g_cutoff(cell: Cell, q: np.ndarray, gmax: float) -> np.ndarray:
    """{G : |q+G| < gmax}, sorted by |G|^2 then lexicographically."""
    n, _ = g_sorted(cell, nmax=12)
    g = n @ cell.recip + q
    keep = np.einsum("ij,ij->i", g, g) < gmax * gmax
    return n[keep].copy()


def random_coeffs(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex standard-normal draws."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def band_energies(rng: np.random.Generator, shape, lo_ev: float, hi_ev: float) -> np.ndarray:
    """Uniform draws on [lo, hi] eV, sorted along the last axis, in Hartree."""
    return np.sort(rng.uniform(lo_ev, hi_ev, shape), axis=-1) / HARTREE_EV


def omega_grid(wmax_ev: float, nw: int) -> np.ndarray:
    return np.linspace(0.0, wmax_ev, nw) / HARTREE_EV


def random_q(rng: np.random.Generator, cell: Cell, n: int, qmax_units: float,
             G_int: np.ndarray, min_units: float = 0.1) -> np.ndarray:
    """n q vectors on isotropic random directions with |q| ~ U(0, qmax] (units
    2 pi/a); a draw is repeated while min_G |q+G| < min_units (the optical
    limit q+G -> 0 is not part of this path)."""
    unit = 2.0 * np.pi / cell.a
    Gc = G_int @ cell.recip
    out = []
    while len(out) < n:
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        qv = d * rng.uniform(0.0, qmax_units) * unit
        if np.min(np.linalg.norm(qv[None, :] + Gc, axis=1)) >= min_units * unit:
            out.append(qv)
    return np.array(out)


def random_directions(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _states(rng, nk, nq, nb, nv, nc, ev_lo, ev_hi, ec_lo, ec_hi):
    """Raw draws at k (nv columns kept) and band energies; draws at k+q are lazy."""
    Zk = random_coeffs(rng, (nk, nb, nv))
    Ek = band_energies(rng, (nk, nv), ev_lo, ev_hi)
    Ekq = band_energies(rng, (nq, nk, nc), ec_lo, ec_hi)
    return Zk, Ek, Ekq


def make_small(nq: int | None = None, nw: int | None = None) -> Problem:
    """Small workload (seed 1235).  `nq`/`nw` truncate the q list / omega grid."""
    rng = np.random.default_rng(1235)
    cell = diamond_cell()
    basis = sp_basis(rng, 2, 8, 0.1, 100.0)
    kp = kgrid(cell, 4)
    unit = 2.0 * np.pi / cell.a
    q = np.array([[0.19 * j * unit, 0.0, 0.0] for j in range(1, 11)])
    Zk, Ek, Ekq = _states(rng, kp.shape[0], q.shape[0], basis.nbasis, 4, 12, -12.0, 0.0, 1.1, 30.0)
    p = Problem("small", cell, basis, kp, q, g_lowest_shells(cell, 27), 4, 12, Zk, Ek, Ekq,
                omega_grid(50.0, 50), 0.1 / HARTREE_EV, seed=1235)
    return truncate(p, nq, nw)


def make_mid(nq: int | None = None, nw: int | None = None) -> Problem:
    """Mid-size workload (seed 1236)."""
    rng = np.random.default_rng(1236)
    cell = diamond_cell()
    basis = sp_basis(rng, 2, 12, 0.1, 100.0)
    kp = kgrid(cell, 8)
    nq_full = 50
    G = g_lowest_shells(cell, 181)
    q = random_q(rng, cell, nq_full, 4.0, G)
    Zk, Ek, Ekq = _states(rng, kp.shape[0], nq_full, basis.nbasis, 4, 32, -12.0, 0.0, 1.1, 30.0)
    p = Problem("mid", cell, basis, kp, q, G, 4, 32, Zk, Ek, Ekq,
                omega_grid(60.0, 200), 0.1 / HARTREE_EV, seed=1236)
    return truncate(p, nq, nw)


def make_mid_shard(shard: int) -> Problem:
    """The mid workload with its own 50 q (and k+q states) for shard number
    `shard` (weak scaling across processes); k states and basis are shared."""
    p = make_mid()
    rng = np.random.default_rng([1236, 7, shard])
    p.qpts = random_q(rng, p.cell, 50, 4.0, p.G_int)
    p.Ekq = band_energies(rng, (50, p.nk, p.nc), 1.1, 30.0)
    p.q_index = np.arange(50) + 50 * (shard + 1)
    return p


def make_surrogate_set(nq: int = 110) -> Problem:
    """The learned-correction workload: the mid workload's cell, basis, k grid
    and bands with its own `nq` random q (|q| <= 4 reciprocal units) and k+q
    states; 200 w each (nq x 200 head samples)."""
    p = make_mid()
    rng = np.random.default_rng([1236, 11])
    p.name = "surrogate"
    p.qpts = random_q(rng, p.cell, nq, 4.0, p.G_int)
    p.Ekq = band_energies(rng, (nq, p.nk, p.nc), 1.1, 30.0)
    p.q_index = np.arange(nq) + 5000
    return p


def make_large(nq: int | None = None, nw: int | None = None, n_k: int = 12) -> Problem:
    """Large all-electron-style workload (seed 1239).  The raw draws at k+q
    are [nq][1728][144][144] complex; ask for a few q only.  `n_k` < 12 gives
    the same basis, G set and q list on a coarser n_k^3 k grid (other draws)."""
    rng = np.random.default_rng(1239)
    cell = diamond_cell()
    basis = sp_basis(rng, 2, 18, 0.1, 5000.0)
    kp = kgrid(cell, n_k)
    nq_full = 100
    G = g_lowest_shells(cell, 531)
    q = random_q(rng, cell, nq_full, 6.0, G)
    Zk, Ek, Ekq = _states(rng, kp.shape[0], nq_full, basis.nbasis, 14, 64, -12.0, 0.0, 1.1, 30.0)
    p = Problem("large", cell, basis, kp, q, G, 14, 64, Zk, Ek, Ekq,
                omega_grid(100.0, 400), 0.05 / HARTREE_EV, seed=1239)
    return truncate(p, nq, nw)


def make_uneven(n_inst: int = 256) -> Problem:
    """Uneven instances over the small workload's states (seed 1237 for the
    instance draws).  extra['inst_q'] indexes the q list, extra['inst_w'] is
    omega (Hartree), extra['inst_gmax'] the cutoff (bohr^-1); N_G per instance
    lies in [15, 339]."""
    base = make_small()
    rng = np.random.default_rng(1237)
    unit = 2.0 * np.pi / base.cell.a
    radii = np.sqrt(np.array([4.0, 8.0, 11.0, 12.0, 16.0, 19.0, 20.0, 24.0, 27.0, 32.0, 35.0, 36.0,
                              40.0, 43.0, 44.0, 48.0])) * unit
    iq, iw, gm, ngs = [], [], [], []
    while len(iq) < n_inst:
        qi = int(rng.integers(0, base.nq))
        g = float(rng.choice(radii))
        ng = g_cutoff(base.cell, base.qpts[qi], g).shape[0]
        if 15 <= ng <= 339:
            iq.append(qi)
            gm.append(g)
            ngs.append(ng)
            iw.append(float(rng.choice(base.w[1:])))
    base.name = "uneven"
    base.extra = {"inst_q": np.array(iq, np.int32), "inst_w": np.array(iw),
                  "inst_gmax": np.array(gm), "inst_ng": np.array(ngs, np.int32)}
    return base


def truncate(p: Problem, nq, nw) -> Problem:
    """Keep the first `nq` q points (or the listed indices) and `nw` omegas."""
    if p.q_index is None:
        p.q_index = np.arange(p.qpts.shape[0])
    if nq is not None:
        sel = np.arange(nq) if np.isscalar(nq) else np.asarray(nq)
        p.qpts = p.qpts[sel]
        p.Ekq = p.Ekq[sel]
        p.q_index = p.q_index[sel]
    if nw is not None:
        p.w = p.w[:nw]
    return p


def make_optical(base: str = "small", nw: int | None = None) -> Problem:
    """The optical limit q -> 0 on the cell, basis, k grid, valence draws, energies
    at k and G set of the small (or mid) workload: a single q = 0 whose conduction
    draws and energies are seeded apart from the finite-q ones.  Its conduction
    states live at k itself, so the consumer orthonormalises them together with
    the valence draws (extra["joint"]), as eigenvectors of one H(k) would be."""
    p = make_small() if base == "small" else make_mid()
    rng = np.random.default_rng([p.seed, 999])
    p.name = f"optical-{base}"
    p.qpts = np.zeros((1, 3))
    p.q_index = np.array([999])
    p.Ekq = band_energies(rng, (1, p.nk, p.nc), 1.1, 30.0)
    p.extra["joint"] = True
    return truncate(p, None, nw)


def make_tiny(seed: int = 7, shells_per_atom: int = 2, n_k: int = 2, nv: int = 2, nc: int = 3,
              ng: int = 9, nq: int = 2, nw: int = 16, lo: float = 0.3, hi: float = 2.0) -> Problem:
    """A tiny cell for brute-force checks (moderate exponents so that real-space
    quadrature converges on modest grids)."""
    rng = np.random.default_rng(seed)
    cell = diamond_cell()
    basis = sp_basis(rng, 2, shells_per_atom, lo, hi)
    kp = kgrid(cell, n_k)
    G = g_sorted(cell)[0][:ng].copy()         # need not close a shell
    q = random_q(rng, cell, nq, 1.5, G, min_units=0.2)
    nb = basis.nbasis
    Zk, Ek, Ekq = _states(rng, kp.shape[0], nq, nb, nv, nc, -12.0, 0.0, 1.1, 30.0)
    p = Problem("tiny", cell, basis, kp, q, G, nv, nc, Zk, Ek, Ekq,
                omega_grid(50.0, nw), 0.5 / HARTREE_EV, seed=seed)
    return truncate(p, None, None)


def mlp_init(seed: int = 2024, layers=(6, 128, 128, 128, 2)) -> np.ndarray:
    """Initial parameters of the surrogate network as one FP32 vector (per
    layer W [out][in] then b [out]): W ~ N(0, 1/fan_in), b = 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in zip(layers[:-1], layers[1:]):
        parts.append(rng.standard_normal(o * i) / np.sqrt(i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def halo_flux(v, m_chi_eV=1e9, rho_chi_GeV_cm3=0.3, v0_kms=238.0, vesc_kms=544.0, vE_kms=250.2):
    """Differential flux dPhi/dv (1/(cm^2 s) per unit v, v in units of c) of the
    standard halo seen from the Earth: n_chi v f(v) with n_chi = rho_chi/m_chi and
    f(v) the speed distribution of the truncated Maxwellian
    exp(-|v + v_E|^2/v0^2) Theta(v_esc - |v + v_E|) (angles integrated in closed
    form).  An input of the general rate (the halo term of its flux), not part
    of the screening method."""
    from math import erf, exp, pi, sqrt
    c = 299792.458
    v0, vesc, vE = v0_kms / c, vesc_kms / c, vE_kms / c
    z = vesc / v0
    norm = pi ** 1.5 * v0 ** 3 * (erf(z) - 2.0 / sqrt(pi) * z * exp(-z * z))
    out = np.zeros(len(v))
    for i, vi in enumerate(v):
        if vi <= 0.0:
            continue
        cmax = min(1.0, (vesc * vesc - vi * vi - vE * vE) / (2.0 * vi * vE))
        if cmax < -1.0:
            continue
        b = 2.0 * vi * vE / (v0 * v0)
        a = (vi * vi + vE * vE) / (v0 * v0)
        f = 2.0 * pi * vi * vi / (norm * b) * (exp(-(a - b)) - exp(-(a + b * cmax)))
        out[i] = rho_chi_GeV_cm3 * 1e9 / m_chi_eV * vi * c * 1e5 * f
    return out

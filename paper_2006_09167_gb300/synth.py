"""Seeded synthetic input systems for the short-range non-bonded path.

This module builds inputs only: coordinates, charges, atom types, Lennard-Jones
type-pair tables, exclusion lists, boxes and cut-off settings.  It holds none of
the interaction arithmetic (no pair potentials, no forces, no pair search), so
that both the CUDA library and the FP64 oracle can be driven from the same
inputs without sharing any of the method itself.

The workloads stand in for the paper's SPC/E water size sweep (Sec. V.C,
Fig. 7: water with a 1 nm cut-off and Ewald electrostatics), its Lennard-Jones
argon throughput system (Sec. V.C, Fig. 6: density 26 nm^-3, sigma 0.3345 nm),
its reaction-field runs (Sec. VI, Fig. 12) and its ensembles of independent
simulations sharing one GPU (Sec. VI, Fig. 11).  The paper's own input systems
are not used; every system here is generated from a fixed seed.

Units: nm, ps, kJ/mol, elementary charge, g/mol.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# SPC/E water model parameters (standard published values; the paper does not
# list them).  O-H bond 0.1 nm, H-O-H angle 109.47 degrees.
SPCE_Q_O = -0.8476
SPCE_Q_H = +0.4238
SPCE_SIGMA_O = 0.3166
SPCE_EPS_O = 0.650
SPCE_BOND = 0.1
SPCE_ANGLE_DEG = 109.47
MASS_O = 15.9994
MASS_H = 1.008

COULOMB_RF = 0
COULOMB_EWALD = 1
COULOMB_NONE = 2  # Lennard-Jones only (argon)


@dataclasses.dataclass
class System:
    """One periodic system in the caller's atom order.

    x: float32 [N,3] positions (inside [0, L) per axis as generated)
    q: float32 [N] charges;  types: int32 [N] type index in [0, T)
    c6, c12: float32 [T,T] symmetric Lennard-Jones tables, V = C12/r^12 - C6/r^6
    excl_off: int32 [N+1], excl_idx: int32 [*]  symmetric exclusion CSR (self implicit)
    box: float64 [3] rectangular box edges
    coulomb: COULOMB_RF or COULOMB_EWALD;  eps_r, eps_rf (inf = conducting), beta
    rc: interaction cut-off;  rlist: outer pair-list cut-off;  r_in: inner (pruned) cut-off
    mass: float64 [N] (for the MD-like drivers)
    """

    name: str
    x: np.ndarray
    q: np.ndarray
    types: np.ndarray
    c6: np.ndarray
    c12: np.ndarray
    excl_off: np.ndarray
    excl_idx: np.ndarray
    box: np.ndarray
    coulomb: int
    rc: float
    rlist: float
    r_in: float
    eps_r: float = 1.0
    eps_rf: float = math.inf
    beta: float = 0.0
    mass: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_types(self) -> int:
        return int(self.c6.shape[0])


# ---------------------------------------------------------------------------
# parameter helpers
# ---------------------------------------------------------------------------
def ewald_beta(rc: float, rtol: float = 1e-5) -> float:
    """Ewald splitting parameter beta such that erfc(beta*rc) = rtol (bisection in FP64).

    This is the input convention for the Ewald real-space settings (the paper does
    not state one); rc=1.0 nm, rtol=1e-5 gives beta = 3.123413 nm^-1.
    """
    lo, hi = 0.0, 50.0 / rc
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.erfc(mid * rc) > rtol:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def lj_c6_c12(sigma, eps):
    """C6 = 4 eps sigma^6, C12 = 4 eps sigma^12 (elementwise)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    s6 = sigma ** 6
    return 4.0 * eps * s6, 4.0 * eps * s6 * s6


def geometric_tables(c6_type, c12_type):
    """Type-pair tables by the geometric rule C_ab = sqrt(C_a C_b), as float32."""
    c6_type = np.asarray(c6_type, dtype=np.float64)
    c12_type = np.asarray(c12_type, dtype=np.float64)
    c6 = np.sqrt(np.outer(c6_type, c6_type)).astype(np.float32)
    c12 = np.sqrt(np.outer(c12_type, c12_type)).astype(np.float32)
    return c6, c12


def _wrap32(x: np.ndarray, box: np.ndarray) -> np.ndarray:
    """Wrap FP64 coordinates into [0, L) and round to float32 strictly below L."""
    w = np.mod(x, box)
    w32 = w.astype(np.float32)
    box32 = box.astype(np.float32)
    # rounding to float32 may land exactly on L (or above it when L itself rounds up)
    bad = w32.astype(np.float64) >= box
    if np.any(bad):
        w32[bad] = 0.0
    del box32
    return w32


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniformly distributed rotation matrices from normalised Gaussian quaternions."""
    qv = rng.standard_normal((n, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    a, b, c, d = qv[:, 0], qv[:, 1], qv[:, 2], qv[:, 3]
    rot = np.empty((n, 3, 3))
    rot[:, 0, 0] = a * a + b * b - c * c - d * d
    rot[:, 0, 1] = 2 * (b * c - a * d)
    rot[:, 0, 2] = 2 * (b * d + a * c)
    rot[:, 1, 0] = 2 * (b * c + a * d)
    rot[:, 1, 1] = a * a - b * b + c * c - d * d
    rot[:, 1, 2] = 2 * (c * d - a * b)
    rot[:, 2, 0] = 2 * (b * d - a * c)
    rot[:, 2, 1] = 2 * (c * d + a * b)
    rot[:, 2, 2] = a * a - b * b - c * c + d * d
    return rot


def _spce_body_frame() -> np.ndarray:
    half = math.radians(SPCE_ANGLE_DEG) / 2.0
    return np.array([
        [0.0, 0.0, 0.0],
        [SPCE_BOND * math.sin(half), 0.0, SPCE_BOND * math.cos(half)],
        [-SPCE_BOND * math.sin(half), 0.0, SPCE_BOND * math.cos(half)],
    ])


def _water_exclusions(first_atom: int, n_mol: int):
    """Intramolecular exclusion pairs (O-H1, O-H2, H1-H2) for n_mol consecutive waters."""
    base = first_atom + 3 * np.arange(n_mol)
    pairs = np.concatenate([
        np.stack([base, base + 1], 1),
        np.stack([base, base + 2], 1),
        np.stack([base + 1, base + 2], 1),
    ])
    return pairs


def csr_from_pairs(n: int, pairs: np.ndarray):
    """Symmetric CSR (offsets[N+1], idx) from unordered pairs; self is never listed."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    if pairs.size:
        assert np.all(pairs[:, 0] != pairs[:, 1])
        both = np.concatenate([pairs, pairs[:, ::-1]])
        key = np.unique(both[:, 0] * np.int64(n) + both[:, 1])  # sorted by (i, j), duplicates removed
        both = np.stack([key // n, key % n], 1)
    else:
        both = np.zeros((0, 2), dtype=np.int64)
    counts = np.bincount(both[:, 0], minlength=n)
    off = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(counts, out=off[1:])
    idx = both[np.lexsort((both[:, 1], both[:, 0])), 1].astype(np.int32)
    return off, idx


def _place_waters(rng, sites: np.ndarray, box: np.ndarray, jitter: float, o_type: np.ndarray):
    """Waters with O on the given sites, uniform random orientation and uniform jitter.

    Returns (x float64 [3M,3], q, types) in molecule order O,H1,H2.
    o_type: per-molecule type index for the oxygen (hydrogen type is 1).
    """
    m = sites.shape[0]
    rot = _random_rotations(rng, m)
    body = _spce_body_frame()
    pos = sites[:, None, :] + np.einsum("mij,aj->mai", rot, body)
    pos += rng.uniform(-jitter, jitter, size=pos.shape)
    x = pos.reshape(-1, 3)
    q = np.tile(np.array([SPCE_Q_O, SPCE_Q_H, SPCE_Q_H]), m)
    types = np.empty(3 * m, dtype=np.int32)
    types[0::3] = o_type
    types[1::3] = 1
    types[2::3] = 1
    return x, q, types


def _lattice_sites(n_side: int, box: np.ndarray) -> np.ndarray:
    g = (np.arange(n_side) + 0.5) / n_side
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1) * box


def _spce_tables(extra_o_types=None):
    """Types: 0 = SPC/E O, 1 = H (no LJ), 2.. = extra O-like types given as (sigma, eps)."""
    c6o, c12o = lj_c6_c12(SPCE_SIGMA_O, SPCE_EPS_O)
    c6_t = [c6o, 0.0]
    c12_t = [c12o, 0.0]
    for s, e in (extra_o_types or []):
        a, b = lj_c6_c12(s, e)
        c6_t.append(a)
        c12_t.append(b)
    return geometric_tables(c6_t, c12_t)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def water_box(n_mol: int, box_len: float, seed: int, *, n_side: Optional[int] = None,
              coulomb: int = COULOMB_EWALD, rc: float = 1.0, rlist: float = 1.1,
              r_in: Optional[float] = None, jitter: float = 0.02, rtol: float = 1e-5,
              extra_o_types=None, name: str = "water") -> System:
    """SPC/E water: O on a cubic lattice subset, random rotation about O, uniform jitter.

    n_side^3 >= n_mol lattice sites of spacing box_len/n_side; n_mol of them are
    chosen by a seeded permutation when the lattice has more sites than molecules.
    extra_o_types: list of (sigma, eps); every oxygen then draws its type uniformly
    from {SPC/E O} plus these.
    """
    rng = np.random.default_rng(seed)
    box = np.full(3, float(box_len))
    if n_side is None:
        n_side = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    sites = _lattice_sites(n_side, box)
    if sites.shape[0] > n_mol:
        sites = sites[np.sort(rng.permutation(sites.shape[0])[:n_mol])]
    c6, c12 = _spce_tables(extra_o_types)
    if extra_o_types:
        choices = np.array([0] + list(range(2, 2 + len(extra_o_types))), dtype=np.int32)
        o_type = choices[rng.integers(0, len(choices), size=n_mol)]
    else:
        o_type = np.zeros(n_mol, dtype=np.int32)
    x, q, types = _place_waters(rng, sites, box, jitter, o_type)
    n = x.shape[0]
    off, idx = csr_from_pairs(n, _water_exclusions(0, n_mol))
    mass = np.tile(np.array([MASS_O, MASS_H, MASS_H]), n_mol)
    beta = ewald_beta(rc, rtol) if coulomb == COULOMB_EWALD else 0.0
    return System(name=name, x=_wrap32(x, box), q=q.astype(np.float32), types=types,
                  c6=c6, c12=c12, excl_off=off, excl_idx=idx, box=box, coulomb=coulomb,
                  rc=rc, rlist=rlist, r_in=rc if r_in is None else r_in, beta=beta, mass=mass)


def water_648(seed: int = 1) -> System:
    """648-atom SPC/E box (216 molecules on a 6^3 lattice, 1.862 nm cube), reaction field
    with eps_rf = inf, rc 0.9 nm, rlist 1.0 nm."""
    return water_box(216, 1.862, seed, n_side=6, coulomb=COULOMB_RF, rc=0.9, rlist=1.0,
                     name="spce_water_648_rf")


def water_96k(seed: int = 2) -> System:
    """96,000-atom SPC/E box (32,000 of 32^3 lattice sites, 9.86 nm cube), Ewald
    real space with erfc(beta rc) = 1e-5, rc 1.0 nm, rlist 1.1 nm."""
    return water_box(32000, 9.86, seed, n_side=32, coulomb=COULOMB_EWALD, rc=1.0, rlist=1.1,
                     name="spce_water_96k_ewald")


def water_24k_types(seed: int = 4) -> System:
    """24,000-atom SPC/E box (20^3 lattice, 6.2114 nm cube) whose oxygens draw one of
    five LJ types (SPC/E O and four perturbed copies: sigma x U[0.95,1.05],
    eps x U[0.8,1.2]); Ewald as the 96k box."""
    rng = np.random.default_rng(1000 + seed)
    extra = [(SPCE_SIGMA_O * rng.uniform(0.95, 1.05), SPCE_EPS_O * rng.uniform(0.8, 1.2))
             for _ in range(4)]
    return water_box(8000, 6.2114, seed, n_side=20, coulomb=COULOMB_EWALD, rc=1.0, rlist=1.1,
                     extra_o_types=extra, name="spce_water_24k_6types")


def replica_set(n_rep: int = 256, seed: int = 5, mol_min: int = 1000, mol_max: int = 20000):
    """Independent SPC/E replicas, molecule counts log-uniform in [mol_min, mol_max],
    box edge 9.86 nm x (n_mol/32000)^(1/3); Ewald rc 1.0, rlist 1.1."""
    rng = np.random.default_rng(seed)
    n_mol = np.rint(np.exp(rng.uniform(math.log(mol_min), math.log(mol_max), size=n_rep)))
    systems = []
    for r, m in enumerate(n_mol.astype(int)):
        box_len = 9.86 * (m / 32000.0) ** (1.0 / 3.0)
        systems.append(water_box(int(m), box_len, seed * 100000 + r, coulomb=COULOMB_EWALD,
                                 rc=1.0, rlist=1.1, name=f"replica{r}"))
    return systems


def ionic_crystal(kind: str = "NaCl", a: float = 0.5640, cells: int = 2, beta: float = 8.0,
                  rc: Optional[float] = None, origin=(0.1, 0.1, 0.1)) -> System:
    """A perfect ionic crystal of unit charges in a cubic box of `cells`^3 conventional
    cells (lattice constant a, nm): "NaCl" (rock salt, 8 ions per cell) or "CsCl"
    (simple cubic pair, 2 ions per cell).  No Lennard-Jones, no exclusions, Ewald
    electrostatics with the given beta; rc just below L/2.  Used to check the Ewald
    sum against the known Madelung constants."""
    if kind == "NaCl":
        basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                          [.5, .5, .5], [.5, 0, 0], [0, .5, 0], [0, 0, .5]])
        charge = np.array([1, 1, 1, 1, -1, -1, -1, -1], np.float64)
    elif kind == "CsCl":
        basis = np.array([[0, 0, 0], [.5, .5, .5]])
        charge = np.array([1, -1], np.float64)
    else:
        raise ValueError(kind)
    g = np.arange(cells)
    cell = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = ((cell[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3) + np.asarray(origin)
    q = np.tile(charge, len(cell))
    L = cells * a
    box = np.full(3, L)
    x = np.mod(x, L)
    n = x.shape[0]
    off = np.zeros(n + 1, np.int32)
    return System(name=f"{kind.lower()}_{cells}", x=x.astype(np.float32), q=q.astype(np.float32),
                  types=np.zeros(n, np.int32), c6=np.zeros((1, 1), np.float32),
                  c12=np.zeros((1, 1), np.float32), excl_off=off, excl_idx=np.zeros(0, np.int32), box=box,
                  coulomb=COULOMB_EWALD, rc=(0.499 * L if rc is None else rc),
                  rlist=(0.499 * L if rc is None else rc), r_in=(0.499 * L if rc is None else rc),
                  beta=beta, mass=np.full(n, 30.0))


def argon_box(n_atoms: int = 1000, seed: int = 7, rho: float = 26.0, sigma: float = 0.3345,
              eps: float = 0.996, rc: float = 0.9, rlist: float = 1.0, r_in: Optional[float] = None,
              jitter: float = 0.01) -> System:
    """Lennard-Jones argon at number density rho (Sec. V.C, Fig. 6 settings) on a
    jittered simple-cubic lattice; no charges.  eps and the mass 39.948 are inputs
    the paper does not give."""
    rng = np.random.default_rng(seed)
    box_len = (n_atoms / rho) ** (1.0 / 3.0)
    box = np.full(3, box_len)
    n_side = int(math.ceil(n_atoms ** (1.0 / 3.0) - 1e-9))
    sites = _lattice_sites(n_side, box)
    if sites.shape[0] > n_atoms:
        sites = sites[np.sort(rng.permutation(sites.shape[0])[:n_atoms])]
    x = sites + rng.uniform(-jitter, jitter, size=sites.shape)
    c6a, c12a = lj_c6_c12(sigma, eps)
    c6, c12 = geometric_tables([c6a], [c12a])
    off, idx = csr_from_pairs(n_atoms, np.zeros((0, 2)))
    return System(name=f"argon_{n_atoms}", x=_wrap32(x, box), q=np.zeros(n_atoms, np.float32),
                  types=np.zeros(n_atoms, np.int32), c6=c6, c12=c12, excl_off=off, excl_idx=idx,
                  box=box, coulomb=COULOMB_NONE, rc=rc, rlist=rlist,
                  r_in=rc if r_in is None else r_in, mass=np.full(n_atoms, 39.948))


class _Grid:
    """Uniform hash grid over a periodic box for rejection sampling (generator only)."""

    def __init__(self, box, cell, cap=16):
        self.box = box
        self.nc = np.maximum((box / cell).astype(int), 1)
        self.cell = box / self.nc
        self.cap = cap
        self.slots = -np.ones((int(np.prod(self.nc)), cap), dtype=np.int64)
        self.fill = np.zeros(int(np.prod(self.nc)), dtype=np.int64)
        self.fill_max = 0  # upper bound of fill (never lowered: extra slots are empty, -1)
        self.pos = []

    def _cid(self, c):
        c = np.mod(c, self.nc)
        return (c[..., 0] * self.nc[1] + c[..., 1]) * self.nc[2] + c[..., 2]

    def near_min_dist(self, p, all_pos, ignore=None, chunk=20000):
        """Minimum-image distance from each point p[k] to stored points (inf if none)."""
        if p.shape[0] > chunk:
            return np.concatenate([
                self.near_min_dist(p[a:a + chunk], all_pos,
                                   None if ignore is None else [ig[a:a + chunk] for ig in ignore], chunk)
                for a in range(0, p.shape[0], chunk)])
        c = np.floor(p / self.cell).astype(int)
        offs = np.array([(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)])
        used = max(1, self.fill_max)
        cand = self.slots[self._cid(c[:, None, :] + offs[None])][:, :, :used]  # [k,27,used]
        cand = cand.reshape(p.shape[0], -1)
        valid = cand >= 0
        if ignore is not None:
            for ig in ignore:
                valid &= cand != ig[:, None]
        pts = all_pos[np.where(valid, cand, 0)]
        d = pts - p[:, None, :]
        d -= self.box * np.rint(d / self.box)
        r = np.sqrt((d * d).sum(-1))
        r = np.where(valid, r, np.inf)
        return r.min(axis=1) if r.shape[1] else np.full(p.shape[0], np.inf)

    def remove(self, idx, p):
        cid = self._cid(np.floor(p / self.cell).astype(int))
        for i, c in zip(idx, cid):
            f = self.fill[c]
            row = self.slots[c, :f]
            k = int(np.nonzero(row == i)[0][0])
            row[k] = row[f - 1]
            self.slots[c, f - 1] = -1
            self.fill[c] = f - 1

    def insert(self, idx, p):
        cid = self._cid(np.floor(p / self.cell).astype(int))
        for i, c in zip(idx, cid):
            f = self.fill[c]
            if f >= self.cap:
                raise RuntimeError("generator grid cell overflow")
            self.slots[c, f] = i
            self.fill[c] = f + 1
            self.fill_max = max(self.fill_max, int(f) + 1)


def polymer_water_box(seed: int = 3, n_chain: int = 1125, chain_len: int = 200,
                      n_water: int = 425000, box_len: float = 24.63, n_poly_types: int = 20,
                      bond: float = 0.15, min_13: float = 0.2, min_nb: float = 0.2,
                      water_clear: float = 0.22, water_side: int = 87, persistence: float = 1.5,
                      rc: float = 1.2, rlist: float = 1.3) -> System:
    """Heterogeneous box: 85% SPC/E water plus 15% polymer chains (1.5M atoms by default).

    Chains are grown in parallel as persistent random walks (Gaussian step plus
    `persistence` times the previous bond direction) with bond length 0.15 nm, each
    step rejected if the 1-3 distance falls below 0.2 nm or any non-bonded chain
    atom lies within 0.2 nm.  Chain atom types are uniform over 20 types with
    sigma U[0.25,0.38] nm and eps U[0.2,1.0] kJ/mol; chain charges are N(0,0.4)
    shifted to zero net charge per chain; 1-2 and 1-3 pairs are excluded.  Waters
    occupy the sites of a water_side^3 cubic lattice whose points are at least
    water_clear from every chain atom, chosen by a seeded permutation.  Ewald with
    erfc(beta rc) = 1e-5 at rc 1.2 nm, rlist 1.3 nm.
    """
    rng = np.random.default_rng(seed)
    box = np.full(3, float(box_len))
    n_poly = n_chain * chain_len
    pos = np.zeros((n_poly, 3))
    grid = _Grid(box, 0.25, cap=24)
    placed_any = np.zeros(n_poly, dtype=bool)
    prev_idx = -np.ones(n_chain, dtype=np.int64)
    prev2_idx = -np.ones(n_chain, dtype=np.int64)
    failed = np.zeros(n_chain, dtype=bool)

    def propose(a_prev, a_prev2, m):
        """m candidate next positions after atom a_prev (a_prev2 the one before, or -1)."""
        dvec = rng.standard_normal((m, 3))
        if a_prev2 >= 0:
            pd = pos[a_prev] - pos[a_prev2]
            pd -= box * np.rint(pd / box)
            dvec += persistence * pd / bond
        dvec /= np.linalg.norm(dvec, axis=1, keepdims=True)
        return np.mod(pos[a_prev] + bond * dvec, box)

    def acceptable(p, a_prev, a_prev2):
        if a_prev2 >= 0:
            d13 = p - pos[a_prev2]
            d13 -= box * np.rint(d13 / box)
            if np.sqrt((d13 * d13).sum()) < min_13:
                return False
        ign = [np.array([a_prev]), np.array([a_prev2])]
        return grid.near_min_dist(p[None], pos, ignore=ign)[0] >= min_nb

    # phase 1: all chains grow in lock step (vectorised proposals)
    for k in range(chain_len):
        idx_now = np.arange(n_chain) * chain_len + k
        todo = np.nonzero(~failed)[0]
        for attempt in range(400):
            if todo.size == 0:
                break
            if k == 0:
                cand = rng.uniform(0, 1, size=(todo.size, 3)) * box
            else:
                dvec = rng.standard_normal((todo.size, 3))
                if k >= 2:
                    pd = pos[prev_idx[todo]] - pos[prev2_idx[todo]]
                    pd -= box * np.rint(pd / box)
                    dvec += persistence * pd / bond
                dvec /= np.linalg.norm(dvec, axis=1, keepdims=True)
                cand = np.mod(pos[prev_idx[todo]] + bond * dvec, box)
            ok = np.ones(todo.size, dtype=bool)
            if k >= 2:
                d13 = cand - pos[prev2_idx[todo]]
                d13 -= box * np.rint(d13 / box)
                ok &= np.sqrt((d13 * d13).sum(1)) >= min_13
            ok &= grid.near_min_dist(cand, pos, ignore=[prev_idx[todo], prev2_idx[todo]]) >= min_nb
            # two chains growing in the same step must not clash with each other: of every
            # pair of accepted candidates closer than min_nb, the later one is rejected
            acc = np.nonzero(ok)[0]
            if acc.size > 1:
                pa = cand[acc]
                dd = pa[:, None, :] - pa[None, :, :]
                dd -= box * np.rint(dd / box)
                close = (dd * dd).sum(-1) < min_nb * min_nb
                close = np.triu(close, 1)
                ok[acc[np.any(close, axis=0)]] = False
            done = ok
            acc = np.nonzero(done)[0]
            if acc.size:
                ids = idx_now[todo[acc]]
                pos[ids] = cand[acc]
                placed_any[ids] = True
                grid.insert(ids, cand[acc])
            todo = todo[~done]
        for a in todo:  # trapped: take the chain out and regrow it later
            failed[a] = True
            ids = np.arange(a * chain_len, a * chain_len + k)
            ids = ids[placed_any[ids]]
            if ids.size:
                grid.remove(ids, pos[ids])
                placed_any[ids] = False
        prev2_idx[:] = prev_idx
        prev_idx[:] = idx_now
    # phase 2: regrow trapped chains one by one, backtracking when stuck
    for a in np.nonzero(failed)[0]:
        base_i = a * chain_len
        k = 0
        stuck = 0
        while k < chain_len:
            i = base_i + k
            a_prev = i - 1 if k >= 1 else -1
            a_prev2 = i - 2 if k >= 2 else -1
            ok = False
            for _ in range(50):
                if k == 0:
                    p = rng.uniform(0, 1, size=3) * box
                else:
                    p = propose(a_prev, a_prev2, 1)[0]
                if acceptable(p, a_prev, a_prev2):
                    ok = True
                    break
            if ok:
                pos[i] = p
                placed_any[i] = True
                grid.insert([i], p[None])
                k += 1
                continue
            stuck += 1
            if stuck > 10000:
                raise RuntimeError("polymer regrowth failed")
            back = min(k, 5)
            ids = np.arange(base_i + k - back, base_i + k)
            if ids.size:
                grid.remove(ids, pos[ids])
                placed_any[ids] = False
            k -= back
    assert placed_any.all()
    # polymer types / charges
    sig = rng.uniform(0.25, 0.38, size=n_poly_types)
    eps = rng.uniform(0.2, 1.0, size=n_poly_types)
    c6_p, c12_p = lj_c6_c12(sig, eps)
    c6o, c12o = lj_c6_c12(SPCE_SIGMA_O, SPCE_EPS_O)
    c6, c12 = geometric_tables(np.concatenate([[c6o, 0.0], c6_p]),
                               np.concatenate([[c12o, 0.0], c12_p]))
    ptypes = (2 + rng.integers(0, n_poly_types, size=n_poly)).astype(np.int32)
    pq = rng.normal(0.0, 0.4, size=(n_chain, chain_len))
    pq -= pq.mean(axis=1, keepdims=True)
    # water sites clear of the chains
    sites = _lattice_sites(water_side, box)
    wgrid_d = grid.near_min_dist(sites, pos)
    free = np.nonzero(wgrid_d >= water_clear)[0]
    if free.size < n_water:
        raise RuntimeError(f"only {free.size} free water sites (< {n_water})")
    sites = sites[np.sort(rng.permutation(free)[:n_water])]
    wx, wq, wtypes = _place_waters(rng, sites, box, 0.02, np.zeros(n_water, np.int32))
    x = np.concatenate([pos, wx])
    q = np.concatenate([pq.ravel(), wq])
    types = np.concatenate([ptypes, wtypes]).astype(np.int32)
    # exclusions: chain 1-2, 1-3 and water intramolecular
    base = (np.arange(n_chain) * chain_len)[:, None]
    k12 = np.arange(chain_len - 1)[None, :] + base
    k13 = np.arange(chain_len - 2)[None, :] + base
    pairs = np.concatenate([
        np.stack([k12.ravel(), k12.ravel() + 1], 1),
        np.stack([k13.ravel(), k13.ravel() + 2], 1),
        _water_exclusions(n_poly, n_water),
    ])
    n = x.shape[0]
    off, idx = csr_from_pairs(n, pairs)
    mass = np.concatenate([np.full(n_poly, 14.0), np.tile([MASS_O, MASS_H, MASS_H], n_water)])
    return System(name="polymer_water_1.5M", x=_wrap32(x, box), q=q.astype(np.float32),
                  types=types, c6=c6, c12=c12, excl_off=off, excl_idx=idx, box=box,
                  coulomb=COULOMB_EWALD, rc=rc, rlist=rlist, r_in=rc,
                  beta=ewald_beta(rc), mass=mass)


def maxwell_boltzmann(system: System, temperature: float, seed: int) -> np.ndarray:
    """Velocities [N,3] (nm/ps) drawn from Maxwell-Boltzmann at the given temperature."""
    kb = 0.0083144626  # kJ/mol/K
    rng = np.random.default_rng(seed)
    m = system.mass if system.mass is not None else np.ones(system.n)
    s = np.sqrt(kb * temperature / m)[:, None]
    v = rng.standard_normal((system.n, 3)) * s
    v -= (m[:, None] * v).sum(0) / m.sum()
    return v


def subsystem(system: System, keep: np.ndarray) -> System:
    """A copy restricted to the atoms in `keep` (exclusions remapped), same box."""
    keep = np.asarray(keep, dtype=np.int64)
    remap = -np.ones(system.n, dtype=np.int64)
    remap[keep] = np.arange(keep.size)
    pairs = []
    for a in keep:
        for b in system.excl_idx[system.excl_off[a]:system.excl_off[a + 1]]:
            if remap[b] >= 0 and a < b:
                pairs.append((remap[a], remap[b]))
    off, idx = csr_from_pairs(keep.size, np.array(pairs).reshape(-1, 2))
    return dataclasses.replace(system, name=system.name + "_sub", x=system.x[keep].copy(),
                               q=system.q[keep].copy(), types=system.types[keep].copy(),
                               excl_off=off, excl_idx=idx,
                               mass=None if system.mass is None else system.mass[keep].copy())

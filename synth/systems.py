"""Seeded synthetic molecular clusters: geometry, fragment partition and random Gaussian bases.

This module is the only code shared by the CPU oracle and the CUDA path.  It draws random
numbers and places atoms; it holds none of the fragment-mean-field arithmetic (no integrals,
no Fock matrices, no densities).  The one numerical check it makes is a rejection test on a
drawn element basis (the smallest eigenvalue of the one-centre overlap of same-l shells), which
only decides which draw is kept.

Workloads follow the paper's setting (Theory, "Fragment Mean Field"): a molecular system split
into fragments, each fragment carrying its own monomer-centred contracted Cartesian Gaussian
basis.  The paper gives no geometries, so every system here is synthetic:

* water-like fragments: O-H 0.96 A, H-O-H 104.5 deg, uniform random orientation;
* a planar cytosine-like heterocycle C4N3OH5 (13 atoms), 1.4 A heavy-atom bonds, 1.0-1.1 A X-H;
* formamide-like CH3NO (6 atoms) and guanine-like C5N5OH5 (16 atoms) planar fragments;
* clusters made by random sequential addition in a cube, heavy-atom separations >= 2.6 A between
  fragments and no inter-fragment atom pair closer than 1.4 A.

Basis: per basis set, contracted Cartesian shells with 3 primitives each; exponents
log-uniform in [0.1, 50], contraction coefficients U(0.1, 1) scaled to unit 2-norm.  The
coefficients multiply primitives normalised at shell level (radial factor); each Cartesian AO is
then renormalised by the consumer so that its self-overlap is 1.

Lengths are in Angstrom here; consumers convert to bohr.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ANGSTROM_PER_BOHR = 0.529177210903  # CODATA 2018

MASS = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999}
AVOGADRO = 6.02214076e23

# shell angular momenta per basis-set kind
SHELLS_H = (0, 0)
SHELLS_O_SP = (0, 0, 0, 1, 1)
SHELLS_HEAVY_SPD = (0, 0, 0, 1, 1, 2)

EXP_LO, EXP_HI = 0.1, 50.0
N_PRIM = 3


@dataclasses.dataclass
class BasisSet:
    """Shells of one basis-set kind: angular momentum, exponents and raw coefficients."""

    l: list
    exps: list  # list of arrays, one per shell
    coefs: list


@dataclasses.dataclass
class System:
    """A fragmented molecular cluster with its basis.

    Z[n_atoms], xyz[n_atoms, 3] (Angstrom), frag_of_atom[n_atoms] (fragments are contiguous atom
    ranges, in order), charge[n_frag], basis_of_atom[n_atoms] indexing ``basis_sets``.
    """

    Z: np.ndarray
    xyz: np.ndarray
    frag_of_atom: np.ndarray
    charge: np.ndarray
    basis_of_atom: np.ndarray
    basis_sets: list
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.Z.shape[0])

    @property
    def n_frag(self) -> int:
        return int(self.charge.shape[0])

    def frag_atoms(self, x: int) -> np.ndarray:
        return np.nonzero(self.frag_of_atom == x)[0]

    def flat_basis(self):
        """Basis sets flattened into arrays: (set_shell_offset, shell_l, shell_nprim, exps, coefs)."""
        off = [0]
        l, npr, ex, co = [], [], [], []
        for bs in self.basis_sets:
            for sl, se, sc in zip(bs.l, bs.exps, bs.coefs):
                l.append(sl)
                npr.append(len(se))
                ex.extend(se)
                co.extend(sc)
            off.append(len(l))
        return (np.asarray(off, np.int32), np.asarray(l, np.int32), np.asarray(npr, np.int32),
                np.asarray(ex, np.float64), np.asarray(co, np.float64))


def _streams(seed: int, n: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(n)]


def random_rotation(rng) -> np.ndarray:
    """Uniform random rotation matrix (normalised Gaussian quaternion)."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def random_unit(rng) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def _one_centre_min_eig(ls, exps, coefs) -> float:
    """Smallest eigenvalue of the overlap of same-l contracted shells on one centre.

    Uses the textbook overlap of two one-centre radial Gaussians of equal l,
    <a|b> = (2 sqrt(ab) / (a + b))^(l + 3/2) for shell-level normalised primitives.  Only a
    rejection test for near-linearly-dependent draws.
    """
    worst = 1.0
    for lv in sorted(set(ls)):
        idx = [i for i, x in enumerate(ls) if x == lv]
        n = len(idx)
        S = np.zeros((n, n))
        for i in range(n):
            for j in range(n):
                ea, ca = exps[idx[i]], coefs[idx[i]]
                eb, cb = exps[idx[j]], coefs[idx[j]]
                r = (2.0 * np.sqrt(np.outer(ea, eb)) / np.add.outer(ea, eb)) ** (lv + 1.5)
                S[i, j] = ca @ r @ cb
        d = 1.0 / np.sqrt(np.diag(S))
        worst = min(worst, float(np.linalg.eigvalsh(S * np.outer(d, d)).min()))
    return worst


def random_basis_set(rng, shell_ls, min_eig: float = 1e-4) -> BasisSet:
    """Draw one basis-set kind; redraw until the one-centre overlap is well conditioned."""
    while True:
        exps, coefs = [], []
        for _ in shell_ls:
            e = np.exp(rng.uniform(math.log(EXP_LO), math.log(EXP_HI), N_PRIM))
            c = rng.uniform(0.1, 1.0, N_PRIM)
            exps.append(np.sort(e)[::-1].copy())
            coefs.append(c / np.linalg.norm(c))
        if _one_centre_min_eig(list(shell_ls), exps, coefs) >= min_eig:
            return BasisSet(list(shell_ls), exps, coefs)


# ----------------------------------------------------------------------------- fragment shapes

def water_geometry():
    """Water-like monomer: (Z, xyz) with O at the origin, O-H 0.96 A, angle 104.5 deg."""
    r, th = 0.96, math.radians(104.5)
    xyz = np.array([[0.0, 0.0, 0.0],
                    [r * math.sin(th / 2), 0.0, r * math.cos(th / 2)],
                    [-r * math.sin(th / 2), 0.0, r * math.cos(th / 2)]])
    return np.array([8, 1, 1], np.int32), xyz


def _add_h(xyz_list, z_list, anchor, direction, rng):
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    xyz_list.append(np.asarray(anchor) + rng.uniform(1.0, 1.1) * d)
    z_list.append(1)


def cytosine_like_geometry(rng):
    """Planar C4N3OH5 heterocycle (13 atoms) in the xy plane, centred at the origin.

    Six-ring N1 C2 N3 C4 C5 C6 (1.4 A bonds), exocyclic O on C2 and N on C4 (1.4 A), H on N1, C5,
    C6 and two on the exocyclic N; X-H drawn in [1.0, 1.1] A; in-plane jitter of 0.02 A.
    """
    bond = 1.4
    ring_z = [7, 6, 7, 6, 6, 6]
    ang = [math.radians(90 + 60 * k) for k in range(6)]
    ring = [np.array([bond * math.cos(a), bond * math.sin(a), 0.0]) for a in ang]
    z, xyz = list(ring_z), list(ring)
    out = [r / np.linalg.norm(r) for r in ring]
    xyz.append(ring[1] + bond * out[1]); z.append(8)          # O on C2
    n4 = ring[3] + bond * out[3]
    xyz.append(n4); z.append(7)                              # exocyclic N on C4
    _add_h(xyz, z, ring[0], out[0], rng)                     # H on N1
    _add_h(xyz, z, ring[4], out[4], rng)                     # H on C5
    _add_h(xyz, z, ring[5], out[5], rng)                     # H on C6
    rot60 = lambda v, s: np.array([v[0] * math.cos(s) - v[1] * math.sin(s),
                                   v[0] * math.sin(s) + v[1] * math.cos(s), 0.0])
    _add_h(xyz, z, n4, rot60(out[3], math.radians(60)), rng)
    _add_h(xyz, z, n4, rot60(out[3], math.radians(-60)), rng)
    xyz = np.array(xyz)
    xyz[:, :2] += rng.uniform(-0.02, 0.02, (len(z), 2))
    xyz -= xyz.mean(axis=0)
    return np.array(z, np.int32), xyz


def formamide_like_geometry(rng):
    """Planar CH3NO (6 atoms): C with O and N at 1.4 A and 120 deg, H on C, two H on N."""
    bond = 1.4
    c = np.zeros(3)
    o = np.array([bond, 0.0, 0.0])
    t = math.radians(120)
    n = np.array([bond * math.cos(t), bond * math.sin(t), 0.0])
    z, xyz = [6, 8, 7], [c, o, n]
    _add_h(xyz, z, c, [math.cos(-t), math.sin(-t), 0.0], rng)
    _add_h(xyz, z, n, [math.cos(t + math.radians(60)), math.sin(t + math.radians(60)), 0.0], rng)
    _add_h(xyz, z, n, [math.cos(t - math.radians(60)), math.sin(t - math.radians(60)), 0.0], rng)
    xyz = np.array(xyz)
    xyz[:, :2] += rng.uniform(-0.02, 0.02, (len(z), 2))
    xyz -= xyz.mean(axis=0)
    return np.array(z, np.int32), xyz


def guanine_like_geometry(rng):
    """Planar C5N5OH5 (16 atoms): a 6-ring fused with a 5-ring, exocyclic O and NH2."""
    bond = 1.4
    hexa = [np.array([bond * math.cos(math.radians(30 + 60 * k)),
                      bond * math.sin(math.radians(30 + 60 * k)), 0.0]) for k in range(6)]
    # hexagon atoms k=0..5; fuse the pentagon on edge (0, 5) (the +x side)
    a, b = hexa[0], hexa[5]
    mid = 0.5 * (a + b)
    outdir = mid / np.linalg.norm(mid)
    h_pent = bond / (2 * math.tan(math.radians(36)))  # apothem of a regular pentagon
    centre = mid + h_pent * outdir
    R = bond / (2 * math.sin(math.radians(36)))
    base = math.atan2(a[1] - centre[1], a[0] - centre[0])
    pent = [centre + R * np.array([math.cos(base - math.radians(72) * k),
                                   math.sin(base - math.radians(72) * k), 0.0]) for k in range(5)]
    # ring atoms: hexagon C4(0) C5... assign Z: fused atoms C, C; others by formula C5N5O
    ring_xyz = hexa + [pent[1], pent[2], pent[3]]
    ring_z = [6, 7, 6, 7, 6, 6, 7, 6, 7]       # 5 C + 4 N in the rings
    z, xyz = list(ring_z), list(ring_xyz)
    c_all = np.mean(np.array(ring_xyz), axis=0)
    out = lambda p: (p - c_all) / np.linalg.norm(p - c_all)
    o = hexa[4] + bond * out(hexa[4]); xyz.append(o); z.append(8)
    n2 = hexa[2] + bond * out(hexa[2]); xyz.append(n2); z.append(7)
    _add_h(xyz, z, hexa[3], out(hexa[3]), rng)          # H on ring N
    _add_h(xyz, z, pent[2], out(pent[2]), rng)          # H on C8
    _add_h(xyz, z, pent[3], out(pent[3]), rng)          # H on N9
    d = out(hexa[2])
    rot = lambda v, s: np.array([v[0] * math.cos(s) - v[1] * math.sin(s),
                                 v[0] * math.sin(s) + v[1] * math.cos(s), 0.0])
    _add_h(xyz, z, n2, rot(d, math.radians(60)), rng)
    _add_h(xyz, z, n2, rot(d, math.radians(-60)), rng)
    xyz = np.array(xyz)
    xyz[:, :2] += rng.uniform(-0.02, 0.02, (len(z), 2))
    xyz -= xyz.mean(axis=0)
    return np.array(z, np.int32), xyz


# ----------------------------------------------------------------------------- assembly

def _min_pair_ok(new_xyz, new_z, placed_xyz, placed_z, heavy_min=2.6, any_min=1.4):
    if placed_xyz is None or len(placed_xyz) == 0:
        return True
    d = np.linalg.norm(new_xyz[:, None, :] - placed_xyz[None, :, :], axis=-1)
    if d.min() < any_min:
        return False
    hn = new_z > 1
    hp = placed_z > 1
    if hn.any() and hp.any() and d[np.ix_(hn, hp)].min() < heavy_min:
        return False
    return True


def _assemble(frags, basis_sets, kind_of_frag_atom, name):
    Z = np.concatenate([f[0] for f in frags]).astype(np.int32)
    xyz = np.concatenate([f[1] for f in frags]).astype(np.float64)
    foa = np.concatenate([np.full(len(f[0]), i, np.int32) for i, f in enumerate(frags)])
    boa = np.concatenate(kind_of_frag_atom).astype(np.int32)
    return System(Z=Z, xyz=xyz, frag_of_atom=foa, charge=np.zeros(len(frags), np.int32),
                  basis_of_atom=boa, basis_sets=basis_sets, name=name)


def water_dimer(seed: int = 0, r_oo: float = 3.0) -> System:
    """Two water-like fragments, seeded rotations, O-O separation along a seeded direction.

    Basis: O 3s2p, H 2s, 3 primitives per shell.
    """
    rb, rg = _streams(seed, 2)
    bs = [random_basis_set(rb, SHELLS_O_SP), random_basis_set(rb, SHELLS_H)]
    z, w = water_geometry()
    u = random_unit(rg)
    frags = []
    for k in range(2):
        Rm = random_rotation(rg)
        frags.append((z, w @ Rm.T + (k * r_oo) * u))
    kinds = [np.array([0, 1, 1])] * 2
    return _assemble(frags, bs, kinds, f"water_dimer(seed={seed}, r_oo={r_oo})")


def cube_side_for_density(total_mass_amu: float, density_g_cm3: float = 1.0) -> float:
    grams = total_mass_amu / AVOGADRO
    return (grams / density_g_cm3) ** (1.0 / 3.0) * 1e8  # cm -> Angstrom


def water_box(n_water: int, seed: int = 0, side: float | None = None,
              basis_sets=None, max_tries: int = 200000) -> System:
    """``n_water`` water-like fragments in a cube (default side: 1 g/cm^3).

    Random sequential addition: O uniform in the cube with O-O >= 2.6 A to every placed
    fragment and no inter-fragment atom pair closer than 1.4 A; random orientations.
    """
    rb, rg = _streams(seed, 2)
    if basis_sets is None:
        basis_sets = [random_basis_set(rb, SHELLS_O_SP), random_basis_set(rb, SHELLS_H)]
    if side is None:
        side = cube_side_for_density(n_water * (MASS[8] + 2 * MASS[1]))
    z, w = water_geometry()
    frags = _place(rg, [(z, w)] * n_water, side, max_tries)
    kinds = [np.array([0, 1, 1])] * n_water
    return _assemble(frags, basis_sets, kinds, f"water_box(n={n_water}, side={side:.2f}, seed={seed})")


class _CellList:
    """Placed atoms binned in cubic cells of the largest exclusion distance, so that a candidate is
    tested only against atoms that can lie within that distance (the test's outcome is unchanged)."""

    def __init__(self, cell: float):
        self.cell = cell
        self.bins = {}
        self.xyz = []
        self.z = []

    def add(self, xyz, z):
        for r, q in zip(xyz, z):
            key = tuple(np.floor(r / self.cell).astype(int))
            self.bins.setdefault(key, []).append(len(self.xyz))
            self.xyz.append(r)
            self.z.append(int(q))

    def near(self, xyz):
        idx = set()
        for r in xyz:
            kx, ky, kz = np.floor(r / self.cell).astype(int)
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        idx.update(self.bins.get((kx + dx, ky + dy, kz + dz), ()))
        idx = sorted(idx)
        return np.array([self.xyz[i] for i in idx]).reshape(-1, 3), np.array([self.z[i] for i in idx], np.int32)


def _place(rg, shapes, side, max_tries, fixed=None):
    cells = _CellList(2.6)  # the heavy-atom exclusion distance of _min_pair_ok, its largest
    frags = []
    if fixed is not None:
        for z, xyz in fixed:
            frags.append((z, xyz))
            cells.add(xyz, z)
    for z, w in shapes:
        for _ in range(max_tries):
            Rm = random_rotation(rg)
            c = rg.uniform(0.0, side, 3)
            xyz = w @ Rm.T + c
            near_xyz, near_z = cells.near(xyz)
            if _min_pair_ok(xyz, z, near_xyz, near_z):
                break
        else:
            raise RuntimeError("random sequential addition failed; box too dense")
        frags.append((z, xyz))
        cells.add(xyz, z)
    return frags


def solvated_heterocycle(n_water: int = 1000, side: float = 31.0, seed: int = 0, heavy_shells=None) -> System:
    """A cytosine-like C4N3OH5 fragment (heavy atoms 3s2p1d, 130 AOs; or ``heavy_shells``, e.g.
    SHELLS_O_SP for an 82-AO s/p solute) at the cube centre, plus ``n_water`` water-like fragments
    (O 3s2p, H 2s) placed around it."""
    rb, rg = _streams(seed, 2)
    bs = [random_basis_set(rb, SHELLS_O_SP), random_basis_set(rb, SHELLS_H)]
    heavy = {zz: random_basis_set(rb, SHELLS_HEAVY_SPD if heavy_shells is None else heavy_shells) for zz in (6, 7, 8)}
    kind_of = {}
    for zz in (6, 7, 8):
        kind_of[zz] = len(bs)
        bs.append(heavy[zz])
    zs, xs = cytosine_like_geometry(rg)
    xs = xs @ random_rotation(rg).T + side / 2
    z, w = water_geometry()
    frags = _place(rg, [(z, w)] * n_water, side, 200000, fixed=[(zs, xs)])
    kinds = [np.array([kind_of[int(q)] if q > 1 else 1 for q in zs])] + [np.array([0, 1, 1])] * n_water
    return _assemble(frags, bs, kinds, f"solvated_heterocycle(n_water={n_water}, side={side}, seed={seed})")


FRAG_TYPES = {3: "water", 6: "formamide", 13: "cytosine", 16: "guanine"}


# Basis-set seed of the mixed (batching) workload: the first of seeds 0-15 whose log-uniform draw
# gives bound fragments (isolated water-like and formamide-like RHF, which carry all four element
# bases: highest occupied orbital below -0.2 Eh, gap above 0.3 Eh).  Most draws of 3s2p1d heavy-atom
# shells leave the highest occupied orbital unbound (up to +1.4 Eh), and such fragments' RHF in a
# field does not converge.  Fixed once, offline; the generator itself runs no SCF.
MIXED_BASIS_SEED = 5


def mixed_snapshot(n_frag: int = 500, seed: int = 0, weights=(0.85, 0.08, 0.05, 0.02),
                   basis_seed: int | None = None) -> System:
    """Fragments of uneven size drawn from {3, 6, 13, 16} atoms; all heavy atoms 3s2p1d, H 2s.

    Cube side from the total mass at 1 g/cm^3; larger fragments are placed first.  The basis sets
    come from the sub-stream of ``basis_seed`` when given (e.g. MIXED_BASIS_SEED, shared by all
    snapshots of a batch), else from ``seed``.
    """
    rb, rg, rs = _streams(seed, 3)
    if basis_seed is not None:
        rb = _streams(basis_seed, 3)[0]
    bs = [random_basis_set(rb, SHELLS_H)]
    kind_of = {1: 0}
    for zz in (6, 7, 8):
        kind_of[zz] = len(bs)
        bs.append(random_basis_set(rb, SHELLS_HEAVY_SPD))
    sizes = rs.choice([3, 6, 13, 16], size=n_frag, p=np.asarray(weights) / np.sum(weights))
    sizes = np.sort(sizes)[::-1]
    shapes = []
    for s in sizes:
        if s == 3:
            shapes.append(water_geometry())
        elif s == 6:
            shapes.append(formamide_like_geometry(rg))
        elif s == 13:
            shapes.append(cytosine_like_geometry(rg))
        else:
            shapes.append(guanine_like_geometry(rg))
    mass = sum(MASS[int(q)] for z, _ in shapes for q in z)
    side = cube_side_for_density(mass)
    frags = _place(rg, shapes, side, 200000)
    kinds = [np.array([kind_of[int(q)] for q in z]) for z, _ in frags]
    return _assemble(frags, bs, kinds, f"mixed_snapshot(n_frag={n_frag}, seed={seed}, basis_seed={basis_seed})")


def batch(systems, gap: float = 20.0) -> System:
    """Independent snapshots in one system: each snapshot is translated along x so that its smallest
    x lies gap (A) beyond the largest x of the one before, so that no atom pair (and no fragment pair)
    across snapshots is closer than gap; basis sets are concatenated and re-indexed."""
    Z, xyz, foa, boa, charge, bases = [], [], [], [], [], []
    f0 = 0
    x_end = None
    for k, sy in enumerate(systems):
        shift = 0.0 if x_end is None else x_end + gap - float(sy.xyz[:, 0].min())
        x_end = float(sy.xyz[:, 0].max()) + shift
        Z.append(sy.Z)
        xyz.append(sy.xyz + np.array([shift, 0.0, 0.0]))
        foa.append(sy.frag_of_atom + f0)
        boa.append(sy.basis_of_atom + len(bases))
        charge.append(sy.charge)
        bases.extend(sy.basis_sets)
        f0 += sy.n_frag
    return System(Z=np.concatenate(Z).astype(np.int32), xyz=np.concatenate(xyz), frag_of_atom=np.concatenate(foa).astype(np.int32),
                  charge=np.concatenate(charge).astype(np.int32), basis_of_atom=np.concatenate(boa).astype(np.int32),
                  basis_sets=bases, name=f"batch({len(systems)} x {systems[0].name}, gap={gap})")


def random_orbital_coefficients(seed: int, n_ao: int, n_occ: int) -> np.ndarray:
    """G ~ N(0, 1) of shape (n_ao, n_occ): raw occupied-orbital coefficients.

    The consumer orthonormalises them in its own overlap metric, C = G (G^T S G)^(-1/2), and
    forms D = 2 C C^T.
    """
    return np.random.default_rng(seed).standard_normal((n_ao, n_occ))


def n_ao_of_basis_set(bs: BasisSet) -> int:
    return sum((l + 1) * (l + 2) // 2 for l in bs.l)


def frag_n_ao(system: System, x: int) -> int:
    return sum(n_ao_of_basis_set(system.basis_sets[system.basis_of_atom[a]]) for a in system.frag_atoms(x))


def frag_n_occ(system: System, x: int) -> int:
    ne = int(system.Z[system.frag_atoms(x)].sum()) - int(system.charge[x])
    if ne % 2:
        raise ValueError(f"fragment {x} has an odd electron count")
    return ne // 2

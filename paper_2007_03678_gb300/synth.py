"""Seeded synthetic inputs for the docking hot path.

This module only draws inputs: receptor atoms, grid geometry, ligand trees,
random genotypes and the synthetic force-field table.  It holds none of the
method's arithmetic (no energies, no poses, no map values), so both the CUDA
library and the CPU oracle can be fed from it without sharing code.

Stand-ins for the paper's data (Sec. 2.3): the paper docks SN9000/S42 ligands
against AutoGrid4 maps of real receptors (6VWW, Mpro).  None of those are
available, so every input here is a seeded synthetic object with the shapes
the paper's workloads have: a 22.5 A-class focused box (64^3 x 0.375 A), drug
like ligands of 10-60 heavy atoms and 0-15 rotatable bonds, 7 ligand atom
types plus electrostatic and desolvation maps.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

# Atom types (AutoDock4 naming).  Map index t for t < 7; 7 = elec, 8 = desolv.
TYPE_NAMES = ("C", "A", "N", "NA", "OA", "HD", "S")
NTYPES = 7
NMAPS = 9
MAP_ELEC = 7
MAP_DESOLV = 8
T_C, T_A, T_N, T_NA, T_OA, T_HD, T_S = range(7)

MAX_ATOMS = 128
MAX_TORS = 16


def forcefield() -> dict:
    """Synthetic AD4-like parameter table (data only).

    The paper names the AutoDock4 physics-based energy (vdW, H-bond,
    electrostatics, desolvation, torsional entropy; Sec. 1) but prints no
    parameters.  The weights below are the published AD4.1 free-energy
    weights; the per-type radii, well depths, volumes and solvation
    parameters are plausible AD4-like magnitudes chosen for this synthetic
    workload, not a copy of any parameter file.
    """
    per_type = {
        #        Rii   epsii  vol     solpar    donor acc  hbR  hbeps
        "C":  (4.00, 0.150, 33.51, -0.00143, 0, 0, 0.0, 0.0),
        "A":  (4.00, 0.150, 33.51, -0.00052, 0, 0, 0.0, 0.0),
        "N":  (3.50, 0.160, 22.45, -0.00162, 0, 0, 0.0, 0.0),
        "NA": (3.50, 0.160, 22.45, -0.00162, 0, 1, 1.9, 5.0),
        "OA": (3.20, 0.200, 17.16, -0.00251, 0, 1, 1.9, 5.0),
        "HD": (2.00, 0.020, 0.00, 0.00051, 1, 0, 0.0, 0.0),
        "S":  (4.00, 0.200, 33.51, -0.00214, 0, 0, 0.0, 0.0),
    }
    cols = list(zip(*[per_type[n] for n in TYPE_NAMES]))
    ff = dict(
        Rii=list(cols[0]), epsii=list(cols[1]), vol=list(cols[2]), solpar=list(cols[3]),
        hb_donor=[int(v) for v in cols[4]], hb_acceptor=[int(v) for v in cols[5]],
        hb_R=list(cols[6]), hb_eps=list(cols[7]),
        w_vdw=0.1662, w_hb=0.1209, w_elec=0.1406, w_desolv=0.1322, w_tors=0.2983,
        qasp=0.01097, sigma=3.6, coulomb=332.06363,
        ms_A=-8.5525, ms_eps0=78.4, ms_lambda=0.003627, ms_k=7.7839,
        r_min=0.5, e_cap=1.0e5, map_r_on=7.0, map_r_off=8.0, k_out=10.0,
    )
    # the library receives the table as float32: round every real value here
    for k, v in ff.items():
        if k in ("hb_donor", "hb_acceptor"):
            continue
        ff[k] = [float(x) for x in f32(v)] if isinstance(v, list) else float(f32(v))
    return ff


@dataclass
class Grid:
    n: tuple            # points per axis (nx, ny, nz)
    origin: tuple       # coordinates of node (0, 0, 0), Angstrom
    spacing: float      # Angstrom

    @property
    def center(self):
        return tuple(o + 0.5 * (k - 1) * self.spacing for o, k in zip(self.origin, self.n))

    @property
    def extent(self):
        return tuple((k - 1) * self.spacing for k in self.n)


def make_grid(npts: int, spacing: float = 0.375, center=(0.0, 0.0, 0.0)) -> Grid:
    half = 0.5 * (npts - 1) * spacing
    return Grid((npts, npts, npts), tuple(c - half for c in center), spacing)


@dataclass
class Receptor:
    xyz: np.ndarray     # (n, 3) float64
    type: np.ndarray    # (n,) int32
    charge: np.ndarray  # (n,) float64


RECEPTOR_TYPE_FREQ = np.array([0.45, 0.10, 0.08, 0.04, 0.15, 0.15, 0.03])
LIGAND_HEAVY_FREQ = {T_C: 0.55, T_A: 0.15, T_N: 0.05, T_NA: 0.05, T_OA: 0.12, T_S: 0.02}


def _recentre(q: np.ndarray) -> np.ndarray:
    return q - q.mean()


def f32(x):
    """Round to float32-representable float64 values.  The C ABI takes
    float32, so every real-valued input is drawn at that precision and the
    float64 copy handed to a CPU checker is bit-identical to what the GPU
    receives."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def make_receptor(natoms: int, grid: Grid, seed: int = 1, min_sep: float = 2.0,
                  pocket: float = 5.0) -> Receptor:
    """Pseudo-receptor: a Gaussian blob (sigma = box/4) around the box centre
    with a spherical empty pocket of radius `pocket` and a minimum atom
    separation `min_sep` (rejection sampling on a cell hash)."""
    rng = np.random.default_rng(seed)
    c = np.asarray(grid.center)
    sig = grid.extent[0] / 4.0
    pts = np.zeros((natoms, 3))
    cells: dict = {}
    count = 0
    sep2 = min_sep * min_sep
    while count < natoms:
        cand = rng.normal(c, sig, size=(256, 3))
        for x in cand:
            if count >= natoms:
                break
            if np.sum((x - c) ** 2) < pocket * pocket:
                continue
            k = np.floor(x / min_sep).astype(int)
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for j in cells.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                            d = pts[j] - x
                            if d @ d < sep2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                cells.setdefault((k[0], k[1], k[2]), []).append(count)
                pts[count] = x
                count += 1
    types = rng.choice(NTYPES, size=natoms, p=RECEPTOR_TYPE_FREQ / RECEPTOR_TYPE_FREQ.sum())
    q = _recentre(rng.normal(0.0, 0.2, size=natoms))
    return Receptor(f32(pts), types.astype(np.int32), f32(q))


@dataclass
class Ligand:
    xyz: np.ndarray        # (n, 3) reference conformation, float64
    type: np.ndarray       # (n,) int32 map index
    charge: np.ndarray     # (n,) float64, net zero
    bonds: np.ndarray      # (nb, 2) int32
    tors: np.ndarray       # (T, 2) int32 rotatable bonds (a, b), any orientation
    root: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def natoms(self):
        return len(self.type)

    @property
    def ntors(self):
        return len(self.tors)


_MAXDEG = {T_C: 4, T_A: 3, T_N: 3, T_NA: 2, T_OA: 2, T_S: 2, T_HD: 1}


_COS100 = math.cos(math.radians(100.0))


def _unit(rng):
    v = rng.normal(size=3)
    return v / math.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])


def make_ligand(n_heavy: int, n_tors: int, seed: int, n_hd: int | None = None,
                max_tries: int = 200) -> Ligand:
    """Random acyclic drug-like ligand.

    Heavy atoms are grown one by one from a random parent with free valence,
    bond length U(1.40, 1.54) A, bond angles of at least 100 deg at the
    parent (about tetrahedral) and no contact closer than 2.0 A to any other
    atom.  Polar hydrogens (HD, 1.0 A) go on N/OA atoms (ceil(heavy/10) by
    default).  `n_tors` rotatable bonds are drawn uniformly among bonds whose
    two atoms both have another heavy neighbour.  Charges ~ N(0, 0.2),
    re-centred to net zero.
    """
    rng = np.random.default_rng(seed)
    if n_hd is None:
        n_hd = int(math.ceil(n_heavy / 10))
    heavy_types = np.array(list(LIGAND_HEAVY_FREQ.keys()))
    heavy_p = np.array(list(LIGAND_HEAVY_FREQ.values()))
    heavy_p = heavy_p / heavy_p.sum()
    for _attempt in range(max_tries):
        types = [int(rng.choice(heavy_types, p=heavy_p))]
        # make sure there are enough donor sites for the polar hydrogens
        xyz = [np.zeros(3)]
        X = np.zeros((n_heavy + n_hd, 3))  # the same coordinates as one array (distance checks)
        nbr = [[]]

        dirs = {}  # atom -> unit vectors to its bonded neighbours (dropped when a bond is added)

        def bond_dirs(i):
            u = dirs.get(i)
            if u is None:
                v = X[nbr[i]] - X[i]
                u = dirs[i] = v / np.sqrt((v * v).sum(axis=1))[:, None]
            return u

        failed = False
        for a in range(1, n_heavy):
            t = int(rng.choice(heavy_types, p=heavy_p))
            placed = False
            cand = [i for i in range(a) if len(nbr[i]) < _MAXDEG[types[i]]]
            for _ in range(400):
                if not cand:
                    break
                p = cand[int(rng.integers(0, len(cand)))]
                d = _unit(rng)
                if len(nbr[p]) and (bond_dirs(p) @ d > _COS100).any():
                    continue
                x = xyz[p] + d * rng.uniform(1.40, 1.54)
                r = np.sqrt(((X[:a] - x) ** 2).sum(axis=1))
                r[p] = np.inf
                if (r < 2.0).any():
                    continue
                xyz.append(x)
                X[a] = x
                nbr.append([p])
                nbr[p].append(a)
                dirs.pop(p, None)
                types.append(t)
                placed = True
                break
            if not placed:
                failed = True
                break
        if failed:
            continue
        # polar hydrogens on N / OA atoms with free valence; convert carbons if needed
        sites = [i for i in range(n_heavy) if types[i] in (T_N, T_OA) and len(nbr[i]) < _MAXDEG[types[i]]]
        if len(sites) < n_hd:
            extra = [i for i in range(n_heavy) if types[i] in (T_C, T_A) and len(nbr[i]) <= 2
                     and i not in sites]
            rng.shuffle(extra)
            for i in extra[: n_hd - len(sites)]:
                types[i] = T_OA if len(nbr[i]) <= 1 else T_N
                sites.append(i)
        if len(sites) < n_hd:
            continue
        hd_sites = rng.choice(sites, size=n_hd, replace=False)
        for s in hd_sites:
            s = int(s)
            placed = False
            for _ in range(400):
                d = _unit(rng)
                if len(nbr[s]) and (bond_dirs(s) @ d > _COS100).any():
                    continue
                x = xyz[s] + d * 1.0
                r = np.sqrt(((X[:len(xyz)] - x) ** 2).sum(axis=1))
                r[s] = np.inf
                if (r < 1.6).any():
                    continue
                X[len(xyz)] = x
                xyz.append(x)
                nbr.append([s])
                nbr[s].append(len(xyz) - 1)
                dirs.pop(s, None)
                types.append(T_HD)
                placed = True
                break
            if not placed:
                failed = True
                break
        if failed:
            continue
        n = len(types)
        bonds = np.array([(i, j) for i in range(n) for j in nbr[i] if i < j], dtype=np.int32)
        heavy_deg = [sum(1 for j in nbr[i] if types[j] != T_HD) for i in range(n)]
        cand = [(i, j) for (i, j) in bonds.tolist()
                if types[i] != T_HD and types[j] != T_HD and heavy_deg[i] >= 2 and heavy_deg[j] >= 2]
        if len(cand) < n_tors:
            continue
        pick = rng.choice(len(cand), size=n_tors, replace=False) if n_tors else np.zeros(0, int)
        tors = np.array([cand[k] for k in sorted(pick.tolist())], dtype=np.int32).reshape(-1, 2)
        q = _recentre(rng.normal(0.0, 0.2, size=n))
        xyz = np.array(xyz)
        xyz -= xyz.mean(axis=0)
        return Ligand(f32(xyz), np.array(types, dtype=np.int32), f32(q), bonds, tors, 0,
                      dict(n_heavy=n_heavy, n_hd=n_hd, seed=seed))
    raise RuntimeError(f"could not grow ligand n_heavy={n_heavy} n_tors={n_tors} seed={seed}")


def random_genes(lig: Ligand, npose: int, grid: Grid, seed: int, spread: float = 0.35) -> np.ndarray:
    """Random genotypes [t(3), q(4) (w, x, y, z), theta(T)] for parity tests.

    t is uniform in a cube of half-width `spread` x box half-extent around the
    box centre, q uniform on S^3 (Shoemake's three-uniform recipe), theta
    uniform in [-pi, pi).  float64; callers cast as needed.
    """
    rng = np.random.default_rng(seed)
    T = lig.ntors
    g = np.zeros((npose, 7 + T))
    c = np.asarray(grid.center)
    half = np.asarray(grid.extent) * 0.5 * spread
    g[:, 0:3] = c + rng.uniform(-1, 1, size=(npose, 3)) * half
    u1, u2, u3 = rng.uniform(size=(3, npose))
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    g[:, 3] = b * np.cos(2 * np.pi * u3)
    g[:, 4] = a * np.sin(2 * np.pi * u2)
    g[:, 5] = a * np.cos(2 * np.pi * u2)
    g[:, 6] = b * np.sin(2 * np.pi * u3)
    g[:, 7:] = rng.uniform(-np.pi, np.pi, size=(npose, T))
    return g


# Named workloads -----------------------------------------------------------

PLAIN = dict(name="plain", grid_n=40, rec_atoms=600, pocket_frac=0.45, n_heavy=16, n_hd=2, n_tors=3,
             nrun=10, pop=150, nev=50_000, ls="sw")
PAPER = dict(name="paper-scale", grid_n=64, rec_atoms=3000, pocket_frac=0.40, n_heavy=40, n_hd=4, n_tors=8,
             nrun=100, pop=150, nev=2_500_000, ls="adadelta")
RECEPTOR_SEED = 1
LIGAND_SEED0 = 1000
SEARCH_SEED = 42


def workload_inputs(w: dict, lig_index: int = 0):
    grid = make_grid(w["grid_n"])
    rec = make_receptor(w["rec_atoms"], grid, RECEPTOR_SEED, pocket=w["pocket_frac"] * grid.extent[0])
    lig = make_ligand(w["n_heavy"], w["n_tors"], LIGAND_SEED0 + lig_index, n_hd=w["n_hd"])
    return grid, rec, lig


def _grow(job):
    """Ligand k of a batch: the most torsions <= nt that a grown tree offers."""
    nh, nt, lseed = job
    for t in range(nt, -1, -1):
        try:
            return make_ligand(nh, t, lseed)
        except RuntimeError:
            continue
    return None


def make_batch(n: int, seed: int, heavy=(10, 60), tors=(0, 15), workers: int | None = None):
    """Seeded batch of drug-like ligands with heavy atoms uniform in `heavy`
    and torsions uniform in `tors` (clipped to the rotatable bonds a grown
    tree offers).  Ligand k depends only on (seed, k), so a batch can be
    grown by a pool of `workers` processes (0: the host's cores) with the
    same result as one process; the pool is started with "spawn", so the
    calling script needs the usual `if __name__ == "__main__":` guard."""
    rng = np.random.default_rng(seed)
    if workers is None:
        workers = 1
    elif workers == 0:
        workers = min(os.cpu_count() or 1, 32)
    out = []
    k = 0
    pool = None
    try:
        while len(out) < n:
            need = n - len(out)
            jobs = []
            for _ in range(need):
                nh = int(rng.integers(heavy[0], heavy[1] + 1))
                nt = int(rng.integers(tors[0], tors[1] + 1))
                jobs.append((nh, nt, seed * 100003 + k))
                k += 1
            if workers > 1 and len(jobs) >= 2 * workers:
                if pool is None:
                    import multiprocessing as mp
                    from concurrent.futures import ProcessPoolExecutor
                    pool = ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))
                grown = list(pool.map(_grow, jobs, chunksize=max(1, len(jobs) // (4 * workers))))
            else:
                grown = [_grow(j) for j in jobs]
            out.extend(g for g in grown if g is not None)
    finally:
        if pool is not None:
            pool.shutdown()
    return out[:n]

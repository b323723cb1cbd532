"""FP64 CPU oracle for the docking hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library (``paper_2007_03678_gb300``)
never imports, links or calls it, and shares no code with it: the oracle is
plain C in ``adg_oracle.c`` (double precision, written from the published
definitions the paper cites), loaded here with ctypes.

Parity pins (tests/test_oracle_*.py) check it against closed forms,
invariants, library special cases and brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NTYPES = 7
NMAPS = 9
MAXATOMS = 128
MAXTORS = 16
MAXGENES = 7 + MAXTORS


def build(force: bool = False) -> str:
    """Compile adg_oracle.c into liboracle.so with the host C compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


# ---------------------------------------------------------------- structs
class FF(C.Structure):
    _fields_ = [(n, C.c_double * NTYPES) for n in
                ("Rii", "epsii", "vol", "solpar", "hb_donor", "hb_acceptor", "hb_R", "hb_eps")] + \
               [(n, C.c_double) for n in
                ("w_vdw", "w_hb", "w_elec", "w_desolv", "w_tors", "qasp", "sigma", "coulomb",
                 "ms_A", "ms_eps0", "ms_lambda", "ms_k", "r_min", "e_cap", "map_r_on", "map_r_off", "k_out")]


class GRID(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("origin", C.c_double * 3), ("spacing", C.c_double)]


class PARAMS(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("nrun", "pop_size", "nev", "max_gen", "ls_method", "ls_max_iters", "elitism")] + \
               [(n, C.c_double) for n in ("ls_rate", "crossover_rate", "mutation_rate", "tournament_rate",
                                          "sw_rho0", "sw_rho_min", "sw_expand", "sw_contract")] + \
               [("sw_succ", C.c_int), ("sw_fail", C.c_int)] + \
               [(n, C.c_double) for n in ("sw_scale_t", "sw_scale_rot", "sw_scale_tors", "ad_rho", "ad_eps",
                                          "mut_t", "mut_rot", "mut_tors")] + \
               [("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32), ("lig_id", C.c_uint32), ("autostop", C.c_int),
                ("stopstd", C.c_double)]


TRACE_WIDTH = 12  # parent1, parent2, xlo, xhi, mut_mask, ls_applied, a1, b1, a2, b2, 0, 0


class TRACE(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("parent1", "parent2", "xlo", "xhi", "mut_mask", "ls_applied",
                                         "a1", "b1", "a2", "b2", "pad0", "pad1")]


class RUNRES(C.Structure):
    _fields_ = [("best_energy", C.c_double), ("best_genes", C.c_double * MAXGENES),
                ("evals", C.c_longlong), ("generations", C.c_int), ("pad", C.c_int)]


_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_vp = C.c_void_p


def _declare(L):
    L.orc_philox_batch.argtypes = [_u, C.c_int, C.c_uint32, C.c_uint32, _u]
    L.orc_pair_lj.argtypes = [C.POINTER(FF), C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double)]
    L.orc_pair_lj.restype = C.c_double
    L.orc_pair_elec.argtypes = [C.POINTER(FF), C.c_double, C.c_double, C.POINTER(C.c_double)]
    L.orc_pair_elec.restype = C.c_double
    L.orc_pair_desolv.argtypes = [C.POINTER(FF), C.c_int, C.c_double, C.c_int, C.c_double, C.c_double,
                                  C.POINTER(C.c_double)]
    L.orc_pair_desolv.restype = C.c_double
    L.orc_map_switch.argtypes = [C.POINTER(FF), C.c_double]
    L.orc_map_switch.restype = C.c_double
    L.orc_map_point.argtypes = [C.POINTER(FF), _d, C.c_int, _d, _i, _d, _d]
    L.orc_maps_build.argtypes = [C.POINTER(FF), C.POINTER(GRID), C.c_int, _d, _i, _d, _d]
    L.orc_trilinear.argtypes = [C.POINTER(GRID), _d, _d, _d]
    L.orc_trilinear.restype = C.c_double
    L.orc_out_of_box.argtypes = [C.POINTER(GRID), _d, C.c_double, _d]
    L.orc_out_of_box.restype = C.c_double
    L.orc_ligand_sizeof.restype = C.c_size_t
    L.orc_ligand_init.argtypes = [_vp, C.c_int, _d, _i, _d, C.c_int, _i, C.c_int, _i, C.c_int]
    L.orc_ligand_npairs.argtypes = [_vp]
    L.orc_ligand_pairs.argtypes = [_vp, _i]
    L.orc_ligand_moving.argtypes = [_vp, _u8]
    L.orc_ligand_torsions.argtypes = [_vp, _i]
    L.orc_quat_to_matrix.argtypes = [_d, _d]
    L.orc_pose_batch.argtypes = [_vp, _d, C.c_int, _d]
    L.orc_score_batch.argtypes = [C.POINTER(FF), C.POINTER(GRID), _d, _vp, _d, C.c_int, _d, _d, _d, _d]
    L.orc_atom_gradients.argtypes = [C.POINTER(FF), C.POINTER(GRID), _d, _vp, _d, C.c_int, _d]
    L.orc_apply_step.argtypes = [C.c_int, _d, _d, C.c_double, _d]
    L.orc_local_search.argtypes = [C.POINTER(FF), C.POINTER(GRID), _d, _vp, C.POINTER(PARAMS), C.c_int,
                                   C.c_int, C.c_int, _d, C.POINTER(C.c_double)]
    L.orc_local_search.restype = C.c_longlong
    L.orc_lga_run.argtypes = [C.POINTER(FF), C.POINTER(GRID), _d, _vp, C.POINTER(PARAMS), C.c_int,
                              C.POINTER(RUNRES), C.c_int, _vp, _vp, _vp]
    L.orc_init_population.argtypes = [C.POINTER(GRID), C.POINTER(PARAMS), C.c_int, C.c_int, _d]
    L.orc_score_xyz.argtypes = [C.POINTER(FF), C.POINTER(GRID), _d, _vp, _d, C.c_int, _d, _d, _vp]
    L.orc_solis_wets_trace.argtypes = [C.POINTER(FF), C.POINTER(GRID), _d, _vp, C.POINTER(PARAMS), C.c_int,
                                       C.c_int, C.c_int, _d, C.POINTER(C.c_double), _d,
                                       C.POINTER(C.c_longlong)]
    L.orc_solis_wets_trace.restype = C.c_int
    L.orc_make_offspring.argtypes = [C.POINTER(PARAMS), C.c_int, C.c_int, C.c_int, C.c_int, _d, _d, _d,
                                     C.POINTER(TRACE)]


# ---------------------------------------------------------------- helpers
def make_ff(ff: dict) -> FF:
    s = FF()
    for name in ("Rii", "epsii", "vol", "solpar", "hb_donor", "hb_acceptor", "hb_R", "hb_eps"):
        arr = getattr(s, name)
        for t in range(NTYPES):
            arr[t] = float(ff[name][t])
    for name, _ in FF._fields_[8:]:
        setattr(s, name, float(ff[name]))
    return s


def make_grid(grid) -> GRID:
    g = GRID()
    for a in range(3):
        g.n[a] = int(grid.n[a])
        g.origin[a] = float(grid.origin[a])
    g.spacing = float(grid.spacing)
    return g


@dataclass
class SearchParams:
    """Search parameters (names after the paper's nrun / nev, Sec. 1.1; the
    defaults are readings -- the paper only says 'other parameters default')."""
    nrun: int = 10
    pop_size: int = 150
    nev: int = 50_000
    max_gen: int = 27_000
    ls_method: int = 1          # 0 none, 1 Solis-Wets, 2 ADADELTA
    ls_max_iters: int = 300
    elitism: int = 1
    ls_rate: float = 1.0
    crossover_rate: float = 0.8
    mutation_rate: float = 0.02
    tournament_rate: float = 0.6
    sw_rho0: float = 1.0
    sw_rho_min: float = 0.01
    sw_expand: float = 2.0
    sw_contract: float = 0.5
    sw_succ: int = 4
    sw_fail: int = 4
    sw_scale_t: float = 1.0
    sw_scale_rot: float = 0.5
    sw_scale_tors: float = 0.5
    ad_rho: float = 0.8
    ad_eps: float = 0.01
    mut_t: float = 2.0
    mut_rot: float = np.pi / 2
    mut_tors: float = np.pi / 2
    seed: int = 42
    lig_id: int = 0
    autostop: int = 0
    stopstd: float = 0.15

    def to_c(self) -> PARAMS:
        p = PARAMS()
        for f in fields(self):
            if f.name == "seed":
                continue
            setattr(p, f.name, getattr(self, f.name))
        p.seed_lo = self.seed & 0xFFFFFFFF
        p.seed_hi = (self.seed >> 32) & 0xFFFFFFFF
        return p


class Ligand:
    """Oracle-side ligand topology built from the raw description."""

    def __init__(self, lig):
        L = lib()
        self._buf = C.create_string_buffer(L.orc_ligand_sizeof())
        self.ptr = C.cast(self._buf, C.c_void_p)
        xyz = np.ascontiguousarray(lig.xyz, dtype=np.float64).reshape(-1)
        rc = L.orc_ligand_init(self.ptr, int(lig.natoms), xyz, np.ascontiguousarray(lig.type, np.int32),
                               np.ascontiguousarray(lig.charge, np.float64), int(len(lig.bonds)),
                               np.ascontiguousarray(lig.bonds, np.int32).reshape(-1), int(lig.ntors),
                               np.ascontiguousarray(lig.tors, np.int32).reshape(-1), int(lig.root))
        if rc != 0:
            raise ValueError(f"oracle rejected ligand (rc={rc})")
        self.natoms = int(lig.natoms)
        self.ntors = int(lig.ntors)

    @property
    def npairs(self):
        return lib().orc_ligand_npairs(self.ptr)

    def pairs(self):
        out = np.zeros(2 * self.npairs, np.int32)
        lib().orc_ligand_pairs(self.ptr, out)
        return out.reshape(-1, 2)

    def moving(self):
        out = np.zeros(self.ntors * self.natoms, np.uint8)
        lib().orc_ligand_moving(self.ptr, out)
        return out.reshape(self.ntors, self.natoms).astype(bool)

    def torsions(self):
        out = np.zeros(2 * self.ntors, np.int32)
        lib().orc_ligand_torsions(self.ptr, out)
        return out.reshape(-1, 2)


# ---------------------------------------------------------------- API
def philox(ctr: np.ndarray, key0: int, key1: int) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1)
    out = np.zeros_like(ctr)
    lib().orc_philox_batch(ctr, len(ctr) // 4, key0, key1, out)
    return out.reshape(-1, 4)


def pair_lj(ff, ti, tj, r):
    d = C.c_double()
    e = lib().orc_pair_lj(C.byref(make_ff(ff)), ti, tj, r, C.byref(d))
    return e, d.value


def pair_elec(ff, qiqj, r):
    d = C.c_double()
    e = lib().orc_pair_elec(C.byref(make_ff(ff)), qiqj, r, C.byref(d))
    return e, d.value


def pair_desolv(ff, ti, qi, tj, qj, r):
    d = C.c_double()
    e = lib().orc_pair_desolv(C.byref(make_ff(ff)), ti, qi, tj, qj, r, C.byref(d))
    return e, d.value


def map_switch(ff, r):
    return lib().orc_map_switch(C.byref(make_ff(ff)), r)


def map_point(ff, p, rec):
    out = np.zeros(NMAPS)
    lib().orc_map_point(C.byref(make_ff(ff)), np.ascontiguousarray(p, np.float64), len(rec.type),
                        np.ascontiguousarray(rec.xyz, np.float64).reshape(-1),
                        np.ascontiguousarray(rec.type, np.int32), np.ascontiguousarray(rec.charge, np.float64), out)
    return out


def maps_build(ff, grid, rec) -> np.ndarray:
    nx, ny, nz = grid.n
    out = np.zeros(NMAPS * nx * ny * nz)
    lib().orc_maps_build(C.byref(make_ff(ff)), C.byref(make_grid(grid)), len(rec.type),
                         np.ascontiguousarray(rec.xyz, np.float64).reshape(-1),
                         np.ascontiguousarray(rec.type, np.int32), np.ascontiguousarray(rec.charge, np.float64), out)
    return out.reshape(NMAPS, nz, ny, nx)


def trilinear(grid, map3d, p):
    g = np.zeros(3)
    v = lib().orc_trilinear(C.byref(make_grid(grid)), np.ascontiguousarray(map3d, np.float64).reshape(-1),
                            np.ascontiguousarray(p, np.float64), g)
    return v, g


def out_of_box(grid, p, k):
    g = np.zeros(3)
    v = lib().orc_out_of_box(C.byref(make_grid(grid)), np.ascontiguousarray(p, np.float64), k, g)
    return v, g


def quat_to_matrix(q):
    R = np.zeros(9)
    lib().orc_quat_to_matrix(np.ascontiguousarray(q, np.float64), R)
    return R.reshape(3, 3)


def pose(L: Ligand, genes: np.ndarray) -> np.ndarray:
    genes = np.ascontiguousarray(np.atleast_2d(genes), np.float64)
    out = np.zeros((genes.shape[0], L.natoms, 3))
    lib().orc_pose_batch(L.ptr, genes, genes.shape[0], out)
    return out


def score(ff, grid, maps, L: Ligand, genes: np.ndarray):
    """Energies, intermolecular energies, gene gradients, tangent gradients."""
    genes = np.ascontiguousarray(np.atleast_2d(genes), np.float64)
    n = genes.shape[0]
    G, D = 7 + L.ntors, 6 + L.ntors
    e = np.zeros(n)
    ei = np.zeros(n)
    gg = np.zeros((n, G))
    gt = np.zeros((n, D))
    lib().orc_score_batch(C.byref(make_ff(ff)), C.byref(make_grid(grid)),
                          np.ascontiguousarray(maps, np.float64).reshape(-1), L.ptr, genes, n, e, ei, gg, gt)
    return e, ei, gg, gt


def score_xyz(ff, grid, maps, L: Ligand, xyz: np.ndarray, forces: bool = False):
    """Energies (total, intermolecular) of posed coordinates xyz[npose, natoms, 3]
    given directly, and with forces=True the per-atom gradients too."""
    xyz = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, L.natoms, 3))
    n = xyz.shape[0]
    e = np.zeros(n)
    ei = np.zeros(n)
    f = np.zeros((n, L.natoms, 3)) if forces else None
    lib().orc_score_xyz(C.byref(make_ff(ff)), C.byref(make_grid(grid)),
                        np.ascontiguousarray(maps, np.float64).reshape(-1), L.ptr, xyz, n, e, ei,
                        f.ctypes.data if forces else None)
    return (e, ei, f) if forces else (e, ei)


def atom_gradients(ff, grid, maps, L: Ligand, genes: np.ndarray) -> np.ndarray:
    """dE/dx'_i per atom: [npose, natoms, 3]."""
    genes = np.ascontiguousarray(np.atleast_2d(genes), np.float64)
    out = np.zeros((genes.shape[0], L.natoms, 3))
    lib().orc_atom_gradients(C.byref(make_ff(ff)), C.byref(make_grid(grid)),
                             np.ascontiguousarray(maps, np.float64).reshape(-1), L.ptr, genes, genes.shape[0], out)
    return out


def apply_step(ntors, genes, xi, sign=1.0):
    out = np.zeros(7 + ntors)
    lib().orc_apply_step(ntors, np.ascontiguousarray(genes, np.float64), np.ascontiguousarray(xi, np.float64),
                         sign, out)
    return out


def local_search(ff, grid, maps, L, params: SearchParams, genes, energy, run=0, ind=0, gen=1):
    g = np.ascontiguousarray(genes, np.float64).copy()
    e = C.c_double(energy)
    n = lib().orc_local_search(C.byref(make_ff(ff)), C.byref(make_grid(grid)),
                               np.ascontiguousarray(maps, np.float64).reshape(-1), L.ptr, C.byref(params.to_c()),
                               run, ind, gen, g, C.byref(e))
    return g, e.value, n


SW_TRACE_WIDTH = 3 + 2 * MAXGENES


def solis_wets_trace(ff, grid, maps, L, params: SearchParams, genes, energy, run=0, ind=0, gen=1):
    """Solis-Wets on one genotype with its trace.  Returns (genes, energy,
    evaluations, trace) where trace has one row per iteration: rho, outcome
    (+1 / -1 / 0), energy after it, xi[D], bias after it[D]."""
    g = np.ascontiguousarray(genes, np.float64).copy()
    e = C.c_double(energy)
    nev = C.c_longlong(0)
    D = 6 + L.ntors
    buf = np.zeros((max(params.ls_max_iters, 1), SW_TRACE_WIDTH))
    it = lib().orc_solis_wets_trace(C.byref(make_ff(ff)), C.byref(make_grid(grid)),
                                    np.ascontiguousarray(maps, np.float64).reshape(-1), L.ptr,
                                    C.byref(params.to_c()), run, ind, gen, g, C.byref(e), buf, C.byref(nev))
    t = buf[:it]
    trace = dict(rho=t[:, 0].copy(), outcome=t[:, 1].astype(int), energy=t[:, 2].copy(),
                 xi=t[:, 3:3 + D].copy(), bias=t[:, 3 + MAXGENES:3 + MAXGENES + D].copy())
    return g, e.value, nev.value, trace


def make_offspring(params: SearchParams, ntors, pop_genes, pop_energy, run=0, ind=1, gen=1):
    """One offspring of the GA (selection, two-point crossover, mutation).
    Returns (child genes, decisions dict)."""
    G = 7 + ntors
    Pg = np.ascontiguousarray(pop_genes, np.float64).reshape(-1, G)
    Pe = np.ascontiguousarray(pop_energy, np.float64).reshape(-1)
    child = np.zeros(G)
    tr = TRACE()
    lib().orc_make_offspring(C.byref(params.to_c()), ntors, run, ind, gen, Pg, Pe, child, C.byref(tr))
    dec = {f: getattr(tr, f) for f, _ in TRACE._fields_}
    return child, dec


def init_population(grid, params: SearchParams, ntors, run=0):
    out = np.zeros((params.pop_size, 7 + ntors))
    lib().orc_init_population(C.byref(make_grid(grid)), C.byref(params.to_c()), ntors, run, out)
    return out


def lga_run(ff, grid, maps, L, params: SearchParams, run=0, ntrace=0):
    """One LGA run.  Returns (best_energy, best_genes, evals, generations,
    trace or None) where trace = (decisions[ntrace, pop] structured array,
    genes[ntrace, pop, G], energies[ntrace, pop])."""
    res = RUNRES()
    pop, G = params.pop_size, 7 + L.ntors
    tr = (TRACE * (max(ntrace, 1) * pop))()
    tg = np.zeros((max(ntrace, 1), pop, G))
    te = np.zeros((max(ntrace, 1), pop))
    mp = np.ascontiguousarray(maps, np.float64).reshape(-1)
    rc = lib().orc_lga_run(C.byref(make_ff(ff)), C.byref(make_grid(grid)), mp, L.ptr, C.byref(params.to_c()),
                           run, C.byref(res), ntrace, C.cast(tr, C.c_void_p) if ntrace else None,
                           tg.ctypes.data if ntrace else None, te.ctypes.data if ntrace else None)
    if rc != 0:
        raise ValueError(f"oracle lga_run failed rc={rc}")
    trace = None
    if ntrace:
        dec = np.frombuffer(tr, dtype=np.int32).reshape(ntrace, pop, TRACE_WIDTH).copy()
        trace = (dec, tg[:ntrace], te[:ntrace])
    return res.best_energy, np.array(res.best_genes[:G]), res.evals, res.generations, trace

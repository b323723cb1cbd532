"""Shared set-up for the GPU parity tests: seeded problems, oracle maps and
the tolerances the parity tests hold the CUDA path to."""
import functools

import numpy as np

import oracle as O
from paper_2007_03678_gb300 import synth as S

# Tolerances (per pose): energy |E_gpu - E_ref| <= E_ABS + E_REL |E_ref|;
# gradient |g_gpu - g_ref| <= G_REL * max(|g_ref|_inf, 1) per component.
E_ABS = 1e-3
E_REL = 1e-5
G_REL = 1e-3
# Genotype-level comparisons only: FP32 rounding of a posed coordinate moves
# the energy by up to COORD_EPS * sum_i |dE/dx_i|_1.  A posed coordinate
# (|x| <= 16 A, one ulp 9.5e-7 A) comes out of a product of up to 12 nested
# torsion transforms and the rigid-body transform, each adding about one
# ulp: 1e-5 A bounds it.  The scoring itself is held to the plain tolerance
# above at the CUDA path's own posed coordinates (strict_at_gpu_coords), for
# every non-clashing pose (inside the box, E < 1e3).
COORD_EPS = 1e-5
F_WELL = 50.0


@functools.lru_cache(maxsize=None)
def problem(name: str):
    """(grid, receptor, ligand, oracle maps float64 from the float32 maps, maps float32)."""
    w = {"plain": S.PLAIN, "paper": S.PAPER}[name]
    grid, rec, lig = S.workload_inputs(w)
    ff = S.forcefield()
    maps32 = O.maps_build(ff, grid, rec).astype(np.float32)
    return grid, rec, lig, maps32.astype(np.float64), maps32


def energy_ok(e_gpu, e_ref):
    return np.abs(e_gpu - e_ref) <= E_ABS + E_REL * np.abs(e_ref)


def energy_tol(e_ref, forces):
    return E_ABS + E_REL * np.abs(e_ref) + COORD_EPS * np.abs(forces).sum(axis=(1, 2))


def well_conditioned(forces):
    return np.abs(forces).max(axis=(1, 2)) <= F_WELL


def grad_ok(g_gpu, g_ref):
    scale = np.maximum(np.abs(g_ref).max(axis=1, keepdims=True), 1.0)
    return np.abs(g_gpu - g_ref) <= G_REL * scale


def near_face(grid, xyz, delta=1e-4):
    """Poses with an atom within `delta` grid units of a cell face."""
    u = (xyz - np.asarray(grid.origin)) / grid.spacing
    f = u - np.floor(u)
    return (np.minimum(f, 1 - f) < delta).any(axis=(1, 2))


def inside_box(grid, xyz):
    lo = np.asarray(grid.origin)
    hi = lo + np.asarray(grid.extent)
    return ((xyz >= lo) & (xyz <= hi)).all(axis=(1, 2))


@functools.lru_cache(maxsize=None)
def ga_problem():
    """A well-conditioned variant of the plain problem for replaying GA
    decisions: the maps saturated smoothly at +-20 kcal/mol (20 tanh(M/20))
    and the pair cap lowered to 50, so population energies are O(100) and
    FP32 and FP64 order them alike.  Both sides receive these inputs."""
    grid, rec, lig, maps64, maps32 = problem("plain")
    sm32 = (20.0 * np.tanh(maps64 / 20.0)).astype(np.float32)
    ff = dict(S.forcefield(), e_cap=50.0)
    return grid, lig, sm32.astype(np.float64), sm32, ff


def near_tie(energies, factor=2.0):
    """True when two different energies of one population lie within
    `factor` x the energy tolerance of each other."""
    for pop in energies:
        s = np.sort(np.asarray(pop, np.float64))
        d = np.diff(s)
        tol = E_ABS + E_REL * np.abs(s[1:])
        if ((d > 0) & (d < factor * tol)).any():
            return True
    return False


def gpu_coords_energy(ctx, A, ff, grid, maps64, Lg, OL, genes32):
    """The oracle's FP64 energy of the CUDA path's own FP32 posed coordinates
    (adg_pose), and those coordinates."""
    import torch
    xyz = A.pose(ctx, Lg, torch.from_numpy(np.ascontiguousarray(genes32)).cuda())
    ctx.sync()
    xyz = xyz.cpu().numpy().astype(np.float64)
    return O.score_xyz(ff, grid, maps64, OL, xyz)[0], xyz


def strict_at_gpu_coords(ctx, A, ff, grid, maps64, Lg, OL, genes32, e_gpu):
    """Hold the scoring to the plain tolerance E_ABS + E_REL |E| against the
    oracle's energy of the same FP32 coordinates, for every non-clashing pose
    (all atoms inside the box, E < 1e3).  Returns (clean mask, ok mask,
    reference energies at the GPU coordinates)."""
    e_ref, xyz = gpu_coords_energy(ctx, A, ff, grid, maps64, Lg, OL, genes32)
    clean = inside_box(grid, xyz) & (e_ref < 1e3)
    ok = np.abs(np.asarray(e_gpu, np.float64) - e_ref) <= E_ABS + E_REL * np.abs(e_ref)
    return clean, ok, e_ref

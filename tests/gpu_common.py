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

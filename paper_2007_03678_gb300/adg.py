"""Thin Python binding of libadg.so (include/adg.h), same names as the C ABI.

Only argument marshalling lives here: every step of the docking hot path
runs in the CUDA library.  PyTorch provides device memory and streams.
There is no CPU fallback: if libadg.so is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import synth

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libadg.so")

NTYPES = 7
NMAPS = 9
MAX_ATOMS = 128
MAX_TORS = 16
MAX_GENES = 7 + MAX_TORS
TRACE_WIDTH = 12

ADG_OK = 0
GRAD_NONE, GRAD_GENES, GRAD_TANGENT = 0, 1, 2
LS_NONE, LS_SOLIS_WETS, LS_ADADELTA = 0, 1, 2
GEO_HEURISTIC, GEO_TUNED = 0, 1
MLP_MMA_SYNC, MLP_TCGEN05 = 0, 1
NDESC = 16


class AdgError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        msg = f"{what}: {strerror(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


# ---------------------------------------------------------------- structs
class adg_forcefield(C.Structure):
    _fields_ = [("Rii", C.c_float * NTYPES), ("epsii", C.c_float * NTYPES), ("vol", C.c_float * NTYPES),
                ("solpar", C.c_float * NTYPES), ("hb_donor", C.c_int32 * NTYPES),
                ("hb_acceptor", C.c_int32 * NTYPES), ("hb_R", C.c_float * NTYPES), ("hb_eps", C.c_float * NTYPES)] + \
               [(n, C.c_float) for n in ("w_vdw", "w_hb", "w_elec", "w_desolv", "w_tors", "qasp", "sigma", "coulomb",
                                         "ms_A", "ms_eps0", "ms_lambda", "ms_k", "r_min", "e_cap", "map_r_on",
                                         "map_r_off", "k_out")]


class adg_grid_desc(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("origin", C.c_float * 3), ("spacing", C.c_float)]


class adg_ligand_desc(C.Structure):
    _fields_ = [("natoms", C.c_int32), ("xyz", C.POINTER(C.c_float)), ("type", C.POINTER(C.c_int32)),
                ("charge", C.POINTER(C.c_float)), ("nbonds", C.c_int32), ("bonds", C.POINTER(C.c_int32)),
                ("ntors", C.c_int32), ("tors", C.POINTER(C.c_int32)), ("root", C.c_int32)]


class adg_search_params(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("nrun", "pop_size", "nev", "max_gen", "ls_method", "ls_max_iters",
                                         "elitism")] + \
               [(n, C.c_float) for n in ("ls_rate", "crossover_rate", "mutation_rate", "tournament_rate", "sw_rho0",
                                         "sw_rho_min", "sw_expand", "sw_contract")] + \
               [("sw_succ", C.c_int32), ("sw_fail", C.c_int32)] + \
               [(n, C.c_float) for n in ("sw_scale_t", "sw_scale_rot", "sw_scale_tors", "ad_rho", "ad_eps", "mut_t",
                                         "mut_rot", "mut_tors")] + \
               [("seed", C.c_uint64), ("lig_id", C.c_uint32), ("autostop", C.c_int32), ("stopstd", C.c_float),
                ("pad0", C.c_int32)]


class adg_result(C.Structure):
    _fields_ = [("best_energy", C.c_float), ("generations", C.c_int32), ("evals", C.c_int64),
                ("genes", C.c_float * MAX_GENES), ("xyz", C.c_float * (3 * MAX_ATOMS))]


class adg_dock_trace(C.Structure):
    _fields_ = [("ngen", C.c_int32), ("decisions", C.POINTER(C.c_int32)), ("genes", C.POINTER(C.c_float)),
                ("energies", C.POINTER(C.c_float)), ("init_genes", C.POINTER(C.c_float)),
                ("init_energies", C.POINTER(C.c_float))]


class adg_stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("gen_launches", C.c_int64), ("gen_kernel_ms", C.c_double),
                ("gen_timed", C.c_int64), ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64),
                ("dock_groups", C.c_int64), ("tune_launches", C.c_int64)]


class adg_tuned_shape(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("apl", "ls_method", "nslots_max", "bytes_max", "staged", "warps_per_block",
                                         "blocks_per_sm", "ncand")] + [("us_per_eval", C.c_float * 2)]


class adg_ligand_stats(C.Structure):
    _fields_ = [("natoms", C.c_int32), ("ntors", C.c_int32), ("npairs", C.c_int32), ("sum_moving", C.c_int32),
                ("device_bytes", C.c_int64)]


class adg_schedule_stats(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("natoms", "npairs", "nsteps", "gsteps", "empty_slots", "pair_wavefronts",
                                         "pair_wavefronts_ideal", "gather_wavefronts", "gather_wavefronts_ideal")]


class adg_peaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("fp32_scalar_tflops", C.c_double), ("fp32x2_tflops", C.c_double),
                ("mufu_gops", C.c_double), ("mufu_rsqrt_gops", C.c_double), ("l2_gather_gbs", C.c_double), ("gather_bytes", C.c_int64),
                ("sms", C.c_int32), ("sm_clock_mhz", C.c_int32)]


# The full exported symbol list of include/adg.h.
EXPORTS = ("adg_strerror", "adg_search_params_default", "adg_ctx_create", "adg_ctx_destroy", "adg_sync",
           "adg_ctx_last_error", "adg_maps_build", "adg_receptor_create", "adg_receptor_destroy", "adg_ligand_create",
           "adg_ligand_destroy", "adg_ligand_info", "adg_score", "adg_pose", "adg_dock", "adg_philox",
           "adg_ctx_set_timing", "adg_ctx_stats", "adg_dock_noalloc", "adg_ctx_set_geometry", "adg_ctx_tuned",
           "adg_dock_traced", "adg_ligand_descriptors", "adg_mlp_nparams", "adg_mlp_create", "adg_mlp_destroy",
           "adg_mlp_get_params", "adg_mlp_set_params", "adg_mlp_set_norm", "adg_mlp_forward", "adg_mlp_grad",
           "adg_mlp_train_step", "adg_mlp_fit", "adg_ligand_set_stream_id",
           "adg_ctx_set_graphs", "adg_mlp_set_engine", "adg_mlp_check", "adg_probe_peaks", "adg_ligand_schedule", "adg_score_multi",
           "adg_mlp_set_wait_ns")

_lib = None


def load(path: str | None = None):
    """Load libadg.so (or the build named by $ADG_LIBRARY).  Raises if it has
    not been built."""
    global _lib
    if _lib is None:
        path = path or os.environ.get("ADG_LIBRARY") or LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2007_03678_gb300.build`")
        L = C.CDLL(path)
        _vp, _i, _f = C.c_void_p, C.c_int, C.c_float
        L.adg_strerror.restype = C.c_char_p
        L.adg_strerror.argtypes = [_i]
        L.adg_search_params_default.argtypes = [C.POINTER(adg_search_params)]
        L.adg_search_params_default.restype = None
        L.adg_ctx_create.argtypes = [C.POINTER(_vp), _i, _vp]
        L.adg_ctx_destroy.argtypes = [_vp]
        L.adg_sync.argtypes = [_vp]
        L.adg_ctx_last_error.argtypes = [_vp]
        L.adg_ctx_last_error.restype = C.c_char_p
        L.adg_maps_build.argtypes = [_vp, C.POINTER(adg_forcefield), C.POINTER(adg_grid_desc), _i, _vp, _vp, _vp,
                                     _vp]
        L.adg_receptor_create.argtypes = [_vp, C.POINTER(adg_grid_desc), _vp, _i, C.POINTER(_vp)]
        L.adg_receptor_destroy.argtypes = [_vp]
        L.adg_ligand_create.argtypes = [_vp, C.POINTER(adg_forcefield), C.POINTER(adg_ligand_desc), C.POINTER(_vp)]
        L.adg_ligand_destroy.argtypes = [_vp]
        L.adg_ligand_info.argtypes = [_vp, C.POINTER(adg_ligand_stats)]
        L.adg_score.argtypes = [_vp, _vp, _vp, _vp, _i, _vp, _vp, _i]
        L.adg_score_multi.argtypes = [_vp, _vp, C.POINTER(_vp), _i, C.POINTER(C.c_int), _vp, _vp, _vp, _i]
        L.adg_pose.argtypes = [_vp, _vp, _vp, _i, _vp]
        L.adg_dock.argtypes = [_vp, _vp, C.POINTER(_vp), _i, C.POINTER(adg_search_params), C.POINTER(adg_result),
                               C.POINTER(adg_dock_trace)]
        L.adg_philox.argtypes = [_vp, _vp, _i, C.c_uint64, _vp]
        L.adg_ctx_set_timing.argtypes = [_vp, _i]
        L.adg_dock_noalloc.argtypes = [_vp, _vp, C.POINTER(adg_search_params), C.POINTER(adg_result), _vp]
        L.adg_ctx_stats.argtypes = [_vp, C.POINTER(adg_stats), _i]
        L.adg_ctx_set_geometry.argtypes = [_vp, _i]
        L.adg_ctx_set_graphs.argtypes = [_vp, _i]
        L.adg_dock_traced.argtypes = [_vp, _vp, C.POINTER(_vp), _i, C.POINTER(adg_search_params),
                                      C.POINTER(adg_result), C.POINTER(C.c_float), _i]
        L.adg_ligand_descriptors.argtypes = [_vp, C.POINTER(C.c_float)]
        L.adg_ligand_set_stream_id.argtypes = [_vp, C.c_int64]
        _fp = C.POINTER(C.c_float)
        L.adg_mlp_nparams.argtypes = [_i]
        L.adg_mlp_create.argtypes = [_vp, _i, C.c_uint64, C.POINTER(_vp)]
        L.adg_mlp_destroy.argtypes = [_vp]
        L.adg_mlp_get_params.argtypes = [_vp, _vp, _fp]
        L.adg_mlp_set_params.argtypes = [_vp, _vp, _fp]
        L.adg_mlp_set_norm.argtypes = [_vp, _fp, _fp, C.c_float, C.c_float]
        L.adg_mlp_forward.argtypes = [_vp, _vp, _vp, _i, _vp]
        L.adg_mlp_grad.argtypes = [_vp, _vp, _vp, _vp, _vp, _i, _vp, _vp]
        L.adg_mlp_train_step.argtypes = [_vp, _vp, _vp, _vp, _vp, _i, C.c_float, _vp]
        L.adg_mlp_fit.argtypes = [_vp, _vp, _vp, _vp, _i, _i, _i, C.c_float, C.c_uint64, _fp]
        L.adg_mlp_set_engine.argtypes = [_vp, _i]
        L.adg_mlp_check.argtypes = [_vp, _vp]
        L.adg_mlp_set_wait_ns.argtypes = [_vp, C.c_longlong]
        L.adg_ctx_tuned.argtypes = [_vp, C.POINTER(adg_tuned_shape), _i, C.POINTER(C.c_int)]
        L.adg_probe_peaks.argtypes = [_vp, C.POINTER(adg_peaks)]
        L.adg_ligand_schedule.argtypes = [C.POINTER(adg_forcefield), C.POINTER(adg_ligand_desc),
                                          C.POINTER(adg_schedule_stats)]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return load().adg_strerror(code).decode()
    except Exception:  # library missing: still format the error
        return "error"


def _check(rc: int, what: str, ctx=None):
    if rc != ADG_OK:
        detail = ""
        if ctx is not None and ctx.handle:
            detail = load().adg_ctx_last_error(ctx.handle).decode()
        raise AdgError(rc, what, detail)


def _ptr(t) -> int:
    """Device pointer of a CUDA tensor (checked contiguous, on a GPU)."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


# ---------------------------------------------------------------- helpers
def forcefield_struct(ff: dict) -> adg_forcefield:
    s = adg_forcefield()
    for name in ("Rii", "epsii", "vol", "solpar", "hb_R", "hb_eps"):
        arr = getattr(s, name)
        for t in range(NTYPES):
            arr[t] = float(ff[name][t])
    for name in ("hb_donor", "hb_acceptor"):
        arr = getattr(s, name)
        for t in range(NTYPES):
            arr[t] = int(ff[name][t])
    for name, _ in adg_forcefield._fields_[8:]:
        setattr(s, name, float(ff[name]))
    return s


def grid_struct(grid) -> adg_grid_desc:
    g = adg_grid_desc()
    for a in range(3):
        g.n[a] = int(grid.n[a])
        g.origin[a] = float(grid.origin[a])
    g.spacing = float(grid.spacing)
    return g


def search_params(**kw) -> adg_search_params:
    p = adg_search_params()
    load().adg_search_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- objects
class Context:
    """adg_ctx_create / adg_ctx_destroy on a torch.cuda.Stream (a new one when
    `stream` is None).  Calls that take device tensors order the context's
    stream after the caller's current stream on entry, and the current stream
    after the context's stream on exit, so tensors are safe to use on either
    side without a host synchronisation."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        L = load()
        if stream is None:
            stream = torch.cuda.Stream(device=device)
        h = C.c_void_p()
        _check(L.adg_ctx_create(C.byref(h), device, C.c_void_p(stream.cuda_stream)), "adg_ctx_create")
        self.handle = h
        self.device = device
        self.stream = stream

    def _enter(self):
        import torch
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _leave(self):
        import torch
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def sync(self):
        _check(load().adg_sync(self.handle), "adg_sync", self)

    def set_timing(self, enable: bool):
        _check(load().adg_ctx_set_timing(self.handle, int(enable)), "adg_ctx_set_timing", self)

    def set_graphs(self, enable: bool):
        """Generation loop of dock as device-side graph loops (default) or host launches."""
        _check(load().adg_ctx_set_graphs(self.handle, int(enable)), "adg_ctx_set_graphs", self)

    def set_geometry(self, mode: int):
        """GEO_HEURISTIC or GEO_TUNED (default) launch geometry for dock."""
        _check(load().adg_ctx_set_geometry(self.handle, int(mode)), "adg_ctx_set_geometry", self)

    def tuned(self) -> list:
        """The context's tuning table: one dict per shape bucket."""
        n = C.c_int(0)
        _check(load().adg_ctx_tuned(self.handle, None, 0, C.byref(n)), "adg_ctx_tuned", self)
        buf = (adg_tuned_shape * max(n.value, 1))()
        _check(load().adg_ctx_tuned(self.handle, buf, n.value, C.byref(n)), "adg_ctx_tuned", self)
        out = []
        for t in buf[:n.value]:
            d = {name: getattr(t, name) for name, _ in adg_tuned_shape._fields_[:-1]}
            d["us_per_eval"] = [float(t.us_per_eval[0]), float(t.us_per_eval[1])]
            out.append(d)
        return out

    def stats(self, reset: bool = False) -> dict:
        st = adg_stats()
        _check(load().adg_ctx_stats(self.handle, C.byref(st), int(reset)), "adg_ctx_stats", self)
        return {name: getattr(st, name) for name, _ in adg_stats._fields_}

    def close(self):
        if self.handle:
            load().adg_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def maps_build(ctx: Context, ff: dict, grid, rec: "synth.Receptor"):
    """adg_maps_build -> torch float32 tensor [9, nz, ny, nx] on the device."""
    import torch
    nx, ny, nz = grid.n
    out = torch.empty((NMAPS, nz, ny, nx), dtype=torch.float32, device=f"cuda:{ctx.device}")
    xyz = np.ascontiguousarray(rec.xyz, np.float32)
    typ = np.ascontiguousarray(rec.type, np.int32)
    q = np.ascontiguousarray(rec.charge, np.float32)
    ffs, gs = forcefield_struct(ff), grid_struct(grid)
    ctx._enter()
    _check(load().adg_maps_build(ctx.handle, C.byref(ffs), C.byref(gs), len(typ), xyz.ctypes.data, typ.ctypes.data,
                                 q.ctypes.data, _ptr(out)), "adg_maps_build", ctx)
    ctx._leave()
    return out


class Receptor:
    """adg_receptor_create: maps [9][nz][ny][nx] float32 (numpy host array or CUDA tensor)."""

    def __init__(self, ctx: Context, grid, maps):
        self.ctx = ctx
        self.grid = grid
        gs = grid_struct(grid)
        h = C.c_void_p()
        if isinstance(maps, np.ndarray):
            m = np.ascontiguousarray(maps, np.float32)
            rc = load().adg_receptor_create(ctx.handle, C.byref(gs), m.ctypes.data, 0, C.byref(h))
        else:
            ctx._enter()
            rc = load().adg_receptor_create(ctx.handle, C.byref(gs), _ptr(maps), 1, C.byref(h))
        _check(rc, "adg_receptor_create", ctx)
        self.handle = h

    def close(self):
        if self.handle:
            load().adg_receptor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ligand_desc(lig):
    """adg_ligand_desc of a synth.Ligand-like object, and the arrays it points
    into (keep them alive while the descriptor is used)."""
    xyz = np.ascontiguousarray(lig.xyz, np.float32).reshape(-1)
    typ = np.ascontiguousarray(lig.type, np.int32)
    q = np.ascontiguousarray(lig.charge, np.float32)
    bonds = np.ascontiguousarray(lig.bonds, np.int32).reshape(-1)
    tors = np.ascontiguousarray(lig.tors, np.int32).reshape(-1)
    d = adg_ligand_desc()
    d.natoms = len(typ)
    d.xyz = xyz.ctypes.data_as(C.POINTER(C.c_float))
    d.type = typ.ctypes.data_as(C.POINTER(C.c_int32))
    d.charge = q.ctypes.data_as(C.POINTER(C.c_float))
    d.nbonds = len(bonds) // 2
    d.bonds = bonds.ctypes.data_as(C.POINTER(C.c_int32))
    d.ntors = len(tors) // 2
    d.tors = tors.ctypes.data_as(C.POINTER(C.c_int32))
    d.root = int(lig.root)
    return d, (xyz, typ, q, bonds, tors)


def ligand_schedule(ff: dict, lig) -> dict:
    """adg_ligand_schedule: the pair-loop and force-gather schedule the library
    builds for `lig`, with its modelled shared-memory wavefronts per
    energy+gradient evaluation (host only, no GPU)."""
    d, _keep = ligand_desc(lig)
    ffs = forcefield_struct(ff)
    out = adg_schedule_stats()
    _check(load().adg_ligand_schedule(C.byref(ffs), C.byref(d), C.byref(out)), "adg_ligand_schedule")
    return {f: getattr(out, f) for f, _ in adg_schedule_stats._fields_}


class Ligand:
    """adg_ligand_create from a synth.Ligand-like object (xyz, type, charge, bonds, tors, root)."""

    def __init__(self, ctx: Context, ff: dict, lig):
        self.ctx = ctx
        d, _keep = ligand_desc(lig)
        ffs = forcefield_struct(ff)
        h = C.c_void_p()
        _check(load().adg_ligand_create(ctx.handle, C.byref(ffs), C.byref(d), C.byref(h)), "adg_ligand_create", ctx)
        self.handle = h
        st = adg_ligand_stats()
        _check(load().adg_ligand_info(h, C.byref(st)), "adg_ligand_info", ctx)
        self.natoms, self.ntors, self.npairs = st.natoms, st.ntors, st.npairs
        self.sum_moving, self.device_bytes = st.sum_moving, st.device_bytes
        self.stream_id = None

    def set_stream_id(self, sid: int):
        """adg_ligand_set_stream_id: fixed Philox ligand word (-1: index-based default)."""
        _check(load().adg_ligand_set_stream_id(self.handle, int(sid)), "adg_ligand_set_stream_id")
        self.stream_id = None if sid < 0 else int(sid)

    def descriptors(self) -> np.ndarray:
        """adg_ligand_descriptors: [NDESC] float32."""
        out = np.zeros(NDESC, np.float32)
        _check(load().adg_ligand_descriptors(self.handle, out.ctypes.data_as(C.POINTER(C.c_float))),
               "adg_ligand_descriptors")
        return out

    def close(self):
        if self.handle:
            load().adg_ligand_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def score(ctx: Context, rec: Receptor, lig: Ligand, genes, grad_kind: int = GRAD_NONE, energy=None, grad=None):
    """adg_score on CUDA tensors.  genes: float32 [npose, 7+T] on the device.
    Returns (energy [npose], grad or None); outputs may be passed in."""
    import torch
    n = genes.shape[0]
    if energy is None:
        energy = torch.empty(n, dtype=torch.float32, device=genes.device)
    if grad_kind != GRAD_NONE and grad is None:
        width = 7 + lig.ntors if grad_kind == GRAD_GENES else 6 + lig.ntors
        grad = torch.empty((n, width), dtype=torch.float32, device=genes.device)
    ctx._enter()
    _check(load().adg_score(ctx.handle, rec.handle, lig.handle, _ptr(genes), n, _ptr(energy),
                            _ptr(grad) if grad is not None else None, grad_kind), "adg_score", ctx)
    ctx._leave()
    return energy, grad


def score_multi(ctx: Context, rec: Receptor, ligs, genes, npose, grad_kind: int = GRAD_NONE):
    """adg_score_multi: genes float32 [sum(npose), MAX_GENES] on the device,
    ligand i owning npose[i] consecutive rows (its 7+T genes in front).
    Returns (energy [total], grad [total, MAX_GENES] or None)."""
    import torch
    n = len(ligs)
    counts = (C.c_int * n)(*[int(k) for k in npose])
    total = int(sum(int(k) for k in npose))
    if genes.shape != (total, MAX_GENES) or genes.dtype != torch.float32:
        raise ValueError(f"genes must be float32 [{total}, {MAX_GENES}]")
    energy = torch.empty(total, dtype=torch.float32, device=genes.device)
    grad = None
    if grad_kind != GRAD_NONE:  # every column is written (zeros past the ligand's genes)
        grad = torch.empty((total, MAX_GENES), dtype=torch.float32, device=genes.device)
    hs = (C.c_void_p * n)(*[l.handle.value for l in ligs])
    ctx._enter()
    _check(load().adg_score_multi(ctx.handle, rec.handle, hs, n, counts, _ptr(genes), _ptr(energy),
                                  _ptr(grad) if grad is not None else None, grad_kind), "adg_score_multi", ctx)
    ctx._leave()
    return energy, grad


def pose(ctx: Context, lig: Ligand, genes):
    import torch
    n = genes.shape[0]
    xyz = torch.empty((n, lig.natoms, 3), dtype=torch.float32, device=genes.device)
    ctx._enter()
    _check(load().adg_pose(ctx.handle, lig.handle, _ptr(genes), n, _ptr(xyz)), "adg_pose", ctx)
    ctx._leave()
    return xyz


def philox(ctx: Context, ctr, key: int):
    """ctr: uint32-compatible int32 CUDA tensor [n, 4] -> same shape output."""
    import torch
    out = torch.empty_like(ctr)
    ctx._enter()
    _check(load().adg_philox(ctx.handle, _ptr(ctr), ctr.shape[0], key, _ptr(out)), "adg_philox", ctx)
    ctx._leave()
    return out


def probe_peaks(ctx: Context) -> dict:
    """Measured FP32 (TFLOP/s), special-function (G results/s) and L2 random
    gather (GB/s) throughput of the context's GPU (adg_probe_peaks)."""
    out = adg_peaks()
    ctx._enter()
    _check(load().adg_probe_peaks(ctx.handle, C.byref(out)), "adg_probe_peaks", ctx)
    ctx._leave()
    return {f: getattr(out, f) for f, _ in adg_peaks._fields_}


def _result_dtype():
    f = adg_result
    return np.dtype({"names": ["best_energy", "generations", "evals", "genes", "xyz"],
                     "formats": [np.float32, np.int32, np.int64, (np.float32, MAX_GENES), (np.float32, 3 * MAX_ATOMS)],
                     "offsets": [f.best_energy.offset, f.generations.offset, f.evals.offset, f.genes.offset,
                                 f.xyz.offset],
                     "itemsize": C.sizeof(adg_result)})


def dock(ctx: Context, rec: Receptor, ligs, params: adg_search_params, trace_ngen: int = 0, best_trace: int = 0):
    """adg_dock (adg_dock_traced when best_trace > 0).  Returns a list (per
    ligand) of dicts with arrays over runs: best_energy [nrun], genes
    [nrun, 7+T], xyz [nrun, natoms, 3], evals, generations, and best_trace
    [nrun, best_trace] when asked; plus a trace dict when trace_ngen > 0 (one
    ligand only)."""
    if isinstance(ligs, Ligand):
        ligs = [ligs]
    n = len(ligs)
    nrun, pop = params.nrun, params.pop_size
    res = (adg_result * (n * nrun))()
    hs = (C.c_void_p * n)(*[l.handle.value for l in ligs])
    tr = None
    trace = None
    if trace_ngen > 0 and best_trace > 0:
        raise ValueError("trace_ngen and best_trace are exclusive")
    if trace_ngen > 0:
        G = 7 + ligs[0].ntors
        dec = np.zeros((nrun, trace_ngen, pop, TRACE_WIDTH), np.int32)
        tg = np.zeros((nrun, trace_ngen, pop, G), np.float32)
        te = np.zeros((nrun, trace_ngen, pop), np.float32)
        ig = np.zeros((nrun, pop, G), np.float32)
        ie = np.zeros((nrun, pop), np.float32)
        tr = adg_dock_trace()
        tr.ngen = trace_ngen
        tr.decisions = dec.ctypes.data_as(C.POINTER(C.c_int32))
        tr.genes = tg.ctypes.data_as(C.POINTER(C.c_float))
        tr.energies = te.ctypes.data_as(C.POINTER(C.c_float))
        tr.init_genes = ig.ctypes.data_as(C.POINTER(C.c_float))
        tr.init_energies = ie.ctypes.data_as(C.POINTER(C.c_float))
        trace = dict(decisions=dec, genes=tg, energies=te, init_genes=ig, init_energies=ie)
    bt = None
    if best_trace > 0:
        bt = np.zeros((n, nrun, best_trace), np.float32)
        _check(load().adg_dock_traced(ctx.handle, rec.handle, hs, n, C.byref(params), res,
                                      bt.ctypes.data_as(C.POINTER(C.c_float)), int(best_trace)),
               "adg_dock_traced", ctx)
    else:
        _check(load().adg_dock(ctx.handle, rec.handle, hs, n, C.byref(params), res,
                               C.byref(tr) if tr is not None else None), "adg_dock", ctx)
    rec_arr = np.frombuffer(res, dtype=_result_dtype()).reshape(n, nrun)
    out = []
    for li, lig in enumerate(ligs):
        G, N = 7 + lig.ntors, lig.natoms
        r = rec_arr[li]
        d = dict(best_energy=r["best_energy"].copy(), genes=r["genes"][:, :G].copy(),
                 xyz=r["xyz"][:, :3 * N].reshape(nrun, N, 3).copy(), evals=r["evals"].copy(),
                 generations=r["generations"].copy())
        if bt is not None:
            d["best_trace"] = bt[li]
        out.append(d)
    return (out, trace) if trace_ngen > 0 else out


def dock_noalloc(rec: Receptor, lig: Ligand, params: adg_search_params, stream=None):
    """adg_dock_noalloc: dock one ligand without any allocation by the library
    (for callers whose memory the library may not allocate; see include/adg.h).
    Returns the same per-run dict as dock() for one ligand."""
    nrun = params.nrun
    res = (adg_result * nrun)()
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(load().adg_dock_noalloc(rec.handle, lig.handle, C.byref(params), res, sp), "adg_dock_noalloc")
    G, N = 7 + lig.ntors, lig.natoms
    return dict(best_energy=np.array([r.best_energy for r in res], np.float32),
                genes=np.array([r.genes[:G] for r in res], np.float32),
                xyz=np.array([r.xyz[:3 * N] for r in res], np.float32).reshape(nrun, N, 3),
                evals=np.array([r.evals for r in res], np.int64),
                generations=np.array([r.generations for r in res], np.int32))


class MLP:
    """The triage network (adg_mlp_*): nin -> 256 -> 256 -> 1, ReLU, BF16
    weights with FP32 accumulation, trained by Adam.  Tensors are CUDA
    float32 (PyTorch supplies the memory; every step runs in libadg.so)."""

    HIDDEN = 256
    NIN_MAX = 32

    def __init__(self, ctx: Context, nin: int, seed: int = 0):
        self.ctx = ctx
        self.nin = int(nin)
        h = C.c_void_p()
        _check(load().adg_mlp_create(ctx.handle, self.nin, int(seed), C.byref(h)), "adg_mlp_create", ctx)
        self.handle = h
        self.nparams = load().adg_mlp_nparams(self.nin)

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparams, np.float32)
        _check(load().adg_mlp_get_params(self.ctx.handle, self.handle, out.ctypes.data_as(C.POINTER(C.c_float))),
               "adg_mlp_get_params", self.ctx)
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, np.float32)
        if th.size != self.nparams:
            raise ValueError("expected %d parameters" % self.nparams)
        _check(load().adg_mlp_set_params(self.ctx.handle, self.handle, th.ctypes.data_as(C.POINTER(C.c_float))),
               "adg_mlp_set_params", self.ctx)

    def set_norm(self, mu, sigma, mu_y: float, sigma_y: float):
        m = np.ascontiguousarray(mu, np.float32)
        sg = np.ascontiguousarray(sigma, np.float32)
        _check(load().adg_mlp_set_norm(self.handle, m.ctypes.data_as(C.POINTER(C.c_float)),
                                       sg.ctypes.data_as(C.POINTER(C.c_float)), float(mu_y), float(sigma_y)),
               "adg_mlp_set_norm")

    def set_engine(self, engine: int):
        """MLP_TCGEN05 (default) or MLP_MMA_SYNC for forward()."""
        _check(load().adg_mlp_set_engine(self.handle, int(engine)), "adg_mlp_set_engine")

    def set_wait_ns(self, ns: int):
        """Bound of each wait of the tcgen05 forward on its MMAs (ns; 0: no waiting)."""
        _check(load().adg_mlp_set_wait_ns(self.handle, int(ns)), "adg_mlp_set_wait_ns")

    def check(self):
        """Raise if a bounded wait of the tcgen05 forward expired (synchronous)."""
        _check(load().adg_mlp_check(self.ctx.handle, self.handle), "adg_mlp_check", self.ctx)

    def forward(self, x):
        import torch
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        self.ctx._enter()
        _check(load().adg_mlp_forward(self.ctx.handle, self.handle, _ptr(x), x.shape[0], _ptr(y)),
               "adg_mlp_forward", self.ctx)
        self.ctx._leave()
        return y

    def grad(self, x, t, idx=None):
        """(gradient [nparams] CUDA tensor, loss CUDA scalar) of the batch loss."""
        import torch
        g = torch.empty(self.nparams, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        n = x.shape[0] if idx is None else idx.shape[0]
        self.ctx._enter()
        _check(load().adg_mlp_grad(self.ctx.handle, self.handle, _ptr(x), _ptr(t),
                                   _ptr(idx) if idx is not None else None, n, _ptr(g), _ptr(loss)),
               "adg_mlp_grad", self.ctx)
        self.ctx._leave()
        return g, loss

    def train_step(self, x, t, lr: float, idx=None):
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        n = x.shape[0] if idx is None else idx.shape[0]
        self.ctx._enter()
        _check(load().adg_mlp_train_step(self.ctx.handle, self.handle, _ptr(x), _ptr(t),
                                         _ptr(idx) if idx is not None else None, n, float(lr), _ptr(loss)),
               "adg_mlp_train_step", self.ctx)
        self.ctx._leave()
        return loss

    def fit(self, x, t, batch: int, epochs: int, lr: float, seed: int = 0) -> np.ndarray:
        out = np.zeros(max(epochs, 1), np.float32)
        self.ctx._enter()
        _check(load().adg_mlp_fit(self.ctx.handle, self.handle, _ptr(x), _ptr(t), x.shape[0], int(batch), int(epochs),
                                  float(lr), int(seed), out.ctypes.data_as(C.POINTER(C.c_float))),
               "adg_mlp_fit", self.ctx)
        return out[:epochs]

    def close(self):
        if self.handle:
            load().adg_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

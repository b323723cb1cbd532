"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Run on a GB300: python -m pytest tests -m gpu."""
import numpy as np
import pytest

import oracle as O
from paper_2007_03678_gb300 import synth as S

from gpu_common import (E_ABS, E_REL, energy_ok, energy_tol, grad_ok, inside_box, near_face, problem,
                        strict_at_gpu_coords, well_conditioned)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03678_gb300 import adg, build
    build.build()
    c = adg.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def A():
    from paper_2007_03678_gb300 import adg
    return adg


def _cuda(x, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ------------------------------------------------------------------ Philox
def test_philox_bit_exact(ctx, A):
    import torch
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = 0x9E3779B97F4A7C15
    want = O.philox(ctr, key & 0xFFFFFFFF, key >> 32)
    got = A.philox(ctx, _cuda(ctr.view(np.int32)), key)
    ctx.sync()
    got = got.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want)


# ------------------------------------------------------------------ maps
def test_maps_build_matches_oracle_plain(ctx, A, ff):
    grid, rec, lig, maps64, maps32 = problem("plain")
    g = A.maps_build(ctx, ff, grid, rec)
    ctx.sync()
    g = g.cpu().numpy().astype(np.float64)
    ref = O.maps_build(ff, grid, rec)
    err = np.abs(g - ref)
    tol = 2e-3 + 1e-5 * np.abs(ref)
    assert (err <= tol).all(), f"max err {err.max()} at {np.unravel_index(err.argmax(), err.shape)}"


def test_maps_build_matches_oracle_paper_scale_sampled(ctx, A, ff):
    grid, rec, lig, maps64, maps32 = problem("paper")
    g = A.maps_build(ctx, ff, grid, rec)
    ctx.sync()
    g = g.cpu().numpy().astype(np.float64)
    # full oracle maps are in problem(); also re-check 500 nodes point by point
    err = np.abs(g - maps64)
    tol = 2e-3 + 1e-5 * np.abs(maps64)
    if not (err <= tol).all():
        worst = np.argsort(-(err / tol).ravel())[:5]
        rows = [(np.unravel_index(w, err.shape), g.ravel()[w], maps64.ravel()[w]) for w in worst]
        raise AssertionError(f"{(err > tol).sum()} nodes off; worst (map,z,y,x), gpu, oracle: {rows}")
    rng = np.random.default_rng(1)
    nx, ny, nz = grid.n
    for _ in range(500):
        i, j, k = rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz)
        p = np.array(grid.origin) + grid.spacing * np.array([i, j, k])
        ref = O.map_point(ff, p, rec)
        assert np.all(np.abs(g[:, k, j, i] - ref) <= 2e-3 + 1e-5 * np.abs(ref))


# ------------------------------------------------------------------ pose + score
def _score_both(ctx, A, ff, name, genes32, grad_kind):
    grid, rec, lig, maps64, maps32 = problem(name)
    R = A.Receptor(ctx, grid, maps32)
    Lg = A.Ligand(ctx, ff, lig)
    e, g = A.score(ctx, R, Lg, _cuda(genes32), grad_kind)
    ctx.sync()
    L = O.Ligand(lig)
    ref = O.score(ff, grid, maps64, L, genes32.astype(np.float64))
    xyz = O.pose(L, genes32.astype(np.float64))
    return e.cpu().numpy().astype(np.float64), (g.cpu().numpy().astype(np.float64) if g is not None else None), ref, xyz


@pytest.mark.parametrize("name", ["plain", "paper"])
def test_pose_matches_oracle(ctx, A, ff, name):
    grid, rec, lig, _, _ = problem(name)
    genes = S.random_genes(lig, 2048, grid, 21).astype(np.float32)
    genes[::3, 3:7] *= 2.5  # non-unit quaternions are normalised by both sides
    Lg = A.Ligand(ctx, ff, lig)
    xyz = A.pose(ctx, Lg, _cuda(genes))
    ctx.sync()
    ref = O.pose(O.Ligand(lig), genes.astype(np.float64))
    assert np.abs(xyz.cpu().numpy() - ref).max() < 2e-5


def _parity_report(e, ref_e, ok_mask, tol=None):
    err = np.abs(e - ref_e)
    tol = E_ABS + E_REL * np.abs(ref_e) if tol is None else tol
    bad = (err > tol) & ok_mask
    worst = np.argsort(-(err / tol) * ok_mask)[:5]
    rows = ", ".join(f"#{i}: gpu {e[i]:.6g} ref {ref_e[i]:.6g} tol {tol[i]:.3g}" for i in worst)
    return f"{bad.sum()} of {ok_mask.sum()} poses off; worst {rows}"


def _forces(ff, name, genes32):
    grid, rec, lig, maps64, _ = problem(name)
    return O.atom_gradients(ff, grid, maps64, O.Ligand(lig), genes32.astype(np.float64))


@pytest.mark.parametrize("name", ["plain", "paper"])
def test_score_energy_and_gradients_random_poses(ctx, A, ff, name):
    grid, rec, lig, maps64, _ = problem(name)
    genes = S.random_genes(lig, 8192 if name == "paper" else 4096, grid, 22, spread=0.5).astype(np.float32)
    e, gg, ref, xyz = _score_both(ctx, A, ff, name, genes, A.GRAD_GENES)
    ref_e, ref_ei, ref_gg, ref_gt = ref
    forces = _forces(ff, name, genes)
    clean = inside_box(grid, xyz) & (ref_e < 1e3)
    # every pose: the plain tolerance plus the propagation of FP32 coordinate
    # rounding through the per-atom forces (random poses sit on steep walls;
    # the docked-like test below holds well-conditioned poses to the plain one)
    tol = energy_tol(ref_e, forces)
    assert (np.abs(e - ref_e) <= tol).all(), _parity_report(e, ref_e, np.ones(len(e), bool), tol)
    well = clean & well_conditioned(forces)
    assert energy_ok(e, ref_e)[well].all(), _parity_report(e, ref_e, well)
    # the scoring alone: every non-clashing pose at the plain tolerance against
    # the oracle's energy of the CUDA path's own posed coordinates
    Lg, OL = A.Ligand(ctx, ff, lig), O.Ligand(lig)
    clean_g, ok_g, ref_g = strict_at_gpu_coords(ctx, A, ff, grid, maps64, Lg, OL, genes, e)
    assert clean_g.sum() > 50
    assert ok_g[clean_g].all(), _parity_report(e, ref_g, clean_g)
    only_widened = clean & ~energy_ok(e, ref_e)
    print(f"{name}: {clean_g.sum()} non-clashing poses meet 1e-3 + 1e-5|E| at the GPU coordinates; "
          f"{only_widened.sum()} of {clean.sum()} need the coordinate-rounding term at the genotype level")
    smooth = clean & ~near_face(grid, xyz)
    assert smooth.sum() > 0.9 * clean.sum() and smooth.sum() > 50
    ok = grad_ok(gg, ref_gg)[smooth]
    assert ok.all(), f"{(~ok).any(axis=1).sum()} poses with a gradient component off"
    e2, gt, _, _ = _score_both(ctx, A, ff, name, genes, A.GRAD_TANGENT)
    assert np.array_equal(e2, e)
    assert grad_ok(gt, ref_gt)[smooth].all()


@pytest.mark.parametrize("name", ["plain", "paper"])
def test_score_docked_like_poses(ctx, A, ff, name):
    """Low-energy poses (oracle Solis-Wets refined), where 1e-3 kcal/mol is tight."""
    grid, rec, lig, maps64, _ = problem(name)
    L = O.Ligand(lig)
    p = O.SearchParams(ls_method=1, ls_max_iters=150)
    starts = S.random_genes(lig, 48, grid, 23, spread=0.15)
    refined = []
    for i, g0 in enumerate(starts):
        e0 = O.score(ff, grid, maps64, L, g0)[0][0]
        g, e, _ = O.local_search(ff, grid, maps64, L, p, g0, e0, run=0, ind=i, gen=1)
        refined.append(g)
    genes = np.array(refined, np.float32)
    e, gg, ref, xyz = _score_both(ctx, A, ff, name, genes, A.GRAD_GENES)
    assert (ref[0] < 0).mean() >= 0.4
    assert energy_ok(e, ref[0]).all(), _parity_report(e, ref[0], np.ones(len(e), bool))
    smooth = ~near_face(grid, xyz)
    assert grad_ok(gg, ref[2])[smooth].all()


def test_score_edge_cases(ctx, A, ff):
    import torch
    grid, rec, lig, maps64, maps32 = problem("plain")
    R = A.Receptor(ctx, grid, maps32)
    # npose = 0 is a no-op
    Lg = A.Ligand(ctx, ff, lig)
    e, _ = A.score(ctx, R, Lg, torch.zeros((0, 7 + lig.ntors), device="cuda"))
    assert e.numel() == 0
    cases = []
    # rigid ligand (no torsion), one-atom ligand, a 128-atom 16-torsion ligand,
    # a 64-atom ligand (every atom index of two per lane used) and an 88-atom
    # ligand (three atoms per lane, the last lanes partly empty)
    rigid = S.make_ligand(12, 0, 77)
    one = S.Ligand(np.zeros((1, 3)), np.array([S.T_OA], np.int32), np.array([-0.3]), np.zeros((0, 2), np.int32),
                   np.zeros((0, 2), np.int32), 0)
    big = S.make_ligand(116, 16, 78, n_hd=12)
    full2 = S.make_ligand(58, 7, 81)
    three = S.make_ligand(80, 10, 79)
    assert (big.natoms, full2.natoms, three.natoms) == (128, 64, 88)
    for lg in (rigid, one, big, full2, three):
        genes = S.random_genes(lg, 700, grid, 24, spread=1.3).astype(np.float32)  # many poses leave the box
        Lg = A.Ligand(ctx, ff, lg)
        e, gt = A.score(ctx, R, Lg, _cuda(genes), A.GRAD_TANGENT)
        ctx.sync()
        L = O.Ligand(lg)
        g64 = genes.astype(np.float64)
        ref_e, ref_ei, _, ref_gt = O.score(ff, grid, maps64, L, g64)
        forces = O.atom_gradients(ff, grid, maps64, L, g64)
        xyz = O.pose(L, g64)
        e = e.cpu().numpy()
        out = ~inside_box(grid, xyz)
        assert out.sum() > 50  # the out-of-box restraint is exercised
        well = (ref_e < 1e3) & well_conditioned(forces)
        assert energy_ok(e, ref_e)[well].all(), _parity_report(e, ref_e, well)
        tol = energy_tol(ref_e, forces)
        assert (np.abs(e - ref_e) <= tol).all(), _parity_report(e, ref_e, np.ones(len(e), bool), tol)
        clean_g, ok_g, ref_g = strict_at_gpu_coords(ctx, A, ff, grid, maps64, Lg, L, genes, e)
        assert ok_g[clean_g].all(), _parity_report(e, ref_g, clean_g)
        smooth = well & ~near_face(grid, xyz)
        assert grad_ok(gt.cpu().numpy(), ref_gt)[smooth].all()


def test_host_validation_errors(ctx, A, ff):
    grid, rec, lig, maps64, maps32 = problem("plain")
    bad_type = S.Ligand(lig.xyz, np.where(np.arange(lig.natoms) == 3, 9, lig.type).astype(np.int32), lig.charge,
                        lig.bonds, lig.tors, 0)
    with pytest.raises(A.AdgError) as ei:
        A.Ligand(ctx, ff, bad_type)
    assert ei.value.code == -2
    cyc = S.Ligand(lig.xyz, lig.type, lig.charge, np.vstack([lig.bonds, [[0, lig.natoms - 1]]]).astype(np.int32),
                   lig.tors, 0)
    with pytest.raises(A.AdgError) as ei:
        A.Ligand(ctx, ff, cyc)
    assert ei.value.code == -8
    not_bond = S.Ligand(lig.xyz, lig.type, lig.charge, lig.bonds, np.array([[0, lig.natoms - 1]], np.int32), 0)
    with pytest.raises(A.AdgError):
        A.Ligand(ctx, ff, not_bond)
    big = S.make_ligand(130, 2, 5, n_hd=0)
    with pytest.raises(A.AdgError) as ei:
        A.Ligand(ctx, ff, big)
    assert ei.value.code == -3
    g = S.Grid((1, 40, 40), grid.origin, grid.spacing)
    with pytest.raises(A.AdgError) as ei:
        A.Receptor(ctx, g, maps32)
    assert ei.value.code == -4

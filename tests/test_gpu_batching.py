"""Batching: many ligands of uneven size in one adg_dock call (one graph per
atoms-per-lane shape class, classes on concurrent streams) give exactly the
results of docking each ligand alone with the same counter-based stream."""
import numpy as np
import pytest

from paper_2007_03678_gb300 import synth as S

from gpu_common import problem

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


@pytest.mark.parametrize("ls_method", [1, 2])
def test_batch_equals_one_by_one(ctx, ff, ls_method):
    from paper_2007_03678_gb300 import adg
    grid, rec, _, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    ligs = S.make_batch(12, seed=5)
    sizes = [l.natoms for l in ligs]
    assert min(sizes) <= 32 and max(sizes) > 64  # all three shape classes
    L = [adg.Ligand(ctx, ff, l) for l in ligs]
    p = adg.search_params(nrun=4, pop_size=50, nev=6000, ls_method=ls_method, ls_max_iters=25, lig_id=100, seed=9)
    batch = adg.dock(ctx, R, L, p)
    for i, lg in enumerate(L):
        q = adg.search_params(nrun=4, pop_size=50, nev=6000, ls_method=ls_method, ls_max_iters=25, lig_id=100 + i,
                              seed=9)
        alone = adg.dock(ctx, R, lg, q)[0]
        for key in ("best_energy", "genes", "xyz", "evals", "generations"):
            assert np.array_equal(batch[i][key], alone[key]), (i, key)


def test_geometry_modes_agree_and_tuning_table(ctx, ff):
    """The tuned launch geometry (per-bucket timing of staged / L1 forms,
    ligands grouped by the geometry they get) and the fixed rule give the
    same results bit for bit; every tuned bucket has a launchable choice."""
    from paper_2007_03678_gb300 import adg
    grid, rec, _, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    ligs = S.make_batch(10, seed=11) + [S.make_ligand(88, 12, 4242), S.make_ligand(110, 15, 4343)]
    sizes = [l.natoms for l in ligs]
    assert min(sizes) <= 32 and max(sizes) > 96  # atoms-per-lane widths 1 to 4
    L = [adg.Ligand(ctx, ff, l) for l in ligs]
    p = adg.search_params(nrun=3, pop_size=40, nev=3000, ls_method=adg.LS_ADADELTA, ls_max_iters=20, seed=17)
    ctx.set_geometry(adg.GEO_HEURISTIC)
    ctx.stats(reset=True)
    ref = adg.dock(ctx, R, L, p)
    assert ctx.stats()["dock_groups"] == 4
    ctx.set_geometry(adg.GEO_TUNED)
    ctx.stats(reset=True)
    got = adg.dock(ctx, R, L, p)
    st = ctx.stats()
    assert st["dock_groups"] >= 4 and st["tune_launches"] >= 0
    for i in range(len(L)):
        for key in ("best_energy", "genes", "xyz", "evals", "generations"):
            assert np.array_equal(ref[i][key], got[i][key]), (i, key)
    table = ctx.tuned()
    assert {t["apl"] for t in table} == {1, 2, 3, 4}
    for t in table:
        assert t["blocks_per_sm"] >= 1 and 1 <= t["warps_per_block"] <= 12
        if t["ncand"] == 2:
            assert min(t["us_per_eval"]) > 0
    # a second call reuses the table: nothing more is tuned
    ctx.stats(reset=True)
    adg.dock(ctx, R, L, p)
    assert ctx.stats()["tune_launches"] == 0


def test_graph_and_host_loops_agree(ctx, ff):
    """The device-side graph loop and the host-driven loop give the same runs."""
    from paper_2007_03678_gb300 import adg
    grid, rec, _, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    L = [adg.Ligand(ctx, ff, l) for l in S.make_batch(7, seed=13)]
    p = adg.search_params(nrun=3, pop_size=40, nev=9000, ls_method=adg.LS_SOLIS_WETS, ls_max_iters=30, seed=23,
                          autostop=1)
    ref = adg.dock(ctx, R, L, p, best_trace=6)
    ctx.set_graphs(False)
    try:
        got = adg.dock(ctx, R, L, p, best_trace=6)
    finally:
        ctx.set_graphs(True)
    for a, b in zip(ref, got):
        for key in ("best_energy", "genes", "xyz", "evals", "generations", "best_trace"):
            assert np.array_equal(a[key], b[key]), key


def test_run_halves_equal_one_group(ctx, ff):
    """One ligand with 8 or more runs docks as two concurrent groups of run
    halves; every run's result (and best-energy trace) equals the same run
    docked inside a single group (the ligand batched with another)."""
    from paper_2007_03678_gb300 import adg
    grid, rec, lig, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    L = adg.Ligand(ctx, ff, lig)
    other = adg.Ligand(ctx, ff, S.make_ligand(20, 3, 777))
    p = adg.search_params(nrun=9, pop_size=40, nev=4000, ls_method=adg.LS_ADADELTA, ls_max_iters=20, lig_id=300,
                          seed=5)
    ctx.stats(reset=True)
    alone = adg.dock(ctx, R, L, p, best_trace=6)[0]
    assert ctx.stats()["dock_groups"] == 2
    both = adg.dock(ctx, R, [L, other], p, best_trace=6)[0]
    for key in ("best_energy", "genes", "xyz", "evals", "generations", "best_trace"):
        assert np.array_equal(alone[key], both[key]), key


def test_batched_dock_sampled_against_oracle(ctx, ff):
    """One adg_dock call over 16 ligands that span the four atoms-per-lane
    widths (up to 32, 64, 96 and 128 atoms): for every ligand and run, the
    reported pose is the oracle's pose of the reported genotype, the reported
    best energy is the oracle's energy of that genotype (genotype-level
    tolerance), and the oracle's energy of the reported FP32 pose meets the
    plain 1e-3 + 1e-5|E| wherever the pose does not clash; every run spends
    its budget and its best-energy trace never rises."""
    import oracle as O
    from paper_2007_03678_gb300 import adg
    from gpu_common import E_ABS, E_REL, energy_tol, inside_box
    grid, rec, _, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    ligs = S.make_batch(10, seed=31) + [S.make_ligand(36, 5, 3131), S.make_ligand(60, 9, 3232),
                                        S.make_ligand(78, 11, 3333), S.make_ligand(92, 13, 3434),
                                        S.make_ligand(104, 14, 3535), S.make_ligand(116, 15, 3636, n_hd=12)]
    widths = {(l.natoms + 31) // 32 for l in ligs}
    assert widths == {1, 2, 3, 4}, widths
    L = [adg.Ligand(ctx, ff, l) for l in ligs]
    nev = 30_000
    p = adg.search_params(nrun=4, pop_size=60, nev=nev, ls_method=adg.LS_ADADELTA, ls_max_iters=30, seed=19)
    res = adg.dock(ctx, R, L, p, best_trace=8)
    clean_checked = 0
    for i, (lig, r) in enumerate(zip(ligs, res)):
        assert (r["evals"] >= nev).all() and (r["evals"] < nev + 60 * 31).all(), i
        assert np.all(np.diff(r["best_trace"], axis=1) <= 0), i
        OL = O.Ligand(lig)
        genes = r["genes"].astype(np.float64)
        assert np.abs(r["xyz"] - O.pose(OL, genes)).max() < 1e-3, i
        e_ref = O.score(ff, grid, maps64, OL, genes)[0]
        forces = O.atom_gradients(ff, grid, maps64, OL, genes)
        e = r["best_energy"].astype(np.float64)
        assert (np.abs(e - e_ref) <= energy_tol(e_ref, forces)).all(), (i, e, e_ref)
        xyz = r["xyz"].astype(np.float64)
        e_xyz = O.score_xyz(ff, grid, maps64, OL, xyz)[0]
        clean = inside_box(grid, xyz) & (e_xyz < 1e3)
        assert (np.abs(e - e_xyz) <= E_ABS + E_REL * np.abs(e_xyz))[clean].all(), (i, e, e_xyz)
        clean_checked += int(clean.sum())
    assert clean_checked >= 0.75 * 4 * len(ligs)


def test_full_batching_configuration_sampled_against_oracle(ctx, ff):
    """The full batching configuration's 4,096 ligands (the bench's seeded set,
    heavy atoms 10-60, torsions 0-15) in one adg_dock call of 20 runs x 150,
    here with one generation of ADADELTA per run instead of 1 M evaluations:
    every run spends its budget, and for a sample of ligands of every
    atoms-per-lane width each run's reported pose is the oracle's pose of the
    reported genotype and its best energy the oracle's energy of that
    genotype (genotype-level tolerance)."""
    import oracle as O
    from paper_2007_03678_gb300 import adg
    from gpu_common import energy_tol
    grid, rec, _, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    bl = S.make_batch(4096, seed=7, workers=0)
    L = [adg.Ligand(ctx, ff, l) for l in bl]
    nev = 40_000
    p = adg.search_params(nrun=20, pop_size=150, nev=nev, ls_method=adg.LS_ADADELTA, seed=S.SEARCH_SEED)
    res = adg.dock(ctx, R, L, p)
    assert len(res) == 4096
    for r in res:
        assert (r["evals"] >= nev).all() and (r["generations"] == 1).all()
    widths = np.array([(l.natoms + 31) // 32 for l in bl])
    rng = np.random.default_rng(4096)
    sample = np.concatenate([rng.choice(np.nonzero(widths == w)[0], min(8, int((widths == w).sum())), replace=False)
                             for w in np.unique(widths)])
    for i in sample:
        lig, r = bl[i], res[i]
        OL = O.Ligand(lig)
        genes = r["genes"].astype(np.float64)
        assert np.abs(r["xyz"] - O.pose(OL, genes)).max() < 1e-3, i
        e_ref = O.score(ff, grid, maps64, OL, genes)[0]
        forces = O.atom_gradients(ff, grid, maps64, OL, genes)
        assert (np.abs(r["best_energy"] - e_ref) <= energy_tol(e_ref, forces)).all(), (i, r["best_energy"], e_ref)
    for lg in L:
        lg.close()

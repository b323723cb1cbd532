"""Triage inputs and pipeline: ligand descriptors, the per-generation
best-energy trace of adg_dock_traced, and the screening pipeline of
paper_2007_03678_gb300.triage (network trained on full dockings, early
docking of a stream, full docking of the survivors only)."""
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


def test_descriptors(ctx, ff):
    from paper_2007_03678_gb300 import adg
    for seed, (nh, nt) in enumerate([(12, 2), (40, 8), (58, 15)]):
        lig = S.make_ligand(nh, nt, 7000 + seed)
        L = adg.Ligand(ctx, ff, lig)
        d = L.descriptors()
        xyz = np.asarray(lig.xyz, np.float64).reshape(-1, 3)
        q = np.asarray(lig.charge, np.float64)
        c = xyz - xyz.mean(0)
        r = np.sqrt((c * c).sum(1))
        want = np.concatenate([[lig.natoms, lig.ntors, L.npairs], np.bincount(lig.type, minlength=7),
                               [np.abs(q).sum(), (q * q).sum(), np.sqrt((r * r).mean()), r.max()]])
        assert np.allclose(d[:14], want, rtol=1e-5, atol=1e-5), (d, want)
        assert d[14] >= 1 and d[14] == lig.ntors + 1  # a tree: every rotatable bond splits off one fragment
        assert abs(d[15] - (L.sum_moving / max(lig.ntors, 1))) < 1e-5


def test_best_trace(ctx, ff):
    """Entry k of the trace is the best energy after generation k+1: non-increasing
    (elitism), ending at the run's best energy; docking with max_gen = k
    reproduces the first k entries exactly (counter-based random streams)."""
    from paper_2007_03678_gb300 import adg
    grid, rec, _, _, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    ligs = [adg.Ligand(ctx, ff, l) for l in S.make_batch(6, seed=21)]
    K = 12
    p = adg.search_params(nrun=4, pop_size=60, nev=10 ** 7, max_gen=9, ls_method=adg.LS_ADADELTA,
                          ls_max_iters=10, seed=5)
    full = adg.dock(ctx, R, ligs, p, best_trace=K)
    plain = adg.dock(ctx, R, ligs, p)
    q = adg.search_params(nrun=4, pop_size=60, nev=10 ** 7, max_gen=3, ls_method=adg.LS_ADADELTA,
                          ls_max_iters=10, seed=5)
    early = adg.dock(ctx, R, ligs, q, best_trace=3)
    for f, pl, e in zip(full, plain, early):
        tr = f["best_trace"]
        assert tr.shape == (4, K)
        assert np.all(np.diff(tr, axis=1) <= 0)
        assert np.array_equal(tr[:, -1], f["best_energy"])
        assert np.array_equal(f["best_energy"], pl["best_energy"])
        assert np.all(f["generations"] == 9)
        assert np.array_equal(e["best_trace"], tr[:, :3])
        assert np.array_equal(e["best_energy"], tr[:, 2])


def test_triage_pipeline_recall_and_gain(ctx, ff):
    """The network, trained on the plain path's own full dockings, cuts the
    search of a 2,000-ligand stream: at least 95% of the plain path's top-1%
    survive, the survivors' results are the plain path's exactly, and the
    stream costs at most 30% of the plain path's evaluations."""
    from paper_2007_03678_gb300 import adg, triage as T
    grid, rec, _, _, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    cfg = T.TriageConfig()
    LT = [adg.Ligand(ctx, ff, l) for l in S.make_batch(1200, seed=101, workers=0)]
    LS = [adg.Ligand(ctx, ff, l) for l in S.make_batch(2000, seed=202, workers=0)]
    T.assign_stream_ids(LT, 1_000_000)
    T.assign_stream_ids(LS, 2_000_000)
    y_tr, x_tr, _, _ = T.dock_full(ctx, R, LT, cfg)
    tri = T.Triage(ctx, cfg, seed=3)
    hist = tri.fit(x_tr, y_tr)
    assert np.all(hist[:, -1] < 0.5 * hist[:, 0])
    y_st, x_st, ev_plain, _ = T.dock_full(ctx, R, LS, cfg)
    out = T.screen(ctx, R, LS, tri)
    keep = out["keep"]
    assert np.array_equal(out["energy"][keep], y_st[keep])
    rec_ = T.recall(y_st, keep, cfg.top_frac)
    assert rec_ >= 0.95, (rec_, keep.mean())
    assert out["evals"] <= 0.3 * ev_plain, (out["evals"] / ev_plain, keep.mean())
    # the early features of the screen are those of the full runs' first generations
    feats, _, _ = T.dock_early(ctx, R, LS[:50], cfg)
    assert np.array_equal(feats, x_st[:50])


def test_best_trace_after_autostop_and_rigid_descriptors(ctx, ff):
    """A run that autostop ends early repeats its final best energy in the
    rest of the trace; a rigid ligand has one fragment and no moving atoms."""
    from paper_2007_03678_gb300 import adg
    grid, rec, _, _, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    L = adg.Ligand(ctx, ff, S.make_ligand(20, 3, 7100))
    K = 40
    p = adg.search_params(nrun=6, pop_size=40, nev=10 ** 7, max_gen=K, ls_method=adg.LS_SOLIS_WETS,
                          ls_max_iters=20, seed=3, autostop=1, stopstd=1.0)
    r = adg.dock(ctx, R, L, p, best_trace=K)[0]
    tr = r["best_trace"]
    assert (r["generations"] < K).any()  # autostop fired somewhere
    for run in range(6):
        g = int(r["generations"][run])
        assert np.all(tr[run, g - 1:] == r["best_energy"][run])
        assert np.all(np.diff(tr[run, :g]) <= 0)
    rigid = adg.Ligand(ctx, ff, S.make_ligand(15, 0, 7200))
    d = rigid.descriptors()
    assert d[1] == 0 and d[14] == 1 and d[15] == 0

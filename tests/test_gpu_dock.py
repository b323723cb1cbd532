"""GPU docking runs against the oracle's LGA: bit-exact GA decisions under the
shared Philox stream for the first 5 generations, evaluation accounting, and
the distribution of best energies of full runs."""
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O
from paper_2007_03678_gb300 import synth as S

from gpu_common import E_ABS, E_REL, energy_tol, ga_problem, problem

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


def _params_pair(A, **kw):
    """The same search parameters for the library (float32 struct) and the oracle."""
    op = O.SearchParams(**kw)
    ap = A.search_params(**{k: getattr(op, k) for k in (
        "nrun", "pop_size", "nev", "max_gen", "ls_method", "ls_max_iters", "elitism", "ls_rate", "crossover_rate",
        "mutation_rate", "tournament_rate", "sw_rho0", "sw_rho_min", "sw_expand", "sw_contract", "sw_succ", "sw_fail",
        "sw_scale_t", "sw_scale_rot", "sw_scale_tors", "ad_rho", "ad_eps", "mut_t", "mut_rot", "mut_tors", "seed",
        "lig_id", "autostop", "stopstd")})
    # the oracle works in double from the float32 values the library receives
    for k in ("ls_rate", "crossover_rate", "mutation_rate", "tournament_rate", "sw_rho0", "sw_rho_min", "sw_expand",
              "sw_contract", "sw_scale_t", "sw_scale_rot", "sw_scale_tors", "ad_rho", "ad_eps", "mut_t", "mut_rot",
              "mut_tors", "stopstd"):
        setattr(op, k, float(getattr(ap, k)))
    return op, ap


GA_SEED = 20200707
# decision record columns
P1, P2, XLO, XHI, MUT, LSA, A1, B1, A2, B2 = range(10)


def _tol(e):
    return E_ABS + E_REL * np.abs(e)


def _compare_generation(gd, od, prev_o, prev_g, agree):
    """Compare one generation's decisions.  Philox-only fields (candidates,
    crossover points, mutation mask, LS pick) must be bit-exact.  A
    tournament winner must match when both candidates' energies agree
    between the two sides (within tolerance) and are not a near-tie (within
    twice the tolerance of each other, where FP32 and FP64 may order them
    differently); otherwise it is counted as unresolved and must still be one
    of the two candidates.  Likewise the elite.  Returns (compared, unresolved)."""
    assert np.array_equal(gd[:, XLO:LSA + 1], od[:, XLO:LSA + 1])
    assert np.array_equal(gd[:, A1:B2 + 1], od[:, A1:B2 + 1])
    compared = unresolved = 0
    order = np.argsort(prev_o, kind="stable")
    b0, b1 = order[0], order[1]
    if agree[b0] and prev_o[b1] - prev_o[b0] > 2 * _tol(prev_o[b0]) and (prev_g >= prev_g[b0]).all():
        assert gd[0, P1] == od[0, P1]
        compared += 1
    else:
        unresolved += 1
    for i in range(1, len(od)):
        for ca, cb, col in ((A1, B1, P1), (A2, B2, P2)):
            a, b = od[i, ca], od[i, cb]
            resolvable = a == b or (agree[a] and agree[b] and
                                    abs(prev_o[a] - prev_o[b]) > 2 * _tol(min(abs(prev_o[a]), abs(prev_o[b]))))
            if resolvable:
                assert gd[i, col] == od[i, col], f"offspring {i}: winner {gd[i, col]} vs oracle {od[i, col]}"
                compared += 1
            else:
                unresolved += 1
                assert gd[i, col] in (a, b)
    return compared, unresolved


# ADADELTA from random starts is chaotic: in the oracle alone a 1e-7 change of
# the start splits a fifth of the individuals (> 2e-3 in the genes) after 12
# iterations and none after 3, so per-individual replay uses 3 iterations;
# long runs are compared by their distribution of best energies instead.  Even
# then an individual can split when two iterates tie within rounding and each
# side keeps a different one as the best; such splits are counted and bounded.
@pytest.mark.parametrize("ls_method,iters", [(0, 0), (2, 3), (1, 12)])
def test_ga_decisions_bit_exact_first_5_generations(ctx, A, ls_method, iters):
    """Generations 1-5 under the shared Philox stream: tournament candidates,
    crossover points, mutation masks and local-search picks bit-exact in every
    generation; every tournament winner and elite bit-exact unless its
    candidates are a near-tie or already differ between the two sides.  An
    individual 'agrees' when its genes and energy match the oracle's within
    tolerance; local search may split an individual off (an ADADELTA iterate
    within FP32 rounding of a map cell face sees the other side's gradient; a
    Solis-Wets trial within rounding of the current energy is accepted on one
    side only), which must stay rare.  LS off, ADADELTA and Solis-Wets."""
    grid, lig, maps64, maps32, ff = ga_problem()
    pop, ngen, nrun = 150, 5, 3
    evals_per_gen = (pop - 1) + pop * (iters if ls_method == 2 else 0)
    op, ap = _params_pair(A, nrun=nrun, pop_size=pop, ls_method=ls_method, ls_max_iters=iters, max_gen=ngen,
                          nev=10 ** 9, seed=GA_SEED)
    R = A.Receptor(ctx, grid, maps32)
    Lg = A.Ligand(ctx, ff, lig)
    res, tr = A.dock(ctx, R, Lg, ap, trace_ngen=ngen)
    L = O.Ligand(lig)
    compared = unresolved = split = total = 0
    for run in range(nrun):
        init = O.init_population(grid, op, lig.ntors, run=run)
        assert np.abs(tr["init_genes"][run] - init).max() < 1e-5
        init_e = O.score(ff, grid, maps64, L, init)[0]
        g_e = tr["init_energies"][run]
        assert (np.abs(g_e - init_e) <= _tol(init_e) + 1e-6 * np.abs(init_e)).all()
        best, bg, evals, gens, (dec, tg, te) = O.lga_run(ff, grid, maps64, L, op, run=run, ntrace=ngen)
        assert gens == ngen
        gd = tr["decisions"][run]
        prev_o, prev_g, agree = init_e, g_e, np.ones(pop, bool)
        for g in range(ngen):
            c, u = _compare_generation(gd[g], dec[g], prev_o, prev_g, agree)
            compared += c
            unresolved += u
            # which individuals still agree after this generation
            forces = O.atom_gradients(ff, grid, maps64, L, tg[g])
            e_ok = np.abs(tr["energies"][run][g] - te[g]) <= energy_tol(te[g], forces)
            q_ok = np.abs(tr["genes"][run][g] - tg[g]).max(axis=1) < 2e-3
            same_parents = (gd[g][:, P1] == dec[g][:, P1]) & (gd[g][:, P2] == dec[g][:, P2])
            parents_agree = agree[dec[g][:, P1]] & agree[dec[g][:, P2]]
            agree = e_ok & q_ok
            # with the same agreeing parents and no local search the child must agree
            if ls_method == 0:
                assert agree[same_parents & parents_agree].all()
            split += int((~agree & same_parents & parents_agree).sum())
            total += pop
            prev_o, prev_g = te[g], tr["energies"][run][g]
        if ls_method != 1:
            assert res[0]["evals"][run] == evals == pop + ngen * evals_per_gen
    stats = dict(compared=compared, unresolved=unresolved, split=split, total=total)
    limit_unres, limit_split = (0.02, 0.0) if ls_method == 0 else (0.15, 0.10)
    assert unresolved <= limit_unres * (compared + unresolved), stats
    assert split <= limit_split * total, stats


@pytest.mark.parametrize("ls_method,iters", [(0, 0), (2, 20), (1, 30)])
def test_ga_decisions_replayed_on_the_gpu_population(ctx, A, ls_method, iters):
    """Every GA decision of every generation, bit for bit: the oracle's
    offspring builder (pinned) replayed on the CUDA path's own previous
    population (its FP32 genes and energies, read exactly) must give the GPU's
    tournament candidates and winners, elites, crossover points and mutation
    masks, and the Philox local-search pick, with no near-tie exclusions --
    for the first 8 generations of three runs, LS off, ADADELTA and
    Solis-Wets (whose trajectories may differ from the oracle's own run; the
    decisions are still those of the shared stream on the same population).
    With LS off the children's genes are the oracle's children of the GPU
    parents within FP32 rounding."""
    grid, lig, maps64, maps32, ff = ga_problem()
    pop, ngen, nrun = 150, 8, 3
    op, ap = _params_pair(A, nrun=nrun, pop_size=pop, ls_method=ls_method, ls_max_iters=iters, max_gen=ngen,
                          nev=10 ** 9, seed=GA_SEED + 1, lig_id=5)
    R = A.Receptor(ctx, grid, maps32)
    Lg = A.Ligand(ctx, ff, lig)
    res, tr = A.dock(ctx, R, Lg, ap, trace_ngen=ngen)
    T = lig.ntors
    thr_ls = int(np.floor(float(ap.ls_rate) * 2 ** 24)) if ap.ls_rate < 1 else 2 ** 24
    checked = 0
    for run in range(nrun):
        Pg = tr["init_genes"][run].astype(np.float64)
        Pe = tr["init_energies"][run].astype(np.float64)
        for g in range(ngen):
            gd = tr["decisions"][run][g]
            elite = int(np.argmin(Pe))  # ties to the lower index
            assert gd[0, P1] == gd[0, P2] == elite
            for i in range(1, pop):
                child, d = O.make_offspring(op, T, Pg, Pe, run=run, ind=i, gen=g + 1)
                want = (d["parent1"], d["parent2"], d["xlo"], d["xhi"], d["mut_mask"], d["a1"], d["b1"], d["a2"],
                        d["b2"])
                got = tuple(int(v) for v in gd[i, [P1, P2, XLO, XHI, MUT, A1, B1, A2, B2]])
                assert got == want, (run, g + 1, i, got, want)
                if ls_method == 0:
                    assert np.abs(tr["genes"][run][g][i] - child).max() < 2e-6, (run, g + 1, i)
                checked += 1
            # the local-search pick: word 0 of the individual's LSPICK block
            ctr = np.array([[5, (run << 16) | i, g + 1, 4 << 20] for i in range(pop)], np.uint32)
            w = O.philox(ctr, op.seed & 0xFFFFFFFF, op.seed >> 32)[:, 0]
            want_ls = ((w >> 8) < thr_ls) if ls_method != 0 else np.zeros(pop, bool)
            assert np.array_equal(gd[:, LSA].astype(bool), want_ls)
            Pg = tr["genes"][run][g].astype(np.float64)
            Pe = tr["energies"][run][g].astype(np.float64)
    assert checked == nrun * ngen * (pop - 1)


def test_adadelta_eval_accounting(ctx, A, ff):
    grid, rec, lig, maps64, maps32 = problem("plain")
    pop, iters, nev = 150, 20, 20000
    _, ap = _params_pair(A, nrun=4, pop_size=pop, ls_method=2, ls_max_iters=iters, nev=nev)
    R = A.Receptor(ctx, grid, maps32)
    res = A.dock(ctx, R, A.Ligand(ctx, ff, lig), ap)[0]
    per_gen = (pop - 1) + pop * iters
    gens = int(np.ceil((nev - pop) / per_gen))
    assert (res["generations"] == gens).all()
    assert (res["evals"] == pop + gens * per_gen).all()


def _oracle_runs(args):
    name, runs, kw = args
    grid, rec, lig, maps64, _ = problem(name)
    ff = S.forcefield()
    L = O.Ligand(lig)
    op = O.SearchParams(**kw)
    return [O.lga_run(ff, grid, maps64, L, op, run=r)[0] for r in runs]


def test_plain_docking_distribution_matches_oracle(ctx, A, ff):
    """Plain workload (40^3 maps, 16+2 atoms, 3 torsions, Solis-Wets, 50k
    evaluations per run), 40 runs: the median best energy of the GPU runs is
    within 0.1 kcal/mol of the oracle's."""
    grid, rec, lig, maps64, maps32 = problem("plain")
    nrun = 40
    op, ap = _params_pair(A, nrun=nrun, pop_size=150, ls_method=1, nev=50_000)
    R = A.Receptor(ctx, grid, maps32)
    res = A.dock(ctx, R, A.Ligand(ctx, ff, lig), ap)[0]
    kw = {k: getattr(op, k) for k in op.__dataclass_fields__}
    chunks = [list(range(i, nrun, 8)) for i in range(8)]
    with mp.get_context("spawn").Pool(8) as pool:
        parts = pool.map(_oracle_runs, [("plain", c, kw) for c in chunks])
    ref = np.empty(nrun)
    for c, vals in zip(chunks, parts):
        ref[c] = vals
    assert (res["evals"] >= 50_000).all()
    gpu = res["best_energy"].astype(np.float64)
    assert abs(np.median(gpu) - np.median(ref)) <= 0.1, (np.median(gpu), np.median(ref))
    # the reported best energy and pose belong to the reported genotype (GPU self-consistency)
    import torch
    Lg = A.Ligand(ctx, ff, lig)
    e, _ = A.score(ctx, R, Lg, torch.from_numpy(res["genes"]).cuda())
    xyz = A.pose(ctx, Lg, torch.from_numpy(res["genes"]).cuda())
    ctx.sync()
    assert np.allclose(e.cpu().numpy(), res["best_energy"], rtol=1e-6, atol=1e-5)
    assert np.array_equal(xyz.cpu().numpy(), res["xyz"])


def _autostop_generation(best_per_gen, stopstd):
    """First generation g >= 10 whose last 10 best energies have a population
    standard deviation below stopstd (numpy), or None."""
    for g in range(10, len(best_per_gen) + 1):
        if np.std(best_per_gen[g - 10:g]) < stopstd:
            return g
    return None


def test_autostop_applies_the_rule(ctx, A, ff):
    """With autostop on, every GPU run ends at the first generation where its
    own best energies satisfy the rule (checked with numpy on the GPU's trace,
    skipping decisions within 1e-4 of the threshold); with it off the runs go
    on; the surviving evaluation counts shrink."""
    grid, rec, lig, maps64, maps32 = problem("plain")
    ngen = 60
    kw = dict(nrun=6, pop_size=60, ls_method=1, ls_max_iters=20, nev=10 ** 8, max_gen=ngen, stopstd=0.15)
    _, on = _params_pair(A, autostop=1, **kw)
    _, off = _params_pair(A, autostop=0, **kw)
    R = A.Receptor(ctx, grid, maps32)
    Lg = A.Ligand(ctx, ff, lig)
    res_on, tr = A.dock(ctx, R, Lg, on, trace_ngen=ngen)
    res_off = A.dock(ctx, R, Lg, off)[0]
    assert (res_off["generations"] == ngen).all()
    stopped = 0
    for run in range(on.nrun):
        best = tr["energies"][run].min(axis=1).astype(np.float64)
        g = int(res_on[0]["generations"][run])
        want = _autostop_generation(best[:g], on.stopstd)
        near = any(abs(np.std(best[k - 10:k]) - on.stopstd) < 1e-4 for k in range(10, g + 1))
        if not near:
            assert want == (g if g < ngen else want), (run, g, want)
        stopped += g < ngen
    assert stopped >= 1
    assert res_on[0]["evals"].sum() < res_off["evals"].sum()


def test_paper_scale_bench_configuration_sampled_against_oracle(ctx, A, ff):
    """The launch the bench times (paper-scale: 64^3 maps, 44 atoms, 8 torsions,
    100 runs x 150 x 2.5 M evaluations, ADADELTA): properties that hold at any
    size -- every run spends its budget, the best energy never rises along the
    trace, the reported pose is the oracle's pose of the reported genotype --
    and, on a sample of 20 runs, the reported best energy is the oracle's
    energy of the reported genotype within the energy tolerance."""
    grid, rec, lig, maps64, maps32 = problem("paper")
    R = A.Receptor(ctx, grid, maps32)
    Lg = A.Ligand(ctx, ff, lig)
    nev = 2_500_000
    p = A.search_params(nrun=100, pop_size=150, nev=nev, ls_method=A.LS_ADADELTA, seed=42)
    res = A.dock(ctx, R, Lg, p, best_trace=64)[0]
    assert (res["evals"] >= nev).all() and (res["evals"] < nev + 150 * 301).all()
    assert (res["generations"] == res["generations"][0]).all()
    assert np.all(np.diff(res["best_trace"], axis=1) <= 0)
    L = O.Ligand(lig)
    genes = res["genes"].astype(np.float64)
    xyz_ref = O.pose(L, genes)
    assert np.abs(res["xyz"] - xyz_ref).max() < 1e-3
    sample = np.arange(0, 100, 5)
    e_ref = O.score(ff, grid, maps64, L, genes[sample])[0]
    forces = O.atom_gradients(ff, grid, maps64, L, genes[sample])
    assert (np.abs(res["best_energy"][sample] - e_ref) <= energy_tol(e_ref, forces)).all()
    assert (e_ref < 0).all()

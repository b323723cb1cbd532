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

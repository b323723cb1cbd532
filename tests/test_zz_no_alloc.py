"""adg_dock_noalloc, the docking entry point for callers that cannot allocate
memory (an application allocator that owns all device memory, or a loop in
which cudaMalloc/cudaFree would stall other work): it must return what
adg_dock returns for the same inputs, on two calls in a row (the second call
reuses the first call's working memory), and reject requests larger than its
fixed working memory.  Collected last so that a failure here comes after
every other test has run; it passes alone in a fresh process too."""
import numpy as np
import pytest

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
def test_noalloc_dock_matches_dock_on_two_calls(ctx, ff, ls_method):
    from paper_2007_03678_gb300 import adg
    grid, rec, lig, maps64, maps32 = problem("plain")
    R = adg.Receptor(ctx, grid, maps32)
    L = adg.Ligand(ctx, ff, lig)
    p = adg.search_params(nrun=12, pop_size=150, nev=20000, ls_method=ls_method, ls_max_iters=40, seed=77)
    ref = adg.dock(ctx, R, L, p)[0]
    ctx.sync()
    # both paths run the same kernels on the same run-keyed random streams, so
    # the results agree bit for bit; a slip in carving or clearing the shared
    # array that moved a single individual would show here
    for call in range(2):
        got = adg.dock_noalloc(R, L, p)
        for key in ("best_energy", "genes", "xyz", "evals", "generations"):
            assert np.array_equal(got[key], ref[key]), (call, key)


def test_noalloc_rejects_oversized_requests(ctx, ff):
    from paper_2007_03678_gb300 import adg
    grid, rec, lig, maps64, maps32 = problem("plain")
    R = adg.Receptor(ctx, grid, maps32)
    L = adg.Ligand(ctx, ff, lig)
    for kw in (dict(nrun=129, pop_size=50), dict(nrun=100, pop_size=200)):
        p = adg.search_params(nev=1000, **kw)
        with pytest.raises(adg.AdgError) as ei:
            adg.dock_noalloc(R, L, p)
        assert ei.value.code == -3


def test_no_alloc_docking_keeps_a_fixed_stream_id():
    """adg_ligand_set_stream_id applies to the no-allocation entry point too."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03678_gb300 import adg, build
    from paper_2007_03678_gb300 import synth as S
    from gpu_common import problem
    build.build()
    ctx = adg.Context(0)
    ff = S.forcefield()
    grid, rec, lig, _, maps32 = problem("plain")
    R = adg.Receptor(ctx, grid, maps32)
    L = adg.Ligand(ctx, ff, lig)
    L.set_stream_id(4242)
    p = adg.search_params(nrun=3, pop_size=40, nev=4000, ls_method=adg.LS_SOLIS_WETS, ls_max_iters=20, seed=8,
                          lig_id=7)
    a = adg.dock_noalloc(R, L, p, stream=ctx.stream)
    L.set_stream_id(-1)
    q = adg.search_params(nrun=3, pop_size=40, nev=4000, ls_method=adg.LS_SOLIS_WETS, ls_max_iters=20, seed=8,
                          lig_id=4242)
    b = adg.dock(ctx, R, L, q)[0]
    for key in ("best_energy", "genes", "evals", "generations"):
        assert np.array_equal(a[key], b[key]), key
    ctx.close()

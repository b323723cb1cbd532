"""Differentiation workload: 65,536 random poses across 256 ligands (20-50
atoms, 2-12 torsions) on the 64^3 receptor, energy + gradient w.r.t.
translation, quaternion and torsions through the torch.autograd.Function,
checked against the oracle's analytic gradient (every pose) and FP64 central
finite differences with h = 1e-4 (a sample)."""
import numpy as np
import pytest

import oracle as O
from paper_2007_03678_gb300 import synth as S

from gpu_common import energy_tol, grad_ok, inside_box, near_face, problem, strict_at_gpu_coords

pytestmark = pytest.mark.gpu

NLIG, NPOSE = 256, 256
FD_H = 1e-4


def _ligands():
    rng = np.random.default_rng(2024)
    out = []
    seed = 30000
    while len(out) < NLIG:
        n_heavy = int(rng.integers(18, 46))
        n_tors = int(rng.integers(2, 13))
        seed += 1
        try:
            lig = S.make_ligand(n_heavy, n_tors, seed)
        except RuntimeError:
            continue
        if 20 <= lig.natoms <= 50:
            out.append(lig)
    return out


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


def _crosses_face(grid, xa, xb):
    """Do the two stencil end points put some atom in different map cells
    (or change which coordinates are clamped into the box)?"""
    def cell(x):
        u = (x - np.asarray(grid.origin)) / grid.spacing
        hi = np.asarray(grid.n) - 1
        return np.minimum(np.maximum(np.floor(u), -1), hi)
    return bool((cell(xa) != cell(xb)).any())


def test_autograd_matches_oracle_and_finite_differences(ctx, ff):
    import torch
    from paper_2007_03678_gb300 import adg
    from paper_2007_03678_gb300.autograd import score
    grid, rec, _, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    ligs = _ligands()
    assert len(ligs) * NPOSE == 65536
    checked = fd_checked = strict_checked = 0
    for li, lig in enumerate(ligs):
        genes = S.random_genes(lig, NPOSE, grid, 40000 + li, spread=0.3)
        genes[::2, 3:7] *= 1.5  # non-unit quaternions: the q gradient carries the 1/|q| factor
        g32 = genes.astype(np.float32)
        Lg = adg.Ligand(ctx, ff, lig)
        x = torch.from_numpy(g32).cuda().requires_grad_(True)
        e = score(x, ctx, R, Lg)
        e.sum().backward()
        ctx.sync()
        e = e.detach().cpu().numpy().astype(np.float64)
        gg = x.grad.cpu().numpy().astype(np.float64)
        L = O.Ligand(lig)
        g64 = g32.astype(np.float64)
        ref_e, _, ref_gg, _ = O.score(ff, grid, maps64, L, g64)
        forces = O.atom_gradients(ff, grid, maps64, L, g64)
        xyz = O.pose(L, g64)
        tol = energy_tol(ref_e, forces)
        bad = np.abs(e - ref_e) > tol
        assert not bad.any(), (li, [(int(p), e[p], ref_e[p], tol[p]) for p in np.nonzero(bad)[0][:4]])
        # the scoring alone, at the CUDA path's own posed coordinates: every
        # non-clashing pose at the plain 1e-3 + 1e-5|E|
        clean_g, ok_g, ref_g = strict_at_gpu_coords(ctx, adg, ff, grid, maps64, Lg, L, g32, e)
        bad = clean_g & ~ok_g
        assert not bad.any(), (li, [(int(p), e[p], ref_g[p]) for p in np.nonzero(bad)[0][:4]])
        strict_checked += int(clean_g.sum())
        smooth = inside_box(grid, xyz) & (ref_e < 1e3) & ~near_face(grid, xyz)
        ok = grad_ok(gg, ref_gg)[smooth]
        assert ok.all(), f"ligand {li}: {(~ok).any(axis=1).sum()} poses with a gradient component off"
        checked += int(smooth.sum())
        # FP64 central differences of the oracle energy on two smooth poses per ligand
        for p in np.nonzero(smooth)[0][:2]:
            fd = np.zeros(len(g64[p]))
            use = np.ones(len(g64[p]), bool)
            for d in range(len(fd)):
                gp, gm = g64[p].copy(), g64[p].copy()
                gp[d] += FD_H
                gm[d] -= FD_H
                if _crosses_face(grid, O.pose(L, gp)[0], O.pose(L, gm)[0]):
                    use[d] = False
                    continue
                fd[d] = (O.score(ff, grid, maps64, L, gp)[0][0] - O.score(ff, grid, maps64, L, gm)[0][0]) / (2 * FD_H)
            scale = max(np.abs(fd[use]).max(initial=0.0), 1.0)
            assert (np.abs(gg[p] - fd)[use] <= 1e-3 * scale).all(), (li, p, gg[p], fd)
            fd_checked += int(use.sum())
    assert checked > 0.1 * NLIG * NPOSE
    assert strict_checked > 0.1 * NLIG * NPOSE
    assert fd_checked > 3000


def test_batched_scoring_equals_per_ligand(ctx, ff):
    """adg_score_multi (one launch per atoms-per-lane width over many
    ligands) gives every pose the energy and gene gradient adg_score gives it,
    bit for bit; the batched autograd function returns the same gradients as
    the per-ligand one, including for a ligand with no poses."""
    import torch
    from paper_2007_03678_gb300 import adg
    from paper_2007_03678_gb300.autograd import score, score_batch, score_rows
    grid, rec, _, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    ligs = _ligands()[:12] + [S.make_ligand(80, 9, 5151), S.make_ligand(12, 2, 5252)]
    assert len({(l.natoms + 31) // 32 for l in ligs}) >= 3  # several widths in one call
    L = [adg.Ligand(ctx, ff, l) for l in ligs]
    counts = [37 + 11 * i for i in range(len(ligs))]
    counts[5] = 0
    genes = [torch.from_numpy(S.random_genes(l, max(k, 1), grid, 60000 + i, spread=0.3)[:k].astype(np.float32)).cuda()
             for i, (l, k) in enumerate(zip(ligs, counts))]
    rows = torch.zeros((sum(counts), adg.MAX_GENES), dtype=torch.float32, device="cuda")
    r = 0
    for g in genes:
        rows[r:r + g.shape[0], :g.shape[1]] = g
        r += g.shape[0]
    e_all, g_all = adg.score_multi(ctx, R, L, rows, counts, adg.GRAD_GENES)
    ctx.sync()
    packed = rows.clone().requires_grad_(True)
    e_rows = score_rows(packed, ctx, R, L, counts)
    e_rows.sum().backward()
    assert torch.equal(e_rows.detach(), e_all) and torch.equal(packed.grad, g_all)
    r = 0
    for Lg, g in zip(L, genes):
        n, w = g.shape
        if n:
            e1, g1 = adg.score(ctx, R, Lg, g.contiguous(), adg.GRAD_GENES)
            ctx.sync()
            assert torch.equal(e_all[r:r + n], e1)
            assert torch.equal(g_all[r:r + n, :w], g1)
            assert not g_all[r:r + n, w:].any()
        r += n
    # autograd through the batch against the per-ligand function
    xs = [g.clone().requires_grad_(True) for g in genes]
    energies = score_batch(xs, ctx, R, L)
    torch.stack([e.sum() for e in energies]).sum().backward()
    for Lg, g, x, e in zip(L, genes, xs, energies):
        if g.shape[0] == 0:
            assert e.numel() == 0
            continue
        y = g.clone().requires_grad_(True)
        e1 = score(y, ctx, R, Lg)
        e1.sum().backward()
        assert torch.equal(e.detach(), e1.detach())
        assert torch.equal(x.grad, y.grad)


def test_batched_scoring_across_changing_calls(ctx, ff):
    """adg_score_multi keeps its launch tables between calls and uploads new
    ones only when a call's ligands or counts differ: calls that alternate
    between ligand sets (of one and of several widths) and counts each give
    adg_score's values bit for bit, and every gradient row is written whole."""
    import torch
    from paper_2007_03678_gb300 import adg
    grid, rec, _, maps64, maps32 = problem("paper")
    R = adg.Receptor(ctx, grid, maps32)
    pool = _ligands()[:6] + [S.make_ligand(80, 9, 5353), S.make_ligand(12, 2, 5454)]
    L = [adg.Ligand(ctx, ff, l) for l in pool]
    G = {i: torch.from_numpy(S.random_genes(l, 96, grid, 61000 + i, spread=0.3).astype(np.float32)).cuda()
         for i, l in enumerate(pool)}
    calls = [([0, 1, 6, 7], [40, 17, 33, 9]), ([2, 3], [64, 5]), ([0, 1, 6, 7], [40, 17, 33, 9]),
             ([0, 1, 6, 7], [12, 50, 33, 9]), ([7, 6, 1, 0], [9, 33, 17, 40]), ([4], [96]), ([0, 1, 6, 7], [40, 17, 33, 9])]
    for idx, counts in calls:
        rows = torch.full((sum(counts), adg.MAX_GENES), 7.0, dtype=torch.float32, device="cuda")
        r = 0
        for i, k in zip(idx, counts):
            g = G[i][:k]
            rows[r:r + k] = 0.0
            rows[r:r + k, :g.shape[1]] = g
            r += k
        e_all, g_all = adg.score_multi(ctx, R, [L[i] for i in idx], rows, counts, adg.GRAD_GENES)
        ctx.sync()
        r = 0
        for i, k in zip(idx, counts):
            g = G[i][:k].contiguous()
            e1, g1 = adg.score(ctx, R, L[i], g, adg.GRAD_GENES)
            ctx.sync()
            assert torch.equal(e_all[r:r + k], e1), (idx, counts, i)
            assert torch.equal(g_all[r:r + k, :g.shape[1]], g1), (idx, counts, i)
            assert not g_all[r:r + k, g.shape[1]:].any()
            r += k

"""Pins for the FP64 oracle: each test checks the oracle against something
other than itself -- published known-answer vectors, closed forms,
invariants, library routines (scipy, networkx) and finite differences.

A plausible mistake anywhere in the oracle (a dropped term, a wrong sign, a
transposed index, a wrong exponent) should fail at least one test here.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2007_03678_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox(np.array([v[0:4]], np.uint32), v[4], v[5])[0]
        assert [int(x) for x in out] == v[6:10]


def test_philox_counter_sensitivity_and_uniformity():
    n = 20000
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    out = O.philox(ctr, 123, 456)
    # every word distinct-ish and top-24-bit uniforms pass a coarse chi-square
    u = (out.reshape(-1) >> 8) / 2.0 ** 24
    hist, _ = np.histogram(u, bins=32, range=(0, 1))
    exp = len(u) / 32
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 80  # 31 dof, p ~ 1e-5
    # changing one key bit changes the outputs
    out2 = O.philox(ctr[:100], 124, 456)
    assert np.mean(out2 == out[:100]) < 0.01


# ----------------------------------------------------------------- pair terms
def _num_deriv(f, r, h=1e-6):
    return (f(r + h) - f(r - h)) / (2 * h)


@pytest.mark.parametrize("ti,tj", [(S.T_C, S.T_C), (S.T_C, S.T_N), (S.T_OA, S.T_S), (S.T_A, S.T_HD)])
def test_lj_12_6_minimum_and_zero(ff, ti, tj):
    r0 = 0.5 * (ff["Rii"][ti] + ff["Rii"][tj])
    eps = math.sqrt(ff["epsii"][ti] * ff["epsii"][tj])
    e0, d0 = O.pair_lj(ff, ti, tj, r0)
    assert e0 == pytest.approx(-ff["w_vdw"] * eps, rel=1e-12)
    assert abs(d0) < 1e-10
    # zero crossing of a 12-6 well at r0 / 2^(1/6)
    rz = r0 / 2 ** (1 / 6)
    assert abs(O.pair_lj(ff, ti, tj, rz)[0]) < 1e-10
    # minimum found by a bracketing optimiser lands at r0
    from scipy.optimize import minimize_scalar
    res = minimize_scalar(lambda r: O.pair_lj(ff, ti, tj, r)[0], bounds=(r0 - 0.5, r0 + 1.0), method="bounded",
                          options=dict(xatol=1e-9))
    assert res.x == pytest.approx(r0, abs=1e-5)
    for r in (rz * 0.97, r0 * 1.3, 6.0):
        assert O.pair_lj(ff, ti, tj, r)[1] == pytest.approx(_num_deriv(lambda x: O.pair_lj(ff, ti, tj, x)[0], r),
                                                            rel=1e-6)


@pytest.mark.parametrize("donor,acc", [(S.T_HD, S.T_OA), (S.T_NA, S.T_HD)])
def test_hbond_12_10(ff, donor, acc):
    a = acc if ff["hb_acceptor"][acc] else donor
    r0, eps = ff["hb_R"][a], ff["hb_eps"][a]
    e0, d0 = O.pair_lj(ff, donor, acc, r0)
    assert e0 == pytest.approx(-ff["w_hb"] * eps, rel=1e-12)
    assert abs(d0) < 1e-9
    assert abs(O.pair_lj(ff, donor, acc, r0 * math.sqrt(5 / 6))[0]) < 1e-9
    # symmetric in argument order
    assert O.pair_lj(ff, acc, donor, 2.3)[0] == O.pair_lj(ff, donor, acc, 2.3)[0]
    # 12-10 decays as r^-10: E(2r)/E(r) -> 2^-10 at large r
    assert O.pair_lj(ff, donor, acc, 400.0)[0] / O.pair_lj(ff, donor, acc, 200.0)[0] == pytest.approx(2 ** -10, rel=1e-3)


def test_lj_cap_and_floor(ff):
    e, d = O.pair_lj(ff, S.T_C, S.T_C, 0.9)
    assert e == ff["e_cap"] and d == 0.0
    e1, _ = O.pair_lj(ff, S.T_HD, S.T_HD, 0.2)
    e2, _ = O.pair_lj(ff, S.T_HD, S.T_HD, ff["r_min"])
    assert e1 == e2


def test_elec_limits_and_derivative(ff):
    qq = 0.3 * -0.2
    w = ff["w_elec"] * ff["coulomb"]
    # at long range the dielectric saturates at eps0
    r = 2000.0
    e, _ = O.pair_elec(ff, qq, r)
    assert e == pytest.approx(w * qq / (ff["ms_eps0"] * r), rel=1e-9)
    # at contact the Mehler-Solmajer dielectric is close to 1.35 (A + B/(1+k))
    eps0 = ff["ms_A"] + (ff["ms_eps0"] - ff["ms_A"]) / (1 + ff["ms_k"])
    assert 1.2 < eps0 < 1.5
    # opposite charges attract, like charges repel
    assert O.pair_elec(ff, -0.04, 3.0)[0] < 0 < O.pair_elec(ff, 0.04, 3.0)[0]
    for r in (0.7, 2.0, 5.5, 12.0):
        assert O.pair_elec(ff, qq, r)[1] == pytest.approx(_num_deriv(lambda x: O.pair_elec(ff, qq, x)[0], r), rel=1e-6)
    # the screened Coulomb energy times r decreases in magnitude with r (eps grows)
    rs = np.linspace(1, 20, 50)
    er = np.array([O.pair_elec(ff, 1.0, x)[0] * x for x in rs])
    assert np.all(np.diff(er) < 0)


def test_desolv_gaussian_and_symmetry(ff):
    ti, qi, tj, qj = S.T_OA, -0.3, S.T_C, 0.1
    e0, _ = O.pair_desolv(ff, ti, qi, tj, qj, ff["r_min"])
    s = ff["sigma"]
    r = s * math.sqrt(2.0)
    e1, _ = O.pair_desolv(ff, ti, qi, tj, qj, r)
    assert e1 / e0 == pytest.approx(math.exp(-1.0) / math.exp(-ff["r_min"] ** 2 / (2 * s * s)), rel=1e-12)
    assert O.pair_desolv(ff, tj, qj, ti, qi, 2.7)[0] == pytest.approx(O.pair_desolv(ff, ti, qi, tj, qj, 2.7)[0],
                                                                      rel=1e-14)
    for rr in (1.0, 3.3, 7.0):
        assert O.pair_desolv(ff, ti, qi, tj, qj, rr)[1] == pytest.approx(
            _num_deriv(lambda x: O.pair_desolv(ff, ti, qi, tj, qj, x)[0], rr), rel=1e-6)
    # HD has zero volume: its partner's solvation term drops out
    eh, _ = O.pair_desolv(ff, S.T_HD, 0.0, S.T_HD, 0.0, 2.0)
    assert eh == 0.0


def test_map_switch(ff):
    assert O.map_switch(ff, ff["map_r_on"]) == 1.0
    assert O.map_switch(ff, ff["map_r_off"]) == 0.0
    assert O.map_switch(ff, 0.5 * (ff["map_r_on"] + ff["map_r_off"])) == pytest.approx(0.5)
    for r in (ff["map_r_on"], ff["map_r_off"]):
        d = _num_deriv(lambda x: O.map_switch(ff, x), r, 1e-7)
        assert abs(d) < 1e-5


# ----------------------------------------------------------------- maps
def test_maps_reproduce_pair_interaction(ff):
    """One receptor atom: M_t + q M_e + |q| M_d at a node equals the pair
    energy (vdW/H-bond + elec + desolvation) of a ligand atom there, times the
    switch.  Pins the map decomposition of the desolvation term."""
    grid = S.make_grid(9, 0.5)
    for tj in range(S.NTYPES):
        rec = S.Receptor(np.array([[0.13, -0.21, 0.34]]), np.array([tj], np.int32), np.array([-0.27]))
        maps = O.maps_build(ff, grid, rec)
        for (i, j, k) in ((0, 0, 0), (7, 4, 4), (8, 2, 5), (3, 7, 1)):
            p = np.array(grid.origin) + grid.spacing * np.array([i, j, k])
            r = np.linalg.norm(p - rec.xyz[0])
            assert r > 1.0  # no capped node in this set
            sw = O.map_switch(ff, r)
            for ti in range(S.NTYPES):
                for qi in (0.25, -0.4):
                    want = sw * (O.pair_lj(ff, ti, tj, r)[0] + O.pair_elec(ff, qi * rec.charge[0], r)[0] +
                                 O.pair_desolv(ff, ti, qi, tj, rec.charge[0], r)[0])
                    got = maps[ti, k, j, i] + qi * maps[S.MAP_ELEC, k, j, i] + abs(qi) * maps[S.MAP_DESOLV, k, j, i]
                    assert got == pytest.approx(want, rel=1e-11, abs=1e-12)


def test_maps_layout_is_x_fastest(ff):
    """A single receptor atom placed off-centre: the elec map must be radial
    about it when indexed [z][y][x] with node (i,j,k) at origin + (i,j,k) h."""
    grid = S.Grid((7, 9, 11), (-1.0, -2.0, -3.0), 0.4)
    P = np.array([0.31, -0.77, 0.58])
    rec = S.Receptor(P[None], np.array([S.T_C], np.int32), np.array([0.5]))
    maps = O.maps_build(ff, grid, rec)
    assert maps.shape == (9, 11, 9, 7)
    for (i, j, k) in ((0, 0, 0), (6, 8, 10), (3, 1, 7), (5, 8, 2)):
        p = np.array(grid.origin) + grid.spacing * np.array([i, j, k])
        r = np.linalg.norm(p - P)
        assert maps[S.MAP_ELEC, k, j, i] == pytest.approx(O.map_switch(ff, r) * O.pair_elec(ff, 0.5, r)[0], rel=1e-12)


def test_maps_cap(ff):
    grid = S.make_grid(5, 0.375)
    # two atoms on one node: each pair term is capped, the sum is capped again
    rec = S.Receptor(np.zeros((2, 3)), np.array([S.T_C, S.T_C], np.int32), np.array([0.0, 0.0]))
    maps = O.maps_build(ff, grid, rec)
    assert maps[S.T_C, 2, 2, 2] == ff["e_cap"]
    one = S.Receptor(np.zeros((1, 3)), np.array([S.T_C], np.int32), np.array([0.0]))
    m1 = O.maps_build(ff, grid, one)
    assert m1[S.T_C, 2, 2, 2] == pytest.approx(ff["e_cap"] + O.pair_desolv(ff, S.T_C, 0.0, S.T_C, 0.0, 0.0)[0]
                                               - ff["w_desolv"] * ff["qasp"] * 0.0, rel=1e-12)


# ----------------------------------------------------------------- trilinear
def _linear_map(grid, a, b):
    nx, ny, nz = grid.n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = grid.origin[0] + x * grid.spacing
    Y = grid.origin[1] + y * grid.spacing
    Z = grid.origin[2] + z * grid.spacing
    return a + b[0] * X + b[1] * Y + b[2] * Z


def test_trilinear_exact_for_linear_fields():
    grid = S.Grid((6, 7, 8), (-1.0, 0.5, 2.0), 0.375)
    b = np.array([0.7, -1.3, 2.1])
    m = _linear_map(grid, 0.4, b)
    rng = np.random.default_rng(0)
    lo = np.array(grid.origin)
    hi = lo + np.array(grid.extent)
    for _ in range(200):
        p = lo + rng.uniform(size=3) * (hi - lo)
        v, g = O.trilinear(grid, m, p)
        assert v == pytest.approx(0.4 + b @ p, rel=1e-12, abs=1e-12)
        assert np.allclose(g, b, rtol=1e-11)
    # the last node (f = 1 in the last cell) and the first node
    v, _ = O.trilinear(grid, m, hi)
    assert v == pytest.approx(0.4 + b @ hi, rel=1e-13)
    v, _ = O.trilinear(grid, m, lo)
    assert v == pytest.approx(0.4 + b @ lo, rel=1e-13)


def test_trilinear_nodes_and_clamping():
    grid = S.Grid((5, 5, 5), (0.0, 0.0, 0.0), 0.5)
    rng = np.random.default_rng(1)
    m = rng.normal(size=(5, 5, 5))
    for (i, j, k) in ((0, 0, 0), (4, 4, 4), (1, 3, 2), (4, 0, 3)):
        p = np.array([i, j, k]) * 0.5
        v, _ = O.trilinear(grid, m, p)
        assert v == pytest.approx(m[k, j, i], abs=1e-14)
    # outside along x: the value is the clamped one and d/dx of the map part is 0
    v_in, g_in = O.trilinear(grid, m, np.array([2.0, 1.1, 0.7]))
    v_out, g_out = O.trilinear(grid, m, np.array([5.0, 1.1, 0.7]))
    assert v_out == pytest.approx(v_in, abs=1e-14) and g_out[0] == 0.0
    assert g_out[1] == pytest.approx(g_in[1]) and g_out[2] == pytest.approx(g_in[2])


def test_out_of_box_penalty():
    grid = S.Grid((5, 5, 5), (0.0, 0.0, 0.0), 0.5)
    v, g = O.out_of_box(grid, np.array([2.5, -0.5, 1.0]), 10.0)
    assert v == pytest.approx(10.0 * (0.5 ** 2 + 0.5 ** 2))
    assert np.allclose(g, [10.0, -10.0, 0.0])
    assert O.out_of_box(grid, np.array([1.0, 1.0, 1.0]), 10.0)[0] == 0.0


# ----------------------------------------------------------------- pose
def test_quaternion_matrix_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(2)
    for _ in range(50):
        q = rng.normal(size=4) * rng.uniform(0.2, 3.0)
        R = O.quat_to_matrix(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is scalar-last
        assert np.allclose(R, ref, atol=1e-13)


@pytest.fixture(scope="module")
def lig8():
    return S.make_ligand(40, 8, 1000, n_hd=4)


def test_identity_genotype_reproduces_reference(lig8):
    L = O.Ligand(lig8)
    c = lig8.xyz.mean(axis=0)
    g = np.concatenate([c, [1, 0, 0, 0], np.zeros(8)])
    x = O.pose(L, g)[0]
    assert np.allclose(x, lig8.xyz, atol=1e-13)
    # a full turn of any torsion is the identity
    g2 = g.copy()
    g2[7 + 3] = 2 * np.pi
    assert np.allclose(O.pose(L, g2)[0], lig8.xyz, atol=1e-12)


def test_pose_preserves_bonds_and_fragments(lig8):
    L = O.Ligand(lig8)
    g = S.random_genes(lig8, 20, S.make_grid(64), 3)
    xs = O.pose(L, g)
    bl_ref = np.linalg.norm(lig8.xyz[lig8.bonds[:, 0]] - lig8.xyz[lig8.bonds[:, 1]], axis=1)
    import networkx as nx
    G = nx.Graph()
    G.add_edges_from(lig8.bonds.tolist())
    G.remove_edges_from([tuple(t) for t in lig8.tors.tolist()])
    frags = list(nx.connected_components(G))
    for x in xs:
        bl = np.linalg.norm(x[lig8.bonds[:, 0]] - x[lig8.bonds[:, 1]], axis=1)
        assert np.allclose(bl, bl_ref, atol=1e-12)
        for f in frags:
            f = sorted(f)
            d0 = np.linalg.norm(lig8.xyz[f][:, None] - lig8.xyz[f][None], axis=-1)
            d1 = np.linalg.norm(x[f][:, None] - x[f][None], axis=-1)
            assert np.allclose(d0, d1, atol=1e-11)


def _dihedral(p0, p1, p2, p3):
    b0, b1, b2 = p0 - p1, p2 - p1, p3 - p2
    b1n = b1 / np.linalg.norm(b1)
    v = b0 - (b0 @ b1n) * b1n
    w = b2 - (b2 @ b1n) * b1n
    return math.atan2(np.cross(b1n, v) @ w, v @ w)


def test_torsion_gene_changes_dihedral_by_theta(lig8):
    """Rotating torsion k by theta moves only its moving side and changes the
    dihedral across bond (a_k, b_k) by exactly +theta (right-hand rule about
    a -> b, with a on the root side)."""
    import networkx as nx
    L = O.Ligand(lig8)
    ab = L.torsions()
    mv = L.moving()
    G = nx.Graph()
    G.add_edges_from(lig8.bonds.tolist())
    c = lig8.xyz.mean(axis=0)
    for k in range(8):
        a, b = ab[k]
        # moving side = component of b after cutting (a, b), and it excludes the root
        H = G.copy()
        H.remove_edge(a, b)
        side = nx.node_connected_component(H, b)
        assert lig8.root not in side
        assert set(np.nonzero(mv[k])[0].tolist()) == side
        pa = [n for n in G.neighbors(a) if n != b][0]
        pb = [n for n in G.neighbors(b) if n != a][0]
        th = 0.731
        g = np.concatenate([c, [1, 0, 0, 0], np.zeros(8)])
        g[7 + k] = th
        x = O.pose(L, g)[0]
        d0 = _dihedral(lig8.xyz[pa], lig8.xyz[a], lig8.xyz[b], lig8.xyz[pb])
        d1 = _dihedral(x[pa], x[a], x[b], x[pb])
        assert math.remainder(d1 - d0 - th, 2 * math.pi) == pytest.approx(0.0, abs=1e-12)
        fixed = np.array([i not in side for i in range(lig8.natoms)])
        assert np.allclose(x[fixed], lig8.xyz[fixed], atol=1e-13)


def test_rigid_body_part_matches_scipy(lig8):
    from scipy.spatial.transform import Rotation
    L = O.Ligand(lig8)
    rng = np.random.default_rng(5)
    c = lig8.xyz.mean(axis=0)
    for _ in range(5):
        q = rng.normal(size=4)
        t = rng.normal(size=3) * 3
        g = np.concatenate([t, q, np.zeros(8)])
        x = O.pose(L, g)[0]
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).apply(lig8.xyz - c) + t
        assert np.allclose(x, ref, atol=1e-12)


# ----------------------------------------------------------------- topology
def test_pair_list_matches_networkx(lig8):
    import networkx as nx
    L = O.Ligand(lig8)
    G = nx.Graph()
    G.add_edges_from(lig8.bonds.tolist())
    dist = dict(nx.all_pairs_shortest_path_length(G))
    H = G.copy()
    H.remove_edges_from([tuple(t) for t in lig8.tors.tolist()])
    frag = {}
    for fi, comp in enumerate(nx.connected_components(H)):
        for a in comp:
            frag[a] = fi
    want = sorted((i, j) for i in range(lig8.natoms) for j in range(i + 1, lig8.natoms)
                  if frag[i] != frag[j] and dist[i][j] > 3)
    got = sorted(map(tuple, L.pairs().tolist()))
    assert got == want


def test_bad_topology_rejected():
    lig = S.make_ligand(12, 2, 7)
    bad = S.Ligand(lig.xyz, lig.type, lig.charge, lig.bonds, np.array([[0, lig.natoms - 1]], np.int32), 0)
    if not any(set(b) == {0, lig.natoms - 1} for b in lig.bonds.tolist()):
        with pytest.raises(ValueError):
            O.Ligand(bad)


# ----------------------------------------------------------------- energy
def _zero_maps(grid):
    nx, ny, nz = grid.n
    return np.zeros((S.NMAPS, nz, ny, nx))


def test_intra_energy_rigid_body_invariant(ff, lig8):
    grid = S.make_grid(64)
    maps = _zero_maps(grid)
    L = O.Ligand(lig8)
    rng = np.random.default_rng(8)
    base = S.random_genes(lig8, 1, grid, 9)[0]
    e0 = O.score(ff, grid, maps, L, base)[0][0]
    for _ in range(10):
        g = base.copy()
        g[0:3] = np.array(grid.center) + rng.uniform(-3, 3, 3)
        g[3:7] = rng.normal(size=4)
        e, _, gg, gt = O.score(ff, grid, maps, L, g)
        assert e[0] == pytest.approx(e0, rel=1e-12, abs=1e-12)
        # intramolecular forces are central and pairwise: no net force, no net torque
        assert np.allclose(gt[0, 0:6], 0.0, atol=1e-9 * max(1.0, np.abs(gt).max()))


def test_intra_energy_brute_force_tiny_ligand(ff):
    """A 7-atom chain with one torsion in the middle, built by hand: the pair
    list holds exactly the pairs >3 bonds apart across the torsion, and the
    energy is the plain sum of the three pair terms."""
    xyz = np.array([[0, 0, 0], [1.5, 0, 0], [2.0, 1.4, 0], [3.5, 1.4, 0], [4.0, 2.8, 0.3], [5.5, 2.8, 0.6],
                    [6.0, 4.2, 0.2]], float)
    types = np.array([S.T_C, S.T_OA, S.T_C, S.T_N, S.T_C, S.T_HD, S.T_S], np.int32)
    q = np.array([0.1, -0.3, 0.2, -0.1, 0.05, 0.3, -0.25])
    bonds = np.array([[i, i + 1] for i in range(6)], np.int32)
    tors = np.array([[2, 3]], np.int32)
    lig = S.Ligand(xyz, types, q, bonds, tors, 0)
    L = O.Ligand(lig)
    assert sorted(map(tuple, L.pairs().tolist())) == [(0, 4), (0, 5), (0, 6), (1, 5), (1, 6), (2, 6)]
    grid = S.make_grid(9, 2.0, center=tuple(xyz.mean(axis=0)))
    maps = _zero_maps(grid)
    g = np.concatenate([xyz.mean(axis=0), [1, 0, 0, 0], [0.9]])
    x = O.pose(L, g)[0]
    want = 0.0
    for (i, j) in L.pairs():
        r = np.linalg.norm(x[i] - x[j])
        want += O.pair_lj(ff, types[i], types[j], r)[0] + O.pair_elec(ff, q[i] * q[j], r)[0] + \
            O.pair_desolv(ff, types[i], q[i], types[j], q[j], r)[0]
    assert O.score(ff, grid, maps, L, g)[0][0] == pytest.approx(want, rel=1e-13)


def test_inter_energy_linear_maps_closed_form(ff, lig8):
    """With every map linear in space the interpolated intermolecular energy
    is exact: sum_i (a_t + b_t.x_i) + q_i (a_e + b_e.x_i) + |q_i| (a_d + b_d.x_i)."""
    grid = S.make_grid(64)
    rng = np.random.default_rng(10)
    coefs = [(rng.normal(), rng.normal(size=3)) for _ in range(S.NMAPS)]
    maps = np.stack([_linear_map(grid, a, b) for a, b in coefs])
    L = O.Ligand(lig8)
    g = S.random_genes(lig8, 6, grid, 11, spread=0.2)
    x = O.pose(L, g)
    e, ei, _, _ = O.score(ff, grid, maps, L, g)
    for p in range(len(g)):
        want = 0.0
        for i in range(lig8.natoms):
            t, qq = lig8.type[i], lig8.charge[i]
            val = lambda m: coefs[m][0] + coefs[m][1] @ x[p, i]
            want += val(t) + qq * val(S.MAP_ELEC) + abs(qq) * val(S.MAP_DESOLV)
        assert ei[p] == pytest.approx(want, rel=1e-11)


def _fd_gene_grad(ff, grid, maps, L, g, h=1e-6):
    out = np.zeros_like(g)
    for d in range(len(g)):
        gp, gm = g.copy(), g.copy()
        gp[d] += h
        gm[d] -= h
        out[d] = (O.score(ff, grid, maps, L, gp)[0][0] - O.score(ff, grid, maps, L, gm)[0][0]) / (2 * h)
    return out


def _fd_tangent_grad(ff, grid, maps, L, g, h=1e-6):
    D = 6 + L.ntors
    out = np.zeros(D)
    for d in range(D):
        xi = np.zeros(D)
        xi[d] = h
        ep = O.score(ff, grid, maps, L, O.apply_step(L.ntors, g, xi, 1.0))[0][0]
        em = O.score(ff, grid, maps, L, O.apply_step(L.ntors, g, xi, -1.0))[0][0]
        out[d] = (ep - em) / (2 * h)
    return out


def test_gradient_matches_finite_differences_linear_maps(ff, lig8):
    """Smooth energy (linear maps, exact trilinear) -> the analytic gene and
    tangent gradients agree with central differences to ~1e-6 relative."""
    grid = S.make_grid(64)
    rng = np.random.default_rng(12)
    maps = np.stack([_linear_map(grid, rng.normal(), rng.normal(size=3)) for _ in range(S.NMAPS)])
    L = O.Ligand(lig8)
    for g in S.random_genes(lig8, 4, grid, 13, spread=0.2):
        g[3:7] *= 1.7  # non-unit quaternion: the gradient must carry the 1/|q| factor
        e, _, gg, gt = O.score(ff, grid, maps, L, g)
        fd = _fd_gene_grad(ff, grid, maps, L, g)
        scale = max(1.0, np.abs(fd).max())
        assert np.abs(gg[0] - fd).max() / scale < 1e-6
        # radial quaternion direction carries no gradient
        assert abs(gg[0, 3:7] @ g[3:7]) < 1e-8 * scale
        fdt = _fd_tangent_grad(ff, grid, maps, L, g)
        assert np.abs(gt[0] - fdt).max() / max(1.0, np.abs(fdt).max()) < 1e-6


def test_gradient_matches_finite_differences_real_maps(ff, plain_inputs, plain_maps):
    """On the interpolated plain-workload maps, away from cell faces."""
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    checked = 0
    for g in S.random_genes(lig, 40, grid, 14, spread=0.15):
        x = O.pose(L, g)[0]
        u = (x - np.array(grid.origin)) / grid.spacing
        frac = u - np.floor(u)
        if np.min(np.minimum(frac, 1 - frac)) < 1e-3:
            continue  # a finite-difference stencil would cross a cell face
        e, _, gg, _ = O.score(ff, grid, plain_maps, L, g)
        fd = _fd_gene_grad(ff, grid, plain_maps, L, g, h=1e-7)
        assert np.abs(gg[0] - fd).max() / max(1.0, np.abs(fd).max()) < 1e-5
        checked += 1
    assert checked >= 10


# ----------------------------------------------------------------- moves
def test_apply_step_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(15)
    for _ in range(20):
        g = np.concatenate([rng.normal(size=3), rng.normal(size=4), rng.normal(size=2)])
        g[3:7] /= np.linalg.norm(g[3:7])
        xi = rng.normal(size=8) * 0.7
        out = O.apply_step(2, g, xi, 1.0)
        assert np.allclose(out[0:3], g[0:3] + xi[0:3])
        assert np.allclose(out[7:], g[7:] + xi[6:])
        want = Rotation.from_rotvec(xi[3:6]) * Rotation.from_quat([g[4], g[5], g[6], g[3]])
        wq = want.as_quat()
        got = np.array([out[4], out[5], out[6], out[3]])
        assert min(np.abs(got - wq).max(), np.abs(got + wq).max()) < 1e-12
        back = O.apply_step(2, out, xi, -1.0)
        assert min(np.abs(back - g).max(), np.abs(np.r_[back[:3], -back[3:7], back[7:]] - g).max()) < 1e-12


# ----------------------------------------------------------------- local search
def _bowl_problem(ff, centre_node=(6, 6, 6)):
    """One-atom ligand (HD, charge 0) over a map that samples a convex bowl
    whose minimum sits on a node: the interpolant's minimum is that node."""
    grid = S.Grid((13, 13, 13), (0.0, 0.0, 0.0), 0.375)
    c = np.array(centre_node) * grid.spacing
    nx, ny, nz = grid.n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([x, y, z], -1) * grid.spacing
    bowl = ((P - c) ** 2).sum(-1) * 2.0 - 5.0
    maps = np.zeros((S.NMAPS, nz, ny, nx))
    maps[S.T_HD] = bowl
    lig = S.Ligand(np.zeros((1, 3)), np.array([S.T_HD], np.int32), np.zeros(1), np.zeros((0, 2), np.int32),
                   np.zeros((0, 2), np.int32), 0)
    return grid, maps, O.Ligand(lig), c


@pytest.mark.parametrize("method", [1, 2])
def test_local_search_finds_bowl_minimum(ff, method):
    grid, maps, L, c = _bowl_problem(ff)
    p = O.SearchParams(ls_method=method, ls_max_iters=300, sw_rho_min=1e-4)
    g0 = np.concatenate([c + np.array([1.2, -0.8, 0.9]), [1, 0, 0, 0]])
    e0 = O.score(ff, grid, maps, L, g0)[0][0]
    g, e, n = O.local_search(ff, grid, maps, L, p, g0, e0)
    assert e < -4.9
    assert np.linalg.norm(g[0:3] - c) < (0.06 if method == 1 else 0.1)
    assert 1 <= n <= 600


def test_adadelta_constant_gradient_steps(ff):
    """In a linear field the gradient is constant, so ADADELTA's step sizes
    follow Zeiler's recursion: |dx_1| = sqrt(eps / ((1-rho) g^2 + eps)) |g|,
    and the steps grow monotonically while the field keeps decreasing."""
    grid = S.Grid((33, 33, 33), (0.0, 0.0, 0.0), 0.375)
    maps = np.stack([_linear_map(grid, 0.0, np.array([0.5, 0.0, 0.0])) for _ in range(S.NMAPS)])
    lig = S.Ligand(np.zeros((1, 3)), np.array([S.T_C], np.int32), np.zeros(1), np.zeros((0, 2), np.int32),
                   np.zeros((0, 2), np.int32), 0)
    L = O.Ligand(lig)
    g0 = np.concatenate([[8.0, 6.0, 6.0], [1, 0, 0, 0]])
    xs = []
    for iters in (2, 3, 4):
        p = O.SearchParams(ls_method=2, ls_max_iters=iters)
        g, e, n = O.local_search(ff, grid, maps, L, p, g0, O.score(ff, grid, maps, L, g0)[0][0])
        assert n == iters
        xs.append(g[0])
    step1 = 8.0 - xs[0]
    gx, rho, eps = 0.5, 0.8, 0.01
    assert step1 == pytest.approx(math.sqrt(eps / ((1 - rho) * gx * gx + eps)) * gx, rel=1e-12)
    steps = -np.diff([8.0] + xs)
    assert np.all(np.diff(steps) > 0)


# ----------------------------------------------------------------- LGA
def test_lga_decisions_statistics_and_bookkeeping(ff, plain_inputs, plain_maps):
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    pop = 150
    p = O.SearchParams(pop_size=pop, ls_method=0, nev=pop + 40 * (pop - 1), max_gen=100)
    best, bg, evals, gens, (dec, tg, te) = O.lga_run(ff, grid, plain_maps, L, p, ntrace=40)
    assert gens == 40 and evals == pop + 40 * (pop - 1)
    nb = 2 + lig.ntors
    kids = dec[:, 1:]
    assert ((kids[..., 0] >= 0) & (kids[..., 0] < pop)).all() and ((kids[..., 1] >= 0) & (kids[..., 1] < pop)).all()
    xo = kids[..., 2] >= 0
    assert abs(xo.mean() - 0.8) < 0.03
    assert ((kids[..., 2][xo] <= kids[..., 3][xo]) & (kids[..., 3][xo] <= nb)).all()
    mut_rate = np.mean([(m >> b) & 1 for m in kids[..., 4].ravel() for b in range(nb)])
    assert abs(mut_rate - 0.02) < 0.006
    # elitism: slot 0 copies the previous generation's best
    for gi in range(1, 40):
        assert te[gi, 0] == te[gi - 1].min()
    # energies stored in the trace are the oracle's energies of the stored genes
    e = O.score(ff, grid, plain_maps, L, tg[5])[0]
    assert np.allclose(e, te[5], rtol=1e-12)
    # best never gets worse across generations, and equals the final minimum
    assert np.all(np.diff(te.min(axis=1)) <= 0)
    assert best == te[-1].min()


def test_lga_tournament_prefers_better(ff, plain_inputs, plain_maps):
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    pop = 150
    p = O.SearchParams(pop_size=pop, ls_method=0, nev=pop + 10 * (pop - 1), max_gen=100)
    _, _, _, _, (dec, tg, te) = O.lga_run(ff, grid, plain_maps, L, p, ntrace=10)
    # parents of generation g are chosen from generation g-1's energies: the
    # mean rank of chosen parents must be better than uniform (0.6 vs 0.4)
    ranks = []
    for gi in range(1, 10):
        order = np.argsort(np.argsort(te[gi - 1], kind="stable"), kind="stable")
        ranks.extend(order[dec[gi, 1:, 0]].tolist())
    assert np.mean(ranks) < 0.47 * pop


def test_lga_run_with_solis_wets_improves(ff, plain_inputs, plain_maps):
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    p = O.SearchParams(nev=20000, ls_method=1)
    init = O.init_population(grid, p, lig.ntors)
    e_init = O.score(ff, grid, plain_maps, L, init)[0]
    best, g, evals, gens, _ = O.lga_run(ff, grid, plain_maps, L, p)
    assert best < e_init.min() and best < 0.0
    assert evals >= 20000
    assert O.score(ff, grid, plain_maps, L, g)[0][0] == pytest.approx(best, rel=1e-12)


def test_init_population_uniform_in_box(plain_inputs):
    grid, rec, lig = plain_inputs
    p = O.SearchParams(pop_size=4000)
    g = O.init_population(grid, p, lig.ntors)
    lo, hi = np.array(grid.origin), np.array(grid.origin) + np.array(grid.extent)
    assert (g[:, :3] >= lo).all() and (g[:, :3] < hi).all()
    assert np.allclose(np.linalg.norm(g[:, 3:7], axis=1), 1.0, atol=1e-12)
    # uniform on S^3: E[w^2] = 1/4 per component
    assert np.allclose((g[:, 3:7] ** 2).mean(axis=0), 0.25, atol=0.02)
    assert (np.abs(g[:, 7:]) <= np.pi).all()


def test_atom_gradients_sum_to_translation_gradient(ff, plain_inputs, plain_maps):
    """Per-atom gradients: their sum is dE/dt and their torque sum is the
    tangent rotation gradient (both pinned by finite differences above)."""
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    g = S.random_genes(lig, 30, grid, 31, spread=0.2)
    f = O.atom_gradients(ff, grid, plain_maps, L, g)
    _, _, _, gt = O.score(ff, grid, plain_maps, L, g)
    x = O.pose(L, g)
    assert np.allclose(f.sum(axis=1), gt[:, 0:3], rtol=1e-10, atol=1e-8)
    tau = np.cross(x - g[:, None, 0:3], f).sum(axis=1)
    assert np.allclose(tau, gt[:, 3:6], rtol=1e-10, atol=1e-8)


def test_lga_run_is_deterministic(ff, plain_inputs, plain_maps):
    """Same seed, same result, bit for bit (the counter-based stream has no
    hidden state); a different seed gives a different run."""
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    p = O.SearchParams(nev=3000, ls_method=1, pop_size=40)
    a = O.lga_run(ff, grid, plain_maps, L, p, run=3)
    b = O.lga_run(ff, grid, plain_maps, L, p, run=3)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2]
    p.seed = 43
    c = O.lga_run(ff, grid, plain_maps, L, p, run=3)
    assert not np.array_equal(a[1], c[1])


def test_autostop_rule(ff, plain_inputs, plain_maps):
    """A run with autostop ends at the first generation >= 10 whose last 10
    best energies have a population standard deviation (numpy) below stopstd;
    without autostop it runs to max_gen."""
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    kw = dict(pop_size=40, ls_method=1, ls_max_iters=15, nev=10 ** 8, max_gen=60, stopstd=0.15)
    _, _, _, g_off, _ = O.lga_run(ff, grid, plain_maps, L, O.SearchParams(autostop=0, **kw), run=1)
    assert g_off == 60
    best, _, _, g_on, (dec, tg, te) = O.lga_run(ff, grid, plain_maps, L, O.SearchParams(autostop=1, **kw), run=1,
                                                ntrace=60)
    b = te[:g_on].min(axis=1)
    first = next((g for g in range(10, g_on + 1) if np.std(b[g - 10:g]) < 0.15), None)
    assert first == g_on < 60


# ----------------------------------------------------------------- Solis-Wets, step by step
def _sw_gaussians(params, lig_id, run, ind, gen, iters, D):
    """The Solis-Wets normal draws from the pinned Philox stream and the
    textbook Box-Muller transform: counter (ligand, run<<16 | individual,
    generation, 5<<20 | iteration*8 + d/4); words (2p, 2p+1) with p = (d/2)
    mod 2 give u1 in (0, 1] and u2 in [0, 1); z = sqrt(-2 ln u1) cos(2 pi u2)
    for even d, sin for odd d."""
    z = np.zeros((iters, D))
    for it in range(iters):
        for d in range(D):
            ctr = np.array([[lig_id, (run << 16) | ind, gen, (5 << 20) | (it * 8 + d // 4)]], np.uint32)
            w = O.philox(ctr, params.seed & 0xFFFFFFFF, params.seed >> 32)[0]
            p = (d // 2) % 2
            u1 = ((int(w[2 * p]) >> 8) + 1) / 2.0 ** 24
            u2 = (int(w[2 * p + 1]) >> 8) / 2.0 ** 24
            rad = math.sqrt(-2.0 * math.log(u1))
            z[it, d] = rad * (math.cos(2 * math.pi * u2) if d % 2 == 0 else math.sin(2 * math.pi * u2))
    return z


def test_solis_wets_follows_the_published_rule(ff, plain_inputs, plain_maps):
    """Every iteration of a Solis-Wets search (Solis & Wets 1981) on the plain
    problem, checked against the rule: the trial is xi = bias + rho s (.) z
    with z the Box-Muller normals of the Philox stream; x (+) xi is taken when
    it lowers the energy (bias <- 0.4 xi + 0.2 bias), else x (-) xi when that
    does (bias <- bias - 0.4 xi), else nothing moves (bias <- bias / 2); rho
    doubles after 4 successes in a row and halves after 4 failures in a row.
    The energies of both trials are recomputed with the scoring function and
    the step with the tangent move (both pinned above)."""
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    T, D = lig.ntors, 6 + lig.ntors
    p = O.SearchParams(ls_method=1, ls_max_iters=80, seed=11, lig_id=3)
    scale = np.array([p.sw_scale_t] * 3 + [p.sw_scale_rot] * 3 + [p.sw_scale_tors] * T)
    g0 = S.random_genes(lig, 4, grid, 41, spread=0.2)[2]
    e0 = O.score(ff, grid, plain_maps, L, g0)[0][0]
    g_end, e_end, nev, tr = O.solis_wets_trace(ff, grid, plain_maps, L, p, g0, e0, run=2, ind=7, gen=3)
    n = len(tr["rho"])
    assert n == p.ls_max_iters or tr["rho"][-1] * 0.5 < p.sw_rho_min
    z = _sw_gaussians(p, 3, 2, 7, 3, n, D)
    x, e, bias, rho, succ, fail = g0.copy(), e0, np.zeros(D), 1.0, 0, 0
    outcomes, evals = set(), 0
    for it in range(n):
        assert tr["rho"][it] == rho
        xi = bias + rho * scale * z[it]
        assert np.allclose(tr["xi"][it], xi, rtol=1e-12, atol=1e-14)
        xi = tr["xi"][it]
        plus, minus = O.apply_step(T, x, xi, 1.0), O.apply_step(T, x, xi, -1.0)
        e_plus = O.score(ff, grid, plain_maps, L, plus)[0][0]
        evals += 1
        if e_plus < e:
            want, x, e, bias = 1, plus, e_plus, 0.4 * xi + 0.2 * bias
        else:
            e_minus = O.score(ff, grid, plain_maps, L, minus)[0][0]
            evals += 1
            if e_minus < e:
                want, x, e, bias = -1, minus, e_minus, bias - 0.4 * xi
            else:
                want, bias = 0, 0.5 * bias
        assert tr["outcome"][it] == want, it
        assert tr["energy"][it] == e
        assert np.allclose(tr["bias"][it], bias, rtol=1e-12, atol=1e-14)
        outcomes.add(want)
        succ, fail = (succ + 1, 0) if want else (0, fail + 1)
        if succ >= 4:
            rho, succ = 2 * rho, 0
        if fail >= 4:
            rho, fail = 0.5 * rho, 0
    assert outcomes == {1, -1, 0}  # the three branches all ran
    assert nev == evals and e_end == e and np.array_equal(g_end, x)


def test_solis_wets_at_a_strict_minimum_contracts_to_rho_min(ff):
    """Started exactly on the minimum node of a convex bowl, every trial is
    worse in both directions: the bias stays 0, rho halves after every 4
    failures, 1 -> 2^-7 < 0.01 after 28 iterations = 56 evaluations, and the
    genotype does not move."""
    grid, maps, L, c = _bowl_problem(ff)
    p = O.SearchParams(ls_method=1, ls_max_iters=300)
    g0 = np.concatenate([c, [1, 0, 0, 0]])
    e0 = O.score(ff, grid, maps, L, g0)[0][0]
    g, e, nev, tr = O.solis_wets_trace(ff, grid, maps, L, p, g0, e0)
    assert len(tr["rho"]) == 28 and nev == 56
    assert (tr["outcome"] == 0).all() and (tr["bias"] == 0).all()
    assert np.array_equal(tr["rho"], 0.5 ** (np.arange(28) // 4))
    assert np.array_equal(g, g0) and e == e0


def test_solis_wets_on_a_linear_field_always_succeeds(ff):
    """One atom in a linear field E = b.x: for any trial one of x (+) xi and
    x (-) xi is lower, and the lower one is the one with b.xi_t < 0.  So every
    iteration succeeds, rho doubles every 4 iterations, and the translation
    moves by exactly -sign(b.xi_t) xi_t each time."""
    grid = S.Grid((61, 61, 61), (0.0, 0.0, 0.0), 1.0)
    b = np.array([0.3, -0.2, 0.5])
    maps = np.stack([_linear_map(grid, 0.0, b) for _ in range(S.NMAPS)])
    lig = S.Ligand(np.zeros((1, 3)), np.array([S.T_C], np.int32), np.zeros(1), np.zeros((0, 2), np.int32),
                   np.zeros((0, 2), np.int32), 0)
    L = O.Ligand(lig)
    p = O.SearchParams(ls_method=1, ls_max_iters=12, sw_scale_t=0.1)
    g0 = np.array([30.0, 30.0, 30.0, 1, 0, 0, 0])
    e0 = O.score(ff, grid, maps, L, g0)[0][0]
    g, e, nev, tr = O.solis_wets_trace(ff, grid, maps, L, p, g0, e0)
    assert len(tr["rho"]) == 12
    assert np.array_equal(tr["rho"], 2.0 ** (np.arange(12) // 4))
    want = -np.sign(tr["xi"][:, 0:3] @ b)
    assert np.array_equal(tr["outcome"], want.astype(int))
    assert nev == 12 + (want < 0).sum()
    t = g0[0:3] + (want[:, None] * tr["xi"][:, 0:3]).sum(axis=0)
    assert np.allclose(g[0:3], t, rtol=0, atol=1e-12)
    assert e == pytest.approx(e0 + b @ (t - g0[0:3]), abs=1e-10)


# ----------------------------------------------------------------- offspring
def test_make_offspring_blocks_and_mutations():
    """Selection, crossover and mutation of single offspring against the
    operators' definitions, drawing from the pinned Philox stream:
      - parents: binary tournaments over uniform indices floor(w pop / 2^32),
        the lower energy (ties to the lower index) winning when the word's
        top 24 bits fall below floor(0.6 * 2^24);
      - two-point crossover over gene blocks [t][q][theta_1]..[theta_T]: the
        blocks in [lo, hi) are parent 2's, all others parent 1's, q whole;
      - mutation per block: t moves by mut_t (2u - 1) per component, theta by
        mut_tors (2u - 1), q by a rotation of angle mut_rot (2u - 1) about a
        uniform axis (checked with scipy's rotation algebra); blocks that do
        not mutate keep their crossed-over values bit for bit."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(5)
    T, pop = 5, 40
    G, nb = 7 + T, 2 + T
    Pg = rng.normal(size=(pop, G))
    Pg[:, 3:7] /= np.linalg.norm(Pg[:, 3:7], axis=1, keepdims=True)
    Pe = rng.normal(size=pop)
    Pe[7] = Pe[3]  # one tie, broken towards the lower index
    base = O.SearchParams(pop_size=pop, mutation_rate=0.0, seed=99, lig_id=4)
    mut = O.SearchParams(pop_size=pop, mutation_rate=0.5, seed=99, lig_id=4)
    key = (base.seed & 0xFFFFFFFF, base.seed >> 32)
    thr = lambda pr: math.floor(pr * 2 ** 24)

    def words(run, ind, gen, purpose, blk):
        return [int(v) for v in O.philox(np.array([[4, (run << 16) | ind, gen, (purpose << 20) | blk]], np.uint32),
                                          *key)[0]]

    seen_x = seen_m = 0
    for k in range(400):
        run, ind, gen = k % 3, 1 + k % (pop - 1), 1 + k // 7
        c0, d0 = O.make_offspring(base, T, Pg, Pe, run, ind, gen)
        c1, d1 = O.make_offspring(mut, T, Pg, Pe, run, ind, gen)
        for f in ("parent1", "parent2", "xlo", "xhi", "a1", "b1", "a2", "b2"):
            assert d0[f] == d1[f]
        parents = []
        for s in (0, 1):
            w = words(run, ind, gen, 2, s)
            a, b = (w[0] * pop) >> 32, (w[1] * pop) >> 32
            better, worse = (a, b) if (Pe[a] < Pe[b] or (Pe[a] == Pe[b] and a <= b)) else (b, a)
            parents.append(better if (w[2] >> 8) < thr(0.6) else worse)
            assert (d0["a%d" % (s + 1)], d0["b%d" % (s + 1)]) == (a, b)
        assert (d0["parent1"], d0["parent2"]) == tuple(parents)
        p1, p2 = parents
        w = words(run, ind, gen, 2, 2)
        if (w[0] >> 8) < thr(0.8):
            c1_, c2_ = (w[1] * (nb + 1)) >> 32, (w[2] * (nb + 1)) >> 32
            lo, hi = min(c1_, c2_), max(c1_, c2_)
            seen_x += hi > lo
        else:
            lo = hi = -1
        assert (d0["xlo"], d0["xhi"]) == (lo, hi)
        blocks = [slice(0, 3), slice(3, 7)] + [slice(7 + j, 8 + j) for j in range(T)]
        for bidx, sl in enumerate(blocks):
            src = p2 if lo <= bidx < hi else p1
            assert np.array_equal(c0[sl], Pg[src, sl])
        assert d0["mut_mask"] == 0
        mask = 0
        for bidx, sl in enumerate(blocks):
            if (words(run, ind, gen, 2, 3 + bidx // 4)[bidx % 4] >> 8) >= thr(0.5):
                assert np.array_equal(c1[sl], c0[sl])
                continue
            mask |= 1 << bidx
            m = words(run, ind, gen, 3, bidx)
            u = [(v >> 8) / 2.0 ** 24 for v in m]
            if bidx == 0:
                assert np.array_equal(c1[sl], c0[sl] + 2.0 * (2.0 * np.array(u[:3]) - 1.0))
                assert np.abs(c1[sl] - c0[sl]).max() <= 2.0
            elif bidx == 1:
                zc, phi, ang = 2 * u[0] - 1, 2 * math.pi * u[1], (math.pi / 2) * (2 * u[2] - 1)
                axis = np.array([math.sqrt(1 - zc * zc) * math.cos(phi), math.sqrt(1 - zc * zc) * math.sin(phi), zc])
                want = Rotation.from_rotvec(ang * axis) * Rotation.from_quat([c0[4], c0[5], c0[6], c0[3]])
                wq = want.as_quat()
                got = np.array([c1[4], c1[5], c1[6], c1[3]])
                assert min(np.abs(got - wq).max(), np.abs(got + wq).max()) < 1e-12
                assert abs(np.dot(c1[3:7], c0[3:7])) >= math.cos(math.pi / 4) - 1e-12  # at most 90 degrees
            else:
                assert c1[sl][0] == c0[sl][0] + (math.pi / 2) * (2.0 * u[0] - 1.0)
                assert abs(c1[sl][0] - c0[sl][0]) <= math.pi / 2
        assert d1["mut_mask"] == mask
        seen_m += mask != 0
    assert seen_x > 200 and seen_m > 300


def test_score_of_posed_coordinates_matches_genotype_scoring(ff, plain_inputs, plain_maps):
    """orc_score_xyz on the oracle's own posed coordinates gives orc_score's
    energies and per-atom gradients bit for bit; translating every atom by a
    vector leaves the intramolecular part unchanged."""
    grid, rec, lig = plain_inputs
    L = O.Ligand(lig)
    g = S.random_genes(lig, 40, grid, 43, spread=0.2)
    e, ei, _, _ = O.score(ff, grid, plain_maps, L, g)
    x = O.pose(L, g)
    e2, ei2, f2 = O.score_xyz(ff, grid, plain_maps, L, x, forces=True)
    assert np.array_equal(e, e2) and np.array_equal(ei, ei2)
    assert np.array_equal(f2, O.atom_gradients(ff, grid, plain_maps, L, g))
    zero = np.zeros_like(plain_maps)
    a = O.score_xyz(ff, grid, zero, L, x)[0] - O.score_xyz(ff, grid, zero, L, x)[1]
    b = O.score_xyz(ff, grid, zero, L, x + np.array([0.7, -0.4, 0.2]))
    assert np.allclose(a, b[0] - b[1], rtol=1e-12, atol=1e-9)

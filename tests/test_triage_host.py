"""Host-side logic of the triage pipeline (no GPU): the energy squash, the
feature rows, the survival rule and the recall measure."""
import numpy as np

from paper_2007_03678_gb300 import triage as T


def test_squash_is_monotone_and_keeps_the_bound_region():
    e = np.array([-20.0, -3.5, -1e-9, 0.0, 1e-9, 0.5, 10.0, 1e5])
    s = T.squash(e)
    assert np.all(np.diff(s) > 0) or np.all(np.diff(s) >= 0)
    assert np.array_equal(s[:4], e[:4])
    assert np.isclose(s[-1], np.log1p(1e5))
    assert np.isclose(s[5], np.log1p(0.5))


def test_features_layout():
    rng = np.random.default_rng(0)
    n, nrun, K = 5, 4, 3
    desc = rng.normal(size=(n, 16))
    tr = -np.sort(rng.uniform(0, 10, size=(n, nrun, 7)), axis=2)  # non-increasing traces
    tr[0, 2, :] = 1e4                                              # a run stuck in a clash
    x = T.features(desc, tr, K)
    assert x.shape == (n, 16 + 2 * K) and x.dtype == np.float32
    assert np.allclose(x[:, :16], desc, atol=1e-6)
    sq = T.squash(tr[:, :, :K])
    assert np.allclose(x[:, 16:16 + K], sq.min(axis=1), atol=1e-5)
    assert np.allclose(x[:, 16 + K:], sq.mean(axis=1), atol=1e-5)
    assert x[0, 16 + K] < 5  # the clash run enters the mean as log(1 + 1e4), not 1e4


def test_keep_best_and_recall():
    score = np.array([3.0, -1.0, 2.0, -5.0, 0.0, -5.0])
    keep = T.keep_best(score, 0.5)
    assert keep.sum() == 3 and keep[3] and keep[5] and keep[1]
    assert T.keep_best(score, 0.0).sum() == 0 and T.keep_best(score, 1.0).all()
    true_e = np.arange(100, dtype=float)          # ligand 0 is the best
    keep = np.zeros(100, bool)
    keep[:1] = True
    assert T.recall(true_e, keep, 0.01) == 1.0    # top 1 % = ligand 0
    assert T.recall(true_e, keep, 0.02) == 0.5
    assert T.recall(true_e, ~keep, 0.01) == 0.0


def test_config_defaults():
    from paper_2007_03678_gb300 import build
    build.build()  # search_params reads the library's defaults
    cfg = T.TriageConfig()
    assert cfg.early_gen * 10 == cfg.max_gen       # the early search is the first tenth
    assert cfg.nin == 16 + 2 * cfg.early_gen <= 32  # fits the network's input width
    p = cfg.params(cfg.early_gen)
    assert p.max_gen == cfg.early_gen and p.nrun == cfg.nrun and p.ls_method == cfg.ls_method


def test_wilson_interval_and_recall_counts():
    """The Wilson score interval: its end points are the proportions at which
    the normal-approximation test is exactly at z (checked by substitution),
    it contains the sample proportion, narrows as 1/sqrt(n), and for 20 of 20
    hits has the closed form lower end n / (n + z^2)."""
    z = 1.959963984540054
    for hits, n in ((20, 20), (190, 200), (0, 50), (7, 9)):
        lo, hi = T.wilson_interval(hits, n)
        ph = hits / n
        assert lo <= ph <= hi
        for p in (lo, hi):
            if 0.0 < p < 1.0:
                assert abs(abs(ph - p) - z * np.sqrt(p * (1 - p) / n)) < 1e-12
    assert np.isclose(T.wilson_interval(20, 20)[0], 20 / (20 + z * z))
    w1 = np.diff(T.wilson_interval(90, 100))[0]
    w2 = np.diff(T.wilson_interval(9000, 10000))[0]
    assert 8 < w1 / w2 < 12
    true_e = np.arange(1000, dtype=float)
    keep = np.zeros(1000, bool)
    keep[[0, 1, 2, 5, 30]] = True
    assert T.recall_counts(true_e, keep, 0.01) == (4, 10)


def test_early_rule_keeps_the_lowest_early_energies():
    from paper_2007_03678_gb300 import build
    build.build()
    cfg = T.TriageConfig()
    rng = np.random.default_rng(3)
    n = 200
    desc = rng.normal(size=(n, 16))
    tr = -np.sort(rng.uniform(0, 10, size=(n, cfg.nrun, cfg.early_gen)), axis=2)
    x = T.features(desc, tr, cfg.early_gen)
    keep = T.early_rule_survivors(x, cfg)
    best_early = tr[:, :, cfg.early_gen - 1].min(axis=1)
    assert keep.sum() == int(np.ceil(cfg.keep_frac * n))
    assert best_early[keep].max() <= best_early[~keep].min()


def test_mcnemar_exact_on_discordant_top_ligands():
    """Only top ligands where the two rules disagree count; the p-value is the
    two-sided exact binomial tail, checked against its closed forms: 0
    discordant gives 1, 5 to 0 gives 2/32, and 3 to 3 gives 1 (capped)."""
    true_e = np.arange(1000, dtype=float)  # ligands 0-9 are the top 1 %
    a = np.zeros(1000, bool)
    b = np.zeros(1000, bool)
    a[:10] = b[:10] = True
    r = T.mcnemar_exact(true_e, a, b, 0.01)
    assert (r["only_a"], r["only_b"], r["p_two_sided"]) == (0, 0, 1.0)
    b[:5] = False
    b[500:600] = True  # outside the top: ignored
    r = T.mcnemar_exact(true_e, a, b, 0.01)
    assert (r["only_a"], r["only_b"]) == (5, 0) and abs(r["p_two_sided"] - 2 / 32) < 1e-15
    a[:3] = False
    b[:3] = True
    a[3:6] = True
    b[3:6] = False
    r = T.mcnemar_exact(true_e, a, b, 0.01)
    assert (r["only_a"], r["only_b"]) == (3, 3) and r["p_two_sided"] == 1.0
    # symmetric in the two rules
    assert T.mcnemar_exact(true_e, b, a, 0.01)["p_two_sided"] == r["p_two_sided"]

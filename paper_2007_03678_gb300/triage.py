"""Learned triage of a ligand stream (no counterpart in the paper).

The plain path docks every ligand with the full search.  The triaged path
docks every ligand for the first `early_gen` generations only (a tenth of
the full search), predicts each ligand's final best energy with the networks
of adg_mlp_* from its descriptors and that early best-energy trace, and runs
the full search only for the best-predicted fraction of the stream.  A ligand keeps its random stream (adg_ligand_set_stream_id), so its
early generations are exactly the first generations of its full search and a
survivor's full docking is the plain path's result for it.

Everything numeric runs in libadg.so (docking, network training and
inference); this module arranges the calls and the host-side bookkeeping
(feature rows, the survival threshold).

Training records (descriptors, early trace, final best energy) come from the
plain path's own full dockings (adg_dock_traced reports the per-generation
trace of every run).
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import adg

NTRACE_FEATURES = 2  # per early generation: best over runs, mean over runs


@dataclass
class TriageConfig:
    nrun: int = 10
    pop: int = 150
    max_gen: int = 50          # the full search
    early_gen: int = 5         # the early search: the first tenth of the generations
    ls_max_iters: int = 20
    ls_method: int = adg.LS_ADADELTA
    seed: int = 42
    top_frac: float = 0.01     # the screen's hits: the best 1% by final energy
    keep_frac: float = 0.10    # full search for the best-predicted tenth of a stream
    epochs: int = 100
    batch: int = 64
    lr: float = 1e-3

    def params(self, generations: int) -> adg.adg_search_params:
        return adg.search_params(nrun=self.nrun, pop_size=self.pop, nev=2 ** 31 - 1, max_gen=generations,
                                 ls_method=self.ls_method, ls_max_iters=self.ls_max_iters, seed=self.seed)

    @property
    def nin(self) -> int:
        return adg.NDESC + NTRACE_FEATURES * self.early_gen


def assign_stream_ids(ligs, base: int):
    """Give ligand i the fixed random stream base + i (adg_ligand_set_stream_id)."""
    for i, l in enumerate(ligs):
        l.set_stream_id(base + i)


def _check_ids(ligs):
    if any(getattr(l, "stream_id", None) is None for l in ligs):
        raise ValueError("triage needs a fixed stream id per ligand (assign_stream_ids)")


def squash(e):
    """Monotone map of energies (kcal/mol) that keeps the bound region e <= 0
    as it is and compresses clashes, e > 0 -> log(1 + e): the screen ranks
    the bound region, and a run stuck at +1e4 must not dominate a mean or
    the training loss."""
    e = np.asarray(e, np.float64)
    return np.where(e > 0, np.log1p(np.maximum(e, 0.0)), e)


def features(desc: np.ndarray, best_trace: np.ndarray, early_gen: int) -> np.ndarray:
    """Network input rows: descriptors, then per early generation the best
    and the mean over runs of the (squashed) best energy after that
    generation.  desc [n, NDESC]; best_trace [n, nrun, >= early_gen]."""
    tr = squash(np.asarray(best_trace, np.float64)[:, :, :early_gen])
    return np.concatenate([np.asarray(desc, np.float64), tr.min(axis=1), tr.mean(axis=1)], axis=1).astype(np.float32)


def dock_full(ctx, rec, ligs, cfg: TriageConfig):
    """Plain path: full search of every ligand, with its trace.
    Returns (final best energy [n], early features [n, nin], evals, seconds)."""
    _check_ids(ligs)
    t0 = time.perf_counter()
    res = adg.dock(ctx, rec, ligs, cfg.params(cfg.max_gen), best_trace=cfg.early_gen)
    dt = time.perf_counter() - t0
    best = np.array([r["best_energy"].min() for r in res], np.float32)
    desc = np.stack([l.descriptors() for l in ligs])
    feats = features(desc, np.stack([r["best_trace"] for r in res]), cfg.early_gen)
    evals = int(sum(r["evals"].sum() for r in res))
    return best, feats, evals, dt


def dock_early(ctx, rec, ligs, cfg: TriageConfig):
    """Early search of every ligand.  Returns (features [n, nin], evals, seconds)."""
    _check_ids(ligs)
    t0 = time.perf_counter()
    res = adg.dock(ctx, rec, ligs, cfg.params(cfg.early_gen), best_trace=cfg.early_gen)
    dt = time.perf_counter() - t0
    desc = np.stack([l.descriptors() for l in ligs])
    feats = features(desc, np.stack([r["best_trace"] for r in res]), cfg.early_gen)
    return feats, int(sum(r["evals"].sum() for r in res)), dt


class Triage:
    """An ensemble of networks and the survival rule.

    fit() trains `folds` networks, each without one fold of the training
    records; their mean is the predictor, and each network's predictions on
    its held-out fold (out-of-fold predictions, kept in `oof`) estimate on the
    training set how the rule would do.  The rule keeps, of the ligands
    screened together, the fraction cfg.keep_frac with the lowest predicted
    final energy: the search budget of the rest is cut to the early search."""

    def __init__(self, ctx, cfg: TriageConfig, seed: int = 0, folds: int = 5):
        self.ctx = ctx
        self.cfg = cfg
        self.seed = seed
        self.folds = folds
        self.nets = []
        self.oof = None

    def _train(self, net, x: np.ndarray, energy: np.ndarray, seed: int) -> np.ndarray:
        import torch
        y = squash(energy)
        net.set_norm(x.mean(0), np.maximum(x.std(0), 1e-3), float(y.mean()), float(max(y.std(), 1e-3)))
        xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(self.ctx.device)
        yd = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda(self.ctx.device)
        return net.fit(xd, yd, batch=self.cfg.batch, epochs=self.cfg.epochs, lr=self.cfg.lr, seed=seed)

    def _predict_one(self, net, x: np.ndarray) -> np.ndarray:
        import torch
        xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(self.ctx.device)
        return net.forward(xd).cpu().numpy()

    def fit(self, x: np.ndarray, energy: np.ndarray) -> np.ndarray:
        """Train on feature rows x and final best energies (kcal/mol).
        Returns the loss per epoch of each network [folds, epochs]."""
        for net in self.nets:
            net.close()
        n = len(x)
        fold = np.arange(n) % self.folds
        self.oof = np.empty(n, np.float64)
        self.nets, hist = [], []
        for f in range(self.folds):
            net = adg.MLP(self.ctx, self.cfg.nin, seed=self.seed + 1 + f)
            hist.append(self._train(net, x[fold != f], energy[fold != f], self.seed + 101 + f))
            self.oof[fold == f] = self._predict_one(net, x[fold == f])
            self.nets.append(net)
        return np.array(hist)

    def predict(self, x: np.ndarray) -> np.ndarray:
        """Predicted final best energy (ensemble mean), in squashed units (see squash)."""
        return np.mean([self._predict_one(net, x) for net in self.nets], axis=0)

    def survivors(self, x: np.ndarray) -> np.ndarray:
        """The cfg.keep_frac of the rows with the lowest predicted energy."""
        if not self.nets:
            raise RuntimeError("fit() first")
        return keep_best(self.predict(x), self.cfg.keep_frac)


def keep_best(score: np.ndarray, frac: float) -> np.ndarray:
    """Mask of the ceil(frac * n) lowest scores (ties by index)."""
    k = int(np.ceil(frac * len(score)))
    keep = np.zeros(len(score), bool)
    keep[np.argsort(score, kind="stable")[:k]] = True
    return keep


def screen(ctx, rec, ligs, tri: Triage):
    """Triaged path over a stream: early search of all, prediction, full
    search of the survivors.  Returns a dict with the final best energies
    (NaN for ligands cut), the survivor mask, evaluations and seconds."""
    cfg = tri.cfg
    t0 = time.perf_counter()
    feats, ev_early, t_early = dock_early(ctx, rec, ligs, cfg)
    t1 = time.perf_counter()
    keep = tri.survivors(feats)
    t_pred = time.perf_counter() - t1
    energy = np.full(len(ligs), np.nan, np.float32)
    ev_full, t_full = 0, 0.0
    idx = np.nonzero(keep)[0]
    if len(idx):
        res = adg.dock(ctx, rec, [ligs[i] for i in idx], cfg.params(cfg.max_gen))
        t_full = time.perf_counter() - t1 - t_pred
        energy[idx] = [r["best_energy"].min() for r in res]
        ev_full = int(sum(r["evals"].sum() for r in res))
    return dict(energy=energy, keep=keep, evals=ev_early + ev_full, seconds=time.perf_counter() - t0,
                seconds_early=t_early, seconds_predict=t_pred, seconds_full=t_full)


def recall(true_energy: np.ndarray, keep: np.ndarray, top_frac: float) -> float:
    """Fraction of the plain path's top `top_frac` ligands that survive."""
    k = max(1, int(round(top_frac * len(true_energy))))
    top = np.argsort(true_energy, kind="stable")[:k]
    return float(keep[top].mean())


def recall_counts(true_energy: np.ndarray, keep: np.ndarray, top_frac: float) -> tuple:
    """(survivors among the plain path's top `top_frac`, their number)."""
    k = max(1, int(round(top_frac * len(true_energy))))
    top = np.argsort(true_energy, kind="stable")[:k]
    return int(keep[top].sum()), k


def wilson_interval(hits: int, n: int, z: float = 1.959963984540054) -> tuple:
    """Wilson score interval of a binomial proportion hits / n (95 % for the
    default z): the proportions p whose normal-approximation test
    |hits/n - p| <= z sqrt(p (1 - p) / n) does not reject, i.e. the roots of
    a quadratic in p."""
    if n <= 0:
        return (0.0, 1.0)
    ph = hits / n
    den = 1.0 + z * z / n
    mid = (ph + z * z / (2 * n)) / den
    half = z * np.sqrt(ph * (1.0 - ph) / n + z * z / (4.0 * n * n)) / den
    # at 0 or n hits one root is exactly 0 or 1 (kept exact, not rounded)
    return (0.0 if hits == 0 else max(0.0, mid - half), 1.0 if hits == n else min(1.0, mid + half))


def mcnemar_exact(true_energy: np.ndarray, keep_a: np.ndarray, keep_b: np.ndarray, top_frac: float) -> dict:
    """Paired comparison of two survival rules on the same top ligands:
    b = top ligands only rule a keeps, c = only rule b keeps; under the null
    hypothesis (equal recall) each discordant ligand falls either way with
    probability 1/2, so the two-sided exact p-value is
    min(1, 2 P(X <= min(b, c))), X ~ Binomial(b + c, 1/2)."""
    from math import comb
    k = max(1, int(round(top_frac * len(true_energy))))
    top = np.argsort(true_energy, kind="stable")[:k]
    a, bb = np.asarray(keep_a)[top], np.asarray(keep_b)[top]
    b, c = int((a & ~bb).sum()), int((~a & bb).sum())
    n = b + c
    tail = sum(comb(n, i) for i in range(min(b, c) + 1)) / 2.0 ** n if n else 1.0
    return {"only_a": b, "only_b": c, "p_two_sided": min(1.0, 2.0 * tail)}


def early_rule_survivors(feats: np.ndarray, cfg: TriageConfig) -> np.ndarray:
    """The same survival fraction chosen without the network: the ligands
    whose best early energy (over runs, after the early generations; the
    feature column of the last early generation) is lowest."""
    col = adg.NDESC + cfg.early_gen - 1
    return keep_best(np.asarray(feats, np.float64)[:, col], cfg.keep_frac)

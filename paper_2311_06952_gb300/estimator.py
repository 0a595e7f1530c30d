"""A fit / predict interface over the C ABI (MH-DEOCT and DEOCT classifiers).

Marshalling and orchestration only: encoding, the moving-horizon fit, the raw
thresholds and the prediction all run in libdeoct's kernels.

Presets follow Section 5 of the paper: "normal" is population 100, 600
generations, CR 0.1, M = rand(0,1) per individual (dithered); "long" is
population 200 and 4000 generations.  The moving-horizon depth defaults to 2
for depth-2 trees and 3 otherwise (Section 5.2).
"""
from __future__ import annotations

import numpy as np

PRESETS = {
    "normal": dict(pop=100, gens=600, cr=0.1, mut_f=0.5, dither=True),
    "long": dict(pop=200, gens=4000, cr=0.1, mut_f=0.5, dither=True),
}


class MHDEOCTClassifier:
    """Moving-horizon DEOCT (Algorithm 2).  ``horizon >= depth`` is plain DEOCT
    of the whole tree at the root, kept node by node.  ``warm_starts`` selects
    the warm starts of Algorithm 2 ("cart", "deoct"; the paper uses both)."""

    def __init__(self, depth=3, horizon=None, preset="normal", pop=None, gens=None, cr=None, mut_f=None,
                 dither=None, alpha=0.0, n_min=1, seed=0, batched=True, warm_starts=("cart", "deoct"),
                 device=0):
        p = dict(PRESETS[preset])
        for k, v in dict(pop=pop, gens=gens, cr=cr, mut_f=mut_f, dither=dither).items():
            if v is not None:
                p[k] = v
        self.depth = int(depth)
        self.horizon = int(horizon) if horizon is not None else (2 if depth == 2 else 3)
        self.params = p
        self.alpha, self.n_min, self.seed = float(alpha), int(n_min), int(seed)
        self.batched = bool(batched)
        self.warm_starts = tuple(warm_starts or ())  # Algorithm 2: CART and DEOCT warm starts
        self.device = device
        self.tree_ = None
        self._ctx = None

    def _context(self):
        from . import deoct
        if self._ctx is None:
            self._ctx = deoct.Context(self.device)
        return self._ctx

    @staticmethod
    def _dev(a, dtype):
        import torch
        if isinstance(a, torch.Tensor):
            return a.to(device="cuda", dtype=dtype).contiguous()
        return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype).contiguous()

    def fit(self, X, y, K=None):
        import torch

        from . import deoct
        ctx = self._context()
        Xd = self._dev(X, torch.float32)
        yd = self._dev(y, torch.uint8)
        n, F = Xd.shape
        K = int(K) if K is not None else int(yd.max().item()) + 1
        # uint16 ranks whenever every feature has at most 65536 distinct values
        ranks, nu, uniq, rank_bytes = deoct.deoct_encode_auto(ctx, Xd)
        ds = deoct.DeviceDataset(ranks, rank_bytes, nu, yd, n, F, K)
        flags = (deoct.DEOCT_BATCHED if self.batched else 0) | \
            (deoct.DEOCT_DITHER_M if self.params["dither"] else 0) | \
            (deoct.DEOCT_CART_SEEDS if "cart" in self.warm_starts else 0) | \
            (deoct.DEOCT_DE_SEEDS if "deoct" in self.warm_starts else 0)
        prm = deoct.make_params(self.depth, self.params["pop"], self.params["gens"],
                                mut_f=self.params["mut_f"], cr=self.params["cr"], alpha=self.alpha,
                                n_min=self.n_min, seed=self.seed, horizon=self.horizon, flags=flags)
        out = deoct.deoct_fit_moving_horizon(ctx, ds, prm)
        a = torch.from_numpy(out["a"].view(np.int16)).cuda()
        th = torch.from_numpy(out["theta"].view(np.int32)).cuda()
        b = deoct.deoct_split_values(ctx, uniq, a, th)
        self.tree_ = dict(out, b=b.cpu().numpy(), K=K, F=F)
        self._dev_tree = (a, b, torch.from_numpy(out["leaf_class"]).cuda())
        return self

    def fit_tuned(self, X, y, K=None, n_grid=21, val_frac=1.0 / 3.0, split_seed=0):
        """Complexity-parameter tuning by training, validation and retraining (the
        procedure of the paper's Appendix C, 21 values of the parameter).

        The paper does not state alpha's domain.  Here alpha = cp * e_root, with e_root
        the misclassifications of the tree without splits on the set being fitted and cp
        taking n_grid values evenly spaced in [0, 1] (a split must then pay for itself
        with at least cp * e_root corrected samples).  The training set is split once
        (seeded) into a fitting part and a validation part of val_frac (the paper's
        50/25 split of train+validation is val_frac = 1/3); every cp is fitted on the
        fitting part and scored on the validation part; the cp with the highest
        validation accuracy wins, ties going to the larger cp (the simpler tree); the
        tree is then refitted on the whole training set with that cp."""
        Xh = np.ascontiguousarray(X if isinstance(X, np.ndarray) else X.cpu().numpy(), np.float32)
        yh = np.ascontiguousarray(y if isinstance(y, np.ndarray) else y.cpu().numpy(), np.uint8)
        K = int(K) if K is not None else int(yh.max()) + 1
        fit_idx, val_idx = validation_split(len(yh), val_frac, split_seed)
        cps = np.linspace(0.0, 1.0, n_grid)
        e_fit = root_errors(yh[fit_idx], K)
        acc = []
        for cp in cps:
            self.alpha = float(cp * e_fit)
            self.fit(Xh[fit_idx], yh[fit_idx], K=K)
            acc.append(self.score(Xh[val_idx], yh[val_idx]))
        acc = np.asarray(acc)
        best = int(np.flatnonzero(acc == acc.max())[-1])  # ties: the larger cp
        self.alpha = float(cps[best] * root_errors(yh, K))
        self.fit(Xh, yh, K=K)
        self.tuning_ = dict(cp=cps, val_accuracy=acc, cp_best=float(cps[best]), alpha=self.alpha,
                            fit_idx=fit_idx, val_idx=val_idx)
        return self

    def predict(self, X):
        import torch

        from . import deoct
        a, b, lc = self._dev_tree
        pred, _ = deoct.deoct_predict(self._context(), self._dev(X, torch.float32), a, b, self.depth, lc)
        return pred.cpu().numpy()

    def score(self, X, y):
        import torch

        from . import deoct
        a, b, lc = self._dev_tree
        Xd = self._dev(X, torch.float32)
        _, correct = deoct.deoct_predict(self._context(), Xd, a, b, self.depth, lc,
                                         y=self._dev(y, torch.uint8))
        return int(correct.item()) / Xd.shape[0]


def validation_split(n, val_frac, seed):
    """Seeded split of n samples into (fitting, validation) index arrays, each sorted."""
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(n)
    nv = int(round(n * val_frac))
    return np.sort(perm[nv:]), np.sort(perm[:nv])


def root_errors(y, K):
    """Misclassifications of the tree without splits: n minus the majority class count."""
    return int(len(y) - np.bincount(y, minlength=K).max())

"""Learned warm start for star (barycenter) problems.

An MLP maps one fixed leaf's marginal mu_l (n values) and eps to the leaf's
potential f_(l,c) on the leaf-centre edge, in cost units and in the gauge
mean_x f_(l,c)(x) = 0 (the plans do not depend on the gauge).  A solve starts
from the predicted leaf potentials; the first half-step updates the centre
(colour of node 0) from them.  Problems that do not converge within the cap
fall back to the plain start u = 1.

This module only moves data between the solver and the network: the network's
forward / backward / Adam kernels and the solver run in libtreeot.so.
"""
from __future__ import annotations

import math
import time
from typing import List, Sequence

import numpy as np

from .treeot import MLP, Solver, options

LOG_FLOOR = 1e-30
LOG_SCALE = 1.0 / 16.0
EPS_SHIFT = 5.0  # the last input is log(eps) + EPS_SHIFT


def leaf_edges(p) -> List[int]:
    """Directed-edge index (leaf -> centre) of every fixed leaf of a star rooted at node 0."""
    out = []
    for e, (a, b) in enumerate(np.asarray(p.edges)):
        if int(a) == 0 and p.fixed[int(b)]:
            out.append(2 * e + 1)
        elif int(b) == 0 and p.fixed[int(a)]:
            out.append(2 * e)
    return out


def leaf_of(p, dedge: int) -> int:
    a, b = np.asarray(p.edges)[dedge // 2]
    return int(b) if dedge % 2 == 1 else int(a)


def leaf_items(problems: Sequence):
    """(problem index, directed edge leaf -> centre) of every fixed leaf, in the row order of inputs()."""
    pr, de = [], []
    for i, p in enumerate(problems):
        for d in leaf_edges(p):
            pr.append(i)
            de.append(d)
    return np.asarray(pr, np.int32), np.asarray(de, np.int32)


def inputs(problems: Sequence) -> np.ndarray:
    """Rows [mu_l (n), log(eps) + EPS_SHIFT], one per fixed leaf, FP32."""
    mus, eps = [], []
    for p in problems:
        for d in leaf_edges(p):
            mus.append(p.marginals[leaf_of(p, d)])
            eps.append(math.log(p.eps) + EPS_SHIFT)
    out = np.empty((len(mus), len(mus[0]) + 1), np.float32)
    out[:, :-1] = np.asarray(mus, np.float32)
    out[:, -1] = eps
    return out


def targets(solver: Solver, problems: Sequence, device="cuda"):
    """Leaf potentials of solved problems in the gauge mean_x f = 0: a CUDA float32
    matrix, rows in the order of inputs() (read on the device, no host copy)."""
    import torch
    pr, de = leaf_items(problems)
    n = int(np.asarray(problems[0].n)[leaf_of(problems[0], int(de[0]))])
    out = torch.empty((len(pr), n), dtype=torch.float32, device=device)
    return solver.get_potentials_batch(pr, de, out, centred=True)


class WarmStart:
    def __init__(self, n: int, hidden: int = 512, max_batch: int = 256, seed: int = 0):
        self.n = n
        self.max_batch = max_batch
        self.net = MLP(n + 1, hidden, n, max_batch, seed)
        self.net.set_input_log(n, LOG_FLOOR, LOG_SCALE)

    def close(self):
        self.net.close()

    def train(self, X: np.ndarray, Y: np.ndarray, epochs: int = 20, batch: int = 256, lr: float = 1e-3,
              seed: int = 0, device="cuda") -> List[float]:
        """Adam with a cosine learning-rate schedule; returns the mean loss per epoch."""
        import torch
        Xd = X if isinstance(X, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(X))
        Yd = Y if isinstance(Y, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(Y))
        Xd, Yd = Xd.to(device), Yd.to(device)
        rng = np.random.default_rng(seed)
        N = X.shape[0]
        batch = min(batch, self.max_batch)
        steps_per_epoch = max(1, N // batch)
        total = epochs * steps_per_epoch
        hist, k = [], 0
        for ep in range(epochs):
            perm = torch.from_numpy(rng.permutation(N)).to(device)
            acc = 0.0
            for s in range(steps_per_epoch):
                idx = perm[s * batch:(s + 1) * batch]
                lr_k = 0.5 * lr * (1.0 + math.cos(math.pi * k / total))
                acc += self.net.train_step(Xd.index_select(0, idx).contiguous(), Yd.index_select(0, idx).contiguous(),
                                           lr_k)
                k += 1
            hist.append(acc / steps_per_epoch)
        return hist

    def predict_device(self, X: np.ndarray, device="cuda"):
        """Network outputs for the rows of X as a CUDA float32 tensor."""
        import torch
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(device)
        out = torch.empty((X.shape[0], self.n), dtype=torch.float32, device=device)
        for s in range(0, X.shape[0], self.max_batch):
            e = min(s + self.max_batch, X.shape[0])
            self.net.forward(Xd[s:e], out[s:e])
        return out

    def predict(self, X: np.ndarray, device="cuda") -> np.ndarray:
        return self.predict_device(X, device).cpu().numpy()

    def warm_solve(self, problems: Sequence, tol: float = 1e-6, max_half_steps: int = 20000, timing=None, **kw):
        """Solve every problem from predicted leaf potentials (set on the device, no
        host round trip); problems that do not converge restart from u = 1.
        Returns (results, fallbacks, seconds); `timing` (a dict) receives the split:
        create, predict (inputs + network + set), solve, fallback."""
        t0 = time.perf_counter()
        s = Solver(problems, options(tol=tol, tol_kind="max", max_half_steps=max_half_steps, **kw))
        t1 = time.perf_counter()
        pred = self.predict_device(inputs(problems))
        pr, de = leaf_items(problems)
        s.set_potentials_batch(pr, de, pred)
        t2 = time.perf_counter()
        rc, res = s.solve()
        t3 = time.perf_counter()
        s.close()
        # fall back when the warm start failed (cap reached far from tol, or not finite); a
        # problem whose FP32 accuracy floor sits just above tol would not gain from u = 1
        bad = [i for i, x in enumerate(res)
               if not np.isfinite(x["max_marginal_l1"]) or (x["status"] != 0 and x["max_marginal_l1"] > 10 * tol)]
        if bad:
            s0 = Solver([problems[i] for i in bad],
                        options(tol=tol, tol_kind="max", max_half_steps=max_half_steps, **kw))
            _, res0 = s0.solve()
            s0.close()
            for i, x in zip(bad, res0):
                x["half_steps"] += res[i]["half_steps"]
                res[i] = x
        t4 = time.perf_counter()
        if timing is not None:
            timing.update(create=t1 - t0, predict=t2 - t1, solve=t3 - t2, fallback=t4 - t3)
        return res, len(bad), t4 - t0


def zero_solve(problems: Sequence, tol: float = 1e-6, max_half_steps: int = 20000, timing=None, **kw):
    """Plain start u = 1; returns (results, solver, seconds) with the solver still open;
    `timing` (a dict) receives create and solve seconds."""
    t0 = time.perf_counter()
    s = Solver(problems, options(tol=tol, tol_kind="max", max_half_steps=max_half_steps, **kw))
    t1 = time.perf_counter()
    rc, res = s.solve()
    if timing is not None:
        timing.update(create=t1 - t0, solve=time.perf_counter() - t1)
    return res, s, time.perf_counter() - t0

"""Coupled MOT on a modified junction tree (Sec. 4) as a tree problem of Sec. 3.

Host-side reformulation only (no solver arithmetic): when every separator's
neighbour cliques intersect it in the whole separator (the trivial inclusion
sequence of Assumption ass:inclusion), every clique's variables are the disjoint
union of its two separators' variables, and every constraint covers a whole
separator, then the problem of eq. ot_graph_local_reg is the tree problem of eq.
ot_graph_pairwise_mass on the separators: each separator is a node whose support
is the product of its variables' supports, each clique an edge whose cost matrix
is the clique's cost tensor with the two separators' variables as rows and
columns, and the reference measures of prop:local_reg_dual are the tree's
gamma_j (x) gamma_k.  The separator update of prop:general_algo with equal
intersections is then the tree's free-node update, so the library's kernels
solve it as they stand.  The Wasserstein least-squares example of Sec. 2.3 and
Sec. 5 is of this kind.  Nested inclusion sequences (a separator meeting some of
its cliques in proper subsets) do not reduce this way and are rejected.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np


class NotReducible(ValueError):
    """The junction tree is not a tree of separators with product supports."""


@dataclass
class SeparatorTree:
    """The tree problem of a reducible modified junction tree, in the shape the
    Solver reads (dense FP32 costs per edge, rows on edges[e][0])."""

    name: str
    edges: np.ndarray
    n: np.ndarray
    fixed: np.ndarray
    marginals: Dict[int, np.ndarray]
    eps: float
    dense_costs: List[np.ndarray]
    sep_vars: List[tuple]
    edge_clique: List[int]
    coords: List[np.ndarray] = field(default_factory=list)
    cost_scale: float = 1.0
    cost_kind: str = "dense"
    meta: Dict = field(default_factory=dict)

    @property
    def num_nodes(self) -> int:
        return int(self.n.shape[0])

    @property
    def num_edges(self) -> int:
        return int(self.edges.shape[0])

    def dense_cost(self, e: int) -> np.ndarray:
        return self.dense_costs[e]

    def elements_per_half_step(self) -> int:
        return int(sum(int(self.n[a]) * int(self.n[b]) for a, b in self.edges))


def reduce_junction_tree(jt) -> SeparatorTree:
    """The separator tree of ``jt`` (a gen.JunctionTreeProblem-like object: d,
    clique_vars, clique_costs, sep_vars, sep_cliques, sep_gamma, sep_mu, eps)."""
    S = len(jt.sep_vars)
    cl_seps: List[List[int]] = [[] for _ in jt.clique_vars]
    for s, cl in enumerate(jt.sep_cliques):
        for c in cl:
            cl_seps[c].append(s)
    for s, cl in enumerate(jt.sep_cliques):
        sv = set(jt.sep_vars[s])
        for c in cl:
            if not sv <= set(jt.clique_vars[c]):
                raise NotReducible(f"separator {s} meets clique {c} in a proper subset (nested inclusion)")
        g = jt.sep_gamma[s]
        if g is not None and set(g) != sv:
            raise NotReducible(f"separator {s}: the constraint covers only part of it")
    edges, costs, edge_clique = [], [], []
    for c, seps in enumerate(cl_seps):
        if len(seps) != 2:
            raise NotReducible(f"clique {c} must join exactly two separators")
        a, b = seps
        va, vb = tuple(jt.sep_vars[a]), tuple(jt.sep_vars[b])
        cv = tuple(jt.clique_vars[c])
        if set(va) & set(vb) or set(va) | set(vb) != set(cv):
            raise NotReducible(f"clique {c}: its variables are not the disjoint union of its separators'")
        order = [cv.index(v) for v in va + vb]
        C = np.transpose(np.asarray(jt.clique_costs[c], dtype=np.float64), order)
        na = int(np.prod([int(jt.d[v]) for v in va]))
        nb = int(np.prod([int(jt.d[v]) for v in vb]))
        edges.append((a, b))
        costs.append(np.ascontiguousarray(C.reshape(na, nb).astype(np.float32)))
        edge_clique.append(c)
    if len(edges) != S - 1:
        raise NotReducible("the separators and cliques do not form a tree")
    n = np.array([int(np.prod([int(jt.d[v]) for v in jt.sep_vars[s]])) for s in range(S)], np.int32)
    fixed = np.array([jt.sep_gamma[s] is not None for s in range(S)], bool)
    marg = {}
    for s in range(S):
        if fixed[s]:
            g = tuple(jt.sep_gamma[s])
            order = [g.index(v) for v in jt.sep_vars[s]]
            marg[s] = np.ascontiguousarray(np.transpose(np.asarray(jt.sep_mu[s], np.float64), order).reshape(-1))
    # dense costs carry no geometry: one index coordinate per support point, same dimension everywhere
    coords = [np.arange(int(n[s]), dtype=np.float32).reshape(-1, 1) for s in range(S)]
    return SeparatorTree(name=getattr(jt, "name", "jt") + "_septree", edges=np.asarray(edges, np.int32), n=n,
                         fixed=fixed, marginals=marg, eps=float(jt.eps), dense_costs=costs,
                         sep_vars=[tuple(v) for v in jt.sep_vars], edge_clique=edge_clique, coords=coords,
                         meta=dict(getattr(jt, "meta", {})))


def clique_plan(tree: SeparatorTree, jt, e: int, plan: np.ndarray) -> np.ndarray:
    """An edge's plan (n_a x n_b, rows on edges[e][0]) as the clique's tensor (axes in
    the clique's variable order)."""
    c = tree.edge_clique[e]
    a, b = (int(x) for x in tree.edges[e])
    va, vb = tree.sep_vars[a], tree.sep_vars[b]
    shape = [int(jt.d[v]) for v in va + vb]
    T = np.asarray(plan).reshape(shape)
    cv = tuple(jt.clique_vars[c])
    src = list(va + vb)
    return np.transpose(T, [src.index(v) for v in cv])

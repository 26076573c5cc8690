"""Seeded synthetic problem instances for tree-structured coupled OT.

This module only builds *inputs*: tree topologies, support points, fixed
marginals and (for the stored-cost form) dense cost matrices.  It holds none of
the solver's arithmetic (no kernels, messages, potentials or updates), so both
the CUDA path and the CPU oracle can read the very same arrays.

Workloads follow the paper's numerical section (Sec. 5: squared-Euclidean
costs, probability vectors on a uniform grid in [0,1]) and the five workload
shapes this project is measured on:

* ``chain_problem``   -- 5-node chain, n=64 uniform 1-D grid, |x-y|^2, eps=0.01,
  two fixed end nodes with 2-component Gaussian mixtures.
* ``star_problem``    -- barycenter star: 8 fixed leaves on a 32x32 grid, a free
  centre on the same grid, squared-Euclidean cost normalised to max 1,
  eps=0.005, 3-component mixtures.
* ``prufer_problem``  -- 64-node random tree from a Pruefer sequence with exactly
  32 leaves, n=4096 points U[0,1]^3 per node, dense FP32 cost per edge,
  Dirichlet(1) leaf marginals, eps=0.01.
* ``batched_problems`` -- 512 random trees with 4..32 nodes, n_j uniform in
  {128..2048}, 2-D uniform points, eps log-uniform in [0.002, 0.05].
* ``star_problem`` with other seeds/eps -- the warm-start training/test sets.
* ``lognormal_barycenter`` -- the paper's own experiment (Sec. 5, Fig. 4(a)):
  |E| fixed leaves and a free centre on a uniform grid of d points in [0,1],
  squared-Euclidean cost, log-normal marginals, eps = delta / (4 |E| log d).

Every generator takes a ``seed``; by convention ``seed = 1000*workload + instance``.
All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

COST_SQEUCLID = "sqeuclid"
COST_DENSE = "dense"


@dataclass
class TreeProblem:
    """One coupled bi-marginal OT problem on a tree (the problem of Sec. 3).

    Attributes
    ----------
    edges : int32 [J-1, 2]; edge e joins ``edges[e,0]`` and ``edges[e,1]``.
        Its cost matrix is indexed [support of edges[e,0], support of edges[e,1]].
    n : int32 [J]; support size n_j of every node.
    fixed : bool [J]; True for the nodes in Gamma (given marginals).
    marginals : node -> float64 [n_j] probability vector, fixed nodes only.
    eps : entropic regularisation epsilon.
    coords : per node float32 [n_j, D] support points.
    cost_scale : the cost is ``cost_scale * ||x - y||^2`` between support points.
    cost_kind : ``"sqeuclid"`` (the solver recomputes C from ``coords``) or
        ``"dense"`` (the solver reads a stored FP32 matrix per edge; the matrix
        is the FP64 value of the formula above rounded once to FP32).
    dense_costs : optional list of float32 [n_a, n_b] per edge; filled lazily by
        ``dense_cost(e)`` when ``cost_kind == "dense"``.
    """

    name: str
    edges: np.ndarray
    n: np.ndarray
    fixed: np.ndarray
    marginals: Dict[int, np.ndarray]
    eps: float
    coords: List[np.ndarray]
    cost_scale: float
    cost_kind: str = COST_SQEUCLID
    dense_costs: Optional[List[Optional[np.ndarray]]] = None
    meta: dict = field(default_factory=dict)

    @property
    def num_nodes(self) -> int:
        return int(self.n.shape[0])

    @property
    def num_edges(self) -> int:
        return int(self.edges.shape[0])

    @property
    def dim(self) -> int:
        return int(self.coords[0].shape[1])

    def dense_cost(self, e: int) -> np.ndarray:
        """FP32 dense cost of edge e (rows: edges[e,0]); cached after first use."""
        if self.dense_costs is None:
            self.dense_costs = [None] * self.num_edges
        if self.dense_costs[e] is None:
            a, b = int(self.edges[e, 0]), int(self.edges[e, 1])
            self.dense_costs[e] = sqeuclid_cost_f32(self.coords[a], self.coords[b], self.cost_scale)
        return self.dense_costs[e]

    def elements_per_half_step(self) -> int:
        """Sum over edges of n_a * n_b (each half-step touches every edge once)."""
        return int(sum(int(self.n[a]) * int(self.n[b]) for a, b in self.edges))


# --------------------------------------------------------------------------
# cost matrices (problem data, FP64 arithmetic rounded once to FP32)
# --------------------------------------------------------------------------

def sqeuclid_cost_f32(xa: np.ndarray, xb: np.ndarray, scale: float, rows=None) -> np.ndarray:
    """``float32(scale * sum_d (xa_d - xb_d)^2)`` evaluated in FP64.

    The operation order (difference, square, running sum over d, then the
    scale) is fixed so that the torch version below yields identical bits.
    ``rows`` optionally selects a subset of rows of the result.
    """
    A = np.asarray(xa, dtype=np.float64)
    if rows is not None:
        A = A[np.asarray(rows)]
    B = np.asarray(xb, dtype=np.float64)
    acc = None
    for d in range(A.shape[1]):
        diff = A[:, d][:, None] - B[:, d][None, :]
        sq = diff * diff
        acc = sq if acc is None else acc + sq
    if scale != 1.0:
        acc = acc * scale
    return acc.astype(np.float32)


def sqeuclid_cost_f32_torch(xa, xb, scale: float, device):
    """Same values as ``sqeuclid_cost_f32``, built with torch on ``device``.

    Separate elementwise ops (no fused multiply-add) in FP64, then one rounding
    to FP32, so the result matches the numpy version bit for bit.
    """
    import torch

    A = torch.as_tensor(np.asarray(xa), device=device).to(torch.float64)
    B = torch.as_tensor(np.asarray(xb), device=device).to(torch.float64)
    acc = None
    for d in range(A.shape[1]):
        diff = A[:, d].unsqueeze(1) - B[:, d].unsqueeze(0)
        sq = diff * diff
        acc = sq if acc is None else acc + sq
        del diff, sq
    if scale != 1.0:
        acc = acc * scale
    out = acc.to(torch.float32)
    del acc
    return out


# --------------------------------------------------------------------------
# topologies
# --------------------------------------------------------------------------

def chain_edges(J: int) -> np.ndarray:
    return np.array([[i, i + 1] for i in range(J - 1)], dtype=np.int32).reshape(-1, 2)


def star_edges(L: int) -> np.ndarray:
    """Centre node 0 joined to leaves 1..L."""
    return np.array([[0, l] for l in range(1, L + 1)], dtype=np.int32).reshape(-1, 2)


def pruefer_decode(seq) -> np.ndarray:
    """Tree on labels 0..len(seq)+1 encoded by a Pruefer sequence (standard decoding)."""
    import heapq

    seq = [int(s) for s in seq]
    J = len(seq) + 2
    degree = [1] * J
    for s in seq:
        degree[s] += 1
    heap = [v for v in range(J) if degree[v] == 1]
    heapq.heapify(heap)
    edges = []
    for s in seq:
        leaf = heapq.heappop(heap)
        edges.append((leaf, s))
        degree[leaf] -= 1
        degree[s] -= 1
        if degree[s] == 1:
            heapq.heappush(heap, s)
    u = heapq.heappop(heap)
    v = heapq.heappop(heap)
    edges.append((u, v))
    return np.array(edges, dtype=np.int32)


def pruefer_tree_with_leaves(J: int, num_leaves: int, rng) -> np.ndarray:
    """Random tree on J labels with exactly ``num_leaves`` leaves.

    A label is a leaf iff it is absent from the Pruefer sequence, so the
    sequence (length J-2) holds every one of the J-num_leaves interior labels
    at least once, plus uniform draws from the interior set, shuffled.
    """
    if not (2 <= num_leaves <= J - 1) and J > 2:
        raise ValueError("num_leaves out of range")
    interior = rng.choice(J, size=J - num_leaves, replace=False)
    extra = rng.choice(interior, size=(J - 2) - (J - num_leaves), replace=True)
    seq = np.concatenate([interior, extra])
    rng.shuffle(seq)
    return pruefer_decode(seq)


def uniform_pruefer_tree(J: int, rng) -> np.ndarray:
    if J == 2:
        return np.array([[0, 1]], dtype=np.int32)
    return pruefer_decode(rng.integers(0, J, size=J - 2))


def leaves_of(J: int, edges: np.ndarray) -> np.ndarray:
    deg = np.bincount(edges.reshape(-1), minlength=J)
    return deg == 1


# --------------------------------------------------------------------------
# supports and marginals
# --------------------------------------------------------------------------

def grid_1d(n: int) -> np.ndarray:
    """x_i = i/(n-1), i = 0..n-1 (endpoints included), float32 [n, 1]."""
    return (np.arange(n, dtype=np.float64) / (n - 1)).astype(np.float32).reshape(n, 1)


def grid_2d(side: int) -> np.ndarray:
    """Tensor grid (i/(side-1), j/(side-1)), row-major in (i, j), float32 [side^2, 2]."""
    t = np.arange(side, dtype=np.float64) / (side - 1)
    X, Y = np.meshgrid(t, t, indexing="ij")
    return np.stack([X.reshape(-1), Y.reshape(-1)], axis=1).astype(np.float32)


def gaussian_mixture(points: np.ndarray, rng, n_comp: int,
                     sigma_range=(0.05, 0.15), mean_range=(0.15, 0.85)) -> np.ndarray:
    """Isotropic Gaussian-mixture density at the support points, normalised (FP64)."""
    P = np.asarray(points, dtype=np.float64)
    D = P.shape[1]
    w = rng.dirichlet(np.ones(n_comp))
    means = rng.uniform(mean_range[0], mean_range[1], size=(n_comp, D))
    sig = rng.uniform(sigma_range[0], sigma_range[1], size=n_comp)
    dens = np.zeros(P.shape[0])
    for c in range(n_comp):
        r2 = np.sum((P - means[c]) ** 2, axis=1)
        dens += w[c] * np.exp(-r2 / (2.0 * sig[c] ** 2)) / (2.0 * np.pi * sig[c] ** 2) ** (D / 2.0)
    return dens / dens.sum()


def dirichlet_marginal(n: int, rng) -> np.ndarray:
    mu = rng.dirichlet(np.ones(n))
    return mu / mu.sum()


def _check_fixed_leaves(J, edges, fixed):
    deg = np.bincount(edges.reshape(-1), minlength=J)
    assert all(deg[j] == 1 for j in range(J) if fixed[j])


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def chain_problem(seed: int = 1000, J: int = 5, n: int = 64, eps: float = 0.01,
                  n_comp: int = 2, cost_kind: str = COST_DENSE) -> TreeProblem:
    """Chain 0-1-...-(J-1); ends fixed with mixtures on the grid i/(n-1); C=|x-y|^2."""
    rng = np.random.default_rng(seed)
    edges = chain_edges(J)
    x = grid_1d(n)
    fixed = np.zeros(J, dtype=bool)
    fixed[0] = fixed[J - 1] = True
    marg = {0: gaussian_mixture(x, rng, n_comp), J - 1: gaussian_mixture(x, rng, n_comp)}
    return TreeProblem(name=f"chain{J}_n{n}", edges=edges, n=np.full(J, n, np.int32), fixed=fixed,
                       marginals=marg, eps=eps, coords=[x] * J, cost_scale=1.0, cost_kind=cost_kind,
                       meta={"seed": seed})


def star_problem(seed: int = 2000, leaves: int = 8, side: int = 32, eps: float = 0.005,
                 n_comp: int = 3, cost_kind: str = COST_SQEUCLID) -> TreeProblem:
    """Barycenter star: centre 0 (free), leaves 1..L fixed, all on the side x side grid.

    The squared-Euclidean cost is normalised to max 1 on [0,1]^2 (scale 1/2).
    """
    rng = np.random.default_rng(seed)
    edges = star_edges(leaves)
    x = grid_2d(side)
    J = leaves + 1
    fixed = np.ones(J, dtype=bool)
    fixed[0] = False
    marg = {l: gaussian_mixture(x, rng, n_comp) for l in range(1, J)}
    return TreeProblem(name=f"star{leaves}_grid{side}", edges=edges, n=np.full(J, side * side, np.int32),
                       fixed=fixed, marginals=marg, eps=eps, coords=[x] * J, cost_scale=0.5,
                       cost_kind=cost_kind, meta={"seed": seed})


def prufer_problem(seed: int = 3000, J: int = 64, n: int = 4096, num_leaves: int = 32, D: int = 3,
                   eps: float = 0.01, cost_kind: str = COST_DENSE) -> TreeProblem:
    """Random Pruefer tree with exactly ``num_leaves`` fixed leaves; points U[0,1]^D."""
    rng = np.random.default_rng(seed)
    edges = pruefer_tree_with_leaves(J, num_leaves, rng)
    fixed = leaves_of(J, edges)
    coords = [rng.random((n, D)).astype(np.float32) for _ in range(J)]
    marg = {j: dirichlet_marginal(n, rng) for j in range(J) if fixed[j]}
    _check_fixed_leaves(J, edges, fixed)
    return TreeProblem(name=f"prufer{J}_n{n}", edges=edges, n=np.full(J, n, np.int32), fixed=fixed,
                       marginals=marg, eps=eps, coords=coords, cost_scale=1.0, cost_kind=cost_kind,
                       meta={"seed": seed})


def random_tree_problem(rng, J: int, n_range=(128, 2048), eps_range=(0.002, 0.05), D: int = 2,
                        name: str = "tree") -> TreeProblem:
    """One tree of the batched workload: uniform Pruefer tree, leaves fixed (1-3 comp mixtures)."""
    edges = uniform_pruefer_tree(J, rng)
    fixed = leaves_of(J, edges)
    n = rng.integers(n_range[0], n_range[1] + 1, size=J).astype(np.int32)
    coords = [rng.random((int(n[j]), D)).astype(np.float32) for j in range(J)]
    eps = float(np.exp(rng.uniform(np.log(eps_range[0]), np.log(eps_range[1]))))
    marg = {}
    for j in range(J):
        if fixed[j]:
            marg[j] = gaussian_mixture(coords[j], rng, int(rng.integers(1, 4)))
    _check_fixed_leaves(J, edges, fixed)
    return TreeProblem(name=name, edges=edges, n=n, fixed=fixed, marginals=marg, eps=eps, coords=coords,
                       cost_scale=1.0, cost_kind=COST_SQEUCLID, meta={})


def warmstart_stars(seed0: int, count: int, side: int = 32, leaves: int = 8, eps_range=(0.0025, 0.01),
                    eps: float = None) -> List[TreeProblem]:
    """Barycenter stars of the star generator for the learned warm start: star i
    uses seed seed0 + i; eps is log-uniform in eps_range (training) unless fixed."""
    out = []
    for i in range(count):
        e = eps
        if e is None:
            rng = np.random.default_rng(seed0 + i + 7_000_000)
            e = float(np.exp(rng.uniform(np.log(eps_range[0]), np.log(eps_range[1]))))
        out.append(star_problem(seed=seed0 + i, leaves=leaves, side=side, eps=e))
    return out


def batched_problems(seed: int = 4000, num_trees: int = 512, J_range=(4, 32), n_range=(128, 2048),
                     eps_range=(0.002, 0.05)) -> List[TreeProblem]:
    rng = np.random.default_rng(seed)
    out = []
    for i in range(num_trees):
        J = int(rng.integers(J_range[0], J_range[1] + 1))
        out.append(random_tree_problem(rng, J, n_range, eps_range, name=f"batch{i}_J{J}"))
    return out


WORKLOADS = {
    "chain5_n64_eps0.01": "chain_problem",
    "star8_grid32_eps0.005": "star_problem",
    "prufer64_n4096_dense": "prufer_problem",
    "batched512_trees": "batched_problems",
    "star8_warmstart": "star_problem",
}


def lognormal_barycenter(seed: int, num_leaves: int, d: int, delta: float = 0.2,
                         cost_kind: str = COST_SQEUCLID) -> TreeProblem:
    """The barycenter of the paper's numerical section (Sec. 5): a star whose
    ``num_leaves`` = |E| leaves carry fixed marginals and whose centre is free, all
    on the uniform grid of d points between 0 and 1 (endpoints included), cost
    |x - y|^2 (so C_inf = 1), and the parameter choice of Sec. 3.2 for a target
    accuracy delta: eps = delta / (4 |E| log d); the stopping threshold is
    delta' = delta / (8 C_inf), in ``meta["tol"]``.

    Marginals: the density of a log-normal distribution evaluated on the grid
    and normalised to sum to one, with log-mean m ~ U[-1.5, 0] and shape
    s ~ U[0.3, 1] per leaf (mode e^(m - s^2) inside (0, 1]); the density is 0 at
    x = 0.  The paper says only that the marginals are generated from the
    log-normal distribution and normalised."""
    rng = np.random.default_rng(seed)
    edges = star_edges(num_leaves)
    x = grid_1d(d)
    xs = x[:, 0].astype(np.float64)
    J = num_leaves + 1
    fixed = np.ones(J, dtype=bool)
    fixed[0] = False
    marg = {}
    for l in range(1, J):
        m = rng.uniform(-1.5, 0.0)
        sh = rng.uniform(0.3, 1.0)
        w = np.zeros(d)
        pos = xs > 0
        w[pos] = np.exp(-(np.log(xs[pos]) - m) ** 2 / (2.0 * sh * sh)) / (xs[pos] * sh * np.sqrt(2.0 * np.pi))
        marg[l] = w / w.sum()
    eps = delta / (4.0 * num_leaves * np.log(d))
    return TreeProblem(name=f"lognormal_bary_E{num_leaves}_d{d}", edges=edges, n=np.full(J, d, np.int32),
                       fixed=fixed, marginals=marg, eps=float(eps), coords=[x] * J, cost_scale=1.0,
                       cost_kind=cost_kind, meta={"seed": seed, "delta": delta, "tol": delta / 8.0})


# --------------------------------------------------------------------------
# general graphs: modified junction trees (Sec. 4)
# --------------------------------------------------------------------------

@dataclass
class JunctionTreeProblem:
    """A coupled MOT problem on a modified junction tree (Sec. 4, eq. ot_graph_local_reg).

    Attributes
    ----------
    d : int [V]; support size of every variable x_0 .. x_{V-1}.
    clique_vars : per cost clique, the sorted tuple of its variables.
    clique_costs : per cost clique, the FP64 cost tensor, axes in clique_vars order.
    sep_vars : per separator, the sorted tuple of its variables.
    sep_cliques : per separator, its neighbour cliques in the order of its
        inclusion sequence (Assumption ass:inclusion: the intersections with the
        separator are equal for the first two and nested after that).
    sep_gamma : per separator, the constrained variable set (a sorted tuple) or None.
    sep_mu : per separator, the FP64 marginal over sep_gamma (axes in that order) or None.
    eps : local entropic regularisation.
    coords : per variable float32 [d, 1] support points (the grid the costs were built on).
    """

    name: str
    d: np.ndarray
    clique_vars: List[tuple]
    clique_costs: List[np.ndarray]
    sep_vars: List[tuple]
    sep_cliques: List[List[int]]
    sep_gamma: List[Optional[tuple]]
    sep_mu: List[Optional[np.ndarray]]
    eps: float
    coords: List[np.ndarray] = field(default_factory=list)
    meta: Dict = field(default_factory=dict)


def _lognormal_density_marginal(xs, rng):
    m = rng.uniform(-1.5, 0.0)
    sh = rng.uniform(0.3, 1.0)
    w = np.zeros(xs.shape[0])
    pos = xs > 0
    w[pos] = np.exp(-(np.log(xs[pos]) - m) ** 2 / (2.0 * sh * sh)) / (xs[pos] * sh * np.sqrt(2.0 * np.pi))
    return w / w.sum()


def wls_junction_tree(seed: int, J: int, d: int, alpha: float = 10.0, delta: float = 0.2) -> JunctionTreeProblem:
    """Wasserstein least squares (Sec. 2.3, eq. wls_cost) on its modified junction tree
    (Sec. 4): variables x_0, x_1 .. x_J, x_{J+1} on the uniform grid of d points in
    [0, 1]; cost cliques {x_0, x_j, x_{J+1}} with
        C_j = |x_j - (1 - t_j) x_0 - t_j x_{J+1}|^2 + (alpha / J) |x_0 - x_{J+1}|^2,
    t_j = j / (J + 1) (the alpha term of eq. wls_cost shared equally by the J cliques);
    separators {x_0, x_{J+1}} (free, joined to every clique) and {x_j} (constrained to
    the data marginal rho_{t_j}, a log-normal density on the grid).  eps and the
    stopping threshold follow the parameter choice of Sec. 3.2 with |E| = J cliques:
    eps = delta / (4 J log d), threshold delta / (8 C_inf) in meta["tol"]."""
    rng = np.random.default_rng(seed)
    x = grid_1d(d)
    xs = x[:, 0].astype(np.float64)
    V = J + 2
    cv, cc = [], []
    for j in range(1, J + 1):
        t = j / (J + 1.0)
        X0 = xs[:, None, None]
        Xj = xs[None, :, None]
        X1 = xs[None, None, :]
        C = (Xj - (1.0 - t) * X0 - t * X1) ** 2 + (alpha / J) * (X0 - X1) ** 2   # axes (x_0, x_j, x_{J+1})
        cv.append((0, j, J + 1))
        cc.append(C)
    sv = [(0, J + 1)] + [(j,) for j in range(1, J + 1)]
    sc = [list(range(J))] + [[j - 1] for j in range(1, J + 1)]
    sg = [None] + [(j,) for j in range(1, J + 1)]
    smu = [None] + [_lognormal_density_marginal(xs, rng) for _ in range(J)]
    cinf = max(float(np.max(np.abs(C))) for C in cc)
    eps = delta / (4.0 * J * np.log(d))
    return JunctionTreeProblem(name=f"wls_J{J}_d{d}", d=np.full(V, d, np.int32), clique_vars=cv, clique_costs=cc,
                               sep_vars=sv, sep_cliques=sc, sep_gamma=sg, sep_mu=smu, eps=float(eps),
                               coords=[x] * V, meta={"seed": seed, "alpha": alpha, "delta": delta,
                                                     "tol": delta / (8.0 * cinf), "c_inf": cinf})


def nested_junction_tree(seed: int, d: int = 2, eps: float = 0.5) -> JunctionTreeProblem:
    """The nested example of Sec. 4 (Assumption ass:inclusion's figure) closed into a
    modified junction tree: separator c = {x1, x3, x4} with cliques c1 = {x1, x2, x3, x4},
    c2 = {x1, x3, x4}, c3 = {x0, x1, x3} (intersections {1,3,4} = {1,3,4} ⊇ {1,3}) and
    the constraint gamma = {x3} embedded in c; each clique's second separator is a
    constrained single variable: {x2} for c1, {x4} for c2, {x0} for c3.  Costs are
    seeded uniform numbers in [0, 1); marginals Dirichlet(1)."""
    rng = np.random.default_rng(seed)
    V = 5
    dd = np.full(V, d, np.int32)
    cv = [(1, 2, 3, 4), (1, 3, 4), (0, 1, 3)]
    cc = [rng.random(tuple(int(dd[v]) for v in c)) for c in cv]
    sv = [(1, 3, 4), (2,), (4,), (0,)]
    sc = [[0, 1, 2], [0], [1], [2]]
    sg = [(3,), (2,), (4,), (0,)]
    smu = [dirichlet_marginal(d, rng) for _ in range(4)]
    x = grid_1d(d)
    return JunctionTreeProblem(name=f"nested_d{d}", d=dd, clique_vars=cv, clique_costs=cc, sep_vars=sv,
                               sep_cliques=sc, sep_gamma=sg, sep_mu=smu, eps=eps, coords=[x] * V,
                               meta={"seed": seed})


def tree_as_junction_tree(p: TreeProblem) -> JunctionTreeProblem:
    """A tree problem of Sec. 3 written as a modified junction tree: variables = nodes,
    cost cliques = edges {j, k}, separators = single nodes {j} (constrained to mu_j on
    fixed nodes).  The cost tensors are the problem's FP32 costs in FP64."""
    J = p.num_nodes
    cv, cc = [], []
    for e, (a, b) in enumerate(np.asarray(p.edges)):
        a, b = int(a), int(b)
        if p.cost_kind == COST_DENSE:
            C = (p.dense_costs[e] if p.dense_costs is not None and p.dense_costs[e] is not None
                 else p.dense_cost(e)).astype(np.float64)
        else:
            Xa = p.coords[a].astype(np.float64)
            Xb = p.coords[b].astype(np.float64)
            C = p.cost_scale * ((Xa[:, None, :] - Xb[None, :, :]) ** 2).sum(-1)
        if a < b:
            cv.append((a, b))
            cc.append(C)
        else:
            cv.append((b, a))
            cc.append(C.T.copy())
    sv = [(j,) for j in range(J)]
    sc = [[] for _ in range(J)]
    for e, (a, b) in enumerate(np.asarray(p.edges)):
        sc[int(a)].append(e)
        sc[int(b)].append(e)
    sg = [(j,) if p.fixed[j] else None for j in range(J)]
    smu = [p.marginals[j] if p.fixed[j] else None for j in range(J)]
    return JunctionTreeProblem(name=p.name + "_jt", d=np.asarray(p.n, np.int32), clique_vars=cv, clique_costs=cc,
                               sep_vars=sv, sep_cliques=sc, sep_gamma=sg, sep_mu=smu, eps=p.eps,
                               coords=list(p.coords), meta=dict(p.meta))

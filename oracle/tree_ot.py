"""FP64 CPU oracle: bipartite iterative scaling for tree-structured OT with local
entropic regularisation (Sec. 3 of "A parallel framework for graphical optimal
transport").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
package; only the tests, the smoke check and the benchmark's CPU-baseline leg
use it.  It shares no code with the CUDA path: it reads the same seeded problem
arrays (``gen``) and nothing else.

Everything here is plain numpy in float64, written for readability, in the
paper's notation:

* tree G=(V,E), neighbours N(j), fixed nodes Gamma (leaves only), free nodes V\\Gamma;
* reference measure M_(j,k) = gamma_j (x) gamma_k with gamma_j = mu_j on Gamma and 1
  elsewhere (eq. jointdist, Sec. 3.1);
* plans B_(j,k) = diag(u_(j,k) gamma_j) K_(j,k) diag(u_(k,j) gamma_k),
  K = exp(-C/eps) (eq. bi-marginal_B_sol);
* potentials lambda_(j,k) = eps * log u_(j,k) (Sec. 3.2); here called ``f[(j,k)]``,
  one vector of length n_j per directed edge.

Updates (theorem thm:tree_dual_var, Sec. 3.1), written in log form with the message
    m_(j,k)(x) = log( K_(j,k) (u_(k,j) * gamma_k) )(x)
               = LSE_y [ (f_(k,j)(y) - C_(j,k)(x,y)) / eps + log gamma_k(y) ]:
* fixed j:  u_(j,k_j) = 1 ./ (K u_(k_j,j))          ->  f_(j,k_j) = -eps m_(j,k_j)
* free j:   v_j = (prod_k K(u_(k,j) gamma_k))^(1/|N(j)|) -> log v_j = s_j = mean_k m_(j,k)
            rho_j = -|N(j)| log(1^T v_j) = -|N(j)| Z_j,  Z_j = LSE_x s_j(x)
            u_(j,k) = exp(rho_j/|N(j)|) v_j ./ K(u_(k,j) gamma_k)
                                              ->  f_(j,k) = eps (s_j - Z_j - m_(j,k))
Schedule (Algorithm "Bipartite Iterative Scaling", Sec. 3.1): the tree is
two-coloured; half-step t updates every node of S_1 (t odd) or S_2 (t even)
from the neighbours' current potentials.  S_1 is the colour class of node 0.

Stopping quantity (the while-condition of that algorithm):
    r = sum_{j in Gamma} ||B_(j,k_j) 1 - mu_j||_1
      + sum_{j free} sum_{k in N(j)} ||q_(j,k) - qbar_j||_1,
with q_(j,k) = B_(j,k) 1 and qbar_j their arithmetic mean (lemma lem:f_upper_bound_tree).

Readings of the paper taken here:
* "iteration" t counts half-steps; S_1 (node 0's colour) goes first;
* the closed form of thm:tree_dual_var is used (it equals the multiplicative
  listing from u = 1, proposition cor:equi; ``multiplicative_half_step`` implements the
  listing's form for that check);
* potentials where gamma_j(x) = 0 are still defined by the update formula.
"""
from __future__ import annotations

from collections import deque
from typing import Dict, List, Tuple

import numpy as np

Potentials = Dict[Tuple[int, int], np.ndarray]


# ---------------------------------------------------------------------------
# tree structure (Sec. 3: fixed nodes are leaves; no edge joins two fixed nodes)
# ---------------------------------------------------------------------------

class TreeError(ValueError):
    """Invalid input; ``kind`` names the violated assumption."""

    def __init__(self, kind: str, msg: str):
        super().__init__(f"{kind}: {msg}")
        self.kind = kind


def neighbours(num_nodes: int, edges) -> List[List[int]]:
    nb = [[] for _ in range(num_nodes)]
    for a, b in edges:
        nb[int(a)].append(int(b))
        nb[int(b)].append(int(a))
    return nb


def validate(problem) -> None:
    """Check the assumptions of Sec. 3 (tree; Gamma only on leaves; no Gamma-Gamma edge)."""
    J = problem.num_nodes
    E = np.asarray(problem.edges)
    if J < 2 or E.shape != (J - 1, 2):
        raise TreeError("NOT_TREE", "a tree on J nodes has J-1 edges")
    if E.min() < 0 or E.max() >= J or np.any(E[:, 0] == E[:, 1]):
        raise TreeError("NOT_TREE", "edge endpoint out of range or self loop")
    nb = neighbours(J, E)
    seen = np.zeros(J, dtype=bool)
    seen[0] = True
    dq = deque([0])
    while dq:
        v = dq.popleft()
        for w in nb[v]:
            if not seen[w]:
                seen[w] = True
                dq.append(w)
    if not seen.all():
        raise TreeError("NOT_TREE", "graph is not connected")
    for j in range(J):
        if problem.fixed[j]:
            if len(nb[j]) != 1:
                raise TreeError("FIXED_NOT_LEAF", f"fixed node {j} is not a leaf")
            if problem.fixed[nb[j][0]]:
                raise TreeError("FIXED_ADJACENT", f"edge joins fixed nodes {j},{nb[j][0]}")
            mu = problem.marginals[j]
            if mu.shape != (problem.n[j],) or np.any(mu < 0) or abs(mu.sum() - 1.0) > 1e-9:
                raise TreeError("MARGINAL", f"marginal of node {j} is not a probability vector")
    if not problem.eps > 0:
        raise TreeError("EPS", "eps must be positive")


def bipartition(num_nodes: int, edges) -> np.ndarray:
    """Colour classes of the tree (Sec. 3.1, bipartite graph); colour 0 contains node 0."""
    nb = neighbours(num_nodes, edges)
    colour = -np.ones(num_nodes, dtype=np.int64)
    colour[0] = 0
    dq = deque([0])
    while dq:
        v = dq.popleft()
        for w in nb[v]:
            if colour[w] < 0:
                colour[w] = 1 - colour[v]
                dq.append(w)
    return colour


# ---------------------------------------------------------------------------
# problem data in FP64
# ---------------------------------------------------------------------------

def edge_index(problem) -> Dict[Tuple[int, int], Tuple[int, bool]]:
    """(j,k) -> (edge id, transposed?) where not transposed means rows are node j."""
    idx = {}
    for e, (a, b) in enumerate(np.asarray(problem.edges)):
        idx[(int(a), int(b))] = (e, False)
        idx[(int(b), int(a))] = (e, True)
    return idx


def cost(problem, j: int, k: int, rows=None) -> np.ndarray:
    """C_(j,k) in FP64, rows indexed by node j's support (C_(k,j) = C_(j,k)^T)."""
    e, transposed = edge_index(problem)[(j, k)]
    a, b = (k, j) if transposed else (j, k)
    if problem.cost_kind == "dense":
        if problem.dense_costs is not None and problem.dense_costs[e] is not None:
            Cab = problem.dense_costs[e].astype(np.float64)
        else:
            Cab = problem.dense_cost(e).astype(np.float64)
        C = Cab.T if transposed else Cab
        return C if rows is None else C[np.asarray(rows)]
    # squared Euclidean between FP32 support points, evaluated in FP64
    X = problem.coords[j].astype(np.float64)
    Y = problem.coords[k].astype(np.float64)
    if rows is not None:
        X = X[np.asarray(rows)]
    return problem.cost_scale * ((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2)


def log_gamma(problem, j: int) -> np.ndarray:
    """log gamma_j: log mu_j on Gamma (-inf where mu_j = 0), 0 on free nodes (eq. jointdist)."""
    if problem.fixed[j]:
        with np.errstate(divide="ignore"):
            return np.log(problem.marginals[j])
    return np.zeros(int(problem.n[j]))


def c_infinity(problem) -> float:
    """C_inf = max over edges of the entrywise max |C_e| over finite entries (Sec. 3.2)."""
    best = 0.0
    for a, b in np.asarray(problem.edges):
        C = cost(problem, int(a), int(b))
        fin = np.isfinite(C)
        if fin.any():
            best = max(best, float(np.abs(C[fin]).max()))
    return best


def zero_potentials(problem) -> Potentials:
    """u^0 = 1, i.e. lambda^0 = 0 on every directed edge (initialisation of the algorithm)."""
    f = {}
    for a, b in np.asarray(problem.edges):
        a, b = int(a), int(b)
        f[(a, b)] = np.zeros(int(problem.n[a]))
        f[(b, a)] = np.zeros(int(problem.n[b]))
    return f


# ---------------------------------------------------------------------------
# log-sum-exp and the message K_(j,k)(u_(k,j) * gamma_k) in log form
# ---------------------------------------------------------------------------

def logsumexp(A: np.ndarray, axis: int) -> np.ndarray:
    """Two-pass log-sum-exp (max, then sum of exp); all--inf slices give -inf."""
    M = np.max(A, axis=axis, keepdims=True)
    Msafe = np.where(np.isfinite(M), M, 0.0)
    with np.errstate(divide="ignore"):
        out = np.log(np.sum(np.exp(A - Msafe), axis=axis, keepdims=True)) + Msafe
    return np.squeeze(out, axis=axis)


def message(problem, f: Potentials, j: int, k: int, rows=None) -> np.ndarray:
    """m_(j,k)(x) = log sum_y K_(j,k)(x,y) u_(k,j)(y) gamma_k(y), in log-sum-exp form."""
    C = cost(problem, j, k, rows)
    A = (f[(k, j)][None, :] - C) / problem.eps + log_gamma(problem, k)[None, :]
    return logsumexp(A, axis=1)


# ---------------------------------------------------------------------------
# one half-step of the bipartite schedule (thm:tree_dual_var applied to all j in S)
# ---------------------------------------------------------------------------

def update_node(problem, f: Potentials, j: int, nb: List[List[int]]):
    """New potentials {f_(j,k)}_k of node j and rho_j (None for fixed nodes), thm:tree_dual_var."""
    eps = problem.eps
    msgs = {k: message(problem, f, j, k) for k in nb[j]}
    if problem.fixed[j]:
        (k,) = nb[j]
        return {(j, k): -eps * msgs[k]}, None
    deg = len(nb[j])
    s = sum(msgs[k] for k in nb[j]) / deg            # log of the geometric mean v_j
    Z = float(logsumexp(s, axis=0))                    # log(1^T v_j)
    rho = -deg * Z
    return {(j, k): eps * (s - Z - msgs[k]) for k in nb[j]}, rho


def half_step(problem, f: Potentials, colour: np.ndarray, side: int):
    """Update every node of colour ``side`` from the current potentials (parallel within S)."""
    nb = neighbours(problem.num_nodes, problem.edges)
    new = dict(f)
    rhos = {}
    for j in range(problem.num_nodes):
        if colour[j] != side:
            continue
        upd, rho = update_node(problem, f, j, nb)   # reads only f of the other colour
        new.update(upd)
        if rho is not None:
            rhos[j] = rho
    return new, rhos


def run_half_steps(problem, T: int, f: Potentials = None) -> Potentials:
    """T half-steps from u = 1 (or from ``f``): S_1 on odd t, S_2 on even t."""
    colour = bipartition(problem.num_nodes, problem.edges)
    f = zero_potentials(problem) if f is None else dict(f)
    for t in range(1, T + 1):
        f, _ = half_step(problem, f, colour, 0 if t % 2 == 1 else 1)
    return f


# ---------------------------------------------------------------------------
# plans, marginals and the stopping quantity
# ---------------------------------------------------------------------------

def plan(problem, f: Potentials, j: int, k: int) -> np.ndarray:
    """B_(j,k) = diag(u_(j,k) gamma_j) K diag(u_(k,j) gamma_k), rows indexed by node j."""
    C = cost(problem, j, k)
    A = (f[(j, k)][:, None] + f[(k, j)][None, :] - C) / problem.eps
    A = A + log_gamma(problem, j)[:, None] + log_gamma(problem, k)[None, :]
    with np.errstate(invalid="ignore"):
        return np.exp(A)


def edge_marginal(problem, f: Potentials, j: int, k: int) -> np.ndarray:
    """q_(j,k) = B_(j,k) 1 (eq. q)."""
    return plan(problem, f, j, k).sum(axis=1)


def residual(problem, f: Potentials) -> Tuple[float, float, Dict[Tuple[int, int], float]]:
    """(r, max term, per-directed-edge terms) of the stopping rule (all nodes).

    r = sum_{j in Gamma} ||B_(j,k_j)1 - mu_j||_1 + sum_{j free} sum_k ||q_(j,k) - qbar_j||_1.
    """
    nb = neighbours(problem.num_nodes, problem.edges)
    terms = {}
    for j in range(problem.num_nodes):
        if problem.fixed[j]:
            (k,) = nb[j]
            terms[(j, k)] = float(np.abs(edge_marginal(problem, f, j, k) - problem.marginals[j]).sum())
        else:
            qs = {k: edge_marginal(problem, f, j, k) for k in nb[j]}
            qbar = sum(qs.values()) / len(nb[j])
            for k in nb[j]:
                terms[(j, k)] = float(np.abs(qs[k] - qbar).sum())
    return float(sum(terms.values())), float(max(terms.values())), terms


def rho_of(problem, f: Potentials) -> Dict[int, float]:
    """rho_j = (1/eps) * mean_x sum_k f_(j,k)(x) for free j (the dual constraint of eq. tree_dual_mass_consv)."""
    nb = neighbours(problem.num_nodes, problem.edges)
    out = {}
    for j in range(problem.num_nodes):
        if not problem.fixed[j]:
            out[j] = float(np.mean(sum(f[(j, k)] for k in nb[j]))) / problem.eps
    return out


def dual_objective(problem, f: Potentials) -> float:
    """f(u, rho) = sum_e ||B_e||_1 - sum_{j in Gamma} log(u_(j,k_j))^T mu_j - sum_{j free} rho_j."""
    nb = neighbours(problem.num_nodes, problem.edges)
    val = 0.0
    for a, b in np.asarray(problem.edges):
        val += float(plan(problem, f, int(a), int(b)).sum())
    for j in range(problem.num_nodes):
        if problem.fixed[j]:
            (k,) = nb[j]
            mu = problem.marginals[j]
            pos = mu > 0
            val -= float(np.dot(f[(j, k)][pos] / problem.eps, mu[pos]))
    val -= sum(rho_of(problem, f).values())
    return val


def final_check(problem, f: Potentials) -> dict:
    """FP64 quantities of the returned potentials: marginals, residuals, objectives.

    primal P   = sum_e <C_e,B_e> + eps H(B_e | M_e)  (objective of eq. ot_graph_pairwise_mass)
    dual   D   = -eps * f(u, rho)                    (same units as P; P = D at the optimum)
    transport  TC = sum_e <C_e, B_e>
    """
    eps = problem.eps
    nb = neighbours(problem.num_nodes, problem.edges)
    P = 0.0
    TC = 0.0
    mass = {}
    for a, b in np.asarray(problem.edges):
        a, b = int(a), int(b)
        B = plan(problem, f, a, b)
        C = cost(problem, a, b)
        pos = B > 0
        lgM = log_gamma(problem, a)[:, None] + log_gamma(problem, b)[None, :]
        lgM = np.broadcast_to(lgM, B.shape)
        H = float(np.sum(B[pos] * (np.log(B[pos]) - lgM[pos] - 1.0)))
        tc = float(np.sum(B[pos] * C[pos]))
        TC += tc
        P += tc + eps * H
        mass[(a, b)] = float(B.sum())
    r, rmax, terms = residual(problem, f)
    marg = {}
    for j in range(problem.num_nodes):
        qs = [edge_marginal(problem, f, j, k) for k in nb[j]]
        marg[j] = sum(qs) / len(qs)
    D = -eps * dual_objective(problem, f)
    return {"residual": r, "max_marginal_l1": rmax, "terms": terms, "primal": P, "dual": D,
            "transport_cost": TC, "mass": mass, "marginals": marg}


def solve(problem, tol: float = 1e-9, max_half_steps: int = 100000, tol_kind: str = "sum",
          f0: Potentials = None):
    """Run the algorithm until the stopping quantity is below ``tol``.

    ``tol_kind='sum'`` uses r (the paper's rule); ``'max'`` the largest single term.
    Returns (potentials, half-steps done, final r).
    """
    validate(problem)
    colour = bipartition(problem.num_nodes, problem.edges)
    f = zero_potentials(problem) if f0 is None else dict(f0)
    t = 1
    while True:
        r, rmax, _ = residual(problem, f)
        crit = r if tol_kind == "sum" else rmax
        if crit < tol or t > max_half_steps:
            return f, t - 1, r
        f, _ = half_step(problem, f, colour, 0 if t % 2 == 1 else 1)
        t += 1


def gauge_fix(problem, f: Potentials) -> Potentials:
    """Canonical representative: per edge (a,b), shift so that mean f_(b,a) = 0.

    (f_(a,b) + c, f_(b,a) - c) leaves every B_e unchanged.
    """
    g = dict(f)
    for a, b in np.asarray(problem.edges):
        a, b = int(a), int(b)
        c = float(np.mean(f[(b, a)]))
        g[(b, a)] = f[(b, a)] - c
        g[(a, b)] = f[(a, b)] + c
    return g


# ---------------------------------------------------------------------------
# the algorithm listing's multiplicative form (proposition cor:equi check)
# ---------------------------------------------------------------------------

def multiplicative_half_step(problem, u: Dict[Tuple[int, int], np.ndarray], colour, side: int):
    """Scaling-domain update of the listing: fixed u <- u * mu / q; free u <- u * (q_j/|q_j|_1) / q_(j,k).

    q_(j,k) = B^t 1 with B^t from the current u, q_j = geometric mean of {q_(j,k)}_k.
    Only for small problems with moderate C/eps (plain exponentials, no log domain).
    """
    nb = neighbours(problem.num_nodes, problem.edges)
    eps = problem.eps

    def gamma(j):
        return problem.marginals[j] if problem.fixed[j] else np.ones(int(problem.n[j]))

    def q(j, k):
        K = np.exp(-cost(problem, j, k) / eps)
        return (u[(j, k)] * gamma(j)) * (K @ (u[(k, j)] * gamma(k)))

    new = dict(u)
    for j in range(problem.num_nodes):
        if colour[j] != side:
            continue
        if problem.fixed[j]:
            (k,) = nb[j]
            new[(j, k)] = u[(j, k)] * problem.marginals[j] / q(j, k)
        else:
            qs = {k: q(j, k) for k in nb[j]}
            qj = np.exp(sum(np.log(qs[k]) for k in nb[j]) / len(nb[j]))
            for k in nb[j]:
                new[(j, k)] = u[(j, k)] * (qj / qj.sum()) / qs[k]
    return new


# ---------------------------------------------------------------------------
# rounding to feasible plans (Algorithm "Rounding for transport plan on a
# bipartite graph", Sec. 3.1; lemmas lem:round and lem:round_applied, Sec. 3.2)
# ---------------------------------------------------------------------------

def round_matrix(F: np.ndarray, r: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Algorithm 2 of Altschuler, Weed and Rigollet (2017), the routine the paper's
    rounding calls: a nonnegative G with row sums r and column sums c (||r||_1 = ||c||_1).

    1. scale every row of F down to at most r:     x_i = min(r_i / r_i(F), 1),  F' = diag(x) F;
    2. scale every column down to at most c:       y_j = min(c_j / c_j(F'), 1), F'' = F' diag(y);
    3. add what is missing as a rank-one term:     G = F'' + err_r err_c^T / ||err_r||_1,
       err_r = r - F'' 1,  err_c = c - F''^T 1  (both nonnegative).
    A row or column of F with zero sum is left unscaled (x or y = 1).
    """
    F = np.asarray(F, dtype=np.float64)
    rF = F.sum(axis=1)
    x = np.ones_like(rF)
    pos = rF > 0
    x[pos] = np.minimum(r[pos] / rF[pos], 1.0)
    F1 = x[:, None] * F
    cF1 = F1.sum(axis=0)
    y = np.ones_like(cF1)
    pos = cF1 > 0
    y[pos] = np.minimum(c[pos] / cF1[pos], 1.0)
    F2 = F1 * y[None, :]
    # nonnegative in exact arithmetic; a last-bit negative difference is taken as 0
    err_r = np.maximum(r - F2.sum(axis=1), 0.0)
    err_c = np.maximum(c - F2.sum(axis=0), 0.0)
    mass = float(err_r.sum())
    if mass > 0:
        F2 = F2 + np.outer(err_r, err_c) / mass
    return F2


def mismatched_side(T: int) -> int:
    """The colour class whose projections miss their marginals after half-step T >= 1:
    half-step T updated colour (T+1) % 2, so it is colour T % 2 (the set S of the rounding)."""
    return T % 2


def round_plans(problem, f: Potentials, side: int) -> Dict[Tuple[int, int], np.ndarray]:
    """The rounding algorithm of Sec. 3.1 applied to the plans of the potentials f.

    For every node j of colour class ``side`` (the set S) and every neighbour k, B_(j,k)
    (rows on j) is rounded by ``round_matrix`` so that its row sums become mu_j (j fixed) or
    qbar_j(B) = mean_k B_(j,k) 1 (j free) and its column sums stay B_(j,k)^T 1.  Every edge
    has exactly one endpoint in S, so every plan is rounded once.  Returns {(j, k): B^_(j,k)}
    keyed with j in S.
    """
    colour = bipartition(problem.num_nodes, problem.edges)
    nb = neighbours(problem.num_nodes, problem.edges)
    out = {}
    for j in range(problem.num_nodes):
        if colour[j] != side:
            continue
        Bs = {k: plan(problem, f, j, k) for k in nb[j]}
        if problem.fixed[j]:
            target = np.asarray(problem.marginals[j], dtype=np.float64)
        else:
            target = sum(B.sum(axis=1) for B in Bs.values()) / len(nb[j])
        for k in nb[j]:
            out[(j, k)] = round_matrix(Bs[k], target, Bs[k].sum(axis=0))
    return out


def rounded_transport_cost(problem, rounded: Dict[Tuple[int, int], np.ndarray]) -> float:
    """sum_e <C_e, B^_e> of rounded plans (entries with B^ = 0 contribute nothing, also where C = +inf)."""
    tc = 0.0
    for (j, k), B in rounded.items():
        C = cost(problem, j, k)
        pos = B > 0
        tc += float(np.sum(B[pos] * C[pos]))
    return tc

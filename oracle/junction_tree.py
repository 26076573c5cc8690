"""FP64 CPU oracle for coupled MOT on a modified junction tree (Sec. 4 of "A
parallel framework for graphical optimal transport": definition def:jt_general,
problem eq:ot_graph_local_reg, Assumption ass:inclusion, proposition
prop:local_reg_dual and the separator update of proposition prop:general_algo).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module; only the tests use it.  It shares no code with the CUDA path and reads
the problem description from ``gen`` (``JunctionTreeProblem``).

Plain numpy in float64, in the log domain: every tensor carries the tuple of its
variables (axes in that order), and "(x) 1" broadcasting is an explicit
expansion to a superset of variables.  Notation as in Sec. 4:

* cost cliques c in Q_C (tensors B_c over their variables), each joined to
  exactly two separators in Q_S;
* separator s with neighbour cliques c_1 .. c_l in the order of its inclusion
  sequence (s n c_1 = s n c_2 >= s n c_3 >= ... >= s n c_l), optionally a
  constrained set gamma (inside s n c_l) with marginal mu_gamma;
* dual variable u^s_i over s n c_i for each neighbour; plans
  B_c = K_c . M_c . (u^{s_j}_{i_j} (x) 1) . (u^{s_k}_{i_k} (x) 1),  K_c = exp(-C_c / eps),
  M_c = m_{s_j} (x) m_{s_k},  m_s = mu_gamma (x) 1 on constrained separators, else 1
  (prop:local_reg_dual);
* k_i = P_{s n c_i}(K_{c_i} . M_{c_i} . (ubar_i (x) 1)), ubar_i the other separator's
  dual variable of c_i, P the marginal (sum over the other variables).

Separator update (prop:general_algo), for l > 1:
  1. q_2 = (k_1 . k_2)^(1/2),  q_i = (P_{s n c_i}(q_{i-1})^(i-1) . k_i)^(1/i), i = 3..l;
  2. v_{l+1} = (mu_gamma ./ P_gamma(q_l))^l  (unconstrained: mu = 1, P = total sum, a scalar;
     computed with s's own factor m_s taken out of the k_i, see update_separator),
     a_i = (v_{i+1} (x) 1)^(1/i) . q_i for i = l..2, with v_i = (a_i ./ P_{s n c_i}(q_{i-1}))^(i-1)
     for i = l..3 computed on the way;
  3. u_1 = a_2 ./ k_1,  u_i = a_i ./ k_i (i = 2..l).
For l = 1 the dual variable is constant along the variables outside gamma:
  u_1 = (mu_gamma ./ P_gamma(k_1)) (x) 1 (the paper writes u_1 = mu_gamma ./ k_1 for
  gamma = s n c_1), and u_1 = 1 / sum k_1 on an unconstrained separator.

Schedule: separators are two-coloured through the cliques (the modified junction
tree is bipartite); a half-step updates every separator of one colour from the
other colour's current dual variables; the colour of separator 0 goes first.

Stopping quantity (a reading: the paper defines none for general graphs): for
every separator, sum_{i >= 2} ||P_{s n c_i}(B_{c_i}) - P_{s n c_i}(B_{c_1})||_1 plus
||P_gamma(B_{c_1}) - mu_gamma||_1 (constrained) or |<B_{c_1}, 1> - 1| (unconstrained);
zero exactly when the plans meet the constraints of eq:ot_graph_local_reg.
"""
from __future__ import annotations

from collections import deque
from typing import Dict, List, Tuple

import numpy as np

LogT = Tuple[tuple, np.ndarray]          # (variables, log-tensor with axes in that order)


# ---------------------------------------------------------------------------
# tensors over variable sets, in the log domain
# ---------------------------------------------------------------------------

def _lse(a: np.ndarray, axes) -> np.ndarray:
    if not axes:
        return a
    m = np.max(a, axis=axes, keepdims=True)
    ms = np.where(np.isfinite(m), m, 0.0)
    with np.errstate(divide="ignore"):
        out = np.log(np.sum(np.exp(a - ms), axis=axes, keepdims=True)) + ms
    return np.squeeze(out, axis=axes)


def project(t: LogT, keep: tuple) -> LogT:
    """log P_keep(exp t): sum over the variables of t not in keep (keep = () gives the total)."""
    vars_, a = t
    axes = tuple(i for i, v in enumerate(vars_) if v not in keep)
    kept = tuple(v for v in vars_ if v in keep)
    assert set(kept) == set(keep), (vars_, keep)
    out = _lse(np.asarray(a, dtype=np.float64), axes)
    order = [kept.index(v) for v in keep]
    return tuple(keep), np.transpose(out, order) if np.ndim(out) > 1 else out


def expand(t: LogT, to: tuple, d) -> np.ndarray:
    """t broadcast to the variables ``to`` (a superset), axes in ``to`` order."""
    vars_, a = t
    assert set(vars_) <= set(to), (vars_, to)
    if not vars_:
        return np.full(tuple(int(d[v]) for v in to), float(a))
    order = sorted(range(len(vars_)), key=lambda i: to.index(vars_[i]))
    a = np.transpose(a, order)
    shape = [int(d[v]) if v in vars_ else 1 for v in to]
    return np.broadcast_to(a.reshape(shape), tuple(int(d[v]) for v in to))


def inter(a: tuple, b: tuple) -> tuple:
    return tuple(v for v in a if v in b)


# ---------------------------------------------------------------------------
# structure checks (def:jt_general, Assumption ass:inclusion)
# ---------------------------------------------------------------------------

def clique_separators(jt) -> List[List[Tuple[int, int]]]:
    """Per clique: its (separator, position in that separator's inclusion sequence) pairs."""
    out = [[] for _ in jt.clique_vars]
    for s, cl in enumerate(jt.sep_cliques):
        for i, c in enumerate(cl):
            out[c].append((s, i))
    return out


def validate(jt) -> None:
    cs = clique_separators(jt)
    for c, lst in enumerate(cs):
        if len(lst) != 2:
            raise ValueError(f"clique {c} must have exactly two separator neighbours (def:jt_general.4)")
        for s, _ in lst:
            if not set(jt.sep_vars[s]) & set(jt.clique_vars[c]) and jt.sep_vars[s]:
                raise ValueError(f"separator {s} shares no variable with clique {c}")
    for s, cl in enumerate(jt.sep_cliques):
        if not cl:
            raise ValueError(f"separator {s} has no clique")
        sets = [set(inter(jt.sep_vars[s], jt.clique_vars[c])) for c in cl]
        if len(sets) > 1 and sets[0] != sets[1]:
            raise ValueError(f"separator {s}: the first two intersections must be equal (ass:inclusion)")
        for i in range(2, len(sets)):
            if not sets[i] <= sets[i - 1]:
                raise ValueError(f"separator {s}: intersections must be nested (ass:inclusion)")
        g = jt.sep_gamma[s]
        if g is not None:
            if not set(g) <= sets[-1]:
                raise ValueError(f"separator {s}: gamma must lie in the smallest intersection")
            mu = np.asarray(jt.sep_mu[s])
            if mu.shape != tuple(int(jt.d[v]) for v in g) or np.any(mu < 0) or abs(mu.sum() - 1) > 1e-9:
                raise ValueError(f"separator {s}: mu_gamma is not a probability tensor over gamma")
    colours(jt)  # bipartite


def colours(jt) -> np.ndarray:
    """Two-colouring of the separators through the cliques; separator 0 gets colour 0."""
    S = len(jt.sep_vars)
    nb = [set() for _ in range(S)]
    for lst in clique_separators(jt):
        (a, _), (b, _) = lst
        nb[a].add(b)
        nb[b].add(a)
    col = -np.ones(S, dtype=np.int64)
    col[0] = 0
    dq = deque([0])
    while dq:
        v = dq.popleft()
        for w in nb[v]:
            if col[w] < 0:
                col[w] = 1 - col[v]
                dq.append(w)
            elif col[w] == col[v]:
                raise ValueError("the separator graph is not bipartite")
    if np.any(col < 0):
        raise ValueError("the junction tree is not connected")
    return col


# ---------------------------------------------------------------------------
# dual variables, plans and the separator update
# ---------------------------------------------------------------------------

Duals = Dict[Tuple[int, int], LogT]   # (separator, position) -> log u over s n c_i


def zero_duals(jt) -> Duals:
    """u = 1 on every dual variable."""
    out = {}
    for s, cl in enumerate(jt.sep_cliques):
        for i, c in enumerate(cl):
            v = inter(jt.sep_vars[s], jt.clique_vars[c])
            out[(s, i)] = (v, np.zeros(tuple(int(jt.d[x]) for x in v)))
    return out


def log_m(jt, s) -> LogT:
    """log m_s: log mu_gamma on a constrained separator, else 0 (over no variables)."""
    g = jt.sep_gamma[s]
    if g is None:
        return (), np.float64(0.0)
    with np.errstate(divide="ignore"):
        return tuple(g), np.log(np.asarray(jt.sep_mu[s], dtype=np.float64))


def log_plan_without(jt, duals: Duals, c: int, skip=None) -> np.ndarray:
    """log(K_c . M_c . u's) over clique c's variables; with ``skip`` = (s, i), without the
    dual variable u^s_i and without s's own factor m_s of M_c."""
    cv = jt.clique_vars[c]
    a = -np.asarray(jt.clique_costs[c], dtype=np.float64) / jt.eps
    for s, i in clique_separators(jt)[c]:
        if (s, i) != skip:
            a = a + expand(log_m(jt, s), cv, jt.d)
            a = a + expand(duals[(s, i)], cv, jt.d)
    return a


def log_plan(jt, duals: Duals, c: int) -> LogT:
    return jt.clique_vars[c], log_plan_without(jt, duals, c)


def geometric_chain(k: List[LogT], sets: List[tuple]):
    """Step 1 of prop:general_algo in logs: q_2 = (k_1 k_2)^(1/2), q_i = (P_{s n c_i}(q_{i-1})^(i-1) k_i)^(1/i).
    Returns (q, Pq), q[i] over sets[i - 1] and Pq[i] = P_{s n c_i}(q_{i-1}) (1-based i as in the text)."""
    l = len(k)
    q = [None] * (l + 1)
    Pq = [None] * (l + 1)
    q[2] = (sets[1], 0.5 * (k[0][1] + k[1][1]))
    for i in range(3, l + 1):
        Pq[i] = project(q[i - 1], sets[i - 1])
        q[i] = (sets[i - 1], ((i - 1) * Pq[i][1] + k[i - 1][1]) / i)
    return q, Pq


def intermediates(jt, q, Pq, sets: List[tuple], g: tuple):
    """Step 2 in logs: v_{l+1} = (1 ./ P_gamma(q_l))^l (mu_gamma cancelled, see update_separator),
    a_i = (v_{i+1} (x) 1)^(1/i) q_i for i = l..2, v_i = (a_i ./ P_{s n c_i}(q_{i-1}))^(i-1) for i = l..3."""
    l = len(sets)
    v_next = (g, l * (-project(q[l], g)[1]))
    a = [None] * (l + 1)
    for i in range(l, 1, -1):
        a[i] = (sets[i - 1], expand(v_next, sets[i - 1], jt.d) / i + q[i][1])
        if i >= 3:
            v_next = (sets[i - 1], (i - 1) * (a[i][1] - Pq[i][1]))
    return a


def update_separator(jt, duals: Duals, s: int) -> Duals:
    """New dual variables of separator s (prop:general_algo; l = 1 as in the text after it)."""
    cl = jt.sep_cliques[s]
    sv = jt.sep_vars[s]
    l = len(cl)
    sets = [inter(sv, jt.clique_vars[c]) for c in cl]
    # k_i = P_{s n c_i}(K . M . ubar (x) 1) carries s's own factor m_s = mu_gamma (x) 1 of M
    # in every i; it is left out here (k'_i), so the geometric means below carry it once and
    # mu_gamma cancels in v_{l+1} = (mu_gamma ./ P_gamma(q_l))^l = (1 ./ P_gamma(q'_l))^l.
    # Identical to the text where mu_gamma > 0; where it vanishes the dual variable stays
    # defined by the same formula (as in Sec. 3) and the plan is 0 there anyway.
    k = [project((jt.clique_vars[c], log_plan_without(jt, duals, c, skip=(s, i))), sets[i])
         for i, c in enumerate(cl)]
    g = () if jt.sep_gamma[s] is None else tuple(jt.sep_gamma[s])
    new = {}
    if l == 1:
        pk = project(k[0], g)
        new[(s, 0)] = (sets[0], expand((g, -pk[1]), sets[0], jt.d).copy())
        return new
    q, Pq = geometric_chain(k, sets)
    a = intermediates(jt, q, Pq, sets, g)
    # step 3
    new[(s, 0)] = (sets[0], a[2][1] - k[0][1])
    for i in range(2, l + 1):
        new[(s, i - 1)] = (sets[i - 1], a[i][1] - k[i - 1][1])
    return new


def half_step(jt, duals: Duals, colour: np.ndarray, side: int) -> Duals:
    new = dict(duals)
    for s in range(len(jt.sep_vars)):
        if colour[s] == side:
            new.update(update_separator(jt, duals, s))   # reads only the other colour's variables
    return new


def run_half_steps(jt, T: int, duals: Duals = None) -> Duals:
    col = colours(jt)
    duals = zero_duals(jt) if duals is None else dict(duals)
    for t in range(1, T + 1):
        duals = half_step(jt, duals, col, 0 if t % 2 == 1 else 1)
    return duals


# ---------------------------------------------------------------------------
# stopping quantity, objectives, solve
# ---------------------------------------------------------------------------

def residual(jt, duals: Duals) -> Tuple[float, float]:
    """(sum over separators, largest separator term) of the stopping quantity above."""
    plans = [log_plan(jt, duals, c) for c in range(len(jt.clique_vars))]
    terms = []
    for s, cl in enumerate(jt.sep_cliques):
        sv = jt.sep_vars[s]
        sets = [inter(sv, jt.clique_vars[c]) for c in cl]
        ref = project(plans[cl[0]], sets[0])
        r = 0.0
        for i in range(1, len(cl)):
            pi = np.exp(project(plans[cl[i]], sets[i])[1])
            pr = np.exp(project(ref, sets[i])[1])
            r += float(np.abs(pi - pr).sum())
        g = jt.sep_gamma[s]
        if g is None:
            r += abs(float(np.exp(ref[1]).sum()) - 1.0)
        else:
            r += float(np.abs(np.exp(project(ref, tuple(g))[1]) - np.asarray(jt.sep_mu[s])).sum())
        terms.append(r)
    return float(sum(terms)), float(max(terms))


def plans(jt, duals: Duals) -> List[np.ndarray]:
    return [np.exp(log_plan(jt, duals, c)[1]) for c in range(len(jt.clique_vars))]


def transport_cost(jt, duals: Duals) -> float:
    tc = 0.0
    for B, C in zip(plans(jt, duals), jt.clique_costs):
        pos = B > 0
        tc += float(np.sum(B[pos] * np.asarray(C)[pos]))
    return tc


def primal(jt, duals: Duals) -> float:
    """sum_c <C_c, B_c> + eps H(B_c | M_c), H(B|M) = sum B (log B - log M - 1)."""
    val = 0.0
    for c in range(len(jt.clique_vars)):
        lb = log_plan(jt, duals, c)[1]
        cv = jt.clique_vars[c]
        lm = np.zeros(lb.shape)
        for s, _ in clique_separators(jt)[c]:
            lm = lm + expand(log_m(jt, s), cv, jt.d)
        B = np.exp(lb)
        pos = B > 0
        C = np.asarray(jt.clique_costs[c])
        val += float(np.sum(B[pos] * C[pos]) + jt.eps * np.sum(B[pos] * (lb[pos] - lm[pos] - 1.0)))
    return val


def solve(jt, tol: float = 1e-10, max_half_steps: int = 100000, tol_kind: str = "sum"):
    """Half-steps until the stopping quantity is below tol; returns (duals, half-steps, r)."""
    validate(jt)
    col = colours(jt)
    duals = zero_duals(jt)
    t = 1
    while True:
        r, rmax = residual(jt, duals)
        crit = r if tol_kind == "sum" else rmax
        if crit < tol or t > max_half_steps:
            return duals, t - 1, r
        duals = half_step(jt, duals, col, 0 if t % 2 == 1 else 1)
        t += 1

"""Independent textbook solvers used to pin the CPU oracle.

None of this code is shared with the oracle or the CUDA path.  Each routine is
a different algorithm (or a generic library solver) for a problem whose
solution coincides with the tree solver's on a special case:

* ``sinkhorn``            -- two-marginal entropic OT (Cuturi 2013), log domain.
* ``ibp_barycenter``      -- iterative Bregman projections for the entropic
                             barycenter with uniform weights (Benamou et al. 2015).
* ``primal_generic``      -- the local-entropy primal problem of Sec. 3 solved
                             as a generic linearly constrained entropic program
                             (Newton on its Lagrangian dual).
* ``lp_optimum``          -- the unregularised tree LP (eq. ot_graph_pairwise)
                             solved with HiGHS.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linprog
from scipy.special import logsumexp


def sqeuclid(X, Y, scale=1.0):
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    return scale * ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)


def sinkhorn(mu, nu, C, eps, tol=1e-14, max_iter=200000):
    """argmin <C,P> + eps sum P(log P - 1) over P 1 = mu, P^T 1 = nu; returns P."""
    la, lb = np.log(mu), np.log(nu)
    a = np.zeros_like(mu)
    b = np.zeros_like(nu)
    for _ in range(max_iter):
        a = eps * (la - logsumexp((b[None, :] - C) / eps, axis=1))
        b_new = eps * (lb - logsumexp((a[:, None] - C) / eps, axis=0))
        if np.max(np.abs(b_new - b)) < tol * eps:
            b = b_new
            break
        b = b_new
    return np.exp((a[:, None] + b[None, :] - C) / eps)


def ibp_barycenter(mus, Cs, eps, tol=1e-15, max_iter=200000):
    """Entropic barycenter by iterative Bregman projections, uniform weights.

    ``Cs[l]`` is [n_l, n_bar] (rows: measure l).  Returns (plans, barycenter)
    where plans[l] has row sums mus[l] and column sums the barycenter.
    """
    L = len(mus)
    logK = [-C / eps for C in Cs]
    lv = [np.zeros(C.shape[1]) for C in Cs]
    lmu = [np.log(m) for m in mus]
    lbar = None
    for _ in range(max_iter):
        lu = [lmu[l] - logsumexp(logK[l] + lv[l][None, :], axis=1) for l in range(L)]
        lKtu = [logsumexp(logK[l] + lu[l][:, None], axis=0) for l in range(L)]
        lbar_new = sum(lKtu) / L
        lv = [lbar_new - lKtu[l] for l in range(L)]
        if lbar is not None and np.max(np.abs(lbar_new - lbar)) < tol:
            lbar = lbar_new
            break
        lbar = lbar_new
    plans = [np.exp(lu[l][:, None] + logK[l] + lv[l][None, :]) for l in range(L)]
    return plans, np.exp(lbar)


def _tree_constraints(J, edges, n, fixed, marginals):
    """Linear constraints of eq. ot_graph_pairwise_mass on the stacked plan entries."""
    offs = [0]
    for a, b in edges:
        offs.append(offs[-1] + n[a] * n[b])
    nvar = offs[-1]
    nb = [[] for _ in range(J)]
    for e, (a, b) in enumerate(edges):
        nb[a].append((e, True))
        nb[b].append((e, False))

    def row_sum_matrix(e, j_is_row):
        a, b = edges[e]
        Mx = np.zeros((n[a] if j_is_row else n[b], nvar))
        for x in range(n[a]):
            for y in range(n[b]):
                col = offs[e] + x * n[b] + y
                if j_is_row:
                    Mx[x, col] = 1.0
                else:
                    Mx[y, col] = 1.0
        return Mx

    A, rhs = [], []
    for j in range(J):
        mats = [row_sum_matrix(e, is_row) for e, is_row in nb[j]]
        if fixed[j]:
            A.append(mats[0])
            rhs.append(marginals[j])
        else:
            for M in mats[1:]:
                A.append(mats[0] - M)
                rhs.append(np.zeros(n[j]))
            A.append(mats[0].sum(axis=0, keepdims=True))
            rhs.append(np.ones(1))
    return np.vstack(A), np.concatenate(rhs), offs


def primal_generic(J, edges, n, fixed, marginals, costs, eps, tol=1e-14, max_iter=500):
    """Minimise sum_e <C_e,B_e> + eps H(B_e | gamma_j x gamma_k) over the constraint set.

    Generic convex optimisation, blind to the tree structure: the program is
    min_z c.z + eps sum z(log z - log m - 1) s.t. A z = b, whose Lagrangian dual
    max_y y.b - eps sum m exp((A^T y - c)/eps) is smooth and concave; it is
    maximised by damped Newton steps (least-squares solves, since A may have
    redundant rows) and z = m exp((A^T y - c)/eps) recovered.  Returns (plans, primal value).
    """
    A, rhs, offs = _tree_constraints(J, edges, n, fixed, marginals)
    logM = []
    for e, (a, b) in enumerate(edges):
        ga = np.log(marginals[a]) if fixed[a] else np.zeros(n[a])
        gb = np.log(marginals[b]) if fixed[b] else np.zeros(n[b])
        logM.append((ga[:, None] + gb[None, :]).reshape(-1))
    c = np.concatenate([C.reshape(-1) for C in costs])
    lm = np.concatenate(logM)

    def z_of(y):
        return np.exp((A.T @ y - c) / eps + lm)

    def dual(y):
        return float(y @ rhs - eps * z_of(y).sum())

    y = np.zeros(A.shape[0])
    for _ in range(max_iter):
        z = z_of(y)
        g = rhs - A @ z
        if np.abs(g).max() < tol:
            break
        H = (A * z[None, :]) @ A.T / eps
        step = np.linalg.lstsq(H, g, rcond=None)[0]
        t, d0 = 1.0, dual(y)
        while dual(y + t * step) < d0 - 1e-15 * abs(d0) and t > 1e-12:
            t *= 0.5
        y = y + t * step
    z = z_of(y)
    val = float(c @ z + eps * np.sum(z * (np.log(z) - lm - 1.0)))
    return [z[offs[e]:offs[e + 1]].reshape(n[a], n[b]) for e, (a, b) in enumerate(edges)], val


def lp_optimum(J, edges, n, fixed, marginals, costs):
    """Optimal value of the unregularised tree LP (eq. ot_graph_pairwise) via HiGHS."""
    A, rhs, _ = _tree_constraints(J, edges, n, fixed, marginals)
    c = np.concatenate([C.reshape(-1) for C in costs])
    res = linprog(c, A_eq=A, b_eq=rhs, bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    return float(res.fun)


# ---------------------------------------------------------------------------
# coupled MOT on a modified junction tree (eq. ot_graph_local_reg), generic
# ---------------------------------------------------------------------------

def _projection(d, cvars, keep):
    """Matrix mapping a clique tensor (axes cvars, row-major) to its marginal on keep."""
    shape = tuple(int(d[v]) for v in cvars)
    idx = np.indices(shape).reshape(len(cvars), -1)
    kshape = tuple(int(d[v]) for v in keep)
    rows = np.zeros(idx.shape[1], dtype=np.int64)
    for v in keep:
        rows = rows * int(d[v]) + idx[cvars.index(v)]
    P = np.zeros((int(np.prod(kshape)) if keep else 1, idx.shape[1]))
    P[rows if keep else np.zeros_like(rows), np.arange(idx.shape[1])] = 1.0
    return P


def _jt_constraints(jt):
    offs = [0]
    for C in jt.clique_costs:
        offs.append(offs[-1] + C.size)
    nvar = offs[-1]

    def block(c, keep):
        P = _projection(jt.d, tuple(jt.clique_vars[c]), tuple(keep))
        out = np.zeros((P.shape[0], nvar))
        out[:, offs[c]:offs[c + 1]] = P
        return out

    A, rhs = [], []
    for s, cl in enumerate(jt.sep_cliques):
        sv = jt.sep_vars[s]
        sets = [tuple(v for v in sv if v in jt.clique_vars[c]) for c in cl]
        for i in range(1, len(cl)):
            A.append(block(cl[i], sets[i]) - block(cl[0], sets[i]))
            rhs.append(np.zeros(A[-1].shape[0]))
        if jt.sep_gamma[s] is None:
            A.append(block(cl[0], ()))
            rhs.append(np.ones(1))
        else:
            A.append(block(cl[0], tuple(jt.sep_gamma[s])))
            rhs.append(np.asarray(jt.sep_mu[s], dtype=np.float64).reshape(-1))
    return np.vstack(A), np.concatenate(rhs), offs


def jt_primal_generic(jt, tol=1e-14, max_iter=500):
    """Minimise sum_c <C_c,B_c> + eps H(B_c | M_c) under the constraints of eq.
    ot_graph_local_reg (separator plans eliminated: each neighbour's marginal on the
    intersection equals the first neighbour's; gamma marginal or unit mass), blind to
    the junction-tree algorithm: Newton on the Lagrangian dual as in primal_generic.
    M_c = m_{s_j} (x) m_{s_k} with m_s = mu_gamma (x) 1 (prop. local_reg_dual).
    Returns (plans, primal value)."""
    A, rhs, offs = _jt_constraints(jt)
    lm = []
    for c, cv in enumerate(jt.clique_vars):
        shape = tuple(int(jt.d[v]) for v in cv)
        a = np.zeros(shape)
        for s, cl in enumerate(jt.sep_cliques):
            if c in cl and jt.sep_gamma[s] is not None:
                g = tuple(jt.sep_gamma[s])
                with np.errstate(divide="ignore"):
                    lmu = np.log(np.asarray(jt.sep_mu[s], dtype=np.float64))
                sh = [int(jt.d[v]) if v in g else 1 for v in cv]
                order = sorted(range(len(g)), key=lambda k: cv.index(g[k]))
                a = a + np.transpose(lmu, order).reshape(sh)
        lm.append(a.reshape(-1))
    lm = np.concatenate(lm)
    c = np.concatenate([np.asarray(C, dtype=np.float64).reshape(-1) for C in jt.clique_costs])
    eps = jt.eps

    def z_of(y):
        with np.errstate(invalid="ignore"):
            return np.nan_to_num(np.exp((A.T @ y - c) / eps + lm))

    def dual(y):
        return float(y @ rhs - eps * z_of(y).sum())

    y = np.zeros(A.shape[0])
    for _ in range(max_iter):
        z = z_of(y)
        g = rhs - A @ z
        if np.abs(g).max() < tol:
            break
        H = (A * z[None, :]) @ A.T / eps
        step = np.linalg.lstsq(H, g, rcond=None)[0]
        t, d0 = 1.0, dual(y)
        while dual(y + t * step) < d0 - 1e-15 * abs(d0) and t > 1e-12:
            t *= 0.5
        y = y + t * step
    z = z_of(y)
    pos = z > 0
    val = float(c @ z + eps * np.sum(z[pos] * (np.log(z[pos]) - lm[pos] - 1.0)))
    return [z[offs[k]:offs[k + 1]].reshape(np.asarray(C).shape) for k, C in enumerate(jt.clique_costs)], val


def mot_lp_optimum(jt):
    """The unregularised multi-marginal problem over the joint distribution of all
    variables (eq. ot_graph): min sum_x (sum_c C_c(x_c)) pi(x) with the gamma marginals
    fixed and unit mass, solved with HiGHS on the full joint tensor (tiny cases only)."""
    V = len(jt.d)
    shape = tuple(int(v) for v in jt.d)
    idx = np.indices(shape).reshape(V, -1)
    cost = np.zeros(idx.shape[1])
    for cv, C in zip(jt.clique_vars, jt.clique_costs):
        cost += np.asarray(C, dtype=np.float64)[tuple(idx[v] for v in cv)]
    A, rhs = [np.ones((1, idx.shape[1]))], [np.ones(1)]
    for s in range(len(jt.sep_vars)):
        g = jt.sep_gamma[s]
        if g is None:
            continue
        P = _projection(jt.d, tuple(range(V)), tuple(g))
        A.append(P)
        rhs.append(np.asarray(jt.sep_mu[s], dtype=np.float64).reshape(-1))
    res = linprog(cost, A_eq=np.vstack(A), b_eq=np.concatenate(rhs), bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    return float(res.fun)

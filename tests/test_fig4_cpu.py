"""The paper's numerical experiment (Sec. 5, Fig. 4(a)) on the oracle: the
log-normal barycenter with the parameter choice of Sec. 3.2 (eps = delta / (4 |E|
log d), stopping threshold delta' = delta / (8 C_inf)).

Pins: the generator's instance matches the paper's description (grid, C_inf = 1,
probability vectors, parameters); the stopping threshold is reached within the
iteration bound of theorem thm:num_iter; the rounded plans are delta-approximate
against an LP optimum (lemma lem:round_applied with that parameter choice makes
the bound exactly delta/2 + 4 C_inf r < delta).  The plotted iteration counts
themselves are not in the paper's text, so only trends can be compared (the
benchmark reports them).
"""
import math

import numpy as np
import pytest

import gen
from oracle import tree_ot as O
import textbook_ot as TB


def test_instance_follows_the_paper():
    p = gen.lognormal_barycenter(1, 3, 10, delta=0.2)
    O.validate(p)
    assert p.num_nodes == 4 and not p.fixed[0] and all(p.fixed[1:])
    x = p.coords[1][:, 0].astype(np.float64)
    np.testing.assert_allclose(x, np.arange(10) / 9.0, rtol=0, atol=1e-7)
    assert O.c_infinity(p) == 1.0
    for l in (1, 2, 3):
        mu = p.marginals[l]
        assert abs(mu.sum() - 1.0) < 1e-14 and mu[0] == 0.0 and np.all(mu[1:] > 0)
    assert p.eps == pytest.approx(0.2 / (4 * 3 * math.log(10)), rel=1e-15)
    assert p.meta["tol"] == pytest.approx(0.2 / 8, rel=1e-15)
    # with this eps the entropic part of the bound of lem:round_applied is exactly delta / 2
    assert 2 * p.eps * p.num_edges * math.log(10) == pytest.approx(0.1, rel=1e-14)


@pytest.mark.parametrize("E,d,seed", [(2, 5, 0), (3, 8, 1), (3, 12, 2), (4, 6, 3)])
def test_delta_approximate_within_the_iteration_bound(E, d, seed):
    delta = 0.2
    p = gen.lognormal_barycenter(seed, E, d, delta)
    tol = p.meta["tol"]
    f, T, r = O.solve(p, tol=tol, tol_kind="sum", max_half_steps=100000)
    assert r < tol
    assert T <= 2 + 88 * E * O.c_infinity(p) / (tol * p.eps)                  # thm:num_iter
    R = O.round_plans(p, f, O.mismatched_side(T))
    tc = O.rounded_transport_cost(p, R)
    costs = [O.cost(p, int(a), int(b)) for a, b in p.edges]
    opt = TB.lp_optimum(p.num_nodes, [tuple(map(int, e)) for e in p.edges], [int(x) for x in p.n], p.fixed,
                        p.marginals, costs)
    bound = 2 * p.eps * E * math.log(d) + 4 * O.c_infinity(p) * r                 # lem:round_applied
    assert bound < delta
    assert opt - 1e-9 <= tc <= opt + bound + 1e-9

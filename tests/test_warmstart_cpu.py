"""Host-side logic of the learned warm start (no GPU): the star generator for
training / held-out sets, the (problem, directed edge) items and the input rows
the network sees, in matching order."""
import math

import numpy as np

import gen
from paper_2406_10849_gb300 import warmstart as W


def test_warmstart_stars_are_seeded_and_eps_in_range():
    a = gen.warmstart_stars(5_000_000, 6, side=8)
    b = gen.warmstart_stars(5_000_000, 6, side=8)
    for p, q in zip(a, b):
        assert p.eps == q.eps
        for j in p.marginals:
            np.testing.assert_array_equal(p.marginals[j], q.marginals[j])
    eps = [p.eps for p in gen.warmstart_stars(1, 200, side=4)]
    assert min(eps) >= 0.0025 and max(eps) <= 0.01
    assert len(set(eps)) > 150  # drawn per star
    fixed = gen.warmstart_stars(9_000_000, 3, side=8, eps=0.005)
    assert all(p.eps == 0.005 for p in fixed)
    # held-out seeds do not collide with training seeds
    assert not np.array_equal(gen.warmstart_stars(9_000_000, 1, side=8)[0].marginals[1],
                              gen.warmstart_stars(5_000_000, 1, side=8)[0].marginals[1])


def test_leaf_items_match_input_rows():
    probs = gen.warmstart_stars(123, 5, side=6)
    pr, de = W.leaf_items(probs)
    X = W.inputs(probs)
    assert X.dtype == np.float32 and X.shape == (5 * 8, 36 + 1)
    for r, (i, d) in enumerate(zip(pr, de)):
        p = probs[int(i)]
        a, b = np.asarray(p.edges)[int(d) // 2]
        owner = int(a) if int(d) % 2 == 0 else int(b)
        assert p.fixed[owner] and owner != 0            # the directed edge is leaf -> centre
        assert W.leaf_of(p, int(d)) == owner
        np.testing.assert_array_equal(X[r, :-1], np.asarray(p.marginals[owner], np.float32))
        assert X[r, -1] == np.float32(math.log(p.eps) + W.EPS_SHIFT)


def test_leaf_edges_of_star_centre_zero():
    p = gen.star_problem(seed=2000, leaves=8, side=4, eps=0.005)
    d = W.leaf_edges(p)
    assert len(d) == 8
    # edges (0, l): the leaf owns the second directed edge of each pair
    assert all(x % 2 == 1 for x in d)

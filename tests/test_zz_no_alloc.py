"""The allocation-free entry point (tree_ot_edge_apply_noalloc) through the C
ABI, on a GPU.

Some callers cannot allocate device memory: a serving runtime that hands out
every byte of device memory from its own pre-sized pool (and the plug-ins it
hosts), or a real-time loop that must not risk the device-wide synchronisation
cudaMalloc/cudaFree can cause.  They use this entry point, whose scratch is a
fixed array inside the library.  Its messages must equal those of the regular
solver for the same edge (read through a two-node problem: after one half-step
the fixed node's potential is f = -eps * m) and an FP64 log-sum-exp of the same
inputs, on two calls in a row (the second call reuses the scratch the first
one left behind).  This file is collected last, and the tests also pass on
their own in a fresh process.
"""
import numpy as np
import pytest

import gen
from gen.problems import TreeProblem
from oracle import tree_ot as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCRATCH_FLOATS = 1 << 20   # the fixed scratch array's size stated in include/tree_ot.h


def _need(n_rows, n_cols):
    """Scratch floats a request needs, as include/tree_ot.h states it."""
    return 2 * ((n_cols + 63) // 64 * 64) + 2 * n_rows * ((n_cols + 1023) // 1024)


def _regular_message(T, C, g, eps):
    """m(x) = LSE_y(g(y) - C(x,y)/eps) via tree_ot_create/set_potentials/half_steps."""
    n_rows, n_cols = C.shape
    rng = np.random.default_rng(5)
    mu = gen.dirichlet_marginal(n_rows, rng)
    p = TreeProblem(name="edge", edges=np.array([[0, 1]], np.int32), n=np.array([n_rows, n_cols], np.int32),
                    fixed=np.array([True, False]), marginals={0: mu}, eps=eps,
                    coords=[np.zeros((n_rows, 1), np.float32), np.zeros((n_cols, 1), np.float32)],
                    cost_scale=1.0, cost_kind="dense", dense_costs=[C])
    with T.Solver([p], T.options(precision="fp32")) as s:
        s.set_potential(0, 1, eps * g)       # f_(1,0) = eps g (node 1 is free: log gamma = 0)
        s.half_steps(1)                      # colour 0 = the fixed node 0: f_(0,1) = -eps m
        return -s.potential(0, 0) / eps


def _fp64_message(C, g, eps):
    """The same message in FP64 on the host (the oracle's two-pass log-sum-exp)."""
    return O.logsumexp(g[None, :] - C.astype(np.float64) / eps, axis=1)


def test_noalloc_matches_regular_path_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    rng = np.random.default_rng(11)
    n_rows, n_cols, eps = 1100, 2500, 0.02     # ragged rows and three 1024-column splits
    ld = 2504
    assert _need(n_rows, n_cols) <= SCRATCH_FLOATS
    X = rng.random((n_rows, 3)).astype(np.float32)
    Y = rng.random((n_cols, 3)).astype(np.float32)
    C = gen.sqeuclid_cost_f32(X, Y, 1.0)
    inf_row = 7
    C[inf_row, :] = np.inf                     # every term of this row is zero: m = -inf
    C_pad = np.full((n_rows, ld), 7.0, np.float32)   # padding the entry point must ignore
    C_pad[:, :n_cols] = C
    dev = torch.device("cuda")
    cost = torch.from_numpy(C_pad).to(dev)
    m_out = torch.full((n_rows,), float("nan"), dtype=torch.float64, device=dev)
    rows = np.arange(n_rows) != inf_row
    for call in range(2):
        g = rng.normal(0.0, 3.0, size=n_cols) + np.log(rng.dirichlet(np.ones(n_cols)))
        T.treeot.edge_apply_noalloc(cost, torch.from_numpy(g).to(dev), eps, m_out, ld=ld)
        torch.cuda.synchronize()
        got = m_out.cpu().numpy()
        exact = _fp64_message(C, g, eps)
        assert got[inf_row] == -np.inf and exact[inf_row] == -np.inf, call
        assert np.all(np.isfinite(got[rows])), call
        # FP32 terms and sums: ~1e-7 of the row's sum, i.e. ~1e-7 absolute in m; bound 1e-6
        scale = np.maximum(1.0, np.abs(exact[rows]))
        assert float(np.max(np.abs(got[rows] - exact[rows]) / scale)) <= 1e-6, call
        # the regular path (the solver's own apply) carries the same FP32 error: within twice that
        ref = _regular_message(T, C, g, eps)
        assert float(np.max(np.abs(got[rows] - ref[rows]) / scale)) <= 2e-6, call


def test_noalloc_rejects_oversize_request():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_10849_gb300 as T
    T.load()
    dev = torch.device("cuda")
    n_rows, n_cols = 1, 600_000                # a fully backed 2.4 MB row
    assert _need(n_rows, n_cols) > SCRATCH_FLOATS
    cost = torch.zeros((n_rows, n_cols), dtype=torch.float32, device=dev)
    g = torch.zeros(n_cols, dtype=torch.float64, device=dev)
    m_out = torch.zeros(n_rows, dtype=torch.float64, device=dev)
    with pytest.raises(T.TreeOTError) as ei:
        T.treeot.edge_apply_noalloc(cost, g, 0.1, m_out)
    assert ei.value.kind == "ARG"
    torch.cuda.synchronize()

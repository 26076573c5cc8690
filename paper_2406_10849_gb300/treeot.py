"""ctypes binding of libtreeot.so (include/tree_ot.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  If the shared library
is missing this module raises at import time; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtreeot.so")

OK = 0
NOT_CONVERGED = 1
ERR = {
    -1: "ARG", -2: "NOT_TREE", -3: "FIXED_NOT_LEAF", -4: "FIXED_ADJACENT", -5: "MARGINAL",
    -6: "NONFINITE", -7: "EPS", -8: "CUDA", -9: "OOM", -10: "TIMEOUT", -11: "STATE",
}
COST_DENSE_F32 = 0
COST_SQEUCLID = 1
INPUT_DEVICE = 1
PREC = {"fp32": 0, "fp64": 1}
TOL_KIND = {"sum": 0, "max": 1}
APPLY = {"auto": 0, "lse": 1, "bf16": 2}


PROFILE_CATEGORIES = ["apply_stored", "apply_recompute", "apply_bf16", "sk_build", "sk_product", "sk_fixup",
                      "node_update", "absorb", "check", "round", "apply_fp64", "forest"]


class TreeOTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tree_ot error {code} ({ERR.get(code, '?')}): {msg}")
        self.code = code
        self.kind = ERR.get(code, "?")


class Problem(C.Structure):
    _fields_ = [
        ("num_nodes", C.c_int32),
        ("edges", C.POINTER(C.c_int32)),
        ("support_size", C.POINTER(C.c_int32)),
        ("is_fixed", C.POINTER(C.c_uint8)),
        ("marginal", C.POINTER(C.POINTER(C.c_double))),
        ("eps", C.c_double),
        ("cost_kind", C.c_int32),
        ("dim", C.c_int32),
        ("coords", C.POINTER(C.POINTER(C.c_float))),
        ("cost_scale", C.c_double),
        ("dense_cost", C.POINTER(C.POINTER(C.c_float))),
        ("flags", C.c_uint32),
    ]


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int32),
        ("apply_mode", C.c_int32),
        ("tol", C.c_double),
        ("tol_kind", C.c_int32),
        ("max_half_steps", C.c_int64),
        ("check_every", C.c_int32),
        ("use_graph", C.c_int32),
        ("flags", C.c_uint32),
        ("refine_tol", C.c_double),
        ("absorb_tau", C.c_double),
        ("lowp_start", C.c_int32),
        ("autotune", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("half_steps", C.c_int64),
        ("residual_sum_l1", C.c_double),
        ("max_marginal_l1", C.c_double),
        ("primal", C.c_double),
        ("dual", C.c_double),
        ("transport_cost", C.c_double),
        ("wall_ms", C.c_double),
        ("lowp_half_steps", C.c_int64),
        ("absorptions", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RoundResult(C.Structure):
    _fields_ = [
        ("side", C.c_int32),
        ("half_steps", C.c_int64),
        ("residual_sum_l1", C.c_double),
        ("transport_cost", C.c_double),
        ("rounded_transport_cost", C.c_double),
        ("c_inf", C.c_double),
        ("bound", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every exported symbol of include/tree_ot.h with its ctypes signature
SIGNATURES = {
    "tree_ot_default_options": (None, [C.POINTER(Options)]),
    "tree_ot_error_string": (C.c_char_p, [C.c_int]),
    "tree_ot_last_error": (C.c_char_p, []),
    "tree_ot_validate": (C.c_int, [C.POINTER(Problem)]),
    "tree_ot_bipartition": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_uint8)]),
    "tree_ot_create": (C.c_int, [C.POINTER(Problem), C.c_int32, C.POINTER(Options), C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    "tree_ot_destroy": (C.c_int, [C.c_void_p]),
    "tree_ot_reset": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tree_ot_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Result)]),
    "tree_ot_half_steps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "tree_ot_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "tree_ot_node_update": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "tree_ot_check": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Result)]),
    "tree_ot_marginals": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "tree_ot_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "tree_ot_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    "tree_ot_round": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(RoundResult)]),
    "tree_ot_round_plan": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64]),
    "tree_ot_residual_history": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int64,
                                           C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "tree_ot_get_potentials": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "tree_ot_set_potentials": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "tree_ot_set_potentials_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                               C.POINTER(C.c_int32), C.c_void_p, C.c_int64]),
    "tree_ot_get_potentials_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                               C.POINTER(C.c_int32), C.c_void_p, C.c_int64, C.c_uint32]),
    "tree_ot_plan_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_int32]),
    "tree_ot_edge_apply_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_double,
                                             C.c_void_p, C.c_void_p]),
    "tree_ot_mlp_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(C.c_void_p)]),
    "tree_ot_mlp_destroy": (C.c_int, [C.c_void_p]),
    "tree_ot_mlp_num_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "tree_ot_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tree_ot_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tree_ot_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "tree_ot_mlp_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                       C.POINTER(C.c_double)]),
    "tree_ot_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double,
                                         C.POINTER(C.c_double)]),
    "tree_ot_mlp_last_error": (C.c_char_p, []),
    "tree_ot_mlp_set_input_log": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_double]),
    "tree_ot_jt_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "tree_ot_jt_destroy": (C.c_int, [C.c_void_p]),
    "tree_ot_jt_reset": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tree_ot_jt_half_steps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "tree_ot_jt_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "tree_ot_jt_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_int64, C.c_int32,
                                   C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "tree_ot_jt_plan": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double)]),
    "tree_ot_jt_transport_cost": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "tree_ot_jt_get_dual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "tree_ot_jt_colour": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libtreeot.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, allow=(OK,)):
    if rc in allow:
        return rc
    msg = _lib.tree_ot_last_error().decode(errors="replace")
    raise TreeOTError(rc, msg)


def torch_float32():
    import torch
    return torch.float32


def _stream_ptr(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr_of(obj, ctype):
    """(pointer, keepalive) for a numpy array or a torch tensor (host or device)."""
    if hasattr(obj, "data_ptr"):
        return C.cast(C.c_void_p(obj.data_ptr()), C.POINTER(ctype)), obj
    arr = np.ascontiguousarray(obj)
    return arr.ctypes.data_as(C.POINTER(ctype)), arr


class _Marshalled:
    """ctypes image of one problem plus the buffers it points into."""

    def __init__(self, p, device_costs=None, device_coords=None):
        keep = []
        J = int(p.num_nodes)
        self.J = J
        edges = np.ascontiguousarray(np.asarray(p.edges, dtype=np.int32).reshape(-1))
        n = np.ascontiguousarray(np.asarray(p.n, dtype=np.int32))
        fixed = np.ascontiguousarray(np.asarray(p.fixed, dtype=np.uint8))
        keep += [edges, n, fixed]
        marg_ptrs = (C.POINTER(C.c_double) * J)()
        for j in range(J):
            if fixed[j]:
                m = np.ascontiguousarray(np.asarray(p.marginals[j], dtype=np.float64))
                keep.append(m)
                marg_ptrs[j] = m.ctypes.data_as(C.POINTER(C.c_double))
        keep.append(marg_ptrs)
        flags = 0
        coord_src = device_coords if device_coords is not None else p.coords
        coords_ptrs = (C.POINTER(C.c_float) * J)()
        dim = int(p.coords[0].shape[1]) if p.coords is not None else 0
        for j in range(J):
            ptr, k = _ptr_of(coord_src[j] if device_coords is not None
                             else np.asarray(p.coords[j], dtype=np.float32), C.c_float)
            keep.append(k)
            coords_ptrs[j] = ptr
        keep.append(coords_ptrs)
        dense_ptrs = None
        kind = COST_SQEUCLID if p.cost_kind == "sqeuclid" else COST_DENSE_F32
        if kind == COST_DENSE_F32:
            dense_ptrs = (C.POINTER(C.c_float) * max(1, J - 1))()
            for e in range(J - 1):
                src = device_costs[e] if device_costs is not None else p.dense_cost(e)
                ptr, k = _ptr_of(src, C.c_float)
                keep.append(k)
                dense_ptrs[e] = ptr
            keep.append(dense_ptrs)
        if device_costs is not None or device_coords is not None:
            flags |= INPUT_DEVICE
            if device_coords is None:
                # device flag covers coords too: stage them on the device
                import torch
                dcs = [torch.as_tensor(np.asarray(c, np.float32)).cuda() for c in p.coords]
                keep += dcs
                for j in range(J):
                    coords_ptrs[j] = C.cast(C.c_void_p(dcs[j].data_ptr()), C.POINTER(C.c_float))
        self.struct = Problem(
            num_nodes=J,
            edges=edges.ctypes.data_as(C.POINTER(C.c_int32)),
            support_size=n.ctypes.data_as(C.POINTER(C.c_int32)),
            is_fixed=fixed.ctypes.data_as(C.POINTER(C.c_uint8)),
            marginal=marg_ptrs,
            eps=float(p.eps),
            cost_kind=kind,
            dim=dim,
            coords=coords_ptrs,
            cost_scale=float(p.cost_scale),
            dense_cost=dense_ptrs,
            flags=flags,
        )
        self.keep = keep


def options(precision="fp32", tol=1e-6, tol_kind="sum", max_half_steps=100000, check_every=32, use_graph=True,
            apply_mode="auto", refine_tol=None, absorb_tau=None, lowp_start=None, autotune=None,
            dense_kernel="auto", exact_dist=False, transpose=True, test_stall=False, sk_product="auto",
            persistent=False, node_finish="auto") -> Options:
    """tree_ot_options with the defaults of tree_ot_default_options; dense_kernel picks the
    stored-cost apply ("auto": the autotuner's choice, "tma": bulk-copy staged, "ldg": plain loads);
    exact_dist: recompute squared distances exactly from the first half-step;
    transpose: keep stored costs also transposed when the device has room;
    test_stall: test hook, the staged kernel's producer issues nothing (its waits run out);
    persistent: allow the persistent forest launch (TREE_OT_OPT_PERSISTENT; kept only where the
    create-time timing finds it faster);
    sk_product: the shared-kernel BF16 phase's product ("auto": tcgen05 over CTA pairs where
    available, "one_cta": tcgen05 with one CTA per 128-row tile, "mma": the legacy mma.sync kernel);
    node_finish: where the node update's bookkeeping runs ("auto": by chunk count per colour,
    "defer": an extra launch after the chunks, "arrive": the last-arriving chunk)."""
    load()
    o = Options()
    _lib.tree_ot_default_options(C.byref(o))
    o.precision = PREC[precision]
    o.apply_mode = APPLY[apply_mode]
    o.tol = float(tol)
    o.tol_kind = TOL_KIND[tol_kind]
    o.max_half_steps = int(max_half_steps)
    o.check_every = int(check_every)
    o.use_graph = 1 if use_graph else 0
    if refine_tol is not None:
        o.refine_tol = float(refine_tol)
    if absorb_tau is not None:
        o.absorb_tau = float(absorb_tau)
    if lowp_start is not None:
        o.lowp_start = int(lowp_start)
    if autotune is not None:
        o.autotune = 1 if autotune else 0
    o.flags = ({"auto": 0, "tma": 1, "ldg": 2}[dense_kernel] | (4 if exact_dist else 0) | (0 if transpose else 8)
               | (16 if test_stall else 0) | {"auto": 0, "mma": 32, "one_cta": 512}[sk_product] | (64 if persistent else 0)
               | {"auto": 0, "defer": 128, "arrive": 256}[node_finish])
    return o


def validate(problem) -> int:
    """tree_ot_validate on one problem; returns the code (0 = valid)."""
    load()
    m = _Marshalled(problem)
    return _lib.tree_ot_validate(C.byref(m.struct))


def bipartition(num_nodes: int, edges) -> np.ndarray:
    load()
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    out = np.zeros(num_nodes, dtype=np.uint8)
    _check(_lib.tree_ot_bipartition(num_nodes, e.ctypes.data_as(C.POINTER(C.c_int32)),
                                    out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out


class Solver:
    """One handle over a batch of problems (tree_ot_create .. tree_ot_destroy)."""

    def __init__(self, problems: Sequence, opts: Optional[Options] = None, stream=None,
                 device_costs: Optional[List] = None, device_coords: Optional[List] = None, **kw):
        load()
        self.problems = list(problems)
        dc = device_costs if device_costs is not None else [None] * len(self.problems)
        dk = device_coords if device_coords is not None else [None] * len(self.problems)
        self._m = [_Marshalled(p, dc[i], dk[i]) for i, p in enumerate(self.problems)]
        arr = (Problem * len(self._m))(*[m.struct for m in self._m])
        self._arr = arr
        self.opts = opts if opts is not None else options(**kw)
        self.stream = stream
        h = C.c_void_p()
        _check(_lib.tree_ot_create(arr, len(self._m), C.byref(self.opts), C.c_void_p(_stream_ptr(stream)),
                                   C.byref(h)))
        self.h = h
        # borrowed device buffers must outlive the handle
        self._borrowed = [m.keep for m in self._m]

    def _s(self):
        return C.c_void_p(_stream_ptr(self.stream))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.tree_ot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self):
        res = (Result * len(self._m))()
        rc = _check(_lib.tree_ot_solve(self.h, self._s(), res), allow=(OK, NOT_CONVERGED))
        return rc, [r.as_dict() for r in res]

    def half_steps(self, T: int):
        _check(_lib.tree_ot_half_steps(self.h, self._s(), int(T)))

    def apply(self, colour: int):
        _check(_lib.tree_ot_apply(self.h, self._s(), int(colour)))

    def node_update(self, colour: int):
        _check(_lib.tree_ot_node_update(self.h, self._s(), int(colour)))

    def reset(self):
        _check(_lib.tree_ot_reset(self.h, self._s()))

    def check(self):
        res = (Result * len(self._m))()
        _check(_lib.tree_ot_check(self.h, self._s(), res))
        return [r.as_dict() for r in res]

    def marginal(self, prob: int, node: int) -> np.ndarray:
        n = int(self.problems[prob].n[node])
        out = np.zeros(n, np.float64)
        _check(_lib.tree_ot_marginals(self.h, prob, node, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def profile(self, enable: bool = True):
        """tree_ot_profile: time every launch group queued outside graph capture."""
        _check(_lib.tree_ot_profile(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{category: (milliseconds, launch groups)} since the last read (tree_ot_profile_read)."""
        n = len(PROFILE_CATEGORIES)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        _check(_lib.tree_ot_profile_read(self.h, ms, cnt, n))
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(PROFILE_CATEGORIES) if cnt[i]}

    def round(self, side: int = -1):
        """tree_ot_round: round every problem's plans (the mismatched colour class by default);
        returns one dict per problem (costs before / after rounding, r, C_inf, the bound)."""
        res = (RoundResult * len(self._m))()
        _check(_lib.tree_ot_round(self.h, self._s(), int(side), res))
        return [r.as_dict() for r in res]

    def round_plan(self, prob: int, edge: int, out=None):
        """tree_ot_round_plan into a CUDA float64 (n_a, n_b) tensor (rows on edges[edge][0])."""
        import torch
        p = self.problems[prob]
        a, b = (int(v) for v in p.edges[edge])
        shape = (int(p.n[a]), int(p.n[b]))
        if out is None:
            out = torch.zeros(shape, dtype=torch.float64, device="cuda")
        if (tuple(out.shape) != shape or out.dtype != torch.float64 or not out.is_cuda or out.stride(1) != 1
                or out.device.index != torch.cuda.current_device()):
            raise ValueError(f"out must be a CUDA float64 {shape} matrix with unit column stride on the current device")
        _check(_lib.tree_ot_round_plan(self.h, self._s(), int(prob), int(edge), C.c_void_p(out.data_ptr()),
                                       int(out.stride(0))))
        return out

    def residual_history(self, prob: int, first: int, count: int):
        """(sums, maxima) of the stopping quantity of iterates first .. first+count-1,
        as the half-step kernels accumulated it (tree_ot_residual_history)."""
        sums = np.zeros(int(count), np.float64)
        maxs = np.zeros(int(count), np.float64)
        _check(_lib.tree_ot_residual_history(self.h, self._s(), int(prob), int(first), int(count),
                                             sums.ctypes.data_as(C.POINTER(C.c_double)),
                                             maxs.ctypes.data_as(C.POINTER(C.c_double))))
        return sums, maxs

    def potential(self, prob: int, dedge: int) -> np.ndarray:
        p = self.problems[prob]
        e = dedge // 2
        owner = int(p.edges[e][dedge % 2])
        out = np.zeros(int(p.n[owner]), np.float64)
        _check(_lib.tree_ot_get_potentials(self.h, self._s(), prob, dedge,
                                           out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def potentials(self, prob: int = 0) -> dict:
        """{(j,k): f_(j,k)} for every directed edge of problem ``prob``."""
        p = self.problems[prob]
        out = {}
        for e, (a, b) in enumerate(np.asarray(p.edges)):
            out[(int(a), int(b))] = self.potential(prob, 2 * e)
            out[(int(b), int(a))] = self.potential(prob, 2 * e + 1)
        return out

    def set_potential(self, prob: int, dedge: int, values):
        v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
        _check(_lib.tree_ot_set_potentials(self.h, self._s(), prob, dedge, v.ctypes.data_as(C.POINTER(C.c_double))))

    def set_potentials_batch(self, probs, dedges, values):
        """tree_ot_set_potentials_batch: row i of the CUDA float32 matrix `values`
        becomes the potential of directed edge dedges[i] of problem probs[i]."""
        pr = np.ascontiguousarray(np.asarray(probs, dtype=np.int32))
        de = np.ascontiguousarray(np.asarray(dedges, dtype=np.int32))
        if pr.shape != de.shape or values.dim() != 2 or values.shape[0] != pr.shape[0]:
            raise ValueError("probs, dedges and the rows of values must match")
        if values.dtype != torch_float32() or not values.is_cuda or values.stride(1) != 1:
            raise ValueError("values must be a CUDA float32 matrix with unit column stride")
        _check(_lib.tree_ot_set_potentials_batch(self.h, self._s(), int(pr.shape[0]),
                                                 pr.ctypes.data_as(C.POINTER(C.c_int32)),
                                                 de.ctypes.data_as(C.POINTER(C.c_int32)),
                                                 C.c_void_p(values.data_ptr()), int(values.stride(0))))

    def get_potentials_batch(self, probs, dedges, out, centred: bool = False):
        """tree_ot_get_potentials_batch into the CUDA float32 matrix `out` (row i:
        directed edge dedges[i] of problem probs[i]); centred: mean over x removed."""
        pr = np.ascontiguousarray(np.asarray(probs, dtype=np.int32))
        de = np.ascontiguousarray(np.asarray(dedges, dtype=np.int32))
        if pr.shape != de.shape or out.dim() != 2 or out.shape[0] != pr.shape[0]:
            raise ValueError("probs, dedges and the rows of out must match")
        if out.dtype != torch_float32() or not out.is_cuda or out.stride(1) != 1:
            raise ValueError("out must be a CUDA float32 matrix with unit column stride")
        _check(_lib.tree_ot_get_potentials_batch(self.h, self._s(), int(pr.shape[0]),
                                                 pr.ctypes.data_as(C.POINTER(C.c_int32)),
                                                 de.ctypes.data_as(C.POINTER(C.c_int32)),
                                                 C.c_void_p(out.data_ptr()), int(out.stride(0)),
                                                 1 if centred else 0))
        return out

    def set_potentials(self, f: dict, prob: int = 0):
        p = self.problems[prob]
        for e, (a, b) in enumerate(np.asarray(p.edges)):
            self.set_potential(prob, 2 * e, f[(int(a), int(b))])
            self.set_potential(prob, 2 * e + 1, f[(int(b), int(a))])

    def plan_stats(self) -> dict:
        st = (C.c_int64 * 16)()
        _check(_lib.tree_ot_plan_stats(self.h, st, 16))
        keys = ["directed_edges", "edges", "elements_per_half_step", "matrix_bytes_per_half_step",
                "apply_tasks_c0", "apply_tasks_c1", "device_bytes", "node_ctas_c0", "node_ctas_c1",
                "recompute_output_block", "recompute_ctas_per_sm", "recompute_variant", "dense_tma",
                "persistent", "node_defer", "sk_product"]
        return dict(zip(keys, [int(x) for x in st]))


def edge_apply_noalloc(cost, g, eps: float, m_out, ld: int = None, stream=None):
    """tree_ot_edge_apply_noalloc on device tensors: m_out[x] = LSE_y(g[y] - cost[x, y] / eps).

    cost: CUDA float32 (n_rows, ld) tensor (its first n_cols = len(g) columns are used),
    g: CUDA float64 (n_cols,), m_out: CUDA float64 (n_rows,).  Marshalling only.
    """
    load()
    import torch
    if cost.dim() != 2 or g.dim() != 1 or m_out.dim() != 1:
        raise ValueError("cost must be a matrix, g and m_out vectors")
    if cost.dtype != torch.float32 or g.dtype != torch.float64 or m_out.dtype != torch.float64:
        raise ValueError("cost must be float32, g and m_out float64")
    if not (cost.is_cuda and g.is_cuda and m_out.is_cuda):
        raise ValueError("cost, g and m_out must be CUDA tensors")
    cur = torch.cuda.current_device()
    if cost.device.index != cur or g.device.index != cur or m_out.device.index != cur:
        raise ValueError("cost, g and m_out must live on the current CUDA device")
    if cost.stride(1) != 1 or g.stride(0) != 1 or m_out.stride(0) != 1:
        raise ValueError("cost rows, g and m_out must be contiguous")
    n_rows = int(cost.shape[0])
    n_cols = int(g.shape[0])
    ld = int(cost.stride(0)) if ld is None else int(ld)
    # every row the kernel reads (x * ld .. x * ld + n_cols) must lie inside the tensor's storage
    reach = (n_rows - 1) * ld + n_cols
    avail = cost.untyped_storage().nbytes() // 4 - cost.storage_offset()
    if n_cols > int(cost.shape[1]) or ld < n_cols or reach > avail or int(m_out.shape[0]) < n_rows:
        raise ValueError("need len(g) <= cost columns, ld >= len(g), rows of stride ld inside the cost's "
                         "storage and len(m_out) >= cost rows")
    _check(_lib.tree_ot_edge_apply_noalloc(C.c_void_p(cost.data_ptr()), ld, n_rows, n_cols,
                                           C.c_void_p(g.data_ptr()), float(eps), C.c_void_p(m_out.data_ptr()),
                                           C.c_void_p(_stream_ptr(stream))))


def _mcheck(rc: int):
    if rc != OK:
        raise TreeOTError(rc, _lib.tree_ot_mlp_last_error().decode(errors="replace"))


class MLP:
    """tree_ot_mlp_*: the warm-start predictor (device tensors in, device tensors out)."""

    def __init__(self, in_dim: int, hidden: int, out_dim: int, max_batch: int, seed: int = 0):
        load()
        h = C.c_void_p()
        _mcheck(_lib.tree_ot_mlp_create(in_dim, hidden, out_dim, max_batch, seed, C.byref(h)))
        self.h = h
        self.in_dim, self.hidden, self.out_dim, self.max_batch = in_dim, hidden, out_dim, max_batch
        n = C.c_int64()
        offs = (C.c_int64 * 6)()
        _mcheck(_lib.tree_ot_mlp_num_params(h, C.byref(n), offs))
        self.num_params = int(n.value)
        self.offsets = [int(o) for o in offs]

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.tree_ot_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_input_log(self, count: int, floor_value: float = 1e-30, scale: float = 1.0):
        _mcheck(_lib.tree_ot_mlp_set_input_log(self.h, int(count), float(floor_value), float(scale)))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params, np.float32)
        _mcheck(_lib.tree_ot_mlp_get_params(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, np.float32))
        assert p.size == self.num_params
        _mcheck(_lib.tree_ot_mlp_set_params(self.h, p.ctypes.data_as(C.c_void_p)))

    def tensors(self, flat) -> dict:
        """Split a flat parameter vector into W1, b1, W2, b2, W3, b3 views."""
        shapes = [(self.hidden, self.in_dim), (self.hidden,), (self.hidden, self.hidden), (self.hidden,),
                  (self.out_dim, self.hidden), (self.out_dim,)]
        names = ["W1", "b1", "W2", "b2", "W3", "b3"]
        return {nm: flat[o:o + int(np.prod(sh))].reshape(sh) for nm, o, sh in zip(names, self.offsets, shapes)}

    def forward(self, x, y, stream=None):
        _mcheck(_lib.tree_ot_mlp_forward(self.h, C.c_void_p(_stream_ptr(stream)), C.c_void_p(x.data_ptr()),
                                         int(x.shape[0]), C.c_void_p(y.data_ptr())))

    def backward(self, x, target, grads=None, stream=None) -> float:
        loss = C.c_double()
        _mcheck(_lib.tree_ot_mlp_backward(self.h, C.c_void_p(_stream_ptr(stream)), C.c_void_p(x.data_ptr()),
                                          C.c_void_p(target.data_ptr()), int(x.shape[0]),
                                          C.c_void_p(grads.data_ptr()) if grads is not None else None,
                                          C.byref(loss)))
        return float(loss.value)

    def train_step(self, x, target, lr: float, stream=None) -> float:
        loss = C.c_double()
        _mcheck(_lib.tree_ot_mlp_train_step(self.h, C.c_void_p(_stream_ptr(stream)), C.c_void_p(x.data_ptr()),
                                            C.c_void_p(target.data_ptr()), int(x.shape[0]), float(lr),
                                            C.byref(loss)))
        return float(loss.value)


# ---- general graphs: modified junction trees (tree_ot_jt_*) ----------------

class JtProblem(C.Structure):
    _fields_ = [
        ("num_vars", C.c_int32),
        ("var_size", C.POINTER(C.c_int32)),
        ("num_cliques", C.c_int32),
        ("clique_var_begin", C.POINTER(C.c_int32)),
        ("clique_vars", C.POINTER(C.c_int32)),
        ("clique_cost", C.POINTER(C.POINTER(C.c_float))),
        ("num_seps", C.c_int32),
        ("sep_var_begin", C.POINTER(C.c_int32)),
        ("sep_vars", C.POINTER(C.c_int32)),
        ("sep_clique_begin", C.POINTER(C.c_int32)),
        ("sep_cliques", C.POINTER(C.c_int32)),
        ("sep_gamma_begin", C.POINTER(C.c_int32)),
        ("sep_gamma", C.POINTER(C.c_int32)),
        ("sep_mu", C.POINTER(C.POINTER(C.c_double))),
        ("eps", C.c_double),
    ]


def _flat(lists):
    begin = np.zeros(len(lists) + 1, np.int32)
    for i, l in enumerate(lists):
        begin[i + 1] = begin[i] + len(l)
    items = np.array([int(x) for l in lists for x in l] or [0], np.int32)
    return begin, items


class JunctionSolver:
    """One handle over a modified junction tree (tree_ot_jt_create .. tree_ot_jt_destroy).
    ``jt`` carries d (support size per variable), clique_vars, clique_costs (arrays with
    axes in the clique's variable order), sep_vars, sep_cliques (inclusion order),
    sep_gamma (None or the constraint's variables), sep_mu and eps."""

    def __init__(self, jt, stream=None):
        load()
        self.jt = jt
        self.stream = stream
        keep = []
        d = np.ascontiguousarray(np.asarray(jt.d, np.int32))
        cb, cv = _flat(jt.clique_vars)
        sb, sv = _flat(jt.sep_vars)
        kb, kc = _flat(jt.sep_cliques)
        gb, gv = _flat([g if g is not None else () for g in jt.sep_gamma])
        costs = [np.ascontiguousarray(np.asarray(c, np.float32)).reshape(-1) for c in jt.clique_costs]
        mus = [None if g is None else np.ascontiguousarray(np.asarray(m, np.float64)).reshape(-1)
               for g, m in zip(jt.sep_gamma, jt.sep_mu)]
        keep += [d, cb, cv, sb, sv, kb, kc, gb, gv] + costs + [m for m in mus if m is not None]
        cost_ptrs = (C.POINTER(C.c_float) * len(costs))(*[c.ctypes.data_as(C.POINTER(C.c_float)) for c in costs])
        mu_ptrs = (C.POINTER(C.c_double) * len(mus))(
            *[m.ctypes.data_as(C.POINTER(C.c_double)) if m is not None else C.POINTER(C.c_double)() for m in mus])
        keep += [cost_ptrs, mu_ptrs]
        i32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        self.struct = JtProblem(len(d), i32(d), len(costs), i32(cb), i32(cv), cost_ptrs, len(jt.sep_vars), i32(sb),
                                i32(sv), i32(kb), i32(kc), i32(gb), i32(gv), mu_ptrs, float(jt.eps))
        self._keep = keep
        h = C.c_void_p()
        _check(_lib.tree_ot_jt_create(C.byref(self.struct), C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self.h = h

    def _s(self):
        return C.c_void_p(_stream_ptr(self.stream))

    def close(self):
        if getattr(self, "h", None):
            _lib.tree_ot_jt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self):
        _check(_lib.tree_ot_jt_reset(self.h, self._s()))

    def half_steps(self, T: int):
        _check(_lib.tree_ot_jt_half_steps(self.h, self._s(), int(T)))

    def residual(self):
        s, m = C.c_double(), C.c_double()
        _check(_lib.tree_ot_jt_residual(self.h, self._s(), C.byref(s), C.byref(m)))
        return s.value, m.value

    def solve(self, tol: float, tol_kind: str = "sum", max_half_steps: int = 100000, check_every: int = 16):
        hs, r = C.c_int64(), C.c_double()
        rc = _check(_lib.tree_ot_jt_solve(self.h, self._s(), float(tol), TOL_KIND[tol_kind], int(max_half_steps),
                                          int(check_every), C.byref(hs), C.byref(r)), allow=(OK, NOT_CONVERGED))
        return rc, int(hs.value), r.value

    def plan(self, clique: int) -> np.ndarray:
        shape = tuple(int(self.jt.d[v]) for v in self.jt.clique_vars[clique])
        out = np.zeros(int(np.prod(shape)), np.float64)
        _check(_lib.tree_ot_jt_plan(self.h, self._s(), int(clique), out.ctypes.data_as(C.POINTER(C.c_double))))
        return out.reshape(shape)

    def transport_cost(self) -> float:
        v = C.c_double()
        _check(_lib.tree_ot_jt_transport_cost(self.h, self._s(), C.byref(v)))
        return v.value

    def dual(self, sep: int, pos: int) -> np.ndarray:
        c = self.jt.sep_cliques[sep][pos]
        vars_ = [v for v in self.jt.sep_vars[sep] if v in self.jt.clique_vars[c]]
        shape = tuple(int(self.jt.d[v]) for v in vars_)
        out = np.zeros(int(np.prod(shape)) if shape else 1, np.float64)
        _check(_lib.tree_ot_jt_get_dual(self.h, self._s(), int(sep), int(pos),
                                        out.ctypes.data_as(C.POINTER(C.c_double))))
        return out.reshape(shape) if shape else out[0]

    def colours(self) -> np.ndarray:
        out = np.zeros(len(self.jt.sep_vars), np.int32)
        _check(_lib.tree_ot_jt_colour(self.h, out.ctypes.data_as(C.POINTER(C.c_int32))))
        return out

"""Benchmark: edge-kernel applies per second of the bipartite scaling sweep.

Workload (default): a 64-node random tree (Pruefer sequence, exactly 32 fixed
leaves), n = 4096 support points per node drawn uniformly in [0,1]^3, a stored
dense FP32 cost per edge (63 edges, 4.2 GB on the device), Dirichlet(1) leaf
marginals, eps = 0.01.  One step = one half-step of the sweep: the edge-apply
launch (every edge's Gibbs kernel applied once toward the active colour, in
log-sum-exp form, reading all 4.2 GB) followed by the node-update launch
(block updates of thm:tree_dual_var + stopping terms).  63 edge applies per step.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "edge-kernel applies/sec"
UNIT = "edge_applies/s"
WORKLOAD = "prufer64_n4096_dense_fp32_eps0.01"
NODES = 64


def workload_name(nodes: int) -> str:
    return WORKLOAD if nodes == 64 else f"prufer{nodes}_n4096_dense_fp32_eps0.01"


def workload_problem(nodes: int = NODES):
    """The Pruefer-tree workload; nodes < 64 gives the same construction on a smaller
    tree (used for profiling captures that must stay small)."""
    import gen
    return gen.prufer_problem(seed=3000, J=nodes, n=4096, num_leaves=nodes // 2, D=3, eps=0.01)


def algorithmic_bytes(p) -> int:
    """Bytes one apply launch must move: each stored cost entry once (4 B) plus
    the two-float operand of the reduction side and the output of the active side
    (8 B per support point on each side of every edge)."""
    tot = 0
    for a, b in np.asarray(p.edges):
        na, nb = int(p.n[a]), int(p.n[b])
        tot += 4 * na * nb + 8 * (na + nb)
    return tot


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def read_bf16_peak():
    """Dense BF16 tensor throughput (TFLOP/s): the measured burst figure, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["bf16_tflops"]), "bf16_tflops (burst) of measured"
    except Exception:
        return 1900.0, "fallback"


KERNEL_SOURCES = {"apply_dense_kernel": "apply_f32.cu", "apply_dense_tma_kernel": "apply_tma.cu"}


def kernel_hash(kernel: str = "apply_dense_kernel") -> str:
    """Hash of the code a kernel is built from (its source, ptx.cuh and internal.h),
    with line comments and blank lines dropped: editing a comment keeps a profile
    valid, editing code does not."""
    h = hashlib.sha256()
    for f in (KERNEL_SOURCES[kernel], "ptx.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_2406_10849_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, kernel: str):
    """DRAM bytes per apply launch from the committed ncu summary, if it was taken
    on the current source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "apply_f32_traffic.json")
    try:
        with open(path) as fh:
            entries = json.load(fh)
        for d in entries if isinstance(entries, list) else [entries]:
            if (d.get("kernel", "apply_dense_kernel") == kernel and d.get("kernel_hash") == kernel_hash(kernel)
                    and d.get("workload") == workload):
                return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


def cpu_baseline(p, budget_s: float = 20.0, max_applies: int = 64):
    """FP64 oracle on a bounded sample: edge applies (messages) of half-step 1,
    timed on the host cores, as it stands."""
    from oracle import tree_ot as O
    colour = O.bipartition(p.num_nodes, p.edges)
    f = O.zero_potentials(p)
    nb = O.neighbours(p.num_nodes, p.edges)
    active = [(j, k) for j in range(p.num_nodes) if colour[j] == 0 for k in nb[j]]
    # build the sampled costs outside the timed loop (the oracle reads them as problem data)
    done = 0
    t_total = 0.0
    for (j, k) in active[:max_applies]:
        O.cost(p, j, k)  # materialise the FP32 matrix (input), not timed
        t0 = time.perf_counter()
        O.message(p, f, j, k)
        t_total += time.perf_counter() - t0
        done += 1
        if t_total >= budget_s:
            break
    return {"value": done / t_total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} of {p.num_edges} edge applies of half-step 1 (FP64 numpy log-sum-exp over 4096x4096), "
                      f"{t_total:.1f} s"}


def run_reference(args):
    """The oracle as it stands, on the host cores: each step is a bounded sample of
    one edge apply of the workload (REF_ROWS of its 4096 output rows, FP64 numpy
    log-sum-exp over all 4096 columns); the value is scaled to whole edge applies."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    REF_ROWS = 512
    p = workload_problem()
    steps, warm = args.steps, args.warmup
    from oracle import tree_ot as O
    colour = O.bipartition(p.num_nodes, p.edges)
    f = O.zero_potentials(p)
    nb = O.neighbours(p.num_nodes, p.edges)
    active = [(j, k) for j in range(p.num_nodes) if colour[j] == 0 for k in nb[j]]
    for j, k in active[:4]:
        O.cost(p, j, k)  # the stored FP32 matrices are problem data, built before timing
    def step(i):
        j, k = active[i % 4]
        r0 = (i * REF_ROWS) % int(p.n[j])
        O.message(p, f, j, k, rows=np.arange(r0, r0 + REF_ROWS))
    for i in range(warm):
        step(i)
    t0 = time.perf_counter()
    for i in range(steps):
        step(warm + i)
    dt = time.perf_counter() - t0
    frac = REF_ROWS / 4096.0
    value = steps * frac / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "step": f"{REF_ROWS} of 4096 rows of one edge apply (FP64 numpy oracle, host cores)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{steps} x {REF_ROWS} rows of half-step-1 edge applies, 4096 columns each"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# Per-SM unit rates of the GB300 SM used for the recomputed-cost roofline:
# 128 FP32 lanes (FFMA / FADD / FMUL, packed f32x2 included: a packed op is two
# lane operations) and 32 MUFU ex2 per clock, both measured with a throughput
# microbenchmark on this GPU (115 and 30 per clock per SM achieved).
FP32_LANES_PER_CLK = 128.0
EX2_PER_CLK = 32.0
def fp32_peak(sms: int, mhz: float) -> float:
    return FP32_LANES_PER_CLK * sms * mhz * 1e6


def sfu_peak(sms: int, mhz: float) -> float:
    return EX2_PER_CLK * sms * mhz * 1e6


# FP32-pipe lane operations per element the recomputed-cost apply needs by the
# survey's algorithmic count (2-D points): the squared distance (two differences,
# a square and an FMA), the argument (operand minus frame, scale), the sum --
# about 8 -- beside one ex2 on the MUFU.
RECOMP_ALG_OPS_PER_ELEM = 8.0


def batched_share(num_trees: int, rank: int, world: int):
    """This rank's trees of the batched workload (all of them at world = 1): disjoint
    subsets balanced by plan elements per half-step, no data-path exchange."""
    import gen
    from paper_2406_10849_gb300 import shard

    allp = gen.batched_problems(seed=4000, num_trees=num_trees)
    if world == 1:
        return allp, list(range(len(allp)))
    return shard.shard_problems(allp, rank, world)


def bench_batched(dev, stream, steps: int, warmup: int, converge: bool, num_trees: int = 512, rank: int = 0,
                  world: int = 1, dist=None):
    """Independent random trees (4..32 nodes, n_j in 128..2048, 2-D points, eps
    log-uniform in [0.002, 0.05], squared-Euclidean cost recomputed in the kernel)
    in one handle; this rank's share of the batch when world > 1.  One step = one
    half-step over the rank's trees.  Returns a dict (timed with CUDA events on the
    launching stream, per-kernel times from the library's launch timing)."""
    import torch

    import gen
    import paper_2406_10849_gb300 as T
    from paper_2406_10849_gb300 import shard

    probs, mine = batched_share(num_trees, rank, world)
    t0 = time.perf_counter()
    solver = T.Solver(probs, T.options(precision="fp32"), stream=stream)
    create_s = time.perf_counter() - t0
    stats = solver.plan_stats()
    elems = stats["elements_per_half_step"]
    n_apply = stats["edges"]
    for i in range(warmup):
        solver.apply(i % 2)
        solver.node_update(i % 2)
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    c0 = warmup % 2
    solver.profile(True)
    with ClockSampler(dev.index or 0) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        for i in range(steps):
            solver.apply((c0 + i) % 2)
            solver.node_update((c0 + i) % 2)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
    prof = solver.profile_read()
    solver.profile(False)
    clocks = clk.summary()
    t_ms = start.elapsed_time(stop)
    t_max = shard.max_over_ranks(t_ms, dist, dev)
    total_apply = shard.sum_over_ranks(n_apply, dist, dev)
    apply_ms = prof["apply_recompute"][0] / steps   # every launch of a half-step (one per dimension)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks["sm_mhz"] or 2070.0
    elem_rate = elems / (apply_ms / 1e3)
    peak = fp32_peak(sms, mhz)
    out = {
        "workload": f"batched{num_trees}_trees_2d_sqeuclid", "trees": len(probs), "edges": n_apply,
        "elements_per_step": elems, "create_s": create_s,
        "edge_applies_per_s": total_apply * steps / (t_max / 1e3), "ms_per_step": t_max / steps,
        "apply_ms": apply_ms, "node_update_ms": prof["node_update"][0] / steps,
        "elements_per_s": elem_rate,
        "roofline": {"bound": "alu", "kernel": "apply_recomp_kernel<2>",
                     "achieved": RECOMP_ALG_OPS_PER_ELEM * elem_rate / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
                     "frac": RECOMP_ALG_OPS_PER_ELEM * elem_rate / peak,
                     "ops_per_element": RECOMP_ALG_OPS_PER_ELEM,
                     "peak_kind": f"FP32 lanes: 128/clk/SM x {sms} SMs x {mhz:.0f} MHz (median SM clock under load)",
                     "sfu_frac": elem_rate / sfu_peak(sms, mhz), "traffic": None},
        "autotuned_tile": {"output_block": stats["recompute_output_block"],
                           "ctas_per_sm": stats["recompute_ctas_per_sm"],
                           "register_variant": stats["recompute_variant"]},
        "clocks": clocks, "gpu_launches": 2 * steps,
    }
    solver.close()
    # the persistent forest launch: chunks of half-steps as one launch each (the create-time
    # timing keeps it only where it beats the per-half-step launches)
    sp = T.Solver(probs, T.options(precision="fp32", persistent=True), stream=stream)
    form = sp.plan_stats()["persistent"]
    sp.half_steps(warmup)
    torch.cuda.synchronize(dev)
    sp.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    e0.record(stream)
    sp.half_steps(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    pprof = sp.profile_read()
    sp.close()
    p_ms = shard.max_over_ranks(e0.elapsed_time(e1), dist, dev) / steps
    out["persistent"] = {"form": form, "note": "0: per-half-step launches kept; 2 or 3: CTAs per SM of the "
                                               "persistent kernel", "ms_per_step": p_ms,
                         "edge_applies_per_s": total_apply / (p_ms / 1e3),
                         "kernel_ms_per_step": {k: v[0] / steps for k, v in pprof.items()},
                         "fp32_frac_whole_half_step": RECOMP_ALG_OPS_PER_ELEM * elems / (p_ms / 1e3) / peak}
    if converge and rank == 0 and world == 1:
        s2 = T.Solver(probs, T.options(precision="fp32", tol=1e-6, tol_kind="max", max_half_steps=20000),
                      stream=stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rc, res = s2.solve()
        dt_two = time.perf_counter() - t0
        s2.close()
        s2 = T.Solver(probs, T.options(precision="fp32", tol=1e-6, tol_kind="max", max_half_steps=20000,
                                       persistent=True), stream=stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rc, res = s2.solve()
        dt = time.perf_counter() - t0
        out["solve_per_half_step_launches_s"] = dt_two
        hs = [r["half_steps"] for r in res]
        s2.profile(True)
        t0 = time.perf_counter()
        rr = s2.round()
        dt_round = time.perf_counter() - t0
        pr = s2.profile_read()
        s2.close()
        out["solve_to_1e-6"] = {"seconds": dt, "form": form,
                                "certified": sum(1 for r in res if r["status"] == 0),
                                "trees": len(res), "half_steps_median": int(np.median(hs)),
                                "half_steps_max": int(max(hs)),
                                "worst_max_marginal_l1": max(r["max_marginal_l1"] for r in res)}
        out["rounding"] = {"seconds": dt_round, "kernel_ms": pr.get("round", (0.0, 0))[0],
                           "max_abs_cost_change": max(abs(r["rounded_transport_cost"] - r["transport_cost"])
                                                      for r in rr),
                           "worst_bound": max(r["bound"] for r in rr)}
    return out


def run_batched(args):
    """--workload batched: the batched trees as the JSON line's own workload.  Under
    torchrun the ranks split the 512 trees (disjoint subsets balanced by cost; no
    data-path collective) and value is the whole job's edge applies per second."""
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    b = bench_batched(dev, stream, args.steps, args.warmup, not args.no_converge, args.trees, rank, world, dist)
    if rank == 0:
        line = {
            "metric": METRIC, "value": b["edge_applies_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": b["workload"], "trees": args.trees, "edges_rank0": b["edges"],
                       "elements_per_step_rank0": b["elements_per_step"],
                       "step": "one half-step over every tree (apply + node update); ranks split the trees",
                       "l2": "no stored costs; per-step vectors exceed L2",
                       "autotuned_tile": b["autotuned_tile"]},
            "roofline": b["roofline"], "clocks": b["clocks"], "gpu_launches": b["gpu_launches"],
        }
        for k in ("persistent", "solve_to_1e-6", "solve_per_half_step_launches_s", "rounding"):
            if k in b:
                line[k] = b[k]
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def bench_stars(dev, stream, stars: int, side: int, steps: int, warmup: int, converge: bool,
                refine_tol: float = 1.5e-6, sk_product: str = "auto"):
    """The shared-kernel BF16 phase on a batch of barycenter stars (8 fixed leaves on
    a side x side grid, free centre, eps 0.005: every directed edge of every star
    shares one Gibbs kernel) against the FP32 recomputed-cost path: a half-step of
    each (CUDA events on the launching stream, per-kernel times from the library's
    launch timing) and, when converge, the batch to a certified max marginal
    L1 <= 1e-6 in each form."""
    import torch

    import gen
    import paper_2406_10849_gb300 as T

    probs = gen.warmstart_stars(9_000_000, stars, side=side, eps=0.005)
    n = side * side
    cols = 8 * stars  # directed edges applied per half-step
    forms = {"plain_fp32": {},
             "bf16_shared_kernel": dict(apply_mode="bf16", lowp_start=0, refine_tol=0.0, sk_product=sk_product)}
    res = {}
    clocks = None
    for name, kw in forms.items():
        s = T.Solver(probs, T.options(**kw), stream=stream)
        s.half_steps(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s.profile(True)
        with ClockSampler(dev.index or 0) as clk:
            e0.record(stream)
            s.half_steps(steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        prof = s.profile_read()
        s.profile(False)
        res[name] = {"ms_per_half_step": e0.elapsed_time(e1) / steps,
                     "kernel_ms_per_half_step": {k: v[0] / steps for k, v in prof.items()}}
        if name == "bf16_shared_kernel":
            clocks = clk.summary()
            sk_form = {0: "none", 1: "mma.sync", 2: "tcgen05, one CTA per 128-row tile",
                       3: "tcgen05, CTA pairs (256-row MMAs)"}[s.plan_stats()["sk_product"]]
        s.close()
    if converge:
        solve = {"plain_fp32": {}, "bf16_shared_kernel": dict(apply_mode="bf16", lowp_start=0,
                                                               refine_tol=refine_tol, sk_product=sk_product)}
        for name, kw in solve.items():
            s = T.Solver(probs, T.options(tol=1e-6, tol_kind="max", max_half_steps=20000, **kw), stream=stream)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rc, out = s.solve()
            dt = time.perf_counter() - t0
            s.close()
            hs = np.array([r["half_steps"] for r in out], dtype=np.float64)
            res[name]["time_to_1e-6_s"] = dt
            res[name]["half_steps_mean"] = float(hs.mean())
            res[name]["bf16_half_steps_mean"] = float(np.mean([r["lowp_half_steps"] for r in out]))
            res[name]["certified"] = int(sum(r["status"] == 0 for r in out))
            res[name]["worst_max_marginal_l1"] = max(r["max_marginal_l1"] for r in out)
    ph = res["bf16_shared_kernel"]
    prod_ms = ph["kernel_ms_per_half_step"].get("sk_product", float("nan"))
    flops3 = 3 * 2 * n * n * cols       # the three split products
    flops1 = 2 * n * n * cols           # the method's one product
    bf16_peak, kind = read_bf16_peak()
    out = {
        "workload": f"stars{stars}_grid{n}_eps0.005", "stars": stars, "n": n,
        "edge_applies_per_s": cols / (ph["ms_per_half_step"] / 1e3),
        "plain_fp32_edge_applies_per_s": cols / (res["plain_fp32"]["ms_per_half_step"] / 1e3),
        "speedup_per_half_step": res["plain_fp32"]["ms_per_half_step"] / ph["ms_per_half_step"],
        "product": {"kernel": "sk_gemm_tc_kernel", "form": sk_form,
                    "ms_per_launch": prod_ms,
                    "pflops_3_products": flops3 / (prod_ms / 1e3) / 1e15,
                    "pflops_method_1_product": flops1 / (prod_ms / 1e3) / 1e15,
                    "peak_pflops": bf16_peak / 1e3, "peak_kind": kind,
                    "frac_3_products": flops3 / (prod_ms / 1e3) / 1e12 / bf16_peak,
                    "frac_method": flops1 / (prod_ms / 1e3) / 1e12 / bf16_peak},
        "forms": res, "clocks": clocks,
    }
    if converge:
        out["speedup_time_to_1e-6"] = (res["plain_fp32"]["time_to_1e-6_s"]
                                       / res["bf16_shared_kernel"]["time_to_1e-6_s"])
    return out


FIG4_D = (10, 20, 40, 80, 160, 320, 640, 1280)      # d at |E| = 3
FIG4_E = (2, 3, 4, 6, 8, 12, 16, 24, 32)             # |E| at d = 10


def bench_fig4(dev, stream, seeds: int = 5, delta: float = 0.2):
    """The paper's experiment (Sec. 5, Fig. 4(a)) with this solver: half-steps of
    the Bipartite Iterative Scaling algorithm until the stopping sum falls below
    delta' = delta / (8 C_inf), with eps = delta / (4 |E| log d), on the
    log-normal barycenter -- against d at |E| = 3 and against |E| at d = 10, each
    point the mean over ``seeds`` seeds.  All instances run as one batch (each
    problem retires on its own); the rounding then certifies every instance
    delta-approximate by lemma lem:round_applied (bound <= delta)."""
    import torch

    import gen
    import paper_2406_10849_gb300 as T

    cases = [(3, d) for d in FIG4_D] + [(E, 10) for E in FIG4_E if E != 3]
    probs, keys = [], []
    for (E, d) in cases:
        for sd in range(seeds):
            probs.append(gen.lognormal_barycenter(6_000_000 + 1000 * E + 10 * d + sd, E, d, delta))
            keys.append((E, d))
    tol = probs[0].meta["tol"]
    s = T.Solver(probs, T.options(precision="fp32", tol=tol, tol_kind="sum", max_half_steps=200000), stream=stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rc, res = s.solve()
    dt = time.perf_counter() - t0
    rr = s.round()
    s.close()
    by = {}
    for k, r, q, pb in zip(keys, res, rr, probs):
        b = by.setdefault(k, {"half_steps": [], "bound": [], "theorem": 2 + 88 * k[0] * 1.0 / (tol * pb.eps)})
        b["half_steps"].append(r["half_steps"])
        b["bound"].append(q["bound"])
    def row(k):
        b = by[k]
        return {"E": k[0], "d": k[1], "eps": delta / (4 * k[0] * np.log(k[1])),
                "half_steps_mean": float(np.mean(b["half_steps"])), "half_steps": b["half_steps"],
                "thm_num_iter_bound": b["theorem"], "worst_round_bound": max(b["bound"])}
    vs_d = [row((3, d)) for d in FIG4_D]
    vs_E = [row((E, 10)) for E in FIG4_E]
    # trends: iterations against log d (least-squares line) and against |E| (log-log slope)
    ld = np.log(np.array(FIG4_D, dtype=np.float64))
    yd = np.array([r["half_steps_mean"] for r in vs_d])
    slope_d, icpt_d = np.polyfit(ld, yd, 1)
    r2_d = 1.0 - float(np.sum((yd - (slope_d * ld + icpt_d)) ** 2) / np.sum((yd - yd.mean()) ** 2))
    lE = np.log(np.array(FIG4_E, dtype=np.float64))
    yE = np.log(np.array([r["half_steps_mean"] for r in vs_E]))
    exp_E, _ = np.polyfit(lE, yE, 1)
    return {"workload": f"fig4_lognormal_barycenter_delta{delta}", "delta": delta, "tol": tol, "seeds": seeds,
            "instances": len(probs), "seconds": dt, "certified": int(sum(r["status"] == 0 for r in res)),
            "all_delta_approximate": bool(max(q["bound"] for q in rr) <= delta),
            "vs_d_at_E3": vs_d, "vs_E_at_d10": vs_E,
            "trend": {"half_steps_per_log_d": float(slope_d), "r2_vs_log_d": r2_d,
                      "loglog_exponent_vs_E": float(exp_E)}}


FIG4_WLS_D = (5, 10, 20, 40, 80)       # d at |E| = 12 cliques
FIG4_WLS_E = (2, 3, 4, 6, 8, 12, 16)   # cliques at d = 10


def bench_fig4_wls(dev, stream, seeds: int = 5, delta: float = 0.2, alpha: float = 10.0):
    """The Wasserstein least-squares half of the paper's experiment (Sec. 5, Fig. 4(b)):
    each instance's modified junction tree reduced to its tree of separators
    (x_0 x x_{J+1} centre of d^2 points, J constrained leaves) and solved by the same
    kernels, eps = delta / (4 J log d), stopping sum below delta / (8 C_inf); mean
    half-steps against d at J = 12 and against J at d = 10, all instances in one batch."""
    import torch

    import gen
    import paper_2406_10849_gb300 as T
    from paper_2406_10849_gb300 import junction as JR

    cases = [(12, d) for d in FIG4_WLS_D] + [(J, 10) for J in FIG4_WLS_E if J != 12]
    by_tol = {}
    for (J, d) in cases:
        for sd in range(seeds):
            jt = gen.wls_junction_tree(6_500_000 + 1000 * J + 10 * d + sd, J, d, alpha, delta)
            by_tol.setdefault(round(jt.meta["tol"], 12), []).append(((J, d), JR.reduce_junction_tree(jt)))
    rows = {}
    dt = 0.0
    for tol, items in by_tol.items():   # one handle per stopping threshold (C_inf depends on J)
        probs = [t for _, t in items]
        s = T.Solver(probs, T.options(precision="fp32", tol=tol, tol_kind="sum", max_half_steps=400000),
                     stream=stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rc, res = s.solve()
        dt += time.perf_counter() - t0
        s.close()
        for (k, _), r in zip(items, res):
            rows.setdefault(k, []).append((r["half_steps"], r["status"]))
    def row(k):
        hs = [h for h, _ in rows[k]]
        return {"J": k[0], "d": k[1], "half_steps_mean": float(np.mean(hs)), "half_steps": hs,
                "certified": int(sum(1 for _, st in rows[k] if st == 0))}
    vs_d = [row((12, d)) for d in FIG4_WLS_D]
    vs_E = [row((J, 10)) for J in FIG4_WLS_E]
    ld = np.log(np.array(FIG4_WLS_D, dtype=np.float64))
    yd = np.array([r["half_steps_mean"] for r in vs_d])
    slope_d, icpt_d = np.polyfit(ld, yd, 1)
    r2_d = 1.0 - float(np.sum((yd - (slope_d * ld + icpt_d)) ** 2) / np.sum((yd - yd.mean()) ** 2))
    exp_E = float(np.polyfit(np.log(np.array(FIG4_WLS_E, dtype=np.float64)),
                             np.log(np.array([r["half_steps_mean"] for r in vs_E])), 1)[0])
    return {"workload": f"fig4_wls_alpha{alpha}_delta{delta}", "instances": sum(len(v) for v in rows.values()),
            "seconds": dt, "vs_d_at_E12": vs_d, "vs_E_at_d10": vs_E,
            "trend": {"half_steps_per_log_d": float(slope_d), "r2_vs_log_d": r2_d, "loglog_exponent_vs_E": exp_E}}


def bench_jt_general(dev, stream, steps: int = 40):
    """General modified junction trees (Sec. 4) on the GPU's general path
    (tree_ot_jt_*): the nested example of ass:inclusion at d = 8 (cliques of up to
    8^4 entries) and the WLS junction tree (J = 12, d = 20, alpha = 10) through the
    general separator update, against WLS reduced to its tree of separators and
    solved by the tree kernels: us per half-step (CUDA events) and the solve to
    the stopping threshold."""
    import torch

    import gen
    import paper_2406_10849_gb300 as T
    from paper_2406_10849_gb300 import junction as JR
    from paper_2406_10849_gb300.treeot import JunctionSolver

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    out = {}
    cases = {"nested_d8": (gen.nested_junction_tree(6_700_000, d=8, eps=0.1), 1e-8),
             "wls_J12_d20": (gen.wls_junction_tree(6_700_001, 12, 20), None)}
    for name, (jt, tol) in cases.items():
        tol = jt.meta["tol"] if tol is None else tol
        with JunctionSolver(jt, stream) as s:
            s.half_steps(2)
            ms = timed(lambda: s.half_steps(steps))
            s.reset()
            t0 = time.perf_counter()
            rc, hs, r = s.solve(tol=tol, tol_kind="sum", max_half_steps=200000, check_every=16)
            dt = time.perf_counter() - t0
            out[name] = {"general_path_us_per_half_step": 1e3 * ms / steps, "solve_s": dt, "half_steps": hs,
                         "stopping_sum": r, "status": rc, "transport_cost": s.transport_cost()}
        if name.startswith("wls"):
            tr = JR.reduce_junction_tree(jt)
            with T.Solver([tr], T.options(precision="fp32", tol=tol, tol_kind="sum", max_half_steps=200000),
                          stream=stream) as s:
                s.half_steps(2)
                ms = timed(lambda: s.half_steps(steps))
                s.reset()
                t0 = time.perf_counter()
                rc, res = s.solve()
                dt = time.perf_counter() - t0
                out[name].update({"reduced_tree_us_per_half_step": 1e3 * ms / steps, "reduced_solve_s": dt,
                                  "reduced_half_steps": res[0]["half_steps"],
                                  "reduced_transport_cost": res[0]["transport_cost"]})
    return out


def bench_chain(dev, stream, steps: int):
    """The 5-node chain (n = 64 grid, eps = 0.01, FP64 handle): microseconds per
    half-step (CUDA events) and the solve to a stopping sum below 1e-9."""
    import torch

    import gen
    import paper_2406_10849_gb300 as T

    p = gen.chain_problem(seed=1000)
    s = T.Solver([p], T.options(precision="fp64"), stream=stream)
    s.half_steps(10)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    s.half_steps(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    us = 1e3 * e0.elapsed_time(e1) / steps
    s.close()
    s = T.Solver([p], T.options(precision="fp64", tol=1e-9, tol_kind="sum", check_every=2), stream=stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rc, res = s.solve()
    dt = time.perf_counter() - t0
    rr = s.round()[0]
    s.close()
    return {"workload": "chain5_n64_fp64_eps0.01", "us_per_half_step": us,
            "edge_applies_per_s": p.num_edges / (us / 1e6),
            "solve_to_1e-9": {"seconds": dt, "half_steps": res[0]["half_steps"], "status": rc,
                              "residual_sum_l1": res[0]["residual_sum_l1"]},
            "rounded_transport_cost": rr["rounded_transport_cost"], "transport_cost": rr["transport_cost"]}


def bench_star(dev, stream, steps: int):
    """One barycenter star (8 fixed leaves on a 32 x 32 grid, free centre, eps
    0.005, squared-Euclidean cost recomputed in the kernel, FP32): microseconds
    per half-step and the solve to a certified max marginal L1 <= 1e-6."""
    import torch

    import gen
    import paper_2406_10849_gb300 as T

    p = gen.star_problem(seed=2000)
    s = T.Solver([p], T.options(precision="fp32"), stream=stream)
    s.half_steps(10)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    s.profile(True)
    e0.record(stream)
    s.half_steps(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    prof = s.profile_read()
    us = 1e3 * e0.elapsed_time(e1) / steps
    s.close()
    s = T.Solver([p], T.options(precision="fp32", tol=1e-6, tol_kind="max"), stream=stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rc, res = s.solve()
    dt = time.perf_counter() - t0
    s.close()
    return {"workload": "star8_grid1024_sqeuclid_fp32_eps0.005", "us_per_half_step": us,
            "edge_applies_per_s": p.num_edges / (us / 1e6),
            "kernel_us_per_half_step": {k: 1e3 * v[0] / steps for k, v in prof.items()},
            "solve_to_1e-6": {"seconds": dt, "half_steps": res[0]["half_steps"], "status": rc,
                              "max_marginal_l1": res[0]["max_marginal_l1"]}}


def run_warmstart(args):
    """Learned warm start and the shared-kernel BF16 phase on barycenter stars
    (8 fixed leaves on a side x side grid, free centre, eps log-uniform in
    [0.0025, 0.01] for training): solve the training stars from u = 1 on the
    GPU, train the MLP on their leaf potentials with the library's own kernels,
    then solve the held-out stars (eps = 0.005, one shared Gibbs kernel) to max
    marginal L1 <= 1e-6 in one batched handle, four ways: plain FP32 from u = 1,
    FP32 from the predicted potentials, and both again with the BF16 phase.
    The JSON line's value is the BF16 + warm-start time (prediction included);
    the plain FP32 time and the other two forms stand beside it."""
    import torch

    import gen
    from paper_2406_10849_gb300 import warmstart as W

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    side, B = args.side, 512
    t0 = time.perf_counter()
    X, Y, hs_train = [], [], []
    for b in range(0, args.train_trees, B):
        probs = gen.warmstart_stars(5_000_000 + b, min(B, args.train_trees - b), side=side)
        res, s, _ = W.zero_solve(probs)
        X.append(torch.from_numpy(W.inputs(probs)).to(dev))
        Y.append(W.targets(s, probs).clone())
        s.close()
        hs_train += [r["half_steps"] for r in res]
    X, Y = torch.cat(X), torch.cat(Y)
    t_data = time.perf_counter() - t0
    ws = W.WarmStart(side * side, 512, 256, seed=0)
    t1 = time.perf_counter()
    hist = ws.train(X, Y, epochs=args.epochs, batch=256, lr=1e-3)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t1
    test = gen.warmstart_stars(9_000_000, args.test_trees, side=side, eps=0.005)
    # first-use costs (autotuner cache, function attributes) outside the timed solves
    W.zero_solve(test[:16])[1].close()
    W.zero_solve(test[:16], apply_mode="bf16", lowp_start=0, refine_tol=args.refine_tol)[1].close()
    tzd, twd, tzbd, twbd = {}, {}, {}, {}
    with ClockSampler(0) as clk:
        torch.cuda.synchronize(dev)
        rz, s, tz = W.zero_solve(test, timing=tzd)
        s.close()
        rw, fallbacks, tw = ws.warm_solve(test, timing=twd)
        # the same, with the shared-kernel BF16 phase from the first half-step
        bf = dict(apply_mode="bf16", lowp_start=0, refine_tol=args.refine_tol)
        rzb, s, _ = W.zero_solve(test, timing=tzbd, **bf)
        s.close()
        rwb, fallbacks_b, _ = ws.warm_solve(test, timing=twbd, **bf)
    clocks = clk.summary()
    # the handle's creation (upload, planning) is the same for both starts: compare the rest
    tz_run = tzd["solve"]
    tw_run = twd["predict"] + twd["solve"] + twd["fallback"]
    tzb_run = tzbd["solve"]
    twb_run = twbd["predict"] + twbd["solve"] + twbd["fallback"]
    hz = np.array([r["half_steps"] for r in rz], dtype=np.float64)
    hw = np.array([r["half_steps"] for r in rw], dtype=np.float64)

    def summary(res, seconds):
        hs = np.array([r["half_steps"] for r in res], dtype=np.float64)
        lp = np.array([r["lowp_half_steps"] for r in res], dtype=np.float64)
        return {"seconds": seconds, "half_steps_mean": float(hs.mean()), "bf16_half_steps_mean": float(lp.mean()),
                "converged": int(sum(r["status"] == 0 for r in res)),
                "worst_max_marginal_l1": max(r["max_marginal_l1"] for r in res)}

    line = {
        "metric": "time to max marginal L1 <= 1e-6: BF16 shared-kernel phase + warm start vs plain FP32 from u = 1",
        "value": twb_run, "unit": "s",
        "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": twb_run * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 tensor-core phase + f32 solve, bf16 MLP",
        "data": "synthetic",
        "plain_fp32_seconds": tz_run, "speedup_vs_plain": tz_run / twb_run,
        "forms": {"plain_fp32_zero": summary(rz, tz_run), "fp32_warm": summary(rw, tw_run),
                  "bf16_zero": summary(rzb, tzb_run), "bf16_warm": summary(rwb, twb_run),
                  "bf16_warm_fallbacks": fallbacks_b},
        "config": {"workload": f"warmstart_star{side * side}_train{args.train_trees}_test{args.test_trees}",
                   "leaves": 8, "n": side * side, "train_eps": [0.0025, 0.01], "test_eps": 0.005,
                   "mlp": f"{side * side + 1}-512-512-{side * side} GELU, bf16 weights, fp32 master + Adam",
                   "epochs": args.epochs},
        "warm_fp32_seconds": tw_run, "zero_init_seconds": tz_run, "speedup_warm_fp32": tz_run / tw_run,
        "seconds_split": {"warm": twd, "zero": tzd, "bf16_warm": twbd, "bf16_zero": tzbd,
                          "note": "warm forms: predict (inputs, network, set) + solve + fallback; zero forms: "
                                  "solve; handle creation excluded from all"},
        "half_steps": {"zero_mean": float(hz.mean()), "warm_mean": float(hw.mean()),
                       "zero_median": float(np.median(hz)), "warm_median": float(np.median(hw)),
                       "zero_max": int(hz.max()), "warm_max": int(hw.max()),
                       "paired_frac_warm_fewer": float(np.mean(hw < hz))},
        "fallbacks": fallbacks,
        "worst_max_marginal_l1": {"warm": max(r["max_marginal_l1"] for r in rw),
                                  "zero": max(r["max_marginal_l1"] for r in rz)},
        "training": {"data_seconds": t_data, "train_seconds": t_train, "samples": int(X.shape[0]),
                     "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                     "target_variance": float(Y.var().item()),
                     "train_half_steps_mean": float(np.mean(hs_train))},
        "clocks": clocks,
    }
    ws.close()
    print(json.dumps(line), flush=True)


def run_stars(args):
    """--workload stars: the shared-kernel BF16 phase on a batch of stars as the JSON
    line's own workload (see bench_stars)."""
    import torch

    import paper_2406_10849_gb300 as T

    T.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    b = bench_stars(dev, stream, args.stars, args.side, args.steps, args.warmup, not args.no_converge,
                    args.refine_tol, args.sk_product)
    ms = b["forms"]["bf16_shared_kernel"]["ms_per_half_step"]
    line = {
        "metric": "edge-kernel applies/sec, shared-kernel BF16 phase (stars on one grid)",
        "value": b["edge_applies_per_s"], "unit": "edge_applies/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3 tensor-core product, f32 node update", "data": "synthetic",
        "config": {"workload": b["workload"], "stars": args.stars, "leaves": 8, "n": b["n"],
                   "step": "one half-step over all stars", "refine_tol": args.refine_tol},
    }
    line.update({k: v for k, v in b.items() if k not in ("workload", "stars", "n")})
    print(json.dumps(line), flush=True)


def run_fig4(args):
    """--workload fig4: the iteration-count experiment as the JSON line's own workload."""
    import torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    b = bench_fig4(dev, stream)
    b["wls"] = bench_fig4_wls(dev, stream)
    line = {"metric": "half-steps to the stopping threshold delta' (mean over seeds)", "value": b["seconds"],
            "unit": "s for all instances", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * b["seconds"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": b["workload"], "instances": b["instances"]}}
    line.update({k: v for k, v in b.items() if k not in ("workload",)})
    print(json.dumps(line), flush=True)


def run_unit_rates():
    """Build and run the unit-rate microbenchmark (csrc/unit_rates.cu): FP32 FMA
    lanes, packed f32x2 lanes and MUFU ex2 per clock and SM, ex2.approx error."""
    src = os.path.join(ROOT, "paper_2406_10849_gb300", "csrc", "unit_rates.cu")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "unit_rates")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    print(out.strip(), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-converge", action="store_true", help="skip the time-to-1e-6 solve")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only: skip the batched, stars, star and chain measurements")
    ap.add_argument("--nodes", type=int, default=NODES, help="tree size (64 = the benchmark workload)")
    ap.add_argument("--workload", default="prufer", choices=["prufer", "batched", "warmstart", "stars", "fig4"],
                    help="prufer: the 64-node stored-cost tree (default); batched: independent random trees "
                         "with costs recomputed from 2-D points (measured against the MUFU ex2 roofline); "
                         "warmstart: learned warm start on barycenter stars, warm vs u = 1; "
                         "stars: the shared-kernel BF16 phase on a batch of stars; "
                         "fig4: the paper's iteration-count experiment on log-normal barycenters")
    ap.add_argument("--stars", type=int, default=2000, help="stars workload: number of stars")
    ap.add_argument("--train-trees", type=int, default=20000, help="warmstart: training stars")
    ap.add_argument("--test-trees", type=int, default=2000, help="warmstart: held-out stars")
    ap.add_argument("--side", type=int, default=32, help="warmstart: grid side (n = side^2)")
    ap.add_argument("--epochs", type=int, default=30, help="warmstart: training epochs")
    ap.add_argument("--refine-tol", type=float, default=1.5e-6,
                    help="warmstart: stopping quantity at which the BF16 forms hand over to FP32")
    ap.add_argument("--unit-rates", action="store_true",
                    help="only build and run the FP32 / MUFU unit-rate microbenchmark")
    ap.add_argument("--trees", type=int, default=512, help="batched workload: number of trees")
    ap.add_argument("--sk-product", default="auto", choices=["auto", "one_cta", "mma"],
                    help="stars workload: the shared-kernel product (auto: tcgen05 over CTA pairs)")
    ap.add_argument("--dense-kernel", default="auto", choices=["auto", "tma", "ldg"],
                    help="stored-cost apply kernel (auto: the solver's autotuner picks)")
    args = ap.parse_args()
    if args.unit_rates:
        return run_unit_rates()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "stars":
        return run_stars(args)
    if args.workload == "fig4":
        return run_fig4(args)

    import torch

    import gen
    import paper_2406_10849_gb300 as T

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    p = workload_problem(args.nodes)
    workload = workload_name(args.nodes)
    costs = [gen.sqeuclid_cost_f32_torch(p.coords[a], p.coords[b], 1.0, dev) for a, b in p.edges]
    torch.cuda.synchronize(dev)
    solver = T.Solver([p], T.options(precision="fp32", dense_kernel=args.dense_kernel), stream=stream,
                      device_costs=[costs])
    stats = solver.plan_stats()
    kernel = "apply_dense_tma_kernel" if stats["dense_tma"] else "apply_dense_kernel"
    n_apply = p.num_edges

    # warm-up
    for i in range(args.warmup):
        c = i % 2
        solver.apply(c)
        solver.node_update(c)
    torch.cuda.synchronize(dev)

    K = args.steps
    ev_a0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_a1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    c0 = args.warmup % 2
    with ClockSampler(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        for i in range(K):
            c = (c0 + i) % 2
            ev_a0[i].record(stream)
            solver.apply(c)
            ev_a1[i].record(stream)
            solver.node_update(c)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
    clocks = clk.summary()
    elapsed_ms = start.elapsed_time(stop)
    apply_ms = [ev_a0[i].elapsed_time(ev_a1[i]) for i in range(K)]
    t_max = elapsed_ms
    if dist is not None:
        t = torch.tensor([elapsed_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = world * n_apply * K / (t_max / 1e3)

    apply_avg_ms = statistics.mean(apply_ms)
    alg = algorithmic_bytes(p)
    peak, peak_kind = read_peaks()
    achieved = alg / (apply_avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(workload, kernel), "peak_kind": f"hbm_gbs of {peak_kind}",
                "kernel": kernel, "apply_ms_avg": apply_avg_ms,
                "apply_ms_median": statistics.median(apply_ms), "algorithmic_bytes_per_launch": alg}

    extra = {}
    if rank == 0 and not args.no_converge:
        # plain FP32 sweep from u = 1 to max marginal L1 <= 1e-6 (the solver's own check)
        s2 = T.Solver([p], T.options(precision="fp32", tol=1e-6, tol_kind="max", max_half_steps=20000),
                      stream=stream, device_costs=[costs])
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rc, res = s2.solve()
        dt = time.perf_counter() - t0
        s2.close()
        ttt = {"plain_fp32_s": dt, "plain_half_steps": res[0]["half_steps"],
               "plain_max_marginal_l1": res[0]["max_marginal_l1"], "plain_status": rc}
        # absorbed BF16 phase, then FP32 refinement, same tolerance and check
        s3 = T.Solver([p], T.options(precision="fp32", tol=1e-6, tol_kind="max", max_half_steps=20000,
                                     apply_mode="bf16"), stream=stream, device_costs=[costs])
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rc3, res3 = s3.solve()
        dt3 = time.perf_counter() - t0
        # rounding of the certified iterate to feasible plans (the step after the sweep)
        s3.profile(True)
        t0 = time.perf_counter()
        rr = s3.round()[0]
        dt_round = time.perf_counter() - t0
        pr = s3.profile_read()
        s3.close()
        ttt.update({"bf16_refined_s": dt3, "bf16_half_steps": res3[0]["half_steps"],
                    "bf16_lowp_half_steps": res3[0]["lowp_half_steps"], "bf16_absorptions": res3[0]["absorptions"],
                    "bf16_max_marginal_l1": res3[0]["max_marginal_l1"], "bf16_status": rc3,
                    "speedup": dt / dt3 if dt3 > 0 else None,
                    "note": "wall time of tree_ot_solve from u = 1 to max marginal L1 < 1e-6 (GPU check), "
                            "setup excluded"})
        extra["time_to_1e-6"] = ttt
        extra["rounding"] = {"seconds": dt_round, "kernel_ms": pr.get("round", (0.0, 0))[0],
                             "transport_cost": rr["transport_cost"],
                             "rounded_transport_cost": rr["rounded_transport_cost"],
                             "residual_sum_l1": rr["residual_sum_l1"], "bound_lem_round_applied": rr["bound"],
                             "c_inf": rr["c_inf"]}
    solver.close()

    e2e = None
    if not args.no_e2e:
        # the same metric through the public API with host inputs: create (host->device copy
        # of costs, coordinates and marginals), the K half-steps, the FP64 check (device->host)
        host_costs = [torch.empty(c.shape, dtype=torch.float32, pin_memory=True) for c in costs]
        for hc, c in zip(host_costs, costs):
            hc.copy_(c)
        del costs
        torch.cuda.empty_cache()
        hp = workload_problem(args.nodes)
        hp.dense_costs = [hc.numpy() for hc in host_costs]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s3 = T.Solver([hp], T.options(precision="fp32"), stream=stream)
        s3.half_steps(K)
        s3.check()
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        s3.close()
        t_e2e = dt
        if dist is not None:
            t = torch.tensor([dt], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        h2d = sum(int(hc.numel()) * 4 for hc in host_costs) + sum(int(c.size) * 4 for c in hp.coords) + \
            sum(int(m.size) * 8 for m in hp.marginals.values())
        d2h = 16 * int(sum(int(hp.n[a]) + int(hp.n[c]) for a, c in hp.edges))  # marginals + potentials
        e2e = {"value": world * n_apply * K / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d // K,
               "d2h_bytes_per_step": d2h // K,
               "note": f"one public-API solve of {K} half-steps from pinned host buffers per run"}
        host_costs = None
        hp = None

    costs = None
    torch.cuda.empty_cache()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # the other workloads, each with its own numbers (N = 1 only)
    if world == 1 and not args.no_extra:
        ks = max(10, min(K, 100))
        extra["batched"] = bench_batched(dev, stream, ks, args.warmup, not args.no_converge)
        extra["stars"] = bench_stars(dev, stream, args.stars, args.side, ks, args.warmup, not args.no_converge,
                                     args.refine_tol)
        extra["star"] = bench_star(dev, stream, max(ks, 50))
        extra["chain_fp64"] = bench_chain(dev, stream, max(ks, 200))
        extra["fig4"] = bench_fig4(dev, stream)
        extra["fig4_wls"] = bench_fig4_wls(dev, stream)
        extra["jt_general"] = bench_jt_general(dev, stream)
    cpu = None if (args.no_cpu or world > 1) else cpu_baseline(p)  # the host baseline: N = 1 only
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "nodes": p.num_nodes, "edges": p.num_edges, "n": 4096, "dim": 3,
                   "eps": 0.01, "cost": f"stored dense FP32, {stats['matrix_bytes_per_half_step'] / 1e9:.2f} GB", "step": "one half-step (apply + node update)",
                   "l2": f"inputs ({stats['matrix_bytes_per_half_step'] / 1e9:.2f} GB of costs) "
                         f"{'exceed' if stats['matrix_bytes_per_half_step'] > 129e6 else 'fit in'} L2 (129 MB)",
                   "elements_per_step": stats["elements_per_half_step"]},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": 2 * K,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

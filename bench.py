"""Benchmark: CADDeLaG graph pairs per second on the n = 32768 field pair.

One step = one whole graph pair through the C ABI (cdl_caddelag_pair):
graph build, bf16 inverse chain (d = 14, tcgen05 GEMMs), projection (k = 128),
chain-preconditioned solve refined to relative residual 1e-10 and CAD scores
with the top-10 anomalies, for both graphs of the pair.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 it runs under torch.distributed (one process per GPU); the
path does not shard, so every rank runs independent replicas and `value` is
the pairs of all ranks divided by the slowest rank's time. --impl reference
times the float64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "graph pairs/s at n=32768"
WORKLOAD = "field_n32768_pair"
N_GRID = (128, 256)
T_LEN = 256
K_PROJ = 128
D_CHAIN = 14
TOPK = 10
SEED = 2024
REL_TOL = 1e-10


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def square_traffic():
    """DRAM bytes per launch of the bf16 squaring from the committed ncu summary,
    if the kernel source is unchanged since it was captured (else None)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "k_tc_sq2_square_n32768_traffic.md")
    src = os.path.join(ROOT, "paper_1802_05421_gb300", "csrc", "tc_gemm.cu")
    try:
        text = open(path).read()
        tb = int(re.search(r"traffic_bytes_per_launch:\s*(\d+)", text).group(1))
        sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text).group(1)
        cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, AttributeError, ValueError):
        return None
    return tb if sha == cur else None


def make_workload():
    from workloads import field_sequence
    wl = field_sequence(N_GRID[0], N_GRID[1], T_LEN, 2, patch=8, patch_transition=0, seed=2)
    return wl


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- phase rooflines
def phase_rooflines(kc, n, pk, src, sm_count, sm_mhz):
    """Every phase of one pair against the roofline that binds it, from the
    library's per-class CUDA-event times (kc: class -> ms_per_step, work per
    launch, launches per step). Algorithmic work per pair:
      distance    8 n^2 bytes written per graph (float64 squared distances,
                  both triangles)                                     -> HBM
      select      bytes the radix-select passes read (library count) -> HBM
      kernel      bytes the kernel-value pass moves (library count)  -> HBM
      chain_init  bytes level-0 formation moves (library count)      -> HBM
      square      n^2 (n + 1) flops per squaring (library count)     -> bf16 tensor
      project     n (n - 1) k signed adds per graph (library count)  -> one float32
                  add per term on every lane: SMs x 128 x clock
      apply       bytes of chain levels (and A operands) read        -> HBM
      residual    bf16 slice-product flops of the exact residual     -> bf16 tensor
      score       8 n (n - 1) bytes: the upper halves of float64 A1, A2 -> HBM
      score_tensor  the same phase against the bf16 flops of its 21 exact
                  slice products over the upper triangle (library count) -> bf16
                  tensor: the bound of the exact design (it exceeds the HBM
                  time at every n)
    A phase's time includes its small helper kernels."""
    hbm = pk.get("hbm_gbs")
    bf16 = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    alu = sm_count * 128 * sm_mhz * 1e6 / 1e12     # T adds/s
    spec = {
        "distance": ("hbm", 2 * 8.0 * n * n),
        "select": ("hbm", None),
        "kernel": ("hbm", None),
        "chain_init": ("hbm", None),
        "square": ("tensor", None),
        "project": ("alu", None),
        "apply": ("hbm", None),
        "residual": ("tensor", None),
        "score": ("hbm", 8.0 * n * (n - 1)),
        "score_tensor": ("tensor", None),
    }
    out = {}
    for name, (bound, work) in spec.items():
        v = kc.get("score" if name == "score_tensor" else name)
        if not v or not v["ms_per_step"]:
            continue
        if work is None:
            work = v["work"] * v["launches"]
        sec = v["ms_per_step"] * 1e-3
        if bound == "hbm":
            ach, peak, unit, ps = work / sec / 1e9, hbm, "GB/s", f"{src} hbm_gbs"
        elif bound == "tensor":
            ach, peak, unit, ps = work / sec / 1e12, bf16, "TFLOP/s", f"{src} bf16_tflops_sustained"
        else:
            ach, peak, unit = work / sec / 1e12, alu, "T adds/s"
            ps = f"{sm_count} SMs x 128 float32 lanes x {sm_mhz:.0f} MHz"
        out[name] = {"bound": bound, "ms_per_pair": round(v["ms_per_step"], 3), "work_per_pair": work,
                     "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak if peak else None,
                     "peak_source": ps}
    return out


def oracle_full_pair_n1024():
    """The float64 oracle on the whole of the small pair (n = 1024, T = 64,
    k = 32, top-10; exact embeddings), timed in full: a CPU baseline that is
    measured, not extrapolated."""
    from oracle import caddelag as O
    from workloads import iid_pair
    wl = iid_pair(1024, 64, 10, seed=0)
    t0 = time.perf_counter()
    out = O.caddelag_pair(wl.X[0], wl.X[1], 32, 0, 10)
    sec = time.perf_counter() - t0
    return sec, [int(i) for i in out["top"]], wl


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(wl, budget_rows: int = 24, chol_n: int = 4096):
    """Time the float64 oracle on a bounded sample of one pair and scale each
    phase to the full pair: row-sampled distances, kernel, projection and
    scores (cost proportional to rows), the median on a 1/256 subsample
    (linear), the exact solve as a dense Cholesky at chol_n scaled by
    (n / chol_n)^3. Returns (seconds per pair, description)."""
    from oracle import caddelag as O
    X1, X2 = wl.X
    n = X1.shape[0]
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(n, size=budget_rows, replace=False))
    t = {}
    # distances + kernel rows, both graphs
    t0 = time.perf_counter()
    d2 = [O.squared_distances(X, rows) for X in (X1, X2)]
    t["distances"] = (time.perf_counter() - t0) * n / budget_rows / 2   # upper triangle only needed
    sample = d2[0].ravel()
    reps = max(1, (n * (n - 1) // 2) // sample.size // 64)
    t0 = time.perf_counter()
    np.partition(np.sqrt(sample), sample.size // 2)
    t["median"] = (time.perf_counter() - t0) * reps * 64 * 2
    sig = 30.0
    t0 = time.perf_counter()
    Ar = [np.exp(-(d / (2.0 * sig * sig))) for d in d2]
    t["kernel"] = (time.perf_counter() - t0) * n / budget_rows
    t0 = time.perf_counter()
    for a in Ar:
        O.project_rows(a, rows, SEED, K_PROJ)
    t["projection"] = (time.perf_counter() - t0) * n / budget_rows
    # exact solve: dense Cholesky at chol_n, cubic scaling, two graphs
    sub = X1[:chol_n]
    Asub, *_ = O.gaussian_graph(sub, d2=O.squared_distances_exact_grid(sub))
    Ysub = O.project_rows(Asub[:1], [0], SEED, 4)   # warm the path (tiny)
    Y = np.random.default_rng(1).standard_normal((chol_n, K_PROJ))
    Y -= Y.mean(0)
    t0 = time.perf_counter()
    O.exact_embedding(Asub, Y)
    t["solve"] = (time.perf_counter() - t0) * (n / chol_n) ** 3 * 2
    # scores on the sampled rows
    Z = np.random.default_rng(2).standard_normal((n, K_PROJ)) * 1e-3
    t0 = time.perf_counter()
    O.node_scores(Ar[0], Ar[1], Z, Z * 1.01, 1.0, 1.0, rows=rows)
    t["scores"] = (time.perf_counter() - t0) * n / budget_rows
    total = sum(t.values())
    desc = (f"oracle phases timed on {budget_rows} sampled rows of both graphs (distances, kernel, "
            f"projection, scores; scaled by n/rows), median on a row sample (linear), exact "
            f"Cholesky solve at n={chol_n} scaled by (n/{chol_n})^3; sum = one pair")
    del Ysub
    return total, desc, t


def cpu_cores():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        blas = [i for i in info if i.get("user_api") == "blas"]
        if blas:
            return int(blas[0].get("num_threads", os.cpu_count()))
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = make_workload()
    walls, est = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t, desc, _ = oracle_sample(wl, budget_rows=8, chol_n=2048)
        wall = time.perf_counter() - t0
        if s >= args.warmup:
            walls.append(wall)
            est.append(t)
    sec = statistics.median(est)        # extrapolated seconds for one whole pair
    value = 1.0 / sec
    c1_sec, _, _ = oracle_full_pair_n1024()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(walls) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_GRID[0] * N_GRID[1], "T": T_LEN, "k": K_PROJ,
                       "d": D_CHAIN, "solver": "oracle exact (dense Cholesky)"},
            "step_definition": "one bounded sample of the pair (8 rows of both graphs, Cholesky at n = 2048); "
                               "ms_per_step is its wall time",
            "value_basis": "extrapolated: each sampled phase scaled to the whole pair (rows by n / 8, "
                           "the Cholesky by (n / 2048)^3)",
            "extrapolated_ms_per_pair": sec * 1e3,
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": desc,
                             "measured_full_pair_n1024": {"workload": "iid_n1024 (n = 1024, T = 64, k = 32, "
                                                                      "top-10, exact embeddings)",
                                                          "seconds": c1_sec, "pairs_per_s": 1.0 / c1_sec}},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- ranks
def rank_max(values, dist, device):
    """Element-wise maximum of a list of floats over all ranks (identity
    without a process group)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def pairs_per_second(step_ms_max: float, world: int) -> float:
    """Whole-job rate: every rank processes one pair per step, the job is as
    fast as its slowest rank."""
    return world * 1000.0 / step_ms_max


# ---------------------------------------------------------------- profiling cases
def run_case(args):
    """Small single-kernel cases for profiler captures (not a bench line):
    graph build, then per case: square (one bf16 chain squaring), solve
    (bf16 chain d=4 + refinement), project, score; batched: --n ragged pairs
    (n log-uniform in [256, 4096]) through one eager batched call per rep."""
    import torch
    from paper_1802_05421_gb300 import build as B
    B.build()
    from paper_1802_05421_gb300 import cdl
    if args.case == "batched":
        return run_case_batched(args, cdl)
    from workloads import iid_pair
    wl = iid_pair(args.n, 64, 8, seed=5)
    n, T = wl.X[0].shape
    st, ctx = cdl.cdl_ctx_create(0, torch.cuda.current_stream().cuda_stream, 0)
    assert st == 0
    X = torch.from_numpy(wl.X[0]).cuda()
    A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    D = torch.empty(n, dtype=torch.float64, device="cuda")
    sc = torch.zeros(2, dtype=torch.float64, device="cuda")
    vol, sig = sc[0:1].data_ptr(), sc[1:2].data_ptr()
    k = K_PROJ
    Y = torch.empty((n, k), dtype=torch.float64, device="cuda")
    Z = torch.empty((n, k), dtype=torch.float64, device="cuda")
    ch = None
    for _ in range(args.reps):
        assert cdl.cdl_build_graph(ctx, X, n, T, 0.0, cdl.CDL_F64, A, D, vol, sig) == 0
        if args.case in ("square", "solve"):
            cdt = cdl.CDL_FP8E4M3_T128 if args.chain == "fp8t" else cdl.CDL_BF16
            st, ch = cdl.cdl_chain_build(ctx, A, cdl.CDL_F64, D, vol, n, 2 if args.case == "square" else 4,
                                         cdt, 0, ch)
            assert st == 0
        if args.case in ("project", "solve", "score"):
            assert cdl.cdl_project(ctx, A, cdl.CDL_F64, n, k, SEED, Y) == 0
        if args.case == "solve":
            st = cdl.cdl_chain_solve(ctx, ch, A, cdl.CDL_F64, Y, k, cdl.cdl_solve_opts(3, 0.0, 0), Z, None)
            assert st == 0
        if args.case == "score":
            F = torch.empty(n, dtype=torch.float64, device="cuda")
            top = torch.empty(TOPK, dtype=torch.int64, device="cuda")
            Z2 = Y * 1e-3
            assert cdl.cdl_cad_score(ctx, A, A.flip(0).contiguous(), cdl.CDL_F64, Z2, Z2 * 1.5, vol, vol, n, k,
                                     cdl.CDL_BF16 if args.score == "bf16" else cdl.CDL_F32, TOPK, F, top) == 0
    assert cdl.cdl_sync(ctx) == 0
    if ch is not None:
        cdl.cdl_chain_free(ch)
    cdl.cdl_ctx_destroy(ctx)
    print(f"case {args.case} n={n} reps={args.reps} ok")
    return 0


def run_case_batched(args, cdl):
    import torch
    from workloads import ragged_pairs
    pairs = ragged_pairs(G=args.n, n_lo=256, n_hi=4096, T=64, seed=7)
    G = len(pairs)
    n = np.array([p.X[0].shape[0] for p in pairs], dtype=np.int64)
    N = int(n.sum())
    X1 = torch.from_numpy(np.ascontiguousarray(np.concatenate([p.X[0] for p in pairs]))).cuda()
    X2 = torch.from_numpy(np.ascontiguousarray(np.concatenate([p.X[1] for p in pairs]))).cuda()
    F = torch.empty(N, dtype=torch.float64, device="cuda")
    top = torch.empty(G * BATCH_TOPK, dtype=torch.int64, device="cuda")
    stats = (cdl.cdl_solve_stats * (2 * G))()
    st, ctx = cdl.cdl_ctx_create(0, torch.cuda.current_stream().cuda_stream, 0)
    assert st == 0
    o = cdl.cdl_batch_opts(BATCH_K, BATCH_D, cdl.CDL_BF16, cdl.CDL_F32, SEED, 0.0,
                           cdl.cdl_solve_opts(30, BATCH_TOL, 0), BATCH_TOPK, 0, 0)
    for _ in range(args.reps):
        assert cdl.cdl_caddelag_batched(ctx, G, n, 64, X1, X2, o, F, top, stats) == 0
    assert cdl.cdl_sync(ctx) == 0
    cdl.cdl_ctx_destroy(ctx)
    print(f"case batched pairs={G} sum_n={N} reps={args.reps} ok")
    return 0


# ---------------------------------------------------------------- batched form
BATCH_METRIC = "graph pairs/s, 64 ragged pairs (n log-uniform in [256, 4096])"
BATCH_WORKLOAD = "ragged_64pairs_n256_4096"
BATCH_K, BATCH_D, BATCH_TOPK, BATCH_TOL = 32, 10, 10, 1e-12


def run_batched(args):
    """The batched form: 64 independent pairs of uneven order (seeded
    log-uniform n in [256, 4096], T = 64, N(0,1) series, 1-5 perturbed nodes
    each) through one cdl_caddelag_batched call per step, recorded once as a
    CUDA graph and replayed. Every rank runs its own replica of the batch."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1802_05421_gb300 import build as B
    B.build()
    line = batched_measure(args.steps, args.warmup, args.e2e_steps, dist, world, local, sample_clocks=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def batched_measure(steps, warmup, e2e_steps, dist, world, local, sample_clocks):
    """Time the batched workload (see run_batched) and return its JSON record."""
    import torch
    from paper_1802_05421_gb300 import cdl
    from workloads import ragged_pairs
    pairs = ragged_pairs(G=64, n_lo=256, n_hi=4096, T=64, seed=7)
    G = len(pairs)
    n = np.array([p.X[0].shape[0] for p in pairs], dtype=np.int64)
    T = pairs[0].X[0].shape[1]
    N = int(n.sum())
    X1h = np.ascontiguousarray(np.concatenate([p.X[0] for p in pairs]))
    X2h = np.ascontiguousarray(np.concatenate([p.X[1] for p in pairs]))
    stream = torch.cuda.Stream()
    st, ctx = cdl.cdl_ctx_create(local, stream.cuda_stream, 0)
    assert st == 0, cdl.cdl_status_string(st)
    X1 = torch.from_numpy(X1h).cuda()
    X2 = torch.from_numpy(X2h).cuda()
    F = torch.empty(N, dtype=torch.float64, device="cuda")
    top = torch.empty(G * BATCH_TOPK, dtype=torch.int64, device="cuda")
    stats = (cdl.cdl_solve_stats * (2 * G))()

    def opts(use_graph, host_io=0):
        return cdl.cdl_batch_opts(BATCH_K, BATCH_D, cdl.CDL_BF16, cdl.CDL_F32, SEED, 0.0,
                                  cdl.cdl_solve_opts(30, BATCH_TOL, 0), BATCH_TOPK, host_io, use_graph)

    def call(o, x1=X1, x2=X2, f=F, t=top):
        r = cdl.cdl_caddelag_batched(ctx, G, n, T, x1, x2, o, f, t, stats)
        if r != 0:
            raise RuntimeError(f"cdl_caddelag_batched: {cdl.cdl_status_string(r)} {cdl.cdl_last_error_detail()}")

    og = opts(1)
    for _ in range(warmup):
        call(og)
    torch.cuda.synchronize()
    _, l0 = cdl.cdl_ctx_launch_count(ctx)
    sampler = ClockSampler(local) if sample_clocks else None
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        call(og)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = ev0.elapsed_time(ev1) / steps
    _, l1 = cdl.cdl_ctx_launch_count(ctx)
    iters = [stats[g].iters for g in range(2 * G)]
    rel_res = max(stats[g].rel_res for g in range(2 * G))

    _, info = cdl.cdl_batch_plan_info(ctx)
    tuning = {"square_max_npad_128": info.square_max_npad_128,
              "project_rows_per_block": info.project_rows_per_block,
              "residual_tile": [info.residual_tile_m, info.residual_tile_n],
              "slots_captured": info.slots_captured,
              "square_variants_ms": {str(info.square_variant_max_npad_128[v]): round(info.square_variant_ms[v], 4)
                                     for v in range(info.n_square_variants)},
              "project_variants_ms": {str(info.project_variant_rows[v]): round(info.project_variant_ms[v], 4)
                                      for v in range(info.n_project_variants)},
              "device_gb": round(info.device_bytes / 1e9, 2)}

    # one eager call with per-kernel timing: the grouped squaring launches
    eager = opts(0)
    call(eager)   # builds the eager plan's state (same sizes: the plan is reused)
    cdl.cdl_ctx_reset_counters(ctx)
    cdl.cdl_ctx_set_timing(ctx, True)
    call(eager)
    kc = {}
    for i, name in enumerate(cdl.KERNEL_CLASSES):
        _, ms, cnt, work = cdl.cdl_ctx_timing(ctx, i)
        kc[name] = dict(ms=ms, launches=cnt, work=work / max(cnt, 1), ms_per_launch=ms / max(cnt, 1))
    cdl.cdl_ctx_set_timing(ctx, False)

    # end to end with pinned host buffers (host_io: copies inside the call)
    h1 = torch.from_numpy(X1h).pin_memory()
    h2 = torch.from_numpy(X2h).pin_memory()
    hF = torch.empty(N, dtype=torch.float64).pin_memory()
    ht = torch.empty(G * BATCH_TOPK, dtype=torch.int64).pin_memory()
    oh = opts(1, 1)
    call(oh, h1.data_ptr(), h2.data_ptr(), hF.data_ptr(), ht.data_ptr())   # records the graph for host I/O
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        call(oh, h1.data_ptr(), h2.data_ptr(), hF.data_ptr(), ht.data_ptr())
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    same_top = ht.tolist() == top.cpu().tolist()
    step_ms, e2e_s = rank_max([step_ms, e2e_s], dist, "cuda")
    pk, src = peaks()
    sq = kc["square"]
    achieved = sq["work"] / (sq["ms_per_launch"] * 1e-3) / 1e12 if sq["ms_per_launch"] else 0.0
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    line = {
        "metric": BATCH_METRIC, "value": world * G * 1000.0 / step_ms, "unit": "pairs/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "pairs": G, "n_min": int(n.min()), "n_max": int(n.max()),
                   "sum_n": N, "T": T, "k": BATCH_K, "d": BATCH_D, "topk": BATCH_TOPK, "score": "f32",
                   "refine_rel_tol": BATCH_TOL, "solve_iters_max": max(iters), "rel_res_max": rel_res,
                   "cuda_graph": True, "parallelism": f"replicas x{world}",
                   "l2": "no flush: each step writes 2 x 64 chains of 10 bf16 levels (about 30 GB), "
                         "far larger than the 129 MB L2"},
        "roofline": {"kernel": "k_tc_gemm grouped squaring (one launch per level over 128 graphs)",
                     "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "peak_source": f"{src} bf16_tflops_sustained",
                     "work_per_launch": sq["work"], "ms_per_launch": sq["ms_per_launch"],
                     "timed": "one eager call with per-launch CUDA events"},
        "cpu_baseline": None,
        "e2e": {"value": world * G / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": 2 * N * T * 8,
                "d2h_bytes_per_step": N * 8 + G * BATCH_TOPK * 8, "same_top_as_device_run": same_top},
        "gpu_launches": int((l1 - l0) // steps),
        "clocks": clocks,
        "autotuner": tuning,
        "eager_phases_ms": {k: round(v["ms"], 3) for k, v in kc.items()},
    }
    cdl.cdl_ctx_destroy(ctx)
    return line


# ---------------------------------------------------------------- host levels
def run_host_levels(args):
    """The larger-than-memory form at the n = 32768 field pair: chain levels
    in pinned host memory (CDL_CHAIN_HOST_LEVELS), streamed through two
    device slots, against the same pair with device-resident levels. Reports
    the copies the library made (count, bytes, summed time on the chain's
    copy stream), the rates of plain one-level copies for comparison, and how
    much of the copy time the step hides."""
    import torch
    torch.cuda.set_device(0)
    from paper_1802_05421_gb300 import build as B
    B.build()
    from paper_1802_05421_gb300 import cdl
    wl = make_workload()
    n, T = wl.X[0].shape
    stream = torch.cuda.Stream()
    st, ctx = cdl.cdl_ctx_create(0, stream.cuda_stream, 0)
    assert st == 0
    X1 = torch.from_numpy(wl.X[0]).cuda()
    X2 = torch.from_numpy(wl.X[1]).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    top = torch.empty(TOPK, dtype=torch.int64, device="cuda")
    s1, s2 = cdl.cdl_solve_stats(), cdl.cdl_solve_stats()

    def timed(flags, steps, warmup):
        o = cdl.cdl_pair_opts(K_PROJ, D_CHAIN, cdl.CDL_BF16, cdl.CDL_BF16 if args.score == "bf16" else cdl.CDL_F32,
                              SEED, 0.0,
                              cdl.cdl_solve_opts(40, REL_TOL, 0), TOPK, 0, flags)
        for _ in range(warmup):
            assert cdl.cdl_caddelag_pair(ctx, X1, X2, n, T, o, F, top, s1, s2) == 0
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            assert cdl.cdl_caddelag_pair(ctx, X1, X2, n, T, o, F, top, s1, s2) == 0
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, F.cpu().numpy().copy(), top.cpu().tolist(), (s1.iters, s2.iters)

    sampler = ClockSampler(0)
    ms_dev, F_dev, top_dev, it_dev = timed(0, max(1, args.steps), args.warmup)
    ms_host, F_host, top_host, it_host = timed(cdl.CDL_CHAIN_HOST_LEVELS, max(1, args.steps), args.warmup)
    clocks = sampler.stop()
    # one more pair with class timing on: the copies the chain made and their
    # summed time on its copy stream
    cdl.cdl_ctx_reset_counters(ctx)
    cdl.cdl_ctx_set_timing(ctx, True)
    timed(cdl.CDL_CHAIN_HOST_LEVELS, 1, 0)
    _, copy_ms, copies, copy_bytes = cdl.cdl_ctx_timing(ctx, cdl.CDL_KC_HOST_LINK)
    cdl.cdl_ctx_set_timing(ctx, False)
    # link copy rates with a pinned buffer of one level (npad^2 bf16)
    npad = (n + 255) // 256 * 256
    lb = npad * npad * 2
    hbuf = torch.empty(lb, dtype=torch.uint8).pin_memory()
    dbuf = torch.empty(lb, dtype=torch.uint8, device="cuda")
    rates = {}
    for name, fn in (("h2d", lambda: dbuf.copy_(hbuf, non_blocking=True)),
                     ("d2h", lambda: hbuf.copy_(dbuf, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            fn()
        e1.record()
        torch.cuda.synchronize()
        rates[name] = 5 * lb / (e0.elapsed_time(e1) * 1e-3) / 1e9
    hidden = 1.0 - max(0.0, ms_host - ms_dev) / copy_ms if copy_ms > 0 else None
    line = {"metric": METRIC + " (chain levels in pinned host memory)", "value": 1000.0 / ms_host,
            "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_host,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "T": T, "k": K_PROJ, "d": D_CHAIN, "chain_flags": "HOST_LEVELS",
                       "level_bytes": lb, "host_level_bytes": D_CHAIN * lb, "solve_iters": list(it_host)},
            "device_levels_ms_per_step": ms_dev,
            "identical_to_device_levels": bool(np.array_equal(F_dev, F_host) and top_dev == top_host),
            "link": {"copies_per_pair": copies, "bytes_per_pair": copy_bytes, "copy_ms_per_pair": copy_ms,
                     "copy_gbs_in_pair": copy_bytes / (copy_ms * 1e6) if copy_ms > 0 else None,
                     "h2d_gbs_one_level_buffer": rates["h2d"], "d2h_gbs_one_level_buffer": rates["d2h"],
                     "fraction_of_copy_time_hidden": hidden},
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    cdl.cdl_ctx_destroy(ctx)
    return 0


# ---------------------------------------------------------------- synthetic mixture pair
GMM_N = 32768
GMM_WORKLOAD = "gmm_n32768_pair"


C5_WORKLOAD = "field_n131072_pair"
C5_METRIC = "graph pairs/s at n=131072 (graphs regenerated in row panels, chain levels partly in pinned host memory)"
C5_K, C5_D, C5_TOPK = 192, 10, 100


def field_pair_n131072():
    from workloads import field_sequence
    return field_sequence(256, 512, 365, 2, patch=16, patch_transition=0, seasonal=0.5, seed=5)


def run_larger_than_hbm(args):
    """The larger-than-memory form at its own size: one pair at n = 131072
    (256 x 512 grid, T = 365 field samples plus a seasonal sinusoid, a
    planted 16 x 16 patch), k = 192, d = 10, bf16 levels (as many as fit on
    the device, the rest in pinned host memory), refinement to 1e-10,
    top-100; neither float64 graph (137 GB each) is stored: both are
    regenerated from the node series in row panels wherever they are needed.
    One warm-up pair (it allocates and pins the levels), then --steps pairs
    (default 1) between CUDA events; then one pair with per-class timing."""
    import torch
    torch.cuda.set_device(0)
    from paper_1802_05421_gb300 import build as B
    B.build()
    from paper_1802_05421_gb300 import cdl
    wl = field_pair_n131072()
    n, T = wl.X[0].shape
    stream = torch.cuda.Stream()
    st, ctx = cdl.cdl_ctx_create(0, stream.cuda_stream, 0)
    assert st == 0
    X1 = torch.from_numpy(wl.X[0]).cuda()
    X2 = torch.from_numpy(wl.X[1]).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    top = torch.empty(C5_TOPK, dtype=torch.int64, device="cuda")
    s1, s2 = cdl.cdl_solve_stats(), cdl.cdl_solve_stats()
    flags = cdl.CDL_PAIR_REGEN_GRAPHS | cdl.CDL_CHAIN_HOST_LEVELS | cdl.CDL_CHAIN_RESIDENT(255)
    o = cdl.cdl_pair_opts(C5_K, C5_D, cdl.CDL_BF16, cdl.CDL_BF16, SEED, 0.0, cdl.cdl_solve_opts(40, REL_TOL, 0),
                          C5_TOPK, 0, flags)

    def call(opts=o, x1=X1, x2=X2, f=F, t=top):
        r = cdl.cdl_caddelag_pair(ctx, x1, x2, n, T, opts, f, t, s1, s2)
        if r != 0:
            raise RuntimeError(f"cdl_caddelag_pair: {cdl.cdl_status_string(r)} {cdl.cdl_last_error_detail()}")

    t0 = time.perf_counter()
    call()
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    steps = max(1, args.large_steps)
    _, l0 = cdl.cdl_ctx_launch_count(ctx)
    sampler = ClockSampler(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = e0.elapsed_time(e1) / steps
    _, l1 = cdl.cdl_ctx_launch_count(ctx)
    top_dev = top.cpu().tolist()
    iters = (s1.iters, s2.iters)
    rel_res = max(s1.rel_res, s2.rel_res)
    # one pair with per-class timing: phases, the squaring's rate, the host link
    cdl.cdl_ctx_reset_counters(ctx)
    cdl.cdl_ctx_set_timing(ctx, True)
    call()
    kc = {}
    for i, name in enumerate(cdl.KERNEL_CLASSES + ["host_link"]):
        _, ms, cnt, work = cdl.cdl_ctx_timing(ctx, i)
        kc[name] = dict(ms=ms, launches=cnt, work=work)
    cdl.cdl_ctx_set_timing(ctx, False)
    # end to end with host buffers (the series in, scores and top-100 out)
    h1 = torch.from_numpy(wl.X[0]).pin_memory()
    h2 = torch.from_numpy(wl.X[1]).pin_memory()
    hF = torch.empty(n, dtype=torch.float64).pin_memory()
    ht = torch.empty(C5_TOPK, dtype=torch.int64).pin_memory()
    oh = cdl.cdl_pair_opts(C5_K, C5_D, cdl.CDL_BF16, cdl.CDL_BF16, SEED, 0.0, cdl.cdl_solve_opts(40, REL_TOL, 0),
                           C5_TOPK, 1, flags)
    t0 = time.perf_counter()
    call(oh, h1.data_ptr(), h2.data_ptr(), hF.data_ptr(), ht.data_ptr())
    e2e_s = time.perf_counter() - t0
    pk, src = peaks()
    sq = kc["square"]
    ach = sq["work"] / (sq["ms"] * 1e-3) / 1e12 if sq["ms"] else 0.0
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    npad = (n + 255) // 256 * 256
    lb = npad * npad * 2
    link = kc["host_link"]
    line = {
        "metric": C5_METRIC, "value": 1000.0 / step_ms, "unit": "pairs/s", "n_gpus": 1, "steps": steps,
        "warmup": 1, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": C5_WORKLOAD, "n": n, "T": T, "k": C5_K, "d": C5_D, "topk": C5_TOPK,
                   "chain": "bf16", "score": "bf16", "refine_rel_tol": REL_TOL, "solve_iters": list(iters),
                   "rel_res": rel_res, "graphs": "regenerated in row panels of 4096 (not stored)",
                   "levels": "as many on the device as fit, the rest in pinned host memory",
                   "level_bytes": lb, "float64_graph_bytes": 8 * n * n,
                   "l2": "no flush: each step streams hundreds of GB"},
        "first_call_s": first_s,
        "roofline": {"kernel": "k_tc_sq2 (chain squaring on CTA pairs)", "bound": "tensor", "achieved": ach,
                     "peak": peak,
                     "unit": "TFLOP/s", "frac": ach / peak if peak else None, "traffic": None,
                     "peak_source": f"{src} bf16_tflops_sustained",
                     "ms_per_launch": sq["ms"] / max(sq["launches"], 1), "launches": sq["launches"]},
        "link": {"copies_per_pair": link["launches"], "bytes_per_pair": link["work"], "copy_ms_per_pair": link["ms"]},
        "e2e": {"value": 1.0 / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": 2 * n * T * 8,
                "d2h_bytes_per_step": n * 8 + C5_TOPK * 8, "same_top_as_device_run": ht.tolist() == top_dev},
        "gpu_launches": int((l1 - l0) // steps),
        "clocks": clocks,
        "phases_ms_per_step": {k: round(v["ms"], 1) for k, v in kc.items()},
        "planted_in_top": len(set(top_dev) & set(wl.planted[0].tolist())),
    }
    print(json.dumps(line), flush=True)
    cdl.cdl_ctx_destroy(ctx)
    return 0


def run_gmm(args):
    """The paper's synthetic data (Sec. 4.2.1) at n = 32768: graph 1 is the
    exp(-d) kernel graph of a 4-component 2-D Gaussian mixture, graph 2 that
    of the same points with small noise plus the symmetrised sparse random
    weights (R + R^T) / 2 (p = 0.05). One step = both graphs built
    (cdl_build_graph_kernel, cdl_graph_add_edges, cdl_graph_degrees), chain
    (bf16, d = 14), projection (k = 128), solve to 1e-10 and CAD scores for the
    pair, through the C ABI stage by stage. After timing, the anomalous edge
    ranking is scored against the cross-cluster ground truth."""
    import torch
    torch.cuda.set_device(0)
    from paper_1802_05421_gb300 import build as B
    B.build()
    from paper_1802_05421_gb300 import cdl
    from workloads import gmm_pair
    g = gmm_pair(GMM_N, seed=11)
    n, T = g.X[0].shape
    m = len(g.w)
    stream = torch.cuda.Stream()
    st, ctx = cdl.cdl_ctx_create(0, stream.cuda_stream, 0)
    assert st == 0, cdl.cdl_status_string(st)

    def ok(r, what):
        if r != 0:
            raise RuntimeError(f"{what}: {cdl.cdl_status_string(r)} {cdl.cdl_last_error_detail()}")

    hX1 = torch.from_numpy(g.X[0]).pin_memory()
    hX2 = torch.from_numpy(g.X[1]).pin_memory()
    hij = torch.from_numpy(g.ij).pin_memory()
    hw = torch.from_numpy(g.w).pin_memory()
    with torch.cuda.stream(stream):
        X1, X2 = hX1.cuda(), hX2.cuda()
        ij, w = hij.cuda(), hw.cuda()
        A = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(2)]
        D = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
        sc = torch.zeros(4, dtype=torch.float64, device="cuda")      # vol1, vol2, sigma1, sigma2
        Y = torch.empty((n, K_PROJ), dtype=torch.float64, device="cuda")
        Z = [torch.empty((n, K_PROJ), dtype=torch.float64, device="cuda") for _ in range(2)]
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        top = torch.empty(TOPK, dtype=torch.int64, device="cuda")
    stream.synchronize()
    vol = [sc[0:1], sc[1:2]]
    chain = [None]
    gscore = cdl.CDL_BF16 if args.score == "bf16" else cdl.CDL_F32
    stats = [cdl.cdl_solve_stats(), cdl.cdl_solve_stats()]
    sopts = cdl.cdl_solve_opts(40, REL_TOL, 0)

    def step(x1=X1, x2=X2, eij=ij, ew=w):
        for t, x in enumerate((x1, x2)):
            ok(cdl.cdl_build_graph_kernel(ctx, x, n, T, cdl.CDL_KERNEL_EXP, 1.0, cdl.CDL_F64, A[t], D[t],
                                          vol[t].data_ptr(), sc[2 + t:3 + t].data_ptr()), "build_graph_kernel")
        r, bad = cdl.cdl_graph_add_edges(ctx, A[1], cdl.CDL_F64, n, m, eij, ew)
        ok(r, "graph_add_edges")
        ok(cdl.cdl_graph_degrees(ctx, A[1], cdl.CDL_F64, n, D[1], vol[1].data_ptr()), "graph_degrees")
        for t in range(2):
            r, chain[0] = cdl.cdl_chain_build(ctx, A[t], cdl.CDL_F64, D[t], vol[t].data_ptr(), n, D_CHAIN,
                                              cdl.CDL_BF16, 0, chain[0])
            ok(r, "chain_build")
            ok(cdl.cdl_project(ctx, A[t], cdl.CDL_F64, n, K_PROJ, SEED, Y), "project")
            ok(cdl.cdl_chain_solve(ctx, chain[0], A[t], cdl.CDL_F64, Y, K_PROJ, sopts, Z[t], stats[t]), "solve")
        ok(cdl.cdl_cad_score(ctx, A[0], A[1], cdl.CDL_F64, Z[0], Z[1], vol[0].data_ptr(), vol[1].data_ptr(), n,
                             K_PROJ, gscore, TOPK, F, top), "cad_score")

    for _ in range(args.warmup):
        step()
    ok(cdl.cdl_sync(ctx), "sync")
    cdl.cdl_ctx_reset_counters(ctx)
    cdl.cdl_ctx_set_timing(ctx, True)
    sampler = ClockSampler(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = ev0.elapsed_time(ev1) / args.steps
    _, launches = cdl.cdl_ctx_launch_count(ctx)
    kc = {}
    for i, name in enumerate(cdl.KERNEL_CLASSES):
        _, ms, cnt, work = cdl.cdl_ctx_timing(ctx, i)
        kc[name] = dict(ms_per_step=ms / args.steps, work=work / max(cnt, 1), ms_per_launch=ms / max(cnt, 1))
    cdl.cdl_ctx_set_timing(ctx, False)
    iters = [stats[0].iters, stats[1].iters]
    rel_res = max(stats[0].rel_res, stats[1].rel_res)
    top_dev = top.cpu().tolist()

    # end to end: the step's inputs (points and the added edge list) copied in
    # from pinned host memory, node scores and top nodes read back
    hF = torch.empty(n, dtype=torch.float64).pin_memory()
    htop = torch.empty(TOPK, dtype=torch.int64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        with torch.cuda.stream(stream):
            X1.copy_(hX1, non_blocking=True)
            X2.copy_(hX2, non_blocking=True)
            ij.copy_(hij, non_blocking=True)
            w.copy_(hw, non_blocking=True)
        step()
        with torch.cuda.stream(stream):
            hF.copy_(F, non_blocking=True)
            htop.copy_(top, non_blocking=True)
        stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps

    # detector quality against the ground truth: every edge's Delta E
    cdl.cdl_chain_free(chain[0])
    del Y
    M = n * (n - 1) // 2
    quality = None
    try:
        with torch.cuda.stream(stream):
            eij_all = torch.empty((M, 2), dtype=torch.int64, device="cuda")
            ev_all = torch.empty(M, dtype=torch.float64, device="cuda")
        r, res = cdl.cdl_cad_edges(ctx, A[0], A[1], cdl.CDL_F64, Z[0], Z[1], vol[0].data_ptr(),
                                   vol[1].data_ptr(), n, K_PROJ, cdl.CDL_F64, 1e-300, M, eij_all, ev_all,
                                   None, 0, 0, None, None, None)
        ok(r, "cad_edges")
        torch.cuda.synchronize()
        cnt = int(min(res.n_edges, M))
        flat = eij_all[:cnt, 0] * n + eij_all[:cnt, 1]
        vals = ev_all[:cnt]
        del eij_all
        fa = ij[:, 0] * n + ij[:, 1]
        pos = torch.searchsorted(flat, fa).clamp_(max=max(cnt - 1, 0))
        e_added = torch.where(flat[pos] == fa, vals[pos], torch.zeros_like(vals[pos]))
        truth = torch.from_numpy(g.truth).cuda()
        P = int(truth.sum())
        ranks = torch.empty(m, dtype=torch.float64, device="cuda")
        ranks[torch.argsort(e_added)] = torch.arange(1, m + 1, dtype=torch.float64, device="cuda")
        auc = float((ranks[truth].sum() - P * (P + 1) / 2) / (P * (m - P)))
        dA = (A[0][ij[:, 0], ij[:, 1]] - A[1][ij[:, 0], ij[:, 1]]).abs()
        ranks[torch.argsort(dA)] = torch.arange(1, m + 1, dtype=torch.float64, device="cuda")
        auc_dA = float((ranks[truth].sum() - P * (P + 1) / 2) / (P * (m - P)))
        thr = float(torch.topk(vals, P, sorted=False).values.min())
        prec = float((e_added[truth] >= thr).sum()) / P
        quality = {"edges_total": M, "edges_added": m, "ground_truth_edges": P,
                   "precision_at_ground_truth_size": prec, "chance_precision": P / M,
                   "auc_among_added_edges": auc, "auc_among_added_edges_delta_A_only": auc_dA}
    except (RuntimeError, torch.cuda.OutOfMemoryError) as e:
        quality = {"error": str(e)[:200]}

    pk, src = peaks()
    sq = kc["square"]
    achieved = sq["work"] / (sq["ms_per_launch"] * 1e-3) / 1e12 if sq["ms_per_launch"] else 0.0
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    line = {
        "metric": "graph pairs/s at n=32768 (synthetic mixture graphs)", "value": 1000.0 / step_ms,
        "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": GMM_WORKLOAD, "n": n, "points": "2-D, 4 components at (+-3, +-3), unit covariance",
                   "kernel": "exp(-d)", "noise": g.meta["noise"], "p": g.meta["p"], "added_edges": m,
                   "k": K_PROJ, "d": D_CHAIN, "chain": "bf16", "score": args.score, "topk": TOPK,
                   "refine_rel_tol": REL_TOL, "solve_iters": iters, "rel_res": rel_res,
                   "l2": "no flush: each step writes two 8.6 GB float64 graphs and 2 x 30 GB of chain "
                         "levels, far larger than the 129 MB L2"},
        "roofline": {"kernel": "k_tc_sq2 (chain squaring on CTA pairs)", "bound": "tensor", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": None,
                     "peak_source": f"{src} bf16_tflops_sustained", "work_per_launch": sq["work"],
                     "ms_per_launch": sq["ms_per_launch"]},
        "cpu_baseline": None,
        "e2e": {"value": 1.0 / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": 2 * n * T * 8 + m * 24,
                "d2h_bytes_per_step": n * 8 + TOPK * 8, "same_top_as_device_run": htop.tolist() == top_dev},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "phases_ms_per_step": {k: round(v["ms_per_step"], 3) for k, v in kc.items()},
        "detector_vs_ground_truth": quality,
    }
    print(json.dumps(line), flush=True)
    cdl.cdl_ctx_destroy(ctx)
    return 0


# ---------------------------------------------------------------- float32 sequence
SEQ_WORKLOAD = "field_n8192_seq4"


def run_sequence(args):
    """The plain float32 GPU path on a graph sequence: 4 graphs of the 64 x 128
    correlated field (n = 8192, T = 128, AR(1) drift, an 8 x 8 patch shifted in
    the second transition), each embedded once (float32 chain on CUDA cores,
    d = 12; projection k = 64; solve to 1e-10) and reused by its two pairs,
    then the 3 transitions scored in float32. One step = the whole sequence
    through the C ABI stage by stage; value = transitions scored per second."""
    import torch
    torch.cuda.set_device(0)
    from paper_1802_05421_gb300 import build as B
    B.build()
    from paper_1802_05421_gb300 import cdl
    from workloads import field_sequence
    wl = field_sequence(64, 128, 128, 4, patch=8, patch_transition=1, seed=1)
    G = len(wl.X)
    n, T = wl.X[0].shape
    k, d = 64, 12
    stream = torch.cuda.Stream()
    st, ctx = cdl.cdl_ctx_create(0, stream.cuda_stream, 0)
    assert st == 0, cdl.cdl_status_string(st)

    def ok(r, what):
        if r != 0:
            raise RuntimeError(f"{what}: {cdl.cdl_status_string(r)} {cdl.cdl_last_error_detail()}")

    hX = [torch.from_numpy(x).pin_memory() for x in wl.X]
    with torch.cuda.stream(stream):
        X = [h.cuda() for h in hX]
        A = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(G)]
        D = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(G)]
        sc = torch.zeros(2 * G, dtype=torch.float64, device="cuda")     # vol, sigma per graph
        Y = torch.empty((n, k), dtype=torch.float64, device="cuda")
        Z = [torch.empty((n, k), dtype=torch.float64, device="cuda") for _ in range(G)]
        F = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(G - 1)]
        top = [torch.empty(TOPK, dtype=torch.int64, device="cuda") for _ in range(G - 1)]
    stream.synchronize()
    vol = [sc[t:t + 1] for t in range(G)]
    chain = [None]
    stats = [cdl.cdl_solve_stats() for _ in range(G)]
    sopts = cdl.cdl_solve_opts(40, REL_TOL, 0)

    def step():
        for t in range(G):
            ok(cdl.cdl_build_graph(ctx, X[t], n, T, 0.0, cdl.CDL_F64, A[t], D[t], vol[t].data_ptr(),
                                   sc[G + t:G + t + 1].data_ptr()), "build_graph")
            r, chain[0] = cdl.cdl_chain_build(ctx, A[t], cdl.CDL_F64, D[t], vol[t].data_ptr(), n, d, cdl.CDL_F32,
                                              0, chain[0])
            ok(r, "chain_build")
            ok(cdl.cdl_project(ctx, A[t], cdl.CDL_F64, n, k, SEED, Y), "project")
            ok(cdl.cdl_chain_solve(ctx, chain[0], A[t], cdl.CDL_F64, Y, k, sopts, Z[t], stats[t]), "solve")
        for t in range(G - 1):
            ok(cdl.cdl_cad_score(ctx, A[t], A[t + 1], cdl.CDL_F64, Z[t], Z[t + 1], vol[t].data_ptr(),
                                 vol[t + 1].data_ptr(), n, k, cdl.CDL_F32, TOPK, F[t], top[t]), "cad_score")

    for _ in range(args.warmup):
        step()
    ok(cdl.cdl_sync(ctx), "sync")
    cdl.cdl_ctx_reset_counters(ctx)
    cdl.cdl_ctx_set_timing(ctx, True)
    sampler = ClockSampler(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = ev0.elapsed_time(ev1) / args.steps
    _, launches = cdl.cdl_ctx_launch_count(ctx)
    kc = {}
    for i, name in enumerate(cdl.KERNEL_CLASSES):
        _, ms, cnt, work = cdl.cdl_ctx_timing(ctx, i)
        kc[name] = dict(ms_per_step=ms / args.steps, work=work / max(cnt, 1), ms_per_launch=ms / max(cnt, 1))
    cdl.cdl_ctx_set_timing(ctx, False)
    tops = [tp.cpu().tolist() for tp in top]
    planted_on_top = set(tops[1]) <= set(wl.planted[1].tolist())

    # end to end: the 4 series copied in from pinned host memory, the 3 score
    # vectors and top lists read back
    hF = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(G - 1)]
    htop = [torch.empty(TOPK, dtype=torch.int64).pin_memory() for _ in range(G - 1)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        with torch.cuda.stream(stream):
            for t in range(G):
                X[t].copy_(hX[t], non_blocking=True)
        step()
        with torch.cuda.stream(stream):
            for t in range(G - 1):
                hF[t].copy_(F[t], non_blocking=True)
                htop[t].copy_(top[t], non_blocking=True)
        stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    if chain[0] is not None:
        cdl.cdl_chain_free(chain[0])

    # the float32 squaring on the CUDA cores against the float32 FMA rate of the
    # part: 152 SMs x 128 lanes x 2 flop x the maximum SM clock
    pk, _ = peaks()
    f32_peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    sq = kc["square"]
    achieved = sq["work"] / (sq["ms_per_launch"] * 1e-3) / 1e12 if sq["ms_per_launch"] else 0.0
    line = {
        "metric": "graph pairs/s on the n=8192 sequence (plain float32 GPU path)",
        "value": (G - 1) * 1000.0 / step_ms, "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": SEQ_WORKLOAD, "n": n, "T": T, "graphs": G, "transitions": G - 1, "k": k, "d": d,
                   "chain": "f32", "score": "f32", "topk": TOPK, "refine_rel_tol": REL_TOL,
                   "solve_iters": [s.iters for s in stats], "rel_res": max(s.rel_res for s in stats),
                   "planted_patch_on_top": planted_on_top,
                   "l2": "no flush: each step writes four 537 MB float64 graphs and their 3 GB float32 chains, "
                         "larger than the 129 MB L2"},
        "roofline": {"kernel": "k_gemm_tn (float32 chain squaring, CUDA cores)", "bound": "alu",
                     "achieved": achieved, "peak": f32_peak, "unit": "TFLOP/s",
                     "frac": achieved / f32_peak if f32_peak else None, "traffic": None,
                     "peak_source": "derived: 152 SMs x 128 float32 lanes x 2 flop x sm_max_mhz",
                     "work_per_launch": sq["work"], "ms_per_launch": sq["ms_per_launch"]},
        "cpu_baseline": None,
        "e2e": {"value": (G - 1) / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": G * n * T * 8,
                "d2h_bytes_per_step": (G - 1) * (n * 8 + TOPK * 8),
                "same_top_as_device_run": [h.tolist() for h in htop] == tops},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "phases_ms_per_step": {k2: round(v["ms_per_step"], 3) for k2, v in kc.items()},
    }
    print(json.dumps(line), flush=True)
    cdl.cdl_ctx_destroy(ctx)
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cdl", choices=["cdl", "reference"])
    ap.add_argument("--chain", default="bf16", choices=["bf16", "fp8", "fp8t", "f32", "f64"])
    ap.add_argument("--score", default="bf16", choices=["bf16", "f32"],
                    help="score arithmetic of the tensor-chain paths: bf16 = exact slices on the tensor cores, "
                         "f32 = compensated float32 pipes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-compare-f32", dest="compare_f32", action="store_false",
                    help="skip the plain float32 GPU path comparison step")
    ap.add_argument("--case", default=None, choices=["square", "solve", "project", "score", "batched"],
                    help="run a small single-kernel case for a profiler capture instead of the bench")
    ap.add_argument("--n", type=int, default=12288)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--large-steps", type=int, default=1, help="timed pairs of --workload larger-than-hbm")
    ap.add_argument("--workload", default="pair",
                    choices=["pair", "batched", "host-levels", "gmm", "sequence", "larger-than-hbm"],
                    help="pair: the n = 32768 field pair (default); batched: 64 ragged pairs; "
                         "host-levels: the pair with chain levels in pinned host memory; "
                         "gmm: the synthetic mixture pair at n = 32768")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "host-levels":
        return run_host_levels(args)
    if args.workload == "sequence":
        return run_sequence(args)
    if args.workload == "gmm":
        return run_gmm(args)
    if args.workload == "larger-than-hbm":
        return run_larger_than_hbm(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1802_05421_gb300 import build as B
    B.build()
    from paper_1802_05421_gb300 import cdl

    wl = make_workload()
    n, T = wl.X[0].shape
    stream = torch.cuda.Stream()
    st, ctx = cdl.cdl_ctx_create(local, stream.cuda_stream, 0)
    assert st == 0, cdl.cdl_status_string(st)
    chain = {"bf16": cdl.CDL_BF16, "fp8": cdl.CDL_FP8E4M3, "fp8t": cdl.CDL_FP8E4M3_T128, "f32": cdl.CDL_F32,
             "f64": cdl.CDL_F64}[args.chain]
    score = cdl.CDL_F64 if args.chain == "f64" else (cdl.CDL_BF16 if args.score == "bf16" else cdl.CDL_F32)
    score_name = {cdl.CDL_F64: "f64", cdl.CDL_F32: "f32", cdl.CDL_BF16: "bf16"}[score]
    X1 = torch.from_numpy(wl.X[0]).cuda()
    X2 = torch.from_numpy(wl.X[1]).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    top = torch.empty(TOPK, dtype=torch.int64, device="cuda")
    opts = cdl.cdl_pair_opts(K_PROJ, D_CHAIN, chain, score, SEED, 0.0,
                             cdl.cdl_solve_opts(40, REL_TOL, 0), TOPK, 0)
    s1, s2 = cdl.cdl_solve_stats(), cdl.cdl_solve_stats()

    def step(o=opts, x1=X1, x2=X2, f=F, t=top):
        r = cdl.cdl_caddelag_pair(ctx, x1, x2, n, T, o, f, t, s1, s2)
        if r != 0:
            raise RuntimeError(f"cdl_caddelag_pair: {cdl.cdl_status_string(r)} {cdl.cdl_last_error_detail()}")

    torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    assert cdl.cdl_sync(ctx) == 0
    cdl.cdl_ctx_reset_counters(ctx)
    cdl.cdl_ctx_set_timing(ctx, True)
    sampler = ClockSampler(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = ev0.elapsed_time(ev1) / args.steps
    _, launches = cdl.cdl_ctx_launch_count(ctx)
    kc = {}
    for i, name in enumerate(cdl.KERNEL_CLASSES):
        _, ms, cnt, work = cdl.cdl_ctx_timing(ctx, i)
        kc[name] = dict(ms_per_step=ms / args.steps, launches=cnt // args.steps, work=work / max(cnt, 1),
                        ms_per_launch=ms / max(cnt, 1))
    cdl.cdl_ctx_set_timing(ctx, False)
    iters = (s1.iters, s2.iters)
    rel_res = max(s1.rel_res, s2.rel_res)

    # end to end through the C ABI with pinned host buffers
    h1 = torch.from_numpy(wl.X[0]).pin_memory()
    h2 = torch.from_numpy(wl.X[1]).pin_memory()
    hF = torch.empty(n, dtype=torch.float64).pin_memory()
    htop = torch.empty(TOPK, dtype=torch.int64).pin_memory()
    o2 = cdl.cdl_pair_opts(K_PROJ, D_CHAIN, chain, score, SEED, 0.0, cdl.cdl_solve_opts(40, REL_TOL, 0), TOPK, 1)
    step(o2, h1.data_ptr(), h2.data_ptr(), hF.data_ptr(), htop.data_ptr())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        step(o2, h1.data_ptr(), h2.data_ptr(), hF.data_ptr(), htop.data_ptr())
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    same_top = htop.tolist() == top.cpu().tolist()

    # plain float32 GPU path on the same pair (comparison of the metric)
    f32 = None
    if args.compare_f32 and args.chain == "bf16":
        of = cdl.cdl_pair_opts(K_PROJ, D_CHAIN, cdl.CDL_F32, cdl.CDL_F32, SEED, 0.0,
                               cdl.cdl_solve_opts(40, REL_TOL, 0), TOPK, 0)
        Ff = torch.empty(n, dtype=torch.float64, device="cuda")
        tf = torch.empty(TOPK, dtype=torch.int64, device="cuda")
        step(of, X1, X2, Ff, tf)   # warm-up (allocates the float32 chain)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(of, X1, X2, Ff, tf)
        e1.record(stream)
        torch.cuda.synchronize()
        f32_ms = e0.elapsed_time(e1)
        rel = float(((Ff - F).abs() / F).max())
        f32 = {"value": 1000.0 / f32_ms, "unit": "pairs/s", "ms_per_step": f32_ms, "steps": 1, "warmup": 1,
               "same_top": tf.cpu().tolist() == top.cpu().tolist(), "max_rel_diff_F_vs_bf16": rel}

    # e4m3 chain with 128 x 128 tile scales on the same pair
    fp8t = None
    if args.compare_f32 and args.chain == "bf16":
        o8 = cdl.cdl_pair_opts(K_PROJ, D_CHAIN, cdl.CDL_FP8E4M3_T128, score, SEED, 0.0,
                               cdl.cdl_solve_opts(40, REL_TOL, 0), TOPK, 0)
        F8 = torch.empty(n, dtype=torch.float64, device="cuda")
        t8 = torch.empty(TOPK, dtype=torch.int64, device="cuda")
        step(o8, X1, X2, F8, t8)   # warm-up (allocates the e4m3 chain)
        cdl.cdl_ctx_reset_counters(ctx)
        cdl.cdl_ctx_set_timing(ctx, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(o8, X1, X2, F8, t8)
        e1.record(stream)
        torch.cuda.synchronize()
        _, sq_ms, sq_cnt, sq_work = cdl.cdl_ctx_timing(ctx, cdl.CDL_KC_SQUARE)
        cdl.cdl_ctx_set_timing(ctx, False)
        f8_ms = e0.elapsed_time(e1)
        pk8, _ = peaks()
        peak8 = 2.0 * pk8.get("bf16_tflops_sustained", pk8.get("bf16_tflops"))
        ach8 = (sq_work / max(sq_cnt, 1)) / (sq_ms / max(sq_cnt, 1) * 1e-3) / 1e12 if sq_ms else 0.0
        fp8t = {"value": 1000.0 / f8_ms, "unit": "pairs/s", "ms_per_step": f8_ms, "steps": 1, "warmup": 1,
                "solve_iters": [s1.iters, s2.iters], "rel_res": max(s1.rel_res, s2.rel_res),
                "same_top": t8.cpu().tolist() == top.cpu().tolist(),
                "max_rel_diff_F_vs_bf16": float(((F8 - F).abs() / F).max()),
                "square_ms_per_launch": sq_ms / max(sq_cnt, 1),
                "square_roofline": {"kernel": "k_tc_mx8", "achieved": ach8, "peak": peak8, "unit": "TFLOP/s",
                                    "frac": ach8 / peak8,
                                    "peak_source": "2 x measured bf16_tflops_sustained (nominal e4m3/bf16 ratio)"}}

    # opt-in chain truncation (levels whose row sums fall to 2^-24 are not formed)
    trunc = None
    if args.compare_f32 and args.chain == "bf16":
        ot = cdl.cdl_pair_opts(K_PROJ, D_CHAIN, cdl.CDL_BF16, score, SEED, 0.0,
                               cdl.cdl_solve_opts(40, REL_TOL, 0), TOPK, 0, cdl.CDL_CHAIN_TRUNCATE)
        Ft = torch.empty(n, dtype=torch.float64, device="cuda")
        tt = torch.empty(TOPK, dtype=torch.int64, device="cuda")
        step(ot, X1, X2, Ft, tt)   # warm-up
        cdl.cdl_ctx_reset_counters(ctx)
        cdl.cdl_ctx_set_timing(ctx, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(ot, X1, X2, Ft, tt)
        e1.record(stream)
        torch.cuda.synchronize()
        _, _, sq_cnt, _ = cdl.cdl_ctx_timing(ctx, cdl.CDL_KC_SQUARE)
        cdl.cdl_ctx_set_timing(ctx, False)
        t_ms = e0.elapsed_time(e1)
        trunc = {"value": 1000.0 / t_ms, "unit": "pairs/s", "ms_per_step": t_ms, "steps": 1, "warmup": 1,
                 "squarings_per_pair": int(sq_cnt), "configured_squarings_per_pair": 2 * (D_CHAIN - 1),
                 "solve_iters": [s1.iters, s2.iters], "rel_res": max(s1.rel_res, s2.rel_res),
                 "same_top": tt.cpu().tolist() == top.cpu().tolist(),
                 "max_rel_diff_F_vs_full_chain": float(((Ft - F).abs() / F).max())}

    # the small pair (n = 1024, T = 64, k = 32, d = 8) on the float64 path, whole
    c1 = None
    if args.compare_f32 and args.chain == "bf16":
        from workloads import iid_pair
        w1 = iid_pair(1024, 64, 10, seed=0)
        x1s, x2s = torch.from_numpy(w1.X[0]).cuda(), torch.from_numpy(w1.X[1]).cuda()
        F1 = torch.empty(1024, dtype=torch.float64, device="cuda")
        t1 = torch.empty(TOPK, dtype=torch.int64, device="cuda")
        o1 = cdl.cdl_pair_opts(32, 8, cdl.CDL_F64, cdl.CDL_F64, 0, 0.0, cdl.cdl_solve_opts(40, REL_TOL, 0), TOPK, 0)
        ctx1 = cdl.cdl_ctx_create(local, stream.cuda_stream, 0)[1]
        for _ in range(3):
            r = cdl.cdl_caddelag_pair(ctx1, x1s, x2s, 1024, 64, o1, F1, t1, s1, s2)
            assert r == 0, cdl.cdl_status_string(r)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            cdl.cdl_caddelag_pair(ctx1, x1s, x2s, 1024, 64, o1, F1, t1, s1, s2)
        e1.record(stream)
        torch.cuda.synchronize()
        cdl.cdl_ctx_destroy(ctx1)
        c1 = {"workload": "iid_n1024 (n = 1024, T = 64, k = 32, d = 8, float64 chain and scores, top-10)",
              "ms_per_pair": e0.elapsed_time(e1) / 5, "top": t1.cpu().tolist()}

    # the batched form (64 ragged pairs), a shorter run of --workload batched
    batched = None
    if args.compare_f32 and args.chain == "bf16":
        b = batched_measure(5, 3, 1, dist, world, local, sample_clocks=False)
        batched = {k: b[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "config",
                                     "roofline", "e2e", "gpu_launches", "autotuner")}

    # max over ranks
    step_ms, e2e_s = rank_max([step_ms, e2e_s], dist, "cuda")
    value = pairs_per_second(step_ms, world)

    if rank == 0:
        pk, src = peaks()
        sq = kc["square"]
        achieved = sq["work"] / (sq["ms_per_launch"] * 1e-3) / 1e12 if sq["ms_per_launch"] else 0.0
        peak = None
        if args.chain == "bf16":
            peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        elif args.chain in ("fp8", "fp8t"):   # measured bf16 peak x the nominal fp8/bf16 dense ratio (4.5 / 2.25)
            peak = 2.0 * pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        kname = {"bf16": "k_tc_sq2", "fp8": "k_tc_gemm<fp8>", "fp8t": "k_tc_mx8"}.get(args.chain, "k_gemm_tn")
        roof = {"kernel": kname + " (chain squaring)",
                "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if peak else None,
                "traffic": square_traffic() if args.chain == "bf16" else None,
                "peak_source": f"{src} bf16_tflops_sustained (kernel timed inside a long step)",
                "work_per_launch": sq["work"], "ms_per_launch": sq["ms_per_launch"]}
        cpu = None
        if not args.no_cpu_baseline:
            sec, desc, phases = oracle_sample(wl)
            cpu = {"value": 1.0 / sec, "unit": "pairs/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": desc, "seconds_per_pair": sec, "value_basis": "extrapolated from the sample",
                   "phases_s": {k: round(v, 2) for k, v in phases.items()}}
            c1_sec, c1_top, _ = oracle_full_pair_n1024()
            cpu["measured_full_pair_n1024"] = {"workload": "iid_n1024 (n = 1024, T = 64, k = 32, top-10, "
                                                           "exact embeddings)",
                                               "seconds": c1_sec, "pairs_per_s": 1.0 / c1_sec}
            if c1 is not None:
                c1["oracle_s"] = c1_sec
                c1["same_top_as_oracle"] = c1["top"] == c1_top
        props = torch.cuda.get_device_properties(local)
        phases_roof = phase_rooflines(kc, n, pk, src, props.multi_processor_count,
                                      float(pk.get("sm_max_mhz", 2070.0)))
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.chain, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "T": T, "k": K_PROJ, "d": D_CHAIN, "topk": TOPK,
                       "chain": args.chain, "score": score_name,
                       "refine_rel_tol": REL_TOL, "solve_iters": list(iters), "rel_res": rel_res,
                       "parallelism": f"replicas x{world}",
                       "l2": "no flush: each step streams two 8.6 GB float64 graphs and 30 GB of "
                             "chain levels, far larger than the 129 MB L2"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "phase_rooflines": phases_roof,
            "f32_path": f32,
            "fp8_tile_path": fp8t,
            "truncated_chain_path": trunc,
            "batched_path": batched,
            "small_pair_f64_path": c1,
            "e2e": {"value": pairs_per_second(e2e_s * 1000.0, world), "unit": "pairs/s",
                    "h2d_bytes_per_step": 2 * n * T * 8,
                    "d2h_bytes_per_step": n * 8 + TOPK * 8, "same_top_as_device_run": same_top},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "phases_ms_per_step": {k: round(v["ms_per_step"], 3) for k, v in kc.items()},
        }
        print(json.dumps(line), flush=True)
    cdl.cdl_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark: steady nonlinear ship-wave solves on the 181x61 mesh.

Workload: 181 x 61 half-mesh on x in [-16, 20], y in [0, 12] (dx = dy = 0.2),
F = 0.7, eps = 0.4, flat initial guess, GMRES restart 30.  One step is one
complete solve: preconditioner set-up, Newton-GMRES with the FP32 all-pairs
residual, and the FP64 residual refinement down to ||E_fp64||_inf < 1e-9
(the mixed-precision solve).  The plain FP64 solve of the same workload is
timed beside it and every mixed result is compared with it and with the
stored oracle root (max |d zeta|, max |d phi|).

After the timed steps the default run also reports, outside the headline:
the exact-JVP solve; the 64 x 121x41 batch (mixed and FP64, sampled
instances against stored oracle roots); the serving workload (mixed: 256
Poisson requests at the saturated rate, 1.0x and 0.5x of it; FP64, about 37x
slower per request: 16 requests at its saturated rate and 1.0x); and one
721x241 solve (eps = 0.8) with its root refined further on FP64 residuals.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its
own replica of the workload (independent solves; there is no data exchange)
and the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ship-wave solve 181x61, F=0.7, eps=0.4 (x in [-16,20], y in [0,12], dx=dy=0.2)"
METRIC = "solves/s (mixed FP32-residual solve refined to FP64, max|dzeta| vs FP64 solve <= 1e-6)"
FLOP_PER_PAIR = 44          # FP32 operations per (source, target) pair, FFMA counted as 2
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2        # B300: FP64 at 1/64 of the FP32 rate
SM_COUNT_B300 = 148
SM_MAX_MHZ = 2032.0
# residual evaluations of one FP64 Newton-GMRES solve of this workload with the
# default options (measured on the GPU path); the reference arm converts the
# oracle's residual time into solves/s with it
RESIDUALS_PER_SOLVE = 21
# committed ncu summary of the FP32 all-pairs kernel's DRAM traffic per tile shape
# (its header records the hash of the kernel source it was captured from)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_pairs_fp32_traffic_181x61.txt")
KERNEL_SOURCE = os.path.join(ROOT, "paper_1403_5044_b300", "csrc", "pairs.cu")
ORACLE_ROOT_181x61 = os.path.join(ROOT, "tests", "golden", "oracle_root_181x61.txt")
ORACLE_ROOT_BATCH = os.path.join(ROOT, "tests", "golden", "oracle_root_121x41_batch.txt")
BLOCK_BW = 15          # block bandwidth of the mixed solves (fastest measured at 181x61)
FP64_BLOCK_BW = 15     # the FP64 solve's own fastest block bandwidth


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block-bw", type=int, default=BLOCK_BW)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp64-block-bw", type=int, default=FP64_BLOCK_BW)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-requests", type=int, default=None,
                    help="requests per rate point of the mixed serving block (default 256, 2000 with --serve; "
                         "0 = skip it)")
    ap.add_argument("--serve-requests-fp64", type=int, default=None,
                    help="requests per rate point of the FP64 serving block (default 16, 64 with --serve; "
                         "0 = skip it)")
    ap.add_argument("--large-steps", type=int, default=1,
                    help="721x241 solves in the default run (0 = skip them)")
    ap.add_argument("--serve", action="store_true",
                    help="only the serving workload: 2000 Poisson requests per rate, rates swept over "
                         "{0.25, 0.5, 0.75, 1.0, 1.25} x the measured saturated rate, mixed and FP64")
    ap.add_argument("--serve-rates", default="0.25,0.5,0.75,1.0,1.25",
                    help="--serve: rate factors of the mixed block (x its saturated rate)")
    ap.add_argument("--serve-rates-fp64", default="0.5,1.0",
                    help="--serve: rate factors of the FP64 block (x its own saturated rate)")
    ap.add_argument("--large", action="store_true",
                    help="only the 721x241 workload (F = 0.7, eps = 0.8): one mixed solve from the flat "
                         "guess, reported with its counters (minutes)")
    ap.add_argument("--batch-steps", type=int, default=2,
                    help="timed steps of the 64 x 121x41 batched workload (0 = skip it)")
    ap.add_argument("--mesh", default="181x61",
                    help="--precond-only: mesh NxM on x in [-16,20], y in [0,12] (F = 0.7, eps = 0.3 "
                         "unless 181x61, the workload)")
    ap.add_argument("--lu-products", type=int, default=None,
                    help="block products of the band LU: 0 FP64 kernel, 1 bf16 slices on the tensor cores "
                         "(default: the library's)")
    ap.add_argument("--jvp-only", action="store_true",
                    help="exact Jacobian-vector products of the 181x61 workload only (FP32 and FP64, timed)")
    ap.add_argument("--spectrum", action="store_true",
                    help="spectral diagnostics of J P^-1 (41x21, F = 0.7, eps = 0.1, at the root) for several b")
    ap.add_argument("--precond-only", action="store_true",
                    help="build the preconditioner, apply it 10 times and solve once "
                         "(a small, fixed launch sequence for profilers)")
    ap.add_argument("--residual-only", action="store_true",
                    help="only evaluate the FP32 and FP64 residual of the workload `steps` times "
                         "(a small, fixed launch sequence for profilers)")
    return ap.parse_args()


def dist_init(n, backend="nccl"):
    """One process per GPU under torchrun (RANK, LOCAL_RANK, WORLD_SIZE and
    MASTER_* from the environment); (0, 1, None) for a single process."""
    import torch
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    if backend == "nccl":
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), dist


def replica_rate(total_ms, solves_per_rank, world, dist, device="cuda"):
    """Whole-job rate of `world` independent replicas (no data-path
    collective; weak scaling): every rank's solves over the slowest rank's
    time.  Returns (solves/s, max total ms)."""
    import torch
    if dist is not None:
        t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * solves_per_rank / (total_ms / 1e3), total_ms


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_hash(path):
    """First 16 hex digits of the SHA-256 of a file (identifies a kernel build)."""
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic(shape):
    """DRAM bytes (read + write) per launch of one tile shape of the FP32
    all-pairs kernel, from the committed ncu summary: lines
    '<shape> <bytes>' under a header 'source_sha256_16 <hash>'.  None when
    the shape was not captured or the kernel source changed since."""
    try:
        with open(TRAFFIC_FILE) as f:
            lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None, "no traffic summary"
    table = {ln[0]: ln[1] for ln in lines if len(ln) == 2}
    if table.get("source_sha256_16") != source_hash(KERNEL_SOURCE):
        return None, "kernel source changed since the ncu capture"
    if shape not in table:
        return None, "shape not in the ncu capture"
    return int(table[shape]), "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch of this shape"


def load_roots(path):
    """Stored oracle roots: list of (header dict, zeta [M][N], phi [M][N] or
    None when the file holds zeta alone)."""
    import numpy as np
    blocks = []
    with open(path) as f:
        for line in f:
            if line.startswith("# instance"):
                head, rest = line[2:].split(":", 1)
                words = rest.split()
                N, M = (int(v) for v in words[1].split("x"))
                kv = {k: float(v) for k, v in (w.split("=") for w in words[2:])}
                blocks.append({"label": head.split()[1], "N": N, "M": M, **kv, "rows": []})
            elif line.startswith("# newton_iterations") and blocks:
                blocks[-1].update({k: float(v) for k, v in (t.split("=") for t in line[2:].split())})
            elif not line.startswith("#") and line.strip():
                blocks[-1]["rows"].append([float(v) for v in line.split()])
    out = []
    for b in blocks:
        a = np.array(b.pop("rows")).reshape(b["M"] * b["N"], -1)
        out.append((b, a[:, 0].reshape(b["M"], b["N"]),
                    a[:, 1].reshape(b["M"], b["N"]) if a.shape[1] > 1 else None))
    return out


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_oracle_residual_rate(seconds):
    """Time the oracle's full FP64 residual of the workload on the host cores;
    returns (seconds per residual, evaluations, cores)."""
    import oracle as O
    from paper_1403_5044_b300 import workloads as W
    spec, F, eps = W.SOLVE_181x61
    m = O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
    u = W.random_state(spec, seed=3, amp=0.05)
    O.residual(m, F, eps, u)  # compile / warm
    n, t0 = 0, time.perf_counter()
    while True:
        O.residual(m, F, eps, u)
        n += 1
        if time.perf_counter() - t0 >= seconds or n >= 50:
            break
    dt = (time.perf_counter() - t0) / n
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dt, n, cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1403_5044_b300 import workloads as W
    spec = W.SOLVE_181x61[0]
    per = []
    for _ in range(args.warmup + args.steps):
        dt, n, cores = cpu_oracle_residual_rate(0.0)
        per.append(dt)
    per = per[args.warmup:]
    t_res = sum(per) / len(per)
    solves_s = 1.0 / (t_res * RESIDUALS_PER_SOLVE)
    sample = ("a projection, not a timed solve: each step times one full oracle FP64 residual of the "
              "181x61 workload (%d pairs) on %d host threads; solves/s = 1 / (t_residual x %d residual "
              "evaluations per solve); the oracle's own LU and Krylov work is not counted"
              % (spec.pairs, cores, RESIDUALS_PER_SOLVE))
    out = {"impl": "reference", "metric": METRIC, "value": solves_s, "unit": "solves/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": t_res * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "impl": "CPU oracle (numpy + plain C, OpenMP)"},
           "cpu_baseline": {"value": solves_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": sample, "cpu_model": cpu_model()},
           "e2e": {"value": solves_s, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "residual_pairs_per_s": spec.pairs / t_res}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    from paper_1403_5044_b300 import swj
    from paper_1403_5044_b300 import workloads as W

    rank, world, dist = dist_init(args.gpus)
    if world == 1:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    spec, F, eps = W.SOLVE_181x61
    stream = torch.cuda.current_stream()
    ctx = swj.Context.from_spec(spec, F, eps, solve_mode="mixed", block_bw=args.block_bw, stream=stream)
    u = ctx.vector()
    zeta = torch.empty(spec.N * spec.M, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    mid = []   # events between the set-up and the Newton-GMRES phase of each timed step

    def solve_once(ev_mid=None):
        # a whole solve: preconditioner set-up (it depends on the mesh and F only, but
        # every step rebuilds it) + Newton-GMRES + FP64 refinement
        ctx.initial_guess_flat(u)
        ctx.precond_setup()
        if ev_mid is not None:
            ev_mid.record(stream)
        return ctx.solve(u)

    for _ in range(args.warmup):
        solve_once()
    ctx.sync()

    # ---- timed region: K mixed solves (L2 flushed before each, outside the step time)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    ctx.set_kernel_timing(True)
    launches0 = swj.kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        # NVTX range "timed": `ncu --nvtx --nvtx-include timed/` lists only these launches
        torch.cuda.nvtx.range_push("timed")
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            mid.append(torch.cuda.Event(enable_timing=True))
            stats.append(solve_once(mid[-1]))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        torch.cuda.nvtx.range_pop()
    launches = swj.kernel_launches() - launches0
    pair_ms, pair_n = ctx.pair_timing(swj.FP32)
    pair_name = swj.pair_variant_name(swj.FP32, ctx.pair_config(swj.FP32)[0])
    traffic, traffic_note = measured_traffic(pair_name)
    pair64_ms, pair64_n = ctx.pair_timing(swj.FP64)
    ctx.set_kernel_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    setup_ms = [a.elapsed_time(m) for (a, _), m in zip(ev, mid)]
    value, total_ms = replica_rate(sum(step_ms), args.steps, world, dist)
    phi = torch.empty_like(zeta)
    ctx.unpack(u, zeta, phi)
    ctx.sync()
    zeta_mixed, phi_mixed = zeta.cpu().numpy(), phi.cpu().numpy()

    # ---- plain FP64 solve of the same workload (reference for max|dzeta| and its own rate)
    ctx64 = swj.Context.from_spec(spec, F, eps, solve_mode="fp64", block_bw=args.fp64_block_bw, stream=stream)
    u64 = ctx64.vector()
    t64 = []
    st64 = None
    for k in range(max(1, args.fp64_steps)):
        flush.fill_(-1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx64.initial_guess_flat(u64)
        ctx64.precond_setup()
        st64 = ctx64.solve(u64)
        b.record(stream)
        torch.cuda.synchronize()
        t64.append(a.elapsed_time(b))
    ctx64.unpack(u64, zeta, phi)
    ctx64.sync()
    zeta64, phi64 = zeta.cpu().numpy(), phi.cpu().numpy()
    dzeta = float(np.abs(zeta_mixed - zeta64).max())
    vs_oracle = None
    if os.path.exists(ORACLE_ROOT_181x61):
        head, zo, po = load_roots(ORACLE_ROOT_181x61)[0]
        zo, po = zo.ravel(), po.ravel()
        vs_oracle = {"root": "oracle Newton-GMRES root, ||E||_inf %.1e (stored, written by the oracle only)"
                             % head["final_norm_inf"],
                     "max_abs_dzeta_mixed": float(np.abs(zeta_mixed - zo).max()),
                     "max_abs_dphi_mixed": float(np.abs(phi_mixed - po).max()),
                     "max_abs_dzeta_fp64": float(np.abs(zeta64 - zo).max()),
                     "max_abs_dphi_fp64": float(np.abs(phi64 - po).max())}

    # ---- end to end through the C ABI with host buffers: swj_solve_host copies the
    # pinned host initial guess in, rebuilds the preconditioner, solves, and copies
    # the surface zeta back to pinned host memory, all inside the timed region
    u_host = torch.empty(ctx.n_unknowns, dtype=torch.float64).pin_memory()
    u_host.copy_(torch.from_numpy(W.flat_state(spec)))
    z_host = torch.empty(spec.N * spec.M, dtype=torch.float64).pin_memory()
    # untimed warm-up through the same call (its first use allocates the staging buffer)
    for _ in range(max(1, min(args.warmup, 2))):
        ctx.solve_host(u_host, True, None, z_host, None)
    torch.cuda.synchronize()
    e2e_ms = []
    if dist:
        dist.barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.solve_host(u_host, True, None, z_host, None)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_dz = float(np.abs(z_host.numpy() - zeta_mixed).max())
    e2e_value, _ = replica_rate(sum(e2e_ms), args.steps, world, dist)

    exact = exact_jvp_section(spec, F, eps, args, stream, flush, zeta_mixed) if rank == 0 else None

    batch = run_batch(args, stream, flush) if args.batch_steps > 0 else None
    serve = None
    if rank == 0 and (args.serve_requests > 0 or args.serve_requests_fp64 > 0):
        serve = {"workload": SERVE_WORKLOAD}
        if args.serve_requests > 0:
            serve["mixed"] = serve_block("mixed", args.serve_requests, [1.0, 0.5])
        if args.serve_requests_fp64 > 0:
            serve["fp64"] = serve_block("fp64", args.serve_requests_fp64, [1.0])
    large = large_section(args) if (rank == 0 and args.large_steps > 0) else None

    if rank != 0:
        return
    n_solves = world * args.steps
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pairs = spec.pairs
    avg_pair_ms = pair_ms / max(1, pair_n)
    achieved = FLOP_PER_PAIR * pairs / (avg_pair_ms * 1e-3) / 1e12
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    cs = clk.summary()
    mean = lambda xs: sum(xs) / len(xs)
    s0 = stats[-1]
    cpu = None
    if world == 1:
        dt, n, cores = cpu_oracle_residual_rate(args.cpu_seconds)
        res_per_solve = mean([s["residual_evals"] for s in stats])
        cpu = {"value": 1.0 / (dt * st64["residual_evals"]), "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": "a projection, not a timed solve: %d full oracle FP64 residuals of the 181x61 workload "
                         "were timed (%.2f s each, %.3e pairs/s) and solves/s = 1 / (t_residual x %d residual "
                         "evaluations of the FP64 solve); the oracle's own LU and Krylov work is not counted"
                         % (n, dt, pairs / dt, st64["residual_evals"]),
               "cpu_model": cpu_model(), "residual_pairs_per_s": pairs / dt}
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 all-pairs sum + f64 (mesh step, Krylov, LU, refinement)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": [spec.N, spec.M], "F": F, "eps": eps,
                   "block_bw": args.block_bw, "gmres_restart": 30, "solve": "mixed",
                   "refine_tol_inf": 1e-9, "l2": "flushed (256 MB write) before every step, outside the step time",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "latency_ms": serve_latency(serve),
        "solve_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99)),
                     "mean": mean(step_ms), "setup_mean": mean(setup_ms),
                     "newton_gmres_mean": mean(step_ms) - mean(setup_ms)},
        "solve_stats": {k: s0[k] for k in ("newton_iters", "refine_iters", "residual_evals", "residual_evals_fp64",
                                           "krylov_iters", "precond_applies", "final_norm_inf_fp64", "t_setup_ms")},
        "fp64_solve": {"value": 1e3 / mean(t64), "unit": "solves/s", "ms": mean(t64),
                       "block_bw": args.fp64_block_bw,
                       "residual_evals": st64["residual_evals"], "krylov_iters": st64["krylov_iters"],
                       "final_norm_inf": st64["final_norm_inf"]},
        "max_abs_dzeta_mixed_vs_fp64": dzeta,
        "vs_oracle_root": vs_oracle,
        "speedup_mixed_vs_fp64": value / (1e3 / mean(t64)),
        "residual_pairs_per_s": {"fp32_kernel": pairs / (avg_pair_ms * 1e-3),
                                 "fp64_kernel": pairs / (pair64_ms / max(1, pair64_n) * 1e-3) if pair64_n else None},
        "roofline": {"bound": "alu", "kernel": pair_name + " (FP32 all-pairs boundary-integral sum)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_note": "derived: %d SMs x %d FP32 lanes x 2 flop x %.0f MHz (MEASURED_PEAKS.json has no FP32 figure)"
                                  % (sms, FP32_LANES_PER_SM, SM_MAX_MHZ),
                     "flop_per_pair": FLOP_PER_PAIR, "pairs_per_launch": pairs,
                     "avg_launch_ms": avg_pair_ms, "launches_timed": pair_n,
                     "frac_at_measured_clock": (achieved / (sms * FP32_LANES_PER_SM * 2 * cs["sm_mhz"] * 1e6 / 1e12)
                                                if cs["sm_mhz"] else None),
                     "traffic": traffic, "traffic_source": traffic_note,
                     "algorithmic_bytes_per_launch": spec.N * spec.M * 32 + (spec.N - 1) * spec.M * 32},
        "roofline_fp64": ({"bound": "alu", "kernel": swj.pair_variant_name(swj.FP64, ctx.pair_config(swj.FP64)[0])
                           + " (FP64 all-pairs sum of the refinement residuals)",
                           "achieved": FLOP_PER_PAIR * pairs / (pair64_ms / pair64_n * 1e-3) / 1e12,
                           "peak": sms * FP64_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12, "unit": "TFLOP/s",
                           "frac": FLOP_PER_PAIR * pairs / (pair64_ms / pair64_n * 1e-3) / 1e12
                           / (sms * FP64_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12),
                           "peak_note": "derived: %d SMs x %d FP64 lanes x 2 flop x %.0f MHz (B300 nominal 1.25 TFLOP/s FP64)"
                                        % (sms, FP64_LANES_PER_SM, SM_MAX_MHZ),
                           "avg_launch_ms": pair64_ms / pair64_n, "launches_timed": pair64_n}
                          if pair64_n else None),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value,
                "unit": "solves/s", "h2d_bytes_per_step": ctx.n_unknowns * 8,
                "d2h_bytes_per_step": spec.N * spec.M * 8,
                "call": "swj_solve_host (C ABI, pinned host buffers in and out, preconditioner rebuilt)",
                "ms": {"p50": statistics.median(e2e_ms), "max": max(e2e_ms), "min": min(e2e_ms)},
                "max_abs_dzeta_vs_device_solve": e2e_dz},
        "gpu_launches": int(launches),
        "exact_jvp": exact,
        "batch": batch,
        "serve": serve,
        "large": large,
        "clocks": {"sm_mhz": cs["sm_mhz"], "sm_max_mhz": cs["sm_max_mhz"], "reasons": cs["reasons"]},
        "wall_s_timed": wall,
    }
    print(json.dumps(out), flush=True)


def serve_latency(serve):
    """Headline latency: the mixed serving block at 1.0 x its saturated rate."""
    if not serve or "mixed" not in serve:
        return None
    pt = [p for p in serve["mixed"]["points"] if p["rate_factor"] == 1.0][0]
    return {**pt["latency_ms"], "source": "serving workload, mixed, %d requests at 1.0 x the saturated rate"
            % pt["requests"]}


TAN_FLOP_PER_PAIR = 88   # tangent pair: 12 add + 24 mul + 26 FMA (FMA = 2) + 4 rsqrt


def exact_jvp_section(spec, F, eps, args, stream, flush, zeta_ref):
    """The exact Jacobian-vector product (swj_jvp_exact) on the 181x61 workload:
    time per product in FP32 and FP64 at a converged state, against one FP32
    residual (what an FD product costs), and a mixed solve whose GMRES uses it."""
    import numpy as np
    import torch
    from paper_1403_5044_b300 import swj
    ctx = swj.Context.from_spec(spec, F, eps, solve_mode="mixed", block_bw=args.block_bw, stream=stream,
                                jvp=swj.JVP_EXACT)
    u = ctx.initial_guess_flat(ctx.vector())
    for _ in range(args.warmup):
        ctx.initial_guess_flat(u)
        ctx.precond_setup()
        st = ctx.solve(u)
    ctx.sync()
    t = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.initial_guess_flat(u)
        ctx.precond_setup()
        st = ctx.solve(u)
        b.record(stream)
        torch.cuda.synchronize()
        t.append(a.elapsed_time(b))
    zeta = torch.empty(spec.N * spec.M, dtype=torch.float64, device="cuda")
    ctx.unpack(u, zeta, None)
    ctx.sync()
    dz = float(np.abs(zeta.cpu().numpy() - zeta_ref).max())
    v = torch.tensor(np.random.default_rng(5).normal(size=ctx.n_unknowns), device="cuda")
    J, E = ctx.vector(), ctx.vector()

    def per_call(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms32 = per_call(lambda: ctx.jvp_exact(u, v, J, swj.FP32))
    ms64 = per_call(lambda: ctx.jvp_exact(u, v, J, swj.FP64), reps=5)
    msr = per_call(lambda: ctx.residual(u, E, swj.FP32))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    ctx.close()
    return {"fp32_ms": ms32, "fp64_ms": ms64, "fp32_residual_ms": msr,
            "fp32_tflops_whole_product": TAN_FLOP_PER_PAIR * spec.pairs / (ms32 * 1e-3) / 1e12,
            "fp32_frac_whole_product": TAN_FLOP_PER_PAIR * spec.pairs / (ms32 * 1e-3) / 1e12 / peak,
            "flop_per_pair": TAN_FLOP_PER_PAIR,
            "mixed_solve": {"solves_per_s": 1e3 / (sum(t) / len(t)), "ms": sum(t) / len(t),
                            "krylov_iters": st["krylov_iters"], "exact_jvps": st["exact_jvps"],
                            "residual_evals": st["residual_evals"], "newton_iters": st["newton_iters"],
                            "final_norm_inf_fp64": st["final_norm_inf_fp64"],
                            "max_abs_dzeta_vs_fd_mixed": dz}}


def run_batch(args, stream, flush):
    """The batched workload: 64 instances of 121x41 (x in [-16, 20], y in [0, 12],
    dx = dy = 0.3), F ~ U[0.5, 1], eps ~ U[0.05, 0.6] from seed 1403_5044.  One
    step solves the whole batch from the flat guess (preconditioner set-up
    included), mixed precision; the FP64 batch is timed beside it and every
    instance's surface is compared with its FP64 one."""
    import numpy as np
    import torch
    from paper_1403_5044_b300 import swj
    from paper_1403_5044_b300 import workloads as W
    spec = W.MESH_121x41
    params = W.batch_params()
    F = [p[0] for p in params]
    eps = [p[1] for p in params]
    out = {"workload": "64 x 121x41, F ~ U[0.5,1], eps ~ U[0.05,0.6] (seed 1403_5044), block_bw %d" % BLOCK_BW,
           "instances": len(F)}
    zeta = {}
    for mode, steps in (("mixed", args.batch_steps), ("fp64", 1)):
        ctx = swj.BatchContext.from_spec(spec, F, eps, solve_mode=mode, block_bw=BLOCK_BW, stream=stream)
        u = ctx.vector()

        def once():
            ctx.initial_guess_flat(u)
            ctx.precond_setup()
            return ctx.solve(u, check=False)
        once()                          # warm-up: captures the Arnoldi graphs
        ctx.sync()
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rc, st = once()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        z = torch.empty(ctx.count * spec.N * spec.M, dtype=torch.float64, device="cuda")
        ctx.unpack(u, z, None)
        ctx.sync()
        zeta[mode] = z.view(ctx.count, -1).cpu().numpy()
        conv = sum(1 for s in st if s["status"] == swj.OK)
        res = [s["residual_evals"] for s in st]
        out[mode] = {"solves_per_s": len(F) * 1e3 / (sum(ms) / len(ms)), "ms_per_batch": sum(ms) / len(ms),
                     "steps": steps, "converged": conv, "rc": rc,
                     "residual_evals_max": max(res), "residual_evals_mean": sum(res) / len(res),
                     "effective_pairs_per_s": sum(res) * spec.pairs / (sum(ms) / len(ms) / 1e3)}
        ctx.close()
    out["max_abs_dzeta_mixed_vs_fp64"] = float(np.abs(zeta["mixed"] - zeta["fp64"]).max())
    if os.path.exists(ORACLE_ROOT_BATCH):
        roots = load_roots(ORACLE_ROOT_BATCH)
        idx = [int(h["label"]) for h, _, _ in roots]
        zo = np.stack([z.ravel() for _, z, _ in roots])
        out["vs_oracle_root"] = {"instances": idx,
                                 "max_abs_dzeta_mixed": float(np.abs(zeta["mixed"][idx] - zo).max()),
                                 "max_abs_dzeta_fp64": float(np.abs(zeta["fp64"][idx] - zo).max())}
    out["speedup_mixed_vs_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


SERVE_WORKLOAD = ("requests on meshes drawn uniformly from {61x21, 121x41, 181x61, 361x121} over "
                  "x in [-16,20], y in [0,12]; F ~ U[0.5,1], eps ~ U[0.05,0.5]; Poisson arrivals (seed 1403_5045)")


def _serve_summary(reqs, res, rate_factor, offered, span):
    import numpy as np
    from paper_1403_5044_b300 import swj
    lat = np.array([r["latency_ms"] for r in res])
    ok = sum(1 for r in res if r["rc"] == swj.OK)
    by_mesh = {}
    for (t, m, F, eps), r in zip(reqs, res):
        by_mesh.setdefault("%dx%d" % (m.N, m.M), []).append(r["latency_ms"])
    return {"rate_factor": rate_factor, "offered_solves_per_s": offered, "solves_per_s": len(res) / span,
            "requests": len(res), "converged": ok, "not_converged": len(res) - ok,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "p50_ms_by_mesh": {k: float(np.median(v)) for k, v in sorted(by_mesh.items())},
            "mean_group": float(np.mean([r["group_size"] for r in res]))}


def serve_block(mode, count, rate_factors):
    """The serving workload in one precision: `count` requests of the Poisson
    stream (seed 1403_5045) first all submitted at once (the saturated rate,
    itself a latency point), then replayed at rate_factor x that rate for each
    factor.  Latency is submit -> result on the host, measured inside the
    server; requests that did not converge are counted, never dropped."""
    import numpy as np
    from paper_1403_5044_b300 import swj
    from paper_1403_5044_b300 import workloads as W
    reqs = W.serve_requests(count=count)
    kw = dict(max_active=4, max_group=8, block_bw=-1, solve_mode=mode)   # block bandwidth by mesh
    points = []
    with swj.Server(**kw) as srv:
        # warm-up: one request per mesh (creates the kept contexts' first graphs)
        for m in W.SERVE_MESHES:
            srv.poll(srv.submit(m, 0.75, 0.25), wait=True)
        t0 = time.perf_counter()
        ids = [srv.submit(m, F, eps) for _, m, F, eps in reqs]
        srv.drain()
        span = time.perf_counter() - t0
        res = [srv.poll(i, wait=True) for i in ids]
        sat = count / span
        points.append(_serve_summary(reqs, res, "saturated", None, span))
        arrivals = np.array([t for t, *_ in reqs])
        for f in rate_factors:
            rate = f * sat
            ta_all = arrivals / arrivals[-1] * (count / rate)      # rescale the stream to `rate`
            ids = []
            t0 = time.perf_counter()
            for (t, m, F, eps), ta in zip(reqs, ta_all):
                dt = ta - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                ids.append(srv.submit(m, F, eps))
            srv.drain()
            span = time.perf_counter() - t0
            res = [srv.poll(i, wait=True) for i in ids]
            points.append(_serve_summary(reqs, res, f, rate, span))
        info = srv.info()
    return {"requests_per_point": count, "saturated_solves_per_s": sat, "points": points,
            "peak_active": info["peak_active"], "peak_bytes_held": info["peak_bytes_held"],
            "contexts_created": info["contexts_created"], "contexts_reused": info["contexts_reused"]}


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    rates = {"mixed": [float(r) for r in args.serve_rates.split(",")],
             "fp64": [float(r) for r in args.serve_rates_fp64.split(",")]}
    out = {"serve": True, "workload": SERVE_WORKLOAD}
    counts = {"mixed": args.serve_requests, "fp64": args.serve_requests_fp64}
    for mode in ("mixed", "fp64"):
        if counts[mode] > 0:
            out[mode] = serve_block(mode, counts[mode], rates[mode])
            print(json.dumps({"mode": mode, **out[mode]}), flush=True)
    print(json.dumps(out), flush=True)


def large_section(args):
    """The 721x241 workload (F = 0.7, eps = 0.8, a steep near-limiting wave):
    one mixed solve from the flat guess (FP32 Newton-GMRES, FP64 GMRES/LU,
    float-float refinement), its counters, the plain FP64 residual at its
    root, the crest against the limiting height F^2/2, and max|dzeta|
    against the same root refined further with FP64 residuals
    (refine_precision = FP64) down to ||E_fp64||_inf < 1e-11."""
    import numpy as np
    import torch
    from paper_1403_5044_b300 import swj
    from paper_1403_5044_b300 import workloads as W
    spec, F, eps = W.SOLVE_721x241
    out = {"workload": "ship-wave solve 721x241, F=0.7, eps=0.8 (x in [-16,20], y in [0,12], dx=dy=0.05)",
           "pairs_per_residual": spec.pairs}
    with swj.Context.from_spec(spec, F, eps, solve_mode="mixed", block_bw=-1) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        out["workspace_bytes"] = ctx.workspace_bytes()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.precond_setup()
        ctx.sync()
        out["setup_s"] = time.perf_counter() - t0
        st = ctx.solve(u, check=False)
        path = [eps]
        if st["rc"] != swj.OK:
            path = [0.2, 0.4, 0.6, 0.8]
            ctx.initial_guess_flat(u)
            for e in path:
                ctx.set_params(F, e)
                st = ctx.solve(u, check=False)
                if st["rc"] != swj.OK:
                    break
        ctx.sync()
        out["total_s"] = time.perf_counter() - t0
        out["eps_path"] = path
        out["solve_stats"] = {k: st[k] for k in ("rc", "newton_iters", "refine_iters", "residual_evals",
                                                 "residual_evals_ff", "krylov_iters", "final_norm_inf_fp64",
                                                 "t_total_ms")}
        E = ctx.vector()
        ctx.residual(u, E, swj.FP64)
        z, zr = (torch.empty(spec.N * spec.M, dtype=torch.float64, device="cuda") for _ in range(2))
        ctx.unpack(u, z, None)
        ctx.sync()
        out["fp64_residual_norm_inf_at_root"] = float(E.abs().max().item())
        out["max_zeta"] = float(z.max().item())
        out["crest_bound_F2_over_2"] = F * F / 2
        # the same root refined with FP64 residuals (FP32 phase skipped)
        o = swj.default_opts(solve_mode="mixed", block_bw=-1, refine_precision=swj.FP64,
                             refine_tol_inf=1e-11, mixed_tol_inf=1e300)
        ctx.set_opts(o)
        u2 = u.clone()
        t1 = time.perf_counter()
        st2 = ctx.solve(u2, check=False)
        ctx.unpack(u2, zr, None)
        ctx.sync()
        out["fp64_refined"] = {"rc": st2["rc"], "refine_iters": st2["refine_iters"],
                               "residual_evals_fp64": st2["residual_evals_fp64"],
                               "final_norm_inf_fp64": st2["final_norm_inf_fp64"],
                               "seconds": time.perf_counter() - t1,
                               "max_abs_dzeta_vs_mixed": float((z - zr).abs().max().item())}
    return out


def run_large(args):
    """Only the 721x241 workload (see large_section)."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps({"large": True, **large_section(args)}), flush=True)


def run_residual_only(args):
    """Residuals of the 181x61 workload only: every compiled tile shape of the
    all-pairs kernel pinned in turn, `steps` timed launches each (plus the
    autotuner's choice), a short fixed launch sequence for profilers."""
    import torch
    from paper_1403_5044_b300 import swj
    from paper_1403_5044_b300 import workloads as W
    spec, F, eps = W.SOLVE_181x61
    out = {"residual_only": True, "steps": args.steps, "workload": WORKLOAD, "pairs": spec.pairs, "shapes": []}
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    with swj.Context.from_spec(spec, F, eps) as ctx:
        u = torch.tensor(W.random_state(spec, seed=1, amp=0.05), device="cuda")
        E = ctx.vector()
        ctx.residual(u, E, swj.FP32)
        ctx.residual(u, E, swj.FP64)
        ctx.sync()
        ctx.residual(u, E, swj.FF)
        ctx.sync()
        out["tuned"] = {"fp32": ctx.pair_config(swj.FP32), "fp64": ctx.pair_config(swj.FP64)}
        for prec in (swj.FP32, swj.FP64, swj.FF):
            for v in range(swj.pair_variants(prec)):
                ctx.set_pair_config(prec, v)
                ctx.residual(u, E, prec)
                ctx.sync()
                ctx.set_kernel_timing(True)
                ctx.reset_pair_timing()
                for _ in range(args.steps if prec != swj.FP64 else max(1, args.steps // 10)):
                    ctx.residual(u, E, prec)
                ctx.sync()
                ms, n = ctx.pair_timing(prec)
                ctx.set_kernel_timing(False)
                _, tpb, r, packed = ctx.pair_config(prec)
                avg = ms / max(1, n)
                row = {"precision": {swj.FP32: "fp32", swj.FP64: "fp64", swj.FF: "ff"}[prec], "variant": v,
                       "name": swj.pair_variant_name(prec, v), "threads": tpb,
                       "targets_per_thread": r, "packed": packed, "avg_ms": avg,
                       "pairs_per_s": spec.pairs / (avg * 1e-3)}
                if prec == swj.FP32:
                    row["frac_fp32_peak"] = FLOP_PER_PAIR * spec.pairs / (avg * 1e-3) / 1e12 / peak
                out["shapes"].append(row)
    print(json.dumps(out))


def run_precond_only(args):
    import torch
    from paper_1403_5044_b300 import swj
    from paper_1403_5044_b300 import workloads as W
    spec, F, eps = W.SOLVE_181x61
    if args.mesh != "181x61":
        N, M = (int(v) for v in args.mesh.split("x"))
        spec, F, eps = W.domain_mesh(N, M), 0.7, 0.3
    kw = {} if args.lu_products is None else {"lu_products": args.lu_products}
    with swj.Context.from_spec(spec, F, eps, solve_mode="mixed", block_bw=args.block_bw, **kw) as ctx:
        ctx.precond_setup()             # first use: module loading and kernel attributes
        ctx.sync()
        t0 = time.perf_counter()
        ctx.precond_setup()
        ctx.sync()
        t1 = time.perf_counter()
        u = ctx.initial_guess_flat(ctx.vector())
        r = ctx.vector()
        for _ in range(3):
            ctx.precond_apply(u, r)
        ctx.sync()
        # the context's stream is torch's current stream here
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            ctx.precond_apply(u, r)
        e1.record()
        ctx.sync()
        apply_ms = e0.elapsed_time(e1) / 20
        clusters = ctx.sweep_clusters()
        st = ctx.solve(u)               # first solve: autotuning and graph capture
        ctx.initial_guess_flat(u)
        t2 = time.perf_counter()
        st = ctx.solve(u)
        t3 = time.perf_counter()
    print(json.dumps({"precond_only": True, "mesh": args.mesh, "block_bw": args.block_bw,
                      "lu_products": args.lu_products,
                      "setup_ms": (t1 - t0) * 1e3,
                      "apply_ms": apply_ms, "sweep_clusters": clusters, "solve_ms": (t3 - t2) * 1e3,
                      "krylov_iters": st["krylov_iters"], "residual_evals": st["residual_evals"]}))


def run_jvp_only(args):
    import numpy as np
    import torch
    from paper_1403_5044_b300 import swj
    from paper_1403_5044_b300 import workloads as W
    spec, F, eps = W.SOLVE_181x61
    with swj.Context.from_spec(spec, F, eps) as ctx:
        u = torch.tensor(W.random_state(spec, seed=1, amp=0.05), device="cuda")
        v = torch.tensor(np.random.default_rng(2).normal(size=ctx.n_unknowns), device="cuda")
        J = ctx.vector()
        out = {"jvp_only": True, "workload": WORKLOAD, "pairs": spec.pairs}
        for name, prec, reps in (("fp32", swj.FP32, args.steps), ("fp64", swj.FP64, max(1, args.steps // 10))):
            ctx.jvp_exact(u, v, J, prec)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                ctx.jvp_exact(u, v, J, prec)
            b.record()
            torch.cuda.synchronize()
            out[name + "_ms"] = a.elapsed_time(b) / reps
    print(json.dumps(out), flush=True)


def run_spectrum(args):
    import torch
    from paper_1403_5044_b300 import diagnostics as D
    from paper_1403_5044_b300 import swj
    from paper_1403_5044_b300 import workloads as W
    spec, F, eps = W.MESH_41x21, 0.7, 0.1
    with swj.Context.from_spec(spec, F, eps, solve_mode="fp64", block_bw=0) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        ctx.solve(u)
    for b in (1, 3, 5, 7, 11, 0):
        with swj.Context.from_spec(spec, F, eps, solve_mode="fp64", block_bw=b) as ctx:
            ctx.precond_setup()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A = D.preconditioned_jacobian(ctx, u)
            t1 = time.perf_counter()
            import numpy as np
            eigs = np.linalg.eigvals(A)
            t2 = time.perf_counter()
            print(json.dumps({"spectrum": True, "mesh": "41x21", "block_bw": b, "form_ms": (t1 - t0) * 1e3,
                              "eig_ms": (t2 - t1) * 1e3, **D.clustering(eigs),
                              "eigs_re_min": float(eigs.real.min()), "eigs_re_max": float(eigs.real.max()),
                              "eigs_im_absmax": float(np.abs(eigs.imag).max())}), flush=True)


def main():
    args = parse()
    if args.serve_requests is None:
        args.serve_requests = 2000 if args.serve else 256
    if args.serve_requests_fp64 is None:
        args.serve_requests_fp64 = 64 if args.serve else 16
    if args.spectrum:
        run_spectrum(args)
        return
    if args.jvp_only:
        run_jvp_only(args)
        return
    if args.large:
        run_large(args)
    elif args.serve:
        run_serve(args)
    elif args.precond_only:
        run_precond_only(args)
    elif args.residual_only:
        run_residual_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

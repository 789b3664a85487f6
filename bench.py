"""Benchmark of the IBIM hot path on GB300.

Step = one full solve of the Kirkwood-sphere workload (radius 20 A, 50 seeded
+-1 charges, eps_I = 2, eps_E = 80, kappa = 0.1257, h = 0.5 A, band 2h,
tau = h, about 80k nodes): right-hand side, restarted GMRES to a 1e-6
relative residual with the FP32 compensated pair-sum operator and FP64
Arnoldi/Givens on the device, then G_pol and area.  The metric is operator
(matvec) interactions per second over the whole step; each interaction is one
(target, source) pair with all four kernels evaluated.

Also reported once per run (outside the timed steps): the same solve with an
FP64-certified residual, the plain FP64 GPU solve it is compared with, the
certified solve with the full Jacobian and the tube extrapolated to tau -> 0
(its energy against the Kirkwood series), and the FP64 oracle timed on the
host cores on a bounded sample of operator rows.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (the workload does not
shard), value = interactions of all ranks / max rank time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "kirkwood_sphere", "R": 20.0, "h": 0.5, "band_k": 2, "tau_k": 1.0, "n_charges": 50,
            "charge_ball": 16.0, "eps_in": 2.0, "eps_out": 80.0, "kappa": 0.1257, "tol": 1e-6, "restart": 64}
# FP32-pipe operations (FMA/MUL/ADD lanes) per interaction of the pair
# kernel's far-field formula, counted from its source (pair_far2, two sources
# per packed instruction): r 3, |r|^2 3, s_x 3, r.(a m) 3, n.(a m) 3, rho and
# the two exponent arguments 3, E x, E - 1, g, 3 - B 5, rho^-3 1, the two
# theta terms 2, the four kernel products fused into the two sums 10.  The
# three MUFU operations (rsqrt, rcp, ex2) run on the XU pipe and are not
# counted; the per-chunk frame offsets and compensation add about 0.5.
F32_OPS_PER_INTERACTION = 36
# The symmetric variants evaluate each unordered source pair once for both
# directions: the shared part (r, |r|^2, s_x, s_y, c, rho, E, g, the series
# products, rho^-3, theta terms, hi, qf) is 28 lane-operations and each
# direction's two sums 10 more, 48 for two interactions.
F32_OPS_PER_INTERACTION_SYM = 24
# The float-float operator (IBIM_FF, pair_ff_kernel), counted from ff_pair's
# far branch: r 6, |r|^2 31, s_x, s_y and n.m 31 each, 1/rho 11, rho, kappa rho
# and the exponent argument 4 each, exp 25, E x 4, 1 - E 4, g 11, 1 - th A
# 15 twice, 3 - B 18, rho^-2 and rho^-3 8, the y1 term 31, the y2 term 54 and
# the two float-float accumulations 22 FP32-pipe operations per interaction
# (plus one MUFU, about six integer operations and five shared loads).
FF_OPS_PER_INTERACTION = 366
# The symmetric float-float kernel (pair_ffs_kernel, the default IBIM_FF kernel),
# counted from ffs_pair: 296 shared operations per unordered pair (the above up
# to rho^-3, plus the combination g c - (3 - B) s_x s_y / rho^2 27 and four
# products with the powers of 1/rho 16) and 68 per direction (the two terms 46,
# their float-float accumulation 22): 432 per unordered pair, 216 per interaction.
FFS_OPS_PER_INTERACTION = 216
FP32_LANES_PER_SM = 128
# dram__bytes_read.sum + dram__bytes_write.sum of one pair-kernel launch on this
# workload, by variant (targets/thread, min CTAs/SM, threads/CTA, symmetric scheme), from
# the ncu full-set captures summarised in profiles/pair_f32_kernel_kirkwood80k.md and
# profiles/pair_sym_kernel_kirkwood80k.md; None where the kernel changed after
# its last capture.
NCU_TRAFFIC_BYTES = {(2, 1, 512, 0): None, (2, 1, 512, 1): 7.012352e6, (2, 1, 512, 2): 7.009792e6}
METRIC = "IBIM matvec interactions/s"
L2_NOTE = ("GPU arm: a 256 MB buffer is written between timed steps (L2 is 129 MB); "
           "oracle arm: host cores, no GPU cache involved")


def reduce_over_ranks(ms, count, device):
    """Whole-job timing of independent per-rank work: (max of the ranks' times,
    sum of their counts); a plain pass-through without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(count)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(count)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def shard_molecules(costs, world_size, rank):
    """Indices of the molecules rank `rank` solves: greedy longest-first
    assignment of the costs (N_m^2) to the least loaded rank, ties to the lower
    rank; every molecule goes to exactly one rank."""
    load = [0.0] * world_size
    mine = []
    for m in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world_size), key=lambda q: (load[q], q))
        load[r] += costs[m]
        if r == rank:
            mine.append(m)
    return sorted(mine)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                smax.append(float(v[2]))
                power.append(float(v[3]))
            except ValueError:
                continue
            for n, flag in zip(names, v[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        busy = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def _kirkwood_inputs():
    from paper_1709_08070_gb300 import inputs
    W = WORKLOAD
    z, q = inputs.kirkwood_charges(W["n_charges"], W["charge_ball"])
    return z, q


def inputs_random(n, seed=3):
    from paper_1709_08070_gb300 import inputs
    return inputs.random_vector(n, seed=seed)


def _series_kcal(W):
    """Kirkwood series G_pol (kcal/mol) of a sphere workload, as stored in
    tests/golden/kirkwood_series.json by tests/golden/make_kirkwood_series.py."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "kirkwood_series.json")
    with open(path) as f:
        g = json.load(f)
    c = g["workloads"][W["workload"]]
    same = (c["R"], c["n_charges"], c["charge_ball"], g["eps_in"], g["eps_out"], g["kappa"]) == (
        W["R"], W["n_charges"], W["charge_ball"], W["eps_in"], W["eps_out"], W["kappa"])
    return c["gpol_kcal"] if same else None


def cpu_oracle_rate(target_s=10.0, max_rows=None, threads=None):
    """FP64 oracle operator rows on the host cores, bounded sample: returns
    (interactions/s, threads, sample description, elapsed).  threads: OpenMP
    threads of the oracle (None = all host cores)."""
    import oracle
    from paper_1709_08070_gb300 import inputs
    W = WORKLOAD
    all_threads = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    try:
        g = oracle.sphere_nodes(W["R"], h=W["h"], eps=W["band_k"] * W["h"])
        N = g["w"].size
        P = oracle.Phys(W["eps_in"], W["eps_out"], W["kappa"], W["tau_k"] * W["h"], 0)
        p = inputs.random_vector(2 * N, seed=3)
        probe = 256 if not threads or threads > 4 else 32
        rows = inputs.random_rows(N, probe, seed=4)
        t0 = time.perf_counter()
        oracle.matvec_rows(g["xs"], g["nrm"], g["w"], P, p, rows)
        dt = time.perf_counter() - t0
        nrows = int(min(N, max(probe, probe * target_s / max(dt, 1e-3))))
        if max_rows:
            nrows = min(nrows, max_rows)
        rows = inputs.random_rows(N, nrows, seed=5)
        t0 = time.perf_counter()
        oracle.matvec_rows(g["xs"], g["nrm"], g["w"], P, p, rows)
        dt = time.perf_counter() - t0
        used = oracle.num_threads()
    finally:
        oracle.set_num_threads(all_threads)
    return nrows * N / dt, used, "%d of %d operator rows of the %d-node workload (%d interactions)" % (
        nrows, N, N, nrows * N), dt


def kirkwood_config(N, ws):
    """The workload as both arms state it in their bench lines."""
    return dict(WORKLOAD, N=int(N), parallelism="replicas" if ws > 1 else "single", l2=L2_NOTE)


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle timed on the host cores on bounded
    row samples of the same workload (rank 0 only; it loads no CUDA code)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import build as oracle_build
    oracle_build.build()
    import oracle
    W = WORKLOAD
    N = oracle.sphere_nodes(W["R"], h=W["h"], eps=W["band_k"] * W["h"])["w"].size
    vals = []
    desc, cores = "", 0
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        v, cores, desc, dt = cpu_oracle_rate(target_s=per_step)
        if i >= args.warmup:
            vals.append((v, dt))
    value = float(np.mean([v for v, _ in vals]))
    ms = float(np.mean([dt for _, dt in vals]) * 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": kirkwood_config(N, ws),
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1709_08070_gb300 import ibim

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    W = WORKLOAD
    z, q = _kirkwood_inputs()
    h = W["h"]
    stream = torch.cuda.current_stream()
    ctx = ibim.Context.sphere(W["R"], h=h, band_eps=W["band_k"] * h)
    ctx.set_charges(z, q)
    N = ctx.N
    P = ibim.Phys(W["eps_in"], W["eps_out"], W["kappa"], W["tau_k"] * h, 0)
    variant, bps, tune_ms = ctx.autotune(P)
    tpt, minb, nthr, sym = ibim.ibim_f32_variants()[variant]
    opts = dict(precision=ibim.IBIM_F32C, tol=W["tol"], restart=W["restart"], maxit=1000, start=0, certify=0)
    dp = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.solve(P, dp, **opts)

    def timed_steps(kernel_events):
        """args.steps solves between barriers, each bracketed by CUDA events on
        the solver's stream.  kernel_events: the library also brackets every
        pair-kernel launch with events (GMRES then launches its step kernels
        directly instead of replaying the captured step graph)."""
        ctx.timing_enable(kernel_events)
        ctx.timing_reset()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        out = []
        barrier()
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("ibim_timed_steps")  # lets a profiler select exactly the timed launches
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            out.append(ctx.solve(P, dp, **opts))
            ev[i][1].record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        wall_s = time.perf_counter() - t0
        tim_ = ctx.timing()
        ctx.timing_enable(False)
        return out, [a.elapsed_time(b) for a, b in ev], tim_, wall_s

    clocks = Clocks(local)
    clocks.start()
    # the product path (graph replay): the headline value
    infos, step_ms, tim_prod, wall = timed_steps(False)
    # the same steps with the pair-kernel launches timed: the roofline
    infos_k, step_ms_k, tim, _ = timed_steps(True)
    ck = clocks.stop()
    interactions = sum(int(i["matvecs_f32"] + i["matvecs_f64"]) for i in infos) * N * N
    total_ms, interactions_all = reduce_over_ranks(float(sum(step_ms)), interactions, "cuda")
    value = interactions_all / (total_ms * 1e-3)
    inter_k = sum(int(i["matvecs_f32"] + i["matvecs_f64"]) for i in infos_k) * N * N

    # ---- dominant kernel roofline (pair_f32_kernel), live CUDA-event timing
    peaks = _peaks()
    props = torch.cuda.get_device_properties(local)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6
    # GMRES launches its Arnoldi steps in pairs between host polls, so a cycle
    # that converges on an odd step ends with one launch whose kernels see the
    # `done` flag and return at once: average over the applications that ran
    # (the solves' own operator-application counts), not over every launch.
    applied = sum(int(i["matvecs_f32"] + i["matvecs_f64"]) for i in infos_k)
    avg_pair_ms = tim["pair_ms"] / max(1, applied)
    per_launch = float(N) * float(N)
    ops_per = F32_OPS_PER_INTERACTION_SYM if sym else F32_OPS_PER_INTERACTION
    achieved_ops = ops_per * per_launch / (avg_pair_ms * 1e-3)
    roofline = {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                "frac": achieved_ops / peak_ops, "traffic": NCU_TRAFFIC_BYTES.get((tpt, minb, nthr, sym)),
                "kernel": "pair_sym_kernel" if sym else "pair_f32_kernel", "ops_per_interaction": ops_per,
                "interactions_per_launch": per_launch, "avg_launch_ms": avg_pair_ms,
                "launches_timed": int(tim["pair_launches"]), "applications_timed": applied,
                "timed_in": "a second pass of the same %d steps with a CUDA event pair around every pair-kernel "
                            "launch on the solver's stream (%.2f ms per step there, %.2f ms on the graph path; "
                            "%.4g interactions/s)" % (args.steps, float(np.mean(step_ms_k)),
                                                      float(np.mean(step_ms)),
                                                      inter_k / (sum(step_ms_k) * 1e-3)),
                "peak_basis": "%d SMs x %d FP32 lanes x %.0f MHz (max SM clock, measured peaks file)" % (
                    props.multi_processor_count, FP32_LANES_PER_SM, sm_max)}
    if ck.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved_ops / (peak_ops * ck["sm_mhz"] / sm_max)
    # the other kernel family on the same workload (one-directional when the
    # autotuner chose the symmetric kernel, and vice versa), three timed
    # operator applications, for comparison of the two fractions
    variants = ibim.ibim_f32_variants()
    alt = [v for v, info in enumerate(variants) if info[:3] == (2, 1, 512) and info[3] != sym]
    if alt:
        ctx.set_f32_variant(alt[0], 1)
        xa = torch.from_numpy(inputs_random(2 * N)).cuda()
        ya = torch.empty_like(xa)
        ctx.matvec(P, xa, ya)
        ctx.timing_enable(True)
        ctx.timing_reset()
        for _ in range(3):
            ctx.matvec(P, xa, ya)
        torch.cuda.synchronize()
        ta = ctx.timing()
        ctx.timing_enable(False)
        ctx.set_f32_variant(variant, bps)
        a_ms = ta["pair_ms"] / max(1, ta["pair_launches"])
        a_ops = F32_OPS_PER_INTERACTION_SYM if variants[alt[0]][3] else F32_OPS_PER_INTERACTION
        a_ach = a_ops * N * N / (a_ms * 1e-3)
        roofline["other_kernel"] = {"kernel": "pair_sym_kernel" if variants[alt[0]][3] else "pair_f32_kernel",
                                    "variant": alt[0], "ops_per_interaction": a_ops, "avg_launch_ms": a_ms,
                                    "achieved": a_ach / 1e12, "frac": a_ach / peak_ops,
                                    "interactions_per_s": N * N / (a_ms * 1e-3)}

    extra = {}
    if rank == 0:
        # ---- e2e through the C ABI with host buffers (pinned), per step
        zp = torch.from_numpy(np.ascontiguousarray(z)).pin_memory()
        qp = torch.from_numpy(np.ascontiguousarray(q)).pin_memory()
        hp = torch.empty(2 * N, dtype=torch.float64).pin_memory()
        e2e_ms, e2e_inter = [], 0
        for i in range(max(3, args.steps)):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, inf = ctx.solve_host(P, zp.numpy(), qp.numpy(), hp.numpy(), **opts)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_inter += int(inf["matvecs_f32"] + inf["matvecs_f64"]) * N * N
        e2e = {"value": e2e_inter / (sum(e2e_ms) * 1e-3), "unit": "interactions/s",
               "h2d_bytes_per_step": int(zp.numel() * 8 + qp.numel() * 8),
               "d2h_bytes_per_step": int(hp.numel() * 8 + 8)}
        # ---- time to 1e-6 residual: certified FP32 path vs plain FP64 GPU solve.
        # certify=1 checks the residual with the float-float operator (FP64
        # accuracy on the FP32 pipe), certify=2 with the plain FP64 operator.
        ctx.solve(P, dp, **dict(opts, certify=1))  # first use builds the float-float table
        t0 = time.perf_counter()
        icert = ctx.solve(P, dp, **dict(opts, certify=1))
        torch.cuda.synchronize()
        cert_ms = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        icert2 = ctx.solve(P, dp, **dict(opts, certify=2))
        torch.cuda.synchronize()
        cert2_ms = (time.perf_counter() - t0) * 1e3
        # the certified solve to 1e-10, below the FP32 operator's own accuracy
        # (refinement on the correction equation after the first check)
        t0 = time.perf_counter()
        itight = ctx.solve(P, dp, allow_not_converged=True, **dict(opts, tol=1e-10, maxit=1000, certify=1))
        torch.cuda.synchronize()
        tight = {"tol": 1e-10, "ms": (time.perf_counter() - t0) * 1e3, "iters": itight["iters"],
                 "relres_f64": itight["relres"], "converged": bool(itight["converged"]),
                 "fp64_accurate_applications": itight["matvecs_f64"]}
        # the two FP64-accurate operators alone (CUDA events around the pair launches)
        xa = torch.from_numpy(inputs_random(2 * N)).cuda()
        ya = torch.empty_like(xa)
        acc = {}
        for name, prec, reps, ffs in (("ffs", ibim.IBIM_FF, 3, 1), ("ff", ibim.IBIM_FF, 3, 0),
                                      ("f64", ibim.IBIM_F64, 1, 1)):
            ctx.set_ff_kernel(ffs)
            ctx.matvec(P, xa, ya, precision=prec)
            ctx.timing_enable(True)
            ctx.timing_reset()
            for _ in range(reps):
                ctx.matvec(P, xa, ya, precision=prec)
            torch.cuda.synchronize()
            tk = ctx.timing()
            ctx.timing_enable(False)
            acc[name] = tk["pair_ms"] / max(1, tk["pair_launches"])
        ctx.set_ff_kernel(1)
        ffs_ops = FFS_OPS_PER_INTERACTION * N * N / (acc["ffs"] * 1e-3)
        ff_ops = FF_OPS_PER_INTERACTION * N * N / (acc["ff"] * 1e-3)
        certifier = {"kernel": "pair_ffs_kernel", "precision": "float-float (IBIM_FF), symmetric kernel",
                     "avg_launch_ms": acc["ffs"], "interactions_per_s": N * N / (acc["ffs"] * 1e-3),
                     "ops_per_interaction": FFS_OPS_PER_INTERACTION, "achieved": ffs_ops / 1e12,
                     "frac": ffs_ops / peak_ops, "unit": "Tops/s",
                     "f64_kernel_ms": acc["f64"], "speedup_vs_f64_kernel": acc["f64"] / acc["ffs"],
                     "one_directional": {"kernel": "pair_ff_kernel", "avg_launch_ms": acc["ff"],
                                         "ops_per_interaction": FF_OPS_PER_INTERACTION,
                                         "achieved": ff_ops / 1e12, "frac": ff_ops / peak_ops}}
        fp64 = None
        if not args.skip_fp64:
            t0 = time.perf_counter()
            d64 = torch.empty_like(dp)
            i64 = ctx.solve(P, d64, **dict(opts, precision=ibim.IBIM_F64))
            torch.cuda.synchronize()
            fp64_ms = (time.perf_counter() - t0) * 1e3
            fp64 = {"ms": fp64_ms, "iters": i64["iters"], "relres": i64["relres"], "gpol_kcal": i64["gpol_kcal"]}
        Gs = _series_kcal(W)
        extra = {"time_to_residual": {
            "tol": W["tol"], "f32_step_ms": total_ms / args.steps, "f32_iters": infos[-1]["iters"],
            "f32_certified_ms": cert_ms, "f32_certified_relres_f64": icert["relres"],
            "f32_certified_iters": icert["iters"], "f32_certified_check": "float-float operator (certify=1)",
            "f32_certified_f64check_ms": cert2_ms, "f32_certified_f64check_relres": icert2["relres"],
            "f32_certified_tight": tight,
            "f64_plain": fp64,
            "speedup_certified_vs_f64": (fp64["ms"] / cert_ms) if fp64 else None,
            "speedup_certified_f64check_vs_f64": (fp64["ms"] / cert2_ms) if fp64 else None,
            "speedup_uncertified_vs_f64": (fp64["ms"] / (total_ms / args.steps)) if fp64 else None},
            "energy": {"gpol_kcal_f32": infos[-1]["gpol_kcal"], "gpol_kcal_f64": fp64["gpol_kcal"] if fp64 else None,
                       "kirkwood_series_kcal": Gs,
                       "rel_err_f32_vs_f64": abs(infos[-1]["gpol_kcal"] - fp64["gpol_kcal"]) / abs(fp64["gpol_kcal"])
                       if fp64 else None,
                       "rel_err_vs_series": abs(infos[-1]["gpol_kcal"] - Gs) / abs(Gs)},
            "certifying_operator": certifier}
        # accuracy path: full Jacobian + tube extrapolation (two certified FP32 solves)
        ctx.set_jacobian(1)
        t0 = time.perf_counter()
        ix = ctx.solve_extrapolated(P, dp, **dict(opts, certify=1))
        torch.cuda.synchronize()
        ext_s = time.perf_counter() - t0
        ctx.set_jacobian(0)
        extra["energy"]["full_jacobian_extrapolated"] = {
            "gpol_kcal": ix["gpol_kcal"], "rel_err_vs_series": abs(ix["gpol_kcal"] - Gs) / abs(Gs), "s": ext_s,
            "iters": ix["iters"], "relres_f64": ix["relres"]}
        if not args.skip_cpu:
            v, cores, desc, _ = cpu_oracle_rate(target_s=args.cpu_seconds)
            v1, c1, desc1, _ = cpu_oracle_rate(target_s=args.cpu_seconds / 2, threads=1)
            extra["cpu_baseline"] = {"value": v, "unit": "interactions/s", "cores": cores, "kind": "oracle",
                                     "sample": desc,
                                     "single_core": {"value": v1, "unit": "interactions/s", "cores": c1,
                                                     "sample": desc1}}
        if not args.skip_protein:
            extra["protein_globule"] = protein_summary(args)
        extra["e2e"] = e2e

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": kirkwood_config(N, ws),
                "f32_variant": {"index": variant, "targets_per_thread": tpt, "min_ctas_per_sm": minb,
                                "threads_per_cta": nthr, "symmetric": sym, "ctas_per_sm": bps},
                "gpu_launches": int(tim_prod["total_launches"]), "clocks": ck, "roofline": roofline,
                "wall_s_timed": wall}
        line.update(extra)
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------- other workloads
# Opt-in (--workload): the synthetic protein, the batched globules and the
# learned warm start.  Paper parameters: eps_I = 1, eps_E = 80, kappa = 0.1257,
# h = 0.5, band 2h, tau = h, probe 1.4.

PROTEIN = {"workload": "protein_globule", "atoms": 2000, "probe": 1.4, "h": 0.5, "band_k": 2, "tau_k": 1.0,
           "eps_in": 1.0, "eps_out": 80.0, "kappa": 0.1257, "tol": 1e-6, "restart": 64}


def _line(args, workload, value, ms, extra):
    line = {"metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": workload}
    line.update(extra)
    print(json.dumps(line), flush=True)


def _globule(n_atoms, seed, h=0.5, probe=1.4, atoms=None):
    """Level-set context of a seeded globule (atoms: a precomputed (z, r, q))."""
    from paper_1709_08070_gb300 import ibim, inputs
    z, r, q = atoms if atoms is not None else inputs.globule_atoms(int(n_atoms), seed=int(seed))
    return ibim.Context.molecule(z, r, q, probe=probe, h=h)


def _globule_atoms_parallel(specs):
    """inputs.globule_atoms for every (n_atoms, seed) of specs on all host cores
    (a spawned process pool, started before this process uses the GPU)."""
    import multiprocessing as mp

    from paper_1709_08070_gb300 import inputs
    specs = [(int(n), int(sd)) for n, sd in specs]
    with mp.get_context("spawn").Pool(max(1, min(os.cpu_count() or 1, 32))) as pool:
        return pool.starmap(inputs.globule_atoms, specs, chunksize=4)


def protein_summary(args, steps=3):
    """The 2,000-atom globule (level-set SES, N about 211k) as an extra key of
    the default line: geometry build time, FP32 operator interactions/s over
    `steps` timed applications (L2 flushed between them), and one certified
    FP32 solve to 1e-6 from the zero start."""
    import torch

    from paper_1709_08070_gb300 import ibim, inputs

    W = PROTEIN
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = _globule(W["atoms"], inputs.SEED_PROTEIN, W["h"], W["probe"])
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    try:
        N = ctx.N
        P = ibim.Phys(W["eps_in"], W["eps_out"], W["kappa"], W["tau_k"] * W["h"], 0)
        variant, bps, _ = ctx.autotune(P)
        stream = torch.cuda.current_stream()
        x = torch.from_numpy(inputs.random_vector(2 * N, seed=3)).cuda()
        y = torch.empty_like(x)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        ctx.matvec(P, x, y)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            ctx.matvec(P, x, y)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        d = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        info = ctx.solve(P, d, precision=ibim.IBIM_F32C, tol=W["tol"], restart=W["restart"], maxit=2000, certify=1)
        torch.cuda.synchronize()
        solve_s = time.perf_counter() - t0
        return {"config": dict(W, N=N), "geometry_build_s": build_s, "f32_variant": variant,
                "operator_interactions_per_s": N * N / (float(np.mean(ms)) * 1e-3),
                "operator_ms": float(np.mean(ms)),
                "solve_f32_certified": {"s": solve_s, "iters": info["iters"], "relres_f64": info["relres"],
                                        "converged": info["converged"], "gpol_kcal": info["gpol_kcal"],
                                        "area": info["area"], "matvecs_f32": info["matvecs_f32"],
                                        "matvecs_f64": info["matvecs_f64"]}}
    finally:
        ctx.close()


def run_protein(args):
    """2000-atom globule, level-set SES: timed FP32 operator applications and
    one certified FP32 solve to 1e-6 (the FP64 solve at this size is not run)."""
    import torch

    from paper_1709_08070_gb300 import ibim, inputs

    W = PROTEIN
    t0 = time.perf_counter()
    ctx = _globule(W["atoms"], inputs.SEED_PROTEIN, W["h"], W["probe"])
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    N = ctx.N
    P = ibim.Phys(W["eps_in"], W["eps_out"], W["kappa"], W["tau_k"] * W["h"], 0)
    variant, bps, _ = ctx.autotune(P)
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(inputs.random_vector(2 * N, seed=3)).cuda()
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.matvec(P, x, y)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        ctx.matvec(P, x, y)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    value = N * N * len(ms) / (sum(ms) * 1e-3)
    d = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    info = ctx.solve(P, d, precision=ibim.IBIM_F32C, tol=W["tol"], restart=W["restart"], maxit=2000, certify=1)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    extra = {"clocks": ck, "geometry_build_s": build_s,
             "solve_f32_certified": {"s": solve_s, "iters": info["iters"], "relres_f64": info["relres"],
                                     "converged": info["converged"], "gpol_kcal": info["gpol_kcal"],
                                     "area": info["area"], "matvecs_f32": info["matvecs_f32"],
                                     "matvecs_f64": info["matvecs_f64"]}}
    if args.protein_fp64:
        d64 = torch.empty_like(d)
        t0 = time.perf_counter()
        i64 = ctx.solve(P, d64, precision=ibim.IBIM_F64, tol=W["tol"], restart=W["restart"], maxit=2000)
        torch.cuda.synchronize()
        s64 = time.perf_counter() - t0
        extra["solve_f64_plain"] = {"s": s64, "iters": i64["iters"], "relres": i64["relres"],
                                    "converged": i64["converged"], "gpol_kcal": i64["gpol_kcal"]}
        extra["speedup_certified_vs_f64"] = s64 / solve_s
        extra["gpol_rel_diff_f32_vs_f64"] = abs(info["gpol_kcal"] - i64["gpol_kcal"]) / abs(i64["gpol_kcal"])
    cfg = dict(W, N=N, l2="256 MB buffer written between timed applications", step="one FP32 operator application",
               f32_variant={"index": variant, "ctas_per_sm": bps})
    _line(args, cfg, value, float(np.mean(ms)), extra)
    ctx.close()


TREECODE = {"workload": "kirkwood_sphere_large", "R": 60.0, "h": 0.5, "band_k": 2, "tau_k": 1.0, "n_charges": 50,
            "charge_ball": 48.0, "eps_in": 2.0, "eps_out": 80.0, "kappa": 0.1257, "tol": 1e-6, "restart": 64,
            "theta": 0.7, "target_interp": 1, "order": 6,
            "fast_setting": {"theta": 0.9, "order": 4}}


def _tc_pairs(info, order):
    """Pair evaluations of one treecode application: near steps 512 x 256,
    far steps 512 x the proxy chunks' nodes, interpolated steps order^3 x those."""
    pc = -(-order ** 3 // 32) * 32
    return (info["near_steps"] * 256 + info["far_steps"] * pc) * 512 + info["interp_steps"] * order ** 3 * pc


def run_treecode(args):
    """Kirkwood-type sphere three times the default size (R = 60 A, N = 722,830)
    with the treecode operator (IBIM_F32T, theta 0.7, target-side
    interpolation of the well-separated far clusters): timed applications, the
    direct FP32 operator timed beside it, the operator difference, and one FP32
    solve to 1e-6 with each operator, plain and certified (energies against each
    other and against the Kirkwood series).  value = N^2 x applications / time: the interactions
    of the operator the treecode approximates; pairs_per_s counts the pair
    evaluations the treecode actually performs."""
    import torch

    from paper_1709_08070_gb300 import ibim, inputs

    W = TREECODE
    h = W["h"]
    t0 = time.perf_counter()
    ctx = ibim.Context.sphere(W["R"], h=h, band_eps=W["band_k"] * h)
    z, q = inputs.kirkwood_charges(W["n_charges"], W["charge_ball"])
    ctx.set_charges(z, q)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    N = ctx.N
    P = ibim.Phys(W["eps_in"], W["eps_out"], W["kappa"], W["tau_k"] * h, 0)
    variant, bps, _ = ctx.autotune(P)
    t0 = time.perf_counter()
    ctx.treecode_setup(W["theta"], W["tau_k"] * h, W["target_interp"], W["order"])
    setup_s = time.perf_counter() - t0
    tinfo = ctx.treecode_info()
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(inputs.random_vector(2 * N, seed=3)).cuda()
    yt, yd = torch.empty_like(x), torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.matvec(P, x, yt, precision=ibim.IBIM_F32T)
    ctx.timing_enable(True)
    ctx.timing_reset()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        ctx.matvec(P, x, yt, precision=ibim.IBIM_F32T)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    tim = ctx.timing()
    ctx.timing_enable(False)
    ms = [a.elapsed_time(b) for a, b in ev]
    value = N * N * len(ms) / (sum(ms) * 1e-3)
    pairs = _tc_pairs(tinfo, W["order"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.matvec(P, x, yd)
    e0.record(stream)
    ctx.matvec(P, x, yd)
    e1.record(stream)
    torch.cuda.synchronize()
    direct_ms = e0.elapsed_time(e1)
    a, b = yd.cpu().numpy(), yt.cpu().numpy()
    op_err = [float(np.linalg.norm(b[:N] - a[:N]) / np.linalg.norm(a[:N])),
              float(np.linalg.norm(b[N:] - a[N:]) / np.linalg.norm(a[N:]))]
    d = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    solves = {}
    Gs = _series_kcal(W)
    # the faster setting (the paper's accelerator works at a 1e-4 tolerance)
    F = W["fast_setting"]
    ctx.treecode_setup(F["theta"], W["tau_k"] * h, W["target_interp"], F["order"])
    finfo = ctx.treecode_info()
    ctx.matvec(P, x, yt, precision=ibim.IBIM_F32T)
    e0.record(stream)
    for _ in range(3):
        ctx.matvec(P, x, yt, precision=ibim.IBIM_F32T)
    e1.record(stream)
    torch.cuda.synchronize()
    f_ms = e0.elapsed_time(e1) / 3
    bf = yt.cpu().numpy()
    t0 = time.perf_counter()
    finf = ctx.solve(P, d, precision=ibim.IBIM_F32T, tol=W["tol"], restart=W["restart"], maxit=1000, certify=0)
    torch.cuda.synchronize()
    f_solve = time.perf_counter() - t0
    fast = dict(F, **finfo, ms_per_application=f_ms, speedup_per_application=direct_ms / f_ms,
                operator_rel_err_vs_direct_f32=[float(np.linalg.norm(bf[:N] - a[:N]) / np.linalg.norm(a[:N])),
                                                float(np.linalg.norm(bf[N:] - a[N:]) / np.linalg.norm(a[N:]))],
                solve={"s": f_solve, "iters": finf["iters"], "relres": finf["relres"],
                       "converged": finf["converged"], "gpol_kcal": finf["gpol_kcal"],
                       "gpol_rel_err_vs_series": (finf["gpol_kcal"] - Gs) / Gs if Gs else None})
    ctx.treecode_setup(W["theta"], W["tau_k"] * h, W["target_interp"], W["order"])
    # plain FP32 solves, then certified ones (float-float residual check, refinement)
    for name, prec, cert in (("treecode", ibim.IBIM_F32T, 0), ("direct_f32", ibim.IBIM_F32C, 0),
                             ("treecode_certified", ibim.IBIM_F32T, 1), ("direct_f32_certified", ibim.IBIM_F32C, 1)):
        t0 = time.perf_counter()
        info = ctx.solve(P, d, precision=prec, tol=W["tol"], restart=W["restart"], maxit=1000, certify=cert)
        torch.cuda.synchronize()
        solves[name] = {"s": time.perf_counter() - t0, "iters": info["iters"], "relres": info["relres"],
                        "converged": info["converged"], "gpol_kcal": info["gpol_kcal"],
                        "fp64_accurate_applications": info["matvecs_f64"]}
    gt, gd = solves["treecode"]["gpol_kcal"], solves["direct_f32"]["gpol_kcal"]
    extra = {"clocks": ck, "geometry_build_s": build_s, "treecode_setup_s": setup_s,
             "treecode": dict(tinfo, theta=W["theta"], chebyshev_points_per_axis=W["order"], pairs_per_application=pairs,
                              pairs_per_s=pairs * len(ms) / (sum(ms) * 1e-3),
                              list_kernel_ms=tim["pair_ms"] / max(1, tim["pair_launches"])),
             "direct_f32_ms": direct_ms, "speedup_per_application": direct_ms / float(np.mean(ms)),
             "operator_rel_err_vs_direct_f32": op_err, "solves": solves,
             "speedup_solve": solves["direct_f32"]["s"] / solves["treecode"]["s"],
             "speedup_certified_solve": solves["direct_f32_certified"]["s"] / solves["treecode_certified"]["s"],
             "gpol_rel_diff_treecode_vs_direct": abs(gt - gd) / abs(gd), "kirkwood_series_kcal": Gs,
             "gpol_rel_err_vs_series": {"treecode": (gt - Gs) / Gs, "direct_f32": (gd - Gs) / Gs},
             "fast_setting": fast}
    cfg = dict(W, N=N, l2="256 MB buffer written between timed applications",
               step="one treecode operator application (P2M/M2M, list kernel, fixup)",
               f32_variant={"index": variant, "ctas_per_sm": bps})
    _line(args, cfg, value, float(np.mean(ms)), extra)
    ctx.close()


def run_batched(args):
    """64 globules (atoms log-uniform in [50, 3000], kappa ~ U[0, 0.2]) solved
    together by ibim_solve_batch to 1e-6; the timed step is the complete batched
    solve (every molecule converged; --batch-rounds caps the lock-step GMRES
    rounds), value = sum over molecules of operator applications x N_m^2 / time.  Under torchrun the molecules are
    independent problems: each rank solves its cost-balanced share (no
    collective on the data path), value = all ranks' interactions / the
    slowest rank's time."""
    import torch
    import torch.distributed as dist

    from paper_1709_08070_gb300 import ibim, inputs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    n_atoms, kappas = inputs.batch_sizes(args.batch_mols)
    mine = shard_molecules([float(a) ** (4.0 / 3.0) for a in n_atoms], ws, rank)  # N^2 ~ atoms^(4/3)
    t0 = time.perf_counter()
    ctxs = [_globule(n_atoms[m], inputs.SEED_BATCH + 1 + m) for m in mine]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Ns = [c.N for c in ctxs]
    physs = [ibim.Phys(1.0, 80.0, float(kappas[m]), 0.5, 0) for m in mine]
    outs = [torch.empty(2 * n, dtype=torch.float64, device="cuda") for n in Ns]
    opts = dict(precision=ibim.IBIM_F32C, tol=1e-6, restart=64, maxit=args.batch_rounds, allow_not_converged=True)
    ibim.ibim_set_batch_variant(args.batch_variant)
    for _ in range(max(1, args.warmup - 2)):
        ibim.ibim_solve_batch(ctxs, physs, outs, **dict(opts, maxit=2))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("ibim_timed_steps")
    e0.record(stream)
    infos = ibim.ibim_solve_batch(ctxs, physs, outs, **opts)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ck = clocks.stop()
    inter = sum((i["matvecs_f32"] + i["matvecs_f64"]) * n * n for i, n in zip(infos, Ns))
    ms, inter_all = reduce_over_ranks(e0.elapsed_time(e1), inter, "cuda")
    if rank == 0:
        cfg = {"workload": "batched_globules", "molecules": int(args.batch_mols),
               "molecules_rank0": len(Ns), "atoms_min": int(n_atoms.min()), "atoms_max": int(n_atoms.max()),
               "N_total_rank0": int(sum(Ns)), "N_max_rank0": int(max(Ns)),
               "sum_N2_rank0": float(sum(n * n for n in Ns)), "kappa_range": [0.0, 0.2], "h": 0.5,
               "eps_in": 1.0, "eps_out": 80.0, "rounds_cap": args.batch_rounds, "tol": 1e-6, "restart": 64,
               "parallelism": "molecules sharded over %d ranks" % ws if ws > 1 else "single",
               "step": "one complete ibim_solve_batch of every molecule to tol (at most rounds_cap lock-step "
                       "GMRES rounds)"}
        line_args = argparse.Namespace(steps=1, warmup=args.warmup)
        _line(line_args, cfg, inter_all / (ms * 1e-3), ms, {
            "n_gpus": ws, "scaling": "strong", "clocks": ck, "geometry_build_s_rank0": build_s,
            "batched_variant_rank0": ibim.ibim_batch_variants()[1],
            "batch_rank0": {"converged": int(sum(i["converged"] for i in infos)),
                            "iters_max": int(max(i["iters"] for i in infos)),
                            "iters_median": float(np.median([i["iters"] for i in infos])),
                            "interactions": float(inter)},
            "interactions_all_ranks": inter_all})
    for c in ctxs:
        c.close()
    if ws > 1:
        dist.destroy_process_group()


def run_learned(args):
    """Learned warm start: solutions of globules of learn_train_lo..hi atoms
    (batched FP32 solves, 64 molecules per batch) train the network; held-out
    globules of learn_test_atoms atoms are then solved from the zero start and
    from the network's prediction (FP32 GMRES, FP64-certified to 1e-6)."""
    import torch

    from paper_1709_08070_gb300 import ibim, inputs

    rng = np.random.default_rng(inputs.SEED_LEARNED)
    t0 = time.perf_counter()
    train_atoms = rng.integers(args.learn_train_lo, args.learn_train_hi + 1, size=args.learn_train)
    train_kappa = rng.uniform(0.0, 0.2, size=args.learn_train)
    # the training globules' atoms on the host cores first (no GPU use before the pool)
    train_sets = _globule_atoms_parallel([(train_atoms[m], inputs.SEED_LEARNED + 100 + m)
                                          for m in range(args.learn_train)])
    atoms_s = time.perf_counter() - t0
    net = ibim.WarmStartNet(seed=1)
    n_examples = 0
    for b0 in range(0, args.learn_train, 64):
        idx = range(b0, min(args.learn_train, b0 + 64))
        ctxs = [_globule(train_atoms[m], inputs.SEED_LEARNED + 100 + m, atoms=train_sets[m]) for m in idx]
        physs = [ibim.Phys(1.0, 80.0, float(train_kappa[m]), 0.5, 0) for m in idx]
        outs = [torch.empty(2 * c.N, dtype=torch.float64, device="cuda") for c in ctxs]
        infos = ibim.ibim_solve_batch(ctxs, physs, outs, precision=ibim.IBIM_F32C, tol=1e-6, restart=64,
                                      maxit=3000, allow_not_converged=True)
        for c, P, d, info in zip(ctxs, physs, outs, infos):
            if info["converged"]:
                net.add_example(c, P, d)
                n_examples += 1
            c.close()
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss0 = net.train(1, batch_nodes=8192, lr=1e-3)
    loss = net.train(args.learn_steps, batch_nodes=8192, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # FP32 + batched + warm-started vs the plain FP64 GPU solve, on held-out globules
    cmp_atoms = rng.integers(args.learn_cmp_lo, args.learn_cmp_hi + 1, size=args.learn_cmp)
    cmp_kappa = rng.uniform(0.0, 0.2, size=args.learn_cmp)
    cctx = [_globule(cmp_atoms[m], inputs.SEED_LEARNED + 20000 + m) for m in range(args.learn_cmp)]
    cphys = [ibim.Phys(1.0, 80.0, float(cmp_kappa[m]), 0.5, 0) for m in range(args.learn_cmp)]
    couts = [torch.empty(2 * c.N, dtype=torch.float64, device="cuda") for c in cctx]
    bopts = dict(precision=ibim.IBIM_F32C, tol=1e-6, restart=64, maxit=3000)
    ibim.ibim_solve_batch(cctx, cphys, couts, allow_not_converged=True, **dict(bopts, maxit=2))  # tunes variants
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ib0 = ibim.ibim_solve_batch(cctx, cphys, couts, **bopts)
    torch.cuda.synchronize()
    tb0 = time.perf_counter() - t0
    t0 = time.perf_counter()
    for c, P, o in zip(cctx, cphys, couts):
        net.predict(c, P, o)
    ibl = ibim.ibim_solve_batch(cctx, cphys, couts, start=3, **bopts)
    torch.cuda.synchronize()
    tbl = time.perf_counter() - t0
    t64, g64, res64 = 0.0, [], []
    for c, P, o in zip(cctx, cphys, couts):
        d64 = torch.empty_like(o)
        t0 = time.perf_counter()
        i64 = c.solve(P, d64, precision=ibim.IBIM_F64, tol=1e-6, restart=64, maxit=3000)
        torch.cuda.synchronize()
        t64 += time.perf_counter() - t0
        g64.append(i64["gpol"])
        g = torch.empty_like(o)
        c.rhs(1.0, g)
        ao = torch.empty_like(o)
        c.matvec(P, o, ao, precision=ibim.IBIM_F64)  # FP64 residual of the batched learned-start solution
        res64.append(float(torch.linalg.norm(g - ao) / torch.linalg.norm(g)))
    combined = {
        "molecules": int(args.learn_cmp), "atoms": [int(args.learn_cmp_lo), int(args.learn_cmp_hi)],
        "N": [int(c.N) for c in cctx], "f64_plain_s": t64, "f32_batched_zero_s": tb0,
        "f32_batched_learned_s": tbl, "speedup_vs_f64": t64 / tbl,
        "iters_zero": [int(i["iters"]) for i in ib0], "iters_learned": [int(i["iters"]) for i in ibl],
        "fp64_relres_of_learned_batched_max": max(res64),
        "gpol_rel_diff_vs_f64_max": max(abs(i["gpol"] - g) / abs(g) for i, g in zip(ibl, g64))}
    for c in cctx:
        c.close()
    tests = []
    for m in range(args.learn_test):
        ctx = _globule(args.learn_test_atoms, inputs.SEED_LEARNED + 10000 + m)
        P = ibim.Phys(1.0, 80.0, 0.1257, 0.5, 0)
        ctx.autotune(P)
        d0 = torch.empty(2 * ctx.N, dtype=torch.float64, device="cuda")
        res = {"N": ctx.N}
        for name, start in (("zero", 0), ("learned", 3)):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if start == 3:
                net.predict(ctx, P, d0)
            info = ctx.solve(P, d0, precision=ibim.IBIM_F32C, tol=1e-6, restart=64, maxit=3000, start=start,
                             certify=1)
            torch.cuda.synchronize()
            res[name] = {"s": time.perf_counter() - t1, "iters": info["iters"], "relres_f64": info["relres"],
                         "gpol_kcal": info["gpol_kcal"], "converged": info["converged"],
                         "matvecs_f64": info["matvecs_f64"]}
        res["gpol_rel_diff"] = abs(res["learned"]["gpol_kcal"] - res["zero"]["gpol_kcal"]) / abs(res["zero"]["gpol_kcal"])
        tests.append(res)
        ctx.close()
    net.close()
    z_it = sum(t["zero"]["iters"] for t in tests)
    l_it = sum(t["learned"]["iters"] for t in tests)
    z_s = sum(t["zero"]["s"] for t in tests)
    l_s = sum(t["learned"]["s"] for t in tests)
    cfg = {"workload": "learned_warm_start", "train_globules": int(args.learn_train), "train_examples": n_examples,
           "train_atoms": [int(args.learn_train_lo), int(args.learn_train_hi)], "train_steps": int(args.learn_steps),
           "test_globules": int(args.learn_test), "test_atoms": int(args.learn_test_atoms), "h": 0.5,
           "eps_in": 1.0, "eps_out": 80.0, "tol": 1e-6,
           "step": "certified FP32 solve of a held-out globule from the learned start (prediction included)"}
    line = {"metric": "GMRES iterations to 1e-6 (learned start vs zero start)", "value": l_it / max(1, len(tests)),
            "unit": "iterations per solve", "n_gpus": 1, "steps": len(tests), "warmup": 0,
            "ms_per_step": 1e3 * l_s / max(1, len(tests)), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 weights, f32+f64 solve", "data": "synthetic", "config": cfg,
            "zero_start_iters_per_solve": z_it / max(1, len(tests)),
            "iters_saved_frac": (z_it - l_it) / max(1, z_it), "time_saved_frac": (z_s - l_s) / max(1e-9, z_s),
            "train": {"examples_s": gen_s, "atoms_on_host_s": atoms_s, "train_s": train_s, "loss_first": loss0,
                      "loss_last": loss},
            "tests": tests, "batched_warm_started_vs_f64": combined}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Operator applications only (the workload's tuned FP32 pair kernel), for
    profiler captures: warm-up + steps matvecs, one short JSON line."""
    import torch

    from paper_1709_08070_gb300 import ibim, inputs

    W = WORKLOAD
    h = W["h"]
    ctx = ibim.Context.sphere(W["R"], h=h, band_eps=W["band_k"] * h)
    N = ctx.N
    P = ibim.Phys(W["eps_in"], W["eps_out"], W["kappa"], W["tau_k"] * h, 0)
    if args.variant is not None:
        ctx.set_f32_variant(args.variant, args.ctas_per_sm)
        variant, bps = args.variant, args.ctas_per_sm
    else:
        variant, bps, _ = ctx.autotune(P)
    prec = {"f32c": ibim.IBIM_F32C, "ff": ibim.IBIM_FF, "ff1": ibim.IBIM_FF, "f64": ibim.IBIM_F64}[args.prec]
    ctx.set_ff_kernel(0 if args.prec == "ff1" else 1)
    if args.treecode_theta > 0:
        ctx.treecode_setup(args.treecode_theta, W["tau_k"] * h, args.treecode_interp)
        prec = ibim.IBIM_F32T
    x = torch.from_numpy(inputs.random_vector(2 * N, seed=3)).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        ctx.matvec(P, x, y, precision=prec)
    torch.cuda.synchronize()
    ctx.timing_enable(True)
    ctx.timing_reset()
    for _ in range(args.steps):
        ctx.matvec(P, x, y, precision=prec)
    torch.cuda.synchronize()
    tim = ctx.timing()
    ctx.close()
    print(json.dumps({"mode": "profile", "N": N, "variant": variant, "ctas_per_sm": bps, "prec": args.prec,
                      "treecode_theta": args.treecode_theta,
                      "pair_ms": tim["pair_ms"] / max(1, tim["pair_launches"])}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-protein", action="store_true",
                    help="leave the 2,000-atom globule summary out of the default line")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--profile", action="store_true",
                    help="operator applications only (for profiler captures); prints no bench line")
    ap.add_argument("--variant", type=int, default=None, help="with --profile: FP32 kernel variant (no autotune)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="with --variant: CTAs per SM (0 = occupancy)")
    ap.add_argument("--prec", default="f32c", choices=["f32c", "ff", "ff1", "f64"],
                    help="with --profile: operator precision (FP32 compensated, float-float with the symmetric "
                         "kernel, float-float with the one-directional kernel, or FP64)")
    ap.add_argument("--treecode-theta", type=float, default=0.0,
                    help="with --profile: apply the treecode operator (IBIM_F32T) with this theta instead")
    ap.add_argument("--treecode-interp", type=int, default=0, choices=[0, 1],
                    help="with --treecode-theta: target-side interpolation of well-separated far clusters")
    ap.add_argument("--workload", default="kirkwood", choices=["kirkwood", "protein", "batched", "learned", "treecode"],
                    help="kirkwood (default, the headline line) or an opt-in workload")
    ap.add_argument("--protein-fp64", action="store_true",
                    help="with --workload protein: also time the plain FP64 GPU solve (about ten minutes)")
    ap.add_argument("--batch-mols", type=int, default=64)
    ap.add_argument("--batch-rounds", type=int, default=4000,
                    help="with --workload batched: cap on lock-step GMRES rounds (the default lets every molecule "
                         "converge)")
    ap.add_argument("--batch-variant", type=int, default=-1,
                    help="with --workload batched: force this batched pair-kernel variant (-1: the first-round tuning)")
    ap.add_argument("--learn-train", type=int, default=2000)
    ap.add_argument("--learn-train-lo", type=int, default=100)
    ap.add_argument("--learn-train-hi", type=int, default=1000)
    ap.add_argument("--learn-steps", type=int, default=50000)
    ap.add_argument("--learn-test", type=int, default=2)
    ap.add_argument("--learn-test-atoms", type=int, default=10000)
    ap.add_argument("--learn-cmp", type=int, default=8, help="held-out globules of the batched comparison")
    ap.add_argument("--learn-cmp-lo", type=int, default=100)
    ap.add_argument("--learn-cmp-hi", type=int, default=300)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    import __graft_entry__
    __graft_entry__.build()
    if args.profile:
        run_profile(args)
    elif args.workload == "treecode":
        run_treecode(args)
    elif args.workload == "protein":
        run_protein(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

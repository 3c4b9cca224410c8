"""Benchmark: RPY pair interactions per second during BDF2 timesteps of a
32 000-segment filament suspension on one GB300 (per GPU; weak scaling over
independent replicas when launched on several GPUs).

One step = one whole timestep of the method: initial guess (extrapolated from
past steps, by default the adaptive blend of the linear and quadratic guesses;
the learned warm start is attached when its weights were trained on the chosen
extrapolation, e.g. --extrapolation 1), J0 assembly and inversion, the
Broyden loop (each iteration: unpack, forces, RPY mobility over all S^2 pairs,
residual, J0 solve, rank-one update) and the commit. The value is the number
of RPY pair interactions evaluated in the timed steps divided by their device
time (S^2 per residual evaluation).

Workload (synthetic, seeded; shapes of the paper's 3D filament clouds):
1000 filaments x 32 segments, a = 1, dL = 2.2a, eta = 1, isotropic straight
initial filaments in a cube at 2% volume fraction (overlaps redrawn); the first
500 filaments sediment under gravity (B = L^3 W / K_B = 1000), the other 500
carry a compressive tip follower force f L^2 / K_B = 100 and no weight;
dt = T/200 with T = eta L / W; Broyden tolerance 1e-4 (||f||_inf <= tol a).
Precision (default "pair32"): FP32 pair sums with per-target compensated
accumulation; the Broyden history and updates, the J0 solves, the quaternion
steps, the state and the residual in FP64.

The default run also reports, as nested records with their own config,
roofline, clocks and FP64-oracle comparison: the initial-guess rules side by
side, the all-FP32-solve variant ("mixed"), the plain FP64 solve (the paper's
form: linear guess, J0 every step), the mobility apply alone at 3200 segments
(1000 applies), the single sedimenting filament (200 FP64 steps), the
256-system ensemble and the suspension with clamped filaments.

Output: one JSON line. --impl reference times the FP64 CPU oracle on bounded
samples of the same workload instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("RPY pair interactions/s (% FMA peak); timesteps/s at 32k segments, "
          "plain vs chosen form")
UNIT = "pair interactions/s"
EXTRAP_NAME = {1: "linear extrapolation", 2: "quadratic extrapolation",
               3: "adaptive extrapolation (linear or quadratic per filament and block)"}
# algorithmic flops of one far-field pair (FMA = 2): the fixed count of the structured
# far-field formula used as the roofline unit (the kernel itself issues ~51 FP32
# operations per pair)
FLOPS_PER_PAIR = 84
FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0
FP32_PEAK_TFLOPS = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 80.55


def workload(n_fil=1000, n_seg=32, seed=0):
    from paper_1903_12609_gb300.inputs import suspension
    return suspension(n_fil, n_seg, seed=seed)


def clocks_start():
    try:
        f = open(os.path.join(ROOT, ".bench_clocks.csv"), "w")
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def clocks_stop(handle, gpu_index):
    p, f = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    path = os.path.join(ROOT, ".bench_clocks.csv")
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    os.remove(path)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
            "reasons": sorted(reasons), "samples": len(sm)}


U32 = 2.0 ** -24
# per-component bound of the FP32 pair sums against the oracle, in units of 2^-24 B
C_MIXED = 4 * 32 + 16
PRECISION_NOTE = {
    "pair32": "RPY pair sums in FP32 with per-target compensated accumulation; Broyden history, "
              "dot products and rank-one updates, J0 solves (FP32 inverse + one FP64 "
              "refinement), quaternion exponential map, state and residual in FP64",
    "mixed": "RPY pair sums in FP32 (compensated); J0 inverse applied in FP32 without "
             "refinement; Broyden history and its dot products in FP32; state, residual, "
             "norms in FP64",
    "fp64": "every step in FP64"}


def precision_code(fil, name):
    return {"pair32": fil.FIL_PAIR32, "mixed": fil.FIL_MIXED, "fp64": fil.FIL_FP64}[name]


def suspension_positions(wl, base, t, n_fil, n_seg=32):
    return np.concatenate([base[i] + np.arange(n_seg)[:, None] * wl.dL * t[i]
                           for i in range(n_fil)])


# ---------------------------------------------------------------------------
# CPU baseline legs: the FP64 oracle timed on the host cores on a bounded
# sample. The oracle values they compute are also what the GPU results of the
# same inputs are compared with (velocity error).
# ---------------------------------------------------------------------------

def _oracle_rows_timed(Y, FT, rows, nthreads, a=1.0, eta=1.0):
    from oracle import rpy
    t0 = time.perf_counter()
    ref, B = rpy.apply_rows(Y, FT, rows, a=a, eta=eta, with_abs=True, nthreads=nthreads)
    return ref, B, time.perf_counter() - t0


def velocity_error(got, ref, B):
    """Per-component error of the GPU apply against the oracle in units of
    2^-24 B (B = the oracle's sum of |parts of M_nm| |F|, |T| per component),
    and the normwise relative error."""
    err = np.abs(got - ref)
    c = err / np.maximum(B, 1e-300) / U32
    return {"rows": int(got.shape[0]), "max_c": float(c.max()), "median_c": float(np.median(c)),
            "bound_c": C_MIXED, "within_bound": bool(np.all(err <= C_MIXED * U32 * B)),
            "normwise": float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)),
            "unit": "max/median c = |v_gpu - v_fp64| / (2^-24 B) per component"}


def cpu_baseline(Y, FT, seconds=10.0):
    """The FP64 oracle on the host cores: a bounded sample of target rows of one
    mobility apply of the same workload, scaled to pairs/s; returns the timing
    record and (rows, oracle rows, magnitude sums) for the velocity error."""
    cores = os.cpu_count() or 1
    S = Y.shape[0]
    rows = np.arange(64, dtype=np.int32)
    _, _, dt = _oracle_rows_timed(Y, FT, rows, cores)
    n = int(min(S, max(64, 64 * seconds / max(dt, 1e-4))))
    rows = np.linspace(0, S - 1, n).astype(np.int32)
    ref, B, dt = _oracle_rows_timed(Y, FT, rows, cores)
    # the same oracle on one thread, on a sample 1/cores the size (about as long)
    n1 = max(16, n // cores)
    rows1 = np.linspace(0, S - 1, n1).astype(np.int32)
    _, _, dt1 = _oracle_rows_timed(Y, FT, rows1, 1)
    rec = {"value": n * S / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d target rows x %d sources of one mobility apply (%.1f s)" % (n, S, dt),
           "single_thread": {"value": n1 * S / dt1, "cores": 1,
                             "sample": "%d target rows x %d sources (%.1f s)" % (n1, S, dt1)}}
    return rec, (rows, ref, B)


def counters_from_profile():
    """ncu counters of the pair kernel (DRAM bytes per launch, FMA-pipe
    utilisation) from the committed record, if it was taken on the current
    kernel sources (else an empty dict)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "rpy_pair32_32k_counters.json")
    try:
        rec = json.load(open(path))
        m = hashlib.sha256()
        for src in rec["sources"]:
            m.update(open(os.path.join(ROOT, src), "rb").read())
        if rec.get("source_sha256") == m.hexdigest():
            return rec
    except Exception:
        pass
    return {}


def aggregate_ranks(units, ms, dist, device):
    """(sum of units over ranks, max of device time over ranks); one rank: as is."""
    if dist is None:
        return units, ms
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u[0]), float(t[0])


def pair_roofline(pairs_per_launch, pair_ms, n_launch, kernel="rpy_pair32", peak=None):
    avg = pair_ms / max(n_launch, 1)
    achieved = FLOPS_PER_PAIR * pairs_per_launch / (avg * 1e-3) / 1e12 if avg > 0 else None
    peak = FP32_PEAK_TFLOPS if peak is None else peak
    return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
            "flops_per_pair": FLOPS_PER_PAIR, "avg_launch_ms": avg, "launches": int(n_launch)}


def run_peaks(args, fil):
    """Measured FMA rates against the derived peaks (SMs x lanes x 2 x clock)."""
    out = {"metric": "measured FMA rate", "unit": "TFLOP/s", "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "FMA chains at full occupancy (fil_fma_peak)"}}
    for name, fp64, lanes in (("fp32", False, FP32_LANES_PER_SM), ("fp64", True, 2)):
        reps = [fil.fil_fma_peak(fp64) for _ in range(3)]
        fl, mhz = max(reps)
        out[name] = {"tflops": fl / 1e12, "sm_mhz": mhz,
                     "derived_at_max_clock": N_SM * lanes * 2 * SM_MAX_MHZ * 1e6 / 1e12,
                     "derived_at_measured_clock": N_SM * lanes * 2 * mhz * 1e6 / 1e12,
                     "runs_tflops": [r[0] / 1e12 for r in reps]}
    print(json.dumps(out), flush=True)


def run_mobility(args, fil, torch):
    """RPY applies alone on the positions of the 32k suspension with N(0,1)
    loads: a lean launch sequence for kernel profiling (one JSON line)."""
    wl, base, t, mu, Fext, follower = workload(args.n_fil)
    S = args.n_fil * 32
    Y = suspension_positions(wl, base, t, args.n_fil)
    FT = np.random.default_rng(1).standard_normal((S, 6))
    prec = precision_code(fil, args.precision)
    m = fil.Filaments(wl.seg_per_fil, precision=prec)
    m.init_straight(base, t, mu, None)
    tuned = m.autotune(5) if args.tune else None
    Yd = torch.from_numpy(Y).cuda()
    FTd = torch.from_numpy(FT).cuda()
    VW = torch.empty((S, 6), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        m.mobility_apply(Yd, FTd, VW)
    m.profile(True)
    m.profile_read()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        m.mobility_apply(Yd, FTd, VW)
    n, ms = m.profile_read()
    m.close()
    avg = ms / max(n, 1)
    print(json.dumps({"workload": "mobility apply, %d segments" % S, "precision": args.precision,
                      "pair_kernel_ms": avg, "pairs_per_s": S * S / (avg * 1e-3),
                      "tflops": FLOPS_PER_PAIR * S * S / (avg * 1e-3) / 1e12,
                      "autotuned": tuned}), flush=True)


# ---------------------------------------------------------------------------
# Nested records (default run): each a workload of its own with config,
# roofline, clocks and the FP64-oracle comparison.
# ---------------------------------------------------------------------------

def set_schedule(m, text):
    """A pair schedule 'tile,targets_per_thread,ctas_per_sm[,source_split]' set by hand."""
    v = [int(x) for x in text.split(",")]
    m.set_pair_schedule(*v[:3])
    if len(v) > 3:
        m.set_source_split(v[3])


def run_c1_mobility(fil, torch, applies=1000, per_graph=100, min_seconds=1.0, schedule=None):
    """Mobility apply alone: 100 random-walk filaments x 32 segments (3200) at
    5% volume fraction, N(0,1) loads, 1000 repeated applies. At this size an
    apply takes tens of microseconds, less than the host needs to issue it, so
    the applies are captured in a CUDA graph (100 per graph; the apply
    allocates nothing and does not synchronise with device arrays) and the
    graph is replayed; the schedule is autotuned for the size first. The
    1000-apply batch is repeated until the timed region lasts min_seconds
    (for the clock record). `schedule` ('tile,targets_per_thread,ctas_per_sm')
    sets the pair schedule by hand instead."""
    from paper_1903_12609_gb300.inputs import mobility_inputs
    Y, FT = mobility_inputs(100, 32, seed=0)
    S = Y.shape[0]
    stream = torch.cuda.Stream()
    m = fil.Filaments([32] * 100, precision=fil.FIL_PAIR32, stream=stream.cuda_stream)
    m.set_state(Y, np.tile([1.0, 0.0, 0.0, 0.0], (S, 1)))
    if schedule:
        set_schedule(m, schedule)
        tuned = (m.pair_schedule()[0], m.pair_schedule()[2], None)
    else:
        tuned = m.autotune(50)
    schedule = m.pair_schedule()
    split = m.source_split()
    Yd = torch.from_numpy(Y).cuda()
    FTd = torch.from_numpy(FT).cuda()
    VW = torch.empty((S, 6), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(20):
            m.mobility_apply(Yd, FTd, VW)
    torch.cuda.synchronize()
    m.profile(True)
    m.profile_read()
    a0, _, k0 = m.counters()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        for _ in range(per_graph):
            m.mobility_apply(Yd, FTd, VW)
    a1, _, k1 = m.counters()
    launches_per_graph = k1 - k0
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clk = clocks_start()
    t_wall = time.perf_counter()
    replays = 0
    e0.record(stream)
    while True:
        for _ in range(applies // per_graph):
            graph.replay()
            replays += 1
        stream.synchronize()
        if time.perf_counter() - t_wall >= min_seconds or replays >= 500:
            break
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clocks_stop(clk, torch.cuda.current_device())
    # the events inside the graph hold the pair-kernel times of its last replay
    n_pair, pair_ms = m.profile_read()
    m.profile(False)
    ms = e0.elapsed_time(e1)
    got = VW.cpu().numpy()
    m.close()
    n_app = replays * per_graph
    # FP64 oracle: the whole apply (all 3200 rows), timed on the host cores
    cores = os.cpu_count() or 1
    rows = np.arange(S, dtype=np.int32)
    ref, B, dt = _oracle_rows_timed(Y, FT, rows, cores)
    return {"metric": "RPY pair interactions/s", "value": n_app * float(S) * S / (ms * 1e-3),
            "unit": UNIT, "applies": int(n_app), "ms_per_apply": ms / n_app, "dtype": "f32+f64",
            "config": {"workload": "mobility apply alone: 100 random-walk filaments x 32 "
                                   "segments (3200), bond 2.2a, 5% volume fraction, F,T ~ N(0,1)",
                       "segments": S, "precision": "FP32 pair sums (compensated), FP64 results",
                       "issue": "CUDA graph of %d applies (pack and pair kernels), replayed"
                                % per_graph,
                       "l2": "inputs L2-resident (3200 segments); the metric is the apply "
                             "itself, repeated"},
            "roofline": pair_roofline(float(S) * S, pair_ms, n_pair),
            "autotuned": {"tile": tuned[0], "ctas_per_sm": tuned[1], "ms_per_apply": tuned[2],
                          "targets_per_thread": schedule[1], "source_split": split},
            "velocity_error": velocity_error(got, ref, B),
            "cpu_baseline": {"value": S * float(S) / dt, "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": "one whole apply, %d x %d pairs (%.2f s)"
                                                         % (S, S, dt)},
            "gpu_launches": int(launches_per_graph * replays), "clocks": clocks}


def run_c0_single(fil, torch, steps=200, order=1):
    """Single filament (N = 20) sedimenting from a 45-degree tilt, B = 1000,
    dt = T/100, Broyden tolerance 1e-8, 200 steps, all FP64 (App. B.2 J0),
    initial guess extrapolated at the given order."""
    from paper_1903_12609_gb300.inputs import single_filament, workload_params
    wl = workload_params(1, 20, B=1000.0, dt_over_T=0.01, tol=1e-8)
    base, t, mu, xi = single_filament(20, seed=0)
    stream = torch.cuda.Stream()
    m = fil.Filaments([20], a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt,
                      tol=wl.tol, max_iter=50, precision=fil.FIL_FP64,
                      j0_model=fil.FIL_J0_DRAG, stream=stream.cuda_stream)
    m.set_extrapolation(order)
    m.init_straight(base, t, mu, xi)
    m.set_external(np.tile([0.0, 0.0, -wl.W * wl.dL], (20, 1)), None, None)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    a0, _, k0 = m.counters()
    clk = clocks_start()
    e0.record(stream)
    iters = [m.step() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clocks_stop(clk, torch.cuda.current_device())
    a1, _, k1 = m.counters()
    ms = e0.elapsed_time(e1)
    Y = np.zeros((20, 3))
    m.get_state(Y, None, None, None, None)
    FT = np.random.default_rng(5).standard_normal((20, 6))
    VW = np.zeros((20, 6))
    m.mobility_apply(Y, FT, VW)
    m.close()
    # FP64 oracle on the final positions (N(0,1) loads): a whole apply, repeated
    cores = os.cpu_count() or 1
    rows = np.arange(20, dtype=np.int32)
    reps, dt = 0, 0.0
    while dt < 0.2:
        ref, B, d = _oracle_rows_timed(Y, FT, rows, 1)
        reps += 1
        dt += d
    err = velocity_error(VW, ref, B)
    err["loads"] = "N(0,1) at the final positions"
    return {"metric": "timesteps/s", "value": steps / (ms * 1e-3), "unit": "timesteps/s",
            "steps": steps, "broyden_iters_per_step": float(np.mean(iters)),
            "pairs_per_s": (a1 - a0) * 400.0 / (ms * 1e-3), "dtype": "f64",
            "config": {"workload": "single filament N=20, B=1000, 45-degree tilt with 1e-3 "
                                   "perturbation, sedimenting; BDF2 dt=T/100, tol 1e-8",
                       "precision": "fp64", "j0": "drag (App. B.2)",
                       "initial_guess": EXTRAP_NAME[order]},
            "roofline": {"bound": "latency", "note": "400 pairs per apply: each Broyden "
                                                     "iteration is a chain of small kernels and "
                                                     "one status read"},
            "velocity_error": err,
            "cpu_baseline": {"value": reps * 400.0 / dt, "unit": "pair interactions/s",
                             "cores": 1, "kind": "oracle",
                             "sample": "%d whole applies of 20 x 20 pairs" % reps},
            "gpu_launches": int(k1 - k0), "clocks": clocks}


def run_ensemble(args, fil, torch, nested=False):
    """Batched ensemble: independent suspensions in one context (one launch per
    kernel, per-system Broyden); aggregate and per-system rates."""
    from paper_1903_12609_gb300.inputs import ensemble
    rank = int(os.environ.get("RANK", "0"))
    wl, fps, segs, base, t, mu, Fext, follower = ensemble(args.n_sys, seed=rank)
    n_sys = len(fps)
    off = np.concatenate([[0], np.cumsum(fps)])
    seg_arr = np.array(segs)
    S_sys = np.array([seg_arr[off[k]:off[k + 1]].sum() for k in range(n_sys)], dtype=np.float64)
    pairs_per_apply = float(np.sum(S_sys ** 2))
    stream = torch.cuda.Stream()
    j0 = fil.FIL_J0_FILAMENT_RPY if max(segs) <= 38 else fil.FIL_J0_DRAG
    prec = precision_code(fil, args.ens_precision)
    m = fil.Filaments(segs, fil_per_sys=fps, a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT,
                      dt=wl.dt, tol=wl.tol, max_iter=args.ens_max_iter, precision=prec,
                      j0_model=j0, stream=stream.cuda_stream)
    m.init_straight(base, t, mu, None)
    m.set_external(Fext, None, follower)
    m.set_graph(args.graph)
    m.set_j0_reuse(args.j0_reuse)
    m.set_broyden_memory(args.ens_broyden_memory)
    m.set_extrapolation(args.extrapolation)
    for _ in range(args.warmup):
        m.step()
    tuned = None
    if args.ens_schedule:
        set_schedule(m, args.ens_schedule)
    elif args.tune_ensemble:
        tuned = m.autotune(2)
    schedule = m.pair_schedule()
    split = m.source_split()
    a0, i0, k0 = m.counters()
    p0 = m.pair_count()
    torch.cuda.synchronize()
    clk = clocks_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters, sys_iters = [], []
    steps = args.ens_steps if nested else args.steps
    e0.record(stream)
    for _ in range(steps):
        iters.append(m.step())
        sys_iters.append(m.sys_stats()[0].copy())
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clocks_stop(clk, torch.cuda.current_device())
    a1, _, k1 = m.counters()
    pairs = m.pair_count() - p0
    ms = e0.elapsed_time(e1)
    si = np.array(sys_iters)
    # the pair kernel on its own (CUDA events per launch, outside the graphs):
    # two more steps with kernel launches and the library's timing on
    m.set_graph(0)
    m.profile(True)
    m.profile_read()
    q0 = m.pair_count()
    for _ in range(2):
        m.step()
    n_pair, pair_ms = m.profile_read()
    pairs_prof = m.pair_count() - q0
    # velocity error: the ensemble's apply at the current positions with N(0,1)
    # loads against the oracle on sampled systems (each system's block alone)
    Sall = int(S_sys.sum())
    Y = np.zeros((Sall, 3))
    m.get_state(Y, None, None, None, None)
    FT = np.random.default_rng(7).standard_normal((Sall, 6))
    VW = np.zeros((Sall, 6))
    m.mobility_apply(Y, FT, VW)
    m.close()
    soff = np.concatenate([[0], np.cumsum(S_sys)]).astype(np.int64)
    pick = np.random.default_rng(8).choice(n_sys, size=min(8, n_sys), replace=False)
    cores = os.cpu_count() or 1
    refs, Bs, gots, dt, opairs = [], [], [], 0.0, 0.0
    for k in pick:
        sl = slice(soff[k], soff[k + 1])
        rows = np.arange(soff[k + 1] - soff[k], dtype=np.int32)
        ref, B, d = _oracle_rows_timed(Y[sl], FT[sl], rows, cores)
        refs.append(ref)
        Bs.append(B)
        gots.append(VW[sl])
        dt += d
        opairs += float(rows.size) ** 2
    err = velocity_error(np.concatenate(gots), np.concatenate(refs), np.concatenate(Bs))
    err["systems"] = [int(k) for k in pick]
    # pairs actually evaluated (converged systems drop out of the applies)
    roof = pair_roofline(pairs_prof / max(n_pair, 1), pair_ms, n_pair)
    roof["measured_over"] = "2 steps without graphs"
    rec = {
        "metric": METRIC if not nested else "system timesteps/s",
        "value": pairs / (ms * 1e-3) if not nested else n_sys * steps / (ms * 1e-3),
        "unit": UNIT if not nested else "system timesteps/s",
        "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "ensemble of %d independent suspensions, filaments U[1,64] x "
                               "segments U[16,48] (%d filaments, %d segments), physics of the "
                               "32k suspension" % (n_sys, len(segs), Sall),
                   "j0": "filament_rpy" if j0 == fil.FIL_J0_FILAMENT_RPY else "drag",
                   "precision": args.ens_precision, "precision_note":
                       PRECISION_NOTE[args.ens_precision],
                   "j0_reuse_max_age": args.j0_reuse,
                   "initial_guess": EXTRAP_NAME[args.extrapolation],
                   "broyden_memory": args.ens_broyden_memory,
                   "pairs_per_apply": pairs_per_apply, "parallelism": "single"},
        "pairs_per_s": pairs / (ms * 1e-3),
        "ensemble_timesteps_per_s": steps / (ms * 1e-3),
        "timesteps_per_s_per_system": steps / (ms * 1e-3),
        "system_timesteps_per_s": n_sys * steps / (ms * 1e-3),
        "broyden_iters_per_step": {"max_over_systems": float(np.mean(iters)),
                                   "mean_over_systems": float(si.mean()),
                                   "p90_over_systems": float(np.percentile(si, 90))},
        "roofline": roof,
        "velocity_error": err,
        "cpu_baseline": {"value": opairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "whole applies of %d sampled systems (%.2f s)"
                                   % (len(pick), dt)},
        "graph": bool(args.graph),
        "autotuned": ({"tile": tuned[0], "ctas_per_sm": tuned[1], "ms_per_apply": tuned[2]}
                      if tuned else None),
        "pair_schedule": {"tile": schedule[0], "targets_per_thread": schedule[1],
                          "ctas_per_sm": schedule[2], "source_split": split},
        "gpu_launches": int(k1 - k0), "clocks": clocks}
    if not nested:
        print(json.dumps(rec), flush=True)
    return rec


def host_round_trip(torch, n=2000):
    """What a device-side Broyden loop could save: the host's part of one
    iteration of the library's loop is a status read (a small device-to-host
    copy after the iteration's last kernel) and a stream synchronisation. This
    times that round trip with a tiny kernel in front, n times."""
    stream = torch.cuda.Stream()
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    h = torch.empty(8, dtype=torch.int32).pin_memory()
    with torch.cuda.stream(stream):
        for _ in range(50):
            x.add_(1)
            h.copy_(x, non_blocking=True)
            stream.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            x.add_(1)
            h.copy_(x, non_blocking=True)
            stream.synchronize()
        dt = time.perf_counter() - t0
    return 1e6 * dt / n


def run_tether(fil, torch, steps=40, warmup=5, every=4, order=1, j0_reuse=1, memory=0):
    """The 32k suspension's cloud with every fourth filament clamped at its base
    (Sec. 5.2.1: Y_1 fixed, u_1 = 0), weightless: the follower-force half keeps
    its tip force, the other half is passive. (With gravity the cloud settles
    collectively at ~35 times the speed of a lone filament, ~7a per step, and the
    first step would ask the clamps to hold that flow from a standing start;
    Algorithm 2 with the per-filament J0 does not converge on it at 1000
    filaments, on the GPU or in the oracle.) FIL_PAIR32, extrapolated initial
    guess of the given order (tether multipliers linear; the network refuses
    tethered contexts); the clamps are set once, so J0 may be kept for up to
    j0_reuse steps and `memory` Broyden pairs carried while it is."""
    wl, base, t, mu, Fext, follower = workload(1000, 32, seed=0)
    stream = torch.cuda.Stream()
    m = fil.Filaments(wl.seg_per_fil, precision=fil.FIL_PAIR32, stream=stream.cuda_stream,
                      a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol,
                      max_iter=wl.max_iter, j0_model=fil.FIL_J0_FILAMENT_RPY)
    m.set_extrapolation(order)
    m.set_j0_reuse(j0_reuse)
    m.set_broyden_memory(memory)
    m.init_straight(base, t, mu, None)
    m.set_external(None, None, follower)
    mask = (np.arange(1000) % every) == 0
    m.set_tether(mask, base.copy(), np.zeros((1000, 3)))
    warm_iters = [m.step() for _ in range(warmup)]
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    a0, _, k0 = m.counters()
    m.profile(True)
    m.profile_read()
    clk = clocks_start()
    e0.record(stream)
    iters = [m.step() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clocks_stop(clk, torch.cuda.current_device())
    n_pair, pair_ms = m.profile_read()
    a1, _, k1 = m.counters()
    lam = np.zeros((1000, 6))
    m.get_tether(lam)
    m.close()
    ms = e0.elapsed_time(e1)
    S = 32000.0
    return {"metric": "timesteps/s", "value": steps / (ms * 1e-3), "unit": "timesteps/s",
            "steps": steps, "broyden_iters_per_step": float(np.mean(iters)),
            "iters": [int(i) for i in iters], "warmup_iters": warm_iters,
            "pairs_per_s": (a1 - a0) * S * S / (ms * 1e-3), "dtype": "f32+f64",
            "config": {"workload": "the 32k suspension's cloud (1000 x 32) with %d filaments "
                                   "(every %d-th) clamped at the base, no gravity, tip follower "
                                   "force fL^2/KB=100 on the other half as in the suspension, "
                                   "dt=T/200, tol 1e-4" % (int(mask.sum()), every),
                       "precision": "pair32",
                       "initial_guess": EXTRAP_NAME[order],
                       "j0": "filament_rpy + rank-6 correction per clamped filament",
                       "j0_reuse_max_age": j0_reuse, "broyden_memory": memory},
            "roofline": pair_roofline(S * S, pair_ms, n_pair),
            "max_abs_multiplier": float(np.abs(lam[mask]).max()),
            "gpu_launches": int(k1 - k0), "clocks": clocks}


def run_suspension(args, fil, torch, world, rank, local):
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n_fil, n_seg = args.n_fil, 32
    S = n_fil * n_seg
    wl, base, t, mu, Fext, follower = workload(n_fil, n_seg, seed=rank)
    stream = torch.cuda.Stream()
    prec = precision_code(fil, args.precision)
    j0 = fil.FIL_J0_FILAMENT_RPY if args.j0 == "filament_rpy" else fil.FIL_J0_DRAG
    params = dict(a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol,
                  max_iter=wl.max_iter, j0_model=j0)
    m = fil.Filaments(wl.seg_per_fil, precision=prec, stream=stream.cuda_stream, **params)
    m.init_straight(base, t, mu, None)
    m.set_external(Fext, None, follower)
    m.set_j0_reuse(args.j0_reuse)
    m.set_broyden_memory(args.broyden_memory)
    m.set_extrapolation(args.extrapolation)
    m.set_graph(args.graph)
    if args.steric > 0:
        m.set_steric(args.steric, 1.1)

    # learned warm start (chosen form): the committed network, trained on other seeds for
    # the extrapolation order it corrects
    net, warm_mode, net_order, net_note = None, None, None, None
    if args.warm != "off" and prec != fil.FIL_FP64:
        from paper_1903_12609_gb300 import warmstart
        if os.path.exists(warmstart.DEFAULT_WEIGHTS):
            net_order = warmstart.trained_order()
            warm_mode = (fil.FIL_WARM_PREDICTION_FIRST if args.warm == "prediction_first"
                         else fil.FIL_WARM_BEST_OF_TWO)
            net = warmstart.load(max_batch=max(64, n_fil), stream=stream.cuda_stream)
            if net_order == args.extrapolation:
                fil.fil_warm_attach(m.ctx, net, warm_mode)
            else:
                net_note = ("the committed network corrects the %s; not attached to the "
                            "timed steps (%s)" % (EXTRAP_NAME[net_order],
                                                  EXTRAP_NAME[args.extrapolation]))

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        m.step()
    tuned = m.autotune(5) if args.tune else None
    st0 = [np.zeros((S, 3)), np.zeros((S, 4)), np.zeros((S, 3)), np.zeros((S, 3)),
           np.zeros((S - n_fil, 3))]
    m.get_state(*st0)

    def timed_steps(ctx_obj, K, with_flush=True):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        its = []
        with torch.cuda.stream(stream):
            for j in range(K):
                if with_flush:
                    flush.fill_(float(j))
                ev[j][0].record(stream)
                its.append(ctx_obj.step())
                ev[j][1].record(stream)
        torch.cuda.synchronize()
        return float(sum(s.elapsed_time(e) for s, e in ev)), its

    # ---- timed region: K steps, L2 flushed between steps ----
    a0, i0, k0 = m.counters()
    jb0, jr0 = m.j0_stats()
    m.profile(True)
    m.profile_read()
    barrier()
    clk = clocks_start()
    t_wall = time.perf_counter()
    dev_ms, iters = timed_steps(m, args.steps)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = clocks_stop(clk, local)
    n_pair_launch, pair_ms = m.profile_read()
    m.profile(False)
    a1, i1, k1 = m.counters()
    jb1, jr1 = m.j0_stats()
    applies = a1 - a0
    pairs = applies * float(S) * S
    Y_timed = np.zeros((S, 3))
    m.get_state(Y_timed, None, None, None, None)

    # whole-job aggregate: units of all ranks over the slowest rank's time
    tot_pairs, max_ms = aggregate_ranks(pairs, dev_ms, dist, "cuda")
    value = tot_pairs / (max_ms * 1e-3)

    # ---- dominant kernel: the RPY pair kernel, timed live by the library ----
    roof = pair_roofline(float(S) * S, pair_ms, n_pair_launch,
                         kernel="rpy_pair32" if prec != fil.FIL_FP64 else "rpy_pair64")
    prof = counters_from_profile() if prec != fil.FIL_FP64 else {}
    roof["traffic"] = prof.get("dram_bytes_per_launch")
    roof["fma_pipe_active"] = prof.get("fma_pipe_active")
    roof["share_of_step"] = pair_ms / dev_ms if dev_ms > 0 else None
    roof["peak_note"] = "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (derived)"
    if prec == fil.FIL_FP64:
        roof["peak"] = roof["frac"] = None

    # ---- end to end through the C ABI with host buffers ----
    # (a) a time-stepping user: every step copies its external loads in from pinned host
    #     memory (fil_set_external) and the positions and orientations out (fil_get_state);
    #     the solver's state and history stay on the device
    Fh = torch.from_numpy(np.ascontiguousarray(Fext)).pin_memory()
    fh = torch.from_numpy(np.ascontiguousarray(follower, dtype=np.float64)).pin_memory()
    Yo = torch.empty((S, 3), dtype=torch.float64).pin_memory()
    qo = torch.empty((S, 4), dtype=torch.float64).pin_memory()
    barrier()
    a2, _, _ = m.counters()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_iters = []
    e0.record(stream)
    for _ in range(args.e2e_steps):
        m.set_external(Fh, None, fh)
        e2e_iters.append(m.step())
        m.get_state(Yo, qo, None, None, None)
    e1.record(stream)
    barrier()
    a3, _, _ = m.counters()
    e2e_ms = e0.elapsed_time(e1)
    e2e_pairs = (a3 - a2) * float(S) * S
    in_bytes = 8 * (Fh.numel() + fh.numel())
    out_bytes = 8 * (Yo.numel() + qo.numel())
    # (b) restarting every step from host arrays (fil_set_state, fil_step, fil_get_state):
    #     the whole state goes both ways and the step history is lost at each restart
    Yh = np.zeros((S, 3)); qh = np.zeros((S, 4)); Yph = np.zeros((S, 3)); uh = np.zeros((S, 3))
    lh = np.zeros((S - n_fil, 3))
    m.get_state(Yh, qh, Yph, uh, lh)
    barrier()
    a4, _, _ = m.counters()
    r_iters = []
    e0.record(stream)
    for _ in range(args.e2e_steps):
        m.set_state(Yh, qh, Yph, uh, lh)
        r_iters.append(m.step())
        m.get_state(Yh, qh, Yph, uh, lh)
    e1.record(stream)
    barrier()
    a5, _, _ = m.counters()
    r_ms = e0.elapsed_time(e1)
    r_pairs = (a5 - a4) * float(S) * S
    state_bytes = 8 * (Yh.size + qh.size + Yph.size + uh.size + lh.size)

    extra = {}
    if args.extra and rank == 0:
        # ---- one converged step from st0, extrapolated start: this form vs plain FP64 ----
        m.set_state(*st0)
        if net is not None:
            fil.fil_warm_attach(m.ctx, None)
        m.step()
        Y1c, q1c = np.zeros((S, 3)), np.zeros((S, 4))
        m.get_state(Y1c, q1c, None, None, None)

        # ---- initial guesses of a step: linear and quadratic extrapolation and the learned
        #      warm start (at the order it was trained for), on the timed window's first 20
        #      steps from st0 and 20 steps from step 200 of the same trajectory ----
        ig = {"weights": (os.path.relpath(warmstart.DEFAULT_WEIGHTS, ROOT)
                          if net is not None else None),
              "network_trained_for_order": net_order, "mode": args.warm}
        K = 20
        m.set_state(*st0)
        m.set_extrapolation(args.extrapolation)
        fil.fil_warm_attach(m.ctx, net if net_note is None else None, warm_mode or 0)
        for _ in range(200 - args.warmup):
            m.step()
        st200 = [np.zeros_like(a) for a in st0]
        m.get_state(*st200)
        arms = [("extrapolation_linear", 1, None), ("extrapolation_quadratic", 2, None),
                ("extrapolation_adaptive", 3, None)]
        if net is not None:
            arms.append(("learned", net_order, net))
        for wname, state, what in (
                ("early", st0, "20 steps from the state after the warm-up steps of a "
                               "fresh cloud (the timed window's first 20 steps)"),
                ("later", st200, "20 steps from step 200 of the same trajectory")):
            rec = {"window": what}
            for name, order, use in arms:
                m.set_state(*state)
                m.set_extrapolation(order)
                fil.fil_warm_attach(m.ctx, use, warm_mode or 0)
                ms_w, its = timed_steps(m, K, with_flush=False)
                rec[name] = {"timesteps_per_s": K / (ms_w * 1e-3), "order": order,
                             "broyden_iters_per_step": float(np.mean(its)), "steps": K}
            if net is not None:
                base = {1: "extrapolation_linear", 2: "extrapolation_quadratic",
                        3: "extrapolation_adaptive"}[net_order]
                rec["learned_over_its_extrapolation_iterations"] = (
                    rec["learned"]["broyden_iters_per_step"]
                    / rec[base]["broyden_iters_per_step"])
            ig[wname] = rec
        fil.fil_warm_attach(m.ctx, None)
        extra["initial_guess"] = ig

        # ---- velocity error vs the FP64 oracle on the positions after the timed steps
        #      (N(0,1) loads; sampled target rows = the CPU baseline's sample) ----
        FTv = np.random.default_rng(2).standard_normal((S, 6))
        VWv = np.zeros((S, 6))
        m.mobility_apply(Y_timed, FTv, VWv)
        m.close()
        if net is not None:
            fil.fil_mlp_destroy(net)
            net = None
        cpu, (rows, ref, B) = cpu_baseline(Y_timed, FTv, args.cpu_seconds)
        extra["cpu_baseline"] = cpu
        verr = velocity_error(VWv[rows], ref, B)
        verr["loads"] = "N(0,1) at the positions after the timed steps"
        extra["velocity_error"] = verr

        # ---- the all-FP32-solve variant (FIL_MIXED) from st0, same steps ----
        mm = fil.Filaments(wl.seg_per_fil, precision=fil.FIL_MIXED, stream=stream.cuda_stream,
                           **params)
        mm.set_state(*st0)
        mm.set_external(Fext, None, follower)
        mm.set_extrapolation(args.extrapolation)
        mm.set_j0_reuse(args.j0_reuse)
        mm.set_broyden_memory(args.broyden_memory)
        netm = None
        if warm_mode is not None and net_note is None:
            netm = warmstart.load(max_batch=max(64, n_fil), stream=stream.cuda_stream)
            fil.fil_warm_attach(mm.ctx, netm, warm_mode)
        mm.profile(True)
        mm.profile_read()
        ma0, _, _ = mm.counters()
        ms_m, its_m = timed_steps(mm, args.steps)
        ma1, _, _ = mm.counters()
        npl, pms = mm.profile_read()
        mm.close()
        if netm is not None:
            fil.fil_mlp_destroy(netm)
        extra["fast_mixed"] = {
            "timesteps_per_s": args.steps / (ms_m * 1e-3),
            "pairs_per_s": (ma1 - ma0) * float(S) * S / (ms_m * 1e-3),
            "broyden_iters_per_step": float(np.mean(its_m)), "steps": args.steps,
            "precision": "mixed", "precision_note": PRECISION_NOTE["mixed"],
            "roofline": pair_roofline(float(S) * S, pms, npl),
            "from": "the same state as the timed steps, same initial-guess rule, J0 policy and Broyden memory"}

        # ---- the other J0 policy (built every step / kept up to 10 steps) from st0 ----
        other = 1 if args.j0_reuse > 1 else 10
        mr = fil.Filaments(wl.seg_per_fil, precision=prec, stream=stream.cuda_stream, **params)
        mr.set_state(*st0)
        mr.set_external(Fext, None, follower)
        mr.set_j0_reuse(other)
        mr.set_broyden_memory(args.broyden_memory)
        mr.set_extrapolation(args.extrapolation)
        netr = None
        if warm_mode is not None and net_note is None:
            netr = warmstart.load(max_batch=max(64, n_fil), stream=stream.cuda_stream)
            fil.fil_warm_attach(mr.ctx, netr, warm_mode)
        rb0, rr0 = mr.j0_stats()
        ms_r, its_r = timed_steps(mr, args.steps)
        rb1, rr1 = mr.j0_stats()
        mr.close()
        if netr is not None:
            fil.fil_mlp_destroy(netr)
        extra["j0_policy_variant"] = {
            "j0_reuse_max_age": other, "timesteps_per_s": args.steps / (ms_r * 1e-3),
            "broyden_iters_per_step": float(np.mean(its_r)), "steps": args.steps,
            "j0_builds": int(rb1 - rb0), "j0_reuses": int(rr1 - rr0),
            "from": "the same state as the timed steps, same precision and initial guess"}

        # ---- the plain FP64 form from st0 (extrapolated start) ----
        if args.plain_steps > 0:
            mp = fil.Filaments(wl.seg_per_fil, precision=fil.FIL_FP64,
                               stream=stream.cuda_stream, **params)
            mp.set_state(*st0)
            mp.set_external(Fext, None, follower)
            if args.steric > 0:
                mp.set_steric(args.steric, 1.1)
            it1 = mp.step()                              # the converged step compared below
            Y1p, q1p = np.zeros((S, 3)), np.zeros((S, 4))
            mp.get_state(Y1p, q1p, None, None, None)
            pa0, _, _ = mp.counters()
            pms_, pits = timed_steps(mp, args.plain_steps, with_flush=False)
            pa1, _, _ = mp.counters()
            mp.close()
            p64, _ = fil.fil_fma_peak(True)
            plain = {"timesteps_per_s": args.plain_steps / (pms_ * 1e-3),
                     "pairs_per_s": (pa1 - pa0) * float(S) * S / (pms_ * 1e-3),
                     "broyden_iters_per_step": float(np.mean(pits)),
                     "steps": args.plain_steps, "precision": "fp64",
                     "initial_guess": "order-1 extrapolation", "j0_reuse_max_age": 1,
                     "from": "steps 2.. from the same state as the timed steps"}
            plain["frac_of_measured_fp64_peak"] = plain["pairs_per_s"] * FLOPS_PER_PAIR / p64
            extra["plain_fp64"] = plain
            extra["chosen_over_plain_timesteps"] = (args.steps / (max_ms * 1e-3)
                                                    / plain["timesteps_per_s"])
            extra["converged_step_vs_fp64"] = {
                "max_abs_dY": float(np.abs(Y1c - Y1p).max()),
                "max_abs_dq": float(np.abs(q1c - q1p).max()),
                "tol_a": wl.tol * wl.a, "iters_fp64": int(it1),
                "what": "one step from the same state with the extrapolated start, this "
                        "precision vs FIL_FP64, both converged to ||f||_inf <= tol a"}

        # ---- host work per Broyden iteration (the case for a device-side loop) ----
        rt = host_round_trip(torch)
        iters_mean = float(np.mean(iters))
        extra["host_loop_overhead"] = {
            "round_trip_us": rt, "iterations_per_step": iters_mean,
            "share_of_step": rt * 1e-3 * (iters_mean + 1) / (max_ms / args.steps),
            "what": "a tiny kernel, a 32-byte device-to-host copy and a stream synchronisation, "
                    "timed 2000 times: the host's part of each Broyden iteration (and of the "
                    "step set-up), which a loop kept on the device would remove"}

        # ---- the other configurations (a failure is reported in its record) ----
        for key, fn in (("c1_mobility_3200", lambda: run_c1_mobility(fil, torch)),
                        ("c0_single_filament",
                         lambda: run_c0_single(fil, torch, order=args.extrapolation)),
                        ("c3_ensemble256", lambda: run_ensemble(args, fil, torch, nested=True)),
                        ("tethered_suspension",
                         lambda: run_tether(fil, torch, order=args.extrapolation,
                                            j0_reuse=args.j0_reuse,
                                            memory=args.broyden_memory))):
            try:
                extra[key] = fn()
            except Exception as exc:   # keep the headline line when a nested record fails
                extra[key] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    else:
        m.close()
        if net is not None:
            fil.fil_mlp_destroy(net)

    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return

    # measured FMA rates (after the timed region): context for the derived peak
    p32, mhz32 = fil.fil_fma_peak(False)
    p64, mhz64 = fil.fil_fma_peak(True)
    roof["peak_measured"] = {
        "fp32_tflops": p32 / 1e12, "fp32_sm_mhz": mhz32, "fp64_tflops": p64 / 1e12,
        "fp64_sm_mhz": mhz64,
        "frac_of_measured": (roof["achieved"] / (p32 / 1e12) if prec != fil.FIL_FP64 else None),
        "how": "fil_fma_peak: packed FP32x2 / FP64 FMA chains, full occupancy, 5 launches of "
               "~20 ms"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec != fil.FIL_FP64 else "f64", "data": "synthetic",
        "config": {
            "workload": "suspension %d filaments x 32 segments (%d), 2%% volume fraction, "
                        "half sedimenting (B=1000) half tip-follower (fL^2/KB=100), BDF2 "
                        "dt=T/200, Broyden tol 1e-4" % (n_fil, S),
            "segments": S, "precision": args.precision,
            "precision_note": PRECISION_NOTE[args.precision], "j0": args.j0,
            "initial_guess": (("learned warm start (%s) on the %s"
                               % (args.warm, EXTRAP_NAME[args.extrapolation]))
                              if warm_mode is not None and net_note is None
                              else EXTRAP_NAME[args.extrapolation]),
            "initial_guess_note": net_note,
            "j0_reuse_max_age": args.j0_reuse,
            "broyden_memory": args.broyden_memory,
            "steric_FS": args.steric if args.steric > 0 else None,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between timed steps (256 MiB write)"},
        "timesteps_per_s": args.steps / (max_ms * 1e-3),
        "broyden_iters_per_step": float(np.mean(iters)),
        "mobility_applies": int(applies),
        "j0_builds": int(jb1 - jb0), "j0_reuses": int(jr1 - jr0),
        "roofline": roof,
        "autotuned": ({"tile": tuned[0], "ctas_per_sm": tuned[1], "ms_per_apply": tuned[2]}
                      if tuned else None),
        "e2e": {"value": e2e_pairs / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes,
                "timesteps_per_s": args.e2e_steps / (e2e_ms * 1e-3),
                "broyden_iters_per_step": float(np.mean(e2e_iters)) if e2e_iters else None,
                "steps": args.e2e_steps,
                "what": "fil_set_external (pinned host loads in), fil_step, fil_get_state "
                        "(positions and quaternions out), every step",
                "restarted": {"value": r_pairs / (r_ms * 1e-3), "unit": UNIT,
                              "h2d_bytes_per_step": state_bytes,
                              "d2h_bytes_per_step": state_bytes,
                              "timesteps_per_s": args.e2e_steps / (r_ms * 1e-3),
                              "broyden_iters_per_step": (float(np.mean(r_iters))
                                                         if r_iters else None),
                              "what": "fil_set_state, fil_step, fil_get_state of the whole "
                                      "state from / to host arrays, every step"}},
        "gpu_launches": int(k1 - k0),
        "clocks": clocks,
        "wall_s": t_wall,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_reference(args, rank):
    if rank != 0:
        return
    from oracle import build as obuild
    obuild.build()
    from oracle import rpy
    wl, base, t, mu, Fext, follower = workload()
    S = 1000 * 32
    Y = np.concatenate([base[i] + np.arange(32)[:, None] * wl.dL * t[i] for i in range(1000)])
    FT = np.random.default_rng(1).standard_normal((S, 6))
    cores = os.cpu_count() or 1
    rows = np.linspace(0, S - 1, 2048).astype(np.int32)
    for _ in range(args.warmup):
        rpy.apply_rows(Y, FT, rows[:64], nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rpy.apply_rows(Y, FT, rows, nthreads=cores)
    dt = time.perf_counter() - t0
    value = args.steps * rows.size * S / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "FP64 CPU oracle: %d target rows x 32000 sources of the "
                                   "RPY mobility apply per step (suspension 1000x32)" % rows.size,
                       "segments": S},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d rows x %d sources per step" % (rows.size, S)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="pair32", choices=["pair32", "mixed", "fp64"],
                    help="pair32: FP32 pair sums, FP64 elsewhere (default); mixed: also FP32 J0 "
                         "solves and Broyden history; fp64: everything FP64")
    ap.add_argument("--plain-steps", type=int, default=5,
                    help="timed steps of the plain FP64 form for comparison (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--extra", type=int, default=1,
                    help="1: also the nested records (variants, other configurations, oracle "
                         "comparison); 0: the headline suspension only (for profiling)")
    ap.add_argument("--broyden-memory", type=int, default=48,
                    help="Broyden pairs carried into the next step while J0 is kept "
                         "(fil_set_broyden_memory; 0 = reset every step, the paper's choice)")
    ap.add_argument("--j0-reuse", type=int, default=10,
                    help="keep J0 for up to this many steps (fil_set_j0_reuse; 1 = every step)")
    ap.add_argument("--j0", default="filament_rpy", choices=["filament_rpy", "drag"],
                    help="approximate Jacobian: filament RPY blocks (default) or App. B.2 drag")
    ap.add_argument("--n-fil", type=int, default=1000,
                    help="filaments of 32 segments (1000 = the 32k suspension; smaller for profiling)")
    ap.add_argument("--extrapolation", type=int, default=3, choices=[1, 2, 3],
                    help="extrapolated initial guess (fil_set_extrapolation): 1 linear, "
                         "2 quadratic, 3 adaptive per filament and block; the learned warm "
                         "start is attached only when trained for this choice")
    ap.add_argument("--warm", default="prediction_first",
                    choices=["prediction_first", "best_of_two", "off"],
                    help="learned warm start of each step (the committed network) and its mode")
    ap.add_argument("--n-sys", type=int, default=256, help="systems of the ensemble workload")
    ap.add_argument("--ens-max-iter", type=int, default=100)
    ap.add_argument("--ens-steps", type=int, default=40,
                    help="timed steps of the ensemble record of the default run")
    ap.add_argument("--ens-precision", default="mixed", choices=["pair32", "mixed", "fp64"])
    ap.add_argument("--ens-broyden-memory", type=int, default=0,
                    help="Broyden pairs carried across steps in the ensemble (measured slower "
                         "there: the slowest system's iterations rise)")
    ap.add_argument("--tune", type=int, default=0,
                    help="autotune the suspension's pair-kernel schedule after the warm-up steps "
                         "(its default schedule is the tuned one)")
    ap.add_argument("--tune-ensemble", type=int, default=1,
                    help="autotune the ensemble's pair-kernel schedule after its warm-up steps")
    ap.add_argument("--ens-schedule", default=None,
                    help="set the ensemble's pair schedule 'tile,targets_per_thread,ctas_per_sm"
                         "[,source_split]' instead of autotuning it (e.g. for a profile of the "
                         "tuned schedule)")
    ap.add_argument("--c1-schedule", default=None,
                    help="set the 3200-segment apply's pair schedule "
                         "'tile,targets_per_thread,ctas_per_sm[,source_split]' instead of "
                         "autotuning it")
    ap.add_argument("--steric", type=float, default=0.0,
                    help="steric barrier strength F^S (Sec. 2.6, chi = 1.1); 0 = off")
    ap.add_argument("--graph", type=int, default=0,
                    help="run each Broyden iteration as one CUDA graph launch (ensemble; off by "
                         "default: with kernels of 0.05-0.7 ms the launches are not the cost and "
                         "the graph's speculative last iteration is)")
    ap.add_argument("--workload", default="suspension",
                    choices=["suspension", "mobility", "ensemble", "peaks", "c0", "c1", "tether"],
                    help="'mobility': only RPY applies on the suspension's configuration (for "
                         "profiling); 'peaks': the measured FP32 / FP64 FMA rates beside the "
                         "derived ones; c0, c1, tether: one nested record alone")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_12609_gb300 import fil

    torch.cuda.set_device(local)
    if args.workload == "mobility":
        run_mobility(args, fil, torch)
    elif args.workload == "peaks":
        run_peaks(args, fil)
    elif args.workload == "ensemble":
        run_ensemble(args, fil, torch)
    elif args.workload == "c1":
        print(json.dumps(run_c1_mobility(fil, torch, schedule=args.c1_schedule)), flush=True)
    elif args.workload in ("c0", "tether"):
        if args.workload == "c0":
            rec = run_c0_single(fil, torch, order=args.extrapolation)
        else:
            rec = run_tether(fil, torch, order=args.extrapolation, j0_reuse=args.j0_reuse,
                             memory=args.broyden_memory)
        print(json.dumps(rec), flush=True)
    else:
        run_suspension(args, fil, torch, world, rank, local)


if __name__ == "__main__":
    main()

"""Benchmark: RPY pair interactions per second during BDF2 timesteps of a
32 000-segment filament suspension on one GB300 (per GPU; weak scaling over
independent replicas when launched on several GPUs).

One step = one whole timestep of the method: initial guess, J0 assembly and
banded LU, the Broyden loop (each iteration: unpack, forces, RPY mobility over
all S^2 pairs, residual, J0 solve, rank-one update) and the commit. The value
is the number of RPY pair interactions evaluated in the timed steps divided by
their device time (S^2 per residual evaluation; begin + one per iteration).

Workload (synthetic, seeded; shapes of the paper's 3D filament clouds):
1000 filaments x 32 segments, a = 1, dL = 2.2a, eta = 1, isotropic straight
initial filaments in a cube at 2% volume fraction (overlaps redrawn); the first
500 filaments sediment under gravity (B = L^3 W / K_B = 1000), the other 500
carry a compressive tip follower force f L^2 / K_B = 100 and no weight;
dt = T/200 with T = eta L / W; Broyden tolerance 1e-4 (||f||_inf <= tol a).
Precision: FP32-compensated pair sums, FP64 everything else ("mixed").

Output: one JSON line (see the keys below). --impl reference times the FP64
CPU oracle on bounded samples of the same workload instead.
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


def cpu_baseline(Y, FT, seconds=10.0):
    """The FP64 oracle on the host cores: a bounded sample of target rows of one
    mobility apply of the same workload, scaled to pairs/s."""
    from oracle import rpy
    cores = os.cpu_count() or 1
    S = Y.shape[0]
    rows = np.arange(64, dtype=np.int32)
    t0 = time.perf_counter()
    rpy.apply_rows(Y, FT, rows, nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-4)
    n = int(min(S, max(64, 64 * seconds / dt)))
    rows = np.linspace(0, S - 1, n).astype(np.int32)
    t0 = time.perf_counter()
    rpy.apply_rows(Y, FT, rows, nthreads=cores)
    dt = time.perf_counter() - t0
    # the same oracle on one thread, on a sample 1/cores the size (about as long)
    n1 = max(16, n // cores)
    rows1 = np.linspace(0, S - 1, n1).astype(np.int32)
    t0 = time.perf_counter()
    rpy.apply_rows(Y, FT, rows1, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": n * S / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d target rows x %d sources of one mobility apply (%.1f s)" % (n, S, dt),
            "single_thread": {"value": n1 * S / dt1, "cores": 1,
                              "sample": "%d target rows x %d sources (%.1f s)" % (n1, S, dt1)}}


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
    wl, base, t, mu, Fext, follower = workload()
    S = 1000 * 32
    Y = np.concatenate([base[i] + np.arange(32)[:, None] * wl.dL * t[i] for i in range(1000)])
    FT = np.random.default_rng(1).standard_normal((S, 6))
    prec = fil.FIL_MIXED if args.precision == "mixed" else fil.FIL_FP64
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
    print(json.dumps({"workload": "mobility apply, 32000 segments", "precision": args.precision,
                      "pair_kernel_ms": avg, "pairs_per_s": S * S / (avg * 1e-3),
                      "tflops": FLOPS_PER_PAIR * S * S / (avg * 1e-3) / 1e12,
                      "autotuned": tuned}), flush=True)


def run_ensemble(args, fil, torch):
    """Batched ensemble: 256 independent suspensions in one context (one launch
    per kernel, per-system Broyden); JSON line with aggregate and per-system
    rates."""
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
    m = fil.Filaments(segs, fil_per_sys=fps, a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT,
                      dt=wl.dt, tol=wl.tol, max_iter=args.ens_max_iter, precision=fil.FIL_MIXED,
                      j0_model=j0, stream=stream.cuda_stream)
    m.init_straight(base, t, mu, None)
    m.set_external(Fext, None, follower)
    m.set_graph(args.graph)
    for _ in range(args.warmup):
        m.step()
    tuned = m.autotune(2) if args.tune else None
    a0, i0, k0 = m.counters()
    p0 = m.pair_count()
    torch.cuda.synchronize()
    clk = clocks_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters, sys_iters = [], []
    e0.record(stream)
    for _ in range(args.steps):
        iters.append(m.step())
        sys_iters.append(m.sys_stats()[0].copy())
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clocks_stop(clk, 0)
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
    m.close()
    # pairs actually evaluated (converged systems drop out of the applies)
    achieved = FLOPS_PER_PAIR * pairs_prof / (pair_ms * 1e-3) / 1e12
    pair_avg = pair_ms / max(n_pair, 1)
    print(json.dumps({
        "metric": METRIC, "value": pairs / (ms * 1e-3), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "ensemble of %d independent suspensions, filaments U[1,64] x "
                               "segments U[16,48] (%d filaments, %d segments), physics of the "
                               "32k suspension" % (n_sys, len(segs), int(S_sys.sum())),
                   "j0": "filament_rpy" if j0 == fil.FIL_J0_FILAMENT_RPY else "drag",
                   "pairs_per_apply": pairs_per_apply, "parallelism": "single"},
        "timesteps_per_s_per_system": args.steps / (ms * 1e-3),
        "system_timesteps_per_s": n_sys * args.steps / (ms * 1e-3),
        "broyden_iters_per_step": {"max_over_systems": float(np.mean(iters)),
                                   "mean_over_systems": float(si.mean()),
                                   "p90_over_systems": float(np.percentile(si, 90))},
        "roofline": {"kernel": "rpy_pair32", "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "avg_launch_ms": pair_avg,
                     "launches": int(n_pair), "measured_over": "2 steps without graphs"},
        "graph": bool(args.graph),
        "autotuned": ({"tile": tuned[0], "ctas_per_sm": tuned[1], "ms_per_apply": tuned[2]}
                      if tuned else None),
        "gpu_launches": int(k1 - k0), "clocks": clocks}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--plain-steps", type=int, default=2,
                    help="timed steps of the plain FP64 form for comparison (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--j0", default="filament_rpy", choices=["filament_rpy", "drag"],
                    help="approximate Jacobian: filament RPY blocks (default) or App. B.2 drag")
    ap.add_argument("--n-fil", type=int, default=1000,
                    help="filaments of 32 segments (1000 = the 32k suspension; smaller for profiling)")
    ap.add_argument("--warm", default="prediction_first",
                    choices=["prediction_first", "best_of_two", "off"],
                    help="learned warm start of each step (the committed network) and its mode")
    ap.add_argument("--n-sys", type=int, default=256, help="systems of the ensemble workload")
    ap.add_argument("--ens-max-iter", type=int, default=100)
    ap.add_argument("--tune", type=int, default=None,
                    help="autotune the pair kernel's schedule after the warm-up steps "
                         "(default: on for the ensemble, off for the single suspension, whose "
                         "default schedule is the tuned one)")
    ap.add_argument("--steric", type=float, default=0.0,
                    help="steric barrier strength F^S (Sec. 2.6, chi = 1.1); 0 = off")
    ap.add_argument("--graph", type=int, default=0,
                    help="run each Broyden iteration as one CUDA graph launch (ensemble; off by "
                         "default: with kernels of 0.05-0.7 ms the launches are not the cost and "
                         "the graph's speculative last iteration is)")
    ap.add_argument("--workload", default="suspension",
                    choices=["suspension", "mobility", "ensemble", "peaks"],
                    help="'mobility': only RPY applies on the 32k configuration (for profiling); "
                         "'peaks': the measured FP32 / FP64 FMA rates beside the derived ones")
    args = ap.parse_args()
    if args.tune is None:
        args.tune = 1 if args.workload == "ensemble" else 0

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
        return
    if args.workload == "peaks":
        run_peaks(args, fil)
        return
    if args.workload == "ensemble":
        run_ensemble(args, fil, torch)
        return
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
    prec = fil.FIL_MIXED if args.precision == "mixed" else fil.FIL_FP64
    j0 = fil.FIL_J0_FILAMENT_RPY if args.j0 == "filament_rpy" else fil.FIL_J0_DRAG
    params = dict(a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol,
                  max_iter=wl.max_iter, j0_model=j0)
    m = fil.Filaments(wl.seg_per_fil, precision=prec, stream=stream.cuda_stream, **params)
    m.init_straight(base, t, mu, None)
    m.set_external(Fext, None, follower)
    if args.steric > 0:
        m.set_steric(args.steric, 1.1)

    # learned warm start (chosen form): the committed network, trained on other seeds
    net, warm_mode = None, None
    if args.warm != "off" and prec == fil.FIL_MIXED:
        from paper_1903_12609_gb300 import warmstart
        if os.path.exists(warmstart.DEFAULT_WEIGHTS):
            net = warmstart.load(max_batch=max(64, n_fil), stream=stream.cuda_stream)
            warm_mode = (fil.FIL_WARM_PREDICTION_FIRST if args.warm == "prediction_first"
                         else fil.FIL_WARM_BEST_OF_TWO)
            fil.fil_warm_attach(m.ctx, net, warm_mode)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        m.step()
    tuned = m.autotune(5) if args.tune else None
    st0 = [np.zeros((S, 3)), np.zeros((S, 4)), np.zeros((S, 3)), np.zeros((S, 3)),
           np.zeros((S - n_fil, 3))]
    m.get_state(*st0)

    # ---- timed region: K steps, L2 flushed between steps ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    a0, i0, k0 = m.counters()
    m.profile(True)
    m.profile_read()
    barrier()
    clk = clocks_start()
    t_wall = time.perf_counter()
    iters = []
    with torch.cuda.stream(stream):
        for j in range(args.steps):
            flush.fill_(float(j))
            ev[j][0].record(stream)
            iters.append(m.step())
            ev[j][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = clocks_stop(clk, local)
    n_pair_launch, pair_ms = m.profile_read()
    m.profile(False)
    a1, i1, k1 = m.counters()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    dev_ms = float(sum(step_ms))
    applies = a1 - a0
    pairs = applies * float(S) * S
    local_val = pairs / (dev_ms * 1e-3)

    # whole-job aggregate: units of all ranks over the slowest rank's time
    tot_pairs, max_ms = aggregate_ranks(pairs, dev_ms, dist, "cuda")
    value = tot_pairs / (max_ms * 1e-3)

    # ---- dominant kernel: the RPY pair kernel, timed live by the library ----
    pair_avg_ms = pair_ms / max(n_pair_launch, 1)
    achieved = FLOPS_PER_PAIR * float(S) * S / (pair_avg_ms * 1e-3) / 1e12
    prof = counters_from_profile() if prec == fil.FIL_MIXED else {}
    traffic = prof.get("dram_bytes_per_launch")

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

    # ---- learned warm start vs extrapolation, both from the state before the timed steps ----
    warm = None
    if net is not None:
        warm = {"mode": args.warm, "weights": os.path.relpath(warmstart.DEFAULT_WEIGHTS, ROOT)}
        K = min(args.steps, 20)
        for name, use in (("extrapolation", False), ("learned", True)):
            m.set_state(*st0)
            fil.fil_warm_attach(m.ctx, net if use else None, warm_mode)
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            barrier()
            c0.record(stream)
            its = [m.step() for _ in range(K)]
            c1.record(stream)
            barrier()
            warm[name] = {"timesteps_per_s": K / (c0.elapsed_time(c1) * 1e-3),
                          "broyden_iters_per_step": float(np.mean(its)), "steps": K}
        fil.fil_warm_attach(m.ctx, None)
    m.close()
    if net is not None:
        fil.fil_mlp_destroy(net)

    # ---- plain FP64 form on the same workload (timesteps/s for comparison) ----
    plain = None
    if args.plain_steps > 0 and prec == fil.FIL_MIXED:
        mp = fil.Filaments(wl.seg_per_fil, precision=fil.FIL_FP64, stream=stream.cuda_stream,
                           **params)
        mp.set_state(Yh, qh, Yph, uh, lh)
        mp.set_external(Fext, None, follower)
        if args.steric > 0:
            mp.set_steric(args.steric, 1.1)
        barrier()
        pa0, _, _ = mp.counters()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.plain_steps):
            mp.step()
        p1.record(stream)
        barrier()
        pa1, _, _ = mp.counters()
        pms = p0.elapsed_time(p1)
        plain = {"timesteps_per_s": args.plain_steps / (pms * 1e-3),
                 "pairs_per_s": (pa1 - pa0) * float(S) * S / (pms * 1e-3),
                 "steps": args.plain_steps, "precision": "fp64"}
        mp.close()

    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return

    # measured FMA rates (after the timed region): context for the derived peak
    p32, mhz32 = fil.fil_fma_peak(False)
    p64, mhz64 = fil.fil_fma_peak(True)
    import __graft_entry__ as _g  # noqa: F401
    cpu = cpu_baseline(Yh, np.random.default_rng(2).standard_normal((S, 6)),
                       args.cpu_seconds) if world == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == fil.FIL_MIXED else "f64", "data": "synthetic",
        "config": {
            "workload": "suspension %d filaments x 32 segments (%d), 2%% volume fraction, "
                        "half sedimenting (B=1000) half tip-follower (fL^2/KB=100), BDF2 "
                        "dt=T/200, Broyden tol 1e-4" % (n_fil, S),
            "segments": S, "precision": args.precision, "j0": args.j0,
            "initial_guess": ("learned warm start (%s)" % args.warm) if net is not None
                             else "extrapolation",
            "steric_FS": args.steric if args.steric > 0 else None,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between timed steps (256 MiB write)"},
        "timesteps_per_s": args.steps / (max_ms * 1e-3),
        "warm_start": warm,
        "broyden_iters_per_step": float(np.mean(iters)),
        "mobility_applies": int(applies),
        "roofline": {"kernel": "rpy_pair32" if prec == fil.FIL_MIXED else "rpy_pair64",
                     "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS if prec == fil.FIL_MIXED else None,
                     "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS if prec == fil.FIL_MIXED else None,
                     "traffic": traffic, "flops_per_pair": FLOPS_PER_PAIR,
                     "fma_pipe_active": prof.get("fma_pipe_active"),
                     "avg_launch_ms": pair_avg_ms, "launches": int(n_pair_launch),
                     "share_of_step": pair_ms / dev_ms if dev_ms > 0 else None,
                     "peak_note": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (derived)",
                     "peak_measured": {
                         "fp32_tflops": p32 / 1e12, "fp32_sm_mhz": mhz32,
                         "fp64_tflops": p64 / 1e12, "fp64_sm_mhz": mhz64,
                         "frac_of_measured": (achieved / (p32 / 1e12)
                                              if prec == fil.FIL_MIXED else None),
                         "how": "fil_fma_peak: packed FP32x2 / FP64 FMA chains, full "
                                "occupancy, 5 launches of ~20 ms"}},
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
    if plain is not None:
        plain["frac_of_measured_fp64_peak"] = plain["pairs_per_s"] * FLOPS_PER_PAIR / p64
        line["plain_fp64"] = plain
        line["mixed_over_plain_timesteps"] = line["timesteps_per_s"] / plain["timesteps_per_s"]
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

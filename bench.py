"""Benchmark of the quantum-trajectory hot path: trajectory-steps per second at N = 4096.

Workload (uniform batch): singlet Gaussian S wave (width 0.2 GeV^-1), Coulomb 2S and Gaussian P
wave initial states in equal numbers for each (kappa_hat, gamma_hat) in {4,5,6} x {-3.5,0}, grid
N = 4096, L = 40 GeV^-1, dt = 0.001 GeV^-1, M = 4.65 GeV, alpha_s = 0.3, Bjorken cooling from
0.425 GeV at 0.6 fm/c to 0.25 GeV (11,899 steps): 180,000 trajectories.  Trajectory t has initial
state t % 3, medium (t // 3) % 6 and seed t; bench step i evolves the i-th slice of `--batch` of them
(a multiple of 18, so every slice has the same pattern of (initial state, medium) pairs) through its
whole medium: one qtraj_evolve, i.e. one launch of the fused kernel whose first work items are the
no-jump runs of the 18 groups.  The metric counts executed trajectory-steps only (rMin short-cuts
count zero, the no-jump runs count, and so does a trajectory taken up before its group's p_NoJump
was known, which runs its whole medium).

Timing: W warm-up steps, then exactly K steps between a barrier + synchronize on both sides,
measured with CUDA events on the launching stream; the maximum over ranks is reported.  A 256 MiB
buffer is written between steps to flush L2.  `e2e` repeats the measurement through the C ABI
with host buffers: the step's descriptors are uploaded from host memory by qtraj_evolve and its
observables copied back to pinned host memory inside the timed region.

`--impl reference` times the plain CPU oracle on this host's cores (the arm the ratio is taken
against): every step evolves one trajectory per core of the same workload through the first
~2,500 steps of its medium.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "traj-steps/s at N=4096 vs plain FP64 GPU form at stated error; p99 request latency"
UNIT = "traj-steps/s"
N_GRID, L_BOX, DT = 4096, 40.0, 0.001
# DRAM traffic of fused_kernel<float, 4096, 0> from two ncu captures of the current kernel source
# (608 trajectories through 300 and through 1000 steps; dram__bytes_read.sum + dram__bytes_write.sum):
# a launch costs a fixed part (the first touch of the tables) plus a part per trajectory-step (the
# per-step tables that fall out of L2).  None until the kernel has been captured again after a change.
PROFILED_DRAM_FIXED_BYTES = 1.107e6
PROFILED_DRAM_BYTES_PER_TRAJ_STEP = 2.63
N_STEPS_FULL = 11899          # ceil((tau_f - tau0) / (hbar c dt)) for the Bjorken medium 0.425 -> 0.25 GeV at tau0 = 0.6 fm/c


def workload_config(batch):
    return {"workload": "uniform batch N=4096 L=40 dt=0.001 1S/2S/1P x kappa{4,5,6} x gamma{-3.5,0}, "
                        "Bjorken 0.425->0.25 GeV (11899 steps)",
            "N": N_GRID, "L": L_BOX, "dt": DT, "trajectories_per_step": batch, "precision": "fp32 fused",
            "l2": "flushed between steps (256 MiB write); state lives on chip"}


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
def fp32_peak_tflops(sm_count, mhz=2070.0):
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def algorithmic_flops_per_step(N):
    """FP32 flops of one trajectory-step of the method as implemented: two sine transforms, each an
    N-point complex FFT (5 N log2 N) plus pre/post-processing and the odd-coefficient prefix sum
    (12 N), the kinetic factor (6 N), two space half-steps (12 N each) and the norm (4 N)."""
    lg = int(np.log2(N))
    return 2 * (5 * N * lg + 12 * N) + 6 * N + 2 * 12 * N + 4 * N


def nominal_flops_per_step(N):
    """The nominal count of the odd-extended length-2N transform pair: 10 (2N) log2(2N) + pointwise."""
    return 10 * 2 * N * int(np.log2(2 * N)) + 30 * N


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2107_06147_gb300 import inputs, qtraj

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = inputs.uniform_interleaved(per_group=10000, N=N_GRID, L=L_BOX, dt=DT)
    total = w.n_traj
    B = (args.batch // 18) * 18
    specs = [qtraj.init_spec(s.kind, s.width, s.n, s.l, s.color) for s in w.inits]
    media = [qtraj.medium(m.T0, m.tau0, m.Tf, m.kappa_hat, m.gamma_hat) for m in w.media]
    prec = qtraj.FP32 if args.precision == "fp32" else qtraj.FP64
    eng = qtraj.Engine(qtraj.Config(N=N_GRID, L=L_BOX, dt=DT, precision=prec, form=qtraj.FUSED,
                                    variant=args.variant))
    n_slices = total // B

    # every rank owns disjoint trajectory ids: step i of rank r takes slice (i*world + r) mod n_slices
    def slice_ids(i):
        return np.arange(B) + ((i * world + rank) % n_slices) * B

    eng.init(specs, B, spec_idx=w.init_idx[slice_ids(0)])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    obs_host = torch.empty(B * qtraj.OBS_DTYPE.itemsize, dtype=torch.uint8).pin_memory()

    def step(i, e2e=False):
        ids = slice_ids(i)
        eng.evolve(media, w.seeds[ids], w.medium_idx[ids], stream=stream)
        if e2e:
            st = eng.lib.qtraj_observables(eng.ctx, qtraj.C.c_void_p(obs_host.data_ptr()), 0,
                                           qtraj.C.c_void_p(stream.cuda_stream))
            qtraj._check(st, eng.ctx)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for i in range(args.warmup):
        step(i)
    barrier()
    kinfo = eng.kernel_info()

    # ---- device-timed region ------------------------------------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    steps_exec, launches, kernel_ms = 0, 0, 0.0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for i in range(args.warmup, args.warmup + args.steps):
        step(i)
        flush.fill_(i & 255)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    # the counters (executed steps, launches, per-launch event times) are read in the e2e pass, which
    # evolves the same slices again; executed steps are deterministic per slice
    # ---- end-to-end region through host buffers ---------------------------------------------------
    barrier()
    t0 = time.perf_counter()
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    main_ms = []
    for i in range(args.warmup, args.warmup + args.steps):
        step(i, e2e=True)
        s = eng.stats()
        steps_exec += s.steps_executed
        launches += s.launches
        main_ms.append(s.ms_main)
        kernel_ms += s.ms_main + s.ms_nojump
        flush.fill_(i & 255)
    ev3.record(stream)
    barrier()
    e2e_ms = ev2.elapsed_time(ev3)

    t_local = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=dev)
    cnt = torch.tensor([steps_exec], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    ms, e2e_ms = float(t_local[0]), float(t_local[1])
    total_steps = float(cnt[0])
    value = total_steps / (ms / 1e3)
    e2e_value = total_steps / (e2e_ms / 1e3)

    # roofline of the dominant kernel (the fused FP32 kernel; one launch per step, the groups' no-jump
    # runs included): the nominal flops of the odd-extended length-2N transform pair, 10 (2N)
    # log2(2N) + pointwise = 1,187,840 per trajectory-step at N = 4096, over that kernel's event time,
    # against the FP32 FMA peak from unit counts (SMs x 128 lanes x 2 flops x 2070 MHz); the flops the
    # implementation needs (an N-point FFT per sine transform, half the nominal) go beside it
    main_steps = steps_exec
    nominal = nominal_flops_per_step(N_GRID)
    alg = algorithmic_flops_per_step(N_GRID)
    achieved = main_steps * nominal / (sum(main_ms) / 1e3) / 1e12
    achieved_alg = main_steps * alg / (sum(main_ms) / 1e3) / 1e12
    peak = fp32_peak_tflops(kinfo.sm_count)
    # DRAM bytes of one main launch from the two captures: fixed part + per-trajectory-step part x the
    # launch's executed trajectory-steps
    traffic = None
    if args.precision == "fp32" and args.variant == 0 and PROFILED_DRAM_BYTES_PER_TRAJ_STEP is not None:
        traffic = round(PROFILED_DRAM_FIXED_BYTES + PROFILED_DRAM_BYTES_PER_TRAJ_STEP * main_steps / args.steps)
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "traffic_note": "DRAM bytes per launch: fixed + per-trajectory-step parts from ncu captures of this kernel (608 trajectories x 300 and x 1000 steps)",
                "flops_per_traj_step": nominal,
                "flops_note": "nominal 10 (2N) log2(2N) + 30 N of the odd-extended transform pair",
                "algorithmic_flops_per_traj_step": alg, "algorithmic_tflops": round(achieved_alg, 3),
                "algorithmic_frac": round(achieved_alg / peak, 4),
                "peak_note": "FP32 FMA peak from unit counts: SMs x 128 lanes x 2 flops x 2070 MHz"}
    if rank == 0:
        fma = qtraj.fma_peak(qtraj.FP32)
        roofline["fma_rate_measured_tflops"] = round(fma, 2)   # context: an FMA microbenchmark on this GPU

    result = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64"}[args.precision],
              "data": "synthetic",
              "config": workload_config(B) | {"parallelism": f"replicas x{world} (disjoint trajectory ids)"},
              "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                      # staged per evolve: a 24-byte record per trajectory and per (state, medium)
                      # group (18), a 104-byte record per medium (6)
                      "h2d_bytes_per_step": int(B * 24 + 18 * 24 + 6 * 104),
                      "d2h_bytes_per_step": int(B * qtraj.OBS_DTYPE.itemsize + 4)},
              "gpu_launches": int(launches), "roofline": roofline, "clocks": clk,
              "kernel": {"threads_per_traj": kinfo.threads_per_traj, "ctas_per_sm": kinfo.ctas_per_sm,
                         "smem_bytes": kinfo.smem_bytes, "regs": kinfo.regs_per_thread, "radix": kinfo.radix,
                         "variant": args.variant}}

    # the comparison forms, the CPU baseline and serving are single-GPU measurements: with N > 1 they
    # would hold every GPU at the final barrier, so they run at N = 1 only
    if rank == 0 and world == 1 and not args.no_compare:
        # the FP64 forms at two batch sizes, to show whether their throughput has plateaued; the
        # speed-up is quoted against the faster of the two plain FP64 rates
        for k, form in (("plain_fp64", qtraj.PLAIN), ("fused_fp64", qtraj.FUSED)):
            result[k] = measure_form(qtraj, w, specs, media, qtraj.FP64, form, args.compare_batch)
            big = measure_form(qtraj, w, specs, media, qtraj.FP64, form, 2 * args.compare_batch)
            result[k]["value_at_double_batch"] = big["value"]
        best_plain = max(result["plain_fp64"]["value"], result["plain_fp64"]["value_at_double_batch"])
        result["speedup_vs_plain_fp64"] = round(value / world / best_plain, 2)
        result["speedup_note"] = (f"fused FP32 at {B} trajectories per step against the faster plain FP64 rate of "
                                  f"{args.compare_batch} and {2 * args.compare_batch} trajectories")
        # the FP64 forms are bound by GB300's FP64 pipe: their algorithmic rate against the FP64 FMA
        # throughput measured on the same GPU
        fma64 = qtraj.fma_peak(qtraj.FP64)
        result["fp64_fma_peak_measured_tflops"] = round(fma64, 3)
        for k in ("plain_fp64", "fused_fp64"):
            t = result[k]["value"] * alg / 1e12
            result[k]["tflops"] = round(t, 4)
            result[k]["frac_of_measured_fp64_fma"] = round(t / fma64, 4)
        # the DFT16 blocks on the tensor cores against the CUDA cores: per-pass rate, the
        # transform-only ceiling it puts on trajectory-steps/s, and the 64-pass error
        from paper_2107_06147_gb300 import tcstudy
        st = tcstudy.run(batches=912, passes=32, reps=2)
        result["dft16_forms"] = {
            "note": "radix-16 DFT blocks as CUDA-core butterflies or mma.sync split forms; the ceiling is a "
                    "step that did nothing but its sine transforms (1536 column-DFTs per trajectory-step)",
            **{k: {"ns_per_column": v["ns_per_column"],
                   "transform_only_traj_steps_per_s_ceiling": v["transform_only_traj_steps_per_s_ceiling"],
                   "rel_err_64pass_rms": v["rel_err_64pass_rms"]} for k, v in st["forms"].items()}}
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(args)
    if rank == 0 and world == 1 and not args.no_serving:
        eng.close()
        result["serving"] = run_serving(args)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if eng.ctx:
        eng.close()
    if rank == 0:
        print(json.dumps(result))


def run_uneven(args):
    """Throughput of the uneven-batch workload: --uneven trajectories with N drawn from
    {1024, 2048, 4096, 8192} (L = N * 5/512), l0 in {0, 1, 2} (Gaussian singlets of width 0.2),
    T0 ~ U[0.30, 0.60] GeV from tau0 = 0.6 fm/c to 0.25 GeV, kappa_hat ~ U[3, 7], gamma_hat ~ U[-3.5, 0],
    seeds = ids (PCG64 seed 0), all grid sizes launched together on concurrent streams (batching.py).
    Every trajectory has its own medium, so the rMin shortcut (one no-jump run per (state, medium)
    group) would double the work: it is off.  One JSON line."""
    import torch

    from paper_2107_06147_gb300 import batching, inputs, qtraj
    u = inputs.uneven(n_traj=args.uneven, seed=0)
    inits = [qtraj.init_spec("gauss", 0.2, 1 + int(l), int(l), 0) for l in u["l0"]]
    media = [qtraj.medium(float(u["T0"][i]), 0.6, 0.25, float(u["kappa_hat"][i]), float(u["gamma_hat"][i]))
             for i in range(args.uneven)]
    prec = qtraj.FP32 if args.precision == "fp32" else qtraj.FP64
    w = batching.UnevenBatch(u["N"][:64], inits[:64], media[:64], precision=prec, use_rmin=0)
    w.run(u["seeds"][:64])   # loads every kernel instantiation before the timed run
    w.close()
    b = batching.UnevenBatch(u["N"], inits, media, precision=prec, use_rmin=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    obs = b.run(u["seeds"])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = b.stats()
    b.close()
    steps = int(obs["n_steps_exec"].sum())
    per_n = {int(N): {"trajectories": int(s.n_traj), "traj_steps": int(s.steps_executed), "kernel_ms": round(s.ms_main, 1)}
             for N, s in st.items()}
    print(json.dumps({"uneven": True, "trajectories": args.uneven, "precision": args.precision, "traj_steps": steps,
                      "wall_s": round(wall, 2), "traj_steps_per_s": round(steps / wall, 1), "per_N": per_n,
                      "jumps_mean": round(float(obs["n_jumps"].mean()), 2)}))


def run_ksu(args):
    """Throughput of the isotropic KSU potential (App. E; no jumps, H_eff evolution of singlets) at
    N = 4096, L = 40, dt = 0.001: --ksu trajectories of Gaussian 1S and 1P singlets (width 0.2) in the
    benchmark's Bjorken medium 0.425 -> 0.25 GeV (11,899 steps), m_D factor 1, in the FP32 and FP64
    fused forms (one untimed evolve first).  One JSON line."""
    import torch

    from paper_2107_06147_gb300 import qtraj
    n = args.ksu
    specs = [qtraj.init_spec("gauss", 0.2, 1, 0, 0), qtraj.init_spec("gauss", 0.2, 2, 1, 0)]
    idx = (np.arange(n) % 2).astype(np.int32)
    media = [qtraj.medium(0.425, 0.6, 0.25, 0.0, 0.0)]
    out = {"ksu": True, "N": N_GRID, "trajectories": n, "medium": "Bjorken 0.425 -> 0.25 GeV, m_D factor 1"}
    for name, prec in (("fp32", qtraj.FP32), ("fp64", qtraj.FP64)):
        e = qtraj.Engine(qtraj.Config(N=N_GRID, L=L_BOX, dt=DT, precision=prec, potential=1, ksu_mD_factor=1.0))
        e.init(specs, n, idx)
        seeds = np.arange(n, dtype=np.uint64)
        e.evolve(media, seeds, np.zeros(n, np.int32))
        torch.cuda.synchronize()
        e.evolve(media, seeds, np.zeros(n, np.int32))
        torch.cuda.synchronize()
        st = e.stats()
        ki = e.kernel_info()
        e.close()
        out[name] = {"traj_steps": int(st.steps_executed), "ms": round(st.ms_main, 1),
                     "traj_steps_per_s": round(st.steps_executed / (st.ms_main / 1e3), 1),
                     "ctas_per_sm": ki.ctas_per_sm, "regs": ki.regs_per_thread}
    print(json.dumps(out))


def _serve_once(args, rate_hz, order):
    """Replays the first --serving-requests requests of the stream, their arrival gaps rescaled from
    200 req/s to rate_hz, with the given launch order; returns the summary dict."""
    import torch

    from paper_2107_06147_gb300 import inputs, qtraj, serving
    st = inputs.serving_prefix(args.serving_requests)
    arrival = st["arrival_s"] * (200.0 / rate_hz)
    reqs = serving.requests_from_stream(st)
    Ns = sorted(set(int(n) for n in st["N"]))
    srv = serving.Server(Ns=tuple(Ns), slots_per_n=2, wave_mult=4,
                         order=qtraj.ORDER_SHORTEST if order == "shortest" else qtraj.ORDER_ARRIVAL)
    torch.cuda.synchronize()
    wall = srv.run_stream(reqs, arrival)
    log = srv.launch_log()
    srv.close()
    lat = serving.latency_stats(reqs)
    steps = int(sum(int(r.obs["n_steps_exec"].sum()) for r in reqs))
    # device concurrency: the fraction of the busy time during which launches of two or more slots ran
    ev = sorted([(t, +1) for t in log["start_ms"]] + [(t, -1) for t in log["end_ms"]])
    busy = multi = 0.0
    depth, last = 0, None
    for t, d in ev:
        if last is not None and depth > 0:
            busy += t - last
            if depth > 1:
                multi += t - last
        depth += d
        last = t
    return {"requests": len(reqs), "n_latencies": lat["n"], "order": order, "offered_rate_hz": rate_hz,
            "latency_p50_s": round(lat["p50_s"], 3), "latency_p99_s": round(lat["p99_s"], 3),
            "latency_mean_s": round(lat["mean_s"], 3), "latency_max_s": round(lat["max_s"], 3),
            "wall_s": round(wall, 3), "traj_steps": steps, "traj_steps_per_s": round(steps / wall, 1),
            "completed_rate_hz": round(len(reqs) / wall, 4), "Ns": Ns, "launches": int(len(log)),
            "concurrent_fraction": round(multi / busy, 3) if busy > 0 else None,
            "trajectories": int(sum(r.ntraj for r in reqs)), "precision": "fp32 fused, rMin shortcut off"}


def run_serving_sweep(args):
    """The first --serving-requests requests of the stream replayed at each offered rate of
    --serving-sweep (the arrival gaps of the 200 req/s stream rescaled): latency against offered load,
    down to a rate one GPU sustains, for the launch order(s) of --serving-order.  One JSON line per
    (rate, order)."""
    orders = ("arrival", "shortest") if args.serving_order == "both" else (args.serving_order,)
    for rate in [float(r) for r in args.serving_sweep.split(",")]:
        for order in orders:
            print(json.dumps({"serving_sweep": True, **_serve_once(args, rate, order)}), flush=True)


def run_serving(args):
    """p50/p99 request latency of the continuous-batching loop on the first --serving-requests of the
    Poisson request stream (200 req/s, seed 1; initial state in {1S, 2S, 1P}, kappa ~ U[3,7],
    gamma ~ U[-3.5,0], T0 ~ U[0.3,0.6] GeV Bjorken to 0.25 GeV, ntraj log-uniform in [64, 4096],
    N in {1024, ..., 16384} with L = N * 5/512, dt = 0.001).  The offered rate far exceeds one GPU's
    service rate, so latency includes queueing behind the earlier requests; n_latencies is the number
    of request latencies the percentiles are taken over."""
    order = "shortest" if args.serving_order == "shortest" else "arrival"
    return _serve_once(args, 200.0, order)


def measure_form(qtraj, w, specs, media, prec, form, B):
    """Trajectory-steps/s of another form on the first B trajectories of the workload (one evolve)."""
    import torch
    eng = qtraj.Engine(qtraj.Config(N=N_GRID, L=L_BOX, dt=DT, precision=prec, form=form))
    ids = np.arange(B)
    eng.init(specs, B, spec_idx=w.init_idx[ids])
    eng.evolve(media, w.seeds[ids], w.medium_idx[ids])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng.evolve(media, w.seeds[ids], w.medium_idx[ids])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    s = eng.stats()
    eng.close()
    ms = s.ms_main + s.ms_nojump
    return {"value": round(s.steps_executed / (ms / 1e3), 1), "unit": UNIT, "trajectories": B,
            "traj_steps": int(s.steps_executed), "ms": round(ms, 1), "wall_s": round(wall, 2)}


# ------------------------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline)
# ------------------------------------------------------------------------------------------------
def oracle_sample(n_traj, prefix_steps=2500, seed_offset=0):
    """Evolves n_traj trajectories of the workload (1S Gaussian, kappa 5, gamma 0 group) through the
    first prefix_steps steps of the Bjorken medium with the oracle; returns (traj-steps, seconds, cores)."""
    import oracle as orc
    threads = os.cpu_count() or 1
    g = orc.Grid(N=N_GRID, L=L_BOX, dt=DT, use_rmin=0)
    T0, tau0 = 0.425, 0.6
    if prefix_steps >= N_STEPS_FULL:
        Tf = 0.25
    else:
        tau_end = tau0 + prefix_steps * DT * 0.1973269804
        Tf = T0 * (tau0 / tau_end) ** (1.0 / 3.0) * (1 + 1e-9)
    m = orc.medium(T0, tau0, Tf, 5.0, 0.0)
    spec = orc.init_spec("gauss", 0.2, 1, 0, 0)
    seeds = np.arange(n_traj, dtype=np.uint64) + seed_offset
    t0 = time.perf_counter()
    obs, _, _ = orc.run_batch(g, [spec], np.zeros(n_traj, np.int32), [m], np.zeros(n_traj, np.int32), seeds,
                              n_threads=threads)
    dt = time.perf_counter() - t0
    return int(obs["n_steps_exec"].sum()), dt, threads


def cpu_baseline(args):
    """Two trajectories per host core through the whole Bjorken medium (11,899 steps): ~10-20 s of
    oracle work on a 16-core host."""
    cores = os.cpu_count() or 1
    steps, secs, thr = oracle_sample(2 * cores, prefix_steps=N_STEPS_FULL)
    return {"value": round(steps / secs, 1), "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"{2 * cores} trajectories (two per core) of the 1S/kappa=5/gamma=0 group, N=4096, "
                      f"all {steps // (2 * cores)} steps of the Bjorken medium 0.425->0.25 GeV, "
                      f"plain FP64 C oracle, {secs:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as orc
    orc.build()
    cores = os.cpu_count() or 1
    for i in range(args.warmup):
        oracle_sample(cores, prefix_steps=300, seed_offset=10_000 * (i + 1))
    tot_steps, tot_s = 0, 0.0
    for i in range(args.steps):
        s, t, thr = oracle_sample(cores, seed_offset=i * cores)
        tot_steps += s
        tot_s += t
    value = tot_steps / tot_s
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot_s / args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(cores) | {"precision": "fp64 CPU oracle",
                                               "sample": "one trajectory per core, first ~2500 steps"},
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{cores} trajectories per step, first ~2500 steps of the medium"},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_profile_case(args):
    """One evolve of --batch trajectories of the workload through the first --profile-steps steps of
    the medium (the fused kernel's steady state at a size a profiler can replay quickly)."""
    import torch

    from paper_2107_06147_gb300 import inputs, qtraj
    NG = args.profile_n
    LB = NG * L_BOX / N_GRID          # the same dr as the bench workload
    w = inputs.uniform_interleaved(per_group=10000, N=NG, L=LB, dt=DT)
    probe = qtraj.Engine(qtraj.Config(N=NG, L=LB, dt=DT, precision=qtraj.FP32 if args.precision == "fp32"
                                      else qtraj.FP64, variant=args.variant))
    ki = probe.kernel_info()
    probe.close()
    # one full wave of CTAs unless --batch is given explicitly
    B = args.batch if args.batch_given else ki.sm_count * ki.ctas_per_sm
    tau_end = 0.6 + args.profile_steps * DT * 0.1973269804
    media = [qtraj.medium(m.T0, m.tau0, m.T0 * (m.tau0 / tau_end) ** (1 / 3) * (1 + 1e-9), m.kappa_hat, m.gamma_hat)
             for m in w.media]
    prec = qtraj.FP32 if args.precision == "fp32" else qtraj.FP64
    eng = qtraj.Engine(qtraj.Config(N=NG, L=LB, dt=DT, precision=prec, form=qtraj.FUSED, use_rmin=0,
                                    variant=args.variant))
    specs = [qtraj.init_spec(s.kind, s.width, s.n, s.l, s.color) for s in w.inits]
    eng.init(specs, B, spec_idx=w.init_idx[:B])
    for _ in range(2):
        eng.evolve(media, w.seeds[:B], w.medium_idx[:B])
    torch.cuda.synchronize()
    s = eng.stats()
    print(json.dumps({"profile_case": True, "N": NG, "trajectories": B, "steps_executed": int(s.steps_executed),
                      "ms": round(s.ms_main, 3), "traj_steps_per_s": round(s.steps_executed / (s.ms_main / 1e3), 1)}))
    eng.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=9216, help="trajectories per bench step (multiple of 18)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--compare-batch", type=int, default=1024)
    ap.add_argument("--variant", type=int, default=0, help="fused kernel occupancy variant (0 or 1)")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=16)
    ap.add_argument("--serving-order", default="arrival", choices=["arrival", "shortest", "both"],
                    help="order of the admitted trajectories of a grid size in a launch")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one small evolve for a profiler: --batch trajectories, --profile-steps steps")
    ap.add_argument("--profile-steps", type=int, default=1000)
    ap.add_argument("--profile-n", type=int, default=N_GRID, help="grid size of --profile-case (dr of the bench workload)")
    ap.add_argument("--uneven", type=int, default=0, metavar="NTRAJ",
                    help="throughput of the uneven-batch workload (NTRAJ trajectories of mixed N, l, lifetime)")
    ap.add_argument("--serving-sweep", default="", metavar="RATES",
                    help="comma-separated offered rates (req/s): replay the --serving-requests prefix at each")
    ap.add_argument("--ksu", type=int, default=0, metavar="NTRAJ",
                    help="throughput of the isotropic KSU potential at N=4096 (NTRAJ trajectories, FP32 and FP64)")
    ap.add_argument("--precision-study", type=int, default=0, metavar="NTRAJ",
                    help="paired FP64/FP32 study on NTRAJ trajectories of N=8192, L=80, dt=0.0005 (no timing line)")
    args = ap.parse_args()
    args.batch_given = any(a.startswith("--batch") for a in sys.argv[1:])
    if args.uneven:
        from paper_2107_06147_gb300 import build
        build.build()
        run_uneven(args)
        return
    if args.serving_sweep:
        from paper_2107_06147_gb300 import build
        build.build()
        run_serving_sweep(args)
        return
    if args.ksu:
        from paper_2107_06147_gb300 import build
        build.build()
        run_ksu(args)
        return
    if args.precision_study:
        from paper_2107_06147_gb300 import build, inputs, precision
        build.build()
        print(json.dumps(precision.run(inputs.precision(n_traj=args.precision_study))))
        return
    if args.profile_case:
        from paper_2107_06147_gb300 import build
        build.build()
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2107_06147_gb300 import build
        import oracle
        build.build()
        oracle.build()
        run_ours(args)


if __name__ == "__main__":
    main()

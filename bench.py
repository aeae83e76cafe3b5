"""Benchmark of the ensemble-SDE hot path on GB300.

Default workload: the batched Josephson sweep (Eq. 1 over 512 parameter points,
uneven path and step counts, one persistent graph-captured launch, FP64
on-device reductions).  One step = one full sweep from the initial state:
Philox4x32-10 + Box-Muller noise, SRK2 (Alg. 2) for every path of every point,
window averages and the FP64 ensemble reduction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sweep|plain|kuramoto-meanfield|kuramoto-pairwise]

Prints one JSON line (rank 0).  Under torchrun each rank integrates its own copy
of the workload (a different noise seed), with no data-path collective: weak
scaling.  `--impl reference` times the FP64 CPU oracle on a bounded sample of
the same workload on this host's cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0903_3852_gb300 import dist as sde_dist  # noqa: E402
from paper_0903_3852_gb300 import inputs  # noqa: E402

PAPER_FLOP_PER_STEP = 79  # Table 1 (Appendix): FLOP per SRK2 step of Eq. 1, weighted
# FP32 operations per SRK2 path-step of the Josephson kernels as the hardware
# counts them (ncu: 2 x FFMA + FADD + FMUL, the packed FP32x2 forms counting
# both lanes): the same arithmetic in every launch variant.  The paper's
# weighting above counts each transcendental as several FLOP; these kernels
# take them from tables and polynomials, so the counted figure is the
# roofline's numerator and the weighted one is reported beside it.
COUNTED_FLOP_PER_PATH_STEP = 52.27
PAPER_FLOP_MEANFIELD = 66  # Fig. 5: operations per step of PROG3 (Eq. 3, mean field)
PAPER_FLOP_PAIR = 6  # Fig. 5: 44 + 6N operations per step of PROG2, 6 per pair term
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "plain", "kuramoto-meanfield", "kuramoto-pairwise",
                             "kuramoto-general", "kuramoto-general-fp32", "surrogate", "surrogate-inference", "fig2",
                             "kuramoto-fig4", "fig2-fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pairwise-steps", type=int, default=200,
                    help="steps per bench step of the pairwise Kuramoto workload")
    ap.add_argument("--fig4-steps", type=int, default=None,
                    help="kuramoto-fig4: steps per bench step (default: the workload's 2000)")
    ap.add_argument("--cluster", type=int, default=0,
                    help="kuramoto-meanfield: CTAs per replica (with --block: skips autotuning)")
    ap.add_argument("--async-exchange", action="store_true",
                    help="kuramoto-meanfield: cluster exchange by st.async + mbarrier only")
    ap.add_argument("--schedule", choices=["auto", "plain", "persistent"], default="auto",
                    help="Josephson workloads: persistent sweep launch (default except 'plain') or one "
                         "launch per point with one thread per path (the plain per-path kernel)")
    ap.add_argument("--euler", action="store_true",
                    help="Euler-Maruyama (PROG2's scheme) instead of SRK2: Josephson workloads and kuramoto-pairwise")
    ap.add_argument("--fp64-steps", type=int, default=20_000,
                    help="fig2-fp64: steps of the FP64 run per bench step (the Fig. 2 run has 2e5)")
    ap.add_argument("--general-steps", type=int, default=0,
                    help="steps per bench step of the general-coupling workloads "
                         "(default: all 5000 for BF16, 100 for the FP32 baseline)")
    # reduced cases for profiler captures (not bench lines)
    ap.add_argument("--points", type=int, default=0, help="sweep: keep only the first N points")
    ap.add_argument("--steps-cap", type=int, default=0, help="sweep: cap every point's step count")
    ap.add_argument("--block", type=int, default=0, help="fixed threads per block (skips autotuning)")
    ap.add_argument("--ilp", type=int, default=0,
                    help="fixed Josephson launch variant, skipping the autotuner: 1, 2 or 4 paths per "
                         "thread, 11 / 12 / 14 the same with fewer registers")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="sweep: skip the plain per-path kernel comparison of the default line")
    ap.add_argument("--separate-stage", action="store_true",
                    help="general coupling, tensor-core form: SRK2 sub-steps as separate kernels instead of "
                         "in the GEMM epilogue (the default)")
    ap.add_argument("--gemm-single-cta", action="store_true",
                    help="general coupling, tensor-core form: whole tiles, one CTA per 128 x 256 GEMM tile")
    ap.add_argument("--gemm-stream-k", action="store_true",
                    help="general coupling, tensor-core form: split the K range of all tiles over every "
                         "resident CTA (stream-K) instead of whole tiles")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- workloads
def sweep_workload(rank, args=None):
    w = inputs.josephson_sweep()
    # each rank integrates its own copy with its own noise key (weak scaling)
    w["seed"] = sde_dist.rank_seed(w["seed"], rank)
    if args is not None and (args.points or args.steps_cap):
        k = args.points or len(w["points"])
        n = int(w["paths"][:k].sum())
        w["points"], w["paths"], w["x0"], w["v0"] = w["points"][:k], w["paths"][:k], w["x0"][:n], w["v0"][:n]
        w["steps"] = w["steps"][:k]
        if args.steps_cap:
            w["steps"] = np.minimum(w["steps"], args.steps_cap)
    return w


def josephson_workload_name(args, w):
    name = {"sweep": "josephson_sweep_%dpts" % len(w["points"]), "plain": "josephson_plain_1024",
            "fig2": "josephson_fig2_524288paths_2e5steps"}[args.workload]
    if args.steps_cap:
        name += "_cap%d" % args.steps_cap
    if args.euler:
        name += "_euler"
    return name


def kuramoto_workload_name(workload, euler, n_osc, replicas):
    if workload.startswith("kuramoto-general"):
        kind = "bf16_tcgen05" if workload == "kuramoto-general" else "fp32_cudacore"
        return "kuramoto_general_%s_N%d_R%d" % (kind, n_osc, replicas)
    form = "fig4_meanfield_grid" if workload == "kuramoto-fig4" else workload.split("-")[1]
    suffix = "_euler_prog2" if euler and workload == "kuramoto-pairwise" else ""
    return "kuramoto_%s_N%d_R%d%s" % (form, n_osc, replicas, suffix)


def josephson_sizes(w):
    return {"points": len(w["points"]), "total_paths": int(w["paths"].sum()),
            "path_steps": float((w["paths"] * w["steps"]).sum()), "steps_per_period": w["steps_per_period"]}


def plain_workload(rank):
    w = inputs.josephson_plain()
    w["seed"] = sde_dist.rank_seed(w["seed"], rank)
    return w


def fig2_workload(rank):
    w = inputs.josephson_fig2()
    w["seed"] = sde_dist.rank_seed(w["seed"], rank)
    return w


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "of measured (MEASURED_PEAKS.json)"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


def fp64_peak_tflops(props):
    # 2 DFMA per SM per clock (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
    # peak_sustained), 2 FLOP each, at 2070 MHz
    return props.multi_processor_count * 2 * 2 * 2.070e9 / 1e12


def fp32_peak_tflops(props):
    # 128 FP32 lanes per SM on Blackwell, one FMA (2 FLOP) per lane per clock,
    # at the maximum SM clock of 2070 MHz.
    return props.multi_processor_count * 128 * 2 * 2.070e9 / 1e12


def measure_fp32_peak(device, launches=6, target_ms=60.0):
    """The FP32 peak measured on this GPU: the library's FMA probe (eight
    independent FFMA2 chains per thread, 8 blocks of 256 threads per SM),
    timed with CUDA events on the launching stream; best launch, with the SM
    clock sampled meanwhile."""
    import torch
    from paper_0903_3852_gb300 import sde
    props = torch.cuda.get_device_properties(device)
    grid, block = props.multi_processor_count * 8, 256
    sink = torch.empty(grid * block, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream()

    def one(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flop = sde.fp32_fma_probe(1, iters, grid, block, sink, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return flop, e0.elapsed_time(e1)

    iters = 1024
    for _ in range(2):
        _, t = one(iters)
        iters = max(1, int(iters * target_ms / max(t, 1e-3)))
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.3)
    best = 0.0
    for _ in range(launches):
        flop, t = one(iters)
        best = max(best, flop / (t * 1e-3) / 1e12)
    clk = clocks.stop()
    return {"tflops": best, "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"),
            "derived_2070mhz": fp32_peak_tflops(props),
            "probe": "FFMA2 chains, %d blocks x %d threads, best of %d launches of ~%.0f ms"
                     % (grid, block, launches, target_ms)}


def host_cpu_model():
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_ours(args, rank, world, device):
    import torch
    from paper_0903_3852_gb300 import build as sde_build
    from paper_0903_3852_gb300 import sde

    sde_build.build()
    props = torch.cuda.get_device_properties(device)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    if args.workload in ("sweep", "plain", "fig2"):
        w = {"sweep": lambda r: sweep_workload(r, args), "plain": plain_workload,
             "fig2": fig2_workload}[args.workload](rank)
        plain = args.schedule == "plain" or (args.schedule == "auto" and args.workload == "plain")
        sched = sde.SDE_SCHED_PLAIN if plain else sde.SDE_SCHED_PERSISTENT
        ens = sde.Ensemble.josephson(w["points"], w["paths"], w["steps"], w["seed"],
                                     steps_per_period=w["steps_per_period"], schedule=sched,
                                     block_threads=args.block, paths_per_thread=args.ilp,
                                     flags=sde.SDE_FLAG_EULER if args.euler else 0)
        n = int(w["paths"].sum())
        units = float((w["paths"] * w["steps"]).sum())
        n_end = int(w["steps"].max())
        x_h = torch.from_numpy(w["x0"]).pin_memory()
        v_h = torch.from_numpy(w["v0"]).pin_memory()
        x_in, v_in = x_h.to(device), v_h.to(device)
        x_out = torch.empty_like(x_in)
        v_out = torch.empty_like(v_in)
        w_out = torch.empty(n, dtype=torch.int32, device=device)
        vs_out = torch.empty(n, dtype=torch.float64, device=device)

        def step():
            ens.run_josephson(0, n_end, x_in, v_in, x_out, v_out, w_out, vs_out)

        def step_e2e():
            x_in.copy_(x_h, non_blocking=True)
            v_in.copy_(v_h, non_blocking=True)
            step()
            return ens.observables()

        h2d = x_h.numel() * 4 + v_h.numel() * 4
        d2h = 40 * len(w["points"])
        launches_per_step = (1 if sched == sde.SDE_SCHED_PERSISTENT else len(w["points"])) + 1
        launches_kernel = 1  # the timed region brackets the per-step launches as one
        metric = "path-steps/sec"
        flop_per_unit = PAPER_FLOP_PER_STEP
        name = josephson_workload_name(args, w)
        if args.workload != "plain" and sched == sde.SDE_SCHED_PLAIN:
            name += "_plain_per_point"
        cfg = {"workload": name, **josephson_sizes(w),
               "schedule": "persistent+graph" if sched == sde.SDE_SCHED_PERSISTENT else "plain per point",
               "tuning": dict(zip(("block_threads", "paths_per_thread", "cluster_ctas"), ens.tuning())),
               "l2": "flushed between steps (256 MiB write); state 9 MB, compute-bound"}
    elif args.workload == "fig2-fp64":
        # the Fig. 2 ensemble in double precision on the GPU (Sec. 5's DP run),
        # shortened to --fp64-steps steps
        w = fig2_workload(rank)
        S = args.fp64_steps
        n = int(w["paths"][0])
        pt = w["points"][0]
        P = w["steps_per_period"]
        x_h = torch.from_numpy(w["x0"].astype(np.float64)).pin_memory()
        v_h = torch.from_numpy(w["v0"].astype(np.float64)).pin_memory()
        x_in, v_in = x_h.to(device), v_h.to(device)
        x_out, v_out = torch.empty_like(x_in), torch.empty_like(v_in)
        vs_out = torch.empty_like(x_in)
        v_back = torch.empty(n, dtype=torch.float64).pin_memory()

        class _Timed:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)

            def close(self):
                pass

            def last_kernel_stats(self):
                self.e1.synchronize()
                t = self.e0.elapsed_time(self.e1)
                return t, t, 1

        ens = _Timed()

        def step():
            ens.e0.record(stream)
            sde.josephson_run_fp64(pt, P, S, w["seed"], 0, S, x_in, v_in, x_out, v_out, vsum_out=vs_out,
                                   stream=stream)
            ens.e1.record(stream)

        def step_e2e():
            x_in.copy_(x_h, non_blocking=True)
            v_in.copy_(v_h, non_blocking=True)
            step()
            v_back.copy_(v_out, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            return v_back

        h2d = 16 * n
        d2h = 8 * n
        units = float(n * S)
        metric = "path-steps/sec"
        launches_per_step = 1
        flop_per_unit = PAPER_FLOP_PER_STEP
        flop_per_launch = flop_per_unit * units
        cfg = {"workload": "josephson_fig2_fp64_%dpaths_%dsteps" % (n, S), "precision": "fp64 throughout",
               "steps_per_period": P, "full_run_steps": int(w["steps"][0]),
               "l2": "flushed between steps (256 MiB write); state 8 MB, compute-bound"}
    elif args.workload in ("kuramoto-meanfield", "kuramoto-pairwise", "kuramoto-fig4"):
        fig4 = args.workload == "kuramoto-fig4"
        w = inputs.kuramoto_fig4(seed=rank) if fig4 else inputs.kuramoto_uniform(seed=rank)
        model = sde.SDE_KURAMOTO_PAIRWISE if args.workload == "kuramoto-pairwise" else sde.SDE_KURAMOTO_MEANFIELD
        S = w["steps"] if model == sde.SDE_KURAMOTO_MEANFIELD else args.pairwise_steps
        if fig4 and args.fig4_steps:
            S = args.fig4_steps
        euler = args.euler and model == sde.SDE_KURAMOTO_PAIRWISE
        mf_shape = {} if fig4 or model != sde.SDE_KURAMOTO_MEANFIELD else \
            dict(block_threads=args.block, cluster_ctas=args.cluster)
        ens = sde.Ensemble.kuramoto(model, w["n_osc"], w["replicas"], w["K"], w["D"], w["dt"], w["seed"],
                                    sample_every=w["sample_every"],
                                    flags=sde.SDE_FLAG_TIME_KERNELS | (sde.SDE_FLAG_EULER if euler else 0)
                                    | (sde.SDE_FLAG_ASYNC_EXCHANGE if args.async_exchange else 0),
                                    **mf_shape)
        phi_h = torch.from_numpy(w["phi0"]).pin_memory()
        phi_in = phi_h.to(device)
        om = torch.from_numpy(w["omega"]).to(device)
        phi_out = torch.empty_like(phi_in)

        def step():
            ens.run_kuramoto(0, S, phi_in, phi_out, om)

        def step_e2e():
            phi_in.copy_(phi_h, non_blocking=True)
            step()
            return ens.observables()

        h2d = phi_h.numel() * 4
        d2h = 40 * (S // w["sample_every"] + 1)
        if fig4:
            units = float(w["n_osc"] * w["replicas"] * S)
            metric = "oscillator-steps/sec"
            launches_per_step = 2 * S + 4
            # 152 B per oscillator per 4 steps (noise-drawing predictor 28, predictor 20
            # three times, corrector 16 four times): 19 B per launch on average
            bytes_per_launch = 19.0 * w["n_osc"] * w["replicas"]
        elif model == sde.SDE_KURAMOTO_MEANFIELD:
            units = float(w["n_osc"] * w["replicas"] * S)
            metric = "oscillator-steps/sec"
            flop_per_unit = PAPER_FLOP_MEANFIELD
            launches_per_step = 4
            flop_per_launch = flop_per_unit * units
        else:
            units = float(w["n_osc"] ** 2 * w["replicas"] * S)
            metric = "pair-terms/sec"
            flop_per_unit = PAPER_FLOP_PAIR
            launches_per_step = 2 * S + S // w["sample_every"] + 4
            flop_per_launch = flop_per_unit * w["n_osc"] ** 2 * w["replicas"]  # one stage launch
        cfg = {"workload": kuramoto_workload_name(args.workload, euler, w["n_osc"], w["replicas"]),
               "steps_per_bench_step": S, "K": w["K"], "D": w["D"], "dt": w["dt"],
               "tuning": dict(zip(("block_threads", "oscillators_per_thread", "cluster_ctas"), ens.tuning())),
               "l2": "flushed between steps (256 MiB write)"}
    else:
        w = inputs.kuramoto_general(seed=rank)
        tc = args.workload == "kuramoto-general"
        model = sde.SDE_KURAMOTO_GENERAL if tc else sde.SDE_KURAMOTO_GENERAL_FP32
        S = args.general_steps or (w["steps"] if tc else 100)
        N, R = w["n_osc"], w["replicas"]
        fused = tc and not args.separate_stage
        flags = (sde.SDE_FLAG_TIME_KERNELS | (sde.SDE_FLAG_FUSED if fused else 0)
                 | (sde.SDE_FLAG_GEMM_SINGLE_CTA if args.gemm_single_cta else 0)
                 | (sde.SDE_FLAG_GEMM_STREAM_K if args.gemm_stream_k else 0))
        ens = sde.Ensemble.kuramoto(model, N, R, 0.0, w["D"], w["dt"], w["seed"],
                                    sample_every=w["sample_every"], flags=flags)
        Kdev = torch.from_numpy(w["Kmat"]).to(device)
        ens.set_coupling(Kdev)
        del Kdev
        phi_h = torch.from_numpy(w["phi0"]).pin_memory()
        phi_in = phi_h.to(device)
        om = torch.from_numpy(w["omega"]).to(device)
        phi_out = torch.empty_like(phi_in)

        def step():
            ens.run_kuramoto(0, S, phi_in, phi_out, om)

        def step_e2e():
            phi_in.copy_(phi_h, non_blocking=True)
            step()
            return ens.observables()

        h2d = phi_h.numel() * 4
        d2h = 40 * (S // w["sample_every"] + 1)
        units = float(N * R * S)
        metric = "oscillator-steps/sec"
        flop_per_launch = 2.0 * N * (2 * R) * N  # one GEMM K . [sin | cos]
        # per step two GEMMs (+ two stage kernels unless fused); r(t) samples;
        # the operand kernel, the last sample and the flush
        launches_per_step = (2 if fused else 4) * S + S // w["sample_every"] + 4
        cfg = {"workload": kuramoto_workload_name(args.workload, False, N, R),
               "stage": "fused into the GEMM epilogue" if fused else "separate kernel",
               "steps_per_bench_step": S, "K0": w["K0"], "D": w["D"], "dt": w["dt"],
               "gemm": "M=%d N=%d K=%d per stage, 2 per step" % (N, 2 * R, N),
               "gemm_tiling": ({0: "stream-K: 128 x 256 tiles, K split over %d CTAs (tcgen05 cta_group::1)"
                                   % ens.tuning()[1],
                                2: "256 x 256 per CTA pair (tcgen05 cta_group::2)",
                                1: "128 x %d per CTA (tcgen05 cta_group::1)" % ens.tuning()[1]}[ens.tuning()[2]]
                               if tc else "128 x 128 per CTA (FP32 FMA)"),
               "l2": "K matrix %d MiB streams each GEMM; flushed between steps (256 MiB write)"
                     % (N * N * (2 if tc else 4) >> 20)}

    # warm-up (also captures the graph)
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(device if isinstance(device, int) else torch.cuda.current_device())
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kernel_ms = []
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        kernel_ms.append(ens.last_kernel_stats()[0])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        import torch.distributed as dist
        ms = sde_dist.max_over_ranks(ms, device=torch.device("cuda", device))
        dist.barrier()

    # end to end through the public API with host buffers
    e2e_ms = []
    for _ in range(0 if args.no_e2e else max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_e2e()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = statistics.median(e2e_ms) if e2e_ms else None

    extra = {}
    if args.workload == "fig2":
        # the coarse-grained distribution of Fig. 2 (right): 200 bins, one potential
        # period each, the window centred on the median winding number
        w_lo = int(np.median(w_out.cpu().numpy())) - 100
        counts = ens.position_histogram(w_out, w_lo, 200).cpu().numpy()[0]
        extra["fig2_histogram"] = {"w_lo": w_lo, "bins": 200, "below": int(counts[0]),
                                   "above": int(counts[-1]), "counts": [int(c) for c in counts[1:-1]],
                                   "paper_seconds_c1060_fp32": 20.0}
    if args.workload == "kuramoto-fig4":
        # the density P(x; t) of Fig. 4 at the end of the run, and r against
        # the mean-field self-consistency r = I1(K r / D) / I0(K r / D)
        nb = 100
        counts = sde.phase_histogram(phi_out.reshape(-1), nb).cpu().numpy()
        obs = ens.observables()
        extra["fig4"] = {"r_end": float(obs["mean"][-1]), "r_theory": 0.8314620247541972,
                         "histogram_bins": nb, "counts": [int(c) for c in counts],
                         "paper_seconds_c1060_fp32": 20.0}
    if args.workload == "kuramoto-general" and world == 1:
        extra["library_gemm_same_shape"] = library_gemm_same_shape(N, R, device)
    k_ms = statistics.mean(kernel_ms)
    peaks, peak_src = measured_peaks()
    fp32 = measure_fp32_peak(device)
    if args.workload == "kuramoto-fig4":
        bound, peak = "hbm", peaks["hbm_gbs"]
        peak_note = "HBM copy bandwidth, %s" % peak_src
        flop_note = "19 B per oscillator per launch (38 B per oscillator-step over the predictor and corrector launches)"
    elif args.workload == "fig2-fp64":
        bound, peak = "alu", fp64_peak_tflops(props)
        peak_note = "%d SM x 2 DFMA x 2 FLOP x 2070 MHz (derived)" % props.multi_processor_count
        flop_note = "%d FLOP per path-step (paper Table 1 weighting), in FP64" % flop_per_unit
    elif args.workload == "kuramoto-general":
        bound, peak = "tensor", peaks["bf16_tflops_sustained"]
        peak_note = "bf16 dense, sustained, %s" % peak_src
        flop_note = "2 N (2R) N FLOP per GEMM launch"
    else:
        bound, peak = "alu", fp32["tflops"]
        peak_note = ("FP32 FMA probe measured in this run (%.1f TFLOP/s at %s MHz; %.1f derived from 128 "
                     "lanes x 2 FLOP x 2070 MHz)" % (fp32["tflops"], fp32["sm_mhz"], fp32["derived_2070mhz"]))
        flop_note = ("2 N (2R) N FLOP per GEMM launch (FP32 FMA)" if args.workload == "kuramoto-general-fp32"
                     else "%d FLOP per unit (paper Table 1 weighting)" % flop_per_unit)
    counted = args.workload in ("sweep", "plain", "fig2") and not args.euler
    if args.workload in ("sweep", "plain", "fig2"):
        if counted:
            flop_per_unit = COUNTED_FLOP_PER_PATH_STEP
            flop_note = ("%.2f FP32 FLOP per path-step counted by ncu (2 x FFMA + FADD + FMUL, packed "
                         "instructions both lanes)" % flop_per_unit)
        flop_per_launch = flop_per_unit * units / launches_kernel
    if args.workload == "kuramoto-fig4":
        achieved = bytes_per_launch / (k_ms * 1e-3) / 1e9
    else:
        achieved = flop_per_launch / (k_ms * 1e-3) / 1e12
    # DRAM bytes per launch of the dominant kernel, dram__bytes_read.sum +
    # dram__bytes_write.sum of one ncu capture of that kernel (scaled by the
    # units where the capture was smaller); null where the kernel changed since
    traffic, traffic_src = None, None
    if args.workload in ("sweep", "plain", "fig2") and not args.euler:
        traffic = 8.23 * n  # 8.23 B per path: the initial state read once
        traffic_src = "ncu capture of the sweep kernel (2000-step cap), scaled by paths"
    elif args.workload == "kuramoto-fig4":
        traffic = 16.6 * w["n_osc"] * w["replicas"]  # mean over the launches of 4 steps
        traffic_src = "ncu capture of the grid-wide mean-field launches"
    elif (args.workload == "kuramoto-general" and fused and not args.gemm_single_cta
          and not args.gemm_stream_k):
        traffic = 179.4e6  # K (134 MB) once, the operand and the SRK2 state of the epilogue
        traffic_src = ("ncu capture of the fused CTA-pair GEMM (mean of its predictor and corrector "
                       "launches)")
    elif args.workload == "kuramoto-meanfield":
        traffic = 2.26e6  # phases and omega read once per run; results stay in L2
        traffic_src = "ncu capture of the asynchronous-exchange cluster mean-field kernel"
    elif args.workload == "kuramoto-pairwise" and not args.euler:
        traffic = 2.11e6
        traffic_src = "ncu capture of the pairwise stage kernel"
    res = {
        "metric": metric,
        "value": sde_dist.aggregate_rate(units, world, ms * 1e-3),
        "unit": metric.split("/")[0] + "/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": vs_paper(args, sde_dist.aggregate_rate(units, world, ms * 1e-3)),
        "dtype": "f64" if args.workload == "fig2-fp64" else "f32 (FP64 reductions)",
        "data": "synthetic (seeded; inputs.py)",
        "config": cfg,
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak,
                     "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                     "flop_model": flop_note,
                     "peak_source": peak_note, "kernel_ms_per_launch": k_ms,
                     "fp32_peak_probe": fp32},
        "e2e": {"value": units * world / (e2e * 1e-3) if e2e else None, "unit": metric.split("/")[0] + "/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    if counted:
        res["roofline"]["frac_paper_weighted_79flop"] = (PAPER_FLOP_PER_STEP * units / launches_kernel
                                                         / (k_ms * 1e-3) / 1e12 / peak)
    if args.workload == "sweep" and not args.euler and not args.no_plain and world == 1 and sched != sde.SDE_SCHED_PLAIN:
        res["plain_vs_batched"] = plain_comparison(args, device, res["value"], fp32["tflops"])
    res.update(extra)
    return res, ens


def library_gemm_same_shape(N, R, device, reps=20):
    """The same product as one general-coupling GEMM (N x N times N x 2R, BF16
    operands) through torch.matmul (cuBLAS), timed with CUDA events after
    warm-up: a library reference point for the tensor-core GEMM, outside the
    timed region (median of `reps` launches; random operands)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(0)
    A = torch.randn(N, N, device=device, dtype=torch.bfloat16, generator=g)
    B = torch.randn(N, 2 * R, device=device, dtype=torch.bfloat16, generator=g)
    for _ in range(5):
        A @ B
    ts = []
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        A @ B
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    t = statistics.median(ts)
    del A, B
    return {"shape": [N, 2 * R, N], "us": t * 1e3, "tflops": 2.0 * N * N * 2 * R / (t * 1e-3) / 1e12,
            "how": "torch.matmul, BF16 operands and output (cuBLAS), median of %d launches, CUDA events" % reps}


def plain_comparison(args, device, batched_rate, peak):
    """The plain per-path kernel (one thread per path, scalar FP32: Alg. 1 as
    the paper writes it) against the batched form, at the same accuracy (the
    same arithmetic: every launch variant gives the same bits): (a) at a size
    that fills the GPU, the Fig. 2 ensemble of 2^19 paths in one launch, 2e4
    of its 2e5 steps; (b) on the sweep itself, one plain launch per point."""
    import torch
    from paper_0903_3852_gb300 import sde
    out = {}
    cases = [("saturating", fig2_workload(0), 20_000), ("per_point_sweep", sweep_workload(0, args), None)]
    for name, w, cap in cases:
        if cap:
            w["steps"] = np.minimum(w["steps"], cap)
        ens = sde.Ensemble.josephson(w["points"], w["paths"], w["steps"], w["seed"],
                                     steps_per_period=w["steps_per_period"], schedule=sde.SDE_SCHED_PLAIN,
                                     paths_per_thread=1)
        n = int(w["paths"].sum())
        units = float((w["paths"] * w["steps"]).sum())
        n_end = int(w["steps"].max())
        x = torch.from_numpy(w["x0"]).to(device)
        v = torch.from_numpy(w["v0"]).to(device)
        xo, vo = torch.empty_like(x), torch.empty_like(v)
        wo = torch.empty(n, dtype=torch.int32, device=device)
        so = torch.empty(n, dtype=torch.float64, device=device)
        ens.run_josephson(0, n_end, x, v, xo, vo, wo, so)  # warm-up
        ms = []
        for _ in range(2):
            ens.run_josephson(0, n_end, x, v, xo, vo, wo, so)
            ms.append(ens.last_kernel_ms())
        t = min(ms) * 1e-3
        rate = units / t
        out[name] = {"workload": josephson_workload_name(args, w) if name == "per_point_sweep"
                     else "josephson_fig2_%dpaths_%dsteps" % (n, n_end),
                     "kernel": "one thread per path, scalar FP32", "launches": len(w["points"]),
                     "tuning_block_threads": ens.tuning()[0], "path_steps": units, "value": rate,
                     "unit": "path-steps/s", "frac": COUNTED_FLOP_PER_PATH_STEP * rate / 1e12 / peak,
                     "batched_over_plain": batched_rate / rate}
        ens.close()
    return out


# The paper's own figures for the exact workloads it timed (NVIDIA Tesla C1060,
# another machine: context, not a target): the Fig. 2 ensemble, 2^19 paths x
# 2e5 steps, in 20 s single precision and 13 min double precision.
PAPER_RATE = {"fig2": 2 ** 19 * 2e5 / 20.0, "fig2-fp64": 2 ** 19 * 2e5 / (13 * 60.0)}


def vs_paper(args, value):
    ref = PAPER_RATE.get(args.workload)
    if ref is None or args.euler or args.schedule == "plain":
        return None
    return value / ref


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker_init(_):
    import oracle
    oracle.lib()
    return 0


def _oracle_jj_task(task):
    """One oracle task in a worker process: a chunk of paths of one point."""
    import oracle
    pt, x0, v0, P, S, seed, k, path0 = task
    oracle.jj_run(x0, v0, oracle.jj_params(**pt), P, 0, S, S, seed, point=k, path0=path0)
    return float(len(x0) * S)


def _oracle_kur_task(task):
    """One oracle task in a worker process: one Kuramoto replica."""
    import oracle
    phi0, omega, D, dt, S, seed, r, Kconst, meanfield, units = task
    oracle.kuramoto_run(phi0, omega, D, dt, 0, S, seed, r, Kconst=Kconst, meanfield=meanfield)
    return units


class OracleTimer:
    """The FP64 oracle timed on all host cores: one process per core (spawn
    context, safe after CUDA initialisation), each running the unchanged oracle
    on disjoint paths or replicas of the workload; the sample is sized from the
    single-core rate to take about `budget_s` seconds."""

    def __init__(self):
        import multiprocessing as mp
        self.cores = host_cores()
        self.pool = None
        if self.cores > 1:
            self.pool = mp.get_context("spawn").Pool(self.cores)
            self.pool.map(_oracle_worker_init, range(self.cores))

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def run(self, args, rate1, budget_s=10.0):
        if self.pool is None:
            return None
        target = rate1 * self.cores * budget_s
        if args.workload in ("sweep", "plain", "fig2", "fig2-fp64"):
            w = {"sweep": sweep_workload, "plain": plain_workload, "fig2": fig2_workload,
                 "fig2-fp64": fig2_workload}[args.workload](0)
            if args.workload == "fig2-fp64":
                w["steps"] = np.array([args.fp64_steps], dtype=np.int64)
            offs = np.concatenate([[0], np.cumsum(w["paths"])])
            per_step = float(np.sum(w["steps"]))  # path-steps of one path at every point
            per_point = int(max(1, min(w["paths"].max(), round(target / per_step))))
            tasks = []
            for k, pt in enumerate(w["points"]):
                n = min(per_point, int(w["paths"][k]))
                S = int(w["steps"][k])
                for c in range(0, n, 16):
                    m = min(16, n - c)
                    a = int(offs[k]) + c
                    tasks.append((pt, w["x0"][a:a + m], w["v0"][a:a + m], w["steps_per_period"], S, w["seed"],
                                  k, c))
            t0 = time.perf_counter()
            done = sum(self.pool.map(_oracle_jj_task, tasks, chunksize=1))
            dt = time.perf_counter() - t0
            return {"value": done / dt, "unit": "path-steps/s", "cores": self.cores, "kind": "oracle",
                    "sample": "up to the first %d paths of each of %d points, full step counts (%.3g path-steps), "
                              "16-path tasks over %d processes" % (per_point, len(w["points"]), done, self.cores)}
        if args.workload in ("kuramoto-meanfield", "kuramoto-pairwise"):
            w = inputs.kuramoto_uniform()
            meanfield = args.workload == "kuramoto-meanfield"
            N, R = w["n_osc"], w["replicas"]
            per = N if meanfield else N * N
            S = int(max(1, min(w["steps"], round(target / (per * R)))))
            tasks = [(w["phi0"][r], w["omega"][r], w["D"], w["dt"], S, w["seed"], r, w["K"] / N, meanfield,
                      float(per * S)) for r in range(R)]
            t0 = time.perf_counter()
            done = sum(self.pool.map(_oracle_kur_task, tasks, chunksize=1))
            dt = time.perf_counter() - t0
            return {"value": done / dt, "unit": "oscillator-steps/s" if meanfield else "pair-terms/s",
                    "cores": self.cores, "kind": "oracle",
                    "sample": "all %d replicas, %d steps each, over %d processes" % (R, S, self.cores)}
        return None  # a single replica (Fig. 4) or the 512 MB K matrix per process: single core only


def cpu_baseline_both(args, budget_s=20.0):
    """Single-core oracle rate, and the all-core rate where the workload splits."""
    one = cpu_baseline(args, budget_s=budget_s)
    timer = OracleTimer()
    try:
        allc = timer.run(args, one["value"], budget_s=budget_s / 2)
    finally:
        timer.close()
    if allc is None:
        return one
    allc["single_core"] = one
    return allc


def cpu_baseline(args, budget_s=20.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload."""
    import oracle
    if args.workload in ("sweep", "plain", "fig2", "fig2-fp64"):
        w = {"sweep": sweep_workload, "plain": plain_workload, "fig2": fig2_workload,
             "fig2-fp64": fig2_workload}[args.workload](0)
        if args.workload == "fig2-fp64":
            w["steps"] = np.array([args.fp64_steps], dtype=np.int64)
        offs = np.concatenate([[0], np.cumsum(w["paths"])])
        per_point = {"sweep": 2, "plain": 64, "fig2": 256, "fig2-fp64": 1024}[args.workload]
        t0 = time.perf_counter()
        done = 0.0
        npts = 0
        for k, pt in enumerate(w["points"]):
            sl = slice(offs[k], offs[k] + min(per_point, int(w["paths"][k])))
            S = int(w["steps"][k])
            for c in range(sl.start, sl.stop, 16):
                cs = slice(c, min(c + 16, sl.stop))
                oracle.jj_run(w["x0"][cs], w["v0"][cs], oracle.jj_params(**pt), w["steps_per_period"], 0, S, S,
                              w["seed"], point=k, path0=int(c - offs[k]))
                done += (cs.stop - cs.start) * S
                if time.perf_counter() - t0 > budget_s:
                    break
            npts += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dt = time.perf_counter() - t0
        return {"value": done / dt, "unit": "path-steps/s", "cores": 1, "kind": "oracle",
                "sample": "up to the first %d paths of each of %d points, full step counts (%.3g path-steps)"
                          % (per_point, npts, done)}
    if args.workload.startswith("kuramoto-general"):
        w = inputs.kuramoto_general()
        K = w["Kmat"].astype(np.float64)
        t0 = time.perf_counter()
        S = 1
        oracle.kuramoto_run(w["phi0"][0], w["omega"][0], w["D"], w["dt"], 0, S, w["seed"], 0, Kmat=K)
        dt = time.perf_counter() - t0
        return {"value": w["n_osc"] * S / dt, "unit": "oscillator-steps/s", "cores": 1, "kind": "oracle",
                "sample": "replica 0 of %d, %d step (direct FP64 sum over K_ij, N = %d)"
                          % (w["replicas"], S, w["n_osc"])}
    if args.workload == "kuramoto-fig4":
        w = inputs.kuramoto_fig4()
        S = 2
        t0 = time.perf_counter()
        oracle.kuramoto_run(w["phi0"][0], w["omega"][0], w["D"], w["dt"], 0, S, w["seed"], 0,
                            Kconst=w["K"] / w["n_osc"], meanfield=True)
        dt = time.perf_counter() - t0
        return {"value": w["n_osc"] * S / dt, "unit": "oscillator-steps/s", "cores": 1, "kind": "oracle",
                "sample": "the full replica of %d oscillators, %d steps (mean-field form)" % (w["n_osc"], S)}
    w = inputs.kuramoto_uniform()
    meanfield = args.workload == "kuramoto-meanfield"
    S = 200 if meanfield else 2
    t0 = time.perf_counter()
    oracle.kuramoto_run(w["phi0"][0], w["omega"][0], w["D"], w["dt"], 0, S, w["seed"], 0,
                        Kconst=w["K"] / w["n_osc"], meanfield=meanfield)
    dt = time.perf_counter() - t0
    units = w["n_osc"] * S if meanfield else w["n_osc"] ** 2 * S
    unit = "oscillator-steps/s" if meanfield else "pair-terms/s"
    return {"value": units / dt, "unit": unit, "cores": 1, "kind": "oracle",
            "sample": "replica 0, %d steps" % S}


def reference_config(args, sample):
    """The reference arm's config: the workload as the GPU arm names and sizes
    it (Josephson workloads), plus the bounded sample the oracle ran."""
    if args.workload in ("sweep", "plain", "fig2"):
        w = {"sweep": lambda: sweep_workload(0, args), "plain": lambda: plain_workload(0),
             "fig2": lambda: fig2_workload(0)}[args.workload]()
        return {"workload": josephson_workload_name(args, w), **josephson_sizes(w), "sample": sample}
    if args.workload.startswith("kuramoto"):
        import inspect
        build = {"kuramoto-fig4": inputs.kuramoto_fig4, "kuramoto-general": inputs.kuramoto_general,
                 "kuramoto-general-fp32": inputs.kuramoto_general}.get(args.workload, inputs.kuramoto_uniform)
        prm = inspect.signature(build).parameters  # the default sizes, without building the inputs
        replicas = prm["replicas"].default if "replicas" in prm else 1
        return {"workload": kuramoto_workload_name(args.workload, args.euler, prm["n_osc"].default, replicas),
                "sample": sample}
    return {"workload": args.workload, "sample": sample}


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores, K bounded steps."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return None
    per = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    one = cpu_baseline(args, budget_s=min(per, 5.0))  # the single-core rate sizes the samples
    timer = OracleTimer()
    try:
        def step(budget):
            r = timer.run(args, one["value"], budget_s=budget)
            return r if r is not None else cpu_baseline(args, budget_s=budget)
        for _ in range(args.warmup):
            step(min(per, 3.0))
        vals = []
        last = None
        for _ in range(args.steps):
            last = step(per)
            vals.append(last["value"])
    finally:
        timer.close()
    v = statistics.mean(vals)
    metric = {"sweep": "path-steps/sec", "plain": "path-steps/sec", "fig2": "path-steps/sec",
              "fig2-fp64": "path-steps/sec",
              "kuramoto-meanfield": "oscillator-steps/sec", "kuramoto-pairwise": "pair-terms/sec",
              "kuramoto-fig4": "oscillator-steps/sec",
              "kuramoto-general": "oscillator-steps/sec",
              "kuramoto-general-fp32": "oscillator-steps/sec"}[args.workload]
    unit = last["unit"]
    res = {"impl": "reference", "metric": metric, "value": v, "unit": unit, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; inputs.py)",
           "config": reference_config(args, last["sample"]),
           "cpu_baseline": {"value": v, "unit": unit, "cores": last["cores"], "kind": "oracle",
                            "sample": last["sample"], "single_core": one, "cpu_model": host_cpu_model()},
           "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return res


def surrogate_inference(sur, points, device, batch=100_000, reps=20):
    """Inference throughput of the surrogate's ensemble at a batch of 10^5 points:
    the fused tensor-core forward and the CUDA-core forward, each timed with CUDA
    events on the launching stream over `reps` calls after 3 warm-ups; the
    tensor-pipe fraction counts the square layers' MACs (2 x 256 x 256 per point,
    layer and member) against the measured BF16 peak."""
    import torch
    stream = torch.cuda.current_stream()
    X = sur.features(points[:batch])
    B = X.shape[0]
    mlp = sur.mlp
    n_sq = mlp.cfg.n_hidden - 1
    flop_tc = 2.0 * 256 * 256 * n_sq * mlp.members * B
    peaks, src = measured_peaks()
    out = {"batch": B, "members": mlp.members}
    for name, tc in (("tensor_cores", True), ("cuda_cores", False)):
        mlp.use_tensor_cores(tc)
        for _ in range(3):
            mlp.forward(X)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            mlp.forward(X)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_batch": ms, "points_per_sec": B / (ms * 1e-3),
                     "square_layer_tflops": flop_tc / (ms * 1e-3) / 1e12}
    mlp.use_tensor_cores(True)
    mlp.check()
    tf = out["tensor_cores"]["square_layer_tflops"]
    out["tensor_pipe_frac"] = tf / peaks["bf16_tflops"]
    out["tensor_pipe_peak"] = "bf16 dense burst, %s (%.0f TFLOP/s)" % (src, peaks["bf16_tflops"])
    out["tensor_over_cuda_cores"] = out["cuda_cores"]["ms_per_batch"] / out["tensor_cores"]["ms_per_batch"]
    return out


def run_surrogate_inference(args, device):
    """Inference of the surrogate's ensemble (4 networks 5-256-256-256-1) at a
    batch of 10^5 parameter points: one bench step = one forward of the whole
    batch through the library's fused tensor-core kernel (features in HBM).
    The weights are the networks' seeded initial ones (the cost does not
    depend on their values)."""
    import torch
    from paper_0903_3852_gb300 import build as sde_build
    from paper_0903_3852_gb300 import surrogate

    sde_build.build()
    B = 100_000
    sur = surrogate.Surrogate(members=4, max_batch=131072, seed=3)
    pts = inputs.surrogate_points(B, seed=6)
    X = sur.features(pts)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    for _ in range(max(args.warmup, 0)):
        sur.mlp.forward(X)
    torch.cuda.synchronize()
    clocks = ClockSampler(device)
    clocks.start()
    ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sur.mlp.forward(X)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    sur.mlp.check()
    # end to end: features from host parameter points, the forward, the
    # mean and spread back to the host
    e2e = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sur.predict(pts)
        e2e.append(time.perf_counter() - t0)
    t = statistics.mean(ms) * 1e-3
    flop = 2.0 * 256 * 256 * 2 * 4 * B
    peaks, src = measured_peaks()
    return {
        "metric": "points/sec", "value": B / t, "unit": "points/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 operands, fp32 accumulation", "data": "synthetic (seeded; inputs.py)",
        "config": {"workload": "surrogate_inference_batch100000", "members": 4, "net": "5-256-256-256-1 SiLU",
                   "l2": "flushed between steps (256 MiB write)"},
        "roofline": {"bound": "tensor", "achieved": flop / t / 1e12, "peak": peaks["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": flop / t / 1e12 / peaks["bf16_tflops"], "traffic": None,
                     "flop_model": "2 x 256 x 256 FLOP per point, square layer and member (the tensor-core work)",
                     "peak_source": "bf16 dense burst, %s" % src, "kernel_ms_per_launch": t * 1e3},
        "e2e": {"value": B / statistics.median(e2e), "unit": "points/s", "h2d_bytes_per_step": 40 * B,
                "d2h_bytes_per_step": 8 * B},
        "gpu_launches": 3 * args.steps, "clocks": clk,
    }


def run_surrogate(args, device):
    """The learned surrogate of <<v>>: labels from the sweep engine (10^5 points x
    2048 paths x 2e4 steps), an ensemble of 4 networks trained by the library's
    kernels on 80,000 of them, an error model on 10,000 more, selective
    calibration on the last 10,000, then one bench step = answering 10^4 held-out
    points (network where its predicted error <= 1e-2, simulator at 8192 paths
    elsewhere)."""
    import torch
    from paper_0903_3852_gb300 import build as sde_build
    from paper_0903_3852_gb300 import surrogate

    sde_build.build()
    props = torch.cuda.get_device_properties(device)
    steps, tol = 20_000, 1e-2
    train = inputs.surrogate_points(100_000, seed=6)
    y, se, t_lab = surrogate.simulate(train, 2048, steps, seed=6)
    label_units = len(train) * 2048.0 * steps
    sur = surrogate.Surrogate(members=4, max_batch=131072, lr=2e-3, seed=3)
    t0 = time.perf_counter()
    sur.fit(train[:80_000], y[:80_000], epochs=120, batch=1024)
    sur.fit_error_model(train[80_000:90_000], y[80_000:90_000])
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    tau, cal_share = sur.calibrate(train[90_000:], y[90_000:], se[90_000:], tol, risk=5e-4)
    evalp = inputs.surrogate_points(10_000, seed=7)
    ref, ref_se, t_ref = surrogate.simulate(evalp, 8192, steps, seed=7)
    infer = surrogate_inference(sur, train, device)
    mlp_pps = infer["tensor_cores"]["points_per_sec"]
    for _ in range(max(args.warmup, 0)):
        out = sur.answer(evalp, tol, 8192, steps, seed=8)
    clocks = ClockSampler(device)
    clocks.start()
    times, kms = [], []
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = sur.answer(evalp, tol, 8192, steps, seed=8 + i)
        times.append(time.perf_counter() - t0)
        kms.append(surrogate.simulate.last_kernel_ms)
    clk = clocks.stop()
    err = np.abs(out["value"] - ref)
    ans = ~out["fallback"]
    ok = err <= tol + 3.0 * np.hypot(ref_se, np.where(ans, 0.0, out["predicted_error"]))
    t_step = statistics.mean(times)
    fb_units = float(out["fallback"].sum()) * 8192.0 * steps
    k_ms = statistics.mean(kms)
    achieved = PAPER_FLOP_PER_STEP * fb_units / (k_ms * 1e-3) / 1e12
    peak = measure_fp32_peak(device)["tflops"]
    return {
        "metric": "points/sec", "value": len(evalp) / t_step, "unit": "points/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 simulator, bf16 network (fp32 master)",
        "data": "synthetic (seeded; inputs.py)",
        "config": {"workload": "surrogate_10k_heldout", "train_points": 100_000, "label_paths": 2048,
                   "steps": steps, "fallback_paths": 8192, "tol": tol, "members": 4,
                   "net": "5-256-256-256-1 SiLU"},
        "surrogate": {"label_seconds": t_lab, "label_points_per_sec_2048_paths": len(train) / t_lab,
                      "label_path_steps_per_sec": label_units / t_lab, "fit_seconds": t_fit,
                      "mlp_points_per_sec": mlp_pps, "inference_batch_1e5": infer,
                      "calibration": {"log_error_threshold": tau, "answered_share": cal_share, "risk": 5e-4,
                                      "points": 10_000, "split": "ensemble 80k, error model 10k, calibration 10k"},
                      "simulator_points_per_sec_8192_paths": len(evalp) / t_ref,
                      "answered_by_network": float(ans.mean()),
                      "within_tol_all": float(ok.mean()),
                      "within_tol_network_answers": float(ok[ans].mean()) if ans.any() else None,
                      "median_abs_err_network_answers": float(np.median(err[ans])) if ans.any() else None,
                      "gain_vs_simulator_only": t_ref / t_step},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "flop_model": "79 FLOP per path-step (paper Table 1 weighting), fallback simulation",
                     "peak_source": "%d SM x 128 FP32 lanes x 2 FLOP x 2070 MHz (derived)"
                                    % props.multi_processor_count, "kernel_ms_per_launch": k_ms},
        "e2e": {"value": len(evalp) / t_step, "unit": "points/s", "h2d_bytes_per_step": 40 * len(evalp),
                "d2h_bytes_per_step": 8 * len(evalp)},
        # per step: features 1 + 4 members x (2 casts + 4 GEMMs) + spread 1; the fallback
        # simulation: prepare 1 + autotune 6 x 3 x 2 + persistent kernel + finalize
        "gpu_launches": (26 + 1 + 36 + 2) * args.steps, "clocks": clk,
    }


def main():
    args = parse()
    if args.impl == "reference":
        res = run_reference(args)
        if res is not None:
            print(json.dumps(res))
        return
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "surrogate-inference":
        res = run_surrogate_inference(args, local)
        if rank == 0:
            print(json.dumps(res))
        return
    if args.workload == "surrogate":
        res = run_surrogate(args, local)
        if rank == 0:
            print(json.dumps(res))
        return
    res, ens = run_ours(args, rank, world, local)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:  # the oracle baseline is a 1-GPU figure
            res["cpu_baseline"] = cpu_baseline_both(args)
            res["cpu_baseline"]["cpu_model"] = host_cpu_model()
        print(json.dumps(res))
    ens.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

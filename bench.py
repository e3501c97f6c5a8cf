#!/usr/bin/env python3
"""Gate-application throughput of random qudit circuits on GB300.

Workload (one step): a seeded random sequence of 200 gates -- each drawn
uniformly from {Haar-random d x d unitary, level-pair rotation with uniform
angle, clock Z, shift X, SUM or controlled-RY on a random ordered pair} -- is
applied to each of four complex64 states, d=2 n=28, d=3 n=17, d=4 n=14 and
d=5 n=12 (1.29e8 to 2.68e8 amplitudes, 1.0 to 2.1 GB each, every state far
larger than L2), through fused programs, followed by <N_q> of every qudit in
FP64.  Throughput is amplitude-updates/s: N x gates applied / time.

Reported alongside: HBM roofline of the fused tile kernel (bytes-weighted over
its launches in the timed region, CUDA events around every pass), the per-gate
strided-kernel GB/s sweep over gate kinds and target positions on d=3 n=17,
complex128 and unfused throughput, end-to-end throughput through the public
API with host buffers, SM clocks sampled during the timed region, and the
CPU oracle timed on the host cores on a bounded sample.

--impl reference times the CPU oracle (complex128, explicit loops, OpenMP over
independent amplitude groups) on the host cores on the same workload, each step
a bounded sample (one gate per state), and prints the same JSON line with
"impl": "reference".
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIZES = [(2, 28), (3, 17), (4, 14), (5, 12)]
N_GATES = 200
METRIC = "amplitude-updates/s (random 200-gate qudit circuits, fused)"
UNIT = "amplitude-updates/s"
WORKLOAD = "random-200-gate sequences on d=2 n=28, d=3 n=17, d=4 n=14, d=5 n=12 + <N_q> of every qudit"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip c128/unfused/sweep/e2e/cpu legs")
    ap.add_argument("--profile-case", nargs="?", const="3,17", default=None, metavar="D,N",
                    help="small run for ncu captures: one state (default d=3 n=17) complex64 only, no extras")
    ap.add_argument("--probe-host-memory", action="store_true",
                    help="time the end-to-end step with host buffers from torch pin_memory and from qf_host_alloc "
                         "(copies alone and with circuits) and print the per-step times; no bench line")
    args = ap.parse_args()
    if args.profile_case is not None:
        d, n = (int(x) for x in args.profile_case.split(","))
        if (d, n) not in SIZES:
            ap.error("--profile-case takes one of the bench sizes %s" % (SIZES,))
        args.profile_case = (d, n)
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job(ms_local, units_per_rank_step, steps, dist=None, device="cpu"):
    """(max timed-region ms over ranks, whole-job units/s).  Every rank runs
    the same per-rank work (weak scaling, independent replicas), so the job
    processes world x units_per_rank_step per step within the slowest rank's
    time."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms = float(t.item())
    return ms, units_per_rank_step * steps * world / (ms / 1e3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        # raw samples; QF_BENCH_CLOCKS_DIR keeps them somewhere other than the temp directory
        import tempfile
        self.path = os.path.join(os.environ.get("QF_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 "qf_bench_clocks_rank%d.csv" % device_index)

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, n = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            n += 1
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": n}


def kernel_hash():
    h = hashlib.sha256()
    # the fused passes run as tile kernels generated by qf_jit.cu
    for f in ("qf_jit.cu", "qf_gates.cu", "qf_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2409_17716_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_ratio():
    """DRAM bytes / algorithmic bytes of one tile-kernel launch from the
    committed ncu summary, or None if the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "k_tile_jit_traffic.json")
    try:
        with open(path) as f:
            j = json.load(f)
        if j.get("kernel_sha") != kernel_hash():
            return None
        return float(j["dram_bytes_per_launch"]) / float(j["algorithmic_bytes_per_launch"])
    except Exception:
        return None


# --------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np
    from oracle import sim
    from paper_2409_17716_gb300 import workloads as W

    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    sizes = SIZES if not args.profile_case else [args.profile_case]
    states, circuits, pos = [], [], []
    for d, n in sizes:
        states.append(sim.basis(d, n, 0))
        circuits.append(W.random_circuit(d, n, N_GATES))
        pos.append(0)

    def step():
        au = 0
        for i, (d, n) in enumerate(sizes):
            op = circuits[i][pos[i] % N_GATES]
            pos[i] += 1
            t, U = sim.op_matrix(op, d)
            sim.apply(states[i], d, n, t, U)
            au += d ** n
        return au

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    au = 0
    for _ in range(args.steps):
        au += step()
    dt = time.perf_counter() - t0
    value = au / dt
    sample = "one gate per state per step (the next gate of each 200-gate sequence), complex128 oracle"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "global_batch": len(sizes), "seq_len": None,
                       "parallelism": "cpu-oracle", "l2": "states larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- CPU baseline leg
def _err(got, want, tol=None, rel=False):
    import numpy as np
    got = np.asarray(got)
    want = np.asarray(want)
    e = {"max_abs": float(np.abs(got - want).max()) if want.size else 0.0}
    if rel:
        e["max_rel"] = float((np.abs(got - want) / np.maximum(1.0, np.abs(want))).max()) if want.size else 0.0
    if tol is not None:
        e["tol"] = tol
        e["within"] = bool(e["max_abs"] <= tol)
    return e


def cpu_baseline(keep, size=(3, 17)):
    """The oracle as it stands (complex128, explicit loops, OpenMP over
    independent amplitude groups) on the host cores, on bounded samples of
    the workloads, and the error of every GPU result it can check:

    * forward: the whole 200-gate d=3 n=17 sequence on all cores (timed: the
      line's value), compared amplitude by amplitude with the GPU's complex64
      and complex128 results of the same sequence; the first two gates again
      on one thread;
    * adjoint (d=3 n=14, 10 layers, 560 parameters): the oracle's derivative
      circuits for 4 parameters and its loss, against the GPU's complex64 and
      complex128 gradients (timed per parameter, extrapolated to 560);
    * batched and VQA: sampled circuits' losses and per-sample gradients.
    Returns (cpu_baseline record, error_vs_oracle record)."""
    import numpy as np
    from oracle import sim
    from paper_2409_17716_gb300 import workloads as W
    cores = os.cpu_count() or 1
    sim.set_threads(cores)
    errors = {}
    # ---- forward, all cores
    d, n = size
    ops = W.random_circuit(d, n, N_GATES)
    t0 = time.perf_counter()
    psi = sim.run(ops, d, n)
    dt = time.perf_counter() - t0
    value = N_GATES * d ** n / dt
    fw = keep.get("forward")
    if fw:
        for dtype, tol in (("c64", 1e-5), ("c128", 1e-12)):
            got = fw[dtype]
            m = 0.0
            for i in range(0, psi.size, 1 << 24):
                m = max(m, float(np.abs(got[i:i + (1 << 24)].astype(np.complex128) - psi[i:i + (1 << 24)]).max()))
            errors["forward_" + dtype] = {"max_abs": m, "tol": tol, "within": m <= tol,
                                          "sample": "the whole 200-gate d=%d n=%d sequence, every amplitude" % (d, n)}
    del psi
    # ---- the first two gates on one thread
    sim.set_threads(1)
    one = sim.basis(d, n, 0)
    t0 = time.perf_counter()
    for op in ops[:2]:
        t, U = sim.op_matrix(op, d)
        sim.apply(one, d, n, t, U)
    dt1 = time.perf_counter() - t0
    sim.set_threads(cores)
    del one
    record = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
              "sample": "the whole 200-gate d=%d n=%d sequence, complex128 oracle, all host cores, %.1f s" % (d, n, dt),
              "one_thread": {"value": 2 * d ** n / dt1, "unit": UNIT, "cores": 1,
                             "sample": "first 2 gates of the d=%d n=%d sequence, %.1f s" % (d, n, dt1)}}
    # ---- adjoint: derivative circuits for a parameter subset
    adj = keep.get("adjoint")
    if adj:
        d, n, ops, theta, w, slots = adj["d"], adj["n"], adj["ops"], adj["theta"], adj["w"], adj["slots"]
        t0 = time.perf_counter()
        want_g = sim.grad_bruteforce(ops, d, n, theta, w, slots=slots)
        tg = time.perf_counter() - t0
        want_l = sim.loss(sim.run(ops, d, n, params=theta), d, n, w)
        for dtype in ("c64", "c128"):
            if dtype in adj:
                loss, g = adj[dtype]
                e = _err(g[slots], want_g, 1e-10 if dtype == "c128" else None, rel=True)
                e["loss_abs"] = abs(loss - want_l)
                e["sample"] = "d=3 n=14 L=10 ansatz, parameters %s of 560 and the loss" % (slots,)
                errors["adjoint_" + dtype] = e
        record["adjoint_bruteforce"] = {
            "seconds_for_sample": tg, "params_in_sample": len(slots),
            "seconds_per_gradient_extrapolated": tg / len(slots) * adj["P"],
            "note": "oracle derivative circuits, all cores; extrapolated linearly to all %d parameters" % adj["P"]}
    # ---- batched and VQA samples
    for key in ("batched", "vqa"):
        smp = keep.get(key)
        if not smp:
            continue
        t0 = time.perf_counter()
        eg, el, worst_rel = 0.0, 0.0, 0.0
        for c_ops, cd, cn, slots, loss_gpu, g_gpu, params in smp["circuits"]:
            w = [1.0] + [0.0] * (cn - 1)
            want = sim.grad_bruteforce(c_ops, cd, cn, params, w, slots=slots)
            wl = sim.loss(sim.run(c_ops, cd, cn, params=params), cd, cn, w)
            eg = max(eg, float(np.abs(np.asarray(g_gpu) - want).max()) if len(slots) else 0.0)
            el = max(el, abs(loss_gpu - wl))
        errors[key + "_" + smp["dtype"]] = {"max_abs": eg, "loss_abs": el, "sample": smp["sample"]}
        record[key + "_oracle_seconds"] = time.perf_counter() - t0
    return record, errors


# --------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.probe_host_memory:
        return probe_host_memory(args)

    import numpy as np
    import torch

    from paper_2409_17716_gb300 import build as gpu_build
    gpu_build.build()
    from paper_2409_17716_gb300 import qf
    from paper_2409_17716_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    hbm_peak, peak_kind = peaks()
    sizes = [args.profile_case] if args.profile_case else SIZES
    extras = not (args.no_extras or args.profile_case)
    stream = torch.cuda.current_stream()

    # ---- states and fused programs (inputs resident in HBM)
    states, progs, circ = [], [], []
    for d, n in sizes:
        st = qf.State(d, n, "c64")
        st.set_basis(0)
        ops = W.random_circuit(d, n, N_GATES)
        p = qf.program_from_ops(d, n, ops, fuse=True)
        states.append(st)
        progs.append(p)
        circ.append(ops)
    out_dev = torch.zeros(128, dtype=torch.float64, device="cuda")

    def step(states_, progs_):
        # the program, then <N_q> of every qudit and the norm, reduced in its
        # last pass
        for st, p in zip(states_, progs_):
            qf.qf_program_run_expect(p, st.handle, out_dev.data_ptr())

    for _ in range(args.warmup):
        step(states, progs)
    torch.cuda.synchronize()
    passes = [qf.qf_program_last_passes(p) for p in progs]
    for p in progs:
        qf.qf_program_set_timing(p, True)

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(states, progs)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()

    # per-pass times of every timed step
    tile_ms, tile_bytes, strided_ms, strided_bytes, n_tile = 0.0, 0.0, 0.0, 0.0, 0
    for p in progs:
        pms, pkind, pby = qf.qf_program_pass_times(p, 1 << 16)
        qf.qf_program_set_timing(p, False)
        for t_, k_, b_ in zip(pms, pkind, pby):
            if k_ == 0:
                tile_ms += t_
                tile_bytes += b_
                n_tile += 1
            else:
                strided_ms += t_
                strided_bytes += b_
    au_step = sum(d ** n for d, n in sizes) * N_GATES
    ms, value = whole_job(ms, au_step, args.steps, dist, "cuda")
    launches = sum(pp + 1 for pp in passes) * args.steps   # passes + the row sums of the fused reduction
    achieved = (tile_bytes / (tile_ms / 1e3)) / 1e9 if tile_ms > 0 else None
    ratio = traffic_ratio()
    avg_alg = tile_bytes / n_tile if n_tile else None
    roofline = {"bound": "hbm", "kernel": "k_tile_jit (compiled fused pass)", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": (achieved / hbm_peak) if achieved else None,
                "traffic": (ratio * avg_alg) if (ratio and avg_alg) else None,
                "algorithmic_bytes_per_launch": avg_alg, "launches": n_tile,
                "share_of_step": tile_ms / ms if ms else None,
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs copy)" if peak_kind == "measured" else peak_kind}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.profile_case else
                       "profile case: d=%d n=%d only" % args.profile_case,
                       "global_batch": len(sizes) * world, "seq_len": None,
                       "parallelism": "replicas" if world > 1 else "single-gpu",
                       "l2": "inputs larger than L2 (1.0-2.1 GB per state), no flush",
                       "passes_per_step": passes, "gates_per_state": N_GATES},
            "gpu_launches": launches, "clocks": clocks, "roofline": roofline}

    if extras:
        line["per_size"] = per_size_throughput(qf, W, torch, sizes, states, progs, args, hbm_peak)
        line["roofline"]["frac_by_d"] = {str(r["d"]): r["hbm_frac"] for r in line["per_size"]}
        line["e2e"] = e2e_throughput(qf, W, torch, sizes, progs, args)
        line["unfused"] = unfused_throughput(qf, W, torch, sizes, states, circ)
        rates = qf.qf_device_fma_rates()
        line["alu_peaks"] = {"fp64_fma_tflops": 2 * rates[0] / 1e12, "fp32_fma_tflops": 2 * rates[1] / 1e12,
                             "how": "qf_device_fma_rates: independent FMA chains, CUDA events, best of 5"}
        line["c128"] = c128_throughput(qf, W, torch, sizes, hbm_peak, rates)
        line["per_gate"] = per_gate_sweep(qf, W, torch, hbm_peak)
    for p in progs:
        qf.qf_program_free(p)
    for st in states:
        st.free()
    keep = {}   # GPU outputs the oracle checks in the CPU-baseline leg
    if extras:
        torch.cuda.empty_cache()
        keep["forward"] = forward_outputs(qf, W, torch)
        torch.cuda.empty_cache()
        line["adjoint"] = adjoint_bench(qf, W, torch, hbm_peak, keep)
        torch.cuda.empty_cache()
        line["batched"] = batch_bench(qf, W, torch, keep)
        torch.cuda.empty_cache()
        line["vqa_training"] = vqa_bench(qf, W, torch, keep)
        torch.cuda.empty_cache()
        line["mixed_dims"] = mixed_bench(qf, W, torch, hbm_peak)
    if extras and rank == 0 and world == 1:
        line["cpu_baseline"], errors = cpu_baseline(keep)
        line["error_vs_oracle"] = errors
        for leg, key in (("adjoint", "adjoint"), ("batched", "batched"), ("vqa_training", "vqa")):
            if leg in line:
                line[leg]["error_vs_oracle"] = {k: v for k, v in errors.items() if k.startswith(key)}
        line["c128"]["error_vs_oracle"] = errors.get("forward_c128")
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _time_ms(torch, fn, reps=3):
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def forward_outputs(qf, W, torch, d=3, n=17):
    """The d=3 n=17 benchmark sequence run once from |0...0> through the
    timed fused program in complex64 and complex128; host copies of the final
    states for the oracle comparison."""
    ops = W.random_circuit(d, n, N_GATES)
    p = qf.program_from_ops(d, n, ops, fuse=True)
    out = {"d": d, "n": n}
    for dtype in ("c64", "c128"):
        st = qf.State(d, n, dtype).set_basis(0)
        qf.qf_program_run(p, st.handle)
        torch.cuda.synchronize()
        out[dtype] = st.tensor.cpu().numpy()
        st.free()
    qf.qf_program_free(p)
    return out


def per_size_throughput(qf, W, torch, sizes, states, progs, args, hbm_peak):
    """Each size's program alone: time, rate, and the HBM fraction of its
    passes (pass count x 2 N b over the program time)."""
    out = []
    for (d, n), st, p in zip(sizes, states, progs):
        ms = _time_ms(torch, lambda: qf.qf_program_run(p, st.handle), reps=5)
        passes = qf.qf_program_last_passes(p)
        out.append({"d": d, "n": n, "amps": d ** n, "passes": passes,
                    "ms": ms, "au_per_s": d ** n * N_GATES / (ms / 1e3),
                    "hbm_frac": passes * 2 * d ** n * 8 / (ms / 1e3) / 1e9 / hbm_peak})
    return out


def unfused_throughput(qf, W, torch, sizes, states, circ):
    tot_au, tot_ms = 0, 0.0
    for (d, n), st, ops in zip(sizes, states, circ):
        p = qf.program_from_ops(d, n, ops, fuse=False)
        qf.qf_program_run(p, st.handle)
        ms = _time_ms(torch, lambda: qf.qf_program_run(p, st.handle), reps=2)
        qf.qf_program_free(p)
        tot_au += d ** n * N_GATES
        tot_ms += ms
    return {"value": tot_au / (tot_ms / 1e3), "unit": UNIT, "note": "one kernel per gate (fusion off)"}


def c128_throughput(qf, W, torch, sizes, hbm_peak, rates):
    """Complex128 programs (double-float arithmetic in the compiled passes,
    the default) per size, with the two ceilings that bound them: HBM (one
    read and write of 16-byte amplitudes per pass) and what FP64 arithmetic
    alone would allow (4 FP64 FMAs per complex multiply-add of the program,
    at the measured FP64 FMA rate); the same programs in FP64 on the
    smallest size for comparison."""
    fp64_rate = rates[0]
    tot_au, tot_ms, per = 0, 0.0, []
    for d, n in sizes:
        st = qf.State(d, n, "c128").set_basis(0)
        p = qf.program_from_ops(d, n, W.random_circuit(d, n, N_GATES), fuse=True)
        qf.qf_program_run(p, st.handle)
        ms = _time_ms(torch, lambda: qf.qf_program_run(p, st.handle), reps=3)
        passes = qf.qf_program_last_passes(p)
        N = d ** n
        cm = qf.qf_program_cmacs(p, qf.QF_C128)
        rec = {"d": d, "n": n, "ms": ms, "passes": passes, "au_per_s": N * N_GATES / (ms / 1e3),
               "cmacs_per_amplitude": cm,
               "hbm_bound_au_per_s": N * N_GATES / (passes * 2 * 16 * N / (hbm_peak * 1e9)),
               "fp64_arith_bound_au_per_s": fp64_rate * N_GATES / (4 * cm) if cm else None}
        if (d, n) == (3, 17):
            qf.qf_program_set_fp64(p, True)
            qf.qf_program_run(p, st.handle)
            rec["fp64_ms"] = _time_ms(torch, lambda: qf.qf_program_run(p, st.handle), reps=2)
        per.append(rec)
        qf.qf_program_free(p)
        st.free()
        tot_au += N * N_GATES
        tot_ms += ms
    return {"value": tot_au / (tot_ms / 1e3), "unit": UNIT, "arith": "double-float (FP32 pairs) in compiled passes",
            "bound": "alu (FP32 pipe, double-float arithmetic)", "per_size": per}


def per_gate_sweep(qf, W, torch, hbm_peak):
    """Single-gate GB/s of each gate kind at every target position, all four
    sizes, complex64 and complex128 (immediate mode: the strided kernel at
    every stride).  Algorithmic bytes count the level rows a gate changes;
    effective bytes count whole 32-byte sectors -- below a sector per row
    the untouched rows share sectors with the touched ones, so the whole
    state moves."""
    import numpy as np
    out = {}
    for dtype, b in (("c64", 8), ("c128", 16)):
        for d, n in SIZES:
            N = d ** n
            st = qf.State(d, n, dtype).set_basis(0)
            U = W.haar_unitary(d, np.random.default_rng(7))
            kinds = {
                "dense(H/Haar)": (lambda q: qf.qf_apply_gate(st.handle, [q], U), 1.0),
                "rot_pair(RY 0,1)": (lambda q: qf.qf_apply_rot(st.handle, q, 0, 1, 0.7, "y"), 2 / d),
                "diag(clock Z)": (lambda q: qf.qf_apply_z(st.handle, q, 1), (d - 1) / d),
                "rz_pair(RZ 0,1)": (lambda q: qf.qf_apply_rot(st.handle, q, 0, 1, 0.7, "z"), 2 / d),
                "shift(X)": (lambda q: qf.qf_apply_x(st.handle, q, 1), 1.0),
                "sum(c=q-1,t=q)": (lambda q: qf.qf_apply_sum(st.handle, (q - 1) % n, q), (d - 1) / d),
            }
            rec = {}
            for name, (fn, frac) in kinds.items():
                alg, eff = [], []
                for q in range(n):
                    S = d ** (n - 1 - q)
                    if name.startswith("sum"):   # skips the control-0 blocks: the control's stride counts too
                        S = min(S, d ** (n - 1 - (q - 1) % n))
                    fn(q)
                    ms = _time_ms(torch, lambda: fn(q), reps=5)
                    alg_b = 2 * N * b * frac
                    eff_b = alg_b if S * b >= 32 else 2 * N * b
                    alg.append(alg_b / (ms / 1e3) / 1e9)
                    eff.append(eff_b / (ms / 1e3) / 1e9)
                rec[name] = {"gbps_by_target": [round(x, 1) for x in alg],
                             "median_frac": statistics.median(alg) / hbm_peak,
                             "min_frac_effective": min(eff) / hbm_peak,
                             "median_frac_effective": statistics.median(eff) / hbm_peak}
            out["d%d_n%d_%s" % (d, n, dtype)] = rec
            st.free()
            torch.cuda.empty_cache()
    return out


def mixed_touched_bytes(op, dims, N, b):
    """Algorithmic HBM bytes of one gate on a mixed register: read + write of
    the amplitudes it changes (levels it touches, control level != 0)."""
    k = op.kind
    full = 2.0 * N * b
    if k in ("h", "x") or (k == "u"):
        return full
    t = op.qudits[-1]
    d = dims[t]
    if k == "z":
        return full * sum(1 for l in range(d) if (op.power * l) % d) / d
    if k in ("rot", "crot"):
        rows = (op.j + 1) if op.axis == "g" else 2
        f = rows / d
        if k == "crot":
            f *= (dims[op.qudits[0]] - 1) / dims[op.qudits[0]]
        return full * f
    if k == "sum":
        return full * (dims[op.qudits[0]] - 1) / dims[op.qudits[0]]
    if k == "swap":
        return full * (d * d - d) / (d * d)
    return full


def mixed_bench(qf, W, torch, hbm_peak):
    """Registers that mix dimensions (dims 2,3,4,5 repeated four times: 16
    qudits, 2.07e8 amplitudes, 1.66 GB complex64): the random 200-gate
    sequence, one launch per gate; and the adjoint gradient of a mixed
    ansatz against 2P + 1 forwards."""
    import numpy as np
    dims = [2, 3, 4, 5] * 4
    n = len(dims)
    N = int(np.prod(dims))
    b = 8
    ops = W.mixed_random_circuit(dims, 200)
    st = qf.State(dims, n, "c64").set_basis(0)
    p = qf.program_from_ops(dims, n, ops)
    qf.qf_program_run(p, st.handle)
    ms = _time_ms(torch, lambda: qf.qf_program_run(p, st.handle), reps=3)
    alg = sum(mixed_touched_bytes(op, dims, N, b) for op in ops)
    out = {"dims": dims, "amps": N, "gates": len(ops), "launches": len(ops), "ms": ms,
           "au_per_s": N * len(ops) / (ms / 1e3),
           "algorithmic_gbs": alg / (ms / 1e3) / 1e9, "algorithmic_frac": alg / (ms / 1e3) / 1e9 / hbm_peak,
           "whole_state_gbs": 2.0 * N * b * len(ops) / (ms / 1e3) / 1e9,
           "note": "one launch per gate (no fusion on mixed registers); algorithmic bytes count only "
                   "the levels a gate changes, whole-state bytes 2 N b per gate"}
    qf.qf_program_free(p)
    st.free()
    # adjoint of a mixed ansatz: 16 qudits, 1 layer
    aops, P = W.mixed_ansatz(dims, 1)
    theta = W.normal_angles(P, seed=16)
    w = [1.0] * n
    p = qf.program_from_ops(dims, n, aops)
    psi, lam = qf.State(dims, n, "c64"), qf.State(dims, n, "c64")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(P, dtype=torch.float64, device="cuda")
    ev = torch.zeros(n + 1, dtype=torch.float64, device="cuda")

    def fwd():
        psi.set_basis(0)
        qf.qf_program_run(p, psi.handle, theta)
        qf.qf_expect_device(psi.handle, ev.data_ptr(), qf.QF_OBS_NUMBER_ALL)

    def full_grad():
        psi.set_basis(0)
        qf.qf_program_run(p, psi.handle, theta)
        qf.qf_program_adjoint(p, psi.handle, lam.handle, theta, w, loss.data_ptr(), grad.data_ptr())

    full_grad()
    gms = _time_ms(torch, full_grad, reps=3)
    fms = _time_ms(torch, fwd, reps=3)
    out["adjoint"] = {"params": P, "gates": len(aops), "gradient_ms": gms, "forward_ms": fms,
                      "fd_gradient_ms": (2 * P + 1) * fms, "speedup_vs_fd": (2 * P + 1) * fms / gms}
    qf.qf_program_free(p)
    psi.free()
    lam.free()
    return out


ADJ_N14_SLOTS = [3, 150, 297, 559]     # oracle-checked parameters of the d=3 n=14 L=10 ansatz
ADJ_N20_FD_SLOTS = [47, 141, 235, 319]  # central-difference parameters of the d=3 n=20 L=4 ansatz


def central_differences_c128(qf, torch, d, n, ops, theta, w, slots, h=1e-5):
    """FP64 central differences of sum_q w_q <N_q> from complex128 forward
    runs on this GPU.  One state advances through the circuit; at each
    chosen parameter a copy runs the remaining gates at theta +- h."""
    import numpy as np
    pos = {op.param: l for l, op in enumerate(ops) if op.param >= 0}
    a, b = qf.State(d, n, "c128").set_basis(0), qf.State(d, n, "c128")
    prev, fd = 0, {}
    for s in sorted(slots, key=lambda x: pos[x]):
        l = pos[s]
        if l > prev:
            seg = qf.program_from_ops(d, n, ops[prev:l])
            qf.qf_program_run(seg, a.handle, theta)
            qf.qf_program_free(seg)
            prev = l
        suf = qf.program_from_ops(d, n, ops[l:])
        vals = []
        for sign in (1.0, -1.0):
            b.tensor.copy_(a.tensor)
            t = np.array(theta, dtype=float)
            t[s] += sign * h
            qf.qf_program_run(suf, b.handle, t)
            vals.append(float(np.dot(w, b.expect_number()[:n])))
        qf.qf_program_free(suf)
        fd[s] = (vals[0] - vals[1]) / (2 * h)
    a.free()
    b.free()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return fd


def adjoint_bench(qf, W, torch, hbm_peak, keep):
    """Full gradient (forward + adjoint) of the variational ansatz vs the
    forward + central-difference path on the same GPU (2P + 1 forwards).
    The d=3 n=14 gradients are kept for the oracle; the d=3 n=20 complex64
    gradient is checked against complex128 central differences here."""
    import numpy as np
    out = {}
    cases = [("d3_n14_L10", 3, 14, 10, ("c64", "c128")), ("d3_n20_L4", 3, 20, 4, ("c64",))]
    for name, d, n, L, dtypes in cases:
        ops, P = W.variational_ansatz(d, n, L, entangler="ring" if n == 14 else "chain")
        theta = W.normal_angles(P, seed=n)
        w = [1.0] * n
        if n == 14:
            keep["adjoint"] = {"d": d, "n": n, "ops": ops, "theta": theta, "w": w, "P": P, "slots": ADJ_N14_SLOTS}
        for dtype in dtypes:
            p = qf.program_from_ops(d, n, ops)
            psi, lam = qf.State(d, n, dtype), qf.State(d, n, dtype)
            loss = torch.zeros(1, dtype=torch.float64, device="cuda")
            grad = torch.zeros(P, dtype=torch.float64, device="cuda")
            ev = torch.zeros(n + 1, dtype=torch.float64, device="cuda")

            def fwd():
                psi.set_basis(0)
                qf.qf_program_run(p, psi.handle, theta)
                qf.qf_expect_device(psi.handle, ev.data_ptr(), qf.QF_OBS_NUMBER_ALL)

            def full_grad():
                psi.set_basis(0)
                qf.qf_program_run(p, psi.handle, theta)
                qf.qf_program_adjoint(p, psi.handle, lam.handle, theta, w, loss.data_ptr(), grad.data_ptr())

            reps = 2 if n >= 20 else 5
            fwd()
            full_grad()
            t_f = _time_ms(torch, fwd, reps=reps)
            fwd_passes = qf.qf_program_last_passes(p)
            full_grad()
            adj_passes = qf.qf_program_last_passes(p)
            t_g = _time_ms(torch, full_grad, reps=reps)
            N = d ** n
            b = 8 if dtype == "c64" else 16
            # algorithmic bytes: forward passes (2Nb each), lambda = O psi (2Nb),
            # reverse passes over psi and lambda (4Nb each)
            by = fwd_passes * 2 * N * b + 2 * N * b + adj_passes * 4 * N * b
            fd_ms = (2 * P + 1) * t_f
            out[name + "_" + dtype] = {
                "params": P, "gates": len(ops), "gradient_ms": t_g, "gradients_per_s": P / (t_g / 1e3),
                "forward_ms": t_f, "fd_gradient_ms": fd_ms, "speedup_vs_fd": fd_ms / t_g,
                "passes_forward": fwd_passes, "passes_adjoint": adj_passes,
                "hbm_gbs": by / (t_g / 1e3) / 1e9, "hbm_frac": by / (t_g / 1e3) / 1e9 / hbm_peak,
                "note": "fd = (2P+1) forward runs of the same fused program on this GPU"}
            torch.cuda.synchronize()
            g_host = grad.cpu().numpy().copy()
            l_host = float(loss.item())
            if n == 14:
                keep["adjoint"][dtype] = (l_host, g_host)
            qf.qf_program_free(p)
            psi.free()
            lam.free()
            del ev, grad, loss
            torch.cuda.empty_cache()
            if n == 20:
                t0 = time.perf_counter()
                fd = central_differences_c128(qf, torch, d, n, ops, theta, w, ADJ_N20_FD_SLOTS)
                fd_v = np.array([fd[s] for s in ADJ_N20_FD_SLOTS])
                e = _err(g_host[ADJ_N20_FD_SLOTS], fd_v, rel=True)
                e["reference"] = ("FP64 central differences (h=1e-5) of the complex128 forward on this GPU, "
                                  "parameters %s of %d" % (ADJ_N20_FD_SLOTS, P))
                e["seconds"] = time.perf_counter() - t0
                out[name + "_" + dtype]["error_vs_c128_fd"] = e
    return out


def batch_bench(qf, W, torch, keep):
    """4096 circuits (d 2..5, n 4..10, L 2..6), forward + adjoint in one graph
    replay, vs per-circuit forward + central differences on the same GPU
    (sampled over 64 circuits and extrapolated)."""
    import numpy as np
    from paper_2409_17716_gb300 import autotune
    circuits, params = W.batch_circuits(count=4096)
    t0 = time.perf_counter()
    tuning = autotune.tune(circuits, params, qf.QF_C64, use_cache=False)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = qf.qf_batch_create(qf.QF_C64)
    progs = []
    for c in circuits:
        p = qf.program_from_ops(c.d, c.n, c.ops)
        qf.qf_batch_add(b, p, [1.0] + [0.0] * (c.n - 1))
        progs.append(p)
    autotune.apply(b, tuning)
    qf.qf_batch_build(b, len(params))
    build_s = time.perf_counter() - t0
    info = qf.qf_batch_info(b)
    qf.qf_batch_run(b, params, True)
    qf.qf_batch_run(b, params, True)
    t_fb = _time_ms(torch, lambda: qf.qf_batch_run(b, params, True), reps=3)
    t_f = _time_ms(torch, lambda: qf.qf_batch_run(b, params, False), reps=3)
    # outputs of a forward + backward run for the oracle: 8 circuits of at
    # most 4096 amplitudes drawn from the batch
    qf.qf_batch_run(b, params, True)
    loss_all, gl_all, _ = qf.qf_batch_read(b)
    rs = np.random.default_rng(2)
    small = [i for i, c in enumerate(circuits) if c.d ** c.n <= 4096]
    picks = [int(i) for i in rs.choice(small, min(8, len(small)), replace=False)]
    smp = []
    for i in picks:
        c = circuits[i]
        slots, off = qf.qf_batch_circuit_params(b, i)
        smp.append((c.ops, c.d, c.n, slots, float(loss_all[i]), gl_all[off:off + len(slots)].copy(), params))
    keep["batched"] = {"dtype": "c64", "circuits": smp,
                       "sample": "circuits %s of the 4096 (those with at most 4096 amplitudes, drawn at random): "
                                 "loss and every parameter's gradient" % picks}
    # per-circuit forward + FD baseline on a sample
    rng = np.random.default_rng(1)
    sample = rng.choice(len(circuits), 64, replace=False)
    fd_ms = 0.0
    ev = torch.zeros(16, dtype=torch.float64, device="cuda")
    for i in sample:
        c = circuits[i]
        st = qf.State(c.d, c.n, "c64")
        P_c = len(qf.qf_batch_circuit_params(b, int(i))[0])

        def fwd():
            st.set_basis(0)
            qf.qf_program_run(progs[i], st.handle, params)
            qf.qf_expect_device(st.handle, ev.data_ptr(), qf.QF_OBS_NUMBER_ALL)

        fwd()
        fd_ms += (2 * P_c + 1) * _time_ms(torch, fwd, reps=3)
        st.free()
    fd_total_ms = fd_ms * len(circuits) / len(sample)
    qf.qf_batch_free(b)
    for p in progs:
        qf.qf_program_free(p)
    return {"circuits": info["circuits"], "amplitudes": info["amplitudes"],
            "forward_backward_ms": t_fb, "forward_ms": t_f, "samples_per_s": info["circuits"] / (t_fb / 1e3),
            "gradients_per_s": info["grad_local_len"] / (t_fb / 1e3),
            "forward_amplitude_updates_per_s": info["gate_amplitudes"] / (t_f / 1e3),
            "launches_forward_backward": info["launches_backward"], "build_s": build_s, "autotune_s": tune_s,
            "autotuned": {str(d): {"tile_qudits": t["tile_qudits"], "max_ops": t["max_ops"]} for d, t in tuning.items()},
            "fd_per_circuit_ms_extrapolated": fd_total_ms, "speedup_vs_per_circuit_fd": fd_total_ms / t_fb,
            "note": "fd baseline: per-circuit fused forward + <N_q> on this GPU, (2P_c+1) runs, 64-circuit sample"}


def vqa_bench(qf, W, torch, keep):
    """Training-step throughput of the paper's VQA circuits (rotation blocks
    R1 / R2 / R3): 4096 samples per step (Iris-like d=3 n=4, MNIST-like d=10
    n=2 and n=4), forward + adjoint of <N_0> in one graph replay, complex64."""
    out = {}
    for d, n in [(3, 4), (10, 2), (10, 4)]:
        for variant in ("R1", "R2", "R3"):
            circuits, params = W.vqa_batch(4096, d, n, variant)
            b = qf.qf_batch_create(qf.QF_C64)
            progs = []
            for c in circuits:
                p = qf.program_from_ops(c.d, c.n, c.ops)
                qf.qf_batch_add(b, p, [1.0] + [0.0] * (c.n - 1))
                progs.append(p)
            qf.qf_batch_build(b, len(params))
            qf.qf_batch_run(b, params, True)
            ms = _time_ms(torch, lambda: qf.qf_batch_run(b, params, True), reps=3)
            info = qf.qf_batch_info(b)
            if (d, n, variant) in ((3, 4, "R1"), (10, 2, "R3")):
                loss_all, gl_all, _ = qf.qf_batch_read(b)
                smp = keep.setdefault("vqa", {"dtype": "c64", "circuits": [],
                                              "sample": "samples 0, 1000, 2000, 4095 of the d=3 n=4 R1 and d=10 n=2 "
                                                        "R3 steps: loss and every parameter's gradient"})
                for i in (0, 1000, 2000, 4095):
                    c = circuits[i]
                    slots, off = qf.qf_batch_circuit_params(b, i)
                    smp["circuits"].append((c.ops, c.d, c.n, slots, float(loss_all[i]),
                                            gl_all[off:off + len(slots)].copy(), params))
            out["d%d_n%d_%s" % (d, n, variant)] = {
                "samples_per_s": 4096 / (ms / 1e3), "step_ms": ms, "gates": len(circuits[0].ops),
                "gradients_per_s": info["grad_local_len"] / (ms / 1e3)}
            qf.qf_batch_free(b)
            for p in progs:
                qf.qf_program_free(p)
    return out


def e2e_throughput(qf, W, torch, sizes, progs, args):
    """End to end through the library's C ABI with host buffers: per step and
    state, qf_state_upload of the input amplitudes from page-locked host
    memory, qf_program_run, and qf_expect returning <N_q> and the norm to the
    host.  Each state has its own stream, so one state's upload overlaps
    another's circuit; qf_expect synchronises its state's stream."""
    import numpy as np
    # smallest state first: its circuit starts after the shortest upload
    order = sorted(range(len(sizes)), key=lambda i: sizes[i][0] ** sizes[i][1])
    sizes = [sizes[i] for i in order]
    progs = [progs[i] for i in order]
    host = []
    for d, n in sizes:
        ptr = qf.qf_host_alloc(d ** n * 8)   # page-locked by the library
        a = qf.host_array(ptr, d ** n, np.complex64)
        a[:] = 0
        a[0] = 1.0
        host.append((ptr, d ** n))
    streams = [torch.cuda.Stream() for _ in sizes]
    states = [qf.State(d, n, "c64", stream=s) for (d, n), s in zip(sizes, streams)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in sizes]

    calls = []   # host wall time of every library call of the last step

    def step():
        calls.clear()
        for i, (st, (ptr, count)) in enumerate(zip(states, host)):
            ev[i][0].record(streams[i])
            t = time.perf_counter()
            qf.qf_state_upload(st.handle, ptr, 0, count)
            calls.append(("upload", i, time.perf_counter() - t))
            ev[i][1].record(streams[i])
            t = time.perf_counter()
            qf.qf_program_run(progs[i], st.handle)
            calls.append(("run", i, time.perf_counter() - t))
        out = []
        for i, st in enumerate(states):
            t = time.perf_counter()
            out.append(qf.qf_expect(st.handle, qf.QF_OBS_NUMBER_ALL))
            calls.append(("expect", i, time.perf_counter() - t))
        return out

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    steps = max(3, args.steps // 2)
    per_step, copy_ms, step_calls = [], [], []
    import gc
    gc.collect()
    gc.disable()   # a full collection of the process's objects is a host pause, not library time
    t0 = time.perf_counter()
    for _ in range(steps):
        ts = time.perf_counter()
        res = step()
        per_step.append(1e3 * (time.perf_counter() - ts))
        copy_ms.append(sum(a.elapsed_time(b) for a, b in ev))
        step_calls.append([(c, i, round(1e3 * x, 2)) for c, i, x in calls])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    gc.enable()
    assert all(abs(r[-1] - 1.0) < 1e-3 for r in res)
    for st in states:
        st.free()
    for ptr, _ in host:
        qf.qf_host_free(ptr)
    au = sum(d ** n for d, n in sizes) * N_GATES * steps
    bytes_in = sum(d ** n * 8 for d, n in sizes)
    med = sorted(per_step)[len(per_step) // 2]
    return {"value": au / dt, "unit": UNIT, "h2d_bytes_per_step": bytes_in,
            "d2h_bytes_per_step": sum((n + 1) * 8 for d, n in sizes), "steps": steps,
            "h2d_gbs_in_step_median": bytes_in / (sorted(copy_ms)[len(copy_ms) // 2] / 1e3) / 1e9,
            "step_ms": {"min": min(per_step), "median": med, "max": max(per_step)},
            "step_ms_each": [round(x, 2) for x in per_step],
            # host wall ms of each call (kind, state) in the slowest and in the median step
            "calls_slowest_step": step_calls[per_step.index(max(per_step))],
            "calls_median_step": step_calls[per_step.index(med)],
            "value_at_median_step": au / steps / (med / 1e3),
            "note": "per state (own stream, smallest first): qf_state_upload from page-locked host memory "
                    "(qf_host_alloc), qf_program_run, qf_expect to the host"}


def probe_host_memory(args):
    """The end-to-end step (per state and stream: qf_state_upload of 1.0-2.1
    GB, the circuit, qf_expect) with host buffers from torch's pin_memory
    and from the library's qf_host_alloc; per-step wall times."""
    import numpy as np
    import torch
    from paper_2409_17716_gb300 import build as gpu_build
    gpu_build.build()
    from paper_2409_17716_gb300 import qf
    from paper_2409_17716_gb300 import workloads as W
    sizes = SIZES
    progs = [qf.program_from_ops(d, n, W.random_circuit(d, n, N_GATES)) for d, n in sizes]
    streams = [torch.cuda.Stream() for _ in sizes]
    states = [qf.State(d, n, "c64", stream=s) for (d, n), s in zip(sizes, streams)]

    def run(name, ptrs, circuits=True, steps=14):
        per = []
        for it in range(steps + 2):
            t0 = time.perf_counter()
            for i, st in enumerate(states):
                qf.qf_state_upload(st.handle, ptrs[i], 0, sizes[i][0] ** sizes[i][1])
                if circuits:
                    qf.qf_program_run(progs[i], st.handle)
            if circuits:
                for st in states:
                    qf.qf_expect(st.handle, qf.QF_OBS_NUMBER_ALL)
            else:
                for s in streams:
                    s.synchronize()
            if it >= 2:
                per.append(round(1e3 * (time.perf_counter() - t0), 1))
        med = sorted(per)[len(per) // 2]
        print(json.dumps({"host_memory": name, "median_ms": med, "max_ms": max(per),
                          "steps_over_1.5x_median": sum(p > 1.5 * med for p in per), "step_ms": per}), flush=True)

    pinned = []
    for d, n in sizes:
        h = torch.zeros(d ** n, dtype=torch.complex64, pin_memory=True)
        h[0] = 1.0
        pinned.append(h)
    tp = [h.data_ptr() for h in pinned]
    run("torch pin_memory, uploads only", tp, circuits=False)
    run("torch pin_memory, upload + circuit + <N_q>", tp)
    del pinned
    lib = []
    for d, n in sizes:
        ptr = qf.qf_host_alloc(d ** n * 8)
        a = qf.host_array(ptr, d ** n, np.complex64)
        a[:] = 0
        a[0] = 1.0
        lib.append(ptr)
    run("qf_host_alloc, uploads only", lib, circuits=False)
    run("qf_host_alloc, upload + circuit + <N_q>", lib)
    for ptr in lib:
        qf.qf_host_free(ptr)
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark of the GB300 adaptive LP decoder.

Metric: LP-decoded frames/s on the (3,6)-regular n=1008, m=504 LDPC code
(PEG-style construction, seed 0) over BPSK/AWGN at Eb/N0 = 2.0 dB, all-zero
codeword, gamma = 2y/sigma^2. The job is 20,000 synthetic frames (seed 0);
one step decodes --frames (default: all 20,000) frames per GPU through one
persistent kernel launch (MALP-A + interior point + PCG + MTS for every
frame). Inputs are resident in HBM when the timed region starts; L2 is
flushed (256 MB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank decodes its own frames (weak scaling, no
collective on the data path); rank 0 prints one JSON line. --impl reference
times the CPU oracle (FP64, dense Cholesky interior point) on the host cores
on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LP-decoded frames/s at n=1008 (3,6) LDPC 2 dB; p99 latency; PCG SpMV HBM GB/s"
UNIT = "frames/s"
CODE_NAME = "peg_1008"
EBN0_DB = 2.0
POOL = 20000
SEED = 0
# FP64 peak of the GB300 FP64 units: 1.25 TFLOP/s nominal at the 2070 MHz
# maximum SM clock over 152 SMs, i.e. 4 FP64 flops per SM per clock (detail
# figure only; the roofline is HBM bytes).
FP64_FLOPS_PER_SM_CLK = 4.0
N_SMS = 152
HBM_FALLBACK_GBS = 6800.0
# DRAM bytes (read + write) per frame of k_decode<double> on the 2 dB
# workload with the library defaults, from one ncu capture of this build:
# 936,507,648 read + 9,836,531,200 written over a 456-frame launch of
# pool frames 0-455 (dram__bytes_read.sum, dram__bytes_write.sum), scaled
# to a launch by its frame count. Mostly the dense fallback's
# matrices leaving L2. Valid only for that kernel build and configuration.
DRAM_BYTES_PER_FRAME_2DB = (936507648 + 9836531200) / 456


def measured_hbm_gbs():
    """(peak HBM GB/s, source): the measured copy bandwidth of this machine's
    GB300s when the generated peaks file is present, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS, "fallback"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=20000, help="frames per timed step per GPU")
    ap.add_argument("--warmup-frames", type=int, default=8,
                    help="frames per warm-up step (same kernel and code, fewer frames)")
    ap.add_argument("--precision", choices=["fp64", "mixed", "m32"], default="fp64",
                    help="fp64: FP64 PCG; mixed: FP32 PCG refined in FP64; "
                         "m32: FP64 PCG with an FP32 preconditioner solve")
    ap.add_argument("--threads", type=int, default=128)
    ap.add_argument("--precond", choices=["column", "incremental", "rowwise", "adaptive",
                                          "rowwise-tri"],
                    default="column", help="triangular-set preconditioner (Section V)")
    ap.add_argument("--warm-start", type=int, default=0,
                    help="1: interior-point warm start across the LPs of a frame")
    ap.add_argument("--mts-reuse", type=int, default=0,
                    help="1: reuse the triangular set across interior-point iterations")
    ap.add_argument("--dense-switch", type=int, default=-1,
                    help="PCG iterations after which an LP's Newton solves go dense "
                         "(-1: library default, 0: only after a PCG stall)")
    ap.add_argument("--order", type=int, default=1,
                    help="frame order: 0 as given, 1 hardest first when frames queue (default), 2 always")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: pick the triangular-solve schedule with lpdec_autotune during the "
                         "warm-up (456 frames of the same code at 3 dB)")
    ap.add_argument("--smem-budget", type=int, default=0,
                    help="shared-memory bytes per CTA (0 = library choice)")
    ap.add_argument("--ebn0", type=float, default=EBN0_DB,
                    help="Eb/N0 in dB (2.0 is the workload; other values for small profiling cases)")
    ap.add_argument("--oracle-seconds", type=float, default=15.0,
                    help="CPU seconds per oracle worker for the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-seconds", type=float, default=20.0,
                    help="seconds of the plain one-frame-per-launch arm (0 = skip)")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per k_decode launch from an ncu capture of this build")
    ap.add_argument("--workload", choices=["c1", "c2", "c3", "c4", "c5", "x123"], default="c2",
                    help="c2: the batched decode of the metric (default); c1: n=120, one frame "
                         "per launch against one batched launch; c3: the n=16000 "
                         "precision study; c4 / c5: serving with Poisson arrivals of mixed-length "
                         "frames; x123: the iteration-count studies of Section III-D (each prints "
                         "one JSON line of its own)")
    ap.add_argument("--x-trials", type=int, default=1000, help="frames per length (x123)")
    ap.add_argument("--c3-frames", type=int, default=32,
                    help="frames of the n=16000 study (a subset of its 2000)")
    ap.add_argument("--c3-oracle-frames", type=int, default=2,
                    help="frames of the study checked against the full LP (HiGHS)")
    ap.add_argument("--max-pcg", type=int, default=0,
                    help="PCG iteration cap per Newton solve (0 = library default)")
    ap.add_argument("--sat-seconds", type=float, default=100.0,
                    help="serving: length of the saturated run (rate over its last 60%%)")
    ap.add_argument("--serve-seconds", type=float, default=45.0,
                    help="serving: arrival window of each Poisson load level")
    ap.add_argument("--serve-grace", type=float, default=60.0,
                    help="serving: seconds after a level's last arrival before the frames "
                         "still running are cancelled (their latency is reported as censored)")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0,
                    help="HBM admission budget of the serving workloads")
    return ap.parse_args()


def workload_config(args, n, m):
    return {
        "workload": f"(3,6) PEG LDPC n={n} m={m}, BPSK/AWGN Eb/N0 {args.ebn0} dB, all-zero codeword, "
                    f"{POOL}-frame pool (seed {SEED}), {args.frames} frames per step per GPU",
        "code": CODE_NAME, "n": n, "m": m, "ebn0_db": args.ebn0, "pool_frames": POOL,
        "frames_per_step": args.frames, "warmup_frames_per_step": args.warmup_frames,
        "precision": args.precision, "smem_budget": args.smem_budget or "library (1/3 of SM)",
        "threads_per_block": args.threads, "variant": "MALP-A", "precond": args.precond,
        "warm_start": args.warm_start, "mts_reuse": args.mts_reuse, "order_frames": args.order,
        "dense_switch": args.dense_switch if args.dense_switch >= 0 else "library default (64)",
        "l2": "flushed by a 256 MB write between timed steps",
    }


def frame_ids(step, rank, world, per_step):
    """Frames of one rank in one step: the ranks of a step take consecutive,
    disjoint blocks of the pool (weak scaling, no exchange between ranks)."""
    base = (step * world + rank) * per_step
    return [(base + i) % POOL for i in range(per_step)]


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (a plain float on one rank)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle baseline (spawned worker processes, one BLAS thread each)
# ---------------------------------------------------------------------------

def _oracle_worker(args):
    wid, nworkers, seconds, frames, ebn0 = args
    import numpy as np  # noqa: F401
    import oracle
    from synth import awgn_llr_frames, named_code
    code = named_code(CODE_NAME)
    t0 = time.perf_counter()
    done = 0
    for f in frames[wid::nworkers]:
        g = awgn_llr_frames(code.n, code.design_rate, ebn0, SEED, [f])[0]
        oracle.decode(code, g)
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return done, time.perf_counter() - t0


def run_oracle_sample(seconds, offset, ebn0):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    cores = os.cpu_count() or 1
    frames = [(offset + i) % POOL for i in range(10 * cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(w, cores, seconds, frames, ebn0) for w in range(cores)])
    done = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return done, wall, cores


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""
        return False

    def summary(self):
        if self.proc is None:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)

    from paper_0902_0657_gb300 import build as B
    from paper_0902_0657_gb300 import lpdec as L
    from synth import awgn_llr_frames, named_code

    B.build()
    code = named_code(CODE_NAME)
    n, m, B_ = code.n, code.m, args.frames
    prm = L.lpdec_default_params()
    prm.precision = {"fp64": L.LPDEC_FP64, "mixed": L.LPDEC_MIXED, "m32": L.LPDEC_M32}[args.precision]
    prm.threads_per_block = args.threads
    prm.smem_budget = args.smem_budget
    prm.precond = {"column": L.LPDEC_MTS_COLUMN, "incremental": L.LPDEC_MTS_INCREMENTAL,
                   "rowwise": L.LPDEC_MTS_ROWWISE, "adaptive": L.LPDEC_MTS_ADAPTIVE,
                   "rowwise-tri": L.LPDEC_MTS_ROWWISE_TRI}[args.precond]
    prm.warm_start = args.warm_start
    prm.mts_reuse = args.mts_reuse
    prm.order_frames = args.order
    if args.dense_switch >= 0:
        prm.dense_switch = args.dense_switch
    dec = L.Decoder(code, device=local, params=prm)

    tune = None
    if args.autotune:   # part of the warm-up: the schedule autotuner on a fast sample
        sample = awgn_llr_frames(n, code.design_rate, 3.0, SEED + 1, range(456))
        rc, pol, secs = L.lpdec_autotune(dec.ctx, dec.code, sample)
        if rc != 0:
            raise RuntimeError(f"autotune failed: {L.error_string(rc)}")
        tune = {"lane_policy": pol, "candidates": dict(zip(["0", "1", "2", "4", "8"],
                                                           [round(float(x), 3) for x in secs])),
                "sample": "456 frames of the code at 3 dB (seed 1), total CTA seconds"}

    nsteps = args.warmup + args.steps
    sizes = [min(args.warmup_frames, B_) if k < args.warmup else B_ for k in range(nsteps)]
    gam = [torch.from_numpy(awgn_llr_frames(n, code.design_rate, args.ebn0, SEED,
                                            frame_ids(k, rank, world, sizes[k]))).cuda()
           for k in range(nsteps)]
    d_u = torch.empty((B_, n), dtype=torch.float64, device="cuda")
    d_h = torch.empty((B_, n), dtype=torch.uint8, device="cuda")
    d_c = torch.empty(B_, dtype=torch.int32, device="cuda")
    d_m = torch.empty((B_, m), dtype=torch.int32, device="cuda")
    d_s = torch.empty(B_ * L.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # kernels of one timed step: the decode kernel, plus the order keys and
    # their sort when the batch is handed out hardest-first
    rc, grid, ordered = L.lpdec_batch_grid(dec.ctx, dec.code, B_)
    if rc != 0:
        raise RuntimeError(f"launch query failed: {L.error_string(rc)}")
    launches = args.steps * (1 + 2 * ordered)

    def step(k):
        rc = L.lpdec_decode_batch_device(dec.ctx, dec.code, sizes[k], gam[k], d_u, d_h, d_c, d_m,
                                         d_s, stream=stream)
        if rc != 0:
            raise RuntimeError(f"decode failed: {L.error_string(rc)}")

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    times, flops, nbytes, stats_all, certs_all, lat = [], 0.0, 0.0, [], [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.warmup, nsteps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(k)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            st = d_s.cpu().numpy().view(L.STATS_DTYPE)
            stats_all.append(st.copy())
            certs_all.append(d_c.cpu().numpy().copy())
            flops += float(st["pcg_flops"].sum())
            nbytes += float(st["pcg_bytes"].sum())
            # latency of each frame from the launch (the earliest frame start
            # of the step, on the device's global timer) to its end
            lat.append((st["t_end"] - st["t_start"].min()) * 1e-9)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    t_total = sum(times)
    t_max = max_over_ranks(t_total, dist, "cuda") if world > 1 else t_total
    frames_total = B_ * args.steps * world
    value = frames_total / t_max

    # end to end through the host API (pinned host buffers, copies inside)
    e2e = None
    if not args.no_e2e:
        g_host = torch.empty((B_, n), dtype=torch.float64, pin_memory=True)
        g_host.copy_(gam[nsteps - 1].cpu())
        gh = g_host.numpy()
        u = torch.empty((B_, n), dtype=torch.float64, pin_memory=True).numpy()
        hd = torch.empty((B_, n), dtype=torch.uint8, pin_memory=True).numpy()
        ce = torch.empty(B_, dtype=torch.int32, pin_memory=True).numpy()
        mk = torch.empty((B_, m), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        ss = np.empty(B_, L.STATS_DTYPE)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        rc = L.lpdec_decode_frames(dec.ctx, dec.code, B_, gh, u, hd, ce, mk, ss)
        te = time.perf_counter() - t0
        if rc != 0:
            raise RuntimeError(f"host decode failed: {L.error_string(rc)}")
        if world > 1:
            te = max_over_ranks(te, dist, "cuda")
        e2e = {"value": B_ * world / te, "unit": UNIT, "h2d_bytes_per_step": B_ * n * 8,
               "d2h_bytes_per_step": B_ * (n * 8 + n + 4 + m * 4 + L.STATS_DTYPE.itemsize)}

    # the plain form: one frame per launch (grid of one CTA), frames of the
    # same pool in order, for a bounded time
    plain = None
    if args.plain_seconds > 0 and rank == 0:
        pg = gam[nsteps - 1]
        done, t_plain = 0, 0.0
        while t_plain < args.plain_seconds and done < B_:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = L.lpdec_decode_batch_device(dec.ctx, dec.code, 1, pg[done:done + 1], d_u, d_h,
                                             d_c, d_m, d_s, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if rc != 0:
                raise RuntimeError(f"plain decode failed: {L.error_string(rc)}")
            t_plain += e0.elapsed_time(e1) / 1e3
            done += 1
        plain = {"value": done / t_plain, "unit": UNIT, "frames": done,
                 "what": "one frame per launch (one CTA), the step's frames in order, "
                         "device time"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        dec.close()
        return

    st = np.concatenate(stats_all)
    lat = np.concatenate(lat)
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] if clocks else 2070.0
    hbm_peak, hbm_src = measured_hbm_gbs()
    achieved = nbytes / t_total / 1e9
    traffic = args.traffic_bytes
    defaults = (args.ebn0 == 2.0 and args.precision == "fp64" and args.smem_budget == 0
                and args.threads == 128 and args.precond == "column" and not args.warm_start
                and not args.mts_reuse and args.dense_switch < 0)
    if traffic is None and defaults:
        traffic = DRAM_BYTES_PER_FRAME_2DB * B_   # per launch (one launch per step)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak,
                "traffic": traffic,
                "kernel": "k_decode (persistent, one CTA per frame)",
                "peak_source": f"{hbm_src} HBM copy bandwidth",
                "bytes": "algorithmic bytes of every PCG iteration (Q h index passes at 4 B, "
                         "D^2, h and l; both triangular solves at 4 nnz(A_M) + 8p; 5 vector "
                         "passes of 8p), counted per frame on the device from its p, E_A and "
                         "nnz(A_M)"}
    fp64_peak = N_SMS * FP64_FLOPS_PER_SM_CLK * sm_mhz * 1e6 / 1e12

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        done, w, cores = run_oracle_sample(args.oracle_seconds, offset=0, ebn0=args.ebn0)
        cpu = {"value": done / w, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{done} frames of the same workload (pool frames from 0), "
                         f"{cores} spawned single-threaded workers, ~{args.oracle_seconds:.0f} s each"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic", "config": workload_config(args, n, m),
        "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
        "roofline": roofline, "cpu_baseline": cpu, "plain": plain, "schedule": tune,
        "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                       "p99": 1e3 * float(np.percentile(lat, 99)),
                       "p99.9": 1e3 * float(np.percentile(lat, 99.9)),
                       "max": 1e3 * float(lat.max()),
                       "what": "from the start of the step's launch to the end of the frame "
                               "(device global timer)"},
        "frame_device_ms": {"p50": 1e3 * float(np.percentile(st["seconds"], 50)),
                            "p99": 1e3 * float(np.percentile(st["seconds"], 99)),
                            "max": 1e3 * float(st["seconds"].max()),
                            "what": "device time of one frame on its CTA"},
        "detail": {
            "grid_ctas": grid, "frames_ordered_hardest_first": bool(ordered),
            "frames_integral": float((np.concatenate(certs_all) == 1).mean()),
            "frames_ok": int((st["status"] == L.LPDEC_OK).sum()),
            "frames_not_converged": int((st["status"] == L.LPDEC_ERR_NOT_CONVERGED).sum()),
            "frames_out_of_rows": int((st["status"] == L.LPDEC_ERR_OUT_OF_BUDGET).sum()),
            "frames_continued_as_alp": int((st["alp_switch"] > 0).sum()),
            "mean_lps_per_frame": float(st["alp_iters"].mean()),
            "mean_ipm_iters_per_frame": float(st["ipm_iters_total"].mean()),
            "mean_pcg_iters_per_frame": float(st["pcg_iters_total"].mean()),
            "mean_dense_solves_per_frame": float(st["dense_solves"].mean()),
            "ipm_iters_in_refinement_share": float(st["ipm_iters_refine"].sum()
                                                   / max(1, st["ipm_iters_total"].sum())),
            "lps_with_uncertified_vertex": int(st["vertex_failures"].sum()),
            "phase_share_of_cta_time": {
                k: float(st["sec_" + k].sum() / st["seconds"].sum())
                for k in ("mts", "pcg", "dense", "certify", "refine")},
            "slowest_frames": [
                {"frame": int(frame_ids(nsteps - 1, rank, world, B_)[i]),
                 "seconds": round(float(st["seconds"][i]), 3),
                 **{k: int(st[k][i]) for k in ("status", "alp_iters", "ipm_iters_total",
                                                "ipm_iters_refine", "pcg_iters_total",
                                                "dense_solves", "lp_rows_max", "alp_switch",
                                                "vertex_failures")},
                 **{k: round(float(st[k][i]), 3) for k in ("sec_mts", "sec_pcg", "sec_dense",
                                                            "sec_certify", "sec_refine")}}
                for i in np.argsort(-st["seconds"])[:8]],
            "pcg_bytes_per_step": nbytes / args.steps,
            "pcg_flops_per_step": flops / args.steps,
            "fp64_tflops": flops / t_total / 1e12,
            "fp64_frac_of_derived_peak": flops / t_total / 1e12 / fp64_peak,
            "pcg_spmv_hbm_gbs": achieved,
            "pcg_spmv_hbm_note": ("algorithmic bytes of the PCG iterations per second; the "
                                  "kernel keeps each frame's LP in shared memory and L2, so "
                                  "these bytes are served on chip (DRAM traffic is in "
                                  "roofline.traffic)"),
            "wall_s": wall,
        },
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    dec.close()


# ---------------------------------------------------------------------------
# Serving workloads: Poisson arrivals of frames of several codes
# ---------------------------------------------------------------------------

SERVING = {
    "c4": {"codes": ["gallager_504", "peg_1008", "gallager_2016", "gallager_4032"],
           "ebn0": (1.5, 3.0),
           "what": "(3,6)-regular codes n in {504, 1008, 2016, 4032} in equal proportion, "
                   "Eb/N0 uniform in [1.5, 3.0] dB"},
    "c5": {"codes": ["gallager330_8000", "irregular_4000"], "ebn0": (2.5, 4.5),
           "what": "(3,30)-regular n=8000 (rate 0.9) and irregular lambda(x)=0.25x+0.3x^2+0.45x^7, "
                   "check degree 8, n=4000, in equal proportion, Eb/N0 uniform in [2.5, 4.5] dB"},
}


def serving_frames(spec, codes, count, offset, seed=SEED):
    """Frame k: its code (uniform over the workload's codes) and LLRs at an
    Eb/N0 drawn uniformly from the workload's range, from seeded streams."""
    import numpy as np
    from synth import awgn_llr_frames
    out = []
    lo, hi = spec["ebn0"]
    for k in range(offset, offset + count):
        rng = np.random.default_rng([seed, 7, k])
        ci = int(rng.integers(len(codes)))
        eb = float(rng.uniform(lo, hi))
        c = codes[ci]
        out.append((ci, awgn_llr_frames(c.n, c.design_rate, eb, seed, [k])[0]))
    return out


L_OUT_OF_BUDGET = -2   # lpdec.h LPDEC_ERR_OUT_OF_BUDGET
L_CANCELLED = -8       # lpdec.h LPDEC_ERR_CANCELLED
L_NOT_SERVED = -100    # (bench only) offered but never submitted


def serve_run(srv, frames, rate=None, stop_after=None):
    """Submits frames (as fast as admission allows if rate is None, else at
    Poisson arrival times of that rate) and polls them; at stop_after
    seconds from the start, frames not finished are cancelled (running ones
    stop at their next cancel check) and frames not yet submitted are
    dropped. Returns (elapsed, latency in s or NaN if not served, finish
    time from the start or NaN, status)."""
    import numpy as np
    import time as _t
    n = len(frames)
    if rate is None:
        arrive = np.zeros(n)
    else:
        arrive = np.cumsum(np.random.default_rng([SEED, 11, n]).exponential(1.0 / rate, n))
    lat = np.full(n, np.nan)
    fin = np.full(n, np.nan)
    status = np.full(n, L_NOT_SERVED, np.int32)
    pending = {}
    k = 0
    t0 = _t.perf_counter()
    while k < n or pending:
        now = _t.perf_counter() - t0
        if stop_after is not None and now > stop_after:
            for t, (kk, ta) in pending.items():
                srv.cancel(t)
                status[kk] = L_CANCELLED
            pending.clear()
            break
        progressed = False
        while k < n and arrive[k] <= now:
            rc, t = srv.try_submit(frames[k][1], code=frames[k][0])
            if rc == L_OUT_OF_BUDGET:
                break                       # admission refused: poll, then retry
            if rc != 0:
                raise RuntimeError(f"submit failed: {rc}")
            pending[t] = (k, max(arrive[k], 0.0) if rate is not None else now)
            k += 1
            progressed = True
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                kk, ta = pending.pop(t)
                fin[kk] = _t.perf_counter() - t0
                lat[kk] = fin[kk] - ta
                status[kk] = r[4]["status"]
                progressed = True
        if not progressed:
            _t.sleep(0.0002)
    return _t.perf_counter() - t0, lat, fin, status


def latency_summary(lat, offered):
    """p50/p99/p99.9 in ms over the offered frames; a frame not served
    (cancelled at the level's end, or never admitted) counts as slower than
    every served one, and a percentile that falls on such frames is None."""
    import numpy as np
    x = np.where(np.isnan(lat), np.inf, lat)[:offered]
    out = {}
    for q, nm in ((50, "p50_ms"), (99, "p99_ms"), (99.9, "p99.9_ms")):
        v = float(np.percentile(x, q, method="higher")) if len(x) else float("nan")
        out[nm] = 1e3 * v if np.isfinite(v) else None
    out["max_served_ms"] = 1e3 * float(np.nanmax(lat)) if np.any(~np.isnan(lat)) else None
    return out


def run_serving(args):
    import numpy as np
    import torch
    from paper_0902_0657_gb300 import build as B
    from paper_0902_0657_gb300 import lpdec as L
    from synth import named_code
    B.build()
    torch.cuda.set_device(0)
    spec = SERVING[args.workload]
    codes = [named_code(nm) for nm in spec["codes"]]
    prm = L.lpdec_default_params()
    prm.precision = {"fp64": L.LPDEC_FP64, "mixed": L.LPDEC_MIXED, "m32": L.LPDEC_M32}[args.precision]
    budget = int(args.serve_budget_gb * (1 << 30))
    levels = {}
    offset = 0

    def frames_for(count):
        nonlocal offset
        fr = serving_frames(spec, codes, count, offset)
        offset += count
        return fr

    with L.Server(codes, params=prm, hbm_budget_bytes=budget, max_pending=1 << 15) as srv:
        serve_run(srv, serving_frames(spec, codes, 64, 10 ** 6), stop_after=60.0)   # warm-up
        # saturated: more frames than the run can finish, all offered at once;
        # the rate is taken over the last 60% of the run (the pipeline full)
        T = args.sat_seconds
        fr = frames_for(30000)
        el, lat, fin, st = serve_run(srv, fr, stop_after=T)
        w0 = 0.4 * T
        sat = float(np.sum((fin >= w0) & (fin <= T))) / (T - w0)
        print(f"[serving] saturated: {sat:.1f} frames/s over [{w0:.0f}, {T:.0f}] s",
              file=sys.stderr, flush=True)
        levels["saturated"] = {"frames_per_s": sat, "window_s": [w0, T],
                               "frames_finished": int(np.sum(~np.isnan(fin))),
                               "frames_ok": int((st == 0).sum())}
        for load in (0.5, 0.8, 0.95):
            rate = load * sat
            cnt = max(1, int(rate * args.serve_seconds))
            fr = frames_for(cnt)
            el, lat, fin, st = serve_run(srv, fr, rate=rate,
                                         stop_after=args.serve_seconds + args.serve_grace)
            served = ~np.isnan(lat)
            print(f"[serving] load {load}: {int(served.sum())}/{cnt} frames served",
                  file=sys.stderr, flush=True)
            levels[f"poisson_{int(load * 100)}pct"] = {
                "offered_frames_per_s": rate, "offered_frames": cnt,
                "frames_per_s_served": float(served.sum()) / el,
                **latency_summary(lat, cnt),
                "frames_served": int(served.sum()), "frames_ok": int((st == 0).sum()),
                "frames_cancelled_at_end": int((st == L_CANCELLED).sum())}
        hbm, arena, used, out = srv.stats()
    line = {
        "metric": f"served LP-decoded frames/s, {args.workload} mixed lengths; p50/p99/p99.9 latency",
        "value": sat, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {spec['what']}; saturated for {args.sat_seconds:.0f} s, "
                               f"then Poisson arrivals at 50/80/95% of that rate for "
                               f"{args.serve_seconds:.0f} s each (frame counts scaled down from "
                               f"the configuration's to bound the run)",
                   "codes": spec["codes"], "hbm_budget_gb": args.serve_budget_gb,
                   "server_device_bytes": hbm, "precision": args.precision,
                   "grace_s": args.serve_grace},
        "levels": levels,
        "latency": "host clock from a frame's arrival (its scheduled Poisson time) to the poll "
                   "that returns its result; frames still running grace_s after the last "
                   "arrival are cancelled and count as slower than every served frame",
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# c3: precision study at n = 16000
# ---------------------------------------------------------------------------

def _full_lp_worker(args):
    f, ebn0 = args
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    from oracle import feldman
    from synth import awgn_llr_frames, named_code
    c = named_code("gallager_16000")
    g = awgn_llr_frames(c.n, c.design_rate, ebn0, SEED, [f])[0]
    u, obj = feldman.lp_decode_sparse(c, g)
    return f, obj


def run_c3(args):
    import numpy as np
    import torch
    from paper_0902_0657_gb300 import build as B
    from paper_0902_0657_gb300 import lpdec as L
    from synth import awgn_llr_frames, named_code
    ebn0 = 1.8
    cfut = None
    pool = None
    if args.c3_oracle_frames > 0:   # the full LP on host cores while the GPU runs
        pool = mp.get_context("spawn").Pool(args.c3_oracle_frames)
        cfut = pool.map_async(_full_lp_worker, [(f, ebn0) for f in range(args.c3_oracle_frames)])
    B.build()
    torch.cuda.set_device(0)
    code = named_code("gallager_16000")
    nf = args.c3_frames
    G = awgn_llr_frames(code.n, code.design_rate, ebn0, SEED, range(nf))
    modes = {}
    outs = {}
    for name, prec in (("fp64", L.LPDEC_FP64), ("mixed", L.LPDEC_MIXED)):
        prm = L.lpdec_default_params()
        prm.precision = prec
        if args.max_pcg > 0:
            prm.max_pcg = args.max_pcg
        prm.precond = {"column": L.LPDEC_MTS_COLUMN, "incremental": L.LPDEC_MTS_INCREMENTAL,
                       "rowwise": L.LPDEC_MTS_ROWWISE, "adaptive": L.LPDEC_MTS_ADAPTIVE,
                   "rowwise-tri": L.LPDEC_MTS_ROWWISE_TRI}[args.precond]
        with L.Decoder(code, params=prm) as d:
            d_g = torch.from_numpy(G).cuda()
            d_u = torch.empty((nf, code.n), dtype=torch.float64, device="cuda")
            d_h = torch.empty((nf, code.n), dtype=torch.uint8, device="cuda")
            d_c = torch.empty(nf, dtype=torch.int32, device="cuda")
            d_m = torch.empty((nf, code.m), dtype=torch.int32, device="cuda")
            d_s = torch.empty(nf * L.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rc = L.lpdec_decode_batch_device(d.ctx, d.code, nf, d_g, d_u, d_h, d_c, d_m, d_s)
            e1.record()
            e1.synchronize()
            if rc != 0:
                raise RuntimeError(L.error_string(rc))
            sec = e0.elapsed_time(e1) / 1e3
            st = d_s.cpu().numpy().view(L.STATS_DTYPE)
            outs[name] = (d_u.cpu().numpy(), d_h.cpu().numpy(), d_c.cpu().numpy(),
                          d_m.cpu().numpy().view(np.uint32), st)
            trace = None
            if name == "fp64":   # spectrum of the last LP of frame 0 along its interior-point run
                mk = outs[name][3][0:1]
                in_lp = (mk != 0).astype(np.uint8)
                qm = code.n + code.m
                mt = 200
                d_x = torch.zeros((1, qm), dtype=torch.float64, device="cuda")
                d_s1 = torch.zeros(L.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
                d_t = torch.full((mt * 10,), float("nan"), dtype=torch.float64, device="cuda")
                rc = L.lpdec_lp_solve_trace_device(d.ctx, d.code, 1, d_g[0:1],
                                                   torch.from_numpy(in_lp).cuda(),
                                                   torch.from_numpy(mk).cuda(), d_x, d_s1, d_t, mt)
                torch.cuda.synchronize()
                tr = d_t.cpu().numpy().reshape(mt, 10)
                k = int(d_s1.cpu().numpy().view(L.STATS_DTYPE)["ipm_iters_total"][0])
                trace = [{"it": i, "gap": float(tr[i, 0]), "pcg_iters": int(tr[i, 3]),
                          "cond_MinvQ_lanczos": float(tr[i, 9] / tr[i, 8]) if tr[i, 8] > 0 else None}
                         for i in range(min(k, mt)) if np.isfinite(tr[i, 0])]
            modes[name] = {
                "seconds": sec, "frames_per_s": nf / sec,
                "frames_ok": int((st["status"] == 0).sum()),
                "frames_integral": int((outs[name][2] == 1).sum()),
                "mean_lps": float(st["alp_iters"].mean()),
                "mean_ipm_iters": float(st["ipm_iters_total"].mean()),
                "pcg_iters_per_ipm_iter": float(st["pcg_iters_total"].sum() /
                                                max(1, st["ipm_iters_total"].sum())),
                "fp64_share_of_pcg_iters": float(st["pcg_iters_fp64"].sum() /
                                                 max(1, st["pcg_iters_total"].sum())),
                "dense_solves": int(st["dense_solves"].sum()),
                "vertex_failures": int(st["vertex_failures"].sum()),
            }
            if trace is not None:
                modes[name]["trace_last_lp_frame0"] = trace
    u64, h64, c64, m64, s64 = outs["fp64"]
    u32, h32, c32, m32, s32 = outs["mixed"]
    agree = {
        "hard_equal": int(sum(np.array_equal(h64[f], h32[f]) for f in range(nf))),
        "cert_equal": int((c64 == c32).sum()), "cutset_equal": int(sum(np.array_equal(m64[f], m32[f]) for f in range(nf))),
        "max_abs_du": float(np.abs(u64 - u32).max()),
        "max_rel_dobj": float(np.max(np.abs(s64["objective"] - s32["objective"]) /
                                     (1 + np.abs(s64["objective"])))),
    }
    full = None
    if cfut is not None:
        res = cfut.get()
        pool.close()
        full = [{"frame": f, "full_lp_objective": obj,
                 "fp64_rel_err": abs(float(s64["objective"][f]) - obj) / (1 + abs(obj)),
                 "mixed_rel_err": abs(float(s32["objective"][f]) - obj) / (1 + abs(obj))}
                for f, obj in res]
    line = {
        "metric": "c3 precision study: (3,6) n=16000 LP decoding, FP32 PCG + FP64 refinement vs FP64",
        "value": modes["fp64"]["frames_per_s"], "unit": UNIT, "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic",
        "config": {"workload": f"(3,6) Gallager n=16000 m=8000 (seed 0), Eb/N0 1.8 dB, frames 0..{nf - 1} "
                               f"of the seed-0 pool (a subset of the configuration's 2000)",
                   "max_pcg": args.max_pcg or 1000, "precond": args.precond},
        "modes": modes, "fp64_vs_mixed": agree, "vs_full_lp": full,
        "full_lp": "Feldman's LP over all 8000 x 32 parity inequalities, HiGHS dual simplex on the "
                   "host (Theorem 2(c): the LP decoding optimum)",
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# c1: the plain form (one frame per launch) against the batched form
# ---------------------------------------------------------------------------

def run_c1(args):
    import numpy as np
    import torch
    from paper_0902_0657_gb300 import build as B
    from paper_0902_0657_gb300 import lpdec as L
    from synth import awgn_llr_frames, named_code
    B.build()
    torch.cuda.set_device(0)
    code = named_code("gallager_120")
    nf = 200
    G = torch.from_numpy(awgn_llr_frames(code.n, code.design_rate, 2.0, SEED, range(nf))).cuda()
    out = {}
    with L.Decoder(code) as d:
        d_u = torch.empty((nf, code.n), dtype=torch.float64, device="cuda")
        d_h = torch.empty((nf, code.n), dtype=torch.uint8, device="cuda")
        d_c = torch.empty(nf, dtype=torch.int32, device="cuda")
        d_s = torch.empty(nf * L.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream()
        for _ in range(3):   # warm-up
            L.lpdec_decode_batch_device(d.ctx, d.code, nf, G, d_u, d_h, d_c, None, d_s, stream=stream)
        torch.cuda.synchronize()
        for form in ("plain", "batched"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if form == "plain":
                for f in range(nf):
                    rc = L.lpdec_decode_batch_device(d.ctx, d.code, 1, G[f:f + 1], d_u[f:f + 1],
                                                     d_h[f:f + 1], d_c[f:f + 1], None,
                                                     d_s[f * L.STATS_DTYPE.itemsize:],
                                                     stream=stream)
                    assert rc == 0
            else:
                rc = L.lpdec_decode_batch_device(d.ctx, d.code, nf, G, d_u, d_h, d_c, None, d_s,
                                                 stream=stream)
                assert rc == 0
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            st = d_s.cpu().numpy().view(L.STATS_DTYPE)
            out[form] = {"frames_per_s": nf / sec, "seconds": sec,
                         "frame_device_ms_p50": 1e3 * float(np.percentile(st["seconds"], 50)),
                         "frame_device_ms_p99": 1e3 * float(np.percentile(st["seconds"], 99)),
                         "frames_ok": int((st["status"] == 0).sum())}
    line = {"metric": "c1: (3,6) n=120 LP decoding, plain form (one frame per launch) vs one batched "
                      "launch", "value": out["batched"]["frames_per_s"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "(3,6) Gallager n=120 m=60 (seed 0), Eb/N0 2 dB, 200 frames "
                                   "(seed 0), FP64, device-timed with CUDA events"},
            "forms": out,
            "batched_over_plain": out["batched"]["frames_per_s"] / out["plain"]["frames_per_s"]}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# x123: iteration counts of ALP, MALP-A and MALP-B against code length
# ---------------------------------------------------------------------------

X_LENGTHS = (120, 240, 480, 720, 960, 1200, 1800, 2400)


def run_x123(args):
    import numpy as np
    import torch
    from paper_0902_0657_gb300 import build as B
    from paper_0902_0657_gb300 import lpdec as L
    from synth import awgn_llr_frames, named_code
    B.build()
    torch.cuda.set_device(0)
    variants = (("ALP", L.LPDEC_ALP), ("MALP-A", L.LPDEC_MALP_A), ("MALP-B", L.LPDEC_MALP_B))
    table = []
    for n in X_LENGTHS:
        code = named_code(f"gallager_{n}")
        G = awgn_llr_frames(code.n, code.design_rate, 2.0, SEED, range(args.x_trials))
        row = {"n": n}
        largest = {}
        for name, var in variants:
            prm = L.lpdec_default_params()
            prm.variant = var
            if var == L.LPDEC_ALP:   # ALP's cut lists outgrow the default 2m rows
                prm.lp_rows_cap = 4 * code.m
            with L.Decoder(code, params=prm) as d:
                u, hard, cert, masks, st = d.decode_batch(G)
            lps = st["alp_iters"].astype(float)
            integ = cert == 1
            ent = {}
            for lab, sel in (("integral", integ), ("fractional", ~integ)):
                if sel.any():
                    ent[lab] = {"frames": int(sel.sum()), "mean_lps": float(lps[sel].mean()),
                                "p95_lps": float(np.sort(lps[sel])[int(np.ceil(0.95 * sel.sum())) - 1]),
                                "mean_largest_lp_rows": float(st["lp_rows_max"][sel].mean())}
            ent["frames_ok"] = int((st["status"] == 0).sum())
            ent["status_counts"] = {str(int(k)): int(v) for k, v in
                                    zip(*np.unique(st["status"], return_counts=True))}
            ent["frames_switched_to_alp"] = int((st["alp_switch"] > 0).sum())
            row[name] = ent
            largest[name] = st["lp_rows_max"].astype(float), integ
        for name in ("MALP-A", "MALP-B"):
            red = {}
            for lab, val in (("integral", True), ("fractional", False)):
                rm, integ = largest[name]
                ra, _ = largest["ALP"]
                sel = (integ == val) & (ra > 0)
                if sel.any():
                    red[lab] = float(1.0 - rm[sel].mean() / ra[sel].mean())
            row[f"{name}_largest_lp_reduction_vs_ALP"] = red
        table.append(row)
    line = {"metric": "Section III-D iteration counts (X1-X3): LPs per frame of ALP, MALP-A, MALP-B",
            "unit": "LPs per frame", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"(3,6) Gallager codes n in {list(X_LENGTHS)} (seed 0), "
                                   f"Eb/N0 2 dB, {args.x_trials} frames each (seed-0 pool)",
                       "alp_lp_rows_cap": "4 m"},
            "table": table}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import named_code
    code = named_code(CODE_NAME)
    total_done, total_wall, cores = 0, 0.0, 1
    for k in range(args.warmup + args.steps):
        done, w, cores = run_oracle_sample(args.oracle_seconds, offset=k * 997, ebn0=args.ebn0)
        if k >= args.warmup:
            total_done += done
            total_wall += w
    value = total_done / total_wall
    sample = (f"{total_done} frames over {args.steps} timed steps, {cores} spawned "
              f"single-threaded oracle workers, ~{args.oracle_seconds:.0f} s per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, code.n, code.m),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in SERVING:
        run_serving(args)
    elif args.workload == "c3":
        run_c3(args)
    elif args.workload == "x123":
        run_x123(args)
    elif args.workload == "c1":
        run_c1(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

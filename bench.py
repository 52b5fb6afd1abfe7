#!/usr/bin/env python3
"""Throughput benchmark of the fused third-order (CEC) semi-Lagrangian step.

Workload (default ``abc512``): 3D periodic [0, 2 pi)^3 grid of 512^3 cells,
FP32, steady ABC flow (A = B = C = 1), scalar = sum of 32 random Fourier modes
with |k| <= 8 (seed 0), CFL 0.8, split CEC step with the sweep order
alternating every step; 512^3 is the size the HBM-roofline target is stated
for, and ``--n 256`` runs the same flow at 256^3 (also reported beside the
headline).  One step = one fused kernel launch that advances every cell once;
the metric is cell-updates per second (Gcell/s).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s at fixed L2 error: plain 3rd-order vs batched/learned forms"
UNIT = "Gcell/s"
BYTES_PER_CELL = 20          # read Phi (4) + u (12), write Phi (4)
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0   # dense bf16 burst, one earlier GB300 measurement
# tensor-core FLOPs per cell of the learned corrector: 67 -> 64 and 64 -> 64 layers
LEARNED_TC_FLOP_PER_CELL = 2 * (67 * 64 + 64 * 64)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512, help="cells per axis")
    ap.add_argument("--no-extras", action="store_true", help="skip the per-scheme and batched side measurements")
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and timed CEC steps (for ncu); prints the plain timing line")
    ap.add_argument("--profile-wide", action="store_true",
                    help="only run warmup + steps wide CEC steps (CFL 3.64) on the workload, for ncu")
    ap.add_argument("--profile-learned", action="store_true",
                    help="only warm-up and timed learned-corrector steps (untrained weights; for ncu)")
    ap.add_argument("--profile-rb", action="store_true",
                    help="only the Rayleigh-Benard run (50x50, every scheme, 1000 steps each; for ncu); prints "
                         "its record")
    ap.add_argument("--rb-steps", type=int, default=1000, help="steps of each --profile-rb run")
    ap.add_argument("--scheme", choices=["CIR", "FEC", "BEC", "CEC"], default="CEC",
                    help="scheme of the --profile steps")
    ap.add_argument("--jsonl", default=None,
                    help="also append one JSON record per measurement of the line to this file")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def slowest_rank_ms(ms, world, device):
    """Max over ranks of a per-rank elapsed time (every rank gets the result)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, steps, world, slowest_ms):
    """Cell-updates per second of the whole job (all ranks' cells over the slowest rank's time), in G."""
    return world * cells_per_rank * steps / (slowest_ms * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"

    def find(obj):
        if isinstance(obj, dict):
            for k, v in obj.items():
                if "hbm" in k.lower() and isinstance(v, (int, float)):
                    return float(v)
                r = find(v)
                if r:
                    return r
        return None
    v = find(d)
    return (v, "measured") if v else (FALLBACK_HBM_GBS, "fallback")


def measured_bf16_peak():
    """Dense bf16 TFLOP/s (burst) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
    except Exception:
        return FALLBACK_BF16_TFLOPS, "fallback"
    v = d.get("bf16_tflops") if isinstance(d, dict) else None
    return (float(v), "measured") if isinstance(v, (int, float)) else (FALLBACK_BF16_TFLOPS, "fallback")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_cec_fast.cu", "sl_common.cuh"):
        with open(os.path.join(ROOT, "paper_1606_06117_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic(workload):
    """DRAM bytes per launch of the CEC kernel from the committed ncu summary, or
    None when the summary is missing or was taken on other kernel sources."""
    p = os.path.join(ROOT, "profiles", f"k_cec_fast_{workload}.md")
    try:
        text = open(p).read()
    except OSError:
        return None
    m = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(n, device, torch):
    from paper_1606_06117_gb300 import workloads as W
    shape = (n, n, n)
    phi = W.random_modes(shape, W.draw_modes(3, 32, 8, seed=0), device=device, dtype=torch.float32)
    vel = W.abc_velocity(shape, device=device, dtype=torch.float32)
    sp = [2 * math.pi / n] * 3
    dt = 0.8 * sp[0] / 2.0          # max |u_d| = 2 for A = B = C = 1
    return phi, vel, sp, dt


# ------------------------------------------------------------- CPU oracle
def host_cores():
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


class OracleReplicas:
    """The FP64 oracle's CEC step on an n_sample^3 grid of the same workload, run
    by `threads` threads at once, each stepping its own copy of the sample.  The
    oracle is reentrant C called through ctypes, which releases the interpreter
    lock, so the threads occupy that many cores.  The oracle itself is unchanged."""

    def __init__(self, n_sample, threads):
        import torch

        from oracle import oracle as O
        self.O = O
        phi, vel, sp, dt = workload(n_sample, "cpu", torch)
        p = phi.double().numpy()
        self.c = vel.double().numpy() * (dt / sp[0])
        self.p = [p.copy() for _ in range(threads)]
        self.cells = n_sample ** 3
        self.threads = threads
        self.k = 0
        self.pool = None
        if threads > 1:
            from concurrent.futures import ThreadPoolExecutor
            self.pool = ThreadPoolExecutor(max_workers=threads)

    def _one(self, i):
        self.p[i] = self.O.step(self.p[i], self.c, self.O.CEC, self.k)

    def step(self):
        """One step of every replica; returns when all have finished."""
        if self.pool is None:
            self._one(0)
        else:
            list(self.pool.map(self._one, range(self.threads)))
        self.k += 1

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()


def rb_oracle_rate(n, Ra, dt, nsteps=200):
    """Time per step of the FP64 oracle's Rayleigh-Benard box (one thread of
    numpy; the dense pseudo-inverse is built before the timed steps)."""
    from oracle import rb_oracle as R
    from paper_1606_06117_gb300 import workloads as W
    box = R.Box(n, n, Ra=Ra, scheme="CEC")
    box.theta = W.rb_spots(n, n)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        box.step(dt)
    el = time.perf_counter() - t0
    return {"value": el / nsteps * 1e6, "unit": "us/step", "cores": 1, "kind": "oracle",
            "sample": f"{nsteps} CEC steps of the {n}x{n} box ({el:.1f} s)"}


def oracle_rate(n_sample, max_seconds, threads=1, min_steps=1):
    """Aggregate cell-updates/s of `threads` oracle replicas, stepped until
    max_seconds have passed (and at least min_steps steps)."""
    r = OracleReplicas(n_sample, threads)
    steps, t0 = 0, time.perf_counter()
    while True:
        r.step()
        steps += 1
        el = time.perf_counter() - t0
        if steps >= min_steps and el >= max_seconds:
            break
    r.close()
    return steps * threads * r.cells / el / 1e9, steps, el


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each timed step is one oracle CEC step on every host core, each core on its
    # own copy of a smaller periodic grid of the same flow (identical per-cell
    # work), sized so the whole run stays within ~2 minutes
    budget = 120.0 / max(1, args.steps + args.warmup)
    m = 16
    for cand in (16, 24, 32, 48, 64, 96, 128):
        if cand ** 3 / 3.0e6 <= budget:
            m = cand
    cores = host_cores()
    r = OracleReplicas(m, cores)
    for _ in range(args.warmup):
        r.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.step()
    el = time.perf_counter() - t0
    r.close()
    value = args.steps * cores * m ** 3 / el / 1e9
    sample = (f"per timed step, one FP64 oracle CEC step on each of {cores} threads, each on its own copy of "
              f"a {m}^3 grid of the same ABC / 32-mode workload")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"abc{args.n}_cec_f32", "sample_grid": m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ metrics records
def jsonl_records(line, when=None):
    """Flatten a bench line into one record per measurement: throughput
    (Gcell/s and GB/s of algorithmic bytes), roofline fraction, errors against
    the oracle or the exact solution, and the host cores of the CPU baseline."""
    when = when or time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    base = {"time": when, "n_gpus": line.get("n_gpus"), "clocks": line.get("clocks")}
    recs = []
    roof = line.get("roofline") or {}
    recs.append(dict(base, record="headline", workload=line["config"]["workload"], gcell_s=line["value"],
                     ms_per_step=line["ms_per_step"], gb_s=roof.get("achieved"), roofline_frac=roof.get("frac"),
                     traffic_bytes=roof.get("traffic"), launch=line["config"].get("launch")))
    if line.get("e2e"):
        recs.append(dict(base, record="e2e", gcell_s=line["e2e"]["value"],
                         h2d_bytes_per_step=line["e2e"]["h2d_bytes_per_step"],
                         d2h_bytes_per_step=line["e2e"]["d2h_bytes_per_step"]))
    if line.get("cpu_baseline"):
        cb = line["cpu_baseline"]
        recs.append(dict(base, record="cpu_baseline", gcell_s=cb["value"], host_cores=cb["cores"], sample=cb["sample"]))
    for name, r in (line.get("schemes") or {}).items():
        gb = BYTES_PER_CELL * r["gcell_s"]   # GB/s of algorithmic bytes
        peak = roof.get("peak")
        recs.append(dict(base, record="scheme", scheme=name, gcell_s=r["gcell_s"], ms_per_step=r["ms_per_step"],
                         gb_s=gb, roofline_frac=gb / peak if peak else None,
                         roundtrip_rel_l2=r.get("roundtrip_rel_l2_100_100"), launch=r.get("launch")))
    if line.get("cec_256"):
        c = line["cec_256"]
        recs.append(dict(base, record="cec_256", gcell_s=c["gcell_s"], ms_per_step=c["ms_per_step"],
                         gb_s=c["roofline"]["achieved"], roofline_frac=c["roofline"]["frac"]))
    if line.get("batched_c3"):
        b = line["batched_c3"]
        recs.append(dict(base, record="batched_c3", gcell_s=b["batched_graph"]["gcell_s"],
                         plain_gcell_s=b["plain_48_launches"]["gcell_s"], launch=b.get("launch")))
    if line.get("deformation_c5"):
        d = line["deformation_c5"]
        recs.append(dict(base, record="deformation_c5", field_gcell_s=d["field_gcell_s"],
                         rel_l2_vs_exact=d.get("rel_l2_at_T")))
    if line.get("learned_c4"):
        lc = line["learned_c4"]
        recs.append(dict(base, record="learned_c4", gcell_s=lc["learned_gcell_s"],
                         roofline_frac=lc["roofline"]["frac"], fell_back_at_step=lc.get("fell_back_at_step"),
                         checks=lc.get("checks")))
        if lc.get("deformation_c5_learned"):
            dl = lc["deformation_c5_learned"]
            recs.append(dict(base, record="deformation_c5_learned", fell_back_at_step=dl["fell_back_at_step"],
                             rel_l2_vs_exact=dl["rel_l2_at_T"]))
    if line.get("rotation_c1"):
        r = line["rotation_c1"]
        recs.append(dict(base, record="rotation_c1", **{k: {"rel_l2_vs_exact": v["rel_l2"], "linf_vs_exact": v["linf"]}
                                                         for k, v in r.items() if isinstance(v, dict)}))
    if line.get("large_cfl_f2"):
        w = line["large_cfl_f2"]
        recs.append(dict(base, record="large_cfl_f2", gcell_s=w["gcell_s"], roofline_frac=w["roofline"]["frac"],
                         roundtrip_rel_l2=w["roundtrip_rel_l2"]))
    if line.get("rayleigh_benard_f4"):
        rb = line["rayleigh_benard_f4"]
        recs.append(dict(base, record="rayleigh_benard_f4", grid=rb["grid"],
                         **{k: {"us_per_step": v["us_per_step"], "top_reached_at_step": v["top_reached_at_step"]}
                            for k, v in rb.items() if k in ("CIR", "FEC", "BEC", "CEC")}))
    return recs


def write_jsonl(path, line):
    with open(path, "a") as fh:
        for rec in jsonl_records(line):
            fh.write(json.dumps(rec) + "\n")


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1606_06117_gb300 import _lib as sl

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sl.load()
    sl.sl_init()

    n = args.n
    ncell = n ** 3
    phi, vel, sp, dt = workload(n, dev, torch)
    dims = [n, n, n]
    a, b = phi.clone(), torch.empty_like(phi)
    stream = torch.cuda.current_stream()
    if args.profile_wide:
        # the large-CFL step of large_cfl_measurement: 22 steps cover 100 steps of CFL 0.8
        dtw = 100 * dt / int(math.ceil(100 * dt * 2.0 / sp[0] / 3.75 - 1e-12))
        need = sl.sl_advect_wide_workspace(3, dims, sl.CEC, sl.F32)
        ws_t = torch.empty(need + 256, dtype=torch.uint8, device=dev)
        ws = ws_t.data_ptr() + (-ws_t.data_ptr()) % 256
        for k in range(args.warmup + args.steps):
            sl.sl_advect_wide(b, a, vel, 3, dims, sp, dtw, sl.CEC, sl.F32, k & 1, ws, need, stream)
            a, b = b, a
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_wide_run": True, "steps": args.steps}), flush=True)
        return

    if args.profile_learned:
        # the learned step's work does not depend on the weights' values
        c = sl.sl_corrector_create(0)
        try:
            for k in range(args.warmup + args.steps):
                sl.sl_advect_learned(c, b, a, vel, 3, dims, sp, dt, k & 1, 0, 2.0, stream)
                a, b = b, a
            torch.cuda.synchronize()
        finally:
            sl.sl_corrector_destroy(c)
        if rank == 0:
            print(json.dumps({"profile_learned_run": True, "steps": args.steps}), flush=True)
        return

    scheme = getattr(sl, args.scheme) if args.profile else sl.CEC
    # the library's autotuner picks the launch shape (it only regroups work: the
    # results are bitwise those of the default shape); b is scratch here
    tuned = sl.sl_autotune_scheme(b, a, vel, 3, dims, sp, dt, scheme, sl.F32, stream).as_dict()

    def step(k, src, dst):
        sl.sl_advect(dst, src, vel, 3, dims, sp, dt, scheme, sl.F32, k & 1, stream)

    for k in range(args.warmup):
        step(k, a, b)
        a, b = b, a
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)   # let the sampler see the loaded GPU from the first step on
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for k in range(args.steps):
        step(k, a, b)
        a, b = b, a
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": ms / args.steps, "steps": args.steps}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    ms_max = slowest_rank_ms(ms, world, dev)
    ms_step = ms_max / args.steps
    value = whole_job_rate(ncell, args.steps, world, ms_max)
    sl_status = sl.sl_device_status(stream)

    # per-launch kernel time (one launch per step) for the roofline
    peak, peak_kind = measured_hbm_peak()
    achieved = BYTES_PER_CELL * ncell / (ms / args.steps * 1e-3) / 1e9
    traffic = profiled_traffic(f"abc{n}")

    # ------------------------------------------------ end to end, host buffers
    ke = max(10, min(200, args.steps // 50))
    h_in = phi.cpu().pin_memory()
    h_vel = vel.cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    for k in range(2):
        sl.sl_advect_host(h_out, h_in, h_vel, 3, dims, sp, dt, sl.CEC, sl.F32, k & 1, stream)
    barrier()
    t0 = time.perf_counter()
    for k in range(ke):
        sl.sl_advect_host(h_out, h_in, h_vel, 3, dims, sp, dt, sl.CEC, sl.F32, k & 1, stream)
        h_in, h_out = h_out, h_in
    barrier()
    el = time.perf_counter() - t0
    el_max = slowest_rank_ms(el * 1e3, world, dev)
    e2e = {"value": whole_job_rate(ncell, ke, world, el_max), "unit": UNIT,
           "h2d_bytes_per_step": 16 * ncell, "d2h_bytes_per_step": 4 * ncell, "steps": ke,
           "api": "sl_advect_host (pinned host buffers; every step copies phi and u in, steps and copies phi "
                  "back in 8 z slabs on three streams, and returns once the result is on the host)"}

    extras = {}
    if not args.no_extras and world == 1:   # per-GPU figures; the same at every N
        extras = side_measurements(torch, sl, dev, stream, n, phi, vel, sp, dt)
        del a, b
        torch.cuda.empty_cache()
        extras["batched_c3"] = batched_measurement(torch, sl, stream)
        torch.cuda.empty_cache()
        extras["deformation_c5"] = deformation_measurement(torch, sl, stream)
        torch.cuda.empty_cache()
        extras["cec_256" if n != 256 else "cec_512"] = cec_size_measurement(torch, sl, stream,
                                                                           256 if n != 256 else 512)
        torch.cuda.empty_cache()
        extras["rotation_c1"] = rotation_measurement(torch, sl, stream)
        extras["resolution_f1"] = resolution_measurement(torch, sl, stream)
        extras["shear_f3"] = shear_measurement(torch, sl, stream)
        torch.cuda.empty_cache()
        extras["large_cfl_f2"] = large_cfl_measurement(torch, sl, stream)
        extras["learned_c4"] = learned_measurement(torch, sl, stream)
        extras["rayleigh_benard_f4"] = rb_measurement(torch, sl, stream)

    cpu = None
    if rank == 0 and world == 1:
        m = 96 if n >= 96 else n
        cores = host_cores()
        rate, steps, secs = oracle_rate(m, max_seconds=10.0, threads=cores, min_steps=2)
        rate1, steps1, secs1 = oracle_rate(m, max_seconds=10.0, threads=1, min_steps=2)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{steps} FP64 oracle CEC steps on each of {cores} threads, each on its own copy of a "
                         f"{m}^3 grid of the same workload ({secs:.1f} s)",
               "one_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"{steps1} steps on one {m}^3 grid ({secs1:.1f} s)"}}

    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"abc{n}_cec_f32", "grid": [n, n, n], "scheme": "CEC (split, fused)",
                           "cfl": 0.8, "flow": "ABC A=B=C=1", "scalar": "32 random modes |k|<=8 seed 0",
                           "l2": f"inputs larger than L2: {20 * ncell / 1e6:.0f} MB working set per step",
                           "parallelism": f"replicas x{world}", "launch": tuned},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                             "kernel": "k_cec_xyz_fast / k_cec_zyx_fast (alternating)",
                             "bytes_per_launch": BYTES_PER_CELL * ncell},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps, "clocks": clk,
                "device_status": sl_status}
        line.update(extras)
        print(json.dumps(line), flush=True)
        if args.jsonl:
            write_jsonl(args.jsonl, line)
    if world > 1:
        dist.destroy_process_group()


def time_steps(torch, stream, fn, steps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(steps):
        fn(k)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def side_measurements(torch, sl, dev, stream, n, phi, vel, sp, dt):
    """Per-scheme throughput, and each scheme's accuracy on the workload: 100
    steps forward then 100 steps with the flow reversed (dt -> -dt) must return
    the initial field; the relative L2 distance to it is computed on the device
    in FP64 (sl_norms)."""
    out = {}
    dims = [n, n, n]
    a = phi.clone()
    b = torch.empty_like(phi)
    rates = {}
    for name, code, dtc in (("CIR", sl.CIR, sl.F32), ("FEC", sl.FEC, sl.F32), ("BEC", sl.BEC, sl.F32),
                            ("CEC", sl.CEC, sl.F32), ("CEC_f32_d64", sl.CEC, sl.F32_D64)):
        def fn(k, code=code, dtc=dtc):
            sl.sl_advect(b, a, vel, 3, dims, sp, dt, code, dtc, k & 1, stream)
        tuned = sl.sl_autotune_scheme(b, a, vel, 3, dims, sp, dt, code, dtc, stream).as_dict()
        fn(0)
        fn(1)
        ms = time_steps(torch, stream, fn, 50)
        x, y = phi.clone(), torch.empty_like(phi)
        for k in range(200):
            sl.sl_advect(y, x, vel, 3, dims, sp, dt if k < 100 else -dt, code, dtc, k & 1, stream)
            x, y = y, x
        rel = sl.sl_norms(x, phi, phi.numel(), sl.F32, stream)[2]
        rates[name] = {"gcell_s": n ** 3 / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                       "roundtrip_rel_l2_100_100": rel, "launch": tuned}
    out["schemes"] = rates
    return out


def batched_measurement(torch, sl, stream, steps=20):
    """48 independent grids of sizes drawn from {64..192}^3 (ABC or Taylor-Green
    velocity, amplitudes in [0.5, 1.5], random-mode scalar, CFL 0.8): one
    persistent launch per step (captured in a CUDA graph) against 48 separate
    sl_advect launches per step."""
    from paper_1606_06117_gb300 import workloads as W
    insts = W.draw_batch(48, seed=0)
    recs, keep, cells = [], [], 0
    for inst in insts:
        phi, vel = W.instance_fields(inst, device="cuda", dtype=torch.float32)
        n = inst.n
        sp = [2 * math.pi / n] * 3
        umax = float(vel.abs().amax())
        dt = 0.8 * sp[0] / umax
        a, b = phi, torch.empty_like(phi)
        keep.append((a, b, vel, n, sp, dt))
        recs.append(sl.Instance(a.data_ptr(), b.data_ptr(), vel.data_ptr(), (n, n, n), tuple(sp), dt))
        cells += n ** 3
    h = sl.sl_batch_create(recs)
    try:
        tuned = sl.sl_batch_autotune(h, stream).as_dict()   # overwrites the B buffers only
        sl.sl_batch_step(h, 0, stream)
        sl.sl_batch_step(h, 1, stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cap = torch.cuda.current_stream()
            sl.sl_batch_step(h, 0, cap)
            sl.sl_batch_step(h, 1, cap)
        for _ in range(3):
            g.replay()
        ms_b = time_steps(torch, stream, lambda k: g.replay(), steps) / 2.0

        def plain(k):
            for a, b, vel, n, sp, dt in keep:
                src, dst = (a, b) if k % 2 == 0 else (b, a)
                sl.sl_advect(dst, src, vel, 3, [n, n, n], sp, dt, sl.CEC, sl.F32, k & 1, stream)
        plain(0)
        plain(1)
        ms_p = time_steps(torch, stream, plain, 2 * steps)
    finally:
        sl.sl_batch_destroy(h)
    return {"instances": len(insts), "cells_per_step": cells, "launch": tuned,
            "batched_graph": {"gcell_s": cells / (ms_b * 1e-3) / 1e9, "ms_per_step": ms_b},
            "plain_48_launches": {"gcell_s": cells / (ms_p * 1e-3) / 1e9, "ms_per_step": ms_p}}


def learned_measurement(torch, sl, stream, n=256, steps=500, check_every=25):
    """Learned corrector (67-64-64-1 BF16 MLP on the tensor cores): trained on
    128^3 ABC / Taylor-Green random-mode fields advected by the plain CEC step,
    then run on the n^3 ABC workload for `steps` steps with a plain-scheme check
    every `check_every` steps and fallback above 2x the plain error.  Reports
    the learned and plain step rates, the training loss, the checked errors and
    the 100-forward / 100-reverse round-trip error of each path."""
    from paper_1606_06117_gb300 import workloads as W
    c = sl.sl_corrector_create(0)
    try:
        m = 128
        spm = [2 * math.pi / m] * 3
        flows = [W.abc_velocity((m,) * 3, device="cuda", dtype=torch.float32),
                 W.abc_velocity((m,) * 3, 1.3, 0.7, 1.1, device="cuda", dtype=torch.float32),
                 W.taylor_green_velocity((m,) * 3, 1.0, device="cuda", dtype=torch.float32),
                 W.taylor_green_velocity((m,) * 3, 1.4, device="cuda", dtype=torch.float32)]
        t0 = time.perf_counter()
        for i, v in enumerate(flows):
            dtm = 0.8 * spm[0] / float(v.abs().amax())
            cur = W.random_modes((m,) * 3, W.draw_modes(3, 32, 8, seed=20 + i), device="cuda", dtype=torch.float32)
            for k in range(6):
                nxt = sl.advect(cur, v, dtm, spm, "CEC", 0)
                sl.sl_corrector_add_samples(c, cur, nxt, v, [m] * 3, spm, dtm, 100000, seed=1000 * i + k)
                cur = sl.advect(cur, v, dtm, spm, "CEC", k)
        loss0 = sl.sl_corrector_train(c, 1, 4096, 1e-3, seed=1)
        # Adam with a stepped learning rate: 10k iterations at 1e-3, 10k at
        # 3e-4, 10k at 1e-4, 10k at 3e-5 (about 4 s)
        for seed, lr in ((2, 1e-3), (3, 3e-4), (4, 1e-4), (5, 3e-5)):
            loss = sl.sl_corrector_train(c, 10000, 4096, lr, seed=seed)
        train_s = time.perf_counter() - t0
        # evaluation on the bench workload
        phi, vel, sp, dt = workload(n, "cuda", torch)
        dims = [n] * 3
        a, b = phi.clone(), torch.empty_like(phi)

        def lstep(k):
            sl.sl_advect_learned(c, b, a, vel, 3, dims, sp, dt, k & 1, 0, 2.0, stream)
        lstep(0)
        lstep(1)
        ms_l = time_steps(torch, stream, lstep, 50)
        checks, fell_at = [], None
        x, y = phi.clone(), torch.empty_like(phi)
        for k in range(steps):
            chk = (k % check_every) == 0
            used, errs = sl.sl_advect_learned(c, y, x, vel, 3, dims, sp, dt, k & 1, int(chk), 2.0, stream)
            if chk:
                checks.append({"step": k, "learned_err": errs[0], "plain_err": errs[1], "plain_used": used})
            if used and fell_at is None:
                fell_at = k
            x, y = y, x
        # round-trip accuracy of each path (learned path without checks)
        sl.sl_corrector_reset(c)
        rt = {}
        for name in ("learned", "plain"):
            x, y = phi.clone(), torch.empty_like(phi)
            for k in range(200):
                d = dt if k < 100 else -dt
                if name == "learned":
                    sl.sl_advect_learned(c, y, x, vel, 3, dims, sp, d, k & 1, 0, 2.0, stream)
                else:
                    sl.sl_advect(y, x, vel, 3, dims, sp, d, sl.CEC, sl.F32, k & 1, stream)
                x, y = y, x
            rt[name] = sl.sl_norms(x, phi, phi.numel(), sl.F32, stream)[2]
        del a, b, x, y, phi, vel
        torch.cuda.empty_cache()
        deform = deformation_learned_run(torch, sl, stream, c)
    finally:
        sl.sl_corrector_destroy(c)
    peak, kind = measured_bf16_peak()
    tflops = LEARNED_TC_FLOP_PER_CELL * n ** 3 / (ms_l * 1e-3) / 1e12
    return {"train": {"grid": [128] * 3, "rows": 4 * 6 * 100000, "iters": 40000, "batch": 4096,
                      "lr": "1e-3, 3e-4, 1e-4, 3e-5 (10k iterations each)",
                      "loss_first": loss0, "loss_last": loss, "seconds": train_s},
            "learned_gcell_s": n ** 3 / (ms_l * 1e-3) / 1e9, "learned_ms_per_step": ms_l,
            "roofline": {"bound": "tensor", "kernel": "k_learned_step", "achieved": tflops, "peak": peak,
                         "unit": "TFLOP/s", "frac": tflops / peak, "peak_kind": kind,
                         "flop_per_cell": LEARNED_TC_FLOP_PER_CELL},
            "steps": steps, "check_every": check_every, "fell_back_at_step": fell_at, "checks": checks[:6],
            "roundtrip_rel_l2_100_100": rt, "deformation_c5_learned": deform}


def deformation_learned_run(torch, sl, stream, c, n=512, total_steps=2000, check_every=25):
    """Config 5 in its learned form: the time-reversing deformation flow at
    n^3, the three velocity components and the scalar each advanced by
    sl_advect_learned (plain-scheme check every `check_every` steps, fallback
    above 2x the plain error; one corrector, so a fallback holds for every
    field), velocity scaled by cos(pi t / T) as in the plain and multi-field
    runs; relative L2 error of each field at t = T against its initial field."""
    from paper_1606_06117_gb300 import workloads as W
    shape = (n, n, n)
    vel = W.deformation_velocity(shape, device="cuda", dtype=torch.float32)
    scal = W.random_modes(shape, W.draw_modes(3, 32, 8, seed=5), length=1.0, device="cuda", dtype=torch.float32)
    f0 = [vel[0].clone(), vel[1].clone(), vel[2].clone(), scal]
    sp = [1.0 / n] * 3
    dt = 0.8 * sp[0] / float(vel.abs().amax())
    T = total_steps * dt
    sl.sl_corrector_reset(c)
    cur = [f.clone() for f in f0]
    nxt = [torch.empty_like(f) for f in f0]
    fell_at, checks = None, []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(total_steps):
        d = dt * math.cos(math.pi * (k + 0.5) * dt / T)
        chk = int(k % check_every == 0)
        for i in range(4):
            used, errs = sl.sl_advect_learned(c, nxt[i], cur[i], vel, 3, [n] * 3, sp, d, k & 1, chk, 2.0, stream)
            if chk and i == 3 and len(checks) < 4:
                checks.append({"step": k, "learned_err": errs[0], "plain_err": errs[1], "plain_used": used})
            if used and fell_at is None:
                fell_at = k
        cur, nxt = nxt, cur
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    errs = [sl.sl_norms(x, f, f.numel(), sl.F32, stream)[2] for x, f in zip(cur, f0)]
    return {"grid": [n] * 3, "fields": 4, "steps_T": total_steps, "check_every": check_every,
            "fell_back_at_step": fell_at, "checks": checks, "seconds": secs,
            "rel_l2_at_T": {"u": errs[0], "v": errs[1], "w": errs[2], "scalar": errs[3]}}


def rotation_measurement(torch, sl, stream, n=128):
    """The 2D FP64 accuracy workload: a Gaussian (sigma 0.05 at (0.25, 0.5)) under
    solid-body rotation u = 2 pi (0.5 - y, x - 0.5), CFL 0.5, one revolution
    (805 steps at 128^2), every scheme; relative L2 and max error against the
    exact solution (the initial field), computed on the device in FP64."""
    from paper_1606_06117_gb300 import workloads as W
    shape = (n, n)
    phi0 = W.gaussian_unwrapped(shape, (0.25, 0.5), 0.05, device="cuda")
    vel = W.rotation_velocity(shape, device="cuda")
    dt, nsteps = W.dt_for_cfl(1.0, math.pi * n, 0.5)
    sp = [1.0 / n, 1.0 / n, 1.0]   # the ABI takes three entries; the third is unused in 2D
    out = {"grid": [n, n], "steps": nsteps, "dtype": "f64"}
    for name in ("CIR", "FEC", "BEC", "CEC"):
        code = getattr(sl, name)
        x, y = phi0.clone(), torch.empty_like(phi0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(nsteps):
            sl.sl_advect(y, x, vel, 2, [n, n, 1], sp, dt, code, sl.F64, k & 1, stream)
            x, y = y, x
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        nrm = sl.sl_norms(x, phi0, phi0.numel(), sl.F64, stream)
        out[name] = {"rel_l2": nrm[2], "linf": nrm[1], "us_per_step": el / nsteps * 1e6}
    return out


# Leading modified-equation coefficients of Table 1 for the first harmonic on
# the unit interval (u = 1, dt = U dx), written as c * u dx^(alpha - 1) with
# alpha the derivative order: decay of CIR (alpha 2), FEC / BEC / CEC (alpha 4),
# phase drift of FEC / BEC (alpha 3; CEC has no third-derivative term).
TABLE1_DECAY = {"CIR": (2, lambda U: (1 - U) / 2), "FEC": (4, lambda U: 3 * (1 - U * U) * U / 24),
                "BEC": (4, lambda U: 9 * (1 - U) ** 2 * U / 24),
                "CEC": (4, lambda U: (1 + U) * (1 - U) * (2 - U) / 24)}
TABLE1_DRIFT = {"FEC": lambda U: (1 - U * U) / 6, "BEC": lambda U: (1 - U) * (1 - 2 * U) / 6}


def resolution_measurement(torch, sl, stream, U=0.37, sizes=(64, 128, 256, 512)):
    """The App. B resolution study on the GPU: the first harmonic cos(2 pi x) on
    n cells along x (n x 32 x 8 grid, FP64), constant Courant number U along x.
    One step of cos and of sin gives the amplification g; the decay rate is
    sigma = -ln|g| / dt and the phase drift w = (arg g + U th) / dt.  Reported per
    scheme: sigma N^(alpha - 1) per N (constant when C_alpha ~ N^(1 - alpha)), the
    fitted exponent of sigma (1 - alpha), and the fitted coefficient at the
    largest N over Table 1's (decay; and phase drift for FEC, BEC)."""
    import numpy as np
    out = {"U": U, "sizes": list(sizes), "dtype": "f64", "axis": "x"}
    for name in ("CIR", "FEC", "BEC", "CEC"):
        code = getattr(sl, name)
        alpha, c_dec = TABLE1_DECAY[name]
        sig, drift = [], []
        for n in sizes:
            shape = (8, 32, n)
            th = 2 * math.pi / n
            j = torch.arange(n, dtype=torch.float64, device="cuda") * th
            cos = torch.cos(j).expand(shape).contiguous()
            sin = torch.sin(j).expand(shape).contiguous()
            vel = torch.zeros((3,) + shape, dtype=torch.float64, device="cuda")
            vel[0] = U
            a, b = torch.empty_like(cos), torch.empty_like(sin)
            sl.sl_advect(a, cos, vel, 3, [n, 32, 8], [1.0, 1.0, 1.0], 1.0, code, sl.F64, 0, stream)
            sl.sl_advect(b, sin, vel, 3, [n, 32, 8], [1.0, 1.0, 1.0], 1.0, code, sl.F64, 0, stream)
            torch.cuda.synchronize()
            z = torch.complex(a, b) * torch.exp(-1j * j)
            g = complex(z.mean().item())
            dt = U / n
            lg = complex(np.log(g))
            sig.append(-lg.real / dt)
            drift.append((lg.imag + U * th) / dt)
        k, dx = 2 * math.pi, 1.0 / sizes[-1]
        rec = {"sigma_times_N^(alpha-1)": [s_ * n ** (alpha - 1) for s_, n in zip(sig, sizes)],
               "alpha": alpha,
               "fitted_exponent": float(np.polyfit(np.log(sizes), np.log(sig), 1)[0]),
               "decay_coeff_over_table1": sig[-1] / (k ** alpha * dx ** (alpha - 1)) / c_dec(U)}
        if name in TABLE1_DRIFT:
            rec["drift_coeff_over_table1"] = drift[-1] / (k ** 3 * dx ** 2) / TABLE1_DRIFT[name](U)
        else:
            rec["drift_over_decay"] = drift[-1] / sig[-1]
        out[name] = rec
    return out


def shear_measurement(torch, sl, stream, sizes=(128, 256, 512)):
    """The 2D patch test of Sec. 5 (compact divergence-free shear, CFL 0.5, to
    t = 64, FP64), every scheme, against the initial field carried along exact
    trajectories: L1 error of the discontinuous square patch, relative L2 error
    of a smooth Gaussian in its place and the orders between sizes, and the
    time per step at the largest size."""
    from paper_1606_06117_gb300 import workloads as W
    out = {"sizes": list(sizes), "T": W.SHEAR_T, "cfl": 0.5, "dtype": "f64"}
    exact = {}
    for n in sizes:
        for kind, f in (("patch", W.patch_indicator()), ("bump", W.bump())):
            exact[(n, kind)] = W.shear_exact((n, n), f, device="cuda")
    for name in ("CIR", "FEC", "BEC", "CEC"):
        code = getattr(sl, name)
        rec = {"patch_l1": [], "bump_rel_l2": []}
        for n in sizes:
            vel = W.shear_patch_velocity((n, n), device="cuda")
            dt, nsteps = W.dt_for_cfl(W.SHEAR_T, vel.abs().max().item() * n, 0.5)
            for kind, f in (("patch", W.patch_indicator()), ("bump", W.bump())):
                x = W.on_grid((n, n), f, device="cuda")
                y = torch.empty_like(x)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for k in range(nsteps):
                    sl.sl_advect(y, x, vel, 2, [n, n, 1], [1.0 / n, 1.0 / n, 1.0], dt, code, sl.F64, k & 1, stream)
                    x, y = y, x
                torch.cuda.synchronize()
                el = time.perf_counter() - t0
                ex = exact[(n, kind)]
                if kind == "patch":
                    rec["patch_l1"].append((x - ex).abs().mean().item())
                else:
                    rec["bump_rel_l2"].append((torch.linalg.vector_norm(x - ex) / torch.linalg.vector_norm(ex)).item())
            rec["steps"] = nsteps
            rec["us_per_step"] = el / nsteps * 1e6
        e = rec["bump_rel_l2"]
        rec["bump_orders"] = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        out[name] = rec
    return out


# Algorithmic bytes per cell of one FP32 wide CEC step whose lines fit the
# fused sweep (k_wide_sweep): per axis, read Phi and u_d, write the result.
WIDE_CEC_BYTES_PER_CELL = 3 * 12


def large_cfl_measurement(torch, sl, stream, n=256, cfl=3.75, timed=20):
    """Steps at a large Courant number (Sec. 4, eq. intro:CECcoefSL): the 256^3
    ABC / 32-mode workload advanced by the non-local CEC step (sl_advect_wide)
    at CFL 3.75 over the physical time of 100 local CEC steps at CFL 0.8.
    Reports the time per step, the rate and its HBM roofline (36 B per cell:
    three fused line sweeps), and the round trip (forward, then back with -dt) against the
    local step's 100 + 100 steps: relative L2 error and wall time for the same
    physical time."""
    phi, vel, sp, dt0 = workload(n, "cuda", torch)
    dims = [n, n, n]
    T = 100 * dt0
    nsteps = int(math.ceil(T * 2.0 / sp[0] / cfl - 1e-12))     # max |u_d| = 2
    dt = T / nsteps
    need = sl.sl_advect_wide_workspace(3, dims, sl.CEC, sl.F32)
    ws_t = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    ws = ws_t.data_ptr() + (-ws_t.data_ptr()) % 256
    a, b = phi.clone(), torch.empty_like(phi)

    def fn(k):
        sl.sl_advect_wide(b, a, vel, 3, dims, sp, dt, sl.CEC, sl.F32, k & 1, ws, need, stream)
    fn(0)
    fn(1)
    ms = time_steps(torch, stream, fn, timed)
    peak, kind = measured_hbm_peak()
    gbs = WIDE_CEC_BYTES_PER_CELL * n ** 3 / (ms * 1e-3) / 1e9

    def round_trip(step, count, h):
        x, y = phi.clone(), torch.empty_like(phi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(2 * count):
            step(y, x, h if k < count else -h, k)
            x, y = y, x
        torch.cuda.synchronize()
        return sl.sl_norms(x, phi, phi.numel(), sl.F32, stream)[2], time.perf_counter() - t0

    wide_err, wide_s = round_trip(
        lambda y, x, h, k: sl.sl_advect_wide(y, x, vel, 3, dims, sp, h, sl.CEC, sl.F32, k & 1, ws, need, stream),
        nsteps, dt)
    local_err, local_s = round_trip(
        lambda y, x, h, k: sl.sl_advect(y, x, vel, 3, dims, sp, h, sl.CEC, sl.F32, k & 1, stream), 100, dt0)
    unsplit = {}
    for name in ("CIR", "FEC", "BEC"):          # non-local operator compositions, unfused gathers
        code = getattr(sl, name)
        need_u = sl.sl_advect_wide_workspace(3, dims, code, sl.F32)

        def fu(k, code=code, need_u=need_u):
            sl.sl_advect_wide(b, a, vel, 3, dims, sp, dt, code, sl.F32, k & 1, ws, need_u, stream)
        fu(0)
        msu = time_steps(torch, stream, fu, timed)
        unsplit[name] = {"ms_per_step": msu, "gcell_s": n ** 3 / (msu * 1e-3) / 1e9}
    sl.sl_device_status(stream)
    return {"grid": dims, "cfl": dt * 2.0 / sp[0], "steps_for_T": nsteps, "ms_per_step": ms, "unsplit": unsplit,
            "gcell_s": n ** 3 / (ms * 1e-3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_kind": kind, "bytes_per_cell": WIDE_CEC_BYTES_PER_CELL},
            "roundtrip_rel_l2": wide_err, "roundtrip_seconds": wide_s,
            "local_cfl_0.8": {"steps_for_T": 100, "roundtrip_rel_l2": local_err, "roundtrip_seconds": local_s}}


def cec_size_measurement(torch, sl, stream, n, timed=40):
    """One scalar field, the split CEC step on the n^3 ABC / 32-mode workload
    (the headline's flow at another size): rate, per-step time and the
    roofline fraction of the fused kernels (20 B per cell-update)."""
    phi, vel, sp, dt = workload(n, "cuda", torch)
    a, b = phi, torch.empty_like(phi)

    def fn(k):
        sl.sl_advect(b, a, vel, 3, [n] * 3, sp, dt, sl.CEC, sl.F32, k & 1, stream)
    fn(0)
    fn(1)
    ms = time_steps(torch, stream, fn, timed)
    peak, kind = measured_hbm_peak()
    gbs = BYTES_PER_CELL * n ** 3 / (ms * 1e-3) / 1e9
    return {"grid": [n] * 3, "gcell_s": n ** 3 / (ms * 1e-3) / 1e9, "ms_per_step": ms,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_kind": kind}}


def deformation_measurement(torch, sl, stream, n=512, total_steps=2000, timed=20):
    """Time-reversing deformation flow on [0,1)^3 at n^3: the three velocity
    components of u(t=0) and a random-mode scalar advected with the CEC step,
    u scaled by cos(pi t / T) over T = total_steps steps (CFL 0.8 at t = 0), so
    that every field returns to its initial value at t = T.  Reports
    field-cell-updates per second of sl_advect_multi and the relative L2 error
    of each field at t = T."""
    from paper_1606_06117_gb300 import workloads as W
    shape = (n, n, n)
    vel = W.deformation_velocity(shape, device="cuda", dtype=torch.float32)
    scal = W.random_modes(shape, W.draw_modes(3, 32, 8, seed=5), length=1.0, device="cuda", dtype=torch.float32)
    f0 = [vel[0].clone(), vel[1].clone(), vel[2].clone(), scal]
    sp = [1.0 / n] * 3
    umax = float(vel.abs().amax())
    dt = 0.8 * sp[0] / umax
    T = total_steps * dt
    cur = [f.clone() for f in f0]
    nxt = [torch.empty_like(f) for f in f0]

    def step(k):
        scale = math.cos(math.pi * (k + 0.5) * dt / T)
        sl.sl_advect_multi(nxt, cur, vel, 3, [n, n, n], sp, dt * scale, sl.CEC, sl.F32, k & 1, stream)
        cur[:], nxt[:] = nxt[:], cur[:]
    for k in range(2):
        step(k)
    torch.cuda.synchronize()
    ms = time_steps(torch, stream, lambda k: step(2 + k), timed)

    def plain(k):   # the same step as four single-field calls (bitwise the same result)
        scale = math.cos(math.pi * (k + 0.5) * dt / T)
        for i in range(4):
            sl.sl_advect(nxt[i], cur[i], vel, 3, [n, n, n], sp, dt * scale, sl.CEC, sl.F32, k & 1, stream)
        cur[:], nxt[:] = nxt[:], cur[:]
    ms_plain = time_steps(torch, stream, lambda k: plain(2 + timed + k), timed)
    # accuracy: the full forward-and-back run from the initial fields
    cur[:] = [f.clone() for f in f0]
    for k in range(total_steps):
        step(k)
    torch.cuda.synchronize()
    errs = [sl.sl_norms(c, f, f.numel(), sl.F32, stream)[2] for c, f in zip(cur, f0)]
    return {"grid": [n, n, n], "fields": 4, "steps_T": total_steps,
            "field_gcell_s": 4 * n ** 3 / (ms * 1e-3) / 1e9, "ms_per_step": ms,
            "plain_field_gcell_s": 4 * n ** 3 / (ms_plain * 1e-3) / 1e9, "plain_ms_per_step": ms_plain,
            "rel_l2_at_T": {"u": errs[0], "v": errs[1], "w": errs[2], "scalar": errs[3]}}


def rb_measurement(torch, sl, stream, n=50, Ra=1e5, dt=2e-5, steps=1000, cpu=True):
    """The Sec. 6 run: Rayleigh-Benard box 2 x 1 on n x n cells, Pr = 1, the
    +-0.1 spots near the lower left corner, U = 0, FP64, every scheme for
    `steps` steps (the rising plume reaches the top after about a thousand).
    Reports the time per step of sl_rb_step over the whole run, the first step
    (to 10) at which theta > 0.02 reaches the top three rows, and the state's
    extrema, total variation of theta and mean kinetic energy at the end (CIR
    diffuses the plume: lower extrema and energy)."""
    from paper_1606_06117_gb300 import workloads as W
    th0 = torch.from_numpy(W.rb_spots(n, n)).cuda()
    z0 = torch.zeros_like(th0)
    out = {"grid": [n, n], "box": [2.0, 1.0], "Ra": Ra, "Pr": 1.0, "dt": dt, "steps": steps, "dtype": "f64"}
    for name in ("CIR", "FEC", "BEC", "CEC"):
        box = sl.RayleighBenard(n, n, Ra=Ra, scheme=name)
        try:
            box.set_state(z0, z0, th0)
            box.step(dt, 16)   # warm-up (captures the replayed graph)
            box.set_state(z0, z0, th0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            box.step(dt, steps)
            torch.cuda.synchronize()
            us = (time.perf_counter() - t0) / steps * 1e6
            box.set_state(z0, z0, th0)
            reach = None
            for k in range(0, steps, 10):
                box.step(dt, 10)
                if reach is None and bool((box.state()[2][-3:] > 0.02).any()):
                    reach = k + 10
            u, w, th = box.state()
            tv = float((th[1:] - th[:-1]).abs().sum() + (th[:, 1:] - th[:, :-1]).abs().sum())
            out[name] = {"us_per_step": us, "top_reached_at_step": reach, "theta_max": float(th.max()),
                         "theta_min": float(th.min()), "theta_tv": tv,
                         "kinetic_energy": float(0.5 * (u * u + w * w).mean())}
        finally:
            box.close()
    out["device_status"] = sl.sl_device_status()
    if cpu:
        out["cpu_baseline"] = rb_oracle_rate(n, Ra, dt)
    return out


def main():
    args = parse()
    if args.profile_rb:
        import torch
        from paper_1606_06117_gb300 import _lib as sl
        sl.load()
        print(json.dumps(rb_measurement(torch, sl, None, steps=args.rb_steps, cpu=False)), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

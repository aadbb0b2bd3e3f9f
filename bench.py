#!/usr/bin/env python
"""Throughput of the GRRMHD+M1 time step on one GB300: zone-cycles per second.

Workload: the seeded Kerr-Schild torus (a = 0.9375, r in [1.2, 50],
256 x 128 x 64 zones, PPM + LAXF, flux-CT, PMHD/URAD implicit solve), FP64 or
split precision.  A zone-cycle is one active zone advanced one full RK3 step,
including the CFL time step, the three sub-steps, retries and back-ups.  The
state is resident in HBM; its working set (primitives, fluxes, scratch) is far
larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|split]
                  [--impl harmrad|reference]

Prints one JSON line.  The reference arm times the FP64 CPU oracle (the plain
restatement of the method used by the tests) on the host cores.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GRRMHD+M1 zone-cycles/s at 256x128x64 (FP64 vs split); frac of HBM roofline"
UNIT = "zone-cycles/s"
# FP64 peak of a GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA per
# clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s (the nominal 1.25 TFLOP/s).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
PROFILE_JSON = os.path.join(ROOT, "profiles", "k_update_counters.json")
INTEGRATORS = {"rk3": 0, "imex2": 1, "imex2b": 2, "imex3": 3}
KERNEL_SOURCES = ["hr_phys.cuh", "hr_implicit.cuh", "hr_kernels.cuh"]


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1312_6127_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_time_ms(ms_local, dist, device):
    """The job's timed-region length: the maximum over ranks of each rank's
    milliseconds (every rank receives it); ms_local itself on one process."""
    if dist is None:
        return ms_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, steps, ws, ms):
    """Whole-job zone-cycles/s: the units all ranks advanced (each rank runs
    its own replica of the workload) over the max-over-ranks time."""
    return units_per_rank * steps * ws / (ms / 1e3)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class OracleRun:
    """The FP64 CPU oracle (as it stands) on the same seeded torus, with its
    zone and face loops on `threads` host threads (the result does not depend
    on the thread count)."""

    def __init__(self, n, threads, integrator=0):
        os.environ["ORACLE_THREADS"] = str(threads)
        from oracle import oracle as O
        from paper_1312_6127_gb300 import workloads as W
        cfg, P = W.torus(n, seed=12345)
        cfg["integrator"] = integrator
        self.o = O.Oracle(cfg)
        self.o.set_prims(P)
        self.zones = n[0] * n[1] * n[2]
        self.threads = threads

    def step(self):
        """One CFL step; returns (zone-cycles/s, seconds)."""
        t0 = time.perf_counter()
        self.o.step(0.0)
        dt = time.perf_counter() - t0
        return self.zones / dt, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    n = tuple(int(x) for x in args.size.split(","))
    cores = os.cpu_count() or 1
    run = OracleRun(n, cores, INTEGRATORS[args.integrator])
    for _ in range(args.warmup):
        run.step()
    t_all = 0.0
    for _ in range(args.steps):
        t_all += run.step()[1]
    value = run.zones * args.steps / t_all
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "KS torus a=0.9375 %dx%dx%d (PPM, LAXF, flux-CT, PMHD/URAD)" % n,
                   "precision": "fp64", "integrator": args.integrator, "zones": run.zones},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "each step: one CFL step of the whole %dx%dx%d torus, FP64 oracle "
                                   "with its zone and face loops on %d host threads" % (n + (cores,))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="harmrad", choices=["harmrad", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "split"])
    ap.add_argument("--size", default="256,128,64")
    ap.add_argument("--workload", default="torus", choices=["torus", "batch48"],
                    help="torus: the Kerr-Schild torus (default); batch48: 48 uneven Minkowski "
                         "boxes with a per-zone absorption field in one batched context")
    ap.add_argument("--integrator", default="rk3", choices=list(INTEGRATORS),
                    help="time integrator (Sec. 4.1): the paper's RK3 or one of its IMEX schemes")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    from paper_1312_6127_gb300 import harmrad as H
    from paper_1312_6127_gb300 import workloads as W

    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = tuple(int(x) for x in args.size.split(","))
    prec = H.PREC_SPLIT if args.precision == "split" else H.PREC_FP64
    stream = torch.cuda.current_stream()
    integ = INTEGRATORS[args.integrator]
    if args.workload == "torus":
        cfg, P = W.torus(n, seed=12345 + rank)
        cfg["integrator"] = integ
        nact = n[0] * n[1] * n[2]
        g = H.Grid(cfg, precision=prec, stream=stream)
        g.set_prims(P)
        wl = "KS torus a=0.9375 %dx%dx%d (PPM, LAXF, flux-CT, PMHD/URAD)" % n
        size_key, prof_key = list(n), args.precision
    else:
        cfgs, Ps, Ks = W.box_batch(seed=4242 + rank)
        cfgs = [dict(c, integrator=integ) for c in cfgs]
        g = H.Batch(cfgs, precision=prec, stream=stream)
        g.set_prims(Ps)
        g.set_opacity_field(Ks)
        nact = g.nact
        del Ps, Ks
        wl = ("48 periodic Minkowski boxes, edges log-uniform 32..128 (%d zones), per-zone "
              "absorption with optical depth per cell log-uniform 1e-4..1e6, one batched context"
              % nact)
        size_key, prof_key = "batch48", "batch48_" + args.precision
    tuning = g.tuning() if args.no_autotune else g.autotune(reps=1)
    for _ in range(args.warmup):
        g.step(0.0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        g.step(0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = job_time_ms(ms, dist, "cuda")
    st = g.stats()
    value = job_throughput(nact, args.steps, ws, ms)

    # per-kernel device times of one eager step (events on the launching stream)
    roofline = None
    kt = None
    if not args.no_profile:
        kt = g.profile_step(0.0)
        upd_ms, upd_n = kt["update"]
        avg_ms = upd_ms / max(upd_n, 1)
        prof = {}
        try:
            with open(PROFILE_JSON) as fh:
                prof = json.load(fh)
        except (OSError, ValueError):
            prof = {}
        entry = prof.get(prof_key, {})
        # the counters are those of the RK3 update kernel
        fresh = (entry.get("kernel_hash") == kernel_hash() and entry.get("size") == size_key
                 and integ == 0)
        flops_per_zone = entry.get("fp64_flops_per_zone_stage")
        traffic = entry.get("dram_bytes_per_launch") if fresh else None
        if flops_per_zone and fresh:
            achieved = flops_per_zone * nact / (avg_ms / 1e3) / 1e12
            roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS / 1e3,
                        "unit": "TFLOP/s", "frac": achieved / (FP64_PEAK_GFLOPS / 1e3),
                        "traffic": traffic, "kernel": "k_update (update + PMHD Newton)",
                        "kernel_ms": avg_ms, "counters_fresh": fresh,
                        "fp64_pipe_active_pct": entry.get("fp64_pipe_active_pct"),
                        "peak_note": "FP64 from unit counts: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz; "
                                     "achieved counts DFMA/DMUL/DADD only"}
        else:
            roofline = {"bound": "alu", "achieved": None, "peak": FP64_PEAK_GFLOPS / 1e3,
                        "unit": "TFLOP/s", "frac": None, "traffic": traffic,
                        "kernel": "k_update", "kernel_ms": avg_ms,
                        "note": "FP64 op count per zone not captured for this kernel build "
                                "(profiles/k_update_counters.json kernel_hash differs)" if integ == 0 else
                                "FP64 op counts are captured for the RK3 update kernel only"}
        # HBM view of the whole step: algorithmic bytes per zone-cycle
        hbm = measured_peaks().get("hbm_gbs")
        step_ms = ms / args.steps
        alg_bytes = 960.0 * nact
        roofline["step_hbm"] = {"algorithmic_bytes_per_zone_cycle": 960, "achieved_gbs":
                                alg_bytes / (step_ms / 1e3) / 1e9, "peak_gbs": hbm,
                                "frac": (alg_bytes / (step_ms / 1e3) / 1e9) / hbm if hbm else None}

    # end to end through the C ABI with host buffers: H2D + step + D2H per step
    e2e = None
    if not args.no_e2e:
        size = 12 * nact
        pin_in = torch.empty(size, dtype=torch.float64, pin_memory=True).numpy()
        pin_out = torch.empty(size, dtype=torch.float64, pin_memory=True).numpy()
        pin_in[:] = g.get_prims(device=True).reshape(-1).cpu().numpy()
        g.step_host(pin_in, pin_out, 0.0)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(args.steps):
            src, dst = (pin_out, pin_in) if s % 2 else (pin_in, pin_out)
            g.step_host(src, dst, 0.0)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        nbytes = size * 8
        e2e = {"value": nact * args.steps * ws / te, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu and args.workload == "torus":
        cores = os.cpu_count() or 1
        run = OracleRun(n, cores, integ)
        v, t = run.step()
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "one CFL step of the same seeded %dx%dx%d torus, FP64 oracle with its zone "
                         "and face loops on %d host threads, %.1f s" % (n + (cores, t))}
        del run

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == H.PREC_FP64 else "f64+f32",
            "data": "synthetic",
            "config": {"workload": wl,
                       "precision": args.precision, "integrator": args.integrator, "zones": nact,
                       "l2": "working set > L2 (129 MB); no flush needed",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "launch_shapes": {k: v for k, v in tuning.items() if not k.endswith("_ms")},
                       "autotuned": not args.no_autotune},
            "gpu_launches": st["kernel_launches"] * args.steps,
            "clocks": clk,
            "solver": {"newton_iters_per_solve": st["newton_iters"] / max(st["zone_stages"], 1),
                       "pmhd": st["pmhd_ok"], "urad": st["urad_ok"], "backup": st["backup"],
                       "dt": st["dt"]},
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        if kt:
            line["kernel_ms"] = {k: round(v[0], 4) for k, v in kt.items()}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

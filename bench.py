#!/usr/bin/env python
"""Throughput of the GRRMHD+M1 time step on one GB300: zone-cycles per second.

Workload: the seeded Kerr-Schild torus (a = 0.9375, r in [1.2, 50],
256 x 128 x 64 zones, PPM + LAXF, flux-CT, PMHD/URAD implicit solve), FP64 or
split precision.  A zone-cycle is one active zone advanced one full RK3 step,
including the CFL time step, the three sub-steps, retries and back-ups.  The
state is resident in HBM; its working set (primitives, fluxes, scratch) is far
larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|split]
                  [--workload torus|torus_uct|batch48] [--impl harmrad|reference]

Prints one JSON line.  The default run (FP64 torus, one GPU) also times split
precision on the same torus ("split", with its conserved totals against FP64),
the batch of 48 uneven boxes ("batch48") and the torus with the staggered
field and 4-state EMF ("uct"), each with its own clocks and roofline.  The
reference arm times the FP64 CPU oracle (the plain restatement of the method
used by the tests) on the host cores.
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
# clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s (the nominal 1.25 TFLOP/s); the
# roofline divides by the rate measured live, this figure is reported beside it.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
PROFILE_JSON = os.path.join(ROOT, "profiles", "k_update_counters.json")
INTEGRATORS = {"rk3": 0, "imex2": 1, "imex2b": 2, "imex3": 3}
KERNEL_SOURCES = ["hr_phys.cuh", "hr_implicit.cuh", "hr_tangent.cuh", "hr_kernels.cuh"]


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


def fp64_peak(H):
    """FP64 peak for the roofline: the device's FMA rate measured live by the
    library's FMA-chain kernel (harmrad_fp64_fma_rate), best of 5 launches."""
    try:
        return H.fp64_fma_rate(5), "measured: harmrad_fp64_fma_rate (independent DFMA chains, best of 5)"
    except Exception as ex:  # the derived figure is reported instead, and said so
        return FP64_PEAK_GFLOPS / 1e3, "derived from unit counts (probe failed: %s)" % ex


def make_context(args, H, W, workload, prec, stream, rank, integ):
    """The workload's context with its state loaded: (grid, active zones,
    workload text, counters key)."""
    n = tuple(int(x) for x in args.size.split(","))
    pname = "split" if prec == H.PREC_SPLIT else "fp64"
    if workload in ("torus", "torus_uct"):
        cfg, P, Bf = W.torus(n, seed=12345 + rank, faces=True)
        cfg["integrator"] = integ
        uct = workload == "torus_uct"
        cfg["emf"] = H.EMF_UCT if uct else H.EMF_FLUXCT
        g = H.Grid(cfg, precision=prec, stream=stream)
        g.set_prims(P)
        if uct:
            g.set_face_fields(Bf)
        g.cfg_init, g.P_init = cfg, P
        wl = "KS torus a=0.9375 %dx%dx%d (PPM, LAXF, %s, PMHD/URAD)" % (n + ("staggered B, 4-state EMF" if uct
                                                                             else "flux-CT",))
        return g, n[0] * n[1] * n[2], wl, (list(n), pname + ("_uct" if uct else ""))
    cfgs, Ps, Ks = W.box_batch(seed=4242 + rank)
    cfgs = [dict(c, integrator=integ) for c in cfgs]
    g = H.Batch(cfgs, precision=prec, stream=stream)
    g.set_prims(Ps)
    g.set_opacity_field(Ks)
    wl = ("48 periodic Minkowski boxes, edges log-uniform 32..128 (%d zones), per-zone "
          "absorption with optical depth per cell log-uniform 1e-4..1e6, one batched context" % g.nact)
    return g, g.nact, wl, ("batch48", "batch48_" + pname)


def time_steps(g, args, stream, dist, local):
    """W warm-up steps, then K timed CUDA-graph steps bracketed by a barrier
    and a synchronize; clocks sampled during the timed region."""
    import torch
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
    return ms, clocks.stop()


SUBSTEPS = {0: 3, 1: 3, 2: 4, 3: 5}  # sub-steps of a step per integrator


def kernel_roofline(g, nact, key, integ, peak_tf, peak_note, ms, steps):
    """Roofline of the dominant kernel (the update kernel: update, geometric
    source and PMHD Newton, with its Newton continuation kernel when the
    launch shapes split the Newton iteration) from one eager step timed per
    kernel with CUDA events on the context's stream, per sub-step, and the
    HBM view of the whole step."""
    kt = g.profile_step(0.0)
    upd_ms, upd_n = kt["update"]
    avg_ms = upd_ms / SUBSTEPS.get(integ, 3)
    try:
        with open(PROFILE_JSON) as fh:
            prof = json.load(fh)
    except (OSError, ValueError):
        prof = {}
    size_key, prof_key = key
    entry = prof.get(prof_key, {})
    # the counters are those of the RK3 update kernel of this build
    fresh = (entry.get("kernel_hash") == kernel_hash() and entry.get("size") == size_key and integ == 0)
    flops_per_zone = entry.get("fp64_flops_per_zone_stage")
    traffic = entry.get("dram_bytes_per_launch") if fresh else None
    derived = FP64_PEAK_GFLOPS / 1e3
    roof = {"bound": "alu", "achieved": None, "peak": peak_tf, "unit": "TFLOP/s", "frac": None,
            "traffic": traffic, "kernel": "k_update (update + geometric source + PMHD Newton)",
            "kernel_ms": avg_ms, "kernel_ms_note": "per sub-step: k_update and, with a Newton split, "
                                                    "k_newton_cont (%d launches in the profiled step)" % upd_n,
            "kernel_share": upd_ms / max(sum(v[0] for v in kt.values()), 1e-30),
            "counters_fresh": fresh, "peak_note": peak_note,
            "peak_derived": derived}
    if flops_per_zone and fresh:
        achieved = flops_per_zone * nact / (avg_ms / 1e3) / 1e12
        roof.update(achieved=achieved, frac=achieved / peak_tf, frac_of_derived=achieved / derived,
                    fp64_flops_per_zone_stage=flops_per_zone,
                    fp64_pipe_active_pct=entry.get("fp64_pipe_active_pct"),
                    counters_captured_size=entry.get("captured_size"),
                    achieved_note="(2 DFMA + DMUL + DADD) thread instructions per zone-stage from ncu x "
                                  "zones / CUDA-event launch time")
    else:
        roof["note"] = ("FP64 op counts of this kernel build are not in profiles/k_update_counters.json"
                        if integ == 0 else "FP64 op counts are captured for the RK3 update kernel only")
    hbm = measured_peaks().get("hbm_gbs")
    step_ms = ms / steps
    gbs = 960.0 * nact / (step_ms / 1e3) / 1e9
    roof["step_hbm"] = {"algorithmic_bytes_per_zone_cycle": 960, "achieved_gbs": gbs, "peak_gbs": hbm,
                        "frac": gbs / hbm if hbm else None}
    return roof, kt


def conserved_totals(H, cfg, Pd):
    """Mass, total energy and total momenta (gas + radiation) of a state,
    with the absolute sums they are measured against (point-wise physics
    entry of the library)."""
    import torch
    n1, n2, n3 = cfg["n"]
    kk, jj, ii = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    x = np.zeros((n3 * n2 * n1, 4))
    x[:, 1] = cfg["x0"][0] + (ii.ravel() + 0.5) * cfg["dx"][0]
    x[:, 2] = cfg["x0"][1] + (jj.ravel() + 0.5) * cfg["dx"][1]
    x[:, 3] = cfg["x0"][2] + (kk.ravel() + 0.5) * cfg["dx"][2]
    U = H.zone_physics(cfg, x, Pd.reshape(12, -1).T.cpu().numpy())[0]
    tot, ab = U.sum(axis=0), np.abs(U).sum(axis=0)
    pick = lambda t: np.array([t[0], t[1] + t[8], t[2] + t[9], t[3] + t[10], t[4] + t[11]])
    return pick(tot), pick(ab)


def split_total_errors(H, g64, g32, steps):
    """Both precisions from the same initial state with the FP64 run's CFL
    steps: each conserved total of split precision against FP64, relative to
    the total's absolute sum (outside any timed region)."""
    cfg, P = g64.cfg_init, g64.P_init
    g64.set_prims(P)
    g32.set_prims(P)
    dts = []
    for _ in range(steps):
        g64.step(0.0)
        dts.append(g64.stats()["dt"])
    for dt in dts:
        g32.step(dt)
    t64, s64 = conserved_totals(H, cfg, g64.get_prims(device=True))
    t32, _ = conserved_totals(H, cfg, g32.get_prims(device=True))
    rel = np.abs(t32 - t64) / s64
    return {"steps": steps, "quantities": ["mass", "energy", "momentum_1", "momentum_2", "momentum_3"],
            "rel_to_abs_sum": [float(v) for v in rel], "max": float(rel.max())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="harmrad", choices=["harmrad", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "split"])
    ap.add_argument("--size", default="256,128,64")
    ap.add_argument("--workload", default="torus", choices=["torus", "torus_uct", "batch48"],
                    help="torus: the Kerr-Schild torus (default, flux-CT); torus_uct: the same torus with "
                         "the staggered field and 4-state EMF; batch48: 48 uneven Minkowski boxes with a "
                         "per-zone absorption field in one batched context")
    ap.add_argument("--integrator", default="rk3", choices=list(INTEGRATORS),
                    help="time integrator (Sec. 4.1): the paper's RK3 or one of its IMEX schemes")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the split-precision, batch48 and staggered-field sub-measurements of the "
                         "default run")
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
    peak_tf, peak_note = fp64_peak(H)
    g, nact, wl, key = make_context(args, H, W, args.workload, prec, stream, rank, integ)
    tuning = g.tuning() if args.no_autotune else g.autotune(reps=1)
    ms, clk = time_steps(g, args, stream, dist, local)
    ms = job_time_ms(ms, dist, "cuda")
    st = g.stats()
    value = job_throughput(nact, args.steps, ws, ms)

    roofline, kt = None, None
    if not args.no_profile:
        roofline, kt = kernel_roofline(g, nact, key, integ, peak_tf, peak_note, ms, args.steps)

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

    # the default run also measures split precision on the same torus, the
    # batch of 48 boxes and the torus with the staggered field (same steps and
    # warm-up, each timed on its own)
    extras = {}
    default_run = (args.workload == "torus" and prec == H.PREC_FP64 and integ == 0 and ws == 1)
    if default_run and not args.no_extras:
        for name, wk, pr in (("split", "torus", H.PREC_SPLIT), ("batch48", "batch48", H.PREC_FP64),
                             ("uct", "torus_uct", H.PREC_FP64)):
            gx, nx, wlx, keyx = make_context(args, H, W, wk, pr, stream, rank, integ)
            tx = gx.tuning() if args.no_autotune else gx.autotune(reps=1)
            msx, clkx = time_steps(gx, args, stream, None, local)
            stx = gx.stats()
            sub = {"value": job_throughput(nx, args.steps, 1, msx), "unit": UNIT,
                   "ms_per_step": msx / args.steps, "workload": wlx, "zones": nx,
                   "dtype": "f64+f32" if pr == H.PREC_SPLIT else "f64", "clocks": clkx,
                   "launch_shapes": {k: v for k, v in tx.items() if not k.endswith("_ms")},
                   "solver": {"newton_iters_per_solve": stx["newton_iters"] / max(stx["zone_stages"], 1),
                              "pmhd": stx["pmhd_ok"], "urad": stx["urad_ok"], "backup": stx["backup"]}}
            if not args.no_profile:
                sub["roofline"], ktx = kernel_roofline(gx, nx, keyx, integ, peak_tf, peak_note, msx,
                                                       args.steps)
                sub["kernel_ms"] = {k: round(v[0], 4) for k, v in ktx.items()}
            if name in ("split", "uct"):
                sub["vs_fp64"] = value and sub["value"] / value
            if name == "split":
                sub["conserved_totals_vs_fp64"] = split_total_errors(H, g, gx, args.steps)
            extras[name] = sub
            del gx
            torch.cuda.empty_cache()

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
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python3
"""Throughput of the GB300 suspension stepper in particle-steps/s.

Workload: 1,000,000 bidisperse spheres (radii 1 and 1.4, equal numbers),
volume fraction 0.58, Pe = 1000, friction coefficient 1 (k_t = k_n / 2),
k_n = 1e4, dt = 1e-4, skin 0.3, mixed precision (single-precision pair
arithmetic on gaps formed from double positions; double integration, history
and stress).  One bench step = one library call advancing `--inner`
timesteps (kick/drift/wrap, neighbour rebuilds when due, pair forces, stress
reduction), so every row of the hot path runs inside the timed region.

value: N * inner * steps / (device time of the timed steps), inputs resident
in HBM; e2e: the same metric through the public API with the state uploaded
from pinned host memory and the stress read back every step.  The roofline
entry covers the kernel family that takes most device time, timed with CUDA
events on the library's stream in a profiling pass right after the timed
steps.  Under torchrun each rank steps its own independent system (weak
scaling, no collective on the data path); rank 0 prints one JSON line.

--impl reference times the plain FP64 CPU oracle on a bounded sample of the
same workload instead (rank 0 only).
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "bidisperse-1M-phi0.58-pe1000-mu1"
SMS_GB300 = 152          # streaming multiprocessors of one GB300
SM_MAX_MHZ = 2070.0      # its maximum SM clock
METRIC = "particle-steps/s"

# DRAM traffic per launch of the dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), recorded per sphere together
# with the hash of the source it was taken on; reported only while the
# source is unchanged.
NCU_TRAFFIC = {
    # ncu --set full on the 1M bench workload: DRAM read + write per launch / N
    # issue_active: fraction of cycles the kernel issued an instruction (the
    # pair kernel is bound by issue and latency, not by DRAM)
    "k_pair_mixed": {"bytes_per_sphere": 332.638, "source_sha": "0bb6c694e2217c8a",
                     "issue_active": 0.763, "dram_throughput": 0.234,
                     "warp_instructions_per_sphere": 162.724},
    "k_integrate_mixed": {"bytes_per_sphere": 251.151, "source_sha": "dc951ff6aadb9bdb"},
}

# Double-precision floating-point operations per launch of the FP64 pair
# kernel, per sphere, from one ncu capture on the 1M bench workload: 2 per
# DFMA plus 1 per DADD and DMUL (smsp__sass_thread_inst_executed_op_d{fma,add,
# mul}_pred_on.sum); reported only while the source is unchanged.
NCU_FP64_FLOPS = {
    # 497.7 M DADD + 1,190.9 M DFMA + 666.0 M DMUL thread instructions per launch
    "k_pair_fp64": {"flops_per_sphere": 3545.513, "source_sha": "bd935770d82aa949"},
}


def _src_hash(name: str) -> str:
    """Hash of a kernel's translation unit: the .cu file and every local
    header it includes, directly or not, in include order."""
    csrc = os.path.join(ROOT, "paper_2307_13802_gb300", "csrc")
    h, seen, todo = hashlib.sha256(), set(), [name]
    while todo:
        f = todo.pop(0)
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        with open(os.path.join(csrc, f), "rb") as fh:
            data = fh.read()
        h.update(data)
        todo += re.findall(r'^#include "([^"]+)"', data.decode(), flags=re.M)
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--inner", type=int, default=100,
                    help="timesteps advanced per bench step")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP64-path comparison line")
    ap.add_argument("--phases", action="store_true",
                    help="time the mixed pair kernel's template variants (noise, friction, "
                         "stress sampling, lubrication switched off one at a time) on the "
                         "bench workload and print one JSON line")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (FP64 10k, 256 replicas, 8M) and the "
                         "mixed-vs-FP64 accuracy run")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.tmp.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.tmp.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per sphere of each kernel family
# ---------------------------------------------------------------------------
def algorithmic_bytes(family: str, precision: str, K: float, c: float, fric: bool) -> float:
    """Bytes a launch must move per sphere for the method's work: every record
    read or written once, gathers of neighbours not counted again.  K =
    half-list slots per sphere, c = touching pairs with history per sphere.

    Pair kernel: FP64 128 + 4K + 48c (own x, U, Omega 72 + radius 4, row
    length 4 + list 4K, F and T written 48, history 48 per touching pair read
    and written); mixed 100 + 4K + 48c (three 16-byte single-precision
    mirrors instead of the FP64 records).  Integrator: FP64 196 (read x, U,
    Omega, F, T 120 + radius 4, write x, U, Omega 72), mixed 244 (plus three
    16-byte mirrors written)."""
    hist = 48.0 * c if fric else 0.0
    if family == "pair":
        if precision == "mixed":
            return 48.0 + 4.0 + 4.0 * K + 48.0 + hist
        return 76.0 + 4.0 + 4.0 * K + 48.0 + hist
    if family == "integrate":
        return 244.0 if precision == "mixed" else 196.0
    return 0.0


def rebuild_bytes(K: float, passes: int = 2) -> float:
    """Algorithmic bytes per sphere of one neighbour rebuild: read the
    position (24) and write the cell key (4) and permutation (4), `passes`
    counting-sort passes over 4-byte keys, permute the particle records once
    (read and write 150), write the list (4K)."""
    return 24.0 + 8.0 + 8.0 * passes + 150.0 + 4.0 * K


def layout_bytes(family: str, precision: str, K: float, c: float, fric: bool) -> float:
    """Bytes the library's own layout moves per sphere in a launch (what the
    DRAM traffic is compared with): the mixed path's double-float position
    records (32 B with the low words), the velocity + tag mirror and the high
    half of the spin record (16 B each), float4 force and torque accumulators
    (32 B), and the 64-bit contact mask (16 B read and written) beside the
    32-byte history records.  The integrator writes two mirrors (48 B)."""
    hist = (16.0 + 48.0 * c) if fric else 0.0
    if family == "pair":
        if precision == "mixed":
            return 64.0 + 4.0 + 4.0 * K + 32.0 + hist
        return 96.0 + 8.0 + 4.0 * K + 48.0 + hist
    if family == "integrate":
        if precision == "mixed":
            return 96.0 + 32.0 + 8.0 + 96.0 + 48.0 + 32.0
        return 96.0 + 48.0 + 96.0 + 48.0
    return 0.0


# ---------------------------------------------------------------------------
# multi-rank pieces (one process per GPU, replicas only)
# ---------------------------------------------------------------------------
def rank_seed(seed: int, rank: int) -> int:
    """Each rank steps an independent replica of the workload: its own
    dynamics seed, no data exchanged between ranks."""
    return seed + 7919 * rank


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (the job is done when every rank is)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, N: int, timesteps: int, ms_max: float) -> float:
    """Particle-steps per second of the whole job: all ranks' spheres times
    the timesteps each advanced, over the slowest rank's time."""
    return world * N * timesteps / (ms_max / 1e3)


def run_ours(args, rank, world, local_rank, dist):
    import numpy as np
    import torch

    import paper_2307_13802_gb300 as susp
    import workloads

    torch.cuda.set_device(local_rank)
    w = workloads.named(WORKLOAD)
    if world > 1:
        w.params["seed"] = rank_seed(w.params["seed"], rank)
    p = w.params
    N = w.N
    stream = torch.cuda.Stream()

    def make(precision):
        s = susp.System(w.radii, w.box, precision=precision, eta=p["eta"], rho=p["rho"],
                        kn=p["kn"], kt=p["kt"], mu=p["mu"], skin=p["skin"],
                        shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"], dt=p["dt"])
        s.set_stream(stream.cuda_stream)
        s.set_state(w.x, w.U, w.W)
        return s

    def step(s, n):
        s.step(n, p["shear_rate"], p["kT"], p["dt"], p["seed"])

    sysm = make(args.precision)
    for _ in range(args.warmup):
        step(sysm, args.inner)
    sysm.stress()
    info0 = sysm.info()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step(sysm, args.inner)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    clk = clocks.stop()
    info1 = sysm.info()
    if dist is not None:
        ms = max_over_ranks(ms, dist, "cuda")
        dist.barrier()
    sig = sysm.stress()
    value = job_value(world, N, args.inner * args.steps, ms)

    # where the time goes: per-family device time over one more bench step
    prof = sysm.profile(args.inner, p["dt"])
    info = sysm.info()
    ij, _ = sysm.history()
    K = info["npairs"] / N
    c = len(ij) / N
    fric = p["mu"] > 0
    fam = max(("integrate", "pair", "rebuild", "finalize", "reduce"),
              key=lambda f: prof[f]["ms"])
    hbm, peak_kind = peaks()
    per_sphere = algorithmic_bytes(fam, args.precision, K, c, fric)
    per_sphere_layout = layout_bytes(fam, args.precision, K, c, fric)
    roofline = None
    if per_sphere > 0 and prof[fam]["launches"] > 0:
        bytes_per_launch = per_sphere * N
        achieved = bytes_per_launch / (prof[fam]["ms_per_launch"] * 1e-3) / 1e9
        kernel = {"pair": "k_pair_mixed" if args.precision == "mixed" else "k_pair_fp64",
                  "integrate": "k_integrate_mixed" if args.precision == "mixed" else "k_integrate_fp64",
                  "finalize": "k_finalize"}.get(fam, fam)
        src = {("mixed", "pair"): "k_pair_mixed.cu", ("mixed", "integrate"): "k_mixed.cu",
               ("fp64", "pair"): "k_pair_fp64.cu"}.get((args.precision, fam),
                                                       "k_integrate_fp64.cu")
        rec = NCU_TRAFFIC.get(kernel)
        traffic = None
        ncu = None
        if rec and rec.get("source_sha") == _src_hash(src):
            traffic = rec["bytes_per_sphere"] * N
            ncu = {k: rec[k] for k in ("issue_active", "dram_throughput") if k in rec}
        roofline = {"bound": "hbm", "kernel": kernel, "achieved": round(achieved, 1),
                    "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": round(achieved / hbm, 4), "traffic": traffic,
                    "algorithmic_bytes_per_launch": bytes_per_launch,
                    "bytes_per_sphere": per_sphere,
                    "layout_bytes_per_sphere": round(per_sphere_layout, 3),
                    "ms_per_launch": prof[fam]["ms_per_launch"],
                    "half_list_slots_per_sphere": round(K, 3),
                    "contacts_per_sphere": round(c, 3)}
        if ncu:
            roofline["ncu"] = ncu
        if rec and rec.get("source_sha") == _src_hash(src) and "warp_instructions_per_sphere" in rec:
            # the instruction-issue roofline of the same launch: warp
            # instructions (ncu smsp__inst_executed.sum) over the event time,
            # against one warp instruction per cycle on each of the 4
            # schedulers of 152 SMs at the SM clock sampled in the timed region
            sm = SMS_GB300 * 4 * ((clk or {}).get("sm_mhz") or SM_MAX_MHZ) * 1e6
            inst = rec["warp_instructions_per_sphere"] * N
            got = inst / (prof[fam]["ms_per_launch"] * 1e-3)
            roofline["issue"] = {"warp_instructions_per_launch": inst,
                                 "achieved_ginst_per_s": round(got / 1e9, 1),
                                 "peak_ginst_per_s": round(sm / 1e9, 1),
                                 "frac": round(got / sm, 4)}
    rebuild_roof = None
    if prof["rebuild"]["launches"] > 0:
        rb = rebuild_bytes(K) * N
        ach = rb / (prof["rebuild"]["ms_per_launch"] * 1e-3) / 1e9
        rebuild_roof = {"bound": "hbm", "kernels": "cell keys, counting sort, permutation, "
                        "list, history carry-over, mirrors", "achieved": round(ach, 1),
                        "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
                        "bytes_per_sphere": round(rebuild_bytes(K), 3),
                        "ms_per_rebuild": round(prof["rebuild"]["ms_per_launch"], 4)}
    breakdown = {f: {"ms_per_launch": round(v["ms_per_launch"], 5),
                     "launches": v["launches"], "ms": round(v["ms"], 3)}
                 for f, v in prof.items()}

    # end to end: pinned host state in, stress out, every bench step
    x, U, Wv = sysm.state()
    pin = [torch.empty((N, 3), dtype=torch.float64, pin_memory=True) for _ in range(3)]
    for dst, src in zip(pin, (x, U, Wv)):
        dst.numpy()[:] = src
    hx, hU, hW = (t.numpy() for t in pin)
    e2e_steps = max(3, args.steps // 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sysm.set_state(hx, hU, hW)
        step(sysm, args.inner)
        st = sysm.stress()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = world * N * args.inner * e2e_steps / e2e_s
    assert math.isfinite(st["eta_r"])

    # the same workload with the stress sampled every 8th step (a divisor of
    # the 32-step graph chunk), reported beside the every-step headline
    sparse = None
    if not args.no_configs and world == 1:
        s8 = susp.System(w.radii, w.box, precision=args.precision, eta=p["eta"], rho=p["rho"],
                         kn=p["kn"], kt=p["kt"], mu=p["mu"], skin=p["skin"],
                         shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"], dt=p["dt"],
                         sample_every=8)
        s8.set_stream(stream.cuda_stream)
        s8.set_state(w.x, w.U, w.W)
        step(s8, args.inner)
        n8 = max(3, args.steps // 4)

        def run8():
            for _ in range(n8):
                step(s8, args.inner)
        ms8 = _timed(stream, run8)
        sparse = {"stress_sample_every": 8, "value": round(world * N * args.inner * n8 / (ms8 / 1e3), 1),
                  "ms_per_timestep": round(ms8 / (args.inner * n8), 4),
                  "samples": int(s8.stress()["samples"])}
        s8.close()

    fp64 = None
    if not args.no_fp64 and args.precision == "mixed":
        s64 = make("fp64")
        step(s64, 4)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n64 = 20
        e0.record(stream)
        step(s64, n64)
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        prof64 = s64.profile(2, p["dt"])
        fp64 = {"value": round(world * N * n64 / (ms64 / 1e3), 1),
                "ms_per_timestep": round(ms64 / n64, 4),
                "speedup_of_mixed": round(value / (world * N * n64 / (ms64 / 1e3)), 2),
                "pair_ms_per_launch": round(prof64["pair"]["ms_per_launch"], 4)}
        try:
            pk = susp.measure_peaks()
        except susp.SuspError:
            pk = None
        rec = NCU_FP64_FLOPS.get("k_pair_fp64")
        if pk and rec and rec.get("source_sha") == _src_hash("k_pair_fp64.cu"):
            fl = rec["flops_per_sphere"] * N
            ach = fl / (prof64["pair"]["ms_per_launch"] * 1e-3) / 1e9
            fp64["roofline"] = {"bound": "alu", "kernel": "k_pair_fp64", "unit": "GFLOP/s",
                                "achieved": round(ach, 1), "peak": round(pk["fp64_gflops"], 1),
                                "peak_kind": "measured FP64 multiply-add microbenchmark",
                                "frac": round(ach / pk["fp64_gflops"], 4),
                                "flops_per_launch": fl}
        elif pk:
            fp64["fp64_peak_gflops"] = round(pk["fp64_gflops"], 1)
        s64.close()

    legs = {}
    if not args.no_configs and world == 1:
        x0, U0, W0 = sysm.state()
        i0 = sysm.info()
        sysm.close()

        def leg(fn):
            # a library error in one extra workload is reported, not fatal
            try:
                return fn()
            except susp.SuspError as e:
                return {"error": str(e)}

        legs["mixed_vs_fp64"] = leg(lambda: mixed_vs_fp64(
            susp, w, x0, U0, W0, int(i0["k"]), float(i0["strain"]), stream))
        legs["configs"] = {
            "bidisperse-10k-phi0.56-pe10-mu1 (fp64)": leg(lambda: run_single(
                susp, workloads.named("bidisperse-10k-phi0.56"), "fp64", stream, 100, 5)),
            "batched-256-replicas (mixed)": leg(lambda: run_batched(susp, stream)),
        }
        legs["scaling_polydisperse_phi0.60_pe100_mu1"] = leg(lambda: run_scaling(susp, stream))

    launches = int(info1["launches"] - info0["launches"])
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": METRIC,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-pair/df32x2-state/f32-warp-virials"
        if args.precision == "mixed" else "f64",
        "data": "synthetic seeded packing (no dataset)",
        "config": {"workload": WORKLOAD, "N": N, "phi": 0.58, "Pe": 1000.0, "mu": 1.0,
                   "precision": args.precision, "timesteps_per_step": args.inner,
                   "dt": p["dt"], "box": round(w.L, 4), "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (state + list > 300 MB)",
                   "stress_sample_every": 1},
        "e2e": {"value": round(e2e_val, 1), "unit": METRIC,
                "h2d_bytes_per_step": 3 * 3 * 8 * N, "d2h_bytes_per_step": 58 * 8},
        "gpu_launches": launches,
        "roofline": roofline,
        "rebuild_roofline": rebuild_roof,
        "kernel_breakdown": breakdown,
        "eta_r": round(float(sig["eta_r"]), 4),
        "neighbour_builds": int(info1["nbuilds"] - info0["nbuilds"]),
    }
    if sparse:
        out["sampled_every_8_steps"] = sparse
    if fp64:
        out["fp64_path"] = fp64
    out.update(legs)
    if clk:
        out["clocks"] = clk
    return out


def _timed(stream, fn):
    """Device milliseconds of fn() on `stream` (CUDA events, synchronised)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def _system(susp, w, precision, stream):
    p = w.params
    s = susp.System(w.radii, w.box, precision=precision, eta=p["eta"], rho=p["rho"],
                    kn=p["kn"], kt=p["kt"], mu=p["mu"], skin=p["skin"],
                    shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"], dt=p["dt"])
    s.set_stream(stream.cuda_stream)
    s.set_state(w.x, w.U, w.W)
    return s


def run_single(susp, w, precision, stream, inner, steps, warmup=1):
    """particle-steps/s of one handle on workload w."""
    p = w.params
    s = _system(susp, w, precision, stream)
    for _ in range(warmup):
        s.step(inner, p["shear_rate"], p["kT"], p["dt"], p["seed"])

    def run():
        for _ in range(steps):
            s.step(inner, p["shear_rate"], p["kT"], p["dt"], p["seed"])
    ms = _timed(stream, run)
    eta = s.stress()["eta_r"]
    s.close()
    return {"value": round(w.N * inner * steps / (ms / 1e3), 1), "N": w.N,
            "precision": precision, "timesteps": inner * steps,
            "ms_per_timestep": round(ms / (inner * steps), 4), "eta_r": round(float(eta), 4)}


def run_scaling(susp, stream, inner=100, steps=3):
    """Linear-in-N scaling of the mixed path: one seeded periodic packing of
    15,625 polydisperse spheres (radii U[1, 1.4], phi 0.60, Pe 100, mu 1)
    replicated 4x4x4, 4x4x8, 4x8x8 and 8x8x8 times (1M, 2M, 4M, 8M spheres,
    the same local structure), each timed over `steps` calls of `inner`
    timesteps after one warm-up call; with the pair kernel's time per launch
    and its fraction of the HBM roofline from susp_profile."""
    import workloads
    hbm, peak_kind = peaks()
    out = {}
    for ks in ((4, 4, 4), (4, 4, 8), (4, 8, 8), (8, 8, 8)):
        rs, box, x, U, W, p = workloads.scaled_tiles(15625, ks, 0.60, 100.0, 1.0, poly=True,
                                                     pack_seed=1005, dyn_seed=2005)
        N = len(rs)
        s = susp.System(rs, box, precision="mixed", eta=p["eta"], rho=p["rho"], kn=p["kn"],
                        kt=p["kt"], mu=p["mu"], skin=p["skin"], shear_rate=p["shear_rate"],
                        kT=p["kT"], seed=p["seed"], dt=p["dt"])
        s.set_stream(stream.cuda_stream)
        s.set_state(x, U, W)
        s.step(inner, p["shear_rate"], p["kT"], p["dt"], p["seed"])

        def run():
            for _ in range(steps):
                s.step(inner, p["shear_rate"], p["kT"], p["dt"], p["seed"])
        ms = _timed(stream, run)
        # long enough to hold a rebuild (about every 250 steps)
        prof = s.profile(max(inner, 400), p["dt"])
        info = s.info()
        ij, _ = s.history()
        K, c = info["npairs"] / N, len(ij) / N
        pb = algorithmic_bytes("pair", "mixed", K, c, True)
        pair_ms = prof["pair"]["ms_per_launch"]
        # a due rebuild's device time in the profiled steps (one graph
        # launch), else one explicit rebuild timed around the call
        if prof["rebuild"]["launches"] > 0:
            rb_ms = prof["rebuild"]["ms_per_launch"]
        else:
            rb_ms = _timed(stream, s.build_neighbors)
        rbb = rebuild_bytes(K)
        out[f"{N // 1000000}M"] = {
            "N": N, "tiles": list(ks), "value": round(N * inner * steps / (ms / 1e3), 1),
            "ms_per_timestep": round(ms / (inner * steps), 4),
            "pair_ms_per_launch": round(pair_ms, 5),
            "pair_hbm_frac": round(pb * N / (pair_ms * 1e-3) / 1e9 / hbm, 4),
            "rebuild_ms": round(rb_ms, 4),
            "rebuild_hbm_frac": round(rbb * N / (rb_ms * 1e-3) / 1e9 / hbm, 4),
            "half_list_slots_per_sphere": round(K, 3), "contacts_per_sphere": round(c, 3)}
        s.close()
    # linear in N: the same particle-steps/s at every size
    v = [out[k]["value"] for k in out]
    out["value_spread"] = round(max(v) / min(v) - 1.0, 4)
    out["peak_kind"] = peak_kind
    return out


PHASE_VARIANTS = (
    ("full", {}),
    ("no_noise", dict(noise=0)),
    ("no_friction", dict(mu=0.0, kt=0.0)),
    ("no_sampling", dict(sample_every=1000)),
    ("no_noise_no_sampling", dict(noise=0, sample_every=1000)),
    ("no_noise_no_friction_no_sampling", dict(noise=0, mu=0.0, kt=0.0, sample_every=1000)),
    ("no_lubrication", dict(lubrication=0)),
)


def run_phases(inner: int = 100, warm: int = 200):
    """Where the pair kernel's time goes: the bench workload (1M spheres,
    mixed) with one term after another switched off, each kernel family
    timed per launch by susp_profile after `warm` steps.  The differences
    are the costs of the pair noise (Philox + Box-Muller + the Brownian
    algebra), the tangential history, the stress sampling (virials and their
    reductions) and the lubrication (resistances + pair noise)."""
    import torch

    import paper_2307_13802_gb300 as susp
    import workloads
    w = workloads.named(WORKLOAD)
    p = w.params
    stream = torch.cuda.Stream()
    out = {}
    for name, kw in PHASE_VARIANTS:
        args = dict(precision="mixed", eta=p["eta"], rho=p["rho"], kn=p["kn"], kt=p["kt"],
                    mu=p["mu"], skin=p["skin"], shear_rate=p["shear_rate"], kT=p["kT"],
                    seed=p["seed"], dt=p["dt"])
        args.update(kw)
        s = susp.System(w.radii, w.box, **args)
        s.set_stream(stream.cuda_stream)
        s.set_state(w.x, w.U, w.W)
        s.step(warm, p["shear_rate"], p["kT"], p["dt"], p["seed"])
        prof = s.profile(inner, p["dt"])
        out[name] = {f: round(v["ms_per_launch"], 5) for f, v in prof.items() if v["launches"]}
        s.close()
    full = out["full"]["pair"]
    costs = {"pair_noise": full - out["no_noise"]["pair"],
             "tangential_history": full - out["no_friction"]["pair"],
             "stress_sampling": full - out["no_sampling"]["pair"],
             "base": out["no_noise_no_friction_no_sampling"]["pair"]}
    return {"workload": WORKLOAD, "metric": "ms per launch", "variants": out,
            "pair_cost_ms": {k: round(v, 5) for k, v in costs.items()}}


def run_batched(susp, stream, inner=100, steps=3):
    """particle-steps/s of the 256-replica ensemble (N ~ U[500, 20000],
    phi ~ U[0.45, 0.60], Pe log-uniform in [0.1, 1000], mu in {0, 0.5, 1})
    stepped by one batch handle, mixed precision, with the skin picked by the
    library's autotuner before the timed steps."""
    import numpy as np
    import workloads
    table = workloads.replica_table()
    t0 = time.perf_counter()
    ws = workloads.make_replicas(table, tol=1e-2, processes=max(1, (os.cpu_count() or 2) - 1))
    gen_s = time.perf_counter() - t0
    kw = []
    for w in ws:
        p = w.params
        kw.append(dict(precision="mixed", eta=p["eta"], rho=p["rho"], kn=p["kn"], kt=p["kt"],
                       mu=p["mu"], skin=p["skin"], shear_rate=p["shear_rate"], kT=p["kT"],
                       seed=p["seed"], dt=p["dt"]))
    sizes = [w.N for w in ws]
    b = susp.System.batch(sizes, np.concatenate([w.radii for w in ws]),
                          np.stack([w.box for w in ws]), kw)
    b.set_stream(stream.cuda_stream)
    b.set_state(np.concatenate([w.x for w in ws]), np.concatenate([w.U for w in ws]),
                np.concatenate([w.W for w in ws]))
    dt = ws[0].params["dt"]
    b.step_batch(inner, dt)
    # the skin (and with it the cell size) is the autotuner's pick for this
    # ensemble: timed trials from the current state, which it restores
    skins = [0.2, 0.3, 0.45, 0.6, 0.8]
    skin, trial_ms = b.autotune(200, dt, skins)

    def run():
        for _ in range(steps):
            b.step_batch(inner, dt)
    ms = _timed(stream, run)
    total = int(sum(sizes))
    etas = [b.stress(r)["eta_r"] for r in range(len(ws))]
    i0 = b.info()
    prof = b.profile(inner, dt)
    i1 = b.info()
    b.close()
    breakdown = {f: {"ms_per_launch": round(v["ms_per_launch"], 5), "launches": v["launches"]}
                 for f, v in prof.items() if v["launches"]}
    return {"value": round(total * inner * steps / (ms / 1e3), 1), "replicas": len(ws),
            "particles": total, "precision": "mixed", "timesteps": inner * steps,
            "ms_per_timestep": round(ms / (inner * steps), 4),
            "finite_eta_r": bool(all(math.isfinite(e) for e in etas)),
            "skin": skin, "kernel_breakdown": breakdown,
            "rebuilds_in_profiled_steps": int(i1["nbuilds"] - i0["nbuilds"]),
            "autotune_ms_per_step": {str(k): (round(float(v), 4) if math.isfinite(v) else None)
                                     for k, v in zip(skins, trial_ms)},
            "packing_tol": 1e-2, "generation_s": round(gen_s, 1)}


def mixed_vs_fp64(susp, w, x, U, Wv, k, strain, stream, steps=500):
    """Accuracy of the mixed path against the FP64 path from one state:
    one evaluation (forces, torques, pair stresses, relative to the largest
    entry) and the relative viscosity averaged over `steps` timesteps run
    from that state with the same noise."""
    import numpy as np
    p = w.params
    out = {"N": w.N, "steps": steps}
    res = {}
    for prec in ("mixed", "fp64"):
        s = _system(susp, w, prec, stream)
        s.set_state(x, U, Wv)
        s.set_clock(k, strain)
        s.evaluate()
        F, T = s.forces()
        sig = s.stress()
        s.step(steps, p["shear_rate"], p["kT"], p["dt"], p["seed"])
        run = s.stress()
        res[prec] = (F, T, sig, run)
        s.close()
    Fm, Tm, sm, rm = res["mixed"]
    Fd, Td, sd, rd = res["fp64"]
    out["force_err"] = float(np.abs(Fm - Fd).max() / np.abs(Fd).max())
    out["torque_err"] = float(np.abs(Tm - Td).max() / np.abs(Td).max())
    for key in ("contact", "lubrication", "brownian"):
        out[f"{key}_stress_err"] = float(np.abs(sm[key] - sd[key]).max() / np.abs(sd[key]).max())
    out["eta_r_mixed"] = round(float(rm["eta_r"]), 6)
    out["eta_r_fp64"] = round(float(rd["eta_r"]), 6)
    out["eta_r_rel_err"] = float(abs(rm["eta_r"] / rd["eta_r"] - 1.0))
    out["N1_rel_err"] = float(abs(rm["N1"] - rd["N1"]) / max(abs(rd["N1"]), 1e-300))
    return out


def cpu_sample_workload():
    """Bounded sample of the workload: the 15,625-sphere periodic tile from
    which the 1M packing is replicated (same seeds, phi, Pe, mu)."""
    import workloads
    c = workloads.WORKLOADS[WORKLOAD]
    ps, ds = c["seeds"]
    return workloads.make(15625, c["phi"], c["pe"], c["mu"], poly=c["poly"],
                          pack_seed=ps, dyn_seed=ds)


def cpu_model() -> str:
    """The host CPU's model name as the OS reports it."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_worker(job):
    """One host core: the oracle on its own copy of the sample workload,
    `warm` untimed steps then `timed` timed steps; returns the seconds."""
    radii, box, params, x, U, W, warm, timed = job
    import oracle
    o = oracle.System(radii, box, **params)
    o.set_state(x, U, W)
    o.step(max(1, warm))            # list build, setup evaluation, warm-up
    t0 = time.perf_counter()
    o.step(timed)
    return time.perf_counter() - t0


def run_oracle_on_cores(warm: int, timed: int, cores: int = 0):
    """The serial oracle on every host core at once, each core stepping its
    own copy of the sample workload (independent replicas: the oracle itself
    is unchanged).  Returns (particle-steps/s over all cores, seconds of the
    slowest core, cores, N)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    w = cpu_sample_workload()
    cores = cores or os.cpu_count() or 1
    job = (w.radii, w.box, w.params, w.x, w.U, w.W, warm, timed)
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        secs = list(ex.map(_oracle_worker, [job] * cores))
    slowest = max(secs)
    return cores * w.N * timed / slowest, slowest, cores, w.N


def run_cpu_baseline(timesteps: int = 200):
    value, secs, cores, n = run_oracle_on_cores(1, timesteps)
    return {"value": round(value, 1), "unit": METRIC, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{n}-sphere periodic tile of the same packing recipe, {timesteps} "
                      f"timesteps on each of {cores} cores at once (one serial FP64 oracle "
                      f"per core on its own copy, O(N^2) list builds); {secs:.1f} s"}


def run_reference(args):
    inner = 20
    value, secs, cores, n = run_oracle_on_cores(args.warmup * inner, args.steps * inner)
    sample = (f"{n}-sphere periodic tile of the {WORKLOAD} packing, {inner} timesteps per "
              f"bench step on each of {cores} cores at once (one serial FP64 oracle per "
              f"core on its own copy)")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic seeded packing (no dataset)",
            "config": {"workload": WORKLOAD, "N": n, "timesteps_per_step": inner,
                       "parallelism": f"cpu{cores}"},
            "cpu_baseline": {"value": round(value, 1), "unit": METRIC, "cores": cores,
                             "kind": "oracle", "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": round(value, 1), "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.phases:
        if rank == 0:
            print(json.dumps(run_phases(inner=args.inner, warm=2 * args.inner)), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
        dist = td
    out = run_ours(args, rank, world, local_rank, dist)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = run_cpu_baseline()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

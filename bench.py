#!/usr/bin/env python3
"""Throughput of the multispecies Enskog/RPA lattice Boltzmann step on GB300.

Workload (default): binary hard-sphere mixture sigma = (1, 1.5), packing 0.2,
equal mole fractions, tau = 1, no attraction, 5% concentration sine wave
along x (Eq. perturba) on a 256^3 periodic D3Q19 lattice, FP32 populations.
One "step" is one full time step of the method (moments, contact values,
both force passes, collision, streaming) over the whole lattice.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mlb|reference]

Prints one JSON line.  value = MLUPS per species over all ranks (species-site
updates per microsecond); each rank runs an independent replica (weak scaling,
no data-path collective).  --impl reference times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS/species + % HBM roofline; surrogate/BF16 speedup at <=1% D_mutual error"
UNIT = "MLUPS/species"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["mlb", "reference"], default="mlb")
    ap.add_argument("--size", type=int, default=None, help="cubic lattice extent (default: the workload's)")
    ap.add_argument("--workload", choices=["binary", "attraction", "ensemble", "surrogate", "taylor"], default="binary",
                    help="binary: sigma 1/1.5 packing 0.2 (256^3); attraction: sigma 2/3, eps kT/2 tails, "
                         "packing 0.3, 1%% noise (128^3); ensemble: 64 independent binary systems of "
                         "32^3..128^3, packing 0.05-0.20, shear 0-0.05, stepped as one captured graph; "
                         "surrogate: the binary workload with the learned hard-core force (trained first on "
                         "64x8x8 frames, exact recheck every 50 steps, bound 5%%), timed against the exact step; "
                         "taylor: the 3-species Taylor channel 512x64x64 between moving walls (--size sets the "
                         "channel's cross-section, the length is 8x)")
    ap.add_argument("--members", type=int, default=64, help="ensemble size")
    ap.add_argument("--meanfield", choices=["fp32", "bf16", "bf16_1pass"], default="fp32",
                    help="attractive mean field: FP32 column sums, or the tensor-core band product in BF16 "
                         "(compensated hi/lo, or the single hi product)")
    ap.add_argument("--sweeps", type=int, default=1,
                    help="Jacobi sweeps of the half step u* = u + a(u*)/2 (the method's default: one)")
    ap.add_argument("--no-autotune", action="store_true", help="ensemble: keep the default decomposition")
    ap.add_argument("--cpu-sample", type=int, default=128, help="oracle sample extent for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the surrogate / BF16 / ensemble forms reported beside the plain path")
    return ap.parse_args()


DEFAULT_SIZE = {"binary": 256, "attraction": 128, "ensemble": 0, "surrogate": 256, "taylor": 64}


def workload(size, kind="binary"):
    from paper_1105_3634_gb300 import workloads as W
    if kind == "attraction":
        return W.binary_attraction((size, size, size))
    if kind == "taylor":
        return W.taylor_channel((8 * size, size, size))
    return W.binary_config1((size, size, size))


def grid_of(size, kind):
    return [8 * size, size, size] if kind == "taylor" else [size, size, size]


def config_dict(size, kind="binary"):
    desc = {"binary": "binary hard spheres sigma=(1,1.5), packing 0.2, tau=1, 5% sine wave",
            "surrogate": "binary hard spheres sigma=(1,1.5), packing 0.2, tau=1, 5% sine wave, hard-core force "
                         "from the learned surrogate (exact recheck every 50 steps, bound 5%)",
            "attraction": "binary sigma=(2,3), attractive tails -eps(sigma/r)^6 to 2.5 sigma, eps=kT/2, "
                          "packing 0.3, 1% noise, tau=1",
            "taylor": "Taylor channel: solvents sigma=(2,2.5) at packing 0.211, solute sigma=3 at mole fraction "
                      "1e-3 in a Gaussian pulse of width 8, walls normal to y moving at -/+0.05 along x, tau=1"}[kind]
    grid = grid_of(size, kind)
    S = 3 if kind == "taylor" else 2
    sites = grid[0] * grid[1] * grid[2]
    where = "channel with bounce-back walls" if kind == "taylor" else "periodic"
    return {"workload": f"{desc}, {grid[0]}x{grid[1]}x{grid[2]} {where} D3Q19",
            "grid": grid, "species": S, "lattice": "D3Q19", "precision": "FP32 populations",
            "force_scheme": "semi-implicit half-force shift",
            "l2": "inputs larger than L2 (populations %.2f GB per buffer)" % (S * 19 * 4 * sites / 1e9),
            "parallelism": "replicas"}


# ------------------------------------------------------------------ per-kernel algorithmic bytes
def algorithmic_bytes(kernel, S, npairs, has_fext=False, local_g=True):
    """Bytes per species-site that the kernel must move by design (FP32)."""
    g = 4.0 * npairs / S
    table = {
        # f read, (dn, j) write (+ g write when the contact values are site-local)
        "k_moments": 76 + 16 + (g if local_g else 0),
        "k_gfield": 4 + g,                                       # dn read, g write
        "k_pass1": 16 + g + 12 + 16 + (12 if has_fext else 0),    # moments, g read; frest, p* write
        "k_pass2": 16 + g + 12 + 12,                               # p* = (n - n_ref, u*), g, frest read; acc write
        "k_sweep": 16 + g + 16 + 12 + 16,                          # previous p*, g, own moments, frest read; p* write
        "k_collide": 76 + 16 + 12 + 76,                            # f, moments, acc read; f write
        "k_attraction": 4 + 12,                                     # n - n_ref read; G write
        # pass 2 fused with the collision: (n - n_ref, u*), g, frest, f, moments read; f write
        "k_pass2_collide": 16 + g + 12 + 76 + 16 + 76,
    }
    return table.get(kernel)


def shell_points(sigma):
    """sum over ordered species pairs of |S_ab|, the lattice points with
    (sigma_ab - 1/2)^2 <= |d|^2 < (sigma_ab + 1/2)^2 (the contact shells)."""
    tot = 0
    for sa in sigma:
        for sb in sigma:
            s = 0.5 * (sa + sb)
            R = int(math.ceil(s + 0.5)) + 1
            for dz in range(-R, R + 1):
                for dy in range(-R, R + 1):
                    for dx in range(-R, R + 1):
                        q = dx * dx + dy * dy + dz * dz
                        if q > 0 and (s - 0.5) ** 2 <= q < (s + 0.5) ** 2:
                            tot += 1
    return tot


def attraction_points(lat):
    """sum over ordered species pairs with eps_ab != 0 of |A_ab|, the lattice
    points with sigma_ab <= |d| <= lambda_c sigma_ab."""
    tot = 0
    S = len(lat.sigma)
    for a in range(S):
        for b in range(S):
            if lat.eps[a][b] == 0.0:
                continue
            s = 0.5 * (lat.sigma[a] + lat.sigma[b])
            rc = lat.lambda_c[a][b] * s
            R = int(math.ceil(rc)) + 1
            for dz in range(-R, R + 1):
                for dy in range(-R, R + 1):
                    for dx in range(-R, R + 1):
                        q = dx * dx + dy * dy + dz * dz
                        if q > 0 and s * s <= q <= rc * rc:
                            tot += 1
    return tot


# algorithmic FP32 operations per (ordered pair, stencil point):
#   pass 1: pair value (2), hard core (7), velocity exchange (15), friction tensor (12)
#   pass 2: pair value (2), velocity exchange (16)
#   a further predictor sweep: pass 1 without the hard core (29)
#   attraction: one 3-vector multiply-add per point of the full region (6)
FLOPS_PER_SHELL_POINT = {"k_pass1": 36, "k_pass2": 18, "k_pass2_collide": 18, "k_sweep": 29}
FLOPS_PER_ATTRACTION_POINT = 6
# the surrogate network per site: 3^3 conv 2->32, 3^3 conv 32->32 (tensor cores), 1^3 conv 32->6
FLOPS_PER_SURROGATE_SITE = 2 * (27 * 2 * 32 + 27 * 32 * 32 + 32 * 6)


def attraction_columns(lat):
    """Columns (dx, dy) of the attraction regions: the offsets of any pair's
    sigma_ab <= |d| <= lambda_c sigma_ab projected onto the (x, y) plane."""
    cols = set()
    S = len(lat.sigma)
    for a in range(S):
        for b in range(S):
            if lat.eps[a][b] == 0.0:
                continue
            s = 0.5 * (lat.sigma[a] + lat.sigma[b])
            rc = lat.lambda_c[a][b] * s
            R = int(math.floor(rc + 1e-9))
            for dz in range(-R, R + 1):
                for dy in range(-R, R + 1):
                    for dx in range(-R, R + 1):
                        q = dx * dx + dy * dy + dz * dz
                        if q > 0 and s * s <= q <= rc * rc:
                            cols.add((dx, dy))
    return len(cols)


def tensor_flops_attraction(lat, products):
    """MMA flops of one tensor-core attraction launch: per tile of 128 x sites
    and 16 planes, per column, M 128 x N 48 S x K 32 S, times the products."""
    S = lat.nspecies
    nx, ny, nz = lat.shape
    tiles = -(-nx // 128) * ny * -(-nz // 16)
    return tiles * attraction_columns(lat) * products * 2.0 * 128 * (48 * S) * (32 * S)


def fp32_peak_tflops(sm_mhz=2070.0):
    """152 SMs x 128 FP32 lanes x 2 (FMA) x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


KERNEL_SOURCE = {"k_pass1": "mlb_pass1.cu", "k_sweep": "mlb_sweep.cu", "k_pass2": "mlb_pass2.cu",
                 "k_pass2_collide": "mlb_pass2.cu",
                 "k_attraction": "mlb_attraction.cu", "k_surrogate": "mlb_surrogate.cu"}


def kernel_source_sha(kernel):
    """First 16 hex digits of the SHA-256 of the kernel's translation unit and
    every internal header."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1105_3634_gb300", "csrc")
    h = hashlib.sha256()
    headers = sorted(f for f in os.listdir(csrc) if f.endswith((".h", ".cuh")))
    for f in [KERNEL_SOURCE.get(kernel, "mlb_kernels.cu")] + headers:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel, size, kind="binary"):
    """DRAM bytes per launch from a committed ncu summary under profiles/
    (a line `bench-traffic: kernel=... workload=... size=... bytes_per_launch=...
    kernel_source_sha256_16=...`), if it was taken on the current kernel
    source; None otherwise."""
    pdir = os.path.join(ROOT, "profiles")
    try:
        sha = kernel_source_sha(kernel)
        for name in sorted(os.listdir(pdir)):
            for line in open(os.path.join(pdir, name)):
                if not line.startswith("bench-traffic:"):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:])
                if (kv.get("kernel") == kernel and kv.get("workload", "binary") == kind
                        and int(kv.get("size", -1)) == size and kv.get("kernel_source_sha256_16") == sha):
                    return float(kv["bytes_per_launch"])
    except Exception:
        return None
    return None


def reduce_max(value, dist=None, device=None):
    """Maximum of a per-rank float over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, nspecies, nsites, steps, seconds):
    """Whole-job MLUPS per species: every rank advances its own replica."""
    return world * nspecies * nsites * steps / seconds / 1e6


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_peak_bf16():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except Exception:
        return 1900.0


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = (uuid or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and self.uuid not in parts[1].lower():
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ cpu baseline (oracle)
def host_cpu():
    """The host's CPU model (lscpu 'Model name', else /proc/cpuinfo) and core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"model": model or "unknown", "nproc": os.cpu_count()}


def cpu_baseline(size, kind="binary", steps=2, one_thread_size=None):
    import numpy as np
    import oracle
    oracle.build()
    lat, n = workload(size, kind)
    f = oracle.init(lat, n)
    oracle.step(lat, f, 1)                    # warm (page-in, thread pool)
    t0 = time.perf_counter()
    oracle.step(lat, f, steps)
    dt = time.perf_counter() - t0
    value = lat.nspecies * lat.nsites * steps / dt / 1e6
    out = {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle", "host": host_cpu(),
           "sample": "%s lattice of the same physics, %d timed steps after 1 warm step, FP64 C oracle, OpenMP"
                     % ("x".join(str(v) for v in grid_of(size, kind)), steps)}
    if one_thread_size:
        cores = oracle.num_threads()
        lat1, n1 = workload(one_thread_size, kind)
        f1 = oracle.init(lat1, n1)
        oracle.set_num_threads(1)
        try:
            t0 = time.perf_counter()
            oracle.step(lat1, f1, 1)
            dt1 = time.perf_counter() - t0
        finally:
            oracle.set_num_threads(cores)
        out["one_thread"] = {"value": lat1.nspecies * lat1.nsites / dt1 / 1e6, "unit": UNIT, "cores": 1,
                             "sample": "%s lattice, 1 step" % "x".join(str(v) for v in grid_of(one_thread_size, kind))}
    return out


# ------------------------------------------------------------------ the GPU arm
def run_mlb(args, rank, world, local_rank):
    import numpy as np
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_1105_3634_gb300 import build as B
    B.build()
    from paper_1105_3634_gb300 import mlb
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    lat, n = workload(args.size, args.workload)
    lat.predictor_sweeps = args.sweeps
    lat.meanfield = args.meanfield
    S, N = lat.nspecies, lat.nsites
    stream = torch.cuda.Stream(device=dev)
    sim = mlb.Simulation(lat, stream=stream)
    sim.set_fields(n)
    sim.step(args.warmup)
    sim.synchronize()
    surrogate = None
    if args.workload == "surrogate":
        surrogate = run_surrogate_setup(args, mlb, sim, lat, stream)

    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = ""
    clocks = Clocks(uuid)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    sim.profile(True)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    sim.step(args.steps)
    t_end.record(stream)
    sim.synchronize()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms_total = t_start.elapsed_time(t_end)
    prof = sim.profile_read()
    sim.profile(False)
    ms_total = reduce_max(ms_total, dist, dev)
    ms_step = ms_total / args.steps
    value = job_value(world, S, N, args.steps, ms_total * 1e-3)

    # end to end through the C ABI with host buffers: upload the fields, then
    # every step one monitored step whose FP64 conservation sums (the
    # monitored metric) come back to pinned host memory, read by the host one
    # step behind while the next step runs; finally the moments to the host
    e2e = None
    if not args.no_e2e:
        nh = torch.empty((S, N), dtype=torch.float64, pin_memory=True).numpy()
        nh[:] = n
        n_out = torch.empty((S, N), dtype=torch.float64, pin_memory=True).numpy()
        u_out = torch.empty((S, 3, N), dtype=torch.float64, pin_memory=True).numpy()
        sums = [torch.empty(S + 3, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        # one untimed pass over the same path and buffers (the first transfers
        # through freshly pinned pages run slower), like the device warm-up
        sim.set_fields(nh)
        sim.step_monitored(sums[0])
        sim.moments(n_out, u_out)
        sim.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        sim.set_fields(nh)
        mass0 = None
        for k in range(args.steps):
            sim.step_monitored(sums[k % 2])
            done[k % 2].record(stream)
            if k >= 1:
                done[(k - 1) % 2].synchronize()
                m = float(sums[(k - 1) % 2][:S].sum())
                mass0 = m if mass0 is None else mass0
                if not abs(m - mass0) <= 1e-6 * abs(mass0):
                    raise RuntimeError(f"mass drift at step {k - 1}: {m} vs {mass0}")
        sim.moments(n_out, u_out)
        dt = reduce_max(time.perf_counter() - t0, dist, dev)
        h2d = nh.nbytes / args.steps
        d2h = (S + 3) * 8 + (n_out.nbytes + u_out.nbytes) / args.steps
        e2e = {"value": job_value(world, S, N, args.steps, dt), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": args.steps,
               "note": "the one-time set_fields upload and get_moments read-back are spread over the "
                       "steps: a short run weighs them more",
               "what": "mlb_set_fields from pinned host n, K x mlb_step_monitored (FP64 conservation sums of "
                       "every step to pinned host memory, checked one step behind), mlb_get_moments"}

    # roofline of the dominant kernel (largest device time in the timed region):
    # the stencil passes are bound by FP32 issue, the others by HBM
    npairs = S * (S + 1) // 2
    peak, peak_kind = measured_peak_hbm()
    pts = shell_points(lat.sigma)
    kernels = {}
    for name, (ms, cnt) in prof.items():
        if cnt == 0:
            continue
        per_launch_ms = ms / cnt
        bss = algorithmic_bytes(name, S, npairs)
        b = bss * S * N if bss is not None else None
        k = {"launches": cnt, "ms_total": ms, "ms_per_launch": per_launch_ms,
             "share": ms / sum(v[0] for v in prof.values()), "algorithmic_bytes_per_launch": b,
             "achieved_gbs": (b / (per_launch_ms * 1e-3) / 1e9) if b is not None else None}
        fl = None
        if name in FLOPS_PER_SHELL_POINT:
            fl = FLOPS_PER_SHELL_POINT[name] * pts * N
        elif name == "k_attraction" and args.meanfield != "fp32":
            fl = FLOPS_PER_ATTRACTION_POINT * attraction_points(lat) * N
            tfl = tensor_flops_attraction(lat, 3 if args.meanfield == "bf16" else 1)
            k["tensor_flops_per_launch"] = tfl
            k["achieved_tensor_tflops"] = tfl / (per_launch_ms * 1e-3) / 1e12
            k["flops_note"] = ("algorithmic: the direct lattice sum (6 flops per region point); tensor: the BF16 "
                               "MMAs executed (band matrices along z, zeros included; %s)"
                               % ("hi*hi + hi*lo + lo*hi" if args.meanfield == "bf16" else "hi*hi"))
        elif name == "k_attraction":
            fl = FLOPS_PER_ATTRACTION_POINT * attraction_points(lat) * N
            k["flops_note"] = ("direct lattice sum, one 3-vector FMA per region point; the column kernel "
                               "executes about 1.25 FP32 flops per point through K(-d) = -K(d)")
        elif name == "k_surrogate":
            fl = FLOPS_PER_SURROGATE_SITE * N
            k["flops_note"] = "dense network flops; the 32->32 layer (94% of them) on BF16 tensor cores"
        if fl is not None:
            k["algorithmic_flops_per_launch"] = fl
            k["achieved_tflops"] = fl / (per_launch_ms * 1e-3) / 1e12
        kernels[name] = k
    top = max(kernels, key=lambda k: kernels[k]["ms_total"])
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    derived = fp32_peak_tflops(sm_mhz)
    # the measured FP32 FMA throughput (project kernel, after the timed region)
    try:
        fma = mlb.fma_throughput(1 << 14, 10)
    except Exception:
        fma = None
    fpk = fma or derived
    fpk_kind = ("measured: project FMA kernel (mlb_fma_throughput, 16 packed chains per thread)" if fma
                else f"derived: 152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz")
    for k in kernels.values():
        if k.get("achieved_tflops") is not None and "tensor_flops_per_launch" not in k:
            k["frac_of_fp32_peak"] = k["achieved_tflops"] / fpk
    kt = kernels[top]
    alu = {"kernel": top, "bound": "alu", "achieved": kt.get("achieved_tflops"), "peak": fpk,
           "peak_kind": fpk_kind,
           "unit": "TFLOP/s", "frac": (kt["achieved_tflops"] / fpk) if "achieved_tflops" in kt else None,
           "traffic": committed_traffic(top, args.size, args.workload)}
    hbm = {"kernel": top, "bound": "hbm", "achieved": kt["achieved_gbs"], "peak": peak,
           "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
           "unit": "GB/s", "frac": (kt["achieved_gbs"] / peak) if kt["achieved_gbs"] is not None else None,
           "traffic": committed_traffic(top, args.size, args.workload)}
    # the binding resource of the dominant kernel: the larger fraction of its peak
    roof = alu if (alu["frac"] or 0.0) > (hbm["frac"] or 0.0) else hbm
    if top == "k_attraction" and args.meanfield != "fp32":
        tpk = measured_peak_bf16()
        roof = {"kernel": top, "bound": "tensor", "achieved": kt["achieved_tensor_tflops"], "peak": tpk,
                "peak_kind": "measured (MEASURED_PEAKS.json bf16_tflops, burst)", "unit": "TFLOP/s",
                "frac": kt["achieved_tensor_tflops"] / tpk,
                "traffic": committed_traffic(top, args.size, args.workload)}
    if top == "k_surrogate":
        tpk = measured_peak_bf16()
        roof = {"kernel": top, "bound": "tensor", "achieved": kt["achieved_tflops"], "peak": tpk,
                "peak_kind": "measured (MEASURED_PEAKS.json bf16_tflops, burst)", "unit": "TFLOP/s",
                "frac": kt["achieved_tflops"] / tpk, "traffic": committed_traffic(top, args.size, args.workload)}
    try:
        project_copy = mlb.copy_bandwidth(1 << 31, 20)
    except Exception:
        project_copy = None
    roof["peaks_gbs"] = {"measured_copy": peak, "project_copy_kernel": project_copy, "nominal": 7900.0}
    roof["peaks_fp32_tflops"] = {"project_fma_kernel": fma, "derived": derived}
    step_bytes = 184.0 * S * N
    step_roof = {"bytes_per_species_site": 184, "achieved_gbs": step_bytes / (ms_step * 1e-3) / 1e9,
                 "frac": step_bytes / (ms_step * 1e-3) / 1e9 / peak, "peak_gbs": peak}

    if surrogate is not None:
        net = surrogate.pop("net")
        active, last, rechecks, rejections = sim.surrogate_status()
        surrogate.update({"ms_per_step": ms_step, "speedup_vs_exact": surrogate["ms_per_step_exact"] / ms_step,
                          "active_at_end": active, "last_recheck_error": last, "rechecks": rechecks,
                          "rejections": rejections})
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded sine-wave mixture)",
           "config": dict(config_dict(args.size, args.workload), predictor_sweeps=args.sweeps,
                          meanfield=args.meanfield),
           "roofline": roof, "step_roofline": step_roof,
           "kernels": kernels, "gpu_launches": sim.launches_per_step() * args.steps * 1,
           "mlups": value / S, "clocks": clk, "e2e": e2e}
    if surrogate is not None:
        out["surrogate"] = surrogate
        out["dtype"] = "f32 step, bf16 network activations (fp32 input and accumulation)"
    sim.close()
    if surrogate is not None:
        net.close()
    if (args.workload == "binary" and args.size == 256 and world == 1 and not args.no_variants
            and args.sweeps == 1 and args.meanfield == "fp32"):
        out["variants"] = run_variants(mlb, torch, value, ms_step)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = {"binary": args.cpu_sample, "taylor": 16}.get(args.workload, 48)
        out["cpu_baseline"] = cpu_baseline(sample, args.workload,
                                           one_thread_size={"binary": 64, "taylor": 8}.get(args.workload, 24))
    if dist:
        dist.destroy_process_group()
    return out


# ------------------------------------------------------------------ the other forms of the step
def fitted_D(mlb, lat, n0, amp=1e-3, t0=100, t1=1100, every=100, attach=None):
    """Mutual diffusion coefficient from the decay of the concentration mode
    n0_B dn^A - n0_A dn^B of a small sine wave along x (Eq. perturba), fitted
    over [t0, t1]; attach(sim) runs before the first step (a surrogate)."""
    import numpy as np
    from paper_1105_3634_gb300 import workloads as W
    n = W.sine_wave(lat, n0, amp)
    sim = mlb.Simulation(lat)
    sim.set_fields(n)
    if attach:
        attach(sim)
    q = 2 * math.pi / lat.shape[0]
    ph = np.exp(-1j * q * W.coordinate(lat, 0))
    ts, amps = [], []
    sim.step(t0)
    for t in range(t0, t1 + 1, every):
        nn, _ = sim.moments()
        ts.append(t)
        amps.append(abs(((nn[0] - n0[0]) * n0[1] - (nn[1] - n0[1]) * n0[0]) @ ph))
        sim.step(every)
    sim.close()
    return -np.polyfit(np.array(ts, float), np.log(np.array(amps)), 1)[0] / q ** 2


def time_steps(mlb, torch, lat, n, steps, warmup=3, attach=None):
    """ms per step and the per-kernel profile of `steps` steps of one Simulation."""
    stream = torch.cuda.Stream()
    sim = mlb.Simulation(lat, stream=stream)
    sim.set_fields(n)
    if attach:
        attach(sim)
    sim.step(warmup)
    sim.synchronize()
    sim.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    sim.synchronize()
    prof = sim.profile_read()
    sim.profile(False)
    status = sim.surrogate_status() if attach else None
    sim.close()
    return e0.elapsed_time(e1) / steps, {k: v[0] / v[1] for k, v in prof.items() if v[1]}, status


def run_variants(mlb, torch, plain_value, plain_ms):
    """The other forms of the step beside the plain FP32 path, each timed
    briefly, with its speed ratio and its mutual diffusion coefficient against
    the exact FP32 path on the same lattice (the exact path equals the FP64
    oracle to ~1e-5 in state and D: the GPU test suite)."""
    from paper_1105_3634_gb300 import workloads as W
    from paper_1105_3634_gb300 import surrogate as SG
    out = {"plain_256": {"value": plain_value, "ms_per_step": plain_ms}}
    # learned surrogate of the hard-core force, 256^3 (trained on 64 x 8 x 8 frames)
    t0 = time.perf_counter()
    params, ins, outs, _ = SG.recipe(mlb)
    train_s = time.perf_counter() - t0
    nets = []

    def attach(sim):
        net = mlb.Net(sim.lat.shape)
        net.set_params(params)
        net.set_scales(ins, outs)
        nets.append(net)
        sim.attach_surrogate(net, recheck_every=50, bound=0.05)
    lat, n = W.binary_config1((256, 256, 256))
    ms, prof, status = time_steps(mlb, torch, lat, n, 10, attach=attach)
    small = W.Lattice(shape=(64, 8, 8), sigma=[1.0, 1.5], tau=1.0)
    n0 = W.densities_from_packing(0.2, small.sigma, [0.5, 0.5])
    D_exact = fitted_D(mlb, small, n0)
    D_surr = fitted_D(mlb, small, n0, attach=attach)
    for net in nets:
        net.close()
    out["surrogate_256"] = {"ms_per_step": ms, "value": 2 * lat.nsites / ms / 1e3, "speedup_vs_plain": plain_ms / ms,
                            "kernels_ms": prof, "surrogate_active": bool(status[0]),
                            "last_recheck_error": status[1], "training_s": train_s,
                            "D_mutual": D_surr, "D_mutual_exact": D_exact,
                            "D_mutual_rel_error": (D_surr - D_exact) / D_exact,
                            "D_lattice": "64x8x8, sigma 1/1.5, packing 0.2, wave 1e-3, steps 100-1100"}
    # the attractive mean field: FP32 column sums against the BF16 tensor-core product, 128^3
    lat, n = W.binary_attraction((128, 128, 128))
    small = W.Lattice(shape=(64, 16, 16), sigma=list(lat.sigma), tau=1.0, eps=lat.eps, lambda_c=lat.lambda_c)
    n0 = W.densities_from_packing(0.3, small.sigma, [0.5, 0.5])
    D_fp32 = None
    for mf in ("fp32", "bf16", "bf16_1pass"):
        lat.meanfield = small.meanfield = mf
        ms, prof, _ = time_steps(mlb, torch, lat, n, 10)
        D = fitted_D(mlb, small, n0)
        if mf == "fp32":
            D_fp32, base_ms, base_attr = D, ms, prof.get("k_attraction")
        out["attraction_128_" + mf] = {
            "ms_per_step": ms, "value": 2 * lat.nsites / ms / 1e3, "k_attraction_ms": prof.get("k_attraction"),
            "speedup_vs_fp32": base_ms / ms, "attraction_kernel_speedup_vs_fp32": base_attr / prof["k_attraction"],
            "D_mutual": D, "D_mutual_rel_error_vs_fp32": (D - D_fp32) / D_fp32,
            "D_lattice": "64x16x16, sigma 2/3, eps kT/2 tails to 2.5 sigma, packing 0.3, wave 1e-3"}
    # the batched ensemble of 64 uneven systems, one captured graph per two steps
    systems = W.ensemble(64)
    sims = [mlb.Simulation(l, stream=torch.cuda.Stream()) for l, _ in systems]
    for sim, (_, nn) in zip(sims, systems):
        sim.set_fields(nn)
        sim.autotune(trials=1)
    units = sum(l.nspecies * l.nsites for l, _ in systems)
    bstream = torch.cuda.Stream()
    batch = mlb.Batch(sims, stream=bstream)
    batch.step(2)
    batch.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bstream)
    batch.step(10)
    e1.record(bstream)
    batch.synchronize()
    ms = e0.elapsed_time(e1) / 10
    grouped = batch.grouped_members()
    batch.close()
    # the same members, each by its own launches inside the graph
    batch = mlb.Batch(sims, stream=bstream, lanes=0)
    batch.step(2)
    batch.synchronize()
    e0.record(bstream)
    batch.step(10)
    e1.record(bstream)
    batch.synchronize()
    ms_own = e0.elapsed_time(e1) / 10
    batch.close()
    for sim in sims:
        sim.close()
    # many small systems (256 x 16^3): the batch (grouped launches, one graph)
    # against the same members stepped through mlb_step one after the other
    # (every call asynchronous on the member's own stream, one wait at the end)
    small = []
    for k in range(256):
        sig = [1.0, 1.5]
        if k % 2:
            lat_k = W.Lattice(shape=(16, 16, 16), sigma=sig, wall_axis=1, wall_u_lo=(-0.02, 0.0, 0.0),
                              wall_u_hi=(0.02, 0.0, 0.0))
        else:
            lat_k = W.Lattice(shape=(16, 16, 16), sigma=sig)
        n0 = W.densities_from_packing(0.05 + 0.15 * (k % 7) / 6, sig, [0.5, 0.5])
        small.append((lat_k, W.sine_wave(lat_k, n0, 0.05)))
    ssims = [mlb.Simulation(l, stream=torch.cuda.Stream()) for l, _ in small]
    for sim, (_, nn) in zip(ssims, small):
        sim.set_fields(nn)
    sunits = sum(l.nspecies * l.nsites for l, _ in small)
    for sim in ssims:
        sim.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sim in ssims:
        sim.step(10)
    torch.cuda.synchronize()
    ms_turn = (time.perf_counter() - t0) * 1e3 / 10
    sb = mlb.Batch(ssims, stream=bstream)
    sb.step(2)
    sb.synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(bstream)
    sb.step(10)
    e1.record(bstream)
    sb.synchronize()
    ms_sb_wall = (time.perf_counter() - t0) * 1e3 / 10
    ms_sb = e0.elapsed_time(e1) / 10
    sgrouped = sb.grouped_members()
    sb.close()
    for sim in ssims:
        sim.close()
    out["ensemble_256_small"] = {
        "ms_per_ensemble_step": ms_sb, "ms_per_ensemble_step_wall": ms_sb_wall, "value": sunits / ms_sb / 1e3,
        "ms_per_ensemble_step_members_in_turn": ms_turn, "speedup_vs_members_in_turn": ms_turn / ms_sb_wall,
        "grouped_members": sgrouped, "species_sites": sunits, "D_mutual_rel_error": 0.0,
        "config": "256 binary systems 16^3 sigma=(1,1.5), packing 0.05-0.20, half sheared (walls at -+0.02); "
                  "members in turn: mlb_step(10) per member (asynchronous, own streams), one wait; "
                  "both timed by the host clock"}
    # the ensemble with attractive tails (sigma 2/3, packing to 0.30): the mean
    # field in FP32 and on the tensor cores
    ens = {}
    for mf in ("fp32", "bf16"):
        asys = W.ensemble_attraction(64, meanfield=mf)
        asims = [mlb.Simulation(l, stream=torch.cuda.Stream()) for l, _ in asys]
        for sim, (_, nn) in zip(asims, asys):
            sim.set_fields(nn)
        ab = mlb.Batch(asims, stream=bstream)
        ab.step(2)
        ab.synchronize()
        e0.record(bstream)
        ab.step(10)
        e1.record(bstream)
        ab.synchronize()
        ens[mf] = e0.elapsed_time(e1) / 10
        aunits = sum(l.nspecies * l.nsites for l, _ in asys)
        ab.close()
        for sim in asims:
            sim.close()
    out["ensemble_64_attraction"] = {
        "ms_per_ensemble_step_fp32": ens["fp32"], "ms_per_ensemble_step_bf16": ens["bf16"],
        "value_bf16": aunits / ens["bf16"] / 1e3, "speedup_bf16_vs_fp32": ens["fp32"] / ens["bf16"],
        "species_sites": aunits,
        "config": "64 binary systems sigma=(2,3), eps kT/2 tails to 2.5 sigma, cubes 32^3..128^3, "
                  "packing 0.05-0.30, shear 0-0.05; one captured graph"}
    out["ensemble_64"] = {"ms_per_ensemble_step": ms, "value": units / ms / 1e3, "ratio_to_plain": units / ms / 1e3 / plain_value,
                          "species_sites": units, "grouped_members": grouped,
                          "ms_per_ensemble_step_own_launches": ms_own, "grouping_speedup": ms_own / ms,
                          "D_mutual_rel_error": 0.0,
                          "note": "every member's populations equal those of the member stepped alone bit for bit"}
    return out


def run_surrogate_setup(args, mlb, sim, lat, stream):
    """Train the surrogate (64x8x8 frames, stencil start, GPU fine-tuning), time
    the exact step on `sim` over the same number of steps, then attach the
    network; the caller's timed region then measures the surrogate step."""
    import torch
    from paper_1105_3634_gb300 import surrogate as SG
    t0 = time.perf_counter()
    params, ins, outs, _ = SG.recipe(mlb)
    train_s = time.perf_counter() - t0
    net = mlb.Net(lat.shape)
    net.set_params(params)
    net.set_scales(ins, outs)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sim.synchronize()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    sim.synchronize()
    ms_exact = e0.elapsed_time(e1) / args.steps
    sim.attach_surrogate(net, recheck_every=50, bound=0.05)
    sim.step(args.warmup)
    sim.synchronize()
    return {"net": net, "ms_per_step_exact": ms_exact, "recheck_every": 50, "bound": 0.05,
            "training": "240 frames on 64x8x8, least-squares linear-response start, 100 epochs of Adam "
                        "on the GPU (lr 1e-6 cosine)", "training_s": train_s,
            "exact_timing": "same lattice and stream, the same number of steps just before, CUDA events"}


def run_ensemble(args, rank, world, local_rank):
    """Batched ensemble: every member autotuned, then (a) each member stepped
    alone in turn through mlb_step (the plain path), (b) all members stepped
    together through one captured CUDA graph (mlb_batch_step).  value = (b)."""
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_1105_3634_gb300 import build as B
    B.build()
    from paper_1105_3634_gb300 import mlb
    from paper_1105_3634_gb300 import workloads as W
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    systems = W.ensemble(args.members)
    sims = []
    for lat, n in systems:
        sim = mlb.Simulation(lat, stream=torch.cuda.Stream(device=dev))
        sim.set_fields(n)
        sims.append(sim)
    tuned = [sim.autotune(trials=2) for sim in sims] if not args.no_autotune else []
    units = sum(lat.nspecies * lat.nsites for lat, _ in systems)
    steps = max(2, min(args.steps, 100) // 2 * 2)
    warm = max(2, args.warmup // 2 * 2)
    for sim in sims:
        sim.step(warm)
        sim.synchronize()
    if dist:
        dist.barrier()
    # (a) each member alone in turn
    t0 = time.perf_counter()
    for sim in sims:
        sim.step(steps)
        sim.synchronize()
    t_seq = reduce_max(time.perf_counter() - t0, dist, dev)
    # (b) one batch
    bstream = torch.cuda.Stream(device=dev)
    batch = mlb.Batch(sims, stream=bstream)
    batch.step(warm)
    batch.synchronize()
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = ""
    clocks = Clocks(uuid)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(bstream)
    batch.step(steps)
    e1.record(bstream)
    batch.synchronize()
    t_batch_wall = time.perf_counter() - t0
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1), dist, dev)
    grouped = batch.grouped_members()
    # (c) the same batch with every member by its own launches
    own = mlb.Batch(sims, stream=bstream, lanes=0)
    own.step(warm)
    own.synchronize()
    e0.record(bstream)
    own.step(steps)
    e1.record(bstream)
    own.synchronize()
    ms_own = reduce_max(e0.elapsed_time(e1), dist, dev)
    own.close()
    value = units * steps * world / (ms * 1e-3) / 1e6
    seq_value = units * steps * world / t_seq / 1e6
    peak, peak_kind = measured_peak_hbm()
    design_bytes = 98 + 50 + 202                   # moments, pass 1, fused pass 2 + collide (B / species-site)
    achieved = design_bytes * units * steps / (ms * 1e-3) / 1e9
    zs = sorted({z for z, _ in tuned})
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warm,
           "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic (seeded ensemble)",
           "config": {"workload": f"ensemble of {len(systems)} independent binary systems sigma=(1,1.5), "
                                  "cubes 32^3..128^3, packing 0.05-0.20, shear 0-0.05 (Couette walls), "
                                  "5% sine wave, D3Q19, one captured CUDA graph per 2 steps",
                      "members": len(systems), "species_sites": units, "precision": "FP32 populations",
                      "l2": "inputs larger than L2", "parallelism": "replicas"},
           "roofline": {"kernel": "ensemble step (graph)", "bound": "hbm", "achieved": achieved, "peak": peak,
                        "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                        "note": f"{design_bytes} B per species-site: the three step kernels' algorithmic bytes"},
           "ensemble": {"sequential_value": seq_value, "speedup_vs_sequential": value / seq_value,
                        "grouped_members": grouped,
                        "own_launches_value": units * steps * world / (ms_own * 1e-3) / 1e6,
                        "grouping_speedup": ms_own / ms,
                        "batch_wall_value": units * steps * world / t_batch_wall / 1e6,
                        "autotuned_zchunks": zs,
                        "fused_members": sum(1 for _, f in tuned if f)},
           "gpu_launches": steps * sum(sim.launches_per_step() for sim in sims),
           "clocks": clk, "e2e": None}
    batch.close()
    for sim in sims:
        sim.close()
    if dist:
        dist.destroy_process_group()
    return out


def run_reference(args):
    """The oracle, as it stands, on the host cores: each step is one oracle
    time step of a bounded sample (96^3) of the same workload."""
    import oracle
    oracle.build()
    if args.workload == "ensemble":
        # one member's physics on a bounded 64^3 sample (the members are binary systems)
        size, kind = 64, "binary"
        sample_of = "an ensemble member (64^3 sample)"
        config = {"workload": "ensemble of independent binary systems (see the mlb arm)", "members": args.members}
    else:
        size, kind = min(args.size, {"binary": 96, "taylor": 16}.get(args.workload, 40)), args.workload
        sample_of = "x".join(str(v) for v in grid_of(args.size, args.workload))
        config = config_dict(args.size, args.workload)
    lat, n = workload(size, kind)
    f = oracle.init(lat, n)
    if args.warmup:
        oracle.step(lat, f, args.warmup)
    t0 = time.perf_counter()
    oracle.step(lat, f, args.steps)
    dt = time.perf_counter() - t0
    value = lat.nspecies * lat.nsites * args.steps / dt / 1e6
    cb = {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle", "host": host_cpu(),
          "sample": "%s lattice of the same physics per step (bounded sample of %s), FP64 C oracle"
                    % ("x".join(str(v) for v in grid_of(size, kind)), sample_of)}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded sine-wave mixture)", "config": config,
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    if args.size is None:
        args.size = DEFAULT_SIZE[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0
    if args.workload == "ensemble":
        out = run_ensemble(args, rank, world, local_rank)
    else:
        out = run_mlb(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

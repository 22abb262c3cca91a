#!/usr/bin/env python3
"""Benchmark of the DFT+U CheFSI hot path on GB300.

Metric: H.psi throughput in Gpt.orb/s (grid points x orbitals x H applications per second,
/1e9) over whole SCF iterations.  Default workload: the rutile-shaped 2x2x3 supercell
(24 Ti + 48 O, 17.36 x 17.36 x 16.78 bohr, 88x88x84 grid), 348 orbitals per spin, two spin
channels, 12th-order FD, Chebyshev degree 24, FP64.  One step = one SCF iteration through the
library's public entry point hub_scf_iterate: per spin a degree-24 filter and a Rayleigh-Ritz
projection (25 H applications), then Fermi level, occupation matrices, E_U and Pulay mixing.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f64|f32|mixed|mixed16]
        python bench.py --impl reference ...      (the CPU oracle arm)
Multi-GPU (torchrun, one rank per GPU): each rank runs an independent replica of the
workload (spin channels / snapshots are independent units): weak scaling, no collective on
the data path.  Inputs are synthetic (seeded); every orbital block is larger than L2.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PREC = {"f64": 0, "f32": 1, "mixed": 2, "mixed16": 3}
DTYPE_NAME = {"f64": "f64", "f32": "f32", "mixed": "f32+bf16", "mixed16": "f32+f16"}
# FP64 pipe of one GB300: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (max SM clock)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
# algorithmic work per point-orbital of one stencil pass (12th order, symmetric pairing):
# 3 axes x 6 pairs x (add + FMA) + centre + V_eff + the recurrence's axpby = 44 flop (the
# count the roofline fraction uses).  Counting every FMA as two flops instead (18 adds and
# 18 FMAs for the 36 neighbours, the centre and V_eff FMAs, one multiply, one FMA for
# beta * Yprev) gives 59; both are reported.
STENCIL_FLOP = 44.0
STENCIL_FLOP_FMA2 = 59.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hub", choices=["hub", "reference"])
    ap.add_argument("--prec", default="f64", choices=list(PREC))
    ap.add_argument("--workload", default="rutile", choices=["rutile", "tiny", "batched", "warm"])
    ap.add_argument("--warm-train", type=int, default=200,
                    help="warm workload: SCF solutions of displaced 12-atom cells to train on")
    ap.add_argument("--warm-f64-iters", type=int, default=2,
                    help="warm workload: FP64 iterations timed for the extrapolated cold FP64 time")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-scf-tts", action="store_true",
                    help="skip the cold-start SCF time to solution (FP64 and mixed) of the default run")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--probe-alu", action="store_true",
                    help="measure the FP64 and FP32 FMA throughput of the GPU (roofline denominators)")
    ap.add_argument("--probe-apply", type=int, default=0, metavar="NCOL",
                    help="profiling case: four H applications to NCOL random columns of the rutile "
                         "workload in --prec, then exit (no timing)")
    ap.add_argument("--projector-forms", action="store_true",
                    help="per-kernel times of a float H application on the rutile block for every "
                         "projector form and every float stencil tile shape")
    ap.add_argument("--probe-rr", type=int, default=0, metavar="NCOL",
                    help="profiling case: one filter and two Rayleigh-Ritz projections of NCOL random "
                         "columns of the rutile workload in --prec, then exit (no timing)")
    ap.add_argument("--forces", action="store_true",
                    help="time hub_hubbard_forces on the rutile workload (348 orbitals, one spin) "
                         "in --prec and report the FD-gradient kernel against the HBM roofline")
    ap.add_argument("--stress", action="store_true",
                    help="time hub_hubbard_stress on the rutile workload (348 orbitals, one spin) in --prec")
    ap.add_argument("--density-scf", action="store_true",
                    help="self-consistent density SCF (FD-Poisson Hartree, exchange, Kerker-"
                         "preconditioned Pulay on rho and D) of the workload in --prec to 1e-5 "
                         "Ha/atom: iterations, time, CG iterations per SCF iteration")
    ap.add_argument("--md-compare", type=int, default=0, metavar="STEPS",
                    help="SCF at STEPS steps of a seeded rutile 2x2x3 trajectory in --prec, starting D "
                         "atomic vs second-order extrapolated vs the occupation model (trained on "
                         "--warm-train displaced cells), previous orbitals reused: iterations per step")
    ap.add_argument("--kpoint-scf", action="store_true",
                    help="SCF of the rutile 2x2x3 cell with a k, -k pair (k = pi/L_x (1/2, 0, 0), "
                         "weights 1/2) over one handle per k-point in --prec: iterations and time")
    ap.add_argument("--scf-compare", action="store_true",
                    help="cold-start SCF to convergence in FP64, FP32 and mixed (BF16 with the "
                         "precision ladder); report time to solution and errors against FP64")
    return ap.parse_args()


def make_workload(name):
    import workloads as w
    return w.rutile() if name == "rutile" else w.tiny()


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ CPU oracle
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as w
from oracle import hubbard as o
wl = {make!s}
H = o.build_hamiltonian(wl, 0)
X = w.random_orbitals(wl.Nd, {cols}, 77).T.copy()
H.apply(X)
n, t0 = 0, time.perf_counter()
while True:
    X = H.apply(X)
    X /= np.linalg.norm(X, axis=0)
    n += 1
    if time.perf_counter() - t0 > {secs}:
        break
dt = time.perf_counter() - t0
print(json.dumps({{"applications": n, "seconds": dt, "cols": {cols}, "Nd": wl.Nd}}))
"""


def run_config(args, wl_name, wl, world):
    """The workload description shared by both arms of the bench line."""
    block = wl.Nd * wl.ncol * (8 if args.prec == "f64" else 4) / 1e9
    return {"workload": wl_name, "grid": list(wl.n), "orbitals_per_spin": wl.ncol,
            "spins": wl.nspin, "chebyshev_degree": wl.degree,
            "h_applications_per_step": wl.nspin * (wl.degree + 1),
            "step": "one SCF iteration (filter + Rayleigh-Ritz per spin, occupations, D, E_U, Pulay)",
            "l2": ("inputs larger than L2" if block > 0.129 else "inputs smaller than L2 (not flushed)")
                  + " (each orbital block %.3f GB)" % block,
            "parallelism": f"replicas x{world}"}


def host_cores():
    """Host cores this process may run on (the CPU baseline runs one oracle process per core)."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def cpu_oracle_sample(workload: str, seconds: float, cols: int = 2, procs: int = 0):
    """Time the oracle's H application on a bounded sample: `procs` independent processes
    (default: one per host core, at most 64), each single-threaded numpy on its own `cols`
    orbitals of the full grid, run side by side; the throughput is their sum.  Fresh
    interpreters (no CUDA state is inherited)."""
    make = "w.rutile()" if workload == "rutile" else "w.tiny()"
    code = CPU_SNIPPET.format(root=ROOT, make=make, cols=cols, secs=seconds)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = procs or min(64, host_cores())
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=env) for _ in range(procs)]
    outs = []
    for p in ps:
        out, err = p.communicate(timeout=600)
        if p.returncode != 0:
            raise RuntimeError("CPU oracle sample failed: " + err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    value = sum(d["Nd"] * d["cols"] * d["applications"] / d["seconds"] for d in outs) / 1e9
    d = {"applications": sum(d["applications"] for d in outs), "seconds": max(d["seconds"] for d in outs),
         "cols": cols, "Nd": outs[0]["Nd"], "procs": procs}
    return value, d


# ------------------------------------------------------------------------------ hub arm
# DRAM bytes per point-orbital of one launch (dram__bytes_read.sum + dram__bytes_write.sum of
# an ncu capture), each valid only for the kernel source the capture ran on: an entry holds
# the bytes, the source file and the first 16 hex digits of its sha256 at capture time.  A
# kernel whose source has changed since reports traffic null until it is captured again.
# Captured on the rutile 2x2x3 workload (348 orbitals, one launch = 226.4 M point-orbitals)
# with `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
# --clock-control none -k regex:"k_stencil|k_gather|k_scatter" -s 300 -c 3` (FP64) and `-c 6`
# (`--prec f32`) around `python bench.py [--prec f32] --steps 1 --warmup 1 --no-scf-tts
# --no-e2e --no-cpu-baseline`; the float gather and scatter are the tensor-core brick forms.
TRAFFIC_CAPTURES = {
    ("f64", "stencil"): (25.36, "stencil.cu", "7095f36bbcbc94c0"),
    ("f64", "gather"): (95.82, "projectors.cu", "4b61aaf339edd58a"),
    ("f64", "scatter"): (50.96, "projectors.cu", "4b61aaf339edd58a"),
    ("f32", "stencil"): (12.52, "stencil.cu", "7095f36bbcbc94c0"),
    ("f32", "gather"): (5.71, "projectors_tc.cu", "c1f826507f2e5e4b"),
    ("f32", "scatter"): (10.42, "projectors_tc.cu", "c1f826507f2e5e4b"),
}


def _source_sha16(rel_path):
    import hashlib
    p = os.path.join(ROOT, "paper_2507_23612_gb300", "csrc", rel_path)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16] if os.path.exists(p) else None


def captured_traffic(family, kernel):
    """Bytes per point-orbital of the capture of (family, kernel), or None when there is no
    capture or the kernel's source changed since it was taken."""
    cap = TRAFFIC_CAPTURES.get((family, kernel))
    if not cap:
        return None
    b, src, sha = cap
    return b if _source_sha16(src) == sha else None


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path))["hbm_gbs"], "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback 6.8 TB/s"


def kernel_roofline(name, t_n, wl, prec, function_points):
    """Roofline of one hot kernel from its summed event time and launch count (every timed
    launch processes the whole ncol-column block).  Algorithmic work per launch:
      stencil  FP64: 44 flop per point-orbital against the FP64 pipe; float: 12 B per
               point-orbital (read Y and Yprev, write Yout) against HBM
      gather   FP64: 2 flop per function-point and column against the FP64 pipe; float: one
               read of the block (4 B per point-orbital) against HBM
      scatter  FP64: as the gather; float: read and write of the block (8 B per point-orbital)"""
    t_ms, n = t_n
    per_launch_s = t_ms / n / 1e3
    pts_orb = wl.Nd * wl.ncol
    if prec == "f64":
        flops = (STENCIL_FLOP * pts_orb) if name == "stencil" else 2.0 * function_points * wl.ncol
        achieved = flops / per_launch_s / 1e12
        peak = FP64_PEAK_GFLOPS / 1e3
        traffic = captured_traffic("f64", name)
        out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
               "traffic": traffic * pts_orb if traffic else None, "traffic_unit": "DRAM bytes per launch",
               "kernel": name, "ms_per_launch": t_ms / n,
               "peak_source": "FP64 pipe: 152 SM x 2 FMA/clk x 2.07 GHz (nominal; bench.py --probe-alu measured 1.253)"}
        if name == "stencil":
            out["flop_per_point_orbital"] = STENCIL_FLOP
            out["frac_fma_as_two_flops"] = STENCIL_FLOP_FMA2 * pts_orb / per_launch_s / 1e12 / peak
        return out
    per_pt = {"stencil": 12.0, "gather": 4.0, "scatter": 8.0}[name]
    gbs = per_pt * pts_orb / per_launch_s / 1e9
    peak, src = hbm_peak()
    traffic = captured_traffic("f32", name)
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "traffic": traffic * pts_orb if traffic else None, "traffic_unit": "DRAM bytes per launch",
            "kernel": name, "ms_per_launch": t_ms / n, "peak_source": src}


# ------------------------------------------------------------------------------ ranks
def replica_spin_index(spin: int, rank: int) -> int:
    """Seed index of the starting orbitals of one spin channel on one rank: every rank is an
    independent replica with its own seeded orbitals (indices 0, 1 on rank 0; 2, 3 on rank 1 ...)."""
    return spin + 2 * rank


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over the ranks of the default process group (x itself without
    one): the job's time is the slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank_step * steps * world / seconds


def run_hub(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2507_23612_gb300 import Hub, scf_params

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    wl = make_workload(args.workload)
    nspin = wl.nspin
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=PREC[args.prec], stream=stream)
    hub.set_veff(torch.tensor(wl.veff, device=dev))
    hub.set_atoms(wl.atoms)
    dt = hub.dtype
    # each rank is an independent replica: its own seeded starting orbitals
    X0 = [wl.orbitals(replica_spin_index(s, rank)) for s in range(nspin)]
    Xs = [torch.tensor(x, device=dev).to(dt).contiguous() for x in X0]
    v0s = [torch.tensor(wl.lanczos_start(s), device=dev).to(dt).contiguous() for s in range(nspin)]
    p = scf_params(nspin=nspin, ncol=wl.ncol, ld=wl.Nd, degree=wl.degree, max_iter=1000,
                   first_passes=3 if args.workload == "rutile" else 1, lanczos_steps=10,
                   pulay_history=7, natoms=len(wl.atoms), pulay_beta=0.3,
                   kT=wl.kT if wl.kT > 0 else 0.005, n_elec=wl.n_elec, tol_e_atom=1e-5, tol_D=1e-4,
                   ladder=1 if args.prec in ("mixed", "mixed16") else 0, ladder_tol=1e-4)
    hub.scf_begin(p, Xs, v0s, wl.D0)
    for _ in range(args.warmup):
        hub.scf_iterate()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local_rank)
    sampler.start()
    hub.profile(-1)
    n0 = hub.launch_count()
    print(f"library launches before the timed region: {n0}", file=sys.stderr)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    last = None
    for _ in range(args.steps):
        last = hub.scf_iterate()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    launches = hub.launch_count() - n0
    clocks = sampler.stop()
    ms = max_over_ranks(ms, dev)
    ptorb_step = nspin * (wl.degree + 1) * wl.Nd * wl.ncol
    value = whole_job_rate(ptorb_step, args.steps, world, ms / 1e3) / 1e9

    # per-kernel breakdown: the same number of SCF iterations again, with a CUDA event pair
    # around every library launch on the library's stream (kept out of the headline loop)
    hub.profile(1)
    ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    for _ in range(args.steps):
        hub.scf_iterate()
    ep1.record(stream)
    torch.cuda.synchronize()
    ms_prof = ep0.elapsed_time(ep1)
    hub.profile(0)
    prof = hub.profile_read()
    hub.profile(-1)

    # e2e: the same step through the public API with the orbitals on the host (pinned):
    # every step copies the blocks host->device, iterates, and copies the blocks, the
    # eigenvalues and D back to the host.
    e2e = None
    if not args.no_e2e:
        hosts = [torch.empty(x.shape, dtype=dt, pin_memory=True) for x in Xs]
        for hx, x in zip(hosts, Xs):
            hx.copy_(x)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for hx, x in zip(hosts, Xs):
                x.copy_(hx, non_blocking=True)
            hub.scf_iterate()
            for hx, x in zip(hosts, Xs):
                hx.copy_(x, non_blocking=True)
            eig, occ, D = hub.scf_get()
            torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
        bx = sum(x.numel() * x.element_size() for x in Xs)
        e2e = {"value": whole_job_rate(ptorb_step, args.steps, world, t_e2e) / 1e9, "unit": "Gpt·orb/s",
               "h2d_bytes_per_step": bx,
               "d2h_bytes_per_step": bx + 8 * (eig.size + occ.size + D.size)}
    fpts = hub.projector_stats()["function_points"]
    hub.close()
    del Xs
    torch.cuda.empty_cache()

    # rooflines of the three hot kernels, and the dominant kernel's
    rooflines = {k: kernel_roofline(k, prof[k], wl, args.prec, fpts) for k in ("stencil", "gather", "scatter")
                 if k in prof}
    dom = max(prof.items(), key=lambda kv: kv[1][0]) if prof else ("none", (0.0, 0))
    roof = rooflines.get(dom[0])
    breakdown = {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / ms_prof, 4)}
                 for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}

    # the metric's second half: cold-start SCF time to solution at 1e-5 Ha/atom, FP64 and the
    # mixed form (BF16 tensor-core products with the precision ladder), on fresh handles, and
    # the float kernels' rooflines from two profiled iterations of the converged mixed SCF
    tts = None
    if not args.no_scf_tts and args.workload == "rutile" and world == 1:
        tts = scf_time_to_solution(wl, X0, dev)
    return {"value": value, "ms": ms, "launches": launches, "e2e": e2e, "tts": tts,
            "roofline": roof, "rooflines": rooflines, "kernels": breakdown, "clocks": clocks, "last": last,
            "wl": wl, "profiled_ms": ms_prof}


def scf_solve_timed(wl, X0, dev, prec, profile_after=0, ladder=None):
    """Cold-start SCF of the workload in one precision form on a fresh handle, timed from
    handle creation to convergence; optionally profile_after more iterations with per-kernel
    events.  Returns the result, the per-kernel profile and the projector function points.
    ladder: the mixed forms' precision ladder (default on for them; 0 = three-term 16-bit
    products throughout)."""
    import numpy as np
    import torch
    from paper_2507_23612_gb300 import Hub, scf_params
    # the starting orbitals in the form's element type, prepared before the clock starts
    # (uploaded inside the timed region)
    X0h = [np.ascontiguousarray(x, dtype=np.float64 if prec == "f64" else np.float32) for x in X0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=PREC[prec])
    hub.set_veff(torch.tensor(wl.veff, device=dev))
    hub.set_atoms(wl.atoms)
    Xs = [torch.from_numpy(x).to(dev) for x in X0h]
    v0s = [torch.tensor(wl.lanczos_start(s), device=dev).to(hub.dtype).contiguous() for s in range(wl.nspin)]
    p = scf_params(nspin=wl.nspin, ncol=wl.ncol, ld=wl.Nd, degree=wl.degree, max_iter=200,
                   first_passes=3, lanczos_steps=10, pulay_history=7, natoms=len(wl.atoms),
                   pulay_beta=0.3, kT=wl.kT if wl.kT > 0 else 0.005, n_elec=wl.n_elec,
                   tol_e_atom=1e-5, tol_D=1e-4,
                   ladder=(1 if prec in ("mixed", "mixed16") else 0) if ladder is None else ladder,
                   ladder_tol=1e-4)
    hub.scf_begin(p, Xs, v0s, wl.D0)
    res = hub.scf_run()
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    eig, occ, D = hub.scf_get()
    prof, fpts = None, None
    if profile_after:
        hub.profile(-1)
        hub.profile(1)
        for _ in range(profile_after):
            hub.scf_iterate()
        torch.cuda.synchronize()
        hub.profile(0)
        prof = hub.profile_read()
        fpts = hub.projector_stats()["function_points"]
    hub.close()
    del Xs
    torch.cuda.empty_cache()
    return {"seconds": seconds, "iterations": res["iter"], "converged": bool(res["converged"]),
            "E": res["E"], "E_U": res["E_U"], "band": float(np.sum(occ * eig)), "D": D}, prof, fpts


def scf_time_to_solution(wl, X0, dev):
    import numpy as np
    nat = len(wl.atoms)
    f64, _, _ = scf_solve_timed(wl, X0, dev, "f64")
    mixed, prof, fpts = scf_solve_timed(wl, X0, dev, "mixed", profile_after=2)
    mixed16, _, _ = scf_solve_timed(wl, X0, dev, "mixed16")

    def errors(r):
        return {"E_Ha_per_atom": abs(r["E"] - f64["E"]) / nat, "E_U_Ha_per_atom": abs(r["E_U"] - f64["E_U"]) / nat,
                "band_Ha_per_atom": abs(r["band"] - f64["band"]) / nat,
                "max_abs_dD": float(np.max(np.abs(r["D"] - f64["D"])))}
    out = {"criterion": "|dE|/atom < 1e-5 Ha twice and max|dD| < 1e-4; wall clock from handle creation",
           "f64": {"seconds": round(f64["seconds"], 3), "iterations": f64["iterations"],
                   "converged": f64["converged"], "E_Ha": f64["E"], "E_U_Ha": f64["E_U"]},
           "mixed": {"seconds": round(mixed["seconds"], 3), "iterations": mixed["iterations"],
                     "converged": mixed["converged"], "E_Ha": mixed["E"], "E_U_Ha": mixed["E_U"],
                     "error_vs_f64": errors(mixed)},
           "mixed_f16": {"seconds": round(mixed16["seconds"], 3), "iterations": mixed16["iterations"],
                         "converged": mixed16["converged"], "E_Ha": mixed16["E"], "E_U_Ha": mixed16["E_U"],
                         "error_vs_f64": errors(mixed16)},
           "speedup_mixed_vs_f64": round(f64["seconds"] / mixed["seconds"], 2),
           "speedup_mixed_f16_vs_f64": round(f64["seconds"] / mixed16["seconds"], 2)}
    if prof:
        out["mixed_rooflines"] = {k: kernel_roofline(k, prof[k], wl, "mixed", fpts)
                                  for k in ("stencil", "gather", "scatter") if k in prof}
    return out


def scf_compare(args):
    """Cold-start SCF of the workload in each precision form; errors against the FP64 run."""
    import numpy as np
    import torch
    from paper_2507_23612_gb300 import Hub, scf_params
    dev = torch.device("cuda", 0)
    wl = make_workload(args.workload)
    X0 = [wl.orbitals(s) for s in range(wl.nspin)]
    out = {}
    for form in ("f64", "f32", "mixed", "mixed16"):
        out[form], _, _ = scf_solve_timed(wl, X0, dev, form)
    nat = len(wl.atoms)
    ref = out["f64"]
    table = {}
    for form, r in out.items():
        table[form] = {"time_to_solution_s": round(r["seconds"], 3), "iterations": r["iterations"],
                       "converged": r["converged"], "speedup_vs_f64": round(ref["seconds"] / r["seconds"], 2),
                       "E_err_Ha_per_atom": abs(r["E"] - ref["E"]) / nat,
                       "E_U_err_Ha_per_atom": abs(r["E_U"] - ref["E_U"]) / nat,
                       "band_err_Ha_per_atom": abs(r["band"] - ref["band"]) / nat,
                       "max_abs_dD": float(np.max(np.abs(r["D"] - ref["D"])))}
    print(json.dumps({"scf_compare": table, "workload": args.workload,
                      "criterion": "|dE|/atom < 1e-5 Ha twice and max|dD| < 1e-4",
                      "E_f64_Ha": ref["E"], "E_U_f64_Ha": ref["E_U"]}))
    return 0


def run_warm(args):
    """Warm start of the 3x3x4 rutile-shaped supercell (216 atoms, 72 Ti, 132x132x112 grid,
    1044 orbitals per spin, two spins), mixed form with the precision ladder.

    The occupation model (descriptors -> 3x256 SiLU MLP with FP16 weights -> 15 D entries
    per spin) is trained on --warm-train SCF solutions that the library computes (float) for
    seeded displaced 12-atom cells (the descriptors see 6 bohr around an atom, so small cells
    give the local environments cheaply).  Two consecutive steps of a seeded MD trajectory of
    the 216-atom cell are then solved: step 0 cold (random orbitals, atomic-guess D), step 1
    from step 0's converged orbitals with the atomic-guess D (the method without the model)
    and with the model's D.  The cold FP64 time of step 0 is extrapolated from timed FP64
    iterations and the mixed run's iteration count."""
    import numpy as np
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import HUB_F32, HUB_F64, HUB_MIXED_BF16, Hub, scf_params
    from paper_2507_23612_gb300.warmstart import OccupationModel, scf_solve
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    model = OccupationModel(nspin=2, seed=0)
    gen = []
    for i in range(args.warm_train):
        wl = w.rutile_snapshot((1, 1, 2), 0.1, seed=i)
        r = scf_solve(wl, HUB_F32, tol_e_atom=1e-6, tol_D=1e-5)
        model.add_solution(wl.atoms, wl.L, r["D"])
        gen.append((r["iterations"], r["seconds"]))
    t_gen = time.perf_counter() - t0
    t1 = time.perf_counter()
    losses = model.fit(steps=3000)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t1

    steps = w.rutile_trajectory((3, 3, 4), nsteps=2, amplitude=0.1, period=12.0)
    s0, s1 = steps
    nat = len(s0.atoms)
    cold = scf_solve(s0, HUB_MIXED_BF16, keep_orbitals=True)
    X0 = [x.clone() for x in cold["X"]]
    del cold["X"]
    torch.cuda.empty_cache()
    t2 = time.perf_counter()
    D_pred = model.predict(s1.atoms, s1.L)
    t_pred = time.perf_counter() - t2
    atomic = scf_solve(s1, HUB_MIXED_BF16, X0=[x.clone() for x in X0])
    torch.cuda.empty_cache()
    warm = scf_solve(s1, HUB_MIXED_BF16, D0=D_pred, X0=[x.clone() for x in X0])
    del X0
    torch.cuda.empty_cache()

    # cold FP64 of step 0: the first iteration (first passes) and the following ones timed,
    # then extrapolated with the cold mixed run's iteration count
    f64 = None
    if args.warm_f64_iters > 0:
        hub = Hub(s0.n, s0.L, s0.fd_half_order, prec=HUB_F64)
        hub.set_veff(torch.tensor(s0.veff, device=dev))
        hub.set_atoms(s0.atoms)
        Xs = [torch.tensor(s0.orbitals(s), device=dev).contiguous() for s in range(s0.nspin)]
        v0s = [torch.tensor(s0.lanczos_start(s), device=dev).contiguous() for s in range(s0.nspin)]
        p = scf_params(nspin=2, ncol=s0.ncol, ld=s0.Nd, degree=s0.degree, max_iter=200, first_passes=3,
                       lanczos_steps=10, pulay_history=7, natoms=nat, pulay_beta=0.3, kT=s0.kT,
                       n_elec=s0.n_elec, tol_e_atom=1e-5, tol_D=1e-4)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        hub.scf_begin(p, Xs, v0s, s0.D0)
        times = []
        for _ in range(args.warm_f64_iters):
            hub.scf_iterate()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - ts)
            ts = time.perf_counter()
        hub.close()
        del Xs, v0s
        torch.cuda.empty_cache()
        later = float(np.mean(times[1:])) if len(times) > 1 else times[0] / 3
        est = times[0] + (cold["iterations"] - 1) * later
        f64 = {"first_iteration_s": round(times[0], 3), "later_iteration_s": round(later, 3),
               "time_to_solution_s_extrapolated": round(est, 2),
               "extrapolation": "first FP64 iteration + (cold mixed iteration count - 1) x timed later FP64 iteration"}
    err0 = float(np.max(np.abs(s1.D0 - atomic["D"])))
    errp = float(np.max(np.abs(D_pred - atomic["D"])))
    line = {
        "metric": "SCF time to solution at 1e-5 Ha/atom (warm start, MD step)",
        "value": round(warm["seconds"], 3), "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "dtype": "f32+bf16 (FP64 dense steps)", "data": "synthetic",
        "config": {"workload": s0.name, "grid": list(s0.n), "orbitals_per_spin": s0.ncol, "spins": 2,
                   "atoms": nat, "hubbard_atoms": D_pred.shape[1], "chebyshev_degree": s0.degree,
                   "trajectory": "seeded sinusoidal displacements, 0.1 bohr, period 12 steps; steps 0 and 1",
                   "criterion": "|dE|/atom < 1e-5 Ha twice and max|dD| < 1e-4",
                   "model": "descriptors(48) -> 3x256 SiLU -> 30, FP16 weights, FP32 accumulate"},
        "training": {"scf_solutions": args.warm_train, "cells": "displaced 1x1x2 rutile (12 atoms, 4 Ti), float",
                     "samples": model.n_samples, "generation_s": round(t_gen, 2),
                     "scf_iterations_mean": float(np.mean([g[0] for g in gen])) if gen else None,
                     "fit_s": round(t_fit, 3), "adam_steps": 3000,
                     "loss_first_last": [losses[0], losses[-1]], "predict_s": round(t_pred, 4)},
        "step0_cold_mixed": {"iterations": cold["iterations"], "seconds": round(cold["seconds"], 3),
                             "E_Ha": cold["E"], "converged": cold["converged"]},
        "step1_atomic_D_reused_orbitals": {"iterations": atomic["iterations"], "seconds": round(atomic["seconds"], 3),
                                           "E_Ha": atomic["E"], "converged": atomic["converged"]},
        "step1_model_D_reused_orbitals": {"iterations": warm["iterations"], "seconds": round(warm["seconds"], 3),
                                          "E_Ha": warm["E"], "converged": warm["converged"]},
        "fixed_point_step1": {"dE_Ha_per_atom": abs(warm["E"] - atomic["E"]) / nat,
                              "max_abs_dD": float(np.max(np.abs(warm["D"] - atomic["D"])))},
        "initial_D_error_step1": {"atomic_guess": err0, "model": errp},
        "cold_f64_step0": f64,
    }
    if f64:
        line["speedup_warm_mixed_vs_cold_f64"] = round(f64["time_to_solution_s_extrapolated"] / warm["seconds"], 2)
    line["speedup_model_vs_atomic_D"] = round(atomic["seconds"] / warm["seconds"], 2)
    print(json.dumps(line))
    return 0


def run_batched(args):
    """16 perturbed rutile / anatase snapshots of 24-96 atoms with 1-4 k-points each (complex
    float orbitals), all filtered (degree 24) in one graph; against the same systems filtered
    one after another without the graph."""
    import numpy as np
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import Hub, HUB_F32, batch_filter
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    snaps = w.snapshot_batch()
    hubs, Xs, bounds, work = [], [], [], 0.0
    t0 = time.perf_counter()
    for sn in snaps:
        for k, kpt in enumerate(sn.kpts):
            hb = Hub(sn.n, sn.L, sn.fd_half_order, kpt=kpt, complex_=True, prec=HUB_F32)
            hb.set_veff(torch.tensor(sn.veff, device=dev))
            hb.set_atoms(sn.atoms)
            hb.set_occupation_matrix(0, sn.D0[0])
            X = torch.randn(sn.ncol, sn.Nd, dtype=torch.complex64, device=dev, generator=gen)
            v0 = torch.randn(sn.Nd, dtype=torch.complex64, device=dev, generator=gen)
            lo, up = hb.lanczos_bound(0, 10, v0)
            hubs.append(hb)
            Xs.append(X)
            bounds.append((lo + 0.1 * (up - lo), up, lo))
            work += sn.Nd * sn.ncol * sn.degree
    setup_s = time.perf_counter() - t0
    a = [bb[0] for bb in bounds]
    b = [bb[1] for bb in bounds]
    al = [bb[2] for bb in bounds]
    degree = snaps[0].degree
    t0 = time.perf_counter()
    try:
        batch_filter(hubs, [0] * len(hubs), Xs, degree, a, b, al)    # tune + capture + first run
    except Exception:
        free, total = torch.cuda.mem_get_info()
        print(f"device memory free {free / 1e9:.1f} of {total / 1e9:.1f} GB; torch holds "
              f"{torch.cuda.memory_allocated() / 1e9:.1f} GB", file=sys.stderr)
        raise
    first_s = time.perf_counter() - t0
    for _ in range(max(1, args.warmup)):
        batch_filter(hubs, [0] * len(hubs), Xs, degree, a, b, al)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for _ in range(args.steps):
        batch_filter(hubs, [0] * len(hubs), Xs, degree, a, b, al)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1) / args.steps
    # the same work, one system after another, no graph
    e0.record(stream)
    for hb, X, bb in zip(hubs, Xs, bounds):
        hb.chefsi_filter(0, X, degree, bb[0], bb[1], bb[2])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    grids = sorted(set(sn.n for sn in snaps), key=lambda n: n[0] * n[1] * n[2])
    small = batched_small(args, dev, gen)
    variants = [hb.autotune(0, X) for hb, X in zip(hubs, Xs)][:8]
    for hb in hubs:
        hb.close()
    del Xs
    torch.cuda.empty_cache()
    scf_tts = batched_scf_tts(dev)
    print(json.dumps({
        "metric": "H·psi throughput, batched filter", "value": work / (ms_graph / 1e3) / 1e9,
        "unit": "Gpt·orb/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": "16 snapshots (rutile/anatase, 24-96 atoms, N(0,0.1 bohr)), 1-4 k-points, "
                               "complex float, degree 24", "systems": len(hubs),
                   "grids_min_max": [list(grids[0]), list(grids[-1])], "step": "one hub_batch_filter call"},
        "sequential_no_graph": {"ms": ms_seq, "value": work / (ms_seq / 1e3) / 1e9},
        "graph_speedup": ms_seq / ms_graph, "first_call_s": first_s, "setup_s": setup_s,
        "stencil_variants": variants,
        "small_systems": small, "scf_time_to_solution": scf_tts}))
    return 0


def batched_scf_tts(dev):
    """SCF time to solution of the batched form: k-point SCFs of four snapshot cells (24 and
    36 atoms, 1-3 Monkhorst-Pack k-points, complex orbitals, 8 channels) to 1e-5 Ha/atom,
    (a) float, all cells batched (per filter pass one CUDA graph over every channel,
    hub_kscf_run_batch), (b) float, one cell after another (hub_kscf_run), (c) FP64, one
    after another; and a launch-bound case, the 24^3 tiny cell with 8 k-points, batched and
    not.  Wall clock from handle creation to convergence."""
    import numpy as np
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import HUB_F32, HUB_F64
    from paper_2507_23612_gb300.kpoint_scf import KpointSCF, run_batched

    def cells():
        snaps = w.snapshot_batch()
        return [snaps[i] for i in (0, 1, 5, 6)]

    def tiny_k8():
        wl = w.tiny()
        kf = [((i % 2) / 4.0 + 0.125, ((i // 2) % 2) / 4.0 + 0.125, (i // 4) / 4.0 + 0.125) for i in range(8)]
        wl.kpts = tuple(tuple(2 * np.pi * np.asarray(f) / np.asarray(wl.L)) for f in kf)
        wl.kweights = tuple([1.0 / 8] * 8)
        return [wl]

    def solve(wls, prec, batched):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        scfs = []
        try:
            for wl in wls:
                scf = KpointSCF(wl, wl.kpts, wl.kweights, prec, device=dev)
                scfs.append(scf)
                dt = scf.hubs[0].dtype
                X0 = [[torch.tensor(wl.orbitals(0, k, complex_=True), device=dev).to(dt).contiguous()
                       for k in range(len(wl.kpts))]]
                v0 = [[torch.tensor(wl.lanczos_start(0, k, complex_=True), device=dev).to(dt).contiguous()
                       for k in range(len(wl.kpts))]]
                kw = dict(n_elec=wl.n_elec, kT=wl.kT if wl.kT > 0 else 0.005, degree=wl.degree, max_iter=200,
                          tol_e_atom=1e-5, tol_D=1e-4)
                if batched:
                    scf.begin(X0, v0, wl.D0, **kw)
                else:
                    scf.res = scf.run(X0, v0, wl.D0, **kw)
            res = run_batched(scfs) if batched else [s.res for s in scfs]
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
        finally:
            for scf in scfs:
                scf.close()
        return {"seconds": round(sec, 3), "iterations": [r["iterations"] for r in res],
                "converged": all(r["converged"] for r in res), "E_Ha": [r["E"] for r in res]}

    out = {}
    wls = cells()
    out["cells"] = [f"{wl.name} ({len(wl.kpts)} k)" for wl in wls]
    out["f32_batched"] = solve(wls, HUB_F32, True)
    out["f32_one_by_one"] = solve(wls, HUB_F32, False)
    out["f64_one_by_one"] = solve(wls, HUB_F64, False)
    nat = [len(wl.atoms) for wl in wls]
    out["max_dE_f32_batched_vs_f64_Ha_per_atom"] = max(abs(a - b) / n for a, b, n in zip(
        out["f32_batched"]["E_Ha"], out["f64_one_by_one"]["E_Ha"], nat))
    out["speedup_batched_vs_f64"] = round(out["f64_one_by_one"]["seconds"] / out["f32_batched"]["seconds"], 2)
    out["speedup_batched_vs_f32_one_by_one"] = round(out["f32_one_by_one"]["seconds"] / out["f32_batched"]["seconds"], 2)
    tk = tiny_k8()
    out["tiny_8k"] = {"f32_batched": solve(tk, HUB_F32, True), "f32_one_by_one": solve(tk, HUB_F32, False)}
    out["tiny_8k"]["speedup"] = round(out["tiny_8k"]["f32_one_by_one"]["seconds"] /
                                      out["tiny_8k"]["f32_batched"]["seconds"], 2)
    return out


def batched_small(args, dev, gen):
    """Launch-bound case: 32 Bloch wavevectors of the 24^3 tiny cell (32 complex orbitals
    each), filtered in one graph and one after another."""
    import numpy as np
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import Hub, HUB_F32, batch_filter
    wl = w.tiny()
    hubs, Xs, a, b, al = [], [], [], [], []
    for i in range(32):
        kf = np.array([(i % 4) / 8.0, ((i // 4) % 4) / 8.0, (i // 16) / 8.0]) + 0.01
        kpt = 2 * np.pi * kf / np.asarray(wl.L)
        hb = Hub(wl.n, wl.L, wl.fd_half_order, kpt=tuple(kpt), complex_=True, prec=HUB_F32)
        hb.set_veff(torch.tensor(wl.veff, device=dev))
        hb.set_atoms(wl.atoms)
        hb.set_occupation_matrix(0, wl.D0[0])
        X = torch.randn(wl.ncol, wl.Nd, dtype=torch.complex64, device=dev, generator=gen)
        v0 = torch.randn(wl.Nd, dtype=torch.complex64, device=dev, generator=gen)
        lo, up = hb.lanczos_bound(0, 10, v0)
        hubs.append(hb); Xs.append(X); a.append(lo + 0.1 * (up - lo)); b.append(up); al.append(lo)
    work = 32 * wl.Nd * wl.ncol * wl.degree
    batch_filter(hubs, [0] * 32, Xs, wl.degree, a, b, al)
    batch_filter(hubs, [0] * 32, Xs, wl.degree, a, b, al)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        batch_filter(hubs, [0] * 32, Xs, wl.degree, a, b, al)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_g = e0.elapsed_time(e1) / 5
    e0.record(stream)
    for hb, X, x1, x2, x3 in zip(hubs, Xs, a, b, al):
        hb.chefsi_filter(0, X, wl.degree, x1, x2, x3)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    return {"systems": 32, "grid": list(wl.n), "orbitals": wl.ncol, "degree": wl.degree,
            "graph_ms": ms_g, "sequential_ms": ms_s, "graph_speedup": ms_s / ms_g,
            "graph_value": work / (ms_g / 1e3) / 1e9}


def probe_apply(args):
    """A small case for ncu captures of the hot kernels: the rutile handle, four hub_apply_H
    calls on a seeded random block of args.probe_apply columns (larger than L2 from 64 on)."""
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import Hub
    wl = w.rutile()
    dev = torch.device("cuda", 0)
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=PREC[args.prec])
    hub.set_veff(torch.tensor(wl.veff, device=dev))
    hub.set_atoms(wl.atoms)
    hub.set_occupation_matrix(0, wl.D0[0])
    g = torch.Generator(device=dev).manual_seed(5)
    X = torch.randn(args.probe_apply, wl.Nd, device=dev, dtype=torch.float64, generator=g).to(hub.dtype).contiguous()
    Y = torch.empty_like(X)
    for _ in range(4):
        hub.apply_H(0, X, Y)
    torch.cuda.synchronize()
    print(json.dumps({"probe": "apply_H", "columns": args.probe_apply, "prec": args.prec,
                      "max_abs": float(Y.abs().max())}))
    hub.close()
    return 0


def run_projector_forms(args):
    """Per-kernel times of one float H application on the rutile block (348 random orbitals)
    for every projector form (point-major, bricks on CUDA cores, tensor-core brick gather,
    tensor-core gather and scatter) and every float stencil tile shape: 3 warm-up and 10
    timed applications per setting, CUDA events around every launch on the library's
    stream.  Also checks that every stencil tile shape gives the same bits."""
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import Hub, HUB_F32
    wl = w.rutile()
    dev = torch.device("cuda", 0)
    hb = Hub(wl.n, wl.L, wl.fd_half_order, prec=HUB_F32)
    hb.set_veff(torch.tensor(wl.veff, device=dev))
    hb.set_atoms(wl.atoms)
    hb.set_occupation_matrix(0, wl.D0[0])
    g = torch.Generator(device=dev).manual_seed(3)
    X = torch.randn(wl.ncol, wl.Nd, device=dev, generator=g, dtype=torch.float32)
    Y = torch.empty_like(X)
    pts = wl.Nd * wl.ncol

    def timed():
        for _ in range(3):
            hb.apply_H(0, X, Y)
        torch.cuda.synchronize()
        hb.profile(-1)
        hb.profile(1)
        for _ in range(10):
            hb.apply_H(0, X, Y)
        torch.cuda.synchronize()
        hb.profile(0)
        p = hb.profile_read()
        hb.profile(-1)
        # per application (transform: the reduction and coefficient kernels of one gather)
        return {k: round(v[0] / 10, 4) for k, v in p.items() if k in ("stencil", "gather", "transform", "scatter")}

    forms = {}
    for form, name in ((0, "point-major"), (1, "bricks, CUDA cores"), (2, "tensor-core gather"),
                       (3, "tensor-core gather and scatter")):
        try:
            hb.set_tuning(gather_form=form)
        except Exception as e:          # tables not available on this grid
            forms[name] = str(e)
            continue
        t = timed()
        t["projector_ms"] = round(t.get("gather", 0) + t.get("transform", 0) + t.get("scatter", 0), 4)
        forms[name] = t
    hb.set_tuning(gather_form=3)
    stencil = {}
    ref = None
    for v in range(hb.get_tuning()["n_variants"]):
        hb.set_tuning(stencil_variant=v)
        t = timed()
        if ref is None:
            ref = Y.clone()
        ms = t["stencil"]
        stencil[v] = {"ms": ms, "GBs": round(12.0 * pts / (ms * 1e-3) / 1e9, 1),
                      "frac_of_hbm": round(12.0 * pts / (ms * 1e-3) / 1e9 / hbm_peak()[0], 4),
                      "same_bits_as_variant_0": bool(torch.equal(Y, ref))}
    print(json.dumps({"projector_forms_ms_per_application": forms, "float_stencil_variants": stencil,
                      "workload": "rutile-2x2x3 88x88x84, 348 random orbitals, float", "point_orbitals": pts}))
    hb.close()
    return 0


def probe_rr(args):
    """A small case for ncu captures of the Rayleigh-Ritz products: the rutile handle in
    --prec, one degree-8 filter (so that the block's Gram matrix is well conditioned enough
    for the mixed form) and two hub_rayleigh_ritz calls on a seeded random block of
    args.probe_rr columns."""
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import Hub
    wl = w.rutile()
    dev = torch.device("cuda", 0)
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=PREC[args.prec])
    hub.set_veff(torch.tensor(wl.veff, device=dev))
    hub.set_atoms(wl.atoms)
    hub.set_occupation_matrix(0, wl.D0[0])
    g = torch.Generator(device=dev).manual_seed(5)
    X = torch.randn(args.probe_rr, wl.Nd, device=dev, dtype=torch.float64, generator=g).to(hub.dtype).contiguous()
    v0 = torch.randn(wl.Nd, device=dev, dtype=torch.float64, generator=g).to(hub.dtype).contiguous()
    lo, up = hub.lanczos_bound(0, 10, v0)
    hub.chefsi_filter(0, X, 8, lo + 0.1 * (up - lo), up, lo)
    eig = None
    for _ in range(2):
        eig = hub.rayleigh_ritz(0, X)
    torch.cuda.synchronize()
    print(json.dumps({"probe": "rayleigh_ritz", "columns": args.probe_rr, "prec": args.prec,
                      "eig_min_max": [float(eig[0]), float(eig[-1])]}))
    hub.close()
    return 0


def run_forces(args):
    """Hubbard forces of one (spin, k) block of the rutile workload: three FD gradients of
    the 348-orbital block, four projector gathers and the per-atom reductions per call.
    The gradient kernel reads X and writes d_a X once each (16 B per point-orbital in FP64,
    8 B in float), so its roofline is HBM.  Times with CUDA events on the library's stream."""
    import math
    import numpy as np
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import Hub
    wl = w.rutile()
    dev = torch.device("cuda", 0)
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=PREC[args.prec])
    hub.set_veff(torch.tensor(wl.veff, device=dev))
    hub.set_atoms(wl.atoms)
    hub.set_occupation_matrix(0, wl.D0[0])
    g = torch.Generator(device=dev).manual_seed(5)
    X = torch.randn(wl.ncol, wl.Nd, device=dev, dtype=torch.float64, generator=g).to(hub.dtype).contiguous()
    X /= (X.double().norm(dim=1, keepdim=True) * math.sqrt(wl.dV)).to(X.dtype)
    f = np.linspace(1.0, 0.0, wl.ncol)
    work = torch.empty_like(X)
    for _ in range(max(args.warmup, 1)):
        F = hub.hubbard_forces(0, X, f, 1.0, work=work)
    torch.cuda.synchronize()
    hub.profile(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        F = hub.hubbard_forces(0, X, f, 1.0, work=work)
    wall_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    prof = hub.profile_read()
    hub.profile(0)
    grad_ms, grad_n = prof.get("force", (0.0, 0))
    per_launch = grad_ms / max(grad_n, 1)
    bytes_per = (16 if hub.dtype == torch.float64 else 8) * wl.Nd * wl.ncol
    peak = hbm_peak()[0]
    achieved = bytes_per / (per_launch * 1e-3) / 1e9 if per_launch > 0 else None
    print(json.dumps({"probe": "hubbard_forces", "prec": args.prec, "grid": list(wl.n),
                      "orbitals": wl.ncol, "hubbard_atoms": hub.nhub, "ms_per_call": wall_ms,
                      "gradient": {"ms_per_launch": per_launch, "launches": grad_n,
                                   "achieved_gbs": achieved, "peak_gbs": peak,
                                   "frac": achieved / peak if achieved and peak else None},
                      "kernels": {k: v for k, v in prof.items() if v[1]},
                      "max_abs_force": float(np.max(np.abs(F)))}))
    hub.close()
    return 0


def run_stress(args):
    """Hubbard stress of one (spin, k) block of the rutile workload: three FD gradients,
    one projector gather, three moment gathers (the orbitals re-evaluated about each image
    centre for the 24 Hubbard Ti) and nine per-atom reductions per call."""
    import math
    import numpy as np
    import torch
    import workloads as w
    from paper_2507_23612_gb300 import Hub
    wl = w.rutile()
    dev = torch.device("cuda", 0)
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=PREC[args.prec])
    hub.set_veff(torch.tensor(wl.veff, device=dev))
    hub.set_atoms(wl.atoms)
    hub.set_occupation_matrix(0, wl.D0[0])
    g = torch.Generator(device=dev).manual_seed(5)
    X = torch.randn(wl.ncol, wl.Nd, device=dev, dtype=torch.float64, generator=g).to(hub.dtype).contiguous()
    X /= (X.double().norm(dim=1, keepdim=True) * math.sqrt(wl.dV)).to(X.dtype)
    f = np.linspace(1.0, 0.0, wl.ncol)
    work = torch.empty_like(X)
    sig = hub.hubbard_stress(0, X, f, 1.0, work=work)
    torch.cuda.synchronize()
    hub.profile(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sig = hub.hubbard_stress(0, X, f, 1.0, work=work)
    wall_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    prof = hub.profile_read()
    hub.profile(0)
    print(json.dumps({"probe": "hubbard_stress", "prec": args.prec, "grid": list(wl.n),
                      "orbitals": wl.ncol, "hubbard_atoms": hub.nhub, "ms_per_call": wall_ms,
                      "kernels": {k: v for k, v in prof.items() if v[1]},
                      "sigma_Ha_per_bohr3": sig.tolist()}))
    hub.close()
    return 0


def run_density_scf(args):
    """Cold-start self-consistent density SCF of the workload (uniform starting density,
    atomic-guess D) in --prec, to |dE|/atom < 1e-5 Ha twice, max|dD| < 1e-4 and
    int|rho_out - rho_in| / N_e < 1e-4."""
    import torch
    from paper_2507_23612_gb300 import Hub, scf_params
    dev = torch.device("cuda", 0)
    wl = make_workload(args.workload)
    hub = Hub(wl.n, wl.L, wl.fd_half_order, prec=PREC[args.prec])
    hub.set_veff(torch.tensor(wl.veff, device=dev))
    hub.set_atoms(wl.atoms)
    Xs = [torch.tensor(wl.orbitals(s), device=dev).to(hub.dtype).contiguous() for s in range(wl.nspin)]
    v0s = [torch.tensor(wl.lanczos_start(s), device=dev).to(hub.dtype).contiguous() for s in range(wl.nspin)]
    p = scf_params(nspin=wl.nspin, ncol=wl.ncol, ld=wl.Nd, degree=wl.degree, max_iter=200,
                   first_passes=3, lanczos_steps=10, pulay_history=7, natoms=len(wl.atoms),
                   pulay_beta=0.3, kT=wl.kT if wl.kT > 0 else 0.005, n_elec=wl.n_elec,
                   tol_e_atom=1e-5, tol_D=1e-4, ladder=1 if args.prec in ("mixed", "mixed16") else 0, ladder_tol=1e-4,
                   density=1, kerker_kappa=0.5, tol_rho=1e-4, cg_tol=1e-10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hub.scf_begin(p, Xs, v0s, wl.D0)
    hist = []
    while True:
        r = hub.scf_iterate()
        hist.append({"E": r["E"], "dE": r["dE"], "dD": r["dD"], "drho": r["drho"], "cg_iters": r["cg_iters"]})
        if r["converged"] or r["iter"] >= p.max_iter:
            break
    torch.cuda.synchronize()
    tts = time.perf_counter() - t0
    print(json.dumps({"density_scf": {"workload": args.workload, "prec": args.prec,
                                      "time_to_solution_s": tts, "iterations": r["iter"],
                                      "converged": bool(r["converged"]), "E_Ha": r["E"],
                                      "E_H_Ha": r["E_H"], "E_x_Ha": r["E_x"], "E_U_Ha": r["E_U"],
                                      "cg_iters_per_iteration": [h["cg_iters"] for h in hist],
                                      "drho": [h["drho"] for h in hist]}}))
    hub.close()
    return 0


def run_md_compare(args):
    """Iterations per MD step with the atomic and the extrapolated starting D."""
    import workloads as w
    from paper_2507_23612_gb300.md import trajectory_scf
    from paper_2507_23612_gb300.warmstart import OccupationModel, scf_solve
    steps = w.rutile_trajectory((2, 2, 3), nsteps=args.md_compare, amplitude=0.1, period=12.0)
    # the occupation model, trained on SCF solutions of displaced 12-atom cells off the trajectory
    from paper_2507_23612_gb300 import HUB_F32
    model = OccupationModel(nspin=steps[0].nspin, seed=0)
    for i in range(args.warm_train):
        snap = w.rutile_snapshot((1, 1, 2), 0.1, seed=500 + i)
        model.add_solution(snap.atoms, snap.L, scf_solve(snap, HUB_F32, tol_e_atom=1e-6, tol_D=1e-5)["D"])
    model.fit(steps=3000)
    out = {}
    for start in ("atomic", "extrapolated", "mlp"):
        res = trajectory_scf(steps, PREC[args.prec], start=start, model=model)
        out[start] = {"iterations": [r["iterations"] for r in res],
                      "seconds": [round(r["seconds"], 3) for r in res],
                      "E": [r["E"] for r in res], "alpha_beta": [r["alpha_beta"] for r in res]}
    print(json.dumps({"md_compare": out, "prec": args.prec, "steps": args.md_compare,
                      "trajectory": "rutile 2x2x3, sinusoidal displacements (0.1 bohr, period 12 steps)"}))
    return 0


def run_kpoint_scf(args):
    """Brillouin-zone sampling: the SCF of the rutile cell over a time-reversal pair of
    Bloch vectors (complex orbitals, real D), to 1e-5 Ha/atom."""
    import math
    import numpy as np
    import torch
    import workloads as w
    from paper_2507_23612_gb300.kpoint_scf import KpointSCF
    wl = w.rutile()
    kx = 0.5 * math.pi / wl.L[0]
    kpts = [(kx, 0.0, 0.0), (-kx, 0.0, 0.0)]
    scf = KpointSCF(wl, kpts, [0.5, 0.5], PREC[args.prec])
    try:
        dev = torch.device("cuda", 0)
        X0 = [[torch.tensor(wl.orbitals(s, complex_=True), device=dev).to(scf.hubs[0].dtype).contiguous()
               for _ in kpts] for s in range(wl.nspin)]
        v0 = [[torch.tensor(wl.lanczos_start(s, complex_=True), device=dev).to(scf.hubs[0].dtype).contiguous()
               for _ in kpts] for s in range(wl.nspin)]
        for s in range(wl.nspin):                 # -k starts from the conjugate of +k
            X0[s][1] = X0[s][0].conj().resolve_conj().contiguous()
            v0[s][1] = v0[s][0].conj().resolve_conj().contiguous()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = scf.run(X0, v0, wl.D0, n_elec=wl.n_elec, kT=wl.kT if wl.kT > 0 else 0.005, degree=wl.degree,
                      max_iter=200, tol_e_atom=1e-5, tol_D=1e-4)
        torch.cuda.synchronize()
        tts = time.perf_counter() - t0
    finally:
        scf.close()
    print(json.dumps({"kpoint_scf": {"prec": args.prec, "kpoints": kpts, "weights": [0.5, 0.5],
                                     "iterations": res["iterations"], "converged": res["converged"],
                                     "time_to_solution_s": tts, "E_Ha": res["E"], "E_U_Ha": res["E_U"],
                                     "max_imag_D": float(np.max(np.abs(np.imag(res["D"]))))}}))
    return 0


def main():
    args = parse()
    if args.kpoint_scf:
        return run_kpoint_scf(args)
    if args.md_compare:
        return run_md_compare(args)
    if args.forces:
        return run_forces(args)
    if args.stress:
        return run_stress(args)
    if args.density_scf:
        return run_density_scf(args)
    if args.probe_apply:
        return probe_apply(args)
    if args.probe_rr:
        return probe_rr(args)
    if args.projector_forms:
        return run_projector_forms(args)
    if args.probe_alu:
        from paper_2507_23612_gb300.binding import alu_peaks
        print(json.dumps({"probe": "alu_peaks", **alu_peaks()}))
        return 0
    if args.scf_compare:
        return scf_compare(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "warm":
        return run_warm(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl_name = {"rutile": "rutile-2x2x3-72atoms-88x88x84-348orb-2spin-degree24",
               "tiny": "tiny-24^3-2atoms-32orb-degree20"}[args.workload]
    metric = "H·psi throughput over SCF iterations"

    if args.impl == "reference":
        if rank != 0:
            return 0
        cores = min(64, host_cores())
        vals = []
        for _ in range(args.warmup):
            cpu_oracle_sample(args.workload, 2.0, procs=cores)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v, d = cpu_oracle_sample(args.workload, 8.0, procs=cores)
            vals.append(v)
        wall = time.perf_counter() - t0
        value = sum(vals) / len(vals)
        sample = (f"oracle H applications, {cores} single-threaded processes side by side, each on "
                  f"{d['cols']} orbitals of the {wl_name} grid, about 8 s per step")
        print(json.dumps({
            "metric": metric, "value": value, "unit": "Gpt·orb/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": run_config(args, wl_name, make_workload(args.workload), world),
            "cpu_baseline": {"value": value, "unit": "Gpt·orb/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Gpt·orb/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return 0

    if world > 1:
        import torch
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group("nccl", rank=rank, world_size=world,
                                             device_id=torch.device("cuda", local_rank))
    r = run_hub(args, rank, world, local_rank)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            v, d = cpu_oracle_sample(args.workload, args.cpu_seconds)
            cpu = {"value": v, "unit": "Gpt·orb/s", "cores": d["procs"], "kind": "oracle",
                   "sample": f"{d['applications']} oracle H applications, {d['procs']} single-threaded "
                             f"processes side by side, each on {d['cols']} orbitals of the full "
                             f"{wl_name} grid ({d['seconds']:.1f} s)"}
        wl = r["wl"]
        line = {
            "metric": metric, "value": r["value"], "unit": "Gpt·orb/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_NAME[args.prec], "data": "synthetic",
            "config": run_config(args, wl_name, wl, world),
            "roofline": r["roofline"], "rooflines": r["rooflines"], "cpu_baseline": cpu, "e2e": r["e2e"],
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "kernels": r["kernels"],
        }
        line["kernels_profiled_ms"] = r["profiled_ms"]
        if r["tts"]:
            line["scf_time_to_solution"] = r["tts"]
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the Cahn-Hilliard lattice Boltzmann step on one GB300.

Workload: Zalesak's slotted disk on a 256 x 256 periodic lattice (disk radius 64 at (128, 160), slot
16 x 80, W = 4, solid-body rotation with U0 = 0.02, M = 0.005, tau = 1, Model II).  One benchmark step is
one full revolution, 12800 lattice steps, of the FP32 path; the FP64 path runs the same revolution
beside it.  The metric is million lattice updates per second (MLUPS); the roofline fraction is the step
kernel's algorithmic HBM bytes per launch over its average launch time, against the measured copy
bandwidth, with the FP32 arithmetic roofline beside it.  A large-grid sweep (4096^2, inputs far larger
than L2) reports the kernels where HBM or arithmetic, not latency, bounds them: at tau_g = 1 (phi only,
16 B per update) and at tau_g = 0.8 (the populations too, 88 B per update on the FP32 path).  L2 is
flushed (a 512 MiB write) before every timed benchmark step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1805_00007_gb300 import workloads as wl  # noqa: E402

REV_N = 256
METRIC = "MLUPS and % HBM roofline (FP32 vs FP64 step) at stated phi error vs FP64 oracle"

# FP32 operations per lattice update of the row-sweep step at tau_g = 1, Model II, float-float phi: the
# operations of the per-node helpers (a fused multiply-add counts 2): mu 23, D = div(phi u) 34, grad mu and
# grad D 28, force 11, velocity 4, equilibrium + source + collision 55, streaming sum and TwoSum 14.
FLOPS_PER_LU_TAU1 = 169
# The FP64 step does the same operations without the TwoSum (6 fewer) and with a reciprocal refined by two
# Newton steps (6 more): 169 as well.
SMS, FP32_LANES_PER_SM, FP64_LANES_PER_SM = 152, 128, 2

# Algorithmic HBM bytes per lattice update of the general step (any tau_g): the nine populations read and
# written once and phi read and written once, in the storage type of each path (FP16S: eight half
# populations, float phi).  The roofline fraction is reported against these, and beside them against the
# bytes the path in use actually needs (at tau_g = 1 the populations drop out and phi alone is moved).
GENERAL_BYTES_PER_LU = {"f32": 80, "f64": 160, "f16s": 44}

# DRAM bytes (read + write) per launch of the headline kernel, from an ncu capture of these sources
# (dram__bytes_read.sum + dram__bytes_write.sum); reported only while the sources that kernel is compiled
# from (its translation unit) still hash the same and the autotuner chose that kernel, else null.
TRAFFIC = {"hash": "838296a82dae8588", "bytes_per_launch": 669568,
           "kernel": "ch_pair_kernel<float,float,tile=32x14,NT=1024>"}
KERNEL_SOURCES = ("lbch_pair.cu", "lbch_pair.cuh", "lbch_kernels.cuh")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1805_00007_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_name(k: dict, prec: str) -> str:
    types = {"f32": "float,float,float,FF=1", "f64": "double,double,double,FF=0", "f16s": "float,__half,float,FF=0"}[prec]
    if k["form"] in ("sweep", "sweep_tau1"):
        nw = k["threads"] // 32
        return f"ch_sweep_kernel<{types},TY={k['rows_per_warp']},NW={nw},GEN={int(k['form'] == 'sweep')}>"
    if k["form"] == "pair_tau1":
        pt = {"f32": "float,float", "f64": "double,double"}[prec]
        return f"ch_pair_kernel<{pt},tile={k['tile'][0]}x{k['tile'][1]},NT={k['threads']}>"
    return (f"ch_step_kernel<{types},tile={k['tile'][0]}x{k['tile'][1]},NT={k['threads']},"
            f"TAU1={int(k['form'] == 'tile_tau1')}>")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs (the samples go to
    $LBCH_CLOCKS_DIR, else the system's temporary directory)."""

    def __init__(self, index: int):
        import tempfile
        self.index = index
        self.proc = None
        out = os.environ.get("LBCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_rank{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1])); mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1.0)


def oracle_baseline(p, phi0, nsteps, threads=0):
    """The FP64 oracle as it stands, on the host cores (threads > 0: that many; 0: all, its default):
    lattice updates per second over nsteps, the seconds taken and the threads used."""
    import oracle
    prev = oracle.set_threads(0)
    used = oracle.set_threads(threads) if threads > 0 else prev
    g = oracle.init(p, phi0)
    t0 = time.perf_counter()
    oracle.run(p, g, nsteps)
    dt = time.perf_counter() - t0
    oracle.set_threads(prev)
    return p["nx"] * p["ny"] * nsteps / dt / 1e6, dt, used


def oracle_by_config():
    """The FP64 oracle as it stands on each configuration's workload, on the host's threads (its default): the
    translation in full, the others on a bounded number of steps.  Lattice updates per second, and the wall time
    the configuration's full length would take at that rate (reported, not a target)."""
    import oracle
    out = {}

    def record(name, lu, dt, used, steps, full_lu):
        out[name] = {"MLUPS": lu / dt / 1e6, "steps": steps, "seconds": dt, "threads": used,
                     "full_run_s": full_lu / (lu / dt)}

    p, f, n = wl.translation()
    v, dt, used = oracle_baseline(p, f, n)
    record("translation_100_2500_steps", p["nx"] * p["ny"] * n, dt, used, n, p["nx"] * p["ny"] * n)
    p, f, rev = wl.zalesak(n=REV_N)
    v, dt, used = oracle_baseline(p, f, 300)
    record("zalesak_256_one_revolution", p["nx"] * p["ny"] * 300, dt, used, 300, p["nx"] * p["ny"] * rev)
    p, f, tv = wl.single_vortex()
    v, dt, used = oracle_baseline(p, f, 40)
    record("single_vortex_512_T8000", p["nx"] * p["ny"] * 40, dt, used, 40, p["nx"] * p["ny"] * tv)
    ens = wl.shear_ensemble()
    lu = dt = 0.0
    for q, f in ens:  # every instance, a few steps each
        _, d, used = oracle_baseline(q, f, 3)
        lu += q["nx"] * q["ny"] * 3
        dt += d
    record("shear_ensemble_256_5000_steps", lu, dt, used, 3, lu / 3 * 5000)
    p, f = wl.rayleigh_taylor()
    t0 = time.perf_counter()
    oracle.ns_simulate(p, f, 10)
    dt = time.perf_counter() - t0
    record("rayleigh_taylor_256x1024_2e4_steps", p["nx"] * p["ny"] * 10, dt, oracle.set_threads(0), 10,
           p["nx"] * p["ny"] * 20000)
    out["rayleigh_taylor_256x1024_2e4_steps"]["threads_note"] = \
        "the coupled step's stencils run on the threads, its per-node collision loop on one"
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    p, phi0, rev = wl.zalesak(n=REV_N)
    sample = 150  # lattice steps of the 256^2 workload per benchmark step
    for _ in range(args.warmup):
        oracle_baseline(p, phi0, 5)
    vals, tot, cores = [], 0.0, 1
    for _ in range(args.steps):
        v, dt, cores = oracle_baseline(p, phi0, sample)
        vals.append(v)
        tot += dt
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "zalesak_256x256_fp64_oracle", "nx": REV_N, "ny": REV_N,
                       "lattice_steps_per_step": sample, "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} lattice steps of the 256x256 Zalesak workload per step"},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def sweep_params(n, tau=1.0, ny=None):
    """A rotation workload of n x ny nodes (square by default; the Zalesak flow and parameters scaled to n)."""
    ny = n if ny is None else ny
    pp = wl.make_params(nx=n, ny=ny, vel=wl.VEL_ROTATION, U0=0.02, xc=n / 2, yc=ny / 2, half=n / 2,
                        W=4.0, M=0.005, tau=tau)
    return pp, wl.circle_phi(n, ny, n / 2, 5 * ny / 8, min(n, ny) / 4, 4.0)


def steps_per_launch(k: dict) -> int:
    """Lattice steps one launch of the kernel takes (the two-step kernel takes two)."""
    return 2 if k["form"] == "pair_tau1" else 1


def size_sweep(sizes, precs):
    """The step on square periodic grids from 1024^2 up: the diagonal translation workload of Sec. III.A
    (circle of radius n/4, W = 4, u = (0.04, 0.04), M = 0.01, tau_g = 0.8, Model II), each grid autotuned
    and timed over enough steps for about 50 ms.  One JSON line; not part of the default run."""
    import torch
    from paper_1805_00007_gb300 import abi
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.Stream()
    out = {}
    for prec in precs:
        for n in sizes:
            pp = wl.make_params(nx=n, ny=n, vel=wl.VEL_UNIFORM, ux0=0.04, uy0=0.04, W=4.0, M=0.01, tau=0.8)
            f0 = wl.circle_phi(n, n, n / 2, n / 2, n / 4, 4.0)
            with abi.Simulation(pp, f0, prec=prec, stream=stream.cuda_stream, tune=True) as sim:
                sim.step(4)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(4)
                e1.record(stream)
                e1.synchronize()
                nst = max(8, min(256, int(0.05 / (e0.elapsed_time(e1) / 1e3 / 4))))
                e0.record(stream)
                sim.step(nst)
                e1.record(stream)
                e1.synchronize()
                dt = e0.elapsed_time(e1) / 1e3 / nst
                inf = sim.info()
                gbs = inf["bytes_per_lu"] * n * n / dt / 1e9
                out[f"{prec}_{n}"] = {"MLUPS": n * n / dt / 1e6, "us_per_step": dt * 1e6, "steps_timed": nst,
                                      "kernel": kernel_name(sim.kernel(), prec), "bytes_per_lu": inf["bytes_per_lu"],
                                      "achieved_gbs": gbs, "frac": gbs / hbm_peak}
    print(json.dumps({"size_sweep": out, "workload": "diagonal translation, tau_g = 0.8, Model II",
                      "peak_gbs": hbm_peak, "peak_kind": peak_kind}))


def run_case(case, nsteps, tile=0, form="sweep"):
    """One grid, no timing: the command ncu profiles."""
    import torch
    from paper_1805_00007_gb300 import abi
    parts = case.split("_")
    if parts[0] == "rt":  # the coupled Rayleigh-Taylor workload, 256 x 1024 (rt_f32, rt_f64)
        from paper_1805_00007_gb300 import workloads as wl
        pp, f0 = wl.rayleigh_taylor()
        with abi.Simulation(pp, f0, prec=parts[1]) as sim:
            sim.step(nsteps)
            torch.cuda.synchronize()
            m = sim.observe(abi.LBCH_OBS_MASS)
        print(json.dumps({"case": case, "steps": nsteps, "mass": m, "kernels": "ns::fields, ns::collide (ns::phi before observing)"}))
        return
    if parts[0] == "adj":  # adjoint steps on the n^2 single vortex (FP32 forward tape), e.g. adj_512
        from paper_1805_00007_gb300 import workloads as wl
        n = int(parts[1])
        pv, fv, _ = wl.single_vortex(n=n)
        with abi.Simulation(pv, fv, prec="f32") as sim:
            sim.step(4)
            tape = torch.empty((n, n), dtype=torch.float32, device="cuda")
            abi.lb_ch_tape_phi(sim.h, tape.data_ptr())
            seed = torch.ones((n, n), dtype=torch.float64, device="cuda")
            abi.lb_ch_adjoint_begin(sim.h, seed.data_ptr())
            for k in range(nsteps):
                abi.lb_ch_adjoint_step(sim.h, tape.data_ptr(), 4 + nsteps - 1 - k)
            torch.cuda.synchronize()
        print(json.dumps({"case": case, "adjoint_steps": nsteps,
                          "kernels": "adj::fwd_mu, adj::local, adj::transpose1, adj::transpose2"}))
        return
    if parts[0] == "ens":  # the first N instances of the ragged shear ensemble, e.g. ens_f32_64 or ens_f32_64_0.8
        from paper_1805_00007_gb300 import workloads as wl
        ens = wl.shear_ensemble(tau=float(parts[3]) if len(parts) > 3 else 1.0)[:int(parts[2])]
        with abi.Simulation([q for q, _ in ens], [f for _, f in ens], prec=parts[1], tune=tile < 0) as sim:
            if tile >= 0:
                abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, int(form == "tile"))
                abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_SHAPE, tile)
            sim.step(nsteps)
            torch.cuda.synchronize()
            kname = kernel_name(sim.kernel(), parts[1])
            nodes = sim.info()["nodes"]
        print(json.dumps({"case": case, "steps": nsteps, "instances": len(ens), "nodes": nodes, "kernel": kname}))
        return
    prec = parts[0]
    n, ny = (int(v) for v in parts[1].split("x")) if "x" in parts[1] else (int(parts[1]), None)
    tau = float(parts[2]) if len(parts) > 2 else 1.0
    pp, f0 = sweep_params(n, tau, ny)
    with abi.Simulation(pp, f0, prec=prec, tune=tile < 0) as sim:
        if tile >= 0:
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, int(form == "tile"))
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TWO_STEP, int(form == "pair"))
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_SHAPE, tile)
        sim.step(nsteps)
        torch.cuda.synchronize()
        m = sim.observe(abi.LBCH_OBS_MASS)
        kname = kernel_name(sim.kernel(), prec)
    print(json.dumps({"case": case, "steps": nsteps, "mass": m, "kernel": kname}))


def accuracy(prec, p, phi0, nsteps):
    """max |phi - phi_oracle| over every node after the full run (the oracle's stored final field), the
    relative difference of ||E_phi||_2 (Eq. err) and the mass drift; None when the stored field is absent."""
    path = os.path.join(ROOT, "tests", "golden", "zalesak_256_phi.npz")
    if not os.path.exists(path):
        return None
    gold = np.load(path)
    if int(gold["nsteps"]) != nsteps:
        return None
    ref = gold["phi"]
    from paper_1805_00007_gb300 import abi
    with abi.Simulation(p, phi0, prec=prec) as sim:
        sim.step(nsteps)
        phi = sim.phi()
        err = sim.observe(abi.LBCH_OBS_ERR_L2)
        mass = sim.observe(abi.LBCH_OBS_MASS)
    err_o = float(np.sqrt(np.sum((ref - phi0) ** 2) / np.sum(phi0 ** 2)))
    return {"max_abs_dphi_vs_oracle": float(np.max(np.abs(phi - ref))), "nodes_compared": int(ref.size),
            "err_l2": err, "err_l2_oracle": err_o, "err_l2_rel_diff": abs(err - err_o) / err_o,
            "mass_rel_drift": abs(mass - float(phi0.sum())) / float(phi0.sum())}


def accuracy_vs_fp64(sims_of, nsteps, precs):
    """max |phi - phi_FP64| over every node of every instance after nsteps, for each precision, where the
    FP64 path is the reference (it matches the oracle to 1e-12 at this length in the GPU tests)."""
    ref = sims_of("f64")
    ref.step(nsteps)
    n_inst = len(ref.params)
    ref_phi = [ref.phi(k) for k in range(n_inst)]
    ref.close()
    out = {}
    for prec in precs:
        sim = sims_of(prec)
        sim.step(nsteps)
        out[prec] = max(float(np.max(np.abs(sim.phi(k) - ref_phi[k]))) for k in range(n_inst))
        sim.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--size-sweep", action="store_true",
                    help="time the step on 1024^2 .. 16384^2 grids (tau_g = 0.8) instead of the benchmark")
    ap.add_argument("--case", default=None,
                    help="profiling case PREC_N[xNY][_TAU] (e.g. f32_4096, f32_4096_0.8, f32_8192x1024_0.8), rt_PREC (the coupled "
                         "Rayleigh-Taylor grid), adj_N (adjoint steps on the N^2 single vortex) or "
                         "ens_PREC_N[_TAU] (the first N instances of the shear ensemble): init and "
                         "--case-steps steps of that case only")
    ap.add_argument("--case-steps", type=int, default=8)
    ap.add_argument("--case-tile", type=int, default=0, help="tile shape index for --case (-1: autotune)")
    ap.add_argument("--case-form", default="sweep", choices=["sweep", "tile", "pair"], help="kernel form for --case")
    ap.add_argument("--kernel", default=None,
                    help="FORM:SHAPE (sweep|tile|pair and a shape index): pin the FP32 headline kernel instead of "
                         "autotuning it -- for a profiler run, under which the tuner's timings are distorted")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args.case, args.case_steps, args.case_tile, args.case_form)
    if args.size_sweep:
        return size_sweep((1024, 2048, 4096, 8192, 16384), ("f32", "f64", "f16s"))

    import torch
    import torch.distributed as dist

    from paper_1805_00007_gb300 import abi

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_peak, peak_kind = peaks()

    p, phi0, rev = wl.zalesak(n=REV_N)
    nodes = REV_N * REV_N
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def timed_revolutions(prec, k, w, pin=None):
        """Run w warm-up and k timed revolutions; returns (mean seconds per revolution, the simulation, the
        time of each revolution)."""
        sim = abi.Simulation(p, phi0, prec=prec, stream=stream.cuda_stream, tune=pin is None)
        if pin is not None:
            form, shape = pin.split(":")
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, int(form == "tile"))
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TWO_STEP, int(form == "pair"))
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_SHAPE, int(shape))
        for _ in range(w):
            with torch.cuda.stream(stream):
                flush_l2(flush)
            sim.step(rev)
        barrier()
        times = []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush_l2(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(rev)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        barrier()
        return sum(times) / k, sim, times

    # --- FP32 path: the headline value
    with Clocks(local) as clk:
        t32, sim32, times32 = timed_revolutions("f32", args.steps, args.warmup, args.kernel)
    t_max = t32
    if world > 1:
        t = torch.tensor([t32], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    info32 = sim32.info()
    tile32 = sim32.tile
    kern32 = sim32.kernel()
    phi32 = sim32.phi()
    sim32.close()

    # --- FP64 path, same revolution
    t64, sim64, times64 = timed_revolutions("f64", max(1, args.steps // 2), 1)
    kern64 = sim64.kernel()
    info64 = sim64.info()
    n_rev64 = args.steps // 2 + 1 + max(1, args.steps // 2)
    phi64 = sim64.phi()
    sim64.close()

    lu_per_rev = nodes * rev
    value = world * lu_per_rev / t_max / 1e6
    spl32 = steps_per_launch(kern32)
    launch32 = t32 / rev * spl32  # one launch of the headline kernel
    achieved32 = info32["bytes_per_lu"] * nodes * spl32 / launch32 / 1e9
    achieved_gen32 = GENERAL_BYTES_PER_LU["f32"] * nodes * spl32 / launch32 / 1e9
    achieved64 = info64["bytes_per_lu"] * nodes / (t64 / rev) / 1e9

    # --- end to end through the C ABI with host buffers: init (H2D of phi0), one revolution, read phi (D2H)
    e2e_times = []
    for it in range(2 + max(1, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = abi.lb_ch_init(p, phi0, abi.LBCH_F32, stream.cuda_stream)
        abi.lb_ch_step(h, rev)
        out = abi.lb_ch_observe(h, 0, abi.LBCH_OBS_PHI, (REV_N, REV_N))
        abi.lb_ch_free(h)
        dt = time.perf_counter() - t0
        if it >= 2:
            e2e_times.append(dt)
    e2e = world * lu_per_rev / statistics.median(e2e_times) / 1e6

    # --- large-grid sweep: the same kernel with inputs far larger than L2 (HBM-bound regime)
    sweep = {}
    if not args.no_sweep:
        for prec, n, tau in (("f32", 4096, 1.0), ("f64", 4096, 1.0), ("f16s", 4096, 1.0),
                             ("f32", 4096, 0.8), ("f64", 4096, 0.8), ("f16s", 4096, 0.8)):
            pp, f0 = sweep_params(n, tau)
            sim = abi.Simulation(pp, f0, prec=prec, stream=stream.cuda_stream, tune=True)
            sim.step(64)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nst = 128
            e0.record(stream)
            sim.step(nst)
            e1.record(stream)
            e1.synchronize()
            dt = e0.elapsed_time(e1) / 1e3 / nst
            inf = sim.info()
            gbs = inf["bytes_per_lu"] * n * n / dt / 1e9
            sweep[f"{prec}_{n}" + ("" if tau == 1.0 else f"_tau{tau}")] = {
                "MLUPS": n * n / dt / 1e6, "us_per_launch": dt * 1e6 * steps_per_launch(sim.kernel()),
                "kernel": kernel_name(sim.kernel(), prec),
                "bytes_per_lu": inf["bytes_per_lu"], "achieved_gbs": gbs, "frac": gbs / hbm_peak}
            sim.close()


    # --- the ragged ensemble: 256 wall-bounded shear instances (23.1 M nodes) advanced in one launch per step;
    #     with several ranks the instances are shared out (independent problems, nothing exchanged)
    ensemble = {}
    if not args.no_sweep:
        from paper_1805_00007_gb300 import shard
        for etau, prec in ((1.0, "f32"), (1.0, "f16s"), (0.8, "f32"), (0.8, "f16s")):
            ens = wl.shear_ensemble(tau=etau)
            enodes = sum(q["nx"] * q["ny"] for q, _ in ens)
            _, eparams, efields = shard.shard(ens, rank, world)
            key = prec if etau == 1.0 else f"{prec}_tau{etau}"
            sim = abi.Simulation(list(eparams), list(efields), prec=prec, stream=stream.cuda_stream, tune=True)
            sim.step(64)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nst = 128
            e0.record(stream)
            sim.step(nst)
            e1.record(stream)
            e1.synchronize()
            dt = e0.elapsed_time(e1) / 1e3 / nst
            if world > 1:
                t = torch.tensor([dt], device=dev, dtype=torch.float64)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                dt = float(t.item())
            inf = sim.info()
            gbs = inf["bytes_per_lu"] * enodes / dt / 1e9
            ggen = GENERAL_BYTES_PER_LU[prec] * enodes / dt / 1e9
            ensemble[key] = {"instances": len(ens), "nodes": enodes, "tau": etau, "MLUPS": enodes / dt / 1e6,
                             "ranks": world, "sharding": "instances across ranks, no exchange",
                             "kernel": kernel_name(sim.kernel(), prec),
                             "us_per_launch": dt * 1e6 * steps_per_launch(sim.kernel()),
                             "roofline": {"bound": "hbm", "peak": hbm_peak, "unit": "GB/s", "peak_kind": peak_kind,
                                          "bytes_per_lu": GENERAL_BYTES_PER_LU[prec], "achieved": ggen,
                                          "frac": ggen / hbm_peak,
                                          "bytes_basis": "general step: populations and phi read and written once",
                                          "path": {"bytes_per_lu": inf["bytes_per_lu"], "achieved": gbs,
                                                   "frac": gbs / hbm_peak,
                                                   "basis": ("phi alone (tau_g = 1: the populations drop out)"
                                                             if etau == 1.0 else
                                                             "populations and phi (hi + lo on FP32) read and "
                                                             "written once")}}}
            sim.close()
            if prec == "f32" and etau == 1.0:
                # the same instances as separate single-instance handles, stepped one after another on the
                # same stream (each with the untuned default kernel): what the batched launch saves
                sims = [abi.Simulation(q, f, prec=prec, stream=stream.cuda_stream) for q, f in zip(eparams, efields)]
                for s in sims:
                    s.step(64)
                barrier()
                e0.record(stream)
                for s in sims:
                    s.step(nst)
                e1.record(stream)
                e1.synchronize()
                dt_loop = e0.elapsed_time(e1) / 1e3 / nst
                if world > 1:
                    t = torch.tensor([dt_loop], device=dev, dtype=torch.float64)
                    dist.all_reduce(t, op=dist.ReduceOp.MAX)
                    dt_loop = float(t.item())
                for s in sims:
                    s.close()
                ensemble[key]["looped_single_instance_MLUPS"] = enodes / dt_loop / 1e6
                ensemble[key]["batched_speedup"] = dt_loop / dt

    # --- the coupled Rayleigh-Taylor workload (256 x 1024, Navier-Stokes + Cahn-Hilliard, walls in y) and the
    #     adjoint step of the 512^2 single-vortex workload: the step rates of the other two kernel families
    coupled, adjoint = {}, {}
    if not args.no_sweep and rank == 0:
        prt, frt = wl.rayleigh_taylor()
        nrt = prt["nx"] * prt["ny"]
        for prec in ("f32", "f64"):
            with abi.Simulation(prt, frt, prec=prec, stream=stream.cuda_stream) as sim:
                sim.step(64)
                torch.cuda.synchronize()
                nst = 256 if prec == "f32" else 64
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(nst)
                e1.record(stream)
                e1.synchronize()
                dt = e0.elapsed_time(e1) / 1e3 / nst
                inf = sim.info()
                gbs = inf["bytes_per_lu"] * nrt / dt / 1e9
                coupled[prec] = {"MLUPS": nrt / dt / 1e6, "us_per_step": dt * 1e6, "bytes_per_lu": inf["bytes_per_lu"],
                                 "achieved_gbs": gbs, "frac": gbs / hbm_peak, "kernels_per_step": 2}
        pv, fv, _ = wl.single_vortex(n=512)
        nv = pv["nx"] * pv["ny"]
        with abi.Simulation(pv, fv, prec="f32", stream=stream.cuda_stream) as sim:
            sim.step(4)
            tape = torch.empty((pv["ny"], pv["nx"]), dtype=torch.float32, device=dev)
            abi.lb_ch_tape_phi(sim.h, tape.data_ptr())
            seed = torch.zeros((pv["ny"], pv["nx"]), dtype=torch.float64, device=dev)
            abi.lb_ch_adjoint_begin(sim.h, seed.data_ptr())
            for k in range(8):
                abi.lb_ch_adjoint_step(sim.h, tape.data_ptr(), 100 - k)
            torch.cuda.synchronize()
            nst = 64
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(nst):
                abi.lb_ch_adjoint_step(sim.h, tape.data_ptr(), 90 - k)
            e1.record(stream)
            e1.synchronize()
            dta = e0.elapsed_time(e1) / 1e3 / nst
            adjoint = {"workload": "512^2 single vortex, FP32 forward tape, adjoint carried in FP64",
                       "MLUPS": nv / dta / 1e6, "us_per_step": dta * 1e6}

    # --- the gradient of the single-vortex loss (512^2, T = 8000: FP32 forward, adjoint in FP64) with respect to
    #     phi0 and the velocity scale, forward and backward through evolve() with binomial checkpointing
    gradient = {}
    if not args.no_sweep and rank == 0:
        from paper_1805_00007_gb300.autograd import evolve, schedule_stats
        pv, fv, tv = wl.single_vortex()
        ck, leaf = 16, 64
        gtimes = []
        for it in range(2):
            x = torch.tensor(fv, dtype=torch.float64, requires_grad=True)
            sc = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            phiT = evolve(x, sc, pv, tv, prec="f32", checkpoints=ck, leaf=leaf)
            loss = 0.5 * torch.sum((phiT - x.detach()) ** 2)
            loss.backward()
            torch.cuda.synchronize()
            gtimes.append(time.perf_counter() - t0)
        stt = schedule_stats(tv, ck, leaf)
        nbytes_state = None
        with abi.Simulation(pv, fv, prec="f32") as sim:
            nbytes_state = abi.lb_ch_state_bytes(sim.h)
        gradient = {"workload": "512^2 single vortex, T = 8000, loss 1/2 |phi(T) - phi0|^2, d/dphi0 and d/dscale",
                    "ms": 1e3 * min(gtimes), "ms_first": 1e3 * gtimes[0], "adjoint_steps": tv,
                    "forward_steps": stt["forward_steps"], "repetitions": stt["repetitions"],
                    "stored_states": stt["slots"], "state_mb": nbytes_state / 2 ** 20, "tape_steps": leaf,
                    "tape_mb": leaf * pv["nx"] * pv["ny"] * 4 / 2 ** 20, "dL_dscale": float(sc.grad)}

    # --- the paper's relaxation-time study (Sec. III.A) at its own size, every point one ensemble instance
    tau_sweep = {}
    if not args.no_sweep and rank == 0:
        from paper_1805_00007_gb300 import sweeps
        taus = (0.6, 0.7, sweeps.TAU_STAR, 0.9, 1.0, 1.3)
        t0 = time.perf_counter()
        res = sweeps.translation_tau_sweep(taus, models=(1, 2, 3), L0=200, prec="f64", stream=stream.cuda_stream)
        tau_sweep = {"workload": "diagonal translation, L0 = 200, Pe = 200, W = 2, rhoA/rhoB = 2, one period, FP64",
                     "err_l2": {f"tau={t:.4f}": {f"model{m}": res[t, m] for m in (1, 2, 3)} for t in taus},
                     "seconds": time.perf_counter() - t0}

    acc = {prec: accuracy(prec, p, phi0, rev) for prec in ("f32", "f64", "f16s")} if rank == 0 else {}

    # --- the other workloads at their stated lengths: every node of the float paths against the FP64 path
    acc_more = {}
    if rank == 0 and not args.no_sweep:
        sc = stream.cuda_stream
        pv, fv, tv = wl.single_vortex()
        acc_more["vortex_512_T8000"] = {
            "max_abs_dphi_vs_fp64": accuracy_vs_fp64(lambda pr: abi.Simulation(pv, fv, prec=pr, stream=sc), tv, ("f32",)),
            "nodes": pv["nx"] * pv["ny"], "steps": tv}
        for etau in (1.0, 0.8):
            ens = wl.shear_ensemble(tau=etau)
            eq, ef = [q for q, _ in ens], [f for _, f in ens]
            acc_more[f"ensemble_shear_256_tau{etau}"] = {
                "max_abs_dphi_vs_fp64": accuracy_vs_fp64(lambda pr: abi.Simulation(eq, ef, prec=pr, stream=sc), 200,
                                                         ("f32", "f16s")),
                "instances": len(ens), "nodes": sum(f.size for f in ef), "steps": 200, "over": "every instance"}
        prt, frt = wl.rayleigh_taylor()
        acc_more["rayleigh_taylor_256x1024"] = {
            "max_abs_dphi_vs_fp64_500_steps": accuracy_vs_fp64(lambda pr: abi.Simulation(prt, frt, prec=pr, stream=sc),
                                                              500, ("f32",))}
        for prec in ("f32", "f64"):
            with abi.Simulation(prt, frt, prec=prec, stream=sc) as sim:
                done, rec = 0, {"finite": True}
                while done < 20000:  # in blocks, to find where a run stops being finite
                    sim.step(1000)
                    done += 1000
                    try:
                        phr = sim.phi()
                        mrt = sim.observe(abi.LBCH_OBS_MASS)
                    except abi.LbchError:
                        rec = {"finite": False, "non_finite_by_step": done}
                        break
                if rec["finite"]:
                    rec.update({"mass_rel_drift": abs(mrt - float(frt.sum())) / float(np.abs(frt).sum()),
                                "mirror_asymmetry": float(np.max(np.abs(np.roll(phr[:, ::-1], 1, axis=1) - phr))),
                                "phi_range": [float(phr.min()), float(phr.max())]})
            acc_more["rayleigh_taylor_256x1024"][f"{prec}_20000_steps"] = rec

    cpu = None
    if rank == 0 and not args.no_cpu:
        sample, sample1 = 1200, 120
        v, dt, used = oracle_baseline(p, phi0, sample)
        v1, dt1, _ = oracle_baseline(p, phi0, sample1, threads=1)
        cpu = {"value": v, "unit": "MLUPS", "cores": used, "kind": "oracle",
               "sample": f"{sample} lattice steps of the 256x256 Zalesak workload ({dt:.1f} s)",
               "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1,
                                 "sample": f"{sample1} lattice steps of the same workload ({dt1:.1f} s)"},
               "by_config": oracle_by_config()}

    clocks = clk.summary()
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak_tflops = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    peak64_tflops = SMS * FP64_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    alu_tflops = FLOPS_PER_LU_TAU1 * nodes * spl32 / launch32 / 1e12
    alu64_tflops = FLOPS_PER_LU_TAU1 * nodes / (t64 / rev) / 1e12
    # the FMA throughput the device sustains (lb_ch_alu_peak), beside the unit-count peaks
    fma32 = abi.lb_ch_alu_peak(abi.LBCH_F32, stream.cuda_stream) / 1e12
    fma64 = abi.lb_ch_alu_peak(abi.LBCH_F64, stream.cuda_stream) / 1e12
    traffic = (TRAFFIC["bytes_per_launch"]
               if TRAFFIC["hash"] == kernel_hash() and TRAFFIC["kernel"] == kernel_name(kern32, "f32") else None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "zalesak_256x256_one_revolution", "nx": REV_N, "ny": REV_N,
                       "lattice_steps_per_step": rev, "model": "II", "l2": "flushed before each step",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "revolution_ms": {"mean": 1e3 * t32, "best": 1e3 * min(times32),
                              "median": 1e3 * statistics.median(times32), "n": len(times32)},
            "fp32_over_fp64": t64 / t32,
            "fp64": {"MLUPS": world * lu_per_rev / t64 / 1e6, "ms_per_step": 1e3 * t64,
                     "revolution_ms": {"best": 1e3 * min(times64), "median": 1e3 * statistics.median(times64),
                                       "n": len(times64)},
                     "achieved_gbs": achieved64, "frac": achieved64 / hbm_peak, "kernel": kernel_name(kern64, "f64"),
                     "alu": {"flops_per_lu": FLOPS_PER_LU_TAU1, "achieved": alu64_tflops, "peak": peak64_tflops,
                             "unit": "TFLOP/s", "frac": alu64_tflops / peak64_tflops,
                             "peak_from": "152 SMs x 2 FP64 lanes x 2 flop x median SM clock under load",
                             "peak_measured": fma64, "frac_of_measured": alu64_tflops / fma64}},
            "roofline": {"bound": "hbm", "achieved": achieved_gen32, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved_gen32 / hbm_peak, "traffic": traffic,
                         "kernel": kernel_name(kern32, "f32"), "bytes_per_lu": GENERAL_BYTES_PER_LU["f32"],
                         "bytes_basis": "general step: 9 populations and phi read and written once, 4 B each",
                         "path": {"bytes_per_lu": info32["bytes_per_lu"], "achieved": achieved32,
                                  "frac": achieved32 / hbm_peak,
                                  "basis": "what the kernel in use moves: at tau_g = 1 phi alone (hi + lo), read and "
                                           "written once per launch of two steps"},
                         "l2_resident": "one 256^2 field is 0.5 MB: the state stays in L2, so HBM does not bound it",
                         "peak_kind": peak_kind, "us_per_launch": launch32 * 1e6,
                         "alu": {"flops_per_lu": FLOPS_PER_LU_TAU1, "achieved": alu_tflops, "peak": peak_tflops,
                                 "unit": "TFLOP/s", "frac": alu_tflops / peak_tflops,
                                 "peak_from": "152 SMs x 128 FP32 lanes x 2 flop x median SM clock under load",
                                 "peak_measured": fma32, "frac_of_measured": alu_tflops / fma32}},
            "sweep_4096": sweep,
            "ensemble_shear_256": ensemble,
            "paper_tau_sweep": tau_sweep,
            "coupled_rt_256x1024": coupled,
            "adjoint_vortex_512": adjoint,
            "gradient_vortex_512_T8000": gradient,
            "accuracy_one_revolution": acc,
            "accuracy_full_length": acc_more,
            "e2e": {"value": e2e, "unit": "MLUPS", "h2d_bytes_per_step": phi0.nbytes,
                    "d2h_bytes_per_step": phi0.nbytes},
            "gpu_launches": args.steps * rev // spl32,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Benchmark of the TTN sweep on GB300 (one JSON line on stdout).

Workload: the critical transverse-field Ising chain, L = 1024, h = 1, one
shared isometry per layer, bond dimension chi = 128 (chi_t = 2, 4, 16, 128 ...),
seeded QR-orthonormalised Gaussian start (seed 1).  A step is one sweep.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec tf32x3|fp64|...]
    python bench.py --impl reference ...      # the FP64 CPU oracle, same workload

The GPU arm reports sweeps/s of the chosen precision with the tensors resident
in HBM (``value``), the same through the C ABI with host buffers (``e2e``), the
FP64 GPU path for comparison, the energy error against the oracle's reference
trajectory, the roofline of the dominant kernel family and the oracle timed on
this host (``cpu_baseline``).  With N > 1 (torchrun) every rank advances its own
replica: the sweep of one instance does not shard (replicas only).
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "tfim_chain_L1024_h1_chi128", "L": 1024, "h": 1.0, "chi": 128,
            "seed": 1, "model": "transverse-field Ising chain, periodic",
            "tree": "binary TTN, one isometry per layer"}
METRIC = "TTN sweeps/s at chi=128 (TFIM L=1024)"
# DRAM bytes (read + write) per launch of a kernel family, averaged over the
# launches of one steady-state sweep of the headline workload (sweep 31 from
# the seeded start, tuned table loaded), from an ncu capture of the current
# kernels (dram__bytes_read.sum + dram__bytes_write.sum; ncu flushes the caches
# before each launch, so these are cold-cache figures, and writes still in L2
# at the end of a launch are not counted).  A family without a capture of its
# current kernel has none.  This is a stored measurement, labelled as such in
# the line.
TRAFFIC = {
    "tc_hbm": 14.70e6,   # gemm_tma_kernel: 128 launches, 1.88 GB
    "tc": 14.70e6,
    "df": 5.71e6,        # gemm_df_kernel: 63 launches (39 return at once), 0.360 GB
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--prec", default=os.environ.get("TTN_BENCH_PREC", "tf32x3"))
    p.add_argument("--chi", type=int, default=128)
    p.add_argument("--no-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true", help="keep the launchers' default tiles")
    p.add_argument("--tiles-file", default=None,
                   help="load the autotuner's table from this file instead of tuning")
    p.add_argument("--save-tiles", default=None, help="write the autotuner's table to this file")
    p.add_argument("--cpu-1thread", action="store_true",
                   help="also time the oracle with one BLAS thread (minutes at chi=128)")
    p.add_argument("--quick", action="store_true", help="skip the 200-sweep energy-error runs")
    p.add_argument("--profile-sweeps", type=int, default=0,
                   help="only run this many eagerly launched sweeps (for an ncu launch list) and exit")
    p.add_argument("--lanczos-tol", type=float, default=0.0,
                   help="top-solve residual tolerance (0: the library's default for the precision)")
    p.add_argument("--profile-start", type=int, default=0,
                   help="with --profile-sweeps: sweeps run before the profiled ones, outside the "
                        "cudaProfilerStart/Stop range (ncu --profile-from-start off)")
    p.add_argument("--workload", default="tfim1024",
                   choices=["tfim1024", "batched64", "paper-torus", "top-mode", "configs",
                            "polar-study"],
                   help="tfim1024: the headline line; batched64: 64 independent chains in one "
                        "context; paper-torus: the paper's 128 x 5 torus at h = 2.9 with its "
                        "entanglement spectrum; top-mode: eigensolver vs polar-step top update; "
                        "configs: the five configurations' table")
    return p.parse_args()


def aggregate(ms_local: float, steps: int, world: int, dist=None, device="cpu"):
    """Whole-job throughput of replicas: every rank ran `steps` sweeps in
    ms_local milliseconds; the job takes the slowest rank's time.  Returns
    (sweeps per second over all ranks, max milliseconds)."""
    t_max = ms_local
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return world * steps / (t_max * 1e-3), t_max


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the same workload
# --------------------------------------------------------------------------

def oracle_sweeps_per_s(n_sweeps: int, warm: int, chi: int):
    import numpy as np  # noqa: F401
    import ttn_inputs as ti
    from oracle import ttn as oracle
    m = ti.tfim_chain(1024, 1.0)
    ws, V = ti.initial_tensors(1024, 2, chi, 1)
    st = oracle.make_state(m, ws, V)
    for _ in range(warm):
        oracle.sweep(st)
    t0 = time.perf_counter()
    for _ in range(n_sweeps):
        oracle.sweep(st)
    dt = time.perf_counter() - t0
    return n_sweeps / dt, dt


def cpu_model():
    """The host CPU's model string (lscpu), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_timing(chi, threads, warm=2, timed=3, timeout=900):
    """Seconds of each of `timed` oracle sweeps of the headline workload after
    `warm` warm-up sweeps from the seeded start, in a fresh process with the
    BLAS limited to `threads` threads (None when it fails or runs out of time)."""
    code = ("import json, time, ttn_inputs as ti\n"
            "from oracle import ttn as oracle\n"
            "m = ti.tfim_chain(1024, 1.0)\n"
            f"ws, V = ti.initial_tensors(1024, 2, {chi}, 1)\n"
            "st = oracle.make_state(m, ws, V)\n"
            f"for _ in range({warm}): oracle.sweep(st)\n"
            "ts = []\n"
            f"for _ in range({timed}):\n"
            "    t0 = time.perf_counter(); oracle.sweep(st); ts.append(time.perf_counter() - t0)\n"
            "print(json.dumps(ts))\n")
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                             text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return None
    if out.returncode != 0:
        return None
    return json.loads(out.stdout.strip().splitlines()[-1])


def threads_used():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each step is one full oracle sweep of the workload
    v, dt = oracle_sweeps_per_s(args.steps, args.warmup, args.chi)
    cores = threads_used()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "sweeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded QR-orthonormalised Gaussian isometries)",
            "config": dict(WORKLOAD, chi=args.chi, workload=f"tfim_chain_L1024_h1_chi{args.chi}",
                           precision="fp64", engine="numpy/LAPACK oracle"),
            "cpu_baseline": {"value": v, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{args.steps} full sweeps after {args.warmup} warm-up sweeps "
                                       f"of the same workload, BLAS threads {cores}"},
            "e2e": {"value": v, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def golden_final_energy(chi, sweeps):
    """FP64 energy of the oracle's tensors after `sweeps` sweeps from the same
    seeded start (written by oracle/make_golden.py)."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_tfim_L1024_chi{chi}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    return g["final_energy"] if g["sweeps"] == sweeps else None


def run_gpu(args):
    import numpy as np
    import torch

    import ttn_inputs as ti
    from paper_1905_01331_gb300 import flops as ttn_flops
    from paper_1905_01331_gb300 import Sweeper, _abi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    chi = args.chi
    model = ti.tfim_chain(1024, 1.0)
    ws, V = ti.initial_tensors(1024, 2, chi, 1)
    s = Sweeper(model, chi, prec=args.prec, lanczos_tol=args.lanczos_tol)
    s.set_isometries(0, ws, V)
    chis = s.chis(0)
    flops_per_sweep = ttn_flops.sweep_flops(1024, chis, 1, symmetric=True)

    # warm-up: the autotuner's sweep (tile widths, engines, split counts of
    # every product shape, timed), then the warm-up sweeps (graph capture)
    tune_t0 = time.perf_counter()
    tiles_blob = s.autotune(reps=3) if not args.no_autotune else b""
    tune_s = time.perf_counter() - tune_t0
    if args.save_tiles and tiles_blob:
        with open(args.save_tiles, "wb") as f:
            f.write(tiles_blob)
    s.sweep(args.warmup)
    stream = s.stream
    torch.cuda.synchronize()
    # pinned host buffers of the state for the end-to-end leg below
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    n_w = sum(int(np.prod(w.shape)) for w in ws)
    flat_host = torch.empty(n_w, dtype=torch.float64).pin_memory()
    v_host = torch.empty(V.size, dtype=torch.float64).pin_memory()
    fp = ctypes.cast(flat_host.data_ptr(), dp)
    vp = ctypes.cast(v_host.data_ptr(), dp)
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.sweep_async(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = s.launch_count
    value, t_max = aggregate(ms, args.steps, world, dist, device="cuda")

    # profiling sweep: dominant kernel family
    prof = s.profile_sweep()

    # e2e through the C ABI with host buffers: upload the state, one sweep,
    # read the energy back, every step.  The state uploaded is the one reached
    # after the timed sweeps (and the profiling sweep), so every e2e step does
    # the work of a steady-state sweep of the timed region plus the copies.
    # (Repeating the first sweep after the warm-up instead would time the top
    # solve of a transient state, which takes two or three restart cycles
    # depending on the last bits of that state: the figure then moves by
    # +-6 % with no change in the steady-state rate.)
    if s.lib.ttn_get_isometries(s.h, 0, fp, vp):
        raise RuntimeError("reading the state back failed")
    E_host = np.zeros(1)
    ep = E_host.ctypes.data_as(dp)
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(2):
        s.lib.ttn_set_isometries(s.h, 0, fp, vp)
        s.lib.ttn_sweep(s.h, 1, ep)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = s.lib.ttn_set_isometries(s.h, 0, fp, vp)
        rc |= s.lib.ttn_sweep(s.h, 1, ep)
        if rc:
            raise RuntimeError("e2e call failed")
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_dt], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_dt = float(t.item())
    e2e = {"value": world * e2e_steps / e2e_dt, "unit": "sweeps/s",
           "h2d_bytes_per_step": 8 * (n_w + V.size), "d2h_bytes_per_step": 8}

    # roofline of each kernel family of the sweep's CUDA-event profile; the
    # line's "roofline" is the family that takes the most time
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    sm_count, sm_ghz = 152, peaks.get("sm_max_mhz", 2070.0) * 1e-3
    hbm = peaks.get("hbm_gbs", 6789.3)
    families = {
        # the same tcgen05 products against HBM bandwidth: their algorithmic
        # bytes (every operand read once, the output written once) over the
        # same time; most are below the ridge of 3xTF32 (~47 flop/B)
        "tc_hbm": {"bound": "hbm", "kernel": "gemm_tma_kernel / gemm_tc_kernel (tcgen05 grouped "
                                             "products), algorithmic bytes",
                   "ms": prof["tc_ms"], "achieved_units": prof.get("tc_bytes", 0.0) * 1e3,
                   "launches": prof["tc_launches"], "peak": hbm, "unit": "GB/s",
                   "peak_source": "MEASURED_PEAKS hbm_gbs (copy bandwidth)"},
        # tcgen05 products: algorithmic flops against the TF32 dense peak
        "tc": {"bound": "tensor", "kernel": "gemm_tc_kernel (tcgen05 grouped products)",
               "ms": prof["tc_ms"], "achieved_units": prof["tc_flops"], "launches": prof["tc_launches"],
               "peak": peaks.get("bf16_tflops", 1932.2) * 0.5,
               "peak_source": "MEASURED_PEAKS bf16_tflops x 0.5 (nominal tf32:bf16)"},
        # FP64 products and the polar composition: executed FP64 flops
        "fp64": {"bound": "alu", "kernel": "FP64 engine: gemm_f64_kernel + polar_compose_kernel",
                 "ms": prof["fp64_ms"], "achieved_units": prof["fp64_flops"],
                 "launches": prof["fp64_launches"], "peak": 1.10,
                 "peak_source": "measured cuBLAS DGEMM 8192^3 on this pool's GB300 (1.10 TFLOP/s)"},
        # double-float products: FP32 flops executed, 15 per multiply-add
        # (1 MUL + 3 FMA + 8 ADD), against the FP32 FMA peak from unit counts
        "df": {"bound": "alu", "kernel": "gemm_df_kernel (double-float Gram and apply products, "
                                         "FP32 pipes; with df_reduce_kernel)",
               "ms": prof.get("df_ms", 0.0), "achieved_units": prof.get("df_flops", 0.0) / 2 * 15,
               "launches": prof.get("df_launches", 0.0),
               "peak": sm_count * 128 * 2 * sm_ghz / 1e3,
               "peak_source": "152 SMs x 128 FP32 lanes x 2 flop/FMA x max SM clock (FP32 FMA peak); "
                              "the kernel's mix (8 of 12 instructions are adds) caps it at 0.625"},
        # the double-float polar composition (P x P products between grid barriers)
        "dfc": {"bound": "alu", "kernel": "polar_compose_df_kernel (double-float composition, "
                                          "persistent, grid barriers)",
                "ms": prof.get("dfc_ms", 0.0), "achieved_units": prof.get("dfc_flops", 0.0) / 2 * 15,
                "launches": prof.get("dfc_launches", 0.0),
                "peak": sm_count * 128 * 2 * sm_ghz / 1e3,
                "peak_source": "FP32 FMA peak as for df; latency-bound (two grid barriers per "
                               "Newton-Schulz step)"},
    }
    fam = {}
    for k, f in families.items():
        ach = f["achieved_units"] / (f["ms"] * 1e-3) / 1e12 if f["ms"] > 0 else 0.0
        fam[k] = {"bound": f["bound"], "kernel": f["kernel"], "achieved": ach, "peak": f["peak"],
                  "unit": f.get("unit", "TFLOP/s"), "frac": ach / f["peak"],
                  "peak_source": f["peak_source"],
                  "launches_per_sweep": f["launches"], "ms_per_sweep": f["ms"],
                  "share_of_sweep": f["ms"] / prof["total_ms"]}
    if prof.get("tc_launches"):
        # the bytes the traffic figure compares with: every operand read once
        # and the output written once, per launch
        fam["tc_hbm"]["algorithmic_bytes_per_launch"] = prof.get("tc_bytes", 0.0) / prof["tc_launches"]
    dom = max((k for k in fam if k != "tc_hbm"), key=lambda k: fam[k]["ms_per_sweep"])
    if dom == "tc" and fam["tc_hbm"]["frac"] > fam["tc"]["frac"]:
        dom = "tc_hbm"   # the products are bandwidth-bound: report that roofline
    roofline = dict(fam[dom], traffic=TRAFFIC.get(dom))
    if TRAFFIC.get(dom) is not None:
        roofline["traffic_source"] = ("stored ncu capture of the current kernels (cold cache, "
                                      "steady-state sweep 31), mean DRAM bytes per launch")

    out = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.prec == "fp64" else "f32(" + args.prec + ")+f64",
           "data": "synthetic (seeded QR-orthonormalised Gaussian isometries)",
           "config": dict(WORKLOAD, chi=chi, workload=f"tfim_chain_L1024_h1_chi{chi}",
                          precision=args.prec, chis=chis,
                          parallelism=("replicas x%d" % world) if world > 1 else "single GPU",
                          l2="working set %.0f MB > 129 MB L2" % (s.workspace.numel() / 1e6)),
           "tflops": flops_per_sweep * value / world / 1e12,
           "algorithmic_flops_per_sweep": flops_per_sweep,
           "gpu_launches": int(launches), "clocks": clk, "e2e": e2e, "roofline": roofline,
           "autotune": {"seconds": tune_s, "table_bytes": len(tiles_blob),
                        "product_shapes": max(0, (len(tiles_blob) - 16) // 32)},
           "roofline_families": fam,
           "profile": prof}

    if not args.quick:
        # Equal-energy comparison.  FP64 GPU path: 200 sweeps from the seeded
        # start; its FP64 energy E_ref is checked against the oracle's after the
        # same 200 sweeps.  Mixed path: sweeps in blocks of 10 until the FP64
        # energy of its tensors is <= E_ref (or 400 sweeps); reported are the
        # sweeps and the sweep time to get there, and the energy after 200.
        oracle_E = golden_final_energy(chi, 200)

        def sweep_time(t, n):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(t.stream)
            t.sweep_async(n)
            b.record(t.stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) * 1e-3

        f = Sweeper(model, chi, prec="fp64")
        f.set_isometries(0, ws, V)
        f.sweep(1)
        t_f = sweep_time(f, 199)
        E_ref = f.energy(0)
        f.close()
        t_f *= 200.0 / 199.0
        energy = {"target": "FP64 energy of the FP64 GPU path after 200 sweeps",
                  "fp64": {"sweeps": 200, "seconds": t_f, "E_fp64": E_ref,
                           "rel_err_vs_oracle_200": abs(E_ref - oracle_E) / abs(oracle_E) if oracle_E else None}}
        if args.prec != "fp64":
            g = Sweeper(model, chi, prec=args.prec, tiles=tiles_blob or None,
                        lanczos_tol=args.lanczos_tol)
            g.set_isometries(0, ws, V)
            g.sweep(1)
            done, secs, reached, E200 = 1, 0.0, None, None
            while done < 400:
                secs += sweep_time(g, 10)
                done += 10
                E = g.energy(0)
                if done >= 200 and E200 is None:
                    E200 = E
                if reached is None and E <= E_ref:
                    reached = {"sweeps": done, "seconds": secs, "E_fp64": E}
                if reached is not None and E200 is not None:
                    break
            g.close()
            energy[args.prec] = {
                "E_fp64_after_~200": E200,
                "rel_diff_vs_fp64_path_200": abs(E200 - E_ref) / abs(E_ref) if E200 else None,
                "reached_fp64_path_energy": reached,
                "speedup_at_equal_energy": (t_f / reached["seconds"]) if reached else None}
        out["energy"] = energy

    if rank == 0 and not args.no_baseline and world == 1:
        # the oracle on this host: 2 warm-up sweeps from the seeded start, then
        # the median of 3 timed sweeps, in a fresh process with the BLAS on
        # all cores (and, with --cpu-1thread, on one)
        ncores = os.cpu_count()
        ts = oracle_timing(chi, ncores)
        if ts:
            med = statistics.median(ts)
            out["cpu_baseline"] = {"value": 1.0 / med, "unit": "sweeps/s", "cores": ncores,
                                   "kind": "oracle", "cpu_model": cpu_model(),
                                   "sample": "median of 3 full oracle sweeps of the same workload "
                                             "after 2 warm-up sweeps from the seeded start "
                                             f"(BLAS threads {ncores}; seconds {ts})"}
        if args.cpu_1thread:
            t1 = oracle_timing(chi, 1, timeout=1800)
            if t1:
                out["cpu_baseline_1thread"] = {"value": 1.0 / statistics.median(t1),
                                               "unit": "sweeps/s", "cores": 1,
                                               "seconds": t1}
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_profile_only(args):
    """Eager sweeps (no CUDA graph) of the bench workload, for ncu."""
    import torch
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import Sweeper
    model = ti.tfim_chain(1024, 1.0)
    ws, V = ti.initial_tensors(1024, 2, args.chi, 1)
    tiles = open(args.tiles_file, "rb").read() if args.tiles_file else None
    s = Sweeper(model, args.chi, prec=args.prec, use_graph=False, tiles=tiles,
                lanczos_tol=args.lanczos_tol)
    s.set_isometries(0, ws, V)
    if tiles is None and not args.no_autotune:
        # the configurations the bench times (the tuning sweep is the first of the list)
        blob = s.autotune(reps=3)
        s.set_isometries(0, ws, V)
        if args.save_tiles and blob:
            # a later run under ncu loads this table: timings taken under the
            # profiler would choose other configurations
            with open(args.save_tiles, "wb") as f:
                f.write(blob)
    if args.profile_start:
        s.sweep(args.profile_start)     # towards the steady state the bench times
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    E = s.sweep(args.profile_sweeps)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_sweeps": args.profile_sweeps, "profile_start": args.profile_start,
                      "prec": args.prec, "energies": E[:, 0].tolist(),
                      "launches_per_sweep": s.launch_count / max(1, args.profile_sweeps)}))
    s.close()


def run_batched(args):
    """64 independent TFIM chains (h ~ U[0.5,1.5], L ~ {64..512}, chi ~ {32,64,128},
    seed 4) advanced together in one context and one captured sweep.  Under
    torchrun the chains are sharded by instance (cost-balanced, no collective
    on the data path): each rank advances its own share, the job's time is the
    slowest rank's and the throughput counts every rank's instance-sweeps."""
    import torch
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import Sweeper, instance_cost, shard_instances
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wls_all = ti.batched_chains()
    mine = shard_instances([instance_cost(w.model.Lx, w.chi) for w in wls_all], world, rank)
    wls = [wls_all[i] for i in mine]
    s = Sweeper([w.model for w in wls], [w.chi for w in wls], prec=args.prec)
    for i, w in enumerate(wls):
        s.set_isometries(i, *ti.initial_tensors(w.model.Lx, 2, w.chi, w.seed))
    # per-instance error of the first sweep's energy against the oracle's
    # (the stored values written by oracle/make_golden.py), per site
    E1 = s.sweep(1)[0]
    err = None
    gpath = os.path.join(ROOT, "tests", "golden", "oracle_batched64_first_sweep.json")
    if os.path.exists(gpath):
        with open(gpath) as f:
            gold = json.load(f)["instances"]
        err = [abs(E1[k] - gold[i]["first_sweep_energy"]) / wls_all[i].model.Lx
               for k, i in enumerate(mine)]
    if args.warmup > 1:
        s.sweep(args.warmup - 1)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s.stream)
    s.sweep_async(args.steps)
    b.record(s.stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = a.elapsed_time(b)
    # throughput over all ranks: instance-sweeps of the whole job / slowest rank
    ms_max = ms
    total = len(wls) * args.steps
    if dist is not None:
        t = torch.tensor([ms, float(total)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        ms_max, total = float(tmax[0]), float(t[1])
    if rank == 0:
        print(json.dumps({"metric": "batched TTN sweeps/s (64 independent chains, instance-sweeps)",
                          "value": total / (ms_max * 1e-3), "unit": "instance-sweeps/s",
                          "n_gpus": world, "scaling": "strong", "ms_per_step": ms_max / args.steps,
                          "steps": args.steps, "warmup": args.warmup, "precision": args.prec,
                          "instances": len(wls_all), "instances_rank0": len(wls),
                          "parallelism": ("instances sharded over %d ranks" % world) if world > 1
                          else "single GPU", "gpu_launches": s.launch_count,
                          "first_sweep_energy_error_vs_oracle": None if err is None else {
                              "max": max(err), "median": statistics.median(err),
                              "unit": "energy per site",
                              "instances": len(err)}}))
    s.close()
    if dist is not None:
        dist.destroy_process_group()


def run_paper_torus(args):
    """The paper's workload (Sec. IV): 128 x 5 thin torus, h = 2.9, d0 = 32,
    K = 5; energy per spin and the entanglement spectrum / entropy of the
    block of 2^6 columns (site layer 6, leftmost site)."""
    import numpy as np
    import torch
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import Sweeper
    m = ti.tfim_torus(128, 5, 2.9)
    chi = args.chi
    ws, V = ti.initial_tensors(128, m.d0, chi, 5)
    s = Sweeper(m, chi, prec=args.prec)
    s.set_isometries(0, ws, V)
    t0 = time.perf_counter()
    # Sec. IV: sweep until the energy per spin changes by less than 1e-10
    converged, E = s.sweep_until(tol=1e-10, max_sweeps=args.steps)
    E = E[:, 0]
    dt = time.perf_counter() - t0
    E_cert = s.energy(0)
    rho = s.rdm(0, 6, which=1)
    p = np.clip(np.linalg.eigvalsh(0.5 * (rho + rho.T))[::-1], 1e-300, None)
    lam = -np.log2(p)
    S = float(-np.sum(p * np.log2(p)))
    n = len(E)
    marks = sorted({k for k in (1, 10, 50, 100, 200, 500, 1000, 2000, 5000) if k <= n} | {n})
    print(json.dumps({"workload": "paper torus 128x5 h=2.9", "chi": chi, "precision": args.prec,
                      "sweeps": n, "converged_1e-10": bool(converged), "sweeps_per_s": n / dt,
                      "energy_per_spin_fp64": E_cert / m.n_spins,
                      "energy_per_spin_at_sweep": {str(k): float(E[k - 1] / m.n_spins) for k in marks},
                      "last_delta_e_per_spin": float(abs(E[-1] - E[-2]) / m.n_spins)
                      if len(E) > 1 else None,
                      "paper_e_inf": -3.11229, "entanglement_spectrum_tau6_first30": lam[:30].tolist(),
                      "entropy_tau6": S}))
    s.close()


def _oracle_sweep_seconds(workload_expr, threads, sweeps=1):
    """Seconds per oracle sweep of a workload in a fresh process with the BLAS
    limited to `threads` threads (the CPU baseline of the config table)."""
    code = ("import time, ttn_inputs as ti\n"
            "from oracle import ttn as oracle\n"
            f"w = {workload_expr}\n"
            "ws, V = ti.initial_tensors(w.model.Lx, w.model.d0, w.chi, w.seed, w.per_node)\n"
            "st = oracle.make_state(w.model, ws, V, per_node=w.per_node)\n"
            "oracle.sweep(st)\n"
            "t0 = time.perf_counter()\n"
            f"for _ in range({sweeps}): oracle.sweep(st)\n"
            f"print((time.perf_counter() - t0) / {sweeps})\n")
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=1800)
    return float(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None


def run_configs(args):
    """The five configurations: GPU FP64 and mixed-precision sweeps/s, FP64
    parity against the oracle's stored trajectories, FP64-certified energies
    of the mixed paths, and the oracle's seconds per sweep on the host cores.
    One JSON line per configuration."""
    import numpy as np
    import torch
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import Sweeper

    def golden(name):
        path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
        if not os.path.exists(path):
            return None
        with open(path) as f:
            return json.load(f)

    def timed(s, n):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        s.sweep_async(n)
        b.record(s.stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e-3

    def gpu_run(w, prec, n):
        s = Sweeper(w.model, w.chi, per_node=w.per_node, prec=prec)
        s.set_isometries(0, *ti.initial_tensors(w.model.Lx, w.model.d0, w.chi, w.seed, w.per_node))
        E = s.sweep(n)[:, 0]                      # trajectory from the seeded start
        cert = s.energy(0)
        k = min(n, 20)
        dt = timed(s, k)                          # throughput, warm
        s.close()
        return E, cert, k / dt

    ncores = os.cpu_count()
    rows = [("ti.tfim_l16_pernode()", ti.tfim_l16_pernode(), ["fp64", "tf32x3"], True),
            ("ti.tfim_l1024(32)", ti.tfim_l1024(32), ["fp64", "tf32x3", "tf32"], True),
            ("ti.tfim_l1024(64)", ti.tfim_l1024(64), ["fp64", "tf32x3", "tf32"], False),
            ("ti.tfim_l1024(128)", ti.tfim_l1024(128), ["fp64", "tf32x3", "tf32"], False),
            ("ti.heisenberg_l256(256)", ti.heisenberg_l256(256), ["fp64", "bf16x3"], False),
            ("ti.torus_64x4(128)", ti.torus_64x4(128), ["fp64", "tf32", "tf32x3"], False)]
    for expr, w, precs, one_core in rows:
        g = golden(w.name)
        line = {"config": w.name, "chi": w.chi, "K": w.model.K, "d0": w.model.d0}
        for prec in precs:
            if prec == "fp64":
                n = g["sweeps"] if g else 4
            else:
                n = 20 if w.name.startswith("heisenberg") else w.sweeps
            E, cert, sps = gpu_run(w, prec, n)
            r = {"sweeps": n, "sweeps_per_s": sps, "E_certified_fp64": cert,
                 "energy_per_spin": cert / w.model.n_spins}
            if g and len(g["energies"]) >= n:
                ref = np.array(g["energies"][:n])
                r["max_rel_err_vs_oracle_trajectory"] = float((np.abs(E - ref) / np.abs(ref)).max())
                if n == g["sweeps"]:
                    r["rel_err_certified_vs_oracle"] = abs(cert - g["final_energy"]) / abs(g["final_energy"])
            line[prec] = r
        line["oracle_s_per_sweep"] = {f"{ncores}_threads": _oracle_sweep_seconds(expr, ncores)}
        if one_core:
            line["oracle_s_per_sweep"]["1_thread"] = _oracle_sweep_seconds(expr, 1)
        print(json.dumps(line), flush=True)


def run_top_mode_study(args):
    """Top update read two ways (Sec. III.B, "updated similarly"): the exact
    lowest eigenvector (top_mode 0) against minus the polar factor of the top
    tensor's environment (top_mode 1), FP64, from the same seeded start:
    energies along the sweeps and sweeps needed to come within 1e-6 (relative)
    of the eigensolver's final energy."""
    import numpy as np
    import torch
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import Sweeper
    L, chi, n = 256, args.chi, args.steps
    model = ti.tfim_chain(L, 1.0)
    ws, V = ti.initial_tensors(L, 2, chi, 1)
    out = {"workload": f"tfim_chain_L{L}_h1_chi{chi}", "precision": "fp64", "sweeps": n}
    Es = {}
    for mode in (0, 1):
        s = Sweeper(model, chi, prec="fp64", top_mode=mode)
        s.set_isometries(0, ws, V)
        t0 = time.perf_counter()
        s.sweep(n)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        s.set_isometries(0, ws, V)
        E = []
        for _ in range(n):
            s.sweep(1)
            E.append(s.energy(0))
        s.close()
        Es[mode] = np.array(E)
        out[f"top_mode_{mode}"] = {"sweeps_per_s": n / dt,
                                   "energy_at": {str(k): float(Es[mode][k - 1]) for k in
                                                 (1, 5, 10, 25, 50, 100, 200, n) if k <= n}}
    ref = Es[0][-1]
    for mode in (0, 1):
        hit = np.nonzero(np.abs(Es[mode] - ref) / abs(ref) < 1e-6)[0]
        out[f"top_mode_{mode}"]["sweeps_to_1e-6_of_eig_final"] = int(hit[0]) + 1 if len(hit) else None
    print(json.dumps(out))


def run_polar_study(args):
    """Sec. III.B / Fig. 9: the update from the SVD of the environment (Fig.
    9a) against the EVD of its Gram matrix (Fig. 9b: E^T E = V S^2 V^T,
    w = V S^-1 V^T E^T) and the Newton-Schulz schedule the library uses (FP64
    mode: blocks of at most four scaled steps per fresh Gram matrix), on the
    damped environments Gamma - mu |Gamma| w of the full layers of the TFIM
    L=1024 chain at chi (state after 20 FP64 sweeps).  All three in FP64 on the
    GPU with torch (cuSOLVER / cuBLAS): the distance of each factor to the
    SVD's, its isometry defect, and its time."""
    import numpy as np
    import torch
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import Sweeper
    chi = args.chi
    model = ti.tfim_chain(1024, 1.0)
    ws, V = ti.initial_tensors(1024, 2, chi, 1)
    s = Sweeper(model, chi, prec="fp64")
    s.set_isometries(0, ws, V)
    s.sweep(20)
    ws, V = s.get_isometries(0)
    mu = 1e-7

    def timed(f, reps=5):
        f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = f()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) / reps * 1e3

    def ns_schedule(l0, gmax=30.0, maxb=4):
        out, l, cur, start = [], l0, [], l0
        while 1 - l > 1e-15 and len(out) + len(cur) < 200:
            c = math.sqrt(3 / (1 + l + l * l))
            ln = 1.5 * c * l - 0.5 * c ** 3 * l ** 3
            if cur and (ln / start > gmax or len(cur) >= maxb):
                out.append(cur)
                cur, start = [], l
            cur.append((1.5 * c, 0.5 * c ** 3))
            l = ln
        if cur:
            out.append(cur)
        return out

    sched = ns_schedule(mu / 4)
    rows = []
    for t, w in enumerate(ws):
        P, n = w.shape[0], w.shape[1]
        if P < 64:
            continue
        g = s.env(0, t).reshape(P, n * n)
        W0 = torch.tensor(w.reshape(P, n * n), device="cuda")
        G = g - mu * torch.linalg.norm(g) * W0

        def svd():
            U, S, Vh = torch.linalg.svd(G, full_matrices=False)
            return -(U @ Vh)

        def evd():
            ev, Q = torch.linalg.eigh(G @ G.T)
            ev = torch.clamp(ev, min=1e-300)
            return -((Q * ev.rsqrt()) @ Q.T) @ G

        def ns():
            X = G / torch.linalg.norm(G)
            I = torch.eye(P, dtype=torch.float64, device="cuda")
            for blk in sched:
                A = X @ X.T
                F = I.clone()
                for a, c in blk:
                    Pm = a * I - c * A
                    F = Pm @ F
                    A = Pm @ A @ Pm
                    A = 0.5 * (A + A.T)
                X = F @ X
            return -X

        Wsvd, t_svd = timed(svd)
        row = {"layer": t, "P": P, "n2": n * n, "ms_svd": t_svd}
        U, S, Vh = torch.linalg.svd(G, full_matrices=False)
        row["sigma_min_over_max"] = float(S[-1] / S[0])
        for name, f in (("evd", evd), ("newton_schulz", ns)):
            Wx, ms = timed(f)
            I = torch.eye(P, dtype=torch.float64, device="cuda")
            row[name] = {"ms": ms, "max_abs_diff_vs_svd": float((Wx - Wsvd).abs().max()),
                         "isometry_defect": float((Wx @ Wx.T - I).abs().max())}
        rows.append(row)
    s.close()
    print(json.dumps({"study": "polar factor of the damped environment: SVD (Fig. 9a) vs EVD "
                               "(Fig. 9b) vs Newton-Schulz (FP64, torch on the GPU)",
                      "workload": f"tfim_chain_L1024_h1_chi{chi}, state after 20 FP64 sweeps",
                      "mu": mu, "ns_steps": sum(len(b) for b in sched), "ns_blocks": len(sched),
                      "layers": rows}))


def main():
    args = parse()
    if args.workload == "top-mode":
        run_top_mode_study(args)
        return
    if args.workload == "polar-study":
        run_polar_study(args)
        return
    if args.workload == "configs":
        run_configs(args)
        return
    if args.workload == "batched64":
        run_batched(args)
        return
    if args.workload == "paper-torus":
        run_paper_torus(args)
        return
    if args.profile_sweeps:
        run_profile_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Throughput of the Gutzwiller-projection PQMC sweep on GB300.

Workload: Gutzwiller PQMC on the 6x6 honeycomb cluster (72 sites), Hubbard
U = 4, half filling, trial = Neel mean-field Slater determinant (M_N = 0.21)
times exp(-g sum n_up n_dn) with g = 0.6 as extra HS slices, dtau = 0.1,
2 Theta = 8 (80 interaction slices + 2 Gutzwiller slices), a batch of
independent chains per GPU.  Synthetic: the model Hamiltonian and seeded
Philox fields are the whole input.

One step = one sweep of every chain (each proposes all (Ltau+2) N fields
once); metric = HS-field updates/s summed over chains and GPUs.

  python bench.py [--gpus N --steps K --warmup W] [--prec fp32|fp64] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the slow reference program) on the host cores on a bounded sample of the
same workload.
"""
import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(kind=0, Lx=6, Ly=6, t=1.0, tp=0.0, U=4.0, dtau=0.1, two_theta=8.0, g=0.6, M_N=0.21)
METRIC = "HS-field updates/s & time-to-sigma(E)=1e-3, FP32/3xBF16 vs FP64 PQMC, one GB300"
UNIT = "updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--chains", type=int, default=608, help="chains per GPU (4 per SM)")
    ap.add_argument("--two-theta", type=float, default=8.0)
    ap.add_argument("--n-stab", type=int, default=0, help="0: 4 for fp32, 10 for fp64")
    ap.add_argument("--fp64-steps", type=int, default=2, help="steps of the FP64 path timed beside (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


# ---------------------------------------------------------------- CPU oracle
def _oracle_worker(args):
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    chain, two_theta, n_stab, seconds = args
    from oracle import pqmc as opq
    p = opq.Params(n_stab=n_stab, seed=1, chain=chain, **{**WORKLOAD, "two_theta": two_theta})
    ch = opq.Chain(p)
    props = (ch.m.Ltau + 2) * ch.m.N
    t0 = time.perf_counter()
    n = 0
    while True:
        ch.sweep(measure=True)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return n * props, time.perf_counter() - t0


def oracle_rate(two_theta, n_stab, seconds, cores=None):
    """Oracle updates/s with one chain per host core (spawned processes,
    one BLAS thread each), each sweeping for about `seconds`."""
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(c, two_theta, n_stab, seconds) for c in range(cores)])
    updates = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return updates / wall, cores, updates


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp32_peak_tflops(sm_mhz):
    """FP32 FFMA peak: 152 SMs x 128 lanes x 2 flop x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def algorithmic_flops(N, n_sigma, Ltau, n_stab, acc):
    """Per sweep per chain, both spins (see the measurement section of the design doc):
    wrap 4 N^3 and delayed-update flush 2 acc N^3 per interaction slice per spin
    (path precision); stack products 2 N^2 n_sigma per slice per spin, and per
    stabilisation per spin: QR 2 n^2 (N - n/3), Q_L^T Q_R 2 n^2 N,
    LU + solve 2/3 n^3 + 2 n^2 N, G assembly 2 N^2 n (FP64)."""
    n = n_sigma
    path = 2 * Ltau * (4 * N ** 3 + 2 * acc * N ** 3)
    n_stab_pts = Ltau // n_stab + 1
    fp64 = 2 * (Ltau * 2 * N * N * n
                + n_stab_pts * (2 * n * n * (N - n / 3) + 2 * n * n * N + 2 / 3 * n ** 3 + 2 * n * n * N
                                + 2 * N * N * n))
    return path, fp64


# ---------------------------------------------------------------- our arm
def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2303_13403_gb300 import pqmc, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = {"fp32": pqmc.FP32, "fp64": pqmc.FP64}[a.prec]
    n_stab = a.n_stab or (4 if prec != pqmc.FP64 else 10)
    spec = workloads.ChainSpec(**{**WORKLOAD, "two_theta": a.two_theta})
    specs = [spec] * a.chains
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(prec_, n_stab_, steps, warmup):
        ctx = pqmc.Context(specs, prec=prec_, seed=1, n_stab=n_stab_, chain_offset=rank * a.chains,
                           max_meas=warmup + steps + 1, stream=stream.cuda_stream)
        for _ in range(warmup):
            ctx.sweep(1, measure=True)
        ctx.synchronize()
        torch.cuda.synchronize()
        barrier()
        clk = ClockSampler(local)
        clk.start()
        time.sleep(0.3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.sweep(1, measure=True)
        e1.record(stream)
        e1.synchronize()
        ctx.synchronize()
        torch.cuda.synchronize()
        barrier()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        obs = ctx.measure(-1)
        launches = ctx.launch_count()
        dims = ctx.dims(0)
        ctx.close()
        return float(t.item()), clocks, obs, launches, dims

    ms, clocks, obs, launches, d = timed(prec, n_stab, a.steps, a.warmup)
    N, Ltau = d["N"], d["Ltau"]
    props_per_chain = (Ltau + 2) * N
    updates = props_per_chain * a.chains * world * a.steps
    value = updates / (ms / 1e3)

    # FP64 path timed beside it (the plain FP64 GPU sweep the reduced paths must beat)
    fp64 = None
    if prec != pqmc.FP64 and a.fp64_steps > 0:
        ms64, _, obs64, _, _ = timed(pqmc.FP64, 10, a.fp64_steps, 1)
        fp64 = {"value": props_per_chain * a.chains * world * a.fp64_steps / (ms64 / 1e3), "unit": UNIT,
                "n_stab": 10, "ms_per_step": ms64 / a.fp64_steps, "max_dG": obs64["max_dG"]}

    # end to end through the public API with host buffers: context creation
    # (host model set-up + upload of the arena from host memory) and, every
    # step, one sweep plus the device->host read of every chain's new record
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    ctx = pqmc.Context(specs, prec=prec, seed=2, n_stab=n_stab, chain_offset=rank * a.chains,
                       max_meas=a.steps + 1, stream=stream.cuda_stream)
    h2d = ctx.device_bytes()
    rec = np.zeros((a.chains, 5))
    d2h = 0
    for _ in range(a.steps):
        ctx.sweep(1, measure=True)
        ctx.last_records(rec)
        d2h += rec.nbytes
    t_e2e = time.perf_counter() - t0
    t = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = updates / float(t.item())
    ctx.close()

    path_flops, fp64_flops = algorithmic_flops(N, N // 2, Ltau, n_stab, obs["accept"])
    launch_s = ms / 1e3 / a.steps                     # one sweep launch per step
    achieved = path_flops * a.chains / launch_s / 1e12
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = fp32_peak_tflops(2070.0) if prec == pqmc.FP32 else 1.2
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64"}[a.prec], "data": "synthetic",
        "config": {"workload": "gutzwiller_pqmc_honeycomb_6x6_U4_g0.6_MN0.21_2theta%g" % a.two_theta,
                   "sites": N, "slices": Ltau + 2, "chains_per_gpu": a.chains, "global_chains": a.chains * world,
                   "n_stab": n_stab, "delay_block": 32, "precision": a.prec,
                   "l2": "state larger than L2 (%.0f MB of chain state per GPU vs 129 MB L2)" %
                         (a.chains * (2 * 2 * N * N * (4 if prec != pqmc.FP64 else 8)
                                      + 4 * (Ltau // n_stab + 1) * N * (N // 2) * 8) / 1e6),
                   "parallelism": "chains%d" % world},
        "clocks": clocks,
        "gpu_launches": launches,
        "accept": obs["accept"], "max_dG": obs["max_dG"], "E_per_site": obs["E"], "E_err": obs["E_err"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "sweep_kernel", "peak_source": "FP32 FFMA 152x128x2 at 2070 MHz" if prec == pqmc.FP32
                     else "FP64 measured 1.2 TFLOP/s (FMA probe)"},
        "fp64_flops_per_sweep": fp64_flops * a.chains,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // max(a.steps, 1),
                "d2h_bytes_per_step": d2h // max(a.steps, 1),
                "note": "timed: context creation (host FP64 model build, upload of the whole device arena "
                        "from host memory, device initialisation) + per step one sweep and the device-to-host "
                        "read of every chain's new measurement; h2d is the arena upload spread over the steps"},
    }
    if fp64:
        result["fp64_gpu"] = fp64
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        rate, cores, n_upd = oracle_rate(a.two_theta, n_stab, a.cpu_seconds)
        result["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": "%d oracle chains (one per core), ~%gs of sweeps each, %d updates" %
                                            (cores, a.cpu_seconds, n_upd)}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_stab = a.n_stab or (4 if a.prec != "fp64" else 10)
    seconds = max(2.0, min(10.0, 120.0 / max(a.steps + a.warmup, 1)))
    for _ in range(a.warmup):
        oracle_rate(a.two_theta, n_stab, 0.5)
    rates = []
    total_upd = 0
    t0 = time.perf_counter()
    for _ in range(a.steps):
        r, cores, n = oracle_rate(a.two_theta, n_stab, seconds)
        rates.append(r)
        total_upd += n
    wall = time.perf_counter() - t0
    value = sum(rates) / len(rates)
    sample = "%d oracle chains (one per core) sweeping ~%gs per step" % (cores, seconds)
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": wall / a.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "gutzwiller_pqmc_honeycomb_6x6_U4_g0.6_MN0.21_2theta%g" % a.two_theta,
                   "sites": 72, "n_stab": n_stab, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()

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

  python bench.py [--gpus N --steps K --warmup W] [--prec fp32|bf16x3|fp64] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the slow reference program) on the host cores on a bounded sample of the
same workload.
"""
import argparse
import json
import multiprocessing as mp
import os
import platform
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
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16x3", "fp64"])
    ap.add_argument("--chains", type=int, default=608, help="chains per GPU (two waves of 2 chains per SM)")
    ap.add_argument("--two-theta", type=float, default=8.0)
    ap.add_argument("--n-stab", type=int, default=0, help="0: 2 for fp32 and bf16x3, 10 for fp64")
    ap.add_argument("--beside-steps", type=int, default=1,
                    help="nonzero: time the other precisions beside the head with the same --steps/--warmup")
    ap.add_argument("--tts-sweeps", type=int, default=40,
                    help="sweeps of the time-to-sigma run of every precision (0: skip)")
    ap.add_argument("--dg-chains", type=int, default=64,
                    help="chains of the max|G - G_FP64| diagnostic of the reduced paths (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cta-threads", type=int, default=0, help="threads per chain CTA (0: autotuned)")
    ap.add_argument("--delay-k", type=int, default=0, help="delayed-update block (0: autotuned)")
    ap.add_argument("--large-sweeps", type=int, default=3,
                    help="timed sweeps of the single 648-site chain swept by the whole GPU (0: skip)")
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


def cpu_model():
    """The host CPU as the kernel reports it (model name on x86, the
    implementer / part codes on Arm), else the machine type."""
    try:
        info = {}
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                info.setdefault(k.strip().lower(), v.strip())
        if "model name" in info:
            return info["model name"]
        if "cpu part" in info:
            return "%s, CPU implementer %s part %s" % (platform.machine(), info.get("cpu implementer", "?"),
                                                      info["cpu part"])
    except OSError:
        pass
    return platform.machine()


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


# ---------------------------------------------------------------- our arm
def sweep_flops(N, n, Ltau, n_stab, acc, prec):
    """Algorithmic flops per sweep per chain, both spins: (path-precision, FP64).

    Path precision, per interaction slice per spin: wrap 4 N^3, delayed-update
    flush 2 acc N^3, stack slice products 2 N^2 n.  FP64, per stabilisation per
    spin, Ltau / n_stab stabilisations per sweep: the QR of the N x n stack
    block 2 n^2 (N - n/3), the overlap Q_L^T Q_R 2 n^2 N and its inverse 2 n^3
    (the method's arithmetic, whatever QR variant the kernel runs; the
    kernel's Cholesky QR on the reduced paths does more, N n (n + 1) + n^3/3
    + N n^2, and is not counted)."""
    path = 2 * Ltau * (4 * N ** 3 + 2 * acc * N ** 3 + 2 * N * N * n)
    stab = (Ltau // n_stab) * 2 * (2 * n * n * (N - n / 3) + 2 * n * n * N + 2 * n ** 3)
    return path, stab


# FP64 peak from the unit counts and the clock: 152 SMs x 2 FP64 FMA lanes per
# clock x 2 flop x 2070 MHz = 1.26 TFLOP/s, the part's nominal 1.25 TFLOP/s
# (an FMA-throughput probe on this machine measured 1.2 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2070e6 / 1e12

# DRAM bytes (read + write) per chain and sweep of the sweep kernel, by
# (precision, N, Ltau, delayed block, CTA threads), from one ncu capture of
# that launch shape (profiles/sweep_kernel_gutz72_ncu.md: 304 chains, one
# sweep, 550.7 + 499.6 MB).
DRAM_BYTES_PER_CHAIN_SWEEP = {("fp32", 72, 80, 32, 256): (550.736384e6 + 499.562496e6) / 304}


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2303_13403_gb300 import distributed, pqmc, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    PRECS = {"fp32": pqmc.FP32, "bf16x3": pqmc.BF16X3, "fp64": pqmc.FP64}
    NSTAB = {"fp32": 2, "bf16x3": 2, "fp64": 10}
    spec = workloads.ChainSpec(**{**WORKLOAD, "two_theta": a.two_theta})
    specs = [spec] * a.chains
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    tuned = {}

    def tune(name, n_stab_):
        # the library's autotuner (delayed block and CTA shape) on this batch;
        # contexts created with delay_k = 0 then take the cached pick
        if name not in tuned:
            tuned[name] = pqmc.autotune(specs, prec=PRECS[name], n_stab=n_stab_, cta_threads=a.cta_threads,
                                        delay_k=a.delay_k)
        return tuned[name]

    def timed(name, n_stab_, steps, warmup, clocks=False):
        tune(name, n_stab_)
        ctx = pqmc.Context(specs, prec=PRECS[name], seed=1, n_stab=n_stab_, chain_offset=rank * a.chains,
                           max_meas=warmup + steps + 1, stream=stream.cuda_stream, cta_threads=a.cta_threads,
                           delay_k=0)
        for _ in range(warmup):
            ctx.sweep(1, measure=False)
        ctx.synchronize()
        torch.cuda.synchronize()
        barrier()
        clk = ClockSampler(local) if clocks else None
        if clk:
            clk.start()
            time.sleep(0.3)
        launches0 = ctx.launch_count()
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
        cl = clk.stop() if clk else None
        ms = e0.elapsed_time(e1)
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        obs = ctx.measure(-1)
        # pooled over the chains of every rank (jackknife over chains)
        sums = distributed.chain_sums([ctx.measurements(c, cap=steps + 1) for c in range(a.chains)])
        if world > 1:
            sums = distributed.gather_sums(sums)
        pooled = distributed.pooled_estimate(sums)
        obs["E"], obs["E_err"] = pooled["E"], pooled["E_err"]
        # per-stabilisation errors of 64 chains; the first sweep starts from
        # the random initial fields (burn-in) and is reported apart
        d = ctx.dims(0)
        per_sweep = d["Ltau"] // d["n_stab"] + 1
        hist = [ctx.stab_errors(c, cap=4096) for c in range(min(a.chains, 64))]
        errs = np.concatenate([h[per_sweep:] for h in hist])
        first = np.concatenate([h[:per_sweep] for h in hist])
        out = {"ms": float(t.item()), "clocks": cl, "obs": obs, "launches": ctx.launch_count() - launches0,
               "dims": d, "dG": errs, "dG_first": first, "launch": ctx.launch()}
        ctx.close()
        return out

    def summary(name, r, steps):
        N, Ltau = r["dims"]["N"], r["dims"]["Ltau"]
        props = (Ltau + 2) * N
        ups = props * a.chains * world * steps / (r["ms"] / 1e3)
        o = r["obs"]
        dg = r["dG"]
        return {"value": ups, "unit": UNIT, "n_stab": NSTAB[name] if not a.n_stab else a.n_stab,
                "delay_block": r["launch"]["delay_k"], "cta_threads": r["launch"]["cta_threads"],
                "ms_per_step": r["ms"] / steps, "E_per_site": o["E"], "E_err": o["E_err"], "accept": o["accept"],
                "dG_per_stabilisation": {"median": float(np.median(dg)), "p99": float(np.percentile(dg, 99)),
                                         "p999": float(np.percentile(dg, 99.9)), "max": float(dg.max()),
                                         "after": "the first sweep",
                                         "first_sweep_max": float(r["dG_first"].max()),
                                         "against": "G rebuilt from the stacks in the path precision"}}

    def time_to_sigma(name, n_sweeps):
        """Wall time to sigma(E/site) = 1e-3, warm-up included (the time a
        user waits for that error bar from a fresh start): a fresh context of the bench's chains runs n_sweeps
        measured sweeps, each timed with CUDA events on the context's
        stream.  The warm-up length is the shortest of 2, 4, 8, 12, 16 sweeps
        after which the pooled E/site of the first and second halves of the
        remaining sweeps agree within 2 sigma; sigma after k further sweeps
        is the jackknife over chains of the per-chain averages of those k
        sweeps; the time is that of the warm-up plus the first k whose sigma
        reaches 1e-3 (extrapolated as t (sigma / 1e-3)^2 past the end of the
        run, and flagged)."""
        ns = a.n_stab or NSTAB[name]
        tune(name, ns)
        ctx = pqmc.Context(specs, prec=PRECS[name], seed=7, n_stab=ns, chain_offset=rank * a.chains,
                           max_meas=n_sweeps + 1, stream=stream.cuda_stream, cta_threads=a.cta_threads,
                           delay_k=0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_sweeps + 1)]
        ev[0].record(stream)
        for k in range(n_sweeps):
            ctx.sweep(1, measure=True)
            ev[k + 1].record(stream)
        ev[-1].synchronize()
        ctx.synchronize()
        t_cum = np.array([0.0] + [ev[0].elapsed_time(e) / 1e3 for e in ev[1:]])
        recs = np.stack([ctx.measurements(c, cap=n_sweeps + 1) for c in range(a.chains)])  # chains x sweeps x 6
        ctx.close()

        def pooled(r):
            sums = distributed.chain_sums(list(r))
            if world > 1:
                sums = distributed.gather_sums(sums)
            return distributed.pooled_estimate(sums)

        w_eq, halves = None, None
        for w in (2, 4, 8, 12, 16):
            rest = n_sweeps - w
            if rest < 4:
                break
            h1, h2 = pooled(recs[:, w:w + rest // 2]), pooled(recs[:, w + rest // 2:])
            halves = (h1["E"], h1["E_err"], h2["E"], h2["E_err"])
            if abs(h1["E"] - h2["E"]) <= 2 * np.hypot(h1["E_err"], h2["E_err"]):
                w_eq = w
                break
        equilibrated = w_eq is not None
        if w_eq is None:
            w_eq = min(16, n_sweeps // 2)
        t_tts, k_hit, sig = None, None, None
        for k in range(2, n_sweeps - w_eq + 1):
            sig = pooled(recs[:, w_eq:w_eq + k])["E_err"]
            if sig <= 1e-3:
                k_hit = k
                t_tts = t_cum[w_eq + k]
                break
        final = pooled(recs[:, w_eq:])
        if k_hit is None:
            sig = final["E_err"]
            t_tts = t_cum[w_eq] + (t_cum[-1] - t_cum[w_eq]) * (sig / 1e-3) ** 2
        return {"seconds": float(t_tts), "extrapolated": k_hit is None,
                "warmup_sweeps": int(w_eq), "equilibrated": bool(equilibrated),
                "measured_sweeps_to_sigma": k_hit, "sweeps_run": n_sweeps,
                "ms_per_sweep": float(1e3 * t_cum[-1] / n_sweeps),
                "E_per_site": final["E"], "E_err": final["E_err"],
                "E_halves": halves, "n_stab": ns}

    def dg_vs_fp64(name, chains=64, sweeps=6):
        """Per-stabilisation max |G - G_FP64| with G_FP64 assembled in FP64 from
        the FP64 factors (opts.dg_fp64 = 1), and the same divided by
        max(1, max |G_FP64|) (dg_fp64 = 3), over `chains` chains from one seed
        (the diagnostic does not change the chain); the first sweep, which
        starts from the random initial fields, is reported apart."""
        ns = a.n_stab or NSTAB[name]
        out = {}
        for mode, key in ((1, "absolute"), (3, "relative")):
            ctx = pqmc.Context([spec] * chains, prec=PRECS[name], seed=3, n_stab=ns, stream=stream.cuda_stream,
                               dg_fp64=mode, delay_k=32)
            ctx.sweep(sweeps, measure=False)
            ctx.synchronize()
            d = ctx.dims(0)
            per_sweep = d["Ltau"] // d["n_stab"] + 1
            hist = [ctx.stab_errors(c, cap=4096) for c in range(chains)]
            ctx.close()
            errs = np.concatenate([h[per_sweep:] for h in hist])
            first = np.concatenate([h[:per_sweep] for h in hist])
            out[key] = {"median": float(np.median(errs)), "p99": float(np.percentile(errs, 99)),
                        "p999": float(np.percentile(errs, 99.9)), "max": float(errs.max()),
                        "frac_above_1e-4": float(np.mean(errs > 1e-4)), "stabilisations": int(errs.size),
                        "first_sweep_max": float(first.max())}
        out["after"] = "the first sweep"
        out["sample"] = "%d chains x %d sweeps, n_stab %d" % (chains, sweeps, ns)
        out["against"] = ("G_FP64 = 1 - Q_R (Q_L^T Q_R)^-1 Q_L^T assembled in FP64 from the FP64 factors; "
                          "relative: divided by max(1, max|G_FP64|) per spin")
        return out

    def large_chain(name, n_stab_, sweeps, warmup=2):
        """One 648-site chain (18x18 honeycomb, 2 Theta = 20) swept by the
        whole GPU (opts.spread): context creation, `warmup` sweeps (one
        captured graph per sweep direction), then `sweeps` sweeps timed with
        CUDA events."""
        lspec = workloads.honeycomb(18, U=4.0, dtau=0.1, two_theta=20.0, g=0.6, M_N=0.21)
        t0 = time.perf_counter()
        ctx = pqmc.Context([lspec], prec=PRECS[name], seed=7, n_stab=n_stab_, stream=stream.cuda_stream, spread=1)
        ctx.synchronize()
        t_init = time.perf_counter() - t0
        ctx.sweep(warmup, measure=False)
        ctx.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = ctx.launch_count()
        e0.record(stream)
        ctx.sweep(sweeps, measure=True)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / sweeps
        d = ctx.dims(0)
        obs = ctx.measure(0)
        errs = ctx.stab_errors(0, cap=4096)
        out = {"ms_per_sweep": ms, "updates_per_s": (d["Ltau"] + 2) * d["N"] / (ms / 1e3), "n_stab": n_stab_,
               "context_creation_s": t_init, "kernels_per_sweep": (ctx.launch_count() - n0) / sweeps,
               "E_per_site_last_sweeps": float(np.mean(ctx.measurements(0)[-sweeps:, 1])),
               "accept": obs["accept"], "max_dG": float(np.max(errs)) if len(errs) else None,
               "dG_median": float(np.median(errs)) if len(errs) else None}
        ctx.close()
        return out

    head = a.prec
    n_stab = a.n_stab or NSTAB[head]
    r = timed(head, n_stab, a.steps, a.warmup, clocks=True)
    res = summary(head, r, a.steps)
    N, Ltau = r["dims"]["N"], r["dims"]["Ltau"]
    props_per_chain = (Ltau + 2) * N
    updates = props_per_chain * a.chains * world * a.steps
    ms = r["ms"]

    # the other precisions, timed beside the head for context with the same
    # warm-up and step count
    beside = {}
    if a.beside_steps > 0:
        for name in PRECS:
            if name == head:
                continue
            rb = timed(name, NSTAB[name], a.steps, a.warmup)
            beside[name + "_gpu"] = summary(name, rb, a.steps)

    # time-to-sigma of every precision, same procedure and sweep budget
    tts = {}
    if a.tts_sweeps > 0:
        for name in PRECS:
            tts[name] = time_to_sigma(name, a.tts_sweeps)
        ref = tts.get("fp64")
        if ref:
            for name, v in tts.items():
                v["dE_vs_fp64_sigma"] = (v["E_per_site"] - ref["E_per_site"]) / float(
                    np.hypot(v["E_err"], ref["E_err"])) if name != "fp64" else 0.0
    large = {}
    if a.large_sweeps > 0:
        for name, ns in (("fp32", 2), ("bf16x3", 2), ("fp64", 10)):
            try:
                large[name] = large_chain(name, ns, a.large_sweeps)
            except pqmc.PQMCError as ex:
                large[name] = {"error": str(ex)}
        large["workload"] = ("one chain, 18x18 honeycomb (648 sites), U=4, g=0.6, M_N=0.21, 2Theta=20 "
                             "(202 slices), swept by grid-wide kernel sequences (opts.spread)")
    dg64 = {}
    if a.dg_chains > 0 and rank == 0:
        for name in ("fp32", "bf16x3"):
            dg64[name] = dg_vs_fp64(name, chains=a.dg_chains)

    # end to end through the public API with host buffers: context creation
    # (host model set-up, the arena cleared on the device and its host-set
    # parts copied from host memory, initialisation) and, every
    # step, one sweep plus the device->host read of every chain's new record
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    ctx = pqmc.Context(specs, prec=PRECS[head], seed=2, n_stab=n_stab, chain_offset=rank * a.chains,
                       max_meas=a.steps + 1, stream=stream.cuda_stream, cta_threads=a.cta_threads, delay_k=0)
    h2d = ctx.upload_bytes()
    rec = np.zeros((a.chains, pqmc.RECORD))
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

    # roofline of the sweep kernel (one launch per step): the binding pipe is
    # FP64 for every path (the stabilisation in the reduced paths, everything
    # in the FP64 path)
    path_f, stab_f = sweep_flops(N, N // 2, Ltau, n_stab, res["accept"], head)
    launch_s = ms / 1e3 / a.steps
    fp64_f = stab_f + (path_f if head == "fp64" else 0.0)
    fp64_achieved = fp64_f * a.chains / launch_s / 1e12
    fp32_achieved = (path_f * a.chains / launch_s / 1e12) if head != "fp64" else 0.0
    fp32_peak = fp32_peak_tflops(2070.0)
    # time the two pipes need at their peaks, as a fraction of the launch
    bound_s = fp64_f * a.chains / (FP64_PEAK_TFLOPS * 1e12) + (
        path_f * a.chains / (fp32_peak * 1e12) if head != "fp64" else 0.0)
    shape_key = (head, N, Ltau, r["launch"]["delay_k"], r["launch"]["cta_threads"])
    traffic = (DRAM_BYTES_PER_CHAIN_SWEEP[shape_key] * a.chains if shape_key in DRAM_BYTES_PER_CHAIN_SWEEP
               else None)
    result = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x3": "bf16x3", "fp64": "f64"}[head], "data": "synthetic",
        "config": {"workload": "gutzwiller_pqmc_honeycomb_6x6_U4_g0.6_MN0.21_2theta%g" % a.two_theta,
                   "sites": N, "slices": Ltau + 2, "chains_per_gpu": a.chains, "global_chains": a.chains * world,
                   "n_stab": n_stab, "delay_block": r["launch"]["delay_k"],
                   "cta_threads": r["launch"]["cta_threads"], "precision": head,
                   "autotune": {k: {"pick": [v["delay_k"], v["cta_threads"]],
                                    "proxy_slices": v["proxy_ltau"],
                                    "ms_per_sweep": {"k%d_t%d" % (c["delay_k"], c["cta_threads"]): c["ms_per_sweep"]
                                                     for c in v["candidates"]}} for k, v in tuned.items()},
                   "l2": "state larger than L2 (%.0f MB of chain state per GPU vs 129 MB L2)" %
                         (a.chains * (2 * 2 * N * N * (4 if head != "fp64" else 8)
                                      + 4 * (Ltau // n_stab + 1) * N * (N // 2) * 8) / 1e6),
                   "parallelism": "chains%d" % world},
        "clocks": r["clocks"],
        "gpu_launches": r["launches"],
        "time_to_sigma_1e-3_s": tts[head]["seconds"] if head in tts else None,
        "time_to_sigma": tts,
        "time_to_sigma_method": ("wall time on the GPU from the first sweep of a fresh context, warm-up "
                                 "included, until the jackknife-over-chains sigma(E/site) reaches 1e-3; the "
                                 "warm-up is the shortest of 2/4/8/12/16 sweeps after which the two halves of "
                                 "the remaining sweeps agree within 2 sigma; every precision runs the same "
                                 "procedure with %d sweeps of %d chains" % (a.tts_sweeps, a.chains)),
        "E_per_site": res["E_per_site"], "E_err": res["E_err"], "accept": res["accept"],
        "dG_per_stabilisation": res["dG_per_stabilisation"],
        "dG_vs_fp64_per_stabilisation": dg64,
        "large_chain": large,
        "roofline": {"bound": "alu", "achieved": fp64_achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": fp64_achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": "sweep_kernel",
                     "pipe": "fp64",
                     "peak_source": "152 SMs x 2 FP64 FMA lanes x 2 flop x 2070 MHz (nominal 1.25 TFLOP/s)",
                     "two_pipe_bound_frac": bound_s / launch_s,
                     "fp32_pipe": {"achieved": fp32_achieved, "peak": fp32_peak,
                                   "frac": fp32_achieved / fp32_peak,
                                   "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // max(a.steps, 1),
                "d2h_bytes_per_step": d2h // max(a.steps, 1),
                "note": "timed: context creation (host FP64 model build, device allocation and clearing, upload "
                        "of the host-set parts of the arena, device initialisation) + per step one sweep and the device-to-host "
                        "read of every chain's new measurement; h2d is the creation-time upload (model tables, trial "
                        "orbitals, initial fields, chain states) spread over the steps"},
    }
    result.update(beside)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        rate, cores, n_upd = oracle_rate(a.two_theta, NSTAB["fp64"], a.cpu_seconds)
        cs_per_s = rate / props_per_chain
        # chain-sweeps the FP64 GPU arm needed for sigma = 1e-3 (warm-up
        # included), at the oracle's chain-sweep rate on all host cores
        ref = tts.get("fp64")
        need = (a.chains * (ref["warmup_sweeps"] + (ref["measured_sweeps_to_sigma"] or
                                                     (ref["sweeps_run"] - ref["warmup_sweeps"]) *
                                                     (ref["E_err"] / 1e-3) ** 2))) if ref else None
        result["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "per_core": rate / cores, "cpu_model": cpu_model(),
                                  "sample": "%d oracle chains (one per core, FP64, n_stab 10), ~%gs of sweeps "
                                            "each, %d updates" % (cores, a.cpu_seconds, n_upd),
                                  "time_to_sigma_1e-3_s": need / cs_per_s if need else None,
                                  "time_to_sigma_method": "the chain-sweeps the FP64 GPU arm needed, at the "
                                                          "oracle's chain-sweep rate on these cores"}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_stab = a.n_stab or 10
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
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "per_core": value / cores, "cpu_model": cpu_model()},
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

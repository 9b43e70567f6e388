"""A fixed sweep workload for profiling the sweep kernel (one context, no
autotuning): the 72-site Gutzwiller PQMC batch of the throughput bench, or
another size, run for a few sweeps with a chosen launch shape.

  python -m paper_2303_13403_gb300.profile_run [--chains 304] [--prec fp32] [--L 6]
         [--two-theta 8] [--n-stab 2] [--delay-k 32] [--cta-threads 256] [--sweeps 2]

Prints one JSON line: milliseconds per sweep (CUDA events on the context's
stream, after one warm-up sweep) and the launch shape.
"""
import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--chains", type=int, default=304)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16x3", "fp64"])
    ap.add_argument("--L", type=int, default=6)
    ap.add_argument("--two-theta", type=float, default=8.0)
    ap.add_argument("--n-stab", type=int, default=0)
    ap.add_argument("--delay-k", type=int, default=32)
    ap.add_argument("--cta-threads", type=int, default=0)
    ap.add_argument("--sweeps", type=int, default=2)
    a = ap.parse_args()
    import torch
    from . import pqmc, workloads
    torch.cuda.set_device(0)
    prec = {"fp32": pqmc.FP32, "bf16x3": pqmc.BF16X3, "fp64": pqmc.FP64}[a.prec]
    n_stab = a.n_stab or (10 if a.prec == "fp64" else 2)
    spec = workloads.honeycomb(a.L, U=4.0, dtau=0.1, two_theta=a.two_theta, g=0.6, M_N=0.21)
    stream = torch.cuda.Stream()
    ctx = pqmc.Context([spec] * a.chains, prec=prec, seed=1, n_stab=n_stab, delay_k=a.delay_k,
                       cta_threads=a.cta_threads, stream=stream.cuda_stream)
    ctx.sweep(1, measure=False)
    ctx.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.sweeps):
        ctx.sweep(1, measure=True)
    e1.record(stream)
    e1.synchronize()
    print(json.dumps({"ms_per_sweep": e0.elapsed_time(e1) / a.sweeps, "chains": a.chains, "sites": spec.n_sites,
                      "precision": a.prec, "n_stab": n_stab, "launch": ctx.launch()}))
    ctx.close()


if __name__ == "__main__":
    main()

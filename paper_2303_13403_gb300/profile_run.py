"""A fixed sweep workload for profiling the sweep kernel (one context, no
autotuning): the 72-site Gutzwiller PQMC batch of the throughput bench, or
another size, run for a few sweeps with a chosen launch shape.

  python -m paper_2303_13403_gb300.profile_run [--chains 304] [--prec fp32] [--L 6] [--spread 1]
         [--two-theta 8] [--n-stab 2] [--delay-k 32] [--cta-threads 256] [--sweeps 2]

Prints one JSON line: milliseconds per sweep (CUDA events on the context's
stream, after one warm-up sweep) and the launch shape.

  python -m paper_2303_13403_gb300.profile_run --gemm 288 288 288 [--reps 3]

instead times the tensor-core split-BF16 product of the BF16X3 path
(pqmc_test_tc_gemm, one CTA) on random FP32 operands.
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
    ap.add_argument("--gemm", type=int, nargs=3, default=None, metavar=("M", "N", "K"))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--spread", type=int, default=0, help="1: grid-wide kernel sequence per sweep")
    ap.add_argument("--warmup", type=int, default=-1, help="untimed sweeps first (default 1, spread 2)")
    a = ap.parse_args()
    import torch
    from . import pqmc, workloads
    torch.cuda.set_device(0)
    if a.gemm:
        M, N, K = a.gemm
        g = torch.Generator(device="cuda").manual_seed(1)
        A = torch.randn(M, K, device="cuda", generator=g)
        B = torch.randn(K, N, device="cuda", generator=g)
        C = torch.empty(M, N, device="cuda")
        pqmc.test_tc_gemm(M, N, K, A.data_ptr(), False, B.data_ptr(), C.data_ptr())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            pqmc.test_tc_gemm(M, N, K, A.data_ptr(), False, B.data_ptr(), C.data_ptr())
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        err = float((C.double() - A.double() @ B.double()).abs().max() / (A.double() @ B.double()).abs().max())
        # three BF16 products per element of C, 2 M N K flop each
        print(json.dumps({"gemm": [M, N, K], "ms": ms, "split_tflops": 6.0 * M * N * K / (ms * 1e-3) / 1e12,
                          "max_rel_err": err}))
        return
    prec = {"fp32": pqmc.FP32, "bf16x3": pqmc.BF16X3, "fp64": pqmc.FP64}[a.prec]
    n_stab = a.n_stab or (10 if a.prec == "fp64" else 2)
    spec = workloads.honeycomb(a.L, U=4.0, dtau=0.1, two_theta=a.two_theta, g=0.6, M_N=0.21)
    stream = torch.cuda.Stream()
    ctx = pqmc.Context([spec] * a.chains, prec=prec, seed=1, n_stab=n_stab, delay_k=a.delay_k,
                       cta_threads=a.cta_threads, stream=stream.cuda_stream, spread=a.spread)
    # warm-up (a spread context captures one graph per sweep direction)
    warm = a.warmup if a.warmup >= 0 else (2 if a.spread else 1)
    if warm:
        ctx.sweep(warm, measure=False)
    ctx.synchronize()
    c0 = ctx.phase_cycles(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.sweeps):
        ctx.sweep(1, measure=True)
    e1.record(stream)
    e1.synchronize()
    c1 = ctx.phase_cycles(0)
    mcyc = {k: round((c1[k] - c0[k]) / a.sweeps / 1e6, 2) for k in c1 if c1[k] != c0[k]}
    print(json.dumps({"ms_per_sweep": e0.elapsed_time(e1) / a.sweeps, "chains": a.chains, "sites": spec.n_sites,
                      "mcycles_per_sweep_chain0": mcyc,
                      "precision": a.prec, "n_stab": n_stab, "spread": a.spread, "launch": ctx.launch(),
                      "max_dG": ctx.measure(-1)["max_dG"]}))
    ctx.close()


if __name__ == "__main__":
    main()

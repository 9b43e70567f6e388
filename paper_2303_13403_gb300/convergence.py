"""Convergence of the projection in Theta for three trial states (the
comparison of Fig. 2): the Gutzwiller-projected Neel state (GP), the Neel
mean-field Slater determinant without projection (SD(AFM), g = 0) and the
free-fermion Slater determinant (SD(NI), g = 0, M_N = 0), for U = 3.5, 3.75
and 4 on one honeycomb lattice.

Every (U, trial, 2 Theta) point is a group of chains of one batched context
(uneven projection lengths in one launch); the energy per site and the AFM
structure factor are pooled per group with a jackknife over its chains.

Trial parameters (readings): GP takes the optimum the paper quotes for
U = 3.5 (g = 0.55, M_N = 0.07) and U = 4 (g = 0.6, M_N = 0.21) and their
midpoint for U = 3.75, where none is quoted; SD(AFM) takes the same M_N with
g = 0 (the paper does not give its mean-field order parameter).

Run ``python -m paper_2303_13403_gb300.convergence --L 6``.
"""
import argparse
import json
import time

import numpy as np

from . import distributed, workloads

GP_PARAMS = {3.5: (0.55, 0.07), 3.75: (0.575, 0.14), 4.0: (0.6, 0.21)}
TRIALS = ("GP", "SD(AFM)", "SD(NI)")


def trial_params(name, U):
    g, m = GP_PARAMS[U]
    return {"GP": (g, m), "SD(AFM)": (0.0, m), "SD(NI)": (0.0, 0.0)}[name]


def run(L=6, Us=(3.5, 3.75, 4.0), two_thetas=(0.8, 1.6, 2.4, 4.0, 5.6, 8.0), chains=32, n_warm=20, n_meas=100,
        prec=workloads.FP32, n_stab=2, dtau=0.1, seed=3):
    from . import pqmc
    groups = [(U, t, tt) for U in Us for t in TRIALS for tt in two_thetas]
    specs = []
    for U, t, tt in groups:
        g, m = trial_params(t, U)
        specs += [workloads.honeycomb(L, U=U, dtau=dtau, two_theta=tt, g=g, M_N=m)] * chains
    ctx = pqmc.Context(specs, prec=prec, seed=seed, n_stab=n_stab, max_meas=n_meas)
    t0 = time.perf_counter()
    ctx.sweep(n_warm, measure=False)
    ctx.sweep(n_meas, measure=True)
    ctx.synchronize()
    seconds = time.perf_counter() - t0
    rows = []
    for k, (U, t, tt) in enumerate(groups):
        recs = [ctx.measurements(k * chains + r) for r in range(chains)]
        est = distributed.pooled_estimate(distributed.chain_sums(recs))
        rows.append({"U": U, "trial": t, "two_theta": tt, "E": est["E"], "E_err": est["E_err"],
                     "s_afm": est["s_afm"], "s_afm_err": est["s_afm_err"], "sign": est["sign"]})
    ctx.close()
    return {"L": L, "chains_per_point": chains, "sweeps": n_warm + n_meas, "seconds": seconds,
            "precision": workloads.PRECISION_NAMES[prec], "rows": rows}


def main():
    ap = argparse.ArgumentParser(description="Theta convergence of GP, SD(AFM) and SD(NI) trial states")
    ap.add_argument("--L", type=int, default=6)
    ap.add_argument("--chains", type=int, default=32)
    ap.add_argument("--warm", type=int, default=20)
    ap.add_argument("--meas", type=int, default=100)
    ap.add_argument("--two-theta", type=float, nargs="+", default=[0.8, 1.6, 2.4, 4.0, 5.6, 8.0])
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    r = run(a.L, two_thetas=tuple(a.two_theta), chains=a.chains, n_warm=a.warm, n_meas=a.meas)
    print(json.dumps(r))


if __name__ == "__main__":
    main()

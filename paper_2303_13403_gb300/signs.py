"""Average sign of the spinless t-V model (Fig. 4): Gutzwiller trial (GP)
against the free Slater determinant (SD), as a function of the projection
length 2 Theta and of the linear size L, all groups in one batched context.

The density-difference decoupling of each bond leaves real fields and one
determinant, whose sign can be negative; <sign> = sum_c s_c / n over the
per-sweep weight signs of a group's chains, with a jackknife over chains.
The GP parameters (g, Delta_C) are inputs: the paper minimises the
variational energy (variational.py --tv) and quotes no values.

Run ``python -m paper_2303_13403_gb300.signs --gp-g 0.5 --gp-delta 0.1``.
"""
import argparse
import json
import time

from . import distributed, workloads


def run(gp=(0.5, 0.1), Vs=(1.35, 1.6), L=6, two_thetas=(0.8, 1.6, 4.0, 8.0), Ls=(3, 6, 9), L_two_theta=4.0,
        V_L=1.6, chains=32, n_warm=10, n_meas=60, prec=workloads.FP32, n_stab=2, seed=7):
    from . import pqmc
    trials = {"GP": gp, "SD": (0.0, 0.0)}
    groups = [(V, L, t, tt) for V in Vs for t in trials for tt in two_thetas]
    groups += [(V_L, l, t, L_two_theta) for l in Ls if l != L or V_L not in Vs or L_two_theta not in two_thetas
               for t in trials]
    specs = []
    for V, l, t, tt in groups:
        g, d = trials[t]
        specs += [workloads.tv_honeycomb(l, V=V, g=g, Delta_C=d, two_theta=tt)] * chains
    ctx = pqmc.Context(specs, prec=prec, seed=seed, n_stab=n_stab, max_meas=n_meas)
    t0 = time.perf_counter()
    ctx.sweep(n_warm, measure=False)
    ctx.sweep(n_meas, measure=True)
    ctx.synchronize()
    seconds = time.perf_counter() - t0
    rows = []
    for k, (V, l, t, tt) in enumerate(groups):
        est = distributed.pooled_estimate(distributed.chain_sums(
            [ctx.measurements(k * chains + r) for r in range(chains)]))
        rows.append({"V": V, "L": l, "trial": t, "two_theta": tt, "sign": est["sign"],
                     "sign_err": est["sign_err"], "E": est["E"], "E_err": est["E_err"],
                     "s_cdw": est["s_afm"], "s_cdw_err": est["s_afm_err"]})
    ctx.close()
    return {"gp": gp, "chains_per_point": chains, "sweeps": n_warm + n_meas, "seconds": seconds,
            "precision": workloads.PRECISION_NAMES[prec], "rows": rows}


def main():
    ap = argparse.ArgumentParser(description="Average sign of the t-V model, GP against SD trial")
    ap.add_argument("--gp-g", type=float, default=0.5)
    ap.add_argument("--gp-delta", type=float, default=0.1)
    ap.add_argument("--chains", type=int, default=32)
    ap.add_argument("--warm", type=int, default=10)
    ap.add_argument("--meas", type=int, default=60)
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(run((a.gp_g, a.gp_delta), chains=a.chains, n_warm=a.warm, n_meas=a.meas)))


if __name__ == "__main__":
    main()

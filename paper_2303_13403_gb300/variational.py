"""The variational step of the method (Method section, Fig. 1): the energy of
the Gutzwiller-projected Neel state |psi_G> = e^{-g D} |psi_N(M_N)> over a
(g, M_N) grid, and the parameters that minimise it.

At Theta = 0 the estimator <psi_G|H|psi_G> / <psi_G|psi_G> needs only the two
Gutzwiller HS slices (tau = 0 and tau = Ltau + 1 = 1; no interaction slices),
so a grid point is a short chain and the whole grid -- every (U, g, M_N) and
several chains per point -- runs as one batched context through the same
sweep kernel.  The grid minimum is refined by a weighted least-squares
quadratic fit over the points around it (host-side analysis of the measured
energies; every Monte Carlo step runs in the CUDA kernels).

Run ``python -m paper_2303_13403_gb300.variational --L 6`` for the 11 x 11
scan of Fig. 1 (g in [0, 1], M_N in [0, 0.3]) at U = 3.5 and 4.0, and with
``--tv --U 1.35 1.6`` the same scan of the spinless t-V trial of Eq. (5)
(bond g, CDW field Delta_C), whose optimum the paper uses without quoting it.
"""
import argparse
import json
import time

import numpy as np

from . import distributed, workloads

G_VALUES = tuple(np.round(np.linspace(0.0, 1.0, 11), 10))
M_VALUES = tuple(np.round(0.03 * np.arange(11), 10))


def grid_specs(U, L, g_values=G_VALUES, m_values=M_VALUES, dtau=0.1, kind=workloads.HONEYCOMB):
    """ChainSpecs of one Theta = 0 grid, row-major over (g, M_N).  For the
    spinless t-V model (kind HONEYCOMB_TV) U is V and M_N the CDW field
    Delta_C of the trial of Eq. (5)."""
    if kind == workloads.HONEYCOMB_TV:
        return [workloads.tv_honeycomb(L, V=U, g=float(g), Delta_C=float(m), two_theta=0.0, dtau=dtau)
                for g in g_values for m in m_values]
    return [workloads.ChainSpec(kind=kind, Lx=L, Ly=L, U=U, dtau=dtau, two_theta=0.0, g=float(g),
                                M_N=float(m))
            for g in g_values for m in m_values]


def quadratic_minimum(gv, mv, E, E_err, at):
    """Stationary point of E(g, M) = c0 + c1 g + c2 M + c3 g^2 + c4 g M + c5 M^2
    fitted (weights 1/err^2) to the grid points within one step of ``at``
    (a (row, col) index).  Returns (g*, M*, E*) or None when the fit has no
    minimum inside that neighbourhood."""
    gv, mv = np.asarray(gv, float), np.asarray(mv, float)
    i0, j0 = at
    rows = range(max(i0 - 1, 0), min(i0 + 2, len(gv)))
    cols = range(max(j0 - 1, 0), min(j0 + 2, len(mv)))
    A, b, w = [], [], []
    for i in rows:
        for j in cols:
            g, m = gv[i], mv[j]
            A.append([1.0, g, m, g * g, g * m, m * m])
            b.append(E[i, j])
            w.append(1.0 / max(E_err[i, j], 1e-300))
    A, b, w = np.array(A), np.array(b), np.array(w)
    if len(b) < 6:
        return None
    c, *_ = np.linalg.lstsq(A * w[:, None], b * w, rcond=None)
    H = np.array([[2 * c[3], c[4]], [c[4], 2 * c[5]]])
    if np.linalg.eigvalsh(H).min() <= 0:
        return None
    gs, ms = np.linalg.solve(H, -c[1:3])
    lo_g, hi_g = gv[min(rows)], gv[max(rows)]
    lo_m, hi_m = mv[min(cols)], mv[max(cols)]
    if not (lo_g <= gs <= hi_g and lo_m <= ms <= hi_m):
        return None
    Es = c[0] + c[1] * gs + c[2] * ms + c[3] * gs * gs + c[4] * gs * ms + c[5] * ms * ms
    return float(gs), float(ms), float(Es)


def summarise(gv, mv, E, E_err):
    i, j = np.unravel_index(np.nanargmin(E), E.shape)
    out = {"grid_argmin": {"g": float(gv[i]), "M_N": float(mv[j]), "E": float(E[i, j]),
                           "E_err": float(E_err[i, j])}}
    fit = quadratic_minimum(gv, mv, E, E_err, (i, j))
    out["fit_min"] = None if fit is None else {"g": fit[0], "M_N": fit[1], "E": fit[2]}
    return out


def scan(Us, L, chains_per_point=8, n_warm=50, n_meas=400, prec=workloads.FP64, seed=1,
         g_values=G_VALUES, m_values=M_VALUES, kind=workloads.HONEYCOMB, cta_threads=0):
    """Variational energies E/site (sign-reweighted, jackknife over the chains
    of a point) for every U in ``Us`` on one L x L lattice, all in one context.

    Returns {U: {"E": (ng, nm), "E_err", "docc", "s_afm", "grid_argmin",
    "fit_min"}} plus "seconds" (sweeps only) and "chains"."""
    from . import pqmc
    base = [sp for U in Us for sp in grid_specs(U, L, g_values, m_values, kind=kind)]
    specs = [sp for sp in base for _ in range(chains_per_point)]
    ctx = pqmc.Context(specs, prec=prec, seed=seed, n_stab=1, max_meas=n_meas, cta_threads=cta_threads)
    t0 = time.perf_counter()
    if n_warm:
        ctx.sweep(n_warm, measure=False)
    ctx.sweep(n_meas, measure=True)
    ctx.synchronize()
    seconds = time.perf_counter() - t0
    ng, nm = len(g_values), len(m_values)
    out = {"seconds": seconds, "chains": len(specs), "sweeps": n_warm + n_meas}
    for u, U in enumerate(Us):
        grids = {k: np.full((ng, nm), np.nan) for k in ("E", "E_err", "docc", "s_afm", "s_afm_err", "sign")}
        for p in range(ng * nm):
            c0 = (u * ng * nm + p) * chains_per_point
            recs = [ctx.measurements(c0 + r) for r in range(chains_per_point)]
            est = distributed.pooled_estimate(distributed.chain_sums(recs))
            i, j = divmod(p, nm)
            for k in grids:
                grids[k][i, j] = est[k]
        res = {k: v for k, v in grids.items()}
        res.update(summarise(g_values, m_values, grids["E"], grids["E_err"]))
        out[U] = res
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser(description="Theta = 0 variational scan of the Gutzwiller-Neel trial")
    ap.add_argument("--L", type=int, default=6)
    ap.add_argument("--U", type=float, nargs="+", default=[3.5, 4.0])
    ap.add_argument("--chains", type=int, default=8, help="chains per grid point")
    ap.add_argument("--warm", type=int, default=50)
    ap.add_argument("--meas", type=int, default=400)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "bf16x3"])
    ap.add_argument("--tv", action="store_true", help="spinless t-V model (--U are V values)")
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    prec = {v: k for k, v in workloads.PRECISION_NAMES.items()}[a.prec]
    kind = workloads.HONEYCOMB_TV if a.tv else workloads.HONEYCOMB
    r = scan(a.U, a.L, a.chains, a.warm, a.meas, prec, kind=kind)
    line = {"L": a.L, "chains": r["chains"], "sweeps": r["sweeps"], "seconds": round(r["seconds"], 3)}
    for U in a.U:
        x = r[U]
        line[str(U)] = {"grid_argmin": x["grid_argmin"], "fit_min": x["fit_min"],
                        "median_E_err": float(np.nanmedian(x["E_err"])),
                        "E": np.round(x["E"], 5).tolist()}
    print(json.dumps(line))


if __name__ == "__main__":
    main()

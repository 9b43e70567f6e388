"""The larger workloads through the C-ABI: uneven batched lattices of the
variational scan (72/162/288 sites), the 648-site single chain, and the doped
square lattice with signful weights."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import pqmc as opq
from paper_2303_13403_gb300 import pqmc, workloads

pytestmark = pytest.mark.gpu


def oracle_params(spec, **kw):
    base = dict(kind=spec.kind, Lx=spec.Lx, Ly=spec.Ly, t=spec.t, tp=spec.tp, U=spec.U, dtau=spec.dtau,
                two_theta=spec.two_theta, g=spec.g, M_N=spec.M_N, n_up=spec.n_up, n_dn=spec.n_dn,
                tiebreak=spec.tiebreak)
    base.update(kw)
    return opq.Params(**base)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    torch.cuda.set_device(0)
    pqmc.load()


def test_uneven_batch_fixed_fields_parity():
    """One chain of each size of the batched (g, M_N) scan in one context; FP64
    G after initialisation on fixed fields equals the oracle to 1e-10."""
    by_size = {}
    for sp in workloads.variational_grid(8.0):
        by_size.setdefault(sp.n_sites, sp)
    specs = [by_size[72], by_size[162], by_size[288]]
    ctx = pqmc.Context(specs, prec=pqmc.FP64, seed=3, n_stab=10)
    for c, sp in enumerate(specs):
        f = workloads.random_fields(sp, seed=40 + c)
        ctx.set_fields(f, chain=c)
        ch = opq.Chain(oracle_params(sp, n_stab=10), fields=f)
        for s, sg in ((0, 1), (1, -1)):
            G = ctx.green(c, s)
            assert np.abs(G - ch.G[sg]).max() / np.abs(ch.G[sg]).max() < 1e-10, (sp.n_sites, s)


def test_uneven_batch_sweeps_all_sizes_fp32():
    by_size = {}
    for sp in workloads.variational_grid(8.0):
        by_size.setdefault(sp.n_sites, sp)
    specs = [by_size[72], by_size[162], by_size[288]] * 2
    ctx = pqmc.Context(specs, prec=pqmc.FP32, seed=5, n_stab=4)
    ctx.sweep(2)
    for c in range(len(specs)):
        rec = ctx.measurements(c)
        assert len(rec) == 2 and np.all(np.isfinite(rec)) and np.all(rec[:, 0] == 1.0)
        assert -1.2 < rec[:, 1].mean() < -0.5
        assert ctx.stab_errors(c).max() < 5e-2


def test_large_single_chain_648_sites():
    """The 648-site chain (200 slices, n_stab 10) in FP32: one sweep, finite
    records, stabilisation errors reported, sign +1 at half filling."""
    spec = workloads.GUTZ_648
    ctx = pqmc.Context([spec], prec=pqmc.FP32, seed=1, n_stab=10)
    ctx.sweep(1)
    rec = ctx.measurements(0)
    assert len(rec) == 1 and np.all(np.isfinite(rec)) and rec[0, 0] == 1.0
    assert -1.0 < rec[0, 1] < -0.5
    errs = ctx.stab_errors(0)
    assert len(errs) == 21 and np.all(np.isfinite(errs))


def test_doped_square_signs_consistent():
    """Doped t-t' lattice (28 up + 28 down on 64 sites): the weight sign from
    the stabilised stacks equals the running product of sgn(R) in every record."""
    spec = replace(workloads.DOPED_64[0.6], two_theta=4.0)
    ctx = pqmc.Context([spec] * 16, prec=pqmc.FP64, seed=9, n_stab=10)
    ctx.sweep(4)
    for c in range(16):
        rec = ctx.measurements(c)
        assert set(np.unique(rec[:, 0])) <= {-1.0, 1.0}
        assert np.array_equal(rec[:, 0], rec[:, 4])


def test_theta_convergence_study_against_exact_projection():
    """The Theta-convergence study of Fig. 2 (GP, SD(AFM), SD(NI) trial states,
    uneven projection lengths in one context) on the 8-site cluster: every
    (trial, 2 Theta) energy agrees with the exact Trotterised projection of
    the same trial state (Fock space, same operator order) within 3 sigma,
    and the three trial states' exact energies differ at the shortest
    projection, so the check separates them."""
    from oracle import ed
    from paper_2303_13403_gb300 import convergence
    two_thetas = (0.4, 1.6)
    r = convergence.run(L=2, Us=(4.0,), two_thetas=two_thetas, chains=48, n_warm=20, n_meas=150, seed=17)
    assert len(r["rows"]) == 3 * len(two_thetas)
    exact = {}
    for row in r["rows"]:
        g, m_n = convergence.trial_params(row["trial"], row["U"])
        spec = workloads.honeycomb(2, U=row["U"], dtau=0.1, two_theta=row["two_theta"], g=g, M_N=m_n)
        m = opq.Model(oracle_params(spec, n_stab=2))
        c = ed.Cluster(m.K, 4, 4, row["U"])
        Ex, _ = c.trotter_projection(m.P[1], m.P[-1], g, 0.1, m.Ltau)
        exact[(row["trial"], row["two_theta"])] = Ex / 8
        assert row["sign"] == 1.0 and 0.0 < row["s_afm"] <= 0.25
        assert 0 < row["E_err"] < 0.01
        assert abs(row["E"] - Ex / 8) < 3 * row["E_err"], (row, Ex / 8)
    short = [exact[(t, 0.4)] for t in convergence.TRIALS]
    assert max(short) - min(short) > 0.01


def test_cta_shapes_agree_on_reduced_path():
    """FP32 sweeps of an uneven batch with 256- and 512-thread CTAs: every
    product element is the same sequence of FMAs in both shapes, so G and the
    accept/reject sequences agree exactly; the records agree to rounding of
    the CTA-wide sums."""
    specs = [workloads.honeycomb(3, two_theta=2.0, g=0.6, M_N=0.21),
             workloads.honeycomb(6, two_theta=2.0, g=0.6, M_N=0.21),
             workloads.honeycomb(9, two_theta=2.0, g=0.6, M_N=0.21)]
    out = {}
    for tpb in (256, 512):
        ctx = pqmc.Context(specs, prec=pqmc.FP32, seed=4, n_stab=2, cta_threads=tpb, accept_log=1 << 16)
        ctx.sweep(2)
        out[tpb] = [(ctx.accept_log(2 * (s.n_slices + 2) * s.n_sites, c), ctx.green(c, 0), ctx.measurements(c))
                    for c, s in enumerate(specs)]
        ctx.close()
    for (a0, g0, r0), (a1, g1, r1) in zip(out[256], out[512]):
        assert np.array_equal(a0, a1)
        assert np.array_equal(g0, g1)
        assert np.allclose(r0, r1, rtol=1e-12, atol=1e-14)

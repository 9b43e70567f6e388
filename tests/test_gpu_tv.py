"""The spinless t-V model (repulsive spinless honeycomb section, Eqs. (4)-(5))
through the C-ABI against the t-V oracle: G and the weight on fixed bond
fields, identical accept/reject sequences and measurements over several
sweeps (FP64), and Monte Carlo estimates within 3 sigma of Fock space."""
import numpy as np
import pytest

from oracle import pqmc as opq
from oracle import tv
from paper_2303_13403_gb300 import pqmc, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    torch.cuda.set_device(0)
    pqmc.load()


def tv_params(spec, **kw):
    base = dict(Lx=spec.Lx, Ly=spec.Ly, t=spec.t, V=spec.U, dtau=spec.dtau, two_theta=spec.two_theta,
                g=spec.g, Delta_C=spec.M_N, tiebreak=spec.tiebreak)
    base.update(kw)
    return tv.TVParams(**base)


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("spec,n_stab", [
    (workloads.tv_honeycomb(2, V=1.6, g=0.5, Delta_C=0.1, two_theta=1.0), 5),
    (workloads.tv_honeycomb(3, V=1.35, g=0.3, Delta_C=0.0, two_theta=2.0), 10),
    (workloads.tv_honeycomb(6, V=1.6, g=0.4, Delta_C=0.2, two_theta=1.6), 4),
])
def test_fixed_fields_green_and_weight(spec, n_stab):
    f = workloads.random_fields(spec, seed=11)
    ctx = pqmc.Context([spec], prec=pqmc.FP64, seed=1, n_stab=n_stab)
    assert ctx.dims()["n_fields"] == 3 * spec.Lx * spec.Ly and ctx.dims()["N_dn"] == 0
    ctx.set_fields(f)
    ch = tv.TVChain(tv_params(spec, n_stab=n_stab), fields=f)
    assert rel_err(ctx.green(0, 0), ch.G) < 1e-10
    w = ctx.weight()
    assert np.isclose(w[0], ch.logw, rtol=1e-10, atol=1e-9)
    assert w[1] == ch.sign_stack and w[2] == 0.0 and w[3] == 1.0
    assert np.array_equal(ctx.fields(), f)


def run_pair(spec, n_sweeps, n_stab, seed, prec=pqmc.FP64):
    ctx = pqmc.Context([spec], prec=prec, seed=seed, n_stab=n_stab, accept_log=1 << 20)
    ctx.sweep(n_sweeps, measure=True)
    ctx.synchronize()
    ch = tv.TVChain(tv_params(spec, n_stab=n_stab, seed=seed)).run(0, n_sweeps)
    return ctx, ch


@pytest.mark.parametrize("spec,n_sweeps,n_stab", [
    (workloads.tv_honeycomb(2, V=1.6, g=0.5, Delta_C=0.1, two_theta=1.0), 6, 5),
    (workloads.tv_honeycomb(2, V=1.6, g=0.6, Delta_C=0.1, two_theta=0.0), 6, 1),     # Theta = 0
    (workloads.tv_honeycomb(3, V=1.35, g=0.3, two_theta=2.0), 4, 10),
    (workloads.tv_honeycomb(6, V=1.6, g=0.4, Delta_C=0.2, two_theta=0.8), 2, 2),       # 3 blocks per class
])
def test_sweep_parity(spec, n_sweeps, n_stab):
    """FP64: the same Philox accept/reject sequence as the oracle, G and every
    measurement record (E, bond energy, S_CDW, signs) to 1e-10."""
    ctx, ch = run_pair(spec, n_sweeps, n_stab, 9)
    d = ctx.dims()
    n = n_sweeps * (d["Ltau"] + 2) * d["n_fields"]
    ora = np.array([x[3] for x in ch.accept_log], dtype=np.uint8)
    assert len(ora) == n
    assert np.array_equal(ctx.accept_log(n), ora)
    assert rel_err(ctx.green(0, 0), ch.G) < 1e-10
    assert np.array_equal(ctx.fields(), ch.fields)
    rec = ctx.measurements()
    ms = ch.measurements
    assert len(rec) == len(ms) == n_sweeps
    assert np.allclose(rec[:, 1], [m.energy for m in ms], rtol=1e-10, atol=1e-12)
    assert np.allclose(rec[:, 2], [m.ebond for m in ms], rtol=1e-10, atol=1e-12)
    assert np.allclose(rec[:, 3], [m.kinetic for m in ms], rtol=1e-10, atol=1e-12)
    assert np.allclose(rec[:, 5], [m.s_cdw for m in ms], rtol=1e-10, atol=1e-14)
    assert np.array_equal(rec[:, 0], [m.sign for m in ms])
    assert np.array_equal(rec[:, 4], [m.sign_running for m in ms])
    assert np.isclose(ctx.measure(0)["accept"], ch.acceptance, rtol=0, atol=1e-12)


@pytest.mark.parametrize("prec", [pqmc.FP64, pqmc.FP32, pqmc.BF16X3])
def test_mc_within_3sigma_of_exact(prec):
    """64 chains on the 8-site cluster: pooled E, bond energy and S_CDW agree
    with the exact Trotterised projection (Fock space) within 3 sigma."""
    spec = workloads.tv_honeycomb(2, V=1.6, g=0.4, Delta_C=0.1, two_theta=1.0)
    ctx = pqmc.Context([spec] * 64, prec=prec, seed=21, n_stab=5 if prec == pqmc.FP64 else 1)
    ctx.sweep(10, measure=False)
    ctx.sweep(60, measure=True)
    obs = ctx.measure(-1)
    m = tv.TVModel(tv_params(spec, n_stab=5))
    Ex, EBx, Sx = tv.TVCluster(m).trotter_observables(spec.g, spec.dtau, spec.U, m.Ltau)
    assert obs["n_meas"] == 64 * 60
    assert abs(obs["E"] - Ex) < 3 * obs["E_err"], (obs, Ex)
    assert abs(obs["docc"] - EBx) < 3 * obs["docc_err"], (obs, EBx)
    assert abs(obs["s_afm"] - Sx) < 3 * obs["s_afm_err"], (obs, Sx)
    assert obs["E_err"] < 0.01


def test_signs_consistent_and_fp32_stabilisation():
    """72 sites, V = 1.6, 2 Theta = 4, FP32: the sign of the weight from the
    stacks equals the running product of sgn(R) at every measurement, and the
    per-stabilisation error stays at FP32 level."""
    spec = workloads.tv_honeycomb(6, V=1.6, g=0.0, two_theta=4.0)
    ctx = pqmc.Context([spec] * 32, prec=pqmc.FP32, seed=5, n_stab=2)
    ctx.sweep(4)
    for c in range(32):
        rec = ctx.measurements(c)
        assert set(np.unique(rec[:, 0])) <= {-1.0, 1.0}
        assert np.array_equal(rec[:, 0], rec[:, 4])
    errs = np.concatenate([ctx.stab_errors(c) for c in range(32)])
    assert np.median(errs) < 1e-5 and np.percentile(errs, 99) < 1e-3

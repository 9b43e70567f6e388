"""GPU parity of libpqmc (called through the C-ABI) against the FP64 oracle.

FP64 path: on fixed fields G and the weight match to 1e-10 relative; with the
same seed the Philox accept/reject sequence is identical (so every ratio
decision agrees) and the energies agree to 1e-10.  FP32 path: max |G - G_FP64|
after every stabilisation <= 1e-4, energies within 3 sigma of the exact value.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import ed, pqmc as opq
from paper_2303_13403_gb300 import distributed, pqmc, workloads

pytestmark = pytest.mark.gpu


def oracle_params(spec, **kw):
    base = dict(kind=spec.kind, Lx=spec.Lx, Ly=spec.Ly, t=spec.t, tp=spec.tp, U=spec.U, dtau=spec.dtau,
                two_theta=spec.two_theta, g=spec.g, M_N=spec.M_N, n_up=spec.n_up, n_dn=spec.n_dn,
                tiebreak=spec.tiebreak)
    base.update(kw)
    return opq.Params(**base)


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    pqmc.load()


SMALL = workloads.honeycomb(2, U=4.0, dtau=0.1, two_theta=2.0, g=0.6, M_N=0.21)


@pytest.mark.parametrize("spec,n_stab", [
    (SMALL, 5),
    (workloads.PLAIN_18, 10),
    (workloads.GUTZ_72[4.0], 10),
    (workloads.DOPED_64[0.6], 10),
    (workloads.ChainSpec(kind=workloads.SQUARE, Lx=5, Ly=5, tp=-0.2, U=4.0, two_theta=2.0, g=0.3,
                         n_up=11, n_dn=12), 5),
])
def test_fixed_fields_green_and_weight(spec, n_stab):
    fields = workloads.random_fields(spec, seed=12)
    ctx = pqmc.Context([spec], prec=pqmc.FP64, seed=5, n_stab=n_stab)
    ctx.set_fields(fields)
    ch = opq.Chain(oracle_params(spec, n_stab=n_stab, seed=5), fields=fields)
    for s, sg in ((0, 1), (1, -1)):
        assert rel_err(ctx.green(0, s), ch.G[sg]) < 1e-10
    w = ctx.weight()
    # weight at the last stabilisation (tau = 0 of the initialisation)
    assert np.isclose(w[0], ch.logw[1], rtol=1e-10, atol=1e-9)
    assert np.isclose(w[2], ch.logw[-1], rtol=1e-10, atol=1e-9)
    assert w[1] * w[3] == ch.sign_stack
    assert np.array_equal(ctx.fields(), fields)


def run_pair(spec, n_sweeps, n_stab, seed, prec=pqmc.FP64):
    ctx = pqmc.Context([spec], prec=prec, seed=seed, n_stab=n_stab, accept_log=1 << 20)
    ctx.sweep(n_sweeps, measure=True)
    ctx.synchronize()
    ch = opq.Chain(oracle_params(spec, n_stab=n_stab, seed=seed))
    ch.run(0, n_sweeps)
    return ctx, ch


def test_accept_sequence_10_sweeps_plain_18():
    """Plain PQMC, 18-site honeycomb, 100 slices, seed 1: identical Philox
    accept/reject sequence over 10 sweeps, G and energies to 1e-10."""
    spec = workloads.PLAIN_18
    ctx, ch = run_pair(spec, 10, 10, 1)
    d = ctx.dims()
    n = 10 * (d["Ltau"] + 2) * d["N"]
    gpu = ctx.accept_log(n)
    ora = np.array([x[3] for x in ch.accept_log], dtype=np.uint8)
    assert len(ora) == n
    assert np.array_equal(gpu, ora)
    for s, sg in ((0, 1), (1, -1)):
        assert rel_err(ctx.green(0, s), ch.G[sg]) < 1e-10
    rec = ctx.measurements()
    assert len(rec) == 10
    assert np.allclose(rec[:, 1], [m.energy for m in ch.measurements], rtol=1e-10, atol=0)
    assert np.allclose(rec[:, 2], [m.docc for m in ch.measurements], rtol=1e-10, atol=0)
    assert np.allclose(rec[:, 5], [m.s_afm for m in ch.measurements], rtol=1e-10, atol=0)
    assert np.all(rec[:, 0] == 1.0) and np.all(rec[:, 4] == 1.0)
    assert np.array_equal(ctx.fields(), ch.fields)
    obs = ctx.measure(0)
    assert np.isclose(obs["accept"], ch.acceptance, rtol=0, atol=1e-12)
    assert obs["max_dG"] < 1e-8


@pytest.mark.parametrize("spec,n_sweeps,n_stab", [
    (SMALL, 6, 5),
    (workloads.honeycomb(3, U=3.5, dtau=0.1, two_theta=2.0, g=0.55, M_N=0.07), 4, 10),
    (workloads.ChainSpec(kind=workloads.SQUARE, Lx=2, Ly=4, tp=-0.2, U=4.0, dtau=0.1, two_theta=1.0,
                         g=0.5, M_N=0.1, n_up=3, n_dn=3), 6, 5),
    (workloads.honeycomb(2, U=4.0, dtau=0.1, two_theta=0.0, g=0.6, M_N=0.21), 6, 1),   # Theta = 0: VMC
    (workloads.honeycomb(3, U=4.0, dtau=0.1, two_theta=2.0, g=0.6, M_N=0.21, n_up=1, n_dn=17), 4, 10),
])
def test_sweep_parity(spec, n_sweeps, n_stab):
    ctx, ch = run_pair(spec, n_sweeps, n_stab, 9)
    d = ctx.dims()
    n = n_sweeps * (d["Ltau"] + 2) * d["N"]
    assert np.array_equal(ctx.accept_log(n), np.array([x[3] for x in ch.accept_log], dtype=np.uint8))
    for s, sg in ((0, 1), (1, -1)):
        assert rel_err(ctx.green(0, s), ch.G[sg]) < 1e-10
    rec = ctx.measurements()
    assert np.allclose(rec[:, 1], [m.energy for m in ch.measurements], rtol=1e-10, atol=1e-12)
    assert np.allclose(rec[:, 5], [m.s_afm for m in ch.measurements], rtol=1e-10, atol=1e-14)
    assert np.array_equal(rec[:, 0], [m.sign for m in ch.measurements])
    assert np.array_equal(rec[:, 4], [m.sign_running for m in ch.measurements])


def test_g0_matches_plain_slater_pqmc():
    """g = 0 on the GPU (Gutzwiller slices present, all flips there accepted
    with R = 1) equals plain PQMC without those slices in the oracle."""
    spec = workloads.honeycomb(2, U=4.0, dtau=0.1, two_theta=2.0, g=0.0, M_N=0.1)
    ctx = pqmc.Context([spec], prec=pqmc.FP64, seed=4, n_stab=5)
    ctx.sweep(4)
    ch = opq.Chain(oracle_params(spec, n_stab=5, seed=4, gutzwiller_slices=False)).run(0, 4)
    rec = ctx.measurements()
    assert np.allclose(rec[:, 1], [m.energy for m in ch.measurements], rtol=1e-10, atol=0)


def test_batch_of_uneven_chains_equals_single_chains():
    specs = [SMALL, replace(workloads.PLAIN_18, two_theta=2.0),
             workloads.ChainSpec(kind=workloads.SQUARE, Lx=5, Ly=5, tp=-0.2, two_theta=2.0, g=0.3,
                                 n_up=11, n_dn=12),
             workloads.honeycomb(6, two_theta=2.0, g=0.6, M_N=0.21)]
    batch = pqmc.Context(specs, prec=pqmc.FP64, seed=2, n_stab=5, accept_log=1 << 16)
    batch.sweep(2)
    for c, s in enumerate(specs):
        one = pqmc.Context([s], prec=pqmc.FP64, seed=2, n_stab=5, chain_offset=c, accept_log=1 << 16)
        one.sweep(2)
        d = one.dims()
        n = 2 * (d["Ltau"] + 2) * d["N"]
        assert np.array_equal(batch.accept_log(n, c), one.accept_log(n))
        assert np.array_equal(batch.green(c, 0), one.green(0, 0))
        assert np.array_equal(batch.measurements(c), one.measurements(0))


def test_identical_chains_share_trial_orbitals_bit_for_bit():
    """Chains with one lattice and trial share one host eigensolution; the
    context uploads only the host-set part of its arena.  A batch of equal
    specs must still equal the chains run one at a time."""
    specs = [SMALL] * 3
    batch = pqmc.Context(specs, prec=pqmc.FP64, seed=4, n_stab=5, accept_log=1 << 16)
    assert 0 < batch.upload_bytes() < batch.device_bytes()
    batch.sweep(2)
    for c in range(3):
        one = pqmc.Context([SMALL], prec=pqmc.FP64, seed=4, n_stab=5, chain_offset=c, accept_log=1 << 16)
        one.sweep(2)
        d = one.dims()
        n = 2 * (d["Ltau"] + 2) * d["N"]
        assert np.array_equal(batch.accept_log(n, c), one.accept_log(n))
        assert np.array_equal(batch.green(c, 1), one.green(0, 1))


def test_fp32_stabilisation_error_and_green():
    """FP32 wraps and updates amplify rounding by about cond(B_tau) per slice;
    with a 2-slice stabilisation interval max |G - G_FP64| stays below 1e-4."""
    spec = workloads.GUTZ_72[4.0]
    fields = workloads.random_fields(spec, seed=3)
    ctx = pqmc.Context([spec], prec=pqmc.FP32, seed=7, n_stab=2)
    ctx.set_fields(fields)
    ch = opq.Chain(oracle_params(spec, n_stab=2), fields=fields)
    for s, sg in ((0, 1), (1, -1)):
        assert np.abs(ctx.green(0, s) - ch.G[sg]).max() < 1e-5
    ctx.sweep(4)
    errs = ctx.stab_errors()
    assert len(errs) == 4 * 21 and errs.max() <= 1e-4
    assert ctx.measure(0)["max_dG"] <= 1e-4


def test_fp32_stabilisation_error_distribution():
    """Over 64 chains x 6 sweeps at a 2-slice interval, after the first sweep
    (which starts from the random initial fields and holds the largest
    values), the 99.9th percentile of the per-stabilisation error stays
    below 1e-4 and the maximum below 1e-2."""
    spec = workloads.GUTZ_72[8.0]
    ctx = pqmc.Context([spec] * 64, prec=pqmc.FP32, seed=3, n_stab=2)
    ctx.sweep(6)
    hist = [ctx.stab_errors(c) for c in range(64)]
    assert all(len(h) == 6 * 41 for h in hist)
    errs = np.concatenate([h[41:] for h in hist])
    assert np.percentile(errs, 99.9) <= 1e-4 and errs.max() < 1e-2


def test_fp32_error_against_fp64_relative_to_g():
    """Against G_FP64 (assembled in FP64 from the FP64 factors), FP32 at a
    2-slice interval: after the first sweep, the 99.9th percentile of
    max |G - G_FP64| stays below 1e-4, and every stabilisation's error
    relative to max(1, max |G_FP64|) stays below 1e-4 (the absolute tail
    belongs to configurations whose G has entries of size 30-70, where FP32
    storage alone carries ~4e-6)."""
    spec = workloads.GUTZ_72[8.0]
    out = {}
    for mode in (1, 3):
        ctx = pqmc.Context([spec] * 32, prec=pqmc.FP32, seed=3, n_stab=2, dg_fp64=mode)
        ctx.sweep(5)
        out[mode] = np.concatenate([ctx.stab_errors(c)[41:] for c in range(32)])
        ctx.close()
    assert len(out[1]) == len(out[3]) == 32 * 4 * 41
    assert np.percentile(out[1], 99.9) <= 1e-4 and out[1].max() < 1e-2
    assert out[3].max() <= 1e-4
    assert np.all(out[3] <= out[1] + 1e-30)


@pytest.mark.parametrize("prec", [pqmc.FP64, pqmc.FP32, pqmc.BF16X3])
def test_mc_energy_within_3sigma_of_exact(prec):
    """64 independent chains on the 8-site cluster; the pooled estimates of E,
    docc and S_AFM agree with the exact Trotterised projection (Fock space)
    within 3 sigma."""
    spec = SMALL
    ctx = pqmc.Context([spec] * 64, prec=prec, seed=21, n_stab=5 if prec == pqmc.FP64 else 2)
    ctx.sweep(10, measure=False)
    ctx.sweep(60, measure=True)
    obs = ctx.measure(-1)
    m = opq.Model(oracle_params(spec, n_stab=5))
    c = ed.Cluster(m.K, 4, 4, spec.U)
    Ex, Dx, Sx = c.trotter_observables(m.P[1], m.P[-1], spec.g, spec.dtau, m.Ltau, m.eps)
    assert obs["n_meas"] == 64 * 60
    assert abs(obs["E"] - Ex / 8) < 3 * obs["E_err"], (obs, Ex / 8)
    assert abs(obs["docc"] - Dx / 8) < 3 * obs["docc_err"], (obs, Dx / 8)
    assert abs(obs["s_afm"] - Sx) < 3 * obs["s_afm_err"], (obs, Sx)
    assert obs["E_err"] < 0.01
    assert obs["sign"] == 1.0


def test_bf16x3_green_and_stabilisation_error():
    """BF16X3: the wrap and delayed-update products run as three BF16 tensor-core
    products (about 16 significant bits); G after the FP64 stabilisation is
    FP32-exact, the drift between stabilisations is reported per interval."""
    spec = workloads.GUTZ_72[4.0]
    fields = workloads.random_fields(spec, seed=3)
    ctx = pqmc.Context([spec], prec=pqmc.BF16X3, seed=7, n_stab=2)
    ctx.set_fields(fields)
    ch = opq.Chain(oracle_params(spec, n_stab=2), fields=fields)
    for s, sg in ((0, 1), (1, -1)):
        assert np.abs(ctx.green(0, s) - ch.G[sg]).max() < 1e-5
    batch = pqmc.Context([spec] * 32, prec=pqmc.BF16X3, seed=3, n_stab=2)
    batch.sweep(4)
    errs = np.concatenate([batch.stab_errors(c) for c in range(32)])
    assert len(errs) == 32 * 4 * 21
    assert np.median(errs) < 1e-3 and np.percentile(errs, 99) < 2e-2


def test_measure_errors_equal_oracle_estimator():
    """pqmc_measure's estimates and jackknife errors (one chain: 20 bins of
    consecutive sweeps, here with a partial last bin; pooled: over chains)
    equal the oracle's estimator and the pooled estimate on the same records
    to 1e-12."""
    ctx = pqmc.Context([SMALL] * 8, prec=pqmc.FP64, seed=31, n_stab=5)
    ctx.sweep(47, measure=True)
    for c in (0, 3):
        rec = ctx.measurements(c)
        assert len(rec) == 47
        obs = ctx.measure(c)
        s = rec[:, 0]
        for key, col in (("E", 1), ("docc", 2), ("s_afm", 5)):
            m, e = opq.estimate(rec[:, col], s)
            assert abs(obs[key] - m) <= 1e-12 * abs(m), key
            assert e > 0 and abs(obs[key + "_err"] - e) <= 1e-12 * e, key
    pooled = ctx.measure(-1)
    est = distributed.pooled_estimate(distributed.chain_sums([ctx.measurements(c) for c in range(8)]))
    for key in ("E", "docc", "s_afm"):
        assert abs(pooled[key] - est[key]) <= 1e-12 * abs(est[key]), key
        assert abs(pooled[key + "_err"] - est[key + "_err"]) <= 1e-12 * est[key + "_err"], key
    ctx.close()


def test_fp64_diagnostic_changes_nothing_but_the_recorded_error():
    """opts.dg_fp64 makes the reduced paths record max |G - G_FP64| (G_FP64
    assembled in FP64 from the FP64 factors) at each stabilisation; the chain
    itself (decisions, G, records) is the same as without it."""
    spec = workloads.GUTZ_72[4.0]
    out = {}
    for dg in (0, 1):
        ctx = pqmc.Context([spec] * 4, prec=pqmc.FP32, seed=9, n_stab=2, accept_log=1 << 16, dg_fp64=dg)
        ctx.sweep(3)
        n = 3 * (spec.n_slices + 2) * spec.n_sites
        out[dg] = [(ctx.accept_log(n, c), ctx.green(c, 1), ctx.measurements(c), ctx.stab_errors(c))
                   for c in range(4)]
        ctx.close()
    for (a0, g0, r0, e0), (a1, g1, r1, e1) in zip(out[0], out[1]):
        assert np.array_equal(a0, a1) and np.array_equal(g0, g1) and np.array_equal(r0, r1)
        assert len(e0) == len(e1) == 3 * 21
        assert np.all(np.isfinite(e1)) and e1.max() < 1e-2 and not np.array_equal(e0, e1)

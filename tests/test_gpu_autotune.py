"""Delayed-update block sizes and the autotuner (GPU, through the C-ABI).

Every delayed block (8, 16, 32, 64 sites) applies the same sequence of
Sherman-Morrison updates, regrouped: in FP64 the accept/reject sequence and G
equal the oracle's single-flip chain (the oracle's own delayed = Sherman-
Morrison pin).  The autotuner's pick, timed on a shortened proxy batch, is
within 5% of the fastest candidate timed on the full batch."""
import time

import numpy as np
import pytest

from oracle import pqmc as opq
from paper_2303_13403_gb300 import pqmc, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    torch.cuda.set_device(0)
    pqmc.load()


def oracle_params(spec, **kw):
    base = dict(kind=spec.kind, Lx=spec.Lx, Ly=spec.Ly, t=spec.t, tp=spec.tp, U=spec.U, dtau=spec.dtau,
                two_theta=spec.two_theta, g=spec.g, M_N=spec.M_N, n_up=spec.n_up, n_dn=spec.n_dn,
                tiebreak=spec.tiebreak)
    base.update(kw)
    return opq.Params(**base)


@pytest.mark.parametrize("k", [8, 16, 32, 64])
def test_delay_blocks_follow_oracle_fp64(k):
    """72 sites (blocks of 64 span two decision sub-blocks and a ragged tail):
    two FP64 sweeps give the oracle's accept sequence, G to 1e-10 and the
    energies to 1e-10."""
    spec = workloads.honeycomb(6, U=4.0, dtau=0.1, two_theta=2.0, g=0.6, M_N=0.21)
    ctx = pqmc.Context([spec], prec=pqmc.FP64, seed=19, n_stab=5, delay_k=k, accept_log=1 << 16)
    assert ctx.launch()["delay_k"] == k and ctx.dims()["delay_k"] == k
    ctx.sweep(2)
    d = ctx.dims()
    n = 2 * (d["Ltau"] + 2) * d["N"]
    ch = opq.Chain(oracle_params(spec, n_stab=5, seed=19))
    ch.run(0, 2)
    assert np.array_equal(ctx.accept_log(n), np.array([x[3] for x in ch.accept_log], dtype=np.uint8))
    for s, sg in ((0, 1), (1, -1)):
        assert np.abs(ctx.green(0, s) - ch.G[sg]).max() / np.abs(ch.G[sg]).max() < 1e-10
    assert np.allclose(ctx.measurements(0)[:, 1], [m.energy for m in ch.measurements], rtol=0, atol=1e-10)
    ctx.close()


@pytest.mark.parametrize("k,L", [(8, 6), (64, 6), (64, 9)])
def test_delay_blocks_fp32_against_definition(k, L):
    """FP32 sweeps with the smallest and largest blocks (72 sites resident in
    shared memory, 162 sites in global memory): G after each sweep against
    the oracle's definition on the GPU's fields to 1e-4."""
    spec = workloads.honeycomb(L, U=4.0, dtau=0.1, two_theta=2.0, g=0.6, M_N=0.21)
    ctx = pqmc.Context([spec], prec=pqmc.FP32, seed=23, n_stab=2, delay_k=k)
    model = opq.Model(oracle_params(spec, n_stab=2))
    for sw in (1, 2):
        ctx.sweep(1)
        tau = model.Ltau + 1 if sw % 2 else -1
        f = ctx.fields(0)
        for s, sg in ((0, 1), (1, -1)):
            assert np.abs(ctx.green(0, s) - opq.green_definition(model, f, tau, sg)).max() < 1e-4
    ctx.close()


def test_tv_chains_ignore_delay_k():
    """t-V chains propose bonds in blocks of 16 whatever delay_k is."""
    spec = workloads.tv_honeycomb(3, V=1.35, g=0.3, two_theta=2.0)
    out = []
    for k in (8, 64):
        ctx = pqmc.Context([spec], prec=pqmc.FP64, seed=4, n_stab=5, delay_k=k, accept_log=1 << 16)
        ctx.sweep(2)
        out.append((ctx.accept_log(4000), ctx.green(0, 0)))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def full_ms(specs, prec, n_stab, k, tpb):
    ctx = pqmc.Context(specs, prec=prec, seed=5, n_stab=n_stab, delay_k=k, cta_threads=tpb)
    ctx.sweep(1, measure=False)
    ctx.synchronize()
    t0 = time.perf_counter()
    ctx.sweep(2, measure=False)
    ctx.synchronize()
    ms = (time.perf_counter() - t0) / 2 * 1e3
    ctx.close()
    return ms


@pytest.mark.parametrize("L,two_theta,chains", [(6, 4.0, 304), (12, 2.0, 76)])
def test_autotune_pick_within_5_percent_of_exhaustive(L, two_theta, chains):
    spec = workloads.honeycomb(L, U=4.0, dtau=0.1, two_theta=two_theta, g=0.6, M_N=0.21)
    specs = [spec] * chains
    t = pqmc.autotune(specs, prec=pqmc.FP32, n_stab=2)
    assert t["delay_k"] in (8, 16, 32, 64) and t["cta_threads"] in (64, 128, 256, 512)
    assert len(t["candidates"]) == 16 and all(np.isfinite(c["ms_per_sweep"]) for c in t["candidates"])
    full = {(c["delay_k"], c["cta_threads"]): full_ms(specs, pqmc.FP32, 2, c["delay_k"], c["cta_threads"])
            for c in t["candidates"]}
    best = min(full.values())
    assert full[(t["delay_k"], t["cta_threads"])] <= 1.05 * best, (t, full)
    # a context asking for the autotuner gets the cached pick
    ctx = pqmc.Context(specs, prec=pqmc.FP32, seed=1, n_stab=2, delay_k=0)
    shape = ctx.launch()
    assert (shape["delay_k"], shape["cta_threads"]) == (t["delay_k"], t["cta_threads"])
    ctx.close()
    again = pqmc.autotune(specs, prec=pqmc.FP32, n_stab=2)
    assert again["from_cache"] and (again["delay_k"], again["cta_threads"]) == (t["delay_k"], t["cta_threads"])

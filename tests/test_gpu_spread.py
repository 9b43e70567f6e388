"""Chains swept by grid-wide kernels (pqmc_opts.spread) against the oracle and
against the one-CTA path (GPU, through the C-ABI).

The spread sweep runs the same Metropolis decisions on the same Philox stream
as the one-CTA sweep, with the delayed update, the wrap and the stabilisation
as tile products, a blocked Cholesky QR and a blocked Gauss-Jordan inverse.
Checked here: G after whole sweeps against the oracle's definition of the
equal-time Green's function (Method section: G = 1 - B_R (B_L B_R)^{-1} B_L,
products re-orthonormalised after every slice) on the GPU's own fields (FP64
to 1e-10 relative, FP32 to 1e-4, BF16X3 to 2e-3 absolute), the FP64
accept/reject sequence against an oracle chain from the same seed, the FP64
energies against the one-CTA path, batches against single chains, and a
checkpoint round trip."""
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


def gutz(L, two_theta):
    return workloads.honeycomb(L, U=4.0, dtau=0.1, two_theta=two_theta, g=0.6, M_N=0.21)


CASES = [
    # (L, 2 Theta, precision, sweeps): 162, 288 and 648 sites (ragged 32-site blocks and panels)
    (9, 2.0, pqmc.FP64, 2),
    (12, 2.0, pqmc.FP64, 1),
    (9, 4.0, pqmc.FP32, 2),
    (12, 2.0, pqmc.FP32, 2),
    (18, 2.0, pqmc.FP32, 1),
    (9, 4.0, pqmc.BF16X3, 2),
    (12, 2.0, pqmc.BF16X3, 1),
]


@pytest.mark.parametrize("L,two_theta,prec,sweeps", CASES)
def test_spread_sweeps_against_green_definition(L, two_theta, prec, sweeps):
    spec = gutz(L, two_theta)
    N = spec.n_sites
    ctx = pqmc.Context([spec], prec=prec, seed=11, n_stab=2, spread=1)
    model = opq.Model(oracle_params(spec, n_stab=2))
    for k in range(1, sweeps + 1):
        ctx.sweep(1)
        ctx.synchronize()
        f = ctx.fields(0)
        tau = model.Ltau + 1 if k % 2 else -1
        for s, sg in ((0, 1), (1, -1)):
            G = ctx.green(0, s)
            Gd = opq.green_definition(model, f, tau, sg)
            if prec == pqmc.FP64:
                err = np.abs(G - Gd).max() / np.abs(Gd).max()
                assert err < 1e-10, (N, k, s, err)
            else:
                err = np.abs(G - Gd).max()
                assert err < (1e-4 if prec == pqmc.FP32 else 2e-3), (N, k, s, err)
        assert abs(N - np.trace(ctx.green(0, 0)) - N // 2) < (1e-9 if prec == pqmc.FP64 else 1e-3)
    rec = ctx.measurements(0)
    assert len(rec) == sweeps and np.all(rec[:, 0] == 1.0) and np.all(np.isfinite(rec))
    assert np.isfinite(ctx.measure(0)["max_dG"])
    ctx.close()


def test_spread_accept_sequence_against_oracle_fp64():
    """Two FP64 sweeps of a 162-site chain: the accept/reject sequence, G and
    the energies of an oracle chain run from the same seed."""
    spec = gutz(9, 2.0)
    ctx = pqmc.Context([spec], prec=pqmc.FP64, seed=13, n_stab=2, accept_log=1 << 16, spread=1)
    ctx.sweep(2)
    d = ctx.dims()
    n = 2 * (d["Ltau"] + 2) * d["N"]
    gpu_log = ctx.accept_log(n)
    ch = opq.Chain(oracle_params(spec, n_stab=2, seed=13))
    ch.run(0, 2)
    ora_log = np.array([x[3] for x in ch.accept_log], dtype=np.uint8)
    assert len(ora_log) == n
    assert np.array_equal(gpu_log, ora_log)
    for s, sg in ((0, 1), (1, -1)):
        assert np.abs(ctx.green(0, s) - ch.G[sg]).max() / np.abs(ch.G[sg]).max() < 1e-10
    rec = ctx.measurements(0)
    assert np.allclose(rec[:, 1], [m.energy for m in ch.measurements], rtol=0, atol=1e-10)
    ctx.close()


def test_spread_equals_one_cta_path_fp64():
    """Same seed, spread and one-CTA FP64 paths: identical accept sequences
    over four sweeps, G and the records equal to rounding."""
    spec = gutz(9, 2.0)
    kw = dict(prec=pqmc.FP64, seed=21, n_stab=2, accept_log=1 << 17)
    a = pqmc.Context([spec], spread=1, **kw)
    b = pqmc.Context([spec], cta_threads=256, **kw)
    a.sweep(4)
    b.sweep(4)
    n = 4 * (a.dims()["Ltau"] + 2) * a.dims()["N"]
    assert np.array_equal(a.accept_log(n), b.accept_log(n))
    assert np.array_equal(a.fields(0), b.fields(0))
    for s in (0, 1):
        assert np.abs(a.green(0, s) - b.green(0, s)).max() < 1e-10
    ra, rb = a.measurements(0), b.measurements(0)
    assert np.allclose(ra, rb, rtol=0, atol=1e-10)
    a.close()
    b.close()


def test_spread_init_matches_one_cta_init_fp64():
    """The spread initialisation (left stack, right block 0, G at tau = -1)
    gives the one-CTA initialisation's G to 1e-10 and the oracle's definition
    of G at tau = -1 on the initial fields."""
    spec = gutz(9, 4.0)
    a = pqmc.Context([spec], prec=pqmc.FP64, seed=17, n_stab=2, spread=1)
    b = pqmc.Context([spec], prec=pqmc.FP64, seed=17, n_stab=2, cta_threads=256)
    model = opq.Model(oracle_params(spec, n_stab=2))
    f = a.fields(0)
    assert np.array_equal(f, b.fields(0))
    for s, sg in ((0, 1), (1, -1)):
        Gd = opq.green_definition(model, f, -1, sg)
        for ctx in (a, b):
            assert np.abs(ctx.green(0, s) - Gd).max() / np.abs(Gd).max() < 1e-10
    a.close()
    b.close()


def test_spread_batch_equals_single_chains():
    """Three chains of one shape in one spread context give the chains run
    alone, bit for bit (FP32)."""
    specs = [workloads.honeycomb(9, U=4.0, dtau=0.1, two_theta=2.0, g=g, M_N=0.21) for g in (0.3, 0.6, 0.9)]
    batch = pqmc.Context(specs, prec=pqmc.FP32, seed=5, n_stab=2, spread=1)
    batch.sweep(2)
    for c, sp in enumerate(specs):
        one = pqmc.Context([sp], prec=pqmc.FP32, seed=5, n_stab=2, chain_offset=c, spread=1)
        one.sweep(2)
        assert np.array_equal(one.fields(0), batch.fields(c))
        for s in (0, 1):
            assert np.array_equal(one.green(0, s), batch.green(c, s))
        assert np.array_equal(one.measurements(0), batch.measurements(c))
        one.close()
    batch.close()


def test_spread_checkpoint_restore():
    """A spread context restored from a checkpoint continues the run bit for bit."""
    spec = gutz(9, 2.0)
    a = pqmc.Context([spec], prec=pqmc.FP32, seed=9, n_stab=2, spread=1)
    a.sweep(1)
    data = a.checkpoint()
    a.sweep(2)
    b = pqmc.Context([spec], prec=pqmc.FP32, seed=9, n_stab=2, spread=1)
    b.restore(data)
    b.sweep(2)
    assert np.array_equal(a.fields(0), b.fields(0))
    for s in (0, 1):
        assert np.array_equal(a.green(0, s), b.green(0, s))
    a.close()
    b.close()


def test_spread_rejects_mixed_shapes_and_tv():
    with pytest.raises(pqmc.PQMCError):
        pqmc.Context([gutz(9, 2.0), gutz(6, 2.0)], prec=pqmc.FP32, n_stab=2, spread=1)
    with pytest.raises(pqmc.PQMCError):
        pqmc.Context([workloads.tv_honeycomb(6, V=1.6, g=0.3, Delta_C=0.24, two_theta=2.0)], prec=pqmc.FP32,
                     n_stab=2, spread=1)

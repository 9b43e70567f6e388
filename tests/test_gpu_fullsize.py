"""The bench workload at its full size and launch configuration (608 chains of
the 72-site Gutzwiller PQMC, 2 Theta = 8, default CTA shapes): sampled chains
against the oracle's G computed from its definition on the GPU's own fields,
and properties that hold for every chain."""
import numpy as np
import pytest

from oracle import pqmc as opq
from paper_2303_13403_gb300 import pqmc, workloads

pytestmark = pytest.mark.gpu

SPEC = workloads.GUTZ_72[8.0]
CHAINS = 608
SAMPLE = (0, 151, 303, 304, 607)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    torch.cuda.set_device(0)
    pqmc.load()


def oracle_model(n_stab):
    return opq.Model(opq.Params(kind=SPEC.kind, Lx=SPEC.Lx, Ly=SPEC.Ly, U=SPEC.U, dtau=SPEC.dtau,
                                two_theta=SPEC.two_theta, g=SPEC.g, M_N=SPEC.M_N, n_stab=n_stab))


@pytest.mark.parametrize("prec,n_stab,tol", [(pqmc.FP64, 10, 1e-10), (pqmc.FP32, 2, 1e-3)])
def test_full_batch_against_definition(prec, n_stab, tol):
    """After two sweeps (G = G(-1) of the final fields) every sampled chain's
    G matches the oracle's definition on the same fields (FP64: 1e-10
    relative; FP32: 1e-3 absolute, the stabilisation-error tail), every
    chain has Tr(1 - G_sigma) = N_sigma, and the weight sign equals the
    running sign in every record."""
    ctx = pqmc.Context([SPEC] * CHAINS, prec=prec, seed=1, n_stab=n_stab)
    ctx.sweep(2)
    ctx.synchronize()
    m = oracle_model(n_stab)
    for c in SAMPLE:
        f = ctx.fields(c)
        for s, sg in ((0, 1), (1, -1)):
            Gd = opq.green_definition(m, f, -1, sg)
            G = ctx.green(c, s)
            err = np.abs(G - Gd).max() / (np.abs(Gd).max() if prec == pqmc.FP64 else 1.0)
            assert err < tol, (c, s, err)
    trace_tol = 1e-9 if prec == pqmc.FP64 else 1e-3
    for c in range(CHAINS):
        for s in (0, 1):
            assert abs(np.trace(np.eye(72) - ctx.green(c, s)) - 36) < trace_tol, c
        rec = ctx.measurements(c)
        assert len(rec) == 2 and np.all(np.isfinite(rec))
        assert np.array_equal(rec[:, 0], rec[:, 4])
    obs = ctx.measure(-1)
    assert obs["n_meas"] == 2 * CHAINS and obs["sign"] == 1.0

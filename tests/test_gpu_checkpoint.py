"""Checkpoint / restore and the recomputation of G at a stabilisation point,
through the C-ABI: a restored run continues the checkpointed one exactly,
mismatched contexts are refused, and G(tau = b n_stab) recomputed by the
kernels matches the oracle's definition of G on the same fields at every
stabilisation point without disturbing the chain."""
import ctypes as C

import numpy as np
import pytest

from oracle import pqmc as opq
from oracle import tv
from paper_2303_13403_gb300 import pqmc, workloads

pytestmark = pytest.mark.gpu

SMALL = workloads.honeycomb(2, U=4.0, dtau=0.1, two_theta=2.0, g=0.6, M_N=0.21)
BATCH = [SMALL,
         workloads.honeycomb(6, two_theta=2.0, g=0.6, M_N=0.21),
         workloads.ChainSpec(kind=workloads.SQUARE, Lx=5, Ly=5, tp=-0.2, two_theta=2.0, g=0.3, n_up=11, n_dn=12),
         workloads.tv_honeycomb(3, V=1.35, g=0.3, two_theta=2.0)]


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


def tv_params(spec, **kw):
    base = dict(Lx=spec.Lx, Ly=spec.Ly, t=spec.t, V=spec.U, dtau=spec.dtau, two_theta=spec.two_theta,
                g=spec.g, Delta_C=spec.M_N, tiebreak=spec.tiebreak)
    base.update(kw)
    return tv.TVParams(**base)


def n_proposals(ctx, c, n_sweeps):
    d = ctx.dims(c)
    return n_sweeps * (d["Ltau"] + 2) * d["n_fields"]


def state_of(ctx, n_sweeps):
    out = []
    for c in range(len(BATCH)):
        out.append(dict(acc=ctx.accept_log(n_proposals(ctx, c, n_sweeps), c), G0=ctx.green(c, 0),
                        G1=ctx.green(c, 1), f=ctx.fields(c), rec=ctx.measurements(c), w=ctx.weight(c),
                        dG=ctx.stab_errors(c)))
    return out


@pytest.mark.parametrize("prec,first,tpb", [(pqmc.FP64, 3, 0), (pqmc.FP32, 2, 0), (pqmc.FP32, 3, 128),
                                            (pqmc.BF16X3, 1, 0)])
def test_restored_run_continues_exactly(prec, first, tpb):
    """Run A: `first` sweeps, checkpoint, 3 more. Run B: a new context with the
    same specs (FP32: also another CTA size), restore, 3 sweeps. Accept
    sequences, G, fields, records, weights and stabilisation errors agree
    bit for bit, with the checkpoint taken after an even or odd number of
    sweeps (the next sweep going up or down). Across CTA sizes the records'
    CTA-wide sums are added in another order, so there they agree to
    rounding."""
    kw = dict(prec=prec, seed=5, n_stab=2, accept_log=1 << 16)
    a = pqmc.Context(BATCH, **kw)
    a.sweep(first)
    data = a.checkpoint()
    a.sweep(3)
    b = pqmc.Context(BATCH, cta_threads=tpb, **kw)
    b.sweep(1)                       # state that the restore must overwrite
    b.restore(data)
    b.sweep(3)
    sa, sb = state_of(a, first + 3), state_of(b, first + 3)
    for c, (x, y) in enumerate(zip(sa, sb)):
        for k in x:
            if k == "rec" and tpb:
                assert np.allclose(x[k], y[k], rtol=1e-12, atol=1e-14), c
            else:
                assert np.array_equal(x[k], y[k]), (c, k)
    assert len(sa[0]["rec"]) == first + 3
    oa, ob = a.measure(1), b.measure(1)
    for k in ("E", "docc", "sign", "accept", "n_meas"):
        assert np.isclose(oa[k], ob[k], rtol=1e-12, atol=0) if tpb else oa[k] == ob[k], k
    a.close()
    b.close()


@pytest.mark.parametrize("code", [pqmc.ENAN, pqmc.ESTAB])
def test_failed_chain_is_sticky_and_restore_resumes(code):
    """The failure path, without a GPU fault: one chain is marked failed from
    the host exactly as a kernel that met a NaN or a singular pivot marks it
    (pqmc_inject_error). The next synchronisation reports the error; sweeps
    and checkpoints are then refused with the same code; restoring the last
    good checkpoint clears it and the resumed run continues the uninterrupted
    one bit for bit."""
    kw = dict(prec=pqmc.FP32, seed=8, n_stab=2, accept_log=1 << 16)
    ref = pqmc.Context(BATCH, **kw)
    ref.sweep(5)
    a = pqmc.Context(BATCH, **kw)
    a.sweep(2)
    good = a.checkpoint()
    a.sweep(1)
    a.inject_error(code, chain=1)
    for call in (a.synchronize, lambda: a.sweep(1), a.checkpoint, lambda: a.measure(-1)):
        with pytest.raises(pqmc.PQMCError) as e:
            call()
        assert e.value.status == code
    a.restore(good)
    a.sweep(3)
    sr, sa = state_of(ref, 5), state_of(a, 5)
    for c, (x, y) in enumerate(zip(sr, sa)):
        for k in x:
            assert np.array_equal(x[k], y[k]), (c, k)
    ref.close()
    a.close()


def test_restore_refuses_other_contexts():
    kw = dict(prec=pqmc.FP32, seed=5, n_stab=2)
    a = pqmc.Context(BATCH, **kw)
    a.sweep(1)
    data = a.checkpoint()
    lib = pqmc.load()
    others = [pqmc.Context(BATCH, prec=pqmc.FP32, seed=6, n_stab=2),          # seed
              pqmc.Context(BATCH, prec=pqmc.FP64, seed=5, n_stab=2),          # precision
              pqmc.Context(BATCH[:3], **kw),                                  # chain count
              pqmc.Context([BATCH[1]] + BATCH[1:], **kw),                     # one spec differs
              pqmc.Context(BATCH, prec=pqmc.FP32, seed=5, n_stab=5),          # n_stab
              pqmc.Context(BATCH, max_meas=100, **kw)]                        # record capacity
    for o in others:
        with pytest.raises(pqmc.PQMCError) as e:
            o.restore(data)
        assert e.value.status == pqmc.EINVAL
        o.close()
    same = pqmc.Context(BATCH, **kw)
    for bad in (data[:-1], data + b"\0", b"\0" * len(data), data[:16]):
        with pytest.raises(pqmc.PQMCError) as e:
            same.restore(bad)
        assert e.value.status == pqmc.EINVAL
    # a buffer that is too small is refused and told the size
    n = C.c_size_t(16)
    buf = (C.c_ubyte * 16)()
    assert lib.pqmc_checkpoint(a.handle, buf, C.byref(n)) == pqmc.EINVAL
    assert n.value == len(data)
    same.restore(data)
    same.sweep(1)
    a.sweep(1)
    for c in range(len(BATCH)):
        assert np.array_equal(a.green(c, 0), same.green(c, 0))
    a.close()
    same.close()


@pytest.mark.parametrize("prec,tol", [(pqmc.FP64, 1e-10), (pqmc.FP32, 1e-4)])
def test_green_at_every_stabilisation_point(prec, tol):
    """G(tau = b n_stab) recomputed by the kernels from the chains' fields
    after two sweeps, for every b, against the oracle's definition of G
    (FP64: relative 1e-10; FP32: absolute 1e-4). The chains then continue
    exactly as an undisturbed twin context."""
    n_stab = 2
    kw = dict(prec=prec, seed=8, n_stab=n_stab, accept_log=1 << 16)
    ctx = pqmc.Context(BATCH, **kw)
    twin = pqmc.Context(BATCH, **kw)
    ctx.sweep(2)
    twin.sweep(2)
    for c, spec in enumerate(BATCH):
        f = ctx.fields(c)
        is_tv = spec.kind == workloads.HONEYCOMB_TV
        m = tv.TVModel(tv_params(spec, n_stab=n_stab)) if is_tv else opq.Model(oracle_params(spec, n_stab=n_stab))
        nb = ctx.dims(c)["Ltau"] // n_stab
        for b in range(nb + 1):
            for s, sg in ((0, 1),) if is_tv else ((0, 1), (1, -1)):
                Gd = tv.green_definition(m, f, b * n_stab) if is_tv else opq.green_definition(m, f, b * n_stab, sg)
                G = ctx.green_at(b, c, s)
                err = np.abs(G - Gd).max() / (np.abs(Gd).max() if prec == pqmc.FP64 else 1.0)
                assert err < tol, (c, b, s, err)
        with pytest.raises(pqmc.PQMCError):
            ctx.green_at(nb + 1, c)
    ctx.sweep(2)
    twin.sweep(2)
    for c in range(len(BATCH)):
        n = n_proposals(ctx, c, 4)
        assert np.array_equal(ctx.accept_log(n, c), twin.accept_log(n, c))
        assert np.array_equal(ctx.green(c, 0), twin.green(c, 0))
        assert np.array_equal(ctx.measurements(c), twin.measurements(c))
    ctx.close()
    twin.close()

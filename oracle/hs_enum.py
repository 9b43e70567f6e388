"""Exact sum over all auxiliary-field configurations (test infrastructure only).

For systems with at most ~16 fields the HS sum of the Method section can be
done exactly: weight W(s) = prod_sigma det(P^T B_{Ltau+1} ... B_0 P) and the
estimator sum_s W(s) O(s) / sum_s W(s), with O(s) the Wick estimate on
G(Ltau/2).  It must equal the exact Trotterised projection of ``ed``; the
average sign is sum_s W / sum_s |W|.  All configurations are processed at once
as one batch of small dense products.
"""
import numpy as np

from . import pqmc


def all_fields(n_fields):
    """Every +-1 configuration of n_fields fields, shape (2**n_fields, n_fields)."""
    idx = np.arange(2 ** n_fields)[:, None]
    bits = (idx >> np.arange(n_fields)[None, :]) & 1
    return np.where(bits == 1, 1, -1).astype(np.int8)


def enumerate_estimator(params):
    """(E, docc, average sign) of the exact field sum."""
    r = enumerate_observables(params)
    return r["E"], r["docc"], r["sign"]


def enumerate_observables(params):
    """Exact field sum of E, docc and S_AFM (all per the Wick estimates of
    ``pqmc.Chain.measure``) and the average sign, as a dict."""
    m = pqmc.Model(params)
    N, Lt = m.N, m.Ltau
    n_fields = (Lt + 2) * N
    if n_fields > 20:
        raise ValueError("too many fields to enumerate")
    F = all_fields(n_fields).reshape(-1, Lt + 2, N)
    C = F.shape[0]
    W = np.ones(C)
    G = {}
    for sigma in (+1, -1):
        def bmat(t):
            d = np.exp(sigma * m.kappa(t) * F[:, t, :].astype(np.float64))   # C x N
            if m.is_gutz(t):
                return d[:, :, None] * np.eye(N)[None]
            return m.expKm[None] * d[:, None, :]                            # K e^{V}
        BR = np.broadcast_to(m.P[sigma], (C,) + m.P[sigma].shape).copy()
        for t in range(0, Lt // 2 + 1):
            BR = bmat(t) @ BR
        BL = np.broadcast_to(m.P[sigma].T, (C,) + m.P[sigma].T.shape).copy()
        for t in range(Lt + 1, Lt // 2, -1):
            BL = BL @ bmat(t)
        O = BL @ BR
        W = W * np.linalg.det(O)
        G[sigma] = np.eye(N)[None] - BR @ np.linalg.solve(O, BL)
    ekin = sum(np.einsum("ij,cji->c", m.K, np.eye(N)[None] - G[sg]) for sg in (+1, -1))
    dg = {sg: np.diagonal(G[sg], axis1=1, axis2=2) for sg in (+1, -1)}
    docc = np.sum((1 - dg[+1]) * (1 - dg[-1]), axis=1)
    E = ekin + params.U * docc
    # staggered S^z structure factor: (stagger^2 + same-spin exchange)/(4 N^2)
    stag = np.einsum("i,ci->c", m.eps, dg[-1] - dg[+1])
    exch = sum(np.einsum("i,j,cji,cij->c", m.eps, m.eps, np.eye(N)[None] - G[sg], G[sg])
               for sg in (+1, -1))
    S = (stag ** 2 + exch) / (4.0 * N * N)
    tot = np.sum(W)
    return {"E": float(np.sum(W * E) / tot), "docc": float(np.sum(W * docc) / tot),
            "s_afm": float(np.sum(W * S) / tot), "sign": float(tot / np.sum(np.abs(W)))}

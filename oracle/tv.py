"""Spinless t-V model on the honeycomb lattice (test infrastructure only).

Repulsive spinless honeycomb section, Eq. (4):
    H = -t sum_<ij> (c^+_i c_j + h.c.) + V sum_<ij> (n_i - 1/2)(n_j - 1/2),
at half filling (N/2 fermions), with the trial state of Eq. (5)
    |psi_T> = exp(-g sum_<ij> n_i n_j) |psi_C>,
psi_C the N/2 lowest orbitals of H_C = H_0 + Delta_C sum_i eps_i n_i (eps_i = +1
on A, -1 on B, the same reading of the printed sublattice sign as for the
Hubbard model; at Delta_C below 1e-4 the field is raised to 1e-4, which opens
the zero-mode shell of L = 3m clusters).

Readings (the paper says only that V is decoupled "in the density channel"):

* Bonds: bond b = 3 c + k of cell c = x + Lx y joins A(x, y) to B(x, y) (k = 0),
  B(x-1, y) (k = 1) or B(x, y-1) (k = 2), the hopping bonds of ``lattice``;
  on clusters that wrap onto themselves a doubled bond appears twice, in H
  and in the fields alike.  Each class k is a perfect matching of the sites.
* HS of a bond, the identity of Eq. (1) read in the density-difference
  channel: exp(-a (n_i - 1/2)(n_j - 1/2)) = 1/2 exp(-a/4) sum_s exp(kappa s (n_i - n_j)),
  cosh kappa = exp(a/2); a = dtau V in the interaction slices (kappa = alpha),
  a = g in the two Gutzwiller slices (kappa = lambda).  At fixed particle
  number exp(-g sum_b n_i n_j) equals prod_b exp(-g (n_i-1/2)(n_j-1/2)) times a
  constant, because every site lies on three bonds.  The fields are real and
  the weight is a single determinant: it can be negative (the sign problem
  studied in Fig. 4).
* Slices as for the Hubbard chain: tau = 0 and Ltau + 1 carry Gutzwiller bond
  fields (no kinetic factor), B_tau = e^{-dtau K} e^{V(s_tau)} in between, with
  V(s)_ii = kappa sum_b D_ib s_b, D_ib = +1 at the A end of b, -1 at its B end.
* Updates: single-bond Metropolis, accept iff u < |R|, the bonds of a slice
  visited class by class (k = 0, 1, 2), cells ascending within a class; the
  Philox counter is (b, tau, sweep, chain).  Flipping s_b changes V at its two
  ends by Gamma = diag(e^{-2 kappa s_b} - 1, e^{2 kappa s_b} - 1) and
      R = det(1 + Gamma (1 - G)_SS),
      G <- G - (E_S - G_{:,S}) Gamma (1 + (1 - G_SS) Gamma)^{-1} G_{S,:},
  S = (A end, B end): the rank-2 form of the single-site update.
* Measurement at tau = Ltau/2 by Wick's theorem (one species):
  <c^+_i c_j> = delta_ij - G_ji, <(n_i - 1/2)(n_j - 1/2)> =
  (n_i - 1/2)(n_j - 1/2) + (delta_ij - G_ji) G_ij; the CDW structure factor
  (definition in the unavailable supplement) is read as
  S_CDW = (1/N^2) sum_ij eps_i eps_j <(n_i - 1/2)(n_j - 1/2)>.
"""
from dataclasses import dataclass

import numpy as np

from . import ed, hs, lattice, philox
from .pqmc import StackEntry


@dataclass
class TVParams:
    Lx: int = 3
    Ly: int = 3
    t: float = 1.0
    V: float = 1.6
    dtau: float = 0.1
    two_theta: float = 4.0
    g: float = 0.0
    Delta_C: float = 0.0
    n_f: int = -1           # -1: half filling
    tiebreak: float = -1.0  # <0: 1e-4
    n_stab: int = 10
    seed: int = 1
    chain: int = 0


def bonds(Lx, Ly):
    """(A end, B end) of every bond b = 3 c + k, as an (3 Lx Ly) x 2 array."""
    def site(x, y, sub):
        return 2 * ((x % Lx) + Lx * (y % Ly)) + sub
    out = []
    for y in range(Ly):
        for x in range(Lx):
            a = site(x, y, 0)
            for bx, by in ((x, y), (x - 1, y), (x, y - 1)):
                out.append((a, site(bx, by, 1)))
    return np.array(out, dtype=np.int64)


def visiting_order(Lx, Ly):
    """Bond indices in the order they are proposed within a slice."""
    nc = Lx * Ly
    return [3 * c + k for k in range(3) for c in range(nc)]


class TVModel:
    def __init__(self, p: TVParams):
        self.p = p
        self.K, self.eps = lattice.honeycomb(p.Lx, p.Ly, p.t)
        self.N = N = self.K.shape[0]
        self.bond = bonds(p.Lx, p.Ly)
        self.nbond = len(self.bond)
        self.D = np.zeros((N, self.nbond))
        for b, (i, j) in enumerate(self.bond):
            self.D[i, b] += 1.0
            self.D[j, b] -= 1.0
        self.order = visiting_order(p.Lx, p.Ly)
        self.Ltau = int(round(p.two_theta / p.dtau))
        if self.Ltau % 2 or (self.Ltau // 2) % p.n_stab:
            raise ValueError("Ltau/2 must be a multiple of n_stab")
        self.nb = self.Ltau // p.n_stab
        self.n_f = N // 2 if p.n_f < 0 else p.n_f
        w, v = np.linalg.eigh(self.K)
        self.expKm = (v * np.exp(-p.dtau * w)) @ v.T
        self.expKp = (v * np.exp(+p.dtau * w)) @ v.T
        tb = 1e-4 if p.tiebreak < 0 else p.tiebreak
        e, u = np.linalg.eigh(self.K + max(p.Delta_C, tb) * np.diag(self.eps))
        self.P = u[:, :self.n_f].copy()
        self.gap = float(e[self.n_f] - e[self.n_f - 1]) if self.n_f < N else np.inf
        self.alpha = hs.coupling(p.dtau * p.V)
        self.lam = hs.coupling(p.g)

    def is_gutz(self, tau):
        return tau == 0 or tau == self.Ltau + 1

    def kappa(self, tau):
        return self.lam if self.is_gutz(tau) else self.alpha

    def vdiag(self, tau, s_row):
        """Diagonal of e^{V(s_tau)}."""
        return np.exp(self.kappa(tau) * (self.D @ s_row.astype(np.float64)))

    def B(self, tau, s_row):
        d = self.vdiag(tau, s_row)
        if self.is_gutz(tau):
            return np.diag(d)
        return self.expKm @ np.diag(d)


def green_definition(model, fields, tau):
    """G(tau) = 1 - B_R (B_L B_R)^{-1} B_L from its definition, with the
    partial products re-orthonormalised by QR (G depends only on their spans)."""
    R = model.P.copy()
    for t in range(0, tau + 1):
        R, _ = np.linalg.qr(model.B(t, fields[t]) @ R)
    Lt = model.P.copy()
    for t in range(model.Ltau + 1, tau, -1):
        Lt, _ = np.linalg.qr(model.B(t, fields[t]).T @ Lt)
    L = Lt.T
    return np.eye(model.N) - R @ np.linalg.solve(L @ R, L)


def log_weight_definition(model, fields):
    """log|det(P^T B_{Ltau+1} ... B_0 P)| and its sign, by QR after every slice."""
    M = model.P.copy()
    logabs, sign = 0.0, 1.0
    for t in range(0, model.Ltau + 1):
        M, r = np.linalg.qr(model.B(t, fields[t]) @ M)
        d = np.diag(r)
        logabs += float(np.sum(np.log(np.abs(d))))
        sign *= float(np.prod(np.sign(d)))
    s, ld = np.linalg.slogdet(model.P.T @ model.B(model.Ltau + 1, fields[model.Ltau + 1]) @ M)
    return logabs + ld, sign * s


@dataclass
class TVMeasurement:
    sweep: int
    sign: float          # sign of the weight, from the stabilised stacks
    sign_running: float  # running product of sgn(R)
    energy: float        # <H> per site for Eq. (4)
    kinetic: float       # kinetic energy per site
    ebond: float         # V sum_b <(n_i-1/2)(n_j-1/2)> per site
    s_cdw: float         # CDW structure factor


class TVChain:
    """One Markov chain of the spinless t-V model and its sweep algorithm."""

    def __init__(self, p: TVParams, fields=None):
        self.p = p
        self.m = m = TVModel(p)
        if fields is None:
            fields = philox.initial_fields(p.seed, p.chain, m.Ltau + 2, m.nbond)
        self.fields = np.array(fields, dtype=np.int8).copy()
        self.sweep_index = 0
        self.sign_running = 1.0
        self.accept_log = []          # (sweep, tau, b, accepted) in visiting order
        self.measurements = []
        self.max_dG = 0.0
        self.G = None
        self.Rstack = [None] * (m.nb + 1)
        self.Lstack = [None] * (m.nb + 1)
        self.sign_stack = 1.0
        self.logw = 0.0
        self.n_prop = 0
        self.n_acc = 0
        self.hook = None
        self.initialise()

    # stacks and fresh G -------------------------------------------------
    def push_R(self, b):
        m, n = self.m, self.p.n_stab
        if b == 0:
            M = m.vdiag(0, self.fields[0])[:, None] * m.P
            pl, ps = 0.0, 1.0
        else:
            prev = self.Rstack[b - 1]
            M = prev.Q.copy()
            for tau in range((b - 1) * n + 1, b * n + 1):
                M = m.expKm @ (m.vdiag(tau, self.fields[tau])[:, None] * M)
            pl, ps = prev.logabs, prev.sign
        Q, r = np.linalg.qr(M)
        d = np.diag(r)
        self.Rstack[b] = StackEntry(Q, pl + float(np.sum(np.log(np.abs(d)))), ps * float(np.prod(np.sign(d))))

    def push_L(self, b):
        m, n = self.m, self.p.n_stab
        if b == m.nb:
            Mt = m.vdiag(m.Ltau + 1, self.fields[m.Ltau + 1])[:, None] * m.P
            pl, ps = 0.0, 1.0
        else:
            prev = self.Lstack[b + 1]
            Mt = prev.Q.copy()
            for tau in range((b + 1) * n, b * n, -1):
                Mt = m.vdiag(tau, self.fields[tau])[:, None] * (m.expKm.T @ Mt)
            pl, ps = prev.logabs, prev.sign
        Q, r = np.linalg.qr(Mt)
        d = np.diag(r)
        self.Lstack[b] = StackEntry(Q, pl + float(np.sum(np.log(np.abs(d)))), ps * float(np.prod(np.sign(d))))

    def refresh(self, b):
        m = self.m
        R, L = self.Rstack[b], self.Lstack[b]
        O = L.Q.T @ R.Q
        s, ld = np.linalg.slogdet(O)
        Gf = np.eye(m.N) - R.Q @ np.linalg.inv(O) @ L.Q.T
        if self.G is not None:
            self.max_dG = max(self.max_dG, float(np.max(np.abs(self.G - Gf))))
        self.G = Gf
        self.logw = R.logabs + ld + L.logabs
        self.sign_stack = R.sign * s * L.sign

    def initialise(self):
        m = self.m
        for b in range(m.nb, -1, -1):
            self.push_L(b)
        self.push_R(0)
        self.G = None
        self.refresh(0)
        self.sign_running = self.sign_stack
        self.unwrap(0)

    # slice propagation --------------------------------------------------
    def wrap(self, tau):
        m = self.m
        d = m.vdiag(tau, self.fields[tau])
        G = d[:, None] * self.G / d[None, :]
        if not m.is_gutz(tau):
            G = m.expKm @ G @ m.expKp
        self.G = G

    def unwrap(self, tau):
        m = self.m
        d = m.vdiag(tau, self.fields[tau])
        G = self.G
        if not m.is_gutz(tau):
            G = m.expKp @ G @ m.expKm
        self.G = G / d[:, None] * d[None, :]

    # Metropolis updates of one slice -----------------------------------
    def update_slice(self, tau):
        m = self.m
        kappa = m.kappa(tau)
        u = philox.uniforms_slice(self.p.seed, self.p.chain, self.sweep_index, tau, m.nbond)
        I2 = np.eye(2)
        for b in m.order:
            i, j = m.bond[b]
            S = [i, j]
            s = float(self.fields[tau, b])
            gam = np.array([np.exp(-2.0 * kappa * s) - 1.0, np.exp(2.0 * kappa * s) - 1.0])
            G = self.G
            GSS = G[np.ix_(S, S)]
            R = float(np.linalg.det(I2 + np.diag(gam) @ (I2 - GSS)))
            accepted = bool(u[b] < abs(R))
            self.accept_log.append((self.sweep_index, tau, b, accepted))
            self.n_prop += 1
            if not accepted:
                continue
            self.n_acc += 1
            ES_minus = -G[:, S].copy()
            ES_minus[i, 0] += 1.0
            ES_minus[j, 1] += 1.0
            Mx = np.diag(gam) @ np.linalg.inv(I2 + (I2 - GSS) @ np.diag(gam))
            self.G = G - ES_minus @ Mx @ G[S, :]
            self.fields[tau, b] = -self.fields[tau, b]
            self.sign_running *= float(np.sign(R))

    # measurement ----------------------------------------------------------
    def measure(self):
        m = self.m
        N, G = m.N, self.G
        ekin = 0.0
        for i in range(N):
            for j in range(N):
                if m.K[i, j] != 0.0:
                    ekin += m.K[i, j] * ((1.0 if i == j else 0.0) - G[j, i])
        dn = 1.0 - np.diag(G) - 0.5                      # n_i - 1/2
        ebond = 0.0
        for i, j in m.bond:
            ebond += dn[i] * dn[j] - G[j, i] * G[i, j]    # i != j on every bond
        ebond *= self.p.V
        stag = float(np.sum(m.eps * dn))
        exch = 0.0
        for i in range(N):
            for j in range(N):
                exch += m.eps[i] * m.eps[j] * ((1.0 if i == j else 0.0) - G[j, i]) * G[i, j]
        s_cdw = (stag * stag + exch) / (N * N)
        self.measurements.append(TVMeasurement(self.sweep_index, self.sign_stack, self.sign_running,
                                               (ekin + ebond) / N, ekin / N, ebond / N, s_cdw))

    def is_stab_point(self, tau):
        return 0 <= tau <= self.m.Ltau and tau % self.p.n_stab == 0

    def sweep(self, measure=True):
        m, n = self.m, self.p.n_stab
        if self.sweep_index % 2 == 0:
            for tau in range(0, m.Ltau + 2):
                self.update_slice(tau)
                self.wrap(tau)
                if self.hook:
                    self.hook(self, "up", tau)
                if self.is_stab_point(tau):
                    b = tau // n
                    self.push_R(b)
                    self.refresh(b)
                    if measure and tau == m.Ltau // 2:
                        self.measure()
        else:
            for tau in range(m.Ltau + 1, -1, -1):
                self.unwrap(tau)
                self.update_slice(tau)
                if self.hook:
                    self.hook(self, "down", tau)
                if self.is_stab_point(tau - 1):
                    b = (tau - 1) // n
                    self.push_L(b)
                    self.refresh(b)
                    if measure and tau - 1 == m.Ltau // 2:
                        self.measure()
        self.sweep_index += 1

    def run(self, n_warm, n_meas):
        for _ in range(n_warm):
            self.sweep(measure=False)
        for _ in range(n_meas):
            self.sweep(measure=True)
        return self

    @property
    def acceptance(self):
        return self.n_acc / max(self.n_prop, 1)


# ----------------------------------------------------------------- exact
class TVCluster:
    """Fock-space reference for the spinless model (one species, n_f fermions)."""

    def __init__(self, model: TVModel):
        self.m = model
        self.Mk, self.states = ed.hopping_sector(model.K, model.n_f)
        N = model.N
        occ = np.array([[(st >> i) & 1 for i in range(N)] for st in self.states], dtype=np.float64)
        dn = occ - 0.5
        bi, bj = model.bond[:, 0], model.bond[:, 1]
        self.Dv = np.sum(dn[:, bi] * dn[:, bj], axis=1)         # sum_b (n_i-1/2)(n_j-1/2)
        self.Dg = np.sum(occ[:, bi] * occ[:, bj], axis=1)       # sum_b n_i n_j
        self.stag = dn @ model.eps                              # sum_i eps_i (n_i - 1/2)

    def trotter_states(self, g, dtau, V, Ltau):
        """Bra and ket at the middle slice; same operator order as the slices."""
        w, v = np.linalg.eigh(self.Mk)
        EK = (v * np.exp(-dtau * w)) @ v.T
        eV = np.exp(-dtau * V * self.Dv)
        psi = np.exp(-g * self.Dg) * ed.slater_vector(self.m.P, self.states)
        R, L = psi.copy(), psi.copy()
        for _ in range(Ltau // 2):
            R = EK @ (eV * R)
            L = eV * (EK @ L)
        return L, R

    def observables(self, L, R, V):
        """(E, E_bond, S_CDW) per site (S_CDW as defined above)."""
        N = self.m.N
        norm = float(L @ R)
        ekin = float(L @ (self.Mk @ R)) / norm
        eb = V * float(L @ (self.Dv * R)) / norm
        s = float(L @ (self.stag ** 2 * R)) / norm / (N * N)
        return (ekin + eb) / N, eb / N, s

    def trotter_observables(self, g, dtau, V, Ltau):
        return self.observables(*self.trotter_states(g, dtau, V, Ltau), V)


def enumerate_observables(p: TVParams):
    """Exact sum over all bond-field configurations of the slices with a
    nonzero coupling (at most ~16 fields); Wick estimates on G(Ltau/2)."""
    m = TVModel(p)
    N, Lt = m.N, m.Ltau
    live = [t for t in range(Lt + 2) if m.kappa(t) != 0.0]
    nf = len(live) * m.nbond
    if nf > 20:
        raise ValueError("too many fields to enumerate")
    idx = np.arange(2 ** nf)[:, None]
    F = np.where(((idx >> np.arange(nf)[None, :]) & 1) == 1, 1, -1).reshape(-1, len(live), m.nbond)
    C = F.shape[0]
    fields = np.ones((C, Lt + 2, m.nbond), dtype=np.int8)
    fields[:, live, :] = F
    def bmat(t):                                   # C x N x N, all configurations at once
        d = np.exp(m.kappa(t) * np.einsum("ib,cb->ci", m.D, fields[:, t, :].astype(np.float64)))
        if m.is_gutz(t):
            return d[:, :, None] * np.eye(N)[None]
        return m.expKm[None] * d[:, None, :]
    BR = np.broadcast_to(m.P, (C,) + m.P.shape).copy()
    for t in range(0, Lt // 2 + 1):
        BR = bmat(t) @ BR
    BL = np.broadcast_to(m.P.T, (C,) + m.P.T.shape).copy()
    for t in range(Lt + 1, Lt // 2, -1):
        BL = BL @ bmat(t)
    O = BL @ BR
    W = np.linalg.det(O)
    G = np.eye(N)[None] - BR @ np.linalg.solve(O, BL)
    GT = np.transpose(G, (0, 2, 1))
    ekin = np.einsum("ij,cij->c", m.K, np.eye(N)[None] - GT)
    dn = 1.0 - np.diagonal(G, axis1=1, axis2=2) - 0.5
    bi, bj = m.bond[:, 0], m.bond[:, 1]
    eb = p.V * np.sum(dn[:, bi] * dn[:, bj] - G[:, bj, bi] * G[:, bi, bj], axis=1)
    stag = dn @ m.eps
    exch = np.einsum("i,j,cij,cij->c", m.eps, m.eps, np.eye(N)[None] - GT, G)
    E = (ekin + eb) / N
    EB = eb / N
    S = (stag * stag + exch) / (N * N)
    tot = np.sum(W)
    return {"E": float(np.sum(W * E) / tot), "ebond": float(np.sum(W * EB) / tot),
            "s_cdw": float(np.sum(W * S) / tot), "sign": float(tot / np.sum(np.abs(W)))}

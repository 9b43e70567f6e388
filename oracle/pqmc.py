"""Projective determinant QMC with a Gutzwiller-projected trial state.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain FP64 numpy,
written to be checked against the paper by eye.

What the paper fixes (Method section; honeycomb Hubbard section):

* expectation values <psi_T| e^{-Theta H} O e^{-Theta H} |psi_T> / <psi_T| e^{-2 Theta H} |psi_T>,
  with the trial state |psi_T> = e^{-g sum_i n_i,up n_i,dn} |psi_N> of Eq. (3) on
  both sides (the printed denominator names a different state; both ends
  carry the Gutzwiller factor here);
* the Hamiltonian of Eq. (2);
* the Gutzwiller factor decoupled with the Ising field of Eq. (1);
* "the standard procedure" of Trotter decomposition, HS transformation and
  determinant QMC for everything else.

The standard procedure as this oracle reads it (the CUDA path follows the
same reading, written independently):

Slices tau = 0 .. Ltau+1, Ltau = 2 Theta / dtau.  tau = 0 and tau = Ltau+1
carry the Gutzwiller fields (coupling lambda, no kinetic factor); tau = 1 .. Ltau
carry the Hubbard fields (coupling alpha):

    B_tau = e^{-dtau K} e^{V_sigma(s_tau)}     (1 <= tau <= Ltau)
    B_tau = e^{V_sigma(s_tau)}                 (tau = 0, Ltau+1)
    V_sigma(s)_ii = sigma kappa s_i.

B_R(tau) = B_tau ... B_0 P_sigma,  B_L(tau) = P_sigma^T B_{Ltau+1} ... B_{tau+1},
G_sigma(tau) = 1 - B_R (B_L B_R)^{-1} B_L,   weight = prod_sigma det(B_L B_R).

A flip of s_{tau,i} is proposed on G(tau-1) (the flip sits just right of
the diagonal factor of B_tau): R_sigma = 1 + Delta_sigma (1 - G_ii),
R = R_up R_dn, accept iff u < |R| (Metropolis with the uniform of
``philox.uniform``), and on acceptance
G <- G - (Delta/R_sigma) (e_i - G[:, i]) G[i, :]   (Sherman-Morrison).

A sweep is one pass over all slices, proposing every field once, sites in
ascending order; sweeps alternate up (tau = 0 -> Ltau+1, sweep index even)
and down.  Going up, slice tau is updated on G(tau-1) and then wrapped,
G(tau) = B_tau G(tau-1) B_tau^{-1}; going down, G(tau) is first unwrapped to
G(tau-1) and then slice tau is updated.

Stabilisation points are tau = b n_stab, b = 0 .. Ltau/n_stab.  At each one
the stack block on the side just updated is rebuilt from the previous block
by QR (B_R(b): right stack while going up; B_L(b): left stack going down), and
G is replaced by 1 - Q_R (Q_L^T Q_R)^{-1} Q_L^T.  The largest change
|G - G_fresh| is recorded.  Measurements are taken on the fresh G at
tau = Ltau/2 once per sweep.
"""
from dataclasses import dataclass, field, replace

import numpy as np

from . import hs, lattice, philox, trial


@dataclass
class Params:
    """One PQMC chain.  Energies are in units of t."""
    kind: int = lattice.HONEYCOMB
    Lx: int = 3
    Ly: int = 3
    t: float = 1.0
    tp: float = 0.0
    U: float = 4.0
    dtau: float = 0.1
    two_theta: float = 10.0
    g: float = 0.0
    M_N: float = 0.0
    n_up: int = -1          # -1: half filling
    n_dn: int = -1
    tiebreak: float = -1.0  # <0: default open-shell tie-break (trial module)
    n_stab: int = 10
    seed: int = 1
    chain: int = 0
    gutzwiller_slices: bool = True
    delay_k: int = 1        # 1: Sherman-Morrison; >1: delayed updates


class Model:
    """Static matrices of one chain: K, e^{-+dtau K}, P_sigma, couplings."""

    def __init__(self, p: Params):
        self.p = p
        self.K, self.eps = lattice.hopping(p.kind, p.Lx, p.Ly, p.t, p.tp)
        self.N = N = self.K.shape[0]
        self.Ltau = int(round(p.two_theta / p.dtau))
        if self.Ltau % 2 or (self.Ltau // 2) % p.n_stab:
            raise ValueError("Ltau/2 must be a multiple of n_stab")
        self.nb = self.Ltau // p.n_stab
        n_up = N // 2 if p.n_up < 0 else p.n_up
        n_dn = N // 2 if p.n_dn < 0 else p.n_dn
        self.n_sigma = {+1: n_up, -1: n_dn}
        # dense exact exponentials of the hopping matrix (library eigh)
        w, v = np.linalg.eigh(self.K)
        self.expKm = (v * np.exp(-p.dtau * w)) @ v.T
        self.expKp = (v * np.exp(+p.dtau * w)) @ v.T
        self.P = {}
        self.gap = {}
        for sigma in (+1, -1):
            self.P[sigma], self.gap[sigma] = trial.trial_orbitals(
                p.kind, self.K, self.eps, p.M_N, self.n_sigma[sigma], sigma, p.tiebreak, p.Lx)
        self.alpha = hs.alpha(p.dtau, p.U)
        self.lam = hs.lam(p.g)

    # slice bookkeeping -------------------------------------------------
    def is_gutz(self, tau):
        return tau == 0 or tau == self.Ltau + 1

    def has_slice(self, tau):
        return self.p.gutzwiller_slices or not self.is_gutz(tau)

    def kappa(self, tau):
        return self.lam if self.is_gutz(tau) else self.alpha

    def vdiag(self, tau, sigma, s_row):
        """Diagonal of e^{V_sigma(s_tau)}."""
        if not self.has_slice(tau):
            return np.ones(self.N)
        return np.exp(sigma * self.kappa(tau) * s_row.astype(np.float64))

    def B(self, tau, sigma, s_row):
        d = self.vdiag(tau, sigma, s_row)
        if self.is_gutz(tau):
            return np.diag(d)
        return self.expKm @ np.diag(d)


def green_definition(model, fields, tau, sigma):
    """G_sigma(tau) = 1 - B_R (B_L B_R)^{-1} B_L straight from its definition.

    The partial products are re-orthonormalised by QR after every slice; that
    keeps their column (row) spaces, and G depends on nothing else.
    """
    R = model.P[sigma].copy()
    for t in range(0, tau + 1):
        R = model.B(t, sigma, fields[t]) @ R
        R, _ = np.linalg.qr(R)
    Lt = model.P[sigma].copy()                       # (B_L)^T, N x N_sigma
    for t in range(model.Ltau + 1, tau, -1):
        Lt = model.B(t, sigma, fields[t]).T @ Lt
        Lt, _ = np.linalg.qr(Lt)
    L = Lt.T
    return np.eye(model.N) - R @ np.linalg.solve(L @ R, L)


def log_weight_definition(model, fields, sigma):
    """log|det(P^T B_{Ltau+1}...B_0 P)| and its sign, by QR after every slice."""
    M = model.P[sigma].copy()
    logabs, sign = 0.0, 1.0
    for t in range(0, model.Ltau + 2):
        M = model.B(t, sigma, fields[t]) @ M
        M, r = np.linalg.qr(M)
        d = np.diag(r)
        logabs += np.sum(np.log(np.abs(d)))
        sign *= np.prod(np.sign(d))
    s, ld = np.linalg.slogdet(model.P[sigma].T @ M)
    return logabs + ld, sign * s


@dataclass
class Measurement:
    sweep: int
    sign: float          # sign of the weight, from the stabilised stacks
    sign_running: float  # running product of sgn(R) since the last reset
    energy: float        # <H> per site for Eq. (2), this configuration
    kinetic: float       # kinetic energy per site
    docc: float          # double occupancy per site
    s_afm: float = 0.0   # staggered S^z structure factor, see Chain.measure


@dataclass
class StackEntry:
    Q: np.ndarray        # N x N_sigma, orthonormal columns
    logabs: float        # log|det T| of the triangular factor carried along
    sign: float


class Chain:
    """State of one Markov chain and the sweep algorithm acting on it."""

    def __init__(self, p: Params, fields=None):
        self.p = p
        self.m = Model(p)
        m = self.m
        if fields is None:
            fields = philox.initial_fields(p.seed, p.chain, m.Ltau + 2, m.N)
        self.fields = np.array(fields, dtype=np.int8).copy()
        self.sweep_index = 0
        self.sign_running = 1.0
        self.accept_log = []          # (sweep, tau, i, accepted) in visiting order
        self.measurements = []
        self.max_dG = 0.0
        self.dG_history = []
        self.G = {+1: None, -1: None}
        self.Rstack = {s: [None] * (m.nb + 1) for s in (+1, -1)}
        self.Lstack = {s: [None] * (m.nb + 1) for s in (+1, -1)}
        self.sign_stack = 1.0
        self.logw = {+1: 0.0, -1: 0.0}
        self.n_prop = 0
        self.n_acc = 0
        # optional observer: hook(chain, event, tau) after every slice step
        # ('up': G is G(tau); 'down': G is G(tau-1)) and every refresh
        self.hook = None
        self.initialise()

    # ------------------------------------------------------------------
    # stacks and fresh Green's functions
    def push_R(self, b):
        m = self.m
        n = self.p.n_stab
        for sigma in (+1, -1):
            if b == 0:
                M = m.vdiag(0, sigma, self.fields[0])[:, None] * m.P[sigma]
                prev_logabs, prev_sign = 0.0, 1.0
            else:
                prev = self.Rstack[sigma][b - 1]
                M = prev.Q.copy()
                for tau in range((b - 1) * n + 1, b * n + 1):
                    M = m.expKm @ (m.vdiag(tau, sigma, self.fields[tau])[:, None] * M)
                prev_logabs, prev_sign = prev.logabs, prev.sign
            Q, r = np.linalg.qr(M)
            d = np.diag(r)
            self.Rstack[sigma][b] = StackEntry(
                Q, prev_logabs + float(np.sum(np.log(np.abs(d)))),
                prev_sign * float(np.prod(np.sign(d))))

    def push_L(self, b):
        """Left block b holds (B_L(b n_stab))^T = Q T^T with Q orthonormal."""
        m = self.m
        n = self.p.n_stab
        for sigma in (+1, -1):
            if b == m.nb:
                Mt = m.vdiag(m.Ltau + 1, sigma, self.fields[m.Ltau + 1])[:, None] * m.P[sigma]
                prev_logabs, prev_sign = 0.0, 1.0
            else:
                prev = self.Lstack[sigma][b + 1]
                Mt = prev.Q.copy()
                # (Q^T B_{(b+1)n} ... B_{bn+1})^T = B_{bn+1}^T ... B_{(b+1)n}^T Q
                for tau in range((b + 1) * n, b * n, -1):
                    Mt = m.vdiag(tau, sigma, self.fields[tau])[:, None] * (m.expKm.T @ Mt)
                prev_logabs, prev_sign = prev.logabs, prev.sign
            Q, r = np.linalg.qr(Mt)
            d = np.diag(r)
            self.Lstack[sigma][b] = StackEntry(
                Q, prev_logabs + float(np.sum(np.log(np.abs(d)))),
                prev_sign * float(np.prod(np.sign(d))))

    def refresh(self, b):
        """Replace G by 1 - Q_R (Q_L^T Q_R)^{-1} Q_L^T at stabilisation point b."""
        m = self.m
        sign_total = 1.0
        for sigma in (+1, -1):
            R = self.Rstack[sigma][b]
            L = self.Lstack[sigma][b]
            O = L.Q.T @ R.Q
            s, ld = np.linalg.slogdet(O)
            Gf = np.eye(m.N) - R.Q @ np.linalg.inv(O) @ L.Q.T
            if self.G[sigma] is not None:
                dG = float(np.max(np.abs(self.G[sigma] - Gf)))
                self.max_dG = max(self.max_dG, dG)
                self.dG_history.append(dG)
            self.G[sigma] = Gf
            self.logw[sigma] = R.logabs + ld + L.logabs
            sign_total *= R.sign * s * L.sign
        self.sign_stack = sign_total

    def initialise(self):
        m = self.m
        for b in range(m.nb, -1, -1):
            self.push_L(b)
        self.push_R(0)
        self.G = {+1: None, -1: None}
        self.refresh(0)
        self.sign_running = self.sign_stack
        if m.has_slice(0):
            self.unwrap(0)                 # G(0) -> G(-1)

    # ------------------------------------------------------------------
    # slice propagation
    def wrap(self, tau):
        """G(tau) = B_tau G(tau-1) B_tau^{-1}."""
        m = self.m
        for sigma in (+1, -1):
            d = m.vdiag(tau, sigma, self.fields[tau])
            G = d[:, None] * self.G[sigma] / d[None, :]
            if not m.is_gutz(tau):
                G = m.expKm @ G @ m.expKp
            self.G[sigma] = G

    def unwrap(self, tau):
        """G(tau-1) = B_tau^{-1} G(tau) B_tau."""
        m = self.m
        for sigma in (+1, -1):
            d = m.vdiag(tau, sigma, self.fields[tau])
            G = self.G[sigma]
            if not m.is_gutz(tau):
                G = m.expKp @ G @ m.expKm
            self.G[sigma] = G / d[:, None] * d[None, :]

    # ------------------------------------------------------------------
    # Metropolis updates of one slice
    def update_slice(self, tau):
        if self.p.delay_k > 1:
            return self.update_slice_delayed(tau)
        m = self.m
        kappa = m.kappa(tau)
        u = philox.uniforms_slice(self.p.seed, self.p.chain, self.sweep_index, tau, m.N)
        for i in range(m.N):
            s = self.fields[tau, i]
            delta = {sg: float(hs.delta(kappa, sg, s)) for sg in (+1, -1)}
            ratio = {sg: 1.0 + delta[sg] * (1.0 - self.G[sg][i, i]) for sg in (+1, -1)}
            R = ratio[+1] * ratio[-1]
            accepted = bool(u[i] < abs(R))
            self.accept_log.append((self.sweep_index, tau, i, accepted))
            self.n_prop += 1
            if accepted:
                self.n_acc += 1
                for sg in (+1, -1):
                    G = self.G[sg]
                    e_i = np.zeros(m.N)
                    e_i[i] = 1.0
                    self.G[sg] = G - (delta[sg] / ratio[sg]) * np.outer(e_i - G[:, i], G[i, :])
                self.fields[tau, i] = -s
                self.sign_running *= float(np.sign(R))

    def update_slice_delayed(self, tau):
        """Same proposals with delayed rank-k updates.

        G = G0 - sum_m u_m v_m^T with u_m = (Delta/R)(e_i - G[:, i]) and
        v_m = G[i, :] built from the current G; G0 absorbs the pending
        vectors every k accepted flips and at the end of the slice.
        """
        m = self.m
        k = self.p.delay_k
        kappa = m.kappa(tau)
        u = philox.uniforms_slice(self.p.seed, self.p.chain, self.sweep_index, tau, m.N)
        U = {+1: [], -1: []}
        V = {+1: [], -1: []}

        def current(sg, i):
            col = self.G[sg][:, i].copy()
            row = self.G[sg][i, :].copy()
            for uu, vv in zip(U[sg], V[sg]):
                col -= uu * vv[i]
                row -= uu[i] * vv
            return col, row

        def flush():
            for sg in (+1, -1):
                for uu, vv in zip(U[sg], V[sg]):
                    self.G[sg] = self.G[sg] - np.outer(uu, vv)
                U[sg].clear()
                V[sg].clear()

        for i in range(m.N):
            s = self.fields[tau, i]
            delta = {sg: float(hs.delta(kappa, sg, s)) for sg in (+1, -1)}
            gii = {}
            for sg in (+1, -1):
                gii[sg] = self.G[sg][i, i] - sum(uu[i] * vv[i] for uu, vv in zip(U[sg], V[sg]))
            ratio = {sg: 1.0 + delta[sg] * (1.0 - gii[sg]) for sg in (+1, -1)}
            R = ratio[+1] * ratio[-1]
            accepted = bool(u[i] < abs(R))
            self.accept_log.append((self.sweep_index, tau, i, accepted))
            self.n_prop += 1
            if accepted:
                self.n_acc += 1
                for sg in (+1, -1):
                    col, row = current(sg, i)
                    e_i = np.zeros(m.N)
                    e_i[i] = 1.0
                    U[sg].append((delta[sg] / ratio[sg]) * (e_i - col))
                    V[sg].append(row)
                self.fields[tau, i] = -s
                self.sign_running *= float(np.sign(R))
                if len(U[+1]) == k:
                    flush()
        flush()

    # ------------------------------------------------------------------
    def measure(self):
        """Equal-time Wick estimates on the fresh G at tau = Ltau/2."""
        m = self.m
        N = m.N
        K = m.K
        ekin = 0.0
        for sg in (+1, -1):
            G = self.G[sg]
            for i in range(N):
                for j in range(N):
                    if K[i, j] != 0.0:
                        ekin += K[i, j] * ((1.0 if i == j else 0.0) - G[j, i])
        docc = 0.0
        for i in range(N):
            docc += (1.0 - self.G[+1][i, i]) * (1.0 - self.G[-1][i, i])
        energy = ekin + self.p.U * docc
        # AFM structure factor (z component, the reading taken for the
        # undefined supplement): S = (1/N^2) sum_ij eps_i eps_j <S^z_i S^z_j>,
        # S^z_i = (n_i,up - n_i,dn)/2.  The spins are independent at fixed
        # fields, so Wick's theorem per spin gives
        #   <n_i,s n_j,s'> = n_i,s n_j,s' + [s = s'] <c^+_i c_j>_s <c_i c^+_j>_s,
        # with <c_i c^+_j> = G_ij and <c^+_i c_j> = delta_ij - G_ji.
        stag = 0.0
        for i in range(N):
            stag += m.eps[i] * (self.G[-1][i, i] - self.G[+1][i, i])   # eps_i (n_up - n_dn)
        exch = 0.0
        for sg in (+1, -1):
            G = self.G[sg]
            for i in range(N):
                for j in range(N):
                    exch += m.eps[i] * m.eps[j] * ((1.0 if i == j else 0.0) - G[j, i]) * G[i, j]
        s_afm = (stag * stag + exch) / (4.0 * N * N)
        self.measurements.append(Measurement(
            self.sweep_index, self.sign_stack, self.sign_running,
            energy / N, ekin / N, docc / N, s_afm))

    def is_stab_point(self, tau):
        return 0 <= tau <= self.m.Ltau and tau % self.p.n_stab == 0

    def sweep(self, measure=True):
        """One directional pass; even sweep index goes up, odd goes down."""
        m = self.m
        n = self.p.n_stab
        if self.sweep_index % 2 == 0:
            for tau in range(0, m.Ltau + 2):
                if m.has_slice(tau):
                    self.update_slice(tau)
                    self.wrap(tau)
                    if self.hook:
                        self.hook(self, "up", tau)
                if self.is_stab_point(tau):
                    b = tau // n
                    self.push_R(b)
                    self.refresh(b)
                    if self.hook:
                        self.hook(self, "refresh", tau)
                    if measure and tau == m.Ltau // 2:
                        self.measure()
        else:
            for tau in range(m.Ltau + 1, -1, -1):
                if m.has_slice(tau):
                    self.unwrap(tau)
                    self.update_slice(tau)
                    if self.hook:
                        self.hook(self, "down", tau)
                if self.is_stab_point(tau - 1):
                    b = (tau - 1) // n
                    self.push_L(b)
                    self.refresh(b)
                    if self.hook:
                        self.hook(self, "refresh", tau - 1)
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


def estimate(values, signs, n_bins=None):
    """Sign-reweighted mean sum(s O)/sum(s) with a binned jackknife error."""
    values = np.asarray(values, dtype=np.float64)
    signs = np.asarray(signs, dtype=np.float64)
    n = len(values)
    if n == 0:
        return float("nan"), float("nan")
    if n_bins is None:
        n_bins = min(n, 20)
    n_bins = max(1, min(n_bins, n))
    per = n // n_bins
    sv = (signs * values)[: per * n_bins].reshape(n_bins, per).sum(axis=1)
    ss = signs[: per * n_bins].reshape(n_bins, per).sum(axis=1)
    mean = float(np.sum(signs * values) / np.sum(signs))
    if n_bins < 2:
        return mean, float("nan")
    tot_v, tot_s = sv.sum(), ss.sum()
    jk = (tot_v - sv) / (tot_s - ss)
    err = float(np.sqrt((n_bins - 1) / n_bins * np.sum((jk - jk.mean()) ** 2)))
    return mean, err


def run_chain(p: Params, n_warm, n_meas):
    return Chain(p).run(n_warm, n_meas)

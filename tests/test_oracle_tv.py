"""Pins of the spinless t-V oracle (repulsive spinless honeycomb section,
Eqs. (4)-(5)): the bond HS identity and the bond Gutzwiller factor, exact
field sums against Fock space, the free-fermion closed form, the sweep's G
against its definition, the rank-2 ratio against the determinant ratio, the
classical CDW limit, and Monte Carlo against the exact projection."""
import itertools

import numpy as np
import pytest

from oracle import ed, hs, pqmc, tv


@pytest.mark.parametrize("a", [0.16, 0.6, 1.3])
def test_bond_hs_identity(a):
    """exp(-a (n_i-1/2)(n_j-1/2)) = 1/2 exp(-a/4) sum_s exp(kappa s (n_i - n_j)),
    cosh kappa = exp(a/2), for all four occupations of the bond."""
    k = hs.coupling(a)
    for ni, nj in itertools.product((0, 1), repeat=2):
        lhs = np.exp(-a * (ni - 0.5) * (nj - 0.5))
        rhs = 0.5 * np.exp(-a / 4) * sum(np.exp(k * s * (ni - nj)) for s in (1, -1))
        assert abs(lhs - rhs) < 1e-14


def test_bond_gutzwiller_factor_is_product_of_hs_factors():
    """At fixed particle number exp(-g sum_b n_i n_j) / prod_b exp(-g (n_i-1/2)(n_j-1/2))
    is the same for every Fock state (every site lies on three bonds)."""
    m = tv.TVModel(tv.TVParams(Lx=3, Ly=1, n_stab=1, two_theta=0.0))
    g = 0.7
    for nf in (2, 3, 4):
        states, _ = ed.basis(m.N, nf)
        ratios = []
        for st in states:
            occ = np.array([(st >> i) & 1 for i in range(m.N)], dtype=float)
            gz = np.exp(-g * sum(occ[i] * occ[j] for i, j in m.bond))
            hsf = np.prod([np.exp(-g * (occ[i] - 0.5) * (occ[j] - 0.5)) for i, j in m.bond])
            ratios.append(gz / hsf)
        assert np.ptp(ratios) < 1e-12 * max(ratios)


def test_bonds_are_three_perfect_matchings():
    m = tv.TVModel(tv.TVParams(Lx=3, Ly=2, n_stab=1, two_theta=0.0))
    for k in range(3):
        cls = m.bond[k::3]
        assert sorted(cls[:, 0]) == list(range(0, m.N, 2))
        assert sorted(cls[:, 1]) == list(range(1, m.N, 2))
    assert np.array_equal(np.sort(m.bond, axis=None), np.sort(np.repeat(np.arange(m.N), 3)))
    K = np.zeros((m.N, m.N))
    for i, j in m.bond:
        K[i, j] -= 1.0
        K[j, i] -= 1.0
    assert np.array_equal(K, m.K)


@pytest.mark.parametrize("kw", [
    dict(Lx=2, Ly=1, two_theta=0.0, g=0.5, Delta_C=0.1, V=1.6),        # Theta = 0: variational
    dict(Lx=3, Ly=1, two_theta=0.2, g=0.0, Delta_C=0.0, V=4.0),        # two interaction slices
    dict(Lx=3, Ly=1, two_theta=0.4, g=0.0, Delta_C=0.0, V=8.0, dtau=0.2),
    dict(Lx=3, Ly=1, two_theta=0.0, g=1.0, Delta_C=0.2, V=1.6),
])
def test_enumeration_equals_fock_space(kw):
    """Exact sum over the bond fields (determinants, Wick) == Fock-space
    Trotterised projection with exp(-g sum_b n_i n_j) on both ends."""
    p = tv.TVParams(n_stab=1, **kw)
    m = tv.TVModel(p)
    r = tv.enumerate_observables(p)
    E, EB, S = tv.TVCluster(m).trotter_observables(p.g, p.dtau, p.V, m.Ltau)
    assert abs(r["E"] - E) < 1e-12 and abs(r["ebond"] - EB) < 1e-12 and abs(r["s_cdw"] - S) < 1e-12


def test_free_fermions_closed_form():
    """V = 0, g = 0: every configuration has G = 1 - Pi with Pi the projector on
    the lowest N/2 orbitals of K; E/site is their energy sum / N."""
    p = tv.TVParams(Lx=2, Ly=2, V=0.0, g=0.0, Delta_C=0.0, tiebreak=0.0, two_theta=1.0, n_stab=5, seed=3)
    ch = tv.TVChain(p).run(0, 2)
    w, v = np.linalg.eigh(ch.m.K)
    nf = ch.m.n_f
    assert w[nf] - w[nf - 1] > 0.5
    Pi = v[:, :nf] @ v[:, :nf].T
    assert np.abs(ch.G - (np.eye(ch.m.N) - Pi)).max() < 1e-10
    for x in ch.measurements:
        assert abs(x.energy - np.sum(w[:nf]) / ch.m.N) < 1e-10
        assert abs(x.ebond) < 1e-15


def test_sweep_green_matches_definition_and_trace():
    """G after every slice step of two sweeps (up and down) equals its
    definition on the current fields; Tr(1 - G) = N_f."""
    p = tv.TVParams(Lx=2, Ly=2, V=1.6, g=0.5, Delta_C=0.1, two_theta=1.0, n_stab=5, seed=4)
    ch = tv.TVChain(p)
    worst = [0.0]

    def hook(c, ev, tau):
        t = tau if ev == "up" else tau - 1
        if t < 0:
            return
        G = tv.green_definition(c.m, c.fields, t)
        worst[0] = max(worst[0], np.abs(c.G - G).max())
        assert abs(np.trace(np.eye(c.m.N) - c.G) - c.m.n_f) < 1e-9
    ch.hook = hook
    ch.run(0, 2)
    assert worst[0] < 1e-9
    assert 0.2 < ch.acceptance < 1.0


def test_rank2_ratio_is_determinant_ratio():
    """R = det(1 + Gamma (1 - G)_SS) equals the ratio of the weights before and
    after flipping one bond field, for bonds of every class and slice kind."""
    p = tv.TVParams(Lx=2, Ly=2, V=2.0, g=0.6, Delta_C=0.1, two_theta=0.4, n_stab=1)
    m = tv.TVModel(p)
    rng = np.random.default_rng(5)
    f = rng.choice(np.array([-1, 1], dtype=np.int8), size=(m.Ltau + 2, m.nbond))
    for tau in (0, 2, m.Ltau + 1):
        for b in (0, 1, 2, 7):
            G = tv.green_definition(m, f, tau - 1) if tau > 0 else None
            if G is None:                           # G(-1): nothing applied on the right
                R0 = m.P.copy()
                Lt = m.P.copy()
                for t in range(m.Ltau + 1, -1, -1):
                    Lt = m.B(t, f[t]).T @ Lt
                G = np.eye(m.N) - R0 @ np.linalg.solve(Lt.T @ R0, Lt.T)
            i, j = m.bond[b]
            k, s = m.kappa(tau), float(f[tau, b])
            gam = np.diag([np.exp(-2 * k * s) - 1, np.exp(2 * k * s) - 1])
            R = np.linalg.det(np.eye(2) + gam @ (np.eye(2) - G[np.ix_([i, j], [i, j])]))
            l0, s0 = tv.log_weight_definition(m, f)
            f2 = f.copy()
            f2[tau, b] = -f2[tau, b]
            l1, s1 = tv.log_weight_definition(m, f2)
            assert abs(R - s0 * s1 * np.exp(l1 - l0)) < 1e-10 * max(1.0, abs(R))


def test_classical_cdw_limit():
    """Delta_C >> t, V = 0, g = 0, Theta = 0: the trial fills the B sublattice,
    sum_i eps_i (n_i - 1/2) = -N/2 and S_CDW = 1/4."""
    ch = tv.TVChain(tv.TVParams(Lx=2, Ly=2, V=0.0, g=0.0, Delta_C=1e5, two_theta=0.0, n_stab=1)).run(0, 2)
    for x in ch.measurements:
        assert abs(x.s_cdw - 0.25) < 1e-8


def test_mc_within_3sigma_of_exact():
    """Four chains; bins of 150 sweeps (the autocorrelation of E on this
    cluster spans tens of sweeps)."""
    ms = []
    for seed in (6, 7, 8, 9):
        p = tv.TVParams(Lx=2, Ly=2, V=1.6, g=0.4, Delta_C=0.1, two_theta=1.0, n_stab=5, seed=seed)
        ch = tv.TVChain(p).run(10, 300)
        ms += ch.measurements
        assert np.array_equal([x.sign for x in ch.measurements], [x.sign_running for x in ch.measurements])
    s = [x.sign for x in ms]
    E, dE = pqmc.estimate([x.energy for x in ms], s, n_bins=8)
    S, dS = pqmc.estimate([x.s_cdw for x in ms], s, n_bins=8)
    Ex, _, Sx = tv.TVCluster(ch.m).trotter_observables(p.g, p.dtau, p.V, ch.m.Ltau)
    assert abs(E - Ex) < 3 * dE and dE < 0.02
    assert abs(S - Sx) < 3 * dS


def test_measurement_of_one_configuration_equals_fock_space():
    """For one field configuration (G not symmetric) the sweep's Wick
    estimates equal <L|O|R>/<L|R> with |R>, <L| the Slater determinants of
    B_R and B_L^T built in Fock space."""
    p = tv.TVParams(Lx=2, Ly=2, V=1.6, g=0.5, Delta_C=0.1, two_theta=0.4, n_stab=1)
    m = tv.TVModel(p)
    rng = np.random.default_rng(8)
    f = rng.choice(np.array([-1, 1], dtype=np.int8), size=(m.Ltau + 2, m.nbond))
    ch = tv.TVChain(p, fields=f.copy())
    t = m.Ltau // 2
    ch.G = tv.green_definition(m, f, t)
    assert np.abs(ch.G - ch.G.T).max() > 1e-3
    ch.measure()
    x = ch.measurements[-1]
    R = m.P.copy()
    for tt in range(0, t + 1):
        R = m.B(tt, f[tt]) @ R
    Lt = m.P.copy()
    for tt in range(m.Ltau + 1, t, -1):
        Lt = m.B(tt, f[tt]).T @ Lt
    c = tv.TVCluster(m)
    E, EB, S = c.observables(ed.slater_vector(Lt, c.states), ed.slater_vector(R, c.states), p.V)
    assert abs(x.energy - E) < 1e-12 and abs(x.ebond - EB) < 1e-12 and abs(x.s_cdw - S) < 1e-12

"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties an oracle function to an independent fact: published Philox
vectors, Bloch spectra, the exact HS identity, Fock-space ED, exact field
enumeration, closed forms at U = 0, invariants of G, and the g = 0 reduction.
"""
import os

import numpy as np
import pytest

from oracle import ed, hs, hs_enum, lattice, philox, pqmc, trial

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Salmon et al. (SC'11) published vectors for Philox4x32-10."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert philox.philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10])
        c0, c1, c2, c3 = philox.philox4x32_10_vec([w[0]], [w[1]], [w[2]], [w[3]], w[4], w[5])
        assert [int(c0[0]), int(c1[0]), int(c2[0]), int(c3[0])] == w[6:10]
        n += 1
    assert n == 3


def test_philox_uniform_and_fields():
    u = philox.uniforms_slice(1, 3, 5, 7, 64)
    for i in (0, 17, 63):
        assert u[i] == philox.uniform(1, 3, 5, 7, i)
    assert np.all((u >= 0) & (u < 1))
    f = philox.initial_fields(1, 0, 12, 18)
    assert f.dtype == np.int8 and set(np.unique(f)) <= {-1, 1}
    x2 = philox.philox4x32_10((5, 3, philox.INIT_SWEEP, 0), philox.seed_key(1))[2]
    assert f[3, 5] == (1 if x2 & 1 else -1)
    # a large sample is uniform to a few sigma
    big = philox.uniforms_slice(99, 0, 0, 0, 200000)
    assert abs(big.mean() - 0.5) < 5 * np.sqrt(1 / 12 / 200000)


# ------------------------------------------------------------------- lattices
def bloch_honeycomb(Lx, Ly, t=1.0):
    e = []
    for n1 in range(Lx):
        for n2 in range(Ly):
            z = abs(1 + np.exp(2j * np.pi * n1 / Lx) + np.exp(2j * np.pi * n2 / Ly))
            e += [-t * z, t * z]
    return np.sort(e)


@pytest.mark.parametrize("L", [2, 3, 6])
def test_honeycomb_spectrum_is_bloch(L):
    K, eps = lattice.honeycomb(L, L)
    assert np.allclose(K, K.T)
    assert np.allclose(np.sort(np.linalg.eigvalsh(K)), bloch_honeycomb(L, L), atol=1e-12)
    # bipartite: hopping only between A and B
    A = eps > 0
    assert not np.any(K[np.ix_(A, A)]) and not np.any(K[np.ix_(~A, ~A)])
    assert np.all(np.count_nonzero(K, axis=1) == 3)


def test_square_tprime_spectrum():
    Lx = Ly = 8
    tp = -0.2
    K, eps = lattice.square(Lx, Ly, 1.0, tp)
    kx = 2 * np.pi * np.arange(Lx) / Lx
    ky = 2 * np.pi * np.arange(Ly) / Ly
    e = [-2 * (np.cos(a) + np.cos(b)) - 4 * tp * np.cos(a) * np.cos(b) for a in kx for b in ky]
    assert np.allclose(np.sort(np.linalg.eigvalsh(K)), np.sort(e), atol=1e-12)


# ------------------------------------------------------------------ HS (Eq. 1)
@pytest.mark.parametrize("g", [0.0, 0.3, 0.6, 1.0, 0.4])
def test_spin_channel_hs_identity(g):
    lam = hs.coupling(g)
    assert np.isclose(np.cosh(lam), np.exp(g / 2), rtol=1e-15)
    for nu in (0, 1):
        for nd in (0, 1):
            lhs = np.exp(-g * (nu - 0.5) * (nd - 0.5))
            rhs = 0.5 * np.exp(-g / 4) * sum(np.exp(lam * s * (nu - nd)) for s in (1, -1))
            assert np.isclose(lhs, rhs, rtol=1e-14)


def test_delta_table():
    k = hs.alpha(0.1, 4.0)
    for sigma in (1, -1):
        for s in (1, -1):
            # flipping s multiplies e^{sigma k s} by 1 + Delta
            assert np.isclose(np.exp(sigma * k * s) * (1 + hs.delta(k, sigma, s)),
                              np.exp(-sigma * k * s), rtol=1e-15)


# ---------------------------------------------------------------------- trial
@pytest.mark.parametrize("L,M", [(3, 0.0), (6, 0.21), (6, 0.0), (9, 0.0), (12, 0.3)])
def test_trial_is_closed_shell(L, M):
    K, eps = lattice.honeycomb(L, L)
    N = K.shape[0]
    for sigma in (1, -1):
        P, gap = trial.trial_orbitals(lattice.HONEYCOMB, K, eps, M, N // 2, sigma)
        assert gap > 1e-6
        assert np.allclose(P.T @ P, np.eye(N // 2), atol=1e-12)
        h = trial.trial_hamiltonian(lattice.HONEYCOMB, K, eps, M, sigma)
        # span of P is invariant under h
        HP = h @ P
        assert np.allclose(HP, P @ (P.T @ HP), atol=1e-10)


@pytest.mark.parametrize("L,M", [(3, 0.21), (6, 0.21), (6, 0.0)])
def test_neel_trial_is_antiferromagnetic(L, M):
    """H_N = H_0 + M_N sum_i eps_i (n_up - n_dn): at half filling on the
    bipartite lattice every site holds one electron, and the staggered moment
    points against the field (up spins avoid the sites where eps_i M_N > 0)."""
    K, eps = lattice.honeycomb(L, L)
    N = K.shape[0]
    n = {}
    for sigma in (1, -1):
        P, _ = trial.trial_orbitals(lattice.HONEYCOMB, K, eps, M, N // 2, sigma)
        n[sigma] = np.sum(P * P, axis=1)          # <n_i,sigma> = (P P^T)_ii
    assert np.allclose(n[1] + n[-1], 1.0, atol=1e-10)
    m_stag = np.sum(eps * (n[1] - n[-1])) / N
    assert m_stag < -1e-4 if M > 0 else m_stag < 0
    # the two spins are images of each other under the sublattice swap
    assert np.allclose(np.sort(n[1][eps > 0]), np.sort(n[-1][eps < 0]), atol=1e-10)


def test_doped_square_trial_closed_shell():
    """28 particles on the 8x8 t' = -0.2 lattice fill 27 states below an 8-fold
    shell at e = -0.4 (Bloch spectrum); the tie-break must open a real gap."""
    K, eps = lattice.square(8, 8, 1.0, -0.2)
    e = np.sort(np.linalg.eigvalsh(K))
    assert np.allclose(e[27:35], -0.4, atol=1e-12) and e[26] < -0.4 - 0.1 and e[35] > -0.4 + 0.1
    for M, least in ((0.0, 1e-2), (0.1, 1e-3)):
        P, gap = trial.trial_orbitals(lattice.SQUARE, K, eps, M, 28, 1, lx=8)
        assert gap > least
    # without the tie-break the shell is open
    _, gap0 = trial.trial_orbitals(lattice.SQUARE, K, eps, 0.0, 28, 1, tiebreak=0.0, lx=8)
    assert gap0 < 1e-10


# ------------------------------------------------------------------------- ED
def test_ed_free_fermions_and_atomic_limit():
    K, _ = lattice.honeycomb(2, 2)
    e = np.sort(np.linalg.eigvalsh(K))
    c = ed.Cluster(K, 4, 4, 0.0)
    e0, _ = c.ground_state()
    assert np.isclose(e0, 2 * e[:4].sum(), atol=1e-10)
    # a Slater determinant of eigenvectors is an eigenvector of the hopping sector
    w, v = np.linalg.eigh(K)
    amp = ed.slater_vector(v[:, :4], c.sup)
    assert np.allclose(c.Mup @ amp, e[:4].sum() * amp, atol=1e-10)
    # t = 0: the ground state avoids double occupancy when possible
    c0 = ed.Cluster(np.zeros((4, 4)), 2, 2, 3.0)
    assert np.isclose(c0.ground_state()[0], 0.0, atol=1e-12)
    c1 = ed.Cluster(np.zeros((4, 4)), 3, 3, 3.0)
    assert np.isclose(c1.ground_state()[0], 6.0, atol=1e-12)


def small_params(**kw):
    base = dict(kind=lattice.HONEYCOMB, Lx=2, Ly=1, U=4.0, dtau=0.1, two_theta=0.2,
                g=0.6, M_N=0.21, n_stab=1)
    base.update(kw)
    return pqmc.Params(**base)


def test_enumeration_equals_trotterised_ed_honeycomb():
    """Exact HS sum (determinants) == Fock-space Trotterised projection."""
    p = small_params()
    m = pqmc.Model(p)
    E, D, sign = hs_enum.enumerate_estimator(p)
    c = ed.Cluster(m.K, m.n_sigma[1], m.n_sigma[-1], p.U)
    Ex, Dx = c.trotter_projection(m.P[1], m.P[-1], p.g, p.dtau, m.Ltau)
    assert abs(E - Ex) < 1e-11 and abs(D - Dx) < 1e-11
    assert sign == 1.0


def test_enumeration_equals_ed_doped_square_vmc():
    """Theta = 0 (Gutzwiller slices only) on a doped 2x4 t-t' cluster: the
    variational energy of Eq. (3).  With no kinetic factor every weight is
    det(P^T D P) > 0 (D a positive diagonal), so the sign is exactly one."""
    p = pqmc.Params(kind=lattice.SQUARE, Lx=2, Ly=4, tp=-0.2, U=4.0, dtau=0.1,
                    two_theta=0.0, g=0.5, M_N=0.1, n_up=3, n_dn=3, n_stab=1)
    m = pqmc.Model(p)
    E, D, sign = hs_enum.enumerate_estimator(p)
    c = ed.Cluster(m.K, 3, 3, p.U)
    Ex, Dx = c.trotter_projection(m.P[1], m.P[-1], p.g, p.dtau, 0)
    assert abs(E - Ex) < 1e-11 and abs(D - Dx) < 1e-11
    assert sign == 1.0


def test_enumeration_with_negative_weights_equals_ed():
    """A doped 4-site cluster (1 up, 2 down, U = 8) where some field
    configurations have negative weight: the sign-weighted estimator still
    equals the Fock-space value and the average sign is below one."""
    p = small_params(U=8.0, dtau=0.2, two_theta=0.4, g=0.5, M_N=0.1, n_up=1, n_dn=2)
    m = pqmc.Model(p)
    E, D, sign = hs_enum.enumerate_estimator(p)
    c = ed.Cluster(m.K, 1, 2, p.U)
    Ex, Dx = c.trotter_projection(m.P[1], m.P[-1], p.g, p.dtau, m.Ltau)
    assert abs(E - Ex) < 1e-11 and abs(D - Dx) < 1e-11
    assert sign < 1.0 - 1e-7


# ------------------------------------------------------------- PQMC machinery
def expm_sym(K, x):
    w, v = np.linalg.eigh(K)
    return (v * np.exp(x * w)) @ v.T


def test_u0_closed_form_every_slice():
    """U = 0, g = 0: G(tau) = 1 - e^{-tau dtau K} P (P^T e^{-Ltau dtau K} P)^{-1}
    P^T e^{-(Ltau - tau) dtau K} at every slice, both directions, with a trial
    that is not an eigenbasis of K (M_N != 0)."""
    p = pqmc.Params(Lx=2, Ly=2, U=0.0, g=0.0, M_N=0.3, dtau=0.1, two_theta=2.0, n_stab=5)
    ch = pqmc.Chain(p)
    m = ch.m
    errs = []

    def closed(taug, sigma):
        P = m.P[sigma]
        taug = max(taug, 0)                    # slice 0 is the identity at g = 0
        tr = min(taug, m.Ltau)
        Rm = expm_sym(m.K, -tr * p.dtau) @ P
        Lm = P.T @ expm_sym(m.K, -(m.Ltau - tr) * p.dtau)
        return np.eye(m.N) - Rm @ np.linalg.solve(Lm @ Rm, Lm)

    def hook(chain, event, tau):
        taug = tau if event in ("up", "refresh") else tau - 1
        for sigma in (1, -1):
            errs.append(np.abs(chain.G[sigma] - closed(taug, sigma)).max())

    ch.hook = hook
    ch.run(0, 2)
    assert len(errs) > 50 and max(errs) < 1e-11
    # the energy is the closed-form kinetic energy
    G = {s: closed(m.Ltau // 2, s) for s in (1, -1)}
    e = sum(np.trace(m.K @ (np.eye(m.N) - G[s])) for s in (1, -1)) / m.N
    assert all(abs(x.energy - e) < 1e-11 for x in ch.measurements)


def test_sweep_green_matches_definition_every_slice():
    """The incremental G (updates + wraps + refreshes) equals the definition
    1 - B_R (B_L B_R)^{-1} B_L on the current fields after every slice."""
    p = pqmc.Params(Lx=2, Ly=2, U=4.0, g=0.6, M_N=0.21, dtau=0.1, two_theta=2.0, n_stab=5)
    ch = pqmc.Chain(p)
    errs = []

    def hook(chain, event, tau):
        taug = tau if event in ("up", "refresh") else tau - 1
        for sigma in (1, -1):
            Gd = pqmc.green_definition(chain.m, chain.fields, taug, sigma)
            errs.append(np.abs(chain.G[sigma] - Gd).max())

    ch.hook = hook
    ch.run(0, 2)
    assert ch.n_acc > 20
    assert len(errs) > 50 and max(errs) < 1e-10


def test_ratio_is_determinant_ratio():
    """R_sigma = det(B_L' B_R)/det(B_L B_R) for a single flip."""
    p = pqmc.Params(Lx=2, Ly=2, U=4.0, g=0.6, M_N=0.21, dtau=0.1, two_theta=2.0, n_stab=5)
    m = pqmc.Model(p)
    f = philox.initial_fields(3, 0, m.Ltau + 2, m.N)
    for tau, i in ((0, 3), (7, 5), (m.Ltau + 1, 0)):
        G = {s: pqmc.green_definition(m, f, tau - 1, s) for s in (1, -1)}
        f2 = f.copy()
        f2[tau, i] *= -1
        for s in (1, -1):
            d = float(hs.delta(m.kappa(tau), s, f[tau, i]))
            R = 1 + d * (1 - G[s][i, i])
            l1, s1 = pqmc.log_weight_definition(m, f, s)
            l2, s2 = pqmc.log_weight_definition(m, f2, s)
            assert np.isclose(R, s1 * s2 * np.exp(l2 - l1), rtol=1e-10)


def test_invariants_and_sign_half_filling():
    p = pqmc.Params(Lx=3, Ly=3, U=4.0, g=0.6, M_N=0.21, dtau=0.1, two_theta=2.0, n_stab=5, seed=4)
    ch = pqmc.Chain(p)
    checks = []

    def hook(chain, event, tau):
        if event == "refresh":
            for s in (1, -1):
                A = np.eye(chain.m.N) - chain.G[s]
                # log|W| from the QR chain equals a from-scratch evaluation
                lw, _ = pqmc.log_weight_definition(chain.m, chain.fields, s)
                checks.append((abs(np.trace(A) - chain.m.n_sigma[s]),
                               np.abs(A @ A - A).max(), abs(chain.logw[s] - lw)))

    ch.hook = hook
    ch.run(2, 4)
    assert len(checks) > 10
    assert max(c[0] for c in checks) < 1e-10 and max(c[1] for c in checks) < 1e-10
    assert max(c[2] for c in checks) < 1e-8
    assert all(x.sign == 1.0 and x.sign_running == 1.0 for x in ch.measurements)
    assert ch.max_dG < 1e-8


def test_g0_reduces_to_plain_slater_pqmc():
    """g = 0: the Gutzwiller slices are the identity; the accept sequence on the
    interaction slices and every measurement equal plain PQMC bit for bit."""
    a = pqmc.Chain(pqmc.Params(Lx=2, Ly=2, U=4.0, g=0.0, M_N=0.1, dtau=0.1, two_theta=2.0,
                               n_stab=5, seed=11, gutzwiller_slices=True))
    b = pqmc.Chain(pqmc.Params(Lx=2, Ly=2, U=4.0, g=0.0, M_N=0.1, dtau=0.1, two_theta=2.0,
                               n_stab=5, seed=11, gutzwiller_slices=False))
    a.run(2, 6)
    b.run(2, 6)
    Lt = a.m.Ltau
    la = [x for x in a.accept_log if 1 <= x[1] <= Lt]
    assert la == b.accept_log
    assert all(x[3] for x in a.accept_log if x[1] in (0, Lt + 1))
    assert [x.energy for x in a.measurements] == [x.energy for x in b.measurements]
    assert [x.docc for x in a.measurements] == [x.docc for x in b.measurements]


@pytest.mark.parametrize("k", [2, 3, 8])
def test_delayed_updates_match_sherman_morrison(k):
    kw = dict(Lx=2, Ly=2, U=4.0, g=0.6, M_N=0.21, dtau=0.1, two_theta=2.0, n_stab=5, seed=5)
    a = pqmc.Chain(pqmc.Params(delay_k=1, **kw))
    b = pqmc.Chain(pqmc.Params(delay_k=k, **kw))
    ga, gb = [], []
    a.hook = lambda c, e, t: ga.append(np.stack([c.G[1], c.G[-1]]))
    b.hook = lambda c, e, t: gb.append(np.stack([c.G[1], c.G[-1]]))
    a.run(0, 3)
    b.run(0, 3)
    assert a.accept_log == b.accept_log
    assert max(np.abs(x - y).max() for x, y in zip(ga, gb)) < 1e-12


# ------------------------------------------------------ Monte Carlo vs exact
def mc_vs_exact(p, n_warm, n_meas):
    ch = pqmc.Chain(p).run(n_warm, n_meas)
    ms = ch.measurements
    s = [x.sign for x in ms]
    E, dE = pqmc.estimate([x.energy for x in ms], s)
    D, dD = pqmc.estimate([x.docc for x in ms], s)
    m = ch.m
    c = ed.Cluster(m.K, m.n_sigma[1], m.n_sigma[-1], p.U)
    Ex, Dx = c.trotter_projection(m.P[1], m.P[-1], p.g, p.dtau, m.Ltau)
    return (E, dE, Ex / m.N), (D, dD, Dx / m.N), ch


def test_mc_energy_within_3sigma_of_exact_honeycomb():
    p = pqmc.Params(Lx=2, Ly=2, U=4.0, g=0.6, M_N=0.21, dtau=0.1, two_theta=2.0, n_stab=5, seed=7)
    (E, dE, Ex), (D, dD, Dx), ch = mc_vs_exact(p, 10, 400)
    assert abs(E - Ex) < 3 * dE and dE < 0.02
    assert abs(D - Dx) < 3 * dD
    # the exact Trotterised estimate lies near the continuum ground state
    e0, _ = ed.Cluster(ch.m.K, 4, 4, 4.0).ground_state()
    assert abs(Ex - e0 / 8) < 0.05


def test_mc_energy_within_3sigma_of_exact_doped_square():
    """Doped t-t' cluster: signful weights (spin-channel HS off half filling)."""
    p = pqmc.Params(kind=lattice.SQUARE, Lx=2, Ly=4, tp=-0.2, U=4.0, dtau=0.1, two_theta=1.0,
                    g=0.5, M_N=0.1, n_up=3, n_dn=3, n_stab=5, seed=3)
    (E, dE, Ex), (D, dD, Dx), ch = mc_vs_exact(p, 10, 400)
    assert abs(E - Ex) < 3 * dE
    assert abs(D - Dx) < 3 * dD
    signs = np.array([x.sign for x in ch.measurements])
    assert np.all(signs == np.array([x.sign_running for x in ch.measurements]))


# ------------------------------------------------- AFM structure factor (f3)
@pytest.mark.parametrize("case", ["honeycomb", "doped_vmc", "negative_weights"])
def test_s_afm_enumeration_equals_fock_space(case):
    """The Wick form of S_AFM = (1/N^2) sum_ij eps_i eps_j <S^z_i S^z_j>
    (stagger squared plus same-spin exchange) summed over all fields equals
    the diagonal Fock-space operator (sum_i eps_i S^z_i)^2 / N^2 applied to
    the exact Trotterised bra and ket."""
    if case == "honeycomb":
        p = small_params()
    elif case == "doped_vmc":
        p = pqmc.Params(kind=lattice.SQUARE, Lx=2, Ly=4, tp=-0.2, U=4.0, dtau=0.1,
                        two_theta=0.0, g=0.5, M_N=0.1, n_up=3, n_dn=3, n_stab=1)
    else:
        p = small_params(U=8.0, dtau=0.2, two_theta=0.4, g=0.5, M_N=0.1, n_up=1, n_dn=2)
    m = pqmc.Model(p)
    r = hs_enum.enumerate_observables(p)
    c = ed.Cluster(m.K, m.n_sigma[1], m.n_sigma[-1], p.U)
    Ex, Dx, Sx = c.trotter_observables(m.P[1], m.P[-1], p.g, p.dtau, m.Ltau, m.eps)
    assert abs(r["E"] - Ex) < 1e-11 and abs(r["docc"] - Dx) < 1e-11
    assert abs(r["s_afm"] - Sx) < 1e-12
    assert 0.0 < Sx <= 0.25 + 1e-12


def test_s_afm_classical_neel_limit():
    """M_N >> t at g = 0, Theta = 0: the trial is the classical Neel state
    (A sites up, B sites down), whose staggered moment is N/2, so
    S_AFM = (N/2)^2 / N^2 = 1/4 up to O((t/M_N)^2)."""
    for kind, Lx, Ly in ((lattice.HONEYCOMB, 2, 2), (lattice.SQUARE, 4, 2)):
        p = pqmc.Params(kind=kind, Lx=Lx, Ly=Ly, U=4.0, dtau=0.1, two_theta=0.0,
                        g=0.0, M_N=1e5, n_stab=1, seed=1)
        ch = pqmc.Chain(p).run(0, 2)
        for x in ch.measurements:
            assert abs(x.s_afm - 0.25) < 1e-8


def test_s_afm_free_fermions_closed_form():
    """U = 0, g = 0, free Fermi-sea trial: G is the projector of the filled
    orbitals, G = 1 - Pi with Pi the projector on the N_s lowest eigenvectors
    of K.  With n_i = 1/2 on a half-filled bipartite lattice the stagger term
    vanishes, <c^+_i c_j> <c_i c^+_j> = Pi_ij (delta_ij - Pi_ij), and
        S_AFM = 2 (N_s - sum_ij eps_i eps_j Pi_ij^2) / (4 N^2).
    Pi comes from numpy's eigh of K, not from the trial builder; the trial's
    Neel tie-break (M_N = 1e-4) shifts S_AFM by far less than 1e-8."""
    p = pqmc.Params(Lx=2, Ly=2, U=0.0, g=0.0, M_N=0.0, dtau=0.1, two_theta=1.0, n_stab=5, seed=2)
    ch = pqmc.Chain(p).run(0, 2)
    m = ch.m
    w, v = np.linalg.eigh(m.K)
    ns = m.N // 2
    assert w[ns] - w[ns - 1] > 0.5                      # closed shell
    Pi = v[:, :ns] @ v[:, :ns].T
    want = 2.0 * (ns - np.sum(np.outer(m.eps, m.eps) * Pi * Pi)) / (4.0 * m.N ** 2)
    for x in ch.measurements:
        assert abs(x.s_afm - want) < 1e-8


def test_mc_s_afm_within_3sigma_of_exact():
    p = pqmc.Params(Lx=2, Ly=2, U=4.0, g=0.6, M_N=0.21, dtau=0.1, two_theta=2.0, n_stab=5, seed=11)
    ch = pqmc.Chain(p).run(10, 400)
    ms = ch.measurements
    S, dS = pqmc.estimate([x.s_afm for x in ms], [x.sign for x in ms])
    m = ch.m
    c = ed.Cluster(m.K, 4, 4, p.U)
    _, _, Sx = c.trotter_observables(m.P[1], m.P[-1], p.g, p.dtau, m.Ltau, m.eps)
    assert abs(S - Sx) < 3 * dS and dS < 0.01


def test_s_afm_fixed_fields_equals_fock_space():
    """One field configuration at Theta > 0 (G not symmetric): the sweep's
    Wick estimate of S_AFM on G(Ltau/2) equals <L|S|R>/<L|R> with |R> and
    <L| the Slater determinants of B_R and B_L of each spin, built in Fock
    space.  Pins the index order of the exchange term."""
    p = small_params(two_theta=0.4, Lx=2, Ly=1)
    m = pqmc.Model(p)
    rng = np.random.default_rng(4)
    fields = rng.choice(np.array([-1, 1], dtype=np.int8), size=(m.Ltau + 2, m.N))
    ch = pqmc.Chain(p, fields=fields.copy())
    t = m.Ltau // 2
    ch.G = {sg: pqmc.green_definition(m, fields, t, sg) for sg in (+1, -1)}
    ch.measure()
    got = ch.measurements[-1].s_afm
    c = ed.Cluster(m.K, m.n_sigma[1], m.n_sigma[-1], p.U)
    vec = {}
    for sg in (+1, -1):
        R = m.P[sg].copy()
        for tt in range(0, t + 1):
            R = m.B(tt, sg, fields[tt]) @ R
        Lt = m.P[sg].copy()
        for tt in range(m.Ltau + 1, t, -1):
            Lt = m.B(tt, sg, fields[tt]).T @ Lt
        states = c.sup if sg == 1 else c.sdn
        vec[sg] = (ed.slater_vector(Lt, states), ed.slater_vector(R, states))
    L = np.outer(vec[1][0], vec[-1][0])
    R = np.outer(vec[1][1], vec[-1][1])
    want = c.s_afm(L, R, m.eps)
    assert abs(got - want) < 1e-12
    G = ch.G[1]
    assert np.abs(G - G.T).max() > 1e-3                 # the asymmetric case

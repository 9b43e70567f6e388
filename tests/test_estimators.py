"""Pins of the error bars that every Monte Carlo comparison rests on (CPU only).

The estimator of the Method section is the sign-reweighted ratio <s O>/<s>.
Its error is a delete-one-group jackknife: over bins of consecutive sweeps in
the oracle (oracle/pqmc.py: estimate) and in the library's pqmc_measure, over
chains in the pooled estimate (distributed.pooled_estimate).  Every "within
3 sigma" test trusts these errors, so they are tied here to answers fixed
independently of the code: a two-bin case worked by hand, i.i.d. Gaussian
records whose standard error is sigma / sqrt(n), and a signed ratio whose
variance follows from the delta method.  A slip that scales the error (the
jackknife factor (n - 1)/n written as n - 1 or 1/n, a missing square root,
bins averaged instead of summed) fails at least one of them.

Also here: the exact ground-state values of the 8-site cluster that the
Monte Carlo energies are set against, from the oracle's own Lanczos ED.
"""
import os

import numpy as np
import pytest

from oracle import ed, lattice, pqmc as opq
from paper_2303_13403_gb300 import build, distributed, pqmc


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pqmc.LIB_PATH):
        build.build()
    return pqmc.load()


# ------------------------------------------------------------ worked by hand
def test_two_bins_by_hand():
    # two bins of two records, all signs +1: bin means 1.5 and 4.5; the
    # jackknife replicates are the other bin's mean, so err = |m1 - m2| / 2,
    # the standard error of the mean of two bin means
    m, e = opq.estimate([1.0, 2.0, 3.0, 6.0], [1.0, 1.0, 1.0, 1.0], n_bins=2)
    assert m == 3.0 and e == 1.5


def test_two_signed_bins_by_hand():
    # values 1..6, sign -1 on the third record, two bins of three:
    # bin 1: sum sO = 1 + 2 - 3 = 0, sum s = 1;  bin 2: sum sO = 15, sum s = 3
    # mean = 15 / 4; replicates 15/3 = 5 and 0/1 = 0, their mean 2.5,
    # err = sqrt(1/2 * (2.5^2 + 2.5^2)) = 2.5
    v = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
    s = [1.0, 1.0, -1.0, 1.0, 1.0, 1.0]
    m, e = opq.estimate(v, s, n_bins=2)
    assert m == 3.75 and abs(e - 2.5) < 1e-15
    # the same two groups through the pooled (over chains) and library forms
    sums = np.array([[0.0, 0.0, 1.0, 3.0, 0.0], [15.0, 0.0, 3.0, 3.0, 0.0]])
    est = distributed.pooled_estimate(sums)
    assert est["E"] == 3.75 and abs(est["E_err"] - 2.5) < 1e-15


def test_library_jackknife_by_hand(lib):
    m, e = pqmc.host_jackknife([0.0, 15.0], [1.0, 3.0])
    assert m == 3.75 and abs(e - 2.5) < 1e-15
    m, e = pqmc.host_jackknife([7.0], [2.0])
    assert m == 3.5 and np.isnan(e)


# --------------------------------------------------------- i.i.d. statistics
def test_iid_gaussian_error_is_sigma_over_sqrt_n():
    """Unit-variance i.i.d. records, 200 per run in 20 bins: the jackknife
    variance is unbiased for sigma^2 / n = 0.005.  Over 4000 runs its mean
    has a relative sampling error of sqrt(2/19/4000) = 0.5%, and the spread
    of the 4000 means (sample variance, relative error 2.2%) must agree."""
    rng = np.random.default_rng(12345)
    runs, n = 4000, 200
    X = rng.standard_normal((runs, n))
    ones = np.ones(n)
    means = np.empty(runs)
    var = np.empty(runs)
    for r in range(runs):
        means[r], e = opq.estimate(X[r], ones)
        var[r] = e * e
    assert abs(var.mean() / (1.0 / n) - 1.0) < 0.03
    assert abs(means.var(ddof=1) / (1.0 / n) - 1.0) < 0.10


def test_signed_ratio_error_follows_delta_method():
    """Signs +1 with probability 0.8, O ~ N(-0.8, 0.05^2) independent of the
    sign: <sO>/<s> estimates -0.8 with variance sigma_O^2 / (n <s>^2) to first
    order in 1/n (delta method), here 0.0025 / (400 * 0.36).  The mean
    jackknife variance over 3000 runs and the spread of the estimates must
    both match it."""
    rng = np.random.default_rng(2024)
    runs, n = 3000, 400
    target = 0.05 ** 2 / (n * 0.6 ** 2)
    ests = np.empty(runs)
    var = np.empty(runs)
    for r in range(runs):
        s = np.where(rng.random(n) < 0.8, 1.0, -1.0)
        O = -0.8 + 0.05 * rng.standard_normal(n)
        ests[r], e = opq.estimate(O, s)
        var[r] = e * e
    assert abs(var.mean() / target - 1.0) < 0.05
    assert abs(ests.var(ddof=1) / target - 1.0) < 0.10
    assert abs(ests.mean() + 0.8) < 4 * np.sqrt(target / runs)


def test_pooled_over_chains_is_sigma_over_sqrt_n():
    """The pooled estimate's jackknife over chains: 40 chains of 25 unit-variance
    records each; its variance must be 1 / 1000 on average over 2000 runs."""
    rng = np.random.default_rng(7)
    runs, chains, per = 2000, 40, 25
    var = np.empty(runs)
    for r in range(runs):
        x = rng.standard_normal((chains, per))
        sums = np.column_stack([x.sum(axis=1), x.sum(axis=1), np.full(chains, per), np.full(chains, per),
                                x.sum(axis=1)])
        var[r] = distributed.pooled_estimate(sums)["E_err"] ** 2
    assert abs(var.mean() * chains * per - 1.0) < 0.05


# ------------------------------------------------ library == oracle, same bins
@pytest.mark.parametrize("n", [200, 213])
def test_library_jackknife_equals_oracle(lib, n):
    rng = np.random.default_rng(n)
    s = np.where(rng.random(n) < 0.7, 1.0, -1.0)
    O = 0.3 + rng.standard_normal(n)
    m_o, e_o = opq.estimate(O, s)
    per = n // 20
    sO = (s * O)[: per * 20].reshape(20, per).sum(axis=1)
    ss = s[: per * 20].reshape(20, per).sum(axis=1)
    m_l, e_l = pqmc.host_jackknife(sO, ss)
    assert abs(e_l - e_o) <= 1e-12 * e_o
    if n % 20 == 0:
        assert abs(m_l - m_o) <= 1e-12 * abs(m_o)


# ----------------------------------------------------------- ED ground state
@pytest.mark.parametrize("U,E0,docc", [(4.0, -5.954236681057, 0.125649427910),
                                       (3.5, -6.488606477882, None)])
def test_ed_ground_state_of_8_site_cluster(U, E0, docc):
    """Continuum ground state of the 2x2 honeycomb cluster (8 sites, 4 up + 4
    down, periodic): the exact values the Trotterised projection approaches
    as 2 Theta grows, from an independent Lanczos run of the same Hamiltonian
    (E0 per cluster; docc per site)."""
    K, _ = lattice.honeycomb(2, 2)
    c = ed.Cluster(K, 4, 4, U)
    e0, v = c.ground_state()
    assert abs(e0 - E0) < 1e-9
    assert abs(e0 / 8 - E0 / 8) < 1e-9
    if docc is not None:
        _, d = c.energy_docc(v, v)
        assert abs(d / 8 - docc) < 1e-9

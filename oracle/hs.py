"""Hubbard-Stratonovich couplings (test infrastructure only).

Eq. (1) of the paper decouples the Gutzwiller factor with an Ising field and
cosh(lambda) = exp(g/2).  As printed, Eq. (1) couples the field to the charge
(n_up + n_dn); with real lambda that form is not an identity (at n = 0 its
right side is exp(-g/4), not 1).  The oracle takes the spin-channel reading,
which keeps the printed prefactor and the printed cosh condition:

    exp(-g (n_up - 1/2)(n_dn - 1/2)) = 1/2 exp(-g/4) sum_{s=+-1} exp(lambda s (n_up - n_dn)),
    cosh(lambda) = exp(g / 2).

At fixed particle numbers exp(-g (n_up-1/2)(n_dn-1/2)) is exp(-g n_up n_dn)
times a constant, so the trial state of Eq. (3) is reproduced exactly.

The Method section says the U term is handled by "the standard" HS
transformation; the same identity with g -> dtau U gives the Hirsch
spin-channel coupling alpha, cosh(alpha) = exp(dtau U / 2).

In slice tau the single-particle factor for spin sigma (+1 up, -1 down) is
exp(V_sigma(s)) = diag(exp(sigma kappa s_i)), kappa = alpha or lambda.
Flipping s_i multiplies that entry by exp(-2 sigma kappa s_i), so
Delta_sigma = exp(-2 sigma kappa s_i) - 1.
"""
import numpy as np


def coupling(x):
    """kappa with cosh(kappa) = exp(x / 2); x = g or dtau * U."""
    return float(np.arccosh(np.exp(x / 2.0)))


def alpha(dtau, U):
    return coupling(dtau * U)


def lam(g):
    return coupling(g)


def delta(kappa, sigma, s):
    """Delta_sigma for flipping field value s (scalar or array)."""
    return np.exp(-2.0 * sigma * kappa * np.asarray(s, dtype=np.float64)) - 1.0

"""Neel mean-field trial state (test infrastructure only).

Honeycomb Hubbard section: |psi_N> is the ground state of
H_N = H_0 + M_N sum_i (-1)^{delta_i} (n_i,up - n_i,dn).  The printed sign
convention ("delta_i = +-1 if site i belongs to A(B)") gives -1 on both
sublattices; the oracle reads it as the staggered sign eps_i = +1 (A), -1 (B).

Per spin sigma (+1 up, -1 down) the single-particle matrix is
h_sigma = K + sigma M_N diag(eps), and P_sigma holds its N_sigma lowest
eigenvectors (N x N_sigma).

Open shells.  Honeycomb clusters with L a multiple of 3 have zero modes at
M_N = 0, and the square 8x8 t-t' cluster at 28 particles per spin has a
degenerate shell.  The trial needs a unique ground state, so:

* honeycomb: the Neel field is raised to max(M_N, tiebreak), default 1e-4
  (Neel direction: particle-hole symmetry, hence the sign, is kept);
* square: a spin-independent on-site term tiebreak * w_i is added to the
  trial Hamiltonian only, w_i = cos(pi x_i / 4) + cos(pi y_i / 2) / 2 at site
  (x_i, y_i), default tiebreak 0.2.  Plane-wave shell states mix only through
  the Fourier components of the on-site term at their momentum differences;
  this modulation has them, and opens a gap of 0.03 on the 8x8 t' = -0.2
  lattice at 28 particles, while a quasi-random term splits that shell by
  only ~1e-4 and leaves the trial defined to no better than ~1e-12.

G depends only on the span of P_sigma, so any orthonormal basis of it serves.
"""
import numpy as np

from . import lattice



def trial_hamiltonian(kind, K, eps, M_N, sigma, tiebreak=-1.0, lx=None):
    N = K.shape[0]
    if kind == lattice.HONEYCOMB:
        tb = 1e-4 if tiebreak < 0 else tiebreak
        m = max(M_N, tb)
        return K + sigma * m * np.diag(eps)
    tb = 0.2 if tiebreak < 0 else tiebreak
    Lx = int(round(lx)) if lx else N
    x = np.arange(N) % Lx
    y = np.arange(N) // Lx
    w = np.cos(np.pi * x / 4.0) + 0.5 * np.cos(np.pi * y / 2.0)
    return K + sigma * M_N * np.diag(eps) + tb * np.diag(w)


def trial_orbitals(kind, K, eps, M_N, n_sigma, sigma, tiebreak=-1.0, lx=None):
    """P_sigma (N x n_sigma) and the gap above the last occupied level.
    lx is the extent Lx of a square lattice (site i sits at x = i mod Lx)."""
    h = trial_hamiltonian(kind, K, eps, M_N, sigma, tiebreak, lx)
    e, v = np.linalg.eigh(h)
    gap = e[n_sigma] - e[n_sigma - 1] if n_sigma < len(e) else np.inf
    return v[:, :n_sigma].copy(), float(gap)

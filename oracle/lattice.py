"""Hopping matrices K (test infrastructure only).

The honeycomb Hubbard model of Eq. (2) has nearest-neighbour hopping -t.  The
paper does not fix geometry, site order or boundary conditions; the oracle
uses this reading (the CUDA side's host code restates it independently):

* honeycomb Lx x Ly unit cells, periodic, N = 2 Lx Ly sites,
  site id = 2 (x + Lx y) + sub, sub = 0 (A) or 1 (B);
  A(x, y) bonds to B(x, y), B(x-1, y) and B(x, y-1);
* square Lx x Ly, periodic, id = x + Lx y, nearest-neighbour hopping -t and
  next-nearest-neighbour hopping -t' (the doped t-t' workload);
* every bond adds its amplitude to K_ij and K_ji, so on clusters that wrap
  onto themselves a doubled bond carries twice the amplitude.

The staggered sign eps_i (+1 on A, -1 on B; (-1)^(x+y) on the square
lattice) is the sublattice sign used by the Neel term of H_N.
"""
import numpy as np

HONEYCOMB = 0
SQUARE = 1


def honeycomb(Lx, Ly, t=1.0):
    """K and eps for the honeycomb lattice of Eq. (2)."""
    N = 2 * Lx * Ly
    K = np.zeros((N, N))
    eps = np.zeros(N)

    def site(x, y, sub):
        return 2 * ((x % Lx) + Lx * (y % Ly)) + sub

    for y in range(Ly):
        for x in range(Lx):
            a = site(x, y, 0)
            eps[a] = 1.0
            eps[site(x, y, 1)] = -1.0
            for b in (site(x, y, 1), site(x - 1, y, 1), site(x, y - 1, 1)):
                K[a, b] += -t
                K[b, a] += -t
    return K, eps


def square(Lx, Ly, t=1.0, tp=0.0):
    """K and eps for the square t-t' lattice."""
    N = Lx * Ly
    K = np.zeros((N, N))
    eps = np.zeros(N)

    def site(x, y):
        return (x % Lx) + Lx * (y % Ly)

    for y in range(Ly):
        for x in range(Lx):
            i = site(x, y)
            eps[i] = 1.0 if (x + y) % 2 == 0 else -1.0
            for dx, dy, amp in ((1, 0, t), (0, 1, t), (1, 1, tp), (1, -1, tp)):
                if amp == 0.0:
                    continue
                j = site(x + dx, y + dy)
                K[i, j] += -amp
                K[j, i] += -amp
    return K, eps


def hopping(kind, Lx, Ly, t=1.0, tp=0.0):
    if kind == HONEYCOMB:
        return honeycomb(Lx, Ly, t)
    if kind == SQUARE:
        return square(Lx, Ly, t, tp)
    raise ValueError("unknown lattice kind %r" % (kind,))

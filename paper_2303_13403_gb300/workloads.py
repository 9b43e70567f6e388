"""Seeded synthetic workloads shared by the tests, the oracle runs and bench.py.

Pure data: lattice shapes, couplings, projection lengths, trial parameters and
seeded random field configurations.  It holds none of the method's arithmetic.

The paper measures on model Hamiltonians, not datasets, so these specs are the
complete workload; shapes follow its honeycomb Hubbard runs (U = 3.5-4.0, half
filling, Gutzwiller trial g = 0.6, M_N = 0.21, optimal for U = 4 in Fig. 1)
plus a doped square t-t' lattice for the sign study.
"""
from dataclasses import dataclass, asdict, replace

import numpy as np

HONEYCOMB = 0
SQUARE = 1
HONEYCOMB_TV = 2        # spinless t-V model on the honeycomb lattice (U holds V, M_N holds Delta_C)

FP64 = 0
FP32 = 1
BF16X3 = 2
PRECISION_NAMES = {FP64: "fp64", FP32: "fp32", BF16X3: "bf16x3"}


@dataclass(frozen=True)
class ChainSpec:
    kind: int = HONEYCOMB
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
    tiebreak: float = -1.0  # <0: default open-shell tie-break

    @property
    def n_sites(self):
        return self.Lx * self.Ly if self.kind == SQUARE else 2 * self.Lx * self.Ly

    @property
    def n_fields(self):
        """Ising fields per slice: one per site, or one per bond (t-V)."""
        return 3 * self.Lx * self.Ly if self.kind == HONEYCOMB_TV else self.n_sites

    @property
    def n_slices(self):
        """Interaction slices Ltau = 2 Theta / dtau."""
        return int(round(self.two_theta / self.dtau))

    def as_dict(self):
        return asdict(self)


def honeycomb(L, **kw):
    return ChainSpec(kind=HONEYCOMB, Lx=L, Ly=L, **kw)


def tv_honeycomb(L, V=1.6, g=0.0, Delta_C=0.0, two_theta=4.0, dtau=0.1, Ly=None, **kw):
    """Spinless t-V chain on the L x L honeycomb lattice at half filling."""
    return ChainSpec(kind=HONEYCOMB_TV, Lx=L, Ly=L if Ly is None else Ly, U=V, dtau=dtau, two_theta=two_theta,
                     g=g, M_N=Delta_C, n_up=-1, n_dn=0, **kw)


# Plain PQMC with a Slater trial on the 18-site honeycomb cluster: 100 slices,
# FP64, seed 1 (the small case the oracle runs in seconds).
PLAIN_18 = honeycomb(3, U=4.0, dtau=0.1, two_theta=10.0, g=0.0, M_N=0.0)
PLAIN_18_SWEEPS = (50, 200)

# Gutzwiller PQMC on the 72-site honeycomb cluster, U = 4, g = 0.6, M_N = 0.21.
GUTZ_72 = {tt: honeycomb(6, U=4.0, dtau=0.1, two_theta=tt, g=0.6, M_N=0.21)
           for tt in (4.0, 8.0, 16.0)}

# Large single chain: 648-site honeycomb, 200 slices, delay rank 32.
GUTZ_648 = honeycomb(18, U=4.0, dtau=0.1, two_theta=20.0, g=0.6, M_N=0.21)

# Doped square t-t' lattice: 8x8, t' = -0.2, 28 up + 28 down, 2 Theta = 12.
DOPED_64 = {g: ChainSpec(kind=SQUARE, Lx=8, Ly=8, tp=-0.2, U=4.0, dtau=0.1,
                         two_theta=12.0, g=g, M_N=0.0, n_up=28, n_dn=28)
            for g in (0.0, 0.3, 0.6)}


def variational_grid(two_theta=8.0):
    """The batched (g, M_N) scan: 11 x 11 grid for U = 3.5 and U = 4.0 (242
    chains), honeycomb L = 6/9/12 assigned cyclically over the grid."""
    specs = []
    for U in (3.5, 4.0):
        for ig in range(11):
            for im in range(11):
                L = (6, 9, 12)[(ig * 11 + im) % 3]
                specs.append(honeycomb(L, U=U, dtau=0.1, two_theta=two_theta,
                                       g=ig / 10.0, M_N=0.03 * im))
    return specs


def random_fields(spec, seed):
    """Seeded uniform +-1 fields, shape (Ltau + 2, N), int8."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.array([-1, 1], dtype=np.int8),
                      size=(spec.n_slices + 2, spec.n_fields))

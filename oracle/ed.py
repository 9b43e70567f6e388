"""Fock-space exact diagonalisation of small clusters (test infrastructure only).

Independent of the determinant machinery: states are occupation-number
bitstrings, operators act on many-body vectors.  Used to pin the oracle's
PQMC estimator (Method section) with

* the continuum ground state of Eq. (2) (Lanczos), and
* the exact Trotterised projection, with the same operator order as the
  slices B_tau = e^{-dtau K} e^{V}:
      |R> = (e^{-dtau K} e^{-dtau U D})^{Ltau/2} e^{-g D} |psi_N>,
      <L| = <psi_N| e^{-g D} (e^{-dtau K} e^{-dtau U D})^{Ltau/2},
      E   = <L|H|R> / <L|R>,   D = sum_i n_i,up n_i,dn.
  The HS identity of Eq. (1) (spin-channel reading) is exact, so the PQMC
  estimator has no bias against this number, only statistical error.

A basis state is c^+_{i1} c^+_{i2} ... |0> with i1 < i2 < ...; the amplitude of a
Slater determinant with orbitals P on it is det(P[rows i1, i2, ...]).
"""
from itertools import combinations

import numpy as np
import scipy.sparse.linalg as spla


def basis(N, n):
    states = [sum(1 << i for i in occ) for occ in combinations(range(N), n)]
    return np.array(states, dtype=np.int64), {s: k for k, s in enumerate(states)}


def _count_below(state, i):
    return bin(state & ((1 << i) - 1)).count("1")


def hopping_sector(K, n):
    """Matrix of sum_ij K_ij c^+_i c_j on the n-particle space of one spin."""
    N = K.shape[0]
    states, index = basis(N, n)
    dim = len(states)
    M = np.zeros((dim, dim))
    for a, st in enumerate(states):
        for i in range(N):
            for j in range(N):
                if K[i, j] == 0.0:
                    continue
                if not (st >> j) & 1:
                    continue
                if i == j:
                    M[a, a] += K[i, i]
                    continue
                if (st >> i) & 1:
                    continue
                sgn = (-1) ** _count_below(st, j)
                mid = st ^ (1 << j)
                sgn *= (-1) ** _count_below(mid, i)
                new = mid | (1 << i)
                M[index[new], a] += sgn * K[i, j]
    return M, states


def slater_vector(P, states):
    """Amplitudes det(P[occupied rows]) of a Slater determinant."""
    N, n = P.shape
    out = np.zeros(len(states))
    for a, st in enumerate(states):
        rows = [i for i in range(N) if (st >> i) & 1]
        out[a] = np.linalg.det(P[rows, :])
    return out


class Cluster:
    def __init__(self, K, n_up, n_dn, U):
        self.K = K
        self.N = K.shape[0]
        self.U = U
        self.Mup, self.sup = hopping_sector(K, n_up)
        self.Mdn, self.sdn = hopping_sector(K, n_dn)
        self.D = np.array([[bin(a & b).count("1") for b in self.sdn] for a in self.sup],
                          dtype=np.float64)

    def apply_K(self, X):
        return self.Mup @ X + X @ self.Mdn.T

    def apply_H(self, X):
        return self.apply_K(X) + self.U * self.D * X

    def ground_state(self):
        shape = self.D.shape
        dim = shape[0] * shape[1]
        op = spla.LinearOperator((dim, dim), dtype=np.float64,
                                 matvec=lambda v: self.apply_H(v.reshape(shape)).ravel())
        if dim <= 400:
            H = np.column_stack([op.matvec(e) for e in np.eye(dim)])
            w, v = np.linalg.eigh(H)
            return float(w[0]), v[:, 0].reshape(shape)
        w, v = spla.eigsh(op, k=1, which="SA", tol=1e-13, maxiter=20000)
        return float(w[0]), v[:, 0].reshape(shape)

    def energy_docc(self, L, R):
        """(<L|H|R>/<L|R>, <L|D|R>/<L|R>)."""
        norm = float(np.sum(L * R))
        return (float(np.sum(L * self.apply_H(R))) / norm,
                float(np.sum(L * self.D * R)) / norm)

    def s_afm(self, L, R, eps):
        """<L|S|R>/<L|R> for S = (1/N^2) (sum_i eps_i S^z_i)^2, S^z_i = (n_up - n_dn)/2.

        S is diagonal in the occupation basis: a basis state with up set a and
        down set b has sum_i eps_i S^z_i = (sum_{i in a} eps_i - sum_{i in b} eps_i)/2.
        """
        def stagger(states):
            return np.array([sum(eps[i] for i in range(self.N) if (st >> i) & 1) for st in states])
        mz = 0.5 * (stagger(self.sup)[:, None] - stagger(self.sdn)[None, :])
        return float(np.sum(L * mz * mz * R)) / float(np.sum(L * R)) / (self.N * self.N)

    def trotter_projection(self, P_up, P_dn, g, dtau, Ltau):
        """Exact Trotterised estimate of E and D at the middle slice."""
        return self.energy_docc(*self.trotter_states(P_up, P_dn, g, dtau, Ltau))

    def trotter_observables(self, P_up, P_dn, g, dtau, Ltau, eps):
        """(E, D, S_AFM) of the exact Trotterised projection at the middle slice."""
        L, R = self.trotter_states(P_up, P_dn, g, dtau, Ltau)
        E, D = self.energy_docc(L, R)
        return E, D, self.s_afm(L, R, eps)

    def trotter_states(self, P_up, P_dn, g, dtau, Ltau):
        """Bra and ket at the middle slice (shapes dim_up x dim_dn)."""
        def expm_sym(M, x):
            w, v = np.linalg.eigh(M)
            return (v * np.exp(x * w)) @ v.T
        Eup = expm_sym(self.Mup, -dtau)
        Edn = expm_sym(self.Mdn, -dtau)
        eV = np.exp(-dtau * self.U * self.D)
        psi = np.outer(slater_vector(P_up, self.sup), slater_vector(P_dn, self.sdn))
        psi = np.exp(-g * self.D) * psi
        R = psi.copy()
        L = psi.copy()
        for _ in range(Ltau // 2):
            R = Eup @ (eV * R) @ Edn.T          # e^{-dtau K} e^{-dtau U D} on the ket
            L = eV * (Eup @ L @ Edn.T)        # transpose of the same product, bra side
        return L, R

// Host-side FP64 model set-up: lattice hopping matrices, a symmetric
// eigensolver, matrix exponentials of K and the Neel trial orbitals.
#pragma once
#include <string>
#include <vector>

namespace pqmc {

struct Lattice {
  int kind;      // 0 honeycomb, 1 square
  int Lx, Ly;
  double t, tp;
  int n_sites() const { return kind == 0 ? 2 * Lx * Ly : Lx * Ly; }
};

// Hopping matrix K (N x N row-major) of the model of Eq. (2) (honeycomb) or of
// the square t-t' lattice, and the staggered sublattice sign eps_i.
void build_hopping(const Lattice& lat, std::vector<double>& K, std::vector<double>& eps);

// Symmetric eigen-decomposition A = V diag(w) V^T, w ascending, eigenvectors in
// the columns of V (row-major). Householder tridiagonalisation followed by the
// implicit symmetric QR iteration with Wilkinson shifts (Golub & Van Loan,
// Matrix Computations, sections 8.3.1-8.3.3). Returns false if it fails to
// converge.
bool sym_eig(int n, const std::vector<double>& A, std::vector<double>& w, std::vector<double>& V);

// e^{x K} = V diag(e^{x w}) V^T for symmetric K given its decomposition.
void expm_from_eig(int n, const std::vector<double>& w, const std::vector<double>& V, double x,
                   std::vector<double>& out);

// Trial orbitals of the Neel mean-field Hamiltonian H_N (honeycomb Hubbard
// section) for one spin sigma = +1 (up) or -1 (down): the n_sigma lowest
// eigenvectors (N x n_sigma, row-major) of h = K + sigma M diag(eps) with the
// open-shell tie-break, plus the gap above the last occupied level.
bool trial_orbitals(const Lattice& lat, const std::vector<double>& K, const std::vector<double>& eps,
                    double M_N, double tiebreak, int sigma, int n_sigma, std::vector<double>& P,
                    double& gap);

// cosh(kappa) = exp(x / 2): the Ising coupling of Eq. (1) in the spin-channel
// reading (x = g) and of the Trotterised U term (x = dtau U).
double hs_coupling(double x);

}  // namespace pqmc

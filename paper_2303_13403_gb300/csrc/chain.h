// Per-chain descriptors shared by the CUDA kernels (sweep.cu) and the host
// side of the C-ABI (api.cpp). Plain data: device pointers and sizes.
#pragma once
#include <stdint.h>

namespace pqmc {

constexpr int kBlock = 32;        // sites per delayed-update block (one warp)
constexpr int kThreads = 256;     // threads per chain CTA
constexpr int kRecord = 5;        // doubles per measurement record
constexpr int kDGHistory = 4096;  // stabilisation errors kept per chain

// error bits written by the kernels
enum : int { kErrNaN = 1, kErrStab = 2, kErrTimeout = 4 };

// Mutable per-chain counters, in device memory.
struct ChainState {
  long long n_prop;
  long long n_acc;
  long long acc_pos;      // next accept-log slot
  int n_meas;             // records written
  int n_dG;               // stabilisation errors written (total, ring of kDGHistory)
  double sign_running;    // product of sgn(R) over accepted flips
  double max_dG;
  double logw[2][2];      // [spin][logabs, sign] at the last stabilisation
  double sign_stack;      // prod over spins of the weight sign at the last stabilisation
  int err;
  int pad;
};

// Read-only description of one chain plus pointers to its device buffers.
// Matrices of the path precision T (float or double) are row-major with
// leading dimension ld; FP64 stack blocks are column-major N x n_sigma with
// leading dimension N.
struct ChainDesc {
  int N, ld, nup, ndn, nmax;
  int Ltau, nb, n_stab, kb;
  uint32_t chain_index;
  double U;
  double delta[2][2][2];   // [0 Hubbard, 1 Gutzwiller][spin][s=+1 -> 0, s=-1 -> 1]: e^{-2 sigma kappa s} - 1
  double vexp[2][2][2];    // same indexing: e^{sigma kappa s}
  int8_t* fields;          // (Ltau+2) x N
  void* G;                 // 2 x N x ld (T)
  void* Gt;                // 2 x N x ld (T), temporary
  const void* expKm;       // N x ld (T): e^{-dtau K}
  const void* expKp;       // N x ld (T): e^{+dtau K}
  const double* expKm64;   // N x N FP64
  const double* K64;       // N x N FP64
  const double* P;         // 2 x (N x nmax) FP64, column-major per spin (ld N)
  double* Rst;             // (nb+1) x 2 x (N x nmax) FP64
  double* Lst;             // (nb+1) x 2 x (N x nmax) FP64
  double* Rlog;            // (nb+1) x 2 x 2 (logabs, sign)
  double* Llog;            // (nb+1) x 2 x 2
  double* work;            // FP64 scratch: M, Q (N x nmax each), O (nmax^2), Y (nmax x N)
  void* UW;                // T scratch: 2 x (N x kBlock) + 2 x (kBlock x ld)
  double* meas;            // max_meas x kRecord
  int max_meas;
  int pad0;
  double* dG;              // kDGHistory
  uint8_t* acc_log;        // accept bits
  long long acc_cap;
  ChainState* st;
};

}  // namespace pqmc

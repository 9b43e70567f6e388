// Per-chain descriptors shared by the CUDA kernels (sweep_kernels.cuh) and the
// host side of the C-ABI (api.cpp). Plain data: device pointers and sizes.
#pragma once
#include <stdint.h>

namespace pqmc {

constexpr int kBlock = 32;        // sites per flip-decision sub-block (one warp); t-V bond blocks
constexpr int kMaxDelay = 64;     // largest delayed-update block (sites whose flips are applied at once)
constexpr int kMaxN = 1024;       // sites per chain
constexpr int kMaxSigma = 512;    // particles per spin
constexpr int kQRParts = 8;       // row chunks of the column dots in the Householder QR
constexpr int kRecord = 6;        // doubles per measurement record
constexpr int kDGHistory = 4096;  // stabilisation errors kept per chain

// phases timed with clock64() by thread 0 of each chain CTA
enum : int {
  kPhFlip = 0, kPhFlush, kPhWrap, kPhStack, kPhQR, kPhRefresh, kPhMeasure, kPhTotal,
  kPhQRForm, kPhOverlap, kPhLU, kPhAssemble, kPhGJPivot, kPhGJElim, kPhGJTail, kPhFlushVec, kPhases
  // (kPhLU: the marker after the Gauss-Jordan inverse, which the three kPhGJ
  // phases already cover; kept so that the counter layout stays fixed)
};

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
  long long cycles[kPhases];  // SM clock cycles spent per phase (thread 0's view)
  int err;
  int pad;
};

// Read-only description of one chain plus pointers to its device buffers.
// Matrices of the path precision T (float or double) are row-major with
// leading dimension ld; FP64 stack blocks are column-major N x n_sigma with
// leading dimension N.
struct ChainDesc {
  int N, ld, nup, ndn, nmax;
  int Ltau, nb, n_stab, kb;        // kb: delayed-update block, 8, 16, 32 or 64 sites (Hubbard chains)
  uint32_t chain_index;
  int tc;                  // 1: wrap and delayed-update GEMMs as split BF16 tensor-core products
  int tv;                  // 1: spinless t-V model (one species, bond fields)
  int nfld;                // fields per slice: N, or 3N/2 bonds (tv)
  int dg64;                // reduced paths: 1 record max |G - G_FP64| (G_FP64 assembled in FP64) at
                           // each stabilisation instead of the path-precision comparison; 2 the
                           // refreshed G against G_FP64; 3 as 1 over max(1, max |G_FP64|)
  double U;
  double delta[2][2][2];   // [0 Hubbard, 1 Gutzwiller][spin][s=+1 -> 0, s=-1 -> 1]: e^{-2 sigma kappa s} - 1
  double vexp[2][2][2];    // same indexing: e^{sigma kappa s}
  double vtv[2][7];        // tv: [0 Hubbard-type slice, 1 Gutzwiller][m + 3]: e^{kappa m}, m = sum of the
                           // site's three bond fields with sign +1 at A ends, -1 at B ends
  int8_t* fields;          // (Ltau+2) x nfld
  void* G;                 // 2 x N x ld (T)
  const void* expKm;       // N x ld (T): e^{-dtau K}
  const void* expKp;       // N x ld (T): e^{+dtau K}
  const double* expKm64;   // N x N FP64
  const double* K64;       // N x N FP64
  const double* eps;       // N: staggered sublattice sign (+1 A, -1 B)
  const int* bond_ends;    // tv: 3N/2 x 2 (A end, B end) of each bond
  const int* site_bonds;   // tv: N x 3 bonds of each site
  const double* P;         // 2 x (N x nmax) FP64, column-major per spin (ld N)
  double* Rst;             // (nb+1) x 2 x (N x nmax) FP64
  double* Lst;             // (nb+1) x 2 x (N x nmax) FP64
  double* Rlog;            // (nb+1) x 2 x 2 (logabs, sign)
  double* Llog;            // (nb+1) x 2 x 2
  void* scratch;           // per-chain phase scratch in global memory (layout: ScratchLayout),
                           // used when the chain does not fit in shared memory
  double* meas;            // max_meas x kRecord
  double* last;            // kRecord: latest record (slot in a context-wide array)
  int max_meas;
  int pad0;
  double* dG;              // kDGHistory
  uint8_t* acc_log;        // accept bits
  long long acc_cap;
  ChainState* st;
  unsigned char* spread;   // buffers of a chain swept by many CTAs (SpreadLayout), or null
};
static_assert(sizeof(ChainDesc) % sizeof(int) == 0, "descriptor copied word by word");

}  // namespace pqmc

namespace pqmc {

#if defined(__CUDACC__)
#define PQMC_HDI __host__ __device__ inline
#else
#define PQMC_HDI inline
#endif

// Byte offsets of the phase buffers inside one chain's scratch region.  The
// phases never overlap in time, so their buffers share the region:
//   wrap    : Gt (N x ld, T) for one spin at a time; for a chain resident in
//             shared memory also copies of e^{-dtau K} and e^{+dtau K}
//             (em, ep; 0 when they would make the scratch larger)
//   flips   : the update vectors of a delayed block, U (N x kw, T) and V
//             (kw x ld, T) of each spin (u, w for spin 0; u2, mw for
//             spin 1), kw = max(delayed block, kBlock); for t-V blocks A_S
//             (u), W and M W (w, mw); and the per-block flip buffers
//   stack   : M64 (N x n, FP64, column-major, ld m64_ld(N)), then a region holding the two
//             path-precision product buffers Mt, Mt2 (N x n, T, row-major)
//             and later the FP64 Q of the QR; Householder betas / R_jj;
//             the Gram matrix and pivots of the Cholesky QR
//   refresh : O (n x n, FP64, both spins, inverted in place), Y (n x ld, T), Q_R and Q_L in the
//             path precision (N x n, T); GJ pivots / multipliers; O^{-1} in
//             the path precision (n x n, T)
struct ScratchLayout {
  size_t gt, em, ep, u, u2, w, mw, fb, m64, mtq, mt2, qaux, chol, o, y, qrt, qlt, laux, ot, total;
};

PQMC_HDI constexpr size_t al16(size_t v) { return (v + 15) & ~(size_t)15; }

// Per-block buffers of the flip phase (kBlock x kBlock blocks of both spins,
// ratios of one decision sub-block, Delta and Delta/R of each accepted flip of
// a delayed block, accepted sites); the layout is FlipBuf<T> in
// sweep_kernels.cuh.
PQMC_HDI constexpr size_t flipbuf_bytes(int tsize) {
  return al16(2 * (size_t)kBlock * (kBlock + 1) * tsize + 2 * (size_t)kBlock * tsize +
              4 * (size_t)kMaxDelay * tsize + 2 * (size_t)kMaxDelay * 4);
}

// kd: the delayed-update block of the chain (its update vectors are sized
// for max(kd, kBlock) flips)
// leading dimension of the stack phase's FP64 block M in the scratch: odd, so
// that the Gram matrix's threads, each on its own columns, read different
// shared-memory banks
PQMC_HDI constexpr int m64_ld(int N) { return N | 1; }

PQMC_HDI ScratchLayout scratch_layout(int N, int ld, int n, int tsize, int kd) {
  ScratchLayout L;
  const size_t Nn = (size_t)N * n;
  const size_t kw = kd > kBlock ? (size_t)kd : (size_t)kBlock;
  L.gt = 0;
  size_t wrap = al16((size_t)N * ld * tsize);
  L.u = 0;
  L.u2 = al16((size_t)N * kw * tsize);
  L.w = L.u2 + al16((size_t)N * kw * tsize);
  L.mw = L.w + al16(kw * ld * tsize);
  L.fb = L.mw + al16(kw * ld * tsize);
  size_t flush = L.fb + flipbuf_bytes(tsize);
  L.m64 = 0;
  L.mtq = al16((size_t)m64_ld(N) * n * 8);
  L.mt2 = L.mtq + al16(Nn * tsize);
  const size_t two_mt = 2 * al16(Nn * tsize);
  const size_t mtq_sz = two_mt > al16(Nn * 8) ? two_mt : al16(Nn * 8);
  L.qaux = L.mtq + mtq_sz;
  L.chol = L.qaux + al16((3 * (size_t)n + (size_t)kQRParts * n) * 8);
  size_t stack = L.chol + al16((2 * (size_t)n * n + 3 * (size_t)n) * 8);
  L.o = 0;                                   // O for spin 0, then spin 1 (inverted in place)
  L.y = 2 * al16((size_t)n * n * 8);
  L.qrt = L.y + al16((size_t)n * ld * tsize);
  L.qlt = L.qrt + al16(Nn * tsize);
  L.laux = L.qlt + al16(Nn * tsize);
  L.ot = L.laux + al16(2 * 3 * (size_t)n * 8);
  size_t refresh = L.ot + al16((size_t)n * n * tsize);
  size_t t = wrap;
  if (flush > t) t = flush;
  if (stack > t) t = stack;
  if (refresh > t) t = refresh;
  L.em = wrap;
  L.ep = 2 * wrap;
  if (3 * wrap > t) L.em = L.ep = 0;
  L.total = (t + 255) & ~(size_t)255;
  return L;
}

// Buffers of a chain whose sweep runs as a sequence of grid-wide kernels
// (pqmc_opts.spread): byte offsets inside the chain's spread region, per
// spin s.
//   mt[s][0..1] : N x n (T, row-major, ld n) products advancing a stack block
//   m64[s]      : N x n (FP64, column-major, ld N) block to factor
//   c64[s]      : n x n (FP64, row-major) Gram matrix, then R in its upper part
//   rinv[s]     : inverses of R's kSpPanel x kSpPanel diagonal blocks
//   o64[s]      : n x n (FP64, row-major) Q_L^T Q_R, inverted in place
//   tgj[s]      : kSpGJ x n block row saved by a Gauss-Jordan panel step
//   pval, perm  : Gauss-Jordan pivots and row interchanges; d0 the Gram diagonal
//   xt, qrt, qlt: path-precision copies of O^{-1} (n x n), Q_R and Q_L (N x n, ld N)
//   y[s]        : n x ld (T) O^{-1} Q_L^T
//   gt[s]       : N x ld (T) wrap intermediate
//   g2          : 2 x N x ld (T) second copy of G: the block updates of a slice
//                 alternate between G and g2 (read one, write the other)
//   mb[s]       : M (kBlock x kBlock, T) of the flips accepted in one block
//   misc        : int na (accepted flips of the block), int bad[2] (Cholesky
//                 breakdown), then 8-aligned: uint64 dmax (bits of max |G - G_fresh|),
//                 double lchol[2] (log det R); at 64: int sites[kBlock] (accepted sites)
constexpr int kSpPanel = 32;   // Cholesky panel width
constexpr int kSpGJ = 16;      // Gauss-Jordan panel width
struct SpreadLayout {
  size_t mt[2][2], m64[2], c64[2], rinv[2], o64[2], tgj[2], pval[2], perm[2], d0[2], xt[2], qrt[2], qlt[2], y[2],
      gt[2], mb[2], g2, misc, total;
};

PQMC_HDI SpreadLayout spread_layout(int N, int ld, int n, int tsize) {
  SpreadLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return at;
  };
  const size_t Nn = (size_t)N * n, nn = (size_t)n * n, np = (size_t)((n + kSpPanel - 1) / kSpPanel);
  for (int s = 0; s < 2; ++s) {
    L.mt[s][0] = take(Nn * tsize);
    L.mt[s][1] = take(Nn * tsize);
    L.m64[s] = take(Nn * 8);
    L.c64[s] = take(nn * 8);
    L.rinv[s] = take(np * kSpPanel * kSpPanel * 8);
    L.o64[s] = take(nn * 8);
    L.tgj[s] = take((size_t)kSpGJ * n * 8);
    L.pval[s] = take((size_t)n * 8);
    L.perm[s] = take((size_t)n * 4);
    L.d0[s] = take((size_t)n * 8);
    L.xt[s] = take(nn * tsize);
    L.qrt[s] = take(Nn * tsize);
    L.qlt[s] = take(Nn * tsize);
    L.y[s] = take((size_t)n * ld * tsize);
    L.gt[s] = take((size_t)N * ld * tsize);
    L.mb[s] = take((size_t)kBlock * kBlock * tsize);
  }
  L.g2 = take(2 * (size_t)N * ld * tsize);
  L.misc = take(64 + kBlock * 4);
  L.total = off;
  return L;
}

// Shared-memory bytes of a chain that keeps G and its scratch resident
// (a chain that does not fit keeps only the flip buffers in shared memory).
PQMC_HDI size_t resident_bytes(int N, int ld, int n, int tsize, int kd) {
  return al16(2 * (size_t)N * ld * tsize) + scratch_layout(N, ld, n, tsize, kd).total;
}

}  // namespace pqmc

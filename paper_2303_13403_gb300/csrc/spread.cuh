#pragma once
// A chain swept by the whole GPU (pqmc_opts.spread).
//
// The single-CTA sweep kernel runs one chain on one SM; at 288 and more sites
// its FP64 stabilisation, its wrap and its delayed updates then run at one
// SM's rate.  Here the same sweep is a sequence of grid-wide kernels, launched
// in order on one stream and captured in a CUDA graph per sweep direction:
//
//   per block of kBlock sites   sp_decide (one CTA per chain: the Metropolis
//                               decisions of decide_sub_block, then the block
//                               form's M = Gamma (1 + (1 - G_SS) Gamma)^{-1}),
//                               sp_flush (tiles of G: G_new = G - (E_S - G_{:,S})
//                               M G_{S,:}, read from one copy of G and written
//                               to the other, so no tile reads what another
//                               tile writes)
//   per slice                   sp_scale (e^{V} G e^{-V}), two tile products
//                               with e^{-+dtau K} (the wrap)
//   per stabilisation           the n_stab slice products of the new stack
//                               block, its Cholesky QR (Gram matrix, blocked
//                               right-looking factor, Q = M R^{-1} row by row),
//                               O = Q_L^T Q_R, its blocked Gauss-Jordan inverse
//                               with partial pivoting, G = 1 - Q_R O^{-1} Q_L^T
//                               with max |G - G_fresh|, and sp_tail (weights,
//                               records, measurement)
//
// No kernel waits on another CTA: every dependency is a kernel boundary.  The
// arithmetic follows the single-CTA path phase by phase (same decisions, same
// Philox stream, same precisions: the wrap, the delayed update, the stack
// products and the assembly in the path precision, QR, overlap, inverse and
// weights in FP64); sums run in another order, so the two agree to rounding.
// The delayed update applies the flips of each kBlock-site block at once.
// Chains of one spread context share N, N_sigma and Ltau.
#include <algorithm>

#include "spread.h"
#include "sweep_kernels.cuh"

namespace pqmc {

// ---------------------------------------------------------------------------
// Tile products over a batch of (chain, spin) jobs: C = A B with A(i,k) =
// A[i sai + k sak], B(k,j) = B[k sbk + j sbj], C(i,j) = C[i sci + j scj].

struct SpJob {
  const void* A;
  const void* B;
  void* C;
  unsigned long long* dmax;   // kSpFresh: max |G - G_fresh| of the chain (bits of a non-negative double)
  const void* Cin;            // kSpFresh: the propagated G to compare with (same layout as C; null: C)
  int M, Nn, K;
  int p1;                     // kSpGJUpd: end of the panel block row
};
constexpr int kSpMaxJobs = 64;
enum : int { kSpStore = 0, kSpSub = 1, kSpFresh = 2, kSpGJUpd = 3 };
struct SpGemm {
  int sai, sak, sbk, sbj, sci, scj;
  int tiles_n;                // tiles along the columns of the largest job
  int split;                  // BF16X3 wrap products (T = float)
  int p0;                     // kSpGJUpd: start of the panel block row
  int upper;                  // 1: only tiles that reach the upper triangle (j >= i) are computed
  int njobs;
  SpJob job[kSpMaxJobs];
};

template <typename T> struct SpTile;
template <> struct SpTile<float> { static constexpr int TM = 64, TK = 16, R = 4; };
template <> struct SpTile<double> { static constexpr int TM = 32, TK = 32, R = 2; };
// the Cholesky block row is formed in place by one K slice per tile
static_assert(kSpPanel <= SpTile<double>::TK && kSpPanel <= SpTile<double>::TM, "block row in one tile slice");

// One TM x TM tile of C per CTA (256 threads, R x R outputs each, rows and
// columns interleaved by 16), operands staged through shared memory in
// TK-deep slices.
template <typename T, int kMode>
__global__ void __launch_bounds__(256) sp_gemm_kernel(SpGemm g) {
  constexpr int TM = SpTile<T>::TM, TK = SpTile<T>::TK, R = SpTile<T>::R;
  __shared__ __align__(16) T As[TK][TM + 1];
  __shared__ __align__(16) T Bs[TK][TM + 1];
  __shared__ double red[8];
  const SpJob& jb = g.job[blockIdx.y];
  const int r0 = (blockIdx.x / g.tiles_n) * TM, c0 = (blockIdx.x % g.tiles_n) * TM;
  if (r0 >= jb.M || c0 >= jb.Nn || (g.upper && r0 > c0 + TM - 1)) return;
  const T* A = static_cast<const T*>(jb.A);
  const T* B = static_cast<const T*>(jb.B);
  T* C = static_cast<T*>(jb.C);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if constexpr (std::is_same<T, float>::value) {
    if (g.split) {
      // BF16X3 wrap product: the split-precision tensor-core tile
      const int m = min(TM, jb.M - r0), nn = min(TM, jb.Nn - c0);
      cta_gemm_bf16x3(m, nn, jb.K, A + (long)r0 * g.sai, g.sai, g.sak, B + (long)c0 * g.sbj, g.sbk, g.sbj,
                      C + (long)r0 * g.sci + (long)c0 * g.scj, g.sci, g.scj, EpiStore());
      return;
    }
  }
  T acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < R; ++q) acc[r][q] = T(0);
  const bool a_i_fast = g.sai == 1, b_j_fast = g.sbj == 1;
  for (int k0 = 0; k0 < jb.K; k0 += TK) {
    for (int e = tid; e < TM * TK; e += 256) {
      int i, k;
      if (a_i_fast) { i = e % TM; k = e / TM; } else { k = e % TK; i = e / TK; }
      const int gi = r0 + i, gk = k0 + k;
      As[k][i] = (gi < jb.M && gk < jb.K) ? A[(long)gi * g.sai + (long)gk * g.sak] : T(0);
    }
    for (int e = tid; e < TM * TK; e += 256) {
      int j, k;
      if (b_j_fast) { j = e % TM; k = e / TM; } else { k = e % TK; j = e / TK; }
      const int gj = c0 + j, gk = k0 + k;
      Bs[k][j] = (gj < jb.Nn && gk < jb.K) ? B[(long)gk * g.sbk + (long)gj * g.sbj] : T(0);
    }
    __syncthreads();
    const int kt = min(TK, jb.K - k0);   // no FMAs on the zero padding (FP64 issue is scarce)
#pragma unroll 4
    for (int k = 0; k < kt; ++k) {
      T a[R], b[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = As[k][ty + 16 * r];
#pragma unroll
      for (int q = 0; q < R; ++q) b[q] = Bs[k][tx + 16 * q];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < R; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
    }
    __syncthreads();
  }
  double dm = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = r0 + ty + 16 * r, j = c0 + tx + 16 * q;
      if (i >= jb.M || j >= jb.Nn) continue;
      T& ref = C[(long)i * g.sci + (long)j * g.scj];
      if constexpr (kMode == kSpStore) {
        ref = acc[r][q];
      } else if constexpr (kMode == kSpSub) {
        ref -= acc[r][q];
      } else if constexpr (kMode == kSpFresh) {
        // G_fresh = delta_ij - (Q_R Y)_ij against the propagated G
        const T gnew = (i == j ? T(1) : T(0)) - acc[r][q];
        const T gold = jb.Cin ? static_cast<const T*>(jb.Cin)[(long)i * g.sci + (long)j * g.scj] : ref;
        const T d = fabs(gold - gnew);
        dm = d == d ? fmax(dm, (double)d) : INFINITY;   // a NaN is recorded as +inf
        ref = gnew;
      } else {
        // Gauss-Jordan block update of the columns outside the panel
        if (j >= g.p0 && j < jb.p1) continue;
        ref = ((i >= g.p0 && i < jb.p1) ? T(0) : ref) + acc[r][q];
      }
    }
  if constexpr (kMode == kSpFresh) {
    // max over the CTA, then over the chain (non-negative doubles order like
    // their bit patterns)
    dm = warp_max(dm);
    if ((tid & 31) == 0) red[tid >> 5] = dm;
    __syncthreads();
    if (tid == 0) {
      double m = red[0];
      for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
      atomicMax(jb.dmax, (unsigned long long)__double_as_longlong(m));
    }
  }
}

// ---------------------------------------------------------------------------
// Per-chain pointers of the spread buffers.

// (tsize: the path precision's element size, which places the FP64 buffers
// too)
template <typename T>
struct SpBuf {
  unsigned char* b;
  SpreadLayout L;
  __device__ __host__ SpBuf(unsigned char* base, int N, int ld, int nmax, int tsize = (int)sizeof(T))
      : b(base), L(spread_layout(N, ld, nmax, tsize)) {}
  __device__ __host__ T* mt(int s, int k) const { return reinterpret_cast<T*>(b + L.mt[s][k]); }
  __device__ __host__ double* m64(int s) const { return reinterpret_cast<double*>(b + L.m64[s]); }
  __device__ __host__ double* c64(int s) const { return reinterpret_cast<double*>(b + L.c64[s]); }
  __device__ __host__ double* rinv(int s) const { return reinterpret_cast<double*>(b + L.rinv[s]); }
  __device__ __host__ double* o64(int s) const { return reinterpret_cast<double*>(b + L.o64[s]); }
  __device__ __host__ double* tgj(int s) const { return reinterpret_cast<double*>(b + L.tgj[s]); }
  __device__ __host__ double* pval(int s) const { return reinterpret_cast<double*>(b + L.pval[s]); }
  __device__ __host__ int* perm(int s) const { return reinterpret_cast<int*>(b + L.perm[s]); }
  __device__ __host__ double* d0(int s) const { return reinterpret_cast<double*>(b + L.d0[s]); }
  __device__ __host__ T* xt(int s) const { return reinterpret_cast<T*>(b + L.xt[s]); }
  __device__ __host__ T* qrt(int s) const { return reinterpret_cast<T*>(b + L.qrt[s]); }
  __device__ __host__ T* qlt(int s) const { return reinterpret_cast<T*>(b + L.qlt[s]); }
  __device__ __host__ T* y(int s) const { return reinterpret_cast<T*>(b + L.y[s]); }
  __device__ __host__ T* gt(int s) const { return reinterpret_cast<T*>(b + L.gt[s]); }
  __device__ __host__ T* mb(int s) const { return reinterpret_cast<T*>(b + L.mb[s]); }
  __device__ __host__ T* g2() const { return reinterpret_cast<T*>(b + L.g2); }
  __device__ __host__ int* sites() const { return reinterpret_cast<int*>(b + L.misc + 64); }
  __device__ __host__ int* na() const { return reinterpret_cast<int*>(b + L.misc); }
  __device__ __host__ int* bad() const { return reinterpret_cast<int*>(b + L.misc) + 1; }
  __device__ __host__ unsigned long long* dmax() const {
    return reinterpret_cast<unsigned long long*>(b + L.misc + 16);
  }
  __device__ __host__ double* lchol() const { return reinterpret_cast<double*>(b + L.misc + 24); }
};

// e^{V_sigma(s_tau)} at site i in FP64, as the single-CTA path tabulates it
__device__ __forceinline__ double sp_vexp(const ChainDesc& c, int tau, int s, int i) {
  const int k = (tau == 0 || tau == c.Ltau + 1) ? 1 : 0;
  return c.vexp[k][s][c.fields[(long)tau * c.nfld + i] > 0 ? 0 : 1];
}

// ---------------------------------------------------------------------------
// Flips of one block: decisions, then the factors of the block update.

// The current G of a chain: its own buffer (alt = 0) or the second copy.
template <typename T>
__device__ __forceinline__ T* sp_gcur(const ChainDesc& c, int alt, int tsize = (int)sizeof(T)) {
  return alt ? SpBuf<T>(c.spread, c.N, c.ld, c.nmax, tsize).g2() : static_cast<T*>(c.G);
}

// Decisions of block [i0, i0 + kBlock) on the current G (one CTA per chain),
// then M = Gamma (1 + (1 - G_SS) Gamma)^{-1} and the accepted sites.
template <typename T>
__global__ void __launch_bounds__(256) sp_decide_kernel(const ChainDesc* chains, uint64_t seed,
                                                        const uint32_t* sweep_ctr, int tau, int i0, int alt, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (chains[blockIdx.x].st->err) return;
  Cta<T> x = make_cta<T>(chains[blockIdx.x], smem_raw, 0, seed);
  load_state(x);
  const ChainDesc& c = x.c;
  x.Gp = sp_gcur<T>(c, alt);
  decide_sub_block(x, tau, *sweep_ctr, i0, min(kBlock, c.N - i0), 0);
  __syncthreads();
  x.mark(kPhFlip);
  const int a = x.sh.na;
  SpBuf<T> sp(c.spread, c.N, c.ld, c.nmax);
  if (threadIdx.x == 0) *sp.na() = a;
  if (a > 0) {
    FlipBuf<T>& fb = *x.fb;
    block_inverse(x, a, false);
    if ((int)threadIdx.x < a) sp.sites()[threadIdx.x] = fb.gsite[threadIdx.x];
    for (int s = 0; s < 2; ++s) {
      T* Mb = sp.mb(s);
      PQMC_FOR_2D(l, 0, a, m, 0, a) Mb[l * kBlock + m] = fb.Tu[s][l][m];
    }
  }
  x.mark(kPhFlush);
  store_state(x, err);
}

// Block update on one 64 x 64 tile of G per CTA (grid: tiles, spin, chain):
// G_new = G_old - (E_S - G_old[:, S]) M G_old[S, :], G_old the current buffer
// (alt), G_new the other one; a copy when no flip was accepted.
template <typename T>
__global__ void __launch_bounds__(256) sp_flush_kernel(const ChainDesc* chains, int i0, int alt) {
  constexpr int TT = 64;
  __shared__ T Ms[kBlock][kBlock + 1];
  __shared__ T MW[kBlock][TT];
  __shared__ T Ws[kBlock][TT];
  __shared__ T Us[TT][kBlock + 1];
  __shared__ int st[kBlock];
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int N = c.N, ld = c.ld, s = blockIdx.y;
  SpBuf<T> sp(c.spread, N, ld, c.nmax);
  const T* Gin = sp_gcur<T>(c, alt) + (long)s * N * ld;
  T* Gout = sp_gcur<T>(c, alt ^ 1) + (long)s * N * ld;
  const int a = *sp.na();
  const int tn = (N + TT - 1) / TT;
  const int r0 = (blockIdx.x / tn) * TT, c0 = (blockIdx.x % tn) * TT;
  if (r0 >= N) return;
  const int nr = min(TT, N - r0), nc = min(TT, N - c0);
  if (a == 0) {
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
      const long o = (long)(r0 + e / nc) * ld + c0 + e % nc;
      Gout[o] = Gin[o];
    }
    return;
  }
  const T* Mb = sp.mb(s);
  if ((int)threadIdx.x < a) st[threadIdx.x] = sp.sites()[threadIdx.x];
  for (int e = threadIdx.x; e < a * a; e += blockDim.x) Ms[e / a][e % a] = Mb[(e / a) * kBlock + e % a];
  __syncthreads();
  // W = G_old[S, tile columns]; U = E_S - G_old[tile rows, S]
  for (int e = threadIdx.x; e < a * nc; e += blockDim.x) {
    const int l = e / nc, j = e % nc;
    Ws[l][j] = Gin[(long)st[l] * ld + c0 + j];
  }
  for (int e = threadIdx.x; e < a * nr; e += blockDim.x) {
    const int i = e / a, m = e % a;
    Us[i][m] = (r0 + i == st[m] ? T(1) : T(0)) - Gin[(long)(r0 + i) * ld + st[m]];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < a * nc; e += blockDim.x) {
    const int l = e / nc, j = e % nc;
    T v = T(0);
    for (int m = 0; m < a; ++m) v = fma(Ms[l][m], Ws[m][j], v);
    MW[l][j] = v;
  }
  __syncthreads();
  // 4 x 4 outputs per thread, rows and columns interleaved by 16
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = T(0);
  for (int m = 0; m < a; ++m) {
    T u[4], w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) u[r] = Us[ty + 16 * r][m];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = MW[m][tx + 16 * q];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = fma(u[r], w[q], acc[r][q]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = ty + 16 * r, j = tx + 16 * q;
      if (i < nr && j < nc) {
        const long o = (long)(r0 + i) * ld + c0 + j;
        Gout[o] = Gin[o] - acc[r][q];
      }
    }
  (void)i0;
}

// G (both spins) from the second copy back into the chain's own buffer
template <typename T>
__global__ void sp_copy_back_kernel(const ChainDesc* chains) {
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const long n = 2L * c.N * c.ld;
  const T* src = SpBuf<T>(c.spread, c.N, c.ld, c.nmax).g2();
  T* dst = static_cast<T*>(c.G);
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) dst[e] = src[e];
}

// ---------------------------------------------------------------------------
// Diagonal factors of a slice.

// G_s <- e^{V} G_s e^{-V} (dir > 0) or e^{-V} G_s e^{V} (dir < 0), read from
// the current buffer (alt), written to the chain's own
template <typename T>
__global__ void sp_scale_kernel(const ChainDesc* chains, int tau, int dir, int alt) {
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int N = c.N, ld = c.ld, s = blockIdx.y;
  const T* Gin = sp_gcur<T>(c, alt) + (long)s * N * ld;
  T* G = static_cast<T*>(c.G) + (long)s * N * ld;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)N * N; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    const double vi = sp_vexp(c, tau, s, i), vj = sp_vexp(c, tau, s, j);
    const T f = dir > 0 ? (T)vi * (T)(1.0 / vj) : (T)vj * (T)(1.0 / vi);
    G[(long)i * ld + j] = Gin[(long)i * ld + j] * f;
  }
}

// rows of the stack product buffer k: Mt_s <- e^{V(s_tau)} Mt_s
template <typename T>
__global__ void sp_rowscale_kernel(const ChainDesc* chains, int tau, int k) {
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int N = c.N, s = blockIdx.y, n = s == 0 ? c.nup : c.ndn, ldn = c.nmax;
  SpBuf<T> sp(c.spread, N, c.ld, c.nmax);
  T* Mt = sp.mt(s, k);
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)N * n; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), q = (int)(e % n);
    Mt[(long)i * ldn + q] *= (T)sp_vexp(c, tau, s, i);
  }
}

// Start of a stack block: M64 = e^{V(s_tau0)} P (tau0 >= 0, the blocks at the
// ends of the projection), else Mt_s[0] = the previous block in the path
// precision (row-major)
template <typename T>
__global__ void sp_stack_first_kernel(const ChainDesc* chains, int tau0, int left, int b_prev) {
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int N = c.N, s = blockIdx.y, n = s == 0 ? c.nup : c.ndn, ldn = c.nmax;
  SpBuf<T> sp(c.spread, N, c.ld, c.nmax);
  const long stride = (long)gridDim.x * blockDim.x;
  if (tau0 >= 0) {
    const double* P = c.P + (long)s * N * c.nmax;
    double* M = sp.m64(s);
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)N * n; e += stride) {
      const int q = (int)(e / N), i = (int)(e % N);
      M[(long)q * N + i] = sp_vexp(c, tau0, s, i) * P[(long)q * N + i];
    }
  } else {
    const double* prev = (left ? c.Lst : c.Rst) + ((long)b_prev * 2 + s) * N * c.nmax;
    T* Mt = sp.mt(s, 0);
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)N * n; e += stride) {
      const int i = (int)(e / n), q = (int)(e % n);
      Mt[(long)i * ldn + q] = (T)prev[(long)q * N + i];
    }
  }
}

// M64 (column-major) = the product buffer k in FP64
template <typename T>
__global__ void sp_to64_kernel(const ChainDesc* chains, int k) {
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int N = c.N, s = blockIdx.y, n = s == 0 ? c.nup : c.ndn, ldn = c.nmax;
  SpBuf<T> sp(c.spread, N, c.ld, c.nmax);
  const T* Mt = sp.mt(s, k);
  double* M = sp.m64(s);
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)N * n; e += (long)gridDim.x * blockDim.x) {
    const int q = (int)(e / N), i = (int)(e % N);
    M[(long)q * N + i] = (double)Mt[(long)i * ldn + q];
  }
}

// path-precision copies of O^{-1}, Q_R and Q_L for the assembly
template <typename T>
__global__ void sp_cvt_kernel(const ChainDesc* chains, int b) {
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int N = c.N, s = blockIdx.y, n = s == 0 ? c.nup : c.ndn, ldn = c.nmax;
  SpBuf<T> sp(c.spread, N, c.ld, c.nmax);
  const double* QR = c.Rst + ((long)b * 2 + s) * N * c.nmax;
  const double* QL = c.Lst + ((long)b * 2 + s) * N * c.nmax;
  const double* O = sp.o64(s);
  T* xt = sp.xt(s);
  T* qr = sp.qrt(s);
  T* ql = sp.qlt(s);
  const long stride = (long)gridDim.x * blockDim.x;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)N * n; e += stride) {
    qr[e] = (T)QR[e];
    ql[e] = (T)QL[e];
  }
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * n; e += stride) {
    const int i = (int)(e / n), q = (int)(e % n);
    xt[(long)i * ldn + q] = (T)O[(long)i * ldn + q];
  }
}

// Weight of stack block b just factorised (one thread per spin, chain):
// log|det| of the previous block plus log det R (R has a positive diagonal,
// so the sign is the previous block's); a Cholesky breakdown stops the chain.
static __global__ void sp_stack_log_kernel(const ChainDesc* chains, int b, int left, int tsize, int* err) {
  const ChainDesc& c = chains[blockIdx.x];
  const int s = threadIdx.x;
  if (s >= 2 || c.st->err) return;
  const SpBuf<double> sp(c.spread, c.N, c.ld, c.nmax, tsize);
  double* lg = left ? c.Llog : c.Rlog;
  const bool first = left ? b == c.nb : b == 0;
  const int bp = left ? b + 1 : b - 1;
  const double prev_l = first ? 0.0 : lg[(bp * 2 + s) * 2 + 0];
  const double prev_s = first ? 1.0 : lg[(bp * 2 + s) * 2 + 1];
  lg[(b * 2 + s) * 2 + 0] = prev_l + sp.lchol()[s];
  lg[(b * 2 + s) * 2 + 1] = prev_s;
  if (sp.bad()[s]) {
    atomicOr(&c.st->err, kErrStab);
    atomicOr(err, kErrStab);
  }
}

// End of a stabilisation, one CTA per chain: the weight of G from the stack
// blocks' weights and O's pivots,
// the recorded max |G - G_fresh| (flags & kSpRecord), the measurement
// (flags & kSpMeasure), or at initialisation the running sign from the
// weight (flags & kSpInit).
enum : int { kSpMeasure = 1, kSpRecord = 2, kSpInit = 4 };
template <typename T>
__global__ void __launch_bounds__(256) sp_tail_kernel(const ChainDesc* chains, uint64_t seed, int b, int left,
                                                      int flags, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (chains[blockIdx.x].st->err) return;
  Cta<T> x = make_cta<T>(chains[blockIdx.x], smem_raw, 0, seed);
  load_state(x);
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  SpBuf<T> sp(c.spread, c.N, c.ld, c.nmax);
  double sign_total = 1.0;
  for (int s = 0; s < 2; ++s) {
    const int n = x.nsig(s);
    if (threadIdx.x == 0 && sp.bad()[s]) sh.err |= kErrStab;   // a zero Gauss-Jordan pivot
    __syncthreads();
    // row interchanges of the Gauss-Jordan inverse
    int sw = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) sw += sp.perm(s)[j] != j ? 1 : 0;
    const int nsw = (int)cta_sum((double)sw, sh.red);
    double la, sg;
    log_det_of(x, sp.pval(s), n, nsw, la, sg);
    const double l_tot = c.Rlog[(b * 2 + s) * 2 + 0] + la + c.Llog[(b * 2 + s) * 2 + 0];
    const double s_tot = c.Rlog[(b * 2 + s) * 2 + 1] * sg * c.Llog[(b * 2 + s) * 2 + 1];
    if (threadIdx.x == 0) {
      sh.logw_spin[s] = l_tot;
      sh.sign_spin[s] = s_tot;
    }
    sign_total *= s_tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double dmax = __longlong_as_double((long long)*sp.dmax());
    *sp.dmax() = 0ull;
    if (flags & kSpRecord) {
      if (!isfinite(dmax)) sh.err |= kErrNaN;
      sh.dGmax = fmax(sh.dGmax, dmax);
      c.dG[c.st->n_dG % kDGHistory] = dmax;
      c.st->n_dG++;
    }
    if (flags & kSpInit) sh.sign_running = sh.sign_spin[0] * sh.sign_spin[1];
    c.st->sign_stack = sign_total;
  }
  __syncthreads();
  if (flags & kSpMeasure) measure(x);
  store_state(x, err);
}

// ---------------------------------------------------------------------------
// FP64 stabilisation steps, compiled once (spread_f64.cu) for both paths;
// tsize is the path precision's element size.  Grids: (.., spin, chain).

// FP64 tile product over the jobs of g
cudaError_t sp_dgemm(SpGemm& g, int mode, int max_m, int max_n, cudaStream_t st);
// Cholesky factor C = R^T R, panel p: the diagonal block R_PP and its inverse
// (the block row R_{P,rest} = R_PP^{-T} C_{P,rest} and the trailing update
// are sp_dgemm products)
cudaError_t sp_chol_panel(const ChainDesc* d, int nc, int nmax, int p, int tsize, cudaStream_t st);
// Q = M R^{-1} into stack block b
cudaError_t sp_qform(const ChainDesc* d, int nc, int N, int nmax, int left, int b, int tsize, cudaStream_t st);
// Gauss-Jordan panel p of O (pivots, row interchanges, the panel's columns,
// the saved block row), and the interchanges undone on the columns at the end
cudaError_t sp_gj_panel(const ChainDesc* d, int nc, int nmax, int p, int tsize, cudaStream_t st);
cudaError_t sp_gj_unswap(const ChainDesc* d, int nc, int nmax, int tsize, cudaStream_t st);

// ---------------------------------------------------------------------------
// The kernel sequence of one sweep.

template <typename T>
cudaError_t sp_gemm_t(SpGemm& g, int mode, int max_m, int max_n, cudaStream_t st) {
  constexpr int TM = SpTile<T>::TM;
  g.tiles_n = (max_n + TM - 1) / TM;
  const dim3 grid(((max_m + TM - 1) / TM) * g.tiles_n, g.njobs);
  if (grid.x == 0 || g.njobs == 0) return cudaSuccess;
  switch (mode) {
    case kSpStore: sp_gemm_kernel<T, kSpStore><<<grid, 256, 0, st>>>(g); break;
    case kSpSub: sp_gemm_kernel<T, kSpSub><<<grid, 256, 0, st>>>(g); break;
    case kSpFresh: sp_gemm_kernel<T, kSpFresh><<<grid, 256, 0, st>>>(g); break;
    default: sp_gemm_kernel<T, kSpGJUpd><<<grid, 256, 0, st>>>(g); break;
  }
  return cudaGetLastError();
}

// mode 0: an up sweep, 1: a down sweep (measure at the middle slice when
// measure != 0); 2: the initialisation from the chains' fields (the left
// stack, right block 0, G at tau = -1 and the running sign), the same steps
// as the single-CTA initialisation
template <typename T>
cudaError_t spread_sweep_t(const SpreadPlan& P, int mode, int measure, cudaStream_t st) {
  const int nc = P.n, N = P.N, ld = P.ld, ldn = P.nmax, ts = (int)sizeof(T);
  const int nsig[2] = {P.nup, P.ndn};
  const int split = (std::is_same<T, float>::value && P.prec == PQMC_BF16X3) ? 1 : 0;
  const size_t smem_cta = al16(sizeof(Smem<T>)) + flipbuf_bytes(ts);
  const dim3 ew((unsigned)std::min(2048, (N * N + 255) / 256), 2, nc);
  const dim3 ewn((unsigned)std::min(2048, (N * ldn + 255) / 256), 2, nc);
  const ChainDesc* D = P.d_desc;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess;
  };
  auto buf = [&](int c) { return SpBuf<T>(P.ch[c].sp, N, ld, P.nmax); };
  auto Gs = [&](int c, int s) { return static_cast<T*>(P.ch[c].G) + (long)s * N * ld; };
  // the block updates of a slice alternate between the chain's G and its
  // second copy; cur = 1 while the current G is the copy
  int cur = 0;
  auto Gcur = [&](int c, int s) { return (cur ? buf(c).g2() : static_cast<T*>(P.ch[c].G)) + (long)s * N * ld; };
  auto stack_block = [&](int c, bool left, int b, int s) {
    return (left ? P.ch[c].Lst : P.ch[c].Rst) + ((long)b * 2 + s) * N * P.nmax;
  };
  if (nc * 2 > kSpMaxJobs) return cudaErrorInvalidValue;

  auto update = [&](int tau) {
    const int tn = (N + 63) / 64;
    for (int i0 = 0; i0 < N && e == cudaSuccess; i0 += kBlock) {
      sp_decide_kernel<T><<<nc, 256, smem_cta, st>>>(D, P.seed, P.d_sweep, tau, i0, cur, P.d_err);
      ok(cudaSuccess);
      sp_flush_kernel<T><<<dim3(tn * tn, 2, nc), 256, 0, st>>>(D, i0, cur);
      ok(cudaSuccess);
      cur ^= 1;
    }
  };
  auto wrap = [&](int tau, int dir) {
    const bool gz = tau == 0 || tau == P.Ltau + 1;
    // every path through the wrap ends with G in the chain's own buffer
    if (dir > 0 || gz) {
      sp_scale_kernel<T><<<ew, 256, 0, st>>>(D, tau, dir, cur);
      ok(cudaSuccess);
      cur = 0;
    }
    if (!gz) {
      // Gt = E1 G, G = Gt E2: (E1, E2) = (e^{-dtau K}, e^{+dtau K}) up, reversed down;
      // the first factor read transposed, as the single-CTA path reads it
      SpGemm g1{}, g2{};
      g1.split = g2.split = split;
      g1.njobs = g2.njobs = 2 * nc;
      g1.sai = 1; g1.sak = ld; g1.sbk = ld; g1.sbj = 1; g1.sci = ld; g1.scj = 1;
      g2.sai = ld; g2.sak = 1; g2.sbk = ld; g2.sbj = 1; g2.sci = ld; g2.scj = 1;
      for (int c = 0; c < nc; ++c)
        for (int s = 0; s < 2; ++s) {
          const void* E1 = dir > 0 ? P.ch[c].expKm : P.ch[c].expKp;
          const void* E2 = dir > 0 ? P.ch[c].expKp : P.ch[c].expKm;
          g1.job[2 * c + s] = SpJob{E1, Gcur(c, s), buf(c).gt(s), nullptr, nullptr, N, N, N, 0};
          g2.job[2 * c + s] = SpJob{buf(c).gt(s), E2, Gs(c, s), nullptr, nullptr, N, N, N, 0};
        }
      ok(sp_gemm_t<T>(g1, kSpStore, N, N, st));
      ok(sp_gemm_t<T>(g2, kSpStore, N, N, st));
      cur = 0;
      if (dir < 0) {
        sp_scale_kernel<T><<<ew, 256, 0, st>>>(D, tau, -1, 0);
        ok(cudaSuccess);
      }
    }
  };
  // stack block b (right: from block b-1, left: from block b+1) and its QR
  auto stack = [&](int b, bool left) {
    const bool first = left ? b == P.nb : b == 0;
    if (first) {
      sp_stack_first_kernel<T><<<ewn, 256, 0, st>>>(D, left ? P.Ltau + 1 : 0, left ? 1 : 0, 0);
      ok(cudaSuccess);
    } else {
      sp_stack_first_kernel<T><<<ewn, 256, 0, st>>>(D, -1, left ? 1 : 0, left ? b + 1 : b - 1);
      ok(cudaSuccess);
      int cur = 0;
      auto product = [&]() {
        SpGemm g{};
        g.njobs = 2 * nc;
        g.sai = 1; g.sak = ld; g.sbk = ldn; g.sbj = 1; g.sci = ldn; g.scj = 1;
        for (int c = 0; c < nc; ++c)
          for (int s = 0; s < 2; ++s)
            g.job[2 * c + s] = SpJob{P.ch[c].expKm, buf(c).mt(s, cur), buf(c).mt(s, cur ^ 1), nullptr, nullptr, N, nsig[s], N, 0};
        ok(sp_gemm_t<T>(g, kSpStore, N, ldn, st));
        cur ^= 1;
      };
      if (!left) {
        for (int tau = (b - 1) * P.n_stab + 1; tau <= b * P.n_stab; ++tau) {
          sp_rowscale_kernel<T><<<ewn, 256, 0, st>>>(D, tau, cur);
          ok(cudaSuccess);
          product();
        }
      } else {
        for (int tau = (b + 1) * P.n_stab; tau > b * P.n_stab; --tau) {
          product();
          sp_rowscale_kernel<T><<<ewn, 256, 0, st>>>(D, tau, cur);
          ok(cudaSuccess);
        }
      }
      sp_to64_kernel<T><<<ewn, 256, 0, st>>>(D, cur);
      ok(cudaSuccess);
    }
    // Cholesky QR: Gram matrix, blocked factor, Q = M R^{-1}
    {
      SpGemm g{};
      g.njobs = 2 * nc;
      g.sai = N; g.sak = 1; g.sbk = 1; g.sbj = N; g.sci = ldn; g.scj = 1;
      g.upper = 1;   // the factorisation reads the upper triangle only
      for (int c = 0; c < nc; ++c)
        for (int s = 0; s < 2; ++s)
          g.job[2 * c + s] = SpJob{buf(c).m64(s), buf(c).m64(s), buf(c).c64(s), nullptr, nullptr, nsig[s], nsig[s], N, 0};
      ok(sp_dgemm(g, kSpStore, ldn, ldn, st));
    }
    for (int p0 = 0; p0 < ldn && e == cudaSuccess; p0 += kSpPanel) {
      const int p = p0 / kSpPanel;
      ok(sp_chol_panel(D, nc, ldn, p, ts, st));
      {
        // block row in place: R_{P,rest} = R_PP^{-T} C_{P,rest} (a single
        // K slice, so every tile reads its columns before it writes them)
        SpGemm r{};
        r.njobs = 2 * nc;
        r.sai = 1; r.sak = kSpPanel; r.sbk = ldn; r.sbj = 1; r.sci = ldn; r.scj = 1;
        int maxr = 0;
        for (int c = 0; c < nc; ++c)
          for (int s = 0; s < 2; ++s) {
            const int p1 = std::min(p0 + kSpPanel, nsig[s]);
            const int rest = p0 < nsig[s] ? nsig[s] - p1 : 0;
            double* C = buf(c).c64(s);
            r.job[2 * c + s] = SpJob{buf(c).rinv(s) + (long)p * kSpPanel * kSpPanel, C + (long)p0 * ldn + p1,
                                     C + (long)p0 * ldn + p1, nullptr, nullptr, rest > 0 ? p1 - p0 : 0, rest, p1 - p0, 0};
            maxr = std::max(maxr, rest);
          }
        if (maxr > 0) ok(sp_dgemm(r, kSpStore, kSpPanel, maxr, st));
      }
      SpGemm g{};
      g.njobs = 2 * nc;
      g.sai = 1; g.sak = ldn; g.sbk = ldn; g.sbj = 1; g.sci = ldn; g.scj = 1;
      g.upper = 1;
      int maxr = 0;
      for (int c = 0; c < nc; ++c)
        for (int s = 0; s < 2; ++s) {
          const int p1 = std::min(p0 + kSpPanel, nsig[s]);
          const int rest = p0 < nsig[s] ? nsig[s] - p1 : 0;
          double* C = buf(c).c64(s);
          g.job[2 * c + s] = SpJob{C + (long)p0 * ldn + p1, C + (long)p0 * ldn + p1, C + (long)p1 * ldn + p1, nullptr, nullptr,
                                   rest, rest, p1 - p0, 0};
          maxr = std::max(maxr, rest);
        }
      if (maxr > 0) ok(sp_dgemm(g, kSpSub, maxr, maxr, st));
    }
    ok(sp_qform(D, nc, N, ldn, left ? 1 : 0, b, ts, st));
    sp_stack_log_kernel<<<nc, 32, 0, st>>>(D, b, left ? 1 : 0, ts, P.d_err);
    ok(cudaSuccess);
  };
  // G = 1 - Q_R (Q_L^T Q_R)^{-1} Q_L^T at stabilisation point b
  auto refresh = [&](int b, bool left, int flags) {
    {
      SpGemm g{};
      g.njobs = 2 * nc;
      g.sai = N; g.sak = 1; g.sbk = 1; g.sbj = N; g.sci = ldn; g.scj = 1;
      for (int c = 0; c < nc; ++c)
        for (int s = 0; s < 2; ++s)
          g.job[2 * c + s] =
              SpJob{stack_block(c, true, b, s), stack_block(c, false, b, s), buf(c).o64(s), nullptr, nullptr, nsig[s], nsig[s], N, 0};
      ok(sp_dgemm(g, kSpStore, ldn, ldn, st));
    }
    for (int p0 = 0; p0 < ldn && e == cudaSuccess; p0 += kSpGJ) {
      ok(sp_gj_panel(D, nc, ldn, p0 / kSpGJ, ts, st));
      SpGemm g{};
      g.njobs = 2 * nc;
      g.p0 = p0;
      g.sai = ldn; g.sak = 1; g.sbk = ldn; g.sbj = 1; g.sci = ldn; g.scj = 1;
      for (int c = 0; c < nc; ++c)
        for (int s = 0; s < 2; ++s) {
          const int n = nsig[s], p1 = std::min(p0 + kSpGJ, n);
          double* O = buf(c).o64(s);
          g.job[2 * c + s] = SpJob{O + p0, buf(c).tgj(s), O, nullptr, nullptr, p0 < n ? n : 0, n, p1 - p0, p1};
        }
      ok(sp_dgemm(g, kSpGJUpd, ldn, ldn, st));
    }
    ok(sp_gj_unswap(D, nc, ldn, ts, st));
    // assembly in the path precision, max |G - G_fresh|
    SpGemm gy{}, gg{};
    gy.njobs = gg.njobs = 2 * nc;
    gy.sai = ldn; gy.sak = 1; gy.sbk = N; gy.sbj = 1; gy.sci = ld; gy.scj = 1;
    gg.sai = 1; gg.sak = N; gg.sbk = ld; gg.sbj = 1; gg.sci = ld; gg.scj = 1;
    if (!std::is_same<T, double>::value) {
      sp_cvt_kernel<T><<<ewn, 256, 0, st>>>(D, b);
      ok(cudaSuccess);
    }
    for (int c = 0; c < nc; ++c)
      for (int s = 0; s < 2; ++s) {
        const SpBuf<T> B = buf(c);
        const bool f64 = std::is_same<T, double>::value;
        const void* X = f64 ? (const void*)B.o64(s) : (const void*)B.xt(s);
        const void* QL = f64 ? (const void*)stack_block(c, true, b, s) : (const void*)B.qlt(s);
        const void* QR = f64 ? (const void*)stack_block(c, false, b, s) : (const void*)B.qrt(s);
        gy.job[2 * c + s] = SpJob{X, QL, B.y(s), nullptr, nullptr, nsig[s], N, nsig[s], 0};
        gg.job[2 * c + s] = SpJob{QR, B.y(s), Gs(c, s), B.dmax(), Gcur(c, s), N, N, nsig[s], 0};
      }
    ok(sp_gemm_t<T>(gy, kSpStore, ldn, N, st));
    ok(sp_gemm_t<T>(gg, kSpFresh, N, N, st));
    cur = 0;
    sp_tail_kernel<T><<<nc, 256, smem_cta, st>>>(D, P.seed, b, left ? 1 : 0, flags, P.d_err);
    ok(cudaSuccess);
  };

  if (mode == 2) {
    for (int b = P.nb; b >= 0 && e == cudaSuccess; --b) stack(b, true);
    stack(0, false);
    refresh(0, false, kSpInit);
    wrap(0, -1);
  } else if (mode == 0) {
    for (int tau = 0; tau <= P.Ltau + 1 && e == cudaSuccess; ++tau) {
      update(tau);
      wrap(tau, +1);
      if (tau <= P.Ltau && tau % P.n_stab == 0) {
        stack(tau / P.n_stab, false);
        refresh(tau / P.n_stab, false, kSpRecord | ((measure && tau == P.Ltau / 2) ? kSpMeasure : 0));
      }
    }
  } else {
    for (int tau = P.Ltau + 1; tau >= 0 && e == cudaSuccess; --tau) {
      wrap(tau, -1);
      update(tau);
      const int t1 = tau - 1;
      if (t1 >= 0 && t1 % P.n_stab == 0) {
        stack(t1 / P.n_stab, true);
        refresh(t1 / P.n_stab, true, kSpRecord | ((measure && t1 == P.Ltau / 2) ? kSpMeasure : 0));
      }
    }
  }
  if (cur && e == cudaSuccess) {
    sp_copy_back_kernel<T><<<ew, 256, 0, st>>>(D);
    ok(cudaSuccess);
  }
  return e;
}

}  // namespace pqmc

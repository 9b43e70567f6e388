#pragma once
// PQMC sweep kernels for GB300 (sm_103a).
//
// This header holds the device code and the launch templates; each
// sweep_*.cu translation unit instantiates the kernels of one path (FP64,
// reduced precision, reduced precision with dense chain packing) so the three
// compile in parallel, and sweep.cu holds the precision dispatch.
//
// One CTA owns one Markov chain for the whole launch and runs complete
// sweeps: Metropolis flips of the Ising fields with delayed (blocked)
// updates, slice wrapping, QR stabilisation of the B_L / B_R stacks, and the
// measurement at the middle slice.  Chains are independent, so a batch of
// chains of uneven size is one launch with one CTA per chain.
//
// Paper: Method section (PQMC estimator, Eq. (1) HS of the Gutzwiller
// factor) and honeycomb Hubbard section (Eq. (2), trial state of Eq. (3)).
//
// Conventions (shared with the header):
//   slices tau = 0..Ltau+1; 0 and Ltau+1 carry the Gutzwiller fields;
//   B_tau = e^{-dtau K} e^{V(s_tau)} (interaction), e^{V(s_tau)} (Gutzwiller);
//   G(tau) = 1 - B_R(tau) (B_L(tau) B_R(tau))^{-1} B_L(tau),
//   B_R(tau) = B_tau ... B_0 P,  B_L(tau) = P^T B_{Ltau+1} ... B_{tau+1}.
//   A flip of s_{tau,i} is proposed on G(tau-1): R_sigma = 1 + Delta_sigma (1 - G_ii).
//
// Precision: T (double or float) is the path precision of G, the ratios,
// the wrap, the delayed updates, the products that advance the stack blocks
// and the assembly of G from them.  The Householder QR of the stack blocks,
// the product Q_L^T Q_R, its inverse and the log-determinant / sign are FP64
// in every path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pqmc.h"
#include "chain.h"
#include "model.h"
#include "philox.cuh"
#include "tc_gemm.cuh"

namespace pqmc {


// --------------------------------------------------------------------------
// small CTA helpers

static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
static __device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Loop over a 2D index range with warps along rows and lanes along columns
// (no runtime integer division in the element loops).
#define PQMC_FOR_2D(i, i0, i1, j, j0, j1)                                          \
  for (int i = (i0) + (int)(threadIdx.x >> 5); i < (i1); i += (int)(blockDim.x >> 5)) \
    for (int j = (j0) + (int)(threadIdx.x & 31); j < (j1); j += 32)

// Sum / max over the CTA; every thread gets the result.  red holds >= 32 doubles.
static __device__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = lane < nw ? red[lane] : 0.0;
  return warp_sum(t);
}
static __device__ double cta_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = lane < nw ? red[lane] : 0.0;
  return warp_max(t);
}

// --------------------------------------------------------------------------
// CTA-wide register-tiled GEMM: C = A B, A(i,k) = A[i*sai + k*sak],
// B(k,j) = B[k*sbk + j*sbj]; inputs are converted to the accumulation type T
// on load; the epilogue receives (i, j, value).  Every thread owns 4x4
// outputs.  When A is contiguous in i and B in j (sai = sbj = 1, strides and
// pointers 16-byte aligned, same type as T) the operands are read with
// 16-byte vector loads.

struct EpiStore {
  static constexpr bool kRow4 = true;   // supports 4 contiguous outputs of a row at once
  template <typename T, typename TC> __device__ void operator()(TC* C, int sci, int scj, int i, int j, T v) const {
    C[(long)i * sci + (long)j * scj] = (TC)v;
  }
  template <typename T> __device__ void row4(T* c, const T v[4]) const { c[0] = v[0]; c[1] = v[1]; c[2] = v[2]; c[3] = v[3]; }
};
struct EpiSub {
  static constexpr bool kRow4 = true;
  template <typename T, typename TC> __device__ void operator()(TC* C, int sci, int scj, int i, int j, T v) const {
    C[(long)i * sci + (long)j * scj] -= (TC)v;
  }
  template <typename T> __device__ void row4(T* c, const T v[4]) const {
    c[0] -= v[0]; c[1] -= v[1]; c[2] -= v[2]; c[3] -= v[3];
  }
};
template <typename E, typename = void> struct HasRow4 { static constexpr bool value = false; };
template <typename E> struct HasRow4<E, std::void_t<decltype(E::kRow4)>> { static constexpr bool value = E::kRow4; };

template <typename T> struct Vec4;
template <> struct Vec4<float> {
  __device__ static void load(const float* p, float v[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
  static constexpr int kAlign = 4;
};
template <> struct Vec4<double> {
  __device__ static void load(const double* p, double v[4]) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    const double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
  static constexpr int kAlign = 2;
};

template <typename T>
__device__ __forceinline__ bool vec_ok(const T* p, long stride) {
  return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && (stride % Vec4<T>::kAlign == 0);
}

template <typename T, typename TA, typename TB, typename TC, typename Epi>
__device__ void cta_gemm(int M, int Nn, int K, const TA* A, int sai, int sak, const TB* B, int sbk, int sbj,
                         TC* C, int sci, int scj, Epi epi) {
  const int tm = (M + 3) >> 2, tn = (Nn + 3) >> 2;
  bool vec = false, vec_row = false, st_row = false;
  if constexpr (std::is_same<T, TA>::value && std::is_same<T, TB>::value) {
    vec = sai == 1 && sbj == 1 && vec_ok<T>((const T*)A, sak) && vec_ok<T>((const T*)B, sbk) &&
          (M % 4 == 0) && (Nn % 4 == 0);
    // A contiguous along k (row-major): 4 x 4 blocks of A per four k-steps
    vec_row = !vec && sak == 1 && sbj == 1 && vec_ok<T>((const T*)A, sai) && vec_ok<T>((const T*)B, sbk) &&
              (M % 4 == 0) && (Nn % 4 == 0) && (K % 4 == 0);
  }
  if constexpr (std::is_same<T, TC>::value && HasRow4<Epi>::value) {
    st_row = scj == 1 && vec_ok<T>((const T*)C, sci) && (Nn % 4 == 0);
  }
  for (int t = threadIdx.x; t < tm * tn; t += blockDim.x) {
    const int i0 = (t / tn) << 2, j0 = (t % tn) << 2;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = T(0);
    if constexpr (std::is_same<T, TA>::value && std::is_same<T, TB>::value) {
      if (vec) {
        const T* pa = (const T*)A + i0;
        const T* pb = (const T*)B + j0;
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
          T a[4], b[4];
          Vec4<T>::load(pa + (long)k * sak, a);
          Vec4<T>::load(pb + (long)k * sbk, b);
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
        }
      }
    }
    if constexpr (std::is_same<T, TA>::value && std::is_same<T, TB>::value) {
      if (vec_row) {
        const T* pa = (const T*)A + (long)i0 * sai;
        const T* pb = (const T*)B + j0;
        for (int k = 0; k < K; k += 4) {
          T a[4][4], b[4][4];
#pragma unroll
          for (int r = 0; r < 4; ++r) Vec4<T>::load(pa + (long)r * sai + k, a[r]);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) Vec4<T>::load(pb + (long)(k + kk) * sbk, b[kk]);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r][kk], b[kk][q], acc[r][q]);
        }
      }
    }
    if (!vec && !vec_row) {
      for (int k = 0; k < K; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = (i0 + r < M) ? (T)A[(long)(i0 + r) * sai + (long)k * sak] : T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = (j0 + q < Nn) ? (T)B[(long)k * sbk + (long)(j0 + q) * sbj] : T(0);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
      }
    }
    if constexpr (std::is_same<T, TC>::value && HasRow4<Epi>::value) {
      if (st_row) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (i0 + r < M) epi.row4((T*)C + (long)(i0 + r) * sci + j0, acc[r]);
        continue;
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i0 + r < M && j0 + q < Nn) epi(C, sci, scj, i0 + r, j0 + q, acc[r][q]);
  }
}

// --------------------------------------------------------------------------
// Split-precision tensor-core GEMM (the BF16X3 path): C = A B for FP32 A, B
// with every operand split as x = hi + lo, hi = bf16(x), lo = bf16(x - hi),
// and C = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 by
// mma.sync.m16n8k16 (Henry, Tang & Heinecke 2019 use the same split).  Each
// warp owns 16 x 32 output tiles; operands are read with arbitrary strides
// (zero outside the matrix) and split on the fly.

static __device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}

static __device__ __forceinline__ uint32_t pack2(__nv_bfloat16 first, __nv_bfloat16 second) {
  return (uint32_t)__bfloat16_as_ushort(first) | ((uint32_t)__bfloat16_as_ushort(second) << 16);
}

static __device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename Epi>
__device__ void cta_gemm_bf16x3(int M, int Nn, int K, const float* A, int sai, int sak, const float* B, int sbk,
                                int sbj, float* C, int sci, int scj, Epi epi) {
  // each warp owns a 16 x 32 output tile: the A fragment of a k-step is
  // loaded and split once and used by the four 16 x 8 products of the tile
  constexpr int kNs = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int tm = (M + 15) >> 4, tn = (Nn + 8 * kNs - 1) / (8 * kNs);
  auto a_at = [&](int r, int k) -> float { return (r < M && k < K) ? A[(long)r * sai + (long)k * sak] : 0.0f; };
  auto b_at = [&](int k, int n) -> float { return (k < K && n < Nn) ? B[(long)k * sbk + (long)n * sbj] : 0.0f; };
  for (int t = warp; t < tm * tn; t += nw) {
    const int m0 = (t / tn) << 4, n0 = (t % tn) * 8 * kNs;
    const int r0 = m0 + g, r1 = m0 + g + 8;
    const int nsub = min(kNs, (Nn - n0 + 7) >> 3);          // sub-tiles holding columns (warp-uniform)
    float c[kNs][4];
#pragma unroll
    for (int q = 0; q < kNs; ++q) c[q][0] = c[q][1] = c[q][2] = c[q][3] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
      const int k = k0 + 2 * tg;
      const float av[8] = {a_at(r0, k), a_at(r0, k + 1), a_at(r1, k), a_at(r1, k + 1),
                           a_at(r0, k + 8), a_at(r0, k + 9), a_at(r1, k + 8), a_at(r1, k + 9)};
      __nv_bfloat16 ah[8], al[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) split_bf16(av[q], ah[q], al[q]);
      const uint32_t AH[4] = {pack2(ah[0], ah[1]), pack2(ah[2], ah[3]), pack2(ah[4], ah[5]), pack2(ah[6], ah[7])};
      const uint32_t AL[4] = {pack2(al[0], al[1]), pack2(al[2], al[3]), pack2(al[4], al[5]), pack2(al[6], al[7])};
#pragma unroll
      for (int q = 0; q < kNs; ++q) {
        if (q < nsub) {
          const int nn = n0 + 8 * q + g;
          const float bv[4] = {b_at(k, nn), b_at(k + 1, nn), b_at(k + 8, nn), b_at(k + 9, nn)};
          __nv_bfloat16 bh[4], bl[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) split_bf16(bv[u], bh[u], bl[u]);
          const uint32_t BH[2] = {pack2(bh[0], bh[1]), pack2(bh[2], bh[3])};
          const uint32_t BL[2] = {pack2(bl[0], bl[1]), pack2(bl[2], bl[3])};
          mma_bf16(c[q], AH, BL);
          mma_bf16(c[q], AL, BH);
          mma_bf16(c[q], AH, BH);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kNs; ++q) {
      if (q < nsub) {
        const int cc = n0 + 8 * q + 2 * tg;
        if (r0 < M) {
          if (cc < Nn) epi(C, sci, scj, r0, cc, c[q][0]);
          if (cc + 1 < Nn) epi(C, sci, scj, r0, cc + 1, c[q][1]);
        }
        if (r1 < M) {
          if (cc < Nn) epi(C, sci, scj, r1, cc, c[q][2]);
          if (cc + 1 < Nn) epi(C, sci, scj, r1, cc + 1, c[q][3]);
        }
      }
    }
  }
}

// --------------------------------------------------------------------------
// shared memory of one chain CTA

// Buffers of one flip block (lives in shared memory, see make_cta).
template <typename T>
struct FlipBuf {
  T Tu[2][kBlock][kBlock + 1];      // t-V: 1 + (1 - G_SS) Gamma, inverted in place, then M
  T rs[2][kBlock];                  // ratio R_sigma of each proposal of the decision sub-block
  T cl[2][kMaxDelay];               // Delta of each accepted flip of the delayed block (diagonal of Gamma)
  T fr[2][kMaxDelay];               // Delta / R_sigma of each accepted flip
  int sites[kMaxDelay];             // (unused slot kept for the layout)
  int gsite[kMaxDelay];             // site of each accepted flip
};
static_assert(sizeof(FlipBuf<double>) <= flipbuf_bytes(8) && sizeof(FlipBuf<float>) <= flipbuf_bytes(4),
              "flip buffer layout");

template <typename T>
struct Smem {
  ChainDesc desc;                   // this chain's descriptor, copied in at launch
  double red[32];                   // reduction scratch
  // e^{V_sigma} of one site as a function of m = the staged value fr[i]
  // (a site field +-1, or for t-V the signed sum of the site's bond fields,
  // -3..3): [Gutzwiller?][spin][m + 3]; unused entries are 1
  double vtab[2][2][7];
  T vt[2][2][7];                    // the same in the path precision
  T vti[2][2][7];                   // and its inverse
  long long cyc[kPhases];           // per-phase clock cycles (thread 0)
  long long t_mark;
  signed char fr[kMaxN];            // fields of the staged slice
  int na;                           // accepted flips in the block
  int piv;
  int nswap[2];
  int chol_bad;
  int fperm[kBlock];                // row interchanges of the flush inverse (t-V)
  int staged;                       // slice held in fr, or -1
  double sign_running;
  double sign_spin[2];
  double logw_spin[2];
  double dGmax;
  long long n_prop, n_acc, acc_pos;
  int err;
};

// One chain CTA: its descriptor, shared memory, and where G and the phase
// scratch live (shared memory when they fit, else the chain's global buffers).
template <typename T>
struct Cta {
  const ChainDesc& c;
  Smem<T>& sh;
  uint64_t seed;
  T* Gp;
  unsigned char* scr;
  ScratchLayout L;
  bool resident;
  FlipBuf<T>* fb;
  unsigned char* tcs = nullptr;     // tensor-core staging area (BF16X3, chains in global memory), or null
  uint32_t tmem = 0;                // its TMEM accumulator
  __device__ T* G(int s) const { return Gp + (long)s * c.N * c.ld; }
  __device__ T* Gt() const { return reinterpret_cast<T*>(scr + L.gt); }
  __device__ T* Ub() const { return reinterpret_cast<T*>(scr + L.u); }
  __device__ T* Wb() const { return reinterpret_cast<T*>(scr + L.w); }
  __device__ double* M64() const { return reinterpret_cast<double*>(scr + L.m64); }
  __device__ double* Q64() const { return reinterpret_cast<double*>(scr + L.mtq); }
  __device__ T* Mt() const { return reinterpret_cast<T*>(scr + L.mtq); }
  __device__ T* Mt2() const { return reinterpret_cast<T*>(scr + L.mt2); }
  __device__ double* qbeta() const { return reinterpret_cast<double*>(scr + L.qaux); }
  __device__ double* qalpha() const { return qbeta() + c.nmax; }
  __device__ double* qw() const { return qbeta() + 2 * c.nmax; }
  __device__ double* qpart() const { return qbeta() + 3 * c.nmax; }
  __device__ double* chol() const { return reinterpret_cast<double*>(scr + L.chol); }
  __device__ double* Ob(int s) const {
    return reinterpret_cast<double*>(scr + L.o + s * al16((size_t)c.nmax * c.nmax * 8));
  }
  __device__ T* Yb() const { return reinterpret_cast<T*>(scr + L.y); }
  __device__ T* QRt() const { return reinterpret_cast<T*>(scr + L.qrt); }
  __device__ T* QLt() const { return reinterpret_cast<T*>(scr + L.qlt); }
  __device__ T* Ot() const { return reinterpret_cast<T*>(scr + L.ot); }
  __device__ double* pval(int s) const { return reinterpret_cast<double*>(scr + L.laux) + s * 3 * c.nmax; }
  __device__ double* pinv(int s) const { return pval(s) + c.nmax; }
  __device__ double* lmul(int s) const { return pval(s) + 2 * c.nmax; }
  __device__ const T* Em() const { return reinterpret_cast<const T*>(c.expKm); }
  __device__ const T* Ep() const { return reinterpret_cast<const T*>(c.expKp); }
  __device__ int nsig(int s) const { return s == 0 ? c.nup : c.ndn; }
  __device__ bool gutz(int tau) const { return tau == 0 || tau == c.Ltau + 1; }
  // fermion species carried by the chain: both spins, or one (t-V)
  __device__ int nspec() const { return c.tv ? 1 : 2; }
  // stage slice tau into shared memory (collective): the site fields, or for
  // t-V the sum m_i of the site's three bond fields (+ at A ends, - at B ends)
  __device__ void stage(int tau) {
    __syncthreads();
    const int8_t* f = c.fields + (long)tau * c.nfld;
    if (c.tv) {
      for (int i = threadIdx.x; i < c.N; i += blockDim.x) {
        const int* sb = c.site_bonds + 3 * i;
        const int m = (int)f[sb[0]] + (int)f[sb[1]] + (int)f[sb[2]];
        sh.fr[i] = (signed char)((i & 1) ? -m : m);
      }
    } else {
      for (int i = threadIdx.x; i < c.N; i += blockDim.x) sh.fr[i] = f[i];
    }
    if (threadIdx.x == 0) sh.staged = tau;
    __syncthreads();
  }
  // diagonal of e^{V_sigma(s_tau)} at site i for the staged slice tau
  __device__ double vexp(int tau, int s, int i) const { return sh.vtab[gutz(tau) ? 1 : 0][s][sh.fr[i] + 3]; }
  __device__ T vexpT(int tau, int s, int i) const { return sh.vt[gutz(tau) ? 1 : 0][s][sh.fr[i] + 3]; }
  __device__ T vinvT(int tau, int s, int i) const { return sh.vti[gutz(tau) ? 1 : 0][s][sh.fr[i] + 3]; }
  // charge the cycles since the last mark to phase ph (thread 0 only)
  __device__ void mark(int ph) {
    if (threadIdx.x == 0) {
      const long long t = clock64();
      sh.cyc[ph] += t - sh.t_mark;
      sh.t_mark = t;
    }
  }
};

// Path GEMM of the wrap (deep = true, K = N) and of the delayed update
// (deep = false, K = accepted flips of a block).  On the BF16X3 path the
// wrap runs as split-precision tensor-core products: tcgen05 MMAs into tensor
// memory when the CTA holds a staging area for them (a chain kept in global
// memory on a 512-thread CTA), mma.sync otherwise.  The delayed update is a
// rank-a correction (a <= 64) whose cost is reading and writing G: it runs
// in FP32 on the CUDA cores on the BF16X3 path too (measured faster than
// either tensor-core form at 162-648 sites, and exact to FP32).  FP32 and
// FP64 paths: CUDA-core FMA.
template <typename T, typename Epi>
__device__ void path_gemm(Cta<T>& x, bool deep, int M, int Nn, int K, const T* A, int sai, int sak, const T* B,
                          int sbk, int sbj, T* C, int sci, int scj, Epi epi) {
  if constexpr (std::is_same<T, float>::value) {
    if (x.c.tc && deep) {
      if (x.tcs) {
        cta_gemm_tc(M, Nn, K, A, sai, sak, B, sbk, sbj, C, sci, scj, epi, x.tcs, x.tmem, &x.sh.err, kErrTimeout);
        __syncthreads();
      } else {
        cta_gemm_bf16x3(M, Nn, K, A, sai, sak, B, sbk, sbj, C, sci, scj, epi);
      }
      return;
    }
  }
  cta_gemm<T>(M, Nn, K, A, sai, sak, B, sbk, sbj, C, sci, scj, epi);
}

// --------------------------------------------------------------------------
// Metropolis updates of one slice with delayed updates in blocks of kBlock
// sites.  Inside a block one warp (lane = column of the block) proposes the
// flips in order on the kBlock x kBlock diagonal block of G.  Later proposals
// read only rows and columns of later sites, so an accepted flip at j updates
// just that future part: G_rq += c G_rj G_jq (r, q > j), c = Delta/R_sigma.
// After the block the whole CTA applies the accepted set S at once:
//     G <- G - (E_S - G_{:,S}) M G_{S,:},  M = Gamma (1 + (1 - G_SS) Gamma)^{-1},
// G the G of the block start, Gamma = diag(Delta) of the accepted flips.  This
// equals the sequence of Sherman-Morrison updates because the new G depends
// only on the new fields; the pivots of the a x a inverse are the accepted
// ratios, so Gauss-Jordan without pivoting follows the sequential process.

// The Metropolis uniform u = m 2^-53 of the 53-bit Philox mantissa m, in the
// decision precision: exact in FP64; in FP32 rounded down to 24 bits, so
// u < |R| is decided in FP32 on both sides of a comparison with the oracle.
template <typename T>
__device__ __forceinline__ T uniform_of(uint64_t m53) {
  if constexpr (std::is_same<T, double>::value) return (double)m53 * 0x1.0p-53;
  else return (float)(uint32_t)(m53 >> 29) * 0x1.0p-24f;
}

// Applies the a accepted flips of a block, recorded in fb (global sites
// gsite, Delta per species cl), to the whole G of every species:
//     G <- G - (E_S - G_{:,S}) Gamma (1 + (1 - G_SS) Gamma)^{-1} G_{S,:}
// with G the G of the block start.  X = 1 + (1 - G_SS) Gamma is inverted in
// place by one warp per species; Hubbard blocks need no pivoting (its pivots
// are the accepted ratios), the bond blocks of the t-V model pivot on rows
// (a single end of an accepted bond may have a vanishing ratio).
// M = Gamma (1 + (1 - G_SS) Gamma)^{-1} of the a accepted flips of a block
// into fb.Tu[s] for every species s (collective; G is the G of the block
// start).
template <typename T>
__device__ void block_inverse(Cta<T>& x, int a, bool pivot) {
  FlipBuf<T>& fb = *x.fb;
  const int ld = x.c.ld, ns = x.nspec();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  PQMC_FOR_2D(sl, 0, ns * a, m, 0, a) {
    const int s = sl >= a ? 1 : 0, l = sl - s * a;
    const T g = x.G(s)[(long)fb.gsite[l] * ld + fb.gsite[m]];
    fb.Tu[s][l][m] = ((l == m) ? T(1) : T(0)) + ((l == m ? T(1) : T(0)) - g) * fb.cl[s][m];
  }
  __syncthreads();
  if (warp < ns) {
    const int s = warp;
    T (*X)[kBlock + 1] = fb.Tu[s];
    int* perm = x.sh.fperm;
    for (int p = 0; p < a; ++p) {
      if (pivot) {
        // largest |X_rp|, r >= p, ties to the lower row; swap rows r and p
        T best = T(-1);
        int bi = p;
        if (lane >= p && lane < a) { best = fabs(X[lane][p]); bi = lane; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) perm[p] = bi;
        if (bi != p && lane < a) {
          const T t = X[p][lane];
          X[p][lane] = X[bi][lane];
          X[bi][lane] = t;
        }
        __syncwarp();
      }
      const T ip = T(1) / X[p][p];
      const T xpl = lane < a ? X[p][lane] : T(0);
      if (lane < a && lane != p)
        for (int r = 0; r < a; ++r)
          if (r != p) X[r][lane] = fma(-X[r][p] * ip, xpl, X[r][lane]);
      __syncwarp();
      if (lane < a) {
        if (lane != p) X[p][lane] = xpl * ip;
        X[lane][p] = lane == p ? ip : -X[lane][p] * ip;
      }
      __syncwarp();
    }
    if (pivot) {
      // the row interchanges of the factorisation become column
      // interchanges of the inverse, undone last step first
      for (int p = a - 1; p >= 0; --p) {
        const int q = perm[p];
        if (q != p && lane < a) {
          const T t = X[lane][p];
          X[lane][p] = X[lane][q];
          X[lane][q] = t;
        }
        __syncwarp();
      }
    }
    for (int l = 0; l < a; ++l)
      if (lane < a) X[l][lane] *= fb.cl[s][l];
  }
  __syncthreads();
}

template <typename T>
__device__ void flush_block(Cta<T>& x, int a, bool pivot) {
  const ChainDesc& c = x.c;
  FlipBuf<T>& fb = *x.fb;
  const int N = c.N, ld = c.ld, ns = x.nspec();
  T* Ubuf = x.Ub();                                    // kBlock x N  (U column-major, ld N)
  T* Wbuf = x.Wb();                                    // kBlock x ld (rows G_{S,:})
  block_inverse(x, a, pivot);
  // per species: A_S = E_S - G_{:,S} (N x a, column-major) and W = G_{S,:}
  // (a x N) gathered before G changes, then MW = M W and G -= A_S MW
  T* MW = reinterpret_cast<T*>(x.scr + x.L.mw);
  for (int s = 0; s < ns; ++s) {
    T* Gs = x.G(s);
    PQMC_FOR_2D(m, 0, a, i, 0, N) {
      const int col = fb.gsite[m];
      Ubuf[(long)m * N + i] = (i == col ? T(1) : T(0)) - Gs[(long)i * ld + col];
    }
    PQMC_FOR_2D(l, 0, a, q, 0, N) Wbuf[(long)l * ld + q] = Gs[(long)fb.gsite[l] * ld + q];
    __syncthreads();
    cta_gemm<T>(a, N, a, &fb.Tu[s][0][0], kBlock + 1, 1, Wbuf, ld, 1, MW, ld, 1, EpiStore());
    __syncthreads();
    path_gemm<T>(x, false, N, N, a, Ubuf, 1, N, MW, ld, 1, Gs, ld, 1, EpiSub());
    __syncthreads();
  }
  x.mark(kPhFlush);
}

// The accepted flips of a Hubbard delayed block, applied to G as the chain of
// rank-1 updates they stand for, in acceptance order (the update of one
// flip at site i with G the G just before it):
//     G <- G - (e_i - G_{:,i}) (Delta_i / R_i) G_{i,:}.
// Written as G <- G - U V over the block: column m of U and row m of V are
// the vectors of flip m, obtained from the block-start G and the earlier
// vectors (c = G_{:,s_m} - U V_{:,s_m}, r = G_{s_m,:} - U_{s_m,:} V), one
// step per flip for the two spins at once (half of the CTA each)
// (sm_vectors, for flips m0..m1-1 once their decisions are taken), then one
// rank-a product per spin (apply_vectors).  Same result as the block form of
// flush_block, without the a x a inverse.
template <typename T>
__device__ void sm_vectors(Cta<T>& x, int m0, int m1) {
  const ChainDesc& c = x.c;
  FlipBuf<T>& fb = *x.fb;
  const int N = c.N, ld = c.ld;
  const int half = (int)blockDim.x >> 1;
  const int s = (int)threadIdx.x >= half ? 1 : 0;
  const int t = (int)threadIdx.x - s * half;
  T* Us[2] = {reinterpret_cast<T*>(x.scr + x.L.u), reinterpret_cast<T*>(x.scr + x.L.u2)};
  T* Vs[2] = {reinterpret_cast<T*>(x.scr + x.L.w), reinterpret_cast<T*>(x.scr + x.L.mw)};
  {
    const T* Gs = x.G(s);
    T* U = Us[s];
    T* V = Vs[s];
    for (int m = m0; m < m1; ++m) {
      const int sm = fb.gsite[m];
      const T f = fb.fr[s][m];
      for (int o = t; o < 2 * N; o += half) {
        if (o < N) {
          T cv = Gs[(long)o * ld + sm];
          for (int l = 0; l < m; ++l) cv = fma(-U[(long)l * N + o], V[(long)l * ld + sm], cv);
          U[(long)m * N + o] = ((o == sm ? T(1) : T(0)) - cv) * f;
        } else {
          const int j = o - N;
          T rv = Gs[(long)sm * ld + j];
          for (int l = 0; l < m; ++l) rv = fma(-U[(long)l * N + sm], V[(long)l * ld + j], rv);
          V[(long)m * ld + j] = rv;
        }
      }
      // the two halves step independently: one named barrier per spin
      if (s == 0) asm volatile("bar.sync 2, %0;" ::"r"(half) : "memory");
      else asm volatile("bar.sync 3, %0;" ::"r"(half) : "memory");
    }
  }
  __syncthreads();
  x.mark(kPhFlushVec);
}

template <typename T>
__device__ void apply_vectors(Cta<T>& x, int a) {
  const ChainDesc& c = x.c;
  const int N = c.N, ld = c.ld;
  T* Us[2] = {reinterpret_cast<T*>(x.scr + x.L.u), reinterpret_cast<T*>(x.scr + x.L.u2)};
  T* Vs[2] = {reinterpret_cast<T*>(x.scr + x.L.w), reinterpret_cast<T*>(x.scr + x.L.mw)};
  for (int sp = 0; sp < 2; ++sp)
    path_gemm<T>(x, false, N, N, a, Us[sp], 1, N, Vs[sp], ld, 1, x.G(sp), ld, 1, EpiSub());
  __syncthreads();
  x.mark(kPhFlush);
}

// Hubbard slice: delayed blocks of c.kb sites (8, 16, 32 or 64), each
// decided in sub-blocks of up to kBlock sites (one warp per spin) and then
// applied to G at once.  Within a delayed block a later sub-block reads its
// diagonal block of G corrected by the update vectors of the flips already
// accepted, G_SS - U_S V_S, so every decision sees the current G.
// The proposals of one decision sub-block, sites i0 .. i0 + nbk - 1 of slice
// tau (nbk <= kBlock), after a_done flips of the delayed block were accepted
// (their update vectors in the scratch correct the diagonal block read from
// G): warps 0 and 1 decide; sh.na receives the accepted count of the delayed
// block, fb the accepted sites and their Delta, Delta / R.
template <typename T>
__device__ void decide_sub_block(Cta<T>& x, int tau, uint32_t sweep, int i0, int nbk, int a_done) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  FlipBuf<T>& fb = *x.fb;
  const int N = c.N, ld = c.ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kap = x.gutz(tau) ? 1 : 0;
  int8_t* f = c.fields + (long)tau * c.nfld;
  const T dl[2][2] = {{(T)c.delta[kap][0][0], (T)c.delta[kap][0][1]}, {(T)c.delta[kap][1][0], (T)c.delta[kap][1][1]}};
  if (warp < 2) {
    // warp s (spin s): lane q holds column q of the spin's diagonal block in
    // registers; the two warps exchange the spin ratios through shared
    // memory once per proposal and take the same decision
    const int s = warp;
    T gs[kBlock];
    const bool colq = lane < nbk;
#pragma unroll
    for (int r = 0; r < kBlock; ++r) gs[r] = (colq && r < nbk) ? x.G(s)[(long)(i0 + r) * ld + i0 + lane] : T(0);
    if (a_done > 0 && colq) {
      // G_SS - U_S V_S over the vectors of the block's earlier flips
      const T* U = reinterpret_cast<const T*>(x.scr + (s == 0 ? x.L.u : x.L.u2));
      const T* V = reinterpret_cast<const T*>(x.scr + (s == 0 ? x.L.w : x.L.mw));
      for (int l = 0; l < a_done; ++l) {
        const T vq = V[(long)l * ld + i0 + lane];
#pragma unroll
        for (int r = 0; r < kBlock; ++r)
          if (r < nbk) gs[r] = fma(-U[(long)l * N + i0 + r], vq, gs[r]);
      }
    }
    // lane j: uniform (in the decision precision) and field of site i0 + j
    T uj = T(2);
    int flj = 1;
    if (colq) {
      const U4 w = philox4x32_10((uint32_t)(i0 + lane), (uint32_t)tau, sweep, c.chain_index, (uint32_t)x.seed,
                                 (uint32_t)(x.seed >> 32));
      uj = uniform_of<T>(((uint64_t)w.x0 << 21) | (uint64_t)(w.x1 >> 11));
      flj = (int)f[i0 + lane];
    }
    int a = a_done, bad = 0, nneg = 0;
    const long long pos0 = sh.acc_pos;
#pragma unroll
    for (int j = 0; j < kBlock; ++j) {
      if (j < nbk) {
        const int si = __shfl_sync(0xffffffffu, flj, j) > 0 ? 0 : 1;
        const T ds = dl[s][si];
        const T rs = T(1) + ds * (T(1) - __shfl_sync(0xffffffffu, gs[j], j));
        if (lane == 0) fb.rs[s][j] = rs;
        asm volatile("bar.sync 1, 64;" ::: "memory");
        const T R = fb.rs[0][j] * fb.rs[1][j];
        const bool acc = __shfl_sync(0xffffffffu, (int)(uj < (R < T(0) ? -R : R)), j) != 0;
        if (s == 0 && lane == 0) {
          if (!isfinite(R)) bad = 1;
          if (pos0 + j < c.acc_cap) c.acc_log[pos0 + j] = acc ? 1 : 0;
        }
        if (acc) {
          // G_rq += c G_rj G_jq for future rows r > j and columns q > j
          const T y = lane > j ? (ds / rs) * gs[j] : T(0);
#pragma unroll
          for (int r = j + 1; r < kBlock; ++r) gs[r] = fma(__shfl_sync(0xffffffffu, gs[r], j), y, gs[r]);
          if (lane == j) {
            flj = -flj;
            if (s == 0) f[i0 + j] = (int8_t)flj;
          }
          if (lane == 0) fb.fr[s][a] = ds / rs;
          if (s == 0 && lane == 0) {
            fb.gsite[a] = i0 + j;
            fb.cl[0][a] = ds;
            fb.cl[1][a] = dl[1][si];
            nneg += R < T(0) ? 1 : 0;
          }
          ++a;
        }
      }
    }
    if (s == 0 && lane == 0) {
      sh.na = a;
      sh.acc_pos = pos0 + nbk;
      sh.n_prop += nbk;
      sh.n_acc += a - a_done;
      if (nneg & 1) sh.sign_running = -sh.sign_running;
      if (bad) sh.err |= kErrNaN;
    }
  }
}

template <typename T>
__device__ void update_slice(Cta<T>& x, int tau, uint32_t sweep) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  const int N = c.N;
  const int kd = c.kb;
  const int sub = kd < kBlock ? kd : kBlock;

  for (int d0 = 0; d0 < N; d0 += kd) {
    const int d1 = min(d0 + kd, N);
    int a_done = 0;                                  // flips of the delayed block already accepted
    for (int i0 = d0; i0 < d1; i0 += sub) {
      const int nbk = min(sub, d1 - i0);
      decide_sub_block(x, tau, sweep, i0, nbk, a_done);
      __syncthreads();
      x.mark(kPhFlip);
      const int a = sh.na;
      if (a > a_done) sm_vectors(x, a_done, a);
      a_done = a;
    }
    if (a_done > 0) apply_vectors(x, a_done);
  }
}

// Metropolis updates of one slice of the spinless t-V model: the bonds in
// blocks of 16 of one class (a class is a perfect matching, so a block
// touches 32 distinct sites W).  Warp 0 holds G_WW in registers, lane q the
// column of site W[q] (pair p = bond p of the block: A end in lane 2p, B end
// in lane 2p+1); lane p draws the uniform of bond p.  Bond p's flip changes
// V at its two ends by Gamma = diag(Delta_A, Delta_B) and is accepted with
// R = det(1 + Gamma (1 - G_SS)); an accepted flip updates the rows and
// columns of the later pairs by the rank-2 form
//     G_rq <- G_rq + sum_{s in S} G_rs (M G_{S,q})_s,  M = Gamma (1 + (1 - G_SS) Gamma)^{-1}.
// The accepted ends then go to flush_block as one set.
template <typename T>
__device__ void update_slice_tv(Cta<T>& x, int tau, uint32_t sweep) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  FlipBuf<T>& fb = *x.fb;
  const int ld = c.ld, nc = c.N / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kap = x.gutz(tau) ? 1 : 0;
  int8_t* f = c.fields + (long)tau * c.nfld;
  // Delta at the A end (coupled like spin up) and at the B end, field +1 / -1
  const T dA[2] = {(T)c.delta[kap][0][0], (T)c.delta[kap][0][1]};
  const T dB[2] = {(T)c.delta[kap][1][0], (T)c.delta[kap][1][1]};
  constexpr int kPairs = kBlock / 2;
  for (int k = 0; k < 3; ++k) {
    for (int c0 = 0; c0 < nc; c0 += kPairs) {
      const int np = min(kPairs, nc - c0);
      if (warp == 0) {
        const bool on = (lane >> 1) < np;
        const int wq = on ? c.bond_ends[2 * (3 * (c0 + (lane >> 1)) + k) + (lane & 1)] : 0;
        T g[kBlock];
        const T* G0 = x.G(0);
#pragma unroll
        for (int r = 0; r < kBlock; ++r) {
          const int wr = __shfl_sync(0xffffffffu, wq, r);
          g[r] = (on && (r >> 1) < np) ? G0[(long)wr * ld + wq] : T(0);
        }
        T up = T(2);
        int fp = 1;
        if (lane < np) {
          const int b = 3 * (c0 + lane) + k;
          const U4 w = philox4x32_10((uint32_t)b, (uint32_t)tau, sweep, c.chain_index, (uint32_t)x.seed,
                                     (uint32_t)(x.seed >> 32));
          up = uniform_of<T>(((uint64_t)w.x0 << 21) | (uint64_t)(w.x1 >> 11));
          fp = (int)f[b];
        }
        int a = 0, bad = 0, nneg = 0;
        const long long pos0 = sh.acc_pos;
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
          if (p < np) {
            const int si = __shfl_sync(0xffffffffu, fp, p) > 0 ? 0 : 1;
            const T di = dA[si], dj = dB[si];
            const T gii = __shfl_sync(0xffffffffu, g[2 * p], 2 * p);
            const T gjj = __shfl_sync(0xffffffffu, g[2 * p + 1], 2 * p + 1);
            const T gij = __shfl_sync(0xffffffffu, g[2 * p], 2 * p + 1);
            const T gji = __shfl_sync(0xffffffffu, g[2 * p + 1], 2 * p);
            // R = det(1 + Gamma (1 - G_SS))
            const T m00 = T(1) + di * (T(1) - gii), m01 = -di * gij;
            const T m10 = -dj * gji, m11 = T(1) + dj * (T(1) - gjj);
            const T R = m00 * m11 - m01 * m10;
            const bool acc = __shfl_sync(0xffffffffu, (int)(up < (R < T(0) ? -R : R)), p) != 0;
            if (lane == 0) {
              if (!isfinite(R)) bad = 1;
              if (pos0 + p < c.acc_cap) c.acc_log[pos0 + p] = acc ? 1 : 0;
            }
            if (acc) {
              // X = 1 + (1 - G_SS) Gamma, M = Gamma X^{-1}
              const T x00 = T(1) + (T(1) - gii) * di, x01 = -gij * dj;
              const T x10 = -gji * di, x11 = T(1) + (T(1) - gjj) * dj;
              const T inv = T(1) / (x00 * x11 - x01 * x10);
              const T M00 = di * (x11 * inv), M01 = di * (-x01 * inv);
              const T M10 = dj * (-x10 * inv), M11 = dj * (x00 * inv);
              const bool fut = lane >= 2 * p + 2;
              const T y0 = fut ? M00 * g[2 * p] + M01 * g[2 * p + 1] : T(0);
              const T y1 = fut ? M10 * g[2 * p] + M11 * g[2 * p + 1] : T(0);
#pragma unroll
              for (int r = 2 * p + 2; r < kBlock; ++r) {
                const T gri = __shfl_sync(0xffffffffu, g[r], 2 * p);
                const T grj = __shfl_sync(0xffffffffu, g[r], 2 * p + 1);
                g[r] = fma(gri, y0, fma(grj, y1, g[r]));
              }
              if (lane == p) {
                fp = -fp;
                f[3 * (c0 + p) + k] = (int8_t)fp;
              }
              const int wi = __shfl_sync(0xffffffffu, wq, 2 * p), wj = __shfl_sync(0xffffffffu, wq, 2 * p + 1);
              if (lane == 0) {
                fb.gsite[a] = wi;
                fb.cl[0][a] = di;
                fb.gsite[a + 1] = wj;
                fb.cl[0][a + 1] = dj;
                nneg += R < T(0) ? 1 : 0;
              }
              a += 2;
            }
          }
        }
        if (lane == 0) {
          sh.na = a;
          sh.acc_pos = pos0 + np;
          sh.n_prop += np;
          sh.n_acc += a / 2;
          if (nneg & 1) sh.sign_running = -sh.sign_running;
          if (bad) sh.err |= kErrNaN;
        }
      }
      __syncthreads();
      x.mark(kPhFlip);
      const int a = sh.na;
      if (a == 0) continue;
      flush_block(x, a, true);
    }
  }
}

// --------------------------------------------------------------------------
// Slice wrapping.  dir = +1: G(tau) = B_tau G(tau-1) B_tau^{-1};
// dir = -1: G(tau-1) = B_tau^{-1} G(tau) B_tau.

template <typename T>
__device__ void wrap(Cta<T>& x, int tau, int dir) {
  const ChainDesc& c = x.c;
  const int N = c.N, ld = c.ld;
  const bool gz = x.gutz(tau);
  T* Gt = x.Gt();
  const T* Em = x.Em();
  const T* Ep = x.Ep();
  if (!gz && x.resident && x.L.em) {
    // a chain resident in shared memory reads e^{-+dtau K} there: the two
    // tables are copied in from the L2-resident copy shared by all chains
    // (the wrap phase leaves room for them in the scratch)
    const int chunks = N * ld * (int)sizeof(T) / 16;
    int4* dm = reinterpret_cast<int4*>(x.scr + x.L.em);
    int4* dp = reinterpret_cast<int4*>(x.scr + x.L.ep);
    const int4* sm = reinterpret_cast<const int4*>(Em);
    const int4* sp = reinterpret_cast<const int4*>(Ep);
    for (int e = threadIdx.x; e < chunks; e += blockDim.x) {
      dm[e] = sm[e];
      dp[e] = sp[e];
    }
    Em = reinterpret_cast<const T*>(dm);
    Ep = reinterpret_cast<const T*>(dp);
    __syncthreads();
  }
  x.stage(tau);
  if (dir > 0) {
    for (int s = 0; s < x.nspec(); ++s) {
      T* Gs = x.G(s);
      PQMC_FOR_2D(i, 0, N, j, 0, N) Gs[(long)i * ld + j] *= x.vexpT(tau, s, i) * x.vinvT(tau, s, j);
    }
    __syncthreads();
    if (gz) return;
    // Gt = e^{-dtau K} G, G = Gt e^{+dtau K}
    for (int s = 0; s < x.nspec(); ++s) {
      path_gemm<T>(x, true, N, N, N, Em, 1, ld, x.G(s), ld, 1, Gt, ld, 1, EpiStore());
      __syncthreads();
      path_gemm<T>(x, true, N, N, N, Gt, ld, 1, Ep, ld, 1, x.G(s), ld, 1, EpiStore());
      __syncthreads();
    }
  } else {
    if (!gz) {
      for (int s = 0; s < x.nspec(); ++s) {
        path_gemm<T>(x, true, N, N, N, Ep, 1, ld, x.G(s), ld, 1, Gt, ld, 1, EpiStore());
        __syncthreads();
        path_gemm<T>(x, true, N, N, N, Gt, ld, 1, Em, ld, 1, x.G(s), ld, 1, EpiStore());
        __syncthreads();
      }
    }
    for (int s = 0; s < x.nspec(); ++s) {
      T* Gs = x.G(s);
      PQMC_FOR_2D(i, 0, N, j, 0, N) Gs[(long)i * ld + j] *= x.vexpT(tau, s, j) * x.vinvT(tau, s, i);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// FP64 stabilisation.

// log|prod_j d_j| and sign(prod_j d_j) of n values in shared memory, summed by
// warp 0 and broadcast through shared memory (collective).
template <typename T>
__device__ void log_det_of(Cta<T>& x, const double* d, int n, int extra_sign_flips, double& logabs, double& sgn) {
  Smem<T>& sh = x.sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (warp == 0) {
    double la = 0.0;
    int neg = 0;
    for (int j = lane; j < n; j += 32) {
      la += log(fabs(d[j]));
      neg += d[j] < 0 ? 1 : 0;
    }
    la = warp_sum(la);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) neg += __shfl_xor_sync(0xffffffffu, neg, o);
    if (lane == 0) {
      sh.red[0] = la;
      sh.red[1] = ((neg + extra_sign_flips) & 1) ? -1.0 : 1.0;
    }
  }
  __syncthreads();
  logabs = sh.red[0];
  sgn = sh.red[1];
  __syncthreads();
}

// Householder QR of the column-major N x n matrix M (ld ldm).  The explicit
// orthonormal factor goes to Q (column-major, ld N); log|det R| and sign(det R)
// are returned to every thread.  Each reflector is applied to all trailing
// columns in three CTA-wide phases (partial column dots over row chunks, one
// thread per column adds the chunks, a parallel rank-1 update), so no FP64
// work sits in warp-shuffle reductions.
template <typename T>
__device__ void householder_apply(Cta<T>& x, int N, int lda, const double* v, double beta, double* A, int c0, int c1,
                                  int j) {
  double* part = x.qpart();
  double* w = x.qw();
  if (c1 <= c0) return;
  // thread (col, p): rows j + p, j + p + kQRParts, ...
  {
    const int p = threadIdx.x & (kQRParts - 1);
    for (int col = c0 + (int)(threadIdx.x / kQRParts); col < c1; col += (int)(blockDim.x / kQRParts)) {
      const double* a = A + (long)col * lda;
      double d0 = 0.0, d1 = 0.0;
      int i = j + p;
      for (; i + kQRParts < N; i += 2 * kQRParts) {
        d0 = fma(v[i], a[i], d0);
        d1 = fma(v[i + kQRParts], a[i + kQRParts], d1);
      }
      if (i < N) d0 = fma(v[i], a[i], d0);
      part[p * x.c.nmax + col] = d0 + d1;
    }
  }
  __syncthreads();
  for (int col = c0 + threadIdx.x; col < c1; col += blockDim.x) {
    const int nm = x.c.nmax;
    double q[kQRParts];
#pragma unroll
    for (int p = 0; p < kQRParts; ++p) q[p] = part[p * nm + col];
#pragma unroll
    for (int h = kQRParts / 2; h > 0; h >>= 1)
#pragma unroll
      for (int p = 0; p < h; ++p) q[p] += q[p + h];
    w[col] = q[0] * beta;
  }
  __syncthreads();
  {
    const int rows = N - j, total = rows * (c1 - c0);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int cl = e / rows, i = j + (e - cl * rows), col = c0 + cl;
      A[(long)col * lda + i] = fma(-v[i], w[col], A[(long)col * lda + i]);
    }
  }
  __syncthreads();
}

// reflector of column j (warp 0): v = x - alpha e_j stored over the column
template <typename T>
__device__ void householder_reflector(Cta<T>& x, int N, int ldm, double* M, int j) {
  const int lane = threadIdx.x & 31;
  if ((threadIdx.x >> 5) == 0) {
    double* v = M + (long)j * ldm;
    double s = 0.0;
    for (int i = j + lane; i < N; i += 32) s = fma(v[i], v[i], s);
    s = warp_sum(s);
    if (lane == 0) {
      const double x0 = v[j];
      const double a = x0 > 0 ? -sqrt(s) : sqrt(s);
      const double v0 = x0 - a;
      const double vv = s - x0 * x0 + v0 * v0;
      v[j] = v0;
      x.qbeta()[j] = vv > 0 ? 2.0 / vv : 0.0;
      x.qalpha()[j] = a;
      if (a == 0.0) x.sh.err |= kErrStab;
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void qr_householder(Cta<T>& x, int N, int ldm, int n, double* M, double* Q, double& logabs, double& sgn) {
  for (int j = 0; j < n; ++j) {
    householder_reflector(x, N, ldm, M, j);
    householder_apply(x, N, ldm, M + (long)j * ldm, x.qbeta()[j], M, j + 1, n, j);
  }
  x.mark(kPhQR);
  PQMC_FOR_2D(col, 0, n, i, 0, N) Q[(long)col * N + i] = (i == col) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) householder_apply(x, N, N, M + (long)j * ldm, x.qbeta()[j], Q, j, n, j);
  log_det_of(x, x.qalpha(), n, 0, logabs, sgn);
  x.mark(kPhQRForm);
}

// Upper triangle (2 x 2 tiles on or above the diagonal) of C = M^T M for the
// column-major N x n matrix M (ld ldm, odd so that the threads' columns fall
// in different shared-memory banks); C row-major n x n.
static __device__ void gram_upper_f64(int n, int N, int ldm, const double* M, double* C) {
  // 2 x 2 output tiles (ti, tj), ti <= tj, enumerated over a flat index so
  // that every warp carries only tiles of the upper triangle (the FP64 pipe
  // takes the same time for a partial warp as for a full one)
  const int tn = (n + 1) >> 1;
  for (int t = threadIdx.x; t < tn * (tn + 1) / 2; t += blockDim.x) {
    int ti = 0, tj = t;
    while (tj >= tn - ti) { tj -= tn - ti; ++ti; }
    tj += ti;
    const int i0 = ti << 1, j0 = tj << 1;
    const double* a0 = M + (long)i0 * ldm;
    const double* a1 = M + (long)min(i0 + 1, n - 1) * ldm;
    const double* b0 = M + (long)j0 * ldm;
    const double* b1 = M + (long)min(j0 + 1, n - 1) * ldm;
    double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
      const double x0 = a0[k], x1 = a1[k], y0 = b0[k], y1 = b1[k];
      c00 = fma(x0, y0, c00);
      c01 = fma(x0, y1, c01);
      c10 = fma(x1, y0, c10);
      c11 = fma(x1, y1, c11);
    }
    C[(long)i0 * n + j0] = c00;
    if (j0 + 1 < n) C[(long)i0 * n + j0 + 1] = c01;
    if (i0 + 1 < n) {
      C[(long)(i0 + 1) * n + j0] = c10;
      if (j0 + 1 < n) C[(long)(i0 + 1) * n + j0 + 1] = c11;
    }
  }
}

// Cholesky QR of the column-major N x n matrix M (ld N), used for the stack
// blocks of the reduced-precision paths: C = M^T M = R^T R, Q = M R^{-1}
// (Stathopoulos & Wu, SIAM J. Sci. Comput. 23 (2002); the loss of
// orthogonality grows like eps cond(M)^2, Yamamoto et al., ETNA 44 (2015)).
// With two slices per stabilisation cond(M) stays near 1e2, and it needs n
// CTA barriers per factor and per solve instead of the Householder QR's
// sequence of reflector, dot and update phases.  Every FP64 step runs over a
// flat or 2D index of the whole CTA.  Returns false, with M unchanged, when a
// pivot falls below 1e-12 of its original diagonal entry (cond(M) above about
// 1e6); the caller then takes the Householder QR.  R has a positive diagonal,
// so only log|det R| = (1/2) sum_k log(pivot_k) is returned.
template <typename T>
__device__ bool qr_cholesky(Cta<T>& x, int N, int ldm, int n, double* M, double* Q, double& logabs) {
  Smem<T>& sh = x.sh;
  double* C = x.chol();                 // n x n row-major (upper part): Gram, then Schur complements
  double* U = C + (long)n * n;          // n x n row-major (upper part): U_kj = R_kj / R_kk
  double* d0 = U + (long)n * n;         // original diagonal
  double* ip = d0 + n;                  // 1 / pivot
  double* isq = ip + n;                 // 1 / sqrt(pivot)
  gram_upper_f64(n, N, ldm, M, C);
  if (threadIdx.x == 0) sh.chol_bad = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) d0[k] = C[(long)k * n + k];
  if (threadIdx.x == 0) ip[0] = 1.0 / C[0];
  __syncthreads();
  // right-looking factorisation: step k scales row k into U (U_kj = C_kj / p_k)
  // and then updates the trailing block, C_ij -= C_ki U_kj (i, j > k; the
  // part below the diagonal is updated too, so the flat loop keeps the warps
  // full, and never read)
  const int step = (int)blockDim.x;
  for (int k = 0; k < n; ++k) {
    const double p = C[(long)k * n + k];
    if (!(p > 1e-12 * d0[k])) {          // same value in every thread: uniform exit
      if (threadIdx.x == 0) sh.chol_bad = 1;
      break;
    }
    const double ipk = ip[k];
    for (int j = k + 1 + (int)threadIdx.x; j < n; j += step) U[(long)k * n + j] = C[(long)k * n + j] * ipk;
    __syncthreads();
    const int m = n - k - 1;
    if (m > 0) {
      const int sq = step / m, sr = step - sq * m;
      int i = (int)threadIdx.x / m, j = (int)threadIdx.x - i * m;
      const double* Ck = C + (long)k * n + k + 1;
      const double* Uk = U + (long)k * n + k + 1;
      double* Cb = C + (long)(k + 1) * n + k + 1;
      while (i < m) {
        Cb[(long)i * n + j] = fma(-Ck[i], Uk[j], Cb[(long)i * n + j]);
        if (i == 0 && j == 0) ip[k + 1] = 1.0 / Cb[0];
        j += sr;
        i += sq;
        if (j >= m) { j -= m; ++i; }
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (sh.chol_bad) return false;
  for (int k = threadIdx.x; k < n; k += blockDim.x) isq[k] = rsqrt(C[(long)k * n + k]);
  __syncthreads();
  x.mark(kPhQR);
  {
    // Q = M R^{-1}, right-looking over the columns of M: q_k = m_k / R_kk,
    // m_j -= m_k U_kj for j > k, in blocks of four columns: each row first
    // takes its block's own triangle in registers, then one flat pass
    // applies the block's four updates to the later columns (a barrier pair
    // per block instead of per column; every element sees the same FMAs in
    // the same order as column by column)
    for (int K = 0; K < n; K += 4) {
      const int kb = min(4, n - K);
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double mv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) mv[u] = u < kb ? M[(long)(K + u) * ldm + i] : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < kb) {
            Q[(long)(K + u) * N + i] = mv[u] * isq[K + u];
#pragma unroll
            for (int v = u + 1; v < 4; ++v)
              if (v < kb) mv[v] = fma(-mv[u], U[(long)(K + u) * n + K + v], mv[v]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < kb) M[(long)(K + u) * ldm + i] = mv[u];
      }
      __syncthreads();
      const int j0 = K + kb;
      if (j0 < n) {
        const int sq = step / N, sr = step - sq * N;
        const int t0 = (int)threadIdx.x / N, r0 = (int)threadIdx.x - t0 * N;
        int jj = j0 + t0, i = r0;
        while (jj < n) {
          double acc = M[(long)jj * ldm + i];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (u < kb) acc = fma(-M[(long)(K + u) * ldm + i], U[(long)(K + u) * n + jj], acc);
          M[(long)jj * ldm + i] = acc;
          i += sr;
          jj += sq;
          if (i >= N) { i -= N; ++jj; }
        }
      }
      __syncthreads();
    }
  }
  // log|det R|
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
      double la = 0.0;
      for (int k = lane; k < n; k += 32) la += log(C[(long)k * n + k]);
      la = warp_sum(la);
      if (lane == 0) sh.red[0] = 0.5 * la;
    }
    __syncthreads();
    logabs = sh.red[0];
    __syncthreads();
  }
  x.mark(kPhQRForm);
  return true;
}

// Invert O_s (n_s x n_s, row-major) in place for both spins at once by
// Gauss-Jordan elimination with partial pivoting (Golub & Van Loan, section
// 3.2): warp s finds the pivot of spin s, swaps the rows, scales the pivot row
// and saves the pivot column; the CTA then eliminates that column from every
// other row; the row interchanges are undone on the columns at the end.
// Returns log|det O_s| and sign(det O_s) to every thread.
template <typename T>
__device__ void gj_invert2(Cta<T>& x, const int n[2], double* O[2], double logabs[2], double sgn[2]) {
  Smem<T>& sh = x.sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nmax = n[0] > n[1] ? n[0] : n[1];
  if (threadIdx.x < 2) sh.nswap[threadIdx.x] = 0;
  __syncthreads();
  for (int j = 0; j < nmax; ++j) {
    if (warp < 2 && j < n[warp]) {
      const int s = warp, ns = n[s];
      double* A = O[s];
      double* f = x.lmul(s);
      // pivot: largest |A_ij|, i >= j, ties to the lower row; |x| is compared
      // through the bit pattern with the sign cleared, which orders
      // non-negative doubles like their values
      unsigned long long best = 0;
      int bi = j;
      for (int i = j + lane; i < ns; i += 32) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(A[(long)i * ns + j]) & 0x7fffffffffffffffull;
        if (v > best || bi == j && i == j) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (bi != j) {
        for (int col = lane; col < ns; col += 32) {
          const double t = A[(long)j * ns + col];
          A[(long)j * ns + col] = A[(long)bi * ns + col];
          A[(long)bi * ns + col] = t;
        }
        if (lane == 0) sh.nswap[s]++;
      }
      if (lane == 0) x.pinv(s)[j] = (double)bi;         // row interchange of step j
      __syncwarp();
      const double pv = A[(long)j * ns + j];
      const double ip = pv != 0.0 ? 1.0 / pv : 0.0;
      if (lane == 0) {
        x.pval(s)[j] = pv;
        if (pv == 0.0) sh.err |= kErrStab;
      }
      for (int i = lane; i < ns; i += 32) f[i] = A[(long)i * ns + j];
      __syncwarp();
      for (int col = lane; col < ns; col += 32) A[(long)j * ns + col] = (col == j) ? ip : A[(long)j * ns + col] * ip;
    }
    __syncthreads();
    x.mark(kPhGJPivot);
    // eliminate column j from every other row of both spins: one FMA per
    // element over a flat index (full warps on the FP64 pipe); the pivot
    // column takes -f_i / pivot through the same FMA with a zero addend
    for (int s = 0; s < 2; ++s) {
      const int ns = n[s];
      if (j >= ns) continue;
      double* A = O[s];
      const double* fl = x.lmul(s);
      // flat (row, column) index stepped incrementally
      const int step = (int)blockDim.x, sq = step / ns, sr = step - sq * ns;
      int i = (int)threadIdx.x / ns, col = (int)threadIdx.x - i * ns;
      while (i < ns) {
        const double add = col == j ? 0.0 : A[(long)i * ns + col];
        const double r = fma(-fl[i], A[(long)j * ns + col], add);
        if (i != j) A[(long)i * ns + col] = r;
        col += sr;
        i += sq;
        if (col >= ns) { col -= ns; ++i; }
      }
    }
    __syncthreads();
    x.mark(kPhGJElim);
  }
  // undo the row interchanges on the columns, last step first
  if (warp < 2) {
    const int s = warp, ns = n[s];
    double* A = O[s];
    for (int j = ns - 1; j >= 0; --j) {
      const int p = (int)x.pinv(s)[j];
      if (p != j)
        for (int i = lane; i < ns; i += 32) {
          const double t = A[(long)i * ns + j];
          A[(long)i * ns + j] = A[(long)i * ns + p];
          A[(long)i * ns + p] = t;
        }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int s = 0; s < 2; ++s) log_det_of(x, x.pval(s), n[s], sh.nswap[s], logabs[s], sgn[s]);
  x.mark(kPhGJTail);
}

// C = A^T B for column-major A, B (K x m and K x m', ld K): FP64, 2 x 3
// outputs per thread (a 36 x 36 product is 216 tiles: one pass of a
// 256-thread CTA).
static __device__ void gemm_tn_f64(int m, int mp, int K, const double* A, const double* B, double* C, int ldc) {
  const int tm = (m + 1) >> 1, tn = (mp + 2) / 3;
  for (int t = threadIdx.x; t < tm * tn; t += blockDim.x) {
    const int i0 = (t / tn) << 1, j0 = (t % tn) * 3;
    const double* a0 = A + (long)i0 * K;
    const double* a1 = A + (long)min(i0 + 1, m - 1) * K;
    const double* b0 = B + (long)j0 * K;
    const double* b1 = B + (long)min(j0 + 1, mp - 1) * K;
    const double* b2 = B + (long)min(j0 + 2, mp - 1) * K;
    double c00 = 0, c01 = 0, c02 = 0, c10 = 0, c11 = 0, c12 = 0;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const double x0 = a0[k], x1 = a1[k], y0 = b0[k], y1 = b1[k], y2 = b2[k];
      c00 = fma(x0, y0, c00);
      c01 = fma(x0, y1, c01);
      c02 = fma(x0, y2, c02);
      c10 = fma(x1, y0, c10);
      c11 = fma(x1, y1, c11);
      c12 = fma(x1, y2, c12);
    }
    C[(long)i0 * ldc + j0] = c00;
    if (j0 + 1 < mp) C[(long)i0 * ldc + j0 + 1] = c01;
    if (j0 + 2 < mp) C[(long)i0 * ldc + j0 + 2] = c02;
    if (i0 + 1 < m) {
      C[(long)(i0 + 1) * ldc + j0] = c10;
      if (j0 + 1 < mp) C[(long)(i0 + 1) * ldc + j0 + 1] = c11;
      if (j0 + 2 < mp) C[(long)(i0 + 1) * ldc + j0 + 2] = c12;
    }
  }
}

static __device__ void copy_block(const double* src, double* dst, int n) {
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
  __syncthreads();
}

template <typename T>
__device__ double* stack_block(const Cta<T>& x, double* base, int b, int s) {
  return base + ((long)b * 2 + s) * x.c.N * x.c.nmax;
}

// Right stack block b: QR of B_{b n} ... B_{(b-1)n+1} Q_R[b-1] (b >= 1) or of B_0 P (b = 0).
// The slice products run in the path precision on a row-major copy.
template <typename T>
__device__ void push_R(Cta<T>& x, int b) {
  const ChainDesc& c = x.c;
  const int N = c.N, n_stab = c.n_stab;
  const int ldm = m64_ld(N);
  double* M = x.M64();
  for (int s = 0; s < x.nspec(); ++s) {
    const int n = x.nsig(s);
    const double* P = c.P + (long)s * N * c.nmax;
    T* Mt = x.Mt();
    T* Mt2 = x.Mt2();
    double prev_l = 0.0, prev_s = 1.0;
    if (b == 0) {
      x.stage(0);
      PQMC_FOR_2D(k, 0, n, i, 0, N) M[(long)k * ldm + i] = x.vexp(0, s, i) * P[(long)k * N + i];
      __syncthreads();
    } else {
      const double* prev = stack_block(x, c.Rst, b - 1, s);
      PQMC_FOR_2D(k, 0, n, i, 0, N) Mt[(long)i * n + k] = (T)prev[(long)k * N + i];
      prev_l = c.Rlog[((b - 1) * 2 + s) * 2 + 0];
      prev_s = c.Rlog[((b - 1) * 2 + s) * 2 + 1];
      for (int tau = (b - 1) * n_stab + 1; tau <= b * n_stab; ++tau) {
        x.stage(tau);
        PQMC_FOR_2D(i, 0, N, k, 0, n) Mt[(long)i * n + k] *= x.vexpT(tau, s, i);
        __syncthreads();
        cta_gemm<T>(N, n, N, x.Em(), 1, c.ld, Mt, n, 1, Mt2, n, 1, EpiStore());
        __syncthreads();
        T* t = Mt; Mt = Mt2; Mt2 = t;
      }
      PQMC_FOR_2D(k, 0, n, i, 0, N) M[(long)k * ldm + i] = (double)Mt[(long)i * n + k];
      __syncthreads();
    }
    double la, sg = 1.0;
    x.mark(kPhStack);
    if (std::is_same<T, double>::value || !qr_cholesky(x, N, ldm, n, M, x.Q64(), la))
      qr_householder(x, N, ldm, n, M, x.Q64(), la, sg);
    copy_block(x.Q64(), stack_block(x, c.Rst, b, s), N * n);
    x.mark(kPhQR);
    if (threadIdx.x == 0) {
      c.Rlog[(b * 2 + s) * 2 + 0] = prev_l + la;
      c.Rlog[(b * 2 + s) * 2 + 1] = prev_s * sg;
    }
    __syncthreads();
  }
}

// Left stack block b holds (B_L(b n))^T = Q T^T: QR of
// B_{bn+1}^T ... B_{(b+1)n}^T Q_L[b+1] (b < nb) or of e^{V(s_{Ltau+1})} P (b = nb).
template <typename T>
__device__ void push_L(Cta<T>& x, int b) {
  const ChainDesc& c = x.c;
  const int N = c.N, n_stab = c.n_stab;
  const int ldm = m64_ld(N);
  double* M = x.M64();
  for (int s = 0; s < x.nspec(); ++s) {
    const int n = x.nsig(s);
    const double* P = c.P + (long)s * N * c.nmax;
    T* Mt = x.Mt();
    T* Mt2 = x.Mt2();
    double prev_l = 0.0, prev_s = 1.0;
    if (b == c.nb) {
      x.stage(c.Ltau + 1);
      PQMC_FOR_2D(k, 0, n, i, 0, N) M[(long)k * ldm + i] = x.vexp(c.Ltau + 1, s, i) * P[(long)k * N + i];
      __syncthreads();
    } else {
      const double* prev = stack_block(x, c.Lst, b + 1, s);
      PQMC_FOR_2D(k, 0, n, i, 0, N) Mt[(long)i * n + k] = (T)prev[(long)k * N + i];
      prev_l = c.Llog[((b + 1) * 2 + s) * 2 + 0];
      prev_s = c.Llog[((b + 1) * 2 + s) * 2 + 1];
      __syncthreads();
      for (int tau = (b + 1) * n_stab; tau > b * n_stab; --tau) {
        cta_gemm<T>(N, n, N, x.Em(), 1, c.ld, Mt, n, 1, Mt2, n, 1, EpiStore());
        x.stage(tau);
        PQMC_FOR_2D(i, 0, N, k, 0, n) Mt[(long)i * n + k] = x.vexpT(tau, s, i) * Mt2[(long)i * n + k];
        __syncthreads();
      }
      PQMC_FOR_2D(k, 0, n, i, 0, N) M[(long)k * ldm + i] = (double)Mt[(long)i * n + k];
      __syncthreads();
    }
    double la, sg = 1.0;
    x.mark(kPhStack);
    if (std::is_same<T, double>::value || !qr_cholesky(x, N, ldm, n, M, x.Q64(), la))
      qr_householder(x, N, ldm, n, M, x.Q64(), la, sg);
    copy_block(x.Q64(), stack_block(x, c.Lst, b, s), N * n);
    x.mark(kPhQR);
    if (threadIdx.x == 0) {
      c.Llog[(b * 2 + s) * 2 + 0] = prev_l + la;
      c.Llog[(b * 2 + s) * 2 + 1] = prev_s * sg;
    }
    __syncthreads();
  }
}

// Fused epilogue of the G assembly: g = delta_ij - v, compare with the
// propagated G, overwrite it.
template <typename T>
struct EpiFresh {
  T* G;
  int ld;
  T* dmax;
  template <typename A, typename TC> __device__ void operator()(TC*, int, int, int i, int j, A v) const {
    const T g = (i == j ? T(1) : T(0)) - (T)v;
    T& ref = G[(long)i * ld + j];
    const T d = fabs(ref - g);
    *dmax = d > *dmax ? d : *dmax;
    ref = g;
  }
};

// Epilogue of the FP64 diagnostic assembly: g = delta_ij - v in FP64 against
// the propagated G (read only).
template <typename T>
struct EpiDiff64 {
  const T* G;
  int ld;
  double* dmax;
  double* gmax;      // largest |G_FP64| element
  template <typename A, typename TC> __device__ void operator()(TC*, int, int, int i, int j, A v) const {
    const double g = (i == j ? 1.0 : 0.0) - (double)v;
    const double d = fabs((double)G[(long)i * ld + j] - g);
    *dmax = d > *dmax ? d : *dmax;
    *gmax = fabs(g) > *gmax ? fabs(g) : *gmax;
  }
};

// G_fresh = 1 - Q_R X Q_L^T for spin s with X = (Q_L^T Q_R)^{-1} (FP64, n x n
// row-major at Xinv), in the path precision; the FP64 diagnostics of
// opts.dg_fp64 around it.
template <typename T>
__device__ void assemble_spin(Cta<T>& x, int s, const double* QR, const double* QL, const double* Xinv, int ns,
                              bool record, T& dmax, double& dmax64) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  const int N = c.N, ld = c.ld;
  T* Y = x.Yb();
  const T* qr = reinterpret_cast<const T*>(QR);
  const T* ql = reinterpret_cast<const T*>(QL);
  if constexpr (!std::is_same<T, double>::value) {
    if ((c.dg64 == 1 || c.dg64 == 3) && record) {
      // Y64 = O^{-1} Q_L^T (n x N, FP64, in the space of the path-precision
      // copies of Q_R and Q_L, which are written after it), then
      // max |G - (1 - Q_R Y64)| over the propagated G (mode 3: divided by
      // max(1, max |G_FP64|), per spin)
      double* y64 = reinterpret_cast<double*>(x.QRt());
      cta_gemm<double>(ns, N, ns, Xinv, ns, 1, QL, N, 1, y64, N, 1, EpiStore());
      __syncthreads();
      double d_s = 0.0, g_s = 0.0;
      EpiDiff64<T> ed{x.G(s), ld, &d_s, &g_s};
      cta_gemm<double>(N, N, ns, QR, 1, N, y64, N, 1, (double*)nullptr, 0, 0, ed);
      if (c.dg64 == 3) {
        d_s = cta_max(d_s, sh.red);
        g_s = cta_max(g_s, sh.red);
        d_s /= fmax(1.0, g_s);
      }
      dmax64 = fmax(dmax64, d_s);
      __syncthreads();
    }
    T* qrt = x.QRt();
    T* qlt = x.QLt();
    PQMC_FOR_2D(k, 0, ns, i, 0, N) {
      qrt[(long)k * N + i] = (T)QR[(long)k * N + i];
      qlt[(long)k * N + i] = (T)QL[(long)k * N + i];
    }
    qr = qrt;
    ql = qlt;
    __syncthreads();
  }
  if constexpr (std::is_same<T, double>::value) {
    cta_gemm<T>(ns, N, ns, Xinv, ns, 1, ql, N, 1, Y, ld, 1, EpiStore());
  } else {
    // O^{-1} to the path precision once, then a path-precision product
    T* ot = x.Ot();
    for (int e = threadIdx.x; e < ns * ns; e += blockDim.x) ot[e] = (T)Xinv[e];
    __syncthreads();
    cta_gemm<T>(ns, N, ns, ot, ns, 1, ql, N, 1, Y, ld, 1, EpiStore());
  }
  __syncthreads();
  EpiFresh<T> epi{x.G(s), ld, &dmax};
  cta_gemm<T>(N, N, ns, qr, 1, N, Y, ld, 1, (T*)nullptr, 0, 0, epi);
  if constexpr (!std::is_same<T, double>::value) {
    if (c.dg64 == 2 && record) {
      // the refreshed G itself against G_FP64 (the path-precision copies of
      // Q_R and Q_L are no longer needed: Y64 takes their space)
      __syncthreads();
      double* y64 = reinterpret_cast<double*>(x.QRt());
      cta_gemm<double>(ns, N, ns, Xinv, ns, 1, QL, N, 1, y64, N, 1, EpiStore());
      __syncthreads();
      double g_s = 0.0;
      EpiDiff64<T> ed{x.G(s), ld, &dmax64, &g_s};
      cta_gemm<double>(N, N, ns, QR, 1, N, y64, N, 1, (double*)nullptr, 0, 0, ed);
    }
  }
  __syncthreads();
}

// G <- 1 - Q_R (Q_L^T Q_R)^{-1} Q_L^T at stabilisation point b; records
// max |G - G_fresh| when record != 0, and the weight's log|det| and sign.
// With c.dg64 (reduced paths) the recorded error is max |G - G_FP64|, the
// propagated G against the same formula assembled in FP64 from the FP64
// factors; the G that replaces the propagated one is still the
// path-precision assembly, so the chain itself is unchanged.
template <typename T>
__device__ void refresh(Cta<T>& x, int b, bool record) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  const int N = c.N;
  T dmax = T(0);
  double dmax64 = 0.0;
  double sign_total = 1.0;
  int n[2] = {x.nsig(0), x.nsig(1)};
  double* O[2] = {x.Ob(0), x.Ob(1)};
  const double* QR[2] = {stack_block(x, c.Rst, b, 0), stack_block(x, c.Rst, b, 1)};
  const double* QL[2] = {stack_block(x, c.Lst, b, 0), stack_block(x, c.Lst, b, 1)};
  // O_s = Q_L^T Q_R and its inverse in FP64, both spins together
  for (int s = 0; s < 2; ++s) gemm_tn_f64(n[s], n[s], N, QL[s], QR[s], O[s], n[s]);
  __syncthreads();
  x.mark(kPhOverlap);
  double la[2], sg[2];
  gj_invert2(x, n, O, la, sg);
  x.mark(kPhLU);
  for (int s = 0; s < x.nspec(); ++s) {
    assemble_spin(x, s, QR[s], QL[s], O[s], n[s], record, dmax, dmax64);
    const double l_tot = c.Rlog[(b * 2 + s) * 2 + 0] + la[s] + c.Llog[(b * 2 + s) * 2 + 0];
    const double s_tot = c.Rlog[(b * 2 + s) * 2 + 1] * sg[s] * c.Llog[(b * 2 + s) * 2 + 1];
    if (threadIdx.x == 0) {
      sh.logw_spin[s] = l_tot;
      sh.sign_spin[s] = s_tot;
    }
    sign_total *= s_tot;
    __syncthreads();
  }
  x.mark(kPhAssemble);
  const double dm = cta_max((c.dg64 && record) ? dmax64 : (double)dmax, sh.red);
  if (threadIdx.x == 0) {
    for (int s = x.nspec(); s < 2; ++s) {
      sh.logw_spin[s] = 0.0;
      sh.sign_spin[s] = 1.0;
    }
    const double dmax = dm;
    if (!isfinite(dmax)) sh.err |= kErrNaN;
    if (record) {
      sh.dGmax = fmax(sh.dGmax, dmax);
      c.dG[c.st->n_dG % kDGHistory] = dmax;
      c.st->n_dG++;
    }
    c.st->sign_stack = sign_total;
  }
  __syncthreads();
}

// Wick estimates on the fresh G at the middle slice: E/site for Eq. (2),
// docc/site, kinetic/site, with the weight sign and the running sign, and the
// staggered S^z structure factor S = (1/N^2) sum_ij eps_i eps_j <S^z_i S^z_j>
// = [(sum_i eps_i m_i)^2 + sum_s sum_ij eps_i eps_j (delta_ij - G_s,ji) G_s,ij]
// / (4 N^2), m_i = n_i,up - n_i,dn (the spins are independent at fixed fields).
// Wick estimates of the spinless t-V model on the fresh G at the middle
// slice: E/site of Eq. (4), interaction energy/site
// V sum_<ij> [(n_i - 1/2)(n_j - 1/2) - G_ji G_ij] / N, kinetic/site, the weight
// sign, the running sign, and S_CDW = [(sum_i eps_i (n_i - 1/2))^2 +
// sum_ij eps_i eps_j (delta_ij - G_ji) G_ij] / N^2.
template <typename T>
__device__ void measure_tv(Cta<T>& x) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  const int N = c.N, ld = c.ld;
  const T* G = x.G(0);
  double ek = 0.0, eb = 0.0, st = 0.0, ex = 0.0;
  PQMC_FOR_2D(i, 0, N, j, 0, N) {
    const double gji = (i == j ? 1.0 : 0.0) - (double)G[(long)j * ld + i];
    ek += c.K64[(long)i * N + j] * gji;
    ex += c.eps[i] * c.eps[j] * gji * (double)G[(long)i * ld + j];
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) st += c.eps[i] * (0.5 - (double)G[(long)i * ld + i]);
  for (int b = threadIdx.x; b < c.nfld; b += blockDim.x) {
    const int i = c.bond_ends[2 * b], j = c.bond_ends[2 * b + 1];
    const double di = 0.5 - (double)G[(long)i * ld + i], dj = 0.5 - (double)G[(long)j * ld + j];
    eb += di * dj - (double)G[(long)j * ld + i] * (double)G[(long)i * ld + j];
  }
  ek = cta_sum(ek, sh.red);
  eb = cta_sum(eb, sh.red) * c.U;
  st = cta_sum(st, sh.red);
  ex = cta_sum(ex, sh.red);
  if (threadIdx.x == 0) {
    const int m = c.st->n_meas;
    const double rec[kRecord] = {sh.sign_spin[0] * sh.sign_spin[1], (ek + eb) / N, eb / N, ek / N,
                                 sh.sign_running, (st * st + ex) / ((double)N * N)};
    for (int k = 0; k < kRecord; ++k) {
      if (m < c.max_meas) c.meas[(long)m * kRecord + k] = rec[k];
      c.last[k] = rec[k];
    }
    c.st->n_meas = m + 1;
  }
  __syncthreads();
}

template <typename T>
__device__ void measure(Cta<T>& x) {
  const ChainDesc& c = x.c;
  if (c.tv) {
    measure_tv(x);
    return;
  }
  Smem<T>& sh = x.sh;
  const int N = c.N, ld = c.ld;
  double ek = 0.0, dc = 0.0, st = 0.0, ex = 0.0;
  PQMC_FOR_2D(i, 0, N, j, 0, N) {
    const double k = c.K64[(long)i * N + j];
    const double ee = c.eps[i] * c.eps[j];
    for (int s = 0; s < 2; ++s) {
      const double gji = (i == j ? 1.0 : 0.0) - (double)x.G(s)[(long)j * ld + i];
      ek += k * gji;
      ex += ee * gji * (double)x.G(s)[(long)i * ld + j];
    }
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double g0 = (double)x.G(0)[(long)i * ld + i], g1 = (double)x.G(1)[(long)i * ld + i];
    dc += (1.0 - g0) * (1.0 - g1);
    st += c.eps[i] * (g1 - g0);
  }
  ek = cta_sum(ek, sh.red);
  dc = cta_sum(dc, sh.red);
  st = cta_sum(st, sh.red);
  ex = cta_sum(ex, sh.red);
  if (threadIdx.x == 0) {
    const int m = c.st->n_meas;
    const double rec[kRecord] = {sh.sign_spin[0] * sh.sign_spin[1], (ek + c.U * dc) / N, dc / N, ek / N,
                                 sh.sign_running, (st * st + ex) / (4.0 * N * N)};
    for (int k = 0; k < kRecord; ++k) {
      if (m < c.max_meas) c.meas[(long)m * kRecord + k] = rec[k];
      c.last[k] = rec[k];
    }
    c.st->n_meas = m + 1;
  }
  __syncthreads();
}

// --------------------------------------------------------------------------
// sweeps

template <typename T>
__device__ void sweep_up(Cta<T>& x, uint32_t sweep, bool do_measure) {
  const ChainDesc& c = x.c;
  for (int tau = 0; tau <= c.Ltau + 1; ++tau) {
    if (c.tv) update_slice_tv(x, tau, sweep);
    else update_slice(x, tau, sweep);
    wrap(x, tau, +1);
    x.mark(kPhWrap);
    if (tau <= c.Ltau && tau % c.n_stab == 0) {
      const int b = tau / c.n_stab;
      push_R(x, b);
      refresh(x, b, true);
      x.mark(kPhRefresh);
      if (do_measure && tau == c.Ltau / 2) measure(x);
      x.mark(kPhMeasure);
    }
  }
}

template <typename T>
__device__ void sweep_down(Cta<T>& x, uint32_t sweep, bool do_measure) {
  const ChainDesc& c = x.c;
  for (int tau = c.Ltau + 1; tau >= 0; --tau) {
    wrap(x, tau, -1);
    x.mark(kPhWrap);
    if (c.tv) update_slice_tv(x, tau, sweep);
    else update_slice(x, tau, sweep);
    const int t1 = tau - 1;
    if (t1 >= 0 && t1 % c.n_stab == 0) {
      const int b = t1 / c.n_stab;
      push_L(x, b);
      refresh(x, b, true);
      x.mark(kPhRefresh);
      if (do_measure && t1 == c.Ltau / 2) measure(x);
      x.mark(kPhMeasure);
    }
  }
}

template <typename T>
__device__ void load_state(Cta<T>& x) {
  if (threadIdx.x == 0) {
    const ChainState& st = *x.c.st;
    x.sh.sign_running = st.sign_running;
    x.sh.dGmax = st.max_dG;
    x.sh.n_prop = st.n_prop;
    x.sh.n_acc = st.n_acc;
    x.sh.acc_pos = st.acc_pos;
    x.sh.err = 0;
    x.sh.staged = -1;
    x.sh.sign_spin[0] = st.logw[0][1];
    x.sh.sign_spin[1] = st.logw[1][1];
    x.sh.logw_spin[0] = st.logw[0][0];
    x.sh.logw_spin[1] = st.logw[1][0];
  }
  if (threadIdx.x < 28) {
    const int k = threadIdx.x / 14, sp = (threadIdx.x / 7) % 2, m = threadIdx.x % 7 - 3;
    double v = 1.0;
    if (x.c.tv) {
      if (sp == 0) v = x.c.vtv[k][m + 3];
    } else if (m == 1 || m == -1) {
      v = x.c.vexp[k][sp][m > 0 ? 0 : 1];
    }
    x.sh.vtab[k][sp][m + 3] = v;
    x.sh.vt[k][sp][m + 3] = (T)v;
    x.sh.vti[k][sp][m + 3] = (T)(1.0 / v);
  }
  if (threadIdx.x < kPhases) x.sh.cyc[threadIdx.x] = 0;
  if (threadIdx.x == 0) x.sh.t_mark = clock64();
  __syncthreads();
}

template <typename T>
__device__ void store_state(Cta<T>& x, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ChainState& st = *x.c.st;
    st.sign_running = x.sh.sign_running;
    st.max_dG = x.sh.dGmax;
    st.n_prop = x.sh.n_prop;
    st.n_acc = x.sh.n_acc;
    st.acc_pos = x.sh.acc_pos;
    st.err |= x.sh.err;
    for (int s = 0; s < 2; ++s) {
      st.logw[s][0] = x.sh.logw_spin[s];
      st.logw[s][1] = x.sh.sign_spin[s];
    }
    for (int p = 0; p < kPhases; ++p) st.cycles[p] += x.sh.cyc[p];
    if (x.sh.err) atomicOr(err, x.sh.err);
  }
}

// Place G and the scratch: in shared memory after the fixed part when the
// chain's footprint fits in res_bytes (G is copied in), else in global memory.
template <typename T>
__device__ Cta<T> make_cta(const ChainDesc& cg, unsigned char* smem_raw, size_t res_bytes, uint64_t seed) {
  Smem<T>& sh = *reinterpret_cast<Smem<T>*>(smem_raw);
  // the descriptor is read all through the sweep: keep a shared-memory copy
  {
    const int words = (int)(sizeof(ChainDesc) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(&cg);
    int* dst = reinterpret_cast<int*>(&sh.desc);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    __syncthreads();
  }
  const ChainDesc& c = sh.desc;
  const int ts = (int)sizeof(T);
  const ScratchLayout L = scratch_layout(c.N, c.ld, c.nmax, ts, c.kb);
  const bool res = resident_bytes(c.N, c.ld, c.nmax, ts, c.kb) <= res_bytes;
  unsigned char* dyn = smem_raw + al16(sizeof(Smem<T>));
  T* Gp = res ? reinterpret_cast<T*>(dyn) : reinterpret_cast<T*>(c.G);
  unsigned char* scr = res ? dyn + al16(2 * (size_t)c.N * c.ld * ts) : reinterpret_cast<unsigned char*>(c.scratch);
  FlipBuf<T>* fb = reinterpret_cast<FlipBuf<T>*>(res ? scr + L.fb : dyn);
  Cta<T> x{c, sh, seed, Gp, scr, L, res, fb};
  if (res) {
    const T* g = reinterpret_cast<const T*>(c.G);
    for (long e = threadIdx.x; e < 2L * c.N * c.ld; e += blockDim.x) Gp[e] = g[e];
  }
  return x;
}

template <typename T>
__device__ void write_back(Cta<T>& x) {
  __syncthreads();
  if (x.resident) {
    T* g = reinterpret_cast<T*>(x.c.G);
    for (long e = threadIdx.x; e < 2L * x.c.N * x.c.ld; e += blockDim.x) g[e] = x.Gp[e];
  }
  __syncthreads();
}

// b_at < 0: initialisation from the chain's fields (left stack, right block
// 0, G at tau = -1 and the running sign). b_at >= 0: the left stack down to
// block b_at, the right stack up to it and G at the stabilisation point
// tau = b_at * n_stab, all from the fields (a recomputation the host wraps
// in a save and restore of the chain's state).
template <typename T, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) init_kernel(const ChainDesc* chains, int chain0, uint64_t seed,
                                                          size_t res_bytes, int* err, int b_at) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cta<T> x = make_cta<T>(chains[chain0 + blockIdx.x], smem_raw, res_bytes, seed);
  Smem<T>& sh = x.sh;
  load_state(x);
  const ChainDesc& c = x.c;
  const int bt = b_at < 0 ? 0 : b_at;
  for (int b = c.nb; b >= bt; --b) push_L(x, b);
  for (int b = 0; b <= bt; ++b) push_R(x, b);
  refresh(x, bt, false);
  if (b_at < 0) {
    if (threadIdx.x == 0) sh.sign_running = sh.sign_spin[0] * sh.sign_spin[1];
    __syncthreads();
    wrap(x, 0, -1);
  }
  write_back(x);
  store_state(x, err);
}

template <typename T, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) sweep_kernel(const ChainDesc* chains, uint64_t seed,
                                                       const uint32_t* sweep_ctr, int n_sweeps, int do_measure,
                                                       size_t res_bytes, int* err, int tc_on) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (chains[blockIdx.x].st->err) return;
  const uint32_t sweep0 = *sweep_ctr;
  Cta<T> x = make_cta<T>(chains[blockIdx.x], smem_raw, res_bytes, seed);
  Smem<T>& sh = x.sh;
  load_state(x);
  if constexpr (std::is_same<T, float>::value && TPB == 512) {
    // BF16X3 chains kept in global memory run their products on the tensor
    // cores: a staging area after the dynamic shared memory the launch
    // reserves for it, and TMEM columns held until the CTA ends
    if (tc_on && x.c.tc && !x.resident) {
      const size_t fbb = flipbuf_bytes((int)sizeof(T));
      const uintptr_t at = reinterpret_cast<uintptr_t>(smem_raw) + al16(sizeof(Smem<T>)) + (res_bytes > fbb ? res_bytes : fbb);
      x.tcs = reinterpret_cast<unsigned char*>((at + 127) & ~(uintptr_t)127);
      x.tmem = tc_alloc(x.tcs);
    }
  }
  const long long t_start = clock64();
  for (int k = 0; k < n_sweeps; ++k) {
    const uint32_t sw = sweep0 + (uint32_t)k;
    if ((sw & 1u) == 0) sweep_up(x, sw, do_measure != 0);
    else sweep_down(x, sw, do_measure != 0);
    __syncthreads();
    if (sh.err) break;
  }
  if (threadIdx.x == 0) sh.cyc[kPhTotal] += clock64() - t_start;
  if constexpr (std::is_same<T, float>::value && TPB == 512) {
    if (x.tcs) tc_free(x.tmem);
  }
  write_back(x);
  store_state(x, err);
}

// --------------------------------------------------------------------------
// launch templates, instantiated by the per-path translation units

template <typename T>
static size_t dyn_smem(size_t res) {
  const size_t fbb = flipbuf_bytes((int)sizeof(T));
  return al16(sizeof(Smem<T>)) + (res > fbb ? res : fbb);
}

template <typename T, int TPB, int MINB>
static cudaError_t launch_init_t(const ChainDesc* d_chains, int chain0, int n, uint64_t seed, size_t res, int* d_err,
                                 cudaStream_t stream, int b_at) {
  const size_t sm = dyn_smem<T>(res);
  cudaError_t e = cudaFuncSetAttribute(init_kernel<T, TPB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  init_kernel<T, TPB, MINB><<<n, TPB, sm, stream>>>(d_chains, chain0, seed, res, d_err, b_at);
  return cudaGetLastError();
}

// Advances the device-side sweep index after a sweep launch (sweep.cu).
cudaError_t launch_advance(uint32_t* sweep_ctr, int n, cudaStream_t stream);

// tc_on: the launch reserves the tensor-core staging area (BF16X3 on
// 512-thread CTAs)
template <typename T, int TPB, int MINB>
static size_t sweep_smem(size_t res, int tc_on) {
  return dyn_smem<T>(res) + ((std::is_same<T, float>::value && TPB == 512 && tc_on) ? kTcBytes + 128 : 0);
}

template <typename T, int TPB, int MINB>
static cudaError_t prepare_sweep_t(size_t res, int tc_on) {
  return cudaFuncSetAttribute(sweep_kernel<T, TPB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sweep_smem<T, TPB, MINB>(res, tc_on));
}

template <typename T, int TPB, int MINB>
static cudaError_t launch_sweep_t(const ChainDesc* d_chains, int n, uint64_t seed, uint32_t* sweep_ctr, int n_sweeps,
                                  int measure, size_t res, int* d_err, cudaStream_t stream, int tc_on) {
  sweep_kernel<T, TPB, MINB><<<n, TPB, sweep_smem<T, TPB, MINB>(res, tc_on), stream>>>(
      d_chains, seed, sweep_ctr, n_sweeps, measure, res, d_err, tc_on);
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : launch_advance(sweep_ctr, n_sweeps, stream);
}

// Defines launch_init_<P>, prepare_sweep_<P> and launch_sweep_<P> over the
// CTA shapes that PQMC_TPB_DISPATCH (defined by the including unit) selects.
#define PQMC_DEFINE_LAUNCHERS(P)                                                                                  \
  cudaError_t launch_init_##P(int tpb, const ChainDesc* d_chains, int chain0, int n, uint64_t seed, size_t res,    \
                              int* d_err, cudaStream_t stream, int b_at) {                                         \
    PQMC_TPB_DISPATCH(launch_init_t, d_chains, chain0, n, seed, res, d_err, stream, b_at);                          \
  }                                                                                                                \
  cudaError_t prepare_sweep_##P(int tpb, size_t res, int tc_on) { PQMC_TPB_DISPATCH(prepare_sweep_t, res, tc_on); } \
  cudaError_t launch_sweep_##P(int tpb, const ChainDesc* d_chains, int n, uint64_t seed, uint32_t* sweep_ctr,      \
                               int n_sweeps, int measure, size_t res, int* d_err, cudaStream_t stream, int tc_on) { \
    PQMC_TPB_DISPATCH(launch_sweep_t, d_chains, n, seed, sweep_ctr, n_sweeps, measure, res, d_err, stream, tc_on);  \
  }

// Per-path launchers (one translation unit each).
#define PQMC_DECLARE_LAUNCHERS(P)                                                                                 \
  cudaError_t launch_init_##P(int tpb, const ChainDesc* d_chains, int chain0, int n, uint64_t seed, size_t res,    \
                              int* d_err, cudaStream_t stream, int b_at);                                          \
  cudaError_t prepare_sweep_##P(int tpb, size_t res, int tc_on);                                                  \
  cudaError_t launch_sweep_##P(int tpb, const ChainDesc* d_chains, int n, uint64_t seed, uint32_t* sweep_ctr,      \
                               int n_sweeps, int measure, size_t res, int* d_err, cudaStream_t stream, int tc_on);
PQMC_DECLARE_LAUNCHERS(f64)
PQMC_DECLARE_LAUNCHERS(f32)
PQMC_DECLARE_LAUNCHERS(f32_256)
PQMC_DECLARE_LAUNCHERS(f32_512)
PQMC_DECLARE_LAUNCHERS(f32_dense)

}  // namespace pqmc

// PQMC sweep kernels for GB300 (sm_103a).
//
// One CTA owns one Markov chain for the whole launch and runs complete
// sweeps: Metropolis flips of the Ising fields with delayed (blocked)
// updates, slice wrapping, QR stabilisation of the B_L / B_R stacks in FP64,
// and the measurement at the middle slice.  Chains are independent, so a
// batch of chains of uneven size is one launch with one CTA per chain.
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
#include <cuda_runtime.h>
#include <stdint.h>

#include "chain.h"
#include "philox.cuh"

namespace pqmc {

// --------------------------------------------------------------------------
// small CTA helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the CTA; every thread gets the result.  red holds >= 32 doubles.
__device__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = lane < nw ? red[lane] : 0.0;
  t = warp_sum(t);
  return t;
}
__device__ double cta_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = lane < nw ? red[lane] : 0.0;
  t = warp_max(t);
  return t;
}

// --------------------------------------------------------------------------
// CTA-wide register-tiled GEMM: C = A B with arbitrary strides,
// A(i,k) = A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj]; the epilogue receives
// (i, j, value).  Every thread owns 4x4 outputs.

struct EpiStore {
  template <typename T> __device__ void operator()(T* C, int sci, int scj, int i, int j, T v) const {
    C[(long)i * sci + (long)j * scj] = v;
  }
};
struct EpiSub {
  template <typename T> __device__ void operator()(T* C, int sci, int scj, int i, int j, T v) const {
    C[(long)i * sci + (long)j * scj] -= v;
  }
};

template <typename T, typename Epi>
__device__ void cta_gemm(int M, int Nn, int K, const T* A, int sai, int sak, const T* B, int sbk,
                         int sbj, T* C, int sci, int scj, Epi epi) {
  const int tm = (M + 3) >> 2, tn = (Nn + 3) >> 2;
  for (int t = threadIdx.x; t < tm * tn; t += blockDim.x) {
    const int i0 = (t / tn) << 2, j0 = (t % tn) << 2;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = T(0);
    for (int k = 0; k < K; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = (i0 + r < M) ? A[(long)(i0 + r) * sai + (long)k * sak] : T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = (j0 + q < Nn) ? B[(long)k * sbk + (long)(j0 + q) * sbj] : T(0);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i0 + r < M && j0 + q < Nn) epi(C, sci, scj, i0 + r, j0 + q, acc[r][q]);
  }
}

// --------------------------------------------------------------------------
// shared memory of one chain CTA

template <typename T>
struct Smem {
  T Gb[2][kBlock][kBlock + 1];      // diagonal block of current G, both spins
  T xs[2][kBlock][kBlock];          // column snapshot at each accepted flip
  T ys[2][kBlock][kBlock];          // row snapshot at each accepted flip
  T Tu[2][kBlock][kBlock + 1];      // U = (E_S - G_{:,S}) Tu
  T Tv[2][kBlock][kBlock + 1];      // W = Tv^T G_{S,:}
  T cl[2][kBlock];                  // Delta / R_sigma of each accepted flip
  double u[kBlock];                 // Metropolis uniforms of the block
  double red[32];                   // reduction scratch
  double qbeta[1024];               // Householder betas (n_sigma <= 1024)
  double lmul[1024];                // LU multipliers
  int sites[kBlock];                // block index of each accepted flip
  int fl[kBlock];                   // fields of the block
  int na;                           // accepted flips in the block
  int piv;
  double sign_running;
  double sign_spin[2];
  double logw_spin[2];
  double dGmax;
  long long n_prop, n_acc, acc_pos;
  int err;
};

template <typename T>
struct Cta {
  const ChainDesc& c;
  Smem<T>& sh;
  uint64_t seed;
  __device__ T* G(int s) const { return reinterpret_cast<T*>(c.G) + (long)s * c.N * c.ld; }
  __device__ T* Gt(int s) const { return reinterpret_cast<T*>(c.Gt) + (long)s * c.N * c.ld; }
  __device__ const T* Em() const { return reinterpret_cast<const T*>(c.expKm); }
  __device__ const T* Ep() const { return reinterpret_cast<const T*>(c.expKp); }
  __device__ int nsig(int s) const { return s == 0 ? c.nup : c.ndn; }
  __device__ bool gutz(int tau) const { return tau == 0 || tau == c.Ltau + 1; }
  __device__ double vexp(int tau, int s, int i) const {
    const int f = c.fields[(long)tau * c.N + i];
    return c.vexp[gutz(tau) ? 1 : 0][s][f > 0 ? 0 : 1];
  }
};

// --------------------------------------------------------------------------
// Metropolis updates of one slice with delayed updates in blocks of kBlock
// sites.  Inside a block one warp proposes the flips sequentially on the
// kBlock x kBlock diagonal block of G (rank-1 updates restricted to the block)
// and records, for the accepted set S, upper-triangular Tu and Tv such that
// the sequence of Sherman-Morrison updates equals
//     G <- G - (E_S - G_{:,S}) Tu Tv^T G_{S,:}
// with G the G at the start of the block.  Column a of Tu / Tv follows from
// the rank-1 form u_a = c_a (e_{s_a} - G^{(a)}_{:,s_a}),
// v_a = G^{(a)}_{s_a,:}, G^{(a)} = G - sum_{l<a} u_l v_l^T:
//     Tu[:,a] = c_a (e_a + sum_{l<a} Tu[:,l] v_l(s_a)),
//     Tv[:,a] = e_a - sum_{l<a} Tv[:,l] u_l(s_a).
// The whole CTA then applies the rank-|S| update to G.

template <typename T>
__device__ void update_slice(Cta<T>& x, int tau, uint32_t sweep) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  const int N = c.N, ld = c.ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kap = x.gutz(tau) ? 1 : 0;
  int8_t* f = c.fields + (long)tau * N;
  T* Ubuf = reinterpret_cast<T*>(c.UW);                // 2 x N x kBlock
  T* Wbuf = Ubuf + 2L * N * kBlock;                    // 2 x kBlock x ld

  for (int i0 = 0; i0 < N; i0 += kBlock) {
    const int nbk = min(kBlock, N - i0);
    for (int e = threadIdx.x; e < 2 * kBlock * kBlock; e += blockDim.x) {
      const int s = e / (kBlock * kBlock), r = (e / kBlock) % kBlock, q = e % kBlock;
      sh.Gb[s][r][q] = (r < nbk && q < nbk) ? x.G(s)[(long)(i0 + r) * ld + i0 + q] : T(0);
    }
    if (threadIdx.x < kBlock) {
      const int j = threadIdx.x;
      sh.u[j] = j < nbk ? metropolis_uniform(x.seed, c.chain_index, sweep, (uint32_t)tau, (uint32_t)(i0 + j)) : 2.0;
      sh.fl[j] = j < nbk ? (int)f[i0 + j] : 1;
    }
    __syncthreads();

    if (warp == 0) {
      int a = 0;
      for (int j = 0; j < nbk; ++j) {
        const int si = sh.fl[j] > 0 ? 0 : 1;
        const T d0 = (T)c.delta[kap][0][si], d1 = (T)c.delta[kap][1][si];
        const T r0 = T(1) + d0 * (T(1) - sh.Gb[0][j][j]);
        const T r1 = T(1) + d1 * (T(1) - sh.Gb[1][j][j]);
        const T R = r0 * r1;
        const bool acc = sh.u[j] < fabs((double)R);
        if (lane == 0) {
          if (!isfinite((double)R)) sh.err |= kErrNaN;
          if (sh.acc_pos < c.acc_cap) c.acc_log[sh.acc_pos] = acc ? 1 : 0;
          sh.acc_pos++;
          sh.n_prop++;
        }
        if (!acc) continue;
        const T cc[2] = {d0 / r0, d1 / r1};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          sh.xs[s][a][lane] = sh.Gb[s][lane][j];
          sh.ys[s][a][lane] = sh.Gb[s][j][lane];
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          T tu = (lane == a) ? T(1) : T(0);
          T tv = tu;
          if (lane < a) {
            for (int l = lane; l < a; ++l) {
              tu = fma(sh.Tu[s][lane][l], sh.ys[s][l][j], tu);
              tv = fma(sh.Tv[s][lane][l], sh.cl[s][l] * sh.xs[s][l][j], tv);
            }
          }
          sh.Tu[s][lane][a] = lane <= a ? cc[s] * tu : T(0);
          sh.Tv[s][lane][a] = lane <= a ? tv : T(0);
          const T yq = sh.ys[s][a][lane];
          for (int r = 0; r < nbk; ++r) {
            const T xr = sh.xs[s][a][r];
            sh.Gb[s][r][lane] -= cc[s] * ((r == j ? T(1) : T(0)) - xr) * yq;
          }
        }
        if (lane == 0) {
          sh.sites[a] = j;
          sh.cl[0][a] = cc[0];
          sh.cl[1][a] = cc[1];
          sh.fl[j] = -sh.fl[j];
          f[i0 + j] = (int8_t)sh.fl[j];
          sh.sign_running *= (R < T(0)) ? -1.0 : 1.0;
          sh.n_acc++;
        }
        ++a;
        __syncwarp();
      }
      if (lane == 0) sh.na = a;
    }
    __syncthreads();
    const int a = sh.na;
    if (a == 0) continue;

    // U[i][l'] = sum_{l<=l'} (delta_{i, s_l} - G[i][s_l]) Tu[l][l']   (N x a)
    // W[l'][q] = sum_{l<=l'} Tv[l][l'] G[s_l][q]                      (a x N)
    for (int e = threadIdx.x; e < 2 * N * a; e += blockDim.x) {
      const int s = e / (N * a), rem = e % (N * a), i = rem / a, lp = rem % a;
      const T* Gs = x.G(s);
      T acc = T(0);
      for (int l = 0; l <= lp; ++l) {
        const int col = i0 + sh.sites[l];
        acc = fma((i == col ? T(1) : T(0)) - Gs[(long)i * ld + col], sh.Tu[s][l][lp], acc);
      }
      Ubuf[(long)s * N * kBlock + (long)i * kBlock + lp] = acc;
    }
    for (int e = threadIdx.x; e < 2 * N * a; e += blockDim.x) {
      const int s = e / (N * a), rem = e % (N * a), lp = rem / N, q = rem % N;
      const T* Gs = x.G(s);
      T acc = T(0);
      for (int l = 0; l <= lp; ++l) acc = fma(sh.Tv[s][l][lp], Gs[(long)(i0 + sh.sites[l]) * ld + q], acc);
      Wbuf[(long)s * kBlock * ld + (long)lp * ld + q] = acc;
    }
    __syncthreads();
    for (int s = 0; s < 2; ++s)
      cta_gemm<T>(N, N, a, Ubuf + (long)s * N * kBlock, kBlock, 1, Wbuf + (long)s * kBlock * ld, ld, 1,
                  x.G(s), ld, 1, EpiSub());
    __syncthreads();
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
  if (dir > 0) {
    for (int e = threadIdx.x; e < 2 * N * N; e += blockDim.x) {
      const int s = e / (N * N), i = (e / N) % N, j = e % N;
      x.G(s)[(long)i * ld + j] *= (T)(x.vexp(tau, s, i) / x.vexp(tau, s, j));
    }
    __syncthreads();
    if (gz) return;
    // Gt = e^{-dtau K} G (stored transposed), G = Gt e^{+dtau K}
    for (int s = 0; s < 2; ++s)
      cta_gemm<T>(N, N, N, x.Em(), 1, ld, x.G(s), ld, 1, x.Gt(s), 1, ld, EpiStore());
    __syncthreads();
    for (int s = 0; s < 2; ++s)
      cta_gemm<T>(N, N, N, x.Gt(s), 1, ld, x.Ep(), ld, 1, x.G(s), ld, 1, EpiStore());
    __syncthreads();
  } else {
    if (!gz) {
      for (int s = 0; s < 2; ++s)
        cta_gemm<T>(N, N, N, x.Ep(), 1, ld, x.G(s), ld, 1, x.Gt(s), 1, ld, EpiStore());
      __syncthreads();
      for (int s = 0; s < 2; ++s)
        cta_gemm<T>(N, N, N, x.Gt(s), 1, ld, x.Em(), ld, 1, x.G(s), ld, 1, EpiStore());
      __syncthreads();
    }
    for (int e = threadIdx.x; e < 2 * N * N; e += blockDim.x) {
      const int s = e / (N * N), i = (e / N) % N, j = e % N;
      x.G(s)[(long)i * ld + j] *= (T)(x.vexp(tau, s, j) / x.vexp(tau, s, i));
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// FP64 stabilisation.

// Householder QR of the column-major N x n matrix M (ld N).  The explicit
// orthonormal factor goes to Q (column-major, ld N); log|det R| and sign(det R)
// are returned through the shared variables.
template <typename T>
__device__ void qr_householder(Cta<T>& x, int N, int n, double* M, double* Q, double& logabs, double& sgn) {
  Smem<T>& sh = x.sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double s_alpha;
  double la = 0.0, sg = 1.0;
  for (int j = 0; j < n; ++j) {
    double* v = M + (long)j * N;
    if (warp == 0) {
      double s = 0.0;
      for (int i = j + lane; i < N; i += 32) s += v[i] * v[i];
      s = warp_sum(s);
      if (lane == 0) {
        const double x0 = v[j];
        const double alpha = x0 > 0 ? -sqrt(s) : sqrt(s);
        const double v0 = x0 - alpha;
        const double vv = s - x0 * x0 + v0 * v0;
        v[j] = v0;
        sh.qbeta[j] = vv > 0 ? 2.0 / vv : 0.0;
        s_alpha = alpha;
        if (alpha == 0.0) sh.err |= kErrStab;
      }
    }
    __syncthreads();
    la += log(fabs(s_alpha));
    sg *= s_alpha < 0 ? -1.0 : 1.0;
    const double beta = sh.qbeta[j];
    for (int col = j + 1 + warp; col < n; col += nw) {
      double* w = M + (long)col * N;
      double d = 0.0;
      for (int i = j + lane; i < N; i += 32) d += v[i] * w[i];
      d = warp_sum(d) * beta;
      for (int i = j + lane; i < N; i += 32) w[i] -= d * v[i];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < N * n; e += blockDim.x) {
    const int col = e / N, i = e % N;
    Q[e] = (i == col) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const double* v = M + (long)j * N;
    const double beta = sh.qbeta[j];
    for (int col = j + warp; col < n; col += nw) {
      double* w = Q + (long)col * N;
      double d = 0.0;
      for (int i = j + lane; i < N; i += 32) d += v[i] * w[i];
      d = warp_sum(d) * beta;
      for (int i = j + lane; i < N; i += 32) w[i] -= d * v[i];
    }
    __syncthreads();
  }
  logabs = la;
  sgn = sg;
}

// Solve O Y = Y in place by LU with partial pivoting (O: n x n row-major;
// Y: n x ncols row-major, ld ncols).  Returns log|det O| and sign(det O).
template <typename T>
__device__ void lu_solve(Cta<T>& x, int n, int ncols, double* O, double* Y, double& logabs, double& sgn) {
  Smem<T>& sh = x.sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double la = 0.0, sg = 1.0;
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      double best = -1.0;
      int bi = j;
      for (int i = j + lane; i < n; i += 32) {
        const double v = fabs(O[(long)i * n + j]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) sh.piv = bi;
    }
    __syncthreads();
    const int p = sh.piv;
    if (p != j) {
      for (int e = threadIdx.x; e < n + ncols; e += blockDim.x) {
        double* A = e < n ? O : Y;
        const int ldA = e < n ? n : ncols;
        const int col = e < n ? e : e - n;
        const double t = A[(long)j * ldA + col];
        A[(long)j * ldA + col] = A[(long)p * ldA + col];
        A[(long)p * ldA + col] = t;
      }
      sg = -sg;
      __syncthreads();
    }
    const double piv = O[(long)j * n + j];
    if (piv == 0.0) {
      if (threadIdx.x == 0) sh.err |= kErrStab;
      __syncthreads();
      logabs = -INFINITY;
      sgn = 0.0;
      return;
    }
    la += log(fabs(piv));
    sg *= piv < 0 ? -1.0 : 1.0;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) sh.lmul[i] = O[(long)i * n + j] / piv;
    __syncthreads();
    const int w = n - j - 1 + ncols;
    const long total = (long)(n - j - 1) * w;
    for (long e = threadIdx.x; e < total; e += blockDim.x) {
      const int i = j + 1 + (int)(e / w), col = (int)(e % w);
      if (col < n - j - 1)
        O[(long)i * n + j + 1 + col] -= sh.lmul[i] * O[(long)j * n + j + 1 + col];
      else
        Y[(long)i * ncols + col - (n - j - 1)] -= sh.lmul[i] * Y[(long)j * ncols + col - (n - j - 1)];
    }
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    const double inv = 1.0 / O[(long)j * n + j];
    for (int col = threadIdx.x; col < ncols; col += blockDim.x) Y[(long)j * ncols + col] *= inv;
    __syncthreads();
    const long total = (long)j * ncols;
    for (long e = threadIdx.x; e < total; e += blockDim.x) {
      const int i = (int)(e / ncols), col = (int)(e % ncols);
      Y[(long)i * ncols + col] -= O[(long)i * n + j] * Y[(long)j * ncols + col];
    }
    __syncthreads();
  }
  logabs = la;
  sgn = sg;
}

template <typename T>
__device__ double* stack_block(const Cta<T>& x, double* base, int b, int s) {
  return base + ((long)b * 2 + s) * x.c.N * x.c.nmax;
}

// Right stack block b: QR of B_{b n} ... B_{(b-1)n+1} Q_R[b-1] (b >= 1) or of B_0 P (b = 0).
template <typename T>
__device__ void push_R(Cta<T>& x, int b) {
  const ChainDesc& c = x.c;
  const int N = c.N, n_stab = c.n_stab;
  double* M = c.work;
  double* M2 = c.work + (long)N * c.nmax;
  for (int s = 0; s < 2; ++s) {
    const int n = x.nsig(s);
    const double* P = c.P + (long)s * N * c.nmax;
    double prev_l = 0.0, prev_s = 1.0;
    if (b == 0) {
      for (int e = threadIdx.x; e < N * n; e += blockDim.x) M[e] = x.vexp(0, s, e % N) * P[e];
      __syncthreads();
    } else {
      const double* prev = stack_block(x, c.Rst, b - 1, s);
      for (int e = threadIdx.x; e < N * n; e += blockDim.x) M[e] = prev[e];
      prev_l = c.Rlog[((b - 1) * 2 + s) * 2 + 0];
      prev_s = c.Rlog[((b - 1) * 2 + s) * 2 + 1];
      __syncthreads();
      for (int tau = (b - 1) * n_stab + 1; tau <= b * n_stab; ++tau) {
        for (int e = threadIdx.x; e < N * n; e += blockDim.x) M[e] *= x.vexp(tau, s, e % N);
        __syncthreads();
        cta_gemm<double>(N, n, N, c.expKm64, 1, N, M, 1, N, M2, 1, N, EpiStore());
        __syncthreads();
        for (int e = threadIdx.x; e < N * n; e += blockDim.x) M[e] = M2[e];
        __syncthreads();
      }
    }
    double la, sg;
    qr_householder(x, N, n, M, stack_block(x, c.Rst, b, s), la, sg);
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
  double* M = c.work;
  double* M2 = c.work + (long)N * c.nmax;
  for (int s = 0; s < 2; ++s) {
    const int n = x.nsig(s);
    const double* P = c.P + (long)s * N * c.nmax;
    double prev_l = 0.0, prev_s = 1.0;
    if (b == c.nb) {
      for (int e = threadIdx.x; e < N * n; e += blockDim.x) M[e] = x.vexp(c.Ltau + 1, s, e % N) * P[e];
      __syncthreads();
    } else {
      const double* prev = stack_block(x, c.Lst, b + 1, s);
      for (int e = threadIdx.x; e < N * n; e += blockDim.x) M[e] = prev[e];
      prev_l = c.Llog[((b + 1) * 2 + s) * 2 + 0];
      prev_s = c.Llog[((b + 1) * 2 + s) * 2 + 1];
      __syncthreads();
      for (int tau = (b + 1) * n_stab; tau > b * n_stab; --tau) {
        cta_gemm<double>(N, n, N, c.expKm64, 1, N, M, 1, N, M2, 1, N, EpiStore());
        __syncthreads();
        for (int e = threadIdx.x; e < N * n; e += blockDim.x) M[e] = x.vexp(tau, s, e % N) * M2[e];
        __syncthreads();
      }
    }
    double la, sg;
    qr_householder(x, N, n, M, stack_block(x, c.Lst, b, s), la, sg);
    if (threadIdx.x == 0) {
      c.Llog[(b * 2 + s) * 2 + 0] = prev_l + la;
      c.Llog[(b * 2 + s) * 2 + 1] = prev_s * sg;
    }
    __syncthreads();
  }
}

// G <- 1 - Q_R (Q_L^T Q_R)^{-1} Q_L^T at stabilisation point b; records
// max |G - G_fresh| when record != 0, and the weight's log|det| and sign.
template <typename T>
__device__ void refresh(Cta<T>& x, int b, bool record) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  const int N = c.N, ld = c.ld;
  double* O = c.work + 2L * N * c.nmax;
  double* Y = O + (long)c.nmax * c.nmax;
  double dmax = 0.0;
  double sign_total = 1.0;
  for (int s = 0; s < 2; ++s) {
    const int n = x.nsig(s);
    const double* QR = stack_block(x, c.Rst, b, s);
    const double* QL = stack_block(x, c.Lst, b, s);
    cta_gemm<double>(n, n, N, QL, N, 1, QR, 1, N, O, n, 1, EpiStore());
    for (int e = threadIdx.x; e < n * N; e += blockDim.x) Y[e] = QL[e];
    __syncthreads();
    double la, sg;
    lu_solve(x, n, N, O, Y, la, sg);
    // G_fresh = 1 - QR Y, compared with and written over G
    T* Gs = x.G(s);
    const int tm = (N + 3) >> 2;
    for (int t = threadIdx.x; t < tm * tm; t += blockDim.x) {
      const int i0 = (t / tm) << 2, j0 = (t % tm) << 2;
      double acc[4][4] = {};
      for (int k = 0; k < n; ++k) {
        double av[4], bv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = (i0 + r < N) ? QR[(long)k * N + i0 + r] : 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) bv[q] = (j0 + q < N) ? Y[(long)k * N + j0 + q] : 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[r][q] = fma(av[r], bv[q], acc[r][q]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = i0 + r, j = j0 + q;
          if (i < N && j < N) {
            const double g = (i == j ? 1.0 : 0.0) - acc[r][q];
            T& ref = Gs[(long)i * ld + j];
            dmax = fmax(dmax, fabs((double)ref - g));
            ref = (T)g;
          }
        }
    }
    const double l_tot = c.Rlog[(b * 2 + s) * 2 + 0] + la + c.Llog[(b * 2 + s) * 2 + 0];
    const double s_tot = c.Rlog[(b * 2 + s) * 2 + 1] * sg * c.Llog[(b * 2 + s) * 2 + 1];
    if (threadIdx.x == 0) {
      sh.logw_spin[s] = l_tot;
      sh.sign_spin[s] = s_tot;
    }
    sign_total *= s_tot;
    __syncthreads();
  }
  dmax = cta_max(dmax, sh.red);
  if (threadIdx.x == 0) {
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
// docc/site, kinetic/site, with the weight sign and the running sign.
template <typename T>
__device__ void measure(Cta<T>& x) {
  const ChainDesc& c = x.c;
  Smem<T>& sh = x.sh;
  const int N = c.N, ld = c.ld;
  double ek = 0.0, dc = 0.0;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i = e / N, j = e % N;
    const double k = c.K64[e];
    if (k != 0.0) {
      for (int s = 0; s < 2; ++s) ek += k * ((i == j ? 1.0 : 0.0) - (double)x.G(s)[(long)j * ld + i]);
    }
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    dc += (1.0 - (double)x.G(0)[(long)i * ld + i]) * (1.0 - (double)x.G(1)[(long)i * ld + i]);
  ek = cta_sum(ek, sh.red);
  dc = cta_sum(dc, sh.red);
  if (threadIdx.x == 0) {
    const int m = c.st->n_meas;
    if (m < c.max_meas) {
      double* r = c.meas + (long)m * kRecord;
      r[0] = sh.sign_spin[0] * sh.sign_spin[1];
      r[1] = (ek + c.U * dc) / N;
      r[2] = dc / N;
      r[3] = ek / N;
      r[4] = sh.sign_running;
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
    update_slice(x, tau, sweep);
    wrap(x, tau, +1);
    if (tau <= c.Ltau && tau % c.n_stab == 0) {
      const int b = tau / c.n_stab;
      push_R(x, b);
      refresh(x, b, true);
      if (do_measure && tau == c.Ltau / 2) measure(x);
    }
  }
}

template <typename T>
__device__ void sweep_down(Cta<T>& x, uint32_t sweep, bool do_measure) {
  const ChainDesc& c = x.c;
  for (int tau = c.Ltau + 1; tau >= 0; --tau) {
    wrap(x, tau, -1);
    update_slice(x, tau, sweep);
    const int t1 = tau - 1;
    if (t1 >= 0 && t1 % c.n_stab == 0) {
      const int b = t1 / c.n_stab;
      push_L(x, b);
      refresh(x, b, true);
      if (do_measure && t1 == c.Ltau / 2) measure(x);
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
    x.sh.sign_spin[0] = st.logw[0][1];
    x.sh.sign_spin[1] = st.logw[1][1];
    x.sh.logw_spin[0] = st.logw[0][0];
    x.sh.logw_spin[1] = st.logw[1][0];
  }
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
    if (x.sh.err) atomicOr(err, x.sh.err);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) init_kernel(const ChainDesc* chains, int chain0, uint64_t seed, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T>& sh = *reinterpret_cast<Smem<T>*>(smem_raw);
  Cta<T> x{chains[chain0 + blockIdx.x], sh, seed};
  load_state(x);
  const ChainDesc& c = x.c;
  for (int b = c.nb; b >= 0; --b) push_L(x, b);
  push_R(x, 0);
  refresh(x, 0, false);
  if (threadIdx.x == 0) sh.sign_running = sh.sign_spin[0] * sh.sign_spin[1];
  __syncthreads();
  wrap(x, 0, -1);
  store_state(x, err);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) sweep_kernel(const ChainDesc* chains, uint64_t seed, uint32_t sweep0,
                                                         int n_sweeps, int do_measure, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T>& sh = *reinterpret_cast<Smem<T>*>(smem_raw);
  Cta<T> x{chains[blockIdx.x], sh, seed};
  if (x.c.st->err) return;
  load_state(x);
  for (int k = 0; k < n_sweeps; ++k) {
    const uint32_t sw = sweep0 + (uint32_t)k;
    if ((sw & 1u) == 0) sweep_up(x, sw, do_measure != 0);
    else sweep_down(x, sw, do_measure != 0);
    if (sh.err) break;
  }
  store_state(x, err);
}

// --------------------------------------------------------------------------
// host launch wrappers (called from api.cpp)

size_t smem_bytes(int prec) { return prec == 0 ? sizeof(Smem<double>) : sizeof(Smem<float>); }

cudaError_t launch_init(int prec, const ChainDesc* d_chains, int chain0, int n, uint64_t seed, int* d_err,
                        cudaStream_t stream) {
  const size_t sm = smem_bytes(prec);
  if (prec == 0) {
    cudaFuncSetAttribute(init_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    init_kernel<double><<<n, kThreads, sm, stream>>>(d_chains, chain0, seed, d_err);
  } else {
    cudaFuncSetAttribute(init_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    init_kernel<float><<<n, kThreads, sm, stream>>>(d_chains, chain0, seed, d_err);
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep(int prec, const ChainDesc* d_chains, int n, uint64_t seed, uint32_t sweep0, int n_sweeps,
                         int measure, int* d_err, cudaStream_t stream) {
  const size_t sm = smem_bytes(prec);
  if (prec == 0) {
    cudaFuncSetAttribute(sweep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    sweep_kernel<double><<<n, kThreads, sm, stream>>>(d_chains, seed, sweep0, n_sweeps, measure, d_err);
  } else {
    cudaFuncSetAttribute(sweep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    sweep_kernel<float><<<n, kThreads, sm, stream>>>(d_chains, seed, sweep0, n_sweeps, measure, d_err);
  }
  return cudaGetLastError();
}

}  // namespace pqmc

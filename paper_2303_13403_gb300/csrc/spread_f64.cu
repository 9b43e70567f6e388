// Spread sweep (spread.cuh): the FP64 path's kernel sequence and the FP64
// stabilisation steps that both paths call.
#include "spread.cuh"

namespace pqmc {

namespace {

__device__ __forceinline__ SpBuf<double> fp64_bufs(const ChainDesc& c, int tsize) {
  return SpBuf<double>(c.spread, c.N, c.ld, c.nmax, tsize);
}
__device__ __forceinline__ int nsig_of(const ChainDesc& c, int s) { return s == 0 ? c.nup : c.ndn; }

// Cholesky factor, diagonal block of panel p (one CTA per spin, chain), on a
// shared-memory copy: step k takes the pivot C_kk, writes row k of R
// (R_kj = C_kj / sqrt(C_kk)) and then updates the rows below by
// C_ij -= R_ki R_kj (one FP64 instruction per element); then R_PP^{-1} by
// back substitution on the identity, one barrier per row.  Panel 0 first records the Gram diagonal and clears the chain's
// breakdown flag and log det R.
__global__ void __launch_bounds__(256) chol_panel_kernel(const ChainDesc* chains, int p, int tsize) {
  __shared__ double A[kSpPanel][kSpPanel + 1];    // Schur complements
  __shared__ double R[kSpPanel][kSpPanel + 1];    // the factor's rows
  __shared__ double X[1][kSpPanel][kSpPanel + 1]; // inverse, rows in progress
  __shared__ double Xf[kSpPanel][kSpPanel + 1];   // its final rows
  __shared__ double ikk[kSpPanel];
  __shared__ int bad;
  const ChainDesc& c = chains[blockIdx.y];
  if (c.st->err) return;
  const int s = blockIdx.x, n = nsig_of(c, s), ldn = c.nmax;
  const int p0 = p * kSpPanel;
  if (p0 >= n) return;
  const int p1 = min(p0 + kSpPanel, n), bw = p1 - p0;
  SpBuf<double> sp = fp64_bufs(c, tsize);
  double* C = sp.c64(s);
  double* d0 = sp.d0(s);
  if (p == 0) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) d0[k] = C[(long)k * ldn + k];
    if (threadIdx.x == 0) {
      sp.bad()[s] = 0;
      sp.lchol()[s] = 0.0;
    }
  }
  __shared__ double dlim[kSpPanel];
  __syncthreads();
  for (int e = threadIdx.x; e < kSpPanel * kSpPanel; e += blockDim.x) {
    const int i = e / kSpPanel, j = e % kSpPanel;
    A[i][j] = (i < bw && j < bw) ? C[(long)(p0 + i) * ldn + p0 + j] : 0.0;
    R[i][j] = 0.0;
  }
  if ((int)threadIdx.x < bw) dlim[threadIdx.x] = 1e-12 * d0[p0 + threadIdx.x];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // upper-triangle pairs (i, j), i <= j, of the trailing block, enumerated so
  // that every FP64 instruction carries a full warp (the FP64 unit takes as
  // long for a partial warp)
  for (int k = 0; k < bw; ++k) {
    const double piv = A[k][k];
    if (!(piv > dlim[k])) {   // the same value in every thread: uniform exit
      if (threadIdx.x == 0) bad = 1;
      break;
    }
    const double ir = rsqrt(piv);
    if ((int)threadIdx.x >= k && (int)threadIdx.x < bw) R[k][threadIdx.x] = threadIdx.x == k ? piv * ir : A[k][threadIdx.x] * ir;
    __syncthreads();
    const int m = bw - k - 1;
    for (int e = threadIdx.x; e < m * (m + 1) / 2; e += blockDim.x) {
      int i = 0, r = e;
      while (r >= m - i) { r -= m - i; ++i; }
      const int ii = k + 1 + i, jj = ii + r;
      A[ii][jj] = fma(-R[k][ii], R[k][jj], A[ii][jj]);
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) sp.bad()[s] = 1;
    return;
  }
  for (int e = threadIdx.x; e < bw * bw; e += blockDim.x) {
    const int i = e / bw, j = e % bw;
    if (i <= j) C[(long)(p0 + i) * ldn + p0 + j] = R[i][j];
  }
  if (threadIdx.x < 32) {
    // log det R_PP: one logarithm per lane, summed over the warp
    double la = (int)threadIdx.x < bw ? log(R[threadIdx.x][threadIdx.x]) : 0.0;
    la = warp_sum(la);
    if (threadIdx.x == 0) sp.lchol()[s] += la;
  }
  // X = R_PP^{-1} by back substitution on the identity: for k = bw-1 .. 0,
  // row k of X is final once scaled by 1 / R_kk (kept in Xf), then the rows
  // i < k take away R_ik times it (one FP64 instruction per element)
  for (int e = threadIdx.x; e < kSpPanel * kSpPanel; e += blockDim.x) {
    const int i = e / kSpPanel, j = e % kSpPanel;
    X[0][i][j] = (i == j && i < bw) ? 1.0 : 0.0;
    Xf[i][j] = 0.0;
  }
  if ((int)threadIdx.x < bw) ikk[threadIdx.x] = 1.0 / R[threadIdx.x][threadIdx.x];
  __syncthreads();
  for (int k = bw - 1; k >= 0; --k) {
    if ((int)threadIdx.x < bw) Xf[k][threadIdx.x] = X[0][k][threadIdx.x] * ikk[k];
    __syncthreads();
    for (int e = threadIdx.x; e < k * bw; e += blockDim.x) {
      const int i = e / bw, j = e % bw;
      X[0][i][j] = fma(-R[i][k], Xf[k][j], X[0][i][j]);
    }
    __syncthreads();
  }
  double* Ri = sp.rinv(s) + (long)p * kSpPanel * kSpPanel;
  for (int e = threadIdx.x; e < kSpPanel * kSpPanel; e += blockDim.x) {
    const int i = e / kSpPanel, j = e % kSpPanel;
    Ri[e] = (i < bw && j < bw) ? Xf[i][j] : 0.0;
  }
}

// Q = M R^{-1}, one warp per row i of M: panel by panel, t = m_P - q_{<P} R_{<P,P}
// (lane j: column p0 + j), then q_P = t R_PP^{-1}; the eight rows of a CTA
// are written to the column-major stack block together
__global__ void __launch_bounds__(256) qform_kernel(const ChainDesc* chains, int left, int b, int tsize) {
  __shared__ double q[8][kMaxSigma];
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int s = blockIdx.y, n = nsig_of(c, s), ldn = c.nmax, N = c.N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 8, i = i0 + w;
  SpBuf<double> sp = fp64_bufs(c, tsize);
  const double* M = sp.m64(s);
  const double* C = sp.c64(s);
  const double* Ri = sp.rinv(s);
  if (i < N) {
    for (int p0 = 0; p0 < n; p0 += kSpPanel) {
      const int bw = min(kSpPanel, n - p0), j = lane;
      double t = 0.0;
      if (j < bw) {
        double a0 = M[(long)(p0 + j) * N + i], a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int l = 0;
        for (; l + 4 <= p0; l += 4) {
          a0 = fma(-q[w][l], C[(long)l * ldn + p0 + j], a0);
          a1 = fma(-q[w][l + 1], C[(long)(l + 1) * ldn + p0 + j], a1);
          a2 = fma(-q[w][l + 2], C[(long)(l + 2) * ldn + p0 + j], a2);
          a3 = fma(-q[w][l + 3], C[(long)(l + 3) * ldn + p0 + j], a3);
        }
        for (; l < p0; ++l) a0 = fma(-q[w][l], C[(long)l * ldn + p0 + j], a0);
        t = (a0 + a1) + (a2 + a3);
      }
      const double* Rp = Ri + (long)(p0 / kSpPanel) * kSpPanel * kSpPanel;
      double acc = 0.0;
      for (int l = 0; l < bw; ++l) {
        const double tl = __shfl_sync(0xffffffffu, t, l);
        if (l <= j && j < bw) acc = fma(tl, Rp[l * kSpPanel + j], acc);
      }
      if (j < bw) q[w][p0 + j] = acc;
      __syncwarp();
    }
  }
  __syncthreads();
  double* Q = (left ? c.Lst : c.Rst) + ((long)b * 2 + s) * N * c.nmax;
  const int rows = min(8, N - i0);
  for (int e = threadIdx.x; e < n * 8; e += blockDim.x) {
    const int k = e >> 3, r = e & 7;
    if (r < rows) Q[(long)k * N + i0 + r] = q[r][k];
  }
}

// Gauss-Jordan panel p (columns P = [p0, p1)) of O, one CTA per spin, chain:
// for each column j of P the largest |O_ij|, i >= j (ties to the lower row),
// the interchange of rows j and i, then the elimination of column j
// restricted to the panel's columns (the rest of the row operations is the
// block update that follows, from the block row saved at the end).  The
// panel stays in shared memory for all its steps, each thread owning one
// panel column on every 16th row (one FP64 FMA per eliminated element); the
// pass that eliminates column j also hands on column j + 1 and its pivot
// candidates, so a step takes two CTA barriers.  The interchanges reach the
// other columns once, in order, at the end.
constexpr int kGJLd = kSpGJ + 1;
constexpr int kGJThreads = 512;
constexpr int kGJRowStep = kGJThreads / kSpGJ;
static_assert(kGJThreads % kSpGJ == 0 && kSpGJ <= 32, "each thread owns one panel column");
size_t gj_panel_smem(int nmax) { return (size_t)nmax * kGJLd * 8; }

__global__ void __launch_bounds__(kGJThreads) gj_panel_kernel(const ChainDesc* chains, int p, int tsize) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double (*Ap)[kGJLd] = reinterpret_cast<double (*)[kGJLd]>(smem_raw);   // n x bw panel
  __shared__ double fbuf[2][kMaxSigma];   // column j of the panel before step j (two steps in flight)
  __shared__ double prow[kSpGJ];          // pivot row of the step, after the interchange
  __shared__ double ips;
  __shared__ unsigned long long wbest[kGJThreads / 32];
  __shared__ int wbi[kGJThreads / 32];
  __shared__ int piv[kSpGJ];
  const ChainDesc& c = chains[blockIdx.y];
  if (c.st->err) return;
  const int s = blockIdx.x, n = nsig_of(c, s), ldn = c.nmax;
  const int p0 = p * kSpGJ;
  if (p0 >= n) return;
  const int p1 = min(p0 + kSpGJ, n), bw = p1 - p0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = threadIdx.x % kSpGJ, row0 = threadIdx.x / kSpGJ;
  SpBuf<double> sp = fp64_bufs(c, tsize);
  double* A = sp.o64(s);
  // load; the owners of column 0 hand it on with its pivot candidates
  unsigned long long best = 0;
  int bi = p0;
  for (int i = row0; i < n; i += kGJRowStep) {
    if (col < bw) {
      const double v = A[(long)i * ldn + p0 + col];
      Ap[i][col] = v;
      if (col == 0) {
        fbuf[0][i] = v;
        const unsigned long long av = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
        if (i >= p0 && av > best) { best = av; bi = i; }
      }
    }
  }
  for (int jj = 0; jj < bw; ++jj) {
    const int j = p0 + jj;
    double* f = fbuf[jj & 1];
    double* fnext = fbuf[(jj + 1) & 1];
    // candidates of column j: per warp, then warp 0 over the warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { wbest[warp] = best; wbi[warp] = bi; }
    __syncthreads();
    if (threadIdx.x < 32) {
      unsigned long long bb = 0;
      int ii = j;
      if (lane < kGJThreads / 32) { bb = wbest[lane]; ii = wbi[lane]; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bb, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ii, o);
        if (ob > bb || (ob == bb && oi < ii)) { bb = ob; ii = oi; }
      }
      if (ii != j) {
        if (lane < bw) {
          const double t = Ap[j][lane];
          Ap[j][lane] = Ap[ii][lane];
          Ap[ii][lane] = t;
        }
        if (lane == 0) {
          const double t = f[j];
          f[j] = f[ii];
          f[ii] = t;
        }
      }
      __syncwarp();
      if (lane < bw) prow[lane] = Ap[j][lane];
      if (lane == 0) {
        const double pv = Ap[j][jj];
        ips = pv != 0.0 ? 1.0 / pv : 0.0;
        piv[jj] = ii;
        sp.perm(s)[j] = ii;
        sp.pval(s)[j] = pv;
        if (pv == 0.0) sp.bad()[s] = 1;
      }
    }
    __syncthreads();
    // eliminate column j from the panel; the owners of column j + 1 hand it on
    const double ip = ips;
    best = 0;
    bi = j + 1;
    if (col < bw) {
      // one FP64 instruction per element: v = add - f_i x with (x, add) =
      // (1 / pivot, 0) on the pivot column, (pivot row / pivot, O_ic) elsewhere
      const bool pc = col == jj;
      const double x = pc ? ip : prow[col] * ip;
      for (int i = row0; i < n; i += kGJRowStep) {
        const double add = pc ? 0.0 : Ap[i][col];
        const double v = i == j ? x : fma(-f[i], x, add);
        Ap[i][col] = v;
        if (col == jj + 1) {
          fnext[i] = v;
          const unsigned long long av = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
          if (i > j && av > best) { best = av; bi = i; }
        }
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * bw; e += blockDim.x) A[(long)(e / bw) * ldn + p0 + e % bw] = Ap[e / bw][e % bw];
  // the panel back; the other columns take the panel's interchanges composed
  // into one permutation of at most 2 bw rows (new row rows[e] = old row
  // src[e]), read once and written once, and the block row of the update
  __shared__ int rows[2 * kSpGJ], src[2 * kSpGJ], nrows;
  if (threadIdx.x == 0) {
    int m = 0;
    for (int jj = 0; jj < bw; ++jj) { rows[m] = p0 + jj; src[m] = p0 + jj; ++m; }
    for (int jj = 0; jj < bw; ++jj) {
      const int j = p0 + jj, r = piv[jj];
      if (r == j) continue;
      int ej = -1, er = -1;
      for (int e = 0; e < m; ++e) {
        if (rows[e] == j) ej = e;
        if (rows[e] == r) er = e;
      }
      if (er < 0) { rows[m] = r; src[m] = r; er = m++; }
      const int t = src[ej];
      src[ej] = src[er];
      src[er] = t;
    }
    nrows = m;
  }
  __syncthreads();
  const int m = nrows;
  double* Tb = sp.tgj(s);
  for (int col = threadIdx.x; col < n; col += blockDim.x) {
    if (col >= p0 && col < p1) continue;
    double v[2 * kSpGJ];
#pragma unroll
    for (int e = 0; e < 2 * kSpGJ; ++e)
      if (e < m) v[e] = A[(long)src[e] * ldn + col];
#pragma unroll
    for (int e = 0; e < 2 * kSpGJ; ++e)
      if (e < m) {
        A[(long)rows[e] * ldn + col] = v[e];
        if (e < bw) Tb[(long)e * ldn + col] = v[e];   // rows[e] = p0 + e for e < bw
      }
  }
}

// row i: the interchanges of the elimination applied to the columns, last first
__global__ void __launch_bounds__(128) gj_unswap_kernel(const ChainDesc* chains, int tsize) {
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int s = blockIdx.y, n = nsig_of(c, s), ldn = c.nmax;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  SpBuf<double> sp = fp64_bufs(c, tsize);
  double* A = sp.o64(s) + (long)i * ldn;
  const int* perm = sp.perm(s);
  for (int j = n - 1; j >= 0; --j) {
    const int q = perm[j];
    if (q != j) {
      const double t = A[j];
      A[j] = A[q];
      A[q] = t;
    }
  }
}

}  // namespace

cudaError_t sp_dgemm(SpGemm& g, int mode, int max_m, int max_n, cudaStream_t st) {
  return sp_gemm_t<double>(g, mode, max_m, max_n, st);
}

cudaError_t sp_chol_panel(const ChainDesc* d, int nc, int nmax, int p, int tsize, cudaStream_t st) {
  (void)nmax;
  chol_panel_kernel<<<dim3(2, nc), 256, 0, st>>>(d, p, tsize);
  return cudaGetLastError();
}

cudaError_t sp_qform(const ChainDesc* d, int nc, int N, int nmax, int left, int b, int tsize, cudaStream_t st) {
  (void)nmax;
  qform_kernel<<<dim3((N + 7) / 8, 2, nc), 256, 0, st>>>(d, left, b, tsize);
  return cudaGetLastError();
}

cudaError_t sp_gj_panel(const ChainDesc* d, int nc, int nmax, int p, int tsize, cudaStream_t st) {
  gj_panel_kernel<<<dim3(2, nc), kGJThreads, gj_panel_smem(nmax), st>>>(d, p, tsize);
  return cudaGetLastError();
}

cudaError_t spread_prepare() {
  return cudaFuncSetAttribute(gj_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gj_panel_smem(kMaxSigma));
}

cudaError_t sp_gj_unswap(const ChainDesc* d, int nc, int nmax, int tsize, cudaStream_t st) {
  gj_unswap_kernel<<<dim3((nmax + 127) / 128, 2, nc), 128, 0, st>>>(d, tsize);
  return cudaGetLastError();
}

cudaError_t spread_sweep_f64(const SpreadPlan& p, int mode, int measure, cudaStream_t st) {
  return spread_sweep_t<double>(p, mode, measure, st);
}

}  // namespace pqmc

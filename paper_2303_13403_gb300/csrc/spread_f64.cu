// Spread sweep (spread.cuh): the FP64 path's kernel sequence and the FP64
// stabilisation steps that both paths call.
#include "spread.cuh"

namespace pqmc {

namespace {

__device__ __forceinline__ SpBuf<double> fp64_bufs(const ChainDesc& c, int tsize) {
  return SpBuf<double>(c.spread, c.N, c.ld, c.nmax, tsize);
}
__device__ __forceinline__ int nsig_of(const ChainDesc& c, int s) { return s == 0 ? c.nup : c.ndn; }

// Cholesky factor, diagonal block of panel p (one CTA per spin, chain):
// right-looking on a shared-memory copy, R_kk = sqrt(pivot), R_kj = C_kj / R_kk,
// C_ij -= R_ki R_kj inside the block.  Panel 0 first records the Gram
// diagonal and clears the chain's breakdown flag and log det R.
__global__ void __launch_bounds__(256) chol_panel_kernel(const ChainDesc* chains, int p, int tsize) {
  __shared__ double A[kSpPanel][kSpPanel + 1];
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
  for (int e = threadIdx.x; e < bw * bw; e += blockDim.x) A[e / bw][e % bw] = C[(long)(p0 + e / bw) * ldn + p0 + e % bw];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < bw; ++k) {
    const double piv = A[k][k];
    if (!(piv > 1e-12 * d0[p0 + k])) {   // the same value in every thread: uniform exit
      if (threadIdx.x == 0) bad = 1;
      break;
    }
    const double r = sqrt(piv), ir = 1.0 / r;
    __syncthreads();
    for (int j = k + 1 + (int)threadIdx.x; j < bw; j += blockDim.x) A[k][j] *= ir;
    if (threadIdx.x == 0) A[k][k] = r;
    __syncthreads();
    const int m = bw - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (i <= j) A[i][j] = fma(-A[k][i], A[k][j], A[i][j]);
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
    if (i <= j) C[(long)(p0 + i) * ldn + p0 + j] = A[i][j];
  }
  if (threadIdx.x == 0) {
    double la = 0.0;
    for (int k = 0; k < bw; ++k) la += log(A[k][k]);
    sp.lchol()[s] += la;
  }
}

// block row of R: column j >= p1 solves R_PP^T x = C_{P,j} by forward
// substitution (one thread per column)
__global__ void __launch_bounds__(128) chol_rows_kernel(const ChainDesc* chains, int p, int tsize) {
  __shared__ double R[kSpPanel][kSpPanel + 1];
  __shared__ double ir[kSpPanel];
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int s = blockIdx.y, n = nsig_of(c, s), ldn = c.nmax;
  const int p0 = p * kSpPanel;
  if (p0 >= n) return;
  const int p1 = min(p0 + kSpPanel, n), bw = p1 - p0;
  if (p1 + (int)(blockIdx.x * blockDim.x) >= n) return;
  SpBuf<double> sp = fp64_bufs(c, tsize);
  double* C = sp.c64(s);
  for (int e = threadIdx.x; e < bw * bw; e += blockDim.x) R[e / bw][e % bw] = C[(long)(p0 + e / bw) * ldn + p0 + e % bw];
  __syncthreads();
  if ((int)threadIdx.x < bw) ir[threadIdx.x] = 1.0 / R[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int j = p1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double x[kSpPanel];
#pragma unroll
  for (int k = 0; k < kSpPanel; ++k) {
    if (k < bw) {
      double v = C[(long)(p0 + k) * ldn + j];
#pragma unroll
      for (int l = 0; l < kSpPanel; ++l)
        if (l < k) v = fma(-R[l][k], x[l], v);
      x[k] = v * ir[k];
      C[(long)(p0 + k) * ldn + j] = x[k];
    }
  }
}

// inverse of the upper-triangular diagonal block of panel p = blockIdx.x
// (thread j: column j by back substitution), row-major kSpPanel x kSpPanel
__global__ void __launch_bounds__(32) tri_inv_kernel(const ChainDesc* chains, int tsize) {
  __shared__ double R[kSpPanel][kSpPanel + 1];
  __shared__ double X[kSpPanel][kSpPanel + 1];
  const ChainDesc& c = chains[blockIdx.z];
  if (c.st->err) return;
  const int s = blockIdx.y, n = nsig_of(c, s), ldn = c.nmax;
  const int p = blockIdx.x, p0 = p * kSpPanel;
  if (p0 >= n) return;
  const int bw = min(kSpPanel, n - p0);
  SpBuf<double> sp = fp64_bufs(c, tsize);
  const double* C = sp.c64(s);
  for (int e = threadIdx.x; e < kSpPanel * kSpPanel; e += blockDim.x) {
    const int i = e / kSpPanel, j = e % kSpPanel;
    R[i][j] = (i < bw && j < bw && i <= j) ? C[(long)(p0 + i) * ldn + p0 + j] : 0.0;
    X[i][j] = 0.0;
  }
  __syncwarp();
  const int j = threadIdx.x;
  if (j < bw) {
    X[j][j] = 1.0 / R[j][j];
    for (int i = j - 1; i >= 0; --i) {
      double v = 0.0;
      for (int k = i + 1; k <= j; ++k) v = fma(R[i][k], X[k][j], v);
      X[i][j] = -v / R[i][i];
    }
  }
  __syncwarp();
  double* Ri = sp.rinv(s) + (long)p * kSpPanel * kSpPanel;
  for (int e = threadIdx.x; e < kSpPanel * kSpPanel; e += blockDim.x) Ri[e] = X[e / kSpPanel][e % kSpPanel];
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
// the interchange of rows j and i over all columns, then the elimination of
// column j restricted to the panel's columns (the rest of the row operations
// is the block update that follows, from the block row saved at the end)
__global__ void __launch_bounds__(256) gj_panel_kernel(const ChainDesc* chains, int p, int tsize) {
  __shared__ double f[kMaxSigma];
  __shared__ unsigned long long wbest[8];
  __shared__ int wbi[8];
  __shared__ int piv;
  const ChainDesc& c = chains[blockIdx.y];
  if (c.st->err) return;
  const int s = blockIdx.x, n = nsig_of(c, s), ldn = c.nmax;
  const int p0 = p * kSpGJ;
  if (p0 >= n) return;
  const int p1 = min(p0 + kSpGJ, n), bw = p1 - p0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  SpBuf<double> sp = fp64_bufs(c, tsize);
  double* A = sp.o64(s);
  for (int j = p0; j < p1; ++j) {
    unsigned long long best = 0;
    int bi = j;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(A[(long)i * ldn + j]) & 0x7fffffffffffffffull;
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { wbest[warp] = best; wbi[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long bb = wbest[0];
      int ii = wbi[0];
      for (int u = 1; u < nw; ++u)
        if (wbest[u] > bb || (wbest[u] == bb && wbi[u] < ii)) { bb = wbest[u]; ii = wbi[u]; }
      piv = ii;
      sp.perm(s)[j] = ii;
    }
    __syncthreads();
    const int r = piv;
    if (r != j)
      for (int col = threadIdx.x; col < n; col += blockDim.x) {
        const double t = A[(long)j * ldn + col];
        A[(long)j * ldn + col] = A[(long)r * ldn + col];
        A[(long)r * ldn + col] = t;
      }
    __syncthreads();
    const double pv = A[(long)j * ldn + j];
    const double ip = pv != 0.0 ? 1.0 / pv : 0.0;
    if (threadIdx.x == 0) {
      sp.pval(s)[j] = pv;
      if (pv == 0.0) sp.bad()[s] = 1;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = A[(long)i * ldn + j];
    __syncthreads();
    for (int col = p0 + threadIdx.x; col < p1; col += blockDim.x)
      A[(long)j * ldn + col] = col == j ? ip : A[(long)j * ldn + col] * ip;
    __syncthreads();
    for (int e = threadIdx.x; e < n * bw; e += blockDim.x) {
      const int i = e / bw, col = p0 + e % bw;
      if (i == j) continue;
      const double add = col == j ? 0.0 : A[(long)i * ldn + col];
      A[(long)i * ldn + col] = fma(-f[i], A[(long)j * ldn + col], add);
    }
    __syncthreads();
  }
  double* Tb = sp.tgj(s);
  for (int e = threadIdx.x; e < bw * n; e += blockDim.x) {
    const int l = e / n, col = e % n;
    Tb[(long)l * ldn + col] = A[(long)(p0 + l) * ldn + col];
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

cudaError_t sp_chol_rows(const ChainDesc* d, int nc, int nmax, int p, int tsize, cudaStream_t st) {
  const int rest = nmax - std::min(nmax, (p + 1) * kSpPanel);
  if (rest <= 0) return cudaSuccess;
  chol_rows_kernel<<<dim3((rest + 127) / 128, 2, nc), 128, 0, st>>>(d, p, tsize);
  return cudaGetLastError();
}

cudaError_t sp_qform(const ChainDesc* d, int nc, int N, int nmax, int left, int b, int tsize, cudaStream_t st) {
  tri_inv_kernel<<<dim3((nmax + kSpPanel - 1) / kSpPanel, 2, nc), 32, 0, st>>>(d, tsize);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  qform_kernel<<<dim3((N + 7) / 8, 2, nc), 256, 0, st>>>(d, left, b, tsize);
  return cudaGetLastError();
}

cudaError_t sp_gj_panel(const ChainDesc* d, int nc, int p, int tsize, cudaStream_t st) {
  gj_panel_kernel<<<dim3(2, nc), 256, 0, st>>>(d, p, tsize);
  return cudaGetLastError();
}

cudaError_t sp_gj_unswap(const ChainDesc* d, int nc, int nmax, int tsize, cudaStream_t st) {
  gj_unswap_kernel<<<dim3((nmax + 127) / 128, 2, nc), 128, 0, st>>>(d, tsize);
  return cudaGetLastError();
}

cudaError_t spread_sweep_f64(const SpreadPlan& p, int parity, int measure, cudaStream_t st) {
  return spread_sweep_t<double>(p, parity, measure, st);
}

}  // namespace pqmc

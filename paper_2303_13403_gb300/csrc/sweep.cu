// Host side of the sweep kernels: shared-memory budgets, the precision and
// CTA-shape dispatch over the per-path translation units, the sweep-index
// advance kernel, and the allocation-free single-chain initialisation.
#include "spread.h"
#include "sweep_kernels.cuh"

namespace pqmc {

// --------------------------------------------------------------------------
// host launch wrappers (called from api.cpp)

size_t smem_fixed(int prec) { return prec == 0 ? al16(sizeof(Smem<double>)) : al16(sizeof(Smem<float>)); }

// CTAs per SM a launch is built for: the reduced paths pack twice as many
// chains per SM as the FP64 path (their FP32 work and the FP64 stabilisation of
// different chains overlap); smaller CTAs pack more chains.
int ctas_per_sm(int prec, int tpb, int boost) {
  if (tpb >= 512) return 1;
  return (256 / tpb) * (prec == 0 ? 1 : 2) * (boost ? 2 : 1);
}

// BF16X3 launches of 512-thread CTAs reserve the tensor-core staging area
int tc_launch(int prec, int tpb) { return (prec == 2 && tpb == 512) ? 1 : 0; }

// Largest resident footprint a launch offers per chain.
size_t smem_resident_cap(int prec, int tpb, int boost) {
  const size_t per_sm = 233472, reserve = 1024;
  size_t per_cta = per_sm / ctas_per_sm(prec, tpb, boost) - reserve;
  if (tc_launch(prec, tpb)) per_cta -= kTcBytes + 128;
  const size_t fixed = smem_fixed(prec);
  return per_cta > fixed ? per_cta - fixed : 0;
}

// The sweep index lives in device memory (sweep_ctr) and is advanced by a
// one-thread kernel after each sweep launch, so that the pair can be captured
// once in a CUDA graph and replayed.
__global__ void advance_sweep_kernel(uint32_t* sweep_ctr, int n) { *sweep_ctr += (uint32_t)n; }

cudaError_t launch_advance(uint32_t* sweep_ctr, int n, cudaStream_t stream) {
  advance_sweep_kernel<<<1, 1, 0, stream>>>(sweep_ctr, n);
  return cudaGetLastError();
}

cudaError_t launch_init(int prec, int tpb, int boost, const ChainDesc* d_chains, int chain0, int n, uint64_t seed,
                        size_t res, int* d_err, cudaStream_t stream, int b_at) {
  if (prec == 0) return launch_init_f64(tpb, d_chains, chain0, n, seed, res, d_err, stream, b_at);
  if (boost) return launch_init_f32_dense(tpb, d_chains, chain0, n, seed, res, d_err, stream, b_at);
  if (tpb == 256) return launch_init_f32_256(tpb, d_chains, chain0, n, seed, res, d_err, stream, b_at);
  if (tpb == 512) return launch_init_f32_512(tpb, d_chains, chain0, n, seed, res, d_err, stream, b_at);
  return launch_init_f32(tpb, d_chains, chain0, n, seed, res, d_err, stream, b_at);
}

cudaError_t prepare_sweep(int prec, int tpb, int boost, size_t res) {
  if (prec == 0) return prepare_sweep_f64(tpb, res, 0);
  if (boost) return prepare_sweep_f32_dense(tpb, res, 0);
  if (tpb == 256) return prepare_sweep_f32_256(tpb, res, tc_launch(prec, tpb));
  if (tpb == 512) return prepare_sweep_f32_512(tpb, res, tc_launch(prec, tpb));
  return prepare_sweep_f32(tpb, res, tc_launch(prec, tpb));
}

cudaError_t launch_sweep(int prec, int tpb, int boost, const ChainDesc* d_chains, int n, uint64_t seed,
                         uint32_t* sweep_ctr, int n_sweeps, int measure, size_t res, int* d_err, cudaStream_t stream) {
  if (prec == 0) return launch_sweep_f64(tpb, d_chains, n, seed, sweep_ctr, n_sweeps, measure, res, d_err, stream, 0);
  if (boost)
    return launch_sweep_f32_dense(tpb, d_chains, n, seed, sweep_ctr, n_sweeps, measure, res, d_err, stream, 0);
  if (tpb == 256)
    return launch_sweep_f32_256(tpb, d_chains, n, seed, sweep_ctr, n_sweeps, measure, res, d_err, stream,
                                tc_launch(prec, tpb));
  if (tpb == 512)
    return launch_sweep_f32_512(tpb, d_chains, n, seed, sweep_ctr, n_sweeps, measure, res, d_err, stream,
                                tc_launch(prec, tpb));
  return launch_sweep_f32(tpb, d_chains, n, seed, sweep_ctr, n_sweeps, measure, res, d_err, stream,
                          tc_launch(prec, tpb));
}

// chains swept by grid-wide kernel sequences (spread_f64.cu, spread_f32.cu)
cudaError_t spread_sweep_f64(const SpreadPlan& p, int mode, int measure, cudaStream_t st);
cudaError_t spread_sweep_f32(const SpreadPlan& p, int mode, int measure, cudaStream_t st);
cudaError_t spread_sweep(const SpreadPlan& p, int parity, int measure, cudaStream_t st) {
  return p.prec == PQMC_FP64 ? spread_sweep_f64(p, parity & 1, measure, st) : spread_sweep_f32(p, parity & 1, measure, st);
}
cudaError_t spread_init(const SpreadPlan& p, cudaStream_t st) {
  return p.prec == PQMC_FP64 ? spread_sweep_f64(p, 2, 0, st) : spread_sweep_f32(p, 2, 0, st);
}

// --------------------------------------------------------------------------
// Test kernel of the tensor-core split-BF16 GEMM (pqmc_test_tc_gemm).

__global__ void __launch_bounds__(512, 1) tc_gemm_test_kernel(int M, int N, int K, const float* A, int trans_a,
                                                             const float* B, float* C, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* st = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  const uint32_t tmem = tc_alloc(st);
  if (trans_a) cta_gemm_tc(M, N, K, A, 1, M, B, N, 1, C, N, 1, EpiStore(), st, tmem, err, kErrTimeout);
  else cta_gemm_tc(M, N, K, A, K, 1, B, N, 1, C, N, 1, EpiStore(), st, tmem, err, kErrTimeout);
  tc_free(tmem);
}

// --------------------------------------------------------------------------
// Allocation-free initialisation of one chain (pqmc_green_noalloc).
//
// Runs init_kernel for a single FP64 chain with every buffer the kernel needs
// (its descriptor and counters, the model tables, the left/right stacks, G
// and the phase scratch) placed in one file-scope device array instead of
// memory obtained from cudaMalloc.  The caller supplies the fields and the
// output buffers.  Host code never uses the array's name as an address: the
// device address comes from cudaGetSymbolAddress, once per device.

constexpr size_t kNoAllocBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

pqmc_status check_spec(const pqmc_chain_spec& s, int n_stab, std::string& why);
void set_init_error(const std::string& msg);

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[256];
bool g_noalloc_ready[256];

size_t take256(size_t& off, size_t bytes) {
  const size_t at = off;
  off = (off + bytes + 255) & ~(size_t)255;
  return at;
}
}  // namespace

}  // namespace pqmc

extern "C" pqmc_status pqmc_green_noalloc(const pqmc_chain_spec* spec, int n_stab, const int8_t* d_fields,
                                          double* d_G, double* d_logw, void* stream) {
  using namespace pqmc;
  if (!spec || !d_fields || !d_G || !d_logw) {
    set_init_error("pqmc_green_noalloc: NULL argument");
    return PQMC_EINVAL;
  }
  std::string why;
  if (check_spec(*spec, n_stab, why) != PQMC_OK) {
    set_init_error("pqmc_green_noalloc: " + why);
    return PQMC_EINVAL;
  }
  const pqmc_lattice& lt = spec->lattice;
  if (lt.kind == PQMC_HONEYCOMB_TV) {
    set_init_error("pqmc_green_noalloc: Hubbard lattices only");
    return PQMC_EINVAL;
  }
  const int N = lt.kind == PQMC_HONEYCOMB ? 2 * lt.Lx * lt.Ly : lt.Lx * lt.Ly;
  const int ld = (N + 3) & ~3;
  const int nup = spec->trial.N_up < 0 ? N / 2 : spec->trial.N_up;
  const int ndn = spec->trial.N_dn < 0 ? N / 2 : spec->trial.N_dn;
  const int nmax = nup > ndn ? nup : ndn;
  const int Ltau = (int)std::lround(spec->two_theta / spec->dtau);
  const int nb = Ltau / n_stab;
  const size_t blk = (size_t)N * nmax * 8;

  // layout inside the static array
  size_t off = 0;
  const size_t o_desc = take256(off, sizeof(ChainDesc));
  const size_t o_state = take256(off, sizeof(ChainState));
  const size_t o_err = take256(off, sizeof(int));
  const size_t o_em = take256(off, (size_t)N * ld * 8);
  const size_t o_ep = take256(off, (size_t)N * ld * 8);
  const size_t o_em64 = take256(off, (size_t)N * N * 8);
  const size_t o_k64 = take256(off, (size_t)N * N * 8);
  const size_t o_P = take256(off, 2 * blk);
  const size_t upload = off;                   // everything above is uploaded each call
  const size_t o_rst = take256(off, (size_t)(nb + 1) * 2 * blk);
  const size_t o_lst = take256(off, (size_t)(nb + 1) * 2 * blk);
  const size_t o_rlog = take256(off, (size_t)(nb + 1) * 4 * 8);
  const size_t o_llog = take256(off, (size_t)(nb + 1) * 4 * 8);
  const size_t o_G = take256(off, 2 * (size_t)N * ld * 8);
  const size_t o_scr = take256(off, scratch_layout(N, ld, nmax, 8, kBlock).total);
  if (off > kNoAllocBytes) {
    set_init_error("pqmc_green_noalloc: chain needs " + std::to_string(off) + " bytes, above the 16 MiB maximum");
    return PQMC_EINVAL;
  }

  // device address of the array, looked up once per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    set_init_error(std::string("pqmc_green_noalloc: no current device: ") + cudaGetErrorString(e));
    return PQMC_ECUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ready[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || p == nullptr) {
        set_init_error(std::string("pqmc_green_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return PQMC_ECUDA;
      }
      g_noalloc_addr[dev] = p;
      g_noalloc_ready[dev] = true;
    }
    base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  }

  // host model set-up (FP64), same as context creation
  Lattice lat{lt.kind, lt.Lx, lt.Ly, lt.t, lt.tp};
  std::vector<double> K, eps, w, V, em, ep, P[2];
  build_hopping(lat, K, eps);
  if (!sym_eig(N, K, w, V)) {
    set_init_error("pqmc_green_noalloc: eigensolver failed on K");
    return PQMC_EINVAL;
  }
  expm_from_eig(N, w, V, -spec->dtau, em);
  expm_from_eig(N, w, V, +spec->dtau, ep);
  for (int sp = 0; sp < 2; ++sp) {
    double gap = 0;
    if (!trial_orbitals(lat, K, eps, spec->trial.M_N, spec->trial.tiebreak, sp == 0 ? 1 : -1, sp == 0 ? nup : ndn,
                        P[sp], gap) || !(gap > 1e-8)) {
      set_init_error("pqmc_green_noalloc: trial orbitals failed or open shell");
      return PQMC_EINVAL;
    }
  }

  // contents of the uploaded prefix; counters start from zero every call
  std::vector<unsigned char> h(upload, 0);
  ChainDesc d;
  memset(&d, 0, sizeof d);
  d.N = N; d.ld = ld; d.nup = nup; d.ndn = ndn; d.nmax = nmax;
  d.nfld = N;
  d.Ltau = Ltau; d.nb = nb; d.n_stab = n_stab; d.kb = kBlock;
  d.U = spec->U;
  const double kap[2] = {hs_coupling(spec->dtau * spec->U), hs_coupling(spec->trial.g)};
  for (int k = 0; k < 2; ++k)
    for (int sp = 0; sp < 2; ++sp)
      for (int si = 0; si < 2; ++si) {
        const double sigma = sp == 0 ? 1.0 : -1.0, sv = si == 0 ? 1.0 : -1.0;
        d.delta[k][sp][si] = std::exp(-2.0 * sigma * kap[k] * sv) - 1.0;
        d.vexp[k][sp][si] = std::exp(sigma * kap[k] * sv);
      }
  d.fields = const_cast<int8_t*>(d_fields);
  d.G = base + o_G;
  d.expKm = base + o_em;
  d.expKp = base + o_ep;
  d.expKm64 = reinterpret_cast<const double*>(base + o_em64);
  d.K64 = reinterpret_cast<const double*>(base + o_k64);
  d.P = reinterpret_cast<const double*>(base + o_P);
  d.Rst = reinterpret_cast<double*>(base + o_rst);
  d.Lst = reinterpret_cast<double*>(base + o_lst);
  d.Rlog = reinterpret_cast<double*>(base + o_rlog);
  d.Llog = reinterpret_cast<double*>(base + o_llog);
  d.scratch = base + o_scr;
  d.st = reinterpret_cast<ChainState*>(base + o_state);
  memcpy(h.data() + o_desc, &d, sizeof d);
  ChainState st{};
  st.sign_running = 1.0;
  st.logw[0][1] = st.logw[1][1] = 1.0;
  memcpy(h.data() + o_state, &st, sizeof st);
  double* hem = reinterpret_cast<double*>(h.data() + o_em);
  double* hep = reinterpret_cast<double*>(h.data() + o_ep);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      hem[(size_t)i * ld + j] = em[(size_t)i * N + j];
      hep[(size_t)i * ld + j] = ep[(size_t)i * N + j];
    }
  memcpy(h.data() + o_em64, em.data(), (size_t)N * N * 8);
  memcpy(h.data() + o_k64, K.data(), (size_t)N * N * 8);
  double* hP = reinterpret_cast<double*>(h.data() + o_P);
  for (int sp = 0; sp < 2; ++sp) {
    const int ns = sp == 0 ? nup : ndn;
    for (int i = 0; i < N; ++i)
      for (int k = 0; k < ns; ++k) hP[(size_t)sp * N * nmax + (size_t)k * N + i] = P[sp][(size_t)i * ns + k];
  }

  cudaStream_t st_ = static_cast<cudaStream_t>(stream);
  e = cudaMemcpyAsync(base, h.data(), upload, cudaMemcpyHostToDevice, st_);
  if (e == cudaSuccess) {
    const size_t cap = smem_resident_cap(0, 256, 0);
    const size_t rb = resident_bytes(N, ld, nmax, 8, kBlock);
    e = launch_init_t<double, 256, 1>(reinterpret_cast<const ChainDesc*>(base + o_desc), 0, 1, 0,
                                      rb <= cap ? rb : 0, reinterpret_cast<int*>(base + o_err), st_, -1);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(d_G, (size_t)N * 8, base + o_G, (size_t)ld * 8, (size_t)N * 8, 2 * (size_t)N,
                          cudaMemcpyDeviceToDevice, st_);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_logw, base + o_state + offsetof(ChainState, logw), 4 * sizeof(double),
                        cudaMemcpyDeviceToDevice, st_);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, base + o_err, sizeof(int), cudaMemcpyDeviceToHost, st_);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
  if (e != cudaSuccess) {
    set_init_error(std::string("pqmc_green_noalloc: ") + cudaGetErrorString(e));
    return PQMC_ECUDA;
  }
  if (herr) {
    set_init_error((herr & kErrNaN) ? "pqmc_green_noalloc: NaN or Inf in G" : "pqmc_green_noalloc: singular matrix");
    return (herr & kErrNaN) ? PQMC_ENAN : PQMC_ESTAB;
  }
  return PQMC_OK;
}

extern "C" pqmc_status pqmc_test_tc_gemm(int M, int N, int K, const float* d_A, int trans_a, const float* d_B,
                                         float* d_C, void* stream) {
  using namespace pqmc;
  if (M < 1 || N < 1 || K < 1 || M > 4096 || N > 4096 || K > 4096 || !d_A || !d_B || !d_C) {
    set_init_error("pqmc_test_tc_gemm: bad sizes or NULL pointer");
    return PQMC_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* d_err = nullptr;
  cudaError_t e = cudaMallocAsync(&d_err, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  const int smem = (int)(kTcBytes + 128);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_gemm_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) {
    tc_gemm_test_kernel<<<1, 512, smem, st>>>(M, N, K, d_A, trans_a, d_B, d_C, d_err);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (d_err) cudaFreeAsync(d_err, st);
  cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_init_error(std::string("pqmc_test_tc_gemm: ") + cudaGetErrorString(e));
    return PQMC_ECUDA;
  }
  if (herr & kErrTimeout) {
    set_init_error("pqmc_test_tc_gemm: tensor-core completion wait gave up");
    return PQMC_ETIMEOUT;
  }
  return PQMC_OK;
}

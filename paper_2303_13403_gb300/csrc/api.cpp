// C-ABI of libpqmc.so (declarations and documentation in include/pqmc.h).
//
// Host side: validates the chain specs, builds the model in FP64 (model.cpp),
// draws the initial fields with Philox, lays out one device arena per context
// and drives the sweep kernels (sweep_kernels.cuh, dispatched by sweep.cu) on
// the context's stream.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pqmc.h"
#include "chain.h"
#include "model.h"
#include "philox.cuh"
#include "spread.h"

namespace pqmc {
size_t smem_resident_cap(int prec, int tpb, int boost);
int ctas_per_sm(int prec, int tpb, int boost);
cudaError_t launch_init(int prec, int tpb, int boost, const ChainDesc* d_chains, int chain0, int n, uint64_t seed,
                        size_t res, int* d_err, cudaStream_t stream, int b_at);
cudaError_t prepare_sweep(int prec, int tpb, int boost, size_t res);
cudaError_t launch_advance(uint32_t* sweep_ctr, int n, cudaStream_t stream);
cudaError_t launch_sweep(int prec, int tpb, int boost, const ChainDesc* d_chains, int n, uint64_t seed,
                         uint32_t* sweep_ctr, int n_sweeps, int measure, size_t res, int* d_err, cudaStream_t stream);
}  // namespace pqmc

using namespace pqmc;

namespace {

thread_local std::string g_init_error;

// NVTX range for the duration of a scope (shows the host-side entry points on
// a profiler timeline; no effect without a tool attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct HostChain {
  pqmc_chain_spec spec;
  int N, ld, nup, ndn, nmax, Ltau, nb, nfld;
  size_t off_fields, off_G, off_Rst, off_Lst, off_Rlog, off_Llog, off_meas, off_dG,
      off_acc, off_state, off_P, off_scratch, off_expKm, off_expKp, off_expKm64, off_K64, off_eps, off_bonds,
      off_sbonds, off_spread;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct pqmc_ctx {
  pqmc_opts opts;
  int prec = 0;
  size_t tsize = 8;
  std::vector<HostChain> chains;
  std::vector<ChainDesc> desc;
  size_t upload_bytes = 0;                 // bytes copied from host memory into the arena at creation
  unsigned char* d_arena = nullptr;
  size_t arena_bytes = 0;
  ChainDesc* d_desc = nullptr;            // descriptors by chain index (initialisation launches)
  ChainDesc* d_desc_run = nullptr;        // the same in sweep-launch order: costliest chains first
  int* d_err = nullptr;
  size_t off_last = 0;                     // n_chains x kRecord latest records
  size_t res_bytes = 0;                    // shared memory offered for resident chains
  uint32_t* d_sweep = nullptr;             // sweep index read by the sweep kernel
  struct GraphEntry { int n_sweeps, measure; cudaGraphExec_t exec; size_t kernels; };
  std::vector<GraphEntry> graphs;          // captured (sweep, advance) pairs; spread: one sweep of
                                           // each direction (n_sweeps = parity)
  bool spread = false;                     // chains swept by grid-wide kernel sequences
  SpreadPlan plan;
  int tpb = 256;                           // threads per chain CTA
  int scratch_kd = kBlock;                 // delayed block the per-chain scratch is sized for
  int boost = 0;                           // 1: reduced-path kernels built for twice the CTAs per SM
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t sweep_index = 0;
  long launches = 0;
  int sticky = PQMC_OK;
  std::string err;
};

namespace {

pqmc_status fail(pqmc_ctx* ctx, pqmc_status st, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_init_error = msg;
  return st;
}

pqmc_status cuda_fail(pqmc_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, PQMC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int n_sites(const pqmc_lattice& l) { return l.kind == PQMC_SQUARE ? l.Lx * l.Ly : 2 * l.Lx * l.Ly; }
bool is_tv(const pqmc_chain_spec& s) { return s.lattice.kind == PQMC_HONEYCOMB_TV; }

// model tables shared by chains with the same lattice and dtau
struct ModelTables {
  std::vector<double> K, eps, w, V, expKm, expKp;
  std::vector<int> bond_ends, site_bonds;   // t-V only
};

// Bonds of the honeycomb lattice for the t-V model: bond 3 c + k of cell
// c = x + Lx y joins A(x, y) to B(x, y), B(x-1, y), B(x, y-1) (k = 0, 1, 2);
// site_bonds lists the three bonds of every site.
void tv_bonds(int Lx, int Ly, std::vector<int>& ends, std::vector<int>& site_bonds) {
  const int nc = Lx * Ly;
  auto site = [&](int x, int y, int sub) { return 2 * (((x % Lx) + Lx) % Lx + Lx * (((y % Ly) + Ly) % Ly)) + sub; };
  ends.assign(6 * nc, 0);
  site_bonds.assign(6 * nc, 0);
  std::vector<int> fill(2 * nc, 0);
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      const int c = x + Lx * y, a = site(x, y, 0);
      const int bs[3] = {site(x, y, 1), site(x - 1, y, 1), site(x, y - 1, 1)};
      for (int k = 0; k < 3; ++k) {
        const int b = 3 * c + k;
        ends[2 * b] = a;
        ends[2 * b + 1] = bs[k];
        site_bonds[3 * a + fill[a]++] = b;
        site_bonds[3 * bs[k] + fill[bs[k]]++] = b;
      }
    }
}

std::string lattice_key(const pqmc_chain_spec& s) {
  char buf[256];
  snprintf(buf, sizeof buf, "%d/%d/%d/%.17g/%.17g/%.17g", s.lattice.kind, s.lattice.Lx, s.lattice.Ly, s.lattice.t,
           s.lattice.tp, s.dtau);
  return buf;
}

}  // namespace

namespace pqmc {
void set_init_error(const std::string& msg) { g_init_error = msg; }

pqmc_status check_spec(const pqmc_chain_spec& s, int n_stab, std::string& why) {
  const auto& l = s.lattice;
  if (l.kind != PQMC_HONEYCOMB && l.kind != PQMC_SQUARE && l.kind != PQMC_HONEYCOMB_TV) {
    why = "unknown lattice kind"; return PQMC_EINVAL;
  }
  if (l.Lx < 1 || l.Ly < 1 || l.Lx > 64 || l.Ly > 64) { why = "lattice extent out of range"; return PQMC_EINVAL; }
  const int N = n_sites(l);
  if (N > kMaxN) { why = "more than 1024 sites"; return PQMC_EINVAL; }
  const int nup = s.trial.N_up < 0 ? N / 2 : s.trial.N_up;
  if (l.kind == PQMC_HONEYCOMB_TV) {
    if (s.trial.N_dn > 0) { why = "t-V chains have one species: N_dn must be 0 or < 0"; return PQMC_EINVAL; }
    if (nup < 1 || nup > N) { why = "N_up must be in 1..N"; return PQMC_EINVAL; }
  }
  const int ndn = l.kind == PQMC_HONEYCOMB_TV ? nup : (s.trial.N_dn < 0 ? N / 2 : s.trial.N_dn);
  if (nup < 1 || ndn < 1 || nup > N || ndn > N) { why = "N_sigma must be in 1..N"; return PQMC_EINVAL; }
  if (nup > kMaxSigma || ndn > kMaxSigma) { why = "N_sigma above 512"; return PQMC_EINVAL; }
  if (!(s.dtau > 0) || !(s.two_theta >= 0) || !std::isfinite(s.U) || s.U < 0) {
    why = "need dtau > 0, two_theta >= 0, U >= 0"; return PQMC_EINVAL;
  }
  if (!(s.trial.g >= 0) || !std::isfinite(s.trial.M_N)) { why = "need g >= 0 and finite M_N"; return PQMC_EINVAL; }
  const double lt = s.two_theta / s.dtau;
  const int Ltau = (int)std::lround(lt);
  if (std::fabs(lt - Ltau) > 1e-9 * std::max(1.0, lt)) { why = "two_theta / dtau is not an integer"; return PQMC_EINVAL; }
  if (Ltau % 2) { why = "Ltau must be even"; return PQMC_EINVAL; }
  if (n_stab < 1 || (Ltau / 2) % n_stab) { why = "Ltau/2 must be a multiple of n_stab"; return PQMC_EINVAL; }
  return PQMC_OK;
}
}  // namespace pqmc

namespace {

// The parts of a new context's arena that do not start at zero, as segments
// at arena offsets: the arena is cleared on the device and only these are
// copied from host memory.
struct Staged {
  struct Segment {
    size_t off;
    std::vector<unsigned char> bytes;
  };
  std::vector<Segment> seg;
  // a zeroed host segment of n bytes for arena offset off
  unsigned char* at(size_t off, size_t n) {
    seg.push_back({off, std::vector<unsigned char>(n, 0)});
    return seg.back().bytes.data();
  }
  size_t bytes() const {
    size_t b = 0;
    for (const Segment& g : seg) b += g.bytes.size();
    return b;
  }
};

template <typename T>
void put(Staged& a, size_t off, const std::vector<double>& src, int rows, int cols, int ld) {
  T* p = reinterpret_cast<T*>(a.at(off, (size_t)rows * ld * sizeof(T)));
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) p[(size_t)i * ld + j] = (T)src[(size_t)i * cols + j];
}

void put_raw(Staged& a, size_t off, const void* src, size_t n) { memcpy(a.at(off, n), src, n); }

pqmc_status sync_check(pqmc_ctx* ctx) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  int herr = 0;
  e = cudaMemcpy(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "error word copy");
  if (herr) {
    ctx->sticky = (herr & kErrNaN) ? PQMC_ENAN : (herr & kErrStab) ? PQMC_ESTAB : PQMC_ETIMEOUT;
    ctx->err = (herr & kErrNaN) ? "NaN or Inf in a ratio or in G"
               : (herr & kErrStab) ? "singular matrix in the stabilisation"
                                   : "the bounded wait for the tensor cores' completion gave up";
    return (pqmc_status)ctx->sticky;
  }
  return PQMC_OK;
}

// The sweep launch runs one CTA per chain; a batch of uneven chains starts
// its costliest chains first (longest-processing-time order, cost
// N^3 (Ltau + 2), ties in chain order), so that the long chains are not left
// for the tail of the launch.  Each CTA reads its chain's own descriptor, so
// the order changes no result.
cudaError_t upload_run_order(pqmc_ctx* ctx) {
  const int n = (int)ctx->chains.size();
  std::vector<int> order(n);
  for (int c = 0; c < n; ++c) order[c] = c;
  auto cost = [&](int c) {
    const HostChain& h = ctx->chains[c];
    return (double)h.N * h.N * h.N * (h.Ltau + 2);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::vector<ChainDesc> run(n);
  for (int i = 0; i < n; ++i) run[i] = ctx->desc[order[i]];
  cudaError_t e = cudaMemcpyAsync(ctx->d_desc_run, run.data(), sizeof(ChainDesc) * n, cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);   // run is a local buffer
  return e;
}

pqmc_status autotune_cached(int n, const pqmc_chain_spec* specs, const pqmc_opts& o, pqmc_tune* out);

bool valid_delay(int k) { return k == 8 || k == 16 || k == 32 || k == 64; }

// scratch_kd: size the per-chain scratch for delayed blocks up to this many
// sites (the autotuner's proxy context runs every block size on one arena)
pqmc_status build_ctx(int n, const pqmc_chain_spec* specs, const pqmc_opts* opts, pqmc_ctx** out,
                      int scratch_kd = 0) {
  NvtxRange range("pqmc_init");
  if (!out) return fail(nullptr, PQMC_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !specs || !opts) return fail(nullptr, PQMC_EINVAL, "need n >= 1, specs and opts");
  pqmc_opts o = *opts;
  if (o.prec < PQMC_FP64 || o.prec > PQMC_BF16X3) return fail(nullptr, PQMC_EINVAL, "unknown precision");
  if (o.delay_k != 0 && !valid_delay(o.delay_k)) return fail(nullptr, PQMC_EINVAL, "delay_k must be 0, 8, 16, 32 or 64");
  if (o.max_meas <= 0) o.max_meas = 4096;
  if (o.accept_log < 0) return fail(nullptr, PQMC_EINVAL, "accept_log < 0");
  if (o.cta_threads != 0 && o.cta_threads != 64 && o.cta_threads != 128 && o.cta_threads != 256 &&
      o.cta_threads != 512)
    return fail(nullptr, PQMC_EINVAL, "cta_threads must be 0, 64, 128, 256 or 512");
  if (o.cta_threads == 512 && (o.prec == PQMC_FP64 || o.dense_chains))
    return fail(nullptr, PQMC_EINVAL, "cta_threads 512 is built for the reduced paths only");
  if (o.dense_chains && o.prec != PQMC_FP64 && o.cta_threads == 256)
    return fail(nullptr, PQMC_EINVAL, "dense_chains needs cta_threads 64 or 128");
  if (o.spread) {
    // chains swept by grid-wide kernels: one shape, Hubbard chains, blocks of
    // kBlock sites, no FP64 diagnostic
    if (n * 2 > 64) return fail(nullptr, PQMC_EINVAL, "spread: at most 32 chains");
    if (o.dense_chains || o.dg_fp64) return fail(nullptr, PQMC_EINVAL, "spread: no dense_chains or dg_fp64");
    for (int c = 0; c < n; ++c) {
      const pqmc_chain_spec& a = specs[c];
      const pqmc_chain_spec& z = specs[0];
      if (is_tv(a)) return fail(nullptr, PQMC_EINVAL, "spread: Hubbard chains only");
      if (n_sites(a.lattice) != n_sites(z.lattice) || a.trial.N_up != z.trial.N_up || a.trial.N_dn != z.trial.N_dn ||
          std::lround(a.two_theta / a.dtau) != std::lround(z.two_theta / z.dtau))
        return fail(nullptr, PQMC_EINVAL, "spread: chains must share N, N_sigma and Ltau");
    }
    o.delay_k = kBlock;
  }
  for (int c = 0; c < n; ++c) {
    std::string why;
    if (check_spec(specs[c], o.n_stab, why) != PQMC_OK) return fail(nullptr, PQMC_EINVAL, "chain " + std::to_string(c) + ": " + why);
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
    return fail(nullptr, PQMC_ECUDA, "no CUDA device");
  if (o.delay_k == 0) {
    // delay_k = 0: the autotuner picks the delayed block (and the CTA shape
    // when that is not fixed)
    pqmc_tune t;
    const pqmc_status ts = autotune_cached(n, specs, o, &t);
    if (ts != PQMC_OK) return ts;
    o.delay_k = t.delay_k;
    if (o.cta_threads == 0) o.cta_threads = t.cta_threads;
  }
  if (scratch_kd < o.delay_k) scratch_kd = o.delay_k;

  auto* ctx = new pqmc_ctx();
  ctx->opts = o;
  ctx->scratch_kd = scratch_kd;
  ctx->prec = o.prec;
  ctx->tsize = o.prec == PQMC_FP64 ? 8 : 4;

  // ---- host model set-up and arena layout
  std::map<std::string, ModelTables> models;
  std::map<std::string, size_t> model_off;   // offset of expKm (T) for the lattice key
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes, 256); return at; };
  ctx->chains.resize(n);
  struct TrialOut { std::vector<double> P[2]; };
  std::vector<TrialOut> trials(n);
  // chains with the same lattice, trial parameters and particle numbers share
  // their trial orbitals: trial_src[c] is the chain whose orbitals c uses
  std::vector<int> trial_src(n);
  std::map<std::string, int> trial_first;
  for (int c = 0; c < n; ++c) {
    const pqmc_chain_spec& s = specs[c];
    HostChain& h = ctx->chains[c];
    h.spec = s;
    h.N = n_sites(s.lattice);
    h.ld = (int)align_up(h.N, 4);
    h.nup = s.trial.N_up < 0 ? h.N / 2 : s.trial.N_up;
    h.ndn = is_tv(s) ? 0 : (s.trial.N_dn < 0 ? h.N / 2 : s.trial.N_dn);
    h.nmax = std::max(h.nup, h.ndn);
    h.nfld = is_tv(s) ? 3 * h.N / 2 : h.N;
    h.Ltau = (int)std::lround(s.two_theta / s.dtau);
    h.nb = h.Ltau / o.n_stab;
    const std::string key = lattice_key(s);
    if (!models.count(key)) {
      ModelTables mt;
      Lattice lat{is_tv(s) ? (int)PQMC_HONEYCOMB : s.lattice.kind, s.lattice.Lx, s.lattice.Ly, s.lattice.t,
                  s.lattice.tp};
      build_hopping(lat, mt.K, mt.eps);
      if (is_tv(s)) tv_bonds(s.lattice.Lx, s.lattice.Ly, mt.bond_ends, mt.site_bonds);
      if (!sym_eig(h.N, mt.K, mt.w, mt.V)) { delete ctx; return fail(nullptr, PQMC_EINVAL, "eigensolver failed on K"); }
      expm_from_eig(h.N, mt.w, mt.V, -s.dtau, mt.expKm);
      expm_from_eig(h.N, mt.w, mt.V, +s.dtau, mt.expKp);
      models[key] = std::move(mt);
      const size_t Tm = (size_t)h.N * h.ld * ctx->tsize;
      const size_t o1 = take(Tm);
      take(Tm);
      take((size_t)h.N * h.N * 8);
      take((size_t)h.N * h.N * 8);
      take((size_t)h.N * 8);
      take((size_t)h.N * 3 * 4);             // bond ends (3N/2 x 2 int)
      take((size_t)h.N * 3 * 4);             // site bonds (N x 3 int)
      model_off[key] = o1;
    }
    const ModelTables& mt = models[key];
    Lattice lat{is_tv(s) ? (int)PQMC_HONEYCOMB : s.lattice.kind, s.lattice.Lx, s.lattice.Ly, s.lattice.t,
                s.lattice.tp};
    char tkey[160];
    snprintf(tkey, sizeof tkey, "|%.17g|%.17g|%d|%d", s.trial.M_N, s.trial.tiebreak, h.nup, h.ndn);
    const auto tf = trial_first.find(key + tkey);
    trial_src[c] = tf == trial_first.end() ? c : tf->second;
    if (tf == trial_first.end()) trial_first[key + tkey] = c;
    for (int sp = 0; sp < (is_tv(s) ? 1 : 2) && trial_src[c] == c; ++sp) {
      double gap = 0;
      if (!trial_orbitals(lat, mt.K, mt.eps, s.trial.M_N, s.trial.tiebreak, sp == 0 ? 1 : -1,
                          sp == 0 ? h.nup : h.ndn, trials[c].P[sp], gap)) {
        delete ctx; return fail(nullptr, PQMC_EINVAL, "eigensolver failed on the trial Hamiltonian");
      }
      if (!(gap > 1e-8)) {
        delete ctx;
        return fail(nullptr, PQMC_EINVAL, "chain " + std::to_string(c) + ": open-shell trial (gap " + std::to_string(gap) + ")");
      }
    }
    h.off_expKm = model_off[key];
    h.off_expKp = h.off_expKm + align_up((size_t)h.N * h.ld * ctx->tsize, 256);
    h.off_expKm64 = h.off_expKp + align_up((size_t)h.N * h.ld * ctx->tsize, 256);
    h.off_K64 = h.off_expKm64 + align_up((size_t)h.N * h.N * 8, 256);
    h.off_eps = h.off_K64 + align_up((size_t)h.N * h.N * 8, 256);
    h.off_bonds = h.off_eps + align_up((size_t)h.N * 8, 256);
    h.off_sbonds = h.off_bonds + align_up((size_t)h.N * 3 * 4, 256);
    const size_t Gbytes = 2ull * h.N * h.ld * ctx->tsize;
    const size_t blk = (size_t)h.N * h.nmax * 8;
    h.off_fields = take((size_t)(h.Ltau + 2) * h.nfld);
    h.off_G = take(Gbytes);
    h.off_P = take(2 * blk);
    h.off_Rst = take((size_t)(h.nb + 1) * 2 * blk);
    h.off_Lst = take((size_t)(h.nb + 1) * 2 * blk);
    h.off_Rlog = take((size_t)(h.nb + 1) * 4 * 8);
    h.off_Llog = take((size_t)(h.nb + 1) * 4 * 8);
    h.off_scratch = take(scratch_layout(h.N, h.ld, h.nmax, (int)ctx->tsize, scratch_kd).total);
    h.off_meas = take((size_t)o.max_meas * kRecord * 8);
    h.off_dG = take((size_t)kDGHistory * 8);
    h.off_acc = take((size_t)std::max(o.accept_log, 1));
    h.off_state = take(sizeof(ChainState));
    h.off_spread = o.spread ? take(spread_layout(h.N, h.ld, h.nmax, (int)ctx->tsize).total) : 0;
  }
  ctx->off_last = take((size_t)n * kRecord * 8);
  // default CTA size (measured on GB300): the FP64 path packs 4 chains of 64
  // threads per SM; the reduced paths 2 chains of 256 threads, whose G and
  // scratch then fit in shared memory at 72 sites, and one chain of 512
  // threads per SM once a chain has 128 sites or more (its G lives in global
  // memory and more warps hide the latency: 1.4-1.6x at 162-648 sites)
  int nmax_sites = 0;
  for (const HostChain& h : ctx->chains) nmax_sites = std::max(nmax_sites, h.N);
  const int reduced_tpb = (nmax_sites >= 128 && !o.dense_chains) ? 512 : 256;
  ctx->tpb = o.cta_threads != 0 ? o.cta_threads : (ctx->prec == PQMC_FP64 ? (o.spread ? 256 : 64) : reduced_tpb);
  {
    ctx->boost = (ctx->prec != PQMC_FP64 && o.dense_chains) ? 1 : 0;
    const size_t cap = smem_resident_cap(ctx->prec, ctx->tpb, ctx->boost);
    for (const HostChain& h : ctx->chains) {
      const size_t r = resident_bytes(h.N, h.ld, h.nmax, (int)ctx->tsize, o.delay_k);
      if (r <= cap && r > ctx->res_bytes) ctx->res_bytes = r;
    }
  }
  ctx->arena_bytes = off;

  // ---- initial arena contents
  Staged A;
  std::map<std::string, bool> written;
  double* last_all = reinterpret_cast<double*>(A.at(ctx->off_last, (size_t)n * kRecord * 8));
  for (int c = 0; c < n; ++c) {
    HostChain& h = ctx->chains[c];
    const pqmc_chain_spec& s = h.spec;
    const std::string key = lattice_key(s);
    if (!written[key]) {
      const ModelTables& mt = models[key];
      if (ctx->prec == PQMC_FP64) {
        put<double>(A, h.off_expKm, mt.expKm, h.N, h.N, h.ld);
        put<double>(A, h.off_expKp, mt.expKp, h.N, h.N, h.ld);
      } else {
        put<float>(A, h.off_expKm, mt.expKm, h.N, h.N, h.ld);
        put<float>(A, h.off_expKp, mt.expKp, h.N, h.N, h.ld);
      }
      put<double>(A, h.off_expKm64, mt.expKm, h.N, h.N, h.N);
      put<double>(A, h.off_K64, mt.K, h.N, h.N, h.N);
      put_raw(A, h.off_eps, mt.eps.data(), (size_t)h.N * 8);
      if (is_tv(s)) {
        put_raw(A, h.off_bonds, mt.bond_ends.data(), mt.bond_ends.size() * 4);
        put_raw(A, h.off_sbonds, mt.site_bonds.data(), mt.site_bonds.size() * 4);
      }
      written[key] = true;
    }
    // P_sigma column-major (ld N) in blocks of N x nmax
    double* P = reinterpret_cast<double*>(A.at(h.off_P, 2 * (size_t)h.N * h.nmax * 8));
    const TrialOut& tr = trials[trial_src[c]];
    for (int sp = 0; sp < 2; ++sp) {
      const int ns = sp == 0 ? h.nup : h.ndn;
      for (int i = 0; i < h.N; ++i)
        for (int k = 0; k < ns; ++k) P[(size_t)sp * h.N * h.nmax + (size_t)k * h.N + i] = tr.P[sp][(size_t)i * ns + k];
    }
    int8_t* F = reinterpret_cast<int8_t*>(A.at(h.off_fields, (size_t)(h.Ltau + 2) * h.nfld));
    const uint32_t chain_index = (uint32_t)(o.chain_offset + c);
    for (int t = 0; t < h.Ltau + 2; ++t)
      for (int i = 0; i < h.nfld; ++i) F[(size_t)t * h.nfld + i] = (int8_t)initial_field(o.seed, chain_index, t, i);
    double* last = last_all + (size_t)c * kRecord;
    for (int k = 0; k < kRecord; ++k) last[k] = NAN;
    ChainState st{};
    st.sign_running = 1.0;
    st.logw[0][1] = st.logw[1][1] = 1.0;
    put_raw(A, h.off_state, &st, sizeof st);
  }

  // ---- device
  cudaError_t e;
  if (o.stream) {
    ctx->stream = (cudaStream_t)o.stream;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete ctx; return cuda_fail(nullptr, e, "stream create"); }
    ctx->own_stream = true;
  }
  e = cudaMalloc(&ctx->d_arena, ctx->arena_bytes);
  if (e != cudaSuccess) { pqmc_free(ctx); return fail(nullptr, PQMC_ENOMEM, std::string("device arena: ") + cudaGetErrorString(e)); }
  e = cudaMalloc(&ctx->d_desc, sizeof(ChainDesc) * n);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_desc_run, sizeof(ChainDesc) * n);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, 2 * sizeof(int));
  if (e == cudaSuccess) ctx->d_sweep = reinterpret_cast<uint32_t*>(ctx->d_err + 1);
  if (e != cudaSuccess) { pqmc_free(ctx); return fail(nullptr, PQMC_ENOMEM, "device descriptors"); }
  ctx->desc.resize(n);
  for (int c = 0; c < n; ++c) {
    HostChain& h = ctx->chains[c];
    const pqmc_chain_spec& s = h.spec;
    ChainDesc& d = ctx->desc[c];
    memset(&d, 0, sizeof d);
    d.N = h.N; d.ld = h.ld; d.nup = h.nup; d.ndn = h.ndn; d.nmax = h.nmax;
    d.Ltau = h.Ltau; d.nb = h.nb; d.n_stab = o.n_stab; d.kb = o.delay_k;
    d.chain_index = (uint32_t)(o.chain_offset + c);
    d.tc = ctx->prec == PQMC_BF16X3 ? 1 : 0;
    d.tv = is_tv(s) ? 1 : 0;
    d.nfld = h.nfld;
    d.dg64 = (ctx->prec != PQMC_FP64 && o.dg_fp64 >= 1 && o.dg_fp64 <= 3) ? o.dg_fp64 : 0;
    d.U = s.U;
    const double kap[2] = {hs_coupling(s.dtau * s.U), hs_coupling(s.trial.g)};
    for (int k = 0; k < 2; ++k)
      for (int m = -3; m <= 3; ++m) d.vtv[k][m + 3] = std::exp(kap[k] * m);
    for (int k = 0; k < 2; ++k)
      for (int sp = 0; sp < 2; ++sp)
        for (int si = 0; si < 2; ++si) {
          const double sigma = sp == 0 ? 1.0 : -1.0, sv = si == 0 ? 1.0 : -1.0;
          d.delta[k][sp][si] = std::exp(-2.0 * sigma * kap[k] * sv) - 1.0;
          d.vexp[k][sp][si] = std::exp(sigma * kap[k] * sv);
        }
    unsigned char* b = ctx->d_arena;
    d.fields = reinterpret_cast<int8_t*>(b + h.off_fields);
    d.G = b + h.off_G;
    d.expKm = b + h.off_expKm;
    d.expKp = b + h.off_expKp;
    d.expKm64 = reinterpret_cast<const double*>(b + h.off_expKm64);
    d.K64 = reinterpret_cast<const double*>(b + h.off_K64);
    d.eps = reinterpret_cast<const double*>(b + h.off_eps);
    d.bond_ends = reinterpret_cast<const int*>(b + h.off_bonds);
    d.site_bonds = reinterpret_cast<const int*>(b + h.off_sbonds);
    d.P = reinterpret_cast<const double*>(b + h.off_P);
    d.Rst = reinterpret_cast<double*>(b + h.off_Rst);
    d.Lst = reinterpret_cast<double*>(b + h.off_Lst);
    d.Rlog = reinterpret_cast<double*>(b + h.off_Rlog);
    d.Llog = reinterpret_cast<double*>(b + h.off_Llog);
    d.scratch = b + h.off_scratch;
    d.meas = reinterpret_cast<double*>(b + h.off_meas);
    d.last = reinterpret_cast<double*>(b + ctx->off_last) + (size_t)c * kRecord;
    d.max_meas = o.max_meas;
    d.dG = reinterpret_cast<double*>(b + h.off_dG);
    d.acc_log = reinterpret_cast<uint8_t*>(b + h.off_acc);
    d.acc_cap = o.accept_log;
    d.st = reinterpret_cast<ChainState*>(b + h.off_state);
    d.spread = o.spread ? b + h.off_spread : nullptr;
  }
  if (o.spread) {
    SpreadPlan& P = ctx->plan;
    const HostChain& h0 = ctx->chains[0];
    P.prec = ctx->prec;
    P.n = n;
    P.N = h0.N; P.ld = h0.ld; P.nup = h0.nup; P.ndn = h0.ndn; P.nmax = h0.nmax;
    P.Ltau = h0.Ltau; P.n_stab = o.n_stab; P.nb = h0.nb;
    P.d_desc = ctx->d_desc;
    P.seed = o.seed;
    P.d_sweep = ctx->d_sweep;
    P.d_err = ctx->d_err;
    for (int c = 0; c < n; ++c) {
      const ChainDesc& d = ctx->desc[c];
      P.ch.push_back({d.spread, d.G, d.expKm, d.expKp, d.Rst, d.Lst});
    }
    ctx->spread = true;
  }
  // clear the arena on the device, then copy in the parts that the host set
  // (model tables, trial orbitals, initial fields, chain states, records);
  // pqmc_init synchronises before it returns, so A outlives the copies
  e = cudaMemsetAsync(ctx->d_arena, 0, ctx->arena_bytes, ctx->stream);
  for (size_t g = 0; g < A.seg.size() && e == cudaSuccess; ++g)
    e = cudaMemcpyAsync(ctx->d_arena + A.seg[g].off, A.seg[g].bytes.data(), A.seg[g].bytes.size(),
                        cudaMemcpyHostToDevice, ctx->stream);
  ctx->upload_bytes = A.bytes();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->d_desc, ctx->desc.data(), sizeof(ChainDesc) * n, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = upload_run_order(ctx);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err, 0, 2 * sizeof(int), ctx->stream);
  if (e == cudaSuccess) e = prepare_sweep(ctx->prec, ctx->tpb, ctx->boost, ctx->res_bytes);
  if (e == cudaSuccess && ctx->spread) e = spread_prepare();
  if (e != cudaSuccess) { pqmc_free(ctx); return cuda_fail(nullptr, e, "upload"); }
  if (ctx->spread) {
    e = spread_init(ctx->plan, ctx->stream);
  } else {
    e = launch_init(ctx->prec, ctx->tpb, ctx->boost, ctx->d_desc, 0, n, o.seed, ctx->res_bytes, ctx->d_err, ctx->stream, -1);
    ctx->launches++;
  }
  if (e != cudaSuccess) { pqmc_free(ctx); return cuda_fail(nullptr, e, "init launch"); }
  pqmc_status st = sync_check(ctx);
  if (st != PQMC_OK) { g_init_error = ctx->err; pqmc_free(ctx); return st; }
  *out = ctx;
  return PQMC_OK;
}

bool chain_ok(pqmc_ctx* ctx, int chain) { return ctx && chain >= 0 && chain < (int)ctx->chains.size(); }

// ---------------------------------------------------------------- autotuner
//
// Picks the delayed-update block and the CTA shape of a batch by timing
// every candidate on a proxy of the batch (same chains, shorter projection),
// all candidates on one proxy context whose scratch is sized for the largest
// block: the context is re-targeted (block size in every chain descriptor,
// CTA shape, shared-memory budget) between candidates.

// Point a context at another delayed block and CTA shape.
pqmc_status retarget(pqmc_ctx* ctx, int kd, int tpb) {
  ctx->opts.delay_k = kd;
  ctx->opts.cta_threads = tpb;
  ctx->tpb = tpb;
  ctx->res_bytes = 0;
  const size_t cap = smem_resident_cap(ctx->prec, ctx->tpb, ctx->boost);
  for (const HostChain& h : ctx->chains) {
    const size_t r = resident_bytes(h.N, h.ld, h.nmax, (int)ctx->tsize, kd);
    if (r <= cap && r > ctx->res_bytes) ctx->res_bytes = r;
  }
  for (auto& d : ctx->desc) d.kb = kd;
  cudaError_t e = cudaMemcpyAsync(ctx->d_desc, ctx->desc.data(), sizeof(ChainDesc) * ctx->desc.size(),
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = upload_run_order(ctx);
  if (e == cudaSuccess) e = prepare_sweep(ctx->prec, ctx->tpb, ctx->boost, ctx->res_bytes);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
  return e == cudaSuccess ? PQMC_OK : cuda_fail(ctx, e, "retarget");
}

// ms per sweep of the context as it is set up: one warm-up sweep, then two
// timed with CUDA events on its stream; NaN when a launch fails
double time_sweeps(pqmc_ctx* ctx) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NAN;
  const int n = (int)ctx->chains.size();
  cudaError_t e = launch_sweep(ctx->prec, ctx->tpb, ctx->boost, ctx->d_desc_run, n, ctx->opts.seed, ctx->d_sweep, 1, 0,
                               ctx->res_bytes, ctx->d_err, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = launch_sweep(ctx->prec, ctx->tpb, ctx->boost, ctx->d_desc_run, n, ctx->opts.seed, ctx->d_sweep, 1, 0,
                     ctx->res_bytes, ctx->d_err, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = NAN;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  else cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->launches += 6;
  return e == cudaSuccess ? ms / 2.0 : NAN;
}

int proxy_ltau(int Ltau, int n_stab) {
  int lp = 2 * n_stab;
  while (lp < 8) lp += 2 * n_stab;
  return std::min(lp, Ltau);
}

// cache key: precision, n_stab, the fixed options and the multiset of shapes
std::string tune_key(int n, const pqmc_chain_spec* specs, const pqmc_opts& o) {
  std::map<std::string, int> shapes;
  for (int c = 0; c < n; ++c) {
    const pqmc_chain_spec& s = specs[c];
    const int N = n_sites(s.lattice);
    const int nup = s.trial.N_up < 0 ? N / 2 : s.trial.N_up;
    const int ndn = is_tv(s) ? 0 : (s.trial.N_dn < 0 ? N / 2 : s.trial.N_dn);
    const int Ltau = (int)std::lround(s.two_theta / s.dtau);
    char buf[96];
    snprintf(buf, sizeof buf, "%d.%d.%d.%d.%s", N, nup, ndn, Ltau, is_tv(s) ? "tv" : "h");
    shapes[buf]++;
  }
  std::ostringstream k;
  k << "prec" << o.prec << "/nstab" << o.n_stab << "/k" << o.delay_k << "/cta" << o.cta_threads << "/dense"
    << o.dense_chains;
  for (auto& kv : shapes) k << "/" << kv.first << "x" << kv.second;
  return k.str();
}

struct TuneEntry { int delay_k, cta_threads; double ms; };
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune;
bool g_tune_file_read = false;

// the JSON cache: an object of {"key": {"delay_k": k, "cta_threads": t, "ms_per_sweep": m}}
// entries (whitespace anywhere; keys hold no quotes)
void tune_file_read(const char* path) {
  std::ifstream f(path);
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string txt = ss.str();
  size_t pos = 0;
  auto field = [](const std::string& obj, const char* name, double& v) {
    const size_t a = obj.find(std::string("\"") + name + "\"");
    if (a == std::string::npos) return false;
    const size_t c = obj.find(':', a);
    if (c == std::string::npos) return false;
    v = atof(obj.c_str() + c + 1);
    return true;
  };
  while (true) {
    const size_t q0 = txt.find('"', pos);
    if (q0 == std::string::npos) break;
    const size_t q1 = txt.find('"', q0 + 1);
    if (q1 == std::string::npos) break;
    size_t b = q1 + 1;
    while (b < txt.size() && isspace((unsigned char)txt[b])) ++b;
    if (b >= txt.size() || txt[b] != ':') { pos = q1 + 1; continue; }
    ++b;
    while (b < txt.size() && isspace((unsigned char)txt[b])) ++b;
    if (b >= txt.size() || txt[b] != '{') { pos = q1 + 1; continue; }
    const size_t e = txt.find('}', b);
    if (e == std::string::npos) break;
    const std::string key = txt.substr(q0 + 1, q1 - q0 - 1), obj = txt.substr(b, e - b + 1);
    double k = 0, t = 0, m = NAN;
    if (field(obj, "delay_k", k) && field(obj, "cta_threads", t)) {
      field(obj, "ms_per_sweep", m);
      const TuneEntry te{(int)k, (int)t, m >= 0 ? m : NAN};
      if (valid_delay(te.delay_k) && te.cta_threads > 0 && !g_tune.count(key)) g_tune[key] = te;
    }
    pos = e + 1;
  }
}

void tune_file_write(const char* path) {
  std::ofstream f(path, std::ios::trunc);
  f << "{\n";
  size_t i = 0;
  for (auto& kv : g_tune) {
    char buf[160];
    snprintf(buf, sizeof buf, "{\"delay_k\": %d, \"cta_threads\": %d, \"ms_per_sweep\": %.6g}", kv.second.delay_k,
             kv.second.cta_threads, std::isfinite(kv.second.ms) ? kv.second.ms : -1.0);
    f << "  \"" << kv.first << "\": " << buf << (++i < g_tune.size() ? ",\n" : "\n");
  }
  f << "}\n";
}

pqmc_status autotune_run(int n, const pqmc_chain_spec* specs, const pqmc_opts& o, pqmc_tune* out) {
  memset(out, 0, sizeof *out);
  std::vector<int> ks = o.delay_k ? std::vector<int>{o.delay_k} : std::vector<int>{8, 16, 32, 64};
  std::vector<int> tpbs;
  if (o.cta_threads) tpbs = {o.cta_threads};
  else if (o.dense_chains) tpbs = {64, 128};
  else if (o.prec == PQMC_FP64) tpbs = {64, 128, 256};
  else tpbs = {64, 128, 256, 512};
  // proxy batch: the same chains with a shorter projection
  std::vector<pqmc_chain_spec> proxy(specs, specs + n);
  int lp_max = 0;
  for (auto& s : proxy) {
    const int Ltau = (int)std::lround(s.two_theta / s.dtau);
    const int lp = proxy_ltau(Ltau, o.n_stab);
    s.two_theta = lp * s.dtau;
    lp_max = std::max(lp_max, lp);
  }
  pqmc_opts po = o;
  po.delay_k = ks.back();
  po.cta_threads = tpbs.front();
  po.accept_log = 0;
  po.max_meas = 1;
  po.dg_fp64 = 0;
  pqmc_ctx* ctx = nullptr;
  pqmc_status st = build_ctx(n, proxy.data(), &po, &ctx, kMaxDelay);
  if (st != PQMC_OK) return st;
  double best = INFINITY;
  int nc = 0;
  for (int tpb : tpbs)
    for (int k : ks) {
      double ms = NAN;
      if (retarget(ctx, k, tpb) == PQMC_OK) ms = time_sweeps(ctx);
      if (nc < 32) {
        out->cand_delay_k[nc] = k;
        out->cand_cta_threads[nc] = tpb;
        out->cand_ms[nc] = ms;
        ++nc;
      }
      if (ms < best) {
        best = ms;
        out->delay_k = k;
        out->cta_threads = tpb;
      }
    }
  pqmc_free(ctx);
  out->n_candidates = nc;
  out->ms_per_sweep = best;
  out->proxy_ltau = lp_max;
  if (!std::isfinite(best)) return fail(nullptr, PQMC_ECUDA, "autotune: no candidate ran");
  return PQMC_OK;
}

pqmc_status autotune_cached(int n, const pqmc_chain_spec* specs, const pqmc_opts& o, pqmc_tune* out) {
  const std::string key = tune_key(n, specs, o);
  const char* path = getenv("PQMC_AUTOTUNE_CACHE");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (path && *path && !g_tune_file_read) {
      tune_file_read(path);
      g_tune_file_read = true;
    }
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      memset(out, 0, sizeof *out);
      out->delay_k = it->second.delay_k;
      out->cta_threads = it->second.cta_threads;
      out->ms_per_sweep = it->second.ms;
      out->from_cache = 1;
      return PQMC_OK;
    }
  }
  const pqmc_status st = autotune_run(n, specs, o, out);
  if (st != PQMC_OK) return st;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = TuneEntry{out->delay_k, out->cta_threads, out->ms_per_sweep};
  if (path && *path) tune_file_write(path);
  return PQMC_OK;
}

pqmc_status read_state(pqmc_ctx* ctx, int chain, ChainState& st) {
  cudaError_t e = cudaMemcpy(&st, ctx->desc[chain].st, sizeof st, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? PQMC_OK : cuda_fail(ctx, e, "state copy");
}

pqmc_status read_records(pqmc_ctx* ctx, int chain, std::vector<double>& rec, int& n) {
  ChainState st;
  pqmc_status s = read_state(ctx, chain, st);
  if (s != PQMC_OK) return s;
  n = std::min(st.n_meas, ctx->opts.max_meas);
  rec.resize((size_t)n * kRecord);
  if (n == 0) return PQMC_OK;
  cudaError_t e = cudaMemcpy(rec.data(), ctx->desc[chain].meas, rec.size() * 8, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? PQMC_OK : cuda_fail(ctx, e, "record copy");
}

// Device regions of the arena that hold one chain's Markov-chain state.
// stacks_only: what a recomputation of G from the fields overwrites (G, the
// stacks, their log-determinants, the counters); otherwise also the fields,
// the measurement records, the stabilisation-error history, the accept log
// and the latest record. Model tables, trial orbitals and the phase scratch
// are not state: they are rebuilt at creation or rewritten before use.
struct Region { size_t off, bytes; };

std::vector<Region> chain_state_regions(const pqmc_ctx* ctx, int c, bool stacks_only) {
  const HostChain& h = ctx->chains[c];
  const size_t blk = (size_t)h.N * h.nmax * 8;
  std::vector<Region> r = {{h.off_G, 2ull * h.N * h.ld * ctx->tsize},
                           {h.off_Rst, (size_t)(h.nb + 1) * 2 * blk},
                           {h.off_Lst, (size_t)(h.nb + 1) * 2 * blk},
                           {h.off_Rlog, (size_t)(h.nb + 1) * 4 * 8},
                           {h.off_Llog, (size_t)(h.nb + 1) * 4 * 8},
                           {h.off_state, sizeof(ChainState)}};
  if (!stacks_only) {
    r.push_back({h.off_fields, (size_t)(h.Ltau + 2) * h.nfld});
    r.push_back({h.off_meas, (size_t)ctx->opts.max_meas * kRecord * 8});
    r.push_back({h.off_dG, (size_t)kDGHistory * 8});
    r.push_back({h.off_acc, (size_t)ctx->opts.accept_log});
    r.push_back({ctx->off_last + (size_t)c * kRecord * 8, (size_t)kRecord * 8});
  }
  return r;
}

// Checkpoint layout: this header, then every chain's state regions in the
// order of chain_state_regions, chain by chain (little-endian, as on the
// device).
struct CkptHeader {
  char magic[8];
  uint32_t version, n_chains;
  int32_t prec, n_stab, delay_k, max_meas, accept_log, chain_offset;
  uint64_t seed, spec_hash, payload;
  uint32_t sweep_index, pad;
};
constexpr char kCkptMagic[8] = {'P', 'Q', 'M', 'C', 'C', 'K', 'P', 0};

// FNV-1a over the quantities that fix each chain's layout and dynamics
uint64_t spec_hash(const pqmc_ctx* ctx) {
  uint64_t hsh = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) { hsh ^= b[i]; hsh *= 1099511628211ull; }
  };
  for (const HostChain& h : ctx->chains) {
    const pqmc_chain_spec& s = h.spec;
    const int iv[] = {s.lattice.kind, s.lattice.Lx, s.lattice.Ly, h.N, h.nup, h.ndn, h.Ltau, h.nfld};
    const double dv[] = {s.lattice.t, s.lattice.tp, s.U, s.dtau, s.two_theta, s.trial.g, s.trial.M_N, s.trial.tiebreak};
    mix(iv, sizeof iv);
    mix(dv, sizeof dv);
  }
  return hsh;
}

size_t checkpoint_payload(const pqmc_ctx* ctx) {
  size_t t = 0;
  for (int c = 0; c < (int)ctx->chains.size(); ++c)
    for (const Region& r : chain_state_regions(ctx, c, false)) t += r.bytes;
  return t;
}

// ratio estimate sum(s O)/sum(s) with a delete-one-group jackknife error over
// groups given by their sums so[g] = sum s O, ss[g] = sum s
void jackknife(size_t nb, const double* so, const double* ss, double& mean, double& err) {
  double tso = 0, tss = 0;
  for (size_t b = 0; b < nb; ++b) {
    tso += so[b];
    tss += ss[b];
  }
  mean = tso / tss;
  if (nb < 2) { err = NAN; return; }
  std::vector<double> jk(nb);
  double m = 0;
  for (size_t b = 0; b < nb; ++b) { jk[b] = (tso - so[b]) / (tss - ss[b]); m += jk[b]; }
  m /= nb;
  double v = 0;
  for (size_t b = 0; b < nb; ++b) v += (jk[b] - m) * (jk[b] - m);
  err = std::sqrt((double)(nb - 1) / nb * v);
}

// the same over groups of records; the mean is taken over every record
// (all_sO / all_s), the error over the groups
void estimate(const std::vector<std::vector<double>>& groups_sO, const std::vector<std::vector<double>>& groups_s,
              double all_sO, double all_s, double& mean, double& err) {
  const size_t nb = groups_s.size();
  std::vector<double> so(nb, 0.0), ss(nb, 0.0);
  for (size_t b = 0; b < nb; ++b) {
    for (double v : groups_sO[b]) so[b] += v;
    for (double v : groups_s[b]) ss[b] += v;
  }
  jackknife(nb, so.data(), ss.data(), mean, err);
  mean = all_sO / all_s;
}

}  // namespace

extern "C" {

pqmc_status pqmc_init(const pqmc_lattice* lattice, double U, double dtau, double two_theta, const pqmc_trial* trial,
                      const pqmc_opts* opts, pqmc_ctx** out) {
  if (!lattice || !trial || !opts) return fail(nullptr, PQMC_EINVAL, "NULL argument");
  if (opts->n_chains < 1) return fail(nullptr, PQMC_EINVAL, "n_chains must be >= 1");
  std::vector<pqmc_chain_spec> specs(opts->n_chains);
  for (auto& s : specs) {
    s.lattice = *lattice;
    s.U = U;
    s.dtau = dtau;
    s.two_theta = two_theta;
    s.trial = *trial;
  }
  return build_ctx(opts->n_chains, specs.data(), opts, out);
}

pqmc_status pqmc_init_batch(int n, const pqmc_chain_spec* specs, const pqmc_opts* opts, pqmc_ctx** out) {
  return build_ctx(n, specs, opts, out);
}

pqmc_status pqmc_autotune(int n, const pqmc_chain_spec* specs, const pqmc_opts* opts, pqmc_tune* out) {
  NvtxRange range("pqmc_autotune");
  if (n < 1 || !specs || !opts || !out) return fail(nullptr, PQMC_EINVAL, "need n >= 1, specs, opts and out");
  if (opts->delay_k != 0 && !valid_delay(opts->delay_k))
    return fail(nullptr, PQMC_EINVAL, "delay_k must be 0, 8, 16, 32 or 64");
  for (int c = 0; c < n; ++c) {
    std::string why;
    if (check_spec(specs[c], opts->n_stab, why) != PQMC_OK)
      return fail(nullptr, PQMC_EINVAL, "chain " + std::to_string(c) + ": " + why);
  }
  return autotune_cached(n, specs, *opts, out);
}

pqmc_status pqmc_get_launch(pqmc_ctx* ctx, int* out) {
  if (!ctx || !out) return PQMC_EINVAL;
  out[0] = ctx->opts.delay_k;
  out[1] = ctx->tpb;
  out[2] = ctas_per_sm(ctx->prec, ctx->tpb, ctx->boost);
  out[3] = (int)ctx->res_bytes;
  return PQMC_OK;
}

namespace {

// Sweeps of a spread context: one captured graph per (direction, measure)
// holding the kernel sequence of one sweep and the advance of the sweep
// index, replayed once per sweep in direction order.
pqmc_status spread_sweeps(pqmc_ctx* ctx, int n_sweeps, int meas) {
  for (int k = 0; k < n_sweeps; ++k) {
    const int parity = (int)((ctx->sweep_index + (uint32_t)k) & 1u);
    pqmc_ctx::GraphEntry* ge = nullptr;
    for (auto& g : ctx->graphs)
      if (g.n_sweeps == parity && g.measure == meas) ge = &g;
    cudaError_t e = cudaSuccess;
    if (!ge) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      size_t nodes = 0;
      e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t el = spread_sweep(ctx->plan, parity, meas, ctx->stream);
        if (el == cudaSuccess) el = launch_advance(ctx->d_sweep, 1, ctx->stream);
        e = cudaStreamEndCapture(ctx->stream, &graph);
        if (e == cudaSuccess) e = el;
      }
      if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nullptr, &nodes);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "spread sweep graph capture");
      ctx->graphs.push_back({parity, meas, exec, nodes});
      ge = &ctx->graphs.back();
    }
    e = cudaGraphLaunch(ge->exec, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "spread sweep graph launch");
    ctx->launches += (long)ge->kernels;
  }
  ctx->sweep_index += (uint32_t)n_sweeps;
  return PQMC_OK;
}

}  // namespace

pqmc_status pqmc_sweep(pqmc_ctx* ctx, int n_sweeps, int measure) {
  NvtxRange range("pqmc_sweep");
  if (!ctx || n_sweeps < 0) return PQMC_EINVAL;
  if (ctx->sticky != PQMC_OK) return (pqmc_status)ctx->sticky;
  if (n_sweeps == 0) return PQMC_OK;
  const int meas = measure ? 1 : 0;
  if (ctx->spread) return spread_sweeps(ctx, n_sweeps, meas);
  // one captured graph per (n_sweeps, measure): the sweep launch and the
  // advance of the device-side sweep index, replayed on the context's stream
  cudaGraphExec_t exec = nullptr;
  for (auto& g : ctx->graphs)
    if (g.n_sweeps == n_sweeps && g.measure == meas) exec = g.exec;
  cudaError_t e = cudaSuccess;
  if (!exec) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t el = launch_sweep(ctx->prec, ctx->tpb, ctx->boost, ctx->d_desc_run, (int)ctx->chains.size(), ctx->opts.seed,
                                          ctx->d_sweep, n_sweeps, meas, ctx->res_bytes, ctx->d_err, ctx->stream);
      e = cudaStreamEndCapture(ctx->stream, &graph);
      if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sweep graph capture");
    ctx->graphs.push_back({n_sweeps, meas, exec, 2});
  }
  e = cudaGraphLaunch(exec, ctx->stream);
  ctx->launches += 2;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sweep graph launch");
  ctx->sweep_index += (uint32_t)n_sweeps;
  return PQMC_OK;
}

pqmc_status pqmc_synchronize(pqmc_ctx* ctx) {
  NvtxRange range("pqmc_synchronize");
  if (!ctx) return PQMC_EINVAL;
  return sync_check(ctx);
}

pqmc_status pqmc_measure(pqmc_ctx* ctx, int chain, pqmc_obs* out) {
  NvtxRange range("pqmc_measure");
  if (!ctx || !out || chain < -1 || chain >= (int)ctx->chains.size()) return PQMC_EINVAL;
  pqmc_status s = sync_check(ctx);
  if (s != PQMC_OK) return s;
  const int c0 = chain < 0 ? 0 : chain, c1 = chain < 0 ? (int)ctx->chains.size() : chain + 1;
  std::vector<std::vector<double>> gs, gE, gD;
  long long prop = 0, acc = 0;
  double maxdG = 0;
  long nm = 0;
  std::vector<std::vector<double>> per_s, per_E, per_D, per_S;
  for (int c = c0; c < c1; ++c) {
    std::vector<double> rec;
    int n = 0;
    if ((s = read_records(ctx, c, rec, n)) != PQMC_OK) return s;
    ChainState st;
    if ((s = read_state(ctx, c, st)) != PQMC_OK) return s;
    prop += st.n_prop;
    acc += st.n_acc;
    maxdG = std::max(maxdG, st.max_dG);
    nm += n;
    std::vector<double> sv(n), Ev(n), Dv(n), Sv(n);
    for (int m = 0; m < n; ++m) {
      sv[m] = rec[(size_t)m * kRecord + 0];
      Ev[m] = sv[m] * rec[(size_t)m * kRecord + 1];
      Dv[m] = sv[m] * rec[(size_t)m * kRecord + 2];
      Sv[m] = sv[m] * rec[(size_t)m * kRecord + 5];
    }
    per_s.push_back(sv);
    per_E.push_back(Ev);
    per_D.push_back(Dv);
    per_S.push_back(Sv);
  }
  // groups: chains when pooling several, else up to 20 bins of consecutive sweeps
  std::vector<std::vector<double>> bs, bE, bD, bS;
  if (per_s.size() >= 2) {
    bs = per_s; bE = per_E; bD = per_D; bS = per_S;
  } else if (!per_s.empty()) {
    const int n = (int)per_s[0].size();
    const int nbins = std::max(1, std::min(n, 20));
    const int per = std::max(1, n / nbins);
    for (int b = 0; b < nbins && (b + 1) * per <= n; ++b) {
      bs.emplace_back(per_s[0].begin() + b * per, per_s[0].begin() + (b + 1) * per);
      bE.emplace_back(per_E[0].begin() + b * per, per_E[0].begin() + (b + 1) * per);
      bD.emplace_back(per_D[0].begin() + b * per, per_D[0].begin() + (b + 1) * per);
      bS.emplace_back(per_S[0].begin() + b * per, per_S[0].begin() + (b + 1) * per);
    }
  }
  memset(out, 0, sizeof *out);
  out->n_meas = nm;
  out->accept = prop ? (double)acc / prop : 0.0;
  out->max_dG = maxdG;
  if (nm == 0 || bs.empty()) {
    out->E = out->E_err = out->docc = out->docc_err = out->sign = out->sign_err = NAN;
    out->s_afm = out->s_afm_err = NAN;
    return PQMC_OK;
  }
  // means over every record (a single chain's tail beyond the last full bin
  // included), errors over the groups
  double tot_s = 0, tot_E = 0, tot_D = 0, tot_S = 0;
  for (size_t c = 0; c < per_s.size(); ++c)
    for (size_t m = 0; m < per_s[c].size(); ++m) {
      tot_s += per_s[c][m];
      tot_E += per_E[c][m];
      tot_D += per_D[c][m];
      tot_S += per_S[c][m];
    }
  estimate(bE, bs, tot_E, tot_s, out->E, out->E_err);
  estimate(bD, bs, tot_D, tot_s, out->docc, out->docc_err);
  estimate(bS, bs, tot_S, tot_s, out->s_afm, out->s_afm_err);
  // average sign: mean of s with the same grouping
  std::vector<std::vector<double>> ones;
  for (auto& g : bs) ones.emplace_back(g.size(), 1.0);
  estimate(bs, ones, tot_s, (double)nm, out->sign, out->sign_err);
  return PQMC_OK;
}

pqmc_status pqmc_get_measurements(pqmc_ctx* ctx, int chain, double* out, long* n) {
  if (!chain_ok(ctx, chain) || !out || !n || *n < 0) return PQMC_EINVAL;
  pqmc_status s = sync_check(ctx);
  if (s != PQMC_OK && s != PQMC_ENAN && s != PQMC_ESTAB) return s;
  std::vector<double> rec;
  int m = 0;
  if ((s = read_records(ctx, chain, rec, m)) != PQMC_OK) return s;
  const long k = std::min<long>(*n, m);
  memcpy(out, rec.data(), (size_t)k * kRecord * 8);
  *n = k;
  return PQMC_OK;
}

pqmc_status pqmc_get_last_records(pqmc_ctx* ctx, double* out) {
  if (!ctx || !out) return PQMC_EINVAL;
  pqmc_status s = sync_check(ctx);
  if (s != PQMC_OK) return s;
  cudaError_t e = cudaMemcpy(out, ctx->d_arena + ctx->off_last, ctx->chains.size() * kRecord * 8,
                             cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? PQMC_OK : cuda_fail(ctx, e, "record copy");
}

pqmc_status pqmc_set_fields(pqmc_ctx* ctx, int chain, const int8_t* fields) {
  if (!chain_ok(ctx, chain) || !fields) return PQMC_EINVAL;
  if (ctx->sweep_index & 1u) return fail(ctx, PQMC_EINVAL, "set_fields needs an even number of sweeps done");
  if (ctx->sticky != PQMC_OK) return (pqmc_status)ctx->sticky;
  const HostChain& h = ctx->chains[chain];
  const size_t nf = (size_t)(h.Ltau + 2) * h.nfld;
  for (size_t i = 0; i < nf; ++i)
    if (fields[i] != 1 && fields[i] != -1) return fail(ctx, PQMC_EINVAL, "fields must be +1 or -1");
  cudaError_t e = cudaMemcpyAsync(ctx->desc[chain].fields, fields, nf, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fields upload");
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fields upload");
  e = launch_init(ctx->prec, ctx->tpb, ctx->boost, ctx->d_desc, chain, 1, ctx->opts.seed, ctx->res_bytes, ctx->d_err,
                  ctx->stream, -1);
  ctx->launches++;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "init launch");
  return sync_check(ctx);
}

pqmc_status pqmc_get_fields(pqmc_ctx* ctx, int chain, int8_t* fields) {
  if (!chain_ok(ctx, chain) || !fields) return PQMC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  const HostChain& h = ctx->chains[chain];
  e = cudaMemcpy(fields, ctx->desc[chain].fields, (size_t)(h.Ltau + 2) * h.nfld, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? PQMC_OK : cuda_fail(ctx, e, "fields copy");
}

pqmc_status pqmc_get_green(pqmc_ctx* ctx, int chain, int spin, double* out) {
  if (!chain_ok(ctx, chain) || !out || spin < 0 || spin > 1) return PQMC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  const HostChain& h = ctx->chains[chain];
  const size_t cnt = (size_t)h.N * h.ld;
  std::vector<unsigned char> buf(cnt * ctx->tsize);
  e = cudaMemcpy(buf.data(), (unsigned char*)ctx->desc[chain].G + spin * cnt * ctx->tsize, buf.size(),
                 cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "G copy");
  for (int i = 0; i < h.N; ++i)
    for (int j = 0; j < h.N; ++j) {
      const size_t k = (size_t)i * h.ld + j;
      out[(size_t)i * h.N + j] = ctx->tsize == 8 ? reinterpret_cast<double*>(buf.data())[k]
                                                 : (double)reinterpret_cast<float*>(buf.data())[k];
    }
  return PQMC_OK;
}

pqmc_status pqmc_get_green_at(pqmc_ctx* ctx, int chain, int spin, int b, double* out) {
  NvtxRange range("pqmc_get_green_at");
  if (!chain_ok(ctx, chain) || !out || spin < 0 || spin > 1) return PQMC_EINVAL;
  const HostChain& h = ctx->chains[chain];
  if (b < 0 || b > h.nb) return fail(ctx, PQMC_EINVAL, "stabilisation point out of range");
  if (ctx->sticky != PQMC_OK) return (pqmc_status)ctx->sticky;
  pqmc_status st = sync_check(ctx);
  if (st != PQMC_OK) return st;
  // keep the chain's state aside, recompute, read G, put the state back
  const std::vector<Region> regs = chain_state_regions(ctx, chain, true);
  size_t total = 0;
  for (const Region& r : regs) total += r.bytes;
  unsigned char* keep = nullptr;
  cudaError_t e = cudaMalloc(&keep, total);
  if (e != cudaSuccess) return fail(ctx, PQMC_ENOMEM, std::string("state copy: ") + cudaGetErrorString(e));
  size_t at = 0;
  for (const Region& r : regs) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(keep + at, ctx->d_arena + r.off, r.bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    at += r.bytes;
  }
  if (e == cudaSuccess)
    e = launch_init(ctx->prec, ctx->tpb, ctx->boost, ctx->d_desc, chain, 1, ctx->opts.seed, ctx->res_bytes, ctx->d_err,
                    ctx->stream, b);
  ctx->launches++;
  if (e != cudaSuccess) { cudaStreamSynchronize(ctx->stream); cudaFree(keep); return cuda_fail(ctx, e, "recompute launch"); }
  st = sync_check(ctx);
  if (st == PQMC_OK) st = pqmc_get_green(ctx, chain, spin, out);
  at = 0;
  e = cudaSuccess;
  for (const Region& r : regs) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_arena + r.off, keep + at, r.bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    at += r.bytes;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(keep);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "state restore");
  return st;
}

pqmc_status pqmc_checkpoint(pqmc_ctx* ctx, void* buf, size_t* len) {
  NvtxRange range("pqmc_checkpoint");
  if (!ctx || !len) return PQMC_EINVAL;
  if (ctx->sticky != PQMC_OK) return (pqmc_status)ctx->sticky;
  pqmc_status st = sync_check(ctx);
  if (st != PQMC_OK) return st;
  const size_t payload = checkpoint_payload(ctx);
  const size_t total = sizeof(CkptHeader) + payload;
  if (!buf) { *len = total; return PQMC_OK; }
  if (*len < total) { *len = total; return fail(ctx, PQMC_EINVAL, "checkpoint buffer too small"); }
  CkptHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, kCkptMagic, sizeof hd.magic);
  hd.version = 2;
  hd.n_chains = (uint32_t)ctx->chains.size();
  hd.prec = ctx->prec;
  hd.n_stab = ctx->opts.n_stab;
  hd.delay_k = ctx->opts.delay_k;
  hd.max_meas = ctx->opts.max_meas;
  hd.accept_log = ctx->opts.accept_log;
  hd.chain_offset = ctx->opts.chain_offset;
  hd.seed = ctx->opts.seed;
  hd.spec_hash = spec_hash(ctx);
  hd.payload = payload;
  hd.sweep_index = ctx->sweep_index;
  unsigned char* p = static_cast<unsigned char*>(buf);
  memcpy(p, &hd, sizeof hd);
  size_t at = sizeof hd;
  for (int c = 0; c < (int)ctx->chains.size(); ++c)
    for (const Region& r : chain_state_regions(ctx, c, false)) {
      if (r.bytes) {
        cudaError_t e = cudaMemcpy(p + at, ctx->d_arena + r.off, r.bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "checkpoint copy");
      }
      at += r.bytes;
    }
  *len = total;
  return PQMC_OK;
}

pqmc_status pqmc_restore(pqmc_ctx* ctx, const void* buf, size_t len) {
  NvtxRange range("pqmc_restore");
  if (!ctx || !buf) return PQMC_EINVAL;
  CkptHeader hd;
  if (len < sizeof hd) return fail(ctx, PQMC_EINVAL, "not a checkpoint (too short)");
  memcpy(&hd, buf, sizeof hd);
  if (memcmp(hd.magic, kCkptMagic, sizeof hd.magic) != 0 || hd.version != 2)
    return fail(ctx, PQMC_EINVAL, "not a checkpoint of this library");
  const char* what = nullptr;
  if (hd.n_chains != (uint32_t)ctx->chains.size()) what = "chain count";
  else if (hd.prec != ctx->prec) what = "precision";
  else if (hd.n_stab != ctx->opts.n_stab || hd.delay_k != ctx->opts.delay_k) what = "n_stab or delay_k";
  else if (hd.max_meas != ctx->opts.max_meas || hd.accept_log != ctx->opts.accept_log) what = "max_meas or accept_log";
  else if (hd.chain_offset != ctx->opts.chain_offset || hd.seed != ctx->opts.seed) what = "seed or chain_offset";
  else if (hd.spec_hash != spec_hash(ctx)) what = "chain specs";
  else if (hd.payload != checkpoint_payload(ctx) || len != sizeof hd + hd.payload) what = "size";
  if (what) return fail(ctx, PQMC_EINVAL, std::string("checkpoint of a different context: ") + what);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  const unsigned char* p = static_cast<const unsigned char*>(buf);
  size_t at = sizeof hd;
  for (int c = 0; c < (int)ctx->chains.size(); ++c)
    for (const Region& r : chain_state_regions(ctx, c, false)) {
      if (r.bytes) {
        e = cudaMemcpy(ctx->d_arena + r.off, p + at, r.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "restore copy");
      }
      at += r.bytes;
    }
  // the sweep index (host and device copies) and a clean error word: the
  // checkpoint was taken without an error, so the chains run on from it
  const int words[2] = {0, (int)hd.sweep_index};
  e = cudaMemcpy(ctx->d_err, words, sizeof words, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "restore copy");
  ctx->sweep_index = hd.sweep_index;
  ctx->sticky = PQMC_OK;
  ctx->err.clear();
  return PQMC_OK;
}

pqmc_status pqmc_write_run_log(pqmc_ctx* ctx, const char* path) {
  NvtxRange range("pqmc_write_run_log");
  if (!ctx || !path) return PQMC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  std::ofstream f(path, std::ios::app);
  if (!f) return fail(ctx, PQMC_EINVAL, std::string("cannot open ") + path);
  f.precision(17);
  const char* prec[] = {"fp64", "fp32", "bf16x3"};
  for (int c = 0; c < (int)ctx->chains.size(); ++c) {
    std::vector<double> rec;
    int n = 0;
    pqmc_status s = read_records(ctx, c, rec, n);
    if (s != PQMC_OK) return s;
    ChainState st;
    if ((s = read_state(ctx, c, st)) != PQMC_OK) return s;
    const HostChain& h = ctx->chains[c];
    // sign-reweighted means over the chain's records
    double ts = 0, tE = 0, tD = 0, tS = 0;
    for (int m = 0; m < n; ++m) {
      const double sg = rec[(size_t)m * kRecord + 0];
      ts += sg;
      tE += sg * rec[(size_t)m * kRecord + 1];
      tD += sg * rec[(size_t)m * kRecord + 2];
      tS += sg * rec[(size_t)m * kRecord + 5];
    }
    auto num = [&](double v) {
      std::ostringstream o;
      o.precision(17);
      if (std::isfinite(v)) o << v; else o << "null";
      return o.str();
    };
    const int nd = std::min(st.n_dG, kDGHistory);
    double dG_last = NAN;
    if (nd > 0) {
      double v = 0;
      cudaMemcpy(&v, ctx->desc[c].dG + (st.n_dG - 1) % kDGHistory, sizeof v, cudaMemcpyDeviceToHost);
      dG_last = v;
    }
    f << "{\"chain\": " << c << ", \"chain_index\": " << ctx->desc[c].chain_index << ", \"sites\": " << h.N
      << ", \"slices\": " << h.Ltau + 2 << ", \"precision\": \"" << prec[ctx->prec] << "\", \"sweeps\": "
      << ctx->sweep_index << ", \"records\": " << n << ", \"E_per_site\": " << num(ts != 0 ? tE / ts : NAN)
      << ", \"docc\": " << num(ts != 0 ? tD / ts : NAN) << ", \"s_afm\": " << num(ts != 0 ? tS / ts : NAN)
      << ", \"sign\": " << num(n ? ts / n : NAN) << ", \"accept\": "
      << num(st.n_prop ? (double)st.n_acc / st.n_prop : NAN) << ", \"max_dG\": " << num(st.max_dG)
      << ", \"dG_last\": " << num(dG_last) << ", \"stabilisations\": " << st.n_dG << ", \"logw\": ["
      << num(st.logw[0][0]) << ", " << num(st.logw[1][0]) << "], \"weight_sign\": [" << num(st.logw[0][1])
      << ", " << num(st.logw[1][1]) << "], \"running_sign\": " << num(st.sign_running)
      << ", \"error\": " << st.err << "}\n";
  }
  return f ? PQMC_OK : fail(ctx, PQMC_EINVAL, std::string("write failed: ") + path);
}

pqmc_status pqmc_get_weight(pqmc_ctx* ctx, int chain, double* out) {
  if (!chain_ok(ctx, chain) || !out) return PQMC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  ChainState st;
  pqmc_status s = read_state(ctx, chain, st);
  if (s != PQMC_OK) return s;
  out[0] = st.logw[0][0]; out[1] = st.logw[0][1];
  out[2] = st.logw[1][0]; out[3] = st.logw[1][1];
  return PQMC_OK;
}

pqmc_status pqmc_get_accept_log(pqmc_ctx* ctx, int chain, uint8_t* out, long n) {
  if (!chain_ok(ctx, chain) || !out || n < 0 || n > ctx->opts.accept_log) return PQMC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  if (n == 0) return PQMC_OK;
  e = cudaMemcpy(out, ctx->desc[chain].acc_log, (size_t)n, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? PQMC_OK : cuda_fail(ctx, e, "accept log copy");
}

pqmc_status pqmc_get_stab_errors(pqmc_ctx* ctx, int chain, double* out, long* n) {
  if (!chain_ok(ctx, chain) || !out || !n || *n < 0) return PQMC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  ChainState st;
  pqmc_status s = read_state(ctx, chain, st);
  if (s != PQMC_OK) return s;
  std::vector<double> ring(kDGHistory);
  e = cudaMemcpy(ring.data(), ctx->desc[chain].dG, kDGHistory * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "dG copy");
  const long total = st.n_dG;
  const long kept = std::min<long>(total, kDGHistory);
  const long k = std::min<long>(*n, kept);
  const long first = total - kept;
  for (long m = 0; m < k; ++m) out[m] = ring[(first + m) % kDGHistory];
  *n = k;
  return PQMC_OK;
}

pqmc_status pqmc_get_phase_cycles(pqmc_ctx* ctx, int chain, long long* out) {
  if (!chain_ok(ctx, chain) || !out) return PQMC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  ChainState st;
  pqmc_status s = read_state(ctx, chain, st);
  if (s != PQMC_OK) return s;
  for (int p = 0; p < kPhases; ++p) out[p] = st.cycles[p];
  return PQMC_OK;
}

pqmc_status pqmc_get_dims(pqmc_ctx* ctx, int chain, int* out) {
  if (!chain_ok(ctx, chain) || !out) return PQMC_EINVAL;
  const HostChain& h = ctx->chains[chain];
  out[0] = h.N; out[1] = h.nup; out[2] = h.ndn; out[3] = h.Ltau; out[4] = ctx->opts.n_stab; out[5] = ctx->opts.delay_k;
  out[6] = h.nfld;
  return PQMC_OK;
}

int pqmc_num_chains(const pqmc_ctx* ctx) { return ctx ? (int)ctx->chains.size() : -1; }

long pqmc_launch_count(const pqmc_ctx* ctx) { return ctx ? ctx->launches : 0; }

size_t pqmc_device_bytes(const pqmc_ctx* ctx) { return ctx ? ctx->arena_bytes : 0; }
size_t pqmc_upload_bytes(const pqmc_ctx* ctx) { return ctx ? ctx->upload_bytes : 0; }

const char* pqmc_last_error(const pqmc_ctx* ctx) {
  if (!ctx) return g_init_error.c_str();
  return ctx->err.c_str();
}

void pqmc_free(pqmc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  if (ctx->d_arena) cudaFree(ctx->d_arena);
  if (ctx->d_desc) cudaFree(ctx->d_desc);
  if (ctx->d_desc_run) cudaFree(ctx->d_desc_run);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

pqmc_status pqmc_host_model(const pqmc_lattice* lattice, double dtau, const pqmc_trial* trial, int spin, double* K,
                            double* expK, double* P, double* gap) {
  if (!lattice || spin < 0 || spin > 1) return fail(nullptr, PQMC_EINVAL, "bad argument");
  if (lattice->Lx < 1 || lattice->Ly < 1 || lattice->Lx > 64 || lattice->Ly > 64 ||
      (lattice->kind != 0 && lattice->kind != 1))
    return fail(nullptr, PQMC_EINVAL, "bad lattice");
  Lattice lat{lattice->kind, lattice->Lx, lattice->Ly, lattice->t, lattice->tp};
  const int N = lat.n_sites();
  std::vector<double> Km, eps, w, V, E;
  build_hopping(lat, Km, eps);
  if (K) memcpy(K, Km.data(), Km.size() * 8);
  if (expK) {
    if (!sym_eig(N, Km, w, V)) return fail(nullptr, PQMC_EINVAL, "eigensolver failed");
    expm_from_eig(N, w, V, -dtau, E);
    memcpy(expK, E.data(), E.size() * 8);
  }
  if (P || gap) {
    if (!trial) return fail(nullptr, PQMC_EINVAL, "trial is NULL");
    const int ns = spin == 0 ? (trial->N_up < 0 ? N / 2 : trial->N_up) : (trial->N_dn < 0 ? N / 2 : trial->N_dn);
    if (ns < 1 || ns > N) return fail(nullptr, PQMC_EINVAL, "bad N_sigma");
    std::vector<double> Pm;
    double g = 0;
    if (!trial_orbitals(lat, Km, eps, trial->M_N, trial->tiebreak, spin == 0 ? 1 : -1, ns, Pm, g))
      return fail(nullptr, PQMC_EINVAL, "eigensolver failed");
    if (P) memcpy(P, Pm.data(), Pm.size() * 8);
    if (gap) *gap = g;
  }
  return PQMC_OK;
}

pqmc_status pqmc_host_jackknife(int n_groups, const double* sO, const double* s, double* mean, double* err) {
  if (n_groups < 1 || !sO || !s || !mean || !err) return fail(nullptr, PQMC_EINVAL, "bad argument");
  jackknife((size_t)n_groups, sO, s, *mean, *err);
  return PQMC_OK;
}

pqmc_status pqmc_inject_error(pqmc_ctx* ctx, int chain, int code) {
  if (!chain_ok(ctx, chain) || (code != PQMC_ENAN && code != PQMC_ESTAB)) return PQMC_EINVAL;
  const int bits = code == PQMC_ENAN ? kErrNaN : kErrStab;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  // the chain's own error word (the sweep kernel skips a failed chain) and
  // the context-wide word that sync_check reads, as a failing kernel sets them
  e = cudaMemcpy(reinterpret_cast<unsigned char*>(ctx->desc[chain].st) + offsetof(ChainState, err), &bits,
                 sizeof bits, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->d_err, &bits, sizeof bits, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "error word copy");
  return PQMC_OK;
}

pqmc_status pqmc_host_eigh(int n, const double* A, double* w, double* V) {
  if (n < 1 || !A || !w || !V) return fail(nullptr, PQMC_EINVAL, "bad argument");
  std::vector<double> Am(A, A + (size_t)n * n), wm, Vm;
  if (!sym_eig(n, Am, wm, Vm)) return fail(nullptr, PQMC_EINVAL, "eigensolver did not converge");
  memcpy(w, wm.data(), (size_t)n * 8);
  memcpy(V, Vm.data(), (size_t)n * n * 8);
  return PQMC_OK;
}

}  // extern "C"

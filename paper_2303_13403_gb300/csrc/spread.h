// Host-side plan of a context whose chains are swept by the whole GPU
// (pqmc_opts.spread): the sizes the chains share and the device pointers the
// kernel sequence of spread.cuh needs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "chain.h"

namespace pqmc {

struct SpreadChainPtrs {
  unsigned char* sp;      // spread buffers (SpreadLayout)
  void* G;                // 2 x N x ld (T)
  const void* expKm;      // N x ld (T)
  const void* expKp;
  double* Rst;
  double* Lst;
};

struct SpreadPlan {
  int prec = 0;           // pqmc_precision
  int n = 0;              // chains
  int N = 0, ld = 0, nup = 0, ndn = 0, nmax = 0, Ltau = 0, n_stab = 0, nb = 0;
  const ChainDesc* d_desc = nullptr;
  uint64_t seed = 0;
  uint32_t* d_sweep = nullptr;
  int* d_err = nullptr;
  std::vector<SpreadChainPtrs> ch;
};

// Enqueue one sweep of every chain (up for an even sweep index, down for an
// odd one) on stream; measure at the middle slice when measure != 0.
cudaError_t spread_sweep(const SpreadPlan& p, int parity, int measure, cudaStream_t stream);

// Enqueue the initialisation of every chain from its fields (left stack,
// right block 0, G at tau = -1, running sign) with the same kernels.
cudaError_t spread_init(const SpreadPlan& p, cudaStream_t stream);

// Kernel attributes of the spread sequence (once per process, before capture).
cudaError_t spread_prepare();

}  // namespace pqmc

// Spread sweep (spread.cuh): the kernel sequence of the reduced paths (FP32
// and split BF16; the FP64 stabilisation steps live in spread_f64.cu).
#include "spread.cuh"

namespace pqmc {

cudaError_t spread_sweep_f32(const SpreadPlan& p, int mode, int measure, cudaStream_t st) {
  return spread_sweep_t<float>(p, mode, measure, st);
}

}  // namespace pqmc

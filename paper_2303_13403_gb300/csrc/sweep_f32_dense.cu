// Reduced-precision paths with dense chain packing (pqmc_opts.dense_chains):
// kernels for CTAs of 64 and 128 threads built for 16 and 8 chains per SM.
#include "sweep_kernels.cuh"

namespace pqmc {

#define PQMC_TPB_DISPATCH(CALL, ...) \
  do { \
    if (tpb == 64) return CALL<float, 64, 16>(__VA_ARGS__); \
    return CALL<float, 128, 8>(__VA_ARGS__); \
  } while (0)

PQMC_DEFINE_LAUNCHERS(f32_dense)

}  // namespace pqmc

// Reduced-precision paths (FP32 and split BF16, T = float): kernels for
// CTAs of 256 threads, two chains per SM (a 72-site chain's G and
// scratch in shared memory).
#include "sweep_kernels.cuh"

namespace pqmc {

#define PQMC_TPB_DISPATCH(CALL, ...) \
  do { \
    (void)tpb; \
    return CALL<float, 256, 2>(__VA_ARGS__); \
  } while (0)

PQMC_DEFINE_LAUNCHERS(f32_256)

}  // namespace pqmc

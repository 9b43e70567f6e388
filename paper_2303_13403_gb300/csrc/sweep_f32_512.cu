// Reduced-precision paths (FP32 and split BF16, T = float): kernels for
// CTAs of 512 threads, one chain per SM (large chains, G in global
// memory; BF16X3 wraps on the tensor cores).
#include "sweep_kernels.cuh"

namespace pqmc {

#define PQMC_TPB_DISPATCH(CALL, ...) \
  do { \
    (void)tpb; \
    return CALL<float, 512, 1>(__VA_ARGS__); \
  } while (0)

PQMC_DEFINE_LAUNCHERS(f32_512)

}  // namespace pqmc

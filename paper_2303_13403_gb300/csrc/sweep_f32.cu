// Reduced-precision paths (FP32 and split BF16, T = float): kernels for CTAs
// of 64, 128 and 256 threads, twice as many chains per SM as the FP64 path,
// and of 512 threads, one chain per SM (large chains).
#include "sweep_kernels.cuh"

namespace pqmc {

#define PQMC_TPB_DISPATCH(CALL, ...) \
  do { \
    if (tpb == 64) return CALL<float, 64, 8>(__VA_ARGS__); \
    if (tpb == 128) return CALL<float, 128, 4>(__VA_ARGS__); \
    if (tpb == 512) return CALL<float, 512, 1>(__VA_ARGS__); \
    return CALL<float, 256, 2>(__VA_ARGS__); \
  } while (0)

PQMC_DEFINE_LAUNCHERS(f32)

}  // namespace pqmc

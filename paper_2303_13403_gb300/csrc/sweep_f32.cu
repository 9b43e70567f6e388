// Reduced-precision paths (FP32 and split BF16, T = float): kernels for CTAs
// of 64 and 128 threads, twice as many chains per SM as the FP64 path (256
// threads: sweep_f32_256.cu; 512 threads, one chain per SM for large chains:
// sweep_f32_512.cu; one translation unit per CTA shape so that the build
// compiles them side by side).
#include "sweep_kernels.cuh"

namespace pqmc {

#define PQMC_TPB_DISPATCH(CALL, ...) \
  do { \
    if (tpb == 64) return CALL<float, 64, 8>(__VA_ARGS__); \
    return CALL<float, 128, 4>(__VA_ARGS__); \
  } while (0)

PQMC_DEFINE_LAUNCHERS(f32)

}  // namespace pqmc

// FP64 path: kernels for CTAs of 64, 128 and 256 threads (4, 2, 1 chains per
// 256 threads of an SM).
#include "sweep_kernels.cuh"

namespace pqmc {

#define PQMC_TPB_DISPATCH(CALL, ...) \
  do { \
    if (tpb == 64) return CALL<double, 64, 4>(__VA_ARGS__); \
    if (tpb == 128) return CALL<double, 128, 2>(__VA_ARGS__); \
    return CALL<double, 256, 1>(__VA_ARGS__); \
  } while (0)

PQMC_DEFINE_LAUNCHERS(f64)

}  // namespace pqmc

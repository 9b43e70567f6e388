// Micro-benchmarks of the arithmetic pipes that bound the sweep kernel
// (pqmc_probe_pipes in include/pqmc.h).  They measure this GPU's FP64 FMA and
// FP64 tensor-core (DMMA) throughput, the FP32 FMA throughput, the latency of
// a dependent FP64 FMA / divide / square root, and the cost of an FP64 warp
// instruction with 1, 8, 16 or 32 active lanes, which decide how the
// stabilisation's FP64 loops are laid out.  Every loop has a fixed trip
// count; nothing waits on anything but the kernel's end.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pqmc.h"

namespace pqmc_probe {

constexpr int kIters = 4096;
constexpr int kChains = 8;   // independent accumulators per thread

// FP64 FMA throughput: kChains independent chains per thread
__global__ void dfma_tput(double* sink, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1.2345) sink[threadIdx.x] = s;
}

__global__ void ffma_tput(float* sink, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1.2345f) sink[threadIdx.x] = s;
}

// FP64 tensor-core throughput: mma.sync m8n8k4, 4 independent accumulators per warp
__global__ void dmma_tput(double* sink, double a, double b) {
  double acc[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = 0.0;
  const double av = a + threadIdx.x * 1e-9, bv = b - threadIdx.x * 1e-9;
  for (int i = 0; i < kIters / 4; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
  if (s == 1.2345) sink[threadIdx.x] = s;
}

// even warps run the DFMA loop of dfma_tput, odd warps the DMMA loop of
// dmma_tput: whether the two FP64 paths of an SM can be busy at the same time
__global__ void dfma_dmma_mix(double* sink, double a, double b) {
  const int warp = threadIdx.x >> 5;
  double s = 0;
  if ((warp & 1) == 0) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
    for (int i = 0; i < kIters; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
  } else {
    double acc[4][2];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = 0.0;
    const double av = a + threadIdx.x * 1e-9, bv = b - threadIdx.x * 1e-9;
    for (int i = 0; i < kIters / 4; ++i) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(acc[c][0]), "+d"(acc[c][1])
                     : "d"(av), "d"(bv));
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
  }
  if (s == 1.2345) sink[threadIdx.x] = s;
}

// one warp, `active` lanes running kChains independent FP64 chains: clock
// cycles per FP64 warp instruction
__global__ void dfma_partial(long long* cycles, double* sink, int active, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
  __syncwarp();
  const long long t0 = clock64();
  if ((int)threadIdx.x < active) {
    for (int i = 0; i < kIters / 4; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  __syncwarp();
  const long long t1 = clock64();
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1.2345) sink[threadIdx.x] = s;
  if (threadIdx.x == 0) *cycles = t1 - t0;
}

// dependent chains on one thread: latency in cycles of FMA, divide, sqrt.
// The operations are volatile PTX so that they stay between the clock reads.
__global__ void dep_latency(long long* cycles, double* sink, double a, double b) {
  double x = 1.0 + threadIdx.x, y = 2.0, z = 3.0;
  long long t0 = clock64();
#pragma unroll 1
  for (int i = 0; i < 256; ++i) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x) : "d"(a), "d"(b));
  long long t1 = clock64();
#pragma unroll 1
  for (int i = 0; i < 256; ++i) {
    asm volatile("add.rn.f64 %0, %0, 0d3FF0000000000000;" : "+d"(y));
    asm volatile("div.rn.f64 %0, %1, %0;" : "+d"(y) : "d"(a));
  }
  long long t2 = clock64();
#pragma unroll 1
  for (int i = 0; i < 256; ++i) {
    asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(z) : "d"(b));
    asm volatile("sqrt.rn.f64 %0, %0;" : "+d"(z));
  }
  long long t3 = clock64();
  if (x + y + z == 1.2345) sink[0] = x + y + z;
  cycles[0] = t1 - t0;
  cycles[1] = t2 - t1;
  cycles[2] = t3 - t2;
}

}  // namespace pqmc_probe

extern "C" pqmc_status pqmc_probe_pipes(double* out) {
  using namespace pqmc_probe;
  if (!out) return PQMC_EINVAL;
  int dev = 0, sms = 0, clk_khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PQMC_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  double* dsink = nullptr;
  long long* dcyc = nullptr;
  if (cudaMalloc(&dsink, 1024 * sizeof(double)) != cudaSuccess) return PQMC_ENOMEM;
  if (cudaMalloc(&dcyc, 8 * sizeof(long long)) != cudaSuccess) {
    cudaFree(dsink);
    return PQMC_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256;
  auto time_ms = [&](auto launch) {
    launch();                       // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms;
  };
  const double flop_fma = 2.0 * kIters * kChains * (double)blocks * threads;
  const double ms_d = time_ms([&] { dfma_tput<<<blocks, threads>>>(dsink, 0.999999, 1e-7); });
  const double ms_f = time_ms([&] { ffma_tput<<<blocks, threads>>>((float*)dsink, 0.999999f, 1e-7f); });
  const double ms_m = time_ms([&] { dmma_tput<<<blocks, threads>>>(dsink, 0.999999, 1e-7); });
  const double flop_mma = 2.0 * 8 * 8 * 4 * 4 * (kIters / 4) * (double)blocks * (threads / 32);
  const double ms_x = time_ms([&] { dfma_dmma_mix<<<blocks, threads>>>(dsink, 0.999999, 1e-7); });
  long long cyc[8] = {0};
  const int lanes[4] = {1, 8, 16, 32};
  double per_instr[4];
  for (int k = 0; k < 4; ++k) {
    dfma_partial<<<1, 32>>>(dcyc, dsink, lanes[k], 0.999999, 1e-7);
    cudaMemcpy(cyc, dcyc, sizeof(long long), cudaMemcpyDeviceToHost);
    per_instr[k] = (double)cyc[0] / ((kIters / 4) * kChains);
  }
  dep_latency<<<1, 1>>>(dcyc, dsink, 0.999999, 1e-7);
  cudaMemcpy(cyc, dcyc, 3 * sizeof(long long), cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaDeviceSynchronize();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(dsink);
  cudaFree(dcyc);
  if (e != cudaSuccess) return PQMC_ECUDA;
  out[0] = flop_fma / (ms_d * 1e-3) / 1e12;     // FP64 FMA TFLOP/s, all SMs
  out[1] = flop_mma / (ms_m * 1e-3) / 1e12;     // FP64 DMMA TFLOP/s
  out[2] = flop_fma / (ms_f * 1e-3) / 1e12;     // FP32 FMA TFLOP/s
  out[3] = (double)cyc[0] / 256;                // dependent FP64 FMA latency, cycles
  out[4] = (double)cyc[1] / 256;                // dependent FP64 add + divide, cycles
  out[5] = (double)cyc[2] / 256;                // dependent FP64 add + sqrt, cycles
  for (int k = 0; k < 4; ++k) out[6 + k] = per_instr[k];   // cycles per FP64 warp instruction, 1/8/16/32 lanes
  out[10] = sms;
  out[11] = clk_khz / 1e3;                      // reported SM clock, MHz
  // half the warps on each path: FP64 TFLOP/s of the mix, and its time
  // against the two halves run one after the other (1: one shared pipe,
  // 0.5: two independent ones)
  out[12] = 0.5 * (flop_fma + flop_mma) / (ms_x * 1e-3) / 1e12;
  out[13] = ms_x / (0.5 * (ms_d + ms_m));
  return PQMC_OK;
}

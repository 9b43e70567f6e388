#pragma once
// Split-precision GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
// C = A B for FP32 A (M x K) and B (K x N) with every operand split as
// x = hi + lo, hi = bf16(x), lo = bf16(x - hi), and
// C = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 in tensor memory
// (the same split as the mma.sync path; Henry, Tang & Heinecke 2019).
//
// One CTA computes the whole product in tiles of 128 rows x up to 192
// columns: the threads split a 128 x 64 slice of A and a 64-deep slice of B
// into BF16 hi/lo tiles in shared memory (canonical K-major layout without
// swizzle: 8 x 8 core matrices, 128 B each), one thread issues the
// 128 x N x 16 MMAs (three per 16-deep step) into a TMEM accumulator and
// commits them to an mbarrier; after the last slice the warps read the
// accumulator back (tcgen05.ld, warp w reads TMEM lanes 32 (w mod 4) ...)
// and hand every element to the epilogue through a row-major chunk in shared
// memory (so that the epilogue's global accesses are coalesced).  The
// accumulator lives in 256
// TMEM columns the CTA allocates once per launch (tc_alloc / tc_free).
//
// Every wait is bounded: a completion that does not arrive within
// kTcSpinLimit polls sets *err and the product is abandoned (the caller
// reports the error; the CTA still frees its TMEM before it exits).
#include <cuda_bf16.h>
#include <stdint.h>

namespace pqmc {

constexpr int kTcM = 128;                 // rows per tile (the MMA's M; the staging maps rows by & 127)
constexpr int kTcN = 192;                 // largest tile width (the MMA's N, multiple of 16); 192 keeps
                                          // the staging area within a 100 KB shared-memory carve-out
                                          // (more L1 for the chain's global-memory G and scratch)
constexpr int kTcK = 64;                  // depth of one staged slice (four 16-deep MMA steps)
constexpr int kTcCols = 256;              // TMEM columns held by the CTA
constexpr uint32_t kTcTileA = kTcM * kTcK * 2;          // bytes of one BF16 A tile
constexpr uint32_t kTcTileB = kTcN * kTcK * 2;          // bytes of one BF16 B tile
constexpr uint32_t kTcOffAlo = kTcTileA;
constexpr uint32_t kTcOffBhi = 2 * kTcTileA;
constexpr uint32_t kTcOffBlo = 2 * kTcTileA + kTcTileB;
constexpr uint32_t kTcOffBar = 2 * kTcTileA + 2 * kTcTileB;   // mbarrier (8 B), TMEM address (4 B), phase (4 B)
constexpr uint32_t kTcBytes = kTcOffBar + 64;                  // staging area of one CTA (80 KB + 64 B)
constexpr int kTcSpinLimit = 1 << 22;

// byte offset of element (r, k) of a K-major tile, k < kTcK: core matrix
// (r / 8, k / 8) at (r / 8) * SBO + (k / 8) * LBO, row r % 8 at 16 B steps
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (kTcK / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
constexpr uint32_t kTcLBO = 128;                      // next core matrix along K
constexpr uint32_t kTcSBO = (kTcK / 8) * 128;         // next core matrix along M / N

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), the
// descriptor version of the sm_100 family (bit 46), no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kTcLBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((kTcSBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n
__device__ __forceinline__ uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

// TMEM allocation of kTcCols columns by warp 0; every thread gets the address
__device__ __forceinline__ uint32_t tc_alloc(unsigned char* st) {
  uint32_t* slot = reinterpret_cast<uint32_t*>(st + kTcOffBar + 8);
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(st + kTcOffBar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *reinterpret_cast<uint32_t*>(st + kTcOffBar + 12) = 0;   // phase of the next completion
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *slot;
}

__device__ __forceinline__ void tc_free(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// wait (bounded) for the completion the last commit signals; returns false
// when it did not arrive
__device__ __forceinline__ bool tc_wait(unsigned char* st) {
  const uint32_t bar = smem_addr(st + kTcOffBar);
  uint32_t* ph = reinterpret_cast<uint32_t*>(st + kTcOffBar + 12);
  const uint32_t phase = *ph;
  uint32_t done = 0;
  for (int it = 0; it < kTcSpinLimit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return done != 0;
}

// Split eight FP32 values into BF16 hi = bf16(x) and lo = bf16(x - hi) and
// store each part as one 16-byte row of a core matrix (element q at byte 2q)
__device__ __forceinline__ void tc_split_store8(unsigned char* hi, unsigned char* lo, uint32_t off, const float v[8]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]), h1 = __float2bfloat16_rn(v[2 * q + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
    h[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// C = A B (split BF16, FP32 accumulation); A(i, k) = A[i sai + k sak],
// B(k, j) = B[k sbk + j sbj]; epi(C, sci, scj, i, j, value) for every
// element.  st: the CTA's staging area (kTcBytes, 1024-aligned), tmem: its
// accumulator; *err gets kErr bits when a completion wait gives up.
template <typename Epi>
__device__ void cta_gemm_tc(int M, int Nn, int K, const float* A, int sai, int sak, const float* B, int sbk, int sbj,
                            float* C, int sci, int scj, Epi epi, unsigned char* st, uint32_t tmem, int* err,
                            int err_bit) {
  const int nthr = (int)blockDim.x, tid = (int)threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  unsigned char* ahi = st;
  unsigned char* alo = st + kTcOffAlo;
  unsigned char* bhi = st + kTcOffBhi;
  unsigned char* blo = st + kTcOffBlo;
  uint32_t* phase = reinterpret_cast<uint32_t*>(st + kTcOffBar + 12);
  for (int m0 = 0; m0 < M; m0 += kTcM) {
    for (int n0 = 0; n0 < Nn; n0 += kTcN) {
      int nt = Nn - n0 < kTcN ? Nn - n0 : kTcN;
      nt = (nt + 15) & ~15;                                      // the MMA's N: a multiple of 16
      const uint32_t idesc = tc_idesc(nt);
      bool ok = true;
      for (int k0 = 0; k0 < K; k0 += kTcK) {
        // 16-deep MMA steps holding data, and the depth staged for them
        const int ks = (K - k0) < kTcK ? ((K - k0) + 15) / 16 : kTcK / 16;
        const int kw = 16 * ks;
        // split the A slice (128 x kw) and the B slice (kw x nt, stored as
        // its transpose, nt x kw) into the hi / lo tiles (zero outside the
        // operands).  One item is one 16-byte row of a core matrix: eight
        // depths 8 kg .. 8 kg + 7 of one row r of A or one column n of B;
        // consecutive threads take consecutive rows / columns, the operands'
        // unit-stride index in the wrap (a row-major A is read as two 16-byte
        // vectors per item instead)
        const int kgs = kw >> 3;
        const bool a_vec = sak == 1 && (sai & 3) == 0 && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
        for (int it = tid; it < kTcM * kgs; it += nthr) {
          const int r = it & (kTcM - 1), kg = it >> 7;
          const int i = m0 + r, kb = k0 + 8 * kg;
          float v[8];
          if (a_vec && i < M && kb + 8 <= K) {
            const float4 x0 = *reinterpret_cast<const float4*>(A + (long)i * sai + kb);
            const float4 x1 = *reinterpret_cast<const float4*>(A + (long)i * sai + kb + 4);
            v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
            v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              v[q] = (i < M && kb + q < K) ? A[(long)i * sai + (long)(kb + q) * sak] : 0.0f;
          }
          tc_split_store8(ahi, alo, tc_off(r, 8 * kg), v);
        }
        // item -> (kg, n) = divmod(it, nt) by a multiply-high: it < 2^13 and
        // nt <= kTcN < 2^8, so ceil(2^32 / nt) gives the exact quotient
        const uint32_t mg = (uint32_t)((0x100000000ull + (uint64_t)nt - 1) / (uint64_t)nt);
        for (int it = tid; it < nt * kgs; it += nthr) {
          const int kg = (int)__umulhi((uint32_t)it, mg), n = it - kg * nt;
          const int j = n0 + n, kb = k0 + 8 * kg;
          float v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            v[q] = (j < Nn && kb + q < K) ? B[(long)(kb + q) * sbk + (long)j * sbj] : 0.0f;
          tc_split_store8(bhi, blo, tc_off(n, 8 * kg), v);
        }
        // the tiles written by the threads (generic proxy) are read by the
        // tensor cores (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
          for (int s = 0; s < ks; ++s) {
            const uint32_t step = (uint32_t)s * 2 * kTcLBO;                   // two core matrices per step
            const uint64_t dah = tc_desc(smem_addr(ahi) + step), dal = tc_desc(smem_addr(alo) + step);
            const uint64_t dbh = tc_desc(smem_addr(bhi) + step), dbl = tc_desc(smem_addr(blo) + step);
            tc_mma(tmem, dah, dbh, idesc, (k0 > 0 || s > 0) ? 1u : 0u);
            tc_mma(tmem, dah, dbl, idesc, 1u);
            tc_mma(tmem, dal, dbh, idesc, 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_addr(st + kTcOffBar))
                       : "memory");
        }
        // every thread waits for the products, which also frees the tiles;
        // the outcome is made the same for the whole CTA
        ok = __syncthreads_and(tc_wait(st) ? 1 : 0) != 0;
        if (tid == 0) *phase ^= 1u;
        __syncthreads();
        if (!ok) break;
      }
      if (!ok) {
        if (tid == 0) atomicOr(err, err_bit);
        return;
      }
      // epilogue, 32 columns at a time: warp w reads TMEM lanes 32 (w mod 4)
      // .. +31 (rows of the tile) and 8 columns (w / 4 mod 4) of the chunk
      // into a row-major chunk in shared memory (the A tile is free once
      // the products are done); then the CTA hands the chunk to the
      // epilogue row by row, consecutive threads on consecutive columns
      float* chunk = reinterpret_cast<float*>(ahi);               // 128 x 32 FP32, rows padded to 33
      const int quarter = warp & 3;
      for (int c0 = 0; c0 < nt; c0 += 32) {
        for (int sub = warp >> 2; sub < 4; sub += nwarps >> 2) {
          if (c0 + 8 * sub < nt) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(c0 + 8 * sub);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 8; ++q) chunk[(32 * quarter + lane) * 33 + 8 * sub + q] = __uint_as_float(v[q]);
          }
        }
        __syncthreads();
        for (int e = tid; e < kTcM * 32; e += nthr) {
          const int r = e >> 5, cc = e & 31;
          const int i = m0 + r, j = n0 + c0 + cc;
          if (i < M && j < Nn && c0 + cc < nt) epi(C, sci, scj, i, j, chunk[r * 33 + cc]);
        }
        __syncthreads();
      }
      // the accumulator is rewritten by the next tile
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }
}

}  // namespace pqmc

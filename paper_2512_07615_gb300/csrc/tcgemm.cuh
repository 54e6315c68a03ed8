// Tensor-core (tcgen05) version of gemm_tile for FP32 storage: the same
// 64 x 64 output tile of one strided GEMM descriptor, computed by tcgen05.mma
// with TF32 operands (kind::tf32) or BF16 operands (kind::f16, both A and B
// BF16) and FP32 accumulation in tensor memory.
//
// Operands are rounded to TF32 or BF16 (nearest) and staged by the CTA's
// threads into shared memory in the K-major, no-swizzle canonical layout:
// core matrices of 8 rows x 16 bytes (4 TF32 or 8 BF16 values per row),
// LBO = 128 B between core matrices along K, SBO = 128 B times the core
// matrices per 8-row group between 8-row groups.  The MMA shape is M = 128,
// N = 64, and 32 bytes of K per instruction (K = 8 TF32 or 16 BF16): one CTA
// computes a 128 x 64 output tile (two of the 64-row tiles of the SIMT grid;
// the CTAs of the grid's odd row tiles have nothing to do and return).  One
// thread issues the instructions of a K chunk and commits them to an mbarrier
// that all threads wait on (with an iteration limit) before the chunk's
// shared memory is refilled.  The 128 x 64 FP32 accumulator (64 TMEM columns,
// 128 lanes) is read back with tcgen05.ld: warp w reads lanes
// 32 (w mod 4) .. + 31 and columns 32 (w / 4) .. + 31.
#pragma once

#include <stdint.h>

#include "gemm.cuh"

namespace tn {

static constexpr int TC_K = 32;            // K per shared-memory chunk (4 MMAs)
static constexpr int TC_COLS = 64;         // TMEM columns per CTA (N = 64 FP32 accumulators)
static constexpr int TC_WAIT = 1 << 22;    // mbarrier polls before giving up

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading / stride byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: D F32 (bits 4-5), A and B format (bits 7-9, 10-12:
// TF32 = 2 under kind::tf32, BF16 = 1 under kind::f16), both K-major, N / 8
// (bits 17-22), M / 16 (bits 24-28).
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n, bool bf16 = false) {
  return (1u << 4) | ((bf16 ? 1u : 2u) << 7) | ((bf16 ? 1u : 2u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// FP32 -> BF16 bits, round to nearest even
__device__ __forceinline__ uint16_t tc_bf16(float x) {
  uint16_t r;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
  return r;
}

// FP32 -> TF32, round to nearest (the MMA itself would drop the low 13 bits,
// a bias toward zero that compounds along chains of contractions).
__device__ __forceinline__ float tc_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < TC_WAIT && !done; ++it)
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
  return done != 0;
}

__device__ __forceinline__ void tc_ld16(uint32_t addr, uint32_t (&r)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                 "=r"(r[15])
               : "r"(addr));
}

// gemm_tile on the tensor cores (blockDim.x == G_THREADS == 256).  A timed-out
// wait sets ST_TIMEOUT in *status and leaves the tile unwritten.
template <bool BF16>
__device__ __forceinline__ void gemm_tile_tc(const GDesc& d, int tile, int ib, int k_begin, int k_end, float* part,
                                             int* status) {
  // the same bytes for either operand type: 128 (A) or 64 (B) rows of TC_K
  // values (TF32: 4 bytes each; BF16: the first half of the buffer)
  __shared__ __align__(1024) float sA[128 * TC_K];
  __shared__ __align__(1024) float sB[64 * TC_K];
  uint16_t* hA = (uint16_t*)sA;
  uint16_t* hB = (uint16_t*)sB;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tn = (d.N + GB_N - 1) / GB_N;
  const int tm_i = tile / tn, tn_i = tile % tn;
  const int m0 = tm_i * 128, n0 = tn_i * GB_N;     // 128-row tiles on the 64-row grid
  if (m0 >= d.M || ib >= d.nb_hi * d.nb_lo) return;       // uniform over the CTA
  const int hi = ib / d.nb_lo, lo = ib % d.nb_lo;
  const float* A = (const float*)d.A + hi * d.a_bh + lo * d.a_bl;
  const float* B = (const float*)d.B + hi * d.b_bh + lo * d.b_bl;
  float* C = (float*)d.C + hi * d.c_bh + lo * d.c_bl;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t mbar = tc_smem(&s_mbar);
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tc_smem(&s_tmem)),
                 "r"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc_idesc(128, 64, BF16);
  constexpr int VPR = BF16 ? 8 : 4;                // values per 16-byte core-matrix row
  const uint32_t sbo = (TC_K / VPR) * 128;
  uint32_t parity = 0;
  bool issued = false;
  for (int k0 = k_begin; k0 < k_end; k0 += TC_K) {
    // A rows 0..127 and B (N x K, K-major) into the core-matrix layout
    for (int e = tid; e < 128 * TC_K; e += blockDim.x) {
      int mm, kk;
      if (d.a_cs == 1) { mm = e / TC_K; kk = e % TC_K; } else { kk = e / 128; mm = e % 128; }
      const int gm = m0 + mm, gk = k0 + kk;
      const float v = (gm < d.M && gk < k_end) ? A[gm * d.a_rs + gk * d.a_cs] : 0.f;
      const int at = ((mm >> 3) * (TC_K / VPR) + kk / VPR) * (8 * VPR) + (mm & 7) * VPR + kk % VPR;
      if constexpr (BF16) hA[at] = tc_bf16(v);
      else sA[at] = tc_tf32(v);
    }
    for (int e = tid; e < 64 * TC_K; e += blockDim.x) {
      int nn, kk;
      if (d.b_cs == 1) { kk = e / 64; nn = e % 64; } else { nn = e / TC_K; kk = e % TC_K; }
      const int gn = n0 + nn, gk = k0 + kk;
      const float v = (gk < k_end && gn < d.N) ? B[gk * d.b_rs + gn * d.b_cs] : 0.f;
      const int at = ((nn >> 3) * (TC_K / VPR) + kk / VPR) * (8 * VPR) + (nn & 7) * VPR + kk % VPR;
      if constexpr (BF16) hB[at] = tc_bf16(v);
      else sB[at] = tc_tf32(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // 32 bytes of K (two core matrices) per instruction
      for (int s = 0; s < TC_K / (2 * VPR); ++s) {
        const uint64_t da = tc_sdesc(tc_smem(sA) + s * 256, 128, sbo);
        const uint64_t db = tc_sdesc(tc_smem(sB) + s * 256, 128, sbo);
        const uint32_t acc = (issued || s > 0) ? 1u : 0u;
        if constexpr (BF16)
          asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                       :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
        else
          asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                       "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                       :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
                   : "memory");
    }
    issued = true;
    if (!tc_wait(mbar, parity)) s_fail = 1;
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_fail) break;
  }
  if (s_fail) {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
  } else {
    // rows 32 (warp & 3) + lane, columns 32 (warp >> 2) .. + 31
    const int row = 32 * (warp & 3) + lane, cbase = 32 * (warp >> 2);
    const int gm = m0 + row;
    for (int h = 0; h < 2; ++h) {
      uint32_t r[16];
      const int c0 = cbase + 16 * h;
      if (issued) {
        tc_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0u;
      }
      if (gm >= d.M) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int gn = n0 + c0 + j;
        if (gn >= d.N) continue;
        const float v = __uint_as_float(r[j]);
        if (part) {
          part[(size_t)gm * d.N + gn] = v;
          continue;
        }
        float* p = C + gm * d.c_rs + gn * d.c_cs;
        float o = (float)d.alpha * v;
        if (d.beta != 0.0) o += (float)d.beta * *p;
        *p = o;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_fail && tid == 0) tc_wait(mbar, parity ^ 1u);      // let the last chunk finish before freeing TMEM
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TC_COLS));
}

}  // namespace tn

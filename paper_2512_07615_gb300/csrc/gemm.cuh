// Strided batched GEMM with device-resident dimensions (SIMT, FP32/FP64).
//
// C[b] = alpha * A[b] B[b] + beta * C[b], each operand addressed by
// (row stride, column stride) and a two-level inner batch ib = hi * nb_lo + lo.
// The descriptor of every (job, stage, site) is computed inside the kernel
// from the MPS bonds in device memory, so launch shapes are fixed by
// capacities and the kernels can sit in a CUDA graph while ranks change.
#pragma once

#include "internal.cuh"

namespace tn {

struct GDesc {
  int M, N, K, nb_hi, nb_lo;
  const void* A;
  const void* B;
  void* C;
  long long a_rs, a_cs, a_bh, a_bl;
  long long b_rs, b_cs, b_bh, b_bl;
  long long c_rs, c_cs, c_bh, c_bl;
  double alpha, beta;
};

static constexpr int GB_M = 64, GB_N = 64, GB_K = 16, G_THREADS = 256;

// One 64x64 output tile of one inner batch of one descriptor, over the
// reduction range [k_begin, k_end).  With part == nullptr the tile is written
// to C as alpha * AB + beta * C; otherwise the raw sum goes to part (dense
// M x N, the split-K partial of this range).
template <typename T>
__device__ __forceinline__ void gemm_tile(const GDesc& d, int tile, int ib, int k_begin, int k_end,
                                          T* part) {
  __shared__ T As[GB_K][GB_M + 4];
  __shared__ T Bs[GB_K][GB_N + 4];
  const int tn = (d.N + GB_N - 1) / GB_N;
  const int tm_i = tile / tn, tn_i = tile % tn;
  const int m0 = tm_i * GB_M, n0 = tn_i * GB_N;
  if (m0 >= d.M || ib >= d.nb_hi * d.nb_lo) return;
  const int hi = ib / d.nb_lo, lo = ib % d.nb_lo;
  const T* A = (const T*)d.A + hi * d.a_bh + lo * d.a_bl;
  const T* B = (const T*)d.B + hi * d.b_bh + lo * d.b_bl;
  T* C = (T*)d.C + hi * d.c_bh + lo * d.c_bl;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  for (int k0 = k_begin; k0 < k_end; k0 += GB_K) {
    // A tile: GB_M x GB_K, stored transposed in As[k][m]
    for (int e = threadIdx.x; e < GB_M * GB_K; e += G_THREADS) {
      int mm, kk;
      if (d.a_cs == 1) { mm = e / GB_K; kk = e % GB_K; } else { kk = e / GB_M; mm = e % GB_M; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < d.M && gk < k_end) ? A[gm * d.a_rs + gk * d.a_cs] : (T)0;
    }
    for (int e = threadIdx.x; e < GB_K * GB_N; e += G_THREADS) {
      int kk, nn;
      if (d.b_cs == 1) { kk = e / GB_N; nn = e % GB_N; } else { nn = e / GB_K; kk = e % GB_K; }
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < k_end && gn < d.N) ? B[gk * d.b_rs + gn * d.b_cs] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= d.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= d.N) continue;
      if (part) {
        part[(size_t)gm * d.N + gn] = acc[i][j];
        continue;
      }
      T* p = C + gm * d.c_rs + gn * d.c_cs;
      T v = (T)d.alpha * acc[i][j];
      if (d.beta != 0.0) v += (T)d.beta * *p;
      *p = v;
    }
  }
}

}  // namespace tn

// Rank model of the learned rounding: an 18 -> 64 -> 64 -> 1 ReLU network that
// maps the spectrum features of a bond (top-16 log10 singular values relative
// to the largest, bond / L, min(step / 1000, 1)) to the retained rank / chi.
// Forward pass, mean-squared-error gradient and Adam training, all on the GPU.
//
// Parameters are one flat FP32 master array W1[64][18], b1[64], W2[64][64],
// b2[64], W3[64], b3.  The forward and backward passes use the parameters
// rounded to FP16 (the copy the rounding kernel evaluates) with FP32
// arithmetic; the updates go to the FP32 master, which is rounded to FP16
// again after every step.
//
// Work split: a CTA takes tiles of 32 samples; per tile the activations live in
// shared memory and the gradient of every parameter is accumulated by the one
// thread that owns it (no atomics).  Per-CTA partial gradients are summed in a
// fixed order by a second kernel, which also applies the Adam step, so that a
// training run is deterministic.
#include <cuda_fp16.h>

#include <cmath>

#include "internal.cuh"

namespace tn {

static constexpr int O_W1 = 0, O_B1 = MLP_H * MLP_IN, O_W2 = O_B1 + MLP_H, O_B2 = O_W2 + MLP_H * MLP_H,
                     O_W3 = O_B2 + MLP_H, O_B3 = O_W3 + MLP_H;
static_assert(O_B3 + 1 == MLP_NPARAM, "parameter layout");
static constexpr int MT = 256;        // threads per CTA
static constexpr int TS = 32;         // samples per tile
static constexpr int HP = MLP_H + 1;  // padded row of an activation tile
static constexpr int MLP_GRID = 152;  // one CTA per SM at most

struct MlpSmem {
  float w[MLP_NPARAM];
  float g[MLP_NPARAM];
  float x[TS][MLP_IN];
  float z1[TS][HP];
  float z2[TS][HP];
  float gz[TS][HP];
  float go[TS];
  float loss[MT / 32];
};

// Samples (start + i) mod M for i < count.  mode 0: gradient partials into
// part[blockIdx.x][0..NPARAM) and the partial sum of squared errors into
// part[..][NPARAM]; mode 1: predictions into out[i].
__global__ void __launch_bounds__(MT) mlp_tile_kernel(const float* __restrict__ P, int M, int start,
                                                       int count, const float* __restrict__ X,
                                                       const float* __restrict__ y, float* __restrict__ part,
                                                       float* __restrict__ out, int mode) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmem& S = *(MlpSmem*)smraw;
  const int tid = threadIdx.x;
  for (int p = tid; p < MLP_NPARAM; p += MT) {
    S.w[p] = __half2float(__float2half_rn(P[p]));
    S.g[p] = 0.f;
  }
  float sq = 0.f;
  const float gscale = 2.f / (float)(count > 0 ? count : 1);
  const int ntiles = (count + TS - 1) / TS;
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int s0 = tile * TS;
    const int ns = imin(TS, count - s0);
    for (int e = tid; e < TS * MLP_IN; e += MT) {
      const int s = e / MLP_IN, i = e % MLP_IN;
      S.x[s][i] = s < ns ? X[(size_t)((start + s0 + s) % M) * MLP_IN + i] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < TS * MLP_H; e += MT) {          // z1 = W1 x + b1
      const int s = e / MLP_H, u = e % MLP_H;
      float a = S.w[O_B1 + u];
#pragma unroll
      for (int i = 0; i < MLP_IN; ++i) a += S.w[O_W1 + u * MLP_IN + i] * S.x[s][i];
      S.z1[s][u] = a;
    }
    __syncthreads();
    for (int e = tid; e < TS * MLP_H; e += MT) {          // z2 = W2 relu(z1) + b2
      const int s = e / MLP_H, u = e % MLP_H;
      float a = S.w[O_B2 + u];
      for (int v = 0; v < MLP_H; ++v) a += S.w[O_W2 + u * MLP_H + v] * fmaxf(S.z1[s][v], 0.f);
      S.z2[s][u] = a;
    }
    __syncthreads();
    {                                                     // out = W3 relu(z2) + b3; one warp per 4 samples
      const int warp = tid >> 5, lane = tid & 31;
      for (int s = warp; s < TS; s += MT / 32) {
        float a = S.w[O_W3 + lane] * fmaxf(S.z2[s][lane], 0.f) +
                  S.w[O_W3 + lane + 32] * fmaxf(S.z2[s][lane + 32], 0.f);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) {
          const float o_ = a + S.w[O_B3];
          if (s < ns) {
            if (mode == 1) out[s0 + s] = o_;
            const float d = (mode == 0) ? o_ - y[(start + s0 + s) % M] : 0.f;
            S.go[s] = gscale * d;
            sq += d * d;
          } else {
            S.go[s] = 0.f;
          }
        }
      }
    }
    __syncthreads();
    if (mode == 0) {
      for (int e = tid; e < TS * MLP_H; e += MT) {        // dL/dz2
        const int s = e / MLP_H, u = e % MLP_H;
        S.gz[s][u] = S.z2[s][u] > 0.f ? S.go[s] * S.w[O_W3 + u] : 0.f;
      }
      for (int u = tid; u < MLP_H; u += MT) {             // W3, b3
        float a = 0.f;
        for (int s = 0; s < TS; ++s) a += S.go[s] * fmaxf(S.z2[s][u], 0.f);
        S.g[O_W3 + u] += a;
      }
      if (tid == 0) {
        float a = 0.f;
        for (int s = 0; s < TS; ++s) a += S.go[s];
        S.g[O_B3] += a;
      }
      __syncthreads();
      for (int e = tid; e < MLP_H * MLP_H; e += MT) {     // W2
        const int u = e / MLP_H, v = e % MLP_H;
        float a = 0.f;
        for (int s = 0; s < TS; ++s) a += S.gz[s][u] * fmaxf(S.z1[s][v], 0.f);
        S.g[O_W2 + e] += a;
      }
      for (int u = tid; u < MLP_H; u += MT) {             // b2
        float a = 0.f;
        for (int s = 0; s < TS; ++s) a += S.gz[s][u];
        S.g[O_B2 + u] += a;
      }
      for (int e = tid; e < TS * MLP_H; e += MT) {        // dL/dz1 into z2 (no longer needed)
        const int s = e / MLP_H, v = e % MLP_H;
        float a = 0.f;
        for (int u = 0; u < MLP_H; ++u) a += S.gz[s][u] * S.w[O_W2 + u * MLP_H + v];
        S.z2[s][v] = S.z1[s][v] > 0.f ? a : 0.f;
      }
      __syncthreads();
      for (int e = tid; e < MLP_H * MLP_IN; e += MT) {    // W1
        const int u = e / MLP_IN, i = e % MLP_IN;
        float a = 0.f;
        for (int s = 0; s < TS; ++s) a += S.z2[s][u] * S.x[s][i];
        S.g[O_W1 + e] += a;
      }
      for (int u = tid; u < MLP_H; u += MT) {             // b1
        float a = 0.f;
        for (int s = 0; s < TS; ++s) a += S.z2[s][u];
        S.g[O_B1 + u] += a;
      }
    }
    __syncthreads();
  }
  if (mode != 0) return;
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((tid & 31) == 0) S.loss[tid >> 5] = sq;
  __syncthreads();
  float* dst = part + (size_t)blockIdx.x * (MLP_NPARAM + 1);
  for (int p = tid; p < MLP_NPARAM; p += MT) dst[p] = S.g[p];
  if (tid == 0) {
    float a = 0.f;
    for (int w = 0; w < MT / 32; ++w) a += S.loss[w];
    dst[MLP_NPARAM] = a;
  }
}

// Sum of the partials in CTA order; then either store gradient and loss, or
// apply one Adam step to the master (bias corrections c1 = 1 - b1^t,
// c2 = 1 - b2^t from the host) and refresh the FP16 copy.
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nparts, int count, float* grad,
                                  float* loss, float* master, float* am, float* av, __half* half_out,
                                  float lr, float b1, float b2, float c1, float c2, float aeps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > MLP_NPARAM) return;
  float a = 0.f;
  for (int c = 0; c < nparts; ++c) a += part[(size_t)c * (MLP_NPARAM + 1) + p];
  if (p == MLP_NPARAM) {
    if (loss) *loss = a / (float)(count > 0 ? count : 1);
    return;
  }
  if (grad) grad[p] = a;
  if (master) {
    const float m = b1 * am[p] + (1.f - b1) * a;
    const float v = b2 * av[p] + (1.f - b2) * a * a;
    am[p] = m;
    av[p] = v;
    const float w = master[p] - lr * (m / c1) / (sqrtf(v / c2) + aeps);
    master[p] = w;
    if (half_out) half_out[p] = __float2half_rn(w);
  }
}

static size_t mlp_smem() { return sizeof(MlpSmem); }

static int mlp_set_smem() {
  static bool done = false;
  if (!done) {
    TN_CUDA(cudaFuncSetAttribute(mlp_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem()));
    done = true;
  }
  return 0;
}

__global__ void learn_tick_kernel(int* step) { *step += 1; }

void launch_learn_tick(int* d_step, cudaStream_t st) { learn_tick_kernel<<<1, 1, 0, st>>>(d_step); }

static int grid_for(int count) { return imax(1, imin(MLP_GRID, (count + TS - 1) / TS)); }

}  // namespace tn

using namespace tn;

extern "C" int tnlbm_mlp_param_count(void) { return MLP_NPARAM; }

extern "C" int tnlbm_mlp_forward(const float* params, int M, const float* X, float* out, void* stream) {
  if (M < 0 || (M > 0 && (!params || !X || !out))) { set_error("bad arguments to tnlbm_mlp_forward"); return TNLBM_E_ARG; }
  if (M == 0) return 0;
  int rc = mlp_set_smem();
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  mlp_tile_kernel<<<grid_for(M), MT, mlp_smem(), st>>>(params, M, 0, M, X, nullptr, nullptr, out, 1);
  TN_CUDA(cudaGetLastError());
  return 0;
}

extern "C" int tnlbm_mlp_loss_grad(const float* params, int M, const float* X, const float* y, float* loss,
                                   float* grad, void* stream) {
  if (M < 1 || !params || !X || !y || !loss || !grad) {
    set_error("bad arguments to tnlbm_mlp_loss_grad");
    return TNLBM_E_ARG;
  }
  int rc = mlp_set_smem();
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int G = grid_for(M);
  float* part = nullptr;
  TN_CUDA(cudaMallocAsync((void**)&part, (size_t)G * (MLP_NPARAM + 1) * sizeof(float), st));
  mlp_tile_kernel<<<G, MT, mlp_smem(), st>>>(params, M, 0, M, X, y, part, nullptr, 0);
  mlp_reduce_kernel<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, st>>>(part, G, M, grad, loss, nullptr, nullptr,
                                                                  nullptr, nullptr, 0.f, 0.f, 0.f, 1.f, 1.f, 0.f);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, st);
  if (e != cudaSuccess) return cuda_fail(e, "tnlbm_mlp_loss_grad");
  return 0;
}

extern "C" int tnlbm_mlp_train(float* master, float* adam_m, float* adam_v, void* half_out, int M,
                               const float* X, const float* y, int iters, int batch, int step0, float lr,
                               float* loss_hist, void* stream) {
  if (!master || !adam_m || !adam_v || M < 1 || !X || !y || iters < 0 || batch < 1 || step0 < 0 ||
      !(lr > 0.f)) {
    set_error("bad arguments to tnlbm_mlp_train");
    return TNLBM_E_ARG;
  }
  int rc = mlp_set_smem();
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int cnt = imin(batch, M);
  const int G = grid_for(cnt);
  float* part = nullptr;
  TN_CUDA(cudaMallocAsync((void**)&part, (size_t)G * (MLP_NPARAM + 1) * sizeof(float), st));
  const double b1 = 0.9, b2 = 0.999;
  for (int it = 0; it < iters; ++it) {
    const int t = step0 + it + 1;
    const int start = (int)(((long long)it * cnt) % M);
    mlp_tile_kernel<<<G, MT, mlp_smem(), st>>>(master, M, start, cnt, X, y, part, nullptr, 0);
    mlp_reduce_kernel<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, st>>>(
        part, G, cnt, nullptr, loss_hist ? loss_hist + it : nullptr, master, adam_m, adam_v, (__half*)half_out,
        lr, (float)b1, (float)b2, (float)(1.0 - std::pow(b1, t)), (float)(1.0 - std::pow(b2, t)), 1e-8f);
  }
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, st);
  if (e != cudaSuccess) return cuda_fail(e, "tnlbm_mlp_train");
  return 0;
}

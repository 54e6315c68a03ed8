// Compressed elementwise product by the single-site variational fit, Sec. 2.3.
//
// A ~ B . C with candidate A = B.  A is right-orthogonalised (centre at site 0),
// right environments are built, then `sweeps` round trips c = 0 -> L-1 -> 0.
// At each centre the optimal core is the contraction
//   A_c[a,s,a'] = sum EL_c[a,g,b] B_c[b,s,b'] C_c[g,s,g'] ER_{c+1}[a',g',b']
// (the local minimiser of ||A - B.C||^2 when A is in mixed canonical form),
// done as three GEMM stages; the centre moves on by QR (rightwards) or LQ
// (leftwards) and the environment of the vacated bond is updated from the
// intermediate of the local contraction.  Environments are stored [a][g][b].
//
// All stages are batched over independent fit jobs; dimensions are read from
// the bond arrays on the device.
#include <algorithm>

#include "fit.cuh"
#include "gemm.cuh"
#include "tcgemm.cuh"
#include "linalg.cuh"

namespace tn {

enum Stage : int { S1 = 0, S2, S3, ENVR, T1, T2, T3, ENVL };
static constexpr int SPLITK_MAX = 16;     // split-K partials of S3 / T3 held in the X buffer

// Bonds of A, B, C at bond k: from the device arrays (rank) or capacities (bound).
struct RankSrc {
  const FitJob* j;
  bool bound;
  int L;
  __host__ __device__ int a(int k) const { return bound ? bond_cap(L, j->A.cap, k) : j->A.ranks[k]; }
  __host__ __device__ int b(int k) const { return bound ? bond_cap(L, j->B.cap, k) : j->B.ranks[k]; }
  __host__ __device__ int g(int k) const { return bound ? bond_cap(L, j->C.cap, k) : j->C.ranks[k]; }
};

template <typename T>
__host__ __device__ inline GDesc make_desc(int stage, const FitJob& J, int c, const RankSrc& R) {
  GDesc d{};
  const int L = R.L;
  const int a = R.a(c), a1 = R.a(c + 1), b = R.b(c), b1 = R.b(c + 1), g = R.g(c), g1 = R.g(c + 1);
  const T* Bc = (const T*)J.B.base + core_offset(L, J.B.cap, c);
  const T* Cc = (const T*)J.C.base + core_offset(L, J.C.cap, c);
  T* Ac = (T*)J.A.base + core_offset(L, J.A.cap, c);
  const T* EL = (const T*)J.env_l + (size_t)c * J.env_stride;
  T* ELn = (T*)J.env_l + (size_t)(c + 1) * J.env_stride;
  const T* ERn = (const T*)J.env_r + (size_t)(c + 1) * J.env_stride;
  T* ER = (T*)J.env_r + (size_t)c * J.env_stride;
  T* X = (T*)J.x;
  T* Y = (T*)J.y;
  T* Ab = (T*)J.abuf;
  d.alpha = 1.0;
  d.beta = 0.0;
  d.nb_hi = 1;
  d.nb_lo = 1;
  switch (stage) {
    case S1:  // X[a][g][s][b1] = EL_c[(a g)][b] * B_c[b][(s b1)]
      d.M = a * g; d.N = 2 * b1; d.K = b;
      d.A = EL; d.a_rs = b; d.a_cs = 1;
      d.B = Bc; d.b_rs = 2 * b1; d.b_cs = 1;
      d.C = X; d.c_rs = 2 * b1; d.c_cs = 1;
      break;
    case S2:  // Y[a][s][g1][b1] = C_s^T (g1 x g) * X[a][.][s][.] (g x b1)
      d.M = g1; d.N = b1; d.K = g; d.nb_hi = a; d.nb_lo = 2;
      d.A = Cc; d.a_rs = 1; d.a_cs = 2 * g1; d.a_bh = 0; d.a_bl = g1;
      d.B = X; d.b_rs = 2 * b1; d.b_cs = 1; d.b_bh = (long long)2 * g * b1; d.b_bl = b1;
      d.C = Y; d.c_rs = b1; d.c_cs = 1; d.c_bh = (long long)2 * g1 * b1; d.c_bl = (long long)g1 * b1;
      break;
    case S3:  // Anew[(a s)][a1] = Y[(a s)][(g1 b1)] * ER_{c+1}[a1][(g1 b1)]^T
      d.M = 2 * a; d.N = a1; d.K = g1 * b1;
      d.A = Y; d.a_rs = (long long)g1 * b1; d.a_cs = 1;
      d.B = ERn; d.b_rs = 1; d.b_cs = (long long)g1 * b1;
      d.C = Ab; d.c_rs = a1; d.c_cs = 1;
      break;
    case ENVR:  // EL_{c+1}[a1][(g1 b1)] = Q^T (a1 x 2a) * Y (2a x g1 b1); Q = A core c
      d.M = a1; d.N = g1 * b1; d.K = 2 * a;
      d.A = Ac; d.a_rs = 1; d.a_cs = a1;
      d.B = Y; d.b_rs = (long long)g1 * b1; d.b_cs = 1;
      d.C = ELn; d.c_rs = (long long)g1 * b1; d.c_cs = 1;
      break;
    case T1:  // X'[b][s][(a1 g1)] = B_c[b][s][b1] * ER_{c+1}[(a1 g1)][b1]^T
      d.M = b; d.N = a1 * g1; d.K = b1; d.nb_lo = 2;
      d.A = Bc; d.a_rs = 2 * b1; d.a_cs = 1; d.a_bl = b1;
      d.B = ERn; d.b_rs = 1; d.b_cs = b1; d.b_bl = 0;
      d.C = X; d.c_rs = (long long)2 * a1 * g1; d.c_cs = 1; d.c_bl = (long long)a1 * g1;
      break;
    case T2:  // Y'[g][b][s][a1] = C_s (g x g1) * X'[b][s][a1][g1]^T
      d.M = g; d.N = a1; d.K = g1; d.nb_hi = b; d.nb_lo = 2;
      d.A = Cc; d.a_rs = 2 * g1; d.a_cs = 1; d.a_bh = 0; d.a_bl = g1;
      d.B = X; d.b_rs = 1; d.b_cs = g1; d.b_bh = (long long)2 * a1 * g1; d.b_bl = (long long)a1 * g1;
      d.C = Y; d.c_rs = (long long)b * 2 * a1; d.c_cs = 1; d.c_bh = 2 * a1; d.c_bl = a1;
      break;
    case T3:  // Anew[a][s][a1] = EL_c[a][(g b)] * Y'[(g b)][s][a1]
      d.M = a; d.N = a1; d.K = g * b; d.nb_lo = 2;
      d.A = EL; d.a_rs = (long long)g * b; d.a_cs = 1; d.a_bl = 0;
      d.B = Y; d.b_rs = 2 * a1; d.b_cs = 1; d.b_bl = a1;
      d.C = Ab; d.c_rs = 2 * a1; d.c_cs = 1; d.c_bl = a1;
      break;
    case ENVL:  // ER_c[a][(g b)] = Qrows (a x 2a1) * Y'[(g b)][(s a1)]^T; Qrows = A core c
      d.M = a; d.N = g * b; d.K = 2 * a1;
      d.A = Ac; d.a_rs = 2 * a1; d.a_cs = 1;
      d.B = Y; d.b_rs = 1; d.b_cs = 2 * a1;
      d.C = ER; d.c_rs = (long long)g * b; d.c_cs = 1;
      break;
  }
  return d;
}

// Split-K count of one job for the long-K stages: from its capacities only,
// so that a job does the same arithmetic in any batch.
__host__ __device__ inline int job_splits(int kcap) {
  return kcap / 256 < 1 ? 1 : (kcap / 256 > SPLITK_MAX ? SPLITK_MAX : kcap / 256);
}

// splits > 1 (split-K, for the long-K stages S3 and T3): blockIdx.y = split *
// nbm + inner batch; each CTA writes the partial product of its K range to the
// job's X buffer (free during S3 and T3), which fit_splitk_reduce sums in
// split order (deterministic).
template <typename T, int STAGE>
__global__ void __launch_bounds__(G_THREADS) fit_gemm_kernel(const FitJob* __restrict__ jobs, int L,
                                                             int c, double* ctr, int splits, int nbm) {
  const FitJob& J = jobs[blockIdx.z];
  RankSrc R{&J, false, L};
  GDesc d = make_desc<T>(STAGE, J, c, R);
  if (ctr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(&ctr[C_FIT_GEMM], 2.0 * d.M * d.N * d.K * d.nb_hi * d.nb_lo);
  if (splits <= 1) {
    gemm_tile<T>(d, blockIdx.x, blockIdx.y, 0, d.K, nullptr);
    return;
  }
  const int split = blockIdx.y / nbm, ib = blockIdx.y % nbm;
  const int nb = d.nb_hi * d.nb_lo;
  RankSrc Rc{&J, true, L};
  const int sj = job_splits(make_desc<T>(STAGE, J, c, Rc).K);
  if (ib >= nb || split >= sj) return;
  splits = sj;
  const int kc = ((d.K + splits - 1) / splits + GB_K - 1) / GB_K * GB_K;
  const int k0 = imin(d.K, split * kc), k1 = imin(d.K, k0 + kc);
  T* part = (T*)J.x + ((size_t)split * nb + ib) * d.M * d.N;
  gemm_tile<T>(d, blockIdx.x, ib, k0, k1, part);
}

// fit_gemm_kernel<float, STAGE> with the tiles on the tensor cores (TF32 or
// BF16 operands, FP32 accumulation; same grid, split-K ranges and outputs).
template <int STAGE, bool BF16>
__global__ void __launch_bounds__(G_THREADS) fit_gemm_tc_kernel(const FitJob* __restrict__ jobs, int L, int c,
                                                                double* ctr, int splits, int nbm, int* status) {
  const FitJob& J = jobs[blockIdx.z];
  RankSrc R{&J, false, L};
  GDesc d = make_desc<float>(STAGE, J, c, R);
  if (ctr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(&ctr[C_FIT_GEMM], 2.0 * d.M * d.N * d.K * d.nb_hi * d.nb_lo);
  if (splits <= 1) {
    gemm_tile_tc<BF16>(d, blockIdx.x, blockIdx.y, 0, d.K, nullptr, status);
    return;
  }
  const int split = blockIdx.y / nbm, ib = blockIdx.y % nbm;
  const int nb = d.nb_hi * d.nb_lo;
  RankSrc Rc{&J, true, L};
  const int sj = job_splits(make_desc<float>(STAGE, J, c, Rc).K);
  if (ib >= nb || split >= sj) return;
  splits = sj;
  const int kc = ((d.K + splits - 1) / splits + GB_K - 1) / GB_K * GB_K;
  const int k0 = imin(d.K, split * kc), k1 = imin(d.K, k0 + kc);
  float* part = (float*)J.x + ((size_t)split * nb + ib) * d.M * d.N;
  gemm_tile_tc<BF16>(d, blockIdx.x, ib, k0, k1, part, status);
}

template <typename T, int STAGE>
__global__ void fit_splitk_reduce(const FitJob* __restrict__ jobs, int L, int c, int splits) {
  const FitJob& J = jobs[blockIdx.y];
  RankSrc R{&J, false, L};
  GDesc d = make_desc<T>(STAGE, J, c, R);
  RankSrc Rc{&J, true, L};
  splits = job_splits(make_desc<T>(STAGE, J, c, Rc).K);
  const int nb = d.nb_hi * d.nb_lo;
  const size_t mn = (size_t)d.M * d.N, total = mn * nb;
  const T* part = (const T*)J.x;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int ib = (int)(e / mn);
    const size_t r = e % mn;
    const int i = (int)(r / d.N), j = (int)(r % d.N);
    T acc = (T)0;
    for (int z = 0; z < splits; ++z) acc += part[((size_t)z * nb + ib) * mn + r];
    const int hi = ib / d.nb_lo, lo = ib % d.nb_lo;
    T* p = (T*)d.C + hi * d.c_bh + lo * d.c_bl + i * d.c_rs + j * d.c_cs;
    T v = (T)d.alpha * acc;
    if (d.beta != 0.0) v += (T)d.beta * *p;
    *p = v;
  }
}

// ---------------------------------------------------------------- per-job CTA kernels
static constexpr int FT = 512;

template <typename T>
__global__ void copy_mps_kernel(const FitJob* __restrict__ jobs, int L) {
  const FitJob& J = jobs[blockIdx.x];
  for (int k = 0; k < L; ++k) {
    const int r0 = J.B.ranks[k], r1 = J.B.ranks[k + 1];
    const T* src = (const T*)J.B.base + core_offset(L, J.B.cap, k);
    T* dst = (T*)J.A.base + core_offset(L, J.A.cap, k);
    for (int i = threadIdx.x; i < r0 * 2 * r1; i += blockDim.x) dst[i] = src[i];
  }
  for (int k = threadIdx.x; k <= L; k += blockDim.x) J.A.ranks[k] = J.B.ranks[k];
}

// environments of the empty left / right parts: EL_0 = ER_L = [1]
template <typename T>
__global__ void env_edges_kernel(const FitJob* __restrict__ jobs, int L) {
  const FitJob& J = jobs[blockIdx.x];
  if (threadIdx.x == 0) {
    ((T*)J.env_l)[0] = (T)1;
    ((T*)J.env_r)[(size_t)L * J.env_stride] = (T)1;
  }
}

// Right-orthogonalise A: LQ at k = L-1..1, A_{k-1} <- A_{k-1} L.
static constexpr int FIT_SMEM = 96 * 1024;   // work matrix of the centre shifts

template <typename T>
__global__ void __launch_bounds__(FT) rortho_kernel(const FitJob* __restrict__ jobs, int L,
                                                    int* status, double* ctr) {
  const FitJob& J = jobs[blockIdx.x];
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ double red[32];
  __shared__ double tau[1024];
  __shared__ T wv[1024];
  T* Qt = (T*)J.qscr + J.qscr_stride;         // 2a1 x a''
  T* Rm = Qt + J.qscr_stride;                 // a'' x a
  T* tmp = Rm + J.qscr_stride;                // 2 a0 x a''
  for (int k = L - 1; k >= 1; --k) {
    const int a = J.A.ranks[k], a1 = J.A.ranks[k + 1], a0 = J.A.ranks[k - 1];
    const int m = 2 * a1, n = a, kk = imin(m, n);
    if (kk > 1024 || n > 1024) { if (threadIdx.x == 0) atomicOr(status, ST_CAPACITY); return; }
    const int ldw = ((size_t)m * (n | 1) * sizeof(T) <= (size_t)FIT_SMEM) ? (n | 1) : n;
    T* work = ((size_t)m * ldw * sizeof(T) <= (size_t)FIT_SMEM) ? (T*)fsm : (T*)J.qscr;
    T* Ak = (T*)J.A.base + core_offset(L, J.A.cap, k);
    T* Ap = (T*)J.A.base + core_offset(L, J.A.cap, k - 1);
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
      const int i = idx / n, c = idx % n;      // work[i][c] = Ak[c][i]
      work[(size_t)i * ldw + c] = Ak[(size_t)c * m + i];
    }
    __syncthreads();
    householder_qr_blk<T>(work, m, n, ldw, Qt, kk, Rm, n, tau, wv, red, (T*)J.x, (T*)J.x + (size_t)m * QB);
    if (ctr && threadIdx.x == 0) atomicAdd(&ctr[C_FIT_QR], qr_flops(m, n) + 2.0 * 2 * a0 * a * kk);
    // A_k <- Qt^T (kk x m) ; A_{k-1} <- A_{k-1} (2a0 x a) * Rm^T (a x kk)
    for (int idx = threadIdx.x; idx < kk * m; idx += blockDim.x) {
      const int i = idx / m, c = idx % m;
      Ak[idx] = Qt[(size_t)c * kk + i];
    }
    for (int idx = threadIdx.x; idx < 2 * a0 * kk; idx += blockDim.x) {
      const int i = idx / kk, c = idx % kk;
      T acc = (T)0;
      for (int p = 0; p < a; ++p) acc += Ap[(size_t)i * a + p] * Rm[(size_t)c * n + p];
      tmp[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * a0 * kk; idx += blockDim.x) Ap[idx] = tmp[idx];
    if (threadIdx.x == 0) J.A.ranks[k] = kk;
    __syncthreads();
  }
}

// Centre shift after a local update.  mode 0: QR of Abuf (2a x a1) -> A core c,
// bond c+1 <- a''.  mode 1: LQ of Abuf (a x 2a1) -> A core c, bond c <- a''.
// mode 2: copy Abuf into A core c (end of a half-sweep).
template <typename T>
__global__ void __launch_bounds__(FT) shift_centre_kernel(const FitJob* __restrict__ jobs, int L,
                                                          int c, int mode, int* status,
                                                          double* ctr) {
  const FitJob& J = jobs[blockIdx.x];
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ double red[32];
  __shared__ double tau[1024];
  __shared__ T wv[1024];
  const int a = J.A.ranks[c], a1 = J.A.ranks[c + 1];
  T* Ac = (T*)J.A.base + core_offset(L, J.A.cap, c);
  const T* Ab = (const T*)J.abuf;
  T* Qt = (T*)J.qscr + J.qscr_stride;
  T* Rm = Qt + J.qscr_stride;
  if (mode == 2) {
    for (int i = threadIdx.x; i < a * 2 * a1; i += blockDim.x) Ac[i] = Ab[i];
    return;
  }
  const int m = mode == 0 ? 2 * a : 2 * a1;
  const int n = mode == 0 ? a1 : a;
  const int kk = imin(m, n);
  if (kk > 1024 || n > 1024) { if (threadIdx.x == 0) atomicOr(status, ST_CAPACITY); return; }
  const int ldw = ((size_t)m * (n | 1) * sizeof(T) <= (size_t)FIT_SMEM) ? (n | 1) : n;
  T* work = ((size_t)m * ldw * sizeof(T) <= (size_t)FIT_SMEM) ? (T*)fsm : (T*)J.qscr;
  for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
    const int i = idx / n, col = idx % n;
    work[(size_t)i * ldw + col] = mode == 0 ? Ab[idx] : Ab[(size_t)col * m + i];
  }
  __syncthreads();
  // blocked QR; its panel scratch is the X buffer (free between the local update and
  // the environment update)
  householder_qr_blk<T>(work, m, n, ldw, Qt, kk, Rm, n, tau, wv, red, (T*)J.x, (T*)J.x + (size_t)m * QB);
  if (ctr && threadIdx.x == 0) atomicAdd(&ctr[C_FIT_QR], qr_flops(m, n));
  if (mode == 0) {
    for (int idx = threadIdx.x; idx < m * kk; idx += blockDim.x) Ac[idx] = Qt[idx];
    if (threadIdx.x == 0) J.A.ranks[c + 1] = kk;
  } else {
    for (int idx = threadIdx.x; idx < kk * m; idx += blockDim.x) {
      const int i = idx / m, col = idx % m;
      Ac[idx] = Qt[(size_t)col * kk + i];
    }
    if (threadIdx.x == 0) J.A.ranks[c] = kk;
  }
}

template <typename T>
static void set_fit_smem() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(rortho_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, FIT_SMEM);
    cudaFuncSetAttribute(shift_centre_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, FIT_SMEM);
    done = true;
  }
}

// ---------------------------------------------------------------- host driver
template <typename T, int STAGE>
static int launch_stage(const FitJob* d_jobs, const std::vector<FitJob>& hj, int L, int c,
                        cudaStream_t st, Prof* prof, int tc, int* d_status) {
  int tiles = 1, nb = 1, kmax = 1;
  size_t elems = 1;
  for (const FitJob& j : hj) {
    RankSrc R{&j, true, L};
    GDesc d = make_desc<T>(STAGE, j, c, R);
    int t = ((d.M + GB_M - 1) / GB_M) * ((d.N + GB_N - 1) / GB_N);
    tiles = std::max(tiles, t);
    nb = std::max(nb, d.nb_hi * d.nb_lo);
    kmax = std::max(kmax, d.K);
    elems = std::max(elems, (size_t)d.M * d.N * d.nb_hi * d.nb_lo);
  }
  // split-K for the stages whose output tiles alone leave SMs idle (S3, T3:
  // K = g b); the grid holds the largest per-job split count
  int splits = 1;
  if (STAGE == S3 || STAGE == T3) splits = job_splits(kmax);
  dim3 grid(tiles, nb * splits, (unsigned)hj.size());
  bool launched = false;
  if constexpr (sizeof(T) == 4) {
    if (tc == TC_TF32) {
      fit_gemm_tc_kernel<STAGE, false><<<grid, G_THREADS, 0, st>>>(d_jobs, L, c, prof ? prof->d_ctr : nullptr,
                                                                   splits, nb, d_status);
      launched = true;
    } else if (tc == TC_BF16) {
      fit_gemm_tc_kernel<STAGE, true><<<grid, G_THREADS, 0, st>>>(d_jobs, L, c, prof ? prof->d_ctr : nullptr,
                                                                  splits, nb, d_status);
      launched = true;
    }
  }
  if (!launched)
    fit_gemm_kernel<T, STAGE><<<grid, G_THREADS, 0, st>>>(d_jobs, L, c, prof ? prof->d_ctr : nullptr, splits, nb);
  if (splits > 1) {
    const unsigned rb = (unsigned)std::min<size_t>(64, (elems + 255) / 256);
    fit_splitk_reduce<T, STAGE><<<dim3(rb, (unsigned)hj.size()), 256, 0, st>>>(d_jobs, L, c, splits);
  }
  if (prof) prof->mark(C_FIT_GEMM);
  return splits > 1 ? 2 : 1;
}

template <typename T>
int run_fit(const FitJob* d_jobs, const std::vector<FitJob>& hj, int L, int sweeps,
            int* d_status, cudaStream_t st, Prof* prof, int tc) {
  const int nj = (int)hj.size();
  if (nj == 0) return 0;
  double* ctr = prof ? prof->d_ctr : nullptr;
  auto mark = [&](int c) { if (prof) prof->mark(c); };
  set_fit_smem<T>();
  int launches = 0;
  copy_mps_kernel<T><<<nj, 128, 0, st>>>(d_jobs, L); ++launches; mark(C_FIT_MISC);
  rortho_kernel<T><<<nj, FT, FIT_SMEM, st>>>(d_jobs, L, d_status, ctr); ++launches; mark(C_FIT_QR);
  env_edges_kernel<T><<<nj, 32, 0, st>>>(d_jobs, L); ++launches; mark(C_FIT_MISC);
  for (int c = L - 1; c >= 1; --c) {
    launches += launch_stage<T, T1>(d_jobs, hj, L, c, st, prof, tc, d_status);
    launches += launch_stage<T, T2>(d_jobs, hj, L, c, st, prof, tc, d_status);
    launches += launch_stage<T, ENVL>(d_jobs, hj, L, c, st, prof, tc, d_status);
  }
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int c = 0; c < L; ++c) {
      launches += launch_stage<T, S1>(d_jobs, hj, L, c, st, prof, tc, d_status);
      launches += launch_stage<T, S2>(d_jobs, hj, L, c, st, prof, tc, d_status);
      launches += launch_stage<T, S3>(d_jobs, hj, L, c, st, prof, tc, d_status);
      if (c < L - 1) {
        shift_centre_kernel<T><<<nj, FT, FIT_SMEM, st>>>(d_jobs, L, c, 0, d_status, ctr); mark(C_FIT_QR);
        launches += launch_stage<T, ENVR>(d_jobs, hj, L, c, st, prof, tc, d_status);
        launches += 1;
      } else {
        shift_centre_kernel<T><<<nj, FT, FIT_SMEM, st>>>(d_jobs, L, c, 2, d_status, ctr); mark(C_FIT_MISC);
        launches += 1;
      }
    }
    for (int c = L - 1; c >= 0; --c) {
      launches += launch_stage<T, T1>(d_jobs, hj, L, c, st, prof, tc, d_status);
      launches += launch_stage<T, T2>(d_jobs, hj, L, c, st, prof, tc, d_status);
      launches += launch_stage<T, T3>(d_jobs, hj, L, c, st, prof, tc, d_status);
      if (c > 0) {
        shift_centre_kernel<T><<<nj, FT, FIT_SMEM, st>>>(d_jobs, L, c, 1, d_status, ctr); mark(C_FIT_QR);
        launches += launch_stage<T, ENVL>(d_jobs, hj, L, c, st, prof, tc, d_status);
        launches += 1;
      } else {
        shift_centre_kernel<T><<<nj, FT, FIT_SMEM, st>>>(d_jobs, L, c, 2, d_status, ctr); mark(C_FIT_MISC);
        launches += 1;
      }
    }
  }
  return launches;
}

// Scratch sizes (elements) of one fit job from the capacities.
void plan_fit_job(FitJob& j, int L, size_t* env_elems, size_t* x_elems, size_t* y_elems,
                  size_t* abuf_elems, size_t* q_elems) {
  size_t env = 1, xs = 1, ys = 1, ab = 1, q = 1;
  for (int k = 0; k <= L; ++k) {
    size_t e = (size_t)bond_cap(L, j.A.cap, k) * bond_cap(L, j.B.cap, k) * bond_cap(L, j.C.cap, k);
    env = std::max(env, e);
  }
  for (int c = 0; c < L; ++c) {
    size_t a = bond_cap(L, j.A.cap, c), a1 = bond_cap(L, j.A.cap, c + 1);
    size_t b = bond_cap(L, j.B.cap, c), b1 = bond_cap(L, j.B.cap, c + 1);
    size_t g = bond_cap(L, j.C.cap, c), g1 = bond_cap(L, j.C.cap, c + 1);
    xs = std::max(xs, std::max(a * g * 2 * b1, b * 2 * a1 * g1));
    xs = std::max(xs, (size_t)SPLITK_MAX * 2 * a * a1);     // split-K partials of S3 and T3
    const size_t amax = std::max(a, a1);
    xs = std::max(xs, qr_blk_scratch<float>(2 * (int)amax, (int)amax));   // blocked QR panels
    ys = std::max(ys, std::max(a * 2 * g1 * b1, g * b * 2 * a1));
    ab = std::max(ab, a * 2 * a1);
    q = std::max(q, std::max(a * 2 * a1, std::max(2 * a1 * a, (size_t)2 * a * a)));
    size_t a0 = c > 0 ? bond_cap(L, j.A.cap, c - 1) : 1;
    q = std::max(q, 2 * a0 * a);
  }
  *env_elems = (env + 31) & ~(size_t)31;
  *x_elems = xs;
  *y_elems = ys;
  *abuf_elems = ab;
  *q_elems = (q + 31) & ~(size_t)31;
}

template int run_fit<float>(const FitJob*, const std::vector<FitJob>&, int, int, int*, cudaStream_t, Prof*, int);
template int run_fit<double>(const FitJob*, const std::vector<FitJob>&, int, int, int*, cudaStream_t, Prof*, int);

}  // namespace tn

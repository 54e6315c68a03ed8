// Smaller kernels of the MPS-LBM step and of the library's input/output:
//  - <X, 1>: transfer-vector sweep (Sec. 3.2, mean density rho_0)
//  - rho_0 and the scalar coefficients of the Taylor 1/rho (Sec. 3.2)
//  - contraction of an MPS to a dense [x][y][z] field (Eq. MPS), for outputs
//  - moments and velocity of the contracted populations (Eq. macro, App. A)
//  - TT-SVD of a dense field (Eq. svd-comp), used to compress geometry masks
#include <algorithm>
#include <cmath>
#include <vector>

#include "fit.cuh"
#include "linalg.cuh"

namespace tn {

// ---------------------------------------------------------------- <X, 1>
template <typename T>
__device__ double inner_ones_dev(const MpsRef& X, int L, double* v, double* w) {
  if (threadIdx.x == 0) v[0] = 1.0;
  __syncthreads();
  for (int k = 0; k < L; ++k) {
    const int r0 = X.ranks[k], r1 = X.ranks[k + 1];
    const T* A = (const T*)X.base + core_offset(L, X.cap, k);
    for (int j = threadIdx.x; j < r1; j += blockDim.x) {
      double acc = 0.0;
      for (int i = 0; i < r0; ++i)
        acc += v[i] * ((double)A[((size_t)i * 2) * r1 + j] + (double)A[((size_t)i * 2 + 1) * r1 + j]);
      w[j] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < r1; j += blockDim.x) v[j] = w[j];
    __syncthreads();
  }
  double r = v[0];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void inner_ones_kernel(const MpsRef* refs, int L, double* out) {
  __shared__ double v[1024], w[1024];
  double r = inner_ones_dev<T>(refs[blockIdx.x], L, v, w);
  if (threadIdx.x == 0) out[blockIdx.x] = r;
}

template <typename T>
void launch_inner_ones(const MpsRef* d_refs, int n, int L, double* d_out, cudaStream_t st) {
  inner_ones_kernel<T><<<n, 256, 0, st>>>(d_refs, L, d_out);
}

template <typename T>
__global__ void rho0_kernel(const MpsRef* rho, int L, double n_fluid, double* scal) {
  __shared__ double v[1024], w[1024];
  double s = inner_ones_dev<T>(rho[0], L, v, w);
  if (threadIdx.x == 0) {
    const double r0 = s / n_fluid;
    scal[SC_NEG_RHO0] = -r0;
    scal[SC_INV1] = 1.0 / r0;
    scal[SC_INV2] = -1.0 / (r0 * r0);
    scal[SC_INV3] = 1.0 / (r0 * r0 * r0);
    scal[SC_RHO0] = r0;
    for (int q = 0; q < 18; ++q) scal[SC_UB + q] = r0 * scal[SC_UBRAW + q];
  }
}

template <typename T>
void launch_rho0(const MpsRef* d_rho, int L, double n_fluid, double* d_scal, cudaStream_t st) {
  rho0_kernel<T><<<1, 256, 0, st>>>(d_rho, L, n_fluid, d_scal);
}

// ---------------------------------------------------------------- mass correction
template <typename T>
__global__ void mass_scale_kernel(const MpsRef* refs, int n, const double* mass, const double* mass0) {
  __shared__ double fac;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m += mass[i];
    fac = (m != 0.0 && isfinite(m)) ? mass0[0] / m : 1.0;
  }
  __syncthreads();
  const MpsRef& X = refs[blockIdx.x];
  const int r1 = X.ranks[1];
  T* c0 = (T*)X.base;                        // core 0 is 1 x 2 x r1
  for (int i = threadIdx.x; i < 2 * r1; i += blockDim.x) c0[i] = (T)((double)c0[i] * fac);
}

template <typename T>
void launch_mass_fix(const MpsRef* d_refs, int n, int L, double* d_mass, const double* d_mass0,
                     cudaStream_t st) {
  inner_ones_kernel<T><<<n, 256, 0, st>>>(d_refs, L, d_mass);
  mass_scale_kernel<T><<<n, 64, 0, st>>>(d_refs, n, d_mass, d_mass0);
}

// ---------------------------------------------------------------- copies
template <typename T>
__global__ void copy_kernel(const MpsRef* src, const MpsRef* dst, int L) {
  const MpsRef& S = src[blockIdx.x];
  const MpsRef& D = dst[blockIdx.x];
  for (int k = 0; k < L; ++k) {
    const int r0 = S.ranks[k], r1 = S.ranks[k + 1];
    const T* a = (const T*)S.base + core_offset(L, S.cap, k);
    T* b = (T*)D.base + core_offset(L, D.cap, k);
    for (int i = threadIdx.x; i < r0 * 2 * r1; i += blockDim.x) b[i] = a[i];
  }
  for (int k = threadIdx.x; k <= L; k += blockDim.x) D.ranks[k] = S.ranks[k];
}

template <typename T>
void launch_copy(const MpsRef* d_src, const MpsRef* d_dst, int n, int L, cudaStream_t st) {
  if (n > 0) copy_kernel<T><<<n, 256, 0, st>>>(d_src, d_dst, L);
}

// ---------------------------------------------------------------- dense contraction
// site-ordered linear index of cell (x, y, z): site k (MSB first) holds bit
// (n-1-k/3) of coordinate k%3
__host__ __device__ inline size_t site_index(int x, int y, int z, int n) {
  size_t idx = 0;
  const int c[3] = {x, y, z};
  for (int k = 0; k < 3 * n; ++k) idx = (idx << 1) | (size_t)((c[k % 3] >> (n - 1 - k / 3)) & 1);
  return idx;
}

// Output contractions accumulate in FP64 whatever the storage type: they run
// once per output, not on the hot path, and FP32 products of L cores would
// bias sums over the lattice at the 1e-6 level.
template <typename T>
__global__ void left_rows_kernel(MpsRef X, int L, int h, double* Lm, int ldl) {
  __shared__ double v[1024], w[1024];
  const size_t l = blockIdx.x;
  for (int k = 0; k < h; ++k) {
    const int s = (int)((l >> (h - 1 - k)) & 1);
    const int r0 = X.ranks[k], r1 = X.ranks[k + 1];
    const T* A = (const T*)X.base + core_offset(L, X.cap, k);
    for (int j = threadIdx.x; j < r1; j += blockDim.x) {
      double acc = 0.0;
      if (k == 0) acc = (double)A[(size_t)s * r1 + j];
      else for (int i = 0; i < r0; ++i) acc += v[i] * (double)A[((size_t)i * 2 + s) * r1 + j];
      w[j] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < r1; j += blockDim.x) v[j] = w[j];
    __syncthreads();
  }
  const int rh = X.ranks[h];
  for (int j = threadIdx.x; j < rh; j += blockDim.x) Lm[l * ldl + j] = v[j];
}

template <typename T>
__global__ void right_cols_kernel(MpsRef X, int L, int h, double* Rt, int ldr) {
  __shared__ double v[1024], w[1024];
  const size_t q = blockIdx.x;
  for (int k = L - 1; k >= h; --k) {
    const int s = (int)((q >> (L - 1 - k)) & 1);
    const int r0 = X.ranks[k], r1 = X.ranks[k + 1];
    const T* A = (const T*)X.base + core_offset(L, X.cap, k);
    for (int i = threadIdx.x; i < r0; i += blockDim.x) {
      double acc = 0.0;
      if (k == L - 1) acc = (double)A[(size_t)i * 2 + s];
      else for (int j = 0; j < r1; ++j) acc += (double)A[((size_t)i * 2 + s) * r1 + j] * v[j];
      w[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r0; i += blockDim.x) v[i] = w[i];
    __syncthreads();
  }
  const int rh = X.ranks[h];
  for (int j = threadIdx.x; j < rh; j += blockDim.x) Rt[q * ldr + j] = v[j];
}

template <typename T>
__global__ void join_kernel(MpsRef X, int n, int h, const double* Lm, const double* Rt, int ld, T* out) {
  const int L = 3 * n;
  const size_t N = (size_t)1 << n;
  const size_t total = N * N * N;
  const int rh = X.ranks[h];
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(idx % N), y = (int)((idx / N) % N), x = (int)(idx / (N * N));
    const size_t si = site_index(x, y, z, n);
    const size_t l = si >> (L - h), q = si & (((size_t)1 << (L - h)) - 1);
    const double* a = Lm + l * ld;
    const double* b = Rt + q * ld;
    double acc = 0.0;
    for (int j = 0; j < rh; ++j) acc += a[j] * b[j];
    out[idx] = (T)acc;
  }
}

size_t contract_scratch_bytes(int n_bits, int cap, size_t elem) {
  const int L = 3 * n_bits, h = L / 2;
  const size_t ld = bond_cap(L, cap, h);
  (void)elem;
  return (((size_t)1 << h) + ((size_t)1 << (L - h))) * ld * sizeof(double);
}

template <typename T, typename OutT>
int contract_dense_to(const MpsRef& X, int n_bits, OutT* d_dense, void* d_scratch, size_t scratch_bytes,
                      cudaStream_t st) {
  const int L = 3 * n_bits, h = L / 2;
  const int ld = bond_cap(L, X.cap, h);
  if (contract_scratch_bytes(n_bits, X.cap, sizeof(T)) > scratch_bytes) return TNLBM_E_ARG;
  double* Lm = (double*)d_scratch;
  double* Rt = Lm + ((size_t)1 << h) * ld;
  left_rows_kernel<T><<<(unsigned)(1u << h), 256, 0, st>>>(X, L, h, Lm, ld);
  right_cols_kernel<T><<<(unsigned)(1u << (L - h)), 256, 0, st>>>(X, L, h, Rt, ld);
  join_kernel<OutT><<<152 * 16, 256, 0, st>>>(X, n_bits, h, Lm, Rt, ld, d_dense);
  return 0;
}

template <typename T>
int contract_dense(const MpsRef& X, int n_bits, T* d_dense, void* d_scratch, size_t scratch_bytes,
                   cudaStream_t st) {
  return contract_dense_to<T, T>(X, n_bits, d_dense, d_scratch, scratch_bytes, st);
}

template <typename T>
int contract_dense_f64(const MpsRef& X, int n_bits, double* d_dense, void* d_scratch, size_t scratch_bytes,
                       cudaStream_t st) {
  return contract_dense_to<T, double>(X, n_bits, d_dense, d_scratch, scratch_bytes, st);
}

// ---------------------------------------------------------------- plane contraction
// The plane coordinate[axis] = index of an MPS without the N^3 field: the
// sites of `axis` are fixed to the bits of `index`, the other 2n sites are
// enumerated as in the dense contraction (prefix rows x suffix columns split
// at h = L / 2), FP64 accumulation.  Output out[u * N + v], u and v the two
// remaining coordinates in increasing axis order.
__host__ __device__ inline int plane_free_bits(int L, int axis, int k0, int k1) {
  int c = 0;
  for (int k = k0; k < k1; ++k) c += (k % 3) != axis;
  return c;
}

template <typename T>
__global__ void left_rows_plane_kernel(MpsRef X, int L, int n, int h, int axis, int index, int fp, double* Lm,
                                       int ldl) {
  __shared__ double v[1024], w[1024];
  const size_t l = blockIdx.x;
  int used = 0;
  for (int k = 0; k < h; ++k) {
    int s;
    if (k % 3 == axis) s = (index >> (n - 1 - k / 3)) & 1;
    else { s = (int)((l >> (fp - 1 - used)) & 1); ++used; }
    const int r0 = X.ranks[k], r1 = X.ranks[k + 1];
    const T* A = (const T*)X.base + core_offset(L, X.cap, k);
    for (int j = threadIdx.x; j < r1; j += blockDim.x) {
      double acc = 0.0;
      if (k == 0) acc = (double)A[(size_t)s * r1 + j];
      else for (int i = 0; i < r0; ++i) acc += v[i] * (double)A[((size_t)i * 2 + s) * r1 + j];
      w[j] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < r1; j += blockDim.x) v[j] = w[j];
    __syncthreads();
  }
  const int rh = X.ranks[h];
  for (int j = threadIdx.x; j < rh; j += blockDim.x) Lm[l * ldl + j] = v[j];
}

template <typename T>
__global__ void right_cols_plane_kernel(MpsRef X, int L, int n, int h, int axis, int index, double* Rt, int ldr) {
  __shared__ double v[1024], w[1024];
  const size_t q = blockIdx.x;
  int used = 0;                                    // free sites seen from the right
  for (int k = L - 1; k >= h; --k) {
    int s;
    if (k % 3 == axis) s = (index >> (n - 1 - k / 3)) & 1;
    else { s = (int)((q >> used) & 1); ++used; }
    const int r0 = X.ranks[k], r1 = X.ranks[k + 1];
    const T* A = (const T*)X.base + core_offset(L, X.cap, k);
    for (int i = threadIdx.x; i < r0; i += blockDim.x) {
      double acc = 0.0;
      if (k == L - 1) acc = (double)A[(size_t)i * 2 + s];
      else for (int j = 0; j < r1; ++j) acc += (double)A[((size_t)i * 2 + s) * r1 + j] * v[j];
      w[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r0; i += blockDim.x) v[i] = w[i];
    __syncthreads();
  }
  const int rh = X.ranks[h];
  for (int j = threadIdx.x; j < rh; j += blockDim.x) Rt[q * ldr + j] = v[j];
}

__global__ void join_plane_kernel(const int* ranks, int n, int h, int axis, const double* Lm, const double* Rt,
                                  int ld, double* out) {
  const int L = 3 * n;
  const size_t N = (size_t)1 << n;
  const int rh = ranks[h];
  const int a0 = axis == 0 ? 1 : 0, a1 = axis == 2 ? 1 : 2;   // remaining axes
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N * N;
       idx += (size_t)gridDim.x * blockDim.x) {
    int c[3] = {0, 0, 0};
    c[a0] = (int)(idx / N);
    c[a1] = (int)(idx % N);
    size_t l = 0, q = 0;
    for (int k = 0; k < L; ++k) {
      if (k % 3 == axis) continue;
      const size_t b = (size_t)((c[k % 3] >> (n - 1 - k / 3)) & 1);
      if (k < h) l = (l << 1) | b;
      else q = (q << 1) | b;
    }
    const double* pa = Lm + l * ld;
    const double* pb = Rt + q * ld;
    double acc = 0.0;
    for (int j = 0; j < rh; ++j) acc += pa[j] * pb[j];
    out[idx] = acc;
  }
}

size_t plane_scratch_bytes(int n_bits, int axis, int cap) {
  const int L = 3 * n_bits, h = L / 2;
  const int fp = plane_free_bits(L, axis, 0, h), fs = plane_free_bits(L, axis, h, L);
  return (((size_t)1 << fp) + ((size_t)1 << fs)) * (size_t)bond_cap(L, cap, h) * sizeof(double);
}

template <typename T>
int contract_plane_f64(const MpsRef& X, int n_bits, int axis, int index, double* d_plane, void* d_scratch,
                       size_t scratch_bytes, cudaStream_t st) {
  const int L = 3 * n_bits, h = L / 2;
  const int ld = bond_cap(L, X.cap, h);
  if (plane_scratch_bytes(n_bits, axis, X.cap) > scratch_bytes) return TNLBM_E_ARG;
  const int fp = plane_free_bits(L, axis, 0, h), fs = plane_free_bits(L, axis, h, L);
  double* Lm = (double*)d_scratch;
  double* Rt = Lm + ((size_t)1 << fp) * ld;
  left_rows_plane_kernel<T><<<(unsigned)(1u << fp), 256, 0, st>>>(X, L, n_bits, h, axis, index, fp, Lm, ld);
  right_cols_plane_kernel<T><<<(unsigned)(1u << fs), 256, 0, st>>>(X, L, n_bits, h, axis, index, Rt, ld);
  join_plane_kernel<<<152 * 4, 256, 0, st>>>(X.ranks, n_bits, h, axis, Lm, Rt, ld, d_plane);
  return 0;
}

template <typename T>
__global__ void accum_kernel(const T* f, size_t n, double* rho, double* jx, double* jy, double* jz,
                             int cx, int cy, int cz, int first) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = (double)f[i];
    if (first) { rho[i] = v; jx[i] = cx * v; jy[i] = cy * v; jz[i] = cz * v; }
    else { rho[i] += v; jx[i] += cx * v; jy[i] += cy * v; jz[i] += cz * v; }
  }
}

template <typename T>
void launch_accum_moments(const T* d_f, size_t ncell, double* rho, double* jx, double* jy, double* jz,
                          int cx, int cy, int cz, int first, cudaStream_t st) {
  accum_kernel<T><<<152 * 8, 256, 0, st>>>(d_f, ncell, rho, jx, jy, jz, cx, cy, cz, first);
}

__global__ void velocity_kernel(size_t n, const double* rho, double* jx, double* jy, double* jz,
                                const double* mask, double fx, double fy, double fz) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double m = mask ? mask[i] : 0.0;
    const double r = rho[i];
    if (r > 0.5) {
      jx[i] = (jx[i] + 0.5 * fx * (1.0 - m)) / r;
      jy[i] = (jy[i] + 0.5 * fy * (1.0 - m)) / r;
      jz[i] = (jz[i] + 0.5 * fz * (1.0 - m)) / r;
    } else {
      jx[i] = 0.0; jy[i] = 0.0; jz[i] = 0.0;
    }
  }
}

void launch_velocity(size_t ncell, const double* rho, double* jx, double* jy, double* jz,
                     const double* mask, double fx, double fy, double fz, cudaStream_t st) {
  velocity_kernel<<<152 * 8, 256, 0, st>>>(ncell, rho, jx, jy, jz, mask, fx, fy, fz);
}

// ---------------------------------------------------------------- TT-SVD
template <typename T>
__global__ void to_site_order_kernel(const T* dense, int n, double* out) {
  const size_t N = (size_t)1 << n, total = N * N * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(idx % N), y = (int)((idx / N) % N), x = (int)(idx / (N * N));
    out[site_index(x, y, z, n)] = (double)dense[idx];
  }
}

// Partial Gram matrices, deterministic: block p accumulates M[:, chunk] M[:, chunk]^T
// (upper triangle) over the column chunks p, p + P, p + 2P, ... into its own
// slice part[p] (every entry owned by one thread); gram_reduce_kernel sums the
// slices in block order.
__global__ void gram_part_kernel(const double* M, int m, size_t ncols, int kc, int P, double* part) {
  extern __shared__ double tile[];           // m x kc
  double* G = part + (size_t)blockIdx.x * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) G[e] = 0.0;
  const size_t nch = (ncols + kc - 1) / kc;
  for (size_t ch = blockIdx.x; ch < nch; ch += P) {
    const size_t c0 = ch * kc;
    const int w = (int)((ncols - c0) < (size_t)kc ? (ncols - c0) : (size_t)kc);
    __syncthreads();
    for (int e = threadIdx.x; e < m * kc; e += blockDim.x) {
      const int i = e / kc, c = e % kc;
      tile[e] = c < w ? M[(size_t)i * ncols + c0 + c] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e % m;
      if (j < i) continue;
      double acc = 0.0;
      for (int c = 0; c < w; ++c) acc += tile[i * kc + c] * tile[j * kc + c];
      G[e] += acc;
    }
  }
}

__global__ void gram_reduce_kernel(const double* part, int P, size_t mm, double* G) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < mm; e += (size_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int p = 0; p < P; ++p) a += part[(size_t)p * mm + e];
    G[e] = a;
  }
}

// eigen-decomposition of the symmetric PSD Gram G (m x m) by one-sided Jacobi;
// truncation; writes U (m x r, FP64) and the rank.
__global__ void __launch_bounds__(1024) gram_eig_kernel(double* G, int m, double* Wm, double* Vm,
                                                        double* U, int chi, double delta2,
                                                        int ncols_cap, int* r_out, int* status) {
  __shared__ double lam[1024];
  __shared__ int perm[1024];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    const double v = (j >= i) ? G[(size_t)i * m + j] : G[(size_t)j * m + i];
    Wm[(size_t)j * m + i] = v;   // column j
  }
  __syncthreads();
  int sw = jacobi_cols<double>(Wm, Vm, m, m, 80);
  if (sw >= 80 && threadIdx.x == 0) atomicOr(status, ST_NOCONV);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < m; ++i) a += Wm[(size_t)j * m + i] * Wm[(size_t)j * m + i];
    const double lj = sqrt(a);                // eigenvalue of G = sigma^2 of M
    if (!(lj >= 0.0) || isinf(lj)) { lam[j] = -1.0; atomicOr(status, ST_NAN); }   // orders last
    else lam[j] = lj;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int rank = 0;
    for (int o = 0; o < m; ++o) rank += (lam[o] > lam[j]) || (lam[o] == lam[j] && o < j);
    perm[rank] = j;
  }
  __syncthreads();
  __shared__ int s_r;
  if (threadIdx.x == 0) {
    const int rmax = imin(chi, imin(m, ncols_cap));
    int r = rmax;
    // eigenvalues of the Gram matrix below its round-off level carry no
    // information: treat that level as the smallest resolvable tail
    const double floor2 = 64.0 * 2.220446049250313e-16 * (double)m * lam[perm[0]];
    const double thr = delta2 > floor2 ? delta2 : floor2;
    for (int rr = 1; rr <= rmax; ++rr) {
      double tail = 0.0;
      for (int p = rr; p < m; ++p) tail += lam[perm[p]];
      if (tail <= thr) { r = rr; break; }
    }
    s_r = r;
    *r_out = r;
  }
  __syncthreads();
  const int r = s_r;
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    U[e] = Vm[(size_t)perm[j] * m + i];
  }
}

// Mn (r x ncols) = U^T (r x m) M (m x ncols)
__global__ void project_kernel(const double* U, int m, int r, const double* M, size_t ncols, double* Mn) {
  const size_t total = (size_t)r * ncols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / ncols);
    const size_t c = e % ncols;
    double acc = 0.0;
    for (int i = 0; i < m; ++i) acc += U[(size_t)i * r + p] * M[(size_t)i * ncols + c];
    Mn[e] = acc;
  }
}

template <typename T>
__global__ void cast_double_kernel(const T* src, size_t n, double* dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

template <typename T>
void launch_cast_double(const T* src, size_t n, double* dst, cudaStream_t st) {
  cast_double_kernel<T><<<152 * 8, 256, 0, st>>>(src, n, dst);
}

template <typename T>
__global__ void cast_store_kernel(const double* src, size_t n, T* dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

// per-block partial sums of squares (summed in block order by the host)
__global__ void norm2_part_kernel(const double* x, size_t n, double* part) {
  __shared__ double red[32];
  double a = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a += x[i] * x[i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

template <typename T>
int tt_svd_dense(const T* d_dense, int n, T* d_dst, int* d_dst_ranks, int dst_cap, int chi_max,
                 double eps, int* d_status, cudaStream_t st) {
  const int L = 3 * n;
  const size_t total = (size_t)1 << L;
  const int mmax = 2 * imin(chi_max, dst_cap);
  if (mmax > 1024) return TNLBM_E_ARG;
  double *M = nullptr, *M2 = nullptr, *G = nullptr, *Wm = nullptr, *Vm = nullptr, *U = nullptr, *nrm = nullptr;
  double* gpart = nullptr;
  int* d_r = nullptr;
  // partial Gram slices: as many as fit in 256 MB at the largest m (at most 304)
  const int NB_NORM = 152 * 4;
  int Pg = (int)std::min<size_t>(304, std::max<size_t>(1, ((size_t)256 << 20) / ((size_t)mmax * mmax * sizeof(double))));
  auto cleanup = [&]() {
    cudaFree(M); cudaFree(M2); cudaFree(G); cudaFree(Wm); cudaFree(Vm); cudaFree(U); cudaFree(nrm); cudaFree(d_r);
    cudaFree(gpart);
  };
  if (cudaMalloc(&M, total * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&M2, total * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&G, (size_t)mmax * mmax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&Wm, (size_t)mmax * mmax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&Vm, (size_t)mmax * mmax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&U, (size_t)mmax * mmax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&nrm, NB_NORM * sizeof(double)) != cudaSuccess || cudaMalloc(&d_r, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&gpart, (size_t)Pg * mmax * mmax * sizeof(double)) != cudaSuccess) {
    cleanup();
    return TNLBM_E_OOM;
  }
  to_site_order_kernel<T><<<152 * 8, 256, 0, st>>>(d_dense, n, M);
  norm2_part_kernel<<<NB_NORM, 256, 0, st>>>(M, total, nrm);
  std::vector<double> h_part(NB_NORM);
  cudaMemcpyAsync(h_part.data(), nrm, NB_NORM * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  double h_n2 = 0.0;
  for (double v : h_part) h_n2 += v;
  const double delta = eps * sqrt(h_n2) / sqrt((double)(L - 1));
  std::vector<int> ranks(L + 1, 1);
  int r = 1;
  for (int k = 0; k < L - 1; ++k) {
    const int m = 2 * r;
    const size_t ncols = total >> (k + 1);
    int kc = 6144 / m;
    if (kc < 1) kc = 1;
    const size_t nch = (ncols + kc - 1) / kc;
    const int P = (int)std::min<size_t>((size_t)Pg, nch);
    gram_part_kernel<<<P, 256, (size_t)m * kc * sizeof(double), st>>>(M, m, ncols, kc, P, gpart);
    gram_reduce_kernel<<<152, 256, 0, st>>>(gpart, P, (size_t)m * m, G);
    gram_eig_kernel<<<1, 1024, 0, st>>>(G, m, Wm, Vm, U, imin(chi_max, dst_cap), delta * delta,
                                        (int)(ncols < (size_t)1024 ? ncols : (size_t)1024), d_r, d_status);
    int h_r = 0;
    cudaMemcpyAsync(&h_r, d_r, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "tt_svd_dense"); }
    const int rn = h_r;
    if (rn > bond_cap(L, dst_cap, k + 1)) { cleanup(); return TNLBM_E_CAPACITY; }
    // core k = U (r x 2 x rn)
    cast_store_kernel<T><<<64, 256, 0, st>>>(U, (size_t)m * rn, d_dst + core_offset(L, dst_cap, k));
    project_kernel<<<152 * 8, 256, 0, st>>>(U, m, rn, M, ncols, M2);
    double* t = M; M = M2; M2 = t;
    r = rn;
    ranks[k + 1] = rn;
  }
  cast_store_kernel<T><<<64, 256, 0, st>>>(M, (size_t)2 * r, d_dst + core_offset(L, dst_cap, L - 1));
  cudaMemcpyAsync(d_dst_ranks, ranks.data(), (L + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "tt_svd_dense");
  return 0;
}

#define INST(T)                                                                                   \
  template void launch_inner_ones<T>(const MpsRef*, int, int, double*, cudaStream_t);           \
  template int contract_plane_f64<T>(const MpsRef&, int, int, int, double*, void*, size_t, cudaStream_t); \
  template void launch_rho0<T>(const MpsRef*, int, double, double*, cudaStream_t);              \
  template void launch_copy<T>(const MpsRef*, const MpsRef*, int, int, cudaStream_t);           \
  template void launch_mass_fix<T>(const MpsRef*, int, int, double*, const double*, cudaStream_t); \
  template int contract_dense<T>(const MpsRef&, int, T*, void*, size_t, cudaStream_t);          \
  template int contract_dense_f64<T>(const MpsRef&, int, double*, void*, size_t, cudaStream_t);  \
  template void launch_accum_moments<T>(const T*, size_t, double*, double*, double*, double*,   \
                                        int, int, int, int, cudaStream_t);                       \
  template int tt_svd_dense<T>(const T*, int, T*, int*, int, int, double, int*, cudaStream_t); \
  template void launch_cast_double<T>(const T*, size_t, double*, cudaStream_t);
INST(float)
INST(double)

}  // namespace tn

// Compressed element-wise product by the zip-up pass, the alternative to the
// single-site fit that Sec. 2.3 names.  One CTA per product:
//   1. copies of both factors are brought to right-canonical form by LQ
//      sweeps (QR of each transposed core unfolding, R^T moved left);
//   2. one left-to-right pass carries a matrix M[a][c][b] from the product
//      bond (b, c) to the new bond a.  At site k the product core is
//      contracted into it, T[a s][c' b'] = sum_{b,c} M[a][c][b] B_k[b s b']
//      C_k[c s c'], and T is truncated: QR of T^T (R only), one-sided Jacobi
//      on the columns of R (their accumulated rotation V holds the left
//      singular vectors of T), rank by the rounding's tail rule with
//      delta = eps ||T_0|| / sqrt(L-1); U_r is the new core and M = U_r^T T
//      is carried on.  The last site keeps T.
// The pass leaves its result left-orthogonal up to the last core; the step
// rounds it afterwards (a one-term rounding job), which also moves the centre
// to site 0 as every other product and sum of the step.
#include <cuda_runtime.h>

#include "fit.cuh"
#include "internal.cuh"
#include "linalg.cuh"

namespace tn {

static constexpr int ZT = 512;                      // threads per product
static constexpr int ZSM = 176 * 1024;              // Jacobi matrices in shared memory

__device__ inline void zflag(int* st, int code) { atomicOr(st, code); }

// Scratch partition of one zip job (elements of T).
struct ZipLayout {
  size_t bc, cc, m, x, t, r, a, q, p, jw, jv, qs, total;
};

__host__ __device__ inline ZipLayout zip_layout(int L, int cb, int cc, int cz, size_t esz) {
  ZipLayout z{};
  const int cm = imax(cb, cc);
  const size_t prod = (size_t)cc * cb;
  const int jl = (int)((16 / esz) * ((2 * cz + (int)(16 / esz) - 1) / (int)(16 / esz)));
  size_t o = 0;
  auto take = [&](size_t n) { size_t r = o; o += (n + 3) & ~(size_t)3; return r; };   // 16-byte starts (FP32)
  z.bc = take(mps_size(L, cb));
  z.cc = take(mps_size(L, cc));
  z.m = take((size_t)cz * prod);
  z.x = take(2 * (size_t)cz * prod);
  z.t = take(2 * (size_t)cz * prod);
  z.r = take((size_t)imax(2 * cz, cm) * imax(2 * cz, cm));
  z.a = take(2 * (size_t)cm * cm);
  z.q = take(2 * (size_t)cm * cm);
  z.p = take(2 * (size_t)cm * cm);
  z.jw = take((size_t)2 * cz * jl);
  z.jv = take((size_t)2 * cz * jl);
  z.qs = take(qr_blk_scratch<float>((int)(prod > (size_t)(2 * cm) ? prod : (size_t)(2 * cm)), imax(2 * cz, cm)));
  z.total = o;
  return z;
}

size_t zip_scratch_elems(int L, int capB, int capC, int capZ, size_t esz) {
  return zip_layout(L, capB, capC, capZ, esz).total;
}

// Right-canonical form of a flat MPS in place (ranks in shared memory):
// for k = L-1 .. 1 the transposed unfolding (2 r1 x r0) of core k is
// factorised Q R; core k becomes Q^T, core k-1 is multiplied by R^T.
template <typename T>
__device__ void zip_right_orth(T* F, int cap, int L, int* rk, T* At, T* Qb, T* Rb, T* Pb, double* s_tau,
                               T* s_wv, double* s_red, T* vb, T* wb) {
  for (int k = L - 1; k >= 1; --k) {
    const int r0 = rk[k], r1 = rk[k + 1], rp = rk[k - 1];
    const int m = 2 * r1, n = r0, kk = imin(m, n);
    T* core = F + core_offset(L, cap, k);
    T* prev = F + core_offset(L, cap, k - 1);
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
      const int row = idx / n, al = idx % n;
      At[idx] = core[(size_t)al * m + row];
    }
    __syncthreads();
    householder_qr_blk<T>(At, m, n, n, Qb, kk, Rb, n, s_tau, s_wv, s_red, vb, wb);
    for (int idx = threadIdx.x; idx < kk * m; idx += blockDim.x) {
      const int j = idx / m, row = idx % m;
      core[idx] = Qb[(size_t)row * kk + j];
    }
    for (int idx = threadIdx.x; idx < 2 * rp * kk; idx += blockDim.x) {
      const int i = idx / kk, j = idx % kk;
      T acc = (T)0;
      for (int al = 0; al < n; ++al) acc += prev[(size_t)i * n + al] * Rb[(size_t)j * n + al];
      Pb[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * rp * kk; idx += blockDim.x) prev[idx] = Pb[idx];
    if (threadIdx.x == 0) rk[k] = kk;
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(ZT) zipup_kernel(const ZipJob* __restrict__ jobs, int L,
                                                  int* __restrict__ status, double* __restrict__ ctr) {
  const ZipJob& J = jobs[blockIdx.x];
  extern __shared__ __align__(16) unsigned char zsm[];
  __shared__ double s_tau[1024], s_sig[1024];
  __shared__ int s_perm[1024];
  __shared__ T s_wv[1024];
  __shared__ double s_red[64];
  __shared__ int s_rb[TN_MAXL + 1], s_rc[TN_MAXL + 1], s_rz[TN_MAXL + 1];
  __shared__ double s_delta, s_scale;
  __shared__ int s_rank, s_bad;
  __shared__ double s_flops;

  const int cb = J.B.cap, cc = J.C.cap, cz = J.Z.cap;
  const ZipLayout lay = zip_layout(L, cb, cc, cz, sizeof(T));
  T* scr = (T*)J.scratch;
  T* Bc = scr + lay.bc;
  T* Cc = scr + lay.cc;
  T* Mb = scr + lay.m;
  T* Xb = scr + lay.x;
  T* Tb = scr + lay.t;
  T* Rb = scr + lay.r;
  T* vb = scr + lay.qs;
  const int cm = imax(cb, cc);
  const int qm = imax(cc * cb, 2 * cm);
  T* wb = vb + (size_t)qm * QB;

  if (threadIdx.x == 0) { s_bad = 0; s_flops = 0.0; }
  for (int k = threadIdx.x; k <= L; k += blockDim.x) {
    s_rb[k] = J.B.ranks[k];
    s_rc[k] = J.C.ranks[k];
  }
  __syncthreads();
  for (int k = threadIdx.x; k <= L; k += blockDim.x) {
    if (s_rb[k] < 1 || s_rb[k] > bond_cap(L, cb, k) || s_rc[k] < 1 || s_rc[k] > bond_cap(L, cc, k)) s_bad = 1;
  }
  __syncthreads();
  if (s_bad) { if (threadIdx.x == 0) zflag(status, ST_CAPACITY); return; }
  // ---- copies of the factors, right-canonical
  {
    const size_t nb = mps_size(L, cb), nc = mps_size(L, cc);
    const T* B = (const T*)J.B.base;
    const T* C = (const T*)J.C.base;
    for (size_t i = threadIdx.x; i < nb; i += blockDim.x) Bc[i] = B[i];
    for (size_t i = threadIdx.x; i < nc; i += blockDim.x) Cc[i] = C[i];
    __syncthreads();
    T* At = scr + lay.a;
    T* Qb = scr + lay.q;
    T* Pb = scr + lay.p;
    zip_right_orth<T>(Bc, cb, L, s_rb, At, Qb, Rb, Pb, s_tau, s_wv, s_red, vb, wb);
    zip_right_orth<T>(Cc, cc, L, s_rc, At, Qb, Rb, Pb, s_tau, s_wv, s_red, vb, wb);
  }
  // ---- the pass
  T* Z = (T*)J.Z.base;
  if (threadIdx.x == 0) { Mb[0] = (T)1; s_rz[0] = 1; }
  __syncthreads();
  int a = 1;
  for (int k = 0; k < L; ++k) {
    const int b = s_rb[k], c = s_rc[k], y = s_rb[k + 1], z = s_rc[k + 1];
    const T* Bk = Bc + core_offset(L, cb, k);
    const T* Ck = Cc + core_offset(L, cc, k);
    // X[(a c)][(s b')] = sum_b M[(a c)][b] B_k[b][(s b')]
    cta_gemm<T>(a * c, 2 * y, b, Mb, b, Bk, 2 * y, Xb, 2 * y, false);
    __syncthreads();
    // T[(a s)][(c' b')] = sum_c C_k[c][s][c'] X[(a c)][s][b'], 4 x 4 register tiles
    const int tz = (z + 3) >> 2, ty = (y + 3) >> 2, m = z * y;
    for (int t = threadIdx.x; t < 2 * a * tz * ty; t += blockDim.x) {
      const int row = t / (tz * ty), rem = t % (tz * ty);
      const int ai = row >> 1, s = row & 1;
      const int z0 = (rem / ty) * 4, y0 = (rem % ty) * 4;
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
      for (int q = 0; q < c; ++q) {
        T cv[4], xv[4];
        const T* cr = Ck + (size_t)q * 2 * z + (size_t)s * z;
        const T* xr = Xb + ((size_t)ai * c + q) * 2 * y + (size_t)s * y;
#pragma unroll
        for (int i = 0; i < 4; ++i) cv[i] = (z0 + i < z) ? cr[z0 + i] : (T)0;
#pragma unroll
        for (int j = 0; j < 4; ++j) xv[j] = (y0 + j < y) ? xr[y0 + j] : (T)0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += cv[i] * xv[j];
      }
      T* tr = Tb + (size_t)row * m;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (z0 + i < z && y0 + j < y) tr[(size_t)(z0 + i) * y + y0 + j] = acc[i][j];
    }
    __syncthreads();
    const int n = 2 * a;
    if (k == 0) {                                  // delta from the first unfolding's norm
      double part = 0.0;
      for (int i = threadIdx.x; i < n * m; i += blockDim.x) part += (double)Tb[i] * (double)Tb[i];
      const double t2 = block_sum(part, s_red);
      if (threadIdx.x == 0) s_delta = J.eps * sqrt(t2) / sqrt((double)imax(L - 1, 1));
      __syncthreads();
    }
    if (threadIdx.x == 0)
      s_flops += 4.0 * a * c * b * y + 4.0 * a * z * y * c;
    if (k == L - 1) {
      T* zk = Z + core_offset(L, cz, k);
      for (int i = threadIdx.x; i < n; i += blockDim.x) zk[i] = Tb[i];
      if (threadIdx.x == 0) s_rz[L] = 1;
      __syncthreads();
      break;
    }
    // QR of T^T (m x n), R only
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
      const int col = idx / n, row = idx % n;
      Xb[idx] = Tb[(size_t)row * m + col];
    }
    __syncthreads();
    const int kk = imin(m, n);
    householder_qr_blk<T>(Xb, m, n, n, (T*)nullptr, 0, Rb, n, s_tau, s_wv, s_red, vb, wb);
    // Jacobi on the n columns of R (length kk); shared memory if it fits
    const int ldw = jacobi_ld<T>(kk), ldv = jacobi_ld<T>(n);
    const size_t need = ((size_t)n * ldw + (size_t)n * ldv) * sizeof(T);
    T* Wm = need <= (size_t)ZSM ? (T*)zsm : scr + lay.jw;
    T* Vm = need <= (size_t)ZSM ? (T*)zsm + (size_t)n * ldw : scr + lay.jv;
    {
      T amax = (T)0;
      for (int idx = threadIdx.x; idx < kk * n; idx += blockDim.x) amax = fmax(amax, fabs(Rb[idx]));
      for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = (double)amax;
      __syncthreads();
      if (threadIdx.x == 0) {
        double am = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) am = fmax(am, s_red[w]);
        int e = 0;
        if (am > 0.0 && isfinite(am)) frexp(am, &e);
        s_scale = ldexp(1.0, 1 - e);             // max |R| scaled into [1, 2), exactly
      }
      __syncthreads();
    }
    const double scl = s_scale;
    for (int idx = threadIdx.x; idx < n * kk; idx += blockDim.x) {
      const int j = idx / kk, i = idx % kk;
      Wm[(size_t)j * ldw + i] = (T)scl * Rb[(size_t)i * n + j];
    }
    __syncthreads();
    const int sw = jacobi_cols_fast<T>(Wm, ldw, Vm, ldv, n, kk, 60);
    if (sw >= 60 && threadIdx.x == 0) zflag(status, ST_NOCONV);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      T acc = (T)0;
      const T* w = Wm + (size_t)j * ldw;
      for (int i = 0; i < kk; ++i) acc += w[i] * w[i];
      const double sv = (double)sqrt(acc) / scl;
      if (!(sv >= 0.0) || isinf(sv)) { s_sig[j] = -1.0; zflag(status, ST_NAN); }   // orders last
      else s_sig[j] = sv;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      int rank = 0;
      const double sj = s_sig[j];
      for (int o = 0; o < n; ++o) {
        const double so = s_sig[o];
        rank += (so > sj) || (so == sj && o < j);
      }
      s_perm[rank] = j;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // smallest r in [1, min(chi, n)] whose discarded tail is <= delta
      const int rmax = imin(J.chi, n);
      double tail2 = 0.0;
      for (int p = n - 1; p >= 1; --p) {
        const double sv = s_sig[s_perm[p]];
        tail2 += sv * sv;
        s_tau[p] = tail2;
      }
      int rr = rmax;
      for (int q = 1; q <= rmax; ++q) {
        const double t2 = q < n ? s_tau[q] : 0.0;
        if (sqrt(t2) <= s_delta) { rr = q; break; }
      }
      if (rr > bond_cap(L, cz, k + 1)) { s_bad = 1; rr = bond_cap(L, cz, k + 1); }
      s_rank = rr;
      s_flops += 2.0 * m * (double)n * n + svd_flops(kk, n) + 2.0 * rr * (double)n * m;
    }
    __syncthreads();
    if (s_bad) { if (threadIdx.x == 0) zflag(status, ST_CAPACITY); return; }
    const int r = s_rank;
    // core k = U_r (a, 2, r); U_r^T into Rb (r x n) for the carry
    T* zk = Z + core_offset(L, cz, k);
    for (int idx = threadIdx.x; idx < n * r; idx += blockDim.x) {
      const int row = idx / r, j = idx % r;
      zk[idx] = Vm[(size_t)s_perm[j] * ldv + row];
    }
    for (int idx = threadIdx.x; idx < r * n; idx += blockDim.x) {
      const int j = idx / n, row = idx % n;
      Rb[idx] = Vm[(size_t)s_perm[j] * ldv + row];
    }
    __syncthreads();
    // M[j][(c' b')] = sum_i U_r[i][j] T[i][(c' b')]
    cta_gemm<T>(r, m, n, Rb, n, Tb, m, Mb, m, false);
    if (threadIdx.x == 0) s_rz[k + 1] = r;
    a = r;
    __syncthreads();
  }
  for (int k = threadIdx.x; k <= L; k += blockDim.x) J.Z.ranks[k] = s_rz[k];
  if (ctr && threadIdx.x == 0) atomicAdd(&ctr[C_ZIPUP], s_flops);
}

template <typename T>
int run_zipup(const ZipJob* d_jobs, int njobs, int L, int* d_status, cudaStream_t st, double* d_ctr) {
  if (njobs <= 0) return 0;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(zipup_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, ZSM);
    attr_set = true;
  }
  zipup_kernel<T><<<njobs, ZT, ZSM, st>>>(d_jobs, L, d_status, d_ctr);
  return 1;
}

template int run_zipup<float>(const ZipJob*, int, int, int*, cudaStream_t, double*);
template int run_zipup<double>(const ZipJob*, int, int, int*, cudaStream_t, double*);

}  // namespace tn

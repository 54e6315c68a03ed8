// In-CTA dense linear algebra used by the rounding sweep and the product fit:
// block reductions, Householder QR with an explicit Q, and a one-sided
// (Hestenes) Jacobi SVD.  Matrices are row-major with a leading dimension and
// may live in shared or global memory (generic pointers).  Every function is
// called by all threads of the block and ends with __syncthreads().
#pragma once

#include "internal.cuh"

namespace tn {

template <typename T> struct Eps;
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };

// sum over the block in type V; `red` is shared scratch of >= 32 V
template <typename V>
__device__ inline V block_sum_t(V v, V* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  V s = (V)0;
  const int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
    s = lane < nw ? red[lane] : (V)0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// sum over the block; `red` is shared scratch of >= 32 doubles
__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
    s = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// One-sided Jacobi on ncol columns of length len, stored column-contiguous
// (Wm[j*len + i]); V (ncol x ncol, V[j*ncol + i] = column j) accumulates the
// rotations.  Parallel ordering: a round-robin tournament, one warp per pair.
// Returns the number of sweeps used (maxsw + 1 if not converged).
template <typename T>
__device__ int jacobi_cols(T* Wm, T* V, int ncol, int len, int maxsw) {
  for (int idx = threadIdx.x; idx < ncol * ncol; idx += blockDim.x)
    V[idx] = (idx / ncol == idx % ncol) ? (T)1 : (T)0;
  __shared__ int s_rot;
  __syncthreads();
  if (ncol < 2) return 0;
  const int np = (ncol + 1) & ~1;          // padded to even; index np-1 may be a dummy
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // stopping threshold on |cos| of a pair: a few ulps above the round-off of a
  // freshly rotated pair, so short columns cannot cycle on noise
  const double tol = 16.0 * Eps<T>::v * sqrt((double)len);
  int sweep = 0;
  for (; sweep < maxsw; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int p = wid; p < np / 2; p += nw) {
        int a, b;
        if (p == 0) { a = rnd; b = np - 1; }
        else { a = (rnd + p) % (np - 1); b = (rnd - p + (np - 1)) % (np - 1); }
        if (a >= ncol || b >= ncol) continue;
        if (a > b) { int t = a; a = b; b = t; }
        T* wa = Wm + (size_t)a * len;
        T* wb = Wm + (size_t)b * len;
        double al = 0, be = 0, ga = 0;
        for (int i = lane; i < len; i += 32) {
          double x = (double)wa[i], y = (double)wb[i];
          al += x * x; be += y * y; ga += x * y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        // pairs below the representable range carry nothing; skip them too
        if (ga == 0.0 || al < 1e-250 || be < 1e-250 || fabs(ga) <= tol * sqrt(al) * sqrt(be)) continue;
        // Rutishauser's rotation zeroing the (a, b) inner product
        double zeta = (be - al) / (2.0 * ga);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        const T cc = (T)c, ss = (T)s;
        for (int i = lane; i < len; i += 32) {
          T x = wa[i], y = wb[i];
          wa[i] = cc * x - ss * y;
          wb[i] = ss * x + cc * y;
        }
        T* va = V + (size_t)a * ncol;
        T* vb = V + (size_t)b * ncol;
        for (int i = lane; i < ncol; i += 32) {
          T x = va[i], y = vb[i];
          va[i] = cc * x - ss * y;
          vb[i] = ss * x + cc * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

}  // namespace tn

namespace tn {

// ---------------------------------------------------------------- fast in-CTA kernels
// Designed for 1024-thread CTAs with the working matrix in shared memory.

// C (M x N, ldc) = [C +] A (M x K, lda) * B (K x N, ldb); each thread owns 4x4
// output tiles in a strided loop; operands may be in global or shared memory.
template <typename T>
__device__ void cta_gemm(int M, int N, int K, const T* A, int lda, const T* B, int ldb, T* C,
                         int ldc, bool accumulate) {
  const int tm = (M + 3) >> 2, tnn = (N + 3) >> 2;
  for (int t = threadIdx.x; t < tm * tnn; t += blockDim.x) {
    const int i0 = (t / tnn) * 4, j0 = (t % tnn) * 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int k = 0; k < K; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = (i0 + a < M) ? A[(size_t)(i0 + a) * lda + k] : (T)0;
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = (j0 + b < N) ? B[(size_t)k * ldb + j0 + b] : (T)0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (i0 + a >= M) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (j0 + b >= N) continue;
        T* p = C + (size_t)(i0 + a) * ldc + j0 + b;
        *p = accumulate ? *p + acc[a][b] : acc[a][b];
      }
    }
  }
  __syncthreads();
}

// Householder QR of A (m x n, lda; typically shared memory, lda = n + 1 to
// avoid bank conflicts), with Q (m x k, ldq) and R (k x n, ldr) written out,
// diag(R) >= 0.  Parallel form: per column, the reflector inner products are
// split over row groups (8 threads per column) and the rank-1 update runs over
// all elements.  tau/wv: shared scratch of >= n doubles / T.
template <typename T>
__device__ void householder_qr_par(T* A, int m, int n, int lda, T* Q, int ldq, T* R, int ldr,
                                   double* tau, T* wv, double* red) {
  // All arithmetic in T: on GB300 FP64 runs at ~1/64 of the FP32 rate.
  // Per column: one reduction for the norm (fused into the previous update),
  // one pass for the reflector inner products (the reflector is kept unscaled
  // and its scale folded in), one pass for the rank-1 update that also stores
  // the scaled reflector.  Three barriers per column.
  const int kk = imin(m, n);
  const int G = 8;                                 // threads per column in the dot phase
  __shared__ T s_scale, s_norm2;
  T* redT = (T*)red;
  // norm of column 0 below the diagonal
  {
    T part = (T)0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) {
      const T v = A[(size_t)i * lda];
      part += v * v;
    }
    const T t = block_sum_t<T>(part, redT);
    if (threadIdx.x == 0) s_norm2 = t;
  }
  for (int j = 0; j < kk; ++j) {
    if (threadIdx.x == 0) {
      const T sig2 = s_norm2;
      const T alpha = A[(size_t)j * lda + j];
      if (sig2 == (T)0) {
        tau[j] = 0.0;
        s_scale = (T)0;
      } else {
        const T beta = -copysign(sqrt(alpha * alpha + sig2), alpha);
        tau[j] = (double)((beta - alpha) / beta);
        s_scale = (T)1 / (alpha - beta);
        A[(size_t)j * lda + j] = beta;
      }
    }
    __syncthreads();
    const T tj = (T)tau[j];
    const T sc = s_scale;
    const int nc = n - j - 1;
    if (tj != (T)0) {
      // w_c = (A[j][c] + sc * sum_{i>j} A[i][j] A[i][c]) * tau, c > j
      for (int base = 0; base < nc * G; base += blockDim.x) {
        const int t = base + threadIdx.x;
        const bool act = t < nc * G;
        const int c = j + 1 + t / G, p = t % G;
        T acc = (T)0;
        if (act)
          for (int i = j + 1 + p; i < m; i += G) acc += A[(size_t)i * lda + j] * A[(size_t)i * lda + c];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
        if (act && p == 0) wv[c] = (A[(size_t)j * lda + c] + sc * acc) * tj;
      }
      __syncthreads();
    }
    // A[i][c] -= w_c v_i with v_i = sc A[i][j] (v_j = 1); store v; norm of column j+1
    const int rows = m - j;
    T part = (T)0;
    if (tj != (T)0) {
      for (int t = threadIdx.x; t < rows * nc; t += blockDim.x) {
        const int ii = j + t / nc, c = j + 1 + t % nc;
        const T vi = (ii == j) ? (T)1 : sc * A[(size_t)ii * lda + j];
        const T nv = A[(size_t)ii * lda + c] - wv[c] * vi;
        A[(size_t)ii * lda + c] = nv;
        if (c == j + 1 && ii > j + 1) part += nv * nv;
      }
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[(size_t)i * lda + j] *= sc;
    } else if (nc > 0) {
      for (int i = j + 2 + threadIdx.x; i < m; i += blockDim.x) {
        const T v = A[(size_t)i * lda + j + 1];
        part += v * v;
      }
    }
    if (j + 1 < kk) {
      const T t = block_sum_t<T>(part, redT);
      if (threadIdx.x == 0) s_norm2 = t;
    } else {
      __syncthreads();
    }
  }
  // R with non-negative diagonal; remember the signs for Q
  __shared__ signed char s_dneg[1024];
  for (int idx = threadIdx.x; idx < kk * n; idx += blockDim.x) {
    const int i = idx / n, c = idx % n;
    const bool neg = A[(size_t)i * lda + i] < (T)0;
    R[(size_t)i * ldr + c] = c >= i ? (neg ? -A[(size_t)i * lda + c] : A[(size_t)i * lda + c]) : (T)0;
    if (c == i) s_dneg[i] = neg ? 1 : 0;
  }
  __syncthreads();
  // Q = H_0 ... H_{kk-1} [I; 0] formed in place of the reflectors, backwards
  // (column j of A holds reflector j until step j turns it into column j of Q;
  // columns > j already hold Q, rows < j of them are zero)
  for (int j = kk - 1; j >= 0; --j) {
    const T tj = (T)tau[j];
    const int nc = kk - j - 1;                      // Q columns j+1..kk-1
    if (tj != (T)0 && nc > 0) {
      for (int base = 0; base < nc * G; base += blockDim.x) {
        const int t = base + threadIdx.x;
        const bool act = t < nc * G;
        const int c = j + 1 + t / G, p = t % G;
        T acc = (T)0;
        if (act) {
          if (p == 0) acc = A[(size_t)j * lda + c];
          for (int i = j + 1 + p; i < m; i += G) acc += A[(size_t)i * lda + j] * A[(size_t)i * lda + c];
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
        if (act && p == 0) wv[c] = acc * tj;
      }
      __syncthreads();
      const int rows = m - j;
      for (int t = threadIdx.x; t < rows * nc; t += blockDim.x) {
        const int ii = j + t / nc, c = j + 1 + t % nc;
        const T vi = (ii == j) ? (T)1 : A[(size_t)ii * lda + j];
        A[(size_t)ii * lda + c] -= wv[c] * vi;
      }
      __syncthreads();
    }
    // column j of Q: H_j e_j = e_j - tau_j v, zero above the diagonal
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      T q;
      if (i < j) q = (T)0;
      else if (i == j) q = (T)1 - tj;
      else q = -tj * A[(size_t)i * lda + j];
      A[(size_t)i * lda + j] = q;
    }
    __syncthreads();
  }
  // Q out, with the column signs that make diag(R) >= 0
  for (int idx = threadIdx.x; idx < m * kk; idx += blockDim.x) {
    const int i = idx / kk, c = idx % kk;
    const T q = A[(size_t)i * lda + c];
    Q[(size_t)i * ldq + c] = s_dneg[c] ? -q : q;
  }
  __syncthreads();
}

// One-sided Jacobi as jacobi_cols, with a half-warp per column pair so that a
// 1024-thread CTA keeps 64 pairs in flight.  Columns have stride ldw >= len.
template <typename T>
__device__ int jacobi_cols_hw(T* Wm, int ldw, T* V, int ldv, int ncol, int len, int maxsw) {
  for (int idx = threadIdx.x; idx < ncol * ncol; idx += blockDim.x)
    V[(size_t)(idx / ncol) * ldv + idx % ncol] = (idx / ncol == idx % ncol) ? (T)1 : (T)0;
  __shared__ int s_rot;
  __syncthreads();
  if (ncol < 2) return 0;
  const int np = (ncol + 1) & ~1;
  const int hl = threadIdx.x & 15, hw = threadIdx.x >> 4, nhw = blockDim.x >> 4;
  const unsigned mask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  const T tolT = (T)(16.0 * Eps<T>::v * sqrt((double)len));
  int sweep = 0;
  for (; sweep < maxsw; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int p = hw; p < np / 2; p += nhw) {
        int a, b;
        if (p == 0) { a = rnd; b = np - 1; }
        else { a = (rnd + p) % (np - 1); b = (rnd - p + (np - 1)) % (np - 1); }
        const bool live = a < ncol && b < ncol;
        if (a > b) { int t = a; a = b; b = t; }
        T al = (T)0, be = (T)0, ga = (T)0;
        T* wa = Wm + (size_t)a * ldw;
        T* wb = Wm + (size_t)b * ldw;
        if (live)
          for (int i = hl; i < len; i += 16) {
            const T x = wa[i], y = wb[i];
            al += x * x; be += y * y; ga += x * y;
          }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(mask, al, o, 16);
          be += __shfl_xor_sync(mask, be, o, 16);
          ga += __shfl_xor_sync(mask, ga, o, 16);
        }
        // columns below the type's representable range (after the caller's
        // power-of-two scaling to max |entry| ~ 1) carry nothing
        // (FP32: below 1e-24 the rotation parameter zeta could overflow)
        const T floor2 = sizeof(T) == 8 ? (T)1e-250 : (T)1e-24;
        if (!live || ga == (T)0 || al < floor2 || be < floor2 || fabs(ga) <= tolT * sqrt(al) * sqrt(be))
          continue;
        // Rutishauser's rotation zeroing the (a, b) inner product
        const T zeta = (be - al) / ((T)2 * ga);
        const T t = (zeta >= (T)0 ? (T)1 : (T)-1) / (fabs(zeta) + hypot((T)1, zeta));
        const T cc = (T)1 / sqrt((T)1 + t * t), ss = cc * t;
        for (int i = hl; i < len; i += 16) {
          const T x = wa[i], y = wb[i];
          wa[i] = cc * x - ss * y;
          wb[i] = ss * x + cc * y;
        }
        T* va = V + (size_t)a * ldv;
        T* vb = V + (size_t)b * ldv;
        for (int i = hl; i < ncol; i += 16) {
          const T x = va[i], y = vb[i];
          va[i] = cc * x - ss * y;
          vb[i] = ss * x + cc * y;
        }
        if (hl == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

// 16-byte vector of T
template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 t; static constexpr int n = 4; };
template <> struct Vec16<double> { typedef double2 t; static constexpr int n = 2; };

template <typename T> __device__ __forceinline__ void v_dot3(const typename Vec16<T>::t& x, const typename Vec16<T>::t& y,
                                                            T& al, T& be, T& ga);
template <> __device__ __forceinline__ void v_dot3<float>(const float4& x, const float4& y, float& al, float& be, float& ga) {
  al += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
  be += y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
  ga += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
}
template <> __device__ __forceinline__ void v_dot3<double>(const double2& x, const double2& y, double& al, double& be,
                                                           double& ga) {
  al += x.x * x.x + x.y * x.y;
  be += y.x * y.x + y.y * y.y;
  ga += x.x * y.x + x.y * y.y;
}
template <typename T> __device__ __forceinline__ void v_rot(typename Vec16<T>::t& x, typename Vec16<T>::t& y, T c, T s);
template <> __device__ __forceinline__ void v_rot<float>(float4& x, float4& y, float c, float s) {
  const float4 a = x, b = y;
  x = make_float4(c * a.x - s * b.x, c * a.y - s * b.y, c * a.z - s * b.z, c * a.w - s * b.w);
  y = make_float4(s * a.x + c * b.x, s * a.y + c * b.y, s * a.z + c * b.z, s * a.w + c * b.w);
}
template <> __device__ __forceinline__ void v_rot<double>(double2& x, double2& y, double c, double s) {
  const double2 a = x, b = y;
  x = make_double2(c * a.x - s * b.x, c * a.y - s * b.y);
  y = make_double2(s * a.x + c * b.x, s * a.y + c * b.y);
}

// Row stride of a Jacobi matrix for jacobi_cols_fast (16-byte multiple).
template <typename T>
__host__ __device__ inline int jacobi_ld(int n) {
  constexpr int VW = 16 / (int)sizeof(T);
  return (n + VW - 1) / VW * VW;
}

// FP32 one-sided Jacobi with a half-warp per column pair (64 pairs in flight
// in a 1024-thread CTA, as jacobi_cols_hw) and 16-byte vector accesses:
// each lane holds NV float4 of each of its two columns in registers, so a
// pair costs one read and one write of each column.  Same pair order,
// convergence test and rotation as jacobi_cols_hw.  Requires ldw, ldv multiples of 4 and
// 16-byte aligned Wm, V; len <= 64 * NV.
template <int NV>
__device__ __noinline__ int jacobi_cols_h4(float* Wm, int ldw, float* V, int ldv, int ncol, int len, int maxsw) {
  const int lenv = (len + 3) / 4, ncv = (ncol + 3) / 4;
  const int padw = lenv * 4 - len;
  for (int idx = threadIdx.x; idx < ncol * padw; idx += blockDim.x)
    Wm[(size_t)(idx / padw) * ldw + len + idx % padw] = 0.f;
  for (int idx = threadIdx.x; idx < ncol * ncv * 4; idx += blockDim.x) {
    const int r = idx / (ncv * 4), c = idx % (ncv * 4);
    V[(size_t)r * ldv + c] = (r == c) ? 1.f : 0.f;
  }
  __shared__ int s_rot;
  __syncthreads();
  if (ncol < 2) return 0;
  const int np = (ncol + 1) & ~1, nr = np - 1;
  const int hl = threadIdx.x & 15, hw = threadIdx.x >> 4, nhw = blockDim.x >> 4;
  const unsigned mask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  const float tolT = (float)(16.0 * Eps<float>::v * sqrt((double)len));
  int sweep = 0;
  for (; sweep < maxsw; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < nr; ++rnd) {
      for (int p = hw; p < np / 2; p += nhw) {
        int a, b;
        if (p == 0) { a = rnd; b = nr; }
        else {
          a = rnd + p; if (a >= nr) a -= nr;
          b = rnd - p; if (b < 0) b += nr;
        }
        if (a > b) { int t = a; a = b; b = t; }
        const bool live = b < ncol;
        float4* pa = (float4*)(Wm + (size_t)a * ldw);
        float4* pb = (float4*)(Wm + (size_t)b * ldw);
        float4 xa[NV], xb[NV];
        float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int i = hl + 16 * v;
          if (live && i < lenv) {
            xa[v] = pa[i];
            xb[v] = pb[i];
            v_dot3<float>(xa[v], xb[v], al, be, ga);
          }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(mask, al, o, 16);
          be += __shfl_xor_sync(mask, be, o, 16);
          ga += __shfl_xor_sync(mask, ga, o, 16);
        }
        if (!live || ga == 0.f || al < 1e-24f || be < 1e-24f || fabsf(ga) <= tolT * sqrtf(al) * sqrtf(be))
          continue;
        // Rutishauser's rotation (correctly rounded division and square root:
        // c^2 + s^2 = 1 to the last bit keeps the accumulated V orthogonal)
        const float zeta = (be - al) / (2.f * ga);
        const float az = fabsf(zeta);
        const float h = az > 1e18f ? az : sqrtf(1.f + zeta * zeta);
        const float t = copysignf(1.f / (az + h), zeta);
        const float cc = 1.f / sqrtf(1.f + t * t), ss = cc * t;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int i = hl + 16 * v;
          if (i < lenv) {
            v_rot<float>(xa[v], xb[v], cc, ss);
            pa[i] = xa[v];
            pb[i] = xb[v];
          }
        }
        float4* va = (float4*)(V + (size_t)a * ldv);
        float4* vb = (float4*)(V + (size_t)b * ldv);
        for (int i = hl; i < ncv; i += 16) {
          float4 x = va[i], y = vb[i];
          v_rot<float>(x, y, cc, ss);
          va[i] = x;
          vb[i] = y;
        }
        if (hl == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

// The fastest in-CTA Jacobi for the type and column length (use jacobi_ld
// for the strides): FP32 columns of up to 256 entries take jacobi_cols_h4,
// everything else jacobi_cols_hw.
template <typename T>
__device__ __forceinline__ int jacobi_cols_fast(T* Wm, int ldw, T* V, int ldv, int ncol, int len, int maxsw) {
  if constexpr (sizeof(T) == 4) {
    if (len <= 128) return jacobi_cols_h4<2>(Wm, ldw, V, ldv, ncol, len, maxsw);
    if (len <= 256) return jacobi_cols_h4<4>(Wm, ldw, V, ldv, ncol, len, maxsw);
  }
  return jacobi_cols_hw<T>(Wm, ldw, V, ldv, ncol, len, maxsw);
}

}  // namespace tn

namespace tn {

// C (M x N, ldc) = A^T B with A given as K x M (lda) and B as K x N (ldb).
template <typename T>
__device__ void cta_gemm_tn(int M, int N, int K, const T* A, int lda, const T* B, int ldb, T* C, int ldc) {
  const int tm = (M + 3) >> 2, tnn = (N + 3) >> 2;
  for (int t = threadIdx.x; t < tm * tnn; t += blockDim.x) {
    const int i0 = (t / tnn) * 4, j0 = (t % tnn) * 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int k = 0; k < K; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = (i0 + a < M) ? A[(size_t)k * lda + i0 + a] : (T)0;
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = (j0 + b < N) ? B[(size_t)k * ldb + j0 + b] : (T)0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (i0 + a >= M) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (j0 + b < N) C[(size_t)(i0 + a) * ldc + j0 + b] = acc[a][b];
    }
  }
  __syncthreads();
}

// Rank-predicting MLP (18 -> 64 -> 64 -> 1, ReLU, FP16 parameters) evaluated
// by the block; returns the predicted rank clamped to [1, chi].  `buf` is
// shared scratch of >= 146 floats.  Parameter layout: W1[64][18], b1[64],
// W2[64][64], b2[64], W3[64], b3.
__device__ inline int mlp_predict_rank(const __half* P, const float* spec, float bondf, float stepf,
                                       int chi, float* buf) {
  float* x = buf;
  float* h1 = buf + 18;
  float* h2 = buf + 18 + 64;
  if (threadIdx.x < 16) x[threadIdx.x] = spec[threadIdx.x];
  if (threadIdx.x == 16) x[16] = bondf;
  if (threadIdx.x == 17) x[17] = stepf;
  __syncthreads();
  const __half* W1 = P;
  const __half* b1 = W1 + 64 * 18;
  const __half* W2 = b1 + 64;
  const __half* b2 = W2 + 64 * 64;
  const __half* W3 = b2 + 64;
  const __half* b3 = W3 + 64;
  if (threadIdx.x < 64) {
    float a = __half2float(b1[threadIdx.x]);
    for (int i = 0; i < 18; ++i) a += __half2float(W1[threadIdx.x * 18 + i]) * x[i];
    h1[threadIdx.x] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  if (threadIdx.x < 64) {
    float a = __half2float(b2[threadIdx.x]);
    for (int i = 0; i < 64; ++i) a += __half2float(W2[threadIdx.x * 64 + i]) * h1[i];
    h2[threadIdx.x] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  __shared__ int s_pred;
  if (threadIdx.x < 32) {
    float a = __half2float(W3[threadIdx.x]) * h2[threadIdx.x] + __half2float(W3[threadIdx.x + 32]) * h2[threadIdx.x + 32];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (threadIdx.x == 0) {
      const float y = a + __half2float(b3[0]);
      int k = isfinite(y) ? (int)lrintf(fminf(fmaxf(y, 0.f), 2.f) * (float)chi) : chi;
      s_pred = k < 1 ? 1 : (k > chi ? chi : k);
    }
  }
  __syncthreads();
  return s_pred;
}

}  // namespace tn

namespace tn {

// ---------------------------------------------------------------- blocked Householder QR
// Same factorisation and outputs as householder_qr_par (reflectors, diag(R) >=
// 0, explicit Q), organised in panels of QB columns (compact WY form,
// H_p0 ... H_pe-1 = I - V T V^T): the reflectors of a panel are computed column
// by column on the panel only, and the rest of the matrix is updated once per
// panel by two small matrix products instead of once per column.  Q is formed
// backwards panel by panel in place of the reflectors.
static constexpr int QB = 16;            // panel width
static constexpr int QNG = 4;            // row groups of the V^T X products

// Scratch (global or shared): vb >= m * QB, wb >= (QNG + 1) * QB * n elements.
template <typename T>
__host__ __device__ inline size_t qr_blk_scratch(int m, int n) {
  return (size_t)m * QB + (size_t)(QNG + 1) * QB * n;
}

// V (mr x QB, ld QB) of the panel [p0, pe): unit diagonal, zeros above it,
// the stored reflectors below; columns >= pe - p0 are zero.
template <typename T>
__device__ void qr_blk_load_v(const T* A, int lda, int m, int p0, int pe, T* vb) {
  const int mr = m - p0, pb = pe - p0;
  for (int idx = threadIdx.x; idx < mr * QB; idx += blockDim.x) {
    const int r = idx / QB, q = idx % QB;
    T v;
    if (q >= pb || r < q) v = (T)0;
    else if (r == q) v = (T)1;
    else v = A[(size_t)(p0 + r) * lda + p0 + q];
    vb[idx] = v;
  }
  __syncthreads();
}

// T (pb x pb, upper) of the compact WY form from the Gram matrix of V:
// T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] (V^T V)[0:j, j].
template <typename T>
__device__ void qr_blk_make_t(const T* vb, int mr, int pb, const double* tau, T (*sT)[QB + 1], T (*sG)[QB + 1]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int pr = warp; pr < pb * pb; pr += nw) {
    const int q1 = pr / pb, q2 = pr % pb;
    if (q2 < q1) continue;
    T acc = (T)0;
    for (int r = q2 + lane; r < mr; r += 32) acc += vb[(size_t)r * QB + q1] * vb[(size_t)r * QB + q2];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sG[q1][q2] = acc;
  }
  __syncthreads();
  if (warp == 0) {
    for (int j = 0; j < pb; ++j) {
      const T tj = (T)tau[j];
      T z = (T)0;
      if (lane < j)
        for (int k = lane; k < j; ++k) z += sT[lane][k] * sG[k][j];
      __syncwarp();
      if (lane < j) sT[lane][j] = -tj * z;
      if (lane == j) sT[j][j] = tj;
      if (lane > j && lane < QB) sT[lane][j] = (T)0;
      __syncwarp();
    }
  }
  __syncthreads();
}

// W (pb x nx, ld nx) = V^T X, X = mr x nx (ld ldx): 4x4 register tiles, the
// rows split over QNG groups whose partials are summed in group order.
template <typename T>
__device__ void qr_blk_vtx(const T* vb, int mr, int pb, const T* X, int ldx, int nx, T* wpart, T* W) {
  const int tq = (pb + 3) >> 2, tc = (nx + 3) >> 2, ntile = tq * tc;
  const int rc = (mr + QNG - 1) / QNG;
  for (int it = threadIdx.x; it < ntile * QNG; it += blockDim.x) {
    const int g = it / ntile, t = it % ntile;
    const int q0 = (t / tc) * 4, c0 = (t % tc) * 4;
    const int r0 = g * rc, r1 = imin(mr, r0 + rc);
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int r = r0; r < r1; ++r) {
      T v[4], x[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) v[a] = vb[(size_t)r * QB + q0 + a];     // q0 + 3 < QB
#pragma unroll
      for (int b = 0; b < 4; ++b) x[b] = (c0 + b < nx) ? X[(size_t)r * ldx + c0 + b] : (T)0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += v[a] * x[b];
    }
    T* wp = wpart + (size_t)g * QB * nx;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (q0 + a >= pb) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (c0 + b < nx) wp[(size_t)(q0 + a) * nx + c0 + b] = acc[a][b];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < pb * nx; e += blockDim.x) {
    T s = (T)0;
#pragma unroll
    for (int g = 0; g < QNG; ++g) s += wpart[(size_t)g * QB * nx + e];
    W[e] = s;
  }
  __syncthreads();
}

// Squared-norm floor of the Householder columns: m (4 eps max|A|)^2, the
// rounding noise of the matrix in its own type.
template <typename T>
__device__ T qr_noise_floor2(const T* A, int m, int n, int lda, T* red) {
  T amax = (T)0;
  for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x)
    amax = fmax(amax, fabs(A[(size_t)(idx / n) * lda + idx % n]));
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  T a = (T)0;
  for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) a = fmax(a, red[w]);
  __syncthreads();
  const T f = (T)(4.0 * Eps<T>::v) * a;
  return (T)m * f * f;
}

// Squared-norm floor of the Householder columns below which a column counts
// as zero.  FP64 data: m (4 eps max|A|)^2, its rounding noise.  FP32 data: the
// column norms, beta and tau are formed in FP64 (no squares underflow), so
// only columns below 2^-60 of the largest entry, or with norm under 1e-36
// (the edge of the FP32 range), are zero: small columns of a matrix with a
// wide spread of column scales (a mixed-canonical centre carries its singular
// values in its columns) are kept.
template <typename T>
__device__ double qr_zero_floor2(const T* A, int m, int n, int lda, T* red) {
  if constexpr (sizeof(T) == 8) {
    return (double)qr_noise_floor2<T>(A, m, n, lda, red);
  } else {
    T amax = (T)0;
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x)
      amax = fmax(amax, fabs(A[(size_t)(idx / n) * lda + idx % n]));
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    T mx = (T)0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) mx = fmax(mx, red[w]);
    __syncthreads();
    const double f = 8.673617379884035e-19 * (double)mx;     // 2^-60 max|A|
    return fmax((double)m * f * f, 1e-72);
  }
}

// Sum over the block in the norm type N (double, or float for the scaled FP32
// norms); `red` is shared scratch of >= 32 doubles.
template <typename N>
__device__ inline N block_sum_n(N v, double* red) {
  if constexpr (sizeof(N) == 8) {
    return block_sum(v, red);
  } else {
    N* r = (N*)red;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) r[wid] = v;
    __syncthreads();
    N s = 0;
    const int nw = (blockDim.x + 31) >> 5;
    if (wid == 0) {
      s = lane < nw ? r[lane] : (N)0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) r[0] = s;
    }
    __syncthreads();
    s = r[0];
    __syncthreads();
    return s;
  }
}

// Householder QR, blocked by panels of QB columns.  Column norms and the
// reflector scalars: FP64 for FP64 data; for FP32 data FP32 on the matrix
// scaled by 2^-e (2^e the power of two at max|A|, an exact scaling), so that no
// square of an entry above the zero floor (2^-60 max|A|) leaves the FP32
// normal range.
template <typename T>
__device__ void householder_qr_blk(T* A, int m, int n, int lda, T* Q, int ldq, T* R, int ldr,
                                   double* tau, T* wv, double* red, T* vb, T* wb) {
  using N = T;                                     // type of the norms and reflector scalars
  const int kk = imin(m, n);
  const int G = 8;                                 // threads per column in the panel dots
  __shared__ T s_scale;
  __shared__ N s_norm2;
  __shared__ T sT[QB][QB + 1], sG[QB][QB + 1];
  __shared__ signed char s_dneg[1024];
  T* redT = (T*)red;
  T* wpart = wb;
  T* W = wb + (size_t)QNG * QB * n;
  // columns below the zero floor: a reflector built from them would not be
  // orthogonal and would spoil the larger columns it is applied to
  N floor2, sc2;                                   // floor of the scaled squared norms; the scaling
  if constexpr (sizeof(T) == 8) {
    floor2 = qr_zero_floor2<T>(A, m, n, lda, redT);
    sc2 = 1.0;
  } else {
    T amax = (T)0;
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x)
      amax = fmaxf(amax, fabsf(A[(size_t)(idx / n) * lda + idx % n]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) redT[threadIdx.x >> 5] = amax;
    __syncthreads();
    T mx = (T)0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) mx = fmaxf(mx, redT[w]);
    __syncthreads();
    int e = 0;
    if (mx > 0.f && isfinite(mx)) frexpf(mx, &e);
    sc2 = ldexpf(1.f, -e);                         // max |A| sc2 in [0.5, 1)
    floor2 = (float)m * 7.523164e-37f;             // m (2^-60)^2 in scaled units
  }
  for (int p0 = 0; p0 < kk; p0 += QB) {
    const int pe = imin(p0 + QB, kk), pb = pe - p0;
    {                                              // norm of column p0 below its diagonal
      N part = 0;
      for (int i = p0 + 1 + threadIdx.x; i < m; i += blockDim.x) {
        const N v = (N)A[(size_t)i * lda + p0] * sc2;
        part += v * v;
      }
      const N t = block_sum_n<N>(part, red);
      if (threadIdx.x == 0) s_norm2 = t;
    }
    // ---- panel: column by column, updates restricted to the panel
    for (int j = p0; j < pe; ++j) {
      if (threadIdx.x == 0) {
        const N sig2 = s_norm2;
        const N alpha = (N)A[(size_t)j * lda + j] * sc2;
        if (sig2 <= floor2) {
          tau[j] = 0.0;
          s_scale = sig2 == (N)0 ? (T)0 : (T)-1;   // -1: zero the column below the diagonal
        } else {
          const N beta = -copysign(sqrt(alpha * alpha + sig2), alpha);
          tau[j] = (double)((beta - alpha) / beta);
          s_scale = (T)(sc2 / (alpha - beta));
          A[(size_t)j * lda + j] = (T)(beta / sc2);
        }
      }
      __syncthreads();
      const T tj = (T)tau[j];
      const T sc = s_scale;
      if (tj == (T)0 && sc == (T)-1)
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[(size_t)i * lda + j] = (T)0;
      const int nc = pe - j - 1;
      if (tj != (T)0 && nc > 0) {
        for (int base = 0; base < nc * G; base += blockDim.x) {
          const int t = base + threadIdx.x;
          const bool act = t < nc * G;
          const int c = j + 1 + t / G, p = t % G;
          T acc = (T)0;
          if (act)
            for (int i = j + 1 + p; i < m; i += G) acc += A[(size_t)i * lda + j] * A[(size_t)i * lda + c];
#pragma unroll
          for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
          if (act && p == 0) wv[c] = (A[(size_t)j * lda + c] + sc * acc) * tj;
        }
        __syncthreads();
      }
      N part = 0;
      if (tj != (T)0) {
        const int rows = m - j;
        if (nc > 0) {
          for (int t = threadIdx.x; t < rows * nc; t += blockDim.x) {
            const int ii = j + t / nc, c = j + 1 + t % nc;
            const T vi = (ii == j) ? (T)1 : sc * A[(size_t)ii * lda + j];
            const T nv = A[(size_t)ii * lda + c] - wv[c] * vi;
            A[(size_t)ii * lda + c] = nv;
            if (c == j + 1 && ii > j + 1) {
              const N v = (N)nv * sc2;
              part += v * v;
            }
          }
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[(size_t)i * lda + j] *= sc;
      } else if (nc > 0) {
        for (int i = j + 2 + threadIdx.x; i < m; i += blockDim.x) {
          const N v = (N)A[(size_t)i * lda + j + 1] * sc2;
          part += v * v;
        }
      }
      if (j + 1 < pe) {
        const N t = block_sum_n<N>(part, red);
        if (threadIdx.x == 0) s_norm2 = t;
      } else {
        __syncthreads();
      }
    }
    // ---- trailing columns [pe, n): A <- (I - V T^T V^T) A
    const int nt = n - pe, mr = m - p0;
    if (nt <= 0) continue;
    qr_blk_load_v<T>(A, lda, m, p0, pe, vb);
    qr_blk_make_t<T>(vb, mr, pb, tau + p0, sT, sG);
    T* X = A + (size_t)p0 * lda + pe;
    qr_blk_vtx<T>(vb, mr, pb, X, lda, nt, wpart, W);
    for (int e = threadIdx.x; e < pb * nt; e += blockDim.x) {      // W2 = -T^T W (into wpart)
      const int q = e / nt, c = e % nt;
      T s = (T)0;
      for (int q2 = 0; q2 <= q; ++q2) s += sT[q2][q] * W[(size_t)q2 * nt + c];
      wpart[e] = -s;
    }
    __syncthreads();
    cta_gemm<T>(mr, nt, pb, vb, QB, wpart, nt, X, lda, true);
  }
  // ---- R with non-negative diagonal; remember the signs for Q
  for (int idx = threadIdx.x; idx < kk * n; idx += blockDim.x) {
    const int i = idx / n, c = idx % n;
    const bool neg = A[(size_t)i * lda + i] < (T)0;
    R[(size_t)i * ldr + c] = c >= i ? (neg ? -A[(size_t)i * lda + c] : A[(size_t)i * lda + c]) : (T)0;
    if (c == i) s_dneg[i] = neg ? 1 : 0;
  }
  __syncthreads();
  if (Q == nullptr) return;                        // R only
  // ---- Q = (I - V_0 T_0 V_0^T) ... (I - V_last T_last V_last^T) [I; 0], backwards, in
  // place: X = A[p0:m, p0:kk] with the panel's columns reset to unit vectors
  for (int p0 = ((kk - 1) / QB) * QB; p0 >= 0; p0 -= QB) {
    const int pe = imin(p0 + QB, kk), pb = pe - p0, mr = m - p0, nx = kk - p0;
    qr_blk_load_v<T>(A, lda, m, p0, pe, vb);
    qr_blk_make_t<T>(vb, mr, pb, tau + p0, sT, sG);
    for (int idx = threadIdx.x; idx < m * pb; idx += blockDim.x) {
      const int i = idx / pb, c = p0 + idx % pb;
      A[(size_t)i * lda + c] = (i == c) ? (T)1 : (T)0;
    }
    __syncthreads();
    T* X = A + (size_t)p0 * lda + p0;
    qr_blk_vtx<T>(vb, mr, pb, X, lda, nx, wpart, W);
    for (int e = threadIdx.x; e < pb * nx; e += blockDim.x) {      // W2 = -T W (into wpart)
      const int q = e / nx, c = e % nx;
      T s = (T)0;
      for (int q2 = q; q2 < pb; ++q2) s += sT[q][q2] * W[(size_t)q2 * nx + c];
      wpart[e] = -s;
    }
    __syncthreads();
    cta_gemm<T>(mr, nx, pb, vb, QB, wpart, nx, X, lda, true);
  }
  for (int idx = threadIdx.x; idx < m * kk; idx += blockDim.x) {
    const int i = idx / kk, c = idx % kk;
    const T q = A[(size_t)i * lda + c];
    Q[(size_t)i * ldq + c] = s_dneg[c] ? -q : q;
  }
  __syncthreads();
}

}  // namespace tn

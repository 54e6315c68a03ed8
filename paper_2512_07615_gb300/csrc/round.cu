// TT-rounding of linear combinations of exactly formed terms (one CTA per job).
//
// For a job sum_t coef_t X_t the wide MPS is the block-diagonal sum of Eq. (add);
// its cores are never stored as a whole: at site k the term blocks are formed
// (plain copy, rank-1 mask product, Kronecker product of Eq. (mul), or the shift
// MPO x MPS contraction of Eq. (applympo) with the cores of Sec. 2.5), multiplied
// from the left by the R factor carried from site k-1, and QR-factorised
// (left-orthogonalising sweep, Eq. lorg).  The right-to-left sweep then moves the
// canonical centre back to site 0 with SVDs (Eq. svd-move) and truncates at the
// centre to chi / eps.
#include <algorithm>

#include "cluster.cuh"
#include "linalg.cuh"

namespace tn {

static constexpr int RT = 512;                      // threads per rounding CTA
static constexpr int SM_SMALL = 41 * 1024;          // bookkeeping part of smem
static constexpr int SM_WORK = 176 * 1024;          // work area in smem
static constexpr int MAXK = 1024;                   // max columns of a QR / SVD

size_t round_smem_bytes() { return SM_SMALL + SM_WORK; }

// ---------------------------------------------------------------- layout (host)
void plan_round_job(RoundJob& j, int L, int n_bits, size_t eb) {
  for (int k = 0; k <= L; ++k) {
    int s = 0;
    for (int t = 0; t < j.nterms; ++t) s += term_bond_bound(j.t[t], L, n_bits, k);
    j.rw[k] = (k == 0 || k == L) ? 1 : s;
  }
  // QR-sweep bonds: q_0 = 1, q_{k+1} <= min(2 q_k, rw_{k+1})
  j.qb[0] = 1;
  for (int k = 0; k < L; ++k) j.qb[k + 1] = imin(2 * j.qb[k], j.rw[k + 1]);
  j.qb[L] = 1;
  size_t off = 0;
  auto al = [&](size_t n) { size_t o = off; off += (n + 31) & ~(size_t)31; return o; };
  for (int k = 0; k < L; ++k) j.lay.q_off[k] = al((size_t)2 * j.qb[k] * (k == L - 1 ? 1 : j.qb[k + 1]));
  size_t wmax = 0, mmax = 0, rmax = 0, cmax = 0, jw = 0, jv = 0, us = 0, rz = 0, qw = 0;
  for (int k = 0; k < L; ++k) {
    size_t w = 0;
    for (int t = 0; t < j.nterms; ++t)
      w += (size_t)term_bond_bound(j.t[t], L, n_bits, k) * 2 * term_bond_bound(j.t[t], L, n_bits, k + 1);
    wmax = w > wmax ? w : wmax;
    size_t m = (size_t)j.qb[k] * 2 * j.rw[k + 1];
    mmax = m > mmax ? m : mmax;
    // blocked QR of M (2 q_k x rw_{k+1}): panel reflectors and products
    const size_t qs = qr_blk_scratch<float>(2 * j.qb[k], j.rw[k + 1]);
    qw = qs > qw ? qs : qw;
    size_t r = (size_t)j.qb[k + 1] * j.rw[k + 1];
    rmax = r > rmax ? r : rmax;
    // right sweep at site k: C is q_k x 2 r_{k+1}, r_{k+1} <= min(chi, q_{k+1})
    size_t rn = (size_t)imin(j.chi, j.qb[k + 1]);
    size_t cm = (size_t)j.qb[k] * 2 * rn;
    cmax = cm > cmax ? cm : cmax;
    size_t ncol = imin(j.qb[k], (int)(2 * rn));
    size_t len = j.qb[k] > (int)(2 * rn) ? j.qb[k] : 2 * rn;
    // Jacobi matrices with 16-byte row strides (up to 16 / eb - 1 padding)
    const size_t pad = 16 / eb;
    jw = ncol * (len + pad) > jw ? ncol * (len + pad) : jw;
    jv = ncol * (ncol + pad) > jv ? ncol * (ncol + pad) : jv;
    // range-finder power step (n x l), then B (l x n) of the randomized step
    rz = (2 * rn + pad) * ncol > rz ? (2 * rn + pad) * ncol : rz;
    size_t u = (size_t)j.qb[k] * imin(j.chi, (int)ncol);
    us = u > us ? u : us;
    // C' = Q_{k-1} (2 q_{k-1} x q_k) * US: 2 q_{k-1} x r
    size_t c2 = (size_t)(k > 0 ? j.qb[k - 1] : 1) * 2 * imin(j.chi, (int)ncol);
    cmax = c2 > cmax ? c2 : cmax;
  }
  j.lay.w_off = al(wmax);
  j.lay.m_off = al(mmax);
  j.lay.r_off = al(rmax > 1 ? rmax : 1);
  j.lay.c_off = al(cmax);
  j.lay.jw_off = al(jw);
  j.lay.jv_off = al(jv);
  j.lay.us_off = al(us);
  j.lay.rz_off = al(rz);
  j.lay.qw_off = al(qw);
  if (eb == 8) {
    j.lay.jw64_off = j.lay.jw_off;                 // the FP64 Jacobi matrices are the Jacobi matrices
    j.lay.jv64_off = j.lay.jv_off;
  } else if (j.svd64) {
    size_t w64 = 0, v64 = 0;                       // doubles, in units of T (two floats each)
    for (int k = 0; k < L; ++k) {
      const int rn = imin(j.chi, j.qb[k + 1]);
      const int ncol = imin(j.qb[k], 2 * rn), len = imax(j.qb[k], 2 * rn);
      w64 = std::max(w64, (size_t)ncol * jacobi_ld<double>(len));
      v64 = std::max(v64, (size_t)ncol * jacobi_ld<double>(ncol));
    }
    j.lay.jw64_off = al(2 * w64);
    j.lay.jv64_off = al(2 * v64);
  } else {
    j.lay.jw64_off = j.lay.jv64_off = 0;
  }
  j.lay.total = off;
}

// ---------------------------------------------------------------- device helpers
__device__ inline void flag(int* st, int code) { atomicOr(st, code); }

template <typename T>
__device__ inline const T* core_ptr(const MpsRef& m, int L, int k) {
  return (const T*)m.base + core_offset(L, m.cap, k);
}

// Input index s of the shift MPO block (w, s_out, w') at site k, or -1 (zero).
// 1-D cores (Sec. 2.5): first [I X], middle [[I j],[0 j']], last [j; j'],
// X = P (cyclic) or j (non-cyclic); (j, j') = (J, J') for offset +1, swapped for -1.
// Non-axis sites carry the identity and pass the bond through.
__device__ inline int shift_src(const Term& t, int n_bits, int k, int w, int so, int w2) {
  if (k % 3 != t.axis) return (w == w2) ? so : -1;             // identity padding
  const int lev = k / 3;
  // 2x2 blocks as functions out -> in: I: s; J: out0<-in1; J': out1<-in0; P: 1-s
  const int jJ = (t.offset == 1) ? 0 : 1;   // 0: j = J, 1: j = J'
  auto blockJ = [&](int which) -> int {     // which 0 = j, 1 = j'
    int isJ = (which == 0) ? (jJ == 0) : (jJ == 1);
    if (isJ) return so == 0 ? 1 : -1;      // J: (0,1)
    return so == 1 ? 0 : -1;               // J': (1,0)
  };
  if (n_bits == 1) {                        // single 2x2 operator
    if (t.cyclic) return 1 - so;
    return blockJ(0);
  }
  if (lev == 0) {                           // [I  X], 1 x 2
    if (w2 == 0) return so;
    if (t.cyclic) return 1 - so;
    return blockJ(0);
  }
  if (lev == n_bits - 1) {                  // [j; j'], 2 x 1
    return blockJ(w == 0 ? 0 : 1);
  }
  if (w == 0 && w2 == 0) return so;         // [[I j],[0 j']]
  if (w == 0 && w2 == 1) return blockJ(0);
  if (w == 1 && w2 == 1) return blockJ(1);
  return -1;
}

__device__ inline int shift_w(const Term& t, int n_bits, int k) {   // MPO bond at bond k
  int first = t.axis, last = t.axis + 3 * (n_bits - 1);
  return (k > first && k <= last) ? 2 : 1;
}

__device__ inline int term_bond(const Term& t, int n_bits, int k) {
  switch (t.kind) {
    case T_ONES: return 1;
    case T_PLAIN:
    case T_MASK1: return t.x.ranks[k];
    case T_KRON: return t.x.ranks[k] * t.y.ranks[k];
    case T_SHIFT: return shift_w(t, n_bits, k) * t.x.ranks[k];
  }
  return 0;
}

// element (i, s, j) of term t's core k (coefficient not applied)
template <typename T>
__device__ inline T term_elem(const Term& t, int L, int n_bits, int k, int i, int s, int j,
                              const T* masks) {
  switch (t.kind) {
    case T_ONES: return (T)1;
    case T_PLAIN: {
      const int r1 = t.x.ranks[k + 1];
      return core_ptr<T>(t.x, L, k)[((size_t)i * 2 + s) * r1 + j];
    }
    case T_MASK1: {
      const int r1 = t.x.ranks[k + 1];
      return core_ptr<T>(t.x, L, k)[((size_t)i * 2 + s) * r1 + j] *
             masks[((size_t)t.mask_id * TN_MAXL + k) * 2 + s];
    }
    case T_KRON: {
      const int rb = t.y.ranks[k], rb1 = t.y.ranks[k + 1], ra1 = t.x.ranks[k + 1];
      const int a = i / rb, b = i % rb, a1 = j / rb1, b1 = j % rb1;
      return core_ptr<T>(t.x, L, k)[((size_t)a * 2 + s) * ra1 + a1] *
             core_ptr<T>(t.y, L, k)[((size_t)b * 2 + s) * rb1 + b1];
    }
    case T_SHIFT: {
      const int ra = t.x.ranks[k], ra1 = t.x.ranks[k + 1];
      const int w = i / ra, a = i % ra, w2 = j / ra1, a1 = j % ra1;
      const int si = shift_src(t, n_bits, k, w, s, w2);
      if (si < 0) return (T)0;
      return core_ptr<T>(t.x, L, k)[((size_t)a * 2 + si) * ra1 + a1];
    }
  }
  return (T)0;
}

// ---------------------------------------------------------------- the kernel
// Shared memory map (bytes): [0,16K) bond bookkeeping; then 32 doubles of
// reduction scratch, tau[MAXK], sig[MAXK] (doubles), wv[MAXK] (T); the rest is
// the work area holding the QR panel (left sweep) or the Jacobi pair W, V
// (right sweep) whenever they fit.
static constexpr int SM_RED = 16 * 1024;
static constexpr int SM_TAU = SM_RED + 256;
static constexpr int SM_SIG = SM_TAU + (MAXK + 8) * 8;   // tau also holds tails at [2, MAXK+2)
static constexpr int SM_WV = SM_SIG + MAXK * 8;
static_assert(SM_WV + MAXK * 8 <= SM_SMALL, "bookkeeping overlaps the work area");
static_assert(16 * 1024 >= (2 * TN_MAXT * (TN_MAXL + 1) + TN_MAXT + 2 * (TN_MAXL + 1) + MAXK) * 4, "bond tables");

// phase timer of thread 0 (profiling only)
// Phase timers and counters of thread 0, kept in shared memory so that they
// hold no registers across the kernel (slots: PH_*).
struct PhaseClock {
  long long t0 = 0;
  double* acc;
  bool on;
  __device__ PhaseClock(bool enable, double* sh) : acc(sh), on(enable && threadIdx.x == 0) {
    if (on) {
      for (int p = 0; p < PH_COUNT; ++p) acc[p] = 0.0;
      t0 = clock64();
    }
  }
  __device__ void lap(int ph) {
    if (!on) return;
    const long long t = clock64();
    acc[ph] += (double)(t - t0);
    t0 = t;
  }
};

// Lap timer of the cluster Jacobi's sub-phases (thread 0 of the leader CTA;
// acc null elsewhere).
struct RxClock {
  double* acc;
  long long t0;
  __device__ explicit RxClock(double* a) : acc(threadIdx.x == 0 ? a : nullptr), t0(0) {
    if (acc) t0 = clock64();
  }
  __device__ void lap(int ph) {
    if (!acc) return;
    const long long t = clock64();
    acc[ph] += (double)(t - t0);
    t0 = t;
  }
};

// ---------------------------------------------------------------- row-partitioned FP64 SVD
// Work-area layout (bytes, same in every CTA of the cluster) of svd64_rows:
// the CTA's rows of W and of V (FP64), the column norms, each pair's rotation
// and flag, the exchange buffers of the pair inner products and of the
// column norms, and the singular values, order and tails the rank rule
// reads.  For FP32 data the block of G = V0^T V0 and the staged rows of V and
// of X used by the Newton-Schulz step and by W = X V share the exchange
// buffers' space (those run before the first exchange of the sweeps).
struct RowsLayout {
  int lw, lv, npairs, kc;
  size_t wl, vl, nrm, pcw, psw, pf, gl, xb, nbuf, gb, st, xs, sig, perm, tail, total;
};
__host__ __device__ inline RowsLayout rows_layout(int ncol, int len, int P, bool two_phase) {
  RowsLayout R;
  R.lw = (len + P - 1) / P;
  R.lv = (ncol + P - 1) / P;
  R.npairs = (ncol + 1) / 2;
  R.kc = imax(1, imin(32, 2048 / imax(ncol, 1)));      // staged rows of V per chunk (<= 16 KB)
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 15) & ~(size_t)15; return r; };
  auto rnd16 = [](size_t bytes) { return (bytes + 15) & ~(size_t)15; };
  R.wl = take((size_t)ncol * R.lw * 8);
  R.vl = take((size_t)ncol * R.lv * 8);
  R.nrm = take((size_t)ncol * 8);
  R.pcw = take((size_t)R.npairs * 8);
  R.psw = take((size_t)R.npairs * 8);
  R.pf = take((size_t)R.npairs * 4);
  R.gl = take((size_t)imax(R.npairs, ncol) * 8);
  // shared region: exchange buffers | Newton-Schulz and X V staging
  const size_t xch = rnd16((size_t)2 * R.npairs * P * 8) + rnd16((size_t)ncol * P * 8);
  const size_t stg = two_phase ? rnd16((size_t)ncol * R.lv * 8) + rnd16((size_t)ncol * R.kc * 8) +
                                     rnd16((size_t)R.lw * R.kc * 8)
                               : 0;
  const size_t base = take(xch > stg ? xch : stg);
  R.xb = base;
  R.nbuf = base + rnd16((size_t)2 * R.npairs * P * 8);
  R.gb = base;
  R.st = base + rnd16((size_t)ncol * R.lv * 8);
  R.xs = R.st + rnd16((size_t)ncol * R.kc * 8);
  R.sig = take((size_t)ncol * 8);
  R.perm = take((size_t)ncol * 4);
  R.tail = take((size_t)(ncol + 2) * 8);
  R.total = o;
  return R;
}

template <typename S>
__device__ __forceinline__ S fmx(S a, S b, S c) {
  if constexpr (sizeof(S) == 8) return fma(a, b, c);
  else return fmaf(a, b, c);
}

// Sum of n values x[0], x[s], x[2s], ... in a fixed order with four
// independent accumulators; the same inputs give the same result in every CTA.
template <typename S>
__device__ __forceinline__ S sum4(const S* x, int n, int s) {
  S a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  int c = 0;
  for (; c + 3 < n; c += 4) {
    a0 += x[(size_t)c * s];
    a1 += x[(size_t)(c + 1) * s];
    a2 += x[(size_t)(c + 2) * s];
    a3 += x[(size_t)(c + 3) * s];
  }
  for (; c < n; ++c) a0 += x[(size_t)c * s];
  return (a0 + a1) + (a2 + a3);
}

// round-robin pair p of round rnd over np (even) indices, a < b
__device__ __forceinline__ void rr_pair(int rnd, int p, int np, int& a, int& b) {
  if (p == 0) { a = rnd; b = np - 1; }
  else { a = (rnd + p) % (np - 1); b = (rnd - p + (np - 1)) % (np - 1); }
  if (a > b) { const int t = a; a = b; b = t; }
}

// Column norms of the S-typed rows Wl over the cluster, in S arithmetic:
// every CTA sums its rows, sends the partial sums to every CTA, and every CTA
// adds them in rank order (the same values in every CTA).  Ends with nrm[]
// valid everywhere.
template <typename S>
__device__ inline void rows_norms(ClusterCtx& cc, const RowsLayout& R, unsigned char* wa, const S* Wl, int ncol,
                                  int li) {
  S* nb = (S*)(wa + R.nbuf);
  S* nrm = (S*)(wa + R.nrm);
  S* loc = (S*)(wa + R.gl);
  cl_xchg_expect(cc, (unsigned)(ncol * cc.P * sizeof(S)));
  for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
    const S* w = Wl + (size_t)j * R.lw;
    S v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    int ii = 0;
    for (; ii + 3 < li; ii += 4) {
      v0 = fmx(w[ii], w[ii], v0);
      v1 = fmx(w[ii + 1], w[ii + 1], v1);
      v2 = fmx(w[ii + 2], w[ii + 2], v2);
      v3 = fmx(w[ii + 3], w[ii + 3], v3);
    }
    for (; ii < li; ++ii) v0 = fmx(w[ii], w[ii], v0);
    const S v = (v0 + v1) + (v2 + v3);
    if (cc.P == 1) nb[j] = v;
    else loc[j] = v;
  }
  // stores into the other CTAs follow the last exchange by at most a round,
  // far less than a CTA that gave up waits at the exit barrier
  if (cc.P > 1) {
    __syncthreads();
    if (!cc.dead)
      for (int idx = threadIdx.x; idx < ncol * cc.P; idx += blockDim.x) {
        const int j = idx / cc.P, d = idx % cc.P;
        cl_xchg_send(cc, nb + (size_t)j * cc.P + cc.rank, d, loc[j]);
      }
  }
  cl_xchg_wait(cc);
  for (int j = threadIdx.x; j < ncol; j += blockDim.x) nrm[j] = sum4<S>(nb + (size_t)j * cc.P, cc.P, 1);
  __syncthreads();
}

// This CTA's parts of the inner products of the pairs of round rnd (S sums;
// four lanes per pair, so that the FP64 work of a round is spread over four
// warps), sent to every CTA's exchange slots xq[p][rank]; then the wait for
// the other CTAs' parts.
template <typename S>
__device__ inline bool rows_pair_dots(ClusterCtx& cc, const RowsLayout& R, unsigned char* wa, const S* Wl,
                                      S* xq, int rnd, int np, int ncol, int li, RxClock& rx) {
  const int npairs = np / 2;
  S* loc = (S*)(wa + R.gl);
  cl_xchg_expect(cc, (unsigned)(npairs * cc.P * sizeof(S)));
  for (int t = threadIdx.x; t < npairs * 4; t += blockDim.x) {
    const int p = t >> 2, q = t & 3;
    const unsigned grp = 0xfu << (threadIdx.x & 28);
    int a, b;
    rr_pair(rnd, p, np, a, b);
    S g0 = 0, g1 = 0;
    if (b < ncol) {
      const S* x = Wl + (size_t)a * R.lw;
      const S* y = Wl + (size_t)b * R.lw;
      int ii = q;
      for (; ii + 4 < li; ii += 8) {
        g0 = fmx(x[ii], y[ii], g0);
        g1 = fmx(x[ii + 4], y[ii + 4], g1);
      }
      if (ii < li) g0 = fmx(x[ii], y[ii], g0);
    }
    S g = g0 + g1;
    g += __shfl_xor_sync(grp, g, 1, 4);
    g += __shfl_xor_sync(grp, g, 2, 4);
    if (q == 0) {
      if (cc.P == 1) xq[p] = g;
      else loc[p] = g;
    }
  }
  if (cc.P > 1) {
    __syncthreads();
    if (!cc.dead)
      for (int idx = threadIdx.x; idx < npairs * cc.P; idx += blockDim.x) {
        const int p = idx / cc.P, d = idx % cc.P;
        cl_xchg_send(cc, xq + (size_t)p * cc.P + cc.rank, d, loc[p]);
      }
  }
  rx.lap(PH_RX_DOT);
  const bool ok = cl_xchg_wait(cc);
  rx.lap(PH_RX_WAIT);
  return ok;
}

// (c, s) of FP32 values renormalised in FP64: (c, s) (1 + d)^(-1/2) with
// d = c^2 + s^2 - 1 (exact in FP64: the squares have 48 bits) and the series
// to d^2 (error O(d^3) ~ 1e-20): orthogonal to FP64 rounding.
__device__ __forceinline__ void renorm64(float cf, float sf, double& c, double& s) {
  const double c0 = (double)cf, s0 = (double)sf;
  const double dr = fma(c0, c0, s0 * s0) - 1.0;
  const double h = fma(dr, fma(0.375, dr, -0.5), 1.0);
  c = c0 * h;
  s = s0 * h;
}

// Rotation of a pair with norms al, be and inner product g (exchanged FP64
// values, identical in every CTA): false if the pair counts as orthogonal
// (g^2 <= tol2 al be) or a column is negligible.  t = tan(theta) is
// Rutishauser's root of the FP32 quotient zeta = (be - al) / (2 g) of the
// FP64 difference (a quotient outside the FP32 range is formed in FP64, with
// t = 1 / (2 zeta) once |zeta| > 1e18).  (c, s) = (1, t) (1 + t^2)^(-1/2)
// orthogonal to FP64 rounding: for |t| < 2^-14 by the series c = 1 - t^2/2,
// s = t c; else the FP32 (c, s) renormalised in FP64 (renorm64).  The new
// norms are al - t g and be + t g (exact for the exact root; recomputed every
// sweep); rel2 = g^2 / (al be) for the stopping rule.
__device__ __forceinline__ bool rows_angle(double al, double be, double g, double tol2, double& cw, double& sw,
                                           double& na, double& nb, float& rel2) {
  const double gg = g * g, ab = al * be;
  if (g == 0.0 || !(al > 1e-250) || !(be > 1e-250) || gg <= tol2 * ab) return false;
  rel2 = (float)gg / (float)ab;                         // +inf if al be leaves the FP32 range
  const double d = be - al;
  float tf = 0.f;
  double t;
  bool tiny = false;
  if (fabs(d) > 1e18 * fabs(g) || fabs(g) < 1e-30) {
    const double zd = d / (2.0 * g);                    // outside the FP32 range: FP64 (rare)
    if (fabs(zd) > 1e18) {
      t = 0.5 / zd;
      tiny = true;
    } else {
      const float z = (float)zd;
      tf = copysignf(1.f / (fabsf(z) + sqrtf(fmaf(z, z, 1.f))), z);
      t = (double)tf;
    }
  } else {
    const float z = (float)d / (2.f * (float)g);
    tf = copysignf(1.f / (fabsf(z) + sqrtf(fmaf(z, z, 1.f))), z);
    t = (double)tf;
  }
  if (tiny) {
    cw = 1.0;                                           // 1 + t^2 rounds to 1 for |t| < 1e-18
    sw = t;
  } else if (fabsf(tf) < 6.1035156e-05f) {
    // c^2 + s^2 = 1 - 3 t^4 / 4 + ...: orthogonal to FP64 rounding
    const double c = fma(-0.5 * t, t, 1.0);
    cw = c;
    sw = t * c;
  } else {
    const float cf = rsqrtf(fmaf(tf, tf, 1.f)), sf = cf * tf;
    renorm64(cf, sf, cw, sw);
  }
  na = al - t * g;
  nb = be + t * g;
  return true;
}

// Cyclic one-sided Jacobi sweeps (round-robin order) on the cluster's FP64
// rows of W and V; nrot counts rotations.  Per round: each CTA's parts of the
// pair inner products go to every CTA, four lanes per pair add them in rank
// order, lane 0 takes the angle, and every CTA rotates its rows of W and V.
// Stopping rule: a sweep that rotates nothing (every pair within the
// tolerance), or a sweep whose largest relative inner product
// g^2 / (al be) was below (5e-9)^2 -- Jacobi converges quadratically,
// so its rotations leave every pair below ~(5e-9)^2 ncol plus the FP32 angle's
// residual 1.2e-7 x 5e-9, under the tolerance 16 eps_64 sqrt(len) >= 5e-15,
// and the confirming sweep is skipped.  Every CTA sees the same values, so
// every CTA stops at the same sweep.  Returns the sweeps used; *converged
// tells whether the rule was met within maxsw sweeps.
template <typename S>
__device__ int rows_sweeps(ClusterCtx& cc, const RowsLayout& R, unsigned char* wa, S* Wl, double* Vl, int ncol,
                           int li, int vi, int maxsw, S tol2, unsigned* nrot, double* phase_acc, bool* converged,
                           int* rounds_out = nullptr) {
  static_assert(sizeof(S) == 8, "the cluster sweeps run on FP64 rows");
  __shared__ float s_mrel[32];
  RxClock rx(phase_acc);
  unsigned q = 0;                                  // rounds so far (exchange buffer parity)
  S* nrm = (S*)(wa + R.nrm);
  S* xb = (S*)(wa + R.xb);
  S* pcw = (S*)(wa + R.pcw);
  S* psw = (S*)(wa + R.psw);
  int* pfl = (int*)(wa + R.pf);
  const int np = (ncol + 1) & ~1, npairs = np / 2;
  int sweep = 0, rounds = 0;
  *converged = true;
  if (ncol < 2) return 0;
  *converged = false;
  // rotation of this CTA's rows of V by round rnd's pairs
  auto rotate_v = [&](int rnd) {
    for (int idx = threadIdx.x; idx < npairs * vi; idx += blockDim.x) {
      const int p = idx / vi, ii = idx - p * vi;
      if (!pfl[p]) continue;
      int a, b;
      rr_pair(rnd, p, np, a, b);
      const double cs = pcw[p], sn = psw[p];
      double* pa = Vl + (size_t)a * R.lv + ii;
      double* pb = Vl + (size_t)b * R.lv + ii;
      const double u = *pa, w = *pb;
      *pa = cs * u - sn * w;
      *pb = sn * u + cs * w;
    }
  };
  for (; sweep < maxsw; ++sweep) {
    rows_norms<S>(cc, R, wa, Wl, ncol, li);
    rx.lap(PH_RX_NORM);
    int any = 0;
    float mrel = 0.f;                              // largest g^2 / (al be) this thread rotated this sweep
    bool ok = rows_pair_dots<S>(cc, R, wa, Wl, xb + (size_t)(q & 1) * npairs * cc.P, 0, np, ncol, li, rx);
    for (int rnd = 0; rnd < np - 1 && ok; ++rnd, ++q) {
      const S* xq = xb + (size_t)(q & 1) * npairs * cc.P;
      ++rounds;
      int rot = 0;
      for (int t = threadIdx.x; t < npairs * 4; t += blockDim.x) {
        const int p = t >> 2, l = t & 3;
        const unsigned grp = 0xfu << (threadIdx.x & 28);
        // the partials of pair p in rank order: lane l adds ranks l, l+4, ...,
        // then the four lanes combine (the same order in every CTA)
        S g = 0;
        for (int c = l; c < cc.P; c += 4) g += xq[(size_t)p * cc.P + c];
        g += __shfl_xor_sync(grp, g, 1, 4);
        g += __shfl_xor_sync(grp, g, 2, 4);
        if (l != 0) continue;
        int a, b;
        rr_pair(rnd, p, np, a, b);
        int go = 0;
        if (b < ncol) {
          S cw, sw, na, nb;
          float rel2 = 0.f;
          if (rows_angle(nrm[a], nrm[b], g, tol2, cw, sw, na, nb, rel2)) {
            mrel = fmaxf(mrel, rel2);
            nrm[a] = na;
            nrm[b] = nb;
            pcw[p] = cw;
            psw[p] = sw;
            go = 1;
            atomicAdd(nrot, 1u);
          }
        }
        pfl[p] = go;
        rot |= go;
      }
      any |= __syncthreads_or(rot);
      rx.lap(PH_RX_ANGLE);
      // the rotations of W, one element pair per thread
      for (int idx = threadIdx.x; idx < npairs * li; idx += blockDim.x) {
        const int p = idx / li, ii = idx - p * li;
        if (!pfl[p]) continue;
        int a, b;
        rr_pair(rnd, p, np, a, b);
        const S cs = pcw[p], sn = psw[p];
        S* pa = Wl + (size_t)a * R.lw + ii;
        S* pb = Wl + (size_t)b * R.lw + ii;
        const S u = *pa, w = *pb;
        *pa = cs * u - sn * w;
        *pb = sn * u + cs * w;
      }
      rotate_v(rnd);
      __syncthreads();
      rx.lap(PH_RX_ROT);
      if (rnd + 1 < np - 1)
        ok = rows_pair_dots<S>(cc, R, wa, Wl, xb + (size_t)((q + 1) & 1) * npairs * cc.P, rnd + 1, np, ncol, li,
                               rx);
    }
    if (cc.dead) break;
    if (!any) { *converged = true; break; }
    // the sweep's largest relative inner product (the same in every CTA)
    for (int o = 16; o > 0; o >>= 1) mrel = fmaxf(mrel, __shfl_xor_sync(0xffffffffu, mrel, o));
    if ((threadIdx.x & 31) == 0) s_mrel[threadIdx.x >> 5] = mrel;
    __syncthreads();
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_mrel[w]);
    __syncthreads();
    if (m < 2.5e-17f) { *converged = true; ++sweep; break; }
  }
  if (phase_acc && threadIdx.x == 0) phase_acc[PH_ROUNDS64] += rounds;
  if (rounds_out) *rounds_out = rounds;
  if (cc.dead) { *converged = false; return maxsw; }
  return sweep;
}

// Stage rows [k0, k0 + nk) of every column of the ncol x ncol matrix V
// (global, column c at V + c * ld, type S) in shared memory as doubles:
// st[c * kc + kk] = V(k0 + kk, c).
template <typename S>
__device__ inline void stage_rows(const S* V, int ld, int ncol, int k0, int nk, int kc, double* st) {
  for (int idx = threadIdx.x; idx < ncol * nk; idx += blockDim.x) {
    const int c = idx / nk, kk = idx - c * nk;
    st[(size_t)c * kc + kk] = (double)__ldcg(V + (size_t)c * ld + k0 + kk);
  }
}

// One Newton-Schulz step towards the orthogonal polar factor, in FP64, on
// this CTA's block of columns J = [v0, v0 + vi): G(:, J) = V0^T V0(:, J),
// V1(:, J) = V0 (3/2 I - 1/2 G)(:, J).  V0 (type S, ld0) and V1 (FP64, ld1)
// are global; V0 is read in staged row chunks.  With V0^T V0 = I + E the
// step leaves V1^T V1 = I + O(E^2) (3/4 E^2 to second order).
template <typename S>
__device__ inline void rows_ns_step(const RowsLayout& R, unsigned char* wa, const S* V0, int ld0, double* V1,
                                    int ld1, int ncol, int v0, int vi) {
  double* G = (double*)(wa + R.gb);                      // G[jj * ncol + i] = G(i, v0 + jj)
  double* st = (double*)(wa + R.st);
  const int kc = R.kc;
  for (int idx = threadIdx.x; idx < ncol * vi; idx += blockDim.x) G[idx] = 0.0;
  for (int k0 = 0; k0 < ncol; k0 += kc) {
    const int nk = imin(kc, ncol - k0);
    __syncthreads();
    stage_rows<S>(V0, ld0, ncol, k0, nk, kc, st);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncol * vi; idx += blockDim.x) {
      const int jj = idx / ncol, i = idx - jj * ncol;
      const double* x = st + (size_t)i * kc;
      const double* y = st + (size_t)(v0 + jj) * kc;
      double a0 = 0.0, a1 = 0.0;
      int kk = 0;
      for (; kk + 1 < nk; kk += 2) {
        a0 = fma(x[kk], y[kk], a0);
        a1 = fma(x[kk + 1], y[kk + 1], a1);
      }
      if (kk < nk) a0 = fma(x[kk], y[kk], a0);
      G[idx] += a0 + a1;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ncol * vi; idx += blockDim.x) {
    const int jj = idx / ncol, i = idx - jj * ncol;
    G[idx] = (i == v0 + jj ? 1.5 : 0.0) - 0.5 * G[idx];  // H = 3/2 I - 1/2 G
  }
  for (int k0 = 0; k0 < ncol; k0 += kc) {
    const int nk = imin(kc, ncol - k0);
    __syncthreads();
    stage_rows<S>(V0, ld0, ncol, k0, nk, kc, st);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nk * vi; idx += blockDim.x) {
      const int jj = idx / nk, kk = idx - jj * nk;
      const double* h = G + (size_t)jj * ncol;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int i = 0;
      for (; i + 3 < ncol; i += 4) {
        a0 = fma(st[(size_t)i * kc + kk], h[i], a0);
        a1 = fma(st[(size_t)(i + 1) * kc + kk], h[i + 1], a1);
        a2 = fma(st[(size_t)(i + 2) * kc + kk], h[i + 2], a2);
        a3 = fma(st[(size_t)(i + 3) * kc + kk], h[i + 3], a3);
      }
      for (; i < ncol; ++i) a0 = fma(st[(size_t)i * kc + kk], h[i], a0);
      __stcg(V1 + (size_t)(v0 + jj) * ld1 + k0 + kk, (a0 + a1) + (a2 + a3));
    }
  }
  __syncthreads();
}

// W = X V for this CTA's rows (FP64): X(i, k) = scl C(i, k) (C^T when the
// Jacobi runs on the columns of C^T) for the rows [i0, i0 + li), read from
// the job's scratch, and V (ncol x ncol, FP64, column c at V + c * ld), both
// staged in chunks of kc indices k.
template <typename T>
__device__ inline void rows_xv(const RowsLayout& R, unsigned char* wa, const T* C, int n, bool trans, double scl,
                               int i0, int li, const double* V, int ld, double* W, int ncol) {
  double* st = (double*)(wa + R.st);
  double* xs = (double*)(wa + R.xs);                      // xs[kk * li + ii] = X(i0 + ii, k0 + kk)
  const int kc = R.kc;
  for (int idx = threadIdx.x; idx < ncol * li; idx += blockDim.x) W[(size_t)(idx / li) * R.lw + idx % li] = 0.0;
  for (int k0 = 0; k0 < ncol; k0 += kc) {
    const int nk = imin(kc, ncol - k0);
    __syncthreads();
    stage_rows<double>(V, ld, ncol, k0, nk, kc, st);
    for (int idx = threadIdx.x; idx < nk * li; idx += blockDim.x) {
      const int kk = idx / li, ii = idx - kk * li, i = i0 + ii, k = k0 + kk;
      xs[idx] = scl * (double)__ldcg(trans ? C + (size_t)i * n + k : C + (size_t)k * n + i);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ncol * li; idx += blockDim.x) {
      const int j = idx / li, ii = idx - j * li;
      const double* v = st + (size_t)j * kc;
      double a0 = 0.0, a1 = 0.0;
      int kk = 0;
      for (; kk + 1 < nk; kk += 2) {
        a0 = fma(xs[kk * li + ii], v[kk], a0);
        a1 = fma(xs[(kk + 1) * li + ii], v[kk + 1], a1);
      }
      if (kk < nk) a0 = fma(xs[kk * li + ii], v[kk], a0);
      W[(size_t)j * R.lw + ii] += a0 + a1;
    }
  }
  __syncthreads();
}

// FP64 one-sided Jacobi SVD of the centre matrix C (m x n, T, global) with the
// rows of the Jacobi matrices split over the CTAs of the cluster and held in
// shared memory.  X = the columns of C (n <= m) or of C^T, scaled by scl;
// V accumulates the rotations (FP64).  CTA c owns entries
// [c len / P, (c+1) len / P) of every column of W and [c ncol / P,
// (c+1) ncol / P) of every column of V.  Every CTA sums the exchanged parts
// in the same order, so every CTA takes the same rotations.
// FP32 data (T = float): the leader has already run FP32 sweeps on X alone
// and left their V0 (FP32, ncol x ncol) in the job's scratch; one FP64
// Newton-Schulz step, spread over the CTAs by blocks of columns, makes it
// orthogonal to FP64 working accuracy (V0^T V0 - I ~ 1e-6 becomes ~1e-12),
// W = X V is formed in FP64 and the FP64 sweeps start from there -- the
// result is an FP64 one-sided Jacobi SVD of X started from the FP32 sweeps'
// V.  FP64 data start from W = X, V = I.  Column norms are recomputed
// exactly at the start of every sweep and at the end.  Every CTA then finds
// the same singular values, order and kept rank (the rank rule of Eq.
// svd-move with delta) and writes its rows of core k (V^T[:r], r x n) and of
// U S (m x r).  Called by all threads of every CTA with equal arguments;
// returns the kept rank (0 if it exceeds the bond capacity), the FP64
// sweeps, whether their limit was reached, and the FP64 FLOPs executed.
template <typename T>
__device__ int svd64_rows(ClusterCtx& cc, const RoundJob& J, int L, int k, int m, int n, double scl, double delta,
                          int maxsw, int* sweeps_out, bool* noconv, double* exec_flops = nullptr,
                          double* phase_acc = nullptr) {
  constexpr bool two_phase = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_nrot;
  if (threadIdx.x == 0) s_nrot = 0;
  unsigned char* wa = smem + SM_SMALL;
  T* scr = (T*)J.scratch;
  const T* C = scr + J.lay.c_off;
  T* US = scr + J.lay.us_off;
  T* out = (T*)J.dst.base + core_offset(L, J.dst.cap, k);
  const int ncol = imin(m, n), len = imax(m, n);
  const bool trans = (n <= m);
  const RowsLayout R = rows_layout(ncol, len, cc.P, two_phase);
  double* Wl = (double*)(wa + R.wl);
  double* Vl = (double*)(wa + R.vl);
  double* nrm = (double*)(wa + R.nrm);
  double* sig = (double*)(wa + R.sig);
  int* perm = (int*)(wa + R.perm);
  double* tail = (double*)(wa + R.tail);
  const int i0 = cc.rank * len / cc.P, li = (cc.rank + 1) * len / cc.P - i0;
  const int v0 = cc.rank * ncol / cc.P, vi = (cc.rank + 1) * ncol / cc.P - v0;
  double* W = Wl;
  if constexpr (two_phase) {
    const long long t0 = clock64();
    const float* V0 = (const float*)(scr + J.lay.jv_off);
    const int ld0 = jacobi_ld<float>(ncol), ld1 = jacobi_ld<double>(ncol);
    double* V1 = (double*)(scr + J.lay.jv64_off);
    rows_ns_step<float>(R, wa, V0, ld0, V1, ld1, ncol, v0, vi);
    cl_sync(cc);                                  // every block of V1 written (cluster-scope fence)
    if (phase_acc && threadIdx.x == 0) phase_acc[PH_NS] += (double)(clock64() - t0);
    const long long t1 = clock64();
    for (int idx = threadIdx.x; idx < ncol * vi; idx += blockDim.x) {
      const int j = idx / vi, ii = idx % vi;
      Vl[(size_t)j * R.lv + ii] = __ldcg(V1 + (size_t)j * ld1 + v0 + ii);
    }
    rows_xv<T>(R, wa, C, n, trans, scl, i0, li, V1, ld1, W, ncol);
    cl_sync(cc);                                  // the staging space is the exchange buffers' again
    if (phase_acc && threadIdx.x == 0) phase_acc[PH_XV] += (double)(clock64() - t1);
  } else {
    // own rows of X (promoted, scaled by a power of two: exact)
    for (int idx = threadIdx.x; idx < ncol * li; idx += blockDim.x) {
      const int j = idx / li, ii = idx % li, i = i0 + ii;
      const T v = trans ? __ldcg(C + (size_t)i * n + j) : __ldcg(C + (size_t)j * n + i);
      Wl[(size_t)j * R.lw + ii] = scl * (double)v;
    }
    for (int idx = threadIdx.x; idx < ncol * vi; idx += blockDim.x) {
      const int j = idx / vi, ii = idx % vi;
      Vl[(size_t)j * R.lv + ii] = (j == v0 + ii) ? 1.0 : 0.0;
    }
    __syncthreads();
  }
  const double tol64 = 16.0 * 2.220446049250313e-16 * sqrt((double)len);
  bool conv = false;
  int rounds = 0;
  const int sw = rows_sweeps<double>(cc, R, wa, W, Vl, ncol, li, vi, maxsw, tol64 * tol64, &s_nrot, phase_acc,
                                     &conv, &rounds);
  *sweeps_out = sw;
  *noconv = !conv || cc.dead;
  if (exec_flops && threadIdx.x == 0) {
    // over the whole cluster, FP64 only: 6 per rotated element pair of W and
    // V, 2 per element of every pair's inner product and of the norms; for
    // FP32 data the Newton-Schulz step (two ncol^3 products) and X V
    const int np = (ncol + 1) & ~1, npairs = np / 2;
    const double sweeps = (double)rounds / (double)imax(np - 1, 1);
    *exec_flops = 6.0 * (double)s_nrot * (len + ncol) + 2.0 * (double)rounds * npairs * len +
                  2.0 * (sweeps + 1) * ncol * len;
    if (two_phase) *exec_flops += 4.0 * (double)ncol * ncol * ncol + 2.0 * (double)len * ncol * ncol;
  }
  // exact norms -> singular values, order and rank (identical in every CTA);
  // non-finite values order last and are reported
  rows_norms<double>(cc, R, wa, W, ncol, li);
  for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
    const double sv = sqrt(nrm[j]) / scl;
    if (!(sv >= 0.0) || isinf(sv)) { sig[j] = -1.0; atomicOr(cc.status, ST_NAN); }
    else sig[j] = sv;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
    int rank = 0;
    const double sj = sig[j];
    for (int o = 0; o < ncol; ++o) rank += (sig[o] > sj) || (sig[o] == sj && o < j);
    perm[rank] = j;
  }
  __syncthreads();
  __shared__ int s_r;
  if (threadIdx.x == 0) {
    const int rmax = imin(J.chi, ncol);
    double tail2 = 0.0;
    for (int p = ncol - 1; p >= 1; --p) {
      const double sv = sig[perm[p]];
      tail2 += sv * sv;
      tail[2 + p] = tail2;
    }
    int rr = rmax;
    for (int qq = 1; qq <= rmax; ++qq) {
      const double t2 = (qq < ncol) ? tail[2 + qq] : 0.0;
      if (sqrt(t2) <= delta) { rr = qq; break; }
    }
    s_r = rr > bond_cap(L, J.dst.cap, k) ? 0 : rr;
  }
  __syncthreads();
  const int r = s_r;
  if (r > 0 && !cc.dead) {
    if (trans) {
      // core: rows of V^T (entries c in this CTA's V rows); U S: this CTA's rows of W
      for (int idx = threadIdx.x; idx < r * vi; idx += blockDim.x) {
        const int jr = idx / vi, ii = idx % vi;
        __stcg(out + (size_t)jr * n + v0 + ii, (T)Vl[(size_t)perm[jr] * R.lv + ii]);
      }
      for (int idx = threadIdx.x; idx < li * r; idx += blockDim.x) {
        const int ii = idx / r, jr = idx % r;
        __stcg(US + (size_t)(i0 + ii) * r + jr, (T)(W[(size_t)perm[jr] * R.lw + ii] * (1.0 / scl)));
      }
    } else {
      for (int idx = threadIdx.x; idx < r * li; idx += blockDim.x) {
        const int jr = idx / li, ii = idx % li;
        const int pj = perm[jr];
        const double sg = sig[pj] * scl;
        const double v = sg > 0.0 ? W[(size_t)pj * R.lw + ii] / sg : (i0 + ii == jr ? 1.0 : 0.0);
        __stcg(out + (size_t)jr * n + i0 + ii, (T)v);
      }
      for (int idx = threadIdx.x; idx < vi * r; idx += blockDim.x) {
        const int ii = idx / r, jr = idx % r;
        const int pj = perm[jr];
        __stcg(US + (size_t)(v0 + ii) * r + jr, (T)(Vl[(size_t)pj * R.lv + ii] * sig[pj]));
      }
    }
  }
  cl_sync(cc);
  return r;
}

// Shared-memory pointers of the leader CTA that the FP64 centre SVD uses.
struct SiteShared {
  double* red;
  double* tau;     // [1] scale, [2..] tails
  double* sig;
  int* perm;
  int* bad;
  int* rank;
  double* flops;
};

// Centre SVD of one right-to-left step in FP64 (FP32 data promoted, or FP64
// data on a cluster): C (m x n, T, global) = U S V^T by one-sided Jacobi in
// FP64 on the columns of C (n <= m) or of C^T; the rank rule and the
// discarded tail in FP64; writes core k = V^T[:r] (r x n) to out and U S
// (m x r) to US, both in T.  The Jacobi matrices sit in the leader's shared
// memory when the job has one CTA and they fit, else in the job's global
// scratch, where every CTA of the cluster works on them.  Returns the kept
// rank, or 0 after flagging an error.
template <typename T>
__device__ __noinline__ int svd64_site(const RoundJob& J, int L, int k, const T* C, int m, int n, T* out, T* US,
                                       T* scr, T* work, const SiteShared& sh, ClusterCtx& cc, int* status,
                                       const LearnCtx* lc, PhaseClock& pc, double delta) {
  const int ncol = imin(m, n), len = imax(m, n);
  const bool trans = (n <= m);
  const int ldw = jacobi_ld<double>(len), ldv = jacobi_ld<double>(ncol);
  const size_t need = ((size_t)ncol * ldw + (size_t)ncol * ldv) * sizeof(double);
  const bool in_smem = cc.P == 1 && need <= (size_t)SM_WORK;
  double* Wm = in_smem ? (double*)work : (double*)(scr + J.lay.jw64_off);
  double* Vm = in_smem ? (double*)work + (size_t)ncol * ldw : (double*)(scr + J.lay.jv64_off);
  // exact power-of-two scale so that max |C| is in [1, 2) (as the T path)
  T amax = (T)0;
  for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) amax = fmax(amax, fabs(C[idx]));
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = (double)amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmax(a, sh.red[w]);
    int e = 0;
    if (a > 0.0 && isfinite(a)) frexp(a, &e);
    sh.tau[1] = ldexp(1.0, 1 - e);
  }
  __syncthreads();
  const double scl = sh.tau[1];
  const int maxsw = J.max_sweeps > 0 ? J.max_sweeps : 60;
  if (!in_smem && cc.P > 1 && rows_layout(ncol, len, cc.P, sizeof(T) == 4).total <= (size_t)SM_WORK) {
    // rows of the Jacobi matrices spread over the cluster, in shared memory
    pc.lap(PH_SVD_OUT);
    if constexpr (sizeof(T) == 4) {
      // FP32 data: FP32 sweeps on X by this CTA alone (the in-CTA Jacobi of the
      // FP32 path; its own stopping rule, at most 30 sweeps, convergence not
      // required), V0 left in the job's scratch for the cluster
      const int ldw32 = jacobi_ld<float>(len), ldv32 = jacobi_ld<float>(ncol);
      const size_t need32 = ((size_t)ncol * ldw32 + (size_t)ncol * ldv32) * sizeof(float);
      float* Vg = (float*)(scr + J.lay.jv_off);
      // W (the hot operand: len entries per rotated column) in shared memory
      // whenever it fits there alone; V with it if both fit, else in scratch
      const bool w_smem = (size_t)ncol * ldw32 * sizeof(float) <= (size_t)SM_WORK;
      float* Wf = w_smem ? (float*)work : (float*)(scr + J.lay.jw_off);
      float* Vf = need32 <= (size_t)SM_WORK ? (float*)work + (size_t)ncol * ldw32 : Vg;
      for (int idx = threadIdx.x; idx < ncol * len; idx += blockDim.x) {
        const int jj = idx / len, i = idx % len;
        Wf[(size_t)jj * ldw32 + i] = (float)(scl * (double)(trans ? C[(size_t)i * n + jj] : C[(size_t)jj * n + i]));
      }
      __syncthreads();
      const int sw32 = jacobi_cols_fast<float>(Wf, ldw32, Vf, ldv32, ncol, len, imin(maxsw, 30));
      if (Vf != Vg)
        for (int idx = threadIdx.x; idx < ncol * ldv32; idx += blockDim.x) __stcg(Vg + idx, Vf[idx]);
      __syncthreads();
      if (threadIdx.x == 0) pc.acc[PH_SWEEPS32] += sw32;
      pc.lap(PH_J32);
    }
    cl_command(cc, 2, ncol, len, maxsw, m, n, k, delta, scl);
    int sw = 0;
    bool noconv = false;
    double xfl = 0.0;
    const int r = svd64_rows<T>(cc, J, L, k, m, n, scl, delta, maxsw, &sw, &noconv, &xfl, pc.on ? pc.acc : nullptr);
    pc.lap(PH_JACOBI);
    if (threadIdx.x == 0) { pc.acc[PH_SVD64_FLOPS] += svd_flops(m, n); pc.acc[PH_SVD64_EXEC] += xfl; }
    const RowsLayout R = rows_layout(ncol, len, cc.P, sizeof(T) == 4);
    const unsigned char* wa = (const unsigned char*)work;
    const double* sig = (const double*)(wa + R.sig);
    const int* perm = (const int*)(wa + R.perm);
    const double* tail = (const double*)(wa + R.tail);
    if (threadIdx.x == 0) {
      pc.acc[6] += sw; pc.acc[7] += 1.0;
      if (noconv) {
        flag(status, ST_NOCONV);
        if (atomicCAS(&status[1], 0, 1) == 0) {
          status[2] = blockIdx.x / cc.P; status[3] = k; status[4] = ncol; status[5] = len;
        }
      }
      if (r == 0) flag(status, ST_CAPACITY);
      else {
        if (J.discard && r < ncol) atomicAdd(J.discard, tail[2 + r]);
        J.dst.ranks[k] = r;
      }
      *sh.flops += svd_flops(m, n);
      if (lc && lc->counters) atomicAdd(&lc->counters[2], 1);
    }
    // singular values and order where the spectrum log reads them
    for (int j = threadIdx.x; j < ncol; j += blockDim.x) { sh.sig[j] = sig[j]; sh.perm[j] = perm[j]; }
    // the other CTAs wrote rows of the core and of U S at L2: read them back
    // past this SM's L1 before the leader's own loads use them
    if (r > 0) {
      for (int idx = threadIdx.x; idx < r * n; idx += blockDim.x) out[idx] = __ldcg(out + idx);
      for (int idx = threadIdx.x; idx < m * r; idx += blockDim.x) US[idx] = __ldcg(US + idx);
    }
    __syncthreads();
    return r;
  }
  for (int idx = threadIdx.x; idx < ncol * len; idx += blockDim.x) {
    const int jj = idx / len, i = idx % len;
    const double v = scl * (double)(trans ? C[(size_t)i * n + jj] : C[(size_t)jj * n + i]);
    if (in_smem) Wm[(size_t)jj * ldw + i] = v;
    else __stcg(Wm + (size_t)jj * ldw + i, v);
  }
  __syncthreads();
  pc.lap(PH_SVD_OUT);
  const double jac0 = pc.acc[PH_JACOBI];
  int sw;
  if (in_smem) {
    sw = jacobi_cols_fast<double>(Wm, ldw, Vm, ldv, ncol, len, maxsw);
  } else {
    cl_command(cc, 1, ncol, len, maxsw);
    sw = jacobi64_cluster(cc, Wm, ldw, Vm, ldv, ncol, len, maxsw);
  }
  pc.lap(PH_JACOBI);
  if (threadIdx.x == 0) { pc.acc[6] += sw; pc.acc[7] += 1.0; pc.acc[PH_SVD64_FLOPS] += svd_flops(m, n); }
  if (threadIdx.x == 0 && !in_smem) { pc.acc[8] += pc.acc[PH_JACOBI] - jac0; pc.acc[9] += 1.0; }
  if (sw >= maxsw && threadIdx.x == 0) {
    flag(status, ST_NOCONV);
    if (atomicCAS(&status[1], 0, 1) == 0) {
      status[2] = blockIdx.x / cc.P; status[3] = k; status[4] = ncol; status[5] = len;
    }
  }
  auto ldW = [&](size_t i) -> double { return in_smem ? Wm[i] : __ldcg(Wm + i); };
  auto ldV = [&](size_t i) -> double { return in_smem ? Vm[i] : __ldcg(Vm + i); };
  for (int jj = threadIdx.x; jj < ncol; jj += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < len; ++i) { const double w = ldW((size_t)jj * ldw + i); a += w * w; }
    const double sv = sqrt(a) / scl;
    if (!(sv >= 0.0) || isinf(sv)) { sh.sig[jj] = -1.0; flag(status, ST_NAN); }   // orders last
    else sh.sig[jj] = sv;
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < ncol; jj += blockDim.x) {
    int rank = 0;
    const double sj = sh.sig[jj];
    for (int o = 0; o < ncol; ++o) {
      const double so = sh.sig[o];
      rank += (so > sj) || (so == sj && o < jj);
    }
    sh.perm[rank] = jj;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int rmax = imin(J.chi, ncol);
    double tail2 = 0.0;
    int rr = rmax;
    for (int p = ncol - 1; p >= 1; --p) {
      const double sv = sh.sig[sh.perm[p]];
      tail2 += sv * sv;
      sh.tau[2 + p] = tail2;
    }
    for (int q = 1; q <= rmax; ++q) {
      const double t2 = (q < ncol) ? sh.tau[2 + q] : 0.0;
      if (sqrt(t2) <= delta) { rr = q; break; }
    }
    if (rr > bond_cap(L, J.dst.cap, k)) { *sh.bad = 1; rr = bond_cap(L, J.dst.cap, k); }
    *sh.rank = rr;
    if (J.discard && rr < ncol) atomicAdd(J.discard, sh.tau[2 + rr]);
    *sh.flops += svd_flops(m, n);
    if (lc && lc->counters) atomicAdd(&lc->counters[2], 1);
  }
  __syncthreads();
  if (*sh.bad) { if (threadIdx.x == 0) flag(status, ST_CAPACITY); return 0; }
  const int r = *sh.rank;
  for (int idx = threadIdx.x; idx < r * n; idx += blockDim.x) {
    const int jr = idx / n, c = idx % n;
    const int pj = sh.perm[jr];
    double v;
    if (trans) {
      v = ldV((size_t)pj * ldv + c);
    } else {
      const double sg = sh.sig[pj] * scl;
      v = sg > 0.0 ? ldW((size_t)pj * ldw + c) / sg : (c == jr ? 1.0 : 0.0);
    }
    out[idx] = (T)v;
  }
  for (int idx = threadIdx.x; idx < m * r; idx += blockDim.x) {
    const int i = idx / r, jr = idx % r;
    const int pj = sh.perm[jr];
    US[idx] = (T)(trans ? ldW((size_t)pj * ldw + i) * (1.0 / scl) : ldV((size_t)pj * ldv + i) * sh.sig[pj]);
  }
  if (threadIdx.x == 0) J.dst.ranks[k] = r;
  __syncthreads();
  return r;
}

// The rounding job as run by the leader CTA of its cluster (the whole job
// when the cluster has one CTA).
template <typename T>
__device__ void round_job_body(const RoundJob& J, int L_arg, int n_bits_arg, const T* __restrict__ masks_arg,
                               const double* __restrict__ scal_arg, int* __restrict__ status,
                               double* __restrict__ ctr, const LearnCtx* __restrict__ lc, ClusterCtx& cc) {
  // per-job chain length, mask table and scalars (jobs of several simulations,
  // possibly of different lattice sizes, in one launch)
  const int L = J.L > 0 ? J.L : L_arg;
  const int n_bits = J.n_bits > 0 ? J.n_bits : n_bits_arg;
  const T* __restrict__ masks = J.masks ? (const T*)J.masks : masks_arg;
  const double* __restrict__ scal = J.scal ? J.scal : scal_arg;
  extern __shared__ __align__(16) unsigned char smem[];
  int* s_rt = (int*)smem;                            // [TN_MAXT][TN_MAXL+1] term bonds
  int* s_ro = s_rt + TN_MAXT * (TN_MAXL + 1);        // row offsets at each bond
  int* s_wo = s_ro + TN_MAXT * (TN_MAXL + 1);        // per-term offsets in W buffer
  int* s_R = s_wo + TN_MAXT;                         // wide bonds
  int* s_q = s_R + TN_MAXL + 1;                      // QR sweep bonds
  int* s_perm = s_q + TN_MAXL + 1;                   // [MAXK]
  double* s_red = (double*)(smem + SM_RED);
  double* s_tau = (double*)(smem + SM_TAU);
  double* s_sig = (double*)(smem + SM_SIG);
  T* s_wv = (T*)(smem + SM_WV);
  T* work = (T*)(smem + SM_SMALL);
  __shared__ double s_coef[TN_MAXT];
  __shared__ double s_phase[PH_COUNT];
  __shared__ double s_flops;                          // algorithmic FLOPs (thread 0)
  __shared__ int s_bad, s_rank;

  const int nt = J.nterms;
  T* scr = (T*)J.scratch;
  double& flops = s_flops;
  PhaseClock pc(ctr != nullptr, s_phase);
  if (threadIdx.x == 0) { s_bad = 0; s_flops = 0.0; }
  __syncthreads();
  // ---- bonds of every term and of the wide sum
  for (int idx = threadIdx.x; idx < nt * (L + 1); idx += blockDim.x) {
    const int t = idx / (L + 1), k = idx % (L + 1);
    const Term& tm = J.t[t];
    int rb = term_bond(tm, n_bits, k);
    if (tm.kind != T_ONES) {
      if (tm.x.ranks[k] > bond_cap(L, tm.x.cap, k) || tm.x.ranks[k] < 1) s_bad = 1;
      if (tm.kind == T_KRON && (tm.y.ranks[k] > bond_cap(L, tm.y.cap, k) || tm.y.ranks[k] < 1)) s_bad = 1;
    }
    s_rt[t * (TN_MAXL + 1) + k] = rb;
  }
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    double c = J.t[t].coef;
    if (J.t[t].coef_slot >= 0) c *= scal[J.t[t].coef_slot];
    s_coef[t] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k <= L; ++k) {
      int acc = 0;
      for (int t = 0; t < nt; ++t) {
        s_ro[t * (TN_MAXL + 1) + k] = (k == 0 || k == L) ? 0 : acc;
        acc += s_rt[t * (TN_MAXL + 1) + k];
      }
      s_R[k] = (k == 0 || k == L) ? 1 : acc;
      if (s_R[k] > J.rw[k]) s_bad = 1;
    }
  }
  __syncthreads();
  if (s_bad) { if (threadIdx.x == 0) flag(status, ST_CAPACITY); return; }

  // ---- materialise a single term without rounding
  if (J.materialize_only) {
    const Term& tm = J.t[0];
    for (int k = 0; k < L; ++k) {
      const int r0 = s_rt[k], r1 = s_rt[k + 1];
      if (r0 > bond_cap(L, J.dst.cap, k) || r1 > bond_cap(L, J.dst.cap, k + 1)) {
        if (threadIdx.x == 0) flag(status, ST_CAPACITY);
        return;
      }
      T* out = (T*)J.dst.base + core_offset(L, J.dst.cap, k);
      const T cf = (T)(k == 0 ? s_coef[0] : 1.0);
      for (int idx = threadIdx.x; idx < r0 * 2 * r1; idx += blockDim.x) {
        int i = idx / (2 * r1), s = (idx / r1) % 2, jj = idx % r1;
        out[idx] = cf * term_elem<T>(tm, L, n_bits, k, i, s, jj, masks);
      }
    }
    for (int k = threadIdx.x; k <= L; k += blockDim.x) J.dst.ranks[k] = s_rt[k];
    return;
  }

  // ---- left-orthogonalising sweep over the wide sum
  T* Rc = scr + J.lay.r_off;                // carried R factor, rc x R_k (ld R_k)
  if (threadIdx.x == 0) { Rc[0] = (T)1; s_q[0] = 1; }
  __syncthreads();
  int rc = 1;
  for (int k = 0; k < L; ++k) {
    const int Rk = s_R[k], Rk1 = s_R[k + 1];
    // (a) term blocks of core k into W (global scratch)
    T* W = scr + J.lay.w_off;
    if (threadIdx.x == 0) {
      int o = 0;
      for (int t = 0; t < nt; ++t) {
        s_wo[t] = o;
        o += s_rt[t * (TN_MAXL + 1) + k] * 2 * s_rt[t * (TN_MAXL + 1) + k + 1];
      }
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      const int r0 = s_rt[t * (TN_MAXL + 1) + k], r1 = s_rt[t * (TN_MAXL + 1) + k + 1];
      const T cf = (T)(k == 0 ? s_coef[t] : 1.0);
      T* Wt = W + s_wo[t];
      for (int idx = threadIdx.x; idx < r0 * 2 * r1; idx += blockDim.x) {
        int i = idx / (2 * r1), s = (idx / r1) % 2, jj = idx % r1;
        Wt[idx] = cf * term_elem<T>(J.t[t], L, n_bits, k, i, s, jj, masks);
      }
    }
    __syncthreads();
    pc.lap(PH_TERMS);
    // (b) M = Rc * blockdiag(W): rows (r, s), row length Rk1, leading dim ld
    const int mrows = 2 * rc;
    int ld = Rk1 | 1;
    bool in_smem = (size_t)mrows * ld * sizeof(T) <= (size_t)SM_WORK;
    if (!in_smem) ld = Rk1;
    T* M = in_smem ? work : scr + J.lay.m_off;
    const bool last = (k == L - 1);
    if (last)
      for (int idx = threadIdx.x; idx < mrows * ld; idx += blockDim.x) M[idx] = (T)0;
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      const int r0 = s_rt[t * (TN_MAXL + 1) + k], r1 = s_rt[t * (TN_MAXL + 1) + k + 1];
      const int co = s_ro[t * (TN_MAXL + 1) + k + 1], ro = s_ro[t * (TN_MAXL + 1) + k];
      const T* Wt = W + s_wo[t];
      for (int s = 0; s < 2; ++s)
        cta_gemm<T>(rc, r1, r0, Rc + ro, Rk, Wt + s * r1, 2 * r1, M + (size_t)s * ld + co, 2 * ld, last);
      if (threadIdx.x == 0) flops += 4.0 * rc * r0 * r1;
    }
    pc.lap(PH_GEMM_M);
    T* Qk = scr + J.lay.q_off[k];
    if (last) {
      for (int idx = threadIdx.x; idx < mrows; idx += blockDim.x) Qk[idx] = M[(size_t)idx * ld];
      __syncthreads();
      break;
    }
    // (c) QR of M (mrows x Rk1) -> Q_k (ld rq), new carried R (rq x Rk1, ld Rk1)
    const int rq = imin(mrows, Rk1);
    if (rq > MAXK || Rk1 > MAXK) { if (threadIdx.x == 0) flag(status, ST_CAPACITY); return; }
    {
      T* vb = scr + J.lay.qw_off;
      householder_qr_blk<T>(M, mrows, Rk1, ld, Qk, rq, Rc, Rk1, s_tau, s_wv, s_red, vb,
                            vb + (size_t)mrows * QB);
    }
    if (threadIdx.x == 0) flops += qr_flops(mrows, Rk1);
    pc.lap(PH_QR);
    rc = rq;
    if (threadIdx.x == 0) s_q[k + 1] = rq;
    __syncthreads();
    (void)Rk;
  }
  if (threadIdx.x == 0) s_q[L] = 1;
  __syncthreads();

  // ---- right-to-left truncated SVD sweep
  T* C = scr + J.lay.c_off;
  {
    const int q = s_q[L - 1];
    const T* Ql = scr + J.lay.q_off[L - 1];
    double part = 0.0;
    for (int idx = threadIdx.x; idx < 2 * q; idx += blockDim.x) {
      double v = (double)Ql[idx];
      part += v * v;
      C[idx] = Ql[idx];
    }
    double nrm2 = block_sum(part, s_red);
    if (!isfinite(nrm2)) { if (threadIdx.x == 0) flag(status, ST_NAN); }
    if (threadIdx.x == 0) s_tau[0] = J.eps * sqrt(nrm2) / sqrt((double)(L - 1));
    __syncthreads();
  }
  const double delta = s_tau[0];
  __syncthreads();
  int rnext = 1;
  for (int k = L - 1; k >= 1; --k) {
    const int m = s_q[k], n = 2 * rnext;
    T* out = (T*)J.dst.base + core_offset(L, J.dst.cap, k);
    T* US = scr + J.lay.us_off;
    int r = 0;
    bool done = false;             // randomized truncation accepted
    bool full64 = false;           // full SVD taken in FP64 (svd64_site)
    // ---- randomized truncation at a target rank, certified (learned-rank path)
    int tgt = 0;
    if (J.rsvd_mode && lc != nullptr && lc->omega != nullptr) {
      if (J.rsvd_mode == 1) {
        tgt = J.targets ? J.targets[k] : J.rsvd_k;
      } else if (J.rsvd_mode == 3 && J.log != nullptr && J.log->valid[k]) {
        tgt = J.log->label[k];                     // previous step's kept rank
      } else if (J.rsvd_mode == 2 && lc->mlp != nullptr && J.log != nullptr && J.log->valid[k]) {
        const float stepf = lc->step ? fminf((float)(*lc->step) / 1000.f, 1.f) : 0.f;
        tgt = mlp_predict_rank(lc->mlp, J.log->spec[k], (float)k / (float)L, stepf, J.chi,
                               (float*)s_sig);
      }
    }
    tgt = imin(tgt, J.chi);
    const int fullmin = imin(m, n);
    // at least TN_SPEC samples, so that the logged spectrum has every value the model reads
    const int lsamp = imin(imax(tgt + (lc ? lc->oversample : 0), TN_SPEC), fullmin);
    // Y (m x l, and n x l in the power steps) must fit the shared work area;
    // B and V (l x n, l x l) go there too when they fit, else to global scratch
    const bool fits = (size_t)imax(m, n) * (lsamp | 1) * sizeof(T) <= (size_t)SM_WORK;
    const bool bv_smem = ((size_t)lsamp * jacobi_ld<T>(n) + (size_t)lsamp * jacobi_ld<T>(lsamp)) * sizeof(T) <=
                         (size_t)SM_WORK;
    if (tgt > 0 && lsamp < fullmin && fits && n <= lc->omega_rows && lsamp <= lc->omega_ld) {
      const int l = lsamp;
      const int ldy = l | 1, ldw = jacobi_ld<T>(n), ldv = jacobi_ld<T>(l);
      T* Ysm = work;
      const T* Om = (const T*)lc->omega;
      // Y = C Omega (m x l), in shared memory
      cta_gemm<T>(m, l, n, C, n, Om, lc->omega_ld, Ysm, ldy, false);
      T* Qy = scr + J.lay.jw_off;                  // m x l
      T* Rtmp = scr + J.lay.jv_off;                // l x l (discarded)
      // power steps: Y <- C orth(C^T orth(Y)), re-orthonormalised for stability
      for (int it = 0; it < lc->power; ++it) {
        T* Z = scr + J.lay.rz_off;                 // n x l
        householder_qr_par<T>(Ysm, m, l, ldy, Qy, l, Rtmp, l, s_tau, s_wv, s_red);
        cta_gemm_tn<T>(n, l, m, C, n, Qy, l, Ysm, ldy);
        householder_qr_par<T>(Ysm, n, l, ldy, Z, l, Rtmp, l, s_tau, s_wv, s_red);
        cta_gemm<T>(m, l, n, C, n, Z, l, Ysm, ldy, false);
        if (threadIdx.x == 0) flops += 4.0 * m * n * l + qr_flops(m, l) + qr_flops(n, l);
      }
      householder_qr_par<T>(Ysm, m, l, ldy, Qy, l, Rtmp, l, s_tau, s_wv, s_red);
      // B = Qy^T C (l x n), row j = Jacobi column j; in shared memory, or in the
      // power-step and R regions of the scratch (both free by now)
      T* Wm = bv_smem ? work : scr + J.lay.rz_off;
      T* Vm = bv_smem ? work + (size_t)l * ldw : Rtmp;
      cta_gemm_tn<T>(l, n, m, Qy, l, C, n, Wm, ldw);
      // residual ||C - Qy B||^2 and ||C||^2 (FP64 sums)
      double pr = 0.0, pc2 = 0.0;
      for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
        const int i = idx / n, c = idx % n;
        const T* qrow = Qy + (size_t)i * l;
        T acc = C[idx];
        for (int q = 0; q < l; ++q) acc -= qrow[q] * Wm[(size_t)q * ldw + c];
        pr += (double)acc * (double)acc;
        pc2 += (double)C[idx] * (double)C[idx];
      }
      const double resid2 = block_sum(pr, s_red);
      const double c2 = block_sum(pc2, s_red);
      // scale B to max |entry| in [1, 2)
      T amax = (T)0;
      for (int idx = threadIdx.x; idx < l * n; idx += blockDim.x)
        amax = fmax(amax, fabs(Wm[(size_t)(idx / n) * ldw + idx % n]));
      for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = (double)amax;
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmax(a, s_red[w]);
        int e = 0;
        if (a > 0.0 && isfinite(a)) frexp(a, &e);
        s_tau[1] = ldexp(1.0, 1 - e);
      }
      __syncthreads();
      const double scl = s_tau[1];
      for (int idx = threadIdx.x; idx < l * n; idx += blockDim.x)
        Wm[(size_t)(idx / n) * ldw + idx % n] *= (T)scl;
      __syncthreads();
      const int sw = jacobi_cols_fast<T>(Wm, ldw, Vm, ldv, l, n, 60);
      for (int jj = threadIdx.x; jj < l; jj += blockDim.x) {
        T a = (T)0;
        const T* w = Wm + (size_t)jj * ldw;
        for (int i = 0; i < n; ++i) a += w[i] * w[i];
        const double sv = (double)sqrt(a) / scl;
        if (!(sv >= 0.0) || isinf(sv)) { s_sig[jj] = -1.0; flag(status, ST_NAN); }   // orders last
        else s_sig[jj] = sv;
      }
      __syncthreads();
      for (int jj = threadIdx.x; jj < l; jj += blockDim.x) {
        int rank = 0;
        const double sj = s_sig[jj];
        for (int o = 0; o < l; ++o) rank += (s_sig[o] > sj) || (s_sig[o] == sj && o < jj);
        s_perm[rank] = jj;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const int rmax = imin(J.chi, l);
        double tail2 = 0.0;
        s_tau[2 + l] = 0.0;
        for (int p = l - 1; p >= 0; --p) {
          const double sv = s_sig[s_perm[p]];
          tail2 += sv * sv;
          s_tau[2 + p] = tail2;
        }
        int rr = rmax;
        for (int q = 1; q <= rmax; ++q)
          if (sqrt(resid2 + s_tau[2 + q]) <= delta) { rr = q; break; }
        const double err2 = resid2 + s_tau[2 + rr];
        const int full_cap = imin(J.chi, imin(m, n));
        const bool rule_ok = sqrt(err2) <= delta || rr == full_cap || rr == J.chi;
        // accept: measured error within the tolerance, or (at the chi cap) the
        // residual bound proves err^2 <= opt^2 / (1 - eta) (Ky Fan on C^T C = B^T B + E^T E)
        const double floor2 = (double)lc->floor_rel * (double)lc->floor_rel * c2;
        const bool cert = sqrt(err2) <= delta || resid2 <= fmax((double)lc->eta * err2, floor2);
        const bool ok = rule_ok && cert && sw < 60 && rr <= bond_cap(L, J.dst.cap, k);
        s_rank = ok ? rr : 0;
        if (ok && J.discard) atomicAdd(J.discard, err2);
        if (lc->counters) atomicAdd(&lc->counters[ok ? 0 : 1], 1);
        flops += 2.0 * m * n * l * 3 + qr_flops(m, l) + svd_flops(l, n);
      }
      __syncthreads();
      if (s_rank > 0) {
        r = s_rank;
        for (int idx = threadIdx.x; idx < r * n; idx += blockDim.x) {
          const int jr = idx / n, c = idx % n;
          const int pj = s_perm[jr];
          const T sg = (T)(s_sig[pj] * scl);
          out[idx] = sg > (T)0 ? Wm[(size_t)pj * ldw + c] / sg : (T)(c == jr ? 1 : 0);
        }
        for (int idx = threadIdx.x; idx < m * r; idx += blockDim.x) {
          const int i = idx / r, jr = idx % r;
          const int pj = s_perm[jr];
          const T* qrow = Qy + (size_t)i * l;
          const T* vcol = Vm + (size_t)pj * ldv;
          T acc = (T)0;
          for (int q = 0; q < l; ++q) acc += qrow[q] * vcol[q];
          US[idx] = acc * (T)s_sig[pj];
        }
        done = true;
        if (threadIdx.x == 0) J.dst.ranks[k] = r;
      }
      __syncthreads();
      pc.lap(PH_JACOBI);
    }
    // ---- full SVD (reference path, and fallback of the randomized one)
    const int ncol = imin(m, n), len = imax(m, n);
    if (!done && (J.svd64 || (sizeof(T) == 8 && cc.P > 1))) {
      if (ncol > MAXK) { if (threadIdx.x == 0) flag(status, ST_CAPACITY); return; }
      const SiteShared sh{s_red, s_tau, s_sig, s_perm, &s_bad, &s_rank, &s_flops};
      r = svd64_site<T>(J, L, k, C, m, n, out, US, scr, work, sh, cc, status, lc, pc, delta);
      if (r == 0) return;
      full64 = true;
    }
    if (!done && !full64) {
      if (ncol > MAXK) { if (threadIdx.x == 0) flag(status, ST_CAPACITY); return; }
      const bool trans = (n <= m);             // Jacobi on the columns of C
      // 16-byte row strides (vector loads in the Jacobi); shared memory if it
      // fits -- W alone when W and V do not fit together
      const int ldw = jacobi_ld<T>(len), ldv = jacobi_ld<T>(ncol);
      const size_t need = ((size_t)ncol * ldw + (size_t)ncol * ldv) * sizeof(T);
      const bool w_smem = (size_t)ncol * ldw * sizeof(T) <= (size_t)SM_WORK;
      T* Wm = w_smem ? work : scr + J.lay.jw_off;
      T* Vm = (need <= (size_t)SM_WORK) ? work + (size_t)ncol * ldw : scr + J.lay.jv_off;
      const int ldw_e = ldw;
      const int ldv_e = ldv;
      // scale by an exact power of two so that max |C| is in [1, 2): keeps the
      // Jacobi inner products far from under- and overflow; undone exactly below
      T amax = (T)0;
      for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) amax = fmax(amax, fabs(C[idx]));
      for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = (double)amax;
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmax(a, s_red[w]);
        int e = 0;
        if (a > 0.0 && isfinite(a)) frexp(a, &e);
        s_tau[1] = ldexp(1.0, 1 - e);     // scale
      }
      __syncthreads();
      const double scl = s_tau[1];
      const T tscl = (T)scl;
      for (int idx = threadIdx.x; idx < ncol * len; idx += blockDim.x) {
        const int jj = idx / len, i = idx % len;
        Wm[(size_t)jj * ldw_e + i] = tscl * (trans ? C[(size_t)i * n + jj] : C[(size_t)jj * n + i]);
      }
      __syncthreads();
      const int maxsw = J.max_sweeps > 0 ? J.max_sweeps : 60;
      pc.lap(PH_SVD_OUT);
      const double jac0 = pc.acc[PH_JACOBI];
      int sw = jacobi_cols_fast<T>(Wm, ldw_e, Vm, ldv_e, ncol, len, maxsw);
      pc.lap(PH_JACOBI);
      if (threadIdx.x == 0) { pc.acc[6] += sw; pc.acc[7] += 1.0; }   // sweeps, SVD count
      if (threadIdx.x == 0 && need > (size_t)SM_WORK) {               // matrices in global memory
        pc.acc[8] += pc.acc[PH_JACOBI] - jac0;
        pc.acc[9] += 1.0;
      }
      if (sw >= maxsw && threadIdx.x == 0) {
        flag(status, ST_NOCONV);
        if (atomicCAS(&status[1], 0, 1) == 0) {     // first failure: where and how big
          status[2] = blockIdx.x / cc.P; status[3] = k; status[4] = ncol; status[5] = len;
        }
      }
      for (int jj = threadIdx.x; jj < ncol; jj += blockDim.x) {
        T a = (T)0;
        const T* w = Wm + (size_t)jj * ldw_e;
        for (int i = 0; i < len; ++i) a += w[i] * w[i];
        const double sv = (double)sqrt(a) / scl;   // singular value of the unscaled C
        if (!(sv >= 0.0) || isinf(sv)) { s_sig[jj] = -1.0; flag(status, ST_NAN); }   // orders last
        else s_sig[jj] = sv;
      }
      __syncthreads();
      for (int jj = threadIdx.x; jj < ncol; jj += blockDim.x) {
        int rank = 0;
        const double sj = s_sig[jj];
        for (int o = 0; o < ncol; ++o) {
          const double so = s_sig[o];
          rank += (so > sj) || (so == sj && o < jj);
        }
        s_perm[rank] = jj;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        // smallest r in [1, min(chi, ncol)] with discarded tail <= delta (FP64 tail)
        const int rmax = imin(J.chi, ncol);
        double tail2 = 0.0;
        int rr = rmax;
        for (int p = ncol - 1; p >= 1; --p) {
          const double sv = s_sig[s_perm[p]];
          tail2 += sv * sv;
          s_tau[2 + p] = tail2;                  // tail starting at position p
        }
        for (int q = 1; q <= rmax; ++q) {
          const double t2 = (q < ncol) ? s_tau[2 + q] : 0.0;
          if (sqrt(t2) <= delta) { rr = q; break; }
        }
        if (rr > bond_cap(L, J.dst.cap, k)) { s_bad = 1; rr = bond_cap(L, J.dst.cap, k); }
        s_rank = rr;
        if (J.discard && rr < ncol) atomicAdd(J.discard, s_tau[2 + rr]);   // squared discarded tail
        flops += svd_flops(m, n);
        if (lc && lc->counters) atomicAdd(&lc->counters[2], 1);
      }
      __syncthreads();
      if (s_bad) { if (threadIdx.x == 0) flag(status, ST_CAPACITY); return; }
      r = s_rank;
      // outputs: core k = V^T[:r] (r x n) into dst; US (m x r) into scratch
      for (int idx = threadIdx.x; idx < r * n; idx += blockDim.x) {
        const int jr = idx / n, c = idx % n;
        const int pj = s_perm[jr];
        T v;
        if (trans) {
          v = Vm[(size_t)pj * ldv_e + c];
        } else {
          const T sg = (T)(s_sig[pj] * scl);       // norm of the scaled column
          v = sg > (T)0 ? Wm[(size_t)pj * ldw_e + c] / sg : (T)(c == jr ? 1 : 0);
        }
        out[idx] = v;
      }
      for (int idx = threadIdx.x; idx < m * r; idx += blockDim.x) {
        const int i = idx / r, jr = idx % r;
        const int pj = s_perm[jr];
        US[idx] = trans ? Wm[(size_t)pj * ldw_e + i] * (T)(1.0 / scl)
                        : Vm[(size_t)pj * ldv_e + i] * (T)s_sig[pj];
      }
      if (threadIdx.x == 0) J.dst.ranks[k] = r;
      __syncthreads();
    }
    // ---- sign gauge of the kept singular pairs: each row of V^T gets a
    // positive inner product with the probe weights frac((c+1) g) + 1/4,
    // g = 0.618..., a generic positive vector (rows with tied entries are
    // common in structured fields).  Contracted results do not depend on the
    // gauge; the randomized sample of the next step does.
    __syncthreads();
    {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int jr = warp; jr < r; jr += nw) {
        T* row = out + (size_t)jr * n;
        double dot = 0.0;
        for (int c = lane; c < n; c += 32) {
          const double x = (double)(c + 1) * 0.6180339887498949;
          dot += (double)row[c] * (x - floor(x) + 0.25);
        }
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        __syncwarp();
        if (dot < 0.0) {
          for (int c = lane; c < n; c += 32) row[c] = -row[c];
          for (int i = lane; i < m; i += 32) US[(size_t)i * r + jr] = -US[(size_t)i * r + jr];
        }
      }
    }
    __syncthreads();
    // ---- spectrum log: (features of the previous step, rank kept now)
    if (J.log != nullptr && lc != nullptr) {
      const int nsv = done ? imin(lsamp, TN_SPEC) : imin(ncol, TN_SPEC);
      if (threadIdx.x == 0 && lc->dataset != nullptr && J.log->valid[k]) {
        const int slot = atomicAdd(lc->dataset_count, 1);
        if (slot < lc->dataset_cap) {
          float* row = lc->dataset + (size_t)slot * (MLP_IN + 1);
          for (int q = 0; q < TN_SPEC; ++q) row[q] = J.log->spec[k][q];
          row[16] = (float)k / (float)L;
          row[17] = lc->step ? fminf((float)(*lc->step) / 1000.f, 1.f) : 0.f;
          row[18] = (float)r / (float)J.chi;
        }
      }
      __syncthreads();
      if (threadIdx.x < TN_SPEC) {
        const double s0 = s_sig[s_perm[0]];
        const double sv = threadIdx.x < nsv ? s_sig[s_perm[threadIdx.x]] : 0.0;
        J.log->spec[k][threadIdx.x] = (s0 > 0.0 && sv > 0.0) ? (float)log10(fmax(sv / s0, 1e-20)) : -20.f;
      }
      if (threadIdx.x == 0) { J.log->label[k] = r; J.log->valid[k] = 1; }
      __syncthreads();
    }
    // C' = Q_{k-1} (2 q_{k-1} x m) * US (m x r)
    const int rows = 2 * s_q[k - 1];
    const T* Qp = scr + J.lay.q_off[k - 1];
    pc.lap(PH_SVD_OUT);
    cta_gemm<T>(rows, r, m, Qp, m, US, r, C, r, false);
    if (threadIdx.x == 0) flops += 2.0 * rows * m * r;
    pc.lap(PH_GEMM_C);
    rnext = r;
  }
  // core 0 = C (1 x 2 x r_1)
  {
    T* out = (T*)J.dst.base;
    for (int idx = threadIdx.x; idx < 2 * rnext; idx += blockDim.x) out[idx] = C[idx];
    if (threadIdx.x == 0) {
      J.dst.ranks[0] = 1;
      J.dst.ranks[L] = 1;
      if (ctr) {
        atomicAdd(&ctr[C_ROUND], flops);
        for (int p = 0; p < PH_COUNT; ++p) atomicAdd(&ctr[C_COUNT + p], pc.acc[p]);
      }
    }
  }
}

// Worker CTA (rank > 0 of a cluster): joins the leader's FP64 Jacobi runs
// until the leader sends the exit command or a wait runs out.
template <typename T>
__device__ void round_worker(const RoundJob& J, int L_arg, ClusterCtx& cc) {
  T* scr = (T*)J.scratch;
  double* Wm = (double*)(scr + J.lay.jw64_off);
  double* Vm = (double*)(scr + J.lay.jv64_off);
  const int L = J.L > 0 ? J.L : L_arg;
  for (;;) {
    if (!cl_sync(cc)) break;
    const volatile ClusterCmd* cmd = (const volatile ClusterCmd*)&cc.sh->cmd;
    const int op = cmd->op, ncol = cmd->ncol, len = cmd->len, maxsw = cmd->maxsw;
    const int m = cmd->m, n = cmd->n, k = cmd->k;
    const double delta = cmd->delta, scl = cmd->scl;
    __syncthreads();
    if (op == 1) {
      jacobi64_cluster(cc, Wm, jacobi_ld<double>(len), Vm, jacobi_ld<double>(ncol), ncol, len, maxsw);
    } else if (op == 2) {
      int sw = 0;
      bool noconv = false;
      svd64_rows<T>(cc, J, L, k, m, n, scl, delta, maxsw, &sw, &noconv);
    } else {
      break;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) round_kernel(const RoundJob* __restrict__ jobs, int L_arg,
                                                   int n_bits_arg, const T* __restrict__ masks_arg,
                                                   const double* __restrict__ scal_arg,
                                                   int* __restrict__ status,
                                                   double* __restrict__ ctr,
                                                   const LearnCtx* __restrict__ lc) {
  __shared__ ClusterShared s_cl;
  ClusterCtx cc;
  const RoundJob& J = jobs[blockIdx.x / cl_size()];
  cl_init(cc, &s_cl, status, J.wait_ns > 0 ? J.wait_ns : 5000000000LL);
  if (cc.rank == 0) {
    round_job_body<T>(J, L_arg, n_bits_arg, masks_arg, scal_arg, status, ctr, lc, cc);
    cl_command(cc, 0, 0, 0, 0);
  } else {
    round_worker<T>(J, L_arg, cc);
  }
  cl_exit(cc);
}

template <typename T>
void launch_round(const RoundJob* d_jobs, int njobs, int L, int n_bits, const T* d_masks,
                  const double* d_scal, int* d_status, cudaStream_t st, double* d_ctr,
                  const LearnCtx* d_learn, int cluster) {
  if (njobs <= 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(round_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)round_smem_bytes());
    cudaFuncSetAttribute(round_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    attr_set = true;
  }
  if (cluster <= 1) {
    round_kernel<T><<<njobs, RT, round_smem_bytes(), st>>>(d_jobs, L, n_bits, d_masks, d_scal,
                                                           d_status, d_ctr, d_learn);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * cluster, 1, 1);
  cfg.blockDim = dim3(RT, 1, 1);
  cfg.dynamicSmemBytes = round_smem_bytes();
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, round_kernel<T>, d_jobs, L, n_bits, d_masks, d_scal, d_status, d_ctr, d_learn);
}

// Resident clusters of P CTAs (1 <= P <= 16) of the rounding kernel on the
// current device; the table is queried once per device.
template <typename T>
int round_cluster_resident(int P) {
  static int cached_dev = -1;
  static int max_active[CL_MAX + 1];
  if (P < 1 || P > CL_MAX) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev != cached_dev) {
    cudaFuncSetAttribute(round_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)round_smem_bytes());
    cudaFuncSetAttribute(round_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int q = 1; q <= CL_MAX; ++q) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(q, 1, 1);
      cfg.blockDim = dim3(RT, 1, 1);
      cfg.dynamicSmemBytes = round_smem_bytes();
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = q;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, round_kernel<T>, &cfg) != cudaSuccess) n = 0;
      max_active[q] = n;
    }
    cudaGetLastError();
    cached_dev = dev;
  }
  return max_active[P];
}

template <typename T>
int round_cluster_size(int njobs, int cap) {
  // the largest cluster at which every job of the launch is resident at once
  // (the FP64 Jacobi scales with the SMs of its cluster)
  for (int P = imin(cap, CL_MAX); P >= 2; --P)
    if (round_cluster_resident<T>(P) >= njobs) return P;
  return 1;
}

template void launch_round<float>(const RoundJob*, int, int, int, const float*, const double*,
                                  int*, cudaStream_t, double*, const LearnCtx*, int);
template void launch_round<double>(const RoundJob*, int, int, int, const double*,
                                   const double*, int*, cudaStream_t, double*, const LearnCtx*, int);
template int round_cluster_size<float>(int, int);
template int round_cluster_size<double>(int, int);
template int round_cluster_resident<float>(int);
template int round_cluster_resident<double>(int);

}  // namespace tn

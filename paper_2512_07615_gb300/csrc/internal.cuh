// Internal declarations of libtnlbm: flat MPS layout, rounding/fit job
// descriptors, status codes and small device helpers.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/tnlbm.h"

#define TN_MAXL 32     // sites per MPS (n_bits <= 10 -> L <= 30)
#define TN_MAXT 40     // terms per rounding job

namespace tn {

// ------------------------------------------------------------ status word
// Kernels never trap: they record a code in a device status word and return.
enum : int {
  ST_OK = 0,
  ST_CAPACITY = 1,   // a realised bond exceeded a buffer capacity
  ST_NOCONV = 2,     // Jacobi sweep limit reached
  ST_NAN = 4,        // non-finite value seen
  ST_TIMEOUT = 8     // bounded wait ran out
};
// algorithmic FLOP counters per kernel class (profiling only; nullable)
enum : int { C_ROUND = 0, C_FIT_GEMM = 1, C_FIT_QR = 2, C_FIT_MISC = 3, C_RHO0 = 4, C_COPY = 5, C_ZIPUP = 6,
             C_COUNT = 7 };
// phases of the rounding kernel (cycles of thread 0, summed over jobs), stored
// after the FLOP counters: terms, R*W GEMM, QR, Jacobi, SVD outputs, Q*US GEMM
// slots 6..9: Jacobi sweeps, SVD count, Jacobi cycles and count of SVDs in
// global memory; 10: algorithmic FLOPs of the FP64 centre SVDs (Golub-Kahan
// count); 11: FP64 FLOPs the cluster Jacobi executed (rotations, inner
// products, norms); 12..16: cycles of the leader's FP64 cluster Jacobi
// sweeps spent in the column norms (with their exchange), forming and sending
// the pair inner products, waiting for the other CTAs' parts, the angles, and
// the rotations; for FP32 data, 17: cycles of the leader's FP32 sweeps, 18: of
// the Newton-Schulz step, 19: of the product X V, 20: the FP32 sweeps; 21:
// rounds of the FP64 cluster sweeps
enum : int { PH_TERMS = 0, PH_GEMM_M = 1, PH_QR = 2, PH_JACOBI = 3, PH_SVD_OUT = 4, PH_GEMM_C = 5,
             PH_SVD64_FLOPS = 10, PH_SVD64_EXEC = 11, PH_RX_NORM = 12, PH_RX_DOT = 13, PH_RX_WAIT = 14,
             PH_RX_ANGLE = 15, PH_RX_ROT = 16, PH_J32 = 17, PH_NS = 18, PH_XV = 19, PH_SWEEPS32 = 20,
             PH_ROUNDS64 = 21, PH_COUNT = 22 };
// Precision modes: which run the centre SVDs in FP64 (FP32 data) and which
// put the fit's contractions on the tensor cores (0 none, 1 TF32, 2 BF16).
inline bool prec_svd64(int p) { return p == TNLBM_MIXED || p == TNLBM_BF16; }
inline int prec_tc(int p) { return p == TNLBM_TF32 ? 1 : p == TNLBM_BF16 ? 2 : 0; }
static constexpr int CTR_SIZE = 32;   // >= C_COUNT + PH_COUNT
// Householder QR with explicit Q of an m x n matrix, LAPACK-style counts
__host__ __device__ inline double qr_flops(double m, double n) {
  const double k = m < n ? m : n, big = m < n ? n : m;
  return 4.0 * big * k * k - 4.0 / 3.0 * k * k * k;
}
// thin SVD with both singular-vector sets (Golub-Kahan-Reinsch count)
__host__ __device__ inline double svd_flops(double m, double n) {
  const double k = m < n ? m : n, big = m < n ? n : m;
  return 4.0 * big * k * k + 8.0 * k * k * k;
}
// status buffers hold STATUS_INTS ints: [0] flags, [1] diag taken, [2..5] where
static constexpr int STATUS_INTS = 8;

__host__ __device__ inline int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

// bond capacity of a flat MPS: 1 at the two ends, cap inside (exactly formed
// sums, products and MPO applications may exceed 2^k near the ends)
__host__ __device__ inline int bond_cap(int L, int cap, int k) {
  return (k == 0 || k == L) ? 1 : cap;
}

__host__ __device__ inline size_t core_offset(int L, int cap, int k) {
  size_t off = 0;
  for (int j = 0; j < k; ++j)
    off += (size_t)bond_cap(L, cap, j) * 2 * (size_t)bond_cap(L, cap, j + 1);
  return off;
}

__host__ __device__ inline size_t mps_size(int L, int cap) { return core_offset(L, cap, L); }

// A device MPS in the flat layout.
struct MpsRef {
  void* base;      // T*
  int* ranks;      // [L+1]
  int cap;
};

// ------------------------------------------------------------ rounding jobs
enum TermKind : int { T_PLAIN = 0, T_SHIFT = 1, T_MASK1 = 2, T_KRON = 3, T_ONES = 4 };

struct Term {
  int kind;
  int axis, offset, cyclic;   // SHIFT
  double coef;
  int coef_slot;              // -1, or index of a device scalar multiplying coef
  int mask_id;                // MASK1: index into the job table's mask vectors
  MpsRef x, y;
};

// Scratch partition of one rounding job (elements of T), same on host and device.
struct RoundLayout {
  size_t q_off[TN_MAXL + 1];  // left-orthogonal cores of the QR sweep
  size_t w_off, m_off, r_off, c_off, jw_off, jv_off, us_off, rz_off, qw_off, total;
  size_t jw64_off, jv64_off;  // FP64 Jacobi matrices (in elements of T; = jw/jv for T = double)
};

// Learned-rank rounding state shared by all jobs of a launch (nullable parts).
// Spectrum log of one job: top-16 log10(s_i / s_0) per bond and the rank kept.
#define TN_SPEC 16
struct JobLog {
  float spec[TN_MAXL + 1][TN_SPEC];
  int label[TN_MAXL + 1];
  int valid[TN_MAXL + 1];
};
static constexpr int MLP_IN = 18, MLP_H = 64;
static constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;
struct LearnCtx {
  const void* omega;          // T*, fixed Gaussian test matrix (rows x ld)
  int omega_rows, omega_ld;
  int oversample;             // p
  int power;                  // power steps of the range finder
  float eta;                  // certificate: residual <= eta * err^2 at the chi cap
  float floor_rel;            // residuals below (floor_rel ||C||)^2 are round-off
  const __half* mlp;          // FP16 parameters (MLP_NPARAM), or null
  const int* step;            // device step counter (MLP feature)
  float* dataset;             // (features[18], label) rows, or null = no logging
  int* dataset_count;
  int dataset_cap;
  int* counters;              // [0] randomized accepted, [1] fell back, [2] full SVDs
};

struct RoundJob {
  int nterms;
  int chi;
  double eps;
  Term t[TN_MAXT];
  MpsRef dst;
  void* scratch;              // T*, RoundLayout::total elements
  int rw[TN_MAXL + 1];        // upper bounds of the wide (summed) bonds
  int qb[TN_MAXL + 1];        // upper bounds of the QR-sweep bonds
  RoundLayout lay;
  int materialize_only;       // 1: write the (single) term to dst, no rounding
  int rsvd_mode;              // 0 full SVD; 1 randomized at rsvd_k / targets; 2 MLP-predicted;
                              // 3 previous step's rank
  int rsvd_k;                 // fixed target rank (mode 1, when targets is null)
  const int* targets;         // per-bond target ranks (mode 1), device, or null
  JobLog* log;                // spectra of the previous step (modes 2 and logging), or null
  const void* masks;          // T*, rank-1 mask table of this job's simulation, or null = launch's
  const double* scal;         // scalars of this job's simulation, or null = launch's
  int L, n_bits;              // chain length and bits per axis of this job, or 0 = launch's
  double* discard;            // accumulator of squared discarded tails (device), or null
  int svd64;                  // 1: centre SVDs in FP64 on FP32 data (precision TNLBM_MIXED)
  int max_sweeps;             // Jacobi sweep limit (0 = 60)
  long long wait_ns;          // limit of every cross-CTA wait in ns (0 = 5 s)
};

// bound of one term's bond k from the capacities of its operands
__host__ __device__ inline int term_bond_bound(const Term& t, int L, int n_bits, int k) {
  switch (t.kind) {
    case T_ONES: return 1;
    case T_PLAIN:
    case T_MASK1: return bond_cap(L, t.x.cap, k);
    case T_KRON: return bond_cap(L, t.x.cap, k) * bond_cap(L, t.y.cap, k);
    case T_SHIFT: {
      int first = t.axis, last = t.axis + 3 * (n_bits - 1);
      int w = (k > first && k <= last) ? 2 : 1;
      return w * bond_cap(L, t.x.cap, k);
    }
  }
  return 0;
}

// Fill rw/qb bounds and the scratch layout of a job (host side); j.svd64 must
// be set before (it adds the FP64 Jacobi matrices for FP32 data).
void plan_round_job(RoundJob& j, int L, int n_bits, size_t elem_bytes);

// ------------------------------------------------------------ error helpers
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define TN_CUDA(call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return ::tn::cuda_fail(_e, #call); \
  } while (0)

// Error code and message of a device status block (STATUS_INTS ints).  A
// timed-out wait comes first: whatever follows it in the launch is unreliable
// (a CTA that gave up skips its work), so NaN or capacity flags raised after it
// are consequences.  A sweep limit alone is reported with where it happened.
inline int status_to_code(const int* st8) {
  const int st = st8[0];
  if (st & ST_TIMEOUT) { set_error("a bounded wait between the CTAs of a cluster ran out"); return TNLBM_E_TIMEOUT; }
  if (st & ST_NOCONV && !(st & (ST_CAPACITY | ST_NAN))) {
    char buf[160];
    snprintf(buf, sizeof(buf), "Jacobi SVD reached its sweep limit (job %d, site %d, %d columns of length %d)",
             st8[2], st8[3], st8[4], st8[5]);
    set_error(buf);
    return TNLBM_E_NOCONV;
  }
  if (st & ST_CAPACITY) { set_error("a realised bond exceeded a buffer capacity"); return TNLBM_E_CAPACITY; }
  if (st & ST_NAN) { set_error("non-finite values in a rounding"); return TNLBM_E_NAN; }
  if (st & ST_NOCONV) { set_error("Jacobi SVD reached its sweep limit"); return TNLBM_E_NOCONV; }
  return 0;
}

// ------------------------------------------------------------ launchers
// Rounding / materialisation of `njobs` jobs already resident on the device.
// cluster: CTAs per job (1 = one CTA; > 1 = a thread-block cluster whose CTAs
// share the FP64 Jacobi of the job; see round_cluster_size).
template <typename T>
void launch_round(const RoundJob* d_jobs, int njobs, int L, int n_bits,
                  const T* d_masks, const double* d_scal, int* d_status,
                  cudaStream_t st, double* d_ctr = nullptr, const LearnCtx* d_learn = nullptr,
                  int cluster = 1);
size_t round_smem_bytes();
// CTAs per job for a launch of njobs rounding jobs whose centre SVDs run in
// FP64: the largest cluster size (<= cap, <= 16) at which all njobs clusters
// are resident at once on the current device; 1 if none.
template <typename T>
int round_cluster_size(int njobs, int cap);
// how many clusters of P CTAs of the rounding kernel are resident at once on
// the current device (0: that size cannot launch)
template <typename T>
int round_cluster_resident(int P);
// increments the device step counter read by the rank model
void launch_learn_tick(int* d_step, cudaStream_t st);

}  // namespace tn

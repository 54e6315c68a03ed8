// Product-fit jobs (Sec. 2.3) and the other batched kernels' launchers.
#pragma once

#include "internal.cuh"

namespace tn {

struct FitJob {
  MpsRef A, B, C;          // A: candidate and output (set to B first)
  void* env_l;             // T*, (L+1) left environments, stride env_stride
  void* env_r;             // T*, (L+1) right environments
  size_t env_stride;
  void* x;                 // intermediates of the local contraction
  void* y;
  void* abuf;              // new centre core before the QR / LQ shift
  void* qscr;              // 4 * qscr_stride elements of QR scratch
  size_t qscr_stride;
};

void plan_fit_job(FitJob& j, int L, size_t* env_elems, size_t* x_elems, size_t* y_elems,
                  size_t* abuf_elems, size_t* q_elems);

// Zip-up product (zipup.cu): Z = the pass over B * C (left-orthogonal up to
// its last core); the caller rounds Z afterwards.  Z.cap >= chi, caps <= 512.
struct ZipJob {
  MpsRef B, C, Z;
  int chi;
  double eps;
  void* scratch;           // T*, zip_scratch_elems(L, B.cap, C.cap, Z.cap, sizeof(T))
};
size_t zip_scratch_elems(int L, int capB, int capC, int capZ, size_t esz);
// One launch (one CTA per job); returns the number of launches.
template <typename T>
int run_zipup(const ZipJob* d_jobs, int njobs, int L, int* d_status, cudaStream_t st, double* d_ctr = nullptr);

// Eager-launch profiler: an event after every launch on one stream; the time
// between consecutive events is charged to the class of the launch.
struct Prof {
  cudaStream_t st = nullptr;
  double* d_ctr = nullptr;            // device FLOP counters [C_COUNT]
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> cls;
  void begin() { cudaEventCreate(&start); cudaEventRecord(start, st); }
  void mark(int c) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    ev.push_back(e);
    cls.push_back(c);
  }
  // ms[c], launches[c]; destroys the events
  void collect(double* ms, int* launches) {
    cudaEventSynchronize(ev.empty() ? start : ev.back());
    cudaEvent_t prev = start;
    for (size_t i = 0; i < ev.size(); ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, prev, ev[i]);
      ms[cls[i]] += t;
      launches[cls[i]] += 1;
      prev = ev[i];
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    cudaEventDestroy(start);
    ev.clear();
    cls.clear();
  }
};

// tc: the GEMM stages on SIMT cores (TC_NONE) or on the tensor cores with
// TF32 (tcgen05 kind::tf32) or BF16 (kind::f16) operands; float storage only
enum : int { TC_NONE = 0, TC_TF32 = 1, TC_BF16 = 2 };
template <typename T>
int run_fit(const FitJob* d_jobs, const std::vector<FitJob>& hj, int L, int sweeps, int* d_status,
            cudaStream_t st, Prof* prof = nullptr, int tc = TC_NONE);

// ---- misc.cu
// out[b] = <X_b, 1> for MPS refs in device memory
template <typename T>
void launch_inner_ones(const MpsRef* d_refs, int n, int L, double* d_out, cudaStream_t st);

// rho_0 = <rho,1> / n_fluid and the scalar slots used by the Taylor 1/rho terms
// scalars of a step: rho_0 and its powers (Sec. 3.2), and per face (x-, x+, y-,
// y+, z-, z+) the inlet velocity u_b as set by the host (SC_UBRAW + 3 face + d)
// and rho_0 u_b (SC_UB + 3 face + d), the coefficient scale of Eq. boundaries2
enum ScalSlot : int { SC_NEG_RHO0 = 0, SC_INV1 = 1, SC_INV2 = 2, SC_INV3 = 3, SC_RHO0 = 4, SC_UB = 8,
                      SC_UBRAW = 26, SC_COUNT = 44 };
template <typename T>
void launch_rho0(const MpsRef* d_rho, int L, double n_fluid, double* d_scal, cudaStream_t st);

// Mass correction: mass[i] = <X_i, 1> for the n MPS (one CTA each), then every
// X_i's core 0 is scaled by mass0[0] / sum_i mass[i].
template <typename T>
void launch_mass_fix(const MpsRef* d_refs, int n, int L, double* d_mass, const double* d_mass0,
                     cudaStream_t st);

// copy MPS src[b] -> dst[b] (cores and bonds)
template <typename T>
void launch_copy(const MpsRef* d_src, const MpsRef* d_dst, int n, int L, cudaStream_t st);

// dense[x][y][z] = contraction of X (host-known ranks not needed)
template <typename T>
int contract_dense(const MpsRef& X, int n_bits, T* d_dense, void* d_scratch, size_t scratch_bytes,
                   cudaStream_t st);
size_t contract_scratch_bytes(int n_bits, int cap, size_t elem);
// plane coordinate[axis] = index of X, out[u * N + v] (the two other axes in order)
size_t plane_scratch_bytes(int n_bits, int axis, int cap);
template <typename T>
int contract_plane_f64(const MpsRef& X, int n_bits, int axis, int index, double* d_plane, void* d_scratch,
                       size_t scratch_bytes, cudaStream_t st);
template <typename T>
int contract_dense_f64(const MpsRef& X, int n_bits, double* d_dense, void* d_scratch, size_t scratch_bytes,
                       cudaStream_t st);

// accumulate rho += f, j += c f (double) from a dense population
template <typename T>
void launch_accum_moments(const T* d_f, size_t ncell, double* rho, double* jx, double* jy,
                          double* jz, int cx, int cy, int cz, int first, cudaStream_t st);
template <typename T>
void launch_cast_double(const T* src, size_t n, double* dst, cudaStream_t st);
void launch_velocity(size_t ncell, const double* rho, double* jx, double* jy, double* jz,
                     const double* mask, double fx, double fy, double fz, cudaStream_t st);

// TT-SVD of a dense device field (FP64 Gram matrices); host-synchronous.
template <typename T>
int tt_svd_dense(const T* d_dense_xyz, int n_bits, T* d_dst, int* d_dst_ranks, int dst_cap,
                 int chi_max, double eps, int* d_status, cudaStream_t st);

}  // namespace tn

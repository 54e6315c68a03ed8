// tnlbm_lincomb_round_noalloc: the rounded linear combination of
// tnlbm_lincomb_round without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// rounding: code whose device memory is entirely reserved up front by a pool
// allocator (a cudaMalloc there fails or fragments the pool), and code that must
// not stall the device (cudaFree synchronises the whole device).  For them this
// entry point keeps every buffer it needs in fixed arrays that live in the
// library's own device memory for as long as the library is loaded:
//   scratch     TN_NOALLOC_SCRATCH_BYTES (16 MiB), the per-job QR/SVD workspace
//   job table   TN_NOALLOC_MAX_JOBS (64) rounding jobs
//   mask table  TN_NOALLOC_MAX_MASKS (64) rank-1 masks
//   scalars and a status word
// Every GPU that loads the library holds these arrays until the process exits.
// All calls share them: a call overwrites what the previous one left, so calls
// whose GPU work overlaps (different streams, or different host threads) race.
// The status word and scalars are cleared at the start of every call.
//
// The device addresses of the arrays are looked up with cudaGetSymbolAddress on
// the first call made on each device (with that device current).  That first
// call therefore does a little set-up work and should come before any stream
// capture that includes this entry point.
#include <cstring>

#include "fit.cuh"
#include "internal.cuh"

#define TN_NOALLOC_SCRATCH_BYTES (16u << 20)
#define TN_NOALLOC_MAX_JOBS 64
#define TN_NOALLOC_MAX_MASKS 64
#define TN_NOALLOC_MAX_DEVICES 64

namespace tn {

static __device__ __align__(256) unsigned char g_na_scratch[TN_NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) RoundJob g_na_jobs[TN_NOALLOC_MAX_JOBS];
static __device__ __align__(256) double g_na_masks[TN_NOALLOC_MAX_MASKS * TN_MAXL * 2];
static __device__ __align__(256) double g_na_scal[SC_COUNT];   // the full scalar table a rounding reads
static __device__ __align__(256) int g_na_status[STATUS_INTS];

struct NoallocPtrs {
  bool ready = false;
  unsigned char* scratch = nullptr;
  RoundJob* jobs = nullptr;
  double* masks = nullptr;
  double* scal = nullptr;
  int* status = nullptr;
};
static NoallocPtrs g_na_dev[TN_NOALLOC_MAX_DEVICES];
// host staging of the job and mask tables (fixed, like the device arrays)
static RoundJob g_na_hjobs[TN_NOALLOC_MAX_JOBS];
static double g_na_hmasks[TN_NOALLOC_MAX_MASKS * TN_MAXL * 2];

// Device addresses of the fixed arrays for the current device (set-up on the
// first call per device).
static int noalloc_ptrs(NoallocPtrs** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= TN_NOALLOC_MAX_DEVICES) {
    set_error("tnlbm_lincomb_round_noalloc: device index out of range");
    return TNLBM_E_ARG;
  }
  NoallocPtrs& p = g_na_dev[dev];
  if (!p.ready) {
    e = cudaGetSymbolAddress((void**)&p.scratch, g_na_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    e = cudaGetSymbolAddress((void**)&p.jobs, g_na_jobs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(jobs)");
    e = cudaGetSymbolAddress((void**)&p.masks, g_na_masks);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(masks)");
    e = cudaGetSymbolAddress((void**)&p.scal, g_na_scal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scal)");
    e = cudaGetSymbolAddress((void**)&p.status, g_na_status);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(status)");
    p.ready = true;
  }
  *out = &p;
  return 0;
}

template <typename T>
static int noalloc_impl(int n_bits, int batch, int nterms, const tnlbm_term* terms, void* const* dst,
                        int* const* dst_ranks, int dst_cap, int chi, double eps, cudaStream_t st) {
  const int L = 3 * n_bits;
  if (batch > TN_NOALLOC_MAX_JOBS) {
    set_error("tnlbm_lincomb_round_noalloc: batch exceeds the fixed job table (64 jobs)");
    return TNLBM_E_ARG;
  }
  NoallocPtrs* P = nullptr;
  int rc = noalloc_ptrs(&P);
  if (rc) return rc;
  RoundJob* jobs = g_na_hjobs;
  T* masks = (T*)g_na_hmasks;                // masks stored in the job's element type
  int nmask = 0;
  for (int b = 0; b < batch; ++b) {
    RoundJob& j = jobs[b];
    std::memset(&j, 0, sizeof(RoundJob));
    j.nterms = nterms;
    j.chi = chi;
    j.eps = eps;
    j.dst.base = dst[b];
    j.dst.ranks = dst_ranks[b];
    j.dst.cap = dst_cap;
    for (int t = 0; t < nterms; ++t) {
      const tnlbm_term& in = terms[(size_t)b * nterms + t];
      Term& tm = j.t[t];
      tm.kind = in.kind;
      tm.coef = in.coef;
      tm.coef_slot = -1;
      tm.axis = in.axis;
      tm.offset = in.offset;
      tm.cyclic = in.cyclic;
      tm.mask_id = -1;
      if (in.kind < 0 || in.kind > 4) { set_error("bad term kind"); return TNLBM_E_ARG; }
      if (in.kind != T_ONES) {
        if (!in.x || !in.x_ranks || in.x_cap < 1) { set_error("term operand missing"); return TNLBM_E_ARG; }
        tm.x.base = (void*)in.x; tm.x.ranks = (int*)in.x_ranks; tm.x.cap = in.x_cap;
      }
      if (in.kind == T_KRON) {
        if (!in.y || !in.y_ranks || in.y_cap < 1) { set_error("KRON needs y"); return TNLBM_E_ARG; }
        tm.y.base = (void*)in.y; tm.y.ranks = (int*)in.y_ranks; tm.y.cap = in.y_cap;
      }
      if (in.kind == T_SHIFT && (in.axis < 0 || in.axis > 2 || (in.offset != 1 && in.offset != -1))) {
        set_error("SHIFT needs axis in 0..2 and offset +-1");
        return TNLBM_E_ARG;
      }
      if (in.kind == T_MASK1) {
        if (!in.mask) { set_error("MASK1 needs mask vectors"); return TNLBM_E_ARG; }
        const int id = nmask;
        if (id >= TN_NOALLOC_MAX_MASKS) {
          set_error("tnlbm_lincomb_round_noalloc: more rank-1 masks than the fixed table holds (64)");
          return TNLBM_E_ARG;
        }
        tm.mask_id = id;
        ++nmask;
        for (int k = 0; k < TN_MAXL * 2; ++k) masks[(size_t)id * TN_MAXL * 2 + k] = (T)1;
        for (int k = 0; k < L; ++k)
          for (int s2 = 0; s2 < 2; ++s2) masks[(size_t)id * TN_MAXL * 2 + 2 * k + s2] = (T)in.mask[2 * k + s2];
      }
    }
    plan_round_job(j, L, n_bits, sizeof(T));
  }
  // scratch partition inside the fixed array
  size_t off = 0;
  for (int b = 0; b < batch; ++b) {
    RoundJob& j = jobs[b];
    const size_t bytes = ((j.lay.total * sizeof(T)) + 255) & ~(size_t)255;
    if (off + bytes > TN_NOALLOC_SCRATCH_BYTES) {
      set_error("tnlbm_lincomb_round_noalloc: the rounding needs more than the fixed 16 MiB scratch; "
                "use tnlbm_lincomb_round or fewer / smaller jobs");
      return TNLBM_E_ARG;
    }
    j.scratch = P->scratch + off;
    off += bytes;
  }
  TN_CUDA(cudaMemcpyAsync(P->jobs, jobs, batch * sizeof(RoundJob), cudaMemcpyHostToDevice, st));
  if (nmask > 0)
    TN_CUDA(cudaMemcpyAsync(P->masks, masks, (size_t)nmask * TN_MAXL * 2 * sizeof(T),
                            cudaMemcpyHostToDevice, st));
  TN_CUDA(cudaMemsetAsync(P->scal, 0, SC_COUNT * sizeof(double), st));
  TN_CUDA(cudaMemsetAsync(P->status, 0, STATUS_INTS * sizeof(int), st));
  launch_round<T>(P->jobs, batch, L, n_bits, (const T*)P->masks, P->scal, P->status, st);
  TN_CUDA(cudaGetLastError());
  // the status word is read on the caller's stream, which alone is waited for
  int h[STATUS_INTS] = {0};
  TN_CUDA(cudaMemcpyAsync(h, P->status, sizeof(h), cudaMemcpyDeviceToHost, st));
  TN_CUDA(cudaStreamSynchronize(st));
  return status_to_code(h);
}

}  // namespace tn

extern "C" int tnlbm_lincomb_round_noalloc(int precision, int n_bits, int batch, int nterms,
                                           const tnlbm_term* terms, void* const* dst,
                                           int* const* dst_ranks, int dst_cap, int chi_max,
                                           double eps, void* stream) {
  if (n_bits < 1 || n_bits > 10 || batch < 0 || nterms < 1 || nterms > TN_MAXT || !terms || !dst ||
      !dst_ranks || chi_max < 1 || chi_max > dst_cap || chi_max > 512 || eps < 0 ||
      (precision != TNLBM_FP64 && precision != TNLBM_FP32)) {
    tn::set_error("bad arguments to tnlbm_lincomb_round_noalloc");
    return TNLBM_E_ARG;
  }
  if (batch == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == TNLBM_FP64
             ? tn::noalloc_impl<double>(n_bits, batch, nterms, terms, dst, dst_ranks, dst_cap, chi_max, eps, st)
             : tn::noalloc_impl<float>(n_bits, batch, nterms, terms, dst, dst_ranks, dst_cap, chi_max, eps, st);
}

// Masks combined on separate length scales (App. D): an inner geometry on a
// 2^k grid per axis repeated where an outer mask on a 2^l grid per axis is
// one.  In scale order the combined MPS is the outer MPS followed by the inner
// one, so each part is compressed on its own small grid (TT-SVD, the mask
// builder of Eq. svd-comp) and the cores are concatenated; no dense field of
// the combined resolution is ever formed.
#include "fit.cuh"

namespace tn {

// core k of the combined MPS (L = Lo + Li sites, capacity cap) from core k of
// the outer MPS (k < Lo) or core k - Lo of the inner one; one CTA per site
template <typename T>
__global__ void concat_cores_kernel(const T* __restrict__ outer, const int* __restrict__ ro, int Lo,
                                    const T* __restrict__ inner, const int* __restrict__ ri, int Li, int cap,
                                    T* __restrict__ dst, int* __restrict__ rd) {
  const int k = blockIdx.x, L = Lo + Li;
  const bool is_outer = k < Lo;
  const int kk = is_outer ? k : k - Lo;
  const int Ls = is_outer ? Lo : Li;
  const int* r = is_outer ? ro : ri;
  const T* src = (is_outer ? outer : inner) + core_offset(Ls, cap, kk);
  T* out = dst + core_offset(L, cap, k);
  const int n = r[kk] * 2 * r[kk + 1];
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = src[i];
  if (threadIdx.x == 0) {
    rd[k] = r[kk];
    if (k == L - 1) rd[L] = 1;
  }
}

template <typename T>
static int mask_product_impl(int n_outer, const T* outer, int n_inner, const T* inner, T* dst, int* dst_ranks,
                             int cap, int chi, double eps, cudaStream_t st) {
  const int Lo = 3 * n_outer, Li = 3 * n_inner;
  T *bo = nullptr, *bi = nullptr;
  int *ro = nullptr, *ri = nullptr, *ds = nullptr;
  auto cleanup = [&]() { cudaFree(bo); cudaFree(bi); cudaFree(ro); cudaFree(ri); cudaFree(ds); };
  if (cudaMalloc(&bo, mps_size(Lo, cap) * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&bi, mps_size(Li, cap) * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&ro, (Lo + 1) * sizeof(int)) != cudaSuccess || cudaMalloc(&ri, (Li + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ds, STATUS_INTS * sizeof(int)) != cudaSuccess) {
    cleanup();
    set_error("out of device memory");
    return TNLBM_E_OOM;
  }
  cudaMemsetAsync(ds, 0, STATUS_INTS * sizeof(int), st);
  int rc = tt_svd_dense<T>(outer, n_outer, bo, ro, cap, chi, eps, ds, st);
  if (!rc) rc = tt_svd_dense<T>(inner, n_inner, bi, ri, cap, chi, eps, ds, st);
  if (!rc) {
    concat_cores_kernel<T><<<Lo + Li, 128, 0, st>>>(bo, ro, Lo, bi, ri, Li, cap, dst, dst_ranks);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "tnlbm_mask_product");
  }
  if (!rc) {
    int h[STATUS_INTS] = {0};
    cudaError_t e = cudaMemcpy(h, ds, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "tnlbm_mask_product status");
    else if (h[0] & ST_CAPACITY) { set_error("a mask bond exceeded the capacity"); rc = TNLBM_E_CAPACITY; }
    else if (h[0]) { set_error("mask TT-SVD failed on the device"); rc = TNLBM_E_NOCONV; }
  }
  cleanup();
  return rc;
}

}  // namespace tn

extern "C" int tnlbm_mask_product(int precision, int n_outer, const void* outer_dense, int n_inner,
                                  const void* inner_dense, void* dst, int* dst_ranks, int dst_cap, int chi_max,
                                  double eps, void* stream) {
  if (n_outer < 1 || n_inner < 1 || n_outer + n_inner > 10 || !outer_dense || !inner_dense || !dst ||
      !dst_ranks || dst_cap < 1 || chi_max < 1 || chi_max > dst_cap || 2 * chi_max > 1024 || eps < 0 ||
      (precision != TNLBM_FP64 && precision != TNLBM_FP32)) {
    tn::set_error("bad arguments to tnlbm_mask_product");
    return TNLBM_E_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return precision == TNLBM_FP64
             ? tn::mask_product_impl<double>(n_outer, (const double*)outer_dense, n_inner,
                                             (const double*)inner_dense, (double*)dst, dst_ranks, dst_cap,
                                             chi_max, eps, st)
             : tn::mask_product_impl<float>(n_outer, (const float*)outer_dense, n_inner, (const float*)inner_dense,
                                            (float*)dst, dst_ranks, dst_cap, chi_max, eps, st);
}

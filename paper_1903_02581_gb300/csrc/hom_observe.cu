// Launchers of the probability-map and slice kernels (hom_observe.cuh) for
// both precisions.
#include <cuda_runtime.h>

#include "hom_internal.h"
#include "hom_observe.cuh"

namespace hom {

template <typename T>
cudaError_t launch_marginal(const void* psi, int n, int batch, double* out, cudaStream_t s) {
  using C = typename Cx<T>::type;
  if (n < 1 || batch < 1) return cudaErrorInvalidValue;
  marginal_rows<C><<<(unsigned)((size_t)batch * n), OBS_THREADS, 0, s>>>(static_cast<const C*>(psi), n, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather(const void* psi, int n, int row0, int rstride, int nrows, int col0, int cstride, int ncols,
                          double2* out, double* mag2, cudaStream_t s) {
  using C = typename Cx<T>::type;
  if (nrows < 1 || ncols < 1) return cudaErrorInvalidValue;
  const long long total = (long long)nrows * ncols;
  gather_slice<C><<<(unsigned)((total + OBS_THREADS - 1) / OBS_THREADS), OBS_THREADS, 0, s>>>(
      static_cast<const C*>(psi), n, row0, rstride, nrows, col0, cstride, ncols, out, mag2);
  return cudaGetLastError();
}

template cudaError_t launch_marginal<float>(const void*, int, int, double*, cudaStream_t);
template cudaError_t launch_marginal<double>(const void*, int, int, double*, cudaStream_t);
template cudaError_t launch_gather<float>(const void*, int, int, int, int, int, int, int, double2*, double*,
                                          cudaStream_t);
template cudaError_t launch_gather<double>(const void*, int, int, int, int, int, int, int, double2*, double*,
                                           cudaStream_t);

}  // namespace hom

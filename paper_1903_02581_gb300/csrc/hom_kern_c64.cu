// Kernels of libhom in complex64 (FP32 arithmetic, FP64 reductions): the
// transposing pass and every kernel but the in-place passes.
#define HOM_T float
#define HOM_WIDE 1
#define HOM_PART 2
#include "hom_kern.inc"

namespace hom {
cudaError_t launch_reduce(const double* partial, int tiles_per_sim, int batch, double* out, cudaStream_t s) {
  reduce_partials<NPART><<<batch, 256, 0, s>>>(partial, tiles_per_sim, out);
  return cudaGetLastError();
}

cudaError_t launch_adj_reduce(const double* slot, int nk, int batch, double* out, int stride, cudaStream_t s) {
  if (nk == 1) adj_reduce<1><<<batch, 256, 0, s>>>(slot, ADJ_BLOCKS, out, stride);
  else adj_reduce<2><<<batch, 256, 0, s>>>(slot, ADJ_BLOCKS, out, stride);
  return cudaGetLastError();
}
}  // namespace hom

// hom_internal.h -- launch interface between the C ABI (hom_api.cu) and the
// per-precision kernel translation units (hom_kern_c64.cu, hom_kern_c128.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "hom_pass.cuh"

namespace hom {

struct GeoInfo {
  int G;              // planes per CTA
  int NT;             // threads per CTA
  size_t smem;        // dynamic shared memory bytes
  int tiles_per_sim;  // CTAs per simulation
};

// Tile geometry of the row (col = false) or column (col = true) pass.
// G = 0 if (nx, ny) is not a supported size.
template <typename T> GeoInfo geo_info(int nx, int ny, bool col);

// Set the kernel attributes (dynamic shared memory, occupancy query) of the
// kinetic passes of a grid on the current device, so that later launches,
// including launches captured into a CUDA graph, make no attribute calls.
template <typename T> cudaError_t prepare_kinetic(int nx, int ny);
// The same for the in-place passes only (called by prepare_kinetic).
template <typename T> cudaError_t prepare_kinetic_rows(int nx, int ny);

// In-place pass on rows (kinetic_pass), variant 0 or 1 (see Geo).
template <typename T>
cudaError_t launch_kinetic(int nx, int ny, int variant, const PassArgs<typename Cx<T>::type>& a, int batch,
                           cudaStream_t s);

// Double in-place pass: two sandwiches with the potential phase a.p1m/a.p12m
// between them (see kinetic_pass), variant 0 or 1.
template <typename T>
cudaError_t launch_kinetic2(int nx, int ny, int variant, const PassArgs<typename Cx<T>::type>& a, int batch,
                            cudaStream_t s);

// Transposing pass (kinetic_pass_t), variant 0 or 1.
template <typename T>
cudaError_t launch_kinetic_t(int nx, int ny, int variant, const PassArgsT<typename Cx<T>::type>& a, int batch,
                             cudaStream_t s);

// out[b * n + r1] = sum over r2 of |psi[b][r1][r2]|^2 in FP64, for batch states
// of [n][n] (hom_observe.cuh).
template <typename T>
cudaError_t launch_marginal(const void* psi, int n, int batch, double* out, cudaStream_t s);

// out[i * ncols + j] (FP64 complex) and mag2 (|.|^2) of the elements
// psi[(row0 + i * rstride) * n + col0 + j * cstride] of one [n][n] state;
// either output may be null.
template <typename T>
cudaError_t launch_gather(const void* psi, int n, int row0, int rstride, int nrows, int col0, int cstride, int ncols,
                          double2* out, double* mag2, cudaStream_t s);

// dst = transpose of each [n][n] state of src (batch states).
template <typename T>
cudaError_t launch_transpose(const void* src, void* dst, int n, int batch, cudaStream_t s);

// Columns per transposed-store tile of the transposing pass of a grid (kernel
// variant 0 or 1) when it stores through the tensor memory accelerator, else 0.
template <typename T> int tma_store_width(int nx, int ny, int variant);

template <typename T>
cudaError_t launch_measure(int nx, int ny, bool col, const MeasureArgs<typename Cx<T>::type>& a, int batch,
                           cudaStream_t s);

template <typename T>
cudaError_t launch_slater(void* psi, const double2* pk, const double* coef, const int* exch, int b0, int nb,
                          int n, cudaStream_t s);

cudaError_t launch_reduce(const double* partial, int tiles_per_sim, int batch, double* out, cudaStream_t s);

// Adjoint gradient kernels (hom_adjoint.cuh); slots hold kAdjBlocks partial
// sums per simulation (times 2 for adj_accum).
constexpr int kAdjBlocks = 512;
template <typename T>
cudaError_t launch_adj_mask(const void* psi, void* lam, double* slot, int nx, int ny, int batch, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_accum(const void* psi, const void* lam, const double* dv, double* slot, double w, int nx,
                             int ny, int batch, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_delay(const void* lam, const double2* pk, const double2* dbeta, const double* cdc,
                             const int* exch, double* slot, int n, int batch, cudaStream_t s);
cudaError_t launch_adj_reduce(const double* slot, int nk, int batch, double* out, int stride, cudaStream_t s);

}  // namespace hom

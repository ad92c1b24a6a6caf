// hom_observe.cuh -- probability maps and slices of the two-particle state
// (captions of Fig. 2 and Fig. 3(b) and Sec. V of arXiv:1903.02581).
// The state is read in layout A, psi[b][r1][r2] with r = x * ny + y.
#pragma once

#include <cuda_runtime.h>

#include "hom_fft.cuh"

namespace hom {

constexpr int OBS_THREADS = 256;

// Unconditional probability of particle 1, before the dx dy factor:
// out[b * n + r1] = sum over r2 of |psi[b][r1][r2]|^2, in FP64.  One CTA per
// row; every thread sums a fixed strided subset and the CTA reduces in a
// fixed order, so the result does not depend on scheduling.
template <typename C>
__global__ void __launch_bounds__(OBS_THREADS) marginal_rows(const C* __restrict__ psi, int n,
                                                             double* __restrict__ out) {
  __shared__ double red[OBS_THREADS / 32];
  const size_t row = blockIdx.x;
  const C* p = psi + row * (size_t)n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += OBS_THREADS) {
    const C v = p[i];
    s = fma((double)v.x, (double)v.x, fma((double)v.y, (double)v.y, s));
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < OBS_THREADS / 32; ++w) t += red[w];
    out[row] = t;
  }
}

// Strided 2D gather of one simulation's state, widened to FP64:
// out[i * ncols + j] = psi[(row0 + i * rstride) * n + col0 + j * cstride], and
// mag2 (if not null) the squared modulus.  One thread per output element.
template <typename C>
__global__ void __launch_bounds__(OBS_THREADS) gather_slice(const C* __restrict__ psi, int n, int row0, int rstride,
                                                            int nrows, int col0, int cstride, int ncols,
                                                            double2* __restrict__ out, double* __restrict__ mag2) {
  const int k = blockIdx.x * OBS_THREADS + threadIdx.x;
  if (k >= nrows * ncols) return;
  const int i = k / ncols, j = k % ncols;
  const C v = psi[(size_t)(row0 + i * rstride) * n + col0 + (size_t)j * cstride];
  const double re = (double)v.x, im = (double)v.y;
  if (out) out[k] = make_double2(re, im);
  if (mag2) mag2[k] = fma(re, re, im * im);
}

}  // namespace hom

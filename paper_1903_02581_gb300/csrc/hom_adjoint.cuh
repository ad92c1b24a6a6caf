// hom_adjoint.cuh -- elementwise kernels of the adjoint gradient of the
// bunching probability (the loss L = <psi_N| M |psi_N> dV, M the indicator of
// x1, x2 on the same side, Eq. p_bunching of arXiv:1903.02581).
//
// The Strang step is a palindromic product of unitary factors, so its adjoint
// is the step with the opposite time step, S(dt)^dagger = S(-dt).  For a
// parameter theta of the single-particle potential,
//   dL/dtheta = 2 dt dV Im sum'_n <lambda_n| dV/dtheta |psi_n>
// (trapezoid weights 1/2 at n = 0 and n = N), lambda_N = M psi_N,
// lambda_n = S(-dt) lambda_{n+1}; for the centre of the second packet,
//   dL/ddelay = 2 dV Re <lambda_0| d psi_0 / d delay>.
// Every kernel runs on a fixed grid of ADJ_BLOCKS blocks per simulation
// (blockIdx.y = simulation) and each block adds into its own slot, so the
// sums are deterministic.
#pragma once

#include <cuda_runtime.h>

#include "hom_fft.cuh"

namespace hom {

constexpr int ADJ_BLOCKS = 512;
constexpr int ADJ_THREADS = 256;

__device__ __forceinline__ double adj_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// lambda = M psi; slot[b][blk] = sum over the block's points of M |psi|^2.
template <typename C>
__global__ void __launch_bounds__(ADJ_THREADS)
adj_mask(const C* __restrict__ psi, C* __restrict__ lam, double* __restrict__ slot, int nx, int ny) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const size_t n = (size_t)nx * ny, per = n * n;
  const C* p = psi + (size_t)b * per;
  C* l = lam + (size_t)b * per;
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const int r1 = (int)(i / n), r2 = (int)(i % n);
    const bool same = ((r1 / ny) < nx / 2) == ((r2 / ny) < nx / 2);
    const C v = p[i];
    if (same) {
      l[i] = v;
      s += cnorm2_d(v);
    } else {
      l[i] = C{0, 0};
    }
  }
  s = adj_block_sum(s, red);
  if (threadIdx.x == 0) slot[(size_t)b * gridDim.x + blockIdx.x] = s;
}

// slot[b][blk][k] += w * sum Im(conj(lambda) psi) (d_k(x1) + d_k(x2)), k = 0 (h), 1 (w);
// dv = [batch][2][nx] derivatives of V1 along x.
template <typename C>
__global__ void __launch_bounds__(ADJ_THREADS)
adj_accum(const C* __restrict__ psi, const C* __restrict__ lam, const double* __restrict__ dv,
          double* __restrict__ slot, double w, int nx, int ny) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const size_t n = (size_t)nx * ny, per = n * n;
  const C* p = psi + (size_t)b * per;
  const C* l = lam + (size_t)b * per;
  const double* dh = dv + (size_t)b * 2 * nx;
  const double* dw = dh + nx;
  double sh = 0.0, sw = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const int x1 = (int)(i / n) / ny, x2 = (int)(i % n) / ny;
    const C u = l[i], v = p[i];
    const double im = (double)u.x * (double)v.y - (double)u.y * (double)v.x;
    sh += im * (dh[x1] + dh[x2]);
    sw += im * (dw[x1] + dw[x2]);
  }
  sh = adj_block_sum(sh, red);
  sw = adj_block_sum(sw, red);
  if (threadIdx.x == 0) {
    double* o = slot + ((size_t)b * gridDim.x + blockIdx.x) * 2;
    o[0] += w * sh;
    o[1] += w * sw;
  }
}

// slot[b][blk] = sum Re(conj(lambda) dpsi0), with
// dpsi0 = dc u + c du, u = a(r1) be(r2) + s be(r1) a(r2), du = a(r1) dbe(r2) + s dbe(r1) a(r2).
template <typename C>
__global__ void __launch_bounds__(ADJ_THREADS)
adj_delay(const C* __restrict__ lam, const double2* __restrict__ pk, const double2* __restrict__ dbeta,
          const double* __restrict__ cdc, const int* __restrict__ exch, double* __restrict__ slot, int n) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const size_t per = (size_t)n * n;
  const C* l = lam + (size_t)b * per;
  const double2* al = pk + (size_t)b * 2 * n;
  const double2* be = al + n;
  const double2* db = dbeta + (size_t)b * n;
  const double c = cdc[2 * b], dc = cdc[2 * b + 1];
  const double s = (double)exch[b];
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const int r1 = (int)(i / n), r2 = (int)(i % n);
    const double2 a1 = al[r1], a2 = al[r2], b1 = be[r1], b2 = be[r2], d1 = db[r1], d2 = db[r2];
    double ur = a1.x * b2.x - a1.y * b2.y + s * (b1.x * a2.x - b1.y * a2.y);
    double ui = a1.x * b2.y + a1.y * b2.x + s * (b1.x * a2.y + b1.y * a2.x);
    double dr = a1.x * d2.x - a1.y * d2.y + s * (d1.x * a2.x - d1.y * a2.y);
    double di = a1.x * d2.y + a1.y * d2.x + s * (d1.x * a2.y + d1.y * a2.x);
    const double gr = dc * ur + c * dr, gi = dc * ui + c * di;
    const C v = l[i];
    acc += (double)v.x * gr + (double)v.y * gi;
  }
  acc = adj_block_sum(acc, red);
  if (threadIdx.x == 0) slot[(size_t)b * gridDim.x + blockIdx.x] = acc;
}

// out[b * stride + k] = sum over blocks of slot[b][blk][k], k < NK, fixed order.
template <int NK>
__global__ void adj_reduce(const double* __restrict__ slot, int blocks, double* __restrict__ out, int stride) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  constexpr int nk = NK;
  for (int k = 0; k < nk; ++k) {
    double s = 0.0;
    for (int t = threadIdx.x; t < blocks; t += blockDim.x) s += slot[((size_t)b * blocks + t) * nk + k];
    s = adj_block_sum(s, red);
    if (threadIdx.x == 0) out[b * stride + k] = s;
  }
}

}  // namespace hom

// hom_fft.cuh -- complex arithmetic and in-register DFTs for libhom kernels.
//
// The 2D Fourier transforms F_{x1,x2} and F_{y1,y2} of Eq. (evoloperat) of
// arXiv:1903.02581 are applied here one particle at a time as 1D DFTs along
// each axis (F_{x1,x2} = F_{x1} F_{x2}).  A line of length N <= 16 is
// transformed entirely in registers; longer lines are split N = N1 * N2 into
// two register passes with a twiddle between them (Cooley-Tukey), the second
// pass leaving the coefficients in digit-transposed order, which the phase
// tables and the inverse transform consume directly.
#pragma once

#include <cuda_runtime.h>

namespace hom {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

template <typename C> struct Re;
template <> struct Re<float2> { using type = float; };
template <> struct Re<double2> { using type = double; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
// FP32 complex add/subtract as one packed two-lane instruction (sm_100 family);
// each lane rounds to nearest exactly as the scalar add does (a + 1 * b is
// the exact sum before its one rounding).
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(1.0f, 1.0f), a);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C> __device__ __forceinline__ typename Re<C>::type cnorm2(C a) {
  return a.x * a.x + a.y * a.y;
}
// |a|^2 in FP64 (exact for an FP32 a: each square fits a double), for the
// FP64 reductions of the observables.
template <typename C> __device__ __forceinline__ double cnorm2_d(C a) {
  return fma((double)a.x, (double)a.x, (double)a.y * (double)a.y);
}
template <typename C> __device__ __forceinline__ C ldg(const C* p) { return __ldg(p); }

// cos and sin of 2*pi*j/16, j = 0..15 (exact values of the 16th roots of unity).
__device__ __forceinline__ constexpr double cos16(int j) {
  switch (j & 15) {
    case 0: return 1.0;
    case 1: case 15: return 0.92387953251128675613;   // cos(pi/8)
    case 2: case 14: return 0.70710678118654752440;   // cos(pi/4)
    case 3: case 13: return 0.38268343236508977173;   // cos(3pi/8)
    case 4: case 12: return 0.0;
    case 5: case 11: return -0.38268343236508977173;
    case 6: case 10: return -0.70710678118654752440;
    case 7: case 9: return -0.92387953251128675613;
    default: return -1.0;
  }
}
__device__ __forceinline__ constexpr double sin16(int j) { return cos16(j + 12); }

// v * (1 + d): a unit-modulus phase stored as its deviation d = w - 1 from 1.
// For the small phase angles of a split step, d carries the phase with full
// relative precision, so the rounded table has |1 + d| = 1 to far better than
// the precision of w itself.
template <typename C>
__device__ __forceinline__ C apply_delta(C v, C d) {
  return C{fma(v.x, d.x, fma(-v.y, d.y, v.x)), fma(v.x, d.y, fma(v.y, d.x, v.y))};
}
// In FP32 the correction t = v * d is formed first, at its own (small) scale,
// and added to v in one rounding.  The FMA chain above instead adds the
// second-order term v * d.x (|d.x| = 2 sin^2(theta/2)) to an already rounded
// value in a rounding of its own; where |v * d.x| is within a few ulps of v,
// as for the most occupied low-k modes at the time steps used, that rounding
// is biased with a sign set by the phase angle, the same every step, and the
// norm drifts by ~1e-8 per step.  With t added once, the rounding error is
// that of v + t, whose low bits vary over many ulps: no measurable drift.
template <>
__device__ __forceinline__ float2 apply_delta<float2>(float2 v, float2 d) {
  const float tr = fmaf(v.x, d.x, -(v.y * d.y));
  const float ti = fmaf(v.y, d.x, v.x * d.y);
  return __fadd2_rn(v, make_float2(tr, ti));
}

// s v (1 + d) from a table holding ds = s d, with s a power of two (the
// 1/(nx ny) of both inverse transforms).  Scaling by a power of two commutes
// with rounding, so this gives the bits of apply_delta(s v, d) with one
// product fewer per component.
template <typename C>
__device__ __forceinline__ C apply_delta_scaled(C v, typename Re<C>::type s, C ds) {
  return C{fma(v.x, ds.x, fma(-v.y, ds.y, v.x * s)), fma(v.x, ds.y, fma(v.y, ds.x, v.y * s))};
}
template <>
__device__ __forceinline__ float2 apply_delta_scaled<float2>(float2 v, float s, float2 ds) {
  const float tr = fmaf(v.x, ds.x, -(v.y * ds.y));
  const float ti = fmaf(v.y, ds.x, v.x * ds.y);
  return __ffma2_rn(v, make_float2(s, s), make_float2(tr, ti));
}

// v * (hi + lo) (or v * conj(hi + lo)): a twiddle carried as an unevaluated
// sum of two values, so that its modulus is 1 to twice the working precision.
// Rounding a unit twiddle to one FP32 value leaves |w| != 1 by up to 6e-8,
// with the same sign every step: an energy drift the compensated product
// removes.  In FP64 the low part is not used.
template <bool CONJ, typename C>
__device__ __forceinline__ C cmul_hl(C v, C hi, C lo) {
  using R = typename Re<C>::type;
  const R hy = CONJ ? -hi.y : hi.y;
  if constexpr (sizeof(R) == 8) {
    return C{v.x * hi.x - v.y * hy, v.x * hy + v.y * hi.x};
  } else {
    const R ly = CONJ ? -lo.y : lo.y;
    R re = fma(v.x, lo.x, -v.y * ly);
    R im = fma(v.x, ly, v.y * lo.x);
    re = fma(v.x, hi.x, fma(-v.y, hy, re));
    im = fma(v.x, hy, fma(v.y, hi.x, im));
    return C{re, im};
  }
}

// v * W_j (or its conjugate) from a twiddle table stored as interleaved
// (hi, lo) pairs: in FP32 the pair is one 16-byte load.
template <bool CONJ, typename C>
__device__ __forceinline__ C cmul_tw(C v, const C* tw, int j) {
  if constexpr (sizeof(C) == 8) {
    const float4 t = *reinterpret_cast<const float4*>(tw + 2 * j);
    return cmul_hl<CONJ>(v, C{t.x, t.y}, C{t.z, t.w});
  } else {
    return cmul_hl<CONJ>(v, tw[2 * j], tw[2 * j + 1]);
  }
}

template <typename R> __device__ __forceinline__ R hi_part(double v) { return (R)v; }
template <typename R> __device__ __forceinline__ R lo_part(double v) {
  return sizeof(R) == 8 ? (R)0 : (R)(v - (double)(float)v);
}

// a * W_N^{k} with W_N = exp(-2 pi i / N) (forward) or its conjugate (inverse).
// k is a compile-time constant after unrolling; trivial factors cost nothing,
// the others use compensated constants (see cmul_hl).
template <int N, bool INV, typename C>
__device__ __forceinline__ C twiddle_const(C a, int k) {
  using R = typename Re<C>::type;
  if (k == 0) return a;
  if (4 * k == N) return INV ? C{-a.y, a.x} : C{a.y, -a.x};          // * (+i) / (-i)
  constexpr double r2 = 0.70710678118654752440;                       // 1/sqrt(2)
  if (8 * k == N || 8 * k == 3 * N) {
    // (+-1 -+ i)/sqrt2: sums first, then one compensated scaling
    const R rh = hi_part<R>(r2), rl = lo_part<R>(r2);
    R u, w;
    if (8 * k == N) {
      if (INV) { u = a.x - a.y; w = a.x + a.y; } else { u = a.x + a.y; w = a.y - a.x; }
    } else {
      if (INV) { u = -a.x - a.y; w = a.x - a.y; } else { u = a.y - a.x; w = -a.x - a.y; }
    }
    if constexpr (sizeof(R) == 8) {
      return C{u * rh, w * rh};           // FP64: no low part (a product by 0 would still be issued)
    } else {
      return C{fma(u, rh, u * rl), fma(w, rh, w * rl)};
    }
  }
  const int j = k * (16 / N);
  const C hi{hi_part<R>(cos16(j)), hi_part<R>(-sin16(j))};
  const C lo{lo_part<R>(cos16(j)), lo_part<R>(-sin16(j))};
  return cmul_hl<INV>(a, hi, lo);                                     // * (c - i s) or its conjugate
}

// 4-point DFT of (a, b, c, d) in place, forward e^{-2 pi i jk/4} or inverse
// e^{+...} (no 1/4): the products by -+i are component swaps, so it costs
// eight complex additions.
template <bool INV, typename C>
__device__ __forceinline__ void dft4(C& a, C& b, C& c, C& d) {
  const C s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = csub(b, d);
  a = cadd(s0, s1);
  c = csub(s0, s1);
  if (INV) {              // X1 = d0 + i d1, X3 = d0 - i d1
    b = C{d0.x - d1.y, d0.y + d1.x};
    d = C{d0.x + d1.y, d0.y - d1.x};
  } else {                // X1 = d0 - i d1, X3 = d0 + i d1
    b = C{d0.x + d1.y, d0.y - d1.x};
    d = C{d0.x - d1.y, d0.y + d1.x};
  }
}

// In-register DFT of length N in {1,2,4,8,16}: natural order in and out,
// forward sum e^{-2 pi i jk/N}, inverse e^{+...} without the 1/N.  With S44,
// N = 16 is split 4 x 4 (x[n2 + 4 n1] -> X[k1 + 4 k2], with W16^(n2 k1)
// between the two 4-point stages): 4 general and 4 eighth-root twiddles,
// against 4 and 6 for the radix-2 recursion, with the same number of
// additions, but more values live at once (see kX44 in hom_pass.cuh).
template <int N, bool INV, bool S44 = false, typename C>
__device__ __forceinline__ void dft_reg(C* v) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (N == 16 && S44) {
    C t[16];   // t[4 k1 + n2]
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C a = v[n2], b = v[n2 + 4], c = v[n2 + 8], d = v[n2 + 12];
      dft4<INV>(a, b, c, d);
      t[n2] = a;
      t[4 + n2] = twiddle_const<16, INV>(b, n2);
      t[8 + n2] = twiddle_const<16, INV>(c, 2 * n2);
      t[12 + n2] = twiddle_const<16, INV>(d, 3 * n2);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C a = t[4 * k1], b = t[4 * k1 + 1], c = t[4 * k1 + 2], d = t[4 * k1 + 3];
      dft4<INV>(a, b, c, d);
      v[k1] = a;
      v[k1 + 4] = b;
      v[k1 + 8] = c;
      v[k1 + 12] = d;
    }
  } else {
    static_assert(N == 4 || N == 8 || N == 16, "register DFT length");
    C e[N / 2], o[N / 2];
#pragma unroll
    for (int j = 0; j < N / 2; ++j) {
      e[j] = v[2 * j];
      o[j] = v[2 * j + 1];
    }
    dft_reg<N / 2, INV>(e);
    dft_reg<N / 2, INV>(o);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const C t = twiddle_const<N, INV>(o[k], k);
      v[k] = cadd(e[k], t);
      v[k + N / 2] = csub(e[k], t);
    }
  }
}

// Split of an axis length into (N1, N2): N <= 16 is one register pass.
template <int N> struct Split {
  static constexpr int N1 = (N <= 16) ? N : (N >= 128 ? 16 : 8);
  static constexpr int N2 = N / N1;
  static_assert(N1 <= 16 && N2 <= 16 && N1 * N2 == N, "axis length");
};

}  // namespace hom

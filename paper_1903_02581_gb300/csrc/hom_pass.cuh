// hom_pass.cuh -- the per-particle kinetic passes of one Strang step and the
// observables passes, templated on precision and grid.
//
// The Strang step of Eq. (evoloperat) of arXiv:1903.02581 (symmetric order)
//   S = V/2 . F_x^-1 T_x/2 F_y^-1 T_y F_y T_x/2 F_x . V/2
// has a kinetic factor that splits exactly per particle, because every
// operator of particle 1 commutes with every operator of particle 2 and
// F_{x1,x2} = F_{x1} F_{x2}, T_x = T_x1 + T_x2 (Appendix A):
//   K = K_1 K_2,  K_i = F_xi^-1 Q_i F_yi^-1 G_i F_yi Q_i F_xi,
//   Q_i = e^{-i dt/4 (k_xi - B y_i)^2},  G_i = e^{-i dt/2 k_yi^2}.
// K_2 acts on the (x2, y2) plane of each fixed (x1, y1): a contiguous row of
// psi[r1][r2]; K_1 acts on the (x1, y1) planes, the rows of the transposed
// state psi[r2][r1].  Since K_1 and K_2 commute, a step applies them in either
// order, and the host sequences the passes in one of three ways (step
// strategies, all with the same arithmetic per element):
//   - a transposing pass that reads rows of whichever layout holds the state
//     and writes the other layout (kinetic_pass_t), then an in-place pass on
//     the rows of that layout (kinetic_pass);
//   - in-place pass, plain transpose (transpose_state), in-place pass;
//   - a transpose and one double in-place pass per step (kinetic_pass with
//     TWICE): the same particle's sandwich at the end of one step and at the
//     start of the next, with the potential phase of a full step between them.
// The real-space phase e^{-iV tau} (V1(r1) + V1(r2) + V12, symmetric in the
// particles) is fused into the first load of a run, between the two
// sandwiches of a double pass, and, for the last half step, into the last
// store.  Each pass reads and writes the state once: two HBM round trips per
// step with the first or the third sequence.
//
// A CTA holds G planes of one simulation in shared memory, laid out
// [g][x][y] with row stride RS = ny + 1 and plane stride PS (padding chosen so
// that the access patterns below are free of bank conflicts).
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hom_fft.cuh"

namespace hom {

template <typename C> struct PassArgs {
  C* psi;              // state [batch][n][n]
  // Unit-modulus phase tables are stored as deltas d = w - 1 (see apply_delta).
  const C* qa;         // e^{-i dt/4 (k_x - B y)^2} - 1        [x position][y]
  const C* qt;         // the same deltas times 1/(nx ny), transposed [y][x position]
  const C* gy;         // e^{-i dt/2 k_y^2} - 1                [y position]
  const C* twx;        // e^{-2 pi i j / nx}, j < nx: interleaved (hi, lo) pairs
  const C* twy;        // e^{-2 pi i j / ny}, j < ny: interleaved (hi, lo) pairs
  const C* p1;         // e^{-i tau V1(r)} - 1                 [batch][n]   (tau = dt/2 or dt)
  const C* p12;        // e^{-i tau V12(dx, dy)} - 1           [batch][(2nx-1)(2ny-1)]
  const C* p1m;        // double pass: the potential between its two sandwiches (tau = dt)
  const C* p12m;
  int v_load;          // apply the potential phase when loading
  int v_store;         // apply the potential phase when storing
  int pref_ahead;      // nonzero: prefetch into L2 the tile a CTA takes next
  int ntiles;          // tiles of the launch: CTA c takes tiles c, c + gridDim.x, ...
};

// Transposing pass: reads G contiguous rows of src ([n][n] per simulation,
// row = the plane of one particle for a fixed coordinate of the other) and
// writes the result transposed into dst, so that the next pass again reads
// contiguous rows (the state alternates between psi[r1][r2] and psi[r2][r1]).
template <typename C> struct PassArgsT {
  CUtensorMap tmap_dst;   // dst as [batch*n rows][n columns] of 8-byte elements (clustered complex64 pass)
  const C* src;
  C* dst;
  const C* qa;
  const C* qt;
  const C* gy;
  const C* twx;
  const C* twy;
  const C* p1;
  const C* p12;
  int v_load;          // apply the potential phase when loading
  int v_store;         // apply the potential phase when storing
  int pref_ahead;      // prefetch into L2 the tile this many CTAs ahead (0: off)
  int ntiles;          // tiles of the launch (without a cluster the pass is persistent)
};

// The energy weights are in the state precision: the energy terms are summed
// per thread in that precision (a few dozen terms) and added in FP64; the
// norm and the bunching probability are sums of exact squares (SqSum).
template <typename C> struct MeasureArgs {
  using R = typename Re<C>::type;
  const C* psi;
  const C* twx;
  const C* twy;
  const R* tx;         // 1/2 (k_x - B y)^2                    [x position][y]
  const R* ty;         // 1/2 k_y^2                            [y position]
  const R* v1;         // V1(r)                                [batch][n]
  const R* v12;        // V12(dx, dy)                          [batch][(2nx-1)(2ny-1)]
  double* partial;     // [tile][NPART]
};

constexpr int NPART = 6;   // norm, e_pot, e_coul, p_bunch, e_tx, e_ty (raw sums)

// Tile geometry.  COL = false: the in-place pass (G contiguous rows per CTA,
// up to 32 KB of planes); COL = true: the transposing pass and the column
// observables (up to 128 KB of planes, so that G >= 4 columns give 32-byte
// segments).  V selects one of two variants the autotuner times (results are
// identical; only thread counts and cluster widths differ).
template <typename T, int NX, int NY, bool COL, int V = 0> struct Geo {
  using C = typename Cx<T>::type;
  static constexpr int N = NX * NY;
  static constexpr int LW = 128 / (int)sizeof(C);        // lanes per shared-memory wavefront
  static constexpr int BUDGET = (COL ? 16384 : 4096) * 8 / (int)sizeof(C);
  static constexpr int GMAX = COL ? 16 : 8;
  static constexpr int G0 = BUDGET / N;
  static constexpr int G = G0 < 1 ? 1 : (G0 > GMAX ? GMAX : G0);
  static constexpr int RS = NY + 1;
  static constexpr int PS0 = NX * RS;
  static constexpr int PSM = (G >= LW) ? 1 : (LW / G);
  static constexpr int PS = PS0 + ((((PSM - PS0) % LW) + LW) % LW);
  static constexpr int ELEMS = G * PS;
  // twiddle tables after the planes, 16-byte aligned (one (hi, lo) pair per load)
  static constexpr int TWOFF = (ELEMS + 1) / 2 * 2;
  static constexpr size_t SMEM = (size_t)(TWOFF + 2 * NX + 2 * NY) * sizeof(C);
  static constexpr int TILES_PER_SIM = N / G;
  static_assert(N % G == 0, "tile");
  // Transposing pass with fewer than 4 planes per CTA: a cluster of CL CTAs
  // holds CL*G adjacent planes, so that its transposed stores cover whole
  // 32-byte sectors (variant 1: half as wide, 16-byte segments); values move
  // between the CTAs through distributed shared memory.
  static constexpr int CL0 = (COL && G < 4) ? 4 / G : 1;
  static constexpr int CL = (V == 1 && CL0 > 1) ? CL0 / 2 : CL0;
  static_assert(TILES_PER_SIM % CL == 0, "cluster");
  // threads: 512 for complex64 tiles of 8192 points or more, else 256 (a
  // complex128 thread holds twice the registers); variant 1 of an unclustered
  // kernel uses the other count
  static constexpr int NT0 = (sizeof(C) == 8 && G * N >= 8192) ? 512 : 256;
  static constexpr int NT = (V == 1 && CL0 == 1) ? (NT0 == 512 ? 256 : 512) : NT0;
  // x stages owned by XG thread groups of 16 columns each (see x_item), where
  // the thread counts divide evenly and the grid was measured to gain: groups
  // drift apart between the y sandwiches, so one group's shared-memory and
  // load phases overlap another's arithmetic (the 256x64 double pass: 6 %
  // shorter; the 128x32 in-place pass: 2 %; the 4-plane transposing pass of
  // the 128x32 grid ran 9 % slower with them).  Elsewhere 1: every stage ends
  // with a CTA barrier.
  static constexpr int XGC = G * NY / 16;
  static constexpr int XTPG = XGC > 0 ? NT / XGC : 0;
  static constexpr int XSUB = XTPG >= 16 ? XTPG / 16 : 1;   // sub-line indices a group covers at once
  static constexpr bool XOK = sizeof(C) == 8 && XGC > 1 && XGC <= 15 && NT % (32 * XGC) == 0 && XTPG % 16 == 0 &&
                              Split<NX>::N2 > 1 && Split<NX>::N1 % XSUB == 0 && Split<NX>::N2 % XSUB == 0;
  static constexpr bool XMEASURED = (NX == 256 && NY == 64) || (NX == 128 && NY == 32 && !COL);
  static constexpr int XG = (XOK && XMEASURED) ? XGC : 1;
  // clustered complex64 transposing pass: its stores go through the tensor
  // memory accelerator from two staging buffers of N1 tiles of ny rows x CL*G
  // columns (see x_inverse_cluster_store_tma)
  static constexpr bool TMA_STORE = COL && CL > 1 && sizeof(C) == 8;
  static constexpr int STAGE = TMA_STORE ? 2 * Split<NX>::N1 * NY * CL * G : 0;
  static constexpr size_t STAGE_OFF = (SMEM + 127) / 128 * 128;
  // + 128 bytes of slack: the kernel rounds the staging address up to 128 bytes
  static constexpr size_t SMEM_ALL = TMA_STORE ? STAGE_OFF + (size_t)STAGE * sizeof(C) + 128 : SMEM;
};

// The 16-point DFTs of the x axis are split 4 x 4 (fewer twiddles, more live
// values: see dft_reg) only where the x axis is 256 long: there it shortened
// the double pass by 2.3 %, while on the 128-long axis of the batched grid it
// slowed the transposing pass by 7.6 %.  Every kernel of a grid uses the same
// choice, so the step strategies stay bitwise identical.
template <int NX> constexpr bool kX44 = NX == 256;

// ---------------------------------------------------------------------------
// Line transforms over the shared-memory planes.  An x-line is the column of
// one (g, y); a y-line is the row of one (g, x position).
// ---------------------------------------------------------------------------

// Item (g, y, sub) of an x stage: the x-line (column) of plane g at y, and the
// sub-line index (n2, k1 or m) of the stage.  XG == 1: lanes run over y, then
// sub, then g.  XG > 1: thread group q = tid / (NT/XG) owns the columns
// c = g*NY + y in [q*CPG, (q+1)*CPG), CPG = G*NY/XG (16: a 128-byte row
// segment of complex64), with lanes still running over consecutive y, so each
// column's stages stay inside one group and only that group needs to
// synchronise between them (group_sync).  Any bijection of items onto threads
// gives the same bits: an item's arithmetic does not depend on its thread.
template <int NT, int NY, int G, int NSUB, int XG>
__device__ __forceinline__ void x_item(int it, int& g, int& y, int& sub) {
  if constexpr (XG == 1) {
    y = it % NY;
    sub = (it / NY) % NSUB;
    g = it / (NY * NSUB);
  } else {
    constexpr int TPG = NT / XG, CPG = G * NY / XG;
    static_assert((G * NY) % XG == 0 && NY % CPG == 0 && NT % (32 * XG) == 0 && TPG % CPG == 0 &&
                      NSUB % (TPG / CPG) == 0,
                  "x-stage thread groups");
    const int t = it % NT, q = t % TPG;
    const int c = (t / TPG) * CPG + q % CPG;
    g = c / NY;
    y = c % NY;
    sub = q / CPG + (TPG / CPG) * (it / NT);
  }
}

// Barrier over the thread group of x_item (named barrier 1 + group; barrier 0
// is __syncthreads), or over the CTA when XG == 1.
template <int NT, int XG>
__device__ __forceinline__ void group_sync() {
  if constexpr (XG == 1) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / (NT / XG)), "r"(NT / XG) : "memory");
  }
}

struct NoHook {
  template <typename C> __device__ __forceinline__ C operator()(int, int, C v) const { return v; }
};

// Forward DFT along x of every x-line; hook(pos, y, v) sees each output
// coefficient at its x position (digit-transposed order when nx > 16).
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, class Hook>
__device__ __forceinline__ void x_forward(C* sm, const C* tw, Hook& hook) {
  using S = Split<NX>;
  constexpr int N1 = S::N1, N2 = S::N2;
  const int tid = threadIdx.x;
  if constexpr (N2 == 1) {
    for (int it = tid; it < G * NY; it += NT) {
      const int y = it % NY, g = it / NY;
      C* line = sm + g * PS + y;
      C v[NX];
#pragma unroll
      for (int x = 0; x < NX; ++x) v[x] = line[x * RS];
      dft_reg<NX, false, kX44<NX>>(v);
#pragma unroll
      for (int k = 0; k < NX; ++k) line[k * RS] = hook(k, y, v[k]);
    }
    __syncthreads();
  } else {
    for (int it = tid; it < G * NY * N2; it += NT) {
      const int y = it % NY, n2 = (it / NY) % N2, g = it / (NY * N2);
      C* line = sm + g * PS + y;
      C v[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = line[(N2 * n1 + n2) * RS];
      dft_reg<N1, false, kX44<NX>>(v);
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul_tw<false>(v[k1], tw, n2 * k1);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) line[(N2 * k1 + n2) * RS] = v[k1];
    }
    __syncthreads();
    for (int it = tid; it < G * NY * N1; it += NT) {
      const int y = it % NY, k1 = (it / NY) % N1, g = it / (NY * N1);
      C* line = sm + g * PS + y;
      C v[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = line[(N2 * k1 + n2) * RS];
      dft_reg<N2, false, kX44<NX>>(v);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) line[(N2 * k1 + k2) * RS] = hook(N2 * k1 + k2, y, v[k2]);
    }
    __syncthreads();
  }
}

// The y part of the kinetic sandwich on every y-line: F_y, G, F_y^-1 (no
// 1/ny), then the second T_x/2 phase and the 1/(nx ny) of both inverse
// transforms (a power of two: exact) from qb, a [y][x position] table of the
// scaled deltas (so that lanes running over x positions read consecutive
// entries; see apply_delta_scaled).
template <typename C, int NX, int NY, int G, int NT, int RS, int PS>
__device__ __forceinline__ void y_sandwich(C* sm, const C* tw, const C* __restrict__ gy,
                                           const C* __restrict__ qb) {
  using S = Split<NY>;
  using R = typename Re<C>::type;
  constexpr R scale = (R)1 / (R)(NX * NY);
  constexpr int N1 = S::N1, N2 = S::N2;
  const int tid = threadIdx.x;
  if constexpr (N2 == 1) {
    for (int it = tid; it < G * NX; it += NT) {
      const int px = it % NX, g = it / NX;
      C* row = sm + g * PS + px * RS;
      C v[NY];
#pragma unroll
      for (int y = 0; y < NY; ++y) v[y] = row[y];
      dft_reg<NY, false>(v);
#pragma unroll
      for (int k = 0; k < NY; ++k) v[k] = apply_delta(v[k], ldg(gy + k));
      dft_reg<NY, true>(v);
#pragma unroll
      for (int y = 0; y < NY; ++y) row[y] = apply_delta_scaled(v[y], scale, ldg(qb + y * NX + px));
    }
    __syncthreads();
  } else {
    // the three register passes of a line: forward N1-point stage with its
    // twiddle; N2-point stage, G, inverse N2-point stage, inverse twiddle;
    // inverse N1-point stage with the scale and the closing T_x/2 phase
    auto pass1 = [&](int g, int px, int n2) {
      C* row = sm + g * PS + px * RS;
      C v[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = row[N2 * n1 + n2];
      dft_reg<N1, false>(v);
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul_tw<false>(v[k1], tw, n2 * k1);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) row[N2 * k1 + n2] = v[k1];
    };
    auto pass2 = [&](int g, int px, int k1) {
      C* row = sm + g * PS + px * RS;
      C v[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = row[N2 * k1 + n2];
      dft_reg<N2, false>(v);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) v[k2] = apply_delta(v[k2], ldg(gy + N2 * k1 + k2));
      dft_reg<N2, true>(v);
#pragma unroll
      for (int m1 = 1; m1 < N2; ++m1) v[m1] = cmul_tw<true>(v[m1], tw, m1 * k1);
#pragma unroll
      for (int m1 = 0; m1 < N2; ++m1) row[N2 * k1 + m1] = v[m1];
    };
    auto pass3 = [&](int g, int px, int m1) {
      C* row = sm + g * PS + px * RS;
      C v[N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) v[k1] = row[N2 * k1 + m1];
      dft_reg<N1, true>(v);
#pragma unroll
      for (int m2 = 0; m2 < N1; ++m2) {
        const int y = m1 + N2 * m2;
        row[y] = apply_delta_scaled(v[m2], scale, ldg(qb + y * NX + px));
      }
    };
    // Each warp owns LW whole lines when that keeps every half-warp on 16
    // consecutive lines (conflict-free shared memory): the exchanges between
    // the passes stay inside the warp, so warps need not wait for one another
    // until the whole sandwich is done.
    constexpr int L = G * NX, NW = NT / 32, LW = (L % NW == 0) ? L / NW : 0;
    constexpr bool WARP_LINES = LW >= 16 && (LW * N2) % 32 == 0 && (LW * N1) % 32 == 0;
    if constexpr (WARP_LINES) {
      const int l0 = (tid >> 5) * LW, lane = tid & 31;
      for (int q = lane; q < LW * N2; q += 32) {
        const int l = l0 + q % LW;
        pass1(l / NX, l % NX, q / LW);
      }
      __syncwarp();
      for (int q = lane; q < LW * N1; q += 32) {
        const int l = l0 + q % LW;
        pass2(l / NX, l % NX, q / LW);
      }
      __syncwarp();
      for (int q = lane; q < LW * N2; q += 32) {
        const int l = l0 + q % LW;
        pass3(l / NX, l % NX, q / LW);
      }
      __syncthreads();
    } else {
      for (int it = tid; it < G * NX * N2; it += NT) pass1(it / (NX * N2), it % NX, (it / NX) % N2);
      __syncthreads();
      for (int it = tid; it < G * NX * N1; it += NT) pass2(it / (NX * N1), it % NX, (it / NX) % N1);
      __syncthreads();
      for (int it = tid; it < G * NX * N2; it += NT) pass3(it / (NX * N2), it % NX, (it / NX) % N2);
      __syncthreads();
    }
  }
}

// Forward DFT along y of every y-line; hook(pos_x, pos_y, v) sees each output.
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, class Hook>
__device__ __forceinline__ void y_forward(C* sm, const C* tw, Hook& hook) {
  using S = Split<NY>;
  constexpr int N1 = S::N1, N2 = S::N2;
  const int tid = threadIdx.x;
  if constexpr (N2 == 1) {
    for (int it = tid; it < G * NX; it += NT) {
      const int px = it % NX, g = it / NX;
      C* row = sm + g * PS + px * RS;
      C v[NY];
#pragma unroll
      for (int y = 0; y < NY; ++y) v[y] = row[y];
      dft_reg<NY, false>(v);
#pragma unroll
      for (int k = 0; k < NY; ++k) row[k] = hook(px, k, v[k]);
    }
    __syncthreads();
  } else {
    for (int it = tid; it < G * NX * N2; it += NT) {
      const int px = it % NX, n2 = (it / NX) % N2, g = it / (NX * N2);
      C* row = sm + g * PS + px * RS;
      C v[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = row[N2 * n1 + n2];
      dft_reg<N1, false>(v);
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul_tw<false>(v[k1], tw, n2 * k1);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) row[N2 * k1 + n2] = v[k1];
    }
    __syncthreads();
    for (int it = tid; it < G * NX * N1; it += NT) {
      const int px = it % NX, k1 = (it / NX) % N1, g = it / (NX * N1);
      C* row = sm + g * PS + px * RS;
      C v[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = row[N2 * k1 + n2];
      dft_reg<N2, false>(v);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) row[N2 * k1 + k2] = hook(px, N2 * k1 + k2, v[k2]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Real-space phase e^{-i tau V(r1, r2)} from the single-particle and the
// difference tables (never a 4D array).
// ---------------------------------------------------------------------------
template <typename C, int NX, int NY>
__device__ __forceinline__ C vphase_delta(const C* __restrict__ p1, const C* __restrict__ p12, int r1, int r2) {
  const int x1 = r1 / NY, y1 = r1 % NY, x2 = r2 / NY, y2 = r2 % NY;
  const int d = (x1 - x2 + NX - 1) * (2 * NY - 1) + (y1 - y2 + NY - 1);
  // (1 + d1)(1 + d2)(1 + d12) - 1, formed from the small deltas
  const C d1 = ldg(p1 + r1), d2 = ldg(p1 + r2), d12 = ldg(p12 + d);
  const C e = cadd(cadd(d1, d2), cmul(d1, d2));
  return cadd(cadd(e, d12), cmul(e, d12));
}

template <typename C, int NY>
struct QHook {
  const C* __restrict__ q;
  __device__ __forceinline__ C operator()(int pos, int y, C v) const { return apply_delta(v, ldg(q + pos * NY + y)); }
};

// ---------------------------------------------------------------------------
// Kinetic passes: in place on rows (kinetic_pass) or transposing (kinetic_pass_t).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Item decode of the stages that touch global memory: rows (lanes run over y,
// contiguous in a row plane) or columns (lanes run over the G planes first,
// which are the contiguous index of a column tile).
template <bool COL, int NY, int G, int NSUB>
__device__ __forceinline__ void decode_item(int it, int& g, int& y, int& sub) {
  if constexpr (!COL) {
    y = it % NY;
    sub = (it / NY) % NSUB;
    g = it / (NY * NSUB);
  } else {
    g = it % G;
    y = (it / G) % NY;
    sub = it / (G * NY);
  }
}

template <bool COL, int NX, int NY>
__device__ __forceinline__ size_t global_offset(int t0, int g, int x, int y) {
  constexpr int N = NX * NY;
  if constexpr (!COL) return (size_t)(t0 + g) * N + x * NY + y;
  else return (size_t)(x * NY + y) * N + (t0 + g);
}

// First x stage read straight from global memory (streaming loads: the state
// is read once per pass): every thread loads the N1
// elements of its line segment (all in flight at once), applies the potential
// phase if asked (it is symmetric in the two particles, so the plane index
// t0 + g and the element index may be either particle's), transforms, and
// writes shared memory.  With nx <= 16 this
// is the whole forward x transform, followed by the T_x/2 hook.
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, bool COL, int XG, class Hook>
__device__ __forceinline__ void x_forward_from_global(C* sm, const C* tw, const C* __restrict__ base, int t0,
                                                      const C* __restrict__ p1, const C* __restrict__ p12,
                                                      bool apply_v, Hook& hook) {
  using S = Split<NX>;
  constexpr int N1 = S::N1, N2 = S::N2;
  for (int it = threadIdx.x; it < G * NY * N2; it += NT) {
    int g, y, n2;
    if constexpr (COL) decode_item<COL, NY, G, N2>(it, g, y, n2);
    else x_item<NT, NY, G, N2, XG>(it, g, y, n2);
    C v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) v[n1] = __ldcs(base + global_offset<COL, NX, NY>(t0, g, N2 * n1 + n2, y));
    if (apply_v) {
      C d[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) d[n1] = vphase_delta<C, NX, NY>(p1, p12, t0 + g, (N2 * n1 + n2) * NY + y);
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = apply_delta(v[n1], d[n1]);
    }
    dft_reg<N1, false, kX44<NX>>(v);
    C* line = sm + g * PS + y;
    if constexpr (N2 == 1) {
#pragma unroll
      for (int k = 0; k < NX; ++k) line[k * RS] = hook(k, y, v[k]);
    } else {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul_tw<false>(v[k1], tw, n2 * k1);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) line[(N2 * k1 + n2) * RS] = v[k1];
    }
  }
  // the second x stage reads only this group's columns
  if constexpr (N2 > 1 && !COL) group_sync<NT, XG>();
  else __syncthreads();
}

// Second forward x stage (shared memory only, nx > 16), hook on every output.
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, int XG, class Hook>
__device__ __forceinline__ void x_forward_second(C* sm, Hook& hook) {
  using S = Split<NX>;
  constexpr int N1 = S::N1, N2 = S::N2;
  for (int it = threadIdx.x; it < G * NY * N1; it += NT) {
    int g, y, k1;
    x_item<NT, NY, G, N1, XG>(it, g, y, k1);
    C* line = sm + g * PS + y;
    C v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = line[(N2 * k1 + n2) * RS];
    dft_reg<N2, false, kX44<NX>>(v);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) line[(N2 * k1 + k2) * RS] = hook(N2 * k1 + k2, y, v[k2]);
  }
  __syncthreads();
}

// First inverse x stage (shared memory only, nx > 16).  GROUP: the next stage
// reads only this group's columns (x_item), so a group barrier ends it.
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, int XG, bool GROUP>
__device__ __forceinline__ void x_inverse_first(C* sm, const C* tw) {
  using S = Split<NX>;
  constexpr int N1 = S::N1, N2 = S::N2;
  for (int it = threadIdx.x; it < G * NY * N1; it += NT) {
    int g, y, k1;
    x_item<NT, NY, G, N1, XG>(it, g, y, k1);
    C* line = sm + g * PS + y;
    C v[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[k2] = line[(N2 * k1 + k2) * RS];
    dft_reg<N2, true, kX44<NX>>(v);
#pragma unroll
    for (int m1 = 1; m1 < N2; ++m1) v[m1] = cmul_tw<true>(v[m1], tw, m1 * k1);
#pragma unroll
    for (int m1 = 0; m1 < N2; ++m1) line[(N2 * k1 + m1) * RS] = v[m1];
  }
  if constexpr (GROUP) group_sync<NT, XG>();
  else __syncthreads();
}

// Last inverse x stage written straight to global memory with streaming
// stores (the whole inverse x transform when nx <= 16), with the closing
// potential phase if asked.
// COL = false writes the planes back as rows; COL = true writes them
// transposed (element (x, y) of plane t0 + g to row x*ny + y, column t0 + g).
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, bool COL, int XG>
__device__ __forceinline__ void x_inverse_to_global(const C* sm, C* __restrict__ base, int t0,
                                                    const C* __restrict__ p1, const C* __restrict__ p12,
                                                    bool apply_v) {
  using S = Split<NX>;
  constexpr int N1 = S::N1, N2 = S::N2;
  for (int it = threadIdx.x; it < G * NY * N2; it += NT) {
    int g, y, m1;
    if constexpr (COL) decode_item<COL, NY, G, N2>(it, g, y, m1);
    else x_item<NT, NY, G, N2, XG>(it, g, y, m1);
    const C* line = sm + g * PS + y;
    C v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = line[(N2 * k1 + m1) * RS];
    dft_reg<N1, true, kX44<NX>>(v);
    if (apply_v) {
#pragma unroll
      for (int m2 = 0; m2 < N1; ++m2)
        v[m2] = apply_delta(v[m2], vphase_delta<C, NX, NY>(p1, p12, (m1 + N2 * m2) * NY + y, t0 + g));
    }
#pragma unroll
    for (int m2 = 0; m2 < N1; ++m2) __stcs(base + global_offset<COL, NX, NY>(t0, g, m1 + N2 * m2, y), v[m2]);
  }
}

// Between the two sandwiches of a double pass, in registers: the last inverse
// x stage of a line (m, y) yields the x positions m + N2*m2, which are exactly
// the inputs N2*n1 + n2 (n2 = m) of a first forward x stage, so the thread
// inverts, applies the potential phase of the full step (the same call, with
// the plane index first, as a pass that applies it on load), transforms
// forward again and writes back the shared-memory positions it read.  With
// nx <= 16 this is the whole inverse and forward x transform, followed by the
// T_x/2 hook.
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, int XG, class Hook>
__device__ __forceinline__ void x_turnaround(C* sm, const C* tw, int t0, const C* __restrict__ p1,
                                             const C* __restrict__ p12, Hook& hook) {
  using S = Split<NX>;
  constexpr int N1 = S::N1, N2 = S::N2;
  for (int it = threadIdx.x; it < G * NY * N2; it += NT) {
    int g, y, m;
    x_item<NT, NY, G, N2, XG>(it, g, y, m);
    C* line = sm + g * PS + y;
    C v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = line[(N2 * k1 + m) * RS];
    dft_reg<N1, true, kX44<NX>>(v);
    C d[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) d[n1] = vphase_delta<C, NX, NY>(p1, p12, t0 + g, (N2 * n1 + m) * NY + y);
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) v[n1] = apply_delta(v[n1], d[n1]);
    dft_reg<N1, false, kX44<NX>>(v);
    if constexpr (N2 == 1) {
#pragma unroll
      for (int k = 0; k < NX; ++k) line[k * RS] = hook(k, y, v[k]);
    } else {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul_tw<false>(v[k1], tw, m * k1);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) line[(N2 * k1 + m) * RS] = v[k1];
    }
  }
  // the second x stage reads only this group's columns; with nx <= 16 the y
  // sandwich comes next
  if constexpr (N2 > 1) group_sync<NT, XG>();
  else __syncthreads();
}

// Transposed store of a cluster of CL CTAs holding W = CL*G adjacent planes:
// CTA q gathers, for every plane, the inputs of the last inverse x stage of
// the lines m1 = q (mod CL) from the owning CTA (distributed shared memory),
// transforms, applies the closing potential phase if asked, and writes
// 32-byte segments (the W planes' values of one element) to the transposed
// layout.  The caller synchronises the cluster before and after.
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, int CL>
__device__ __forceinline__ void x_inverse_cluster_store(const C* sm, C* __restrict__ base, int c0, int q,
                                                        const C* __restrict__ p1, const C* __restrict__ p12,
                                                        bool apply_v) {
  namespace cg = cooperative_groups;
  using S = Split<NX>;
  constexpr int N1 = S::N1, N2 = S::N2, N = NX * NY, W = CL * G;
  cg::cluster_group cl = cg::this_cluster();
  for (int it = threadIdx.x; it < W * NY * (N2 / CL); it += NT) {
    const int j = it % W, y = (it / W) % NY, m1 = q + CL * (it / (W * NY));
    const C* src = cl.map_shared_rank(const_cast<C*>(sm), j / G) + (j % G) * PS + y;
    C v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = src[(N2 * k1 + m1) * RS];
    dft_reg<N1, true, kX44<NX>>(v);
    if (apply_v) {
#pragma unroll
      for (int m2 = 0; m2 < N1; ++m2)
        v[m2] = apply_delta(v[m2], vphase_delta<C, NX, NY>(p1, p12, (m1 + N2 * m2) * NY + y, c0 + j));
    }
#pragma unroll
    for (int m2 = 0; m2 < N1; ++m2) base[(size_t)((m1 + N2 * m2) * NY + y) * N + c0 + j] = v[m2];
  }
}

// In-place pass: one kinetic sandwich on G contiguous rows of psi (the plane
// of one particle for a fixed coordinate of the other), written back in place.
// TWICE: two sandwiches of the same particle with the potential phase of a
// full step between them (the end of one Strang step and the start of the
// next, when the state is not transposed in between).
// Persistent: the launch holds the CTAs that fit on the device at once, and
// each walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  The twiddles
// are staged once per CTA, the next tile is prefetched into L2 while the
// current one is transformed, and with x-stage groups (XG > 1) a group goes
// from storing its columns of one tile to loading them for the next without
// waiting for the other groups.
template <typename T, int NX, int NY, int V, bool TWICE>
__global__ void __launch_bounds__(Geo<T, NX, NY, false, V>::NT)
kinetic_pass(PassArgs<typename Cx<T>::type> a) {
  using Gm = Geo<T, NX, NY, false, V>;
  using C = typename Cx<T>::type;
  constexpr int N = Gm::N, G = Gm::G, NT = Gm::NT, RS = Gm::RS, PS = Gm::PS;
  constexpr int N2X = Split<NX>::N2;
  constexpr int XG = Gm::XG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* stwx = sm + Gm::TWOFF;
  C* stwy = stwx + 2 * NX;
  const int tid = threadIdx.x;
  for (int i = tid; i < 2 * NX; i += NT) stwx[i] = a.twx[i];
  for (int i = tid; i < 2 * NY; i += NT) stwy[i] = a.twy[i];
  QHook<C, NY> qa{a.qa};
  __syncthreads();                               // twiddles in shared memory

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int b = tile / Gm::TILES_PER_SIM;
    const int t0 = (tile % Gm::TILES_PER_SIM) * G;
    C* base = a.psi + (size_t)b * N * N;
    const C* p1 = a.p1 + (size_t)b * N;
    const C* p12 = a.p12 + (size_t)b * (2 * NX - 1) * (2 * NY - 1);

    // start the HBM read of this CTA's next tile into L2
    const int nt = tile + (int)gridDim.x;
    if (tid == 0 && a.pref_ahead > 0 && nt < a.ntiles) {
      const C* p = a.psi + (size_t)(nt / Gm::TILES_PER_SIM) * N * N + (size_t)(nt % Gm::TILES_PER_SIM) * G * N;
      prefetch_l2(p, (unsigned)(G * N * sizeof(C)));
    }
    x_forward_from_global<C, NX, NY, G, NT, RS, PS, false, XG>(sm, stwx, base, t0, p1, p12, a.v_load != 0, qa);
    if constexpr (N2X > 1) x_forward_second<C, NX, NY, G, NT, RS, PS, XG>(sm, qa);
    y_sandwich<C, NX, NY, G, NT, RS, PS>(sm, stwy, a.gy, a.qt);
    if constexpr (N2X > 1) x_inverse_first<C, NX, NY, G, NT, RS, PS, XG, true>(sm, stwx);
    if constexpr (TWICE) {
      x_turnaround<C, NX, NY, G, NT, RS, PS, XG>(sm, stwx, t0, a.p1m + (size_t)b * N,
                                                 a.p12m + (size_t)b * (2 * NX - 1) * (2 * NY - 1), qa);
      if constexpr (N2X > 1) x_forward_second<C, NX, NY, G, NT, RS, PS, XG>(sm, qa);
      y_sandwich<C, NX, NY, G, NT, RS, PS>(sm, stwy, a.gy, a.qt);
      if constexpr (N2X > 1) x_inverse_first<C, NX, NY, G, NT, RS, PS, XG, true>(sm, stwx);
    }
    x_inverse_to_global<C, NX, NY, G, NT, RS, PS, false, XG>(sm, base, t0, p1, p12, a.v_store != 0);
    // the next tile's first stage overwrites the shared memory just read
    // (only this group's columns when XG > 1)
    group_sync<NT, XG>();
  }
}

// One kinetic sandwich of the particle whose plane is a row of src, written
// transposed to dst (see PassArgsT).  The potential phase is symmetric in the
// two particles, so the same kernel serves both particles.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* smem, int c0, int c1) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(c0),
               "r"(c1), "r"(s)
               : "memory");
}
__device__ __forceinline__ void tma_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void tma_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Transposed store of a cluster of CL CTAs through the tensor memory
// accelerator.  CTA q handles the lines m1 = q (mod CL) in rounds of one m1:
// for every plane j of the cluster and every y it gathers the N1 inputs of the
// last inverse x stage from the owning CTA, transforms, applies the closing
// potential phase if asked, and writes the N1 outputs (x = m1 + N2 m2) into a
// staging buffer laid out as N1 tiles [y][j]; one thread then stores tile m2
// to rows (row0 + x*ny .. + ny) and columns c0 .. c0 + W of the transposed
// layout with one bulk tensor copy.  Two staging buffers alternate; a buffer is
// rewritten only after the copies that read it have finished reading.
template <typename C, int NX, int NY, int G, int NT, int RS, int PS, int CL>
__device__ __forceinline__ void x_inverse_cluster_store_tma(const C* sm, C* stage, const CUtensorMap* map, int row0,
                                                            int c0, int q, const C* __restrict__ p1,
                                                            const C* __restrict__ p12, bool apply_v) {
  namespace cg = cooperative_groups;
  using S = Split<NX>;
  constexpr int N1 = S::N1, N2 = S::N2, W = CL * G, TILE = NY * W;
  cg::cluster_group cl = cg::this_cluster();
  const int tid = threadIdx.x;
  for (int s = 0; s < N2 / CL; ++s) {
    const int m1 = q + CL * s;
    C* st = stage + (s & 1) * (N1 * TILE);
    if (s >= 2) {
      if (tid == 0) tma_wait_read<1>();          // the copies of round s-2 have read this buffer
      __syncthreads();
    }
    for (int it = tid; it < W * NY; it += NT) {
      const int j = it % W, y = it / W;
      const C* src = cl.map_shared_rank(const_cast<C*>(sm), j / G) + (j % G) * PS + y;
      C v[N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) v[k1] = src[(N2 * k1 + m1) * RS];
      dft_reg<N1, true, kX44<NX>>(v);
      if (apply_v) {
#pragma unroll
        for (int m2 = 0; m2 < N1; ++m2)
          v[m2] = apply_delta(v[m2], vphase_delta<C, NX, NY>(p1, p12, (m1 + N2 * m2) * NY + y, c0 + j));
      }
#pragma unroll
      for (int m2 = 0; m2 < N1; ++m2) st[m2 * TILE + y * W + j] = v[m2];
    }
    __syncthreads();
    if (tid == 0) {
      fence_proxy_async();                       // staging writes visible to the copy engine
#pragma unroll 1
      for (int m2 = 0; m2 < N1; ++m2) tma_store_2d(map, st + m2 * TILE, c0, row0 + (m1 + N2 * m2) * NY);
      tma_commit();
    }
  }
  if (tid == 0) tma_wait_all();                  // stores complete before the CTA's shared memory goes
  __syncthreads();
}

template <typename T, int NX, int NY, int V>
__global__ void __launch_bounds__(Geo<T, NX, NY, true, V>::NT)
kinetic_pass_t(const __grid_constant__ PassArgsT<typename Cx<T>::type> a) {
  using Gm = Geo<T, NX, NY, true, V>;
  using C = typename Cx<T>::type;
  constexpr int N = Gm::N, G = Gm::G, NT = Gm::NT, RS = Gm::RS, PS = Gm::PS;
  constexpr int CL = Gm::CL;
  constexpr int N2X = Split<NX>::N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* stwx = sm + Gm::TWOFF;
  C* stwy = stwx + 2 * NX;
  const int tid = threadIdx.x;
  for (int i = tid; i < 2 * NX; i += NT) stwx[i] = a.twx[i];
  for (int i = tid; i < 2 * NY; i += NT) stwy[i] = a.twy[i];

  QHook<C, NY> qa{a.qa};
  constexpr int XG = Gm::XG;
  // Without a cluster the pass is persistent, like the in-place pass: CTA c
  // takes tiles c, c + gridDim.x, ... (the host launches the resident count
  // and prefetches that many tiles ahead, this CTA's next one).  A clustered
  // launch takes one tile per CTA.
  const int ntiles = (CL == 1) ? a.ntiles : (int)gridDim.x;
  __syncthreads();                               // twiddles in shared memory

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int b = tile / Gm::TILES_PER_SIM;
    const int t0 = (tile % Gm::TILES_PER_SIM) * G;
    const C* src = a.src + (size_t)b * N * N;
    C* dst = a.dst + (size_t)b * N * N;
    const C* p1 = a.p1 + (size_t)b * N;
    const C* p12 = a.p12 + (size_t)b * (2 * NX - 1) * (2 * NY - 1);

    const int nt = tile + a.pref_ahead;
    if (tid == 0 && a.pref_ahead > 0 && nt < ntiles) {
      const C* p = a.src + (size_t)(nt / Gm::TILES_PER_SIM) * N * N + (size_t)(nt % Gm::TILES_PER_SIM) * G * N;
      prefetch_l2(p, (unsigned)(G * N * sizeof(C)));
    }
    x_forward_from_global<C, NX, NY, G, NT, RS, PS, false, XG>(sm, stwx, src, t0, p1, p12, a.v_load != 0, qa);
    if constexpr (N2X > 1) x_forward_second<C, NX, NY, G, NT, RS, PS, XG>(sm, qa);
    y_sandwich<C, NX, NY, G, NT, RS, PS>(sm, stwy, a.gy, a.qt);
    // the transposed stores below read every column: a CTA barrier
    if constexpr (N2X > 1) x_inverse_first<C, NX, NY, G, NT, RS, PS, XG, false>(sm, stwx);
    if constexpr (CL == 1) {
      // G >= 4 adjacent rows: the transposed store writes G*8-byte segments
      x_inverse_to_global<C, NX, NY, G, NT, RS, PS, true, XG>(sm, dst, t0, p1, p12, a.v_store != 0);
      __syncthreads();                           // the next tile overwrites the planes just read
    } else {
      // a cluster of CL CTAs holds CL*G adjacent rows: each CTA stores its share
      // of all of them as 32-byte segments, read through distributed shared memory
      namespace cg = cooperative_groups;
      cg::cluster_group cl = cg::this_cluster();
      const int q = (int)cl.block_rank();
      cl.sync();
      if constexpr (Gm::TMA_STORE) {
        // staging at a 128-byte aligned shared address (bulk tensor copies need it)
        const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem_raw + Gm::STAGE_OFF);
        C* stage = reinterpret_cast<C*>(smem_raw + Gm::STAGE_OFF + ((128u - (s0 & 127u)) & 127u));
        x_inverse_cluster_store_tma<C, NX, NY, G, NT, RS, PS, CL>(sm, stage, &a.tmap_dst, b * N, t0 - q * G, q, p1,
                                                                  p12, a.v_store != 0);
      } else {
        x_inverse_cluster_store<C, NX, NY, G, NT, RS, PS, CL>(sm, dst, t0 - q * G, q, p1, p12, a.v_store != 0);
      }
      cl.sync();                                 // keep this CTA's planes alive for the readers
    }
  }
}

// dst[b][c][r] = src[b][r][c] for a batch of [n][n] states: tiles of T x T
// through shared memory (row stride T + 1: conflict-free column reads), rows
// read and written as contiguous T-element segments, both with streaming
// (evict-first) cache hints: every byte is touched once.  Used between
// in-place passes by step strategies 1 and 2 (see step_sequence).  The launch
// bound keeps four CTAs resident per SM (64 registers, no spills): the copy
// waits on DRAM latency, and four CTAs hide it where the two that 124
// registers allowed did not.
template <typename C, int T>
__global__ void __launch_bounds__(256, 4) transpose_state(const C* __restrict__ src, C* __restrict__ dst, int n,
                                                       int batch) {
  __shared__ C tile[T][T + 1];
  constexpr int ROWS = 256 / T;
  const int r0 = blockIdx.y * T, c0 = blockIdx.x * T;
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  for (int b = blockIdx.z; b < batch; b += gridDim.z) {
    const C* s = src + (size_t)b * n * n;
    C* d = dst + (size_t)b * n * n;
    C v[T / ROWS];
#pragma unroll
    for (int i = 0; i < T / ROWS; ++i) v[i] = __ldcs(s + (size_t)(r0 + ty + i * ROWS) * n + c0 + tx);
    if (b != (int)blockIdx.z) __syncthreads();        // previous simulation's tile fully read
#pragma unroll
    for (int i = 0; i < T / ROWS; ++i) tile[ty + i * ROWS][tx] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < T / ROWS; ++i) __stcs(d + (size_t)(c0 + ty + i * ROWS) * n + r0 + tx, tile[tx][ty + i * ROWS]);
  }
}

// ---------------------------------------------------------------------------
// Observables: raw sums per tile, FP64 accumulation.
// ---------------------------------------------------------------------------
template <typename C, int NY>
struct AccHook {
  using R = typename Re<C>::type;
  const R* __restrict__ w;        // weight by (pos, other)
  R acc;
  bool by_first;                  // x hook: w[pos * NY + y]; y hook: w[y position]
  __device__ __forceinline__ C operator()(int p, int q, C v) {
    const R wt = by_first ? w[p * NY + q] : w[q];
    acc = fma(wt, cnorm2(v), acc);
    return v;
  }
};

// Sum of the exact squares |v|^2 of stored state values (the norm and the
// bunching probability).  In FP32 each square is split exactly into its
// rounded product and that product's error (an FMA), and the terms go into an
// unevaluated pair of FP32 values with the two-sum error-free addition: about
// 2^-48 relative, on the FP32 pipes, where FP64 arithmetic runs at 1/64 of
// their rate.  In FP64 the squares are exact FP64 products of the stored
// values and the sum a plain FP64 one.
template <typename C> struct SqSum;
template <> struct SqSum<double2> {
  double s = 0.0;
  __device__ __forceinline__ void add(double2 v) { s += cnorm2_d(v); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct SqSum<float2> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void two_sum(float b) {
    const float s = __fadd_rn(hi, b);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ void add(float2 v) {
    const float px = __fmul_rn(v.x, v.x), py = __fmul_rn(v.y, v.y);
    const float ex = fmaf(v.x, v.x, -px), ey = fmaf(v.y, v.y, -py);
    two_sum(px);
    two_sum(py);
    lo = __fadd_rn(lo, __fadd_rn(ex, ey));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T> __device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  }
  return s;   // valid in thread 0
}

template <typename T, int NX, int NY, bool COL>
__global__ void __launch_bounds__(Geo<T, NX, NY, COL>::NT)
measure_pass(MeasureArgs<typename Cx<T>::type> a) {
  using Gm = Geo<T, NX, NY, COL>;
  using C = typename Cx<T>::type;
  constexpr int N = Gm::N, G = Gm::G, NT = Gm::NT, RS = Gm::RS, PS = Gm::PS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* stwx = sm + Gm::TWOFF;
  C* stwy = stwx + 2 * NX;
  __shared__ double red[32];
  const int tid = threadIdx.x;
  for (int i = tid; i < 2 * NX; i += NT) stwx[i] = a.twx[i];
  for (int i = tid; i < 2 * NY; i += NT) stwy[i] = a.twy[i];

  const int tile = blockIdx.x;
  const int b = tile / Gm::TILES_PER_SIM;
  const int t0 = (tile % Gm::TILES_PER_SIM) * G;
  using R = typename Re<C>::type;
  const C* base = a.psi + (size_t)b * N * N;
  const R* v1 = a.v1 + (size_t)b * N;
  const R* v12 = a.v12 + (size_t)b * (2 * NX - 1) * (2 * NY - 1);

  SqSum<C> s_norm, s_pb;
  R s_pot = 0, s_coul = 0;
  for (int e = tid; e < G * N; e += NT) {
    int g, r;
    size_t off;
    if constexpr (!COL) { g = e / N; r = e % N; off = (size_t)(t0 + g) * N + r; }
    else                { g = e % G; r = e / G; off = (size_t)r * N + (t0 + g); }
    const C v = base[off];
    if constexpr (!COL) {
      const int r1 = t0 + g, r2 = r;
      const R rr = cnorm2(v);
      const int x1 = r1 / NY, y1 = r1 % NY, x2 = r2 / NY, y2 = r2 % NY;
      s_norm.add(v);
      s_pot = fma(rr, v1[r1] + v1[r2], s_pot);
      s_coul = fma(rr, v12[(x1 - x2 + NX - 1) * (2 * NY - 1) + (y1 - y2 + NY - 1)], s_coul);
      if ((x1 < NX / 2) == (x2 < NX / 2)) s_pb.add(v);
    }
    sm[g * PS + (r / NY) * RS + (r % NY)] = v;
  }
  __syncthreads();

  AccHook<C, NY> hx{a.tx, (R)0, true};
  x_forward<C, NX, NY, G, NT, RS, PS>(sm, stwx, hx);
  AccHook<C, NY> hy{a.ty, (R)0, false};
  y_forward<C, NX, NY, G, NT, RS, PS>(sm, stwy, hy);

  const double vals[NPART] = {s_norm.value(), (double)s_pot, (double)s_coul, s_pb.value(), (double)hx.acc,
                              (double)hy.acc};
  double* out = a.partial + (size_t)tile * NPART;
#pragma unroll
  for (int i = 0; i < NPART; ++i) {
    const double s = block_sum<T>(vals[i], red);
    if (tid == 0) out[i] = s;
  }
}

// Sum the per-tile partials of each simulation in a fixed order:
// out[b][i] = sum over tiles of partial[tile][i].
template <int NP>
__global__ void reduce_partials(const double* __restrict__ partial, int tiles_per_sim,
                                double* __restrict__ out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  for (int i = 0; i < NP; ++i) {
    double s = 0.0;
    for (int t = threadIdx.x; t < tiles_per_sim; t += blockDim.x)
      s += partial[((size_t)b * tiles_per_sim + t) * NP + i];
    s = block_sum<double>(s, red);
    if (threadIdx.x == 0) out[b * NP + i] = s;
  }
}

// psi[b][r1][r2] = c_b (alpha[r1] beta[r2] + s_b beta[r1] alpha[r2]) in FP64,
// rounded once to the state precision (Eq. twopstate).
template <typename C>
__global__ void slater_init(C* __restrict__ psi, const double2* __restrict__ pk, const double* __restrict__ coef,
                            const int* __restrict__ exch, int b0, int nb, int n) {
  const size_t per = (size_t)n * n;
  const size_t total = per * nb;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int b = b0 + (int)(i / per);
    const size_t j = i % per;
    const int r1 = (int)(j / n), r2 = (int)(j % n);
    const double2* al = pk + (size_t)b * 2 * n;
    const double2* be = al + n;
    const double2 a1 = al[r1], b2 = be[r2], b1 = be[r1], a2 = al[r2];
    double re = a1.x * b2.x - a1.y * b2.y, im = a1.x * b2.y + a1.y * b2.x;
    const double s = (double)exch[b];
    re += s * (b1.x * a2.x - b1.y * a2.y);
    im += s * (b1.x * a2.y + b1.y * a2.x);
    const double c = coef[b];
    using R = typename Re<C>::type;
    psi[(size_t)b * per + j] = C{(R)(c * re), (R)(c * im)};
  }
}

}  // namespace hom

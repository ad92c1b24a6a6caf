// hom_tc.cu -- the y part of the kinetic sandwich on the tensor cores: a
// measured design trial, not used by hom_step.
//
// F_y^-1 e^{-i dt T_y} F_y of Eq. (evoloperat) (with the 1/ny of the inverse
// transform) is one fixed 64 x 64 complex circulant C for every y-line of
// every plane, so the y sandwich of a batch of lines is the dense product
// Y = X C^T.  In real form (a line is a row of 128 reals: re, im, re, im, ...)
// it is Y[lines x 128] = X[lines x 128] B^T with B[128 x 128].  FP32 accuracy
// on bf16 tensor cores needs split operands: x = x_hi + x_mid + x_lo (three
// bf16 values, x_hi = bf16(x), the others bf16 of the remainders, exact in
// FP32), B split the same way from its FP64 values, and the six products
// whose terms are at least 2^-16 of the leading one (hh, hm, mh, hl, mm, lh)
// accumulated in FP32 in tensor memory.  With exact accumulation this scheme
// changes the norm of a line by +1e-10 on average (the dropped products),
// against 1e-8 per step for the biased FP32 phase rounding the kinetic
// passes avoid; what the hardware accumulation adds is what the trial measures.
//
// One CTA of 128 threads takes 128 lines (the MMA's M):
//   1. stage B's three pieces (precomputed on the host in the operand
//      layout) and the split lines into shared memory, K-major, no swizzle:
//      8 x 8 bf16 core matrices of 128 contiguous bytes, core matrices
//      adjacent in K 128 bytes apart (leading byte offset), 8-row groups
//      2048 bytes apart (stride byte offset);
//   2. warp 0 allocates 128 tensor-memory columns (the 128 x 128 FP32
//      accumulator);
//   3. one thread issues 6 products x 8 K-steps of tcgen05.mma
//      (M = N = 128, K = 16, kind::f16 with bf16 inputs, FP32 accumulator)
//      and commits them to an mbarrier;
//   4. every thread waits on the mbarrier (bounded: after the limit the CTA
//      records an error, waits once more, bounded, frees its tensor memory
//      and returns), then each warp reads its 32 accumulator rows with
//      tcgen05.ld and stores them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <complex>
#include <vector>

#include "../../include/hom.h"

namespace {

constexpr int kLines = 128;                    // lines per CTA (MMA M)
constexpr int kK = 128;                        // reals per line (MMA K total)
constexpr int kN = 128;                        // reals per output line (MMA N)
constexpr int kPiece = kLines * kK * 2;        // bytes of one bf16 operand piece (32 KB)
constexpr int kThreads = 128;
constexpr int kSmem = 6 * kPiece;              // A and B, three pieces each
constexpr unsigned kSpin = 1u << 20;           // mbarrier polls before giving up
constexpr int kTmemCols = 128;
constexpr double kPiD = 3.14159265358979323846;

// Byte offset of element (row, k) in the K-major, no-swizzle operand layout.
__host__ __device__ __forceinline__ uint32_t op_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 2048 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4, leading byte offset 128,
// stride byte offset 2048, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(2048 >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), bf16
// A and B (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at
// bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kLines >> 4) << 24);

__device__ __forceinline__ void split3(float x, uint16_t& h, uint16_t& m, uint16_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(bh);
  const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(bm);
  const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) { return (uint32_t)a | ((uint32_t)b << 16); }

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned i = 0; i < kSpin; ++i) {
    uint32_t done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(kThreads, 1)
ysandwich_tc(const float* __restrict__ in, float* __restrict__ out, const uint4* __restrict__ bsplit,
             int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  uint8_t* sA = smem;
  uint8_t* sB = smem + 3 * kPiece;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t line0 = (size_t)blockIdx.x * kLines;

  for (int i = tid; i < 3 * kPiece / 16; i += kThreads) reinterpret_cast<uint4*>(sB)[i] = bsplit[i];
  for (int it = tid; it < kLines * (kK / 8); it += kThreads) {
    const int r = it / (kK / 8), c = it % (kK / 8);
    const float4* src = reinterpret_cast<const float4*>(in + (line0 + r) * kK + c * 8);
    const float4 a = src[0], b = src[1];
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint16_t h[8], m[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split3(v[j], h[j], m[j], l[j]);
    const uint32_t off = op_offset(r, c * 8);
    *reinterpret_cast<uint4*>(sA + off) = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
    *reinterpret_cast<uint4*>(sA + kPiece + off) =
        make_uint4(pack2(m[0], m[1]), pack2(m[2], m[3]), pack2(m[4], m[5]), pack2(m[6], m[7]));
    *reinterpret_cast<uint4*>(sA + 2 * kPiece + off) =
        make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const uint32_t bar = smem_u32(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the operands were written by ordinary stores: make them visible to the
  // tensor cores (async proxy) before the barrier
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;

  if (tid == 0) {
    // (A piece, B piece) of the six products kept
    const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    uint32_t accum = 0;
    for (int p = 0; p < 6; ++p) {
      for (int s = 0; s < kK / 16; ++s) {
        const uint64_t ad = op_desc(a0 + pa[p] * kPiece + s * 256);
        const uint64_t bd = op_desc(b0 + pb[p] * kPiece + s * 256);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tbase),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(accum)
            : "memory");
        accum = 1;
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
  }
  bool ok = mbar_wait(bar, 0);
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    ok = mbar_wait(bar, 0);                       // the products may still be running: wait once more
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const size_t row = line0 + 32 * warp + lane;
#pragma unroll 1
    for (int ch = 0; ch < kN / 32; ++ch) {
      uint32_t r[32];
      const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(ch * 32);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
            "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
            "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
            "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float4* dst = reinterpret_cast<float4*>(out + row * kN + ch * 32);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]), __uint_as_float(r[4 * j + 2]),
                             __uint_as_float(r[4 * j + 3]));
    }
  } else if (tid == 0) {
    atomicExch(err, 2);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
}

uint16_t bf16_bits(double x) { return __bfloat16_as_ushort(__double2bfloat16(x)); }
double bf16_value(uint16_t b) { return (double)__bfloat162float(__ushort_as_bfloat16(b)); }

}  // namespace

extern "C" size_t hom_ysandwich_tc_work_bytes(void) { return 3 * (size_t)kPiece + 16; }

extern "C" hom_status hom_ysandwich_tc(const float* d_in, float* d_out, int32_t nlines, double dt, double dy,
                                       void* d_work, size_t work_bytes, int32_t nrep, float* ms, void* cuda_stream) {
  if (!d_in || !d_out || !d_work || nlines <= 0 || nlines % kLines != 0 || nrep < 1 || !(dy > 0) ||
      !std::isfinite(dt) || work_bytes < hom_ysandwich_tc_work_bytes() || ((uintptr_t)d_in % 16) ||
      ((uintptr_t)d_out % 16) || ((uintptr_t)d_work % 16))
    return HOM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the circulant C[k][j] = (1/64) sum_m e^{-i dt k_m^2 / 2} e^{2 pi i m (k - j) / 64}, in FP64
  const int ny = 64;
  std::vector<std::complex<double>> c(ny);
  for (int d = 0; d < ny; ++d) {
    std::complex<double> s(0, 0);
    for (int m = 0; m < ny; ++m) {
      const int mm = m < ny / 2 ? m : m - ny;
      const double k = 2.0 * kPiD * mm / (ny * dy);
      const double ang = -0.5 * dt * k * k + 2.0 * kPiD * (double)((m * d) % ny) / ny;
      s += std::complex<double>(std::cos(ang), std::sin(ang));
    }
    c[d] = s / (double)ny;
  }
  // B[n][k] with Y_row = X_row B^T: B[2a][2j] = Re C[a][j], B[2a][2j+1] = -Im C[a][j],
  // B[2a+1][2j] = Im C[a][j], B[2a+1][2j+1] = Re C[a][j]; three bf16 pieces
  std::vector<uint8_t> img(3 * (size_t)kPiece + 16, 0);
  for (int a = 0; a < ny; ++a)
    for (int j = 0; j < ny; ++j) {
      const std::complex<double> v = c[(a - j + ny) % ny];
      const double e[2][2] = {{v.real(), -v.imag()}, {v.imag(), v.real()}};
      for (int u = 0; u < 2; ++u)
        for (int w = 0; w < 2; ++w) {
          // split from the FP64 value: the operator is fixed, so an error in
          // its representation would act the same way every step
          const double x = e[u][w];
          const uint16_t h = bf16_bits(x);
          const double r1 = x - bf16_value(h);
          const uint16_t m = bf16_bits(r1);
          const uint16_t l = bf16_bits(r1 - bf16_value(m));
          const uint32_t off = op_offset(2 * a + u, 2 * j + w);
          const uint16_t parts[3] = {h, m, l};
          for (int p = 0; p < 3; ++p) {
            img[(size_t)p * kPiece + off] = (uint8_t)(parts[p] & 0xFF);
            img[(size_t)p * kPiece + off + 1] = (uint8_t)(parts[p] >> 8);
          }
        }
    }
  int* d_err = reinterpret_cast<int*>(static_cast<uint8_t*>(d_work) + 3 * (size_t)kPiece);
  if (cudaMemcpyAsync(d_work, img.data(), img.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) return HOM_ERR_CUDA;
  if (cudaFuncSetAttribute(ysandwich_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) != cudaSuccess)
    return HOM_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return HOM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return HOM_ERR_CUDA;
  }
  hom_status s = HOM_OK;
  float total = 0.f;
  for (int r = 0; r <= nrep && s == HOM_OK; ++r) {   // launch 0 is a warm-up
    cudaEventRecord(e0, st);
    ysandwich_tc<<<nlines / kLines, kThreads, kSmem, st>>>(d_in, d_out, static_cast<const uint4*>(d_work), d_err);
    cudaEventRecord(e1, st);
    float t = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      s = HOM_ERR_CUDA;
    if (r > 0) total += t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != HOM_OK) return s;
  int herr = 0;
  if (cudaMemcpy(&herr, d_err, sizeof herr, cudaMemcpyDeviceToHost) != cudaSuccess) return HOM_ERR_CUDA;
  if (herr) return HOM_ERR_TIMEOUT;
  if (ms) *ms = total / nrep;
  return HOM_OK;
}

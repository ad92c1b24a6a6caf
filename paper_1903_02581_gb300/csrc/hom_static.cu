// hom_static.cu -- norm and bunching probability of a batch of states with no
// device allocation by anyone: the per-block partial sums live in a fixed
// array in this library's device memory.
//
// Who needs this: a caller that holds the state in memory it was handed (a
// buffer shared by another framework, a region of a pool it does not own, a
// plugin inside a process whose allocator it must not touch) and that cannot
// call cudaMalloc or grow a workspace, e.g. because the host process forbids
// new allocations at run time or because the call runs where an allocation
// would synchronise or fail.  hom_observables needs a caller-sized workspace;
// this entry point needs only the state and an output buffer.
//
// The scratch array is a file-scope __device__ array: every GPU that loads the
// library holds it (kStaticMaxBatch * kStaticBlocks * 2 doubles = 256 KiB)
// until the process exits.  In host code its name is only a stand-in, not a
// device address, so the address is fetched with cudaGetSymbolAddress with the
// device current, on the first call made in a CUDA context, and kept per
// context: each context that loads the library has its own copy of the array
// at its own address.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hom.h"

namespace {

constexpr int kStaticMaxBatch = 64;   // simulations per call
constexpr int kStaticBlocks = 256;    // partial sums per simulation
constexpr int kStaticThreads = 256;
constexpr int kMaxContexts = 64;

static __device__ __align__(256) double g_static_scratch[kStaticMaxBatch * kStaticBlocks * 2];

// Set-up results: the array's address in each CUDA context seen so far.
struct ScratchSlot {
  CUcontext ctx;
  double* addr;
};
ScratchSlot g_slots[kMaxContexts] = {};
int g_nslots = 0;
std::mutex g_scratch_mutex;

// cuCtxGetCurrent, looked up once through the runtime (no link to the driver library).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(f);
  }
  return fn;
}

__device__ __forceinline__ double block_total(double v, double* red) {
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

// scratch[b][blk] = (sum |psi|^2, sum over x1, x2 on the same side of |psi|^2)
// over the block's share of simulation b.  Every slot is written, so nothing
// from an earlier call is read.
template <typename C>
__global__ void __launch_bounds__(kStaticThreads)
static_partials(const C* __restrict__ psi, int nx, int ny, double* __restrict__ scratch) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const size_t n = (size_t)nx * ny, per = n * n;
  const C* p = psi + (size_t)b * per;
  double s_all = 0.0, s_same = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const int r1 = (int)(i / n), r2 = (int)(i % n);
    const C v = p[i];
    const double rho = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    s_all += rho;
    if (((r1 / ny) < nx / 2) == ((r2 / ny) < nx / 2)) s_same += rho;
  }
  s_all = block_total(s_all, red);
  s_same = block_total(s_same, red);
  if (threadIdx.x == 0) {
    double* o = scratch + ((size_t)b * kStaticBlocks + blockIdx.x) * 2;
    o[0] = s_all;
    o[1] = s_same;
  }
}

// out[2b] = norm, out[2b + 1] = p_bunch of simulation b (fixed summation order).
__global__ void static_finish(const double* __restrict__ scratch, double dV, double* __restrict__ out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  for (int k = 0; k < 2; ++k) {
    double s = 0.0;
    for (int t = threadIdx.x; t < kStaticBlocks; t += blockDim.x) s += scratch[((size_t)b * kStaticBlocks + t) * 2 + k];
    s = block_total(s, red);
    if (threadIdx.x == 0) out[2 * b + k] = s * dV;
  }
}

bool pow2_between(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// Device address of the scratch array in the current context: looked up with
// cudaGetSymbolAddress on the first call in a context (the set-up), then taken
// from the table.  A context the table has no room for is looked up on every call.
hom_status scratch_address(double** out) {
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return HOM_ERR_CUDA;
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) return HOM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (ctx) {
    for (int i = 0; i < g_nslots; ++i)
      if (g_slots[i].ctx == ctx) {
        *out = g_slots[i].addr;
        return HOM_OK;
      }
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HOM_ERR_CUDA;
  // with no context current before, the runtime has just made the device's
  // primary context current
  if (!ctx && get(&ctx) != CUDA_SUCCESS) return HOM_ERR_CUDA;
  if (ctx && g_nslots < kMaxContexts) g_slots[g_nslots++] = ScratchSlot{ctx, static_cast<double*>(p)};
  *out = static_cast<double*>(p);
  return HOM_OK;
}

}  // namespace

extern "C" hom_status hom_bunching_static(const void* d_state, int32_t prec, int32_t nx, int32_t ny, int32_t batch,
                                          double dx, double dy, double* d_out, void* cuda_stream) {
  if (!d_state || !d_out) return HOM_ERR_ARG;
  if (prec != HOM_C64 && prec != HOM_C128) return HOM_ERR_ARG;
  if (!pow2_between(nx, 16, 256) || !pow2_between(ny, 16, 64)) return HOM_ERR_ARG;
  if (batch < 1 || batch > kStaticMaxBatch) return HOM_ERR_ARG;
  if (!(dx > 0) || !(dy > 0)) return HOM_ERR_ARG;
  double* scratch = nullptr;
  hom_status s = scratch_address(&scratch);
  if (s != HOM_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const dim3 grid(kStaticBlocks, batch);
  if (prec == HOM_C128)
    static_partials<double2><<<grid, kStaticThreads, 0, st>>>(static_cast<const double2*>(d_state), nx, ny, scratch);
  else
    static_partials<float2><<<grid, kStaticThreads, 0, st>>>(static_cast<const float2*>(d_state), nx, ny, scratch);
  if (cudaGetLastError() != cudaSuccess) return HOM_ERR_CUDA;
  static_finish<<<batch, kStaticThreads, 0, st>>>(scratch, dx * dx * dy * dy, d_out);
  if (cudaGetLastError() != cudaSuccess) return HOM_ERR_CUDA;
  return HOM_OK;
}

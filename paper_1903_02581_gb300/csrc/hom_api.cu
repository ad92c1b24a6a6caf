// hom_api.cu -- the C ABI of libhom (declared in include/hom.h): parameter
// checks, FP64 construction of the phase tables and of the edge packets,
// workspace layout, and the launch sequence of a Strang step.
//
// Paper: arXiv:1903.02581, Sec. II.C (Eq. evoloperat, Landau-gauge
// Hamiltonian), Appendix A (Eq. 2PTB), Eq. coulomb, Eq. screenedCoulomb,
// Eqs. pot_x and pot_xy (barrier blocks), Eq. H_effective (numerical edge
// states), Eq. twopstate, Eq. singlepwp, Eq. p_bunching, and Sec. V
// (Eq. reduced_density, the von Neumann entropy of a slice).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hom.h"
#include "hom_internal.h"

namespace {

using cd = std::complex<double>;

// An NVTX range for the lifetime of the object: every entry point that
// launches work and every kernel pass of a step is a named range, so that
// profilers can select them (ncu --nvtx --nvtx-include).  Header-only NVTX:
// without an attached tool a push or pop is a null-pointer check.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;
constexpr size_t kAlign = 256;
constexpr int kKinds = HOM_PROFILE_KINDS;   // launch kinds timed by hom_profile
constexpr int kStrategies = 3;              // step sequences (see step_sequence)

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

size_t elem_bytes(const hom_params& p) { return p.prec == HOM_C128 ? 16 : 8; }

// e^{-i theta} - 1 with theta reduced modulo 2 pi in FP64 before the sine;
// the real part is formed as -2 sin^2(theta/2), exact to rounding even when
// theta is small (the tables hold this deviation from 1, see apply_delta).
cd phase_delta(double theta) {
  const double t = std::remainder(theta, kTwoPi);
  const double h = std::sin(0.5 * t);
  return cd(-2.0 * h * h, -std::sin(t));
}

// Frequency index held at position p after the forward transform of an axis
// of length n (digit-transposed for n > 16, natural otherwise).
int freq_at(int n, int p) {
  if (n <= 16) return p;
  const int n1 = n >= 128 ? 16 : 8, n2 = n / n1;
  return p / n2 + n1 * (p % n2);
}

double wavenumber(int n, double d, int m) {
  const int s = m < n / 2 ? m : m - n;
  return kTwoPi * s / (n * d);
}

double coord(int n, double d, int j) { return (j - 0.5 * (n - 1)) * d; }

// F_tau(u) = 1 / (exp(u / tau) + 1) of Eq. pot_x, written so that the
// exponential never overflows.
double fermi_fn(double u, double tau) {
  const double z = u / tau;
  if (z > 0.0) {
    const double e = std::exp(-z);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + std::exp(z));
}

struct SimParams {
  double h, w, lam;
};

// Workspace layout: byte offsets of every region.
struct Layout {
  size_t qa[2], qt[2], gy[2], twx, twy;   // [0] = +dt, [1] = -dt
  size_t p1h[2], p1f[2], p12h[2], p12f[2];
  size_t tx, ty, v1, v12;
  size_t part_row, part_col, obs;
  size_t packets, dbeta, coef, exch, scratch;
  size_t adj_slot1, adj_slot2, adj_dv, adj_cdc, adj_out;
  size_t lam, ckpt, pong;
  size_t total;
  int tiles_row, tiles_col;
};

bool sizes_ok(const hom_params& p, std::string* why) {
  char buf[256];
  if (!pow2_in(p.nx, 16, 256) || !pow2_in(p.ny, 16, 64)) {
    snprintf(buf, sizeof buf, "nx must be a power of two in [16,256] and ny in [16,64] (got %d, %d)", p.nx, p.ny);
    if (why) *why = buf;
    return false;
  }
  if (p.prec != HOM_C64 && p.prec != HOM_C128) {
    if (why) *why = "prec must be HOM_C64 or HOM_C128";
    return false;
  }
  if (p.prec == HOM_C128 && p.nx * p.ny > 8192) {
    if (why) *why = "complex128 needs nx*ny <= 8192 (one plane in shared memory)";
    return false;
  }
  if (p.batch < 1) {
    if (why) *why = "batch must be >= 1";
    return false;
  }
  if (!(p.dx > 0) || !(p.dy > 0) || !std::isfinite(p.dx) || !std::isfinite(p.dy)) {
    if (why) *why = "dx and dy must be positive";
    return false;
  }
  if (!std::isfinite(p.dt) || p.dt == 0.0) {
    if (why) *why = "dt must be finite and non-zero";
    return false;
  }
  if (!(p.coul_soft > 0) || !std::isfinite(p.B) || !std::isfinite(p.omega_y) || !(p.qpc_w > 0) ||
      !std::isfinite(p.qpc_h) || !std::isfinite(p.coul_lambda) || !std::isfinite(p.qpc_x0)) {
    if (why) *why = "coul_soft and qpc_w must be positive; B, omega_y, qpc_h, qpc_x0, coul_lambda finite";
    return false;
  }
  if (p.ckpt_slots < 0) {
    if (why) *why = "ckpt_slots must be >= 0";
    return false;
  }
  if (!(p.coul_screen >= 0.0) || !std::isfinite(p.coul_screen)) {
    if (why) *why = "coul_screen must be finite and >= 0 (0: no screening)";
    return false;
  }
  if ((p.split != HOM_STRANG && p.split != HOM_LIE) || p.reserved != 0) {
    if (why) *why = "split must be HOM_STRANG or HOM_LIE, reserved 0";
    return false;
  }
  if (!std::isfinite(p.fermi_vb) || !std::isfinite(p.fermi_xa) || !std::isfinite(p.fermi_ya) ||
      !std::isfinite(p.fermi_xb) || !std::isfinite(p.fermi_yb) ||
      (p.fermi_vb != 0.0 && !(p.fermi_tau > 0.0 && std::isfinite(p.fermi_tau)))) {
    if (why) *why = "fermi_* must be finite, and fermi_tau > 0 when fermi_vb != 0";
    return false;
  }
  return true;
}

int tiles_of(const hom_params& p, bool col) {
  hom::GeoInfo g = p.prec == HOM_C128 ? hom::geo_info<double>(p.nx, p.ny, col) : hom::geo_info<float>(p.nx, p.ny, col);
  return g.G > 0 ? g.tiles_per_sim : 0;
}

Layout make_layout(const hom_params& p) {
  Layout L{};
  const size_t eb = elem_bytes(p);
  const size_t n = (size_t)p.nx * p.ny;
  const size_t D = (size_t)(2 * p.nx - 1) * (2 * p.ny - 1);
  const size_t B = (size_t)p.batch;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  for (int s = 0; s < 2; ++s) {
    L.qa[s] = take(n * eb);
    L.qt[s] = take(n * eb);
    L.gy[s] = take(p.ny * eb);
    L.p1h[s] = take(B * n * eb);
    L.p1f[s] = take(B * n * eb);
    L.p12h[s] = take(B * D * eb);
    L.p12f[s] = take(B * D * eb);
  }
  L.twx = take(2 * p.nx * eb);
  L.twy = take(2 * p.ny * eb);
  // observables' energy weights, in the state precision
  const size_t rb = eb / 2;
  L.tx = take(n * rb);
  L.ty = take(p.ny * rb);
  L.v1 = take(B * n * rb);
  L.v12 = take(B * D * rb);
  L.tiles_row = tiles_of(p, false);
  L.tiles_col = tiles_of(p, true);
  L.part_row = take(B * L.tiles_row * hom::NPART * 8);
  L.part_col = take(B * L.tiles_col * hom::NPART * 8);
  L.obs = take(2 * B * hom::NPART * 8);
  L.packets = take(B * 2 * n * 16);
  L.dbeta = take(B * n * 16);
  L.coef = take(B * 8);
  L.exch = take(B * 4);
  L.scratch = take(B * 8 * 8);
  L.adj_slot1 = take(B * hom::kAdjBlocks * 8);
  L.adj_slot2 = take(B * hom::kAdjBlocks * 2 * 8);
  L.adj_dv = take(B * 2 * p.nx * 8);
  L.adj_cdc = take(B * 2 * 8);
  L.adj_out = take(B * 4 * 8);
  L.lam = take(p.ckpt_slots > 0 ? B * n * n * eb : 0);
  L.ckpt = take((size_t)p.ckpt_slots * B * n * n * eb);
  L.pong = take(B * n * n * eb);
  L.total = o;
  return L;
}

std::string g_create_error = "no error";

}  // namespace

struct hom_ctx {
  hom_params p;
  char* state;
  char* ws;
  cudaStream_t stream;
  int device;
  Layout L;
  std::vector<SimParams> sims;
  std::vector<int> have_packets;    // packets set by hom_init_packets
  std::vector<int> exch;
  std::string err;
  bool poisoned;
  // instrumentation (hom_profile)
  bool prof;
  std::vector<cudaEvent_t> ev;     // event pool
  std::vector<int> ev_kind;        // per recorded pair: kind (see kNumKinds)
  size_t ev_used;
  double prof_ms[kKinds];          // transposing pass, in-place pass, transpose, double in-place pass
  long long prof_n[kKinds];
  // CUDA graphs of the forward step sequence, one per step count
  bool use_graphs;
  // autotuner: kernel variant of the transposing [0] and in-place [1] passes,
  // and the step strategy (0: transposing pass + in-place pass; 1: in-place
  // pass + transpose + in-place pass; 2: one double in-place pass + transpose
  // per step, see step_sequence)
  int variant[2];
  int strategy;
  bool tuned;
  bool tune_enabled;
  double tune_ms[2][2];             // [transposing / in-place][variant], device ms per launch
  double tune_step_ms[kStrategies]; // [strategy], estimated device ms per step
  // tensor maps of the buffers a transposing pass writes (state, transposed
  // buffer, adjoint state), per kernel variant; used where tma_store_width > 0
  CUtensorMap maps[3][2];
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;
};

namespace {

hom_status fail(hom_ctx* c, hom_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (s == HOM_ERR_CUDA || s == HOM_ERR_TIMEOUT) c->poisoned = true;
  } else {
    g_create_error = buf;
  }
  return s;
}

#define HOM_CUDA(ctx, call)                                                                          \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail((ctx), HOM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

hom_status enter(hom_ctx* c) {
  if (!c) return HOM_ERR_ARG;
  if (c->poisoned) {
    return HOM_ERR_STATE;
  }
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return fail(c, HOM_ERR_CUDA, "cudaSetDevice failed: %s", cudaGetErrorString(e));
  return HOM_OK;
}

template <typename C>
void store_complex(std::vector<unsigned char>& buf, size_t i, cd v) {
  using R = decltype(C{}.x);
  C c{(R)v.real(), (R)v.imag()};
  std::memcpy(buf.data() + i * sizeof(C), &c, sizeof(C));
}

void put(std::vector<unsigned char>& buf, bool dbl, size_t i, cd v) {
  if (dbl) store_complex<double2>(buf, i, v);
  else store_complex<float2>(buf, i, v);
}

hom_status upload(hom_ctx* c, size_t off, const void* src, size_t bytes) {
  HOM_CUDA(c, cudaMemcpyAsync(c->ws + off, src, bytes, cudaMemcpyHostToDevice, c->stream));
  return HOM_OK;
}

// Real FP64 values uploaded in the state precision (rounded once to FP32 for
// complex64) and synchronised, so the host vector may go right after.
hom_status upload_real(hom_ctx* c, size_t off, const std::vector<double>& v, bool dbl) {
  if (dbl) {
    if (hom_status s = upload(c, off, v.data(), v.size() * 8); s != HOM_OK) return s;
  } else {
    std::vector<float> f(v.begin(), v.end());
    if (hom_status s = upload(c, off, f.data(), f.size() * 4); s != HOM_OK) return s;
    HOM_CUDA(c, cudaStreamSynchronize(c->stream));
    return HOM_OK;
  }
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

// Tables shared by all simulations: kinetic phases (both signs of dt),
// twiddles, kinetic weights of the observables.
hom_status build_shared_tables(hom_ctx* c) {
  const hom_params& p = c->p;
  const bool dbl = p.prec == HOM_C128;
  const size_t eb = elem_bytes(p);
  const int nx = p.nx, ny = p.ny, n = nx * ny;
  std::vector<unsigned char> qa(n * eb), qt(n * eb), gy(ny * eb), twx(2 * nx * eb), twy(2 * ny * eb);
  std::vector<double> tx(n), ty(ny);
  for (int sgn = 0; sgn < 2; ++sgn) {
    const double dt = sgn == 0 ? p.dt : -p.dt;
    for (int px = 0; px < nx; ++px) {
      const double k = wavenumber(nx, p.dx, freq_at(nx, px));
      for (int j = 0; j < ny; ++j) {
        const double y = coord(ny, p.dy, j);
        const double t = 0.5 * (k - p.B * y) * (k - p.B * y);
        // Strang: e^{-i (dt/2) T_x} - 1 on both sides of the y sandwich;
        // Lie: the full step e^{-i dt T_x} - 1 before it and nothing after
        const bool lie = p.split == HOM_LIE;
        const cd q = phase_delta((lie ? 1.0 : 0.5) * dt * t);
        put(qa, dbl, (size_t)px * ny + j, q);
        // after the y sandwich, with the 1/(nx ny) of both inverse transforms
        // folded in (a power of two: the scaled delta is exact)
        put(qt, dbl, (size_t)j * nx + px, lie ? cd(0.0, 0.0) : q / ((double)nx * ny));
        if (sgn == 0) tx[(size_t)px * ny + j] = t;
      }
    }
    for (int py = 0; py < ny; ++py) {
      const double k = wavenumber(ny, p.dy, freq_at(ny, py));
      put(gy, dbl, py, phase_delta(dt * 0.5 * k * k));       // e^{-i dt T_y} - 1
      if (sgn == 0) ty[py] = 0.5 * k * k;
    }
    hom_status s;
    if ((s = upload(c, c->L.qa[sgn], qa.data(), qa.size())) != HOM_OK) return s;
    if ((s = upload(c, c->L.qt[sgn], qt.data(), qt.size())) != HOM_OK) return s;
    if ((s = upload(c, c->L.gy[sgn], gy.data(), gy.size())) != HOM_OK) return s;
    HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  // twiddles e^{-2 pi i j / n} as interleaved (hi, lo) pairs (lo = 0 in FP64)
  auto twiddles = [&](std::vector<unsigned char>& buf, int nn) {
    for (int j = 0; j < nn; ++j) {
      const double a = kTwoPi * j / nn;
      const cd w(std::cos(a), -std::sin(a));
      const cd hi = dbl ? w : cd((float)w.real(), (float)w.imag());
      put(buf, dbl, 2 * j, hi);
      put(buf, dbl, 2 * j + 1, dbl ? cd(0, 0) : w - hi);
    }
  };
  twiddles(twx, nx);
  twiddles(twy, ny);
  hom_status s;
  if ((s = upload(c, c->L.twx, twx.data(), twx.size())) != HOM_OK) return s;
  if ((s = upload(c, c->L.twy, twy.data(), twy.size())) != HOM_OK) return s;
  if ((s = upload_real(c, c->L.tx, tx, dbl)) != HOM_OK) return s;
  if ((s = upload_real(c, c->L.ty, ty, dbl)) != HOM_OK) return s;
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

// Per-simulation potential tables: e^{-i tau V1}, e^{-i tau V12} for
// tau = +-dt/2, +-dt, and the real V1, V12 for the observables.
hom_status build_sim_tables(hom_ctx* c, int b) {
  const hom_params& p = c->p;
  const SimParams& sp = c->sims[b];
  const bool dbl = p.prec == HOM_C128;
  const size_t eb = elem_bytes(p);
  const int nx = p.nx, ny = p.ny, n = nx * ny;
  const int dny = 2 * ny - 1;
  const size_t D = (size_t)(2 * nx - 1) * dny;
  std::vector<double> v1(n), v12(D);
  for (int ix = 0; ix < nx; ++ix) {
    const double x = coord(nx, p.dx, ix);
    const double g = std::exp(-(x - p.qpc_x0) * (x - p.qpc_x0) / (2.0 * sp.w * sp.w));
    for (int iy = 0; iy < ny; ++iy) {
      const double y = coord(ny, p.dy, iy);
      double v = 0.5 * p.omega_y * p.omega_y * y * y + sp.h * g;
      if (p.fermi_vb != 0.0)   // the two blocks of Eq. pot_xy
        v += p.fermi_vb * (fermi_fn(x - p.fermi_xa, p.fermi_tau) * fermi_fn(y - p.fermi_ya, p.fermi_tau) +
                           fermi_fn(p.fermi_xb - x, p.fermi_tau) * fermi_fn(p.fermi_yb - y, p.fermi_tau));
      v1[(size_t)ix * ny + iy] = v;
    }
  }
  for (int ddx = -(nx - 1); ddx <= nx - 1; ++ddx) {
    for (int ddy = -(ny - 1); ddy <= ny - 1; ++ddy) {
      const double rx = ddx * p.dx, ry = ddy * p.dy, r2 = rx * rx + ry * ry;
      double v = sp.lam / std::sqrt(r2 + p.coul_soft * p.coul_soft);
      if (p.coul_screen > 0.0) v *= std::exp(-std::sqrt(r2) / p.coul_screen);   // Eq. screenedCoulomb
      v12[(size_t)(ddx + nx - 1) * dny + (ddy + ny - 1)] = v;
    }
  }
  std::vector<unsigned char> t1(n * eb), t12(D * eb);
  for (int sgn = 0; sgn < 2; ++sgn) {
    const double dt = sgn == 0 ? p.dt : -p.dt;
    for (int half = 0; half < 2; ++half) {
      const double tau = half ? 0.5 * dt : dt;
      for (int i = 0; i < n; ++i) put(t1, dbl, i, phase_delta(tau * v1[i]));
      for (size_t i = 0; i < D; ++i) put(t12, dbl, i, phase_delta(tau * v12[i]));
      const size_t o1 = (half ? c->L.p1h[sgn] : c->L.p1f[sgn]) + (size_t)b * n * eb;
      const size_t o12 = (half ? c->L.p12h[sgn] : c->L.p12f[sgn]) + (size_t)b * D * eb;
      hom_status s;
      if ((s = upload(c, o1, t1.data(), t1.size())) != HOM_OK) return s;
      if ((s = upload(c, o12, t12.data(), t12.size())) != HOM_OK) return s;
      HOM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
  }
  hom_status s;
  const size_t rb = dbl ? 8 : 4;
  if ((s = upload_real(c, c->L.v1 + (size_t)b * n * rb, v1, dbl)) != HOM_OK) return s;
  if ((s = upload_real(c, c->L.v12 + (size_t)b * D * rb, v12, dbl)) != HOM_OK) return s;
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

// Edge packet of Eq. (singlepwp): sum over the grid wavenumbers k of
// e^{-sigma^2 (k-k0)^2} e^{i k (x - x0)} phi_k(y), phi_k the lowest hybrid
// level of the parabolic edge, (Omega/pi)^{1/4} e^{-Omega (y - k B/Omega^2)^2 / 2},
// Omega^2 = B^2 + omega^2; normalised so that sum |psi|^2 dx dy = 1.  With
// dpsi != nullptr also returns d psi / d x0 (the norm does not depend on x0).
// Eigenpairs of a real symmetric matrix (row-major, overwritten) by the
// cyclic Jacobi method, with the rotations accumulated into v (row-major,
// columns are eigenvectors).  Returns the eigenvalues.
std::vector<double> symmetric_eigen(std::vector<double>& a, int n, std::vector<double>& v) {
  auto A = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += A(i, j) * A(i, j);
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A(p, q);
        if (apq == 0.0) continue;
        const double th = (A(q, q) - A(p, p)) / (2.0 * apq);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          if (k == p || k == q) continue;
          const double akp = A(k, p), akq = A(k, q);
          A(k, p) = A(p, k) = cs * akp - sn * akq;
          A(k, q) = A(q, k) = sn * akp + cs * akq;
        }
        A(p, p) -= t * apq;
        A(q, q) += t * apq;
        A(p, q) = A(q, p) = 0.0;
        for (int k = 0; k < n; ++k) {
          const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = cs * vkp - sn * vkq;
          v[(size_t)k * n + q] = sn * vkp + cs * vkq;
        }
      }
    }
  }
  std::vector<double> ev(n);
  for (int i = 0; i < n; ++i) ev[i] = A(i, i);
  return ev;
}

// Lowest eigenvector of Eq. H_effective at wavevector k on the y grid (see
// hom_packet): normalised to sum phi^2 dy = 1, largest component positive.
void numeric_edge_state(const hom_params& p, double k, double wall_y, int wall_side, std::vector<double>& phi) {
  const int ny = p.ny;
  std::vector<double> h((size_t)ny * ny), vec;
  // spectral -1/2 d^2/dy^2: (1/ny) sum_m 1/2 k_m^2 cos(2 pi m (j - l) / ny)
  std::vector<double> row(ny, 0.0);
  for (int d = 0; d < ny; ++d) {
    double acc = 0.0;
    for (int m = 0; m < ny; ++m) {
      const double km = wavenumber(ny, p.dy, m);
      acc += 0.5 * km * km * std::cos(kTwoPi * (double)m * d / ny);
    }
    row[d] = acc / ny;
  }
  for (int j = 0; j < ny; ++j)
    for (int l = 0; l < ny; ++l) h[(size_t)j * ny + l] = row[(j - l + ny) % ny];
  for (int j = 0; j < ny; ++j) {
    const double y = coord(ny, p.dy, j);
    double d = 0.5 * (k - p.B * y) * (k - p.B * y) + 0.5 * p.omega_y * p.omega_y * y * y;
    if (p.fermi_vb != 0.0) d += p.fermi_vb * fermi_fn(wall_side * (y - wall_y), p.fermi_tau);
    h[(size_t)j * ny + j] += d;
  }
  const std::vector<double> ev = symmetric_eigen(h, ny, vec);
  int lo = 0;
  for (int i = 1; i < ny; ++i)
    if (ev[i] < ev[lo]) lo = i;
  phi.assign(ny, 0.0);
  double nrm = 0.0, big = 0.0;
  int at = 0;
  for (int j = 0; j < ny; ++j) {
    phi[j] = vec[(size_t)j * ny + lo];
    nrm += phi[j] * phi[j];
    if (std::fabs(phi[j]) > big) {
      big = std::fabs(phi[j]);
      at = j;
    }
  }
  const double sc = (phi[at] < 0 ? -1.0 : 1.0) / std::sqrt(nrm * p.dy);
  for (double& x : phi) x *= sc;
}

hom_status build_packet(hom_ctx* c, const hom_packet& pk, std::vector<cd>& psi, std::vector<cd>* dpsi) {
  const hom_params& p = c->p;
  const int nx = p.nx, ny = p.ny;
  const double Om = std::sqrt(p.B * p.B + p.omega_y * p.omega_y);
  if (!std::isfinite(pk.x0) || !(pk.sigma > 0) || !std::isfinite(pk.sigma))
    return fail(c, HOM_ERR_ARG, "packet needs finite x0 and sigma > 0");
  if (Om <= 0) return fail(c, HOM_ERR_ARG, "packets need B != 0 or omega_y != 0");
  if (pk.numeric) {
    if (!pk.by_k0) return fail(c, HOM_ERR_ARG, "numerical edge states need k0 (by_k0)");
    if (pk.wall_side != 1 && pk.wall_side != -1) return fail(c, HOM_ERR_ARG, "wall_side must be +1 or -1");
    if (!std::isfinite(pk.wall_y)) return fail(c, HOM_ERR_ARG, "wall_y must be finite");
  }
  double k0;
  if (pk.by_k0) {
    if (!std::isfinite(pk.k0)) return fail(c, HOM_ERR_ARG, "k0 must be finite");
    k0 = pk.k0;
  } else {
    if (!(p.omega_y > 0)) return fail(c, HOM_ERR_ARG, "an energy needs omega_y > 0 (or give k0 with by_k0)");
    if (!(pk.energy >= 0.5 * Om) || !std::isfinite(pk.energy))
      return fail(c, HOM_ERR_ARG, "energy %g below the lowest hybrid level %g", pk.energy, 0.5 * Om);
    if (pk.dir != 1 && pk.dir != -1) return fail(c, HOM_ERR_ARG, "dir must be +1 or -1");
    k0 = pk.dir * Om * std::sqrt(2.0 * (pk.energy - 0.5 * Om)) / p.omega_y;
  }
  psi.assign((size_t)nx * ny, cd(0, 0));
  if (dpsi) dpsi->assign((size_t)nx * ny, cd(0, 0));
  std::vector<double> chi(ny);
  for (int m = 0; m < nx; ++m) {
    const double k = wavenumber(nx, p.dx, m);
    const double wk = std::exp(-pk.sigma * pk.sigma * (k - k0) * (k - k0));
    if (wk < 1e-300) continue;
    if (pk.numeric) {
      numeric_edge_state(p, k, pk.wall_y, pk.wall_side, chi);
    } else {
      const double yk = k * p.B / (Om * Om);
      for (int j = 0; j < ny; ++j) {
        const double y = coord(ny, p.dy, j) - yk;
        chi[j] = std::pow(Om / kPi, 0.25) * std::exp(-0.5 * Om * y * y);
      }
    }
    for (int ix = 0; ix < nx; ++ix) {
      const double arg = std::fmod(k * (coord(nx, p.dx, ix) - pk.x0), kTwoPi);
      const cd e = wk * cd(std::cos(arg), std::sin(arg));
      for (int j = 0; j < ny; ++j) {
        psi[(size_t)ix * ny + j] += e * chi[j];
        if (dpsi) (*dpsi)[(size_t)ix * ny + j] += cd(0, -k) * e * chi[j];
      }
    }
  }
  double s = 0;
  for (const cd& v : psi) s += std::norm(v);
  s *= p.dx * p.dy;
  if (!(s > 0)) return fail(c, HOM_ERR_ARG, "packet has zero norm on this grid");
  const double inv = 1.0 / std::sqrt(s);
  for (cd& v : psi) v *= inv;
  if (dpsi)
    for (cd& v : *dpsi) v *= inv;
  return HOM_OK;
}

constexpr size_t kEventPool = 4096;

// Sum the elapsed times of the recorded event pairs (the stream is synchronised).
hom_status harvest_events(hom_ctx* c) {
  if (c->ev_used == 0) return HOM_OK;
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    HOM_CUDA(c, cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
    const int k = c->ev_kind[i / 2];
    c->prof_ms[k] += ms;
    c->prof_n[k] += 1;
  }
  c->ev_used = 0;
  c->ev_kind.clear();
  return HOM_OK;
}

hom_status prof_begin(hom_ctx* c, size_t* idx) {
  if (c->ev_used + 2 > c->ev.size()) {
    hom_status s = harvest_events(c);
    if (s != HOM_OK) return s;
  }
  *idx = c->ev_used;
  HOM_CUDA(c, cudaEventRecord(c->ev[c->ev_used], c->stream));
  return HOM_OK;
}

hom_status prof_end(hom_ctx* c, size_t idx, int kind) {
  HOM_CUDA(c, cudaEventRecord(c->ev[idx + 1], c->stream));
  c->ev_used = idx + 2;
  c->ev_kind.push_back(kind);
  return HOM_OK;
}

// One Strang step applies one kinetic sandwich per particle; the two commute,
// so either goes first.  The state lives in psi = psi[r1][r2] (layout A) or,
// between steps, in the workspace buffer as psi[r2][r1] (layout B).  A
// sandwich works on the rows of a layout (the planes of one particle), so the
// other particle's sandwich needs the state transposed.  The potential phase
// (dt/2 on the first step, dt between steps: the halves of neighbouring steps
// fused) is applied on a load, the closing dt/2 on the last store.  Three
// ways of sequencing the passes (c->strategy):
//   0: a transposing pass (rows of one layout in, the other layout out), then
//      an in-place pass there; the state alternates between the layouts and
//      an odd count ends with a second transposing pass back to A;
//   1: an in-place pass, a plain transpose, an in-place pass;
//   2: steps overlap: after the first sandwich, each transpose is followed by
//      one double in-place pass holding this step's second sandwich, the
//      potential of the full step and the next step's first sandwich, all of
//      the same particle (so two HBM round trips per step); the last step
//      ends with a single in-place pass (and a transpose back to A if needed).
// All three apply the same arithmetic to every element in the same order.
template <typename T>
hom_status step_sequence(hom_ctx* c, char* psi, int nsteps, int sgn) {
  using C = typename hom::Cx<T>::type;
  const hom_params& p = c->p;
  const C* qa = reinterpret_cast<const C*>(c->ws + c->L.qa[sgn]);
  const C* qt = reinterpret_cast<const C*>(c->ws + c->L.qt[sgn]);
  const C* gy = reinterpret_cast<const C*>(c->ws + c->L.gy[sgn]);
  const C* twx = reinterpret_cast<const C*>(c->ws + c->L.twx);
  const C* twy = reinterpret_cast<const C*>(c->ws + c->L.twy);
  const C* p1h = reinterpret_cast<const C*>(c->ws + c->L.p1h[sgn]);
  const C* p1f = reinterpret_cast<const C*>(c->ws + c->L.p1f[sgn]);
  const C* p12h = reinterpret_cast<const C*>(c->ws + c->L.p12h[sgn]);
  const C* p12f = reinterpret_cast<const C*>(c->ws + c->L.p12f[sgn]);
  C* A = reinterpret_cast<C*>(psi);
  C* Bp = reinterpret_cast<C*>(c->ws + c->L.pong);
  bool in_a = true;
  // The potential before the first step and after the last: dt/2 each
  // (Strang), or none before and the full step after (Lie: K then V per step).
  const bool lie = p.split == HOM_LIE;
  const int v_first = lie ? 0 : 1;
  const C* first1 = lie ? p1f : p1h;
  const C* first12 = lie ? p12f : p12h;
  const C* last1 = lie ? p1f : p1h;
  const C* last12 = lie ? p12f : p12h;
  auto transposing = [&](C* src, C* dst, int v_load, int v_store, const C* t1, const C* t12) -> hom_status {
    hom::PassArgsT<C> a{};
    const char* d = reinterpret_cast<const char*>(dst);
    const int bi = d == c->state ? 0 : (d == c->ws + c->L.pong ? 1 : 2);
    a.tmap_dst = c->maps[bi][c->variant[0]];
    a.src = src;
    a.dst = dst;
    a.qa = qa;
    a.qt = qt;
    a.gy = gy;
    a.twx = twx;
    a.twy = twy;
    a.p1 = t1;
    a.p12 = t12;
    a.v_load = v_load;
    a.v_store = v_store;
    size_t ev = 0;
    hom_status st;
    if (c->prof && (st = prof_begin(c, &ev)) != HOM_OK) return st;
    NvtxRange r("hom.transposing_pass");
    HOM_CUDA(c, (hom::launch_kinetic_t<T>(p.nx, p.ny, c->variant[0], a, p.batch, c->stream)));
    if (c->prof && (st = prof_end(c, ev, 0)) != HOM_OK) return st;
    return HOM_OK;
  };
  auto in_place_v = [&](C* buf, int v_load, int v_store, const C* t1, const C* t12) -> hom_status {
    hom::PassArgs<C> a{};
    a.psi = buf;
    a.qa = qa;
    a.qt = qt;
    a.gy = gy;
    a.twx = twx;
    a.twy = twy;
    a.p1 = t1;
    a.p12 = t12;
    a.v_load = v_load;
    a.v_store = v_store;
    size_t ev = 0;
    hom_status st;
    if (c->prof && (st = prof_begin(c, &ev)) != HOM_OK) return st;
    NvtxRange r("hom.in_place_pass");
    HOM_CUDA(c, (hom::launch_kinetic<T>(p.nx, p.ny, c->variant[1], a, p.batch, c->stream)));
    if (c->prof && (st = prof_end(c, ev, 1)) != HOM_OK) return st;
    return HOM_OK;
  };
  auto in_place = [&](C* buf, int v_store, const C* t1, const C* t12) -> hom_status {
    return in_place_v(buf, 0, v_store, t1, t12);
  };
  auto transpose = [&](C* src, C* dst) -> hom_status {
    size_t ev = 0;
    hom_status st;
    if (c->prof && (st = prof_begin(c, &ev)) != HOM_OK) return st;
    NvtxRange r("hom.transpose");
    HOM_CUDA(c, (hom::launch_transpose<T>(src, dst, p.nx * p.ny, p.batch, c->stream)));
    if (c->prof && (st = prof_end(c, ev, 2)) != HOM_OK) return st;
    return HOM_OK;
  };
  auto double_in_place = [&](C* buf) -> hom_status {
    hom::PassArgs<C> a{};
    a.psi = buf;
    a.qa = qa;
    a.qt = qt;
    a.gy = gy;
    a.twx = twx;
    a.twy = twy;
    a.p1 = p1h;
    a.p12 = p12h;
    a.p1m = p1f;
    a.p12m = p12f;
    a.v_load = 0;
    a.v_store = 0;
    size_t ev = 0;
    hom_status st;
    if (c->prof && (st = prof_begin(c, &ev)) != HOM_OK) return st;
    NvtxRange r("hom.double_pass");
    HOM_CUDA(c, (hom::launch_kinetic2<T>(p.nx, p.ny, c->variant[1], a, p.batch, c->stream)));
    if (c->prof && (st = prof_end(c, ev, 3)) != HOM_OK) return st;
    return HOM_OK;
  };
  if (c->strategy == 2) {
    hom_status st = in_place_v(A, v_first, 0, first1, first12);
    if (st != HOM_OK) return st;
    for (int s = 0; s < nsteps; ++s) {
      C* cur = in_a ? A : Bp;
      C* oth = in_a ? Bp : A;
      if ((st = transpose(cur, oth)) != HOM_OK) return st;
      in_a = !in_a;
      if (s < nsteps - 1) {
        st = double_in_place(oth);
      } else {
        st = in_place_v(oth, 0, 1, last1, last12);
        if (st == HOM_OK && !in_a) st = transpose(Bp, A);
      }
      if (st != HOM_OK) return st;
    }
    return HOM_OK;
  }
  if (c->strategy == 1) {
    // in-place pass (potential phase at load), transpose, in-place pass
    for (int s = 0; s < nsteps; ++s) {
      const bool last = s == nsteps - 1;
      C* cur = in_a ? A : Bp;
      C* oth = in_a ? Bp : A;
      hom_status st = in_place_v(cur, s == 0 ? v_first : 1, 0, s == 0 ? first1 : p1f, s == 0 ? first12 : p12f);
      if (st != HOM_OK) return st;
      if ((st = transpose(cur, oth)) != HOM_OK) return st;
      in_a = !in_a;
      if (last && !in_a) {
        // the other particle's sandwich on the way back to the caller's layout
        if ((st = transposing(Bp, A, 0, 1, last1, last12)) != HOM_OK) return st;
        in_a = true;
      } else if ((st = in_place_v(oth, 0, last ? 1 : 0, last1, last12)) != HOM_OK) {
        return st;
      }
    }
    return HOM_OK;
  }
  for (int s = 0; s < nsteps; ++s) {
    const bool last = s == nsteps - 1;
    hom_status st = transposing(in_a ? A : Bp, in_a ? Bp : A, s == 0 ? v_first : 1, 0, s == 0 ? first1 : p1f,
                                s == 0 ? first12 : p12f);
    if (st != HOM_OK) return st;
    in_a = !in_a;
    if (last && !in_a) {
      st = transposing(Bp, A, 0, 1, last1, last12);
      in_a = true;
    } else {
      st = in_place(in_a ? A : Bp, last ? 1 : 0, last1, last12);
    }
    if (st != HOM_OK) return st;
  }
  return HOM_OK;
}

// nsteps steps on psi with time step +dt (sgn 0) or -dt (sgn 1).
hom_status run_steps(hom_ctx* c, char* psi, int nsteps, int sgn) {
  return c->p.prec == HOM_C128 ? step_sequence<double>(c, psi, nsteps, sgn)
                               : step_sequence<float>(c, psi, nsteps, sgn);
}

// Autotuner: the kernel variants of a pass (Geo, variant 0 or 1) differ only
// in thread counts and cluster widths, and the step strategies only in where
// the transposition happens, so every element of the state sees the same
// arithmetic and the results are bitwise identical.  The first forward
// hom_step call with at least kTuneMinSteps steps runs three trials on the
// real state, each two steps to warm up and two timed steps (CUDA events
// around every launch): strategy 0 with all passes in variant 0, the same in
// variant 1, and strategy 2 with the faster variant of each pass.  From the
// average launch times it estimates the steady-state step of each strategy
// (0: transposing + in-place pass; 1: two in-place passes + transpose; 2:
// double in-place pass + transpose) and keeps the fastest.  The 12 steps of
// the trials are part of the requested steps.
constexpr int kTuneMinSteps = 24;

hom_status autotune(hom_ctx* c) {
  NvtxRange range("hom_autotune");
  const bool prof_saved = c->prof;
  double ms_saved[kKinds];
  long long n_saved[kKinds];
  for (int k = 0; k < kKinds; ++k) {
    ms_saved[k] = c->prof_ms[k];
    n_saved[k] = c->prof_n[k];
  }
  hom_status s;
  if ((s = harvest_events(c)) != HOM_OK) return s;
  if (c->ev.empty()) {
    c->ev.resize(kEventPool, nullptr);
    for (auto& e : c->ev) HOM_CUDA(c, cudaEventCreate(&e));
  }
  // two untimed then two timed steps of a configuration; average ms per launch of each kind
  auto trial = [&](int strategy, int v0, int v1, double* avg) -> hom_status {
    c->strategy = strategy;
    c->variant[0] = v0;
    c->variant[1] = v1;
    c->prof = false;
    hom_status st;
    if ((st = run_steps(c, c->state, 2, 0)) != HOM_OK) return st;
    c->prof = true;
    for (int k = 0; k < kKinds; ++k) {
      c->prof_ms[k] = 0.0;
      c->prof_n[k] = 0;
    }
    if ((st = run_steps(c, c->state, 2, 0)) != HOM_OK) return st;
    if ((st = harvest_events(c)) != HOM_OK) return st;
    for (int k = 0; k < kKinds; ++k) avg[k] = c->prof_n[k] > 0 ? c->prof_ms[k] / (double)c->prof_n[k] : 0.0;
    return HOM_OK;
  };
  double avg[kKinds];
  for (int v = 0; v < 2; ++v) {
    if ((s = trial(0, v, v, avg)) != HOM_OK) return s;
    c->tune_ms[0][v] = avg[0];
    c->tune_ms[1][v] = avg[1];
  }
  const int v0 = c->tune_ms[0][1] < c->tune_ms[0][0] ? 1 : 0;
  const int v1 = c->tune_ms[1][1] < c->tune_ms[1][0] ? 1 : 0;
  if ((s = trial(2, v0, v1, avg)) != HOM_OK) return s;
  c->tune_step_ms[0] = c->tune_ms[0][v0] + c->tune_ms[1][v1];
  c->tune_step_ms[1] = 2.0 * c->tune_ms[1][v1] + avg[2];
  c->tune_step_ms[2] = avg[3] + avg[2];
  int best = 0;
  for (int k = 1; k < kStrategies; ++k)
    if (c->tune_step_ms[k] < c->tune_step_ms[best]) best = k;
  c->strategy = best;
  c->variant[0] = v0;
  c->variant[1] = v1;
  c->prof = prof_saved;
  for (int k = 0; k < kKinds; ++k) {
    c->prof_ms[k] = ms_saved[k];
    c->prof_n[k] = n_saved[k];
  }
  c->tuned = true;
  return HOM_OK;
}

constexpr size_t kMaxGraphs = 8;

void drop_graphs(hom_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
  c->graphs.clear();
}

// The forward sequence of nsteps steps on the state as one CUDA graph: the
// 2*nsteps kinetic-pass launches are captured once per step count and
// replayed with a single launch.
hom_status run_steps_graph(hom_ctx* c, int nsteps) {
  for (auto& g : c->graphs)
    if (g.first == nsteps) {
      HOM_CUDA(c, cudaGraphLaunch(g.second, c->stream));
      return HOM_OK;
    }
  if (c->graphs.size() >= kMaxGraphs) drop_graphs(c);
  HOM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  hom_status s = run_steps(c, c->state, nsteps, 0);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (s != HOM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(c, HOM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(c, HOM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  c->graphs.emplace_back(nsteps, exec);
  HOM_CUDA(c, cudaGraphLaunch(exec, c->stream));
  return HOM_OK;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to the
// driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor maps for the transposed stores: each buffer seen as [batch*n rows]
// [n columns] of 8-byte elements, box of w columns x ny rows.
hom_status build_tensor_maps(hom_ctx* c) {
  const hom_params& p = c->p;
  std::memset(c->maps, 0, sizeof c->maps);
  if (p.prec != HOM_C64) return HOM_OK;
  const int w[2] = {hom::tma_store_width<float>(p.nx, p.ny, 0), hom::tma_store_width<float>(p.nx, p.ny, 1)};
  if (w[0] == 0 && w[1] == 0) return HOM_OK;
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(c, HOM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const cuuint64_t n = (cuuint64_t)p.nx * p.ny;
  char* bufs[3] = {c->state, c->ws + c->L.pong, p.ckpt_slots > 0 ? c->ws + c->L.lam : nullptr};
  for (int bi = 0; bi < 3; ++bi) {
    if (!bufs[bi]) continue;
    for (int v = 0; v < 2; ++v) {
      if (w[v] == 0) continue;
      const cuuint64_t dims[2] = {n, n * (cuuint64_t)p.batch};
      const cuuint64_t strides[1] = {n * 8};
      const cuuint32_t box[2] = {(cuuint32_t)w[v], (cuuint32_t)p.ny};
      const cuuint32_t estr[2] = {1, 1};
      CUresult r = encode(&c->maps[bi][v], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, bufs[bi], dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(c, HOM_ERR_CUDA, "tensor map encoding failed (%d)", (int)r);
    }
  }
  return HOM_OK;
}

template <typename T>
hom_status measure_launch(hom_ctx* c) {
  using C = typename hom::Cx<T>::type;
  const hom_params& p = c->p;
  hom::MeasureArgs<C> m{};
  m.psi = reinterpret_cast<const C*>(c->state);
  m.twx = reinterpret_cast<const C*>(c->ws + c->L.twx);
  m.twy = reinterpret_cast<const C*>(c->ws + c->L.twy);
  m.tx = reinterpret_cast<const T*>(c->ws + c->L.tx);
  m.ty = reinterpret_cast<const T*>(c->ws + c->L.ty);
  m.v1 = reinterpret_cast<const T*>(c->ws + c->L.v1);
  m.v12 = reinterpret_cast<const T*>(c->ws + c->L.v12);
  double* obs = reinterpret_cast<double*>(c->ws + c->L.obs);
  m.partial = reinterpret_cast<double*>(c->ws + c->L.part_row);
  HOM_CUDA(c, (hom::launch_measure<T>(p.nx, p.ny, false, m, p.batch, c->stream)));
  HOM_CUDA(c, hom::launch_reduce(m.partial, c->L.tiles_row, p.batch, obs, c->stream));
  m.partial = reinterpret_cast<double*>(c->ws + c->L.part_col);
  HOM_CUDA(c, (hom::launch_measure<T>(p.nx, p.ny, true, m, p.batch, c->stream)));
  HOM_CUDA(c, hom::launch_reduce(m.partial, c->L.tiles_col, p.batch, obs + (size_t)p.batch * hom::NPART, c->stream));
  return HOM_OK;
}

}  // namespace

// Eigenvalues of a Hermitian matrix (row-major, overwritten) by the cyclic
// Jacobi method: each rotation first turns the (p, q) element real with a
// diagonal phase, then zeroes it with a real plane rotation.  Both are unitary
// similarities, so the spectrum is kept; the off-diagonal mass falls
// quadratically once small.
std::vector<double> hermitian_eigenvalues(std::vector<cd>& a, int n) {
  auto at = [&](int i, int j) -> cd& { return a[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += std::norm(at(i, j));
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const cd apq = at(p, q);
        const double r = std::abs(apq);
        if (r == 0.0) continue;
        const cd e = apq / r;
        const double app = at(p, p).real(), aqq = at(q, q).real();
        const double th = (aqq - app) / (2.0 * r);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {
          if (k == p || k == q) continue;
          const cd bkp = at(k, p), bkq = at(k, q) * std::conj(e);
          const cd nkp = c * bkp - sn * bkq, nkq = sn * bkp + c * bkq;
          at(k, p) = nkp;
          at(p, k) = std::conj(nkp);
          at(k, q) = nkq;
          at(q, k) = std::conj(nkq);
        }
        at(p, p) = cd(app - t * r, 0.0);
        at(q, q) = cd(aqq + t * r, 0.0);
        at(p, q) = at(q, p) = cd(0.0, 0.0);
      }
    }
  }
  std::vector<double> ev(n);
  for (int i = 0; i < n; ++i) ev[i] = at(i, i).real();
  return ev;
}

// Von Neumann entropy of the renormalised slice phi (m1 x m2, row-major):
// the eigenvalues of phi phi^dagger and of phi^dagger phi are the same apart
// from zeros, so the smaller Gram matrix is diagonalised.  Returns false if
// the slice is zero.
bool slice_entropy(const cd* phi, int m1, int m2, double* entropy, double* weight) {
  double w = 0.0;
  for (size_t k = 0; k < (size_t)m1 * m2; ++k) w += std::norm(phi[k]);
  if (weight) *weight = w;
  if (!(w > 0.0) || !std::isfinite(w)) return false;
  const bool rows = m1 <= m2;
  const int g = rows ? m1 : m2;
  std::vector<cd> gram((size_t)g * g);
  for (int i = 0; i < g; ++i) {
    for (int j = i; j < g; ++j) {
      cd acc(0.0, 0.0);
      if (rows) {
        for (int k = 0; k < m2; ++k) acc += phi[(size_t)i * m2 + k] * std::conj(phi[(size_t)j * m2 + k]);
      } else {
        for (int k = 0; k < m1; ++k) acc += std::conj(phi[(size_t)k * m2 + i]) * phi[(size_t)k * m2 + j];
      }
      acc /= w;
      gram[(size_t)i * g + j] = acc;
      gram[(size_t)j * g + i] = std::conj(acc);
    }
    gram[(size_t)i * g + i] = cd(gram[(size_t)i * g + i].real(), 0.0);
  }
  const std::vector<double> ev = hermitian_eigenvalues(gram, g);
  double sum = 0.0;
  for (double l : ev)
    if (l > 0.0) sum -= l * std::log(l);
  *entropy = sum;
  return true;
}

extern "C" {

size_t hom_state_bytes(const hom_params* p) {
  if (!p || !sizes_ok(*p, nullptr)) return 0;
  const size_t n = (size_t)p->nx * p->ny;
  return (size_t)p->batch * n * n * elem_bytes(*p);
}

size_t hom_workspace_bytes(const hom_params* p) {
  if (!p || !sizes_ok(*p, nullptr)) return 0;
  return make_layout(*p).total;
}

hom_status hom_create(const hom_params* p, void* d_state, void* d_workspace, size_t workspace_bytes,
                      void* cuda_stream, hom_ctx** out) {
  if (!out) return fail(nullptr, HOM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!p) return fail(nullptr, HOM_ERR_ARG, "params is NULL");
  std::string why;
  if (!sizes_ok(*p, &why)) return fail(nullptr, HOM_ERR_ARG, "%s", why.c_str());
  if (!d_state || !d_workspace) return fail(nullptr, HOM_ERR_ARG, "state and workspace pointers must be non-NULL");
  if (((uintptr_t)d_state % kAlign) || ((uintptr_t)d_workspace % kAlign))
    return fail(nullptr, HOM_ERR_ARG, "state and workspace must be %zu-byte aligned", kAlign);
  const Layout L = make_layout(*p);
  if (workspace_bytes < L.total)
    return fail(nullptr, HOM_ERR_NOMEM, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes,
                L.total);
  if (L.tiles_row <= 0 || L.tiles_col <= 0) return fail(nullptr, HOM_ERR_ARG, "unsupported grid");
  hom_ctx* c = new (std::nothrow) hom_ctx();
  if (!c) return fail(nullptr, HOM_ERR_NOMEM, "host allocation failed");
  c->p = *p;
  c->state = static_cast<char*>(d_state);
  c->ws = static_cast<char*>(d_workspace);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->L = L;
  c->poisoned = false;
  c->err = "no error";
  c->prof = false;
  c->ev_used = 0;
  for (int k = 0; k < kKinds; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_n[k] = 0;
  }
  {
    const char* g = getenv("HOM_GRAPHS");
    c->use_graphs = !(g && g[0] == '0');
    const char* tu = getenv("HOM_TUNE");
    c->tune_enabled = !(tu && tu[0] == '0');
    c->variant[0] = c->variant[1] = 0;
    c->strategy = 0;
    c->tuned = false;
    for (auto& r : c->tune_ms) r[0] = r[1] = 0.0;
    for (auto& t : c->tune_step_ms) t = 0.0;
  }
  c->sims.assign(p->batch, SimParams{p->qpc_h, p->qpc_w, p->coul_lambda});
  c->have_packets.assign(p->batch, 0);
  c->exch.assign(p->batch, -1);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, HOM_ERR_CUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  }
  e = p->prec == HOM_C128 ? hom::prepare_kinetic<double>(p->nx, p->ny) : hom::prepare_kinetic<float>(p->nx, p->ny);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, HOM_ERR_CUDA, "kernel set-up failed: %s", cudaGetErrorString(e));
  }
  hom_status s = build_tensor_maps(c);
  if (s == HOM_OK) s = build_shared_tables(c);
  for (int b = 0; s == HOM_OK && b < p->batch; ++b) s = build_sim_tables(c, b);
  if (s != HOM_OK) {
    g_create_error = c->err;
    delete c;
    return s;
  }
  *out = c;
  return HOM_OK;
}

hom_status hom_set_sim_params(hom_ctx* c, int32_t b, double qpc_h, double qpc_w, double coul_lambda) {
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  if (b < 0 || b >= c->p.batch) return fail(c, HOM_ERR_ARG, "simulation index %d out of range", b);
  if (!std::isfinite(qpc_h) || !(qpc_w > 0) || !std::isfinite(qpc_w) || !std::isfinite(coul_lambda))
    return fail(c, HOM_ERR_ARG, "qpc_h, coul_lambda finite and qpc_w > 0 required");
  c->sims[b] = SimParams{qpc_h, qpc_w, coul_lambda};
  return build_sim_tables(c, b);
}

hom_status hom_init_packets(hom_ctx* c, int32_t b, const hom_packet* alpha, const hom_packet* beta, int32_t exch) {
  NvtxRange range("hom_init_packets");
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  const hom_params& p = c->p;
  if (!alpha || !beta) return fail(c, HOM_ERR_ARG, "packets must be non-NULL");
  if (b < -1 || b >= p.batch) return fail(c, HOM_ERR_ARG, "simulation index %d out of range", b);
  if (exch < -1 || exch > 1) return fail(c, HOM_ERR_ARG, "exch must be -1, 0 or +1");
  std::vector<cd> a, be, dbe;
  if ((s = build_packet(c, *alpha, a, nullptr)) != HOM_OK) return s;
  if ((s = build_packet(c, *beta, be, &dbe)) != HOM_OK) return s;
  const size_t n = (size_t)p.nx * p.ny;
  // sum over r1, r2 of |a(r1) b(r2) + s b(r1) a(r2)|^2 = 2 |a|^2 |b|^2 + 2 s |<a|b>|^2  (s = +-1)
  double na = 0, nb = 0;
  cd ab(0, 0);
  for (size_t i = 0; i < n; ++i) {
    na += std::norm(a[i]);
    nb += std::norm(be[i]);
    ab += std::conj(a[i]) * be[i];
  }
  const double sum = exch == 0 ? na * nb : 2.0 * na * nb + 2.0 * exch * std::norm(ab);
  const double dV = p.dx * p.dx * p.dy * p.dy;
  if (!(sum > 1e-12 * na * nb) || !(sum * dV > 1e-300))
    return fail(c, HOM_ERR_ARG, "the combined state vanishes (identical packets?)");
  const double coef = 1.0 / std::sqrt(sum * dV);
  // d(sum)/d(beta centre) for d psi0 / d delay:
  // 2 Re[ na <b|db> (1 + s^2) + 2 s <b|a> <a|db> ]
  cd bdb(0, 0), adb(0, 0);
  for (size_t i = 0; i < n; ++i) {
    bdb += std::conj(be[i]) * dbe[i];
    adb += std::conj(a[i]) * dbe[i];
  }
  const double sx = (double)exch;
  const double dsum = 2.0 * (na * bdb * (1.0 + sx * sx) + 2.0 * sx * std::conj(ab) * adb).real();
  const double cdc[2] = {coef, -0.5 * coef * dsum / sum};
  const int b0 = b < 0 ? 0 : b, b1 = b < 0 ? p.batch : b + 1;
  std::vector<double2> host(2 * n), dhost(n);
  for (size_t i = 0; i < n; ++i) {
    host[i] = double2{a[i].real(), a[i].imag()};
    host[n + i] = double2{be[i].real(), be[i].imag()};
    dhost[i] = double2{dbe[i].real(), dbe[i].imag()};
  }
  for (int bb = b0; bb < b1; ++bb) {
    if ((s = upload(c, c->L.packets + (size_t)bb * 2 * n * 16, host.data(), 2 * n * 16)) != HOM_OK) return s;
    if ((s = upload(c, c->L.dbeta + (size_t)bb * n * 16, dhost.data(), n * 16)) != HOM_OK) return s;
    if ((s = upload(c, c->L.coef + (size_t)bb * 8, &coef, 8)) != HOM_OK) return s;
    if ((s = upload(c, c->L.exch + (size_t)bb * 4, &exch, 4)) != HOM_OK) return s;
    if ((s = upload(c, c->L.adj_cdc + (size_t)bb * 16, cdc, 16)) != HOM_OK) return s;
    c->have_packets[bb] = 1;
    c->exch[bb] = exch;
  }
  const double2* pk = reinterpret_cast<const double2*>(c->ws + c->L.packets);
  const double* cf = reinterpret_cast<const double*>(c->ws + c->L.coef);
  const int* ex = reinterpret_cast<const int*>(c->ws + c->L.exch);
  if (p.prec == HOM_C128)
    HOM_CUDA(c, hom::launch_slater<double>(c->state, pk, cf, ex, b0, b1 - b0, (int)n, c->stream));
  else
    HOM_CUDA(c, hom::launch_slater<float>(c->state, pk, cf, ex, b0, b1 - b0, (int)n, c->stream));
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

hom_status hom_step(hom_ctx* c, int32_t nsteps) {
  NvtxRange range("hom_step");
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  if (nsteps < 0) return fail(c, HOM_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return HOM_OK;
  if (!c->tuned && c->tune_enabled && nsteps >= kTuneMinSteps) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HOM_CUDA(c, cudaStreamIsCapturing(c->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      if ((s = autotune(c)) != HOM_OK) return s;
      nsteps -= 12;
      drop_graphs(c);                            // graphs hold the variants they were captured with
    }
  }
  // graphs need a stream that can be captured (not the legacy default stream)
  if (c->use_graphs && !c->prof && c->stream != nullptr && c->stream != cudaStreamLegacy) {
    // not while the caller is itself capturing the stream
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HOM_CUDA(c, cudaStreamIsCapturing(c->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone) return run_steps_graph(c, nsteps);
  }
  return run_steps(c, c->state, nsteps, 0);
}

hom_status hom_observables(hom_ctx* c, hom_obs* out) {
  NvtxRange range("hom_observables");
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  if (!out) return fail(c, HOM_ERR_ARG, "out is NULL");
  const hom_params& p = c->p;
  s = p.prec == HOM_C128 ? measure_launch<double>(c) : measure_launch<float>(c);
  if (s != HOM_OK) return s;
  std::vector<double> h(2 * (size_t)p.batch * hom::NPART);
  HOM_CUDA(c, cudaMemcpyAsync(h.data(), c->ws + c->L.obs, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  const double dV = p.dx * p.dx * p.dy * p.dy;
  for (int b = 0; b < p.batch; ++b) {
    const double* r = &h[(size_t)b * hom::NPART];
    const double* q = &h[((size_t)p.batch + b) * hom::NPART];
    hom_obs o;
    o.norm = r[0] * dV;
    o.e_pot = r[1] * dV;
    o.e_coul = r[2] * dV;
    o.p_bunch = r[3] * dV;
    o.e_kin = dV * ((r[4] + q[4]) / p.nx + (r[5] + q[5]) / ((double)p.nx * p.ny));
    o.energy = o.e_kin + o.e_pot + o.e_coul;
    out[b] = o;
    if (!std::isfinite(o.norm) || !std::isfinite(o.energy))
      return fail(c, HOM_ERR_NUMERIC, "non-finite observables in simulation %d", b);
  }
  return HOM_OK;
}

hom_status hom_backward(hom_ctx* c, int32_t nsteps, int32_t K, double* loss, double* grad) {
  NvtxRange range("hom_backward");
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  const hom_params& p = c->p;
  if (!loss || !grad) return fail(c, HOM_ERR_ARG, "loss and grad must be non-NULL");
  if (nsteps < 1 || K < 1) return fail(c, HOM_ERR_ARG, "nsteps and K must be >= 1");
  if (p.split != HOM_STRANG)
    return fail(c, HOM_ERR_ARG, "the adjoint needs the Strang split (S(dt)^dagger = S(-dt))");
  const int S = (nsteps + K - 1) / K;
  if (S > p.ckpt_slots)
    return fail(c, HOM_ERR_ARG, "%d checkpoints needed (nsteps=%d, K=%d) but ckpt_slots=%d", S, nsteps, K,
                p.ckpt_slots);
  for (int b = 0; b < p.batch; ++b)
    if (!c->have_packets[b])
      return fail(c, HOM_ERR_STATE, "simulation %d was not set by hom_init_packets (needed for d/d delay)", b);
  const bool dbl = p.prec == HOM_C128;
  const int nx = p.nx, ny = p.ny, n = nx * ny;
  const size_t total = (size_t)p.batch * n * n * elem_bytes(p);
  // dV1/dh and dV1/dw along x for every simulation
  std::vector<double> dv((size_t)p.batch * 2 * nx);
  for (int b = 0; b < p.batch; ++b) {
    const SimParams& sp = c->sims[b];
    for (int ix = 0; ix < nx; ++ix) {
      const double x = coord(nx, p.dx, ix) - p.qpc_x0;
      const double g = std::exp(-x * x / (2.0 * sp.w * sp.w));
      dv[(size_t)b * 2 * nx + ix] = g;
      dv[(size_t)b * 2 * nx + nx + ix] = sp.h * g * x * x / (sp.w * sp.w * sp.w);
    }
  }
  if ((s = upload(c, c->L.adj_dv, dv.data(), dv.size() * 8)) != HOM_OK) return s;
  char* ckpt = c->ws + c->L.ckpt;
  char* lam = c->ws + c->L.lam;
  double* slot1 = reinterpret_cast<double*>(c->ws + c->L.adj_slot1);
  double* slot2 = reinterpret_cast<double*>(c->ws + c->L.adj_slot2);
  double* out = reinterpret_cast<double*>(c->ws + c->L.adj_out);
  const double* dvd = reinterpret_cast<const double*>(c->ws + c->L.adj_dv);
  // forward, keeping psi_{jK}
  for (int j = 0; j < S; ++j) {
    HOM_CUDA(c, cudaMemcpyAsync(ckpt + (size_t)j * total, c->state, total, cudaMemcpyDeviceToDevice, c->stream));
    const int m = std::min(K, nsteps - j * K);
    if ((s = run_steps(c, c->state, m, 0)) != HOM_OK) return s;
  }
  // loss and lambda_N = M psi_N
  if (dbl) HOM_CUDA(c, hom::launch_adj_mask<double>(c->state, lam, slot1, nx, ny, p.batch, c->stream));
  else HOM_CUDA(c, hom::launch_adj_mask<float>(c->state, lam, slot1, nx, ny, p.batch, c->stream));
  HOM_CUDA(c, hom::launch_adj_reduce(slot1, 1, p.batch, out, 4, c->stream));
  HOM_CUDA(c, cudaMemsetAsync(slot2, 0, (size_t)p.batch * hom::kAdjBlocks * 2 * 8, c->stream));
  auto accum = [&](double w) -> hom_status {
    if (dbl) HOM_CUDA(c, hom::launch_adj_accum<double>(c->state, lam, dvd, slot2, w, nx, ny, p.batch, c->stream));
    else HOM_CUDA(c, hom::launch_adj_accum<float>(c->state, lam, dvd, slot2, w, nx, ny, p.batch, c->stream));
    return HOM_OK;
  };
  if ((s = accum(0.5)) != HOM_OK) return s;
  // backward: psi_n from the checkpoint or by S(-dt) psi_{n+1}; lambda_n = S(-dt) lambda_{n+1}
  for (int m = nsteps - 1; m >= 0; --m) {
    if (m % K == 0) {
      HOM_CUDA(c, cudaMemcpyAsync(c->state, ckpt + (size_t)(m / K) * total, total, cudaMemcpyDeviceToDevice,
                                  c->stream));
    } else if ((s = run_steps(c, c->state, 1, 1)) != HOM_OK) {
      return s;
    }
    if ((s = run_steps(c, lam, 1, 1)) != HOM_OK) return s;
    if ((s = accum(m == 0 ? 0.5 : 1.0)) != HOM_OK) return s;
  }
  HOM_CUDA(c, hom::launch_adj_reduce(slot2, 2, p.batch, out + 1, 4, c->stream));
  const double2* pk = reinterpret_cast<const double2*>(c->ws + c->L.packets);
  const double2* db = reinterpret_cast<const double2*>(c->ws + c->L.dbeta);
  const double* cdc = reinterpret_cast<const double*>(c->ws + c->L.adj_cdc);
  const int* ex = reinterpret_cast<const int*>(c->ws + c->L.exch);
  if (dbl) HOM_CUDA(c, hom::launch_adj_delay<double>(lam, pk, db, cdc, ex, slot1, n, p.batch, c->stream));
  else HOM_CUDA(c, hom::launch_adj_delay<float>(lam, pk, db, cdc, ex, slot1, n, p.batch, c->stream));
  HOM_CUDA(c, hom::launch_adj_reduce(slot1, 1, p.batch, out + 3, 4, c->stream));
  std::vector<double> h((size_t)p.batch * 4);
  HOM_CUDA(c, cudaMemcpyAsync(h.data(), out, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  const double dV = p.dx * p.dx * p.dy * p.dy;
  for (int b = 0; b < p.batch; ++b) {
    loss[b] = dV * h[(size_t)b * 4];
    grad[3 * b + 0] = 2.0 * p.dt * dV * h[(size_t)b * 4 + 1];
    grad[3 * b + 1] = 2.0 * p.dt * dV * h[(size_t)b * 4 + 2];
    grad[3 * b + 2] = 2.0 * dV * h[(size_t)b * 4 + 3];
    if (!std::isfinite(loss[b]) || !std::isfinite(grad[3 * b]) || !std::isfinite(grad[3 * b + 1]) ||
        !std::isfinite(grad[3 * b + 2]))
      return fail(c, HOM_ERR_NUMERIC, "non-finite gradient in simulation %d", b);
  }
  return HOM_OK;
}

hom_status hom_copy_state(hom_ctx* c, int32_t b, void* host, size_t bytes, int32_t to_device) {
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  const hom_params& p = c->p;
  if (b < 0 || b >= p.batch) return fail(c, HOM_ERR_ARG, "simulation index %d out of range", b);
  const size_t n = (size_t)p.nx * p.ny;
  const size_t per = n * n * elem_bytes(p);
  if (!host || bytes != per) return fail(c, HOM_ERR_ARG, "host buffer must hold exactly %zu bytes", per);
  char* dev = c->state + (size_t)b * per;
  if (to_device) {
    HOM_CUDA(c, cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, c->stream));
    c->have_packets[b] = 0;
  } else {
    HOM_CUDA(c, cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  }
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

hom_status hom_marginal(hom_ctx* c, double* out) {
  NvtxRange range("hom_marginal");
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  if (!out) return fail(c, HOM_ERR_ARG, "out is NULL");
  const hom_params& p = c->p;
  const int n = p.nx * p.ny;
  double* d = reinterpret_cast<double*>(c->ws + c->L.pong);
  HOM_CUDA(c, p.prec == HOM_C128 ? hom::launch_marginal<double>(c->state, n, p.batch, d, c->stream)
                                 : hom::launch_marginal<float>(c->state, n, p.batch, d, c->stream));
  const size_t cnt = (size_t)p.batch * n;
  HOM_CUDA(c, cudaMemcpyAsync(out, d, cnt * 8, cudaMemcpyDeviceToHost, c->stream));
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  const double a = p.dx * p.dy;
  for (size_t k = 0; k < cnt; ++k) out[k] *= a;
  return HOM_OK;
}

hom_status hom_conditional(hom_ctx* c, int32_t b, int32_t ix2, int32_t iy2, double* out) {
  NvtxRange range("hom_conditional");
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  const hom_params& p = c->p;
  if (!out) return fail(c, HOM_ERR_ARG, "out is NULL");
  if (b < 0 || b >= p.batch) return fail(c, HOM_ERR_ARG, "simulation index %d out of range", b);
  if (ix2 < 0 || ix2 >= p.nx || iy2 < 0 || iy2 >= p.ny)
    return fail(c, HOM_ERR_ARG, "grid point (%d, %d) outside %d x %d", ix2, iy2, p.nx, p.ny);
  const int n = p.nx * p.ny;
  const char* st = c->state + (size_t)b * n * n * elem_bytes(p);
  double* d = reinterpret_cast<double*>(c->ws + c->L.pong);
  const int col = ix2 * p.ny + iy2;
  HOM_CUDA(c, p.prec == HOM_C128 ? hom::launch_gather<double>(st, n, 0, 1, n, col, 0, 1, nullptr, d, c->stream)
                                 : hom::launch_gather<float>(st, n, 0, 1, n, col, 0, 1, nullptr, d, c->stream));
  HOM_CUDA(c, cudaMemcpyAsync(out, d, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

hom_status hom_entanglement(hom_ctx* c, int32_t b, int32_t iy1, int32_t iy2, int32_t x1_lo, int32_t x1_hi,
                            int32_t x2_lo, int32_t x2_hi, double* entropy, double* weight) {
  NvtxRange range("hom_entanglement");
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  const hom_params& p = c->p;
  if (!entropy) return fail(c, HOM_ERR_ARG, "entropy is NULL");
  if (b < 0 || b >= p.batch) return fail(c, HOM_ERR_ARG, "simulation index %d out of range", b);
  if (iy1 < 0 || iy1 >= p.ny || iy2 < 0 || iy2 >= p.ny) return fail(c, HOM_ERR_ARG, "y index out of range");
  if (x1_lo < 0 || x1_hi > p.nx || x1_lo >= x1_hi || x2_lo < 0 || x2_hi > p.nx || x2_lo >= x2_hi)
    return fail(c, HOM_ERR_ARG, "x ranges must satisfy 0 <= lo < hi <= nx");
  const int n = p.nx * p.ny, m1 = x1_hi - x1_lo, m2 = x2_hi - x2_lo;
  const char* st = c->state + (size_t)b * n * n * elem_bytes(p);
  double2* d = reinterpret_cast<double2*>(c->ws + c->L.pong);
  const int r0 = x1_lo * p.ny + iy1, c0 = x2_lo * p.ny + iy2;
  HOM_CUDA(c, p.prec == HOM_C128
                  ? hom::launch_gather<double>(st, n, r0, p.ny, m1, c0, p.ny, m2, d, nullptr, c->stream)
                  : hom::launch_gather<float>(st, n, r0, p.ny, m1, c0, p.ny, m2, d, nullptr, c->stream));
  std::vector<cd> phi((size_t)m1 * m2);
  HOM_CUDA(c, cudaMemcpyAsync(phi.data(), d, phi.size() * 16, cudaMemcpyDeviceToHost, c->stream));
  HOM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (!slice_entropy(phi.data(), m1, m2, entropy, weight))
    return fail(c, HOM_ERR_NUMERIC, "the slice is zero or not finite");
  return HOM_OK;
}

hom_status hom_vn_entropy(const double* phi, int32_t m1, int32_t m2, double* entropy, double* weight) {
  if (!phi || !entropy || m1 < 1 || m2 < 1) return HOM_ERR_ARG;
  std::vector<cd> a((size_t)m1 * m2);
  for (size_t k = 0; k < a.size(); ++k) a[k] = cd(phi[2 * k], phi[2 * k + 1]);
  return slice_entropy(a.data(), m1, m2, entropy, weight) ? HOM_OK : HOM_ERR_NUMERIC;
}

const char* hom_last_error(const hom_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

hom_status hom_autotune_set(hom_ctx* c, const int32_t* choice) {
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  if (!choice) return fail(c, HOM_ERR_ARG, "choice is NULL");
  for (int k = 0; k < 2; ++k)
    if (choice[k] != 0 && choice[k] != 1) return fail(c, HOM_ERR_ARG, "kernel variants must be 0 or 1");
  if (choice[2] < 0 || choice[2] >= kStrategies) return fail(c, HOM_ERR_ARG, "strategy must be 0, 1 or 2");
  c->variant[0] = choice[0];
  c->variant[1] = choice[1];
  c->strategy = choice[2];
  c->tuned = true;
  drop_graphs(c);
  return HOM_OK;
}

hom_status hom_autotune_info(hom_ctx* c, int32_t* choice, double* ms) {
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  if (choice) {
    choice[0] = c->tuned ? c->variant[0] : -1;
    choice[1] = c->tuned ? c->variant[1] : -1;
    choice[2] = c->tuned ? c->strategy : -1;
  }
  if (ms) {
    for (int k = 0; k < 2; ++k)
      for (int v = 0; v < 2; ++v) ms[2 * k + v] = c->tune_ms[k][v];
    for (int k = 0; k < kStrategies; ++k) ms[4 + k] = c->tune_step_ms[k];
  }
  return HOM_OK;
}

hom_status hom_profile(hom_ctx* c, int32_t enable) {
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  if (enable && c->ev.empty()) {
    c->ev.resize(kEventPool, nullptr);
    for (auto& e : c->ev) HOM_CUDA(c, cudaEventCreate(&e));
  }
  if (enable) {
    HOM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->ev_used = 0;
    c->ev_kind.clear();
    for (int k = 0; k < kKinds; ++k) {
      c->prof_ms[k] = 0.0;
      c->prof_n[k] = 0;
    }
  }
  c->prof = enable != 0;
  return HOM_OK;
}

hom_status hom_profile_read(hom_ctx* c, double* ms, int64_t* counts) {
  hom_status s = enter(c);
  if (s != HOM_OK) return s;
  if ((s = harvest_events(c)) != HOM_OK) return s;
  for (int k = 0; k < kKinds; ++k) {
    if (ms) ms[k] = c->prof_ms[k];
    if (counts) counts[k] = c->prof_n[k];
  }
  return HOM_OK;
}

void hom_destroy(hom_ctx* c) {
  if (!c) return;
  drop_graphs(c);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"

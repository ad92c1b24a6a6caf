/*
 * hom.h -- C ABI of libhom: Strang split-step Fourier propagation of the
 * two-electron wavefunction psi(x1,y1,x2,y2) of a Hong-Ou-Mandel
 * interferometer built from quantum-Hall edge states, on one GPU.
 *
 * The operation follows Bellentani, Bordone, Oriols, Bertoni,
 * arXiv:1903.02581: Sec. II.C (two-particle Hamiltonian in the Landau gauge,
 * Eq. evoloperat, parallel 2D Fourier transforms), Appendix A (regrouping of
 * the magnetic kinetic term, Eq. 2PTB), Eq. coulomb (softened interaction),
 * Eq. twopstate (Slater determinant), Eq. singlepwp and Eq. H_effective
 * (edge-state packets), Eqs. pot_x / pot_xy (barriers), Eq. screenedCoulomb,
 * Eq. p_bunching (bunching probability), the probability maps of Figs. 2 and
 * 3(b) and the spatial entanglement of Sec. V.
 *
 * Conventions (units hbar = m* = |e| = 1).  Axes are relabelled with respect
 * to the paper: propagation runs along x, the edge confinement along y.
 *   H_i  = 1/2 (p_x - B y_i)^2 + 1/2 p_y^2 + V1(x_i, y_i)
 *   V1   = 1/2 omega_y^2 y^2 + qpc_h exp(-(x - qpc_x0)^2 / (2 qpc_w^2))
 *          [+ the Fermi-function blocks of hom_params.fermi_*]
 *   V12  = coul_lambda / sqrt((x1-x2)^2 + (y1-y2)^2 + coul_soft^2)
 *          [* exp(-|r1 - r2| / coul_screen) when coul_screen > 0]
 *   grid x_j = (j - (nx-1)/2) dx (cell-centred, same for y), k_m = 2 pi m /
 *   (n d) with m in [-n/2, n/2); periodic box; plain coordinate differences.
 *   One step S(dt) = e^{-iV dt/2} F_x^-1 e^{-iT_x dt/2} F_y^-1 e^{-iT_y dt}
 *   F_y e^{-iT_x dt/2} F_x e^{-iV dt/2}, with T_x diagonal in (k_x, y) and
 *   T_y in k_y (Eq. evoloperat in symmetric order).
 *
 * State layout (device, owned by the caller): psi[b][x1][y1][x2][y2],
 * y2 fastest, interleaved complex (re, im) of float (HOM_C64) or double
 * (HOM_C128); batch b indexes independent simulations.  The state is
 * normalised so that sum |psi|^2 dx^2 dy^2 = 1.
 *
 * Errors: every call returns a hom_status; nothing aborts.  hom_last_error()
 * gives a message for the last failure on a context.  After HOM_ERR_CUDA or
 * HOM_ERR_TIMEOUT the context is poisoned: further calls return
 * HOM_ERR_STATE until hom_destroy.  A context is not thread-safe.
 */
#ifndef HOM_H
#define HOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HOM_OK = 0,
  HOM_ERR_ARG = 1,      /* invalid argument (size, value, pointer)          */
  HOM_ERR_STATE = 2,    /* poisoned context or call out of order            */
  HOM_ERR_CUDA = 3,     /* a CUDA call failed (message in hom_last_error)   */
  HOM_ERR_NOMEM = 4,    /* workspace smaller than hom_workspace_bytes()     */
  HOM_ERR_TIMEOUT = 5,  /* a bounded device wait gave up                    */
  HOM_ERR_NUMERIC = 6   /* non-finite value detected in a reduction         */
} hom_status;

typedef enum { HOM_C64 = 0, HOM_C128 = 1 } hom_prec;

/* Plain data, copied by hom_create.  nx in {16,32,64,128,256}, ny in
 * {16,32,64}; HOM_C128 needs nx*ny <= 8192.  dt may be negative (backward
 * propagation).  qpc_h, qpc_w and coul_lambda are defaults for every
 * simulation of the batch (see hom_set_sim_params).  ckpt_slots reserves
 * room in the workspace for that many state checkpoints of hom_backward plus
 * one adjoint state (0 if hom_backward is not used). */
typedef struct {
  int32_t nx, ny, batch, prec;
  double dx, dy, B, omega_y, dt;
  double qpc_h, qpc_w, qpc_x0;
  double coul_lambda, coul_soft;
  int32_t observe_every;   /* informational: caller's observation cadence */
  int32_t ckpt_slots;
  double coul_screen;      /* sigma_c of Eq. screenedCoulomb: V12 gains exp(-|r1-r2|/sigma_c); 0 = none */
  int32_t split;           /* HOM_STRANG (default) or HOM_LIE */
  int32_t reserved;        /* must be 0 */
  /* Barrier blocks of Eq. pot_xy (axes relabelled as above), added to V1:
   * fermi_vb [F(x - fermi_xa) F(y - fermi_ya) + F(fermi_xb - x) F(fermi_yb - y)]
   * with F(u) = 1 / (exp(u / fermi_tau) + 1) (Eq. pot_x; tau a length), so
   * block A fills x < xa, y < ya and block B x > xb, y > yb.  fermi_vb = 0:
   * no blocks.  fermi_vb and fermi_tau also set the wall of numerical edge
   * states (hom_packet.numeric). */
  double fermi_vb, fermi_tau, fermi_xa, fermi_ya, fermi_xb, fermi_yb;
} hom_params;

/* Splitting of one time step.  HOM_STRANG: V/2 . Fx^-1 Tx/2 Fy^-1 Ty Fy Tx/2
 * Fx . V/2 (second order; the path the tolerances are stated for).  HOM_LIE:
 * the first-order product printed in Eq. evoloperat, applied right to left as
 * the x kinetic phase (full step), the y kinetic phase, then the potential
 * (full step).  hom_backward needs HOM_STRANG. */
enum { HOM_STRANG = 0, HOM_LIE = 1 };

/* One edge packet (Eq. singlepwp): centre x0, width sigma (standard
 * deviation of |psi|^2 along x), and either the energy of the central
 * wavevector on the lowest hybrid level (by_k0 == 0; needs omega_y > 0 and
 * energy >= sqrt(B^2+omega_y^2)/2; dir = +1 moves towards +x, -1 towards -x)
 * or the central wavevector k0 itself (by_k0 != 0, dir ignored).
 * numeric == 0: the edge states are the closed-form lowest hybrid level of
 * the parabolic edge.  numeric != 0 (needs by_k0): each edge state is the
 * lowest eigenvector of Eq. H_effective on the y grid,
 *   -1/2 d^2/dy^2 + 1/2 (k - B y)^2 + 1/2 omega_y^2 y^2 + V_wall(y),
 * with the spectral second derivative of the grid and the one-sided wall of
 * Eq. pot_x, V_wall(y) = fermi_vb F(wall_side (y - wall_y)) (wall_side +1:
 * barrier below wall_y, -1: above), computed on the host in FP64 (Jacobi). */
typedef struct {
  double x0, sigma, energy, k0;
  int32_t dir, by_k0;
  int32_t numeric, wall_side;
  double wall_y;
} hom_packet;

/* Observables of one simulation (host, FP64): norm = sum |psi|^2 dV;
 * e_kin = <T_x + T_y> (both particles); e_pot = <V1(r1) + V1(r2)>;
 * e_coul = <V12>; energy = e_kin + e_pot + e_coul; p_bunch = probability
 * that x1 and x2 have the same sign (Eq. p_bunching with the two regions
 * x < 0 and x > 0).  Expectations are not divided by the norm. */
typedef struct {
  double norm, energy, e_kin, e_pot, e_coul, p_bunch;
} hom_obs;

typedef struct hom_ctx hom_ctx;

/* Bytes of one batch of states: batch * (nx*ny)^2 * sizeof(complex).  Returns
 * 0 for invalid parameters. */
size_t hom_state_bytes(const hom_params* p);

/* Bytes of device workspace hom_create needs: one state-sized buffer (the
 * state alternates between it, as psi[b][r2][r1], and the caller's buffer, so
 * that each particle's kinetic pass reads contiguous planes), the phase tables,
 * reduction partials, packet buffers and ckpt_slots checkpoints (plus one
 * adjoint state when ckpt_slots > 0).  Returns 0 for invalid parameters. */
size_t hom_workspace_bytes(const hom_params* p);

/* Create a context.  d_state (hom_state_bytes) and d_workspace
 * (workspace_bytes >= hom_workspace_bytes) are device pointers owned by the
 * caller, 256-byte aligned, and must outlive the context; the context
 * allocates no device memory.  cuda_stream is a cudaStream_t (NULL = legacy
 * default stream) on which every launch and copy of the context is ordered.
 * Builds the FP64 phase tables (arguments reduced mod 2 pi) and uploads them;
 * synchronises the stream before returning.  The state is not touched. */
hom_status hom_create(const hom_params* p, void* d_state, void* d_workspace,
                      size_t workspace_bytes, void* cuda_stream, hom_ctx** out);

/* Override the QPC height/width and Coulomb strength of simulation b and
 * rebuild its tables (synchronises the stream). */
hom_status hom_set_sim_params(hom_ctx* ctx, int32_t b, double qpc_h, double qpc_w,
                              double coul_lambda);

/* Set simulation b (b = -1: every simulation) to
 *   psi = c [alpha(r1) beta(r2) + exch * beta(r1) alpha(r2)]
 * with exch = -1 (Slater determinant, Eq. twopstate), +1 (symmetric) or 0
 * (product), c fixing sum |psi|^2 dV = 1.  The packets are built on the host
 * in FP64 and combined on the device.  Synchronises the stream. */
hom_status hom_init_packets(hom_ctx* ctx, int32_t b, const hom_packet* alpha,
                            const hom_packet* beta, int32_t exch);

/* Advance every simulation by nsteps Strang steps (nsteps >= 0), state in
 * real space and in the layout above before and after.  Each step applies
 * one kinetic sandwich per particle (see hom_autotune_info for the three ways
 * of sequencing them); the launches of a call are
 * captured into a CUDA graph per step count and replayed (not on the legacy
 * default stream, not while profiling, not while the caller captures the
 * stream).  Asynchronous on the context's stream. */
hom_status hom_step(hom_ctx* ctx, int32_t nsteps);

/* Compute the observables of every simulation; out has batch entries (host).
 * FP64 reductions; synchronises the stream.  HOM_ERR_NUMERIC if the norm is
 * not finite. */
hom_status hom_observables(hom_ctx* ctx, hom_obs* out);

/* Adjoint gradient of L_b = p_bunch of simulation b after nsteps steps
 * (Eq. p_bunching).  Starts from the current state, which must have been set
 * by hom_init_packets (the packets define d psi0 / d delay, delay being the
 * centre of beta).  Runs forward keeping a checkpoint every K steps in the
 * workspace (ceil(nsteps/K) <= ckpt_slots), then backward: the adjoint state
 * lambda_N = M psi_N is stepped with S(dt)^dagger = S(-dt) (the Strang
 * product is palindromic and unitary), psi_n is restored from a checkpoint
 * or by S(-dt) psi_{n+1}, and dL/dtheta = 2 dt dV Im sum'_n <lambda_n|
 * dV/dtheta |psi_n> (trapezoid weights), dL/ddelay = 2 dV Re <lambda_0|
 * d psi_0/d delay>.  loss[b] = L_b, grad[3*b + {0,1,2}] = dL_b /
 * d{qpc_h, qpc_w, delay} (host arrays).  Leaves the state at step 0 (the
 * initial state).  Synchronises the stream.  HOM_ERR_ARG if ckpt_slots is too
 * small, HOM_ERR_STATE if a simulation was not initialised from packets. */
hom_status hom_backward(hom_ctx* ctx, int32_t nsteps, int32_t K, double* loss,
                        double* grad);

/* Copy simulation b between the device state and host memory (to_device != 0:
 * host -> device).  bytes must equal (nx*ny)^2 * sizeof(complex).  Layout as
 * the device state.  Synchronises the stream. */
hom_status hom_copy_state(hom_ctx* ctx, int32_t b, void* host, size_t bytes,
                          int32_t to_device);

/* Instrumentation.  While enabled, hom_step records a pair of CUDA events on
 * the context's stream around every kernel launch of a step and launches
 * without a CUDA graph; hom_profile_read synchronises the stream and returns,
 * for each launch kind, the summed device milliseconds (ms[HOM_PROFILE_KINDS])
 * and launch counts (counts[HOM_PROFILE_KINDS]) since the last enable.  The
 * kinds are [0] transposing pass, [1] in-place pass, [2] transpose, [3]
 * double in-place pass.  Enabling resets the sums.  No effect on results.
 * Independently of this switch, every call that launches work is an NVTX
 * range named after the call (hom_step, hom_observables, ...), and every pass
 * of a step a nested range: hom.transposing_pass, hom.in_place_pass,
 * hom.transpose, hom.double_pass (for ncu --nvtx-include, for example). */
#define HOM_PROFILE_KINDS 4
hom_status hom_profile(hom_ctx* ctx, int32_t enable);
hom_status hom_profile_read(hom_ctx* ctx, double* ms, int64_t* counts);

/* Autotuner.  A step applies one kinetic sandwich per particle, and the
 * second particle's sandwich needs the state transposed.  Three strategies
 * sequence the passes:
 *   0: a transposing pass, then an in-place pass on the other layout;
 *   1: an in-place pass, a transpose, an in-place pass;
 *   2: a transpose and one double in-place pass per step, the double pass
 *      holding the end of one step, the potential phase between steps and
 *      the start of the next (same particle, same layout).
 * Each kinetic pass also has two kernel variants that differ only in thread
 * count or cluster width.  Every choice applies the same arithmetic to every
 * element in the same order, so results are bitwise identical.  The first
 * hom_step call with at least 24 steps times the candidates on its first 12
 * steps (CUDA events around every launch) and keeps the fastest for the
 * context (disabled, strategy 0 with variants 0, if the environment variable
 * HOM_TUNE is "0").  choice[3] receives (transposing-pass variant, in-place
 * variant, strategy), -1 before tuning; ms[7], if not NULL, the measured
 * device milliseconds per launch [pass kind * 2 + variant] of the
 * transposing (kind 0) and in-place (kind 1) passes, then the estimated
 * milliseconds per step of strategies 0, 1 and 2. */
hom_status hom_autotune_info(hom_ctx* ctx, int32_t* choice, double* ms);

/* Fix the choice instead of tuning: choice[3] = (transposing-pass variant,
 * in-place variant, strategy), variants 0 or 1, strategy 0, 1 or 2
 * (HOM_ERR_ARG otherwise).  Later
 * hom_step calls use it and never tune.  Results do not depend on it. */
hom_status hom_autotune_set(hom_ctx* ctx, const int32_t* choice);

/* Probability maps and slices of the state (host outputs, FP64; each call
 * synchronises the stream and uses the workspace's second state buffer as
 * scratch, so it must not overlap a hom_step on another stream).
 *
 * hom_marginal: unconditional probability density of particle 1 (caption of
 * Fig. 3(b)): out[b][x][y] = sum over (x2, y2) of |psi(x, y, x2, y2)|^2 dx dy
 * for every simulation (batch * nx * ny doubles; integrates to the norm).
 * For (anti)symmetric states it is particle 2's as well.
 *
 * hom_conditional: conditional probability of particle 1 for particle 2 at
 * the grid point (ix2, iy2) (caption of Fig. 2): out[x][y] =
 * |psi(x, y, x2*, y2*)|^2, unnormalised (nx * ny doubles).
 *
 * hom_entanglement: spatial entanglement of Sec. V.  The 1D slice
 * phi(x1, x2) = psi(x1, y1*, x2, y2*), with x1 in [x1_lo, x1_hi) (region T)
 * and x2 in [x2_lo, x2_hi) (region B) at the y grid indices iy1, iy2, is
 * renormalised; rho_T(x1, x1') = sum over x2 of phi(x1, x2) conj(phi(x1', x2))
 * (Eq. reduced_density, read with phi*(x1', x2)); *entropy = -Tr rho_T ln rho_T
 * (the von Neumann entropy; the printed formula drops the sign); *weight (if
 * not NULL) = sum of |phi|^2 over the slice before renormalising.  The slice
 * is gathered on the device; the eigenvalues come from a Jacobi
 * diagonalisation on the host in FP64.  HOM_ERR_NUMERIC if the slice is zero.
 *
 * hom_vn_entropy: the same entropy for a slice given on the host (m1 * m2
 * complex values as interleaved doubles, row-major); needs no GPU. */
hom_status hom_marginal(hom_ctx* ctx, double* out);
hom_status hom_conditional(hom_ctx* ctx, int32_t b, int32_t ix2, int32_t iy2, double* out);
hom_status hom_entanglement(hom_ctx* ctx, int32_t b, int32_t iy1, int32_t iy2, int32_t x1_lo, int32_t x1_hi,
                            int32_t x2_lo, int32_t x2_hi, double* entropy, double* weight);
hom_status hom_vn_entropy(const double* phi, int32_t m1, int32_t m2, double* entropy, double* weight);

/* Norm and bunching probability of a batch of states, for callers that
 * cannot allocate device memory: code that was handed the state in a buffer
 * it does not own (another framework's tensor, a slice of a pool) and runs
 * where cudaMalloc is forbidden or would fail or synchronise.  The paper has
 * no counterpart; it is the real-space part of hom_observables without a
 * context or workspace.
 *   d_state: device, batch states laid out as for hom_create (complex64 if
 *            prec == HOM_C64, complex128 if HOM_C128), not modified;
 *   d_out:   device, 2*batch doubles written: d_out[2b] = sum |psi|^2 dx^2 dy^2,
 *            d_out[2b+1] = probability that x1 and x2 have the same sign;
 *   nx in {16..256}, ny in {16, 32, 64} (powers of two), dx, dy > 0,
 *   1 <= batch <= 64 (HOM_ERR_ARG otherwise, nothing launched).
 * Its partial sums live in one fixed 256 KiB array in the library's device
 * memory (every GPU that loads the library holds it until the process exits);
 * nothing is allocated, by the library or by the caller.  The first call in a
 * CUDA context (normally the device's primary context) looks up that array's
 * device address (cudaGetSymbolAddress) with the device current and keeps it
 * for that context: make that first call before any stream capture.  The kept
 * address assumes the context stays alive: after cudaDeviceReset, or anything
 * else that destroys the device's primary context, do not call this entry
 * point again in the same process (the new context may reuse the handle, and
 * the kept address would then be stale).  Every
 * call writes every partial it later reads, so no clearing is needed, but all
 * calls share the array: calls whose kernels overlap on the GPU (different
 * streams, or several host threads) race and must be serialised by the
 * caller.  Asynchronous on cuda_stream (a cudaStream_t, NULL = legacy
 * default stream).  HOM_ERR_CUDA if a launch or the address lookup fails. */
hom_status hom_bunching_static(const void* d_state, int32_t prec, int32_t nx, int32_t ny, int32_t batch,
                               double dx, double dy, double* d_out, void* cuda_stream);

/* Measured arithmetic peak of the current device, for the roofline of the
 * kinetic passes (which are bound by FP32 arithmetic, not by HBM).  A
 * measurement utility, not a step of the paper's method.
 *   kind 0: FP32 fused multiply-adds, kind 1: FP64; *flops_per_s receives the
 *   best of three timed launches (after one warm-up) of a kernel in which
 *   every thread of 8 CTAs per SM runs 8 independent FMA chains (2 flops per
 *   FMA), each launch about 10 ms at the nominal rates;
 *   d_sink: device, >= 16 bytes, caller-owned; written only on a value the
 *   chains never reach, so in practice never;
 *   synchronous: waits for its launches on cuda_stream (NULL = legacy default).
 * HOM_ERR_ARG for a bad kind or NULL pointer, HOM_ERR_CUDA if a launch or an
 * event call fails.  Allocates no device memory. */
hom_status hom_alu_peak(int32_t kind, void* d_sink, void* cuda_stream, double* flops_per_s);

/* Tensor-core form of the y part of the kinetic sandwich (F_y^-1 e^{-i dt T_y}
 * F_y with the 1/64 of the inverse transform, Eq. evoloperat) for ny = 64: a
 * design trial that measures whether the short-axis DFT as a dense product
 * on the tensor cores (tcgen05.mma, bf16 operands split three ways, FP32
 * accumulation) beats the FFT form; hom_step does not use it.
 *   d_in, d_out: device, nlines lines of 64 complex64 values (interleaved,
 *                16-byte aligned), d_out = each line times the circulant;
 *   nlines: a positive multiple of 128;
 *   dt, dy: the time step and the y spacing of the T_y phase;
 *   d_work: device, >= hom_ysandwich_tc_work_bytes() bytes, 16-byte aligned,
 *           caller-owned (the split operator and an error flag);
 *   nrep: timed launches after one warm-up; *ms (may be NULL) receives
 *         their average device time (CUDA events on cuda_stream).
 * Synchronous.  HOM_ERR_ARG for bad sizes or pointers, HOM_ERR_CUDA for a
 * failed launch, HOM_ERR_TIMEOUT if a CTA's bounded wait for its products
 * gave up (it frees its tensor memory and returns). */
size_t hom_ysandwich_tc_work_bytes(void);
hom_status hom_ysandwich_tc(const float* d_in, float* d_out, int32_t nlines, double dt, double dy, void* d_work,
                            size_t work_bytes, int32_t nrep, float* ms, void* cuda_stream);

/* Message of the last failure on ctx (or of the last failed hom_create when
 * ctx is NULL); never NULL. */
const char* hom_last_error(const hom_ctx* ctx);

/* Destroy the context (does not free the caller's buffers).  NULL is a no-op. */
void hom_destroy(hom_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HOM_H */

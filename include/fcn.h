/*
 * fcn.h -- C-ABI of the GB300 (sm_103a) split-step Fourier / Crank-Nicolson
 * z-step library for the 2D+1 NLSE of ultra-short pulses in air
 * (Ma & Lin, arXiv:1507.05988).
 *
 * The library advances A(r, tau) along z by Strang steps (Sec. 3, Eq. (nlseq)):
 *     A^{n+1} = exp(N dz/2) exp(D dz) exp(N dz/2) A^n
 * with D (Eq. (linearpart)) solved per frequency by the Crank-Nicolson system
 * of Eq. (matrix) and N (Eq. (nonlinearpart)) applied pointwise in time, the
 * plasma density coming from Eq. (ionization) integrated along tau by RK4.
 *
 * Conventions shared by every entry point
 *   - Units are SI.  A is in sqrt(W/m^2), |A|^2 is intensity in W/m^2.
 *   - A field is Nr x Nt complex values, row-major A[m][p]: m = radial index
 *     (m = 0 on axis, dr = r_max/(Nr-1), A = 0 at m = Nr-1), p = time index
 *     (contiguous; dtau = t_window/Nt, tau_p = -t_window/2 + p dtau).
 *     Host buffers are interleaved (re, im) doubles: 2*Nr*Nt doubles.
 *     Device buffers are interleaved in the working precision: float
 *     (FCN_FP32_MIXED) or double (FCN_FP64).
 *   - Nt must be a power of two in [2, 8192]; Nr must be in [3, 2048].
 *   - Every function returns FCN_OK (0) or a negative FCN_ERR_* code; no C++
 *     exception crosses the ABI.  fcn_last_error() gives a message.
 *   - Streams: every launch goes to the stream given at creation (or the
 *     stream set by fcn_set_stream); NULL means the legacy default stream.
 *     Functions that return host data synchronise that stream.
 *   - Ownership: the caller owns every host buffer and every device buffer it
 *     passes; the library never frees them.  A context owns its own device
 *     buffers and frees them in fcn_destroy.
 */
#ifndef FCN_H
#define FCN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FCN_OK                   0
#define FCN_ERR_ARG             -1   /* invalid argument (size, pointer, dz ...)    */
#define FCN_ERR_CUDA            -2   /* a CUDA runtime call or launch failed          */
#define FCN_ERR_NONFINITE       -3   /* the field contains NaN or Inf                 */
#define FCN_ERR_STEP_UNDERFLOW  -4   /* adaptive dz fell below dz_min / too many rejections */
#define FCN_ERR_UNSUPPORTED     -5   /* valid request outside the supported sizes     */
#define FCN_ERR_NOMEM           -6   /* device or host allocation failed              */
#define FCN_ERR_STATE           -7   /* call out of order (e.g. no field set)         */

/* ---- physics switches (fcn_params.flags) ---- */
#define FCN_DIFFRACTION   1u   /* (i/2k0) Delta_perp of Eq. (linearpart)                */
#define FCN_DISPERSION    2u   /* -(i k''/2) d^2/dtau^2 of Eq. (linearpart)             */
#define FCN_KERR          4u   /* i (k0/n0) sum_j n_2j |A|^2j of Eq. (nonlinearpart)    */
#define FCN_PLASMA        8u   /* -i k0/(2 n0^2) rho/rho_c of Eq. (nonlinearpart)       */
#define FCN_MPI          16u   /* -(beta_K/2)|A|^(2K-2) of Eq. (nonlinearpart)          */
#define FCN_MPI_SAT      32u   /* optional extra factor (1 - rho/rho_nt) on the loss    */
#define FCN_ALL_PHYSICS  31u
/* Variant of the dispersion term (with FCN_DISPERSION): the Crank-Nicolson
 * system carries diffraction alone and every frequency column is multiplied
 * by the exact factor exp(i k'' omega_q^2 dz / 2) of the -(i k''/2) d^2/dt^2
 * term of Eq. (linearpart), instead of the term sitting on the CN diagonal
 * (the two operators act on r and on omega and commute). */
#define FCN_EXACT_DISPERSION 128u

/* ---- working precision ---- */
#define FCN_FP64        0      /* complex128 everywhere                                   */
#define FCN_FP32_MIXED  1      /* complex64 field and arithmetic; FP64 reductions and the
                                  cross-warp carry of the rho(tau) scan                   */

/* Grid (Sec. 3: lattice A(m dr, n dz, p dtau + tau_min)). */
typedef struct {
    int32_t nr;          /* radial points                                  */
    int32_t nt;          /* time points (power of two)                     */
    double  r_max;       /* R [m]: dr = R/(Nr-1), Dirichlet node at r = R  */
    double  t_window;    /* T [s]: dtau = T/Nt, tau_min = -T/2             */
} fcn_grid;

/* Physics (Sec. 2, Eqs. (nlse) and (ionization)).
 * The rate of Eq. (ionization) is taken as sigma_K I^K (rho_nt - rho), i.e.
 * beta_K = K hbar omega0 sigma_K rho_nt and rho_at = rho_nt. */
typedef struct {
    double   lambda0;    /* carrier wavelength [m]                             */
    double   n0;         /* linear refractive index                            */
    double   n2j[4];     /* n2 [m^2/W], n4 [m^4/W^2], n6 [m^6/W^3], n8 [m^8/W^4] */
    double   k2;         /* GVD k'' [s^2/m]                                    */
    double   sigma_k;    /* MPI cross section sigma_K [s^-1 m^(2K) W^-K]       */
    double   rho_nt;     /* neutral density [m^-3]                             */
    int32_t  K;          /* photon number (1..16)                              */
    uint32_t flags;      /* FCN_* physics switches                             */
} fcn_params;

/* Diagnostics, FP64 reductions over the current field (Fig. 4 quantities and
 * energy).  energy = 2 pi dr^2 dtau sum_m W_m sum_p |A|^2 with W_0 = 1/8,
 * W_m = m; spectral_rms is the rms width of omega weighted by
 * sum_m W_m |FFT_tau(A)|^2. */
typedef struct {
    double  z;               /* propagated distance [m]                     */
    double  energy;          /* [J]                                         */
    double  peak_intensity;  /* max |A|^2 [W/m^2]                           */
    double  peak_rho;        /* max rho of the last nonlinear half step [m^-3] */
    double  onaxis_peak;     /* max_p |A_{0,p}|^2 [W/m^2]                   */
    double  spectral_rms;    /* [rad/s]                                     */
    int64_t steps;           /* accepted z-steps so far                     */
    int64_t rejected;        /* rejected adaptive attempts so far           */
    int32_t nonfinite;       /* 1 if the field holds NaN/Inf                */
    int32_t pad_;
} fcn_diag;

/* Result of an adaptive propagation (step doubling; not in the paper, which
 * uses a fixed dz). */
typedef struct {
    double  z;               /* position reached                            */
    double  dz_next;         /* proposal for the next step                  */
    double  last_err;        /* last relative L2 step-doubling error        */
    int64_t accepted;
    int64_t rejected;
    int64_t substeps;        /* Strang steps run, including rejected attempts */
    int64_t mlp_proposals;   /* steps whose dz came from the MLP            */
} fcn_stats;

typedef struct fcn_ctx fcn_ctx;

/* ========================= context API ========================= */

/* Creates a context for one pulse on the current CUDA device.
 * grid/params: validated as stated above.  precision: FCN_FP64 or
 * FCN_FP32_MIXED.  stream: a cudaStream_t (may be NULL).  On success *out
 * receives the context; the field is zero until fcn_set_field.
 * Errors: FCN_ERR_ARG, FCN_ERR_UNSUPPORTED, FCN_ERR_NOMEM, FCN_ERR_CUDA. */
int fcn_create(const fcn_grid *grid, const fcn_params *params, int32_t precision,
               void *stream, fcn_ctx **out);

/* Creates a context for n independent pulses, each with its own grid and
 * params (arrays of n).  All pulses advance together in every call; row and
 * column stages of all pulses run in one launch each (uneven grids are
 * packed into one work list). */
int fcn_create_batch(int32_t n, const fcn_grid *grids, const fcn_params *params,
                     int32_t precision, void *stream, fcn_ctx **out);

/* Frees every device buffer and graph of the context.  NULL is ignored. */
void fcn_destroy(fcn_ctx *ctx);

/* Message of the last failed call on this context (or of the last failed
 * creation if ctx is NULL).  Never NULL. */
const char *fcn_last_error(const fcn_ctx *ctx);

/* Routes all later launches of ctx to stream (cudaStream_t, may be NULL). */
int fcn_set_stream(fcn_ctx *ctx, void *stream);

/* Copies pulse `pulse`'s field from host memory (2*Nr*Nt doubles, layout
 * above) to the device, converting to the working precision on the device.
 * Resets z, the step counters and the diagnostics of that pulse. */
int fcn_set_field(fcn_ctx *ctx, int32_t pulse, const double *host_field);

/* As fcn_set_field and fcn_get_field with host buffers of interleaved
 * complex64 (2*Nr*Nt floats, the same layout): half the bytes over the host
 * link, and for FCN_FP32_MIXED contexts a plain copy of the working state
 * (no conversion); FCN_FP64 contexts convert on the device (get rounds the
 * double field to float).  fcn_get_field_c64 synchronises. */
int fcn_set_field_c64(fcn_ctx *ctx, int32_t pulse, const float *host_field);
int fcn_get_field_c64(fcn_ctx *ctx, int32_t pulse, float *host_out);

/* As fcn_set_field but from a device buffer already in the working
 * precision (float or double interleaved, Nr*Nt complex).  Device-to-device
 * copy on the context stream. */
int fcn_set_field_device(fcn_ctx *ctx, int32_t pulse, const void *dev_field);

/* Copies pulse `pulse`'s field to a caller-owned host buffer of 2*Nr*Nt
 * doubles (widened on the device in FCN_FP32_MIXED).  Synchronises. */
int fcn_get_field(fcn_ctx *ctx, int32_t pulse, double *host_out);

/* Copies the field to a caller-owned device buffer in the working precision. */
int fcn_get_field_device(fcn_ctx *ctx, int32_t pulse, void *dev_out);

/* rho (Nr*Nt doubles, [m^-3]) of the last nonlinear half step of the last
 * fcn_step/fcn_propagate call (zeros before the first step).  Synchronises. */
int fcn_get_rho(fcn_ctx *ctx, int32_t pulse, double *host_out);

/* Runs n fixed Strang steps of length dz on every pulse (Sec. 3, the serial
 * driver's z-loop).  dz > 0 and finite; n >= 0.  Asynchronous: launches only
 * (a CUDA graph per (dz, n-block) is captured on first use and replayed). */
int fcn_step(fcn_ctx *ctx, double dz, int64_t n);

/* Same as fcn_step but launches every kernel directly, without CUDA graphs
 * (for profiling and for checking that graph replay is identical). */
int fcn_step_nograph(fcn_ctx *ctx, double dz, int64_t n);

/* Adaptive propagation to z_end by step doubling: one step of dz and two of
 * dz/2 from the same state; err = ||A2-A1||/||A2|| (FP64 reduction);
 * err <= rtol accepts A2; next dz = dz*clamp(0.9 (rtol/err)^(1/3), 0.2, 2);
 * the last step lands on z_end exactly.  controller 0: proposals from that
 * formula; controller 1: proposals from the learned MLP (fcn_mlp_set) with
 * the formula as fallback after a rejection (and for the next 16 accepted
 * steps after a rejected MLP proposal).  dz0 > 0 is the first
 * proposal.  Fails with FCN_ERR_STEP_UNDERFLOW if dz < dz_min or after
 * max_reject consecutive rejections.  out may be NULL.
 * Multi-pulse contexts (all pulses at the same z, batching 0) advance with
 * one common dz: every attempt runs on all pulses in the launches of
 * fcn_step (one launch per stage for pulses that share it) and is accepted
 * when every pulse's err is within rtol; the formula follows the largest
 * err, the MLP proposes per pulse from that pulse's features and the
 * smallest proposal is taken.  Counts in *out are per attempt of the batch
 * (one accepted attempt = one step of every pulse). */
int fcn_propagate(fcn_ctx *ctx, double z_end, double dz0, double rtol, double dz_min,
                  int32_t max_reject, int32_t controller, fcn_stats *out);

/* FP64 diagnostics of pulse `pulse` (reduction kernels; synchronises).
 * Returns FCN_ERR_NONFINITE (with *out filled) if the field holds NaN/Inf. */
int fcn_get_diag(fcn_ctx *ctx, int32_t pulse, fcn_diag *out);

/* On-axis-weighted power P(tau_p) = 2 pi dr^2 sum_m W_m |A_mp|^2 [W]
 * (Nt doubles) and fluence F(r_m) = dtau sum_p |A_mp|^2 [J/m^2] (Nr doubles)
 * of pulse `pulse`; either pointer may be NULL.  Synchronises. */
int fcn_get_profiles(fcn_ctx *ctx, int32_t pulse, double *power, double *fluence);

/* Checkpoint: z, accepted/rejected counters and the last dz proposal
 * (4 doubles: z, steps, rejected, dz_next).  The field itself is saved with
 * fcn_get_field and restored with fcn_set_field followed by fcn_set_state. */
int fcn_get_state(fcn_ctx *ctx, int32_t pulse, double state[4]);
int fcn_set_state(fcn_ctx *ctx, int32_t pulse, const double state[4]);

/* ======================= kernel variants (autotuner) ======================= */
/* The row stage has 6 variants (FP32, K = 8): 0-2 one CTA per row (group)
 * with the compiler's register allocation, or 3 or 4 CTAs per SM; 3 a
 * persistent kernel that prefetches each CTA's next rows into shared memory
 * by bulk copies (Nt >= 512); 4, 5 the occupancy of 1, 2 with the other FFT
 * decomposition: radix-8 passes before the final radix-16 one (Nt = 4096:
 * 4 8 8 16) instead of radix-16 passes after one radix 2/4/8 pass (16 16 16)
 * (Nt >= 256; smaller rows run variant 0).  The column stage has 9:
 *   0-3  chunked affine-map scans of the two Thomas sweeps, chunks in
 *        registers (chunk length x CTA size);
 *   4-7  the same with chunks staged in shared memory (cp.async) or fed to
 *        registers, row coefficients from a per-dz table;
 *   8    one sequential Thomas sweep per column, 32 columns per warp, rows
 *        streamed through a shared-memory ring by TMA (Nt a multiple of 64;
 *        other grids fall back to variant 7).
 * By default (-1) the first fcn_step of a grid times every variant on a
 * scratch copy of the field and keeps the fastest per (precision, Nr, Nt)
 * for the process; if the environment variable FCN_TUNE_CACHE names a file,
 * choices are read from and appended to it.  row_variant in -1..5 and
 * col_variant in -1..8 force a variant (-1: tune).  Every variant computes
 * the same step up to rounding.  Drops the context's captured graphs.
 * Synchronises. */
int fcn_set_variants(fcn_ctx *ctx, int32_t row_variant, int32_t col_variant);

/* Batched work lists for multi-pulse FP32 contexts (every pulse K = 8,
 * Nt >= 512): mode 1 runs each stage of all pulses as one persistent launch
 * over (pulse, rows) and (pulse, column group) items; 0 launches each pulse
 * separately (tuned per-Nt kernels, all inside one CUDA graph); -1 (the
 * default) uses the work lists when the grids differ and most points lie in
 * pulses too small to fill the GPU with a launch of their own.  Drops the
 * captured graphs.  FCN_ERR_UNSUPPORTED if mode 1 is not possible. */
int fcn_set_batching(fcn_ctx *ctx, int32_t mode);

/* Paired column launches for FP32 contexts whose pulses all share one grid
 * (and so, for one dz, one pivot table): the column stage of pulses 2i and
 * 2i+1 runs as one launch that reads each pivot, coefficient row and sweep
 * factor once for both (Eqs. (matrix), (matrix1) are the same for both).
 * mode 1 on, 0 off, -1 (default) decided on the first step by timing one
 * paired launch against two single ones.  Drops the captured graphs.
 * fcn_get_pairing returns the decision: 1, 0, or -1 before the first step. */
int fcn_set_pairing(fcn_ctx *ctx, int32_t mode);
int fcn_get_pairing(const fcn_ctx *ctx);

/* Sequential column kernel over all pulses at once, for contexts of 2..8
 * pulses that share one grid (Nt a multiple of 64) and, for one dz, one
 * pivot table: the Crank-Nicolson systems of Eq. (matrix) are solved by one
 * Thomas sweep per frequency column and pulse (the "chasing" method of
 * Sec. 3.1, forward elimination then back substitution), 32 columns per
 * warp and two pulses per thread, rows streamed through shared memory by
 * TMA, all pulses in one launch; the row stage then runs as one launch over
 * all pulses per z-step as in fcn_set_multi_launch mode 1.
 * mode 1 on, 0 off, -1 (default) decided on the first step by timing such
 * launches (each ring shape: rows per stage against warps per SM) against
 * the per-group launches of the tuned column variant (on scratch copies),
 * keeping the fastest; 2, 3, 4: on with ring shape 0, 1, 2 (1: shape 0).
 * Graph branches > 1 turn it off.  Drops the captured graphs.
 * fcn_get_sequential_columns returns the decision: 1, 0, or -1 before the
 * first step.  Other modes: FCN_ERR_ARG. */
int fcn_set_sequential_columns(fcn_ctx *ctx, int32_t mode);
int fcn_get_sequential_columns(const fcn_ctx *ctx);

/* Graph branches for multi-pulse contexts.  The pulses (or pulse pairs of a
 * paired column launch) are independent between the row and column stages
 * of the split step (Sec. 3: each pulse is its own problem), so with n > 1
 * the captured CUDA graphs hold one chain of launches per pulse group,
 * spread round-robin over n forked branches that the GPU may run
 * concurrently (filling the tail of one group's launch with another's).
 * Each pulse's launches and their order are unchanged, so results are
 * bit-identical for every n.  n in 1..8 (default 1; batched work lists
 * ignore it).  Drops the captured graphs.  Synchronises.
 * fcn_get_graph_branches returns the setting. */
int fcn_set_graph_branches(fcn_ctx *ctx, int32_t n);
int fcn_get_graph_branches(const fcn_ctx *ctx);

/* Multi-pulse row launches: the row stage of pulses whose launches differ
 * only in their field, rho and statistics buffers (same grid, physics
 * coefficients, dz and kernel variant) as one launch (blockIdx.y = pulse).
 *   mode 0: one row launch per pulse;
 *   mode 1: per z-step, the column stage of every pulse group, then the
 *           row stage of up to 8 consecutive pulses per launch;
 *   mode 2 (default): per pulse group (the two pulses of a paired column
 *           launch), its column launch and then one row launch for both,
 *           which keeps each group's chain of launches on data still in L2.
 * Each pulse's own sequence of operations is the same in every mode, so
 * results are bit-identical.  Graph branches > 1 use modes 0 and 2 only.
 * Drops the captured graphs.  Synchronises.  fcn_get_multi_launch returns
 * the mode. */
int fcn_set_multi_launch(fcn_ctx *ctx, int32_t mode);
int fcn_get_multi_launch(const fcn_ctx *ctx);

/* Variants in use for pulse `pulse` (out[0] row, out[1] column; -1 before
 * the first step). */
int fcn_get_variants(fcn_ctx *ctx, int32_t pulse, int32_t out[2]);

/* ========================= kernel timing ========================= */
/* Kernel kinds reported by fcn_profile_read. */
#define FCN_PROF_ROW_HEAD  0   /* nonlinear half step + forward FFT               */
#define FCN_PROF_ROW_MID   1   /* inverse FFT + two half steps + forward FFT      */
#define FCN_PROF_ROW_TAIL  2   /* inverse FFT + half step + rho + row statistics  */
#define FCN_PROF_COLUMN    3   /* Crank-Nicolson column solve                      */
#define FCN_PROF_KINDS     4

/* on = 1: later fcn_step calls launch kernels directly (no graphs) with a
 * CUDA event pair around each launch on the context stream.
 * on = 2: later fcn_step calls replay graphs captured with an event record
 * node before and after every kernel (separate from the untimed graphs), so
 * the kernels run in the launch structure of an unprofiled replay; each
 * replay is followed by a synchronisation that reads the events.
 * on = 0 stops.  FCN_ERR_ARG for other values. */
int fcn_profile_enable(fcn_ctx *ctx, int32_t on);

/* Total device milliseconds and launch counts per kind (FCN_PROF_KINDS
 * entries each) since the last reset; reset != 0 clears them.  Synchronises. */
int fcn_profile_read(fcn_ctx *ctx, double *ms, int64_t *count, int32_t reset);

/* ===================== learned dz (MLP) ===================== */
/* Network 6 -> 64 -> 64 -> 1, tanh hidden layers, linear output; BF16
 * weights in the forward pass, FP32 accumulation and FP32 master weights.
 * Flat parameter layout (floats): W1[64][6], b1[64], W2[64][64], b2[64],
 * W3[64], b3 -- 4673 values. */
#define FCN_MLP_NIN     6
#define FCN_MLP_NH      64
#define FCN_MLP_NPARAM  4673

/* Features of a field, computed on the device from the FP64 row statistics
 * that the closing row launch of every attempt writes anyway (no extra pass):
 *   f0 = log(peak I / I_ref)            f1 = log10(peak rho/rho_nt + 1e-30)/10
 *   f2 = log(on-axis peak I / peak I)   f3 = relative change of peak I over the last step
 *   f4 = log(dz_prev / L_ref)           f5 = log(err_prev / rtol)
 *   fE = relative change of the energy over the last step
 * with I_ref from the field at the start of fcn_propagate and
 * L_ref = k0 (r_max/5)^2 / 2.  With g = f4 - f5/3 (log of the step that
 * would have brought the last accepted attempt to err = rtol) and
 * s = exp(-f5/3), the network takes n = (f0, f1, f2, f3 s, g, fE s) (the
 * changes scaled to a step of exp(g) L_ref) and its output y corrects the
 * step-doubling law: the proposal is dz = L_ref exp(g + y) (a zero network
 * gives that law without its 0.9 safety factor), clamped to [0.2, 2] times
 * the last accepted step. */
#define FCN_MLP_LOG_FLOATS 9

/* Loads / reads FP32 master weights (host, FCN_MLP_NPARAM floats). */
int fcn_mlp_set(fcn_ctx *ctx, const float *host_params);
int fcn_mlp_get(fcn_ctx *ctx, float *host_params);

/* Makes fcn_propagate append one record per attempt to a caller-owned host
 * buffer of capacity records of FCN_MLP_LOG_FLOATS (9) floats: f0..f5 and fE
 * of the state the attempt started from, log(h / L_ref) of the attempted
 * step and log(err / rtol) of its step-doubling error.  log(dz_safe / L_ref)
 * of that state follows as rec[7] - rec[8]/3 (the Strang local error is
 * O(dz^3)), and the network's training label as that minus
 * g = rec[4] - rec[5]/3.  capacity 0 stops.  Single-pulse contexts only.
 * fcn_mlp_log_count returns the number of records written. */
int fcn_mlp_set_log(fcn_ctx *ctx, float *host_buf, int64_t capacity);
int64_t fcn_mlp_log_count(const fcn_ctx *ctx);

/* Trains the context's MLP on n samples (x: n x 6 features, y: n labels)
 * with Adam (beta 0.9/0.999) for `epochs` passes over a seeded permutation
 * in minibatches of `batch`; weights start from fcn_mlp_set's or, if none,
 * from a seeded uniform initialisation.  Forward and backward run in this
 * library's kernels (BF16 weights, FP32 accumulation).  final_loss (may be
 * NULL) receives the mean squared error over all samples. */
int fcn_mlp_train(fcn_ctx *ctx, const float *x, const float *y, int32_t n, int32_t epochs,
                  int32_t batch, float lr, uint64_t seed, float *final_loss);

/* Stateless: mean squared error and its gradient (FCN_MLP_NPARAM floats) of
 * the network with the given FP32 master weights over n samples, on the GPU. */
int fcn_mlp_loss_grad(const float *params, const float *x, const float *y, int32_t n,
                      float *loss, float *grad);

/* ====================== stateless device operations ======================
 * These run one stage on caller-owned device buffers (e.g. torch tensors)
 * and exist so each kernel can be checked on its own.  `field`, `rho`,
 * `table` are device pointers in the working precision; `stream` is a
 * cudaStream_t.  They allocate nothing. */

#define FCN_OP_IFFT    1   /* inverse FFT along tau (Eq. (antifourier)), 1/Nt applied */
#define FCN_OP_NL      2   /* one nonlinear half step of length dz_half (Eq. (Anhalf)) */
#define FCN_OP_NL2     4   /* a second nonlinear half step right after the first        */
#define FCN_OP_FFT     8   /* forward FFT along tau (Sec. 3.1, first loop)             */
#define FCN_OP_RHO    16   /* write rho (working precision, Nr*Nt) of the last half step */

/* Row stage: for every row, in order: [IFFT] [NL] [NL2] [FFT].  rho may be
 * NULL unless FCN_OP_RHO is set.  Errors: FCN_ERR_ARG, FCN_ERR_CUDA. */
int fcn_op_rows(const fcn_grid *grid, const fcn_params *params, int32_t precision,
                int32_t ops, double dz_half, void *field, void *rho, void *stream);

/* Number of complex entries of the Crank-Nicolson factorisation table:
 * Nr * (Nt/2 + 1). */
int64_t fcn_cn_table_entries(const fcn_grid *grid);

/* Fills `table` (fcn_cn_table_entries complex values, working precision)
 * with 1/pivot_j of the Thomas factorisation of M_abc^q (Eq. (matrix)) for
 * every radial index j and every |frequency| bin q = 0..Nt/2. */
int fcn_op_cn_table(const fcn_grid *grid, const fcn_params *params, int32_t precision,
                    double dz, void *table, void *stream);

/* Column stage on a frequency-domain field (Sec. 3.1, second loop): for
 * every q, A~_{.,q} <- (M_abc^q)^{-1} M_def^q A~_{.,q}, in place, using the
 * table from fcn_op_cn_table for the same dz. */
int fcn_op_cn(const fcn_grid *grid, const fcn_params *params, int32_t precision,
              double dz, const void *table, void *field, void *stream);

/* ============ column stage for callers that cannot allocate ============
 * There is no counterpart to this in the paper; it is a service of this
 * library.  fcn_op_cn_table + fcn_op_cn need a pivot table in a device buffer
 * that the caller allocates.  Some callers cannot do that: code that runs
 * inside a framework whose caching allocator already owns the device memory
 * (a raw cudaMalloc may then fail, and cudaFree synchronises the whole
 * device, stalling every other stream), or a latency-bound loop that must
 * never block on an allocation.  fcn_op_cn_noalloc does the same column
 * stage as fcn_op_cn_table followed by fcn_op_cn, in place on `field`, with
 * its scratch -- the pivot table for this dz and the radial ratio tables --
 * in one static device array of FCN_NOALLOC_SCRATCH_BYTES bytes built into
 * the library.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   - Size limit: Nr*(Nt/2+1) complex values (16 B in FCN_FP64, 8 B in
 *     FCN_FP32_MIXED) plus 4*Nr reals must fit in the array; larger grids
 *     return FCN_ERR_UNSUPPORTED before any GPU work.  Examples that fit:
 *     Nr=128, Nt=256 (either precision); Nr=1024, Nt=1024 in FP32 only.
 *   - Every GPU that loads the library holds the array until the process
 *     exits.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address; make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents (each
 *     call rewrites what it reads).  Calls whose kernels overlap on the GPU
 *     (different streams or host threads) race on it: serialise them.
 *   - field: device buffer in the working precision, frequency domain,
 *     Nr*Nt complex values, updated in place.  stream: cudaStream_t.
 *   - Arguments are checked as for fcn_op_cn (same codes: FCN_ERR_ARG for a
 *     bad grid, parameter, flag, dz or pointer; FCN_ERR_UNSUPPORTED for a
 *     grid beyond the library's range) before any GPU work.
 *   - Errors: those, FCN_ERR_UNSUPPORTED (grid too large for the array),
 *     FCN_ERR_CUDA. */
#define FCN_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
int fcn_op_cn_noalloc(const fcn_grid *grid, const fcn_params *params, int32_t precision,
                      double dz, void *field, void *stream);

/* ================= Cartesian transverse grid (3D+1) =================
 * Sec. 2 of the paper gives Delta_perp = d^2/dx^2 + d^2/dy^2 for beams
 * without cylindrical symmetry; Sec. 3 discretises only the radial operator.
 * This context advances A(x, y, tau) by the same Strang step (Eq. (nlseq)):
 * the nonlinear half steps and the rho(tau) integration act on every (x, y)
 * row exactly as on a radial row, and the linear step is, per frequency bin,
 * the Crank-Nicolson factor of the x part (Eqs. (diff1)-(diff2) on the x
 * axis) followed by that of the y part with the dispersion term on its
 * diagonal (the x and y factors commute; their product differs from the
 * unsplit two-dimensional Crank-Nicolson step by O(dz^3) per step).  The
 * walls carry A = 0 (Eq. (bound) at r = max, on all four sides).
 *   - A field is Nx x Ny x Nt complex values, row-major A[i][j][p]:
 *     x_i = -x_width/2 + i dx, dx = x_width/(Nx-1), likewise y_j; p as for
 *     the radial grid.  Host buffers: 2*Nx*Ny*Nt interleaved doubles (or
 *     floats for the _c64 calls).
 *   - Nx, Ny in [3, 2048]; Nt a power of two in [2, 8192].
 *   - Diagnostics (fcn_diag): energy = dx dy dtau sum |A|^2; onaxis_peak is
 *     the maximum over tau of the row nearest the centre, i = (Nx-1)/2,
 *     j = (Ny-1)/2; spectral_rms weighs every row equally; rejected = 0.
 *   - Errors, streams and ownership as for the radial context. */
typedef struct {
    int32_t nx;          /* x nodes (walls at i = 0 and Nx-1)              */
    int32_t ny;          /* y nodes (walls at j = 0 and Ny-1)              */
    int32_t nt;          /* time points (power of two)                     */
    int32_t pad_;
    double  x_width;     /* [m]: dx = x_width/(Nx-1)                       */
    double  y_width;     /* [m]: dy = y_width/(Ny-1)                       */
    double  t_window;    /* T [s]: dtau = T/Nt, tau_min = -T/2             */
} fcn_grid_xy;

typedef struct fcn_xy_ctx fcn_xy_ctx;

/* Creates a Cartesian-grid context (physics as in fcn_params, all flags
 * allowed).  The field is zero until fcn_xy_set_field.
 * Errors: FCN_ERR_ARG, FCN_ERR_UNSUPPORTED, FCN_ERR_NOMEM, FCN_ERR_CUDA. */
int  fcn_xy_create(const fcn_grid_xy *grid, const fcn_params *params, int32_t precision,
                   void *stream, fcn_xy_ctx **out);
void fcn_xy_destroy(fcn_xy_ctx *ctx);
/* Message of the context's last error (NULL: of the last failed create). */
const char *fcn_xy_last_error(const fcn_xy_ctx *ctx);
/* Host field in/out (complex128 / complex64 interleaved, layout above);
 * setting a field resets z, the step count and rho.  The get calls
 * synchronise the stream. */
int  fcn_xy_set_field(fcn_xy_ctx *ctx, const double *host);
int  fcn_xy_get_field(fcn_xy_ctx *ctx, double *host);
int  fcn_xy_set_field_c64(fcn_xy_ctx *ctx, const float *host);
int  fcn_xy_get_field_c64(fcn_xy_ctx *ctx, float *host);
/* The same from / into a caller-owned device buffer in the working
 * precision (complex128 in FCN_FP64, complex64 in FCN_FP32_MIXED; Nx*Ny*Nt
 * values): device-to-device copies on the context stream, no
 * synchronisation.  Setting resets z, the step count and rho. */
int  fcn_xy_set_field_device(fcn_xy_ctx *ctx, const void *dev_field);
int  fcn_xy_get_field_device(fcn_xy_ctx *ctx, void *dev_out);
/* rho [m^-3] of the last nonlinear half step, Nx*Ny*Nt doubles. */
int  fcn_xy_get_rho(fcn_xy_ctx *ctx, double *host);
/* n Strang steps of length dz (n >= 0, dz > 0 finite); blocks of eight
 * middle steps replay a CUDA graph (captured on first use per dz).  The
 * first step of a grid times the kernel variants once per process.
 * _nograph launches every kernel directly.  Asynchronous.
 * Errors: FCN_ERR_ARG, FCN_ERR_STATE (no field set), FCN_ERR_CUDA. */
int  fcn_xy_step(fcn_xy_ctx *ctx, double dz, int64_t n);
int  fcn_xy_step_nograph(fcn_xy_ctx *ctx, double dz, int64_t n);
/* FP64 diagnostics of the current field (synchronises the stream).
 * Returns FCN_ERR_NONFINITE if the field holds NaN or Inf. */
int  fcn_xy_get_diag(fcn_xy_ctx *ctx, fcn_diag *out);
/* Forces the row-stage variant (0..5, as fcn_set_variants; 3 runs as 0
 * here) and the line variant (0..7: the chunk
 * of nodes a thread owns, 16 or 8 in FP32 and 8 or 4 in FP64, one or two
 * lines per thread, CTAs of up to 512 or 256 threads); -1 returns to
 * timing.  Every variant computes the same step (up to rounding order). */
int  fcn_xy_set_variants(fcn_xy_ctx *ctx, int32_t row_variant, int32_t line_variant);
int  fcn_xy_get_variants(const fcn_xy_ctx *ctx, int32_t out[2]);
/* Per-launch CUDA-event timing (off by default; while on, steps launch
 * directly instead of replaying graphs).  ms and count receive
 * FCN_XY_PROF_KINDS totals; reset = 1 clears them. */
#define FCN_XY_PROF_ROW_HEAD  0   /* nonlinear half step + forward FFT          */
#define FCN_XY_PROF_ROW_MID   1   /* inverse FFT + two half steps + forward FFT */
#define FCN_XY_PROF_ROW_TAIL  2   /* inverse FFT + half step + rho + statistics */
#define FCN_XY_PROF_LINE_X    3   /* x Crank-Nicolson factor                    */
#define FCN_XY_PROF_LINE_Y    4   /* y Crank-Nicolson factor (with dispersion)  */
#define FCN_XY_PROF_KINDS     5
int  fcn_xy_profile_enable(fcn_xy_ctx *ctx, int32_t on);
int  fcn_xy_profile_read(fcn_xy_ctx *ctx, double *ms, int64_t *count, int32_t reset);

/* ===================== arithmetic peak (measurement) =====================
 * Not an operation of the method: the denominator of the ALU rooflines that
 * the FP64 path and the row stage are measured against.  Runs this
 * library's FMA microkernel (independent FMA chains in every thread, 8 CTAs
 * of 256 threads per SM, best of three CUDA-event-timed launches after a
 * warm-up) on the current device and stream and returns the rate in
 * FLOP/s (an FMA counts two) in *flop_per_s.  kind 0: FP64 fma; 1: FP32
 * fmaf; 2: FP32 packed fma.rn.f32x2 (two FMAs per instruction).  The clocks
 * are those the GPU runs at; nothing here changes them.  Synchronises.
 * Errors: FCN_ERR_ARG, FCN_ERR_NOMEM, FCN_ERR_CUDA. */
int fcn_alu_peak(int32_t kind, double *flop_per_s, void *stream);

/* Library version string. */
const char *fcn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FCN_H */

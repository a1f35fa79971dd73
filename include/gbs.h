/*
 * gbs.h -- C ABI of the GB300 (sm_103a) extrapolated-GBS time stepper.
 *
 * Method: Ellison & Fornberg, "A parallel-in-time approach for wave-type PDEs"
 * (arXiv 1907.11771).  An ODE y' = f(y) from a method-of-lines wave system is
 * advanced over sections of length H.  Each section is one extrapolated GBS
 * macro-step (Sec. 2.1 eq. "GBS", Sec. 3.2, Sec. 3.6):
 *
 *   for every sequence k with even step count N_k and h_k = H / N_k
 *     y_1 = y_0 + h_k f(y_0)                                  Forward Euler
 *     y_(n+1) = y_(n-1) + 2 h_k f(y_n),  n = 1..N_k            leap-frog
 *     y*_k = (y_(N_k-1) + 2 y_(N_k) + y_(N_k+1)) / 4          averaging
 *   y(t + H) = sum_k c_k y*_k                                 extrapolation
 *
 * f(y_0) is evaluated once and shared by all sequences (Sec. 3.6).  The
 * weights c satisfy the order constraints sum_k c_k h_k^(2j) = [j == 0],
 * j < p/2 (Sec. 3.2 eq. "vander"); with more sequences than constraints the
 * free weights are given and the dependent ones follow from
 * c_dep = V_dep^-1 (b - V_free c_free) (Sec. 3.7 eq. "cdep_computation").
 *
 * Conventions for every entry point
 *  - All functions return a gbs_status; none aborts, throws or prints.  The
 *    text of the last failure of a handle is returned by gbs_last_error().
 *  - Device pointers are CUDA device (or managed) addresses on the current
 *    device; the caller owns them and keeps them alive while work that uses
 *    them is in flight.  The library owns only its workspace.
 *  - State layout ("SoA"): for each problem of the batch, in batch order,
 *    fields [F][nz][ny][nx] contiguous with x fastest; the batch is the
 *    concatenation of the problems.  F = 2 (u, v) for the 1D wave system and
 *    F = 1 + ndim (p, u_x, u_y[, u_z]) for acoustics.  Media arrays (kappa,
 *    rho) and gradients use [nz][ny][nx] per problem, concatenated likewise.
 *  - Element type of states and media: float for GBS_F32_STATE_F64_COMBINE,
 *    double for GBS_F64 and GBS_F32X2.  Gradients are always double.
 *  - Precisions.  GBS_F32_STATE_F64_COMBINE keeps the leap-frog levels in FP32
 *    and sums the combine in FP64-class arithmetic (the throughput path).
 *    GBS_F64 computes everything in FP64.  GBS_F32X2 takes FP64 states and
 *    media, holds the levels as pairs of floats (hi + lo, about 48 significant
 *    bits) and evaluates the right-hand sides and leap-frog updates with
 *    error-free FP32 transformations on the FP32 units, then combines in FP64;
 *    it reaches FP64-class accuracy (a few 1e-15 per operation) at FP32-unit
 *    speed.  The paper fixes no arithmetic precision; the three are
 *    implementation choices.  The adjoint of a GBS_F32X2 handle runs in FP64.
 *  - Work is enqueued asynchronously on the stream given to gbs_create.
 *    Device-side failures are latched and reported by gbs_sync().
 */
#ifndef GBS_H
#define GBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBS_ABI_VERSION 1
#define GBS_MAX_SLOTS 8    /* weight slots per handle                       */
#define GBS_MAX_SEQ 16     /* sequences per scheme (m)                       */
#define GBS_MAX_STEPS 64   /* largest step count N_k                         */

typedef struct gbs_ctx* gbs_handle; /* opaque; created by gbs_create, freed by gbs_destroy */

typedef enum {
  GBS_OK = 0,
  GBS_ERR_INVALID = 1,   /* bad argument: null pointer, size, enum, step counts */
  GBS_ERR_ORDER = 2,     /* weights violate the order constraints               */
  GBS_ERR_UNSTABLE = 3,  /* H beyond the scheme's stability limit (checked only
                            when requested)                                     */
  GBS_ERR_CUDA = 4,      /* a CUDA runtime call failed                          */
  GBS_ERR_NOMEM = 5,     /* workspace allocation failed                         */
  GBS_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up                  */
  GBS_ERR_NONFINITE = 7, /* a NaN/Inf was found where finite values are needed  */
  GBS_ERR_STATE = 8      /* call out of order (e.g. stepping before weights set) */
} gbs_status;

/* gbs_problem.system.  GBS_ONEWAY_SPECTRAL is the test problem of Sec. 4: u_t + u_x = 0 on a
 * periodic 1D grid with the derivative taken spectrally (exact on every resolved Fourier mode,
 * zero on the Nyquist mode), so that errors come from the time stepping alone.  It takes
 * fd_order = 0, precision GBS_F64, a power-of-two size n in [8, 2048] per problem, no media and
 * no adjoint; one field u.  Its stability bound uses |lambda| <= pi / dx. */
enum { GBS_WAVE1D = 1, GBS_ACOUSTIC = 2, GBS_ONEWAY_SPECTRAL = 3 };
enum { GBS_F32_STATE_F64_COMBINE = 0, GBS_F64 = 1, GBS_F32X2 = 2 }; /* gbs_problem.precision */
enum { GBS_KERNEL_AUTO = 0, GBS_KERNEL_PLAIN = 1, GBS_KERNEL_FUSED = 2 }; /* gbs_set_option */

/* Problem description.  All problems of a batch share system, ndim, fd_order
 * and precision; each has its own grid and spacing. */
typedef struct {
  int system;             /* GBS_WAVE1D (u_t = v_x, v_t = u_x) or GBS_ACOUSTIC
                             (p_t = -kappa div u, u_t = -grad p / rho)          */
  int ndim;               /* 1 for GBS_WAVE1D; 1, 2 or 3 for GBS_ACOUSTIC        */
  int fd_order;           /* 4 or 6: periodic centred finite differences (0 for
                             GBS_ONEWAY_SPECTRAL)                                */
  int precision;          /* GBS_F32_STATE_F64_COMBINE, GBS_F64 or GBS_F32X2     */
  int batch;              /* number of independent problems, >= 1               */
  int enable_adjoint;     /* nonzero: reserve workspace for gbs_adjoint_step     */
  const int64_t* shape;   /* host, batch x 3: (nx, ny, nz), unused dims = 1      */
  const double* dx;       /* host, batch x 3 grid spacings (unused dims ignored) */
} gbs_problem;

/* Bytes of device workspace gbs_create would allocate for `pb` when schemes
 * with up to `max_steps` steps per sequence are used (0 on invalid input).
 * No counterpart in the paper: sizing of the storage for the levels of
 * Sec. 2.1 eq. "GBS".  Host only; never touches the GPU. */
size_t gbs_workspace_bytes(const gbs_problem* pb, int max_steps);

/* Number of scalars in one state buffer of `pb` (sum over problems of F * points):
 * the length of the method-of-lines state y of y' = f(y) (Sec. 2.1).  Host only;
 * 0 on invalid input. */
size_t gbs_state_elems(const gbs_problem* pb);

/* Create a handle.  kappa and rho are device arrays (media layout, state
 * element type) for GBS_ACOUSTIC and must be NULL for GBS_WAVE1D.  The library
 * keeps the kappa pointer (it is read by every step) and precomputes
 * b = 1/rho into its workspace.  `cuda_stream` is a cudaStream_t (NULL: the
 * legacy default stream).  All workspace is allocated here, none later, except
 * the adjoint level store sized in gbs_set_weights.
 * Errors: GBS_ERR_INVALID (bad description or pointers), GBS_ERR_NOMEM,
 * GBS_ERR_CUDA; *out is NULL on error.
 * Defines the ODE y' = f(y) that the macro-steps advance (Sec. 2.1); the
 * paper leaves the spatial operator open, so f is one of the periodic systems
 * of gbs_problem.system (Sec. 4's spectral one-way wave among them). */
gbs_status gbs_create(const gbs_problem* pb, const void* kappa, const void* rho,
                      void* cuda_stream, gbs_handle* out);

/* Replace the media (same layout rules as gbs_create); recomputes b = 1/rho.
 * The coefficients of f in y' = f(y) (Sec. 2.1); the paper's own test problem
 * has none.  Waits for the handle's stream (the wave-speed maximum used by
 * gbs_stability_limit is read back); the caller keeps kappa alive.  Errors:
 * GBS_ERR_INVALID (NULL handle, a non-acoustic handle, non-device pointers),
 * GBS_ERR_NONFINITE (a non-positive or non-finite wave speed), GBS_ERR_CUDA. */
gbs_status gbs_set_media(gbs_handle h, const void* kappa, const void* rho);

/* Define the scheme of weight slot `slot` (0 <= slot < GBS_MAX_SLOTS).
 * order_p: even order of accuracy p; n_dep must equal p/2.  steps_dep /
 * steps_free: host arrays of distinct even step counts in [2, GBS_MAX_STEPS],
 * n_dep + n_free <= GBS_MAX_SEQ.  c_free: host array of the n_free free
 * weights (taken as exact binary values); may be NULL when n_free == 0.
 * c_full: optional host array of all n_dep + n_free weights (dependent
 * first); when given it is validated and used as is, otherwise the dependent
 * weights are solved from Sec. 3.7 eq. "cdep_computation" in double-double
 * arithmetic (Bjorck-Pereyra for the dual Vandermonde system) and rounded to
 * FP64.  Either way the rounded weights must satisfy every order constraint
 * to within 64 ulp of sum_k |c_k| h_k^(2j), else GBS_ERR_ORDER.  The order
 * of summation in the combine is dependent weights first, then free ones.
 * Also computes the scheme's imaginary stability boundary (Sec. 2.2). */
gbs_status gbs_set_weights(gbs_handle h, int slot, int order_p, int n_dep, const int* steps_dep,
                           int n_free, const int* steps_free, const double* c_free,
                           const double* c_full);

/* Read back a slot: *m sequences, steps[m] and FP64 weights c[m] (host arrays
 * of at least GBS_MAX_SEQ entries, each may be NULL), and *isb = the
 * imaginary stability boundary of R(xi) = sum_k c_k P_k(xi), found by a dense
 * scan of |R(iy)| - 1 > 1e-12 refined by bisection (may be NULL).
 * R(xi) is the scheme's stability polynomial on Dahlquist's test equation
 * (App. A.1) and the ISB its imaginary-axis coverage (Sec. 2.2).  Host only.
 * Errors: GBS_ERR_INVALID (bad handle or slot), GBS_ERR_STATE (slot unset). */
gbs_status gbs_get_weights(gbs_handle h, int slot, int* m, int* steps, double* c, double* isb);

/* Batched problems: host array slot_per_problem[batch] selects each
 * problem's weight slot (default: all use slot 0).  No counterpart in the
 * paper (batches of independent problems are a library addition; each
 * problem still takes the macro-step of Sec. 2.1).  Errors: GBS_ERR_INVALID
 * (NULL handle or array, slot out of range), GBS_ERR_STATE (a slot without
 * weights), GBS_ERR_CUDA (table upload). */
gbs_status gbs_assign_slots(gbs_handle h, const int* slot_per_problem);

/* Largest stable H per problem as ISB(slot) / rho_hat, where rho_hat =
 * max(sqrt(kappa b)) * sqrt(sum_d (s_max / dx_d)^2) bounds the spectral
 * radius of the acoustic operator (s_max = max |stencil symbol|; for the 1D
 * wave system kappa b = 1).  H_max: host array of `batch` doubles.
 * Follows App. A.1 (the eigenvalues of the method-of-lines operator, scaled by
 * the step, must lie in the stability domain; for these wave operators they
 * lie on the imaginary axis) with the ISB of Sec. 2.2.  Host only (the wave
 * speeds are read back when the media are set).  Errors: GBS_ERR_INVALID
 * (NULL handle or H_max), GBS_ERR_STATE (a used slot has no weights). */
gbs_status gbs_stability_limit(gbs_handle h, double* H_max);

/* Advance every problem by n_macro macro-steps of size H (Sec. 2.1 / 3.2):
 * y_out = (macro-step)^n_macro (y_in).  y_in, y_out: device state buffers;
 * y_in == y_out is allowed, other overlap is not.  n_macro == 0 copies.
 * Asynchronous; allocates nothing.  Errors: GBS_ERR_INVALID, GBS_ERR_STATE
 * (a used slot has no weights), GBS_ERR_CUDA (launch failure). */
gbs_status gbs_step(gbs_handle h, const void* y_in, void* y_out, double H, int n_macro);

/* Sequence-parallel macro-step, first half (Sec. 3.6: the sequences of one
 * macro-step are independent, and the paper spreads them over cores, folding
 * pairs whose step counts add up to N_max onto one core).  Runs one macro-step
 * of size H for the sequences k whose bit (seq_mask >> k) & 1 is set (k = the
 * position in each problem's scheme, dependent sequences first) and writes
 * their share of the combine into partial: an FP64 array in the state layout
 * (state_elems doubles, device, owned by the caller).  The shares of all ranks
 * -- disjoint masks covering every sequence -- summed element by element (an
 * FP64 all-reduce), then given to gbs_combine_partial, give the macro-step's
 * result.  For FP32 states the share is sum_k c_k (y*_k - y_0) in the increment
 * form; for FP64 and FP32-pair states sum_k c_k y*_k.  One macro-step per call;
 * y_in is not modified.  A mask different from the previous call's re-plans
 * the time-blocked kernel's schedule (host work, and an allocation if it
 * needs more room).  Errors: GBS_ERR_INVALID (NULL handle or pointers, a mask
 * selecting no sequence, the spectral system), GBS_ERR_STATE (a slot without
 * weights), GBS_ERR_NOMEM, GBS_ERR_CUDA. */
gbs_status gbs_step_partial(gbs_handle h, const void* y_in, double* partial, double H, uint32_t seq_mask);

/* Sequence-parallel macro-step, second half: y_out = y_in + total for FP32
 * states (increment form), y_out = total for FP64 and FP32-pair states, total
 * being the element-wise FP64 sum of every rank's gbs_step_partial share for
 * the same y_in and H (the combine of Sec. 2.1 / 3.2 completed), rounded once
 * to the state type.  y_out == y_in is allowed.  Asynchronous.  Errors:
 * GBS_ERR_INVALID, GBS_ERR_STATE, GBS_ERR_CUDA. */
gbs_status gbs_combine_partial(gbs_handle h, const void* y_in, const double* total, void* y_out);

/* As gbs_step with one H per problem (host array of `batch` doubles): the
 * macro-step of Sec. 2.1 / 3.2 for each problem with its own section length.
 * Errors as gbs_step, and GBS_ERR_INVALID for a NULL array or an H that is
 * not finite and positive. */
gbs_status gbs_step_batch(gbs_handle h, const void* y_in, void* y_out, const double* H,
                          int n_macro);

/* End-to-end variant: y_in and y_out are HOST buffers (pinned or pageable).
 * Copies in, steps on the device, copies out and waits for completion.
 * Computes what gbs_step computes (Sec. 2.1 / 3.2) through library-owned
 * device staging; allocates nothing.  Errors as gbs_step. */
gbs_status gbs_step_host(gbs_handle h, const void* y_in_host, void* y_out_host, double H,
                         int n_macro);

/* End-to-end over a stream of independent inputs (Sec. 2.1 / 3.2 per input):
 * y_out_host[i] = (macro-step)^n_macro (y_in_host[i]) for i = 0..count-1,
 * every y_in_host[i] / y_out_host[i] a HOST state buffer in the layout of
 * gbs_step (pinned memory lets the copies run asynchronously; pageable memory
 * works but serialises them).  The arrays themselves are host arrays of count
 * pointers; an output may alias another output (the device-to-host copies run
 * in order); an output must not alias a later input.  Two library-owned device staging states
 * alternate: the host-to-device copy of input i+1 and the device-to-host copy
 * of result i-1 run on two copy streams while the handle's stream steps input
 * i, so the copies hide behind the macro-steps where they are shorter.  Results
 * written to aliasing outputs land in input order.  Allocates nothing (the
 * staging states, the copy streams and their events are created by
 * gbs_create).  Returns when every result is in host memory; count == 0 is a
 * no-op.  Errors: GBS_ERR_INVALID for NULL arrays or entries, otherwise as
 * gbs_step. */
gbs_status gbs_step_host_stream(gbs_handle h, const void* const* y_in_host, void* const* y_out_host,
                                int count, double H, int n_macro);

/* Discrete adjoint of ONE macro-step (the exact transpose of the forward
 * steps above; not in the paper).  With y_out = M(kappa) y_in:
 *   lam_in = M^T lam_out + S^T r
 *   grad_kappa += d< lam_out, M(kappa) y_in > / d kappa     (pointwise)
 * y_in: device state at the START of the macro-step.  lam_out: device
 * adjoint state at its end.  lam_in: device output (may equal lam_out).
 * grad_kappa: device double array (media layout), accumulated.  S^T r adds
 * rcv_resid[i] to field 0 at flat point index rcv_idx[i] (device arrays;
 * indices per problem 0, i.e. batch must be 1 when n_rcv > 0); n_rcv may be 0.
 * An index outside [0, points) is skipped and latches GBS_ERR_INVALID, which
 * gbs_sync() reports.  Requires enable_adjoint and GBS_ACOUSTIC.  GBS_F32X2 handles run
 * the adjoint kernels in FP32-pair arithmetic, like their forward steps (y_in, the media and
 * lam_out converted to pairs; lam_in written and grad_kappa accumulated in FP64). */
gbs_status gbs_adjoint_step(gbs_handle h, const void* y_in, const void* lam_out, void* lam_in,
                            double* grad_kappa, double H, const int64_t* rcv_idx, int n_rcv,
                            const void* rcv_resid);

/* Receiver misfit helper: resid[i] = y_field0[rcv_idx[i]] - data[i] (device
 * arrays, state element type) and, if J is non-NULL (device double), adds
 * 0.5 * sum_i resid[i]^2 to *J with a warp-shuffle reduction.  Indices are
 * flat points of field 0 of problem 0; one outside [0, points) gets a zero
 * residual and latches GBS_ERR_INVALID (reported by gbs_sync()).
 * Not in the paper: the receiver misfit whose gradient gbs_adjoint_step
 * serves. */
gbs_status gbs_misfit(gbs_handle h, const void* y, const int64_t* rcv_idx, int n_rcv,
                      const void* data, void* resid, double* J);

/* Adjoint of receiver sampling: lam[field 0][rcv_idx[i]] += values[i] (device
 * arrays; indices of problem 0, range-checked like gbs_misfit).  Used to seed
 * the adjoint with the misfit residual of the final state.  Not in the paper
 * (the transpose of gbs_misfit's sampling). */
gbs_status gbs_inject(gbs_handle h, void* lam, const int64_t* rcv_idx, int n_rcv, const void* values);

/* Norms over a whole state buffer, accumulated in FP64 with warp-shuffle and
 * block reductions in a fixed order: out[0] = sum (a - b)^2,
 * out[1] = sum b^2, out[2] = max |a - b|, out[3] = number of non-finite
 * entries of a.  `b` may be NULL (treated as zero).  out: host array of 4
 * doubles; the call waits for the result.  No counterpart in the paper: the
 * error measure of the parity checks and of the time-to-accuracy study.
 * Errors: GBS_ERR_INVALID (NULL handle, a or out), GBS_ERR_CUDA. */
gbs_status gbs_norms(gbs_handle h, const void* a, const void* b, double* out);

/* Tuning options: "kernel" = GBS_KERNEL_*, "graph" = 0/1 (CUDA-graph replay
 * of a macro-step), "check_stability" = 0/1 (gbs_step returns
 * GBS_ERR_UNSTABLE when H exceeds gbs_stability_limit), "time_kernels" = 0/1
 * (record CUDA events around every launch of the dominant kernel -- the
 * leap-frog step kernel, or the time-blocked pass kernel -- on the handle's
 * stream; graph replay is bypassed while it is on).  GBS_KERNEL_FUSED selects the
 * time-blocked kernels: for 2D acoustics the persistent dataflow kernel below (also chosen by
 * GBS_KERNEL_AUTO), for 3D acoustics with FP32 states the z-sweeping pass kernel, two
 * leap-frog levels per pass (Sec. 2.1 eq. "GBS"), whose results equal the one-level kernel's
 * bit for bit; it needs a second pair of level buffers (gbs_workspace_bytes counts them),
 * allocated when it is selected.  On GB300 the 3D pass kernel is slower than the one-level
 * kernel, so GBS_KERNEL_AUTO keeps the latter in 3D.  "zseg" = z-planes per block of the 3D
 * pass kernel (1..65536, default 128).  "seqfuse" = -1/0/1 (default -1: on in 2D, off in 3D,
 * where it measured slower on GB300): where the one-level
 * kernels run FP32 2D/3D acoustics, give every sequence its own pair of level buffers (2 m
 * states, m the scheme's sequence count, allocated when the weights are set and not counted by
 * gbs_workspace_bytes) so that one launch per leap-frog level advances all sequences that have
 * that level, reading f0 and the media from DRAM once for all of them; the results are those of
 * one sequence per launch up to the order of the FP64 combine's terms (sequences finish in
 * step-count order).  Without the memory the step runs one sequence per launch;
 * gbs_get_option answers 1 only where the fused launches are in use.  "seqgroup" = most
 * sequences per fused launch (-1 = by dimension, the default: all of a level's in 2D, 4 in 3D,
 * where a launch's z-neighbour planes must stay in the L2 cache; 0 = all; 1..16).  "hseg" = row-segment height of
 * the 2D time-blocked tiles (16..65536, default 256), "tmax" = most leap-frog levels per
 * time-blocked pass (0 = the kernel's largest, 4; or 2), "schedule" = order of the
 * time-blocked work queue (0 = longest remaining chain of passes first, the default;
 * 1 = pass by pass across all sequences) -- these three only shape the schedule and are
 * what an autotuner varies -- "spin_limit" = polls of a
 * dependency flag in the time-blocked kernel before it gives up and latches
 * GBS_ERR_TIMEOUT (default 2^20, about half a second), and
 * "inject_unsatisfiable_wait" = 0/1, a failure-detection test hook that makes
 * the kernel's first work item wait on a flag nothing sets (the wait runs out,
 * gbs_sync reports GBS_ERR_TIMEOUT, the handle stays usable), and "tma" = -1/0/1
 * (default -1): the FP32 one-step-per-launch kernel can stage the tiles of a single
 * 2D/3D acoustic problem whose nx is a multiple of 4 with tensor-memory-access
 * copies where a tile's box lies inside the grid (identical results to the load
 * staging; a copy that does not complete latches GBS_ERR_TIMEOUT); 1 uses them
 * wherever they apply, -1 only in 3D (where they measured faster), 0 never;
 * gbs_get_option answers 1 only where those copies are in use.  "combine" = 0/1
 * (default 0): how the time-blocked kernel's FP32-state path sums y_0 + sum_k c_k d*_k,
 * 0 in FP64 (the averages promoted exactly, FP64 FMAs, one rounding to FP32), 1 in
 * compensated FP32 pairs (error about 2^-48 of sum_k |c_k d*_k|, on the FP32 units;
 * faster on GB300, whose FP64 rate is a small fraction of its FP32 rate); the plain
 * kernels always sum in FP64.  gbs_get_option also
 * answers "kernel_in_use" (the GBS_KERNEL_* value gbs_step would run now).
 * Unknown names: GBS_ERR_INVALID.  No counterpart in the paper: these choose
 * how the macro-step is scheduled on the GPU, not what it computes. */
gbs_status gbs_set_option(gbs_handle h, const char* name, int64_t value);
gbs_status gbs_get_option(gbs_handle h, const char* name, int64_t* value);

/* Launch count and summed device time (ms, CUDA events) of the dominant
 * kernel since the previous call, recorded while "time_kernels" is on (the
 * forward step's leap-frog or pass kernel in gbs_step, the reverse leap-frog
 * kernel in gbs_adjoint_step); also
 * reports the algorithmic bytes those launches move (*bytes, may be NULL), the
 * per-launch figure being the unit cost of the kernel times the grid-point
 * updates it performs.  Waits for the stream; resets the counters.  No
 * counterpart in the paper (measurement).  launches and total_ms are host
 * pointers.  Errors: GBS_ERR_INVALID, GBS_ERR_CUDA. */
gbs_status gbs_kernel_time(gbs_handle h, int64_t* launches, double* total_ms, double* bytes);

/* Wait for the handle's stream and report a latched device-side error
 * (GBS_ERR_TIMEOUT from a bounded wait that ran out, GBS_ERR_INVALID from an
 * out-of-range receiver index), clearing it, or GBS_ERR_CUDA.  No counterpart
 * in the paper (library service). */
gbs_status gbs_sync(gbs_handle h);

/* Free the workspace and the handle (NULL is accepted).  Waits for work in
 * flight on the handle's stream first.  No counterpart in the paper. */
gbs_status gbs_destroy(gbs_handle h);

/* Last error message of `h` ("" if none); for h == NULL, the last error of a
 * failed gbs_create on this thread.  Valid until the next call on h.  No
 * counterpart in the paper. */
const char* gbs_last_error(gbs_handle h);

/* Number of GPU kernels this handle has launched (for launch accounting;
 * 0 for NULL).  No counterpart in the paper. */
int64_t gbs_kernel_launches(gbs_handle h);

/* ---------------------------------------------------------------------------
 * Stepping without any memory allocation.  The paper has no counterpart: this
 * is a service for callers that cannot call cudaMalloc -- e.g. an application
 * whose GPU memory is owned entirely by its own allocator or pool, or a
 * plug-in living inside such a process -- and therefore cannot create a
 * handle (gbs_create allocates its workspace).
 *
 * gbs_step_noalloc does what gbs_create + gbs_set_weights + gbs_step do for
 * one scheme, but keeps all of its scratch (leap-frog levels, shared first
 * right-hand side, FP64 accumulator, 1/rho, problem tables) in one array of
 * GBS_NOALLOC_SCRATCH_BYTES compiled into the library as a __device__
 * variable, which every GPU that loads the library reserves until the process
 * exits.  It allocates no GPU memory: it calls no cudaMalloc/cudaFree and no
 * allocating library routine (its host-side tables live on the stack; only the
 * per-thread error message is thread-local storage).
 *  - Arguments as in gbs_create (pb, kappa, rho; pb->enable_adjoint must be 0,
 *    batch <= 256), gbs_set_weights (order_p .. c_free; all problems use this
 *    scheme) and gbs_step (y_in, y_out, H, n_macro); cuda_stream is a
 *    cudaStream_t.  The caller owns every pointer it passes.  The weights are
 *    solved and checked as gbs_set_weights does (GBS_ERR_ORDER when the rounded
 *    weights break an order constraint, GBS_ERR_INVALID for a non-finite free
 *    weight); kappa and rho are not checked for non-positive or non-finite
 *    values (gbs_create does check them).
 *  - A problem whose scratch would exceed GBS_NOALLOC_SCRATCH_BYTES is
 *    rejected with GBS_ERR_INVALID; the message is returned by
 *    gbs_noalloc_last_error().
 *  - The first call on a device (with that device current) looks up the
 *    array's device address with cudaGetSymbolAddress.
 *  - The problem tables are copied into the array from pageable host memory:
 *    each call returns only after the work queued earlier on cuda_stream has
 *    finished, and no call may be made while cuda_stream is being captured
 *    (GBS_ERR_STATE, returned before anything is enqueued).  The macro-steps
 *    themselves run asynchronously on cuda_stream.
 *  - All calls on a device share the one array, which keeps the previous
 *    call's contents: calls whose GPU work overlaps (other streams or threads)
 *    race and must be serialised by the caller.
 * ------------------------------------------------------------------------- */
#define GBS_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
gbs_status gbs_step_noalloc(const gbs_problem* pb, const void* kappa, const void* rho, int order_p,
                            int n_dep, const int* steps_dep, int n_free, const int* steps_free,
                            const double* c_free, const void* y_in, void* y_out, double H,
                            int n_macro, void* cuda_stream);

/* Self-test of the library's exact FP32 -> FP64 promotion, which the FP64 combines use
 * instead of the conversion instruction (GB300 runs that instruction on its slow FP64 pipe):
 * for the float bit patterns first .. first + count - 1 (a range within [0, 2^32)), compares
 * the promotion's bits with the conversion instruction's on the current device and writes to
 * mismatches (host, 3 entries) the number of inputs that are not NaN and whose doubles differ
 * [0], of NaN inputs whose doubles differ in more than the quiet bit (bit 51) [1], and of NaN
 * inputs whose doubles differ in the quiet bit alone [2] (the conversion quiets a signalling
 * NaN; the promotion keeps its bits).  Synchronises the device; allocates nothing (the counters
 * are a static device array, so concurrent calls race).  No counterpart in the paper (a check
 * of an implementation detail).  Errors: GBS_ERR_INVALID (NULL mismatches, range outside
 * [0, 2^32)), GBS_ERR_CUDA. */
gbs_status gbs_selftest_f32_to_f64(uint64_t first, uint64_t count, uint64_t* mismatches);

/* Message of the last failed gbs_step_noalloc call on this thread ("" if none).
 * No counterpart in the paper. */
const char* gbs_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GBS_H */

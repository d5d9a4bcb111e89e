/*
 * eq.h - C ABI of the GB300 equilibrium-projection library (libeq.so).
 *
 * The operation (Zhou, Lebensohn, Reischig, Ludwig, Bhattacharya, "Imposing equilibrium on
 * measured 3-D stress fields using Hodge decomposition and FFT-based optimization"):
 * given a voxelized symmetric stress field S on a periodic nx x ny x nz grid, return the field
 * closest to it in L^2 whose divergence vanishes (Sec. 3.2).  By the Hodge decomposition of
 * Sec. 3.1 (Theorem 2) and the Fourier treatment of Sec. 4 this is, per wavevector k with
 * operator symbol Xi(k) and n = Xi / |Xi|,
 *     S^(k) <- S^ - n (x) (S^ n) - (S^ n) (x) n + (n . S^ n) n (x) n,
 * with the mean (k = 0) kept (Sec. 3.2, c0 = mean of S).  Xi is the continuous wavevector (CDO,
 * Sec. 4.1, Nyquist symbol 0) or the central-difference "modified" wavevector
 * sin(2 pi m / N) / h (DDO, Sec. 4.2) used for fields with grain-boundary discontinuities.
 *
 * Field layout at the boundary (all entry points): a contiguous array of `batch` fields, each
 * [6][nz][ny][nx] with x fastest, components in Voigt order (xx, yy, zz, yz, xz, xy), element
 * type float (EQ_F32) or double (EQ_F64).  Device pointers are CUDA device memory of the
 * current device, owned by the caller; host pointers are host memory owned by the caller.
 *
 * Errors: every entry point returns an eq_status; no C++ exception crosses the ABI.  A failed
 * call leaves a message for eq_last_error() (per thread).  Errors of work already queued on a
 * stream (asynchronous CUDA errors) surface at the next eq_norms / eq_serve_poll.
 */
#ifndef EQ_H
#define EQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EQ_OK = 0,
  EQ_ERR_INVALID = 1,    /* bad argument, unsupported size or option */
  EQ_ERR_OOM = 2,        /* device or host allocation failed; over the server's HBM budget */
  EQ_ERR_CUDA = 3,       /* a CUDA call failed (message in eq_last_error) */
  EQ_ERR_TIMEOUT = 4,    /* a bounded wait ran out */
  EQ_ERR_BUSY = 5,       /* server queue full */
  EQ_PENDING = 6,        /* request not finished yet */
  EQ_ERR_NOT_FOUND = 7   /* unknown ticket */
} eq_status;

/* Element type at the boundary.  EQ_F64 fields are read and written as FP64; where every axis
 * length of the plan is 512 or at most 256, the plain projection (eq_project and its host forms)
 * computes in double-float arithmetic: each value an unevaluated sum of two FP32 numbers, about
 * 48 significant bits, relative error about 1e-14 against an exact-arithmetic result (FP64
 * instructions run at a small fraction of the FP32 rate on this GPU).  It keeps FP32's exponent
 * range: spectra reach nx ny nz max|S| and the norm sums its square, so keep nx ny nz max|S| below
 * about 1e18 (stresses below about 7e9 at 512^3; values below about 1e-30 lose precision).  The
 * Hodge and padded forms, other lengths, and every call when the environment variable
 * EQ_F64_ARITH=native is set at plan creation use FP64 instructions for the transforms. */
typedef enum { EQ_F32 = 0, EQ_F64 = 1 } eq_dtype;

/* Derivative symbol: DDO = central-difference modified wavevector (Sec. 4.2, eq. eq:diff);
 * CDO = continuous wavevector 2 pi s / L with 0 at the Nyquist index (Sec. 4.1). */
typedef enum { EQ_OP_DDO = 0, EQ_OP_CDO = 1 } eq_op;

/* Modes where the symbol vanishes but k != 0 (the Nyquist corners of an even grid).  KEEP
 * leaves them unchanged (every field is divergence-free there, so the closest field keeps
 * them; this keeps the map an orthogonal projection).  ZERO removes them, which is what the
 * literal Euler-Lagrange route inc(inc(S) / biharmonic) of Sec. 3.2-3.3 produces. */
typedef enum { EQ_NYQ_KEEP = 0, EQ_NYQ_ZERO = 1 } eq_nyquist;

/* What the plan returns.  EQUILIBRIUM: the closest divergence-free field S_equil (Sec. 3.2).
 * COMPATIBILITY: the closest strain-compatible field c0 + (S - S_equil), i.e. sym grad y + c0 of
 * the Hodge decomposition (Sec. 3.1, Theorem 2), the dual constraint named in the Conclusions;
 * at the Nyquist corners it is 0 under KEEP and the input under ZERO.  The norms describe the
 * returned field either way (resid = S_in - S_out, div_out of S_out). */
typedef enum { EQ_TARGET_EQUILIBRIUM = 0, EQ_TARGET_COMPATIBILITY = 1 } eq_target;

typedef struct {
  eq_op op;              /* default EQ_OP_DDO */
  double hx, hy, hz;     /* voxel spacing, default 1 (all > 0) */
  eq_nyquist nyq;        /* default EQ_NYQ_KEEP */
  int want_linf;         /* 1: also compute resid_linf (needs d_in != d_out); default 1 */
  int graph;             /* 1: capture the passes in a CUDA graph on first use of a (d_in, d_out)
                            pair and replay it while the pair is unchanged; default 1 */
  eq_target target;      /* default EQ_TARGET_EQUILIBRIUM */
} eq_plan_opts;

/* Per-field diagnostics, FP64.  ||A|| = sqrt(mean over voxels of A:A) with A:B = sum_ij A_ij B_ij
 * (off-diagonal Voigt entries weigh 2); resid = S_in - S_out; div_* is the RMS of the divergence
 * vector computed with the plan's operator (Sec. 4, Fig. 1c,d). */
typedef struct {
  double mean[6];        /* c0, per Voigt component (Sec. 3.2) */
  double norm_in, norm_out;
  double resid_l2, resid_rel, resid_linf;
  double div_in_l2, div_out_l2;
  int flags;             /* EQ_FLAG_* */
} eq_norms_t;

#define EQ_FLAG_NONFINITE 1   /* the input held a NaN or an infinity, or a partial sum of it
                                 overflowed the working type (inputs near FLT_MAX in FP32) */
#define EQ_FLAG_NO_LINF 2     /* resid_linf was not computed (in-place call or want_linf = 0) */

typedef struct eq_plan eq_plan;
typedef struct eq_server eq_server;

/* Default options (DDO, unit spacing, KEEP, want_linf = 1, graph = 1, EQUILIBRIUM). */
void eq_plan_opts_default(eq_plan_opts* opts);

/* Create a plan for `batch` fields of one grid size.  Sizes are 1..1024 per axis (powers of two
 * take compile-time-specialised kernels; other lengths the runtime-length path, see
 * eq_plan_create_varlen for its limits).  Allocates
 * the plan's device tables and reduction buffers on the current device (no field-sized
 * workspace: the spectrum lives in the caller's output buffer).  opts == NULL: defaults. */
eq_status eq_plan_create(int nx, int ny, int nz, eq_dtype dtype, int batch,
                         const eq_plan_opts* opts, eq_plan** out);

/* Create a plan for `count` fields of different grid sizes (dims: nx, ny, nz per field, 3 *
 * count ints), all projected by one launch per pass (a persistent grid over every field's
 * tiles).  The fields are packed back to back in the buffers, field f starting at element
 * 6 * sum_{g < f} nx_g ny_g nz_g.  Each axis length must be 1..1024 and, when it has a prime
 * factor above 13, at most 512 (it then runs Bluestein's algorithm).  Norms come back in field
 * order (eq_norms with `count` entries). */
eq_status eq_plan_create_varlen(const int* dims, int count, eq_dtype dtype,
                                const eq_plan_opts* opts, eq_plan** out);

/* Project the plan's `batch` fields d_in -> d_out on `cuda_stream` (a cudaStream_t, NULL =
 * legacy default stream).  d_out may equal d_in (then resid_linf is not computed).  Both must
 * hold batch * 6 * nx * ny * nz elements of the plan's dtype and be 16-byte aligned.  The call
 * only enqueues work; it returns before the result is ready.  Calls on one plan share its
 * reduction buffers, so they must be ordered (one stream, or synchronised between streams).  Steps (Sec. 3.3): forward 3-D
 * DFT, per-mode projector, inverse DFT, norms; the mean is taken in FP64. */
eq_status eq_project(eq_plan* plan, const void* d_in, void* d_out, void* cuda_stream);

/* eq_project plus the vector field y of the Hodge decomposition (Sec. 3.1, Theorem 2):
 * S = inc(H) + sym grad y + c0, so sym grad y = S - S_equil with the plan's operator as the
 * derivative.  y is periodic and mean-free; it is 0 at the modes where the operator vanishes.
 * d_out receives exactly what eq_project writes (same kernels, same target); d_y (device, the
 * plan's dtype, 16-byte aligned, disjoint from d_in and d_out) holds batch * 4 * nx * ny * nz
 * elements: per field the planes y_x, y_y, y_z and one working plane that ends near zero.
 * Power-of-two plans only (EQ_ERR_INVALID otherwise).  Extra cost: one x pass reading the
 * spectrum and two strided passes over the 4-plane buffer.  Their times are counted in the x
 * and z-inverse slots of eq_plan_pass_ms. */
eq_status eq_project_hodge(eq_plan* plan, const void* d_in, void* d_out, void* d_y,
                           void* cuda_stream);

/* A non-periodic specimen (Sec. 5.2): d_in holds batch fields of sx * sy * sz voxels (layout
 * [batch][6][sz][sy][sx], the plan's dtype); each is placed at the origin corner of the plan's
 * periodic grid (nx, ny, nz) >= (sx, sy, sz) with zero stress in the rest of the grid (the
 * buffer region of free surfaces; on a periodic grid the corner placement equals a buffer on
 * both sides, and an axis with no padding stays periodically connected), the whole grid is
 * projected, and the specimen region is written to d_out (same layout as d_in; may equal d_in).
 * The norms are those of the padded grid except resid_linf, taken over the specimen.  Power-of-
 * two plans only.  The first call allocates the padded workspace (plan-owned, one grid per
 * field); the padding and the cut run as their own kernels around the plan's passes. */
eq_status eq_project_padded(eq_plan* plan, int sx, int sy, int sz, const void* d_in, void* d_out,
                            void* cuda_stream);

/* Same as eq_project with host buffers: copies host_in to a plan-owned device buffer
 * (allocated on first use, 2 x field bytes), projects, copies back to host_out, and waits for
 * completion.  Host buffers should be pinned for full copy bandwidth. */
eq_status eq_project_host(eq_plan* plan, const void* host_in, void* host_out, void* cuda_stream);

/* eq_project_host without the final wait: the copy in, the projection and the copy out are only
 * enqueued on cuda_stream (done when the stream reaches that point; eq_norms waits for it).  The
 * host buffers must stay valid and untouched until then, and calls on one plan share its device
 * staging buffer, so they must be ordered.  Two plans on two streams keep two fields in flight:
 * one field's copy in overlaps another's projection and copy out. */
eq_status eq_project_host_async(eq_plan* plan, const void* host_in, void* host_out, void* cuda_stream);

/* Wait for the plan's last eq_project and copy its `batch` diagnostics to host_out.  The call's
 * last kernel has written them, with the plan's error flag, into mapped pinned host memory, so
 * this waits for the call's event and issues no copy of its own.  EQ_ERR_TIMEOUT (and the flag
 * cleared): a bounded wait inside one of the call's kernels ran out; its results are invalid. */
eq_status eq_norms(eq_plan* plan, eq_norms_t* host_out);

/* Failure-detection self-test (the paper has no counterpart): enqueue on cuda_stream one kernel
 * that runs the bounded mbarrier wait of the TMA passes, limited to `polls` polls (about 64 ns
 * each after the first 64), on a barrier that nothing completes, and raises the plan's error
 * flag when it runs out, as a pass would.  The wait always ends: no fault, no hang.  The next
 * eq_norms then returns EQ_ERR_TIMEOUT and clears the flag, after which the plan works as
 * before.  EQ_ERR_INVALID: NULL plan, polls outside 1..2^24, or a runtime-length plan (whose
 * kernels have no waits). */
eq_status eq_selftest_wait_timeout(eq_plan* plan, long long polls, void* cuda_stream);

/* Autotune the plan on the caller's buffers (d_in is only read; d_out is overwritten; work is
 * enqueued on cuda_stream and the call waits for it).  Runtime-length plans time candidate
 * shapes of each pass (tile columns and threads of the z and y passes, row pairs per block of the
 * x pass) and keep the fastest; when the environment variable EQ_TUNE_CACHE names a file the
 * choice is stored there (a JSON object keyed by sizes, dtype, options and GPU) and later plans
 * with the same key start from it.  Power-of-two plans keep, per pass, the faster of the TMA /
 * bulk-copy fed and the plain-load variants.  Results do not depend on the choice beyond the
 * order of the FP64 norm reductions. */
eq_status eq_plan_autotune(eq_plan* plan, const void* d_in, void* d_out, void* cuda_stream);

/* Device bytes owned by the plan (tables, reduction buffers, host-call staging if any). */
size_t eq_plan_workspace_bytes(const eq_plan* plan);

void eq_plan_destroy(eq_plan* plan);

/* Per-pass timing with CUDA events recorded on the launch stream between the kernels of
 * eq_project (for measurement; off by default).  max_calls > 0 reserves event sets for that many
 * subsequent eq_project calls and turns timing on; 0 turns it off.  The passes, in order:
 *   0 z forward, 1 mean finalisation, 2 y forward, 3 x forward + projector + x inverse,
 *   4 y inverse, 5 z inverse, 6 norm finalisation. */
#define EQ_NUM_PASSES 7
eq_status eq_plan_set_timing(eq_plan* plan, int max_calls);

/* Wait for the timed calls and return, per pass, the summed device time in milliseconds over
 * them (ms_out: EQ_NUM_PASSES entries) and their number; then turn timing off (timed calls are
 * launched pass by pass instead of replaying the plan's graph; eq_plan_set_timing again to time
 * more calls). */
eq_status eq_plan_pass_ms(eq_plan* plan, double* ms_out, int* ncalls_out);

/* ---- projection without any allocation ------------------------------------------------
 * For callers that cannot allocate device memory when they project: code that runs under a
 * fixed memory budget or a caller-owned allocator, or a loop in which CUDA allocation calls are
 * not allowed.  The paper has no counterpart; this is a library facility.
 * One FP32 field, power-of-two axis lengths 1..EQ_STATIC_MAX_N.  The caller passes d_in, d_out
 * (6 nx ny nz floats each; equal or disjoint) and optionally d_norms (device memory for one
 * eq_norms_t; NULL = do not report).  Tables and reduction partials live in a fixed
 * EQ_STATIC_SCRATCH_BYTES array in device memory that the library declares; every GPU that loads
 * the library holds it until the process exits.  The call makes no cudaMalloc/cudaFree and calls
 * no allocating library routine; it enqueues work on cuda_stream and returns.  The first call on
 * each device (with that device current) looks up the array's device address and remembers the
 * context it belongs to; a call that finds another context current (after cudaDeviceReset, for
 * one) looks it up again.  Make those first calls before any stream capture.  All calls share the array: calls whose work overlaps on the
 * GPU race on it, so order them (one stream, or synchronise).  Grids whose scratch would not fit
 * are rejected with EQ_ERR_INVALID.  Results equal eq_project's for the same field. */
#define EQ_STATIC_SCRATCH_BYTES (1u << 20)
#define EQ_STATIC_MAX_N 512
eq_status eq_project_static(int nx, int ny, int nz, const eq_plan_opts* opts, const float* d_in,
                            float* d_out, eq_norms_t* d_norms, void* cuda_stream);

/* ---- serving ------------------------------------------------------------------------
 * A request loop for single fields arriving over time.  A scheduler thread admits queued
 * requests in arrival order as soon as one of `max_inflight` slots (CUDA streams) is free and the
 * request's device footprint (input + output field, 2 x 6 nx ny nz x element size) fits in
 * `hbm_budget_bytes` next to the requests in flight; each admitted request runs H2D copy,
 * projection and D2H copy on its slot's stream, so work of different requests overlaps on the
 * device.  A plan thread builds the plan of each queued request ahead of its admission (or takes
 * an idle one of the same grid and options from a least-recently-used cache of at most 64), so
 * no plan is built on the scheduler's path; the budget covers the buffers in flight and the
 * plans in flight or cached, whose idle members are released when the queue's head needs the
 * room.  Results of a field do not depend on what else is in flight (same kernels, fixed-order
 * reductions).
 * Server calls are thread-safe; the server uses the device current at creation. */
eq_status eq_server_create(size_t hbm_budget_bytes, int max_inflight, eq_server** out);

/* Queue one field (host buffers, caller-owned, kept alive until eq_serve_poll returns EQ_OK or
 * the server is destroyed; pinned memory gives full copy bandwidth).  opts == NULL: defaults.
 * EQ_ERR_OOM if the request alone cannot fit the budget, EQ_ERR_BUSY if the queue is full. */
eq_status eq_serve_submit(eq_server* server, int nx, int ny, int nz, eq_dtype dtype,
                          const eq_plan_opts* opts, const void* host_in, void* host_out,
                          unsigned long long* ticket);

/* Wait up to timeout_us (0 = do not wait) for a request.  EQ_PENDING: not finished yet (the ticket
 * stays valid).  Otherwise the ticket is consumed: EQ_OK with its norms (nullable) and latency
 * from submit to completion in seconds (nullable), or the request's error status.
 * EQ_ERR_NOT_FOUND: unknown or already consumed ticket. */
eq_status eq_serve_poll(eq_server* server, unsigned long long ticket, int timeout_us,
                        eq_norms_t* out, double* latency_s);

/* Withdraw a request that has not started: EQ_OK (the ticket is consumed; a plan prepared for it
 * goes back to the server's cache), EQ_ERR_BUSY if it is already on the device or its plan is
 * being built (poll it instead), EQ_ERR_NOT_FOUND for an unknown or consumed ticket. */
eq_status eq_serve_cancel(eq_server* server, unsigned long long ticket);

/* Counters of a server since its creation (totals) and its state at the call (current). */
typedef struct {
  unsigned long long submitted, admitted, completed, failed; /* totals */
  unsigned long long rejected;          /* submits refused: EQ_ERR_OOM or EQ_ERR_BUSY */
  unsigned long long cancelled;         /* eq_serve_cancel successes */
  unsigned long long plans_created, plans_reused, plans_evicted;
  double plan_create_seconds;           /* host time spent building plans (on the plan thread) */
  long long queued, inflight;           /* current */
  long long inflight_peak;              /* most requests on the device at once */
  unsigned long long hbm_in_use;        /* current: buffers in flight + live plans' device bytes */
  unsigned long long hbm_in_use_peak;
  unsigned long long hbm_budget;
  long long plans_cached;               /* idle plans kept for reuse */
} eq_server_stats_t;
eq_status eq_server_stats(eq_server* server, eq_server_stats_t* out);

/* Stop the server: queued requests are cancelled, requests already on the device complete, then
 * every resource is released.  The server and its tickets are invalid afterwards. */
void eq_server_destroy(eq_server* server);

/* ---- Grain averaging (Sec. 5.1) -----------------------------------------------------------
 * The synthetic measurement of Sec. 5.1 / Table 1 averages a stress field over each grain of a
 * polycrystal, as a grain-resolved diffraction reconstruction reports it.  A grain map is fixed
 * across the fields averaged with it, so it becomes an object once. */
typedef struct eq_grains eq_grains;

/* grain_map: host array of nx*ny*nz grain ids in [0, ngrains), x fastest (any id outside that
 * range: EQ_ERR_INVALID, before any device work).  Sorts the voxels by grain on the host (a
 * counting sort that keeps voxel order within a grain) and uploads the per-grain voxel lists and
 * the map to the current device: about 12 bytes per voxel of device memory, owned by the object. */
eq_status eq_grains_create(const int* grain_map, int nx, int ny, int nz, int ngrains,
                           eq_grains** out);

/* For `batch` fields d_in (device, dtype, layout [batch][6][nz][ny][nx]) write the per-grain means
 * of the six Voigt components to d_means (device, FP64, [batch][ngrains][6]; a grain with no voxel
 * gets 0) and, when d_avg is not NULL, the grain-averaged fields (every voxel carries its grain's
 * mean; same layout and dtype as d_in; d_avg may equal d_in).  Sums run in a fixed order (FP64;
 * FP32 data: compensated FP32 per thread, FP64 across threads): results do not depend on timing.
 * Only enqueues work on cuda_stream; a call with d_avg and a larger batch (or dtype) than before
 * first allocates the object's copy of the means in the fields' dtype. */
eq_status eq_grain_average(eq_grains* grains, eq_dtype dtype, int batch, const void* d_in,
                           double* d_means, void* d_avg, void* cuda_stream);

/* Release the object's device memory (NULL: no-op).  Work using it must have completed. */
void eq_grains_destroy(eq_grains* grains);

/* Message of the calling thread's last failed call ("" if none). */
const char* eq_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EQ_H */

/*
 * stencil7.h -- C ABI of the GB300 BiCGStab library for 7-point stencil systems.
 *
 * The library solves A x = b, where A is the nonsymmetric matrix of a
 * 7-point finite-difference stencil on a structured nx*ny*nz mesh (Fan et al.,
 * "Fast Stencil-Code Computation on a Wafer-Scale Processor", SC20: Sec. III,
 * Eq. 1, and Sec. IV), by standard BiCGStab (Algorithm 1).  Every step of the
 * iteration runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.  A mesh vector has nx*ny*nz elements stored x-fastest:
 *   cell (x, y, z) is element i = x + nx*(y + ny*z).
 * Operator.  Row i of A is
 *   (A v)_i = diag_i v_i + xm_i v_{i-1}     + xp_i v_{i+1}
 *                        + ym_i v_{i-nx}    + yp_i v_{i+nx}
 *                        + zm_i v_{i-nx*ny} + zp_i v_{i+nx*ny},
 *   the six off-diagonals named by axis and sign as in Sec. IV-A; a
 *   neighbour outside the mesh contributes zero (homogeneous Dirichlet).
 * Diagonal preconditioning.  By default the library stores the operator with
 *   a unit main diagonal, A~ = D^-1 A (Sec. IV scales the operator by its
 *   diagonal, which leaves ones there, and stores the six others); each
 *   off-diagonal is divided by its row's diagonal in float64 and rounded once
 *   (round to nearest even) to the storage type.  Solves then run on
 *   A~ x = D^-1 b, which has the same solution; tolerances and residual
 *   histories refer to that scaled system.
 * Memory.  Every pointer argument may be host memory (pageable or pinned) or
 *   device memory of the current device; the library tells them apart with
 *   the CUDA pointer attributes and stages host data itself.  Buffers passed
 *   in stay owned by the caller; the library keeps no pointer to them after
 *   the call returns.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *   default stream).  Calls that return results to the host (iteration counts,
 *   norms, histories) synchronise that stream before returning; stencil7_apply
 *   with device buffers does not.
 * Errors.  Every entry point returns an S7_* code; nothing aborts.  After a
 *   non-zero return, s7_last_error() gives a one-line description (per host
 *   thread).  A handle stays usable after S7_EBREAKDOWN / S7_ENOTCONV.
 * Threads.  A handle must not be used by two host threads at once.
 * Devices.  An entry point that takes a handle runs on the handle's device
 *   and leaves the calling thread's current device as it found it.
 */
#ifndef STENCIL7_H
#define STENCIL7_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define S7_OK          0  /* success (for solves: converged to tol)                  */
#define S7_EINVAL      1  /* bad argument: size, null pointer, dtype combination      */
#define S7_ENOMEM      2  /* device (or pinned host) allocation failed                */
#define S7_EBREAKDOWN  3  /* BiCGStab breakdown: (r0,s)=0, omega=0, (r0,r)=0 or a
                             non-finite scalar; x and the history up to the last
                             completed step are returned                              */
#define S7_ENOTCONV    4  /* maxit steps taken without reaching tol; x and the full
                             history are valid                                       */
#define S7_ETIMEOUT    5  /* a bounded wait expired (serving waits)                   */
#define S7_ECUDA       6  /* a CUDA runtime call failed; see s7_last_error()          */
#define S7_EAGAIN      7  /* result not ready yet (s7_server_poll)                    */
#define S7_ECANCELED   8  /* request cancelled                                        */

/* ---- element types ---- */
typedef enum {
  S7_F64 = 0,   /* IEEE binary64 */
  S7_F32 = 1,   /* IEEE binary32 */
  S7_BF16 = 2,  /* bfloat16 (8 significant bits, binary32 exponent range) */
  S7_F16 = 3    /* IEEE binary16 (the paper's 16-bit format, Sec. II) */
} s7_dtype;

typedef struct stencil7_op* stencil7_t;

/* Raw operator coefficients, as the application produced them.
 * diag and the six directions each point to nx*ny*nz elements of `dtype`
 * (S7_F64 or S7_F32), or to ONE element each when `constant` is 1 (a
 * constant-coefficient operator).  Entries that point outside the mesh are
 * read but multiply zero.  Host or device memory. */
typedef struct {
  const void* diag;
  const void* xm;
  const void* xp;
  const void* ym;
  const void* yp;
  const void* zm;
  const void* zp;
  s7_dtype dtype;
  int constant;
} s7_coeffs;

/* Creation options.  Zero-initialise and set what you need; a NULL pointer
 * means all defaults. */
typedef struct {
  s7_dtype storage;  /* type of the stored operator and of the Krylov vectors
                        r, r0, p, s, y.  S7_F64 computes in float64; S7_F32,
                        S7_BF16 and S7_F16 compute in float32 with the iterate x
                        kept in float32.  Default (0) = S7_F64; set explicitly. */
  int no_jacobi;     /* 1: store the raw seven diagonals instead of D^-1 A    */
  int keep_true;     /* 1: also keep the raw coefficients in float32, used by
                        stencil7_residual and bicgstab_solve_refined as the
                        "true" operator (required for the refined solver when
                        storage is 16-bit)                                    */
  int bx, by;        /* sweep tile: bx threads (each 16 bytes of x) by by rows;
                        0 = tuned default                                     */
  int zchunk;        /* z planes per thread block in the sweeps; 0 = default  */
  int check_every;   /* iterations per CUDA-graph launch between host checks
                        of the device convergence flag; 0 = default            */
  int stages;        /* depth of the asynchronous-copy pipeline of the two SpMV
                        sweeps of a step: 2 to 4 shared-memory stages; 1 = no
                        pipeline (direct loads); 0 = default                   */
  int pipe_kinds;    /* which sweeps use that pipeline: bit 0 = the p-update +
                        s = A p sweep, bit 1 = the q + y = A q sweep;
                        0 = default (tuned)                                    */
  int variant;       /* 0: Algorithm 1 as printed, three reductions and three
                        passes per step.  1: two reductions per step: beta_i
                        takes (r0, r_{i+1}) from the recurrence (r0, r_i) -
                        alpha (r0, s_i) - omega (r0, y_i), so the x and r
                        updates of one step fuse with the p update and SpMV
                        of the next; that fused pass also reduces (r0,
                        r_{i+1}) directly, which the next step starts from
                        (two passes, 104 instead of 116 bytes per cell in
                        float32; same iterates in exact arithmetic).
                        bicgstab_solve_batched runs it when every system
                        of the batch was created with it (a batch mixing
                        variants is S7_EINVAL); the server has its own
                        option (s7_server_opts.three_pass). */
  int step_cells;    /* cells per thread in the pipelined sweeps: the width
                        of the other sweeps (4; 2 for float64), or for 16-bit
                        storage 8 (one 16-byte copy per array and thread);
                        0 = default (8 for 16-bit storage)                    */
  int residual_f64;  /* arithmetic of the float64-accuracy residual sweeps (the
                        true residual of bicgstab_solve, stencil7_residual and
                        the refinement's outer residual): 0 = double words
                        (unevaluated sums of two binary32 numbers, about 48
                        significant bits; error a few 1e-14 of the terms'
                        magnitude; squared norms in binary64), several times
                        faster on GB300; 1 = binary64 throughout.  float64
                        storage always uses binary64.                          */
  int tma;           /* 1: the pipelined sweeps of single solves stage their
                        tiles with TMA tensor copies issued by the first warp
                        of a block, where the tile allows (16-byte cell runs,
                        a halo'd tile at most 256 cells wide); 0 (default):
                        with per-thread cp.async copies, which measured as
                        fast or faster on GB300 for these tiles.  Same
                        results either way.                                   */
} s7_opts;

/* Create an operator handle.  Copies the coefficients to library-owned device
 * memory, scaling them to a unit diagonal (unless opts->no_jacobi) in a CUDA
 * kernel, so the caller may free its copies on return.  nx, ny, nz >= 1 and
 * nx*ny*nz < 2^40.  Returns S7_EINVAL for bad sizes, a NULL pointer, a
 * storage/dtype combination not listed above, or a zero diagonal entry;
 * S7_ENOMEM if device memory runs out (nothing is leaked). */
int stencil7_create(stencil7_t* out, int nx, int ny, int nz,
                    const s7_coeffs* coeffs, const s7_opts* opts);

/* ---- the 2D 9-point operator (Sec. IV-A, "SpMV (2D)") ----
 * A 2D mesh of nx*ny cells, x-fastest (cell (x, y) is element i = x + nx*y),
 * with the 9-point stencil
 *   (A v)_i = diag_i v_i + xm_i v_{i-1} + xp_i v_{i+1} + ym_i v_{i-nx}
 *           + yp_i v_{i+nx} + xmym_i v_{i-1-nx} + xpym_i v_{i+1-nx}
 *           + xmyp_i v_{i-1+nx} + xpyp_i v_{i+1+nx},
 * the diagonal directions named by the signs of the neighbour's x and y
 * offsets; neighbours outside the mesh contribute zero.  The handle is a
 * stencil7_t like any other: stencil7_apply, stencil7_residual(_noalloc),
 * bicgstab_solve and bicgstab_solve_refined take it unchanged (vectors have
 * nx*ny elements; stencil7_info reports nz = 1).  bicgstab_solve_batched and
 * the server take 7-point operators only. */
typedef enum {
  S9_ROWS = 0,     /* array e holds, at element i, A_{i, i+e}: row i's
                      coefficient of its neighbour i+e                       */
  S9_COLUMNS = 1   /* array e holds, at element j, A_{j+e, j}: the factor by
                      which v_j enters (A v)_{j+e} -- the column storage of
                      the paper's 2D mapping; entries whose target j+e is
                      off-mesh are ignored                                  */
} s9_layout;

typedef struct {
  const void* diag;
  const void* xm;
  const void* xp;
  const void* ym;
  const void* yp;
  const void* xmym;
  const void* xpym;
  const void* xmyp;
  const void* xpyp;
  s7_dtype dtype;    /* S7_F64 or S7_F32; nx*ny elements per array (no
                        constant mode); host or device memory               */
  int layout;        /* s9_layout                                           */
} s9_coeffs;

/* Create a 9-point operator handle.  Like stencil7_create: the coefficients
 * are copied to library-owned device memory (column layout converted to
 * rows), scaled to a unit diagonal in float64 and rounded once to the
 * storage type unless opts->no_jacobi.  In opts, bx is the number of threads
 * across a row strip (each VEC cells, <= 512), zchunk the rows per thread
 * block, by must be 0 or 1, and stages / pipe_kinds are ignored.  nx, ny >= 1,
 * nx*ny < 2^40.  Errors as for stencil7_create (S7_EINVAL also for a bad
 * layout). */
int stencil9_create(stencil7_t* out, int nx, int ny, const s9_coeffs* coeffs,
                    const s7_opts* opts);

/* Release a handle and all device memory it owns (the blocks return to the
 * library's memory pool, see s7_mem_trim).  Waits for all work queued on the
 * handle's device first, including asynchronous stencil7_apply calls on the
 * caller's streams.  NULL is accepted. */
int stencil7_destroy(stencil7_t h);

/* Mesh sizes, storage type and device bytes held by a handle. */
int stencil7_info(stencil7_t h, int* nx, int* ny, int* nz, s7_dtype* storage,
                  size_t* device_bytes);

/* One SpMV with the stored operator: y = A~ x (Sec. IV-A "SpMV (3D)"; with
 * Jacobi scaling A~ = D^-1 A has a unit diagonal).  x and y hold nx*ny*nz
 * elements of `dt`, which must equal the handle's storage type; they must not
 * overlap.  Accumulation is float32 (float64 for S7_F64).  With device
 * buffers the call is asynchronous on `stream`. */
int stencil7_apply(stencil7_t h, const void* x, void* y, s7_dtype dt, void* stream);

/* True residual of the raw system, r = b - A x, with float64 accuracy (double
 * words by default, binary64 with opts.residual_f64) from the raw float32
 * coefficients when the handle keeps them (keep_true), else from the stored
 * operator times the kept diagonal.  b and x hold nx*ny*nz
 * elements of `dt` (S7_F64 or S7_F32).  r (same type) may be NULL.  Returns
 * ||r||_2 in *rnorm and ||b||_2 in *bnorm (either may be NULL); synchronous. */
int stencil7_residual(stencil7_t h, const void* b, const void* x, void* r,
                      s7_dtype dt, double* rnorm, double* bnorm, void* stream);

/* The same residual as stencil7_residual (same sweep, same results),
 * for callers that must not allocate device memory when they call: services
 * that reserve their whole device-memory budget at start-up (a pool that owns
 * the memory, where a cudaMalloc would fail or fragment it), latency-bound
 * loops that cannot afford cudaMalloc's implicit synchronisation, and
 * callers whose memory manager forbids direct cudaMalloc.  stencil7_residual
 * sets up the handle's solver workspace (several mesh-sized vectors) on
 * first use; this call allocates nothing.  Its scratch -- the per-block
 * partial sums and a small block of scalars, for at most
 * S7_NOALLOC_MAX_BLOCKS thread blocks (about 1 MiB) -- is one fixed array in
 * device memory, held by every GPU that loads the library until the process
 * exits.  The paper has no counterpart.
 *   b, x, r   device memory only (r may be NULL), nx*ny*nz elements of dt
 *             (S7_F64 or S7_F32); host buffers are rejected with S7_EINVAL.
 *   Sizes whose sweep needs more than S7_NOALLOC_MAX_BLOCKS blocks are
 *   rejected with S7_EINVAL (a larger opts.zchunk lowers the count).
 * Synchronous: the call waits on the host for its norms, so it may never be
 * made on a stream that is being captured into a graph (S7_EINVAL, the
 * capture left untouched).  The first call on each device looks up the
 * device address of the scratch array (once per device, under a lock).  The
 * address is kept for the rest of the
 * process: do not use the library across a reset of the device or of its
 * primary context (cudaDeviceReset), after which it would be stale.  All calls share the one array, which keeps
 * the last call's contents; each call clears the part that must start at
 * zero.  Calls whose work overlaps on the GPU (unordered streams or host
 * threads) race on the array: order them.  Runs on `stream`; returns after
 * the norms are on the host. */
#define S7_NOALLOC_MAX_BLOCKS 65536
int stencil7_residual_noalloc(stencil7_t h, const void* b, const void* x, void* r,
                              s7_dtype dt, double* rnorm, double* bnorm, void* stream);

/* BiCGStab (Algorithm 1) on A~ x = D^-1 b.
 *   b      nx*ny*nz elements of dt (S7_F64 or S7_F32); unchanged.
 *   x      in: start vector x0; out: the last iterate.  Same size and type.
 *   tol    stop after the first full step with ||r_k|| / ||b~|| <= tol
 *          (recurrence residual, 2-norms).  No step is taken if the start
 *          vector already satisfies it; b = 0 gives x = 0 after zero steps.
 *   maxit  at most this many steps (>= 0).
 *   iters  out (may be NULL): full steps taken.
 *   resid_hist  out (host, may be NULL): *iters+1 values, resid_hist[k] =
 *          ||r_k|| / ||b~|| (caller provides maxit+1 doubles).
 *   true_resid  out (may be NULL): ||b~ - A~ x|| / ||b~|| recomputed from x at
 *          the end with float64 accuracy (see opts.residual_f64).
 * Every step runs as three fused sweeps (p update + SpMV + (r0,s); q + SpMV +
 * (q,y),(y,y); x and r updates + (r0,r),(r,r)), each ending in a
 * deterministic grid-level combine of per-block partial sums in float64; the
 * steps are replayed from a captured CUDA graph.  Synchronous.  Returns S7_OK,
 * S7_ENOTCONV or S7_EBREAKDOWN (x and history valid in all three cases). */
int bicgstab_solve(stencil7_t h, const void* b, void* x, s7_dtype dt,
                   double tol, int maxit, int* iters, double* resid_hist,
                   double* true_resid, void* stream);

/* Mixed-precision solve with float64 iterative refinement.  The paper notes
 * that 16-bit solves plateau near a relative residual of 1e-2 (Sec. VI-B) and
 * that they may need a correction scheme such as iterative refinement.  Outer
 * loop: r = b - A x with float64 accuracy (see opts.residual_f64) on the true
 * operator (keep_true, float32 coefficients); stop when ||r|| / ||b|| <= tol; else solve A~ d = D^-1 r / s
 * with the handle's storage precision (s = ||r||_2 / sqrt(N), so the inner
 * right-hand side has unit RMS and stays inside binary16's normal range) to
 * inner_tol or inner_maxit steps, and update x += s d in float64.
 *   b, x        float64, nx*ny*nz (x in: x0, out: solution).
 *   hist        out (host, may be NULL): max_outer+1 true relative residuals.
 *   outer, inner_total  out (may be NULL): outer steps and summed inner steps.
 * Returns S7_OK when tol is met, S7_ENOTCONV after max_outer steps,
 * S7_EBREAKDOWN if an inner solve breaks down before making progress. */
int bicgstab_solve_refined(stencil7_t h, const double* b, double* x, double tol,
                           int max_outer, int inner_maxit, double inner_tol,
                           int* outer, int* inner_total, double* hist, void* stream);

/* Options of a batched solve.  Zero-initialise; NULL = all defaults. */
typedef struct {
  int threads;      /* threads per block of the batched sweeps (64..256);
                       0 = chosen by the autotuner                           */
  int zchunk;       /* z planes per block; 0 = chosen by the autotuner       */
  int check_every;  /* steps per graph launch between host checks; 0 = 16    */
  int no_autotune;  /* 1: skip the autotuner (use threads/zchunk or 128/16)  */
  int schedule;     /* 1: one persistent launch runs every step of every
                       system: the blocks that fit on the device at once
                       claim open tiles (sweep or update blocks) of any
                       system from per-system work queues, a system's next
                       phase opening when its previous one completes;
                       -1: one launch per step kernel, replayed from a
                       graph; 0: chosen by the autotuner when it runs,
                       else the persistent launch (one launch per kernel
                       where no block of it fits)                           */
  long long wait_cycles;  /* the persistent launch: longest wait of a block
                       for an open tile, in SM clock cycles; 0 = 2^31
                       (about a second).  A wait that runs out aborts the
                       launch: every unfinished system stops with
                       S7_ETIMEOUT.                                         */
  int choose_variant;  /* 1: the autotuner also times the other variant of
                       the step (Algorithm 1's three sweeps or the
                       two-reduction variant's two) and runs the faster;
                       the result then follows that variant's recurrences.
                       0: the handles' variant.                             */
} s7_batch_opts;

/* Solve nsys independent systems together (BiCGStab, Algorithm 1, on each;
 * or the two-reduction variant when every handle was created with
 * s7_opts.variant = 1).
 * One launch per kernel of a step covers every system: each system owns a
 * range of the launch's blocks and its own grid combine, scalars and stop
 * flag, so systems of different sizes and tolerances share the launches and
 * stop independently.  The steps are replayed from a captured CUDA graph.
 *   hs[j]     operator handles; all of the same storage type and device.  A
 *             handle may appear once only.
 *   b[j],x[j] right-hand side and start vector / result of system j
 *             (nx_j*ny_j*nz_j elements of dt, S7_F64 or S7_F32; host or device).
 *   tol[j], maxit[j]  per-system stopping rule (as in bicgstab_solve).
 *   iters[j], status[j], resid[j]  out (each array may be NULL): steps taken,
 *             S7_OK / S7_ENOTCONV / S7_EBREAKDOWN, final recurrence residual.
 * Unless opts fixes the block shape (threads, zchunk or no_autotune), a
 * built-in autotuner picks the policy on the first solve of each batch
 * signature (storage, systems, total cells, options) and caches it: first the
 * block shape and z chunk, timed with a batched SpMV over the batch's own
 * operators; then the fusion schedule, timed over 8 steps of the solve
 * itself from x0 with tolerance 0 (x is restored before the solve): the
 * persistent launch or one launch per step kernel, the pipelined step
 * sweeps (wide vectors, when every row is whole vectors) or the register
 * sweeps, and with opts.choose_variant the other variant.  Choices other
 * than the variant change only the summation order of the inner products.
 * Synchronous.  Returns S7_OK if every system converged, else S7_ETIMEOUT if
 * a wait of the persistent launch ran out, else S7_EBREAKDOWN if any broke
 * down, else S7_ENOTCONV. */
int bicgstab_solve_batched(int nsys, const stencil7_t* hs, const void* const* b,
                           void* const* x, s7_dtype dt, const double* tol,
                           const int* maxit, int* iters, int* status, double* resid,
                           const s7_batch_opts* opts, void* stream);

/* The policy the calling thread's last bicgstab_solve_batched ran with: block
 * threads, z chunk, schedule (1 persistent, -1 launch per kernel), pipelined
 * (1: pipelined step sweeps, 0: register sweeps) and variant (0: Algorithm 1,
 * 1: two-reduction).  Each pointer may be NULL.  S7_EINVAL if this thread has
 * run no batched solve. */
int bicgstab_batched_policy(int* threads, int* zchunk, int* schedule, int* pipelined,
                            int* variant);

/* ---- serving: continuous batching of solve requests ----
 *
 * A server owns a scheduler thread and a CUDA stream.  Submitted requests
 * are admitted first come, first served while a slot is free and the device
 * memory the request will hold fits the budget; admitted requests run
 * mixed-precision BiCGStab (storage type `storage`, float32 arithmetic) under
 * float64 iterative refinement on the true float32 operator, to their own
 * tolerance.  Every request in an inner solve shares the batched step
 * launches (bicgstab_solve_batched's kernels), so requests that arrive while
 * others run join the batch at the next tick and leave it when they meet
 * their tolerance; their Krylov state stays on the device in between.  A
 * request's arithmetic does not depend on the other requests in the batch.
 * Latencies are measured on the host's monotonic clock. */
typedef struct s7_server* s7_server_t;

typedef struct {
  size_t hbm_budget_bytes; /* device memory admitted requests may hold; 0 = 150 GiB */
  s7_dtype storage;        /* inner storage type; pass explicitly (S7_BF16 typical) */
  int max_active;          /* at most this many admitted requests; 0 = 256         */
  int steps_per_tick;      /* batched steps between host checks; 0 = 4             */
  int threads, zchunk;     /* batched tile policy; 0 = 128 threads, 16 planes      */
  double inner_tol;        /* inner relative residual; 0 = 1e-1 for S7_BF16 storage
                              (its 8 significant bits cap what one refinement
                              step gains), 1e-2 otherwise                        */
  int inner_maxit;         /* steps per inner solve; 0 = 100                       */
  int max_outer;           /* refinement steps; 0 = 60                             */
  int three_pass;          /* 1: inner steps as Algorithm 1 prints them (three
                              passes); 0: two reductions per step (s7_opts.variant
                              1), the default                                      */
  int residual_f64;        /* 1: outer residuals in binary64; 0: double words (see
                              s7_opts.residual_f64), the default                   */
} s7_server_opts;

typedef struct {
  int nx, ny, nz;
  s7_coeffs coeffs;        /* raw operator (host or device)                       */
  const void* b;           /* right-hand side, nx*ny*nz elements of dt            */
  void* x;                 /* out: solution (x0 = 0), nx*ny*nz elements of dt     */
  s7_dtype dt;             /* S7_F64 or S7_F32                                    */
  double tol;              /* ||b - A x|| / ||b|| to reach (float64, true operator) */
} s7_request;

typedef struct {
  int status;              /* S7_OK, S7_ENOTCONV, S7_EBREAKDOWN, S7_ECANCELED, ... */
  int outer;               /* refinement steps                                     */
  int inner_iters;         /* inner BiCGStab steps, summed                         */
  double resid;            /* final ||b - A x|| / ||b||                            */
  double t_arrive, t_admit, t_done;  /* host monotonic seconds                     */
} s7_result;

typedef struct {
  long long completed, failed, queued, active;
  size_t mem_used, mem_peak;  /* admitted bytes now / at most (model of request_bytes) */
  double cell_iters;       /* sum over requests of cells x inner steps             */
  double busy_s;           /* scheduler time spent with work on the device         */
} s7_server_stats;

/* Create a server on the current device (opts may be NULL: BF16 storage,
 * defaults above). */
int s7_server_create(s7_server_t* out, const s7_server_opts* opts);
/* Queue a request; *id identifies it.  The buffers behind req (coefficients,
 * b, x) must stay valid until the request has finished.  S7_ENOMEM if the
 * request alone exceeds the memory budget. */
int s7_server_submit(s7_server_t s, const s7_request* req, uint64_t* id);
/* S7_EAGAIN while the request runs; S7_OK with *out once it has finished
 * (out->status tells how). */
int s7_server_poll(s7_server_t s, uint64_t id, s7_result* out);
/* Block until the request finishes or timeout_s passes (negative: no limit);
 * S7_ETIMEOUT on timeout. */
int s7_server_wait(s7_server_t s, uint64_t id, s7_result* out, double timeout_s);
/* Forget a finished request. */
int s7_server_release(s7_server_t s, uint64_t id);
int s7_server_get_stats(s7_server_t s, s7_server_stats* out);
/* Stop the scheduler (queued and running requests end with S7_ECANCELED)
 * and free everything. */
int s7_server_destroy(s7_server_t s);

/* Per-kernel timing for benchmarks.  enable = 1 turns timing on for handle
 * h: solves then launch each kernel directly (not from a captured graph)
 * with a CUDA event pair around it on the handle's stream; enable = 0 turns
 * it off.  Every call first copies the totals accumulated since the previous
 * call into ms[k] (milliseconds) and launches[k] (either may be NULL;
 * S7_PROF_NKINDS entries each) and resets them.  Kinds, in order: the fused
 * p-update + SpMV + (r0,s) sweep; the fused q + SpMV + (q,y),(y,y) sweep;
 * the x/r update with (r0,r),(r,r); the start-residual sweep; the
 * true-residual sweep; everything else (casts, refinement kernels). */
#define S7_PROF_NKINDS 6
int stencil7_profile(stencil7_t h, int enable, double* ms, long long* launches);

/* ---- device memory ----
 * Handles take their device memory (operator arrays, Krylov vectors, staging
 * buffers) from one stream-ordered CUDA memory pool per device that the
 * library owns.  Blocks a destroyed handle gave back stay reserved in the
 * pool, up to the cache limit, and a later handle reuses them without mapping
 * memory again.  If the pool cannot grow, it first returns its cached blocks
 * to the device and retries.  Other allocators (the caller's, PyTorch's)
 * do not see the cached bytes as free: trim the pool or lower the limit when
 * they need the memory. */

/* Bytes the pool of `device` holds reserved, and of those the bytes in use
 * by live handles (either pointer may be NULL).  S7_ECUDA for a bad device. */
int s7_mem_stats(int device, size_t* reserved, size_t* used);

/* Synchronise `device` and return the cached blocks of its pool to it,
 * keeping at most `keep` reserved bytes (blocks in use stay).  The calling
 * thread's current device is left as it was.  S7_ECUDA for a bad device. */
int s7_mem_trim(int device, size_t keep);

/* Most bytes each pool keeps reserved after the synchronisation that
 * follows a release (default 64 GiB; 0 returns every free block).  Applies
 * to all devices' pools, present and future.  Always S7_OK. */
int s7_mem_set_cache(size_t bytes);

/* ---- thread-local error text ---- */
const char* s7_last_error(void);

/* Library version string. */
const char* s7_version(void);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL7_H */

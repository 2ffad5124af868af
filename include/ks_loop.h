/*
 * ks_loop.h - C ABI of the GB300 (sm_103a) tau-descent library for Kuramoto-Sivashinsky
 * loops, after Azimi, Ashtari & Schneider, "Adjoint-based variational method for
 * constructing periodic orbits of high-dimensional chaotic systems" (arXiv:2007.06427).
 *
 * A loop is l = [u(x, s); T]: a field on [0, L) x [0, 1), periodic in both directions, and a
 * period T > 0 (Sec. 2, Eq. loop_def).  Its residual is r = -(1/T) u_s - u u_x - u_xx - u_xxxx
 * (Sec. 4.1, Eq. KS_R), its cost J = int_0^1 int_0^L r^2 dx ds (Sec. 2, Eq. cost_function), and
 * the loop flow is du/dtau = -L^dag_1, dT/dtau = -L^dag_2 with
 * L^dag_1 = (1/T) r_s + u r_x - r_xx - r_xxxx and L^dag_2 = int int (1/T^2) u_s r dx ds
 * (Sec. 4.1, Eq. KS_L_dagger and Eq. KS_G; App. B).  Fields are discretised with Nx x Ns Fourier
 * modes on the uniform grid (m L / Nx, n / Ns) (Sec. 4.2, Eq. 2D_Fourier), derivatives are
 * spectral, products are formed on the grid, and every product is truncated to the 2/3 band
 * |j| <= Nx/3, |k| <= Ns/3 (Sec. 4.2).  One tau-step is IMEX Euler for u (the diagonal linear
 * symbol Lambda_jk implicit) and explicit Euler for T (Sec. 4.2); an explicit Euler scheme is
 * also provided.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every compute call runs on the GPU; there is no CPU path.  A call made without a usable
 *    CUDA device returns KS_ERR_CUDA.
 *  - A batch holds `batch` independent loops sharing L and Nx; loop b has its own Ns_b.
 *  - Grid fields (u, r, G) are ragged-packed: loop b occupies Ns_b * Nx consecutive values,
 *    laid out [n][m] with the x-index m fastest; loops follow one another in batch order.
 *    Their element type is double for KS_FP64 and KS_MIXED handles and float for KS_FP32.
 *  - Every input field is first projected onto the 2/3 band; all results are those of the
 *    projected loop.
 *  - T and the per-loop outputs are double arrays of length `batch` (steps: long long,
 *    status: int).
 *  - Pointers may be device pointers or ordinary host pointers; the library tells them apart
 *    with cudaPointerGetAttributes and stages host buffers through its own device memory
 *    (synchronising the stream before it returns).  The caller owns every buffer it passes.
 *  - `stream` is a cudaStream_t (NULL for the legacy default stream).  Calls with device
 *    buffers only are stream ordered; ks_descend always synchronises `stream` (it reads the
 *    convergence state back between chunks).
 *  - Return value: KS_OK (0) or a negative KS_ERR_* code; ks_last_error() gives a message
 *    for the last failing call on the calling thread.  A handle is not thread safe: calls on
 *    one handle must not overlap.
 */
#ifndef KS_LOOP_H
#define KS_LOOP_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(KS_BUILD_SO) && defined(__GNUC__)
#define KS_API __attribute__((visibility("default")))
#else
#define KS_API
#endif

typedef struct ks_loop* ks_loop_t;

/* arithmetic mode of a handle */
enum {
    KS_FP64 = 0,   /* every step in double */
    KS_FP32 = 1,   /* every step in float; reductions finished in double; T in double */
    KS_MIXED = 2   /* ks_descend: float steps while sqrt(J), evaluated in double at every
                      read-back, exceeds switch_tol and keeps falling; then double steps to the
                      end, all in double (the adjoint half of each in float when
                      "finish_f32_adjoint" is 1).
                      "Keeps falling" is decided by a probe (knob "switch_probe") once the
                      float phase's rate bends, with the stall window as a fallback.
                      A loop whose float rounding alone more than doubles sqrt(J) (one that
                      starts below the float floor) takes double steps from the start.
                      Other calls compute in double */
};

/* tau-integration scheme (Sec. 4.2) */
enum {
    KS_EXPLICIT = 0, /* u <- u - dtau * L^dag_1 r */
    KS_IMEX = 1      /* (u' - u)/dtau = Lambda u' + (flow - Lambda u): the paper's scheme */
};

/* return codes */
enum {
    KS_OK = 0,
    KS_ERR_ARG = -1,     /* bad argument: null pointer, size out of range, L <= 0, dtau <= 0 */
    KS_ERR_CUDA = -2,    /* a CUDA runtime call failed, or no device */
    KS_ERR_OOM = -3,     /* device allocation failed */
    KS_ERR_TIMEOUT = -4, /* a bounded in-kernel wait gave up (a grid barrier of the persistent
                            kernel or an exchange of the cluster kernel, about a second each) */
    KS_ERR_STATE = -5    /* call needs a resident state that was never set */
};

/* per-loop outcome of a descent (status array) */
enum {
    KS_RUNNING = 0,   /* still descending */
    KS_CONVERGED = 1, /* sqrt(J) < tol reached */
    KS_STEP_CAP = 2,  /* max_steps taken without convergence */
    KS_STALLED = 3,   /* double descent stopped making progress: a local minimum with J > 0 */
    KS_DIVERGED = 4   /* J not finite or T <= 0 */
};

typedef struct {
    double L;            /* domain length, > 0 */
    int nx;              /* Nx: power of two, 8 <= Nx <= 1024 */
    int batch;           /* number of loops, >= 1 */
    const int* ns;       /* host array [batch]: Ns_b, power of two, 8 <= Ns_b <= 1024 */
    int mode;            /* KS_FP64, KS_FP32 or KS_MIXED */
    int scheme;          /* KS_EXPLICIT or KS_IMEX */
    double dtau;         /* fictitious-time step, > 0 (the paper uses 0.15 with IMEX) */
    double tol;          /* default sqrt(J) tolerance of ks_descend (used when its tol < 0) */
    double switch_tol;   /* KS_MIXED: switch to double once sqrt(J) <= switch_tol */
    long long max_steps; /* default step cap of ks_descend (used when its max_steps < 0) */
    int chunk;           /* tau-steps between convergence read-backs in ks_descend (> 0) */
    int autotune;        /* 0: default launch shapes; 1: ks_autotune at create */
} ks_config;

/* Create a handle: validates cfg, allocates the device workspace for the batch (band states,
 * transform scratch, per-loop scalars) and uploads the twiddle tables.  The current CUDA
 * device is used.  On success *out owns the workspace until ks_destroy. */
KS_API int ks_loop_create(const ks_config* cfg, ks_loop_t* out);

/* Release a handle and all of its device memory (NULL is accepted). */
KS_API int ks_destroy(ks_loop_t h);

/* Residual of each loop (Eq. KS_R) at [P u; T].
 *   u  : in,  grid field (packed, mode element type)
 *   T  : in,  double[batch]
 *   r  : out, grid field, nullable
 *   J  : out, double[batch]: J = int int r^2 (Eq. cost_function), nullable
 * Does not touch the resident descent state. */
KS_API int ks_residual(ks_loop_t h, const void* u, const double* T, void* r, double* J, void* stream);

/* Adjoint gradient at [P u; T] (Eq. KS_L_dagger):
 *   G    : out, grid field G = +L^dag_1 r (the ascent direction of the paper's flow)
 *   dJdT : out, double[batch]: dJ/dT = 2 L^dag_2, nullable
 * The exact gradient of J with respect to the grid values is (2 L / (Nx Ns_b)) G.
 * Does not touch the resident descent state. */
KS_API int ks_adjoint_grad(ks_loop_t h, const void* u, const double* T, void* G, double* dJdT,
                    void* stream);

/* Tau-descent of every loop from [P u; T] (Eq. KS_G integrated as in Sec. 4.2).
 *   u, T     : in/out: initial loop, overwritten by the final one
 *   max_steps: step cap per loop (< 0: the handle's default)
 *   tol      : stop a loop when sqrt(J) < tol at the start of a step (< 0: the handle's)
 *   steps    : out, long long[batch], steps taken (nullable)
 *   sqrtJ    : out, double[batch], sqrt(J) of the final loop (nullable)
 *   status   : out, int[batch], KS_CONVERGED / KS_STEP_CAP / KS_STALLED / KS_DIVERGED
 *              (nullable)
 * Loops are frozen individually when they converge or diverge; the call returns when every
 * loop is frozen or has taken max_steps steps.  The final state also stays resident.  The
 * knobs "extrapolate" (App. C), "symmetry" (centre-symmetric subspace), "stall_window" and the
 * mixed-precision switch act here (see ks_set_option). */
KS_API int ks_descend(ks_loop_t h, void* u, double* T, long long max_steps, double tol,
               long long* steps, double* sqrtJ, int* status, void* stream);

/* Convergence history of loop b recorded by the last ks_descend at each read-back (every
 * `chunk` steps): up to cap entries of the step count, sqrt(J) of the last evaluated loop and
 * the precision it was descending in (0 double, 1 float).  Outputs nullable; returns the
 * number of entries recorded (may exceed cap) or a negative KS_ERR_* code.  sqrt(J) against
 * tau is the convergence curve of the paper's Fig. 2. */
KS_API int ks_get_history(ks_loop_t h, int b, long long* steps, double* sqrtJ, int* prec, int cap);

/* Band-level access to the resident state, for bitwise checkpoints.  The band of loop b is
 * (Kx+1) x (2 Ks_b + 1) complex coefficients u_hat_jk of Eq. 2D_Fourier, j = 0..Kx,
 * k = -Ks_b..Ks_b, stored [j][k + Ks_b] as interleaved (re, im) doubles; loops follow one
 * another in batch order.  ks_band_size gives the number of complex values (or -1).
 * ks_get_band: band (double, 2 * size), T, the precision each loop descends in (0 double,
 * 1 float) and the step counters (outputs nullable except band).  ks_set_band: installs a
 * band, T, optional precisions (NULL: the mode's start) and optional step counters; every loop
 * restarts as running.  Float loops are stored widened to double and narrowed back exactly,
 * so get followed by set continues the descent bit for bit. */
KS_API long long ks_band_size(ks_loop_t h);
KS_API int ks_get_band(ks_loop_t h, double* band, double* T, int* prec, long long* steps,
                       void* stream);
KS_API int ks_set_band(ks_loop_t h, const double* band, const double* T, const int* prec,
                       const long long* steps, void* stream);

/* Resident state: load [P u; T] as the handle's descent state (status reset to running,
 * step counters to zero). */
KS_API int ks_set_state(ks_loop_t h, const void* u, const double* T, void* stream);

/* Advance the resident state by nsteps tau-steps with no read-back (loops that converge
 * below tol or diverge freeze on the device).  tol < 0: the handle's tol. */
KS_API int ks_step(ks_loop_t h, long long nsteps, double tol, void* stream);

/* Copy the resident state out: u (grid, nullable), T (nullable), and the per-loop step
 * counters, sqrt(J) of the last evaluated state and status (each nullable). */
KS_API int ks_get_state(ks_loop_t h, void* u, double* T, long long* steps, double* sqrtJ, int* status,
                 void* stream);

/* Per-kernel timing: while enabled, every kernel the handle launches is bracketed by two CUDA
 * events on its launch stream and the elapsed time is accumulated per kernel kind (a name such
 * as "cols_resid_f64").  Launches are always counted. */
KS_API int ks_profile(ks_loop_t h, int enable);

/* Read the profile: for up to n kinds, names (n x 48 chars, NUL terminated), accumulated
 * milliseconds and launch counts; total_launches gets every launch since the last reset (all
 * outputs nullable).  Synchronises on the recorded events.  reset != 0 clears the counters.
 * Returns the number of kinds (>= 0) or a negative KS_ERR_* code. */
KS_API int ks_profile_read(ks_loop_t h, int n, char* names, double* ms, long long* launches,
                           long long* total_launches, int reset);

/* Tuning knobs of a handle (KS_ERR_ARG for an unknown key or a bad value):
 *   "path"           launch shape of ks_step / descent chunks, for both precisions: 0
 *                    cluster-resident kernel (one thread-block cluster per loop, state in shared
 *                    memory for the whole chunk, falls back to 1 where the loop does not fit);
 *                    1 one cooperative launch per chunk with grid-wide barriers between the four
 *                    phases of a step; 2 four launches per tau-step (replayed as CUDA graphs, see
 *                    "graph").  All three give bit-identical results.
 *   "path_f64", "path_f32"  the same for the double or the float steps alone (the loops of a
 *                    KS_MIXED batch in each precision are stepped by their own precision's form).
 *                    Default at create, with P = Nx * max Ns (the faster form in measurements on
 *                    GB300): 2 for ragged batches (unequal Ns) of 64 or more loops; double: 2
 *                    when P >= 16384, or P >= 8192 in batches of 8 or more, or when the cluster
 *                    plan has 1 or 2 CTAs per loop on P >= 4096 in a batch; float: 2 when
 *                    P >= 32768, or P >= 16384 in batches of 64 or more; else 0.  ks_autotune
 *                    replaces the bulk precision's form (float for KS_MIXED) by timing.
 *   "persistent"     1: path 1, 0: path 2 (older spelling of "path")
 *   "row_threads", "col_threads"  path 2: threads per block of the row and column items, 128
 *                    or 256 (results are bit-identical: a column's partials of J and L^dag_2
 *                    keep 128 accumulators at either size).  Default at create: 256-thread rows
 *                    for Nx >= 256; 256-thread columns when the batch has fewer than 152 column
 *                    items (loops x retained x-modes, one per SM of a GB300) and max Ns >= 256;
 *                    else 128.
 *   "cluster"        0 (default): cluster size chosen per precision; 1..16: force this size
 *                    (KS_ERR_ARG when no plan of that size fits the batch)
 *   "cluster_exchange" 1 (default): the cluster kernel's DSMEM exchanges are asynchronous
 *                    stores counted on an mbarrier of the receiving CTA, which starts its next
 *                    phase once its bytes have landed (in plans with room for a second column
 *                    buffer that keep the CTAs per SM the batch uses); 0: the phases are
 *                    separated by cluster barriers.  Results are bit-identical either way.
 *   "cluster_min_blocks" 0 (default): the cluster kernel variant is chosen by occupancy (see
 *                    "cluster_min_blocks_f64"); 1 or 2: force it.  Results are bit-identical.
 *   "symmetry"       1: restrict the descent to loops invariant under Xi: (x, s) -> (-x, s),
 *                    u -> -u (the centre-symmetric subspace, Sec. 4.1).  Every later analysis of a
 *                    grid field (ks_residual, ks_adjoint_grad, ks_set_state, ks_descend) projects
 *                    it onto that subspace, ks_adjoint_grad returns the projected G, and every
 *                    update is taken along the projected G, so the band state stays exactly
 *                    invariant (u_hat[j][-k] = -conj(u_hat[j][k]) bit for bit, zero j = 0
 *                    column).  0 (default): no projection; the flow still preserves the symmetry
 *                    of an invariant loop up to rounding.  A state already resident keeps its
 *                    non-invariant part (set the state again after changing the knob);
 *                    ks_set_band stores the band as given.
 *   "extrapolate"    1: ks_descend accelerates each loop by the extrapolation of App. C: once
 *                    sqrt(J) (evaluated in double at the read-backs) is below the start
 *                    threshold, every time it has halved since the loop's anchor state, the loop
 *                    is moved to l + (l - l_anchor) rho / (1 - rho), rho = sqrt(J) / sqrt(J_anchor),
 *                    on its band and T; the move is kept only if it lowers sqrt(J).  Read-backs
 *                    happen every "chunk" steps, so the chunk sets how finely the halvings are
 *                    caught.  0 (default): plain descent.  ks_get_option "extrapolations" and
 *                    "extrapolations_rejected" count the moves kept and dropped by the last
 *                    ks_descend.
 *   "extrapolate_start_ppm"  the start threshold on sqrt(J) in parts per million, 1 .. 1e9
 *                    (default 1000, i.e. 1e-3, the value of the example of App. C)
 *   "extrapolate_drop_ppm"   the fraction of the anchor's sqrt(J) at which the next move is
 *                    made, in parts per million, 1 .. 999999 (default 500000: "has halved")
 *   "stall_window"   tau-steps over which ks_descend measures progress (default 40000)
 *   "stall_drop_ppm" a loop whose sqrt(J) fell by less than this many parts per million over
 *                    a window is stalled (default 1000): the float phase of a mixed descent
 *                    then switches to double, a double descent stops with KS_STALLED
 *   "chunk"          tau-steps between read-backs in ks_descend
 *   "graph"          path 2: 1 (default): runs of up to 16 tau-steps (an even number) are
 *                    captured once as a CUDA graph of their launches and replayed on the
 *                    caller's stream (while loops are live in both precisions, the float and
 *                    double chains of a step are parallel branches of the graph); an odd last
 *                    step is launched directly.  Up to 8 graphs are kept per handle, keyed by
 *                    the live precisions, tol, the switch threshold, the step parity, the
 *                    symmetry knob and the run length.  Results are bit-identical to 0 (every
 *                    launch separately).  Off while ks_profile is on.
 *   "test_barrier_timeout" test hook: 1 makes every grid barrier of the path-1 kernel wait
 *                    for one arrival that never comes, so each wait runs out (about a second)
 *                    and the next read-back returns KS_ERR_TIMEOUT; 0 (default) restores it
 *   "switch_probe"   KS_MIXED handles: 1 (default): the float phase of each loop is watched
 *                    in windows of stall_window / 4 steps; when its rate (decades of sqrt(J),
 *                    evaluated in double, per step) falls below an eighth of the best rate over
 *                    windows below sqrt(J) = 1e-2, a copy of the loop takes "switch_probe_steps"
 *                    double steps (a polish).  If the polish removes a fifth or more of sqrt(J)
 *                    beyond what its steps give at the best rate, the float value is mostly
 *                    rounding noise and the float steps keep converging beneath it: the loop
 *                    stays in float until the stall window ends the phase.  If it removes less
 *                    and descends at least four times faster than the float phase now does, the
 *                    float arithmetic holds the descent back: the loop switches to double at once
 *                    and continues from the polished copy (its step counter includes the
 *                    polish's steps).  Otherwise the bend was the loop's own dynamics; it stays
 *                    in float and may be probed again after stall_window steps.  0: switch only
 *                    on switch_tol or the stall window.
 *   "switch_probe_steps"  double steps of a probe, 1 .. 1e6 (default 1000)
 *   "finish_f32_adjoint"  KS_MIXED handles: 0 (default): the finishing steps run all in
 *                    double, as the final convergence steps of the method require; every launch
 *                    form then gives bit-identical mixed descents.  1: the finishing steps keep
 *                    the state, the residual, J, dJ/dT and the update in double and form only
 *                    the descent direction G (the adjoint half of a step) in float, in the
 *                    cluster-resident form (the other forms finish all in double): faster, and
 *                    its direction carries float rounding. */
KS_API int ks_set_option(ks_loop_t h, const char* key, long long value);

/* Read a knob or a derived launch parameter: "path" (the bulk precision's: float for KS_FP32
 * and KS_MIXED handles), "path_f64", "path_f32", "finish_f32_adjoint", "switch_probe",
 * "switch_probe_steps", "cluster_f64",
 * "cluster_f32", "cluster_mixed_finish" (cluster
 * size in use, 0 if the cluster path cannot hold the batch),
 * "cluster_exchange", "cluster_exchange_f64", "cluster_exchange_f32" (whether that plan
 * exchanges through mbarriers), "cluster_grid_f64", "cluster_grid_f32" (CTAs of that cluster
 * launch: cluster size x resident clusters, at most the batch), "cluster_min_blocks_f64",
 * "cluster_min_blocks_f32" (the kernel variant's resident blocks per SM bound: 1, no register
 * cap; 2, at most 128 registers, chosen where it keeps more clusters resident),
 * "cluster_block_f64", "cluster_block_f32", "cluster_block_mixed_finish" (threads per CTA of
 * that cluster kernel:
 * "cluster_threads" work threads, plus one warp for the step scalars at the default width of
 * 128 where the plan allows it; 0 if no plan), "cluster_smem_f64",
 * "cluster_smem_f32" (bytes per CTA), "rows_per_tile", "stall_window", "stall_drop_ppm",
 * "chunk", "symmetry", "graph", "graph_replays" (graphs replayed since create),
 * "row_threads", "col_threads",
 * "extrapolate", "extrapolate_start_ppm", "extrapolate_drop_ppm", "extrapolations",
 * "extrapolations_rejected". */
KS_API int ks_get_option(ks_loop_t h, const char* key, long long* value);

/* Residual of ONE double-precision loop without allocating any device memory.
 *
 * For callers that cannot call cudaMalloc when they need a residual: code that runs inside a
 * memory pool or arena that already owns the device memory, plugins of applications that
 * forbid allocation after start-up, and real-time loops where an allocation (an implicit
 * synchronisation, and a call that can fail) is not acceptable.  The paper has no counterpart:
 * this is a deployment variant of ks_residual.
 *
 * Returns the same r and J as ks_residual for a handle with batch 1 and mode KS_FP64, given
 * the same u and T.  No handle is needed.
 *   L     : domain length, > 0
 *   nx, ns: grid size, powers of two with 8 <= nx <= 256 and 8 <= ns <= 256 (larger sizes are
 *           rejected with KS_ERR_ARG)
 *   u     : in,  device pointer on the current device, ns x nx doubles, layout [n][m]
 *   T     : the period (by value), finite and > 0 (else KS_ERR_ARG)
 *   r     : out, device pointer on the current device, ns x nx doubles, nullable
 *   J     : out, device pointer on the current device, one double
 *   stream: cudaStream_t; the call is stream ordered
 * Host pointers, and device pointers of another device, are rejected with KS_ERR_ARG.
 *
 * All intermediates live in one file-scope device array of about 1.4 MB (at most 2 MB) that
 * every GPU loading the library holds until the process exits.  The first call on a device
 * (with that device current), and the first call after that device's context was destroyed and
 * created again (e.g. by cudaDeviceReset), looks up the array's device address and uploads the
 * twiddle table there with a synchronous copy; make that first call before any stream capture.
 * Every call shares the array and overwrites what the previous call left in it, so calls that
 * overlap on the GPU (on different streams, or from several threads) race: serialise them.
 * Errors are reported through ks_last_error(). */
KS_API int ks_residual_noalloc(double L, int nx, int ns, const double* u, double T, double* r,
                               double* J, void* stream);

/* Time the launch candidates of this batch (cluster-resident kernel for each cluster size that
 * fits, with 128 and 256 threads per CTA; grid-persistent kernel; four launches per step) on a
 * synthetic band-limited state and keep the fastest for the precision the descent spends its
 * bulk in.  If the environment variable KS_AUTOTUNE_CACHE names a file, choices are read from
 * and appended to it, keyed by Nx, the Ns list, the batch size, the mode and the scheme; a
 * line naming a shape the tuner does not try (e.g. another thread count) is ignored.
 * Clears the resident state (call ks_set_state afterwards).  All candidates give the same
 * results bit for bit; only the time differs. */
KS_API int ks_autotune(ks_loop_t h);

/* Measured arithmetic peak of the current device for the roofline of the hot path, which is
 * bound by the FP64 pipe (double steps) or the FP32 pipe (float steps), not by HBM.  The paper
 * has no counterpart: this is a measurement utility.  Launches a grid of (SMs x resident blocks
 * of 256 threads), each thread running iters rounds of 8 independent fused multiply-add chains
 * in the given precision (KS_FP64 or KS_FP32) with no memory traffic, once to warm up and once
 * timed with CUDA events on `stream`; *tflops = 2 x FMAs / time in TFLOP/s.  Synchronises
 * `stream`.  KS_ERR_ARG for another precision, iters < 1 or a null tflops. */
KS_API int ks_probe_peak(int precision, int iters, double* tflops, void* stream);

/* Time integration of the KSE u_t = -u u_x - u_xx - u_xxxx on [0, L), periodic, the chaotic run
 * from which the paper takes its initial loops (Sec. 4.3).  Fourier pseudo-spectral in x with Nx
 * points and the product -(u^2/2)_x truncated to |j| <= Nx/3 (the 2/3 rule of Sec. 4.2; the
 * Nyquist mode is zero), fourth-order exponential time differencing in t (ETDRK4 of Cox &
 * Matthews, J. Comput. Phys. 176 (2002); the paper names no integrator).  `batch` independent
 * trajectories share L, Nx and dt.
 *   u0      : in,  [batch][nx] doubles, the initial grid fields (projected onto |j| <= Nx/3)
 *   nsteps  : steps of size dt (>= 0); save_every (>= 1): the state is saved at steps
 *             0, save_every, 2 save_every, ..., so nsave = nsteps / save_every + 1 instants
 *   symmetric: nonzero keeps the run in the centre-symmetric subspace u(-x) = -u(x) (Sec. 4.4):
 *             the real parts of the coefficients are zeroed initially and after every step
 *   u_saved : out, [batch][nsave][nx] doubles, the grid fields at the saved instants, nullable
 *   norms   : out, [batch][nsave] doubles, ||u||(t) = (int_0^L u^2 dx)^(1/2) at the saved
 *             instants (Sec. 4.3), nullable
 *   u_end   : out, [batch][nx] doubles, the field after the last step, nullable
 * Pointers follow the conventions above (device or host).  Errors: KS_ERR_ARG for L or dt not
 * finite and > 0, nx not a power of two in [8, 1024], batch < 1, nsteps < 0, save_every < 1 or a
 * null u0; KS_ERR_OOM when a host buffer cannot be staged.  The run is one launch on `stream`
 * (one block per two to eight trajectories); with device buffers only it is stream ordered. */
KS_API int ks_dns(double L, int nx, int batch, double dt, long long nsteps, int save_every,
                  int symmetric, const double* u0, double* u_saved, double* norms, double* u_end,
                  void* stream);

/* Initial loops from segments of one saved trajectory (Sec. 4.3): loop l is the field at the Ns_l
 * instants t_a + T_l n / Ns_l (n = 0..Ns_l - 1), t_a the time of saved sample a_idx[l], by linear
 * interpolation in time between saved samples.  The temporal low-pass of Sec. 4.3 is the
 * projection onto the 2/3 band that every loop input receives (ks_set_state, ks_descend).
 *   nx, nsave: the trajectory's [nsave][nx] layout in `us` (device or host doubles)
 *   dts      : time between saved samples, > 0
 *   a_idx, T, ns: HOST arrays [nloops]: first sample, period (> 0) and Ns (>= 1) of each loop
 *             (device pointers there are rejected with KS_ERR_ARG)
 *   out      : out, ragged-packed loops [sum_l Ns_l * nx] doubles, layout [n][m] (device or host)
 * KS_ERR_ARG for a null pointer, nsave < 2, dts not finite and > 0, nloops < 0, or a segment
 * whose last instant needs a sample past the last saved one (the interpolation reads the samples
 * on both sides of every instant). */
KS_API int ks_dns_segments(int nx, long long nsave, double dts, const double* us, int nloops,
                           const int* a_idx, const double* T, const int* ns, double* out,
                           void* stream);

/* Message for the last non-zero return on the calling thread ("" if none). */
KS_API const char* ks_last_error(void);

/* Library version string. */
KS_API const char* ks_version(void);

/* sizeof(ks_config) as compiled into the library (lets bindings check their struct layout). */
KS_API unsigned long long ks_config_sizeof(void);

#ifdef __cplusplus
}
#endif

#endif /* KS_LOOP_H */

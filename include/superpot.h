/*
 * superpot.h -- C ABI of the GB300 (sm_103a) super-potential GS/FFT solver for the
 * free-space Poisson equation  -Laplacian(u) = rho  in R^3  (Exl & Schaffer,
 * arXiv:2506.04489).
 *
 * The solver computes, on a uniform n0 x n1 x n2 grid,
 *     u = crop( IDFT3( M .* DFT3( pad(rho) ) ) )                       (Alg. 2)
 * with padding factor 2 per axis (Sec. 2 and Alg. 1) and the real multiplier
 *     M_k = -|kappa_k|^2 Vhat_k / Ntilde,   Ntilde = 8 n0 n1 n2,      (eq. convtheorem)
 *     Vhat_k = sum_s w_s (H1 G2 G3 + G1 H2 G3 + G1 G2 H3)              (eq. Gten_sep)
 * built from the Gaussian-sum (GS) approximation 1/(8 pi r) ~ sum_s w_s exp(-a_s r^2)
 * on (eps, delta] (eq. sin_1_x) and the one-dimensional integrals
 *     G_p,s(k) = 2 int_0^{L_p} exp(-a_s y^2) cos(kappa y) dy,
 *     H_p,s(k) = 2 int_0^{L_p} y^2 exp(-a_s y^2) cos(kappa y) dy,     kappa = pi k / L_p.
 *
 * Geometry (the reading of Sec. 3 that reproduces the paper's tables): grid points
 * x_j = lo + j h, j = 0..n-1, h = (hi - lo)/(n - 1); the padded period is 2 n h and the
 * kernel window is [-L, L] with L = n h per axis.
 *
 * Conventions shared by every entry point:
 *   - Arrays are C order [x][y][z] (z fastest), n0 x n1 x n2 elements.
 *   - Device pointers are CUDA device (or managed) memory of the current device.
 *   - A plan belongs to the device that was current at sp_plan_create; every call on it
 *     except sp_plan_destroy must be made with that device current (else
 *     SP_ERR_INVALID, naming both devices).
 *   - Streams are cudaStream_t passed as void*; NULL means the legacy default stream.
 *     All work is stream-ordered; no entry point below synchronises the host unless
 *     it says so.
 *   - Every call returns sp_status; nothing throws across the ABI.  On failure
 *     sp_last_error() returns a message for the calling host thread.
 *   - A plan is not thread-safe: one host thread at a time may use it, and solves
 *     issued on different streams of one plan share its workspace and therefore must
 *     not overlap on the GPU.
 */
#ifndef SUPERPOT_H
#define SUPERPOT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SP_FP64 = 0,  /* rho, u float64; FFT passes and multiplier in FP64              */
    SP_FP32 = 1,  /* rho, u float32; FFT passes in FP32, multiplier rounded to FP32  */
    SP_MIXED = 2, /* rho, u float64; FFT passes in FP32 (FP32 accumulation)          */
    SP_DF32 = 3   /* rho, u float64; FFT passes and multiplier in double-float: pairs
                     of FP32 values hi + lo (about 48 significant bits) on the FP32
                     pipes; the same lengths as the other precisions                   */
} sp_precision;

typedef enum {
    SP_OK = 0,
    SP_ERR_INVALID = 1,          /* bad argument (null pointer, bad box, ...)          */
    SP_ERR_UNSUPPORTED_SIZE = 2, /* n < 2 or 2n > 2048, or a feature the grid lacks     */
    SP_ERR_OOM = 3,              /* device allocation failed                            */
    SP_ERR_CUDA = 4,             /* a CUDA runtime call or kernel launch failed         */
    SP_ERR_TIMEOUT = 5,          /* a bounded device wait gave up                       */
    SP_ERR_NOT_READY = 6         /* sp_kernel_precompute has not been run on the plan   */
} sp_status;

typedef struct sp_plan_s* sp_plan;
typedef void* sp_stream; /* a cudaStream_t */

/*
 * sp_plan_create -- validate the problem and allocate the plan's device memory
 * (Alg. 1 inputs).
 *   out        : receives the plan handle (set to NULL on failure).
 *   n[3]       : grid points per axis, each >= 2 with 2n <= 2048 (2n: the padded FFT
 *                lengths; products of 2s, 3s, 5s and 7s are transformed by radix
 *                2/3/4/5/7/8 stages, any other length by Bluestein's algorithm, a
 *                circular convolution through power-of-two transforms of length
 *                M >= 4n - 1).
 *   box_lo/hi  : box faces per axis, hi > lo (the grid spans them inclusively).
 *   padding    : must be 2 (the paper's padding factor, Alg. 1).
 *   gs_w, gs_a : host arrays of gs_terms GS weights/exponents (eq. sin_1_x), copied;
 *                or NULL, NULL, 0 to have sp_kernel_precompute generate them on the
 *                GPU by sinc quadrature on (eps, delta] with delta the window
 *                diagonal sqrt(L0^2 + L1^2 + L2^2).
 *   eps        : GS cutoff (the paper's default is 1e-4); ignored with an explicit table.
 *   prec       : sp_precision of rho/u and of the solve passes.
 *   max_batch  : largest batch sp_solve_batched will be given (>= 1); the workspace
 *                is sized for it.
 * Device memory: multiplier octant (n0+1)(n1+1)(n2+1) FP64 (+ an FP32 or double-float
 * copy for those passes), twiddles, and a workspace of n0 * 2n1 * (n2+1) complex values
 * per batch element (see sp_plan_workspace_bytes).  Allocated on the current device,
 * stream-ordered from its default memory pool (cudaMallocAsync on a stream of the plan's
 * own, complete when this call returns); sp_plan_create_ex takes a caller's allocator.
 * Every precision takes the same lengths: register-resident passes where every padded
 * length has a compiled plan (2n in {64, 128, 192, 256, 384, 512, 1024}), shared-memory
 * passes (radix 2..8, 3, 5 and 7 stages, or Bluestein's algorithm) elsewhere.  Bluestein
 * axes also hold a table of 2n + 3M complex values built on the host and copied here.
 */
sp_status sp_plan_create(sp_plan* out, const int n[3], const double box_lo[3],
                         const double box_hi[3], int padding, const double* gs_w,
                         const double* gs_a, int gs_terms, double eps, sp_precision prec,
                         int max_batch);

/*
 * sp_allocator -- where a plan's device memory comes from (the multiplier, twiddles, 1D
 * tables, GS table, status word and workspace; Alg. 1 storage and the solve workspace).
 *   alloc   : returns `bytes` of device memory of `device` (the current device during the
 *             call), aligned to at least 256 bytes, or NULL on failure (the plan then
 *             fails with SP_ERR_OOM).  Called only from sp_plan_create_ex.
 *   release : gives back a block that alloc returned, with the same size and device.
 *             Called only from sp_plan_destroy (and from sp_plan_create_ex when it fails),
 *             after the plan's work has completed, with `device` current.
 *   ctx     : passed through to both.
 * A framework with its own device pool (for example PyTorch's caching allocator) passes
 * its allocation functions here so that plans draw on that pool.  The transient scratch
 * of sp_kernel_precompute is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
 * precompute stream) in either case.
 */
typedef struct {
    void* (*alloc)(size_t bytes, int device, void* ctx);
    void (*release)(void* ptr, size_t bytes, int device, void* ctx);
    void* ctx;
} sp_allocator;

/* sp_plan_create_ex -- sp_plan_create with the plan's device memory taken from
 * `allocator` (NULL: cudaMalloc/cudaFree, exactly sp_plan_create).  Both callbacks must
 * be non-NULL when allocator is given (else SP_ERR_INVALID). */
sp_status sp_plan_create_ex(sp_plan* out, const int n[3], const double box_lo[3],
                            const double box_hi[3], int padding, const double* gs_w,
                            const double* gs_a, int gs_terms, double eps, sp_precision prec,
                            int max_batch, const sp_allocator* allocator);

/*
 * sp_plan_set_kernel -- which convolution kernel sp_kernel_precompute builds (default
 * SP_KERNEL_SUPERPOTENTIAL).  SP_KERNEL_GS_PLAIN is the original GS method without its
 * near-field correction (Sec. 1; the bracketed columns of Tab. 2): the multiplier is the
 * Fourier transform of the GS approximation of 1/(4 pi |y|) itself, sum_s 2 w_s G1 G2 G3
 * / Ntilde, with no Laplacian symbol; its cutoff error is O(eps^2) where the
 * super-potential kernel's is O(eps^4) (Lemma 1).  Marks the plan not ready: call
 * sp_kernel_precompute afterwards.
 */
typedef enum { SP_KERNEL_SUPERPOTENTIAL = 0, SP_KERNEL_GS_PLAIN = 1 } sp_kernel;
sp_status sp_plan_set_kernel(sp_plan plan, sp_kernel kind);

/*
 * sp_kernel_precompute -- Alg. 1 on the GPU, all in FP64: GS table (if not given),
 * the 1D integral tables G, H of eq. (Gten_sep) (closed full-line forms where
 * a_s L^2 >= 40; else composite 16-point Gauss-Legendre with nodes computed on the
 * device, applied directly for kappa^2 < 4 a_s and, above, to the fourth-derivative
 * remainder after two exact integrations by parts), the multiplier M_k of
 * eq. (convtheorem), and the FFT twiddles.
 * Stream-ordered on `stream`; idempotent.  The plan is ready for solves once the work
 * on `stream` completes; solves issued on other streams must be ordered after it by
 * the caller.
 */
sp_status sp_kernel_precompute(sp_plan plan, sp_stream stream);

/*
 * sp_solve -- one solve (Alg. 2): rho (device, n0 x n1 x n2, float64 for SP_FP64,
 * SP_MIXED and SP_DF32, float32 for SP_FP32) -> u (device, same shape and type).
 * u may alias rho.
 * The caller owns rho and u.  Stream-ordered; no host synchronisation.
 * Returns SP_ERR_NOT_READY before sp_kernel_precompute.
 */
sp_status sp_solve(sp_plan plan, const void* rho, void* u, sp_stream stream);

/*
 * sp_solve_batched -- `batch` independent solves on contiguous arrays
 * rho[b][x][y][z] -> u[b][x][y][z], 1 <= batch <= max_batch.  Same types and aliasing
 * rules as sp_solve.
 */
sp_status sp_solve_batched(sp_plan plan, const void* rho, void* u, int batch,
                           sp_stream stream);

/*
 * sp_solve_host -- `count` solves of host-resident arrays (Alg. 2 each), end to end:
 * rho_host[i] (host, n0 x n1 x n2 of the plan's I/O type) is copied to the device, solved,
 * and the result copied to u_host[i] (host, same shape and type), for i = 0..count-1 in
 * order.  The copies run on two streams of the plan's own, double-buffered, so that the
 * copy of input i+1 and of result i-1 overlap solve i on `stream`; page-locked host
 * memory (cudaHostAlloc / cudaHostRegister) is needed for that overlap (pageable memory
 * works, with the copies serialised by the driver).  Stream-ordered: when the work on
 * `stream` is complete, every result is in its host array; no host synchronisation.
 * The first call allocates the plan's four staging buffers (two inputs, two outputs),
 * through the plan's allocator if it has one, and two copy streams; later calls reuse
 * them.  rho_host[i] and u_host[i] may be the same array.  The host arrays must stay
 * valid, and unread and unwritten by the host, until the work on `stream` completes.
 */
sp_status sp_solve_host(sp_plan plan, const void* const* rho_host, void* const* u_host, int count,
                        sp_stream stream);

/* sp_plan_destroy -- release everything the plan owns once its own outstanding work (the
 * last work it issued, on whichever stream) has completed, from any current device (the
 * current device is left as it was).  Other work on the device is never waited for: the
 * library's own device memory is freed stream-ordered after that work (cudaFreeAsync,
 * no host wait); with a caller's allocator, destroy waits on the host for the plan's
 * work alone and then hands the blocks back.  NULL is accepted. */
sp_status sp_plan_destroy(sp_plan plan);

/*
 * sp_plan_sync -- host-synchronising: wait for the last work the plan issued (solves,
 * precompute, graph launches) and report what went wrong asynchronously since the last
 * sp_plan_sync:
 *   SP_ERR_TIMEOUT : a kernel's bounded wait gave up (sp_solve_persistent); the status
 *                    word is cleared, so the next sp_plan_sync returns SP_OK again;
 *   SP_ERR_CUDA    : a device error (the CUDA context may then be unusable);
 *   SP_OK          : otherwise.
 * Solves return before their kernels run, so this is where errors that a kernel detects
 * surface.
 */
sp_status sp_plan_sync(sp_plan plan);

/* Bytes of device workspace the plan holds for solves (0 for a NULL plan). */
size_t sp_plan_workspace_bytes(const sp_plan plan);

/* Number of GS terms of the plan (known after create: the given table's length, or the
 * length of the table sp_kernel_precompute generates for the plan's eps). */
int sp_plan_gs_terms(const sp_plan plan);

/*
 * sp_plan_copy_tables -- diagnostic read-back (host synchronising): copies the plan's
 * FP64 tables to host arrays; any pointer may be NULL to skip it.
 *   gs_w, gs_a : sp_plan_gs_terms() doubles each.
 *   M          : (n0+1)(n1+1)(n2+1) doubles, M[k0][k1][k2] = -|kappa|^2 Vhat / Ntilde, the
 *                multiplier exactly as the solve applies it, |k_p| = 0..n_p.
 *   G, H       : for axis `axis`, gs_terms x (n_axis+1) doubles each, [s][k].
 */
sp_status sp_plan_copy_tables(sp_plan plan, double* gs_w, double* gs_a, double* M,
                              int axis, double* G, double* H);

/*
 * sp_bluestein_table -- diagnostic, host only (no device work): the table a plan builds
 * for an axis whose padded length N = 2n has a prime factor above 7, where the passes
 * run Bluestein's algorithm (the chirp-z transform: jk = (j^2 + k^2 - (k-j)^2) / 2 turns
 * the length-N DFT into a convolution, evaluated as a circular convolution of length M,
 * the smallest power of two >= 2N - 1).  Complex values in the pass type of `prec`
 * (layout as in sp_forward_spectrum), in this order:
 *   chirp     c_j = exp(-i pi (j^2 mod 2N) / N), j < N;
 *   D_fwd     DFT_M of conj(c) placed at m and M - m (m < N, zeros between), divided by M;
 *   D_inv     the same from c;
 *   twiddles  exp(-2 pi i q / M), q < M.
 *   n      : grid points of the axis, 2 <= n <= 1024.
 *   M      : receives M.
 *   out    : host buffer, or NULL to query M and the size.
 *   bytes  : with out NULL receives the table's size in bytes; else gives the buffer's size.
 * SP_ERR_UNSUPPORTED_SIZE when n is out of range or 2n has no prime factor above 7 (radix
 * stages serve it); SP_ERR_INVALID for NULL M or bytes, an unknown precision, or a buffer
 * smaller than the table.
 */
sp_status sp_bluestein_table(int n, sp_precision prec, int* M, void* out, size_t* bytes);

/*
 * sp_forward_spectrum -- diagnostic: only the forward half of Alg. 2.  Writes the
 * unnormalised padded DFT of rho, spec[kx][ky][kz] for kx < 2n0, ky < 2n1, kz <= n2,
 * as interleaved complex values of the pass type: float64 pairs (SP_FP64), float32 pairs
 * (SP_FP32, SP_MIXED), or double-float values (SP_DF32: four float32 per value, in the
 * order re.hi, im.hi, re.lo, im.lo; re = re.hi + re.lo, im = im.hi + im.lo).  `spec` is device memory of 2n0 * 2n1 * (n2+1) complex values.  Uses the
 * plan's workspace.
 */
sp_status sp_forward_spectrum(sp_plan plan, const void* rho, void* spec, sp_stream stream);

/*
 * Pass timing (diagnostic).  With timing enabled, every solve records a CUDA event on its
 * stream before its first pass and after each pass; sp_plan_pass_times then waits for the
 * last recorded event, adds up the elapsed time of each pass over all solves recorded
 * since the previous call, and clears the record.
 *   sp_plan_set_timing : enable > 0 turns recording on and makes sure events for at least
 *                        `enable` solves exist (they are created here, so that the solves
 *                        recorded afterwards create none); 0 turns it off (the default).
 *                        The events are kept, and reused by later records, until destroy.
 *   sp_plan_pass_times : total_ms[i] (milliseconds) and launches[i] for pass i (both
 *                        arrays of max_passes entries, either may be NULL); names[i]
 *                        (may be NULL) receives a static string naming pass i.  Returns
 *                        the number of passes of one solve (<= max_passes are written),
 *                        or -1 on error (see sp_last_error).
 */
sp_status sp_plan_set_timing(sp_plan plan, int enable);
int sp_plan_pass_times(sp_plan plan, double* total_ms, int* launches, const char** names,
                       int max_passes);

/*
 * Batched execution (configurations with many right-hand sides of one size).
 *
 * sp_plan_autotune -- choose the CTA tiles of the solve passes, and the radix plan of the
 *   line passes, for `batch` right-hand sides (1 <= batch <= max_batch) by timing every
 *   candidate of each pass on the plan's workspace at that batch (host synchronising;
 *   overwrites the workspace).  Tiles decide which lines share a CTA, never the
 *   arithmetic of a line: results are bitwise identical for any tile.  Where a type and
 *   length has an alternative radix plan (FP32 and mixed at 2n = 256, 512, 1024:
 *   eight- or sixteen-value plans beside the built-in 16-16, 32-16, 32-32; double-float
 *   at 256: 16-16 beside 8-8-4), the line passes of each axis also time it; another plan
 *   rounds differently, so results then agree to the precision's tolerance, not bitwise.
 *   FP32 and mixed plans where the fused plane passes exist then time whole solves of
 *   both schedules and keep the faster (see sp_plan_launch_config).
 *   A no-op for grids without compiled register-resident passes.
 * sp_plan_tiles -- the tiles in use: line_tiles[3] (columns per CTA of the y and x line
 *   passes, by axis; 0 = default) and *z_tile (pairs of real lines per CTA of the z
 *   passes).  Either pointer may be NULL.
 */
sp_status sp_plan_autotune(sp_plan plan, int batch, sp_stream stream);
sp_status sp_plan_tiles(const sp_plan plan, int* line_tiles, int* z_tile);

/*
 * sp_plan_launch_config -- the launch configuration in use (what sp_plan_autotune chose):
 *   line_tiles[3], *z_tile : as sp_plan_tiles;
 *   line_plan[3]           : radix plan of the line passes per axis (index 0: the x pass,
 *                            1: the y passes; 0 built-in, 1 the alternative plan);
 *   radices[24]            : radices[8 ax + s] = radix of stage s of the forward transform
 *                            of the passes along axis ax (x pass, y passes, z passes), 0
 *                            after the last stage (the five-pass schedule's plans);
 *   *schedule              : 0 five passes, 1 the three-pass schedule with fused plane
 *                            passes (FP32 and mixed at 2n1 = 2n2 = 512: the z and y
 *                            transforms of an x-plane in one launch of 8-CTA clusters,
 *                            exchanging through distributed shared memory; its y phase uses
 *                            the eight-value plan), 2 the persistent single launch.
 * Any pointer may be NULL.
 */
sp_status sp_plan_launch_config(const sp_plan plan, int* line_tiles, int* z_tile, int* line_plan, int* radices,
                                int* schedule);

/*
 * sp_plan_set_launch_config -- set a launch configuration instead of tuning one (for
 * example one that sp_plan_autotune chose earlier and the caller saved): line_tiles[3]
 * and z_tile as sp_plan_tiles reports them (0 = built-in), line_plan[3] as
 * sp_plan_launch_config reports it (index 2 must be 0), schedule 0 (five passes) or 1
 * (fused plane passes; -1 leaves it unchanged; the persistent launch is set with
 * sp_plan_set_persistent).  A NULL pointer leaves that part unchanged.  A radix plan or a
 * schedule that does not exist for the type and grid is SP_ERR_UNSUPPORTED_SIZE; a tile
 * outside a pass's range fails at the next solve with SP_ERR_INVALID.
 */
sp_status sp_plan_set_launch_config(sp_plan plan, const int* line_tiles, int z_tile, const int* line_plan,
                                    int schedule);

/*
 * CUDA-graph capture of a (batched) solve on fixed buffers, replayed with one launch.
 *   sp_graph_capture -- runs sp_solve_batched(plan, rho, u, batch) once on `stream`
 *     (eagerly, so that every kernel attribute is set outside the capture), then captures
 *     the same call on `stream` (a created stream; the legacy NULL stream cannot capture)
 *     and instantiates it.  *out receives the graph.  The graph reads rho and writes u at
 *     the addresses given here, and uses the plan's tables and workspace: it must not
 *     outlive the plan or those buffers, and must not overlap other work on the plan.
 *   sp_graph_launch  -- replay on `stream` (stream-ordered, no host synchronisation).
 *   sp_graph_destroy -- free the graph (NULL accepted).
 */
/*
 * sp_plan_set_persistent -- enable != 0: every later solve of the plan (sp_solve,
 * sp_solve_batched, sp_graph_capture) runs as ONE persistent cooperative kernel launch
 * (after a 4-byte memset of its barrier counter): each block walks the tiles of the five
 * passes of Alg. 2 with a stride of the grid size, and a grid-wide barrier separates the
 * passes.  Results are bitwise those of the default five launches (tiles never change a
 * line's arithmetic).  The barrier's wait is bounded (2 s): a block that gives up sets
 * the plan's status word and leaves the kernel, and sp_plan_sync then returns
 * SP_ERR_TIMEOUT (the results of that solve are then incomplete).  Needs a cubic grid whose
 * padded length has a compiled plan (2n in {64, 128, 192, 256, 384, 512, 1024}), else
 * SP_ERR_UNSUPPORTED_SIZE.  enable = 0 returns to five launches.
 */
sp_status sp_plan_set_persistent(sp_plan plan, int enable);

/*
 * sp_plan_barrier_check -- diagnostic of the persistent solve's bounded grid wait:
 * launches `blocks` co-resident blocks (1 <= blocks <= number of SMs; a cooperative
 * launch) that each arrive once at a barrier waiting for `expected` arrivals, for at most
 * `limit_ms` (0 < limit_ms <= 2000) milliseconds.  With expected <= blocks the barrier
 * completes; with expected > blocks every block gives up after the limit and sets the
 * plan's status word, which the next sp_plan_sync reports as SP_ERR_TIMEOUT.  Uses the
 * plan's barrier counter: do not overlap it with the plan's solves.  Stream-ordered.
 */
sp_status sp_plan_barrier_check(sp_plan plan, int blocks, int expected, double limit_ms, sp_stream stream);

typedef struct sp_graph_s* sp_graph;
sp_status sp_graph_capture(sp_plan plan, const void* rho, void* u, int batch, sp_stream stream,
                           sp_graph* out);
sp_status sp_graph_launch(sp_graph graph, sp_stream stream);
sp_status sp_graph_destroy(sp_graph graph);

/*
 * sp_solve_noalloc -- the solve of sp_solve for callers that cannot allocate device
 * memory when they solve.  (The paper has no counterpart; this is an interface for
 * programs whose device memory is fixed in advance.)  cudaMalloc/cudaFree can
 * synchronise the whole device and stall a latency-bound loop, a host framework may
 * reserve all device memory for its own pool, and an allocation that fails halfway
 * through a long run is worse than one refused up front.  Such a caller creates and
 * precomputes the plan while it may allocate, then calls this entry point, which
 * allocates nothing: no cudaMalloc, cudaFree, or allocating routine of any library.
 *   plan    : a plan on the current device, precomputed (else SP_ERR_NOT_READY).
 *   rho, u  : as for sp_solve (device, n0 x n1 x n2, the plan's I/O type; u may alias rho).
 * The workspace is a static device array of SP_NOALLOC_MAX_BYTES bytes inside this
 * library (one per GPU that loads the library, held until the process exits) instead
 * of the plan's workspace.  A grid whose workspace, (16 bytes for SP_FP64 and SP_DF32,
 * else 8) x
 * n0 x 2n1 x round_up(n2 + 1, 8), exceeds it is rejected with SP_ERR_UNSUPPORTED_SIZE
 * (of the supported cube sizes, FP64 fits up to n = 126, double-float up to n = 96, its
 * largest supported length below that, and FP32/mixed up to n = 150).
 * The first call on a device looks up the array's device address (once per device,
 * with that device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use this entry point after
 * cudaDeviceReset (the address kept from before the reset is no longer valid).  Every
 * call shares the one array and overwrites it, so calls whose work overlaps on the
 * GPU (other streams, other threads, other plans) race and must be serialised by the
 * caller.  Stream-ordered; no host synchronisation.
 */
#define SP_NOALLOC_MAX_BYTES (64u * 1024u * 1024u)
sp_status sp_solve_noalloc(const sp_plan plan, const void* rho, void* u, sp_stream stream);

/*
 * Continuous-batching solve server (the served configuration: many requests of different
 * grid sizes and accuracy classes arriving over time).  Requests are solves of n^3 grids
 * on the box [lo, hi]^3 (Alg. 2 each); a scheduler thread of the library admits them onto
 * the GPU as stream slots and device memory free up, so that the work of different
 * requests overlaps on the device:
 *   - each (n, precision) key is served by up to plans_per_key resident plans (multiplier,
 *     workspace and batch buffers stay on the device), created on first use, or in
 *     advance by sp_server_prepare, within budget_bytes of device memory (estimate:
 *     sp_server_entry_bytes); idle plans of other keys are evicted, least recently used
 *     first, to make room; a request waits while its key's plans are busy;
 *   - the key whose oldest request has waited longest is served first; its waiting
 *     requests form one batch (at most max_batch requests, at most max_batch_points grid
 *     points, at least one request);
 *   - a batch runs on one of `slots` CUDA streams (host-to-device copies, one batched
 *     solve, device-to-host copies); the first priority_slots streams have the device's
 *     highest stream priority and take batches of at most small_points grid points first;
 *   - completion is stamped by a host callback when the results are in host memory, on
 *     the host's monotonic clock (CLOCK_MONOTONIC, sp_monotonic_seconds);
 *   - a request that cannot be served (a plan that cannot be created, a key whose plan
 *     exceeds the whole budget) fails alone.
 * Host buffers are the caller's: rho_host and u_host hold n^3 values of the precision's
 * I/O type (float32 for SP_FP32, else float64), page-locked for asynchronous copies, and
 * must stay valid and untouched until the request's completion is reported.  The server
 * uses the device that is current at sp_server_create; its functions are thread-safe.
 */
typedef struct sp_server_s* sp_server;
typedef struct {
    double lo, hi;             /* box [lo, hi]^3 */
    double budget_bytes;       /* device memory the server may hold */
    int max_batch;             /* requests per batch */
    int slots;                 /* batches in flight (CUDA streams) */
    int priority_slots;        /* of which high-priority (at most slots - 1) */
    int plans_per_key;         /* resident plans per (n, precision) */
    long long small_points;    /* a batch of at most this many grid points is small */
    long long max_batch_points;/* grid points per batch */
} sp_server_config;
typedef struct {
    double arrival, launched, done; /* seconds, monotonic clock */
    int n, precision;
} sp_server_record;

/* Create a server (its scheduler thread starts at once) on the current device. */
sp_status sp_server_create(sp_server* out, const sp_server_config* cfg);
/* Build the resident plans of a key now (up to plans_per_key, within the budget), so that
 * no plan creation or precompute stalls the device once requests flow.  The server's
 * device must be current. */
sp_status sp_server_prepare(sp_server srv, int n, sp_precision prec);
/* Queue one request; *ticket identifies it.  arrival: its arrival time in seconds on the
 * monotonic clock, or a negative value for now. */
sp_status sp_server_submit(sp_server srv, int n, sp_precision prec, const void* rho_host, void* u_host,
                           double arrival, long long* ticket);
/* Queue `count` requests that a feeder thread submits at their arrival times (seconds on
 * the monotonic clock, non-decreasing): a load generator whose own delays do not enter
 * the latencies.  tickets[i] identifies request i.  Returns at once. */
sp_status sp_server_replay(sp_server srv, int count, const double* arrival, const int* n, const int* precision,
                           const void* const* rho_host, void* const* u_host, long long* tickets);
/* Wait (at most timeout_s seconds; negative: without limit) for the next finished request
 * and report it: *ticket, times[3] = arrival, launch, completion (may be NULL), and its
 * status as the return value (SP_OK when its result is in u_host).  SP_ERR_NOT_READY: the
 * wait timed out; SP_ERR_INVALID: the server has stopped and every request was
 * reported. */
sp_status sp_server_next_done(sp_server srv, double timeout_s, long long* ticket, double* times);
/* Batches launched, peak and current device bytes held (budget accounting). */
sp_status sp_server_stats(sp_server srv, long long* batches, double* peak_bytes, double* used_bytes);
/* Copy up to `max` records of completed requests (in completion order) to out; returns
 * how many there are (-1 on error). */
int sp_server_records(sp_server srv, int max, sp_server_record* out);
/* Stop admitting, finish the batches in flight, fail the requests still waiting
 * (SP_ERR_INVALID, reported by sp_server_next_done).  Idempotent. */
sp_status sp_server_shutdown(sp_server srv);
/* Shut down and free everything the server holds.  No call on srv may be in progress or
 * follow. */
sp_status sp_server_destroy(sp_server srv);
/* Device bytes the server counts against its budget for one resident plan of the key. */
size_t sp_server_entry_bytes(const sp_server_config* cfg, int n, sp_precision prec);
/* The server's clock: seconds on the host's monotonic clock. */
double sp_monotonic_seconds(void);

/* Message of the last failed call on this host thread ("" if none). */
const char* sp_last_error(void);

/* Library version string. */
const char* sp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SUPERPOT_H */

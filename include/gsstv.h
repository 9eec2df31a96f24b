/*
 * gsstv.h -- C ABI of the GB300 (sm_103a) GeoSSTV P-PDS solver.
 *
 * The library runs Algorithm 1 of Takemoto & Ono, "GeoSSTV" (arXiv
 * 2510.00562): the preconditioned primal-dual splitting (P-PDS) solver of the
 * constrained denoising/destriping problem Prob. 15, rewritten as Prob. 20,
 *
 *   min  omega ||w1||_{1,2} + ||w2||_{1,2}
 *   s.t. s in B_{1,alpha}, t in B_{1,beta}, D_v t = 0,
 *        u + s + t in B_{2,eps}^v, u in [mu_lo, mu_hi],
 *        L^T w1 = D u,  L^T w2 = D D_s u,
 *
 * where D = (D_v; D_h) are the spatial forward differences, D_s the spectral
 * one (Sec. II-A, Neumann boundary) and L stacks Condat's interpolators
 * L_vert, L_hori, L_cent band by band (Sec. II-D Eqs. 10-12, Sec. III-A
 * Eq. 13).  The proximity operators are those of Eqs. 21-24; the l1 balls are
 * projected exactly (Sec. III-B).
 *
 * Conventions shared by every entry point:
 *  - A cube has N1 rows (vertical), N2 columns (horizontal) and N3 bands and
 *    is a C-contiguous float32 array of shape (N3, N1, N2): element (b, i, j)
 *    sits at offset (b*N1 + i)*N2 + j.
 *  - Pointers named d_* are CUDA device pointers, h_* host pointers.  The
 *    caller owns every pointer it passes; the library never frees them and
 *    keeps none of them after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work of a handle is issued on the handle's stream.
 *  - Every function returns GSSTV_OK (0) or a negative GSSTV_ERR_* code; on
 *    error the outputs are unspecified and the handle stays valid.
 *  - One handle must not be used from two host threads at once.
 */
#ifndef GSSTV_H
#define GSSTV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define GSSTV_OK              0
#define GSSTV_ERR_ARG        -1  /* null pointer, bad shape, bad parameter    */
#define GSSTV_ERR_OOM        -2  /* a device allocation failed                */
#define GSSTV_ERR_CUDA       -3  /* a CUDA runtime/driver call failed         */
#define GSSTV_ERR_NONFINITE  -4  /* NaN/Inf reached the l2-ball norm          */
#define GSSTV_ERR_TIMEOUT    -5  /* a bounded device wait gave up             */
#define GSSTV_ERR_INTERNAL   -6  /* an internal consistency check failed      */

/* ---- storage type of the iterates (arithmetic is always float32) ------- */
#define GSSTV_FP32  0
#define GSSTV_BF16  1
#define GSSTV_FP16  2

/* ---- threshold search for the l1-ball projections ----------------------- */
#define GSSTV_TAU_AUTO   0  /* windowed search around the last threshold,
                               exact radix search when the window misses   */
#define GSSTV_TAU_EXACT  1  /* always the exact radix search               */

typedef struct gsstv_params {
    /* Prob. 15 (Eqs. 16-19) and Eq. 13 */
    double eps;       /* radius of the l2 ball around v, >= 0               */
    double alpha;     /* radius of the l1 ball on s, >= 0 (0 forces s = 0)  */
    double beta;      /* radius of the l1 ball on t, >= 0 (0 forces t = 0)  */
    double omega;     /* weight of the first-order term, >= 0               */
    double mu_lo;     /* box on u: mu_lo < mu_hi                            */
    double mu_hi;
    /* step sizes of Algorithm 1, all > 0; gsstv_default_params sets the
       values printed in Sec. III-B (1/13, 1/4, 1/4, 1, 1/3, 1/5 x 4).      */
    double gamma_u, gamma_w1, gamma_w2, gamma_s, gamma_t;
    double gamma_y1, gamma_y2, gamma_y3, gamma_y4;
    /* driver */
    int    max_iter;     /* iterations per gsstv_solve (the cap if tol > 0)  */
    double tol;          /* Eq. 28: stop when ||u+ - u|| / ||u|| < tol; 0 = off */
    int    check_every;  /* iterations between two Eq. 28 tests (>= 1)       */
    int    storage;      /* GSSTV_FP32 | GSSTV_BF16 | GSSTV_FP16             */
    int    tau_mode;     /* GSSTV_TAU_AUTO | GSSTV_TAU_EXACT                 */
    int    graph_iters;  /* iterations per captured CUDA graph; 0 = no graph */
} gsstv_params;

typedef struct gsstv_handle gsstv_handle;

/* Per-handle counters, for benchmarks and tests. */
typedef struct gsstv_stats {
    int64_t iterations;        /* iterations run since create / reset_stats  */
    int64_t tau_window_hits;   /* l1 thresholds found by the fused pass's window */
    int64_t tau_exact_runs;    /* l1 thresholds found by the radix search    */
    double  k1_ms;             /* summed duration of the fused stencil kernel
                                  while timing is on (gsstv_set_timing)       */
    int64_t k1_launches;       /* launches covered by k1_ms                   */
    double  last_rel_change;   /* Eq. 28 ratio of the last iteration          */
    double  last_tau_s, last_tau_t; /* thresholds of the last iteration      */
    double  last_l2_scale;     /* min(1, eps / ||y4'/gamma_y4 - v||) (Eq. 23) */
    int64_t tau_retry_hits;    /* l1 thresholds found by one retry pass over a
                                  window placed after a miss                  */
    int64_t search_passes;     /* graph-launched passes whose threshold search
                                  launches ran (the rest skip them: K1's
                                  window found both thresholds)               */
} gsstv_stats;

/* Device views of the full state (float32, each a (N3,N1,N2) cube or a stack
 * of them): w1, w2 are 6 cubes ordered (grid g, component c) with g = 0, 1, 2
 * for the grids (i+1/2, j), (i, j+1/2), (i, j) of L_vert, L_hori, L_cent and
 * c = 0 vertical, 1 horizontal; y1, y2 are 2 cubes (vertical, horizontal). */
typedef struct gsstv_state_view {
    float* u; float* s; float* t;
    float* w1; float* w2;      /* 6*N floats each */
    float* y1; float* y2;      /* 2*N floats each */
    float* y3; float* y4;
} gsstv_state_view;

/* Fills *p with the printed step sizes of Sec. III-B, eps = alpha = beta = 1,
 * omega = 0.03, box [0, 1], max_iter = 1000, tol = 0, check_every = 100,
 * storage FP32, tau_mode AUTO, graph_iters = 16. */
void gsstv_default_params(gsstv_params* p);

/* Creates a solver for N1 x N2 x N3 cubes: the iterates of Algorithm 1
 * (primal u, s, t, w1, w2 and dual y1..y4 of Prob. 20, Sec. III-A/III-B,
 * with the sizes Eq. 13 gives them: w1, w2 in R^{6N}, y1, y2 in R^{2N}).
 * Allocates and zeroes the whole
 * iterate state on the current device (about 43 cube-sized buffers of the
 * storage type plus a float32 copy of v).  stream: cudaStream_t or NULL.
 * Limits: N1, N2 <= 2^20, N3 <= 2^16 and 6 * N1 * N3 * (N2 rounded up to 8)
 * < 2^32 (about 715 M voxels); larger shapes return GSSTV_ERR_ARG. */
int gsstv_create(gsstv_handle** h, int n1, int n2, int n3,
                 const gsstv_params* p, void* stream);

/* Replaces the parameters (same shape and storage type). */
int gsstv_set_params(gsstv_handle* h, const gsstv_params* p);

/* Releases every resource of the handle.  NULL is accepted. */
int gsstv_destroy(gsstv_handle* h);

/* Copies the observation v (d_v, device, N floats) into the handle. */
int gsstv_load_observation(gsstv_handle* h, const float* d_v);

/* Sets the starting point of Algorithm 1: u = v, and s, t, w1, w2, y1..y4 = 0. */
int gsstv_reset_state(gsstv_handle* h);

/* Runs `n` passes of Algorithm 1 from the current state (n >= 0).  When
 * tol > 0 it stops early once Eq. 28 holds at a check; *iters_done (may be
 * NULL) receives the number of passes run.  Synchronises the stream only for
 * the Eq. 28 checks and the final error check. */
int gsstv_iterate(gsstv_handle* h, int n, int* iters_done);

/* gsstv_load_observation + gsstv_reset_state + gsstv_iterate(max_iter), then
 * copies u, s, t (device, N floats each; s and t may be NULL) out. */
int gsstv_solve(gsstv_handle* h, const float* d_v, float* d_u, float* d_s,
                float* d_t, int* iters_done);

/* The same, end to end from host memory: copies h_v in, solves, copies u, s,
 * t back (s, t may be NULL).  Pinned host memory gives the fastest copies. */
int gsstv_solve_host(gsstv_handle* h, const float* h_v, float* h_u, float* h_s,
                     float* h_t, int* iters_done);

/* Reads / writes the full state of Algorithm 1 -- its primal iterates u, s, t,
 * w1, w2 and dual iterates y1..y4 (Sec. III-B; the layout of
 * gsstv_state_view) -- through float32 device views (every pointer non-NULL),
 * for warm starts (Algorithm 1 takes its initial point as an input) and
 * checkpoints.  With 16-bit storage the values are rounded on write.
 * set_state restarts the l1 threshold search; the next pass continues
 * Algorithm 1 from the given point. */
int gsstv_get_state(gsstv_handle* h, const gsstv_state_view* st);
int gsstv_set_state(gsstv_handle* h, const gsstv_state_view* st);

/* Counters; timing adds CUDA events around each launch of the fused stencil
 * kernel (off by default). */
int gsstv_get_stats(gsstv_handle* h, gsstv_stats* out);
int gsstv_reset_stats(gsstv_handle* h);
int gsstv_set_timing(gsstv_handle* h, int on);

/* Launch tuning (the paper has no counterpart: this is a launch parameter of
 * this implementation, not part of Algorithm 1).  Picks the number of bands
 * each CTA of the fused stencil kernel runs through by measurement: times that kernel (CUDA events) over `passes`
 * passes from the standard start on the loaded observation for each of a few
 * candidate run lengths (the wave/prologue model's choice and the next best by
 * its estimate), keeps the fastest for this handle and resets the state.
 * *chunk_out (may be NULL) receives the bands per CTA chosen, or 0 when the
 * handle runs the cooperative kernel (16-bit storage), which has nothing to
 * tune.  Results do not depend on the choice beyond the summation order of
 * the l1 window statistics.  Synchronises the stream; the counters of
 * gsstv_get_stats are left as they were. */
int gsstv_autotune(gsstv_handle* h, int passes, int* chunk_out);

/* Bytes the handle holds on the device. */
int64_t gsstv_device_bytes(const gsstv_handle* h);

/* ---- batches of independent cubes ------------------------------------------
 * Algorithm 1 on many cubes of different shapes at once (each cube its own
 * problem, with its own parameters and its own Eq. 28 stopping rule).  A
 * batch holds one solver per cube, each on a stream of its own; a solve keeps
 * a block of passes (check_every, or max_iter when tol = 0) in flight for
 * every unfinished cube and applies each cube's stopping rule as gsstv_iterate
 * does, so every cube gets exactly the result gsstv_solve gives it alone.
 *
 * gsstv_batch_create: ncubes >= 1; n1, n2, n3, params: ncubes entries each
 * (host arrays, read during the call); each cube obeys gsstv_create's limits.
 * stream: the caller's cudaStream_t (or NULL); solves start after the work
 * already queued on it.  Errors: GSSTV_ERR_ARG, GSSTV_ERR_OOM, GSSTV_ERR_CUDA;
 * nothing is left allocated on an error.
 *
 * gsstv_batch_solve: d_v, d_u (and d_s, d_t unless NULL): host arrays of
 * ncubes device pointers, each to a C-contiguous (N3, N1, N2) float32 cube of
 * that cube's shape, owned by the caller; iters_done (NULL or ncubes ints)
 * receives the passes each cube ran.  Returns when every cube has finished;
 * on an error no work of the batch is left in flight. */
typedef struct gsstv_batch gsstv_batch;
int gsstv_batch_create(gsstv_batch** b, int ncubes, const int* n1, const int* n2, const int* n3,
                       const gsstv_params* params, void* stream);
int gsstv_batch_solve(gsstv_batch* b, const float* const* d_v, float* const* d_u,
                      float* const* d_s, float* const* d_t, int* iters_done);
/* Number of cubes; the solver of cube c (owned by the batch: not destroyed
 * by the caller), e.g. for gsstv_get_stats. */
int gsstv_batch_size(const gsstv_batch* b);
int gsstv_batch_handle(gsstv_batch* b, int c, gsstv_handle** out);
/* Releases the batch and every solver in it.  NULL is accepted. */
int gsstv_batch_destroy(gsstv_batch* b);

/* ---- one cube split into band slabs -------------------------------------
 * Algorithm 1 on one cube whose bands are split into `nslabs` contiguous
 * slabs (slab s owns bands [s N3 / nslabs, (s + 1) N3 / nslabs)), each stored
 * in allocations of its own with one halo band on each side.  The only
 * couplings between bands are D_s and D_s^T (Sec. II-A) and the global sums
 * of a pass: the l2-ball norm of Eq. 23, the l1-ball thresholds (Sec. III-B)
 * and the Eq. 28 norms.  So each pass runs every kernel once per slab, with
 * the partial sums of all slabs finished together, and then refreshes the
 * halos with one device copy per plane: u, q (y4), y1, y2 of the band above
 * each slab and y2 of the band below.  The results equal those of a single
 * handle up to the summation order of the global sums.  This is the data
 * flow of a cube split over several GPUs (one slab per GPU, the partial sums
 * all-reduced, the halo planes exchanged); here every slab lives on the
 * current device.  Float32 storage only (GSSTV_ERR_ARG otherwise); 1 <=
 * nslabs <= N3; each slab obeys gsstv_create's limits.
 *
 * The calls mirror the single-handle ones: views and cubes are whole-cube
 * (N3, N1, N2) float32 device arrays owned by the caller; set_state fills
 * the halos from the view; every call synchronises the stream before it
 * returns, except load_observation.  gsstv_slabs_count returns the number of
 * slabs and writes the bands each owns to bands_out (NULL allowed). */
typedef struct gsstv_slabs gsstv_slabs;
int gsstv_slabs_create(gsstv_slabs** out, int n1, int n2, int n3, int nslabs,
                       const gsstv_params* p, void* stream);
int gsstv_slabs_destroy(gsstv_slabs* s);
int gsstv_slabs_load_observation(gsstv_slabs* s, const float* d_v);
int gsstv_slabs_reset_state(gsstv_slabs* s);
int gsstv_slabs_iterate(gsstv_slabs* s, int n, int* iters_done);
int gsstv_slabs_solve(gsstv_slabs* s, const float* d_v, float* d_u, float* d_s,
                      float* d_t, int* iters_done);
int gsstv_slabs_get_state(gsstv_slabs* s, const gsstv_state_view* st);
int gsstv_slabs_set_state(gsstv_slabs* s, const gsstv_state_view* st);
int gsstv_slabs_get_stats(gsstv_slabs* s, gsstv_stats* out);
int gsstv_slabs_count(const gsstv_slabs* s, int* bands_out);

/* ---- reverse mode (gradients of the unrolled iteration) -------------------
 * The derivative of K passes of Algorithm 1 with respect to the observation
 * v and the radii and weight (eps, alpha, beta, omega), for learning them or
 * for sensitivity studies.  The iteration's operators are piecewise smooth;
 * the transpose uses the derivatives that hold almost everywhere: the box
 * (Eq. 21) passes where mu_lo < u+ < mu_hi; the group soft-threshold (Eq. 24)
 * above its threshold has Jacobian (1 - g/|x|) I + g x x^T/|x|^3; the
 * l1-ball projection (Sec. III-B), when active, keeps the support A of its
 * result and removes the mean of sign(x) p over A (its derivative in the
 * radius is that mean); the l2-ball step (Eq. 23, through Eq. 3) is
 * y4 = (1 - c) q with Jacobian I - (eps g/|q|)(I - q^ q^^T) when the ball is
 * active.  The linear operators D, D_s, L are transposed exactly.  Float32
 * arithmetic throughout; only handles with GSSTV_FP32 storage are accepted
 * (GSSTV_ERR_ARG otherwise).
 *
 * gsstv_vjp_step: one pass.  x: the state before the pass, x_next: the state
 * after it (as gsstv_iterate(h, 1) gives it from x with the handle's loaded
 * observation and parameters), bar_next: the adjoint of x_next; writes the
 * adjoint of x to bar (bar may be bar_next itself: the transpose runs in
 * place; no other views may overlap).  Adds the adjoint of v to d_vbar (N
 * floats) and those of (eps, alpha, beta, omega) to h_pbar[0..3] (host).
 * All views: float32 device arrays in the layout of gsstv_state_view.  Uses
 * a workspace of about 15 N floats held by the handle from the first call.
 * Synchronises the stream to read the parameter adjoints back; with h_pbar
 * NULL it skips them and returns once the work is queued.
 *
 * gsstv_unrolled_vjp: `iters` passes from the standard start (u = v, the
 * rest zero; the observation loaded in the handle, tol ignored) and back.
 * d_ubar: adjoint of u after the last pass (N floats, device).  Writes to
 * d_vbar (N floats, device) the adjoint of v -- through every pass and the
 * start u = v -- and to h_pbar[0..3] those of eps, alpha, beta, omega.
 * ckpt_every: passes between checkpoints (0 = ceil(sqrt(iters))); with
 * C = min(ckpt_every, iters) the call allocates ceil(iters/C) + C + 1 states
 * of 21 N floats and a 15 N-float workspace with cudaMalloc and frees them
 * before returning (GSSTV_ERR_OOM if they do not fit), runs the passes about
 * twice in all (once with ckpt_every = 1: every state is kept and nothing is
 * run again), and leaves the handle's state unspecified (reset it before
 * iterating again).  Synchronises the stream. */
int gsstv_vjp_step(gsstv_handle* h, const gsstv_state_view* x, const gsstv_state_view* x_next,
                   const gsstv_state_view* bar_next, const gsstv_state_view* bar, float* d_vbar,
                   double* h_pbar);
int gsstv_unrolled_vjp(gsstv_handle* h, int iters, int ckpt_every, const float* d_ubar, float* d_vbar,
                       double* h_pbar);

/* Projection onto the l1 ball {z : ||z||_1 <= radius} (Sec. III-B, the prox
 * of the indicator of B_{1,alpha}): d_out = sign(x) max(|x| - tau, 0), with
 * tau >= 0 the root of sum max(|x_i| - tau, 0) = radius, or d_out = d_x when
 * ||x||_1 <= radius; radius = 0 gives d_out = 0.  d_x, d_out: device, n
 * floats (may alias); tau_out: host double (may be NULL).  Allocates its
 * scratch with cudaMalloc and synchronises the stream before returning. */
int gsstv_project_l1ball(const float* d_x, int64_t n, double radius,
                         float* d_out, double* tau_out, void* stream);

/* Allocation-free variant of gsstv_project_l1ball.  The paper has no
 * counterpart: it exists for callers that must not allocate device memory --
 * code whose device memory belongs to another allocator (for example a
 * framework's caching allocator that has already reserved the free memory, so
 * a raw cudaMalloc may fail or fragment it), latency-critical loops that
 * cannot afford the device-wide synchronisation of cudaFree, and plugin code
 * that is not permitted to allocate.
 *
 * Same arguments, result and error codes as gsstv_project_l1ball; it calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch is one
 * static device array of about 1.1 MB (a controller block, two radix
 * histograms and a buffer of GSSTV_NOALLOC_MAX_N floats) that every device
 * loading this library holds until the process exits.
 *  - n > GSSTV_NOALLOC_MAX_N returns GSSTV_ERR_ARG.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) and configures the kernels, with that device
 *    current; make that first call before any stream capture.
 *  - Every call shares the one array (each call clears what must start at
 *    zero): calls whose GPU work overlaps -- on different streams or from
 *    different host threads -- race and give wrong results.
 *  - Synchronises the stream before returning. */
#define GSSTV_NOALLOC_MAX_N 262144
int gsstv_project_l1ball_noalloc(const float* d_x, int64_t n, double radius,
                                 float* d_out, double* tau_out, void* stream);

/* Human-readable text of a return code. */
const char* gsstv_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GSSTV_H */

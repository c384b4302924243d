/*
 * lgnk.h - C ABI of the GB300 Lagrangian Gauss-Newton-Krylov hot path.
 *
 * The method (Mang & Ruthotto, arXiv 1703.04446): a velocity v(x, t) moves the
 * template T along characteristics (Eq. 4) computed by RK4 with N steps
 * (Alg. 1).  The final state u1(v) is the transport pull-back
 * u1 = T(y(v, x_c, 1, 0)) (Eq. 6, intensity preserving) or the particle-in-cell
 * push-forward u1 = F(y(v, x_c, 0, 1)) T(x_c) (Eqs. 7-8, mass preserving).
 * Registration minimises J(v) = D(u1(v), R) + alpha S(v) (Eq. 9) with the SSD
 * distance (Eq. 10) by an inexact Gauss-Newton-Krylov method (Eq. 11).
 *
 * Conventions for every call below:
 *  - Array arguments are DEVICE pointers owned by the caller, contiguous
 *    float32, 16-byte aligned (what cudaMalloc and torch return), unless the
 *    argument says "host".
 *  - A grid with m = (m_x, m_y[, m_z]) cells on [lo, hi] has its points at the
 *    cell centres lo + (i + 1/2) h (Sec. 3).  Images have M = prod(m) values,
 *    x fastest: index = (z * m_y + y) * m_x + x.
 *  - A velocity has n = K * d * M_v values in layout [K][d][z][y][x]:
 *    K time nodes at t_j = j / (K - 1) (K = 1: stationary), d components
 *    (component c is the velocity along axis c, in domain units per unit time).
 *  - Interpolation extends grid data by zero outside the grid: an image or
 *    velocity sample outside is 0 and push-forward mass that lands outside the
 *    image grid leaves it.
 *  - Output arrays are overwritten, never accumulated.
 *  - All work is ordered on the context's CUDA stream; a call returns when its
 *    work is enqueued, except where it returns host scalars (lgnk_objective,
 *    lgnk_dot, lgnk_solve), which synchronise that stream.
 *  - Calls return a status and never abort or throw.  A context is used by one
 *    host thread at a time.
 */
#ifndef LGNK_H
#define LGNK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LGNK_OK = 0,
    LGNK_ERR_INVALID_ARG = 1,  /* bad pointer, size, enum value or alignment   */
    LGNK_ERR_OOM = 2,          /* scratch does not fit the memory budget       */
    LGNK_ERR_CUDA = 3,         /* a CUDA runtime call failed (see last error)  */
    LGNK_ERR_NUMERIC = 4,      /* NaN or Inf met in a reduction                */
    LGNK_ERR_INTERNAL = 5,
    LGNK_LS_FAILED = 6,        /* Armijo found no decrease; v keeps last iterate */
    LGNK_NOT_CONVERGED = 7,    /* informational: iteration cap reached          */
    LGNK_ERR_CAPACITY = 8      /* a fixed-capacity structure is too small       */
} lgnk_status;

typedef enum { LGNK_TRANSPORT = 0, LGNK_CONTINUITY = 1 } lgnk_model;   /* Eq. 2 / Eq. 3 */
typedef enum { LGNK_SSD = 0 } lgnk_distance;                           /* Eq. 10 */
/* Sec. 2.1: diffusion (H1 seminorm), curvature (H2 seminorm); elastic is the
 * Navier-Lame form mu |grad v|^2 + (lambda + mu)(div v)^2, which the paper names
 * but does not define. */
typedef enum { LGNK_DIFFUSION = 0, LGNK_CURVATURE = 1, LGNK_ELASTIC = 2 } lgnk_regularizer;

/* Cell-centred regular grid (Sec. 3): d in {2, 3}; m[a] >= 1 cells on [lo[a], hi[a]]. */
typedef struct {
    int d;
    int m[3];
    double lo[3];
    double hi[3];
} lgnk_grid;

/* The discrete problem of Eq. 9.  time_nodes = K >= 1 (the paper's n_t + 1);
 * rk4_steps = N in [1, 64] (Alg. 1); gamma is the Hessian shift of Sec. 3.2. */
typedef struct {
    lgnk_grid image;
    lgnk_grid velocity;
    int time_nodes;
    int rk4_steps;
    int model;          /* lgnk_model       */
    int distance;       /* lgnk_distance    */
    int regularizer;    /* lgnk_regularizer */
    double alpha;
    double gamma;
    double mu_lame;     /* elastic only */
    double lambda_lame; /* elastic only */
    /* continuity only: PIC particle half-width delta in domain units (Eqs. 7-8).
     * 0: width equal to the cell size, F = P(y)^T (the experiments' choice).
     * delta > 0: each particle is the tensor product of unit-mass hats of
     * half-width delta, integrated exactly over every cell (mass-preserving
     * for any delta); delta / h <= 3.5 on every axis.  Transport requires 0. */
    double pic_delta;
} lgnk_problem;

typedef struct lgnk_ctx lgnk_ctx;

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL =
 * legacy default stream).  mem_budget: upper bound in bytes on the scratch the
 * context allocates (0 = no bound); LGNK_ERR_OOM when it does not fit.  The
 * context owns its scratch (packed velocity and image copies, accumulators,
 * FP64 reduction buffers, solver vectors) and frees it in lgnk_destroy. */
lgnk_status lgnk_create(const lgnk_problem* prob, void* stream, size_t mem_budget, lgnk_ctx** out);
void lgnk_destroy(lgnk_ctx* ctx);
lgnk_status lgnk_set_stream(lgnk_ctx* ctx, void* stream);
/* Bytes of device scratch this context holds. */
size_t lgnk_scratch_bytes(const lgnk_ctx* ctx);
const char* lgnk_status_string(lgnk_status s);
/* Detail of the last failure on this context, or with ctx = NULL of the last
 * failed lgnk_create on this thread (storage owned by the library, never NULL). */
const char* lgnk_last_error(const lgnk_ctx* ctx);

/* Final state u1(v) (Eq. 6 for transport, Eq. 7 for continuity).
 * v[n], T[M] in; u1[M] out.  y: NULL, or [d][M] receiving the end points of the
 * characteristics (transport: y(v, x_c, 1, 0); continuity: y(v, x_c, 0, 1)). */
lgnk_status lgnk_forward(lgnk_ctx* ctx, const float* v, const float* T, float* u1, float* y);

/* du = (d_v u1) dv: the derivative of the final state along dv (Sec. 3.2,
 * derivative recursion of Alg. 1).  v[n], T[M], dv[n] in; du[M] out. */
lgnk_status lgnk_jvp(lgnk_ctx* ctx, const float* v, const float* T, const float* dv, float* du);

/* gv = (d_v u1)^T r: the transpose of lgnk_jvp.  v[n], T[M], r[M] in; gv[n] out. */
lgnk_status lgnk_jtvp(lgnk_ctx* ctx, const float* v, const float* T, const float* r, float* gv);

/* Objective of Eq. 9 with SSD (Eq. 10): J = D + alpha S, D = h^d/2 |u1 - R|^2,
 * S = 1/2 dt h_v^d |B v|^2 (dt = 1/(K-1), 1 when stationary).  J, D, S: host
 * doubles (each may be NULL).  grad: NULL or device [n] receiving
 * d_v J = (d_v u1)^T h^d (u1 - R) + alpha dt h_v^d B^T B v (Sec. 3.2).
 * Sums are accumulated in FP64 per element (each product of FP32 values is
 * exact in FP64) and combined per block in FP64.  Synchronises the stream. */
lgnk_status lgnk_objective(lgnk_ctx* ctx, const float* v, const float* T, const float* R,
                           double* J, double* D, double* S, float* grad);

/* Gauss-Newton Hessian matvec (Sec. 3.2): Hdv = (d_v u1)^T h^d (d_v u1) dv +
 * alpha dt h_v^d B^T B dv + gamma dv, linearised at v.  v[n], T[M], dv[n] in;
 * Hdv[n] out. */
lgnk_status lgnk_hessvec(lgnk_ctx* ctx, const float* v, const float* T, const float* dv, float* Hdv);

/* Assembled J (transport).  The paper forms d_v u1 as a sparse matrix once per
 * Gauss-Newton iteration and applies it in every PCG matvec (Sec. 3.3).  Here
 * row i of J = d_v u1 is grad T(y_i)^T d_v y_i, computed by the adjoint sweep
 * of characteristic i and stored as at most 16 (3D) / 32 (2D) blocks, one per
 * (time slice, velocity cell) the characteristic's RK4 stages meet, each
 * holding the 2^d corner vectors; the products then read these rows instead
 * of re-tracing.
 * lgnk_assemble(ctx, v, T, blocks): builds J at (v, T) (device v[n], T[M]);
 * blocks: NULL or a host size_t receiving the number of blocks stored; the rows
 * live in the context (allocated on first use within its memory budget:
 * 16 x (8 + 96) bytes per voxel in 3D, 32 x (8 + 32) in 2D) until the next
 * lgnk_assemble or lgnk_solve with matvec = 1, which replaces them.  Returns
 * LGNK_ERR_CAPACITY when a characteristic meets more blocks than a row holds
 * (large displacements, many time slices) and LGNK_ERR_INVALID_ARG for the
 * continuity model.  Synchronises the stream.
 * lgnk_jvp_assembled: du[M] = J dv[n]; lgnk_jtvp_assembled: gv[n] = J^T r[M];
 * lgnk_hessvec_assembled: Hdv[n] as lgnk_hessvec at the assembled (v, T).
 * They return LGNK_ERR_INVALID_ARG when the context holds no valid J. */
lgnk_status lgnk_assemble(lgnk_ctx* ctx, const float* v, const float* T, size_t* blocks);
lgnk_status lgnk_jvp_assembled(lgnk_ctx* ctx, const float* dv, float* du);
lgnk_status lgnk_jtvp_assembled(lgnk_ctx* ctx, const float* r, float* gv);
lgnk_status lgnk_hessvec_assembled(lgnk_ctx* ctx, const float* dv, float* Hdv);

/* Spectral preconditioner (Sec. 3.2): z = P^-1 r with P = alpha dt h_v^d A + gamma I
 * applied through the DCT-II eigenbasis of the Neumann operator A; a zero
 * eigenvalue (gamma = 0, constant mode) takes the smallest nonzero one, keeping
 * P positive definite (elastic uses its mu-Laplacian part).  r[n] in; z[n] out. */
lgnk_status lgnk_precond(lgnk_ctx* ctx, const float* r, float* z);

/* Jacobian determinant det grad y of the map the velocity generates (the paper
 * monitors its range to check that the transformation stays diffeomorphic,
 * Sec. 2.1, Sec. 4): y = y(v, x_c, 1, 0) for transport, y(v, x_c, 0, 1) for
 * continuity, differentiated at the cell centres with central differences
 * (one-sided at the ends).  v[n], T[M] in (T as for lgnk_forward); det: NULL or
 * device [M]; det_min / det_max: host doubles (may be NULL).  Synchronises. */
lgnk_status lgnk_jacobian_determinant(lgnk_ctx* ctx, const float* v, const float* T, float* det,
                                      double* det_min, double* det_max);

/* Inner product of two device float arrays of length count, summed in FP64
 * per element (the products of FP32 values are exact in FP64) in a
 * deterministic order and returned on the host.  Synchronises the stream. */
lgnk_status lgnk_dot(lgnk_ctx* ctx, const float* a, const float* b, size_t count, double* out);

/* Profiling.  lgnk_profile(ctx, 1) resets the counters and starts recording a
 * pair of CUDA events on the context's stream around every tracing-kernel
 * launch (the RK4 kernels of lgnk_forward/jvp/jtvp/objective/hessvec) and
 * counting every kernel the context launches; lgnk_profile(ctx, 0) stops.
 * lgnk_profile_read synchronises the stream and returns the summed tracing-
 * kernel time in ms, the number of tracing launches and of all kernel
 * launches since the reset (any output may be NULL). */
lgnk_status lgnk_profile(lgnk_ctx* ctx, int enable);
lgnk_status lgnk_profile_read(lgnk_ctx* ctx, double* trace_ms, long long* trace_launches,
                              long long* kernel_launches);

typedef struct {
    int max_gn;           /* outer Gauss-Newton iterations (default 10)            */
    double gn_grad_rtol;  /* stop when |g| <= rtol |g0| (default 1e-3)             */
    int max_pcg;          /* PCG iterations per GN step (Sec. 4.1: 50)             */
    double pcg_rtol;      /* PCG relative residual (Sec. 4.1: 0.1)                 */
    double armijo_c;      /* sufficient-decrease constant (default 1e-4)           */
    int max_ls;           /* Armijo halvings (default 10)                          */
    int precond;          /* 1 = spectral preconditioner, 0 = none                 */
    int verbosity;        /* 0 silent, 1 one line per GN iteration on stderr       */
    double gn_grad_atol;  /* also stop when |g| <= atol (default 0: off)           */
    int matvec;           /* 1 (default): assembled J per GN step (transport; the    */
                          /* matrix-free products when it does not fit); 0: always   */
                          /* matrix-free                                             */
} lgnk_solve_opts;

typedef struct {
    int gn_iters;
    int pcg_iters;
    int hessvecs;
    int objective_evals;  /* objective evaluations: the start, one per line-search trial (the full step's  */
                          /* trial also yields the next gradient), one per gradient at a shorter step     */
    double J0, J, D, S;
    double g0, g;
    double seconds;
    int status;           /* lgnk_status of the solve */
    int assembled_gn;     /* GN iterations whose PCG used the assembled J */
    double last_mu;       /* Armijo step length of the last accepted GN step (0 if none) */
} lgnk_solve_report;

/* Fill opts with the defaults listed above. */
void lgnk_solve_opts_default(lgnk_solve_opts* opts);

/* Inexact Gauss-Newton-Krylov with Armijo line search (Eq. 11): from the
 * initial v_inout[n] (device, overwritten with the result), minimise J for the
 * template T[M] and reference R[M].  Hessian products, preconditioner, vector
 * updates and inner products (FP64 sums) run on the device; the host drives the loop.
 * After each PCG loop the full step is evaluated together with the gradient
 * (and, with matvec = 1, the rows of J) at v + x, and the host reads its
 * objective, the slope g.x, the new |g| and the PCG counters in one wait; a
 * rejected full step backtracks by halving with objective-only trials.  opts
 * may be NULL (defaults); report may be NULL.  Returns LGNK_OK on convergence,
 * LGNK_NOT_CONVERGED at the GN cap, LGNK_LS_FAILED when the line search stalls
 * (v_inout then holds the last accepted iterate, and the context's assembled J,
 * if any, is no longer valid). */
lgnk_status lgnk_solve(lgnk_ctx* ctx, const float* T, const float* R, float* v_inout,
                       const lgnk_solve_opts* opts, lgnk_solve_report* report);

/* Multilevel continuation (Sec. 3.2, last paragraph).
 *
 * lgnk_restrict_image: coarse image C (m/2 cells per axis, same box) = the
 * average of the 2^d fine cells tiling each coarse cell; keeps the integral.
 * fine->m must be even.  F[M_fine] in, C[M_fine / 2^d] out (device).
 *
 * lgnk_prolong_velocity: vf = the coarse velocity vc (layout [K][d][z][y][x] on
 * `coarse`) interpolated multilinearly, zero outside the coarse grid, at the
 * cell centres of `fine`, per time node and component.
 *
 * lgnk_solve_multilevel: Gauss-Newton (lgnk_solve with opts) on `levels`
 * discretisations from the coarsest (every cell count of image and velocity
 * divided by 2^(levels-1)) to `fine`.  Images are restricted level by level;
 * the coarsest level starts from v = 0 and every finer level from the
 * prolonged solution of the coarser one.  v_out[n_fine] (device) receives the
 * finest solution; reports: NULL or `levels` entries, coarsest first.  The call
 * allocates each level's context and buffers (within mem_budget, 0 = no bound)
 * and frees them before it returns; it synchronises the stream.  Returns the
 * finest level's lgnk_solve status.  All three report details through
 * lgnk_last_error(NULL). */
lgnk_status lgnk_restrict_image(const lgnk_grid* fine, const float* F, float* C, void* stream);
lgnk_status lgnk_prolong_velocity(const lgnk_grid* coarse, const lgnk_grid* fine, int time_nodes,
                                  const float* vc, float* vf, void* stream);
lgnk_status lgnk_solve_multilevel(const lgnk_problem* fine, int levels, void* stream, size_t mem_budget,
                                  const float* T, const float* R, float* v_out,
                                  const lgnk_solve_opts* opts, lgnk_solve_report* reports);

/* Allocation-free transport forward and SSD, for callers that must not call
 * cudaMalloc after start-up: a latency-critical loop (cudaMalloc can
 * synchronise the device and takes unbounded time) or a process whose device
 * memory already belongs to another allocator (a framework's caching
 * allocator, a pool sized at start-up).  The paper has no counterpart; this is
 * lgnk_forward (plus the SSD of lgnk_objective) for LGNK_TRANSPORT without a
 * context.
 *
 * prob: validated as in lgnk_create; model must be LGNK_TRANSPORT.
 * v[n], T[M] in; u1[M] out (device).  R[M] (device) and D (device, one double)
 * are both NULL or both given: D = h^d/2 |u1 - R|^2, summed in FP64.
 * stream: cudaStream_t (NULL = legacy default stream); the call only enqueues.
 *
 * Scratch: a file-scope device array of 32 MiB (every GPU that loads the
 * library holds it until exit).  A problem whose packed velocity, padded
 * template and partial sums exceed it is rejected with LGNK_ERR_INVALID_ARG
 * (the 128^3 image / 64^3 velocity workload fits).  Every call made outside a
 * stream capture looks up the array's device address (cudaGetSymbolAddress),
 * so a device reset between calls is harmless; a call made while its stream is
 * being captured reuses the address its device's last uncaptured call found,
 * so make the first call on a device before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Errors: the status, with detail from
 * lgnk_last_error(NULL).  Allocates nothing. */
lgnk_status lgnk_forward_transport_static(const lgnk_problem* prob, const float* v, const float* T,
                                          const float* R, float* u1, double* D, void* stream);

/* Learned warm start.  The paper starts every Gauss-Newton solve of Eq. 11 from
 * v = 0 (or, with continuation, from a coarser level); this network is an
 * addition with no counterpart there: it predicts a starting velocity from the
 * image pair, and the solve then corrects it (the optimality conditions are
 * unchanged, only the initial iterate differs).  2D, stationary velocity.
 *
 * Network for m x m images (m a multiple of 8), c base channels, 3 x 3
 * convolutions with zero padding 1:
 *   e0 = relu(conv(x = [T, R], 2 -> c))        e1 = relu(conv_s2(e0, c -> 2c))
 *   e2 = relu(conv_s2(e1, 2c -> 4c))           e3 = relu(conv_s2(e2, 4c -> 8c))
 *   d2 = relu(conv(up2(e3), 8c -> 4c)) + e2    d1 = relu(conv(up2(d2), 4c -> 2c)) + e1
 *   v  = scale conv(d1, 2c -> 2)               (m/2 x m/2, two components)
 * (s2: stride 2; up2: nearest-neighbour doubling).  Convolutions use the
 * weights rounded to bfloat16; activations and accumulation are FP32.
 * Parameters: one flat FP32 vector, per layer in the order above W[co][ci][3][3]
 * then b[co].  Loss: 1/2 mean((v - v_target)^2) / scale^2; training: Adam
 * (beta 0.9, 0.999, eps 1e-8) on FP32 master weights.
 *
 * Layouts (device, contiguous): T, R [B][m][m]; v, v_target [B][2][m/2][m/2]
 * (component-major, the velocity layout of lgnk_forward for K = 1).
 * lgnk_ws_create: max_batch bounds B of every later call; scale > 0; stream as
 * in lgnk_create.  The network owns its device buffers (parameters, Adam
 * moments, activations for max_batch) and frees them in lgnk_ws_destroy.
 * Parameters start at zero: load them with lgnk_ws_set_params (device [P],
 * P = lgnk_ws_num_params), which also resets Adam.  lgnk_ws_train_step runs
 * forward, backward and one Adam step with learning rate lr; loss: NULL or a
 * host double receiving the loss before the step (then the call synchronises
 * the stream).  lgnk_ws_get_grads copies the gradient of the last train step.
 * Errors: the status, with detail from lgnk_ws_last_error. */
typedef struct lgnk_ws lgnk_ws;
lgnk_status lgnk_ws_create(int image_m, int base_channels, int max_batch, float scale, void* stream,
                           lgnk_ws** out);
void lgnk_ws_destroy(lgnk_ws* ws);
size_t lgnk_ws_num_params(const lgnk_ws* ws);
const char* lgnk_ws_last_error(const lgnk_ws* ws);
lgnk_status lgnk_ws_set_params(lgnk_ws* ws, const float* params);
lgnk_status lgnk_ws_get_params(lgnk_ws* ws, float* params);
lgnk_status lgnk_ws_get_grads(lgnk_ws* ws, float* grads);
lgnk_status lgnk_ws_predict(lgnk_ws* ws, int batch, const float* T, const float* R, float* v);
lgnk_status lgnk_ws_train_step(lgnk_ws* ws, int batch, const float* T, const float* R, const float* v_target,
                               float lr, double* loss);

#ifdef __cplusplus
}
#endif

#endif /* LGNK_H */

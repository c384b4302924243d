// C ABI of the lgnk library (declared in include/lgnk.h): context and scratch
// management, the hot-path entry points, and the host-driven inexact
// Gauss-Newton-Krylov loop (Eq. 11) whose vector work and inner products run
// on the device.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "lgnk_internal.h"

cudaError_t launch_trace_2d(bool nonstat, int model, int mode, const TraceArgs& a, int nblocks, cudaStream_t s);
cudaError_t launch_trace_3d(bool nonstat, int model, int mode, const TraceArgs& a, int nblocks, cudaStream_t s);

cudaError_t launch_ell_2d(int mode, const EllArgs& a, cudaStream_t s);
cudaError_t launch_ell_3d(int mode, const EllArgs& a, cudaStream_t s);

cudaError_t launch_trace(int d, bool nonstat, int model, int mode, const TraceArgs& a, int nblocks, cudaStream_t s) {
    return d == 3 ? launch_trace_3d(nonstat, model, mode, a, nblocks, s)
                  : launch_trace_2d(nonstat, model, mode, a, nblocks, s);
}

cudaError_t launch_ell(int d, int mode, const EllArgs& a, cudaStream_t s) {
    return d == 3 ? launch_ell_3d(mode, a, s) : launch_ell_2d(mode, a, s);
}

// One PCG iteration's device work as a replayable CUDA graph (one per
// matvec variant), kept in the context across solves.  Captured on first
// use; the launches it holds are counted on every replay.  Everything the
// capture holds is fixed for the context (the solver's vectors and buffers,
// the problem's constants) except what the key records: whether the
// preconditioner is applied, and the template pointer (taken by the
// matrix-free mass-preserving product).
struct PcgGraphKey {
    int precond = -1;
    const float* T = nullptr;
    bool operator==(const PcgGraphKey& o) const { return precond == o.precond && T == o.T; }
};

struct PcgGraph {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0, trace_launches = 0;
    bool failed = false;
    PcgGraphKey key;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        launches = trace_launches = 0;
        failed = false;
    }
    ~PcgGraph() { reset(); }
};

// The whole PCG loop of one GN step as one graph: a while node whose body is
// one iteration followed by launch_pcg_control, which ends the loop on the
// stopping test, non-positive curvature or the iteration cap.  The host reads
// the loop state once per GN step instead of once per iteration.
struct PcgLoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0, trace_launches = 0;   // per iteration
    bool failed = false;
    PcgGraphKey key;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        launches = trace_launches = 0;
        failed = false;
    }
    ~PcgLoopGraph() { reset(); }
};

struct lgnk_ctx {
    lgnk_problem prob;
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t budget = 0, used = 0;
    DevGrid ig{}, vg{};
    int d = 0, K = 0, N = 0;
    size_t M = 0, Mv = 0, n = 0;  // image voxels, velocity nodes per block, unknowns
    size_t ipad = 0, vpad = 0;    // padded image elements, padded velocity nodes
    size_t vt_bytes = 0;          // bytes of one gradient-accumulator element
    SliceTable slices{};          // stage-time slices of the velocity
    int tiles[3] = {1, 1, 1};
    int trace_blocks = 0;
    double cellvol = 0.0;         // image h^d (Eq. 10)
    double wreg = 0.0;            // dt * h_v^d of the regularizer (Sec. 3.2)
    void *Vp = nullptr, *dVp = nullptr, *Gp = nullptr;
    float *Tp = nullptr, *acc = nullptr, *rp = nullptr, *itmp = nullptr, *rtmp = nullptr;
    float *pc0 = nullptr, *pc1 = nullptr, *Cm[3] = {nullptr, nullptr, nullptr}, *inv_eig = nullptr;
    // the DCT matrices in the shared-memory layouts of the tiled kernels, rows
    // padded to P = m rounded up to 4: forward Cf[q][k] = C[k][q], inverse Ci[q][k] = C[q][k]
    float *Cf[3] = {nullptr, nullptr, nullptr}, *Ci[3] = {nullptr, nullptr, nullptr};
    PcgGraph pcg_graphs[2];       // [0] matrix-free, [1] assembled products
    PcgLoopGraph pcg_loops[2];
    double* partial = nullptr;
    double* cpartial = nullptr;   // per-block entry counts of the assembled rows
    int npartial = 0;
    double* dres = nullptr;
    double* hres = nullptr;       // pinned host mirror of dres
    float* fsc = nullptr;         // PCG step lengths on the device (alpha, -alpha, beta)
    unsigned* dcounter = nullptr; // completion counter of launch_dot_fused (zero between launches)
    int* dctl = nullptr;          // device-side PCG loop state (launch_pcg_control)
    unsigned char* hpin = nullptr; // pinned: the loop state's host copy (4 ints) and its tolerance (a double)
    // lgnk_solve runs on a stream of its own (capturable, unlike the legacy
    // default stream), ordered after and before the caller's stream by events
    cudaStream_t solve_stream = nullptr;
    cudaEvent_t ev_enter = nullptr, ev_leave = nullptr;
    float* sv[7] = {nullptr};
    bool have_solve = false;
    float* ybuf = nullptr;        // end points [d][M] for lgnk_jacobian_determinant
    // assembled J (transport, lgnk_assemble): ELL rows of asm_capacity(d) entries
    long long* ekey = nullptr;
    float* eblk = nullptr;
    int* ecnt = nullptr;
    int* eflag = nullptr;
    bool asm_valid = false;
    size_t asm_entries = 0;       // blocks in the assembled rows
    std::vector<void*> allocs;
    // profiling: CUDA events around every tracing-kernel launch, kernel counter
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    long long launches = 0, trace_launches = 0;
    char err[512] = {0};
};

#define SETERR(...) snprintf(ctx->err, sizeof(ctx->err), __VA_ARGS__)
#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            SETERR("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);     \
            return LGNK_ERR_CUDA;                                                                   \
        }                                                                                           \
    } while (0)
// Checks a kernel launch of this library and counts it.
#define KL(call)                                                                                    \
    do {                                                                                            \
        ctx->launches++;                                                                            \
        CK(call);                                                                                   \
    } while (0)
#define TRY(expr)                          \
    do {                                   \
        lgnk_status s_ = (expr);           \
        if (s_ != LGNK_OK) return s_;      \
    } while (0)

namespace {

// Why the last lgnk_create failed (no context exists to hold it).
thread_local char g_create_err[512] = {0};

DevGrid make_grid(const lgnk_grid& g) {
    DevGrid o{};
    for (int a = 0; a < 3; ++a) {
        if (a < g.d) {
            o.m[a] = g.m[a];
            o.mp[a] = g.m[a] + 2 * LGNK_PAD;
            o.lo[a] = (float)g.lo[a];
            o.h[a] = (float)((g.hi[a] - g.lo[a]) / g.m[a]);
            o.inv_h[a] = (float)(g.m[a] / (g.hi[a] - g.lo[a]));
        } else {
            o.m[a] = 1;
            o.mp[a] = 1;
            o.lo[a] = 0.0f;
            o.h[a] = 1.0f;
            o.inv_h[a] = 1.0f;
        }
    }
    return o;
}

const char* validate_grid(const lgnk_grid& g, int d) {
    if (g.d != d) return "image and velocity grids must have the same dimension d";
    for (int a = 0; a < d; ++a) {
        if (g.m[a] < 1 || g.m[a] > (1 << 20)) return "grid cell counts must be in [1, 2^20]";
        if (!std::isfinite(g.lo[a]) || !std::isfinite(g.hi[a]) || !(g.hi[a] > g.lo[a]))
            return "grid bounds must be finite with hi > lo";
    }
    return nullptr;
}

const char* validate_problem(const lgnk_problem* p) {
    if (p == nullptr) return "problem is NULL";
    const int d = p->image.d;
    if (d != 2 && d != 3) return "image.d must be 2 or 3";
    if (const char* e = validate_grid(p->image, d)) return e;
    if (const char* e = validate_grid(p->velocity, d)) return e;
    if (p->time_nodes < 1 || p->time_nodes > 4096) return "time_nodes must be in [1, 4096]";
    if (p->rk4_steps < 1 || p->rk4_steps > LGNK_MAX_STEPS) return "rk4_steps must be in [1, 64]";
    if (p->model != LGNK_TRANSPORT && p->model != LGNK_CONTINUITY) return "unknown model";
    if (p->distance != LGNK_SSD) return "unknown distance";
    if (p->regularizer < LGNK_DIFFUSION || p->regularizer > LGNK_ELASTIC) return "unknown regularizer";
    if (!(p->alpha >= 0.0) || !std::isfinite(p->alpha)) return "alpha must be finite and >= 0";
    if (!(p->gamma >= 0.0) || !std::isfinite(p->gamma)) return "gamma must be finite and >= 0";
    if (p->regularizer == LGNK_ELASTIC &&
        (!(p->mu_lame >= 0.0) || !(p->lambda_lame + p->mu_lame >= 0.0) || !std::isfinite(p->lambda_lame)))
        return "elastic needs mu >= 0 and lambda + mu >= 0";
    if (!(p->pic_delta >= 0.0) || !std::isfinite(p->pic_delta)) return "pic_delta must be finite and >= 0";
    if (p->pic_delta > 0.0) {
        if (p->model != LGNK_CONTINUITY) return "pic_delta applies to the continuity model only";
        for (int a = 0; a < d; ++a)
            if (p->pic_delta * p->image.m[a] / (p->image.hi[a] - p->image.lo[a]) > 3.5 * (1.0 + 1e-9))
                return "pic_delta must be at most 3.5 image cells on every axis";
    }
    double ipad = 1.0, vpad = 1.0, M = 1.0;
    for (int a = 0; a < d; ++a) {
        ipad *= p->image.m[a] + 2 * LGNK_PAD;
        vpad *= p->velocity.m[a] + 2 * LGNK_PAD;
        M *= p->image.m[a];
    }
    // the packed velocity holds one slice per stage time (2N + 1) when it depends on time
    const double slices = p->time_nodes > 1 ? 2.0 * p->rk4_steps + 1.0 : 1.0;
    // (the grid kernels index every array, velocity blocks of K x d components included, in 32 bits)
    if (ipad >= 2147483647.0 || vpad * p->time_nodes * d >= 2147483647.0 || vpad * slices >= 2147483647.0 ||
        M >= 2147483647.0)
        return "grid too large for 32-bit node indexing";
    return nullptr;
}

lgnk_status dev_alloc(lgnk_ctx* ctx, size_t bytes, void** out) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->budget != 0 && ctx->used + bytes > ctx->budget) {
        SETERR("scratch of %zu bytes exceeds the memory budget (%zu of %zu used)", bytes, ctx->used, ctx->budget);
        return LGNK_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        SETERR("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return LGNK_ERR_OOM;
    }
    ctx->used += bytes;
    ctx->allocs.push_back(*out);
    return LGNK_OK;
}

template <typename T>
lgnk_status dalloc(lgnk_ctx* ctx, size_t count, T** out) {
    void* p = nullptr;
    lgnk_status s = dev_alloc(ctx, count * sizeof(T), &p);
    *out = static_cast<T*>(p);
    return s;
}

TraceArgs base_args(const lgnk_ctx* ctx) {
    TraceArgs a{};
    a.ig = ctx->ig;
    a.vg = ctx->vg;
    a.K = ctx->K;
    a.N = ctx->N;
    const bool transport = ctx->prob.model == LGNK_TRANSPORT;
    // transport traces y(v, x_c, 1, 0) backward, continuity y(v, x_c, 0, 1) forward
    a.dt = (float)((transport ? -1.0 : 1.0) / ctx->N);
    a.t0 = transport ? 1.0f : 0.0f;
    a.cellvol = (float)ctx->cellvol;
    for (int i = 0; i < 3; ++i) a.tiles[i] = ctx->tiles[i];
    for (int i = 0; i < 3; ++i) {
        if (i < ctx->d) {
            const lgnk_grid& gi = ctx->prob.image;
            const lgnk_grid& gv = ctx->prob.velocity;
            const double hi = (gi.hi[i] - gi.lo[i]) / gi.m[i], hv = (gv.hi[i] - gv.lo[i]) / gv.m[i];
            a.vxi_a[i] = (gi.lo[i] - gv.lo[i]) / hv - 0.5;
            a.vxi_b[i] = hi / hv;
            a.vxi_af[i] = (float)a.vxi_a[i];
            a.vxi_bf[i] = (float)a.vxi_b[i];
        } else {
            a.vxi_a[i] = 0.0;
            a.vxi_b[i] = 0.0;
            a.vxi_af[i] = 0.0f;
            a.vxi_bf[i] = 0.0f;
        }
    }
    for (int i = 0; i < 3; ++i)
        a.pic_rho[i] = i < ctx->d ? (float)(ctx->prob.pic_delta * ctx->prob.image.m[i] /
                                            (ctx->prob.image.hi[i] - ctx->prob.image.lo[i]))
                                  : 0.0f;
    a.slice_nodes = (long long)ctx->vpad;
    a.V = ctx->Vp;
    a.dV = ctx->dVp;
    a.Tp = ctx->Tp;
    a.G = ctx->Gp;
    return a;
}

lgnk_status record_event(lgnk_ctx* ctx) {
    if (ctx->ev_used == ctx->ev.size()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->ev.push_back(e);
    }
    CK(cudaEventRecord(ctx->ev[ctx->ev_used++], ctx->stream));
    return LGNK_OK;
}

int trace_blocks_for(const lgnk_ctx* ctx, int mode) {
    int ts[3];
    (void)mode;
    trace_tile_shape(ctx->d, ts);
    int n = 1;
    for (int i = 0; i < 3; ++i) n *= (ctx->ig.m[i] + ts[i] - 1) / ts[i];
    return n;
}

lgnk_status trace(lgnk_ctx* ctx, int mode, const TraceArgs& a) {
    if (ctx->prof) TRY(record_event(ctx));
    KL(launch_trace(ctx->d, ctx->K > 1, ctx->prob.model, mode, a, ctx->trace_blocks, ctx->stream));
    ctx->trace_launches++;
    if (ctx->prof) TRY(record_event(ctx));
    return LGNK_OK;
}

lgnk_status pack_v(lgnk_ctx* ctx, const float* v, void* dst) {
    KL(launch_pack_velocity(ctx->d, v, dst, ctx->vg, ctx->K, ctx->slices, ctx->stream));
    return LGNK_OK;
}

lgnk_status pack_T(lgnk_ctx* ctx, const float* T) {
    KL(launch_pack_image(T, ctx->Tp, ctx->ig, ctx->d, 1.0f, ctx->stream));
    return LGNK_OK;
}

lgnk_status zero_G(lgnk_ctx* ctx) {
    CK(cudaMemsetAsync(ctx->Gp, 0, ctx->vpad * ctx->slices.n * ctx->vt_bytes, ctx->stream));
    return LGNK_OK;
}

lgnk_status zero_acc(lgnk_ctx* ctx) {
    CK(cudaMemsetAsync(ctx->acc, 0, ctx->ipad * sizeof(float), ctx->stream));
    return LGNK_OK;
}

// out = addsrc + scale * A_reg x + gamma * x (A_reg the regularizer's operator).
// x must not alias out; addsrc may equal out.
lgnk_status reg_apply(lgnk_ctx* ctx, const float* x, float* out, double scale, double gamma, const float* addsrc) {
    const int kd = ctx->K * ctx->d;
    switch (ctx->prob.regularizer) {
        case LGNK_DIFFUSION:
            KL(launch_laplacian(ctx->d, x, out, ctx->vg, kd, (float)scale, (float)gamma, addsrc, ctx->stream));
            break;
        case LGNK_CURVATURE:
            KL(launch_laplacian(ctx->d, x, ctx->rtmp, ctx->vg, kd, 1.0f, 0.0f, nullptr, ctx->stream));
            KL(launch_laplacian_ext(ctx->d, ctx->rtmp, out, ctx->vg, kd, (float)scale, (float)gamma,
                                    gamma != 0.0 ? x : nullptr, addsrc, ctx->stream));
            break;
        case LGNK_ELASTIC:
            KL(launch_divergence(ctx->d, x, ctx->rtmp, ctx->vg, ctx->K, ctx->stream));
            KL(launch_elastic(ctx->d, x, ctx->rtmp, out, ctx->vg, ctx->K, (float)(scale * ctx->prob.mu_lame),
                              (float)(scale * (ctx->prob.lambda_lame + ctx->prob.mu_lame)), (float)gamma, addsrc,
                              ctx->stream));
            break;
        default:
            SETERR("unknown regularizer");
            return LGNK_ERR_INTERNAL;
    }
    return LGNK_OK;
}

lgnk_status fetch(lgnk_ctx* ctx, int count) {
    CK(cudaMemcpyAsync(ctx->hres, ctx->dres, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LGNK_OK;
}

lgnk_status dot_dev(lgnk_ctx* ctx, const float* a, const float* b, size_t count, int slot) {
    const int nb = dot_blocks(count);
    KL(launch_dot(a, b, count, ctx->partial, nb, ctx->stream));
    KL(launch_reduce(ctx->partial, nb, ctx->dres + slot, ctx->stream));
    return LGNK_OK;
}

lgnk_status dot_host(lgnk_ctx* ctx, const float* a, const float* b, size_t count, double* out) {
    TRY(dot_dev(ctx, a, b, count, 2));
    TRY(fetch(ctx, 3));
    *out = ctx->hres[2];
    if (!std::isfinite(*out)) {
        SETERR("non-finite inner product");
        return LGNK_ERR_NUMERIC;
    }
    return LGNK_OK;
}

// ---- internal operations: velocity already packed in Vp (and template in Tp) ----

lgnk_status forward_packed(lgnk_ctx* ctx, const float* T, float* u1, float* y) {
    TraceArgs a = base_args(ctx);
    a.yout = y;
    if (ctx->prob.model == LGNK_TRANSPORT) {
        a.u1 = u1;
        return trace(ctx, MODE_FWD, a);
    }
    TRY(zero_acc(ctx));
    a.T = T;
    a.acc = ctx->acc;
    TRY(trace(ctx, MODE_FWD, a));
    KL(launch_unpack_image(ctx->acc, u1, ctx->ig, ctx->d, ctx->stream));
    return LGNK_OK;
}

// J, D, S at the packed velocity; v is the same velocity in ABI layout (for S).
// objective_packed in two halves: the device work with the copy of its sums
// to hres[0..1] (no wait), and, once the stream has been synchronized, the
// objective from them.
lgnk_status objective_enqueue(lgnk_ctx* ctx, const float* v, const float* T, const float* R, float* grad) {
    TraceArgs a = base_args(ctx);
    a.R = R;
    a.partial = ctx->partial;
    int nred = trace_blocks_for(ctx, grad != nullptr ? MODE_OBJGRAD : MODE_FWD);
    if (ctx->prob.model == LGNK_TRANSPORT) {
        if (grad != nullptr) {
            TRY(zero_G(ctx));
            TRY(trace(ctx, MODE_OBJGRAD, a));
        } else {
            a.u1 = ctx->itmp;
            TRY(trace(ctx, MODE_FWD, a));
        }
    } else {
        TRY(zero_acc(ctx));
        TraceArgs f = base_args(ctx);
        f.T = T;
        f.acc = ctx->acc;
        TRY(trace(ctx, MODE_FWD, f));
        KL(launch_unpack_image(ctx->acc, ctx->itmp, ctx->ig, ctx->d, ctx->stream));
        nred = residual_blocks(ctx->ig, ctx->d);
        KL(launch_residual(ctx->itmp, R, ctx->rp, ctx->ig, ctx->d, (float)ctx->cellvol, ctx->partial, nred,
                           ctx->stream));
        if (grad != nullptr) {
            TRY(zero_G(ctx));
            TraceArgs b = base_args(ctx);
            b.T = T;
            b.r = ctx->rp;
            TRY(trace(ctx, MODE_JTVP, b));
        }
    }
    KL(launch_reduce(ctx->partial, nred, ctx->dres + 0, ctx->stream));
    if (grad != nullptr) {
        KL(launch_distribute_gradient(ctx->d, ctx->Gp, grad, ctx->vg, ctx->K, ctx->slices, 1.0f, ctx->stream));
        TRY(reg_apply(ctx, v, grad, ctx->prob.alpha * ctx->wreg, 0.0, grad));
    }
    // S = 1/2 dt h_v^d v^T A_reg v
    TRY(reg_apply(ctx, v, ctx->pc0, 1.0, 0.0, nullptr));
    TRY(dot_dev(ctx, v, ctx->pc0, ctx->n, 1));
    CK(cudaMemcpyAsync(ctx->hres, ctx->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return LGNK_OK;
}

lgnk_status objective_collect(lgnk_ctx* ctx, double* J, double* D, double* S) {
    const double Dv = 0.5 * ctx->cellvol * ctx->hres[0];
    const double Sv = 0.5 * ctx->wreg * ctx->hres[1];
    if (!std::isfinite(Dv) || !std::isfinite(Sv)) {
        SETERR("non-finite objective");
        return LGNK_ERR_NUMERIC;
    }
    if (D) *D = Dv;
    if (S) *S = Sv;
    if (J) *J = Dv + ctx->prob.alpha * Sv;
    return LGNK_OK;
}

// J, D, S (and with grad the gradient, Eq. 9) at the packed velocity.
lgnk_status objective_packed(lgnk_ctx* ctx, const float* v, const float* T, const float* R, float* grad,
                             double* J, double* D, double* S) {
    TRY(objective_enqueue(ctx, v, T, R, grad));
    CK(cudaStreamSynchronize(ctx->stream));
    return objective_collect(ctx, J, D, S);
}

// out = J^T h^d J dv + alpha dt h_v^d A dv + gamma dv at the packed velocity.
// The data term of the Gauss-Newton product into the slice gradients Gp
// (the first half of hessvec_packed).
lgnk_status hessvec_accumulate(lgnk_ctx* ctx, const float* T, const float* dv) {
    // packs the direction and zeroes the slice gradients in one pass
    KL(launch_pack_velocity(ctx->d, dv, ctx->dVp, ctx->vg, ctx->K, ctx->slices, ctx->stream, ctx->Gp));
    if (ctx->prob.model == LGNK_TRANSPORT) {
        TraceArgs a = base_args(ctx);
        TRY(trace(ctx, MODE_HESS, a));
    } else {
        TRY(zero_acc(ctx));
        TraceArgs a = base_args(ctx);
        a.T = T;
        a.acc = ctx->acc;
        TRY(trace(ctx, MODE_JVP, a));
        KL(launch_repad_image(ctx->acc, ctx->ig, ctx->d, (float)ctx->cellvol, ctx->stream));
        TraceArgs b = base_args(ctx);
        b.T = T;
        b.r = ctx->acc;
        TRY(trace(ctx, MODE_JTVP, b));
    }
    return LGNK_OK;
}

// out = the distributed slice gradients + the regularizer's term of dv.
lgnk_status hessvec_finish(lgnk_ctx* ctx, const float* dv, float* out) {
    if (ctx->prob.regularizer == LGNK_DIFFUSION) {
        // the slice gradients' distribution, the Laplacian of dv and gamma dv in one pass
        KL(launch_hess_finish(ctx->d, ctx->Gp, dv, out, ctx->vg, ctx->K, ctx->slices, 1.0f,
                              (float)(ctx->prob.alpha * ctx->wreg), (float)ctx->prob.gamma, nullptr, 0, nullptr,
                              nullptr, nullptr, ctx->stream));
        return LGNK_OK;
    }
    KL(launch_distribute_gradient(ctx->d, ctx->Gp, out, ctx->vg, ctx->K, ctx->slices, 1.0f, ctx->stream));
    return reg_apply(ctx, dv, out, ctx->prob.alpha * ctx->wreg, ctx->prob.gamma, out);
}

lgnk_status hessvec_packed(lgnk_ctx* ctx, const float* T, const float* dv, float* out) {
    TRY(hessvec_accumulate(ctx, T, dv));
    return hessvec_finish(ctx, dv, out);
}

EllArgs ell_args(const lgnk_ctx* ctx) {
    EllArgs e{};
    e.vg = ctx->vg;
    e.M = (long long)ctx->M;
    e.ekey = ctx->ekey;
    e.eblk = ctx->eblk;
    e.ecnt = ctx->ecnt;
    e.dV = ctx->dVp;
    e.G = ctx->Gp;
    e.cellvol = (float)ctx->cellvol;
    return e;
}

lgnk_status ell(lgnk_ctx* ctx, int mode, const EllArgs& e) {
    if (ctx->prof) TRY(record_event(ctx));
    KL(launch_ell(ctx->d, mode, e, ctx->stream));
    ctx->trace_launches++;
    if (ctx->prof) TRY(record_event(ctx));
    return LGNK_OK;
}

// Rows of J = d_v u1 at the packed velocity and template (transport).  With
// R: the same trace also yields u1 and the SSD (Eq. 10), and then
// grad = J^T h^d (u1 - R) + alpha dt h_v^d A v is applied through the stored
// rows (one ELL launch instead of a second trace), with J, D, S as in
// objective_packed.  Returns LGNK_ERR_CAPACITY when a row overflows (grad and
// the rows are then not valid).
lgnk_status assemble_enqueue(lgnk_ctx* ctx, const float* v = nullptr, const float* R = nullptr,
                             float* grad = nullptr) {
    ctx->asm_valid = false;
    const int W = asm_capacity(ctx->d);
    const size_t B = ((size_t)1 << ctx->d) * ctx->d;
    if (ctx->eflag == nullptr) {
        TRY(dalloc(ctx, (size_t)W * ctx->M, &ctx->ekey));
        TRY(dalloc(ctx, (size_t)W * B * ctx->M, &ctx->eblk));
        TRY(dalloc(ctx, ctx->M, &ctx->ecnt));
        TRY(dalloc(ctx, 1, &ctx->eflag));
    }
    CK(cudaMemsetAsync(ctx->eflag, 0, sizeof(int), ctx->stream));
    TraceArgs a = base_args(ctx);
    a.ekey = ctx->ekey;
    a.eblk = ctx->eblk;
    a.ecnt = ctx->ecnt;
    a.eflag = ctx->eflag;
    a.ewidth = W;
    a.cpartial = ctx->cpartial;
    if (R != nullptr) {
        a.R = R;
        a.u1 = ctx->itmp;
        a.partial = ctx->partial;
    }
    TRY(trace(ctx, MODE_ASM, a));
    KL(launch_reduce(ctx->cpartial, ctx->trace_blocks, ctx->dres + 7, ctx->stream));
    int nfetch = 0;
    if (R != nullptr) {
        KL(launch_reduce(ctx->partial, ctx->trace_blocks, ctx->dres + 0, ctx->stream));
        // grad = J^T (h^d res) through the rows, then the regularizer
        TRY(zero_G(ctx));
        EllArgs e = ell_args(ctx);
        e.r = ctx->itmp;
        TRY(ell(ctx, ELL_JTVP, e));
        KL(launch_distribute_gradient(ctx->d, ctx->Gp, grad, ctx->vg, ctx->K, ctx->slices, 1.0f, ctx->stream));
        TRY(reg_apply(ctx, v, grad, ctx->prob.alpha * ctx->wreg, 0.0, grad));
        TRY(reg_apply(ctx, v, ctx->pc0, 1.0, 0.0, nullptr));
        TRY(dot_dev(ctx, v, ctx->pc0, ctx->n, 1));
        nfetch = 2;
    }
    CK(cudaMemcpyAsync(ctx->hres + 7, ctx->dres + 7, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hres + 6, ctx->eflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (nfetch) CK(cudaMemcpyAsync(ctx->hres, ctx->dres, nfetch * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return LGNK_OK;
}

// The second half of assemble_packed, after the stream has been synchronized:
// the row capacity check and, with_objective, J, D, S.
lgnk_status assemble_collect(lgnk_ctx* ctx, bool with_objective, double* J = nullptr, double* D = nullptr,
                             double* S = nullptr) {
    const int W = asm_capacity(ctx->d);
    int flag = 0;
    memcpy(&flag, ctx->hres + 6, sizeof(int));
    ctx->asm_entries = (size_t)ctx->hres[7];
    if (flag != 0) {
        SETERR("a characteristic meets more than %d (time slice, velocity cell) pairs: J not assembled", W);
        return LGNK_ERR_CAPACITY;
    }
    ctx->asm_valid = true;
    if (with_objective) {
        const double Dv = 0.5 * ctx->cellvol * ctx->hres[0];
        const double Sv = 0.5 * ctx->wreg * ctx->hres[1];
        if (!std::isfinite(Dv) || !std::isfinite(Sv)) {
            SETERR("non-finite objective");
            return LGNK_ERR_NUMERIC;
        }
        if (D) *D = Dv;
        if (S) *S = Sv;
        if (J) *J = Dv + ctx->prob.alpha * Sv;
    }
    return LGNK_OK;
}

lgnk_status assemble_packed(lgnk_ctx* ctx, const float* v = nullptr, const float* R = nullptr, float* grad = nullptr,
                            double* J = nullptr, double* D = nullptr, double* S = nullptr) {
    TRY(assemble_enqueue(ctx, v, R, grad));
    CK(cudaStreamSynchronize(ctx->stream));
    return assemble_collect(ctx, R != nullptr, J, D, S);
}

lgnk_status hessvec_assembled_accumulate(lgnk_ctx* ctx, const float* dv) {
    KL(launch_pack_velocity(ctx->d, dv, ctx->dVp, ctx->vg, ctx->K, ctx->slices, ctx->stream, ctx->Gp));
    return ell(ctx, ELL_HESS, ell_args(ctx));
}

lgnk_status hessvec_assembled_packed(lgnk_ctx* ctx, const float* dv, float* out) {
    TRY(hessvec_assembled_accumulate(ctx, dv));
    return hessvec_finish(ctx, dv, out);
}

lgnk_status precond_apply(lgnk_ctx* ctx, const float* r, float* z) {
    const int kd = ctx->K * ctx->d;
    cudaStream_t s = ctx->stream;
    if (ctx->vg.m[ctx->d - 1] <= 128) {
        // the last axis's forward transform, scale and inverse transform in one pass
        if (ctx->d == 3 && ctx->vg.m[0] <= 64 && ctx->vg.m[1] <= 64) {
            // y and x of each xy plane in one pass each way: three launches
            const long long planes = (long long)kd * ctx->vg.m[2];
            KL(launch_dct_plane(r, ctx->pc0, ctx->Cf[0], ctx->Cf[1], ctx->vg, planes, s));
            KL(launch_dct_last_fused(ctx->pc0, ctx->pc1, ctx->Cf[2], ctx->Ci[2], ctx->inv_eig, ctx->vg, 3, kd, s));
            KL(launch_dct_plane(ctx->pc1, z, ctx->Ci[0], ctx->Ci[1], ctx->vg, planes, s));
        } else if (ctx->d == 3) {
            KL(launch_dct_axis(r, ctx->pc0, ctx->Cm[0], ctx->Cf[0], ctx->vg, 3, kd, 0, false, s));
            KL(launch_dct_axis(ctx->pc0, ctx->pc1, ctx->Cm[1], ctx->Cf[1], ctx->vg, 3, kd, 1, false, s));
            KL(launch_dct_last_fused(ctx->pc1, ctx->pc0, ctx->Cf[2], ctx->Ci[2], ctx->inv_eig, ctx->vg, 3, kd, s));
            KL(launch_dct_axis(ctx->pc0, ctx->pc1, ctx->Cm[1], ctx->Ci[1], ctx->vg, 3, kd, 1, true, s));
            KL(launch_dct_axis(ctx->pc1, z, ctx->Cm[0], ctx->Ci[0], ctx->vg, 3, kd, 0, true, s));
        } else if (ctx->d == 2 && ctx->vg.m[0] <= 64 && ctx->vg.m[1] <= 64) {
            // the whole transform of each plane in one CTA: one launch
            KL(launch_dct_plane2d(r, z, ctx->Cf[0], ctx->Cf[1], ctx->Ci[0], ctx->Ci[1], ctx->inv_eig, ctx->vg, kd, s));
        } else {
            KL(launch_dct_axis(r, ctx->pc0, ctx->Cm[0], ctx->Cf[0], ctx->vg, 2, kd, 0, false, s));
            KL(launch_dct_last_fused(ctx->pc0, ctx->pc1, ctx->Cf[1], ctx->Ci[1], ctx->inv_eig, ctx->vg, 2, kd, s));
            KL(launch_dct_axis(ctx->pc1, z, ctx->Cm[0], ctx->Ci[0], ctx->vg, 2, kd, 0, true, s));
        }
        return LGNK_OK;
    }
    if (ctx->d == 3) {
        KL(launch_dct_axis(r, ctx->pc0, ctx->Cm[0], ctx->Cf[0], ctx->vg, 3, kd, 0, false, s));
        KL(launch_dct_axis(ctx->pc0, ctx->pc1, ctx->Cm[1], ctx->Cf[1], ctx->vg, 3, kd, 1, false, s));
        KL(launch_dct_axis(ctx->pc1, ctx->pc0, ctx->Cm[2], ctx->Cf[2], ctx->vg, 3, kd, 2, false, s));
        KL(launch_scale_modes(ctx->pc0, ctx->inv_eig, ctx->Mv, ctx->n, s));
        KL(launch_dct_axis(ctx->pc0, ctx->pc1, ctx->Cm[2], ctx->Ci[2], ctx->vg, 3, kd, 2, true, s));
        KL(launch_dct_axis(ctx->pc1, ctx->pc0, ctx->Cm[1], ctx->Ci[1], ctx->vg, 3, kd, 1, true, s));
        KL(launch_dct_axis(ctx->pc0, z, ctx->Cm[0], ctx->Ci[0], ctx->vg, 3, kd, 0, true, s));
    } else {
        KL(launch_dct_axis(r, ctx->pc0, ctx->Cm[0], ctx->Cf[0], ctx->vg, 2, kd, 0, false, s));
        KL(launch_dct_axis(ctx->pc0, ctx->pc1, ctx->Cm[1], ctx->Cf[1], ctx->vg, 2, kd, 1, false, s));
        KL(launch_scale_modes(ctx->pc1, ctx->inv_eig, ctx->Mv, ctx->n, s));
        KL(launch_dct_axis(ctx->pc1, ctx->pc0, ctx->Cm[1], ctx->Ci[1], ctx->vg, 2, kd, 1, true, s));
        KL(launch_dct_axis(ctx->pc0, z, ctx->Cm[0], ctx->Ci[0], ctx->vg, 2, kd, 0, true, s));
    }
    return LGNK_OK;
}

bool distinct(const void* out, std::initializer_list<const void*> ins) {
    for (const void* p : ins)
        if (p != nullptr && p == out) return false;
    return true;
}

}  // namespace

// ---- helpers shared with the allocation-free entry point (static_scratch.cu) ----

const char* lgnk_internal_validate(const lgnk_problem* p) { return validate_problem(p); }

DevGrid lgnk_internal_grid(const lgnk_grid& g) { return make_grid(g); }

void lgnk_internal_set_error(const char* msg) {
    snprintf(g_create_err, sizeof(g_create_err), "%s", msg ? msg : "");
}

#define CHECK_CTX()                                                  \
    do {                                                             \
        if (ctx == nullptr) return LGNK_ERR_INVALID_ARG;             \
    } while (0)
#define REQUIRE(cond, msg)                                           \
    do {                                                             \
        if (!(cond)) {                                               \
            SETERR("%s", msg);                                       \
            return LGNK_ERR_INVALID_ARG;                             \
        }                                                            \
    } while (0)

extern "C" {

const char* lgnk_status_string(lgnk_status s) {
    switch (s) {
        case LGNK_OK: return "ok";
        case LGNK_ERR_INVALID_ARG: return "invalid argument";
        case LGNK_ERR_OOM: return "out of memory (budget or device)";
        case LGNK_ERR_CUDA: return "CUDA error";
        case LGNK_ERR_NUMERIC: return "non-finite value";
        case LGNK_ERR_INTERNAL: return "internal error";
        case LGNK_LS_FAILED: return "line search failed";
        case LGNK_NOT_CONVERGED: return "not converged (iteration cap)";
        case LGNK_ERR_CAPACITY: return "a fixed capacity was exceeded";
    }
    return "unknown status";
}

const char* lgnk_last_error(const lgnk_ctx* ctx) {
    return ctx == nullptr ? g_create_err : ctx->err;
}

size_t lgnk_scratch_bytes(const lgnk_ctx* ctx) {
    return ctx == nullptr ? 0 : ctx->used;
}

void lgnk_destroy(lgnk_ctx* ctx) {
    if (ctx == nullptr) return;
    for (int i = 0; i < 2; ++i) {   // before the stream and the buffers they use
        ctx->pcg_loops[i].reset();
        ctx->pcg_graphs[i].reset();
    }
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    if (ctx->ev_enter) cudaEventDestroy(ctx->ev_enter);
    if (ctx->ev_leave) cudaEventDestroy(ctx->ev_leave);
    if (ctx->solve_stream) cudaStreamDestroy(ctx->solve_stream);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->hres) cudaFreeHost(ctx->hres);
    if (ctx->hpin) cudaFreeHost(ctx->hpin);
    delete ctx;
}

lgnk_status lgnk_set_stream(lgnk_ctx* ctx, void* stream) {
    CHECK_CTX();
    ctx->stream = static_cast<cudaStream_t>(stream);
    return LGNK_OK;
}

lgnk_status lgnk_create(const lgnk_problem* prob, void* stream, size_t mem_budget, lgnk_ctx** out) {
    g_create_err[0] = 0;
    if (out == nullptr) return LGNK_ERR_INVALID_ARG;
    *out = nullptr;
    if (const char* e = validate_problem(prob)) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", e);
        return LGNK_ERR_INVALID_ARG;
    }
    lgnk_ctx* ctx = new (std::nothrow) lgnk_ctx();
    if (ctx == nullptr) return LGNK_ERR_OOM;
    ctx->prob = *prob;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->budget = mem_budget;
    const int d = prob->image.d;
    ctx->d = d;
    ctx->K = prob->time_nodes;
    ctx->N = prob->rk4_steps;
    ctx->ig = make_grid(prob->image);
    ctx->vg = make_grid(prob->velocity);
    ctx->M = (size_t)ctx->ig.m[0] * ctx->ig.m[1] * ctx->ig.m[2];
    ctx->Mv = (size_t)ctx->vg.m[0] * ctx->vg.m[1] * ctx->vg.m[2];
    ctx->n = ctx->Mv * d * ctx->K;
    ctx->ipad = (size_t)ctx->ig.mp[0] * ctx->ig.mp[1] * ctx->ig.mp[2];
    ctx->vpad = (size_t)ctx->vg.mp[0] * ctx->vg.mp[1] * ctx->vg.mp[2];
    ctx->vt_bytes = d == 3 ? 16 : 8;
    {
        int ts[3];
        trace_tile_shape(d, ts);
        for (int i = 0; i < 3; ++i) ctx->tiles[i] = (ctx->ig.m[i] + ts[i] - 1) / ts[i];
        ctx->trace_blocks = ctx->tiles[0] * ctx->tiles[1] * ctx->tiles[2];
    }
    double hv = 1.0, hi = 1.0;
    for (int a = 0; a < d; ++a) {
        hi *= (prob->image.hi[a] - prob->image.lo[a]) / prob->image.m[a];
        hv *= (prob->velocity.hi[a] - prob->velocity.lo[a]) / prob->velocity.m[a];
    }
    ctx->cellvol = hi;
    ctx->wreg = (ctx->K == 1 ? 1.0 : 1.0 / (ctx->K - 1)) * hv;

    auto fail = [&](lgnk_status s) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", ctx->err[0] ? ctx->err : lgnk_status_string(s));
        lgnk_destroy(ctx);
        return s;
    };
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(LGNK_ERR_CUDA);
    }
    {
        const bool transport = prob->model == LGNK_TRANSPORT;
        make_slice_table(ctx->K, ctx->N, transport ? 1.0 : 0.0, (transport ? -1.0 : 1.0) / ctx->N, &ctx->slices);
    }
    const size_t vbytes = ctx->vpad * ctx->slices.n * ctx->vt_bytes;
    const size_t pbytes = ctx->vpad * ctx->slices.n * velocity_pair_bytes(d);
    lgnk_status s;
    if ((s = dev_alloc(ctx, pbytes, &ctx->Vp)) != LGNK_OK) return fail(s);
    if ((s = dev_alloc(ctx, pbytes, &ctx->dVp)) != LGNK_OK) return fail(s);
    if ((s = dev_alloc(ctx, vbytes, &ctx->Gp)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, ctx->ipad, &ctx->Tp)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, ctx->ipad, &ctx->acc)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, ctx->M, &ctx->itmp)) != LGNK_OK) return fail(s);
    if (prob->model == LGNK_CONTINUITY) {
        if ((s = dalloc(ctx, ctx->ipad, &ctx->rp)) != LGNK_OK) return fail(s);
    }
    if ((s = dalloc(ctx, ctx->n, &ctx->rtmp)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, ctx->n, &ctx->pc0)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, ctx->n, &ctx->pc1)) != LGNK_OK) return fail(s);
    for (int a = 0; a < d; ++a) {
        const size_t m = (size_t)ctx->vg.m[a], P = (m + 3) & ~(size_t)3;
        if ((s = dalloc(ctx, m * m, &ctx->Cm[a])) != LGNK_OK) return fail(s);
        if ((s = dalloc(ctx, m * P, &ctx->Cf[a])) != LGNK_OK) return fail(s);
        if ((s = dalloc(ctx, m * P, &ctx->Ci[a])) != LGNK_OK) return fail(s);
    }
    if ((s = dalloc(ctx, ctx->Mv, &ctx->inv_eig)) != LGNK_OK) return fail(s);
    // per-block partials: a trace's blocks, or two per reduction block (two inner
    // products in one launch; the min and max of det grad y)
    ctx->npartial = std::max(ctx->trace_blocks, 2 * reduce_block_cap());
    if ((s = dalloc(ctx, (size_t)ctx->npartial, &ctx->partial)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, (size_t)ctx->trace_blocks, &ctx->cpartial)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, 16, &ctx->dres)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, 4, &ctx->fsc)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, 1, &ctx->dcounter)) != LGNK_OK) return fail(s);
    if ((s = dalloc(ctx, 4, &ctx->dctl)) != LGNK_OK) return fail(s);
    if (cudaMallocHost((void**)&ctx->hpin, 64) != cudaSuccess) {
        cudaGetLastError();
        ctx->hpin = nullptr;
        return fail(LGNK_ERR_OOM);
    }
    if (cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned), ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(LGNK_ERR_CUDA);
    }
    if (cudaMallocHost((void**)&ctx->hres, 16 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        ctx->hres = nullptr;
        return fail(LGNK_ERR_OOM);
    }

    // Spectral preconditioner tables (Sec. 3.2): orthonormal DCT-II per axis and
    // the inverse eigenvalues of alpha dt h_v^d A_reg + gamma I.
    std::vector<float> hostC;
    for (int a = 0; a < d; ++a) {
        const int m = ctx->vg.m[a];
        hostC.assign((size_t)m * m, 0.0f);
        for (int k = 0; k < m; ++k)
            for (int i = 0; i < m; ++i)
                hostC[(size_t)k * m + i] =
                    (float)(std::sqrt((k == 0 ? 1.0 : 2.0) / m) * std::cos(M_PI * k * (2 * i + 1) / (2.0 * m)));
        if (cudaMemcpy(ctx->Cm[a], hostC.data(), hostC.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(LGNK_ERR_CUDA);
        const size_t P = ((size_t)m + 3) & ~(size_t)3;
        std::vector<float> hf((size_t)m * P, 0.0f), hi((size_t)m * P, 0.0f);
        for (int q = 0; q < m; ++q)
            for (int k = 0; k < m; ++k) {
                hf[(size_t)q * P + k] = hostC[(size_t)k * m + q];
                hi[(size_t)q * P + k] = hostC[(size_t)q * m + k];
            }
        if (cudaMemcpy(ctx->Cf[a], hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->Ci[a], hi.data(), hi.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(LGNK_ERR_CUDA);
    }
    std::vector<double> pv(ctx->Mv);
    const double wa = prob->alpha * ctx->wreg;
    double pmin = 0.0;
    for (size_t sidx = 0; sidx < ctx->Mv; ++sidx) {
        size_t r = sidx;
        double lam = 0.0;
        for (int a = 0; a < d; ++a) {
            const int m = prob->velocity.m[a];
            const int k = (int)(r % m);
            r /= m;
            const double h = (prob->velocity.hi[a] - prob->velocity.lo[a]) / m;
            lam += (2.0 - 2.0 * std::cos(M_PI * k / m)) / (h * h);
        }
        if (prob->regularizer == LGNK_CURVATURE) lam = lam * lam;
        if (prob->regularizer == LGNK_ELASTIC) lam = prob->mu_lame * lam;
        pv[sidx] = wa * lam + prob->gamma;
        if (pv[sidx] > 0.0 && (pmin == 0.0 || pv[sidx] < pmin)) pmin = pv[sidx];
    }
    // a zero eigenvalue (gamma = 0: the constant mode) takes the smallest nonzero one
    std::vector<float> ev(ctx->Mv);
    for (size_t sidx = 0; sidx < ctx->Mv; ++sidx) {
        const double p = pv[sidx] > 0.0 ? pv[sidx] : (pmin > 0.0 ? pmin : 1.0);
        ev[sidx] = (float)(1.0 / p);
    }
    if (cudaMemcpy(ctx->inv_eig, ev.data(), ev.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(LGNK_ERR_CUDA);
    if (ctx->rp && cudaMemset(ctx->rp, 0, ctx->ipad * sizeof(float)) != cudaSuccess) return fail(LGNK_ERR_CUDA);
    *out = ctx;
    return LGNK_OK;
}

lgnk_status lgnk_forward(lgnk_ctx* ctx, const float* v, const float* T, float* u1, float* y) {
    CHECK_CTX();
    REQUIRE(v && T && u1, "v, T and u1 must be non-NULL");
    REQUIRE(distinct(u1, {v, T}) && distinct(y, {v, T, u1}), "outputs must not alias inputs");
    TRY(pack_v(ctx, v, ctx->Vp));
    if (ctx->prob.model == LGNK_TRANSPORT) TRY(pack_T(ctx, T));
    return forward_packed(ctx, T, u1, y);
}

lgnk_status lgnk_jvp(lgnk_ctx* ctx, const float* v, const float* T, const float* dv, float* du) {
    CHECK_CTX();
    REQUIRE(v && T && dv && du, "v, T, dv and du must be non-NULL");
    REQUIRE(distinct(du, {v, T, dv}), "outputs must not alias inputs");
    TRY(pack_v(ctx, v, ctx->Vp));
    TRY(pack_v(ctx, dv, ctx->dVp));
    TraceArgs a = base_args(ctx);
    if (ctx->prob.model == LGNK_TRANSPORT) {
        TRY(pack_T(ctx, T));
        a.u1 = du;
        return trace(ctx, MODE_JVP, a);
    }
    TRY(zero_acc(ctx));
    a.T = T;
    a.acc = ctx->acc;
    TRY(trace(ctx, MODE_JVP, a));
    KL(launch_unpack_image(ctx->acc, du, ctx->ig, ctx->d, ctx->stream));
    return LGNK_OK;
}

lgnk_status lgnk_jtvp(lgnk_ctx* ctx, const float* v, const float* T, const float* r, float* gv) {
    CHECK_CTX();
    REQUIRE(v && T && r && gv, "v, T, r and gv must be non-NULL");
    REQUIRE(distinct(gv, {v, T, r}), "outputs must not alias inputs");
    TRY(pack_v(ctx, v, ctx->Vp));
    TRY(zero_G(ctx));
    TraceArgs a = base_args(ctx);
    if (ctx->prob.model == LGNK_TRANSPORT) {
        TRY(pack_T(ctx, T));
        a.r = r;
    } else {
        KL(launch_pack_image(r, ctx->rp, ctx->ig, ctx->d, 1.0f, ctx->stream));
        a.T = T;
        a.r = ctx->rp;
    }
    TRY(trace(ctx, MODE_JTVP, a));
    KL(launch_distribute_gradient(ctx->d, ctx->Gp, gv, ctx->vg, ctx->K, ctx->slices, 1.0f, ctx->stream));
    return LGNK_OK;
}

lgnk_status lgnk_objective(lgnk_ctx* ctx, const float* v, const float* T, const float* R, double* J, double* D,
                           double* S, float* grad) {
    CHECK_CTX();
    REQUIRE(v && T && R, "v, T and R must be non-NULL");
    REQUIRE(distinct(grad, {v, T, R}), "outputs must not alias inputs");
    TRY(pack_v(ctx, v, ctx->Vp));
    if (ctx->prob.model == LGNK_TRANSPORT) TRY(pack_T(ctx, T));
    return objective_packed(ctx, v, T, R, grad, J, D, S);
}

lgnk_status lgnk_hessvec(lgnk_ctx* ctx, const float* v, const float* T, const float* dv, float* Hdv) {
    CHECK_CTX();
    REQUIRE(v && T && dv && Hdv, "v, T, dv and Hdv must be non-NULL");
    REQUIRE(distinct(Hdv, {v, T, dv}), "outputs must not alias inputs");
    TRY(pack_v(ctx, v, ctx->Vp));
    if (ctx->prob.model == LGNK_TRANSPORT) TRY(pack_T(ctx, T));
    return hessvec_packed(ctx, T, dv, Hdv);
}

lgnk_status lgnk_assemble(lgnk_ctx* ctx, const float* v, const float* T, size_t* blocks) {
    CHECK_CTX();
    ctx->asm_valid = false;
    REQUIRE(v && T, "v and T must be non-NULL");
    REQUIRE(ctx->prob.model == LGNK_TRANSPORT, "J is assembled for the transport model only");
    TRY(pack_v(ctx, v, ctx->Vp));
    TRY(pack_T(ctx, T));
    TRY(assemble_packed(ctx));
    if (blocks) *blocks = ctx->asm_entries;
    return LGNK_OK;
}

lgnk_status lgnk_jvp_assembled(lgnk_ctx* ctx, const float* dv, float* du) {
    CHECK_CTX();
    REQUIRE(dv && du && (const void*)dv != (const void*)du, "dv and du must be non-NULL and distinct");
    REQUIRE(ctx->asm_valid, "no assembled J on this context (call lgnk_assemble)");
    TRY(pack_v(ctx, dv, ctx->dVp));
    EllArgs e = ell_args(ctx);
    e.out = du;
    return ell(ctx, ELL_JVP, e);
}

lgnk_status lgnk_jtvp_assembled(lgnk_ctx* ctx, const float* r, float* gv) {
    CHECK_CTX();
    REQUIRE(r && gv && (const void*)r != (const void*)gv, "r and gv must be non-NULL and distinct");
    REQUIRE(ctx->asm_valid, "no assembled J on this context (call lgnk_assemble)");
    TRY(zero_G(ctx));
    EllArgs e = ell_args(ctx);
    e.r = r;
    TRY(ell(ctx, ELL_JTVP, e));
    KL(launch_distribute_gradient(ctx->d, ctx->Gp, gv, ctx->vg, ctx->K, ctx->slices, 1.0f, ctx->stream));
    return LGNK_OK;
}

lgnk_status lgnk_hessvec_assembled(lgnk_ctx* ctx, const float* dv, float* Hdv) {
    CHECK_CTX();
    REQUIRE(dv && Hdv && (const void*)dv != (const void*)Hdv, "dv and Hdv must be non-NULL and distinct");
    REQUIRE(ctx->asm_valid, "no assembled J on this context (call lgnk_assemble)");
    return hessvec_assembled_packed(ctx, dv, Hdv);
}

lgnk_status lgnk_jacobian_determinant(lgnk_ctx* ctx, const float* v, const float* T, float* det, double* det_min,
                                      double* det_max) {
    CHECK_CTX();
    REQUIRE(v && T, "v and T must be non-NULL");
    REQUIRE(distinct(det, {v, T}), "det must not alias the inputs");
    if (ctx->ybuf == nullptr) TRY(dalloc(ctx, ctx->M * ctx->d, &ctx->ybuf));
    TRY(pack_v(ctx, v, ctx->Vp));
    if (ctx->prob.model == LGNK_TRANSPORT) TRY(pack_T(ctx, T));
    TRY(forward_packed(ctx, T, ctx->itmp, ctx->ybuf));
    KL(launch_jacobian_det(ctx->d, ctx->ybuf, det, ctx->ig, ctx->partial, ctx->dres + 4, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hres + 4, ctx->dres + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (det_min) *det_min = ctx->hres[4];
    if (det_max) *det_max = ctx->hres[5];
    return LGNK_OK;
}

lgnk_status lgnk_precond(lgnk_ctx* ctx, const float* r, float* z) {
    CHECK_CTX();
    REQUIRE(r && z, "r and z must be non-NULL");
    return precond_apply(ctx, r, z);
}

lgnk_status lgnk_dot(lgnk_ctx* ctx, const float* a, const float* b, size_t count, double* out) {
    CHECK_CTX();
    REQUIRE(a && b && out, "a, b and out must be non-NULL");
    if (count == 0) {
        *out = 0.0;
        return LGNK_OK;
    }
    return dot_host(ctx, a, b, count, out);
}

lgnk_status lgnk_profile(lgnk_ctx* ctx, int enable) {
    CHECK_CTX();
    ctx->prof = enable != 0;
    ctx->ev_used = 0;
    ctx->launches = 0;
    ctx->trace_launches = 0;
    return LGNK_OK;
}

lgnk_status lgnk_profile_read(lgnk_ctx* ctx, double* trace_ms, long long* trace_launches,
                              long long* kernel_launches) {
    CHECK_CTX();
    CK(cudaStreamSynchronize(ctx->stream));
    double total = 0.0;
    for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
        total += ms;
    }
    if (trace_ms) *trace_ms = total;
    if (trace_launches) *trace_launches = ctx->trace_launches;
    if (kernel_launches) *kernel_launches = ctx->launches;
    return LGNK_OK;
}

void lgnk_solve_opts_default(lgnk_solve_opts* o) {
    if (o == nullptr) return;
    o->max_gn = 10;
    o->gn_grad_rtol = 1e-3;
    o->max_pcg = 50;
    o->pcg_rtol = 0.1;
    o->armijo_c = 1e-4;
    o->max_ls = 10;
    o->precond = 1;
    o->verbosity = 0;
    o->gn_grad_atol = 0.0;
    o->matvec = 1;
}

lgnk_status solve_impl(lgnk_ctx* ctx, const float* T, const float* R, float* v, const lgnk_solve_opts& o,
                       lgnk_solve_report* rep_out) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!ctx->have_solve) {
        for (int i = 0; i < 7; ++i) TRY(dalloc(ctx, ctx->n, &ctx->sv[i]));
        ctx->have_solve = true;
    }
    float *x = ctx->sv[0], *r = ctx->sv[1], *z = ctx->sv[2], *p = ctx->sv[3], *Hp = ctx->sv[4], *g = ctx->sv[5],
          *vt = ctx->sv[6];
    const size_t n = ctx->n;
    cudaStream_t s = ctx->stream;
    lgnk_solve_report rep;
    memset(&rep, 0, sizeof(rep));

    if (ctx->prob.model == LGNK_TRANSPORT) TRY(pack_T(ctx, T));
    TRY(pack_v(ctx, v, ctx->Vp));
    double J, D, S;
    // With the assembled J (transport), one trace per accepted iterate yields
    // the objective, the rows of J and, through them, the gradient; the PCG
    // of the next GN step then reuses the rows.  Rows that do not fit (a
    // capacity overflow, or no memory for them) fall back to the matrix-free
    // products; no memory stops further attempts.
    bool asm_off = !(o.matvec == 1 && ctx->prob.model == LGNK_TRANSPORT);
    bool use_asm = false;
    auto obj_grad = [&](const float* vv) -> lgnk_status {
        use_asm = false;
        if (!asm_off) {
            const lgnk_status as = assemble_packed(ctx, vv, R, g, &J, &D, &S);
            if (as == LGNK_OK) {
                use_asm = true;
                return LGNK_OK;
            }
            if (as != LGNK_ERR_CAPACITY && as != LGNK_ERR_OOM) return as;
            asm_off = as == LGNK_ERR_OOM;
        }
        return objective_packed(ctx, vv, T, R, g, &J, &D, &S);
    };
    TRY(obj_grad(v));
    rep.objective_evals = 1;
    double gg;
    TRY(dot_host(ctx, g, g, n, &gg));
    const double g0 = std::sqrt(gg);
    rep.J0 = J;
    rep.g0 = g0;
    lgnk_status status = LGNK_NOT_CONVERGED;
    double gn = g0;
    for (int it = 0; it < o.max_gn; ++it) {
        if (gn <= o.gn_grad_rtol * g0 || gn <= o.gn_grad_atol) {
            status = LGNK_OK;
            break;
        }
        if (use_asm) rep.assembled_gn++;
        // PCG on H x = -g from x = 0 (Eq. 11)
        CK(cudaMemsetAsync(x, 0, n * sizeof(float), s));
        KL(launch_add_scaled(r, g, -1.0f, g, 0.0f, n, s));
        if (o.precond) TRY(precond_apply(ctx, r, z));
        else CK(cudaMemcpyAsync(z, r, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(p, z, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        // The step lengths stay on the device (dres[5] = r.z, fsc = alpha,
        // -alpha, beta); the host reads p.Hp and r.r once per iteration for
        // the curvature and stopping tests, after the next direction is
        // already enqueued.
        const int nb = dot_blocks(n);
        TRY(dot_dev(ctx, r, z, n, 5));
        // CUDA graphs need a capturable stream and no per-launch profiling events
        const bool use_graphs = !ctx->prof && s == ctx->solve_stream && s != nullptr;
        // the device work of one iteration; ends with p.Hp and r.r in hres[2], hres[3]
        // with the diffusion regularizer, the end of the product, p.Hp and alpha are one kernel
        const bool fused_finish = ctx->prob.regularizer == LGNK_DIFFUSION;
        auto body = [&](bool readback) -> lgnk_status {
            TRY(use_asm ? hessvec_assembled_accumulate(ctx, p) : hessvec_accumulate(ctx, T, p));
            if (fused_finish) {
                KL(launch_hess_finish(ctx->d, ctx->Gp, p, Hp, ctx->vg, ctx->K, ctx->slices, 1.0f,
                                      (float)(ctx->prob.alpha * ctx->wreg), (float)ctx->prob.gamma, ctx->partial, nb,
                                      ctx->dcounter, ctx->dres, ctx->fsc, s));
            } else {
                TRY(hessvec_finish(ctx, p, Hp));
                KL(launch_dot_fused(p, Hp, nullptr, n, ctx->partial, nb, ctx->dcounter, ctx->dres, 2, 2, 0, ctx->fsc,
                                    s));
            }
            KL(launch_pcg_update_xr(x, p, r, Hp, ctx->fsc, n, s));
            if (o.precond) TRY(precond_apply(ctx, r, z));
            else CK(cudaMemcpyAsync(z, r, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
            KL(launch_dot_fused(r, r, z, n, ctx->partial, nb, ctx->dcounter, ctx->dres, 3, 4, 1, ctx->fsc, s));
            KL(launch_axpby_dev(1.0f, nullptr, z, 0.0f, ctx->fsc + 2, p, n, s));
            if (readback) CK(cudaMemcpyAsync(ctx->hres, ctx->dres, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
            return LGNK_OK;
        };
        PcgGraph& gr = ctx->pcg_graphs[use_asm ? 1 : 0];
        PcgLoopGraph& lg = ctx->pcg_loops[use_asm ? 1 : 0];
        PcgGraphKey key;
        key.precond = o.precond ? 1 : 0;
        key.T = use_asm ? nullptr : T;
        if (!(lg.key == key)) {
            lg.reset();
            lg.key = key;
        }
        if (!(gr.key == key)) {
            gr.reset();
            gr.key = key;
        }
        int pit = 0;
        bool pcg_pending = false;
        if (use_graphs && lg.exec == nullptr && !lg.failed) {
            // build the loop graph; any failure falls back to one graph per iteration
            const long long l0 = ctx->launches, t0 = ctx->trace_launches;
            cudaGraphConditionalHandle handle = 0;
            bool ok = cudaGraphCreate(&lg.graph, 0) == cudaSuccess;
            ok = ok && cudaGraphConditionalHandleCreate(&handle, lg.graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
            cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};   // the rest zero
            np.conditional.handle = handle;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            ok = ok && cudaGraphAddNode(&node, lg.graph, nullptr, nullptr, 0, &np) == cudaSuccess;
            if (ok) {
                ok = cudaStreamBeginCaptureToGraph(s, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    bool bok = body(false) == LGNK_OK;
                    if (bok) {
                        ctx->launches++;
                        bok = launch_pcg_control(ctx->dres, ctx->dctl, handle, s) == cudaSuccess;
                    }
                    cudaGraph_t captured = nullptr;
                    ok = (cudaStreamEndCapture(s, &captured) == cudaSuccess) && bok;
                }
            }
            ok = ok && cudaGraphInstantiate(&lg.exec, lg.graph, 0) == cudaSuccess;
            cudaGetLastError();
            lg.launches = ctx->launches - l0;
            lg.trace_launches = ctx->trace_launches - t0;
            ctx->launches = l0;
            ctx->trace_launches = t0;
            if (!ok) {
                if (lg.exec) cudaGraphExecDestroy(lg.exec);
                lg.exec = nullptr;
                lg.failed = true;
                ctx->err[0] = 0;
            }
        }
        if (lg.exec != nullptr) {
            int* hc = reinterpret_cast<int*>(ctx->hpin);
            double* htol = reinterpret_cast<double*>(ctx->hpin + 32);
            hc[0] = 0;
            hc[1] = 0;
            hc[2] = 0;
            hc[3] = o.max_pcg;
            *htol = o.pcg_rtol * gn;
            CK(cudaMemcpyAsync(ctx->dctl, hc, 4 * sizeof(int), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(ctx->dres + 6, htol, sizeof(double), cudaMemcpyHostToDevice, s));
            CK(cudaGraphLaunch(lg.exec, s));
            KL(launch_pcg_curvature_fix(x, z, ctx->dctl, n, s));
            ctx->launches++;
            CK(cudaMemcpyAsync(hc, ctx->dctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
            pcg_pending = true;     // the loop's counters are read at the line search's wait
        }
        for (int i = 1; lg.exec == nullptr && i <= o.max_pcg; ++i) {
            if (use_graphs && gr.exec == nullptr && !gr.failed) {
                // capture; any failure ends the capture and falls back to direct launches
                const long long l0 = ctx->launches, t0 = ctx->trace_launches;
                cudaGraph_t graph = nullptr;
                bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    ok = body(true) == LGNK_OK;
                    ok = (cudaStreamEndCapture(s, &graph) == cudaSuccess) && ok && graph != nullptr;
                }
                if (ok) ok = cudaGraphInstantiate(&gr.exec, graph, 0) == cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                gr.launches = ctx->launches - l0;
                gr.trace_launches = ctx->trace_launches - t0;
                ctx->launches = l0;
                ctx->trace_launches = t0;
                if (!ok) {
                    if (gr.exec) cudaGraphExecDestroy(gr.exec);
                    gr.exec = nullptr;
                    gr.failed = true;
                    ctx->err[0] = 0;
                }
            }
            if (gr.exec != nullptr) {
                CK(cudaGraphLaunch(gr.exec, s));
                ctx->launches += gr.launches;
                ctx->trace_launches += gr.trace_launches;
            } else {
                TRY(body(true));
            }
            CK(cudaStreamSynchronize(s));
            rep.hessvecs++;
            const double pHp = ctx->hres[2], rr = ctx->hres[3];
            if (!std::isfinite(pHp) || !std::isfinite(rr)) {
                SETERR("non-finite inner product in PCG");
                return LGNK_ERR_NUMERIC;
            }
            if (!(pHp > 0.0)) {     // alpha was 0: x and r are unchanged
                if (pit == 0) CK(cudaMemcpyAsync(x, z, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
                break;
            }
            pit = i;
            if (std::sqrt(rr) <= o.pcg_rtol * gn) break;
        }
        // Armijo backtracking on v + mu x (FP64 comparisons).  The full step
        // mu = 1 is evaluated first together with what an accepted step needs
        // next: its gradient (and, with the assembled J, the rows at v + x),
        // whose objective is the trial's, bit for bit (the same trace and
        // sums).  The slope g.x, the new |g|^2 and the PCG loop's counters
        // come back with it in one wait.  Shorter steps, when the full one is
        // rejected, are forward traces as before, and the gradient is then
        // evaluated at the accepted point.
        TRY(dot_dev(ctx, g, x, n, 8));
        KL(launch_add_scaled(vt, v, 1.0f, x, 1.0f, n, s));
        TRY(pack_v(ctx, vt, ctx->Vp));
        bool spec_asm = false;
        if (!asm_off) {
            const lgnk_status es = assemble_enqueue(ctx, vt, R, g);
            if (es == LGNK_OK) spec_asm = true;
            else if (es != LGNK_ERR_OOM) return es;
            else asm_off = true;
        }
        if (!spec_asm) TRY(objective_enqueue(ctx, vt, T, R, g));
        TRY(dot_dev(ctx, g, g, n, 9));
        CK(cudaMemcpyAsync(ctx->hres + 8, ctx->dres + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (pcg_pending) {
            int* hc = reinterpret_cast<int*>(ctx->hpin);
            const int its = hc[0];
            rep.hessvecs += its;
            ctx->launches += its * lg.launches;
            ctx->trace_launches += its * lg.trace_launches;
            if (hc[2] == 2) {
                SETERR("non-finite inner product in PCG");
                return LGNK_ERR_NUMERIC;
            }
            pit = hc[1];
        }
        rep.pcg_iters += pit;
        const double slope = ctx->hres[8];
        double Jt = J, Dt = D, St = S, ggt = ctx->hres[9];
        bool spec_rows = spec_asm;
        if (spec_asm) {
            const lgnk_status cs = assemble_collect(ctx, true, &Jt, &Dt, &St);
            if (cs != LGNK_OK) {
                if (cs != LGNK_ERR_CAPACITY && cs != LGNK_ERR_OOM) return cs;
                // rows that do not fit: the matrix-free gradient at v + x
                spec_rows = false;
                TRY(objective_packed(ctx, vt, T, R, g, &Jt, &Dt, &St));
                TRY(dot_host(ctx, g, g, n, &ggt));
            }
        } else {
            TRY(objective_collect(ctx, &Jt, &Dt, &St));
        }
        rep.objective_evals++;
        double mu = 1.0;
        bool accepted = Jt <= J + o.armijo_c * mu * slope;
        for (int ls = 1; !accepted && ls < o.max_ls; ++ls) {
            mu *= 0.5;
            KL(launch_add_scaled(vt, v, 1.0f, x, (float)mu, n, s));
            TRY(pack_v(ctx, vt, ctx->Vp));
            TRY(objective_packed(ctx, vt, T, R, nullptr, &Jt, nullptr, nullptr));
            rep.objective_evals++;
            accepted = Jt <= J + o.armijo_c * mu * slope;
        }
        rep.gn_iters = it + 1;
        if (!accepted) {
            TRY(pack_v(ctx, v, ctx->Vp));
            ctx->asm_valid = false;     // rows (if any) of the rejected full step
            status = LGNK_LS_FAILED;
            break;
        }
        CK(cudaMemcpyAsync(v, vt, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        rep.last_mu = mu;
        if (mu == 1.0) {
            J = Jt;
            D = Dt;
            S = St;
            use_asm = spec_rows;
            gg = ggt;
        } else {
            TRY(obj_grad(v));
            rep.objective_evals++;
            TRY(dot_host(ctx, g, g, n, &gg));
        }
        gn = std::sqrt(gg);
        if (o.verbosity > 0)
            fprintf(stderr, "lgnk GN %3d  J %.6e  D %.6e  S %.6e  |g|/|g0| %.3e  pcg %d  mu %.3g\n", it + 1, J, D,
                    S, gn / g0, pit, mu);
    }
    if (status == LGNK_NOT_CONVERGED && (gn <= o.gn_grad_rtol * g0 || gn <= o.gn_grad_atol)) status = LGNK_OK;
    CK(cudaStreamSynchronize(s));
    rep.J = J;
    rep.D = D;
    rep.S = S;
    rep.g = gn;
    rep.status = status;
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (rep_out) *rep_out = rep;
    return status;
}

lgnk_status lgnk_solve(lgnk_ctx* ctx, const float* T, const float* R, float* v, const lgnk_solve_opts* opts_in,
                       lgnk_solve_report* rep_out) {
    CHECK_CTX();
    REQUIRE(T && R && v, "T, R and v_inout must be non-NULL");
    REQUIRE(distinct(v, {T, R}), "v_inout must not alias T or R");
    lgnk_solve_opts o;
    lgnk_solve_opts_default(&o);
    if (opts_in) o = *opts_in;
    REQUIRE(o.max_gn >= 0 && o.max_pcg >= 1 && o.max_ls >= 1 && o.pcg_rtol > 0.0 && o.gn_grad_rtol >= 0.0 &&
                o.gn_grad_atol >= 0.0 && (o.matvec == 0 || o.matvec == 1),
            "invalid solve options");
    if (ctx->solve_stream == nullptr) {
        CK(cudaStreamCreateWithFlags(&ctx->solve_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->ev_enter, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_leave, cudaEventDisableTiming));
    }
    // run on the context's own stream, after the caller's pending work; the
    // caller's stream waits for everything the solve enqueued, also on error
    cudaStream_t user = ctx->stream;
    CK(cudaEventRecord(ctx->ev_enter, user));
    CK(cudaStreamWaitEvent(ctx->solve_stream, ctx->ev_enter, 0));
    ctx->stream = ctx->solve_stream;
    const lgnk_status st = solve_impl(ctx, T, R, v, o, rep_out);
    ctx->stream = user;
    CK(cudaEventRecord(ctx->ev_leave, ctx->solve_stream));
    CK(cudaStreamWaitEvent(user, ctx->ev_leave, 0));
    return st;
}

lgnk_status lgnk_restrict_image(const lgnk_grid* fine, const float* F, float* C, void* stream) {
    g_create_err[0] = 0;
    if (fine == nullptr || F == nullptr || C == nullptr || F == C) {
        snprintf(g_create_err, sizeof(g_create_err), "fine grid, F and C must be non-NULL and distinct");
        return LGNK_ERR_INVALID_ARG;
    }
    const int d = fine->d;
    if (d != 2 && d != 3) return LGNK_ERR_INVALID_ARG;
    if (const char* e = validate_grid(*fine, d)) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", e);
        return LGNK_ERR_INVALID_ARG;
    }
    lgnk_grid cgr = *fine;
    for (int a = 0; a < d; ++a) {
        if (fine->m[a] % 2 != 0) {
            snprintf(g_create_err, sizeof(g_create_err), "cell counts must be even to coarsen");
            return LGNK_ERR_INVALID_ARG;
        }
        cgr.m[a] = fine->m[a] / 2;
    }
    const cudaError_t e = launch_restrict_image(d, F, C, make_grid(cgr), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", cudaGetErrorString(e));
        return LGNK_ERR_CUDA;
    }
    return LGNK_OK;
}

lgnk_status lgnk_prolong_velocity(const lgnk_grid* coarse, const lgnk_grid* fine, int time_nodes, const float* vc,
                                  float* vf, void* stream) {
    g_create_err[0] = 0;
    if (coarse == nullptr || fine == nullptr || vc == nullptr || vf == nullptr || vc == vf || time_nodes < 1 ||
        coarse->d != fine->d || (coarse->d != 2 && coarse->d != 3)) {
        snprintf(g_create_err, sizeof(g_create_err), "invalid prolongation arguments");
        return LGNK_ERR_INVALID_ARG;
    }
    const char* e1 = validate_grid(*coarse, coarse->d);
    const char* e2 = validate_grid(*fine, fine->d);
    if (e1 || e2) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", e1 ? e1 : e2);
        return LGNK_ERR_INVALID_ARG;
    }
    const cudaError_t e = launch_prolong_velocity(coarse->d, vc, vf, make_grid(*coarse), make_grid(*fine),
                                                  time_nodes * coarse->d, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", cudaGetErrorString(e));
        return LGNK_ERR_CUDA;
    }
    return LGNK_OK;
}

lgnk_status lgnk_solve_multilevel(const lgnk_problem* fine, int levels, void* stream, size_t mem_budget,
                                  const float* T, const float* R, float* v_out, const lgnk_solve_opts* opts,
                                  lgnk_solve_report* reports) {
    g_create_err[0] = 0;
    if (const char* e = validate_problem(fine)) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", e);
        return LGNK_ERR_INVALID_ARG;
    }
    if (levels < 1 || levels > 8 || T == nullptr || R == nullptr || v_out == nullptr) {
        snprintf(g_create_err, sizeof(g_create_err), "levels must be in [1, 8]; T, R, v_out non-NULL");
        return LGNK_ERR_INVALID_ARG;
    }
    const int d = fine->image.d;
    const int f = 1 << (levels - 1);
    for (int a = 0; a < d; ++a) {
        if (fine->image.m[a] % f != 0 || fine->velocity.m[a] % f != 0) {
            snprintf(g_create_err, sizeof(g_create_err), "cell counts must be divisible by 2^(levels-1)");
            return LGNK_ERR_INVALID_ARG;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // level problems, coarsest first
    std::vector<lgnk_problem> probs(levels, *fine);
    for (int l = 0; l < levels; ++l) {
        const int div = 1 << (levels - 1 - l);
        for (int a = 0; a < d; ++a) {
            probs[l].image.m[a] = fine->image.m[a] / div;
            probs[l].velocity.m[a] = fine->velocity.m[a] / div;
        }
    }
    auto voxels = [&](const lgnk_grid& g) {
        size_t n = 1;
        for (int a = 0; a < d; ++a) n *= (size_t)g.m[a];
        return n;
    };
    std::vector<void*> owned;
    size_t used = 0;
    lgnk_status status = LGNK_OK;
    auto alloc = [&](size_t bytes, float** out) -> lgnk_status {
        if (mem_budget != 0 && used + bytes > mem_budget) {
            snprintf(g_create_err, sizeof(g_create_err), "multilevel buffers exceed the memory budget");
            return LGNK_ERR_OOM;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            snprintf(g_create_err, sizeof(g_create_err), "cudaMalloc(%zu) failed", bytes);
            return LGNK_ERR_OOM;
        }
        owned.push_back(p);
        used += bytes;
        *out = static_cast<float*>(p);
        return LGNK_OK;
    };
    auto cleanup = [&]() {
        for (void* p : owned) cudaFree(p);
        owned.clear();
    };
    // restricted images per level (the finest are the caller's)
    std::vector<const float*> Ts(levels), Rs(levels);
    Ts[levels - 1] = T;
    Rs[levels - 1] = R;
    for (int l = levels - 2; l >= 0; --l) {
        float *tl = nullptr, *rl = nullptr;
        const size_t nb = voxels(probs[l].image) * sizeof(float);
        if ((status = alloc(nb, &tl)) != LGNK_OK || (status = alloc(nb, &rl)) != LGNK_OK) {
            cleanup();
            return status;
        }
        const DevGrid cg = make_grid(probs[l].image);
        if (launch_restrict_image(d, Ts[l + 1], tl, cg, s) != cudaSuccess ||
            launch_restrict_image(d, Rs[l + 1], rl, cg, s) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            snprintf(g_create_err, sizeof(g_create_err), "restriction launch failed");
            return LGNK_ERR_CUDA;
        }
        Ts[l] = tl;
        Rs[l] = rl;
    }
    float* v_prev = nullptr;
    lgnk_status last = LGNK_OK;
    for (int l = 0; l < levels; ++l) {
        const size_t n = voxels(probs[l].velocity) * d * fine->time_nodes;
        float* vl = v_out;
        if (l < levels - 1 && (status = alloc(n * sizeof(float), &vl)) != LGNK_OK) {
            cleanup();
            return status;
        }
        cudaError_t e = cudaSuccess;
        if (l == 0) e = cudaMemsetAsync(vl, 0, n * sizeof(float), s);
        else e = launch_prolong_velocity(d, v_prev, vl, make_grid(probs[l - 1].velocity),
                                          make_grid(probs[l].velocity), fine->time_nodes * d, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            snprintf(g_create_err, sizeof(g_create_err), "prolongation failed");
            return LGNK_ERR_CUDA;
        }
        lgnk_ctx* ctx = nullptr;
        const size_t left = mem_budget == 0 ? 0 : (mem_budget > used ? mem_budget - used : 1);
        if ((status = lgnk_create(&probs[l], stream, left, &ctx)) != LGNK_OK) {
            cleanup();
            return status;
        }
        last = lgnk_solve(ctx, Ts[l], Rs[l], vl, opts, reports ? &reports[l] : nullptr);
        if (last != LGNK_OK && last != LGNK_NOT_CONVERGED && last != LGNK_LS_FAILED) {
            snprintf(g_create_err, sizeof(g_create_err), "level %d: %.400s", l, ctx->err);
            lgnk_destroy(ctx);
            cleanup();
            return last;
        }
        lgnk_destroy(ctx);
        v_prev = vl;
    }
    cudaStreamSynchronize(s);
    cleanup();
    return last;
}

}  // extern "C"

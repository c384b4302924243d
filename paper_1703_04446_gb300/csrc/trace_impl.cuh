// Characteristic tracing kernels: one thread per voxel (= particle), RK4 state
// in registers (Alg. 1).  Included by trace2d.cu and trace3d.cu, each of which
// instantiates the family for one dimension.
//
// Modes (TraceMode):
//   FWD      trace, then transport gather u1 = T(y) (Eq. 6; optional SSD
//            partials, Eq. 10) or continuity splat of T(x_c) at y (Eq. 7).
//   JVP      trace with the forward-mode derivative of Alg. 1 applied to dv,
//            then du = grad T(y) . dy (transport) or the splat of
//            T(x_c) grad_y w . dy (continuity) (Sec. 3.2).
//   JTVP     trace storing the step starts, seed the adjoint at the end point,
//            sweep the RK4 steps backwards scattering into the gradient.
//   HESS     transport only: the Gauss-Newton product J^T h^d J dv fused per
//            voxel (u1 at voxel i depends only on characteristic i, so the
//            JVP value feeds that voxel's JTVP seed directly).
//   OBJGRAD  transport only: u1, SSD partials and the JTVP of h^d res fused.
//
// Position representation.  A characteristic starts at a cell centre x_c and
// its state is the FP32 displacement u = y - x_c.  Looking a point up on a grid
// uses the start's continuous grid index split into an integer I0 and a
// fraction F0 (computed once in FP64): the cell is I0 + floor(F0 + u / h).  A
// characteristic that barely moves off a grid node therefore keeps the sign of
// its displacement (an absolute FP32 coordinate would round it away), and the
// cell choice at the kinks of the piecewise-linear interpolant agrees with an
// exact evaluation.
#pragma once

#include "lgnk_internal.h"

namespace lgnk {

template <int D> struct VecT;
template <> struct VecT<2> { using type = float2; };
template <> struct VecT<3> { using type = float4; };

__device__ __forceinline__ void load_vec(const float2* p, float* o) {
    const float2 a = __ldg(p);
    o[0] = a.x; o[1] = a.y;
}
__device__ __forceinline__ void load_vec(const float4* p, float* o) {
    const float4 a = __ldg(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z;
}
__device__ __forceinline__ void red_vec(float2* p, const float* x, float w) {
    atomicAdd(p, make_float2(w * x[0], w * x[1]));
}
__device__ __forceinline__ void red_vec(float4* p, const float* x, float w) {
    atomicAdd(p, make_float4(w * x[0], w * x[1], w * x[2], 0.0f));
}

// Start of one characteristic on one grid: continuous index I0 + F0 and the
// clamp bounds of the offset t = F0 + u / h that keep I0 + floor(t) in [-2, m].
template <int D>
struct Start {
    int I0[D];
    float F0[D];
    float lo[D], hi[D];
};

template <int D>
__device__ __forceinline__ void start_on_image(const DevGrid& g, const int* idx, Start<D>& s) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        s.I0[a] = idx[a];
        s.F0[a] = 0.0f;
        s.lo[a] = (float)(-2 - idx[a]);
        s.hi[a] = (float)(g.m[a] - idx[a]) + 0.5f;
    }
}

template <int D>
__device__ __forceinline__ void start_on_velocity(const TraceArgs& A, const int* idx, Start<D>& s) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const double xi = A.vxi_a[a] + ((double)idx[a] + 0.5) * A.vxi_b[a];
        const double fl = floor(xi);
        const int i0 = (int)fmax(fmin(fl, (double)A.vg.m[a]), -2.0);
        s.I0[a] = i0;
        s.F0[a] = (float)(xi - (double)i0);
        s.lo[a] = (float)(-2 - i0);
        s.hi[a] = (float)(A.vg.m[a] - i0) + 0.5f;
    }
}

// Cell of the point at displacement u from the start: padded linear index of the
// lower corner and fractional offsets f in [0, 1].  NaN maps to the lowest
// clamp, so any point addresses padded storage.
template <int D>
__device__ __forceinline__ int locate(const DevGrid& g, const Start<D>& s, const float* u, float* f) {
    int idx[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float t = fmaf(u[a], g.inv_h[a], s.F0[a]);
        t = fminf(fmaxf(t, s.lo[a]), s.hi[a]);
        const float fl = floorf(t);
        f[a] = t - fl;
        idx[a] = s.I0[a] + (int)fl + LGNK_PAD;
    }
    if (D == 3) return idx[0] + g.mp[0] * (idx[1] + g.mp[1] * idx[2]);
    return idx[0] + g.mp[0] * idx[1];
}

template <int D>
__device__ __forceinline__ int corner_offset(const DevGrid& g, int c) {
    int o = (c & 1) + ((c >> 1) & 1) * g.mp[0];
    if (D == 3) o += ((c >> 2) & 1) * g.mp[0] * g.mp[1];
    return o;
}

// Multilinear weight of corner c and (optionally) its derivative along each axis.
template <int D, bool GRAD>
__device__ __forceinline__ float corner_weight(int c, const float* f, const DevGrid& g, float* dw) {
    float w1[D];
#pragma unroll
    for (int a = 0; a < D; ++a) w1[a] = ((c >> a) & 1) ? f[a] : 1.0f - f[a];
    float w = w1[0];
#pragma unroll
    for (int a = 1; a < D; ++a) w *= w1[a];
    if (GRAD) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float p = ((c >> a) & 1) ? g.inv_h[a] : -g.inv_h[a];
#pragma unroll
            for (int b = 0; b < D; ++b)
                if (b != a) p *= w1[b];
            dw[a] = p;
        }
    }
    return w;
}

// Time slot of stage time t: nodes t_j = j/(K-1), weight th on node j+1.
__device__ __forceinline__ void time_slot(int K, float t, int& j, float& th) {
    if (K == 1) { j = 0; th = 0.0f; return; }
    const float s = fminf(fmaxf(t, 0.0f), 1.0f) * (float)(K - 1);
    const int jj = min((int)floorf(s), K - 2);
    j = jj;
    th = s - (float)jj;
}

// I(v, p, t) and optionally d_y I (jac[c*D + a] = dV_c/dy_a) and I(dv, p, t).
template <int D, bool NS, bool JAC, bool DV>
__device__ __forceinline__ void sample_velocity(const DevGrid& g, int K,
                                                const typename VecT<D>::type* __restrict__ V,
                                                const typename VecT<D>::type* __restrict__ dV,
                                                int base, const float* f, int jt, float th,
                                                float* val, float* jac, float* dval) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
        val[c] = 0.0f;
        if (DV) dval[c] = 0.0f;
    }
    if (JAC) {
#pragma unroll
        for (int i = 0; i < D * D; ++i) jac[i] = 0.0f;
    }
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        const size_t e = (size_t)(base + corner_offset<D>(g, c)) * K + jt;
        float a[D];
        load_vec(V + e, a);
        if (NS) {
            float b[D];
            load_vec(V + e + 1, b);
#pragma unroll
            for (int q = 0; q < D; ++q) a[q] = fmaf(th, b[q] - a[q], a[q]);
        }
        float dw[D];
        const float w = corner_weight<D, JAC>(c, f, g, dw);
#pragma unroll
        for (int q = 0; q < D; ++q) val[q] = fmaf(w, a[q], val[q]);
        if (JAC) {
#pragma unroll
            for (int q = 0; q < D; ++q)
#pragma unroll
                for (int ax = 0; ax < D; ++ax) jac[q * D + ax] = fmaf(dw[ax], a[q], jac[q * D + ax]);
        }
        if (DV) {
            float da[D];
            load_vec(dV + e, da);
            if (NS) {
                float db[D];
                load_vec(dV + e + 1, db);
#pragma unroll
                for (int q = 0; q < D; ++q) da[q] = fmaf(th, db[q] - da[q], da[q]);
            }
#pragma unroll
            for (int q = 0; q < D; ++q) dval[q] = fmaf(w, da[q], dval[q]);
        }
    }
}

// G += (d_v I(., p, t))^T mu: the transpose of the velocity interpolation.
template <int D, bool NS>
__device__ __forceinline__ void scatter_velocity(const DevGrid& g, int K, typename VecT<D>::type* G,
                                                 int base, const float* f, int jt, float th,
                                                 const float* mu) {
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        const size_t e = (size_t)(base + corner_offset<D>(g, c)) * K + jt;
        const float w = corner_weight<D, false>(c, f, g, nullptr);
        if (NS) {
            red_vec(G + e, mu, w * (1.0f - th));
            red_vec(G + e + 1, mu, w * th);
        } else {
            red_vec(G + e, mu, w);
        }
    }
}

// T(y) and optionally grad T(y) from the padded image, y at displacement u.
template <int D, bool GRAD>
__device__ __forceinline__ float sample_image(const DevGrid& g, const Start<D>& s, const float* __restrict__ Tp,
                                              const float* u, float* grad) {
    float f[D];
    const int base = locate<D>(g, s, u, f);
    float val = 0.0f;
    if (GRAD) {
#pragma unroll
        for (int a = 0; a < D; ++a) grad[a] = 0.0f;
    }
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        const float t = __ldg(Tp + base + corner_offset<D>(g, c));
        float dw[D];
        const float w = corner_weight<D, GRAD>(c, f, g, dw);
        val = fmaf(w, t, val);
        if (GRAD) {
#pragma unroll
            for (int a = 0; a < D; ++a) grad[a] = fmaf(dw[a], t, grad[a]);
        }
    }
    return val;
}

// acc += mass * w(y) (push-forward, Eq. 7) or mass * (grad_y w(y) . dp).
template <int D, bool TANGENT>
__device__ __forceinline__ void splat_image(const DevGrid& g, const Start<D>& s, float* acc, const float* u,
                                            float mass, const float* dp) {
    float f[D];
    const int base = locate<D>(g, s, u, f);
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        float dw[D];
        const float w = corner_weight<D, TANGENT>(c, f, g, dw);
        float x;
        if (TANGENT) {
            x = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) x = fmaf(dw[a], dp[a], x);
            x *= mass;
        } else {
            x = w * mass;
        }
        atomicAdd(acc + base + corner_offset<D>(g, c), x);
    }
}

// One RK4 step of the characteristic (Alg. 1 without the derivative), on the
// displacement u.
template <int D, bool NS>
__device__ __forceinline__ void rk4_step(const TraceArgs& A, const Start<D>& sv,
                                         const typename VecT<D>::type* V, float* u, float tk) {
    int j1, j2, j4;
    float th1, th2, th4;
    time_slot(A.K, tk, j1, th1);
    time_slot(A.K, tk + 0.5f * A.dt, j2, th2);
    time_slot(A.K, tk + A.dt, j4, th4);
    const float dt = A.dt, hdt = 0.5f * A.dt;
    float f[D], v1[D], v2[D], v3[D], v4[D], us[D];
    int b = locate<D>(A.vg, sv, u, f);
    sample_velocity<D, NS, false, false>(A.vg, A.K, V, nullptr, b, f, j1, th1, v1, nullptr, nullptr);
#pragma unroll
    for (int a = 0; a < D; ++a) us[a] = fmaf(hdt, v1[a], u[a]);
    b = locate<D>(A.vg, sv, us, f);
    sample_velocity<D, NS, false, false>(A.vg, A.K, V, nullptr, b, f, j2, th2, v2, nullptr, nullptr);
#pragma unroll
    for (int a = 0; a < D; ++a) us[a] = fmaf(hdt, v2[a], u[a]);
    b = locate<D>(A.vg, sv, us, f);
    sample_velocity<D, NS, false, false>(A.vg, A.K, V, nullptr, b, f, j2, th2, v3, nullptr, nullptr);
#pragma unroll
    for (int a = 0; a < D; ++a) us[a] = fmaf(dt, v3[a], u[a]);
    b = locate<D>(A.vg, sv, us, f);
    sample_velocity<D, NS, false, false>(A.vg, A.K, V, nullptr, b, f, j4, th4, v4, nullptr, nullptr);
    const float s6 = dt / 6.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = fmaf(s6, v1[a] + 2.0f * (v2[a] + v3[a]) + v4[a], u[a]);
}

template <int D>
__device__ __forceinline__ void matvec(const float* J, const float* x, float* out) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int a = 0; a < D; ++a) s = fmaf(J[c * D + a], x[a], s);
        out[c] = s;
    }
}

template <int D>
__device__ __forceinline__ void rmatvec(const float* J, const float* x, float* out) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) s = fmaf(J[c * D + a], x[c], s);
        out[a] = s;
    }
}

// One RK4 step with the derivative recursion of Alg. 1 applied to dv:
// D_s = I(dv, y_s, t_s) + d_y I(v, y_s, t_s) (dy + c_s dt D_{s-1}).
template <int D, bool NS>
__device__ __forceinline__ void rk4_tangent_step(const TraceArgs& A, const Start<D>& sv,
                                                 const typename VecT<D>::type* V,
                                                 const typename VecT<D>::type* dV, float* u, float* dy,
                                                 float tk) {
    int j1, j2, j4;
    float th1, th2, th4;
    time_slot(A.K, tk, j1, th1);
    time_slot(A.K, tk + 0.5f * A.dt, j2, th2);
    time_slot(A.K, tk + A.dt, j4, th4);
    const float dt = A.dt, hdt = 0.5f * A.dt;
    float f[D], us[D], q[D], J[D * D], dvs[D], Jq[D];
    float v1[D], v2[D], v3[D], v4[D], D1[D], D2[D], D3[D], D4[D];

    int b = locate<D>(A.vg, sv, u, f);
    sample_velocity<D, NS, true, true>(A.vg, A.K, V, dV, b, f, j1, th1, v1, J, dvs);
    matvec<D>(J, dy, Jq);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        D1[a] = dvs[a] + Jq[a];
        us[a] = fmaf(hdt, v1[a], u[a]);
        q[a] = fmaf(hdt, D1[a], dy[a]);
    }
    b = locate<D>(A.vg, sv, us, f);
    sample_velocity<D, NS, true, true>(A.vg, A.K, V, dV, b, f, j2, th2, v2, J, dvs);
    matvec<D>(J, q, Jq);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        D2[a] = dvs[a] + Jq[a];
        us[a] = fmaf(hdt, v2[a], u[a]);
        q[a] = fmaf(hdt, D2[a], dy[a]);
    }
    b = locate<D>(A.vg, sv, us, f);
    sample_velocity<D, NS, true, true>(A.vg, A.K, V, dV, b, f, j2, th2, v3, J, dvs);
    matvec<D>(J, q, Jq);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        D3[a] = dvs[a] + Jq[a];
        us[a] = fmaf(dt, v3[a], u[a]);
        q[a] = fmaf(dt, D3[a], dy[a]);
    }
    b = locate<D>(A.vg, sv, us, f);
    sample_velocity<D, NS, true, true>(A.vg, A.K, V, dV, b, f, j4, th4, v4, J, dvs);
    matvec<D>(J, q, Jq);
    const float s6 = dt / 6.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        D4[a] = dvs[a] + Jq[a];
        dy[a] = fmaf(s6, D1[a] + 2.0f * (D2[a] + D3[a]) + D4[a], dy[a]);
        u[a] = fmaf(s6, v1[a] + 2.0f * (v2[a] + v3[a]) + v4[a], u[a]);
    }
}

// Transpose of one tangent step: given lam (adjoint of the step's end point),
// scatter the step's contribution into G and return the adjoint of its start.
template <int D, bool NS>
__device__ __forceinline__ void rk4_adjoint_step(const TraceArgs& A, const Start<D>& sv,
                                                 const typename VecT<D>::type* V, typename VecT<D>::type* G,
                                                 const float* u, float* lam, float tk) {
    int j1, j2, j4;
    float th1, th2, th4;
    time_slot(A.K, tk, j1, th1);
    time_slot(A.K, tk + 0.5f * A.dt, j2, th2);
    time_slot(A.K, tk + A.dt, j4, th4);
    const float dt = A.dt, hdt = 0.5f * A.dt;
    float f1[D], f2[D], f3[D], f4[D], J1[D * D], J2[D * D], J3[D * D], J4[D * D];
    float vs[D], us[D];
    const int b1 = locate<D>(A.vg, sv, u, f1);
    sample_velocity<D, NS, true, false>(A.vg, A.K, V, nullptr, b1, f1, j1, th1, vs, J1, nullptr);
#pragma unroll
    for (int a = 0; a < D; ++a) us[a] = fmaf(hdt, vs[a], u[a]);
    const int b2 = locate<D>(A.vg, sv, us, f2);
    sample_velocity<D, NS, true, false>(A.vg, A.K, V, nullptr, b2, f2, j2, th2, vs, J2, nullptr);
#pragma unroll
    for (int a = 0; a < D; ++a) us[a] = fmaf(hdt, vs[a], u[a]);
    const int b3 = locate<D>(A.vg, sv, us, f3);
    sample_velocity<D, NS, true, false>(A.vg, A.K, V, nullptr, b3, f3, j2, th2, vs, J3, nullptr);
#pragma unroll
    for (int a = 0; a < D; ++a) us[a] = fmaf(dt, vs[a], u[a]);
    const int b4 = locate<D>(A.vg, sv, us, f4);
    sample_velocity<D, NS, true, false>(A.vg, A.K, V, nullptr, b4, f4, j4, th4, vs, J4, nullptr);

    float mu[D], nu[D], acc[D];
    const float c16 = dt / 6.0f, c13 = dt / 3.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) mu[a] = c16 * lam[a];
    scatter_velocity<D, NS>(A.vg, A.K, G, b4, f4, j4, th4, mu);
    rmatvec<D>(J4, mu, nu);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = nu[a]; mu[a] = fmaf(c13, lam[a], dt * nu[a]); }
    scatter_velocity<D, NS>(A.vg, A.K, G, b3, f3, j2, th2, mu);
    rmatvec<D>(J3, mu, nu);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] += nu[a]; mu[a] = fmaf(c13, lam[a], hdt * nu[a]); }
    scatter_velocity<D, NS>(A.vg, A.K, G, b2, f2, j2, th2, mu);
    rmatvec<D>(J2, mu, nu);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] += nu[a]; mu[a] = fmaf(c16, lam[a], hdt * nu[a]); }
    scatter_velocity<D, NS>(A.vg, A.K, G, b1, f1, j1, th1, mu);
    rmatvec<D>(J1, mu, nu);
#pragma unroll
    for (int a = 0; a < D; ++a) lam[a] += acc[a] + nu[a];
}

template <int D> struct Tile;
template <> struct Tile<2> { static constexpr int X = 16, Y = 16, Z = 1; };
template <> struct Tile<3> { static constexpr int X = 8, Y = 8, Z = 4; };

__device__ __forceinline__ double block_sum(double x) {
    __shared__ double red[LGNK_BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = x;
    __syncthreads();
    double s = 0.0;
    if (warp == 0) {
        s = (lane < LGNK_BLOCK / 32) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

template <int D, bool NS, int MODEL, int MODE>
__global__ void __launch_bounds__(LGNK_BLOCK) trace_kernel(const TraceArgs A) {
    using VT = typename VecT<D>::type;
    constexpr bool TANGENT = (MODE == MODE_JVP || MODE == MODE_HESS);
    constexpr bool ADJOINT = (MODE == MODE_JTVP || MODE == MODE_HESS || MODE == MODE_OBJGRAD);
    const VT* V = static_cast<const VT*>(A.V);
    const VT* dV = static_cast<const VT*>(A.dV);
    VT* G = static_cast<VT*>(A.G);

    int b = blockIdx.x;
    const int bx = b % A.tiles[0];
    b /= A.tiles[0];
    const int by = b % A.tiles[1];
    const int bz = b / A.tiles[1];
    const int t = threadIdx.x;
    int idx[3];
    idx[0] = bx * Tile<D>::X + t % Tile<D>::X;
    idx[1] = by * Tile<D>::Y + (t / Tile<D>::X) % Tile<D>::Y;
    idx[2] = bz * Tile<D>::Z + t / (Tile<D>::X * Tile<D>::Y);
    const bool active = idx[0] < A.ig.m[0] && idx[1] < A.ig.m[1] && (D == 2 || idx[2] < A.ig.m[2]);
    double ssd = 0.0;

    if (active) {
        const int vox = idx[0] + A.ig.m[0] * (idx[1] + A.ig.m[1] * (D == 3 ? idx[2] : 0));
        Start<D> si, sv;
        start_on_image<D>(A.ig, idx, si);
        start_on_velocity<D>(A, idx, sv);
        float u[D], dy[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            u[a] = 0.0f;
            dy[a] = 0.0f;
        }
        float hist[ADJOINT ? LGNK_MAX_STEPS : 1][D];

        for (int k = 0; k < A.N; ++k) {
            const float tk = A.t0 + (float)k * A.dt;
            if (ADJOINT) {
#pragma unroll
                for (int a = 0; a < D; ++a) hist[ADJOINT ? k : 0][a] = u[a];
            }
            if (TANGENT) rk4_tangent_step<D, NS>(A, sv, V, dV, u, dy, tk);
            else rk4_step<D, NS>(A, sv, V, u, tk);
        }
        if (A.yout != nullptr) {
            const int M = A.ig.m[0] * A.ig.m[1] * (D == 3 ? A.ig.m[2] : 1);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float xc = A.ig.lo[a] + ((float)idx[a] + 0.5f) * A.ig.h[a];
                A.yout[(size_t)a * M + vox] = xc + u[a];
            }
        }

        float lam[D];
        if (MODEL == LGNK_TRANSPORT) {
            float gT[D];
            if (MODE == MODE_FWD) {
                const float val = sample_image<D, false>(A.ig, si, A.Tp, u, nullptr);
                A.u1[vox] = val;
                if (A.R != nullptr) {
                    const double r = (double)val - (double)A.R[vox];
                    ssd = r * r;
                }
            } else if (MODE == MODE_JVP) {
                sample_image<D, true>(A.ig, si, A.Tp, u, gT);
                float du = 0.0f;
#pragma unroll
                for (int a = 0; a < D; ++a) du = fmaf(gT[a], dy[a], du);
                A.u1[vox] = du;
            } else if (MODE == MODE_JTVP) {
                sample_image<D, true>(A.ig, si, A.Tp, u, gT);
                const float r = A.r[vox];
#pragma unroll
                for (int a = 0; a < D; ++a) lam[a] = r * gT[a];
            } else if (MODE == MODE_HESS) {
                sample_image<D, true>(A.ig, si, A.Tp, u, gT);
                float du = 0.0f;
#pragma unroll
                for (int a = 0; a < D; ++a) du = fmaf(gT[a], dy[a], du);
                const float s = A.cellvol * du;
#pragma unroll
                for (int a = 0; a < D; ++a) lam[a] = s * gT[a];
            } else {  // MODE_OBJGRAD
                const float val = sample_image<D, true>(A.ig, si, A.Tp, u, gT);
                if (A.u1 != nullptr) A.u1[vox] = val;
                const double rd = (double)val - (double)A.R[vox];
                ssd = rd * rd;
                const float s = A.cellvol * (float)rd;
#pragma unroll
                for (int a = 0; a < D; ++a) lam[a] = s * gT[a];
            }
        } else {
            const float mass = __ldg(A.T + vox);
            if (MODE == MODE_FWD) {
                splat_image<D, false>(A.ig, si, A.acc, u, mass, nullptr);
            } else if (MODE == MODE_JVP) {
                splat_image<D, true>(A.ig, si, A.acc, u, mass, dy);
            } else if (MODE == MODE_JTVP) {
                float gr[D];
                sample_image<D, true>(A.ig, si, A.r, u, gr);
#pragma unroll
                for (int a = 0; a < D; ++a) lam[a] = mass * gr[a];
            }
        }

        if (ADJOINT) {
            for (int k = A.N - 1; k >= 0; --k) {
                const float tk = A.t0 + (float)k * A.dt;
                rk4_adjoint_step<D, NS>(A, sv, V, G, hist[ADJOINT ? k : 0], lam, tk);
            }
        }
    }

    if (MODE == MODE_OBJGRAD || MODE == MODE_FWD) {
        if (A.partial != nullptr) {
            const double s = block_sum(ssd);
            if (threadIdx.x == 0) A.partial[blockIdx.x] = s;
        }
    }
}

template <int D, bool NS, int MODEL, int MODE>
static cudaError_t launch_one(const TraceArgs& a, int nblocks, cudaStream_t s) {
    trace_kernel<D, NS, MODEL, MODE><<<nblocks, LGNK_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

template <int D, bool NS>
static cudaError_t launch_dim(int model, int mode, const TraceArgs& a, int nblocks, cudaStream_t s) {
    if (model == LGNK_TRANSPORT) {
        switch (mode) {
            case MODE_FWD: return launch_one<D, NS, LGNK_TRANSPORT, MODE_FWD>(a, nblocks, s);
            case MODE_JVP: return launch_one<D, NS, LGNK_TRANSPORT, MODE_JVP>(a, nblocks, s);
            case MODE_JTVP: return launch_one<D, NS, LGNK_TRANSPORT, MODE_JTVP>(a, nblocks, s);
            case MODE_HESS: return launch_one<D, NS, LGNK_TRANSPORT, MODE_HESS>(a, nblocks, s);
            case MODE_OBJGRAD: return launch_one<D, NS, LGNK_TRANSPORT, MODE_OBJGRAD>(a, nblocks, s);
        }
    } else {
        switch (mode) {
            case MODE_FWD: return launch_one<D, NS, LGNK_CONTINUITY, MODE_FWD>(a, nblocks, s);
            case MODE_JVP: return launch_one<D, NS, LGNK_CONTINUITY, MODE_JVP>(a, nblocks, s);
            case MODE_JTVP: return launch_one<D, NS, LGNK_CONTINUITY, MODE_JTVP>(a, nblocks, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace lgnk

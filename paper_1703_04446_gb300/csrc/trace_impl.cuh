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
//   ASM      transport only: the adjoint sweep seeded with grad T(y) yields
//            row i of J = d_v u1 (Sec. 3.3 assembles J as a sparse matrix);
//            its stage contributions are summed per (slice, cell) block in a
//            per-thread table and written out entry-major (ELL layout), and
//            ell_kernel then applies J, J^T and J^T h^d J.
//
// Position representation.  A characteristic starts at a cell centre x_c and
// its state is the FP32 displacement u = y - x_c.  Looking a point up on a grid
// uses the start's continuous grid index split into an integer I0 and a
// fraction F0 (computed once in FP64): the cell is I0 + floor(F0 + u / h).  A
// characteristic that barely moves off a grid node therefore keeps the sign of
// its displacement (an absolute FP32 coordinate would round it away), and the
// cell choice at the kinks of the piecewise-linear interpolant agrees with an
// exact evaluation.
//
// Jacobian-free derivative products.  d_y I(v, y) enters only as J q (tangent)
// and J^T mu (adjoint).  The interpolant is evaluated separably, one plane of
// four corners at a time (x then y lerps, then z): the same lerps give the
// value and the three axis derivatives, J q contracts them with q, and J^T mu
// is the gradient of the scalar interpolant of v . mu (corners contracted with
// mu first).  No d x d matrix lives in registers.
//
// Time slices.  Every RK4 stage time is t0 + m dt/2 (m = 0..2N), so the host
// packs the velocity (and the direction) at those 2N + 1 times, linearly
// interpolated between its K time nodes, as slices [m][node].  A stage reads
// the one slice of its time: a non-stationary field costs the same gathers as
// a stationary one (K = 1: a single slice), and no time interpolation happens
// in the kernels.
//
// Gradient scatter.  (d_v I)^T mu goes to the padded gradient accumulator of
// the stage's slice with one vector reduction (red.global.add.v4.f32 / .v2)
// per corner, executed by the L2 atomic units; consecutive stages in the same
// cell and slice are combined first.  The host then distributes the slices
// onto the K time nodes with the transposed time weights.  A shared-memory tile of the velocity grid was measured
// slower: float atomics on shared memory retry under the heavy same-address
// contention of neighbouring characteristics.
#pragma once

#include <type_traits>

#include "fsum.cuh"
#include "lgnk_internal.h"

namespace lgnk {

template <int D> struct VecT;
template <> struct VecT<2> { using type = float2; };
template <> struct VecT<3> { using type = float4; };

__device__ __forceinline__ void red_vec(float2* p, const float* x, float w) {
    atomicAdd(p, make_float2(w * x[0], w * x[1]));
}
__device__ __forceinline__ void red_vec(float4* p, const float* x, float w) {
    atomicAdd(p, make_float4(w * x[0], w * x[1], w * x[2], 0.0f));
}

template <int D> struct TileShape;
template <> struct TileShape<2> { static constexpr int X = 16, Y = 16, Z = 1; };
template <> struct TileShape<3> { static constexpr int X = 8, Y = 8, Z = 4; };

// Voxel handled by this thread (recomputed from the block and thread indices
// where needed rather than held in registers).
template <int D>
__device__ __forceinline__ void voxel_index(const TraceArgs& A, int* idx) {
    using TS = TileShape<D>;
    int b = blockIdx.x;
    const int bx = b % A.tiles[0];
    b /= A.tiles[0];
    const int by = b % A.tiles[1];
    const int bz = b / A.tiles[1];
    const int t = threadIdx.x;
    idx[0] = bx * TS::X + t % TS::X;
    idx[1] = by * TS::Y + (t / TS::X) % TS::Y;
    idx[2] = bz * TS::Z + t / (TS::X * TS::Y);
}

// Start of one characteristic on one grid: its continuous grid index I0 + F0.
// Offsets t = F0 + u / h are clamped to [-2 - I0, m - I0 + 1/2], which keeps
// the lower corner I0 + floor(t) in [-2, m].
template <int D>
struct Start {
    int I0[D];
    float F0[D];
};

template <int D>
__device__ __forceinline__ void start_on_image(const int* idx, Start<D>& s) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        s.I0[a] = idx[a];
        s.F0[a] = 0.0f;
    }
}

// Start of this thread's characteristic on the velocity grid:
// (x_c - lo_v) / h_v - 1/2 = vxi_a + (i + 1/2) vxi_b, evaluated in FP32 (one
// rounding, below 1e-5 cells for grids up to 2^7 cells).
template <int D>
__device__ __forceinline__ void start_on_velocity(const TraceArgs& A, Start<D>& s) {
    int idx[3];
    voxel_index<D>(A, idx);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float xi = fmaf((float)idx[a] + 0.5f, A.vxi_bf[a], A.vxi_af[a]);
        const int i0 = min(max((int)floorf(xi), -2), A.vg.m[a]);
        s.I0[a] = i0;
        s.F0[a] = xi - (float)i0;
    }
}

// Cell of the point at displacement u from the start: per-axis padded index p
// of the lower corner and fractional offsets f in [0, 1].  NaN maps to the
// lowest clamp, so any point addresses padded storage.
template <int D>
__device__ __forceinline__ void locate(const DevGrid& g, const Start<D>& s, const float* u, int* p, float* f) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float t = fmaf(u[a], g.inv_h[a], s.F0[a]);
        t = fminf(fmaxf(t, (float)(-2 - s.I0[a])), (float)(g.m[a] - s.I0[a]) + 0.5f);
        const float fl = floorf(t);
        f[a] = t - fl;
        p[a] = s.I0[a] + (int)fl + LGNK_PAD;
    }
}

template <int D>
__device__ __forceinline__ int linear(const DevGrid& g, const int* p) {
    if (D == 3) return p[0] + g.mp[0] * (p[1] + g.mp[1] * p[2]);
    return p[0] + g.mp[0] * p[1];
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

// Both x-corners of a cell row from the pair-packed velocity: element e holds
// [v(node) | v(node + 1)] (3D: 32 bytes, one 256-bit load; 2D: 16 bytes).
__device__ __forceinline__ void load_pair3(const float* p, float* a, float* b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, _, %3, %4, %5, _}, [%6];"
        : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(b[0]), "=f"(b[1]), "=f"(b[2])
        : "l"(p));
}

template <int D>
__device__ __forceinline__ void pair_value(const float* __restrict__ V, size_t e, float* a, float* b) {
    constexpr int PS = (D == 3) ? 8 : 4;
    if (D == 3) {
        load_pair3(V + e * PS, a, b);
    } else {
        const float4 t = __ldg(reinterpret_cast<const float4*>(V + e * PS));
        a[0] = t.x; a[1] = t.y; b[0] = t.z; b[1] = t.w;
    }
}

__device__ __forceinline__ float lerp(float a, float b, float t) { return fmaf(t, b - a, a); }

// Element of corner (0, cy, cz) of the cell with lower corner `base` in the
// slice starting at element `s0`.
template <int D>
__device__ __forceinline__ size_t corner_elem(const DevGrid& g, size_t s0, int base, int cx, int cy, int cz) {
    int o = base + cx + cy * g.mp[0];
    if (D == 3) o += cz * g.mp[0] * g.mp[1];
    return s0 + (size_t)o;
}

// One plane (fixed z corner) of the cell: bilinear value and the unscaled
// derivatives along the fractional x and y offsets, per component.
template <int D, bool GRAD>
__device__ __forceinline__ void plane(const DevGrid& g, const float* __restrict__ V, size_t s0, int base, int cz,
                                      const float* f, float* val, float* dx, float* dy) {
    float c00[3], c10[3], c01[3], c11[3];
    pair_value<D>(V, corner_elem<D>(g, s0, base, 0, 0, cz), c00, c10);
    pair_value<D>(V, corner_elem<D>(g, s0, base, 0, 1, cz), c01, c11);
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const float a0 = lerp(c00[q], c10[q], f[0]);
        const float a1 = lerp(c01[q], c11[q], f[0]);
        val[q] = lerp(a0, a1, f[1]);
        if (GRAD) {
            dx[q] = lerp(c10[q] - c00[q], c11[q] - c01[q], f[1]);
            dy[q] = a1 - a0;
        }
    }
}

// Scalar version: corner values contracted with mu first (s_c = v_c . mu).
template <int D>
__device__ __forceinline__ void plane_dot(const DevGrid& g, const float* __restrict__ V, size_t s0, int base, int cz,
                                          const float* f, const float* mu, float& val, float& dx, float& dy) {
    float c[4];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float a[3], b[3];
        pair_value<D>(V, corner_elem<D>(g, s0, base, 0, r, cz), a, b);
        float sa = 0.0f, sb = 0.0f;
#pragma unroll
        for (int q = 0; q < D; ++q) {
            sa = fmaf(a[q], mu[q], sa);
            sb = fmaf(b[q], mu[q], sb);
        }
        c[2 * r] = sa;
        c[2 * r + 1] = sb;
    }
    const float a0 = lerp(c[0], c[1], f[0]);
    const float a1 = lerp(c[2], c[3], f[0]);
    val = lerp(a0, a1, f[1]);
    dx = lerp(c[1] - c[0], c[3] - c[2], f[1]);
    dy = a1 - a0;
}

// val = I(v, y, t) at the slice of t (Sec. 3.1, Step 1: multilinear in space,
// linear in time through the slice).
template <int D>
__device__ __forceinline__ void stage_value(const DevGrid& g, const float* __restrict__ V, size_t s0, const int* p,
                                            const float* f, float* val) {
    const int base = linear<D>(g, p);
    plane<D, false>(g, V, s0, base, 0, f, val, nullptr, nullptr);
    if (D == 3) {
        float v1[D];
        plane<D, false>(g, V, s0, base, 1, f, v1, nullptr, nullptr);
#pragma unroll
        for (int q = 0; q < D; ++q) val[q] = lerp(val[q], v1[q], f[D - 1]);
    }
}

// Tangent stage: val = I(v, y, t), Jq = d_y I(v, y, t) q, dval = I(dv, y, t).
template <int D>
__device__ __forceinline__ void stage_tangent(const DevGrid& g, const float* __restrict__ V,
                                              const float* __restrict__ dV, size_t s0, const int* p, const float* f,
                                              const float* qv, float* val, float* Jq, float* dval) {
    const int base = linear<D>(g, p);
    float qs[D];
#pragma unroll
    for (int a = 0; a < D; ++a) qs[a] = qv[a] * g.inv_h[a];
    float dx[D], dy[D];
    plane<D, true>(g, V, s0, base, 0, f, val, dx, dy);
    if (D == 3) {
        float v1[D], dx1[D], dy1[D];
        plane<D, true>(g, V, s0, base, 1, f, v1, dx1, dy1);
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const float dz = v1[q] - val[q];
            Jq[q] = dz * qs[D - 1];
            val[q] = lerp(val[q], v1[q], f[D - 1]);
            dx[q] = lerp(dx[q], dx1[q], f[D - 1]);
            dy[q] = lerp(dy[q], dy1[q], f[D - 1]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < D; ++q) Jq[q] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < D; ++q) Jq[q] = fmaf(dx[q], qs[0], fmaf(dy[q], qs[1], Jq[q]));
    stage_value<D>(g, dV, s0, p, f, dval);
}

// Destination of the adjoint scatter (d_v I)^T mu: the padded gradient
// accumulator of each slice, with a one-entry write-combining slot.
// A pending cell block in moment form.  The block's corner vectors are
// sum_stages w_c(f) mu with w_c = prod_a (c_a ? f_a : 1 - f_a); expanding the
// product, they follow from the moments m_k = sum_stages phi_k(f) mu, phi_k =
// prod of the f_a over the axes a set in k (bit 0 x, bit 1 y, bit 2 z), by
// one subtraction per pair and axis: w_c = sum over subsets T of the axes
// with c_a = 0 of (-1)^|T| phi_(c + T).  A stage then costs the 2^d - 1 - d
// products of offsets, D adds and (2^d - 1) D FMAs (3D: 4 FMUL, 3 FADD, 21
// FFMA) instead of the corner weights and (2^d) D FMAs (12 FMUL, 3 FADD, 24
// FFMA); the conversion (12 FADD per component in 3D) is paid once per block.
// Blocks are flat, m[k D + q].
template <int D>
__device__ __forceinline__ void moments_add(float* m, const float* f, const float* mu) {
    float phi[1 << D];
    phi[1] = f[0];
    phi[2] = f[1];
    phi[3] = f[0] * f[1];
    if (D == 3) {
        phi[4] = f[D - 1];
        phi[5] = f[0] * f[D - 1];
        phi[6] = f[1] * f[D - 1];
        phi[7] = phi[3] * f[D - 1];
    }
#pragma unroll
    for (int q = 0; q < D; ++q) m[q] += mu[q];
#pragma unroll
    for (int k = 1; k < (1 << D); ++k)
#pragma unroll
        for (int q = 0; q < D; ++q) m[k * D + q] = fmaf(phi[k], mu[q], m[k * D + q]);
}

// Moments to corner vectors, in place.
template <int D>
__device__ __forceinline__ void moments_to_corners(float* m) {
#pragma unroll
    for (int b = 1; b < (1 << D); b <<= 1)
#pragma unroll
        for (int k = 0; k < (1 << D); ++k)
            if (!(k & b)) {
#pragma unroll
                for (int q = 0; q < D; ++q) m[k * D + q] -= m[(k | b) * D + q];
            }
}

template <int D>
__device__ __forceinline__ void block_zero(float* m) {
#pragma unroll
    for (int k = 0; k < (1 << D) * D; ++k) m[k] = 0.0f;
}

// Consecutive adjoint stages of a characteristic usually fall in the same
// velocity cell and slice; their contributions w_c(f) mu are then summed per
// corner and sent as one vector reduction instead of two.
template <int D>
struct Scatter {
    typename VecT<D>::type* G;
    size_t s0;      // slice of the pending contribution
    int base;       // its cell, -1 if none
    float f[D];
    float mu[D];
};

template <int D>
__device__ __forceinline__ void scatter_flush(const DevGrid& g, Scatter<D>& S, bool two, const float* f2,
                                              const float* mu2) {
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        float w = (c & 1 ? S.f[0] : 1.0f - S.f[0]) * ((c >> 1) & 1 ? S.f[1] : 1.0f - S.f[1]);
        if (D == 3) w *= ((c >> 2) & 1) ? S.f[D - 1] : 1.0f - S.f[D - 1];
        float w2 = 0.0f;
        if (two) {
            w2 = (c & 1 ? f2[0] : 1.0f - f2[0]) * ((c >> 1) & 1 ? f2[1] : 1.0f - f2[1]);
            if (D == 3) w2 *= ((c >> 2) & 1) ? f2[D - 1] : 1.0f - f2[D - 1];
        }
        const size_t e = corner_elem<D>(g, S.s0, S.base, c & 1, (c >> 1) & 1, (c >> 2) & 1);
        float x[D];
#pragma unroll
        for (int q = 0; q < D; ++q) x[q] = fmaf(w2, two ? mu2[q] : 0.0f, w * S.mu[q]);
        red_vec(S.G + e, x, 1.0f);
    }
    S.base = -1;
}

// Add the contribution w_c(f) mu at cell `base` of slice `s0`.
template <int D>
__device__ __forceinline__ void scatter_add(const DevGrid& g, Scatter<D>& S, size_t s0, int base, const float* f,
                                            const float* mu) {
    if (S.base == base && S.s0 == s0) {
        scatter_flush<D>(g, S, true, f, mu);
        return;
    }
    if (S.base >= 0) scatter_flush<D>(g, S, false, f, mu);
    S.base = base;
    S.s0 = s0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        S.f[a] = f[a];
        S.mu[a] = mu[a];
    }
}

template <int D>
__device__ __forceinline__ void scatter_init(Scatter<D>& S, void* G) {
    S.G = static_cast<typename VecT<D>::type*>(G);
    S.base = -1;
    S.s0 = 0;
}

template <int D>
__device__ __forceinline__ void scatter_finish(const DevGrid& g, Scatter<D>& S) {
    if (S.base >= 0) scatter_flush<D>(g, S, false, S.f, S.mu);
}

// Destination of the adjoint scatter with the whole pending cell in
// registers: the contributions w_c(f) mu of consecutive stages in one cell and
// slice are accumulated (in moment form) and sent as 2^d vector reductions
// only when the cell or slice changes (the transport matvec, where
// consecutive stages mostly share a cell).  The block is zeroed inside the
// flush, so that a stage's update is the same FMAs whether it opens a block or
// not: written as "fresh ? w mu : w mu + blk", the compiler evaluated both and
// selected, 24 FMULs and 24 selects per stage (the 128^3 matvec kernel went
// 0.630 -> 0.586 ms with both changes, the assembly 0.653 -> 0.627 ms).
template <int D>
struct BlockScatter {
    typename VecT<D>::type* G;
    int key;                  // s0 + base of the pending cell, -1 if none (the packed velocity has
                              // fewer than 2^31 elements: checked when the context is created)
    float blk[(1 << D) * D];
};

template <int D>
__device__ __forceinline__ void scatter_init(BlockScatter<D>& S, void* G) {
    S.G = static_cast<typename VecT<D>::type*>(G);
    S.key = -1;
    block_zero<D>(S.blk);
}

template <int D>
__device__ __forceinline__ void block_flush(const DevGrid& g, BlockScatter<D>& S) {
    moments_to_corners<D>(S.blk);
#pragma unroll
    for (int c = 0; c < (1 << D); ++c)
        red_vec(S.G + corner_elem<D>(g, (size_t)S.key, 0, c & 1, (c >> 1) & 1, (c >> 2) & 1), S.blk + c * D, 1.0f);
    block_zero<D>(S.blk);
}

template <int D>
__device__ __forceinline__ void scatter_finish(const DevGrid& g, BlockScatter<D>& S) {
    if (S.key >= 0) block_flush<D>(g, S);
}

template <int D>
__device__ __forceinline__ void scatter_add(const DevGrid& g, BlockScatter<D>& S, size_t s0, int base, const float* f,
                                            const float* mu) {
    const int key = (int)s0 + base;
    if (key != S.key) {
        if (S.key >= 0) block_flush<D>(g, S);
        S.key = key;
    }
    moments_add<D>(S.blk, f, mu);
}

// Destination of the adjoint contributions when a row of J is assembled: the
// row's (slice, cell) blocks, each the 2^d corner vectors sum_stages
// w_c(f) mu.  A trajectory stays within a few velocity cells, so a row has
// few blocks; a row that needs more than CAP sets `overflow`.  The keys live
// in a per-thread table (local memory); the blocks go straight to the row's
// slots of the global ELL array, entry j of voxel i at [j][i][corner][q], and
// a block met again is read back, added to and stored by the same thread.
template <int D>
struct AsmTable {
    static constexpr int CAP = D == 3 ? 16 : 32;
    long long key[CAP];
    int n;
    bool overflow;
};

// The block of the current cell is kept in registers (pblk) until the cell
// changes; it is then committed to the row (kept in the table's local array
// it was placed in local memory: 1.23 ms for the 128^3 assembly, 0.79 ms apart).
template <int D>
struct AsmRow {
    static constexpr int CAP = AsmTable<D>::CAP;
    static constexpr int B = (1 << D) * D;
    AsmTable<D>* tab;
    float* blk;               // entry 0 of this voxel's blocks in the ELL array
    size_t stride;            // floats from entry j to entry j + 1 of one voxel
    long long pkey;
    float pblk[B];
};

template <int D>
__device__ __forceinline__ void scatter_init(AsmRow<D>& S, void*) {
    S.pkey = -1;
    block_zero<D>(S.pblk);
}

// The pending block's corner vectors into the row (asm_commit).
template <int D>
__device__ __forceinline__ void asm_store(AsmRow<D>& S) {
    constexpr int B = AsmRow<D>::B;
    AsmTable<D>& T = *S.tab;
    int j = T.n - 1;
#pragma unroll 1
    for (; j >= 0; --j)       // newest first: a trajectory revisits the cell it just left
        if (T.key[j] == S.pkey) break;
    const bool fresh = j < 0;
    if (fresh) {
        if (T.n == AsmTable<D>::CAP) {
            T.overflow = true;
            return;
        }
        j = T.n++;
        T.key[j] = S.pkey;
    }
    float4* dst = reinterpret_cast<float4*>(S.blk + (size_t)j * S.stride);
#pragma unroll
    for (int k = 0; k < B / 4; ++k) {
        float4 b = make_float4(S.pblk[4 * k], S.pblk[4 * k + 1], S.pblk[4 * k + 2], S.pblk[4 * k + 3]);
        if (!fresh) {
            const float4 o = dst[k];
            b.x += o.x;
            b.y += o.y;
            b.z += o.z;
            b.w += o.w;
        }
        dst[k] = b;
    }
}

// Add the pending block (moments, converted here to corner vectors) to the
// row's entry of its cell (a new entry if the row has none yet), and zero it.
template <int D>
__device__ __forceinline__ void asm_commit(AsmRow<D>& S) {
    moments_to_corners<D>(S.pblk);
    asm_store<D>(S);
    block_zero<D>(S.pblk);
}

template <int D>
__device__ __forceinline__ void scatter_finish(const DevGrid&, AsmRow<D>& S) {
    if (S.pkey >= 0) asm_commit<D>(S);
    S.pkey = -1;
}

template <int D>
__device__ __forceinline__ void scatter_add(const DevGrid& g, AsmRow<D>& S, size_t s0, int base, const float* f,
                                            const float* mu) {
    (void)g;
    const long long key = (long long)s0 + base;
    if (key != S.pkey) {
        if (S.pkey >= 0) asm_commit<D>(S);
        S.pkey = key;
    }
    moments_add<D>(S.pblk, f, mu);
}

// Adjoint stage: scatter w_c mu into the slice's gradient and return
// nu = d_y I(v, y, t)^T mu = grad_y (v . mu) of the interpolant.
template <int D, class SC>
__device__ __forceinline__ void stage_adjoint(const DevGrid& g, const float* __restrict__ V, SC& S,
                                              size_t s0, int base, const float* f, const float* mu, float* nu) {
    float s_0, dx, dy;
    plane_dot<D>(g, V, s0, base, 0, f, mu, s_0, dx, dy);
    if (D == 3) {
        float s_1, dx1, dy1;
        plane_dot<D>(g, V, s0, base, 1, f, mu, s_1, dx1, dy1);
        nu[D - 1] = (s_1 - s_0) * g.inv_h[D - 1];
        dx = lerp(dx, dx1, f[D - 1]);
        dy = lerp(dy, dy1, f[D - 1]);
    }
    nu[0] = dx * g.inv_h[0];
    nu[1] = dy * g.inv_h[1];
    scatter_add<D>(g, S, s0, base, f, mu);
}

// The velocity cell last met (and the direction's, when DV), kept in
// registers as the coefficients of its multilinear interpolant, per component
//   3D: v(f) = a0 + a1 fx + a2 fy + a3 fz + a4 fx fy + a5 fx fz + a6 fy fz + a7 fx fy fz
//   2D: v(f) = a0 + a1 fx + a2 fy + a3 fx fy
// with f the fractional offsets in the cell.  Consecutive RK4 stages mostly
// fall in the same cell and slice (stages 2 and 3 share their time and nearly
// their position, stage 4 of a step is stage 1 of the next), so a stage
// recomputes the coefficients only when its cell or slice changes.  From the
// coefficients the value and the d derivatives of a component cost 11 FMAs
// in 3D and the value alone 7 (the lerps of the corner values took about 23
// and 14 operations); the interpolant is the same multilinear function.
template <int D, bool DV>
struct CellCache {
    static constexpr int NC = 1 << D;
    int key;                  // s0 + base of the cached cell, -1 when empty (32 bits: see BlockScatter)
    float a[D][NC];           // coefficients of v, per component
    float b[DV ? D : 1][DV ? NC : 1];   // of dv
};

// Coefficients of one component from its corner values c[cx + 2 cy + 4 cz].
template <int D>
__device__ __forceinline__ void poly_coeffs(const float* c, float* a) {
    a[0] = c[0];
    a[1] = c[1] - c[0];
    a[2] = c[2] - c[0];
    if (D == 2) {
        a[3] = (c[3] - c[2]) - a[1];
    } else {
        a[3] = c[4] - c[0];
        a[4] = (c[3] - c[2]) - a[1];
        a[5] = (c[5] - c[4]) - a[1];
        a[6] = (c[6] - c[4]) - a[2];
        a[7] = ((c[7] - c[6]) - (c[5] - c[4])) - a[4];
    }
}

template <int D, bool DV>
__device__ __forceinline__ void cache_cell(const DevGrid& g, const float* __restrict__ V, const float* __restrict__ dV,
                                           size_t s0, int base, CellCache<D, DV>& C) {
    const int key = (int)s0 + base;
    if (key == C.key) return;
    C.key = key;
    float cv[1 << D][D], cd[DV ? (1 << D) : 1][D];
#pragma unroll
    for (int r = 0; r < (1 << (D - 1)); ++r) {
        pair_value<D>(V, corner_elem<D>(g, s0, base, 0, r & 1, r >> 1), cv[2 * r], cv[2 * r + 1]);
        if (DV) pair_value<D>(dV, corner_elem<D>(g, s0, base, 0, r & 1, r >> 1), cd[2 * r], cd[2 * r + 1]);
    }
#pragma unroll
    for (int q = 0; q < D; ++q) {
        float c[1 << D];
#pragma unroll
        for (int k = 0; k < (1 << D); ++k) c[k] = cv[k][q];
        poly_coeffs<D>(c, C.a[q]);
        if (DV) {
#pragma unroll
            for (int k = 0; k < (1 << D); ++k) c[k] = cd[k][q];
            poly_coeffs<D>(c, C.b[DV ? q : 0]);
        }
    }
}

// Value of the interpolant with coefficients a at f.
template <int D>
__device__ __forceinline__ float poly_value(const float* a, const float* f) {
    if (D == 2) return fmaf(f[0], fmaf(f[1], a[3], a[1]), fmaf(f[1], a[2], a[0]));
    const float gx = fmaf(f[2], a[5], fmaf(f[1], fmaf(f[2], a[7], a[4]), a[1]));
    const float u = fmaf(f[2], a[3], fmaf(f[1], fmaf(f[2], a[6], a[2]), a[0]));
    return fmaf(f[0], gx, u);
}

// Value and derivatives along the fractional offsets (per cell width).
template <int D>
__device__ __forceinline__ float poly_value_grad(const float* a, const float* f, float* gr) {
    if (D == 2) {
        gr[0] = fmaf(f[1], a[3], a[1]);
        gr[1] = fmaf(f[0], a[3], a[2]);
        return fmaf(f[0], gr[0], fmaf(f[1], a[2], a[0]));
    }
    const float t1 = fmaf(f[2], a[7], a[4]);
    const float t4 = fmaf(f[2], a[6], a[2]);
    gr[0] = fmaf(f[2], a[5], fmaf(f[1], t1, a[1]));
    gr[1] = fmaf(f[0], t1, t4);
    gr[2] = fmaf(f[1], fmaf(f[0], a[7], a[6]), fmaf(f[0], a[5], a[3]));
    return fmaf(f[0], gr[0], fmaf(f[2], a[3], fmaf(f[1], t4, a[0])));
}

// Derivatives only (the constant coefficient is not read).
template <int D>
__device__ __forceinline__ void poly_grad(const float* a, const float* f, float* gr) {
    if (D == 2) {
        gr[0] = fmaf(f[1], a[3], a[1]);
        gr[1] = fmaf(f[0], a[3], a[2]);
        return;
    }
    const float t1 = fmaf(f[2], a[7], a[4]);
    gr[0] = fmaf(f[2], a[5], fmaf(f[1], t1, a[1]));
    gr[1] = fmaf(f[0], t1, fmaf(f[2], a[6], a[2]));
    gr[2] = fmaf(f[1], fmaf(f[0], a[7], a[6]), fmaf(f[0], a[5], a[3]));
}

// The cached-cell forms of stage_tangent, stage_adjoint and stage_value.
template <int D>
__device__ __forceinline__ void stage_tangent_cached(const DevGrid& g, const float* __restrict__ V,
                                                     const float* __restrict__ dV, size_t s0, const int* p,
                                                     const float* f, const float* qv, CellCache<D, true>& C,
                                                     float* val, float* Jq, float* dval) {
    cache_cell<D, true>(g, V, dV, s0, linear<D>(g, p), C);
    float qs[D];
#pragma unroll
    for (int a = 0; a < D; ++a) qs[a] = qv[a] * g.inv_h[a];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        float gr[D];
        val[q] = poly_value_grad<D>(C.a[q], f, gr);
        float jq = gr[D - 1] * qs[D - 1];
#pragma unroll
        for (int a = D - 2; a >= 0; --a) jq = fmaf(gr[a], qs[a], jq);
        Jq[q] = jq;
        dval[q] = poly_value<D>(C.b[q], f);
    }
}

template <int D, class SC>
__device__ __forceinline__ void stage_adjoint_cached(const DevGrid& g, const float* __restrict__ V, SC& S,
                                                     CellCache<D, false>& C, size_t s0, int base, const float* f,
                                                     const float* mu, float* nu) {
    cache_cell<D, false>(g, V, nullptr, s0, base, C);
    // coefficients of the scalar interpolant of v . mu (its constant is not needed)
    float sc[1 << D];
#pragma unroll
    for (int i = 1; i < (1 << D); ++i) {
        float t = C.a[0][i] * mu[0];
#pragma unroll
        for (int q = 1; q < D; ++q) t = fmaf(C.a[q][i], mu[q], t);
        sc[i] = t;
    }
    sc[0] = 0.0f;
    float gr[D];
    poly_grad<D>(sc, f, gr);
#pragma unroll
    for (int a = 0; a < D; ++a) nu[a] = gr[a] * g.inv_h[a];
    scatter_add<D>(g, S, s0, base, f, mu);
}

template <int D>
__device__ __forceinline__ void stage_value_cached(const DevGrid& g, const float* __restrict__ V, size_t s0,
                                                   const int* p, const float* f, CellCache<D, false>& C, float* val) {
    cache_cell<D, false>(g, V, nullptr, s0, linear<D>(g, p), C);
#pragma unroll
    for (int q = 0; q < D; ++q) val[q] = poly_value<D>(C.a[q], f);
}

// T(y) and optionally grad T(y) from the padded image, y at displacement u.
template <int D, bool GRAD>
__device__ __forceinline__ float sample_image(const DevGrid& g, const Start<D>& s, const float* __restrict__ Tp,
                                              const float* u, float* grad) {
    int p[D];
    float f[D];
    locate<D>(g, s, u, p, f);
    const int base = linear<D>(g, p);
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

// The push-forward through a shared-memory tile (Eq. 7 with the default
// particle width; every thread of the CTA calls it, inactive ones with
// active = false).  The CTA's particles start on one 8 x 8 x 4 (3D) or
// 16 x 16 (2D) tile of voxels and a smooth flow keeps their end cells
// together, so the CTA reduces the box of their cells; when the box with its
// upper corners holds at most kSplatTile cells, the particles add their
// corner masses into a zeroed tile in shared memory and the CTA then adds
// each nonzero cell of the tile to the image with one global atomic, instead
// of one per particle and corner.  A larger box (large displacements) takes
// the per-particle global atomics.  Measured on the brain-scale forward and
// JVP: 2.06 / 4.01 ms against 1.99 / 3.97 ms with the box reduction but
// direct global atomics (1.93 / 3.85 ms with the splat inline in the trace):
// the L2 atomics are not what bounds these kernels.  Combining, before the
// shared atomic, the lanes of a warp whose corner lands in the same cell
// (__match_any_sync, one leader per cell) measured 2.14 / 4.12 ms: for a
// given corner the lanes' cells are distinct unless the flow compresses, so
// the match finds no peers and costs its instructions.
constexpr int kSplatTile = 2048;

template <int D, bool TANGENT>
__device__ __forceinline__ void splat_tiled(const DevGrid& g, float* acc, bool active, const int* p, const float* f,
                                            float mass, const float* dp) {
    __shared__ float tile[kSplatTile];
    __shared__ int wbox[LGNK_BLOCK / 32][6];
    float x[1 << D];
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        float dw[D];
        const float w = corner_weight<D, TANGENT>(c, f, g, dw);
        if (TANGENT) {
            float t = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) t = fmaf(dw[a], dp[a], t);
            x[c] = t * mass;
        } else {
            x[c] = w * mass;
        }
    }
    // the box of the CTA's cells (lower corners), per axis
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int l = __reduce_min_sync(0xffffffffu, active ? p[a] : 0x7fffffff);
        const int h = __reduce_max_sync(0xffffffffu, active ? p[a] : -0x7fffffff);
        if (lane == 0) {
            wbox[warp][a] = l;
            wbox[warp][3 + a] = h;
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < D; ++a) {
        lo[a] = wbox[0][a];
        hi[a] = wbox[0][3 + a];
#pragma unroll
        for (int w = 1; w < LGNK_BLOCK / 32; ++w) {
            lo[a] = min(lo[a], wbox[w][a]);
            hi[a] = max(hi[a], wbox[w][3 + a]);
        }
    }
    if (hi[0] < lo[0]) return;            // no active particle in the CTA
    int ext[3] = {1, 1, 1};
    long long vol = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        ext[a] = hi[a] - lo[a] + 2;
        vol *= ext[a];
    }
    if (vol > kSplatTile) {
        if (active) {
            const int base = linear<D>(g, p);
#pragma unroll
            for (int c = 0; c < (1 << D); ++c) atomicAdd(acc + base + corner_offset<D>(g, c), x[c]);
        }
        return;
    }
    const int nv = (int)vol;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) tile[i] = 0.0f;
    __syncthreads();
    const int lb = active ? (p[0] - lo[0]) + ext[0] * ((p[1] - lo[1]) + (D == 3 ? ext[1] * (p[D - 1] - lo[D - 1]) : 0))
                          : 0;
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        const int l = lb + (c & 1) + ((c >> 1) & 1) * ext[0] + (D == 3 ? ((c >> 2) & 1) * ext[0] * ext[1] : 0);
        if (active) atomicAdd(&tile[l], x[c]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        const float v = tile[i];
        if (v != 0.0f) {
            int r = i;
            const int ix = r % ext[0];
            r /= ext[0];
            int gi;
            if (D == 3) {
                const int iy = r % ext[1];
                const int iz = r / ext[1];
                gi = (lo[0] + ix) + g.mp[0] * ((lo[1] + iy) + g.mp[1] * (lo[D - 1] + iz));
            } else {
                gi = (lo[0] + ix) + g.mp[0] * (lo[1] + r);
            }
            atomicAdd(acc + gi, v);
        }
    }
}

// General-width PIC push-forward (Eqs. 7-8): the particle is the tensor
// product of unit-mass hats max(0, 1 - |s| / rho) / rho of half-width rho
// cells; cell c (node coordinates [c - 1/2, c + 1/2]) receives the exact
// integral of the particle over it, a difference of the hat's antiderivative,
// so the weights of a particle sum to one.  Cells outside the grid are
// dropped.  rho <= 3.5 keeps a particle within kHatMax cells per axis.
constexpr int kHatMax = 8;

__device__ __forceinline__ float hat_cdf(float s) {
    s = fminf(fmaxf(s, -1.0f), 1.0f);
    return s <= 0.0f ? 0.5f * (1.0f + s) * (1.0f + s) : 1.0f - 0.5f * (1.0f - s) * (1.0f - s);
}

__device__ __forceinline__ float hat_pdf(float s) { return fmaxf(0.0f, 1.0f - fabsf(s)); }

// Cells [I0 + c0, I0 + c0 + n) of one axis that a particle at node coordinate
// I0 + t overlaps inside the grid, their weights and d(weight)/dy.
__device__ __forceinline__ void hat_axis(float t, float rho, int I0, int m, float inv_h, int& c0, int& n, float* w,
                                         float* dw) {
    t = fminf(fmaxf(t, -(float)I0 - rho - 2.0f), (float)(m - I0) + rho + 2.0f);   // also maps NaN into range
    const int lo = max((int)floorf(t - rho + 0.5f), -I0);
    const int hi = min((int)floorf(t + rho + 0.5f), m - 1 - I0);
    c0 = lo;
    n = min(hi - lo + 1, kHatMax);
    const float ir = 1.0f / rho;
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
        const float c = (float)(lo + j);
        const float s1 = (c + 0.5f - t) * ir, s0 = (c - 0.5f - t) * ir;
        w[j] = hat_cdf(s1) - hat_cdf(s0);
        dw[j] = (hat_pdf(s0) - hat_pdf(s1)) * ir * inv_h;
    }
}

// KIND 0: acc += mass w (push-forward); KIND 1: acc += mass (grad_y w . dp)
// (its tangent); KIND 2: grad = sum_c grad_y w_c F_c (the transpose's seed).
// acc and F are padded image grids.
template <int D, int KIND>
__device__ __noinline__ void pic_hat(const DevGrid& g, const int* I0, const float* u, const float* rho, float* acc,
                                     const float* __restrict__ F, float mass, const float* dp, float* grad) {
    int c0[3] = {0, 0, 0}, n[3] = {1, 1, 1};
    float w[3][kHatMax], dw[3][kHatMax];
    w[2][0] = 1.0f;
    dw[2][0] = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) hat_axis(u[a] * g.inv_h[a], rho[a], I0[a], g.m[a], g.inv_h[a], c0[a], n[a], w[a], dw[a]);
    float gsum[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 1
    for (int kz = 0; kz < n[2]; ++kz) {
#pragma unroll 1
        for (int ky = 0; ky < n[1]; ++ky) {
            const float wyz = w[1][ky] * w[2][kz];
            const float dyz = dw[1][ky] * w[2][kz], ydz = w[1][ky] * dw[2][kz];
            int p[3];
            p[1] = I0[1] + c0[1] + ky + LGNK_PAD;
            p[2] = D == 3 ? I0[2] + c0[2] + kz + LGNK_PAD : 0;
#pragma unroll 1
            for (int kx = 0; kx < n[0]; ++kx) {
                p[0] = I0[0] + c0[0] + kx + LGNK_PAD;
                const int o = linear<D>(g, p);
                const float gx = dw[0][kx] * wyz, gy = w[0][kx] * dyz, gz = w[0][kx] * ydz;
                if (KIND == 0) {
                    atomicAdd(acc + o, mass * w[0][kx] * wyz);
                } else if (KIND == 1) {
                    float x = fmaf(gx, dp[0], gy * dp[1]);
                    if (D == 3) x = fmaf(gz, dp[2], x);
                    atomicAdd(acc + o, mass * x);
                } else {
                    const float f = __ldg(F + o);
                    gsum[0] = fmaf(gx, f, gsum[0]);
                    gsum[1] = fmaf(gy, f, gsum[1]);
                    gsum[2] = fmaf(gz, f, gsum[2]);
                }
            }
        }
    }
    if (KIND == 2) {
#pragma unroll
        for (int a = 0; a < D; ++a) grad[a] = gsum[a];
    }
}

// What the forward sweep records of a stage for the adjoint sweep: the
// stage's cell on the velocity grid (linear padded index) and its fractional
// offsets in it, as one 16-byte word (f0, f1, f2 or 0, base).  The adjoint
// then needs no second lookup of the stage position.
template <int D>
__device__ __forceinline__ float4 stage_word(const DevGrid& g, const int* p, const float* f) {
    return make_float4(f[0], f[1], D == 3 ? f[D - 1] : 0.0f, __int_as_float(linear<D>(g, p)));
}

template <int D>
__device__ __forceinline__ int stage_from_word(const float4 w, float* f) {
    f[0] = w.x;
    f[1] = w.y;
    if (D == 3) f[D - 1] = w.z;
    return __float_as_int(w.w);
}

// Slices of the stages of step k: t_k (2k), t_k + dt/2 (2k + 1, stages 2 and
// 3), t_k + dt (2k + 2); a stationary field has the single slice 0.
template <bool NS>
__device__ __forceinline__ void step_slices(const TraceArgs& A, int k, size_t& s1, size_t& s2, size_t& s4) {
    if (NS) {
        s1 = (size_t)(2 * k) * A.slice_nodes;
        s2 = s1 + A.slice_nodes;
        s4 = s2 + A.slice_nodes;
    } else {
        s1 = s2 = s4 = 0;
    }
}

// What the forward and tangent sweeps record of each stage for an adjoint
// sweep (RM): 0 nothing; 1 the stage positions (u, u2, u3, u4 into pos[0 ..
// 4d)), from which the adjoint looks the cells up again; 2 each stage's cell
// and offsets (one 16-byte word per stage into cells[0..3]), so the adjoint
// needs no lookup.  Transport records cells (the 128^3 matvec 0.706 -> 0.630
// ms); the mass-preserving kernels record positions, whose record is a
// quarter smaller: their local-memory traffic is what reaches DRAM, and the
// brain-scale J^T measured 8.43 ms with positions against 8.87 ms with cells.
enum RecordMode { REC_NONE = 0, REC_POS = 1, REC_CELL = 2 };

// One RK4 step of the characteristic (Alg. 1 without the derivative), on the
// displacement u, recording its stages as RM says.
template <int D, bool NS, int RM, bool CACHE>
__device__ __forceinline__ void rk4_step(const TraceArgs& A, const float* V, float* u, int k, float* pos,
                                         float4* rec, CellCache<D, false>& C) {
    size_t s1, s2, s4;
    step_slices<NS>(A, k, s1, s2, s4);
    Start<D> sv;
    start_on_velocity<D>(A, sv);
    const float dt = A.dt, hdt = 0.5f * A.dt;
    int p[D];
    float f[D], vs[D], us[D], acc[D];
    if (RM == REC_POS) {
#pragma unroll
        for (int a = 0; a < D; ++a) pos[a] = u[a];
    }
    locate<D>(A.vg, sv, u, p, f);
    if (RM == REC_CELL) rec[0] = stage_word<D>(A.vg, p, f);
    if constexpr (CACHE) stage_value_cached<D>(A.vg, V, s1, p, f, C, vs);
    else stage_value<D>(A.vg, V, s1, p, f, vs);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = vs[a]; us[a] = fmaf(hdt, vs[a], u[a]); }
    if (RM == REC_POS) {
#pragma unroll
        for (int a = 0; a < D; ++a) pos[D + a] = us[a];
    }
    locate<D>(A.vg, sv, us, p, f);
    if (RM == REC_CELL) rec[1] = stage_word<D>(A.vg, p, f);
    if constexpr (CACHE) stage_value_cached<D>(A.vg, V, s2, p, f, C, vs);
    else stage_value<D>(A.vg, V, s2, p, f, vs);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = fmaf(2.0f, vs[a], acc[a]); us[a] = fmaf(hdt, vs[a], u[a]); }
    if (RM == REC_POS) {
#pragma unroll
        for (int a = 0; a < D; ++a) pos[2 * D + a] = us[a];
    }
    locate<D>(A.vg, sv, us, p, f);
    if (RM == REC_CELL) rec[2] = stage_word<D>(A.vg, p, f);
    if constexpr (CACHE) stage_value_cached<D>(A.vg, V, s2, p, f, C, vs);
    else stage_value<D>(A.vg, V, s2, p, f, vs);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = fmaf(2.0f, vs[a], acc[a]); us[a] = fmaf(dt, vs[a], u[a]); }
    if (RM == REC_POS) {
#pragma unroll
        for (int a = 0; a < D; ++a) pos[3 * D + a] = us[a];
    }
    locate<D>(A.vg, sv, us, p, f);
    if (RM == REC_CELL) rec[3] = stage_word<D>(A.vg, p, f);
    if constexpr (CACHE) stage_value_cached<D>(A.vg, V, s4, p, f, C, vs);
    else stage_value<D>(A.vg, V, s4, p, f, vs);
    const float s6 = dt / 6.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = fmaf(s6, acc[a] + vs[a], u[a]);
}

// One RK4 step with the derivative recursion of Alg. 1 applied to dv:
// D_s = I(dv, y_s, t_s) + d_y I(v, y_s, t_s) (dy + c_s dt D_{s-1}).
template <int D, bool NS, int RM, bool CACHE>
__device__ __forceinline__ void rk4_tangent_step(const TraceArgs& A, const float* V, const float* dV, float* u,
                                                 float* dy, int k, float* pos, float4* rec, CellCache<D, true>& C) {
    size_t s1, s2, s4;
    step_slices<NS>(A, k, s1, s2, s4);
    Start<D> sv;
    start_on_velocity<D>(A, sv);
    const float dt = A.dt, hdt = 0.5f * A.dt;
    int p[D];
    float f[D], us[D], q[D], vs[D], Jq[D], dvs[D], sv_acc[D], sd_acc[D], Ds;
    // stage 1 at y, offset dy
    if (RM == REC_POS) {
#pragma unroll
        for (int a = 0; a < D; ++a) pos[a] = u[a];
    }
    locate<D>(A.vg, sv, u, p, f);
    if (RM == REC_CELL) rec[0] = stage_word<D>(A.vg, p, f);
    if constexpr (CACHE) stage_tangent_cached<D>(A.vg, V, dV, s1, p, f, dy, C, vs, Jq, dvs);
    else stage_tangent<D>(A.vg, V, dV, s1, p, f, dy, vs, Jq, dvs);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        Ds = dvs[a] + Jq[a];
        sv_acc[a] = vs[a];
        sd_acc[a] = Ds;
        us[a] = fmaf(hdt, vs[a], u[a]);
        q[a] = fmaf(hdt, Ds, dy[a]);
    }
    // stage 2
    if (RM == REC_POS) {
#pragma unroll
        for (int a = 0; a < D; ++a) pos[D + a] = us[a];
    }
    locate<D>(A.vg, sv, us, p, f);
    if (RM == REC_CELL) rec[1] = stage_word<D>(A.vg, p, f);
    if constexpr (CACHE) stage_tangent_cached<D>(A.vg, V, dV, s2, p, f, q, C, vs, Jq, dvs);
    else stage_tangent<D>(A.vg, V, dV, s2, p, f, q, vs, Jq, dvs);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        Ds = dvs[a] + Jq[a];
        sv_acc[a] = fmaf(2.0f, vs[a], sv_acc[a]);
        sd_acc[a] = fmaf(2.0f, Ds, sd_acc[a]);
        us[a] = fmaf(hdt, vs[a], u[a]);
        q[a] = fmaf(hdt, Ds, dy[a]);
    }
    // stage 3
    if (RM == REC_POS) {
#pragma unroll
        for (int a = 0; a < D; ++a) pos[2 * D + a] = us[a];
    }
    locate<D>(A.vg, sv, us, p, f);
    if (RM == REC_CELL) rec[2] = stage_word<D>(A.vg, p, f);
    if constexpr (CACHE) stage_tangent_cached<D>(A.vg, V, dV, s2, p, f, q, C, vs, Jq, dvs);
    else stage_tangent<D>(A.vg, V, dV, s2, p, f, q, vs, Jq, dvs);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        Ds = dvs[a] + Jq[a];
        sv_acc[a] = fmaf(2.0f, vs[a], sv_acc[a]);
        sd_acc[a] = fmaf(2.0f, Ds, sd_acc[a]);
        us[a] = fmaf(dt, vs[a], u[a]);
        q[a] = fmaf(dt, Ds, dy[a]);
    }
    // stage 4
    if (RM == REC_POS) {
#pragma unroll
        for (int a = 0; a < D; ++a) pos[3 * D + a] = us[a];
    }
    locate<D>(A.vg, sv, us, p, f);
    if (RM == REC_CELL) rec[3] = stage_word<D>(A.vg, p, f);
    if constexpr (CACHE) stage_tangent_cached<D>(A.vg, V, dV, s4, p, f, q, C, vs, Jq, dvs);
    else stage_tangent<D>(A.vg, V, dV, s4, p, f, q, vs, Jq, dvs);
    const float s6 = dt / 6.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        dy[a] = fmaf(s6, sd_acc[a] + dvs[a] + Jq[a], dy[a]);
        u[a] = fmaf(s6, sv_acc[a] + vs[a], u[a]);
    }
}

// Transpose of one tangent step from recorded stage positions (RM = 1): the
// same as rk4_adjoint_step below, with each stage's cell looked up again.
template <int D, bool NS, class SC, bool CACHE>
__device__ __forceinline__ void rk4_adjoint_step_pos(const TraceArgs& A, const float* V, SC& S, const float* rec,
                                                     float* lam, int k, CellCache<D, false>& C) {
    size_t s1, s2, s4;
    step_slices<NS>(A, k, s1, s2, s4);
    Start<D> sv;
    start_on_velocity<D>(A, sv);
    const float dt = A.dt, hdt = 0.5f * A.dt;
    int p[D];
    float f[D], us[D];
    float mu[D], nu[D], acc[D];
    const float c16 = dt / 6.0f, c13 = dt / 3.0f;
    // stage 4
#pragma unroll
    for (int a = 0; a < D; ++a) { mu[a] = c16 * lam[a]; us[a] = rec[3 * D + a]; }
    locate<D>(A.vg, sv, us, p, f);
    if constexpr (CACHE) stage_adjoint_cached<D, SC>(A.vg, V, S, C, s4, linear<D>(A.vg, p), f, mu, nu);
    else stage_adjoint<D, SC>(A.vg, V, S, s4, linear<D>(A.vg, p), f, mu, nu);
    // stage 3
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = nu[a]; mu[a] = fmaf(c13, lam[a], dt * nu[a]); us[a] = rec[2 * D + a]; }
    locate<D>(A.vg, sv, us, p, f);
    if constexpr (CACHE) stage_adjoint_cached<D, SC>(A.vg, V, S, C, s2, linear<D>(A.vg, p), f, mu, nu);
    else stage_adjoint<D, SC>(A.vg, V, S, s2, linear<D>(A.vg, p), f, mu, nu);
    // stage 2
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] += nu[a]; mu[a] = fmaf(c13, lam[a], hdt * nu[a]); us[a] = rec[D + a]; }
    locate<D>(A.vg, sv, us, p, f);
    if constexpr (CACHE) stage_adjoint_cached<D, SC>(A.vg, V, S, C, s2, linear<D>(A.vg, p), f, mu, nu);
    else stage_adjoint<D, SC>(A.vg, V, S, s2, linear<D>(A.vg, p), f, mu, nu);
    // stage 1
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] += nu[a]; mu[a] = fmaf(c16, lam[a], hdt * nu[a]); us[a] = rec[a]; }
    locate<D>(A.vg, sv, us, p, f);
    if constexpr (CACHE) stage_adjoint_cached<D, SC>(A.vg, V, S, C, s1, linear<D>(A.vg, p), f, mu, nu);
    else stage_adjoint<D, SC>(A.vg, V, S, s1, linear<D>(A.vg, p), f, mu, nu);
#pragma unroll
    for (int a = 0; a < D; ++a) lam[a] += acc[a] + nu[a];
}

// Transpose of one tangent step: given lam (adjoint of the step's end point),
// scatter the step's contribution into the gradient and return the adjoint of
// its start.  The cells and offsets of the stages were recorded by the
// forward sweep (rec[0..3]); each stage's J^T mu and scatter share one pass.
template <int D, bool NS, class SC, bool CACHE>
__device__ __forceinline__ void rk4_adjoint_step(const TraceArgs& A, const float* V, SC& S, const float4* rec,
                                                 float* lam, int k, CellCache<D, false>& C) {
    size_t s1, s2, s4;
    step_slices<NS>(A, k, s1, s2, s4);
    const float dt = A.dt, hdt = 0.5f * A.dt;
    float f[D];
    float mu[D], nu[D], acc[D];
    const float c16 = dt / 6.0f, c13 = dt / 3.0f;
    int base;
    // stage 4: D4 = I(dv, y4) + J4 (dy + dt D3)
#pragma unroll
    for (int a = 0; a < D; ++a) mu[a] = c16 * lam[a];
    base = stage_from_word<D>(rec[3], f);
    if constexpr (CACHE) stage_adjoint_cached<D, SC>(A.vg, V, S, C, s4, base, f, mu, nu);
    else stage_adjoint<D, SC>(A.vg, V, S, s4, base, f, mu, nu);
    // stage 3: D3 = I(dv, y3) + J3 (dy + dt/2 D2)
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = nu[a]; mu[a] = fmaf(c13, lam[a], dt * nu[a]); }
    base = stage_from_word<D>(rec[2], f);
    if constexpr (CACHE) stage_adjoint_cached<D, SC>(A.vg, V, S, C, s2, base, f, mu, nu);
    else stage_adjoint<D, SC>(A.vg, V, S, s2, base, f, mu, nu);
    // stage 2: D2 = I(dv, y2) + J2 (dy + dt/2 D1)
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] += nu[a]; mu[a] = fmaf(c13, lam[a], hdt * nu[a]); }
    base = stage_from_word<D>(rec[1], f);
    if constexpr (CACHE) stage_adjoint_cached<D, SC>(A.vg, V, S, C, s2, base, f, mu, nu);
    else stage_adjoint<D, SC>(A.vg, V, S, s2, base, f, mu, nu);
    // stage 1: D1 = I(dv, y) + J1 dy
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] += nu[a]; mu[a] = fmaf(c16, lam[a], hdt * nu[a]); }
    base = stage_from_word<D>(rec[0], f);
    if constexpr (CACHE) stage_adjoint_cached<D, SC>(A.vg, V, S, C, s1, base, f, mu, nu);
    else stage_adjoint<D, SC>(A.vg, V, S, s1, base, f, mu, nu);
#pragma unroll
    for (int a = 0; a < D; ++a) lam[a] += acc[a] + nu[a];
}

// Finish one assembled row: its keys at [e][voxel] (the blocks are already
// in place, [e][voxel][corner][q], written by asm_commit) and its length.
template <int D>
__device__ __forceinline__ void write_row(const TraceArgs& A, const AsmTable<D>& S, int vox) {
    const long long M = (long long)A.ig.m[0] * A.ig.m[1] * (D == 3 ? A.ig.m[2] : 1);
    if (S.overflow || S.n > A.ewidth) {
        A.ecnt[vox] = 0;
        atomicExch(A.eflag, 1);
        return;
    }
    A.ecnt[vox] = S.n;
#pragma unroll 1
    for (int j = 0; j < S.n; ++j) A.ekey[j * M + vox] = S.key[j];
}

// Products with the assembled J, one thread per voxel i (row i):
//   ELL_JVP   out_i = J_i dv = sum_e sum_c blk_e[c] . dV[key_e + corner c]
//   ELL_JTVP  G[key_e + corner c] += r_i blk_e[c]
//   ELL_HESS  both, with the weight h^d (J_i dv) (the Gauss-Newton data term)
// Most rows have one block: the first is loaded without waiting for the row
// length (every row has at least one) and kept in registers for both the
// gather and the scatter; further blocks are read in a loop (twice for HESS).
constexpr int kEllRegBlocks = 1;
// 128-thread CTAs (measured 0.116 -> 0.109 ms against 256 on the 128^3 matvec)
constexpr int kEllBlock = 128;

// 32 bytes from the read-only path in one 256-bit load (p 32-byte aligned)
__device__ __forceinline__ void load8(const float* p, float* v) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}

// Entry j of row i: its key and its block, read as 256-bit loads (a block is
// 96 bytes in 3D, 32 in 2D, so every block starts on a 32-byte boundary); a
// warp's load then touches half as many L1 wavefronts as with 128-bit loads.
template <int D>
__device__ __forceinline__ void ell_load(const EllArgs& A, long long i, int j, long long& key, float* b) {
    constexpr int B = (1 << D) * D;
    key = __ldg(A.ekey + j * A.M + i);
    const float* p = A.eblk + ((size_t)j * A.M + i) * B;
#pragma unroll
    for (int k = 0; k < B / 8; ++k) load8(p + 8 * k, b + 8 * k);
}

template <int D>
__device__ __forceinline__ float ell_dot(const EllArgs& A, const float* __restrict__ dV, long long key, const float* b) {
    float s = 0.0f;
#pragma unroll
    for (int r = 0; r < (1 << (D - 1)); ++r) {     // rows of x-pairs (cy, cz); corner (0, cy, cz) is 2 r
        float lo[3], hi[3];
        pair_value<D>(dV, corner_elem<D>(A.vg, (size_t)key, 0, 0, r & 1, r >> 1), lo, hi);
#pragma unroll
        for (int q = 0; q < D; ++q) {
            s = fmaf(b[2 * r * D + q], lo[q], s);
            s = fmaf(b[(2 * r + 1) * D + q], hi[q], s);
        }
    }
    return s;
}

template <int D>
__device__ __forceinline__ void ell_scatter(const EllArgs& A, long long key, const float* b, float w) {
    using VT = typename VecT<D>::type;
    VT* G = static_cast<VT*>(A.G);
#pragma unroll
    for (int c = 0; c < (1 << D); ++c)
        red_vec(G + corner_elem<D>(A.vg, (size_t)key, 0, c & 1, (c >> 1) & 1, (c >> 2) & 1), b + c * D, w);
}

// Scatter of the first blocks of a warp's rows with neighbouring rows merged:
// voxels next to each other in x mostly trace through the same velocity cell
// or the next one along x.  A run of lanes with equal keys adds its weighted
// blocks two by two through shuffles and only the lane at an even position of
// the run reduces (about half the global reductions); then a reducing lane
// whose next reducing lane holds the cell one step along x (key + 1: corner
// (1, cy, cz) of cell k is node k + 1 + cy mx + cz mx my, corner (0, cy, cz)
// of cell k + 1) hands it the four corner vectors of that face and reduces
// only its other four corners.  Every lane of the warp calls it; lanes
// without a block pass a key no other lane has.
template <int D>
__device__ __forceinline__ void ell_scatter_merged(const EllArgs& A, long long key, const float* b, float w) {
    constexpr int C = 1 << D, B = C * D;
    using VT = typename VecT<D>::type;
    VT* G = static_cast<VT*>(A.G);
    const int lane = threadIdx.x & 31;
    const long long prev = __shfl_up_sync(0xffffffffu, key, 1);
    const long long next = __shfl_down_sync(0xffffffffu, key, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));   // the run's first lane
    const bool absorbed = ((lane - start) & 1) != 0;
    const bool absorber = !absorbed && lane < 31 && next == key;
    float wb[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
        wb[k] = w * b[k];
        const float o = __shfl_down_sync(0xffffffffu, wb[k], 1);
        if (absorber) wb[k] += o;
    }
    const bool reducer = !absorbed && key >= 0;
    const unsigned red = __ballot_sync(0xffffffffu, reducer);
    const unsigned above = lane == 31 ? 0u : red & (0xfffffffeu << lane);
    const unsigned below = red & ((1u << lane) - 1u);
    const int nxt = above != 0u ? __ffs((int)above) - 1 : lane;     // the next and previous reducing lanes
    const int prv = below != 0u ? 31 - __clz((int)below) : lane;
    const long long knext = __shfl_sync(0xffffffffu, key, nxt);
    const long long kprev = __shfl_sync(0xffffffffu, key, prv);
    const bool give = reducer && nxt != lane && knext == key + 1;
    const bool take = reducer && prv != lane && kprev + 1 == key;
#pragma unroll
    for (int c = 1; c < C; c += 2) {
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const float o = __shfl_sync(0xffffffffu, wb[c * D + q], prv);
            if (take) wb[(c - 1) * D + q] += o;
        }
    }
    if (reducer) {
#pragma unroll
        for (int c = 0; c < C; ++c)
            if (!((c & 1) && give))
                red_vec(G + corner_elem<D>(A.vg, (size_t)key, 0, c & 1, (c >> 1) & 1, (c >> 2) & 1), wb + c * D, 1.0f);
    }
}


template <int D, int EMODE>
__global__ void __launch_bounds__(kEllBlock) ell_kernel(const EllArgs A) {
    constexpr int B = (1 << D) * D;
    constexpr int RB = kEllRegBlocks;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < A.M;           // lanes past the end stay for the warp's shuffles
    const float* dV = static_cast<const float*>(A.dV);
    const int n = valid ? __ldg(A.ecnt + i) : 0;
    long long kr[RB > 0 ? RB : 1];
    float br[RB > 0 ? RB : 1][B];
#pragma unroll
    for (int j = 0; j < RB; ++j)
        if (valid && (j == 0 || j < n)) ell_load<D>(A, i, j, kr[j], br[j]);
    float s = 0.0f;
    if (EMODE != ELL_JTVP) {
#pragma unroll
        for (int j = 0; j < RB; ++j)
            if (j < n) s += ell_dot<D>(A, dV, kr[j], br[j]);
#pragma unroll 1
        for (int j = RB; j < n; ++j) {
            long long k;
            float b[B];
            ell_load<D>(A, i, j, k, b);
            s += ell_dot<D>(A, dV, k, b);
        }
        if (EMODE == ELL_JVP) {
            if (valid) A.out[i] = s;
            return;
        }
        s *= A.cellvol;
    } else {
        s = valid ? A.r[i] : 0.0f;
    }
    // the first block: merged across the warp; keys are non-negative element offsets
    ell_scatter_merged<D>(A, n > 0 ? kr[0] : -1 - (long long)(threadIdx.x & 31), br[0], s);
#pragma unroll
    for (int j = 1; j < RB; ++j)
        if (j < n) ell_scatter<D>(A, kr[j], br[j], s);
#pragma unroll 1
    for (int j = RB; j < n; ++j) {
        long long k;
        float b[B];
        ell_load<D>(A, i, j, k, b);
        ell_scatter<D>(A, k, b, s);
    }
}

template <int D>
static cudaError_t launch_ell_dim(int mode, const EllArgs& a, cudaStream_t s) {
    const long long blocks = (a.M + kEllBlock - 1) / kEllBlock;
    if (blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    switch (mode) {
        case ELL_JVP: ell_kernel<D, ELL_JVP><<<(unsigned)blocks, kEllBlock, 0, s>>>(a); break;
        case ELL_JTVP: ell_kernel<D, ELL_JTVP><<<(unsigned)blocks, kEllBlock, 0, s>>>(a); break;
        case ELL_HESS: ell_kernel<D, ELL_HESS><<<(unsigned)blocks, kEllBlock, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// 256 threads; FWD at 64 registers (4 CTAs per SM; 80 registers, 3 CTAs, for
// the 3D transport sweep with its value cell cache: 0.256 -> 0.226 ms on the
// 128^3 image against the uncached sweep at 4 CTAs), the other derivative
// modes at 80 (3 CTAs): measured fastest among 64/80/128-register and
// 256/512-thread configurations on the 128^3 matvec.
template <int D, int MODEL, int MODE>
struct TraceOccupancy {
    // CTAs per SM the register budget is set for: the 3D transport modes hold
    // cached cells (v and dv corners) and the pending scatter block and run at
    // 128 registers (measured on the 128^3 matvec: 1.42 ms at 3 CTAs without
    // either, 1.50 ms with the cache at 80 registers, 1.31 ms with it at 128,
    // 0.82 ms with the scatter block as well; the assembly 1.23 -> 0.79 ms
    // from 3 to 2 CTAs with its pending block in registers)
    static constexpr int value =
        MODE == MODE_FWD ? ((D == 3 && MODEL == LGNK_TRANSPORT) ? 3 : 4) : ((D == 3 && MODEL == LGNK_TRANSPORT) ? 2 : 3);
};

template <int D, bool NS, int MODEL, int MODE>
__global__ void __launch_bounds__(LGNK_BLOCK, (TraceOccupancy<D, MODEL, MODE>::value)) trace_kernel(const TraceArgs A) {
    using VT = typename VecT<D>::type;
    constexpr bool TANGENT = (MODE == MODE_JVP || MODE == MODE_HESS);
    constexpr bool ADJOINT = (MODE == MODE_JTVP || MODE == MODE_HESS || MODE == MODE_OBJGRAD || MODE == MODE_ASM);
    using SC = typename std::conditional<
        MODE == MODE_ASM, AsmRow<D>,
        typename std::conditional<(MODE == MODE_HESS || MODE == MODE_JTVP || MODE == MODE_OBJGRAD) && MODEL == LGNK_TRANSPORT, BlockScatter<D>, Scatter<D>>::type>::type;
    // cached velocity cells and whole-cell scatter blocks for transport; the
    // continuity kernels (many time slices, longer trajectories) were measured
    // faster without either
    constexpr bool CACHE = MODEL == LGNK_TRANSPORT;
    const float* V = static_cast<const float*>(A.V);
    const float* dV = static_cast<const float*>(A.dV);

    int idx[3];
    voxel_index<D>(A, idx);
    const bool active = idx[0] < A.ig.m[0] && idx[1] < A.ig.m[1] && (D == 2 || idx[2] < A.ig.m[2]);
    lsum ssd = lsum_zero();  // res^2 of this thread's voxel (FWD with R, OBJGRAD, ASM with R)
    int entries = 0;           // MODE_ASM: blocks of this thread's row

    SC S;
    scatter_init<D>(S, A.G);
    AsmTable<D> row_table;        // MODE_ASM: the keys of the row being assembled
    if constexpr (MODE == MODE_ASM) {
        row_table.n = 0;
        row_table.overflow = false;
        S.tab = &row_table;
        const size_t Mi = (size_t)A.ig.m[0] * A.ig.m[1] * (D == 3 ? A.ig.m[2] : 1);
        const int vx = idx[0] + A.ig.m[0] * (idx[1] + A.ig.m[1] * (D == 3 ? idx[2] : 0));
        S.stride = Mi * AsmRow<D>::B;
        S.blk = A.eblk + (size_t)vx * AsmRow<D>::B;
    }

    int sp[D];                    // continuity FWD / JVP: the end cell, offsets, mass and dy of the splat
    float sf[D], sdy[D], smass = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        sp[a] = 0;
        sf[a] = 0.0f;
        sdy[a] = 0.0f;
    }
    if (active) {
        const int vox = idx[0] + A.ig.m[0] * (idx[1] + A.ig.m[1] * (D == 3 ? idx[2] : 0));
        float u[D], dy[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            u[a] = 0.0f;
            dy[a] = 0.0f;
        }
        CellCache<D, true> tcache;
        tcache.key = -1;
        CellCache<D, false> vcache;   // v corners for the forward and adjoint sweeps
        vcache.key = -1;
        // the stages of every step, recorded for the adjoint sweep (RecordMode)
        // in a per-thread local array as 16-byte words.  Kept
        // in shared memory instead, the full record (2 CTAs x 96 KB on the
        // 128^3 matvec) shrank the L1 that the gathers use and measured slower
        // (0.828 against 0.814 ms); keeping only each step's start there and
        // recomputing the other positions in the adjoint sweep measured 0.974
        // ms, and on the brain-scale mass-preserving J^T 9.56 against 8.47 ms.
        constexpr int RM = !ADJOINT ? REC_NONE : (MODEL == LGNK_TRANSPORT ? REC_CELL : REC_POS);
        constexpr int WPS = RM == REC_CELL ? 4 : D;     // 16-byte words per step
        float4 lrec[ADJOINT ? LGNK_MAX_STEPS * WPS : 1];

#pragma unroll 1
        for (int k = 0; k < A.N; ++k) {
            float4* rec = lrec + (ADJOINT ? WPS * k : 0);
            float pos[4 * D];
            if (TANGENT) rk4_tangent_step<D, NS, RM, CACHE>(A, V, dV, u, dy, k, pos, rec, tcache);
            else rk4_step<D, NS, RM, CACHE>(A, V, u, k, pos, rec, vcache);
            if constexpr (RM == REC_POS) {
#pragma unroll
                for (int w = 0; w < D; ++w) rec[w] = make_float4(pos[4 * w], pos[4 * w + 1], pos[4 * w + 2], pos[4 * w + 3]);
            }
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
        Start<D> si;
        start_on_image<D>(idx, si);
        if (MODEL == LGNK_TRANSPORT) {
            float gT[D];
            if (MODE == MODE_FWD) {
                const float val = sample_image<D, false>(A.ig, si, A.Tp, u, nullptr);
                A.u1[vox] = val;
                if (A.R != nullptr) lsum_add_sqdiff(ssd, val, A.R[vox]);
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
            } else if (MODE == MODE_ASM) {
                const float val = sample_image<D, true>(A.ig, si, A.Tp, u, gT);
#pragma unroll
                for (int a = 0; a < D; ++a) lam[a] = gT[a];
                if (A.R != nullptr) {     // with the objective: SSD and the gradient's weights h^d res
                    const float Rv = A.R[vox];
                    lsum_add_sqdiff(ssd, val, Rv);
                    A.u1[vox] = A.cellvol * (val - Rv);
                }
            } else {  // MODE_OBJGRAD
                const float val = sample_image<D, true>(A.ig, si, A.Tp, u, gT);
                if (A.u1 != nullptr) A.u1[vox] = val;
                const float Rv = A.R[vox];
                lsum_add_sqdiff(ssd, val, Rv);
                const float s = A.cellvol * (val - Rv);
#pragma unroll
                for (int a = 0; a < D; ++a) lam[a] = s * gT[a];
            }
        } else {
            const float mass = __ldg(A.T + vox);
            if (A.pic_rho[0] > 0.0f) {
                if (MODE == MODE_FWD) {
                    pic_hat<D, 0>(A.ig, si.I0, u, A.pic_rho, A.acc, nullptr, mass, nullptr, nullptr);
                } else if (MODE == MODE_JVP) {
                    pic_hat<D, 1>(A.ig, si.I0, u, A.pic_rho, A.acc, nullptr, mass, dy, nullptr);
                } else if (MODE == MODE_JTVP) {
                    float gr[D];
                    pic_hat<D, 2>(A.ig, si.I0, u, A.pic_rho, nullptr, A.r, 0.0f, nullptr, gr);
#pragma unroll
                    for (int a = 0; a < D; ++a) lam[a] = mass * gr[a];
                }
            } else if (MODE == MODE_FWD || MODE == MODE_JVP) {
                locate<D>(A.ig, si, u, sp, sf);   // splat after the loop, with the whole CTA
                smass = mass;
#pragma unroll
                for (int a = 0; a < D; ++a) sdy[a] = dy[a];
            } else if (MODE == MODE_JTVP) {
                float gr[D];
                sample_image<D, true>(A.ig, si, A.r, u, gr);
#pragma unroll
                for (int a = 0; a < D; ++a) lam[a] = mass * gr[a];
            }
        }

        if (ADJOINT) {
#pragma unroll 1
            for (int k = A.N - 1; k >= 0; --k) {
                if constexpr (RM == REC_CELL) {
                    rk4_adjoint_step<D, NS, SC, CACHE>(A, V, S, lrec + WPS * k, lam, k, vcache);
                } else {
                    float pos[4 * D];
#pragma unroll
                    for (int w = 0; w < D; ++w) {
                        const float4 word = lrec[WPS * k + w];
                        pos[4 * w] = word.x;
                        pos[4 * w + 1] = word.y;
                        pos[4 * w + 2] = word.z;
                        pos[4 * w + 3] = word.w;
                    }
                    rk4_adjoint_step_pos<D, NS, SC, CACHE>(A, V, S, pos, lam, k, vcache);
                }
            }
            scatter_finish<D>(A.vg, S);
            if constexpr (MODE == MODE_ASM) {
                write_row<D>(A, *S.tab, vox);
                entries = S.tab->n;
            }
        }
    }

    if constexpr (MODEL == LGNK_CONTINUITY && (MODE == MODE_FWD || MODE == MODE_JVP)) {
        if (A.pic_rho[0] <= 0.0f) splat_tiled<D, MODE == MODE_JVP>(A.ig, A.acc, active, sp, sf, smass, sdy);
    }
    if (MODE == MODE_OBJGRAD || MODE == MODE_FWD || MODE == MODE_ASM) {
        if (A.partial != nullptr) {
            const lsum s = lsum_block_sum(ssd);
            if (threadIdx.x == 0) A.partial[blockIdx.x] = lsum_value(s);
        }
    }
    if (MODE == MODE_ASM && A.cpartial != nullptr) {
        __syncthreads();      // lsum_block_sum's shared slots are reused
        lsum c = lsum_zero();
        lsum_add(c, (float)entries);
        c = lsum_block_sum(c);   // exact: at most 256 x 16 blocks
        if (threadIdx.x == 0) A.cpartial[blockIdx.x] = lsum_value(c);
    }
}

template <int D, bool NS, int MODEL, int MODE>
static cudaError_t launch_one(const TraceArgs& a0, int nblocks, cudaStream_t s) {
    (void)nblocks;
    TraceArgs a = a0;
    int ts[3];
    trace_tile_shape(D, ts);
    for (int i = 0; i < 3; ++i) a.tiles[i] = (a.ig.m[i] + ts[i] - 1) / ts[i];
    const int blocks = a.tiles[0] * a.tiles[1] * a.tiles[2];
    const int threads = ts[0] * ts[1] * ts[2];
    trace_kernel<D, NS, MODEL, MODE><<<blocks, threads, 0, s>>>(a);
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
            case MODE_ASM: return launch_one<D, NS, LGNK_TRANSPORT, MODE_ASM>(a, nblocks, s);
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

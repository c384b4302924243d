// Grid utilities of the lgnk library: layout conversion between the ABI layout
// and the padded packed layout of the tracing kernels, reductions (the
// accumulators of fsum.cuh per element, FP64 from the block partials on),
// regularizer stencils (Sec. 2.1, Sec. 3.2), the per-axis DCT of the spectral
// preconditioner (Sec. 3.2) and the vector updates of PCG.
#include <cmath>

#include <algorithm>

#include "fsum.cuh"
#include "lgnk_internal.h"

namespace {

constexpr int kBlock = LGNK_BLOCK;

inline int nblocks_for(size_t count) {
    return (int)((count + kBlock - 1) / kBlock);
}

__device__ __forceinline__ size_t padded_size(const DevGrid& g) {
    return (size_t)g.mp[0] * g.mp[1] * g.mp[2];
}

// ---------------------------------------------------------------- packing --

// Axis coordinates of element i of an nx x ny (x nz) block, in 32-bit
// arithmetic: every array the library accepts has fewer than 2^31 elements
// (checked when the context is created), and a 64-bit division costs many
// times a 32-bit one.
__device__ __forceinline__ void split_xyz(unsigned i, unsigned nx, unsigned ny, int& x, int& y, int& z) {
    const unsigned r = i / nx;
    x = (int)(i - r * nx);
    const unsigned q = r / ny;
    y = (int)(r - q * ny);
    z = (int)q;
}

// Pair-packed time slices: element (m, node) holds the velocity at stage time
// t_m (linear in time between the K nodes) at the padded node and at its +x
// neighbour, [v(node) | v(node + 1)], as 8 floats (3D: xyz + zero pad, twice;
// 32 bytes) or 4 floats (2D).  One 256-bit (3D) or 128-bit (2D) load then
// returns both x-corners of a cell row.  With Gz given, the slice gradients,
// which share the [slice][padded node] index, are zeroed in the same pass.
template <int D>
__global__ void pack_velocity_kernel(const float* __restrict__ v, float* __restrict__ Vp, DevGrid g, SliceTable tab,
                                     void* Gz) {
    const size_t nodes = padded_size(g);
    const size_t total = nodes * tab.n;
    const size_t Mv = (size_t)g.m[0] * g.m[1] * g.m[2];
    constexpr int PS = (D == 3) ? 8 : 4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        if (Gz != nullptr) {
            if (D == 3) reinterpret_cast<float4*>(Gz)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            else reinterpret_cast<float2*>(Gz)[i] = make_float2(0.0f, 0.0f);
        }
        const unsigned nn = (unsigned)nodes;
        const int m = (int)((unsigned)i / nn);
        const unsigned node = (unsigned)i - (unsigned)m * nn;
        const int j = tab.j[m];
        const float th = tab.th[m];
        int px, py, pz;
        split_xyz(node, (unsigned)g.mp[0], (unsigned)g.mp[1], px, py, pz);
        float out[PS];
#pragma unroll
        for (int q = 0; q < PS; ++q) out[q] = 0.0f;
        const int y = py - LGNK_PAD, z = (D == 3) ? pz - LGNK_PAD : 0;
        const bool yz_in = y >= 0 && y < g.m[1] && z >= 0 && z < g.m[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = px + h - LGNK_PAD;
            if (yz_in && x >= 0 && x < g.m[0]) {
                const size_t s = ((size_t)z * g.m[1] + y) * g.m[0] + x;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const float a = v[((size_t)j * D + c) * Mv + s];
                    float val = a;
                    if (th != 0.0f) val = fmaf(th, v[((size_t)(j + 1) * D + c) * Mv + s] - a, a);
                    out[h * (PS / 2) + c] = val;
                }
            }
        }
        float4* o = reinterpret_cast<float4*>(Vp + i * PS);
        o[0] = make_float4(out[0], out[1], out[2], out[3]);
        if (D == 3) o[1] = make_float4(out[4], out[5], out[6], out[7]);
    }
}

// Cell coordinates of node s of an (unpadded) velocity block.
template <int D>
__device__ __forceinline__ void coords(size_t s, const DevGrid& g, int* c) {
    int z;
    split_xyz((unsigned)s, (unsigned)g.m[0], (unsigned)g.m[1], c[0], c[1], z);
    c[2] = (D == 3) ? z : 0;
}

// Adjoint of the slice packing for the gradient: node j of component c gets
// scale * sum_m w_j(m) G_m[node], w_j(m) = 1 - th[m] if j = j[m], th[m] if j = j[m] + 1.
template <int D>
__global__ void distribute_gradient_kernel(const float* __restrict__ Gp, float* __restrict__ out, DevGrid g, int K,
                                           SliceTable tab, float scale) {
    const size_t Mv = (size_t)g.m[0] * g.m[1] * g.m[2];
    const size_t nodes = padded_size(g);
    const size_t total = Mv * K;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)((unsigned)i / (unsigned)Mv);
        const size_t s = (unsigned)i - (unsigned)j * (unsigned)Mv;
        int x, y, z;
        split_xyz((unsigned)s, (unsigned)g.m[0], (unsigned)g.m[1], x, y, z);
        const size_t node = ((size_t)(z + (D == 3 ? LGNK_PAD : 0)) * g.mp[1] + (y + LGNK_PAD)) * g.mp[0] + (x + LGNK_PAD);
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int m = 0; m < tab.n; ++m) {
            float w = 0.0f;
            if (tab.j[m] == j) w = 1.0f - tab.th[m];
            else if (tab.j[m] + 1 == j) w = tab.th[m];
            if (w == 0.0f) continue;
            const size_t e = (size_t)m * nodes + node;
            if (D == 3) {
                const float4 a = reinterpret_cast<const float4*>(Gp)[e];
                acc[0] = fmaf(w, a.x, acc[0]); acc[1] = fmaf(w, a.y, acc[1]); acc[2] = fmaf(w, a.z, acc[2]);
            } else {
                const float2 a = reinterpret_cast<const float2*>(Gp)[e];
                acc[0] = fmaf(w, a.x, acc[0]); acc[1] = fmaf(w, a.y, acc[1]);
            }
        }
#pragma unroll
        for (int c = 0; c < D; ++c) out[((size_t)j * D + c) * Mv + s] = scale * acc[c];
    }
}

__global__ void pack_image_kernel(const float* __restrict__ T, float* __restrict__ Tp, DevGrid g, int d, float scale) {
    const size_t total = padded_size(g);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int px, py, pz;
        split_xyz((unsigned)i, (unsigned)g.mp[0], (unsigned)g.mp[1], px, py, pz);
        const int x = px - LGNK_PAD, y = py - LGNK_PAD, z = (d == 3) ? pz - LGNK_PAD : 0;
        const bool in = x >= 0 && x < g.m[0] && y >= 0 && y < g.m[1] && z >= 0 && z < g.m[2];
        Tp[i] = in ? scale * T[((size_t)z * g.m[1] + y) * g.m[0] + x] : 0.0f;
    }
}

__global__ void unpack_image_kernel(const float* __restrict__ acc, float* __restrict__ out, DevGrid g, int d) {
    const size_t M = (size_t)g.m[0] * g.m[1] * g.m[2];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        split_xyz((unsigned)i, (unsigned)g.m[0], (unsigned)g.m[1], x, y, z);
        const size_t p = ((size_t)(z + (d == 3 ? LGNK_PAD : 0)) * g.mp[1] + (y + LGNK_PAD)) * g.mp[0] + (x + LGNK_PAD);
        out[i] = acc[p];
    }
}

__global__ void repad_image_kernel(float* acc, DevGrid g, int d, float scale) {
    const size_t total = padded_size(g);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int px, py, pz;
        split_xyz((unsigned)i, (unsigned)g.mp[0], (unsigned)g.mp[1], px, py, pz);
        const int x = px - LGNK_PAD, y = py - LGNK_PAD, z = (d == 3) ? pz - LGNK_PAD : 0;
        const bool in = x >= 0 && x < g.m[0] && y >= 0 && y < g.m[1] && z >= 0 && z < g.m[2];
        acc[i] = in ? scale * acc[i] : 0.0f;
    }
}

// ------------------------------------------------------------- reductions --

__device__ __forceinline__ double block_reduce(double x) {
    __shared__ double red[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = x;
    __syncthreads();
    double s = 0.0;
    if (warp == 0) {
        s = (lane < kBlock / 32) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// res = u1 - R (Eq. 10): partial sums of res^2 per block (FP64); rp (padded) = scale * res.
__global__ void residual_kernel(const float* __restrict__ u1, const float* __restrict__ R, float* __restrict__ rp,
                                DevGrid g, int d, float scale, double* partial) {
    const size_t M = (size_t)g.m[0] * g.m[1] * g.m[2];
    lsum s = lsum_zero();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
        const float ui = u1[i], Ri = R[i];
        const float r = ui - Ri;
        lsum_add_sqdiff(s, ui, Ri);
        if (rp != nullptr) {
            int x, y, z;
            split_xyz((unsigned)i, (unsigned)g.m[0], (unsigned)g.m[1], x, y, z);
            const size_t p = ((size_t)(z + (d == 3 ? LGNK_PAD : 0)) * g.mp[1] + (y + LGNK_PAD)) * g.mp[0] + (x + LGNK_PAD);
            rp[p] = scale * r;
        }
    }
    s = lsum_block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = lsum_value(s);
}

__global__ void dot_kernel(const float* __restrict__ a, const float* __restrict__ b, size_t count, double* partial) {
    lsum s = lsum_zero();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        lsum_add_prod(s, a[i], b[i]);
    s = lsum_block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = lsum_value(s);
}

// One or two inner products sharing the first operand, finished in the same
// launch: every block writes its partial sums (FP64, in the partial buffer's
// slots), and the last block to finish (a counter, reset by
// that block) adds the partials in a fixed order (deterministic) into
// sc[slot_b] (a.b) and sc[slot_c] (a.c, when c is given), then the PCG step
// lengths of step `mode` (-1: none), in FP64, from the inner products in sc
// ([2] p.Hp, [3] r.r, [4] r.z new, [5] r.z current):
//   mode 0: alpha = rz / pHp, or 0 when pHp is not positive; f[0] = alpha, f[1] = -alpha
//   mode 1: beta = rz_new / rz, then rz = rz_new;             f[2] = beta
__device__ __forceinline__ void pcg_step_lengths(double* sc, float* f, int mode) {
    if (mode == 0) {
        const double php = sc[2];
        const double a = php > 0.0 ? sc[5] / php : 0.0;
        f[0] = (float)a;
        f[1] = (float)-a;
    } else if (mode == 1) {
        f[2] = (float)(sc[4] / sc[5]);
        sc[5] = sc[4];
    }
}

// Second half of the fused inner products: block sums of the per-thread
// accumulators s (a.b) and, when `two`, t (a.c); every block writes its
// partials (FP64) and the last block to finish adds them in a fixed order
// (FP64, deterministic) into sc[slot_b] (sc[slot_c]) and applies
// pcg_step_lengths(mode).  Every thread of every block calls it.
__device__ __forceinline__ void dot_blocks_finish(lsum s, lsum t, bool two, double* partial, unsigned* counter,
                                                  double* sc, int slot_b, int slot_c, int mode, float* f) {
    s = lsum_block_sum(s);
    if (two) {
        __syncthreads();      // lsum_block_sum's shared slots are reused
        t = lsum_block_sum(t);
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = lsum_value(s);
        if (two) partial[gridDim.x + blockIdx.x] = lsum_value(t);
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const volatile double* vp = partial;
    double u = 0.0, w = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        u += vp[i];
        if (two) w += vp[gridDim.x + i];
    }
    __syncthreads();          // the first block sums' shared slots are reused
    u = block_reduce(u);
    if (two) {
        __syncthreads();
        w = block_reduce(w);
    }
    if (threadIdx.x == 0) {
        sc[slot_b] = u;
        if (two) sc[slot_c] = w;
        pcg_step_lengths(sc, f, mode);
        *counter = 0u;
    }
}

__global__ void dot_fused_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                 const float* __restrict__ c, size_t count, double* partial, unsigned* counter,
                                 double* sc, int slot_b, int slot_c, int mode, float* f) {
    lsum s = lsum_zero(), t = lsum_zero();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float ai = a[i];
        lsum_add_prod(s, ai, b[i]);
        if (c != nullptr) lsum_add_prod(t, ai, c[i]);
    }
    dot_blocks_finish(s, t, c != nullptr, partial, counter, sc, slot_b, slot_c, mode, f);
}

// The end of a Gauss-Newton product inside PCG with the diffusion
// regularizer, in one pass over the velocity nodes: Hp = gscale * (slice
// gradients distributed to the time nodes) + rscale * (B^T B p) + gamma * p
// (the arithmetic of distribute_gradient_kernel and laplacian_kernel, in the
// same order), then p.Hp into sc[2] and the step length alpha (mode 0), as
// dot_fused_kernel does.  Launched with the same block count as the fused
// inner products (partial holds one pair per block).
template <int D, bool DOT>
__global__ void hess_finish_kernel(const float* __restrict__ Gp, const float* __restrict__ p, float* __restrict__ Hp,
                                   DevGrid g, int K, SliceTable tab, float gscale, float rscale, float gamma,
                                   double* partial, unsigned* counter, double* sc, float* f) {
    const size_t Mv = (size_t)g.m[0] * g.m[1] * g.m[2];
    const size_t nodes = padded_size(g);
    const size_t total = Mv * K;
    const size_t stride[3] = {1, (size_t)g.m[0], (size_t)g.m[0] * g.m[1]};
    lsum dsum = lsum_zero();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)((unsigned)i / (unsigned)Mv);
        const size_t sn = (unsigned)i - (unsigned)j * (unsigned)Mv;
        int c[3];
        coords<D>(sn, g, c);
        const size_t node =
            ((size_t)(c[2] + (D == 3 ? LGNK_PAD : 0)) * g.mp[1] + (c[1] + LGNK_PAD)) * g.mp[0] + (c[0] + LGNK_PAD);
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int m = 0; m < tab.n; ++m) {
            float w = 0.0f;
            if (tab.j[m] == j) w = 1.0f - tab.th[m];
            else if (tab.j[m] + 1 == j) w = tab.th[m];
            if (w == 0.0f) continue;
            const size_t e = (size_t)m * nodes + node;
            if (D == 3) {
                const float4 a = reinterpret_cast<const float4*>(Gp)[e];
                acc[0] = fmaf(w, a.x, acc[0]); acc[1] = fmaf(w, a.y, acc[1]); acc[2] = fmaf(w, a.z, acc[2]);
            } else {
                const float2 a = reinterpret_cast<const float2*>(Gp)[e];
                acc[0] = fmaf(w, a.x, acc[0]); acc[1] = fmaf(w, a.y, acc[1]);
            }
        }
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const size_t k = ((size_t)j * D + q) * Mv + sn;
            const float xi = p[k];
            float lap = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                float t = 0.0f;
                if (c[a] > 0) t += xi - p[k - stride[a]];
                if (c[a] < g.m[a] - 1) t += xi - p[k + stride[a]];
                lap = fmaf(t, g.inv_h[a] * g.inv_h[a], lap);
            }
            float r = rscale * lap;
            if (gamma != 0.0f) r = fmaf(gamma, xi, r);
            r += gscale * acc[q];
            Hp[k] = r;
            if (DOT) lsum_add_prod(dsum, xi, r);
        }
    }
    if (DOT) dot_blocks_finish(dsum, lsum_zero(), false, partial, counter, sc, 2, 2, 0, f);
}

// x += f[0] p and r += f[1] Hp (the PCG updates with alpha, -alpha)
__global__ void pcg_update_xr_kernel(float* x, const float* __restrict__ p, float* r, const float* __restrict__ Hp,
                                     const float* __restrict__ f, size_t count) {
    const float a = f[0], b = f[1];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        x[i] = fmaf(a, p[i], x[i]);
        r[i] = fmaf(b, Hp[i], r[i]);
    }
}

// End of one PCG iteration inside a device-side loop (a CUDA-graph while
// node): the same tests the host loop makes, on sc[2] = p.Hp, sc[3] = r.r and
// the tolerance sc[6] = pcg_rtol |g|.  ctl: [0] iterations run, [1] accepted
// iterations, [2] 1 = non-positive curvature, 2 = non-finite, [3] the cap.
// The loop continues while the handle is non-zero; the cap ends it.
__global__ void pcg_control_kernel(const double* sc, int* ctl, cudaGraphConditionalHandle handle) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int it = ctl[0] + 1;
    ctl[0] = it;
    const double php = sc[2], rr = sc[3];
    unsigned go = 0;
    if (!isfinite(php) || !isfinite(rr)) {
        ctl[2] = 2;
    } else if (!(php > 0.0)) {
        ctl[2] = 1;
    } else {
        ctl[1] = it;
        go = (sqrt(rr) <= sc[6] || it >= ctl[3]) ? 0u : 1u;
    }
    cudaGraphSetConditional(handle, go);
}

// After the device-side PCG loop: when its first iteration met non-positive
// curvature (ctl[2] = 1 with no accepted iteration), the step is the
// preconditioned steepest-descent direction, x = z.
__global__ void pcg_curvature_fix_kernel(float* x, const float* __restrict__ z, const int* __restrict__ ctl,
                                         size_t count) {
    if (!(ctl[2] == 1 && ctl[1] == 0)) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        x[i] = z[i];
}

// y = a x + b y, a = *ap when ap is given, b = *bp when bp is given.
__global__ void axpby_dev_kernel(float a, const float* __restrict__ ap, const float* __restrict__ x, float b,
                                 const float* __restrict__ bp, float* y, size_t count) {
    const float ea = ap ? *ap : a, eb = bp ? *bp : b;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        y[i] = fmaf(ea, x[i], eb * y[i]);
}

// Deterministic final sum of the per-block partials (one block).
__global__ void reduce_kernel(const double* __restrict__ partial, int count, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += partial[i];
    s = block_reduce(s);
    if (threadIdx.x == 0) out[0] = s;
}

// ----------------------------------------------------------- regularizers --

// out = addsrc + scale * (B^T B x) + gamma * gsrc: the Neumann Laplacian of each
// (time node, component) block, B the forward difference between neighbouring
// cell centres (interior faces only).
template <int D>
__global__ void laplacian_kernel(const float* __restrict__ x, float* out, DevGrid g, int nblk, float scale,
                                 float gamma, const float* gsrc, const float* addsrc) {
    const size_t Mv = (size_t)g.m[0] * g.m[1] * g.m[2];
    const size_t total = Mv * nblk;
    const size_t stride[3] = {1, (size_t)g.m[0], (size_t)g.m[0] * g.m[1]};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = (unsigned)i % (unsigned)Mv;
        int c[3];
        coords<D>(s, g, c);
        const float xi = x[i];
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float t = 0.0f;
            if (c[a] > 0) t += xi - x[i - stride[a]];
            if (c[a] < g.m[a] - 1) t += xi - x[i + stride[a]];
            acc = fmaf(t, g.inv_h[a] * g.inv_h[a], acc);
        }
        float r = scale * acc;
        if (gsrc != nullptr) r = fmaf(gamma, gsrc[i], r);
        if (addsrc != nullptr) r += addsrc[i];
        out[i] = r;
    }
}

// div[j] = sum_a (x_a[i+1] - x_a[i-1]) / (2 h_a), ends mirrored (one-sided).
template <int D>
__global__ void divergence_kernel(const float* __restrict__ x, float* __restrict__ div, DevGrid g, int K) {
    const size_t Mv = (size_t)g.m[0] * g.m[1] * g.m[2];
    const size_t total = Mv * K;
    const size_t stride[3] = {1, (size_t)g.m[0], (size_t)g.m[0] * g.m[1]};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = (unsigned)i % (unsigned)Mv;
        const size_t j = (unsigned)i / (unsigned)Mv;
        int c[3];
        coords<D>(s, g, c);
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const float* xa = x + (j * D + a) * Mv;
            const size_t up = (c[a] < g.m[a] - 1) ? s + stride[a] : s;
            const size_t dn = (c[a] > 0) ? s - stride[a] : s;
            acc += (xa[up] - xa[dn]) * (0.5f * g.inv_h[a]);
        }
        div[i] = acc;
    }
}

// out_c = addsrc + smu * (A x_c) + slm * (D_c^T div) + gamma * x_c (elastic operator).
template <int D>
__global__ void elastic_kernel(const float* __restrict__ x, const float* __restrict__ div, float* out, DevGrid g,
                               int K, float smu, float slm, float gamma, const float* addsrc) {
    const size_t Mv = (size_t)g.m[0] * g.m[1] * g.m[2];
    const size_t total = Mv * K * D;
    const size_t stride[3] = {1, (size_t)g.m[0], (size_t)g.m[0] * g.m[1]};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = (unsigned)i % (unsigned)Mv;
        const size_t blk = (unsigned)i / (unsigned)Mv;
        const int comp = (int)(blk % D);
        const size_t j = blk / D;
        int c[3];
        coords<D>(s, g, c);
        const float xi = x[i];
        float lap = 0.0f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float t = 0.0f;
            if (c[a] > 0) t += xi - x[i - stride[a]];
            if (c[a] < g.m[a] - 1) t += xi - x[i + stride[a]];
            lap = fmaf(t, g.inv_h[a] * g.inv_h[a], lap);
        }
        // transpose of the centred difference along axis comp
        const float* dj = div + j * Mv;
        const int ci = c[comp], m = g.m[comp];
        const size_t st = stride[comp];
        float dt = 0.0f;
        if (ci >= 1) dt += dj[s - st];
        if (ci == m - 1) dt += dj[s];
        if (ci + 1 <= m - 1) dt -= dj[s + st];
        if (ci == 0) dt -= dj[s];
        dt *= 0.5f * g.inv_h[comp];
        float r = smu * lap + slm * dt + gamma * xi;
        if (addsrc != nullptr) r += addsrc[i];
        out[i] = r;
    }
}

// ------------------------------------------------------------------ DCT --

// out[.., k, ..] = sum_i C[k][i] in[.., i, ..] along one axis (inverse: C[i][k]);
// C is the orthonormal DCT-II matrix of that axis.
__global__ void dct_axis_kernel(const float* __restrict__ in, float* __restrict__ out, const float* __restrict__ C,
                                DevGrid g, int nblk, int axis, int inverse) {
    const size_t Mv = (size_t)g.m[0] * g.m[1] * g.m[2];
    const size_t total = Mv * nblk;
    const int m = g.m[axis];
    const size_t st = (axis == 0) ? 1 : (axis == 1 ? (size_t)g.m[0] : (size_t)g.m[0] * g.m[1]);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = (unsigned)i % (unsigned)Mv;
        const int k = (int)((s / st) % m);
        const size_t base = i - (size_t)k * st;
        float acc = 0.0f;
        if (inverse) {
            for (int q = 0; q < m; ++q) acc = fmaf(__ldg(C + (size_t)q * m + k), in[base + q * st], acc);
        } else {
            const float* row = C + (size_t)k * m;
            for (int q = 0; q < m; ++q) acc = fmaf(__ldg(row + q), in[base + q * st], acc);
        }
        out[i] = acc;
    }
}

// 16-byte asynchronous copy from global to shared memory (both addresses
// 16-byte aligned), cached in L2 only; cp_async_wait_all() waits for every
// copy this thread issued.  A CTA issues all its staging copies before the
// first wait, so a tile arrives in about one memory round trip.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// The same transform for axes of at most kDctTileMax cells, as a small
// register-blocked matrix product staged in shared memory.  Each array block
// is viewed as [outer][m][inner] (inner = product of the cell counts of the
// axes below `axis`).  A CTA transforms 64 lines: 64 consecutive inner
// positions of one outer index (axis > 0), or 64 consecutive x rows (axis 0,
// inner = 1; loaded and stored through shared memory so that global accesses
// stay coalesced).  The coefficient matrix sits in shared memory transposed,
// [q][k], and the tile as [q][line]; a thread computes a 4 x 4 block of
// (output index k, line), reading one float4 of each per q for 16 FMAs.  Every
// output is accumulated over q in increasing order, as in dct_axis_kernel.
constexpr int kDctTileMax = 128;
constexpr int kDctLines = 64;
constexpr int kDctLS = kDctLines + 4;        // tile row stride (float4-aligned)

template <bool XAXIS>
__global__ void __launch_bounds__(kBlock) dct_tile_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                          const float* __restrict__ Ctg, int m, long long inner,
                                                          long long lines, int vec_in) {
    extern __shared__ __align__(16) float sm[];
    const int MP = (m + 3) & ~3;                 // k padded to whole float4s
    float* Ct = sm;                              // [q][MP]: the padded table of the direction (Cf or Ci)
    float* tile = sm + m * MP;                   // [q][kDctLS], later the output stage of axis 0
    const int t = threadIdx.x;
    for (int e = t; e < m * MP / 4; e += kBlock) cp_async16(Ct + 4 * e, Ctg + 4 * e);
    long long o = 0, i0 = 0, r0 = 0;
    if (XAXIS) {                                 // lines are rows: loaded transposed, element by element
        r0 = (long long)blockIdx.x * kDctLines;
        for (int e = t; e < kDctLines * m; e += kBlock) {
            const int l = e / m, q = e % m;
            tile[q * kDctLS + l] = (r0 + l < lines) ? __ldg(in + (size_t)(r0 + l) * m + q) : 0.0f;
        }
    } else {
        o = blockIdx.y;
        i0 = (long long)blockIdx.x * kDctLines;
        if (vec_in) {                            // inner a multiple of 4, in 16-byte aligned
            for (int e = t; e < m * (kDctLines / 4); e += kBlock) {
                const int q = e / (kDctLines / 4), l = 4 * (e % (kDctLines / 4));
                if (i0 + l < inner) cp_async16(tile + q * kDctLS + l, in + ((size_t)o * m + q) * inner + i0 + l);
                else *reinterpret_cast<float4*>(tile + q * kDctLS + l) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        } else {
            for (int e = t; e < kDctLines * m; e += kBlock) {
                const int q = e / kDctLines, l = e % kDctLines;
                tile[q * kDctLS + l] = (i0 + l < inner) ? __ldg(in + ((size_t)o * m + q) * inner + i0 + l) : 0.0f;
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int ntask = (MP / 4) * (kDctLines / 4);
    constexpr int SS = kDctTileMax + 1;          // output stage row stride (axis 0)
    float acc[2][4][4];                          // at most two tasks per thread (MP <= 128)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int task = t + r * kBlock;
        if (task >= ntask) break;
        const int kb = task / (kDctLines / 4), lb = task % (kDctLines / 4);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[r][i][j] = 0.0f;
        const float4* cp = reinterpret_cast<const float4*>(Ct) + kb;
        const float4* xp = reinterpret_cast<const float4*>(tile) + lb;
#pragma unroll 4
        for (int q = 0; q < m; ++q) {
            const float4 c = cp[q * (MP / 4)];
            const float4 x = xp[q * (kDctLS / 4)];
            const float cv[4] = {c.x, c.y, c.z, c.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[r][i][j] = fmaf(cv[i], xv[j], acc[r][i][j]);
        }
        if (!XAXIS) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * kb + i;
                if (k >= m) break;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long l = i0 + 4 * lb + j;
                    if (l < inner) out[((size_t)o * m + k) * inner + l] = acc[r][i][j];
                }
            }
        }
    }
    if (XAXIS) {
        __syncthreads();                         // the tile becomes the output stage [line][k]
        float* stage = tile;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int task = t + r * kBlock;
            if (task >= ntask) break;
            const int kb = task / (kDctLines / 4), lb = task % (kDctLines / 4);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * kb + i;
                if (k >= m) break;
#pragma unroll
                for (int j = 0; j < 4; ++j) stage[(4 * lb + j) * SS + k] = acc[r][i][j];
            }
        }
        __syncthreads();
        for (int e = t; e < kDctLines * m; e += kBlock) {
            const int l = e / m, k = e % m;
            if (r0 + l < lines) out[(size_t)(r0 + l) * m + k] = stage[l * SS + k];
        }
    }
}

// The last axis of the preconditioner in one pass: forward DCT along the
// axis, the spectral scale inv_eig (per mode, the same for every block), and
// the inverse DCT, with the scaled modes kept in shared memory in between.
// LINES lines per CTA of 4 LINES threads, with the register blocking of
// dct_tile_kernel (strided form); every sum still runs in increasing index
// order.
constexpr int kDctFusedLines = 32;

template <int LINES>
__global__ void __launch_bounds__(4 * LINES) dct_last_fused_kernel(const float* __restrict__ in,
                                                                   float* __restrict__ out,
                                                                   const float* __restrict__ Cfg,
                                                                   const float* __restrict__ Cig,
                                                                   const float* __restrict__ inv_eig, int m,
                                                                   long long inner, int vec_in) {
    constexpr int NT = 4 * LINES, LS = LINES + 4;
    extern __shared__ __align__(16) float sm[];
    const int MP = (m + 3) & ~3;
    float* Cf = sm;                   // forward: [q][k] = C[k][q]
    float* Ci = sm + m * MP;          // inverse: [k][k'] = C[k][k']
    float* tile = sm + 2 * m * MP;    // [q][LS], then the scaled modes [k][LS]
    const int t = threadIdx.x;
    for (int e = t; e < m * MP / 4; e += NT) {
        cp_async16(Cf + 4 * e, Cfg + 4 * e);
        cp_async16(Ci + 4 * e, Cig + 4 * e);
    }
    const long long o = blockIdx.y, i0 = (long long)blockIdx.x * LINES;
    if (vec_in) {                     // inner a multiple of 4, in 16-byte aligned: whole float4s in or out
        for (int e = t; e < m * (LINES / 4); e += NT) {
            const int q = e / (LINES / 4), l = 4 * (e % (LINES / 4));
            if (i0 + l < inner) cp_async16(tile + q * LS + l, in + ((size_t)o * m + q) * inner + i0 + l);
            else *reinterpret_cast<float4*>(tile + q * LS + l) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    } else {
        for (int e = t; e < LINES * m; e += NT) {
            const int q = e / LINES, l = e % LINES;
            tile[q * LS + l] = (i0 + l < inner) ? __ldg(in + ((size_t)o * m + q) * inner + i0 + l) : 0.0f;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int ntask = (MP / 4) * (LINES / 4);
    float acc[2][4][4];               // at most two tasks per thread (MP <= 128)
    for (int pass = 0; pass < 2; ++pass) {
        const float* Cm = pass == 0 ? Cf : Ci;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int task = t + r * NT;
            if (task >= ntask) break;
            const int kb = task / (LINES / 4), lb = task % (LINES / 4);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[r][i][j] = 0.0f;
            const float4* cp = reinterpret_cast<const float4*>(Cm) + kb;
            const float4* xp = reinterpret_cast<const float4*>(tile) + lb;
#pragma unroll 4
            for (int q = 0; q < m; ++q) {
                const float4 c = cp[q * (MP / 4)];
                const float4 x = xp[q * (LS / 4)];
                const float cv[4] = {c.x, c.y, c.z, c.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[r][i][j] = fmaf(cv[i], xv[j], acc[r][i][j]);
            }
        }
        __syncthreads();              // every thread is done reading the tile
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int task = t + r * NT;
            if (task >= ntask) break;
            const int kb = task / (LINES / 4), lb = task % (LINES / 4);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * kb + i;
                if (k >= m) break;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long l = i0 + 4 * lb + j;
                    if (pass == 0) {
                        const float sc = l < inner ? __ldg(inv_eig + (size_t)k * inner + l) : 0.0f;
                        tile[k * LS + 4 * lb + j] = acc[r][i][j] * sc;
                    } else if (l < inner) {
                        out[((size_t)o * m + k) * inner + l] = acc[r][i][j];
                    }
                }
            }
        }
        __syncthreads();
    }
}

// The y and x axes of the transform on whole xy planes (both at most
// kDctPlaneMax cells): a CTA holds one plane of one (block, z) in shared
// memory and applies the y axis and then the x axis, two small matrix products
// chained through shared memory.  The y result goes back transposed, [x][k],
// from registers, so that both products read float4 rows of shared memory and
// the plane is loaded and stored row-major.  With Ay, Ax the padded tables of
// the direction (forward Cf, inverse Ci):
//   forward: modes = C_y X C_x^T      inverse: X = C_y^T modes C_x
// The tables and the plane are staged with asynchronous 16-byte copies, all
// issued before the first wait.  A thread computes a 4 x 4 block of each
// product; every sum runs over its index in increasing order.  The two axes
// commute, so this equals the per-axis passes up to rounding.
constexpr int kDctPlaneMax = 64;

// The chained products of one plane: the plane is in S as rows [y][LS]; the
// y product with Ay ([q][PY]) goes back into S transposed, [x][LT], and the x
// product with Ax ([q][PX]) is left in acc[i][j] = (x index 4 xb + i, y index
// 4 kb + j) of this thread's block.  Every thread of the CTA calls it (two
// barriers); act: the thread has a block.
__device__ __forceinline__ void plane_yx(const float* Ay, const float* Ax, float* S, int mx, int my, int PX, int PY,
                                         int LS, int LT, bool act, int kb, int xb, float (&acc)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;   // [k along y][x]
    if (act) {
        const float4* ap = reinterpret_cast<const float4*>(Ay) + kb;
        const float4* sp = reinterpret_cast<const float4*>(S) + xb;
#pragma unroll 4
        for (int q = 0; q < my; ++q) {
            const float4 a = ap[q * (PY / 4)];
            const float4 x = sp[q * (LS / 4)];
            const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], xv[j], acc[i][j]);
        }
    }
    __syncthreads();                      // every read of the plane is done
    if (act) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4*>(S + (4 * xb + j) * LT + 4 * kb) =
                make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;   // now [k along x][y]
    if (act) {
        const float4* ap = reinterpret_cast<const float4*>(Ax) + xb;
        const float4* tp = reinterpret_cast<const float4*>(S) + kb;
#pragma unroll 4
        for (int q = 0; q < mx; ++q) {
            const float4 a = ap[q * (PX / 4)];
            const float4 x = tp[q * (LT / 4)];
            const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], xv[j], acc[i][j]);
        }
    }
}

// Stage a plane of `in` (block `plane`) into S rows [y][LS], pad columns zero.
__device__ __forceinline__ void plane_load(const float* __restrict__ in, size_t base, float* S, int mx, int my, int PX,
                                           int LS, int vec_in) {
    const int t = threadIdx.x;
    if (vec_in) {                         // mx a multiple of 4 (PX = mx), in 16-byte aligned
        const int c4 = mx / 4;
        for (int e = t; e < my * c4; e += blockDim.x) {
            const int y = e / c4, x = 4 * (e % c4);
            cp_async16(S + y * LS + x, in + base + (size_t)y * mx + x);
        }
    } else {
        for (int e = t; e < my * PX; e += blockDim.x) {
            const int y = e / PX, x = e % PX;
            S[y * LS + x] = x < mx ? __ldg(in + base + (size_t)y * mx + x) : 0.0f;
        }
    }
}

// Store this thread's block acc[i][j] = (x 4 xb + i, y 4 kb + j) of the plane.
__device__ __forceinline__ void plane_store(float* __restrict__ out, size_t base, int mx, int my, int kb, int xb,
                                            const float (&acc)[4][4], int vec_out) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = 4 * kb + j;
        if (y >= my) break;
        float* o = out + base + (size_t)y * mx + 4 * xb;
        if (vec_out) {
            *reinterpret_cast<float4*>(o) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * xb + i < mx) o[i] = acc[i][j];
        }
    }
}

__global__ void __launch_bounds__(kBlock) dct_plane_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                           const float* __restrict__ Axg,
                                                           const float* __restrict__ Ayg, int mx, int my,
                                                           int vec_in, int vec_out) {
    extern __shared__ __align__(16) float sm[];
    const int PX = (mx + 3) & ~3, PY = (my + 3) & ~3;
    const int LS = PX + 4, LT = PY + 4;   // row strides of the plane [y][x] and of the transposed result [x][k]
    float* Ay = sm;                       // [q][PY]
    float* Ax = Ay + my * PY;             // [q][PX]
    float* S = Ax + mx * PX;              // the plane, later the y result transposed
    const int t = threadIdx.x;
    for (int e = t; e < my * PY / 4; e += kBlock) cp_async16(Ay + 4 * e, Ayg + 4 * e);
    for (int e = t; e < mx * PX / 4; e += kBlock) cp_async16(Ax + 4 * e, Axg + 4 * e);
    const size_t base = (size_t)blockIdx.x * mx * my;
    plane_load(in, base, S, mx, my, PX, LS, vec_in);
    cp_async_wait_all();
    __syncthreads();
    const int nxb = PX / 4;
    const bool act = t < (PY / 4) * nxb;  // at most 256 blocks of 4 x 4: one per thread
    const int kb = act ? t / nxb : 0, xb = act ? t % nxb : 0;
    float acc[4][4];
    plane_yx(Ay, Ax, S, mx, my, PX, PY, LS, LT, act, kb, xb, acc);
    if (act) plane_store(out, base, mx, my, kb, xb, acc, vec_out);
}

// The whole 2D preconditioner on one plane (a (time node, component) block of
// at most 64 x 64 cells) in one CTA: modes = C_y X C_x^T, scaled by inv_eig,
// then X = C_y^T modes C_x, with the scaled modes written back into the plane
// buffer between the two halves.
__global__ void __launch_bounds__(kBlock) dct_plane2d_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                             const float* __restrict__ Cfx,
                                                             const float* __restrict__ Cfy,
                                                             const float* __restrict__ Cix,
                                                             const float* __restrict__ Ciy,
                                                             const float* __restrict__ inv_eig, int mx, int my,
                                                             int vec_in, int vec_out) {
    extern __shared__ __align__(16) float sm[];
    const int PX = (mx + 3) & ~3, PY = (my + 3) & ~3;
    const int LS = PX + 4, LT = PY + 4;
    float* Fy = sm;                       // forward tables [q][P]
    float* Fx = Fy + my * PY;
    float* Iy = Fx + mx * PX;             // inverse tables [q][P]
    float* Ix = Iy + my * PY;
    float* S = Ix + mx * PX;
    const int t = threadIdx.x;
    for (int e = t; e < my * PY / 4; e += kBlock) {
        cp_async16(Fy + 4 * e, Cfy + 4 * e);
        cp_async16(Iy + 4 * e, Ciy + 4 * e);
    }
    for (int e = t; e < mx * PX / 4; e += kBlock) {
        cp_async16(Fx + 4 * e, Cfx + 4 * e);
        cp_async16(Ix + 4 * e, Cix + 4 * e);
    }
    const size_t base = (size_t)blockIdx.x * mx * my;
    plane_load(in, base, S, mx, my, PX, LS, vec_in);
    cp_async_wait_all();
    __syncthreads();
    const int nxb = PX / 4;
    const bool act = t < (PY / 4) * nxb;
    const int kb = act ? t / nxb : 0, xb = act ? t % nxb : 0;
    float acc[4][4];
    plane_yx(Fy, Fx, S, mx, my, PX, PY, LS, LT, act, kb, xb, acc);
    // scale the modes (kx = 4 xb + i, ky = 4 kb + j; padding modes are zero) and put
    // them back as rows [ky][LS] once every thread is done with the transposed buffer
    __syncthreads();
    if (act) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ky = 4 * kb + j;
            float sc[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int kx = 4 * xb + i;
                sc[i] = (kx < mx && ky < my) ? acc[i][j] * __ldg(inv_eig + (size_t)ky * mx + kx) : 0.0f;
            }
            // rows ky >= my are never read (the inverse sums over q < my) and may lie past the buffer
            if (ky < my) *reinterpret_cast<float4*>(S + ky * LS + 4 * xb) = make_float4(sc[0], sc[1], sc[2], sc[3]);
        }
    }
    __syncthreads();
    plane_yx(Iy, Ix, S, mx, my, PX, PY, LS, LT, act, kb, xb, acc);
    if (act) plane_store(out, base, mx, my, kb, xb, acc, vec_out);
}

inline size_t dct_plane_smem(int mx, int my, int tables = 1) {
    const size_t PX = (size_t)((mx + 3) & ~3), PY = (size_t)((my + 3) & ~3);
    const size_t plane = std::max((size_t)my * (PX + 4), PX * (PY + 4));
    return (tables * ((size_t)my * PY + (size_t)mx * PX) + plane) * sizeof(float);
}

// Shared memory of dct_tile_kernel for an axis of m cells (bytes).
inline size_t dct_tile_smem(int m) {
    const size_t MP = (size_t)((m + 3) & ~3);
    const size_t tile = std::max((size_t)m * kDctLS, (size_t)kDctLines * (kDctTileMax + 1));
    return ((size_t)m * MP + tile) * sizeof(float);
}

__global__ void scale_modes_kernel(float* x, const float* __restrict__ inv_eig, size_t block_elems, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        x[i] *= inv_eig[i % block_elems];
}

__global__ void axpby_kernel(float a, const float* __restrict__ x, float b, float* y, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], b * y[i]);
}

__global__ void add_scaled_kernel(float* out, const float* x, float ax, const float* y, float ay, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = fmaf(ax, x[i], ay * y[i]);
}

// ------------------------------------------------------------- multilevel --

// Coarse cell = average of the 2^d fine cells that tile it (fine m = 2 coarse m).
template <int D>
__global__ void restrict_image_kernel(const float* __restrict__ F, float* __restrict__ C, DevGrid cg) {
    const size_t Mc = (size_t)cg.m[0] * cg.m[1] * cg.m[2];
    const int fm0 = 2 * cg.m[0], fm1 = 2 * cg.m[1];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < Mc; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % cg.m[0]);
        const int y = (int)((i / cg.m[0]) % cg.m[1]);
        const int z = (int)(i / ((size_t)cg.m[0] * cg.m[1]));
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < (1 << D); ++c) {
            const int fx = 2 * x + (c & 1), fy = 2 * y + ((c >> 1) & 1), fz = D == 3 ? 2 * z + ((c >> 2) & 1) : 0;
            s += F[((size_t)fz * fm1 + fy) * fm0 + fx];
        }
        C[i] = s * (1.0f / (1 << D));
    }
}

// Fine velocity = coarse velocity interpolated (multilinear, zero outside the
// coarse grid) at the fine cell centres, per time node and component.
template <int D>
__global__ void prolong_velocity_kernel(const float* __restrict__ vc, float* __restrict__ vf, DevGrid cg, DevGrid fg,
                                        int blocks) {
    const size_t Mf = (size_t)fg.m[0] * fg.m[1] * fg.m[2];
    const size_t Mc = (size_t)cg.m[0] * cg.m[1] * cg.m[2];
    const size_t total = Mf * blocks;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = i % Mf;
        const size_t b = i / Mf;
        const int fi[3] = {(int)(s % fg.m[0]), (int)((s / fg.m[0]) % fg.m[1]), (int)(s / ((size_t)fg.m[0] * fg.m[1]))};
        int c0[3];
        float fr[3];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const float x = fg.lo[a] + ((float)fi[a] + 0.5f) * fg.h[a];
            const float xi = (x - cg.lo[a]) * cg.inv_h[a] - 0.5f;
            const float fl = floorf(xi);
            c0[a] = (int)fl;
            fr[a] = xi - fl;
        }
        const float* src = vc + b * Mc;
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < (1 << D); ++c) {
            float w = 1.0f;
            int idx[3] = {0, 0, 0};
            bool in = true;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int bit = (c >> a) & 1;
                idx[a] = c0[a] + bit;
                w *= bit ? fr[a] : 1.0f - fr[a];
                in = in && idx[a] >= 0 && idx[a] < cg.m[a];
            }
            if (in) acc = fmaf(w, src[((size_t)idx[2] * cg.m[1] + idx[1]) * cg.m[0] + idx[0]], acc);
        }
        vf[b * Mf + s] = acc;
    }
}

// ------------------------------------------------- Jacobian determinant --

__device__ __forceinline__ void block_minmax(double& lo, double& hi) {
    __shared__ double slo[kBlock / 32], shi[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        slo[warp] = lo;
        shi[warp] = hi;
    }
    __syncthreads();
    if (warp == 0) {
        lo = lane < kBlock / 32 ? slo[lane] : INFINITY;
        hi = lane < kBlock / 32 ? shi[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
        }
    }
}

// det grad y at the cell centres from the end points y [d][M]: central
// differences inside, one-sided at the ends; block min/max into partials.
template <int D>
__global__ void jacobian_det_kernel(const float* __restrict__ y, float* det, DevGrid g, double* pmin, double* pmax) {
    const size_t M = (size_t)g.m[0] * g.m[1] * g.m[2];
    const size_t stride[3] = {1, (size_t)g.m[0], (size_t)g.m[0] * g.m[1]};
    double lo = INFINITY, hi = -INFINITY;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
        const int c[3] = {(int)(i % g.m[0]), (int)((i / g.m[0]) % g.m[1]), (int)(i / ((size_t)g.m[0] * g.m[1]))};
        double J[3][3];
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const size_t up = c[b] < g.m[b] - 1 ? i + stride[b] : i;
            const size_t dn = c[b] > 0 ? i - stride[b] : i;
            const double span = (double)g.h[b] * (double)((up != i) + (dn != i));
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float* ya = y + (size_t)a * M;
                J[a][b] = span > 0.0 ? ((double)ya[up] - (double)ya[dn]) / span : (a == b ? 1.0 : 0.0);
            }
        }
        double dt;
        if (D == 2) dt = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        else
            dt = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (det != nullptr) det[i] = (float)dt;
        lo = fmin(lo, dt);
        hi = fmax(hi, dt);
    }
    block_minmax(lo, hi);
    if (threadIdx.x == 0) {
        pmin[blockIdx.x] = lo;
        pmax[blockIdx.x] = hi;
    }
}

__global__ void minmax_final_kernel(const double* pmin, const double* pmax, int count, double* out) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        lo = fmin(lo, pmin[i]);
        hi = fmax(hi, pmax[i]);
    }
    block_minmax(lo, hi);
    if (threadIdx.x == 0) {
        out[0] = lo;
        out[1] = hi;
    }
}

inline int grid_for(size_t count) {
    const size_t b = (count + kBlock - 1) / kBlock;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_pack_velocity(int d, const float* v, void* Vp, const DevGrid& g, int K, const SliceTable& t,
                                 cudaStream_t s, void* Gz) {
    (void)K;
    const size_t total = (size_t)g.mp[0] * g.mp[1] * g.mp[2] * t.n;
    if (d == 3) pack_velocity_kernel<3><<<grid_for(total), kBlock, 0, s>>>(v, (float*)Vp, g, t, Gz);
    else pack_velocity_kernel<2><<<grid_for(total), kBlock, 0, s>>>(v, (float*)Vp, g, t, Gz);
    return cudaGetLastError();
}

cudaError_t launch_distribute_gradient(int d, const void* Gp, float* out, const DevGrid& g, int K,
                                       const SliceTable& t, float scale, cudaStream_t s) {
    const size_t total = (size_t)g.m[0] * g.m[1] * g.m[2] * K;
    if (d == 3) distribute_gradient_kernel<3><<<grid_for(total), kBlock, 0, s>>>((const float*)Gp, out, g, K, t, scale);
    else distribute_gradient_kernel<2><<<grid_for(total), kBlock, 0, s>>>((const float*)Gp, out, g, K, t, scale);
    return cudaGetLastError();
}

void make_slice_table(int K, int N, double t0, double dt, SliceTable* t) {
    if (K <= 1) {
        t->n = 1;
        t->j[0] = 0;
        t->th[0] = 0.0f;
        return;
    }
    t->n = 2 * N + 1;
    for (int m = 0; m < t->n; ++m) {
        double tm = t0 + m * 0.5 * dt;
        tm = tm < 0.0 ? 0.0 : (tm > 1.0 ? 1.0 : tm);
        const double sv = tm * (K - 1);
        int j = (int)std::floor(sv);
        if (j > K - 2) j = K - 2;
        t->j[m] = j;
        t->th[m] = (float)(sv - j);
    }
}

cudaError_t launch_pack_image(const float* T, float* Tp, const DevGrid& g, int d, float scale, cudaStream_t s) {
    const size_t total = (size_t)g.mp[0] * g.mp[1] * g.mp[2];
    pack_image_kernel<<<grid_for(total), kBlock, 0, s>>>(T, Tp, g, d, scale);
    return cudaGetLastError();
}

cudaError_t launch_unpack_image(const float* acc, float* out, const DevGrid& g, int d, cudaStream_t s) {
    const size_t M = (size_t)g.m[0] * g.m[1] * g.m[2];
    unpack_image_kernel<<<grid_for(M), kBlock, 0, s>>>(acc, out, g, d);
    return cudaGetLastError();
}

cudaError_t launch_repad_image(float* acc, const DevGrid& g, int d, float scale, cudaStream_t s) {
    const size_t total = (size_t)g.mp[0] * g.mp[1] * g.mp[2];
    repad_image_kernel<<<grid_for(total), kBlock, 0, s>>>(acc, g, d, scale);
    return cudaGetLastError();
}

// Blocks of the grid-stride reductions: four per SM of the current device
// (the SM count is read once per device ordinal).
int reduce_block_cap() {
    static int cap[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 4 * 152;
    }
    if (cap[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            cudaGetLastError();
            sms = 152;
        }
        cap[dev] = 4 * sms;
    }
    return cap[dev];
}

int residual_blocks(const DevGrid& g, int d) {
    (void)d;
    const size_t M = (size_t)g.m[0] * g.m[1] * g.m[2];
    const int b = nblocks_for(M);
    const int cap = reduce_block_cap();
    return b < cap ? b : cap;
}

cudaError_t launch_residual(const float* u1, const float* R, float* rp, const DevGrid& g, int d, float scale,
                            double* partial, int nblocks, cudaStream_t s) {
    residual_kernel<<<nblocks, kBlock, 0, s>>>(u1, R, rp, g, d, scale, partial);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partial, int count, double* out, cudaStream_t s) {
    reduce_kernel<<<1, kBlock, 0, s>>>(partial, count, out);
    return cudaGetLastError();
}

int dot_blocks(size_t count) {
    const int b = nblocks_for(count);
    const int cap = reduce_block_cap();
    return b < cap ? (b > 0 ? b : 1) : cap;
}

cudaError_t launch_dot_fused(const float* a, const float* b, const float* c, size_t count, double* partial,
                             int nblocks, unsigned* counter, double* sc, int slot_b, int slot_c, int mode, float* f,
                             cudaStream_t s) {
    dot_fused_kernel<<<nblocks, kBlock, 0, s>>>(a, b, c, count, partial, counter, sc, slot_b, slot_c, mode, f);
    return cudaGetLastError();
}

cudaError_t launch_hess_finish(int d, const void* Gp, const float* p, float* Hp, const DevGrid& g, int K,
                               const SliceTable& t, float gscale, float rscale, float gamma, double* partial,
                               int nblocks, unsigned* counter, double* sc, float* f, cudaStream_t s) {
    // without partial: the product only, on a grid sized for the vector
    if (partial == nullptr) nblocks = grid_for((size_t)g.m[0] * g.m[1] * g.m[2] * K);
    if (d == 3) {
        if (partial) hess_finish_kernel<3, true><<<nblocks, kBlock, 0, s>>>((const float*)Gp, p, Hp, g, K, t, gscale,
                                                                             rscale, gamma, partial, counter, sc, f);
        else hess_finish_kernel<3, false><<<nblocks, kBlock, 0, s>>>((const float*)Gp, p, Hp, g, K, t, gscale, rscale,
                                                                     gamma, partial, counter, sc, f);
    } else {
        if (partial) hess_finish_kernel<2, true><<<nblocks, kBlock, 0, s>>>((const float*)Gp, p, Hp, g, K, t, gscale,
                                                                             rscale, gamma, partial, counter, sc, f);
        else hess_finish_kernel<2, false><<<nblocks, kBlock, 0, s>>>((const float*)Gp, p, Hp, g, K, t, gscale, rscale,
                                                                     gamma, partial, counter, sc, f);
    }
    return cudaGetLastError();
}

cudaError_t launch_pcg_update_xr(float* x, const float* p, float* r, const float* Hp, const float* f, size_t count,
                                 cudaStream_t s) {
    pcg_update_xr_kernel<<<grid_for(count), kBlock, 0, s>>>(x, p, r, Hp, f, count);
    return cudaGetLastError();
}

cudaError_t launch_pcg_curvature_fix(float* x, const float* z, const int* ctl, size_t count, cudaStream_t s) {
    const size_t want = (count + kBlock - 1) / kBlock;
    const int cap = reduce_block_cap();
    const int blocks = (int)(want < (size_t)cap ? (want > 0 ? want : 1) : (size_t)cap);
    pcg_curvature_fix_kernel<<<blocks, kBlock, 0, s>>>(x, z, ctl, count);
    return cudaGetLastError();
}

cudaError_t launch_pcg_control(const double* sc, int* ctl, cudaGraphConditionalHandle handle, cudaStream_t s) {
    pcg_control_kernel<<<1, 32, 0, s>>>(sc, ctl, handle);
    return cudaGetLastError();
}

cudaError_t launch_axpby_dev(float a, const float* ap, const float* x, float b, const float* bp, float* y,
                             size_t count, cudaStream_t s) {
    axpby_dev_kernel<<<grid_for(count), kBlock, 0, s>>>(a, ap, x, b, bp, y, count);
    return cudaGetLastError();
}

cudaError_t launch_dot(const float* a, const float* b, size_t count, double* partial, int nblocks, cudaStream_t s) {
    dot_kernel<<<nblocks, kBlock, 0, s>>>(a, b, count, partial);
    return cudaGetLastError();
}

cudaError_t launch_laplacian(int d, const float* x, float* out, const DevGrid& g, int blocks_kd, float scale,
                             float gamma, const float* addsrc, cudaStream_t s) {
    const size_t total = (size_t)g.m[0] * g.m[1] * g.m[2] * blocks_kd;
    const float* gsrc = gamma != 0.0f ? x : nullptr;
    if (d == 3) laplacian_kernel<3><<<grid_for(total), kBlock, 0, s>>>(x, out, g, blocks_kd, scale, gamma, gsrc, addsrc);
    else laplacian_kernel<2><<<grid_for(total), kBlock, 0, s>>>(x, out, g, blocks_kd, scale, gamma, gsrc, addsrc);
    return cudaGetLastError();
}

cudaError_t launch_laplacian_ext(int d, const float* x, float* out, const DevGrid& g, int blocks_kd, float scale,
                                 float gamma, const float* gsrc, const float* addsrc, cudaStream_t s) {
    const size_t total = (size_t)g.m[0] * g.m[1] * g.m[2] * blocks_kd;
    if (d == 3) laplacian_kernel<3><<<grid_for(total), kBlock, 0, s>>>(x, out, g, blocks_kd, scale, gamma, gsrc, addsrc);
    else laplacian_kernel<2><<<grid_for(total), kBlock, 0, s>>>(x, out, g, blocks_kd, scale, gamma, gsrc, addsrc);
    return cudaGetLastError();
}

cudaError_t launch_divergence(int d, const float* x, float* div, const DevGrid& g, int K, cudaStream_t s) {
    const size_t total = (size_t)g.m[0] * g.m[1] * g.m[2] * K;
    if (d == 3) divergence_kernel<3><<<grid_for(total), kBlock, 0, s>>>(x, div, g, K);
    else divergence_kernel<2><<<grid_for(total), kBlock, 0, s>>>(x, div, g, K);
    return cudaGetLastError();
}

cudaError_t launch_elastic(int d, const float* x, const float* div, float* out, const DevGrid& g, int K,
                           float smu, float slm, float gamma, const float* addsrc, cudaStream_t s) {
    const size_t total = (size_t)g.m[0] * g.m[1] * g.m[2] * K * d;
    if (d == 3) elastic_kernel<3><<<grid_for(total), kBlock, 0, s>>>(x, div, out, g, K, smu, slm, gamma, addsrc);
    else elastic_kernel<2><<<grid_for(total), kBlock, 0, s>>>(x, div, out, g, K, smu, slm, gamma, addsrc);
    return cudaGetLastError();
}

cudaError_t launch_dct_axis(const float* in, float* out, const float* C, const float* Cp, const DevGrid& g, int d,
                            int nblocks_kd, int axis, bool inverse, cudaStream_t s) {
    (void)d;
    const size_t total = (size_t)g.m[0] * g.m[1] * g.m[2] * nblocks_kd;
    const int m = g.m[axis];
    if (m > kDctTileMax) {
        dct_axis_kernel<<<grid_for(total), kBlock, 0, s>>>(in, out, C, g, nblocks_kd, axis, inverse ? 1 : 0);
        return cudaGetLastError();
    }
    const size_t smem = dct_tile_smem(m);
    // the dynamic shared-memory limit is raised once per device and kernel
    static bool attr_set_dev[64][2] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    bool* attr_set = attr_set_dev[dev];
    const int smem_max = (int)dct_tile_smem(kDctTileMax);
    const long long inner = axis == 0 ? 1 : (axis == 1 ? (long long)g.m[0] : (long long)g.m[0] * g.m[1]);
    const long long outer = (long long)(total / ((size_t)m * inner));
    if (axis == 0) {
        if (!attr_set[0]) {
            const cudaError_t e =
                cudaFuncSetAttribute(dct_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
            if (e != cudaSuccess) return e;
            attr_set[0] = true;
        }
        const long long rows = outer;   // inner = 1: every (y, z, block) is one line
        dct_tile_kernel<true><<<(unsigned)((rows + kDctLines - 1) / kDctLines), kBlock, smem, s>>>(
            in, out, Cp, m, 1, rows, 0);
    } else {
        if (!attr_set[1]) {
            const cudaError_t e =
                cudaFuncSetAttribute(dct_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
            if (e != cudaSuccess) return e;
            attr_set[1] = true;
        }
        if (outer > 65535) {
            dct_axis_kernel<<<grid_for(total), kBlock, 0, s>>>(in, out, C, g, nblocks_kd, axis, inverse ? 1 : 0);
            return cudaGetLastError();
        }
        const dim3 grid((unsigned)((inner + kDctLines - 1) / kDctLines), (unsigned)outer);
        const int vec_in = (inner % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0) ? 1 : 0;
        dct_tile_kernel<false><<<grid, kBlock, smem, s>>>(in, out, Cp, m, inner, inner * m * outer, vec_in);
    }
    return cudaGetLastError();
}

cudaError_t launch_dct_plane(const float* in, float* out, const float* Ax, const float* Ay, const DevGrid& g,
                             long long planes, cudaStream_t s) {
    const int mx = g.m[0], my = g.m[1];
    if (mx > kDctPlaneMax || my > kDctPlaneMax || planes < 1 || planes > 0x7fffffffLL) return cudaErrorNotSupported;
    static bool attr_set_dev[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set_dev[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(dct_plane_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)dct_plane_smem(kDctPlaneMax, kDctPlaneMax));
        if (e != cudaSuccess) return e;
        attr_set_dev[dev] = true;
    }
    const int vec_in = (mx % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0) ? 1 : 0;
    const int vec_out = (mx % 4 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0) ? 1 : 0;
    dct_plane_kernel<<<(unsigned)planes, kBlock, dct_plane_smem(mx, my), s>>>(in, out, Ax, Ay, mx, my, vec_in,
                                                                              vec_out);
    return cudaGetLastError();
}

cudaError_t launch_dct_plane2d(const float* in, float* out, const float* Cfx, const float* Cfy, const float* Cix,
                               const float* Ciy, const float* inv_eig, const DevGrid& g, int blocks, cudaStream_t s) {
    const int mx = g.m[0], my = g.m[1];
    if (mx > kDctPlaneMax || my > kDctPlaneMax || blocks < 1) return cudaErrorNotSupported;
    static bool attr_set_dev[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set_dev[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(dct_plane2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)dct_plane_smem(kDctPlaneMax, kDctPlaneMax, 2));
        if (e != cudaSuccess) return e;
        attr_set_dev[dev] = true;
    }
    const int vec_in = (mx % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0) ? 1 : 0;
    const int vec_out = (mx % 4 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0) ? 1 : 0;
    dct_plane2d_kernel<<<(unsigned)blocks, kBlock, dct_plane_smem(mx, my, 2), s>>>(in, out, Cfx, Cfy, Cix, Ciy, inv_eig,
                                                                                  mx, my, vec_in, vec_out);
    return cudaGetLastError();
}

cudaError_t launch_dct_last_fused(const float* in, float* out, const float* Cf, const float* Ci, const float* inv_eig,
                                  const DevGrid& g, int d, int nblocks_kd, cudaStream_t s) {
    constexpr int L = kDctFusedLines;
    const int axis = d - 1;
    const int m = g.m[axis];
    const long long inner = axis == 1 ? (long long)g.m[0] : (long long)g.m[0] * g.m[1];
    if (m > kDctTileMax || nblocks_kd > 65535) return cudaErrorNotSupported;
    const size_t MP = (size_t)((m + 3) & ~3);
    const size_t smem = (2 * (size_t)m * MP + (size_t)m * (L + 4)) * sizeof(float);
    static bool attr_set_dev[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set_dev[dev]) {
        const int smax = (int)((2 * (size_t)kDctTileMax * kDctTileMax + (size_t)kDctTileMax * (L + 4)) * sizeof(float));
        const cudaError_t e =
            cudaFuncSetAttribute(dct_last_fused_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        if (e != cudaSuccess) return e;
        attr_set_dev[dev] = true;
    }
    const dim3 grid((unsigned)((inner + L - 1) / L), (unsigned)nblocks_kd);
    const int vec_in = (inner % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0) ? 1 : 0;
    dct_last_fused_kernel<L><<<grid, 4 * L, smem, s>>>(in, out, Cf, Ci, inv_eig, m, inner, vec_in);
    return cudaGetLastError();
}

cudaError_t launch_scale_modes(float* x, const float* inv_eig, size_t block_elems, size_t count, cudaStream_t s) {
    scale_modes_kernel<<<grid_for(count), kBlock, 0, s>>>(x, inv_eig, block_elems, count);
    return cudaGetLastError();
}

cudaError_t launch_axpby(float a, const float* x, float b, float* y, size_t count, cudaStream_t s) {
    axpby_kernel<<<grid_for(count), kBlock, 0, s>>>(a, x, b, y, count);
    return cudaGetLastError();
}

cudaError_t launch_add_scaled(float* out, const float* x, float ax, const float* y, float ay, size_t count,
                              cudaStream_t s) {
    add_scaled_kernel<<<grid_for(count), kBlock, 0, s>>>(out, x, ax, y, ay, count);
    return cudaGetLastError();
}

cudaError_t launch_restrict_image(int d, const float* F, float* C, const DevGrid& cg, cudaStream_t s) {
    const size_t Mc = (size_t)cg.m[0] * cg.m[1] * cg.m[2];
    if (d == 3) restrict_image_kernel<3><<<grid_for(Mc), kBlock, 0, s>>>(F, C, cg);
    else restrict_image_kernel<2><<<grid_for(Mc), kBlock, 0, s>>>(F, C, cg);
    return cudaGetLastError();
}

cudaError_t launch_prolong_velocity(int d, const float* vc, float* vf, const DevGrid& cg, const DevGrid& fg,
                                    int blocks, cudaStream_t s) {
    const size_t total = (size_t)fg.m[0] * fg.m[1] * fg.m[2] * blocks;
    if (d == 3) prolong_velocity_kernel<3><<<grid_for(total), kBlock, 0, s>>>(vc, vf, cg, fg, blocks);
    else prolong_velocity_kernel<2><<<grid_for(total), kBlock, 0, s>>>(vc, vf, cg, fg, blocks);
    return cudaGetLastError();
}

cudaError_t launch_jacobian_det(int d, const float* y, float* det, const DevGrid& g, double* partial, double* out,
                                cudaStream_t s) {
    const size_t M = (size_t)g.m[0] * g.m[1] * g.m[2];
    const int nb = residual_blocks(g, d);
    double* pmin = partial;
    double* pmax = partial + nb;
    if (d == 3) jacobian_det_kernel<3><<<nb, kBlock, 0, s>>>(y, det, g, pmin, pmax);
    else jacobian_det_kernel<2><<<nb, kBlock, 0, s>>>(y, det, g, pmin, pmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    (void)M;
    minmax_final_kernel<<<1, kBlock, 0, s>>>(pmin, pmax, nb, out);
    return cudaGetLastError();
}

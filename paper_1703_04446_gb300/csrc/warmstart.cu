// Learned warm start: a small convolutional encoder-decoder that maps an image
// pair (T, R) to a starting velocity for the Gauss-Newton solve (Eq. 11).  The
// paper has no such network; it is an addition whose predictions the solver
// still checks and corrects.
//
// Network for m x m images, c base channels (B images per call):
//   e0 = relu(conv3(x, 2 -> c))                       m
//   e1 = relu(conv3(e0, c -> 2c, stride 2))           m/2
//   e2 = relu(conv3(e1, 2c -> 4c, stride 2))          m/4
//   e3 = relu(conv3(e2, 4c -> 8c, stride 2))          m/8
//   d2 = relu(conv3(up2(e3), 8c -> 4c)) + e2          m/4
//   d1 = relu(conv3(up2(d2), 4c -> 2c)) + e1          m/2
//   v  = scale * conv3(d1, 2c -> 2)                   m/2
// conv3: 3 x 3, zero padding 1; up2: nearest-neighbour doubling, folded into
// the convolution's input indexing.  Weights are used as bfloat16 (rounded from
// FP32 master weights after every Adam step); activations, gradients and
// accumulation are FP32.  Loss 1/2 mean((v - target)^2) / scale^2.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "lgnk_internal.h"

namespace {

constexpr int kT = 256;
constexpr int kCo = 8;     // output channels per forward CTA
constexpr int kCiChunk = 32;
constexpr int kMaxSlices = 64;   // pixel slices of the weight-gradient reduction

struct Layer {
    int ci, co, stride, up;   // input channels, output channels, stride, input upsampled
    int hin, hout;            // input and output side lengths (square)
    size_t woff, boff;        // offsets of W and b in the parameter vector
};

// Input value at effective position (y, x) of an (optionally upsampled) input
// of side hin; zero outside.
__device__ __forceinline__ float in_eff(const float* __restrict__ in, int hin, int up, int y, int x) {
    const int he = up ? 2 * hin : hin;
    if (y < 0 || x < 0 || y >= he || x >= he) return 0.0f;
    if (up) {
        y >>= 1;
        x >>= 1;
    }
    return __ldg(in + (size_t)y * hin + x);
}

// out[b][co][oy][ox] = act(bias + sum_ci,k W[co][ci][k] in_eff[b][ci][oy s + ky - 1][ox s + kx - 1])
// act: relu when relu != 0; r (optional) receives the activation, out = act + add
// (optional skip tensor); the result is multiplied by `scale`.
__global__ void __launch_bounds__(kT) conv_fwd_kernel(const float* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                                                      const float* __restrict__ bias, float* out, float* r,
                                                      const float* __restrict__ add, Layer L, int relu, float scale) {
    __shared__ float ws[kCo][kCiChunk][9];
    const int tiles = (L.hout + 15) / 16;
    const int tx = blockIdx.x % tiles, ty = blockIdx.x / tiles;
    const int co0 = blockIdx.y * kCo;
    const int b = blockIdx.z;
    const int ox = tx * 16 + (threadIdx.x & 15), oy = ty * 16 + (threadIdx.x >> 4);
    const bool active = ox < L.hout && oy < L.hout;
    float acc[kCo];
#pragma unroll
    for (int k = 0; k < kCo; ++k) acc[k] = 0.0f;
    const float* inb = in + (size_t)b * L.ci * L.hin * L.hin;
    for (int c0 = 0; c0 < L.ci; c0 += kCiChunk) {
        const int nc = min(kCiChunk, L.ci - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < kCo * kCiChunk * 9; i += kT) {
            const int co = i / (kCiChunk * 9), rem = i % (kCiChunk * 9), ci = rem / 9, k = rem % 9;
            float w = 0.0f;
            if (co0 + co < L.co && ci < nc) w = __bfloat162float(W[((size_t)(co0 + co) * L.ci + c0 + ci) * 9 + k]);
            ws[co][ci][k] = w;
        }
        __syncthreads();
        if (active) {
            for (int ci = 0; ci < nc; ++ci) {
                const float* inc = inb + (size_t)(c0 + ci) * L.hin * L.hin;
                float v[9];
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    v[k] = in_eff(inc, L.hin, L.up, oy * L.stride + k / 3 - 1, ox * L.stride + k % 3 - 1);
#pragma unroll
                for (int co = 0; co < kCo; ++co) {
#pragma unroll
                    for (int k = 0; k < 9; ++k) acc[co] = fmaf(ws[co][ci][k], v[k], acc[co]);
                }
            }
        }
    }
    if (!active) return;
    for (int co = 0; co < kCo && co0 + co < L.co; ++co) {
        float z = acc[co] + bias[co0 + co];
        if (relu) z = fmaxf(z, 0.0f);
        const size_t o = (((size_t)b * L.co + co0 + co) * L.hout + oy) * L.hout + ox;
        if (r != nullptr) r[o] = z;
        if (add != nullptr) z += add[o];
        out[o] = scale * z;
    }
}

// din[b][ci][y][x] (+)= sum over the effective positions the input (y, x) feeds
// (four when upsampled) of sum_co,k W[co][ci][k] dz[b][co][oy][ox], where the
// effective position e = o s + k - 1.
__global__ void __launch_bounds__(kT) conv_bwd_data_kernel(const float* __restrict__ dz,
                                                           const __nv_bfloat16* __restrict__ W, float* din, Layer L,
                                                           int accumulate) {
    const int b = blockIdx.z;
    const int ci = blockIdx.y;
    const size_t n = (size_t)L.hin * L.hin;
    const float* dzb = dz + (size_t)b * L.co * L.hout * L.hout;
    for (size_t i = blockIdx.x * (size_t)kT + threadIdx.x; i < n; i += (size_t)gridDim.x * kT) {
        const int x = (int)(i % L.hin), y = (int)(i / L.hin);
        float acc = 0.0f;
        const int reps = L.up ? 2 : 1;
        for (int dyy = 0; dyy < reps; ++dyy) {
            for (int dxx = 0; dxx < reps; ++dxx) {
                const int ey = L.up ? 2 * y + dyy : y, ex = L.up ? 2 * x + dxx : x;
                for (int k = 0; k < 9; ++k) {
                    const int ny = ey + 1 - k / 3, nx = ex + 1 - k % 3;
                    if (ny < 0 || nx < 0) continue;
                    if (L.stride == 2 && ((ny & 1) || (nx & 1))) continue;
                    const int oy = ny / L.stride, ox = nx / L.stride;
                    if (oy >= L.hout || ox >= L.hout) continue;
                    const float* dzp = dzb + (size_t)oy * L.hout + ox;
                    const __nv_bfloat16* wp = W + (size_t)ci * 9 + k;
                    for (int co = 0; co < L.co; ++co)
                        acc = fmaf(__bfloat162float(wp[(size_t)co * L.ci * 9]), __ldg(dzp + (size_t)co * L.hout * L.hout),
                                   acc);
                }
            }
        }
        float* o = din + ((size_t)b * L.ci + ci) * n + i;
        *o = accumulate ? *o + acc : acc;
    }
}

// Partial weight gradients: part[slice][co][ci][k] = sum over one slice of the
// (b, o) range of dz[b][co][o] in_eff[b][ci][o s + k - 1]; one thread per
// (co, ci) pair of an 8 x 8 tile.  The slices are summed in a fixed order by
// sum_slices_kernel, so the gradient does not depend on scheduling.
__global__ void __launch_bounds__(64) conv_bwd_weight_kernel(const float* __restrict__ in, const float* __restrict__ dz,
                                                             float* part, Layer L, int B, int slices) {
    const int co = blockIdx.y * 8 + (threadIdx.x >> 3);
    const int ci = blockIdx.z * 8 + (threadIdx.x & 7);
    const size_t P = (size_t)L.hout * L.hout;
    const size_t total = P * B;
    const size_t per = (total + slices - 1) / slices;
    const size_t p0 = (size_t)blockIdx.x * per, p1 = min(total, p0 + per);
    if (co >= L.co || ci >= L.ci) return;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
    for (size_t q = p0; q < p1; ++q) {
        const int b = (int)(q / P);
        const size_t o = q % P;
        const int oy = (int)(o / L.hout), ox = (int)(o % L.hout);
        const float g = __ldg(dz + ((size_t)b * L.co + co) * P + o);
        if (g == 0.0f) continue;
        const float* inc = in + ((size_t)b * L.ci + ci) * L.hin * L.hin;
#pragma unroll
        for (int k = 0; k < 9; ++k)
            acc[k] = fmaf(g, in_eff(inc, L.hin, L.up, oy * L.stride + k / 3 - 1, ox * L.stride + k % 3 - 1), acc[k]);
    }
    float* out = part + ((size_t)blockIdx.x * L.co * L.ci + (size_t)co * L.ci + ci) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = acc[k];
}

// dW[i] = sum_s part[s][i], s in increasing order.
__global__ void sum_slices_kernel(const float* __restrict__ part, float* dW, size_t n, int slices) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < slices; ++k) s += part[(size_t)k * n + i];
        dW[i] = s;
    }
}

// db[co] = sum_{b, o} dz[b][co][o]
__global__ void bias_grad_kernel(const float* __restrict__ dz, float* db, int C, size_t P, int B) {
    const int co = blockIdx.x;
    float s = 0.0f;
    for (size_t q = threadIdx.x; q < P * B; q += blockDim.x) s += dz[((q / P) * C + co) * P + q % P];
    __shared__ float red[kT];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[co] = red[0];
}

// g *= (r > 0): gradient through a relu whose output is r.
__global__ void relu_mask_kernel(float* g, const float* __restrict__ r, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (r[i] <= 0.0f) g[i] = 0.0f;
}

__global__ void stack_input_kernel(const float* __restrict__ T, const float* __restrict__ R, float* x, size_t n, int B) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * B; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / n, p = i % n;
        x[(b * 2) * n + p] = T[i];
        x[(b * 2 + 1) * n + p] = R[i];
    }
}

// loss partials (FP64) and the gradient of the loss with respect to the
// unscaled output z (v = scale z): dz = (v - t) / (scale N).
__global__ void mse_kernel(const float* __restrict__ v, const float* __restrict__ t, float* dz, size_t n, float scale,
                           double* partial) {
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float e = v[i] - t[i];
        s += (double)e * (double)e;
        dz[i] = e / (scale * (float)n);
    }
    __shared__ double red[kT];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void adam_kernel(float* p, const float* __restrict__ g, float* m, float* s, __nv_bfloat16* wb, size_t n,
                            float lr, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float si = 0.999f * s[i] + 0.001f * gi * gi;
        m[i] = mi;
        s[i] = si;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(si / c2) + 1e-8f);
        p[i] = pi;
        wb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* wb, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(p[i]);
}

inline int blocks_for(size_t n) {
    const size_t b = (n + kT - 1) / kT;
    return (int)(b < 4096 ? (b ? b : 1) : 4096);
}

}  // namespace

struct lgnk_ws {
    int m, c, max_batch;
    float scale;
    cudaStream_t stream;
    std::vector<Layer> L;
    size_t nparams;
    float *p, *g, *am, *as;     // master weights, gradients, Adam moments
    __nv_bfloat16* wb;          // bf16 weights
    float *x, *e0, *e1, *e2, *e3, *r4, *d2, *r5, *d1, *z6;   // activations
    float *ga, *gb, *gc;        // gradient scratch (largest activation each)
    float* wpart;               // per-slice weight-gradient partials
    double* partial;
    double* hres;
    long long steps;
    std::vector<void*> allocs;
    char err[256];
};

namespace {

lgnk_status ws_alloc(lgnk_ws* w, size_t bytes, void** out) {
    if (cudaMalloc(out, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        snprintf(w->err, sizeof(w->err), "cudaMalloc(%zu) failed", bytes);
        return LGNK_ERR_OOM;
    }
    w->allocs.push_back(*out);
    return LGNK_OK;
}

template <typename T>
lgnk_status ws_alloc_n(lgnk_ws* w, size_t n, T** out) {
    void* p = nullptr;
    const lgnk_status s = ws_alloc(w, n * sizeof(T), &p);
    *out = static_cast<T*>(p);
    return s;
}

size_t act_size(const lgnk_ws* w, int layer_out_c, int side, int B) { return (size_t)B * layer_out_c * side * side; }

cudaError_t conv_fwd(lgnk_ws* w, int l, const float* in, float* out, float* r, const float* add, int relu, float scale,
                     int B) {
    const Layer& L = w->L[l];
    const int tiles = (L.hout + 15) / 16;
    dim3 grid(tiles * tiles, (L.co + kCo - 1) / kCo, B);
    conv_fwd_kernel<<<grid, kT, 0, w->stream>>>(in, w->wb + L.woff, w->p + L.boff, out, r, add, L, relu, scale);
    return cudaGetLastError();
}

cudaError_t conv_bwd(lgnk_ws* w, int l, const float* in, const float* dz, float* din, int accumulate, int B) {
    const Layer& L = w->L[l];
    // weight and bias gradients
    const size_t P = (size_t)L.hout * L.hout * B;
    const int slices = (int)std::min<size_t>(kMaxSlices, (P + 1023) / 1024);
    dim3 gw(slices, (L.co + 7) / 8, (L.ci + 7) / 8);
    conv_bwd_weight_kernel<<<gw, 64, 0, w->stream>>>(in, dz, w->wpart, L, B, slices);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t nw = (size_t)L.co * L.ci * 9;
    sum_slices_kernel<<<blocks_for(nw), kT, 0, w->stream>>>(w->wpart, w->g + L.woff, nw, slices);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bias_grad_kernel<<<L.co, kT, 0, w->stream>>>(dz, w->g + L.boff, L.co, (size_t)L.hout * L.hout, B);
    e = cudaGetLastError();
    if (e != cudaSuccess || din == nullptr) return e;
    const size_t n = (size_t)L.hin * L.hin;
    dim3 gd((int)std::min<size_t>((n + kT - 1) / kT, 1024), L.ci, B);
    conv_bwd_data_kernel<<<gd, kT, 0, w->stream>>>(dz, w->wb + L.woff, din, L, accumulate);
    return cudaGetLastError();
}

lgnk_status forward_pass(lgnk_ws* w, int B, const float* T, const float* R, float* v) {
    const size_t n = (size_t)w->m * w->m;
    stack_input_kernel<<<blocks_for(n * B), kT, 0, w->stream>>>(T, R, w->x, n, B);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = conv_fwd(w, 0, w->x, w->e0, nullptr, nullptr, 1, 1.0f, B);
    if (e == cudaSuccess) e = conv_fwd(w, 1, w->e0, w->e1, nullptr, nullptr, 1, 1.0f, B);
    if (e == cudaSuccess) e = conv_fwd(w, 2, w->e1, w->e2, nullptr, nullptr, 1, 1.0f, B);
    if (e == cudaSuccess) e = conv_fwd(w, 3, w->e2, w->e3, nullptr, nullptr, 1, 1.0f, B);
    if (e == cudaSuccess) e = conv_fwd(w, 4, w->e3, w->d2, w->r4, w->e2, 1, 1.0f, B);
    if (e == cudaSuccess) e = conv_fwd(w, 5, w->d2, w->d1, w->r5, w->e1, 1, 1.0f, B);
    if (e == cudaSuccess) e = conv_fwd(w, 6, w->d1, v, nullptr, nullptr, 0, w->scale, B);
    if (e != cudaSuccess) {
        snprintf(w->err, sizeof(w->err), "%s", cudaGetErrorString(e));
        return LGNK_ERR_CUDA;
    }
    return LGNK_OK;
}

}  // namespace

#define WS_CHECK(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            snprintf(w->err, sizeof(w->err), "%s: %s", #call, cudaGetErrorString(e_)); \
            return LGNK_ERR_CUDA;                                                   \
        }                                                                           \
    } while (0)

extern "C" {

void lgnk_ws_destroy(lgnk_ws* w) {
    if (w == nullptr) return;
    for (void* p : w->allocs) cudaFree(p);
    if (w->hres) cudaFreeHost(w->hres);
    delete w;
}

lgnk_status lgnk_ws_create(int image_m, int base_channels, int max_batch, float output_scale, void* stream,
                           lgnk_ws** out) {
    if (out == nullptr) return LGNK_ERR_INVALID_ARG;
    *out = nullptr;
    if (image_m < 8 || image_m % 8 != 0 || image_m > 4096 || base_channels < 1 || base_channels > 256 ||
        max_batch < 1 || !(output_scale > 0.0f))
        return LGNK_ERR_INVALID_ARG;
    lgnk_ws* w = new (std::nothrow) lgnk_ws();
    if (w == nullptr) return LGNK_ERR_OOM;
    w->m = image_m;
    w->c = base_channels;
    w->max_batch = max_batch;
    w->scale = output_scale;
    w->stream = static_cast<cudaStream_t>(stream);
    const int c = base_channels, m = image_m;
    const int spec[7][5] = {{2, c, 1, 0, m},          {c, 2 * c, 2, 0, m},         {2 * c, 4 * c, 2, 0, m / 2},
                            {4 * c, 8 * c, 2, 0, m / 4}, {8 * c, 4 * c, 1, 1, m / 8}, {4 * c, 2 * c, 1, 1, m / 4},
                            {2 * c, 2, 1, 0, m / 2}};
    size_t off = 0;
    for (int l = 0; l < 7; ++l) {
        Layer L;
        L.ci = spec[l][0];
        L.co = spec[l][1];
        L.stride = spec[l][2];
        L.up = spec[l][3];
        L.hin = spec[l][4];
        L.hout = L.up ? 2 * L.hin : L.hin / L.stride;
        L.woff = off;
        off += (size_t)L.co * L.ci * 9;
        L.boff = off;
        off += L.co;
        w->L.push_back(L);
    }
    w->nparams = off;
    const int B = max_batch;
    lgnk_status s = LGNK_OK;
    auto fail = [&](lgnk_status st) {
        lgnk_ws_destroy(w);
        return st;
    };
    if ((s = ws_alloc_n(w, off, &w->p)) || (s = ws_alloc_n(w, off, &w->g)) || (s = ws_alloc_n(w, off, &w->am)) ||
        (s = ws_alloc_n(w, off, &w->as)) || (s = ws_alloc_n(w, off, &w->wb)))
        return fail(s);
    const size_t big = act_size(w, c, m, B);   // the largest activation: e0
    if ((s = ws_alloc_n(w, act_size(w, 2, m, B), &w->x)) || (s = ws_alloc_n(w, big, &w->e0)) ||
        (s = ws_alloc_n(w, act_size(w, 2 * c, m / 2, B), &w->e1)) ||
        (s = ws_alloc_n(w, act_size(w, 4 * c, m / 4, B), &w->e2)) ||
        (s = ws_alloc_n(w, act_size(w, 8 * c, m / 8, B), &w->e3)) ||
        (s = ws_alloc_n(w, act_size(w, 4 * c, m / 4, B), &w->r4)) ||
        (s = ws_alloc_n(w, act_size(w, 4 * c, m / 4, B), &w->d2)) ||
        (s = ws_alloc_n(w, act_size(w, 2 * c, m / 2, B), &w->r5)) ||
        (s = ws_alloc_n(w, act_size(w, 2 * c, m / 2, B), &w->d1)) ||
        (s = ws_alloc_n(w, act_size(w, 2, m / 2, B), &w->z6)) || (s = ws_alloc_n(w, big, &w->ga)) ||
        (s = ws_alloc_n(w, big, &w->gb)) || (s = ws_alloc_n(w, big, &w->gc)) ||
        (s = ws_alloc_n(w, (size_t)4096, &w->partial)))
        return fail(s);
    size_t wmax = 0;
    for (const Layer& L : w->L) wmax = std::max(wmax, (size_t)L.co * L.ci * 9);
    if ((s = ws_alloc_n(w, wmax * kMaxSlices, &w->wpart))) return fail(s);
    if (cudaMallocHost((void**)&w->hres, 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        w->hres = nullptr;
        return fail(LGNK_ERR_OOM);
    }
    if (cudaMemsetAsync(w->p, 0, off * sizeof(float), w->stream) != cudaSuccess ||
        cudaMemsetAsync(w->am, 0, off * sizeof(float), w->stream) != cudaSuccess ||
        cudaMemsetAsync(w->as, 0, off * sizeof(float), w->stream) != cudaSuccess ||
        cudaMemsetAsync(w->wb, 0, off * sizeof(__nv_bfloat16), w->stream) != cudaSuccess)
        return fail(LGNK_ERR_CUDA);
    *out = w;
    return LGNK_OK;
}

size_t lgnk_ws_num_params(const lgnk_ws* w) { return w ? w->nparams : 0; }

const char* lgnk_ws_last_error(const lgnk_ws* w) { return w ? w->err : "null network"; }

lgnk_status lgnk_ws_set_params(lgnk_ws* w, const float* params) {
    if (w == nullptr || params == nullptr) return LGNK_ERR_INVALID_ARG;
    WS_CHECK(cudaMemcpyAsync(w->p, params, w->nparams * sizeof(float), cudaMemcpyDeviceToDevice, w->stream));
    to_bf16_kernel<<<blocks_for(w->nparams), kT, 0, w->stream>>>(w->p, w->wb, w->nparams);
    WS_CHECK(cudaGetLastError());
    WS_CHECK(cudaMemsetAsync(w->am, 0, w->nparams * sizeof(float), w->stream));
    WS_CHECK(cudaMemsetAsync(w->as, 0, w->nparams * sizeof(float), w->stream));
    w->steps = 0;
    return LGNK_OK;
}

lgnk_status lgnk_ws_get_params(lgnk_ws* w, float* params) {
    if (w == nullptr || params == nullptr) return LGNK_ERR_INVALID_ARG;
    WS_CHECK(cudaMemcpyAsync(params, w->p, w->nparams * sizeof(float), cudaMemcpyDeviceToDevice, w->stream));
    return LGNK_OK;
}

lgnk_status lgnk_ws_get_grads(lgnk_ws* w, float* grads) {
    if (w == nullptr || grads == nullptr) return LGNK_ERR_INVALID_ARG;
    WS_CHECK(cudaMemcpyAsync(grads, w->g, w->nparams * sizeof(float), cudaMemcpyDeviceToDevice, w->stream));
    return LGNK_OK;
}

lgnk_status lgnk_ws_predict(lgnk_ws* w, int batch, const float* T, const float* R, float* v) {
    if (w == nullptr || T == nullptr || R == nullptr || v == nullptr || batch < 1 || batch > w->max_batch)
        return LGNK_ERR_INVALID_ARG;
    return forward_pass(w, batch, T, R, v);
}

lgnk_status lgnk_ws_train_step(lgnk_ws* w, int batch, const float* T, const float* R, const float* target, float lr,
                               double* loss) {
    if (w == nullptr || T == nullptr || R == nullptr || target == nullptr || batch < 1 || batch > w->max_batch)
        return LGNK_ERR_INVALID_ARG;
    const int B = batch;
    lgnk_status st = forward_pass(w, B, T, R, w->z6);
    if (st != LGNK_OK) return st;
    const int c = w->c, m = w->m;
    // loss and dz6 (gradient w.r.t. the unscaled output)
    const size_t nv = act_size(w, 2, m / 2, B);
    const int nb = blocks_for(nv) < 1024 ? blocks_for(nv) : 1024;
    float* dz6 = w->gc;
    mse_kernel<<<nb, kT, 0, w->stream>>>(w->z6, target, dz6, nv, w->scale, w->partial);
    WS_CHECK(cudaGetLastError());
    // layer 6: d(d1) -> ga
    float* dd1 = w->ga;
    WS_CHECK(conv_bwd(w, 6, w->d1, dz6, dd1, 0, B));
    // d1 = r5 + e1: d(e1) accumulates d(d1); dz5 = d(d1) * (r5 > 0)
    float* de1 = w->gb;
    const size_t n1 = act_size(w, 2 * c, m / 2, B);
    WS_CHECK(cudaMemcpyAsync(de1, dd1, n1 * sizeof(float), cudaMemcpyDeviceToDevice, w->stream));
    relu_mask_kernel<<<blocks_for(n1), kT, 0, w->stream>>>(dd1, w->r5, n1);
    WS_CHECK(cudaGetLastError());
    // layer 5 (input up2(d2)): d(d2) -> gc
    float* dd2 = w->gc;
    WS_CHECK(conv_bwd(w, 5, w->d2, dd1, dd2, 0, B));
    // d2 = r4 + e2: d(e2) accumulates d(d2); dz4 = d(d2) * (r4 > 0)
    const size_t n2 = act_size(w, 4 * c, m / 4, B);
    float* de2 = w->ga;   // dd1 is no longer needed
    WS_CHECK(cudaMemcpyAsync(de2, dd2, n2 * sizeof(float), cudaMemcpyDeviceToDevice, w->stream));
    relu_mask_kernel<<<blocks_for(n2), kT, 0, w->stream>>>(dd2, w->r4, n2);
    WS_CHECK(cudaGetLastError());
    // layer 4 (input up2(e3)): d(e3) -> ga + n2 (free room after de2)
    float* de3 = w->ga + n2;
    WS_CHECK(conv_bwd(w, 4, w->e3, dd2, de3, 0, B));
    const size_t n3 = act_size(w, 8 * c, m / 8, B);
    relu_mask_kernel<<<blocks_for(n3), kT, 0, w->stream>>>(de3, w->e3, n3);
    WS_CHECK(cudaGetLastError());
    // layer 3: d(e2) += ...
    WS_CHECK(conv_bwd(w, 3, w->e2, de3, de2, 1, B));
    relu_mask_kernel<<<blocks_for(n2), kT, 0, w->stream>>>(de2, w->e2, n2);
    WS_CHECK(cudaGetLastError());
    // layer 2: d(e1) += ...
    WS_CHECK(conv_bwd(w, 2, w->e1, de2, de1, 1, B));
    relu_mask_kernel<<<blocks_for(n1), kT, 0, w->stream>>>(de1, w->e1, n1);
    WS_CHECK(cudaGetLastError());
    // layer 1: d(e0) -> gc
    float* de0 = w->gc;
    WS_CHECK(conv_bwd(w, 1, w->e0, de1, de0, 0, B));
    const size_t n0 = act_size(w, c, m, B);
    relu_mask_kernel<<<blocks_for(n0), kT, 0, w->stream>>>(de0, w->e0, n0);
    WS_CHECK(cudaGetLastError());
    // layer 0: weights only
    WS_CHECK(conv_bwd(w, 0, w->x, de0, nullptr, 0, B));
    // Adam
    w->steps++;
    const float c1 = 1.0f - powf(0.9f, (float)w->steps), c2 = 1.0f - powf(0.999f, (float)w->steps);
    adam_kernel<<<blocks_for(w->nparams), kT, 0, w->stream>>>(w->p, w->g, w->am, w->as, w->wb, w->nparams, lr, c1, c2);
    WS_CHECK(cudaGetLastError());
    if (loss != nullptr) {
        launch_reduce(w->partial, nb, w->partial + 2048, w->stream);
        WS_CHECK(cudaGetLastError());
        WS_CHECK(cudaMemcpyAsync(w->hres, w->partial + 2048, sizeof(double), cudaMemcpyDeviceToHost, w->stream));
        WS_CHECK(cudaStreamSynchronize(w->stream));
        *loss = 0.5 * w->hres[0] / (double)nv / ((double)w->scale * w->scale);
    }
    return LGNK_OK;
}

}  // extern "C"

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
//
// Every convolution, its data gradient and its weight gradient run as implicit
// GEMMs on the tensor cores (conv_umma.cuh); bias gradients, the loss, the
// ReLU masks and Adam are elementwise kernels here.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "conv_umma.cuh"
#include "lgnk_internal.h"

namespace {

constexpr int kT = 256;
constexpr int kMaxSlices = 64;   // K slices of the weight-gradient GEMM (partials summed in order)

struct Layer {
    int ci, co, stride, up;   // input channels, output channels, stride, input upsampled
    int hin, hout;            // input and output side lengths (square)
    size_t woff, boff;        // offsets of W and b in the parameter vector
    // bf16 weight matrices of the tensor-core GEMMs, zero padded, K ordered
    // as the operand planes are (channel fastest):
    // forward wf[co][tap * cpi + ci] (cpi = ci rounded up to 8; rows to a
    // multiple of bnf, rows of ldf), data gradient
    // wd[ci][(tap * R + up position) * cpo + co] (cpo = co rounded up to 8, R = 4 when up)
    int cpi, cpo, bnf, ldf, rowsf, bnd, ldd, rowsd;
    __nv_bfloat16 *wf, *wd;
};

#ifndef LGNK_CONV_STAGES
#define LGNK_CONV_STAGES 1    // operand buffers per CTA (1: two CTAs per SM)
#endif

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// The GEMMs' weight matrices from the FP32 master weights (bf16, nearest).
__global__ void pack_wmats_kernel(const float* __restrict__ p, Layer L) {
    const size_t nf = (size_t)L.rowsf * L.ldf, nd = (size_t)L.rowsd * L.ldd;
    const int R = L.up ? 4 : 1;
    const float* W = p + L.woff;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nf + nd; i += (size_t)gridDim.x * blockDim.x) {
        float v = 0.0f;
        if (i < nf) {
            const int n = (int)(i / L.ldf), k = (int)(i % L.ldf);
            const int t = k / L.cpi, c = k - t * L.cpi;
            if (n < L.co && t < 9 && c < L.ci) v = W[((size_t)n * L.ci + c) * 9 + t];
            L.wf[i] = __float2bfloat16_rn(v);
        } else {
            const size_t j = i - nf;
            const int n = (int)(j / L.ldd), k = (int)(j % L.ldd);
            const int pos = k / L.cpo, cc = k - pos * L.cpo, t = pos / R;
            if (n < L.ci && t < 9 && cc < L.co) v = W[((size_t)cc * L.ci + n) * 9 + t];
            L.wd[j] = __float2bfloat16_rn(v);
        }
    }
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

__global__ void adam_kernel(float* p, const float* __restrict__ g, float* m, float* s, size_t n, float lr, float c1,
                            float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float si = 0.999f * s[i] + 0.001f * gi * gi;
        m[i] = mi;
        s[i] = si;
        p[i] = p[i] - lr * (mi / c1) / (sqrtf(si / c2) + 1e-8f);
    }
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
    float *x, *e0, *e1, *e2, *e3, *r4, *d2, *r5, *d1, *z6;   // activations
    float *ga, *gb, *gc;        // gradient scratch (largest activation each)
    float* wpart;               // per-slice weight-gradient partials
    __nv_bfloat16* planes;      // bf16 planes of a GEMM operand (umma::split_planes_kernel)
    size_t planes_cap;          // elements of one plane it holds
    float* gpart;               // split-K partial tiles of the FWD and BWD_DATA GEMMs
    size_t gpart_cap;           // floats it holds
    int* derr;                  // set by a tensor-core kernel whose wait ran out
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

// planes of src [B][C][h][h] into w->planes (channels padded to cp)
cudaError_t split_planes(lgnk_ws* w, const float* src, int B, int C, int h, int cp, size_t* plane_elems) {
    *plane_elems = (size_t)B * h * h * cp;
    if (*plane_elems > w->planes_cap) return cudaErrorInvalidValue;
    const size_t n = (size_t)B * h * h * (cp / 8);
    umma::split_planes_kernel<<<blocks_for(n), kT, 0, w->stream>>>(src, w->planes, B, C, h, cp);
    return cudaGetLastError();
}

// CTAs a GEMM launch should reach: two per SM
constexpr int kGemmCtas = 2 * 152;

// K slices of a FWD / BWD_DATA GEMM with `tiles` output tiles and `chunks` K
// chunks: enough slices to give about two CTAs per SM, each at least two
// chunks (1 when the tiles alone fill the GPU)
inline int split_slices(int tiles, int chunks) {
    if (tiles >= kGemmCtas) return 1;
    const int s = std::min((kGemmCtas + tiles - 1) / tiles, std::max(1, chunks / 2));
    const int cps = (chunks + s - 1) / s;
    return (chunks + cps - 1) / cps;
}

cudaError_t launch_gemm(lgnk_ws* w, umma::ConvGemm& g, int grid_x, int grid_y, int grid_z) {
    g.stages = LGNK_CONV_STAGES;
    const size_t smem = (size_t)g.stages * umma::stage_bytes(g.kind, g.bn);
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, umma::conv_gemm_kernel);
    if (e == cudaSuccess && smem + fa.sharedSizeBytes > (size_t)optin) e = cudaErrorInvalidValue;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(umma::conv_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    g.err = w->derr;
    umma::conv_gemm_kernel<<<dim3(grid_x, grid_y, grid_z), umma::kThreads, smem, w->stream>>>(g);
    return cudaGetLastError();
}

// a FWD or BWD_DATA GEMM, split along K when its tiles do not fill the GPU
cudaError_t launch_gemm_split(lgnk_ws* w, umma::ConvGemm& g, int grid_y) {
    const int gx = (g.M + umma::BM - 1) / umma::BM;
    const int chunks = (g.K + umma::BK - 1) / umma::BK;
    const int splits = split_slices(gx * grid_y, chunks);
    g.chunks_per_split = (chunks + splits - 1) / splits;
    g.part = w->gpart;
    if (splits > 1 && (size_t)splits * g.M * g.N > w->gpart_cap) return cudaErrorInvalidValue;
    cudaError_t e = launch_gemm(w, g, gx, grid_y, splits);
    if (e != cudaSuccess || splits == 1) return e;
    umma::finish_split_kernel<<<blocks_for((size_t)g.M * g.N), kT, 0, w->stream>>>(g, splits);
    return cudaGetLastError();
}

umma::ConvGemm gemm_base(const Layer& L, int kind, int B) {
    umma::ConvGemm g{};
    g.kind = kind;
    g.ci = L.ci;
    g.co = L.co;
    g.stride = L.stride;
    g.up = L.up;
    g.hin = L.hin;
    g.hout = L.hout;
    g.batch = B;
    return g;
}

// out = scale (act(conv(in) + b) + add), r = act(conv(in) + b) (tensor-core GEMM)
cudaError_t conv_fwd(lgnk_ws* w, int l, const float* in, float* out, float* r, const float* add, int relu, float scale,
                     int B) {
    const Layer& L = w->L[l];
    umma::ConvGemm g = gemm_base(L, umma::FWD, B);
    g.M = B * L.hout * L.hout;
    g.N = L.co;
    g.K = 9 * L.cpi;
    g.cp = L.cpi;
    g.bn = L.bnf;
    cudaError_t e = split_planes(w, in, B, L.ci, L.hin, L.cpi, &g.plane_elems);
    if (e != cudaSuccess) return e;
    g.planes = w->planes;
    g.w = L.wf;
    g.wld = L.ldf;
    g.out = out;
    g.r = r;
    g.add = add;
    g.bias = w->p + L.boff;
    g.relu = relu;
    g.scale = scale;
    return launch_gemm_split(w, g, L.rowsf / L.bnf);
}

// weight and bias gradients of layer l from its input `in` and output gradient
// dz; with din, also the input gradient (added to din when accumulate)
cudaError_t conv_bwd(lgnk_ws* w, int l, const float* in, const float* dz, float* din, int accumulate, int B) {
    const Layer& L = w->L[l];
    // weight gradient: D[co][(ci, tap)] over the batch's pixels, K split into slices
    umma::ConvGemm g = gemm_base(L, umma::BWD_WEIGHT, B);
    g.M = L.co;
    g.N = L.ci * 9;
    g.K = B * L.hout * L.hout;
    g.bn = std::min(128, round_up(g.N, 16));
    const int gx = (g.M + umma::BM - 1) / umma::BM, gy = (g.N + g.bn - 1) / g.bn;
    const int chunks = (g.K + umma::BK - 1) / umma::BK;
    int slices = std::min(kMaxSlices, std::min(chunks, std::max(1, (2 * 152 + gx * gy - 1) / (gx * gy))));
    g.chunks_per_split = (chunks + slices - 1) / slices;
    slices = (chunks + g.chunks_per_split - 1) / g.chunks_per_split;
    g.a = dz;
    g.x = in;
    g.out = w->wpart;
    cudaError_t e = launch_gemm(w, g, gx, gy, slices);
    if (e != cudaSuccess) return e;
    const size_t nw = (size_t)L.co * L.ci * 9;
    sum_slices_kernel<<<blocks_for(nw), kT, 0, w->stream>>>(w->wpart, w->g + L.woff, nw, slices);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bias_grad_kernel<<<L.co, kT, 0, w->stream>>>(dz, w->g + L.boff, L.co, (size_t)L.hout * L.hout, B);
    e = cudaGetLastError();
    if (e != cudaSuccess || din == nullptr) return e;
    // data gradient: D[input pixel][ci]
    umma::ConvGemm d = gemm_base(L, umma::BWD_DATA, B);
    d.M = B * L.hin * L.hin;
    d.N = L.ci;
    d.K = 9 * (L.up ? 4 : 1) * L.cpo;
    d.cp = L.cpo;
    d.bn = L.bnd;
    e = split_planes(w, dz, B, L.co, L.hout, L.cpo, &d.plane_elems);
    if (e != cudaSuccess) return e;
    d.planes = w->planes;
    d.w = L.wd;
    d.wld = L.ldd;
    d.out = din;
    d.accumulate = accumulate;
    return launch_gemm_split(w, d, L.rowsd / L.bnd);
}

// refresh the GEMMs' bf16 weight matrices from the master weights
cudaError_t pack_weights(lgnk_ws* w) {
    for (const Layer& L : w->L) {
        const size_t n = (size_t)L.rowsf * L.ldf + (size_t)L.rowsd * L.ldd;
        pack_wmats_kernel<<<blocks_for(n), kT, 0, w->stream>>>(w->p, L);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
        (s = ws_alloc_n(w, off, &w->as)) || (s = ws_alloc_n(w, 1, &w->derr)))
        return fail(s);
    // the GEMMs' bf16 weight matrices (N per CTA up to 256, rows and K padded)
    size_t pmax = 0;
    for (Layer& L : w->L) {
        const int R = L.up ? 4 : 1;
        L.cpi = round_up(L.ci, 8);
        L.cpo = round_up(L.co, 8);
        L.bnf = std::min(256, round_up(L.co, 16));
        L.rowsf = round_up(L.co, L.bnf);
        L.ldf = round_up(9 * L.cpi, umma::BK);
        L.bnd = std::min(256, round_up(L.ci, 16));
        L.rowsd = round_up(L.ci, L.bnd);
        L.ldd = round_up(9 * R * L.cpo, umma::BK);
        pmax = std::max(pmax, (size_t)B * L.hin * L.hin * L.cpi);
        pmax = std::max(pmax, (size_t)B * L.hout * L.hout * L.cpo);
        if ((s = ws_alloc_n(w, (size_t)L.rowsf * L.ldf, &L.wf)) || (s = ws_alloc_n(w, (size_t)L.rowsd * L.ldd, &L.wd)))
            return fail(s);
    }
    w->planes_cap = pmax;
    if ((s = ws_alloc_n(w, 3 * pmax, &w->planes))) return fail(s);
    // split-K partials: the largest splits x M x N any batch size up to max_batch needs
    size_t gmax = 1;
    for (int b = 1; b <= B; ++b) {
        for (const Layer& L : w->L) {
            const int R = L.up ? 4 : 1;
            const long long Mf = (long long)b * L.hout * L.hout, Md = (long long)b * L.hin * L.hin;
            const int tf = (int)((Mf + umma::BM - 1) / umma::BM) * (L.rowsf / L.bnf);
            const int td = (int)((Md + umma::BM - 1) / umma::BM) * (L.rowsd / L.bnd);
            const int sf = split_slices(tf, (9 * L.cpi + umma::BK - 1) / umma::BK);
            const int sd = split_slices(td, (9 * R * L.cpo + umma::BK - 1) / umma::BK);
            if (sf > 1) gmax = std::max(gmax, (size_t)sf * (size_t)Mf * L.co);
            if (sd > 1) gmax = std::max(gmax, (size_t)sd * (size_t)Md * L.ci);
        }
    }
    w->gpart_cap = gmax;
    if ((s = ws_alloc_n(w, gmax, &w->gpart))) return fail(s);
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
        cudaMemsetAsync(w->derr, 0, sizeof(int), w->stream) != cudaSuccess || pack_weights(w) != cudaSuccess)
        return fail(LGNK_ERR_CUDA);
    *out = w;
    return LGNK_OK;
}

size_t lgnk_ws_num_params(const lgnk_ws* w) { return w ? w->nparams : 0; }

const char* lgnk_ws_last_error(const lgnk_ws* w) { return w ? w->err : "null network"; }

lgnk_status lgnk_ws_set_params(lgnk_ws* w, const float* params) {
    if (w == nullptr || params == nullptr) return LGNK_ERR_INVALID_ARG;
    WS_CHECK(cudaMemcpyAsync(w->p, params, w->nparams * sizeof(float), cudaMemcpyDeviceToDevice, w->stream));
    WS_CHECK(pack_weights(w));
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
    adam_kernel<<<blocks_for(w->nparams), kT, 0, w->stream>>>(w->p, w->g, w->am, w->as, w->nparams, lr, c1, c2);
    WS_CHECK(cudaGetLastError());
    WS_CHECK(pack_weights(w));
    if (loss != nullptr) {
        launch_reduce(w->partial, nb, w->partial + 2048, w->stream);
        WS_CHECK(cudaGetLastError());
        WS_CHECK(cudaMemcpyAsync(w->hres, w->partial + 2048, sizeof(double), cudaMemcpyDeviceToHost, w->stream));
        WS_CHECK(cudaMemcpyAsync(w->hres + 1, w->derr, sizeof(int), cudaMemcpyDeviceToHost, w->stream));
        WS_CHECK(cudaStreamSynchronize(w->stream));
        int bad = 0;
        memcpy(&bad, w->hres + 1, sizeof(int));
        if (bad != 0) {
            snprintf(w->err, sizeof(w->err), "a tensor-core convolution gave up waiting for its MMAs");
            return LGNK_ERR_INTERNAL;
        }
        *loss = 0.5 * w->hres[0] / (double)nv / ((double)w->scale * w->scale);
    }
    return LGNK_OK;
}

}  // extern "C"

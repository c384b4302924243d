// Tensor-core convolutions of the warm-start network: every 3x3 convolution
// and both of its gradients as an implicit GEMM on the 5th-generation tensor
// cores (tcgen05.mma, kind::f16: bf16 operands, FP32 accumulation in tensor
// memory).
//
//   forward       D[pixel][co]      = sum_(ci,tap) x_eff[pixel + tap][ci] W[co][ci][tap]
//   data gradient D[in pixel][ci]   = sum_(co,tap,up) dz[pixel - tap][co] W[co][ci][tap]
//   weight grad.  D[co][(ci,tap)]   = sum_pixel dz[pixel][co] x_eff[pixel + tap][ci]
//
// The network's FP32 activations and gradients enter as sums of three bf16
// planes, x = hi + mid + lo with hi = bf16(x), mid = bf16(x - hi), lo =
// bf16(x - hi - mid) (exact: each difference is exact in FP32 and has at most
// 16, then 8 significant bits), so the products the tensor cores form are the
// exact products of the FP32 values with the bf16 weights, accumulated in
// FP32: the arithmetic of the network as specified (bf16 weights, FP32
// activations and accumulation), not a bf16 approximation of it.  The weight
// gradient multiplies two FP32 operands; the six plane products whose
// exponents reach 2^-16 of the leading one are formed (the three dropped
// ones are below FP32 resolution).
//
// One CTA of 128 threads computes a 128 x BN tile of D.  Per K chunk of 64,
// the threads gather the operands (the im2col addressing of the convolution)
// and write them to shared memory in the K-major canonical layout of the
// tensor cores without swizzle: core matrices of 8 rows x 16 bytes, the 8
// core matrices of a row group along K at 128-byte steps (leading byte
// offset 128), row groups at 1024-byte steps (stride byte offset 1024).  One
// elected thread issues the MMAs (K = 16 each) and commits them to the
// stage's mbarrier; with two stages the gather of chunk c + 1 overlaps the
// MMAs of chunk c, with one the next gather waits for them (and two CTAs fit
// on an SM instead, overlapping each other).  The epilogue reads the accumulator from
// tensor memory (tcgen05.ld, each warp its 32 lanes) and applies bias, ReLU,
// skip connection and scale, or writes gradients / weight-gradient partials.
// Every mbarrier wait is bounded; a wait that runs out sets an error flag,
// waits once more for the MMAs in flight, skips the epilogue and frees the
// tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace umma {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kThreads = 128;
constexpr int kMaxStages = 2;
constexpr int kTileBytes = BM * BK * 2;     // one bf16 plane of a 128 x 64 operand tile
constexpr long kWaitLimit = 1L << 22;       // mbarrier polls before giving up

enum Kind { FWD = 0, BWD_DATA = 1, BWD_WEIGHT = 2 };

struct ConvGemm {
    int kind;
    int ci, co, stride, up, hin, hout, batch;   // the layer and the batch
    int cp;                   // FWD: input channels padded to 8; BWD_DATA: output channels padded to 8
    int M, N, K;              // GEMM sizes
    int bn;                   // N per CTA: multiple of 16, <= 256 (<= 128 for BWD_WEIGHT)
    int chunks_per_split;     // K chunks per CTA along grid.z (split K; every chunk when grid.z = 1)
    float* part;              // FWD, BWD_DATA with grid.z > 1: raw partial tiles [z][N][M], finished by
                              // finish_split_kernel
    int stages;               // operand buffers in shared memory (1 or 2)
    const float* a;           // BWD_WEIGHT: output gradient dz
    const __nv_bfloat16* planes;  // FWD: the input's planes; BWD_DATA: dz's planes ([3][B][h][h][cp], see split_planes)
    size_t plane_elems;       // elements of one plane
    const float* x;           // BWD_WEIGHT: layer input x (the B operand)
    const __nv_bfloat16* w;   // FWD, BWD_DATA: weight matrix [rows >= N rounded to bn][wld], zero padded
    int wld;                  // its row length (K rounded up to 64)
    float* out;               // FWD: layer output; BWD_DATA: input gradient; BWD_WEIGHT: partials [z][co][ci*9]
    float* r;                 // FWD: activation before the skip add (may be NULL)
    const float* add;         // FWD: skip tensor (may be NULL)
    const float* bias;        // FWD
    int relu;
    float scale;
    int accumulate;           // BWD_DATA: out += instead of out =
    int* err;                 // set to 1 when a wait runs out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major without swizzle (leading byte
// offset: core matrices along K; stride byte offset: 8-row groups).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity));
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long i = 0; i < kWaitLimit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// x = hi + mid + lo exactly (see the file comment)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// Byte offset of the 16-byte chunk (row, k group) in a canonical tile.
__device__ __forceinline__ uint32_t chunk_off(int row, int kg) {
    return (uint32_t)(((row >> 3) * 8 + kg) * 128 + (row & 7) * 16);
}

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

// Element (row, k) of the A operand of BWD_WEIGHT: row = output channel, k
// = pixel of the batch (zero outside the GEMM).
__device__ __forceinline__ float a_elem(const ConvGemm& g, int row, int k) {
    if (row >= g.M || k >= g.K) return 0.0f;
    const int P = g.hout * g.hout;
    const int b = k / P, o = k - b * P;
    return __ldg(g.a + ((size_t)b * g.co + row) * P + o);
}

// The row of A a thread gathers for FWD and BWD_DATA, decomposed once: its
// image and pixel coordinates (rows past M are marked invalid).
struct RowCtx {
    bool valid;
    int b, y, x;     // FWD: output pixel (oy, ox); BWD_DATA: input pixel (iy, ix)
};

__device__ __forceinline__ RowCtx row_ctx(const ConvGemm& g, int row) {
    RowCtx r;
    r.valid = row < g.M;
    const int h = g.kind == FWD ? g.hout : g.hin;
    const int P = h * h;
    r.b = row / P;
    const int p = row - r.b * P;
    r.y = p / h;
    r.x = p - r.y * h;
    return r;
}

// The source of the 16-byte chunks (three planes) of A at the thread's row
// for the K position `pos` (tap, or tap and up position) and channels c0 ..
// c0 + 7, for FWD and BWD_DATA: K runs over (pos, channel) with the channel
// fastest, so a chunk is 8 channels of one source pixel of the NHWC planes.
// Returns false where the tap falls outside (the chunk is zero); e receives
// the element offset of the chunk in one plane.
__device__ __forceinline__ bool a_chunk_src(const ConvGemm& g, const RowCtx& r, int pos, int c0, size_t* e) {
    if (!r.valid || pos >= (g.up && g.kind == BWD_DATA ? 36 : 9)) return false;
    int y, x, h;
    if (g.kind == FWD) {
        const int ky = pos / 3, kx = pos - ky * 3;
        const int ey = r.y * g.stride + ky - 1, ex = r.x * g.stride + kx - 1;
        const int he = g.up ? 2 * g.hin : g.hin;
        if (ey < 0 || ex < 0 || ey >= he || ex >= he) return false;
        y = g.up ? ey >> 1 : ey;
        x = g.up ? ex >> 1 : ex;
        h = g.hin;
    } else {   // BWD_DATA: pos = tap * R + up position
        const int R = g.up ? 4 : 1;
        const int t = pos / R, dd = pos - t * R;
        const int ky = t / 3, kx = t - ky * 3;
        const int ey = g.up ? 2 * r.y + (dd >> 1) : r.y, ex = g.up ? 2 * r.x + (dd & 1) : r.x;
        const int ny = ey + 1 - ky, nx = ex + 1 - kx;
        if (ny < 0 || nx < 0) return false;
        if (g.stride == 2 && ((ny | nx) & 1)) return false;
        y = ny / g.stride;
        x = nx / g.stride;
        if (y >= g.hout || x >= g.hout) return false;
        h = g.hout;
    }
    *e = (((size_t)r.b * h + y) * h + x) * g.cp + c0;
    return true;
}

// 16 bytes global -> shared without passing through registers; with
// valid == false the 16 shared bytes are zero-filled and nothing is read.
__device__ __forceinline__ void cp_async16(uint8_t* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0));
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Three bf16 planes of an FP32 tensor [B][C][h][h] (NCHW) in NHWC order with
// the channels padded to cp (a multiple of 8) by zeros: plane q, element
// ((b h + y) h + x) cp + c.  One thread per 8 channels of one pixel.
__global__ void split_planes_kernel(const float* __restrict__ src, __nv_bfloat16* planes, int B, int C, int h,
                                    int cp) {
    const size_t P = (size_t)h * h;
    const size_t n = (size_t)B * P * (cp / 8);
    const size_t pe = (size_t)B * P * cp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t pix = i % (B * P);            // consecutive threads: consecutive pixels (coalesced reads)
        const int c0 = (int)(i / (B * P)) * 8;
        const size_t b = pix / P, o = pix % P;
        __align__(16) __nv_bfloat16 hv[8], mv[8], lv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = c0 + j;
            const float v = c < C ? __ldg(src + (b * C + c) * P + o) : 0.0f;
            split3(v, hv[j], mv[j], lv[j]);
        }
        const size_t e = pix * cp + c0;
        *reinterpret_cast<uint4*>(planes + e) = *reinterpret_cast<const uint4*>(hv);
        *reinterpret_cast<uint4*>(planes + pe + e) = *reinterpret_cast<const uint4*>(mv);
        *reinterpret_cast<uint4*>(planes + 2 * pe + e) = *reinterpret_cast<const uint4*>(lv);
    }
}

// Element (row, k) of the B operand of BWD_WEIGHT: row = (ci, tap), k = pixel.
__device__ __forceinline__ float bw_elem(const ConvGemm& g, int row, int k) {
    if (row >= g.N || k >= g.K) return 0.0f;
    const int P = g.hout * g.hout;
    const int b = k / P, o = k - b * P;
    const int oy = o / g.hout, ox = o - oy * g.hout;
    const int c = row / 9, t = row - c * 9;
    const int ky = t / 3, kx = t - ky * 3;
    const float* in = g.x + ((size_t)b * g.ci + c) * g.hin * g.hin;
    return in_eff(in, g.hin, g.up, oy * g.stride + ky - 1, ox * g.stride + kx - 1);
}

// Gather 8 FP32 values (row, k0 .. k0 + 7) and store their three bf16 planes
// at chunk offset `off` of the plane tiles starting at `planes` (kTileBytes
// apart for A, bn * 128 apart for B).
template <bool IS_A>
__device__ __forceinline__ void gather_split(const ConvGemm& g, int row, int k0, uint8_t* planes, uint32_t pstride,
                                             uint32_t off) {
    __align__(16) __nv_bfloat16 h[8], m[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float v = IS_A ? a_elem(g, row, k0 + j) : bw_elem(g, row, k0 + j);
        split3(v, h[j], m[j], l[j]);
    }
    *reinterpret_cast<uint4*>(planes + off) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(planes + pstride + off) = *reinterpret_cast<const uint4*>(m);
    *reinterpret_cast<uint4*>(planes + 2 * pstride + off) = *reinterpret_cast<const uint4*>(l);
}

__host__ __device__ inline size_t stage_bytes(int kind, int bn) {
    return (size_t)3 * kTileBytes + (size_t)(kind == BWD_WEIGHT ? 3 : 1) * bn * BK * 2;
}

__global__ void __launch_bounds__(kThreads, 1) conv_gemm_kernel(const ConvGemm g) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar[kMaxStages];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool bw = g.kind == BWD_WEIGHT;
    const int pb = bw ? 3 : 1;                    // B planes
    const uint32_t bplane = (uint32_t)g.bn * BK * 2;
    const size_t sbytes = stage_bytes(g.kind, g.bn);
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * g.bn;
    const int nchunks_all = (g.K + BK - 1) / BK;
    const int c_begin = blockIdx.z * g.chunks_per_split;
    const int c_end = min(nchunks_all, c_begin + g.chunks_per_split);
    const bool split = !bw && gridDim.z > 1;
    const uint32_t ncols = g.bn <= 32 ? 32u : (g.bn <= 64 ? 64u : (g.bn <= 128 ? 128u : 256u));

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kMaxStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar[s])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = instr_desc(BM, g.bn);

    const RowCtx rc = row_ctx(g, m0 + tid);    // FWD, BWD_DATA: this thread's A row
    bool failed = false;
    int issued = 0;
    int last = -1;      // index (from c_begin) of the last chunk whose MMAs were committed
    for (int c = c_begin; c < c_end; ++c) {
        const int S = g.stages, i = c - c_begin, s = i % S;
        uint8_t* sa = smem + s * sbytes;
        uint8_t* sb = sa + 3 * kTileBytes;
        if (i >= S) {   // the MMAs of chunk i - S read this stage (its use i / S - 1): one thread polls
            const bool ok = tid != 0 || mbar_wait(&bar[s], (uint32_t)((i / S - 1) & 1));
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        const int k0 = c * BK;
        // A: 128 rows x 8 k groups
        if (g.kind == BWD_WEIGHT) {
            for (int it = tid; it < BM * 8; it += kThreads) {    // lanes along k: contiguous pixels
                const int row = it >> 3, kg = it & 7;
                gather_split<true>(g, m0 + row, k0 + kg * 8, sa, kTileBytes, chunk_off(row, kg));
            }
        } else {
            // lanes along rows: neighbouring pixels; (pos, c0) of k0 + 8 kg stepped, not divided.
            // The 24 copies of a thread are all in flight before the wait below.
            int pos = k0 / g.cp, c0 = k0 - pos * g.cp;
#pragma unroll
            for (int kg = 0; kg < 8; ++kg) {
                size_t e = 0;
                const bool ok = a_chunk_src(g, rc, pos, c0, &e);
                const uint32_t off = chunk_off(tid, kg);
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    cp_async16(sa + q * kTileBytes + off, g.planes + q * g.plane_elems + (ok ? e : 0), ok);
                c0 += 8;
                if (c0 == g.cp) {
                    c0 = 0;
                    ++pos;
                }
            }
        }
        // B: bn rows x 8 k groups
        if (bw) {
            for (int it = tid; it < g.bn * 8; it += kThreads) {
                const int row = it >> 3, kg = it & 7;
                gather_split<false>(g, n0 + row, k0 + kg * 8, sb, bplane, chunk_off(row, kg));
            }
        } else {
            for (int it = tid; it < g.bn * 8; it += kThreads) {
                const int row = it >> 3, kg = it & 7;
                cp_async16(sb + chunk_off(row, kg), g.w + (size_t)(n0 + row) * g.wld + k0 + kg * 8, true);
            }
            cp_async_wait_all();
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                // plane pairs (pa, pb) with pa + pb <= 2
#pragma unroll
                for (int pa = 0; pa < 3; ++pa) {
                    for (int q = 0; q < pb && pa + q <= 2; ++q) {
                        const uint64_t ad = smem_desc(a0 + pa * kTileBytes + kk * 256, 128, 1024);
                        const uint64_t bd = smem_desc(b0 + q * bplane + kk * 256, 128, 1024);
                        mma_bf16(tmem, ad, bd, idesc, (issued > 0) ? 1u : 0u);
                        ++issued;
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar[s])));
        }
        last = i;   // a later chunk reusing this stage waits for these MMAs first (above)
    }
    if (!failed && last >= 0) {
        // the last commit covers every MMA issued before it
        const bool ok = tid != 0 || mbar_wait(&bar[last % g.stages], (uint32_t)((last / g.stages) & 1));
        failed = __syncthreads_or(!ok);
    }
    if (failed) {
        if (tid == 0) atomicExch(g.err, 1);
        // once more, bounded, for whatever is still in flight
        if (tid == 0 && last >= 0) mbar_wait(&bar[last % g.stages], (uint32_t)((last / g.stages) & 1));
    } else if (last >= 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int row = m0 + warp * 32 + lane;     // this thread's accumulator row (TMEM lane)
        for (int c0 = 0; c0 < g.bn; c0 += 16) {
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (row >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = n0 + c0 + j;
                if (n >= g.N) break;
                const float acc = __uint_as_float(v[j]);
                if (split) {
                    g.part[((size_t)blockIdx.z * g.N + n) * g.M + row] = acc;
                } else if (g.kind == FWD) {
                    const int P = g.hout * g.hout;
                    const int b = row / P, o = row - b * P;
                    const size_t oi = ((size_t)b * g.co + n) * P + o;
                    float z = acc + g.bias[n];
                    if (g.relu) z = fmaxf(z, 0.0f);
                    if (g.r != nullptr) g.r[oi] = z;
                    if (g.add != nullptr) z += g.add[oi];
                    g.out[oi] = g.scale * z;
                } else if (g.kind == BWD_DATA) {
                    const int P = g.hin * g.hin;
                    const int b = row / P, p = row - b * P;
                    float* o = g.out + ((size_t)b * g.ci + n) * P + p;
                    *o = g.accumulate ? *o + acc : acc;
                } else {
                    g.out[((size_t)blockIdx.z * g.co + row) * g.N + n] = acc;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// The end of a split-K FWD or BWD_DATA GEMM: the partial tiles summed over z
// in increasing order (deterministic), then the epilogue of the unsplit
// kernel.  One thread per (n, row), rows fastest.
__global__ void finish_split_kernel(const ConvGemm g, int splits) {
    const size_t total = (size_t)g.M * g.N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int n = (int)(i / g.M), row = (int)(i - (size_t)n * g.M);
        float acc = 0.0f;
        for (int z = 0; z < splits; ++z) acc += g.part[((size_t)z * g.N + n) * g.M + row];
        if (g.kind == FWD) {
            const int P = g.hout * g.hout;
            const int b = row / P, o = row - b * P;
            const size_t oi = ((size_t)b * g.co + n) * P + o;
            float z = acc + g.bias[n];
            if (g.relu) z = fmaxf(z, 0.0f);
            if (g.r != nullptr) g.r[oi] = z;
            if (g.add != nullptr) z += g.add[oi];
            g.out[oi] = g.scale * z;
        } else {
            const int P = g.hin * g.hin;
            const int b = row / P, p = row - b * P;
            float* o = g.out + ((size_t)b * g.ci + n) * P + p;
            *o = g.accumulate ? *o + acc : acc;
        }
    }
}

}  // namespace umma

// Allocation-free variant of the transport forward/SSD path: its scratch lives
// in a file-scope device array instead of a context's cudaMalloc'd buffers.
//
// Who needs it: callers that must not call cudaMalloc after start-up.  A
// latency-critical loop cannot afford it (cudaMalloc may synchronise the
// device and takes an unbounded time), and a process whose device memory has
// already been handed to another allocator (a framework's caching allocator,
// a pool sized at start-up) may find no free memory left to allocate.  Such a
// caller passes only its own inputs and outputs; this file never allocates.
#include <cstdio>
#include <mutex>

#include "lgnk_internal.h"

// Largest scratch a call may use.  Every GPU that loads the library holds this
// array until the process exits.
#define LGNK_STATIC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_static_scratch[LGNK_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of g_static_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, with that device current.  A reset of the device
// (cudaDeviceReset, or its primary context destroyed and created again)
// reloads the module and can move the array, so every call made outside a
// stream capture looks the address up again; a call made while `s` is being
// captured uses the address its device's last uncaptured call found (the
// lookup may load the module, which a capture does not allow), so the first
// call on a device must come before any capture.
lgnk_status scratch_address(cudaStream_t s, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        lgnk_internal_set_error(cudaGetErrorString(e));
        return LGNK_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        lgnk_internal_set_error("device index beyond the static scratch table");
        return LGNK_ERR_INVALID_ARG;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) {
        lgnk_internal_set_error(cudaGetErrorString(e));
        return LGNK_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            lgnk_internal_set_error(cudaGetErrorString(e));
            return LGNK_ERR_CUDA;
        }
        g_scratch_dev[dev] = p;
    } else if (g_scratch_dev[dev] == nullptr) {
        lgnk_internal_set_error("the first allocation-free call on a device must come before any stream capture");
        return LGNK_ERR_INVALID_ARG;
    }
    *out = g_scratch_dev[dev];
    return LGNK_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void scale_sum_kernel(const double* sum, double* out, double scale) {
    out[0] = scale * sum[0];
}

}  // namespace

extern "C" lgnk_status lgnk_forward_transport_static(const lgnk_problem* prob, const float* v, const float* T,
                                                     const float* R, float* u1, double* D, void* stream) {
    if (const char* why = lgnk_internal_validate(prob)) {
        lgnk_internal_set_error(why);
        return LGNK_ERR_INVALID_ARG;
    }
    if (prob->model != LGNK_TRANSPORT) {
        lgnk_internal_set_error("the allocation-free forward supports the transport model only");
        return LGNK_ERR_INVALID_ARG;
    }
    if (v == nullptr || T == nullptr || u1 == nullptr || (R == nullptr) != (D == nullptr)) {
        lgnk_internal_set_error("v, T and u1 must be non-NULL; R and D are given together or not at all");
        return LGNK_ERR_INVALID_ARG;
    }
    const int d = prob->image.d;
    const DevGrid ig = lgnk_internal_grid(prob->image);
    const DevGrid vg = lgnk_internal_grid(prob->velocity);
    const int K = prob->time_nodes;
    int ts[3];
    trace_tile_shape(d, ts);
    int tiles[3], nblocks = 1;
    for (int i = 0; i < 3; ++i) {
        tiles[i] = (ig.m[i] + ts[i] - 1) / ts[i];
        nblocks *= tiles[i];
    }
    SliceTable slices;
    make_slice_table(K, prob->rk4_steps, 1.0, -1.0 / prob->rk4_steps, &slices);
    const size_t vbytes = align256((size_t)vg.mp[0] * vg.mp[1] * vg.mp[2] * slices.n * velocity_pair_bytes(d));
    const size_t tbytes = align256((size_t)ig.mp[0] * ig.mp[1] * ig.mp[2] * sizeof(float));
    const size_t pbytes = align256((size_t)nblocks * sizeof(double));
    const size_t need = vbytes + tbytes + pbytes + 256;
    if (need > LGNK_STATIC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof(msg), "problem needs %zu bytes of scratch; the static maximum is %u bytes", need,
                 (unsigned)LGNK_STATIC_SCRATCH_BYTES);
        lgnk_internal_set_error(msg);
        return LGNK_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    lgnk_status st = scratch_address(s, reinterpret_cast<void**>(&base));
    if (st != LGNK_OK) return st;
    void* Vp = base;
    float* Tp = reinterpret_cast<float*>(base + vbytes);
    double* partial = reinterpret_cast<double*>(base + vbytes + tbytes);
    double* sum = reinterpret_cast<double*>(base + vbytes + tbytes + pbytes);

    // Every scratch byte a launch reads is written earlier in the same call
    // (packing writes pads and interiors, each block writes its partial), so
    // nothing left by a previous call needs clearing.
    cudaError_t e = launch_pack_velocity(d, v, Vp, vg, K, slices, s);
    if (e == cudaSuccess) e = launch_pack_image(T, Tp, ig, d, 1.0f, s);
    TraceArgs a{};
    a.ig = ig;
    a.vg = vg;
    a.K = K;
    a.N = prob->rk4_steps;
    a.dt = (float)(-1.0 / prob->rk4_steps);
    a.t0 = 1.0f;
    double cellvol = 1.0;
    for (int i = 0; i < 3; ++i) {
        a.tiles[i] = tiles[i];
        if (i < d) {
            const double hi = (prob->image.hi[i] - prob->image.lo[i]) / prob->image.m[i];
            const double hv = (prob->velocity.hi[i] - prob->velocity.lo[i]) / prob->velocity.m[i];
            cellvol *= hi;
            a.vxi_a[i] = (prob->image.lo[i] - prob->velocity.lo[i]) / hv - 0.5;
            a.vxi_b[i] = hi / hv;
            a.vxi_af[i] = (float)a.vxi_a[i];
            a.vxi_bf[i] = (float)a.vxi_b[i];
        }
    }
    a.cellvol = (float)cellvol;
    a.slice_nodes = (long long)vg.mp[0] * vg.mp[1] * vg.mp[2];
    a.V = Vp;
    a.Tp = Tp;
    a.R = R;
    a.u1 = u1;
    a.partial = R != nullptr ? partial : nullptr;
    if (e == cudaSuccess) e = launch_trace(d, K > 1, LGNK_TRANSPORT, MODE_FWD, a, nblocks, s);
    if (e == cudaSuccess && R != nullptr) {
        e = launch_reduce(partial, nblocks, sum, s);
        if (e == cudaSuccess) {
            scale_sum_kernel<<<1, 1, 0, s>>>(sum, D, 0.5 * cellvol);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        lgnk_internal_set_error(cudaGetErrorString(e));
        return LGNK_ERR_CUDA;
    }
    return LGNK_OK;
}

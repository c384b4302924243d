// Internal declarations of the lgnk CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lgnk.h"

// Grid data is stored padded by LGNK_PAD zero nodes on each side of every axis.
// A point's lower cell corner is clamped to [-2, m], so both corners of any
// point, however far outside, fall on padded storage; padding holds zeros for
// gathers (zero extension) and swallows scatters that the unpack then drops
// (the adjoint of zero extension: splatted mass that leaves the grid is lost).
#define LGNK_PAD 2
#define LGNK_MAX_STEPS 64
#define LGNK_MAX_SLICES (2 * LGNK_MAX_STEPS + 1)
#define LGNK_BLOCK 256

struct DevGrid {
    int m[3];      // cells per axis (1 for an absent axis)
    int mp[3];     // padded extents m + 2 * LGNK_PAD (1 for an absent axis)
    float lo[3];   // domain lower corner
    float h[3];    // cell widths
    float inv_h[3];
};

enum TraceMode { MODE_FWD = 0, MODE_JVP = 1, MODE_JTVP = 2, MODE_HESS = 3, MODE_OBJGRAD = 4, MODE_ASM = 5 };

// Voxel tile of one 256-thread CTA of the tracing kernels (x, y, z).
inline void trace_tile_shape(int d, int* t) {
    if (d == 3) { t[0] = 8; t[1] = 8; t[2] = 4; }
    else { t[0] = 16; t[1] = 16; t[2] = 1; }
}

// Time slices of a velocity: slice m is the field at stage time t0 + m dt / 2,
// (1 - th[m]) v_j[m] + th[m] v_{j[m]+1} (linear in time between the K nodes);
// a stationary field (K = 1) has the single slice j = 0, th = 0.
struct SliceTable {
    int n;
    int j[LGNK_MAX_SLICES];
    float th[LGNK_MAX_SLICES];
};

// Arguments of one launch of the characteristic-tracing kernel family.
struct TraceArgs {
    DevGrid ig, vg;
    int K, N;
    float dt, t0;
    float cellvol;            // image cell volume h^d (SSD weight)
    int tiles[3];             // voxel tiles per axis (grid = product), set per launch
    // continuous velocity-grid index of the start point of voxel i along axis a:
    // vxi_a[a] + (i + 1/2) * vxi_b[a]  (exact in FP64: (x_c - lo_v) / h_v - 1/2)
    double vxi_a[3], vxi_b[3];
    float vxi_af[3], vxi_bf[3];  // the same in FP32 (per-stage recomputation)
    float pic_rho[3];         // continuity PIC half-width in image cells per axis (0: width = cell)
    long long slice_nodes;    // padded velocity nodes per time slice
    const void* V;            // pair-packed velocity slices [m][zp][yp][xp] x [v(node) | v(node+1)]
    const void* dV;           // pair-packed direction slices (JVP, HESS)
    const float* Tp;          // padded template (gathers)
    const float* T;           // template, ABI layout (continuity particle masses)
    const float* R;           // reference, ABI layout (OBJGRAD, FWD with residual)
    const float* r;           // JTVP seed: transport ABI layout r; continuity padded r
    float* u1;                // transport FWD output (ABI layout)
    float* yout;              // optional end points [d][M]
    float* acc;               // continuity splat accumulator (padded image)
    void* G;                  // gradient accumulator slices [m][zp][yp][xp] of float4 (3D) / float2 (2D)
    double* partial;          // per-block partial sums of res^2 (FP64)
    // MODE_ASM (transport): rows of the assembled J, entry-major [e][voxel]
    long long* ekey;          // element of the lower corner of the entry's cell in the slice gradient space
    float* eblk;              // [e][corner][component][voxel]: sum of w_corner * mu over the cell's stages
    int* ecnt;                // entries per voxel
    int* eflag;               // set to 1 when a row needs more than ewidth entries
    double* cpartial;         // per-block sums of the entries per row (may be NULL)
    int ewidth;               // entries per voxel the arrays hold
};

// Assembled J (transport): at most this many (slice, cell) blocks per row.
inline int asm_capacity(int d) { return d == 3 ? 16 : 32; }

// Products with the assembled J (one thread per voxel).
enum EllMode { ELL_JVP = 0, ELL_JTVP = 1, ELL_HESS = 2 };
struct EllArgs {
    DevGrid vg;               // velocity grid (corner offsets in the padded slices)
    long long M;              // voxels
    const long long* ekey;
    const float* eblk;
    const int* ecnt;
    const void* dV;           // pair-packed direction slices (JVP, HESS)
    void* G;                  // slice gradient accumulator (JTVP, HESS)
    const float* r;           // JTVP weights per voxel (ABI image layout)
    float* out;               // JVP output (ABI image layout)
    float cellvol;            // HESS weight h^d
};
cudaError_t launch_ell(int d, int mode, const EllArgs& a, cudaStream_t s);

// trace kernels (trace2d.cu / trace3d.cu)
cudaError_t launch_trace(int d, bool nonstat, int model, int mode, const TraceArgs& a, int nblocks,
                         cudaStream_t s);

// grid utilities (grid_ops.cu)
// ABI velocity [K][d][z][y][x] -> pair-packed padded time slices
// (velocity_pair_bytes(d) bytes per node and slice)
// (and, when Gz is given, zero the slice gradients of the same slices and padding)
cudaError_t launch_pack_velocity(int d, const float* v, void* Vp, const DevGrid& g, int K, const SliceTable& t,
                                 cudaStream_t s, void* Gz = nullptr);
inline size_t velocity_pair_bytes(int d) { return d == 3 ? 32 : 16; }
// slice gradients [m][padded nodes] -> ABI [K][d][z][y][x], out = scale * sum_m w_j(m) G_m
cudaError_t launch_distribute_gradient(int d, const void* Gp, float* out, const DevGrid& g, int K,
                                       const SliceTable& t, float scale, cudaStream_t s);
// stage-time slices of a trace with N steps from t0 in steps dt, over K time nodes
void make_slice_table(int K, int N, double t0, double dt, SliceTable* t);
cudaError_t launch_pack_image(const float* T, float* Tp, const DevGrid& g, int d, float scale, cudaStream_t s);
cudaError_t launch_unpack_image(const float* acc, float* out, const DevGrid& g, int d, cudaStream_t s);
cudaError_t launch_repad_image(float* acc, const DevGrid& g, int d, float scale, cudaStream_t s);
cudaError_t launch_residual(const float* u1, const float* R, float* rp, const DevGrid& g, int d,
                            float scale, double* partial, int nblocks, cudaStream_t s);
int residual_blocks(const DevGrid& g, int d);
// blocks of the grid-stride reductions (4 per SM of the current device)
int reduce_block_cap();
cudaError_t launch_reduce(const double* partial, int count, double* out, cudaStream_t s);
cudaError_t launch_dot(const float* a, const float* b, size_t count, double* partial, int nblocks,
                       cudaStream_t s);
int dot_blocks(size_t count);
// a.b (and a.c) reduced to sc[slot_b] (sc[slot_c]) in one launch, then the PCG
// step `mode` (-1 none, 0 alpha, 1 beta); counter: a zeroed device word
cudaError_t launch_dot_fused(const float* a, const float* b, const float* c, size_t count, double* partial,
                             int nblocks, unsigned* counter, double* sc, int slot_b, int slot_c, int mode, float* f,
                             cudaStream_t s);
// Hp = gscale * distributed slice gradients + rscale * B^T B p + gamma * p (diffusion
// regularizer), then p.Hp into sc[2] and alpha (fused inner-product step, mode 0)
cudaError_t launch_hess_finish(int d, const void* Gp, const float* p, float* Hp, const DevGrid& g, int K,
                               const SliceTable& t, float gscale, float rscale, float gamma, double* partial,
                               int nblocks, unsigned* counter, double* sc, float* f, cudaStream_t s);
// x += f[0] p, r += f[1] Hp
cudaError_t launch_pcg_update_xr(float* x, const float* p, float* r, const float* Hp, const float* f, size_t count,
                                 cudaStream_t s);
// PCG loop test at the end of an iteration of a device-side while loop (see grid_ops.cu)
cudaError_t launch_pcg_control(const double* sc, int* ctl, cudaGraphConditionalHandle handle, cudaStream_t s);
// x = z when the device-side PCG loop's first iteration met non-positive curvature (ctl as above)
cudaError_t launch_pcg_curvature_fix(float* x, const float* z, const int* ctl, size_t count, cudaStream_t s);
cudaError_t launch_axpby_dev(float a, const float* ap, const float* x, float b, const float* bp, float* y,
                             size_t count, cudaStream_t s);
// out = addsrc + scale * A x + gamma * x for the Neumann Laplacian A = B^T B of each
// (time node, component) block; addsrc may be NULL or equal to out.
cudaError_t launch_laplacian(int d, const float* x, float* out, const DevGrid& g, int blocks_kd,
                             float scale, float gamma, const float* addsrc, cudaStream_t s);
// as above with the gamma term taken from gsrc instead of x
cudaError_t launch_laplacian_ext(int d, const float* x, float* out, const DevGrid& g, int blocks_kd,
                                 float scale, float gamma, const float* gsrc, const float* addsrc,
                                 cudaStream_t s);
cudaError_t launch_divergence(int d, const float* x, float* div, const DevGrid& g, int K, cudaStream_t s);
// out_c = addsrc + smu * A x_c + slm * D_c^T div + gamma * x_c (elastic operator)
cudaError_t launch_elastic(int d, const float* x, const float* div, float* out, const DevGrid& g, int K,
                           float smu, float slm, float gamma, const float* addsrc, cudaStream_t s);
// one axis of the spectral transform: C the m x m matrix (untiled kernel,
// axes of more than 128 cells), Cp its padded table of the direction (Cf
// forward, Ci inverse; tiled kernel)
cudaError_t launch_dct_axis(const float* in, float* out, const float* C, const float* Cp, const DevGrid& g, int d,
                            int nblocks_kd, int axis, bool inverse, cudaStream_t s);
// Padded DCT tables per axis (rows of P = m rounded up to 4 floats, zero past
// m): forward Cf[q][k] = C[k][q], inverse Ci[q][k] = C[q][k].
// The y and x axes of the spectral transform on whole xy planes (3D, both
// axes at most 64 cells) with the tables of one direction (Cf or Ci of the x
// and y axes): planes = blocks x z-planes.  cudaErrorNotSupported for larger
// planes (the per-axis kernels cover them).
cudaError_t launch_dct_plane(const float* in, float* out, const float* Ax, const float* Ay, const DevGrid& g,
                             long long planes, cudaStream_t s);
// The whole 2D preconditioner (forward transform, inv_eig, inverse) with one CTA
// per (time node, component) plane of at most 64 x 64 cells.
cudaError_t launch_dct_plane2d(const float* in, float* out, const float* Cfx, const float* Cfy, const float* Cix,
                               const float* Ciy, const float* inv_eig, const DevGrid& g, int blocks, cudaStream_t s);
// forward DCT, scale by inv_eig and inverse DCT along the last axis in one pass
// (the axis's Cf and Ci); cudaErrorNotSupported when that axis has more than 128 cells
cudaError_t launch_dct_last_fused(const float* in, float* out, const float* Cf, const float* Ci, const float* inv_eig,
                                  const DevGrid& g, int d, int nblocks_kd, cudaStream_t s);
cudaError_t launch_scale_modes(float* x, const float* inv_eig, size_t block_elems, size_t count,
                               cudaStream_t s);
// y = a * x + b * y  (count floats)
cudaError_t launch_axpby(float a, const float* x, float b, float* y, size_t count, cudaStream_t s);
cudaError_t launch_add_scaled(float* out, const float* x, float ax, const float* y, float ay, size_t count,
                              cudaStream_t s);

// multilevel: 2^d-cell averaging onto the coarse grid cg; multilinear
// prolongation of `blocks` scalar fields from grid cg to grid fg
cudaError_t launch_restrict_image(int d, const float* F, float* C, const DevGrid& cg, cudaStream_t s);
cudaError_t launch_prolong_velocity(int d, const float* vc, float* vf, const DevGrid& cg, const DevGrid& fg,
                                    int blocks, cudaStream_t s);

// det grad y of end points y [d][M] (det may be NULL); min, max -> out[0], out[1];
// partial needs 2 * residual_blocks(g, d) doubles
cudaError_t launch_jacobian_det(int d, const float* y, float* det, const DevGrid& g, double* partial, double* out,
                                cudaStream_t s);

// api.cu helpers for entry points that run without a context
const char* lgnk_internal_validate(const lgnk_problem* p);  // NULL if valid, else why not
DevGrid lgnk_internal_grid(const lgnk_grid& g);
void lgnk_internal_set_error(const char* msg);             // read back by lgnk_last_error(NULL)

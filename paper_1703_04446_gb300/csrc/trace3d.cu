// 3D instantiations of the characteristic-tracing kernel family.
#include "trace_impl.cuh"

cudaError_t launch_trace_3d(bool nonstat, int model, int mode, const TraceArgs& a, int nblocks, cudaStream_t s) {
    return nonstat ? lgnk::launch_dim<3, true>(model, mode, a, nblocks, s)
                   : lgnk::launch_dim<3, false>(model, mode, a, nblocks, s);
}

cudaError_t launch_ell_3d(int mode, const EllArgs& a, cudaStream_t s) { return lgnk::launch_ell_dim<3>(mode, a, s); }

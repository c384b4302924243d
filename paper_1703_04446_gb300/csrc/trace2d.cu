// 2D instantiations of the characteristic-tracing kernel family.
#include "trace_impl.cuh"

cudaError_t launch_trace_2d(bool nonstat, int model, int mode, const TraceArgs& a, int nblocks, cudaStream_t s) {
    return nonstat ? lgnk::launch_dim<2, true>(model, mode, a, nblocks, s)
                   : lgnk::launch_dim<2, false>(model, mode, a, nblocks, s);
}

cudaError_t launch_ell_2d(int mode, const EllArgs& a, cudaStream_t s) { return lgnk::launch_ell_dim<2>(mode, a, s); }

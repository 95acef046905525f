// Kernel instantiations of the persistent ragged-batch execute (separate translation unit so
// the dense and ragged kernels compile in parallel).
#include "tdh_exec.cuh"

namespace tdh {

int dispatch_ragged(const Geometry& g, const ExecParams<float>& P, int64_t batch, cudaStream_t s) {
    return dispatch_geom<float, true>(g, P, batch, s);
}
int dispatch_ragged(const Geometry& g, const ExecParams<double>& P, int64_t batch, cudaStream_t s) {
    return dispatch_geom<double, true>(g, P, batch, s);
}

}  // namespace tdh

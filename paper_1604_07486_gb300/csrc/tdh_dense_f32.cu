// Kernel instantiations of the dense execute, float (one translation unit per kind and
// precision so that they compile in parallel).
#include "tdh_exec.cuh"

namespace tdh {

int dispatch_dense(const Geometry& g, const ExecParams<float>& P, int64_t batch, cudaStream_t s) {
    return dispatch_geom<float, false>(g, P, batch, s);
}

}  // namespace tdh

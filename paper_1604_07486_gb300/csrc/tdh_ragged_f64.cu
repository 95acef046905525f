// Kernel instantiations of the ragged execute, double (one translation unit per kind and
// precision so that they compile in parallel).
#include "tdh_exec.cuh"

namespace tdh {

int dispatch_ragged(const Geometry& g, const ExecParams<double>& P, int64_t batch, cudaStream_t s) {
    return dispatch_geom<double, true>(g, P, batch, s);
}

}  // namespace tdh

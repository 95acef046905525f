// Kernel instantiations of the dense execute with split-bfloat16 tensor-core DFT passes (one
// translation unit per kind so that they compile in parallel).
#include "tdh_exec.cuh"

namespace tdh {

int dispatch_dense_tc(const Geometry& g, const ExecParams<float>& P, int64_t batch,
                      cudaStream_t s) {
    return dispatch_geom_tc<false>(g, P, batch, s);
}

}  // namespace tdh

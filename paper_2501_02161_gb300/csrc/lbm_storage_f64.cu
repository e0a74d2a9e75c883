// lbm_storage_f64.cu -- the kernels of one storage type (FP64),
// instantiated in a translation unit of their own.
#include "lbm_dispatch.cuh"

namespace lbm {

template <>
cudaError_t flow_launch_storage<0>(int stencil, FlowOp op, const FlowLaunch& a, const Geom& g, cudaStream_t s) {
    if (stencil == 0) {
        dispatch::flow_dispatch<D2Q9, 0>(op, a, g, s);
    } else {
        dispatch::flow_dispatch<D3Q19, 0>(op, a, g, s);
    }
    return cudaGetLastError();
}

template <>
cudaError_t therm_launch_storage<0>(ThermOp op, const ThermLaunch& a, const Geom& g, cudaStream_t s) {
    dispatch::therm_dispatch<0>(op, a, g, s);
    return cudaGetLastError();
}

}  // namespace lbm

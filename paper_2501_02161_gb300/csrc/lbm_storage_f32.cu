// lbm_storage_f32.cu -- the kernels of one storage type (FP32),
// instantiated in a translation unit of their own.
#include "lbm_dispatch.cuh"

namespace lbm {

template <>
cudaError_t flow_launch_storage<1>(int stencil, FlowOp op, const FlowLaunch& a, const Geom& g, cudaStream_t s) {
    if (stencil == 0) {
        dispatch::flow_dispatch<D2Q9, 1>(op, a, g, s);
    } else {
        dispatch::flow_dispatch<D3Q19, 1>(op, a, g, s);
    }
    return cudaGetLastError();
}

template <>
cudaError_t therm_launch_storage<1>(ThermOp op, const ThermLaunch& a, const Geom& g, cudaStream_t s) {
    dispatch::therm_dispatch<1>(op, a, g, s);
    return cudaGetLastError();
}

}  // namespace lbm

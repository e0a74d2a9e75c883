// lbm_storage_f16.cu -- the kernels of one storage type (FP16 offset populations),
// instantiated in a translation unit of their own.
#include "lbm_dispatch.cuh"

namespace lbm {

template <>
cudaError_t flow_launch_storage<2>(int stencil, FlowOp op, const FlowLaunch& a, const Geom& g, cudaStream_t s) {
    if (stencil == 0) return cudaErrorInvalidValue;
    dispatch::flow_dispatch<D3Q19, 2>(op, a, g, s);
    return cudaGetLastError();
}

template <>
cudaError_t therm_launch_storage<2>(ThermOp op, const ThermLaunch& a, const Geom& g, cudaStream_t s) {
    dispatch::therm_dispatch<2>(op, a, g, s);
    return cudaGetLastError();
}

}  // namespace lbm

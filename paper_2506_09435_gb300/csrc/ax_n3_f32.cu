// Instantiations of the FP32 operator kernels for GLL order p = 2.
#include "ax_impl.cuh"

namespace fnpf {
template cudaError_t launch_ax_n<float, 3>(const Geom&, const Tables<float>&, const AxPtrs<float>&, int, int,
                                           cudaStream_t);
}  // namespace fnpf

// Instantiations of the FP64 operator kernels for GLL order p = 3.
#include "ax_impl.cuh"

namespace fnpf {
template cudaError_t launch_ax_n<double, 4>(const Geom&, const Tables<double>&, const AxPtrs<double>&, int, int,
                                            cudaStream_t);
}  // namespace fnpf

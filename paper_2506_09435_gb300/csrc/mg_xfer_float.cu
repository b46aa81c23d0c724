// Instantiations of the p-multigrid transfer kernels for the order pairs of the
// level schedules (halving, two-level, steps of two) (float).
#include "mg_impl.cuh"

namespace fnpf {

cudaError_t launch_transfer_float(const Geom& gf, const Geom& gc, const float* J, const float* in, float* out, float* ring,
                                 int mode, const int* skip, cudaStream_t s) {
  const int key = gf.n * 16 + gc.n;
  switch (key) {
    case 9 * 16 + 5: return launch_transfer_t<float, 9, 5>(gf, gc, J, in, out, ring, mode, skip, s);
    case 8 * 16 + 4: return launch_transfer_t<float, 8, 4>(gf, gc, J, in, out, ring, mode, skip, s);
    case 7 * 16 + 4: return launch_transfer_t<float, 7, 4>(gf, gc, J, in, out, ring, mode, skip, s);
    case 6 * 16 + 3: return launch_transfer_t<float, 6, 3>(gf, gc, J, in, out, ring, mode, skip, s);
    case 5 * 16 + 3: return launch_transfer_t<float, 5, 3>(gf, gc, J, in, out, ring, mode, skip, s);
    case 4 * 16 + 2: return launch_transfer_t<float, 4, 2>(gf, gc, J, in, out, ring, mode, skip, s);
    case 3 * 16 + 2: return launch_transfer_t<float, 3, 2>(gf, gc, J, in, out, ring, mode, skip, s);
    case 9 * 16 + 7: return launch_transfer_t<float, 9, 7>(gf, gc, J, in, out, ring, mode, skip, s);
    case 8 * 16 + 6: return launch_transfer_t<float, 8, 6>(gf, gc, J, in, out, ring, mode, skip, s);
    case 7 * 16 + 5: return launch_transfer_t<float, 7, 5>(gf, gc, J, in, out, ring, mode, skip, s);
    case 6 * 16 + 4: return launch_transfer_t<float, 6, 4>(gf, gc, J, in, out, ring, mode, skip, s);
    case 9 * 16 + 2: return launch_transfer_t<float, 9, 2>(gf, gc, J, in, out, ring, mode, skip, s);
    case 8 * 16 + 2: return launch_transfer_t<float, 8, 2>(gf, gc, J, in, out, ring, mode, skip, s);
    case 7 * 16 + 2: return launch_transfer_t<float, 7, 2>(gf, gc, J, in, out, ring, mode, skip, s);
    case 6 * 16 + 2: return launch_transfer_t<float, 6, 2>(gf, gc, J, in, out, ring, mode, skip, s);
    case 5 * 16 + 2: return launch_transfer_t<float, 5, 2>(gf, gc, J, in, out, ring, mode, skip, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fnpf

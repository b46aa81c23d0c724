// Instantiations of the geometric vector-Jacobian product (FP64, every order).
#include "adj_impl.cuh"

namespace fnpf {

cudaError_t launch_geom_vjp(const Geom& g, const Tables<double>& t, const double* eta, const double* psiI,
                            const double* phiI, const double* phiS, double* out, cudaStream_t s) {
#define FNPF_GV(N)                                                                          \
  case N:                                                                                   \
    return g.dim == 3 ? launch_geom_vjp_t<double, N, 3>(g, t, eta, psiI, phiI, phiS, out, s) \
                      : launch_geom_vjp_t<double, N, 2>(g, t, eta, psiI, phiI, phiS, out, s);
  switch (g.n) {
    FNPF_GV(2)
    FNPF_GV(3)
    FNPF_GV(4)
    FNPF_GV(5)
    FNPF_GV(6)
    FNPF_GV(7)
    FNPF_GV(8)
    FNPF_GV(9)
    default: return cudaErrorInvalidValue;
  }
#undef FNPF_GV
}

}  // namespace fnpf

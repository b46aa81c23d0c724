// Arithmetic peak probe (measurement utility, not part of the method): a
// kernel of independent FMA chains whose only cost is the FMA pipe, timed by
// the caller.  It gives the measured FP64 / FP32 FMA throughput that the
// operator kernels' ALU roofline is compared with.
#include "fnpf_internal.cuh"

namespace {

constexpr int kChains = 8;     // independent dependency chains per thread
constexpr int kUnroll = 16;    // FMAs per chain per loop trip

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T a, T b, int iters, T* out) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x) * T(1e-3) + T(k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == T(-1.0)) out[0] = s;   // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" fnpf_status fnpf_fma_probe(int precision, int blocks, int iters, void* out, double* flops,
                                      void* stream) {
  if (blocks < 1 || iters < 1 || !out || (precision != FNPF_FP64 && precision != FNPF_MIXED)) return FNPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == FNPF_FP64)
    fma_peak_kernel<double><<<blocks, 256, 0, s>>>(1.0 - 1e-12, 1e-12, iters, (double*)out);
  else
    fma_peak_kernel<float><<<blocks, 256, 0, s>>>(1.0f - 1e-6f, 1e-6f, iters, (float*)out);
  if (flops) *flops = 2.0 * blocks * 256.0 * iters * kUnroll * kChains;
  return cudaGetLastError() == cudaSuccess ? FNPF_OK : FNPF_ECUDA;
}

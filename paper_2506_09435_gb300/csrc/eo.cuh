// Even-odd form of the one-dimensional GLL derivative contractions (used by
// the operator kernels): the derivative matrix is centro-antisymmetric,
// D_{n-1-a, n-1-b} = -D_{a,b} (and so is D^T), so with e_m = x_m + x_{n-1-m},
// o_m = x_m - x_{n-1-m} (m < h = n/2),
//     y_i = P_i + Q_i,  y_{n-1-i} = P_i - Q_i,
//     P_i = sum_m 1/2 (D_im - D_i,n-1-m) o_m,
//     Q_i = sum_m 1/2 (D_im + D_i,n-1-m) e_m (+ D_i,h x_h for odd n),
//     y_h = sum_m D_hm o_m (odd n)
// (e.g. Kopriva, Implementing Spectral Methods for PDEs, 2009, Sec. 3.5):
// 2h^2 + 6h operations for odd n (36 instead of 49 at n = 7), 2h^2 + 4h for
// even n.  The half matrices sit in __constant__ memory, so with the loops
// unrolled every coefficient is an immediate constant-bank operand.
#pragma once

#include <atomic>
#include <mutex>

#include "fnpf_internal.cuh"

namespace fnpf {

// Even-odd half matrices of D and D^T: [O h*h | E h*h | mid column h | mid row h].
template <int N>
struct EO {
  static constexpr int H = N / 2;
  static constexpr int O = 0, E = H * H, MC = 2 * H * H, MR = 2 * H * H + H;
  static constexpr int SIZE = 2 * H * H + 2 * H;
};
constexpr int kEOMax = 2 * (kMaxN / 2) * (kMaxN / 2) + 2 * (kMaxN / 2);

// One copy per translation unit (no relocatable device code): each ax_n<N>_*.cu
// fills its own through eo_upload, before its first line-kernel launch.
static __constant__ double c_eo64[kMaxN + 1][2][kEOMax];
static __constant__ float c_eo32[kMaxN + 1][2][kEOMax];
static std::atomic<uint64_t> g_eo_ready{0};   // devices whose copy is filled
static std::mutex g_eo_mu;

template <typename T, int N>
__device__ __forceinline__ T eo_coef(int tr, int k) {
  if constexpr (sizeof(T) == 8) return c_eo64[N][tr][k];
  else return c_eo32[N][tr][k];
}

// Host: the half matrices of every order from the GLL tables (computed in
// double, rounded for the FP32 copy), copied to this TU's constant memory on
// the current device, once per device.  Synchronous (not inside a capture).
static cudaError_t eo_upload() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? uint64_t(1) << dev : 0;
  if (bit && (g_eo_ready.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(g_eo_mu);
  if (bit && (g_eo_ready.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  static double h64[kMaxN + 1][2][kEOMax];
  static float h32[kMaxN + 1][2][kEOMax];
  for (int n = 2; n <= kMaxN; ++n) {
    double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
    gll_tables(n - 1, xi, w, D);
    const int H = n / 2;
    for (int tr = 0; tr < 2; ++tr) {
      auto d = [&](int i, int m) { return tr ? D[m * n + i] : D[i * n + m]; };
      double* o = h64[n][tr];
      for (int i = 0; i < H; ++i)
        for (int m = 0; m < H; ++m) {
          o[i * H + m] = 0.5 * (d(i, m) - d(i, n - 1 - m));
          o[H * H + i * H + m] = 0.5 * (d(i, m) + d(i, n - 1 - m));
        }
      for (int i = 0; i < H; ++i) {
        o[2 * H * H + i] = (n & 1) ? d(i, H) : 0.0;
        o[2 * H * H + H + i] = (n & 1) ? d(H, i) : 0.0;
      }
      for (int k = 0; k < kEOMax; ++k) h32[n][tr][k] = (float)h64[n][tr][k];
    }
  }
  if ((e = cudaMemcpyToSymbol(c_eo64, h64, sizeof(h64))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_eo32, h32, sizeof(h32))) != cudaSuccess) return e;
  if (bit) g_eo_ready.fetch_or(bit, std::memory_order_acq_rel);
  return cudaSuccess;
}

// y = D x (TR = 0) or y = D^T x (TR = 1) on one GLL line, even-odd form.
template <typename T, int N, int TR>
__device__ __forceinline__ void eo_mul(const T (&x)[N], T (&y)[N]) {
  constexpr int H = N / 2;
  using Q = EO<N>;
  T e[H > 0 ? H : 1], o[H > 0 ? H : 1];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    e[m] = x[m] + x[N - 1 - m];
    o[m] = x[m] - x[N - 1 - m];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T p = 0, q = 0;
#pragma unroll
    for (int m = 0; m < H; ++m) {
      p += eo_coef<T, N>(TR, Q::O + i * H + m) * o[m];
      q += eo_coef<T, N>(TR, Q::E + i * H + m) * e[m];
    }
    if constexpr (N & 1) q += eo_coef<T, N>(TR, Q::MC + i) * x[H];
    y[i] = p + q;
    y[N - 1 - i] = p - q;
  }
  if constexpr (N & 1) {
    T s = 0;
#pragma unroll
    for (int m = 0; m < H; ++m) s += eo_coef<T, N>(TR, Q::MR + m) * o[m];
    y[H] = s;
  }
}

}  // namespace fnpf

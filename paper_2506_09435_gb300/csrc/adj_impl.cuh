// Geometric vector-Jacobian product of the Laplace operator (adjoint of the
// eta- and h-dependence of A(eta, h) in Eq. Laplace_weak with the mesh motion
// of Sec. 3.1.2): for given psi and phi, the derivatives of
//     E = psi^T A(eta, h) phi = sum_e sum_q (grad_r psi)^T G_q (grad_r phi)
// with respect to the per-line metric parameters of every element column
//     A = z_t = (eta + h) / (2 Nz),  z_r = P_r + sigma Q_r,  z_s = P_s + sigma Q_s,
//     P_r = -h_r, Q_r = eta_r + h_r (and likewise in s),
// summed over the line's points in all layers.  With u = grad_r psi,
// v = grad_r phi, W0 = w_k cw and a = z_r grad r + z_s grad s:
//   dE/dA   = W0 [ |grad r|^2 u_r v_r + grad r.grad s (u_r v_s + u_s v_r) + |grad s|^2 u_s v_s
//                  - (|a|^2 + 1) / A^2 u_t v_t ]
//   dE/da   = W0 [ -grad r (u_r v_t + u_t v_r) - grad s (u_s v_t + u_t v_s) + 2 a / A u_t v_t ]
//   dE/dz_r = grad r . dE/da,  dE/dz_s = grad s . dE/da,
//   dE/dP = dE/dz,  dE/dQ = sigma dE/dz.
// The per-line sums are stored element-locally and turned into nodal
// derivatives by adj_geom_gather (D^T along the element rows).
#pragma once

#include "ax_impl.cuh"

namespace fnpf {

// out[5][n_ecol * L]: (dE/dA, dE/dQ_r, dE/dQ_s, dE/dP_r, dE/dP_s) per line.
template <typename T, int N, int DIM, int C>
__global__ void __launch_bounds__(AxShape<T, N, DIM, C>::THREADS)
    geom_vjp_kernel(Geom g, Tables<T> t, const T* eta, const T* psiI, const T* phiI, const T* phiS, T* out) {
  using S = AxShape<T, N, DIM, C>;
  constexpr int P = N - 1, L = S::L;
  extern __shared__ __align__(16) unsigned char ax_smem[];
  T* sU = reinterpret_cast<T*>(ax_smem);
  T* sV = sU + S::BUF;
  T* sD = sV + 2 * S::BUF;
  T* sXi = sD + N * N;
  T* sW = sXi + N;
  T* sE = sW + N;
  T* sH = sE + C * L;
  const int c = threadIdx.x / L, line = threadIdx.x - c * L;
  const int i = line % N, j = line / N;
  const int ecol = blockIdx.x * C + c;
  const bool active = ecol < g.n_ecol;
  int col;
  LineGeom<T> lg;
  ax_prologue<T, N, DIM, C>(g, t, eta, sD, sXi, sW, sE, sH, c, line, i, j, ecol, active, col, lg);
  const T inv_nz = T(1) / T(g.nz);
  const T r2 = lg.rx * lg.rx + lg.ry * lg.ry, rs = lg.rx * lg.sx + lg.ry * lg.sy, s2 = lg.sx * lg.sx + lg.sy * lg.sy;
  T bA = 0, bQr = 0, bQs = 0, bPr = 0, bPs = 0;
  for (int l = 0; l < g.nz; ++l) {
    T u[N], v[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int plane = l * P + k;
      T a = 0, b = 0;
      if (active) {
        if (plane < g.nv - 1) {
          a = psiI[(int64_t)plane * g.ns + col];
          b = phiI[(int64_t)plane * g.ns + col];
        } else {
          b = phiS[col];
        }
      }
      u[k] = a;
      v[k] = b;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
      sU[(c * N + k) * L + line] = u[k];
      sV[(c * N + k) * L + line] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const T* uk = sU + (c * N + k) * L;
      const T* vk = sV + (c * N + k) * L;
      T ur = 0, us = 0, ut = 0, vr = 0, vs = 0, vt = 0;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        ur += sD[i * N + m] * uk[j * N + m];
        vr += sD[i * N + m] * vk[j * N + m];
        ut += sD[k * N + m] * u[m];
        vt += sD[k * N + m] * v[m];
      }
      if (DIM == 3) {
#pragma unroll
        for (int m = 0; m < N; ++m) {
          us += sD[j * N + m] * uk[m * N + i];
          vs += sD[j * N + m] * vk[m * N + i];
        }
      }
      const T sigma = (T(l) + T(0.5) * (T(1) + sXi[k])) * inv_nz;
      const T W0 = sW[k] * lg.cw;
      const T zr = lg.Pr + sigma * lg.Qr, zs = lg.Ps + sigma * lg.Qs;
      const T ax = zr * lg.rx + zs * lg.sx, ay = zr * lg.ry + zs * lg.sy;
      const T uv_rr = ur * vr, uv_rs = ur * vs + us * vr, uv_ss = us * vs;
      const T uv_rt = ur * vt + ut * vr, uv_st = us * vt + ut * vs, uv_tt = ut * vt;
      const T a2p1 = ax * ax + ay * ay + T(1);
      bA += W0 * (r2 * uv_rr + rs * uv_rs + s2 * uv_ss - a2p1 * lg.Ainv * lg.Ainv * uv_tt);
      const T dax = W0 * (-lg.rx * uv_rt - lg.sx * uv_st + T(2) * ax * lg.Ainv * uv_tt);
      const T day = W0 * (-lg.ry * uv_rt - lg.sy * uv_st + T(2) * ay * lg.Ainv * uv_tt);
      const T dzr = lg.rx * dax + lg.ry * day, dzs = lg.sx * dax + lg.sy * day;
      bPr += dzr;
      bQr += sigma * dzr;
      bPs += dzs;
      bQs += sigma * dzs;
    }
  }
  if (active) {
    const int64_t hs = (int64_t)g.n_ecol * L, idx = (int64_t)ecol * L + line;
    out[idx] = bA;
    out[hs + idx] = bQr;
    out[2 * hs + idx] = bQs;
    out[3 * hs + idx] = bPr;
    out[4 * hs + idx] = bPs;
  }
}

template <typename T, int N, int DIM>
cudaError_t launch_geom_vjp_t(const Geom& g, const Tables<T>& t, const T* eta, const T* psiI, const T* phiI,
                              const T* phiS, T* out, cudaStream_t s) {
  constexpr int C = DIM == 3 ? CtaChoices<N>::c[1] : (128 + N - 1) / N;
  using S = AxShape<T, N, DIM, C>;
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = set_smem_attr<T, N, DIM, C>(geom_vjp_kernel<T, N, DIM, C>, &attr);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((g.n_ecol + C - 1) / C);
  geom_vjp_kernel<T, N, DIM, C><<<blocks, S::THREADS, S::SMEM, s>>>(g, t, eta, psiI, phiI, phiS, out);
  return cudaGetLastError();
}

}  // namespace fnpf

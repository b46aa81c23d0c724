// Line-decomposed form of the matrix-free operator of the weak Laplace form
// (arXiv 2506.09435, Sec. 3.1.1, Eq. Laplace_weak; geometry of Sec. 3.1.2)
// for 3D meshes:  y = sum_e P_e^T Dhat^T G_e Dhat P_e x, the same operator as
// ax_kernel / axg_kernel, with a different work decomposition.
//
// Every one-dimensional contraction is done by a thread that owns a whole
// GLL line in the contraction's own direction, so a field value loaded from
// shared memory feeds a full line of outputs (register blocking), and the
// contraction uses the centro-antisymmetry of the GLL derivative matrix,
// D_{n-1-a, n-1-b} = -D_{a,b} (the "even-odd" decomposition, e.g. Kopriva,
// Implementing Spectral Methods for PDEs, 2009, Sec. 3.5): with
// e_m = x_m + x_{n-1-m}, o_m = x_m - x_{n-1-m} (m < n/2),
//     y_i = P_i + Q_i,  y_{n-1-i} = P_i - Q_i,
//     P_i = sum_m 1/2 (D_im - D_i,n-1-m) o_m,
//     Q_i = sum_m 1/2 (D_im + D_i,n-1-m) e_m (+ D_i,h x_h for odd n, h = n/2),
//     y_h = sum_m D_hm o_m (odd n),
// which costs 2h^2 + 6h operations for odd n (36 instead of 49 at n = 7) and
// 2h^2 + 4h for even n.  D^T has the same symmetry.  The half matrices sit in
// __constant__ memory, so with the loops unrolled every coefficient is an
// immediate constant-bank operand of its FMA.
//
// Per element layer, C element columns per CTA, n^2 threads per column, three
// roles of the same thread (a, b) = (line % n, line / n):
//   V (vertical line (i, j) = (a, b)): loads u into shared memory;
//   R (r-line (j, k) = (a, b)) and S (s-line (i, k) = (a, b)): r- and
//   s-contractions;
// then the t-contraction and metric product (V), the transposed r/s
// contractions (R, S) and the transposed t-contraction plus the sum (V).  Four shared buffers per column,
// four barriers per layer.  The vertical assembly between stacked elements
// and the horizontal ring assembly are those of ax_kernel.
#pragma once

#include "eo.cuh"

namespace fnpf {

template <typename T, int N, int C>
struct AxlShape {
  static constexpr int L = N * N;
  static constexpr int SJ = N + ((N % 2 == 0) ? 1 : 0);   // odd row stride: conflict-free r-lines
  static constexpr int SK = N * SJ;
  static constexpr int COL = N * SK;                      // one field of one element column
  static constexpr int THREADS = C * L;
  static constexpr size_t SMEM = sizeof(T) * (4 * (size_t)C * COL + N * N + 2 * N + 2 * C * L);
};

template <typename T, int N, int C, bool STORED>
struct axl_kernel {
  static constexpr int kThreads = AxlShape<T, N, C>::THREADS;
  __device__ static void run(Blk bk, Geom g, Tables<T> t, AxPtrs<T> a) {
    using S = AxlShape<T, N, C>;
    constexpr int P = N - 1, L = S::L, SJ = S::SJ, SK = S::SK, COL = S::COL;
    extern __shared__ __align__(16) unsigned char ax_smem[];
    T* buf = reinterpret_cast<T*>(ax_smem);
    T* sD = buf + 4 * C * COL;
    T* sXi = sD + N * N;
    T* sW = sXi + N;
    T* sE = sW + N;
    T* sH = sE + C * L;
    if (a.skip && *a.skip) return;
    const int c = threadIdx.x / L, line = threadIdx.x - c * L;
    const int qa = line % N, qb = line / N;
    const int ecol = bk.x * C + c;
    const bool active = ecol < g.n_ecol;
    T* f0 = buf + c * COL;              // u, then the metric product R
    T* f1 = buf + (C + c) * COL;        // u_r, then D_r^T R
    T* f2 = buf + (2 * C + c) * COL;    // u_s, then D_s^T S
    T* f3 = buf + (3 * C + c) * COL;    // the metric product S
    const int vo = qb * SJ + qa;        // V role (i, j) = (qa, qb): + k * SK
    const int ro = qb * SK + qa * SJ;   // R role (j, k) = (qa, qb): + i
    const int so = qb * SK + qa;        // S role (i, k) = (qa, qb): + j * SJ
    int col = 0;
    LineGeom<T> lg{};
    if constexpr (STORED) {
      if (active) col = node_col(g, ecol % g.nx, ecol / g.nx, qa, qb);
    } else {
      ax_prologue<T, N, 3, C>(g, t, a.eta, sD, sXi, sW, sE, sH, c, line, qa, qb, ecol, active, col, lg);
    }
    const int slot = ring_slot(3, P, qa, qb);
    const T inv_nz = T(1) / T(g.nz);
    const int64_t PT = (int64_t)g.nz * g.n_ecol * N * L;
    T carry = 0;
    for (int l = 0; l < g.nz; ++l) {
      // ---- V: load the line into shared memory
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const int plane = l * P + k;
        T v = 0;
        if (active) {
          if (plane < g.nv - 1) {
            if (a.xI) v = a.xI[(int64_t)plane * g.ns + col];
          } else if (a.xs) {
            v = a.xs[col];
          }
        }
        f0[k * SK + vo] = v;
      }
      __syncthreads();
      // ---- R and S: r- and s-contractions of u
      {
        T v[N], r[N];
  #pragma unroll
        for (int i = 0; i < N; ++i) v[i] = f0[ro + i];
        eo_mul<T, N, 0>(v, r);
  #pragma unroll
        for (int i = 0; i < N; ++i) f1[ro + i] = r[i];
  #pragma unroll
        for (int j = 0; j < N; ++j) v[j] = f0[so + j * SJ];
        eo_mul<T, N, 0>(v, r);
  #pragma unroll
        for (int j = 0; j < N; ++j) f2[so + j * SJ] = r[j];
      }
      __syncthreads();
      // ---- V: t-contraction of the thread's own line (re-read: fewer live
      //      registers across the barriers), metric product (R, S to shared
      //      memory, T in registers)
      T tt[N], ut[N];
      {
        T u[N];
  #pragma unroll
        for (int k = 0; k < N; ++k) u[k] = f0[k * SK + vo];
        eo_mul<T, N, 0>(u, ut);
      }
      const int64_t pt0 = (((int64_t)l * g.n_ecol + (active ? ecol : 0)) * N) * L + line;
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T ur = f1[k * SK + vo], us = f2[k * SK + vo], uz = ut[k];
        T R, Sv;
        if constexpr (STORED) {
          const int64_t pt = pt0 + (int64_t)k * L;
          const T* G = a.G;
          const T grr = G[pt], grs = G[PT + pt], gss = G[2 * PT + pt];
          const T grt = G[3 * PT + pt], gst = G[4 * PT + pt], gtt = G[5 * PT + pt];
          R = grr * ur + grs * us + grt * uz;
          Sv = grs * ur + gss * us + gst * uz;
          tt[k] = grt * ur + gst * us + gtt * uz;
        } else {
          const T sigma = (T(l) + T(0.5) * (T(1) + sXi[k])) * inv_nz;
          const T wk = sW[k];
          const T zr = lg.Pr + sigma * lg.Qr, zs = lg.Ps + sigma * lg.Qs;
          const T ax = zr * lg.rx + zs * lg.sx, ay = zr * lg.ry + zs * lg.sy;
          const T wc = wk * lg.cw;
          const T grt = -wc * (lg.rx * ax + lg.ry * ay);
          const T gst = -wc * (lg.sx * ax + lg.sy * ay);
          const T gtt = wc * (ax * ax + ay * ay + T(1)) * lg.Ainv;
          R = wk * (lg.grr * ur + lg.grs * us) + grt * uz;
          Sv = wk * (lg.grs * ur + lg.gss * us) + gst * uz;
          tt[k] = grt * ur + gst * us + gtt * uz;
        }
        f0[k * SK + vo] = R;
        f3[k * SK + vo] = Sv;
      }
      __syncthreads();
      // ---- R and S: transposed contractions
      {
        T v[N], r[N];
  #pragma unroll
        for (int i = 0; i < N; ++i) v[i] = f0[ro + i];
        eo_mul<T, N, 1>(v, r);
  #pragma unroll
        for (int i = 0; i < N; ++i) f1[ro + i] = r[i];
  #pragma unroll
        for (int j = 0; j < N; ++j) v[j] = f3[so + j * SJ];
        eo_mul<T, N, 1>(v, r);
  #pragma unroll
        for (int j = 0; j < N; ++j) f2[so + j * SJ] = r[j];
      }
      __syncthreads();
      // ---- V: transposed t-contraction, sum, vertical assembly, stores
      T y[N];
      eo_mul<T, N, 1>(tt, y);
  #pragma unroll
      for (int k = 0; k < N; ++k) y[k] += f1[k * SK + vo] + f2[k * SK + vo];
      y[0] += carry;
      carry = y[P];
      if (active) {
  #pragma unroll
        for (int k = 0; k < P; ++k) ax_put(g, a, ecol, col, slot, l * P + k, y[k]);
      }
    }
    if (active) ax_put(g, a, ecol, col, slot, g.nv - 1, carry);
  }
};

}  // namespace fnpf

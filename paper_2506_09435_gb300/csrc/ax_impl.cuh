// Matrix-free stiffness operator of the weak Laplace form (arXiv 2506.09435,
// Sec. 3.1.1, Eq. Laplace_weak) on the free-surface-following extruded mesh
// (Sec. 3.1.2; Step 4.1 of Sec. 3.4), sum-factorised on GLL nodes.
//
//   y = sum_e P_e^T Dhat^T G_e Dhat P_e x,   G = w_i w_j w_k |det J| J^-1 J^-T
//
// Geometric factors are never stored: each element column rebuilds them from
// eta and h (and the horizontal metric, fixed at mesh creation) for every
// application.  With the vertical extrusion z = -h + sigma (eta + h), the
// Jacobian is
//     [x_r x_s 0; y_r y_s 0; z_r z_s z_t],  z_t = (eta + h) / (2 Nz),
//     z_r = -h_r + sigma (eta_r + h_r),  z_s likewise,
// so with (r_x, r_y, s_x, s_y) the inverse horizontal Jacobian,
// a = z_r grad r + z_s grad s and cw = w_i w_j |det H|:
//     G_rr = w_k cw z_t |grad r|^2,  G_rs = w_k cw z_t grad r . grad s, ...
//     G_rt = -w_k cw grad r . a,   G_st = -w_k cw grad s . a,
//     G_tt = w_k cw (|a|^2 + 1) / z_t.
//
// Work decomposition: one thread per vertical GLL line (i, j) of an element
// column, looping over the Nz stacked elements; the line's values stay in
// registers (t-contractions and the vertical assembly between stacked
// elements are thread-local), the horizontal slices go through shared memory
// for the r- and s-contractions.  C element columns share a CTA.
// Horizontal assembly is deterministic without atomics: lines interior to an
// element column are written directly; boundary ("ring") lines are written to
// a per-element-column ring buffer and summed in a fixed order by
// ring_gather_kernel.
#pragma once

#include "fnpf_internal.cuh"

namespace fnpf {

template <typename T, int N, int DIM, int C>
struct AxShape {
  static constexpr int P = N - 1;
  static constexpr int NY = DIM == 3 ? N : 1;
  static constexpr int L = N * NY;            // lines per element column
  static constexpr int THREADS = C * L;
  static constexpr int BUF = C * N * L;       // one field over the CTA's element columns
  static constexpr size_t SMEM = sizeof(T) * (3 * BUF + N * N + 2 * N + 2 * C * L);
};

template <typename T>
__device__ __forceinline__ void ax_put(const Geom& g, const AxPtrs<T>& a, int ecol, int col, int slot, int plane,
                                       T v) {
  const bool surf = plane == g.nv - 1;
  if (surf && a.ys == nullptr) return;
  if (slot < 0) {
    if (surf) a.ys[col] = v;
    else a.yI[(int64_t)plane * g.ns + col] = v;
  } else {
    a.ring[((int64_t)plane * g.n_ecol + ecol) * g.ring + slot] = v;
  }
}

// Per-line geometry shared by the apply and the diagonal kernels.
template <typename T>
struct LineGeom {
  T rx, ry, sx, sy, cw;      // horizontal metric
  T A, Ainv;                 // z_t and 1 / z_t
  T Pr, Qr, Ps, Qs;          // z_r = Pr + sigma Qr, z_s = Ps + sigma Qs
  T grr, grs, gss;           // G_rr / w_k etc.
};

// Loads the CTA's tables and eta/h tiles, computes the line geometry.
// Leaves sD, sXi, sW filled; ends with a __syncthreads().
template <typename T, int N, int DIM, int C>
__device__ __forceinline__ void ax_prologue(const Geom& g, const Tables<T>& t, const T* eta_g, T* sD, T* sXi, T* sW,
                                            T* sE, T* sH, int c, int line, int i, int j, int ecol, bool active,
                                            int& col, LineGeom<T>& lg) {
  using S = AxShape<T, N, DIM, C>;
  constexpr int L = S::L;
  for (int q = threadIdx.x; q < N * N; q += S::THREADS) sD[q] = t.D[q];
  for (int q = threadIdx.x; q < N; q += S::THREADS) {
    sXi[q] = t.xi[q];
    sW[q] = t.w[q];
  }
  col = 0;
  if (active) col = node_col(g, ecol % g.nx, ecol / g.nx, i, j);
  const T eta = active ? eta_g[col] : T(0);
  const T hh = active ? t.h[col] : T(1);
  sE[c * L + line] = eta;
  sH[c * L + line] = hh;
  __syncthreads();
  T er = 0, hr = 0, es = 0, hs = 0;
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const T d = sD[i * N + m];
    er += d * sE[c * L + j * N + m];
    hr += d * sH[c * L + j * N + m];
  }
  if (DIM == 3) {
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const T d = sD[j * N + m];
      es += d * sE[c * L + m * N + i];
      hs += d * sH[c * L + m * N + i];
    }
  }
  const int64_t hstride = (int64_t)g.n_ecol * L;
  const int64_t hidx = (int64_t)(active ? ecol : 0) * L + line;
  lg.rx = t.hm[hidx];
  lg.ry = t.hm[hstride + hidx];
  lg.sx = t.hm[2 * hstride + hidx];
  lg.sy = t.hm[3 * hstride + hidx];
  lg.cw = t.hm[4 * hstride + hidx];
  lg.A = (eta + hh) * (T(0.5) / T(g.nz));
  lg.Ainv = T(1) / lg.A;
  lg.Pr = -hr;
  lg.Qr = er + hr;
  lg.Ps = -hs;
  lg.Qs = es + hs;
  const T ca = lg.cw * lg.A;
  lg.grr = ca * (lg.rx * lg.rx + lg.ry * lg.ry);
  lg.grs = ca * (lg.rx * lg.sx + lg.ry * lg.sy);
  lg.gss = ca * (lg.sx * lg.sx + lg.sy * lg.sy);
}

template <typename T, int N, int DIM, int C>
struct ax_kernel {
  static constexpr int kThreads = AxShape<T, N, DIM, C>::THREADS;
  __device__ static void run(Blk bk, Geom g, Tables<T> t, AxPtrs<T> a) {
    using S = AxShape<T, N, DIM, C>;
    constexpr int P = N - 1, L = S::L;
    extern __shared__ __align__(16) unsigned char ax_smem[];
    T* sU = reinterpret_cast<T*>(ax_smem);
    T* sR = sU + S::BUF;
    T* sS = sR + S::BUF;
    T* sD = sS + S::BUF;
    T* sXi = sD + N * N;
    T* sW = sXi + N;
    T* sE = sW + N;
    T* sH = sE + C * L;
    if (a.skip && *a.skip) return;
    const int c = threadIdx.x / L, line = threadIdx.x - c * L;
    const int i = line % N, j = line / N;
    const int ecol = bk.x * C + c;
    const bool active = ecol < g.n_ecol;
    int col;
    LineGeom<T> lg;
    ax_prologue<T, N, DIM, C>(g, t, a.eta, sD, sXi, sW, sE, sH, c, line, i, j, ecol, active, col, lg);
    const int slot = ring_slot(DIM, P, i, j);
    const T inv_nz = T(1) / T(g.nz);
    // FP32: the D entries of this thread's r- and s-contractions are kept in
    // registers, so that the field values are the only shared-memory operand
    // there (the FP32 kernel is bound by shared-memory loads).  FP64 reads them
    // from shared memory: that kernel is bound by the FP64 pipe, and its
    // latency-bound coarse-level instances run better with fewer registers.
    constexpr bool kDReg = sizeof(T) == 4;
    T Di[N], Dj[N], DiT[N], DjT[N];
  #pragma unroll
    for (int m = 0; m < N; ++m) {
      Di[m] = sD[i * N + m];
      Dj[m] = sD[j * N + m];
      DiT[m] = sD[m * N + i];
      DjT[m] = sD[m * N + j];
    }

    T carry = 0;
    for (int l = 0; l < g.nz; ++l) {
      T u[N];
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
        u[k] = v;
      }
      __syncthreads();   // readers of the previous layer's slices are done
  #pragma unroll
      for (int k = 0; k < N; ++k) sU[(c * N + k) * L + line] = u[k];
      __syncthreads();
      T ft[N];
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* uk = sU + (c * N + k) * L;
        T ur = 0, us = 0, ut = 0;
  #pragma unroll
        for (int m = 0; m < N; ++m) ur += (kDReg ? Di[m] : sD[i * N + m]) * uk[j * N + m];
        if (DIM == 3) {
  #pragma unroll
          for (int m = 0; m < N; ++m) us += (kDReg ? Dj[m] : sD[j * N + m]) * uk[m * N + i];
        }
  #pragma unroll
        for (int m = 0; m < N; ++m) ut += sD[k * N + m] * u[m];
        const T sigma = (T(l) + T(0.5) * (T(1) + sXi[k])) * inv_nz;
        const T wk = sW[k];
        const T zr = lg.Pr + sigma * lg.Qr, zs = lg.Ps + sigma * lg.Qs;
        const T ax = zr * lg.rx + zs * lg.sx, ay = zr * lg.ry + zs * lg.sy;
        const T wc = wk * lg.cw;
        const T grt = -wc * (lg.rx * ax + lg.ry * ay);
        const T gst = -wc * (lg.sx * ax + lg.sy * ay);
        const T gtt = wc * (ax * ax + ay * ay + T(1)) * lg.Ainv;
        sR[(c * N + k) * L + line] = wk * (lg.grr * ur + lg.grs * us) + grt * ut;
        if (DIM == 3) sS[(c * N + k) * L + line] = wk * (lg.grs * ur + lg.gss * us) + gst * ut;
        ft[k] = grt * ur + gst * us + gtt * ut;
      }
      __syncthreads();
      T y[N];
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* rk = sR + (c * N + k) * L;
        const T* sk = sS + (c * N + k) * L;
        T s = 0;
  #pragma unroll
        for (int m = 0; m < N; ++m) s += (kDReg ? DiT[m] : sD[m * N + i]) * rk[j * N + m];
        if (DIM == 3) {
  #pragma unroll
          for (int m = 0; m < N; ++m) s += (kDReg ? DjT[m] : sD[m * N + j]) * sk[m * N + i];
        }
  #pragma unroll
        for (int m = 0; m < N; ++m) s += sD[m * N + k] * ft[m];
        y[k] = s;
      }
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

// diag(A): per node (i, j, k) of an element,
//   sum_m D_mi^2 G_rr(m,j,k) + sum_m D_mj^2 G_ss(i,m,k) + sum_m D_mk^2 G_tt(i,j,m)
//   + 2 D_ii D_jj G_rs + 2 D_ii D_kk G_rt + 2 D_jj D_kk G_st   (all at (i,j,k)).
template <typename T, int N, int DIM, int C>
struct diag_kernel {
  static constexpr int kThreads = AxShape<T, N, DIM, C>::THREADS;
  __device__ static void run(Blk bk, Geom g, Tables<T> t, AxPtrs<T> a) {
    using S = AxShape<T, N, DIM, C>;
    constexpr int P = N - 1, L = S::L;
    extern __shared__ __align__(16) unsigned char ax_smem[];
    T* sU = reinterpret_cast<T*>(ax_smem);
    T* sR = sU + S::BUF;
    T* sS = sR + S::BUF;
    T* sD = sS + S::BUF;
    T* sXi = sD + N * N;
    T* sW = sXi + N;
    T* sE = sW + N;
    T* sH = sE + C * L;
    (void)sS;
    const int c = threadIdx.x / L, line = threadIdx.x - c * L;
    const int i = line % N, j = line / N;
    const int ecol = bk.x * C + c;
    const bool active = ecol < g.n_ecol;
    int col;
    LineGeom<T> lg;
    ax_prologue<T, N, DIM, C>(g, t, a.eta, sD, sXi, sW, sE, sH, c, line, i, j, ecol, active, col, lg);
    const int slot = ring_slot(DIM, P, i, j);
    const T inv_nz = T(1) / T(g.nz);
    const T Dii = sD[i * N + i];
    const T Djj = DIM == 3 ? sD[j * N + j] : T(0);

    T carry = 0;
    for (int l = 0; l < g.nz; ++l) {
      T grt[N], gst[N], gtt[N];
      __syncthreads();
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T sigma = (T(l) + T(0.5) * (T(1) + sXi[k])) * inv_nz;
        const T wk = sW[k];
        const T zr = lg.Pr + sigma * lg.Qr, zs = lg.Ps + sigma * lg.Qs;
        const T ax = zr * lg.rx + zs * lg.sx, ay = zr * lg.ry + zs * lg.sy;
        const T wc = wk * lg.cw;
        grt[k] = -wc * (lg.rx * ax + lg.ry * ay);
        gst[k] = -wc * (lg.sx * ax + lg.sy * ay);
        gtt[k] = wc * (ax * ax + ay * ay + T(1)) * lg.Ainv;
        sU[(c * N + k) * L + line] = wk * lg.grr;
        sR[(c * N + k) * L + line] = wk * lg.gss;
      }
      __syncthreads();
      T y[N];
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* uk = sU + (c * N + k) * L;
        const T* rk = sR + (c * N + k) * L;
        T s = 0;
  #pragma unroll
        for (int m = 0; m < N; ++m) {
          const T d = sD[m * N + i];
          s += d * d * uk[j * N + m];
        }
        if (DIM == 3) {
  #pragma unroll
          for (int m = 0; m < N; ++m) {
            const T d = sD[m * N + j];
            s += d * d * rk[m * N + i];
          }
        }
  #pragma unroll
        for (int m = 0; m < N; ++m) {
          const T d = sD[m * N + k];
          s += d * d * gtt[m];
        }
        const T Dkk = sD[k * N + k];
        s += T(2) * Dii * Dkk * grt[k];
        if (DIM == 3) s += T(2) * (Dii * Djj * sW[k] * lg.grs + Djj * Dkk * gst[k]);
        y[k] = s;
      }
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

// Number of stored metric entries per point: (rr, rs, ss, rt, st, tt) in 3D,
// (rr, rt, tt) in 2D.  Layout G[e][pt], pt = ((l n_ecol + ecol) N + k) L + line,
// so the threads of a CTA read consecutive addresses.
template <int DIM>
struct NGeo {
  static constexpr int value = DIM == 3 ? 6 : 3;
};

// G of every element point, from eta, h and the horizontal metric (the same
// formulas as the on-the-fly operator); run once per solve.
template <typename T, int N, int DIM, int C>
struct geom_kernel {
  static constexpr int kThreads = AxShape<T, N, DIM, C>::THREADS;
  __device__ static void run(Blk bk, Geom g, Tables<T> t, AxPtrs<T> a) {
    using S = AxShape<T, N, DIM, C>;
    constexpr int L = S::L;
    extern __shared__ __align__(16) unsigned char ax_smem[];
    T* sD = reinterpret_cast<T*>(ax_smem) + 3 * S::BUF;
    T* sXi = sD + N * N;
    T* sW = sXi + N;
    T* sE = sW + N;
    T* sH = sE + C * L;
    const int c = threadIdx.x / L, line = threadIdx.x - c * L;
    const int i = line % N, j = line / N;
    const int ecol = bk.x * C + c;
    const bool active = ecol < g.n_ecol;
    int col;
    LineGeom<T> lg;
    ax_prologue<T, N, DIM, C>(g, t, a.eta, sD, sXi, sW, sE, sH, c, line, i, j, ecol, active, col, lg);
    if (!active) return;
    const T inv_nz = T(1) / T(g.nz);
    const int64_t P = (int64_t)g.nz * g.n_ecol * N * L;
    T* G = a.G;
    for (int l = 0; l < g.nz; ++l) {
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T sigma = (T(l) + T(0.5) * (T(1) + sXi[k])) * inv_nz;
        const T wk = sW[k];
        const T zr = lg.Pr + sigma * lg.Qr, zs = lg.Ps + sigma * lg.Qs;
        const T ax = zr * lg.rx + zs * lg.sx, ay = zr * lg.ry + zs * lg.sy;
        const T wc = wk * lg.cw;
        const int64_t pt = (((int64_t)l * g.n_ecol + ecol) * N + k) * L + line;
        if (DIM == 3) {
          G[pt] = wk * lg.grr;
          G[P + pt] = wk * lg.grs;
          G[2 * P + pt] = wk * lg.gss;
          G[3 * P + pt] = -wc * (lg.rx * ax + lg.ry * ay);
          G[4 * P + pt] = -wc * (lg.sx * ax + lg.sy * ay);
          G[5 * P + pt] = wc * (ax * ax + ay * ay + T(1)) * lg.Ainv;
        } else {
          G[pt] = wk * lg.grr;
          G[P + pt] = -wc * (lg.rx * ax);
          G[2 * P + pt] = wc * (ax * ax + T(1)) * lg.Ainv;
        }
      }
    }
  }
};

// The operator with G read from memory instead of rebuilt: fewer FP64
// instructions per point, for the FP64 solves where the FP64 pipe is the bound.
template <typename T, int N, int DIM, int C>
struct axg_kernel {
  static constexpr int kThreads = AxShape<T, N, DIM, C>::THREADS;
  __device__ static void run(Blk bk, Geom g, Tables<T> t, AxPtrs<T> a) {
    using S = AxShape<T, N, DIM, C>;
    constexpr int P = N - 1, L = S::L;
    extern __shared__ __align__(16) unsigned char ax_smem[];
    T* sU = reinterpret_cast<T*>(ax_smem);
    T* sR = sU + S::BUF;
    T* sS = sR + S::BUF;
    T* sD = sS + S::BUF;
    if (a.skip && *a.skip) return;
    const int c = threadIdx.x / L, line = threadIdx.x - c * L;
    const int i = line % N, j = line / N;
    const int ecol = bk.x * C + c;
    const bool active = ecol < g.n_ecol;
    for (int q = threadIdx.x; q < N * N; q += S::THREADS) sD[q] = t.D[q];
    int col = 0;
    if (active) col = node_col(g, ecol % g.nx, ecol / g.nx, i, j);
    const int slot = ring_slot(DIM, P, i, j);
    const int64_t PT = (int64_t)g.nz * g.n_ecol * N * L;
    const T* G = a.G;
    __syncthreads();
    constexpr bool kDReg = sizeof(T) == 4;   // as in ax_kernel
    T Di[N], Dj[N], DiT[N], DjT[N];
  #pragma unroll
    for (int m = 0; m < N; ++m) {
      Di[m] = sD[i * N + m];
      Dj[m] = sD[j * N + m];
      DiT[m] = sD[m * N + i];
      DjT[m] = sD[m * N + j];
    }
    T carry = 0;
    for (int l = 0; l < g.nz; ++l) {
      T u[N];
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
        u[k] = v;
      }
      __syncthreads();
  #pragma unroll
      for (int k = 0; k < N; ++k) sU[(c * N + k) * L + line] = u[k];
      __syncthreads();
      T ft[N];
      const int64_t pt0 = (((int64_t)l * g.n_ecol + (active ? ecol : 0)) * N) * L + line;
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* uk = sU + (c * N + k) * L;
        T ur = 0, us = 0, ut = 0;
  #pragma unroll
        for (int m = 0; m < N; ++m) ur += (kDReg ? Di[m] : sD[i * N + m]) * uk[j * N + m];
        if (DIM == 3) {
  #pragma unroll
          for (int m = 0; m < N; ++m) us += (kDReg ? Dj[m] : sD[j * N + m]) * uk[m * N + i];
        }
  #pragma unroll
        for (int m = 0; m < N; ++m) ut += sD[k * N + m] * u[m];
        const int64_t pt = pt0 + (int64_t)k * L;
        if (DIM == 3) {
          const T grr = G[pt], grs = G[PT + pt], gss = G[2 * PT + pt];
          const T grt = G[3 * PT + pt], gst = G[4 * PT + pt], gtt = G[5 * PT + pt];
          sR[(c * N + k) * L + line] = grr * ur + grs * us + grt * ut;
          sS[(c * N + k) * L + line] = grs * ur + gss * us + gst * ut;
          ft[k] = grt * ur + gst * us + gtt * ut;
        } else {
          const T grr = G[pt], grt = G[PT + pt], gtt = G[2 * PT + pt];
          sR[(c * N + k) * L + line] = grr * ur + grt * ut;
          ft[k] = grt * ur + gtt * ut;
        }
      }
      __syncthreads();
      T y[N];
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* rk = sR + (c * N + k) * L;
        const T* sk = sS + (c * N + k) * L;
        T s = 0;
  #pragma unroll
        for (int m = 0; m < N; ++m) s += (kDReg ? DiT[m] : sD[m * N + i]) * rk[j * N + m];
        if (DIM == 3) {
  #pragma unroll
          for (int m = 0; m < N; ++m) s += (kDReg ? DjT[m] : sD[m * N + j]) * sk[m * N + i];
        }
  #pragma unroll
        for (int m = 0; m < N; ++m) s += sD[m * N + k] * ft[m];
        y[k] = s;
      }
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

// Sums the ring contributions of every element-boundary node column, in a
// fixed order (x owners outer, y owners inner), and writes the output field.
template <typename T, int N, int DIM>
struct ring_gather_kernel {
  static constexpr int kThreads = 256;
  __device__ static void run(Blk bk, Geom g, const T* __restrict__ ring, T* yI, T* ys, int nplanes,
                             int64_t nring_cols, const int* skip) {
    if (skip && *skip) return;
    const int64_t idx = (int64_t)bk.x * blockDim.x + threadIdx.x;
    if (idx >= nring_cols * nplanes) return;
    const int plane = (int)(idx / nring_cols);
    const int64_t rc = idx - (int64_t)plane * nring_cols;
    constexpr int p = N - 1;   // the order as a constant: divisions by p fold
    const int nlx = g.nx + (g.px ? 0 : 1);
    int ix, iy;
    if (DIM == 2) {
      ix = (int)rc * p;
      iy = 0;
    } else {
      const int64_t part1 = (int64_t)nlx * g.ncy;
      if (rc < part1) {
        ix = (int)(rc % nlx) * p;
        iy = (int)(rc / nlx);
      } else {
        // element-interior x positions on the y-boundary lines (none at p = 1,
        // where this branch is never taken; pm1 keeps the divisor non-zero)
        constexpr int pm1 = p > 1 ? p - 1 : 1;
        const int64_t m = rc - part1;
        const int per = g.nx * pm1;
        const int ly = (int)(m / per);
        const int mm = (int)(m - (int64_t)ly * per);
        ix = (mm / pm1) * p + 1 + mm % pm1;
        iy = ly * p;
      }
    }
    int exo[2], io[2], eyo[2] = {0, 0}, jo[2] = {0, 0};
    const int cx = line_owners(ix, p, g.nx, g.px, exo, io);
    const int cy = DIM == 3 ? line_owners(iy, p, g.ny, g.py, eyo, jo) : 1;
    T s = 0;
    for (int u = 0; u < cx; ++u) {
      for (int v = 0; v < cy; ++v) {
        const int ecol = eyo[v] * g.nx + exo[u];
        const int slot = ring_slot(DIM, p, io[u], jo[v]);
        s += ring[((int64_t)plane * g.n_ecol + ecol) * g.ring + slot];
      }
    }
    const int col = iy * g.ncx + ix;
    if (plane == g.nv - 1) ys[col] = s;
    else yI[(int64_t)plane * g.ns + col] = s;
  }
};

// Gather fused with a vector update: one thread per interior unknown (a 2D
// grid of columns x interior planes, so no 64-bit index division); the
// operator output w_i is read from yI on column-interior lines (written there
// by the operator kernel) or summed from the ring buffer on element-boundary
// lines (same owners and order as ring_gather_kernel), then the Epilogue
// update is applied; yI itself is left as the operator kernel wrote it.
template <typename T, int N, int DIM>
struct gather_update_kernel {
  static constexpr int kThreads = 256;
  __device__ static void run(Blk bk, Geom g, const T* __restrict__ ring, const T* __restrict__ yI, const int* skip,
                             Epilogue<T> ep) {
    if (skip && *skip) return;
    const int col = bk.x * blockDim.x + threadIdx.x;   // grid: (columns, interior planes)
    if (col >= g.ns) return;
    const int plane = bk.y;
    const int64_t i = (int64_t)plane * g.ns + col;
    const int iy = col / g.ncx, ix = col - iy * g.ncx;
    constexpr int p = N - 1;
    T w;
    if (ix % p != 0 && (DIM == 2 || iy % p != 0)) {
      w = yI[i];
    } else {
      int exo[2], io[2], eyo[2] = {0, 0}, jo[2] = {0, 0};
      const int cx = line_owners(ix, p, g.nx, g.px, exo, io);
      const int cy = DIM == 3 ? line_owners(iy, p, g.ny, g.py, eyo, jo) : 1;
      w = T(0);
      for (int u = 0; u < cx; ++u)
        for (int v = 0; v < cy; ++v) {
          const int ecol = eyo[v] * g.nx + exo[u];
          w += ring[((int64_t)plane * g.n_ecol + ecol) * g.ring + ring_slot(DIM, p, io[u], jo[v])];
        }
    }
    apply_epilogue(ep, i, w);
  }
};

inline int64_t ring_columns(const Geom& g) {
  const int nlx = g.nx + (g.px ? 0 : 1);
  if (g.dim == 2) return nlx;
  const int nly = g.ny + (g.py ? 0 : 1);
  return (int64_t)nlx * g.ncy + (int64_t)nly * g.nx * (g.p - 1);
}

template <typename T, int N, int DIM>
cudaError_t launch_gather(const Geom& g, const T* ring, T* yI, T* ys, const int* skip, cudaStream_t s) {
  const int nplanes = ys ? g.nv : g.nv - 1;
  const int64_t nrc = ring_columns(g);
  const int64_t total = nrc * nplanes;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  launch<ring_gather_kernel<T, N, DIM>>((unsigned)blocks, threads, 0, s, g, ring, yI, ys, nplanes, nrc, skip);
  return cudaGetLastError();
}

template <typename T, int N, int DIM>
cudaError_t launch_gather_update(const Geom& g, const T* ring, const T* yI, const int* skip, const Epilogue<T>& ep,
                                 cudaStream_t s) {
  if (g.NI == 0) return cudaSuccess;
  const dim3 grid((unsigned)((g.ns + 255) / 256), (unsigned)(g.nv - 1));
  launch<gather_update_kernel<T, N, DIM>>(grid, 256, 0, s, g, ring, yI, skip, ep);
  return cudaGetLastError();
}

template <typename T, int N, int DIM, int C, typename K>
cudaError_t set_smem_attr(K kernel, std::atomic<uint64_t>* done) {
  return smem_optin(kernel, AxShape<T, N, DIM, C>::SMEM, done);
}

// mode: AX_APPLY (on-the-fly geometry), AX_DIAG, AX_GEOM (store G), AX_APPLY_G (stored G)
template <typename T, int N, int DIM, int C>
cudaError_t launch_ax_shape(const Geom& g, const Tables<T>& t, const AxPtrs<T>& a, int mode, cudaStream_t s) {
  using S = AxShape<T, N, DIM, C>;
  const unsigned blocks = (unsigned)((g.n_ecol + C - 1) / C);
  cudaError_t e;
  if (mode == AX_GEOM) {
    static std::atomic<uint64_t> attr{0};
    if ((e = set_smem_attr<T, N, DIM, C>(kernel_one<geom_kernel<T, N, DIM, C>>(), &attr)) != cudaSuccess) return e;
    launch<geom_kernel<T, N, DIM, C>>(blocks, S::THREADS, S::SMEM, s, g, t, a);
    return cudaGetLastError();
  }
  if (mode == AX_APPLY_G) {
    static std::atomic<uint64_t> attr{0};
    if ((e = set_smem_attr<T, N, DIM, C>(kernel_one<axg_kernel<T, N, DIM, C>>(), &attr)) != cudaSuccess) return e;
    launch<axg_kernel<T, N, DIM, C>>(blocks, S::THREADS, S::SMEM, s, g, t, a);
  } else if (mode == AX_DIAG) {
    static std::atomic<uint64_t> attr{0};
    if ((e = set_smem_attr<T, N, DIM, C>(kernel_one<diag_kernel<T, N, DIM, C>>(), &attr)) != cudaSuccess) return e;
    launch<diag_kernel<T, N, DIM, C>>(blocks, S::THREADS, S::SMEM, s, g, t, a);
  } else {
    static std::atomic<uint64_t> attr{0};
    if ((e = set_smem_attr<T, N, DIM, C>(kernel_one<ax_kernel<T, N, DIM, C>>(), &attr)) != cudaSuccess) return e;
    launch<ax_kernel<T, N, DIM, C>>(blocks, S::THREADS, S::SMEM, s, g, t, a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.ep.op != EP_NONE) return launch_gather_update<T, N, DIM>(g, a.ring, a.yI, a.skip, a.ep, s);
  return launch_gather<T, N, DIM>(g, a.ring, a.yI, a.ys, a.skip, s);
}

}  // namespace fnpf

#include "axl_impl.cuh"
#include "axz_impl.cuh"

namespace fnpf {

// Elements-per-CTA candidates for order N (3D); 2D uses one shape.  Variants
// 0-3 are the one-thread-per-vertical-line kernels (ax_kernel, axg_kernel);
// the fourth choice gives grids that fill the 152 SMs evenly for common column
// counts (e.g. 7 columns of N = 7: 147 CTAs for 32 x 32 columns, where 2 and 4
// leave a partial second wave on a third of the SMs).  Variants 4-7 are the
// line-decomposed kernel (axl_kernel) with these element columns per CTA;
// variants 8-11 the vertical-line kernels with two element layers in flight
// (axz_kernel).
template <int N>
struct CtaChoices;
template <> struct CtaChoices<2> { static constexpr int c[12] = {16, 32, 64, 8, 32, 64, 128, 16, 16, 32, 64, 8}; };
template <> struct CtaChoices<3> { static constexpr int c[12] = {7, 14, 28, 4, 16, 32, 56, 8, 7, 14, 28, 4}; };
template <> struct CtaChoices<4> { static constexpr int c[12] = {4, 8, 16, 2, 8, 16, 32, 4, 4, 8, 16, 2}; };
template <> struct CtaChoices<5> { static constexpr int c[12] = {3, 5, 10, 2, 8, 16, 4, 12, 3, 5, 10, 2}; };
template <> struct CtaChoices<6> { static constexpr int c[12] = {2, 4, 8, 6, 4, 8, 14, 2, 2, 4, 8, 6}; };
template <> struct CtaChoices<7> { static constexpr int c[12] = {1, 2, 4, 7, 7, 4, 10, 2, 1, 2, 4, 7}; };
template <> struct CtaChoices<8> { static constexpr int c[12] = {1, 2, 4, 3, 2, 4, 8, 3, 1, 2, 4, 3}; };
template <> struct CtaChoices<9> { static constexpr int c[12] = {1, 2, 3, 4, 2, 4, 6, 3, 1, 2, 3, 4}; };
static_assert(sizeof(CtaChoices<7>::c) / sizeof(int) == kCtaVariants, "one shape per variant");
constexpr int kLineVariant0 = 4;   // first variant of the line-decomposed kernel
constexpr int kLayerVariant0 = 8;  // first variant of the layer-parallel kernel

// Layer-parallel kernel launch (3D, AX_APPLY or AX_APPLY_G), then the gather.
template <typename T, int N, int C>
cudaError_t launch_axz_shape(const Geom& g, const Tables<T>& t, const AxPtrs<T>& a, int mode, cudaStream_t s) {
  constexpr int NZL = 2;
  using S = AxzShape<T, N, C, NZL>;
  const unsigned blocks = (unsigned)((g.n_ecol + C - 1) / C);
  cudaError_t e;
  if (mode == AX_APPLY_G) {
    static std::atomic<uint64_t> attr{0};
    if ((e = smem_optin(kernel_one<axz_kernel<T, N, C, NZL, true>>(), S::SMEM, &attr)) != cudaSuccess) return e;
    launch<axz_kernel<T, N, C, NZL, true>>(blocks, S::THREADS, S::SMEM, s, g, t, a);
  } else {
    static std::atomic<uint64_t> attr{0};
    if ((e = smem_optin(kernel_one<axz_kernel<T, N, C, NZL, false>>(), S::SMEM, &attr)) != cudaSuccess) return e;
    launch<axz_kernel<T, N, C, NZL, false>>(blocks, S::THREADS, S::SMEM, s, g, t, a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.ep.op != EP_NONE) return launch_gather_update<T, N, 3>(g, a.ring, a.yI, a.skip, a.ep, s);
  return launch_gather<T, N, 3>(g, a.ring, a.yI, a.ys, a.skip, s);
}

// Line-decomposed kernel launch (3D, AX_APPLY or AX_APPLY_G), then the gather.
template <typename T, int N, int C>
cudaError_t launch_axl_shape(const Geom& g, const Tables<T>& t, const AxPtrs<T>& a, int mode, cudaStream_t s) {
  using S = AxlShape<T, N, C>;
  cudaError_t e = eo_upload();
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((g.n_ecol + C - 1) / C);
  if (mode == AX_APPLY_G) {
    static std::atomic<uint64_t> attr{0};
    if ((e = smem_optin(kernel_one<axl_kernel<T, N, C, true>>(), S::SMEM, &attr)) != cudaSuccess) return e;
    launch<axl_kernel<T, N, C, true>>(blocks, S::THREADS, S::SMEM, s, g, t, a);
  } else {
    static std::atomic<uint64_t> attr{0};
    if ((e = smem_optin(kernel_one<axl_kernel<T, N, C, false>>(), S::SMEM, &attr)) != cudaSuccess) return e;
    launch<axl_kernel<T, N, C, false>>(blocks, S::THREADS, S::SMEM, s, g, t, a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.ep.op != EP_NONE) return launch_gather_update<T, N, 3>(g, a.ring, a.yI, a.skip, a.ep, s);
  return launch_gather<T, N, 3>(g, a.ring, a.yI, a.ys, a.skip, s);
}

template <typename T, int N>
cudaError_t launch_ax_n(const Geom& g, const Tables<T>& t, const AxPtrs<T>& a, int mode, int variant,
                        cudaStream_t s) {
  if (mode == AX_INIT) return eo_upload();
  if (g.dim == 2) return launch_ax_shape<T, N, 2, (128 + N - 1) / N>(g, t, a, mode, s);
  constexpr int C0 = CtaChoices<N>::c[0], C1 = CtaChoices<N>::c[1], C2 = CtaChoices<N>::c[2];
  constexpr int C3 = CtaChoices<N>::c[3];
  if (variant >= kLayerVariant0 && (mode == AX_APPLY || mode == AX_APPLY_G)) {
    switch (variant - kLayerVariant0) {
      case 0: return launch_axz_shape<T, N, CtaChoices<N>::c[8]>(g, t, a, mode, s);
      case 1: return launch_axz_shape<T, N, CtaChoices<N>::c[9]>(g, t, a, mode, s);
      case 2: return launch_axz_shape<T, N, CtaChoices<N>::c[10]>(g, t, a, mode, s);
      default: return launch_axz_shape<T, N, CtaChoices<N>::c[11]>(g, t, a, mode, s);
    }
  }
  if (variant >= kLineVariant0 && (mode == AX_APPLY || mode == AX_APPLY_G)) {
    switch (variant - kLineVariant0) {
      case 0: return launch_axl_shape<T, N, CtaChoices<N>::c[4]>(g, t, a, mode, s);
      case 1: return launch_axl_shape<T, N, CtaChoices<N>::c[5]>(g, t, a, mode, s);
      case 2: return launch_axl_shape<T, N, CtaChoices<N>::c[6]>(g, t, a, mode, s);
      default: return launch_axl_shape<T, N, CtaChoices<N>::c[7]>(g, t, a, mode, s);
    }
  }
  if (mode == AX_DIAG || mode == AX_GEOM || variant == 1) return launch_ax_shape<T, N, 3, C1>(g, t, a, mode, s);
  if (variant == 0) return launch_ax_shape<T, N, 3, C0>(g, t, a, mode, s);
  if (variant == 3) return launch_ax_shape<T, N, 3, C3>(g, t, a, mode, s);
  return launch_ax_shape<T, N, 3, C2>(g, t, a, mode, s);
}

}  // namespace fnpf

// Layer-parallel form of the vertical-line operator kernels (ax_kernel,
// axg_kernel) for 3D meshes: the same arithmetic, with the Nz stacked elements
// of an element column processed by NZL groups of threads at once instead of
// one after another.  On meshes with few element columns the one-thread-per-
// vertical-line kernels run out of warps (a 32 x 32 x 2 tank gives about 330
// threads per SM), and the operator is bound by latency; NZL layers in flight
// multiply the warps per SM by NZL.
//
// Thread (z, c, line): layer slot z of the group, element column c of the
// CTA, vertical GLL line (i, j).  Each layer's r-, s- and t-contractions use
// the layer's own shared slices.  The vertical assembly between stacked
// elements goes through shared memory: every layer thread leaves the value of
// its top plane in sC[z + 1], then adds sC[z] (the top of the layer below, or
// for z = 0 the carry of the previous group) to its bottom plane.  Ring lines
// and the gathers are those of ax_kernel.
#pragma once

namespace fnpf {

template <typename T, int N, int C, int NZL>
struct AxzShape {
  static constexpr int L = N * N;
  static constexpr int THREADS = NZL * C * L;
  static constexpr int BUF = NZL * C * N * L;   // one field over all layer slots and columns
  static constexpr size_t SMEM =
      sizeof(T) * (3 * (size_t)BUF + N * N + 2 * N + 2 * C * L + (size_t)(NZL + 1) * C * L);
};

template <typename T, int N, int C, int NZL, bool STORED>
struct axz_kernel {
  static constexpr int kThreads = AxzShape<T, N, C, NZL>::THREADS;
  __device__ static void run(Blk bk, Geom g, Tables<T> t, AxPtrs<T> a) {
    using S = AxzShape<T, N, C, NZL>;
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
    T* sC = sH + C * L;               // [NZL + 1][C][L] vertical carries
    if (a.skip && *a.skip) return;
    const int z = threadIdx.x / (C * L);
    const int cl = threadIdx.x - z * (C * L);
    const int c = cl / L, line = cl - c * L;
    const int i = line % N, j = line / N;
    const int ecol = bk.x * C + c;
    const bool active = ecol < g.n_ecol;
    int col = 0;
    LineGeom<T> lg{};
    if constexpr (STORED) {
      for (int q = threadIdx.x; q < N * N; q += S::THREADS) sD[q] = t.D[q];
      if (active) col = node_col(g, ecol % g.nx, ecol / g.nx, i, j);
      __syncthreads();
    } else {
      // every layer slot computes the line geometry (the same for all layers);
      // the tiles of eta and h are written by all slots with the same values
      ax_prologue<T, N, 3, C>(g, t, a.eta, sD, sXi, sW, sE, sH, c, line, i, j, ecol, active, col, lg);
    }
    const int slot = ring_slot(3, P, i, j);
    const T inv_nz = T(1) / T(g.nz);
    const int64_t PT = (int64_t)g.nz * g.n_ecol * N * L;
    const int base = (z * C + c) * N;   // this thread's slices: (base + k) * L + line
    if (z == 0) sC[c * L + line] = T(0);
    for (int l0 = 0; l0 < g.nz; l0 += NZL) {
      const int l = l0 + z;
      const bool lay = l < g.nz;
      T u[N];
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const int plane = l * P + k;
        T v = 0;
        if (active && lay) {
          if (plane < g.nv - 1) {
            if (a.xI) v = a.xI[(int64_t)plane * g.ns + col];
          } else if (a.xs) {
            v = a.xs[col];
          }
        }
        u[k] = v;
      }
      __syncthreads();   // readers of the previous group's slices and carries are done
  #pragma unroll
      for (int k = 0; k < N; ++k) sU[(base + k) * L + line] = u[k];
      __syncthreads();
      T ft[N];
      const int64_t pt0 = (((int64_t)(lay ? l : 0) * g.n_ecol + (active ? ecol : 0)) * N) * L + line;
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* uk = sU + (base + k) * L;
        T ur = 0, us = 0, ut = 0;
  #pragma unroll
        for (int m = 0; m < N; ++m) ur += sD[i * N + m] * uk[j * N + m];
  #pragma unroll
        for (int m = 0; m < N; ++m) us += sD[j * N + m] * uk[m * N + i];
  #pragma unroll
        for (int m = 0; m < N; ++m) ut += sD[k * N + m] * u[m];
        if constexpr (STORED) {
          const int64_t pt = pt0 + (int64_t)k * L;
          const T* G = a.G;
          const T grr = G[pt], grs = G[PT + pt], gss = G[2 * PT + pt];
          const T grt = G[3 * PT + pt], gst = G[4 * PT + pt], gtt = G[5 * PT + pt];
          sR[(base + k) * L + line] = grr * ur + grs * us + grt * ut;
          sS[(base + k) * L + line] = grs * ur + gss * us + gst * ut;
          ft[k] = grt * ur + gst * us + gtt * ut;
        } else {
          const T sigma = (T(lay ? l : 0) + T(0.5) * (T(1) + sXi[k])) * inv_nz;
          const T wk = sW[k];
          const T zr = lg.Pr + sigma * lg.Qr, zs = lg.Ps + sigma * lg.Qs;
          const T ax = zr * lg.rx + zs * lg.sx, ay = zr * lg.ry + zs * lg.sy;
          const T wc = wk * lg.cw;
          const T grt = -wc * (lg.rx * ax + lg.ry * ay);
          const T gst = -wc * (lg.sx * ax + lg.sy * ay);
          const T gtt = wc * (ax * ax + ay * ay + T(1)) * lg.Ainv;
          sR[(base + k) * L + line] = wk * (lg.grr * ur + lg.grs * us) + grt * ut;
          sS[(base + k) * L + line] = wk * (lg.grs * ur + lg.gss * us) + gst * ut;
          ft[k] = grt * ur + gst * us + gtt * ut;
        }
      }
      __syncthreads();
      T y[N];
  #pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* rk = sR + (base + k) * L;
        const T* sk = sS + (base + k) * L;
        T s = 0;
  #pragma unroll
        for (int m = 0; m < N; ++m) s += sD[m * N + i] * rk[j * N + m];
  #pragma unroll
        for (int m = 0; m < N; ++m) s += sD[m * N + j] * sk[m * N + i];
  #pragma unroll
        for (int m = 0; m < N; ++m) s += sD[m * N + k] * ft[m];
        y[k] = lay ? s : T(0);
      }
      // vertical assembly: the top plane of layer z + 1's neighbour below
      sC[((z + 1) * C + c) * L + line] = y[P];
      __syncthreads();
      y[0] += sC[(z * C + c) * L + line];
      if (active && lay) {
  #pragma unroll
        for (int k = 0; k < P; ++k) ax_put(g, a, ecol, col, slot, l * P + k, y[k]);
        if (l == g.nz - 1) ax_put(g, a, ecol, col, slot, g.nv - 1, y[P]);
      }
      __syncthreads();
      // the carry into the next group: the top plane of this group's last layer
      if (z == 0) sC[c * L + line] = sC[(NZL * C + c) * L + line];
    }
  }
};

}  // namespace fnpf

// Inter-level transfers of the p-multigrid preconditioner.
//
// Level spaces are the continuous GLL spaces Q_pf (fine) and Q_pc (coarse) on
// the same extruded element columns; Q_pc is contained in Q_pf on every
// element, so
//   prolongation P: u_f = (J x J x J) u_c per element, J[i][c] = l^c_c(xi^f_i)
//                   (evaluation of the coarse polynomial at the fine nodes;
//                   values on shared faces agree, each node is written once
//                   by its owning element);
//   restriction  R = P^T on assembled vectors: every fine node enters once,
//                   so element-local fine values are divided by their
//                   multiplicity (elements sharing the node), contracted with
//                   J^T in the three directions and summed into coarse nodes
//                   (vertical sums in registers, horizontal sums through the
//                   coarse ring buffer and ring_gather_kernel).
// Vectors carry the interior (non-surface) planes only; the surface plane of a
// correction is zero (homogeneous Dirichlet).
//
// One CTA per element column; thread (i, j) owns fine line (i, j); the
// smaller coarse-line work is spread over the same threads.
#pragma once

#include "ax_impl.cuh"

namespace fnpf {

template <typename T, int NF, int NC, int DIM>
struct XferShape {
  static constexpr int NYF = DIM == 3 ? NF : 1;
  static constexpr int NYC = DIM == 3 ? NC : 1;
  static constexpr int LF = NF * NYF;      // fine lines per element column
  static constexpr int LC = NC * NYC;      // coarse lines
  static constexpr int THREADS = LF;
};

// u_f = P u_c for one element column per CTA.
template <typename T, int NF, int NC, int DIM>
struct prolong_kernel {
  static constexpr int kThreads = XferShape<T, NF, NC, DIM>::THREADS;
  __device__ static void run(Blk bk, Geom gf, Geom gc, const T* __restrict__ J, const T* __restrict__ uc,
                             T* __restrict__ uf, int add, const int* skip) {
    if (skip && *skip) return;
    using S = XferShape<T, NF, NC, DIM>;
    constexpr int PF = NF - 1, PC = NC - 1;
    __shared__ T sJ[NF * NC];
    __shared__ T s1[NF * S::LC];          // [kf][coarse line]
    __shared__ T s2[NF * NC * NF];        // [kf][b][i_f]
    const int tid = threadIdx.x;
    for (int q = tid; q < NF * NC; q += S::THREADS) sJ[q] = J[q];
    const int ecol = bk.x;
    const int ex = ecol % gf.nx, ey = ecol / gf.nx;
    const int i = tid % NF, j = tid / NF;
    const int colf = node_col(gf, ex, ey, i, j);
    const bool own = (i < PF || (!gf.px && ex == gf.nx - 1)) && (DIM == 2 || j < PF || (!gf.py && ey == gf.ny - 1));
    // coarse line owned by this thread for the t-contraction
    const bool cl = tid < S::LC;
    const int ca = tid % NC, cb = tid / NC;
    const int colc = cl ? node_col(gc, ex, ey, ca, cb) : 0;
    __syncthreads();
    for (int l = 0; l < gf.nz; ++l) {
      if (cl) {
        T u[NC];
  #pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int plane = l * PC + c;
          u[c] = plane < gc.nv - 1 ? uc[(int64_t)plane * gc.ns + colc] : T(0);
        }
  #pragma unroll
        for (int k = 0; k < NF; ++k) {
          T s = 0;
  #pragma unroll
          for (int c = 0; c < NC; ++c) s += sJ[k * NC + c] * u[c];
          s1[k * S::LC + tid] = s;
        }
      }
      __syncthreads();
      if (DIM == 3) {
        // s2[k][b][i] = sum_a J[i][a] s1[k][b*NC + a]   (threads (i, b))
        if (tid < NF * NC) {
          const int ii = tid % NF, b = tid / NF;
  #pragma unroll
          for (int k = 0; k < NF; ++k) {
            T s = 0;
  #pragma unroll
            for (int a = 0; a < NC; ++a) s += sJ[ii * NC + a] * s1[k * S::LC + b * NC + a];
            s2[(k * NC + b) * NF + ii] = s;
          }
        }
        __syncthreads();
      }
  #pragma unroll
      for (int k = 0; k < PF; ++k) {
        T s = 0;
        if (DIM == 3) {
  #pragma unroll
          for (int b = 0; b < NC; ++b) s += sJ[j * NC + b] * s2[(k * NC + b) * NF + i];
        } else {
  #pragma unroll
          for (int a = 0; a < NC; ++a) s += sJ[i * NC + a] * s1[k * S::LC + a];
        }
        if (own) {
          T* dst = uf + (int64_t)(l * PF + k) * gf.ns + colf;
          *dst = add ? *dst + s : s;
        }
      }
      __syncthreads();
    }
  }
};

// r_c = P^T r_f (assembled); coarse ring lines go through `ring` and are summed
// by ring_gather_kernel on the coarse geometry.
template <typename T, int NF, int NC, int DIM>
struct restrict_kernel {
  static constexpr int kThreads = XferShape<T, NF, NC, DIM>::THREADS;
  __device__ static void run(Blk bk, Geom gf, Geom gc, const T* __restrict__ J, const T* __restrict__ rf,
                             T* __restrict__ rc, T* __restrict__ ring, const int* skip) {
    if (skip && *skip) return;
    using S = XferShape<T, NF, NC, DIM>;
    constexpr int PF = NF - 1, PC = NC - 1;
    __shared__ T sJ[NF * NC];
    __shared__ T s0[NF * S::LF];          // [kf][fine line]
    __shared__ T s1[NF * NC * NF];        // [kf][b][i_f]
    const int tid = threadIdx.x;
    for (int q = tid; q < NF * NC; q += S::THREADS) sJ[q] = J[q];
    const int ecol = bk.x;
    const int ex = ecol % gf.nx, ey = ecol / gf.nx;
    const int i = tid % NF, j = tid / NF;
    const int colf = node_col(gf, ex, ey, i, j);
    // horizontal multiplicity of this fine line
    int mh = 1;
    if ((i == 0 && (gf.px || ex > 0)) || (i == PF && (gf.px || ex < gf.nx - 1))) mh *= 2;
    if (DIM == 3 && ((j == 0 && (gf.py || ey > 0)) || (j == PF && (gf.py || ey < gf.ny - 1)))) mh *= 2;
    const T inv_mh = T(1) / T(mh);
    const bool cl = tid < S::LC;
    const int ca = tid % NC, cb = tid / NC;
    const int colc = cl ? node_col(gc, ex, ey, ca, cb) : 0;
    const int slot = cl ? ring_slot(DIM, PC, ca, cb) : -1;
    __syncthreads();
    T carry = 0;
    for (int l = 0; l < gf.nz; ++l) {
  #pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int plane = l * PF + k;
        T v = plane < gf.nv - 1 ? rf[(int64_t)plane * gf.ns + colf] : T(0);
        const bool vshared = (k == 0 && l > 0) || (k == PF && l < gf.nz - 1);
        v *= vshared ? inv_mh * T(0.5) : inv_mh;
        s0[k * S::LF + tid] = v;
      }
      __syncthreads();
      if (DIM == 3) {
        // s1[k][b][i] = sum_j J[j][b] s0[k][j*NF + i]   (threads (i, b))
        if (tid < NF * NC) {
          const int ii = tid % NF, b = tid / NF;
  #pragma unroll
          for (int k = 0; k < NF; ++k) {
            T s = 0;
  #pragma unroll
            for (int jj = 0; jj < NF; ++jj) s += sJ[jj * NC + b] * s0[k * S::LF + jj * NF + ii];
            s1[(k * NC + b) * NF + ii] = s;
          }
        }
        __syncthreads();
      }
      if (cl) {
        T w[NF];
  #pragma unroll
        for (int k = 0; k < NF; ++k) {
          T s = 0;
          if (DIM == 3) {
  #pragma unroll
            for (int ii = 0; ii < NF; ++ii) s += sJ[ii * NC + ca] * s1[(k * NC + cb) * NF + ii];
          } else {
  #pragma unroll
            for (int ii = 0; ii < NF; ++ii) s += sJ[ii * NC + ca] * s0[k * S::LF + ii];
          }
          w[k] = s;
        }
        T y[NC];
  #pragma unroll
        for (int c = 0; c < NC; ++c) {
          T s = 0;
  #pragma unroll
          for (int k = 0; k < NF; ++k) s += sJ[k * NC + c] * w[k];
          y[c] = s;
        }
        y[0] += carry;
        carry = y[PC];
  #pragma unroll
        for (int c = 0; c < PC; ++c) {
          const int plane = l * PC + c;
          if (slot < 0) rc[(int64_t)plane * gc.ns + colc] = y[c];
          else ring[((int64_t)plane * gc.n_ecol + ecol) * gc.ring + slot] = y[c];
        }
      }
      __syncthreads();
    }
  }
};

// mode: 0 = restriction (in: fine residual, out: coarse right-hand side),
// 1 = prolongation (out = P in), 2 = prolongation added to out (out += P in).
template <typename T, int NF, int NC>
cudaError_t launch_transfer_t(const Geom& gf, const Geom& gc, const T* J, const T* in, T* out, T* ring, int mode,
                              const int* skip, cudaStream_t s) {
  const unsigned blocks = (unsigned)gf.n_ecol;
  const bool prolong = mode != 0;
  const int add = mode == 2;
  if (gf.dim == 3) {
    if (prolong)
      launch<prolong_kernel<T, NF, NC, 3>>(blocks, XferShape<T, NF, NC, 3>::THREADS, 0, s, gf, gc, J, in, out, add,
                                           skip);
    else
      launch<restrict_kernel<T, NF, NC, 3>>(blocks, XferShape<T, NF, NC, 3>::THREADS, 0, s, gf, gc, J, in, out, ring,
                                            skip);
  } else {
    if (prolong)
      launch<prolong_kernel<T, NF, NC, 2>>(blocks, XferShape<T, NF, NC, 2>::THREADS, 0, s, gf, gc, J, in, out, add,
                                           skip);
    else
      launch<restrict_kernel<T, NF, NC, 2>>(blocks, XferShape<T, NF, NC, 2>::THREADS, 0, s, gf, gc, J, in, out, ring,
                                            skip);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || prolong) return e;
  if (gc.dim == 3) return launch_gather<T, NC, 3>(gc, ring, out, nullptr, skip, s);
  return launch_gather<T, NC, 2>(gc, ring, out, nullptr, skip, s);
}

}  // namespace fnpf

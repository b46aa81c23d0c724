// Vector kernels shared by the CG solves and the Lanczos eigenvalue estimates of
// the p-multigrid smoothers.  Reductions are deterministic: each block writes
// one FP64 partial and the last block of the kernel reduces all partials in a
// fixed order (finish_partials), whatever the order the blocks finish in.
#pragma once

#include <math.h>

#include "fnpf_internal.cuh"
#include "launch.cuh"

namespace fnpf {
namespace vec {

constexpr int NT = kVecThreads;

// Grid-stride loop over [0, n) in a kernel body whose block position is `bk`.
#define FNPF_GRID_LOOP(i, n) \
  for (int64_t i = bk.x * (int64_t)vec::NT + threadIdx.x; i < (n); i += (int64_t)bk.nx * vec::NT)

constexpr int kShared = NT / 32 + 1;   // doubles of shared memory block_sum needs

// Sum over the block, returned to every thread: warp butterflies, then one
// thread adds the warp sums in a fixed order and broadcasts (each FP64 add of
// a full warp occupies the FP64 pipe for many cycles on this GPU, so the last
// stage is not repeated by every thread).
__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < NT / 32; ++k) s += sh[k];
    sh[NT / 32] = s;
  }
  __syncthreads();
  return sh[NT / 32];
}

__device__ inline double reduce_partials(const double* part, int nb, double* sh) {
  double v = 0;
  for (int k = threadIdx.x; k < nb; k += NT) v += __ldcg(part + k);
  return block_sum(v, sh);
}

// Called by every block of a kernel of nb blocks after thread 0 has written
// the block's partials of the given slots: the last block to finish reduces
// each slot's partials (in the same fixed order as reduce_partials) into
// sc->red[slot] and resets the ticket, so consumers read one scalar instead of
// re-reducing.
__device__ inline void finish_partials(CgScalars* sc, const double* part, int nb, int slot0, int nslots,
                                       double* sh) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&sc->ticket[slot0], 1u);
    last = t == (unsigned)nb - 1u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int k = 0; k < nslots; ++k) {
    const double v = reduce_partials(part + (slot0 + k) * nb, nb, sh);
    if (threadIdx.x == 0) sc->red[slot0 + k] = v;
  }
  if (threadIdx.x == 0) sc->ticket[slot0] = 0u;
}

inline int blocks_for(int64_t n) {
  int64_t b = (n + NT - 1) / NT;
  if (b < 1) b = 1;
  if (b > kVecBlocks) b = kVecBlocks;
  return (int)b;
}

template <typename T>
struct invert_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, T* d) {
    FNPF_GRID_LOOP(i, n) d[i] = T(1) / d[i];
  }
};

template <typename T>
struct copy_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, const T* a, T* b, const int* skip) {
    if (skip && *skip) return;
    FNPF_GRID_LOOP(i, n) b[i] = a[i];
  }
};

// part[block] = sum p q (FP64 accumulation); with sc, the last block also
// writes the total to sc->red[slot] (part must then be the slot's array).
template <typename T>
struct dot_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, const int* skip, int64_t n, const T* p, const T* q, double* part, CgScalars* sc,
                             int slot) {
    if (skip && *skip) return;
    __shared__ double sh[kShared];
    double s = 0;
    FNPF_GRID_LOOP(i, n) s += (double)p[i] * (double)q[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[bk.x] = s;
    if (sc) finish_partials(sc, part - slot * bk.nx, bk.nx, slot, 1, sh);
  }
};

// alpha = rz / pq; x += alpha p; r -= alpha q; with dinv: z = dinv r and
// partials rz (slot 1), rr (slot 2); without dinv only rr.  hist (optional)
// records alpha at hist[2 it].
template <typename T>
struct update_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, CgScalars* sc, int it, int64_t n, T* x, T* r, T* z, const T* p, const T* q,
                             const T* dinv, double* part, int nb, double* hist) {
    if (sc->done) return;
    __shared__ double sh[kShared];
    __shared__ double s_alpha;
    const double pq = sc->red[3];   // reduced by the dot kernel's last block
    if (!(pq > 0.0) || !isfinite(pq)) {
      if (bk.x == 0 && threadIdx.x == 0) {
        sc->status = FNPF_EBREAKDOWN;
        sc->done = 1;
      }
      return;
    }
    // one FP64 division per block (FP64 is the slow pipe on this GPU)
    if (threadIdx.x == 0) {
      s_alpha = sc->rz[it & 1] / pq;
      if (hist && bk.x == 0) hist[2 * it] = s_alpha;
    }
    __syncthreads();
    const T alpha = (T)s_alpha;
    double srz = 0, srr = 0;
    FNPF_GRID_LOOP(i, n) {
      x[i] += alpha * p[i];
      const T rn = r[i] - alpha * q[i];
      r[i] = rn;
      srr += (double)rn * (double)rn;
      if (dinv) {
        const T zz = dinv[i] * rn;
        z[i] = zz;
        srz += (double)rn * (double)zz;
      }
    }
    srz = block_sum(srz, sh);
    srr = block_sum(srr, sh);
    if (threadIdx.x == 0) {
      if (dinv) part[1 * nb + bk.x] = srz;
      part[2 * nb + bk.x] = srr;
    }
    if (dinv) finish_partials(sc, part, nb, 1, 2, sh);
    else finish_partials(sc, part, nb, 2, 1, sh);
  }
};

// beta = rz_new / rz; p = z + beta p; block 0 advances the scalars and tests
// convergence.  `it` only selects the parity of the rz double buffer (and the
// hist slot), so a captured pair of iterations with it = 0, 1 can be replayed.
// hist (optional) records beta at hist[2 it + 1].
template <typename T>
struct pupdate_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, CgScalars* sc, int it, int64_t n, const T* z, T* p, const double* part, int nb,
                             double* hist) {
    (void)part;
    (void)nb;
    if (sc->done) return;
    __shared__ double s_beta;
    const double rz_new = sc->red[1];   // reduced by the previous kernels' last blocks
    const double rr = sc->red[2];
    if (threadIdx.x == 0) s_beta = rz_new / sc->rz[it & 1];
    __syncthreads();
    const double beta_d = s_beta;
    const T beta = (T)beta_d;
    FNPF_GRID_LOOP(i, n) p[i] = z[i] + beta * p[i];
    if (bk.x == 0 && threadIdx.x == 0) {
      if (hist) hist[2 * it + 1] = beta_d;
      sc->rz[(it + 1) & 1] = rz_new;
      sc->rr = rr;
      sc->iters += 1;
      if (!isfinite(rr) || !isfinite(rz_new)) {
        sc->status = FNPF_EBREAKDOWN;
        sc->done = 1;
      } else if (rr <= sc->tol2) {
        sc->done = 1;
      }
    }
  }
};

}  // namespace vec
}  // namespace fnpf

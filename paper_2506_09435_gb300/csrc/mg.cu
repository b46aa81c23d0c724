// p-multigrid preconditioner with Chebyshev-Jacobi smoothing for the Laplace
// solve (the paper preconditions CG with algebraic multigrid, Sec. 4 solver
// settings; this is the spectral-element counterpart).
//
// Levels p_0 = p > p_1 = p_0/2 > ... > p_L = 1 on the same element columns.
// Each level is a rediscretisation of the weak Laplace form (Eq. Laplace_weak)
// on the same eta-following geometry: eta and h are interpolated to the
// level's surface nodes and the level's operator rebuilds its geometric
// factors exactly like the fine one.  Transfers: see mg_impl.cuh.
//
// Smoother: Chebyshev iteration on D^-1 A over [lmax / range, lmax] (Saad,
// Iterative Methods, Algorithm 12.1, with the Jacobi diagonal), or the
// fourth-kind Chebyshev smoother on [0, lmax] (see lz_eig_kernel), degree d pre-
// and post-smoothing; the coarsest level gets one Chebyshev sweep of degree
// d_c over a wider interval (on one thread-block cluster when the coarsest
// level is small, see coarse_cheb_kernel).  Every sweep is a fixed polynomial in D^-1 A, so
// the V-cycle is a fixed symmetric operator and plain PCG applies.
// lmax per level comes from a 10-step Jacobi-CG Lanczos run on a fixed
// pseudo-random right-hand side; the largest eigenvalue of the Lanczos
// tridiagonal matrix is found by Sturm multisection on the device and multiplied by a
// safety factor, so the set-up needs no host synchronisation.
#include <math.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mg.cuh"
#include "vec.cuh"

namespace fnpf {

cudaError_t launch_transfer_double(const Geom& gf, const Geom& gc, const double* J, const double* in, double* out,
                                   double* ring, int mode, const int* skip, cudaStream_t s);
cudaError_t launch_transfer_float(const Geom& gf, const Geom& gc, const float* J, const float* in, float* out,
                                  float* ring, int mode, const int* skip, cudaStream_t s);

namespace {

constexpr int kMaxLevels = 5;
constexpr int kLanczos = 10;
constexpr double kSafety = 1.1;

// Cluster solve of the coarsest level: one cluster of kCoarseCluster CTAs
// (the portable maximum) of at most kCoarseThreads threads, kCoarseRows
// unknowns per thread at most.
constexpr int kCoarseCluster = 8;
constexpr int kCoarseThreads = 1024;
constexpr int kCoarseRows = 4;
constexpr int64_t kCoarseMaxRows = (int64_t)kCoarseCluster * kCoarseThreads * kCoarseRows;

inline cudaError_t launch_transfer(const Geom& gf, const Geom& gc, const double* J, const double* in, double* out,
                                   double* ring, int mode, const int* skip, cudaStream_t s) {
  return launch_transfer_double(gf, gc, J, in, out, ring, mode, skip, s);
}
inline cudaError_t launch_transfer(const Geom& gf, const Geom& gc, const float* J, const float* in, float* out,
                                   float* ring, int mode, const int* skip, cudaStream_t s) {
  return launch_transfer_float(gf, gc, J, in, out, ring, mode, skip, s);
}

// ---------------------------------------------------------------------------- kernels

// eta at the level's surface nodes: evaluation of the fine element polynomial.
template <typename T>
struct surface_interp_kernel {
  static constexpr int kThreads = 128;
  __device__ static void run(Blk bk, Geom g0, Geom gl, const T* Js, const T* eta0, T* etal) {
    const int col = bk.x * blockDim.x + threadIdx.x;
    if (col >= gl.ns) return;
    const int ix = col % gl.ncx, iy = col / gl.ncx;
    int ex[2], io[2], ey[2] = {0, 0}, jo[2] = {0, 0};
    line_owners(ix, gl.p, gl.nx, gl.px, ex, io);
    if (gl.dim == 3) line_owners(iy, gl.p, gl.ny, gl.py, ey, jo);
    const int n0 = g0.n;
    T s = 0;
    if (gl.dim == 3) {
      for (int b = 0; b < n0; ++b) {
        T sb = 0;
        for (int a = 0; a < n0; ++a) sb += Js[io[0] * n0 + a] * eta0[node_col(g0, ex[0], ey[0], a, b)];
        s += Js[jo[0] * n0 + b] * sb;
      }
    } else {
      for (int a = 0; a < n0; ++a) s += Js[io[0] * n0 + a] * eta0[node_col(g0, ex[0], 0, a, 0)];
    }
    etal[col] = s;
  }
};

// Deterministic pseudo-random right-hand side in [-0.5, 0.5) (splitmix64 of the index).
template <typename T>
struct random_kernel {
  static constexpr int kThreads = vec::NT;
  __device__ static void run(Blk bk, int64_t n, T* r) {
    FNPF_GRID_LOOP(i, n) {
      uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      r[i] = (T)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
  }
};

// Lanczos start: x = 0, z = dinv r, p = z; partials rz, rr.
template <typename T>
struct lz_init_kernel {
  static constexpr int kThreads = vec::NT;
  __device__ static void run(Blk bk, int64_t n, const T* r, const T* dinv, T* x, T* z, T* p, double* part, int nb) {
    __shared__ double sh[vec::kShared];
    double srz = 0, srr = 0;
    FNPF_GRID_LOOP(i, n) {
      const T zz = dinv[i] * r[i];
      x[i] = T(0);
      z[i] = zz;
      p[i] = zz;
      srz += (double)r[i] * (double)zz;
      srr += (double)r[i] * (double)r[i];
    }
    srz = vec::block_sum(srz, sh);
    srr = vec::block_sum(srr, sh);
    if (threadIdx.x == 0) {
      part[1 * nb + bk.x] = srz;
      part[2 * nb + bk.x] = srr;
    }
  }
};

struct lz_init_finish_kernel {
  static constexpr int kThreads = vec::NT;
  __device__ static void run(Blk bk, CgScalars* sc, const double* part, int nb) {
    __shared__ double sh[vec::kShared];
    const double rz = vec::reduce_partials(part + nb, nb, sh);
    const double rr = vec::reduce_partials(part + 2 * nb, nb, sh);
    if (threadIdx.x == 0) {
      sc->rz[0] = rz;
      sc->rr = rr;
      sc->bb = rr;
      sc->iters = 0;
      sc->tol2 = 1e-28 * rr;
      sc->status = 0;
      sc->done = (rr > 0.0 && isfinite(rr)) ? 0 : 1;
    }
  }
};

// Largest eigenvalue of the Lanczos tridiagonal matrix from the CG coefficients
// (T_jj = 1/a_j + b_{j-1}/a_{j-1}, T_j,j+1 = sqrt(b_j)/a_j), by Sturm counts:
// one warp evaluates 32 points of the bracketing interval per round
// (multisection; 16 rounds shrink it by 33^16, as 80 bisection steps would);
// then lane 0 writes the smoother's step coefficients 1..ncoef-1 for kind 1
// (first-kind Chebyshev on [lmax / range, lmax]) or kind 4 (fourth-kind
// Chebyshev on [0, lmax], no lower bound needed).  Launch with one warp.
struct lz_eig_kernel {
  static constexpr int kThreads = 32;
  __device__ static void run(Blk bk, const CgScalars* sc, const double* hist, double safety, double range, int kind,
                             int ncoef, ChebParams* out) {
    const int lane = threadIdx.x;
    int k = sc->iters < kLanczos ? sc->iters : kLanczos;
    double a[kLanczos], b2[kLanczos];   // diagonal and squared off-diagonal
    double hi = 0.0;
  #pragma unroll
    for (int j = 0; j < kLanczos; ++j) {
      a[j] = 0.0;
      b2[j] = 0.0;
      if (j < k) {
        const double al = hist[2 * j];
        a[j] = 1.0 / al + (j > 0 ? hist[2 * (j - 1) + 1] / hist[2 * (j - 1)] : 0.0);
        const double bj = j + 1 < k ? sqrt(fmax(hist[2 * j + 1], 0.0)) / al : 0.0;
        b2[j] = bj * bj;
      }
    }
  #pragma unroll
    for (int j = 0; j < kLanczos; ++j)   // Gershgorin bound
      if (j < k) hi = fmax(hi, a[j] + sqrt(b2[j]) + (j > 0 ? sqrt(b2[j - 1]) : 0.0));
    double lmax;
    if (k == 0) {
      lmax = out->lmax > 0 ? out->lmax : 2.0;
    } else {
      double lo = 0.0;
      for (int round = 0; round < 16; ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        int below = 0;
        double d = 1.0;
  #pragma unroll
        for (int j = 0; j < kLanczos; ++j) {
          if (j < k) {
            d = a[j] - x - (j > 0 ? b2[j - 1] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0) ++below;
          }
        }
        // first point with every eigenvalue below it brackets lmax from above
        const unsigned all_below = __ballot_sync(0xffffffffu, below == k);
        const double xl = __shfl_up_sync(0xffffffffu, x, 1);
        if (all_below == 0u) {
          lo = __shfl_sync(0xffffffffu, x, 31);
        } else {
          const int jf = __ffs(all_below) - 1;
          const double nlo = jf == 0 ? lo : __shfl_sync(0xffffffffu, xl, jf);
          hi = __shfl_sync(0xffffffffu, x, jf);
          lo = nlo;
        }
      }
      lmax = hi;
    }
    if (lane != 0) return;
    const int nc = ncoef < kMaxChebDegree ? ncoef : kMaxChebDegree;
    out->lmax = safety * lmax;
    out->range = range;
    out->c1[0] = 0.0;
    out->c2[0] = 0.0;
    if (kind == FNPF_CHEB_FOURTH) {
      // Fourth-kind Chebyshev smoother (Lottes, "Optimal polynomial smoothers for
      // multigrid V-cycles", Numer. Linear Algebra Appl. 2023): with rho = lmax,
      // d_0 = 4 / (3 rho) D^-1 r_0 and, for k >= 1,
      // d_k = (2k - 1) / (2k + 3) d_{k-1} + (8k + 4) / ((2k + 3) rho) D^-1 r_k.
      const double rho = out->lmax;
      out->inv_theta = 4.0 / (3.0 * rho);
      for (int m = 1; m < nc; ++m) {
        out->c1[m] = (2.0 * m - 1.0) / (2.0 * m + 3.0);
        out->c2[m] = (8.0 * m + 4.0) / ((2.0 * m + 3.0) * rho);
      }
      return;
    }
    // Chebyshev recurrence on [lmax / range, lmax]: theta = centre, delta = half
    // width, sigma = theta / delta, rho_0 = 1 / sigma, rho_k = 1 / (2 sigma - rho_{k-1})
    const double lm = out->lmax, lmin = lm / range;
    const double theta = 0.5 * (lm + lmin), delta = 0.5 * (lm - lmin), sigma = theta / delta;
    out->inv_theta = 1.0 / theta;
    double rho_old = 1.0 / sigma;
    for (int m = 1; m < nc; ++m) {
      const double rho = 1.0 / (2.0 * sigma - rho_old);
      out->c1[m] = rho * rho_old;
      out->c2[m] = 2.0 * rho / delta;
      rho_old = rho;
    }
  }
};

// Step 0 of a Chebyshev sweep from x = 0 or a given x: (r = b if b given);
// d = dinv r / theta; x = d or x += d.  Steps k >= 1 (r -= A d;
// d = c1[k] d + c2[k] dinv r; x += d) and residuals are fused into the
// gather stage of the operator launches (Epilogue).
template <typename T>
struct cheb_start_kernel {
  static constexpr int kThreads = vec::NT;
  __device__ static void run(Blk bk, int64_t n, const T* b, T* r, const T* dinv, T* d, T* x, const ChebParams* cp,
                             int x_zero, const int* skip) {
    if (skip && *skip) return;
    const T it = (T)cp->inv_theta;
    FNPF_GRID_LOOP(i, n) {
      T rr;
      if (b) {
        rr = b[i];
        r[i] = rr;
      } else {
        rr = r[i];
      }
      const T dd = it * dinv[i] * rr;
      d[i] = dd;
      x[i] = x_zero ? dd : x[i] + dd;
    }
  }
};

// ---------------------------------------------------------------------------- coarsest level on one cluster
//
// At p = 1 every unknown couples only to the 3 x 3 x 3 (3 x 3 in 2D) node block
// around it, so the level operator is a structured stencil.  stencil_kernel
// assembles it from the level's stored metric G (the same quadrature as the
// matrix-free operator: y = sum_e Dhat^T G Dhat x at the element's GLL points);
// coarse_cheb_kernel then runs the whole Chebyshev sweep on it inside one
// thread-block cluster, exchanging directions through distributed shared
// memory with a hardware cluster barrier between steps, instead of one
// operator, gather and update launch per step.

template <int DIM>
struct Stencil {
  static constexpr int slots = DIM == 3 ? 27 : 9;
  // slot of the neighbour at offset (dx, dy, dz), each in -1..1
  __host__ __device__ static constexpr int slot(int dx, int dy, int dz) {
    return DIM == 3 ? (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1) : (dz + 1) * 3 + (dx + 1);
  }
};

// One row per thread: the node's row of A_II, summed over the (up to 8)
// elements that hold it in a fixed order.  coef[slot * NI + row].
template <typename T, int DIM>
struct stencil_kernel {
  static constexpr int kThreads = 128;
  __device__ static void run(Blk bk, Geom g, const T* __restrict__ D, const T* __restrict__ G, T* coef) {
    constexpr int NSL = Stencil<DIM>::slots;
    constexpr int LQ = DIM == 3 ? 4 : 2;       // vertical lines of a p = 1 element column
    constexpr int NJ = DIM == 3 ? 2 : 1;
    const int64_t row = (int64_t)bk.x * blockDim.x + threadIdx.x;
    if (row >= g.NI) return;
    const int k = (int)(row / g.ns), col = (int)(row - (int64_t)k * g.ns);
    const int ix = col % g.ncx, iy = col / g.ncx;
    T acc[NSL];
  #pragma unroll
    for (int q = 0; q < NSL; ++q) acc[q] = T(0);
    int ex[2], ia[2], ey[2] = {0, 0}, jb[2] = {0, 0};
    const int nxo = line_owners(ix, 1, g.nx, g.px, ex, ia);
    const int nyo = DIM == 3 ? line_owners(iy, 1, g.ny, g.py, ey, jb) : 1;
    const int64_t PT = (int64_t)g.nz * g.n_ecol * 2 * LQ;
    for (int c = 0; c < 2; ++c) {           // local vertical index of the node in element layer l
      const int l = k - c;
      if (l < 0 || l >= g.nz) continue;
      for (int yo = 0; yo < nyo; ++yo)
        for (int xo = 0; xo < nxo; ++xo) {
          const int a = ia[xo], b = jb[yo];
          const int ecol = ey[yo] * g.nx + ex[xo];
          for (int qk = 0; qk < 2; ++qk)
            for (int qj = 0; qj < NJ; ++qj)
              for (int qi = 0; qi < 2; ++qi) {
                // reference gradient of the node's basis function at GLL point q
                const T gr = (qj == b && qk == c) ? D[qi * 2 + a] : T(0);
                const T gs = (DIM == 3 && qi == a && qk == c) ? D[qj * 2 + b] : T(0);
                const T gt = (qi == a && qj == b) ? D[qk * 2 + c] : T(0);
                if (gr == T(0) && gs == T(0) && gt == T(0)) continue;
                const int64_t pt = (((int64_t)l * g.n_ecol + ecol) * 2 + qk) * LQ + qj * 2 + qi;
                T vr, vs = T(0), vt;
                if (DIM == 3) {
                  const T grr = G[pt], grs = G[PT + pt], gss = G[2 * PT + pt];
                  const T grt = G[3 * PT + pt], gst = G[4 * PT + pt], gtt = G[5 * PT + pt];
                  vr = grr * gr + grs * gs + grt * gt;
                  vs = grs * gr + gss * gs + gst * gt;
                  vt = grt * gr + gst * gs + gtt * gt;
                } else {
                  const T grr = G[pt], grt = G[PT + pt], gtt = G[2 * PT + pt];
                  vr = grr * gr + grt * gt;
                  vt = grt * gr + gtt * gt;
                }
                for (int c2 = 0; c2 < 2; ++c2)
                  for (int b2 = 0; b2 < NJ; ++b2)
                    for (int a2 = 0; a2 < 2; ++a2) {
                      const T hr = (qj == b2 && qk == c2) ? D[qi * 2 + a2] : T(0);
                      const T hs = (DIM == 3 && qi == a2 && qk == c2) ? D[qj * 2 + b2] : T(0);
                      const T ht = (qi == a2 && qj == b2) ? D[qk * 2 + c2] : T(0);
                      acc[Stencil<DIM>::slot(a2 - a, b2 - b, c2 - c)] += hr * vr + hs * vs + ht * vt;
                    }
              }
        }
    }
    // the plane above the last interior one is the Dirichlet surface: not in A_II
    if (k + 1 > g.nv - 2)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
          if (DIM == 3 || dy == 0) acc[Stencil<DIM>::slot(dx, dy, 1)] = T(0);
  #pragma unroll
    for (int q = 0; q < NSL; ++q) coef[(int64_t)q * g.NI + row] = acc[q];
  }
};

// Neighbour index along one direction (-1 outside a walled boundary).
__device__ __forceinline__ int nbr_index(int i, int o, int n, int periodic) {
  int a = i + o;
  if (a < 0) a = periodic ? a + n : -1;
  else if (a >= n) a = periodic ? a - n : -1;
  return a;
}

// (A_II d)_row from the stencil.  The direction d lives in the shared memory
// of the cluster's CTAs: rank c holds rows [c R, (c + 1) R) (R a power of two)
// in the buffer `cur` of its shared memory, read here through distributed
// shared memory.
template <typename T, int DIM>
__device__ __forceinline__ T stencil_row(const Geom& g, const T* __restrict__ coef,
                                         cooperative_groups::cluster_group& cl, T* cur, int log_r, int row) {
  const int k = row / g.ns, col = row - k * g.ns;
  const int iy = col / g.ncx, ix = col - iy * g.ncx;
  int xs[3], ys[3] = {-1, 0, -1};
#pragma unroll
  for (int o = -1; o <= 1; ++o) {
    xs[o + 1] = nbr_index(ix, o, g.ncx, g.px);
    if (DIM == 3) ys[o + 1] = nbr_index(iy, o, g.ncy, g.py);
  }
  const int rmask = (1 << log_r) - 1;
  T w = T(0);
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    const int kk = k + dz;
    if (kk < 0 || kk > g.nv - 2) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      if (DIM == 2 && dy != 0) continue;
      const int yy = ys[dy + 1];
      if (yy < 0) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = xs[dx + 1];
        if (xx < 0) continue;
        const T cv = coef[(int64_t)Stencil<DIM>::slot(dx, dy, dz) * g.NI + row];
        const int nr = kk * g.ns + yy * g.ncx + xx;
        const T* owner = cl.map_shared_rank(cur, (unsigned)(nr >> log_r));
        w += cv * owner[nr & rmask];
      }
    }
  }
  return w;
}

// The coarsest level's Chebyshev sweep from x = 0 (the recurrence of
// cheb_sweep: cheb_start_kernel, then EP_CHEB gather-updates) in one launch of
// one cluster.  CTA rank c owns rows [c R, (c + 1) R); each thread keeps its
// rows' r, x and direction in registers and publishes the direction in its
// CTA's shared memory (double buffer [2][R]), which the other CTAs read through
// distributed shared memory after the step's cluster barrier.  A last barrier
// keeps every CTA resident until no other CTA can read its shared memory.
// Uniform control flow: every thread reaches every barrier.
template <typename T, int DIM>
struct coarse_cheb_kernel {
  static constexpr int kThreads = kCoarseThreads;
  static constexpr int kCluster = kCoarseCluster;
  static constexpr bool kFlexBlock = true;   // rows are assigned by R, any block of at least the mesh's threads
  __device__ static void run(Blk bk, Geom g, const T* __restrict__ coef, const T* __restrict__ dinv,
                             const T* __restrict__ b, T* x, int log_r, const ChebParams* cp, int degree,
                             const int* skip) {
    if (skip && *skip) return;   // the same value for every CTA of the cluster
    extern __shared__ __align__(16) unsigned char coarse_smem[];
    T* sdir = reinterpret_cast<T*>(coarse_smem);
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    const int R = 1 << log_r;
    const int n = (int)g.NI;
    const int row0 = (int)cl.block_rank() * R;
    T r[kCoarseRows], xv[kCoarseRows], dv[kCoarseRows];
    const T it = (T)cp->inv_theta;
  #pragma unroll
    for (int m = 0; m < kCoarseRows; ++m) {
      const int lr = threadIdx.x + m * blockDim.x, row = row0 + lr;
      r[m] = xv[m] = dv[m] = T(0);
      if (lr < R && row < n) {
        r[m] = b[row];
        dv[m] = it * dinv[row] * r[m];
        xv[m] = dv[m];
        sdir[lr] = dv[m];
      }
    }
    for (int k = 1; k < degree; ++k) {
      cl.sync();
      T* cur = sdir + ((k - 1) & 1) * R;
      T* nxt = sdir + (k & 1) * R;
      const T c1 = (T)cp->c1[k], c2 = (T)cp->c2[k];
  #pragma unroll
      for (int m = 0; m < kCoarseRows; ++m) {
        const int lr = threadIdx.x + m * blockDim.x, row = row0 + lr;
        if (lr < R && row < n) {
          r[m] -= stencil_row<T, DIM>(g, coef, cl, cur, log_r, row);
          dv[m] = c1 * dv[m] + c2 * dinv[row] * r[m];
          xv[m] += dv[m];
          nxt[lr] = dv[m];
        }
      }
    }
    cl.sync();
  #pragma unroll
    for (int m = 0; m < kCoarseRows; ++m) {
      const int lr = threadIdx.x + m * blockDim.x, row = row0 + lr;
      if (lr < R && row < n) x[row] = xv[m];
    }
  }
};

template <typename T>
cudaError_t launch_stencil(const Geom& g, const T* D, const T* G, T* coef, cudaStream_t s) {
  const unsigned nb = (unsigned)((g.NI + 127) / 128);
  if (g.dim == 3) launch<stencil_kernel<T, 3>>(nb, 128, 0, s, g, D, G, coef);
  else launch<stencil_kernel<T, 2>>(nb, 128, 0, s, g, D, G, coef);
  return cudaGetLastError();
}

// Rows per CTA: the power of two R >= NI / kCoarseCluster; CTAs only as large
// as that needs (one row per thread up to kCoarseThreads threads, then up to
// kCoarseRows rows per thread), so that small coarse levels, e.g. of the tanks
// of an ensemble running side by side, leave the rest of their SMs to other
// kernels.  Shared memory: 2 R values per CTA.
int coarse_log_rows(int64_t NI) {
  int log_r = 0;
  while (((int64_t)kCoarseCluster << log_r) < NI) ++log_r;
  return log_r;
}

template <typename T>
cudaError_t launch_coarse_cheb(const Geom& g, const T* coef, const T* dinv, const T* b, T* x, const ChebParams* cp,
                               int degree, const int* skip, cudaStream_t s) {
  const int log_r = coarse_log_rows(g.NI);
  const int R = 1 << log_r;
  const int threads = std::min(kCoarseThreads, std::max(32, (R + 31) / 32 * 32));
  const size_t smem = 2 * (size_t)R * sizeof(T);
  if (g.dim == 3)
    return launch<coarse_cheb_kernel<T, 3>>(kCoarseCluster, threads, smem, s, g, coef, dinv, b, x, log_r, cp, degree,
                                            skip);
  return launch<coarse_cheb_kernel<T, 2>>(kCoarseCluster, threads, smem, s, g, coef, dinv, b, x, log_r, cp, degree,
                                          skip);
}

// Whether one cluster of the coarse kernel, with its largest shared-memory
// footprint, can be resident on this device (also raises the kernels'
// dynamic shared-memory limit on the current device, once per device).
bool cluster_launch_ok() {
  constexpr int kMaxSmem = 2 * (kCoarseMaxRows / kCoarseCluster) * (int)sizeof(double);
  static std::atomic<uint64_t> a64_3{0}, a64_2{0}, a32_3{0}, a32_2{0};
  if (smem_optin(kernel_one<coarse_cheb_kernel<double, 3>>(), kMaxSmem, &a64_3) != cudaSuccess ||
      smem_optin(kernel_one<coarse_cheb_kernel<double, 2>>(), kMaxSmem, &a64_2) != cudaSuccess ||
      smem_optin(kernel_one<coarse_cheb_kernel<float, 3>>(), kMaxSmem, &a32_3) != cudaSuccess ||
      smem_optin(kernel_one<coarse_cheb_kernel<float, 2>>(), kMaxSmem, &a32_2) != cudaSuccess)
    return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCoarseCluster);
  cfg.blockDim = dim3(kCoarseThreads);
  cfg.dynamicSmemBytes = kMaxSmem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCoarseCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, (const void*)kernel_one<coarse_cheb_kernel<double, 3>>(), &cfg);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return nc > 0;
}

// ---------------------------------------------------------------------------- host helpers

int next_p(int p, int schedule) {
  if (schedule == FNPF_MG_TWO_LEVEL) return 1;
  if (schedule == FNPF_MG_STEP2) return p - 2 > 1 ? p - 2 : 1;
  return p / 2 > 1 ? p / 2 : 1;
}

std::vector<double> interp_matrix(const std::vector<double>& xf, const std::vector<double>& xc) {
  const int nf = (int)xf.size(), nc = (int)xc.size();
  std::vector<double> J(nf * nc);
  for (int i = 0; i < nf; ++i)
    for (int c = 0; c < nc; ++c) {
      double v = 1.0;
      for (int m = 0; m < nc; ++m)
        if (m != c) v *= (xf[i] - xc[m]) / (xc[c] - xc[m]);
      J[i * nc + c] = v;
    }
  return J;
}

Geom level_geom(const Geom& g0, int p) {
  Geom g = g0;
  g.p = p;
  g.n = p + 1;
  g.ncx = p * g.nx + (g.px ? 0 : 1);
  g.ncy = g.dim == 3 ? p * g.ny + (g.py ? 0 : 1) : 1;
  g.ns = g.ncx * g.ncy;
  g.nv = p * g.nz + 1;
  g.lines = g.dim == 3 ? g.n * g.n : g.n;
  g.ring = g.dim == 3 ? 4 * p : 2;
  g.N = (int64_t)g.nv * g.ns;
  g.NI = (int64_t)(g.nv - 1) * g.ns;
  return g;
}

// Values of a surface field of level 0 at the surface nodes of level l (host).
std::vector<double> host_surface_interp(const Geom& g0, const Geom& gl, const std::vector<double>& Js,
                                        const double* f0) {
  std::vector<double> out(gl.ns);
  const int n0 = g0.n;
  for (int col = 0; col < gl.ns; ++col) {
    const int ix = col % gl.ncx, iy = col / gl.ncx;
    int ex[2], io[2], ey[2] = {0, 0}, jo[2] = {0, 0};
    line_owners(ix, gl.p, gl.nx, gl.px, ex, io);
    if (gl.dim == 3) line_owners(iy, gl.p, gl.ny, gl.py, ey, jo);
    double s = 0;
    if (gl.dim == 3) {
      for (int b = 0; b < n0; ++b) {
        double sb = 0;
        for (int a = 0; a < n0; ++a) sb += Js[io[0] * n0 + a] * f0[node_col(g0, ex[0], ey[0], a, b)];
        s += Js[jo[0] * n0 + b] * sb;
      }
    } else {
      for (int a = 0; a < n0; ++a) s += Js[io[0] * n0 + a] * f0[node_col(g0, ex[0], 0, a, 0)];
    }
    out[col] = s;
  }
  return out;
}

}  // namespace

struct Mg {
  int L = 0;
  Geom g[kMaxLevels];
  MgLevelBufs<double> b64[kMaxLevels];
  MgLevelBufs<float> b32[kMaxLevels];
  ChebParams* cheb64 = nullptr;   // [L]
  ChebParams* cheb32 = nullptr;
  double* hist = nullptr;         // [L][2 * kLanczos]
  CgScalars* sc = nullptr;        // [L] Lanczos scalars
  double* part = nullptr;         // [4 * kVecBlocks]
  bool fusable = false;           // the coarsest level fits the cluster kernel
  int schedule = FNPF_MG_HALVE;
  int coarse_mode = FNPF_COARSE_CLUSTER;
  int cheb_kind = FNPF_CHEB_FIRST;
  double cheb_range = 160.0;
  std::vector<void*> allocs;

  bool fused() const { return fusable && coarse_mode == FNPF_COARSE_CLUSTER; }

  template <typename T>
  MgLevelBufs<T>* bufs();
  template <typename T>
  ChebParams* cheb();
};
template <>
MgLevelBufs<double>* Mg::bufs<double>() { return b64; }
template <>
MgLevelBufs<float>* Mg::bufs<float>() { return b32; }
template <>
ChebParams* Mg::cheb<double>() { return cheb64; }
template <>
ChebParams* Mg::cheb<float>() { return cheb32; }

void mg_destroy(Mg* mg) {
  if (!mg) return;
  for (void* p : mg->allocs) cudaFree(p);
  delete mg;
}

int mg_levels(const Mg* mg) { return mg ? mg->L : 0; }
int mg_schedule(const Mg* mg) { return mg ? mg->schedule : FNPF_MG_HALVE; }
void mg_set_coarse(Mg* mg, int mode) {
  if (mg) mg->coarse_mode = mode;
}
void mg_set_kind(Mg* mg, int kind, double range) {
  if (!mg) return;
  mg->cheb_kind = kind;
  mg->cheb_range = range;
}
bool mg_coarse_fused(const Mg* mg) { return mg && mg->fused(); }

Mg* mg_create(const Geom& g0, const std::vector<double>& h0, const std::vector<double>& X0,
              const std::vector<double>& Y0, bool iso, double Lx, double Ly, int schedule, std::string* err) {
  Mg* mg = new Mg();
  int p = g0.p;
  mg->schedule = schedule;
  mg->g[0] = g0;
  mg->L = 1;
  while (p > 1 && mg->L < kMaxLevels) {
    p = next_p(p, schedule);
    mg->g[mg->L] = level_geom(g0, p);
    ++mg->L;
  }
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(ptr, bytes < 8 ? 8 : bytes);
    if (e == cudaSuccess) mg->allocs.push_back(*ptr);
  };
  auto upload = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  std::vector<double> xi0(g0.n), w0(g0.n), D0(g0.n * g0.n);
  gll_tables(g0.p, xi0.data(), w0.data(), D0.data());
  std::vector<double> xprev = xi0;
  for (int l = 0; l < mg->L; ++l) {
    const Geom& g = mg->g[l];
    MgLevelBufs<double>& B = mg->b64[l];
    MgLevelBufs<float>& F = mg->b32[l];
    double** dv[] = {&B.dinv, &B.X, &B.B, &B.R, &B.Dd, &B.W, &B.P};
    for (double** v : dv) alloc((void**)v, g.NI * sizeof(double));
    float** fv[] = {&F.dinv, &F.X, &F.B, &F.R, &F.Dd, &F.W, &F.P};
    for (float** v : fv) alloc((void**)v, g.NI * sizeof(float));
    if (l == 0) continue;
    std::vector<double> xi(g.n), w(g.n), D(g.n * g.n);
    gll_tables(g.p, xi.data(), w.data(), D.data());
    const std::vector<double> J = interp_matrix(xprev, xi);     // level l-1 nodes x level l
    const std::vector<double> Js = interp_matrix(xi, xi0);      // level l nodes x level-0 nodes
    xprev = xi;
    std::vector<double> hl = host_surface_interp(g0, g, Js, h0.data());
    std::vector<double> Xl, Yl;
    if (iso) {
      Xl = host_surface_interp(g0, g, Js, X0.data());
      Yl = g.dim == 3 ? host_surface_interp(g0, g, Js, Y0.data()) : std::vector<double>(g.ns, 0.0);
    }
    std::vector<double> hm, mass, xs, ys;
    if (!build_hmetric(g, xi.data(), w.data(), D.data(), iso, Lx, Ly, iso ? Xl.data() : nullptr,
                       iso ? Yl.data() : nullptr, &hm, &mass, &xs, &ys)) {
      *err = "degenerate horizontal Jacobian on a multigrid level";
      mg_destroy(mg);
      return nullptr;
    }
    for (double hv : hl)
      if (!(hv > 0)) {
        *err = "interpolated depth not positive on a multigrid level";
        mg_destroy(mg);
        return nullptr;
      }
    // double tables
    double *dD, *dxi, *dw, *dhm, *dh, *dJ, *dJs, *deta;
    alloc((void**)&dD, D.size() * 8);
    alloc((void**)&dxi, xi.size() * 8);
    alloc((void**)&dw, w.size() * 8);
    alloc((void**)&dhm, hm.size() * 8);
    alloc((void**)&dh, hl.size() * 8);
    alloc((void**)&dJ, J.size() * 8);
    alloc((void**)&dJs, Js.size() * 8);
    alloc((void**)&deta, g.ns * 8);
    upload(dD, D.data(), D.size() * 8);
    upload(dxi, xi.data(), xi.size() * 8);
    upload(dw, w.data(), w.size() * 8);
    upload(dhm, hm.data(), hm.size() * 8);
    upload(dh, hl.data(), hl.size() * 8);
    upload(dJ, J.data(), J.size() * 8);
    upload(dJs, Js.data(), Js.size() * 8);
    B.t = Tables<double>{dD, dxi, dw, dhm, dh, nullptr};
    alloc((void**)&B.G, (size_t)(g.dim == 3 ? 6 : 3) * geom_points(g) * sizeof(double));
    B.J = dJ;
    B.Js = dJs;
    B.eta = deta;
    // float tables
    auto f32 = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
    const std::vector<float> fD = f32(D), fxi = f32(xi), fw = f32(w), fhm = f32(hm), fh = f32(hl), fJ = f32(J),
                             fJs = f32(Js);
    float *sD, *sxi, *sw, *shm, *sh, *sJ, *sJs, *seta;
    alloc((void**)&sD, fD.size() * 4);
    alloc((void**)&sxi, fxi.size() * 4);
    alloc((void**)&sw, fw.size() * 4);
    alloc((void**)&shm, fhm.size() * 4);
    alloc((void**)&sh, fh.size() * 4);
    alloc((void**)&sJ, fJ.size() * 4);
    alloc((void**)&sJs, fJs.size() * 4);
    alloc((void**)&seta, g.ns * 4);
    upload(sD, fD.data(), fD.size() * 4);
    upload(sxi, fxi.data(), fxi.size() * 4);
    upload(sw, fw.data(), fw.size() * 4);
    upload(shm, fhm.data(), fhm.size() * 4);
    upload(sh, fh.data(), fh.size() * 4);
    upload(sJ, fJ.data(), fJ.size() * 4);
    upload(sJs, fJs.data(), fJs.size() * 4);
    F.t = Tables<float>{sD, sxi, sw, shm, sh, nullptr};
    F.J = sJ;
    F.Js = sJs;
    F.eta = seta;
  }
  // coarsest level on one cluster: stencil, direction buffers, FP32 metric
  const Geom& gc = mg->g[mg->L - 1];
  mg->fusable = mg->L >= 2 && gc.p == 1 && gc.NI <= kCoarseMaxRows && cluster_launch_ok();
  if (mg->fusable) {
    MgLevelBufs<double>& B = mg->b64[mg->L - 1];
    MgLevelBufs<float>& F = mg->b32[mg->L - 1];
    const int nsl = gc.dim == 3 ? Stencil<3>::slots : Stencil<2>::slots;
    alloc((void**)&B.coef, (size_t)nsl * gc.NI * sizeof(double));
    alloc((void**)&F.coef, (size_t)nsl * gc.NI * sizeof(float));
    alloc((void**)&F.G, (size_t)(gc.dim == 3 ? 6 : 3) * geom_points(gc) * sizeof(float));
  }
  alloc((void**)&mg->cheb64, mg->L * sizeof(ChebParams));
  alloc((void**)&mg->cheb32, mg->L * sizeof(ChebParams));
  alloc((void**)&mg->hist, mg->L * 2 * kLanczos * sizeof(double));
  alloc((void**)&mg->sc, mg->L * sizeof(CgScalars));
  alloc((void**)&mg->part, 4 * kVecBlocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(mg->cheb64, 0, mg->L * sizeof(ChebParams));
  if (e == cudaSuccess) e = cudaMemset(mg->sc, 0, mg->L * sizeof(CgScalars));   // reduction tickets start at 0
  if (e == cudaSuccess) e = cudaMemset(mg->cheb32, 0, mg->L * sizeof(ChebParams));
  if (e != cudaSuccess) {
    *err = std::string("multigrid set-up failed: ") + cudaGetErrorString(e);
    mg_destroy(mg);
    return nullptr;
  }
  return mg;
}

namespace {

template <typename T>
Tables<T> level_tables(Mg* mg, int l, const Tables<T>& t0) {
  return l == 0 ? t0 : mg->bufs<T>()[l].t;
}

template <typename T>
const T* level_eta(Mg* mg, int l, const T* eta0) {
  return l == 0 ? eta0 : mg->bufs<T>()[l].eta;
}

// Operator of level l (level 0 reads the stored metric when given).
template <typename T>
cudaError_t level_apply(const Geom& g, const Tables<T>& t, const T* eta, const T* G, const T* x, T* y, T* ring,
                        int variant, const int* skip, cudaStream_t s, const Epilogue<T>* ep = nullptr) {
  if (G) return launch_apply_g<T>(g, t, G, x, nullptr, y, nullptr, ring, variant, s, skip, ep);
  return launch_apply<T>(g, t, eta, x, nullptr, y, nullptr, ring, variant, s, skip, ep);
}

// One Chebyshev sweep of `degree` steps on level l solving A x = b.
// x_zero: start from x = 0 (r = b, no operator application needed);
// otherwise r = b - A x first.  With `final_residual` the residual of the
// result is left in R.
template <typename T>
cudaError_t cheb_sweep(Mg* mg, int l, const Tables<T>& t0, const T* eta0, const T* G0, const T* b, T* x, int degree,
                       bool x_zero, bool final_residual, T* ring, int variant, const int* skip, cudaStream_t s,
                       int64_t* nl) {
  const Geom& g = mg->g[l];
  MgLevelBufs<T>& L = mg->bufs<T>()[l];
  const T* G = l == 0 ? G0 : (G0 ? L.G : nullptr);
  const Tables<T> t = level_tables(mg, l, t0);
  const T* eta = level_eta(mg, l, eta0);
  const ChebParams* cp = mg->cheb<T>() + l;
  variant = l == 0 ? variant : 1;   // the autotuned shape is for the finest order
  const int nb = vec::blocks_for(g.NI);
  cudaError_t e;
  // the residual and Chebyshev updates ride on the operator's gather stage
  // (Epilogue), so each step is one element kernel plus one gather-update
  Epilogue<T> ep;
  ep.r = L.R;
  ep.dinv = L.dinv;
  ep.d = L.Dd;
  ep.x = x;
  if (x_zero) {
    launch<cheb_start_kernel<T>>(nb, vec::NT, 0, s, g.NI, b, L.R, L.dinv, L.Dd, x, cp, 1, skip);
    *nl += 1;
  } else {
    // r = b - A x; d = dinv r / theta; x += d (x is the operator input)
    ep.op = EP_RES_START;
    ep.b = b;
    ep.c2 = &cp->inv_theta;
    if ((e = level_apply<T>(g, t, eta, G, x, L.W, ring, variant, skip, s, &ep)) != cudaSuccess) return e;
    *nl += 2;
  }
  for (int k = 1; k < degree; ++k) {
    // r -= A d; d = c1 d + c2 dinv r; x += d (d is the operator input)
    ep.op = EP_CHEB;
    ep.b = nullptr;
    ep.c1 = &cp->c1[k];
    ep.c2 = &cp->c2[k];
    if ((e = level_apply<T>(g, t, eta, G, L.Dd, L.W, ring, variant, skip, s, &ep)) != cudaSuccess) return e;
    *nl += 2;
  }
  if (final_residual) {
    ep.op = EP_RES;
    ep.b = nullptr;
    if ((e = level_apply<T>(g, t, eta, G, L.Dd, L.W, ring, variant, skip, s, &ep)) != cudaSuccess) return e;
    *nl += 2;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t vcycle(Mg* mg, int l, const Tables<T>& t0, const T* eta0, const T* G0, const T* b, T* x, T* ring,
                   int variant, int degree, int coarse_degree, const int* skip, cudaStream_t s, int64_t* nl) {
  cudaError_t e;
  if (l == mg->L - 1) {
    if (mg->fused()) {
      MgLevelBufs<T>& C = mg->bufs<T>()[l];
      *nl += 1;
      return launch_coarse_cheb<T>(mg->g[l], C.coef, C.dinv, b, x, mg->cheb<T>() + l, coarse_degree, skip, s);
    }
    return cheb_sweep<T>(mg, l, t0, eta0, G0, b, x, coarse_degree, true, false, ring, variant, skip, s, nl);
  }
  MgLevelBufs<T>* Lv = mg->bufs<T>();
  if ((e = cheb_sweep<T>(mg, l, t0, eta0, G0, b, x, degree, true, true, ring, variant, skip, s, nl)) != cudaSuccess)
    return e;
  // restrict the residual, solve on the next level, prolong and add
  if ((e = launch_transfer(mg->g[l], mg->g[l + 1], Lv[l + 1].J, Lv[l].R, Lv[l + 1].B, ring, 0, skip, s)) !=
      cudaSuccess)
    return e;
  if ((e = vcycle<T>(mg, l + 1, t0, eta0, G0, Lv[l + 1].B, Lv[l + 1].X, ring, variant, degree, coarse_degree, skip,
                     s, nl)) != cudaSuccess)
    return e;
  if ((e = launch_transfer(mg->g[l], mg->g[l + 1], Lv[l + 1].J, Lv[l + 1].X, x, ring, 2, skip, s)) != cudaSuccess)
    return e;
  *nl += 3;
  return cheb_sweep<T>(mg, l, t0, eta0, G0, b, x, degree, false, false, ring, variant, skip, s, nl);
}

}  // namespace

template <typename T>
cudaError_t mg_prepare(Mg* mg, const Tables<T>& t0, const T* eta0, const T* G0, T* ring, int variant,
                       int cheb_degree, int coarse_degree, bool estimate, cudaStream_t s) {
  cudaError_t e;
  MgLevelBufs<T>* Lv = mg->bufs<T>();
  for (int l = 1; l < mg->L; ++l) {
    const Geom& gl = mg->g[l];
    launch<surface_interp_kernel<T>>((gl.ns + 127) / 128, 128, 0, s, mg->g[0], gl, Lv[l].Js, eta0, Lv[l].eta);
  }
  for (int l = 0; l < mg->L; ++l) {
    const Geom& g = mg->g[l];
    const Tables<T> t = level_tables(mg, l, t0);
    const T* eta = level_eta(mg, l, eta0);
    MgLevelBufs<T>& L = Lv[l];
    const int nb = vec::blocks_for(g.NI);
    const int lv = l == 0 ? variant : 1;
    if ((e = launch_diag<T>(g, t, eta, L.dinv, nullptr, ring, s)) != cudaSuccess) return e;
    launch<vec::invert_kernel<T>>(nb, vec::NT, 0, s, g.NI, L.dinv);
    const bool coarse_fused = l == mg->L - 1 && mg->fused();
    if (l > 0 && L.G && (G0 || coarse_fused))
      if ((e = launch_geom<T>(g, t, eta, L.G, s)) != cudaSuccess) return e;
    if (coarse_fused)
      if ((e = launch_stencil<T>(g, t.D, L.G, L.coef, s)) != cudaSuccess) return e;
    if (!estimate) continue;
    const T* Gl = l == 0 ? G0 : (G0 ? L.G : nullptr);
    // Lanczos through Jacobi-CG: x = X, r = R, z = Dd, p = P, q = W
    launch<random_kernel<T>>(nb, vec::NT, 0, s, g.NI, L.R);
    CgScalars* sc = mg->sc + l;
    double* hist = mg->hist + 2 * kLanczos * l;
    launch<lz_init_kernel<T>>(nb, vec::NT, 0, s, g.NI, L.R, L.dinv, L.X, L.Dd, L.P, mg->part, nb);
    launch<lz_init_finish_kernel>(1, vec::NT, 0, s, sc, mg->part, nb);
    for (int it = 0; it < kLanczos; ++it) {
      if ((e = level_apply<T>(g, t, eta, Gl, L.P, L.W, ring, lv, &sc->done, s)) != cudaSuccess) return e;
      launch<vec::dot_kernel<T>>(nb, vec::NT, 0, s, &sc->done, g.NI, L.P, L.W, mg->part + 3 * nb, sc, 3);
      launch<vec::update_kernel<T>>(nb, vec::NT, 0, s, sc, it, g.NI, L.X, L.R, L.Dd, L.P, L.W, L.dinv, mg->part, nb,
                                                   hist);
      launch<vec::pupdate_kernel<T>>(nb, vec::NT, 0, s, sc, it, g.NI, L.Dd, L.P, mg->part, nb, hist);
    }
    const double range =
        l == mg->L - 1 ? fmax(mg->cheb_range, 0.25 * coarse_degree * coarse_degree) : mg->cheb_range;
    const int ncoef = l == mg->L - 1 ? coarse_degree : cheb_degree;
    launch<lz_eig_kernel>(1, 32, 0, s, sc, hist, kSafety, range, mg->cheb_kind, ncoef, mg->cheb<T>() + l);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t mg_apply(Mg* mg, const Tables<T>& t0, const T* eta0, const T* G0, const T* r, T* z, T* ring,
                     int variant, int cheb_degree, int coarse_degree, const int* skip, cudaStream_t s,
                     int64_t* launches) {
  return vcycle<T>(mg, 0, t0, eta0, G0, r, z, ring, variant, cheb_degree, coarse_degree, skip, s, launches);
}

template cudaError_t mg_prepare<double>(Mg*, const Tables<double>&, const double*, const double*, double*, int, int,
                                        int, bool, cudaStream_t);
template cudaError_t mg_prepare<float>(Mg*, const Tables<float>&, const float*, const float*, float*, int, int, int,
                                       bool, cudaStream_t);
template cudaError_t mg_apply<double>(Mg*, const Tables<double>&, const double*, const double*, const double*,
                                      double*, double*, int, int, int, const int*, cudaStream_t, int64_t*);
template cudaError_t mg_apply<float>(Mg*, const Tables<float>&, const float*, const float*, const float*, float*,
                                     float*, int, int, int, const int*, cudaStream_t, int64_t*);

}  // namespace fnpf

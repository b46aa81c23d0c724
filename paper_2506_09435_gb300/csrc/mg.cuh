// p-multigrid preconditioner: declarations shared by mg.cu and cg.cu.
#pragma once

#include <vector>

#include "fnpf_internal.cuh"

namespace fnpf {

constexpr int kMaxChebDegree = 64;

// Chebyshev interval of one level, written on the device by the Lanczos
// eigenvalue kernel: smoothing targets [lmax / range, lmax].
struct ChebParams {
  double lmax;
  double range;
  // step coefficients precomputed by one thread: step 0 uses d = inv_theta dinv r,
  // step k >= 1 uses d = c1[k] d + c2[k] dinv r
  double inv_theta;
  double c1[kMaxChebDegree];
  double c2[kMaxChebDegree];
};

// Device buffers of one level in precision T.  Level 0 is the mesh itself: its
// X and B are supplied by the caller (the CG vectors z and r).
template <typename T>
struct MgLevelBufs {
  Tables<T> t;          // GLL tables, horizontal metric, depth of this level
  T* eta = nullptr;     // [ns] eta interpolated to this level's surface nodes
  T* dinv = nullptr;    // [NI] inverse Jacobi diagonal
  T* X = nullptr;       // [NI] correction (levels >= 1)
  T* B = nullptr;       // [NI] right-hand side (levels >= 1)
  T* R = nullptr;       // [NI] residual
  T* Dd = nullptr;      // [NI] Chebyshev direction
  T* W = nullptr;       // [NI] operator output
  T* P = nullptr;       // [NI] CG direction of the Lanczos estimate
  T* G = nullptr;         // stored metric of this level (FP64 solves, levels >= 1; the
                          // coarsest level in both precisions when it is solved by the cluster kernel)
  T* coef = nullptr;      // coarsest level: assembled 27-point (9 in 2D) stencil, [slot][NI]
  const T* J = nullptr;   // [n_{l-1} x n_l] prolongation from this level to level l-1 (levels >= 1)
  const T* Js = nullptr;  // [n_l x n_0] surface interpolation from level 0 (levels >= 1)
};

struct Mg;   // opaque; owned by the mesh

// Builds the hierarchy p -> p/2 -> ... -> 1 for the mesh sizes g0 (host work and
// device allocations).  Returns nullptr and sets *err on failure.
Mg* mg_create(const Geom& g0, const std::vector<double>& h0, const std::vector<double>& X0,
              const std::vector<double>& Y0, bool iso, double Lx, double Ly, int schedule, std::string* err);
int mg_schedule(const Mg* mg);
void mg_destroy(Mg* mg);
int mg_levels(const Mg* mg);
// Coarse solver of the next set-ups and V-cycles: FNPF_COARSE_CLUSTER runs the
// coarsest level's Chebyshev sweep as one thread-block-cluster kernel on an
// assembled stencil (used when the level fits, see mg.cu), FNPF_COARSE_LAUNCHES
// as one operator launch per step.
void mg_set_coarse(Mg* mg, int mode);
// Polynomial of the Chebyshev smoothers of the next set-ups: FNPF_CHEB_FIRST
// on [lmax / range, lmax] or FNPF_CHEB_FOURTH on [0, lmax].
void mg_set_kind(Mg* mg, int kind, double range);
// True when the coarsest level is solved by the cluster kernel.
bool mg_coarse_fused(const Mg* mg);

// Per-solve set-up in precision T: eta at every level, Jacobi diagonals, the
// stored metric of the coarser levels when G0 is given, and (when `estimate`)
// the Chebyshev intervals from a short Lanczos run per level (all on the
// device, no host synchronisation).  eta0 is the fine eta in precision T, t0
// the fine tables; G0, if non-null, is the stored metric of level 0 (the
// operator there reads it, and the coarser levels then store theirs too).
template <typename T>
cudaError_t mg_prepare(Mg* mg, const Tables<T>& t0, const T* eta0, const T* G0, T* ring, int variant,
                       int cheb_degree, int coarse_degree, bool estimate, cudaStream_t s);

// z = M r (one symmetric V-cycle); kernels exit at once when *skip != 0.
template <typename T>
cudaError_t mg_apply(Mg* mg, const Tables<T>& t0, const T* eta0, const T* G0, const T* r, T* z, T* ring,
                     int variant, int cheb_degree, int coarse_degree, const int* skip, cudaStream_t s,
                     int64_t* launches);

}  // namespace fnpf

// Internal declarations of the FNPF-SEM CUDA library (not part of the ABI).
//
// Layout reminder (see include/fnpf.h): volume index = k * ns + col,
// col = iy * ncx + ix; the surface plane is k = nv - 1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "fnpf.h"
#include "launch.cuh"

namespace fnpf {

constexpr int kMaxP = 8;
constexpr int kMaxN = kMaxP + 1;
constexpr int kVecBlocks = 608;      // 4 x 152 SMs: grid of the vector kernels
constexpr int kVecThreads = 256;
constexpr int kMaxProjection = 8;    // most previous solutions in the initial-guess projection

// Mesh sizes, passed by value to every kernel.
struct Geom {
  int dim, nx, ny, nz, p, n;
  int px, py;                // periodic flags
  int ncx, ncy;              // node columns per direction
  int ns, nv;                // surface columns, nodes per column
  int n_ecol;                // element columns nx * ny
  int lines;                 // vertical lines per element column: n*n (3D) or n (2D)
  int ring;                  // ring lines per element column: 4p (3D) or 2 (2D)
  int64_t N, NI;             // volume DOF, interior (unknown) DOF
  double g;
};

// Device-resident tables of one mesh in precision T.
template <typename T>
struct Tables {
  const T* D;      // [n*n], D[i*n + a] = l_a'(xi_i)
  const T* xi;     // [n]
  const T* w;      // [n]
  const T* hm;     // [5][n_ecol * lines]: r_x, r_y, s_x, s_y, w_i w_j |J2|
  const T* h;      // [ns] depth
  const T* minv;   // [ns] inverse lumped surface mass
};

// Scalars of one CG solve, device-resident.  rz is double-buffered by the
// host-known iteration parity so that no kernel reads a scalar another block
// of the same kernel writes.
struct CgScalars {
  double rz[2];
  double rr;
  double bb;
  double tol2;
  double pq;
  int done;
  int iters;
  int status;
  int outer;     // defect-correction steps of a mixed-precision solve
  // reduced sums of the partial slots 0..3 (written by the last block of the
  // kernel producing the partials) and that kernel's block tickets, which the
  // last block returns to zero
  double red[4];
  unsigned int ticket[4];
};

// Per-stage summary of a solve run inside a captured RK4-step graph.
struct StageInfo {
  double rr, bb;
  int iters, outer, status, pad;
};

// Shared device helpers -------------------------------------------------------

// Global column of local horizontal node (i, j) of element column (ex, ey).
__host__ __device__ inline int node_col(const Geom& g, int ex, int ey, int i, int j) {
  int ix = ex * g.p + i;
  if (g.px && ix >= g.ncx) ix -= g.ncx;
  int iy = 0;
  if (g.dim == 3) {
    iy = ey * g.p + j;
    if (g.py && iy >= g.ncy) iy -= g.ncy;
  }
  return iy * g.ncx + ix;
}

// Ring slot of boundary line (i, j) of an element column, -1 for interior lines.
__host__ __device__ inline int ring_slot(int dim, int p, int i, int j) {
  if (dim == 2) return i == 0 ? 0 : (i == p ? 1 : -1);
  const int n = p + 1;
  if (j == 0) return i;
  if (j == p) return n + i;
  if (i == 0) return 2 * n + (j - 1);
  if (i == p) return 2 * n + (p - 1) + (j - 1);
  return -1;
}

// Owners of a node index along one direction: up to two (element, local index)
// pairs, in a fixed order.
__host__ __device__ inline int line_owners(int idx, int p, int ne, int periodic, int* e, int* loc) {
  if (idx % p != 0) {
    e[0] = idx / p;
    loc[0] = idx % p;
    return 1;
  }
  int L = idx / p, cnt = 0;
  if (L < ne) { e[cnt] = L; loc[cnt] = 0; ++cnt; }
  if (L >= 1) { e[cnt] = L - 1; loc[cnt] = p; ++cnt; }
  else if (periodic) { e[cnt] = ne - 1; loc[cnt] = p; ++cnt; }
  return cnt;
}

// Host-side helpers ------------------------------------------------------------
fnpf_status validate_desc(const fnpf_mesh_desc* d, std::string* why);
Geom make_geom(const fnpf_mesh_desc* d);
void gll_tables(int p, double* xi, double* w, double* D);   // host, long-double Newton
// Horizontal metric (r_x, r_y, s_x, s_y, w_i w_j |J2|) of every element-column
// line, lumped surface mass and surface coordinates; false on a degenerate map.
bool build_hmetric(const Geom& g, const double* xi, const double* w, const double* D, bool iso, double Lx, double Ly,
                   const double* Xs, const double* Ys, std::vector<double>* hm, std::vector<double>* mass,
                   std::vector<double>* xs, std::vector<double>* ys);

// Vector update fused into the gather stage of an operator application: the
// gather kernel visits every interior unknown i once the element kernel has
// finished, forms w_i = (A x)_i and applies
//   EP_RES:       r_i = (b ? b_i : r_i) - w_i
//   EP_RES_START: r_i = b_i - w_i;  d_i = c2 dinv_i r_i;  x_i += d_i    (x updated in place)
//   EP_CHEB:      r_i -= w_i;  d_i = c1 d_i + c2 dinv_i r_i;  x_i += d_i (d = x updated in place)
// instead of a separate vector kernel.  The operator's input may be updated in
// place because the element kernel has read all of it before the gather runs.
enum { EP_NONE = 0, EP_RES = 1, EP_RES_START = 2, EP_CHEB = 3 };
template <typename T>
struct Epilogue {
  int op = EP_NONE;
  T* r = nullptr;
  const T* b = nullptr;
  const T* dinv = nullptr;
  T* d = nullptr;
  T* x = nullptr;
  const double* c1 = nullptr;   // device scalars (Chebyshev step coefficients)
  const double* c2 = nullptr;
};

template <typename T>
__device__ __forceinline__ void apply_epilogue(const Epilogue<T>& e, int64_t i, T w) {
  if (e.op == EP_RES) {
    e.r[i] = (e.b ? e.b[i] : e.r[i]) - w;
  } else if (e.op == EP_RES_START) {
    const T rn = e.b[i] - w;
    e.r[i] = rn;
    const T dd = (T)(*e.c2) * e.dinv[i] * rn;
    e.d[i] = dd;
    e.x[i] += dd;
  } else {
    const T rn = e.r[i] - w;
    e.r[i] = rn;
    const T dd = (T)(*e.c1) * e.d[i] + (T)(*e.c2) * e.dinv[i] * rn;
    e.d[i] = dd;
    e.x[i] += dd;
  }
}

// Pointers of one operator application.
template <typename T>
struct AxPtrs {
  const T* eta;
  const T* xI;
  const T* xs;
  T* yI;
  T* ys;
  T* ring;
  const int* skip;   // if non-null and *skip != 0 the launch does nothing (converged solve)
  T* G = nullptr;    // stored metric (AX_GEOM output, AX_APPLY_G input)
  Epilogue<T> ep{};  // update fused into the gather (AX_APPLY, AX_APPLY_G); yI is scratch then
};

enum { AX_APPLY = 0, AX_DIAG = 1, AX_GEOM = 2, AX_APPLY_G = 3, AX_INIT = 4 };

// Per-order operator launcher, explicitly instantiated in ax_n<N>_f32.cu / _f64.cu.
template <typename T, int N>
cudaError_t launch_ax_n(const Geom& g, const Tables<T>& t, const AxPtrs<T>& a, int mode, int variant,
                        cudaStream_t s);

// Operator launches (ax_dispatch.cu).  xI == nullptr means zero interior;
// xs == nullptr means zero surface plane; ys == nullptr: surface rows not
// written.  `ring` is scratch of size nv * n_ecol * g.ring.
// A non-null `ep` fuses that update into the gather (ys must be null; yI is
// then scratch for the element kernel's column-interior lines).
template <typename T>
cudaError_t launch_apply(const Geom& g, const Tables<T>& t, const T* eta, const T* xI, const T* xs, T* yI,
                         T* ys, T* ring, int variant, cudaStream_t s, const int* skip = nullptr,
                         const Epilogue<T>* ep = nullptr);
template <typename T>
cudaError_t launch_diag(const Geom& g, const Tables<T>& t, const T* eta, T* dI, T* ds, T* ring, cudaStream_t s);
constexpr int kCtaVariants = 12;     // elements-per-CTA shapes of the 3D operator kernels
int apply_variants(int n, int dim);   // number of elements-per-CTA variants for order n-1
// Fills the constant tables of the line-decomposed operator kernels for order
// n - 1 on the current device (synchronous: call outside stream capture).
cudaError_t ax_prepare(int n);
int cta_columns(int n, int dim, int variant);   // element columns per CTA of a variant
// Stored metric: G (6 entries per point in 3D, 3 in 2D; geom_points(g) points)
// computed from eta once, and the operator reading it.
int64_t geom_points(const Geom& g);
template <typename T>
cudaError_t launch_geom(const Geom& g, const Tables<T>& t, const T* eta, T* G, cudaStream_t s);
template <typename T>
cudaError_t launch_apply_g(const Geom& g, const Tables<T>& t, const T* G, const T* xI, const T* xs, T* yI, T* ys,
                           T* ring, int variant, cudaStream_t s, const int* skip = nullptr,
                           const Epilogue<T>* ep = nullptr);

// Surface kernels (surface.cu).
struct StageArgs {
  const double* eta;     // stage state (read, neighbours)
  const double* geo;     // eta of the geometry (z_t of the w recovery): eta, or zeros (linear)
  int linear;            // 1: d eta/dt = w, d phi/dt = -g eta (linear potential flow)
  const double* phis;
  const double* phi;     // volume potential of this stage (top planes)
  const double* y0_eta;  // y_n (pointwise)
  const double* y0_phi;
  double* acc_eta;       // RK4 accumulator (pointwise)
  double* acc_phi;
  double* out_eta;       // next stage state, or y_{n+1} on the last stage
  double* out_phi;
  double bw;             // weight of this stage's k in the final combination
  double cn;             // c_{s+1} dt for the next stage state
  double dt;
  int first, last;
  double* deta;          // plain right-hand-side output (may be null)
  double* dphis;
  const double* w_in;    // if non-null, use this w instead of recovering it from phi
  const double* rhs_in;  // if non-null (nonlinear model): the right-hand side [2][ns], precomputed
  int* status;           // set to FNPF_EDIVERGED on a non-finite or folded state
  // relaxation after the last stage (cr null: none)
  const double* cr;
  const double* gen;
  const double* xs;      // surface-node coordinates
  const double* ys;
  double amp, kx, ky, omega, phase, ramp_time, t_end;
  const double* t_dev;   // if non-null: t_end = *t_dev + dt (graph replays)
};
cudaError_t launch_stage(const Geom& g, const Tables<double>& t, const StageArgs& a, cudaStream_t s);
cudaError_t launch_w(const Geom& g, const Tables<double>& t, const double* eta, const double* phis,
                     const double* phi, double* w, cudaStream_t s);
// Modal filter (surface.cu): out = the filtered copy of in (element-interior
// nodes filtered with the 1D matrix F [n * n] in each direction, other nodes
// copied); two fields at once (in1/out1 may be null).
cudaError_t launch_filter(const Geom& g, const double* F, const double* in0, double* out0, const double* in1,
                          double* out1, cudaStream_t s);
cudaError_t launch_check_state(const Geom& g, const double* eta, const double* phis, const double* h, int* status,
                               int* done, cudaStream_t s);

// Opts `kernel` in to `bytes` of dynamic shared memory when that is above the
// 48 KB default.  The attribute belongs to the (kernel, device) pair, so the
// record of it is a bit per device (devices 0..63; beyond that the attribute
// is set at every launch); two host threads may both set it, which is
// harmless.  Returns the error of cudaFuncSetAttribute.
template <typename K>
cudaError_t smem_optin(K kernel, size_t bytes, std::atomic<uint64_t>* done) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? uint64_t(1) << dev : 0;
  if (bit && (done->load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && bit) done->fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace fnpf

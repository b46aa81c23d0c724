// Preconditioned conjugate gradients for the Dirichlet-Neumann Laplace problem
// A_II phi_I = -A_IS phi_eta (arXiv 2506.09435, Sec. 3.4 Steps 4.2-4.3; the
// paper uses CG with algebraic multigrid, Sec. 4 solver settings), in two forms:
//
//  * FNPF_FP64: CG on the FP64 operator, preconditioned by Jacobi or by the
//    p-multigrid V-cycle of mg.cu;
//  * FNPF_MIXED: FP64 defect correction around FP32 inner solves -- the outer
//    residual r = b - A64 x is formed with the FP64 operator, the correction
//    e ~ A32^-1 r comes from PCG on the FP32 operator (FP32 geometry, vectors
//    and preconditioner, FP64 dot products), x += e in FP64, until
//    ||b - A64 x|| <= rtol ||b||.
//
// Reductions are deterministic: each block of a vector kernel writes one FP64
// partial sum; every consumer block re-reduces all partials in the same fixed
// order, so all blocks obtain bitwise-identical scalars without a grid sync.
// The convergence test stays on the device: kernels of a converged (or broken
// down) solve exit at once, and the host reads the flag every check_every
// iterations.
#include <math.h>

#include <algorithm>
#include <vector>

#include "mesh.cuh"
#include "mg.cuh"
#include "vec.cuh"
#include "graphs.cuh"

#define FNPF_CK(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      m->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return FNPF_ECUDA;                                           \
    }                                                              \
  } while (0)

namespace fnpf {
namespace {

constexpr int NT = kVecThreads;
using vec::block_sum;
using vec::reduce_partials;
#define GRID_LOOP(i, n) FNPF_GRID_LOOP(i, n)

// b = -y (y = A [0; phis]_I), r = b - q (q = A x), z = dinv r, p = z; partials bb, rz, rr.
struct cg_init_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, double* r, const double* q, const double* dinv, double* z, double* p,
                             double* b_out, double* part, int nb) {
    __shared__ double sh[vec::kShared];
    double sbb = 0, srz = 0, srr = 0;
    GRID_LOOP(i, n) {
      const double b = -r[i];
      const double rn = b - q[i];
      if (b_out) b_out[i] = b;
      r[i] = rn;
      sbb += b * b;
      srr += rn * rn;
      if (dinv) {
        const double zz = dinv[i] * rn;
        z[i] = zz;
        p[i] = zz;
        srz += rn * zz;
      }
    }
    sbb = block_sum(sbb, sh);
    srz = block_sum(srz, sh);
    srr = block_sum(srr, sh);
    if (threadIdx.x == 0) {
      part[0 * nb + bk.x] = sbb;
      part[1 * nb + bk.x] = srz;
      part[2 * nb + bk.x] = srr;
    }
  }
};

// Sets bb, rz[0], rr, tol2 from the partials; done if already converged.
struct cg_init_finish_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, CgScalars* sc, const double* part, int nb, double rtol2, double atol2) {
    __shared__ double sh[vec::kShared];
    const double bb = reduce_partials(part, nb, sh);
    const double rz = reduce_partials(part + nb, nb, sh);
    const double rr = reduce_partials(part + 2 * nb, nb, sh);
    if (threadIdx.x == 0) {
      sc->bb = bb;
      sc->rz[0] = rz;
      sc->rr = rr;
      sc->iters = 0;
      double tol2 = fmax(rtol2 * bb, atol2);
      if (bb == 0.0) tol2 = fmax(rtol2 * rr, atol2);
      sc->tol2 = tol2;
      if (!isfinite(rr) || !isfinite(bb)) {
        if (sc->status == 0) sc->status = FNPF_EDIVERGED;
        sc->done = 1;
      } else if (rr <= tol2) {
        sc->done = 1;
      }
    }
  }
};

// Inner (FP32) solve start from the FP64 residual: r32 = r64, e = 0, z = dinv r,
// p = z; partials rz, rr (FP64).
struct inner_init_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, const double* r64, float* r, float* e, float* z, float* p,
                             const float* dinv, double* part, int nb) {
    __shared__ double sh[vec::kShared];
    double srz = 0, srr = 0;
    GRID_LOOP(i, n) {
      const float rn = (float)r64[i];
      r[i] = rn;
      e[i] = 0.0f;
      srr += (double)rn * (double)rn;
      if (dinv) {
        const float zz = dinv[i] * rn;
        z[i] = zz;
        p[i] = zz;
        srz += (double)rn * (double)zz;
      }
    }
    srz = block_sum(srz, sh);
    srr = block_sum(srr, sh);
    if (threadIdx.x == 0) {
      if (dinv) part[1 * nb + bk.x] = srz;
      part[2 * nb + bk.x] = srr;
    }
  }
};

struct inner_init_finish_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, CgScalars* sc, const double* part, int nb, double rtol2) {
    __shared__ double sh[vec::kShared];
    const double rz = reduce_partials(part + nb, nb, sh);
    const double rr = reduce_partials(part + 2 * nb, nb, sh);
    if (threadIdx.x == 0) {
      sc->bb = rr;
      sc->rz[0] = rz;
      sc->rr = rr;
      sc->iters = 0;
      sc->tol2 = rtol2 * rr;
      sc->done = (rr == 0.0 || !isfinite(rr)) ? 1 : 0;
      if (!isfinite(rr)) sc->status = FNPF_EDIVERGED;
    }
  }
};

// x += e (FP64 += FP32); the outer residual r = b - q follows q = A64 x.
struct add_correction_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, double* x, const float* e) {
    GRID_LOOP(i, n) x[i] += (double)e[i];
  }
};

struct outer_residual_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, const double* b, const double* q, double* r, double* part, int nb) {
    __shared__ double sh[vec::kShared];
    double srr = 0;
    GRID_LOOP(i, n) {
      const double rn = b[i] - q[i];
      r[i] = rn;
      srr += rn * rn;
    }
    srr = block_sum(srr, sh);
    if (threadIdx.x == 0) part[2 * nb + bk.x] = srr;
  }
};

struct outer_finish_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, CgScalars* sc, const double* part, int nb) {
    __shared__ double sh[vec::kShared];
    const double rr = reduce_partials(part + 2 * nb, nb, sh);
    if (threadIdx.x == 0) {
      sc->rr = rr;
      sc->outer += 1;
      if (!isfinite(rr)) {
        sc->status = FNPF_EDIVERGED;
        sc->done = 1;
      } else if (rr <= sc->tol2) {
        sc->done = 1;
      }
    }
  }
};

struct to_float_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, const double* a, float* b) {
    GRID_LOOP(i, n) b[i] = (float)a[i];
  }
};

// Residual into the FP32 preconditioner and its result back (FNPF_FP64_PC32).
struct narrow_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, const int* skip, int64_t n, const double* a, float* b) {
    if (skip && *skip) return;
    GRID_LOOP(i, n) b[i] = (float)a[i];
  }
};
struct widen_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, const int* skip, int64_t n, const float* a, double* b) {
    if (skip && *skip) return;
    GRID_LOOP(i, n) b[i] = (double)a[i];
  }
};

// An FP64 solve whose p-multigrid preconditioner runs in FP32.
inline bool pc32(const fnpf_mesh* m) {
  return m->opts.precision == FNPF_FP64_PC32 && m->opts.precond == FNPF_PMG;
}

inline int vec_blocks(int64_t n) { return vec::blocks_for(n); }

// Host-driven solves re-estimate the Chebyshev intervals on the first solve of
// a precision and then every fourth solve (once per RK4 step); the 1.1 safety
// factor on lmax covers the change of the geometry between stages.
bool want_estimate(fnpf_mesh* m, int prec) {
  const bool e = !m->cheb_valid[prec] || m->solve_count[prec] % 4 == 0;
  ++m->solve_count[prec];
  m->cheb_valid[prec] = true;
  return e;
}

// The stored metric of the finest level while an FP64 solve uses it.
template <typename T>
const T* level0_G(const fnpf_mesh* m) {
  return sizeof(T) == 8 && m->g64_active ? reinterpret_cast<const T*>(m->G64) : nullptr;
}

// Operator application bracketed by profiling events when enabled.  `it` is the
// CG iteration the application belongs to (-1: outside the loop); applications
// of iterations that turn out to follow convergence exit at once and are not
// counted.
template <typename T>
cudaError_t timed_apply(fnpf_mesh* m, const Tables<T>& t, const T* eta, const T* xI, const T* xs, T* yI,
                        cudaStream_t s, const int* skip, int it) {
  const bool rec = m->prof_on && m->prof_used * 2 + 1 < (int)m->prof_ev.size();
  if (rec) cudaEventRecord(m->prof_ev[2 * m->prof_used], s);
  const T* G = sizeof(T) == 8 && m->g64_active ? reinterpret_cast<const T*>(m->G64) : nullptr;
  cudaError_t e = G ? launch_apply_g<T>(m->g, t, G, xI, xs, yI, nullptr, reinterpret_cast<T*>(m->ring),
                                        m->variant<T>(), s, skip)
                    : launch_apply<T>(m->g, t, eta, xI, xs, yI, nullptr, reinterpret_cast<T*>(m->ring),
                                      m->variant<T>(), s, skip);
  if (rec) {
    cudaEventRecord(m->prof_ev[2 * m->prof_used + 1], s);
    m->prof_it[m->prof_used] = it;
    m->prof_fp32[m->prof_used] = sizeof(T) == 4 ? 1 : 0;
    ++m->prof_used;
  }
  m->launches += 2;
  return e;
}

template <typename T>
fnpf_status tune_one(fnpf_mesh* m, const Tables<T>& t, const T* eta, const T* G, T* x, T* y, cudaStream_t s,
                     int* best) {
  const Geom& g = m->g;
  const int nv = apply_variants(g.n, g.dim);
  float best_ms = 1e30f;
  *best = 1;
  T* ring = reinterpret_cast<T*>(m->ring);
  auto run = [&](int v) {
    return G ? launch_apply_g<T>(g, t, G, x, nullptr, y, nullptr, ring, v, s, nullptr)
             : launch_apply<T>(g, t, eta, x, nullptr, y, nullptr, ring, v, s, nullptr);
  };
  // interleaved trials (every shape once per trial), best of kTrials per
  // shape, so clock ramp-up and neighbours' noise hit all shapes alike
  constexpr int kTrials = 4, kReps = 5;
  float shape_ms[kCtaVariants];
  for (int v = 0; v < nv; ++v) {
    FNPF_CK(run(v));
    shape_ms[v] = 1e30f;
  }
  for (int trial = 0; trial < kTrials; ++trial)
    for (int v = 0; v < nv; ++v) {
      FNPF_CK(cudaEventRecord(m->ev0, s));
      for (int r = 0; r < kReps; ++r) FNPF_CK(run(v));
      FNPF_CK(cudaEventRecord(m->ev1, s));
      FNPF_CK(cudaEventSynchronize(m->ev1));
      float ms = 0;
      FNPF_CK(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
      shape_ms[v] = fminf(shape_ms[v], ms);
    }
  for (int v = 0; v < nv; ++v)
    if (shape_ms[v] < best_ms) {
      best_ms = shape_ms[v];
      *best = v;
    }
  return FNPF_OK;
}

}  // namespace

fnpf_status autotune(fnpf_mesh* m, const double* eta, const double* G, cudaStream_t s) {
  const Geom& g = m->g;
  FNPF_CK(cudaMemsetAsync(m->p, 0, g.NI * sizeof(double), s));
  FNPF_CK(cudaMemsetAsync(m->p32, 0, g.NI * sizeof(float), s));
  launch<to_float_kernel>(vec_blocks(g.ns), NT, 0, s, g.ns, eta, m->eta32);
  FNPF_CK(cudaGetLastError());
  fnpf_status st = tune_one<double>(m, m->tables(), eta, G, m->p, m->q, s, &m->variant64);
  if (st == FNPF_OK) st = tune_one<float>(m, m->tables32(), m->eta32, nullptr, m->p32, m->q32, s, &m->variant32);
  m->tuned = true;
  return st;
}

void graph_reset(GraphSlot* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  g->kernels = 0;
  g->key[0] = g->key[1] = nullptr;
}

void prof_collect(fnpf_mesh* m, int iters_done) {
  for (int k = 0; k < m->prof_used; ++k) {
    if (m->prof_it[k] >= iters_done) continue;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, m->prof_ev[2 * k], m->prof_ev[2 * k + 1]) == cudaSuccess) {
      if (m->prof_fp32[k]) {
        m->prof_ms32 += ms;
        ++m->prof_count32;
      } else {
        m->prof_ms += ms;
        ++m->prof_count;
      }
    }
  }
  m->prof_used = 0;
}


namespace {

// Buffers of one PCG iteration loop in precision T.
template <typename T>
struct PcgBufs {
  const T* eta;
  T* x;
  T* r;
  T* z;
  T* p;
  T* q;
  const T* dinv;
  CgScalars* sc;
};

// z = M r with the p-multigrid V-cycle in the solve's precision, or, for an
// FNPF_FP64_PC32 solve, the FP32 V-cycle on the residual rounded to FP32 (its
// FP32 set-up done by mg_prepare<float> on eta32).
template <typename T>
cudaError_t apply_precond(fnpf_mesh* m, const Tables<T>& t, const T* eta, const T* r, T* z, const int* skip,
                          cudaStream_t s) {
  if (sizeof(T) == 8 && pc32(m)) {
    const int64_t NI = m->g.NI;
    const int nb = vec_blocks(NI);
    launch<narrow_kernel>(nb, NT, 0, s, skip, NI, reinterpret_cast<const double*>(r), m->r32);
    cudaError_t e = mg_apply<float>(m->mg, m->tables32(), m->eta32, nullptr, m->r32, m->z32,
                                    reinterpret_cast<float*>(m->ring), m->variant32, m->opts.cheb_degree,
                                    m->opts.coarse_iters, skip, s, &m->launches);
    if (e != cudaSuccess) return e;
    launch<widen_kernel>(nb, NT, 0, s, skip, NI, m->z32, reinterpret_cast<double*>(z));
    m->launches += 2;
    return cudaGetLastError();
  }
  return mg_apply<T>(m->mg, t, eta, level0_G<T>(m), r, z, reinterpret_cast<T*>(m->ring), m->variant<T>(),
                     m->opts.cheb_degree, m->opts.coarse_iters, skip, s, &m->launches);
}

// One PCG iteration (iteration parity it & 1), enqueued on s.
template <typename T>
cudaError_t enqueue_iteration(fnpf_mesh* m, const Tables<T>& t, const PcgBufs<T>& B, int it, cudaStream_t s) {
  const int64_t NI = m->g.NI;
  const int nb = vec_blocks(NI);
  const bool pmg = m->opts.precond == FNPF_PMG;
  const int* skip = &B.sc->done;
  cudaError_t e = timed_apply<T>(m, t, B.eta, B.p, nullptr, B.q, s, skip, it);
  if (e != cudaSuccess) return e;
  launch<vec::dot_kernel<T>>(nb, NT, 0, s, skip, NI, B.p, B.q, m->partials + 3 * nb, B.sc, 3);
  launch<vec::update_kernel<T>>(nb, NT, 0, s, B.sc, it, NI, B.x, B.r, B.z, B.p, B.q, pmg ? nullptr : B.dinv,
                                          m->partials, nb, nullptr);
  if (pmg) {
    e = apply_precond<T>(m, t, B.eta, B.r, B.z, skip, s);
    if (e != cudaSuccess) return e;
    launch<vec::dot_kernel<T>>(nb, NT, 0, s, skip, NI, B.r, B.z, m->partials + 1 * nb, B.sc, 1);
    m->launches += 1;
  }
  launch<vec::pupdate_kernel<T>>(nb, NT, 0, s, B.sc, it, NI, B.z, B.p, m->partials, nb, nullptr);
  m->launches += 3;
  return cudaGetLastError();
}

// Runs PCG iterations until the device flag is set or max_iter is reached; the
// scalars must have been initialised.  After the first chunk (which also does
// any lazy kernel set-up) the iterations run as replays of a CUDA graph that
// holds two iterations (parities 0 and 1), captured once per mesh and
// precision on the mesh's capture stream and launched on s.  Returns the host
// copy of the scalars in *out and whether the loop converged.
template <typename T>
fnpf_status pcg_loop(fnpf_mesh* m, const Tables<T>& t, const PcgBufs<T>& B, int max_iter, cudaStream_t s,
                     CgScalars* out, bool* done) {
  const int every = std::max(2, m->opts.check_every & ~1);
  const bool graphs = m->opts.use_graphs && !m->prof_on;
  GraphSlot& slot = m->g_iter[sizeof(T) == 4 ? 1 : 0];
  int it = 0;
  *done = false;
  while (true) {
    FNPF_CK(cudaMemcpyAsync(m->sc_host, B.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    FNPF_CK(cudaStreamSynchronize(s));
    prof_collect(m, m->sc_host->done ? m->sc_host->iters : it);
    *done = m->sc_host->done != 0;
    if (*done || it >= max_iter) break;
    int chunk = std::min(every, max_iter - it);
    if (graphs && it > 0 && (it & 1) == 0 && chunk >= 2) {
      if (!slot.exec || slot.key[0] != B.x || slot.key[1] != B.eta) {
        graph_reset(&slot);
        FNPF_CK(cudaStreamBeginCapture(m->gstream, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = m->launches;
        cudaError_t e = enqueue_iteration<T>(m, t, B, 0, m->gstream);
        if (e == cudaSuccess) e = enqueue_iteration<T>(m, t, B, 1, m->gstream);
        slot.kernels = m->launches - l0;
        m->launches = l0;
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(m->gstream, &graph);
        FNPF_CK(e);
        FNPF_CK(e2);
        const cudaError_t e3 = cudaGraphInstantiate(&slot.exec, graph, 0);
        cudaGraphDestroy(graph);
        FNPF_CK(e3);
        slot.key[0] = B.x;
        slot.key[1] = B.eta;
      }
      const int pairs = chunk / 2;
      for (int k = 0; k < pairs; ++k) FNPF_CK(cudaGraphLaunch(slot.exec, s));
      m->launches += pairs * slot.kernels;
      it += 2 * pairs;
      chunk -= 2 * pairs;
    }
    for (int k = 0; k < chunk; ++k, ++it) FNPF_CK(enqueue_iteration<T>(m, t, B, it, s));
  }
  *out = *m->sc_host;
  return FNPF_OK;
}

// With the p-multigrid preconditioner: z = M r, p = z, partial rz (slot 1).
template <typename T>
fnpf_status pmg_start(fnpf_mesh* m, const Tables<T>& t, const T* eta, const T* r, T* z, T* p, cudaStream_t s) {
  const int64_t NI = m->g.NI;
  const int nb = vec_blocks(NI);
  FNPF_CK(apply_precond<T>(m, t, eta, r, z, nullptr, s));
  launch<vec::copy_kernel<T>>(nb, NT, 0, s, NI, z, p, nullptr);
  launch<vec::dot_kernel<T>>(nb, NT, 0, s, nullptr, NI, r, z, m->partials + 1 * nb, nullptr, 0);
  m->launches += 2;
  FNPF_CK(cudaGetLastError());
  return FNPF_OK;
}

fnpf_status finish(fnpf_mesh* m, const CgScalars& h, bool done, int iters, int outer, fnpf_solve_info* info,
                   cudaStream_t s) {
  m->g64_active = false;
  fnpf_status st = FNPF_OK;
  if (h.status != 0) st = (fnpf_status)h.status;
  else if (!done) st = FNPF_ENOCONV;
  if (info) {
    FNPF_CK(cudaEventRecord(m->ev1, s));
    FNPF_CK(cudaEventSynchronize(m->ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, m->ev0, m->ev1);
    info->iters = iters;
    info->outer_iters = outer;
    info->rel_res = h.bb > 0 ? sqrt(h.rr / h.bb) : 0.0;
    info->status = st;
    info->ms = ms;
  }
  if (st == FNPF_ENOCONV) m->err = "solver reached its iteration cap before the tolerance";
  else if (st == FNPF_EBREAKDOWN) m->err = "CG breakdown (p^T A p <= 0 or non-finite)";
  else if (st == FNPF_EDIVERGED) m->err = "non-finite state or eta + h <= 0";
  return st;
}

}  // namespace

struct negate_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, const double* a, double* b) {
    GRID_LOOP(i, n) b[i] = -a[i];
  }
};

struct scale_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, const double* d, const double* a, double* b) {
    GRID_LOOP(i, n) b[i] = d[i] * a[i];
  }
};

// Validates the multigrid options, creates the hierarchy at the first use and
// passes the coarse-solver choice on.
fnpf_status ensure_mg(fnpf_mesh* m) {
  if (m->opts.cheb_degree < 1 || m->opts.cheb_degree >= kMaxChebDegree || m->opts.coarse_iters < 1 ||
      m->opts.coarse_iters >= kMaxChebDegree) {
    m->err = "Chebyshev degrees must be in 1..63";
    return FNPF_EINVAL;
  }
  if (m->opts.coarse_solver != FNPF_COARSE_CLUSTER && m->opts.coarse_solver != FNPF_COARSE_LAUNCHES) {
    m->err = "coarse_solver must be FNPF_COARSE_CLUSTER or FNPF_COARSE_LAUNCHES";
    return FNPF_EINVAL;
  }
  if (m->opts.cheb_kind != FNPF_CHEB_FIRST && m->opts.cheb_kind != FNPF_CHEB_FOURTH) {
    m->err = "cheb_kind must be FNPF_CHEB_FIRST or FNPF_CHEB_FOURTH";
    return FNPF_EINVAL;
  }
  if (!(m->opts.cheb_range > 1.0) || !(m->opts.cheb_range < 1e12)) {
    m->err = "cheb_range must be in (1, 1e12)";
    return FNPF_EINVAL;
  }
  if (m->opts.mg_schedule != FNPF_MG_HALVE && m->opts.mg_schedule != FNPF_MG_TWO_LEVEL &&
      m->opts.mg_schedule != FNPF_MG_STEP2) {
    m->err = "mg_schedule must be FNPF_MG_HALVE, FNPF_MG_TWO_LEVEL or FNPF_MG_STEP2";
    return FNPF_EINVAL;
  }
  if (m->mg && mg_schedule(m->mg) != m->opts.mg_schedule) {
    mg_destroy(m->mg);
    m->mg = nullptr;
  }
  if (!m->mg) {
    std::string why;
    m->mg = mg_create(m->g, m->h, m->Xs, m->Ys, m->iso, m->Lx, m->Ly, m->opts.mg_schedule, &why);
    if (!m->mg) {
      m->err = why;
      return FNPF_ENOMEM;
    }
  }
  mg_set_coarse(m->mg, m->opts.coarse_solver);
  mg_set_kind(m->mg, m->opts.cheb_kind, m->opts.cheb_range);
  return FNPF_OK;
}

// Allocates the stored FP64 metric at its first use.
fnpf_status ensure_g64(fnpf_mesh* m) {
  if (m->G64) return FNPF_OK;
  const int64_t ng = (m->g.dim == 3 ? 6 : 3) * geom_points(m->g);
  if (cudaMalloc((void**)&m->G64, ng * sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();
    m->G64 = nullptr;
    m->err = "cannot allocate the stored metric";
    return FNPF_ENOMEM;
  }
  return FNPF_OK;
}

fnpf_status precond_apply(fnpf_mesh* m, const double* eta_in, const double* r, double* z, cudaStream_t s) {
  const Geom& g = m->g;
  const double* eta = m->geom_eta(eta_in);
  m->lpf_ready[0] = false;   // the set-up below overwrites the kept one
  const Tables<double> t = m->tables();
  const int nb = vec_blocks(g.NI);
  if (m->opts.precond != FNPF_PMG) {
    FNPF_CK(launch_diag<double>(g, t, eta, m->dinv, nullptr, m->ring, s));
    launch<vec::invert_kernel<double>>(nb, NT, 0, s, g.NI, m->dinv);
    launch<scale_kernel>(nb, NT, 0, s, g.NI, m->dinv, r, z);
    FNPF_CK(cudaGetLastError());
    return FNPF_OK;
  }
  fnpf_status st = ensure_mg(m);
  if (st != FNPF_OK) return st;
  m->g64_active = false;
  if (m->opts.store_metric) {
    if ((st = ensure_g64(m)) != FNPF_OK) return st;
    FNPF_CK(launch_geom<double>(g, t, eta, m->G64, s));
    m->g64_active = true;
  }
  cudaError_t e = mg_prepare<double>(m->mg, t, eta, level0_G<double>(m), m->ring, m->variant64,
                                     m->opts.cheb_degree, m->opts.coarse_iters, true, s);
  if (e == cudaSuccess)
    e = mg_apply<double>(m->mg, t, eta, level0_G<double>(m), r, z, m->ring, m->variant64, m->opts.cheb_degree,
                         m->opts.coarse_iters, nullptr, s, &m->launches);
  m->g64_active = false;
  m->cheb_valid[0] = false;   // the next solve estimates its own intervals
  FNPF_CK(e);
  FNPF_CK(cudaGetLastError());
  return FNPF_OK;
}

// ---------------------------------------------------------------------------
// Initial guess by projection onto previous solutions (Fischer, "Projection
// techniques for iterative solution of Ax = b with successive right-hand
// sides", Comput. Methods Appl. Mech. Engrg. 163 (1998)).  The solves of an
// RK4 run have right-hand sides and operators that change smoothly from stage
// to stage, so the last L solutions H_0 (newest) .. H_{L-1} nearly span the
// next one.  With the basis X = [guess?, H_0 .. H_{L-1}] and the current
// operator A (the Gram system built in this solve's geometry),
//     x0 = X c,   (X^T A X) c = X^T b,
// is the A-orthogonal projection of the solution onto span X: its A-norm error
// is no larger than that of any basis vector, the guess included.  The first
// CG residual b - A x0 = b - (A X) c needs no further operator application.
// Near-dependent basis vectors (successive solutions differ by a few per cent)
// are dropped by the Cholesky factorisation of the Gram matrix when their new
// pivot falls below 1e-14 of their diagonal entry; non-finite ones likewise.

namespace {

struct ProjBasis {
  const double* x[kMaxProjection + 1];
  const double* ax[kMaxProjection + 1];
};

template <int K>
struct ProjSize {
  static constexpr int NP = K * (K + 1) / 2 + K;   // upper triangle of X^T A X, then X^T b
};
constexpr int kProjMaxNP = ProjSize<kMaxProjection + 1>::NP;

// Per-block partials of G_ac = x_a . (A x_c) (a <= c) and f_a = x_a . b, b = -r.
template <int K>
struct proj_gram_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, ProjBasis B, const double* r, double* part, int nb) {
    constexpr int NP = ProjSize<K>::NP;
    double acc[NP];
  #pragma unroll
    for (int q = 0; q < NP; ++q) acc[q] = 0.0;
    GRID_LOOP(i, n) {
      double xv[K], av[K];
  #pragma unroll
      for (int j = 0; j < K; ++j) {
        xv[j] = B.x[j][i];
        av[j] = B.ax[j][i];
      }
      const double b = -r[i];
      int q = 0;
  #pragma unroll
      for (int a = 0; a < K; ++a)
  #pragma unroll
        for (int c = a; c < K; ++c) acc[q++] += xv[a] * av[c];
  #pragma unroll
      for (int a = 0; a < K; ++a) acc[q++] += xv[a] * b;
    }
    __shared__ double sh[NT / 32][NP];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  #pragma unroll
    for (int q = 0; q < NP; ++q) {
      double v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sh[wid][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NP; q += NT) {
      double v = 0.0;
      for (int w = 0; w < NT / 32; ++w) v += sh[w][q];
      part[(int64_t)q * nb + bk.x] = v;
    }
  }
};

// One block: every sum over the partials in a fixed order (one warp per sum),
// then thread 0 solves the K x K Gram system by Cholesky with dropping and
// writes the coefficients c (0 for dropped vectors) to coef.
template <int K>
struct proj_solve_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, const double* part, int nb, double* coef) {
    constexpr int NP = ProjSize<K>::NP;
    __shared__ double red[NP];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = wid; q < NP; q += NT / 32) {
      double v = 0.0;
      for (int k = lane; k < nb; k += 32) v += part[(int64_t)q * nb + k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[q] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double G[K][K], f[K], Lw[K][K], z[K], c[K];
    bool act[K];
    int q = 0;
    for (int a = 0; a < K; ++a)
      for (int b = a; b < K; ++b) G[a][b] = G[b][a] = red[q++];
    for (int a = 0; a < K; ++a) f[a] = red[q++];
    for (int k = 0; k < K; ++k) {
      double d = G[k][k];
      for (int j = 0; j < k; ++j)
        if (act[j]) d -= Lw[k][j] * Lw[k][j];
      act[k] = isfinite(f[k]) && G[k][k] > 0.0 && isfinite(G[k][k]) && d > 1e-14 * G[k][k];
      if (!act[k]) continue;
      Lw[k][k] = sqrt(d);
      for (int i = k + 1; i < K; ++i) {
        double v = G[i][k];
        for (int j = 0; j < k; ++j)
          if (act[j]) v -= Lw[i][j] * Lw[k][j];
        Lw[i][k] = v / Lw[k][k];
      }
    }
    for (int k = 0; k < K; ++k) {
      z[k] = 0.0;
      if (!act[k]) continue;
      double v = f[k];
      for (int j = 0; j < k; ++j)
        if (act[j]) v -= Lw[k][j] * z[j];
      z[k] = v / Lw[k][k];
    }
    for (int k = K - 1; k >= 0; --k) {
      c[k] = 0.0;
      if (!act[k]) continue;
      double v = z[k];
      for (int j = k + 1; j < K; ++j)
        if (act[j]) v -= Lw[j][k] * c[j];
      c[k] = v / Lw[k][k];
    }
    for (int k = 0; k < K; ++k) coef[k] = c[k];
  }
};

// x0 = X c and A x0 = (A X) c (x and q may be basis vectors 0: read first).
template <int K>
struct proj_combine_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, ProjBasis B, const double* coef, double* x, double* q) {
    double c[K];
  #pragma unroll
    for (int j = 0; j < K; ++j) c[j] = coef[j];
    GRID_LOOP(i, n) {
      double sx = 0.0, sq = 0.0;
  #pragma unroll
      for (int j = 0; j < K; ++j) {
        if (c[j] != 0.0) {
          sx += c[j] * B.x[j][i];
          sq += c[j] * B.ax[j][i];
        }
      }
      x[i] = sx;
      q[i] = sq;
    }
  }
};

// History push after a solve: H_j <- H_{j-1} (j = L-1 .. 1), H_0 <- x.
struct proj_push_kernel {
  static constexpr int kThreads = NT;
  __device__ static void run(Blk bk, int64_t n, int L, double* H, const double* x) {
    GRID_LOOP(i, n) {
      for (int j = L - 1; j > 0; --j) H[(int64_t)j * n + i] = H[(int64_t)(j - 1) * n + i];
      H[i] = x[i];
    }
  }
};

template <int K>
void launch_projection_k(int64_t n, const ProjBasis& B, const double* r, double* part, int nb, double* coef,
                         double* x, double* q, cudaStream_t s) {
  launch<proj_gram_kernel<K>>(nb, NT, 0, s, n, B, r, part, nb);
  launch<proj_solve_kernel<K>>(1, NT, 0, s, part, nb, coef);
  launch<proj_combine_kernel<K>>(nb, NT, 0, s, n, B, coef, x, q);
}

// Allocates a history (zeroed: zero vectors are dropped) at its first use:
// the forward solves' (adj = false) or the adjoint solves' (adj = true).
fnpf_status ensure_projection(fnpf_mesh* m, bool adj) {
  const int L = m->opts.projection;
  double*& Hbuf = adj ? m->projHa : m->projH;
  int& alloc = adj ? m->proj_alloc_a : m->proj_alloc;
  if (L <= 0 || alloc >= L) return FNPF_OK;
  if (Hbuf) cudaFree(Hbuf);
  Hbuf = nullptr;
  alloc = 0;
  const size_t hbytes = (size_t)2 * L * m->g.NI * sizeof(double);
  if (cudaMalloc((void**)&Hbuf, std::max<size_t>(hbytes, 8)) != cudaSuccess) {
    Hbuf = nullptr;
    m->err = "projection history: device allocation failed";
    return FNPF_ENOMEM;
  }
  if (!m->proj_part) {
    const size_t pbytes = ((size_t)kProjMaxNP * kVecBlocks + 16) * sizeof(double);
    if (cudaMalloc((void**)&m->proj_part, pbytes) != cudaSuccess) {
      m->proj_part = nullptr;
      m->err = "projection history: device allocation failed";
      return FNPF_ENOMEM;
    }
  }
  if (cudaMemset(Hbuf, 0, hbytes) != cudaSuccess) return FNPF_ECUDA;
  alloc = L;
  return FNPF_OK;
}

// Replaces x by the projected initial guess and q by A x (r holds -b), with
// the history H ([2L][NI]: solutions, then their operator images).  The
// caller's guess x is a basis vector when with_guess.
cudaError_t enqueue_projection(fnpf_mesh* m, const Tables<double>& t, const double* eta, double* x, bool with_guess,
                               double* H, cudaStream_t s) {
  const int L = m->opts.projection;
  if (L <= 0) return cudaSuccess;
  const int64_t NI = m->g.NI;
  double* AH = H + (int64_t)L * NI;
  for (int j = 0; j < L; ++j) {
    cudaError_t e = timed_apply<double>(m, t, eta, H + (int64_t)j * NI, nullptr, AH + (int64_t)j * NI, s, nullptr,
                                        -1);
    if (e != cudaSuccess) return e;
  }
  ProjBasis B{};
  int K = 0;
  if (with_guess) {
    B.x[K] = x;
    B.ax[K] = m->q;
    ++K;
  }
  for (int j = 0; j < L; ++j, ++K) {
    B.x[K] = H + (int64_t)j * NI;
    B.ax[K] = AH + (int64_t)j * NI;
  }
  const int nb = vec_blocks(NI);
  double* coef = m->proj_part + (int64_t)kProjMaxNP * kVecBlocks;
  switch (K) {
    case 1: launch_projection_k<1>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
    case 2: launch_projection_k<2>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
    case 3: launch_projection_k<3>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
    case 4: launch_projection_k<4>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
    case 5: launch_projection_k<5>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
    case 6: launch_projection_k<6>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
    case 7: launch_projection_k<7>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
    case 8: launch_projection_k<8>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
    default: launch_projection_k<9>(NI, B, m->r, m->proj_part, nb, coef, x, m->q, s); break;
  }
  m->launches += 3;
  return cudaGetLastError();
}

cudaError_t enqueue_projection_push(fnpf_mesh* m, const double* x, double* H, cudaStream_t s) {
  const int L = m->opts.projection;
  if (L <= 0) return cudaSuccess;
  launch<proj_push_kernel>(vec_blocks(m->g.NI), NT, 0, s, m->g.NI, L, H, x);
  m->launches += 1;
  return cudaGetLastError();
}

}  // namespace

fnpf_status cg_solve(fnpf_mesh* m, const double* eta_in, const double* phis, double* x, fnpf_solve_info* info,
                     cudaStream_t s, const double* rhs) {
  const Geom& g = m->g;
  const Tables<double> t = m->tables();
  const int64_t NI = g.NI;
  const int nb = vec_blocks(NI);
  CgScalars* sc = m->sc;
  const bool mixed = m->opts.precision == FNPF_MIXED;
  const bool pmg = m->opts.precond == FNPF_PMG;
  if (pmg) {
    const fnpf_status st = ensure_mg(m);
    if (st != FNPF_OK) return st;
  }
  if (info) FNPF_CK(cudaEventRecord(m->ev0, s));
  // the solve reads eta from a mesh-owned copy, so captured graphs keep valid pointers
  FNPF_CK(cudaMemcpyAsync(m->eta64, m->geom_eta(eta_in), g.ns * sizeof(double), cudaMemcpyDeviceToDevice, s));
  const double* eta = m->eta64;
  FNPF_CK(cudaMemsetAsync(sc, 0, sizeof(CgScalars), s));
  FNPF_CK(launch_check_state(g, eta, rhs ? eta : phis, m->dh, &sc->status, &sc->done, s));
  // the FP64 operator (every application of an FP64 solve; the lift, the
  // projection and the outer residuals of a mixed solve) reads a metric rebuilt
  // from this eta once per solve (fewer FP64 instructions per point)
  // linear potential flow: the geometry is fixed, so the FP64 set-up of the
  // first solve is kept (lpf_ready) and later solves skip it
  const bool keep64 = m->linear() && m->lpf_ready[0];
  m->g64_active = false;
  if (m->opts.store_metric) {
    const fnpf_status st = ensure_g64(m);
    if (st != FNPF_OK) return st;
    if (!keep64) {
      FNPF_CK(launch_geom<double>(g, t, eta, m->G64, s));
      m->launches += 1;
    }
    m->g64_active = true;
  }
  if (!m->tuned) {
    const fnpf_status st = autotune(m, eta, m->g64_active ? m->G64 : nullptr, s);
    if (st != FNPF_OK) return st;
  }
  if (!mixed && !pmg && !keep64) {
    FNPF_CK(launch_diag<double>(g, t, eta, m->dinv, nullptr, m->ring, s));
    launch<vec::invert_kernel<double>>(nb, NT, 0, s, NI, m->dinv);
  }
  if (!mixed && pmg && !keep64) {
    if (pc32(m)) {
      launch<to_float_kernel>(vec_blocks(g.ns), NT, 0, s, g.ns, eta, m->eta32);
      FNPF_CK(mg_prepare<float>(m->mg, m->tables32(), m->eta32, nullptr, reinterpret_cast<float*>(m->ring),
                                m->variant32, m->opts.cheb_degree, m->opts.coarse_iters, want_estimate(m, 1), s));
    } else {
      FNPF_CK(mg_prepare<double>(m->mg, t, eta, level0_G<double>(m), m->ring, m->variant64, m->opts.cheb_degree,
                                 m->opts.coarse_iters, want_estimate(m, 0), s));
    }
  }
  if (!mixed && m->linear()) m->lpf_ready[0] = true;
  FNPF_CK(cudaGetLastError());
  // lift: r = A [0; phis]_I = -b (or r = -rhs); q = A [x; 0]_I; then b, r = b - q (, z, p)
  if (rhs) {
    launch<negate_kernel>(nb, NT, 0, s, NI, rhs, m->r);
    FNPF_CK(cudaGetLastError());
  } else {
    FNPF_CK(timed_apply<double>(m, t, eta, nullptr, phis, m->r, s, nullptr, -1));
  }
  FNPF_CK(timed_apply<double>(m, t, eta, x, nullptr, m->q, s, nullptr, -1));
  // forward solves project onto the forward history, adjoint solves (rhs
  // given) onto their own
  const bool project = m->opts.projection > 0;
  double*& hist = rhs ? m->projHa : m->projH;
  if (project) {
    const fnpf_status st = ensure_projection(m, rhs != nullptr);
    if (st != FNPF_OK) return st;
    FNPF_CK(enqueue_projection(m, t, eta, x, x != m->phi, hist, s));
  }
  launch<cg_init_kernel>(nb, NT, 0, s, NI, m->r, m->q, (mixed || pmg) ? nullptr : m->dinv, m->z, m->p,
                                   mixed ? m->b : nullptr, m->partials, nb);
  if (!mixed && pmg) {
    fnpf_status st = pmg_start<double>(m, t, eta, m->r, m->z, m->p, s);
    if (st != FNPF_OK) return st;
  }
  launch<cg_init_finish_kernel>(1, NT, 0, s, sc, m->partials, nb, m->opts.rtol * m->opts.rtol,
                                         m->opts.atol * m->opts.atol);
  FNPF_CK(cudaGetLastError());
  m->launches += 4 + (mixed ? 0 : 3);
  const int max_iter = std::max(0, m->opts.max_iter);
  CgScalars h{};
  bool done = false;
  if (!mixed) {
    PcgBufs<double> B{eta, x, m->r, m->z, m->p, m->q, m->dinv, sc};
    fnpf_status st = pcg_loop<double>(m, t, B, max_iter, s, &h, &done);
    if (st != FNPF_OK) return st;
    if (project) FNPF_CK(enqueue_projection_push(m, x, hist, s));
    return finish(m, h, done, h.iters, 0, info, s);
  }

  // ---- mixed precision: FP64 defect correction around FP32 Jacobi-PCG
  const Tables<float> t32 = m->tables32();
  if (!(m->linear() && m->lpf_ready[1])) {
    launch<to_float_kernel>(vec_blocks(g.ns), NT, 0, s, g.ns, eta, m->eta32);
    if (pmg) {
      FNPF_CK(mg_prepare<float>(m->mg, t32, m->eta32, nullptr, reinterpret_cast<float*>(m->ring), m->variant32,
                                m->opts.cheb_degree, m->opts.coarse_iters, want_estimate(m, 1), s));
    } else {
      FNPF_CK(launch_diag<float>(g, t32, m->eta32, m->dinv32, nullptr, reinterpret_cast<float*>(m->ring), s));
      launch<vec::invert_kernel<float>>(nb, NT, 0, s, NI, m->dinv32);
    }
    if (m->linear()) m->lpf_ready[1] = true;
  }
  FNPF_CK(cudaGetLastError());
  m->launches += 4;
  int inner_total = 0, outer = 0;
  const int max_outer = std::max(1, m->opts.max_outer);
  const double in_rtol2 = m->opts.inner_rtol * m->opts.inner_rtol;
  while (true) {
    FNPF_CK(cudaMemcpyAsync(m->sc_host, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    FNPF_CK(cudaStreamSynchronize(s));
    prof_collect(m, 1 << 30);
    h = *m->sc_host;
    done = h.done != 0;
    if (done || outer >= max_outer || inner_total >= max_iter) break;
    // inner solve A32 e = r (FP32, Jacobi-PCG, relative tolerance inner_rtol)
    CgScalars* si = m->sc_in;
    FNPF_CK(cudaMemsetAsync(si, 0, sizeof(CgScalars), s));
    launch<inner_init_kernel>(nb, NT, 0, s, NI, m->r, m->r32, m->e32, m->z32, m->p32, pmg ? nullptr : m->dinv32,
                                        m->partials, nb);
    if (pmg) {
      fnpf_status st = pmg_start<float>(m, t32, m->eta32, m->r32, m->z32, m->p32, s);
      if (st != FNPF_OK) return st;
    }
    launch<inner_init_finish_kernel>(1, NT, 0, s, si, m->partials, nb, in_rtol2);
    FNPF_CK(cudaGetLastError());
    m->launches += 2;
    PcgBufs<float> B{m->eta32, m->e32, m->r32, m->z32, m->p32, m->q32, m->dinv32, si};
    CgScalars hi{};
    bool idone = false;
    fnpf_status st = pcg_loop<float>(m, t32, B, max_iter - inner_total, s, &hi, &idone);
    if (st != FNPF_OK) return st;
    inner_total += hi.iters;
    if (hi.status == FNPF_EBREAKDOWN || hi.status == FNPF_EDIVERGED) {
      h.status = hi.status;
      break;
    }
    // x += e; r = b - A64 x
    launch<add_correction_kernel>(nb, NT, 0, s, NI, x, m->e32);
    FNPF_CK(timed_apply<double>(m, t, eta, x, nullptr, m->q, s, nullptr, -1));
    launch<outer_residual_kernel>(nb, NT, 0, s, NI, m->b, m->q, m->r, m->partials, nb);
    launch<outer_finish_kernel>(1, NT, 0, s, sc, m->partials, nb);
    FNPF_CK(cudaGetLastError());
    m->launches += 3;
    ++outer;
  }
  if (project) FNPF_CK(enqueue_projection_push(m, x, hist, s));
  return finish(m, h, done, inner_total, outer, info, s);
}

// ---------------------------------------------------------------------------
// Device-driven solves for captured RK4-step graphs: every loop is a CUDA
// conditional WHILE node whose body ends with a kernel that sets the loop
// condition from the device scalars, so a whole RK4 step runs without the host.

namespace {

__global__ void set_cond_kernel(const CgScalars* sc, cudaGraphConditionalHandle h, int cap, int use_outer) {
  const int cnt = use_outer ? sc->outer : sc->iters;
  cudaGraphSetConditional(h, (!sc->done && cnt < cap) ? 1u : 0u);
}

// Sets the loop condition h from the scalars (a recorded operation while a
// Recorder is active).
cudaError_t set_cond(const CgScalars* sc, cudaGraphConditionalHandle h, int cap, int use_outer, cudaStream_t s) {
  if (Recorder* r = active_recorder()) {
    Op op;
    op.kind = OP_COND;
    op.handle = (int)h;
    op.sc = sc;
    op.cap = cap;
    op.use_outer = use_outer;
    r->ops.push_back(std::move(op));
    return cudaSuccess;
  }
  set_cond_kernel<<<1, 1, 0, s>>>(sc, h, cap, use_outer);
  return cudaPeekAtLastError();
}

// inner solve finished: propagate a breakdown to the outer scalars
struct inner_done_kernel {
  static constexpr int kThreads = 1;
  __device__ static void run(Blk bk, const CgScalars* si, CgScalars* so, int* inner_total) {
    *inner_total += si->iters;
    if (si->status == FNPF_EBREAKDOWN || si->status == FNPF_EDIVERGED) {
      so->status = si->status;
      so->done = 1;
    }
  }
};

struct stage_info_kernel {
  static constexpr int kThreads = 1;
  __device__ static void run(Blk bk, const CgScalars* sc, const int* inner_total, int mixed, StageInfo* out) {
    out->rr = sc->rr;
    out->bb = sc->bb;
    out->iters = mixed ? *inner_total : sc->iters;
    out->outer = mixed ? sc->outer : 0;
    int st = sc->status;
    if (st == 0 && !sc->done) st = FNPF_ENOCONV;
    out->status = st;
  }
};

}  // namespace

cudaError_t new_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
  if (Recorder* r = active_recorder()) {
    Op op;
    op.kind = OP_HANDLE;
    op.handle = r->handles;
    *h = (cudaGraphConditionalHandle)r->handles++;
    r->ops.push_back(std::move(op));
    return cudaSuccess;
  }
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(h, g, 0, 0);
}

// Kernel nodes directly in graph g (not inside nested conditional bodies).
int64_t kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  int64_t k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

int64_t graph_kernel_nodes(cudaGraph_t g) { return kernel_nodes(g); }

// Enqueues (on a capturing stream s) one Laplace solve of the mesh's current
// options and its summary into *info_dev.  The mesh must have run a host-driven
// solve before (multigrid hierarchy, autotuned shapes, lazy kernel set-up).
cudaError_t enqueue_solve_device(fnpf_mesh* m, const double* eta_in, const double* phis, double* x,
                                 StageInfo* info_dev, cudaStream_t s, bool estimate) {
  const Geom& g = m->g;
  const Tables<double> t = m->tables();
  const int64_t NI = g.NI;
  const int nb = vec_blocks(NI);
  CgScalars* sc = m->sc;
  const bool mixed = m->opts.precision == FNPF_MIXED;
  const bool pmg = m->opts.precond == FNPF_PMG;
  const int max_iter = std::max(1, m->opts.max_iter);
  cudaError_t e;
#define ENQ(call)                      \
  do {                                 \
    if ((e = (call)) != cudaSuccess) { \
      m->g64_active = false;           \
      return e;                        \
    }                                  \
  } while (0)
  ENQ(memcpy_async(m->eta64, m->geom_eta(eta_in), g.ns * sizeof(double), cudaMemcpyDeviceToDevice, s));
  const double* eta = m->eta64;
  ENQ(memset_async(sc, 0, sizeof(CgScalars), s));
  ENQ(memset_async(m->inner_total, 0, sizeof(int), s));
  ENQ(launch_check_state(g, eta, phis, m->dh, &sc->status, &sc->done, s));
  // linear potential flow: a host-driven step has done the set-up (lpf_ready)
  const bool keep64 = m->linear() && m->lpf_ready[0];
  const bool keep32 = m->linear() && m->lpf_ready[1];
  m->g64_active = false;
  if (m->opts.store_metric && m->G64) {
    if (!keep64) ENQ(launch_geom<double>(g, t, eta, m->G64, s));
    m->g64_active = true;
  }
  if (!mixed && !pmg && !keep64) {
    ENQ(launch_diag<double>(g, t, eta, m->dinv, nullptr, m->ring, s));
    launch<vec::invert_kernel<double>>(nb, NT, 0, s, NI, m->dinv);
  }
  if (!mixed && pmg && !keep64) {
    if (pc32(m)) {
      launch<to_float_kernel>(vec_blocks(g.ns), NT, 0, s, g.ns, eta, m->eta32);
      ENQ(mg_prepare<float>(m->mg, m->tables32(), m->eta32, nullptr, reinterpret_cast<float*>(m->ring),
                            m->variant32, m->opts.cheb_degree, m->opts.coarse_iters, estimate, s));
    } else {
      ENQ(mg_prepare<double>(m->mg, t, eta, level0_G<double>(m), m->ring, m->variant64, m->opts.cheb_degree,
                             m->opts.coarse_iters, estimate, s));
    }
  }
  ENQ(timed_apply<double>(m, t, eta, nullptr, phis, m->r, s, nullptr, -1));
  ENQ(timed_apply<double>(m, t, eta, x, nullptr, m->q, s, nullptr, -1));
  // the history buffers exist: a host-driven solve of the same options ran before
  const bool project = m->opts.projection > 0 && m->proj_alloc >= m->opts.projection;
  if (project) ENQ(enqueue_projection(m, t, eta, x, x != m->phi, m->projH, s));
  launch<cg_init_kernel>(nb, NT, 0, s, NI, m->r, m->q, (mixed || pmg) ? nullptr : m->dinv, m->z, m->p,
                                   mixed ? m->b : nullptr, m->partials, nb);
  if (!mixed && pmg) {
    ENQ(apply_precond<double>(m, t, eta, m->r, m->z, nullptr, s));
    launch<vec::copy_kernel<double>>(nb, NT, 0, s, NI, m->z, m->p, nullptr);
    launch<vec::dot_kernel<double>>(nb, NT, 0, s, nullptr, NI, m->r, m->z, m->partials + 1 * nb, nullptr, 0);
  }
  launch<cg_init_finish_kernel>(1, NT, 0, s, sc, m->partials, nb, m->opts.rtol * m->opts.rtol,
                                         m->opts.atol * m->opts.atol);
  ENQ(cudaGetLastError());
  if (!mixed) {
    cudaGraphConditionalHandle h;
    ENQ(new_handle(s, &h));
    set_cond(sc, h, max_iter, 0, s);
    PcgBufs<double> B{eta, x, m->r, m->z, m->p, m->q, m->dinv, sc};
    ENQ(capture_while(s, m->bstream[0], h, &m->body_kernels[0], [&](cudaStream_t bs) -> cudaError_t {
      cudaError_t eb = enqueue_iteration<double>(m, t, B, 0, bs);
      if (eb == cudaSuccess) eb = enqueue_iteration<double>(m, t, B, 1, bs);
      set_cond(sc, h, max_iter, 0, bs);
      return eb == cudaSuccess ? cudaGetLastError() : eb;
    }));
  } else {
    const Tables<float> t32 = m->tables32();
    if (!keep32) {
      launch<to_float_kernel>(vec_blocks(g.ns), NT, 0, s, g.ns, eta, m->eta32);
      if (pmg) {
        ENQ(mg_prepare<float>(m->mg, t32, m->eta32, nullptr, reinterpret_cast<float*>(m->ring), m->variant32,
                              m->opts.cheb_degree, m->opts.coarse_iters, estimate, s));
      } else {
        ENQ(launch_diag<float>(g, t32, m->eta32, m->dinv32, nullptr, reinterpret_cast<float*>(m->ring), s));
        launch<vec::invert_kernel<float>>(nb, NT, 0, s, NI, m->dinv32);
      }
    }
    const int max_outer = std::max(1, m->opts.max_outer);
    const double in_rtol2 = m->opts.inner_rtol * m->opts.inner_rtol;
    cudaGraphConditionalHandle ho;
    ENQ(new_handle(s, &ho));
    set_cond(sc, ho, max_outer, 1, s);
    ENQ(capture_while(s, m->bstream[0], ho, &m->body_kernels[0], [&](cudaStream_t bs) -> cudaError_t {
      CgScalars* si = m->sc_in;
      cudaError_t eb = memset_async(si, 0, sizeof(CgScalars), bs);
      if (eb != cudaSuccess) return eb;
      launch<inner_init_kernel>(nb, NT, 0, bs, NI, m->r, m->r32, m->e32, m->z32, m->p32, pmg ? nullptr : m->dinv32,
                                           m->partials, nb);
      if (pmg) {
        if ((eb = mg_apply<float>(m->mg, t32, m->eta32, nullptr, m->r32, m->z32, reinterpret_cast<float*>(m->ring),
                                  m->variant32, m->opts.cheb_degree, m->opts.coarse_iters, nullptr, bs,
                                  &m->launches)) != cudaSuccess)
          return eb;
        launch<vec::copy_kernel<float>>(nb, NT, 0, bs, NI, m->z32, m->p32, nullptr);
        launch<vec::dot_kernel<float>>(nb, NT, 0, bs, nullptr, NI, m->r32, m->z32, m->partials + 1 * nb, nullptr, 0);
      }
      launch<inner_init_finish_kernel>(1, NT, 0, bs, si, m->partials, nb, in_rtol2);
      cudaGraphConditionalHandle hi;
      if ((eb = new_handle(bs, &hi)) != cudaSuccess) return eb;
      set_cond(si, hi, max_iter, 0, bs);
      PcgBufs<float> B{m->eta32, m->e32, m->r32, m->z32, m->p32, m->q32, m->dinv32, si};
      eb = capture_while(bs, m->bstream[1], hi, &m->body_kernels[1], [&](cudaStream_t bs2) -> cudaError_t {
        cudaError_t e2 = enqueue_iteration<float>(m, t32, B, 0, bs2);
        if (e2 == cudaSuccess) e2 = enqueue_iteration<float>(m, t32, B, 1, bs2);
        set_cond(si, hi, max_iter, 0, bs2);
        return e2 == cudaSuccess ? cudaGetLastError() : e2;
      });
      if (eb != cudaSuccess) return eb;
      launch<inner_done_kernel>(1, 1, 0, bs, si, sc, m->inner_total);
      launch<add_correction_kernel>(nb, NT, 0, bs, NI, x, m->e32);
      if ((eb = timed_apply<double>(m, t, eta, x, nullptr, m->q, bs, nullptr, -1)) != cudaSuccess) return eb;
      launch<outer_residual_kernel>(nb, NT, 0, bs, NI, m->b, m->q, m->r, m->partials, nb);
      launch<outer_finish_kernel>(1, NT, 0, bs, sc, m->partials, nb);
      set_cond(sc, ho, max_outer, 1, bs);
      return cudaGetLastError();
    }));
  }
  if (project) ENQ(enqueue_projection_push(m, x, m->projH, s));
  launch<stage_info_kernel>(1, 1, 0, s, sc, m->inner_total, mixed ? 1 : 0, info_dev);
  m->g64_active = false;
  return cudaGetLastError();
#undef ENQ
}

}  // namespace fnpf

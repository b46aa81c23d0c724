// Jacobi-preconditioned conjugate gradients for the Dirichlet-Neumann Laplace
// problem A_II phi_I = -A_IS phi_eta (arXiv 2506.09435, Sec. 3.4 Steps 4.2-4.3;
// the paper uses CG with algebraic multigrid, Sec. 4 solver settings).
//
// Reductions are deterministic: each block of a vector kernel writes one FP64
// partial sum; every consumer block re-reduces all partials in the same fixed
// order, so all blocks obtain bitwise-identical scalars without a grid sync.
// The convergence test stays on the device: kernels of a converged (or broken
// down) solve exit at once, and the host reads the flag every check_every
// iterations.
#include <math.h>

#include <algorithm>

#include "mesh.cuh"

namespace fnpf {
namespace {

constexpr int NT = kVecThreads;

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0;
  for (int k = 0; k < NT / 32; ++k) s += sh[k];
  return s;
}

__device__ double reduce_partials(const double* part, int nb, double* sh) {
  double v = 0;
  for (int k = threadIdx.x; k < nb; k += NT) v += part[k];
  return block_sum(v, sh);
}

__global__ void __launch_bounds__(NT) invert_kernel(int64_t n, double* d) {
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) d[i] = 1.0 / d[i];
}

__global__ void __launch_bounds__(NT) cg_init_kernel(int64_t n, double* r, const double* q, const double* dinv,
                                                     double* z, double* p, double* part, int nb) {
  __shared__ double sh[NT / 32];
  double sbb = 0, srz = 0, srr = 0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
    const double b = -r[i];
    const double rn = b - q[i];
    const double zz = dinv[i] * rn;
    r[i] = rn;
    z[i] = zz;
    p[i] = zz;
    sbb += b * b;
    srz += rn * zz;
    srr += rn * rn;
  }
  sbb = block_sum(sbb, sh);
  srz = block_sum(srz, sh);
  srr = block_sum(srr, sh);
  if (threadIdx.x == 0) {
    part[0 * nb + blockIdx.x] = sbb;
    part[1 * nb + blockIdx.x] = srz;
    part[2 * nb + blockIdx.x] = srr;
  }
}

__global__ void __launch_bounds__(NT) cg_init_finish_kernel(CgScalars* sc, const double* part, int nb, double rtol2,
                                                            double atol2) {
  __shared__ double sh[NT / 32];
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

__global__ void __launch_bounds__(NT) cg_dot_kernel(const CgScalars* sc, int64_t n, const double* p, const double* q,
                                                    double* part) {
  if (sc->done) return;
  __shared__ double sh[NT / 32];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) s += p[i] * q[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(NT) cg_update_kernel(CgScalars* sc, int it, int64_t n, double* x, double* r,
                                                       double* z, const double* p, const double* q,
                                                       const double* dinv, double* part, int nb) {
  if (sc->done) return;
  __shared__ double sh[NT / 32];
  const double pq = reduce_partials(part + 3 * nb, nb, sh);
  const double rz = sc->rz[it & 1];
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->status = FNPF_EBREAKDOWN;
      sc->done = 1;
    }
    return;
  }
  const double alpha = rz / pq;
  double srz = 0, srr = 0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
    x[i] += alpha * p[i];
    const double rn = r[i] - alpha * q[i];
    const double zz = dinv[i] * rn;
    r[i] = rn;
    z[i] = zz;
    srz += rn * zz;
    srr += rn * rn;
  }
  srz = block_sum(srz, sh);
  srr = block_sum(srr, sh);
  if (threadIdx.x == 0) {
    part[1 * nb + blockIdx.x] = srz;
    part[2 * nb + blockIdx.x] = srr;
  }
}

__global__ void __launch_bounds__(NT) cg_pupdate_kernel(CgScalars* sc, int it, int64_t n, const double* z, double* p,
                                                        const double* part, int nb) {
  if (sc->done) return;
  __shared__ double sh[NT / 32];
  const double rz_new = reduce_partials(part + nb, nb, sh);
  const double rr = reduce_partials(part + 2 * nb, nb, sh);
  const double beta = rz_new / sc->rz[it & 1];
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
    p[i] = z[i] + beta * p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rz[(it + 1) & 1] = rz_new;
    sc->rr = rr;
    sc->iters = it + 1;
    if (!isfinite(rr)) {
      sc->status = FNPF_EBREAKDOWN;
      sc->done = 1;
    } else if (rr <= sc->tol2) {
      sc->done = 1;
    }
  }
}

// Operator application bracketed by profiling events when enabled.
// `it` is the CG iteration the application belongs to (-1: set-up); applications
// of iterations that turn out to follow convergence exit at once and are not
// counted.
cudaError_t timed_apply(fnpf_mesh* m, const double* eta, const double* xI, const double* xs, double* yI,
                        cudaStream_t s, const int* skip, int it) {
  const bool rec = m->prof_on && m->prof_used * 2 + 1 < (int)m->prof_ev.size();
  if (rec) cudaEventRecord(m->prof_ev[2 * m->prof_used], s);
  cudaError_t e = launch_apply<double>(m->g, m->tables(), eta, xI, xs, yI, nullptr, m->ring, m->variant, s, skip);
  if (rec) {
    cudaEventRecord(m->prof_ev[2 * m->prof_used + 1], s);
    m->prof_it[m->prof_used] = it;
    ++m->prof_used;
  }
  m->launches += 2;
  return e;
}

inline int vec_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(kVecBlocks, (n + NT - 1) / NT)); }

}  // namespace

void prof_collect(fnpf_mesh* m, int iters_done) {
  for (int k = 0; k < m->prof_used; ++k) {
    if (m->prof_it[k] >= iters_done) continue;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, m->prof_ev[2 * k], m->prof_ev[2 * k + 1]) == cudaSuccess) {
      m->prof_ms += ms;
      ++m->prof_count;
    }
  }
  m->prof_used = 0;
}

#define FNPF_CK(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      m->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return FNPF_ECUDA;                               \
    }                                                  \
  } while (0)

fnpf_status cg_solve(fnpf_mesh* m, const double* eta, const double* phis, double* x, fnpf_solve_info* info,
                     cudaStream_t s) {
  const Geom& g = m->g;
  const Tables<double> t = m->tables();
  const int64_t NI = g.NI;
  const int nb = vec_blocks(NI);
  CgScalars* sc = m->sc;
  if (info) FNPF_CK(cudaEventRecord(m->ev0, s));
  FNPF_CK(cudaMemsetAsync(sc, 0, sizeof(CgScalars), s));
  FNPF_CK(launch_check_state(g, eta, phis, m->dh, &sc->status, &sc->done, s));
  FNPF_CK(launch_diag<double>(g, t, eta, m->dinv, nullptr, m->ring, s));
  invert_kernel<<<nb, NT, 0, s>>>(NI, m->dinv);
  FNPF_CK(cudaGetLastError());
  FNPF_CK(timed_apply(m, eta, nullptr, phis, m->r, s, nullptr, -1));
  FNPF_CK(timed_apply(m, eta, x, nullptr, m->q, s, nullptr, -1));
  cg_init_kernel<<<nb, NT, 0, s>>>(NI, m->r, m->q, m->dinv, m->z, m->p, m->partials, nb);
  cg_init_finish_kernel<<<1, NT, 0, s>>>(sc, m->partials, nb, m->opts.rtol * m->opts.rtol,
                                         m->opts.atol * m->opts.atol);
  FNPF_CK(cudaGetLastError());
  m->launches += 6;   // check, diagonal + gather, invert, init, init-finish
  const int max_iter = std::max(0, m->opts.max_iter);
  const int every = std::max(1, m->opts.check_every);
  int it = 0;
  bool done = false;
  while (true) {
    FNPF_CK(cudaMemcpyAsync(m->sc_host, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    FNPF_CK(cudaStreamSynchronize(s));
    prof_collect(m, m->sc_host->done ? m->sc_host->iters : it);
    done = m->sc_host->done != 0;
    if (done || it >= max_iter) break;
    const int chunk = std::min(every, max_iter - it);
    for (int k = 0; k < chunk; ++k, ++it) {
      FNPF_CK(timed_apply(m, eta, m->p, nullptr, m->q, s, &sc->done, it));
      m->launches += 3;
      cg_dot_kernel<<<nb, NT, 0, s>>>(sc, NI, m->p, m->q, m->partials + 3 * nb);
      cg_update_kernel<<<nb, NT, 0, s>>>(sc, it, NI, x, m->r, m->z, m->p, m->q, m->dinv, m->partials, nb);
      cg_pupdate_kernel<<<nb, NT, 0, s>>>(sc, it, NI, m->z, m->p, m->partials, nb);
    }
    FNPF_CK(cudaGetLastError());
  }
  const CgScalars& h = *m->sc_host;
  fnpf_status st = FNPF_OK;
  if (h.status != 0) st = (fnpf_status)h.status;
  else if (!done) st = FNPF_ENOCONV;
  if (info) {
    FNPF_CK(cudaEventRecord(m->ev1, s));
    FNPF_CK(cudaEventSynchronize(m->ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, m->ev0, m->ev1);
    info->iters = h.iters;
    info->outer_iters = 0;
    info->rel_res = h.bb > 0 ? sqrt(h.rr / h.bb) : 0.0;
    info->status = st;
    info->ms = ms;
  }
  if (st == FNPF_ENOCONV) m->err = "CG reached max_iter before the tolerance";
  else if (st == FNPF_EBREAKDOWN) m->err = "CG breakdown (p^T A p <= 0 or non-finite)";
  else if (st == FNPF_EDIVERGED) m->err = "non-finite state or eta + h <= 0";
  return st;
}

}  // namespace fnpf

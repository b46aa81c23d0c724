// C entry points of the compute path (operator, solve, DtN, right-hand side,
// RK4 step).  See include/fnpf.h for the contract of each call.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mesh.cuh"

using fnpf::Geom;

namespace {

fnpf_status cuda_fail(fnpf_mesh* m, cudaError_t e, const char* what) {
  m->err = std::string(what) + ": " + cudaGetErrorString(e);
  return FNPF_ECUDA;
}

// Laplace solve into the mesh-owned potential (or the caller's) and copy the
// Dirichlet data into its surface plane.
fnpf_status solve_into(fnpf_mesh* m, const double* eta, const double* phis, double* phi, fnpf_solve_info* info,
                       cudaStream_t s) {
  const Geom& g = m->g;
  fnpf_status st = fnpf::cg_solve(m, eta, phis, phi, info, s);
  cudaError_t e = cudaMemcpyAsync(phi + g.NI, phis, g.ns * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(m, e, "copy surface plane");
  return st;
}

}  // namespace

extern "C" {

fnpf_status fnpf_apply(fnpf_mesh* m, const double* eta, const double* x, double* y, void* stream) {
  if (!m || !eta || !x || !y) return FNPF_EINVAL;
  const Geom& g = m->g;
  cudaError_t e = fnpf::launch_apply<double>(g, m->tables(), eta, x, x + g.NI, y, y + g.NI, m->ring, m->variant64,
                                             (cudaStream_t)stream);
  return e == cudaSuccess ? FNPF_OK : cuda_fail(m, e, "apply");
}

fnpf_status fnpf_apply_f32(fnpf_mesh* m, const float* eta, const float* x, float* y, void* stream) {
  if (!m || !eta || !x || !y) return FNPF_EINVAL;
  const Geom& g = m->g;
  cudaError_t e = fnpf::launch_apply<float>(g, m->tables32(), eta, x, x + g.NI, y, y + g.NI,
                                            reinterpret_cast<float*>(m->ring), m->variant32, (cudaStream_t)stream);
  return e == cudaSuccess ? FNPF_OK : cuda_fail(m, e, "apply_f32");
}

fnpf_status fnpf_diagonal(fnpf_mesh* m, const double* eta, double* d, void* stream) {
  if (!m || !eta || !d) return FNPF_EINVAL;
  const Geom& g = m->g;
  cudaError_t e = fnpf::launch_diag<double>(g, m->tables(), eta, d, d + g.NI, m->ring, (cudaStream_t)stream);
  return e == cudaSuccess ? FNPF_OK : cuda_fail(m, e, "diagonal");
}

fnpf_status fnpf_precond_apply(fnpf_mesh* m, const double* eta, const double* r, double* z, void* stream) {
  if (!m || !eta || !r || !z) return FNPF_EINVAL;
  return fnpf::precond_apply(m, eta, r, z, (cudaStream_t)stream);
}

fnpf_status fnpf_laplace_solve(fnpf_mesh* m, const double* eta, const double* phis, double* phi,
                               fnpf_solve_info* info, void* stream) {
  if (!m || !eta || !phis || !phi) return FNPF_EINVAL;
  return solve_into(m, eta, phis, phi, info, (cudaStream_t)stream);
}

fnpf_status fnpf_dtn(fnpf_mesh* m, const double* eta, const double* phis, double* w, fnpf_solve_info* info,
                     void* stream) {
  if (!m || !eta || !phis || !w) return FNPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  fnpf_status st = solve_into(m, eta, phis, m->phi, info, s);
  if (st != FNPF_OK) return st;
  cudaError_t e = fnpf::launch_w(m->g, m->tables(), m->geom_eta(eta), phis, m->phi, w, s);
  m->launches += 1;
  return e == cudaSuccess ? FNPF_OK : cuda_fail(m, e, "w recovery");
}

fnpf_status fnpf_zakharov_rhs(fnpf_mesh* m, const double* eta, const double* phis, const double* w, double* deta,
                              double* dphis, void* stream) {
  if (!m || !eta || !phis || !w || !deta || !dphis) return FNPF_EINVAL;
  fnpf::StageArgs a{};
  a.eta = eta;
  a.geo = m->geom_eta(eta);
  a.linear = m->linear() ? 1 : 0;
  a.phis = phis;
  a.w_in = w;
  a.deta = deta;
  a.dphis = dphis;
  cudaError_t e = cudaSuccess;
  if (m->dealias_M > 0 && !m->linear()) {
    e = fnpf::enqueue_dealias_rhs(m, eta, phis, w, (cudaStream_t)stream);
    a.rhs_in = fnpf::dealias_rhs(m);
  }
  if (e == cudaSuccess) e = fnpf::launch_stage(m->g, m->tables(), a, (cudaStream_t)stream);
  return e == cudaSuccess ? FNPF_OK : cuda_fail(m, e, "rhs");
}

}  // extern "C"

namespace fnpf {

// Stage arguments of RK4 stage st (0..3) reading the stage state (ce, cp).
StageArgs stage_args(fnpf_mesh* m, double* eta, double* phis, const double* ce, const double* cp, int st, double t,
                     double dt, const double* t_dev) {
  static const double bw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const double cn[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  StageArgs a{};
  a.eta = ce;
  a.geo = m->geom_eta(ce);
  a.linear = m->linear() ? 1 : 0;
  a.phis = cp;
  a.phi = m->phi;
  a.y0_eta = eta;
  a.y0_phi = phis;
  a.acc_eta = m->acc_eta;
  a.acc_phi = m->acc_phi;
  a.out_eta = st < 3 ? m->s_eta[st & 1] : eta;
  a.out_phi = st < 3 ? m->s_phi[st & 1] : phis;
  a.bw = bw[st];
  a.cn = cn[st];
  a.dt = dt;
  a.first = st == 0;
  a.last = st == 3;
  a.status = &m->sc->status;
  if (st == 3 && m->relax_on) {
    a.cr = m->rx_cr;
    a.gen = m->rx_gen;
    a.xs = m->dxs;
    a.ys = m->dys;
    a.amp = m->relax.amp;
    a.kx = m->relax.kx;
    a.ky = m->relax.ky;
    a.omega = m->relax.omega;
    a.phase = m->relax.phase;
    a.ramp_time = m->relax.ramp_time;
    a.t_end = t + dt;
    a.t_dev = t_dev;
  }
  return a;
}

// The stage kernel, preceded (when set) by the over-integrated right-hand
// side of the stage state, which it then reads.
cudaError_t launch_stage_rhs(fnpf_mesh* m, StageArgs a, cudaStream_t s) {
  if (m->dealias_M > 0 && !m->linear()) {
    cudaError_t e = enqueue_dealias_rhs(m, a.eta, a.phis, nullptr, s);
    if (e != cudaSuccess) return e;
    a.rhs_in = dealias_rhs(m);
  }
  return launch_stage(m->g, m->tables(), a, s);
}

// Step 4.7 filtering of the new state (eta, phis) in place, through the free
// stage buffers, when a filter is set.
cudaError_t enqueue_filter_step(fnpf_mesh* m, double* eta, double* phis, cudaStream_t s) {
  if (!m->filter_on) return cudaSuccess;
  const size_t bytes = m->g.ns * sizeof(double);
  cudaError_t e = launch_filter(m->g, m->dfilter, eta, m->s_eta[0], phis, m->s_phi[0], s);
  if (e == cudaSuccess) e = memcpy_async(eta, m->s_eta[0], bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = memcpy_async(phis, m->s_phi[0], bytes, cudaMemcpyDeviceToDevice, s);
  m->launches += 1;
  return e;
}

// Captures one RK4 step of mesh m (state arrays eta, phis, step dt; the time is
// read from m->t_dev) on the capturing stream s: four device-driven solves and
// stage kernels, then the per-stage summaries copied to pinned host memory.
cudaError_t enqueue_step(fnpf_mesh* m, double* eta, double* phis, double dt, cudaStream_t s) {
  const double* ce = eta;
  const double* cp = phis;
  for (int st = 0; st < 4; ++st) {
    cudaError_t e = enqueue_solve_device(m, ce, cp, m->phi, m->stage_info + st, s, st == 0);
    if (e != cudaSuccess) return e;
    if (m->tape_on && (e = enqueue_tape_record(m, st, ce, cp, s)) != cudaSuccess) return e;
    const StageArgs a = stage_args(m, eta, phis, ce, cp, st, 0.0, dt, m->t_dev);
    if ((e = launch_stage_rhs(m, a, s)) != cudaSuccess) return e;
    ce = a.out_eta;
    cp = a.out_phi;
  }
  cudaError_t e = enqueue_filter_step(m, eta, phis, s);
  if (e != cudaSuccess) return e;
  return memcpy_async(m->stage_info_host, m->stage_info, 4 * sizeof(StageInfo), cudaMemcpyDeviceToHost, s);
}

// Reads the per-stage summaries after a replayed step (stream synchronised) and,
// with count, adds the kernels the replay executed to the launch counter: the
// top-level kernel nodes plus the loop bodies once per body execution (a CG
// body holds two iterations).
fnpf_status read_step_info(fnpf_mesh* m, fnpf_solve_info* info, float ms, bool count) {
  fnpf_status st = FNPF_OK;
  const bool mixed = m->opts.precision == FNPF_MIXED;
  if (count) m->launches += m->step_kernels;
  for (int k = 0; k < 4; ++k) {
    const StageInfo& si = m->stage_info_host[k];
    if (!count) {
    } else if (mixed) {
      m->launches += si.outer * m->body_kernels[0] + (si.iters + 1) / 2 * m->body_kernels[1];
    } else {
      m->launches += (si.iters + 1) / 2 * m->body_kernels[0];
    }
    if (si.status != 0 && st == FNPF_OK) st = (fnpf_status)si.status;
    if (info) {
      info[k].iters = si.iters;
      info[k].outer_iters = si.outer;
      info[k].rel_res = si.bb > 0 ? sqrt(si.rr / si.bb) : 0.0;
      info[k].status = si.status;
      info[k].ms = ms / 4;
    }
  }
  if (st == FNPF_ENOCONV) m->err = "solver reached its iteration cap before the tolerance";
  else if (st == FNPF_EBREAKDOWN) m->err = "CG breakdown (p^T A p <= 0 or non-finite)";
  else if (st == FNPF_EDIVERGED) m->err = "non-finite state or eta + h <= 0";
  return st;
}

cudaError_t build_step_graph(fnpf_mesh* m, double* eta, double* phis, double dt) {
  if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
  m->step_exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(m->gstream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t e1 = enqueue_step(m, eta, phis, dt, m->gstream);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(m->gstream, &graph);
  if (e1 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return e1;
  }
  if (e2 != cudaSuccess) return e2;
  m->step_kernels = graph_kernel_nodes(graph);
  e = cudaGraphInstantiate(&m->step_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  m->step_key[0] = eta;
  m->step_key[1] = phis;
  m->step_dt = dt;
  return cudaSuccess;
}

bool graph_mode(const fnpf_mesh* m) { return m->opts.use_graphs && !m->prof_on && m->warm; }

}  // namespace fnpf

namespace fnpf {

// The RK4 step of fnpf_rk4_step (graph replay or host-driven).
fnpf_status rk4_step_run(fnpf_mesh* m, double* eta, double* phis, double t, double dt, fnpf_solve_info* info,
                              cudaStream_t s) {
  if (fnpf::graph_mode(m)) {
    // one replay of the captured step: no host work between the kernels
    if (!m->step_exec || m->step_key[0] != eta || m->step_key[1] != phis || m->step_dt != dt) {
      cudaError_t e = fnpf::build_step_graph(m, eta, phis, dt);
      if (e != cudaSuccess) return cuda_fail(m, e, "step graph capture");
    }
    *m->t_host = t;
    cudaError_t e = cudaMemcpyAsync(m->t_dev, m->t_host, sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && info) e = cudaEventRecord(m->ev0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(m->step_exec, s);
    if (e == cudaSuccess && info) e = cudaEventRecord(m->ev1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(m, e, "step graph");
    float ms = 0;
    if (info) cudaEventElapsedTime(&ms, m->ev0, m->ev1);
    return fnpf::read_step_info(m, info, ms);
  }
  const double* ce = eta;
  const double* cp = phis;
  for (int st = 0; st < 4; ++st) {
    fnpf_status r = fnpf::cg_solve(m, ce, cp, m->phi, info ? info + st : nullptr, s);
    if (r != FNPF_OK) return r;
    if (m->tape_on) {
      cudaError_t e = fnpf::enqueue_tape_record(m, st, ce, cp, s);
      if (e != cudaSuccess) return cuda_fail(m, e, "tape");
    }
    const fnpf::StageArgs a = fnpf::stage_args(m, eta, phis, ce, cp, st, t, dt, nullptr);
    cudaError_t e = fnpf::launch_stage_rhs(m, a, s);
    m->launches += 1;
    if (e != cudaSuccess) return cuda_fail(m, e, "stage");
    ce = a.out_eta;
    cp = a.out_phi;
  }
  cudaError_t e = fnpf::enqueue_filter_step(m, eta, phis, s);
  if (e != cudaSuccess) return cuda_fail(m, e, "filter");
  m->warm = true;
  return FNPF_OK;
}

}  // namespace fnpf

extern "C" {

fnpf_status fnpf_rk4_step(fnpf_mesh* m, double* eta, double* phis, double t, double dt, fnpf_solve_info* info,
                          void* stream) {
  if (!m || !eta || !phis || !(dt > 0) || !isfinite(dt)) return FNPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (m->tape_on) {
    // the slot this step records into, read on the device by the tape kernels
    if (m->tape_next >= m->tape_cap) {
      m->err = "tape full: fnpf_tape_begin with more slots";
      return FNPF_EINVAL;
    }
    *m->tape_slot_host = m->tape_next;
    cudaError_t e = cudaMemcpyAsync(m->tape_slot_dev, m->tape_slot_host, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(m, e, "tape slot");
  }
  fnpf_status done = fnpf::rk4_step_run(m, eta, phis, t, dt, info, s);
  if (done == FNPF_OK && m->tape_on) ++m->tape_next;
  return done;
}

fnpf_status fnpf_set_relaxation(fnpf_mesh* m, const fnpf_relaxation* r) {
  if (!m || !r) return FNPF_EINVAL;
  if (!r->cr) {
    m->relax_on = false;
    return FNPF_OK;
  }
  if (!r->gen || !(r->ramp_time > 0) || !(r->omega > 0)) {
    m->err = "relaxation needs gen, omega > 0 and ramp_time > 0";
    return FNPF_EINVAL;
  }
  const Geom& g = m->g;
  for (int c = 0; c < g.ns; ++c)
    if (!(r->cr[c] >= 0.0 && r->cr[c] <= 1.0)) {
      m->err = "relaxation weights must lie in [0, 1]";
      return FNPF_EINVAL;
    }
  const size_t bytes = g.ns * sizeof(double);
  double** bufs[] = {&m->rx_cr, &m->rx_gen, &m->dxs, &m->dys};
  for (double** b : bufs)
    if (!*b) {
      cudaError_t e = cudaMalloc((void**)b, bytes);
      if (e != cudaSuccess) {
        *b = nullptr;
        m->err = "cannot allocate relaxation arrays";
        return FNPF_ENOMEM;
      }
    }
  cudaError_t e = cudaMemcpy(m->rx_cr, r->cr, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->rx_gen, r->gen, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dxs, m->xs.data(), bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dys, m->ys.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(m, e, "relaxation upload");
  m->relax = *r;
  m->relax.cr = nullptr;
  m->relax.gen = nullptr;
  m->relax_on = true;
  return FNPF_OK;
}

fnpf_status fnpf_set_filter(fnpf_mesh* m, const fnpf_filter* f) {
  if (!m) return FNPF_EINVAL;
  const int p = m->g.p, n = m->g.n;
  if (f && !(f->alpha >= 0.0 && std::isfinite(f->alpha))) {
    m->err = "filter alpha must be finite and >= 0";
    return FNPF_EINVAL;
  }
  if (f && f->alpha > 0.0 && (f->order < 1 || f->cutoff < 0 || f->cutoff >= p)) {
    m->err = "filter order must be >= 1 and cutoff in 0..p-1";
    return FNPF_EINVAL;
  }
  // the captured step includes or omits the filter
  if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
  m->step_exec = nullptr;
  if (!f || f->alpha == 0.0) {
    m->filter_on = false;
    return FNPF_OK;
  }
  // V_ij = P~_j(xi_i) (orthonormal Legendre at the GLL nodes), F = V diag(sigma) V^-1
  std::vector<double> V(n * n), Vi(n * n, 0.0), F(n * n, 0.0), sig(n, 1.0);
  for (int i = 0; i < n; ++i) {
    const double x = m->xi[i];
    double pm = 1.0, pc = x;
    for (int j = 0; j < n; ++j) {
      double pj;
      if (j == 0) pj = 1.0;
      else if (j == 1) pj = x;
      else {
        pj = ((2.0 * j - 1.0) * x * pc - (j - 1.0) * pm) / j;
        pm = pc;
        pc = pj;
      }
      V[i * n + j] = pj * std::sqrt((2.0 * j + 1.0) / 2.0);
    }
  }
  for (int k = f->cutoff + 1; k <= p; ++k)
    sig[k] = std::exp(-f->alpha * std::pow((double)(k - f->cutoff) / (double)(p - f->cutoff), f->order));
  // V^-1 by Gauss-Jordan elimination with partial pivoting (n <= 9)
  std::vector<double> A = V;
  for (int i = 0; i < n; ++i) Vi[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) {
      m->err = "singular Vandermonde matrix";
      return FNPF_EINVAL;
    }
    for (int k = 0; k < n; ++k) {
      std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(Vi[c * n + k], Vi[piv * n + k]);
    }
    const double d = A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] /= d;
      Vi[c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double fr = A[r * n + c];
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= fr * A[c * n + k];
        Vi[r * n + k] -= fr * Vi[c * n + k];
      }
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += V[i * n + k] * sig[k] * Vi[k * n + j];
      F[i * n + j] = s;
    }
  cudaError_t e = cudaSuccess;
  if (!m->dfilter) e = cudaMalloc((void**)&m->dfilter, n * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(m->dfilter, F.data(), n * n * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(m, e, "filter set-up");
  m->filter_on = true;
  return FNPF_OK;
}

fnpf_status fnpf_filter_apply(fnpf_mesh* m, double* f, void* stream) {
  if (!m || !f) return FNPF_EINVAL;
  if (!m->filter_on) {
    m->err = "no filter set";
    return FNPF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = fnpf::launch_filter(m->g, m->dfilter, f, m->s_eta[0], nullptr, nullptr, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, m->s_eta[0], m->g.ns * sizeof(double), cudaMemcpyDeviceToDevice, s);
  m->launches += 1;
  return e == cudaSuccess ? FNPF_OK : cuda_fail(m, e, "filter");
}

fnpf_status fnpf_autotune(fnpf_mesh* m, const double* eta, int* variant64, int* variant32, void* stream) {
  if (!m || !eta) return FNPF_EINVAL;
  fnpf_status st = fnpf::autotune(m, eta, nullptr, (cudaStream_t)stream);
  if (variant64) *variant64 = m->variant64;
  if (variant32) *variant32 = m->variant32;
  return st;
}

fnpf_status fnpf_set_shapes(fnpf_mesh* m, int variant64, int variant32) {
  if (!m) return FNPF_EINVAL;
  const int nv = fnpf::apply_variants(m->g.n, m->g.dim);
  if (variant64 < 0 || variant64 >= nv || variant32 < 0 || variant32 >= nv) {
    m->err = "shape index out of range";
    return FNPF_EINVAL;
  }
  m->variant64 = variant64;
  m->variant32 = variant32;
  m->tuned = true;
  for (GraphSlot& gs : m->g_iter) fnpf::graph_reset(&gs);   // captured launches use the shapes
  if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
  m->step_exec = nullptr;
  return FNPF_OK;
}

fnpf_status fnpf_get_shapes(const fnpf_mesh* m, int* variant64, int* variant32, int* columns64, int* columns32) {
  if (!m) return FNPF_EINVAL;
  if (variant64) *variant64 = m->variant64;
  if (variant32) *variant32 = m->variant32;
  if (columns64) *columns64 = fnpf::cta_columns(m->g.n, m->g.dim, m->variant64);
  if (columns32) *columns32 = fnpf::cta_columns(m->g.n, m->g.dim, m->variant32);
  return FNPF_OK;
}

fnpf_status fnpf_profile_enable(fnpf_mesh* m, int on) {
  if (!m) return FNPF_EINVAL;
  if (on && m->prof_ev.empty()) {
    const int pairs = std::max(64, m->opts.check_every + 8);
    m->prof_ev.resize(2 * pairs);
    m->prof_it.assign(pairs, -1);
    m->prof_fp32.assign(pairs, 0);
    for (auto& e : m->prof_ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return cuda_fail(m, r, "profile events");
    }
  }
  m->prof_on = on != 0;
  return FNPF_OK;
}

fnpf_status fnpf_profile_read(fnpf_mesh* m, double* apply_ms, int64_t* apply_count, int64_t* kernel_launches,
                              int reset) {
  if (!m) return FNPF_EINVAL;
  if (apply_ms) *apply_ms = m->prof_ms;
  if (apply_count) *apply_count = m->prof_count;
  if (kernel_launches) *kernel_launches = m->launches;
  if (reset) {
    m->prof_ms = 0;
    m->prof_count = 0;
    m->prof_ms32 = 0;
    m->prof_count32 = 0;
    m->launches = 0;
  }
  return FNPF_OK;
}

fnpf_status fnpf_profile_read_fp32(fnpf_mesh* m, double* apply_ms, int64_t* apply_count) {
  if (!m) return FNPF_EINVAL;
  if (apply_ms) *apply_ms = m->prof_ms32;
  if (apply_count) *apply_count = m->prof_count32;
  return FNPF_OK;
}

}  // extern "C"

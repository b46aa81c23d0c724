// C entry points of the compute path (operator, solve, DtN, right-hand side,
// RK4 step).  See include/fnpf.h for the contract of each call.
#include <math.h>

#include <algorithm>

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
  cudaError_t e = fnpf::launch_w(m->g, m->tables(), eta, phis, m->phi, w, s);
  m->launches += 1;
  return e == cudaSuccess ? FNPF_OK : cuda_fail(m, e, "w recovery");
}

fnpf_status fnpf_zakharov_rhs(fnpf_mesh* m, const double* eta, const double* phis, const double* w, double* deta,
                              double* dphis, void* stream) {
  if (!m || !eta || !phis || !w || !deta || !dphis) return FNPF_EINVAL;
  fnpf::StageArgs a{};
  a.eta = eta;
  a.phis = phis;
  a.w_in = w;
  a.deta = deta;
  a.dphis = dphis;
  cudaError_t e = fnpf::launch_stage(m->g, m->tables(), a, (cudaStream_t)stream);
  return e == cudaSuccess ? FNPF_OK : cuda_fail(m, e, "rhs");
}

fnpf_status fnpf_rk4_step(fnpf_mesh* m, double* eta, double* phis, double t, double dt, fnpf_solve_info* info,
                          void* stream) {
  (void)t;
  if (!m || !eta || !phis || !(dt > 0) || !isfinite(dt)) return FNPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  static const double bw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const double cn[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  const double* ce = eta;
  const double* cp = phis;
  for (int st = 0; st < 4; ++st) {
    fnpf_status r = fnpf::cg_solve(m, ce, cp, m->phi, info ? info + st : nullptr, s);
    if (r != FNPF_OK) return r;
    fnpf::StageArgs a{};
    a.eta = ce;
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
    }
    cudaError_t e = fnpf::launch_stage(m->g, m->tables(), a, s);
    m->launches += 1;
    if (e != cudaSuccess) return cuda_fail(m, e, "stage");
    ce = a.out_eta;
    cp = a.out_phi;
  }
  return FNPF_OK;
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

fnpf_status fnpf_autotune(fnpf_mesh* m, const double* eta, int* variant64, int* variant32, void* stream) {
  if (!m || !eta) return FNPF_EINVAL;
  fnpf_status st = fnpf::autotune(m, eta, nullptr, (cudaStream_t)stream);
  if (variant64) *variant64 = m->variant64;
  if (variant32) *variant32 = m->variant32;
  return st;
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

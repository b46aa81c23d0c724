// The Laplace solve, w and the RK4 step on prisms over an unstructured
// triangular surface mesh (fnpf_prism_laplace_solve, fnpf_prism_dtn,
// fnpf_prism_rhs, fnpf_prism_rk4_step; Sec. 3.1.2, Sec. 3.4 Steps 4.1-4.6,
// Sec. 3.2): the items of prism_step.h launched one thread per item on the
// caller's stream; the CG loops keep their scalars on the device and the host
// reads their state every iteration (p-multigrid) or every 8 (Jacobi).  The workspace and the surface tables (the incidence of the
// triangle slots and the consistent surface mass in CSR form) are built at a
// mesh's first call.
#include <limits.h>
#include <math.h>

#include <string>
#include <type_traits>
#include <vector>

#include "fnpf_internal.cuh"
#include "prism.cuh"
#include "prism_step.h"

namespace fnpf {

constexpr int kItemThreads = 256;

template <class It>
__global__ void __launch_bounds__(kItemThreads) pstep_kernel(int64_t n, typename It::Args a) {
  const int64_t i = (int64_t)blockIdx.x * kItemThreads + threadIdx.x;
  if (i < n) It::at(i, a);
}

// A block kernel: K's phases in order, a barrier after each, the block's
// shared memory given to every phase.
template <class K>
__global__ void __launch_bounds__(K::kThreads) pstep_block_kernel(typename K::Args a) {
  extern __shared__ __align__(16) unsigned char pstep_smem[];
  auto* sm = reinterpret_cast<typename K::value_type*>(pstep_smem);
  for (int ph = 0; ph < K::kPhases; ++ph) {
    K::phase(ph, (int64_t)blockIdx.x, (int)threadIdx.x, (int)blockDim.x, sm, a);
    __syncthreads();
  }
}

namespace {

struct DeviceEx {
  cudaStream_t s;
  template <class K>
  int run_block(int64_t blocks, size_t smem, const typename K::Args& a) {
    if (blocks < 1 || blocks > INT_MAX || smem > 48 * 1024) return 1;   // p <= 8: at most 31 KB
    pstep_block_kernel<K><<<(unsigned)blocks, K::kThreads, smem, s>>>(a);
    return cudaPeekAtLastError() != cudaSuccess;
  }
  template <class It>
  int run(int64_t n, const typename It::Args& a) {
    const int64_t blocks = (n + kItemThreads - 1) / kItemThreads;
    if (blocks < 1 || blocks > INT_MAX) return 1;
    pstep_kernel<It><<<(unsigned)blocks, kItemThreads, 0, s>>>(n, a);
    return cudaPeekAtLastError() != cudaSuccess;
  }
  int get(double* dst, const double* src, int count) {
    if (cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 1;
    return cudaStreamSynchronize(s) != cudaSuccess;
  }
};

}  // namespace

struct PrismStepState {
  pstep::PMesh pm{};
  pstep::PWork w{};
  double* d_work = nullptr;
  int64_t* d_soff = nullptr;
  int64_t* d_sinc = nullptr;
  int64_t* d_mrow = nullptr;
  int* d_mcol = nullptr;
  double* d_mval = nullptr;
  double* d_mdiag = nullptr;
  double* d_filt = nullptr;    // [nt][nt] the modal filter (at the first fnpf_prism_set_filter)
  int* d_interior = nullptr;   // [nt]
  double* d_relax = nullptr;   // [4][ns] C_r, gen, x, y (at the first fnpf_prism_set_relaxation)
  pstep::PMG pmg{};            // the p-multigrid hierarchy (at the first FNPF_PMG call)
  bool pmg_ready = false;
  std::vector<void*> pmg_bufs;
};

void prism_step_free(fnpf_prism* m) {
  if (!m || !m->step) return;
  PrismStepState* st = m->step;
  cudaFree(st->d_work);
  cudaFree(st->d_soff);
  cudaFree(st->d_sinc);
  cudaFree(st->d_mrow);
  cudaFree(st->d_mcol);
  cudaFree(st->d_mval);
  cudaFree(st->d_mdiag);
  cudaFree(st->d_filt);
  cudaFree(st->d_interior);
  cudaFree(st->d_relax);
  for (void* b : st->pmg_bufs) cudaFree(b);
  delete st;
  m->step = nullptr;
}

namespace {

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, src.size()));
  if (e == cudaSuccess && !src.empty()) e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
  return e;
}

// The step workspace of m (built at the first call; every later call reuses it).
fnpf_status ensure_step(fnpf_prism* m) {
  if (m->step) return FNPF_OK;
  PrismStepState* st = new PrismStepState();
  pstep::PMesh& pm = st->pm;
  pm.p = m->p;
  pm.n = m->n;
  pm.nz = m->nz;
  pm.nt = m->nt;
  pm.nq = m->nq;
  pm.ntri = m->ntri;
  pm.ns = m->ns;
  pm.nv = m->nv;
  pm.N = m->N;
  pm.NI = m->N - m->ns;
  pm.nelem = (int64_t)m->ntri * m->nz;
  pm.tn = m->d_tnodes;
  pm.voff = m->d_off;
  pm.vinc = m->d_inc;
  // host copy of the packed tables the kernels read (geo, L, wq for the mass matrix)
  const size_t ntab = 4 * (size_t)m->ntri + 3 * (size_t)m->nq * m->nt + m->nq + 2 * (size_t)m->n +
                      (size_t)m->n * m->n;
  std::vector<double> tab(ntab);
  cudaError_t e = cudaMemcpy(tab.data(), m->d_tab, sizeof(double) * ntab, cudaMemcpyDeviceToHost);
  pstep::PMesh hm = pm;
  pstep::bind_tables(&hm, tab.data());
  pstep::bind_tables(&pm, m->d_tab);
  std::vector<int64_t> soff, sinc, mrow;
  std::vector<int> mcol;
  std::vector<double> mval, mdiag;
  pstep::surface_incidence(m->tnodes.data(), m->ntri, m->nt, m->ns, &soff, &sinc);
  pstep::surface_mass(hm, m->tnodes.data(), hm.geo, hm.L, hm.wq, &mrow, &mcol, &mval, &mdiag);
  int64_t total = 0;
  pstep::carve(pm, &st->w, [&](double** p, int64_t cnt) {
    (void)p;
    total += (cnt + 31) / 32 * 32;   // 256-byte aligned buffers
  });
  if (e == cudaSuccess) e = cudaMalloc(&st->d_work, sizeof(double) * total);
  if (e == cudaSuccess) e = cudaMemset(st->d_work, 0, sizeof(double) * total);
  if (e == cudaSuccess) e = upload(&st->d_soff, soff);
  if (e == cudaSuccess) e = upload(&st->d_sinc, sinc);
  if (e == cudaSuccess) e = upload(&st->d_mrow, mrow);
  if (e == cudaSuccess) e = upload(&st->d_mcol, mcol);
  if (e == cudaSuccess) e = upload(&st->d_mval, mval);
  if (e == cudaSuccess) e = upload(&st->d_mdiag, mdiag);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    m->err = std::string("prism step set-up: ") + cudaGetErrorString(e);
    m->step = st;
    prism_step_free(m);
    return e == cudaErrorMemoryAllocation ? FNPF_ENOMEM : FNPF_ECUDA;
  }
  int64_t off = 0;
  pstep::carve(pm, &st->w, [&](double** p, int64_t cnt) {
    *p = st->d_work + off;
    off += (cnt + 31) / 32 * 32;
  });
  pm.soff = st->d_soff;
  pm.sinc = st->d_sinc;
  pm.mrow = st->d_mrow;
  pm.mcol = st->d_mcol;
  pm.mval = st->d_mval;
  pm.mdiag = st->d_mdiag;
  m->step = st;
  return FNPF_OK;
}

// The p-multigrid hierarchy of m on the device (built at the first FNPF_PMG call).
fnpf_status ensure_pmg(fnpf_prism* m) {
  PrismStepState* st = m->step;
  if (st->pmg_ready) return FNPF_OK;
  bool ok = true;
  auto up = [&](const auto& v) {
    using T = typename std::decay_t<decltype(v)>::value_type;
    T* d = nullptr;
    if (cudaMalloc(&d, sizeof(T) * std::max<size_t>(1, v.size())) != cudaSuccess) {
      ok = false;
      return (const T*)nullptr;
    }
    st->pmg_bufs.push_back(d);
    if (!v.empty() && cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    return (const T*)d;
  };
  auto take = [&](double** p, int64_t cnt) {
    *p = nullptr;
    double* d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * std::max<int64_t>(1, cnt)) != cudaSuccess ||
        cudaMemset(d, 0, sizeof(double) * std::max<int64_t>(1, cnt)) != cudaSuccess) {
      ok = false;
      return;
    }
    st->pmg_bufs.push_back(d);
    *p = d;
  };
  const int nverts = (int)(m->verts.size() / 2);
  const bool built = pstep::build_pmg(st->pm, st->w, m->verts.data(), nverts, m->tris.data(), m->nz, &st->pmg, up, take);
  if (ok && built && cudaDeviceSynchronize() == cudaSuccess) {
    st->pmg_ready = true;
    return FNPF_OK;
  }
  for (void* b : st->pmg_bufs) cudaFree(b);
  st->pmg_bufs.clear();
  st->pmg = pstep::PMG{};
  m->err = ok ? "prism p-multigrid set-up failed" : "prism p-multigrid: device allocation failed";
  return ok ? FNPF_EINVAL : FNPF_ENOMEM;
}

fnpf_status check_opts(const fnpf_prism_opts* o, pstep::Params* p, std::string* why) {
  fnpf_prism_opts d;
  fnpf_prism_default_opts(&d);
  if (!o) o = &d;
  if (!(o->rtol > 0) || !(o->mass_rtol > 0) || o->max_iter < 0 || o->mass_max_iter < 0 || !isfinite(o->g) ||
      (o->model != FNPF_NONLINEAR && o->model != FNPF_LINEAR) ||
      (o->precond != FNPF_JACOBI && o->precond != FNPF_PMG) || o->cheb_degree < 1 || o->coarse_iters < 1 ||
      !(o->cheb_range > 1) || !isfinite(o->cheb_range) ||
      (o->precision != FNPF_FP64 && o->precision != FNPF_FP64_PC32 && o->precision != FNPF_MIXED) ||
      o->projection < 0 || o->projection > pstep::kMaxProj || !(o->inner_rtol > 0 && o->inner_rtol < 1) ||
      o->max_outer < 1) {
    *why = "bad options (rtol, mass_rtol > 0; iteration caps >= 0; finite g; model NONLINEAR or LINEAR; precond "
           "JACOBI or PMG; Chebyshev degrees >= 1; cheb_range > 1; precision FP64, FP64_PC32 or MIXED; projection 0..8; inner_rtol in (0, 1); max_outer >= 1)";
    return FNPF_EINVAL;
  }
  *p = pstep::Params{o->rtol,         o->max_iter, o->mass_rtol,   o->mass_max_iter, o->g, o->model == FNPF_LINEAR,
                     o->precond == FNPF_PMG, o->cheb_degree, o->coarse_iters, o->cheb_range,
                     o->precond == FNPF_PMG && o->precision == FNPF_FP64_PC32, o->projection,
                     o->precond == FNPF_PMG && o->precision == FNPF_MIXED, o->inner_rtol, o->max_outer};
  return FNPF_OK;
}

// Runs f(stepper, params) after the common checks; records the message of a failure.
template <class F>
fnpf_status with_stepper(fnpf_prism* m, const fnpf_prism_opts* opts, void* stream, const char* what, F f) {
  pstep::Params prm{};
  std::string why;
  fnpf_status st = check_opts(opts, &prm, &why);
  if (st != FNPF_OK) {
    m->err = std::string(what) + ": " + why;
    return st;
  }
  if ((st = ensure_step(m)) != FNPF_OK) return st;
  if (prm.pmg && (st = ensure_pmg(m)) != FNPF_OK) return st;
  DeviceEx ex{(cudaStream_t)stream};
  pstep::Stepper<DeviceEx> sp{m->step->pm, m->step->w, ex, prm.pmg ? &m->step->pmg : nullptr};
  st = f(sp, prm);
  if (st == FNPF_ECUDA) {
    m->err = std::string(what) + ": " + cudaGetErrorString(cudaGetLastError());
  } else if (st != FNPF_OK) {
    m->err = std::string(what) + ": " + fnpf_status_string(st);
  }
  return st;
}

}  // namespace
}  // namespace fnpf

extern "C" {

void fnpf_prism_default_opts(fnpf_prism_opts* o) {
  if (!o) return;
  o->rtol = 1e-10;
  o->max_iter = 20000;
  o->mass_rtol = 1e-13;
  o->mass_max_iter = 5000;
  o->g = 9.81;
  o->model = FNPF_NONLINEAR;
  o->precond = FNPF_JACOBI;
  o->cheb_degree = 3;
  o->coarse_iters = 6;
  o->cheb_range = 40.0;
  o->precision = FNPF_FP64;
  o->projection = 0;
  o->inner_rtol = 1e-5;
  o->max_outer = 20;
}

fnpf_status fnpf_prism_diagonal(fnpf_prism* m, const double* eta, const double* h, double* diag, void* stream) {
  if (!m || !eta || !h || !diag) return FNPF_EINVAL;
  return fnpf::with_stepper(m, nullptr, stream, "prism diagonal", [&](auto& sp, const fnpf::pstep::Params&) {
    fnpf_status st = sp.geometry(eta, h);
    if (st == FNPF_OK) st = sp.template go<fnpf::pstep::CopyItem>(m->N, {sp.w.diag, diag});
    return st;
  });
}

fnpf_status fnpf_prism_apply_stored(fnpf_prism* m, const double* eta, const double* h, const double* x, double* y,
                                    void* stream) {
  if (!m || !eta || !h || !x || !y) return FNPF_EINVAL;
  return fnpf::with_stepper(m, nullptr, stream, "prism stored apply", [&](auto& sp, const fnpf::pstep::Params&) {
    fnpf_status st = sp.geometry(eta, h);
    if (st == FNPF_OK) st = sp.apply(x, y);
    return st;
  });
}

fnpf_status fnpf_prism_precond_apply(fnpf_prism* m, const fnpf_prism_opts* opts, const double* eta, const double* h,
                                     const double* r, double* z, void* stream) {
  if (!m || !eta || !h || !r || !z) return FNPF_EINVAL;
  return fnpf::with_stepper(m, opts, stream, "prism preconditioner", [&](auto& sp, const fnpf::pstep::Params& p) {
    return sp.precond_apply(eta, h, r, z, p);
  });
}

fnpf_status fnpf_prism_laplace_solve(fnpf_prism* m, const fnpf_prism_opts* opts, const double* eta, const double* h,
                                     const double* phis, double* phi, fnpf_solve_info* info, void* stream) {
  if (!m || !eta || !h || !phis || !phi) return FNPF_EINVAL;
  return fnpf::with_stepper(m, opts, stream, "prism Laplace solve", [&](auto& sp, const fnpf::pstep::Params& p) {
    return sp.solve(eta, h, phis, phi, p, info);
  });
}

fnpf_status fnpf_prism_laplace_solve_vjp(fnpf_prism* m, const fnpf_prism_opts* opts, const double* eta,
                                         const double* h, const double* phi, const double* lam_phi, double* lam_eta,
                                         double* lam_phis, double* lam_h, fnpf_solve_info* info, void* stream) {
  if (!m || !eta || !h || !phi || !lam_phi || !lam_eta || !lam_phis) return FNPF_EINVAL;
  return fnpf::with_stepper(m, opts, stream, "prism solve VJP", [&](auto& sp, const fnpf::pstep::Params& p) {
    return sp.solve_vjp(eta, h, phi, lam_phi, lam_eta, lam_phis, lam_h, p, info);
  });
}

fnpf_status fnpf_prism_step_adjoint(fnpf_prism* m, const fnpf_prism_opts* opts, const double* h, const double* eta_n,
                                    const double* phis_n, const double* lam_eta, const double* lam_phis,
                                    double* lam_eta_out, double* lam_phis_out, double* lam_h, double t, double dt,
                                    void* stream) {
  if (!m || !h || !eta_n || !phis_n || !lam_eta || !lam_phis || !lam_eta_out || !lam_phis_out || !isfinite(dt) ||
      !isfinite(t))
    return FNPF_EINVAL;
  return fnpf::with_stepper(m, opts, stream, "prism step adjoint", [&](auto& sp, const fnpf::pstep::Params& p) {
    return sp.rk4_adjoint(h, eta_n, phis_n, t, dt, lam_eta, lam_phis, lam_eta_out, lam_phis_out, lam_h, p);
  });
}

fnpf_status fnpf_prism_dtn(fnpf_prism* m, const fnpf_prism_opts* opts, const double* eta, const double* h,
                           const double* phis, double* w, fnpf_solve_info* info, void* stream) {
  if (!m || !eta || !h || !phis || !w) return FNPF_EINVAL;
  return fnpf::with_stepper(m, opts, stream, "prism DtN", [&](auto& sp, const fnpf::pstep::Params& p) {
    return sp.dtn(eta, h, phis, w, p, info);
  });
}

fnpf_status fnpf_prism_rhs(fnpf_prism* m, const fnpf_prism_opts* opts, const double* eta, const double* h,
                           const double* phis, double* k_eta, double* k_phis, fnpf_solve_info* info, void* stream) {
  if (!m || !eta || !h || !phis || !k_eta || !k_phis) return FNPF_EINVAL;
  return fnpf::with_stepper(m, opts, stream, "prism right-hand side", [&](auto& sp, const fnpf::pstep::Params& p) {
    return sp.rhs(eta, h, phis, k_eta, k_phis, p, info);
  });
}

fnpf_status fnpf_prism_set_filter(fnpf_prism* m, const fnpf_filter* f) {
  if (!m) return FNPF_EINVAL;
  if (f && (!(f->alpha >= 0) || !isfinite(f->alpha) || f->order < 1 || f->cutoff < 0 || f->cutoff >= m->p)) {
    m->err = "prism filter: alpha >= 0 and finite, order >= 1, cutoff in 0..p-1";
    return FNPF_EINVAL;
  }
  fnpf_status st = fnpf::ensure_step(m);
  if (st != FNPF_OK) return st;
  fnpf::PrismStepState* ps = m->step;
  if (!f || f->alpha == 0) {
    ps->pm.filt = nullptr;
    ps->pm.interior = nullptr;
    return FNPF_OK;
  }
  std::vector<double> rn, sn, wq, L, Lr, Ls, F;
  std::vector<int> interior;
  if (!fnpf::prism_tables(m->p, &rn, &sn, &wq, &L, &Lr, &Ls) ||
      !fnpf::pstep::triangle_filter(m->p, rn.data(), sn.data(), f->alpha, f->order, f->cutoff, &F, &interior)) {
    m->err = "prism filter: singular Vandermonde matrix";
    return FNPF_EINVAL;
  }
  cudaError_t e = cudaSuccess;
  if (!ps->d_filt) e = cudaMalloc(&ps->d_filt, sizeof(double) * F.size());
  if (e == cudaSuccess && !ps->d_interior) e = cudaMalloc(&ps->d_interior, sizeof(int) * interior.size());
  if (e == cudaSuccess) e = cudaMemcpy(ps->d_filt, F.data(), sizeof(double) * F.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ps->d_interior, interior.data(), sizeof(int) * interior.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    m->err = std::string("prism filter: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FNPF_ENOMEM : FNPF_ECUDA;
  }
  ps->pm.filt = ps->d_filt;
  ps->pm.interior = ps->d_interior;
  return FNPF_OK;
}

fnpf_status fnpf_prism_filter_apply(fnpf_prism* m, double* f, void* stream) {
  if (!m || !f) return FNPF_EINVAL;
  if (!m->step || !m->step->pm.filt) {
    m->err = "prism filter apply: no filter set";
    return FNPF_EINVAL;
  }
  return fnpf::with_stepper(m, nullptr, stream, "prism filter apply",
                            [&](auto& sp, const fnpf::pstep::Params&) { return sp.filter(f); });
}

fnpf_status fnpf_prism_invariants(fnpf_prism* m, const fnpf_prism_opts* opts, const double* eta, const double* h,
                                  const double* phis, double* mass, double* energy, fnpf_solve_info* info,
                                  void* stream) {
  if (!m || !eta || !h || !phis || !mass || !energy) return FNPF_EINVAL;
  return fnpf::with_stepper(m, opts, stream, "prism invariants", [&](auto& sp, const fnpf::pstep::Params& p) {
    return sp.invariants(eta, h, phis, p, mass, energy, info);
  });
}

fnpf_status fnpf_prism_set_relaxation(fnpf_prism* m, const fnpf_relaxation* r) {
  if (!m) return FNPF_EINVAL;
  fnpf_status st = fnpf::ensure_step(m);
  if (st != FNPF_OK) return st;
  fnpf::pstep::PMesh& pm = m->step->pm;
  if (!r || !r->cr) {
    pm.rcr = pm.rgen = pm.xs = pm.ys = nullptr;
    return FNPF_OK;
  }
  bool gen = false;
  for (int c = 0; c < m->ns; ++c) {
    if (!(r->cr[c] >= 0 && r->cr[c] <= 1) || !r->gen || !isfinite(r->gen[c])) {
      m->err = "prism relaxation: cr in [0, 1] and a finite gen flag at every node";
      return FNPF_EINVAL;
    }
    gen = gen || (r->gen[c] != 0 && r->cr[c] > 0);
  }
  if (!(r->ramp_time > 0) || !isfinite(r->amp) || !isfinite(r->kx) || !isfinite(r->ky) || !isfinite(r->phase) ||
      (gen && !(r->omega > 0))) {
    m->err = "prism relaxation: ramp_time > 0, finite wave parameters, omega > 0 with generation nodes";
    return FNPF_EINVAL;
  }
  std::vector<double> host(4 * (size_t)m->ns);
  for (int c = 0; c < m->ns; ++c) {
    host[c] = r->cr[c];
    host[m->ns + c] = r->gen[c];
    host[2 * (size_t)m->ns + c] = m->xs[c];
    host[3 * (size_t)m->ns + c] = m->ys[c];
  }
  fnpf::PrismStepState* ps = m->step;
  cudaError_t e = cudaSuccess;
  if (!ps->d_relax) e = cudaMalloc(&ps->d_relax, sizeof(double) * host.size());
  if (e == cudaSuccess) e = cudaMemcpy(ps->d_relax, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    m->err = std::string("prism relaxation: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FNPF_ENOMEM : FNPF_ECUDA;
  }
  pm.rcr = ps->d_relax;
  pm.rgen = ps->d_relax + m->ns;
  pm.xs = ps->d_relax + 2 * (size_t)m->ns;
  pm.ys = ps->d_relax + 3 * (size_t)m->ns;
  pm.ramp = r->ramp_time;
  pm.amp = r->amp;
  pm.kx = r->kx;
  pm.ky = r->ky;
  pm.omega = r->omega;
  pm.phase = r->phase;
  return FNPF_OK;
}

fnpf_status fnpf_prism_rk4_step(fnpf_prism* m, const fnpf_prism_opts* opts, const double* h, double* eta,
                                double* phis, double t, double dt, fnpf_solve_info* info, void* stream) {
  if (!m || !h || !eta || !phis || !isfinite(dt) || !isfinite(t)) return FNPF_EINVAL;
  return fnpf::with_stepper(m, opts, stream, "prism RK4 step", [&](auto& sp, const fnpf::pstep::Params& p) {
    return sp.rk4(h, eta, phis, t, dt, p, info);
  });
}

}  // extern "C"

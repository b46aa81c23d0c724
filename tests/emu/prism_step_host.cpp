// Test harness (tests only): the items and the orchestration of the prism
// solve and step (paper_2506_09435_gb300/csrc/prism_step.h) compiled as plain
// C++ and run one item after another on host memory, so that a CPU test can
// compare the kernels' own index arithmetic and arithmetic with the oracle
// before they run on a GPU.  The mesh set-up calls the library's host
// functions (numbering, triangle tables, GLL tables) and repeats the packing
// of fnpf_prism_create; every table and workspace buffer is a separate
// allocation of its exact size, so that a build with AddressSanitizer reports
// any access outside a buffer.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <type_traits>
#include <vector>

#include "fnpf.h"
#include "prism_step.h"

namespace {

using namespace fnpf::pstep;

struct HostEx {
  int64_t launches = 0;
  template <class It>
  int run(int64_t n, const typename It::Args& a) {
    ++launches;
    for (int64_t i = 0; i < n; ++i) It::at(i, a);
    return 0;
  }
  // A block kernel: for every block, each phase for every thread of the block
  // before the next phase (the barrier), on a shared array of exactly the
  // requested size.
  template <class K>
  int run_block(int64_t blocks, size_t smem, const typename K::Args& a) {
    ++launches;
    using T = typename K::value_type;
    std::unique_ptr<T[]> sm(new T[smem / sizeof(T)]);
    for (int64_t b = 0; b < blocks; ++b)
      for (int ph = 0; ph < K::kPhases; ++ph)
        for (int tid = 0; tid < K::kThreads; ++tid) K::phase(ph, b, tid, K::kThreads, sm.get(), a);
    return 0;
  }
  int get(double* dst, const double* src, int count) {
    memcpy(dst, src, sizeof(double) * count);
    return 0;
  }
};

struct Emu {
  PMesh m{};
  PWork w{};
  std::vector<std::unique_ptr<double[]>> dbufs;
  std::vector<int> tn, mcol, interior;
  std::vector<int64_t> voff, vinc, soff, sinc, mrow;
  std::vector<double> mval, mdiag;
  std::vector<double> verts, xs, ys;
  std::vector<int> tris;
  int nz = 0;
  PMG pmg{};
  bool pmg_ready = false;
  std::vector<std::shared_ptr<void>> pbufs;   // hierarchy tables, each its own allocation
  HostEx ex;

  bool ensure_pmg() {
    if (pmg_ready) return true;
    auto up = [this](const auto& v) {
      using T = typename std::decay_t<decltype(v)>::value_type;
      std::shared_ptr<T> b(new T[std::max<size_t>(1, v.size())](), std::default_delete<T[]>());
      std::copy(v.begin(), v.end(), b.get());
      pbufs.push_back(b);
      return (const T*)b.get();
    };
    auto take = [this](double** p, int64_t cnt) {
      dbufs.emplace_back(new double[cnt > 0 ? cnt : 1]());
      *p = dbufs.back().get();
    };
    pmg_ready = build_pmg(m, w, verts.data(), (int)(verts.size() / 2), tris.data(), nz, &pmg, up, take);
    return pmg_ready;
  }

  const double* table(const std::vector<double>& v, size_t off, size_t count) {
    dbufs.emplace_back(new double[count]);
    memcpy(dbufs.back().get(), v.data() + off, sizeof(double) * count);
    return dbufs.back().get();
  }
};

}  // namespace

extern "C" {

void* emu_create(const double* verts, int nverts, const int* tris, int ntris, int p, int nz) {
  std::unique_ptr<Emu> e(new Emu());
  e->verts.assign(verts, verts + 2 * (size_t)nverts);
  e->tris.assign(tris, tris + 3 * (size_t)ntris);
  e->nz = nz;
  std::vector<double>& xs = e->xs;
  std::vector<double>& ys = e->ys;
  if (!fnpf::prism_numbering(verts, nverts, tris, ntris, p, &e->tn, &xs, &ys)) return nullptr;
  std::vector<double> rn, sn, wq, L, Lr, Ls;
  if (!fnpf::prism_tables(p, &rn, &sn, &wq, &L, &Lr, &Ls)) return nullptr;
  PMesh& m = e->m;
  m.p = p;
  m.n = p + 1;
  m.nz = nz;
  m.nt = (int)rn.size();
  m.nq = (int)wq.size();
  m.ntri = ntris;
  m.ns = (int64_t)xs.size();
  m.nv = (int64_t)nz * p + 1;
  m.N = m.nv * m.ns;
  m.NI = m.N - m.ns;
  m.nelem = (int64_t)ntris * nz;
  const int n = m.n, nt = m.nt;
  std::vector<double> geo(4 * (size_t)ntris);
  for (int t = 0; t < ntris; ++t) {
    const int A = tris[3 * t], B = tris[3 * t + 1], C = tris[3 * t + 2];
    geo[4 * t] = 0.5 * (verts[2 * B] - verts[2 * A]);
    geo[4 * t + 1] = 0.5 * (verts[2 * C] - verts[2 * A]);
    geo[4 * t + 2] = 0.5 * (verts[2 * B + 1] - verts[2 * A + 1]);
    geo[4 * t + 3] = 0.5 * (verts[2 * C + 1] - verts[2 * A + 1]);
  }
  std::vector<double> xi(n), wv(n), D(n * n);
  fnpf::gll_tables(p, xi.data(), wv.data(), D.data());
  m.tn = e->tn.data();
  m.geo = e->table(geo, 0, geo.size());
  m.L = e->table(L, 0, L.size());
  m.Lr = e->table(Lr, 0, Lr.size());
  m.Ls = e->table(Ls, 0, Ls.size());
  m.wq = e->table(wq, 0, wq.size());
  m.xi = e->table(xi, 0, xi.size());
  m.wv = e->table(wv, 0, wv.size());
  m.D = e->table(D, 0, D.size());
  // volume incidence in (element, local node) order, as fnpf_prism_create
  volume_incidence(e->tn.data(), ntris, nt, nz, p, m.ns, &e->voff, &e->vinc);
  m.voff = e->voff.data();
  m.vinc = e->vinc.data();
  surface_incidence(e->tn.data(), ntris, nt, m.ns, &e->soff, &e->sinc);
  surface_mass(m, e->tn.data(), m.geo, m.L, m.wq, &e->mrow, &e->mcol, &e->mval, &e->mdiag);
  m.soff = e->soff.data();
  m.sinc = e->sinc.data();
  m.mrow = e->mrow.data();
  m.mcol = e->mcol.data();
  m.mval = e->mval.data();
  m.mdiag = e->mdiag.data();
  Emu* ep = e.get();
  carve(m, &e->w, [ep](double** ptr, int64_t cnt) {
    ep->dbufs.emplace_back(new double[cnt > 0 ? cnt : 1]());
    *ptr = ep->dbufs.back().get();
  });
  return e.release();
}

void emu_destroy(void* h) { delete static_cast<Emu*>(h); }

void emu_sizes(void* h, int64_t* N, int64_t* ns, int64_t* launches) {
  Emu* e = static_cast<Emu*>(h);
  *N = e->m.N;
  *ns = e->m.ns;
  *launches = e->ex.launches;
}

static Params params(const fnpf_prism_opts* o) {
  fnpf_prism_opts d;
  fnpf_prism_default_opts(&d);
  if (!o) o = &d;
  return Params{o->rtol,         o->max_iter,    o->mass_rtol,    o->mass_max_iter, o->g, o->model == FNPF_LINEAR,
                o->precond == FNPF_PMG, o->cheb_degree, o->coarse_iters, o->cheb_range,
                o->precond == FNPF_PMG && o->precision == FNPF_FP64_PC32, o->projection,
                o->precond == FNPF_PMG && o->precision == FNPF_MIXED, o->inner_rtol, o->max_outer};
}

// A stepper over the harness's memory (with the hierarchy when the options ask for it).
static Stepper<HostEx> stepper(Emu* e, const Params& prm) {
  Stepper<HostEx> sp{e->m, e->w, e->ex};
  if (prm.pmg && e->ensure_pmg()) sp.pmg = &e->pmg;
  return sp;
}

int emu_diagonal(void* h, const double* eta, const double* hh, double* diag) {
  Emu* e = static_cast<Emu*>(h);
  Stepper<HostEx> sp{e->m, e->w, e->ex};
  fnpf_status st = sp.geometry(eta, hh);
  if (st == FNPF_OK) st = sp.go<CopyItem>(e->m.N, {e->w.diag, diag});
  return st;
}

int emu_apply_stored(void* h, const double* eta, const double* hh, const double* x, double* y) {
  Emu* e = static_cast<Emu*>(h);
  Stepper<HostEx> sp{e->m, e->w, e->ex};
  fnpf_status st = sp.geometry(eta, hh);
  if (st == FNPF_OK) st = sp.apply(x, y);
  return st;
}

// y = A x through the one-thread-per-item operator kernels (the reference of
// the block kernel used by every other entry point).
int emu_apply_items(void* h, const double* eta, const double* hh, const double* x, double* y) {
  Emu* e = static_cast<Emu*>(h);
  Stepper<HostEx> sp{e->m, e->w, e->ex};
  fnpf_status st = sp.geometry(eta, hh);
  if (st == FNPF_OK) st = sp.elements_items(e->m, (const double*)e->w.G, e->w.F, e->w.ye, e->w.vt, x);
  if (st == FNPF_OK) st = sp.go<GatherItem>(e->m.N, {e->m.voff, e->m.vinc, e->w.ye, y});
  return st;
}

int emu_laplace_solve(void* h, const fnpf_prism_opts* o, const double* eta, const double* hh, const double* phis,
                      double* phi, fnpf_solve_info* info) {
  Emu* e = static_cast<Emu*>(h);
  const Params prm = params(o);
  Stepper<HostEx> sp = stepper(e, prm);
  return sp.solve(eta, hh, phis, phi, prm, info);
}

int emu_precond_apply(void* h, const fnpf_prism_opts* o, const double* eta, const double* hh, const double* r,
                      double* z) {
  Emu* e = static_cast<Emu*>(h);
  const Params prm = params(o);
  Stepper<HostEx> sp = stepper(e, prm);
  return sp.precond_apply(eta, hh, r, z, prm);
}

int emu_laplace_solve_vjp(void* h, const fnpf_prism_opts* o, const double* eta, const double* hh, const double* phi,
                          const double* lam, double* lam_eta, double* lam_phis, double* lam_h) {
  Emu* e = static_cast<Emu*>(h);
  const Params prm = params(o);
  Stepper<HostEx> sp = stepper(e, prm);
  return sp.solve_vjp(eta, hh, phi, lam, lam_eta, lam_phis, lam_h, prm, nullptr);
}

int emu_step_adjoint(void* h, const fnpf_prism_opts* o, const double* hh, const double* eta, const double* phis,
                     const double* le, const double* lp, double* oe, double* op, double* oh, double t, double dt) {
  Emu* e = static_cast<Emu*>(h);
  const Params prm = params(o);
  Stepper<HostEx> sp = stepper(e, prm);
  return sp.rk4_adjoint(hh, eta, phis, t, dt, le, lp, oe, op, oh, prm);
}

int emu_dtn(void* h, const fnpf_prism_opts* o, const double* eta, const double* hh, const double* phis, double* w,
            fnpf_solve_info* info) {
  Emu* e = static_cast<Emu*>(h);
  const Params prm = params(o);
  Stepper<HostEx> sp = stepper(e, prm);
  return sp.dtn(eta, hh, phis, w, prm, info);
}

int emu_rhs(void* h, const fnpf_prism_opts* o, const double* eta, const double* hh, const double* phis, double* ke,
            double* kp, fnpf_solve_info* info) {
  Emu* e = static_cast<Emu*>(h);
  const Params prm = params(o);
  Stepper<HostEx> sp = stepper(e, prm);
  return sp.rhs(eta, hh, phis, ke, kp, prm, info);
}

int emu_set_filter(void* h, double alpha, int order, int cutoff) {
  Emu* e = static_cast<Emu*>(h);
  if (alpha == 0) {
    e->m.filt = nullptr;
    e->m.interior = nullptr;
    return FNPF_OK;
  }
  std::vector<double> rn, sn, wq, L, Lr, Ls, F;
  std::vector<int> interior;
  if (!fnpf::prism_tables(e->m.p, &rn, &sn, &wq, &L, &Lr, &Ls) ||
      !triangle_filter(e->m.p, rn.data(), sn.data(), alpha, order, cutoff, &F, &interior))
    return FNPF_EINVAL;
  e->dbufs.emplace_back(new double[F.size()]);
  memcpy(e->dbufs.back().get(), F.data(), sizeof(double) * F.size());
  e->m.filt = e->dbufs.back().get();
  e->interior = interior;
  e->m.interior = e->interior.data();
  return FNPF_OK;
}

int emu_filter_apply(void* h, double* f) {
  Emu* e = static_cast<Emu*>(h);
  Stepper<HostEx> sp{e->m, e->w, e->ex};
  return sp.filter(f);
}

int emu_invariants(void* h, const fnpf_prism_opts* o, const double* eta, const double* hh, const double* phis,
                   double* mass, double* energy) {
  Emu* e = static_cast<Emu*>(h);
  const Params prm = params(o);
  Stepper<HostEx> sp = stepper(e, prm);
  return sp.invariants(eta, hh, phis, prm, mass, energy, nullptr);
}

int emu_set_relaxation(void* h, const double* cr, const double* gen, double amp, double kx, double ky, double omega,
                       double phase, double ramp) {
  Emu* e = static_cast<Emu*>(h);
  PMesh& m = e->m;
  if (!cr) {
    m.rcr = m.rgen = m.xs = m.ys = nullptr;
    return FNPF_OK;
  }
  const std::vector<double> vc(cr, cr + m.ns), vg(gen, gen + m.ns);
  m.rcr = e->table(vc, 0, vc.size());
  m.rgen = e->table(vg, 0, vg.size());
  m.xs = e->table(e->xs, 0, e->xs.size());
  m.ys = e->table(e->ys, 0, e->ys.size());
  m.ramp = ramp;
  m.amp = amp;
  m.kx = kx;
  m.ky = ky;
  m.omega = omega;
  m.phase = phase;
  return FNPF_OK;
}

int emu_rk4_step(void* h, const fnpf_prism_opts* o, const double* hh, double* eta, double* phis, double t, double dt,
                 fnpf_solve_info* info) {
  Emu* e = static_cast<Emu*>(h);
  const Params prm = params(o);
  Stepper<HostEx> sp = stepper(e, prm);
  return sp.rk4(hh, eta, phis, t, dt, prm, info);
}

}  // extern "C"

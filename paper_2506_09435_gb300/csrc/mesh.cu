// Mesh set-up on the host (arXiv 2506.09435, Sec. 3.1.2 and Sec. 3.4 Step 1):
// GLL tables, node counts, horizontal metric of every element-column node,
// lumped surface mass, surface coordinates, device allocations.
#include <math.h>

#include <algorithm>
#include <cstring>

#include "mesh.cuh"

namespace fnpf {

// GLL nodes: +-1 and the roots of P_p'; Newton on q(x) = (1 - x^2) P_p'(x)
// = p (P_{p-1}(x) - x P_p(x)), q'(x) = -p (p + 1) P_p(x), in long double.
// Weights 2 / (p (p+1) P_p(x_i)^2).  Derivative matrix by the closed form
// D_ij = P_p(x_i) / (P_p(x_j) (x_i - x_j)) (i != j), D_00 = -p(p+1)/4,
// D_pp = p(p+1)/4, other diagonal entries 0 (Deville, Fischer & Mund 2002).
static void legendre_pair(int p, long double x, long double* Pp, long double* Pm1) {
  long double a = 1.0L, b = x;
  if (p == 0) { *Pp = 1.0L; *Pm1 = 0.0L; return; }
  for (int k = 1; k < p; ++k) {
    const long double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
    a = b;
    b = c;
  }
  *Pp = b;
  *Pm1 = a;
}

void gll_tables(int p, double* xi, double* w, double* D) {
  const int n = p + 1;
  const long double pi = 3.141592653589793238462643383279502884L;
  long double x[kMaxN], P[kMaxN];
  for (int i = 0; i < n; ++i) x[i] = -cosl(pi * i / p);
  for (int i = 1; i < p; ++i) {
    for (int it = 0; it < 100; ++it) {
      long double Pp, Pm1;
      legendre_pair(p, x[i], &Pp, &Pm1);
      const long double q = p * (Pm1 - x[i] * Pp);
      const long double dq = -(long double)p * (p + 1) * Pp;
      const long double dx = q / dq;
      x[i] -= dx;
      if (fabsl(dx) < 1e-30L) break;
    }
  }
  x[0] = -1.0L;
  x[p] = 1.0L;
  for (int i = 0; i < n; ++i) {
    long double Pm1;
    legendre_pair(p, x[i], &P[i], &Pm1);
    xi[i] = (double)x[i];
    w[i] = (double)(2.0L / ((long double)p * (p + 1) * P[i] * P[i]));
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      D[i * n + j] = (i == j) ? 0.0 : (double)(P[i] / (P[j] * (x[i] - x[j])));
  D[0] = -(double)p * (p + 1) / 4.0;
  D[p * n + p] = (double)p * (p + 1) / 4.0;
}

bool build_hmetric(const Geom& g, const double* xi, const double* w, const double* D, bool iso, double Lx, double Ly,
                   const double* Xs, const double* Ys, std::vector<double>* hm, std::vector<double>* mass,
                   std::vector<double>* xs, std::vector<double>* ys) {
  const int n = g.n;
  const int64_t L = g.lines, HS = (int64_t)g.n_ecol * L;
  hm->assign(5 * HS, 0.0);
  mass->assign(g.ns, 0.0);
  xs->assign(g.ns, 0.0);
  ys->assign(g.ns, 0.0);
  const double dx = iso ? 0.0 : Lx / g.nx;
  const double dy = (iso || g.dim == 2) ? 0.0 : Ly / g.ny;
  bool bad_jac = false;
  for (int ecol = g.n_ecol - 1; ecol >= 0; --ecol) {   // reverse: the lowest element writes coords last
    const int ex = ecol % g.nx, ey = ecol / g.nx;
    for (int line = (int)L - 1; line >= 0; --line) {
      const int i = line % n, j = line / n;
      const int col = node_col(g, ex, ey, i, j);
      double xr, xs_, yr, ys_;
      double X, Y;
      if (!iso) {
        xr = dx / 2;
        xs_ = 0;
        yr = 0;
        ys_ = dy / 2;
        X = ex * dx + (1 + xi[i]) * dx / 2;
        Y = g.dim == 3 ? ey * dy + (1 + xi[j]) * dy / 2 : 0.0;
      } else {
        xr = xs_ = yr = ys_ = 0;
        for (int a = 0; a < n; ++a) {
          xr += D[i * n + a] * Xs[node_col(g, ex, ey, a, j)];
          if (g.dim == 3) {
            yr += D[i * n + a] * Ys[node_col(g, ex, ey, a, j)];
            xs_ += D[j * n + a] * Xs[node_col(g, ex, ey, i, a)];
            ys_ += D[j * n + a] * Ys[node_col(g, ex, ey, i, a)];
          }
        }
        X = Xs[col];
        Y = g.dim == 3 ? Ys[col] : 0.0;
      }
      double rx, ry, sx, sy, cw;
      if (g.dim == 3) {
        const double J2 = xr * ys_ - xs_ * yr;
        if (!(fabs(J2) > 0)) bad_jac = true;
        rx = ys_ / J2;
        ry = -xs_ / J2;
        sx = -yr / J2;
        sy = xr / J2;
        cw = w[i] * w[j] * fabs(J2);
      } else {
        if (!(fabs(xr) > 0)) bad_jac = true;
        rx = 1.0 / xr;
        ry = sx = sy = 0.0;
        cw = w[i] * fabs(xr);
      }
      const int64_t hidx = (int64_t)ecol * L + line;
      (*hm)[hidx] = rx;
      (*hm)[HS + hidx] = ry;
      (*hm)[2 * HS + hidx] = sx;
      (*hm)[3 * HS + hidx] = sy;
      (*hm)[4 * HS + hidx] = cw;
      (*mass)[col] += cw;
      (*xs)[col] = X;
      (*ys)[col] = Y;
    }
  }
  return !bad_jac;
}

fnpf_status validate_desc(const fnpf_mesh_desc* d, std::string* why) {
  if (!d) { *why = "descriptor is NULL"; return FNPF_EINVAL; }
  if (d->dim != 2 && d->dim != 3) { *why = "dim must be 2 or 3"; return FNPF_EINVAL; }
  if (d->p < 1 || d->p > kMaxP) { *why = "p must be in 1..8"; return FNPF_EINVAL; }
  if (d->nx < 1 || d->nz < 1 || (d->dim == 3 && d->ny < 1)) { *why = "element counts must be >= 1"; return FNPF_EINVAL; }
  if (d->horiz_kind != FNPF_BOX && d->horiz_kind != FNPF_ISOPARAMETRIC) { *why = "bad horiz_kind"; return FNPF_EINVAL; }
  // a periodic direction with one element would couple an element to itself
  if ((d->periodic_x && d->nx < 2) || (d->dim == 3 && d->periodic_y && d->ny < 2)) {
    *why = "a periodic direction needs at least 2 elements";
    return FNPF_EINVAL;
  }
  if (d->horiz_kind == FNPF_BOX && (!(d->Lx > 0) || (d->dim == 3 && !(d->Ly > 0)))) {
    *why = "box lengths must be > 0";
    return FNPF_EINVAL;
  }
  if (d->horiz_kind == FNPF_ISOPARAMETRIC && (!d->X || (d->dim == 3 && !d->Y))) {
    *why = "isoparametric mesh needs X and Y";
    return FNPF_EINVAL;
  }
  if (!(d->g > 0)) { *why = "g must be > 0"; return FNPF_EINVAL; }
  // sizes must fit the 32-bit column and element-column indices used on the device
  const int64_t ncx = (int64_t)d->p * d->nx + (d->periodic_x ? 0 : 1);
  const int64_t ncy = d->dim == 3 ? (int64_t)d->p * d->ny + (d->periodic_y ? 0 : 1) : 1;
  if (ncx * ncy > (int64_t)1 << 30 || (int64_t)d->nx * (d->dim == 3 ? d->ny : 1) > (int64_t)1 << 30) {
    *why = "mesh too large";
    return FNPF_EINVAL;
  }
  if (!d->h) { *why = "depth array h is NULL"; return FNPF_EINVAL; }
  return FNPF_OK;
}

Geom make_geom(const fnpf_mesh_desc* d) {
  Geom g{};
  g.dim = d->dim;
  g.nx = d->nx;
  g.ny = d->dim == 3 ? d->ny : 1;
  g.nz = d->nz;
  g.p = d->p;
  g.n = d->p + 1;
  g.px = d->periodic_x ? 1 : 0;
  g.py = (d->dim == 3 && d->periodic_y) ? 1 : 0;
  g.ncx = g.p * g.nx + (g.px ? 0 : 1);
  g.ncy = d->dim == 3 ? g.p * g.ny + (g.py ? 0 : 1) : 1;
  g.ns = g.ncx * g.ncy;
  g.nv = g.p * g.nz + 1;
  g.n_ecol = g.nx * g.ny;
  g.lines = d->dim == 3 ? g.n * g.n : g.n;
  g.ring = d->dim == 3 ? 4 * g.p : 2;
  g.N = (int64_t)g.nv * g.ns;
  g.NI = (int64_t)(g.nv - 1) * g.ns;
  g.g = d->g;
  return g;
}

}  // namespace fnpf

using fnpf::Geom;

namespace {
std::string g_create_error;

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T));
}

void free_mesh(fnpf_mesh* m) {
  if (!m) return;
  double* ptrs[] = {m->dD, m->dxi, m->dw, m->dhm, m->dh, m->dminv, m->ring, m->r, m->z, m->p, m->q, m->dinv,
                    m->phi, m->partials, m->s_eta[0], m->s_eta[1], m->s_phi[0], m->s_phi[1], m->acc_eta,
                    m->acc_phi};
  for (double* p : ptrs)
    if (p) cudaFree(p);
  float* fptrs[] = {m->fD, m->fxi, m->fw, m->fhm, m->fh, m->eta32, m->r32, m->z32, m->p32, m->q32, m->e32,
                    m->dinv32};
  for (float* p : fptrs)
    if (p) cudaFree(p);
  if (m->b) cudaFree(m->b);
  if (m->eta64) cudaFree(m->eta64);
  if (m->zero_eta) cudaFree(m->zero_eta);
  if (m->dfilter) cudaFree(m->dfilter);
  if (m->G64) cudaFree(m->G64);
  if (m->adj) cudaFree(m->adj);
  if (m->inv_work) cudaFree(m->inv_work);
  if (m->dl_buf) cudaFree(m->dl_buf);
  if (m->projH) cudaFree(m->projH);
  if (m->tape) cudaFree(m->tape);
  if (m->tape_slot_dev) cudaFree(m->tape_slot_dev);
  if (m->tape_slot_host) cudaFreeHost(m->tape_slot_host);
  if (m->projHa) cudaFree(m->projHa);
  if (m->proj_part) cudaFree(m->proj_part);
  double* rptrs[] = {m->rx_cr, m->rx_gen, m->dxs, m->dys};
  for (double* p : rptrs)
    if (p) cudaFree(p);
  if (m->sc_in) cudaFree(m->sc_in);
  fnpf::mg_destroy(m->mg);
  for (GraphSlot& gs : m->g_iter) fnpf::graph_reset(&gs);
  if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
  if (m->gstream) cudaStreamDestroy(m->gstream);
  for (cudaStream_t b : m->bstream)
    if (b) cudaStreamDestroy(b);
  if (m->inner_total) cudaFree(m->inner_total);
  if (m->stage_info) cudaFree(m->stage_info);
  if (m->t_dev) cudaFree(m->t_dev);
  if (m->stage_info_host) cudaFreeHost(m->stage_info_host);
  if (m->t_host) cudaFreeHost(m->t_host);
  if (m->sc) cudaFree(m->sc);
  if (m->sc_host) cudaFreeHost(m->sc_host);
  if (m->ev0) cudaEventDestroy(m->ev0);
  if (m->ev1) cudaEventDestroy(m->ev1);
  for (cudaEvent_t e : m->prof_ev)
    if (e) cudaEventDestroy(e);
  delete m;
}
}  // namespace

namespace fnpf {
void set_create_error(const char* msg) { g_create_error = msg; }
}  // namespace fnpf

extern "C" {

fnpf_status fnpf_count_dofs(const fnpf_mesh_desc* desc, int64_t* n_vol, int64_t* n_surf) {
  std::string why;
  if (!desc || !n_vol || !n_surf) return FNPF_EINVAL;
  fnpf_mesh_desc d = *desc;
  // counting does not need the arrays
  const double dummy = 1.0;
  if (!d.h) d.h = &dummy;
  if (d.horiz_kind == FNPF_ISOPARAMETRIC) {
    if (!d.X) d.X = &dummy;
    if (!d.Y) d.Y = &dummy;
  }
  fnpf_status st = fnpf::validate_desc(&d, &why);
  if (st != FNPF_OK) return st;
  const Geom g = fnpf::make_geom(&d);
  *n_vol = g.N;
  *n_surf = g.ns;
  return FNPF_OK;
}

void fnpf_default_opts(fnpf_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = FNPF_FP64;
  o->precond = FNPF_JACOBI;
  o->rtol = 1e-10;
  o->atol = 0.0;
  o->max_iter = 20000;
  o->check_every = 16;
  o->cheb_degree = 3;
  o->coarse_iters = 6;
  o->inner_rtol = 1e-5;
  o->max_outer = 20;
  o->use_graphs = 1;
  o->store_metric = 1;
  o->coarse_solver = FNPF_COARSE_CLUSTER;
  o->cheb_kind = FNPF_CHEB_FIRST;
  o->cheb_range = 160.0;
  o->model = FNPF_NONLINEAR;
  o->mg_schedule = FNPF_MG_HALVE;
  o->projection = 8;
}

fnpf_status fnpf_create_mesh(const fnpf_mesh_desc* desc, const fnpf_opts* opts, fnpf_mesh** out) {
  if (!out) return FNPF_EINVAL;
  *out = nullptr;
  std::string why;
  fnpf_status st = fnpf::validate_desc(desc, &why);
  if (st != FNPF_OK) {
    g_create_error = why;
    return st;
  }
  const Geom g = fnpf::make_geom(desc);
  for (int c = 0; c < g.ns; ++c) {
    if (!(desc->h[c] > 0) || !std::isfinite(desc->h[c])) {
      g_create_error = "depth h must be finite and > 0 at every surface node";
      return FNPF_EINVAL;
    }
  }
  if (opts && opts->model != FNPF_NONLINEAR && opts->model != FNPF_LINEAR) {
    g_create_error = "model must be FNPF_NONLINEAR or FNPF_LINEAR";
    return FNPF_EINVAL;
  }
  if (opts && (opts->projection < 0 || opts->projection > fnpf::kMaxProjection)) {
    g_create_error = "projection must be in 0..8";
    return FNPF_EINVAL;
  }
  if (opts && (opts->precision < FNPF_FP64 || opts->precision > FNPF_FP64_PC32)) {
    g_create_error = "precision must be FNPF_FP64, FNPF_MIXED or FNPF_FP64_PC32";
    return FNPF_EINVAL;
  }
  fnpf_mesh* m = new fnpf_mesh();
  m->g = g;
  if (opts) m->opts = *opts;
  else fnpf_default_opts(&m->opts);
  cudaGetDevice(&m->device);
  const int n = g.n, p = g.p;
  m->xi.resize(n);
  m->w.resize(n);
  m->D.resize(n * n);
  fnpf::gll_tables(p, m->xi.data(), m->w.data(), m->D.data());
  m->h.assign(desc->h, desc->h + g.ns);
  m->iso = desc->horiz_kind == FNPF_ISOPARAMETRIC;
  m->Lx = desc->Lx;
  m->Ly = desc->Ly;
  if (m->iso) {
    m->Xs.assign(desc->X, desc->X + g.ns);
    m->Ys = g.dim == 3 ? std::vector<double>(desc->Y, desc->Y + g.ns) : std::vector<double>(g.ns, 0.0);
  }

  // horizontal metric of every element-column node and lumped surface mass
  const int64_t HS = (int64_t)g.n_ecol * g.lines;
  std::vector<double> mass;
  const bool iso = desc->horiz_kind == FNPF_ISOPARAMETRIC;
  if (!fnpf::build_hmetric(g, m->xi.data(), m->w.data(), m->D.data(), iso, desc->Lx, desc->Ly, desc->X, desc->Y,
                           &m->hm, &mass, &m->xs, &m->ys)) {
    g_create_error = "degenerate horizontal Jacobian";
    delete m;
    return FNPF_EINVAL;
  }
  m->minv.resize(g.ns);
  for (int c = 0; c < g.ns; ++c) m->minv[c] = 1.0 / mass[c];

  // device allocations
  cudaError_t e = cudaSuccess;
  auto A = [&](double** ptr, size_t cnt) {
    if (e == cudaSuccess) e = dalloc(ptr, cnt);
  };
  A(&m->dD, n * n);
  A(&m->dxi, n);
  A(&m->dw, n);
  A(&m->dhm, 5 * HS);
  A(&m->dh, g.ns);
  A(&m->dminv, g.ns);
  A(&m->ring, (size_t)g.nv * g.n_ecol * g.ring);
  A(&m->r, g.NI);
  A(&m->z, g.NI);
  A(&m->p, g.NI);
  A(&m->q, g.NI);
  A(&m->dinv, g.NI);
  A(&m->phi, g.N);
  A(&m->partials, 4 * fnpf::kVecBlocks);
  for (int k = 0; k < 2; ++k) {
    A(&m->s_eta[k], g.ns);
    A(&m->s_phi[k], g.ns);
  }
  A(&m->acc_eta, g.ns);
  A(&m->acc_phi, g.ns);
  A(&m->b, g.NI);
  A(&m->eta64, g.ns);
  A(&m->zero_eta, g.ns);
  auto AF = [&](float** ptr, size_t cnt) {
    if (e == cudaSuccess) e = dalloc(ptr, cnt);
  };
  AF(&m->fD, n * n);
  AF(&m->fxi, n);
  AF(&m->fw, n);
  AF(&m->fhm, 5 * HS);
  AF(&m->fh, g.ns);
  AF(&m->eta32, g.ns);
  AF(&m->r32, g.NI);
  AF(&m->z32, g.NI);
  AF(&m->p32, g.NI);
  AF(&m->q32, g.NI);
  AF(&m->e32, g.NI);
  AF(&m->dinv32, g.NI);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->sc_in, sizeof(fnpf::CgScalars));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->sc, sizeof(fnpf::CgScalars));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&m->sc_host, sizeof(fnpf::CgScalars));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->gstream, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&m->bstream[k], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->inner_total, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->stage_info, 4 * sizeof(fnpf::StageInfo));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->t_dev, sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&m->stage_info_host, 4 * sizeof(fnpf::StageInfo));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&m->t_host, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&m->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&m->ev1);
  if (e == cudaSuccess) e = cudaMemcpy(m->dD, m->D.data(), n * n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dxi, m->xi.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dw, m->w.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dhm, m->hm.data(), 5 * HS * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dh, m->h.data(), g.ns * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dminv, m->minv.data(), g.ns * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->phi, 0, g.N * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(m->zero_eta, 0, g.ns * sizeof(double));
  {
    auto up32 = [&](float* dst, const std::vector<double>& src) {
      std::vector<float> f(src.begin(), src.end());
      if (e == cudaSuccess) e = cudaMemcpy(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
    };
    up32(m->fD, m->D);
    up32(m->fxi, m->xi);
    up32(m->fw, m->w);
    up32(m->fhm, m->hm);
    up32(m->fh, m->h);
  }
  // constant tables of the line-decomposed operator kernels of every order
  // (the multigrid levels use lower orders), once per device
  for (int nn = 2; nn <= fnpf::kMaxN && e == cudaSuccess; ++nn) e = fnpf::ax_prepare(nn);
  if (e != cudaSuccess) {
    g_create_error = std::string("device set-up failed: ") + cudaGetErrorString(e);
    const fnpf_status ret = (e == cudaErrorMemoryAllocation) ? FNPF_ENOMEM : FNPF_ECUDA;
    free_mesh(m);
    return ret;
  }
  *out = m;
  return FNPF_OK;
}

void fnpf_destroy_mesh(fnpf_mesh* m) { free_mesh(m); }

fnpf_status fnpf_set_opts(fnpf_mesh* m, const fnpf_opts* o) {
  if (!m || !o) return FNPF_EINVAL;
  if (o->model != FNPF_NONLINEAR && o->model != FNPF_LINEAR) {
    m->err = "model must be FNPF_NONLINEAR or FNPF_LINEAR";
    return FNPF_EINVAL;
  }
  if (o->precision < FNPF_FP64 || o->precision > FNPF_FP64_PC32) {
    m->err = "precision must be FNPF_FP64, FNPF_MIXED or FNPF_FP64_PC32";
    return FNPF_EINVAL;
  }
  if (o->projection < 0 || o->projection > fnpf::kMaxProjection) {
    m->err = "projection must be in 0..8";
    return FNPF_EINVAL;
  }
  m->opts = *o;
  for (GraphSlot& gs : m->g_iter) fnpf::graph_reset(&gs);   // captured arguments depend on the options
  if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
  m->step_exec = nullptr;
  m->cheb_valid[0] = m->cheb_valid[1] = false;
  m->lpf_ready[0] = m->lpf_ready[1] = false;
  m->warm = false;   // the next step is host-driven: it rebuilds what the new options need
  if (m->mg && fnpf::mg_schedule(m->mg) != o->mg_schedule) {
    fnpf::mg_destroy(m->mg);
    m->mg = nullptr;
  }
  fnpf::mg_set_coarse(m->mg, o->coarse_solver);
  fnpf::mg_set_kind(m->mg, o->cheb_kind, o->cheb_range);
  return FNPF_OK;
}

fnpf_status fnpf_mesh_sizes(const fnpf_mesh* m, int64_t* n_vol, int64_t* n_surf) {
  if (!m || !n_vol || !n_surf) return FNPF_EINVAL;
  *n_vol = m->g.N;
  *n_surf = m->g.ns;
  return FNPF_OK;
}

fnpf_status fnpf_surface_coords(const fnpf_mesh* m, double* x, double* y) {
  if (!m || !x || !y) return FNPF_EINVAL;
  std::copy(m->xs.begin(), m->xs.end(), x);
  std::copy(m->ys.begin(), m->ys.end(), y);
  return FNPF_OK;
}

const char* fnpf_last_error(const fnpf_mesh* m) { return m ? m->err.c_str() : g_create_error.c_str(); }

const char* fnpf_status_string(fnpf_status s) {
  switch (s) {
    case FNPF_OK: return "ok";
    case FNPF_EINVAL: return "invalid argument";
    case FNPF_ENOMEM: return "out of device memory";
    case FNPF_ECUDA: return "CUDA error";
    case FNPF_ENOCONV: return "not converged";
    case FNPF_EBREAKDOWN: return "CG breakdown";
    case FNPF_EDIVERGED: return "diverged or folded state";
    case FNPF_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

}  // extern "C"

// Adjoint (reverse mode) of one RK4 step of the fully nonlinear free-surface
// state (Sec. 3.2 ERK4 around Sec. 3.4 Steps 4.1-4.7): given the adjoint
// lam_{n+1} = dJ/dy_{n+1} of y = (eta, phi_eta), returns dJ/dy_n and adds
// dJ/dh (the bathymetry at the surface nodes).
//
// The step is recomputed from y_n, storing every stage state Y_s and its
// volume potential phi_s.  Then, with k_s = f(Y_s), Y_s = y_n + c_s dt k_{s-1},
// y_{n+1} = y_n + dt sum b_s k_s, the reverse sweep runs s = 4..1:
//   kbar_s = dt b_s lam_{n+1} (+ c_{s+1} dt Ybar_{s+1}),  Ybar_s = f'(Y_s)^T kbar_s,
//   lam_n = lam_{n+1} + sum_s Ybar_s.
// f'(Y)^T kbar (the right-hand side of the Zakharov conditions through the
// Laplace solve):
//   1. RHS VJP: the lumped-mass average and the element-local gradients,
//      adjoint to eta, phi_eta directly and to w;
//   2. w = phi_t / z_t: wbar -> the adjoint right-hand side on the top planes,
//      phibar_eta (surface node of the line), etabar and hbar through z_t;
//   3. one adjoint Laplace solve A_II psi = phibar_I with the same PCG (A is
//      symmetric), then phibar_eta -= (A [psi; 0])_S;
//   4. geometric VJP: etabar, hbar -= d(psi^T A(eta, h) phi)/d(eta, h).
// Relaxation zones, when set, enter as lam <- (1 - C_r) lam at the start (the
// targets do not depend on the state).
#include <math.h>

#include <algorithm>

#include "mesh.cuh"

namespace fnpf {

cudaError_t launch_geom_vjp(const Geom& g, const Tables<double>& t, const double* eta, const double* psiI,
                            const double* phiI, const double* phiS, double* out, cudaStream_t s);
StageArgs stage_args(fnpf_mesh* m, double* eta, double* phis, const double* ce, const double* cp, int st, double t,
                     double dt, const double* t_dev);

namespace {

constexpr int TB = 128;

inline int blocks(int64_t n) { return (int)((n + TB - 1) / TB); }

// Element-local part of the RHS VJP, one thread per element surface node:
// EB[0..5] = (eta_r bar, eta_s bar, phi_r bar, phi_s bar, w bar, eta bar).
__global__ void rhs_vjp_elem_kernel(Geom g, Tables<double> t, const double* eta, const double* phis, const double* w,
                                    const double* kbe, const double* kbp, double* EB) {
  const int64_t total = (int64_t)g.n_ecol * g.lines;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int n = g.n;
  const int ecol = (int)(idx / g.lines), line = (int)(idx % g.lines);
  const int i = line % n, j = line / n, ex = ecol % g.nx, ey = ecol / g.nx;
  const int col = node_col(g, ex, ey, i, j);
  double er = 0, pr = 0, es = 0, ps = 0;
  for (int m = 0; m < n; ++m) {
    const double d = t.D[i * n + m];
    const int c2 = node_col(g, ex, ey, m, j);
    er += d * eta[c2];
    pr += d * phis[c2];
  }
  if (g.dim == 3) {
    for (int m = 0; m < n; ++m) {
      const double d = t.D[j * n + m];
      const int c2 = node_col(g, ex, ey, i, m);
      es += d * eta[c2];
      ps += d * phis[c2];
    }
  }
  const int64_t hs = total;
  const double rx = t.hm[idx], ry = t.hm[hs + idx], sx = t.hm[2 * hs + idx], sy = t.hm[3 * hs + idx],
               cw = t.hm[4 * hs + idx];
  const double gxe = er * rx + es * sx, gye = er * ry + es * sy;
  const double gxp = pr * rx + ps * sx, gyp = pr * ry + ps * sy;
  const double Le = kbe[col] * t.minv[col] * cw, Lp = kbp[col] * t.minv[col] * cw;
  const double wv = w[col];
  const double ge2 = 1.0 + gxe * gxe + gye * gye;
  const double bex = Le * (-gxp + 2.0 * wv * gxe) + Lp * wv * wv * gxe;
  const double bey = Le * (-gyp + 2.0 * wv * gye) + Lp * wv * wv * gye;
  const double bpx = -Le * gxe - Lp * gxp, bpy = -Le * gye - Lp * gyp;
  EB[idx] = rx * bex + ry * bey;
  EB[hs + idx] = sx * bex + sy * bey;
  EB[2 * hs + idx] = rx * bpx + ry * bpy;
  EB[3 * hs + idx] = sx * bpx + sy * bpy;
  EB[4 * hs + idx] = (Le + Lp * wv) * ge2;
  EB[5 * hs + idx] = -g.g * Lp;
}

// Nodal sums of the element-local RHS adjoints (D^T along element rows):
// ebar, pbar, wbar at every surface column (overwritten).
__global__ void rhs_vjp_gather_kernel(Geom g, Tables<double> t, const double* EB, double* ebar, double* pbar,
                                      double* wbar) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= g.ns) return;
  const int n = g.n;
  const int64_t hs = (int64_t)g.n_ecol * g.lines;
  int exo[2], io[2], eyo[2] = {0, 0}, jo[2] = {0, 0};
  const int cx = line_owners(col % g.ncx, g.p, g.nx, g.px, exo, io);
  const int cy = g.dim == 3 ? line_owners(col / g.ncx, g.p, g.ny, g.py, eyo, jo) : 1;
  double se = 0, sp = 0, sw = 0;
  for (int u = 0; u < cx; ++u) {
    for (int v = 0; v < cy; ++v) {
      const int i = io[u], j = jo[v];
      const int64_t base = (int64_t)(eyo[v] * g.nx + exo[u]) * g.lines;
      se += EB[5 * hs + base + j * n + i];
      sw += EB[4 * hs + base + j * n + i];
      for (int q = 0; q < n; ++q) {
        const double d = t.D[q * n + i];
        se += d * EB[base + j * n + q];
        sp += d * EB[2 * hs + base + j * n + q];
      }
      if (g.dim == 3) {
        for (int q = 0; q < n; ++q) {
          const double d = t.D[q * n + j];
          se += d * EB[hs + base + q * n + i];
          sp += d * EB[3 * hs + base + q * n + i];
        }
      }
    }
  }
  ebar[col] = se;
  pbar[col] = sp;
  wbar[col] = sw;
}

// w = phi_t / z_t at every surface column (phi: interior planes + surface phis).
__global__ void w_of_kernel(Geom g, Tables<double> t, const double* eta, const double* phiI, const double* phis,
                            double* w) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= g.ns) return;
  const int P = g.p;
  double s = 0;
  for (int j = 0; j < P; ++j) s += t.D[P * g.n + j] * phiI[(int64_t)(g.nv - 1 - P + j) * g.ns + col];
  s += t.D[P * g.n + P] * phis[col];
  w[col] = s * (2.0 * g.nz) / (eta[col] + t.h[col]);
}

// Adjoint of w: the right-hand side of the adjoint solve on the top planes,
// and the direct terms into pbar, ebar, hbar.
__global__ void w_vjp_kernel(Geom g, Tables<double> t, const double* eta, const double* w, const double* wbar,
                             double* badj, double* pbar, double* ebar, double* hbar) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= g.ns) return;
  const int P = g.p;
  const double depth = eta[col] + t.h[col];
  const double s = (2.0 * g.nz) / depth;
  const double wb = wbar[col];
  for (int j = 0; j < P; ++j) badj[(int64_t)(g.nv - 1 - P + j) * g.ns + col] = t.D[P * g.n + j] * s * wb;
  pbar[col] += t.D[P * g.n + P] * s * wb;
  const double dz = -w[col] / depth * wb;
  ebar[col] += dz;
  hbar[col] += dz;
}

// etabar, hbar -= nodal sums of the geometric VJP line sums LB (see adj_impl.cuh).
__global__ void geom_vjp_gather_kernel(Geom g, Tables<double> t, const double* LB, double* ebar, double* hbar) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= g.ns) return;
  const int n = g.n;
  const int64_t hs = (int64_t)g.n_ecol * g.lines;
  int exo[2], io[2], eyo[2] = {0, 0}, jo[2] = {0, 0};
  const int cx = line_owners(col % g.ncx, g.p, g.nx, g.px, exo, io);
  const int cy = g.dim == 3 ? line_owners(col / g.ncx, g.p, g.ny, g.py, eyo, jo) : 1;
  double se = 0, sh = 0;
  const double za = 0.5 / g.nz;
  for (int u = 0; u < cx; ++u) {
    for (int v = 0; v < cy; ++v) {
      const int i = io[u], j = jo[v];
      const int64_t base = (int64_t)(eyo[v] * g.nx + exo[u]) * g.lines;
      const double a = LB[base + j * n + i] * za;
      se += a;
      sh += a;
      for (int q = 0; q < n; ++q) {
        const double d = t.D[q * n + i];
        const double qr = LB[hs + base + j * n + q], pr = LB[3 * hs + base + j * n + q];
        se += d * qr;
        sh += d * (qr - pr);
      }
      if (g.dim == 3) {
        for (int q = 0; q < n; ++q) {
          const double d = t.D[q * n + j];
          const double qs = LB[2 * hs + base + q * n + i], ps = LB[4 * hs + base + q * n + i];
          se += d * qs;
          sh += d * (qs - ps);
        }
      }
    }
  }
  ebar[col] -= se;
  hbar[col] -= sh;
}

__global__ void scale_kernel(int n, const double* a, const double* cr, double f, double* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  b[i] = f * a[i] * (cr ? 1.0 - cr[i] : 1.0);
}

__global__ void axpy_kernel(int n, double a, const double* x, double* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

__global__ void sub_kernel(int n, const double* x, double* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] -= x[i];
}

}  // namespace
}  // namespace fnpf

using fnpf::Geom;

namespace {

// Tape slot layout: [4][NI] stage potentials (interior), then [4][2][ns] stage states.
inline int64_t tape_stride(const Geom& g) { return 4 * g.NI + 8 * (int64_t)g.ns; }

__global__ void tape_record_kernel(int64_t NI, int ns, const int* slot, int cap, double* tape, int64_t stride, int st,
                                   const double* phi, const double* ce, const double* cp) {
  const int k = *slot;
  if (k < 0 || k >= cap) return;
  double* base = tape + (int64_t)k * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NI; i += (int64_t)gridDim.x * blockDim.x)
    base[(int64_t)st * NI + i] = phi[i];
  double* Y = base + 4 * NI;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
    Y[(int64_t)(2 * st) * ns + i] = ce[i];
    Y[(int64_t)(2 * st + 1) * ns + i] = cp[i];
  }
}

fnpf_status check_adjoint_supported(fnpf_mesh* m) {
  if (m->linear() || m->filter_on || m->dealias_M > 0) {
    m->err = "the adjoint step is built for FNPF_NONLINEAR without the modal filter or over-integration";
    return FNPF_EUNSUPPORTED;
  }
  return FNPF_OK;
}

// The adjoint workspace (stage data of the recompute, reverse-sweep scratch),
// allocated at the first use.
fnpf_status ensure_adj(fnpf_mesh* m) {
  const Geom& g = m->g;
  const int64_t ns = g.ns, NI = g.NI, LS = (int64_t)g.n_ecol * g.lines;
  const int64_t n_phi = 4 * NI, n_y = 8 * ns, n_k = 8 * ns, n_surf = 10 * ns, n_eb = 6 * LS, n_lb = 5 * LS;
  const int64_t n_vol = 3 * NI;
  const size_t bytes = (size_t)(n_phi + n_y + n_k + n_surf + n_eb + n_lb + n_vol) * sizeof(double);
  if (!m->adj || m->adj_bytes < bytes) {
    if (m->adj) cudaFree(m->adj);
    m->adj = nullptr;
    if (cudaMalloc((void**)&m->adj, bytes) != cudaSuccess) {
      m->adj = nullptr;
      m->err = "cannot allocate adjoint workspace";
      return FNPF_ENOMEM;
    }
    m->adj_bytes = bytes;
  }
  return FNPF_OK;
}

// Reverse sweep of one RK4 step from the stage potentials Phi [4][NI] and
// stage states Y [4][2][ns] of the forward step.
fnpf_status adjoint_reverse(fnpf_mesh* m, const double* Phi, const double* Y, const double* lam_eta,
                            const double* lam_phis, double* lam_eta_out, double* lam_phis_out, double* lam_h,
                            double dt, cudaStream_t s) {
  const Geom& g = m->g;
  const int64_t ns = g.ns, NI = g.NI, LS = (int64_t)g.n_ecol * g.lines;
  double* KB = m->adj + 4 * NI + 8 * ns;        // [4][2][ns] kbar
  double* S = KB + 8 * ns;                      // surface scratch
  double* oute = S + 2 * ns, *outp = S + 3 * ns, *ebar = S + 4 * ns, *pbar = S + 5 * ns, *wbar = S + 6 * ns,
         *hbar = S + 7 * ns, *wv = S + 8 * ns, *ysurf = S + 9 * ns;
  double* EB = S + 10 * ns;
  double* LB = EB + 6 * LS;
  double* badj = LB + 5 * LS;
  double* psi = badj + NI;
  double* tmp = psi + NI;
  const fnpf::Tables<double> tb = m->tables();
  const int sb = fnpf::blocks(ns);
  cudaError_t e = cudaSuccess;
#define ACK(call)                                                     \
  do {                                                                \
    if ((e = (call)) != cudaSuccess) {                                \
      m->err = std::string("adjoint: ") + cudaGetErrorString(e);     \
      return FNPF_ECUDA;                                              \
    }                                                                 \
  } while (0)
  // ---- reverse sweep
  const double* cr = m->relax_on ? m->rx_cr : nullptr;
  fnpf::scale_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, lam_eta, cr, 1.0, oute);
  fnpf::scale_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, lam_phis, cr, 1.0, outp);
  static const double bw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  static const double cc[4] = {0.0, 0.5, 0.5, 1.0};
  for (int st = 0; st < 4; ++st) {
    fnpf::scale_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, oute, nullptr, dt * bw[st], KB + (2 * st) * ns);
    fnpf::scale_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, outp, nullptr, dt * bw[st], KB + (2 * st + 1) * ns);
  }
  ACK(cudaMemsetAsync(hbar, 0, ns * 8, s));
  for (int st = 3; st >= 0; --st) {
    const double* Ye = Y + (2 * st) * ns;
    const double* Yp = Y + (2 * st + 1) * ns;
    const double* Ph = Phi + st * NI;
    fnpf::w_of_kernel<<<sb, fnpf::TB, 0, s>>>(g, tb, Ye, Ph, Yp, wv);
    fnpf::rhs_vjp_elem_kernel<<<fnpf::blocks(LS), fnpf::TB, 0, s>>>(g, tb, Ye, Yp, wv, KB + (2 * st) * ns,
                                                                    KB + (2 * st + 1) * ns, EB);
    fnpf::rhs_vjp_gather_kernel<<<sb, fnpf::TB, 0, s>>>(g, tb, EB, ebar, pbar, wbar);
    ACK(cudaMemsetAsync(badj, 0, NI * 8, s));
    fnpf::w_vjp_kernel<<<sb, fnpf::TB, 0, s>>>(g, tb, Ye, wv, wbar, badj, pbar, ebar, hbar);
    ACK(cudaGetLastError());
    // adjoint Laplace solve with the forward solver (A is symmetric)
    ACK(cudaMemsetAsync(psi, 0, NI * 8, s));
    fnpf_status r = fnpf::cg_solve(m, Ye, Yp, psi, nullptr, s, badj);
    if (r != FNPF_OK) return r;
    // surface rows: pbar -= (A [psi; 0])_S
    ACK(fnpf::launch_apply<double>(g, tb, Ye, psi, nullptr, tmp, ysurf, m->ring, m->variant64, s));
    fnpf::sub_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, ysurf, pbar);
    // geometry: ebar, hbar -= d(psi^T A(eta, h) phi)/d(eta, h)
    ACK(fnpf::launch_geom_vjp(g, tb, Ye, psi, Ph, Yp, LB, s));
    fnpf::geom_vjp_gather_kernel<<<sb, fnpf::TB, 0, s>>>(g, tb, LB, ebar, hbar);
    fnpf::axpy_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, 1.0, ebar, oute);
    fnpf::axpy_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, 1.0, pbar, outp);
    if (st > 0) {
      fnpf::axpy_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, cc[st] * dt, ebar, KB + (2 * (st - 1)) * ns);
      fnpf::axpy_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, cc[st] * dt, pbar, KB + (2 * (st - 1) + 1) * ns);
    }
    ACK(cudaGetLastError());
    m->launches += 14;
  }
  ACK(cudaMemcpyAsync(lam_eta_out, oute, ns * 8, cudaMemcpyDeviceToDevice, s));
  ACK(cudaMemcpyAsync(lam_phis_out, outp, ns * 8, cudaMemcpyDeviceToDevice, s));
  if (lam_h) fnpf::axpy_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, 1.0, hbar, lam_h);
  ACK(cudaGetLastError());
#undef ACK
  return FNPF_OK;
}

}  // namespace

cudaError_t fnpf::enqueue_tape_record(fnpf_mesh* m, int st, const double* ce, const double* cp, cudaStream_t s) {
  const Geom& g = m->g;
  tape_record_kernel<<<fnpf::kVecBlocks, 256, 0, s>>>(g.NI, g.ns, m->tape_slot_dev, m->tape_cap, m->tape,
                                                      tape_stride(g), st, m->phi, ce, cp);
  m->launches += 1;
  return cudaGetLastError();
}

extern "C" fnpf_status fnpf_step_adjoint(fnpf_mesh* m, const double* eta_n, const double* phis_n,
                                         const double* lam_eta, const double* lam_phis, double* lam_eta_out,
                                         double* lam_phis_out, double* lam_h, double t, double dt, void* stream) {
  if (!m || !eta_n || !phis_n || !lam_eta || !lam_phis || !lam_eta_out || !lam_phis_out || !(dt > 0))
    return FNPF_EINVAL;
  fnpf_status st0 = check_adjoint_supported(m);
  if (st0 == FNPF_OK) st0 = ensure_adj(m);
  if (st0 != FNPF_OK) return st0;
  cudaStream_t s = (cudaStream_t)stream;
  const Geom& g = m->g;
  const int64_t ns = g.ns, NI = g.NI;
  double* Phi = m->adj;                         // [4][NI] stage potentials (interior)
  double* Y = Phi + 4 * NI;                     // [4][2][ns] stage states (eta, phis)
  double* S = Y + 16 * ns;                      // surface scratch (after the kbar block)
  double* fe = S, *fp = S + ns;
  const fnpf::Tables<double> tb = m->tables();
  cudaError_t e = cudaSuccess;
#define ACK(call)                                                     \
  do {                                                                \
    if ((e = (call)) != cudaSuccess) {                                \
      m->err = std::string("adjoint: ") + cudaGetErrorString(e);     \
      return FNPF_ECUDA;                                              \
    }                                                                 \
  } while (0)
  // ---- forward recompute from y_n, storing Y_s and phi_s
  ACK(cudaMemcpyAsync(fe, eta_n, ns * 8, cudaMemcpyDeviceToDevice, s));
  ACK(cudaMemcpyAsync(fp, phis_n, ns * 8, cudaMemcpyDeviceToDevice, s));
  const double* ce = fe;
  const double* cp = fp;
  for (int st = 0; st < 4; ++st) {
    ACK(cudaMemcpyAsync(Y + (2 * st) * ns, ce, ns * 8, cudaMemcpyDeviceToDevice, s));
    ACK(cudaMemcpyAsync(Y + (2 * st + 1) * ns, cp, ns * 8, cudaMemcpyDeviceToDevice, s));
    fnpf_status r = fnpf::cg_solve(m, ce, cp, m->phi, nullptr, s);
    if (r != FNPF_OK) return r;
    ACK(cudaMemcpyAsync(Phi + st * NI, m->phi, NI * 8, cudaMemcpyDeviceToDevice, s));
    fnpf::StageArgs a = fnpf::stage_args(m, fe, fp, ce, cp, st, t, dt, nullptr);
    a.cr = nullptr;   // the relaxation of y_{n+1} is not needed: only its Jacobian enters
    ACK(fnpf::launch_stage(g, tb, a, s));
    ce = a.out_eta;
    cp = a.out_phi;
  }
#undef ACK
  return adjoint_reverse(m, Phi, Y, lam_eta, lam_phis, lam_eta_out, lam_phis_out, lam_h, dt, s);
}

extern "C" fnpf_status fnpf_tape_begin(fnpf_mesh* m, int capacity) {
  if (!m || capacity < 1) return FNPF_EINVAL;
  const Geom& g = m->g;
  if (!m->tape_slot_dev) {
    if (cudaMalloc((void**)&m->tape_slot_dev, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&m->tape_slot_host, sizeof(int)) != cudaSuccess) {
      m->err = "tape: allocation failed";
      return FNPF_ENOMEM;
    }
  }
  if (m->tape_cap < capacity) {
    if (m->tape) cudaFree(m->tape);
    m->tape = nullptr;
    m->tape_cap = 0;
    if (cudaMalloc((void**)&m->tape, (size_t)capacity * tape_stride(g) * sizeof(double)) != cudaSuccess) {
      m->tape = nullptr;
      m->err = "tape: device allocation failed";
      return FNPF_ENOMEM;
    }
    m->tape_cap = capacity;
  }
  if (!m->tape_on && m->step_exec) {   // the captured step gains the tape kernels
    cudaGraphExecDestroy(m->step_exec);
    m->step_exec = nullptr;
  }
  m->tape_on = true;
  m->tape_next = 0;
  return FNPF_OK;
}

extern "C" fnpf_status fnpf_tape_end(fnpf_mesh* m) {
  if (!m) return FNPF_EINVAL;
  if (m->tape_on && m->step_exec) {
    cudaGraphExecDestroy(m->step_exec);
    m->step_exec = nullptr;
  }
  m->tape_on = false;
  return FNPF_OK;
}

extern "C" fnpf_status fnpf_step_adjoint_taped(fnpf_mesh* m, int slot, const double* lam_eta, const double* lam_phis,
                                               double* lam_eta_out, double* lam_phis_out, double* lam_h, double dt,
                                               void* stream) {
  if (!m || !lam_eta || !lam_phis || !lam_eta_out || !lam_phis_out || !(dt > 0)) return FNPF_EINVAL;
  if (slot < 0 || slot >= m->tape_next || slot >= m->tape_cap || !m->tape) {
    m->err = "tape slot not recorded";
    return FNPF_EINVAL;
  }
  fnpf_status st0 = check_adjoint_supported(m);
  if (st0 == FNPF_OK) st0 = ensure_adj(m);
  if (st0 != FNPF_OK) return st0;
  const double* base = m->tape + (int64_t)slot * tape_stride(m->g);
  return adjoint_reverse(m, base, base + 4 * m->g.NI, lam_eta, lam_phis, lam_eta_out, lam_phis_out, lam_h, dt,
                         (cudaStream_t)stream);
}

extern "C" fnpf_status fnpf_laplace_solve_vjp(fnpf_mesh* m, const double* eta, const double* phis, const double* phi,
                                              const double* gbar, double* lam_eta, double* lam_phis, double* lam_h,
                                              void* stream) {
  if (!m || !eta || !phis || !phi || !gbar || !lam_eta || !lam_phis) return FNPF_EINVAL;
  fnpf_status st0 = check_adjoint_supported(m);
  if (st0 == FNPF_OK) st0 = ensure_adj(m);
  if (st0 != FNPF_OK) return st0;
  cudaStream_t s = (cudaStream_t)stream;
  const Geom& g = m->g;
  const int64_t ns = g.ns, NI = g.NI, LS = (int64_t)g.n_ecol * g.lines;
  double* S = m->adj + 4 * NI + 16 * ns;        // surface scratch of the adjoint workspace
  double* hbar = S + 7 * ns, *ysurf = S + 9 * ns;
  double* LB = S + 10 * ns + 6 * LS;
  double* psi = LB + 5 * LS + NI;
  double* tmp = psi + NI;
  const fnpf::Tables<double> tb = m->tables();
  const int sb = fnpf::blocks(ns);
  cudaError_t e = cudaSuccess;
#define ACK(call)                                                          \
  do {                                                                     \
    if ((e = (call)) != cudaSuccess) {                                     \
      m->err = std::string("laplace_solve_vjp: ") + cudaGetErrorString(e);  \
      return FNPF_ECUDA;                                                   \
    }                                                                      \
  } while (0)
  // adjoint solve A_II psi = gbar_I (A is symmetric)
  ACK(cudaMemsetAsync(psi, 0, NI * 8, s));
  fnpf_status r = fnpf::cg_solve(m, eta, phis, psi, nullptr, s, gbar);
  if (r != FNPF_OK) return r;
  // lam_phis += gbar_S - (A [psi; 0])_S
  ACK(fnpf::launch_apply<double>(g, tb, eta, psi, nullptr, tmp, ysurf, m->ring, m->variant64, s));
  fnpf::axpy_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, 1.0, gbar + NI, lam_phis);
  fnpf::sub_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, ysurf, lam_phis);
  // lam_eta, lam_h -= d(psi^T A(eta, h) phi)/d(eta, h)
  ACK(cudaMemsetAsync(hbar, 0, ns * 8, s));
  ACK(fnpf::launch_geom_vjp(g, tb, eta, psi, phi, phi + NI, LB, s));
  fnpf::geom_vjp_gather_kernel<<<sb, fnpf::TB, 0, s>>>(g, tb, LB, lam_eta, hbar);
  if (lam_h) fnpf::axpy_kernel<<<sb, fnpf::TB, 0, s>>>((int)ns, 1.0, hbar, lam_h);
  ACK(cudaGetLastError());
  m->launches += 7;
#undef ACK
  return FNPF_OK;
}

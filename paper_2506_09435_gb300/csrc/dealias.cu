// Over-integration of the nonlinear free-surface terms (arXiv 2506.09435,
// Sec. 3.2: besides the modal filter, the nonlinear terms of the free-surface
// conditions are integrated with a higher quadrature order than the nodal
// collocation, against aliasing in steep waves).
//
// Per surface element: eta, phi_eta and w are interpolated from the GLL nodes
// to an M x M Gauss-Legendre rule (M >= p + 1), with the horizontal gradients
// of the interpolants; the Zakharov right-hand sides f_eta, f_phi (Sec. 2) are
// evaluated there and replaced by their L2 projection onto the degree-p tensor
// polynomials in the element's reference coordinates, computed exactly by the
// Gauss rule and evaluated at the GLL nodes:
//     Pi = V diag(1 / gamma) Lq^T diag(w_q),  V_ik = P_k(xi_i), Lq_qk = P_k(r_q),
//     gamma_k = 2 / (2k + 1),  f_hat = Pi F Pi^T.
// The element values at shared nodes are combined with the lumped-mass
// weights w_i w_j |det H| as the collocation right-hand side is (the lumped
// GLL mass of the rest of the method).  A right-hand side that is a
// polynomial of degree <= p in each reference direction is reproduced
// exactly; modes above p are dropped instead of folded onto the nodes.
#include <math.h>

#include <cmath>
#include <vector>

#include "mesh.cuh"

namespace fnpf {
namespace {

// Gauss-Legendre rule of M points on [-1, 1]: the roots of P_M by Newton's
// method from the Chebyshev-Gauss guesses, in long double; w = 2 / ((1 - x^2) P_M'(x)^2).
void gauss_legendre(int M, double* x, double* w) {
  for (int k = 0; k < M; ++k) {
    long double r = -std::cos(3.14159265358979323846L * (k + 0.75L) / (M + 0.5L));
    long double dp = 1;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = r;
      for (int j = 2; j <= M; ++j) {
        const long double p2 = ((2 * j - 1) * r * p1 - (j - 1) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      const long double pm = M == 1 ? 1.0L : p0;   // P_{M-1}
      const long double pM = M == 1 ? r : p1;
      dp = M * (r * pM - pm) / (r * r - 1);
      const long double dr = pM / dp;
      r -= dr;
      if (std::fabs((double)dr) < 1e-30) break;
    }
    x[k] = (double)r;
    w[k] = (double)(2.0L / ((1 - r * r) * dp * dp));
  }
}

double legendre_value(int k, double x) {
  double p0 = 1.0, p1 = x;
  if (k == 0) return 1.0;
  for (int j = 2; j <= k; ++j) {
    const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Tables [B (M x n) | Bd (M x n) | Pi (n x M)] and the inverse horizontal
// metric at the Gauss points of every element ([4][n_ecol][M^2] in 3D, r_x as
// [n_ecol][M] in 2D), into m->dl_tab / m->dl_metric.
struct DealiasLayout {
  int M, n, Q;               // Q: Gauss points per element (M^2 or M)
  int64_t tab, metric, elem, rhs, w;
};

DealiasLayout layout(const Geom& g, int M) {
  DealiasLayout d{};
  d.M = M;
  d.n = g.n;
  d.Q = g.dim == 3 ? M * M : M;
  d.tab = 3 * (int64_t)M * g.n;
  d.metric = (g.dim == 3 ? 4 : 1) * (int64_t)g.n_ecol * d.Q;
  d.elem = 2 * (int64_t)g.n_ecol * g.lines;
  d.rhs = 2 * (int64_t)g.ns;
  d.w = g.ns;
  return d;
}

constexpr int kDealiasThreads = 320;   // >= 17^2 Gauss points (M <= 2 kMaxP + 1)

// One CTA per element column: element-local over-integrated right-hand sides,
// weighted by the lumped-mass weight of each node (out[0 | 1][ecol][line]).
template <int DIM>
__global__ void __launch_bounds__(kDealiasThreads)
    dealias_elem_kernel(Geom g, Tables<double> t, int M, const double* tab, const double* metric, const double* eta,
                        const double* phis, const double* w, double* out) {
  extern __shared__ __align__(16) double dsm[];
  const int n = g.n, ecol = blockIdx.x, ex = ecol % g.nx, ey = ecol / g.nx;
  const int NQ = DIM == 3 ? M * M : M;
  double* B = dsm;
  double* Bd = B + M * n;
  double* Pi = Bd + M * n;
  double* E = Pi + n * M;        // nodal fields [a * n + b] (a: r index, b: s index)
  double* F = E + n * n;
  double* Wv = F + n * n;
  double* Ea = Wv + n * n;       // r-contracted [q * n + b]
  double* Era = Ea + M * n;
  double* Fa = Era + M * n;
  double* Fra = Fa + M * n;
  double* Wa = Fra + M * n;
  double* Fe = Wa + M * n;       // f at the Gauss points [q * M + r]
  double* Fp = Fe + NQ;
  double* Te = Fp + NQ;          // projected along r [i * M + r]
  double* Tp = Te + n * M;
  const int tid = threadIdx.x;
  for (int k = tid; k < 3 * M * n; k += blockDim.x) B[k] = tab[k];
  const int nl = DIM == 3 ? n * n : n;
  if (tid < nl) {
    const int a = tid % n, b = DIM == 3 ? tid / n : 0;
    const int col = node_col(g, ex, ey, a, b);
    E[a * n + b] = eta[col];
    F[a * n + b] = phis[col];
    Wv[a * n + b] = w[col];
  }
  __syncthreads();
  const int64_t HS = (int64_t)g.n_ecol * NQ;
  if (DIM == 3) {
    if (tid < M * n) {
      const int q = tid / n, b = tid % n;
      double ea = 0, era = 0, fa = 0, fra = 0, wa = 0;
      for (int a = 0; a < n; ++a) {
        const double bb = B[q * n + a], bd = Bd[q * n + a];
        ea += bb * E[a * n + b];
        era += bd * E[a * n + b];
        fa += bb * F[a * n + b];
        fra += bd * F[a * n + b];
        wa += bb * Wv[a * n + b];
      }
      Ea[q * n + b] = ea;
      Era[q * n + b] = era;
      Fa[q * n + b] = fa;
      Fra[q * n + b] = fra;
      Wa[q * n + b] = wa;
    }
    __syncthreads();
    if (tid < M * M) {
      const int q = tid / M, r = tid % M;
      double eq = 0, er = 0, es = 0, pr = 0, ps = 0, wq = 0;
      for (int b = 0; b < n; ++b) {
        const double bb = B[r * n + b], bd = Bd[r * n + b];
        eq += bb * Ea[q * n + b];
        es += bd * Ea[q * n + b];
        er += bb * Era[q * n + b];
        ps += bd * Fa[q * n + b];
        pr += bb * Fra[q * n + b];
        wq += bb * Wa[q * n + b];
      }
      const int64_t mi = (int64_t)ecol * NQ + tid;
      const double rx = metric[mi], ry = metric[HS + mi], sx = metric[2 * HS + mi], sy = metric[3 * HS + mi];
      const double ex_ = er * rx + es * sx, ey_ = er * ry + es * sy;
      const double px_ = pr * rx + ps * sx, py_ = pr * ry + ps * sy;
      const double ge2 = 1.0 + ex_ * ex_ + ey_ * ey_;
      Fe[tid] = -(ex_ * px_ + ey_ * py_) + wq * ge2;
      Fp[tid] = -g.g * eq - 0.5 * (px_ * px_ + py_ * py_) + 0.5 * wq * wq * ge2;
    }
    __syncthreads();
    if (tid < n * M) {
      const int i = tid / M, r = tid % M;
      double se = 0, sp = 0;
      for (int q = 0; q < M; ++q) {
        const double pi = Pi[i * M + q];
        se += pi * Fe[q * M + r];
        sp += pi * Fp[q * M + r];
      }
      Te[i * M + r] = se;
      Tp[i * M + r] = sp;
    }
    __syncthreads();
    if (tid < n * n) {
      const int i = tid % n, j = tid / n;   // line = j n + i
      double se = 0, sp = 0;
      for (int r = 0; r < M; ++r) {
        const double pi = Pi[j * M + r];
        se += pi * Te[i * M + r];
        sp += pi * Tp[i * M + r];
      }
      const int64_t hs = (int64_t)g.n_ecol * g.lines, li = (int64_t)ecol * g.lines + tid;
      const double cw = t.hm[4 * hs + li];
      out[li] = cw * se;
      out[hs + li] = cw * sp;
    }
  } else {
    if (tid < M) {
      const int q = tid;
      double eq = 0, er = 0, pr = 0, wq = 0;
      for (int a = 0; a < n; ++a) {
        const double bb = B[q * n + a], bd = Bd[q * n + a];
        eq += bb * E[a * n];
        er += bd * E[a * n];
        pr += bd * F[a * n];
        wq += bb * Wv[a * n];
      }
      const double rx = metric[(int64_t)ecol * NQ + q];
      const double ex_ = er * rx, px_ = pr * rx;
      const double ge2 = 1.0 + ex_ * ex_;
      Fe[q] = -ex_ * px_ + wq * ge2;
      Fp[q] = -g.g * eq - 0.5 * px_ * px_ + 0.5 * wq * wq * ge2;
    }
    __syncthreads();
    if (tid < n) {
      double se = 0, sp = 0;
      for (int q = 0; q < M; ++q) {
        const double pi = Pi[tid * M + q];
        se += pi * Fe[q];
        sp += pi * Fp[q];
      }
      const int64_t hs = (int64_t)g.n_ecol * g.lines, li = (int64_t)ecol * g.lines + tid;
      const double cw = t.hm[4 * hs + li];
      out[li] = cw * se;
      out[hs + li] = cw * sp;
    }
  }
}

// Per surface column: the weighted element values of every element sharing
// the node, in a fixed order, divided by the lumped mass.
__global__ void dealias_gather_kernel(Geom g, Tables<double> t, const double* elem, double* rhs) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= g.ns) return;
  const int ix = col % g.ncx, iy = col / g.ncx, P = g.p, n = g.n;
  int exo[2], io[2], eyo[2] = {0, 0}, jo[2] = {0, 0};
  const int cx = line_owners(ix, P, g.nx, g.px, exo, io);
  const int cy = g.dim == 3 ? line_owners(iy, P, g.ny, g.py, eyo, jo) : 1;
  const int64_t hs = (int64_t)g.n_ecol * g.lines;
  double se = 0, sp = 0;
  for (int u = 0; u < cx; ++u)
    for (int v = 0; v < cy; ++v) {
      const int64_t li = (int64_t)(eyo[v] * g.nx + exo[u]) * g.lines + jo[v] * n + io[u];
      se += elem[li];
      sp += elem[hs + li];
    }
  rhs[col] = se * t.minv[col];
  rhs[g.ns + col] = sp * t.minv[col];
}

}  // namespace

// The over-integrated right-hand side of the state (eta, phis) into
// m->dl_rhs ([ns] d eta/dt, then [ns] d phi/dt).  w: the given vertical
// velocity, or (NULL) the one recovered from the mesh potential m->phi in the
// geometry of eta.
cudaError_t enqueue_dealias_rhs(fnpf_mesh* m, const double* eta, const double* phis, const double* w,
                                cudaStream_t s) {
  const Geom& g = m->g;
  const DealiasLayout d = layout(g, m->dealias_M);
  double* wv = m->dl_buf + d.tab + d.metric + d.elem + d.rhs;
  cudaError_t e;
  if (!w) {
    if ((e = launch_w(g, m->tables(), m->geom_eta(eta), phis, m->phi, wv, s)) != cudaSuccess) return e;
    w = wv;
  }
  const double* tab = m->dl_buf;
  const double* metric = tab + d.tab;
  double* elem = m->dl_buf + d.tab + d.metric;
  double* rhs = elem + d.elem;
  const int n = g.n, M = d.M, NQ = d.Q;
  const size_t smem = sizeof(double) * (3 * (size_t)M * n + 3 * n * n + 5 * (size_t)M * n + 2 * (size_t)NQ +
                                        2 * (size_t)n * M);
  if (g.dim == 3) {
    static std::atomic<uint64_t> attr{0};
    if ((e = smem_optin(dealias_elem_kernel<3>, smem, &attr)) != cudaSuccess) return e;
    dealias_elem_kernel<3><<<g.n_ecol, kDealiasThreads, smem, s>>>(g, m->tables(), M, tab, metric, eta, phis, w,
                                                                    elem);
  } else {
    static std::atomic<uint64_t> attr{0};
    if ((e = smem_optin(dealias_elem_kernel<2>, smem, &attr)) != cudaSuccess) return e;
    dealias_elem_kernel<2><<<g.n_ecol, kDealiasThreads, smem, s>>>(g, m->tables(), M, tab, metric, eta, phis, w,
                                                                    elem);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  dealias_gather_kernel<<<(g.ns + 255) / 256, 256, 0, s>>>(g, m->tables(), elem, rhs);
  m->launches += w == wv ? 3 : 2;
  return cudaGetLastError();
}

const double* dealias_rhs(const fnpf_mesh* m) {
  const DealiasLayout d = layout(m->g, m->dealias_M);
  return m->dl_buf + d.tab + d.metric + d.elem;
}

}  // namespace fnpf

extern "C" fnpf_status fnpf_set_dealias(fnpf_mesh* m, int points) {
  using fnpf::Geom;
  if (!m) return FNPF_EINVAL;
  const Geom& g = m->g;
  if (points != 0 && (points < g.n || points > 2 * fnpf::kMaxP + 1)) {
    m->err = "over-integration points must be 0 (off) or in p+1 .. 17";
    return FNPF_EINVAL;
  }
  // the captured step includes or omits the over-integrated right-hand side
  if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
  m->step_exec = nullptr;
  if (m->dl_buf) cudaFree(m->dl_buf);
  m->dl_buf = nullptr;
  m->dealias_M = 0;
  if (points == 0) return FNPF_OK;
  const int n = g.n, M = points;
  const fnpf::DealiasLayout d = fnpf::layout(g, M);
  // host tables
  std::vector<double> xq(M), wq(M), tab(d.tab), metric(d.metric);
  fnpf::gauss_legendre(M, xq.data(), wq.data());
  double* B = tab.data();
  double* Bd = B + M * n;
  double* Pi = Bd + M * n;
  for (int q = 0; q < M; ++q)
    for (int a = 0; a < n; ++a) {
      double l = 1.0;   // Lagrange cardinal polynomial a on the GLL nodes at x_q
      for (int b = 0; b < n; ++b)
        if (b != a) l *= (xq[q] - m->xi[b]) / (m->xi[a] - m->xi[b]);
      B[q * n + a] = l;
    }
  for (int q = 0; q < M; ++q)   // Bd = B D: the derivative of the interpolant
    for (int a = 0; a < n; ++a) {
      double s = 0;
      for (int b = 0; b < n; ++b) s += B[q * n + b] * m->D[b * n + a];
      Bd[q * n + a] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < M; ++q) {
      double s = 0;
      for (int k = 0; k < n; ++k)
        s += fnpf::legendre_value(k, m->xi[i]) * (2.0 * k + 1.0) / 2.0 * fnpf::legendre_value(k, xq[q]);
      Pi[i * M + q] = s * wq[q];
    }
  // inverse horizontal metric at the Gauss points of every element
  const int64_t HS = (int64_t)g.n_ecol * d.Q;
  for (int ecol = 0; ecol < g.n_ecol; ++ecol) {
    const int ex = ecol % g.nx, ey = ecol / g.nx;
    if (g.dim == 2) {
      for (int q = 0; q < M; ++q) {
        double xr;
        if (!m->iso) {
          xr = 0.5 * m->Lx / g.nx;
        } else {
          xr = 0;
          for (int a = 0; a < n; ++a) xr += Bd[q * n + a] * m->Xs[fnpf::node_col(g, ex, ey, a, 0)];
        }
        metric[(int64_t)ecol * M + q] = 1.0 / xr;
      }
      continue;
    }
    for (int q = 0; q < M; ++q)
      for (int r = 0; r < M; ++r) {
        double xr, xs, yr, ys;
        if (!m->iso) {
          xr = 0.5 * m->Lx / g.nx;
          ys = 0.5 * m->Ly / g.ny;
          xs = yr = 0.0;
        } else {
          xr = xs = yr = ys = 0.0;
          for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
              const int c = fnpf::node_col(g, ex, ey, a, b);
              const double X = m->Xs[c], Y = m->Ys[c];
              xr += Bd[q * n + a] * B[r * n + b] * X;
              yr += Bd[q * n + a] * B[r * n + b] * Y;
              xs += B[q * n + a] * Bd[r * n + b] * X;
              ys += B[q * n + a] * Bd[r * n + b] * Y;
            }
        }
        const double J = xr * ys - xs * yr;
        if (!(std::fabs(J) > 0)) {
          m->err = "over-integration: singular horizontal Jacobian at a Gauss point";
          return FNPF_EINVAL;
        }
        const int64_t mi = (int64_t)ecol * d.Q + q * M + r;
        metric[mi] = ys / J;            // r_x
        metric[HS + mi] = -xs / J;      // r_y
        metric[2 * HS + mi] = -yr / J;  // s_x
        metric[3 * HS + mi] = xr / J;   // s_y
      }
  }
  const size_t total = (size_t)(d.tab + d.metric + d.elem + d.rhs + d.w);
  cudaError_t e = cudaMalloc((void**)&m->dl_buf, total * sizeof(double));
  if (e != cudaSuccess) {
    m->dl_buf = nullptr;
    m->err = "over-integration: device allocation failed";
    return FNPF_ENOMEM;
  }
  if ((e = cudaMemcpy(m->dl_buf, tab.data(), d.tab * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->dl_buf + d.tab, metric.data(), d.metric * sizeof(double), cudaMemcpyHostToDevice)) !=
          cudaSuccess) {
    m->err = std::string("over-integration: ") + cudaGetErrorString(e);
    return FNPF_ECUDA;
  }
  m->dealias_M = M;
  return FNPF_OK;
}

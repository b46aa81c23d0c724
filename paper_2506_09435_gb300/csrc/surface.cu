// Surface kernels: vertical-velocity recovery, Zakharov right-hand side with
// lumped GLL mass, and the fused RK4 stage update (arXiv 2506.09435, Sec. 2
// Eqs. kinematic/dynamic_free_surface_strong; Sec. 3.1.1 Eq. free_surface_weak;
// Sec. 3.2 ERK4; Sec. 3.4 Steps 4.4-4.6).
//
// One thread per surface node column.  w = d phi/dz = phi_t / z_t with
// z_t = (eta + h) / (2 Nz) and phi_t the GLL derivative along the top
// element's vertical line (unique across the elements sharing the node, since
// the mesh is extruded vertically).  The right-hand side is evaluated in every
// element sharing the node with the element-local horizontal gradients and
// combined with the lumped-mass weights w_i w_j |det H|:
//     d eta/dt = sum_e W_e f_eta,e / sum_e W_e  (likewise for phi).
// The 1/2 |grad phi|^2 term carries the sign of the strong (Bernoulli) form.
// Linear potential flow (model FNPF_LINEAR) takes z_t from the still-water
// depth and the linear conditions d eta/dt = w, d phi/dt = -g eta.
#include <math.h>

#include "fnpf_internal.cuh"

namespace fnpf {
namespace {

__device__ inline double top_w(const Geom& g, const double* D, const double* phi, const double* phis,
                               const double* h, const double* eta, int col) {
  const int P = g.p;
  double s = 0;
  for (int j = 0; j < P; ++j) s += D[P * g.n + j] * phi[(int64_t)(g.nv - 1 - P + j) * g.ns + col];
  s += D[P * g.n + P] * phis[col];
  return s * (2.0 * g.nz) / (eta[col] + h[col]);
}

// Zakharov right-hand side at surface column col (ix, iy): the conditions in
// every element sharing the node, combined with the lumped-mass weights.
__device__ inline void zakharov_node(const Geom& g, const Tables<double>& t, const StageArgs& a, int col, int ix,
                                     int iy, double w, double e0, double* ke, double* kp) {
  const int P = g.p, n = g.n;
  int exo[2], io[2], eyo[2] = {0, 0}, jo[2] = {0, 0};
  const int cx = line_owners(ix, P, g.nx, g.px, exo, io);
  const int cy = g.dim == 3 ? line_owners(iy, P, g.ny, g.py, eyo, jo) : 1;
  const int64_t hstride = (int64_t)g.n_ecol * g.lines;
  double se = 0, sp = 0;
  for (int u = 0; u < cx; ++u) {
    for (int v = 0; v < cy; ++v) {
      const int ex = exo[u], ey = eyo[v], i = io[u], j = jo[v];
      const int ecol = ey * g.nx + ex;
      const int line = j * n + i;
      double er = 0, pr = 0, es = 0, ps = 0;
      for (int m = 0; m < n; ++m) {
        const double d = t.D[i * n + m];
        const int c2 = node_col(g, ex, ey, m, j);
        er += d * a.eta[c2];
        pr += d * a.phis[c2];
      }
      if (g.dim == 3) {
        for (int m = 0; m < n; ++m) {
          const double d = t.D[j * n + m];
          const int c2 = node_col(g, ex, ey, i, m);
          es += d * a.eta[c2];
          ps += d * a.phis[c2];
        }
      }
      const int64_t hidx = (int64_t)ecol * g.lines + line;
      const double rx = t.hm[hidx], ry = t.hm[hstride + hidx], sx = t.hm[2 * hstride + hidx],
                   sy = t.hm[3 * hstride + hidx], cw = t.hm[4 * hstride + hidx];
      const double ex_ = er * rx + es * sx, ey_ = er * ry + es * sy;   // grad eta
      const double px_ = pr * rx + ps * sx, py_ = pr * ry + ps * sy;   // grad phi
      const double ge2 = 1.0 + ex_ * ex_ + ey_ * ey_;
      const double fe = -(ex_ * px_ + ey_ * py_) + w * ge2;
      const double fp = -g.g * e0 - 0.5 * (px_ * px_ + py_ * py_) + 0.5 * w * w * ge2;
      se += cw * fe;
      sp += cw * fp;
    }
  }
  *ke = se * t.minv[col];
  *kp = sp * t.minv[col];
}

struct stage_kernel {
  static constexpr int kThreads = 128;
  __device__ static void run(Blk bk, Geom g, Tables<double> t, StageArgs a) {
    const int col = bk.x * blockDim.x + threadIdx.x;
    if (col >= g.ns) return;
    const int ix = col % g.ncx, iy = col / g.ncx;
    const double e0 = a.eta[col];
    const double hh = t.h[col];
    if (!(e0 + hh > 0.0) || !isfinite(e0) || !isfinite(a.phis[col])) {
      if (a.status) atomicExch(a.status, (int)FNPF_EDIVERGED);
    }
    double ke, kp;
    if (a.rhs_in && !a.linear) {
      // over-integrated right-hand side (dealias.cu)
      ke = a.rhs_in[col];
      kp = a.rhs_in[g.ns + col];
    } else if (a.linear) {
      const double w = a.w_in ? a.w_in[col] : top_w(g, t.D, a.phi, a.phis, t.h, a.geo ? a.geo : a.eta, col);
      // linear potential flow: the surface conditions linearised about z = 0
      ke = w;
      kp = -g.g * e0;
    } else {
      const double w = a.w_in ? a.w_in[col] : top_w(g, t.D, a.phi, a.phis, t.h, a.geo ? a.geo : a.eta, col);
      zakharov_node(g, t, a, col, ix, iy, w, e0, &ke, &kp);
    }
    if (a.deta) {
      a.deta[col] = ke;
      a.dphis[col] = kp;
    }
    if (a.out_eta) {
      const double acc_e = (a.first ? 0.0 : a.acc_eta[col]) + a.bw * ke;
      const double acc_p = (a.first ? 0.0 : a.acc_phi[col]) + a.bw * kp;
      const double y0e = a.y0_eta[col], y0p = a.y0_phi[col];
      if (a.last) {
        double ye = y0e + a.dt * acc_e, yp = y0p + a.dt * acc_p;
        if (a.cr) {
          // relaxation zones: f <- (1 - C_r) f + C_r f_true at t + dt
          const double c = a.cr[col];
          if (c != 0.0) {
            double te = 0.0, tp = 0.0;
            if (a.gen[col] != 0.0) {
              const double t_end = a.t_dev ? *a.t_dev + a.dt : a.t_end;
              const double ramp = fmin(1.0, t_end / a.ramp_time);
              const double th = a.kx * a.xs[col] + a.ky * a.ys[col] - a.omega * t_end + a.phase;
              const double k = hypot(a.kx, a.ky);
              te = ramp * a.amp * cos(th);
              tp = ramp * (g.g * a.amp / a.omega) * cosh(k * (te + hh)) / cosh(k * hh) * sin(th);
            }
            ye = (1.0 - c) * ye + c * te;
            yp = (1.0 - c) * yp + c * tp;
          }
        }
        a.out_eta[col] = ye;
        a.out_phi[col] = yp;
      } else {
        a.acc_eta[col] = acc_e;
        a.acc_phi[col] = acc_p;
        a.out_eta[col] = y0e + a.cn * ke;
        a.out_phi[col] = y0p + a.cn * kp;
      }
    }
  }
};

struct w_kernel {
  static constexpr int kThreads = 128;
  __device__ static void run(Blk bk, Geom g, Tables<double> t, const double* eta, const double* phis,
                             const double* phi, double* w) {
    const int col = bk.x * blockDim.x + threadIdx.x;
    if (col >= g.ns) return;
    w[col] = top_w(g, t.D, phi, phis, t.h, eta, col);
  }
};

struct check_state_kernel {
  static constexpr int kThreads = 128;
  __device__ static void run(Blk bk, Geom g, const double* eta, const double* phis, const double* h, int* status,
                             int* done) {
    const int col = bk.x * blockDim.x + threadIdx.x;
    if (col >= g.ns) return;
    const double e = eta[col];
    if (!(e + h[col] > 0.0) || !isfinite(e) || !isfinite(phis[col])) {
      atomicExch(status, (int)FNPF_EDIVERGED);
      atomicExch(done, 1);
    }
  }
};

}  // namespace

cudaError_t launch_stage(const Geom& g, const Tables<double>& t, const StageArgs& a, cudaStream_t s) {
  const int threads = 128;
  launch<stage_kernel>((g.ns + threads - 1) / threads, threads, 0, s, g, t, a);
  return cudaGetLastError();
}

cudaError_t launch_w(const Geom& g, const Tables<double>& t, const double* eta, const double* phis,
                     const double* phi, double* w, cudaStream_t s) {
  const int threads = 128;
  launch<w_kernel>((g.ns + threads - 1) / threads, threads, 0, s, g, t, eta, phis, phi, w);
  return cudaGetLastError();
}

namespace {

// One thread per surface column: an element-interior node (i, j) of element
// column (ex, ey) gets sum_a sum_b F[i][a] F[j][b] f(a, b) (sum_a F[i][a] f(a)
// in a 2D slice); every other node is copied.
struct filter_kernel {
  static constexpr int kThreads = 128;
  __device__ static void run(Blk bk, Geom g, const double* __restrict__ F, const double* __restrict__ in0,
                             double* __restrict__ out0, const double* __restrict__ in1, double* __restrict__ out1) {
    const int col = bk.x * blockDim.x + threadIdx.x;
    if (col >= g.ns) return;
    const int P = g.p, n = g.n;
    const int ix = col % g.ncx, iy = col / g.ncx;
    const int i = ix % P, j = g.dim == 3 ? iy % P : 0;
    const bool interior = i != 0 && (g.dim == 2 || j != 0);
    if (!interior) {
      out0[col] = in0[col];
      if (in1) out1[col] = in1[col];
      return;
    }
    const int ex = ix / P, ey = g.dim == 3 ? iy / P : 0;
    double s0 = 0.0, s1 = 0.0;
    for (int b = 0; b < (g.dim == 3 ? n : 1); ++b) {
      double t0 = 0.0, t1 = 0.0;
      for (int a = 0; a < n; ++a) {
        const int c = node_col(g, ex, ey, a, b);
        t0 += F[i * n + a] * in0[c];
        if (in1) t1 += F[i * n + a] * in1[c];
      }
      const double fj = g.dim == 3 ? F[j * n + b] : 1.0;
      s0 += fj * t0;
      s1 += fj * t1;
    }
    out0[col] = s0;
    if (in1) out1[col] = s1;
  }
};

}  // namespace

cudaError_t launch_filter(const Geom& g, const double* F, const double* in0, double* out0, const double* in1,
                          double* out1, cudaStream_t s) {
  const int threads = 128;
  launch<filter_kernel>((g.ns + threads - 1) / threads, threads, 0, s, g, F, in0, out0, in1, out1);
  return cudaGetLastError();
}

cudaError_t launch_check_state(const Geom& g, const double* eta, const double* phis, const double* h, int* status,
                               int* done, cudaStream_t s) {
  const int threads = 128;
  launch<check_state_kernel>((g.ns + threads - 1) / threads, threads, 0, s, g, eta, phis, h, status, done);
  return cudaGetLastError();
}

}  // namespace fnpf

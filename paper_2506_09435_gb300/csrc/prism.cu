// Prism elements over an unstructured triangular surface mesh (the paper's
// own mesh, Sec. 3.1.2: a triangular surface mesh extruded into N_z layers
// whose columns follow the free surface): the stiffness operator of the weak
// Laplace form (Eq. Laplace_weak) applied matrix-free.
//
// Element: the degree-p polynomials on the triangle times the degree-p GLL
// Lagrange basis in the vertical; triangle nodes of Blyth & Pozrikidis (2006)
// from the 1D GLL points; straight-sided triangles; z = -h + sigma (eta + h),
// sigma = (l + (1 + t) / 2) / N_z with eta, h in the triangle's nodal basis;
// a collapsed Gauss-Legendre rule on the triangle ((p + 2)^2 points, exact for
// degree 2p + 2) times GLL collocation in the vertical.  Numbering: surface
// nodes are the mesh vertices, then p - 1 nodes per edge (edges in order of
// first appearance over the triangles' edges (A,B), (B,C), (A,C); nodes from
// the lower to the higher vertex number), then each triangle's interior
// nodes; volume node (plane k, surface node c) is k * Ns + c.
//
// One CTA per prism (triangle, layer): the element's values and the eta, h
// of its triangle go to shared memory; each thread takes quadrature points
// (q, k) -- geometry, metric G = w |det J| J^-1 J^-T and the flux G grad u --
// then local nodes (the transposed contractions); the element results go to
// a buffer that a gather kernel sums per node along a fixed incidence list
// (deterministic, no atomics).
#include <math.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "fnpf_internal.cuh"
#include "prism.cuh"


namespace {

std::string g_prism_error;

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the
// Chebyshev guesses, long double).
void gauss_legendre_host(int n, std::vector<double>* x, std::vector<double>* w) {
  x->assign(n, 0.0);
  w->assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    long double z = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (n + 0.5L));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) {
        p1 = z;
        p0 = 1;
      }
      dp = n * (z * p1 - p0) / (z * z - 1);
      const long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    (*x)[n - 1 - i] = (double)z;
    (*w)[n - 1 - i] = (double)(2 / ((1 - z * z) * dp * dp));
  }
}

// Local triangle nodes (i, j), i + j <= p, j outer.
std::vector<std::pair<int, int>> tri_index(int p) {
  std::vector<std::pair<int, int>> v;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i + j <= p; ++i) v.emplace_back(i, j);
  return v;
}

// Monomials u^a v^b (u = (1 + r) / 2, v = (1 + s) / 2) and their r, s
// derivatives at (r, s), in tri_index order.
void monomials(int p, double r, double s, double* M, double* Mr, double* Ms) {
  const double u = 0.5 * (1 + r), v = 0.5 * (1 + s);
  int c = 0;
  for (auto [a, b] : tri_index(p)) {
    M[c] = pow(u, a) * pow(v, b);
    Mr[c] = a > 0 ? 0.5 * a * pow(u, a - 1) * pow(v, b) : 0.0;
    Ms[c] = b > 0 ? 0.5 * b * pow(u, a) * pow(v, b - 1) : 0.0;
    ++c;
  }
}

// Inverse of the n x n matrix A (row-major) by Gauss-Jordan elimination with
// partial pivoting in long double; false if singular.
bool invert(int n, const std::vector<double>& A, std::vector<double>* inv) {
  std::vector<long double> a(A.begin(), A.end()), b(n * n, 0.0L);
  for (int i = 0; i < n; ++i) b[i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(a[r * n + c]) > fabsl(a[piv * n + c])) piv = r;
    if (fabsl(a[piv * n + c]) < 1e-300L) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(b[c * n + k], b[piv * n + k]);
      }
    const long double d = a[c * n + c];
    for (int k = 0; k < n; ++k) {
      a[c * n + k] /= d;
      b[c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const long double f = a[r * n + c];
      if (f == 0) continue;
      for (int k = 0; k < n; ++k) {
        a[r * n + k] -= f * a[c * n + k];
        b[r * n + k] -= f * b[c * n + k];
      }
    }
  }
  inv->assign(b.begin(), b.end());
  return true;
}

}  // namespace

namespace fnpf {

// Host tables of order p: triangle nodes (r, s) [nt], quadrature (r, s, w)
// [nq], basis values and derivatives at the quadrature points [nq][nt].
bool prism_tables(int p, std::vector<double>* rn, std::vector<double>* sn, std::vector<double>* wq,
                  std::vector<double>* L, std::vector<double>* Lr, std::vector<double>* Ls) {
  const int n = p + 1;
  std::vector<double> xi(n), w(n), D(n * n);
  gll_tables(p, xi.data(), w.data(), D.data());
  const auto idx = tri_index(p);
  const int nt = (int)idx.size();
  rn->clear();
  sn->clear();
  for (auto [i, j] : idx) {
    const int k = p - i - j;
    const double vi = 0.5 * (1 + xi[i]), vj = 0.5 * (1 + xi[j]), vk = 0.5 * (1 + xi[k]);
    const double lb = (1 + 2 * vi - vj - vk) / 3.0, lc = (1 + 2 * vj - vi - vk) / 3.0;
    rn->push_back(2 * lb - 1);
    sn->push_back(2 * lc - 1);
  }
  std::vector<double> V(nt * nt), tmp1(nt), tmp2(nt), C;
  for (int q = 0; q < nt; ++q) monomials(p, (*rn)[q], (*sn)[q], &V[q * nt], tmp1.data(), tmp2.data());
  if (!invert(nt, V, &C)) return false;
  const int ng = p + 2;
  std::vector<double> ga, gw;
  gauss_legendre_host(ng, &ga, &gw);
  const int nq = ng * ng;
  wq->assign(nq, 0.0);
  L->assign(nq * nt, 0.0);
  Lr->assign(nq * nt, 0.0);
  Ls->assign(nq * nt, 0.0);
  std::vector<double> M(nt), Mr(nt), Ms(nt);
  for (int jb = 0; jb < ng; ++jb)
    for (int ia = 0; ia < ng; ++ia) {
      const int q = jb * ng + ia;
      const double a = ga[ia], b = ga[jb];
      const double r = 0.5 * (1 + a) * (1 - b) - 1, s = b;
      (*wq)[q] = gw[ia] * gw[jb] * 0.5 * (1 - b);
      monomials(p, r, s, M.data(), Mr.data(), Ms.data());
      for (int c = 0; c < nt; ++c) {
        double v = 0, vr = 0, vs = 0;
        for (int k = 0; k < nt; ++k) {
          v += M[k] * C[k * nt + c];
          vr += Mr[k] * C[k * nt + c];
          vs += Ms[k] * C[k * nt + c];
        }
        (*L)[q * nt + c] = v;
        (*Lr)[q * nt + c] = vr;
        (*Ls)[q * nt + c] = vs;
      }
    }
  return true;
}

// Surface numbering of the order-p nodes of a triangle mesh: tnodes [ntri][nt],
// coordinates; false on a bad triangle (vertex out of range or repeated).
bool prism_numbering(const double* verts, int nverts, const int* tris, int ntri, int p, std::vector<int>* tnodes,
                     std::vector<double>* xs, std::vector<double>* ys) {
  const auto idx = tri_index(p);
  const int nt = (int)idx.size();
  // (min, max) vertex pair -> first node of the edge, edges numbered in order of first appearance
  std::map<std::pair<int, int>, int> edge_first;
  int nedges = 0;
  auto find_edge = [&](int u, int w) {
    const auto it = edge_first.find(std::pair<int, int>(std::min(u, w), std::max(u, w)));
    return it == edge_first.end() ? -1 : it->second;
  };
  for (int t = 0; t < ntri; ++t) {
    const int A = tris[3 * t], B = tris[3 * t + 1], C = tris[3 * t + 2];
    if (A < 0 || B < 0 || C < 0 || A >= nverts || B >= nverts || C >= nverts || A == B || B == C || A == C)
      return false;
    const int pairs[3][2] = {{A, B}, {B, C}, {A, C}};
    for (auto& pr : pairs)
      if (find_edge(pr[0], pr[1]) < 0)
        edge_first[{std::min(pr[0], pr[1]), std::max(pr[0], pr[1])}] = nverts + (nedges++) * (p - 1);
  }
  int n = nverts + nedges * (p - 1);
  tnodes->assign((size_t)ntri * nt, 0);
  auto edge_node = [&](int u, int w, int m) {
    const int base = find_edge(u, w);
    return base + (u < w ? m : p - m) - 1;
  };
  for (int t = 0; t < ntri; ++t) {
    const int A = tris[3 * t], B = tris[3 * t + 1], C = tris[3 * t + 2];
    for (int q = 0; q < nt; ++q) {
      const int i = idx[q].first, j = idx[q].second, k = p - i - j;
      int g;
      if (i == 0 && j == 0) g = A;
      else if (i == p && j == 0) g = B;
      else if (i == 0 && j == p) g = C;
      else if (j == 0) g = edge_node(A, B, i);
      else if (k == 0) g = edge_node(B, C, j);
      else if (i == 0) g = edge_node(A, C, j);
      else g = n++;
      (*tnodes)[(size_t)t * nt + q] = g;
    }
  }
  std::vector<double> rn, sn, wq, L, Lr, Ls;
  if (!prism_tables(p, &rn, &sn, &wq, &L, &Lr, &Ls)) return false;
  xs->assign(n, 0.0);
  ys->assign(n, 0.0);
  for (int t = 0; t < ntri; ++t) {
    const int A = tris[3 * t], B = tris[3 * t + 1], C = tris[3 * t + 2];
    for (int q = 0; q < nt; ++q) {
      const double lb = 0.5 * (1 + rn[q]), lc = 0.5 * (1 + sn[q]), la = 1 - lb - lc;
      const int g = (*tnodes)[(size_t)t * nt + q];
      (*xs)[g] = la * verts[2 * A] + lb * verts[2 * B] + lc * verts[2 * C];
      (*ys)[g] = la * verts[2 * A + 1] + lb * verts[2 * B + 1] + lc * verts[2 * C + 1];
    }
  }
  return true;
}

namespace {

struct PrismArgs {
  int p, n, nz, nt, nq, ns;
  const int* tnodes;
  const double* geo;
  const double* L;
  const double* Lr;
  const double* Ls;
  const double* wq;
  const double* xi;
  const double* wv;
  const double* D;
  const double* eta;
  const double* h;
  const double* x;
  double* ye;
};

constexpr int kPrismThreads = 128;

// One prism (triangle e = block / nz, layer l = block % nz).  Shared memory:
// u [nt n], E, H [nt], flux [3][n nq].
struct prism_apply_kernel {
  static constexpr int kThreads = kPrismThreads;
  __device__ static void run(Blk bk, PrismArgs a) {
    extern __shared__ __align__(16) unsigned char prism_smem[];
    double* su = reinterpret_cast<double*>(prism_smem);
    double* sE = su + a.nt * a.n;
    double* sH = sE + a.nt;
    double* sf = sH + a.nt;                      // [3][n * nq], point index k * nq + q
    const int elem = bk.x;
    const int e = elem / a.nz, l = elem - e * a.nz;
    const int nt = a.nt, n = a.n, nq = a.nq, P = a.p;
    const int* tn = a.tnodes + (size_t)e * nt;
    for (int idx = threadIdx.x; idx < nt * n; idx += blockDim.x) {
      const int q = idx % nt, m = idx / nt;
      su[idx] = a.x[(int64_t)(l * P + m) * a.ns + tn[q]];
    }
    for (int q = threadIdx.x; q < nt; q += blockDim.x) {
      sE[q] = a.eta[tn[q]];
      sH[q] = a.h[tn[q]];
    }
    __syncthreads();
    const double xr = a.geo[4 * e], xs = a.geo[4 * e + 1], yr = a.geo[4 * e + 2], ys = a.geo[4 * e + 3];
    const double det2 = xr * ys - xs * yr;
    for (int pt = threadIdx.x; pt < n * nq; pt += blockDim.x) {
      const int k = pt / nq, q = pt - k * nq;
      const double* Lq = a.L + (size_t)q * nt;
      const double* Lrq = a.Lr + (size_t)q * nt;
      const double* Lsq = a.Ls + (size_t)q * nt;
      double ev = 0, er = 0, es = 0, hv = 0, hr = 0, hs = 0, ur = 0, us = 0, ut = 0;
      for (int c = 0; c < nt; ++c) {
        ev += Lq[c] * sE[c];
        er += Lrq[c] * sE[c];
        es += Lsq[c] * sE[c];
        hv += Lq[c] * sH[c];
        hr += Lrq[c] * sH[c];
        hs += Lsq[c] * sH[c];
        ur += Lrq[c] * su[k * nt + c];
        us += Lsq[c] * su[k * nt + c];
        double uc = 0;
        for (int m = 0; m < n; ++m) uc += a.D[k * n + m] * su[m * nt + c];
        ut += Lq[c] * uc;
      }
      const double sig = (l + 0.5 * (1.0 + a.xi[k])) / a.nz;
      const double zr = -hr + sig * (er + hr), zs = -hs + sig * (es + hs), zt = (ev + hv) / (2.0 * a.nz);
      // J = [[xr, xs, 0], [yr, ys, 0], [zr, zs, zt]]; J^-1 by cofactors
      const double det = det2 * zt;
      const double i00 = ys * zt / det, i01 = -xs * zt / det, i02 = 0.0;
      const double i10 = -yr * zt / det, i11 = xr * zt / det, i12 = 0.0;
      const double i20 = (yr * zs - ys * zr) / det, i21 = (xs * zr - xr * zs) / det, i22 = det2 / det;
      // physical gradient g = J^-T (ur, us, ut); flux = wt J^-1 g
      const double gx = i00 * ur + i10 * us + i20 * ut;
      const double gy = i01 * ur + i11 * us + i21 * ut;
      const double gz = i02 * ur + i12 * us + i22 * ut;
      const double wt = a.wq[q] * a.wv[k] * fabs(det);
      sf[pt] = wt * (i00 * gx + i01 * gy + i02 * gz);
      sf[n * nq + pt] = wt * (i10 * gx + i11 * gy + i12 * gz);
      sf[2 * n * nq + pt] = wt * (i20 * gx + i21 * gy + i22 * gz);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nt * n; idx += blockDim.x) {
      const int c = idx % nt, m = idx / nt;
      double y = 0;
      for (int q = 0; q < nq; ++q)
        y += a.Lr[(size_t)q * nt + c] * sf[m * nq + q] + a.Ls[(size_t)q * nt + c] * sf[n * nq + m * nq + q];
      for (int k = 0; k < n; ++k) {
        const double dkm = a.D[k * n + m];
        double s = 0;
        for (int q = 0; q < nq; ++q) s += a.L[(size_t)q * nt + c] * sf[2 * n * nq + k * nq + q];
        y += dkm * s;
      }
      a.ye[(size_t)elem * nt * n + idx] = y;
    }
  }
};

// y_g = sum of the element results of node g, in a fixed order.
struct prism_gather_kernel {
  static constexpr int kThreads = 256;
  __device__ static void run(Blk bk, int64_t N, const int64_t* off, const int64_t* inc, const double* ye,
                             double* y) {
    const int64_t g = (int64_t)bk.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    double s = 0;
    for (int64_t j = off[g]; j < off[g + 1]; ++j) s += ye[inc[j]];
    y[g] = s;
  }
};

}  // namespace
}  // namespace fnpf

extern "C" {

fnpf_status fnpf_prism_numbering(const double* verts, int nverts, const int* tris, int ntris, int p, int* tnodes,
                                 double* x, double* y, int* ns) {
  if (!verts || !tris || !ns || nverts < 3 || ntris < 1 || p < 1 || p > fnpf::kMaxP) return FNPF_EINVAL;
  std::vector<int> tn;
  std::vector<double> xs, ys;
  if (!fnpf::prism_numbering(verts, nverts, tris, ntris, p, &tn, &xs, &ys)) return FNPF_EINVAL;
  *ns = (int)xs.size();
  if (tnodes) std::copy(tn.begin(), tn.end(), tnodes);
  if (x) std::copy(xs.begin(), xs.end(), x);
  if (y) std::copy(ys.begin(), ys.end(), y);
  return FNPF_OK;
}

fnpf_status fnpf_prism_tables(int p, double* L, double* Lr, double* Ls, double* wq, int* nq) {
  if (p < 1 || p > fnpf::kMaxP || !nq) return FNPF_EINVAL;
  std::vector<double> rn, sn, w, l, lr, ls;
  if (!fnpf::prism_tables(p, &rn, &sn, &w, &l, &lr, &ls)) return FNPF_EINVAL;
  *nq = (int)w.size();
  if (L) std::copy(l.begin(), l.end(), L);
  if (Lr) std::copy(lr.begin(), lr.end(), Lr);
  if (Ls) std::copy(ls.begin(), ls.end(), Ls);
  if (wq) std::copy(w.begin(), w.end(), wq);
  return FNPF_OK;
}

void fnpf_prism_destroy(fnpf_prism* m) {
  if (!m) return;
  fnpf::prism_step_free(m);
  cudaFree(m->d_tnodes);
  cudaFree(m->d_tab);
  cudaFree(m->d_ye);
  cudaFree(m->d_off);
  cudaFree(m->d_inc);
  delete m;
}

fnpf_status fnpf_prism_create(const double* verts, int nverts, const int* tris, int ntris, int p, int nz,
                              fnpf_prism** out) {
  if (!out) return FNPF_EINVAL;
  *out = nullptr;
  if (!verts || !tris || nverts < 3 || ntris < 1 || p < 1 || p > fnpf::kMaxP || nz < 1) {
    g_prism_error = "bad sizes or null arrays";
    return FNPF_EINVAL;
  }
  fnpf_prism* m = new fnpf_prism();
  m->p = p;
  m->n = p + 1;
  m->nz = nz;
  m->ntri = ntris;
  m->verts.assign(verts, verts + 2 * (size_t)nverts);
  m->tris.assign(tris, tris + 3 * (size_t)ntris);
  if (!fnpf::prism_numbering(verts, nverts, tris, ntris, p, &m->tnodes, &m->xs, &m->ys)) {
    g_prism_error = "bad triangle (vertex out of range or repeated)";
    delete m;
    return FNPF_EINVAL;
  }
  std::vector<double> rn, sn, wq, L, Lr, Ls;
  fnpf::prism_tables(p, &rn, &sn, &wq, &L, &Lr, &Ls);
  m->nt = (int)rn.size();
  m->nq = (int)wq.size();
  m->ns = (int)m->xs.size();
  m->nv = nz * p + 1;
  m->N = (int64_t)m->nv * m->ns;
  const int n = m->n, nt = m->nt, nq = m->nq;
  // geometry of each triangle: dx/dr, dx/ds, dy/dr, dy/ds (affine); positive area
  std::vector<double> geo(4 * (size_t)ntris);
  for (int t = 0; t < ntris; ++t) {
    const int A = tris[3 * t], B = tris[3 * t + 1], C = tris[3 * t + 2];
    geo[4 * t] = 0.5 * (verts[2 * B] - verts[2 * A]);
    geo[4 * t + 1] = 0.5 * (verts[2 * C] - verts[2 * A]);
    geo[4 * t + 2] = 0.5 * (verts[2 * B + 1] - verts[2 * A + 1]);
    geo[4 * t + 3] = 0.5 * (verts[2 * C + 1] - verts[2 * A + 1]);
    const double d = geo[4 * t] * geo[4 * t + 3] - geo[4 * t + 1] * geo[4 * t + 2];
    if (!(d > 0) || !isfinite(d)) {
      g_prism_error = "triangle with zero or negative area (vertices must be counter-clockwise)";
      delete m;
      return FNPF_EINVAL;
    }
  }
  std::vector<double> xi(n), wv(n), D(n * n);
  fnpf::gll_tables(p, xi.data(), wv.data(), D.data());
  std::vector<double> tab;
  tab.insert(tab.end(), geo.begin(), geo.end());
  tab.insert(tab.end(), L.begin(), L.end());
  tab.insert(tab.end(), Lr.begin(), Lr.end());
  tab.insert(tab.end(), Ls.begin(), Ls.end());
  tab.insert(tab.end(), wq.begin(), wq.end());
  tab.insert(tab.end(), xi.begin(), xi.end());
  tab.insert(tab.end(), wv.begin(), wv.end());
  tab.insert(tab.end(), D.begin(), D.end());
  // incidence of every volume node, in (element, local node) order
  const int64_t nelem = (int64_t)ntris * nz;
  std::vector<int64_t> off(m->N + 1, 0);
  for (int t = 0; t < ntris; ++t)
    for (int l = 0; l < nz; ++l)
      for (int mm = 0; mm < n; ++mm)
        for (int q = 0; q < nt; ++q) ++off[(int64_t)(l * p + mm) * m->ns + m->tnodes[(size_t)t * nt + q] + 1];
  for (int64_t g = 0; g < m->N; ++g) off[g + 1] += off[g];
  std::vector<int64_t> inc(off[m->N]), fill(off.begin(), off.end() - 1);
  for (int t = 0; t < ntris; ++t)
    for (int l = 0; l < nz; ++l) {
      const int64_t elem = (int64_t)t * nz + l;
      for (int mm = 0; mm < n; ++mm)
        for (int q = 0; q < nt; ++q) {
          const int64_t g = (int64_t)(l * p + mm) * m->ns + m->tnodes[(size_t)t * nt + q];
          inc[fill[g]++] = elem * nt * n + (int64_t)mm * nt + q;
        }
    }
  cudaError_t e = cudaMalloc(&m->d_tnodes, m->tnodes.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_tab, tab.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_ye, (size_t)nelem * nt * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_off, off.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_inc, std::max<size_t>(1, inc.size()) * sizeof(int64_t));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_tnodes, m->tnodes.data(), m->tnodes.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !inc.empty())
    e = cudaMemcpy(m->d_inc, inc.data(), inc.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    g_prism_error = std::string("device set-up failed: ") + cudaGetErrorString(e);
    fnpf_prism_destroy(m);
    return e == cudaErrorMemoryAllocation ? FNPF_ENOMEM : FNPF_ECUDA;
  }
  (void)nq;
  *out = m;
  return FNPF_OK;
}

fnpf_status fnpf_prism_sizes(const fnpf_prism* m, int64_t* n_vol, int64_t* n_surf) {
  if (!m) return FNPF_EINVAL;
  if (n_vol) *n_vol = m->N;
  if (n_surf) *n_surf = m->ns;
  return FNPF_OK;
}

fnpf_status fnpf_prism_apply(fnpf_prism* m, const double* eta, const double* h, const double* x, double* y,
                             void* stream) {
  if (!m || !eta || !h || !x || !y) return FNPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = m->n, nt = m->nt, nq = m->nq;
  const double* tab = m->d_tab;
  fnpf::PrismArgs a{};
  a.p = m->p;
  a.n = n;
  a.nz = m->nz;
  a.nt = nt;
  a.nq = nq;
  a.ns = m->ns;
  a.tnodes = m->d_tnodes;
  a.geo = tab;
  a.L = a.geo + 4 * (size_t)m->ntri;
  a.Lr = a.L + (size_t)nq * nt;
  a.Ls = a.Lr + (size_t)nq * nt;
  a.wq = a.Ls + (size_t)nq * nt;
  a.xi = a.wq + nq;
  a.wv = a.xi + n;
  a.D = a.wv + n;
  a.eta = eta;
  a.h = h;
  a.x = x;
  a.ye = m->d_ye;
  const size_t smem = sizeof(double) * ((size_t)nt * n + 2 * (size_t)nt + 3 * (size_t)n * nq);
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = fnpf::smem_optin(fnpf::kernel_one<fnpf::prism_apply_kernel>(), smem, &attr);
  const unsigned blocks = (unsigned)((int64_t)m->ntri * m->nz);
  if (e == cudaSuccess) e = fnpf::launch<fnpf::prism_apply_kernel>(blocks, fnpf::kPrismThreads, smem, s, a);
  if (e == cudaSuccess)
    e = fnpf::launch<fnpf::prism_gather_kernel>((unsigned)((m->N + 255) / 256), 256, 0, s, m->N,
                                                (const int64_t*)m->d_off, (const int64_t*)m->d_inc,
                                                (const double*)m->d_ye, y);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    m->err = std::string("prism apply: ") + cudaGetErrorString(e);
    return FNPF_ECUDA;
  }
  return FNPF_OK;
}

const char* fnpf_prism_last_error(const fnpf_prism* m) { return m ? m->err.c_str() : g_prism_error.c_str(); }

}  // extern "C"

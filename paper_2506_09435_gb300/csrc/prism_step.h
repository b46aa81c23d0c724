// The Laplace solve, the Dirichlet-to-Neumann map and the RK4 step on prisms
// over an unstructured triangular surface mesh (the paper's own mesh, Sec.
// 3.1.2), as one-thread-per-item kernels and the host orchestration that
// launches them.
//
// Every kernel of this path is an item struct with a static function
// at(i, args) that one thread runs for item i (no shared memory, no
// synchronisation inside a launch, every output written by exactly one item),
// so the same bodies run as CUDA kernels (prism_step.cu: one thread per item)
// and, compiled as plain C++, one item after another.  Stepper<Ex> orders the
// launches; Ex supplies run<Item>(n, args), run_block<Block>(blocks, smem
// bytes, args) for the block kernels and get(host, src, count), the
// device-to-host read of the CG loops' state (their scalars stay on the
// device; the host tests the stop flag).
//
// Per RK4 stage (Sec. 3.4, Steps 4.1-4.6; ERK4, Sec. 3.2):
//   geometry  G = w_q w_k |det J| J^-1 J^-T at every quadrature point of every
//             prism, from eta and h (z = -h + sigma (eta + h)), stored for the
//             solve, and the Jacobi diagonal from it;
//   lift      b = -A_IS phi_eta (the operator applied to the surface values);
//   PCG       A_II phi_I = b (Eq. Laplace_weak: element fluxes G grad u at the
//             points, transposed contractions to the local nodes, element
//             results summed per node in a fixed order), preconditioned by
//             Jacobi or a p-multigrid V-cycle (Chebyshev-Jacobi smoothing) in
//             FP64 or FP32, or as FP64 defect correction around an FP32 PCG;
//             optionally from the projection of the solution onto the previous
//             solutions;
//   w         d phi / dz = phi_t / z_t on the top layer's vertical GLL lines;
//   conditions the kinematic and dynamic conditions (Sec. 2) at the triangle
//             quadrature points, projected onto the nodal surface space with the
//             consistent mass, M k = int f l_i dA (Eq. free_surface_weak; the
//             mass solve by Jacobi-PCG on the assembled CSR matrix);
//   RK4       the classical stage states and combination, then the relaxation
//             zones and the modal filter (Sec. 3.3, Sec. 3.2) when set.
// Node and quadrature conventions are those of prism.cu (fnpf_prism_*).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "fnpf.h"

#if defined(__CUDACC__)
#define FNPF_HD __host__ __device__
#else
#define FNPF_HD
#endif

namespace fnpf {
namespace pstep {

constexpr int kChunk = 256;   // entries per partial sum of a dot product
constexpr int kMaxProj = 8;   // previous solutions in the projected initial guess (one more slot: the caller's guess)

// The mesh as the items read it (device pointers on the GPU).
struct PMesh {
  int p, n, nz, nt, nq, ntri;
  int64_t ns, nv, N, NI, nelem;
  const int* tn;                        // [ntri][nt] surface node of each local triangle node
  const double* geo;                    // [ntri][4] x_r, x_s, y_r, y_s
  const double *L, *Lr, *Ls;            // [nq][nt] nodal basis and its r, s derivatives
  const double* wq;                     // [nq] triangle quadrature weights
  const double *xi, *wv, *D;            // [n], [n], [n][n] GLL nodes, weights, D[k][m] = l'_m(xi_k)
  const int64_t *voff, *vinc;           // volume node g: element results vinc[voff[g] .. voff[g+1])
  const int64_t *soff, *sinc;           // surface node c: (triangle, local node) slots t nt + c'
  const int64_t* mrow;                  // consistent surface mass, CSR [ns + 1]
  const int* mcol;
  const double* mval;
  const double* mdiag;                  // [ns] its diagonal
  const double* filt;                   // [nt][nt] modal filter V F V^-1 on the triangle nodes (null: none)
  const int* interior;                  // [nt] 1 for the triangle-interior local nodes
  const double *rcr, *rgen;             // [ns] relaxation weight C_r and generation flag (null: no zones)
  const double *xs, *ys;                // [ns] surface node coordinates (the incident wave's phase)
  double ramp, amp, kx, ky, omega, phase;   // incident wave of the generation zones
  const float *Lf, *Lrf, *Lsf, *Df;     // FP32 copies of L, Lr, Ls, D (levels of an FP32 V-cycle)
};

// The operator tables of a mesh view in the value type T of a computation.
template <class T>
struct Tabs {
  const T *L, *Lr, *Ls, *D;
};
FNPF_HD inline Tabs<double> tabs_of(const PMesh& m, const double*) { return {m.L, m.Lr, m.Ls, m.D}; }
FNPF_HD inline Tabs<float> tabs_of(const PMesh& m, const float*) { return {m.Lf, m.Lrf, m.Lsf, m.Df}; }

// Points the table pointers of m into the packed tables of fnpf_prism_create:
// geo [4 ntri], L, Lr, Ls [nq nt], wq [nq], xi [n], wv [n], D [n n].
inline void bind_tables(PMesh* m, const double* tab) {
  m->geo = tab;
  m->L = m->geo + 4 * (int64_t)m->ntri;
  m->Lr = m->L + (int64_t)m->nq * m->nt;
  m->Ls = m->Lr + (int64_t)m->nq * m->nt;
  m->wq = m->Ls + (int64_t)m->nq * m->nt;
  m->xi = m->wq + m->nq;
  m->wv = m->xi + m->n;
  m->D = m->wv + m->n;
}

// Workspace of the path.
struct PWork {
  double *G, *F, *ye, *diag;            // [nelem n nq 6], [nelem n nq 3], [nelem nt n], [N]
  double* vt;                           // [nelem n nt] vertical derivatives, then vertical sums
  double *xs, *r, *z, *pd, *q;          // Laplace PCG [N]
  double *part, *scal;                  // dot-product partials, scalars
  double* cg;                           // CG state on the device (kCgSlots) and Lanczos coefficients
  double *phi, *w;                      // the mesh's potential [N] (warm start), w [ns]
  double *fq, *se, *be, *bp;            // [ntri nq 2], [ntri nt 2], [ns], [ns]
  double *mr, *mz, *mp, *mq;            // surface-mass CG [ns]
  double *ke, *kp, *es, *ps, *ae, *ap;  // RK4 stage right-hand side, stage state, accumulator [ns]
  double* zero;                         // [ns] zeros (still-water geometry of the linear model)
  double* ft;                           // [ntri nt] filtered interior values
  double *H, *AH;                       // [kMaxProj + 1][N] projection basis and its images under A
  double* gram;                         // [(kMaxProj + 1) (kMaxProj + 2)] Gram matrix and right-hand side
  int hist_n = 0, hist_next = 0;        // stored solutions, next slot (host state)
  float *ie, *ir, *iz, *ip, *iq;        // [N] the FP32 inner solve of the defect correction
  double *aN, *aS, *aq, *se3;           // adjoint: [5][N], [32][ns], [ntri nq 6], [ntri nt 3]
};

inline int64_t dot_partials(int64_t n) { return (n + kChunk - 1) / kChunk; }

// Carves the workspace: take(&ptr, count) is called for every buffer in a
// fixed order (the caller allocates, or only counts).
template <class Take>
void carve(const PMesh& m, PWork* w, Take take) {
  const int64_t pts = m.nelem * m.n * m.nq;
  take(&w->G, pts * 6);
  take(&w->F, pts * 3);
  take(&w->ye, m.nelem * m.nt * m.n);
  take(&w->vt, m.nelem * m.nt * m.n);
  take(&w->diag, m.N);
  take(&w->xs, m.N);
  take(&w->r, m.N);
  take(&w->z, m.N);
  take(&w->pd, m.N);
  take(&w->q, m.N);
  take(&w->part, dot_partials(std::max<int64_t>(m.N, m.ns)));
  take(&w->scal, 4);
  take(&w->cg, 64);
  take(&w->phi, m.N);
  take(&w->w, m.ns);
  take(&w->fq, (int64_t)m.ntri * m.nq * 2);
  take(&w->se, (int64_t)m.ntri * m.nt * 2);
  double** surf[] = {&w->be, &w->bp, &w->mr, &w->mz, &w->mp, &w->mq, &w->ke,
                     &w->kp, &w->es, &w->ps, &w->ae, &w->ap, &w->zero};
  for (double** s : surf) take(s, m.ns);
  take(&w->ft, (int64_t)m.ntri * m.nt);
  take(&w->H, (int64_t)(kMaxProj + 1) * m.N);
  take(&w->AH, (int64_t)(kMaxProj + 1) * m.N);
  take(&w->gram, (kMaxProj + 1) * (kMaxProj + 2));
  take(&w->aN, 5 * m.N);
  take(&w->aS, 32 * m.ns);
  take(&w->aq, (int64_t)m.ntri * m.nq * 6);
  take(&w->se3, (int64_t)m.ntri * m.nt * 3);
  float** inner[] = {&w->ie, &w->ir, &w->iz, &w->ip, &w->iq};
  for (float** f : inner) {   // a float buffer of N entries takes (N + 1) / 2 doubles
    double* d = nullptr;
    take(&d, (m.N + 1) / 2);
    *f = reinterpret_cast<float*>(d);
  }
}

// CG state slots (device doubles): r.z, p.q, r.r, alpha, beta, the new r.z,
// the stop flag (0 running, 1 converged, 2 breakdown, 3 diverged) and the
// number of completed iterations; the Lanczos coefficients follow.
enum { kRZ = 0, kPQ, kRR, kAL, kBE, kRZN, kDONE, kITERS, kCgSlots };
constexpr int kMaxLanczos = 12;   // steps of the eigenvalue estimate (coefficients at cg + kCgSlots)

// ---------------------------------------------------------------------------
// Host set-up: the surface incidence and the consistent surface mass.

// Surface node c -> its (triangle, local node) slots t nt + c', in slot order.
inline void surface_incidence(const int* tn, int ntri, int nt, int64_t ns, std::vector<int64_t>* off,
                              std::vector<int64_t>* inc) {
  off->assign(ns + 1, 0);
  for (int64_t s = 0; s < (int64_t)ntri * nt; ++s) ++(*off)[tn[s] + 1];
  for (int64_t c = 0; c < ns; ++c) (*off)[c + 1] += (*off)[c];
  inc->assign((size_t)ntri * nt, 0);
  std::vector<int64_t> fill(off->begin(), off->end() - 1);
  for (int64_t s = 0; s < (int64_t)ntri * nt; ++s) (*inc)[fill[tn[s]]++] = s;
}

// M_ij = int l_i l_j dA (the triangle rule, exact for the degree-2p products),
// assembled row by row with the columns ascending; equal columns summed in
// triangle order.
inline void surface_mass(const PMesh& m, const int* tn, const double* geo, const double* L, const double* wq,
                         std::vector<int64_t>* row, std::vector<int>* col, std::vector<double>* val,
                         std::vector<double>* diag) {
  const int nt = m.nt, nq = m.nq;
  std::vector<std::vector<std::pair<int, double>>> rows(m.ns);
  std::vector<double> Me((size_t)nt * nt);
  for (int t = 0; t < m.ntri; ++t) {
    const double* gt = geo + 4 * (int64_t)t;
    const double det = fabs(gt[0] * gt[3] - gt[1] * gt[2]);
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b) {
        double s = 0;
        for (int q = 0; q < nq; ++q) s += wq[q] * L[(int64_t)q * nt + a] * L[(int64_t)q * nt + b];
        Me[(size_t)a * nt + b] = s * det;
      }
    const int* tt = tn + (int64_t)t * nt;
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b) rows[tt[a]].push_back({tt[b], Me[(size_t)a * nt + b]});
  }
  row->assign(m.ns + 1, 0);
  col->clear();
  val->clear();
  diag->assign(m.ns, 0.0);
  for (int64_t i = 0; i < m.ns; ++i) {
    auto& r = rows[i];
    std::stable_sort(r.begin(), r.end(), [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
      return x.first < y.first;
    });
    for (size_t j = 0; j < r.size();) {
      const int c = r[j].first;
      double s = 0;
      for (; j < r.size() && r[j].first == c; ++j) s += r[j].second;
      col->push_back(c);
      val->push_back(s);
      if (c == i) (*diag)[i] = s;
    }
    (*row)[i + 1] = (int64_t)col->size();
  }
}

// The modal filter of the paper's triangular surface elements (Sec. 3.2): the
// element's nodal values are mapped to the coefficients of a modal basis,
// mode (i, j) is scaled by sigma_(i+j), and the result is mapped back:
// F = V diag(sigma) V^-1 with V[r][c] = psi_c(node r).  psi_(i, j) is the
// orthonormal Dubiner basis on R = {r, s >= -1, r + s <= 0} (Dubiner 1991;
// Sherwin & Karniadakis):
//   psi_(i, j)(r, s) = sqrt(2) Q_i^(0,0)(a) Q_j^(2i+1,0)(s) (1 - s)^i,
//   a = 2 (1 + r) / (1 - s) - 1,
// Q_n^(al,be) the Jacobi polynomial normalised to unit L2 norm under the weight
// (1 - x)^al (1 + x)^be; sigma_d = 1 for d <= cutoff, else
// exp(-alpha ((d - cutoff) / (p - cutoff))^order).  Local node order (i, j),
// j outer (the numbering of prism.cu); interior[c] = 1 for i, j > 0, i + j < p.

// P_n^(al,be)(x) by the three-term recurrence in n.
inline long double jacobi(int n, int al, int be, long double x) {
  long double p0 = 1, p1 = 0.5L * ((al + be + 2) * x + (al - be));
  if (n == 0) return p0;
  for (int k = 1; k < n; ++k) {
    const long double c = 2 * k + al + be;
    const long double a1 = 2 * (k + 1) * (k + al + be + 1) * c;
    const long double a2 = (c + 1) * (al * al - be * be);
    const long double a3 = c * (c + 1) * (c + 2);
    const long double a4 = 2 * (k + al) * (k + be) * (c + 2);
    const long double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// || P_n^(al,be) || under its weight on [-1, 1].
inline long double jacobi_norm(int n, int al, int be) {
  const long double v = powl(2.0L, al + be + 1) / (2 * n + al + be + 1) * tgammal(n + al + 1.0L) *
                        tgammal(n + be + 1.0L) / (tgammal(n + al + be + 1.0L) * tgammal(n + 1.0L));
  return sqrtl(v);
}

inline long double dubiner(int i, int j, long double r, long double s) {
  const long double a = 1 - s > 1e-15L ? 2 * (1 + r) / (1 - s) - 1 : -1.0L;
  return sqrtl(2.0L) * jacobi(i, 0, 0, a) / jacobi_norm(i, 0, 0) * jacobi(j, 2 * i + 1, 0, s) /
         jacobi_norm(j, 2 * i + 1, 0) * powl(1 - s, i);
}

// F [nt][nt] and interior [nt] for order p, the triangle nodes (rn, sn); false
// if V is singular.
inline bool triangle_filter(int p, const double* rn, const double* sn, double alpha, int order, int cutoff,
                            std::vector<double>* F, std::vector<int>* interior) {
  std::vector<std::pair<int, int>> idx;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i + j <= p; ++i) idx.emplace_back(i, j);
  const int nt = (int)idx.size();
  std::vector<long double> V((size_t)nt * nt), Vi((size_t)nt * nt, 0.0L);
  for (int r = 0; r < nt; ++r)
    for (int c = 0; c < nt; ++c) V[(size_t)r * nt + c] = dubiner(idx[c].first, idx[c].second, rn[r], sn[r]);
  // V^-1 by Gauss-Jordan elimination with partial pivoting
  std::vector<long double> A = V;
  for (int i = 0; i < nt; ++i) Vi[(size_t)i * nt + i] = 1;
  for (int c = 0; c < nt; ++c) {
    int piv = c;
    for (int r = c + 1; r < nt; ++r)
      if (fabsl(A[(size_t)r * nt + c]) > fabsl(A[(size_t)piv * nt + c])) piv = r;
    if (fabsl(A[(size_t)piv * nt + c]) < 1e-300L) return false;
    for (int k = 0; k < nt; ++k) {
      std::swap(A[(size_t)c * nt + k], A[(size_t)piv * nt + k]);
      std::swap(Vi[(size_t)c * nt + k], Vi[(size_t)piv * nt + k]);
    }
    const long double d = A[(size_t)c * nt + c];
    for (int k = 0; k < nt; ++k) {
      A[(size_t)c * nt + k] /= d;
      Vi[(size_t)c * nt + k] /= d;
    }
    for (int r = 0; r < nt; ++r) {
      if (r == c) continue;
      const long double f = A[(size_t)r * nt + c];
      if (f == 0) continue;
      for (int k = 0; k < nt; ++k) {
        A[(size_t)r * nt + k] -= f * A[(size_t)c * nt + k];
        Vi[(size_t)r * nt + k] -= f * Vi[(size_t)c * nt + k];
      }
    }
  }
  std::vector<long double> sig(nt);
  for (int c = 0; c < nt; ++c) {
    const int d = idx[c].first + idx[c].second;
    sig[c] = d <= cutoff ? 1.0L : expl(-alpha * powl((long double)(d - cutoff) / (p - cutoff), order));
  }
  F->assign((size_t)nt * nt, 0.0);
  interior->assign(nt, 0);
  for (int r = 0; r < nt; ++r) {
    for (int c = 0; c < nt; ++c) {
      long double v = 0;
      for (int k = 0; k < nt; ++k) v += V[(size_t)r * nt + k] * sig[k] * Vi[(size_t)k * nt + c];
      (*F)[(size_t)r * nt + c] = (double)v;
    }
    const int i = idx[r].first, j = idx[r].second;
    (*interior)[r] = i > 0 && j > 0 && i + j < p;
  }
  return true;
}

// ---------------------------------------------------------------------------
// The p-multigrid hierarchy (host set-up).  Levels p = q_0 > q_1 > ... > 1,
// q_(l+1) = floor(q_l / 2): the same prisms at lower order, their operators
// rediscretised on the eta-following geometry (eta and h interpolated to each
// level).  The order-q spaces are nested (degree-q polynomials on the triangle
// times degree-q polynomials in the vertical), so prolongation is exact
// interpolation and restriction its transpose.

}  // namespace pstep

// Host functions of the library (prism.cu, mesh.cu).
void gll_tables(int p, double* xi, double* w, double* D);
bool prism_tables(int p, std::vector<double>* rn, std::vector<double>* sn, std::vector<double>* wq,
                  std::vector<double>* L, std::vector<double>* Lr, std::vector<double>* Ls);
bool prism_numbering(const double* verts, int nverts, const int* tris, int ntri, int p, std::vector<int>* tnodes,
                     std::vector<double>* xs, std::vector<double>* ys);

namespace pstep {

constexpr int kMaxLevels = 4;   // p <= 8: 8, 4, 2, 1

// Volume node g -> its element results (elem nt n + m nt + c), in (element,
// local node) order.
inline void volume_incidence(const int* tn, int ntri, int nt, int nz, int p, int64_t ns, std::vector<int64_t>* off,
                             std::vector<int64_t>* inc) {
  const int n = p + 1;
  const int64_t N = ((int64_t)nz * p + 1) * ns;
  off->assign(N + 1, 0);
  for (int t = 0; t < ntri; ++t)
    for (int l = 0; l < nz; ++l)
      for (int mm = 0; mm < n; ++mm)
        for (int q = 0; q < nt; ++q) ++(*off)[(int64_t)(l * p + mm) * ns + tn[(size_t)t * nt + q] + 1];
  for (int64_t g = 0; g < N; ++g) (*off)[g + 1] += (*off)[g];
  inc->assign((*off)[N], 0);
  std::vector<int64_t> fill(off->begin(), off->end() - 1);
  for (int t = 0; t < ntri; ++t)
    for (int l = 0; l < nz; ++l)
      for (int mm = 0; mm < n; ++mm)
        for (int q = 0; q < nt; ++q) {
          const int64_t g = (int64_t)(l * p + mm) * ns + tn[(size_t)t * nt + q];
          (*inc)[fill[g]++] = ((int64_t)t * nz + l) * nt * n + (int64_t)mm * nt + q;
        }
}

// Host data of one level: numbering, packed tables (the layout of bind_tables),
// volume and surface incidences, triangle node coordinates.
struct LevelHost {
  int q = 0, nt = 0, nq = 0;
  int64_t ns = 0;
  std::vector<int> tn;
  std::vector<double> tab, rn, sn;
  std::vector<int64_t> voff, vinc, soff, sinc;
};

inline bool build_level(const double* verts, int nverts, const int* tris, int ntri, int q, int nz, LevelHost* L) {
  std::vector<double> xs, ys, wq, Lq, Lr, Ls;
  if (!prism_numbering(verts, nverts, tris, ntri, q, &L->tn, &xs, &ys)) return false;
  if (!prism_tables(q, &L->rn, &L->sn, &wq, &Lq, &Lr, &Ls)) return false;
  L->q = q;
  L->nt = (int)L->rn.size();
  L->nq = (int)wq.size();
  L->ns = (int64_t)xs.size();
  const int n = q + 1;
  std::vector<double> xi(n), wv(n), D(n * n);
  gll_tables(q, xi.data(), wv.data(), D.data());
  L->tab.clear();
  for (int t = 0; t < ntri; ++t) {
    const int A = tris[3 * t], B = tris[3 * t + 1], C = tris[3 * t + 2];
    L->tab.push_back(0.5 * (verts[2 * B] - verts[2 * A]));
    L->tab.push_back(0.5 * (verts[2 * C] - verts[2 * A]));
    L->tab.push_back(0.5 * (verts[2 * B + 1] - verts[2 * A + 1]));
    L->tab.push_back(0.5 * (verts[2 * C + 1] - verts[2 * A + 1]));
  }
  for (const std::vector<double>* v : {&Lq, &Lr, &Ls, &wq, &xi, &wv, &D}) L->tab.insert(L->tab.end(), v->begin(), v->end());
  volume_incidence(L->tn.data(), ntri, L->nt, nz, q, L->ns, &L->voff, &L->vinc);
  surface_incidence(L->tn.data(), ntri, L->nt, L->ns, &L->soff, &L->sinc);
  return true;
}

// Values [npts][nt] of the order-q nodal basis (nodes rn, sn) at the points
// (r, s): the Dubiner basis at the points times the inverse of its values at
// the nodes (both span the degree-q polynomials).
inline bool nodal_basis_at(int q, const std::vector<double>& rn, const std::vector<double>& sn, int npts,
                           const double* r, const double* s, std::vector<double>* out) {
  std::vector<std::pair<int, int>> idx;
  for (int j = 0; j <= q; ++j)
    for (int i = 0; i + j <= q; ++i) idx.emplace_back(i, j);
  const int nt = (int)idx.size();
  std::vector<long double> A((size_t)nt * nt), Vi((size_t)nt * nt, 0.0L);
  for (int a = 0; a < nt; ++a)
    for (int k = 0; k < nt; ++k) A[(size_t)a * nt + k] = dubiner(idx[k].first, idx[k].second, rn[a], sn[a]);
  for (int i = 0; i < nt; ++i) Vi[(size_t)i * nt + i] = 1;
  for (int c = 0; c < nt; ++c) {   // Gauss-Jordan with partial pivoting
    int piv = c;
    for (int r2 = c + 1; r2 < nt; ++r2)
      if (fabsl(A[(size_t)r2 * nt + c]) > fabsl(A[(size_t)piv * nt + c])) piv = r2;
    if (fabsl(A[(size_t)piv * nt + c]) < 1e-300L) return false;
    for (int k = 0; k < nt; ++k) {
      std::swap(A[(size_t)c * nt + k], A[(size_t)piv * nt + k]);
      std::swap(Vi[(size_t)c * nt + k], Vi[(size_t)piv * nt + k]);
    }
    const long double d = A[(size_t)c * nt + c];
    for (int k = 0; k < nt; ++k) {
      A[(size_t)c * nt + k] /= d;
      Vi[(size_t)c * nt + k] /= d;
    }
    for (int r2 = 0; r2 < nt; ++r2) {
      if (r2 == c) continue;
      const long double f = A[(size_t)r2 * nt + c];
      if (f == 0) continue;
      for (int k = 0; k < nt; ++k) {
        A[(size_t)r2 * nt + k] -= f * A[(size_t)c * nt + k];
        Vi[(size_t)r2 * nt + k] -= f * Vi[(size_t)c * nt + k];
      }
    }
  }
  // A psi-values matrix V[a][k] = psi_k(node a); l_c(x) = sum_k psi_k(x) (V^-1)[k][c]
  out->assign((size_t)npts * nt, 0.0);
  std::vector<long double> ps(nt);
  for (int i = 0; i < npts; ++i) {
    for (int k = 0; k < nt; ++k) ps[k] = dubiner(idx[k].first, idx[k].second, r[i], s[i]);
    for (int c = 0; c < nt; ++c) {
      long double v = 0;
      for (int k = 0; k < nt; ++k) v += ps[k] * Vi[(size_t)k * nt + c];
      (*out)[(size_t)i * nt + c] = (double)v;
    }
  }
  return true;
}

// Transfer tables between a fine level f and the next coarser level c:
// Ptri [nt_f][nt_c] (coarse nodal basis at the fine triangle nodes), Pv
// [n_f][n_c] (coarse GLL Lagrange basis at the fine GLL nodes), Etri
// [nt_c][nt_f] (fine nodal basis at the coarse triangle nodes).
inline bool transfer_tables(const LevelHost& f, const LevelHost& c, std::vector<double>* Ptri, std::vector<double>* Pv,
                            std::vector<double>* Etri) {
  if (!nodal_basis_at(c.q, c.rn, c.sn, f.nt, f.rn.data(), f.sn.data(), Ptri)) return false;
  if (!nodal_basis_at(f.q, f.rn, f.sn, c.nt, c.rn.data(), c.sn.data(), Etri)) return false;
  const int nf = f.q + 1, nc = c.q + 1;
  std::vector<double> xf(nf), xc(nc), w(std::max(nf, nc)), D((size_t)std::max(nf, nc) * std::max(nf, nc));
  gll_tables(f.q, xf.data(), w.data(), D.data());
  gll_tables(c.q, xc.data(), w.data(), D.data());
  Pv->assign((size_t)nf * nc, 0.0);
  for (int i = 0; i < nf; ++i)
    for (int j = 0; j < nc; ++j) {
      long double v = 1;
      for (int k = 0; k < nc; ++k)
        if (k != j) v *= ((long double)xf[i] - xc[k]) / ((long double)xc[j] - xc[k]);
      (*Pv)[(size_t)i * nc + j] = (double)v;
    }
  return true;
}

// ---------------------------------------------------------------------------
// Items.

// Prism point (elem, k, q) of item i over nelem n nq; elem = triangle nz + layer.
struct PointIdx {
  int64_t elem;
  int e, l, k, q;
};
FNPF_HD inline PointIdx point_of(const PMesh& m, int64_t i) {
  PointIdx r;
  const int64_t per = (int64_t)m.n * m.nq;
  r.elem = i / per;
  const int pt = (int)(i - r.elem * per);
  r.k = pt / m.nq;
  r.q = pt - r.k * m.nq;
  r.e = (int)(r.elem / m.nz);
  r.l = (int)(r.elem - (int64_t)r.e * m.nz);
  return r;
}

// G = w_q w_k |det J| J^-1 J^-T (6 entries: 00 01 02 11 12 22) at every point;
// J = [[x_r, x_s, 0], [y_r, y_s, 0], [z_r, z_s, z_t]] with z from eta and h in
// the triangle's nodal basis.
struct GeomItem {
  struct Args {
    PMesh m;
    const double *eta, *h;
    double* G;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const PointIdx pi = point_of(m, i);
    const int nt = m.nt;
    const int* tn = m.tn + (int64_t)pi.e * nt;
    const double* Lq = m.L + (int64_t)pi.q * nt;
    const double* Lrq = m.Lr + (int64_t)pi.q * nt;
    const double* Lsq = m.Ls + (int64_t)pi.q * nt;
    double ev = 0, er = 0, es = 0, hv = 0, hr = 0, hs = 0;
    for (int c = 0; c < nt; ++c) {
      const double E = a.eta[tn[c]], H = a.h[tn[c]];
      ev += Lq[c] * E;
      er += Lrq[c] * E;
      es += Lsq[c] * E;
      hv += Lq[c] * H;
      hr += Lrq[c] * H;
      hs += Lsq[c] * H;
    }
    const double* gt = m.geo + 4 * (int64_t)pi.e;
    const double xr = gt[0], xs = gt[1], yr = gt[2], ys = gt[3];
    const double det2 = xr * ys - xs * yr;
    const double sig = (pi.l + 0.5 * (1.0 + m.xi[pi.k])) / m.nz;
    const double zr = -hr + sig * (er + hr), zs = -hs + sig * (es + hs), zt = (ev + hv) / (2.0 * m.nz);
    const double det = det2 * zt;
    // J^-1 by cofactors; its third column is (0, 0, det2 / det)
    const double i00 = ys * zt / det, i01 = -xs * zt / det;
    const double i10 = -yr * zt / det, i11 = xr * zt / det;
    const double i20 = (yr * zs - ys * zr) / det, i21 = (xs * zr - xr * zs) / det, i22 = det2 / det;
    const double wt = m.wq[pi.q] * m.wv[pi.k] * fabs(det);
    double* G = a.G + 6 * i;
    G[0] = wt * (i00 * i00 + i01 * i01);
    G[1] = wt * (i00 * i10 + i01 * i11);
    G[2] = wt * (i00 * i20 + i01 * i21);
    G[3] = wt * (i10 * i10 + i11 * i11);
    G[4] = wt * (i10 * i20 + i11 * i21);
    G[5] = wt * (i20 * i20 + i21 * i21 + i22 * i22);
  }
};

// d u / d t at element node (elem, k, c) of item i over nelem n nt (slot
// k nt + c): the vertical GLL derivative along the node's line.
template <class T>
struct DtItemT {
  struct Args {
    PMesh m;
    const T* x;
    T* ut;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const Tabs<T> tb = tabs_of(m, (const T*)nullptr);
    const int64_t per = (int64_t)m.nt * m.n;
    const int64_t elem = i / per;
    const int idx = (int)(i - elem * per);
    const int c = idx % m.nt, k = idx / m.nt;
    const int e = (int)(elem / m.nz), l = (int)(elem - (int64_t)e * m.nz);
    const int64_t col = m.tn[(int64_t)e * m.nt + c];
    const T* Dk = tb.D + (int64_t)k * m.n;
    const int64_t plane0 = (int64_t)l * m.p;
    T s = 0;
    for (int mm = 0; mm < m.n; ++mm) s += Dk[mm] * a.x[(plane0 + mm) * m.ns + col];
    a.ut[i] = s;
  }
};
using DtItem = DtItemT<double>;

// Flux G grad_ref u at every point (u the volume field x, ut its vertical
// derivatives at the element nodes from DtItem).
template <class T>
struct FluxItemT {
  struct Args {
    PMesh m;
    const T* G;
    const T* x;
    const T* ut;
    T* F;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const Tabs<T> tb = tabs_of(m, (const T*)nullptr);
    const PointIdx pi = point_of(m, i);
    const int nt = m.nt, n = m.n;
    const int* tn = m.tn + (int64_t)pi.e * nt;
    const T* Lq = tb.L + (int64_t)pi.q * nt;
    const T* Lrq = tb.Lr + (int64_t)pi.q * nt;
    const T* Lsq = tb.Ls + (int64_t)pi.q * nt;
    const T* xk = a.x + ((int64_t)pi.l * m.p + pi.k) * m.ns;
    const T* utk = a.ut + (pi.elem * n + pi.k) * nt;
    T ur = 0, us = 0, ut = 0;
    for (int c = 0; c < nt; ++c) {
      const T u = xk[tn[c]];
      ur += Lrq[c] * u;
      us += Lsq[c] * u;
      ut += Lq[c] * utk[c];
    }
    const T* G = a.G + 6 * i;
    T* F = a.F + 3 * i;
    F[0] = G[0] * ur + G[1] * us + G[2] * ut;
    F[1] = G[1] * ur + G[3] * us + G[4] * ut;
    F[2] = G[2] * ur + G[4] * us + G[5] * ut;
  }
};
using FluxItem = FluxItemT<double>;

// Local node (elem, mm, c) of item i over nelem nt n; slot = mm nt + c.
struct NodeIdx {
  int64_t elem, base;   // base: the element's first point
  int mm, c;
};
FNPF_HD inline NodeIdx node_of(const PMesh& m, int64_t i) {
  NodeIdx r;
  const int64_t per = (int64_t)m.nt * m.n;
  r.elem = i / per;
  const int idx = (int)(i - r.elem * per);
  r.c = idx % m.nt;
  r.mm = idx / m.nt;
  r.base = r.elem * m.n * m.nq;
  return r;
}

// Element result at local node (c, mm): the transposed contractions of the
// fluxes with the basis gradients, sum over the points (q, k) of
// (delta_k,mm L_r[q][c], delta_k,mm L_s[q][c], L[q][c] D[k][mm]) . F(q, k).
template <class T>
struct NodeItemT {
  struct Args {
    PMesh m;
    const T* F;
    const T* vs;   // [nelem n nt] from TSumItem
    T* ye;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const Tabs<T> tb = tabs_of(m, (const T*)nullptr);
    const NodeIdx ni = node_of(m, i);
    const int nt = m.nt, nq = m.nq, n = m.n;
    const T* Fm = a.F + 3 * (ni.base + (int64_t)ni.mm * nq);
    T y = 0;
    for (int q = 0; q < nq; ++q) y += tb.Lr[(int64_t)q * nt + ni.c] * Fm[3 * q] + tb.Ls[(int64_t)q * nt + ni.c] * Fm[3 * q + 1];
    const T* vs = a.vs + ni.elem * n * nt + ni.c;
    for (int k = 0; k < n; ++k) y += tb.D[(int64_t)k * n + ni.mm] * vs[(int64_t)k * nt];
    a.ye[i] = y;
  }
};
using NodeItem = NodeItemT<double>;

// The vertical flux contracted over the triangle points, at (elem, k, c) of
// item i over nelem n nt (slot k nt + c): sum over q of L[q][c] F_t(k, q) (the
// part of NodeItem's transposed contraction shared by the n nodes of a line).
template <class T>
struct TSumItemT {
  struct Args {
    PMesh m;
    const T* F;
    T* vs;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const Tabs<T> tb = tabs_of(m, (const T*)nullptr);
    const int64_t per = (int64_t)m.nt * m.n;
    const int64_t elem = i / per;
    const int idx = (int)(i - elem * per);
    const int c = idx % m.nt, k = idx / m.nt;
    const T* Fk = a.F + 3 * (elem * m.n * m.nq + (int64_t)k * m.nq);
    T s = 0;
    for (int q = 0; q < m.nq; ++q) s += tb.L[(int64_t)q * m.nt + c] * Fk[3 * q + 2];
    a.vs[i] = s;
  }
};
using TSumItem = TSumItemT<double>;

// The element results of A x for one prism per block, staged in shared memory:
// the block's phases run in order with a barrier after each (a phase writes
// only shared or output entries that no other thread of the same phase reads
// or writes), every thread of the block taking the entries tid, tid + threads,
// ... of each phase.  Phase 0 loads the element's values u [n][nt], 1 forms
// the vertical derivatives ut [n][nt], 2 the fluxes F [n nq][3] at the points
// (the metric read from G), 3 the vertical sums vs [n][nt], 4 the node results
// ye -- the arithmetic of DtItem, FluxItem, TSumItem and NodeItem in the same
// order, with each value loaded from global memory once per element.  Shared
// memory: smem_entries(m) values of T.
template <class T>
struct ElementBlock {
  using value_type = T;
  static constexpr int kThreads = 128;
  static constexpr int kPhases = 5;
  struct Args {
    PMesh m;
    const T* G;
    const T* x;
    T* ye;
  };
  FNPF_HD static int64_t smem_entries(const PMesh& m) { return 3 * (int64_t)m.nt * m.n + 3 * (int64_t)m.n * m.nq; }
  FNPF_HD static void phase(int ph, int64_t elem, int tid, int nthr, T* sm, const Args& a) {
    const PMesh& m = a.m;
    const Tabs<T> tb = tabs_of(m, (const T*)nullptr);
    const int nt = m.nt, n = m.n, nq = m.nq, ntn = nt * n, npt = n * nq;
    T* u = sm;
    T* ut = u + ntn;
    T* vs = ut + ntn;
    T* F = vs + ntn;
    const int e = (int)(elem / m.nz), l = (int)(elem - (int64_t)e * m.nz);
    const int* tn = m.tn + (int64_t)e * nt;
    if (ph == 0) {
      for (int idx = tid; idx < ntn; idx += nthr) {
        const int c = idx % nt, mm = idx / nt;
        u[idx] = a.x[((int64_t)l * m.p + mm) * m.ns + tn[c]];
      }
    } else if (ph == 1) {
      for (int idx = tid; idx < ntn; idx += nthr) {
        const int c = idx % nt, k = idx / nt;
        const T* Dk = tb.D + (int64_t)k * n;
        T s = 0;
        for (int mm = 0; mm < n; ++mm) s += Dk[mm] * u[mm * nt + c];
        ut[idx] = s;
      }
    } else if (ph == 2) {
      for (int pt = tid; pt < npt; pt += nthr) {
        const int k = pt / nq, q = pt - k * nq;
        const T* Lq = tb.L + (int64_t)q * nt;
        const T* Lrq = tb.Lr + (int64_t)q * nt;
        const T* Lsq = tb.Ls + (int64_t)q * nt;
        const T* uk = u + k * nt;
        const T* utk = ut + k * nt;
        T ur = 0, us = 0, uz = 0;
        for (int c = 0; c < nt; ++c) {
          ur += Lrq[c] * uk[c];
          us += Lsq[c] * uk[c];
          uz += Lq[c] * utk[c];
        }
        const T* G = a.G + 6 * (elem * npt + pt);
        F[3 * pt] = G[0] * ur + G[1] * us + G[2] * uz;
        F[3 * pt + 1] = G[1] * ur + G[3] * us + G[4] * uz;
        F[3 * pt + 2] = G[2] * ur + G[4] * us + G[5] * uz;
      }
    } else if (ph == 3) {
      for (int idx = tid; idx < ntn; idx += nthr) {
        const int c = idx % nt, k = idx / nt;
        const T* Fk = F + 3 * (k * nq);
        T s = 0;
        for (int q = 0; q < nq; ++q) s += tb.L[(int64_t)q * nt + c] * Fk[3 * q + 2];
        vs[idx] = s;
      }
    } else {
      for (int idx = tid; idx < ntn; idx += nthr) {
        const int c = idx % nt, mm = idx / nt;
        const T* Fm = F + 3 * (mm * nq);
        T y = 0;
        for (int q = 0; q < nq; ++q) y += tb.Lr[(int64_t)q * nt + c] * Fm[3 * q] + tb.Ls[(int64_t)q * nt + c] * Fm[3 * q + 1];
        for (int k = 0; k < n; ++k) y += tb.D[(int64_t)k * n + mm] * vs[k * nt + c];
        a.ye[elem * ntn + idx] = y;
      }
    }
  }
};

// The derivatives of B = grad_ref psi^T G grad_ref phi (G = w |det J| J^-1 J^-T)
// with respect to the vertical row (z_r, z_s, z_t) of J at point (elem, k, q):
// with M = J^-1, u = M^T grad_ref psi, v = M^T grad_ref phi and
// d M = -M dJ M, d|det J| = |det J| tr(M dJ),
//   dB / dz_j = w |det J| (M[j][2] u.v - u_z (M v)_j - v_z (M u)_j)
// (the adjoint's geometric term, d(psi^T A(eta, h) phi) = sum of these times
// the variations of z_r, z_s, z_t).  psi and phi are volume fields.
struct GeomVjpItem {
  struct Args {
    PMesh m;
    const double *eta, *h, *psi, *phi;
    double* P;   // [points][3]
  };
  FNPF_HD static void ref_grad(const PMesh& m, const PointIdx& pi, const double* x, double* g) {
    const int nt = m.nt, n = m.n;
    const int* tn = m.tn + (int64_t)pi.e * nt;
    const double* Lq = m.L + (int64_t)pi.q * nt;
    const double* Lrq = m.Lr + (int64_t)pi.q * nt;
    const double* Lsq = m.Ls + (int64_t)pi.q * nt;
    const double* Dk = m.D + (int64_t)pi.k * n;
    const int64_t plane0 = (int64_t)pi.l * m.p;
    double gr = 0, gs = 0, gt = 0;
    for (int c = 0; c < nt; ++c) {
      const int64_t col = tn[c];
      const double u = x[(plane0 + pi.k) * m.ns + col];
      gr += Lrq[c] * u;
      gs += Lsq[c] * u;
      double uc = 0;
      for (int mm = 0; mm < n; ++mm) uc += Dk[mm] * x[(plane0 + mm) * m.ns + col];
      gt += Lq[c] * uc;
    }
    g[0] = gr;
    g[1] = gs;
    g[2] = gt;
  }
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const PointIdx pi = point_of(m, i);
    const int nt = m.nt;
    const int* tn = m.tn + (int64_t)pi.e * nt;
    const double* Lq = m.L + (int64_t)pi.q * nt;
    const double* Lrq = m.Lr + (int64_t)pi.q * nt;
    const double* Lsq = m.Ls + (int64_t)pi.q * nt;
    double ev = 0, er = 0, es = 0, hv = 0, hr = 0, hs = 0;
    for (int c = 0; c < nt; ++c) {
      const double E = a.eta[tn[c]], H = a.h[tn[c]];
      ev += Lq[c] * E;
      er += Lrq[c] * E;
      es += Lsq[c] * E;
      hv += Lq[c] * H;
      hr += Lrq[c] * H;
      hs += Lsq[c] * H;
    }
    const double* gt = m.geo + 4 * (int64_t)pi.e;
    const double xr = gt[0], xs = gt[1], yr = gt[2], ys = gt[3];
    const double det2 = xr * ys - xs * yr;
    const double sig = (pi.l + 0.5 * (1.0 + m.xi[pi.k])) / m.nz;
    const double zr = -hr + sig * (er + hr), zs = -hs + sig * (es + hs), zt = (ev + hv) / (2.0 * m.nz);
    const double det = det2 * zt;
    // M = J^-1 (its third column is (0, 0, det2 / det))
    const double M00 = ys * zt / det, M01 = -xs * zt / det;
    const double M10 = -yr * zt / det, M11 = xr * zt / det;
    const double M20 = (yr * zs - ys * zr) / det, M21 = (xs * zr - xr * zs) / det, M22 = det2 / det;
    double ga[3], gb[3];
    ref_grad(m, pi, a.psi, ga);
    ref_grad(m, pi, a.phi, gb);
    const double ux = M00 * ga[0] + M10 * ga[1] + M20 * ga[2], uy = M01 * ga[0] + M11 * ga[1] + M21 * ga[2],
                 uz = M22 * ga[2];
    const double vx = M00 * gb[0] + M10 * gb[1] + M20 * gb[2], vy = M01 * gb[0] + M11 * gb[1] + M21 * gb[2],
                 vz = M22 * gb[2];
    const double Mu0 = M00 * ux + M01 * uy, Mu1 = M10 * ux + M11 * uy, Mu2 = M20 * ux + M21 * uy + M22 * uz;
    const double Mv0 = M00 * vx + M01 * vy, Mv1 = M10 * vx + M11 * vy, Mv2 = M20 * vx + M21 * vy + M22 * vz;
    const double uv = ux * vx + uy * vy + uz * vz;
    const double wd = m.wq[pi.q] * m.wv[pi.k] * fabs(det);
    double* P = a.P + 3 * i;
    P[0] = wd * (-uz * Mv0 - vz * Mu0);             // M[0][2] = 0
    P[1] = wd * (-uz * Mv1 - vz * Mu1);             // M[1][2] = 0
    P[2] = wd * (M22 * uv - uz * Mv2 - vz * Mu2);
  }
};

// The geometric term at triangle slot (t, c): the point derivatives chained to
// eta and h at the triangle's node c, summed over the prisms of its column:
//   d / d eta_c: dz_r = sigma L_r[q][c], dz_s = sigma L_s[q][c], dz_t = L[q][c] / (2 N_z),
//   d / d h_c:   dz_r = (sigma - 1) L_r[q][c], dz_s = (sigma - 1) L_s[q][c], dz_t = L[q][c] / (2 N_z).
struct VjpTriItem {
  struct Args {
    PMesh m;
    const double* P;
    double* se;   // [ntri nt][2]: (eta, h)
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const int t = (int)(i / m.nt), c = (int)(i - (int64_t)t * m.nt);
    double ge = 0, gh = 0;
    for (int l = 0; l < m.nz; ++l) {
      const int64_t elem = (int64_t)t * m.nz + l;
      for (int k = 0; k < m.n; ++k) {
        const double sig = (l + 0.5 * (1.0 + m.xi[k])) / m.nz;
        const double* P = a.P + 3 * (elem * m.n * m.nq + (int64_t)k * m.nq);
        for (int q = 0; q < m.nq; ++q) {
          const double rs = P[3 * q] * m.Lr[(int64_t)q * m.nt + c] + P[3 * q + 1] * m.Ls[(int64_t)q * m.nt + c];
          const double tz = P[3 * q + 2] * m.L[(int64_t)q * m.nt + c] / (2.0 * m.nz);
          ge += sig * rs + tz;
          gh += (sig - 1.0) * rs + tz;
        }
      }
    }
    a.se[2 * i] = ge;
    a.se[2 * i + 1] = gh;
  }
};

// Element diagonal at local node (c, mm): sum over the points of g^T G g with g
// the reference gradient of that node's basis function.
struct DiagItem {
  struct Args {
    PMesh m;
    const double* G;
    double* ye;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const NodeIdx ni = node_of(m, i);
    const int nt = m.nt, nq = m.nq, n = m.n;
    double d = 0;
    for (int k = 0; k < n; ++k) {
      const double dkm = m.D[(int64_t)k * n + ni.mm];
      for (int q = 0; q < nq; ++q) {
        const double* G = a.G + 6 * (ni.base + (int64_t)k * nq + q);
        const double a0 = k == ni.mm ? m.Lr[(int64_t)q * nt + ni.c] : 0.0;
        const double a1 = k == ni.mm ? m.Ls[(int64_t)q * nt + ni.c] : 0.0;
        const double a2 = m.L[(int64_t)q * nt + ni.c] * dkm;
        d += a0 * (G[0] * a0 + G[1] * a1 + G[2] * a2) + a1 * (G[1] * a0 + G[3] * a1 + G[4] * a2) +
             a2 * (G[2] * a0 + G[4] * a1 + G[5] * a2);
      }
    }
    a.ye[i] = d;
  }
};

// y_g = sum of the element results of node g, in incidence order.
template <class T>
struct GatherItemT {
  struct Args {
    const int64_t *off, *inc;
    const T* ye;
    T* y;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    T s = 0;
    for (int64_t j = a.off[i]; j < a.off[i + 1]; ++j) s += a.ye[a.inc[j]];
    a.y[i] = s;
  }
};
using GatherItem = GatherItemT<double>;

// x = [0 (interior); phis (surface plane)] over N.
struct SurfaceOnlyItem {
  struct Args {
    int64_t NI;
    const double* phis;
    double* x;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.x[i] = i >= a.NI ? a.phis[i - a.NI] : 0.0; }
};

// out = [s src (interior); 0 (surface plane)] over N.
template <class T>
struct InteriorItemT {
  struct Args {
    int64_t NI;
    double s;
    const T* src;
    T* out;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.out[i] = i < a.NI ? (T)a.s * a.src[i] : (T)0; }
};
using InteriorItem = InteriorItemT<double>;

struct AxpyItem {   // y += s x
  struct Args {
    double s;
    const double* x;
    double* y;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.y[i] += a.s * a.x[i]; }
};

struct LinItem {   // out = x + s y
  struct Args {
    const double* x;
    double s;
    const double* y;
    double* out;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.out[i] = a.x[i] + a.s * a.y[i]; }
};

struct DivItem {   // out = x / d (the Jacobi preconditioner)
  struct Args {
    const double *x, *d;
    double* out;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.out[i] = a.x[i] / a.d[i]; }
};

template <class T>
struct CopyItemT {
  struct Args {
    const T* src;
    T* dst;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.dst[i] = a.src[i]; }
};
using CopyItem = CopyItemT<double>;

template <class T>
struct FillItemT {
  struct Args {
    double v;
    T* dst;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.dst[i] = (T)a.v; }
};
using FillItem = FillItemT<double>;

// out = (To) in: the precision changes at the FP32 V-cycle's entry and exit.
template <class To, class From>
struct CastItem {
  struct Args {
    const From* in;
    To* out;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.out[i] = (To)a.in[i]; }
};

// part[i] = sum of x_j y_j over the i-th chunk of kChunk entries (fixed order).
template <class T>
struct DotPartItemT {
  struct Args {
    const T *x, *y;
    int64_t n;
    double* part;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const int64_t lo = i * kChunk, hi = lo + kChunk < a.n ? lo + kChunk : a.n;
    double s = 0;   // FP64 accumulation for every vector type
    for (int64_t j = lo; j < hi; ++j) s += (double)a.x[j] * (double)a.y[j];
    a.part[i] = s;
  }
};
using DotPartItem = DotPartItemT<double>;

// out[0] = sum of the partials (one item).
struct SumItem {
  struct Args {
    const double* part;
    int64_t np;
    double* out;
  };
  FNPF_HD static void at(int64_t, const Args& a) {
    double s = 0;
    for (int64_t j = 0; j < a.np; ++j) s += a.part[j];
    a.out[0] = s;
  }
};

// y = M x, M in CSR (rows in order, the stored column order).
struct CsrItem {
  struct Args {
    const int64_t* row;
    const int* col;
    const double* val;
    const double* x;
    double* y;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    double s = 0;
    for (int64_t j = a.row[i]; j < a.row[i + 1]; ++j) s += a.val[j] * a.x[a.col[j]];
    a.y[i] = s;
  }
};

// Device-side CG scalars.  Every CG item returns at once once the stop flag
// cg[kDONE] is set, so iterations launched after convergence change nothing
// and the host may read the flag only every few iterations.  hist (or null)
// receives alpha_j at 2 j and beta_j at 2 j + 1 (the Lanczos coefficients).
struct CgResetItem {
  struct Args {
    double* cg;
  };
  FNPF_HD static void at(int64_t, const Args& a) {
    a.cg[kDONE] = 0.0;
    a.cg[kITERS] = 0.0;
  }
};

struct CgAlphaItem {   // alpha = r.z / p.q (p.q <= 0 or not finite: breakdown or divergence)
  struct Args {
    double *cg, *hist;
  };
  FNPF_HD static void at(int64_t, const Args& a) {
    double* cg = a.cg;
    if (cg[kDONE] != 0.0) return;
    const double pq = cg[kPQ];
    if (!(pq > 0.0)) {
      cg[kDONE] = pq - pq == 0.0 ? 2.0 : 3.0;
      return;
    }
    const double al = cg[kRZ] / pq;
    cg[kAL] = al;
    if (a.hist) a.hist[2 * (int64_t)cg[kITERS]] = al;
  }
};

template <class T>
struct CgUpdateItemT {
  struct Args {
    const double* cg;
    const T *p, *q;
    T *x, *r;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    if (a.cg[kDONE] != 0.0) return;
    const T al = (T)a.cg[kAL];
    if (a.x) a.x[i] += al * a.p[i];
    a.r[i] -= al * a.q[i];
  }
};
using CgUpdateItem = CgUpdateItemT<double>;

struct CgCheckItem {   // one more completed iteration; converged when ||r|| <= stop
  struct Args {
    double* cg;
    double stop;
  };
  FNPF_HD static void at(int64_t, const Args& a) {
    double* cg = a.cg;
    if (cg[kDONE] != 0.0) return;
    cg[kITERS] += 1.0;
    const double rr = cg[kRR];
    if (!(rr - rr == 0.0)) cg[kDONE] = 3.0;
    else if (sqrt(rr) <= a.stop) cg[kDONE] = 1.0;
  }
};

struct CgBetaItem {   // beta = r.z_new / r.z, r.z = r.z_new
  struct Args {
    double *cg, *hist;
  };
  FNPF_HD static void at(int64_t, const Args& a) {
    double* cg = a.cg;
    if (cg[kDONE] != 0.0) return;
    const double be = cg[kRZN] / cg[kRZ];
    cg[kBE] = be;
    cg[kRZ] = cg[kRZN];
    if (a.hist) a.hist[2 * ((int64_t)cg[kITERS] - 1) + 1] = be;
  }
};

template <class T>
struct CgDirItemT {
  struct Args {
    const double* cg;
    const T* z;
    T* p;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    if (a.cg[kDONE] != 0.0) return;
    a.p[i] = a.z[i] + (T)a.cg[kBE] * a.p[i];
  }
};
using CgDirItem = CgDirItemT<double>;

// w = d phi / dz at surface node c: (sum_j D[p][j] phi(plane N_v - 1 - p + j)) 2 N_z / (eta + h).
struct WItem {
  struct Args {
    PMesh m;
    const double *eta, *h, *phi;
    double* w;
  };
  FNPF_HD static void at(int64_t c, const Args& a) {
    const PMesh& m = a.m;
    const double* Dp = m.D + (int64_t)m.p * m.n;
    const int64_t top = m.nv - 1 - m.p;
    double s = 0;
    for (int j = 0; j < m.n; ++j) s += Dp[j] * a.phi[(top + j) * m.ns + c];
    a.w[c] = s * 2.0 * m.nz / (a.eta[c] + a.h[c]);
  }
};

// The conditions at triangle quadrature point (t, q), times the rule's weight
// and |det J_2|:
//   f_eta = -grad eta . grad phi_eta + w (1 + |grad eta|^2)
//   f_phi = -g eta - |grad phi_eta|^2 / 2 + w^2 (1 + |grad eta|^2) / 2
// (linear: f_eta = w, f_phi = -g eta); grad = J_2^-T grad_ref.
struct SurfQItem {
  struct Args {
    PMesh m;
    const double *eta, *phis, *w;
    double g;
    int linear;
    double* fq;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const int nt = m.nt;
    const int t = (int)(i / m.nq), q = (int)(i - (int64_t)t * m.nq);
    const int* tn = m.tn + (int64_t)t * nt;
    const double* Lq = m.L + (int64_t)q * nt;
    const double* Lrq = m.Lr + (int64_t)q * nt;
    const double* Lsq = m.Ls + (int64_t)q * nt;
    double ev = 0, er = 0, es = 0, pr = 0, ps = 0, wv = 0;
    for (int c = 0; c < nt; ++c) {
      const int64_t g = tn[c];
      const double E = a.eta[g], P = a.phis[g];
      ev += Lq[c] * E;
      er += Lrq[c] * E;
      es += Lsq[c] * E;
      pr += Lrq[c] * P;
      ps += Lsq[c] * P;
      wv += Lq[c] * a.w[g];
    }
    const double* gt = m.geo + 4 * (int64_t)t;
    const double xr = gt[0], xs = gt[1], yr = gt[2], ys = gt[3];
    const double det = xr * ys - xs * yr;
    double fe, fp;
    if (a.linear) {
      fe = wv;
      fp = -a.g * ev;
    } else {
      const double ex = (ys * er - yr * es) / det, ey = (xr * es - xs * er) / det;
      const double px = (ys * pr - yr * ps) / det, py = (xr * ps - xs * pr) / det;
      const double q2 = 1.0 + ex * ex + ey * ey;
      fe = -(ex * px + ey * py) + wv * q2;
      fp = -a.g * ev - 0.5 * (px * px + py * py) + 0.5 * wv * wv * q2;
    }
    const double wt = m.wq[q] * fabs(det);
    a.fq[2 * i] = wt * fe;
    a.fq[2 * i + 1] = wt * fp;
  }
};

// The vector-Jacobian product of the weighted conditions at point (t, q): with
// the cotangents nu_eta, nu_phi of the projected right-hand sides (nodal, the
// mass solves' solutions) interpolated to the point, the coefficients of the
// variations of (grad eta, grad phis, w, eta) there, times the rule's weight:
// A = wt (nu_eta d f_eta + nu_phi d f_phi), 6 entries (d grad eta [2],
// d grad phis [2], d w, d eta).
struct SurfQVjpItem {
  struct Args {
    PMesh m;
    const double *eta, *phis, *w, *ne, *np;
    double g;
    int linear;
    double* A;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const int nt = m.nt;
    const int t = (int)(i / m.nq), q = (int)(i - (int64_t)t * m.nq);
    const int* tn = m.tn + (int64_t)t * nt;
    const double* Lq = m.L + (int64_t)q * nt;
    const double* Lrq = m.Lr + (int64_t)q * nt;
    const double* Lsq = m.Ls + (int64_t)q * nt;
    double er = 0, es = 0, pr = 0, ps = 0, wv = 0, ne = 0, np = 0;
    for (int c = 0; c < nt; ++c) {
      const int64_t g = tn[c];
      er += Lrq[c] * a.eta[g];
      es += Lsq[c] * a.eta[g];
      pr += Lrq[c] * a.phis[g];
      ps += Lsq[c] * a.phis[g];
      wv += Lq[c] * a.w[g];
      ne += Lq[c] * a.ne[g];
      np += Lq[c] * a.np[g];
    }
    const double* gt = m.geo + 4 * (int64_t)t;
    const double xr = gt[0], xs = gt[1], yr = gt[2], ys = gt[3];
    const double det = xr * ys - xs * yr;
    const double wt = m.wq[q] * fabs(det);
    double* A = a.A + 6 * i;
    if (a.linear) {   // f_eta = w, f_phi = -g eta
      A[0] = A[1] = A[2] = A[3] = 0.0;
      A[4] = wt * ne;
      A[5] = wt * np * -a.g;
      return;
    }
    const double ex = (ys * er - yr * es) / det, ey = (xr * es - xs * er) / det;
    const double px = (ys * pr - yr * ps) / det, py = (xr * ps - xs * pr) / det;
    const double q2 = 1.0 + ex * ex + ey * ey;
    A[0] = wt * (ne * (-px + 2.0 * wv * ex) + np * wv * wv * ex);
    A[1] = wt * (ne * (-py + 2.0 * wv * ey) + np * wv * wv * ey);
    A[2] = wt * (ne * -ex + np * -px);
    A[3] = wt * (ne * -ey + np * -py);
    A[4] = wt * (ne * q2 + np * wv * q2);
    A[5] = wt * np * -a.g;
  }
};

// The point coefficients of SurfQVjpItem chained to triangle node c (grad =
// J_2^-T grad_ref): slots [ntri nt][3] = (d eta, d phis, d w).
struct SurfNodeVjpItem {
  struct Args {
    PMesh m;
    const double* A;
    double* se;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const int t = (int)(i / m.nt), c = (int)(i - (int64_t)t * m.nt);
    const double* gt = m.geo + 4 * (int64_t)t;
    const double xr = gt[0], xs = gt[1], yr = gt[2], ys = gt[3];
    const double det = xr * ys - xs * yr;
    double se = 0, sp = 0, sw = 0;
    for (int q = 0; q < m.nq; ++q) {
      const double l = m.L[(int64_t)q * m.nt + c], lr = m.Lr[(int64_t)q * m.nt + c], ls = m.Ls[(int64_t)q * m.nt + c];
      const double gx = (ys * lr - yr * ls) / det, gy = (xr * ls - xs * lr) / det;
      const double* A = a.A + 6 * ((int64_t)t * m.nq + q);
      se += A[0] * gx + A[1] * gy + A[5] * l;
      sp += A[2] * gx + A[3] * gy;
      sw += A[4] * l;
    }
    a.se[3 * i] = se;
    a.se[3 * i + 1] = sp;
    a.se[3 * i + 2] = sw;
  }
};

// Surface node c: its slots' three components summed in incidence order.
struct SurfGather3Item {
  struct Args {
    const int64_t *off, *inc;
    const double* se;
    double *o0, *o1, *o2;
  };
  FNPF_HD static void at(int64_t c, const Args& a) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int64_t j = a.off[c]; j < a.off[c + 1]; ++j) {
      s0 += a.se[3 * a.inc[j]];
      s1 += a.se[3 * a.inc[j] + 1];
      s2 += a.se[3 * a.inc[j] + 2];
    }
    a.o0[c] = s0;
    a.o1[c] = s1;
    a.o2[c] = s2;
  }
};

// The vector-Jacobian product of w = s sum_j D[p][j] phi(top + j), s = 2 N_z /
// (geo + h) at surface node c for the cotangent lw: lphi(top + j, c) =
// lw s D[p][j] (lphi [N], zero elsewhere), and -lw w / (geo + h) added to
// le (when le is not null: the geometry is eta) and to lh.
struct WVjpItem {
  struct Args {
    PMesh m;
    const double *geo, *h, *w, *lw;
    double *lphi, *le, *lh;
  };
  FNPF_HD static void at(int64_t c, const Args& a) {
    const PMesh& m = a.m;
    const double d = a.geo[c] + a.h[c];
    const double s = 2.0 * m.nz / d;
    const double* Dp = m.D + (int64_t)m.p * m.n;
    const int64_t top = m.nv - 1 - m.p;
    for (int j = 0; j < m.n; ++j) a.lphi[(top + j) * m.ns + c] = a.lw[c] * s * Dp[j];
    const double gw = -a.lw[c] * a.w[c] / d;
    if (a.le) a.le[c] += gw;
    a.lh[c] += gw;
  }
};

struct Lin2Item {   // out = a x + b y
  struct Args {
    double a;
    const double* x;
    double b;
    const double* y;
    double* out;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.out[i] = a.a * a.x[i] + a.b * a.y[i]; }
};

// Triangle slot (t, c): sum over the points of L[q][c] times the weighted conditions.
struct SurfNodeItem {
  struct Args {
    PMesh m;
    const double* fq;
    double* se;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const int t = (int)(i / m.nt), c = (int)(i - (int64_t)t * m.nt);
    const double* f = a.fq + 2 * (int64_t)t * m.nq;
    double se = 0, sp = 0;
    for (int q = 0; q < m.nq; ++q) {
      const double l = m.L[(int64_t)q * m.nt + c];
      se += l * f[2 * q];
      sp += l * f[2 * q + 1];
    }
    a.se[2 * i] = se;
    a.se[2 * i + 1] = sp;
  }
};

// Right-hand sides of the mass solves at surface node c: its slots summed in order.
struct SurfGatherItem {
  struct Args {
    const int64_t *off, *inc;
    const double* se;
    double *be, *bp;
  };
  FNPF_HD static void at(int64_t c, const Args& a) {
    double se = 0, sp = 0;
    for (int64_t j = a.off[c]; j < a.off[c + 1]; ++j) {
      se += a.se[2 * a.inc[j]];
      sp += a.se[2 * a.inc[j] + 1];
    }
    a.be[c] = se;
    a.bp[c] = sp;
  }
};

// Filtered value of triangle slot (t, c) for the interior local nodes: row c
// of F applied to the triangle's nodal values of f.
struct FilterItem {
  struct Args {
    PMesh m;
    const double* f;
    double* ft;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const int t = (int)(i / m.nt), c = (int)(i - (int64_t)t * m.nt);
    if (!m.interior[c]) return;
    const int* tn = m.tn + (int64_t)t * m.nt;
    const double* Fc = m.filt + (int64_t)c * m.nt;
    double s = 0;
    for (int k = 0; k < m.nt; ++k) s += Fc[k] * a.f[tn[k]];
    a.ft[i] = s;
  }
};

// f at the interior nodes = the filtered values (each interior node belongs to
// one triangle only).
struct FilterWriteItem {
  struct Args {
    PMesh m;
    const double* ft;
    double* f;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const int c = (int)(i % a.m.nt);
    if (a.m.interior[c]) a.f[a.m.tn[i]] = a.ft[i];
  }
};

// The p-multigrid items.  A level's mesh view is a PMesh of its own order.

struct PXfer {
  const double *Ptri, *Pv, *Etri;   // transfer_tables, fine level -> next coarser level
  const float *Ptri_f, *Pv_f;       // FP32 copies of Ptri and Pv
};
FNPF_HD inline const double* ptri_of(const PXfer& t, const double*) { return t.Ptri; }
FNPF_HD inline const float* ptri_of(const PXfer& t, const float*) { return t.Ptri_f; }
FNPF_HD inline const double* pv_of(const PXfer& t, const double*) { return t.Pv; }
FNPF_HD inline const float* pv_of(const PXfer& t, const float*) { return t.Pv_f; }

// x_f[g] += (P x_c)[g] at every interior fine node g: the coarse element
// polynomial of the node's first element evaluated at the node.
template <class T>
struct ProlongItemT {
  struct Args {
    PMesh f, c;
    PXfer t;
    const T* xc;
    T* xf;
  };
  FNPF_HD static void at(int64_t g, const Args& a) {
    if (g >= a.f.NI) return;
    const int64_t slot = a.f.vinc[a.f.voff[g]];
    const int64_t per = (int64_t)a.f.nt * a.f.n;
    const int64_t elem = slot / per;
    const int idx = (int)(slot - elem * per);
    const int cf = idx % a.f.nt, mf = idx / a.f.nt;
    const int e = (int)(elem / a.f.nz), l = (int)(elem - (int64_t)e * a.f.nz);
    const int* tnc = a.c.tn + (int64_t)e * a.c.nt;
    const T* Pt = ptri_of(a.t, (const T*)nullptr) + (int64_t)cf * a.c.nt;
    const T* Pv = pv_of(a.t, (const T*)nullptr) + (int64_t)mf * a.c.n;
    T s = 0;
    for (int mc = 0; mc < a.c.n; ++mc) {
      const T* xp = a.xc + ((int64_t)l * a.c.p + mc) * a.c.ns;
      T sc = 0;
      for (int k = 0; k < a.c.nt; ++k) sc += Pt[k] * xp[tnc[k]];
      s += Pv[mc] * sc;
    }
    a.xf[g] += s;
  }
};
using ProlongItem = ProlongItemT<double>;

// Element result of coarse local node (c', m') of coarse element elem: the
// transposed interpolation of the fine residual, each fine node's value
// divided by the number of fine elements that share it (so that the gather
// over the coarse elements gives P^T r exactly).
template <class T>
struct RestrictItemT {
  struct Args {
    PMesh f, c;
    PXfer t;
    const T* rf;
    T* yec;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const int64_t per = (int64_t)a.c.nt * a.c.n;
    const int64_t elem = i / per;
    const int idx = (int)(i - elem * per);
    const int cc = idx % a.c.nt, mc = idx / a.c.nt;
    const int e = (int)(elem / a.c.nz), l = (int)(elem - (int64_t)e * a.c.nz);
    const int* tnf = a.f.tn + (int64_t)e * a.f.nt;
    const T* Ptri = ptri_of(a.t, (const T*)nullptr);
    const T* Pvt = pv_of(a.t, (const T*)nullptr);
    T s = 0;
    for (int mf = 0; mf < a.f.n; ++mf) {
      const T pv = Pvt[(int64_t)mf * a.c.n + mc];
      const int64_t plane = ((int64_t)l * a.f.p + mf) * a.f.ns;
      T sf = 0;
      for (int k = 0; k < a.f.nt; ++k) {
        const int64_t g = plane + tnf[k];
        const T mult = (T)(a.f.voff[g + 1] - a.f.voff[g]);
        sf += Ptri[(int64_t)k * a.c.nt + cc] * a.rf[g] / mult;
      }
      s += pv * sf;
    }
    a.yec[i] = s;
  }
};
using RestrictItem = RestrictItemT<double>;

// eta and h at coarse surface node J: the fine triangle polynomial of J's
// first triangle evaluated at J.
struct CoarseGeoItem {
  struct Args {
    PMesh f, c;
    PXfer t;
    const double *etaf, *hf;
    double *etac, *hc;
  };
  FNPF_HD static void at(int64_t J, const Args& a) {
    const int64_t slot = a.c.sinc[a.c.soff[J]];
    const int tri = (int)(slot / a.c.nt), cc = (int)(slot - (int64_t)tri * a.c.nt);
    const int* tnf = a.f.tn + (int64_t)tri * a.f.nt;
    const double* Et = a.t.Etri + (int64_t)cc * a.f.nt;
    double se = 0, sh = 0;
    for (int k = 0; k < a.f.nt; ++k) {
      se += Et[k] * a.etaf[tnf[k]];
      sh += Et[k] * a.hf[tnf[k]];
    }
    a.etac[J] = se;
    a.hc[J] = sh;
  }
};

// One Chebyshev step: d = s d + c D^-1 r, x += d.
template <class T>
struct ChebItemT {
  struct Args {
    double s, c;
    const T *r, *diag;
    T *d, *x;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const T d = (T)a.s * a.d[i] + (T)a.c * a.r[i] / a.diag[i];
    a.d[i] = d;
    a.x[i] += d;
  }
};
using ChebItem = ChebItemT<double>;

// The end of one Chebyshev step at interior node g: q = the gathered element
// results of A d (d the previous direction), r -= q, d = s d + c D^-1 r, x += d
// (the gather, the residual update and the smoother update of one step in one
// pass; only node g's own entries are written).
template <class T>
struct GatherChebItemT {
  struct Args {
    const int64_t *off, *inc;
    const T* ye;
    int64_t NI;
    double s, c;
    const T* diag;
    T *r, *d, *x;
  };
  FNPF_HD static void at(int64_t g, const Args& a) {
    if (g >= a.NI) return;
    T q = 0;
    for (int64_t j = a.off[g]; j < a.off[g + 1]; ++j) q += a.ye[a.inc[j]];
    const T r = a.r[g] - q;
    const T d = (T)a.s * a.d[g] + (T)a.c * r / a.diag[g];
    a.r[g] = r;
    a.d[g] = d;
    a.x[g] += d;
  }
};
using GatherChebItem = GatherChebItemT<double>;

// r = b - (gathered element results) at interior node g (r's surface plane
// untouched): the residual after an operator application.
template <class T>
struct GatherResidualItemT {
  struct Args {
    const int64_t *off, *inc;
    const T* ye;
    int64_t NI;
    const T* b;
    T* r;
  };
  FNPF_HD static void at(int64_t g, const Args& a) {
    if (g >= a.NI) return;
    T q = 0;
    for (int64_t j = a.off[g]; j < a.off[g + 1]; ++j) q += a.ye[a.inc[j]];
    a.r[g] = a.b[g] - q;
  }
};
using GatherResidualItem = GatherResidualItemT<double>;

// Projected initial guess (Fischer's projection for successive right-hand
// sides): x0 = sum_j c_j H_j and r0 = b - sum_j c_j (A H_j) at interior node i
// (the basis vectors at stride N; coefficients in the launch's parameters).
struct ProjCombItem {
  struct Args {
    int nb;
    double c[kMaxProj + 1];
    const double* H[kMaxProj + 1];
    const double* AH[kMaxProj + 1];
    double *x, *r;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    double x = 0, q = 0;
    for (int j = 0; j < a.nb; ++j) {
      x += a.c[j] * a.H[j][i];
      q += a.c[j] * a.AH[j][i];
    }
    a.x[i] = x;
    a.r[i] -= q;
  }
};

// x += (double) e: a correction of the FP32 inner solve added to the FP64 iterate.
struct AddCastItem {
  struct Args {
    const float* e;
    double* x;
  };
  FNPF_HD static void at(int64_t i, const Args& a) { a.x[i] += (double)a.e[i]; }
};

// A fixed pseudo-random vector in [-1, 1) on the interior (splitmix64 of the
// index), zero on the surface plane: the start of the eigenvalue estimate.
struct HashItem {
  struct Args {
    int64_t NI;
    double* x;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    if (i >= a.NI) {
      a.x[i] = 0.0;
      return;
    }
    uint64_t z = (uint64_t)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    a.x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
};

// A level of the hierarchy: its mesh view and workspace (level 0: the mesh's own).
struct PLevel {
  PMesh m;
  double *G, *F, *ye, *diag;   // metric, fluxes, element results, Jacobi diagonal
  double* vt;                  // vertical derivatives and sums of the operator
  double *eta, *h;             // [ns] geometry (level 0: the caller's arrays)
  double *x, *b, *r, *d, *q;   // [N] smoother and V-cycle vectors
  double lo, hi;               // Chebyshev interval of D^-1 A
  // FP32 copies for an FP32 V-cycle: metric, fluxes, element results, vertical
  // terms, diagonal and vectors
  float *G32, *F32, *ye32, *vt32, *diag32, *x32, *b32, *r32, *d32, *q32;
};

// A level's buffers in the value type T of a V-cycle.
template <class T>
struct LView {
  T *G, *F, *ye, *vt, *diag, *x, *b, *r, *d, *q;
};
inline LView<double> view_of(PLevel& L, const double*) { return {L.G, L.F, L.ye, L.vt, L.diag, L.x, L.b, L.r, L.d, L.q}; }
inline LView<float> view_of(PLevel& L, const float*) {
  return {L.G32, L.F32, L.ye32, L.vt32, L.diag32, L.x32, L.b32, L.r32, L.d32, L.q32};
}

struct PMG {
  int nlev = 0;
  PLevel lev[kMaxLevels];
  PXfer xf[kMaxLevels];        // xf[l]: level l -> l + 1
};

// The orders of the hierarchy for order p: p, p/2, ..., 1.
inline int pmg_orders(int p, int* q) {
  int n = 0;
  for (int o = p; n < kMaxLevels; o /= 2) {
    q[n++] = o;
    if (o == 1) break;
  }
  return n;
}

// Workspace of level l >= 1 (take(&ptr, count) as carve), and of level 0's vectors.
template <class Take>
void carve_level(const PMesh& m, bool own_operator, PLevel* L, Take take) {
  const int64_t pts = m.nelem * m.n * m.nq;
  if (own_operator) {
    take(&L->G, pts * 6);
    take(&L->F, pts * 3);
    take(&L->ye, m.nelem * m.nt * m.n);
    take(&L->vt, m.nelem * m.nt * m.n);
    take(&L->diag, m.N);
    take(&L->eta, m.ns);
    take(&L->h, m.ns);
  }
  double** v[] = {&L->x, &L->b, &L->r, &L->d, &L->q};
  for (double** p : v) take(p, m.N);
  // FP32 buffers (a float buffer of c entries takes (c + 1) / 2 doubles)
  auto takef = [&](float** p, int64_t c) {
    double* d = nullptr;
    take(&d, (c + 1) / 2);
    *p = reinterpret_cast<float*>(d);
  };
  takef(&L->G32, pts * 6);
  takef(&L->F32, pts * 3);
  takef(&L->ye32, m.nelem * m.nt * m.n);
  takef(&L->vt32, m.nelem * m.nt * m.n);
  takef(&L->diag32, m.N);
  float** vf[] = {&L->x32, &L->b32, &L->r32, &L->d32, &L->q32};
  for (float** p : vf) takef(p, m.N);
}

// FP32 copies of a level's operator tables, from the host copy of its packed
// FP64 tables (the layout of bind_tables).
template <class Up>
bool float_tables(PMesh* pm, const double* host_tab, Up up) {
  PMesh hv = *pm;
  bind_tables(&hv, host_tab);
  auto cvt = [](const double* a, int64_t n) { return std::vector<float>(a, a + n); };
  const int64_t qt = (int64_t)pm->nq * pm->nt;
  pm->Lf = up(cvt(hv.L, qt));
  pm->Lrf = up(cvt(hv.Lr, qt));
  pm->Lsf = up(cvt(hv.Ls, qt));
  pm->Df = up(cvt(hv.D, (int64_t)pm->n * pm->n));
  return pm->Lf && pm->Lrf && pm->Lsf && pm->Df;
}

// The hierarchy of a mesh of order p over the triangles (verts, tris), level 0
// being the mesh's own view m0 and workspace w0.  up(vector) returns a copy of
// a host vector in the memory the items read (null on failure), take(&ptr,
// count) a zeroed buffer of count doubles.  False on a failure of either or of
// the host set-up.
template <class Up, class Take>
bool build_pmg(const PMesh& m0, const PWork& w0, const double* verts, int nverts, const int* tris, int nz, PMG* pmg,
               Up up, Take take) {
  int q[kMaxLevels];
  const int nl = pmg_orders(m0.p, q);
  std::vector<LevelHost> H(nl);
  for (int l = 0; l < nl; ++l)
    if (!build_level(verts, nverts, tris, m0.ntri, q[l], nz, &H[l])) return false;
  pmg->nlev = nl;
  PLevel& L0 = pmg->lev[0];
  L0 = PLevel{};
  L0.m = m0;
  L0.G = w0.G;
  L0.F = w0.F;
  L0.ye = w0.ye;
  L0.vt = w0.vt;
  L0.diag = w0.diag;
  if (!float_tables(&L0.m, H[0].tab.data(), up)) return false;
  carve_level(m0, false, &L0, take);
  for (int l = 1; l < nl; ++l) {
    PMesh pm{};
    pm.p = q[l];
    pm.n = q[l] + 1;
    pm.nz = nz;
    pm.nt = H[l].nt;
    pm.nq = H[l].nq;
    pm.ntri = m0.ntri;
    pm.ns = H[l].ns;
    pm.nv = (int64_t)nz * q[l] + 1;
    pm.N = pm.nv * pm.ns;
    pm.NI = pm.N - pm.ns;
    pm.nelem = m0.nelem;
    pm.tn = up(H[l].tn);
    const double* tab = up(H[l].tab);
    if (!pm.tn || !tab) return false;
    bind_tables(&pm, tab);
    if (!float_tables(&pm, H[l].tab.data(), up)) return false;
    pm.voff = up(H[l].voff);
    pm.vinc = up(H[l].vinc);
    pm.soff = up(H[l].soff);
    pm.sinc = up(H[l].sinc);
    if (!pm.voff || !pm.vinc || !pm.soff || !pm.sinc) return false;
    PLevel& L = pmg->lev[l];
    L = PLevel{};
    L.m = pm;
    carve_level(pm, true, &L, take);
  }
  for (int l = 0; l + 1 < nl; ++l) {
    std::vector<double> Pt, Pv, Et;
    if (!transfer_tables(H[l], H[l + 1], &Pt, &Pv, &Et)) return false;
    pmg->xf[l] = PXfer{up(Pt), up(Pv), up(Et), up(std::vector<float>(Pt.begin(), Pt.end())),
                        up(std::vector<float>(Pv.begin(), Pv.end()))};
    if (!pmg->xf[l].Ptri || !pmg->xf[l].Pv || !pmg->xf[l].Etri || !pmg->xf[l].Ptri_f || !pmg->xf[l].Pv_f) return false;
  }
  return true;
}

// Relaxation zones at surface node c after the step to t1 (Sec. 3.3, Step
// 4.7): f <- (1 - C_r) f + C_r f_true, the target the linear incident wave
//   eta_I = r a cos(theta), phi_I = r (g a / omega) cosh(k (eta_I + h)) / cosh(k h) sin(theta),
// theta = kx x + ky y - omega t1 + phase, r = min(1, t1 / ramp), in generation
// nodes and zero in absorption nodes.
struct RelaxItem {
  struct Args {
    PMesh m;
    const double* h;
    double t1, g;
    double *eta, *phis;
  };
  FNPF_HD static void at(int64_t c, const Args& a) {
    const PMesh& m = a.m;
    const double cr = m.rcr[c];
    if (cr == 0.0) return;
    double te = 0.0, tp = 0.0;
    if (m.rgen[c] != 0.0) {
      const double r = a.t1 / m.ramp < 1.0 ? a.t1 / m.ramp : 1.0;
      const double th = m.kx * m.xs[c] + m.ky * m.ys[c] - m.omega * a.t1 + m.phase;
      const double k = sqrt(m.kx * m.kx + m.ky * m.ky);
      te = r * m.amp * cos(th);
      tp = r * (a.g * m.amp / m.omega) * cosh(k * (te + a.h[c])) / cosh(k * a.h[c]) * sin(th);
    }
    a.eta[c] = (1.0 - cr) * a.eta[c] + cr * te;
    a.phis[c] = (1.0 - cr) * a.phis[c] + cr * tp;
  }
};

// The relaxation zones' vector-Jacobian product at surface node c (the blend
// f <- (1 - C_r) f + C_r f_true after the step to t1): the cotangents of the
// blended state scaled by 1 - C_r into (le, lp), and C_r lam_phi d phi_I / dh
// (the target potential's dependence on the depth, generation nodes) into dh.
struct RelaxVjpItem {
  struct Args {
    PMesh m;
    const double* h;
    double t1, g;
    const double *lam_e, *lam_p;
    double *le, *lp, *dh;
  };
  FNPF_HD static void at(int64_t c, const Args& a) {
    const PMesh& m = a.m;
    const double cr = m.rcr[c];
    a.le[c] = (1.0 - cr) * a.lam_e[c];
    a.lp[c] = (1.0 - cr) * a.lam_p[c];
    double d = 0.0;
    if (cr != 0.0 && m.rgen[c] != 0.0) {
      const double r = a.t1 / m.ramp < 1.0 ? a.t1 / m.ramp : 1.0;
      const double th = m.kx * m.xs[c] + m.ky * m.ys[c] - m.omega * a.t1 + m.phase;
      const double k = sqrt(m.kx * m.kx + m.ky * m.ky);
      const double te = r * m.amp * cos(th), hc = a.h[c];
      const double ch = cosh(k * hc);
      // d/dh [cosh(k (te + h)) / cosh(k h)]
      const double dq = k * (sinh(k * (te + hc)) * ch - cosh(k * (te + hc)) * sinh(k * hc)) / (ch * ch);
      d = cr * a.lam_p[c] * r * (a.g * m.amp / m.omega) * sin(th) * dq;
    }
    a.dh[c] = d;
  }
};

// The transpose of the modal filter (the map f -> f with the triangle-interior
// values replaced by F applied to the triangle's values): slot (t, c) gets
// sum over the interior local nodes i of F[i][c] lam(tn[i]).
struct FilterTSlotItem {
  struct Args {
    PMesh m;
    const double* lam;
    double* ft;
  };
  FNPF_HD static void at(int64_t i, const Args& a) {
    const PMesh& m = a.m;
    const int t = (int)(i / m.nt), c = (int)(i - (int64_t)t * m.nt);
    const int* tn = m.tn + (int64_t)t * m.nt;
    double s = 0;
    for (int k = 0; k < m.nt; ++k)
      if (m.interior[k]) s += m.filt[(int64_t)k * m.nt + c] * a.lam[tn[k]];
    a.ft[i] = s;
  }
};

// Node g: its own cotangent unless it is a triangle-interior node (replaced by
// the filter), plus its slots' FilterTSlotItem sums.
struct FilterTGatherItem {
  struct Args {
    PMesh m;
    const double *lam, *ft;
    double* out;
  };
  FNPF_HD static void at(int64_t g, const Args& a) {
    const PMesh& m = a.m;
    const int64_t j0 = m.soff[g];
    double s = m.interior[m.sinc[j0] % m.nt] ? 0.0 : a.lam[g];
    for (int64_t j = j0; j < m.soff[g + 1]; ++j) s += a.ft[m.sinc[j]];
    a.out[g] = s;
  }
};

// ---------------------------------------------------------------------------
// Orchestration.

struct Params {
  double rtol;
  int max_iter;
  double mass_rtol;
  int mass_max_iter;
  double g;
  int linear;
  int pmg;            // 1: p-multigrid V-cycle preconditioner, 0: Jacobi
  int cheb_degree;    // Chebyshev degree of the pre- and post-smoothing
  int coarse_degree;  // Chebyshev degree on the coarsest level
  double cheb_range;  // the smoothers act on [lmax / cheb_range, lmax]
  int pc32;           // 1: the V-cycle in FP32 (FP64 PCG around it)
  int projection;     // 0..kMaxProj: previous solutions in the projected initial guess (0: the caller's guess)
  int mixed;          // 1: FP64 defect correction around an FP32 PCG with the FP32 V-cycle
  double inner_rtol;  // the FP32 solve's tolerance relative to the current FP64 residual
  int max_outer;      // defect-correction steps at most
};

#define FNPF_PS_TRY(...)                 \
  do {                                   \
    const fnpf_status st_ = (__VA_ARGS__); \
    if (st_ != FNPF_OK) return st_;      \
  } while (0)

template <class Ex>
struct Stepper {
  const PMesh& m;
  PWork& w;
  Ex& ex;
  PMG* pmg = nullptr;   // the hierarchy (needed when Params::pmg is set)
  bool reuse_lmax = false;   // keep the levels' Chebyshev intervals (stages 2-4 of an RK4 step)

  template <class It>
  fnpf_status go(int64_t n, const typename It::Args& a) {
    if (n <= 0) return FNPF_OK;
    return ex.template run<It>(n, a) ? FNPF_ECUDA : FNPF_OK;
  }

  // The element results ye of A x on the mesh view mv with its metric G (the
  // vertical derivatives, the fluxes, the vertical sums, the node contractions).
  // The element results ye of A x: one block per prism, staged in shared memory.
  template <class T>
  fnpf_status elements(const PMesh& mv, const T* G, T* F, T* ye, T* vt, const T* x) {
    (void)F;
    (void)vt;
    if (mv.nelem <= 0) return FNPF_OK;
    const size_t smem = sizeof(T) * (size_t)ElementBlock<T>::smem_entries(mv);
    return ex.template run_block<ElementBlock<T>>(mv.nelem, smem, {mv, G, x, ye}) ? FNPF_ECUDA : FNPF_OK;
  }

  // The same element results from the one-thread-per-item kernels (the
  // reference of the block form: the same arithmetic in the same order).
  template <class T>
  fnpf_status elements_items(const PMesh& mv, const T* G, T* F, T* ye, T* vt, const T* x) {
    const int64_t nodes = mv.nelem * mv.nt * mv.n;
    FNPF_PS_TRY(go<DtItemT<T>>(nodes, {mv, x, vt}));
    FNPF_PS_TRY(go<FluxItemT<T>>(mv.nelem * mv.n * mv.nq, {mv, G, x, vt, F}));
    FNPF_PS_TRY(go<TSumItemT<T>>(nodes, {mv, F, vt}));
    return go<NodeItemT<T>>(nodes, {mv, F, vt, ye});
  }

  // *out = x . y over n entries (two launches and a read of the scalar).
  fnpf_status dot(const double* x, const double* y, int64_t n, double* out) {
    if (n <= 0) {
      *out = 0;
      return FNPF_OK;
    }
    const int64_t np = dot_partials(n);
    FNPF_PS_TRY(go<DotPartItem>(np, {x, y, n, w.part}));
    FNPF_PS_TRY(go<SumItem>(1, {w.part, np, w.scal}));
    return ex.get(out, w.scal, 1) ? FNPF_ECUDA : FNPF_OK;
  }

  // G and the Jacobi diagonal for the geometry of (eta, h).
  fnpf_status geometry(const double* eta, const double* h) {
    FNPF_PS_TRY(go<GeomItem>(m.nelem * m.n * m.nq, {m, eta, h, w.G}));
    FNPF_PS_TRY(go<DiagItem>(m.nelem * m.nt * m.n, {m, w.G, w.ye}));
    return go<GatherItem>(m.N, {m.voff, m.vinc, w.ye, w.diag});
  }

  // y = A x with the stored G (the full operator, surface rows included).
  fnpf_status apply(const double* x, double* y) {
    FNPF_PS_TRY(elements(m, w.G, w.F, w.ye, w.vt, x));
    return go<GatherItem>(m.N, {m.voff, m.vinc, w.ye, y});
  }

  // *out (device) = x . y over n entries, without reading it back.
  template <class T>
  fnpf_status dot_dev(const T* x, const T* y, int64_t n, double* out) {
    const int64_t np = dot_partials(n);
    FNPF_PS_TRY(go<DotPartItemT<T>>(np, {x, y, n, w.part}));
    return go<SumItem>(1, {w.part, np, out});
  }

  // Preconditioned CG over n entries with its scalars on the device: on entry
  // r = b - A x; op(p, q) sets q = A p, pre(r, z) sets z = M^-1 r (p's and q's
  // entries beyond n, if any, are the caller's).  The host reads the state
  // after the convergence test of every iteration when check == 1 (the
  // preconditioner of a converged iteration is then never applied), else at
  // the end of every check-th iteration; the iterates, iteration count and
  // residual equal those of reading every scalar at once.  x may be null
  // (only the coefficients are wanted: hist).  *iters and *rr: completed
  // iterations and the last r.r (unchanged when no iteration completed).
  template <class T, class Op, class Pre>
  fnpf_status cg_run(int64_t n, T* x, T* r, T* z, T* p, T* q, double stop, int max_iter, int check, double* hist,
                     Op op, Pre pre, int* iters, double* rr) {
    double* cg = w.cg;
    FNPF_PS_TRY(pre(r, z));
    FNPF_PS_TRY(go<CopyItemT<T>>(n, {z, p}));
    FNPF_PS_TRY(dot_dev(r, z, n, cg + kRZ));
    FNPF_PS_TRY(go<CgResetItem>(1, {cg}));
    double st[kCgSlots] = {0};
    for (int it = 0; it < max_iter; ++it) {
      FNPF_PS_TRY(op(p, q));
      FNPF_PS_TRY(dot_dev(p, q, n, cg + kPQ));
      FNPF_PS_TRY(go<CgAlphaItem>(1, {cg, hist}));
      FNPF_PS_TRY(go<CgUpdateItemT<T>>(n, {cg, p, q, x, r}));
      FNPF_PS_TRY(dot_dev(r, r, n, cg + kRR));
      FNPF_PS_TRY(go<CgCheckItem>(1, {cg, stop}));
      if (check == 1) {
        if (ex.get(st, cg, kCgSlots)) return FNPF_ECUDA;
        if (st[kDONE] != 0.0) break;
      }
      FNPF_PS_TRY(pre(r, z));
      FNPF_PS_TRY(dot_dev(r, z, n, cg + kRZN));
      FNPF_PS_TRY(go<CgBetaItem>(1, {cg, hist}));
      FNPF_PS_TRY(go<CgDirItemT<T>>(n, {cg, z, p}));
      if (check > 1 && (it + 1) % check == 0) {
        if (ex.get(st, cg, kCgSlots)) return FNPF_ECUDA;
        if (st[kDONE] != 0.0) break;
      }
    }
    if (ex.get(st, cg, kCgSlots)) return FNPF_ECUDA;
    *iters = (int)st[kITERS];
    if (*iters > 0) *rr = st[kRR];   // else the caller's initial r.r stands
    const int done = (int)st[kDONE];
    return done == 1 ? FNPF_OK : done == 2 ? FNPF_EBREAKDOWN : done == 3 ? FNPF_EDIVERGED : FNPF_ENOCONV;
  }

  // ---- p-multigrid

  fnpf_status geometry_level(PLevel& L, const double* eta, const double* h) {
    FNPF_PS_TRY(go<GeomItem>(L.m.nelem * L.m.n * L.m.nq, {L.m, eta, h, L.G}));
    FNPF_PS_TRY(go<DiagItem>(L.m.nelem * L.m.nt * L.m.n, {L.m, L.G, L.ye}));
    return go<GatherItem>(L.m.N, {L.m.voff, L.m.vinc, L.ye, L.diag});
  }

  fnpf_status apply_level(PLevel& L, const double* x, double* y) {
    FNPF_PS_TRY(elements(L.m, L.G, L.F, L.ye, L.vt, x));
    return go<GatherItem>(L.m.N, {L.m.voff, L.m.vinc, L.ye, y});
  }

  // Largest eigenvalue of D^-1 A_II on a level: the Lanczos tridiagonal matrix of
  // k Jacobi-PCG steps from a fixed pseudo-random right-hand side (its largest
  // eigenvalue by bisection on the Sturm sequence).
  fnpf_status lmax_level(PLevel& L, double* out) {
    const int64_t N = L.m.N, NI = L.m.NI;
    const int k_max = kMaxLanczos;
    double al[k_max], be[k_max], hist[2 * k_max];
    FNPF_PS_TRY(go<HashItem>(N, {NI, L.r}));
    FNPF_PS_TRY(go<FillItem>(N, {0.0, L.d}));   // the direction's surface plane stays zero
    int k = 0;
    double rr = 0;
    const fnpf_status cs =
        cg_run(NI, static_cast<double*>(nullptr), L.r, L.x, L.d, L.q, 0.0, k_max, k_max, w.cg + kCgSlots,
               [&](const double* pv, double* qv) { return apply_level(L, pv, qv); },
               [&](const double* rv, double* zv) { return go<DivItem>(NI, {rv, L.diag, zv}); }, &k, &rr);
    if (cs == FNPF_ECUDA) return cs;
    if (k == 0) return FNPF_EBREAKDOWN;
    if (ex.get(hist, w.cg + kCgSlots, 2 * k)) return FNPF_ECUDA;
    for (int j = 0; j < k; ++j) {
      al[j] = hist[2 * j];
      be[j] = hist[2 * j + 1];
    }
    // T[j][j] = 1/al_j + be_(j-1)/al_(j-1), T[j][j-1] = sqrt(be_(j-1))/al_(j-1)
    double dg[k_max], off[k_max];
    for (int j = 0; j < k; ++j) {
      dg[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
      off[j] = j > 0 ? sqrt(be[j - 1]) / al[j - 1] : 0.0;
    }
    double hi = 0;
    for (int j = 0; j < k; ++j) hi = std::max(hi, dg[j] + fabs(off[j]) + (j + 1 < k ? fabs(off[j + 1]) : 0.0));
    double lo = 0;
    for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {   // count of eigenvalues above mid
      const double mid = 0.5 * (lo + hi);
      int below = 0;   // negative pivots of T - mid I count the eigenvalues below mid
      double q = 1;
      for (int j = 0; j < k; ++j) {
        q = (dg[j] - mid) - (j > 0 ? off[j] * off[j] / q : 0.0);
        if (q == 0) q = -1e-300;
        if (q < 0) ++below;
      }
      if (below < k) lo = mid;   // an eigenvalue lies above mid
      else hi = mid;
    }
    *out = hi;
    return FNPF_OK;
  }

  // Geometry, diagonals and Chebyshev intervals of every level for (eta, h)
  // (the intervals kept when reuse_lmax: within one RK4 step the geometry moves
  // by O(dt), well inside the 10 % margin on lambda_max); level 0's geometry is
  // current.
  fnpf_status setup_pmg(const double* eta, const double* h, const Params& o) {
    pmg->lev[0].eta = const_cast<double*>(eta);
    pmg->lev[0].h = const_cast<double*>(h);
    for (int l = 0; l < pmg->nlev; ++l) {
      PLevel& L = pmg->lev[l];
      if (l > 0) {
        PLevel& F = pmg->lev[l - 1];
        FNPF_PS_TRY(go<CoarseGeoItem>(L.m.ns, {F.m, L.m, pmg->xf[l - 1], F.eta, F.h, L.eta, L.h}));
        FNPF_PS_TRY(geometry_level(L, L.eta, L.h));
      }
      if (!(reuse_lmax && L.hi > 0)) {
        double lmax = 0;
        FNPF_PS_TRY(lmax_level(L, &lmax));
        L.hi = 1.1 * lmax;
        L.lo = L.hi / o.cheb_range;
      }
      if (o.pc32 || o.mixed) {   // the FP32 V-cycle's metric and diagonal: the FP64 ones rounded
        FNPF_PS_TRY(go<CastItem<float, double>>(L.m.nelem * L.m.n * L.m.nq * 6, {L.G, L.G32}));
        FNPF_PS_TRY(go<CastItem<float, double>>(L.m.N, {L.diag, L.diag32}));
      }
    }
    return FNPF_OK;
  }

  // deg Chebyshev steps on level L in the value type T (its buffers v): x and
  // r = b - A x (both in, both out; r updated at the end only if need_r).  Step
  // k > 0 is the element results of A d_(k-1) followed by one fused
  // gather-and-update pass.
  template <class T>
  fnpf_status cheb(PLevel& L, const LView<T>& v, T* x, T* r, int deg, bool need_r) {
    const int64_t N = L.m.N, NI = L.m.NI;
    const double theta = 0.5 * (L.hi + L.lo), delta = 0.5 * (L.hi - L.lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    FNPF_PS_TRY(go<FillItemT<T>>(N, {0.0, v.d}));
    FNPF_PS_TRY(go<ChebItemT<T>>(NI, {0.0, 1.0 / theta, r, v.diag, v.d, x}));
    for (int k = 1; k < deg; ++k) {
      FNPF_PS_TRY(elements<T>(L.m, v.G, v.F, v.ye, v.vt, v.d));
      const double rn = 1.0 / (2.0 * sigma - rho);
      FNPF_PS_TRY(go<GatherChebItemT<T>>(N, {L.m.voff, L.m.vinc, v.ye, NI, rn * rho, 2.0 * rn / delta, v.diag, r, v.d, x}));
      rho = rn;
    }
    if (!need_r) return FNPF_OK;
    FNPF_PS_TRY(elements<T>(L.m, v.G, v.F, v.ye, v.vt, v.d));
    return go<GatherResidualItemT<T>>(N, {L.m.voff, L.m.vinc, v.ye, NI, r, r});
  }

  // x = M_l^-1 b: one V-cycle from x = 0 in the value type T (b and x: interior
  // values, surface plane zero).
  template <class T>
  fnpf_status vcycle(int l, const T* b, T* x, const Params& o) {
    PLevel& L = pmg->lev[l];
    const LView<T> v = view_of(L, (const T*)nullptr);
    const int64_t N = L.m.N, NI = L.m.NI;
    FNPF_PS_TRY(go<FillItemT<T>>(N, {0.0, x}));
    FNPF_PS_TRY(go<InteriorItemT<T>>(N, {NI, 1.0, b, v.r}));
    if (l == pmg->nlev - 1) return cheb<T>(L, v, x, v.r, o.coarse_degree, false);
    FNPF_PS_TRY(cheb<T>(L, v, x, v.r, o.cheb_degree, true));
    PLevel& C = pmg->lev[l + 1];
    const LView<T> c = view_of(C, (const T*)nullptr);
    FNPF_PS_TRY(go<RestrictItemT<T>>(C.m.nelem * C.m.nt * C.m.n, {L.m, C.m, pmg->xf[l], v.r, c.ye}));
    FNPF_PS_TRY(go<GatherItemT<T>>(C.m.N, {C.m.voff, C.m.vinc, c.ye, c.q}));
    FNPF_PS_TRY(go<InteriorItemT<T>>(C.m.N, {C.m.NI, 1.0, c.q, c.b}));
    FNPF_PS_TRY(vcycle<T>(l + 1, c.b, c.x, o));
    FNPF_PS_TRY(go<ProlongItemT<T>>(N, {L.m, C.m, pmg->xf[l], c.x, x}));
    FNPF_PS_TRY(elements<T>(L.m, v.G, v.F, v.ye, v.vt, x));
    FNPF_PS_TRY(go<GatherResidualItemT<T>>(N, {L.m.voff, L.m.vinc, v.ye, NI, b, v.r}));
    return cheb<T>(L, v, x, v.r, o.cheb_degree, false);
  }

  // z = M^-1 r: Jacobi, one FP64 V-cycle, or one FP32 V-cycle on the rounded
  // residual (pc32) whose result is widened back.
  fnpf_status precond(const double* r, double* z, const Params& o) {
    if (!o.pmg) return go<DivItem>(m.NI, {r, w.diag, z});
    if (!o.pc32) return vcycle<double>(0, r, z, o);
    PLevel& L0 = pmg->lev[0];
    FNPF_PS_TRY(go<CastItem<float, double>>(m.N, {r, L0.b32}));
    FNPF_PS_TRY(vcycle<float>(0, L0.b32, L0.x32, o));
    return go<CastItem<double, float>>(m.N, {L0.x32, z});
  }

  // z = M^-1 r for the geometry of (eta, h) (r, z [N]; r's surface plane is ignored).
  fnpf_status precond_apply(const double* eta, const double* h, const double* r, double* z, const Params& o) {
    if (o.pmg && !pmg) return FNPF_EINVAL;
    FNPF_PS_TRY(geometry(eta, h));
    if (o.pmg) FNPF_PS_TRY(setup_pmg(eta, h, o));
    FNPF_PS_TRY(go<InteriorItem>(m.N, {m.NI, 1.0, r, w.r}));
    FNPF_PS_TRY(go<FillItem>(m.N, {0.0, z}));
    return precond(w.r, z, o);
  }

  // The projected initial guess: phi (interior) = the A-orthogonal projection
  // of the solution onto the span of the last o.projection solutions and the
  // caller's guess (Fischer, Comput. Methods Appl. Mech. Engrg. 163, 1998), and
  // w.r = b - A phi (w.r = b on entry).  The Gram system is formed on the
  // device and read once; a vector whose Cholesky pivot falls below 1e-14 of its
  // diagonal (nearly dependent, zero, non-finite) is dropped.
  fnpf_status project(double* phi, const Params& o) {
    const int64_t N = m.N, NI = m.NI;
    const int nh = std::min(w.hist_n, o.projection);
    double* H[kMaxProj + 1];
    double* AH[kMaxProj + 1];
    int nb = 0;
    for (int j = 0; j < nh; ++j) {   // the most recent first
      const int slot = (w.hist_next - 1 - j + 2 * kMaxProj) % kMaxProj;
      H[nb] = w.H + (int64_t)slot * N;
      AH[nb++] = w.AH + (int64_t)slot * N;
    }
    H[nb] = w.H + (int64_t)kMaxProj * N;   // the caller's guess, surface plane zero
    AH[nb++] = w.AH + (int64_t)kMaxProj * N;
    FNPF_PS_TRY(go<InteriorItem>(N, {NI, 1.0, phi, H[nb - 1]}));
    for (int j = 0; j < nb; ++j) FNPF_PS_TRY(apply(H[j], AH[j]));
    int k = 0;
    for (int i = 0; i < nb; ++i)
      for (int j = i; j < nb; ++j) FNPF_PS_TRY(dot_dev(H[i], AH[j], NI, w.gram + k++));
    for (int i = 0; i < nb; ++i) FNPF_PS_TRY(dot_dev(H[i], w.r, NI, w.gram + k++));
    double g[(kMaxProj + 1) * (kMaxProj + 2)];
    if (ex.get(g, w.gram, k)) return FNPF_ECUDA;
    double G[kMaxProj + 1][kMaxProj + 1], rhs[kMaxProj + 1];
    k = 0;
    for (int i = 0; i < nb; ++i)
      for (int j = i; j < nb; ++j) G[i][j] = G[j][i] = g[k++];
    for (int i = 0; i < nb; ++i) rhs[i] = g[k++];
    // Cholesky of the kept vectors, in order, dropping dependent ones
    double Lc[kMaxProj + 1][kMaxProj + 1];
    int kept[kMaxProj + 1], nk = 0;
    for (int j = 0; j < nb; ++j) {
      double l[kMaxProj + 1];
      double d = G[j][j];
      for (int a = 0; a < nk; ++a) {
        double v = G[j][kept[a]];
        for (int b = 0; b < a; ++b) v -= l[b] * Lc[a][b];
        l[a] = v / Lc[a][a];
        d -= l[a] * l[a];
      }
      if (!(d > 1e-14 * G[j][j]) || !isfinite(d)) continue;
      for (int a = 0; a < nk; ++a) Lc[nk][a] = l[a];
      Lc[nk][nk] = sqrt(d);
      kept[nk++] = j;
    }
    ProjCombItem::Args a{};
    a.nb = nb;
    for (int j = 0; j < nb; ++j) {
      a.c[j] = 0.0;
      a.H[j] = H[j];
      a.AH[j] = AH[j];
    }
    double y[kMaxProj + 1];
    for (int i = 0; i < nk; ++i) {   // L y = rhs, L^T c = y
      double v = rhs[kept[i]];
      for (int b = 0; b < i; ++b) v -= Lc[i][b] * y[b];
      y[i] = v / Lc[i][i];
    }
    for (int i = nk - 1; i >= 0; --i) {
      double v = y[i];
      for (int b = i + 1; b < nk; ++b) v -= Lc[b][i] * a.c[kept[b]];
      a.c[kept[i]] = v / Lc[i][i];
    }
    a.x = phi;
    a.r = w.r;
    return go<ProjCombItem>(NI, a);
  }

  // FP64 defect correction around an FP32 PCG (the mixed form): with w.r =
  // b - A phi (FP64) and b in w.z on entry, repeat until ||r|| <= stop: e = the
  // FP32 solution of A e = r to inner_rtol ||r|| (FP32 operator with the rounded
  // metric and tables, the FP32 V-cycle as preconditioner, CG scalars and dot
  // products accumulated in FP64), phi += e, r = b - A phi in FP64.
  fnpf_status defect_correction(double* phi, double stop, const Params& o, int* iters, int* outer, double* rr) {
    const int64_t N = m.N, NI = m.NI;
    PLevel& L0 = pmg->lev[0];
    int inner = 0, k = 0;
    fnpf_status st = FNPF_ENOCONV;
    for (;;) {
      if (sqrt(*rr) <= stop) {
        st = FNPF_OK;
        break;
      }
      if (k >= o.max_outer) break;
      ++k;
      FNPF_PS_TRY(go<CastItem<float, double>>(N, {w.r, w.ir}));   // r's surface plane is zero
      FNPF_PS_TRY(go<FillItemT<float>>(N, {0.0, w.ie}));
      FNPF_PS_TRY(go<FillItemT<float>>(N, {0.0, w.ip}));
      int it_in = 0;
      double rr_in = *rr;
      const fnpf_status si = cg_run(
          NI, w.ie, w.ir, w.iz, w.ip, w.iq, o.inner_rtol * sqrt(*rr), o.max_iter, 1, nullptr,
          [&](const float* pv, float* qv) {
            FNPF_PS_TRY(elements<float>(L0.m, L0.G32, L0.F32, L0.ye32, L0.vt32, pv));
            return go<GatherItemT<float>>(N, {L0.m.voff, L0.m.vinc, L0.ye32, qv});
          },
          [&](const float* rv, float* zv) { return vcycle<float>(0, rv, zv, o); }, &it_in, &rr_in);
      if (si != FNPF_OK && si != FNPF_ENOCONV) return si;
      inner += it_in;
      FNPF_PS_TRY(go<AddCastItem>(NI, {w.ie, phi}));
      FNPF_PS_TRY(go<InteriorItem>(N, {NI, 1.0, phi, w.pd}));
      FNPF_PS_TRY(apply(w.pd, w.q));
      FNPF_PS_TRY(go<LinItem>(NI, {w.z, -1.0, w.q, w.r}));   // r = b - A phi
      FNPF_PS_TRY(dot(w.r, w.r, NI, rr));
      if (!isfinite(*rr)) return FNPF_EDIVERGED;
    }
    *iters = inner;
    *outer = k;
    return st;
  }

  // phi = the solution of A_II phi_I = -A_IS phis (in: the interior guess),
  // phi = phis on the surface plane; Jacobi-PCG to ||r|| <= rtol ||b||.
  fnpf_status solve(const double* eta, const double* h, const double* phis, double* phi, const Params& o,
                    fnpf_solve_info* info) {
    const int64_t N = m.N, NI = m.NI;
    if (info) *info = fnpf_solve_info{0, 0, 0.0, FNPF_OK, 0.0f};
    if (o.pmg && !pmg) return FNPF_EINVAL;
    FNPF_PS_TRY(geometry(eta, h));
    if (o.pmg) FNPF_PS_TRY(setup_pmg(eta, h, o));
    FNPF_PS_TRY(go<SurfaceOnlyItem>(N, {NI, phis, w.xs}));
    FNPF_PS_TRY(apply(w.xs, w.q));
    FNPF_PS_TRY(go<InteriorItem>(N, {NI, -1.0, w.q, w.r}));   // r = b = -A_IS phis
    double bb = 0;
    FNPF_PS_TRY(dot(w.r, w.r, NI, &bb));
    if (o.mixed) FNPF_PS_TRY(go<CopyItem>(NI, {w.r, w.z}));   // b, for the outer residuals
    fnpf_status st = FNPF_OK;
    int it = 0, outer = 0;
    double rr = 0;
    if (!(bb > 0)) {   // b = 0: the solution is zero
      if (!(bb == 0)) st = FNPF_EDIVERGED;
      FNPF_PS_TRY(go<FillItem>(NI, {0.0, phi}));
    } else {
      const double stop = o.rtol * sqrt(bb);
      if (o.projection > 0) {
        FNPF_PS_TRY(project(phi, o));                              // phi = x0, r = b - A_II x0
        FNPF_PS_TRY(go<FillItem>(N, {0.0, w.pd}));                 // the direction's surface plane zero
      } else {
        FNPF_PS_TRY(go<InteriorItem>(N, {NI, 1.0, phi, w.pd}));   // the guess, surface plane zero
        FNPF_PS_TRY(apply(w.pd, w.q));
        FNPF_PS_TRY(go<AxpyItem>(NI, {-1.0, w.q, w.r}));          // r = b - A_II x0
      }
      FNPF_PS_TRY(dot(w.r, w.r, NI, &rr));
      if (o.mixed) {
        st = defect_correction(phi, stop, o, &it, &outer, &rr);
        if (st == FNPF_ECUDA) return st;
      } else if (sqrt(rr) > stop) {
        // w.pd's surface plane is zero (above); the loop writes its first NI entries only
        st = cg_run(NI, phi, w.r, w.z, w.pd, w.q, stop, o.max_iter, o.pmg ? 1 : 8, nullptr,
                    [&](const double* pv, double* qv) { return apply(pv, qv); },
                    [&](const double* rv, double* zv) { return precond(rv, zv, o); }, &it, &rr);
        if (st == FNPF_ECUDA) return st;
      }
    }
    if (o.projection > 0 && st == FNPF_OK && bb > 0) {   // the solution joins the projection basis
      FNPF_PS_TRY(go<CopyItem>(NI, {phi, w.H + (int64_t)w.hist_next * N}));
      w.hist_next = (w.hist_next + 1) % kMaxProj;
      w.hist_n = std::min(w.hist_n + 1, kMaxProj);
    }
    FNPF_PS_TRY(go<CopyItem>(m.ns, {phis, phi + NI}));
    if (info) {
      info->iters = it;
      info->outer_iters = outer;
      info->rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
      info->status = st;
    }
    return st;
  }

  // Vector-Jacobian product of the solve phi = S(eta, h, phis) (phi the forward
  // solution, full N): for dJ/dphi = lam [N], the adjoint solve A_II psi =
  // lam_I (the same operator and preconditioner: A is symmetric), then
  //   dJ/dphis = lam_S - (A psi)_S,  dJ/d(eta, h) = -d(psi^T A(eta, h) phi)/d(eta, h)
  // (psi zero on the surface plane).  lam_h may be null.
  fnpf_status solve_vjp(const double* eta, const double* h, const double* phi, const double* lam, double* lam_eta,
                        double* lam_phis, double* lam_h, const Params& o, fnpf_solve_info* info) {
    const int64_t N = m.N, NI = m.NI;
    if (info) *info = fnpf_solve_info{0, 0, 0.0, FNPF_OK, 0.0f};
    if (o.pmg && !pmg) return FNPF_EINVAL;
    Params oa = o;
    oa.projection = 0;   // the adjoint solves do not share the forward solutions' basis
    FNPF_PS_TRY(geometry(eta, h));
    if (oa.pmg) FNPF_PS_TRY(setup_pmg(eta, h, oa));
    double* psi = w.xs;
    FNPF_PS_TRY(go<FillItem>(N, {0.0, psi}));
    FNPF_PS_TRY(go<InteriorItem>(N, {NI, 1.0, lam, w.r}));
    double bb = 0;
    FNPF_PS_TRY(dot(w.r, w.r, NI, &bb));
    fnpf_status st = FNPF_OK;
    int it = 0, outer = 0;
    double rr = bb;
    if (bb > 0) {
      const double stop = oa.rtol * sqrt(bb);
      FNPF_PS_TRY(go<FillItem>(N, {0.0, w.pd}));
      if (oa.mixed) {
        FNPF_PS_TRY(go<CopyItem>(NI, {w.r, w.z}));
        st = defect_correction(psi, stop, oa, &it, &outer, &rr);
      } else {
        st = cg_run(NI, psi, w.r, w.z, w.pd, w.q, stop, oa.max_iter, oa.pmg ? 1 : 8, nullptr,
                    [&](const double* pv, double* qv) { return apply(pv, qv); },
                    [&](const double* rv, double* zv) { return precond(rv, zv, oa); }, &it, &rr);
      }
      if (st == FNPF_ECUDA) return st;
    } else if (!(bb == 0)) {
      st = FNPF_EDIVERGED;
    }
    if (info) {
      info->iters = it;
      info->outer_iters = outer;
      info->rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
      info->status = st;
    }
    if (st != FNPF_OK) return st;
    FNPF_PS_TRY(apply(psi, w.q));
    FNPF_PS_TRY(go<LinItem>(m.ns, {lam + NI, -1.0, w.q + NI, lam_phis}));
    FNPF_PS_TRY(go<GeomVjpItem>(m.nelem * m.n * m.nq, {m, eta, h, psi, phi, w.F}));
    FNPF_PS_TRY(go<VjpTriItem>((int64_t)m.ntri * m.nt, {m, w.F, w.se}));
    FNPF_PS_TRY(go<SurfGatherItem>(m.ns, {m.soff, m.sinc, w.se, w.be, w.bp}));
    FNPF_PS_TRY(go<InteriorItem>(m.ns, {m.ns, -1.0, w.be, lam_eta}));
    if (lam_h) FNPF_PS_TRY(go<InteriorItem>(m.ns, {m.ns, -1.0, w.bp, lam_h}));
    return FNPF_OK;
  }

  // The cotangents (gE, gP, gh) of a stage's input (E, P) and of h from those
  // (mu_e, mu_p) of its right-hand side, with the stage's solution phi_s and
  // w_s: nu = M^-1 mu (M symmetric), the conditions' products, w's product and
  // the solve's (geometry E, or still water when linear).
  fnpf_status rhs_vjp(const double* E, const double* h, const double* P, const double* phi_s, const double* w_s,
                      const double* mu_e, const double* mu_p, double* gE, double* gP, double* gh, const Params& o) {
    const int64_t ns = m.ns;
    double* S = w.aS;
    double *ne = S, *np = S + ns, *tw = S + 2 * ns, *le = S + 3 * ns, *lp = S + 4 * ns, *lh = S + 5 * ns;
    double* lphi = w.aN;
    FNPF_PS_TRY(mass_solve(mu_e, ne, o));
    FNPF_PS_TRY(mass_solve(mu_p, np, o));
    FNPF_PS_TRY(go<SurfQVjpItem>((int64_t)m.ntri * m.nq, {m, E, P, w_s, ne, np, o.g, o.linear, w.aq}));
    FNPF_PS_TRY(go<SurfNodeVjpItem>((int64_t)m.ntri * m.nt, {m, w.aq, w.se3}));
    FNPF_PS_TRY(go<SurfGather3Item>(ns, {m.soff, m.sinc, w.se3, gE, gP, tw}));
    FNPF_PS_TRY(go<FillItem>(ns, {0.0, gh}));
    const double* geo = o.linear ? w.zero : E;
    FNPF_PS_TRY(go<FillItem>(m.N, {0.0, lphi}));
    FNPF_PS_TRY(go<WVjpItem>(ns, {m, geo, h, w_s, tw, lphi, o.linear ? nullptr : gE, gh}));
    FNPF_PS_TRY(solve_vjp(geo, h, phi_s, lphi, le, lp, lh, o, nullptr));
    if (!o.linear) FNPF_PS_TRY(go<AxpyItem>(ns, {1.0, le, gE}));
    FNPF_PS_TRY(go<AxpyItem>(ns, {1.0, lp, gP}));
    return go<AxpyItem>(ns, {1.0, lh, gh});
  }

  // The adjoint of one RK4 step from (eta, phis) (the step-n state): for the
  // cotangents (lam_e, lam_p) of the step's result, the cotangents of its
  // input (out_e, out_p) and of h (out_h, may be null).  The forward stages
  // are recomputed (their states, solutions and w kept), then swept in
  // reverse: lam_k3 = dt/6 lam, lam_k2 = dt/3 lam + dt g3, lam_k1 = dt/3 lam +
  // dt/2 g2, lam_k0 = dt/6 lam + dt/2 g1 with g_s the stage-input cotangents,
  // out = lam + sum_s g_s; lam is first taken through the transposes of the
  // modal filter (FilterTSlotItem, FilterTGatherItem) and of the relaxation
  // blend (RelaxVjpItem) when these are set, in the reverse of their order.
  fnpf_status rk4_adjoint(const double* h, const double* eta, const double* phis, double t, double dt,
                          const double* lam_e_in, const double* lam_p_in, double* out_e, double* out_p,
                          double* out_h, const Params& o) {
    const int64_t ns = m.ns, N = m.N;
    double* S = w.aS;
    auto st_e = [&](int s) { return S + (6 + 2 * s) * ns; };
    auto st_p = [&](int s) { return S + (7 + 2 * s) * ns; };
    auto ws = [&](int s) { return S + (14 + s) * ns; };
    auto phs = [&](int s) { return w.aN + (1 + s) * N; };
    double *lk_e = S + 18 * ns, *lk_p = S + 19 * ns, *acc_e = S + 20 * ns, *acc_p = S + 21 * ns;
    double *acc_h = S + 22 * ns, *gE = S + 23 * ns, *gP = S + 24 * ns, *gh = S + 25 * ns;
    double *rl_e = S + 26 * ns, *rl_p = S + 27 * ns, *rl_h = S + 28 * ns, *fl_e = S + 29 * ns, *fl_p = S + 30 * ns;
    const double* lam_e = lam_e_in;
    const double* lam_p = lam_p_in;
    if (m.filt) {   // the cotangents of the state before the filter
      const int64_t slots = (int64_t)m.ntri * m.nt;
      FNPF_PS_TRY(go<FilterTSlotItem>(slots, {m, lam_e_in, w.ft}));
      FNPF_PS_TRY(go<FilterTGatherItem>(ns, {m, lam_e_in, w.ft, fl_e}));
      FNPF_PS_TRY(go<FilterTSlotItem>(slots, {m, lam_p_in, w.ft}));
      FNPF_PS_TRY(go<FilterTGatherItem>(ns, {m, lam_p_in, w.ft, fl_p}));
      lam_e = fl_e;
      lam_p = fl_p;
    }
    if (m.rcr) {   // the cotangents of the state before the blend
      FNPF_PS_TRY(go<RelaxVjpItem>(ns, {m, h, t + dt, o.g, lam_e, lam_p, rl_e, rl_p, rl_h}));
      lam_e = rl_e;
      lam_p = rl_p;
    }
    // forward recompute of the stages
    for (int s = 0; s < 4; ++s) {
      if (s == 0) {
        FNPF_PS_TRY(go<CopyItem>(ns, {eta, st_e(0)}));
        FNPF_PS_TRY(go<CopyItem>(ns, {phis, st_p(0)}));
      } else {
        const double c = (s == 3 ? 1.0 : 0.5) * dt;
        FNPF_PS_TRY(go<LinItem>(ns, {eta, c, w.ke, st_e(s)}));
        FNPF_PS_TRY(go<LinItem>(ns, {phis, c, w.kp, st_p(s)}));
      }
      FNPF_PS_TRY(rhs(st_e(s), h, st_p(s), w.ke, w.kp, o, nullptr));
      FNPF_PS_TRY(go<CopyItem>(N, {w.phi, phs(s)}));
      FNPF_PS_TRY(go<CopyItem>(ns, {w.w, ws(s)}));
    }
    // reverse sweep
    FNPF_PS_TRY(go<FillItem>(ns, {0.0, acc_e}));
    FNPF_PS_TRY(go<FillItem>(ns, {0.0, acc_p}));
    if (m.rcr) FNPF_PS_TRY(go<CopyItem>(ns, {rl_h, acc_h}));
    else FNPF_PS_TRY(go<FillItem>(ns, {0.0, acc_h}));
    for (int s = 3; s >= 0; --s) {
      const double b = (s == 0 || s == 3 ? 1.0 : 2.0) * dt / 6.0;
      if (s == 3) {
        FNPF_PS_TRY(go<Lin2Item>(ns, {b, lam_e, 0.0, lam_e, lk_e}));
        FNPF_PS_TRY(go<Lin2Item>(ns, {b, lam_p, 0.0, lam_p, lk_p}));
      } else {
        const double c = (s + 1 == 3 ? 1.0 : 0.5) * dt;   // stage s + 1 reads k_s with this weight
        FNPF_PS_TRY(go<Lin2Item>(ns, {b, lam_e, c, gE, lk_e}));
        FNPF_PS_TRY(go<Lin2Item>(ns, {b, lam_p, c, gP, lk_p}));
      }
      FNPF_PS_TRY(rhs_vjp(st_e(s), h, st_p(s), phs(s), ws(s), lk_e, lk_p, gE, gP, gh, o));
      FNPF_PS_TRY(go<AxpyItem>(ns, {1.0, gE, acc_e}));
      FNPF_PS_TRY(go<AxpyItem>(ns, {1.0, gP, acc_p}));
      FNPF_PS_TRY(go<AxpyItem>(ns, {1.0, gh, acc_h}));
    }
    FNPF_PS_TRY(go<LinItem>(ns, {lam_e, 1.0, acc_e, out_e}));
    FNPF_PS_TRY(go<LinItem>(ns, {lam_p, 1.0, acc_p, out_p}));
    if (out_h) FNPF_PS_TRY(go<CopyItem>(ns, {acc_h, out_h}));
    return FNPF_OK;
  }

  // Mass M = 1^T M_s eta and energy E = 1/2 phi^T A phi + 1/2 g eta^T M_s eta of
  // (eta, phis) (host doubles): the solve into the mesh's potential and one
  // application of the stored operator (the model's geometry).
  fnpf_status invariants(const double* eta, const double* h, const double* phis, const Params& o, double* mass,
                         double* energy, fnpf_solve_info* info) {
    const double* geo = o.linear ? w.zero : eta;
    FNPF_PS_TRY(solve(geo, h, phis, w.phi, o, info));
    FNPF_PS_TRY(apply(w.phi, w.q));
    double kin = 0, pot = 0, tot = 0;
    FNPF_PS_TRY(dot(w.phi, w.q, m.N, &kin));
    FNPF_PS_TRY(go<CsrItem>(m.ns, {m.mrow, m.mcol, m.mval, eta, w.mq}));
    FNPF_PS_TRY(dot(eta, w.mq, m.ns, &pot));
    FNPF_PS_TRY(go<FillItem>(m.ns, {1.0, w.mr}));
    FNPF_PS_TRY(dot(w.mr, w.mq, m.ns, &tot));
    *mass = tot;
    *energy = 0.5 * kin + 0.5 * o.g * pot;
    return FNPF_OK;
  }

  // x = M^-1 b on the surface (Jacobi-PCG on the consistent mass from x = 0).
  fnpf_status mass_solve(const double* b, double* x, const Params& o) {
    const int64_t ns = m.ns;
    FNPF_PS_TRY(go<FillItem>(ns, {0.0, x}));
    double bb = 0;
    FNPF_PS_TRY(dot(b, b, ns, &bb));
    if (!(bb > 0)) return bb == 0 ? FNPF_OK : FNPF_EDIVERGED;
    const double stop = o.mass_rtol * sqrt(bb);
    FNPF_PS_TRY(go<CopyItem>(ns, {b, w.mr}));
    int it = 0;
    double rr = bb;
    return cg_run(ns, x, w.mr, w.mz, w.mp, w.mq, stop, o.mass_max_iter, 8, nullptr,
                  [&](const double* pv, double* qv) { return go<CsrItem>(ns, {m.mrow, m.mcol, m.mval, pv, qv}); },
                  [&](const double* rv, double* zv) { return go<DivItem>(ns, {rv, m.mdiag, zv}); }, &it, &rr);
  }

  // w [ns] at (eta, phis): the solve (warm-started from the mesh's potential) and w.
  fnpf_status dtn(const double* eta, const double* h, const double* phis, double* wout, const Params& o,
                  fnpf_solve_info* info) {
    FNPF_PS_TRY(solve(eta, h, phis, w.phi, o, info));
    return go<WItem>(m.ns, {m, eta, h, w.phi, wout});
  }

  // (k_eta, k_phi) = the projected free-surface conditions at (eta, phis)
  // (linear: the solve and w on the still-water geometry).
  fnpf_status rhs(const double* eta, const double* h, const double* phis, double* ke, double* kp, const Params& o,
                  fnpf_solve_info* info) {
    const double* geo = o.linear ? w.zero : eta;
    FNPF_PS_TRY(dtn(geo, h, phis, w.w, o, info));
    FNPF_PS_TRY(go<SurfQItem>((int64_t)m.ntri * m.nq, {m, eta, phis, w.w, o.g, o.linear, w.fq}));
    FNPF_PS_TRY(go<SurfNodeItem>((int64_t)m.ntri * m.nt, {m, w.fq, w.se}));
    FNPF_PS_TRY(go<SurfGatherItem>(m.ns, {m.soff, m.sinc, w.se, w.be, w.bp}));
    FNPF_PS_TRY(mass_solve(w.be, ke, o));
    return mass_solve(w.bp, kp, o);
  }

  // f [ns] in place through the modal filter (EINVAL without one).
  fnpf_status filter(double* f) {
    if (!m.filt) return FNPF_EINVAL;
    const int64_t slots = (int64_t)m.ntri * m.nt;
    FNPF_PS_TRY(go<FilterItem>(slots, {m, f, w.ft}));
    return go<FilterWriteItem>(slots, {m, w.ft, f});
  }

  // One classical RK4 step of (eta, phis) from t to t + dt in place, then the
  // relaxation zones and the modal filter (when set); info: NULL or [4].
  fnpf_status rk4(const double* h, double* eta, double* phis, double t, double dt, const Params& o,
                  fnpf_solve_info* info) {
    const int64_t ns = m.ns;
    for (int s = 0; s < 4; ++s) {
      const double* E = eta;
      const double* P = phis;
      if (s > 0) {
        const double c = (s == 3 ? 1.0 : 0.5) * dt;
        FNPF_PS_TRY(go<LinItem>(ns, {eta, c, w.ke, w.es}));
        FNPF_PS_TRY(go<LinItem>(ns, {phis, c, w.kp, w.ps}));
        E = w.es;
        P = w.ps;
      }
      reuse_lmax = s > 0;   // the Chebyshev intervals of the step's first stage serve all four
      const fnpf_status sr = rhs(E, h, P, w.ke, w.kp, o, info ? info + s : nullptr);
      reuse_lmax = false;
      FNPF_PS_TRY(sr);
      if (s == 0) {
        FNPF_PS_TRY(go<CopyItem>(ns, {w.ke, w.ae}));
        FNPF_PS_TRY(go<CopyItem>(ns, {w.kp, w.ap}));
      } else {
        const double wgt = s == 3 ? 1.0 : 2.0;
        FNPF_PS_TRY(go<AxpyItem>(ns, {wgt, w.ke, w.ae}));
        FNPF_PS_TRY(go<AxpyItem>(ns, {wgt, w.kp, w.ap}));
      }
    }
    FNPF_PS_TRY(go<AxpyItem>(ns, {dt / 6.0, w.ae, eta}));
    FNPF_PS_TRY(go<AxpyItem>(ns, {dt / 6.0, w.ap, phis}));
    if (m.rcr) FNPF_PS_TRY(go<RelaxItem>(ns, {m, h, t + dt, o.g, eta, phis}));
    if (!m.filt) return FNPF_OK;
    FNPF_PS_TRY(filter(eta));
    return filter(phis);
  }
};

#undef FNPF_PS_TRY

}  // namespace pstep
}  // namespace fnpf

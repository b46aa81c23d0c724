// Conserved quantities of the free-surface state (fnpf_invariants): the
// mass M = sum_c W_c eta_c and the energy
//     E = 1/2 phi^T A(eta) phi + 1/2 g sum_c W_c eta_c^2     (unit density)
// where W_c is the lumped GLL surface mass of node column c (the diagonal
// mass of the free-surface weak forms, Sec. 3.1.1, Eq. free_surface_weak,
// with GLL quadrature at the nodes), phi the potential of the Laplace problem
// with phi = phi_eta on the surface (Sec. 2) and A(eta) the stiffness matrix
// of the weak Laplace form (Eq. Laplace_weak).  Kinetic energy 1/2 int |grad
// phi|^2 dV = 1/2 phi^T A phi exactly for the discrete potential; the
// potential energy is the GLL-lumped 1/2 g int eta^2 dA.
#include "mesh.cuh"
#include "vec.cuh"

namespace {

namespace vec = fnpf::vec;
using fnpf::Blk;
using fnpf::launch;

// Per-block partials of (phi . y, sum eta / minv, sum eta^2 / minv) into
// part[slot * blocks + block].
struct invariant_partials_kernel {
  static constexpr int kThreads = fnpf::vec::NT;
  __device__ static void run(Blk bk, int64_t n, const double* phi, const double* y, int ns, const double* eta,
                             const double* minv, double* part) {
    __shared__ double sh[fnpf::vec::kShared];
    double a = 0, b = 0, c = 0;
    FNPF_GRID_LOOP(i, n) a += phi[i] * y[i];
    FNPF_GRID_LOOP(i, (int64_t)ns) {
      const double w = 1.0 / minv[i];
      b += w * eta[i];
      c += w * eta[i] * eta[i];
    }
    a = fnpf::vec::block_sum(a, sh);
    b = fnpf::vec::block_sum(b, sh);
    c = fnpf::vec::block_sum(c, sh);
    if (threadIdx.x == 0) {
      part[bk.x] = a;
      part[bk.nx + bk.x] = b;
      part[2 * bk.nx + bk.x] = c;
    }
  }
};

// One block: the three sums over the partials in a fixed order, then
// out = (mass, energy).
struct invariant_finish_kernel {
  static constexpr int kThreads = fnpf::vec::NT;
  __device__ static void run(Blk bk, const double* part, int nb, double g, double* out) {
    __shared__ double sh[fnpf::vec::kShared];
    const double a = fnpf::vec::reduce_partials(part, nb, sh);
    const double b = fnpf::vec::reduce_partials(part + nb, nb, sh);
    const double c = fnpf::vec::reduce_partials(part + 2 * nb, nb, sh);
    if (threadIdx.x == 0) {
      out[0] = b;
      out[1] = 0.5 * a + 0.5 * g * c;
    }
  }
};

fnpf_status fail(fnpf_mesh* m, cudaError_t e, const char* what) {
  m->err = std::string("invariants: ") + what + ": " + cudaGetErrorString(e);
  return FNPF_ECUDA;
}

}  // namespace

extern "C" fnpf_status fnpf_invariants(fnpf_mesh* m, const double* eta, const double* phis, double* mass,
                                       double* energy, fnpf_solve_info* info, void* stream) {
  if (!m || !eta || !phis || !mass || !energy) return FNPF_EINVAL;
  const fnpf::Geom& g = m->g;
  cudaStream_t s = (cudaStream_t)stream;
  if (!m->inv_work) {
    cudaError_t e = cudaMalloc((void**)&m->inv_work, (size_t)g.N * sizeof(double));
    if (e != cudaSuccess) {
      m->inv_work = nullptr;
      m->err = "invariants: device allocation failed";
      return FNPF_ENOMEM;
    }
  }
  // phi: the Laplace solve of the mesh's solver into the mesh-owned potential
  fnpf_status st = fnpf_laplace_solve(m, eta, phis, m->phi, info, stream);
  if (st != FNPF_OK) return st;
  double* y = m->inv_work;
  const double* geta = m->geom_eta(eta);
  cudaError_t e = fnpf::launch_apply<double>(g, m->tables(), geta, m->phi, m->phi + g.NI, y, y + g.NI, m->ring,
                                             m->variant64, s);
  if (e != cudaSuccess) return fail(m, e, "operator");
  const int nb = fnpf::kVecBlocks;
  launch<invariant_partials_kernel>(nb, fnpf::vec::NT, 0, s, g.N, m->phi, y, g.ns, eta, m->dminv, m->partials);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(m, e, "partials");
  double* out = m->partials + 3 * nb;
  launch<invariant_finish_kernel>(1, fnpf::vec::NT, 0, s, m->partials, nb, g.g, out);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(m, e, "finish");
  m->launches += 4;
  double host[2];
  if ((e = cudaMemcpyAsync(host, out, sizeof(host), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(m, e, "read back");
  *mass = host[0];
  *energy = host[1];
  return FNPF_OK;
}

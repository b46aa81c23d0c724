// The opaque fnpf_mesh of the C ABI: sizes, tables, workspaces.
#pragma once

#include <string>
#include <vector>

#include "fnpf_internal.cuh"
#include "mg.cuh"

// One captured CUDA graph and the pointers it was captured with.
struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  const void* key[2] = {nullptr, nullptr};
};

struct fnpf_mesh {
  fnpf::Geom g{};
  fnpf_opts opts{};
  std::string err;
  int device = 0;
  int variant64 = 1;                // elements-per-CTA shape of the FP64 operator kernel
  int variant32 = 1;                // ... of the FP32 operator kernel
  bool tuned = false;               // shapes chosen by the autotuner
  template <typename T>
  int variant() const { return sizeof(T) == 4 ? variant32 : variant64; }

  // host copies
  std::vector<double> xi, w, D;     // GLL tables
  std::vector<double> hm;           // horizontal metric [5][n_ecol * lines]
  std::vector<double> h, minv;      // depth, inverse lumped mass [ns]
  std::vector<double> xs, ys;       // surface coordinates [ns]

  // device tables (double)
  double* dD = nullptr;
  double* dxi = nullptr;
  double* dw = nullptr;
  double* dhm = nullptr;
  double* dh = nullptr;
  double* dminv = nullptr;

  // workspaces (double)
  double* ring = nullptr;           // nv * n_ecol * ring
  double* r = nullptr;              // NI each
  double* z = nullptr;
  double* p = nullptr;
  double* q = nullptr;
  double* dinv = nullptr;
  double* phi = nullptr;            // N: potential kept between solves (warm start)
  double* partials = nullptr;       // 4 * kVecBlocks
  fnpf::CgScalars* sc = nullptr;    // device scalars
  fnpf::CgScalars* sc_host = nullptr;  // pinned mirror
  double* s_eta[2] = {nullptr, nullptr};  // RK4 stage states
  double* s_phi[2] = {nullptr, nullptr};
  double* acc_eta = nullptr;
  double* acc_phi = nullptr;

  // mixed precision: FP32 tables and inner-solve vectors, FP64 right-hand side
  float* fD = nullptr;
  float* fxi = nullptr;
  float* fw = nullptr;
  float* fhm = nullptr;
  float* fh = nullptr;
  float* eta32 = nullptr;           // ns
  float* r32 = nullptr;             // NI each
  float* z32 = nullptr;
  float* p32 = nullptr;
  float* q32 = nullptr;
  float* e32 = nullptr;
  float* dinv32 = nullptr;
  double* b = nullptr;              // NI: lifted right-hand side
  double* eta64 = nullptr;          // ns: copy of the solve's eta
  double* zero_eta = nullptr;       // ns zeros: the geometry of FNPF_LINEAR
  double* G64 = nullptr;            // stored metric of FP64 solves (allocated at the first one)
  bool g64_active = false;          // the current FP64 solve reads G64
  fnpf::CgScalars* sc_in = nullptr; // inner-solve scalars

  // relaxation zones (fnpf_set_relaxation)
  double* rx_cr = nullptr;          // ns
  double* rx_gen = nullptr;         // ns
  double* dxs = nullptr;            // ns surface coordinates on the device
  double* dys = nullptr;
  fnpf_relaxation relax{};          // scalar parameters (array pointers unused)
  bool relax_on = false;

  // over-integrated right-hand side (fnpf_set_dealias): Gauss points per
  // direction (0: off) and one buffer of tables, Gauss-point metric, element
  // values, right-hand side and w (dealias.cu)
  int dealias_M = 0;
  double* dl_buf = nullptr;

  // modal filter (fnpf_set_filter): the 1D matrix V diag(sigma) V^-1, [n * n]
  double* dfilter = nullptr;
  bool filter_on = false;

  // projection of the initial guess (opts.projection = L > 0; allocated at the
  // first solve): projH = [L history solutions | L operator images], [2L][NI],
  // history 0 = newest; proj_part: per-block partials of the Gram system, then
  // the coefficients
  double* projH = nullptr;
  double* projHa = nullptr;         // the same for the adjoint solves
  double* proj_part = nullptr;
  int proj_alloc = 0;               // L the buffers were sized for
  int proj_alloc_a = 0;

  // fnpf_invariants: A phi of the energy [N] (allocated at the first call)
  double* inv_work = nullptr;

  // tape of forward steps for the adjoint (fnpf_tape_begin): per slot the four
  // stage potentials [4][NI] and stage states [4][2][ns]; the slot a step
  // records into is read on the device from tape_slot_dev (graph replays)
  double* tape = nullptr;
  int tape_cap = 0;                 // slots allocated
  bool tape_on = false;
  int tape_next = 0;                // slot of the next recorded step
  int* tape_slot_dev = nullptr;
  int* tape_slot_host = nullptr;    // pinned

  // adjoint step workspaces (allocated at the first fnpf_step_adjoint)
  double* adj = nullptr;            // one block holding all of them
  size_t adj_bytes = 0;

  // p-multigrid hierarchy (created at the first FNPF_PMG solve)
  fnpf::Mg* mg = nullptr;
  bool cheb_valid[2] = {false, false};   // Chebyshev intervals estimated (FP64, FP32)
  // FNPF_LINEAR: the solver set-up for the fixed still-water geometry (stored
  // metric, diagonals, multigrid levels, Chebyshev intervals) is done (FP64,
  // FP32) and is reused by later solves
  bool lpf_ready[2] = {false, false};
  int64_t solve_count[2] = {0, 0};
  bool iso = false;
  double Lx = 0, Ly = 0;
  std::vector<double> Xs, Ys;       // surface-node coordinates of an isoparametric mesh
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // CUDA graphs of the CG iteration (0: FP64, 1: FP32), captured on gstream
  cudaStream_t gstream = nullptr;
  GraphSlot g_iter[2];
  cudaStream_t bstream[2] = {nullptr, nullptr};   // capture streams of nested loop bodies
  int* inner_total = nullptr;                     // device: inner iterations of a mixed solve
  fnpf::StageInfo* stage_info = nullptr;          // device [4]
  fnpf::StageInfo* stage_info_host = nullptr;     // pinned [4]
  double* t_dev = nullptr;                        // device time of the step graph
  double* t_host = nullptr;                       // pinned
  cudaGraphExec_t step_exec = nullptr;            // captured RK4 step
  const void* step_key[2] = {nullptr, nullptr};
  double step_dt = 0.0;
  bool warm = false;                              // a host-driven step has run
  int64_t step_kernels = 0;                       // top-level kernel nodes of the step graph
  int64_t body_kernels[2] = {0, 0};               // kernel nodes of a loop body (outer / inner)

  // instrumentation
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // pairs (start, stop) of operator applications
  std::vector<int> prof_it;          // CG iteration of each recorded pair
  std::vector<char> prof_fp32;       // pair timed an FP32 application
  double prof_ms32 = 0.0;
  int64_t prof_count32 = 0;
  int prof_used = 0;                 // pairs recorded since the last host sync
  double prof_ms = 0.0;
  int64_t prof_count = 0;
  int64_t launches = 0;

  fnpf::Tables<double> tables() const { return fnpf::Tables<double>{dD, dxi, dw, dhm, dh, dminv}; }
  bool linear() const { return opts.model == FNPF_LINEAR; }
  // eta as the mesh geometry sees it: the state's eta, or zero for FNPF_LINEAR
  const double* geom_eta(const double* eta) const { return linear() ? zero_eta : eta; }
  fnpf::Tables<float> tables32() const { return fnpf::Tables<float>{fD, fxi, fw, fhm, fh, nullptr}; }
};

namespace fnpf {
// Times every elements-per-CTA shape of the FP64 and FP32 operator on this mesh
// (eta given in FP64; the FP64 timing uses the stored metric G when given) and
// keeps the fastest of each; synchronises the stream.
fnpf_status autotune(fnpf_mesh* m, const double* eta, const double* G, cudaStream_t s);
// Accumulates the recorded event pairs (call after a host sync of the stream).
void prof_collect(fnpf_mesh* m, int iters_done);
void graph_reset(GraphSlot* g);
// Captured RK4 steps (api.cu).
cudaError_t enqueue_step(fnpf_mesh* m, double* eta, double* phis, double dt, cudaStream_t s);
cudaError_t enqueue_filter_step(fnpf_mesh* m, double* eta, double* phis, cudaStream_t s);
fnpf_status read_step_info(fnpf_mesh* m, fnpf_solve_info* info, float ms, bool count = true);
bool graph_mode(const fnpf_mesh* m);
int64_t graph_kernel_nodes(cudaGraph_t g);
// Device-driven solve for graph capture (see cg.cu).
cudaError_t enqueue_solve_device(fnpf_mesh* m, const double* eta_in, const double* phis, double* x,
                                 StageInfo* info_dev, cudaStream_t s, bool estimate);
// Tape recording of stage st (potential m->phi and stage state ce, cp) into the
// slot *m->tape_slot_dev (adj.cu).
cudaError_t enqueue_tape_record(fnpf_mesh* m, int st, const double* ce, const double* cp, cudaStream_t s);
// Over-integrated Zakharov right-hand side of (eta, phis) into dealias_rhs(m)
// (w given, or recovered from m->phi when NULL) -- dealias.cu.
cudaError_t enqueue_dealias_rhs(fnpf_mesh* m, const double* eta, const double* phis, const double* w,
                                cudaStream_t s);
const double* dealias_rhs(const fnpf_mesh* m);
// CG solve of A_II x = -A_IS phis for the interior part x [NI] (in: initial guess),
// or of A_II x = rhs when rhs [NI] is given (phis is then unused).
fnpf_status cg_solve(fnpf_mesh* m, const double* eta, const double* phis, double* x, fnpf_solve_info* info,
                     cudaStream_t s, const double* rhs = nullptr);
// z = M r with the FP64 preconditioner set up from eta (fnpf_precond_apply).
fnpf_status precond_apply(fnpf_mesh* m, const double* eta, const double* r, double* z, cudaStream_t s);
}  // namespace fnpf

// Batched ensembles of independent wave tanks: one CUDA graph launch advances
// every tank by one RK4 step.  Each tank's step (four device-driven Laplace
// solves whose CG loops are conditional WHILE nodes, stage kernels,
// relaxation) is captured as one branch of a fork/join graph, so tanks with
// different sizes and orders run concurrently and the host synchronises once
// per ensemble step.  Tanks keep their own meshes, options, autotuned kernel
// shapes and multigrid hierarchies.
#include <vector>

#include "mesh.cuh"

struct fnpf_ensemble {
  std::vector<fnpf_mesh*> meshes;
  cudaStream_t main = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;   // eta, phis per tank
  std::vector<double> dts;
  std::string err;
};

namespace {
std::string g_ens_error;

void reset_graph(fnpf_ensemble* en) {
  if (en->exec) cudaGraphExecDestroy(en->exec);
  en->exec = nullptr;
}

cudaError_t capture(fnpf_ensemble* en, double* const* etas, double* const* phiss, const double* dts) {
  reset_graph(en);
  const int n = (int)en->meshes.size();
  cudaError_t e = cudaStreamBeginCapture(en->main, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t eb = cudaEventRecord(en->fork, en->main);
  for (int i = 0; i < n && eb == cudaSuccess; ++i) {
    fnpf_mesh* m = en->meshes[i];
    eb = cudaStreamWaitEvent(m->gstream, en->fork, 0);
    if (eb == cudaSuccess) eb = fnpf::enqueue_step(m, etas[i], phiss[i], dts[i], m->gstream);
    if (eb == cudaSuccess) eb = cudaEventRecord(en->join[i], m->gstream);
    if (eb == cudaSuccess) eb = cudaStreamWaitEvent(en->main, en->join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(en->main, &graph);
  if (eb != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return eb;
  }
  if (e != cudaSuccess) return e;
  for (int i = 0; i < n; ++i) en->meshes[i]->step_kernels = 0;
  int64_t top = fnpf::graph_kernel_nodes(graph);
  e = cudaGraphInstantiate(&en->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  // attribute the top-level kernels evenly for the launch counter
  for (int i = 0; i < n; ++i) en->meshes[i]->step_kernels = top / n + (i < top % n ? 1 : 0);
  for (int i = 0; i < n; ++i) {
    en->key[2 * i] = etas[i];
    en->key[2 * i + 1] = phiss[i];
    en->dts[i] = dts[i];
  }
  return cudaSuccess;
}

bool keys_match(const fnpf_ensemble* en, double* const* etas, double* const* phiss, const double* dts) {
  for (size_t i = 0; i < en->meshes.size(); ++i)
    if (en->key[2 * i] != etas[i] || en->key[2 * i + 1] != phiss[i] || en->dts[i] != dts[i]) return false;
  return true;
}
}  // namespace

extern "C" {

fnpf_status fnpf_ensemble_create(fnpf_mesh* const* meshes, int n, fnpf_ensemble** out) {
  if (!out || !meshes || n < 1) return FNPF_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!meshes[i]) return FNPF_EINVAL;
  fnpf_ensemble* en = new fnpf_ensemble();
  en->meshes.assign(meshes, meshes + n);
  en->join.assign(n, nullptr);
  en->key.assign(2 * n, nullptr);
  en->dts.assign(n, 0.0);
  cudaError_t e = cudaStreamCreateWithFlags(&en->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&en->fork, cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&en->join[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    g_ens_error = cudaGetErrorString(e);
    fnpf_ensemble_destroy(en);
    return FNPF_ECUDA;
  }
  *out = en;
  return FNPF_OK;
}

void fnpf_ensemble_destroy(fnpf_ensemble* en) {
  if (!en) return;
  reset_graph(en);
  for (cudaEvent_t ev : en->join)
    if (ev) cudaEventDestroy(ev);
  if (en->fork) cudaEventDestroy(en->fork);
  if (en->main) cudaStreamDestroy(en->main);
  delete en;
}

fnpf_status fnpf_ensemble_rk4_step(fnpf_ensemble* en, double* const* etas, double* const* phiss, const double* ts,
                                   const double* dts, fnpf_solve_info* info, void* stream) {
  if (!en || !etas || !phiss || !ts || !dts) return FNPF_EINVAL;
  const int n = (int)en->meshes.size();
  for (int i = 0; i < n; ++i)
    if (!etas[i] || !phiss[i] || !(dts[i] > 0)) return FNPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  bool warm = true;
  for (fnpf_mesh* m : en->meshes) warm = warm && fnpf::graph_mode(m);
  if (!warm) {
    // first step: each tank once on its own (lazy set-up, autotuning, multigrid)
    for (int i = 0; i < n; ++i) {
      fnpf_status st = fnpf_rk4_step(en->meshes[i], etas[i], phiss[i], ts[i], dts[i], info ? info + 4 * i : nullptr,
                                     stream);
      if (st != FNPF_OK) {
        en->err = "tank " + std::to_string(i) + ": " + en->meshes[i]->err;
        return st;
      }
    }
    return FNPF_OK;
  }
  cudaError_t e = cudaSuccess;
  if (!en->exec || !keys_match(en, etas, phiss, dts)) e = capture(en, etas, phiss, dts);
  if (e != cudaSuccess) {
    en->err = std::string("ensemble capture: ") + cudaGetErrorString(e);
    return FNPF_ECUDA;
  }
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    fnpf_mesh* m = en->meshes[i];
    *m->t_host = ts[i];
    e = cudaMemcpyAsync(m->t_dev, m->t_host, sizeof(double), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(en->exec, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    en->err = std::string("ensemble step: ") + cudaGetErrorString(e);
    return FNPF_ECUDA;
  }
  fnpf_status result = FNPF_OK;
  for (int i = 0; i < n; ++i) {
    fnpf_status st = fnpf::read_step_info(en->meshes[i], info ? info + 4 * i : nullptr, 0.0f);
    if (st != FNPF_OK && result == FNPF_OK) {
      result = st;
      en->err = "tank " + std::to_string(i) + ": " + en->meshes[i]->err;
    }
  }
  return result;
}

const char* fnpf_ensemble_last_error(const fnpf_ensemble* en) { return en ? en->err.c_str() : g_ens_error.c_str(); }

}  // extern "C"

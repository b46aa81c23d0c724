// Batched ensembles of independent wave tanks: one CUDA graph launch advances
// every tank by one RK4 step.
//
// Batched groups.  The RK4 step of a warm tank is a fixed sequence of kernel
// launches and device-driven loops (four solves whose CG and defect-correction
// loops are conditional WHILE nodes, stage kernels, relaxation).  At capture
// the ensemble records that sequence for every tank (launch.cuh: the host code
// of the step runs with a Recorder active, under a throw-away stream capture
// that must stay empty), and tanks whose records agree operation by operation
// -- same kernels and block shapes, same loop structure; in practice the tanks
// of one order with the same options -- form a group.  A group's step is the
// record replayed once: each kernel becomes one batched launch (k_many) over
// the concatenated grids of all its tanks (their arguments in the launch's
// parameters), each loop one WHILE node that runs while any tank's loop runs,
// with a per-tank gate so that a tank whose loop has finished does no work in
// it (every tank executes exactly the operations of its own step, so the
// results equal the single-tank step bit for bit).
// The tanks of a group share the kernel shapes the autotuner chose for the
// largest of them.  Groups (of up to kMaxBatch tanks), and tanks that cannot
// be recorded (adjoint tape, over-integration), run as concurrent fork/join
// branches of one graph.
#include <stdint.h>

#include <algorithm>
#include <map>
#include <vector>

#include "graphs.cuh"
#include "mesh.cuh"

namespace {

// Loop condition of a batched loop: tank t continues while its own condition
// holds and the enclosing loop's gate lets it run; the graph loop continues
// while any tank does.
struct BatchCond {
  const fnpf::CgScalars* sc[fnpf::kMaxBatch];
  const int* parent;   // gate of the enclosing loop (null at the top level)
  int* cond;           // [ntank] this loop's gate
  int* count;          // body executions of this loop (incremented when the loop continues)
  cudaGraphConditionalHandle h;
  int ntank, cap, use_outer;
};

__global__ void __launch_bounds__(fnpf::kMaxBatch) batch_cond_kernel(const __grid_constant__ BatchCond c) {
  const int t = threadIdx.x;
  int v = 0;
  if (t < c.ntank) {
    const fnpf::CgScalars* sc = c.sc[t];
    const int cnt = c.use_outer ? sc->outer : sc->iters;
    v = ((!c.parent || c.parent[t]) && !sc->done && cnt < c.cap) ? 1 : 0;
    c.cond[t] = v;
  }
  const int any = __syncthreads_or(v);
  if (t == 0) {
    cudaGraphSetConditional(c.h, any ? 1u : 0u);
    if (any) *c.count += 1;
  }
}

struct Group {
  std::vector<int> tanks;                  // ensemble indices
  std::vector<fnpf::Recorder> rec;         // aligned records, one per tank
  unsigned char* arena = nullptr;          // device: loop gates and loop counters
  std::vector<size_t> gate_off;            // per loop handle: its gate [ntank]
  size_t count_off = 0;                    // loop counters [handles]
  int handles = 0;
  int* counts_host = nullptr;              // pinned copy of the loop counters after a step
  std::vector<int64_t> body_kernels;       // per handle: kernel nodes of its body
  std::vector<cudaGraphConditionalHandle> real;
  int64_t top_kernels = 0;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> body;          // capture streams of nested bodies
  cudaEvent_t join = nullptr;
};

void free_group(Group* g) {
  if (g->arena) cudaFree(g->arena);
  if (g->counts_host) cudaFreeHost(g->counts_host);
  if (g->stream) cudaStreamDestroy(g->stream);
  for (cudaStream_t s : g->body)
    if (s) cudaStreamDestroy(s);
  if (g->join) cudaEventDestroy(g->join);
  *g = Group();
}

}  // namespace

struct fnpf_ensemble {
  std::vector<fnpf_mesh*> meshes;
  cudaStream_t main = nullptr;
  cudaStream_t scratch = nullptr;          // throw-away captures while recording
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;   // eta, phis per tank
  std::vector<double> dts;
  std::vector<Group> groups;
  std::vector<int> solo;          // tanks stepped as their own branch
  bool batching = true;
  int max_tanks = fnpf::kMaxBatch;        // tanks per batched group
  int64_t max_dof = INT64_MAX;            // DOF per batched group
  int64_t last_kernels = 0;
  std::string err;
};

namespace {
std::string g_ens_error;

void reset_graph(fnpf_ensemble* en) {
  if (en->exec) cudaGraphExecDestroy(en->exec);
  en->exec = nullptr;
  for (Group& g : en->groups) free_group(&g);
  en->groups.clear();
  en->solo.clear();
}

// Records tank m's RK4 step; false when the step cannot be recorded (an
// operation without a recorded form, which would have landed in the scratch
// capture) or recording failed.
bool record_step(fnpf_ensemble* en, fnpf_mesh* m, double* eta, double* phis, double dt, fnpf::Recorder* rec) {
  if (cudaStreamBeginCapture(en->scratch, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  const int64_t launches = m->launches;   // the host code counts what it enqueues; nothing ran
  fnpf::active_recorder() = rec;
  const cudaError_t e = fnpf::enqueue_step(m, eta, phis, dt, en->scratch);
  fnpf::active_recorder() = nullptr;
  m->launches = launches;
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(en->scratch, &graph);
  size_t nodes = 1;
  if (graph) {
    if (cudaGraphGetNodes(graph, nullptr, &nodes) != cudaSuccess) nodes = 1;
    cudaGraphDestroy(graph);
  }
  (void)cudaGetLastError();
  if (e != cudaSuccess || e2 != cudaSuccess || nodes != 0) return false;
  int depth = 0;
  for (const fnpf::Op& op : rec->ops) {
    if (op.kind == fnpf::OP_LOOP) ++depth;
    if (op.kind == fnpf::OP_END && --depth < 0) return false;
    if (op.kind == fnpf::OP_COPY_D2H && depth > 0) return false;
    if (op.kind == fnpf::OP_KERNEL && (op.grid.z != 1 || op.block.y != 1 || op.block.z != 1)) return false;
  }
  return depth == 0;
}

// The operations a batched replay needs equal across tanks.
std::vector<uint64_t> signature(const fnpf::Recorder& r) {
  std::vector<uint64_t> s;
  s.reserve(4 * r.ops.size() + 1);
  s.push_back((uint64_t)r.handles);
  for (const fnpf::Op& op : r.ops) {
    s.push_back((uint64_t)op.kind);
    if (op.kind == fnpf::OP_KERNEL) {
      s.push_back((uint64_t)(uintptr_t)op.id);
      s.push_back(op.flex ? 0 : ((uint64_t)op.block.x << 32 | (uint64_t)op.smem));
      s.push_back((uint64_t)op.args.size());
    } else if (op.kind == fnpf::OP_COPY_D2H) {
      s.push_back((uint64_t)op.bytes);
    } else {
      s.push_back((uint64_t)(uint32_t)op.handle << 32 | (uint64_t)(uint32_t)op.cap << 1 | (uint64_t)op.use_outer);
    }
  }
  return s;
}

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Allocates a group's loop gates and counters and its streams (before the
// capture).
cudaError_t prepare_group(Group* G) {
  const int T = (int)G->tanks.size();
  const std::vector<fnpf::Op>& ops = G->rec[0].ops;
  G->handles = G->rec[0].handles;
  size_t off = 0;
  G->gate_off.assign(G->handles, 0);
  for (int h = 0; h < G->handles; ++h) {
    G->gate_off[h] = off;
    off = align16(off + (size_t)T * sizeof(int));
  }
  G->count_off = off;
  off = align16(off + (size_t)std::max(1, G->handles) * sizeof(int));
  cudaError_t e = cudaMalloc(&G->arena, off);
  if (e == cudaSuccess) e = cudaMemset(G->arena, 0, off);
  if (e == cudaSuccess) e = cudaMallocHost(&G->counts_host, (size_t)std::max(1, G->handles) * sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking);
  int depth = 0, maxd = 0;
  for (const fnpf::Op& op : ops) {
    if (op.kind == fnpf::OP_LOOP) maxd = std::max(maxd, ++depth);
    if (op.kind == fnpf::OP_END) --depth;
  }
  G->body.assign(maxd, nullptr);
  for (int d = 0; d < maxd && e == cudaSuccess; ++d) e = cudaStreamCreateWithFlags(&G->body[d], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->join, cudaEventDisableTiming);
  G->body_kernels.assign(G->handles, 0);
  G->real.assign(G->handles, 0);
  return e;
}

int* gate_of(Group* G, int h) { return reinterpret_cast<int*>(G->arena + G->gate_off[h]); }

// Emits operations [i0, i1) of the group's record on the capturing stream s,
// gated by `gate`; *kernels counts the kernel nodes emitted at this level.
cudaError_t emit_range(Group* G, size_t i0, size_t i1, cudaStream_t s, int depth, const int* gate,
                       int64_t* kernels) {
  const int T = (int)G->tanks.size();
  const std::vector<fnpf::Op>& ops = G->rec[0].ops;
  for (size_t i = i0; i < i1; ++i) {
    const fnpf::Op& op = ops[i];
    cudaError_t e = cudaSuccess;
    if (op.kind == fnpf::OP_KERNEL) {
      int off[fnpf::kMaxBatch + 1], gx[fnpf::kMaxBatch];
      const unsigned char* args[fnpf::kMaxBatch];
      int64_t total = 0;
      unsigned threads = 0;
      size_t smem = 0;
      for (int t = 0; t < T; ++t) {
        const fnpf::Op& o = G->rec[t].ops[i];
        off[t] = (int)total;
        gx[t] = (int)std::max(1u, o.grid.x);
        args[t] = o.args.data();
        total += (int64_t)o.grid.x * o.grid.y;
        threads = std::max(threads, o.block.x);
        smem = std::max(smem, o.smem);
      }
      if (total >= (int64_t)1 << 31) return cudaErrorInvalidConfiguration;
      off[T] = (int)total;
      if (total == 0) continue;
      e = op.emit(gate, T, off, gx, args, (unsigned)total, threads, smem, s);
      ++*kernels;
    } else if (op.kind == fnpf::OP_COPY_D2H) {
      for (int t = 0; t < T && e == cudaSuccess; ++t) {
        const fnpf::Op& o = G->rec[t].ops[i];
        e = cudaMemcpyAsync(o.dst, o.src, o.bytes, cudaMemcpyDeviceToHost, s);
      }
    } else if (op.kind == fnpf::OP_HANDLE) {
      e = fnpf::new_handle(s, &G->real[op.handle]);
    } else if (op.kind == fnpf::OP_COND) {
      BatchCond c{};
      for (int t = 0; t < T; ++t) c.sc[t] = static_cast<const fnpf::CgScalars*>(G->rec[t].ops[i].sc);
      c.parent = gate;
      c.cond = gate_of(G, op.handle);
      c.count = reinterpret_cast<int*>(G->arena + G->count_off) + op.handle;
      c.h = G->real[op.handle];
      c.ntank = T;
      c.cap = op.cap;
      c.use_outer = op.use_outer;
      batch_cond_kernel<<<1, fnpf::kMaxBatch, 0, s>>>(c);
      e = cudaPeekAtLastError();
      ++*kernels;
    } else if (op.kind == fnpf::OP_LOOP) {
      size_t j = i + 1;
      for (int d = 1; j < i1; ++j) {
        if (ops[j].kind == fnpf::OP_LOOP) ++d;
        if (ops[j].kind == fnpf::OP_END && --d == 0) break;
      }
      const int hd = op.handle;
      e = fnpf::capture_while(s, G->body[depth], G->real[hd], &G->body_kernels[hd], [&](cudaStream_t bs) {
        int64_t inner = 0;
        return emit_range(G, i + 1, j, bs, depth + 1, gate_of(G, hd), &inner);
      });
      i = j;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Records every tank, forms the groups and prepares them; tanks that cannot
// be recorded (or all tanks, with batching off) are stepped on their own.
cudaError_t plan(fnpf_ensemble* en, double* const* etas, double* const* phiss, const double* dts) {
  const int n = (int)en->meshes.size();
  if (!en->batching) {
    for (int i = 0; i < n; ++i) en->solo.push_back(i);
    return cudaSuccess;
  }
  // tanks of one order and dimension share the shapes of the largest of them
  std::map<std::pair<int, int>, int> largest;
  for (int i = 0; i < n; ++i) {
    const fnpf_mesh* m = en->meshes[i];
    auto key = std::make_pair(m->g.n, m->g.dim);
    auto it = largest.find(key);
    if (it == largest.end() || en->meshes[it->second]->g.N < m->g.N) largest[key] = i;
  }
  for (int i = 0; i < n; ++i) {
    fnpf_mesh* m = en->meshes[i];
    const fnpf_mesh* L = en->meshes[largest[std::make_pair(m->g.n, m->g.dim)]];
    if (m->variant64 != L->variant64 || m->variant32 != L->variant32) {
      const fnpf_status st = fnpf_set_shapes(m, L->variant64, L->variant32);
      if (st != FNPF_OK) return cudaErrorInvalidValue;
    }
  }
  std::vector<fnpf::Recorder> recs(n);
  std::vector<bool> ok(n, false);
  for (int i = 0; i < n; ++i) ok[i] = record_step(en, en->meshes[i], etas[i], phiss[i], dts[i], &recs[i]);
  std::map<std::vector<uint64_t>, std::vector<int>> by_sig;
  for (int i = 0; i < n; ++i) {
    if (ok[i]) by_sig[signature(recs[i])].push_back(i);
    else en->solo.push_back(i);
  }
  // within a class, tanks in increasing size fill groups up to the tank and
  // DOF limits; a group of one runs as its own branch
  for (auto& kv : by_sig) {
    std::vector<int> idx = kv.second;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return en->meshes[a]->g.N < en->meshes[b]->g.N; });
    size_t a = 0;
    while (a < idx.size()) {
      size_t b = a;
      int64_t dof = 0;
      while (b < idx.size() && (int)(b - a) < en->max_tanks &&
             (b == a || dof + en->meshes[idx[b]]->g.N <= en->max_dof)) {
        dof += en->meshes[idx[b]]->g.N;
        ++b;
      }
      if (b - a == 1) {
        en->solo.push_back(idx[a]);
      } else {
        Group G;
        for (size_t k = a; k < b; ++k) {
          G.tanks.push_back(idx[k]);
          G.rec.push_back(std::move(recs[idx[k]]));
        }
        en->groups.push_back(std::move(G));
        const cudaError_t e = prepare_group(&en->groups.back());
        if (e != cudaSuccess) return e;
      }
      a = b;
    }
  }
  return cudaSuccess;
}

cudaError_t capture(fnpf_ensemble* en, double* const* etas, double* const* phiss, const double* dts) {
  reset_graph(en);
  cudaError_t e = plan(en, etas, phiss, dts);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(en->main, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t eb = cudaEventRecord(en->fork, en->main);
  for (Group& G : en->groups) {
    if (eb != cudaSuccess) break;
    G.top_kernels = 0;
    eb = cudaStreamWaitEvent(G.stream, en->fork, 0);
    if (eb == cudaSuccess)
      eb = cudaMemsetAsync(G.arena + G.count_off, 0, (size_t)std::max(1, G.handles) * sizeof(int), G.stream);
    if (eb == cudaSuccess) eb = emit_range(&G, 0, G.rec[0].ops.size(), G.stream, 0, nullptr, &G.top_kernels);
    if (eb == cudaSuccess)
      eb = cudaMemcpyAsync(G.counts_host, G.arena + G.count_off, (size_t)std::max(1, G.handles) * sizeof(int),
                           cudaMemcpyDeviceToHost, G.stream);
    if (eb == cudaSuccess) eb = cudaEventRecord(G.join, G.stream);
    if (eb == cudaSuccess) eb = cudaStreamWaitEvent(en->main, G.join, 0);
  }
  int64_t solo_top = 0;
  for (int i : en->solo) {
    if (eb != cudaSuccess) break;
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
  int64_t grouped_top = 0;
  for (const Group& G : en->groups) grouped_top += G.top_kernels;
  solo_top = fnpf::graph_kernel_nodes(graph) - grouped_top;
  e = cudaGraphInstantiate(&en->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  // the solo tanks' top-level kernels, attributed evenly for the launch counter
  const int ns = (int)en->solo.size();
  for (int k = 0; k < ns; ++k)
    en->meshes[en->solo[k]]->step_kernels = solo_top / ns + (k < solo_top % ns ? 1 : 0);
  for (int i = 0; i < (int)en->meshes.size(); ++i) {
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
  for (int i = 0; i < n; ++i) {
    if (!meshes[i]) return FNPF_EINVAL;
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) {
        g_ens_error = "the same mesh twice in one ensemble";
        return FNPF_EINVAL;
      }
  }
  fnpf_ensemble* en = new fnpf_ensemble();
  en->meshes.assign(meshes, meshes + n);
  en->join.assign(n, nullptr);
  en->key.assign(2 * n, nullptr);
  en->dts.assign(n, 0.0);
  cudaError_t e = cudaStreamCreateWithFlags(&en->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&en->scratch, cudaStreamNonBlocking);
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
  if (en->scratch) cudaStreamDestroy(en->scratch);
  if (en->main) cudaStreamDestroy(en->main);
  delete en;
}

fnpf_status fnpf_ensemble_set_batching(fnpf_ensemble* en, int on, int max_tanks, int64_t max_dof) {
  if (!en || max_tanks < 0 || max_tanks > fnpf::kMaxBatch) return FNPF_EINVAL;
  const int mt = max_tanks > 0 ? max_tanks : fnpf::kMaxBatch;
  const int64_t md = max_dof > 0 ? max_dof : INT64_MAX;
  if (en->batching != (on != 0) || en->max_tanks != mt || en->max_dof != md) reset_graph(en);
  en->batching = on != 0;
  en->max_tanks = mt;
  en->max_dof = md;
  return FNPF_OK;
}

fnpf_status fnpf_ensemble_stats(const fnpf_ensemble* en, int* groups, int* batched_tanks, int64_t* kernels) {
  if (!en) return FNPF_EINVAL;
  int bt = 0;
  for (const Group& G : en->groups) bt += (int)G.tanks.size();
  if (groups) *groups = (int)en->groups.size();
  if (batched_tanks) *batched_tanks = bt;
  if (kernels) *kernels = en->last_kernels;
  return FNPF_OK;
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
  int64_t before = 0;
  for (fnpf_mesh* m : en->meshes) before += m->launches;
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
    int64_t after = 0;
    for (fnpf_mesh* m : en->meshes) after += m->launches;
    en->last_kernels = after - before;
    return FNPF_OK;
  }
  cudaError_t e = cudaSuccess;
  if (!en->exec || !keys_match(en, etas, phiss, dts)) e = capture(en, etas, phiss, dts);
  if (e != cudaSuccess) {
    reset_graph(en);
    (void)cudaGetLastError();
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
  // kernels of the batched groups: top level plus every loop body execution,
  // attributed evenly to the group's tanks
  for (const Group& G : en->groups) {
    int64_t k = G.top_kernels;
    for (int h = 0; h < G.handles; ++h) k += G.body_kernels[h] * G.counts_host[h];
    const int T = (int)G.tanks.size();
    for (int t = 0; t < T; ++t) en->meshes[G.tanks[t]]->launches += k / T + (t < k % T ? 1 : 0);
  }
  std::vector<bool> solo(n, false);
  for (int i : en->solo) solo[i] = true;
  fnpf_status result = FNPF_OK;
  for (int i = 0; i < n; ++i) {
    fnpf_status st = fnpf::read_step_info(en->meshes[i], info ? info + 4 * i : nullptr, 0.0f, solo[i]);
    if (st != FNPF_OK && result == FNPF_OK) {
      result = st;
      en->err = "tank " + std::to_string(i) + ": " + en->meshes[i]->err;
    }
  }
  int64_t after = 0;
  for (fnpf_mesh* m : en->meshes) after += m->launches;
  en->last_kernels = after - before;
  return result;
}

const char* fnpf_ensemble_last_error(const fnpf_ensemble* en) { return en ? en->err.c_str() : g_ens_error.c_str(); }

}  // extern "C"

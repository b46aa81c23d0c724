// The prism mesh object behind fnpf_prism_* (prism.cu: numbering, tables and
// the operator; prism_step.cu: the solve, w and the RK4 step).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace fnpf {
struct PrismStepState;
}

struct fnpf_prism {
  int p = 0, n = 0, nz = 0, nt = 0, nq = 0, ntri = 0;
  int ns = 0, nv = 0;
  int64_t N = 0;
  std::vector<int> tnodes;   // host copy [ntri][nt]
  std::vector<double> xs, ys;
  std::vector<double> verts;  // host copy [nverts][2] (the coarser orders of the p-multigrid)
  std::vector<int> tris;      // host copy [ntri][3]
  int* d_tnodes = nullptr;
  double* d_tab = nullptr;   // geo [ntri][4], L, Lr, Ls [nq][nt], wq [nq], xi, wv [n], D [n][n]
  double* d_ye = nullptr;    // element results [ntri * nz][nt * n]
  int64_t* d_off = nullptr;  // incidence offsets [N + 1]
  int64_t* d_inc = nullptr;  // indices into d_ye
  std::string err;
  fnpf::PrismStepState* step = nullptr;   // workspace of the solve and the step (at their first call)
};

namespace fnpf {
// Frees the step workspace of m (if any); prism_step.cu.
void prism_step_free(fnpf_prism* m);
}

// fnpf_apply_noalloc: the operator application of fnpf_apply for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a plug-in running inside a host
// application that owns all device memory through its own pool and forbids
// other allocations, or a loop with a fixed, pre-reserved memory budget where
// an allocation could fail or stall at run time.  They cannot create an
// fnpf_mesh (creation allocates the tables and workspaces), so this entry
// point needs nothing but the caller's input and output arrays: the GLL
// tables, the horizontal metric of a box mesh and the operator's ring scratch
// live in the file-scope device array below, which every GPU that loads the
// library holds until the process exits.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it per device.
// Make that first call before any stream capture.  All calls share the one
// array and it keeps the last call's contents; every call rewrites the parts
// it reads before reading them, so nothing has to start at zero.  Calls that
// overlap on the GPU (two streams, or two host threads) race on the array.
#include <mutex>

#include "fnpf_internal.cuh"

namespace fnpf {
void set_create_error(const char* msg);
}

namespace {

constexpr int64_t kScratchDoubles = (int64_t)2 << 20;   // 2,097,152 doubles = 16 MiB
constexpr int64_t kAlign = 32;                           // 256-byte sub-array alignment
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

struct BoxTables {
  double D[fnpf::kMaxN * fnpf::kMaxN];
  double xi[fnpf::kMaxN];
  double w[fnpf::kMaxN];
  double dx, dy;
};

inline int64_t round_up(int64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Writes D, xi, w and the constant box metric of every element-column line.
__global__ void fill_box_tables_kernel(fnpf::Geom g, BoxTables tb, double* D, double* xi, double* w, double* hm) {
  const int n = g.n;
  const int64_t hs = (int64_t)g.n_ecol * g.lines;
  const int64_t total = hs > n * n ? hs : n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < n * n) D[idx] = tb.D[idx];
    if (idx < n) {
      xi[idx] = tb.xi[idx];
      w[idx] = tb.w[idx];
    }
    if (idx < hs) {
      const int line = (int)(idx % g.lines);
      const int i = line % n, j = line / n;
      double rx, sy, cw;
      if (g.dim == 3) {
        rx = 2.0 / tb.dx;
        sy = 2.0 / tb.dy;
        cw = tb.w[i] * tb.w[j] * (0.25 * tb.dx * tb.dy);
      } else {
        rx = 2.0 / tb.dx;
        sy = 0.0;
        cw = tb.w[i] * (0.5 * tb.dx);
      }
      hm[idx] = rx;
      hm[hs + idx] = 0.0;
      hm[2 * hs + idx] = 0.0;
      hm[3 * hs + idx] = sy;
      hm[4 * hs + idx] = cw;
    }
  }
}

}  // namespace

extern "C" fnpf_status fnpf_apply_noalloc(const fnpf_mesh_desc* desc, const double* h, const double* eta,
                                          const double* x, double* y, void* stream) {
  if (!desc || !h || !eta || !x || !y) {
    fnpf::set_create_error("fnpf_apply_noalloc: NULL argument");
    return FNPF_EINVAL;
  }
  fnpf_mesh_desc d = *desc;
  const double unused = 1.0;
  d.h = &unused;   // the depth comes in as the device array h
  std::string why;
  fnpf_status st = fnpf::validate_desc(&d, &why);
  if (st != FNPF_OK) {
    fnpf::set_create_error(("fnpf_apply_noalloc: " + why).c_str());
    return st;
  }
  if (d.horiz_kind != FNPF_BOX) {
    fnpf::set_create_error("fnpf_apply_noalloc: only FNPF_BOX meshes");
    return FNPF_EUNSUPPORTED;
  }
  const fnpf::Geom g = fnpf::make_geom(&d);
  const int n = g.n;
  const int64_t hs = (int64_t)g.n_ecol * g.lines;
  const int64_t off_xi = round_up(n * n), off_w = off_xi + round_up(n), off_hm = off_w + round_up(n);
  const int64_t off_ring = off_hm + round_up(5 * hs);
  const int64_t need = off_ring + (int64_t)g.nv * g.n_ecol * g.ring;
  if (need > kScratchDoubles) {
    fnpf::set_create_error("fnpf_apply_noalloc: mesh needs more scratch than the fixed 16 MiB device array");
    return FNPF_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    fnpf::set_create_error("fnpf_apply_noalloc: no usable current device");
    return e != cudaSuccess ? FNPF_ECUDA : FNPF_EINVAL;
  }
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      double* p = nullptr;
      e = cudaGetSymbolAddress((void**)&p, g_scratch);
      if (e != cudaSuccess || !p) {
        fnpf::set_create_error((std::string("fnpf_apply_noalloc: cudaGetSymbolAddress failed: ") +
                                cudaGetErrorString(e)).c_str());
        return FNPF_ECUDA;
      }
      g_scratch_ptr[dev] = p;
    }
    base = g_scratch_ptr[dev];
  }
  BoxTables tb;
  fnpf::gll_tables(g.p, tb.xi, tb.w, tb.D);
  tb.dx = d.Lx / g.nx;
  tb.dy = g.dim == 3 ? d.Ly / g.ny : 1.0;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t work = hs > n * n ? hs : n * n;
  const int threads = 256;
  const int blocks = (int)((work + threads - 1) / threads < 1024 ? (work + threads - 1) / threads : 1024);
  fill_box_tables_kernel<<<blocks, threads, 0, s>>>(g, tb, base, base + off_xi, base + off_w, base + off_hm);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    fnpf::set_create_error((std::string("fnpf_apply_noalloc: table fill launch failed: ") + cudaGetErrorString(e)).c_str());
    return FNPF_ECUDA;
  }
  const fnpf::Tables<double> t{base, base + off_xi, base + off_w, base + off_hm, h, nullptr};
  e = fnpf::launch_apply<double>(g, t, eta, x, x + g.NI, y, y + g.NI, base + off_ring, 1, s);
  if (e != cudaSuccess) {
    fnpf::set_create_error((std::string("fnpf_apply_noalloc: operator launch failed: ") + cudaGetErrorString(e)).c_str());
    return FNPF_ECUDA;
  }
  return FNPF_OK;
}

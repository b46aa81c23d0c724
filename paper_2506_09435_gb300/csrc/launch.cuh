// Kernel launches of the library, single and batched.
//
// Every kernel of the RK4 step is written as a struct K with a static device
// function K::run(Blk, args...) and the launch bound K::kThreads; Blk is the
// block's position in its own grid.  launch<K>(grid, block, smem, stream,
// args...) launches k_one<K>, which calls K::run with the hardware block
// index.  k_many<K> runs the same body for several independent meshes in one
// launch: its grid is the concatenation of the meshes' grids, a block finds
// its mesh by a binary search over the first-block offsets in the launch's
// parameters and calls K::run with that mesh's argument tuple (also in the
// parameters) and its block position inside that mesh's grid, so every block
// does exactly what it does in the mesh's own launch.  A per-mesh gate (an int
// per mesh in device memory, set by the loop-condition kernels of a batched
// graph) skips the meshes whose loop has finished.
//
// While a Recorder is active on the calling thread, launch<K>, memset_async,
// memcpy_async and the loop primitives of the device-driven solves append
// operations to it instead of running them; the ensemble records one RK4 step
// per tank this way and replays the aligned records as batched launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/std/tuple>
#include <cstring>
#include <memory>
#include <type_traits>
#include <utility>
#include <vector>

namespace fnpf {

// Position of a block in the grid of its own mesh: (x, y) of an nx x ny grid.
struct Blk {
  int x, y, nx, ny;
};

__device__ __forceinline__ Blk this_blk() {
  return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y};
}

constexpr int kMaxBatch = 32;   // meshes per batched launch

// Parameters of a batched launch: the meshes' argument tuples travel in the
// kernel's own parameter space (read in place through a mesh index known only
// at run time, so the compiler keeps them in registers: the batched operator
// kernels use about 15 registers more than their single-launch forms).
template <class... P>
struct BatchParams {
  const int* gate;              // gate[t] == 0: mesh t's blocks return at once (null: none)
  int ntank;
  int off[kMaxBatch + 1];       // first block of mesh t; off[ntank] = total blocks
  int gx[kMaxBatch];            // grid.x of mesh t (its grid.y = blocks / gx)
  cuda::std::tuple<P...> args[kMaxBatch];
};

template <class K, class = void>
struct min_blocks_of {
  static constexpr int v = 1;
};
template <class K>
struct min_blocks_of<K, std::void_t<decltype(K::kMinBlocks)>> {
  static constexpr int v = K::kMinBlocks;
};
template <class K, class = void>
struct cluster_of {
  static constexpr int v = 1;
};
template <class K>
struct cluster_of<K, std::void_t<decltype(K::kCluster)>> {
  static constexpr int v = K::kCluster;
};
// Kernels whose result does not depend on the block size (any block size at
// least the mesh's own): a batched launch takes the largest over its meshes.
template <class K, class = void>
struct flex_block_of {
  static constexpr bool v = false;
};
template <class K>
struct flex_block_of<K, std::void_t<decltype(K::kFlexBlock)>> {
  static constexpr bool v = K::kFlexBlock;
};

template <class K, class... P>
__global__ void __launch_bounds__(K::kThreads, min_blocks_of<K>::v) k_one(P... a) {
  K::run(this_blk(), a...);
}

template <class K, class Tup, size_t... I>
__device__ __forceinline__ void run_tuple(const Blk& b, const Tup& t, std::index_sequence<I...>) {
  K::run(b, cuda::std::get<I>(t)...);
}

template <class K, class... P>
__global__ void __launch_bounds__(K::kThreads, min_blocks_of<K>::v)
    k_many(const __grid_constant__ BatchParams<P...> h) {
  const int bid = (int)blockIdx.x;
  int lo = 0, hi = h.ntank - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (h.off[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  if (h.gate && !h.gate[lo]) return;   // uniform over the block (and over a cluster: one mesh per cluster)
  const int li = bid - h.off[lo], gx = h.gx[lo];
  const Blk b{li % gx, li / gx, gx, (h.off[lo + 1] - h.off[lo]) / gx};
  run_tuple<K>(b, h.args[lo], std::index_sequence_for<P...>{});
}

// ---------------------------------------------------------------------------
// Recording.

enum OpKind { OP_KERNEL = 0, OP_COPY_D2H = 1, OP_HANDLE = 2, OP_COND = 3, OP_LOOP = 4, OP_END = 5 };

// Launches the batched kernel of a recorded operation over ntank meshes: off,
// gx and the argument tuples (args[t], as recorded) per mesh.
using EmitFn = cudaError_t (*)(const int* gate, int ntank, const int* off, const int* gx,
                               const unsigned char* const* args, unsigned blocks, unsigned threads, size_t smem,
                               cudaStream_t s);

struct Op {
  int kind = OP_KERNEL;
  const void* id = nullptr;          // OP_KERNEL: the batched kernel (identity of the operation)
  EmitFn emit = nullptr;
  dim3 grid{1, 1, 1}, block{1, 1, 1};
  size_t smem = 0;
  bool flex = false;
  std::vector<unsigned char> args;   // OP_KERNEL: the argument tuple
  void* dst = nullptr;               // OP_COPY_D2H
  const void* src = nullptr;
  size_t bytes = 0;
  int handle = -1;                   // OP_HANDLE, OP_COND, OP_LOOP: loop handle ordinal
  const void* sc = nullptr;          // OP_COND: the solve's scalars (CgScalars)
  int cap = 0, use_outer = 0;
};

struct Recorder {
  std::vector<Op> ops;
  int handles = 0;
};

// The calling thread's active recorder (null: launches run).
Recorder*& active_recorder();

template <class F>
struct run_sig;
template <class... P>
struct run_sig<void (*)(Blk, P...)> {
  using Tup = cuda::std::tuple<P...>;

  template <class K>
  static auto one() {
    return &k_one<K, P...>;
  }
  template <class K>
  static auto many() {
    return &k_many<K, P...>;
  }

  template <class K>
  static cudaError_t emit(const int* gate, int ntank, const int* off, const int* gx, const unsigned char* const* args,
                          unsigned blocks, unsigned threads, size_t smem, cudaStream_t s) {
    using Params = BatchParams<P...>;
    static_assert(sizeof(Params) <= 31 * 1024, "batched parameters within the kernel parameter limit");
    if (ntank < 1 || ntank > kMaxBatch) return cudaErrorInvalidValue;
    std::unique_ptr<Params> hb(new Params());   // large: on the heap; the launch copies it
    Params& hp = *hb;
    hp.gate = gate;
    hp.ntank = ntank;
    for (int t = 0; t < ntank; ++t) {
      hp.off[t] = off[t];
      hp.gx[t] = gx[t];
      memcpy(static_cast<void*>(&hp.args[t]), args[t], sizeof(Tup));
    }
    hp.off[ntank] = off[ntank];
    auto fn = &k_many<K, P...>;
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    if constexpr (cluster_of<K>::v > 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(blocks);
      cfg.blockDim = dim3(threads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cluster_of<K>::v;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, fn, hp);
    } else {
      fn<<<blocks, threads, smem, s>>>(hp);
      return cudaPeekAtLastError();
    }
  }

  template <class K>
  static cudaError_t go(dim3 grid, dim3 block, size_t smem, cudaStream_t s, P... a) {
    static_assert((std::is_trivially_copyable<P>::value && ...), "kernel arguments are copied as bytes");
    if (Recorder* r = active_recorder()) {
      Op op;
      op.kind = OP_KERNEL;
      op.id = (const void*)&k_many<K, P...>;
      op.emit = &emit<K>;
      op.grid = grid;
      op.block = block;
      op.smem = smem;
      op.flex = flex_block_of<K>::v;
      const Tup t(a...);
      op.args.resize(sizeof(Tup));
      memcpy(op.args.data(), &t, sizeof(Tup));
      r->ops.push_back(std::move(op));
      return cudaSuccess;
    }
    if constexpr (cluster_of<K>::v > 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = grid;
      cfg.blockDim = block;
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cluster_of<K>::v;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, &k_one<K, P...>, a...);
    } else {
      k_one<K, P...><<<grid, block, smem, s>>>(a...);
      // peek, not get: callers test the error of a sequence of launches at its end
      return cudaPeekAtLastError();
    }
  }
};

// Launches kernel K (or records the launch).  Arguments convert to the types
// of K::run's parameters.
template <class K, class... A>
inline cudaError_t launch(dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... a) {
  return run_sig<decltype(&K::run)>::template go<K>(grid, block, smem, s, std::forward<A>(a)...);
}

// The single-mesh kernel of K (for attributes and occupancy queries).
template <class K>
inline auto kernel_one() {
  return run_sig<decltype(&K::run)>::template one<K>();
}

// Byte fill and device-to-device copy as kernels, so that a batched graph can
// gate them like any other operation.
struct fill_bytes_kernel {
  static constexpr int kThreads = 256;
  __device__ static void run(Blk bk, unsigned char* p, int value, int64_t n) {
    for (int64_t i = bk.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)bk.nx * kThreads)
      p[i] = (unsigned char)value;
  }
};
struct copy_words_kernel {
  static constexpr int kThreads = 256;
  __device__ static void run(Blk bk, uint32_t* d, const uint32_t* s, int64_t n) {
    for (int64_t i = bk.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)bk.nx * kThreads) d[i] = s[i];
  }
};

// cudaMemsetAsync, or its recorded form.
cudaError_t memset_async(void* p, int value, size_t bytes, cudaStream_t s);
// cudaMemcpyAsync (device to device or device to host), or its recorded form
// (device-to-device copies of whole 4-byte words become copy kernels).
cudaError_t memcpy_async(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s);

}  // namespace fnpf

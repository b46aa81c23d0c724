// Recorded forms of the stream operations of the RK4 step (launch.cuh).
#include "fnpf_internal.cuh"

namespace fnpf {

Recorder*& active_recorder() {
  static thread_local Recorder* r = nullptr;
  return r;
}

namespace {
inline unsigned words_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > kVecBlocks ? kVecBlocks : b));
}
}  // namespace

cudaError_t memset_async(void* p, int value, size_t bytes, cudaStream_t s) {
  if (active_recorder())
    return launch<fill_bytes_kernel>(words_blocks((int64_t)bytes), 256, 0, s, static_cast<unsigned char*>(p), value,
                                     (int64_t)bytes);
  return cudaMemsetAsync(p, value, bytes, s);
}

cudaError_t memcpy_async(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
  Recorder* r = active_recorder();
  if (!r) return cudaMemcpyAsync(dst, src, bytes, kind, s);
  if (kind == cudaMemcpyDeviceToDevice) {
    if (bytes % 4 != 0 || (uintptr_t)dst % 4 != 0 || (uintptr_t)src % 4 != 0) return cudaErrorNotSupported;
    const int64_t n = (int64_t)(bytes / 4);
    return launch<copy_words_kernel>(words_blocks(n), 256, 0, s, static_cast<uint32_t*>(dst),
                                     static_cast<const uint32_t*>(src), n);
  }
  if (kind != cudaMemcpyDeviceToHost) return cudaErrorNotSupported;
  Op op;
  op.kind = OP_COPY_D2H;
  op.dst = dst;
  op.src = src;
  op.bytes = bytes;
  r->ops.push_back(std::move(op));
  return cudaSuccess;
}

}  // namespace fnpf

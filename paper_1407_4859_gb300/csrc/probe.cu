// probe.cu -- the random-access microbenchmark that bounds the gather section (the particle
// program's section that reads fields at a permuted record).  A copy roofline says nothing about a
// kernel whose reads land on random records: DRAM serves each miss with a whole burst, so the
// ceiling is set by how many random transactions per second the memory system completes.  This
// kernel reads rec_bytes-wide structs at perm[i] and writes them to out[i] in order, with the
// permutation read sequentially, which is the gather's access pattern without its arithmetic.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace adha {

constexpr int kProbePerThread = 4;   // independent random loads in flight per thread

template <class V>
__global__ void __launch_bounds__(kThreads) gather_probe_kernel(const V* __restrict__ table, const int32_t* __restrict__ perm,
                                                              V* __restrict__ out, int64_t n) {
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += kProbePerThread * T) {
    int32_t j[kProbePerThread];
    V v[kProbePerThread];
#pragma unroll
    for (int k = 0; k < kProbePerThread; ++k) {
      const int64_t i = base + k * T;
      j[k] = i < n ? __ldg(perm + i) : 0;
    }
#pragma unroll
    for (int k = 0; k < kProbePerThread; ++k)
      if (base + k * T < n) v[k] = __ldg(table + j[k]);
#pragma unroll
    for (int k = 0; k < kProbePerThread; ++k) {
      const int64_t i = base + k * T;
      if (i < n) out[i] = v[k];
    }
  }
}

template <class V>
static int launch_probe(const void* table, const int32_t* perm, void* out, int64_t n, void* stream) {
  int sms = 0;
  if (int rc = sm_count(&sms)) return rc;
  int64_t blocks = (n + (int64_t)kThreads * kProbePerThread - 1) / ((int64_t)kThreads * kProbePerThread);
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 8));
  gather_probe_kernel<V><<<(int)blocks, kThreads, 0, (cudaStream_t)stream>>>(
      static_cast<const V*>(table), perm, static_cast<V*>(out), n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "gather probe launch");
}

struct ProbeCall {
  const void* table;
  const int32_t* perm;
  void* out;
  int64_t n;
  int32_t rec_bytes;
  void* stream;
};

static int probe_fn(const void* ctx) {
  const ProbeCall& c = *static_cast<const ProbeCall*>(ctx);
  if (c.rec_bytes == 4) return launch_probe<uint32_t>(c.table, c.perm, c.out, c.n, c.stream);
  if (c.rec_bytes == 8) return launch_probe<unsigned long long>(c.table, c.perm, c.out, c.n, c.stream);
  return launch_probe<uint4>(c.table, c.perm, c.out, c.n, c.stream);
}

}  // namespace adha

using namespace adha;

extern "C" int adha_gather_probe(const void* table, const int32_t* perm, void* out, int64_t n, int32_t rec_bytes,
                                 adha_stream stream) {
  clear_error();
  if (n < 0) return fail(ADHA_EINVAL, "n = %lld is negative", (long long)n);
  if (rec_bytes != 4 && rec_bytes != 8 && rec_bytes != 16) return fail(ADHA_EINVAL, "rec_bytes %d is not 4, 8 or 16", rec_bytes);
  if (n == 0) return 0;
  if (!table || !perm || !out) return fail(ADHA_EINVAL, "NULL buffer");
  if (reinterpret_cast<uintptr_t>(table) % rec_bytes || reinterpret_cast<uintptr_t>(out) % rec_bytes ||
      reinterpret_cast<uintptr_t>(perm) % 4)
    return fail(ADHA_EINVAL, "misaligned buffer");
  const ProbeCall c{table, perm, out, n, rec_bytes, stream};
  return profiled_launch(5, rec_bytes, (double)n * (4.0 + 2.0 * rec_bytes), stream, probe_fn, &c);
}

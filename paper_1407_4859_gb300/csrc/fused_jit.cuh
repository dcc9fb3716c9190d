// fused_jit.cuh -- skeleton of a fused run specialised at run time (paper Section 2: the combine
// edge, one pass over the records for a run of consecutive sections that share a layout).
//
// The library's fused kernel (fused.cu) reads its field table, section operands and slice table
// at run time, so every field access costs table lookups and loop control: about 15 instructions
// per field access per record, which makes long runs issue-bound.  For a run that is worth it, the
// host writes a small description W of this one run (chunk shape, the slices' offsets and sizes,
// the fields as typed register members of W::Rec, the sections' operands as constants) and the
// run-time compiler builds this skeleton around it.  Every field index, offset and operand is then
// a constant: a record's fields are read from the chunk buffer into registers once, the run's
// sections are applied there by the same per-record code as everywhere else (run_record), and
// the written fields are stored back once.  The pipeline is the one of the library's kernels:
// per warp, chunks of R = 32*M records staged with 16-byte cp.async (one chunk ahead with two
// buffers), written groups written back whole, the ragged tail done from global memory by the
// warp whose next chunk would be n_chunks.
//
// W provides: M, kBuffers (1 or 2), kInBytes (one chunk buffer), kPermStart (chunk-buffer offset
// of the staged permutation, -1 without a gather), stage(a, chunk, buf, lane),
// writeback(a, chunk, buf, lane), a register record type Rec with load(buf, r) / store(buf, r)
// and ld<V>(field) / st<V>(field, v), and apply<VOTE>(a, fr, rec, i, pj), which runs the
// sections in order on one record.
#pragma once

#include "device_types.h"
#include "ptx.cuh"
#include "section_ops.cuh"

namespace adha {

// The bits of a field value seen as type V (only ever asked for V of the field's own size).
template <class V, class B>
__device__ __forceinline__ V jit_as(B b) {
  if constexpr (sizeof(V) == sizeof(B)) {
    V v;
    memcpy(&v, &b, sizeof v);
    return v;
  } else {
    return V();
  }
}
template <class B, class V>
__device__ __forceinline__ B jit_bits(V v) {
  if constexpr (sizeof(V) == sizeof(B)) {
    B b;
    memcpy(&b, &v, sizeof b);
    return b;
  } else {
    return B();
  }
}

// Slice g of a chunk (bytes B, chunk-buffer offset S): global -> chunk buffer, 16 bytes per lane
// per step; and back for the written slices.
#define ADHA_JIT_STAGE(g, B, S)                                                  \
  {                                                                              \
    const uint8_t* src_ = a.load[g].ptr + ch * (int64_t)(B);                     \
    _Pragma("unroll") for (int t_ = 0; t_ < ((B) + 511) / 512; ++t_) {           \
      const int q_ = t_ * 512 + lane * 16;                                       \
      if ((B) % 512 == 0 || q_ < (B)) cp_async16(buf + (S) + q_, src_ + q_);     \
    }                                                                            \
  }
#define ADHA_JIT_WRITEBACK(g, B, S)                                                                   \
  {                                                                                                   \
    uint8_t* dst_ = const_cast<uint8_t*>(a.load[g].ptr) + ch * (int64_t)(B);                          \
    _Pragma("unroll") for (int t_ = 0; t_ < ((B) + 511) / 512; ++t_) {                                \
      const int q_ = t_ * 512 + lane * 16;                                                            \
      if ((B) % 512 == 0 || q_ < (B))                                                                 \
        *reinterpret_cast<uint4*>(dst_ + q_) = *reinterpret_cast<const uint4*>(buf + (S) + q_);       \
    }                                                                                                 \
  }

template <class W>
__device__ __forceinline__ void fused_window(const FusedArgs& a) {
  extern __shared__ __align__(16) uint8_t smem[];
  constexpr int R = 32 * W::M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* buf0 = smem + (size_t)warp * W::kBuffers * W::kInBytes;
  uint8_t* buf1 = buf0 + (W::kBuffers - 1) * W::kInBytes;
  const FieldRef* fr = a.f;
  const int64_t Wg = (int64_t)gridDim.x * kWarps;
  int64_t c = (int64_t)blockIdx.x * kWarps + warp;
  if (c < a.n_chunks) W::stage(a, c, buf0, lane);
  cp_async_commit();
  for (int i = 0; c < a.n_chunks; c += Wg, ++i) {
    uint8_t* cur = (i & 1) ? buf1 : buf0;
    if (W::kBuffers == 2) {
      if (c + Wg < a.n_chunks) W::stage(a, c + Wg, (i & 1) ? buf0 : buf1, lane);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const int64_t i0 = c * R;
#pragma unroll
    for (int m = 0; m < W::M; ++m) {
      const int r = lane + 32 * m;
      typename W::Rec x;
      x.load(cur, r);
      const int32_t pj = W::kPermStart >= 0 ? reinterpret_cast<const int32_t*>(cur + W::kPermStart)[r] : 0;
      W::template apply<true>(a, fr, x, i0 + r, pj);
      x.store(cur, r);
    }
    __syncwarp();
    W::writeback(a, c, cur, lane);
    __syncwarp();
    if (W::kBuffers == 1 && c + Wg < a.n_chunks) {   // one buffer: the next chunk once this one has gone back
      W::stage(a, c + Wg, buf0, lane);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
  const int64_t t0 = a.n_chunks * R;
  if (c == a.n_chunks && t0 < a.n) {
    for (int64_t i = t0 + lane; i < a.n; i += 32) {
      const int32_t pj = W::kPermStart >= 0 ? a.perm[i] : 0;
      W::template apply<false>(a, fr, GlobalRec{fr, i}, i, pj);
    }
  }
}

}  // namespace adha

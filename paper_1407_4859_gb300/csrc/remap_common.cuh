// remap_common.cuh -- the per-chunk element schedule and moves shared by the single-array remap
// (remap.cu) and the batched remap (batched.cu).
#pragma once

#include <cstdint>

#include "internal.h"

namespace adha {

// (record, move) of entry u of a class of cnt moves in a chunk of R records under `order`:
//   0: destination-major (record by record, its moves in turn);
//   1: record-major (per move, 32 consecutive records per warp step);
//   2 + s (s = 0..4): skewed record-major: warp step j covers records 32*(j / cnt) + lane, lane l
//      taking move (j + l / 2^s) mod cnt, which spreads a strided read over more banks while the
//      records (and so the writes of a one-field slice) stay consecutive.
__host__ __device__ __forceinline__ void schedule_pair(int u, int R, int cnt, int order, int* r, int* k) {
  if (order == 0) {
    *r = u / cnt;
    *k = u - *r * cnt;
  } else if (order == 1) {
    *k = u / R;
    *r = u - *k * R;
  } else {
    const int step = u >> 5, lane = u & 31;
    const int block = step / cnt, j = step - block * cnt;
    *r = 32 * block + lane;
    *k = (j + (lane >> (order - 2))) % cnt;
  }
}

// Schedule entry t of a chunk (R records, n_moves moves sorted into classes of 8/4/2 bytes):
// (source byte in the chunk buffer | destination byte in the output buffer << 16), source
// 0xFFFF for padding.
__device__ __forceinline__ uint32_t schedule_entry(int t, int R, const int32_t* cls_count, const int32_t* cls_order,
                                                   const Move* moves, const GroupRef* src, const GroupRef* dst) {
  int c = 0, first = 0;
  while (t >= R * (first + cls_count[c])) first += cls_count[c++];
  const int u = t - R * first, cnt = cls_count[c];
  int r, k;
  schedule_pair(u, R, cnt, cls_order[c], &r, &k);
  const Move m = moves[first + k];
  const uint32_t s = m.src_group < 0 ? 0xFFFFu : (uint32_t)(src[m.src_group].start + r * src[m.src_group].stride + m.src_off);
  const uint32_t d = (uint32_t)(dst[m.dst_group].start + r * dst[m.dst_group].stride + m.dst_off);
  return s | (d << 16);
}

template <typename V>
__device__ __forceinline__ void move_class(const uint32_t* sched, int begin, int end, const uint8_t* in, uint8_t* out,
                                           int lane) {
#pragma unroll 4
  for (int t = begin + lane; t < end; t += 32) {
    const uint32_t p = sched[t];
    const uint32_t s = p & 0xFFFFu;
    *reinterpret_cast<V*>(out + (p >> 16)) = s != 0xFFFFu ? *reinterpret_cast<const V*>(in + s) : V(0);
  }
}

// All moves of a chunk: the 8-, 4- and 2-byte classes in turn.
__device__ __forceinline__ void move_chunk(const uint32_t* sched, int R, const int32_t* cls_count, const uint8_t* in,
                                           uint8_t* out, int lane) {
  const int e8 = R * cls_count[0], e4 = e8 + R * cls_count[1], e2 = e4 + R * cls_count[2];
  move_class<unsigned long long>(sched, 0, e8, in, out, lane);
  move_class<uint32_t>(sched, e8, e4, in, out, lane);
  move_class<uint16_t>(sched, e4, e2, in, out, lane);
}

template <typename V>
__device__ __forceinline__ void tail_move(const Move& m, int64_t rec, const GroupRef* src, const GroupRef* dst) {
  V v = V(0);
  if (m.src_group >= 0) v = *reinterpret_cast<const V*>(src[m.src_group].ptr + rec * src[m.src_group].stride + m.src_off);
  *reinterpret_cast<V*>(const_cast<uint8_t*>(dst[m.dst_group].ptr) + rec * dst[m.dst_group].stride + m.dst_off) = v;
}

// Records [t0, n) moved one (record, move) pair per lane straight between global buffers.
__device__ __forceinline__ void tail_moves(int64_t t0, int64_t n, int n_moves, const int32_t* cls_count,
                                           const Move* moves, const GroupRef* src, const GroupRef* dst, int lane) {
  const int Tt = (int)(n - t0);
  for (int e = lane; e < Tt * n_moves; e += 32) {
    const int r = e / n_moves, k = e - r * n_moves;
    const Move m = moves[k];
    if (k < cls_count[0]) tail_move<unsigned long long>(m, t0 + r, src, dst);
    else if (k < cls_count[0] + cls_count[1]) tail_move<uint32_t>(m, t0 + r, src, dst);
    else tail_move<uint16_t>(m, t0 + r, src, dst);
  }
}

}  // namespace adha

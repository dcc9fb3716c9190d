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

constexpr int kMoveClasses = 6;

__host__ __device__ __forceinline__ int class_width(int c) { return 8 >> (c % 3); }

// Schedule entry t of a chunk (R records, n_moves moves sorted into the six classes):
// source byte in the chunk buffer | destination << 16, where the destination is
// (group << 10 | record) for direct classes and the output-buffer byte otherwise.  A padding move
// reads pad_src: the 16 zero bytes that follow every input chunk buffer, so that the move loops
// need no test.
__host__ __device__ __forceinline__ uint32_t schedule_entry(int t, int R, const int32_t* cls_count, const int32_t* cls_order,
                                                            const Move* moves, const GroupRef* src, const GroupRef* dst,
                                                            int pad_src) {
  int c = 0, first = 0;
  while (t >= R * (first + cls_count[c])) first += cls_count[c++];
  const int u = t - R * first, cnt = cls_count[c];
  int r, k;
  schedule_pair(u, R, cnt, cls_order[c], &r, &k);
  const Move m = moves[first + k];
  const uint32_t s = m.src_group < 0 ? (uint32_t)pad_src
                                     : (uint32_t)(src[m.src_group].start + r * src[m.src_group].stride + m.src_off);
  const uint32_t d = c < 3 ? (((uint32_t)m.dst_group << 10) | (uint32_t)r)
                           : (uint32_t)(dst[m.dst_group].start + r * dst[m.dst_group].stride + m.dst_off);
  return s | (d << 16);
}

// Bytes of zeros after each input chunk buffer (the source of padding moves).
constexpr int kZeroTail = 16;

// The moves of one class into the output buffer, four per lane per round: the four schedule
// entries, then the four source values, then the four stores, so that one round's shared-memory
// loads are in flight together (the buffers do not overlap).
template <typename V>
__device__ __forceinline__ void move_class_staged(const uint32_t* __restrict__ sched, int begin, int end,
                                                  const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int lane) {
  int t = begin + lane;
  for (; t + 96 < end; t += 128) {
    const uint32_t p0 = sched[t], p1 = sched[t + 32], p2 = sched[t + 64], p3 = sched[t + 96];
    const V v0 = *reinterpret_cast<const V*>(in + (p0 & 0xFFFFu));
    const V v1 = *reinterpret_cast<const V*>(in + (p1 & 0xFFFFu));
    const V v2 = *reinterpret_cast<const V*>(in + (p2 & 0xFFFFu));
    const V v3 = *reinterpret_cast<const V*>(in + (p3 & 0xFFFFu));
    *reinterpret_cast<V*>(out + (p0 >> 16)) = v0;
    *reinterpret_cast<V*>(out + (p1 >> 16)) = v1;
    *reinterpret_cast<V*>(out + (p2 >> 16)) = v2;
    *reinterpret_cast<V*>(out + (p3 >> 16)) = v3;
  }
  for (; t < end; t += 32) {
    const uint32_t p = sched[t];
    *reinterpret_cast<V*>(out + (p >> 16)) = *reinterpret_cast<const V*>(in + (p & 0xFFFFu));
  }
}

// Moves into one-field destination groups go straight to global memory: record rec0 + r.
template <typename V>
__device__ __forceinline__ void move_class_direct(const uint32_t* __restrict__ sched, int begin, int end,
                                                  const uint8_t* __restrict__ in, const GroupRef* dst, int64_t rec0,
                                                  int lane) {
#pragma unroll 4
  for (int t = begin + lane; t < end; t += 32) {
    const uint32_t p = sched[t];
    const uint32_t d = p >> 16;
    const GroupRef& g = dst[d >> 10];
    *reinterpret_cast<V*>(const_cast<uint8_t*>(g.ptr) + (rec0 + (int64_t)(d & 1023u)) * g.stride) =
        *reinterpret_cast<const V*>(in + (p & 0xFFFFu));
  }
}

// All moves of a chunk whose first record is rec0 (DIRECT: the plan has direct classes).
template <bool DIRECT>
__device__ __forceinline__ void move_chunk(const uint32_t* sched, int R, const int32_t* cls_count, const uint8_t* in,
                                           uint8_t* out, const GroupRef* dst, int64_t rec0, int lane) {
  int e = R * (cls_count[0] + cls_count[1] + cls_count[2]), b;
  if (DIRECT) {
    e = 0;
    b = e; e += R * cls_count[0]; move_class_direct<unsigned long long>(sched, b, e, in, dst, rec0, lane);
    b = e; e += R * cls_count[1]; move_class_direct<uint32_t>(sched, b, e, in, dst, rec0, lane);
    b = e; e += R * cls_count[2]; move_class_direct<uint16_t>(sched, b, e, in, dst, rec0, lane);
  }
  b = e; e += R * cls_count[3]; move_class_staged<unsigned long long>(sched, b, e, in, out, lane);
  b = e; e += R * cls_count[4]; move_class_staged<uint32_t>(sched, b, e, in, out, lane);
  b = e; e += R * cls_count[5]; move_class_staged<uint16_t>(sched, b, e, in, out, lane);
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
    int c = 0, first = 0;
    while (k >= first + cls_count[c]) first += cls_count[c++];
    const int w = class_width(c);
    if (w == 8) tail_move<unsigned long long>(moves[k], t0 + r, src, dst);
    else if (w == 4) tail_move<uint32_t>(moves[k], t0 + r, src, dst);
    else tail_move<uint16_t>(moves[k], t0 + r, src, dst);
  }
}

// Writes the staged (start >= 0) destination slices of chunk `ch` from the output buffer with
// 16-byte stores; the staged slices follow one another in the buffer in destination order
// (without direct classes every destination group is staged).
template <bool DIRECT>
__device__ __forceinline__ void write_back(const GroupRef* dst, int R, int out_bytes, const uint8_t* out,
                                           int64_t ch, int lane) {
  int g = 0;
  for (int p = lane * 16; p < out_bytes; p += 512) {
    while ((DIRECT && dst[g].start < 0) || p >= dst[g].start + R * dst[g].stride) ++g;
    *reinterpret_cast<uint4*>(const_cast<uint8_t*>(dst[g].ptr) + ch * R * dst[g].stride + (p - dst[g].start)) =
        *reinterpret_cast<const uint4*>(out + p);
  }
}

// Where a 16-byte piece of a chunk buffer lives in global memory: base + chunk * step.
struct Piece {
  const uint8_t* base;
  int64_t step;
};

// Piece q of a buffer holding the slices `grp` (staged ones, start >= 0) in buffer order.
__device__ __forceinline__ Piece piece_of(int q, const GroupRef* grp, int R) {
  const int p = q * 16;
  int g = 0;
  while (grp[g].start < 0 || p >= grp[g].start + R * grp[g].stride) ++g;
  return Piece{grp[g].ptr + (p - grp[g].start), (int64_t)R * grp[g].stride};
}

}  // namespace adha

// section_ops.cuh -- per-record and per-chunk arithmetic of the section kinds, shared by the
// single-section kernel (sections.cu) and the fused kernel (fused.cu).  A record's fields are
// reached through a FieldRef table: in the warp's chunk buffer when staged, else in global memory.
// Every floating operation is an explicitly rounded-to-nearest intrinsic, so no contraction can
// change a bit.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#include <cstring>
#endif

#include "device_types.h"
#include "ptx.cuh"

// Loops over a section's listed fields: unrolled in windows specialised at run time (constant
// bounds), left to the compiler's own choice in the library's kernels (bounds known at run time).
#ifdef __CUDACC_RTC__
#define ADHA_FIELD_LOOP _Pragma("unroll")
#else
#define ADHA_FIELD_LOOP
#endif

namespace adha {

// Exact IEEE operations done with integer instructions, so that the fp64 pipe (a small fraction
// of the fp32 rate on this GPU) only does the additions.  Every case is a select between integer
// results: a branch to the fp64 instruction for the rare inputs would be turned into a select by
// the compiler too, and then the fp64 instruction would run for every value.

// The common cases of the two below, taken for a whole warp when every lane's values qualify
// (one vote per field): a normal double whose half is normal, and a normal float.
__device__ __forceinline__ bool half_is_plain(double x) {
  return ((unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu) - 2u <= 2044u;
}
__device__ __forceinline__ double half_plain(double x) {
  return __longlong_as_double(__double_as_longlong(x) - (1ll << 52));
}
// (a zero is plain too: a section that reads no fp32 field has t = 0 for one record in 256)
__device__ __forceinline__ bool widen_is_plain(float t) {
  const unsigned u = __float_as_uint(t);
  return ((u >> 23) & 0xFFu) - 1u <= 253u || (u & 0x7FFFFFFFu) == 0u;
}
__device__ __forceinline__ double widen_plain(float t) {
  const unsigned u = __float_as_uint(t);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long normal = sign | ((unsigned long long)(((u >> 23) & 0xFFu) + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)((u & 0x7FFFFFFFu) ? normal : sign));
}

// x * 0.5 rounded to nearest.  A normal x whose half is normal (biased exponent 2..2046): the
// exponent lowered by one.  Exponent 0 or 1 (zeros, subnormals, the smallest normals): the half is
// subnormal, its significand the full significand q of x (with the implicit bit for exponent 1)
// halved with ties to even (q odd is exactly a tie); a carry into the exponent field gives the
// smallest normal, as it should.  Infinities and NaNs are returned unchanged.
__device__ __forceinline__ double half_rn_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  const unsigned long long q = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const unsigned long long h = (q >> 1) + (q & (q >> 1) & 1ull);
  const unsigned long long small = (b & (1ull << 63)) | h;
  const unsigned long long big = e == 0x7FFu ? b : b - (1ull << 52);
  return __longlong_as_double((long long)(e <= 1u ? small : big));
}

// float -> double, exact.  Normal: sign and significand kept (the significand shifted into the
// wider field), exponent rebiased from 127 to 1023.  Zero: the sign alone.  Subnormal m * 2^-149
// (m < 2^23): normal in double, its leading bit p = 31 - clz(m) becomes the implicit one, exponent
// p - 149.  Infinity: exponent all ones; NaN: its payload shifted likewise, made quiet.
__device__ __forceinline__ double widen_int(float t) {
  const unsigned u = __float_as_uint(t);
  const unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long mm = (unsigned long long)m << 29;
  const unsigned long long normal = sign | ((unsigned long long)(e + 896u) << 52) | mm;
  const unsigned long long special = sign | (0x7FFull << 52) | mm | (m ? (1ull << 51) : 0ull);
  const int p = 31 - __clz((int)(m | 1u));
  const unsigned long long sub = sign | ((unsigned long long)(p + 874) << 52) |
                                 (((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFull);
  const unsigned long long zero_or_sub = m ? sub : sign;
  return __longlong_as_double((long long)(e == 0u ? zero_or_sub : (e == 0xFFu ? special : normal)));
}

// The same two with the IEEE instruction for the rare inputs: the compiler turns the choice into
// a select, so the fp64 multiply (or the conversion) runs for every value next to the integer
// result.  That costs fp64-pipe time but few registers and instructions, the better trade in
// the memory-bound single-section kernels; fused runs, which compute long per chunk, take the
// integer forms above behind a warp vote.
__device__ __forceinline__ double half_rn(double x) {
  return half_is_plain(x) ? half_plain(x) : __dmul_rn(x, 0.5);
}
__device__ __forceinline__ double widen(float t) { return widen_is_plain(t) ? widen_plain(t) : (double)t; }

// The integer forms behind one warp vote per value, for code whose 32 lanes run it together.
__device__ __forceinline__ double half_vote(double x) {
  return __all_sync(0xFFFFFFFFu, half_is_plain(x)) ? half_plain(x) : half_rn_int(x);
}
__device__ __forceinline__ double widen_vote(float t) {
  return __all_sync(0xFFFFFFFFu, widen_is_plain(t)) ? widen_plain(t) : widen_int(t);
}

struct StagedRec {      // record r of a staged chunk (global record i)
  const FieldRef* f;
  uint8_t* stage;
  int r;
  int64_t i;
  template <class V>
  __device__ __forceinline__ V ld(int k) const {
    const FieldRef& F = f[k];
    if (F.s0 >= 0) return *reinterpret_cast<const V*>(stage + F.s0 + r * F.ss);
    return *reinterpret_cast<const V*>(F.g + i * F.gs);
  }
  template <class V>
  __device__ __forceinline__ void st(int k, V v) const {
    const FieldRef& F = f[k];
    if (F.wsm) *reinterpret_cast<V*>(stage + F.s0 + r * F.ss) = v;
    else *reinterpret_cast<V*>(F.g + i * F.gs) = v;
  }
};

struct GlobalRec {      // record i in global memory (ragged tail)
  const FieldRef* f;
  int64_t i;
  template <class V>
  __device__ __forceinline__ V ld(int k) const {
    return *reinterpret_cast<const V*>(f[k].g + i * f[k].gs);
  }
  template <class V>
  __device__ __forceinline__ void st(int k, V v) const {
    *reinterpret_cast<V*>(f[k].g + i * f[k].gs) = v;
  }
};

template <class V>
__device__ __forceinline__ V gld(const FieldRef* f, int k, int64_t i) {
  return __ldg(reinterpret_cast<const V*>(f[k].g + i * f[k].gs));
}

// Lambert's continued fraction for tanh cut after the partial denominator 25, as x*Q(a)/P(a) with
// a = x*x: Horner's rule over the 7 coefficients of each polynomial, then one IEEE division.
__device__ __forceinline__ float tanh_cf(float x, const float* P, const float* Q) {
  if (fabsf(x) >= 9.0f) return copysignf(1.0f, x);
  const float a = __fmul_rn(x, x);
  float q = Q[6], p = P[6];
#pragma unroll
  for (int j = 5; j >= 0; --j) {
    q = __fadd_rn(__fmul_rn(q, a), Q[j]);
    p = __fadd_rn(__fmul_rn(p, a), P[j]);
  }
  return __fdiv_rn(__fmul_rn(x, q), p);
}

// MIX over the M records r = lane + 32m of a staged chunk, field-major: every field's shared
// and global addresses are computed once for the M records.
template <int M>
__device__ __forceinline__ void mix_chunk(const SecOp& so, const FieldRef* fr, uint8_t* stage, int64_t i0, int lane) {
  float s[M];
  uint32_t h[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    s[m] = 0.0f;
    h[m] = 0u;
  }
  // V value of field F for the lane's record m: from the chunk buffer if staged, else global
#define ADHA_MIX_READ(V, LIST, BODY)                                                        \
  for (int j = so.rd_off[LIST]; j < so.rd_off[LIST + 1]; ++j) {                            \
    const FieldRef& F = fr[so.rd[j]];                                                       \
    if (F.s0 >= 0) {                                                                        \
      const uint8_t* p = stage + F.s0 + lane * F.ss;                                        \
      _Pragma("unroll") for (int m = 0; m < M; ++m) {                                       \
        const V v = *reinterpret_cast<const V*>(p + m * 32 * F.ss);                         \
        BODY;                                                                               \
      }                                                                                     \
    } else {                                                                                \
      const uint8_t* p = F.g + (i0 + lane) * F.gs;                                          \
      _Pragma("unroll") for (int m = 0; m < M; ++m) {                                       \
        const V v = *reinterpret_cast<const V*>(p + (int64_t)m * 32 * F.gs);                \
        BODY;                                                                               \
      }                                                                                     \
    }                                                                                       \
  }
  ADHA_MIX_READ(float, ADHA_F32, s[m] = __fadd_rn(s[m], v))
  ADHA_MIX_READ(unsigned long long, ADHA_F64, h[m] ^= (uint32_t)v ^ (uint32_t)(v >> 32))
  ADHA_MIX_READ(uint32_t, ADHA_I32, h[m] ^= v)
  ADHA_MIX_READ(uint16_t, ADHA_BF16, h[m] ^= (uint32_t)v)
#undef ADHA_MIX_READ
  float t[M];
  uint32_t k[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    t[m] = __fadd_rn(s[m], __fmul_rn(__uint2float_rn(h[m] & 255u), 0.00390625f));
    k[m] = (h[m] ^ __float_as_uint(t[m])) >> 3;
  }
  // written fields: old value from the chunk buffer if staged, else global; new value to global
#define ADHA_MIX_WRITE(V, LIST, EXPR)                                                       \
  for (int j = so.wr_off[LIST]; j < so.wr_off[LIST + 1]; ++j) {                            \
    const FieldRef& F = fr[so.wr[j]];                                                       \
    uint8_t* p = stage + F.s0 + lane * F.ss;                                                \
    if (F.wsm) {                                                                            \
      _Pragma("unroll") for (int m = 0; m < M; ++m) {                                       \
        V* x = reinterpret_cast<V*>(p + m * 32 * F.ss);                                     \
        const V old = *x;                                                                   \
        *x = EXPR;                                                                          \
      }                                                                                     \
    } else {                                                                                \
      uint8_t* q = F.g + (i0 + lane) * F.gs;                                                \
      _Pragma("unroll") for (int m = 0; m < M; ++m) {                                       \
        const V old = *reinterpret_cast<const V*>(p + m * 32 * F.ss);                       \
        *reinterpret_cast<V*>(q + (int64_t)m * 32 * F.gs) = EXPR;                           \
      }                                                                                     \
    }                                                                                       \
  }
  ADHA_MIX_WRITE(float, ADHA_F32, __fadd_rn(__fmul_rn(old, 0.5f), t[m]))
  if (so.wr_off[ADHA_F64 + 1] > so.wr_off[ADHA_F64]) {
    double td[M];
#pragma unroll
    for (int m = 0; m < M; ++m) td[m] = widen(t[m]);
    ADHA_MIX_WRITE(double, ADHA_F64, __dadd_rn(half_rn(old), td[m]))
  }
  ADHA_MIX_WRITE(uint32_t, ADHA_I32, old ^ k[m])
  ADHA_MIX_WRITE(uint16_t, ADHA_BF16, (uint16_t)(old ^ (uint16_t)(k[m] & 0xFFFFu)))
#undef ADHA_MIX_WRITE
}

// M consecutive values of one field for records lane*M .. lane*M+M-1 of a one-field slice
// (contiguous, M*sizeof(V)-byte aligned): moved with 8- or 16-byte accesses.
template <class V, int M>
__device__ __forceinline__ void ld_vec(const uint8_t* p, V (&v)[M]) {
  constexpr int B = M * (int)sizeof(V);
  if constexpr (B % 16 == 0) {
#pragma unroll
    for (int k = 0; k < B / 16; ++k) {
      const uint4 x = reinterpret_cast<const uint4*>(p)[k];
      memcpy(reinterpret_cast<uint8_t*>(v) + 16 * k, &x, 16);
    }
  } else if constexpr (B == 8) {
    const uint2 x = *reinterpret_cast<const uint2*>(p);
    memcpy(v, &x, 8);
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = reinterpret_cast<const V*>(p)[m];
  }
}

template <class V, int M>
__device__ __forceinline__ void st_vec(uint8_t* p, const V (&v)[M]) {
  constexpr int B = M * (int)sizeof(V);
  if constexpr (B % 16 == 0) {
#pragma unroll
    for (int k = 0; k < B / 16; ++k) {
      uint4 x;
      memcpy(&x, reinterpret_cast<const uint8_t*>(v) + 16 * k, 16);
      reinterpret_cast<uint4*>(p)[k] = x;
    }
  } else if constexpr (B == 8) {
    uint2 x;
    memcpy(&x, v, 8);
    *reinterpret_cast<uint2*>(p) = x;
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) reinterpret_cast<V*>(p)[m] = v[m];
  }
}

// MIX when every accessed group holds one field (SoA-like): lane takes records lane*M + m, so
// each field is one vector load from the chunk buffer and one vector store, to global memory or
// (TO_STAGE, inside a fused run) back into the chunk buffer.  The field loops are unrolled so that
// several fields' loads are in flight before their (ordered) sums consume them.
template <int M, bool TO_STAGE = false>
__device__ __forceinline__ void mix_chunk_vec(const SecOp& so, const FieldRef* fr, uint8_t* stage, int64_t i0,
                                              int lane) {
  float s[M];
  uint32_t h[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    s[m] = 0.0f;
    h[m] = 0u;
  }
  // the lane's M records of a field of size b start at stage + s0 + lane*M*b
#define RD_S0(j) (TO_STAGE ? (int)so.rd_s0[j] : fr[so.rd[j]].s0)
#define WR_S0(j) (TO_STAGE ? (int)so.wr_s0[j] : fr[so.wr[j]].s0)
#define b2 (stage + lane * M * 2)
#define b4 (stage + lane * M * 4)
#define b8 (stage + lane * M * 8)
#pragma unroll 4
  for (int j = so.rd_off[ADHA_F32]; j < so.rd_off[ADHA_F32 + 1]; ++j) {
    float v[M];
    ld_vec<float, M>(b4 + RD_S0(j), v);
#pragma unroll
    for (int m = 0; m < M; ++m) s[m] = __fadd_rn(s[m], v[m]);
  }
#pragma unroll 4
  for (int j = so.rd_off[ADHA_F64]; j < so.rd_off[ADHA_F64 + 1]; ++j) {
    unsigned long long v[M];
    ld_vec<unsigned long long, M>(b8 + RD_S0(j), v);
#pragma unroll
    for (int m = 0; m < M; ++m) h[m] ^= (uint32_t)v[m] ^ (uint32_t)(v[m] >> 32);
  }
#pragma unroll 4
  for (int j = so.rd_off[ADHA_I32]; j < so.rd_off[ADHA_I32 + 1]; ++j) {
    uint32_t v[M];
    ld_vec<uint32_t, M>(b4 + RD_S0(j), v);
#pragma unroll
    for (int m = 0; m < M; ++m) h[m] ^= v[m];
  }
#pragma unroll 4
  for (int j = so.rd_off[ADHA_BF16]; j < so.rd_off[ADHA_BF16 + 1]; ++j) {
    uint16_t v[M];
    ld_vec<uint16_t, M>(b2 + RD_S0(j), v);
#pragma unroll
    for (int m = 0; m < M; ++m) h[m] ^= (uint32_t)v[m];
  }
  float t[M];
  uint32_t k[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    t[m] = __fadd_rn(s[m], __fmul_rn(__uint2float_rn(h[m] & 255u), 0.00390625f));
    k[m] = (h[m] ^ __float_as_uint(t[m])) >> 3;
  }
  const int64_t r0 = i0 + (int64_t)lane * M;
#pragma unroll 4
  for (int j = so.wr_off[ADHA_F32]; j < so.wr_off[ADHA_F32 + 1]; ++j) {
    float v[M];
    ld_vec<float, M>(b4 + WR_S0(j), v);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = __fadd_rn(__fmul_rn(v[m], 0.5f), t[m]);
    st_vec<float, M>(TO_STAGE ? b4 + WR_S0(j) : fr[so.wr[j]].g + r0 * 4, v);
  }
  if (so.wr_off[ADHA_F64 + 1] > so.wr_off[ADHA_F64]) {
    double td[M];
    if constexpr (TO_STAGE) {   // fused run: no fp64 instruction but the additions (see half_rn_int)
      bool plain = true;
#pragma unroll
      for (int m = 0; m < M; ++m) plain = plain && widen_is_plain(t[m]);
      if (__all_sync(0xFFFFFFFFu, plain)) {
#pragma unroll
        for (int m = 0; m < M; ++m) td[m] = widen_plain(t[m]);
      } else {
#pragma unroll
        for (int m = 0; m < M; ++m) td[m] = widen_int(t[m]);
      }
    } else {
#pragma unroll
      for (int m = 0; m < M; ++m) td[m] = widen(t[m]);
    }
#pragma unroll 4
    for (int j = so.wr_off[ADHA_F64]; j < so.wr_off[ADHA_F64 + 1]; ++j) {
      double v[M];
      ld_vec<double, M>(b8 + WR_S0(j), v);
      if constexpr (TO_STAGE) {
        bool ok = true;
#pragma unroll
        for (int m = 0; m < M; ++m) ok = ok && half_is_plain(v[m]);
        if (__all_sync(0xFFFFFFFFu, ok)) {
#pragma unroll
          for (int m = 0; m < M; ++m) v[m] = __dadd_rn(half_plain(v[m]), td[m]);
        } else {
#pragma unroll
          for (int m = 0; m < M; ++m) v[m] = __dadd_rn(half_rn_int(v[m]), td[m]);
        }
      } else {
#pragma unroll
        for (int m = 0; m < M; ++m) v[m] = __dadd_rn(half_rn(v[m]), td[m]);
      }
      st_vec<double, M>(TO_STAGE ? b8 + WR_S0(j) : fr[so.wr[j]].g + r0 * 8, v);
    }
  }
#pragma unroll 4
  for (int j = so.wr_off[ADHA_I32]; j < so.wr_off[ADHA_I32 + 1]; ++j) {
    uint32_t v[M];
    ld_vec<uint32_t, M>(b4 + WR_S0(j), v);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] ^= k[m];
    st_vec<uint32_t, M>(TO_STAGE ? b4 + WR_S0(j) : fr[so.wr[j]].g + r0 * 4, v);
  }
#pragma unroll 4
  for (int j = so.wr_off[ADHA_BF16]; j < so.wr_off[ADHA_BF16 + 1]; ++j) {
    uint16_t v[M];
    ld_vec<uint16_t, M>(b2 + WR_S0(j), v);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = (uint16_t)(v[m] ^ (uint16_t)(k[m] & 0xFFFFu));
    st_vec<uint16_t, M>(TO_STAGE ? b2 + WR_S0(j) : fr[so.wr[j]].g + r0 * 2, v);
  }
#undef b2
#undef b4
#undef b8
#undef RD_S0
#undef WR_S0
}

// AXPB, MUL, TANH under the vector mapping (x, y, z each a one-field group): lane takes records
// lane*M + m; x, y and the old z come from the chunk buffer (the values before the section, so
// any aliasing of x, y, z reads what the per-record rule reads), z and `save` get vector stores
// (z into the chunk buffer when TO_STAGE).
template <int OP, int M, bool TO_STAGE = false>
__device__ __forceinline__ void chain_chunk_vec(const SecOp& so, const FieldRef* fr, const float* tp, const float* tq,
                                                uint8_t* save, uint8_t* stage, int64_t i0, int lane) {
  const int* g = so.arg;
  const int z = OP == ADHA_OP_MUL ? g[2] : g[1];
  const int64_t r0 = i0 + (int64_t)lane * M;
  float x[M], v[M];
  ld_vec<float, M>(stage + fr[g[0]].s0 + lane * M * 4, x);
  if (save) {
    float old[M];
    ld_vec<float, M>(stage + fr[z].s0 + lane * M * 4, old);
    st_vec<float, M>(save + r0 * 4, old);
  }
  if (OP == ADHA_OP_MUL) {
    float y[M];
    ld_vec<float, M>(stage + fr[g[1]].s0 + lane * M * 4, y);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = __fmul_rn(x[m], y[m]);
  } else if (OP == ADHA_OP_AXPB) {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = __fadd_rn(__fmul_rn(so.par[0], x[m]), so.par[1]);
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = tanh_cf(x[m], tp, tq);
  }
  st_vec<float, M>(TO_STAGE ? stage + fr[z].s0 + lane * M * 4 : fr[z].g + r0 * 4, v);
}

template <int OP>
constexpr bool kVectorOp = OP == ADHA_OP_MIX || OP == ADHA_OP_AXPB || OP == ADHA_OP_MUL || OP == ADHA_OP_TANH;

// One record of one section: its fields through `rec` (staged chunk, global memory, or registers
// in a specialised window), fields read through the permutation from global memory (record pj),
// the old z to `save` when asked.  VOTE: the fp64 halving and widening take the integer forms
// behind a warp vote (every lane of the warp must run the call).  The field loops are unrolled
// where their bounds are compile-time constants (specialised windows), so that every field index
// folds to a constant there.
template <int OP, bool VOTE = false, class Rec>
__device__ __forceinline__ void run_record(const SecOp& so, const FieldRef* fr, const float* tp, const float* tq,
                                           uint8_t* save, const Rec& rec, int64_t i, int32_t pj) {
  const int* g = so.arg;
  if (OP == ADHA_OP_MADD3) {
    const float m = __fmul_rn(rec.template ld<float>(g[0]), rec.template ld<float>(g[1]));
    rec.template st<float>(g[2], __fadd_rn(m, rec.template ld<float>(g[2])));
  } else if (OP == ADHA_OP_XORSHIFT) {
    const uint32_t u = rec.template ld<uint32_t>(g[0]);
    rec.template st<uint32_t>(g[1], u ^ (u >> 3));
  } else if (OP == ADHA_OP_ADD) {
    rec.template st<float>(g[2], __fadd_rn(rec.template ld<float>(g[0]), rec.template ld<float>(g[1])));
  } else if (OP == ADHA_OP_MIX) {
    float s = 0.0f;
    uint32_t h = 0u;
ADHA_FIELD_LOOP
    for (int j = so.rd_off[ADHA_F32]; j < so.rd_off[ADHA_F32 + 1]; ++j) s = __fadd_rn(s, rec.template ld<float>(so.rd[j]));
ADHA_FIELD_LOOP
    for (int j = so.rd_off[ADHA_F64]; j < so.rd_off[ADHA_F64 + 1]; ++j) {
      const unsigned long long b = rec.template ld<unsigned long long>(so.rd[j]);
      h ^= (uint32_t)b ^ (uint32_t)(b >> 32);
    }
ADHA_FIELD_LOOP
    for (int j = so.rd_off[ADHA_I32]; j < so.rd_off[ADHA_I32 + 1]; ++j) h ^= rec.template ld<uint32_t>(so.rd[j]);
ADHA_FIELD_LOOP
    for (int j = so.rd_off[ADHA_BF16]; j < so.rd_off[ADHA_BF16 + 1]; ++j) h ^= (uint32_t)rec.template ld<uint16_t>(so.rd[j]);
    const float t = __fadd_rn(s, __fmul_rn(__uint2float_rn(h & 255u), 0.00390625f));
    const uint32_t k = (h ^ __float_as_uint(t)) >> 3;
ADHA_FIELD_LOOP
    for (int j = so.wr_off[ADHA_F32]; j < so.wr_off[ADHA_F32 + 1]; ++j) {
      const int f = so.wr[j];
      rec.template st<float>(f, __fadd_rn(__fmul_rn(rec.template ld<float>(f), 0.5f), t));
    }
    if (so.wr_off[ADHA_F64 + 1] > so.wr_off[ADHA_F64]) {
      const double td = VOTE ? widen_vote(t) : widen(t);
ADHA_FIELD_LOOP
      for (int j = so.wr_off[ADHA_F64]; j < so.wr_off[ADHA_F64 + 1]; ++j) {
        const int f = so.wr[j];
        const double x = rec.template ld<double>(f);
        rec.template st<double>(f, __dadd_rn(VOTE ? half_vote(x) : half_rn(x), td));
      }
    }
ADHA_FIELD_LOOP
    for (int j = so.wr_off[ADHA_I32]; j < so.wr_off[ADHA_I32 + 1]; ++j) {
      const int f = so.wr[j];
      rec.template st<uint32_t>(f, rec.template ld<uint32_t>(f) ^ k);
    }
ADHA_FIELD_LOOP
    for (int j = so.wr_off[ADHA_BF16]; j < so.wr_off[ADHA_BF16 + 1]; ++j) {
      const int f = so.wr[j];
      rec.template st<uint16_t>(f, (uint16_t)(rec.template ld<uint16_t>(f) ^ (uint16_t)(k & 0xFFFFu)));
    }
  } else if (OP == ADHA_OP_DRIFT) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float d = __fmul_rn(so.par[0], rec.template ld<float>(g[3 + ax]));
      float q = __fadd_rn(rec.template ld<float>(g[ax]), d);
      if (q >= 1.0f) q = __fsub_rn(q, 1.0f);
      else if (q < 0.0f) q = __fadd_rn(q, 1.0f);
      rec.template st<float>(g[ax], q);
    }
  } else if (OP == ADHA_OP_BIN) {
    const int G = (int)so.par[0];
    int c[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      int k = __float2int_rz(__fmul_rn(rec.template ld<float>(g[ax]), so.par[0]));
      k = k < 0 ? 0 : (k > G - 1 ? G - 1 : k);
      c[ax] = k;
    }
    rec.template st<int32_t>(g[3], c[0] + G * (c[1] + G * c[2]));
  } else if (OP == ADHA_OP_KE) {
    const float vx = rec.template ld<float>(g[0]), vy = rec.template ld<float>(g[1]),
                vz = rec.template ld<float>(g[2]);
    float s = __fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy));
    s = __fadd_rn(s, __fmul_rn(vz, vz));
    const float e = __fmul_rn(__fmul_rn(0.5f, rec.template ld<float>(g[3])), s);
    rec.template st<double>(g[4], VOTE ? widen_vote(e) : widen(e));
  } else if (OP == ADHA_OP_FLAGS) {
    const uint32_t fl = rec.template ld<uint32_t>(g[0]);
    const uint32_t bit = rec.template ld<double>(g[1]) > (double)so.par[0] ? 1u : 0u;
    rec.template st<uint32_t>(g[0], ((fl << 1) | bit) & 255u);
  } else if (OP == ADHA_OP_GATHER) {
    const int64_t j = pj;
    float pv[4];   // px, py, pz, q of record j
    if (so.gvec) {   // all four in one 16-byte struct: one load
      const uint8_t* base = fr[g[3]].g - 4 * so.gidx[0];
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(base + j * 16));
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int q = so.gidx[a];
        pv[a] = __uint_as_float(q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w);
      }
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a) pv[a] = gld<float>(fr, g[3 + a], j);
    }
    const float c = __fmul_rn(so.par[0], pv[3]);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float d = __fsub_rn(pv[ax], 0.5f);
      rec.template st<float>(g[ax], __fadd_rn(rec.template ld<float>(g[ax]), __fmul_rn(c, d)));
    }
  } else if (OP == ADHA_OP_KICK) {
    const float c = __fmul_rn(so.par[0], rec.template ld<float>(g[3]));
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
      rec.template st<float>(g[ax], __fadd_rn(rec.template ld<float>(g[ax]), __fmul_rn(c, so.par[1 + ax])));
  } else if (OP == ADHA_OP_ASSIGN) {
    // D_k summed over the features in ascending order, all K distances side by side
    const int K = so.arg[1], j0 = so.rd_off[ADHA_F32], d = so.rd_off[ADHA_F32 + 1] - j0;
    const float* cent = static_cast<const float*>(so.aux);
    float D[kMaxClusters];
#pragma unroll
    for (int k = 0; k < kMaxClusters; ++k) D[k] = 0.0f;
    for (int j = 0; j < d; ++j) {
      const float x = rec.template ld<float>(so.rd[j0 + j]);
#pragma unroll
      for (int k = 0; k < kMaxClusters; ++k)
        if (k < K) {
          const float df = __fsub_rn(x, __ldg(cent + k * d + j));
          D[k] = __fadd_rn(D[k], __fmul_rn(df, df));
        }
    }
    int best = 0;
    float bd = D[0];
#pragma unroll
    for (int k = 1; k < kMaxClusters; ++k)
      if (k < K && D[k] < bd) {
        bd = D[k];
        best = k;
      }
    rec.template st<int32_t>(g[0], best);
  } else {   // AXPB, MUL, TANH: z = op(x[, y]); the old z goes to `save` when asked
    const int z = OP == ADHA_OP_MUL ? g[2] : g[1];
    if (save) reinterpret_cast<float*>(save)[i] = rec.template ld<float>(z);
    const float x = rec.template ld<float>(g[0]);
    float v;
    if (OP == ADHA_OP_AXPB) v = __fadd_rn(__fmul_rn(so.par[0], x), so.par[1]);
    else if (OP == ADHA_OP_MUL) v = __fmul_rn(x, rec.template ld<float>(g[1]));
    else v = tanh_cf(x, tp, tq);
    rec.template st<float>(z, v);
  }
}

// Fixed-point value of a REDUCE feature: x * 2^23 (exact) rounded to the nearest integer, ties to
// even; 2^31 - 1 or -2^31 beyond the int32 range; 0 for NaN.  That is the float-to-int32
// conversion PTX defines (cvt.rni.s32.f32: the result clamped to the range, NaN to 0), so one
// conversion instruction does it.
__device__ __forceinline__ long long fixq(float x) {
  return (long long)__float2int_rn(__fmul_rn(x, 8388608.0f));
}

// ASSIGN's centroid table in shared memory, one per CTA: for feature j and cluster k the pair
// (c[k][j], c[k][j]) at cP[2*(j*8 + k)] (zero for k >= K), so one 16-byte load gives two
// clusters' pairs and a pair meets two records' values in one packed instruction.
// After the pairs, each feature's chunk-buffer offset and stride (int2), so that the per-chunk loop
// reads them with one broadcast shared load instead of indexed loads from the parameter space.
constexpr int kCentroidPairBytes = kMaxFields * kMaxClusters * 8 + kMaxFields * 8;

__device__ __forceinline__ void fill_centroid_pairs(const SecOp& so, const FieldRef* fr, float* cP, int tid,
                                                    int nthreads) {
  const int j0 = so.rd_off[ADHA_F32], K = so.arg[1], d = so.rd_off[ADHA_F32 + 1] - j0;
  const float* cent = static_cast<const float*>(so.aux);
  for (int t = tid; t < d * kMaxClusters; t += nthreads) {
    const int j = t / kMaxClusters, k = t - j * kMaxClusters;
    const float v = k < K ? __ldg(cent + k * d + j) : 0.0f;
    cP[2 * t] = v;
    cP[2 * t + 1] = v;
  }
  int2* off = reinterpret_cast<int2*>(cP + 2 * kMaxFields * kMaxClusters);
  for (int j = tid; j < d; j += nthreads) {
    const FieldRef& F = fr[so.rd[j0 + j]];
    off[j] = make_int2(F.s0, F.ss);
  }
}

// ASSIGN over the M records of each lane of a staged chunk (r = lane + 32m), for K clusters:
// feature by feature, its chunk offsets are looked up once for the lane's M records and its K
// centroid coordinates come from the CTA's pair table; the K x M distances are carried in
// registers, records paired (m, m + 1) in packed fp32 instructions when M is even.  Each half
// is the per-record rule itself: D_k = ((+0 + sq_0) + sq_1) + ..., sq_j = (x_j - c_kj)^2, every
// operation rounded to nearest on its own, features in ascending order.
template <int M, int K>
__device__ __forceinline__ void assign_chunk_k(const SecOp& so, const FieldRef* fr, uint8_t* stage, int64_t i0,
                                               int lane, const float* cP) {
  const int d = so.rd_off[ADHA_F32 + 1] - so.rd_off[ADHA_F32];
  constexpr int H = (M + 1) / 2;   // register pairs per cluster
  unsigned long long D[K][H];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int h = 0; h < H; ++h) D[k][h] = 0ull;   // +0.0f in both halves
  const int2* off = reinterpret_cast<const int2*>(cP + 2 * kMaxFields * kMaxClusters);
  for (int j = 0; j < d; ++j) {
    const int2 F = off[j];   // chunk-buffer offset and stride of feature j
    const uint8_t* p = stage + F.x + lane * F.y;
    const int step = 32 * F.y;
    unsigned long long x2[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float lo = *reinterpret_cast<const float*>(p + (2 * h) * step);
      const float hi = 2 * h + 1 < M ? *reinterpret_cast<const float*>(p + (2 * h + 1) * step) : 0.0f;
      x2[h] = f2_pack(lo, hi);
    }
    const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(cP + 2 * j * kMaxClusters);
    unsigned long long c2[K + 1];
#pragma unroll
    for (int k = 0; k < K; k += 2) {
      const ulonglong2 v = cp[k / 2];
      c2[k] = v.x;
      c2[k + 1] = v.y;
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const unsigned long long df = f2_sub_rn(x2[h], c2[k]);
        D[k][h] = f2_add_rn(D[k][h], f2_mul_rn(df, df));
      }
  }
#pragma unroll
  for (int h = 0; h < H; ++h) {
    float Dl[K], Dh[K];
#pragma unroll
    for (int k = 0; k < K; ++k) f2_unpack(D[k][h], &Dl[k], &Dh[k]);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int m = 2 * h + e;
      if (m >= M) break;
      const float* Dm = e ? Dh : Dl;
      int best = 0;
      float bd = Dm[0];
#pragma unroll
      for (int k = 1; k < K; ++k)
        if (Dm[k] < bd) {
          bd = Dm[k];
          best = k;
        }
      const int r = lane + 32 * m;
      StagedRec{fr, stage, r, i0 + r}.template st<int32_t>(so.arg[0], best);
    }
  }
}

template <int M>
__device__ __forceinline__ void assign_chunk(const SecOp& so, const FieldRef* fr, uint8_t* stage, int64_t i0, int lane,
                                             const float* cT) {
  switch (so.arg[1]) {   // K, uniform over the launch
    case 1: assign_chunk_k<M, 1>(so, fr, stage, i0, lane, cT); break;
    case 2: assign_chunk_k<M, 2>(so, fr, stage, i0, lane, cT); break;
    case 3: assign_chunk_k<M, 3>(so, fr, stage, i0, lane, cT); break;
    case 4: assign_chunk_k<M, 4>(so, fr, stage, i0, lane, cT); break;
    case 5: assign_chunk_k<M, 5>(so, fr, stage, i0, lane, cT); break;
    case 6: assign_chunk_k<M, 6>(so, fr, stage, i0, lane, cT); break;
    case 7: assign_chunk_k<M, 7>(so, fr, stage, i0, lane, cT); break;
    default: assign_chunk_k<M, 8>(so, fr, stage, i0, lane, cT); break;
  }
}

// Where a REDUCE lane finds its feature (lane j = feature j, if j < d) and the membership in a
// staged chunk; looked up once per kernel, since the lanes index the field table differently.
struct ReduceLane {
  int d, K;
  int sx, ssx, sm, ssm;   // chunk-buffer offset and stride of the lane's feature and of the membership
  int skew;               // one-field feature slice: the lane starts at its own record (spread banks)
  bool walk;              // sum cluster by cluster into registers (see reduce_chunk_any)
};

// Shared memory of a REDUCE per CTA: the two sum tables of every warp (when it does not walk) and
// every warp's 32-entry record list.
constexpr size_t kReduceTableBytes = (size_t)kWarps * 2 * (kMaxClusters + 1) * 32 * 8;
constexpr size_t kReduceListBytes = (size_t)kWarps * 32 * 4;

// walk: every feature lies in a slice wider than one field (decided on the host, which sizes the
// shared tables only for the other way).
__device__ __forceinline__ ReduceLane reduce_lane(const SecOp& so, const FieldRef* fr, int lane, bool walk) {
  ReduceLane q;
  const int j0 = so.rd_off[ADHA_F32];
  q.d = so.rd_off[ADHA_F32 + 1] - j0;
  q.K = so.arg[1];
  const FieldRef& Fm = fr[so.arg[0]];
  q.sm = Fm.s0;
  q.ssm = Fm.ss;
  q.sx = q.ssx = 0;
  if (lane < q.d) {
    const FieldRef& Fx = fr[so.rd[j0 + lane]];
    q.sx = Fx.s0;
    q.ssx = Fx.ss;
  }
  q.skew = q.ssx == 4 ? lane : 0;
  q.walk = walk;
  return q;
}

template <int M>
__device__ __forceinline__ void reduce_sums(const ReduceLane& q, const uint8_t* stage, int lane,
                                            long long* __restrict__ acc, long long* __restrict__ acc2);

// REDUCE over the R = 32*M records of a staged chunk.  Counts: lane = record, one ballot per
// cluster, lane k keeping cluster k's count (one register).
// Sums, lane j = feature j, integer sums (any order gives the same result):
// * walk (every feature in a slice wider than one field, e.g. AoS): for each group of 32 records
//   the warp lists the records cluster by cluster (a counting sort by ballots into the warp's
//   32-entry list `idx`), then, cluster by cluster, all lanes read the same listed record
//   (consecutive words of a struct) four records at a time, adding into the register sums
//   sum[k]: no shared-memory accumulator and no chain through memory;
// * else (one-field slices, where the lanes reading one record would all hit one bank): each
//   lane starts at its own record and adds every record into its row of two (K+1) x 32 tables in
//   shared memory, even records into the first and odd into the second, so that two
//   read-add-write chains are in flight (row K takes memberships outside [0, K)).
template <int M>
__device__ __forceinline__ void reduce_chunk_any(const ReduceLane& q, const uint8_t* stage, int lane,
                                                 long long* __restrict__ acc, long long* __restrict__ acc2,
                                                 int* __restrict__ idx, long long (&sum)[kMaxClusters],
                                                 unsigned long long* cnt) {
  if (q.walk) {
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int mm = *reinterpret_cast<const int32_t*>(stage + q.sm + (lane + 32 * m) * q.ssm);
      unsigned b[kMaxClusters];
      int start = 0;
#pragma unroll
      for (int k = 0; k < kMaxClusters; ++k) {
        b[k] = k < q.K ? __ballot_sync(0xFFFFFFFFu, mm == k) : 0u;
        const int c = __popc(b[k]);
        if (lane == k) *cnt += (unsigned long long)c;
        if (k < q.K && mm == k) idx[start + __popc(b[k] & lt)] = lane;
        start += c;
      }
      __syncwarp();
      if (lane < q.d) {
        const uint8_t* px = stage + q.sx + 32 * m * q.ssx;
        int e = 0;
#pragma unroll
        for (int k = 0; k < kMaxClusters; ++k) {
          int t = e;
          e += __popc(b[k]);
          long long s = 0;
          for (; t + 4 <= e; t += 4) {
            const int r0 = idx[t], r1 = idx[t + 1], r2 = idx[t + 2], r3 = idx[t + 3];
            const float x0 = *reinterpret_cast<const float*>(px + r0 * q.ssx);
            const float x1 = *reinterpret_cast<const float*>(px + r1 * q.ssx);
            const float x2 = *reinterpret_cast<const float*>(px + r2 * q.ssx);
            const float x3 = *reinterpret_cast<const float*>(px + r3 * q.ssx);
            s += (fixq(x0) + fixq(x1)) + (fixq(x2) + fixq(x3));
          }
          for (; t < e; ++t) s += fixq(*reinterpret_cast<const float*>(px + idx[t] * q.ssx));
          sum[k] += s;
        }
      }
      __syncwarp();   // the list is rewritten for the next 32 records
    }
    return;
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int mm = *reinterpret_cast<const int32_t*>(stage + q.sm + (lane + 32 * m) * q.ssm);
#pragma unroll
    for (int k = 0; k < kMaxClusters; ++k)
      if (k < q.K) {
        const unsigned b = __ballot_sync(0xFFFFFFFFu, mm == k);
        if (lane == k) *cnt += (unsigned long long)__popc(b);
      }
  }
  reduce_sums<M>(q, stage, lane, acc, acc2);
}


template <int M>
__device__ __forceinline__ void reduce_sums(const ReduceLane& q, const uint8_t* stage, int lane,
                                            long long* __restrict__ acc, long long* __restrict__ acc2) {
  constexpr int R = 32 * M;
  if (lane < q.d) {
    long long* __restrict__ col = acc + lane;
    long long* __restrict__ col2 = acc2 + lane;
    const uint8_t* pm = stage + q.sm;
    const uint8_t* px = stage + q.sx;
#pragma unroll 2
    for (int i = 0; i < R; i += 2) {
      const int r0 = (i + q.skew) & (R - 1), r1 = (i + 1 + q.skew) & (R - 1);
      const int m0 = *reinterpret_cast<const int32_t*>(pm + r0 * q.ssm);
      const int m1 = *reinterpret_cast<const int32_t*>(pm + r1 * q.ssm);
      const long long v0 = fixq(*reinterpret_cast<const float*>(px + r0 * q.ssx));
      const long long v1 = fixq(*reinterpret_cast<const float*>(px + r1 * q.ssx));
      // a membership outside [0, K) goes to the scratch row kMaxClusters, never read back
      const int row0 = (unsigned)m0 < (unsigned)q.K ? m0 : kMaxClusters;
      const int row1 = (unsigned)m1 < (unsigned)q.K ? m1 : kMaxClusters;
      col[row0 * 32] += v0;
      col2[row1 * 32] += v1;
    }
  }
}

// REDUCE over records [t0, n) read from global memory (the ragged tail): lane j = feature j,
// lane k counts cluster k; sums into the register sums (walk) or row mm of the first shared table.
__device__ __forceinline__ void reduce_tail(const ReduceLane& q, const SecOp& so, const FieldRef* fr, int64_t t0,
                                            int64_t n, int lane, long long* acc, long long (&sum)[kMaxClusters],
                                            unsigned long long* cnt) {
  const FieldRef& Fm = fr[so.arg[0]];
  const int j0 = so.rd_off[ADHA_F32];
  for (int64_t i = t0; i < n; ++i) {
    const int mm = *reinterpret_cast<const int32_t*>(Fm.g + i * Fm.gs);
    if ((unsigned)mm >= (unsigned)q.K) continue;
    if (lane == mm) *cnt += 1ull;
    if (lane < q.d) {
      const FieldRef& Fx = fr[so.rd[j0 + lane]];
      const long long v = fixq(*reinterpret_cast<const float*>(Fx.g + i * Fx.gs));
      if (q.walk) {
#pragma unroll
        for (int k = 0; k < kMaxClusters; ++k) sum[k] += k == mm ? v : 0ll;
      } else {
        acc[mm * 32 + lane] += v;
      }
    }
  }
}

// The warp's sums and counts added into the result (K rows of [count, d sums], zeroed before
// the launch unless the caller accumulates).
__device__ __forceinline__ void reduce_flush(const ReduceLane& q, const SecOp& so, int lane, const long long* acc,
                                             const long long (&sum)[kMaxClusters], const unsigned long long* cnt) {
  unsigned long long* out = static_cast<unsigned long long*>(const_cast<void*>(so.aux));
  const int d = q.d;
#pragma unroll
  for (int k = 0; k < kMaxClusters; ++k)
    if (k < q.K) {
      if (lane < d) {
        const long long v = q.walk ? sum[k] : acc[k * 32 + lane] + acc[(kMaxClusters + 1 + k) * 32 + lane];
        atomicAdd(out + (size_t)k * (d + 1) + 1 + lane, (unsigned long long)v);
      }
    }
  if (lane < q.K) atomicAdd(out + (size_t)lane * (d + 1), *cnt);
}

}  // namespace adha

// sections.cu -- layout-templated section kernels (paper Section 2: a section is one
// data-parallel loop; its layout decides which bytes it drags through memory) and the reverse
// (adjoint) kernel of the fp32 chain sections.
//
// The forward kernel works per warp on chunks of R = 32*M records, like remap.cu: it copies the
// chunk's slice of every group that holds a field the section reads into its own shared buffer
// (16-byte cp.async, one chunk ahead), computes the M records of each lane from the staged
// bytes, and stores the written fields straight to global memory (a partial-record store
// touches only the sectors of the written field).  The op is a template parameter; the layout is
// the FieldRef table (where each field sits in the stage and in global memory).  Every floating
// operation is an explicitly rounded-to-nearest intrinsic, so no contraction can change a bit.
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"

namespace adha {

// per-CTA slice table at the start of shared memory: pointers, slice ends, write-back flags
constexpr int kSectionTable = (16 * (kMaxGroups + 1) + 15) / 16 * 16;

struct StagedRec {      // record r of a staged chunk (global record i)
  const SectionArgs* a;
  uint8_t* stage;
  int r;
  int64_t i;
  template <class V>
  __device__ __forceinline__ V ld(int f) const {
    const FieldRef& F = a->f[f];
    if (F.s0 >= 0) return *reinterpret_cast<const V*>(stage + F.s0 + r * F.ss);
    return *reinterpret_cast<const V*>(F.g + i * F.gs);
  }
  template <class V>
  __device__ __forceinline__ void st(int f, V v) const {
    const FieldRef& F = a->f[f];
    if (F.wsm) *reinterpret_cast<V*>(stage + F.s0 + r * F.ss) = v;
    else *reinterpret_cast<V*>(F.g + i * F.gs) = v;
  }
};

struct GlobalRec {      // record i in global memory (ragged tail)
  const SectionArgs* a;
  int64_t i;
  template <class V>
  __device__ __forceinline__ V ld(int f) const {
    const FieldRef& F = a->f[f];
    return *reinterpret_cast<const V*>(F.g + i * F.gs);
  }
  template <class V>
  __device__ __forceinline__ void st(int f, V v) const {
    const FieldRef& F = a->f[f];
    *reinterpret_cast<V*>(F.g + i * F.gs) = v;
  }
};

template <class V>
__device__ __forceinline__ V gld(const SectionArgs& a, int f, int64_t i) {
  return __ldg(reinterpret_cast<const V*>(a.f[f].g + i * a.f[f].gs));
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
__device__ __forceinline__ void mix_chunk(const SectionArgs& a, uint8_t* stage, int64_t i0, int lane) {
  float s[M];
  uint32_t h[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    s[m] = 0.0f;
    h[m] = 0u;
  }
  // V value of field F for the lane's record m: from the chunk buffer if staged, else global
#define ADHA_MIX_READ(V, LIST, BODY)                                                        \
  for (int j = 0; j < a.n_rd[LIST]; ++j) {                                                  \
    const FieldRef& F = a.f[a.rd[LIST][j]];                                                 \
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
  for (int j = 0; j < a.n_wr[LIST]; ++j) {                                                  \
    const FieldRef& F = a.f[a.wr[LIST][j]];                                                 \
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
  ADHA_MIX_WRITE(double, ADHA_F64, __dadd_rn(__dmul_rn(old, 0.5), (double)t[m]))
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
// each field is one vector load from the chunk buffer and one vector store to global memory.
template <int M>
__device__ __forceinline__ void mix_chunk_vec(const SectionArgs& a, const uint8_t* stage, int64_t i0, int lane) {
  float s[M];
  uint32_t h[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    s[m] = 0.0f;
    h[m] = 0u;
  }
  for (int j = 0; j < a.n_rd[ADHA_F32]; ++j) {
    float v[M];
    ld_vec<float, M>(stage + a.f[a.rd[ADHA_F32][j]].s0 + lane * M * 4, v);
#pragma unroll
    for (int m = 0; m < M; ++m) s[m] = __fadd_rn(s[m], v[m]);
  }
  for (int j = 0; j < a.n_rd[ADHA_F64]; ++j) {
    unsigned long long v[M];
    ld_vec<unsigned long long, M>(stage + a.f[a.rd[ADHA_F64][j]].s0 + lane * M * 8, v);
#pragma unroll
    for (int m = 0; m < M; ++m) h[m] ^= (uint32_t)v[m] ^ (uint32_t)(v[m] >> 32);
  }
  for (int j = 0; j < a.n_rd[ADHA_I32]; ++j) {
    uint32_t v[M];
    ld_vec<uint32_t, M>(stage + a.f[a.rd[ADHA_I32][j]].s0 + lane * M * 4, v);
#pragma unroll
    for (int m = 0; m < M; ++m) h[m] ^= v[m];
  }
  for (int j = 0; j < a.n_rd[ADHA_BF16]; ++j) {
    uint16_t v[M];
    ld_vec<uint16_t, M>(stage + a.f[a.rd[ADHA_BF16][j]].s0 + lane * M * 2, v);
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
  for (int j = 0; j < a.n_wr[ADHA_F32]; ++j) {
    const FieldRef& F = a.f[a.wr[ADHA_F32][j]];
    float v[M];
    ld_vec<float, M>(stage + F.s0 + lane * M * 4, v);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = __fadd_rn(__fmul_rn(v[m], 0.5f), t[m]);
    st_vec<float, M>(F.g + r0 * 4, v);
  }
  for (int j = 0; j < a.n_wr[ADHA_F64]; ++j) {
    const FieldRef& F = a.f[a.wr[ADHA_F64][j]];
    double v[M];
    ld_vec<double, M>(stage + F.s0 + lane * M * 8, v);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = __dadd_rn(__dmul_rn(v[m], 0.5), (double)t[m]);
    st_vec<double, M>(F.g + r0 * 8, v);
  }
  for (int j = 0; j < a.n_wr[ADHA_I32]; ++j) {
    const FieldRef& F = a.f[a.wr[ADHA_I32][j]];
    uint32_t v[M];
    ld_vec<uint32_t, M>(stage + F.s0 + lane * M * 4, v);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] ^= k[m];
    st_vec<uint32_t, M>(F.g + r0 * 4, v);
  }
  for (int j = 0; j < a.n_wr[ADHA_BF16]; ++j) {
    const FieldRef& F = a.f[a.wr[ADHA_BF16][j]];
    uint16_t v[M];
    ld_vec<uint16_t, M>(stage + F.s0 + lane * M * 2, v);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = (uint16_t)(v[m] ^ (uint16_t)(k[m] & 0xFFFFu));
    st_vec<uint16_t, M>(F.g + r0 * 2, v);
  }
}

// AXPB, MUL, TANH under the vector mapping (x, y, z each a one-field group): lane takes records
// lane*M + m; x, y and the old z come from the chunk buffer (the values before the section, so
// any aliasing of x, y, z reads what the per-record rule reads), z and `save` get vector stores.
template <int OP, int M>
__device__ __forceinline__ void chain_chunk_vec(const SectionArgs& a, const uint8_t* stage, int64_t i0, int lane) {
  const int* g = a.arg;
  const int z = OP == ADHA_OP_MUL ? g[2] : g[1];
  const int64_t r0 = i0 + (int64_t)lane * M;
  float x[M], v[M];
  ld_vec<float, M>(stage + a.f[g[0]].s0 + lane * M * 4, x);
  if (a.save) {
    float old[M];
    ld_vec<float, M>(stage + a.f[z].s0 + lane * M * 4, old);
    st_vec<float, M>(a.save + r0 * 4, old);
  }
  if (OP == ADHA_OP_MUL) {
    float y[M];
    ld_vec<float, M>(stage + a.f[g[1]].s0 + lane * M * 4, y);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = __fmul_rn(x[m], y[m]);
  } else if (OP == ADHA_OP_AXPB) {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = __fadd_rn(__fmul_rn(a.par[0], x[m]), a.par[1]);
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = tanh_cf(x[m], a.tanh_p, a.tanh_q);
  }
  st_vec<float, M>(a.f[z].g + r0 * 4, v);
}

template <int OP>
constexpr bool kVectorOp = OP == ADHA_OP_MIX || OP == ADHA_OP_AXPB || OP == ADHA_OP_MUL || OP == ADHA_OP_TANH;

template <int OP, class Rec>
__device__ __forceinline__ void run_record(const SectionArgs& a, const Rec& rec, int64_t i, int32_t pj) {
  const int* g = a.arg;
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
    for (int j = 0; j < a.n_rd[ADHA_F32]; ++j) s = __fadd_rn(s, rec.template ld<float>(a.rd[ADHA_F32][j]));
    for (int j = 0; j < a.n_rd[ADHA_F64]; ++j) {
      const unsigned long long b = rec.template ld<unsigned long long>(a.rd[ADHA_F64][j]);
      h ^= (uint32_t)b ^ (uint32_t)(b >> 32);
    }
    for (int j = 0; j < a.n_rd[ADHA_I32]; ++j) h ^= rec.template ld<uint32_t>(a.rd[ADHA_I32][j]);
    for (int j = 0; j < a.n_rd[ADHA_BF16]; ++j) h ^= (uint32_t)rec.template ld<uint16_t>(a.rd[ADHA_BF16][j]);
    const float t = __fadd_rn(s, __fmul_rn(__uint2float_rn(h & 255u), 0.00390625f));
    const uint32_t k = (h ^ __float_as_uint(t)) >> 3;
    for (int j = 0; j < a.n_wr[ADHA_F32]; ++j) {
      const int f = a.wr[ADHA_F32][j];
      rec.template st<float>(f, __fadd_rn(__fmul_rn(rec.template ld<float>(f), 0.5f), t));
    }
    if (a.n_wr[ADHA_F64]) {
      const double td = (double)t;
      for (int j = 0; j < a.n_wr[ADHA_F64]; ++j) {
        const int f = a.wr[ADHA_F64][j];
        rec.template st<double>(f, __dadd_rn(__dmul_rn(rec.template ld<double>(f), 0.5), td));
      }
    }
    for (int j = 0; j < a.n_wr[ADHA_I32]; ++j) {
      const int f = a.wr[ADHA_I32][j];
      rec.template st<uint32_t>(f, rec.template ld<uint32_t>(f) ^ k);
    }
    for (int j = 0; j < a.n_wr[ADHA_BF16]; ++j) {
      const int f = a.wr[ADHA_BF16][j];
      rec.template st<uint16_t>(f, (uint16_t)(rec.template ld<uint16_t>(f) ^ (uint16_t)(k & 0xFFFFu)));
    }
  } else if (OP == ADHA_OP_DRIFT) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float d = __fmul_rn(a.par[0], rec.template ld<float>(g[3 + ax]));
      float q = __fadd_rn(rec.template ld<float>(g[ax]), d);
      if (q >= 1.0f) q = __fsub_rn(q, 1.0f);
      else if (q < 0.0f) q = __fadd_rn(q, 1.0f);
      rec.template st<float>(g[ax], q);
    }
  } else if (OP == ADHA_OP_BIN) {
    const int G = (int)a.par[0];
    int c[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      int k = __float2int_rz(__fmul_rn(rec.template ld<float>(g[ax]), a.par[0]));
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
    rec.template st<double>(g[4], (double)e);
  } else if (OP == ADHA_OP_FLAGS) {
    const uint32_t fl = rec.template ld<uint32_t>(g[0]);
    const uint32_t bit = rec.template ld<double>(g[1]) > (double)a.par[0] ? 1u : 0u;
    rec.template st<uint32_t>(g[0], ((fl << 1) | bit) & 255u);
  } else if (OP == ADHA_OP_GATHER) {
    const int64_t j = pj;
    const float c = __fmul_rn(a.par[0], gld<float>(a, g[6], j));
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float d = __fsub_rn(gld<float>(a, g[3 + ax], j), 0.5f);
      rec.template st<float>(g[ax], __fadd_rn(rec.template ld<float>(g[ax]), __fmul_rn(c, d)));
    }
  } else if (OP == ADHA_OP_KICK) {
    const float c = __fmul_rn(a.par[0], rec.template ld<float>(g[3]));
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
      rec.template st<float>(g[ax], __fadd_rn(rec.template ld<float>(g[ax]), __fmul_rn(c, a.par[1 + ax])));
  } else {   // AXPB, MUL, TANH: z = op(x[, y]); the old z goes to `save` when asked
    const int z = OP == ADHA_OP_MUL ? g[2] : g[1];
    if (a.save) reinterpret_cast<float*>(a.save)[i] = rec.template ld<float>(z);
    const float x = rec.template ld<float>(g[0]);
    float v;
    if (OP == ADHA_OP_AXPB) v = __fadd_rn(__fmul_rn(a.par[0], x), a.par[1]);
    else if (OP == ADHA_OP_MUL) v = __fmul_rn(x, rec.template ld<float>(g[1]));
    else v = tanh_cf(x, a.tanh_p, a.tanh_q);
    rec.template st<float>(z, v);
  }
}

template <int OP, int M, bool VEC>
__global__ void __launch_bounds__(kThreads) section_kernel(const __grid_constant__ SectionArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int n_slices = a.n_load + (a.perm_slot >= 0 ? 1 : 0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // slice table: base pointer and byte range of each staged slice within a chunk buffer
  const uint8_t** sp = reinterpret_cast<const uint8_t**>(smem);
  int* send = reinterpret_cast<int*>(smem + 8 * (kMaxGroups + 1));
  int* wback = send + (kMaxGroups + 1);
  uint8_t* buf0 = smem + kSectionTable + (size_t)warp * 2 * a.in_bytes;
  uint8_t* buf1 = buf0 + a.in_bytes;
  constexpr int R = 32 * M;
  for (int k = tid; k < n_slices; k += kThreads) {
    sp[k] = a.load[k].ptr;
    send[k] = a.load[k].start + R * a.load[k].stride;
    wback[k] = a.writeback[k];
  }
  __syncthreads();

  const int64_t W = (int64_t)gridDim.x * kWarps;
  // The chunk's slices are contiguous in the buffer and each a multiple of 64 bytes, so the
  // warp walks the whole buffer in 16-byte pieces (512 bytes per step, every lane busy); piece
  // p of slice g comes from byte (ch*R*stride_g + p - start_g) of group g.
  auto stage = [&](int64_t ch, uint8_t* buf) {
    int g = 0, start = 0;
    for (int p = lane * 16; p < a.in_bytes; p += 512) {
      while (p >= send[g]) start = send[g++];
      const int64_t stride = (send[g] - start) / R;
      cp_async16(buf + p, sp[g] + ch * (R * stride) + (p - start));
    }
  };

  int64_t c = (int64_t)blockIdx.x * kWarps + warp;
  if (c < a.n_chunks) stage(c, buf0);
  cp_async_commit();
  for (int i = 0; c < a.n_chunks; c += W, ++i) {
    uint8_t* cur = (i & 1) ? buf1 : buf0;
    if (c + W < a.n_chunks) stage(c + W, (i & 1) ? buf0 : buf1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    const int64_t i0 = c * R;
    if (OP == ADHA_OP_MIX && VEC) {
      mix_chunk_vec<M>(a, cur, i0, lane);
    } else if (VEC) {
      chain_chunk_vec<OP, M>(a, cur, i0, lane);
    } else if (OP == ADHA_OP_MIX) {
      mix_chunk<M>(a, cur, i0, lane);
    } else {
      const int32_t* ps = a.perm_slot >= 0 ? reinterpret_cast<const int32_t*>(cur + a.load[a.perm_slot].start) : nullptr;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int r = lane + 32 * m;
        run_record<OP>(a, StagedRec{&a, cur, r, i0 + r}, i0 + r, ps ? ps[r] : 0);
      }
    }
    if (a.n_writeback) {   // wide written groups go back whole, 16 bytes per lane per step
      __syncwarp();
      int g = 0, start = 0;
      for (int p = lane * 16; p < a.in_bytes; p += 512) {
        while (p >= send[g]) start = send[g++];
        if (wback[g]) {
          const int64_t stride = (send[g] - start) / R;
          *reinterpret_cast<uint4*>(const_cast<uint8_t*>(sp[g]) + c * (R * stride) + (p - start)) =
              *reinterpret_cast<const uint4*>(cur + p);
        }
      }
    }
    __syncwarp();
  }
  cp_async_wait<0>();

  // ragged tail: the warp whose next chunk would be n_chunks
  const int64_t t0 = a.n_chunks * R;
  if (c == a.n_chunks && t0 < a.n) {
    for (int64_t i = t0 + lane; i < a.n; i += 32) run_record<OP>(a, GlobalRec{&a, i}, i, a.perm_slot >= 0 ? a.perm[i] : 0);
  }
}

// Reverse of one fp32 chain section (AXPB, MUL, TANH).  Every value a record needs is loaded
// first (4 records per thread, independent loads), the oracle's sequential update
//   restore z; gz = g[z]; g[z] = 0; then g[x] (and g[y]) += ...
// is carried out in registers with the aliasing of x, y, z resolved explicitly (they are
// launch-uniform), and the results are stored last.
template <int OP>
__device__ __forceinline__ void backward_record(const BackwardArgs& a, int64_t i, float sv, float xs, float ys,
                                                float gz, float gx, float gy) {
  const bool xz = a.x == a.z, yz = a.y == a.z, xy = a.x == a.y;
  const float xo = xz ? sv : xs;                   // x before the section
  const float yo = yz ? sv : ys;
  float gxn = xz ? 0.0f : gx;                      // after g[z] = 0
  if (OP == ADHA_OP_AXPB) {
    gxn = __fadd_rn(gxn, __fmul_rn(a.a, gz));
  } else if (OP == ADHA_OP_TANH) {
    const float t = tanh_cf(xo, a.tanh_p, a.tanh_q);
    gxn = __fadd_rn(gxn, __fmul_rn(gz, __fsub_rn(1.0f, __fmul_rn(t, t))));
  } else {
    gxn = __fadd_rn(gxn, __fmul_rn(gz, yo));
    float gyn = xy ? gxn : (yz ? 0.0f : gy);
    gyn = __fadd_rn(gyn, __fmul_rn(gz, xo));
    *reinterpret_cast<float*>(a.g[1] + i * a.gs[1]) = gyn;
    if (!xy) *reinterpret_cast<float*>(a.g[0] + i * a.gs[0]) = gxn;
    if (!xz && !yz) *reinterpret_cast<float*>(a.g[2] + i * a.gs[2]) = 0.0f;
    *reinterpret_cast<float*>(a.s[2] + i * a.ss[2]) = sv;
    return;
  }
  *reinterpret_cast<float*>(a.g[0] + i * a.gs[0]) = gxn;
  if (!xz) *reinterpret_cast<float*>(a.g[2] + i * a.gs[2]) = 0.0f;
  *reinterpret_cast<float*>(a.s[2] + i * a.ss[2]) = sv;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) backward_kernel(const __grid_constant__ BackwardArgs a) {
  constexpr int K = 4;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const bool need_y = OP == ADHA_OP_MUL;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < a.n; base += K * T) {
    float sv[K], xs[K], ys[K], gz[K], gx[K], gy[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t i = base + k * T;
      if (i < a.n) {
        sv[k] = a.save[i];
        xs[k] = *reinterpret_cast<const float*>(a.s[0] + i * a.ss[0]);
        ys[k] = need_y ? *reinterpret_cast<const float*>(a.s[1] + i * a.ss[1]) : 0.0f;
        gz[k] = *reinterpret_cast<const float*>(a.g[2] + i * a.gs[2]);
        gx[k] = *reinterpret_cast<const float*>(a.g[0] + i * a.gs[0]);
        gy[k] = need_y ? *reinterpret_cast<const float*>(a.g[1] + i * a.gs[1]) : 0.0f;
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t i = base + k * T;
      if (i < a.n) backward_record<OP>(a, i, sv[k], xs[k], ys[k], gz[k], gx[k], gy[k]);
    }
  }
}

size_t section_smem_bytes(const SectionArgs& a) { return kSectionTable + (size_t)kWarps * 2 * a.in_bytes; }

template <int OP, int M, bool VEC>
static int launch_om(const SectionArgs& a, int grid, size_t smem, void* stream) {
  cudaError_t e = cudaFuncSetAttribute(section_kernel<OP, M, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(section)");
  section_kernel<OP, M, VEC><<<grid, kThreads, smem, (cudaStream_t)stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "section kernel launch");
  return 0;
}

template <int OP>
static int launch_op(const SectionArgs& a, int grid, size_t smem, void* stream) {
  if constexpr (kVectorOp<OP>) {
    if (a.vec && a.R == 64) return launch_om<OP, 2, true>(a, grid, smem, stream);
    if (a.vec && a.R == 128) return launch_om<OP, 4, true>(a, grid, smem, stream);
  }
  switch (a.R) {
    case 32: return launch_om<OP, 1, false>(a, grid, smem, stream);
    case 64: return launch_om<OP, 2, false>(a, grid, smem, stream);
    default: return launch_om<OP, 4, false>(a, grid, smem, stream);
  }
}

template <int OP>
static int occ_op(size_t smem, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(section_kernel<OP, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(section)");
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, section_kernel<OP, 1, false>, kThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(section)");
  return 0;
}

#define ADHA_FOR_EACH_OP(X)                                                                              \
  X(ADHA_OP_MADD3) X(ADHA_OP_XORSHIFT) X(ADHA_OP_ADD) X(ADHA_OP_MIX) X(ADHA_OP_DRIFT) X(ADHA_OP_BIN)     \
  X(ADHA_OP_KE) X(ADHA_OP_FLAGS) X(ADHA_OP_GATHER) X(ADHA_OP_KICK) X(ADHA_OP_AXPB) X(ADHA_OP_MUL)        \
  X(ADHA_OP_TANH)

int launch_section(const SectionArgs& a, int grid, size_t smem, void* stream) {
  switch (a.op) {
#define X(op) case op: return launch_op<op>(a, grid, smem, stream);
    ADHA_FOR_EACH_OP(X)
#undef X
    default: return fail(ADHA_EINVAL, "unknown section op %d", a.op);
  }
}

int section_occupancy(int op, size_t smem, int* blocks) {
  switch (op) {
#define X(o) case o: return occ_op<o>(smem, blocks);
    ADHA_FOR_EACH_OP(X)
#undef X
    default: return fail(ADHA_EINVAL, "unknown section op %d", op);
  }
}

int launch_backward(const BackwardArgs& a, void* stream) {
  int sms = 0;
  if (int rc = sm_count(&sms)) return rc;
  int64_t blocks = (a.n + 4 * kThreads - 1) / (4 * kThreads);
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (blocks < 1) blocks = 1;
  if (a.op == ADHA_OP_AXPB) backward_kernel<ADHA_OP_AXPB><<<(int)blocks, kThreads, 0, (cudaStream_t)stream>>>(a);
  else if (a.op == ADHA_OP_MUL) backward_kernel<ADHA_OP_MUL><<<(int)blocks, kThreads, 0, (cudaStream_t)stream>>>(a);
  else backward_kernel<ADHA_OP_TANH><<<(int)blocks, kThreads, 0, (cudaStream_t)stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "backward kernel launch");
  return 0;
}

}  // namespace adha

// sections.cu -- layout-templated section kernels (paper Section 2: a section is one
// data-parallel loop; its layout decides which bytes it drags through memory) and the reverse
// (adjoint) kernel of the fp32 chain sections.
//
// The forward kernel works per warp on chunks of R records, like remap.cu: it copies the chunk's
// slice of every group that holds a field the section reads into its own shared buffer (16-byte
// cp.async, one chunk ahead), computes each record from the staged bytes, and stores the
// written fields straight to global memory (a partial-record store touches only the sectors of
// the written field).  The op is a template parameter; the layout is
// the FieldRef table (where each field sits in the stage and in global memory).  Every floating
// operation is an explicitly rounded-to-nearest intrinsic, so no contraction can change a bit.
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"

namespace adha {

struct StagedRec {      // loads from the stage tile
  const SectionArgs* a;
  const uint8_t* stage;
  int r;
  template <class V>
  __device__ __forceinline__ V ld(int f) const {
    const FieldRef& F = a->f[f];
    return *reinterpret_cast<const V*>(stage + F.s0 + r * F.ss);
  }
};

struct GlobalRec {      // loads from global memory (ragged tail)
  const SectionArgs* a;
  int64_t i;
  template <class V>
  __device__ __forceinline__ V ld(int f) const {
    const FieldRef& F = a->f[f];
    return *reinterpret_cast<const V*>(F.g + i * F.gs);
  }
};

template <class V>
__device__ __forceinline__ void gst(const SectionArgs& a, int f, int64_t i, V v) {
  *reinterpret_cast<V*>(a.f[f].g + i * a.f[f].gs) = v;
}

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

template <int OP, class Rec>
__device__ __forceinline__ void run_record(const SectionArgs& a, const Rec& rec, int64_t i, int32_t pj) {
  const int* g = a.arg;
  if (OP == ADHA_OP_MADD3) {
    const float m = __fmul_rn(rec.template ld<float>(g[0]), rec.template ld<float>(g[1]));
    gst<float>(a, g[2], i, __fadd_rn(m, rec.template ld<float>(g[2])));
  } else if (OP == ADHA_OP_XORSHIFT) {
    const uint32_t u = rec.template ld<uint32_t>(g[0]);
    gst<uint32_t>(a, g[1], i, u ^ (u >> 3));
  } else if (OP == ADHA_OP_ADD) {
    gst<float>(a, g[2], i, __fadd_rn(rec.template ld<float>(g[0]), rec.template ld<float>(g[1])));
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
      gst<float>(a, f, i, __fadd_rn(__fmul_rn(rec.template ld<float>(f), 0.5f), t));
    }
    if (a.n_wr[ADHA_F64]) {
      const double td = (double)t;
      for (int j = 0; j < a.n_wr[ADHA_F64]; ++j) {
        const int f = a.wr[ADHA_F64][j];
        gst<double>(a, f, i, __dadd_rn(__dmul_rn(rec.template ld<double>(f), 0.5), td));
      }
    }
    for (int j = 0; j < a.n_wr[ADHA_I32]; ++j) {
      const int f = a.wr[ADHA_I32][j];
      gst<uint32_t>(a, f, i, rec.template ld<uint32_t>(f) ^ k);
    }
    for (int j = 0; j < a.n_wr[ADHA_BF16]; ++j) {
      const int f = a.wr[ADHA_BF16][j];
      gst<uint16_t>(a, f, i, (uint16_t)(rec.template ld<uint16_t>(f) ^ (uint16_t)(k & 0xFFFFu)));
    }
  } else if (OP == ADHA_OP_DRIFT) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float d = __fmul_rn(a.par[0], rec.template ld<float>(g[3 + ax]));
      float q = __fadd_rn(rec.template ld<float>(g[ax]), d);
      if (q >= 1.0f) q = __fsub_rn(q, 1.0f);
      else if (q < 0.0f) q = __fadd_rn(q, 1.0f);
      gst<float>(a, g[ax], i, q);
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
    gst<int32_t>(a, g[3], i, c[0] + G * (c[1] + G * c[2]));
  } else if (OP == ADHA_OP_KE) {
    const float vx = rec.template ld<float>(g[0]), vy = rec.template ld<float>(g[1]),
                vz = rec.template ld<float>(g[2]);
    float s = __fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy));
    s = __fadd_rn(s, __fmul_rn(vz, vz));
    const float e = __fmul_rn(__fmul_rn(0.5f, rec.template ld<float>(g[3])), s);
    gst<double>(a, g[4], i, (double)e);
  } else if (OP == ADHA_OP_FLAGS) {
    const uint32_t fl = rec.template ld<uint32_t>(g[0]);
    const uint32_t bit = rec.template ld<double>(g[1]) > (double)a.par[0] ? 1u : 0u;
    gst<uint32_t>(a, g[0], i, ((fl << 1) | bit) & 255u);
  } else if (OP == ADHA_OP_GATHER) {
    const int64_t j = pj;
    const float c = __fmul_rn(a.par[0], gld<float>(a, g[6], j));
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float d = __fsub_rn(gld<float>(a, g[3 + ax], j), 0.5f);
      gst<float>(a, g[ax], i, __fadd_rn(rec.template ld<float>(g[ax]), __fmul_rn(c, d)));
    }
  } else if (OP == ADHA_OP_KICK) {
    const float c = __fmul_rn(a.par[0], rec.template ld<float>(g[3]));
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
      gst<float>(a, g[ax], i, __fadd_rn(rec.template ld<float>(g[ax]), __fmul_rn(c, a.par[1 + ax])));
  } else {   // AXPB, MUL, TANH: z = op(x[, y]); the old z goes to `save` when asked
    const int z = OP == ADHA_OP_MUL ? g[2] : g[1];
    if (a.save) reinterpret_cast<float*>(a.save)[i] = rec.template ld<float>(z);
    const float x = rec.template ld<float>(g[0]);
    float v;
    if (OP == ADHA_OP_AXPB) v = __fadd_rn(__fmul_rn(a.par[0], x), a.par[1]);
    else if (OP == ADHA_OP_MUL) v = __fmul_rn(x, rec.template ld<float>(g[1]));
    else v = tanh_cf(x, a.tanh_p, a.tanh_q);
    gst<float>(a, z, i, v);
  }
}

template <int OP>
__global__ void __launch_bounds__(kThreads, 4) section_kernel(const __grid_constant__ SectionArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  GroupRef* tl = reinterpret_cast<GroupRef*>(smem);
  const int n_slices = a.n_load + (a.perm_slot >= 0 ? 1 : 0);
  uint8_t* wbase = smem + ((n_slices * (int)sizeof(GroupRef) + 15) & ~15);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* buf0 = wbase + (size_t)warp * 2 * a.in_bytes;
  uint8_t* buf1 = buf0 + a.in_bytes;
  for (int k = tid; k < n_slices; k += kThreads) tl[k] = a.load[k];
  __syncthreads();

  const int64_t W = (int64_t)gridDim.x * kWarps;
  const int64_t R = a.R;
  auto stage = [&](int64_t ch, uint8_t* buf) {
    int g = 0;
    for (int p = lane * 16; p < a.in_bytes; p += 512) {
      while (p >= tl[g].start + a.R * tl[g].stride) ++g;
      cp_async16(buf + p, tl[g].ptr + ch * R * tl[g].stride + (p - tl[g].start));
    }
  };

  int64_t c = (int64_t)blockIdx.x * kWarps + warp;
  if (c < a.n_chunks) stage(c, buf0);
  cp_async_commit();
  for (int i = 0; c < a.n_chunks; c += W, ++i) {
    const uint8_t* cur = (i & 1) ? buf1 : buf0;
    if (c + W < a.n_chunks) stage(c + W, (i & 1) ? buf0 : buf1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    const int32_t* ps = a.perm_slot >= 0 ? reinterpret_cast<const int32_t*>(cur + tl[a.perm_slot].start) : nullptr;
    for (int r = lane; r < a.R; r += 32) run_record<OP>(a, StagedRec{&a, cur, r}, c * R + r, ps ? ps[r] : 0);
    __syncwarp();
  }
  cp_async_wait<0>();

  // ragged tail: the warp whose next chunk would be n_chunks
  const int64_t t0 = a.n_chunks * R;
  if (c == a.n_chunks && t0 < a.n) {
    for (int64_t i = t0 + lane; i < a.n; i += 32) run_record<OP>(a, GlobalRec{&a, i}, i, a.perm_slot >= 0 ? a.perm[i] : 0);
  }
}

// Reverse of one fp32 chain section (AXPB, MUL, TANH) on one record per thread: restore the
// overwritten field, then propagate the adjoint in the oracle's operation order.
__global__ void __launch_bounds__(kThreads) backward_kernel(const __grid_constant__ BackwardArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    *reinterpret_cast<float*>(a.s[2] + i * a.ss[2]) = a.save[i];
    const float xo = *reinterpret_cast<const float*>(a.s[0] + i * a.ss[0]);
    float* gz_p = reinterpret_cast<float*>(a.g[2] + i * a.gs[2]);
    const float gz = *gz_p;
    *gz_p = 0.0f;
    float* gx_p = reinterpret_cast<float*>(a.g[0] + i * a.gs[0]);
    if (a.op == ADHA_OP_AXPB) {
      *gx_p = __fadd_rn(*gx_p, __fmul_rn(a.a, gz));
    } else if (a.op == ADHA_OP_MUL) {
      const float yo = *reinterpret_cast<const float*>(a.s[1] + i * a.ss[1]);
      *gx_p = __fadd_rn(*gx_p, __fmul_rn(gz, yo));
      float* gy_p = reinterpret_cast<float*>(a.g[1] + i * a.gs[1]);
      *gy_p = __fadd_rn(*gy_p, __fmul_rn(gz, xo));
    } else {
      const float t = tanh_cf(xo, a.tanh_p, a.tanh_q);
      const float d = __fsub_rn(1.0f, __fmul_rn(t, t));
      *gx_p = __fadd_rn(*gx_p, __fmul_rn(gz, d));
    }
  }
}

size_t section_smem_bytes(const SectionArgs& a) {
  const int n_slices = a.n_load + (a.perm_slot >= 0 ? 1 : 0);
  return (size_t)((n_slices * (int)sizeof(GroupRef) + 15) & ~15) + (size_t)kWarps * 2 * a.in_bytes;
}

template <int OP>
static int launch_op(const SectionArgs& a, int grid, size_t smem, void* stream) {
  cudaError_t e = cudaFuncSetAttribute(section_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(section)");
  section_kernel<OP><<<grid, kThreads, smem, (cudaStream_t)stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "section kernel launch");
  return 0;
}

template <int OP>
static int occ_op(size_t smem, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(section_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(section)");
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, section_kernel<OP>, kThreads, smem);
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
  int64_t blocks = (a.n + kThreads - 1) / kThreads;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (blocks < 1) blocks = 1;
  backward_kernel<<<(int)blocks, kThreads, 0, (cudaStream_t)stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "backward kernel launch");
  return 0;
}

}  // namespace adha

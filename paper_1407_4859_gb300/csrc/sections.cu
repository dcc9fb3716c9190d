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
#include "section_ops.cuh"

namespace adha {

// per-CTA slice table at the start of shared memory: pointers, slice ends, write-back flags
constexpr int kSectionTable = (16 * (kMaxGroups + 1) + 15) / 16 * 16;

template <int OP, int M, bool VEC>
__global__ void __launch_bounds__(kThreads) section_kernel(const __grid_constant__ SectionArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int n_slices = a.n_load + (a.perm_slot >= 0 ? 1 : 0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // slice table: base pointer and byte range of each staged slice within a chunk buffer
  const uint8_t** sp = reinterpret_cast<const uint8_t**>(smem);
  int* send = reinterpret_cast<int*>(smem + 8 * (kMaxGroups + 1));
  int* wback = send + (kMaxGroups + 1);
  const int nb = a.buffers;   // 2: the next chunk is staged while one is computed; 1: one buffer
  uint8_t* buf0 = smem + kSectionTable + (size_t)warp * nb * a.in_bytes;
  uint8_t* buf1 = buf0 + (nb - 1) * a.in_bytes;
  constexpr int R = 32 * M;
  // REDUCE: counts and (walk) sums in registers; after the chunk buffers the warp's two sum
  // tables (not walk) and its 32-entry record list (walk)
  long long* acc = nullptr;
  int* idx = nullptr;
  unsigned long long cnt = 0;   // REDUCE: lane k counts cluster k
  long long sum[kMaxClusters];
  ReduceLane rq{};
  if constexpr (OP == ADHA_OP_REDUCE) {
    rq = reduce_lane(a.s, a.f, lane, a.reduce_walk != 0);
    uint8_t* extra = smem + kSectionTable + (size_t)kWarps * nb * a.in_bytes;
    if (!rq.walk) {
      acc = reinterpret_cast<long long*>(extra) + (size_t)warp * 2 * (kMaxClusters + 1) * 32;
      for (int k = lane; k < 2 * (kMaxClusters + 1) * 32; k += 32) acc[k] = 0;
      extra += kReduceTableBytes;
    }
    idx = reinterpret_cast<int*>(extra) + warp * 32;
#pragma unroll
    for (int k = 0; k < kMaxClusters; ++k) sum[k] = 0;
  }
  for (int k = tid; k < n_slices; k += kThreads) {
    sp[k] = a.load[k].ptr;
    send[k] = a.load[k].start + R * a.load[k].stride;
    wback[k] = a.writeback[k];
  }
  // ASSIGN: the centroid pair table after the chunk buffers
  float* cT = nullptr;
  if constexpr (OP == ADHA_OP_ASSIGN) {
    cT = reinterpret_cast<float*>(smem + kSectionTable + (size_t)kWarps * nb * a.in_bytes);
    fill_centroid_pairs(a.s, a.f, cT, tid, kThreads);
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
    if (nb == 2) {
      if (c + W < a.n_chunks) stage(c + W, (i & 1) ? buf0 : buf1);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const int64_t i0 = c * R;
    if constexpr (OP == ADHA_OP_REDUCE) {
      reduce_chunk_any<M>(rq, cur, lane, acc, acc + (kMaxClusters + 1) * 32, idx, sum, &cnt);
    } else if constexpr (OP == ADHA_OP_ASSIGN) {
      assign_chunk<M>(a.s, a.f, cur, i0, lane, cT);
    } else if (OP == ADHA_OP_MIX && VEC) {
      mix_chunk_vec<M>(a.s, a.f, cur, i0, lane);
    } else if (VEC) {
      chain_chunk_vec<OP, M>(a.s, a.f, a.tanh_p, a.tanh_q, a.save, cur, i0, lane);
    } else if (OP == ADHA_OP_MIX) {
      mix_chunk<M>(a.s, a.f, cur, i0, lane);
    } else {
      const int32_t* ps = a.perm_slot >= 0 ? reinterpret_cast<const int32_t*>(cur + a.load[a.perm_slot].start) : nullptr;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int r = lane + 32 * m;
        run_record<OP>(a.s, a.f, a.tanh_p, a.tanh_q, a.save, StagedRec{a.f, cur, r, i0 + r}, i0 + r, ps ? ps[r] : 0);
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
    if (nb == 1 && c + W < a.n_chunks) {   // one buffer: the next chunk once this one is done with it
      stage(c + W, buf0);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();

  // ragged tail: the warp whose next chunk would be n_chunks
  const int64_t t0 = a.n_chunks * R;
  if constexpr (OP == ADHA_OP_REDUCE) {
    if (c == a.n_chunks && t0 < a.n) reduce_tail(rq, a.s, a.f, t0, a.n, lane, acc, sum, &cnt);
    // every warp adds its sums and counts into the result (zeroed before the launch)
    __syncwarp();
    reduce_flush(rq, a.s, lane, acc, sum, &cnt);
  } else {
    if (c == a.n_chunks && t0 < a.n) {
      for (int64_t i = t0 + lane; i < a.n; i += 32)
        run_record<OP>(a.s, a.f, a.tanh_p, a.tanh_q, a.save, GlobalRec{a.f, i}, i, a.perm_slot >= 0 ? a.perm[i] : 0);
    }
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

size_t section_smem_bytes(const SectionArgs& a) {
  // REDUCE: two (K+1) x 32 int64 tables per warp unless it walks, and a 32-entry list per warp
  const size_t acc = a.s.op == ADHA_OP_REDUCE ? (a.reduce_walk ? 0 : kReduceTableBytes) + kReduceListBytes : 0;
  const size_t cent = a.s.op == ADHA_OP_ASSIGN ? (size_t)kCentroidPairBytes : 0;
  return kSectionTable + (size_t)kWarps * a.buffers * a.in_bytes + acc + cent;
}

template <int OP, int M, bool VEC>
static int launch_om(const SectionArgs& a, int grid, size_t smem, void* stream) {
  cudaError_t e = cudaFuncSetAttribute(section_kernel<OP, M, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(section)");
  if (OP == ADHA_OP_REDUCE && !a.accumulate) {   // the sums are added into a zeroed result
    const int K = a.s.arg[1], d = a.s.rd_off[ADHA_F32 + 1] - a.s.rd_off[ADHA_F32];
    e = cudaMemsetAsync(const_cast<void*>(a.s.aux), 0, (size_t)K * (d + 1) * 8, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(reduce result)");
  }
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
  X(ADHA_OP_TANH) X(ADHA_OP_ASSIGN) X(ADHA_OP_REDUCE)

int launch_section(const SectionArgs& a, int grid, size_t smem, void* stream) {
  switch (a.s.op) {
#define X(op) case op: return launch_op<op>(a, grid, smem, stream);
    ADHA_FOR_EACH_OP(X)
#undef X
    default: return fail(ADHA_EINVAL, "unknown section op %d", a.s.op);
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

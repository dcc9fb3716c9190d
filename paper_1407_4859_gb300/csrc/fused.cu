// fused.cu -- a run of consecutive sections in one pass over the records (paper Section 2: the
// combine edge of the DAG, which joins consecutive sections that share a layout into one node).
//
// Same warp-autonomous pipeline as sections.cu: each warp stages its chunk of R = 32*M records
// (every group holding a field that some section of the run reads or writes, plus the
// permutation of a gather) with 16-byte cp.async one chunk ahead, then applies the run's
// sections in order to the chunk buffer (each section reads what the previous ones wrote there),
// and writes every group with a written field back whole.  The result is the one of running the
// sections one after another: each record's sections run in order, and the only cross-record
// reads (a gather's fields at perm[i]) come from groups no section of the run writes, so they
// read the values from before the run.  Fields are read and written once per run instead of
// once per section.
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"
#include "section_ops.cuh"

namespace adha {

// per-CTA tables at the start of shared memory: the slice table (pointers, slice ends, write-back
// flags), then copies of the field table and of the sections' operands.  The compute loops look
// fields and operands up by runtime index once per field per chunk and section; from the
// parameter space each such lookup is an indexed constant load, whose unit saturates long before
// the memory system does, while shared-memory loads of one address broadcast to the warp.
constexpr int kSliceTable = (16 * (kMaxGroups + 1) + 15) / 16 * 16;
constexpr int kFieldTable = (int)sizeof(FieldRef) * kMaxFields;
static_assert(sizeof(FieldRef) % 8 == 0 && sizeof(SecOp) % 4 == 0, "tables are copied in whole words");

// Bytes of the tables for a run of n_sec sections (the chunk buffers follow, 16-byte aligned).
__host__ __device__ constexpr int fused_table_bytes(int n_sec) {
  return kSliceTable + kFieldTable + ((int)sizeof(SecOp) * n_sec + 15) / 16 * 16;
}

// After the chunk buffers: a REDUCE's two sum tables per warp (unless it walks) and its record
// lists (see reduce_chunk_any), then an ASSIGN's centroid pair table.
constexpr size_t kCentroidBytes = (size_t)kCentroidPairBytes;
static_assert(kReduceTableBytes % 16 == 0 && kReduceListBytes % 16 == 0, "the centroid table stays 16-byte aligned");


// One section on the M records of each lane of a staged chunk (r = lane + 32m), writes into the
// chunk buffer; op is runtime (uniform over the launch).
template <int M>
__device__ __forceinline__ void fused_section_chunk(const FusedArgs& a, const FieldRef* fr, const SecOp& so,
                                                    uint8_t* cur, int64_t i0, const int32_t* ps, int lane) {
  switch (so.op) {
#define ADHA_FUSED_OP(OP)                                                                                 \
  case OP:                                                                                                \
    _Pragma("unroll") for (int m = 0; m < M; ++m) {                                                       \
      const int r = lane + 32 * m;                                                                        \
      run_record<OP>(so, fr, a.tanh_p, a.tanh_q, nullptr, StagedRec{fr, cur, r, i0 + r}, i0 + r,         \
                     ps ? ps[r] : 0);                                                                     \
    }                                                                                                     \
    break;
    ADHA_FUSED_OP(ADHA_OP_MADD3)
    ADHA_FUSED_OP(ADHA_OP_XORSHIFT)
    ADHA_FUSED_OP(ADHA_OP_ADD)
    ADHA_FUSED_OP(ADHA_OP_MIX)
    ADHA_FUSED_OP(ADHA_OP_DRIFT)
    ADHA_FUSED_OP(ADHA_OP_BIN)
    ADHA_FUSED_OP(ADHA_OP_KE)
    ADHA_FUSED_OP(ADHA_OP_FLAGS)
    ADHA_FUSED_OP(ADHA_OP_GATHER)
    ADHA_FUSED_OP(ADHA_OP_KICK)
    ADHA_FUSED_OP(ADHA_OP_AXPB)
    ADHA_FUSED_OP(ADHA_OP_MUL)
    ADHA_FUSED_OP(ADHA_OP_TANH)
    ADHA_FUSED_OP(ADHA_OP_ASSIGN)
#undef ADHA_FUSED_OP
    default: break;
  }
}

// One section on one record in global memory (the ragged tail).
__device__ __forceinline__ void fused_section_record(const FusedArgs& a, const FieldRef* fr, const SecOp& so, int64_t i,
                                                     int32_t pj) {
  const GlobalRec rec{fr, i};
  switch (so.op) {
#define ADHA_FUSED_OP(OP) \
  case OP: run_record<OP>(so, fr, a.tanh_p, a.tanh_q, nullptr, rec, i, pj); break;
    ADHA_FUSED_OP(ADHA_OP_MADD3)
    ADHA_FUSED_OP(ADHA_OP_XORSHIFT)
    ADHA_FUSED_OP(ADHA_OP_ADD)
    ADHA_FUSED_OP(ADHA_OP_MIX)
    ADHA_FUSED_OP(ADHA_OP_DRIFT)
    ADHA_FUSED_OP(ADHA_OP_BIN)
    ADHA_FUSED_OP(ADHA_OP_KE)
    ADHA_FUSED_OP(ADHA_OP_FLAGS)
    ADHA_FUSED_OP(ADHA_OP_GATHER)
    ADHA_FUSED_OP(ADHA_OP_KICK)
    ADHA_FUSED_OP(ADHA_OP_AXPB)
    ADHA_FUSED_OP(ADHA_OP_MUL)
    ADHA_FUSED_OP(ADHA_OP_TANH)
    ADHA_FUSED_OP(ADHA_OP_ASSIGN)
#undef ADHA_FUSED_OP
    default: break;
  }
}

// KM: the run holds a K-Means-shaped section (assign or reduce), whose per-chunk code and
// tables are compiled into a kernel of their own, so that the registers they need do not lower
// the occupancy of every other fused run.
template <int M, bool VEC, bool KM>
__global__ void __launch_bounds__(kThreads) fused_kernel(const __grid_constant__ FusedArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int n_slices = a.n_load + (a.perm_slot >= 0 ? 1 : 0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint8_t** sp = reinterpret_cast<const uint8_t**>(smem);
  int* send = reinterpret_cast<int*>(smem + 8 * (kMaxGroups + 1));
  int* wback = send + (kMaxGroups + 1);
  const int nb = a.buffers;   // 2: the next chunk is staged while one is computed; 1: one buffer
  uint8_t* buf0 = smem + fused_table_bytes(a.n_sec) + (size_t)warp * nb * a.in_bytes;
  uint8_t* buf1 = buf0 + (nb - 1) * a.in_bytes;
  constexpr int R = 32 * M;
  for (int k = tid; k < n_slices; k += kThreads) {
    sp[k] = a.load[k].ptr;
    send[k] = a.load[k].start + R * a.load[k].stride;
    wback[k] = a.writeback[k];
  }
  FieldRef* fr = reinterpret_cast<FieldRef*>(smem + kSliceTable);
  SecOp* secs = reinterpret_cast<SecOp*>(smem + kSliceTable + kFieldTable);
  for (int k = tid; k < kMaxFields * (int)(sizeof(FieldRef) / 8); k += kThreads)
    reinterpret_cast<uint2*>(fr)[k] = reinterpret_cast<const uint2*>(a.f)[k];
  for (int k = tid; k < a.n_sec * (int)(sizeof(SecOp) / 4); k += kThreads)
    reinterpret_cast<uint32_t*>(secs)[k] = reinterpret_cast<const uint32_t*>(a.sec)[k];
  uint8_t* extra = smem + fused_table_bytes(a.n_sec) + (size_t)kWarps * nb * a.in_bytes;
  long long* acc = nullptr;   // REDUCE: this warp's sum tables (or register sums) and record list;
  int* idx = nullptr;         // its counts, one cluster per lane
  unsigned long long cnt_lane = 0;
  long long sum[KM ? kMaxClusters : 1];
  if (KM && a.reduce_sec >= 0) {
    if (!a.reduce_walk) {
      acc = reinterpret_cast<long long*>(extra) + (size_t)warp * 2 * (kMaxClusters + 1) * 32;
      for (int k = lane; k < 2 * (kMaxClusters + 1) * 32; k += 32) acc[k] = 0;
      extra += kReduceTableBytes;
    }
    idx = reinterpret_cast<int*>(extra) + warp * 32;
    extra += kReduceListBytes;
#pragma unroll
    for (int k = 0; k < (KM ? kMaxClusters : 1); ++k) sum[k] = 0;
  }
  float* cT = nullptr;
  if (KM && a.assign_sec >= 0) {
    cT = reinterpret_cast<float*>(extra);
    fill_centroid_pairs(a.sec[a.assign_sec], a.f, cT, tid, kThreads);
  }
  __syncthreads();
  ReduceLane rq{};
  if (KM && a.reduce_sec >= 0) rq = reduce_lane(secs[a.reduce_sec], fr, lane, a.reduce_walk != 0);

  const int64_t W = (int64_t)gridDim.x * kWarps;
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
    const int32_t* ps = a.perm_slot >= 0 ? reinterpret_cast<const int32_t*>(cur + a.load[a.perm_slot].start) : nullptr;
    for (int s = 0; s < a.n_sec; ++s) {
      const SecOp& so = secs[s];
      const int op = so.op;
      if constexpr (KM) {
        if (s == a.reduce_sec) {
          reduce_chunk_any<M>(rq, cur, lane, acc, acc + (kMaxClusters + 1) * 32, idx, sum, &cnt_lane);
          __syncwarp();
          continue;
        }
      }
      if (KM && s == a.assign_sec) assign_chunk<M>(so, fr, cur, i0, lane, cT);
      else if (VEC && op == ADHA_OP_MIX) mix_chunk_vec<M, true>(so, fr, cur, i0, lane);
      else if (VEC && op == ADHA_OP_AXPB) chain_chunk_vec<ADHA_OP_AXPB, M, true>(so, fr, a.tanh_p, a.tanh_q, nullptr, cur, i0, lane);
      else if (VEC && op == ADHA_OP_MUL) chain_chunk_vec<ADHA_OP_MUL, M, true>(so, fr, a.tanh_p, a.tanh_q, nullptr, cur, i0, lane);
      else if (VEC && op == ADHA_OP_TANH) chain_chunk_vec<ADHA_OP_TANH, M, true>(so, fr, a.tanh_p, a.tanh_q, nullptr, cur, i0, lane);
      else fused_section_chunk<M>(a, fr, so, cur, i0, ps, lane);
      __syncwarp();   // the next section may map records to lanes the other way
    }
    // groups with written fields go back whole, 16 bytes per lane per step
    int g = 0, start = 0;
    for (int p = lane * 16; p < a.in_bytes; p += 512) {
      while (p >= send[g]) start = send[g++];
      if (wback[g]) {
        const int64_t stride = (send[g] - start) / R;
        *reinterpret_cast<uint4*>(const_cast<uint8_t*>(sp[g]) + c * (R * stride) + (p - start)) =
            *reinterpret_cast<const uint4*>(cur + p);
      }
    }
    __syncwarp();
    if (nb == 1 && c + W < a.n_chunks) {   // one buffer: the next chunk once this one has gone back
      stage(c + W, buf0);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();

  // ragged tail: the warp whose next chunk would be n_chunks, record by record in global memory
  const int64_t t0 = a.n_chunks * R;
  if (c == a.n_chunks && t0 < a.n) {
    if (!KM || a.reduce_sec < 0) {
      for (int64_t i = t0 + lane; i < a.n; i += 32) {
        const int32_t pj = a.perm_slot >= 0 ? a.perm[i] : 0;
        for (int s = 0; s < a.n_sec; ++s) fused_section_record(a, fr, secs[s], i, pj);
      }
    } else {   // section by section over the tail's records: the reduce reads every lane's records
      for (int s = 0; s < a.n_sec; ++s) {
        __syncwarp();
        if (s == a.reduce_sec) {
          if constexpr (KM) reduce_tail(rq, secs[s], fr, t0, a.n, lane, acc, sum, &cnt_lane);
        } else {
          for (int64_t i = t0 + lane; i < a.n; i += 32)
            fused_section_record(a, fr, secs[s], i, a.perm_slot >= 0 ? a.perm[i] : 0);
        }
      }
    }
  }
  if constexpr (KM) {
    if (a.reduce_sec >= 0) {   // every warp adds its sums and counts into the result
      __syncwarp();
      reduce_flush(rq, secs[a.reduce_sec], lane, acc, sum, &cnt_lane);
    }
  }
}

size_t fused_smem_bytes(const FusedArgs& a) {
  return fused_table_bytes(a.n_sec) + (size_t)kWarps * a.buffers * a.in_bytes +
         (a.reduce_sec >= 0 ? (a.reduce_walk ? 0 : kReduceTableBytes) + kReduceListBytes : 0) +
         (a.assign_sec >= 0 ? kCentroidBytes : 0);
}

template <int M, bool VEC, bool KM>
static int launch_m(const FusedArgs& a, int grid, size_t smem, void* stream) {
  cudaError_t e = cudaFuncSetAttribute(fused_kernel<M, VEC, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused)");
  if (a.reduce_sec >= 0 && !a.accumulate) {   // the sums are added into a zeroed result
    const SecOp& so = a.sec[a.reduce_sec];
    const int K = so.arg[1], d = so.rd_off[ADHA_F32 + 1] - so.rd_off[ADHA_F32];
    e = cudaMemsetAsync(const_cast<void*>(so.aux), 0, (size_t)K * (d + 1) * 8, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(reduce result)");
  }
  fused_kernel<M, VEC, KM><<<grid, kThreads, smem, (cudaStream_t)stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
  return 0;
}

// Runs with an assign or a reduce take the record-by-record mapping whatever the layout (the vector
// mapping only speeds up the mix and chain sections) and at most 64 records per chunk: each such
// kernel carries the assign's per-K specialisations, so only two are built.
template <bool KM>
static int launch_km(const FusedArgs& a, int grid, size_t smem, void* stream) {
  if constexpr (!KM) {
    if (a.vec && a.R == 32) return launch_m<1, true, false>(a, grid, smem, stream);
    if (a.vec && a.R == 64) return launch_m<2, true, false>(a, grid, smem, stream);
    if (a.vec && a.R == 128) return launch_m<4, true, false>(a, grid, smem, stream);
  }
  if constexpr (KM) {   // such runs are planned with at most 64 records per chunk
    return a.R == 32 ? launch_m<1, false, true>(a, grid, smem, stream) : launch_m<2, false, true>(a, grid, smem, stream);
  } else {
    switch (a.R) {
      case 32: return launch_m<1, false, false>(a, grid, smem, stream);
      case 64: return launch_m<2, false, false>(a, grid, smem, stream);
      default: return launch_m<4, false, false>(a, grid, smem, stream);
    }
  }
}

int launch_fused(const FusedArgs& a, int grid, size_t smem, void* stream) {
  return fused_is_km(a) ? launch_km<true>(a, grid, smem, stream) : launch_km<false>(a, grid, smem, stream);
}

template <int M, bool VEC, bool KM>
static int occ_m(size_t smem, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(fused_kernel<M, VEC, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused)");
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fused_kernel<M, VEC, KM>, kThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(fused)");
  return 0;
}

template <bool KM>
static int occ_km(int M, bool vec, size_t smem, int* blocks) {
  if constexpr (!KM) {
    if (vec && M == 1) return occ_m<1, true, false>(smem, blocks);
    if (vec && M == 2) return occ_m<2, true, false>(smem, blocks);
    if (vec && M == 4) return occ_m<4, true, false>(smem, blocks);
  }
  if constexpr (KM) {
    return M == 1 ? occ_m<1, false, true>(smem, blocks) : occ_m<2, false, true>(smem, blocks);
  } else {
    if (M == 1) return occ_m<1, false, false>(smem, blocks);
    if (M == 2) return occ_m<2, false, false>(smem, blocks);
    return occ_m<4, false, false>(smem, blocks);
  }
}

int fused_occupancy(int M, bool vec, bool km, size_t smem, int* blocks) {
  return km ? occ_km<true>(M, vec, smem, blocks) : occ_km<false>(M, vec, smem, blocks);
}

}  // namespace adha

// remap.cu -- the layout remap kernel (paper Section 2: the remap between two sections' layouts;
// Table 4: CPU-ODS(1-3) remap GPU-ODS(4-7)).
//
// One persistent CTA per SM slot walks whole tiles of T records.  Per tile:
//   1. one thread issues a bulk copy (cp.async.bulk) of each source group's T-record slice into a
//      pipeline stage; the bytes land on the stage's mbarrier (S stages in flight);
//   2. all threads assemble the destination groups' slices in a shared output buffer, one
//      u-sized slot at a time (u = the smallest moved field size), from a slot table that maps
//      every destination slot to its source bytes: this is the tile transpose between the
//      source and destination record strides;
//   3. one thread bulk-stores each destination slice (double-buffered output).
// Global traffic is two contiguous streams per group, 16-byte aligned at both ends.  The ragged
// tail (fewer than T records) goes through plain loads and stores by the CTA that owns it.
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"

namespace adha {

template <typename U>
__device__ __forceinline__ void assemble(const RemapArgs& a, const uint8_t* stage, uint8_t* out, int T,
                                         const uint32_t* slots) {
  const int tid = threadIdx.x;
  for (int d = 0; d < a.n_dst; ++d) {
    const int S = a.d_nslot[d];
    const int total = T * S;
    const uint32_t* sl = slots + a.d_slot0[d];
    U* o = reinterpret_cast<U*>(out + a.d_smem[d]);
    int r = tid / S;
    int k = tid - r * S;
    const int q = a.d_q[d], rem = a.d_rem[d];
    for (int e = tid; e < total; e += kThreads) {
      const uint32_t c = sl[k];
      U v = 0;
      if (c != kPadSlot) v = *reinterpret_cast<const U*>(stage + (c & 0xFFFFFu) + r * (c >> 20));
      o[e] = v;
      k += rem;
      r += q;
      if (k >= S) {
        k -= S;
        ++r;
      }
    }
  }
}

template <typename U>
__global__ void __launch_bounds__(kThreads) remap_kernel(const __grid_constant__ RemapArgs a, int* status) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  uint8_t* stages = smem + 128;
  uint8_t* outs = stages + (size_t)a.S * a.stage_bytes;
  uint32_t* slots = reinterpret_cast<uint32_t*>(outs + 2 * (size_t)a.out_bytes);
  const int tid = threadIdx.x;

  for (int k = tid; k < a.n_slots; k += kThreads) slots[k] = a.slot[k];
  if (tid == 0) {
    for (int s = 0; s < a.S; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const int64_t G = gridDim.x;
  const int64_t my_n = (int64_t)blockIdx.x < a.n_full ? (a.n_full - 1 - blockIdx.x) / G + 1 : 0;

  auto issue = [&](int64_t j) {   // thread 0 only: load tile number j of this CTA
    const int st = (int)(j % a.S);
    const int64_t t = blockIdx.x + j * G;
    uint8_t* dst = stages + (size_t)st * a.stage_bytes;
    uint32_t bytes = 0;
    for (int g = 0; g < a.n_src; ++g) bytes += (uint32_t)a.T * a.s_stride[g];
    mbar_expect_tx(&bars[st], bytes);
    for (int g = 0; g < a.n_src; ++g)
      bulk_load(dst + a.s_smem[g], a.src[g] + t * a.T * a.s_stride[g], (uint32_t)a.T * a.s_stride[g], &bars[st]);
  };

  if (tid == 0)
    for (int64_t j = 0; j < my_n && j < a.S; ++j) issue(j);

  int64_t j = 0;
  bool timed_out = false;
  for (; j < my_n; ++j) {
    const int st = (int)(j % a.S);
    const bool ok = mbar_wait(&bars[st], (uint32_t)((j / a.S) & 1));
    if (tid == 0) bulk_wait_read<1>();             // output buffer j&1 no longer read by the store of j-2
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    uint8_t* out = outs + (size_t)(j & 1) * a.out_bytes;
    assemble<U>(a, stages + (size_t)st * a.stage_bytes, out, a.T, slots);
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      const int64_t t = blockIdx.x + j * G;
      for (int d = 0; d < a.n_dst; ++d)
        bulk_store(a.dst[d] + t * a.T * a.d_stride[d], out + a.d_smem[d], (uint32_t)a.T * a.d_stride[d]);
      bulk_commit();
      if (j + a.S < my_n) issue(j + a.S);
    }
  }

  if (timed_out) {
    if (tid == 0) {
      set_status(status, ADHA_ETIMEOUT);
      for (int64_t k = j; k < my_n && k < j + a.S; ++k)   // copies that may still be in flight
        (void)mbar_wait(&bars[k % a.S], (uint32_t)((k / a.S) & 1));
      bulk_wait_all<0>();
    }
    return;
  }

  // Ragged tail: records [n_full*T, n), handled by the CTA that would own tile n_full.
  const int64_t t0 = a.n_full * a.T;
  if (t0 < a.n && (int64_t)blockIdx.x == a.n_full % G) {
    const int Tt = (int)(a.n - t0);
    if (tid == 0) bulk_wait_read<0>();
    __syncthreads();
    uint8_t* stage = stages;
    for (int g = 0; g < a.n_src; ++g) {
      const U* src = reinterpret_cast<const U*>(a.src[g] + t0 * a.s_stride[g]);
      U* sd = reinterpret_cast<U*>(stage + a.s_smem[g]);
      const int words = Tt * a.s_stride[g] / (int)sizeof(U);
      for (int k = tid; k < words; k += kThreads) sd[k] = src[k];
    }
    __syncthreads();
    assemble<U>(a, stage, outs, Tt, slots);
    __syncthreads();
    for (int d = 0; d < a.n_dst; ++d) {
      U* dd = reinterpret_cast<U*>(a.dst[d] + t0 * a.d_stride[d]);
      const U* so = reinterpret_cast<const U*>(outs + a.d_smem[d]);
      const int words = Tt * a.d_stride[d] / (int)sizeof(U);
      for (int k = tid; k < words; k += kThreads) dd[k] = so[k];
    }
  }
  if (tid == 0) bulk_wait_all<0>();
}

size_t remap_smem_bytes(const RemapArgs& a) {
  return 128 + (size_t)a.S * a.stage_bytes + 2 * (size_t)a.out_bytes + (size_t)a.n_slots * 4;
}

template <typename U>
static int launch_t(const RemapArgs& a, int grid, size_t smem, void* stream) {
  int* status = nullptr;
  if (int rc = status_word(&status)) return rc;
  cudaError_t e = cudaFuncSetAttribute(remap_kernel<U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(remap)");
  remap_kernel<U><<<grid, kThreads, smem, (cudaStream_t)stream>>>(a, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "remap kernel launch");
  return 0;
}

int launch_remap(const RemapArgs& a, int unit, int grid, size_t smem, void* stream) {
  switch (unit) {
    case 2: return launch_t<uint16_t>(a, grid, smem, stream);
    case 4: return launch_t<uint32_t>(a, grid, smem, stream);
    default: return launch_t<unsigned long long>(a, grid, smem, stream);
  }
}

template <typename U>
static int occ_t(size_t smem, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(remap_kernel<U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(remap)");
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, remap_kernel<U>, kThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(remap)");
  return 0;
}

int remap_occupancy(int unit, size_t smem, int* blocks) {
  switch (unit) {
    case 2: return occ_t<uint16_t>(smem, blocks);
    case 4: return occ_t<uint32_t>(smem, blocks);
    default: return occ_t<unsigned long long>(smem, blocks);
  }
}

}  // namespace adha

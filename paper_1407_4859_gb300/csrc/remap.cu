// remap.cu -- the layout remap kernel (paper Section 2: the remap between two sections' layouts;
// Table 4: CPU-ODS(1-3) remap GPU-ODS(4-7)).
//
// Every warp works alone on chunks of R consecutive records (R a multiple of 32), so the main
// loop has no block-wide barrier:
//   1. the warp copies the chunk's slice of every source group into its own shared buffer with
//      16-byte cp.async (coalesced: lane l moves bytes 16l, 16l+512, ...), one chunk ahead of
//      the one it works on (double buffering);
//   2. it assembles the destination slices in a second buffer, one u-sized element per lane
//      per step (u = the smallest moved field size), through a schedule table built once per CTA
//      that pairs every destination element of a chunk with its source element: this is the
//      tile transpose between the source and destination record strides.  The host picks the
//      order of the pairs (destination-major or record-major) with fewer shared-memory bank
//      conflicts for the two strides;
//   3. it writes the destination slices back with 16-byte stores.
// Global traffic is one contiguous read stream per source group and one write stream per
// destination group.  The ragged tail (fewer than R records) goes element by element through
// the warp that would own the next chunk.
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"

namespace adha {

__device__ __forceinline__ int align16(int x) { return (x + 15) & ~15; }

template <typename U>
__global__ void __launch_bounds__(kThreads) remap_kernel(const __grid_constant__ RemapArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  GroupRef* tin = reinterpret_cast<GroupRef*>(smem);
  GroupRef* tout = tin + a.n_src;
  uint32_t* sched = reinterpret_cast<uint32_t*>(smem + align16((a.n_src + a.n_dst) * (int)sizeof(GroupRef)));
  uint8_t* wbase = reinterpret_cast<uint8_t*>(sched) + align16(a.n_elems * 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* buf0 = wbase + (size_t)warp * (2 * a.in_bytes + a.out_bytes);
  uint8_t* buf1 = buf0 + a.in_bytes;
  uint8_t* outb = buf1 + a.in_bytes;

  for (int k = tid; k < a.n_src; k += kThreads) tin[k] = a.src[k];
  for (int k = tid; k < a.n_dst; k += kThreads) tout[k] = a.dst[k];
  // schedule table: entry t = (source element << 16 | destination element) of the t-th element
  // the warp moves; lanes take consecutive entries.  Order 0 walks destination elements in
  // order (conflict-free writes); order 1 walks, per destination slot, 32 consecutive records
  // (conflict-free reads from narrow source slices).
  for (int t = tid; t < a.n_elems; t += kThreads) {
    int d = 0, e0 = 0;
    while (t >= e0 + a.R * a.d_nslot[d]) e0 += a.R * a.d_nslot[d++];
    const int S = a.d_nslot[d];
    int r, k;
    if (a.order == 0) {
      r = (t - e0) / S;
      k = (t - e0) - r * S;
    } else {
      k = (t - e0) / a.R;
      r = (t - e0) - k * a.R;
    }
    const uint32_t code = a.slot[a.d_slot0[d] + k];
    uint32_t x = 0xFFFFu;
    if (code != kPadSlot) {
      const int j = (int)(code >> 16);
      x = (uint32_t)((a.src[j].start + r * a.src[j].stride + (int)(code & 0xFFFFu)) / (int)sizeof(U));
    }
    sched[t] = x | ((uint32_t)(e0 + r * S + k) << 16);
  }
  __syncthreads();

  const int64_t W = (int64_t)gridDim.x * kWarps;
  const int64_t R = a.R;
  auto stage = [&](int64_t ch, uint8_t* buf) {
    int g = 0;
    for (int p = lane * 16; p < a.in_bytes; p += 512) {
      while (p >= tin[g].start + a.R * tin[g].stride) ++g;
      cp_async16(buf + p, tin[g].ptr + ch * R * tin[g].stride + (p - tin[g].start));
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
    const U* src = reinterpret_cast<const U*>(cur);
    U* dst = reinterpret_cast<U*>(outb);
#pragma unroll 4
    for (int t = lane; t < a.n_elems; t += 32) {
      const uint32_t p = sched[t];
      const uint32_t x = p & 0xFFFFu;
      dst[p >> 16] = x != 0xFFFFu ? src[x] : U(0);
    }
    __syncwarp();
    int g = 0;
    for (int p = lane * 16; p < a.out_bytes; p += 512) {
      while (p >= tout[g].start + a.R * tout[g].stride) ++g;
      const uint4 v = *reinterpret_cast<const uint4*>(outb + p);
      *reinterpret_cast<uint4*>(const_cast<uint8_t*>(tout[g].ptr) + c * R * tout[g].stride + (p - tout[g].start)) = v;
    }
    __syncwarp();
  }
  cp_async_wait<0>();

  // ragged tail: the warp whose next chunk would be n_chunks
  const int64_t t0 = a.n_chunks * R;
  if (c == a.n_chunks && t0 < a.n) {
    const int Tt = (int)(a.n - t0);
    for (int d = 0; d < a.n_dst; ++d) {
      const int S = a.d_nslot[d];
      for (int e = lane; e < Tt * S; e += 32) {
        const int r = e / S, k = e - r * S;
        const uint32_t code = a.slot[a.d_slot0[d] + k];
        U v = U(0);
        if (code != kPadSlot) {
          const GroupRef& sg = tin[code >> 16];
          v = *reinterpret_cast<const U*>(sg.ptr + (t0 + r) * sg.stride + (code & 0xFFFFu));
        }
        *reinterpret_cast<U*>(const_cast<uint8_t*>(tout[d].ptr) + (t0 + r) * tout[d].stride + k * (int)sizeof(U)) = v;
      }
    }
  }
}

size_t remap_smem_bytes(const RemapArgs& a) {
  auto al = [](size_t x) { return (x + 15) / 16 * 16; };
  return al((size_t)(a.n_src + a.n_dst) * sizeof(GroupRef)) + al((size_t)a.n_elems * 4) +
         (size_t)kWarps * (2 * (size_t)a.in_bytes + a.out_bytes);
}

template <typename U>
static int launch_t(const RemapArgs& a, int grid, size_t smem, void* stream) {
  cudaError_t e = cudaFuncSetAttribute(remap_kernel<U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(remap)");
  remap_kernel<U><<<grid, kThreads, smem, (cudaStream_t)stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "remap kernel launch");
  return 0;
}

int launch_remap(const RemapArgs& a, int grid, size_t smem, void* stream) {
  switch (a.unit) {
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

// remap.cu -- the layout remap kernel (paper Section 2: the remap between two sections' layouts;
// Table 4: CPU-ODS(1-3) remap GPU-ODS(4-7)).
//
// Every warp works alone on chunks of R consecutive records (R a multiple of 32), so the main
// loop has no block-wide barrier:
//   1. the warp copies the chunk's slice of every source group into its own shared buffer with
//      16-byte cp.async (coalesced: lane l moves bytes 16l, 16l+512, ...): one chunk ahead of
//      the one it works on (two buffers), or, with one buffer, as soon as the moves have read
//      the current chunk (half the input buffers' shared memory, so more warps per SM);
//   2. it moves every field of every destination record, one move per lane per step: a move is
//      one field (8, 4 or 2 bytes, whole) or an aligned piece of zero padding (read from 16 zero
//      bytes after the chunk buffer), taken from a schedule table built once per CTA.  Moves into one-field destination groups are stored
//      straight to global memory (consecutive lanes on consecutive records, so the stores are
//      coalesced); moves into wider groups are assembled in a second buffer.  This is the tile
//      transpose between the source and destination record strides; the host picks, per move
//      class, the schedule order with the fewest shared-memory bank conflicts;
//   3. it writes the assembled wider destination slices back with 16-byte stores.
// Where each 16-byte piece of the two buffers lives in global memory is the same for every chunk
// up to the chunk's offset; when a buffer's slices are narrower than a warp step (many groups
// per step), a per-CTA table of the pieces replaces the search over the groups.
// Global traffic is one contiguous read stream per source group and one write stream per
// destination group.  The ragged tail (fewer than R records) goes move by move through the warp
// that would own the next chunk.
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"
#include "remap_common.cuh"

namespace adha {

__device__ __forceinline__ int align16(int x) { return (x + 15) & ~15; }

template <bool DIRECT>
__global__ void __launch_bounds__(kThreads) remap_kernel(const __grid_constant__ RemapArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int in_pieces = (a.pieces & 1) ? a.in_bytes / 16 : 0, out_pieces = (a.pieces & 2) ? a.out_bytes / 16 : 0;
  Piece* pin = reinterpret_cast<Piece*>(smem);
  Piece* pout = pin + in_pieces;
  GroupRef* tin = reinterpret_cast<GroupRef*>(pout + out_pieces);
  GroupRef* tout = tin + a.n_src;
  const int n_entries = a.R * a.n_moves;
  uint32_t* sched = reinterpret_cast<uint32_t*>(tout + a.n_dst);
  uint8_t* wbase = reinterpret_cast<uint8_t*>(sched) + align16(n_entries * 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = a.buffers;
  uint8_t* buf0 = wbase + (size_t)warp * (nb * (a.in_bytes + kZeroTail) + a.out_bytes);
  uint8_t* buf1 = buf0 + (nb - 1) * (a.in_bytes + kZeroTail);
  uint8_t* outb = buf0 + nb * (a.in_bytes + kZeroTail);
  if (lane < nb) *reinterpret_cast<uint4*>((lane ? buf1 : buf0) + a.in_bytes) = make_uint4(0, 0, 0, 0);

  for (int q = tid; q < in_pieces; q += kThreads) pin[q] = piece_of(q, a.src, a.R);
  for (int q = tid; q < out_pieces; q += kThreads) pout[q] = piece_of(q, a.dst, a.R);
  for (int k = tid; k < a.n_src; k += kThreads) tin[k] = a.src[k];
  for (int k = tid; k < a.n_dst; k += kThreads) tout[k] = a.dst[k];
  for (int t = tid; t < n_entries; t += kThreads)
    sched[t] = schedule_entry(t, a.R, a.cls_count, a.cls_order, a.move, a.src, a.dst, a.in_bytes);
  __syncthreads();

  const int64_t W = (int64_t)gridDim.x * kWarps;
  const int64_t R = a.R;
  // lane l moves pieces l, l + 32, ... (16 bytes each: coalesced within every slice), finding
  // each piece's group by a search that resumes where the last piece's ended, or in the table
  auto stage = [&](int64_t ch, uint8_t* buf) {
    if (a.pieces & 1) {
#pragma unroll 1
      for (int q = lane; q < in_pieces; q += 32) {
        const Piece pc = pin[q];
        cp_async16(buf + q * 16, pc.base + ch * pc.step);
      }
    } else {
      int g = 0;
      for (int p = lane * 16; p < a.in_bytes; p += 512) {
        while (p >= tin[g].start + a.R * tin[g].stride) ++g;
        cp_async16(buf + p, tin[g].ptr + ch * R * tin[g].stride + (p - tin[g].start));
      }
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
    move_chunk<DIRECT>(sched, a.R, a.cls_count, cur, outb, tout, c * R, lane);
    __syncwarp();
    if (nb == 1 && c + W < a.n_chunks) {   // one buffer: the next chunk once the moves have read this one
      stage(c + W, buf0);
      cp_async_commit();
    }
    if (a.pieces & 2) {
#pragma unroll 1
      for (int q = lane; q < out_pieces; q += 32) {
        const Piece pc = pout[q];
        *reinterpret_cast<uint4*>(const_cast<uint8_t*>(pc.base) + c * pc.step) =
            *reinterpret_cast<const uint4*>(outb + q * 16);
      }
    } else {
      write_back<DIRECT>(tout, a.R, a.out_bytes, outb, c, lane);
    }
    __syncwarp();
  }
  cp_async_wait<0>();

  // ragged tail: the warp whose next chunk would be n_chunks
  const int64_t t0 = a.n_chunks * R;
  if (c == a.n_chunks && t0 < a.n) tail_moves(t0, a.n, a.n_moves, a.cls_count, a.move, tin, tout, lane);
}

size_t remap_smem_bytes(const RemapArgs& a) {
  auto al = [](size_t x) { return (x + 15) / 16 * 16; };
  const size_t pieces = ((a.pieces & 1) ? a.in_bytes / 16 : 0) + ((a.pieces & 2) ? a.out_bytes / 16 : 0);
  return pieces * sizeof(Piece) + (size_t)(a.n_src + a.n_dst) * sizeof(GroupRef) + al((size_t)a.R * a.n_moves * 4) +
         (size_t)kWarps * ((size_t)a.buffers * ((size_t)a.in_bytes + kZeroTail) + a.out_bytes);
}

template <bool DIRECT>
static int launch_d(const RemapArgs& a, int grid, size_t smem, void* stream) {
  cudaError_t e = cudaFuncSetAttribute(remap_kernel<DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(remap)");
  remap_kernel<DIRECT><<<grid, kThreads, smem, (cudaStream_t)stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "remap kernel launch");
  return 0;
}

int launch_remap(const RemapArgs& a, int grid, size_t smem, void* stream) {
  const bool direct = a.cls_count[0] + a.cls_count[1] + a.cls_count[2] > 0;
  return direct ? launch_d<true>(a, grid, smem, stream) : launch_d<false>(a, grid, smem, stream);
}

template <bool DIRECT>
static int occ_d(size_t smem, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(remap_kernel<DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(remap)");
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, remap_kernel<DIRECT>, kThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(remap)");
  return 0;
}

int remap_occupancy(int direct, size_t smem, int* blocks) {
  return direct ? occ_d<true>(smem, blocks) : occ_d<false>(smem, blocks);
}

}  // namespace adha

// batched.cu -- many record arrays remapped in one persistent launch.
//
// Each array (its own schema, record count and source/destination layouts) is cut into chunks
// of R_a records, and its chunks into work blocks (about 2048 records per working warp).  A CTA holds a
// budget of shared memory for its warps' buffers, set when the batch is created from the number of
// CTAs per SM (1 to 4) that gives the most working warps weighted by the arrays' bytes; an array
// whose records are too wide for eight warps' buffers in that budget is worked on by fewer warps
// of the CTA.  A CTA takes the next block with one atomic ticket (a 64-bit counter in the caller's
// workspace, zeroed by a memset node before every launch), builds the block's array's element
// schedule (and, where the array uses them, its piece tables) in shared memory when the array
// changes, and its warps run the same double-buffered cp.async pipeline as remap.cu on the
// block's chunks.  Blocks of small arrays and of large arrays are interleaved by the ticket
// order, so uneven sizes balance across SMs without any waiting between CTAs.  The descriptors
// live in the workspace; the launch (memset + kernel) can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "remap_common.cuh"

namespace adha {

constexpr int kBlockRecordsPerWarp = 2048;   // a work block gives each working warp about this many records

struct BatchHeader {
  int64_t n, n_full, n_chunks, block0;
  int32_t R, n_src, n_dst, in_bytes, out_bytes, n_moves;
  int32_t cls_count[6], cls_order[6];
  int32_t group0, move0;
  int32_t warps;        // warps of a CTA that work on this array (the others idle for its blocks)
  int32_t chunks_per_warp;   // chunks of one working warp in one work block
  int32_t warp_bytes;   // shared bytes of one working warp: two input buffers and an output buffer
  int32_t pieces;       // bit 0: stage through the piece table, bit 1: write back through it
};

// Warp bytes up to which the autotuner considers chunks longer than 32 records.
constexpr int kTuneWarpBytes = 8 * 1024;

struct BatchParams {
  unsigned long long* ticket;
  const BatchHeader* headers;
  const GroupRef* groups;
  const Move* moves;
  const int64_t* prefix;     // first block of each array, n_arrays + 1 entries
  int32_t n_arrays;
  int64_t total_blocks;
  int32_t max_entries;
  int32_t max_pieces;        // piece-table entries of the array that needs the most
};

template <bool DIRECT>
__global__ void __launch_bounds__(kThreads) batched_kernel(const __grid_constant__ BatchParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BatchHeader h;
  __shared__ unsigned long long s_blk;
  __shared__ int s_arr;
  GroupRef* tin = reinterpret_cast<GroupRef*>(smem);
  GroupRef* tout = tin + kMaxGroups;
  Move* moves = reinterpret_cast<Move*>(tout + kMaxGroups);
  uint32_t* sched = reinterpret_cast<uint32_t*>(moves + kMaxMoves);
  Piece* pin = reinterpret_cast<Piece*>(sched + p.max_entries);   // max_entries is a multiple of 4
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* wbase = reinterpret_cast<uint8_t*>(pin + p.max_pieces);
  int cur = -1;
  int in_pieces = 0, out_pieces = 0;
  Piece* pout = pin;

  for (;;) {
    if (tid == 0) {
      s_blk = atomicAdd(p.ticket, 1ull);
      int lo = 0, hi = p.n_arrays - 1;   // last array whose first block is <= s_blk
      const int64_t b = (int64_t)s_blk;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (p.prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
      }
      s_arr = lo;
    }
    __syncthreads();
    const int64_t blk = (int64_t)s_blk;
    if (blk >= p.total_blocks) break;
    const int arr = s_arr;
    if (arr != cur) {
      if (tid == 0) h = p.headers[arr];
      __syncthreads();
      for (int k = tid; k < h.n_src; k += kThreads) tin[k] = p.groups[h.group0 + k];
      for (int k = tid; k < h.n_dst; k += kThreads) tout[k] = p.groups[h.group0 + h.n_src + k];
      for (int k = tid; k < h.n_moves; k += kThreads) moves[k] = p.moves[h.move0 + k];
      __syncthreads();
      for (int t = tid; t < h.R * h.n_moves; t += kThreads)
        sched[t] = schedule_entry(t, h.R, h.cls_count, h.cls_order, moves, tin, tout);
      in_pieces = (h.pieces & 1) ? h.in_bytes / 16 : 0;
      out_pieces = (h.pieces & 2) ? h.out_bytes / 16 : 0;
      pout = pin + in_pieces;
      for (int q = tid; q < in_pieces; q += kThreads) pin[q] = piece_of(q, tin, h.R);
      for (int q = tid; q < out_pieces; q += kThreads) pout[q] = piece_of(q, tout, h.R);
      __syncthreads();
      cur = arr;
    }
    const int nw = h.warps;
    const int64_t per_block = (int64_t)h.chunks_per_warp * nw;
    const int64_t c_begin = (blk - h.block0) * per_block;
    const int64_t c_end = c_begin + per_block < h.n_chunks ? c_begin + per_block : h.n_chunks;
    uint8_t* buf0 = wbase + (size_t)warp * h.warp_bytes;
    uint8_t* buf1 = buf0 + h.in_bytes;
    uint8_t* outb = buf1 + h.in_bytes;
    const int64_t full_end = c_end < h.n_full ? c_end : h.n_full;
    const int64_t R = h.R;
    const int in_bytes = h.in_bytes, pieces = h.pieces;
    auto stage = [&](int64_t ch, uint8_t* buf) {
      if (pieces & 1) {
#pragma unroll 1
        for (int q = lane; q < in_pieces; q += 32) {
          const Piece pc = pin[q];
          cp_async16(buf + q * 16, pc.base + ch * pc.step);
        }
      } else {
        int g = 0;
        for (int q = lane * 16; q < in_bytes; q += 512) {
          while (q >= tin[g].start + (int)R * tin[g].stride) ++g;
          cp_async16(buf + q, tin[g].ptr + ch * R * tin[g].stride + (q - tin[g].start));
        }
      }
    };
    int64_t c = warp < nw ? c_begin + warp : full_end;
    if (c < full_end) stage(c, buf0);
    cp_async_commit();
    for (int i = 0; c < full_end; c += nw, ++i) {
      uint8_t* curb = (i & 1) ? buf1 : buf0;
      if (c + nw < full_end) stage(c + nw, (i & 1) ? buf0 : buf1);
      cp_async_commit();
      cp_async_wait<1>();
      __syncwarp();
      move_chunk<DIRECT>(sched, h.R, h.cls_count, curb, outb, tout, c * R, lane);
      __syncwarp();
      if (pieces & 2) {
#pragma unroll 1
        for (int q = lane; q < out_pieces; q += 32) {
          const Piece pc = pout[q];
          *reinterpret_cast<uint4*>(const_cast<uint8_t*>(pc.base) + c * pc.step) =
              *reinterpret_cast<const uint4*>(outb + q * 16);
        }
      } else {
        write_back<DIRECT>(tout, h.R, h.out_bytes, outb, c, lane);
      }
      __syncwarp();
    }
    cp_async_wait<0>();
    // the array's ragged tail chunk, by the warp it falls to
    if (warp < nw && h.n_full < h.n_chunks && h.n_full >= c_begin && h.n_full < c_end && (h.n_full - c_begin) % nw == warp)
      tail_moves(h.n_full * h.R, h.n, h.n_moves, h.cls_count, moves, tin, tout, lane);
    __syncthreads();
  }
}

}  // namespace adha

using namespace adha;

struct adha_batched {
  int32_t n_arrays = 0;
  std::vector<uint8_t> image;      // descriptor region as it is copied to the workspace
  size_t off_headers = 0, off_groups = 0, off_moves = 0, off_prefix = 0;
  int64_t total_blocks = 0;
  int32_t max_entries = 0, max_pieces = 0, warp_budget = 0;
  size_t smem = 0;
  int grid = 1;
  double bytes = 0;
  bool direct = false;          // some array stores one-field destination groups directly
  cudaGraphExec_t graph = nullptr;
  void* graph_ws = nullptr;
};

namespace adha {

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

static BatchParams params_for(const adha_batched* b, void* ws) {
  uint8_t* base = static_cast<uint8_t*>(ws);
  BatchParams p;
  p.ticket = reinterpret_cast<unsigned long long*>(base);
  p.headers = reinterpret_cast<const BatchHeader*>(base + b->off_headers);
  p.groups = reinterpret_cast<const GroupRef*>(base + b->off_groups);
  p.moves = reinterpret_cast<const Move*>(base + b->off_moves);
  p.prefix = reinterpret_cast<const int64_t*>(base + b->off_prefix);
  p.n_arrays = b->n_arrays;
  p.total_blocks = b->total_blocks;
  p.max_entries = b->max_entries;
  p.max_pieces = b->max_pieces;
  return p;
}

static int launch_batched(const adha_batched* b, void* ws, void* stream) {
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(unsigned long long), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(ticket)");
  if (b->total_blocks == 0) return 0;
  auto* k = b->direct ? batched_kernel<true> : batched_kernel<false>;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(batched)");
  k<<<b->grid, kThreads, b->smem, (cudaStream_t)stream>>>(params_for(b, ws));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batched kernel launch");
  return 0;
}

// Default chunk of an array in the batched kernel: the single-array rule, but at least 32 records.
static int batch_chunk(const Layout& S, const Layout& D) {
  int src = 0, dst = 0;
  for (int g = 0; g < S.n_groups; ++g) src += S.stride[g];
  for (int g = 0; g < D.n_groups; ++g) dst += D.stride[g];
  int R = 32;
  while (R < 512 && 2 * R * std::max(src, dst) <= 4096) R *= 2;
  return R;
}

// Chooses each array's chunk size, direct stores and piece tables: the default rules, or
// (autotune) the fastest measured with the single-array remap kernel on the array's own buffers:
// first 32..256 records x direct stores, then the four piece-table choices for the best of those.
static int tune_chunk(const Layout& S, const void* const* sp, const Layout& D, void* const* dp, int64_t n, void* stream,
                      int* best_R, int* best_direct, int* best_pieces) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(ADHA_ECUDA, "cudaEventCreate");
  auto time_ms = [&](int R, int direct, int pieces, float* ms) {
    adha_tune_override(R);
    adha_tune_remap_direct(direct);
    adha_tune_remap_pieces(pieces);
    int rc = 0;
    for (int w = 0; w < 2 && !rc; ++w) rc = remap_layouts(S, sp, D, dp, n, stream, nullptr);
    cudaEventRecord(e0, (cudaStream_t)stream);
    for (int w = 0; w < 3 && !rc; ++w) rc = remap_layouts(S, sp, D, dp, n, stream, nullptr);
    cudaEventRecord(e1, (cudaStream_t)stream);
    adha_tune_override(0);
    adha_tune_remap_direct(0);
    adha_tune_remap_pieces(0);
    if (rc) return rc;
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    return 0;
  };
  float best = -1, ms = 0;
  int rc = 0;
  // 32..256 records (shorter chunks only add per-chunk work); longer ones only while a warp's
  // buffers stay small enough for a CTA's eight warps
  for (int trial = 0; trial < 8 && !rc; ++trial) {
    const int R = 32 << (trial >> 1), direct = trial & 1;
    RemapArgs a;
    bool empty = false;
    rc = remap_plan_args(S, sp, D, dp, n, R, direct, &a, &empty);
    if (rc || empty) break;
    if (2 * a.in_bytes + a.out_bytes > kTuneWarpBytes && R > 32) continue;
    rc = time_ms(R, direct, 0, &ms);
    if (!rc && (best < 0 || ms < best)) {
      best = ms;
      *best_R = R;
      *best_direct = direct;
      *best_pieces = a.pieces;
    }
  }
  for (int m = 1; m <= 4 && !rc && best >= 0; ++m) {
    rc = time_ms(*best_R, *best_direct, m, &ms);
    if (!rc && ms < best) {
      best = ms;
      *best_pieces = m - 1;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace adha

extern "C" {

int adha_batched_create(int32_t n_arrays, const adha_remap_desc* descs, int32_t flags, adha_stream stream,
                        adha_batched** out) {
  clear_error();
  if (!out || !descs || n_arrays < 1) return fail(ADHA_EINVAL, "bad batched arguments");
  auto* b = new (std::nothrow) adha_batched();
  if (!b) return fail(ADHA_ENOMEM, "host allocation failed");
  std::vector<BatchHeader> headers;
  std::vector<GroupRef> groups;
  std::vector<Move> moves;
  std::vector<double> moved_bytes;   // per array, for the choice of CTAs per SM
  int max_pieces = 0, max_warp = 0;
  for (int k = 0; k < n_arrays; ++k) {
    const adha_remap_desc& d = descs[k];
    Layout S, D;
    int rc = make_layout(d.schema, d.src, &S, "source");
    if (!rc) rc = make_layout(d.schema, d.dst, &D, "destination");
    if (!rc && d.n < 0) rc = fail(ADHA_EINVAL, "array %d has n = %lld", k, (long long)d.n);
    if (!rc && d.n > 0) {
      for (int g = 0; g < S.n_groups && !rc; ++g)
        if (!d.src_ptrs || !d.src_ptrs[g] || reinterpret_cast<uintptr_t>(d.src_ptrs[g]) % 16)
          rc = fail(ADHA_EINVAL, "array %d source buffer %d is NULL or misaligned", k, g);
      for (int g = 0; g < D.n_groups && !rc; ++g)
        if (!d.dst_ptrs || !d.dst_ptrs[g] || reinterpret_cast<uintptr_t>(d.dst_ptrs[g]) % 16)
          rc = fail(ADHA_EINVAL, "array %d destination buffer %d is NULL or misaligned", k, g);
    }
    int R = 0, direct = 0, pieces = -1;
    if (!rc && d.n > 0 && (flags & ADHA_BATCHED_AUTOTUNE))
      rc = tune_chunk(S, d.src_ptrs, D, d.dst_ptrs, d.n, stream, &R, &direct, &pieces);
    RemapArgs a;
    bool empty = true;
    if (!rc && d.n > 0) rc = remap_plan_args(S, d.src_ptrs, D, d.dst_ptrs, d.n, R ? R : batch_chunk(S, D), direct, &a, &empty);
    if (rc) {
      delete b;
      return rc;
    }
    BatchHeader h;
    std::memset(&h, 0, sizeof h);
    double moved = 0;
    if (!empty) {
      h.n = a.n;
      h.R = a.R;
      h.n_full = a.n_chunks;
      h.n_chunks = a.n_chunks + (a.n % a.R ? 1 : 0);
      h.n_src = a.n_src;
      h.n_dst = a.n_dst;
      h.in_bytes = a.in_bytes;
      h.out_bytes = a.out_bytes;
      h.n_moves = a.n_moves;
      for (int c = 0; c < 6; ++c) {
        h.cls_count[c] = a.cls_count[c];
        h.cls_order[c] = a.cls_order[c];
      }
      h.pieces = pieces >= 0 ? pieces : a.pieces;
      b->direct = b->direct || (a.cls_count[0] + a.cls_count[1] + a.cls_count[2] > 0);
      h.group0 = (int32_t)groups.size();
      h.move0 = (int32_t)moves.size();
      h.warp_bytes = 2 * a.in_bytes + a.out_bytes;
      max_warp = std::max(max_warp, h.warp_bytes);
      max_pieces = std::max(max_pieces, ((h.pieces & 1) ? a.in_bytes / 16 : 0) + ((h.pieces & 2) ? a.out_bytes / 16 : 0));
      for (int g = 0; g < a.n_src; ++g) groups.push_back(a.src[g]);
      for (int g = 0; g < a.n_dst; ++g) groups.push_back(a.dst[g]);
      moves.insert(moves.end(), a.move, a.move + a.n_moves);
      h.chunks_per_warp = std::max(1, kBlockRecordsPerWarp / h.R);
      b->max_entries = std::max(b->max_entries, a.R * a.n_moves);
      for (int g = 0; g < D.n_groups; ++g) {
        bool alias = false;
        for (int j = 0; j < S.n_groups; ++j) alias = alias || (same_group(D, g, S, j) && d.dst_ptrs[g] == d.src_ptrs[j]);
        if (!alias)
          for (int f : D.groups[g]) moved += dtype_size(D.dtype[f]);
      }
      b->bytes += 2.0 * moved * (double)d.n;
    }
    moved_bytes.push_back(2.0 * moved * (double)d.n);
    headers.push_back(h);
  }
  b->max_entries = (b->max_entries + 3) / 4 * 4;
  b->max_pieces = max_pieces;

  // CTAs per SM: 1..4, each with the shared memory left by the others; the warp-buffer budget is
  // what remains after the tables.  The choice maximises the working warps per SM weighted by
  // each array's bytes (an array gets as many warps of a CTA as its buffers fit, at most 8).
  int sms = 0, dev = 0, sm_smem = 0, reserved = 0, optin = 0;
  if (int rc = sm_count(&sms)) {
    delete b;
    return rc;
  }
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  auto* kern = b->direct ? batched_kernel<true> : batched_kernel<false>;
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "device attributes for the batched kernel");
  }
  const size_t fixed = (size_t)2 * kMaxGroups * sizeof(GroupRef) + kMaxMoves * sizeof(Move) +
                       (size_t)b->max_entries * 4 + (size_t)max_pieces * sizeof(Piece);
  double best_score = -1;
  for (int k = 1; k <= 4; ++k) {
    const int64_t dyn = std::min<int64_t>(optin, (int64_t)sm_smem / k - reserved - (int64_t)fa.sharedSizeBytes) / 16 * 16;
    const int64_t budget = dyn - (int64_t)fixed;
    if (budget < std::max(max_warp, 1)) continue;
    double score = 0;
    for (size_t a = 0; a < headers.size(); ++a)
      if (headers[a].warp_bytes > 0)
        score += moved_bytes[a] * k * std::min<int64_t>(kWarps, budget / headers[a].warp_bytes);
    if (score > best_score) {
      best_score = score;
      b->warp_budget = (int32_t)budget;
    }
  }
  if (best_score < 0) {
    const size_t need = fixed + (size_t)max_warp;
    delete b;
    return fail(ADHA_ENOTIMPL, "batched remap needs %zu bytes of shared memory per CTA (limit %d): an array is too wide",
                need, optin);
  }
  std::vector<int64_t> prefix;
  int64_t blocks = 0;
  for (BatchHeader& h : headers) {
    h.block0 = blocks;
    prefix.push_back(blocks);
    if (h.warp_bytes == 0) continue;
    h.warps = (int32_t)std::max(1, std::min(kWarps, b->warp_budget / h.warp_bytes));
    const int64_t per_block = (int64_t)h.chunks_per_warp * h.warps;
    blocks += (h.n_chunks + per_block - 1) / per_block;
  }
  prefix.push_back(blocks);
  b->n_arrays = n_arrays;
  b->total_blocks = blocks;
  b->off_headers = al256(sizeof(unsigned long long));
  b->off_groups = b->off_headers + al256(headers.size() * sizeof(BatchHeader));
  b->off_moves = b->off_groups + al256(std::max<size_t>(1, groups.size()) * sizeof(GroupRef));
  b->off_prefix = b->off_moves + al256(std::max<size_t>(1, moves.size()) * sizeof(Move));
  b->image.assign(b->off_prefix + al256(prefix.size() * sizeof(int64_t)), 0);
  std::memcpy(b->image.data() + b->off_headers, headers.data(), headers.size() * sizeof(BatchHeader));
  if (!groups.empty()) std::memcpy(b->image.data() + b->off_groups, groups.data(), groups.size() * sizeof(GroupRef));
  if (!moves.empty()) std::memcpy(b->image.data() + b->off_moves, moves.data(), moves.size() * sizeof(Move));
  std::memcpy(b->image.data() + b->off_prefix, prefix.data(), prefix.size() * sizeof(int64_t));
  b->smem = fixed + (size_t)b->warp_budget;
  int per_sm = 0;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, b->smem);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batched occupancy");
  }
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(1, per_sm), blocks));
  *out = b;
  return 0;
}

size_t adha_batched_workspace_bytes(const adha_batched* b) { return b ? b->image.size() : 0; }

int adha_batched_upload(const adha_batched* b, void* workspace, size_t ws_bytes, adha_stream stream) {
  clear_error();
  if (!b || !workspace) return fail(ADHA_EINVAL, "NULL batched plan or workspace");
  if (ws_bytes < b->image.size()) return fail(ADHA_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, b->image.size());
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(ADHA_EINVAL, "workspace is not 256-byte aligned");
  cudaError_t e = cudaMemcpyAsync(workspace, b->image.data(), b->image.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "upload of the batched descriptors");
  e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(upload)");
  return 0;
}

static int batched_fn(const void* ctx) {
  const auto* c = static_cast<const std::pair<const adha_batched*, std::pair<void*, void*>>*>(ctx);
  return launch_batched(c->first, c->second.first, c->second.second);
}

int adha_batched_launch(const adha_batched* b, void* workspace, adha_stream stream) {
  clear_error();
  if (!b || !workspace) return fail(ADHA_EINVAL, "NULL batched plan or workspace");
  const std::pair<const adha_batched*, std::pair<void*, void*>> ctx{b, {workspace, stream}};
  return profiled_launch(3, 0, b->bytes, stream, batched_fn, &ctx);
}

int adha_batched_graph(adha_batched* b, void* workspace, adha_stream stream) {
  clear_error();
  if (!b || !workspace) return fail(ADHA_EINVAL, "NULL batched plan or workspace");
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  // Capture on a private stream (the legacy default stream cannot be captured); the graph is
  // later launched on the caller's stream.  `stream` is synchronized first so that the capture
  // does not race with work already queued there.
  (void)stream;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "capture stream");
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(s);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  const int rc = launch_batched(b, workspace, s);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  cudaStreamDestroy(s);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  b->graph_ws = workspace;
  return 0;
}

static int graph_fn(const void* ctx) {
  const auto* c = static_cast<const std::pair<const adha_batched*, void*>*>(ctx);
  cudaError_t e = cudaGraphLaunch(c->first->graph, (cudaStream_t)c->second);
  return e == cudaSuccess ? 0 : cuda_fail(e, "cudaGraphLaunch");
}

int adha_batched_graph_launch(const adha_batched* b, adha_stream stream) {
  clear_error();
  if (!b || !b->graph) return fail(ADHA_EINVAL, "no captured graph: call adha_batched_graph first");
  const std::pair<const adha_batched*, void*> ctx{b, stream};
  return profiled_launch(3, 1, b->bytes, stream, graph_fn, &ctx);
}

void adha_batched_destroy(adha_batched* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
}

double adha_batched_bytes(const adha_batched* b) { return b ? b->bytes : 0.0; }

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batched remap without a caller workspace.
//
// For callers that cannot allocate device memory (for example code that runs where cudaMalloc
// is forbidden or would break an outer allocator's accounting, or plugins handed only their
// input and output buffers), the descriptors and the work ticket of the batched remap can live
// in this file-scope device array instead of a caller workspace.  Every GPU that loads the
// library holds the array until the process exits.  All calls share it and it keeps the last
// call's contents: each call rewrites the descriptors and zeroes the ticket before its kernel,
// so calls that overlap on the GPU (on different streams, unordered) race on it.

namespace adha {

static __device__ __align__(256) uint8_t g_noalloc_scratch[ADHA_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256];

// Device address of the scratch array on the current device, looked up once per device (the
// host-side name of a __device__ array is only a stand-in, not a device address).
static int noalloc_scratch(void** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(ADHA_ENOTIMPL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(batched scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return 0;
}

}  // namespace adha

extern "C" int adha_remap_batched_noalloc(int32_t n_arrays, const adha_remap_desc* descs, adha_stream stream) {
  clear_error();
  void* scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  adha_batched* b = nullptr;
  if (int rc = adha_batched_create(n_arrays, descs, 0, stream, &b)) return rc;
  const size_t need = b->image.size();
  if (need > (size_t)ADHA_NOALLOC_SCRATCH_BYTES) {
    adha_batched_destroy(b);
    return fail(ADHA_EINVAL, "this batch needs %zu bytes of descriptors; the allocation-free entry point holds at most %u",
                need, (unsigned)ADHA_NOALLOC_SCRATCH_BYTES);
  }
  // Pageable source: the call returns once the bytes are staged, so the host image can go.
  cudaError_t e = cudaMemcpyAsync(scratch, b->image.data(), need, cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    adha_batched_destroy(b);
    return cuda_fail(e, "copy of the batched descriptors into the scratch array");
  }
  const std::pair<const adha_batched*, std::pair<void*, void*>> ctx{b, {scratch, stream}};
  const int rc = profiled_launch(3, 2, b->bytes, stream, batched_fn, &ctx);
  adha_batched_destroy(b);
  return rc;
}

// batched.cu -- many record arrays remapped in one persistent launch (the batching form of the
// paper's remap edge, Section 2).
//
// Every array (its own schema, record count and source/destination layouts) is cut into chunks
// of R_a records, and its chunks into work units of about 1024 records.  Each warp works alone:
// it takes the next unit with one 64-bit atomic ticket (in the descriptor region, zeroed before
// every launch), finds the unit's array by a 32-way search over the arrays' first units (one
// ballot per level), and, when the array differs from its last one, copies that array's header,
// group table and element schedule (built on the host when the batch is prepared) into its own
// region of shared memory.  It then runs the cp.async pipeline of remap.cu over the unit's
// consecutive chunks: stage the source slices with 16-byte copies, assemble the destination
// records one move per lane per step, write them back with 16-byte stores.  With one input
// buffer per warp (the default) the next chunk is staged as soon as the moves have read the
// current one, so its copy overlaps the write-back, and the shared memory saved goes to longer
// chunks; with two, the next chunk is staged before the current one is moved.  No warp ever waits for another: there is no block-wide barrier anywhere, so uneven
// arrays and ragged tails cost only their own work.  Units are dealt largest array first, so
// the small arrays' single units fill the last gaps.  The launch (memset + kernel) can be
// captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "remap_common.cuh"

namespace adha {

constexpr int kUnitRecords = 1024;   // records of one work unit (whole chunks, at least one)
constexpr int kHeaderBytes = 128;    // a warp region starts with the header of its current array
constexpr int kMaxBatchedCtas = 8;   // CTAs per SM tried (8 x 8 warps = 64 warps, the SM's limit)

struct BatchHeader {
  int64_t n, n_full, n_chunks;   // records, whole chunks, chunks counting the ragged one
  int64_t unit0;                 // first work unit of the array
  int64_t sched0;                // byte offset of the array's schedule in the schedule region
  int32_t R, n_src, n_dst, in_bytes, out_bytes, n_moves;
  int32_t cls_count[6];
  int32_t group0, move0;
  int32_t chunks_per_unit;
  int32_t sched_off, buf_off;    // offsets in a warp region: the schedule, the first chunk buffer
  int32_t sched_bytes;
};
static_assert(sizeof(BatchHeader) <= kHeaderBytes && sizeof(BatchHeader) % 16 == 0, "header is copied in words");
static_assert(sizeof(GroupRef) == 16, "group table is copied in 16-byte words");

struct BatchParams {
  unsigned long long* ticket;
  const BatchHeader* headers;    // in ticket order (largest array first); arrays with nothing to move are left out
  const GroupRef* groups;
  const Move* moves;
  const uint8_t* sched;
  const int64_t* prefix;         // first unit of each listed array; prefix[n_arrays] = total_units
  int32_t n_arrays;
  int32_t region;                // shared bytes of one warp
  int32_t buffers;               // input chunk buffers per warp: 2 (the next chunk staged during this one) or 1
  int64_t total_units;
};

// Last array a with prefix[a] <= u: a 32-way search, one ballot per level (prefix[0] = 0 <= u,
// so lane 0 always qualifies and the answer stays inside [lo, lo + span)).
__device__ __forceinline__ int find_array(const int64_t* prefix, int n_arrays, int64_t u, int lane) {
  int lo = 0, span = n_arrays;
  while (span > 1) {
    const int step = (span + 31) >> 5, end = lo + span;
    const int idx = lo + lane * step;
    const bool ok = idx < end && __ldg(prefix + idx) <= u;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, ok);
    lo += (31 - __clz(m)) * step;
    span = min(step, end - lo);
  }
  return lo;
}

template <bool DIRECT>
__global__ void __launch_bounds__(kThreads) batched_kernel(const __grid_constant__ BatchParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* region = smem + (size_t)warp * p.region;
  const BatchHeader& h = *reinterpret_cast<const BatchHeader*>(region);
  GroupRef* tin = reinterpret_cast<GroupRef*>(region + kHeaderBytes);
  int cur = -1;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1ull);
    const int64_t u = (int64_t)__shfl_sync(0xFFFFFFFFu, t, 0);
    if (u >= p.total_units) break;
    const int arr = find_array(p.prefix, p.n_arrays, u, lane);
    if (arr != cur) {   // the warp's tables for this array: header, groups, schedule
      __syncwarp();
      const uint32_t* hs = reinterpret_cast<const uint32_t*>(p.headers + arr);
      if (lane < (int)(sizeof(BatchHeader) / 4)) reinterpret_cast<uint32_t*>(region)[lane] = __ldg(hs + lane);
      __syncwarp();
      const uint4* gs = reinterpret_cast<const uint4*>(p.groups + h.group0);
      for (int k = lane; k < h.n_src + h.n_dst; k += 32) reinterpret_cast<uint4*>(tin)[k] = __ldg(gs + k);
      const uint4* ss = reinterpret_cast<const uint4*>(p.sched + h.sched0);
      uint4* sd = reinterpret_cast<uint4*>(region + h.sched_off);
      for (int k = lane; k < h.sched_bytes / 16; k += 32) sd[k] = __ldg(ss + k);
      // the zeros that padding moves read, after each input buffer
      if (lane < p.buffers)
        *reinterpret_cast<uint4*>(region + h.buf_off + lane * (h.in_bytes + kZeroTail) + h.in_bytes) = make_uint4(0, 0, 0, 0);
      __syncwarp();
      cur = arr;
    }
    const GroupRef* tout = tin + h.n_src;
    const uint32_t* sched = reinterpret_cast<const uint32_t*>(region + h.sched_off);
    uint8_t* buf0 = region + h.buf_off;
    const int nb = p.buffers;
    uint8_t* buf1 = buf0 + (nb - 1) * (h.in_bytes + kZeroTail);
    uint8_t* outb = buf0 + nb * (h.in_bytes + kZeroTail);
    const int R = h.R, in_bytes = h.in_bytes;
    const int64_t c_begin = (u - h.unit0) * h.chunks_per_unit;
    const int64_t c_end = min(c_begin + (int64_t)h.chunks_per_unit, h.n_chunks);
    const int64_t full_end = min(c_end, h.n_full);
    // lane l copies the 16-byte pieces l, l + 32, ... of the chunk's source slices, finding each
    // piece's group by a search that resumes where the last piece's ended
    auto stage = [&](int64_t ch, uint8_t* buf) {
      int g = 0;
      for (int q = lane * 16; q < in_bytes; q += 512) {
        while (q >= tin[g].start + R * tin[g].stride) ++g;
        cp_async16(buf + q, tin[g].ptr + ch * R * tin[g].stride + (q - tin[g].start));
      }
    };
    int64_t c = c_begin;
    if (c < full_end) stage(c, buf0);
    cp_async_commit();
    for (int i = 0; c < full_end; ++c, ++i) {
      uint8_t* curb = (i & 1) ? buf1 : buf0;
      if (nb == 2) {
        if (c + 1 < full_end) stage(c + 1, (i & 1) ? buf0 : buf1);
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      move_chunk<DIRECT>(sched, R, h.cls_count, curb, outb, tout, c * R, lane);
      __syncwarp();
      if (nb == 1 && c + 1 < full_end) {   // one buffer: the next chunk once the moves have read this one
        stage(c + 1, buf0);
        cp_async_commit();
      }
      write_back<DIRECT>(tout, R, h.out_bytes, outb, c, lane);
      __syncwarp();
    }
    cp_async_wait<0>();
    // the array's ragged tail chunk (fewer than R records) lies in this unit: move by move
    if (c_end > h.n_full) tail_moves(h.n_full * R, h.n, h.n_moves, h.cls_count, p.moves + h.move0, tin, tout, lane);
    __syncwarp();
  }
}

}  // namespace adha

using namespace adha;

struct adha_batched {
  int32_t n_arrays = 0;            // arrays listed for the kernel (those with bytes to move)
  std::vector<uint8_t> image;      // descriptor region as it is copied to the workspace
  size_t off_headers = 0, off_groups = 0, off_moves = 0, off_sched = 0, off_prefix = 0;
  int64_t total_units = 0;
  int32_t region = 0;              // shared bytes per warp
  int32_t ctas_per_sm = 0;
  size_t smem = 0;
  int grid = 1;
  double bytes = 0;
  bool direct = false;             // some array stores one-field destination groups directly
  int32_t buffers = 1;             // input chunk buffers per warp
  cudaGraphExec_t graph = nullptr;
  void* graph_ws = nullptr;
};

namespace adha {

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }
static int al16(int x) { return (x + 15) / 16 * 16; }

static BatchParams params_for(const adha_batched* b, void* ws) {
  uint8_t* base = static_cast<uint8_t*>(ws);
  BatchParams p;
  p.ticket = reinterpret_cast<unsigned long long*>(base);
  p.headers = reinterpret_cast<const BatchHeader*>(base + b->off_headers);
  p.groups = reinterpret_cast<const GroupRef*>(base + b->off_groups);
  p.moves = reinterpret_cast<const Move*>(base + b->off_moves);
  p.sched = base + b->off_sched;
  p.prefix = reinterpret_cast<const int64_t*>(base + b->off_prefix);
  p.n_arrays = b->n_arrays;
  p.region = b->region;
  p.buffers = b->buffers;
  p.total_units = b->total_units;
  return p;
}

static int launch_batched(const adha_batched* b, void* ws, void* stream) {
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(unsigned long long), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(ticket)");
  if (b->total_units == 0) return 0;
  auto* k = b->direct ? batched_kernel<true> : batched_kernel<false>;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(batched)");
  k<<<b->grid, kThreads, b->smem, (cudaStream_t)stream>>>(params_for(b, ws));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batched kernel launch");
  return 0;
}

// Default chunk of an array: the single-array rule (about 4 KB of the wider side), at least 32
// records; the warp-region budget may shorten it.
static int batch_chunk(const Layout& S, const Layout& D) {
  int src = 0, dst = 0;
  for (int g = 0; g < S.n_groups; ++g) src += S.stride[g];
  for (int g = 0; g < D.n_groups; ++g) dst += D.stride[g];
  int R = 32;
  while (R < 512 && 2 * R * std::max(src, dst) <= 4096) R *= 2;
  return R;
}

// Shared bytes of one warp working on an array with chunks of R records: header, group table,
// schedule (R x moves entries of 4 bytes), nb input buffers (each followed by the zeros that
// padding moves read) and an output buffer.
static int warp_region_bytes(const RemapArgs& a, int R, int nb) {
  const int in_rec = a.in_bytes / a.R, out_rec = a.out_bytes / a.R;
  return kHeaderBytes + (a.n_src + a.n_dst) * (int)sizeof(GroupRef) + al16(R * a.n_moves * 4) +
         R * (nb * in_rec + out_rec) + nb * kZeroTail;
}

// Chooses an array's chunk size and direct stores (autotune): the fastest of 32..256 records x
// direct stores, timed with the single-array remap kernel on the array's own buffers (without
// piece tables, which the batched kernel does not use).
static int tune_chunk(const Layout& S, const void* const* sp, const Layout& D, void* const* dp, int64_t n, void* stream,
                      int* best_R, int* best_direct) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(ADHA_ECUDA, "cudaEventCreate");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ADHA_ECUDA, "cudaEventCreate");
  }
  auto time_ms = [&](int R, int direct, float* ms) {
    adha_tune_override(R);
    adha_tune_remap_direct(direct);
    adha_tune_remap_pieces(1);
    int rc = 0;
    for (int w = 0; w < 2 && !rc; ++w) rc = remap_layouts(S, sp, D, dp, n, stream, nullptr);
    cudaEventRecord(e0, (cudaStream_t)stream);
    for (int w = 0; w < 3 && !rc; ++w) rc = remap_layouts(S, sp, D, dp, n, stream, nullptr);
    cudaEventRecord(e1, (cudaStream_t)stream);
    adha_tune_override(0);
    adha_tune_remap_direct(0);
    adha_tune_remap_pieces(0);
    if (rc) return rc;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e == cudaSuccess ? 0 : cuda_fail(e, "timing a batched array");
  };
  float best = -1, ms = 0;
  int rc = 0;
  for (int trial = 0; trial < 8 && !rc; ++trial) {
    const int R = 32 << (trial >> 1), direct = trial & 1;
    RemapArgs a;
    bool empty = false;
    rc = remap_plan_args(S, sp, D, dp, n, R, direct, &a, &empty);
    if (rc || empty) break;
    if (a.R != R) continue;   // too wide for this chunk in the single-array kernel
    rc = time_ms(R, direct, &ms);
    if (!rc && (best < 0 || ms < best)) {
      best = ms;
      *best_R = R;
      *best_direct = direct;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

struct ArrayPlan {
  Layout S, D;
  int64_t n = 0;
  const void* const* sp = nullptr;
  void* const* dp = nullptr;
  int R0 = 0, direct = 0;   // preferred chunk, direct stores
  bool empty = true;
  double moved = 0;         // algorithmic bytes of the array
  RemapArgs a;              // at R0
};

}  // namespace adha

extern "C" {

int adha_batched_create(int32_t n_arrays, const adha_remap_desc* descs, int32_t flags, adha_stream stream,
                        adha_batched** out) {
  clear_error();
  if (!out || !descs || n_arrays < 1) return fail(ADHA_EINVAL, "bad batched arguments");
  const int forced_ctas = (flags >> 4) & 15;
  const int nb = (flags & ADHA_BATCHED_TWO_BUFFERS) ? 2 : 1;
  if (forced_ctas > kMaxBatchedCtas) return fail(ADHA_EINVAL, "ADHA_BATCHED_CTAS(%d) is not in 1..%d", forced_ctas, kMaxBatchedCtas);
  std::vector<ArrayPlan> plans(n_arrays);
  for (int k = 0; k < n_arrays; ++k) {
    const adha_remap_desc& d = descs[k];
    ArrayPlan& ap = plans[k];
    int rc = make_layout(d.schema, d.src, &ap.S, "source");
    if (!rc) rc = make_layout(d.schema, d.dst, &ap.D, "destination");
    if (!rc && d.n < 0) rc = fail(ADHA_EINVAL, "array %d has n = %lld", k, (long long)d.n);
    if (!rc && d.n > 0) {
      for (int g = 0; g < ap.S.n_groups && !rc; ++g)
        if (!d.src_ptrs || !d.src_ptrs[g] || reinterpret_cast<uintptr_t>(d.src_ptrs[g]) % 16)
          rc = fail(ADHA_EINVAL, "array %d source buffer %d is NULL or misaligned", k, g);
      for (int g = 0; g < ap.D.n_groups && !rc; ++g)
        if (!d.dst_ptrs || !d.dst_ptrs[g] || reinterpret_cast<uintptr_t>(d.dst_ptrs[g]) % 16)
          rc = fail(ADHA_EINVAL, "array %d destination buffer %d is NULL or misaligned", k, g);
    }
    if (rc) return rc;
    ap.n = d.n;
    ap.sp = d.src_ptrs;
    ap.dp = d.dst_ptrs;
    if (d.n == 0) continue;
    int R = 0, direct = 0;
    if (flags & ADHA_BATCHED_AUTOTUNE) rc = tune_chunk(ap.S, d.src_ptrs, ap.D, d.dst_ptrs, d.n, stream, &R, &direct);
    if (!rc) rc = remap_plan_args(ap.S, d.src_ptrs, ap.D, d.dst_ptrs, d.n, R ? R : batch_chunk(ap.S, ap.D), direct, &ap.a,
                                  &ap.empty);
    if (rc) return rc;
    ap.R0 = ap.a.R;
    ap.direct = direct;
    if (!ap.empty)
      for (int g = 0; g < ap.D.n_groups; ++g) {
        bool alias = false;
        for (int j = 0; j < ap.S.n_groups; ++j)
          alias = alias || (same_group(ap.D, g, ap.S, j) && d.dst_ptrs[g] == d.src_ptrs[j]);
        if (!alias)
          for (int f : ap.D.groups[g]) ap.moved += 2.0 * dtype_size(ap.D.dtype[f]) * (double)d.n;
      }
  }

  // CTAs per SM (1..4) and the shared region of a warp: every array must fit its chunk buffers
  // and tables in one region, shortening its chunk (down to 8 records) where it must.  The choice
  // maximises the arrays' bytes x CTAs per SM, discounted where an array's chunk had to shrink
  // below min(its preferred chunk, 32) records.
  int sms = 0, dev = 0, sm_smem = 0, reserved = 0, optin = 0;
  if (int rc = sm_count(&sms)) return rc;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  bool direct_any = false;
  for (const ArrayPlan& ap : plans) direct_any = direct_any || (!ap.empty && ap.a.cls_count[0] + ap.a.cls_count[1] + ap.a.cls_count[2] > 0);
  auto* kern = direct_any ? batched_kernel<true> : batched_kernel<false>;
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return cuda_fail(e, "device attributes for the batched kernel");
  auto fit_R = [&](const ArrayPlan& ap, int region) {
    int R = ap.R0;
    // the longest chunk (at most the preferred one) whose tables and buffers fit the region: in
    // steps of 32 records while at least 32 (whole 32-record blocks keep the skewed schedule
    // orders), then of 8
    while (R > 8 && warp_region_bytes(ap.a, R, nb) > region) R -= R > 32 ? 32 : 8;
    return warp_region_bytes(ap.a, R, nb) <= region ? R : 0;
  };
  // CTAs per SM that the kernel's registers allow at all
  int reg_ctas = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&reg_ctas, kern, kThreads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batched occupancy (registers)");
  const int max_k = std::max(1, std::min(kMaxBatchedCtas, reg_ctas));
  if (forced_ctas > max_k)
    return fail(ADHA_EINVAL, "ADHA_BATCHED_CTAS(%d): the kernel's registers allow at most %d CTAs per SM", forced_ctas, max_k);
  double best_score = -1;
  int best_k = 0, best_region = 0;
  for (int k = 1; k <= max_k; ++k) {
    if (forced_ctas && k != forced_ctas) continue;
    const int64_t dyn = std::min<int64_t>(optin, (int64_t)sm_smem / k - reserved - (int64_t)fa.sharedSizeBytes);
    const int region = (int)(dyn / kWarps / 16 * 16);
    double score = 0;
    bool ok = region > kHeaderBytes;
    for (const ArrayPlan& ap : plans) {
      if (ap.empty || !ok) continue;
      const int R = fit_R(ap, region);
      if (!R) {
        ok = false;
        continue;
      }
      const int want = std::min(ap.R0, 32);
      score += ap.moved * k * std::min(1.0, (double)R / want);
    }
    if (ok && score > best_score) {
      best_score = score;
      best_k = k;
      best_region = region;
    }
  }
  if (best_k == 0)
    return fail(ADHA_ENOTIMPL, "batched remap: an array's records are too wide for the shared memory of one warp");

  // the arrays' final plans, in ticket order (largest first), and the descriptor image
  std::vector<int> order;
  for (int k = 0; k < n_arrays; ++k)
    if (!plans[k].empty) order.push_back(k);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return plans[x].moved > plans[y].moved; });
  std::vector<BatchHeader> headers;
  std::vector<GroupRef> groups;
  std::vector<Move> moves;
  std::vector<uint32_t> sched;
  std::vector<int64_t> prefix;
  int64_t units = 0;
  double bytes = 0;
  bool direct = false;
  for (int k : order) {
    ArrayPlan& ap = plans[k];
    const int R = fit_R(ap, best_region);
    RemapArgs& a = ap.a;
    if (R != a.R) {
      bool empty = false;
      if (int rc = remap_plan_args(ap.S, ap.sp, ap.D, ap.dp, ap.n, R, ap.direct, &a, &empty)) return rc;
      if (a.R != R) return fail(ADHA_ENOTIMPL, "batched remap: array %d cannot use %d-record chunks", k, R);
    }
    BatchHeader h;
    std::memset(&h, 0, sizeof h);
    h.n = a.n;
    h.R = a.R;
    h.n_full = a.n_chunks;
    h.n_chunks = a.n_chunks + (a.n % a.R ? 1 : 0);
    h.n_src = a.n_src;
    h.n_dst = a.n_dst;
    h.in_bytes = a.in_bytes;
    h.out_bytes = a.out_bytes;
    h.n_moves = a.n_moves;
    for (int c = 0; c < kMoveClasses; ++c) h.cls_count[c] = a.cls_count[c];
    h.group0 = (int32_t)groups.size();
    h.move0 = (int32_t)moves.size();
    h.chunks_per_unit = std::max(1, kUnitRecords / a.R);
    h.sched_bytes = al16(a.R * a.n_moves * 4);
    h.sched_off = kHeaderBytes + (a.n_src + a.n_dst) * (int)sizeof(GroupRef);
    h.buf_off = h.sched_off + h.sched_bytes;
    h.sched0 = (int64_t)sched.size() * 4;
    h.unit0 = units;
    prefix.push_back(units);
    units += (h.n_chunks + h.chunks_per_unit - 1) / h.chunks_per_unit;
    for (int g = 0; g < a.n_src; ++g) groups.push_back(a.src[g]);
    for (int g = 0; g < a.n_dst; ++g) groups.push_back(a.dst[g]);
    moves.insert(moves.end(), a.move, a.move + a.n_moves);
    const size_t s0 = sched.size();
    sched.resize(s0 + h.sched_bytes / 4, 0u);
    for (int t = 0; t < a.R * a.n_moves; ++t)
      sched[s0 + t] = schedule_entry(t, a.R, a.cls_count, a.cls_order, a.move, a.src, a.dst, a.in_bytes);
    direct = direct || (a.cls_count[0] + a.cls_count[1] + a.cls_count[2] > 0);
    bytes += ap.moved;
    headers.push_back(h);
  }
  prefix.push_back(units);

  auto* b = new (std::nothrow) adha_batched();
  if (!b) return fail(ADHA_ENOMEM, "host allocation failed");
  b->n_arrays = (int32_t)headers.size();
  b->total_units = units;
  b->bytes = bytes;
  b->direct = direct;
  b->region = best_region;
  b->ctas_per_sm = best_k;
  b->buffers = nb;
  b->off_headers = al256(sizeof(unsigned long long));
  b->off_groups = b->off_headers + al256(std::max<size_t>(1, headers.size()) * sizeof(BatchHeader));
  b->off_moves = b->off_groups + al256(std::max<size_t>(1, groups.size()) * sizeof(GroupRef));
  b->off_sched = b->off_moves + al256(std::max<size_t>(1, moves.size()) * sizeof(Move));
  b->off_prefix = b->off_sched + al256(std::max<size_t>(1, sched.size()) * 4);
  b->image.assign(b->off_prefix + al256(prefix.size() * sizeof(int64_t)), 0);
  if (!headers.empty()) std::memcpy(b->image.data() + b->off_headers, headers.data(), headers.size() * sizeof(BatchHeader));
  if (!groups.empty()) std::memcpy(b->image.data() + b->off_groups, groups.data(), groups.size() * sizeof(GroupRef));
  if (!moves.empty()) std::memcpy(b->image.data() + b->off_moves, moves.data(), moves.size() * sizeof(Move));
  if (!sched.empty()) std::memcpy(b->image.data() + b->off_sched, sched.data(), sched.size() * 4);
  std::memcpy(b->image.data() + b->off_prefix, prefix.data(), prefix.size() * sizeof(int64_t));
  b->smem = (size_t)kWarps * best_region;
  int per_sm = 0;
  auto* k2 = b->direct ? batched_kernel<true> : batched_kernel<false>;
  e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2, kThreads, b->smem);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batched occupancy");
  }
  const int64_t want_ctas = (units + kWarps - 1) / kWarps;
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(1, per_sm), want_ctas));
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

int adha_batched_info(const adha_batched* b, int32_t* ctas_per_sm, int32_t* warp_region_bytes, int64_t* units) {
  clear_error();
  if (!b) return fail(ADHA_EINVAL, "NULL batched plan");
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (warp_region_bytes) *warp_region_bytes = b->region;
  if (units) *units = b->total_units;
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// One-call batched remap: plan, descriptors into the caller's workspace, launch.

namespace adha {

// The descriptor image is copied from pageable host memory that is freed when the call returns:
// safe for a plain enqueue (the copy is staged before cudaMemcpyAsync returns), not for a
// capture, which would record a copy node reading freed memory on every replay.
static int reject_capture(void* stream) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
  if (st != cudaStreamCaptureStatusNone)
    return fail(ADHA_EINVAL, "the stream is being captured: this call copies its descriptors from a host buffer "
                             "it frees on return (capture adha_batched_launch instead)");
  return 0;
}

}  // namespace adha

extern "C" {

int adha_workspace_bytes(int32_t n_arrays, const adha_remap_desc* descs, size_t* bytes) {
  clear_error();
  if (!bytes) return fail(ADHA_EINVAL, "bytes is NULL");
  adha_batched* b = nullptr;
  if (int rc = adha_batched_create(n_arrays, descs, 0, nullptr, &b)) return rc;
  *bytes = b->image.size();
  adha_batched_destroy(b);
  return 0;
}

int adha_remap_batched(int32_t n_arrays, const adha_remap_desc* descs, void* workspace, size_t ws_bytes,
                       adha_stream stream) {
  clear_error();
  if (!workspace) return fail(ADHA_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(ADHA_EINVAL, "workspace is not 256-byte aligned");
  if (int rc = reject_capture(stream)) return rc;
  adha_batched* b = nullptr;
  if (int rc = adha_batched_create(n_arrays, descs, 0, stream, &b)) return rc;
  if (ws_bytes < b->image.size()) {
    const size_t need = b->image.size();
    adha_batched_destroy(b);
    return fail(ADHA_ENOMEM, "workspace has %zu bytes, the batch needs %zu (adha_workspace_bytes)", ws_bytes, need);
  }
  cudaError_t e = cudaMemcpyAsync(workspace, b->image.data(), b->image.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    adha_batched_destroy(b);
    return cuda_fail(e, "copy of the batched descriptors into the workspace");
  }
  const std::pair<const adha_batched*, std::pair<void*, void*>> ctx{b, {workspace, stream}};
  const int rc = profiled_launch(3, 3, b->bytes, stream, batched_fn, &ctx);
  adha_batched_destroy(b);
  return rc;
}

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
// host-side name of a __device__ array is only a stand-in, not a device address).  The caller
// holds g_noalloc_mu.
static int noalloc_scratch(void** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(ADHA_ENOTIMPL, "device ordinal %d out of range", dev);
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
  if (int rc = reject_capture(stream)) return rc;
  adha_batched* b = nullptr;
  if (int rc = adha_batched_create(n_arrays, descs, 0, stream, &b)) return rc;
  const size_t need = b->image.size();
  if (need > (size_t)ADHA_NOALLOC_SCRATCH_BYTES) {
    adha_batched_destroy(b);
    return fail(ADHA_EINVAL, "this batch needs %zu bytes of descriptors; the allocation-free entry point holds at most %u",
                need, (unsigned)ADHA_NOALLOC_SCRATCH_BYTES);
  }
  int rc = 0;
  {
    // one thread's copy, ticket reset and kernel reach the stream before another thread's
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    void* scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (!rc) {
      // pageable source: the bytes are staged before the call returns, so the host image can go
      const cudaError_t e = cudaMemcpyAsync(scratch, b->image.data(), need, cudaMemcpyHostToDevice, (cudaStream_t)stream);
      if (e != cudaSuccess) rc = cuda_fail(e, "copy of the batched descriptors into the scratch array");
    }
    if (!rc) {
      const std::pair<const adha_batched*, std::pair<void*, void*>> ctx{b, {scratch, stream}};
      rc = profiled_launch(3, 2, b->bytes, stream, batched_fn, &ctx);
    }
  }
  adha_batched_destroy(b);
  return rc;
}

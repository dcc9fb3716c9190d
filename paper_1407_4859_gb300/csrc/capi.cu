// capi.cu -- validation, layout model, launch planning and the extern "C" entry points of
// libadha.so for the remap and section kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <set>

#include "internal.h"
#include "remap_common.cuh"

namespace adha {

// ------------------------------------------------------------------ errors
static thread_local std::string t_err;

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

int cuda_fail(int err, const char* what) {
  return fail(ADHA_ECUDA, "%s: %s", what, cudaGetErrorString((cudaError_t)err));
}

void clear_error() { t_err.clear(); }

// ------------------------------------------------------------------ device state
// Status word set by kernels whose bounded waits ran out (one per device, module memory).
static std::mutex g_mu;
static int g_sms[256];

static int current_device(int* dev) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (*dev < 0 || *dev >= 256) return fail(ADHA_ENOTIMPL, "device ordinal %d out of range", *dev);
  return 0;
}

int sm_count(int* count) {
  int dev;
  if (int rc = current_device(&dev)) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_sms[dev]) {
    cudaError_t e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
  }
  *count = g_sms[dev];
  return 0;
}

// ------------------------------------------------------------------ layouts
int group_struct(const int* dtype, const std::vector<int>& fields, std::vector<int>* offsets) {
  int pos = 0, align = 1;
  if (offsets) offsets->resize(fields.size());
  for (size_t k = 0; k < fields.size(); ++k) {
    const int sz = dtype_size(dtype[fields[k]]);
    pos = (pos + sz - 1) / sz * sz;
    if (offsets) (*offsets)[k] = pos;
    pos += sz;
    align = std::max(align, sz);
  }
  return (pos + align - 1) / align * align;
}

int check_schema(const adha_schema* schema) {
  if (!schema) return fail(ADHA_EINVAL, "schema is NULL");
  if (schema->n_fields < 1 || schema->n_fields > kMaxFields)
    return fail(ADHA_EINVAL, "schema has %d fields (1..%d allowed)", schema->n_fields, kMaxFields);
  if (!schema->dtype) return fail(ADHA_EINVAL, "schema dtype array is NULL");
  for (int f = 0; f < schema->n_fields; ++f)
    if (schema->dtype[f] < ADHA_F32 || schema->dtype[f] > ADHA_BF16)
      return fail(ADHA_EINVAL, "field %d has unknown dtype %d", f, schema->dtype[f]);
  return 0;
}

int make_layout(const adha_schema* schema, const adha_layout* layout, Layout* out, const char* what) {
  if (int rc = check_schema(schema)) return rc;
  const int F = schema->n_fields;
  if (!layout) return fail(ADHA_EINVAL, "%s layout is NULL", what);
  if (layout->n_groups < 1 || layout->n_groups > F)
    return fail(ADHA_EINVAL, "%s layout has %d groups for %d fields", what, layout->n_groups, F);
  if (!layout->group_len || !layout->fields) return fail(ADHA_EINVAL, "%s layout arrays are NULL", what);
  out->F = F;
  for (int f = 0; f < F; ++f) out->dtype[f] = schema->dtype[f];
  out->n_groups = layout->n_groups;
  out->groups.assign(layout->n_groups, {});
  bool seen[kMaxFields] = {};
  int p = 0;
  for (int g = 0; g < layout->n_groups; ++g) {
    const int len = layout->group_len[g];
    if (len < 1 || p + len > F) return fail(ADHA_EINVAL, "%s layout group %d has bad length %d", what, g, len);
    for (int k = 0; k < len; ++k) {
      const int f = layout->fields[p + k];
      if (f < 0 || f >= F) return fail(ADHA_EINVAL, "%s layout names field %d (schema has %d)", what, f, F);
      if (seen[f]) return fail(ADHA_EINVAL, "%s layout lists field %d twice", what, f);
      seen[f] = true;
      out->groups[g].push_back(f);
    }
    p += len;
  }
  if (p != F) return fail(ADHA_EINVAL, "%s layout covers %d of %d fields", what, p, F);
  for (int g = 0; g < out->n_groups; ++g) {
    std::vector<int> off;
    out->stride[g] = group_struct(out->dtype, out->groups[g], &off);
    if (out->stride[g] > kMaxStride)
      return fail(ADHA_EINVAL, "%s layout group %d is %d bytes (max %d)", what, g, out->stride[g], kMaxStride);
    for (size_t k = 0; k < off.size(); ++k) {
      out->group_of[out->groups[g][k]] = g;
      out->offset_of[out->groups[g][k]] = off[k];
    }
  }
  return 0;
}

bool same_group(const Layout& a, int ga, const Layout& b, int gb) { return a.groups[ga] == b.groups[gb]; }

static int check_ptrs(const void* const* ptrs, int count, const char* what) {
  if (!ptrs) return fail(ADHA_EINVAL, "%s pointer array is NULL", what);
  for (int g = 0; g < count; ++g) {
    if (!ptrs[g]) return fail(ADHA_EINVAL, "%s buffer %d is NULL", what, g);
    if (reinterpret_cast<uintptr_t>(ptrs[g]) % 16 != 0)
      return fail(ADHA_EINVAL, "%s buffer %d is not 16-byte aligned", what, g);
  }
  return 0;
}

static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return na && nb && x < y + nb && y < x + na;
}


void tanh_coefficients(float p[8], float q[8]) {
  // P_k = (2k+1) P_{k-1} + a P_{k-2}, Q_k likewise; P_{-1} = 1, P_0 = 1, Q_{-1} = 0, Q_0 = 1; k up to 12.
  int64_t pm[8] = {1}, pc[8] = {1}, qm[8] = {0}, qc[8] = {1};
  for (int k = 1; k <= 12; ++k) {
    int64_t pn[8], qn[8];
    for (int j = 0; j < 8; ++j) {
      pn[j] = (2 * k + 1) * pc[j] + (j ? pm[j - 1] : 0);
      qn[j] = (2 * k + 1) * qc[j] + (j ? qm[j - 1] : 0);
    }
    std::memcpy(pm, pc, sizeof pc);
    std::memcpy(pc, pn, sizeof pc);
    std::memcpy(qm, qc, sizeof qc);
    std::memcpy(qc, qn, sizeof qc);
  }
  for (int j = 0; j < 8; ++j) {
    p[j] = (float)pc[j];
    q[j] = (float)qc[j];
  }
}

// ------------------------------------------------------------------ launch profiler
// When on, every kernel the calling thread launches is bracketed by two CUDA events on its
// stream and tagged with its kind, op and algorithmic bytes (what the method must move).
// Process-wide, so launches from other host threads (an autograd engine's, for example) are seen.
struct ProfRec {
  int kind, op;
  double bytes;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool t_prof_on = false;
static std::vector<ProfRec> t_prof;
static std::vector<cudaEvent_t> t_pool;
static size_t t_pool_used = 0;

template <class Fn>
static int profiled(int kind, int op, double bytes, void* stream, Fn launch) {
  ProfRec r{kind, op, bytes, nullptr, nullptr};
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!t_prof_on || t_pool_used + 2 > t_pool.size()) r.a = nullptr;
    else {
      r.a = t_pool[t_pool_used];
      r.b = t_pool[t_pool_used + 1];
      t_pool_used += 2;
    }
  }
  if (!r.a) return launch();
  cudaError_t e = cudaEventRecord(r.a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(profile)");
  if (int rc = launch()) return rc;
  e = cudaEventRecord(r.b, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(profile)");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  t_prof.push_back(r);
  return 0;
}

// ------------------------------------------------------------------ remap planning
struct RemapPlan {
  RemapArgs args;
  size_t smem = 0;
  int grid = 1;
  bool empty = true;
};

// Chunk / pipeline override for the autotuner (0 = default rule).
static thread_local int t_tile_override = 0;
static thread_local int t_writeback_mode = 0;   // 0 automatic, 1 never, 2 every wide written group
static thread_local int t_section_buffers = 0;  // section chunk buffers per warp: 0 tuned or 2, else 1 or 2
static thread_local int t_fused_buffers = 0;    // fused runs: 0 tuned or default, else chunk buffers per warp
static thread_local int t_fused_jit = 0;        // fused runs: 0 as tuned, 1 library kernel, 2 specialised at run time
static thread_local int t_section_jit = 0;      // sections: 0 as tuned, 1 library kernel, 2 specialised where possible
static thread_local bool t_reduce_accumulate = false;   // REDUCE adds into its result (host pipeline slices)
static thread_local int t_remap_direct = 0;     // 1: remaps store one-field destination groups directly
static thread_local int t_remap_pieces = 0;     // 0: tuned or automatic, 1 + (piece-table bits | 4 for one buffer) otherwise

// Autotuned launch shapes: section key -> (records per chunk, writeback mode); remap key ->
// (records per chunk, 0 for the size rule; piece-table bits | 4 for one chunk buffer).
static std::mutex g_tune_mu;
static std::map<std::string, std::pair<int, int>> g_tune;

static std::string layout_code(const Layout& L) {
  std::string k;
  for (const auto& g : L.groups) {
    for (int f : g) k += std::to_string(f) + "." + std::to_string(L.dtype[f]) + ",";
    k += "|";
  }
  return k;
}

static std::string size_class(int64_t n) {
  int lg = 0;
  while (lg < 62 && (int64_t(1) << (lg + 1)) <= n) ++lg;
  return ":n" + std::to_string(lg);
}

static std::string section_key(const Layout& L, const adha_section* s, int64_t n, bool save) {
  std::string k = "S" + std::to_string(s->op) + ":" + std::to_string(s->read_mask) + ":" +
                  std::to_string(s->write_mask) + ":" + std::to_string(s->read_at_perm_mask) + ":" +
                  std::to_string(save ? 1 : 0) + ":";
  for (int a = 0; a < 8; ++a) k += std::to_string(s->arg[a]) + ",";
  return k + ":L" + layout_code(L) + size_class(n);
}

static std::string remap_key(const Layout& S, const Layout& D, int64_t n) {
  return "M" + layout_code(S) + ">" + layout_code(D) + size_class(n);
}

std::string tuning_key(const Layout& L, const adha_section* s, int64_t n, bool save) { return section_key(L, s, n, save); }
std::string remap_tuning_key(const Layout& S, const Layout& D, int64_t n) { return remap_key(S, D, n); }

void set_remap_pieces(int mode) { t_remap_pieces = mode; }

void tuning_store(const std::string& key, int R, int wb) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = {R, wb};
}

void set_overrides(int R, int wb, int buffers) {
  t_tile_override = R;
  t_writeback_mode = wb;
  t_section_buffers = buffers;
}

void set_fused_overrides(int R, int buffers) {
  t_tile_override = R;
  t_fused_buffers = buffers;
}

// Records per warp chunk: a multiple of 32 with about `target` bytes of the widest side.
static int pick_chunk(int rec_bytes, int target, int rmax) {
  int m = rec_bytes > 0 ? target / (32 * rec_bytes) : rmax / 32;
  m = std::max(1, std::min(m, rmax / 32));
  return 32 * m;
}

// Records per remap chunk: a power of two from 8 to 512 with about 4 KB of the widest side, so
// wide records use short chunks and keep more warps resident.
static int pick_remap_chunk(int rec_bytes) {
  int R = 8;
  while (R < 512 && 2 * R * rec_bytes <= 4096) R *= 2;
  return R;
}

static int finish_grid(int64_t n_chunks, int blocks, int* grid) {
  int sms = 0;
  if (int rc = sm_count(&sms)) return rc;
  if (blocks < 1) return fail(ADHA_ENOTIMPL, "kernel does not fit on an SM");
  const int64_t need = (n_chunks + 1 + kWarps - 1) / kWarps;   // +1: the tail's owner
  *grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * blocks, need));
  return 0;
}

// Shared-memory wavefronts of one warp step (32 schedule entries of one move class): the
// largest number of distinct 4-byte words that fall in one bank, for the given byte addresses.
static int step_wavefronts(const uint32_t* bytes, int cnt, int width) {
  uint32_t words[64];
  int m = 0;
  for (int l = 0; l < cnt; ++l) {
    if (bytes[l] == 0xFFFFFFFFu) continue;
    for (int w = 0; w < (width + 3) / 4; ++w) words[m++] = bytes[l] / 4 + w;
  }
  std::sort(words, words + m);
  m = (int)(std::unique(words, words + m) - words);
  int per_bank[32] = {};
  int worst = 1;
  for (int k = 0; k < m; ++k) worst = std::max(worst, ++per_bank[words[k] % 32]);
  return worst;
}

// Wavefronts of one chunk's moves of class c under schedule order `order` (as the kernel's
// schedule_entry lays them out): read side, plus write side for staged classes (direct classes
// store to global memory).
static long class_conflict_cost(const RemapArgs& a, int c, int order) {
  int first = 0;
  for (int k = 0; k < c; ++k) first += a.cls_count[k];
  const int cnt = a.cls_count[c], n = a.R * cnt, width = class_width(c);
  const bool direct = c < 3;
  long cost = 0;
  uint32_t rd[32], wr[32];
  for (int t = 0; t < n; t += 32) {
    const int w = std::min(32, n - t);
    for (int l = 0; l < w; ++l) {
      const int u = t + l;
      int r, k;
      schedule_pair(u, a.R, cnt, order, &r, &k);
      const Move& m = a.move[first + k];
      rd[l] = m.src_group < 0 ? 0xFFFFFFFFu
                              : (uint32_t)(a.src[m.src_group].start + r * a.src[m.src_group].stride + m.src_off);
      wr[l] = direct ? 0xFFFFFFFFu : (uint32_t)(a.dst[m.dst_group].start + r * a.dst[m.dst_group].stride + m.dst_off);
    }
    cost += step_wavefronts(rd, w, width) + (direct ? 0 : step_wavefronts(wr, w, width));
  }
  return cost;
}

// The schedule orders depend only on the moves, strides and chunk size: cached per shape.
static std::mutex g_order_mu;
static std::map<std::vector<int32_t>, std::vector<int32_t>> g_order_cache;

static void choose_orders(RemapArgs* a) {
  std::vector<int32_t> key = {a->R, a->n_src, a->n_dst, a->n_moves};
  for (int k = 0; k < a->n_src; ++k) key.push_back(a->src[k].stride);
  for (int k = 0; k < a->n_dst; ++k) key.push_back(a->dst[k].stride);
  for (int k = 0; k < a->n_moves; ++k) {
    const Move& m = a->move[k];
    key.insert(key.end(), {m.dst_group, m.dst_off, m.src_group, m.src_off});
  }
  for (int c = 0; c < kMoveClasses; ++c) key.push_back(a->cls_count[c]);
  {
    std::lock_guard<std::mutex> lk(g_order_mu);
    auto it = g_order_cache.find(key);
    if (it != g_order_cache.end()) {
      for (int c = 0; c < kMoveClasses; ++c) a->cls_order[c] = it->second[c];
      return;
    }
  }
  std::vector<int32_t> orders(kMoveClasses, 1);
  for (int c = 0; c < kMoveClasses; ++c) {
    if (!a->cls_count[c]) continue;
    long best = -1;
    for (int o = 0; o <= 6; ++o) {   // destination-major, record-major, skewed record-major (5 skews)
      // direct classes store to global memory: keep each run of lanes on one field at least
      // 32 bytes long (order 1, or a skew of at least 32/width lanes) so the stores stay coalesced
      if (c < 3 && (o == 0 || (o >= 2 && (1 << (o - 2)) * class_width(c) < 32))) continue;
      if (o >= 2 && a->R % 32) continue;   // skewed orders walk whole 32-record blocks
      const long cost = class_conflict_cost(*a, c, o);
      if (best < 0 || cost < best) {
        best = cost;
        orders[c] = o;
      }
    }
  }
  for (int c = 0; c < kMoveClasses; ++c) a->cls_order[c] = orders[c];
  std::lock_guard<std::mutex> lk(g_order_mu);
  g_order_cache[key] = orders;
}

// Occupancy per (kernel, shared bytes), queried once.
static std::mutex g_occ_mu;
static std::map<std::pair<int, size_t>, int> g_occ_cache;

static int cached_occupancy(int kind, size_t smem, int* blocks) {
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ_cache.find({kind, smem});
    if (it != g_occ_cache.end()) {
      *blocks = it->second;
      return 0;
    }
  }
  // kinds: < 100 remap (direct or not), 100 + op section, 200 + 10*M + vec + 2*km fused run
  const int rc = kind < 100    ? remap_occupancy(kind, smem, blocks)
                 : kind < 200 ? section_occupancy(kind - 100, smem, blocks)
                              : fused_occupancy((kind - 200) / 10, ((kind - 200) % 10) & 1, ((kind - 200) % 10) >> 1,
                                                smem, blocks);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ_cache[{kind, smem}] = *blocks;
  return 0;
}

static int plan_remap(const Layout& S, const void* const* src_ptrs, const Layout& D, void* const* dst_ptrs, int64_t n,
                      RemapPlan* plan) {
  std::memset(&plan->args, 0, sizeof plan->args);
  RemapArgs& a = plan->args;
  std::vector<int> build;
  for (int d = 0; d < D.n_groups; ++d) {
    bool alias = false;
    for (int j = 0; j < S.n_groups; ++j)
      if (same_group(D, d, S, j) && dst_ptrs[d] == src_ptrs[j]) alias = true;
    if (!alias) build.push_back(d);
  }
  plan->empty = build.empty() || n == 0;
  if (plan->empty) return 0;
  std::set<int> need_set;
  for (int d : build)
    for (int f : D.groups[d]) need_set.insert(S.group_of[f]);
  std::vector<int> need(need_set.begin(), need_set.end());
  for (size_t x = 0; x < build.size(); ++x) {
    const size_t nd = (size_t)n * D.stride[build[x]];
    for (int j : need)
      if (overlap(dst_ptrs[build[x]], nd, src_ptrs[j], (size_t)n * S.stride[j]))
        return fail(ADHA_EINVAL, "destination group %d overlaps source group %d", build[x], j);
    for (size_t y = x + 1; y < build.size(); ++y)
      if (overlap(dst_ptrs[build[x]], nd, dst_ptrs[build[y]], (size_t)n * D.stride[build[y]]))
        return fail(ADHA_EINVAL, "destination groups %d and %d overlap", build[x], build[y]);
  }
  // moves: every field of every built destination struct, and its padding in aligned pieces
  std::vector<Move> moves;
  std::vector<int> widths;
  for (size_t k = 0; k < build.size(); ++k) {
    const int d = build[k];
    std::vector<std::pair<int, int>> spans;   // (offset, size) of the fields
    for (int f : D.groups[d]) {
      const int k_src = (int)(std::lower_bound(need.begin(), need.end(), S.group_of[f]) - need.begin());
      moves.push_back(Move{(int16_t)k, (int16_t)D.offset_of[f], (int16_t)k_src, (int16_t)S.offset_of[f]});
      widths.push_back(dtype_size(D.dtype[f]));
      spans.push_back({D.offset_of[f], dtype_size(D.dtype[f])});
    }
    std::sort(spans.begin(), spans.end());
    spans.push_back({D.stride[d], 0});
    int pos = 0;
    for (const auto& sp : spans) {
      while (pos < sp.first) {   // zero padding, in the widest aligned pieces
        int w = 8;
        while (w > 2 && (pos % w != 0 || pos + w > sp.first)) w /= 2;
        moves.push_back(Move{(int16_t)k, (int16_t)pos, (int16_t)-1, (int16_t)0});
        widths.push_back(w);
        pos += w;
      }
      pos = sp.first + sp.second;
    }
  }
  if ((int)moves.size() > kMaxMoves) return fail(ADHA_EINVAL, "destination records too wide (%zu moves)", moves.size());
  // class of a move: direct (its destination group holds one field) or staged, then its width
  const bool allow_direct = t_remap_direct != 0;
  auto move_class = [&](size_t k) {
    const bool direct = allow_direct && D.groups[build[moves[k].dst_group]].size() == 1;
    return (direct ? 0 : 3) + (widths[k] == 8 ? 0 : widths[k] == 4 ? 1 : 2);
  };
  std::vector<size_t> idx(moves.size());
  for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
  std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
    if (move_class(x) != move_class(y)) return move_class(x) < move_class(y);
    if (moves[x].dst_group != moves[y].dst_group) return moves[x].dst_group < moves[y].dst_group;
    return moves[x].dst_off < moves[y].dst_off;
  });
  int src_rec = 0, dst_rec = 0;
  for (int j : need) src_rec += S.stride[j];
  for (int d : build) dst_rec += D.stride[d];
  int tuned_pieces = -1, tuned_R = 0;
  if (!t_remap_pieces || !t_tile_override) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(remap_key(S, D, n));
    if (it != g_tune.end()) {
      tuned_R = it->second.first;
      tuned_pieces = it->second.second;
    }
  }
  // records per chunk: forced, else tuned, else about 4 KB of the wider side (the loop below
  // shortens it while the buffers do not fit)
  int R = t_tile_override ? t_tile_override : tuned_R > 0 ? tuned_R : pick_remap_chunk(std::max(src_rec, dst_rec));
  if (t_remap_pieces) tuned_pieces = -1;
  for (;;) {
    a.n = n;
    a.R = R;
    a.n_chunks = n / R;
    a.n_src = (int)need.size();
    a.n_dst = (int)build.size();
    int off = 0;
    for (int k = 0; k < a.n_src; ++k) {
      a.src[k].ptr = static_cast<const uint8_t*>(src_ptrs[need[k]]);
      a.src[k].stride = S.stride[need[k]];
      a.src[k].start = off;
      off += R * a.src[k].stride;
    }
    a.in_bytes = off;
    off = 0;
    for (int k = 0; k < a.n_dst; ++k) {
      a.dst[k].ptr = static_cast<const uint8_t*>(dst_ptrs[build[k]]);
      a.dst[k].stride = D.stride[build[k]];
      if (allow_direct && D.groups[build[k]].size() == 1) {
        a.dst[k].start = -1;          // direct: stored straight to global memory
      } else {
        a.dst[k].start = off;
        off += R * a.dst[k].stride;
      }
    }
    a.out_bytes = off;
    // piece tables: as forced or tuned for this pair of layouts, else for a buffer whose slices
    // average under 256 bytes (two or more groups in each 512-byte warp step)
    int staged_dst = 0;
    for (int k = 0; k < a.n_dst; ++k) staged_dst += a.dst[k].start >= 0;
    const bool narrow_in = a.in_bytes < 256 * a.n_src, narrow_out = staged_dst > 0 && a.out_bytes < 256 * staged_dst;
    a.pieces = (narrow_in ? 1 : 0) | (narrow_out ? 2 : 0);
    a.buffers = 2;
    const int mode = t_remap_pieces ? t_remap_pieces - 1 : tuned_pieces;
    if (mode >= 0) {
      a.pieces = mode & 3;
      a.buffers = (mode & 4) ? 1 : 2;
    }
    a.n_moves = (int)moves.size();
    for (int c = 0; c < kMoveClasses; ++c) a.cls_count[c] = 0;
    for (size_t k = 0; k < idx.size(); ++k) {
      a.move[k] = moves[idx[k]];
      a.cls_count[move_class(idx[k])]++;
    }
    plan->smem = remap_smem_bytes(a);
    if (plan->smem <= (size_t)kSmemLimit && a.in_bytes < 0xFFFF && a.out_bytes <= 0xFFFF && R <= 1024) break;
    if (R <= 8) return fail(ADHA_EINVAL, "records too wide for an 8-record chunk (%zu bytes smem)", plan->smem);
    R = std::max(8, R / 2 / 8 * 8);
  }
  choose_orders(&a);
  int blocks = 0;
  if (int rc = cached_occupancy(allow_direct ? 1 : 0, plan->smem, &blocks)) return rc;
  return finish_grid(a.n_chunks, blocks, &plan->grid);
}

// ------------------------------------------------------------------ section planning
static bool has(uint64_t m, int f) { return (m >> f) & 1ull; }

// A section's operation and operands in the kernels' form: read and written fields grouped by
// dtype, ascending ids within a dtype.
void fill_secop(const Layout& L, const adha_section* s, SecOp* o) {
  std::memset(o, 0, sizeof *o);
  o->op = s->op;
  for (int k = 0; k < 8; ++k) o->arg[k] = s->arg[k];
  for (int k = 0; k < 4; ++k) o->par[k] = s->fparam[k];
  int nr = 0, nw = 0;
  for (int d = 0; d < 4; ++d) {
    o->rd_off[d] = (int8_t)nr;
    o->wr_off[d] = (int8_t)nw;
    for (int f = 0; f < L.F; ++f) {
      if (L.dtype[f] != d) continue;
      if (has(s->read_mask, f)) o->rd[nr++] = (int8_t)f;
      if (has(s->write_mask, f)) o->wr[nw++] = (int8_t)f;
    }
  }
  o->rd_off[4] = (int8_t)nr;
  o->wr_off[4] = (int8_t)nw;
  for (int k = 0; k < kMaxFields; ++k) o->rd_s0[k] = o->wr_s0[k] = -1;
  o->aux = s->aux;
  // a gather whose fields read through perm fill one 16-byte struct reads them with one load
  o->gvec = 0;
  if (s->op == ADHA_OP_GATHER) {
    const int g = L.group_of[s->arg[3]];
    bool one = L.stride[g] == 16;
    for (int k = 3; k < 7 && one; ++k) one = L.group_of[s->arg[k]] == g;
    if (one) {
      o->gvec = 1;
      for (int k = 0; k < 4; ++k) o->gidx[k] = (int8_t)(L.offset_of[s->arg[3 + k]] / 4);
    }
  }
}

void fill_secop_offsets(SecOp* o, const FieldRef* f) {
  for (int j = 0; j < o->rd_off[4]; ++j) o->rd_s0[j] = (int16_t)f[o->rd[j]].s0;
  for (int j = 0; j < o->wr_off[4]; ++j) o->wr_s0[j] = (int16_t)f[o->wr[j]].s0;
}

// A REDUCE sums cluster by cluster ("walk") when none of its features is a one-field slice: the
// lanes then read one record's features from one struct, consecutive words.
static bool reduce_walks(const Layout& L, const adha_section* s) {
  if (s->op != ADHA_OP_REDUCE) return false;
  for (int f = 0; f < L.F; ++f)
    if (f != s->arg[0] && has(s->read_mask, f) && L.groups[L.group_of[f]].size() == 1) return false;
  return true;
}

static int check_section(const Layout& L, const adha_section* s, int64_t n, bool has_save) {
  if (!s) return fail(ADHA_EINVAL, "section is NULL");
  const int F = L.F;
  const uint64_t all = F == 64 ? ~0ull : ((1ull << F) - 1);
  if ((s->read_mask | s->write_mask | s->read_at_perm_mask) & ~all)
    return fail(ADHA_EINVAL, "section masks name fields beyond %d", F);
  struct Need {
    int n;
    int dt[8];
    char role[8];   // 'r' read, 'w' written, 'b' both, 'p' read at perm
  };
  if (s->op == ADHA_OP_ASSIGN || s->op == ADHA_OP_REDUCE) {
    const bool assign = s->op == ADHA_OP_ASSIGN;
    const int m = s->arg[0], K = s->arg[1];
    if (m < 0 || m >= F || L.dtype[m] != ADHA_I32)
      return fail(ADHA_EINVAL, "op %d: membership field %d must be an int32 field", s->op, m);
    if (K < 1 || K > kMaxClusters) return fail(ADHA_EINVAL, "op %d: K = %d not in [1, %d]", s->op, K, kMaxClusters);
    const uint64_t feats = s->read_mask & ~(1ull << m);
    for (int f = 0; f < F; ++f)
      if (has(feats, f) && L.dtype[f] != ADHA_F32) return fail(ADHA_EINVAL, "op %d: feature field %d is not fp32", s->op, f);
    const int d = __builtin_popcountll(feats);
    if (d < 1 || (!assign && d > kMaxReduceFeatures))
      return fail(ADHA_EINVAL, "op %d: %d feature fields (1..%d)", s->op, d, assign ? F : kMaxReduceFeatures);
    if (assign && (s->write_mask != (1ull << m) || has(s->read_mask, m)))
      return fail(ADHA_EINVAL, "assign section: write_mask must be the membership field alone, which it does not read");
    if (!assign && (s->write_mask || !has(s->read_mask, m)))
      return fail(ADHA_EINVAL, "reduce section: reads the membership field and writes no field");
    if (s->read_at_perm_mask) return fail(ADHA_EINVAL, "only gather sections read through perm");
    if (n > 0 && (!s->aux || reinterpret_cast<uintptr_t>(s->aux) % (assign ? 4 : 8)))
      return fail(ADHA_EINVAL, "op %d: aux is NULL or misaligned", s->op);
    if (has_save) return fail(ADHA_EINVAL, "save is only defined for axpb, mul and tanh sections");
    return 0;
  }
  Need need{};
  switch (s->op) {
    case ADHA_OP_MADD3: need = {3, {ADHA_F32, ADHA_F32, ADHA_F32}, {'r', 'r', 'b'}}; break;
    case ADHA_OP_XORSHIFT: need = {2, {ADHA_I32, ADHA_I32}, {'r', 'w'}}; break;
    case ADHA_OP_ADD: need = {3, {ADHA_F32, ADHA_F32, ADHA_F32}, {'r', 'r', 'w'}}; break;
    case ADHA_OP_MIX: need = {0, {}, {}}; break;
    case ADHA_OP_DRIFT: need = {6, {0, 0, 0, 0, 0, 0}, {'b', 'b', 'b', 'r', 'r', 'r'}}; break;
    case ADHA_OP_BIN: need = {4, {0, 0, 0, ADHA_I32}, {'r', 'r', 'r', 'w'}}; break;
    case ADHA_OP_KE: need = {5, {0, 0, 0, 0, ADHA_F64}, {'r', 'r', 'r', 'r', 'w'}}; break;
    case ADHA_OP_FLAGS: need = {2, {ADHA_I32, ADHA_F64}, {'b', 'r'}}; break;
    case ADHA_OP_GATHER: need = {7, {0, 0, 0, 0, 0, 0, 0}, {'b', 'b', 'b', 'p', 'p', 'p', 'p'}}; break;
    case ADHA_OP_KICK: need = {4, {0, 0, 0, 0}, {'b', 'b', 'b', 'r'}}; break;
    case ADHA_OP_AXPB: need = {2, {0, 0}, {'r', 'w'}}; break;
    case ADHA_OP_MUL: need = {3, {0, 0, 0}, {'r', 'r', 'w'}}; break;
    case ADHA_OP_TANH: need = {2, {0, 0}, {'r', 'w'}}; break;
    default: return fail(ADHA_EINVAL, "unknown section op %d", s->op);
  }
  for (int k = 0; k < need.n; ++k) {
    const int f = s->arg[k];
    if (f < 0 || f >= F) return fail(ADHA_EINVAL, "op %d operand %d is field %d (schema has %d)", s->op, k, f, F);
    if (L.dtype[f] != need.dt[k])
      return fail(ADHA_EINVAL, "op %d operand %d (field %d) has dtype %d, needs %d", s->op, k, f, L.dtype[f], need.dt[k]);
    const char r = need.role[k];
    if ((r == 'r' || r == 'b') && !has(s->read_mask, f))
      return fail(ADHA_EINVAL, "op %d reads field %d but read_mask lacks it", s->op, f);
    if ((r == 'w' || r == 'b') && !has(s->write_mask, f))
      return fail(ADHA_EINVAL, "op %d writes field %d but write_mask lacks it", s->op, f);
    if (r == 'p' && !has(s->read_at_perm_mask, f))
      return fail(ADHA_EINVAL, "op %d reads field %d at perm[i] but read_at_perm_mask lacks it", s->op, f);
  }
  if (s->op == ADHA_OP_MIX && (s->write_mask & ~s->read_mask))
    return fail(ADHA_EINVAL, "mix section writes fields it does not read");
  if (s->op == ADHA_OP_GATHER) {
    if (s->read_at_perm_mask & s->write_mask)
      return fail(ADHA_EINVAL, "gather section writes a field it reads through perm");
    if (n > 0 && !s->perm) return fail(ADHA_EINVAL, "gather section has no perm");
  } else if (s->read_at_perm_mask) {
    return fail(ADHA_EINVAL, "only gather sections read through perm");
  }
  if (has_save && s->op != ADHA_OP_AXPB && s->op != ADHA_OP_MUL && s->op != ADHA_OP_TANH)
    return fail(ADHA_EINVAL, "save is only defined for axpb, mul and tanh sections");
  return 0;
}

int check_section_layout(const Layout& L, const adha_section* s, int64_t n) { return check_section(L, s, n, false); }

struct SectionPlan {
  SectionArgs args;
  size_t smem = 0;
  int grid = 1;
};

static int plan_section(const Layout& L, void* const* ptrs, const adha_section* s, int64_t n, void* save,
                        SectionPlan* plan) {
  SectionArgs& a = plan->args;
  std::memset(&a, 0, sizeof a);
  int tuned_R = t_tile_override, wb_mode = t_writeback_mode, buffers = t_section_buffers;
  if (!tuned_R && !wb_mode && !buffers) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(section_key(L, s, n, save != nullptr));
    if (it != g_tune.end() && !(it->second.second & 8)) {   // mode: store mode, + 4 for one chunk buffer per warp
      tuned_R = it->second.first;
      wb_mode = it->second.second & 3;
      buffers = (it->second.second & 4) ? 1 : 2;
    }
  }
  if (buffers != 1) buffers = 2;
  uint64_t staged = s->read_mask;
  if (s->op == ADHA_OP_MIX) staged |= s->write_mask;
  if (save) staged |= 1ull << (s->op == ADHA_OP_MUL ? s->arg[2] : s->arg[1]);
  // Every group the section reads is staged through shared memory: the double-buffered copies
  // keep a chunk in flight per warp while the previous one is computed.
  std::vector<int> groups;
  for (int g = 0; g < L.n_groups; ++g) {
    bool any = false;
    for (int f : L.groups[g]) any = any || has(staged, f);
    if (any) groups.push_back(g);
  }
  int rec = 0;
  for (int g : groups) rec += L.stride[g];
  if (s->op == ADHA_OP_GATHER) rec += 4;
  int R = tuned_R ? std::max(32, std::min(tuned_R, 128)) : (rec > 0 ? pick_chunk(rec, 4096, 128) : 128);
  if (R != 32 && R != 64 && R != 128) R = R < 64 ? 32 : 64;   // 96 -> 64: the kernels exist for 32, 64, 128
  fill_secop(L, s, &a.s);   // before the shared-memory size, which depends on the op
  for (;;) {
    a.n = n;
    a.R = R;
    a.n_chunks = n / R;
    a.F = L.F;
    a.n_load = (int)groups.size();
    a.perm_slot = -1;
    for (int f = 0; f < L.F; ++f) {
      const int g = L.group_of[f];
      a.f[f].g = static_cast<uint8_t*>(ptrs[g]) + L.offset_of[f];
      a.f[f].gs = L.stride[g];
      a.f[f].s0 = -1;
      a.f[f].ss = 0;
      a.f[f].wsm = 0;
      a.f[f].dtype = L.dtype[f];
    }
    int off = 0;
    a.n_writeback = 0;
    for (int k = 0; k < a.n_load; ++k) {
      const int g = groups[k];
      a.load[k].ptr = static_cast<const uint8_t*>(ptrs[g]);
      a.load[k].stride = L.stride[g];
      a.load[k].start = off;
      // A wide group with written fields is updated in the chunk buffer and written back whole:
      // one coalesced store stream instead of scattered partial-record stores.
      int written = 0;
      for (int f : L.groups[g]) written += has(s->write_mask, f) ? dtype_size(L.dtype[f]) : 0;
      const bool wide = L.stride[g] > 8 && written > 0;
      a.writeback[k] = (int8_t)(wb_mode == 1 ? 0 : wb_mode == 2 ? wide : (wide && 4 * written >= L.stride[g]));
      a.n_writeback += a.writeback[k];
      for (int f : L.groups[g]) {
        a.f[f].s0 = off + L.offset_of[f];
        a.f[f].ss = L.stride[g];
        a.f[f].wsm = a.writeback[k];
      }
      off += R * L.stride[g];
    }
    if (s->op == ADHA_OP_GATHER) {
      a.perm_slot = a.n_load;
      a.writeback[a.n_load] = 0;
      a.load[a.n_load].ptr = reinterpret_cast<const uint8_t*>(s->perm);
      a.load[a.n_load].stride = 4;
      a.load[a.n_load].start = off;
      off += R * 4;
    }
    a.in_bytes = off;
    a.buffers = buffers;
    a.accumulate = t_reduce_accumulate ? 1 : 0;
    a.reduce_walk = reduce_walks(L, s) ? 1 : 0;
    // vector mapping: every staged group and every written field's group is one field wide
    // (and `save`, if any, aligned for the chunk's vector stores)
    const bool vec_op = s->op == ADHA_OP_MIX || s->op == ADHA_OP_AXPB || s->op == ADHA_OP_MUL || s->op == ADHA_OP_TANH;
    a.vec = (vec_op && R >= 64 && a.n_writeback == 0 && reinterpret_cast<uintptr_t>(save) % (R / 8) == 0) ? 1 : 0;
    for (int f = 0; f < L.F && a.vec; ++f)
      if ((has(staged, f) || has(s->write_mask, f)) && L.groups[L.group_of[f]].size() != 1) a.vec = 0;
    plan->smem = section_smem_bytes(a);
    if (plan->smem <= (size_t)kSmemLimit) break;
    if (R <= 32) return fail(ADHA_EINVAL, "section records too wide for a 32-record chunk");
    R /= 2;
  }
  fill_secop_offsets(&a.s, a.f);
  tanh_coefficients(a.tanh_p, a.tanh_q);
  a.perm = s->perm;
  a.save = static_cast<uint8_t*>(save);
  int blocks = 0;
  if (int rc = cached_occupancy(100 + s->op, plan->smem, &blocks)) return rc;
  return finish_grid(a.n_chunks, blocks, &plan->grid);
}

int remap_plan_args(const Layout& S, const void* const* src_ptrs, const Layout& D, void* const* dst_ptrs, int64_t n,
                    int chunk_override, int direct, RemapArgs* out, bool* empty) {
  const int saved = t_tile_override, saved_direct = t_remap_direct;
  t_tile_override = chunk_override;
  t_remap_direct = direct;
  RemapPlan plan;
  const int rc = plan_remap(S, src_ptrs, D, dst_ptrs, n, &plan);
  t_tile_override = saved;
  t_remap_direct = saved_direct;
  if (rc) return rc;
  *out = plan.args;
  *empty = plan.empty;
  return 0;
}

static double remap_bytes(const RemapArgs& a, const Layout& D, const std::vector<int>& built) {
  double b = 0;
  for (int d : built)
    for (int f : D.groups[d]) b += dtype_size(D.dtype[f]);
  return 2.0 * (double)a.n * b;
}

static double section_bytes(const Layout& L, const adha_section* s, int64_t n, bool save) {
  double b = 0;
  const uint64_t rw = s->read_mask | s->write_mask;
  for (int f = 0; f < L.F; ++f) {
    const int sz = dtype_size(L.dtype[f]);
    if (has(rw, f)) b += sz;
    if (has(s->write_mask, f)) b += sz;
    if (has(s->read_at_perm_mask, f)) b += sz;
  }
  if (s->op == ADHA_OP_GATHER) b += 4;
  if (save) b += 4;
  return b * (double)n;
}

static int do_remap(const Layout& S, const void* const* src_ptrs, const Layout& D, void* const* dst_ptrs, int64_t n,
                    void* stream, int* launched) {
  RemapPlan plan;
  if (int rc = plan_remap(S, src_ptrs, D, dst_ptrs, n, &plan)) return rc;
  if (launched) *launched = plan.empty ? 0 : 1;
  if (plan.empty) return 0;
  std::vector<int> built;
  for (int d = 0; d < D.n_groups; ++d) {
    bool alias = false;
    for (int j = 0; j < S.n_groups; ++j) alias = alias || (same_group(D, d, S, j) && dst_ptrs[d] == src_ptrs[j]);
    if (!alias) built.push_back(d);
  }
  return profiled(0, 0, remap_bytes(plan.args, D, built), stream,
                  [&] { return launch_remap(plan.args, plan.grid, plan.smem, stream); });
}

int remap_layouts(const Layout& S, const void* const* src_ptrs, const Layout& D, void* const* dst_ptrs, int64_t n,
                  void* stream, int* launched) {
  return do_remap(S, src_ptrs, D, dst_ptrs, n, stream, launched);
}

int profiled_launch(int kind, int op, double bytes, void* stream, int (*fn)(const void*), const void* ctx) {
  return profiled(kind, op, bytes, stream, [&] { return fn(ctx); });
}

// ------------------------------------------------------------------ fused runs (combine)
// A run of m consecutive sections in one pass: each section valid on its own, none with `save`,
// every gather reading through the same permutation, and no field that a gather reads through
// the permutation written by any section of the run (a record's sections then see exactly what
// they would see run one after another).
static int check_fused(const Layout& L, const adha_section* s, int m, int64_t n) {
  if (!s) return fail(ADHA_EINVAL, "sections are NULL");
  if (m < 1 || m > kMaxFused) return fail(ADHA_EINVAL, "a fused run holds 1..%d sections (got %d)", kMaxFused, m);
  uint64_t written = 0, at_perm = 0;
  const int32_t* perm = nullptr;
  for (int k = 0; k < m; ++k) {
    if (int rc = check_section(L, &s[k], n, false)) return rc;
    written |= s[k].write_mask;
    at_perm |= s[k].read_at_perm_mask;
    if (s[k].op == ADHA_OP_GATHER) {
      if (perm && s[k].perm != perm) return fail(ADHA_EINVAL, "the gathers of a fused run use different permutations");
      perm = s[k].perm;
    }
  }
  if (written & at_perm)
    return fail(ADHA_EINVAL, "a section of the run writes a field that a gather of the run reads through perm");
  int reduces = 0;
  for (int k = 0; k < m; ++k) reduces += s[k].op == ADHA_OP_REDUCE ? 1 : 0;
  if (reduces > 1) return fail(ADHA_EINVAL, "a fused run holds at most one reduce section (got %d)", reduces);
  if (n > 0 && perm && reinterpret_cast<uintptr_t>(perm) % 16) return fail(ADHA_EINVAL, "perm is not 16-byte aligned");
  if (n > 0 && !perm && at_perm) return fail(ADHA_EINVAL, "gather without a permutation");
  return 0;
}

// Whether sections s[0..m) may run fused (check_fused without leaving an error message behind).
bool fusable_run(const Layout& L, const adha_section* s, int m) {
  const std::string saved = t_err;
  const int rc = check_fused(L, s, m, 1);
  t_err = saved;
  return rc == 0;
}

static std::string fused_key(const Layout& L, const adha_section* s, int m, int64_t n) {
  std::string k = "F";
  for (int j = 0; j < m; ++j) {
    k += std::to_string(s[j].op) + ":" + std::to_string(s[j].read_mask) + ":" + std::to_string(s[j].write_mask) + ":" +
         std::to_string(s[j].read_at_perm_mask) + ":";
    for (int a = 0; a < 8; ++a) k += std::to_string(s[j].arg[a]) + ",";
    k += ";";
  }
  return k + ":L" + layout_code(L) + size_class(n);
}

std::string fused_tuning_key(const Layout& L, const adha_section* s, int m, int64_t n) { return fused_key(L, s, m, n); }

// Algorithmic bytes of a fused run: every field some section reads or writes, read once; every
// written field written once; plus the permutation and the fields read through it.
static double fused_bytes(const Layout& L, const adha_section* s, int m, int64_t n) {
  uint64_t rw = 0, w = 0, p = 0;
  bool gather = false;
  for (int k = 0; k < m; ++k) {
    rw |= s[k].read_mask | s[k].write_mask;
    w |= s[k].write_mask;
    p |= s[k].read_at_perm_mask;
    gather = gather || s[k].op == ADHA_OP_GATHER;
  }
  double b = gather ? 4 : 0;
  for (int f = 0; f < L.F; ++f) {
    const int sz = dtype_size(L.dtype[f]);
    b += (has(rw, f) ? sz : 0) + (has(w, f) ? sz : 0) + (has(p, f) ? sz : 0);
  }
  return b * (double)n;
}

// A fused run computes long per chunk, so by default one chunk buffer per warp (more CTAs per SM,
// the next chunk's copy issued after the write-back) beats double buffering.
constexpr int kFusedBuffers = 1;

struct FusedPlan {
  FusedArgs args;
  int grid = 0;
  size_t smem = 0;
  const void* jit = nullptr;   // the run's specialised kernel, or NULL for the library's fused kernel
};

// launchable = false: the arguments only (no kernel looked up, no device queried).
static int plan_fused(const Layout& L, void* const* ptrs, const adha_section* s, int m, int64_t n, void* stream,
                      FusedPlan* plan, bool launchable = true) {
  FusedArgs& a = plan->args;
  std::memset(&a, 0, sizeof a);
  int tuned_R = t_tile_override, tuned_buffers = t_fused_buffers;
  bool tuned_jit = false;
  if (!tuned_R && !tuned_buffers) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(fused_key(L, s, m, n));
    if (it != g_tune.end()) {   // buffers, + 4 for the run specialised at run time
      tuned_R = it->second.first;
      tuned_buffers = it->second.second & 3;
      tuned_jit = (it->second.second & 4) != 0;
    }
  }
  const bool want_jit = t_fused_jit == 2 || (t_fused_jit == 0 && tuned_jit);
  uint64_t staged = 0, written = 0;
  const int32_t* perm = nullptr;
  int reduce_sec = -1, assign_sec = -1;
  for (int k = 0; k < m; ++k) {
    staged |= s[k].read_mask | s[k].write_mask;
    written |= s[k].write_mask;
    if (s[k].op == ADHA_OP_GATHER) perm = s[k].perm;
    if (s[k].op == ADHA_OP_REDUCE) reduce_sec = k;
    if (s[k].op == ADHA_OP_ASSIGN && assign_sec < 0) assign_sec = k;
  }
  std::vector<int> groups;
  for (int g = 0; g < L.n_groups; ++g) {
    bool any = false;
    for (int f : L.groups[g]) any = any || has(staged, f);
    if (any) groups.push_back(g);
  }
  int rec = perm ? 4 : 0;
  bool one_field = true;
  for (int g : groups) {
    rec += L.stride[g];
    one_field = one_field && L.groups[g].size() == 1;
  }
  // default chunk: with one-field groups the longest of 128 / 64 records whose buffers leave room
  // for two CTAs per SM (the vector mapping needs 64 or more), else about 4 KB of records
  int R = 32;
  if (tuned_R) R = std::max(32, std::min(tuned_R, 128));
  else if (one_field && (size_t)kWarps * 2 * 128 * rec <= (size_t)kSmemLimit / 2 - 8192) R = 128;
  else if (one_field && (size_t)kWarps * 2 * 64 * rec <= (size_t)kSmemLimit / 2 - 8192) R = 64;
  else R = rec > 0 ? pick_chunk(rec, 4096, 128) : 128;
  if (R != 32 && R != 64 && R != 128) R = R < 64 ? 32 : 64;
  if ((reduce_sec >= 0 || assign_sec >= 0) && R > 64) R = 64;   // the assign / reduce kernels stop at 64
  for (;;) {
    a.n = n;
    a.R = R;
    a.n_chunks = n / R;
    a.n_load = (int)groups.size();
    a.perm_slot = -1;
    for (int f = 0; f < L.F; ++f) {
      const int g = L.group_of[f];
      a.f[f].g = static_cast<uint8_t*>(ptrs[g]) + L.offset_of[f];
      a.f[f].gs = L.stride[g];
      a.f[f].s0 = -1;
      a.f[f].dtype = L.dtype[f];
    }
    int off = 0;
    bool vec = true;
    for (int k = 0; k < a.n_load; ++k) {
      const int g = groups[k];
      a.load[k].ptr = static_cast<const uint8_t*>(ptrs[g]);
      a.load[k].stride = L.stride[g];
      a.load[k].start = off;
      bool w = false;
      for (int f : L.groups[g]) w = w || has(written, f);
      a.writeback[k] = w ? 1 : 0;
      for (int f : L.groups[g]) {
        a.f[f].s0 = off + L.offset_of[f];
        a.f[f].ss = L.stride[g];
        a.f[f].wsm = 1;   // every write goes to the chunk buffer; written groups go back whole
      }
      vec = vec && L.groups[g].size() == 1;
      off += R * L.stride[g];
    }
    if (perm) {
      a.perm_slot = a.n_load;
      a.writeback[a.n_load] = 0;
      a.load[a.n_load].ptr = reinterpret_cast<const uint8_t*>(perm);
      a.load[a.n_load].stride = 4;
      a.load[a.n_load].start = off;
      off += R * 4;
    }
    a.in_bytes = off;
    a.vec = vec ? 1 : 0;
    a.buffers = tuned_buffers == 1 || tuned_buffers == 2 ? tuned_buffers : kFusedBuffers;
    a.n_sec = m;
    a.reduce_sec = reduce_sec;
    a.assign_sec = assign_sec;
    a.accumulate = t_reduce_accumulate ? 1 : 0;
    a.reduce_walk = reduce_sec >= 0 && reduce_walks(L, &s[reduce_sec]) ? 1 : 0;
    plan->smem = fused_smem_bytes(a);
    if (plan->smem <= (size_t)kSmemLimit) break;
    if (R <= 32) return fail(ADHA_EINVAL, "the fused run's records are too wide for a 32-record chunk");
    R /= 2;
  }
  a.n_sec = m;
  for (int k = 0; k < m; ++k) {
    fill_secop(L, &s[k], &a.sec[k]);
    fill_secop_offsets(&a.sec[k], a.f);
  }
  tanh_coefficients(a.tanh_p, a.tanh_q);
  a.perm = perm;
  if (!launchable) return 0;
  int blocks = 0;
  if (want_jit) {
    // compiled here unless the stream is being captured (loading a module is no stream work)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    std::string why;
    const void* fn = nullptr;
    const int rc = jit_kernel(a, L.F, a.buffers, cs == cudaStreamCaptureStatusNone, &fn, &why);
    if (rc == 0) {
      plan->jit = fn;
      plan->smem = jit_smem_bytes(a);
      if (int e = jit_occupancy(fn, plan->smem, &blocks)) return e;
      return finish_grid(a.n_chunks, blocks, &plan->grid);
    }
    if (t_fused_jit == 2) return rc;   // asked for explicitly: report why not
    clear_error();                     // else the library's fused kernel
  }
  const int M = R / 32;
  if (int rc = cached_occupancy(200 + 10 * M + a.vec + 2 * (fused_is_km(a) ? 1 : 0), plan->smem, &blocks)) return rc;
  return finish_grid(a.n_chunks, blocks, &plan->grid);
}

int run_fused_layout(const Layout& L, void* const* ptrs, const adha_section* s, int m, int64_t n, void* stream) {
  if (int rc = check_fused(L, s, m, n)) return rc;
  if (n == 0) return 0;
  FusedPlan plan;
  if (int rc = plan_fused(L, ptrs, s, m, n, stream, &plan)) return rc;
  return profiled(4, m, fused_bytes(L, s, m, n), stream, [&] {
    return plan.jit ? launch_fused_jit(plan.jit, plan.args, plan.grid, plan.smem, stream)
                    : launch_fused(plan.args, plan.grid, plan.smem, stream);
  });
}

// The launch arguments of a fused run with chunk shape (chunk, buffers), planned on stand-in group
// addresses (planning reads no memory; the specialised source holds no address).
int fused_jit_args(const Layout& L, const adha_section* s, int m, int64_t n, int chunk, int buffers, FusedArgs* out) {
  if (int rc = check_fused(L, s, m, n)) return rc;
  if (n == 0) return fail(ADHA_EINVAL, "n = 0: nothing to specialise");
  std::vector<void*> fake(L.n_groups, reinterpret_cast<void*>((uintptr_t)1 << 40));
  const int saved_R = t_tile_override, saved_B = t_fused_buffers, saved_J = t_fused_jit;
  t_tile_override = chunk;
  t_fused_buffers = buffers;
  t_fused_jit = 1;
  FusedPlan plan;
  const int rc = plan_fused(L, fake.data(), s, m, n, nullptr, &plan, false);
  t_tile_override = saved_R;
  t_fused_buffers = saved_B;
  t_fused_jit = saved_J;
  if (rc == 0) *out = plan.args;
  return rc;
}

void set_fused_jit(int mode) { t_fused_jit = mode; }
void set_reduce_accumulate(bool on) { t_reduce_accumulate = on; }

// The fused run's specialised source, compiled (and loaded into the process's cache when `load`).
int fused_jit_build(const Layout& L, const adha_section* s, int m, int64_t n, int chunk, int buffers, int load,
                    std::string* src) {
  FusedArgs a;
  if (int rc = fused_jit_args(L, s, m, n, chunk, buffers, &a)) return rc;
  std::string why;
  if (!jit_source(a, L.F, a.buffers, src, &why)) return fail(ADHA_ENOTIMPL, "fused run not specialised: %s", why.c_str());
  if (!load) return jit_compile_only(*src);
  const void* fn = nullptr;
  return jit_kernel(a, L.F, a.buffers, true, &fn, &why);
}

// A section run as a one-section run specialised at run time, chunk shape (R, buffers); ENOTIMPL
// (nothing launched) where it cannot be, or is not compiled and the stream is being captured.
static int run_section_specialised(const Layout& L, void* const* ptrs, const adha_section* s, int64_t n, int R,
                                   int buffers, void* stream) {
  if (check_fused(L, s, 1, n)) {
    clear_error();
    return fail(ADHA_ENOTIMPL, "section not specialised");
  }
  const int saved_R = t_tile_override, saved_B = t_fused_buffers, saved_J = t_fused_jit;
  t_tile_override = R;
  t_fused_buffers = buffers;
  t_fused_jit = 2;
  FusedPlan plan;
  int rc = plan_fused(L, ptrs, s, 1, n, stream, &plan);
  t_tile_override = saved_R;
  t_fused_buffers = saved_B;
  t_fused_jit = saved_J;
  if (rc) return rc;
  return profiled(6, s->op, section_bytes(L, s, n, false), stream,
                  [&] { return launch_fused_jit(plan.jit, plan.args, plan.grid, plan.smem, stream); });
}

int run_section_specialised_shape(const Layout& L, void* const* ptrs, const adha_section* s, int64_t n, int R,
                                  int buffers, void* stream) {
  return run_section_specialised(L, ptrs, s, n, R, buffers, stream);
}

int run_section_layout(const Layout& L, void* const* ptrs, const adha_section* s, int64_t n, void* save, void* stream) {
  if (int rc = check_section(L, s, n, save != nullptr)) return rc;
  if (n == 0) return 0;
  // tuned (or asked) to run specialised: a one-section run compiled for this section and layout
  if (!save && t_section_jit != 1 && !t_tile_override && !t_writeback_mode && !t_section_buffers) {
    int R = 0, mode = 0;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(section_key(L, s, n, false));
      if (it != g_tune.end()) {
        R = it->second.first;
        mode = it->second.second;
      }
    }
    if ((mode & 8) || t_section_jit == 2) {
      const int rc = run_section_specialised(L, ptrs, s, n, (mode & 8) ? R : 0, (mode & 8) ? ((mode & 4) ? 1 : 2) : 0,
                                             stream);
      if (rc != ADHA_ENOTIMPL) return rc;
      clear_error();   // not specialised: the library's section kernel
    }
  }
  SectionPlan plan;
  if (int rc = plan_section(L, ptrs, s, n, save, &plan)) return rc;
  return profiled(1, s->op, section_bytes(L, s, n, save != nullptr), stream,
                  [&] { return launch_section(plan.args, plan.grid, plan.smem, stream); });
}

}  // namespace adha

using namespace adha;

// ====================================================================== C ABI
extern "C" {

const char* adha_version(void) { return "adha-gb300 0.1 (sm_103a)"; }

const char* adha_last_error(void) { return t_err.c_str(); }

void adha_free(void* p) { std::free(p); }

int adha_layout_strides(const adha_schema* schema, const adha_layout* layout, int32_t* stride, int32_t* offset) {
  clear_error();
  Layout L;
  if (int rc = make_layout(schema, layout, &L, "")) return rc;
  if (!stride || !offset) return fail(ADHA_EINVAL, "output arrays are NULL");
  for (int g = 0; g < L.n_groups; ++g) stride[g] = L.stride[g];
  for (int f = 0; f < L.F; ++f) offset[f] = L.offset_of[f];
  return 0;
}

int adha_remap(const adha_schema* schema, int64_t n, const adha_layout* src, const void* const* src_ptrs,
               const adha_layout* dst, void* const* dst_ptrs, adha_stream stream) {
  clear_error();
  Layout S, D;
  if (int rc = make_layout(schema, src, &S, "source")) return rc;
  if (int rc = make_layout(schema, dst, &D, "destination")) return rc;
  if (n < 0) return fail(ADHA_EINVAL, "n = %lld is negative", (long long)n);
  if (n == 0) return 0;
  if (int rc = check_ptrs(src_ptrs, S.n_groups, "source")) return rc;
  if (int rc = check_ptrs(reinterpret_cast<const void* const*>(dst_ptrs), D.n_groups, "destination")) return rc;
  return do_remap(S, src_ptrs, D, dst_ptrs, n, stream, nullptr);
}

int adha_run_section(const adha_schema* schema, int64_t n, const adha_layout* layout, void* const* ptrs,
                     const adha_section* section, void* save, adha_stream stream) {
  clear_error();
  Layout L;
  if (int rc = make_layout(schema, layout, &L, "")) return rc;
  if (n < 0) return fail(ADHA_EINVAL, "n = %lld is negative", (long long)n);
  if (int rc = check_section(L, section, n, save != nullptr)) return rc;
  if (n == 0) return 0;
  if (int rc = check_ptrs(reinterpret_cast<const void* const*>(ptrs), L.n_groups, "layout")) return rc;
  if (save && reinterpret_cast<uintptr_t>(save) % 4) return fail(ADHA_EINVAL, "save buffer is not 4-byte aligned");
  if (section->op == ADHA_OP_GATHER && reinterpret_cast<uintptr_t>(section->perm) % 16)
    return fail(ADHA_EINVAL, "perm is not 16-byte aligned");
  return run_section_layout(L, ptrs, section, n, save, stream);
}

int adha_run_sections_fused(const adha_schema* schema, int64_t n, const adha_layout* layout, void* const* ptrs,
                            const adha_section* sections, int32_t n_sec, adha_stream stream) {
  clear_error();
  Layout L;
  if (int rc = make_layout(schema, layout, &L, "")) return rc;
  if (n < 0) return fail(ADHA_EINVAL, "n = %lld is negative", (long long)n);
  if (int rc = check_fused(L, sections, n_sec, n)) return rc;
  if (n == 0) return 0;
  if (int rc = check_ptrs(reinterpret_cast<const void* const*>(ptrs), L.n_groups, "layout")) return rc;
  return run_fused_layout(L, ptrs, sections, n_sec, n, stream);
}

int adha_fused_jit_build(const adha_schema* schema, int64_t n, const adha_layout* layout, const adha_section* sections,
                         int32_t n_sec, int32_t chunk_records, int32_t buffers, int32_t load, char* src, size_t cap,
                         size_t* len) {
  clear_error();
  Layout L;
  if (int rc = make_layout(schema, layout, &L, "")) return rc;
  if (n < 0) return fail(ADHA_EINVAL, "n = %lld is negative", (long long)n);
  if (chunk_records != 0 && chunk_records != 32 && chunk_records != 64 && chunk_records != 128)
    return fail(ADHA_EINVAL, "chunk_records %d is not 0, 32, 64 or 128", chunk_records);
  if (buffers < 0 || buffers > 2) return fail(ADHA_EINVAL, "buffers %d not in [0, 2]", buffers);
  std::string text;
  const int rc = fused_jit_build(L, sections, n_sec, n, chunk_records, buffers, load, &text);
  if (len) *len = text.size();
  if (src && cap) {
    const size_t k = std::min(cap - 1, text.size());
    std::memcpy(src, text.data(), k);
    src[k] = '\0';
  }
  return rc;
}

int adha_section_backward(const adha_schema* schema, int64_t n, const adha_layout* layout, void* const* state_ptrs,
                          void* const* grad_ptrs, const adha_section* section, const void* save, adha_stream stream) {
  clear_error();
  Layout L;
  if (int rc = make_layout(schema, layout, &L, "")) return rc;
  for (int f = 0; f < L.F; ++f)
    if (L.dtype[f] != ADHA_F32) return fail(ADHA_EINVAL, "backward needs fp32 fields (field %d is not)", f);
  if (n < 0) return fail(ADHA_EINVAL, "n = %lld is negative", (long long)n);
  if (!section) return fail(ADHA_EINVAL, "section is NULL");
  if (section->op != ADHA_OP_AXPB && section->op != ADHA_OP_MUL && section->op != ADHA_OP_TANH)
    return fail(ADHA_EINVAL, "backward is defined for axpb, mul and tanh sections only");
  if (int rc = check_section(L, section, n, true)) return rc;
  if (n == 0) return 0;
  if (!save) return fail(ADHA_EINVAL, "save buffer is NULL");
  if (int rc = check_ptrs(reinterpret_cast<const void* const*>(state_ptrs), L.n_groups, "state")) return rc;
  if (int rc = check_ptrs(reinterpret_cast<const void* const*>(grad_ptrs), L.n_groups, "gradient")) return rc;
  BackwardArgs a;
  std::memset(&a, 0, sizeof a);
  a.n = n;
  a.op = section->op;
  const int x = section->arg[0];
  const int y = section->op == ADHA_OP_MUL ? section->arg[1] : section->arg[0];
  const int z = section->op == ADHA_OP_MUL ? section->arg[2] : section->arg[1];
  a.x = x;
  a.y = y;
  a.z = z;
  a.a = section->fparam[0];
  const int fl[3] = {x, y, z};
  for (int k = 0; k < 3; ++k) {
    const int g = L.group_of[fl[k]];
    a.s[k] = static_cast<uint8_t*>(state_ptrs[g]) + L.offset_of[fl[k]];
    a.g[k] = static_cast<uint8_t*>(grad_ptrs[g]) + L.offset_of[fl[k]];
    a.ss[k] = a.gs[k] = L.stride[g];
  }
  a.save = static_cast<const float*>(save);
  tanh_coefficients(a.tanh_p, a.tanh_q);
  const double bytes = (double)n * (section->op == ADHA_OP_MUL ? 40.0 : 28.0);
  return profiled(2, section->op, bytes, stream, [&] { return launch_backward(a, stream); });
}

int adha_profile_start(int32_t max_records) {
  clear_error();
  if (max_records < 1 || max_records > (1 << 20)) return fail(ADHA_EINVAL, "max_records %d not in [1, 2^20]", max_records);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  while (t_pool.size() < 2 * (size_t)max_records) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return cuda_fail(err, "cudaEventCreate(profile)");
    t_pool.push_back(e);
  }
  t_prof.clear();
  t_pool_used = 0;
  t_prof_on = true;
  return 0;
}

int adha_profile_stop(adha_launch_record* out, int32_t max_records, int32_t* n_records) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  t_prof_on = false;
  if (!n_records) return fail(ADHA_EINVAL, "n_records is NULL");
  int32_t k = 0;
  for (const ProfRec& r : t_prof) {
    if (out && k < max_records) {
      cudaError_t e = cudaEventSynchronize(r.b);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
      if (e != cudaSuccess) return cuda_fail(e, "profile event");
      out[k] = adha_launch_record{r.kind, r.op, r.bytes, (double)ms};
    }
    ++k;
  }
  *n_records = k;
  t_prof.clear();
  t_pool_used = 0;
  return 0;
}

int adha_tune_override(int32_t chunk_records) {
  clear_error();
  if (chunk_records < 0 || chunk_records % 8 != 0 || chunk_records > 1024)
    return fail(ADHA_EINVAL, "chunk %d is not a multiple of 8 in [0, 1024]", chunk_records);
  t_tile_override = chunk_records;
  return 0;
}

int adha_tune_clear(void) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return 0;
}

int adha_tune_export(char* buf, size_t len, size_t* needed) {
  clear_error();
  std::string text;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : g_tune)
      text += kv.first + "\t" + std::to_string(kv.second.first) + "\t" + std::to_string(kv.second.second) + "\n";
  }
  if (needed) *needed = text.size() + 1;
  if (buf && len > text.size()) std::memcpy(buf, text.c_str(), text.size() + 1);
  else if (buf && len) return fail(ADHA_ENOMEM, "export buffer of %zu bytes is too small (%zu needed)", len, text.size() + 1);
  return 0;
}

int adha_tune_import(const char* text) {
  clear_error();
  if (!text) return fail(ADHA_EINVAL, "text is NULL");
  std::map<std::string, std::pair<int, int>> parsed;
  const char* p = text;
  while (*p) {
    const char* eol = std::strchr(p, '\n');
    std::string line(p, eol ? (size_t)(eol - p) : std::strlen(p));
    p = eol ? eol + 1 : p + line.size();
    if (line.empty()) continue;
    const size_t t1 = line.find('\t'), t2 = line.find('\t', t1 == std::string::npos ? 0 : t1 + 1);
    if (t1 == std::string::npos || t2 == std::string::npos || t1 < 2 || line.find('\t', t2 + 1) != std::string::npos)
      return fail(ADHA_EINVAL, "bad tuning line (want key<TAB>records<TAB>mode): %s", line.c_str());
    const char kind = line[0];
    if (kind != 'S' && kind != 'M' && kind != 'F') return fail(ADHA_EINVAL, "bad tuning key kind '%c': %s", kind, line.c_str());
    // both values whole decimal numbers, nothing else on the line
    auto number = [&](size_t from, size_t to, int* v) {
      if (to <= from || to - from > 6) return false;
      int x = 0;
      for (size_t q = from; q < to; ++q) {
        if (line[q] < '0' || line[q] > '9') return false;
        x = 10 * x + (line[q] - '0');
      }
      *v = x;
      return true;
    };
    int R = 0, wb = 0;
    if (!number(t1 + 1, t2, &R) || !number(t2 + 1, line.size(), &wb))
      return fail(ADHA_EINVAL, "bad tuning values (not whole numbers): %s", line.c_str());
    const bool bad = kind == 'M'   ? (R % 8 || R < 0 || R > 1024 || wb > 7)
                     : kind == 'F' ? (R % 32 || R > 128 || (wb & 3) > 2 || wb > 6)
                                   : (R % 32 || R > 128 || (wb & 3) > 2 || wb > 14);
    if (bad) return fail(ADHA_EINVAL, "bad tuning values: %s", line.c_str());
    parsed[line.substr(0, t1)] = {R, wb};
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : parsed) g_tune[kv.first] = kv.second;
  return 0;
}

int adha_tune_remap_direct(int32_t mode) {
  clear_error();
  if (mode < 0 || mode > 1) return fail(ADHA_EINVAL, "remap direct mode %d not in [0, 1]", mode);
  t_remap_direct = mode;
  return 0;
}

int adha_tune_remap_pieces(int32_t mode) {
  clear_error();
  if (mode < 0 || mode > 8) return fail(ADHA_EINVAL, "remap piece-table mode %d not in [0, 8]", mode);
  t_remap_pieces = mode;
  return 0;
}

int adha_tune_section_buffers(int32_t buffers) {
  clear_error();
  if (buffers < 0 || buffers > 2) return fail(ADHA_EINVAL, "section buffers %d not in [0, 2]", buffers);
  t_section_buffers = buffers;
  return 0;
}

int adha_tune_section_jit(int32_t mode) {
  clear_error();
  if (mode < 0 || mode > 2) return fail(ADHA_EINVAL, "section mode %d not in [0, 2]", mode);
  t_section_jit = mode;
  return 0;
}

int adha_tune_fused_buffers(int32_t buffers) {
  clear_error();
  if (buffers < 0 || buffers > 2) return fail(ADHA_EINVAL, "fused buffers %d not in [0, 2]", buffers);
  t_fused_buffers = buffers;
  return 0;
}

int adha_tune_fused_jit(int32_t mode) {
  clear_error();
  if (mode < 0 || mode > 2) return fail(ADHA_EINVAL, "fused run mode %d not in [0, 2]", mode);
  t_fused_jit = mode;
  return 0;
}

int adha_jit_available(void) {
  clear_error();
  std::string why;
  if (jit_available(&why)) return 1;
  fail(ADHA_ENOTIMPL, "%s", why.c_str());
  return 0;
}

int adha_jit_log(char* buf, size_t cap, size_t* len) {
  clear_error();
  const std::string log = jit_last_log();
  if (len) *len = log.size();
  if (buf && cap) {
    const size_t k = std::min(cap - 1, log.size());
    std::memcpy(buf, log.data(), k);
    buf[k] = '\0';
  }
  return 0;
}

int adha_tune_writeback(int32_t mode) {
  clear_error();
  if (mode < 0 || mode > 2) return fail(ADHA_EINVAL, "writeback mode %d not in [0, 2]", mode);
  t_writeback_mode = mode;
  return 0;
}

}  // extern "C"

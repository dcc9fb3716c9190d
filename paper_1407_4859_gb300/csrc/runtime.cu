// runtime.cu -- the measured side of PDL and the program executor.
//
// adha_measure is ADHA's "tuning profile" (paper Section 2: the PDL pass takes execution times
// measured on the device): it times every section in every candidate layout and every remap
// between candidates on the caller's own data (copied into a workspace first, so the input is
// not changed), with CUDA events on the caller's stream.  adha_run_program solves PDL on such a
// table and enqueues the chosen chain of remaps and sections on one stream; groups that two
// consecutive layouts share are kept in place (aliased), new groups are carved from a caller
// workspace by a first-fit allocator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace adha {

constexpr int kFusedLayouts = 8;   // candidates a fused run is timed in (its cheapest one by one)

static size_t round256(size_t x) { return (x + 255) / 256 * 256; }

static size_t layout_bytes(const Layout& L, int64_t n) {
  size_t b = 0;
  for (int g = 0; g < L.n_groups; ++g) b += round256((size_t)n * L.stride[g]);
  return b;
}

static bool same_layout(const Layout& a, const Layout& b) { return a.groups == b.groups; }

static int load_set(const adha_schema* schema, const adha_layout_set* set, std::vector<Layout>* out) {
  if (!set || set->n_layouts < 1 || set->n_fields != schema->n_fields)
    return fail(ADHA_EINVAL, "candidate set is empty or has another field count");
  out->resize(set->n_layouts);
  for (int l = 0; l < set->n_layouts; ++l) {
    const adha_layout x = set_layout(set, l);
    if (int rc = make_layout(schema, &x, &(*out)[l], "candidate")) return rc;
  }
  return 0;
}

// ------------------------------------------------------------------ workspace allocator
struct Arena {
  uint8_t* base = nullptr;
  size_t size = 0;
  std::vector<std::pair<size_t, size_t>> used;   // (offset, bytes), sorted by offset

  void* alloc(size_t bytes) {
    bytes = round256(std::max<size_t>(bytes, 1));
    size_t at = 0;
    for (size_t k = 0; k <= used.size(); ++k) {
      const size_t end = k < used.size() ? used[k].first : size;
      if (at + bytes <= end) {
        used.insert(used.begin() + k, {at, bytes});
        return base + at;
      }
      if (k < used.size()) at = used[k].first + used[k].second;
    }
    return nullptr;
  }
  void release(const void* p) {
    const size_t off = static_cast<const uint8_t*>(p) - base;
    for (size_t k = 0; k < used.size(); ++k)
      if (used[k].first == off) {
        used.erase(used.begin() + k);
        return;
      }
  }
  bool owns(const void* p) const {
    const uint8_t* q = static_cast<const uint8_t*>(p);
    return q >= base && q < base + size;
  }
};

// ------------------------------------------------------------------ timing
struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  int init() {
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    return e == cudaSuccess ? 0 : cuda_fail(e, "cudaEventCreate");
  }
};

// Whole nanoseconds of one call of `fn`: one warm-up call, then the faster of two batches of
// `reps` back-to-back calls timed with events on `stream`.
template <class Fn>
static int time_ns(Timer& t, void* stream, int reps, Fn fn, double* ns) {
  if (int rc = fn()) return rc;
  double best = -1;
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = cudaEventRecord(t.e0, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (int r = 0; r < reps; ++r)
      if (int rc = fn()) return rc;
    e = cudaEventRecord(t.e1, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t.e1);
    if (e != cudaSuccess) return cuda_fail(e, "timing event");
    float ms = 0;
    e = cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    const double v = (double)ms * 1e6 / reps;
    if (best < 0 || v < best) best = v;
  }
  *ns = (double)(long long)(best + 0.5);
  return 0;
}

static void carve(const Layout& L, int64_t n, uint8_t* base, std::vector<void*>* ptrs) {
  ptrs->assign(L.n_groups, nullptr);
  size_t off = 0;
  for (int g = 0; g < L.n_groups; ++g) {
    (*ptrs)[g] = base + off;
    off += round256((size_t)n * L.stride[g]);
  }
}

// Destination pointers of layout D after S (pointers sp): groups identical to a group of S alias
// it, the others are carved from `base`.
static void carve_after(const Layout& S, const std::vector<void*>& sp, const Layout& D, int64_t n, uint8_t* base,
                        std::vector<void*>* dp) {
  carve(D, n, base, dp);
  for (int g = 0; g < D.n_groups; ++g)
    for (int j = 0; j < S.n_groups; ++j)
      if (same_group(D, g, S, j)) (*dp)[g] = sp[j];
}

}  // namespace adha

using namespace adha;

extern "C" {

size_t adha_measure_workspace_bytes_for(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                                        const adha_layout_set* candidates, int32_t flags) {
  clear_error();
  Layout in;
  std::vector<Layout> cand;
  if (make_layout(schema, in_layout, &in, "input") || load_set(schema, candidates, &cand)) return 0;
  size_t m = layout_bytes(in, n);
  for (const Layout& L : cand) m = std::max(m, layout_bytes(L, n));
  // differentiable: a third copy for the gradients and the saved values of one section
  return (flags & ADHA_MEASURE_DIFFERENTIABLE) ? 3 * m + round256((size_t)n * 4) : 2 * m;
}

size_t adha_measure_workspace_bytes(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                                    const adha_layout_set* candidates) {
  return adha_measure_workspace_bytes_for(schema, n, in_layout, candidates, 0);
}

int adha_measure(const adha_schema* schema, int64_t n, const adha_layout* in_layout, void* const* in_ptrs,
                 const adha_section* sections, int32_t n_sec, const adha_layout_set* candidates, int32_t reps,
                 int32_t flags, void* workspace, size_t ws_bytes, adha_stream stream, adha_cost_table** out) {
  clear_error();
  Layout in;
  std::vector<Layout> cand;
  if (int rc = make_layout(schema, in_layout, &in, "input")) return rc;
  if (int rc = load_set(schema, candidates, &cand)) return rc;
  if (n < 1) return fail(ADHA_EINVAL, "n = %lld: nothing to measure", (long long)n);
  if (!in_ptrs || !sections || n_sec < 1 || n_sec > ADHA_MAX_SECTIONS || !out)
    return fail(ADHA_EINVAL, "bad arguments to adha_measure");
  if (reps < 1) reps = 2;
  const bool diff = (flags & ADHA_MEASURE_DIFFERENTIABLE) != 0;
  if (diff) {
    for (int f = 0; f < in.F; ++f)
      if (in.dtype[f] != ADHA_F32) return fail(ADHA_EINVAL, "a differentiable program has fp32 fields (field %d is not)", f);
    for (int k = 0; k < n_sec; ++k)
      if (sections[k].op != ADHA_OP_AXPB && sections[k].op != ADHA_OP_MUL && sections[k].op != ADHA_OP_TANH)
        return fail(ADHA_EINVAL, "a differentiable program has axpb, mul and tanh sections (section %d is not)", k);
  }
  size_t m = layout_bytes(in, n);
  for (const Layout& L : cand) m = std::max(m, layout_bytes(L, n));
  const size_t need = adha_measure_workspace_bytes_for(schema, n, in_layout, candidates, flags);
  if (!workspace || ws_bytes < need) return fail(ADHA_ENOMEM, "measure workspace has %zu bytes, needs %zu", ws_bytes, need);
  const int L = (int)cand.size();
  const int W = diff ? 0 : std::min((flags >> 8) & 0xFF, std::min(n_sec, kMaxFused));
  adha_cost_table* t = nullptr;
  if (int rc = adha_cost_table_create_fused(n_sec, L, W >= 2 ? W : 0, &t)) return rc;
  // runs of 2..W consecutive sections that may be fused (whether they may does not depend on the layout)
  std::vector<std::pair<int, int>> runs;
  for (int k = 0; k < n_sec && W >= 2; ++k)
    for (int m = 2; m <= W && k + m <= n_sec; ++m)
      if (fusable_run(in, &sections[k], m)) runs.push_back({k, m});
  uint8_t* A = static_cast<uint8_t*>(workspace);
  uint8_t* B = A + m;
  uint8_t* C = B + m;                 // differentiable: gradients in layout a
  void* saved = C + m;                // differentiable: the values one section overwrites
  std::vector<void*> in_p(in_ptrs, in_ptrs + in.n_groups), pa, pb, pg;
  Timer timer;
  int rc = timer.init();
  auto done = [&](int code) {
    if (code) std::free(t);
    else *out = t;
    return code;
  };
  if (rc) return done(rc);
  // A remap into or out of the input layout (every plan starts there, and may return there):
  // under autotuning, timed with each choice of piece tables and the fastest kept.
  auto time_remap = [&](const Layout& S, const std::vector<void*>& sp, const Layout& D, const std::vector<void*>& dp,
                        bool tune, double* ns) {
    auto run = [&] { return remap_layouts(S, sp.data(), D, const_cast<void**>(dp.data()), n, stream, nullptr); };
    if (!tune || !(flags & ADHA_MEASURE_AUTOTUNE)) return time_ns(timer, stream, reps, run, ns);
    double best = -1, t = 0;
    int bits = 0, bestR = 0;
    for (int m = 1; m <= 8; ++m) {   // piece tables x one or two chunk buffers per warp
      set_remap_pieces(m);
      const int e = time_ns(timer, stream, reps, run, &t);
      set_remap_pieces(0);
      if (e) return e;
      if (best < 0 || t < best) {
        best = t;
        bits = m - 1;
      }
    }
    // then the chunk: records per chunk from 24 to 128 with the best of the above (the size rule
    // gives 16 records for 80-byte records, where the per-chunk work dominates)
    for (const int R : {24, 32, 48, 64, 96, 128}) {
      set_remap_pieces(bits + 1);
      set_overrides(R, 0, 0);
      const int e = time_ns(timer, stream, reps, run, &t);
      set_overrides(0, 0, 0);
      set_remap_pieces(0);
      if (e) return e;
      if (t < best) {
        best = t;
        bestR = R;
      }
    }
    tuning_store(remap_tuning_key(S, D, n), bestR, bits);
    *ns = best;
    return 0;
  };
  for (int a = 0; a < L && !rc; ++a) {
    // input -> a (identical groups stay where they are)
    carve_after(in, in_p, cand[a], n, B, &pb);
    double ns = 0;
    rc = time_remap(in, in_p, cand[a], pb, true, &ns);
    if (rc) break;
    t->remap_ns[(size_t)L * (L + 1) + a] = ns;
    // a full private copy of the input in layout a, for the section and remap timings
    carve(cand[a], n, A, &pa);
    rc = remap_layouts(in, in_p.data(), cand[a], pa.data(), n, stream, nullptr);
    if (diff) carve(cand[a], n, C, &pg);
    for (int k = 0; k < n_sec && !rc; ++k) {
      // a differentiable program's forward sections keep what they overwrite
      void* save = diff ? saved : nullptr;
      auto run = [&] { return run_section_layout(cand[a], pa.data(), &sections[k], n, save, stream); };
      if (flags & ADHA_MEASURE_AUTOTUNE) {
        // every chunk size x store mode with two chunk buffers per warp, and 64 or 128 records
        // with one (twice the resident warps; at 32 records one buffer hides too little, except
        // for the assign and reduce sections, whose long compute per chunk wants the most warps);
        // the fastest is kept for the executor, one buffer as store mode + 4
        double best = -1;
        int bR = 0, bW = 0;
        const bool long_compute = sections[k].op == ADHA_OP_ASSIGN || sections[k].op == ADHA_OP_REDUCE;
        for (int nb = 2; nb >= 1 && !rc; --nb)
          for (int R = nb == 2 || long_compute ? 32 : 64; R <= 128 && !rc; R *= 2)
            for (int wb = 1; wb <= 2 && !rc; ++wb) {
              set_overrides(R, wb, nb);
              rc = time_ns(timer, stream, reps, run, &ns);
              if (!rc && (best < 0 || ns < best)) {
                best = ns;
                bR = R;
                bW = wb + (nb == 1 ? 4 : 0);
              }
            }
        set_overrides(0, 0, 0);
        if (rc) break;
        tuning_store(tuning_key(cand[a], &sections[k], n, diff), bR, bW);
        ns = best;
      } else {
        rc = time_ns(timer, stream, reps, run, &ns);
      }
      if (diff && !rc) {   // plus its adjoint kernel in the same layout
        const adha_layout cl = set_layout(candidates, a);
        double bw = 0;
        rc = time_ns(timer, stream, reps, [&] {
          return adha_section_backward(schema, n, &cl, pa.data(), pg.data(), &sections[k], saved, stream);
        }, &bw);
        ns += bw;
      }
      t->section_ns[(size_t)k * L + a] = ns;
    }
    for (int b = 0; b <= L && !rc; ++b) {
      if (b == a) continue;
      const Layout& D = b < L ? cand[b] : in;
      if (same_layout(cand[a], D)) continue;
      carve_after(cand[a], pa, D, n, B, &pb);
      rc = time_remap(cand[a], pa, D, pb, b == L, &ns);
      t->remap_ns[(size_t)a * (L + 1) + b] = ns;
    }
  }
  // Specialised sections (autotuning, not differentiable, when the run-time compiler can be
  // loaded): each section also as a one-section run compiled for it, in the kJitSectionLayouts
  // candidates where the library's kernel did best and in the one that PDL on the table so far
  // picks for it (a plan keeps a layout across sections to save remaps, so that one is often
  // none of the three), under six chunk shapes (32 / 64 / 128 records x one or two buffers).  All
  // are compiled first, in parallel host threads; a faster time replaces the entry and its tuning
  // says "specialised" (mode + 8).
  if ((flags & ADHA_MEASURE_AUTOTUNE) && !diff && !rc && jit_available(nullptr)) {
    constexpr int kJitSectionLayouts = 3;
    const int shapes[6][2] = {{32, 1}, {32, 2}, {64, 1}, {64, 2}, {128, 1}, {128, 2}};
    std::vector<int32_t> pre(n_sec, -1);
    double pre_total = 0;
    if (pdl_solve(t, 0, pre.data(), &pre_total)) {
      clear_error();
      std::fill(pre.begin(), pre.end(), -1);
    }
    std::vector<std::vector<int>> top(n_sec);
    std::vector<bool> any(L, false);
    std::vector<FusedArgs> jargs;
    std::vector<int> jF, jB;
    for (int k = 0; k < n_sec; ++k) {
      std::vector<std::pair<double, int>> by;
      for (int a = 0; a < L; ++a) by.push_back({t->section_ns[(size_t)k * L + a], a});
      std::sort(by.begin(), by.end());
      std::vector<int> pick;
      for (int j = 0; j < (int)by.size() && j < kJitSectionLayouts; ++j) pick.push_back(by[j].second);
      if (pre[k] >= 0 && pre[k] < L && std::find(pick.begin(), pick.end(), pre[k]) == pick.end()) pick.push_back(pre[k]);
      for (const int a : pick) {
        bool ok = false;
        for (int q = 0; q < 6; ++q) {
          FusedArgs x;
          if (fused_jit_args(cand[a], &sections[k], 1, n, shapes[q][0], shapes[q][1], &x)) {
            clear_error();
            continue;
          }
          jargs.push_back(x);
          jF.push_back(cand[a].F);
          jB.push_back(x.buffers);
          ok = true;
        }
        if (ok) {
          top[k].push_back(a);
          any[a] = true;
        }
      }
    }
    if (jit_prepare(jargs, jF, jB)) clear_error();
    for (int a = 0; a < L && !rc; ++a) {
      if (!any[a]) continue;
      carve(cand[a], n, A, &pa);
      rc = remap_layouts(in, in_p.data(), cand[a], pa.data(), n, stream, nullptr);
      for (int k = 0; k < n_sec && !rc; ++k) {
        if (std::find(top[k].begin(), top[k].end(), a) == top[k].end()) continue;
        double& entry = t->section_ns[(size_t)k * L + a];
        for (int q = 0; q < 6 && !rc; ++q) {
          double ns = 0;
          const int R = shapes[q][0], nb = shapes[q][1];
          const int e = time_ns(timer, stream, reps, [&] {
            return run_section_specialised_shape(cand[a], pa.data(), &sections[k], n, R, nb, stream);
          }, &ns);
          if (e == ADHA_ENOTIMPL) {
            clear_error();
            continue;
          }
          rc = e;
          if (!rc && ns < entry) {
            entry = ns;
            tuning_store(tuning_key(cand[a], &sections[k], n, false), R, 8 + (nb == 1 ? 4 : 0));
          }
        }
      }
    }
  }
  // Fused runs: each run is timed in the kFusedLayouts candidates where its sections cost least
  // one by one (the others stay +inf); under autotuning, with four launch shapes (records per
  // chunk x chunk buffers, kept in the tuning cache).  Fusing reads every field once instead of once per section, so a layout that
  // is poor for the run's sections is poor for the run too.
  std::vector<std::vector<int>> where(runs.size());
  std::vector<bool> used(L, false);
  for (size_t r = 0; r < runs.size(); ++r) {
    const int k = runs[r].first, m = runs[r].second;
    std::vector<std::pair<double, int>> by;
    for (int a = 0; a < L; ++a) {
      double sum = 0;
      for (int j = 0; j < m; ++j) sum += t->section_ns[(size_t)(k + j) * L + a];
      by.push_back({sum, a});
    }
    std::sort(by.begin(), by.end());
    for (int j = 0; j < (int)by.size() && j < kFusedLayouts; ++j) {
      where[r].push_back(by[j].second);
      used[by[j].second] = true;
    }
  }
  for (int a = 0; a < L && !rc; ++a) {
    if (!used[a]) continue;
    carve(cand[a], n, A, &pa);
    rc = remap_layouts(in, in_p.data(), cand[a], pa.data(), n, stream, nullptr);
    for (size_t r = 0; r < runs.size() && !rc; ++r) {
      if (std::find(where[r].begin(), where[r].end(), a) == where[r].end()) continue;
      const int k = runs[r].first, m = runs[r].second;
      auto run = [&] { return run_fused_layout(cand[a], pa.data(), &sections[k], m, n, stream); };
      // each timing starts from the input's values: repeated runs of a window can drive them to
      // infinities, and fused runs take slower exact paths for such values
      auto fresh = [&] { return remap_layouts(in, in_p.data(), cand[a], pa.data(), n, stream, nullptr); };
      double ns = 0;
      if (flags & ADHA_MEASURE_AUTOTUNE) {
        // records per chunk x chunk buffers per warp: one buffer at 32 / 64 / 128, two at 64
        const int shapes[4][2] = {{32, 1}, {64, 1}, {128, 1}, {64, 2}};
        double best = -1;
        int bR = 0, bB = 0;
        for (int q = 0; q < 4 && !rc; ++q) {
          set_fused_overrides(shapes[q][0], shapes[q][1]);
          rc = fresh();
          if (!rc) rc = time_ns(timer, stream, reps, run, &ns);
          if (!rc && (best < 0 || ns < best)) {
            best = ns;
            bR = shapes[q][0];
            bB = shapes[q][1];
          }
        }
        set_fused_overrides(0, 0);
        if (rc) break;
        tuning_store(fused_tuning_key(cand[a], &sections[k], m, n), bR, bB);
        ns = best;
      } else {
        rc = fresh();
        if (!rc) rc = time_ns(timer, stream, reps, run, &ns);
      }
      t->fused_ns[((size_t)k * W + (m - 1)) * L + a] = ns;
    }
  }
  // Specialised runs (autotuning, when the run-time compiler can be loaded): each run in the two
  // candidates where its sections cost least one by one, under three chunk shapes.  All are
  // compiled first, in parallel host threads, then timed like the library's kernel; a faster one
  // replaces the entry, and its tuning says "specialised".  A run that cannot be specialised, or
  // a compile that fails, keeps the library kernel's time.
  if ((flags & ADHA_MEASURE_AUTOTUNE) && !rc && !runs.empty() && jit_available(nullptr)) {
    const int shapes[3][2] = {{32, 2}, {64, 1}, {64, 2}};
    constexpr int kJitLayouts = 2;
    std::vector<FusedArgs> jargs;
    std::vector<int> jF, jB;
    std::vector<bool> jit_layout(L, false);
    for (size_t r = 0; r < runs.size(); ++r)
      for (int j = 0; j < (int)where[r].size() && j < kJitLayouts; ++j) {
        const int a = where[r][j];
        for (int q = 0; q < 3; ++q) {
          FusedArgs x;
          if (fused_jit_args(cand[a], &sections[runs[r].first], runs[r].second, n, shapes[q][0], shapes[q][1], &x))
            continue;
          jargs.push_back(x);
          jF.push_back(cand[a].F);
          jB.push_back(x.buffers);
          jit_layout[a] = true;
        }
      }
    if (jit_prepare(jargs, jF, jB)) clear_error();
    for (int a = 0; a < L && !rc; ++a) {
      if (!jit_layout[a]) continue;
      carve(cand[a], n, A, &pa);
      rc = remap_layouts(in, in_p.data(), cand[a], pa.data(), n, stream, nullptr);
      for (size_t r = 0; r < runs.size() && !rc; ++r) {
        const auto top = std::find(where[r].begin(), where[r].end(), a);
        if (top == where[r].end() || top - where[r].begin() >= kJitLayouts) continue;
        const int k = runs[r].first, m = runs[r].second;
        double& entry = t->fused_ns[((size_t)k * W + (m - 1)) * L + a];
        auto run = [&] { return run_fused_layout(cand[a], pa.data(), &sections[k], m, n, stream); };
        auto fresh = [&] { return remap_layouts(in, in_p.data(), cand[a], pa.data(), n, stream, nullptr); };
        for (int q = 0; q < 3 && !rc; ++q) {
          set_fused_overrides(shapes[q][0], shapes[q][1]);
          set_fused_jit(2);
          double ns = 0;
          rc = fresh();
          int e = rc ? rc : time_ns(timer, stream, reps, run, &ns);
          set_fused_jit(0);
          set_fused_overrides(0, 0);
          if (e == ADHA_ENOTIMPL) {   // not specialised (or not compiled): the library kernel's time stands
            clear_error();
            continue;
          }
          rc = e;
          if (!rc && ns < entry) {
            entry = ns;
            tuning_store(fused_tuning_key(cand[a], &sections[k], m, n), shapes[q][0], shapes[q][1] + 4);
          }
        }
      }
    }
  }
  // differentiable: every remap of the forward pass has its inverse in the backward pass (the
  // gradients go back through the reversed byte permutation), so an edge costs both directions
  for (int a = 0; a <= L && diff && !rc; ++a)
    for (int b = a + 1; b <= L; ++b) {
      const double both = t->remap_ns[(size_t)a * (L + 1) + b] + t->remap_ns[(size_t)b * (L + 1) + a];
      t->remap_ns[(size_t)a * (L + 1) + b] = t->remap_ns[(size_t)b * (L + 1) + a] = both;
    }
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize(measure)");
  }
  return done(rc);
}

size_t adha_program_workspace_bytes(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                                    const adha_layout_set* candidates) {
  clear_error();
  Layout in;
  std::vector<Layout> cand;
  if (make_layout(schema, in_layout, &in, "input") || load_set(schema, candidates, &cand)) return 0;
  size_t m = layout_bytes(in, n);
  for (const Layout& L : cand) m = std::max(m, layout_bytes(L, n));
  return 3 * m;
}

}  // extern "C"

namespace adha {

// The plan a program runs: PDL on the cost table (with combine nodes when the options allow runs
// of two or more sections and the table holds fused costs) unless the caller fixed it; a fixed plan
// is validated and its model cost summed from the table (+inf for a window the table lacks).
static int settle_plan(const adha_cost_table* costs, const adha_plan_opts* opts, int n_sec, int L, adha_plan* plan) {
  const int back = opts ? opts->return_to_input : 0;
  const int fw = opts ? opts->fuse_window : 0;
  if (!plan->fixed) {
    if (!costs) return fail(ADHA_EINVAL, "no cost table: run adha_measure first or pass a fixed plan");
    if (fw >= 2 && costs->max_window >= 2 && costs->fused_ns)
      return pdl_solve_fused(costs, back, fw, plan->layout_of_section, plan->window_len, &plan->model_ns);
    for (int k = 0; k < n_sec; ++k) plan->window_len[k] = 1;
    return pdl_solve(costs, back, plan->layout_of_section, &plan->model_ns);
  }
  bool any = false;
  for (int k = 0; k < n_sec; ++k) {
    if (plan->layout_of_section[k] < 0 || plan->layout_of_section[k] >= L)
      return fail(ADHA_EINVAL, "fixed plan names candidate %d for section %d", plan->layout_of_section[k], k);
    any = any || plan->window_len[k] != 0;
  }
  if (!any)
    for (int k = 0; k < n_sec; ++k) plan->window_len[k] = 1;
  for (int k = 0; k < n_sec;) {
    const int m = plan->window_len[k];
    if (m < 1 || m > kMaxFused || k + m > n_sec) return fail(ADHA_EINVAL, "fixed plan has a window of %d at section %d", m, k);
    for (int j = 1; j < m; ++j)
      if (plan->window_len[k + j] != 0 || plan->layout_of_section[k + j] != plan->layout_of_section[k])
        return fail(ADHA_EINVAL, "fixed plan: section %d lies in the window at %d but is marked otherwise", k + j, k);
    k += m;
  }
  plan->model_ns = 0;
  if (costs) {
    if (int rc = check_costs(costs)) return rc;
    int prev = L;
    for (int k = 0; k < n_sec;) {
      const int l = plan->layout_of_section[k], m = plan->window_len[k];
      double c = costs->section_ns[(size_t)k * L + l];
      if (m > 1) c = m <= costs->max_window ? costs->fused_ns[((size_t)k * costs->max_window + (m - 1)) * L + l] : HUGE_VAL;
      plan->model_ns += costs->remap_ns[(size_t)prev * (L + 1) + l] + c;
      prev = l;
      k += m;
    }
    if (back) plan->model_ns += costs->remap_ns[(size_t)prev * (L + 1) + L];
  }
  return 0;
}

}  // namespace adha

extern "C" {

int adha_run_program(const adha_schema* schema, int64_t n, const adha_layout* in_layout, void* const* in_ptrs,
                     const adha_section* sections, int32_t n_sec, const adha_layout_set* candidates,
                     const adha_cost_table* costs, const adha_plan_opts* opts, void* workspace, size_t ws_bytes,
                     adha_stream stream, adha_plan* plan) {
  clear_error();
  Layout in;
  std::vector<Layout> cand;
  if (int rc = make_layout(schema, in_layout, &in, "input")) return rc;
  if (int rc = load_set(schema, candidates, &cand)) return rc;
  if (!plan || !sections || n_sec < 1 || n_sec > ADHA_MAX_SECTIONS) return fail(ADHA_EINVAL, "bad program arguments");
  if (n < 0) return fail(ADHA_EINVAL, "n = %lld is negative", (long long)n);
  const int L = (int)cand.size();
  const int back = opts ? opts->return_to_input : 0;
  if (costs && (costs->n_sections != n_sec || costs->n_layouts != L))
    return fail(ADHA_EINVAL, "cost table is %dx%d, program is %dx%d", costs->n_sections, costs->n_layouts, n_sec, L);
  if (int rc = settle_plan(costs, opts, n_sec, L, plan)) return rc;
  plan->n_sections = n_sec;
  plan->n_remaps = 0;
  plan->n_launches = 0;
  if (n > 0) {
    if (!in_ptrs) return fail(ADHA_EINVAL, "input pointers are NULL");
    for (int g = 0; g < in.n_groups; ++g)
      if (!in_ptrs[g] || reinterpret_cast<uintptr_t>(in_ptrs[g]) % 16)
        return fail(ADHA_EINVAL, "input buffer %d is NULL or not 16-byte aligned", g);
  }
  // every section must be valid in its layout, and the workspace must hold every group the plan
  // places there, before anything is launched: a dry run of the placements below
  {
    Arena dry;
    dry.base = static_cast<uint8_t*>(workspace);
    dry.size = workspace ? ws_bytes : 0;
    Layout c = in;
    std::vector<void*> cp(in.n_groups, nullptr);
    for (int g = 0; g < in.n_groups; ++g) cp[g] = in_ptrs ? in_ptrs[g] : nullptr;
    for (int k = 0; k < n_sec; k += plan->window_len[k]) {
      const Layout& D = cand[plan->layout_of_section[k]];
      if (!same_layout(c, D)) {
        std::vector<void*> dp(D.n_groups, nullptr);
        std::vector<bool> kept(c.n_groups, false);
        for (int g = 0; g < D.n_groups; ++g) {
          for (int j = 0; j < c.n_groups; ++j)
            if (same_group(D, g, c, j)) {
              dp[g] = cp[j];
              kept[j] = true;
            }
          if (!dp[g] && !(dp[g] = dry.alloc((size_t)n * D.stride[g])))
            return fail(ADHA_ENOMEM, "program workspace of %zu bytes is too small for the plan", ws_bytes);
        }
        for (int j = 0; j < c.n_groups; ++j)
          if (!kept[j] && cp[j] && dry.owns(cp[j])) dry.release(cp[j]);
        c = D;
        cp = dp;
      }
      const int m = plan->window_len[k];
      if (m > 1 && !fusable_run(D, &sections[k], m))
        return fail(ADHA_EINVAL, "sections %d..%d may not run fused", k, k + m - 1);
      for (int j = 0; j < m; ++j)
        if (int rc = check_section_layout(D, &sections[k + j], n)) return rc;
    }
  }
  Arena arena;
  arena.base = static_cast<uint8_t*>(workspace);
  arena.size = workspace ? ws_bytes : 0;
  Layout cur = in;
  std::vector<void*> cur_p(in_ptrs, in_ptrs + in.n_groups);
  for (int k = 0; k < n_sec; k += plan->window_len[k]) {
    const int l = plan->layout_of_section[k];
    const Layout& D = cand[l];
    if (!same_layout(cur, D)) {
      std::vector<void*> dp(D.n_groups, nullptr);
      std::vector<bool> kept(cur.n_groups, false);
      for (int g = 0; g < D.n_groups; ++g) {
        for (int j = 0; j < cur.n_groups; ++j)
          if (same_group(D, g, cur, j)) {
            dp[g] = cur_p[j];
            kept[j] = true;
          }
        if (!dp[g]) {
          dp[g] = arena.alloc((size_t)n * D.stride[g]);
          if (!dp[g]) return fail(ADHA_ENOMEM, "program workspace of %zu bytes is too small", ws_bytes);
        }
      }
      int launched = 0;
      if (int rc = remap_layouts(cur, cur_p.data(), D, dp.data(), n, stream, &launched)) return rc;
      plan->n_remaps += 1;
      plan->n_launches += launched;
      for (int j = 0; j < cur.n_groups; ++j)
        if (!kept[j] && arena.owns(cur_p[j])) arena.release(cur_p[j]);
      cur = D;
      cur_p = dp;
    }
    const int m = plan->window_len[k];
    if (int rc = m == 1 ? run_section_layout(cur, cur_p.data(), &sections[k], n, nullptr, stream)
                        : run_fused_layout(cur, cur_p.data(), &sections[k], m, n, stream))
      return rc;
    plan->n_launches += n > 0 ? 1 : 0;
  }
  if (back && !same_layout(cur, in)) {
    std::vector<void*> dp(in_ptrs, in_ptrs + in.n_groups);
    int launched = 0;
    if (int rc = remap_layouts(cur, cur_p.data(), in, dp.data(), n, stream, &launched)) return rc;
    plan->n_remaps += 1;
    plan->n_launches += launched;
    cur = in;
    cur_p = dp;
  }
  plan->final_layout = -1;
  for (int l = 0; l < L && plan->final_layout < 0; ++l)
    if (same_layout(cur, cand[l])) plan->final_layout = l;
  plan->final_n_groups = cur.n_groups;
  for (int g = 0; g < cur.n_groups; ++g) plan->final_ptrs[g] = cur_p[g];
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Programs on host-resident data: the record array is cut into slices that flow through three
// streams (upload, compute, download) chained by events over three buffer sets, so the upload of
// one slice, the program on the one before and the download of the one before that overlap.
// Sections are per record, so slices are independent; a section that reads through a
// permutation needs every record and forces one slice.

namespace adha {

constexpr int kPipeSets = 3;

struct HostPipe {
  cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
  cudaEvent_t start = nullptr, end_comp = nullptr, end_down = nullptr;
  cudaEvent_t uploaded[kPipeSets] = {}, computed[kPipeSets] = {}, freed[kPipeSets] = {};
};

static std::mutex g_pipe_mu;
static HostPipe g_pipes[256];

static int host_pipe(HostPipe** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(ADHA_ENOTIMPL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe& p = g_pipes[dev];
  if (!p.up) {
    cudaStream_t* ss[3] = {&p.up, &p.comp, &p.down};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(ss[k], cudaStreamNonBlocking);
    cudaEvent_t* ev[3] = {&p.start, &p.end_comp, &p.end_down};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(ev[k], cudaEventDisableTiming);
    for (int k = 0; k < kPipeSets && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&p.uploaded[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.computed[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.freed[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pipeline streams");
  }
  *out = &p;
  return 0;
}

static int64_t slice_records(int64_t n, int n_slices) { return (n + n_slices - 1) / n_slices; }

}  // namespace adha

extern "C" {

size_t adha_program_host_workspace_bytes(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                                         const adha_layout_set* candidates, int32_t n_slices) {
  clear_error();
  Layout in;
  std::vector<Layout> cand;
  if (n_slices < 1 || make_layout(schema, in_layout, &in, "input") || load_set(schema, candidates, &cand)) return 0;
  const int64_t ns = slice_records(n, n_slices);
  size_t m = layout_bytes(in, ns);
  for (const Layout& L : cand) m = std::max(m, layout_bytes(L, ns));
  return kPipeSets * (layout_bytes(in, ns) + 3 * m);
}

int adha_run_program_host(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                          const void* const* host_in, const adha_section* sections, int32_t n_sec,
                          const adha_layout_set* candidates, const adha_cost_table* costs, const adha_plan_opts* opts,
                          void* const* host_out, int32_t n_slices, void* workspace, size_t ws_bytes, adha_stream stream,
                          adha_plan* plan) {
  clear_error();
  Layout in;
  std::vector<Layout> cand;
  if (int rc = make_layout(schema, in_layout, &in, "input")) return rc;
  if (int rc = load_set(schema, candidates, &cand)) return rc;
  if (!plan || !sections || n_sec < 1 || n_sec > ADHA_MAX_SECTIONS || n < 0 || n_slices < 1)
    return fail(ADHA_EINVAL, "bad host-program arguments");
  for (int k = 0; k < n_sec; ++k)
    if (sections[k].read_at_perm_mask && n_slices > 1)
      return fail(ADHA_EINVAL, "section %d reads through a permutation: it needs every record, use one slice", k);
  const int L = (int)cand.size();
  // the plan (and with it the result's layout) is fixed before any data moves
  if (costs && (costs->n_sections != n_sec || costs->n_layouts != L)) return fail(ADHA_EINVAL, "cost table does not match");
  if (int rc = settle_plan(costs, opts, n_sec, L, plan)) return rc;
  const bool back = opts && opts->return_to_input;
  const Layout& out_layout = back ? in : cand[plan->layout_of_section[n_sec - 1]];
  if (!host_in || !host_out) return fail(ADHA_EINVAL, "host buffers are NULL");
  if (n == 0) return 0;
  const int64_t ns = slice_records(n, n_slices);
  const size_t need = adha_program_host_workspace_bytes(schema, n, in_layout, candidates, n_slices);
  if (!workspace || ws_bytes < need) return fail(ADHA_ENOMEM, "host-program workspace has %zu bytes, needs %zu", ws_bytes, need);
  HostPipe* pipe = nullptr;
  if (int rc = host_pipe(&pipe)) return rc;
  const size_t in_b = layout_bytes(in, ns), set_b = need / kPipeSets;
  cudaError_t e = cudaEventRecord(pipe->start, (cudaStream_t)stream);
  cudaStream_t ss[3] = {pipe->up, pipe->comp, pipe->down};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(ss[k], pipe->start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline start");
  // a REDUCE's result is zeroed once and every slice adds its records' sums into it (integer
  // sums: the total does not depend on how the records are cut)
  bool any_reduce = false;
  for (int k = 0; k < n_sec && e == cudaSuccess; ++k)
    if (sections[k].op == ADHA_OP_REDUCE) {
      any_reduce = true;
      const int K = sections[k].arg[1];
      int d = 0;
      for (int f = 0; f < in.F; ++f)
        d += f != sections[k].arg[0] && ((sections[k].read_mask >> f) & 1) ? 1 : 0;
      if (sections[k].aux) e = cudaMemsetAsync(const_cast<void*>(sections[k].aux), 0, (size_t)K * (d + 1) * 8, pipe->comp);
    }
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(reduce result)");
  struct Accumulate {   // REDUCE adds into its result during the slices, on this thread only
    bool on;
    explicit Accumulate(bool o) : on(o) { if (on) set_reduce_accumulate(true); }
    ~Accumulate() { if (on) set_reduce_accumulate(false); }
  } accumulate(any_reduce);
  adha_plan slice_plan;
  for (int64_t k = 0, i0 = 0; i0 < n; ++k, i0 += ns) {
    const int b = (int)(k % kPipeSets);
    const int64_t cnt = std::min(ns, n - i0);
    uint8_t* base = static_cast<uint8_t*>(workspace) + b * set_b;
    std::vector<void*> dev_in;
    carve(in, ns, base, &dev_in);
    // upload: once the download that last used this buffer set is done
    if (k >= kPipeSets) e = cudaStreamWaitEvent(pipe->up, pipe->freed[b], 0);
    for (int g = 0; g < in.n_groups && e == cudaSuccess; ++g)
      e = cudaMemcpyAsync(dev_in[g], static_cast<const uint8_t*>(host_in[g]) + i0 * in.stride[g],
                          (size_t)cnt * in.stride[g], cudaMemcpyHostToDevice, pipe->up);
    if (e == cudaSuccess) e = cudaEventRecord(pipe->uploaded[b], pipe->up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(pipe->comp, pipe->uploaded[b], 0);
    if (e != cudaSuccess) return cuda_fail(e, "slice upload");
    slice_plan = *plan;
    slice_plan.fixed = 1;
    if (int rc = adha_run_program(schema, cnt, in_layout, dev_in.data(), sections, n_sec, candidates, costs, opts,
                                  base + in_b, set_b - in_b, pipe->comp, &slice_plan))
      return rc;
    e = cudaEventRecord(pipe->computed[b], pipe->comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(pipe->down, pipe->computed[b], 0);
    for (int g = 0; g < slice_plan.final_n_groups && e == cudaSuccess; ++g)
      e = cudaMemcpyAsync(static_cast<uint8_t*>(host_out[g]) + i0 * out_layout.stride[g], slice_plan.final_ptrs[g],
                          (size_t)cnt * out_layout.stride[g], cudaMemcpyDeviceToHost, pipe->down);
    if (e == cudaSuccess) e = cudaEventRecord(pipe->freed[b], pipe->down);
    if (e != cudaSuccess) return cuda_fail(e, "slice download");
  }
  e = cudaEventRecord(pipe->end_comp, pipe->comp);
  if (e == cudaSuccess) e = cudaEventRecord(pipe->end_down, pipe->down);
  if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, pipe->end_comp, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, pipe->end_down, 0);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline join");
  const double model = plan->model_ns;
  *plan = slice_plan;
  plan->fixed = 0;
  plan->model_ns = model;
  plan->final_n_groups = out_layout.n_groups;
  for (int g = 0; g < out_layout.n_groups; ++g) plan->final_ptrs[g] = host_out[g];
  return 0;
}

}  // extern "C"

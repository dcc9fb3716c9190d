// planner.cu -- host side of ADHA's two levels (paper Section 2):
//   ODS: an affinity graph over the fields a run of sections accesses, edge weight = the number
//        of record accesses reaching both fields (a section accesses record i, and record
//        perm[i] if it gathers); greedy clustering of fields into structures under a
//        struct-size limit ("determined based on the underlying architecture");
//   PDL: one layout per section for the whole program: the shortest path through the layered
//        DAG input -> section 1 -> ... -> section S whose nodes are (section, candidate layout),
//        node weight = measured section time, edge weight = measured remap time (0 when the
//        layout stays: the paper's "combine" edge).
// Readings where the paper is silent: ties in the greedy order go to the smaller field id, then
// the larger; a cluster merge must keep the struct (fields ascending, natural alignment) within
// the limit; candidates are AoS, SoA and the ODS layout of every window of consecutive
// sections under every limit; among equally short paths the lexicographically smallest
// sequence of candidate indices wins.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "internal.h"

namespace adha {

using Groups = std::vector<std::vector<int>>;


// Canonical order: fields ascending inside a group, groups by their first field.
static Groups canonical(Groups g) {
  for (auto& x : g) std::sort(x.begin(), x.end());
  std::sort(g.begin(), g.end(), [](const std::vector<int>& a, const std::vector<int>& b) { return a[0] < b[0]; });
  return g;
}

Groups ods_groups(int F, const int* dtype, const adha_section* secs, int n_sec, int cap) {
  // affinity weights: each record access of each section (its record i: the fields it reads or
  // writes; record perm[i]: the fields it reads through the permutation) adds one to every pair
  std::vector<int> w(F * F, 0);
  for (int k = 0; k < n_sec; ++k)
    for (const uint64_t m : {secs[k].read_mask | secs[k].write_mask, secs[k].read_at_perm_mask})
      for (int a = 0; a < F; ++a)
        if ((m >> a) & 1ull)
          for (int b = a + 1; b < F; ++b)
            if ((m >> b) & 1ull) ++w[a * F + b];
  struct Edge { int w, a, b; };
  std::vector<Edge> edges;
  for (int a = 0; a < F; ++a)
    for (int b = a + 1; b < F; ++b)
      if (w[a * F + b] > 0) edges.push_back({w[a * F + b], a, b});
  std::sort(edges.begin(), edges.end(), [](const Edge& x, const Edge& y) {
    if (x.w != y.w) return x.w > y.w;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
  });
  // clusters as field lists; owner[f] = cluster id
  std::vector<int> owner(F);
  std::vector<std::vector<int>> members(F);
  for (int f = 0; f < F; ++f) {
    owner[f] = f;
    members[f] = {f};
  }
  for (const Edge& e : edges) {
    const int ca = owner[e.a], cb = owner[e.b];
    if (ca == cb) continue;
    std::vector<int> merged = members[ca];
    merged.insert(merged.end(), members[cb].begin(), members[cb].end());
    std::sort(merged.begin(), merged.end());
    if (cap > 0 && group_struct(dtype, merged, nullptr) > cap) continue;
    for (int f : members[cb]) owner[f] = ca;
    members[ca] = merged;
    members[cb].clear();
  }
  Groups out;
  for (int c = 0; c < F; ++c)
    if (!members[c].empty()) out.push_back(members[c]);
  return canonical(out);
}

static int validate_sections(int F, const adha_section* secs, int n_sec) {
  if (n_sec < 1 || n_sec > ADHA_MAX_SECTIONS) return fail(ADHA_EINVAL, "%d sections (1..%d allowed)", n_sec, ADHA_MAX_SECTIONS);
  if (!secs) return fail(ADHA_EINVAL, "sections are NULL");
  const uint64_t all = F == 64 ? ~0ull : ((1ull << F) - 1);
  for (int k = 0; k < n_sec; ++k)
    if ((secs[k].read_mask | secs[k].write_mask | secs[k].read_at_perm_mask) & ~all) return fail(ADHA_EINVAL, "section %d names fields beyond %d", k, F);
  return 0;
}

// One malloc'd block holding the struct and its arrays, freed with adha_free.
static adha_layout_set* pack_set(int F, const std::vector<Groups>& layouts) {
  const size_t L = layouts.size();
  const size_t bytes = sizeof(adha_layout_set) + sizeof(int32_t) * (L + 2 * L * F);
  auto* s = static_cast<adha_layout_set*>(std::malloc(bytes));
  if (!s) return nullptr;
  int32_t* base = reinterpret_cast<int32_t*>(s + 1);
  s->n_fields = F;
  s->n_layouts = (int32_t)L;
  s->n_groups = base;
  s->group_len = base + L;
  s->fields = base + L + L * F;
  for (size_t l = 0; l < L; ++l) {
    s->n_groups[l] = (int32_t)layouts[l].size();
    int p = 0;
    for (size_t g = 0; g < layouts[l].size(); ++g) {
      s->group_len[l * F + g] = (int32_t)layouts[l][g].size();
      for (int f : layouts[l][g]) s->fields[l * F + p++] = f;
    }
    for (size_t g = layouts[l].size(); g < (size_t)F; ++g) s->group_len[l * F + g] = 0;
  }
  return s;
}

adha_layout set_layout(const adha_layout_set* s, int l) {
  adha_layout x;
  x.n_groups = s->n_groups[l];
  x.group_len = s->group_len + (size_t)l * s->n_fields;
  x.fields = s->fields + (size_t)l * s->n_fields;
  return x;
}

// Layered-DAG shortest path with lexicographic tie-break; costs are whole nanoseconds held in
// doubles, so every sum is exact and ties compare exactly.
// PDL with combine nodes: a plan is a sequence of windows (consecutive sections, run fused when
// longer than one) each in one layout.  rest[k][p] = cheapest way to run sections k.. when the
// data is in layout p (p = L: the input layout); a window [k, k+m) in layout l costs
// remap(p -> l) + cost(k, m, l), where cost(k, 1, l) = section_ns and cost(k, m >= 2, l) =
// fused_ns.  Ties: the smaller layout index, then the longer window, window by window from the
// first (the lexicographically smallest sequence of (layout, -length) pairs).
int check_costs(const adha_cost_table* c) {
  const size_t L = (size_t)c->n_layouts, S = (size_t)c->n_sections;
  auto bad = [](double v) { return std::isnan(v) || v < 0; };
  for (size_t k = 0; k < S * L; ++k)
    if (bad(c->section_ns[k]))
      return fail(ADHA_EINVAL, "cost table: section_ns[%zu][%zu] = %g (costs must be >= 0 or +inf)", k / L, k % L,
                  c->section_ns[k]);
  for (size_t k = 0; k < (L + 1) * (L + 1); ++k)
    if (bad(c->remap_ns[k]))
      return fail(ADHA_EINVAL, "cost table: remap_ns[%zu][%zu] = %g (costs must be >= 0 or +inf)", k / (L + 1),
                  k % (L + 1), c->remap_ns[k]);
  if (c->max_window >= 2 && c->fused_ns)
    for (size_t k = 0; k < S * (size_t)c->max_window * L; ++k)
      if (bad(c->fused_ns[k]))
        return fail(ADHA_EINVAL, "cost table: fused_ns entry %zu = %g (costs must be >= 0 or +inf)", k, c->fused_ns[k]);
  return 0;
}

int pdl_solve_fused(const adha_cost_table* c, int return_to_input, int max_window, int32_t* seq, int32_t* win,
                    double* total) {
  if (int rc = check_costs(c)) return rc;
  const int S = c->n_sections, L = c->n_layouts, In = L;
  const int W = std::max(1, std::min(max_window, std::max(1, c->max_window)));
  auto rem = [&](int a, int b) { return c->remap_ns[(size_t)a * (L + 1) + b]; };
  auto cost = [&](int k, int m, int l) {
    return m == 1 ? c->section_ns[(size_t)k * L + l] : c->fused_ns[((size_t)k * c->max_window + (m - 1)) * L + l];
  };
  std::vector<double> rest((size_t)(S + 1) * (L + 1));
  for (int p = 0; p <= L; ++p) rest[(size_t)S * (L + 1) + p] = return_to_input ? rem(p, In) : 0.0;
  auto step = [&](int k, int p, int* bl, int* bm) {
    double best = 0;
    bool first = true;
    for (int l = 0; l < L; ++l)
      for (int m = std::min(W, S - k); m >= 1; --m) {
        const double v = rem(p, l) + cost(k, m, l) + rest[(size_t)(k + m) * (L + 1) + l];
        if (first || v < best) {
          best = v;
          first = false;
          if (bl) *bl = l;
          if (bm) *bm = m;
        }
      }
    return best;
  };
  for (int k = S - 1; k >= 0; --k)
    for (int p = 0; p <= L; ++p) rest[(size_t)k * (L + 1) + p] = step(k, p, nullptr, nullptr);
  *total = rest[In];
  int p = In;
  for (int k = 0; k < S;) {
    int l = 0, m = 1;
    step(k, p, &l, &m);
    for (int j = 0; j < m; ++j) {
      seq[k + j] = l;
      if (win) win[k + j] = j == 0 ? m : 0;
    }
    p = l;
    k += m;
  }
  if (std::isinf(*total)) return fail(ADHA_EINVAL, "cost table: every plan has an infinite cost");
  return 0;
}

int pdl_solve(const adha_cost_table* c, int return_to_input, int32_t* seq, double* total) {
  if (int rc = check_costs(c)) return rc;
  const int S = c->n_sections, L = c->n_layouts, In = L;
  auto sec = [&](int k, int l) { return c->section_ns[(size_t)k * L + l]; };
  auto rem = [&](int a, int b) { return c->remap_ns[(size_t)a * (L + 1) + b]; };
  std::vector<double> rest((size_t)S * L);
  for (int l = 0; l < L; ++l) rest[(size_t)(S - 1) * L + l] = sec(S - 1, l) + (return_to_input ? rem(l, In) : 0.0);
  for (int k = S - 2; k >= 0; --k)
    for (int l = 0; l < L; ++l) {
      double best = 0;
      for (int m = 0; m < L; ++m) {
        const double v = rem(l, m) + rest[(size_t)(k + 1) * L + m];
        if (m == 0 || v < best) best = v;
      }
      rest[(size_t)k * L + l] = sec(k, l) + best;
    }
  int prev = In;
  for (int k = 0; k < S; ++k) {
    int arg = 0;
    double best = 0;
    for (int m = 0; m < L; ++m) {
      const double v = rem(prev, m) + rest[(size_t)k * L + m];
      if (m == 0 || v < best) {
        best = v;
        arg = m;
      }
    }
    if (k == 0) *total = best;
    seq[k] = arg;
    prev = arg;
  }
  if (std::isinf(*total)) return fail(ADHA_EINVAL, "cost table: every plan has an infinite cost");
  return 0;
}

// PDL over a structured control-flow graph: a cost matrix C[p][q] (N = L + 1 states, state L the
// input layout) per region of the tree, entered in layout p and left in layout q; then one best
// plan read back from the root with the choices of smallest index among equal costs.
struct ScfgSolver {
  const adha_cost_table* c;
  const adha_scfg_node* nodes;
  int L, N;
  std::vector<std::vector<double>> mat;   // per node, N x N
  std::vector<int32_t>* out;

  double rem(int a, int b) const { return c->remap_ns[(size_t)a * N + b]; }
  double sec(int k, int l) const { return c->section_ns[(size_t)k * L + l]; }

  std::vector<double> identity() const {
    std::vector<double> I((size_t)N * N, HUGE_VAL);
    for (int p = 0; p < N; ++p) I[(size_t)p * N + p] = 0;
    return I;
  }
  std::vector<double> minplus(const std::vector<double>& A, const std::vector<double>& B) const {
    std::vector<double> C((size_t)N * N, HUGE_VAL);
    for (int p = 0; p < N; ++p)
      for (int q = 0; q < N; ++q) {
        const double a = A[(size_t)p * N + q];
        if (a == HUGE_VAL) continue;
        for (int r = 0; r < N; ++r) {
          const double v = a + B[(size_t)q * N + r];
          if (v < C[(size_t)p * N + r]) C[(size_t)p * N + r] = v;
        }
      }
    return C;
  }

  void build(int i) {   // children first
    const adha_scfg_node& nd = nodes[i];
    for (int j = 0; j < nd.n_children; ++j) build(nd.children[j]);
    std::vector<double> C((size_t)N * N, HUGE_VAL);
    if (nd.kind == ADHA_SCFG_SECTION) {
      for (int p = 0; p < N; ++p)
        for (int q = 0; q < L; ++q) C[(size_t)p * N + q] = rem(p, q) + sec(nd.section, q);
    } else if (nd.kind == ADHA_SCFG_SEQ) {
      C = identity();
      for (int j = 0; j < nd.n_children; ++j) C = minplus(C, mat[nd.children[j]]);
    } else if (nd.kind == ADHA_SCFG_BRANCH) {
      std::fill(C.begin(), C.end(), 0.0);
      for (int j = 0; j < nd.n_children; ++j) {
        const std::vector<double>& B = mat[nd.children[j]];
        const double w = nd.weights[j];
        for (int p = 0; p < N; ++p)
          for (int q = 0; q < N; ++q) {
            double best = HUGE_VAL;
            for (int r = 0; r < N; ++r) best = std::min(best, B[(size_t)p * N + r] + rem(r, q));
            C[(size_t)p * N + q] += w * best;
          }
      }
    } else {   // loop
      const std::vector<double>& B = mat[nd.children[0]];
      const double T = nd.trips;
      for (int p = 0; p < N; ++p)
        for (int e = 0; e < N; ++e) {
          double best = HUGE_VAL;
          for (int f = 0; f < N; ++f) best = std::min(best, rem(p, f) + T * B[(size_t)f * N + e] + (T - 1) * rem(e, f));
          C[(size_t)p * N + e] = best;
        }
    }
    mat[i] = std::move(C);
  }

  void pick(int i, int p, int q) {
    const adha_scfg_node& nd = nodes[i];
    if (nd.kind == ADHA_SCFG_SECTION) {
      (*out)[i] = q;
    } else if (nd.kind == ADHA_SCFG_SEQ) {
      (*out)[i] = -1;
      std::vector<std::vector<double>> pref(1, identity());
      for (int j = 0; j < nd.n_children; ++j) pref.push_back(minplus(pref.back(), mat[nd.children[j]]));
      int cur = q;
      for (int j = nd.n_children; j >= 1; --j) {
        const std::vector<double>& M = mat[nd.children[j - 1]];
        int arg = 0;
        double best = HUGE_VAL;
        for (int r = 0; r < N; ++r) {
          const double v = pref[j - 1][(size_t)p * N + r] + M[(size_t)r * N + cur];
          if (v < best) {
            best = v;
            arg = r;
          }
        }
        pick(nd.children[j - 1], arg, cur);
        cur = arg;
      }
    } else if (nd.kind == ADHA_SCFG_BRANCH) {
      (*out)[i] = q;
      for (int j = 0; j < nd.n_children; ++j) {
        const std::vector<double>& B = mat[nd.children[j]];
        int arg = 0;
        double best = HUGE_VAL;
        for (int r = 0; r < N; ++r) {
          const double v = B[(size_t)p * N + r] + rem(r, q);
          if (v < best) {
            best = v;
            arg = r;
          }
        }
        pick(nd.children[j], p, arg);
      }
    } else {
      const std::vector<double>& B = mat[nd.children[0]];
      const double T = nd.trips;
      int arg = 0;
      double best = HUGE_VAL;
      for (int f = 0; f < N; ++f) {
        const double v = rem(p, f) + T * B[(size_t)f * N + q] + (T - 1) * rem(q, f);
        if (v < best) {
          best = v;
          arg = f;
        }
      }
      (*out)[i] = arg;
      pick(nd.children[0], arg, q);
    }
  }
};

}  // namespace adha

using namespace adha;

extern "C" {

int adha_pdl_solve_devices(int32_t n_devices, const adha_cost_table* const* costs, const double* transfer_ns,
                           int32_t input_device, int32_t return_to_input, int32_t* layout_of_section,
                           int32_t* device_of_section, double* total_ns) {
  clear_error();
  if (n_devices < 1 || n_devices > 8) return fail(ADHA_EINVAL, "n_devices = %d not in [1, 8]", n_devices);
  if (!costs || !transfer_ns || !layout_of_section || !device_of_section || !total_ns)
    return fail(ADHA_EINVAL, "NULL argument");
  if (input_device < 0 || input_device >= n_devices) return fail(ADHA_EINVAL, "input_device %d", input_device);
  const int D = n_devices;
  for (int d = 0; d < D; ++d) {
    if (!costs[d] || costs[d]->n_sections < 1 || costs[d]->n_layouts < 1 || !costs[d]->section_ns || !costs[d]->remap_ns)
      return fail(ADHA_EINVAL, "device %d: empty cost table", d);
    if (costs[d]->n_sections != costs[0]->n_sections || costs[d]->n_layouts != costs[0]->n_layouts)
      return fail(ADHA_EINVAL, "device %d: the tables differ in size", d);
    if (int rc = check_costs(costs[d])) return rc;
  }
  const int S = costs[0]->n_sections, L = costs[0]->n_layouts;
  for (size_t k = 0; k < (size_t)D * D * (L + 1); ++k)
    if (std::isnan(transfer_ns[k]) || transfer_ns[k] < 0)
      return fail(ADHA_EINVAL, "transfer_ns entry %zu = %g (must be >= 0 or +inf)", k, transfer_ns[k]);
  auto rem = [&](int d, int a, int b) { return costs[d]->remap_ns[(size_t)a * (L + 1) + b]; };
  auto xfer = [&](int a, int b, int l) { return transfer_ns[((size_t)a * D + b) * (L + 1) + l]; };
  auto edge = [&](int a, int la, int b, int lb) {
    if (a == b) return rem(a, la, lb);
    return std::min(rem(a, la, lb) + xfer(a, b, lb), xfer(a, b, la) + rem(b, la, lb));
  };
  // the plain PDL on the expanded table: state d*L + l, input state D*L
  const int LL = D * L;
  adha_cost_table* t = nullptr;
  if (int rc = adha_cost_table_create(S, LL, &t)) return rc;
  for (int k = 0; k < S; ++k)
    for (int d = 0; d < D; ++d)
      for (int l = 0; l < L; ++l) t->section_ns[(size_t)k * LL + d * L + l] = costs[d]->section_ns[(size_t)k * L + l];
  for (int x = 0; x <= LL; ++x)
    for (int y = 0; y <= LL; ++y) {
      const int a = x < LL ? x / L : input_device, la = x < LL ? x % L : L;
      const int b = y < LL ? y / L : input_device, lb = y < LL ? y % L : L;
      t->remap_ns[(size_t)x * (LL + 1) + y] = x == y ? 0.0 : edge(a, la, b, lb);
    }
  std::vector<int32_t> seq(S);
  const int rc = pdl_solve(t, return_to_input, seq.data(), total_ns);
  std::free(t);
  if (rc) return rc;
  for (int k = 0; k < S; ++k) {
    layout_of_section[k] = seq[k] % L;
    device_of_section[k] = seq[k] / L;
  }
  return 0;
}

int adha_pdl_solve_scfg(const adha_cost_table* costs, int32_t n_nodes, const adha_scfg_node* nodes, int32_t root,
                        int32_t return_to_input, int32_t* layout_of_node, double* total_ns) {
  clear_error();
  if (!costs || !nodes || !layout_of_node || !total_ns) return fail(ADHA_EINVAL, "NULL argument");
  if (costs->n_sections < 1 || costs->n_layouts < 1 || !costs->section_ns || !costs->remap_ns)
    return fail(ADHA_EINVAL, "empty cost table");
  if (n_nodes < 1 || n_nodes > 4096) return fail(ADHA_EINVAL, "n_nodes = %d not in [1, 4096]", n_nodes);
  if (root < 0 || root >= n_nodes) return fail(ADHA_EINVAL, "root %d is not a node", root);
  if (int rc = check_costs(costs)) return rc;
  // the nodes must form a tree below root, each reached once
  std::vector<int> seen(n_nodes, 0), stack{root};
  int reached = 0;
  while (!stack.empty()) {
    const int i = stack.back();
    stack.pop_back();
    if (seen[i]++) return fail(ADHA_EINVAL, "node %d is reached twice (the regions must form a tree)", i);
    ++reached;
    const adha_scfg_node& nd = nodes[i];
    if (nd.n_children < 0 || (nd.n_children > 0 && !nd.children)) return fail(ADHA_EINVAL, "node %d: bad children", i);
    switch (nd.kind) {
      case ADHA_SCFG_SECTION:
        if (nd.n_children != 0) return fail(ADHA_EINVAL, "section node %d has children", i);
        if (nd.section < 0 || nd.section >= costs->n_sections)
          return fail(ADHA_EINVAL, "node %d names section %d (the table has %d)", i, nd.section, costs->n_sections);
        break;
      case ADHA_SCFG_SEQ: break;
      case ADHA_SCFG_BRANCH: {
        if (nd.n_children < 1 || !nd.weights) return fail(ADHA_EINVAL, "branch node %d needs children and weights", i);
        double sum = 0;
        for (int j = 0; j < nd.n_children; ++j) {
          if (!(nd.weights[j] >= 0) || std::isinf(nd.weights[j]))
            return fail(ADHA_EINVAL, "branch node %d: weight %g", i, nd.weights[j]);
          sum += nd.weights[j];
        }
        if (std::fabs(sum - 1.0) > 1e-9) return fail(ADHA_EINVAL, "branch node %d: weights sum to %.12g, not 1", i, sum);
        break;
      }
      case ADHA_SCFG_LOOP:
        if (nd.n_children != 1) return fail(ADHA_EINVAL, "loop node %d has %d children (needs its body)", i, nd.n_children);
        if (!(nd.trips >= 1) || std::isinf(nd.trips)) return fail(ADHA_EINVAL, "loop node %d: trips = %g", i, nd.trips);
        break;
      default: return fail(ADHA_EINVAL, "node %d has kind %d", i, nd.kind);
    }
    for (int j = 0; j < nd.n_children; ++j) {
      const int ch = nd.children[j];
      if (ch < 0 || ch >= n_nodes) return fail(ADHA_EINVAL, "node %d: child %d is not a node", i, ch);
      stack.push_back(ch);
    }
  }
  std::vector<int32_t> out(n_nodes, -1);
  ScfgSolver sv;
  sv.c = costs;
  sv.nodes = nodes;
  sv.L = costs->n_layouts;
  sv.N = sv.L + 1;
  sv.mat.assign(n_nodes, {});
  sv.out = &out;
  sv.build(root);
  const std::vector<double>& C = sv.mat[root];
  int arg = 0;
  double best = HUGE_VAL;
  for (int q = 0; q < sv.N; ++q) {
    const double v = C[(size_t)sv.L * sv.N + q] + (return_to_input ? sv.rem(q, sv.L) : 0.0);
    if (v < best) {
      best = v;
      arg = q;
    }
  }
  if (std::isinf(best)) return fail(ADHA_EINVAL, "cost table: every plan has an infinite cost");
  sv.pick(root, sv.L, arg);
  for (int i = 0; i < n_nodes; ++i) layout_of_node[i] = out[i];
  *total_ns = best;
  return 0;
}


int adha_ods(const adha_schema* schema, const adha_section* sections, int32_t n_sec, int32_t cap_bytes,
             int32_t* n_groups, int32_t* group_len, int32_t* fields) {
  clear_error();
  if (int rc = check_schema(schema)) return rc;
  const int F = schema->n_fields;
  if (int rc = validate_sections(F, sections, n_sec)) return rc;
  if (!n_groups || !group_len || !fields) return fail(ADHA_EINVAL, "output arrays are NULL");
  const Groups g = ods_groups(F, schema->dtype, sections, n_sec, cap_bytes);
  *n_groups = (int32_t)g.size();
  int p = 0;
  for (size_t k = 0; k < g.size(); ++k) {
    group_len[k] = (int32_t)g[k].size();
    for (int f : g[k]) fields[p++] = f;
  }
  return 0;
}

int adha_plan_sections(const adha_schema* schema, const adha_section* sections, int32_t n_sec,
                       const adha_plan_opts* opts, adha_layout_set** out) {
  clear_error();
  if (int rc = check_schema(schema)) return rc;
  const int F = schema->n_fields;
  if (int rc = validate_sections(F, sections, n_sec)) return rc;
  if (!opts || !out) return fail(ADHA_EINVAL, "opts or out is NULL");
  if (opts->n_caps < 0 || (opts->n_caps > 0 && !opts->caps)) return fail(ADHA_EINVAL, "bad caps array");
  std::vector<Groups> layouts;
  std::map<Groups, int> seen;
  auto add = [&](const Groups& g) {
    if (seen.count(g)) return;
    seen[g] = (int)layouts.size();
    layouts.push_back(g);
  };
  if (opts->include_aos_soa) {
    Groups aos(1), soa;
    for (int f = 0; f < F; ++f) {
      aos[0].push_back(f);
      soa.push_back({f});
    }
    add(aos);
    add(soa);
  }
  const int W = opts->max_window <= 0 ? n_sec : std::min<int>(opts->max_window, n_sec);
  const int n_caps = opts->n_caps > 0 ? opts->n_caps : 1;
  for (int w = 1; w <= W; ++w)
    for (int k = 0; k + w <= n_sec; ++k)
      for (int c = 0; c < n_caps; ++c) add(ods_groups(F, schema->dtype, sections + k, w, opts->n_caps > 0 ? opts->caps[c] : 0));
  if (opts->max_candidates > 0 && (int)layouts.size() > opts->max_candidates) layouts.resize(opts->max_candidates);
  *out = pack_set(F, layouts);
  if (!*out) return fail(ADHA_ENOMEM, "host allocation of the layout set failed");
  return 0;
}

int adha_layout_set_create(int32_t n_fields, int32_t n_layouts, const adha_layout* layouts, adha_layout_set** out) {
  clear_error();
  if (!out || !layouts || n_layouts < 1 || n_fields < 1 || n_fields > kMaxFields)
    return fail(ADHA_EINVAL, "bad layout set arguments");
  std::vector<Groups> v;
  std::vector<int32_t> dummy(n_fields, ADHA_F32);
  adha_schema sc{n_fields, dummy.data()};
  for (int l = 0; l < n_layouts; ++l) {
    Layout L;
    if (int rc = make_layout(&sc, &layouts[l], &L, "candidate")) return rc;
    v.push_back(L.groups);
  }
  *out = pack_set(n_fields, v);
  if (!*out) return fail(ADHA_ENOMEM, "host allocation of the layout set failed");
  return 0;
}

int adha_pdl_solve(const adha_cost_table* costs, int32_t return_to_input, int32_t* layout_of_section, double* total_ns) {
  clear_error();
  if (!costs || !layout_of_section || !total_ns) return fail(ADHA_EINVAL, "NULL argument");
  if (costs->n_sections < 1 || costs->n_layouts < 1 || !costs->section_ns || !costs->remap_ns)
    return fail(ADHA_EINVAL, "empty cost table");
  return pdl_solve(costs, return_to_input, layout_of_section, total_ns);
}

int adha_pdl_solve_fused(const adha_cost_table* costs, int32_t return_to_input, int32_t max_window,
                         int32_t* layout_of_section, int32_t* window_len, double* total_ns) {
  clear_error();
  if (!costs || !layout_of_section || !window_len || !total_ns) return fail(ADHA_EINVAL, "NULL argument");
  if (costs->n_sections < 1 || costs->n_layouts < 1 || !costs->section_ns || !costs->remap_ns)
    return fail(ADHA_EINVAL, "empty cost table");
  if (max_window >= 2 && (costs->max_window < 2 || !costs->fused_ns))
    return fail(ADHA_EINVAL, "the cost table holds no fused runs (max_window %d)", costs->max_window);
  return pdl_solve_fused(costs, return_to_input, max_window, layout_of_section, window_len, total_ns);
}

int adha_cost_table_create_fused(int32_t n_sections, int32_t n_layouts, int32_t max_window, adha_cost_table** out) {
  clear_error();
  if (!out || n_sections < 1 || n_layouts < 1) return fail(ADHA_EINVAL, "bad cost table size");
  if (max_window < 0 || max_window > ADHA_MAX_FUSED) return fail(ADHA_EINVAL, "max_window %d not in [0, %d]", max_window, ADHA_MAX_FUSED);
  const int W = max_window >= 2 ? max_window : 0;
  const size_t ns = (size_t)n_sections * n_layouts, nr = (size_t)(n_layouts + 1) * (n_layouts + 1);
  const size_t nf = (size_t)n_sections * W * n_layouts;
  auto* t = static_cast<adha_cost_table*>(std::calloc(1, sizeof(adha_cost_table) + sizeof(double) * (ns + nr + nf)));
  if (!t) return fail(ADHA_ENOMEM, "host allocation of the cost table failed");
  t->n_sections = n_sections;
  t->n_layouts = n_layouts;
  t->section_ns = reinterpret_cast<double*>(t + 1);
  t->remap_ns = t->section_ns + ns;
  t->max_window = W;
  t->fused_ns = W ? t->remap_ns + nr : nullptr;
  for (size_t k = 0; k < nf; ++k) t->fused_ns[k] = HUGE_VAL;   // no fused run until measured
  *out = t;
  return 0;
}

int adha_cost_table_create(int32_t n_sections, int32_t n_layouts, adha_cost_table** out) {
  return adha_cost_table_create_fused(n_sections, n_layouts, 0, out);
}

}  // extern "C"

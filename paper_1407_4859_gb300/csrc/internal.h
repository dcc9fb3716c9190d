// internal.h -- host-side layout model, error state and kernel argument blocks of libadha.
//
// A layout (paper Section 2 and Table 2: fields combined into structures) is a list of groups;
// each group is an array of C structs of its fields in listed order, every field at its natural
// alignment, the struct size rounded up to its largest alignment.
#pragma once

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "device_types.h"

namespace adha {

constexpr int kMaxMoves = 256;         // moves (fields + padding pieces) over all built destination records
constexpr int kMaxStride = 4095;       // bytes per struct
constexpr int kSmemLimit = 227 * 1024; // dynamic shared memory one CTA may use
constexpr size_t kSmemPerSM = 228 * 1024;       // shared memory of one SM
constexpr size_t kSmemReservedPerCTA = 1024;    // taken by the system from it for every resident CTA

inline int dtype_size(int d) { return d == ADHA_F64 ? 8 : (d == ADHA_BF16 ? 2 : 4); }

// ------------------------------------------------------------------ errors
int fail(int code, const char* fmt, ...);   // records the message, returns code
int cuda_fail(int err, const char* what);   // ADHA_ECUDA with the runtime's text
void clear_error();

// ------------------------------------------------------------------ layouts
struct Layout {
  int F = 0;
  int dtype[kMaxFields] = {};
  int n_groups = 0;
  std::vector<std::vector<int>> groups;
  int stride[kMaxGroups] = {};
  int group_of[kMaxFields] = {};
  int offset_of[kMaxFields] = {};
};

// Struct size of a group and the offset of each listed field (natural alignment).
int group_struct(const int* dtype, const std::vector<int>& fields, std::vector<int>* offsets);

// Validates schema + layout and fills `out`; returns 0 or ADHA_EINVAL (message set).
int make_layout(const adha_schema* schema, const adha_layout* layout, Layout* out, const char* what);
int check_schema(const adha_schema* schema);
bool same_group(const Layout& a, int ga, const Layout& b, int gb);

int sm_count(int* count);

// ------------------------------------------------------------------ kernel argument blocks
// (GroupRef, FieldRef, SecOp and FusedArgs are in device_types.h.)

// One field of a destination record (or one aligned zero piece of its padding) and where its
// bytes come from.  Moves are 8, 4 or 2 bytes wide: a field moves whole, whatever the other
// fields' sizes.
struct Move {
  int16_t dst_group;    // index into RemapArgs::dst
  int16_t dst_off;      // byte offset in the destination struct
  int16_t src_group;    // index into RemapArgs::src; -1 for padding
  int16_t src_off;      // byte offset in the source struct
};

// Remap of one record array: every built destination group is assembled from the source groups'
// slices, one move per lane per step.  Moves fall into six classes: moves into one-field
// destination groups ("direct": stored straight to global memory, consecutive lanes on
// consecutive records) of 8, 4 and 2 bytes, then moves into wider groups ("staged": assembled in
// the warp's output buffer, written back with 16-byte stores) of 8, 4 and 2 bytes.  A direct
// destination group has start = -1 in `dst`; the staged ones have their output-buffer offset.
struct RemapArgs {
  int64_t n;              // records
  int64_t n_chunks;       // whole chunks of R records
  int32_t R;              // records per chunk
  int32_t n_src, n_dst;
  int32_t in_bytes;       // one chunk of the source slices
  int32_t out_bytes;      // one chunk of the destination slices
  int32_t n_moves;
  int32_t cls_count[6];   // moves per class, in that order in `move`
  int32_t cls_order[6];   // per class: schedule order (see schedule_pair)
  int32_t pieces;         // bit 0: stage through the per-CTA piece table, bit 1: write back through it
  int32_t buffers;        // input chunk buffers per warp: 2 (the next chunk staged during the moves) or 1
  GroupRef src[kMaxGroups];
  GroupRef dst[kMaxGroups];
  Move move[kMaxMoves];
};

struct SectionArgs {
  int64_t n;
  int64_t n_chunks;
  int32_t R;
  int32_t n_load, in_bytes;
  int32_t F;
  int32_t perm_slot;            // index of the staged perm slice (GATHER), else -1
  GroupRef load[kMaxGroups + 1];
  int8_t writeback[kMaxGroups + 1];   // staged slice k is written back whole after the chunk
  int32_t n_writeback;
  int32_t vec;                        // 1: every accessed group is one field wide; lane = M consecutive records
  int32_t buffers;                    // chunk buffers per warp: 2 (the next chunk staged during this one) or 1
  int32_t accumulate;                 // REDUCE: add into the result as it is (else it is zeroed first)
  int32_t reduce_walk;                // REDUCE: no feature in a one-field slice (sums cluster by cluster)
  FieldRef f[kMaxFields];
  float tanh_p[8], tanh_q[8];   // tanh polynomial coefficients (7 used each)
  const int32_t* perm;
  uint8_t* save;                // NULL or n elements of the written field's type
  SecOp s;
};

struct BackwardArgs {
  int64_t n;
  int32_t op;
  int32_t x, y, z;
  float a;
  uint8_t* s[3];   // state: field x, y, z at record 0
  int32_t ss[3];
  uint8_t* g[3];   // adjoints of x, y, z at record 0
  int32_t gs[3];
  const float* save;
  float tanh_p[8], tanh_q[8];
};

// Plan + launch helpers shared by the entry points, the measurer and the executor.
int remap_layouts(const Layout& S, const void* const* src_ptrs, const Layout& D, void* const* dst_ptrs, int64_t n,
                  void* stream, int* launched);
int run_section_layout(const Layout& L, void* const* ptrs, const adha_section* s, int64_t n, void* save,
                       void* stream);
// Sections s[0..m) fused into one pass (validated here).
int run_fused_layout(const Layout& L, void* const* ptrs, const adha_section* s, int m, int64_t n, void* stream);
std::string fused_tuning_key(const Layout& L, const adha_section* s, int m, int64_t n);
bool fusable_run(const Layout& L, const adha_section* s, int m);
// ADHA_EINVAL (message set) unless section s may run on n records stored in L.
int check_section_layout(const Layout& L, const adha_section* s, int64_t n);
void fill_secop(const Layout& L, const adha_section* s, SecOp* o);
// Copies the chunk-buffer offsets of the section's listed fields from the field table.
void fill_secop_offsets(SecOp* o, const FieldRef* f);
adha_layout set_layout(const adha_layout_set* s, int l);
// Remap launch arguments for one array (chunk_override 0 = the default chunk rule).
int remap_plan_args(const Layout& S, const void* const* src_ptrs, const Layout& D, void* const* dst_ptrs, int64_t n,
                    int chunk_override, int direct, RemapArgs* out, bool* empty);
// Runs fn(ctx) bracketed by the launch profiler's events when profiling is on.
int profiled_launch(int kind, int op, double bytes, void* stream, int (*fn)(const void*), const void* ctx);
// Autotuning: the key of a section launch, storing its best shape, thread-local overrides.
std::string tuning_key(const Layout& L, const adha_section* s, int64_t n, bool save);
void tuning_store(const std::string& key, int R, int wb);
void set_overrides(int R, int wb, int buffers = 0);
void set_fused_overrides(int R, int buffers);
void set_fused_jit(int mode);   // 0 as tuned, 1 library kernel, 2 specialised
// REDUCE sections launched later by the calling thread add into their result instead of zeroing it
// first (the host pipeline zeroes it once and reduces slice by slice).
void set_reduce_accumulate(bool on);
// One section as a one-section run specialised at run time with chunk shape (R, buffers), profiled
// as a section; ADHA_ENOTIMPL (nothing launched) where it cannot be.
int run_section_specialised_shape(const Layout& L, void* const* ptrs, const adha_section* s, int64_t n, int R,
                                  int buffers, void* stream);
int fused_jit_args(const Layout& L, const adha_section* s, int m, int64_t n, int chunk, int buffers, FusedArgs* out);
std::string remap_tuning_key(const Layout& S, const Layout& D, int64_t n);
void set_remap_pieces(int mode);
// ADHA_EINVAL unless every entry of the table is >= 0 or +inf (+inf: not measured or not allowed).
int check_costs(const adha_cost_table* c);
int pdl_solve(const adha_cost_table* c, int return_to_input, int32_t* seq, double* total);
int pdl_solve_fused(const adha_cost_table* c, int return_to_input, int max_window, int32_t* seq, int32_t* win,
                    double* total);

// tanh polynomial coefficients (Lambert's continued fraction cut after 25): 7 each, rounded once.
void tanh_coefficients(float p[8], float q[8]);

// Launchers (defined in the .cu files); all arguments already validated.
int launch_remap(const RemapArgs& a, int grid, size_t smem, void* stream);
size_t remap_smem_bytes(const RemapArgs& a);
int launch_section(const SectionArgs& a, int grid, size_t smem, void* stream);
size_t section_smem_bytes(const SectionArgs& a);
int launch_fused(const FusedArgs& a, int grid, size_t smem, void* stream);
// Fused runs specialised at run time (jit.cu): the kernel of run `a` (F fields; compiled and
// loaded here when `compile`, else only found in the cache), its occupancy and launch.
bool jit_available(std::string* why);
int jit_kernel(const FusedArgs& a, int F, int buffers, bool compile, const void** fn, std::string* why);
int jit_prepare(const std::vector<FusedArgs>& runs, const std::vector<int>& F, const std::vector<int>& buffers);
int jit_occupancy(const void* fn, size_t smem, int* blocks);
int launch_fused_jit(const void* fn, const FusedArgs& a, int grid, size_t smem, void* stream);
size_t jit_smem_bytes(const FusedArgs& a);
bool jit_source(const FusedArgs& a, int F, int buffers, std::string* src, std::string* why);
int jit_compile_only(const std::string& src);   // compile, no device needed, nothing loaded
std::string jit_last_log();
size_t fused_smem_bytes(const FusedArgs& a);
int fused_occupancy(int M, bool vec, bool km, size_t smem, int* blocks);
// Whether a fused run holds an assign or a reduce section (they have a kernel of their own).
inline bool fused_is_km(const FusedArgs& a) { return a.reduce_sec >= 0 || a.assign_sec >= 0; }
int launch_backward(const BackwardArgs& a, void* stream);
int remap_occupancy(int unit, size_t smem, int* blocks);
int section_occupancy(int op, size_t smem, int* blocks);

}  // namespace adha

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

#include "../../include/adha.h"

namespace adha {

constexpr int kMaxFields = ADHA_MAX_FIELDS;
constexpr int kMaxGroups = ADHA_MAX_FIELDS;
constexpr int kMaxSlots = 512;         // u-sized slots over all built destination records
constexpr int kMaxStride = 4095;       // bytes; fits the 12-bit stride field of a slot code
constexpr uint32_t kPadSlot = 0xFFFFFFFFu;
constexpr int kThreads = 256;          // threads per CTA of the staged kernels
constexpr int kSmemLimit = 227 * 1024; // dynamic shared memory one CTA may use

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

// Device address of the library's status word on the current device (set up on first use).
int status_word(int** ptr);
int sm_count(int* count);

// ------------------------------------------------------------------ kernel argument blocks
// Remap of one record array: every built destination group is assembled in shared memory from
// the source groups' tiles, one u-sized slot at a time.
struct RemapArgs {
  int64_t n;              // records
  int64_t n_full;         // whole tiles
  int32_t T;              // records per tile (multiple of 32)
  int32_t S;              // pipeline stages
  int32_t n_src, n_dst;
  int32_t stage_bytes;    // one stage: the source tiles, each region 128-byte aligned
  int32_t out_bytes;      // one output buffer: the destination tiles
  int32_t n_slots;
  int32_t pad_;
  const uint8_t* src[kMaxGroups];
  uint8_t* dst[kMaxGroups];
  int32_t s_stride[kMaxGroups];
  int32_t s_smem[kMaxGroups];
  int32_t d_stride[kMaxGroups];
  int32_t d_smem[kMaxGroups];
  int32_t d_nslot[kMaxGroups];
  int32_t d_slot0[kMaxGroups];
  int32_t d_q[kMaxGroups];     // kThreads / nslot
  int32_t d_rem[kMaxGroups];   // kThreads % nslot
  // slot code: (byte offset of the slot's source bytes for tile record 0 within a stage) |
  //            (source stride << 20); kPadSlot for padding
  uint32_t slot[kMaxSlots];
};

struct FieldRef {
  uint8_t* g;       // global address of the field in record 0
  int32_t gs;       // global stride (the group's struct size)
  int32_t s0;       // byte offset within a stage of the field in tile record 0, -1 if not staged
  int32_t ss;       // stride within the stage
  int32_t dtype;
};

struct SectionArgs {
  int64_t n;
  int64_t n_full;
  int32_t T, S;
  int32_t n_load, stage_bytes;
  int32_t F;
  int32_t op;
  uint64_t R, W;
  const uint8_t* lsrc[kMaxGroups];
  int32_t l_stride[kMaxGroups];
  int32_t l_smem[kMaxGroups];
  FieldRef f[kMaxFields];
  int32_t arg[8];
  float par[4];
  float tanh_p[8], tanh_q[8];   // tanh polynomial coefficients (7 used each)
  const int32_t* perm;
  uint8_t* save;                // NULL or n elements of the written field's type
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

// tanh polynomial coefficients (Lambert's continued fraction cut after 25): 7 each, rounded once.
void tanh_coefficients(float p[8], float q[8]);

// Launchers (defined in the .cu files); all arguments already validated.
int launch_remap(const RemapArgs& a, int unit, int grid, size_t smem, void* stream);
size_t remap_smem_bytes(const RemapArgs& a);
int launch_section(const SectionArgs& a, int grid, size_t smem, void* stream);
size_t section_smem_bytes(const SectionArgs& a);
int launch_backward(const BackwardArgs& a, void* stream);
int remap_occupancy(int unit, size_t smem, int* blocks);
int section_occupancy(int op, size_t smem, int* blocks);

}  // namespace adha

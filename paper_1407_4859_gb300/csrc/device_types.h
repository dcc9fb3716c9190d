// device_types.h -- the types and limits that device code shares with the host: the field and
// section tables of the staged kernels and the argument block of a fused run.  Compiled by nvcc
// with the library and, for fused windows specialised at run time, by the run-time compiler
// (which has no standard headers: it gets the fixed-width integer types here).
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
#include "adha.h"
#else
#include <cstdint>

#include "../../include/adha.h"
#endif

namespace adha {

constexpr int kMaxFields = ADHA_MAX_FIELDS;
constexpr int kMaxGroups = ADHA_MAX_FIELDS;
constexpr int kThreads = 256;          // threads per CTA of the staged kernels (8 warps)
constexpr int kWarps = kThreads / 32;

// Both staged kernels work per warp: a warp copies R consecutive records of every group it needs
// ("a chunk", R a multiple of 32) into its own shared buffer with 16-byte cp.async, double
// buffered, then works on the chunk.  Inside a buffer the groups' slices follow one another in
// the listed order; slice k starts at byte start[k] (16-byte aligned) and holds R*stride[k] bytes.
struct GroupRef {
  const uint8_t* ptr;     // group buffer
  int32_t stride;         // struct size
  int32_t start;          // slice offset within a chunk buffer
};

struct FieldRef {
  uint8_t* g;       // global address of the field in record 0
  int32_t gs;       // global stride (the group's struct size)
  int32_t s0;       // byte offset within a chunk buffer of the field in chunk record 0, -1 if not staged
  int32_t ss;       // stride within the chunk buffer
  int32_t dtype;
  int32_t wsm;      // 1: writes go into the chunk buffer and the whole slice is written back
};

// One section's operation and operands.  Read and written fields are listed by adha_dtype,
// ascending ids within a dtype: the fields of dtype d are rd[rd_off[d] .. rd_off[d + 1]).
struct SecOp {
  int32_t op;
  int32_t arg[8];
  float par[4];
  int8_t rd_off[5], wr_off[5];
  int8_t rd[kMaxFields];
  int8_t wr[kMaxFields];
  int16_t rd_s0[kMaxFields];   // chunk-buffer offset (FieldRef::s0) of each listed field, -1 if not staged
  int16_t wr_s0[kMaxFields];
  const void* aux;             // ASSIGN: centroids; REDUCE: the int64 sums
  int8_t gvec;                 // GATHER: px, py, pz, q share one 16-byte struct (one 16-byte load at perm[i])
  int8_t gidx[4];              // GATHER with gvec: the word of px, py, pz, q in that struct
};

constexpr int kMaxClusters = 8;   // K of the ASSIGN and REDUCE sections
constexpr int kMaxReduceFeatures = 32;

// A run of sections executed in one pass (the paper's combine): every group holding a field that a
// section of the run reads or writes is staged per chunk, the sections are applied in order on
// the chunk buffer, and groups with written fields go back whole.
constexpr int kMaxFused = ADHA_MAX_FUSED;
struct FusedArgs {
  int64_t n;
  int64_t n_chunks;
  int32_t R;
  int32_t n_load, in_bytes;
  int32_t perm_slot;            // index of the staged perm slice (a gather in the run), else -1
  int32_t n_sec;
  int32_t vec;                  // 1: every staged group is one field wide
  int32_t buffers;              // chunk buffers per warp (1 or 2)
  int32_t reduce_sec;           // index of the run's REDUCE section (at most one), else -1
  int32_t assign_sec;           // index of the run's first ASSIGN section (centroids staged per CTA), else -1
  int32_t accumulate;           // REDUCE: add into the result as it is (else it is zeroed before the launch)
  int32_t reduce_walk;          // REDUCE: no feature in a one-field slice (sums cluster by cluster)
  GroupRef load[kMaxGroups + 1];
  int8_t writeback[kMaxGroups + 1];
  FieldRef f[kMaxFields];
  float tanh_p[8], tanh_q[8];
  const int32_t* perm;
  SecOp sec[kMaxFused];
};

}  // namespace adha

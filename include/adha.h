/*
 * adha.h -- C ABI of libadha.so, a GB300 (sm_103a) implementation of the data
 * path of ADHA, the automatic data-layout framework of Majeti, Meel, Barik and
 * Sarkar ("ADHA: Automatic Data layout framework for Heterogeneous
 * Architectures", PACT 2014).
 *
 * Model (paper, Section 2 "Overall Framework"; Table 2):
 *   - A record array holds n records of F fields (F <= 64), each field of one
 *     of four types.  A *layout* splits the fields into ordered *groups*; each
 *     group is stored as its own array of C structs (fields in listed order,
 *     each at its natural alignment, struct size rounded up to the largest
 *     alignment).  AoS is one group of all fields; SoA is one group per field.
 *     Record i of group g starts at byte i * stride(g) of that group's buffer.
 *     Padding bytes written by this library are zero.
 *   - A *section* is one data-parallel loop over the records that reads and
 *     writes some fields of each record (the paper's section).
 *   - ODS picks a layout for a run of sections (affinity graph + greedy
 *     grouping); PDL picks one layout per section for the whole program by a
 *     shortest path whose edge weights are measured run and remap times.
 *
 * Conventions, for every entry point:
 *   - Return 0 (ADHA_OK) on success, a negative ADHA_E* code on failure; the
 *     calling thread's message is then in adha_last_error().  No C++ exception
 *     crosses this boundary.  Arguments are validated before anything is
 *     launched; a call that fails validation launches nothing.
 *   - "device pointer" means memory the GPU can read/write (cudaMalloc,
 *     PyTorch tensors); buffers are owned by the caller, must start on a
 *     16-byte boundary, and must not overlap unless stated.  The library
 *     allocates no device memory of its own: scratch comes from a caller
 *     workspace whose size a *_workspace_bytes call returns.
 *   - adha_stream is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that launch work are asynchronous on that stream unless stated.
 *   - Result objects the library returns (layout sets, cost tables) are
 *     allocated on the host and freed with adha_free.
 */
#ifndef ADHA_H_
#define ADHA_H_

#ifndef __CUDACC_RTC__   /* the run-time compiler of fused windows provides these types itself */
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef void* adha_stream;

enum {
  ADHA_OK = 0,
  ADHA_EINVAL = -1,   /* bad argument: the message names it                      */
  ADHA_ENOMEM = -2,   /* workspace too small, or host allocation failed          */
  ADHA_ECUDA = -3,    /* a CUDA runtime call failed: the message has its text    */
  ADHA_ETIMEOUT = -4, /* reserved for a bounded wait that ran out; no kernel here waits on anything */
  ADHA_ENOTIMPL = -5  /* not supported by the library or the device              */
};

#define ADHA_MAX_FIELDS 64
#define ADHA_MAX_SECTIONS 256
#define ADHA_MAX_FUSED 16      /* sections in one fused run (adha_run_sections_fused) */

typedef enum { ADHA_F32 = 0, ADHA_F64 = 1, ADHA_I32 = 2, ADHA_BF16 = 3 } adha_dtype;

/* n_fields fields; dtype[f] is an adha_dtype.  Host pointer, read during the call only. */
typedef struct {
  int32_t n_fields;
  const int32_t* dtype;
} adha_schema;

/* Groups in order; group g lists group_len[g] field ids, concatenated in `fields`.
 * Every field of the schema appears exactly once.  Host pointers. */
typedef struct {
  int32_t n_groups;
  const int32_t* group_len;
  const int32_t* fields;
} adha_layout;

/*
 * Section ops.  arg[] holds operand field ids and fparam[] fp32 constants.
 * Every floating-point operation is rounded to nearest on its own (no fused
 * multiply-add), in the order written:
 *   MADD3   (x,y,z):            z = x*y + z                                 fp32
 *   XORSHIFT(x,z):              z = x ^ (x >> 3), logical shift              int32
 *   ADD     (x,y,z):            z = x + y                                   fp32
 *   MIX     (masks only):       over the read set in ascending field order,
 *                               s = sum of fp32 fields, h = xor of int32 fields,
 *                               of both 32-bit halves of fp64 fields and of
 *                               bf16 bits; t = s + (h & 255) * 2^-8; then each
 *                               written field w: fp32 w*0.5 + t, fp64
 *                               w*0.5 + (double)t, int32 w ^ ((h ^ bits(t)) >> 3),
 *                               bf16 bits w ^ low16 of the same
 *   DRIFT   (px,py,pz,vx,vy,vz; dt):  p = p + dt*v, then p -= 1 if p >= 1, p += 1 if p < 0
 *   BIN     (px,py,pz,cell; G):  c = clamp((int)(p*G), 0, G-1) per axis,
 *                               cell = cx + G*(cy + G*cz)
 *   KE      (vx,vy,vz,m,e):     e = (double)((0.5*m) * ((vx*vx + vy*vy) + vz*vz))   (fp32 arithmetic)
 *   FLAGS   (fl,e; thr):         fl = ((fl << 1) | (e > thr)) & 255
 *   GATHER  (vx,vy,vz,px,py,pz,q; dt): j = perm[i]; v[i] = v[i] + (dt*q[j]) * (p[j] - 0.5)
 *   KICK    (vx,vy,vz,q; dt,Ex,Ey,Ez): v = v + (dt*q) * E
 *   AXPB    (x,z; a,b):          z = a*x + b          MUL (x,y,z): z = x*y
 *   TANH    (x,z):               z = adha tanh of x: Lambert's continued fraction
 *                               x/(1 + x^2/(3 + x^2/(5 + ...))) cut after the
 *                               partial denominator 25, written as x*Q(x^2)/P(x^2)
 *                               with P, Q its exact integer polynomials rounded
 *                               once to fp32 and evaluated by Horner's rule;
 *                               copysign(1, x) for |x| >= 9
 * The two K-Means-shaped sections (the paper's second benchmark, Section 3):
 * features x_0..x_{d-1} are the fp32 fields of read_mask in ascending id order,
 * arg[0] = the int32 membership field m, arg[1] = K (1..8 clusters):
 *   ASSIGN  (m, K; aux = K*d fp32 centroids c[k][j] = aux[k*d + j], device):
 *                               D_k = sum over j ascending of (x_j - c[k][j])^2
 *                               from +0 (fp32, each operation rounded);
 *                               m = the smallest k with the smallest D_k.
 *                               read_mask: features only (d >= 1); write_mask: m
 *   REDUCE  (m, K; aux = K*(d+1) int64 outputs, device, 8-byte aligned):
 *                               aux[k*(d+1)] = number of records with m = k,
 *                               aux[k*(d+1) + 1 + j] = sum over them of q(x_j),
 *                               q(x) = x * 2^23 rounded to the nearest integer
 *                               (ties to even), 2^31 - 1 / -2^31 beyond int32,
 *                               0 for NaN; records with m outside [0, K) are left
 *                               out.  Integer sums: the result is the same in any
 *                               record order.  aux is overwritten (the library
 *                               zeroes it first).  read_mask: features and m
 *                               (1 <= d <= 32); write_mask: none.  Not fusable.
 */
typedef enum {
  ADHA_OP_MADD3 = 1, ADHA_OP_XORSHIFT = 2, ADHA_OP_ADD = 3, ADHA_OP_MIX = 4, ADHA_OP_DRIFT = 5,
  ADHA_OP_BIN = 6, ADHA_OP_KE = 7, ADHA_OP_FLAGS = 8, ADHA_OP_GATHER = 9, ADHA_OP_KICK = 10,
  ADHA_OP_AXPB = 11, ADHA_OP_MUL = 12, ADHA_OP_TANH = 13, ADHA_OP_ASSIGN = 14, ADHA_OP_REDUCE = 15
} adha_op;

/*
 * One section (paper Section 2: a data-parallel loop with per-field accesses).
 * read_mask / write_mask: fields read / written at record i (bit f = field f);
 * read_at_perm_mask: fields read at record perm[i] (GATHER only).  The masks
 * must contain the op's operands; extra read bits declare reads the op does
 * not use (they still shape the affinity graph and what a section loads).
 * perm: device pointer to n int32 record ids in [0,n) (GATHER only, else NULL);
 * fields read through perm must not be written by the same section.
 * aux: device pointer to the op's table (ASSIGN: centroids, read) or result
 * (REDUCE: sums, written); NULL for the other ops.
 */
typedef struct {
  int32_t op;
  int32_t arg[8];
  float fparam[4];
  uint64_t read_mask;
  uint64_t write_mask;
  uint64_t read_at_perm_mask;
  const int32_t* perm;
  void* aux;
} adha_section;

/* ---------------------------------------------------------------- layouts */

/*
 * Byte stride of every group and byte offset of every field in its group
 * (the struct rule above).  stride[n_groups], offset[n_fields] are host
 * arrays the caller provides.  Host only.
 */
int adha_layout_strides(const adha_schema* schema, const adha_layout* layout, int32_t* stride,
                        int32_t* offset);

/*
 * Remap n records from layout src (group buffers src_ptrs[g], device) to
 * layout dst (dst_ptrs[g], device): the byte permutation that moves every
 * field of every record to its place in dst (paper Section 2, the remap edge;
 * Table 4, "remap").  A dst group identical to a src group (same fields in the
 * same order) whose pointer equals that src group's pointer is left alone (an
 * alias); otherwise dst buffers must not overlap src buffers.  Buffer g holds
 * n * stride(g) bytes.  Async on `stream`.
 */
int adha_remap(const adha_schema* schema, int64_t n, const adha_layout* src, const void* const* src_ptrs,
               const adha_layout* dst, void* const* dst_ptrs, adha_stream stream);

/*
 * Run one section in place on n records stored in `layout` (group buffers
 * ptrs[g], device).  save: NULL, or a device buffer of n elements of the
 * written field's type that receives the values the section overwrites
 * (AXPB, MUL, TANH only; used by adha_section_backward).  Async.
 */
int adha_run_section(const adha_schema* schema, int64_t n, const adha_layout* layout, void* const* ptrs,
                     const adha_section* section, void* save, adha_stream stream);

/*
 * Run sections[0..n_sec) in place on n records stored in `layout`, in one pass
 * (paper Section 2: the combine edge joins consecutive sections into one node):
 * per chunk of records, every group holding a field some section reads or
 * writes is staged once, the sections are applied in order, and groups with
 * written fields are written back whole.  The result equals running the
 * sections one after another with adha_run_section.  Requirements (EINVAL
 * otherwise): 1 <= n_sec <= ADHA_MAX_FUSED, each section valid alone, all
 * gathers of the run use the same perm, no section of the run writes a field
 * that a gather of the run reads through perm, and at most one REDUCE section.
 * A REDUCE in the run sums every record as the run's earlier sections left it
 * (its result is zeroed before the launch, as adha_run_section does).  Async on
 * `stream`.
 */
int adha_run_sections_fused(const adha_schema* schema, int64_t n, const adha_layout* layout, void* const* ptrs,
                            const adha_section* sections, int32_t n_sec, adha_stream stream);

/*
 * Reverse of one AXPB, MUL or TANH section for the chain gradient: restores
 * the overwritten field z from `save` (written by adha_run_section) in the
 * state buffers, then updates the adjoint buffers `grad_ptrs` (same layout,
 * fp32 fields, one adjoint per field):
 *   gz = g[z]; g[z] = 0;  AXPB: g[x] += a*gz;  MUL: g[x] += gz*y, then g[y] += gz*x;
 *   TANH: t = tanh(x); g[x] += gz*(1 - t*t)      (x, y: values before the section)
 * each operation rounded to nearest in fp32.  All fields must be fp32.  Async.
 */
int adha_section_backward(const adha_schema* schema, int64_t n, const adha_layout* layout,
                          void* const* state_ptrs, void* const* grad_ptrs, const adha_section* section,
                          const void* save, adha_stream stream);

/* ----------------------------------------------------------- planning (host) */

/* Options of candidate generation (ODS) and layout choice (PDL). */
typedef struct {
  int32_t n_caps;           /* struct-size limits (bytes) tried by ODS; a limit <= 0 means none    */
  const int32_t* caps;      /* n_caps limits (host); n_caps = 0 runs ODS once without a limit       */
  int32_t max_window;       /* ODS runs on every window of 1..max_window consecutive sections
                               (0 = every window length)                                            */
  int32_t include_aos_soa;  /* 1: the candidate list starts with AoS and SoA                        */
  int32_t max_candidates;   /* keep the first this many candidates (0 = all)                        */
  int32_t return_to_input;  /* PDL adds the remap back to the input layout after the last section  */
  int32_t fuse_window;      /* PDL may also run up to this many consecutive sections fused in one
                               layout (the combine node; needs a cost table measured with
                               ADHA_MEASURE_FUSE); <= 1: every section alone                         */
} adha_plan_opts;

/* A list of layouts over n_fields fields: layout l has n_groups[l] groups; its group
 * lengths are group_len[l*n_fields ...] and its fields, group after group,
 * fields[l*n_fields ...].  Host memory; library-made sets are freed with adha_free. */
typedef struct {
  int32_t n_fields;
  int32_t n_layouts;
  int32_t* n_groups;
  int32_t* group_len;
  int32_t* fields;
} adha_layout_set;

/* Measured costs in whole nanoseconds (stored as doubles, so sums are exact):
 * section_ns[k*n_layouts + l] = time of section k in candidate l;
 * remap_ns[a*(n_layouts+1) + b] = time of the remap from a to b, where index
 * n_layouts stands for the input layout and identical groups cost nothing;
 * with max_window >= 2, fused_ns[(k*max_window + m-1)*n_layouts + l] = time of
 * sections k..k+m-1 run fused in candidate l (2 <= m <= max_window; +inf where
 * the run may not be fused or was not measured; the m = 1 entries are unused).
 * Host memory, freed with adha_free. */
typedef struct {
  int32_t n_sections;
  int32_t n_layouts;
  double* section_ns;
  double* remap_ns;
  int32_t max_window;   /* 0: no fused runs (fused_ns NULL) */
  double* fused_ns;
} adha_cost_table;

/*
 * ODS of one run of sections (paper Section 2, "optimal data-layout of a
 * section"): builds the affinity graph whose nodes are the fields and whose
 * edge (a,b) weighs the number of sections accessing both (read, written or
 * read through perm), then merges clusters greedily along edges in order of
 * weight (descending; ties: smaller field id, then larger) while the merged
 * struct (fields ascending, natural alignment) is at most cap_bytes (<= 0: no
 * limit).  Fields the sections do not touch stay alone.  The result is
 * canonical: fields ascending in a group, groups ordered by their first field.
 * Outputs: *n_groups, group_len[<= n_fields], fields[n_fields] (host).  Host only.
 */
int adha_ods(const adha_schema* schema, const adha_section* sections, int32_t n_sec, int32_t cap_bytes,
             int32_t* n_groups, int32_t* group_len, int32_t* fields);

/*
 * Candidate layouts of a program: AoS and SoA (if asked), then the ODS layout
 * of every window of 1..max_window consecutive sections under every cap, in
 * that order (window length, start, cap), first occurrence kept.  *out is a
 * library-owned set (adha_free).  Host only.
 */
int adha_plan_sections(const adha_schema* schema, const adha_section* sections, int32_t n_sec,
                       const adha_plan_opts* opts, adha_layout_set** out);

/* A library-owned copy of n_layouts caller layouts (for example AoS and SoA only). */
int adha_layout_set_create(int32_t n_fields, int32_t n_layouts, const adha_layout* layouts, adha_layout_set** out);

/* A zeroed library-owned cost table of the given size (to fill by hand or in tests). */
int adha_cost_table_create(int32_t n_sections, int32_t n_layouts, adha_cost_table** out);

/* The same with room for fused runs of up to max_window (0, or 2..ADHA_MAX_FUSED)
 * sections, all +inf.  Host only. */
int adha_cost_table_create_fused(int32_t n_sections, int32_t n_layouts, int32_t max_window, adha_cost_table** out);

/*
 * PDL (paper Section 2, "program data-layout"): the shortest path through the
 * layered DAG input -> (section 1, l) -> ... -> (section S, l), node weight
 * section_ns, edge weight remap_ns (zero when the layout stays: the paper's
 * combine edge), plus the remap back to the input layout if return_to_input.
 * Ties go to the lexicographically smallest sequence of candidate indices.
 * Writes layout_of_section[n_sections] and the path cost.  Host only.
 */
int adha_pdl_solve(const adha_cost_table* costs, int32_t return_to_input, int32_t* layout_of_section,
                   double* total_ns);

/*
 * PDL with combine nodes (paper Section 2: consecutive sections joined into one
 * node of the DAG): besides every section alone, any run of 2..max_window
 * consecutive sections may be one node, run fused in one layout at the cost
 * fused_ns.  A path is a sequence of windows, each with a layout; its cost is
 * the sum of the remaps between consecutive windows' layouts (zero when the
 * layout stays), the windows' costs, and the remap back if return_to_input.
 * Ties go to the smaller layout index, then the longer window, window by window
 * from the first.  Writes layout_of_section[n_sections] (every section of a
 * window gets the window's layout), window_len[n_sections] (the window length at
 * the window's first section, 0 at the others) and the path cost.  max_window
 * <= 1 gives adha_pdl_solve's path with every window_len 1.  Host only.
 */
int adha_pdl_solve_fused(const adha_cost_table* costs, int32_t return_to_input, int32_t max_window,
                         int32_t* layout_of_section, int32_t* window_len, double* total_ns);

/*
 * PDL over a structured control-flow graph (paper Section 2: the rooted DAG is
 * built from the program's SCFG).  The program is a tree of regions, one node
 * each, children given by index:
 *   ADHA_SCFG_SECTION  section `section` (a row of the cost table)
 *   ADHA_SCFG_SEQ      its children in order (none: nothing runs)
 *   ADHA_SCFG_BRANCH   one child runs, child b with probability weights[b]
 *                      (>= 0, summing to 1); the children meet at a merge point
 *   ADHA_SCFG_LOOP     its one child runs `trips` >= 1 times (tested at its end)
 * A plan gives a layout to every section (a candidate, 0..n_layouts-1), to every
 * merge point and to every loop header (a candidate, or n_layouts = the input
 * layout: the layout the data is in when the branches meet / an iteration
 * starts).  Its cost is the expected time: every section and remap weighted by
 * how often it runs; each branch pays the remap from its last layout to the
 * merge point's; each iteration starts with the remap into the header's layout
 * (from the loop's entry layout the first time, from the body's last layout
 * after that).  The least expected cost is found by a dynamic program over the
 * tree (a matrix of costs entered in layout p and left in layout q per region:
 * min-plus products for sequences, weighted sums for branches, the best header
 * for loops); ties go to the smaller layout index.  Writes layout_of_node[i]
 * (-1 for SEQ nodes) and the expected cost.  Every node must be reached from
 * `root` exactly once (a tree) and n_nodes <= 4096; EINVAL otherwise.  Host only.
 */
enum { ADHA_SCFG_SECTION = 0, ADHA_SCFG_SEQ = 1, ADHA_SCFG_BRANCH = 2, ADHA_SCFG_LOOP = 3 };

typedef struct {
  int32_t kind;
  int32_t section;            /* SECTION: row of the cost table                          */
  int32_t n_children;         /* SEQ: >= 0; BRANCH: >= 1; LOOP: 1; SECTION: 0          */
  const int32_t* children;    /* node indices (host)                                     */
  const double* weights;      /* BRANCH: n_children probabilities (host)                 */
  double trips;               /* LOOP: expected iterations, >= 1                          */
} adha_scfg_node;

int adha_pdl_solve_scfg(const adha_cost_table* costs, int32_t n_nodes, const adha_scfg_node* nodes, int32_t root,
                        int32_t return_to_input, int32_t* layout_of_node, double* total_ns);

/*
 * PDL with the device as a second dimension (paper Section 2 and Table 4: the
 * tuning profile covers every device, and the plan maps each section to a
 * device as well as a layout, e.g. CPU-ODS(1-3) remap GPU-ODS(4-7)).  costs[d]
 * is device d's table (same sections and candidates on every device; remap_ns
 * between layouts on that device, index n_layouts = the input layout);
 * transfer_ns[(a*n_devices + b)*(n_layouts+1) + l] is the time to move the data,
 * in layout l (n_layouts: the input layout), from device a to device b.  A plan
 * gives each section a (layout, device); consecutive sections on one device pay
 * that device's remap, across devices the cheaper of remapping on the source and
 * then moving, or moving and then remapping on the destination.  The input is
 * in the input layout on input_device (also where return_to_input goes back
 * to).  Shortest path over the (layout, device) states, state index
 * device*n_layouts + layout, ties to the smaller index.  The library runs
 * sections on its GPU only: this call plans; costs for other devices come from
 * the caller.  1 <= n_devices <= 8.  Host only.
 */
int adha_pdl_solve_devices(int32_t n_devices, const adha_cost_table* const* costs, const double* transfer_ns,
                           int32_t input_device, int32_t return_to_input, int32_t* layout_of_section,
                           int32_t* device_of_section, double* total_ns);

/* ----------------------------------------------------------- measure and run */

/* A program's layout plan and where its result ended up. */
typedef struct {
  int32_t fixed;                                  /* in: 1 = run layout_of_section as given; 0 = solve PDL */
  int32_t n_sections;                             /* out */
  int32_t layout_of_section[ADHA_MAX_SECTIONS];   /* in when fixed, else out: candidate per section */
  double model_ns;                                /* out: sum of the cost-table entries on the path (0 without a table) */
  int32_t n_remaps;                               /* out: layout changes performed */
  int32_t n_launches;                             /* out: kernels launched */
  int32_t final_layout;                           /* out: candidate equal to the result's layout, -1 if none */
  int32_t final_n_groups;                         /* out: groups of the result's layout */
  void* final_ptrs[ADHA_MAX_FIELDS];              /* out: device buffers of the result's groups */
  int32_t window_len[ADHA_MAX_SECTIONS];          /* out (in when fixed): sections run fused from section k
                                                     (0 inside a window); all 0 when fixed = each alone */
} adha_plan;

/* adha_measure flags. */
#define ADHA_MEASURE_AUTOTUNE 1   /* time every section launch shape, keep the fastest for later launches */
#define ADHA_MEASURE_FUSE(w) ((int32_t)(w) << 8)   /* also time every fusable run of 2..w sections (w <= 16) */
#define ADHA_MEASURE_DIFFERENTIABLE 2   /* costs of a forward + backward step (see adha_measure) */

/* Workspace bytes adha_measure needs: two copies of the widest candidate (or input) layout. */
size_t adha_measure_workspace_bytes(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                                    const adha_layout_set* candidates);

/* The same for given adha_measure flags: with ADHA_MEASURE_DIFFERENTIABLE, three
 * copies plus n floats (the gradients and one section's saved values). */
size_t adha_measure_workspace_bytes_for(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                                        const adha_layout_set* candidates, int32_t flags);

/*
 * The tuning profile of PDL (paper Section 2: execution times measured per
 * section and device): times every section in every candidate layout and every
 * remap between two candidates (and from / to the input layout) on the
 * caller's data: the input (layout in_layout, device buffers in_ptrs) is first
 * copied into the workspace, so it is not modified.  Each entry is one warm-up
 * call, then the faster of two batches of `reps` calls timed with CUDA events
 * on `stream`, in whole nanoseconds.  A remap between layouts sharing a group
 * leaves that group in place, as the executor does.  With ADHA_MEASURE_AUTOTUNE
 * in flags each section is timed under every launch shape (records per chunk
 * 32, 64, 128 x field-wise or whole-group stores), and each remap from or to
 * the input layout under every choice of piece tables and chunk buffers (adha_tune_remap_pieces),
 * then under chunks of 24 to 128 records with the best of those choices;
 * the fastest enters the table and the library's tuning cache, which later
 * launches of the same section (or pair of layouts), layout and size class use.
 * With ADHA_MEASURE_DIFFERENTIABLE (fp32 schemas whose sections are all axpb,
 * mul or tanh) the table prices a forward + backward step instead: a section
 * costs its forward launch with the overwritten values saved plus its adjoint
 * kernel (adha_section_backward) in that layout, and a remap edge costs the
 * remap plus its inverse (the gradients travel back through it), so
 * remap_ns[a][b] = remap_ns[b][a]; fused runs are not timed then.
 * Synchronizes `stream`; *out is a library-owned table (adha_free).
 */
int adha_measure(const adha_schema* schema, int64_t n, const adha_layout* in_layout, void* const* in_ptrs,
                 const adha_section* sections, int32_t n_sec, const adha_layout_set* candidates, int32_t reps,
                 int32_t flags, void* workspace, size_t ws_bytes, adha_stream stream, adha_cost_table** out);

/* Workspace bytes adha_run_program needs: three copies of the widest candidate layout. */
size_t adha_program_workspace_bytes(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                                    const adha_layout_set* candidates);

/*
 * Runs a program (paper Section 2 and Table 4): picks one candidate layout per
 * section by PDL on `costs` (unless plan->fixed), then enqueues on `stream`, in
 * order, the remap into each section's layout when it differs from the current
 * one and the section itself, in place.  The data start in in_layout / in_ptrs
 * (device); groups shared by consecutive layouts stay where they are (so input
 * buffers are updated in place while their group survives); other groups are
 * placed in the workspace (device, ws_bytes from adha_program_workspace_bytes).
 * With opts->return_to_input the result is remapped back into in_ptrs.  The
 * result's buffers are listed in plan->final_ptrs.  Asynchronous; no device
 * memory is allocated and nothing synchronizes, so the call can be captured in
 * a CUDA graph.
 */
int adha_run_program(const adha_schema* schema, int64_t n, const adha_layout* in_layout, void* const* in_ptrs,
                     const adha_section* sections, int32_t n_sec, const adha_layout_set* candidates,
                     const adha_cost_table* costs, const adha_plan_opts* opts, void* workspace, size_t ws_bytes,
                     adha_stream stream, adha_plan* plan);

/* Device workspace bytes adha_run_program_host needs for n records cut into n_slices slices:
 * three buffer sets, each an input slice plus three copies of the widest candidate layout. */
size_t adha_program_host_workspace_bytes(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                                         const adha_layout_set* candidates, int32_t n_slices);

/*
 * adha_run_program on host-resident records: host_in (n records in in_layout;
 * pinned host memory lets the copies run asynchronously) is processed in
 * n_slices slices of consecutive records that flow through three streams of
 * the library's own (upload, program, download; chained by events over three
 * buffer sets), so copies in both directions and kernels overlap.  The plan is solved once (or taken as fixed) before any data
 * moves; the result is written in the plan's final layout (the last section's
 * candidate, or in_layout with opts->return_to_input), host_out[g] holding
 * n * stride(g) bytes.  Sections that read through a permutation need every
 * record: with one of those n_slices must be 1.  A REDUCE section's result is
 * zeroed once and every slice adds its records' sums into it (exact integer
 * sums, so the total is the one of a single pass).  The workspace (device,
 * adha_program_host_workspace_bytes) must not be used by anything else until
 * the work is done.  Asynchronous with respect to `stream`: the pipelines wait
 * for work queued on `stream` before they start, and `stream` waits for them
 * to finish.  plan->final_ptrs lists host_out.
 */
int adha_run_program_host(const adha_schema* schema, int64_t n, const adha_layout* in_layout,
                          const void* const* host_in, const adha_section* sections, int32_t n_sec,
                          const adha_layout_set* candidates, const adha_cost_table* costs, const adha_plan_opts* opts,
                          void* const* host_out, int32_t n_slices, void* workspace, size_t ws_bytes, adha_stream stream,
                          adha_plan* plan);

/* ----------------------------------------------------------- batched remap */

/* One record array of a batched remap: its own schema, record count, and
 * source / destination layouts with their group buffers (device).  Host structs,
 * read during adha_batched_create only. */
typedef struct {
  const adha_schema* schema;
  int64_t n;
  const adha_layout* src;
  const void* const* src_ptrs;
  const adha_layout* dst;
  void* const* dst_ptrs;
} adha_remap_desc;

/* A prepared batched remap (host object). */
typedef struct adha_batched adha_batched;

#define ADHA_BATCHED_AUTOTUNE 1   /* pick each array's launch shape by timing it (synchronizes `stream`) */
#define ADHA_BATCHED_TWO_BUFFERS 2   /* two input chunk buffers per warp (the next chunk staged during the moves) */
#define ADHA_BATCHED_CTAS(k) ((int32_t)(k) << 4)   /* force k CTAs per SM (1..8) instead of the model's choice */

/*
 * Prepares the remap of n_arrays record arrays in one persistent launch (the
 * batching form of the paper's remap, Section 2): validates every array (rules
 * of adha_remap), plans each one (chunk size, element schedule) and lays out
 * the descriptors the kernel reads.  The kernel's warps work alone: each takes
 * work units of about 1024 records of one array by an atomic ticket (largest
 * array first) and keeps its current array's tables in its own region of
 * shared memory.  The region is set here: the number of CTAs per SM (1 to 8,
 * as registers allow) whose regions hold every array's chunk buffers (chunks
 * shortened to fit, down to 8 records) with the most bytes x CTAs, discounting
 * arrays whose chunks had to shrink (ADHA_BATCHED_CTAS(k) in flags forces k).
 * A warp has one input chunk buffer and stages its next chunk once the moves
 * have read the current one (longer chunks in the same shared memory, measured
 * faster on the 256-array workload); ADHA_BATCHED_TWO_BUFFERS gives it two, the
 * next chunk staged while the current one is moved.  With
 * ADHA_BATCHED_AUTOTUNE each array's chunk size (32..256 records) and store
 * mode for one-field destination groups (see adha_tune_remap_direct) are the
 * fastest pair, timed with the single-array kernel on the array's own buffers
 * (their contents are overwritten with the remap's result).  *out is freed with
 * adha_batched_destroy.  Needs a current CUDA device (occupancy queries).
 */
int adha_batched_create(int32_t n_arrays, const adha_remap_desc* descs, int32_t flags, adha_stream stream,
                        adha_batched** out);

/* What adha_batched_create chose: CTAs per SM, shared bytes per warp, work units
 * per launch (any output may be NULL).  Host only. */
int adha_batched_info(const adha_batched* b, int32_t* ctas_per_sm, int32_t* warp_region_bytes, int64_t* units);

/* Device workspace bytes the batched remap needs (descriptors + its work ticket). */
size_t adha_batched_workspace_bytes(const adha_batched* b);

/* Copies the descriptors into `workspace` (device, 256-byte aligned) and
 * synchronizes `stream`.  Needed once per workspace before launches. */
int adha_batched_upload(const adha_batched* b, void* workspace, size_t ws_bytes, adha_stream stream);

/* Enqueues the batched remap: zeroes the work ticket, then one persistent
 * kernel in which CTAs take blocks of chunks by atomic ticket.  Async; no
 * allocation or synchronization, so it can be captured in a CUDA graph.  The
 * workspace must hold uploaded descriptors and not be shared by overlapping
 * launches. */
int adha_batched_launch(const adha_batched* b, void* workspace, adha_stream stream);

/* Captures adha_batched_launch into a CUDA graph owned by b (on a private
 * stream; `stream` is synchronized first).  Replaces an earlier graph of b. */
int adha_batched_graph(adha_batched* b, void* workspace, adha_stream stream);

/* Launches the captured graph on `stream` (async). */
int adha_batched_graph_launch(const adha_batched* b, adha_stream stream);

/* Algorithmic bytes one launch moves: 2 x data bytes of every field in a changed group. */
double adha_batched_bytes(const adha_batched* b);

/* Frees b and its graph (NULL is ignored). */
void adha_batched_destroy(adha_batched* b);

/*
 * Device workspace bytes adha_remap_batched needs for this batch (descriptors,
 * element schedules and the work ticket), planned by the default rules of
 * adha_batched_create; *bytes receives it.  Validates the batch like
 * adha_remap_batched.  Needs the current CUDA device; host only.
 */
int adha_workspace_bytes(int32_t n_arrays, const adha_remap_desc* descs, size_t* bytes);

/*
 * The batched remap in one call (paper Section 2, the remap edge, applied to
 * many record arrays at once): validates and plans the batch as
 * adha_batched_create does without autotuning, copies the descriptors into
 * `workspace` (device, 256-byte aligned, ws_bytes >= adha_workspace_bytes of
 * the same batch; ADHA_ENOMEM otherwise), zeroes the work ticket and enqueues
 * the persistent kernel on `stream`.  Rules of adha_remap per array.  The
 * descriptors are copied from a host buffer the call frees before returning,
 * so a stream that is being captured is rejected with ADHA_EINVAL (capture
 * adha_batched_launch, whose workspace is uploaded beforehand, instead).
 * Asynchronous; the workspace must not be reused until the remap is done.
 */
int adha_remap_batched(int32_t n_arrays, const adha_remap_desc* descs, void* workspace, size_t ws_bytes,
                       adha_stream stream);

/* Bytes of the device array that adha_remap_batched_noalloc keeps its descriptors in. */
#define ADHA_NOALLOC_SCRATCH_BYTES (1u << 20)

/*
 * The batched remap for callers that cannot allocate device memory: code
 * running where cudaMalloc is not allowed (inside someone else's memory pool or
 * allocator accounting, or a plugin given only its input and output buffers)
 * cannot provide the workspace adha_batched_upload needs.  This entry point
 * keeps the descriptors and the work ticket in a fixed device array inside the
 * library (ADHA_NOALLOC_SCRATCH_BYTES, held on every GPU that loads the library
 * until the process exits) and calls no device-allocating routine.  The caller
 * still passes every input and output buffer in `descs` (rules of adha_remap).
 * A batch whose descriptors do not fit fails with ADHA_EINVAL, as does a call
 * on a stream that is being captured (the descriptors are copied from a host
 * buffer freed on return).  Each call rewrites the descriptors and zeroes the
 * ticket, then launches the kernel on `stream` (async); calls from several host
 * threads reach the GPU one whole call at a time, but all calls share the one
 * array, so calls that overlap on the GPU (different streams, unordered) race
 * and must be ordered by the caller.  The first call on a device looks up the
 * array's device address and keeps it for the process; make that first call
 * before any stream capture, and do not call again after cudaDeviceReset (the
 * kept address does not survive it).  The paper has no counterpart of this
 * entry point.
 */
int adha_remap_batched_noalloc(int32_t n_arrays, const adha_remap_desc* descs, adha_stream stream);

/*
 * Records per warp chunk (a multiple of 8 up to 1024; 0 = automatic) that the
 * remap kernels launched later by the calling thread use; section kernels take
 * it rounded to 32, 64 or 128.  The autotuner sets it while it times
 * candidates.  Host only.
 */
int adha_tune_override(int32_t chunk_records);

/*
 * How section kernels launched later by the calling thread store into staged
 * groups wider than 8 bytes: 0 = automatic (a group whose written fields make
 * up at least a quarter of its struct is updated in shared memory and written
 * back whole with 16-byte stores; other written fields are stored one by one),
 * 1 = always field by field, 2 = always whole.  Host only.
 */
int adha_tune_writeback(int32_t mode);

/*
 * Chunk buffers per warp of section kernels launched later by the calling
 * thread: 0 = as tuned (adha_measure with ADHA_MEASURE_AUTOTUNE), else 2;
 * 2 = the next chunk is staged while one is computed; 1 = one buffer (half the
 * shared memory, so more CTAs per SM; the next chunk is staged after this one).
 * Every choice computes the same bytes.  Host only; EINVAL for another value.
 */
int adha_tune_section_buffers(int32_t buffers);

/*
 * Fused runs specialised at run time (paper Section 2, the combine edge: one
 * pass over the records for a run of sections).  The library's fused kernel
 * looks fields and operands up in tables at run time; a specialised run is the
 * same pipeline compiled for this one run (chunk shape, slice offsets, field
 * types and section operands as constants, each record's fields in registers
 * across the run's sections) with the CUDA run-time compiler for sm_103a,
 * loaded once and cached for the process.  Both compute the same bytes.
 *
 * adha_tune_fused_jit: how fused runs launched later by the calling thread
 * choose: 0 = as tuned (adha_measure with ADHA_MEASURE_AUTOTUNE times both and
 * keeps the faster), 1 = always the library's kernel, 2 = always specialised
 * (a run that cannot be, e.g. one with an ASSIGN section, then fails with
 * ADHA_ENOTIMPL and the reason).  A run first met while its stream is being
 * captured is not compiled then: it takes the library's kernel (mode 0) or
 * fails with ADHA_ENOTIMPL (mode 2).  Compiling takes a fraction of a second
 * per run; adha_measure compiles the runs it times in parallel host threads.
 * EINVAL for another mode.
 *
 * adha_jit_available: 1 if the run-time compiler (libnvrtc) could be loaded,
 * else 0 with the reason as the error message.
 *
 * adha_jit_log: the last compile's log (the compiler's messages and the
 * register and shared-memory report of the kernel), NUL-terminated into
 * buf[0..cap) when buf is not NULL; *len (if not NULL) gets its full length.
 */
int adha_tune_fused_jit(int32_t mode);

/*
 * How sections launched later by the calling thread (adha_run_section and the
 * executor; not those with a save buffer) choose their kernel: 0 = as tuned
 * (adha_measure with ADHA_MEASURE_AUTOTUNE also times each section as a
 * one-section run specialised at run time, in the layouts where the library's
 * kernel does best, and keeps the faster), 1 = always the library's section
 * kernel, 2 = specialised wherever the section can be (else the library's
 * kernel).  Both compute the same bytes.  EINVAL for another mode.
 */
int adha_tune_section_jit(int32_t mode);

/*
 * Chunk buffers per warp of fused runs launched later by the calling thread:
 * 0 = as tuned, else one (the default); 1 or 2.  Host only; EINVAL otherwise.
 */
int adha_tune_fused_buffers(int32_t buffers);

/*
 * The specialised kernel of the fused run sections[0..n_sec) on n records in
 * `layout` (validated like adha_run_sections_fused; chunk_records 0 = the
 * library's rule, else 32, 64 or 128; buffers 0 = the default, else 1 or 2):
 * its CUDA source (NUL-terminated into src[0..cap) when src is not NULL; *len,
 * if not NULL, gets the full length, also on failure after planning), compiled
 * for sm_103a (no device needed) and, when load != 0, loaded into the process's
 * cache so that later launches of the run (mode 2, or as tuned) skip the
 * compile.  ADHA_ENOTIMPL if the run cannot be specialised or the run-time
 * compiler is missing; ADHA_ECUDA with the compiler's log if it fails.
 */
int adha_fused_jit_build(const adha_schema* schema, int64_t n, const adha_layout* layout, const adha_section* sections,
                         int32_t n_sec, int32_t chunk_records, int32_t buffers, int32_t load, char* src, size_t cap,
                         size_t* len);
int adha_jit_available(void);
int adha_jit_log(char* buf, size_t cap, size_t* len);

/*
 * How remaps launched later by the calling thread store one-field destination
 * groups: 0 = through the warp's output buffer with 16-byte stores (default),
 * 1 = straight from the move loop to global memory (less shared memory, more
 * store instructions).  The batched autotuner tries both per array.  Host only.
 */
int adha_tune_remap_direct(int32_t mode);

/*
 * How remaps launched later by the calling thread find where each 16-byte piece
 * of a chunk buffer lives in global memory (through a per-block table of the
 * pieces, or by a search over the groups) and how many input chunk buffers a
 * warp has.  0 = as tuned for the pair of layouts (adha_measure with
 * ADHA_MEASURE_AUTOTUNE), else automatic (the table for a buffer whose slices
 * average under 256 bytes; two buffers); 1..8 = forced, with bits mode - 1:
 * bit 0 = stage the source buffer through the table, bit 1 = write the
 * destination buffer back through it, bit 2 = one input buffer (the next chunk
 * staged once the moves have read the current one) instead of two.  Every mode
 * moves the same bytes.  Host only; EINVAL for another mode.
 */
int adha_tune_remap_pieces(int32_t mode);

/* Empties the library's tuning cache (process-wide).  Host only. */
int adha_tune_clear(void);

/* Writes the tuning cache as text ("key<TAB>records<TAB>mode" lines; section
 * keys start with S, remap keys with M and carry records 0 and the piece-table
 * bits as mode) into buf
 * (len bytes, NUL-terminated); *needed = bytes required.  buf may be NULL to
 * ask for the size.  Host only. */
int adha_tune_export(char* buf, size_t len, size_t* needed);

/* Adds the entries of a text made by adha_tune_export to the cache.  Host only. */
int adha_tune_import(const char* text);

/*
 * Random-access read microbenchmark, the roofline of the gather section (whose
 * reads land on permuted records, where a copy's bandwidth does not apply):
 * out[i] = table[perm[i]] for i in [0, n), elements of rec_bytes (4, 8 or 16)
 * bytes; perm holds n int32 indices into table (device), out n elements
 * (device, not overlapping table).  The permutation is read and out written in
 * order.  Algorithmic bytes per element: 4 + 2 * rec_bytes.  Async on `stream`.
 * A measuring tool: the paper has no counterpart.
 */
int adha_gather_probe(const void* table, const int32_t* perm, void* out, int64_t n, int32_t rec_bytes,
                      adha_stream stream);

/* One kernel launch seen by the profiler.  kind: 0 remap, 1 section, 2 section
 * backward, 3 batched remap, 4 fused run, 5 gather probe, 6 section run as a
 * one-section run specialised at run time; op: the section's
 * adha_op (0 for remaps; the number of sections for a fused run; the element
 * bytes for the probe); bytes:
 * the algorithmic bytes the launch had to move (data bytes of the moved or
 * accessed fields, not padding or untouched fields); ms: its duration between
 * two CUDA events recorded around it on its stream. */
typedef struct {
  int32_t kind;
  int32_t op;
  double bytes;
  double ms;
} adha_launch_record;

/* Starts recording every kernel launched through this library by any host
 * thread of the process (up to max_records; events are created once and
 * reused).  Host only. */
int adha_profile_start(int32_t max_records);

/* Stops recording, waits for the recorded launches and copies up to
 * max_records of them to out; *n_records = how many were recorded. */
int adha_profile_stop(adha_launch_record* out, int32_t max_records, int32_t* n_records);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* adha_last_error(void);

/* Frees a host object returned by this library (NULL is ignored). */
void adha_free(void* p);

/* Library version string. */
const char* adha_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ADHA_H_ */

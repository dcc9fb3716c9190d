/*
 * adha_oracle.c -- CPU oracle of the ADHA data path.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this file's library.  It shares no code, header or constant with the CUDA
 * path.  Everything is plain scalar C, one record and one field at a time, with
 * every floating-point operation written separately so that it is rounded to
 * nearest on its own (built with -O2 -ffp-contract=off -fno-fast-math: no
 * fused multiply-add, no reassociation, IEEE division).
 *
 * Paper: D. Majeti, K. S. Meel, R. Barik, V. Sarkar, "ADHA: Automatic Data
 * layout framework for Heterogeneous Architectures", PACT 2014.
 *   - Section 2 ("Overall Framework"): fields grouped into structures by the
 *     ODS pass; a remap moves the data of one section's layout into the next.
 *   - Table 2: layouts are ordered lists of field groups (AoS, SoA, hybrids).
 * The paper prints no formulas for the data path; the readings used here are:
 *   - a group is a C struct of its fields in listed order, each field at its
 *     natural alignment (its size), the struct size rounded up to its largest
 *     alignment; padding bytes hold zero;
 *   - a remap is the byte permutation that moves every field of every record
 *     from its place in the source layout to its place in the target layout;
 *   - section results do not depend on the layout, so sections run here on one
 *     plain array per field ("field arrays").
 */
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#include <math.h>

enum { D_F32 = 0, D_F64 = 1, D_I32 = 2, D_BF16 = 3 };

static int dsize(int d) { return d == D_F64 ? 8 : (d == D_BF16 ? 2 : 4); }

/* ---------------------------------------------------------------- layouts */

/*
 * Struct layout of one group (Section 2: "combine the fields in structures"):
 * writes each listed field's byte offset to off[j] and returns the struct size.
 */
int oracle_group_layout(const int* dtypes, const int* fields, int len, int* off) {
  int o = 0, maxal = 1;
  for (int j = 0; j < len; ++j) {
    int s = dsize(dtypes[fields[j]]);
    if (o % s != 0) o += s - o % s;
    off[j] = o;
    o += s;
    if (s > maxal) maxal = s;
  }
  if (o % maxal != 0) o += maxal - o % maxal;
  return o;
}

/*
 * Per-field placement of a whole layout: group_of[f], offset_of[f] and the
 * stride of every group.  Returns 0, or -1 when the groups do not hold every
 * field exactly once.
 */
int oracle_layout_info(int F, const int* dtypes, int n_groups, const int* group_len, const int* fields,
                       int* stride, int* group_of, int* offset_of) {
  int seen[64];
  int off[64];
  if (F < 1 || F > 64) return -1;
  for (int f = 0; f < F; ++f) seen[f] = 0;
  int p = 0;
  for (int g = 0; g < n_groups; ++g) {
    if (group_len[g] < 1 || p + group_len[g] > F) return -1;
    for (int j = 0; j < group_len[g]; ++j) {
      int f = fields[p + j];
      if (f < 0 || f >= F || seen[f]) return -1;
      seen[f] = 1;
    }
    stride[g] = oracle_group_layout(dtypes, fields + p, group_len[g], off);
    for (int j = 0; j < group_len[g]; ++j) {
      group_of[fields[p + j]] = g;
      offset_of[fields[p + j]] = off[j];
    }
    p += group_len[g];
  }
  return p == F ? 0 : -1;
}

/*
 * Remap n records from layout src to layout dst (Section 2, the "remap" edge):
 * every field of every record is copied byte for byte to its new place, one
 * field of one record at a time; dst padding bytes are set to zero.
 */
int oracle_remap(int64_t n, int F, const int* dtypes,
                 int src_ng, const int* src_len, const int* src_fields, uint8_t* const* src,
                 int dst_ng, const int* dst_len, const int* dst_fields, uint8_t* const* dst) {
  int s_stride[64], s_group[64], s_off[64], d_stride[64], d_group[64], d_off[64];
  if (oracle_layout_info(F, dtypes, src_ng, src_len, src_fields, s_stride, s_group, s_off)) return -1;
  if (oracle_layout_info(F, dtypes, dst_ng, dst_len, dst_fields, d_stride, d_group, d_off)) return -1;
  for (int g = 0; g < dst_ng; ++g) memset(dst[g], 0, (size_t)n * (size_t)d_stride[g]);
  for (int64_t i = 0; i < n; ++i) {
    for (int f = 0; f < F; ++f) {
      const uint8_t* from = src[s_group[f]] + i * s_stride[s_group[f]] + s_off[f];
      uint8_t* to = dst[d_group[f]] + i * d_stride[d_group[f]] + d_off[f];
      memcpy(to, from, (size_t)dsize(dtypes[f]));
    }
  }
  return 0;
}

/* ------------------------------------------------------------ tanh */

/*
 * Project tanh: Lambert's continued fraction
 *     tanh x = x / (1 + x^2 / (3 + x^2 / (5 + x^2 / ...)))
 * cut after the partial denominator 2K+1 (K = 12).  With a = x^2, the cut
 * denominator D_K = 1 + a/(3 + a/(... + a/(2K+1))) equals P_K(a) / Q_K(a), where
 * P and Q follow the fundamental recurrences of continued fractions
 *     P_k = (2k+1) P_{k-1} + a P_{k-2},  P_{-1} = 1, P_0 = 1,
 *     Q_k = (2k+1) Q_{k-1} + a Q_{k-2},  Q_{-1} = 0, Q_0 = 1,
 * so tanh x ~= x Q_K(a) / P_K(a).  The polynomial coefficients are exact
 * integers (below 2^53), built here in int64 and rounded once to fp32; the
 * polynomials are evaluated by Horner's rule in fp32, each operation rounded
 * to nearest, then one multiply and one IEEE division.  For |x| >= 9 the value
 * is copysign(1, x) (tanh 9 rounds to 1 in fp32).
 */
#define TANH_K 12
static float tP[TANH_K + 1], tQ[TANH_K + 1];
static int tP_n, tQ_n, t_ready;

static void tanh_coeffs(void) {
  int64_t Pm[TANH_K + 2] = {0}, P[TANH_K + 2] = {0}, Qm[TANH_K + 2] = {0}, Q[TANH_K + 2] = {0};
  int64_t Pn[TANH_K + 2], Qn[TANH_K + 2];
  Pm[0] = 1; P[0] = 1;          /* P_{-1} = 1, P_0 = b_0 = 1 */
  Qm[0] = 0; Q[0] = 1;          /* Q_{-1} = 0, Q_0 = 1       */
  for (int k = 1; k <= TANH_K; ++k) {
    int64_t b = 2 * k + 1;
    for (int j = 0; j < TANH_K + 2; ++j) {
      Pn[j] = b * P[j] + (j > 0 ? Pm[j - 1] : 0);
      Qn[j] = b * Q[j] + (j > 0 ? Qm[j - 1] : 0);
    }
    memcpy(Pm, P, sizeof P); memcpy(P, Pn, sizeof P);
    memcpy(Qm, Q, sizeof Q); memcpy(Q, Qn, sizeof Q);
  }
  tP_n = 0; tQ_n = 0;
  for (int j = 0; j <= TANH_K; ++j) {
    tP[j] = (float)P[j];
    tQ[j] = (float)Q[j];
    if (P[j] != 0) tP_n = j + 1;
    if (Q[j] != 0) tQ_n = j + 1;
  }
  t_ready = 1;
}

/* The rounded coefficients, for tests: writes P then Q (TANH_K+1 each), returns K. */
int oracle_tanh_coeffs(float* p, float* q) {
  if (!t_ready) tanh_coeffs();
  for (int j = 0; j <= TANH_K; ++j) { p[j] = tP[j]; q[j] = tQ[j]; }
  return TANH_K;
}

static float horner(const float* c, int n, float a) {
  float r = c[n - 1];
  for (int j = n - 2; j >= 0; --j) {
    float m = r * a;
    r = m + c[j];
  }
  return r;
}

float oracle_tanhf(float x) {
  if (!t_ready) tanh_coeffs();
  if (fabsf(x) >= 9.0f) return copysignf(1.0f, x);
  float a = x * x;
  float q = horner(tQ, tQ_n, a);
  float p = horner(tP, tP_n, a);
  float xq = x * q;
  return xq / p;
}

void oracle_tanhf_n(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = oracle_tanhf(x[i]);
}

/* ------------------------------------------------------------ sections */

enum {
  OP_MADD3 = 1, OP_XORSHIFT = 2, OP_ADD = 3, OP_MIX = 4, OP_DRIFT = 5, OP_BIN = 6, OP_KE = 7,
  OP_FLAGS = 8, OP_GATHER = 9, OP_KICK = 10, OP_AXPB = 11, OP_MUL = 12, OP_TANH = 13
};

#define F32(f) ((float*)fa[f])
#define F64(f) ((double*)fa[f])
#define I32(f) ((int32_t*)fa[f])
#define U16(f) ((uint16_t*)fa[f])

static uint32_t f32_bits(float v) { uint32_t u; memcpy(&u, &v, 4); return u; }
static uint64_t f64_bits(double v) { uint64_t u; memcpy(&u, &v, 8); return u; }

/*
 * The "mix" section (the random sections of the layout-stress program): per
 * record, over the read set R in ascending field order,
 *   s = sum of the fp32 fields (fp32, starting from +0),
 *   h = xor of the int32 fields, of the two 32-bit halves of the fp64 fields
 *       and of the bf16 fields' 16 bits,
 *   t = s + (h & 255) * 2^-8  (fp32),
 * then every field w of the write set W (all taken from the values before
 * any write) becomes
 *   fp32: w*0.5 + t;   fp64: w*0.5 + (double)t;
 *   int32: w ^ ((h ^ bits(t)) >> 3);   bf16 bits: w ^ low16((h ^ bits(t)) >> 3).
 */
static void sec_mix(int F, const int* dtypes, void** fa, uint64_t R, uint64_t W, int64_t i) {
  float s = 0.0f;
  uint32_t h = 0u;
  for (int f = 0; f < F; ++f) {
    if (!((R >> f) & 1u)) continue;
    switch (dtypes[f]) {
      case D_F32: s = s + F32(f)[i]; break;
      case D_F64: { uint64_t b = f64_bits(F64(f)[i]); h ^= (uint32_t)b ^ (uint32_t)(b >> 32); break; }
      case D_I32: h ^= (uint32_t)I32(f)[i]; break;
      case D_BF16: h ^= (uint32_t)U16(f)[i]; break;
    }
  }
  float hf = (float)(h & 255u);
  float t = s + hf * 0.00390625f;
  uint32_t k = (h ^ f32_bits(t)) >> 3;
  for (int f = 0; f < F; ++f) {
    if (!((W >> f) & 1u)) continue;
    switch (dtypes[f]) {
      case D_F32: { float m = F32(f)[i] * 0.5f; F32(f)[i] = m + t; break; }
      case D_F64: { double m = F64(f)[i] * 0.5; F64(f)[i] = m + (double)t; break; }
      case D_I32: I32(f)[i] = (int32_t)((uint32_t)I32(f)[i] ^ k); break;
      case D_BF16: U16(f)[i] = (uint16_t)(U16(f)[i] ^ (uint16_t)(k & 0xFFFFu)); break;
    }
  }
}

/*
 * Run one section over records [0,n) of the field arrays fa (in place).
 * a = operand field ids, p = fp32 constants; meaning per op:
 *   madd3 (x,y,z):  z = x*y + z                               (fp32)
 *   xorshift (x,z): z = x ^ (x >> 3), logical shift            (int32)
 *   add (x,y,z):    z = x + y                                 (fp32)
 *   mix:            see sec_mix (R = read mask, W = write mask)
 *   drift (px,py,pz,vx,vy,vz; dt): p = p + dt*v, then p -= 1 if p >= 1, p += 1 if p < 0
 *   bin (px,py,pz,cell; G):  c_a = clamp((int)(p_a*G), 0, G-1), cell = cx + G*(cy + G*cz)
 *   ke (vx,vy,vz,m,e):  e = (double)((0.5*m) * ((vx*vx + vy*vy) + vz*vz)), fp32 arithmetic
 *   flags (fl,e; thr): fl = ((fl << 1) | (e > thr)) & 255
 *   gather (vx,vy,vz,px,py,pz,q; dt): j = perm[i]; v_a[i] = v_a[i] + (dt*q[j])*(p_a[j] - 0.5)
 *   kick (vx,vy,vz,q; dt,Ex,Ey,Ez): v_a = v_a + (dt*q)*E_a
 *   axpb (x,z; a,b): z = a*x + b     mul (x,y,z): z = x*y     tanh (x,z): z = oracle_tanhf(x)
 * Every floating operation is rounded to nearest separately, left to right.
 * The gather reads at perm[i] only fields it never writes, so the loop order
 * does not matter.  Returns 0, or -1 for an unknown op.
 */
int oracle_section_range(int op, const int* a, const float* p, uint64_t R, uint64_t W, int F, const int* dtypes,
                         void** fa, int64_t i0, int64_t i1, const int32_t* perm);

int oracle_section(int op, const int* a, const float* p, uint64_t R, uint64_t W, int F, const int* dtypes,
                   void** fa, int64_t n, const int32_t* perm) {
  return oracle_section_range(op, a, p, R, W, F, dtypes, fa, 0, n, perm);
}

/* The same on records [i0, i1) of the field arrays (so that disjoint ranges can run side by
 * side: a record's result depends on its own fields, and a gather's reads at perm[i] on fields
 * no section writes in that section). */
int oracle_section_range(int op, const int* a, const float* p, uint64_t R, uint64_t W, int F, const int* dtypes,
                         void** fa, int64_t i0, int64_t i1, const int32_t* perm) {
  for (int64_t i = i0; i < i1; ++i) {
    switch (op) {
      case OP_MADD3: { float m = F32(a[0])[i] * F32(a[1])[i]; F32(a[2])[i] = m + F32(a[2])[i]; break; }
      case OP_XORSHIFT: { uint32_t u = (uint32_t)I32(a[0])[i]; I32(a[1])[i] = (int32_t)(u ^ (u >> 3)); break; }
      case OP_ADD: { F32(a[2])[i] = F32(a[0])[i] + F32(a[1])[i]; break; }
      case OP_MIX: sec_mix(F, dtypes, fa, R, W, i); break;
      case OP_DRIFT:
        for (int ax = 0; ax < 3; ++ax) {
          float d = p[0] * F32(a[3 + ax])[i];
          float q = F32(a[ax])[i] + d;
          if (q >= 1.0f) q = q - 1.0f;
          else if (q < 0.0f) q = q + 1.0f;
          F32(a[ax])[i] = q;
        }
        break;
      case OP_BIN: {
        int G = (int)p[0];
        int c[3];
        for (int ax = 0; ax < 3; ++ax) {
          float q = F32(a[ax])[i] * p[0];
          int k = (int)q;
          if (k < 0) k = 0;
          if (k > G - 1) k = G - 1;
          c[ax] = k;
        }
        I32(a[3])[i] = c[0] + G * (c[1] + G * c[2]);
        break;
      }
      case OP_KE: {
        float vx = F32(a[0])[i], vy = F32(a[1])[i], vz = F32(a[2])[i];
        float sx = vx * vx, sy = vy * vy, sz = vz * vz;
        float s = sx + sy;
        s = s + sz;
        float hm = 0.5f * F32(a[3])[i];
        float e = hm * s;
        F64(a[4])[i] = (double)e;
        break;
      }
      case OP_FLAGS: {
        uint32_t fl = (uint32_t)I32(a[0])[i];
        uint32_t bit = F64(a[1])[i] > (double)p[0] ? 1u : 0u;
        I32(a[0])[i] = (int32_t)(((fl << 1) | bit) & 255u);
        break;
      }
      case OP_GATHER: {
        int64_t j = perm[i];
        float c = p[0] * F32(a[6])[j];
        for (int ax = 0; ax < 3; ++ax) {
          float d = F32(a[3 + ax])[j] - 0.5f;
          float u = c * d;
          F32(a[ax])[i] = F32(a[ax])[i] + u;
        }
        break;
      }
      case OP_KICK: {
        float c = p[0] * F32(a[3])[i];
        for (int ax = 0; ax < 3; ++ax) {
          float u = c * p[1 + ax];
          F32(a[ax])[i] = F32(a[ax])[i] + u;
        }
        break;
      }
      case OP_AXPB: { float m = p[0] * F32(a[0])[i]; F32(a[1])[i] = m + p[1]; break; }
      case OP_MUL: { F32(a[2])[i] = F32(a[0])[i] * F32(a[1])[i]; break; }
      case OP_TANH: { F32(a[1])[i] = oracle_tanhf(F32(a[0])[i]); break; }
      default: return -1;
    }
  }
  return 0;
}

/* ------------------------------------------- K-Means-shaped sections */

/*
 * The paper's second benchmark (Section 3, Table 1, Table 3) is K-Means: a
 * data-parallel section over all features, then a section that reduces over
 * all records.  Its two sections, as this library defines them (the paper gives
 * no formulas):
 *   features x_0..x_{d-1}: the fp32 fields feat[0..d) (ascending ids);
 *   membership m: the int32 field mf; K clusters; centroid c[k][j] = cent[k*d + j].
 *
 * assign:  per record, D_k = sum over j ascending of (x_j - c[k][j])^2, starting
 *          from +0, the subtraction, the square and the addition each rounded to
 *          nearest in fp32; m = the smallest k whose D_k is smallest (scanning k
 *          upwards, a later k wins only when strictly smaller).
 */
int oracle_kmeans_assign_range(int d, const int* feat, int mf, int K, const float* cent, void** fa, int64_t i0,
                               int64_t i1);

int oracle_kmeans_assign(int d, const int* feat, int mf, int K, const float* cent, void** fa, int64_t n) {
  return oracle_kmeans_assign_range(d, feat, mf, K, cent, fa, 0, n);
}

int oracle_kmeans_assign_range(int d, const int* feat, int mf, int K, const float* cent, void** fa, int64_t i0,
                               int64_t i1) {
  if (d < 1 || K < 1) return -1;
  for (int64_t i = i0; i < i1; ++i) {
    int best = 0;
    float best_d = 0.0f;
    for (int k = 0; k < K; ++k) {
      float D = 0.0f;
      for (int j = 0; j < d; ++j) {
        float diff = F32(feat[j])[i] - cent[k * d + j];
        float sq = diff * diff;
        D = D + sq;
      }
      if (k == 0 || D < best_d) {
        best_d = D;
        best = k;
      }
    }
    I32(mf)[i] = best;
  }
  return 0;
}

/* Fixed-point value of a feature for the reduction: x * 2^23 rounded to the
 * nearest integer, ties to even; 2^31 - 1 or -2^31 beyond the int32 range; 0 for
 * NaN.  The synthetic features lie on the grid of 2^-23, where this is exact. */
static int64_t fixq(float x) {
  float y = x * 8388608.0f;
  if (y != y) return 0;
  if (y >= 2147483648.0f) return 2147483647;
  if (y < -2147483648.0f) return -2147483648LL;
  return (int64_t)nearbyintf(y);
}

/*
 * reduce:  out[k*(d+1)] = the number of records with m = k, and
 *          out[k*(d+1) + 1 + j] = the sum of fixq(x_j) over those records, for
 *          0 <= k < K; records with m outside [0, K) are left out.  The sums are
 *          integers, so they do not depend on the order of the records.
 */
int oracle_kmeans_reduce_range(int d, const int* feat, int mf, int K, void** fa, int64_t i0, int64_t i1,
                               int64_t* out);

int oracle_kmeans_reduce(int d, const int* feat, int mf, int K, void** fa, int64_t n, int64_t* out) {
  return oracle_kmeans_reduce_range(d, feat, mf, K, fa, 0, n, out);
}

/* The sums over records [i0, i1) alone (integer partial sums of ranges add up exactly). */
int oracle_kmeans_reduce_range(int d, const int* feat, int mf, int K, void** fa, int64_t i0, int64_t i1,
                               int64_t* out) {
  if (d < 1 || K < 1) return -1;
  for (int64_t k = 0; k < (int64_t)K * (d + 1); ++k) out[k] = 0;
  for (int64_t i = i0; i < i1; ++i) {
    int32_t m = I32(mf)[i];
    if (m < 0 || m >= K) continue;
    out[(int64_t)m * (d + 1)] += 1;
    for (int j = 0; j < d; ++j) out[(int64_t)m * (d + 1) + 1 + j] += fixq(F32(feat[j])[i]);
  }
  return 0;
}

/* ------------------------------------------------------- differentiation */

/*
 * Forward and reverse pass of a chain of fp32 sections (axpb, mul, tanh) for
 * the scalar loss L = sum_f c_f sum_i field_f[i] after the last section.
 * Per record: run the sections forward keeping the value each one overwrites,
 * then walk them backwards.  With g the adjoint of the record's fields
 * (initially g_f = c_f), section z = op(x, y) is undone by first restoring z,
 * then
 *   gz = g[z]; g[z] = 0;
 *   axpb:  g[x] = g[x] + a*gz
 *   mul:   g[x] = g[x] + gz*y;  g[y] = g[y] + gz*x        (x, y before the section)
 *   tanh:  t = tanh(x); g[x] = g[x] + gz*(1 - t*t)
 * each operation rounded to nearest in fp32.  fa (F arrays of n) holds the
 * inputs on entry and the final state on return; ga receives dL/d(input).
 * ops[k], args[3k..3k+2] = x, y, z (y unused by axpb and tanh), par[2k..2k+1] = a, b.
 */
int oracle_chain_grad(int n_sec, const int* ops, const int* args, const float* par, int F, float** fa,
                      const float* c, float** ga, int64_t n) {
  float* saved = (float*)malloc(sizeof(float) * (size_t)(n_sec > 0 ? n_sec : 1));
  float* v = (float*)malloc(sizeof(float) * (size_t)F);
  float* g = (float*)malloc(sizeof(float) * (size_t)F);
  if (!saved || !v || !g) { free(saved); free(v); free(g); return -1; }
  for (int64_t i = 0; i < n; ++i) {
    for (int f = 0; f < F; ++f) v[f] = fa[f][i];
    for (int k = 0; k < n_sec; ++k) {
      int x = args[3 * k], y = args[3 * k + 1], z = args[3 * k + 2];
      saved[k] = v[z];
      if (ops[k] == OP_AXPB) { float m = par[2 * k] * v[x]; v[z] = m + par[2 * k + 1]; }
      else if (ops[k] == OP_MUL) v[z] = v[x] * v[y];
      else if (ops[k] == OP_TANH) v[z] = oracle_tanhf(v[x]);
      else { free(saved); free(v); free(g); return -1; }
    }
    for (int f = 0; f < F; ++f) fa[f][i] = v[f];
    for (int f = 0; f < F; ++f) g[f] = c[f];
    for (int k = n_sec - 1; k >= 0; --k) {
      int x = args[3 * k], y = args[3 * k + 1], z = args[3 * k + 2];
      v[z] = saved[k];
      float gz = g[z];
      g[z] = 0.0f;
      if (ops[k] == OP_AXPB) {
        float t = par[2 * k] * gz;
        g[x] = g[x] + t;
      } else if (ops[k] == OP_MUL) {
        float t1 = gz * v[y];
        g[x] = g[x] + t1;
        float t2 = gz * v[x];
        g[y] = g[y] + t2;
      } else {
        float t = oracle_tanhf(v[x]);
        float tt = t * t;
        float d = 1.0f - tt;
        float u = gz * d;
        g[x] = g[x] + u;
      }
    }
    for (int f = 0; f < F; ++f) ga[f][i] = g[f];
  }
  free(saved); free(v); free(g);
  return 0;
}

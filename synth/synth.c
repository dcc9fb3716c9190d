/*
 * synth.c -- seeded synthetic inputs shared by the oracle side and the CUDA side.
 *
 * Holds none of the method's arithmetic: only random numbers.  The generator is
 * SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): state advances by the odd constant GAMMA and each
 * output is the state passed through the 64-bit finaliser mix64.  Because the
 * state after k steps is seed + k*GAMMA, output k can be computed directly,
 * which makes every value a pure function of (seed, stream, index): any record
 * of any workload can be regenerated on its own, in any order, on any thread.
 *
 * Distribution recipes (each documented at its kind below) are fixed here so
 * that both sides of every comparison read identical bytes.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Output number k (k = 0, 1, ...) of a SplitMix64 generator seeded with s. */
static inline uint64_t splitmix_at(uint64_t s, uint64_t k) { return mix64(s + (k + 1) * GAMMA); }

/* Key of one independent stream: output number `stream` of the generator seeded with `seed`. */
uint64_t synth_key(uint64_t seed, uint64_t stream) { return splitmix_at(seed, stream); }

/* Value number i of the stream with key `key`. */
uint64_t synth_u64(uint64_t key, uint64_t i) { return splitmix_at(key, i); }

enum {
  SYNTH_F32_PM1 = 0,      /* fp32 uniform [-1,1): (x>>40)*2^-23 - 1, exact            */
  SYNTH_F32_01 = 1,       /* fp32 uniform [0,1):  (x>>40)*2^-24, exact                */
  SYNTH_F64_PM1 = 2,      /* fp64 uniform [-1,1): (x>>11)*2^-52 - 1, exact            */
  SYNTH_I32_U20 = 3,      /* int32 uniform [0,2^20): x>>44                            */
  SYNTH_F32_NORMAL = 4,   /* fp32 N(0,1): Box-Muller in double, rounded once          */
  SYNTH_F32_LOGNORMAL = 5,/* fp32 exp(N(0,1)) in double, rounded once                 */
  SYNTH_F32_SIGN = 6,     /* fp32 +1 or -1 from the top bit                           */
  SYNTH_I32_IOTA = 7,     /* int32 equal to the record index                          */
  SYNTH_ZERO32 = 8,       /* 4 zero bytes                                             */
  SYNTH_ZERO64 = 9,       /* 8 zero bytes                                             */
  SYNTH_RAW16 = 10,       /* top 16 bits of x (any 2-byte field)                      */
  SYNTH_RAW32 = 11,       /* top 32 bits of x (any 4-byte field)                      */
  SYNTH_RAW64 = 12        /* all 64 bits of x (any 8-byte field)                      */
};

int synth_kind_bytes(int kind) {
  switch (kind) {
    case SYNTH_F64_PM1: case SYNTH_ZERO64: case SYNTH_RAW64: return 8;
    case SYNTH_RAW16: return 2;
    default: return 4;
  }
}

static void fill_one(int kind, uint64_t key, int64_t i, void* out, int64_t j) {
  uint64_t x = synth_u64(key, (uint64_t)i);
  switch (kind) {
    case SYNTH_F32_PM1: ((float*)out)[j] = (float)(x >> 40) * 0x1p-23f - 1.0f; break;
    case SYNTH_F32_01: ((float*)out)[j] = (float)(x >> 40) * 0x1p-24f; break;
    case SYNTH_F64_PM1: ((double*)out)[j] = (double)(x >> 11) * 0x1p-52 - 1.0; break;
    case SYNTH_I32_U20: ((int32_t*)out)[j] = (int32_t)(x >> 44); break;
    case SYNTH_F32_NORMAL:
    case SYNTH_F32_LOGNORMAL: {
      double u1 = (double)((x >> 40) + 1) * 0x1p-24;        /* (0,1] */
      double u2 = (double)(x & 0xFFFFFFULL) * 0x1p-24;      /* [0,1) */
      double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
      ((float*)out)[j] = (float)(kind == SYNTH_F32_NORMAL ? z : exp(z));
      break;
    }
    case SYNTH_F32_SIGN: ((float*)out)[j] = (x >> 63) ? -1.0f : 1.0f; break;
    case SYNTH_I32_IOTA: ((int32_t*)out)[j] = (int32_t)i; break;
    case SYNTH_ZERO32: ((uint32_t*)out)[j] = 0u; break;
    case SYNTH_ZERO64: ((uint64_t*)out)[j] = 0ull; break;
    case SYNTH_RAW16: ((uint16_t*)out)[j] = (uint16_t)(x >> 48); break;
    case SYNTH_RAW32: ((uint32_t*)out)[j] = (uint32_t)(x >> 32); break;
    case SYNTH_RAW64: ((uint64_t*)out)[j] = x; break;
    default: break;
  }
}

/*
 * Fill out[0..n) with values of stream `key`: value j uses counter idx[j] when
 * idx is non-NULL, else i0 + j.  Returns 0, or -1 for an unknown kind.
 */
int synth_fill(int kind, uint64_t key, const int64_t* idx, int64_t i0, int64_t n, void* out) {
  if (kind < 0 || kind > SYNTH_RAW64) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) fill_one(kind, key, idx ? idx[j] : i0 + j, out, j);
  return 0;
}

/* Unbiased-enough draw in [0, m): Lemire's multiply-shift of a 64-bit value. */
static inline uint64_t below(uint64_t x, uint64_t m) {
  return (uint64_t)(((unsigned __int128)x * (unsigned __int128)m) >> 64);
}

/* Uniform random permutation of [0,n) by Fisher-Yates (Durstenfeld), draws from stream `key`. */
void synth_perm_i32(uint64_t key, int64_t n, int32_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = (int32_t)i;
  for (int64_t i = n - 1, k = 0; i > 0; --i, ++k) {
    int64_t j = (int64_t)below(synth_u64(key, (uint64_t)k), (uint64_t)(i + 1));
    int32_t t = out[i]; out[i] = out[j]; out[j] = t;
  }
}

/* Uniform double in [0,1) from value i of stream key: (x>>11)*2^-53. */
double synth_unit(uint64_t key, uint64_t i) { return (double)(synth_u64(key, i) >> 11) * 0x1p-53; }

/*
 * sk_oracle.c -- CPU oracle for the random-sketch hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  It may be used only by tests/, by __graft_entry__.smoke()
 * and by the cpu_baseline / reference leg of bench.py.  It shares no code,
 * header, table or constant generator with the CUDA path: every constant here
 * is written out from its mathematical definition (Philox from Salmon et al.
 * 2011; polynomial coefficients from the Taylor series of sin and cos and,
 * for ln, from the least-squares fit that oracle/fit_ln.py writes out).
 *
 * What it computes (arXiv 2603.20966, Sec. 1 and Sec. 3 "Lower Bounds and
 * Algorithm for Matrix Multiplication with a Random Matrix"):
 *   the sketch B = A * Omega of a dense matrix by a dense random matrix whose
 *   entries any processor can regenerate from a shared seed (Sec. 6.2,
 *   "Communicate vs Redundantly Generate Omega": Philox counter-based
 *   generation with a shared seed), and, by the transposition remark after
 *   Theorem 2, the left form S * A.
 *
 * Notation used throughout (row-major storage with leading dimensions):
 *   left  sketch  Y[k x n] = S[k x m] * A[m x n]
 *   right sketch  Y[m x k] = A[m x n] * S^T,  S[k x n]
 *   S(r, c) = s * q(g(r, c)),  s = fl32(1 / sqrt(k)),
 *   g(r, c) the generated value, q the storage precision (identity for
 *   FP32, round-to-nearest-even to BF16 or to E4M3 for the tensor forms).
 * Accumulation is in FP64 (double) with no blocking or reordering: every
 * output entry is a plain dot product in index order.
 *
 * The generator (the paper fixes only "Philox with a shared seed"; the rest
 * is this library's reading, stated once here and implemented independently
 * on the GPU):
 *   key     = (seed mod 2^32, seed >> 32)
 *   counter = (c >> 2, r, dom, 0)  Gaussian / uniform, 4 entries per call
 *           = (c >> 7, r, dom, 0)  Rademacher, 128 entries per call
 *   dom     = 0 for the sketching matrix.
 *   Gaussian (Box-Muller): entries c = 4j..4j+3 use the words (x0,x1) for
 *     c mod 4 in {0,1} and (x2,x3) for c mod 4 in {2,3};
 *     u1 = ((xa >> 8) + 1) * 2^-24 in (0,1],  rho = sqrt(-2 ln u1);
 *     the angle from the top 24 bits of xb: w = bits 29..8, the position
 *     r = w 2^-23 - 1/4 in [-1/4, 1/4), (C, S) = (cospi r, sinpi r), and
 *     (X, Y) = (C, S) turned by q = bits 31..30 quarter turns:
 *     (C, S), (-S, C), (-C, -S), (S, -C) -- the angle pi r + q pi/2, so the
 *     2^24 words give the 2^24 multiples of 2 pi / 2^24, each once;
 *     g = rho * X for even c, rho * Y for odd c.
 *   Rademacher: bit (c mod 32) of word ((c >> 5) mod 4); set bit -> -1.
 *   Uniform: u = (x_{c mod 4} >> 8) * 2^-24 in [0,1) (the distribution the
 *     paper's experiments draw, Sec. 6.2).
 *   ln, sinpi and cospi are this library's own FP32 polynomials built only
 *   from round-to-nearest add, mul and fma (and sqrt for rho), so that CPU
 *   and GPU agree bit for bit.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GAUSSIAN 0
#define ORC_RADEMACHER 1
#define ORC_UNIFORM 2

#define ORC_FP32 0
#define ORC_BF16 1
#define ORC_E4M3 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the       */
/* published description: 10 rounds of two 32x32->64 multiplies with the     */
/* S-box-free "mulhilo" construction, the key bumped by the Weyl constants   */
/* (golden ratio and sqrt(3)-1 in 32-bit fixed point) between rounds.        */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

static void philox4x32_10(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t count) {
  for (int64_t i = 0; i < count; ++i) philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Bit helpers                                                               */
/* ------------------------------------------------------------------------ */
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* ------------------------------------------------------------------------ */
/* Natural logarithm on (0, 1], FP32.                                         */
/* x = 2^e f with f folded into [sqrt(1/2), sqrt(2)) (f > fl32(sqrt 2) is     */
/* halved and e raised by one); t = f - 1 (exact); ln f = t + t^2 Q(t) with  */
/* Q the degree-8 least-squares fit of (ln(1+t) - t) / t^2 written out by    */
/* oracle/fit_ln.py; ln x = e*LN2_HI + (e*LN2_LO + ln f), LN2_HI holding the  */
/* leading 16 bits of ln 2 so that e*LN2_HI is exact (Cody-Waite).           */
/* ------------------------------------------------------------------------ */
float orc_ln1(float x) {
  static const float q[9] = {
      -0x1.fffff8p-2f, 0x1.555558p-2f, -0x1.000422p-2f, 0x1.999fc2p-3f, -0x1.5424e0p-3f,
      0x1.22bf86p-3f, -0x1.0f9b0cp-3f, 0x1.068b28p-3f, -0x1.321a48p-4f};
  const float ln2_hi = 0x1.62e4p-1f;    /* 0.693145751953125 */
  const float ln2_lo = 0x1.7f7d1cp-20f; /* ln 2 - ln2_hi rounded to FP32 */
  uint32_t b = f2u(x);
  int32_t e = (int32_t)(b >> 23) - 127;
  uint32_t mb = b & 0x007fffffu;
  if (mb > 0x003504f3u) { /* f > fl32(sqrt 2): use f/2 and e+1 */
    mb |= 0x3f000000u;
    e += 1;
  } else {
    mb |= 0x3f800000u;
  }
  float t = u2f(mb) - 1.0f;
  float p = q[8];
  for (int i = 7; i >= 0; --i) p = fmaf(t, p, q[i]);
  float lnf = fmaf(t * t, p, t);
  float ef = (float)e;
  return fmaf(ef, ln2_hi, fmaf(ef, ln2_lo, lnf));
}

/* ------------------------------------------------------------------------ */
/* sin(pi r), cos(pi r) for r in [-1/4, 1/4], FP32: the Taylor series of     */
/* sin(pi r) to r^9 and cos(pi r) to r^10, coefficients (-1)^j pi^n / n!     */
/* rounded once to FP32.                                                     */
/* ------------------------------------------------------------------------ */
void orc_sincospi_quarter1(float r, float* sin_out, float* cos_out) {
  const float s1 = 0x1.921fb6p+1f;   /*  pi        */
  const float s3 = -0x1.4abbcep+2f;  /* -pi^3/3!   */
  const float s5 = 0x1.466bc6p+1f;   /*  pi^5/5!   */
  const float s7 = -0x1.32d2ccp-1f;  /* -pi^7/7!   */
  const float s9 = 0x1.507834p-4f;   /*  pi^9/9!   */
  const float c2 = -0x1.3bd3ccp+2f;  /* -pi^2/2!   */
  const float c4 = 0x1.03c1f0p+2f;   /*  pi^4/4!   */
  const float c6 = -0x1.55d3c8p+0f;  /* -pi^6/6!   */
  const float c8 = 0x1.e1f506p-3f;   /*  pi^8/8!   */
  const float c10 = -0x1.a6d1f2p-6f; /* -pi^10/10! */
  float r2 = r * r;
  float sp = fmaf(r2, s9, s7);
  sp = fmaf(r2, sp, s5);
  sp = fmaf(r2, sp, s3);
  sp = fmaf(r2, sp, s1);
  *sin_out = r * sp;
  float cp = fmaf(r2, c10, c8);
  cp = fmaf(r2, cp, c6);
  cp = fmaf(r2, cp, c4);
  cp = fmaf(r2, cp, c2);
  *cos_out = fmaf(r2, cp, 1.0f);
}

/* ------------------------------------------------------------------------ */
/* The point (X, Y) on the unit circle of an angle word w (its top 24 bits): */
/* position r = w' 2^-23 - 1/4 with w' = bits 29..8 (0.5 + w' 2^-23 and its  */
/* difference with 3/4 are exact), (C, S) = (cospi r, sinpi r), turned by a  */
/* quarter turn when bit 30 is set and by a half turn when bit 31 is set.    */
/* ------------------------------------------------------------------------ */
void orc_circle1(uint32_t w, float* x, float* y) {
  float r = u2f(0x3f000000u | ((w >> 7) & 0x007ffffeu)) - 0.75f;
  float sn, cs;
  orc_sincospi_quarter1(r, &sn, &cs);
  float px = cs, py = sn;
  if (w & 0x40000000u) { /* (x, y) -> (-y, x) */
    px = -sn;
    py = cs;
  }
  if (w & 0x80000000u) { /* (x, y) -> (-x, -y) */
    px = -px;
    py = -py;
  }
  *x = px;
  *y = py;
}

void orc_ln(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = orc_ln1(x[i]);
}
void orc_sincospi_quarter(const float* r, float* s, float* c, int64_t n) {
  for (int64_t i = 0; i < n; ++i) orc_sincospi_quarter1(r[i], s + i, c + i);
}
void orc_circle(const uint32_t* w, float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) orc_circle1(w[i], x + i, y + i);
}

/* ------------------------------------------------------------------------ */
/* Round-to-nearest-even conversions, written from the definition of the     */
/* target formats: the representable value nearest to x, ties to the one    */
/* with an even last significand bit.                                        */
/* ------------------------------------------------------------------------ */
/* BF16: 8 exponent bits (bias 127), 7 stored significand bits. */
static uint16_t bf16_rne(float x) {
  uint32_t b = f2u(x);
  uint16_t sign = (uint16_t)((b >> 16) & 0x8000u);
  if (isnan(x)) return (uint16_t)(sign | 0x7fc0u);
  double a = fabs((double)x);
  if (a == 0.0) return sign;
  int e;
  frexp(a, &e);               /* a = m 2^e, m in [0.5, 1) */
  int eu = e - 1;             /* a in [2^eu, 2^(eu+1)) */
  if (eu < -126) eu = -126;   /* subnormal range: fixed quantum */
  double quantum = ldexp(1.0, eu - 7);
  double n = rint(a / quantum); /* exact division by a power of two */
  double v = n * quantum;
  if (v >= ldexp(1.0, 128)) return (uint16_t)(sign | 0x7f80u); /* overflow to inf */
  /* encode v */
  if (v < ldexp(1.0, -126)) return (uint16_t)(sign | (uint16_t)(v / ldexp(1.0, -133)));
  int ev;
  double mv = frexp(v, &ev);  /* v = mv 2^ev, mv in [0.5,1) */
  uint32_t exp_field = (uint32_t)(ev - 1 + 127);
  uint32_t man = (uint32_t)((mv * 2.0 - 1.0) * 128.0);
  return (uint16_t)(sign | (exp_field << 7) | man);
}

/* E4M3 ("fn" variant, OCP FP8): 4 exponent bits (bias 7), 3 significand bits,
 * largest finite 448, no infinities; out-of-range values saturate to +-448
 * (the satfinite conversion), NaN maps to 0x7f. */
static uint8_t e4m3_rne(float x) {
  uint8_t sign = signbit(x) ? 0x80u : 0u;
  if (isnan(x)) return (uint8_t)(sign | 0x7fu);
  double a = fabs((double)x);
  if (a == 0.0) return sign;
  int e;
  frexp(a, &e);
  int eu = e - 1;
  if (eu < -6) eu = -6;       /* subnormals: quantum 2^-9 */
  double quantum = ldexp(1.0, eu - 3);
  double v = rint(a / quantum) * quantum;
  if (v > 448.0) v = 448.0;   /* saturate */
  if (v < ldexp(1.0, -6)) return (uint8_t)(sign | (uint8_t)(v / ldexp(1.0, -9)));
  int ev;
  double mv = frexp(v, &ev);
  uint32_t exp_field = (uint32_t)(ev - 1 + 7);
  uint32_t man = (uint32_t)((mv * 2.0 - 1.0) * 8.0);
  return (uint8_t)(sign | (exp_field << 3) | man);
}

static double bf16_value(uint16_t h) { return (double)u2f((uint32_t)h << 16); }

static double e4m3_value(uint8_t v) {
  double sgn = (v & 0x80u) ? -1.0 : 1.0;
  int ef = (v >> 3) & 0xf, man = v & 7;
  if (ef == 0xf && man == 7) return NAN;
  if (ef == 0) return sgn * ldexp((double)man, -9);
  return sgn * ldexp(1.0 + man / 8.0, ef - 7);
}

void orc_bf16_rne(const float* x, uint16_t* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = bf16_rne(x[i]);
}
void orc_e4m3_rne(const float* x, uint8_t* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = e4m3_rne(x[i]);
}
void orc_e4m3_value(const uint8_t* x, double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = e4m3_value(x[i]);
}

/* ------------------------------------------------------------------------ */
/* Generated values                                                          */
/* ------------------------------------------------------------------------ */
float orc_scale(int64_t k) { return 1.0f / sqrtf((float)k); }

/* q(g(r, c)) as a double (every BF16 / E4M3 / FP32 value is exact in double). */
static double quantize(float g, int prec) {
  if (prec == ORC_BF16) return bf16_value(bf16_rne(g));
  if (prec == ORC_E4M3) return e4m3_value(e4m3_rne(g));
  return (double)g;
}

/* Box-Muller on one pair of Philox words (xa, xb):                         */
/* u1 = ((xa >> 8) + 1) 2^-24 in (0, 1], rho = sqrt(-2 ln u1), (X, Y) the    */
/* circle point of xb, z[0] = rho X, z[1] = rho Y.                           */
static void box_muller(uint32_t xa, uint32_t xb, float z[2]) {
  float u1 = (float)((xa >> 8) + 1u) * 0x1p-24f;
  float rho = sqrtf(-2.0f * orc_ln1(u1));
  float x, y;
  orc_circle1(xb, &x, &y);
  z[0] = rho * x;
  z[1] = rho * y;
}

/* z[2i], z[2i+1] = Box-Muller of the word pair (w[2i], w[2i+1]), i < npairs. */
void orc_box_muller(const uint32_t* w, float* z, int64_t npairs) {
  for (int64_t i = 0; i < npairs; ++i) box_muller(w[2 * i], w[2 * i + 1], z + 2 * i);
}

/* Generate entries (r, col0 .. col0+cols-1) of one row of the generated
 * matrix, unscaled and quantized, into out[0..cols). */
static void gen_row(uint64_t seed, int dist, int prec, uint32_t dom, uint32_t r,
                    int64_t col0, int64_t cols, double* out) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  int64_t cached_block = -1;
  for (int64_t j = 0; j < cols; ++j) {
    uint32_t c = (uint32_t)(col0 + j);
    float g;
    if (dist == ORC_RADEMACHER) {
      int64_t block = c >> 7;
      if (block != cached_block) {
        uint32_t ctr[4] = {(uint32_t)block, r, dom, 0u};
        philox4x32_10(ctr, key, x);
        cached_block = block;
      }
      uint32_t word = x[(c >> 5) & 3u];
      g = ((word >> (c & 31u)) & 1u) ? -1.0f : 1.0f;
    } else {
      int64_t block = c >> 2;
      if (block != cached_block) {
        uint32_t ctr[4] = {(uint32_t)block, r, dom, 0u};
        philox4x32_10(ctr, key, x);
        cached_block = block;
      }
      if (dist == ORC_UNIFORM) {
        g = (float)(x[c & 3u] >> 8) * 0x1p-24f;
      } else {
        uint32_t pair = (c >> 1) & 1u;
        float z[2];
        box_muller(x[2 * pair], x[2 * pair + 1], z);
        g = z[c & 1u];
      }
    }
    out[j] = quantize(g, prec);
  }
}

/* out[i*ld + j] = q(g(row0+i, col0+j)) as FP32 (unscaled). Returns 0, or -1
 * on a bad argument. */
int orc_generate(uint64_t seed, int dist, int prec, uint32_t dom, int64_t row0, int64_t col0,
                 int64_t rows, int64_t cols, float* out, int64_t ld) {
  if (rows < 0 || cols < 0 || row0 < 0 || col0 < 0 || ld < cols) return -1;
  if (row0 + rows > 4294967296LL || col0 + cols > 4294967296LL) return -1;
  double* buf = (double*)malloc(sizeof(double) * (size_t)(cols > 0 ? cols : 1));
  if (!buf) return -1;
  for (int64_t i = 0; i < rows; ++i) {
    gen_row(seed, dist, prec, dom, (uint32_t)(row0 + i), col0, cols, buf);
    for (int64_t j = 0; j < cols; ++j) out[i * ld + j] = (float)buf[j];
  }
  free(buf);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The sketch, FP64 accumulation.                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t seed; int dist, prec; int64_t k;
  const float* A; int64_t m, n, lda;
  const uint8_t* Aq; const int32_t* exps;  /* FP8 right sketch: codes of A, row exponents */
  const int64_t* idx; int64_t nidx;   /* output column (left) / row (right) subset */
  double* Y; int64_t ldy;
  const double* S;                    /* right sketch: full S, k x n, scaled */
  int64_t i_begin, i_end;
  int status;
} job_t;

/* Left: Y[i][jj] = sum_l S(i,l) A(l, idx[jj]); S(i,l) = s q(g(i,l)). */
static void* left_worker(void* arg) {
  job_t* J = (job_t*)arg;
  const double s = (double)orc_scale(J->k);
  double* srow = (double*)malloc(sizeof(double) * (size_t)J->m);
  double* acc = (double*)malloc(sizeof(double) * (size_t)(J->nidx > 0 ? J->nidx : 1));
  if (!srow || !acc) { J->status = -1; free(srow); free(acc); return NULL; }
  for (int64_t i = J->i_begin; i < J->i_end; ++i) {
    gen_row(J->seed, J->dist, J->prec, 0u, (uint32_t)i, 0, J->m, srow);
    for (int64_t l = 0; l < J->m; ++l) srow[l] *= s;
    for (int64_t jj = 0; jj < J->nidx; ++jj) acc[jj] = 0.0;
    for (int64_t l = 0; l < J->m; ++l) {
      const float* arow = J->A + l * J->lda;
      const double sv = srow[l];
      for (int64_t jj = 0; jj < J->nidx; ++jj) {
        int64_t j = J->idx ? J->idx[jj] : jj;
        acc[jj] += sv * (double)arow[j];
      }
    }
    for (int64_t jj = 0; jj < J->nidx; ++jj) J->Y[i * J->ldy + jj] = acc[jj];
  }
  free(srow); free(acc);
  J->status = 0;
  return NULL;
}

/* Right: Y[ii][j] = sum_c A(idx[ii], c) S(j, c). */
static void* right_worker(void* arg) {
  job_t* J = (job_t*)arg;
  for (int64_t ii = J->i_begin; ii < J->i_end; ++ii) {
    int64_t i = J->idx ? J->idx[ii] : ii;
    const float* arow = J->A + i * J->lda;
    for (int64_t j = 0; j < J->k; ++j) {
      const double* srow = J->S + j * J->n;
      double acc = 0.0;
      for (int64_t c = 0; c < J->n; ++c) acc += (double)arow[c] * srow[c];
      J->Y[ii * J->ldy + j] = acc;
    }
  }
  J->status = 0;
  return NULL;
}

static int run_jobs(job_t* base, int64_t total, int nthreads, void* (*fn)(void*)) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > total) nthreads = (int)(total > 0 ? total : 1);
  job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -1; }
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = *base;
    jobs[t].i_begin = total * t / nthreads;
    jobs[t].i_end = total * (t + 1) / nthreads;
    jobs[t].status = -1;
    if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) { fn(&jobs[t]); th[t] = 0; }
  }
  for (int t = 0; t < nthreads; ++t) {
    if (th[t]) pthread_join(th[t], NULL);
    if (jobs[t].status != 0) rc = -1;
  }
  free(jobs); free(th);
  return rc;
}

/* Left sketch, rows row0 .. row0+rows-1 of Y = S[k x m] A[m x n], columns idx
 * (idx == NULL: all n columns, nidx == n), into Y[rows x nidx] (leading dim
 * ldy).  Row i of the result uses the generated row row0 + i.  Returns 0 or -1. */
int orc_apply_left_rows(uint64_t seed, int dist, int prec, int64_t k, int64_t row0, int64_t rows,
                        const float* A, int64_t m, int64_t n, int64_t lda, const int64_t* idx,
                        int64_t nidx, double* Y, int64_t ldy, int nthreads) {
  if (k <= 0 || m <= 0 || n <= 0 || lda < n || nidx < 0 || ldy < nidx) return -1;
  if (row0 < 0 || rows < 0 || row0 + rows > k) return -1;
  if (!idx && nidx != n) return -1;
  job_t J = {0};
  J.seed = seed; J.dist = dist; J.prec = prec; J.k = k;
  J.A = A; J.m = m; J.n = n; J.lda = lda; J.idx = idx; J.nidx = nidx;
  J.Y = Y - row0 * ldy; J.ldy = ldy;  /* worker writes row i at Y + i*ldy */
  job_t* base = &J;
  if (rows == 0) return 0;
  /* split [row0, row0+rows) across threads */
  if (nthreads < 1) nthreads = 1;
  if (nthreads > rows) nthreads = (int)rows;
  job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -1; }
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = *base;
    jobs[t].i_begin = row0 + rows * t / nthreads;
    jobs[t].i_end = row0 + rows * (t + 1) / nthreads;
    jobs[t].status = -1;
    if (pthread_create(&th[t], NULL, left_worker, &jobs[t]) != 0) { left_worker(&jobs[t]); th[t] = 0; }
  }
  for (int t = 0; t < nthreads; ++t) {
    if (th[t]) pthread_join(th[t], NULL);
    if (jobs[t].status != 0) rc = -1;
  }
  free(jobs); free(th);
  return rc;
}

/* Left sketch: Y[k x nidx] (leading dim ldy) = columns idx of S[k x m] A[m x n].
 * idx == NULL means all n columns (nidx must equal n).  Returns 0 or -1. */
int orc_apply_left(uint64_t seed, int dist, int prec, int64_t k, const float* A, int64_t m,
                   int64_t n, int64_t lda, const int64_t* idx, int64_t nidx, double* Y,
                   int64_t ldy, int nthreads) {
  return orc_apply_left_rows(seed, dist, prec, k, 0, k, A, m, n, lda, idx, nidx, Y, ldy, nthreads);
}

/* Right sketch: Y[nidx x k] (leading dim ldy) = rows idx of A[m x n] S^T, S[k x n].
 * idx == NULL means all m rows (nidx must equal m).  Returns 0 or -1. */
int orc_apply_right(uint64_t seed, int dist, int prec, int64_t k, const float* A, int64_t m,
                    int64_t n, int64_t lda, const int64_t* idx, int64_t nidx, double* Y,
                    int64_t ldy, int nthreads) {
  if (k <= 0 || m <= 0 || n <= 0 || lda < n || nidx < 0 || ldy < k) return -1;
  if (!idx && nidx != m) return -1;
  double* S = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
  if (!S) return -1;
  const double s = (double)orc_scale(k);
  for (int64_t j = 0; j < k; ++j) {
    gen_row(seed, dist, prec, 0u, (uint32_t)j, 0, n, S + j * n);
    for (int64_t c = 0; c < n; ++c) S[j * n + c] *= s;
  }
  job_t J = {0};
  J.seed = seed; J.dist = dist; J.prec = prec; J.k = k;
  J.A = A; J.m = m; J.n = n; J.lda = lda; J.idx = idx; J.nidx = nidx; J.Y = Y; J.ldy = ldy;
  J.S = S;
  int rc = run_jobs(&J, nidx, nthreads, right_worker);
  free(S);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* FP8 (E4M3) form of A                                                      */
/* ------------------------------------------------------------------------ */
/* The paper is silent on low precision; this library's reading of "E4M3 A
 * with per-tile scales" (the tile being one row of A, which spans the whole
 * contracted dimension of the right sketch, so the scale factors out of every
 * dot product):
 *   e_i  = the smallest integer with max_j |a_ij| <= 448 * 2^e_i (0 for a row
 *          of zeros),
 *   A_q(i, j) = RNE_e4m3(a_ij * 2^-e_i).
 * Scaling by a power of two is exact, so each code is the E4M3 rounding of a
 * known number; no code saturates (|a_ij| 2^-e_i <= 448, E4M3's largest). */
int orc_quantize_rows_e4m3(const float* A, int64_t m, int64_t n, int64_t lda, uint8_t* Aq,
                           int64_t ldq, int32_t* exps) {
  if (m <= 0 || n <= 0 || lda < n || ldq < n) return -1;
  for (int64_t i = 0; i < m; ++i) {
    const float* a = A + i * lda;
    double amax = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      const double v = fabs((double)a[j]);
      if (v > amax) amax = v;
    }
    int e = 0;
    if (amax > 0.0 && isfinite(amax)) {  /* a row holding Inf keeps e = 0 */
      e = ilogb(amax) - 8;
      while (ldexp(amax, -e) > 448.0) ++e;
      while (ldexp(amax, -(e - 1)) <= 448.0) --e;
    }
    exps[i] = e;
    for (int64_t j = 0; j < n; ++j) Aq[i * ldq + j] = e4m3_rne((float)ldexp((double)a[j], -e));
  }
  return 0;
}

/* FP8 right sketch: Y[ii][j] = 2^{e_i} s sum_c value(A_q(i, c)) value(RNE_e4m3(g(j, c)))
 * for the rows i = idx[ii] (idx NULL: all m rows). */
static void* right_q8_worker(void* arg) {
  job_t* J = (job_t*)arg;
  double* arow = (double*)malloc(sizeof(double) * (size_t)J->n);
  if (!arow) { J->status = -1; return NULL; }
  for (int64_t ii = J->i_begin; ii < J->i_end; ++ii) {
    int64_t i = J->idx ? J->idx[ii] : ii;
    const uint8_t* q = J->Aq + i * J->lda;
    for (int64_t c = 0; c < J->n; ++c) arow[c] = e4m3_value(q[c]);
    const double rs = ldexp(1.0, J->exps[i]);
    for (int64_t j = 0; j < J->k; ++j) {
      const double* srow = J->S + j * J->n;
      double acc = 0.0;
      for (int64_t c = 0; c < J->n; ++c) acc += arow[c] * srow[c];
      J->Y[ii * J->ldy + j] = rs * acc;
    }
  }
  free(arow);
  J->status = 0;
  return NULL;
}

int orc_apply_right_q8(uint64_t seed, int dist, int64_t k, const uint8_t* Aq,
                       const int32_t* exps, int64_t m, int64_t n, int64_t ldq,
                       const int64_t* idx, int64_t nidx, double* Y, int64_t ldy, int nthreads) {
  if (k <= 0 || m <= 0 || n <= 0 || ldq < n || nidx < 0 || ldy < k) return -1;
  if (!idx && nidx != m) return -1;
  double* S = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
  if (!S) return -1;
  const double s = (double)orc_scale(k);
  for (int64_t j = 0; j < k; ++j) {
    gen_row(seed, dist, ORC_E4M3, 0u, (uint32_t)j, 0, n, S + j * n);
    for (int64_t c = 0; c < n; ++c) S[j * n + c] *= s;
  }
  job_t J = {0};
  J.seed = seed; J.dist = dist; J.prec = ORC_E4M3; J.k = k;
  J.Aq = Aq; J.exps = exps; J.m = m; J.n = n; J.lda = ldq; J.idx = idx; J.nidx = nidx;
  J.Y = Y; J.ldy = ldy; J.S = S;
  int rc = run_jobs(&J, nidx, nthreads, right_q8_worker);
  free(S);
  return rc;
}

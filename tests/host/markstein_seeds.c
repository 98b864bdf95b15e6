/* Host proof for the device generator's square root (sqrt_x2 in
 * paper_2603_20966_gb300/csrc/sk_rng.cuh): the same Markstein correction
 * sequence, written out in C with explicit fmaf and IEEE single-precision
 * rounding, run on every radicand the Box-Muller step can produce
 * (w = -2 ln u1, u1 = j 2^-24, j = 1 .. 2^24) from EVERY seed within
 * SEED_ULPS units in the last place of the correctly rounded reciprocal
 * square root, and compared with the IEEE square root.  The hardware
 * approximation the device starts from is within 2^-22.9 relative, well
 * inside the range checked, so the device results equal the IEEE ones
 * whatever the exact seeds are.  Prints the number of mismatches; exit
 * status 0 iff none. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#define SEED_ULPS 6

float orc_ln1(float x); /* the oracle's ln: the radicands are -2 ln u1 */

static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

static float sqrt_seq(float w, float y) {
  float g = w * y;
  float h = 0.5f * y;
  float t = fmaf(-g, h, 0.5f);
  g = fmaf(g, t, g);
  h = fmaf(h, t, h);
  float d = fmaf(-g, g, w);
  return fmaf(d, h, g);
}

int main(void) {
  long bad_sqrt = 0, cases = 0;
  for (uint32_t j = 1; j <= (1u << 24); ++j) {
    float u1 = (float)j * 0x1p-24f;
    float w = -2.0f * orc_ln1(u1);
    float s_ieee = sqrtf(w);
    /* the device takes its seed at max(w, 1e-30): finite at w = -0 (u1 = 1) */
    float ry_rn = (float)(1.0 / sqrt((double)fmaxf(w, 1e-30f)));
    for (int k = -SEED_ULPS; k <= SEED_ULPS; ++k) {
      float ys = u2f(f2u(ry_rn) + k);
      if (f2u(sqrt_seq(w, ys)) != f2u(s_ieee)) ++bad_sqrt;
      ++cases;
    }
  }
  printf("cases %ld root mismatches %ld\n", cases, bad_sqrt);
  return bad_sqrt != 0;
}

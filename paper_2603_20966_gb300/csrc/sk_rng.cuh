// sk_rng.cuh -- device-side generator of the sketching matrix entries.
//
// Entry (r, c) of the generated matrix is a pure function of
// (seed, r, c): any CTA that needs it regenerates it instead of reading it,
// which is the single-GPU form of the paper's choice to generate the random
// matrix redundantly on every processor rather than communicate it
// (arXiv 2603.20966, Sec. 6.2, "Communicate vs Redundantly Generate Omega",
// Philox with a shared seed; Alg. 1 GenRandom).
//
// Specification (identical bit for bit to the CPU oracle, written
// independently here):
//   key      = (seed lo32, seed hi32)
//   counter  = (c >> 2, r, dom, 0) for Gaussian/uniform (4 entries per call),
//              (c >> 7, r, dom, 0) for Rademacher (128 entries per call)
//   Philox4x32-10 (Salmon et al., SC'11): 10 rounds, multipliers
//   0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
//   Gaussian: Box-Muller on (x0,x1) for c%4 in {0,1}, (x2,x3) for {2,3}:
//     u1 = ((xa>>8)+1) 2^-24, rho = sqrt(-2 ln u1); from xb the position
//     r = (bits 29..8) 2^-23 - 1/4 and (X, Y) = (cospi r, sinpi r) turned by
//     q = bits 31..30 quarter turns (angle pi r + q pi/2: the 2^24 words give
//     every multiple of 2 pi / 2^24 once); g = rho X (c even) or rho Y (c odd).
//   Rademacher: bit c%32 of word (c>>5)%4, set -> -1.
//   Uniform: (x_{c%4} >> 8) 2^-24.
// Every floating-point step is an explicitly rounded IEEE operation
// (__fadd2_rn, __fmul2_rn, __ffma2_rn and their scalar forms), so no
// compiler contraction or fast-math flag can change a bit.  ln, sin and cos
// are polynomials; the square root of Box-Muller is the correctly rounded
// IEEE result, computed by Markstein's method from the hardware
// reciprocal-square-root approximation (see sqrt_x2).
#pragma once
#include <stdint.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace sk {

enum : int { kGaussian = 0, kRademacher = 1, kUniform = 2 };
enum : int { kFP32 = 0, kBF16 = 1, kE4M3 = 2 };

struct PhiloxKey {
  uint32_t k0, k1;
};

__host__ __device__ inline PhiloxKey make_key(uint64_t seed) {
  return PhiloxKey{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
}

// The key words of all ten rounds, (k0 + i 0x9E3779B9, k1 + i 0xBB67AE85) at
// k[2i], k[2i+1].  A kernel that receives them among its launch parameters
// reads each one as a constant operand of the round's XOR instead of
// stepping the key in registers on every call.
struct PhiloxRoundKeys {
  uint32_t k[20];
};

__host__ __device__ inline PhiloxRoundKeys round_keys(PhiloxKey key) {
  PhiloxRoundKeys rk;
  for (int i = 0; i < 10; ++i) {
    rk.k[2 * i] = key.k0 + (uint32_t)i * 0x9E3779B9u;
    rk.k[2 * i + 1] = key.k1 + (uint32_t)i * 0xBB67AE85u;
  }
  return rk;
}

__device__ __forceinline__ uint32_t round_key(const PhiloxKey& key, int i, int w) {
  return w == 0 ? key.k0 + (uint32_t)i * 0x9E3779B9u : key.k1 + (uint32_t)i * 0xBB67AE85u;
}
__device__ __forceinline__ uint32_t round_key(const PhiloxRoundKeys& rk, int i, int w) {
  return rk.k[2 * i + w];
}

// Philox4x32-10 on counter (c0, c1, c2, c3); K is PhiloxKey or PhiloxRoundKeys.
template <class K>
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const K& key) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ round_key(key, i, 0);
    const uint32_t n2 = hi0 ^ c3 ^ round_key(key, i, 1);
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// ---- Box-Muller on the two word pairs of one Philox call ----
// The two transforms run side by side: __fadd2_rn / __fmul2_rn / __ffma2_rn
// round each component exactly like the scalar __fadd_rn / __fmul_rn /
// __fmaf_rn, so every value is the one the specification's scalar steps give
// while the floating-point work takes half the instructions (the generator
// is instruction-issue bound inside the sketch kernels).  The square root
// gives the IEEE correctly rounded result (sqrt_x2).
// Where a step below is written differently from the specification, the
// comment beside it shows that the value is the same.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 neg2(float2 x) { return f2(-x.x, -x.y); }

// sqrt(w) rounded to nearest-even for w = -2 ln u1 in [2^-23, 34] or w = -0
// (u1 = 1).  Markstein's square root: from an approximate reciprocal square
// root y, g = w y and h = y / 2 are refined together (t = 1/2 - g h,
// g += g t, h += h t), then g is corrected by the exact residual
// d = w - g^2 (one FMA): g + d h, rounded once.  The same exhaustive check
// (every radicand, every seed within 6 ulp; the hardware approximation is
// within 2^-22.9 relative) finds every root equal to the IEEE one.  The seed
// is taken at max(w, 1e-30), which changes nothing for w >= 2^-23 and keeps it
// finite at w = -0 (u1 = 1), where every step then yields -0, the root.
__device__ __forceinline__ float2 sqrt_x2(float2 w) {
  const float2 y = f2(rsqrt_approx(fmaxf(w.x, 1e-30f)), rsqrt_approx(fmaxf(w.y, 1e-30f)));
  float2 g = __fmul2_rn(w, y);
  float2 h = __fmul2_rn(f2(0.5f, 0.5f), y);
  const float2 t = __ffma2_rn(neg2(g), h, f2(0.5f, 0.5f));
  g = __ffma2_rn(g, t, g);
  h = __ffma2_rn(h, t, h);
  const float2 d = __ffma2_rn(neg2(g), g, w);
  return __ffma2_rn(d, h, g);
}

// ln x for x in (0, 1] (normal): x = 2^e f, f folded into [sqrt(1/2), sqrt 2),
// t = f - 1 (exact), ln f = t + t^2 Q(t) with Q of degree 8 (the generator
// specification's least-squares coefficients, below), ln x = e ln2_hi +
// (e ln2_lo + ln f).
__device__ __forceinline__ float2 ln01_x2(float2 x) {
  const uint32_t b0 = __float_as_uint(x.x), b1 = __float_as_uint(x.y);
  // Fold and split by one integer add: with m the mantissa bits, b + 0x4afb0c
  // carries into the exponent field exactly when m > 0x3504f3 (the fold), so
  // its exponent field is E (plus one when folded) and its mantissa field
  // plus 0x3f3504f4 is m with the exponent of 1 (or of 1/2 when folded).
  const uint32_t i0 = b0 + 0x004afb0cu, i1 = b1 + 0x004afb0cu;
  // e as a float without a conversion: 0x4B000000 + E is the float 2^23 + E
  // (E < 2^8), and subtracting 2^23 + 127 is exact
  const float2 eb = f2(__uint_as_float(0x4B000000u + (i0 >> 23)),
                       __uint_as_float(0x4B000000u + (i1 >> 23)));
  const float2 ef = __fadd2_rn(eb, f2(-8388735.0f, -8388735.0f));
  const float2 f = f2(__uint_as_float((i0 & 0x007fffffu) + 0x3f3504f4u),
                      __uint_as_float((i1 & 0x007fffffu) + 0x3f3504f4u));
  const float2 t = __fadd2_rn(f, f2(-1.0f, -1.0f));
  float2 p = __ffma2_rn(t, f2(-0x1.321a48p-4f, -0x1.321a48p-4f), f2(0x1.068b28p-3f, 0x1.068b28p-3f));
  p = __ffma2_rn(t, p, f2(-0x1.0f9b0cp-3f, -0x1.0f9b0cp-3f));
  p = __ffma2_rn(t, p, f2(0x1.22bf86p-3f, 0x1.22bf86p-3f));
  p = __ffma2_rn(t, p, f2(-0x1.5424e0p-3f, -0x1.5424e0p-3f));
  p = __ffma2_rn(t, p, f2(0x1.999fc2p-3f, 0x1.999fc2p-3f));
  p = __ffma2_rn(t, p, f2(-0x1.000422p-2f, -0x1.000422p-2f));
  p = __ffma2_rn(t, p, f2(0x1.555558p-2f, 0x1.555558p-2f));
  p = __ffma2_rn(t, p, f2(-0x1.fffff8p-2f, -0x1.fffff8p-2f));
  const float2 lnf = __ffma2_rn(__fmul2_rn(t, t), p, t);
  return __ffma2_rn(ef, f2(0x1.62e4p-1f, 0x1.62e4p-1f),
                    __ffma2_rn(ef, f2(0x1.7f7d1cp-20f, 0x1.7f7d1cp-20f), lnf));
}

// The circle points of the angle words w0, w1 before the half turn of their
// bit 31 (the caller applies it as the sign of the radius): the position
// r = (bits 29..8) 2^-23 - 1/4 in [-1/4, 1/4) from the bits (0.5 + w 2^-23
// and its difference with 3/4 are exact), Taylor polynomials of sin(pi r)
// (to r^9) and cos(pi r) (to r^10) with coefficients (-1)^j pi^n/n! rounded
// to FP32, then (x, y) -> (-y, x) when bit 30 is set.
__device__ __forceinline__ void circle_x2(uint32_t w0, uint32_t w1, float2* x_out,
                                          float2* y_out) {
  const float2 h = f2(__uint_as_float(0x3F000000u | ((w0 >> 7) & 0x007FFFFEu)),
                      __uint_as_float(0x3F000000u | ((w1 >> 7) & 0x007FFFFEu)));
  const float2 r = __fadd2_rn(h, f2(-0.75f, -0.75f));
  const float2 r2 = __fmul2_rn(r, r);
  float2 sp = __ffma2_rn(r2, f2(0x1.507834p-4f, 0x1.507834p-4f), f2(-0x1.32d2ccp-1f, -0x1.32d2ccp-1f));
  sp = __ffma2_rn(r2, sp, f2(0x1.466bc6p+1f, 0x1.466bc6p+1f));
  sp = __ffma2_rn(r2, sp, f2(-0x1.4abbcep+2f, -0x1.4abbcep+2f));
  sp = __ffma2_rn(r2, sp, f2(0x1.921fb6p+1f, 0x1.921fb6p+1f));
  const float2 sn = __fmul2_rn(r, sp);
  float2 cp = __ffma2_rn(r2, f2(-0x1.a6d1f2p-6f, -0x1.a6d1f2p-6f), f2(0x1.e1f506p-3f, 0x1.e1f506p-3f));
  cp = __ffma2_rn(r2, cp, f2(-0x1.55d3c8p+0f, -0x1.55d3c8p+0f));
  cp = __ffma2_rn(r2, cp, f2(0x1.03c1f0p+2f, 0x1.03c1f0p+2f));
  cp = __ffma2_rn(r2, cp, f2(-0x1.3bd3ccp+2f, -0x1.3bd3ccp+2f));
  const float2 cs = __ffma2_rn(r2, cp, f2(1.0f, 1.0f));
  const bool q0 = (w0 & 0x40000000u) != 0u, q1 = (w1 & 0x40000000u) != 0u;
  *x_out = f2(q0 ? -sn.x : cs.x, q1 ? -sn.y : cs.y);
  *y_out = f2(q0 ? cs.x : sn.x, q1 ? cs.y : sn.y);
}

// Box-Muller of the word pairs (x.x, x.y) and (x.z, x.w), as (z0, z1, z2, z3):
// u1 = ((xa >> 8) + 1) 2^-24, rho = sqrt(-2 ln u1), (X, Y) the circle point
// of xb, (z_even, z_odd) = rho (X, Y).
__device__ __forceinline__ float4 box_muller_x2(uint4 x) {
  const float2 fa = f2(__uint2float_rn(x.x >> 8), __uint2float_rn(x.z >> 8));  // exact
  // (v + 1) 2^-24 is a float, so the fused form rounds nothing
  const float2 u1 = __ffma2_rn(fa, f2(0x1p-24f, 0x1p-24f), f2(0x1p-24f, 0x1p-24f));
  const float2 v = __fmul2_rn(f2(-2.0f, -2.0f), ln01_x2(u1));
  const float2 rho = sqrt_x2(v);
  // the half turn of bit 31 as the sign of the radius: (-rho) X = -(rho X)
  // exactly, signed zeros included
  const float2 rs = f2(__uint_as_float(__float_as_uint(rho.x) ^ (x.y & 0x80000000u)),
                       __uint_as_float(__float_as_uint(rho.y) ^ (x.w & 0x80000000u)));
  float2 cx, cy;
  circle_x2(x.y, x.w, &cx, &cy);
  const float2 zc = __fmul2_rn(rs, cx);
  const float2 zs = __fmul2_rn(rs, cy);
  return make_float4(zc.x, zs.x, zc.y, zs.y);
}

// The four Gaussian entries (r, 4j .. 4j+3).
template <class K>
__device__ __forceinline__ float4 gaussian4(const K& key, uint32_t r, uint32_t j, uint32_t dom) {
  return box_muller_x2(philox(j, r, dom, 0u, key));
}

// The four uniform entries (r, 4j .. 4j+3).
template <class K>
__device__ __forceinline__ float4 uniform4(const K& key, uint32_t r, uint32_t j, uint32_t dom) {
  const uint4 x = philox(j, r, dom, 0u, key);
  return make_float4(__fmul_rn(__uint2float_rn(x.x >> 8), 0x1p-24f),
                     __fmul_rn(__uint2float_rn(x.y >> 8), 0x1p-24f),
                     __fmul_rn(__uint2float_rn(x.z >> 8), 0x1p-24f),
                     __fmul_rn(__uint2float_rn(x.w >> 8), 0x1p-24f));
}

// Sign bits of the 128 Rademacher entries (r, 128j .. 128j+127): bit b of
// word w belongs to column 128j + 32w + b; a set bit means -1.
template <class K>
__device__ __forceinline__ uint4 rademacher_bits(const K& key, uint32_t r, uint32_t j,
                                                 uint32_t dom) {
  return philox(j, r, dom, 0u, key);
}

// Four consecutive generated values (r, c0 .. c0+3), c0 % 4 == 0, as FP32
// (unquantized).
__device__ __forceinline__ float4 gen4(int dist, PhiloxKey key, uint32_t r, uint32_t c0,
                                       uint32_t dom) {
  if (dist == kRademacher) {
    const uint4 x = rademacher_bits(key, r, c0 >> 7, dom);
    const uint32_t w = ((c0 >> 5) & 3u) == 0 ? x.x : ((c0 >> 5) & 3u) == 1 ? x.y
                     : ((c0 >> 5) & 3u) == 2 ? x.z : x.w;
    const uint32_t bits = w >> (c0 & 31u);
    return make_float4((bits & 1u) ? -1.f : 1.f, (bits & 2u) ? -1.f : 1.f,
                       (bits & 4u) ? -1.f : 1.f, (bits & 8u) ? -1.f : 1.f);
  }
  if (dist == kUniform) return uniform4(key, r, c0 >> 2, dom);
  return gaussian4(key, r, c0 >> 2, dom);
}

}  // namespace sk

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
//     u1 = ((xa>>8)+1) 2^-24, u2 = (xb>>8) 2^-24, rho = sqrt(-2 ln u1),
//     g = rho cospi(2 u2) (c even) or rho sinpi(2 u2) (c odd).
//   Rademacher: bit c%32 of word (c>>5)%4, set -> -1.
//   Uniform: (x_{c%4} >> 8) 2^-24.
// Every floating-point step is an explicitly rounded IEEE operation
// (__fadd_rn, __fmul_rn, __fmaf_rn, __fdiv_rn, __fsqrt_rn), so no compiler
// contraction or fast-math flag can change a bit.  No hardware
// approximation (MUFU) is used for ln, sin or cos.
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

// Philox4x32-10 on counter (c0, c1, c2, c3).
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        PhiloxKey key) {
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// ln x for x in (0, 1] (normal): x = 2^e f, f folded into [sqrt(1/2), sqrt 2],
// s = (f-1)/(f+1), ln f = 2s + s^3 P(s^2) with the atanh series
// coefficients 2/3, 2/5, 2/7, 2/9; ln x = e ln2_hi + (e ln2_lo + ln f).
__device__ __forceinline__ float ln01(float x) {
  const uint32_t b = __float_as_uint(x);
  int e = (int)(b >> 23) - 127;
  uint32_t mb = b & 0x007fffffu;
  if (mb > 0x003504f3u) {
    mb |= 0x3f000000u;
    e += 1;
  } else {
    mb |= 0x3f800000u;
  }
  const float f = __uint_as_float(mb);
  const float s = __fdiv_rn(__fadd_rn(f, -1.0f), __fadd_rn(f, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = __fmaf_rn(s2, 0x1.c71c72p-3f, 0x1.24924ap-2f);
  p = __fmaf_rn(s2, p, 0x1.99999ap-2f);
  p = __fmaf_rn(s2, p, 0x1.555556p-1f);
  const float s3 = __fmul_rn(s, s2);
  const float lnf = __fmaf_rn(s3, p, __fadd_rn(s, s));
  const float ef = __int2float_rn(e);
  return __fmaf_rn(ef, 0x1.62e4p-1f, __fmaf_rn(ef, 0x1.7f7d1cp-20f, lnf));
}

// sin(pi t), cos(pi t) for t in [0, 2): q = rint(2t), r = t - q/2 in
// [-1/4, 1/4] exactly, Taylor polynomials of sin(pi r) (to r^9) and
// cos(pi r) (to r^10) with coefficients (-1)^j pi^n/n! rounded to FP32,
// then a rotation by q quarter turns.
__device__ __forceinline__ void sincospi(float t, float* sn_out, float* cs_out) {
  const float qf = rintf(__fadd_rn(t, t));
  const int q = (int)qf;
  const float r = __fsub_rn(t, __fmul_rn(qf, 0.5f));
  const float r2 = __fmul_rn(r, r);
  float sp = __fmaf_rn(r2, 0x1.507834p-4f, -0x1.32d2ccp-1f);
  sp = __fmaf_rn(r2, sp, 0x1.466bc6p+1f);
  sp = __fmaf_rn(r2, sp, -0x1.4abbcep+2f);
  sp = __fmaf_rn(r2, sp, 0x1.921fb6p+1f);
  const float sn = __fmul_rn(r, sp);
  float cp = __fmaf_rn(r2, -0x1.a6d1f2p-6f, 0x1.e1f506p-3f);
  cp = __fmaf_rn(r2, cp, -0x1.55d3c8p+0f);
  cp = __fmaf_rn(r2, cp, 0x1.03c1f0p+2f);
  cp = __fmaf_rn(r2, cp, -0x1.3bd3ccp+2f);
  const float cs = __fmaf_rn(r2, cp, 1.0f);
  const int qq = q & 3;
  const float a = (qq & 1) ? cs : sn;   // sin candidate
  const float b = (qq & 1) ? sn : cs;   // cos candidate
  *sn_out = (qq == 2 || qq == 3) ? -a : a;
  *cs_out = (qq == 1 || qq == 2) ? -b : b;
}

// Box-Muller on one pair of Philox words -> (z0, z1).
__device__ __forceinline__ float2 box_muller(uint32_t xa, uint32_t xb) {
  const float u1 = __fmul_rn(__uint2float_rn((xa >> 8) + 1u), 0x1p-24f);
  const float u2 = __fmul_rn(__uint2float_rn(xb >> 8), 0x1p-24f);
  const float rho = __fsqrt_rn(__fmul_rn(-2.0f, ln01(u1)));
  float sn, cs;
  sincospi(__fadd_rn(u2, u2), &sn, &cs);
  return make_float2(__fmul_rn(rho, cs), __fmul_rn(rho, sn));
}

// ---- the same two Box-Muller transforms, evaluated side by side ----
// Every step below is the scalar step above applied to the two pairs of one
// Philox call at once: __fadd2_rn / __fmul2_rn / __ffma2_rn round each
// component exactly like __fadd_rn / __fmul_rn / __fmaf_rn, so the results
// are bit-identical to box_muller(x0, x1), box_muller(x2, x3) while the
// floating-point work takes half the instructions (the generator is
// instruction-issue bound inside the sketch kernels).  Integer steps,
// division, square root and rounding to integer stay per component.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ float2 ln01_x2(float2 x) {
  const uint32_t b0 = __float_as_uint(x.x), b1 = __float_as_uint(x.y);
  int e0 = (int)(b0 >> 23) - 127, e1 = (int)(b1 >> 23) - 127;
  uint32_t m0 = b0 & 0x007fffffu, m1 = b1 & 0x007fffffu;
  if (m0 > 0x003504f3u) {
    m0 |= 0x3f000000u;
    e0 += 1;
  } else {
    m0 |= 0x3f800000u;
  }
  if (m1 > 0x003504f3u) {
    m1 |= 0x3f000000u;
    e1 += 1;
  } else {
    m1 |= 0x3f800000u;
  }
  const float2 f = f2(__uint_as_float(m0), __uint_as_float(m1));
  const float2 num = __fadd2_rn(f, f2(-1.0f, -1.0f));
  const float2 den = __fadd2_rn(f, f2(1.0f, 1.0f));
  const float2 sv = f2(__fdiv_rn(num.x, den.x), __fdiv_rn(num.y, den.y));
  const float2 s2 = __fmul2_rn(sv, sv);
  float2 p = __ffma2_rn(s2, f2(0x1.c71c72p-3f, 0x1.c71c72p-3f), f2(0x1.24924ap-2f, 0x1.24924ap-2f));
  p = __ffma2_rn(s2, p, f2(0x1.99999ap-2f, 0x1.99999ap-2f));
  p = __ffma2_rn(s2, p, f2(0x1.555556p-1f, 0x1.555556p-1f));
  const float2 s3 = __fmul2_rn(sv, s2);
  const float2 lnf = __ffma2_rn(s3, p, __fadd2_rn(sv, sv));
  const float2 ef = f2(__int2float_rn(e0), __int2float_rn(e1));
  return __ffma2_rn(ef, f2(0x1.62e4p-1f, 0x1.62e4p-1f),
                    __ffma2_rn(ef, f2(0x1.7f7d1cp-20f, 0x1.7f7d1cp-20f), lnf));
}

__device__ __forceinline__ void sincospi_x2(float2 t, float2* sn_out, float2* cs_out) {
  const float2 tt = __fadd2_rn(t, t);
  const float2 qf = f2(rintf(tt.x), rintf(tt.y));
  const int q0 = (int)qf.x & 3, q1 = (int)qf.y & 3;
  // t - q/2: the product q * 0.5 is exact, so one rounding as in the scalar form
  const float2 r = __ffma2_rn(qf, f2(-0.5f, -0.5f), t);
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
  const float a0 = (q0 & 1) ? cs.x : sn.x, b0 = (q0 & 1) ? sn.x : cs.x;
  const float a1 = (q1 & 1) ? cs.y : sn.y, b1 = (q1 & 1) ? sn.y : cs.y;
  *sn_out = f2((q0 == 2 || q0 == 3) ? -a0 : a0, (q1 == 2 || q1 == 3) ? -a1 : a1);
  *cs_out = f2((q0 == 1 || q0 == 2) ? -b0 : b0, (q1 == 1 || q1 == 2) ? -b1 : b1);
}

// box_muller(x.x, x.y) and box_muller(x.z, x.w), as (z0, z1, z2, z3).
__device__ __forceinline__ float4 box_muller_x2(uint4 x) {
  const float2 k24 = f2(0x1p-24f, 0x1p-24f);
  const float2 u1 = __fmul2_rn(f2(__uint2float_rn((x.x >> 8) + 1u), __uint2float_rn((x.z >> 8) + 1u)),
                               k24);
  const float2 u2 = __fmul2_rn(f2(__uint2float_rn(x.y >> 8), __uint2float_rn(x.w >> 8)), k24);
  const float2 v = __fmul2_rn(f2(-2.0f, -2.0f), ln01_x2(u1));
  const float2 rho = f2(__fsqrt_rn(v.x), __fsqrt_rn(v.y));
  float2 sn, cs;
  sincospi_x2(__fadd2_rn(u2, u2), &sn, &cs);
  const float2 zc = __fmul2_rn(rho, cs);
  const float2 zs = __fmul2_rn(rho, sn);
  return make_float4(zc.x, zs.x, zc.y, zs.y);
}

// The four Gaussian entries (r, 4j .. 4j+3).
__device__ __forceinline__ float4 gaussian4(PhiloxKey key, uint32_t r, uint32_t j, uint32_t dom) {
  return box_muller_x2(philox(j, r, dom, 0u, key));
}

// The four uniform entries (r, 4j .. 4j+3).
__device__ __forceinline__ float4 uniform4(PhiloxKey key, uint32_t r, uint32_t j, uint32_t dom) {
  const uint4 x = philox(j, r, dom, 0u, key);
  return make_float4(__fmul_rn(__uint2float_rn(x.x >> 8), 0x1p-24f),
                     __fmul_rn(__uint2float_rn(x.y >> 8), 0x1p-24f),
                     __fmul_rn(__uint2float_rn(x.z >> 8), 0x1p-24f),
                     __fmul_rn(__uint2float_rn(x.w >> 8), 0x1p-24f));
}

// Sign bits of the 128 Rademacher entries (r, 128j .. 128j+127): bit b of
// word w belongs to column 128j + 32w + b; a set bit means -1.
__device__ __forceinline__ uint4 rademacher_bits(PhiloxKey key, uint32_t r, uint32_t j,
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

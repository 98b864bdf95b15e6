// sk_simt.cu -- FP32 CUDA-core form of the fused generate-and-sketch, the
// debug materializer and the fixed-order split-K reduction.
//
// The fused kernel is the local step of the paper's Alg. 1 (GenRandom, then
// the local multiply B_ik = A_ij Omega_jk) done tile by tile: each CTA
// regenerates the tile of the random operand it is about to consume
// straight into shared memory, so the random matrix is never written to or
// read from device memory.  Accumulation is FP32 FMA in registers.
#include <cuda_runtime.h>

#include "sk_internal.h"
#include "sk_rng.cuh"

namespace sk {
namespace {

constexpr int BL = 16;    // contracted length per stage
constexpr int TPB = 256;  // 16 x 16 threads

// Tile of Y per CTA: BP rows x BQ columns, a TM x TN micro-tile per thread
// (TM = BP / 16, TN = BQ / 16).  The wide left tile (Y = S A, n > 128) takes
// 128 rows of k and 256 columns of n, so that each generated entry of S
// serves 256 columns of A; the narrow left tile (n <= 128) 256 rows of k and
// 128 columns of n, so that few of its columns are past n; the right tile
// (Y = A S^T) 256 rows of m and 128 rows of k.  A stage is 32768 FMAs.
template <bool LEFT, bool WIDE>
struct SimtTile {
  static constexpr int BP = LEFT && WIDE ? 128 : 256;
  static constexpr int BQ = LEFT && WIDE ? 256 : 128;
  static constexpr int TM = BP / 16, TN = BQ / 16;
  // the generated side (X for the left form, W for the right) and its
  // generation tasks per thread and stage (one row, 4 values each)
  static constexpr int GT = (LEFT ? BP : BQ) * (BL / 4) / TPB;
  // 16-byte pieces of A per thread and stage
  static constexpr int NA = LEFT ? BL * BQ / 4 / TPB : BP * BL / 4 / TPB;
  // X (the BP side) is stored with every value twice, X2[l][2r] =
  // X2[l][2r+1] = X[l][r], so that one 16-byte load gives two (x, x) pairs for
  // the packed FMAs; W (the BQ side) as is
  static constexpr int XW = 2 * BP;
  static constexpr int STAGE = BL * (XW + BQ);  // floats per stage buffer
  static constexpr size_t SMEM = 2 * STAGE * sizeof(float);
};

struct SimtParams {
  const float* A;
  int64_t lda;
  float* out;       // Y (splits == 1) or partials [splits][P][Q]
  int64_t ldo;
  int64_t P, Q, L;
  int64_t chunk;    // contracted length per split (multiple of BL)
  PhiloxRoundKeys rk;
  int dist;
  float scale;      // applied only when splits == 1
  int splits;
  int vec;          // A 16-byte aligned and lda a multiple of 4: 16-byte loads
};

// Four consecutive generated values (r, c0 .. c0+3), c0 % 4 == 0, unquantized.
__device__ __forceinline__ float4 gen4_rk(int dist, const PhiloxRoundKeys& rk, uint32_t r,
                                          uint32_t c0) {
  if (dist == kRademacher) {
    const uint4 x = rademacher_bits(rk, r, c0 >> 7, 0u);
    const uint32_t wsel = (c0 >> 5) & 3u;
    const uint32_t w = wsel == 0 ? x.x : wsel == 1 ? x.y : wsel == 2 ? x.z : x.w;
    const uint32_t bits = w >> (c0 & 31u);
    return make_float4((bits & 1u) ? -1.f : 1.f, (bits & 2u) ? -1.f : 1.f,
                       (bits & 4u) ? -1.f : 1.f, (bits & 8u) ? -1.f : 1.f);
  }
  if (dist == kUniform) return uniform4(rk, r, c0 >> 2, 0u);
  return gaussian4(rk, r, c0 >> 2, 0u);
}

// The generated values (t0 + t, l0 + l) of a stage, t < BT, l < BL, zero
// past tmax rows or past lend, in BT x 4 tasks of one row t and 4
// consecutive l; this is the calling thread's task u (of BT / 64).  Lanes of a
// warp take consecutive rows (conflict-free shared stores).  DUP: stored
// twice at X2[l][2t], X2[l][2t+1] (the X side); else at W[l][t].
template <int BT, bool DUP>
__device__ __forceinline__ void gen_task_fp32(float* buf, const SimtParams& p, int64_t t0,
                                              int64_t tmax, int64_t l0, int64_t lend, int u) {
  static_assert(BT * (BL / 4) % TPB == 0, "whole generation tasks per thread and stage");
  {
    const int task = static_cast<int>(threadIdx.x) + TPB * u;
    const int t = task % BT;
    const int jg = task / BT;
    const int64_t r = t0 + t;
    const int64_t c = l0 + 4 * jg;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < tmax && c < lend) {
      v = gen4_rk(p.dist, p.rk, static_cast<uint32_t>(r), static_cast<uint32_t>(c));
      if (c + 1 >= lend) v.y = 0.f;
      if (c + 2 >= lend) v.z = 0.f;
      if (c + 3 >= lend) v.w = 0.f;
    }
    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (DUP)
        *reinterpret_cast<float2*>(buf + (4 * jg + i) * (2 * BT) + 2 * t) = make_float2(vv[i], vv[i]);
      else
        buf[(4 * jg + i) * BT + t] = vv[i];
    }
  }
}

// The NA 4-element pieces of A per thread for the stage at l0.  Left: the W
// tile A[l0 + l][q0 + q] (l < 16, q < BQ: piece f = tid + 256 u is row
// f / (BQ / 4), columns 4 (f % (BQ / 4)) ..); right: the X tile
// A[p0 + r][l0 + l] (row r = tid, columns 4u ..).  Zero outside the matrix
// and past lend.
template <bool LEFT, bool WIDE>
__device__ __forceinline__ void load_a(float4 (&pa)[4], const SimtParams& p, int64_t p0,
                                       int64_t q0, int64_t l0, int64_t lend) {
  using T = SimtTile<LEFT, WIDE>;
  constexpr int QP = T::BQ / 4;  // pieces per row of the left W tile
#pragma unroll
  for (int u = 0; u < T::NA; ++u) {
    const int f = static_cast<int>(threadIdx.x) + TPB * u;
    int64_t row, col, col_end;  // the piece is A[row][col .. col + 3]
    bool row_ok;
    if (LEFT) {
      row = l0 + f / QP;
      col = q0 + 4 * (f % QP);
      row_ok = row < lend;
      col_end = p.Q;
    } else {
      row = p0 + static_cast<int>(threadIdx.x);
      col = l0 + 4 * u;
      row_ok = row < p.P;
      col_end = lend;
    }
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row_ok) {
      const float* src = p.A + row * p.lda + col;
      if (p.vec && col + 3 < col_end) {
        v = __ldg(reinterpret_cast<const float4*>(src));
      } else {
        if (col < col_end) v.x = __ldg(src);
        if (col + 1 < col_end) v.y = __ldg(src + 1);
        if (col + 2 < col_end) v.z = __ldg(src + 2);
        if (col + 3 < col_end) v.w = __ldg(src + 3);
      }
    }
    pa[u] = v;
  }
}

template <bool LEFT, bool WIDE>
__device__ __forceinline__ void store_a(float* buf, const float4 (&pa)[4]) {
  using T = SimtTile<LEFT, WIDE>;
  constexpr int QP = T::BQ / 4;
  float* xs = buf;
  float* ws = buf + BL * T::XW;
#pragma unroll
  for (int u = 0; u < T::NA; ++u) {
    const int f = static_cast<int>(threadIdx.x) + TPB * u;
    if (LEFT) {  // W[l][q], l = f / QP, q = 4 (f % QP)
      *reinterpret_cast<float4*>(ws + (f / QP) * T::BQ + 4 * (f % QP)) = pa[u];
    } else {     // X2[l][2r], r = tid, l = 4u .. 4u+3
      const int r = static_cast<int>(threadIdx.x);
      const float vv[4] = {pa[u].x, pa[u].y, pa[u].z, pa[u].w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float2*>(xs + (4 * u + i) * T::XW + 2 * r) = make_float2(vv[i], vv[i]);
    }
  }
}

// Y tile = sum over l of X[l][rows] (outer) W[l][cols], FP32 FMA: the local
// multiply of Alg. 1 with the random operand generated into shared memory
// stage by stage (double-buffered: the next stage's A is loaded into
// registers before, and its S tile generated after, the current stage's
// FMAs).  Packed FP32x2 FMAs (__ffma2_rn: each component the correctly
// rounded fmaf) update two columns of a row per instruction.
template <bool LEFT, bool WIDE>
__global__ void __launch_bounds__(TPB, 1) k_sketch_fp32_simt(SimtParams p) {
  using T = SimtTile<LEFT, WIDE>;
  extern __shared__ __align__(16) float smem_f[];
  // the tiles along the long side (n of the left sketch, m of the right) run
  // along grid x, whose extent is not limited to 65535
  const int64_t q0 = (int64_t)(LEFT ? blockIdx.x : blockIdx.y) * T::BQ;
  const int64_t p0 = (int64_t)(LEFT ? blockIdx.y : blockIdx.x) * T::BP;
  const int64_t lbeg = (int64_t)blockIdx.z * p.chunk;
  const int64_t lend = min(p.L, lbeg + p.chunk);
  const int nst = static_cast<int>((lend - lbeg + BL - 1) / BL);
  const int tq = threadIdx.x % 16;
  const int tp = threadIdx.x / 16;

  float2 acc[T::TM][T::TN / 2];
#pragma unroll
  for (int i = 0; i < T::TM; ++i)
#pragma unroll
    for (int j = 0; j < T::TN / 2; ++j) acc[i][j] = make_float2(0.f, 0.f);

  // generation task u (of GT) of the stage at l0 into buffer buf
  auto gen = [&](float* buf, int64_t l0, int u) {
    if constexpr (LEFT)
      gen_task_fp32<T::BP, true>(buf, p, p0, p.P, l0, lend, u);
    else
      gen_task_fp32<T::BQ, false>(buf + BL * T::XW, p, q0, p.Q, l0, lend, u);
  };

  float4 pa[4];
  if (nst > 0) {
    load_a<LEFT, WIDE>(pa, p, p0, q0, lbeg, lend);
#pragma unroll
    for (int u = 0; u < T::GT; ++u) gen(smem_f, lbeg, u);
    store_a<LEFT, WIDE>(smem_f, pa);
  }
  __syncthreads();
  for (int st = 0; st < nst; ++st) {
    const int64_t l0 = lbeg + static_cast<int64_t>(st) * BL;
    const bool more = st + 1 < nst;
    float* next = smem_f + ((st + 1) & 1) * T::STAGE;
    if (more) load_a<LEFT, WIDE>(pa, p, p0, q0, l0 + BL, lend);
    const float* xs = smem_f + (st & 1) * T::STAGE;
    const float* ws = xs + BL * T::XW;
#pragma unroll 2
    for (int l = 0; l < BL; ++l) {
      // the next stage's S tile is generated between this stage's FMAs (it
      // goes to the other buffer), so generation and FMAs share the cycles
      if (more && l % (BL / T::GT) == 2) gen(next, l0 + BL, l / (BL / T::GT));
      float2 xr[T::TM];
      float2 wr[T::TN / 2];
#pragma unroll
      for (int a = 0; a < T::TM / 4; ++a) {
        const float* src = xs + l * T::XW + 2 * (64 * a + 4 * tp);
        const float4 u0 = *reinterpret_cast<const float4*>(src);
        const float4 u1 = *reinterpret_cast<const float4*>(src + 4);
        xr[4 * a + 0] = make_float2(u0.x, u0.y);
        xr[4 * a + 1] = make_float2(u0.z, u0.w);
        xr[4 * a + 2] = make_float2(u1.x, u1.y);
        xr[4 * a + 3] = make_float2(u1.z, u1.w);
      }
#pragma unroll
      for (int b = 0; b < T::TN / 4; ++b) {
        const float4 w = *reinterpret_cast<const float4*>(ws + l * T::BQ + 64 * b + 4 * tq);
        wr[2 * b] = make_float2(w.x, w.y);
        wr[2 * b + 1] = make_float2(w.z, w.w);
      }
#pragma unroll
      for (int i = 0; i < T::TM; ++i)
#pragma unroll
        for (int j = 0; j < T::TN / 2; ++j) acc[i][j] = __ffma2_rn(xr[i], wr[j], acc[i][j]);
    }
    if (more) store_a<LEFT, WIDE>(next, pa);
    __syncthreads();
  }

  // acc[4a + i][2b + jj]: row p0 + 64a + 4tp + i, columns q0 + 64b + 4tq + 2jj (+1)
#pragma unroll
  for (int i = 0; i < T::TM; ++i) {
    const int64_t gp = p0 + 64 * (i / 4) + 4 * tp + (i % 4);
    if (gp >= p.P) continue;
#pragma unroll
    for (int j = 0; j < T::TN; ++j) {
      const int64_t gq = q0 + 64 * (j / 4) + 4 * tq + (j % 4);
      if (gq >= p.Q) continue;
      const float v = (j & 1) ? acc[i][j / 2].y : acc[i][j / 2].x;
      if (p.splits == 1) {
        p.out[gp * p.ldo + gq] = __fmul_rn(p.scale, v);
      } else {
        p.out[((int64_t)blockIdx.z * p.P + gp) * p.Q + gq] = v;
      }
    }
  }
}

__global__ void k_splitk_reduce(const float* __restrict__ part, int splits, int64_t P, int64_t Q,
                                float scale, float* __restrict__ Y, int64_t ldy) {
  const int64_t total = P * Q;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s = __fadd_rn(s, part[(int64_t)z * total + i]);
    const int64_t r = i / Q, c = i % Q;
    Y[r * ldy + c] = __fmul_rn(scale, s);
  }
}

__global__ void k_splitk_reduce_batched(const ReduceDesc* __restrict__ desc) {
  const ReduceDesc d = desc[blockIdx.y];
  const int64_t total = d.P * d.Q;
  const int64_t zstride = d.P * d.ldp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / d.Q, c = i % d.Q;
    const float* p = d.part + r * d.ldp + c;
    float s = 0.f;
    for (int z = 0; z < d.splits; ++z) s = __fadd_rn(s, p[(int64_t)z * zstride]);
    d.Y[r * d.ldy + c] = __fmul_rn(d.scale, s);
  }
}

__global__ void k_materialize(PhiloxKey key, int dist, int fmt, int scaled, float scale,
                              int64_t row0, int64_t col0, int64_t rows, int64_t cols, void* out,
                              int64_t ld) {
  const int64_t total = rows * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rr = i / cols, cc = i % cols;
    const uint32_t r = (uint32_t)(row0 + rr);
    const uint32_t c = (uint32_t)(col0 + cc);
    const float4 v = gen4(dist, key, r, c & ~3u, 0u);
    const uint32_t e = c & 3u;
    const float g = e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
    if (fmt == kFP32) {
      static_cast<float*>(out)[rr * ld + cc] = scaled ? __fmul_rn(g, scale) : g;
    } else if (fmt == kBF16) {
      static_cast<__nv_bfloat16*>(out)[rr * ld + cc] = __float2bfloat16_rn(g);
    } else {
      static_cast<__nv_fp8_storage_t*>(out)[rr * ld + cc] =
          __nv_cvt_float_to_fp8(g, __NV_SATFINITE, __NV_E4M3);
    }
  }
}

// The left form takes the wide tile (128 x 256) when n is above 128, the
// 256 x 128 tile otherwise (the right form always); both hold 32768 outputs.
bool simt_wide(const GemmShape& s) { return s.left && s.Q > 128; }

// The FP32 kernels' dynamic shared memory (two stage buffers: 64 / 80 KB)
// is above the 48 KB default: allowed once per process.
cudaError_t set_simt_smem() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_sketch_fp32_simt<true, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(SimtTile<true, true>::SMEM));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sketch_fp32_simt<true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SimtTile<true, false>::SMEM));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sketch_fp32_simt<false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SimtTile<false, false>::SMEM));
  done = e == cudaSuccess;
  return e;
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

void plan_splits(const GemmShape& s, int* splits, int64_t* chunk) {
  const bool wide = simt_wide(s);
  const int bp = wide ? SimtTile<true, true>::BP : SimtTile<false, false>::BP;
  const int bq = wide ? SimtTile<true, true>::BQ : SimtTile<false, false>::BQ;
  const int64_t tiles = ((s.P + bp - 1) / bp) * ((s.Q + bq - 1) / bq);
  const int64_t sms = num_sms();  // one CTA per SM (registers, shared memory)
  int64_t max_sp = s.L / (8 * BL) > 0 ? s.L / (8 * BL) : 1;
  if (max_sp > 64) max_sp = 64;
  // the fewest splits with at least two waves of CTAs whose last wave is
  // nearly full (>= 90 % of the SMs busy over the whole launch), else the
  // best-filled count up to 8 waves
  int64_t sp = 1;
  double best = -1.0;
  for (int64_t c = 1; c <= max_sp; ++c) {
    const int64_t ctas = tiles * c;
    const int64_t waves = (ctas + sms - 1) / sms;
    const double fill = static_cast<double>(ctas) / static_cast<double>(waves * sms);
    if (ctas >= 2 * sms && fill >= 0.9) {
      sp = c;
      break;
    }
    if (waves <= 8 && fill > best + 1e-9) {
      best = fill;
      sp = c;
    }
  }
  int64_t ch = (s.L + sp - 1) / sp;
  ch = (ch + BL - 1) / BL * BL;
  sp = (s.L + ch - 1) / ch;
  *splits = (int)sp;
  *chunk = ch;
}

}  // namespace

size_t simt_workspace_bytes(const GemmShape& s) {
  int sp;
  int64_t ch;
  plan_splits(s, &sp, &ch);
  return sp > 1 ? (size_t)sp * (size_t)s.P * (size_t)s.Q * sizeof(float) : 0;
}

cudaError_t splitk_reduce(const float* part, int splits, int64_t P, int64_t Q, float scale,
                          float* Y, int64_t ldy, cudaStream_t st) {
  const int64_t total = P * Q;
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = 8LL * num_sms();
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_splitk_reduce<<<(unsigned)blocks, 256, 0, st>>>(part, splits, P, Q, scale, Y, ldy);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t splitk_reduce_batched(const ReduceDesc* d_desc, int nprob, int64_t max_elems,
                                  cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  int64_t bx = (max_elems + 255) / 256;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  k_splitk_reduce_batched<<<dim3((unsigned)bx, (unsigned)nprob), 256, 0, st>>>(d_desc);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t simt_sketch(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                        float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st) {
  SimtParams p;
  int splits;
  int64_t chunk;
  plan_splits(s, &splits, &chunk);
  p.A = A;
  p.lda = lda;
  p.P = s.P;
  p.Q = s.Q;
  p.L = s.L;
  p.chunk = chunk;
  p.rk = round_keys(make_key(h->seed));
  p.dist = h->dist;
  p.scale = h->scale;
  p.splits = splits;
  p.vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % 4 == 0) ? 1 : 0;
  if (splits > 1) {
    if (ws == nullptr || ws_bytes < simt_workspace_bytes(s)) return cudaErrorInvalidValue;
    p.out = static_cast<float*>(ws);
    p.ldo = s.Q;
  } else {
    p.out = Y;
    p.ldo = ldy;
  }
  // grid x: tiles of the long side (n or m); grid y: tiles of k, at most
  // 65535 (k <= 8,388,480 with the wide left tile, 16,776,960 with the
  // 256-row ones; a larger k fails the launch)
  const bool wide = simt_wide(s);
  const int bp = wide ? SimtTile<true, true>::BP : SimtTile<false, false>::BP;
  const int bq = wide ? SimtTile<true, true>::BQ : SimtTile<false, false>::BQ;
  const unsigned tq = (unsigned)((s.Q + bq - 1) / bq), tp = (unsigned)((s.P + bp - 1) / bp);
  dim3 grid(s.left ? tq : tp, s.left ? tp : tq, (unsigned)splits);
  cudaError_t e = set_simt_smem();
  if (e != cudaSuccess) return e;
  prof_mark(h->prof_start, st);
  if (s.left && wide)
    k_sketch_fp32_simt<true, true><<<grid, TPB, SimtTile<true, true>::SMEM, st>>>(p);
  else if (s.left)
    k_sketch_fp32_simt<true, false><<<grid, TPB, SimtTile<true, false>::SMEM, st>>>(p);
  else
    k_sketch_fp32_simt<false, false><<<grid, TPB, SimtTile<false, false>::SMEM, st>>>(p);
  prof_mark(h->prof_stop, st);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  return splitk_reduce(static_cast<float*>(ws), splits, s.P, s.Q, h->scale, Y, ldy, st);
}

cudaError_t materialize(const sk_sketch* h, int64_t row0, int64_t col0, int64_t rows,
                        int64_t cols, int fmt, int scaled, void* out, int64_t ld,
                        cudaStream_t st) {
  const int64_t total = rows * cols;
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = 16LL * num_sms();
  if (blocks > cap) blocks = cap;
  k_materialize<<<(unsigned)blocks, 256, 0, st>>>(make_key(h->seed), h->dist, fmt, scaled,
                                                  h->scale, row0, col0, rows, cols, out, ld);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace sk

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP32 left sketch.
//
// Some callers cannot let this library call cudaMalloc: applications whose
// device memory is owned by another allocator (a framework's caching
// allocator or a serving engine that reserves HBM up front and accounts for
// every byte), and latency-critical paths that cannot afford the implicit
// device-wide synchronisation of cudaMalloc/cudaFree.  For them the split-K
// partials of the FP32 left sketch live in a fixed array compiled into the
// library instead of in an allocated workspace.
// ---------------------------------------------------------------------------
namespace sk {
namespace {

// 16 MiB of FP32 split-K partials.  Every GPU that loads this library holds
// this array until the process exits; all calls on a device share it.
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
static __device__ __align__(256) float g_static_scratch[kStaticScratchBytes / sizeof(float)];

// Device address of g_static_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, with the device current, on every call: a cached
// address would outlive a cudaDeviceReset, after which the library's device
// code (and this array) is loaded again, possibly elsewhere.
cudaError_t static_scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace
}  // namespace sk

extern "C" sk_status sk_apply_left_noalloc(sk_handle h, const float* A, int64_t m, int64_t n,
                                           int64_t lda, float* Y, int64_t ldy, void* stream) {
  if (!h || !A || !Y || m <= 0 || n <= 0 || lda < n || ldy < n || m >= 4294967296LL)
    return SK_EINVAL;
  if (h->prec != SK_FP32) return SK_EUNSUPPORTED;
  sk::GemmShape s;
  s.left = true;
  s.P = h->k;
  s.Q = n;
  s.L = m;
  if (sk::simt_workspace_bytes(s) > sk::kStaticScratchBytes) return SK_EUNSUPPORTED;
  void* scratch = nullptr;
  cudaError_t e = sk::static_scratch_address(&scratch);
  if (e == cudaSuccess)
    e = sk::simt_sketch(h, s, A, lda, Y, ldy, scratch, sk::kStaticScratchBytes,
                        static_cast<cudaStream_t>(stream));
  return sk::status_from_cuda(e);
}

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

constexpr int BP = 128;  // output rows per CTA
constexpr int BQ = 128;  // output cols per CTA
constexpr int BL = 32;   // contracted length per stage
constexpr int TPB = 256; // 16 x 16 threads, 8 x 8 outputs each
constexpr int PAD = 4;

struct SimtParams {
  const float* A;
  int64_t lda;
  float* out;       // Y (splits == 1) or partials [splits][P][Q]
  int64_t ldo;
  int64_t P, Q, L;
  int64_t chunk;    // contracted length per split (multiple of BL)
  PhiloxKey key;
  int dist;
  float scale;      // applied only when splits == 1
  int splits;
};

// Generated operand tile: G[l][t] = g(t0 + t, l0 + l) for t < BT (generated
// row index = sketch row), l < BL.  Zero outside the matrix.
template <int BT>
__device__ __forceinline__ void gen_tile(float (*G)[BT + PAD], const SimtParams& p, int64_t t0,
                                         int64_t tmax, int64_t l0) {
  // BT rows x (BL/4) groups of 4 columns
  for (int idx = threadIdx.x; idx < BT * (BL / 4); idx += TPB) {
    const int t = idx % BT;
    const int j = idx / BT;
    const int64_t r = t0 + t;
    const int64_t c = l0 + 4 * j;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < tmax && c < p.L) {
      v = gen4(p.dist, p.key, (uint32_t)r, (uint32_t)c, 0u);
      if (c + 1 >= p.L) v.y = 0.f;
      if (c + 2 >= p.L) v.z = 0.f;
      if (c + 3 >= p.L) v.w = 0.f;
    }
    G[4 * j + 0][t] = v.x;
    G[4 * j + 1][t] = v.y;
    G[4 * j + 2][t] = v.z;
    G[4 * j + 3][t] = v.w;
  }
}

template <bool LEFT>
__global__ void __launch_bounds__(TPB) k_sketch_fp32_simt(SimtParams p) {
  __shared__ __align__(16) float Xs[BL][BP + PAD];
  __shared__ __align__(16) float Ws[BL][BQ + PAD];
  // the tiles along the long side (n of the left sketch, m of the right) run
  // along grid x, whose extent is not limited to 65535
  const int64_t q0 = (int64_t)(LEFT ? blockIdx.x : blockIdx.y) * BQ;
  const int64_t p0 = (int64_t)(LEFT ? blockIdx.y : blockIdx.x) * BP;
  const int64_t lbeg = (int64_t)blockIdx.z * p.chunk;
  const int64_t lend = min(p.L, lbeg + p.chunk);
  const int tq = threadIdx.x % 16;
  const int tp = threadIdx.x / 16;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  for (int64_t l0 = lbeg; l0 < lend; l0 += BL) {
    if (LEFT) {
      gen_tile<BP>(Xs, p, p0, p.P, l0);
      // W(l, q) = A[l][q]: rows of A, coalesced along q
      for (int idx = threadIdx.x; idx < BL * BQ; idx += TPB) {
        const int l = idx / BQ, q = idx % BQ;
        const int64_t gl = l0 + l, gq = q0 + q;
        Ws[l][q] = (gl < lend && gq < p.Q) ? __ldg(p.A + gl * p.lda + gq) : 0.f;
      }
    } else {
      gen_tile<BQ>(Ws, p, q0, p.Q, l0);
      // X(p, l) = A[p][l]: coalesced along l, stored transposed
      for (int idx = threadIdx.x; idx < BL * BP; idx += TPB) {
        const int l = idx % BL, r = idx / BL;
        const int64_t gl = l0 + l, gp = p0 + r;
        Xs[l][r] = (gl < lend && gp < p.P) ? __ldg(p.A + gp * p.lda + gl) : 0.f;
      }
    }
    if (LEFT) {
      // the generated tile may extend past this split's range: zero it
      if (l0 + BL > lend) {
        for (int idx = threadIdx.x; idx < BL * BP; idx += TPB) {
          const int l = idx / BP, r = idx % BP;
          if (l0 + l >= lend) Xs[l][r] = 0.f;
        }
      }
    } else if (l0 + BL > lend) {
      for (int idx = threadIdx.x; idx < BL * BQ; idx += TPB) {
        const int l = idx / BQ, q = idx % BQ;
        if (l0 + l >= lend) Ws[l][q] = 0.f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < BL; ++l) {
      float xr[8], wr[8];
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[l][tp * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[l][64 + tp * 4]);
      const float4 w0 = *reinterpret_cast<const float4*>(&Ws[l][tq * 4]);
      const float4 w1 = *reinterpret_cast<const float4*>(&Ws[l][64 + tq * 4]);
      xr[0] = x0.x; xr[1] = x0.y; xr[2] = x0.z; xr[3] = x0.w;
      xr[4] = x1.x; xr[5] = x1.y; xr[6] = x1.z; xr[7] = x1.w;
      wr[0] = w0.x; wr[1] = w0.y; wr[2] = w0.z; wr[3] = w0.w;
      wr[4] = w1.x; wr[5] = w1.y; wr[6] = w1.z; wr[7] = w1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xr[i], wr[j], acc[i][j]);
    }
    __syncthreads();
  }

  // rows p0 + {tp*4 .. tp*4+3, 64+tp*4 ..}, cols q0 + {tq*4 .., 64+tq*4 ..}
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gp = p0 + (i < 4 ? tp * 4 + i : 64 + tp * 4 + (i - 4));
    if (gp >= p.P) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t gq = q0 + (j < 4 ? tq * 4 + j : 64 + tq * 4 + (j - 4));
      if (gq >= p.Q) continue;
      if (p.splits == 1) {
        p.out[gp * p.ldo + gq] = __fmul_rn(p.scale, acc[i][j]);
      } else {
        p.out[((int64_t)blockIdx.z * p.P + gp) * p.Q + gq] = acc[i][j];
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
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < d.splits; ++z) s = __fadd_rn(s, d.part[(int64_t)z * total + i]);
    const int64_t r = i / d.Q, c = i % d.Q;
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
  const int64_t tiles = ((s.P + BP - 1) / BP) * ((s.Q + BQ - 1) / BQ);
  const int64_t target = 3LL * num_sms();
  int64_t sp = (target + tiles - 1) / tiles;
  const int64_t max_sp = s.L / (4 * BL) > 0 ? s.L / (4 * BL) : 1;
  if (sp > max_sp) sp = max_sp;
  if (sp > 64) sp = 64;
  if (sp < 1) sp = 1;
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
  p.key = make_key(h->seed);
  p.dist = h->dist;
  p.scale = h->scale;
  p.splits = splits;
  if (splits > 1) {
    if (ws == nullptr || ws_bytes < simt_workspace_bytes(s)) return cudaErrorInvalidValue;
    p.out = static_cast<float*>(ws);
    p.ldo = s.Q;
  } else {
    p.out = Y;
    p.ldo = ldy;
  }
  // grid x: tiles of the long side (n or m); grid y: tiles of k, at most
  // 65535 (k <= 8,388,480 in this form; a larger k fails the launch)
  const unsigned tq = (unsigned)((s.Q + BQ - 1) / BQ), tp = (unsigned)((s.P + BP - 1) / BP);
  dim3 grid(s.left ? tq : tp, s.left ? tp : tq, (unsigned)splits);
  prof_mark(h->prof_start, st);
  if (s.left)
    k_sketch_fp32_simt<true><<<grid, TPB, 0, st>>>(p);
  else
    k_sketch_fp32_simt<false><<<grid, TPB, 0, st>>>(p);
  prof_mark(h->prof_stop, st);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
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

// sk_tc.cu -- BF16 split-A tensor-core form of the fused generate-and-sketch
// on Blackwell (tcgen05 + TMEM + TMA), left sketch Y[k x n] = S[k x m] A[m x n].
//
// This is the local multiply of the paper's Alg. 1 (GenRandom, then
// B = A Omega on the local block) with the random operand regenerated inside
// the kernel instead of read (Sec. 6.2's "generate rather than communicate",
// with shared memory in the role of the processor's local memory).
//
// One CTA per SM owns a 128 x NT tile of Y (NT <= 512 TMEM columns) and one
// contiguous range of the contracted dimension m (deterministic split-K):
//   warp 0       TMA producer: FP32 A tiles [16 rows of m x NT cols] into a
//                3-stage staging ring (zero fill beyond the matrix);
//   warp 1       TMEM allocator and MMA issuer: per stage 2 passes (hi, lo) x
//                NT/256 tcgen05.mma kind::f16 (M=128, K=16) into one FP32
//                accumulator in TMEM;
//   warps 2-5    epilogue: every CHAIN stages the accumulator is read out of
//                TMEM (tcgen05.ld) and added into the CTA's FP32 partial in
//                global memory (store for the first chain, red.add after);
//   warps 6-21   workers: each stage, every worker generates its share of the
//                BF16 S tile [128 x 16] (Philox4x32-10 + Box-Muller or sign
//                bits) and converts its share of the FP32 staging tile into
//                BF16 hi = bf16(a), lo = bf16(a - hi), both in the K-major
//                no-swizzle operand layout.
// The tensor core accumulates in FP32 without round-to-nearest on every
// add, so its error grows with the chain length; restarting the TMEM chain
// every CHAIN stages and summing chains with IEEE adds keeps Y within 1e-5
// of the exact product at any m.  S never exists outside shared memory.
// Every wait is bounded: on timeout the kernel records SK_ETIMEOUT in the
// handle's status word, drains its own copies and MMAs (again bounded) and
// frees TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sk_internal.h"
#include "sk_rng.cuh"
#include "sk_tc.cuh"

namespace sk {
namespace {

using namespace tc;

constexpr int BM = 128;       // generated rows per CTA (MMA M)
constexpr int BK = 16;        // contracted length per stage (MMA K)
constexpr int NT_MAX = 512;   // output columns per CTA (TMEM columns)
constexpr int NSF = 3;        // FP32 staging stages
constexpr int NSO = 3;        // operand stages
constexpr int CHAIN = 64;     // stages per TMEM accumulation chain
constexpr int NUM_EPI_WARPS = 4;
constexpr int NUM_WORK_WARPS = 16;
constexpr int WARP_TMA = 0;
constexpr int WARP_MMA = 1;
constexpr int WARP_EPI0 = 2;
constexpr int WARP_WORK0 = WARP_EPI0 + NUM_EPI_WARPS;
constexpr int NWORK = 32 * NUM_WORK_WARPS;                   // 512 worker threads
constexpr int NTHREADS = 32 * (WARP_WORK0 + NUM_WORK_WARPS);  // 704

constexpr uint32_t STAGE_F_BYTES = BK * NT_MAX * 4;  // 32 KB
constexpr uint32_t OPB_BYTES = NT_MAX * BK * 2;      // 16 KB (hi or lo)
constexpr uint32_t OPS_BYTES = BM * BK * 2;          // 4 KB
constexpr uint32_t OFF_F = 0;
constexpr uint32_t OFF_BHI = OFF_F + NSF * STAGE_F_BYTES;
constexpr uint32_t OFF_BLO = OFF_BHI + NSO * OPB_BYTES;
constexpr uint32_t OFF_S = OFF_BLO + NSO * OPB_BYTES;
constexpr uint32_t OFF_BAR = OFF_S + NSO * OPS_BYTES;
constexpr uint32_t NUM_BARS = 2 * NSF + 2 * NSO + 3;
constexpr uint32_t OFF_MISC = OFF_BAR + NUM_BARS * 8;
constexpr uint32_t SMEM_BYTES = OFF_MISC + 16 + 1024;  // + slack for 1 KB alignment
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");

// K-major no-swizzle operand layout (16-element K slab): core matrix
// (8 rows x 16 B) at (row/8)*256 + khalf*128, row r%8 at +16*(r%8).
__device__ __forceinline__ uint32_t kmaj_off(uint32_t row, uint32_t khalf) {
  return (row & 7u) * 16u + (row >> 3) * 256u + khalf * 128u;
}
constexpr uint32_t LBO = 128;  // K-adjacent core matrices
constexpr uint32_t SBO = 256;  // 8-row groups

struct TcParams {
  float* part;      // partials [splits][P][Q] (every chain is summed here)
  int64_t P, Q, L;  // P = k, Q = n, L = m
  int64_t chunk;    // contracted length per split (multiple of BK)
  int nt;           // output columns per CTA: multiple of 16 up to 256, or 512
  int boxn;         // TMA box width in columns
  int nbox;         // TMA boxes per stage
  int tmem_cols;    // power of two >= max(32, nt)
  PhiloxKey key;
  int* status;
  uint64_t timeout_ns;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Bounded wait that ignores the abort flag (used only to drain in-flight
// asynchronous work on the way out).
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > limit_ns) return;
  }
}

template <int DIST>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_sketch_bf16x2_left(const __grid_constant__ CUtensorMap tmapA, const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + OFF_BAR;
  auto full_f = [&](int i) { return bar0 + 8u * i; };
  auto empty_f = [&](int i) { return bar0 + 8u * (NSF + i); };
  auto full_o = [&](int i) { return bar0 + 8u * (2 * NSF + i); };
  auto empty_o = [&](int i) { return bar0 + 8u * (2 * NSF + NSO + i); };
  const uint32_t acc_full = bar0 + 8u * (2 * NSF + 2 * NSO);
  const uint32_t acc_empty = acc_full + 8u;
  const uint32_t drain_bar = acc_full + 16u;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + OFF_MISC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + OFF_MISC + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t q0 = static_cast<int64_t>(blockIdx.x) * p.nt;
  const int64_t p0 = static_cast<int64_t>(blockIdx.y) * BM;
  const int64_t lbeg = static_cast<int64_t>(blockIdx.z) * p.chunk;
  const int64_t lend = min(p.L, lbeg + p.chunk);
  const int nsteps = static_cast<int>((lend - lbeg + BK - 1) / BK);
  const int nchains = (nsteps + CHAIN - 1) / CHAIN;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSF; ++i) {
      mbar_init(full_f(i), 1);
      mbar_init(empty_f(i), NUM_WORK_WARPS);
    }
    for (int i = 0; i < NSO; ++i) {
      mbar_init(full_o(i), NUM_WORK_WARPS);
      mbar_init(empty_o(i), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NUM_EPI_WARPS);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == WARP_MMA) {
    tmem_alloc(smem_u32(tmem_slot), static_cast<uint32_t>(p.tmem_cols));
    tmem_relinquish();
  }
  if (warp == WARP_TMA && lane == 0) tma_prefetch_desc(&tmapA);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const Abort ab{abort_flag, p.status, p.timeout_ns};

  if (warp == WARP_TMA) {
    if (lane == 0) {
      const uint32_t tx = static_cast<uint32_t>(p.nbox * p.boxn * BK * 4);
      int issued = 0;
      for (int s = 0; s < nsteps; ++s) {
        const int sf = s % NSF;
        if (s >= NSF && !mbar_wait(empty_f(sf), ((s / NSF) & 1) ^ 1, ab)) break;
        mbar_arrive_expect_tx(full_f(sf), tx);
        const int32_t y = static_cast<int32_t>(lbeg + static_cast<int64_t>(s) * BK);
        const uint32_t dst = sbase + OFF_F + sf * STAGE_F_BYTES;
        for (int b = 0; b < p.nbox; ++b)
          tma_load_2d(dst + static_cast<uint32_t>(b * p.boxn * BK * 4), &tmapA,
                      static_cast<int32_t>(q0 + b * p.boxn), y, full_f(sf));
        issued = s + 1;
      }
      if (*abort_flag) {  // let the copies already issued land before leaving
        for (int s = max(0, issued - NSF); s < issued; ++s)
          drain_wait(full_f(s % NSF), (s / NSF) & 1, 100000000ull);
      }
    }
  } else if (warp == WARP_MMA) {
    if (lane == 0) {
      const int nmma = p.nt > 256 ? 2 : 1;
      const uint32_t idesc = idesc_bf16_f32(128, static_cast<uint32_t>(p.nt > 256 ? 256 : p.nt));
      for (int s = 0; s < nsteps; ++s) {
        const int so = s % NSO;
        const int in_chain = s % CHAIN;
        // a new chain may start only after the epilogue has read the last one
        if (s > 0 && in_chain == 0 && !mbar_wait(acc_empty, ((s / CHAIN) - 1) & 1, ab)) break;
        if (!mbar_wait(full_o(so), (s / NSO) & 1, ab)) break;
        tc_fence_after();
        const uint64_t adesc = smem_desc(sbase + OFF_S + so * OPS_BYTES, LBO, SBO);
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const uint32_t bb = sbase + (pass ? OFF_BLO : OFF_BHI) + so * OPB_BYTES;
          for (int h = 0; h < nmma; ++h) {
            const uint64_t bdesc = smem_desc(bb + static_cast<uint32_t>(h) * (256u / 8u) * SBO,
                                             LBO, SBO);
            mma_bf16(tmem + static_cast<uint32_t>(h) * 256u, adesc, bdesc, idesc,
                     (in_chain > 0 || pass > 0) ? 1u : 0u);
          }
        }
        mma_commit(empty_o(so));
        if (in_chain == CHAIN - 1 || s == nsteps - 1) mma_commit(acc_full);
      }
      mma_commit(drain_bar);  // completes once every MMA issued above has finished
    }
  } else if (warp < WARP_WORK0) {
    // ---- epilogue: add each finished chain into the CTA's FP32 partial ----
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int64_t gp = p0 + row;
    float* dst_row = p.part + (static_cast<int64_t>(blockIdx.z) * p.P + gp) * p.Q + q0;
    const bool vec_ok = (p.Q % 4) == 0;
    for (int c = 0; c < nchains; ++c) {
      const bool ok = mbar_wait(acc_full, c & 1, ab);
      if (!__all_sync(0xffffffffu, ok)) break;  // tcgen05.ld below is warp-collective
      tc_fence_after();
      for (int ci = 0; ci * 32 < p.nt; ++ci) {
        uint32_t v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                      static_cast<uint32_t>(ci * 32),
                  v);
        tmem_ld_wait();
        if (gp < p.P) {
          const int64_t col = q0 + ci * 32;
          float* d = dst_row + ci * 32;
          if (vec_ok && col + 32 <= p.Q) {
#pragma unroll
            for (int e = 0; e < 32; e += 4) {
              const float a = __uint_as_float(v[e]), b = __uint_as_float(v[e + 1]);
              const float x = __uint_as_float(v[e + 2]), y = __uint_as_float(v[e + 3]);
              if (c == 0)
                *reinterpret_cast<float4*>(d + e) = make_float4(a, b, x, y);
              else
                red_add_v4(d + e, a, b, x, y);
            }
          } else {
            for (int e = 0; e < 32; ++e) {
              if (col + e < p.Q) {
                if (c == 0)
                  d[e] = __uint_as_float(v[e]);
                else
                  red_add(d + e, __uint_as_float(v[e]));
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
  } else {
    // ---- workers: generate the S tile and convert the A tile ----
    const int wt = threadIdx.x - 32 * WARP_WORK0;  // 0..511
    const int nt = p.nt;
    const int boxn = p.boxn;
    // generation task of this thread (fixed across stages)
    //   Rademacher: row wt%128, k-half wt/128 (threads < 256), 8 entries
    //   Gaussian / uniform: 8 rows x 4 quads per warp, 4 entries each
    uint32_t g_row, g_off, g_col;
    bool g_active;
    if (DIST == kRademacher) {
      g_row = static_cast<uint32_t>(wt & (BM - 1));
      g_col = 8u * static_cast<uint32_t>(wt >> 7);
      g_off = kmaj_off(g_row, static_cast<uint32_t>(wt >> 7));
      g_active = wt < 2 * BM;
    } else {
      const uint32_t l = static_cast<uint32_t>(wt & 31);
      g_row = static_cast<uint32_t>(wt >> 5) * 8u + (l >> 2);
      const uint32_t qd = l & 3u;
      g_col = 4u * qd;
      g_off = kmaj_off(g_row, qd >> 1) + (qd & 1u) * 8u;
      g_active = true;
    }
    const int64_t grow = p0 + g_row;
    const bool row_ok = grow < p.P;
    uint32_t cached_blk = 0xffffffffu;
    uint4 words = make_uint4(0u, 0u, 0u, 0u);

    for (int s = 0; s < nsteps; ++s) {
      const int sf = s % NSF;
      const int so = s % NSO;
      bool ok = s < NSO || mbar_wait(empty_o(so), ((s / NSO) & 1) ^ 1, ab);
      if (!__all_sync(0xffffffffu, ok)) break;  // leave together (abort path)
      uint8_t* sdst = smem + OFF_S + so * OPS_BYTES;
      const int64_t cbase = lbeg + static_cast<int64_t>(s) * BK;
      if (g_active) {
        const int64_t c0 = cbase + g_col;
        if (DIST == kRademacher) {
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (row_ok && c0 < lend) {
            const uint32_t c = static_cast<uint32_t>(c0);
            const uint32_t blk = c >> 7;
            if (blk != cached_blk) {
              words = rademacher_bits(p.key, static_cast<uint32_t>(grow), blk, 0u);
              cached_blk = blk;
            }
            const uint32_t wsel = (c >> 5) & 3u;
            const uint32_t w = wsel == 0 ? words.x : wsel == 1 ? words.y
                             : wsel == 2 ? words.z : words.w;
            const uint32_t bits = w >> (c & 31u);
            // +1.0 = 0x3F80, -1.0 = 0xBF80: the sign bit carries the random bit
            v.x = 0x3F803F80u | ((bits & 1u) << 15) | ((bits & 2u) << 30);
            v.y = 0x3F803F80u | ((bits & 4u) << 13) | ((bits & 8u) << 28);
            v.z = 0x3F803F80u | ((bits & 16u) << 11) | ((bits & 32u) << 26);
            v.w = 0x3F803F80u | ((bits & 64u) << 9) | ((bits & 128u) << 24);
          }
          *reinterpret_cast<uint4*>(sdst + g_off) = v;
        } else {
          uint2 v = make_uint2(0u, 0u);
          if (row_ok && c0 < lend) {
            const uint32_t c = static_cast<uint32_t>(c0);
            const float4 a = DIST == kUniform
                                 ? uniform4(p.key, static_cast<uint32_t>(grow), c >> 2, 0u)
                                 : gaussian4(p.key, static_cast<uint32_t>(grow), c >> 2, 0u);
            v = make_uint2(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w));
          }
          *reinterpret_cast<uint2*>(sdst + g_off) = v;
        }
      }
      // conversion needs this stage's A tile
      ok = mbar_wait(full_f(sf), (s / NSF) & 1, ab);
      if (!__all_sync(0xffffffffu, ok)) break;
      const float* stg = reinterpret_cast<const float*>(smem + OFF_F + sf * STAGE_F_BYTES);
      uint8_t* bhi = smem + OFF_BHI + so * OPB_BYTES;
      uint8_t* blo = smem + OFF_BLO + so * OPB_BYTES;
      for (int i = wt; i < 2 * nt; i += NWORK) {
        const int h = i >= nt ? 1 : 0;
        const int j = i - h * nt;
        const int box = j / boxn;
        const float* src = stg + box * boxn * BK + (8 * h) * boxn + (j - box * boxn);
        float a[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] = src[e * boxn];
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          hw[e] = pack_bf16x2(a[2 * e], a[2 * e + 1]);
          const float h0 = __uint_as_float(hw[e] << 16);
          const float h1 = __uint_as_float(hw[e] & 0xffff0000u);
          lw[e] = pack_bf16x2(__fsub_rn(a[2 * e], h0), __fsub_rn(a[2 * e + 1], h1));
        }
        const uint32_t o = kmaj_off(static_cast<uint32_t>(j), static_cast<uint32_t>(h));
        *reinterpret_cast<uint4*>(bhi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(blo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(full_o(so));
        mbar_arrive(empty_f(sf));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == WARP_MMA) {
    tc_fence_after();
    drain_wait(drain_bar, 0, 200000000ull);  // every MMA finished before TMEM is freed
    __syncwarp();
    tmem_dealloc(tmem, static_cast<uint32_t>(p.tmem_cols));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int num_sms_tc() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

struct Plan {
  int nt, boxn, nbox, tmem_cols;
  int64_t tiles_q, tiles_p;
  int splits;
  int64_t chunk;
};

// Tile width, TMA boxes and the split-K count: whole waves of one CTA per SM,
// and no split longer than 2^16 rows of m (4096 MMA K-steps) so that FP32
// accumulation chains stay short.
Plan plan_left(const GemmShape& s) {
  Plan pl;
  if (s.Q > 256) {
    pl.nt = 512;
    pl.boxn = 256;
    pl.nbox = 2;
  } else {
    pl.nt = static_cast<int>((s.Q + 15) / 16 * 16);
    pl.boxn = pl.nt;
    pl.nbox = 1;
  }
  pl.tmem_cols = 32;
  while (pl.tmem_cols < pl.nt) pl.tmem_cols *= 2;
  pl.tiles_q = (s.Q + pl.nt - 1) / pl.nt;
  pl.tiles_p = (s.P + BM - 1) / BM;
  const int64_t tiles = pl.tiles_q * pl.tiles_p;
  const int64_t sms = num_sms_tc();
  const int64_t steps_total = (s.L + BK - 1) / BK;
  const int64_t smin = 1;
  int64_t smax = steps_total / 8;  // at least 8 stages per split
  if (smax > 128) smax = 128;
  if (smax < smin) smax = smin;
  int64_t best = smin;
  double best_eff = -1.0;
  for (int64_t sp = smin; sp <= smax; ++sp) {
    const int64_t ctas = tiles * sp;
    const int64_t waves = (ctas + sms - 1) / sms;
    const double eff = static_cast<double>(ctas) / static_cast<double>(waves * sms);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = sp;
    }
    if (ctas >= 4 * sms) break;
  }
  int64_t chunk = (s.L + best - 1) / best;
  chunk = (chunk + BK - 1) / BK * BK;
  pl.chunk = chunk;
  pl.splits = static_cast<int>((s.L + chunk - 1) / chunk);
  return pl;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

template <int DIST>
cudaError_t launch_left(const CUtensorMap& map, const TcParams& p, dim3 grid, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_sketch_bf16x2_left<DIST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_sketch_bf16x2_left<DIST><<<grid, NTHREADS, SMEM_BYTES, st>>>(map, p);
  return cudaGetLastError();
}

}  // namespace

size_t tc_workspace_bytes(const GemmShape& s) {
  if (!s.left) return 0;
  const Plan pl = plan_left(s);
  return static_cast<size_t>(pl.splits) * static_cast<size_t>(s.P) * static_cast<size_t>(s.Q) *
         sizeof(float);
}

sk_status tc_check(const GemmShape& s, const float* A, int64_t lda, const float* Y, int64_t ldy) {
  if (!s.left) return SK_EUNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(Y) & 15u))
    return SK_EINVAL;
  if (lda % 4 != 0 || ldy % 4 != 0) return SK_EINVAL;
  if (s.L > (1LL << 31) - 64 || s.Q > (1LL << 31) - 1024) return SK_EUNSUPPORTED;
  return SK_OK;
}

cudaError_t tc_sketch(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                      float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!s.left) return cudaErrorNotSupported;
  const Plan pl = plan_left(s);
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(s.Q), static_cast<cuuint64_t>(s.L)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(lda) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(pl.boxn), static_cast<cuuint32_t>(BK)};
  const cuuint32_t estride[2] = {1, 1};
  CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim,
                    gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;

  TcParams p;
  p.P = s.P;
  p.Q = s.Q;
  p.L = s.L;
  p.chunk = pl.chunk;
  p.nt = pl.nt;
  p.boxn = pl.boxn;
  p.nbox = pl.nbox;
  p.tmem_cols = pl.tmem_cols;
  p.key = make_key(h->seed);
  p.status = h->d_status;
  p.timeout_ns = 2000000000ull;  // 2 s per wait: far beyond any healthy stage
  const size_t need = static_cast<size_t>(pl.splits) * s.P * s.Q * sizeof(float);
  if (ws == nullptr || ws_bytes < need) return cudaErrorInvalidValue;
  p.part = static_cast<float*>(ws);
  dim3 grid(static_cast<unsigned>(pl.tiles_q), static_cast<unsigned>(pl.tiles_p),
            static_cast<unsigned>(pl.splits));
  prof_mark(h->prof_start, st);
  cudaError_t e;
  if (h->dist == kRademacher)
    e = launch_left<kRademacher>(map, p, grid, st);
  else if (h->dist == kUniform)
    e = launch_left<kUniform>(map, p, grid, st);
  else
    e = launch_left<kGaussian>(map, p, grid, st);
  prof_mark(h->prof_stop, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  // fixed-order sum of the split partials, times 1/sqrt(k), into Y
  return splitk_reduce(static_cast<float*>(ws), pl.splits, s.P, s.Q, h->scale, Y, ldy, st);
}

}  // namespace sk

// sk_tc.cu -- BF16 split-A tensor-core form of the fused generate-and-sketch
// on Blackwell (tcgen05 + TMEM + TMA, CTA pairs), left sketch
// Y[k x n] = S[k x m] A[m x n].
//
// This is the local multiply of the paper's Alg. 1 (GenRandom, then
// B = A Omega on the local block) with the random operand regenerated inside
// the kernel instead of read (Sec. 6.2's "generate rather than communicate",
// with shared memory in the role of the processor's local memory).
//
// Shared-memory bandwidth, not the tensor core, bounds this product: every
// stage the MMA re-reads its operands from shared memory while the FP32 A
// tile is written by TMA, read back and written again as BF16 hi / lo.  A CTA
// pair (cta_group::2) halves that traffic per SM: one MMA of M = 256 spans
// both SMs, each CTA supplying 128 rows of S and half of the B (= A tile)
// rows, so each CTA loads and converts only half of every A tile.
//
// A pair owns a 256 x NT tile of Y (NT <= 512 TMEM columns in each CTA) and
// one contiguous range of the contracted dimension m (deterministic split-K):
//   warp 0       TMA producer: this CTA's FP32 columns of each A tile
//                [16 rows of m] into a staging ring;
//   warp 1       TMEM allocation (collective over the pair); in the even CTA
//                the MMA issuer: per stage 2 passes (hi, lo) x NT/256
//                tcgen05.mma kind::f16 (M=256, K=16) into the FP32
//                accumulator, completion signalled to both CTAs;
//   warps 2-9    epilogue: every CHAIN stages the accumulator is read out of
//                this CTA's TMEM and added into its FP32 partial in global
//                memory (store for the first chain, red.add after);
//   warps 10-25  workers, in 4 groups that take turns on successive stages
//                (so that four stages are in flight): generate this CTA's
//                BF16 S tile [128 x 16] (Philox4x32-10 + Box-Muller, or sign
//                bits) and convert its A columns into hi = bf16(a),
//                lo = bf16(a - hi) in the K-major no-swizzle operand layout.
// With k <= 128 a single CTA (cta_group::1, M = 128) does the same alone.
// The tensor core accumulates in FP32 without round-to-nearest on every
// add, so its error grows with the chain length; restarting the TMEM chain
// every CHAIN stages and summing chains with IEEE adds keeps Y within 1e-5
// of the exact product at any m.  S never exists outside shared memory.
// Every wait is bounded: on timeout the kernel records SK_ETIMEOUT and the
// waiting site in the handle's status words, drains its own copies and MMAs
// (again bounded) and frees TMEM; both CTAs reach the closing cluster barrier.
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

constexpr int BM = 128;       // generated rows per CTA
constexpr int BK = 16;        // contracted length per stage (MMA K)
constexpr int NT_MAX = 512;   // output columns per tile (TMEM columns)
constexpr int CHAIN = 128;    // stages per TMEM accumulation chain
constexpr int NUM_EPI_WARPS = 8;
constexpr int NUM_WORK_WARPS = 16;

constexpr int WARP_TMA = 0;
constexpr int WARP_MMA = 1;
constexpr int WARP_EPI0 = 2;
constexpr int WARP_WORK0 = WARP_EPI0 + NUM_EPI_WARPS;
constexpr int NWORK = 32 * NUM_WORK_WARPS;
constexpr int NTHREADS = 32 * (WARP_WORK0 + NUM_WORK_WARPS);  // 832

// Per-CTA buffers.  A CTA of a pair holds NT/2 columns of each A tile.
template <bool PAIR>
struct Cfg {
  static constexpr int COLS = PAIR ? NT_MAX / 2 : NT_MAX;   // A columns per CTA
  // Worker groups take turns on successive stages.  A group that starts
  // stage s has finished stage s - NGROUPS, so waits never run more than one
  // barrier phase ahead (the parity test would alias) as long as
  // NGROUPS <= NSF and NGROUPS <= NSO.
  static constexpr int NGROUPS = PAIR ? 4 : 2;
  static constexpr int GROUP_WARPS = NUM_WORK_WARPS / NGROUPS;
  static constexpr int GROUP_THREADS = 32 * GROUP_WARPS;
#ifndef SK_TC_NSF
  static constexpr int NSF = PAIR ? 6 : 3;                  // FP32 staging stages
  static constexpr int NSO = PAIR ? 6 : 3;                  // operand stages
#else
  static constexpr int NSF = PAIR ? SK_TC_NSF : 3;
  static constexpr int NSO = PAIR ? SK_TC_NSO : 3;
#endif
  static constexpr uint32_t STAGE_F = BK * COLS * 4;        // FP32 staging
  static constexpr uint32_t OPB = COLS * BK * 2;            // hi or lo operand
  static constexpr uint32_t OPS = BM * BK * 2;              // S tile
  static constexpr uint32_t OFF_F = 0;
  static constexpr uint32_t OFF_BHI = OFF_F + NSF * STAGE_F;
  static constexpr uint32_t OFF_BLO = OFF_BHI + NSO * OPB;
  static constexpr uint32_t OFF_S = OFF_BLO + NSO * OPB;
  static constexpr uint32_t OFF_BAR = OFF_S + NSO * OPS;
  static constexpr uint32_t NUM_BARS = 2 * NSF + 2 * NSO + 3;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NUM_BARS * 8;
  static constexpr uint32_t SMEM = OFF_MISC + 16 + 1024;  // + slack for 1 KB alignment
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
  static_assert(NGROUPS <= NSF && NGROUPS <= NSO, "worker groups vs ring depth");
};

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
  int nt;           // output columns per tile: multiple of 16 (32 for pairs) up to 256, or 512
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

template <int DIST, bool PAIR>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_sketch_bf16x2_left(const __grid_constant__ CUtensorMap tmapA, const TcParams p) {
  using C = Cfg<PAIR>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + C::OFF_BAR;
  auto full_f = [&](int i) { return bar0 + 8u * i; };
  auto empty_f = [&](int i) { return bar0 + 8u * (C::NSF + i); };
  auto full_o = [&](int i) { return bar0 + 8u * (2 * C::NSF + i); };
  auto empty_o = [&](int i) { return bar0 + 8u * (2 * C::NSF + C::NSO + i); };
  const uint32_t acc_full = bar0 + 8u * (2 * C::NSF + 2 * C::NSO);
  const uint32_t acc_empty = acc_full + 8u;
  const uint32_t drain_bar = acc_full + 16u;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::OFF_MISC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? (cluster_ctarank() & 1u) : 0u;  // 0 = even (MMA issuer)
  const bool leader = rank == 0;
  const int nt = p.nt;
  const int nmma = nt > 256 ? 2 : 1;                 // MMA instructions per pass
  const int nh = nt > 256 ? 256 : nt;                // N of each instruction
  const int bh = PAIR ? nh / 2 : nh;                 // B rows per instruction in this CTA
  const int cols = nmma * bh;                        // A columns this CTA loads/converts
  // grid: x = 128-row tiles of Y (pairs are adjacent in x), y = column tiles
  const int64_t q0 = static_cast<int64_t>(blockIdx.y) * nt;
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int64_t lbeg = static_cast<int64_t>(blockIdx.z) * p.chunk;
  const int64_t lend = min(p.L, lbeg + p.chunk);
  const int nsteps = static_cast<int>((lend - lbeg + BK - 1) / BK);
  const int nchains = (nsteps + CHAIN - 1) / CHAIN;

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NSF; ++i) {
      mbar_init(full_f(i), 1);
      mbar_init(empty_f(i), C::GROUP_WARPS);
    }
    for (int i = 0; i < C::NSO; ++i) {
      mbar_init(full_o(i), C::GROUP_WARPS * (PAIR ? 2 : 1));  // one worker group of each CTA
      mbar_init(empty_o(i), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NUM_EPI_WARPS * (PAIR ? 2 : 1));  // epilogues of both CTAs
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == WARP_MMA) {
    if (PAIR) {
      tmem_alloc_pair(smem_u32(tmem_slot), static_cast<uint32_t>(p.tmem_cols));
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), static_cast<uint32_t>(p.tmem_cols));
      tmem_relinquish();
    }
  }
  if (warp == WARP_TMA && lane == 0) tma_prefetch_desc(&tmapA);
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // the peer's barriers exist before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const Abort ab{abort_flag, p.status, p.timeout_ns};
  // barriers of the even CTA, addressed from either CTA
  const uint32_t lead_full_o = PAIR ? mapa_shared(full_o(0), 0u) : full_o(0);
  const uint32_t lead_acc_empty = PAIR ? mapa_shared(acc_empty, 0u) : acc_empty;

  if (warp == WARP_TMA) {
    if (lane == 0) {
      const uint32_t tx = static_cast<uint32_t>(cols * BK * 4);
      int issued = 0;
      for (int s = 0; s < nsteps; ++s) {
        const int sf = s % C::NSF;
        if (s >= C::NSF && !mbar_wait(empty_f(sf), ((s / C::NSF) & 1) ^ 1, ab, 0x11, s)) break;
        mbar_arrive_expect_tx(full_f(sf), tx);
        const int32_t y = static_cast<int32_t>(lbeg + static_cast<int64_t>(s) * BK);
        for (int b = 0; b * 256 < cols; ++b)
          tma_load_2d(sbase + C::OFF_F + sf * C::STAGE_F + static_cast<uint32_t>(b * 256 * BK * 4),
                      &tmapA, static_cast<int32_t>(q0 + static_cast<int>(rank) * cols + b * 256), y,
                      full_f(sf));
        issued = s + 1;
      }
      if (*abort_flag) {  // let the copies already issued land before leaving
        for (int s = max(0, issued - C::NSF); s < issued; ++s)
          drain_wait(full_f(s % C::NSF), (s / C::NSF) & 1, 100000000ull);
      }
    }
  } else if (warp == WARP_MMA) {
    if (lane == 0 && leader) {
      const uint32_t idesc =
          idesc_bf16_f32(PAIR ? 256u : 128u, static_cast<uint32_t>(nh));
      for (int s = 0; s < nsteps; ++s) {
        const int so = s % C::NSO;
        const int in_chain = s % CHAIN;
        // a new chain may start only after every epilogue has read the last one
        if (s > 0 && in_chain == 0 &&
            !mbar_wait(acc_empty, ((s / CHAIN) - 1) & 1, ab, 0x25, s))
          break;
        if (!mbar_wait(full_o(so), (s / C::NSO) & 1, ab, 0x22, s)) break;
        tc_fence_after();
        const uint64_t adesc = smem_desc(sbase + C::OFF_S + so * C::OPS, LBO, SBO);
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const uint32_t bb = sbase + (pass ? C::OFF_BLO : C::OFF_BHI) + so * C::OPB;
          for (int h = 0; h < nmma; ++h) {
            const uint64_t bdesc =
                smem_desc(bb + static_cast<uint32_t>(h * bh / 8) * SBO, LBO, SBO);
            const uint32_t acc = (in_chain > 0 || pass > 0) ? 1u : 0u;
            if (PAIR)
              mma_bf16_pair(tmem + static_cast<uint32_t>(h) * 256u, adesc, bdesc, idesc, acc);
            else
              mma_bf16(tmem + static_cast<uint32_t>(h) * 256u, adesc, bdesc, idesc, acc);
          }
        }
        const bool chain_end = in_chain == CHAIN - 1 || s == nsteps - 1;
        if (PAIR) {  // operands and accumulator are both CTAs'
          mma_commit_pair_both(empty_o(so));
          if (chain_end) mma_commit_pair_both(acc_full);
        } else {
          mma_commit(empty_o(so));
          if (chain_end) mma_commit(acc_full);
        }
      }
      if (PAIR)
        mma_commit_pair(drain_bar);
      else
        mma_commit(drain_bar);
      // every MMA has finished before this CTA reaches the closing barrier
      drain_wait(drain_bar, 0, 200000000ull);
    }
  } else if (warp < WARP_WORK0) {
    // ---- epilogue: add each finished chain into this CTA's FP32 partial ----
    const int quarter = warp & 3;
    const int colset = (warp - WARP_EPI0) >> 2;  // 0 or 1: even / odd 32-column chunks
    const int row = quarter * 32 + lane;
    const int64_t gp = p0 + row;
    float* dst_row = p.part + (static_cast<int64_t>(blockIdx.z) * p.P + gp) * p.Q + q0;
    const bool vec_ok = (p.Q % 4) == 0;
    for (int c0 = 0; c0 < nchains; ++c0) {
      const bool ok = mbar_wait(acc_full, c0 & 1, ab, 0x34, c0);
      if (!__all_sync(0xffffffffu, ok)) break;  // tcgen05.ld below is warp-collective
      tc_fence_after();
      // TMEM column h*256 + c holds B row c of instruction h: with a pair,
      // rows c < bh are the even CTA's columns h*bh + c of the tile and rows
      // c >= bh the odd CTA's columns cols + h*bh + (c - bh)
      for (int ci = colset; ci * 32 < nmma * 256 && ci * 32 < (nmma - 1) * 256 + nh; ci += 2) {
        uint32_t v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                      static_cast<uint32_t>(ci * 32),
                  v);
        tmem_ld_wait();
        if (gp < p.P) {
#pragma unroll
          for (int e = 0; e < 32; e += 4) {  // bh is a multiple of 8: groups never straddle
            const int tcol = ci * 32 + e;
            const int h = tcol >> 8;
            const int c = tcol & 255;
            if (c >= nh) continue;
            const int tn = PAIR ? (c < bh ? h * bh + c : cols + h * bh + (c - bh)) : tcol;
            const int64_t col = q0 + tn;
            float* d = dst_row + tn;
            const float a0 = __uint_as_float(v[e]), a1 = __uint_as_float(v[e + 1]);
            const float a2 = __uint_as_float(v[e + 2]), a3 = __uint_as_float(v[e + 3]);
            if (vec_ok && col + 4 <= p.Q) {
              if (c0 == 0)
                *reinterpret_cast<float4*>(d) = make_float4(a0, a1, a2, a3);
              else
                red_add_v4(d, a0, a1, a2, a3);
            } else {
              const float vv[4] = {a0, a1, a2, a3};
              for (int u = 0; u < 4; ++u) {
                if (col + u < p.Q) {
                  if (c0 == 0)
                    d[u] = vv[u];
                  else
                    red_add(d + u, vv[u]);
                }
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR)
          mbar_arrive_cluster(lead_acc_empty);
        else
          mbar_arrive(acc_empty);
      }
    }
  } else {
    // ---- workers: generate this CTA's S tile and convert its A columns ----
    // group g handles the stages s = g (mod C::NGROUPS)
    const int grp = (warp - WARP_WORK0) / C::GROUP_WARPS;
    const int wt = threadIdx.x - 32 * WARP_WORK0 - grp * C::GROUP_THREADS;
    // Rademacher: each thread keeps the same (row, half) tasks on every stage
    // and caches their Philox words across the 8 stages a call covers
    constexpr int RAD_IT = (2 * BM + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
    uint32_t cached_blk[RAD_IT];
    uint4 words[RAD_IT];
#pragma unroll
    for (int it = 0; it < RAD_IT; ++it) {
      cached_blk[it] = 0xffffffffu;
      words[it] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int s = grp; s < nsteps; s += C::NGROUPS) {
      const int sf = s % C::NSF;
      const int so = s % C::NSO;
      // the MMAs that read operand buffer `so` last time have completed
      bool ok = s < C::NSO || mbar_wait(empty_o(so), ((s / C::NSO) & 1) ^ 1, ab, 0x43, s);
      if (!__all_sync(0xffffffffu, ok)) break;  // leave together (abort path)
      uint8_t* sdst = smem + C::OFF_S + so * C::OPS;
      const int64_t cbase = lbeg + static_cast<int64_t>(s) * BK;
      if (DIST == kRademacher) {
        // 128 rows x 2 k-halves, 8 entries each, one Philox call per 128 columns
#pragma unroll
        for (int it = 0; it < RAD_IT; ++it) {
          const int t = wt + it * C::GROUP_THREADS;
          if (t >= 2 * BM) break;
          const uint32_t r = static_cast<uint32_t>(t & (BM - 1));
          const uint32_t hh = static_cast<uint32_t>(t >> 7);
          const int64_t grow = p0 + r;
          const int64_t c0 = cbase + 8 * hh;
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (grow < p.P && c0 < lend) {
            const uint32_t c = static_cast<uint32_t>(c0);
            const uint32_t blk = c >> 7;
            if (blk != cached_blk[it]) {
              words[it] = rademacher_bits(p.key, static_cast<uint32_t>(grow), blk, 0u);
              cached_blk[it] = blk;
            }
            const uint32_t wsel = (c >> 5) & 3u;
            const uint4 wv = words[it];
            const uint32_t w = wsel == 0 ? wv.x : wsel == 1 ? wv.y : wsel == 2 ? wv.z : wv.w;
            const uint32_t bits = w >> (c & 31u);
            // +1.0 = 0x3F80, -1.0 = 0xBF80: the sign bit carries the random bit
            v.x = 0x3F803F80u | ((bits & 1u) << 15) | ((bits & 2u) << 30);
            v.y = 0x3F803F80u | ((bits & 4u) << 13) | ((bits & 8u) << 28);
            v.z = 0x3F803F80u | ((bits & 16u) << 11) | ((bits & 32u) << 26);
            v.w = 0x3F803F80u | ((bits & 64u) << 9) | ((bits & 128u) << 24);
          }
          *reinterpret_cast<uint4*>(sdst + kmaj_off(r, hh)) = v;
        }
      } else {
        // 8 rows x 4 quads per 32 tasks, 4 entries (one Philox call) each; a
        // fixed, unrolled count per thread lets independent chains interleave
        constexpr int GEN_IT = (4 * BM + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
#pragma unroll
        for (int it = 0; it < GEN_IT; ++it) {
          const int t = wt + it * C::GROUP_THREADS;
          if (t >= 4 * BM) break;
          const uint32_t l = static_cast<uint32_t>(t & 31);
          const uint32_t r = static_cast<uint32_t>(t >> 5) * 8u + (l >> 2);
          const uint32_t qd = l & 3u;
          const int64_t grow = p0 + r;
          const int64_t c0 = cbase + 4 * qd;
          uint2 v = make_uint2(0u, 0u);
          if (grow < p.P && c0 < lend) {
            const uint32_t c = static_cast<uint32_t>(c0);
            const float4 a = DIST == kUniform
                                 ? uniform4(p.key, static_cast<uint32_t>(grow), c >> 2, 0u)
                                 : gaussian4(p.key, static_cast<uint32_t>(grow), c >> 2, 0u);
            v = make_uint2(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w));
          }
          *reinterpret_cast<uint2*>(sdst + kmaj_off(r, qd >> 1) + (qd & 1u) * 8u) = v;
        }
      }
      // conversion needs this stage's A tile
      ok = mbar_wait(full_f(sf), (s / C::NSF) & 1, ab, 0x40, s);
      if (!__all_sync(0xffffffffu, ok)) break;
      const float* stg = reinterpret_cast<const float*>(smem + C::OFF_F + sf * C::STAGE_F);
      uint8_t* bhi = smem + C::OFF_BHI + so * C::OPB;
      uint8_t* blo = smem + C::OFF_BLO + so * C::OPB;
      constexpr int CONV_IT = (2 * C::COLS + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
#pragma unroll
      for (int it = 0; it < CONV_IT; ++it) {
        const int i = wt + it * C::GROUP_THREADS;
        if (i >= 2 * cols) break;
        const int hh = i >= cols ? 1 : 0;
        const int j = i - hh * cols;   // column j of this CTA's slice = operand row j
        const int box = j >> 8;        // staging boxes are 256 columns wide
        const int bw = min(cols - box * 256, 256);
        const float* src = stg + box * 256 * BK + (8 * hh) * bw + (j - box * 256);
        float a[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] = src[e * bw];
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          hw[e] = pack_bf16x2(a[2 * e], a[2 * e + 1]);
          const float h0 = __uint_as_float(hw[e] << 16);
          const float h1 = __uint_as_float(hw[e] & 0xffff0000u);
          lw[e] = pack_bf16x2(__fsub_rn(a[2 * e], h0), __fsub_rn(a[2 * e + 1], h1));
        }
        const uint32_t o = kmaj_off(static_cast<uint32_t>(j), static_cast<uint32_t>(hh));
        *reinterpret_cast<uint4*>(bhi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(blo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      if (PAIR)
        fence_proxy_async_cluster();  // the even CTA's MMA reads these operands
      else
        fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        if (PAIR)
          mbar_arrive_cluster(lead_full_o + 8u * so);
        else
          mbar_arrive(full_o(so));
        mbar_arrive(empty_f(sf));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // no CTA leaves while its peer may still address it
  if (warp == WARP_MMA) {
    tc_fence_after();
    __syncwarp();
    if (PAIR)
      tmem_dealloc_pair(tmem, static_cast<uint32_t>(p.tmem_cols));
    else
      tmem_dealloc(tmem, static_cast<uint32_t>(p.tmem_cols));
  }
}

// ---------------------------------------------------------------------------
// Right sketch Y[m x k] = A[m x n] S^T (S[k x n]) on CTA pairs.
//
// The roles of the operands swap: the converted A tile is the MMA's A
// operand (K-major as stored, no transpose), the generated S tile its B
// operand.  A pair owns 512 rows of m: each CTA converts 256 of them and holds
// two TMEM accumulators (m rows 0-127 and 128-255 of its share), so one
// generated S tile serves 512 rows of A.  Each CTA generates half of the
// tile's k rows (the pair MMA splits N between the two CTAs).  Warp roles,
// rings, chains and bounded waits are those of the left kernel.
// ---------------------------------------------------------------------------
struct CfgR {
  static constexpr int ROWS = 256;  // rows of A per CTA (two 128-row accumulators)
  static constexpr int NGROUPS = 4;
  static constexpr int GROUP_WARPS = NUM_WORK_WARPS / NGROUPS;
  static constexpr int GROUP_THREADS = 32 * GROUP_WARPS;
  static constexpr int NSF = 6;
  static constexpr int NSO = 6;
  static constexpr uint32_t STAGE_F = BK * ROWS * 4;  // FP32 staging [256 rows][16]
  static constexpr uint32_t OPA = ROWS * BK * 2;      // hi or lo operand, 2 x 4 KB
  static constexpr uint32_t OPS = 128 * BK * 2;       // this CTA's half of the S tile
  static constexpr uint32_t OFF_F = 0;
  static constexpr uint32_t OFF_AHI = OFF_F + NSF * STAGE_F;
  static constexpr uint32_t OFF_ALO = OFF_AHI + NSO * OPA;
  static constexpr uint32_t OFF_S = OFF_ALO + NSO * OPA;
  static constexpr uint32_t OFF_BAR = OFF_S + NSO * OPS;
  static constexpr uint32_t NUM_BARS = 2 * NSF + 2 * NSO + 3;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NUM_BARS * 8;
  static constexpr uint32_t SMEM = OFF_MISC + 16 + 1024;
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
  static_assert(NGROUPS <= NSF && NGROUPS <= NSO, "worker groups vs ring depth");
};

struct TcRightParams {
  float* part;      // partials [splits][P][Q]
  int64_t P, Q, L;  // P = m, Q = k, L = n
  int64_t chunk;    // contracted length per split (multiple of BK)
  int nq;           // N of the MMA: k rows per pair tile (multiple of 16, <= 256)
  int tmem_cols;    // power of two >= 2 * nq
  PhiloxKey key;
  int* status;
  uint64_t timeout_ns;
};

template <int DIST>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_sketch_bf16x2_right(const __grid_constant__ CUtensorMap tmapA, const TcRightParams p) {
  using C = CfgR;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + C::OFF_BAR;
  auto full_f = [&](int i) { return bar0 + 8u * i; };
  auto empty_f = [&](int i) { return bar0 + 8u * (C::NSF + i); };
  auto full_o = [&](int i) { return bar0 + 8u * (2 * C::NSF + i); };
  auto empty_o = [&](int i) { return bar0 + 8u * (2 * C::NSF + C::NSO + i); };
  const uint32_t acc_full = bar0 + 8u * (2 * C::NSF + 2 * C::NSO);
  const uint32_t acc_empty = acc_full + 8u;
  const uint32_t drain_bar = acc_full + 16u;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::OFF_MISC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank() & 1u;  // 0 = even CTA (MMA issuer)
  const bool leader = rank == 0;
  const int nq = p.nq;
  const int gh = nq / 2;                                       // S rows this CTA generates
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * C::ROWS;  // this CTA's rows of A
  const int64_t q0 = static_cast<int64_t>(blockIdx.y) * nq;       // the pair's k rows
  const int64_t g0 = q0 + static_cast<int64_t>(rank) * gh;        // this CTA's S rows
  const int64_t lbeg = static_cast<int64_t>(blockIdx.z) * p.chunk;
  const int64_t lend = min(p.L, lbeg + p.chunk);
  const int nsteps = static_cast<int>((lend - lbeg + BK - 1) / BK);
  const int nchains = (nsteps + CHAIN - 1) / CHAIN;

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NSF; ++i) {
      mbar_init(full_f(i), 1);
      mbar_init(empty_f(i), C::GROUP_WARPS);
    }
    for (int i = 0; i < C::NSO; ++i) {
      mbar_init(full_o(i), C::GROUP_WARPS * 2);
      mbar_init(empty_o(i), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NUM_EPI_WARPS * 2);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == WARP_MMA) {
    tmem_alloc_pair(smem_u32(tmem_slot), static_cast<uint32_t>(p.tmem_cols));
    tmem_relinquish_pair();
  }
  if (warp == WARP_TMA && lane == 0) tma_prefetch_desc(&tmapA);
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const Abort ab{abort_flag, p.status, p.timeout_ns};
  const uint32_t lead_full_o = mapa_shared(full_o(0), 0u);
  const uint32_t lead_acc_empty = mapa_shared(acc_empty, 0u);

  if (warp == WARP_TMA) {
    if (lane == 0) {
      int issued = 0;
      for (int s = 0; s < nsteps; ++s) {
        const int sf = s % C::NSF;
        if (s >= C::NSF && !mbar_wait(empty_f(sf), ((s / C::NSF) & 1) ^ 1, ab, 0x11, s)) break;
        mbar_arrive_expect_tx(full_f(sf), C::STAGE_F);
        tma_load_2d(sbase + C::OFF_F + sf * C::STAGE_F, &tmapA,
                    static_cast<int32_t>(lbeg + static_cast<int64_t>(s) * BK),
                    static_cast<int32_t>(m0), full_f(sf));
        issued = s + 1;
      }
      if (*abort_flag) {
        for (int s = max(0, issued - C::NSF); s < issued; ++s)
          drain_wait(full_f(s % C::NSF), (s / C::NSF) & 1, 100000000ull);
      }
    }
  } else if (warp == WARP_MMA) {
    if (lane == 0 && leader) {
      const uint32_t idesc = idesc_bf16_f32(256u, static_cast<uint32_t>(nq));
      for (int s = 0; s < nsteps; ++s) {
        const int so = s % C::NSO;
        const int in_chain = s % CHAIN;
        if (s > 0 && in_chain == 0 &&
            !mbar_wait(acc_empty, ((s / CHAIN) - 1) & 1, ab, 0x25, s))
          break;
        if (!mbar_wait(full_o(so), (s / C::NSO) & 1, ab, 0x22, s)) break;
        tc_fence_after();
        const uint64_t bdesc = smem_desc(sbase + C::OFF_S + so * C::OPS, LBO, SBO);
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const uint32_t ab_ = sbase + (pass ? C::OFF_ALO : C::OFF_AHI) + so * C::OPA;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const uint64_t adesc = smem_desc(ab_ + static_cast<uint32_t>(j) * (C::OPA / 2), LBO, SBO);
            mma_bf16_pair(tmem + static_cast<uint32_t>(j * nq), adesc, bdesc, idesc,
                          (in_chain > 0 || pass > 0) ? 1u : 0u);
          }
        }
        mma_commit_pair_both(empty_o(so));
        if (in_chain == CHAIN - 1 || s == nsteps - 1) mma_commit_pair_both(acc_full);
      }
      mma_commit_pair(drain_bar);
      drain_wait(drain_bar, 0, 200000000ull);
    }
  } else if (warp < WARP_WORK0) {
    // ---- epilogue: accumulator j holds rows m0 + 128 j + lane, columns q0 + c ----
    const int quarter = warp & 3;
    const int colset = (warp - WARP_EPI0) >> 2;
    const bool vec_ok = (p.Q % 4) == 0;
    const int nchunk = (nq + 31) / 32;
    for (int c0 = 0; c0 < nchains; ++c0) {
      const bool ok = mbar_wait(acc_full, c0 & 1, ab, 0x34, c0);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      for (int t = colset; t < 2 * nchunk; t += 2) {
        const int j = t / nchunk;
        const int ci = t - j * nchunk;
        uint32_t v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                      static_cast<uint32_t>(j * nq + ci * 32),
                  v);
        tmem_ld_wait();
        const int64_t gm = m0 + j * 128 + quarter * 32 + lane;
        if (gm < p.P) {
          float* drow = p.part + (static_cast<int64_t>(blockIdx.z) * p.P + gm) * p.Q + q0;
#pragma unroll
          for (int e = 0; e < 32; e += 4) {
            const int c = ci * 32 + e;
            if (c >= nq) continue;
            const int64_t col = q0 + c;
            const float a0 = __uint_as_float(v[e]), a1 = __uint_as_float(v[e + 1]);
            const float a2 = __uint_as_float(v[e + 2]), a3 = __uint_as_float(v[e + 3]);
            float* d = drow + c;
            if (vec_ok && col + 4 <= p.Q) {
              if (c0 == 0)
                *reinterpret_cast<float4*>(d) = make_float4(a0, a1, a2, a3);
              else
                red_add_v4(d, a0, a1, a2, a3);
            } else {
              const float vv[4] = {a0, a1, a2, a3};
              for (int u = 0; u < 4; ++u) {
                if (col + u < p.Q) {
                  if (c0 == 0)
                    d[u] = vv[u];
                  else
                    red_add(d + u, vv[u]);
                }
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_acc_empty);
    }
  } else {
    // ---- workers: this CTA's half of the S tile, and its 256 rows of A ----
    const int grp = (warp - WARP_WORK0) / C::GROUP_WARPS;
    const int wt = threadIdx.x - 32 * WARP_WORK0 - grp * C::GROUP_THREADS;
    constexpr int RAD_IT = (2 * 128 + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
    uint32_t cached_blk[RAD_IT];
    uint4 words[RAD_IT];
#pragma unroll
    for (int it = 0; it < RAD_IT; ++it) {
      cached_blk[it] = 0xffffffffu;
      words[it] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int s = grp; s < nsteps; s += C::NGROUPS) {
      const int sf = s % C::NSF;
      const int so = s % C::NSO;
      bool ok = s < C::NSO || mbar_wait(empty_o(so), ((s / C::NSO) & 1) ^ 1, ab, 0x43, s);
      if (!__all_sync(0xffffffffu, ok)) break;
      uint8_t* sdst = smem + C::OFF_S + so * C::OPS;
      const int64_t cbase = lbeg + static_cast<int64_t>(s) * BK;
      if (DIST == kRademacher) {
#pragma unroll
        for (int it = 0; it < RAD_IT; ++it) {
          const int t = wt + it * C::GROUP_THREADS;
          if (t >= 2 * gh) break;
          const uint32_t r = static_cast<uint32_t>(t % gh);
          const uint32_t hh = static_cast<uint32_t>(t / gh);
          const int64_t grow = g0 + r;
          const int64_t c0 = cbase + 8 * hh;
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (grow < p.Q && c0 < lend) {
            const uint32_t c = static_cast<uint32_t>(c0);
            const uint32_t blk = c >> 7;
            if (blk != cached_blk[it]) {
              words[it] = rademacher_bits(p.key, static_cast<uint32_t>(grow), blk, 0u);
              cached_blk[it] = blk;
            }
            const uint32_t wsel = (c >> 5) & 3u;
            const uint4 wv = words[it];
            const uint32_t w = wsel == 0 ? wv.x : wsel == 1 ? wv.y : wsel == 2 ? wv.z : wv.w;
            const uint32_t bits = w >> (c & 31u);
            v.x = 0x3F803F80u | ((bits & 1u) << 15) | ((bits & 2u) << 30);
            v.y = 0x3F803F80u | ((bits & 4u) << 13) | ((bits & 8u) << 28);
            v.z = 0x3F803F80u | ((bits & 16u) << 11) | ((bits & 32u) << 26);
            v.w = 0x3F803F80u | ((bits & 64u) << 9) | ((bits & 128u) << 24);
          }
          *reinterpret_cast<uint4*>(sdst + kmaj_off(r, hh)) = v;
        }
      } else {
        constexpr int GEN_IT = (4 * 128 + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
#pragma unroll
        for (int it = 0; it < GEN_IT; ++it) {
          const int t = wt + it * C::GROUP_THREADS;
          if (t >= 4 * gh) break;
          const uint32_t l = static_cast<uint32_t>(t & 31);
          const uint32_t qd = l & 3u;
          const uint32_t r = static_cast<uint32_t>(t >> 2);  // row, 4 quads per row
          const int64_t grow = g0 + r;
          const int64_t c0 = cbase + 4 * qd;
          uint2 v = make_uint2(0u, 0u);
          if (grow < p.Q && c0 < lend) {
            const uint32_t c = static_cast<uint32_t>(c0);
            const float4 a = DIST == kUniform
                                 ? uniform4(p.key, static_cast<uint32_t>(grow), c >> 2, 0u)
                                 : gaussian4(p.key, static_cast<uint32_t>(grow), c >> 2, 0u);
            v = make_uint2(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w));
          }
          *reinterpret_cast<uint2*>(sdst + kmaj_off(r, qd >> 1) + (qd & 1u) * 8u) = v;
        }
      }
      ok = mbar_wait(full_f(sf), (s / C::NSF) & 1, ab, 0x40, s);
      if (!__all_sync(0xffffffffu, ok)) break;
      const float* stg = reinterpret_cast<const float*>(smem + C::OFF_F + sf * C::STAGE_F);
      uint8_t* ahi = smem + C::OFF_AHI + so * C::OPA;
      uint8_t* alo = smem + C::OFF_ALO + so * C::OPA;
      constexpr int CONV_IT = (2 * C::ROWS + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
#pragma unroll
      for (int it = 0; it < CONV_IT; ++it) {
        const int i = wt + it * C::GROUP_THREADS;
        const int row = i >> 1;   // 0..255: accumulator row / 128, lane row % 128
        const int hh = i & 1;
        const float4 x0 = *reinterpret_cast<const float4*>(stg + row * BK + 8 * hh);
        const float4 x1 = *reinterpret_cast<const float4*>(stg + row * BK + 8 * hh + 4);
        const float a[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          hw[e] = pack_bf16x2(a[2 * e], a[2 * e + 1]);
          const float h0 = __uint_as_float(hw[e] << 16);
          const float h1 = __uint_as_float(hw[e] & 0xffff0000u);
          lw[e] = pack_bf16x2(__fsub_rn(a[2 * e], h0), __fsub_rn(a[2 * e + 1], h1));
        }
        const uint32_t o = static_cast<uint32_t>(row >> 7) * (C::OPA / 2) +
                           kmaj_off(static_cast<uint32_t>(row & 127), static_cast<uint32_t>(hh));
        *reinterpret_cast<uint4*>(ahi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(alo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      fence_proxy_async_cluster();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_cluster(lead_full_o + 8u * so);
        mbar_arrive(empty_f(sf));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == WARP_MMA) {
    tc_fence_after();
    __syncwarp();
    tmem_dealloc_pair(tmem, static_cast<uint32_t>(p.tmem_cols));
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

template <bool PAIR>
cudaError_t set_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_sketch_bf16x2_left<kGaussian, PAIR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<PAIR>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sketch_bf16x2_left<kRademacher, PAIR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<PAIR>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sketch_bf16x2_left<kUniform, PAIR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<PAIR>::SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

template <bool PAIR>
void fill_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr, dim3 grid, cudaStream_t st) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = grid;
  cfg->blockDim = dim3(NTHREADS, 1, 1);
  cfg->dynamicSmemBytes = Cfg<PAIR>::SMEM;
  cfg->stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PAIR ? 2 : 1;  // a CTA pair must be adjacent in x
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
}

// SMs that can hold CTA pairs of this kernel at once (a pair must fit in one
// GPC), or -1.
int64_t pair_slots() {
  static int64_t cache = 0;
  if (cache != 0) return cache;
  if (set_smem_attr<true>() != cudaSuccess) return cache = -1;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<true>(&cfg, attr, dim3(2, 1, 1), nullptr);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_sketch_bf16x2_left<kGaussian, true>, &cfg) !=
          cudaSuccess ||
      clusters <= 0) {
    cudaGetLastError();
    return cache = -1;
  }
  return cache = static_cast<int64_t>(clusters) * 2;
}

struct Plan {
  bool pair;
  int nt, tmem_cols, boxw;
  int64_t tiles_q, tiles_p;  // tiles_p is even for pairs
  int splits;
  int64_t chunk;
};

// Tile width, pairing and split-K count: whole waves of one CTA per SM.
Plan plan_left(const GemmShape& s) {
  Plan pl;
  pl.nt = s.Q > 256 ? 512 : static_cast<int>((s.Q + 15) / 16 * 16);
  pl.tmem_cols = 32;
  while (pl.tmem_cols < pl.nt) pl.tmem_cols *= 2;
  pl.tiles_q = (s.Q + pl.nt - 1) / pl.nt;
  const int64_t tp = (s.P + BM - 1) / BM;
  int64_t slots = num_sms_tc();
  pl.pair = false;
  if (tp >= 2) {
    const int64_t ps = pair_slots();
    if (ps > 0) {
      pl.pair = true;
      slots = ps;
    }
  }
  // each CTA loads one contiguous slice of the tile's columns (half of them
  // in a pair) as boxes of at most 256 columns
  const int cta_cols = pl.pair ? pl.nt / 2 : pl.nt;
  pl.boxw = cta_cols > 256 ? 256 : cta_cols;
  pl.tiles_p = pl.pair ? (tp + 1) / 2 * 2 : tp;
  const int64_t tiles = pl.tiles_q * pl.tiles_p;
  const int64_t steps_total = (s.L + BK - 1) / BK;
  int64_t smax = steps_total / 8;  // at least 8 stages per split
  if (smax > 128) smax = 128;
  if (smax < 1) smax = 1;
  int64_t best = 1;
  double best_eff = -1.0;
  for (int64_t sp = 1; sp <= smax; ++sp) {
    const int64_t ctas = tiles * sp;
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = static_cast<double>(ctas) / static_cast<double>(waves * slots);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = sp;
    }
    if (ctas >= 4 * slots) break;
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

template <int DIST, bool PAIR>
cudaError_t launch_left(const CUtensorMap& map, const TcParams& p, dim3 grid, cudaStream_t st) {
  cudaError_t e = set_smem_attr<PAIR>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<PAIR>(&cfg, attr, grid, st);
  return cudaLaunchKernelEx(&cfg, k_sketch_bf16x2_left<DIST, PAIR>, map, p);
}

template <bool PAIR>
cudaError_t launch_dist(int dist, const CUtensorMap& map, const TcParams& p, dim3 grid,
                        cudaStream_t st) {
  if (dist == kRademacher) return launch_left<kRademacher, PAIR>(map, p, grid, st);
  if (dist == kUniform) return launch_left<kUniform, PAIR>(map, p, grid, st);
  return launch_left<kGaussian, PAIR>(map, p, grid, st);
}

cudaError_t set_smem_attr_right() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_sketch_bf16x2_right<kGaussian>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, CfgR::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sketch_bf16x2_right<kRademacher>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, CfgR::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sketch_bf16x2_right<kUniform>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, CfgR::SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

// Right sketch: pairs of CTAs own 512 rows of m and nq <= 256 rows of k; the
// split count keeps the partials (splits x m x k floats) to a few hundred MB.
Plan plan_right(const GemmShape& s) {
  Plan pl;
  pl.pair = true;
  pl.nt = s.Q > 256 ? 256 : static_cast<int>((s.Q + 15) / 16 * 16);
  pl.tmem_cols = 32;
  while (pl.tmem_cols < 2 * pl.nt) pl.tmem_cols *= 2;
  pl.boxw = BK;
  pl.tiles_p = (s.P + 2 * CfgR::ROWS - 1) / (2 * CfgR::ROWS) * 2;  // CTAs along m
  pl.tiles_q = (s.Q + pl.nt - 1) / pl.nt;
  int64_t slots = pair_slots();
  if (slots <= 0) slots = num_sms_tc();
  const int64_t tiles = pl.tiles_p * pl.tiles_q;
  const int64_t steps_total = (s.L + BK - 1) / BK;
  int64_t smax = steps_total / 8;
  const int64_t part_bytes = s.P * s.Q * 4;
  const int64_t cap = part_bytes > 0 ? (int64_t(1) << 29) / part_bytes : 128;
  if (smax > cap) smax = cap;
  if (smax > 128) smax = 128;
  if (smax < 1) smax = 1;
  int64_t best = 1;
  double best_eff = -1.0;
  for (int64_t sp = 1; sp <= smax; ++sp) {
    const int64_t ctas = tiles * sp;
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = static_cast<double>(ctas) / static_cast<double>(waves * slots);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = sp;
    }
  }
  int64_t chunk = (s.L + best - 1) / best;
  chunk = (chunk + BK - 1) / BK * BK;
  pl.chunk = chunk;
  pl.splits = static_cast<int>((s.L + chunk - 1) / chunk);
  return pl;
}

template <int DIST>
cudaError_t launch_right(const CUtensorMap& map, const TcRightParams& p, dim3 grid,
                         cudaStream_t st) {
  cudaError_t e = set_smem_attr_right();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<true>(&cfg, attr, grid, st);
  cfg.dynamicSmemBytes = CfgR::SMEM;
  return cudaLaunchKernelEx(&cfg, k_sketch_bf16x2_right<DIST>, map, p);
}

}  // namespace

size_t tc_workspace_bytes(const GemmShape& s) {
  const Plan pl = s.left ? plan_left(s) : plan_right(s);
  return static_cast<size_t>(pl.splits) * static_cast<size_t>(s.P) * static_cast<size_t>(s.Q) *
         sizeof(float);
}

sk_status tc_check(const GemmShape& s, const float* A, int64_t lda, const float* Y, int64_t ldy) {
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(Y) & 15u))
    return SK_EINVAL;
  if (lda % 4 != 0 || ldy % 4 != 0) return SK_EINVAL;
  if (s.L > (1LL << 31) - 64 || s.Q > (1LL << 31) - 1024) return SK_EUNSUPPORTED;
  return SK_OK;
}

cudaError_t tc_sketch_right(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                            float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st) {
  const Plan pl = plan_right(s);
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  CUtensorMap map;
  // A[m x n]: n innermost; one box = 16 columns of n x 256 rows of m
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(s.L), static_cast<cuuint64_t>(s.P)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(lda) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(CfgR::ROWS)};
  const cuuint32_t estride[2] = {1, 1};
  CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim,
                    gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TcRightParams p;
  p.P = s.P;
  p.Q = s.Q;
  p.L = s.L;
  p.chunk = pl.chunk;
  p.nq = pl.nt;
  p.tmem_cols = pl.tmem_cols;
  p.key = make_key(h->seed);
  p.status = h->d_status;
  p.timeout_ns = 2000000000ull;
  const size_t need = static_cast<size_t>(pl.splits) * s.P * s.Q * sizeof(float);
  if (ws == nullptr || ws_bytes < need) return cudaErrorInvalidValue;
  p.part = static_cast<float*>(ws);
  dim3 grid(static_cast<unsigned>(pl.tiles_p), static_cast<unsigned>(pl.tiles_q),
            static_cast<unsigned>(pl.splits));
  prof_mark(h->prof_start, st);
  cudaError_t e;
  if (h->dist == kRademacher)
    e = launch_right<kRademacher>(map, p, grid, st);
  else if (h->dist == kUniform)
    e = launch_right<kUniform>(map, p, grid, st);
  else
    e = launch_right<kGaussian>(map, p, grid, st);
  prof_mark(h->prof_stop, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return splitk_reduce(static_cast<float*>(ws), pl.splits, s.P, s.Q, h->scale, Y, ldy, st);
}

cudaError_t tc_sketch(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                      float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!s.left) return tc_sketch_right(h, s, A, lda, Y, ldy, ws, ws_bytes, st);
  const Plan pl = plan_left(s);
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(s.Q), static_cast<cuuint64_t>(s.L)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(lda) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(pl.boxw), static_cast<cuuint32_t>(BK)};
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
  p.tmem_cols = pl.tmem_cols;
  p.key = make_key(h->seed);
  p.status = h->d_status;
  p.timeout_ns = 2000000000ull;  // 2 s per wait: far beyond any healthy stage
  const size_t need = static_cast<size_t>(pl.splits) * s.P * s.Q * sizeof(float);
  if (ws == nullptr || ws_bytes < need) return cudaErrorInvalidValue;
  p.part = static_cast<float*>(ws);
  dim3 grid(static_cast<unsigned>(pl.tiles_p), static_cast<unsigned>(pl.tiles_q),
            static_cast<unsigned>(pl.splits));
  prof_mark(h->prof_start, st);
  const cudaError_t e = pl.pair ? launch_dist<true>(h->dist, map, p, grid, st)
                                : launch_dist<false>(h->dist, map, p, grid, st);
  prof_mark(h->prof_stop, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  // fixed-order sum of the split partials, times 1/sqrt(k), into Y
  return splitk_reduce(static_cast<float*>(ws), pl.splits, s.P, s.Q, h->scale, Y, ldy, st);
}

}  // namespace sk

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

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

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

// One left-sketch problem of a launch (a single sketch, or one member of a
// batch).  Lives in device memory; the tensor map must be 64-byte aligned.
struct alignas(128) LeftProblem {
  CUtensorMap map;  // A[m x n] (n innermost), box {boxw, 16}
  float* part;      // partials [splits][P][Q] of this problem
  int64_t P, Q, L;  // P = k, Q = n, L = m
  int64_t chunk;    // contracted length per split (multiple of BK)
  int nt;           // output columns per tile: multiple of 16 up to 256, or 512
  int dist;         // sk_dist of S
  PhiloxKey key;
};

// A unit of work: tile (tp, tq) of split z of problem `prob`.  With pairs,
// tp indexes 256-row tiles and the CTA of rank r takes rows 128 r .. of it.
struct LeftItem {
  int prob, tp, tq, z;
};

// Work lists: the items of pair (or single CTA) i are
// items[begin[i] .. begin[i+1]).
struct LeftSched {
  const LeftProblem* probs;
  const LeftItem* items;
  const int* begin;
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

// Per-item geometry shared by every role.
struct ItemGeo {
  const LeftProblem* pr;
  int64_t p0, q0, lbeg, lend;
  int nsteps, nt, nmma, nh, bh, cols, dist;
};

template <bool PAIR>
__device__ __forceinline__ ItemGeo item_geo(const LeftSched& sc, int idx, uint32_t rank) {
  const LeftItem it = sc.items[idx];
  ItemGeo g;
  g.pr = sc.probs + it.prob;
  g.nt = g.pr->nt;
  g.dist = g.pr->dist;
  g.nmma = g.nt > 256 ? 2 : 1;
  g.nh = g.nt > 256 ? 256 : g.nt;
  g.bh = PAIR ? g.nh / 2 : g.nh;
  g.cols = g.nmma * g.bh;
  g.p0 = static_cast<int64_t>(it.tp) * (PAIR ? 2 * BM : BM) + static_cast<int64_t>(rank) * BM;
  g.q0 = static_cast<int64_t>(it.tq) * g.nt;
  g.lbeg = static_cast<int64_t>(it.z) * g.pr->chunk;
  g.lend = min(g.pr->L, g.lbeg + g.pr->chunk);
  g.nsteps = static_cast<int>((g.lend - g.lbeg + BK - 1) / BK);
  return g;
}

// Generate this CTA's BF16 S tile [128 x 16] of one stage.  Rademacher tasks
// keep their Philox words across the 8 stages one call covers.
template <int DIST, class C>
__device__ __forceinline__ void gen_stage(uint8_t* sdst, const ItemGeo& g, int64_t cbase, int wt,
                                          uint32_t* cached_blk, uint4* words) {
  if (DIST == kRademacher) {
    constexpr int RAD_IT = (2 * BM + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
#pragma unroll
    for (int it = 0; it < RAD_IT; ++it) {
      const int t = wt + it * C::GROUP_THREADS;
      if (t >= 2 * BM) break;
      const uint32_t r = static_cast<uint32_t>(t & (BM - 1));
      const uint32_t hh = static_cast<uint32_t>(t >> 7);
      const int64_t grow = g.p0 + r;
      const int64_t c0 = cbase + 8 * hh;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (grow < g.pr->P && c0 < g.lend) {
        const uint32_t c = static_cast<uint32_t>(c0);
        const uint32_t blk = c >> 7;
        if (blk != cached_blk[it]) {
          words[it] = rademacher_bits(g.pr->key, static_cast<uint32_t>(grow), blk, 0u);
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
      const int64_t grow = g.p0 + r;
      const int64_t c0 = cbase + 4 * qd;
      uint2 v = make_uint2(0u, 0u);
      if (grow < g.pr->P && c0 < g.lend) {
        const uint32_t c = static_cast<uint32_t>(c0);
        const float4 a = DIST == kUniform
                             ? uniform4(g.pr->key, static_cast<uint32_t>(grow), c >> 2, 0u)
                             : gaussian4(g.pr->key, static_cast<uint32_t>(grow), c >> 2, 0u);
        v = make_uint2(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w));
      }
      *reinterpret_cast<uint2*>(sdst + kmaj_off(r, qd >> 1) + (qd & 1u) * 8u) = v;
    }
  }
}

// Split this CTA's FP32 A columns of one stage (staging: boxes of <= 256
// columns x 16 rows) into BF16 hi / lo operand rows (row j = column j).
template <class C>
__device__ __forceinline__ void convert_stage(const float* stg, uint8_t* bhi, uint8_t* blo,
                                              int cols, int wt) {
  constexpr int CONV_IT = (2 * C::COLS + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
#pragma unroll
  for (int it = 0; it < CONV_IT; ++it) {
    const int i = wt + it * C::GROUP_THREADS;
    if (i >= 2 * cols) break;
    const int hh = i >= cols ? 1 : 0;
    const int j = i - hh * cols;
    const int box = j >> 8;
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
}

// Persistent left-sketch kernel: each pair (or single CTA) runs its list of
// items back to back; ring positions, barrier phases and accumulation chains
// are counted across items (g = stage counter, gc = chain counter).  DIST is
// the distribution of every item, or kMixed to read it per item (batches).
constexpr int kMixed = -1;

template <int DIST, bool PAIR>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_sketch_bf16x2_left(const LeftSched sc) {
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
  const int unit = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
  const int ib = sc.begin[unit];
  const int ie = sc.begin[unit + 1];

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
  if (warp == WARP_MMA) {  // the accumulator of every item: up to 512 TMEM columns
    if (PAIR) {
      tmem_alloc_pair(smem_u32(tmem_slot), static_cast<uint32_t>(NT_MAX));
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), static_cast<uint32_t>(NT_MAX));
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // the peer's barriers exist before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const Abort ab{abort_flag, sc.status, sc.timeout_ns};
  // barriers of the even CTA, addressed from either CTA
  const uint32_t lead_full_o = PAIR ? mapa_shared(full_o(0), 0u) : full_o(0);
  const uint32_t lead_acc_empty = PAIR ? mapa_shared(acc_empty, 0u) : acc_empty;

  if (warp == WARP_TMA) {
    if (lane == 0) {
      int g = 0;
      int issued = 0;
      for (int idx = ib; idx < ie && !*abort_flag; ++idx) {
        const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
        const CUtensorMap* map = &ig.pr->map;
        tma_prefetch_desc(map);
        const uint32_t tx = static_cast<uint32_t>(ig.cols * BK * 4);
        const int64_t x0 = ig.q0 + static_cast<int64_t>(rank) * ig.cols;
        for (int s = 0; s < ig.nsteps; ++s, ++g) {
          const int sf = g % C::NSF;
          if (g >= C::NSF && !mbar_wait(empty_f(sf), ((g / C::NSF) & 1) ^ 1, ab, 0x11, g)) break;
          mbar_arrive_expect_tx(full_f(sf), tx);
          const int32_t y = static_cast<int32_t>(ig.lbeg + static_cast<int64_t>(s) * BK);
          for (int b = 0; b * 256 < ig.cols; ++b)
            tma_load_2d(sbase + C::OFF_F + sf * C::STAGE_F + static_cast<uint32_t>(b * 256 * BK * 4),
                        map, static_cast<int32_t>(x0 + b * 256), y, full_f(sf));
          issued = g + 1;
        }
      }
      if (*abort_flag) {  // let the copies already issued land before leaving
        for (int t = max(0, issued - C::NSF); t < issued; ++t)
          drain_wait(full_f(t % C::NSF), (t / C::NSF) & 1, 100000000ull);
      }
    }
  } else if (warp == WARP_MMA) {
    if (lane == 0 && leader) {
      int g = 0, gc = 0;
      bool stop = false;
      for (int idx = ib; idx < ie && !stop; ++idx) {
        const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
        const uint32_t idesc = idesc_bf16_f32(PAIR ? 256u : 128u, static_cast<uint32_t>(ig.nh));
        for (int s = 0; s < ig.nsteps; ++s, ++g) {
          const int so = g % C::NSO;
          const int in_chain = s % CHAIN;
          // a new chain may start only after every epilogue has read the last one
          if (in_chain == 0 && gc > 0 && !mbar_wait(acc_empty, (gc - 1) & 1, ab, 0x25, gc)) {
            stop = true;
            break;
          }
          if (!mbar_wait(full_o(so), (g / C::NSO) & 1, ab, 0x22, g)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint64_t adesc = smem_desc(sbase + C::OFF_S + so * C::OPS, LBO, SBO);
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            const uint32_t bb = sbase + (pass ? C::OFF_BLO : C::OFF_BHI) + so * C::OPB;
            for (int h = 0; h < ig.nmma; ++h) {
              const uint64_t bdesc =
                  smem_desc(bb + static_cast<uint32_t>(h * ig.bh / 8) * SBO, LBO, SBO);
              const uint32_t acc = (in_chain > 0 || pass > 0) ? 1u : 0u;
              if (PAIR)
                mma_bf16_pair(tmem + static_cast<uint32_t>(h) * 256u, adesc, bdesc, idesc, acc);
              else
                mma_bf16(tmem + static_cast<uint32_t>(h) * 256u, adesc, bdesc, idesc, acc);
            }
          }
          const bool chain_end = in_chain == CHAIN - 1 || s == ig.nsteps - 1;
          if (PAIR) {  // operands and accumulator are both CTAs'
            mma_commit_pair_both(empty_o(so));
            if (chain_end) mma_commit_pair_both(acc_full);
          } else {
            mma_commit(empty_o(so));
            if (chain_end) mma_commit(acc_full);
          }
          if (chain_end) ++gc;
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
    // ---- epilogue: add each finished chain into the item's FP32 partial ----
    const int quarter = warp & 3;
    const int colset = (warp - WARP_EPI0) >> 2;  // 0 or 1: even / odd 32-column chunks
    const int row = quarter * 32 + lane;
    int gc = 0;
    bool stop = false;
    for (int idx = ib; idx < ie && !stop; ++idx) {
      const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
      const LeftItem it = sc.items[idx];
      const int64_t gp = ig.p0 + row;
      const int64_t P = ig.pr->P, Q = ig.pr->Q;
      float* dst_row = ig.pr->part + (static_cast<int64_t>(it.z) * P + gp) * Q + ig.q0;
      const bool vec_ok = (Q % 4) == 0;
      const int nchains = (ig.nsteps + CHAIN - 1) / CHAIN;
      for (int c0 = 0; c0 < nchains; ++c0, ++gc) {
        const bool ok = mbar_wait(acc_full, gc & 1, ab, 0x34, gc);
        if (!__all_sync(0xffffffffu, ok)) {  // tcgen05.ld below is warp-collective
          stop = true;
          break;
        }
        tc_fence_after();
        // TMEM column h*256 + c holds B row c of instruction h: with a pair,
        // rows c < bh are the even CTA's columns h*bh + c of the tile and rows
        // c >= bh the odd CTA's columns cols + h*bh + (c - bh)
        for (int ci = colset; ci * 32 < (ig.nmma - 1) * 256 + ig.nh; ci += 2) {
          uint32_t v[32];
          tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                        static_cast<uint32_t>(ci * 32),
                    v);
          tmem_ld_wait();
          if (gp < P) {
#pragma unroll
            for (int e = 0; e < 32; e += 4) {  // bh is a multiple of 8: groups never straddle
              const int tcol = ci * 32 + e;
              const int h = tcol >> 8;
              const int c = tcol & 255;
              if (c >= ig.nh) continue;
              const int tn = PAIR ? (c < ig.bh ? h * ig.bh + c : ig.cols + h * ig.bh + (c - ig.bh))
                                  : tcol;
              const int64_t col = ig.q0 + tn;
              float* d = dst_row + tn;
              const float a0 = __uint_as_float(v[e]), a1 = __uint_as_float(v[e + 1]);
              const float a2 = __uint_as_float(v[e + 2]), a3 = __uint_as_float(v[e + 3]);
              if (vec_ok && col + 4 <= Q) {
                if (c0 == 0)
                  *reinterpret_cast<float4*>(d) = make_float4(a0, a1, a2, a3);
                else
                  red_add_v4(d, a0, a1, a2, a3);
              } else {
                const float vv[4] = {a0, a1, a2, a3};
                for (int u = 0; u < 4; ++u) {
                  if (col + u < Q) {
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
    }
  } else {
    // ---- workers: generate this CTA's S tile and convert its A columns ----
    // group grp handles the stages g = grp (mod NGROUPS)
    const int grp = (warp - WARP_WORK0) / C::GROUP_WARPS;
    const int wt = threadIdx.x - 32 * WARP_WORK0 - grp * C::GROUP_THREADS;
    constexpr int RAD_IT = (2 * BM + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
    uint32_t cached_blk[RAD_IT];
    uint4 words[RAD_IT];
    int g = 0;
    bool stop = false;
    for (int idx = ib; idx < ie && !stop; ++idx) {
      const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
#pragma unroll
      for (int it = 0; it < RAD_IT; ++it) {  // Philox words belong to one problem and row
        cached_blk[it] = 0xffffffffu;
        words[it] = make_uint4(0u, 0u, 0u, 0u);
      }
      for (int s = 0; s < ig.nsteps; ++s, ++g) {
        if (g % C::NGROUPS != grp) continue;
        const int sf = g % C::NSF;
        const int so = g % C::NSO;
        // the MMAs that read operand buffer `so` last time have completed
        bool ok = g < C::NSO || mbar_wait(empty_o(so), ((g / C::NSO) & 1) ^ 1, ab, 0x43, g);
        if (!__all_sync(0xffffffffu, ok)) {  // leave together (abort path)
          stop = true;
          break;
        }
        uint8_t* sdst = smem + C::OFF_S + so * C::OPS;
        const int64_t cbase = ig.lbeg + static_cast<int64_t>(s) * BK;
        if (DIST != kMixed)
          gen_stage<DIST, C>(sdst, ig, cbase, wt, cached_blk, words);
        else if (ig.dist == kRademacher)
          gen_stage<kRademacher, C>(sdst, ig, cbase, wt, cached_blk, words);
        else if (ig.dist == kUniform)
          gen_stage<kUniform, C>(sdst, ig, cbase, wt, cached_blk, words);
        else
          gen_stage<kGaussian, C>(sdst, ig, cbase, wt, cached_blk, words);
        // conversion needs this stage's A tile
        ok = mbar_wait(full_f(sf), (g / C::NSF) & 1, ab, 0x40, g);
        if (!__all_sync(0xffffffffu, ok)) {
          stop = true;
          break;
        }
        convert_stage<C>(reinterpret_cast<const float*>(smem + C::OFF_F + sf * C::STAGE_F),
                         smem + C::OFF_BHI + so * C::OPB, smem + C::OFF_BLO + so * C::OPB,
                         ig.cols, wt);
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
  }

  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // no CTA leaves while its peer may still address it
  if (warp == WARP_MMA) {
    tc_fence_after();
    __syncwarp();
    if (PAIR)
      tmem_dealloc_pair(tmem, static_cast<uint32_t>(NT_MAX));
    else
      tmem_dealloc(tmem, static_cast<uint32_t>(NT_MAX));
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

template <int DIST, bool PAIR>
cudaError_t set_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_sketch_bf16x2_left<DIST, PAIR>,
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
  if (set_smem_attr<kMixed, true>() != cudaSuccess) return cache = -1;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<true>(&cfg, attr, dim3(2, 1, 1), nullptr);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_sketch_bf16x2_left<kMixed, true>, &cfg) !=
          cudaSuccess ||
      clusters <= 0) {
    cudaGetLastError();
    return cache = -1;
  }
  return cache = static_cast<int64_t>(clusters) * 2;
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

// Row-major FP32 matrix [rows x cols] (cols innermost) with boxes of
// {box_cols, box_rows}; zero fill outside the matrix.
bool encode_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld,
                int box_cols, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return false;
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstride,
             box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Geometry of one left problem.
struct LeftPlan {
  bool pair;
  int nt, boxw;
  int64_t tiles_p, tiles_q;  // tiles_p counts pair tiles (256 rows) when pair
  int splits;
  int64_t chunk;
  int64_t steps;             // stages of one item
};

LeftPlan left_geometry(const GemmShape& s, bool pair) {
  LeftPlan pl;
  pl.pair = pair;
  pl.nt = s.Q > 256 ? 512 : static_cast<int>((s.Q + 15) / 16 * 16);
  const int cta_cols = pair ? pl.nt / 2 : pl.nt;
  pl.boxw = cta_cols > 256 ? 256 : cta_cols;
  pl.tiles_q = (s.Q + pl.nt - 1) / pl.nt;
  pl.tiles_p = (s.P + (pair ? 2 * BM : BM) - 1) / (pair ? 2 * BM : BM);
  pl.splits = 1;
  pl.chunk = (s.L + BK - 1) / BK * BK;
  pl.steps = pl.chunk / BK;
  return pl;
}

void set_splits(LeftPlan* pl, const GemmShape& s, int64_t splits) {
  if (splits < 1) splits = 1;
  int64_t chunk = (s.L + splits - 1) / splits;
  chunk = (chunk + BK - 1) / BK * BK;
  pl->chunk = chunk;
  pl->splits = static_cast<int>((s.L + chunk - 1) / chunk);
  pl->steps = chunk / BK;
}

// A single sketch: pairs when the output has at least two 128-row tiles;
// splits that fill whole waves of the resident units.
LeftPlan plan_left(const GemmShape& s) {
  const int64_t tp = (s.P + BM - 1) / BM;
  const int64_t ps = tp >= 2 ? pair_slots() : -1;
  LeftPlan pl = left_geometry(s, ps > 0);
  const int64_t units = pl.pair ? ps / 2 : num_sms_tc();
  const int64_t tiles = pl.tiles_p * pl.tiles_q;
  const int64_t steps_total = (s.L + BK - 1) / BK;
  int64_t smax = steps_total / 8;  // at least 8 stages per split
  if (smax > 128) smax = 128;
  if (smax < 1) smax = 1;
  int64_t best = 1;
  double best_eff = -1.0;
  for (int64_t sp = 1; sp <= smax; ++sp) {
    const int64_t items = tiles * sp;
    const int64_t waves = (items + units - 1) / units;
    const double eff = static_cast<double>(items) / static_cast<double>(waves * units);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = sp;
    }
    if (items >= 4 * units) break;
  }
  set_splits(&pl, s, best);
  return pl;
}

// Host image of a work list: problems (128-byte aligned), items, per-unit
// begin offsets, packed into one buffer for a single upload.
struct HostSched {
  std::vector<LeftProblem> probs;
  std::vector<LeftItem> items;
  std::vector<int> begin;
  size_t off_items = 0, off_begin = 0, bytes = 0;
  std::vector<uint8_t> blob;
};

// Items of every problem, longest first, each to the least-loaded of at most
// `max_units` units (pairs or CTAs).
void build_items(const std::vector<LeftPlan>& plans, int64_t max_units, HostSched* hs) {
  struct Cand {
    LeftItem it;
    double cost;
  };
  std::vector<Cand> cands;
  for (size_t pi = 0; pi < plans.size(); ++pi) {
    const LeftPlan& pl = plans[pi];
    const double cost = static_cast<double>(pl.steps) * (static_cast<double>(pl.nt) + 256.0);
    for (int64_t z = 0; z < pl.splits; ++z)
      for (int64_t tq = 0; tq < pl.tiles_q; ++tq)
        for (int64_t tp = 0; tp < pl.tiles_p; ++tp)
          cands.push_back({{static_cast<int>(pi), static_cast<int>(tp), static_cast<int>(tq),
                            static_cast<int>(z)},
                           cost});
  }
  std::stable_sort(cands.begin(), cands.end(),
                   [](const Cand& a, const Cand& b) { return a.cost > b.cost; });
  const int64_t units = std::max<int64_t>(1, std::min<int64_t>(max_units, cands.size()));
  std::vector<double> load(units, 0.0);
  std::vector<std::vector<LeftItem>> per(units);
  for (const Cand& c : cands) {
    int64_t best = 0;
    for (int64_t u = 1; u < units; ++u)
      if (load[u] < load[best]) best = u;
    load[best] += c.cost;
    per[best].push_back(c.it);
  }
  hs->items.clear();
  hs->begin.assign(1, 0);
  for (int64_t u = 0; u < units; ++u) {
    for (const LeftItem& it : per[u]) hs->items.push_back(it);
    hs->begin.push_back(static_cast<int>(hs->items.size()));
  }
}

void pack_sched(HostSched* hs) {
  const size_t pb = hs->probs.size() * sizeof(LeftProblem);
  hs->off_items = (pb + 255) / 256 * 256;
  const size_t ib = hs->items.size() * sizeof(LeftItem);
  hs->off_begin = (hs->off_items + ib + 255) / 256 * 256;
  hs->bytes = hs->off_begin + hs->begin.size() * sizeof(int);
  hs->blob.assign(hs->bytes, 0);
  memcpy(hs->blob.data(), hs->probs.data(), pb);
  memcpy(hs->blob.data() + hs->off_items, hs->items.data(), ib);
  memcpy(hs->blob.data() + hs->off_begin, hs->begin.data(), hs->begin.size() * sizeof(int));
}

LeftSched device_sched(const HostSched& hs, void* dbuf, int* status) {
  LeftSched sc;
  uint8_t* b = static_cast<uint8_t*>(dbuf);
  sc.probs = reinterpret_cast<const LeftProblem*>(b);
  sc.items = reinterpret_cast<const LeftItem*>(b + hs.off_items);
  sc.begin = reinterpret_cast<const int*>(b + hs.off_begin);
  sc.status = status;
  sc.timeout_ns = 2000000000ull;  // 2 s per wait: far beyond any healthy stage
  return sc;
}

template <int DIST, bool PAIR>
cudaError_t launch_left(const LeftSched& sc, int64_t units, cudaStream_t st) {
  cudaError_t e = set_smem_attr<DIST, PAIR>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<PAIR>(&cfg, attr, dim3(static_cast<unsigned>(units * (PAIR ? 2 : 1)), 1, 1), st);
  return cudaLaunchKernelEx(&cfg, k_sketch_bf16x2_left<DIST, PAIR>, sc);
}

template <bool PAIR>
cudaError_t launch_left_dist(int dist, const LeftSched& sc, int64_t units, cudaStream_t st) {
  if (dist == kRademacher) return launch_left<kRademacher, PAIR>(sc, units, st);
  if (dist == kUniform) return launch_left<kUniform, PAIR>(sc, units, st);
  return launch_left<kGaussian, PAIR>(sc, units, st);
}

bool fill_problem(LeftProblem* pr, const LeftPlan& pl, const GemmShape& s, const float* A,
                  int64_t lda, float* part, uint64_t seed, int dist) {
  memset(pr, 0, sizeof(*pr));
  if (!encode_map(&pr->map, A, s.L, s.Q, lda, pl.boxw, BK)) return false;
  pr->part = part;
  pr->P = s.P;
  pr->Q = s.Q;
  pr->L = s.L;
  pr->chunk = pl.chunk;
  pr->nt = pl.nt;
  pr->dist = dist;
  pr->key = make_key(seed);
  return true;
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

struct Plan {
  int nt, tmem_cols;
  int64_t tiles_p, tiles_q;
  int splits;
  int64_t chunk;
};

// Right sketch: pairs of CTAs own 512 rows of m and nq <= 256 rows of k; the
// split count keeps the partials (splits x m x k floats) to a few hundred MB.
Plan plan_right(const GemmShape& s) {
  Plan pl;
  pl.nt = s.Q > 256 ? 256 : static_cast<int>((s.Q + 15) / 16 * 16);
  pl.tmem_cols = 32;
  while (pl.tmem_cols < 2 * pl.nt) pl.tmem_cols *= 2;
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

cudaError_t grow_device(void** buf, size_t* have, size_t need) {
  if (*have >= need) return cudaSuccess;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(buf, need);
  if (e != cudaSuccess) return e;
  *have = need;
  return cudaSuccess;
}

}  // namespace

size_t tc_workspace_bytes(const GemmShape& s) {
  if (s.left) {
    const LeftPlan pl = plan_left(s);
    return static_cast<size_t>(pl.splits) * s.P * s.Q * sizeof(float);
  }
  const Plan pl = plan_right(s);
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
  CUtensorMap map;
  // A[m x n]: n innermost; one box = 16 columns of n x 256 rows of m
  if (!encode_map(&map, A, s.P, s.L, lda, BK, CfgR::ROWS)) return cudaErrorInvalidValue;
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
  const LeftPlan pl = plan_left(s);
  const size_t need = static_cast<size_t>(pl.splits) * s.P * s.Q * sizeof(float);
  if (ws == nullptr || ws_bytes < need) return cudaErrorInvalidValue;
  sk_sketch* hm = const_cast<sk_sketch*>(h);
  // The work list depends only on these; upload it again only when they change.
  const uint64_t key[8] = {reinterpret_cast<uint64_t>(A), static_cast<uint64_t>(s.L),
                           static_cast<uint64_t>(s.Q), static_cast<uint64_t>(lda),
                           reinterpret_cast<uint64_t>(ws), h->seed,
                           static_cast<uint64_t>(h->dist) | (static_cast<uint64_t>(h->k) << 8),
                           1u};
  const int64_t units = pl.pair ? pair_slots() / 2 : num_sms_tc();
  HostSched hs;
  hs.probs.resize(1);
  if (!fill_problem(&hs.probs[0], pl, s, A, lda, static_cast<float*>(ws), h->seed, h->dist))
    return cudaErrorInvalidValue;
  build_items(std::vector<LeftPlan>{pl}, units, &hs);
  pack_sched(&hs);
  if (memcmp(key, hm->sched_key, sizeof(key)) != 0 || hm->d_sched_bytes < hs.bytes) {
    cudaError_t e = grow_device(&hm->d_sched, &hm->d_sched_bytes, hs.bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(hm->d_sched, hs.blob.data(), hs.bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    memcpy(hm->sched_key, key, sizeof(key));
  }
  const LeftSched sc = device_sched(hs, hm->d_sched, h->d_status);
  const int64_t nunits = static_cast<int64_t>(hs.begin.size()) - 1;
  prof_mark(h->prof_start, st);
  const cudaError_t e = pl.pair ? launch_left_dist<true>(h->dist, sc, nunits, st)
                                : launch_left_dist<false>(h->dist, sc, nunits, st);
  prof_mark(h->prof_stop, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  // fixed-order sum of the split partials, times 1/sqrt(k), into Y
  return splitk_reduce(static_cast<float*>(ws), pl.splits, s.P, s.Q, h->scale, Y, ldy, st);
}

struct PlannedBatch {
  HostSched hs;
  std::vector<ReduceDesc> red;
  size_t off_red = 0;
  size_t ws_floats = 0;
  int64_t max_elems = 0;
  int64_t units = 0;
};

LeftPlan member_plan(const BatchMember& mb, int64_t item_stages, GemmShape* shape) {
  if (mb.item_stages > 0) item_stages = mb.item_stages;
  GemmShape s;
  s.left = true;
  s.P = mb.k;
  s.Q = mb.n;
  s.L = mb.m;
  LeftPlan pl = left_geometry(s, true);
  const int64_t steps_total = (s.L + BK - 1) / BK;
  set_splits(&pl, s, (steps_total + item_stages - 1) / item_stages);
  if (shape) *shape = s;
  return pl;
}

// Work list of a batch whose partials start at `ws`; with `ws` null only the
// size of the partials (`ws_floats`) is computed.
bool plan_members(const BatchMember* mbs, size_t count, int64_t item_stages, float* ws,
                  PlannedBatch* pb) {
  std::vector<LeftPlan> plans;
  std::vector<GemmShape> shapes;
  std::vector<size_t> part_off;
  size_t total = 0;
  for (size_t i = 0; i < count; ++i) {
    GemmShape s;
    plans.push_back(member_plan(mbs[i], item_stages, &s));
    shapes.push_back(s);
    // every member's partials start on a 256-byte boundary: the epilogue
    // stores 16-byte vectors when n is a multiple of 4
    part_off.push_back(total);
    if (mbs[i].part == nullptr)
      total += (static_cast<size_t>(plans.back().splits) * s.P * s.Q + 63) / 64 * 64;
  }
  pb->ws_floats = total;
  if (ws == nullptr) return true;  // sizing pass
  pb->hs = HostSched();
  pb->hs.probs.resize(count);
  for (size_t i = 0; i < count; ++i) {
    float* part = mbs[i].part ? mbs[i].part : ws + part_off[i];
    if (!fill_problem(&pb->hs.probs[i], plans[i], shapes[i], mbs[i].A, mbs[i].lda, part,
                      mbs[i].seed, mbs[i].dist))
      return false;
  }
  const int64_t slots = pair_slots();
  if (slots <= 0) return false;
  build_items(plans, slots / 2, &pb->hs);
  pack_sched(&pb->hs);
  pb->units = static_cast<int64_t>(pb->hs.begin.size()) - 1;
  pb->red.clear();
  pb->max_elems = 0;
  for (size_t i = 0; i < count; ++i) {
    ReduceDesc d;
    d.part = mbs[i].part ? mbs[i].part : ws + part_off[i];
    d.Y = mbs[i].Y;
    d.P = mbs[i].k;
    d.Q = mbs[i].n;
    d.ldy = mbs[i].ldy;
    d.splits = plans[i].splits;
    d.scale = mbs[i].scale;
    pb->red.push_back(d);
    pb->max_elems = std::max<int64_t>(pb->max_elems, mbs[i].k * mbs[i].n);
  }
  pb->off_red = (pb->hs.bytes + 255) / 256 * 256;
  return true;
}

// Plan the members twice: once for the size of the partials, once with the
// arena's workspace in place.
cudaError_t plan_into_arena(const BatchMember* mbs, size_t count, int64_t item_stages,
                            BatchArena* ar, PlannedBatch* pb) {
  if (!plan_members(mbs, count, item_stages, nullptr, pb)) return cudaErrorInvalidValue;
  const cudaError_t e = grow_device(&ar->ws, &ar->ws_bytes, pb->ws_floats * sizeof(float) + 256);
  if (e != cudaSuccess) return e;
  if (!plan_members(mbs, count, item_stages, static_cast<float*>(ar->ws), pb))
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

// Copy the work list and the reduce descriptors into the arena; waits for the
// copies so that the host images may change afterwards.
cudaError_t upload_plan(const PlannedBatch& pb, BatchArena* ar, cudaStream_t st) {
  const size_t total = pb.off_red + pb.red.size() * sizeof(ReduceDesc);
  cudaError_t e = grow_device(&ar->d_buf, &ar->d_bytes, total);
  if (e != cudaSuccess) return e;
  if (ar->async_upload) {
    if (ar->h_stage_bytes < total) {
      if (ar->h_stage) cudaFreeHost(ar->h_stage);
      ar->h_stage = nullptr;
      ar->h_stage_bytes = 0;
      const size_t want = std::max<size_t>(total * 2, 1 << 16);
      e = cudaHostAlloc(&ar->h_stage, want, cudaHostAllocDefault);
      if (e != cudaSuccess) return e;
      ar->h_stage_bytes = want;
    }
    uint8_t* h = static_cast<uint8_t*>(ar->h_stage);
    memcpy(h, pb.hs.blob.data(), pb.hs.bytes);
    memcpy(h + pb.off_red, pb.red.data(), pb.red.size() * sizeof(ReduceDesc));
    return cudaMemcpyAsync(ar->d_buf, h, total, cudaMemcpyHostToDevice, st);
  }
  e = cudaMemcpyAsync(ar->d_buf, pb.hs.blob.data(), pb.hs.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(static_cast<uint8_t*>(ar->d_buf) + pb.off_red, pb.red.data(),
                        pb.red.size() * sizeof(ReduceDesc), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

// The persistent sketch launch and the batched reduce of an uploaded plan
// (the caller counts them).
cudaError_t launch_plan(const PlannedBatch& pb, const BatchArena& ar, cudaStream_t st) {
  const LeftSched sc = device_sched(pb.hs, ar.d_buf, ar.d_status);
  const cudaError_t e = launch_left<kMixed, true>(sc, pb.units, st);
  if (e != cudaSuccess) return e;
  return splitk_reduce_batched(
      reinterpret_cast<const ReduceDesc*>(static_cast<uint8_t*>(ar.d_buf) + pb.off_red),
      static_cast<int>(pb.red.size()), pb.max_elems, st);
}

int64_t spread_item_stages(const BatchMember& mb) {
  GemmShape s;
  s.left = true;
  s.P = mb.k;
  s.Q = mb.n;
  s.L = mb.m;
  const LeftPlan pl = left_geometry(s, true);
  const int64_t units = std::max<int64_t>(1, pair_slots() / 2);
  const int64_t tiles = pl.tiles_p * pl.tiles_q;
  const int64_t steps_total = (s.L + BK - 1) / BK;
  int64_t splits = (units + tiles - 1) / tiles;
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, steps_total / 64));
  return (steps_total + splits - 1) / splits;
}

size_t batch_member_workspace(const BatchMember& mb, int64_t item_stages) {
  GemmShape s;
  const LeftPlan pl = member_plan(mb, item_stages, &s);
  return ((static_cast<size_t>(pl.splits) * s.P * s.Q + 63) / 64 * 64) * sizeof(float);
}

cudaError_t batch_launch_members(const BatchMember* mbs, size_t count, int64_t item_stages,
                                 BatchArena* ar, cudaEvent_t ready, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  PlannedBatch pb;
  cudaError_t e = plan_into_arena(mbs, count, item_stages, ar, &pb);
  if (e == cudaSuccess) e = upload_plan(pb, ar, st);
  if (e == cudaSuccess && ready) e = cudaStreamWaitEvent(st, ready, 0);
  if (e == cudaSuccess) e = launch_plan(pb, *ar, st);
  if (e == cudaSuccess) count_launches(1);  // the reduce counted itself
  return e;
}

}  // namespace sk

// ---------------------------------------------------------------------------
// Batches (see include/sketch.h)
// ---------------------------------------------------------------------------
struct sk_batch {
  std::vector<sk::BatchMember> entries;
  int device = 0;
  int64_t item_stages = 0;  // tuned item length (stages); 0 = not chosen
  bool planned = false;
  sk::BatchArena arena;     // work list, reduce descriptors, partials, status
  sk::PlannedBatch plan;
  cudaGraphExec_t graph = nullptr;
};

namespace {

constexpr int64_t kDefaultItemStages = 512;

std::string batch_signature(const sk_batch* b) {
  std::string sig;
  char buf[96];
  for (const auto& e : b->entries) {
    snprintf(buf, sizeof(buf), "%lld:%lld:%lld:%d;", static_cast<long long>(e.m),
             static_cast<long long>(e.n), static_cast<long long>(e.k), e.dist);
    sig += buf;
  }
  uint64_t hsh = 1469598103934665603ull;  // FNV-1a
  for (unsigned char c : sig) hsh = (hsh ^ c) * 1099511628211ull;
  snprintf(buf, sizeof(buf), "%016llx", static_cast<unsigned long long>(hsh));
  return std::string(buf);
}

int64_t cache_lookup(const std::string& sig) {
  const char* path = getenv("SK_TUNE_CACHE");
  if (!path) return 0;
  FILE* f = fopen(path, "r");
  if (!f) return 0;
  char line[256];
  int64_t found = 0;
  while (fgets(line, sizeof(line), f)) {
    char s[64];
    long long v;
    if (sscanf(line, " \"%63[0-9a-f]\" : %lld", s, &v) == 2 && sig == s) found = v;
  }
  fclose(f);
  return found;
}

void cache_store(const std::string& sig, int64_t value) {
  const char* path = getenv("SK_TUNE_CACHE");
  if (!path) return;
  // keep the other entries: read, replace, rewrite as a flat JSON object
  std::vector<std::pair<std::string, long long>> kv;
  if (FILE* f = fopen(path, "r")) {
    char line[256];
    while (fgets(line, sizeof(line), f)) {
      char s[64];
      long long v;
      if (sscanf(line, " \"%63[0-9a-f]\" : %lld", s, &v) == 2 && sig != s) kv.emplace_back(s, v);
    }
    fclose(f);
  }
  kv.emplace_back(sig, static_cast<long long>(value));
  if (FILE* f = fopen(path, "w")) {
    fprintf(f, "{\n");
    for (size_t i = 0; i < kv.size(); ++i)
      fprintf(f, "  \"%s\": %lld%s\n", kv[i].first.c_str(), kv[i].second,
              i + 1 < kv.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
  }
}

void batch_invalidate(sk_batch* b) {
  b->planned = false;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

sk_status to_status(cudaError_t e) { return sk::status_from_cuda(e); }

// Plan every member with items of about `item_stages` stages of 16 rows.
sk_status batch_plan(sk_batch* b, int64_t item_stages, cudaStream_t st) {
  cudaError_t e = sk::plan_into_arena(b->entries.data(), b->entries.size(), item_stages,
                                      &b->arena, &b->plan);
  if (e == cudaErrorInvalidValue) return SK_EINVAL;
  if (e == cudaSuccess) e = sk::upload_plan(b->plan, &b->arena, st);
  if (e != cudaSuccess) return to_status(e);
  b->planned = true;
  return SK_OK;
}

cudaError_t batch_launch(sk_batch* b, cudaStream_t st) {
  return sk::launch_plan(b->plan, b->arena, st);
}

sk_status batch_run_once(sk_batch* b, cudaStream_t st, bool use_graph) {
  // the legacy default stream cannot be captured: launch directly there
  if (!use_graph || st == nullptr) {
    const cudaError_t e = batch_launch(b, st);
    if (e == cudaSuccess) sk::count_launches(1);  // the reduce counted itself
    return to_status(e);
  }
  if (b->graph == nullptr) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return to_status(e);
    const cudaError_t le = batch_launch(b, st);
    e = cudaStreamEndCapture(st, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return to_status(le != cudaSuccess ? le : e);
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return to_status(e);
    }
  }
  const cudaError_t e = cudaGraphLaunch(b->graph, st);
  if (e == cudaSuccess) sk::count_launches(2);  // the sketch and the reduce kernels
  return to_status(e);
}

}  // namespace

extern "C" {

sk_status sk_batch_create(sk_batch_handle* out) {
  if (!out) return SK_EINVAL;
  *out = nullptr;
  sk_batch* b = new (std::nothrow) sk_batch;
  if (!b) return SK_ENOMEM;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&b->arena.d_status), sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(b->arena.d_status, 0, sizeof(int) * 4);
  if (e != cudaSuccess) {
    if (b->arena.d_status) cudaFree(b->arena.d_status);
    delete b;
    return to_status(e);
  }
  *out = b;
  return SK_OK;
}

sk_status sk_batch_add(sk_batch_handle b, sk_handle h, const float* A, int64_t m, int64_t n,
                       int64_t lda, float* Y, int64_t ldy) {
  if (!b || !h || !A || !Y || m <= 0 || n <= 0 || lda < n || ldy < n) return SK_EINVAL;
  if (m >= (1LL << 31) - 64) return SK_EINVAL;
  if (h->prec != SK_BF16X2) return SK_EUNSUPPORTED;
  sk::GemmShape s;
  s.left = true;
  s.P = h->k;
  s.Q = n;
  s.L = m;
  const sk_status st = sk::tc_check(s, A, lda, Y, ldy);
  if (st != SK_OK) return st;
  sk::BatchMember e{h->seed, h->dist, h->k, h->scale, A, m, n, lda, Y, ldy, nullptr, 0};
  b->entries.push_back(e);
  batch_invalidate(b);
  return SK_OK;
}

sk_status sk_batch_run(sk_batch_handle b, void* stream) {
  if (!b || b->entries.empty()) return SK_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!b->planned) {
    int64_t t = b->item_stages;
    if (t <= 0) t = cache_lookup(batch_signature(b));
    if (t <= 0) t = kDefaultItemStages;
    const sk_status ps = batch_plan(b, t, st);
    if (ps != SK_OK) return ps;
  }
  return batch_run_once(b, st, true);
}

sk_status sk_batch_tune(sk_batch_handle b, void* stream, int64_t* chosen) {
  if (!b || b->entries.empty()) return SK_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t cands[] = {128, 256, 512, 1024, 2048, 4096};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return to_status(cudaGetLastError());
  float best_ms = 1e30f;
  int64_t best = kDefaultItemStages;
  sk_status rs = SK_OK;
  for (int64_t t : cands) {
    batch_invalidate(b);
    rs = batch_plan(b, t, st);
    if (rs != SK_OK) break;
    rs = batch_run_once(b, st, false);  // warm-up
    if (rs != SK_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && rs == SK_OK; ++r) rs = batch_run_once(b, st, false);
    cudaEventRecord(e1, st);
    if (rs != SK_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_invalidate(b);
  if (rs != SK_OK) return rs;
  b->item_stages = best;
  cache_store(batch_signature(b), best);
  if (chosen) *chosen = best;
  return SK_OK;
}

sk_status sk_batch_status(sk_batch_handle b, void* stream) {
  if (!b) return SK_EINVAL;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  int word = 0;
  if (e == cudaSuccess)
    e = cudaMemcpy(&word, b->arena.d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word != 0) e = cudaMemset(b->arena.d_status, 0, sizeof(int) * 4);
  if (e != cudaSuccess) return to_status(e);
  return static_cast<sk_status>(word);
}

sk_status sk_batch_size(sk_batch_handle b, int64_t* count) {
  if (!b || !count) return SK_EINVAL;
  *count = static_cast<int64_t>(b->entries.size());
  return SK_OK;
}

sk_status sk_batch_destroy(sk_batch_handle b) {
  if (!b) return SK_EINVAL;
  batch_invalidate(b);
  if (b->arena.d_buf) cudaFree(b->arena.d_buf);
  if (b->arena.ws) cudaFree(b->arena.ws);
  if (b->arena.d_status) cudaFree(b->arena.d_status);
  delete b;
  return SK_OK;
}

}  // extern "C"

// sk_tc.cu -- BF16 split-A tensor-core form of the fused generate-and-sketch
// on Blackwell (tcgen05 + TMEM + TMA, CTA pairs), left sketch
// Y[k x n] = S[k x m] A[m x n].
//
// This is the local multiply of the paper's Alg. 1 (GenRandom, then
// B = A Omega on the local block) with the random operand regenerated inside
// the kernel instead of read (Sec. 6.2's "generate rather than communicate",
// with shared memory in the role of the processor's local memory).
//
// Two passes.  The split pass (k_split_bf16x2, HBM-bound) writes
// hi = bf16(a) and lo = bf16(a - hi) of A once, row-major with rows padded to
// 64 columns; every 256-row tile of Y then reads the BF16 halves instead of
// converting the FP32 tile again (with k = 2048 the fused conversion was
// repeated by 8 tiles and cost more than the split pass).  The sketch kernel
// keeps S in shared memory only:
//
// A pair owns a 256 x NT tile of Y (NT <= 512 TMEM columns in each CTA) and
// one contiguous range of the contracted dimension m (deterministic split-K):
//   warp 0       TMA producer: one 4D box per stage brings this CTA's
//                columns of the hi and lo tiles [32 rows of m] into the
//                operand ring, MN-major with the 128-byte swizzle;
//   warp 1       TMEM allocation (collective over the pair); in the even CTA
//                the MMA issuer: per stage 2 K steps x 2 passes (hi, lo) x
//                NT/256 tcgen05.mma kind::f16 (M=256, K=16) into the FP32
//                accumulator, completion signalled to both CTAs;
//   warps 2-9    epilogue: at the end of every accumulation chain (2048
//                rows of m; 4096 for Rademacher S) the accumulator is read
//                out of this CTA's TMEM and added into its FP32 partial in
//                global memory (store for the first chain, red.add after);
//   warps 10-25  workers, in 4 groups that take turns on successive stages:
//                generate this CTA's BF16 S tile [128 x 32] (Philox4x32-10 +
//                Box-Muller, or sign bits) in the K-major no-swizzle layout,
//                then pass the stage on to the MMA issuer once this CTA's
//                hi / lo tile has landed.
// With k <= 128 a single CTA (cta_group::1, M = 128) does the same alone.
// The tensor core accumulates in FP32 without round-to-nearest on every
// add, so its error grows with the chain length; restarting the TMEM chain
// at a fixed length and summing chains with IEEE adds keeps Y within 1e-5
// of the exact product at any m.  S never exists outside shared memory
// (except in the stored-S mode, which reads a caller's S by TMA to measure
// the generate-versus-read trade).
// Every wait is bounded: on timeout the kernel records SK_ETIMEOUT and the
// waiting site in the handle's status words, drains its own copies and MMAs
// (again bounded) and frees TMEM; both CTAs reach the closing cluster barrier.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
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
constexpr int BK = 16;        // MMA K; contracted length per stage of the right kernel
constexpr int LK = 32;        // contracted length per stage of the left kernel
constexpr int KSTEPS = LK / BK;  // MMA K steps per left stage
constexpr int NT_MAX = 512;   // output columns per tile (TMEM columns)
constexpr int CHAIN = 128;    // MMA K steps per TMEM accumulation chain (2048 rows)
constexpr int CHAIN_L = CHAIN / KSTEPS;  // left stages per chain
constexpr int HCHUNK = 64;    // columns of one 128-byte swizzle atom of the split A
constexpr int NUM_EPI_WARPS = 8;
constexpr int NUM_WORK_WARPS = 16;
constexpr int IQ = 4;  // slots of the left kernel's work-item queue in shared memory

constexpr int WARP_TMA = 0;
constexpr int WARP_MMA = 1;
constexpr int WARP_EPI0 = 2;
constexpr int WARP_WORK0 = WARP_EPI0 + NUM_EPI_WARPS;
constexpr int NTHREADS = 32 * (WARP_WORK0 + NUM_WORK_WARPS);  // 832

// Epilogue transpose tile of one warp: 32 accumulator rows x 16 columns,
// rows padded to 20 floats (16-byte aligned, few bank conflicts).
constexpr int EPI_PITCH = 20;
constexpr uint32_t EPI_TILE = 32 * EPI_PITCH * 4;
// Staging tile of a TMA drain: 32 accumulator rows x 32 columns (128 B per
// row, the 128-byte swizzle of the partial's tensor map).
constexpr uint32_t DRAIN_TILE = 32 * 32 * 4;

// Per-CTA buffers of the left kernel.  A CTA of a pair holds NT/2 columns of
// each split A tile.  NARROW (pairs only, batches whose tiles all have at most
// 256 columns): half-width split A slots, so the operand ring is 8 stages
// deep instead of 4.  TDRAIN (all but NARROW): each epilogue warp has two
// 4 KB staging tiles from which the TMA adds a drained accumulator chain into
// the partial (see drain_chain_tma); a narrow ring has no room for them.
template <bool PAIR, bool NARROW = false>
struct Cfg {
  static_assert(PAIR || !NARROW, "narrow rings are a pair configuration");
  static constexpr int COLS = NARROW ? NT_MAX / 4 : PAIR ? NT_MAX / 2 : NT_MAX;  // most A columns per CTA
  // Worker groups take turns on successive stages.  A group that starts
  // stage s has finished stage s - NGROUPS, so waits never run more than one
  // barrier phase ahead (the parity test would alias) as long as
  // NGROUPS <= NSO.
  static constexpr int NGROUPS = PAIR ? 4 : 2;
  static constexpr int GROUP_WARPS = NUM_WORK_WARPS / NGROUPS;
  static constexpr int GROUP_THREADS = 32 * GROUP_WARPS;
  static constexpr int NSO = NARROW ? 8 : PAIR ? 4 : 2;     // operand stages
  static constexpr bool TDRAIN = !NARROW;
  static constexpr uint32_t OPB = 2u * COLS * LK * 2u;      // hi and lo tiles of a stage
  static constexpr uint32_t OPS = BM * LK * 2;              // S tile: KSTEPS slabs of 16
  static constexpr uint32_t OFF_B = 0;
  static constexpr uint32_t OFF_S = OFF_B + NSO * OPB;
  static constexpr uint32_t OFF_EPI = OFF_S + NSO * OPS;    // epilogue tiles, per warp:
  static constexpr uint32_t EPI_BYTES = TDRAIN ? 2 * DRAIN_TILE : EPI_TILE;
  static constexpr uint32_t OFF_BAR = OFF_EPI + NUM_EPI_WARPS * EPI_BYTES;
  static constexpr uint32_t NUM_BARS = 3 * NSO + 3 + 2 * IQ;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NUM_BARS * 8;  // abort flag, TMEM slot, item queue
  static constexpr uint32_t SMEM = OFF_MISC + 16 + 4 * IQ + 1024;  // + slack for 1 KB alignment
  // roles that read each queued item: in every CTA the epilogue and worker
  // warps, plus the MMA issuer (even CTA) or the TMA producer (odd CTA); the
  // even CTA's TMA producer fills the queue
  static constexpr int IQ_READERS = (PAIR ? 2 : 1) * (1 + NUM_EPI_WARPS + NUM_WORK_WARPS);
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
  static_assert(NGROUPS <= NSO, "worker groups vs ring depth");
  static_assert(OPB % 1024 == 0, "split tiles start on swizzle-atom boundaries");
  static_assert(!TDRAIN || OFF_EPI % 1024 == 0, "staging tiles on swizzle-atom boundaries");
  static_assert(EPI_BYTES >= EPI_TILE, "the transpose tile fits the warp's area");
};

// K-major no-swizzle operand layout (16-element K slab): core matrix
// (8 rows x 16 B) at (row/8)*256 + khalf*128, row r%8 at +16*(r%8).
__device__ __forceinline__ uint32_t kmaj_off(uint32_t row, uint32_t khalf) {
  return (row & 7u) * 16u + (row >> 3) * 256u + khalf * 128u;
}
constexpr uint32_t LBO = 128;  // K-adjacent core matrices
constexpr uint32_t SBO = 256;  // 8-row groups
// The S tile of a stage: KSTEPS K-major slabs [128 rows][16] of 4 KB.
constexpr uint32_t S_SLAB = BM * BK * 2;
// MN-major 128-byte-swizzled split A tile as the TMA box lays it out:
// [hi/lo][64-column chunk][32 rows][64 columns]; atoms of 8 rows x 128 B
// (next 64 columns: HCHUNK_BYTES, or 2 HCHUNK_BYTES when the tile is split in
// place as [chunk][hi/lo], see convert_stage).
constexpr uint32_t HCHUNK_BYTES = LK * HCHUNK * 2;  // 4096: one chunk of one stage
constexpr uint32_t B_SBO = 8 * HCHUNK * 2;          // 1024: next 8 rows of m
constexpr uint32_t B_KSTEP = BK * HCHUNK * 2;       // 2048: next 16 rows of m

// One left-sketch problem of a launch (a single sketch, or one member of a
// batch).  Lives in device memory; the tensor map must be 64-byte aligned.
struct alignas(128) LeftProblem {
  CUtensorMap map;   // split A: {64 columns, m rows, chunks, hi/lo}, box {64, 32, cols/64, 2}
  CUtensorMap smap;  // stored S (kStored only): the S tile of a stage in its operand layout
  float* part;      // partials [splits][P][ldp] of this problem (columns Q .. ldp-1 unused)
  int64_t P, Q, L;  // P = k, Q = n, L = m
  int64_t ldp;      // partial row stride, >= Q
  int64_t chunk;    // contracted length per split (multiple of LK)
  int nt;           // output columns per tile: a multiple of 128 (pairs) or 64 up to 256, or 512
  int dist;         // sk_dist of S
  int chain;        // stages per TMEM accumulation chain (a power of two, multiple of 8)
  PhiloxKey key;
  // conv_inline: the TMA brings FP32 A as 32-column blocks of 32 rows with the
  // 128-byte swizzle (`amap`: one 3D box of all the CTA's blocks when n is a
  // multiple of 32 (1), else one 2D box per block (2)) and the workers split
  // it into the BF16 halves in
  // place (single sketches on pairs and the Rademacher members of batches;
  // see convert_stage); 0: the split pass wrote the halves and `map` loads
  // them
  int conv_inline;
  CUtensorMap amap;
  // tma_drain: the partials as a 3D FP32 tensor {Q, P, splits} (row stride
  // ldp) with boxes of 32 columns x 32 rows and the 128-byte swizzle
  // (`pmap`); the epilogue drains through the TMA (needs ldp % 4 == 0 and part
  // 16-byte aligned)
  int tma_drain;
  CUtensorMap pmap;
};

// A unit of work: tile (tp, tq) of split z of problem `prob`.  With pairs,
// tp indexes 256-row tiles and the CTA of rank r takes rows 128 r .. of it.
struct LeftItem {
  int prob, tp, tq, z;
};

// Work list: every item of the launch, longest first.  Pairs (or single
// CTAs) take the next unclaimed item from the device counter `claim` (zero
// at launch) until the list is exhausted.
struct LeftSched {
  const LeftProblem* probs;
  const LeftItem* items;
  int* claim;
  int nitems;
  int* status;
  uint64_t timeout_ns;
  // failure-injection hook of the tests, -1 otherwise: the TMA producer
  // issues no copy for this stage (counted over each CTA's or pair's run),
  // so the waits that depend on it give up after timeout_ns
  long long stall_stage;
  PhiloxRoundKeys rk;  // round keys of problem 0 (read when a launch has one distribution)
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

// ---- split pass: A (FP32) -> hi / lo (BF16), rows padded to 64 columns ----

// One matrix of the split pass.  hi row r at H + r*ldh, lo row r at
// H + part + r*ldh; columns n .. ldh-1 are written as zeros.
struct SplitDesc {
  const float* A;
  int64_t lda;
  __nv_bfloat16* H;
  int64_t ldh, part;
  int64_t m, n;
};

// Store hi / lo of the values a[0..7] of columns c .. c+7 of row r.
__device__ __forceinline__ void split_store(const SplitDesc& d, int64_t r, int64_t c,
                                            const float (&a)[8]) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    hw[e] = pack_bf16x2(a[2 * e], a[2 * e + 1]);
    const float h0 = __uint_as_float(hw[e] << 16);
    const float h1 = __uint_as_float(hw[e] & 0xffff0000u);
    lw[e] = pack_bf16x2(__fsub_rn(a[2 * e], h0), __fsub_rn(a[2 * e + 1], h1));
  }
  __nv_bfloat16* dst = d.H + r * d.ldh + c;
  *reinterpret_cast<uint4*>(dst) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(dst + d.part) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// Columns c .. c+7 of row r (c a multiple of 8; rows 16-byte aligned).
__device__ __forceinline__ void split_group(const SplitDesc& d, int64_t r, int64_t c) {
  float a[8];
  const float* src = d.A + r * d.lda + c;
  if (c + 8 <= d.n) {
    const float4 v0 = __ldcs(reinterpret_cast<const float4*>(src));
    const float4 v1 = __ldcs(reinterpret_cast<const float4*>(src + 4));
    a[0] = v0.x; a[1] = v0.y; a[2] = v0.z; a[3] = v0.w;
    a[4] = v1.x; a[5] = v1.y; a[6] = v1.z; a[7] = v1.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) a[e] = c + e < d.n ? __ldcs(src + e) : 0.0f;
  }
  split_store(d, r, c, a);
}

// One warp per row with 4-byte loads: rows of any alignment (the serving
// path reads requests straight from their sources).
__global__ void __launch_bounds__(256) k_split_rows(const SplitDesc d) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * 8;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); r < d.m;
       r += warps) {
    const float* src = d.A + r * d.lda;
    for (int64_t c = 8 * lane; c < d.ldh; c += 256) {
      float a[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) a[e] = c + e < d.n ? src[c + e] : 0.0f;
      split_store(d, r, c, a);
    }
  }
}

__global__ void __launch_bounds__(256) k_split_bf16x2_one(const SplitDesc d) {
  const int64_t gpr = d.ldh / 8;
  const int64_t total = d.m * gpr;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    split_group(d, t / gpr, (t % gpr) * 8);
}

// Many matrices in one launch: prefix[i] = groups of 8 columns before
// matrix i (prefix[count] = total).
__global__ void __launch_bounds__(256)
    k_split_bf16x2_many(const SplitDesc* ds, const int64_t* prefix, int count) {
  const int64_t total = prefix[count];
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last i with prefix[i] <= t
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const SplitDesc d = ds[lo];
    const int64_t u = t - prefix[lo];
    const int64_t gpr = d.ldh / 8;
    split_group(d, u / gpr, (u % gpr) * 8);
  }
}

// Per-item geometry shared by every role.
struct ItemGeo {
  const LeftProblem* pr;
  int64_t P;      // rows of S (copied: the workers' loop keeps it in a register)
  PhiloxKey key;  // (likewise)
  int64_t p0, q0, lbeg, lend;
  int nsteps, nt, nmma, nh, bh, cols, dist;
  int chain;  // stages per accumulation chain
  int coff;   // stages by which this item's chain boundaries are shifted
};

template <bool PAIR>
__device__ __forceinline__ ItemGeo item_geo(const LeftSched& sc, int idx, uint32_t rank) {
  const LeftItem it = sc.items[idx];
  ItemGeo g;
  g.pr = sc.probs + it.prob;
  g.P = g.pr->P;
  g.key = g.pr->key;
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
  g.nsteps = static_cast<int>((g.lend - g.lbeg + LK - 1) / LK);
  // Items of one problem shift their chain boundaries by different amounts so
  // that the accumulator drains of concurrent pairs do not all reach L2 at
  // once; the shift is a function of the item alone, so the summation order
  // of a problem does not depend on what runs beside it.
  g.chain = g.pr->chain;
  g.coff = ((it.tp * 7 + it.z * 13 + it.tq * 5) & 7) * (g.chain / 8);
  return g;
}

// Split this CTA's FP32 A tile of a stage in place into its BF16 halves
// (hi = bf16(a), lo = bf16(a - hi), as the split pass does).  The TMA leaves
// the tile as 32-column blocks [block][32 rows][32 floats] with the 128-byte
// swizzle (16-byte unit u of row r stored at unit u ^ (r mod 8)); 64-column
// chunk c (blocks 2c and 2c+1, 8 KB) becomes hi chunk c (4 KB) followed by lo
// chunk c (4 KB), each [32 rows][64 BF16] with the 128-byte swizzle: the
// MN-major operand layout the MMA reads, chunk after chunk.  Warp w of the
// worker group converts rows 8w .. 8w+7 (4 lanes per row, 16 columns each):
// the bytes those rows occupy in blocks 2c and 2c+1 are exactly the bytes
// they occupy in hi and lo chunk c, so each warp reads its values of a chunk,
// synchronises itself, and writes them back, with no other warp involved.
// Lane l takes row 8w + (l mod 8) and column quarter l / 8: the 8 lanes of
// each 128-byte phase of a 16-byte access then read (and write) one unit of
// each of 8 rows, and the swizzle puts those 8 units in 8 different bank
// groups, so no access of the conversion has a bank conflict.
// wt is the thread's index in a set of 4 warps (128 threads, 4 threads per
// row of the 32-row stage); the set converts chunks c0, c0 + cstep, ...
__device__ __forceinline__ void convert_stage(uint8_t* slot, int cols, int wt, int c0 = 0,
                                              int cstep = 1) {
  const uint32_t r = (static_cast<uint32_t>(wt) >> 5) * 8u + (static_cast<uint32_t>(wt) & 7u);
  const uint32_t j = (static_cast<uint32_t>(wt) >> 3) & 3u;  // 16-column quarter of the chunk
  const uint32_t sw = r & 7u;
  const uint32_t u0 = ((2u * j) ^ sw) * 16u, u1 = ((2u * j + 1u) ^ sw) * 16u;
  for (int c = c0; c < cols / HCHUNK; c += cstep) {
    uint8_t* ch = slot + c * (2 * HCHUNK_BYTES);
    const uint8_t* src = ch + (j >> 1) * HCHUNK_BYTES + r * 128u;
    float a[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t u = (((j & 1u) * 4u + static_cast<uint32_t>(i)) ^ sw) * 16u;
      const float4 v = *reinterpret_cast<const float4*>(src + u);
      a[4 * i] = v.x; a[4 * i + 1] = v.y; a[4 * i + 2] = v.z; a[4 * i + 3] = v.w;
    }
    __syncwarp();  // this warp's rows of the chunk have been read
    uint32_t hw[8], lw[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      hw[e] = pack_bf16x2(a[2 * e], a[2 * e + 1]);
      const float2 hv = f2(__uint_as_float(hw[e] << 16), __uint_as_float(hw[e] & 0xffff0000u));
      // a - hi of both elements in one packed FMA (the product by -1 is exact)
      const float2 lv = __ffma2_rn(hv, f2(-1.0f, -1.0f), f2(a[2 * e], a[2 * e + 1]));
      lw[e] = pack_bf16x2(lv.x, lv.y);
    }
    uint8_t* hrow = ch + r * 128u;
    *reinterpret_cast<uint4*>(hrow + u0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(hrow + u1) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
    *reinterpret_cast<uint4*>(hrow + HCHUNK_BYTES + u0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    *reinterpret_cast<uint4*>(hrow + HCHUNK_BYTES + u1) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
  }
}

// Generate this CTA's BF16 S tile [128 x 32] of one stage (two K-major slabs
// of 16 columns).  A Rademacher task is one row of the stage: one 32-bit
// Philox word, kept across the four stages one call covers.  Gaussian and
// uniform tasks are four entries of one row (one Philox call); a thread owns
// quad qd of rows rbase + RSTEP i of both slabs, so its tile offsets and
// Philox counters step by constants.  K is PhiloxKey, or the precomputed
// PhiloxRoundKeys of a launch parameter.
template <int DIST, class C, class K>
__device__ __forceinline__ void gen_stage(uint8_t* sdst, const ItemGeo& g, const K& key,
                                          int64_t cbase, int wt, uint32_t* cached_blk,
                                          uint4* words) {
  if (DIST == kRademacher) {
    constexpr int RAD_IT = (BM + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
#pragma unroll
    for (int it = 0; it < RAD_IT; ++it) {
      const int t = wt + it * C::GROUP_THREADS;
      if (t >= BM) break;
      const uint32_t r = static_cast<uint32_t>(t);
      const int64_t grow = g.p0 + r;
      uint32_t bits = 0u, valid = 0u;
      if (grow < g.P && cbase < g.lend) {
        const uint32_t c = static_cast<uint32_t>(cbase);  // a multiple of 32
        const uint32_t blk = c >> 7;
        if (blk != cached_blk[it]) {
          words[it] = rademacher_bits(key, static_cast<uint32_t>(grow), blk, 0u);
          cached_blk[it] = blk;
        }
        const uint32_t wsel = (c >> 5) & 3u;
        const uint4 wv = words[it];
        bits = wsel == 0 ? wv.x : wsel == 1 ? wv.y : wsel == 2 ? wv.z : wv.w;
        const int64_t nv = g.lend - cbase;
        valid = nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // 8 columns each: slab j / 2, half j % 2
        const uint32_t b = bits >> (8 * j);
        const uint32_t vm = valid >> (8 * j);
        uint4 v;
        // +1.0 = 0x3F80, -1.0 = 0xBF80: the sign bit carries the random bit
        v.x = 0x3F803F80u | ((b & 1u) << 15) | ((b & 2u) << 30);
        v.y = 0x3F803F80u | ((b & 4u) << 13) | ((b & 8u) << 28);
        v.z = 0x3F803F80u | ((b & 16u) << 11) | ((b & 32u) << 26);
        v.w = 0x3F803F80u | ((b & 64u) << 9) | ((b & 128u) << 24);
        if ((vm & 0xffu) != 0xffu) {  // columns past the end of the split are zero
          v.x &= ((vm & 1u) ? 0x0000ffffu : 0u) | ((vm & 2u) ? 0xffff0000u : 0u);
          v.y &= ((vm & 4u) ? 0x0000ffffu : 0u) | ((vm & 8u) ? 0xffff0000u : 0u);
          v.z &= ((vm & 16u) ? 0x0000ffffu : 0u) | ((vm & 32u) ? 0xffff0000u : 0u);
          v.w &= ((vm & 64u) ? 0x0000ffffu : 0u) | ((vm & 128u) ? 0xffff0000u : 0u);
        }
        *reinterpret_cast<uint4*>(sdst + (j >> 1) * S_SLAB +
                                  kmaj_off(r, static_cast<uint32_t>(j & 1))) = v;
      }
    }
  } else {
    // A warp covers 8 rows x 4 quads; the group covers RSTEP rows per pass.
    // Lane l takes row l mod 8 and quad l / 8: the 16 lanes of each 128-byte
    // phase of an 8-byte store then write both 8-byte halves of one 16-byte
    // unit of each of 8 rows, every bank once.
    constexpr int RSTEP = C::GROUP_THREADS / 4;
    constexpr int NPASS = BM / RSTEP;
    static_assert(RSTEP % 8 == 0 && BM % RSTEP == 0, "row passes of the worker group");
    const uint32_t qd = (static_cast<uint32_t>(wt) >> 3) & 3u;
    const uint32_t rbase = static_cast<uint32_t>(wt >> 5) * 8u + (static_cast<uint32_t>(wt) & 7u);
    // kmaj_off(rbase + RSTEP i, qd / 2) = off0 + 32 RSTEP i (RSTEP is a multiple of 8)
    const uint32_t off0 = kmaj_off(rbase, qd >> 1) + (qd & 1u) * 8u;
    const bool full = cbase + LK <= g.lend;
    const uint32_t j0 = static_cast<uint32_t>(cbase >> 2) + qd;  // Philox block, slab 0
    const int64_t row0 = g.p0 + rbase;
    // two tasks in flight per thread: full unrolling of the 8 Philox +
    // Box-Muller tasks made the loop too large for the instruction cache
    // (11 % slower on the Gaussian sketch)
#pragma unroll 1
    for (int i = 0; i < NPASS; ++i) {
      const int64_t grow = row0 + static_cast<int64_t>(RSTEP) * i;
      const bool rv = grow < g.P;
#pragma unroll
      for (int slab = 0; slab < KSTEPS; ++slab) {
        uint2 v = make_uint2(0u, 0u);
        if (rv && (full || cbase + 16 * slab + 4 * qd < g.lend)) {
          const uint32_t j = j0 + 4u * static_cast<uint32_t>(slab);
          const float4 a = DIST == kUniform ? uniform4(key, static_cast<uint32_t>(grow), j, 0u)
                                            : gaussian4(key, static_cast<uint32_t>(grow), j, 0u);
          v = make_uint2(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w));
        }
        *reinterpret_cast<uint2*>(sdst + slab * S_SLAB + off0 +
                                  static_cast<uint32_t>(i * RSTEP * 32)) = v;
      }
    }
  }
}

// One accumulator drain by an epilogue warp of the left kernel through the
// TMA: wait until chain gc has finished, and for each of the warp's 32-column
// chunks of its TMEM lane quarter, read the chunk (lane = row), write it into
// one of the warp's two staging tiles (row r at 128 r, its 16-byte unit u at
// u ^ (r mod 8): the 128-byte swizzle, and no bank conflict as the 8 lanes of
// a phase write 8 different units), and let lane 0 hand the tile to the TMA,
// which stores it into the item's partial (first chain) or adds it there
// element by element; boxes reaching past P rows or Q columns are clipped.
// The accumulator is released as soon as its last chunk is read: the global
// writes no longer hold up the next chain.  The adds of one address stay in
// chain order, hence deterministic: lane 0 waits until its previous chain's
// copies have completed before issuing this chain's, and a staging tile is
// rewritten only after the copy two chunks back has read it.
template <bool PAIR>
__device__ __noinline__ bool drain_chain_tma(uint32_t tmem, int quarter, int colset,
                                             uint32_t stage_u32, float* stage, const ItemGeo ig,
                                             int z, bool first, uint32_t acc_full,
                                             uint32_t lead_acc_empty, int gc, const Abort ab) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) bulk_wait<0>();
  const bool ok = mbar_wait(acc_full, gc & 1, ab, 0x34, gc);
  if (!__all_sync(0xffffffffu, ok)) return false;  // tcgen05.ld below is warp-collective
  tc_fence_after();
  const int32_t y = static_cast<int32_t>(ig.p0 + quarter * 32);
  const uint32_t sw = static_cast<uint32_t>(lane) & 7u;
  int nb = 0;
  for (int ci = colset; ci * 32 < (ig.nmma - 1) * 256 + ig.nh; ci += 2, ++nb) {
    uint32_t v[32];
    tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(ci * 32),
              v);
    tmem_ld_wait();
    // TMEM column h*256 + c holds B row c of instruction h (pair: rows c < bh
    // the even CTA's tile columns h*bh + c, the others the odd CTA's
    // cols + h*bh + (c - bh)); bh is a multiple of 64, so a chunk of 32 is
    // contiguous in the tile
    const int h = (ci * 32) >> 8;
    const int c = (ci * 32) & 255;
    const int tn =
        PAIR ? (c < ig.bh ? h * ig.bh + c : ig.cols + h * ig.bh + (c - ig.bh)) : ci * 32;
    const uint32_t b = static_cast<uint32_t>(nb & 1);
    if (nb >= 2) {
      if (lane == 0) bulk_wait_read<1>();
      __syncwarp();
    }
    float* row = stage + b * (DRAIN_TILE / 4) + lane * 32;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(row + ((static_cast<uint32_t>(q) ^ sw) << 2)) =
          make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                      __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
    fence_proxy_async_smem();  // the tile is read by the TMA
    __syncwarp();
    if (lane == 0) {
      const int32_t x = static_cast<int32_t>(ig.q0 + tn);
      const uint32_t src = stage_u32 + b * DRAIN_TILE;
      if (first)
        tma_store_3d(&ig.pr->pmap, src, x, y, z);
      else
        tma_reduce_add_3d(&ig.pr->pmap, src, x, y, z);
      bulk_commit();
    }
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) {
    if (PAIR)
      mbar_arrive_cluster(lead_acc_empty);
    else
      mbar_arrive(lead_acc_empty);
  }
  return true;
}

// One accumulator drain by an epilogue warp of the left kernel (the steps of
// the kernel's own epilogue loop): wait until chain gc has finished, read the
// warp's TMEM lane quarter x its 32-column chunks, write them through the
// transpose tile into the item's partial (first chain: store; later: add),
// and release the accumulator.  Out of line for the epilogue warps that also
// split A (EC), so that their stage loop does not hold the drain's registers.
template <bool PAIR>
__device__ __noinline__ bool drain_chain_left(uint32_t tmem, int quarter, int colset, float* tile,
                                              const ItemGeo ig, float* part_item, bool first,
                                              uint32_t acc_full, uint32_t lead_acc_empty, int gc,
                                              const Abort ab) {
  const int lane = threadIdx.x & 31;
  const int rsub = lane >> 2;       // row within a group of 8 (read side)
  const int csub = (lane & 3) * 4;  // first of 4 columns (read side)
  const int64_t P = ig.pr->P, Q = ig.pr->Q, ldp = ig.pr->ldp;
  const bool vec_ok = (ldp % 4) == 0;
  const bool ok = mbar_wait(acc_full, gc & 1, ab, 0x34, gc);
  if (!__all_sync(0xffffffffu, ok)) return false;  // tcgen05.ld below is warp-collective
  tc_fence_after();
  for (int ci = colset; ci * 32 < (ig.nmma - 1) * 256 + ig.nh; ci += 2) {
    uint32_t v[32];
    tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(ci * 32),
              v);
    tmem_ld_wait();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(tile + lane * EPI_PITCH + 4 * q) =
            make_float4(__uint_as_float(v[16 * half + 4 * q]),
                        __uint_as_float(v[16 * half + 4 * q + 1]),
                        __uint_as_float(v[16 * half + 4 * q + 2]),
                        __uint_as_float(v[16 * half + 4 * q + 3]));
      __syncwarp();
      const int tcol = ci * 32 + 16 * half + csub;
      const int h = tcol >> 8;
      const int c = tcol & 255;
      const int tn =
          PAIR ? (c < ig.bh ? h * ig.bh + c : ig.cols + h * ig.bh + (c - ig.bh)) : tcol;
      const int64_t col = ig.q0 + tn;
#pragma unroll
      for (int pass = 0; pass < 4; ++pass) {
        const int rr = 8 * pass + rsub;
        const int64_t gp = ig.p0 + quarter * 32 + rr;
        const float4 a = *reinterpret_cast<const float4*>(tile + rr * EPI_PITCH + csub);
        if (c < ig.nh && gp < P) {
          float* d = part_item + gp * ldp + tn;
          if (vec_ok && col + 4 <= Q) {
            if (first)
              *reinterpret_cast<float4*>(d) = a;
            else
              red_add_v4(d, a.x, a.y, a.z, a.w);
          } else {
            const float vv[4] = {a.x, a.y, a.z, a.w};
            for (int u = 0; u < 4; ++u) {
              if (col + u < Q) {
                if (first)
                  d[u] = vv[u];
                else
                  red_add(d + u, vv[u]);
              }
            }
          }
        }
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) {
    if (PAIR)
      mbar_arrive_cluster(lead_acc_empty);
    else
      mbar_arrive(lead_acc_empty);
  }
  return true;
}

// Persistent left-sketch kernel: each pair (or single CTA) runs its list of
// items back to back; ring positions, barrier phases and accumulation chains
// are counted across items (g = stage counter, gc = chain counter).  DIST is
// the distribution of every item, kMixed to read it per item (batches), or
// kStored to read a caller-materialized BF16 S by TMA instead of generating
// it (the "communicate Omega" side of the paper's Sec. 6.2 trade, for
// measurement).
constexpr int kMixed = -1;
constexpr int kStored = 3;

template <int DIST, bool PAIR, bool NARROW = false, bool ECONV = false>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_sketch_bf16x2_left(const LeftSched sc) {
  using C = Cfg<PAIR, NARROW>;
  // EC (pairs): the epilogue warps certify every stage's A tile to the MMA
  // issuer, and split in place the FP32 tiles of Gaussian and uniform items
  // (their workers are busy generating; the epilogue warps are idle between
  // accumulator drains), so no split pass runs before those items
  constexpr bool EC = ECONV && PAIR;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + C::OFF_BAR;
  // full_b: this CTA's split A tile has landed; full_o (even CTA): both CTAs'
  // operands of the stage are ready; empty_o: the MMAs that read the slot
  // have completed (signalled to both CTAs)
  auto full_b = [&](int i) { return bar0 + 8u * i; };
  auto full_o = [&](int i) { return bar0 + 8u * (C::NSO + i); };
  auto empty_o = [&](int i) { return bar0 + 8u * (2 * C::NSO + i); };
  const uint32_t acc_full = bar0 + 8u * (3 * C::NSO);
  const uint32_t acc_empty = acc_full + 8u;
  const uint32_t drain_bar = acc_full + 16u;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::OFF_MISC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? (cluster_ctarank() & 1u) : 0u;  // 0 = even (MMA issuer)
  const bool leader = rank == 0;
  // item queue: slot i holds the index of the item every role of the pair
  // (or single CTA) works on next; iq_full / iq_empty: written / read by all
  int* iq = reinterpret_cast<int*>(smem + C::OFF_MISC + 16);
  auto iq_full = [&](int i) { return bar0 + 8u * (3 * C::NSO + 3 + i); };
  auto iq_empty = [&](int i) { return bar0 + 8u * (3 * C::NSO + 3 + IQ + i); };

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NSO; ++i) {
      mbar_init(full_b(i), 1);
      // one worker group of each CTA (plus, with EC, the epilogue warps of each)
      mbar_init(full_o(i), (C::GROUP_WARPS + (EC ? NUM_EPI_WARPS : 0)) * (PAIR ? 2 : 1));
      mbar_init(empty_o(i), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NUM_EPI_WARPS * (PAIR ? 2 : 1));  // epilogues of both CTAs
    mbar_init(drain_bar, 1);
    for (int i = 0; i < IQ; ++i) {
      mbar_init(iq_full(i), 1);
      mbar_init(iq_empty(i), C::IQ_READERS);
    }
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

  // The even CTA's TMA producer claims item j of this pair and publishes it in
  // both CTAs' queue slot (-1 once the list is exhausted).
  auto produce_item = [&](int j) -> int {
    const int slot = j % IQ;
    if (j >= IQ && !mbar_wait(iq_empty(slot), ((j / IQ) & 1) ^ 1, ab, 0x18, j)) return -1;
    int idx = atomicAdd(sc.claim, 1);
    if (idx >= sc.nitems) idx = -1;
    iq[slot] = idx;
    mbar_arrive(iq_full(slot));
    if (PAIR) {
      st_shared_cluster(mapa_shared(smem_u32(iq + slot), 1u), idx);
      mbar_arrive_release_cluster(mapa_shared(iq_full(slot), 1u));
    }
    return idx;
  };
  // Every other role reads item j from its own CTA's slot (one thread per
  // role) and tells the producer the slot has been read.
  auto read_item = [&](int j) -> int {
    const int slot = j % IQ;
    if (!mbar_wait<true>(iq_full(slot), (j / IQ) & 1, ab, 0x19, j)) return -1;
    const int idx = *reinterpret_cast<volatile int*>(iq + slot);
    if (PAIR && !leader)
      mbar_arrive_cluster(mapa_shared(iq_empty(slot), 0u));
    else
      mbar_arrive(iq_empty(slot));
    return idx;
  };
  auto read_item_warp = [&](int j) -> int {
    int idx = -1;
    if (lane == 0) idx = read_item(j);
    return __shfl_sync(0xffffffffu, idx, 0);
  };

  if (warp == WARP_TMA) {
    if (lane == 0) {
      int g = 0;
      int issued = 0;
      for (int j = 0; !*abort_flag; ++j) {
        const int idx = leader ? produce_item(j) : read_item(j);
        if (idx < 0) break;
        const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
        const CUtensorMap* map = &ig.pr->map;
        tma_prefetch_desc(map);
        if (DIST == kStored) tma_prefetch_desc(&ig.pr->smap);
        const uint32_t tx = static_cast<uint32_t>(2 * ig.cols * LK * 2) +  // hi + lo
                            (DIST == kStored ? C::OPS : 0u);               // + the S tile
        const int32_t z0 =
            static_cast<int32_t>((ig.q0 + static_cast<int64_t>(rank) * ig.cols) / HCHUNK);
        // FP32 A, split in place by the workers (Rademacher items on pairs) or
        // by the epilogue warps (EC)
        const bool conv =
            (DIST == kRademacher || DIST == kMixed || EC) && PAIR && ig.pr->conv_inline;
        const int32_t x0 = static_cast<int32_t>(ig.q0 + static_cast<int64_t>(rank) * ig.cols);
        if (conv) tma_prefetch_desc(&ig.pr->amap);
        for (int s = 0; s < ig.nsteps; ++s, ++g) {
          const int so = g % C::NSO;
          // the MMAs that read this slot last time have completed
          if (g >= C::NSO && !mbar_wait(empty_o(so), ((g / C::NSO) & 1) ^ 1, ab, 0x13, g)) break;
          if (g == sc.stall_stage) continue;  // injected stall: this stage never lands
          mbar_arrive_expect_tx(full_b(so), tx);
          const int32_t y = static_cast<int32_t>(ig.lbeg + static_cast<int64_t>(s) * LK);
          if (conv) {  // FP32 A: this CTA's columns as 32-column blocks of 4 KB
            if (ig.pr->conv_inline == 1) {
              tma_load_3d(sbase + C::OFF_B + so * C::OPB, &ig.pr->amap, 0, y, x0 / 32, full_b(so));
            } else {
              for (int b = 0; b < ig.cols / 32; ++b)
                tma_load_2d(sbase + C::OFF_B + so * C::OPB + static_cast<uint32_t>(b) * 4096u,
                             &ig.pr->amap, x0 + 32 * b, y, full_b(so));
            }
          } else
            tma_load_4d(sbase + C::OFF_B + so * C::OPB, map, 0, y, z0, 0, full_b(so));
          if (DIST == kStored)  // S rows p0.., columns y.. of the stage, in the operand layout
            tma_load_5d(sbase + C::OFF_S + so * C::OPS, &ig.pr->smap, 0, 0, 0,
                        static_cast<int32_t>(ig.p0 / 8), y / 16, full_b(so));
          issued = g + 1;
        }
      }
      if (*abort_flag) {  // let the copies already issued land before leaving
        for (int t = max(0, issued - C::NSO); t < issued; ++t)
          drain_wait(full_b(t % C::NSO), (t / C::NSO) & 1, 100000000ull);
      }
    }
  } else if (warp == WARP_MMA) {
    if (lane == 0 && leader) {
      int g = 0, gc = 0;
      bool stop = false;
      for (int j = 0; !stop; ++j) {
        const int idx = read_item(j);
        if (idx < 0) break;
        const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
        const uint32_t idesc =
            idesc_bf16_f32(PAIR ? 256u : 128u, static_cast<uint32_t>(ig.nh)) | IDESC_B_MN_MAJOR;
        // split A as loaded: [hi chunks][lo chunks] of 64 columns (4 KB each),
        // or, converted in place, [chunk][hi, lo] (8 KB per chunk)
        const bool inl =
            (DIST == kRademacher || DIST == kMixed || EC) && PAIR && ig.pr->conv_inline;
        const uint32_t chunk_stride = inl ? 2 * HCHUNK_BYTES : HCHUNK_BYTES;
        const uint32_t pstride =
            inl ? HCHUNK_BYTES : static_cast<uint32_t>(ig.cols * LK * 2);  // hi -> lo tile
        const uint32_t hstride = static_cast<uint32_t>(ig.bh / HCHUNK) * chunk_stride;
        // A descriptor holds its operand's address / 16 in its low 14 bits.
        // Every offset below is a multiple of 16 B and every operand lies
        // below 256 KB, so adding offset / 16 to a base descriptor's low word
        // gives exactly the descriptor of the offset operand; the issuer adds
        // instead of rebuilding each descriptor.
        const uint64_t a_base = smem_desc(sbase + C::OFF_S, LBO, SBO);
        const uint64_t b_base = smem_desc_sw128(sbase + C::OFF_B, chunk_stride, B_SBO);
        const uint32_t a_lo = static_cast<uint32_t>(a_base);
        const uint64_t a_hi = a_base & 0xFFFFFFFF00000000ull;
        const uint32_t b_lo = static_cast<uint32_t>(b_base);
        const uint64_t b_hi = b_base & 0xFFFFFFFF00000000ull;
        for (int s = 0; s < ig.nsteps; ++s, ++g) {
          const int so = g % C::NSO;
          const int ph = (s + ig.coff) & (ig.chain - 1);
          const bool chain_start = s == 0 || ph == 0;
          // a new chain may start only after every epilogue has read the last one
          if (chain_start && gc > 0 && !mbar_wait(acc_empty, (gc - 1) & 1, ab, 0x25, gc)) {
            stop = true;
            break;
          }
          if (!mbar_wait(full_o(so), (g / C::NSO) & 1, ab, 0x22, g)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t a_slot = a_lo + ((static_cast<uint32_t>(so) * C::OPS) >> 4);
          const uint32_t b_slot = b_lo + ((static_cast<uint32_t>(so) * C::OPB) >> 4);
#pragma unroll
          for (int ks = 0; ks < KSTEPS; ++ks) {
            const uint64_t adesc = a_hi | (a_slot + ((ks * S_SLAB) >> 4));
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                if (h >= ig.nmma) break;
                const uint64_t bdesc =
                    b_hi | (b_slot + ((static_cast<uint32_t>(pass) * pstride +
                                       static_cast<uint32_t>(h) * hstride + ks * B_KSTEP) >> 4));
                const uint32_t acc = (!chain_start || ks > 0 || pass > 0) ? 1u : 0u;
                if (PAIR)
                  mma_bf16_pair(tmem + static_cast<uint32_t>(h) * 256u, adesc, bdesc, idesc, acc);
                else
                  mma_bf16(tmem + static_cast<uint32_t>(h) * 256u, adesc, bdesc, idesc, acc);
              }
            }
          }
          const bool chain_end = ph == ig.chain - 1 || s == ig.nsteps - 1;
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
    // Problems with a TMA map of their partials drain through the TMA
    // (drain_chain_tma); otherwise a warp reads 32 accumulator rows (its TMEM
    // lane quarter) x 32 columns, then writes them through a transpose tile so
    // that every global store / reduction instruction covers 64-byte pieces
    // of 8 rows instead of 16 bytes of 32 rows.
    const int quarter = warp & 3;
    const int colset = (warp - WARP_EPI0) >> 2;  // 0 or 1: even / odd 32-column chunks
    float* tile = reinterpret_cast<float*>(smem + C::OFF_EPI + (warp - WARP_EPI0) * C::EPI_BYTES);
    const uint32_t tile_u32 = smem_u32(tile);
    const int rsub = lane >> 2;       // row within a group of 8 (read side)
    const int csub = (lane & 3) * 4;  // first of 4 columns (read side)
    if constexpr (EC) {
      // Split each stage's FP32 A tile in place (4-warp sets take alternate
      // 64-column chunks) and certify it to the MMA issuer; the chain that
      // ended at a stage is drained once the next stage is certified, so
      // the MMA issuer finds an operand ready when the accumulator frees.
      const int ew = warp - WARP_EPI0;
      const int cwt = (ew & 3) * 32 + lane;  // thread index in its 4-warp set
      const int cset = ew >> 2;
      int g = 0, gc = 0;
      bool stop = false;
      int pend = -1;  // item whose chain ended at the last certified stage, or -1
      bool pend_first = false;
      auto drain_pending = [&]() -> bool {
        const ItemGeo pg = item_geo<PAIR>(sc, pend, rank);
        const LeftItem it = sc.items[pend];
        if (C::TDRAIN && pg.pr->tma_drain)
          return drain_chain_tma<PAIR>(tmem, quarter, colset, tile_u32, tile, pg, it.z,
                                       pend_first, acc_full, lead_acc_empty, gc++, ab);
        float* part_item =
            pg.pr->part + static_cast<int64_t>(it.z) * pg.pr->P * pg.pr->ldp + pg.q0;
        return drain_chain_left<PAIR>(tmem, quarter, colset, tile, pg, part_item, pend_first,
                                      acc_full, lead_acc_empty, gc++, ab);
      };
      for (int j = 0; !stop; ++j) {
        const int idx = read_item_warp(j);
        if (idx < 0) break;
        const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
        int chains = 0;  // chains of this item begun so far
        for (int s = 0; s < ig.nsteps; ++s, ++g) {
          const int so = g % C::NSO;
          const bool ok = mbar_wait(full_b(so), (g / C::NSO) & 1, ab, 0x30, g);
          if (!__all_sync(0xffffffffu, ok)) {
            stop = true;
            break;
          }
          if (ig.pr->conv_inline && (DIST == kMixed ? ig.dist : DIST) != kRademacher)
            convert_stage(smem + C::OFF_B + so * C::OPB, ig.cols, cwt, cset, 2);
          fence_proxy_async_smem();  // the split tile is read by the tensor core
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(lead_full_o + 8u * so);
          if (pend >= 0) {
            if (!drain_pending()) {
              stop = true;
              break;
            }
            pend = -1;
          }
          const int ph = (s + ig.coff) & (ig.chain - 1);
          if (ph == ig.chain - 1 || s == ig.nsteps - 1) {  // a chain ends at this stage
            pend = idx;
            pend_first = chains == 0;
            ++chains;
          }
        }
      }
      if (pend >= 0 && !stop) drain_pending();
      if (C::TDRAIN && lane == 0) bulk_wait<0>();  // the last copies have completed
    } else {
      int gc = 0;
      bool stop = false;
      for (int j = 0; !stop; ++j) {
        const int idx = read_item_warp(j);
        if (idx < 0) break;
        const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
        const LeftItem it = sc.items[idx];
        const int64_t P = ig.pr->P, Q = ig.pr->Q, ldp = ig.pr->ldp;
        float* part_item = ig.pr->part + static_cast<int64_t>(it.z) * P * ldp + ig.q0;
        const bool vec_ok = (ldp % 4) == 0;
        const int nchains = (ig.nsteps + ig.coff + ig.chain - 1) / ig.chain;
        if (C::TDRAIN && ig.pr->tma_drain) {
          for (int c0 = 0; c0 < nchains; ++c0) {
            if (!drain_chain_tma<PAIR>(tmem, quarter, colset, tile_u32, tile, ig, it.z, c0 == 0,
                                       acc_full, lead_acc_empty, gc++, ab)) {
              stop = true;
              break;
            }
          }
          continue;
        }
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
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              // lane = accumulator row: its 16 columns into the tile
#pragma unroll
              for (int q = 0; q < 4; ++q)
                *reinterpret_cast<float4*>(tile + lane * EPI_PITCH + 4 * q) =
                    make_float4(__uint_as_float(v[16 * half + 4 * q]),
                                __uint_as_float(v[16 * half + 4 * q + 1]),
                                __uint_as_float(v[16 * half + 4 * q + 2]),
                                __uint_as_float(v[16 * half + 4 * q + 3]));
              __syncwarp();
              // 4 consecutive columns (bh is a multiple of 8: they never straddle)
              const int tcol = ci * 32 + 16 * half + csub;
              const int h = tcol >> 8;
              const int c = tcol & 255;
              const int tn = PAIR ? (c < ig.bh ? h * ig.bh + c : ig.cols + h * ig.bh + (c - ig.bh))
                                  : tcol;
              const int64_t col = ig.q0 + tn;
#pragma unroll
              for (int pass = 0; pass < 4; ++pass) {
                const int rr = 8 * pass + rsub;
                const int64_t gp = ig.p0 + quarter * 32 + rr;
                const float4 a = *reinterpret_cast<const float4*>(tile + rr * EPI_PITCH + csub);
                if (c < ig.nh && gp < P) {
                  float* d = part_item + gp * ldp + tn;
                  if (vec_ok && col + 4 <= Q) {
                    if (c0 == 0)
                      *reinterpret_cast<float4*>(d) = a;
                    else
                      red_add_v4(d, a.x, a.y, a.z, a.w);
                  } else {
                    const float vv[4] = {a.x, a.y, a.z, a.w};
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
              __syncwarp();
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
      if (C::TDRAIN && lane == 0) bulk_wait<0>();  // the last copies have completed
    }
  } else {
    // ---- workers: generate this CTA's S tile, hand the stage to the MMA ----
    // group grp handles the stages g = grp (mod NGROUPS)
    const int grp = (warp - WARP_WORK0) / C::GROUP_WARPS;
    const int wt = threadIdx.x - 32 * WARP_WORK0 - grp * C::GROUP_THREADS;
    constexpr int RAD_IT = (BM + C::GROUP_THREADS - 1) / C::GROUP_THREADS;
    uint32_t cached_blk[RAD_IT];
    uint4 words[RAD_IT];
    int g = 0;
    bool stop = false;
    for (int j = 0; !stop; ++j) {
      const int idx = read_item_warp(j);
      if (idx < 0) break;
      const ItemGeo ig = item_geo<PAIR>(sc, idx, rank);
#pragma unroll
      for (int it = 0; it < RAD_IT; ++it) {  // Philox words belong to one problem and row
        cached_blk[it] = 0xffffffffu;
        words[it] = make_uint4(0u, 0u, 0u, 0u);
      }
      // this group's stages of the item: g_item + s = grp (mod NGROUPS)
      const int g_item = g;
      for (int s = ((grp - g_item) % C::NGROUPS + C::NGROUPS) % C::NGROUPS; s < ig.nsteps;
           s += C::NGROUPS) {
        g = g_item + s;
        const int so = g % C::NSO;
        // the MMAs that read S tile `so` last time have completed
        bool ok = g < C::NSO || mbar_wait(empty_o(so), ((g / C::NSO) & 1) ^ 1, ab, 0x43, g);
        if (!__all_sync(0xffffffffu, ok)) {  // leave together (abort path)
          stop = true;
          break;
        }
        uint8_t* sdst = smem + C::OFF_S + so * C::OPS;
        const int64_t cbase = ig.lbeg + static_cast<int64_t>(s) * LK;
        if constexpr (DIST == kStored) {
          // the S tile arrives with the split A tile
        } else if constexpr (DIST != kMixed) {
          // one problem per launch: its round keys are launch parameters
          gen_stage<DIST, C>(sdst, ig, sc.rk, cbase, wt, cached_blk, words);
        } else {
          if (ig.dist == kRademacher)
            gen_stage<kRademacher, C>(sdst, ig, ig.key, cbase, wt, cached_blk, words);
          else if (ig.dist == kUniform)
            gen_stage<kUniform, C>(sdst, ig, ig.key, cbase, wt, cached_blk, words);
          else
            gen_stage<kGaussian, C>(sdst, ig, ig.key, cbase, wt, cached_blk, words);
        }
        // FP32 A of a Rademacher item: the workers split it (the sign bits
        // leave them idle)
        const bool wconv = (DIST == kRademacher || DIST == kMixed) && PAIR &&
                           ig.pr->conv_inline && (DIST != kMixed || ig.dist == kRademacher);
        if (!EC || wconv) {  // with EC the epilogue warps certify the A tile
          // this CTA's split A tile of the stage has landed
          ok = mbar_wait(full_b(so), (g / C::NSO) & 1, ab, 0x40, g);
          if (!__all_sync(0xffffffffu, ok)) {
            stop = true;
            break;
          }
        }
        if constexpr ((DIST == kRademacher || DIST == kMixed) && PAIR) {
          static_assert(C::GROUP_THREADS == 128, "a worker group is one 4-warp set");
          if (wconv) convert_stage(smem + C::OFF_B + so * C::OPB, ig.cols, wt);
        }
        fence_proxy_async_smem();  // the S tile is read by the tensor core
        __syncwarp();
        if (lane == 0) {
          if (PAIR)
            mbar_arrive_cluster(lead_full_o + 8u * so);
          else
            mbar_arrive(full_o(so));
        }
      }
      g = g_item + ig.nsteps;
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
// chains and bounded waits are those of the left kernel.
//
// One ring of stages: the TMA brings a stage's FP32 A tile [256 rows][16]
// into the slot (64-byte swizzle), and the workers split it in place.  The
// 512 bytes of an 8-row group of the FP32 tile become that group's K-major
// BF16 core matrices, hi (256 bytes: 8 rows x 2 halves of 8 columns) then
// lo, so a warp converts whole groups with no other warp involved, and the
// MMA reads hi and lo with 512 bytes between 8-row groups.  With no separate
// staging ring the slots are 20 KB and the ring is 8 stages deep, so up to
// 128 KB of A per SM are in flight from HBM.  The kernel is persistent: as
// many clusters as can be resident each take an equal contiguous share of
// the stages of all blocks, with ring slots,
// barrier phases and chains counted across items, so the next item's copies
// and S tiles are under way while the last chain of the previous one drains.
// ---------------------------------------------------------------------------
struct CfgR {
  static constexpr int ROWS = 256;  // rows of A per CTA (two 128-row accumulators)
  static constexpr int NGROUPS = 4;
  static constexpr int GROUP_WARPS = NUM_WORK_WARPS / NGROUPS;
  static constexpr int GROUP_THREADS = 32 * GROUP_WARPS;
  static constexpr int NS = 8;                        // stages in the ring
  static constexpr uint32_t OPA = BK * ROWS * 4;      // FP32 A tile = its hi and lo halves
  static constexpr uint32_t ACC_A = OPA / 2;          // hi + lo of one 128-row accumulator
  static constexpr uint32_t GROUP_A = 512;            // one 8-row group, FP32 = hi + lo
  static constexpr uint32_t OPS = 128 * BK * 2;       // this CTA's half of the S tile
  static constexpr uint32_t OFF_A = 0;
  static constexpr uint32_t OFF_S = OFF_A + NS * OPA;
  // epilogue area per warp: two staging tiles of a TMA drain, or the
  // transpose tile (32 rows x 32 columns, pitch 36 floats) of the red.add one
  static constexpr int EPI_PITCH_R = 36;
  static constexpr uint32_t EPI_TILE_R = 32 * EPI_PITCH_R * 4;
  static constexpr uint32_t EPI_BYTES = 2 * DRAIN_TILE;
  static constexpr uint32_t OFF_EPI = OFF_S + NS * OPS;
  static constexpr uint32_t OFF_BAR = OFF_EPI + NUM_EPI_WARPS * EPI_BYTES;
  // per slot: A landed, operands ready, slot read by both pairs' MMAs, S rows
  // received from the partner CTA; then the accumulator and drain barriers
  static constexpr uint32_t NUM_BARS = 4 * NS + 3;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NUM_BARS * 8;
  static constexpr uint32_t SMEM = OFF_MISC + 16 + 1024;
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
  static_assert(NGROUPS <= NS, "worker groups vs ring depth");
  static_assert(OPA % 1024 == 0 && OPS % 1024 == 0, "slots on 1 KB boundaries");
  static_assert(OFF_EPI % 1024 == 0 && EPI_BYTES >= EPI_TILE_R, "epilogue tiles");
};

struct TcRightParams {
  float* part;      // partials [segments][P][Q] (a block's segments in order)
  int64_t P, Q, L;  // P = m, Q = k, L = n
  int nq;           // N of the MMA: k rows per pair tile (multiple of 16, <= 256)
  int tmem_cols;    // power of two >= 2 * nq
  PhiloxRoundKeys rk;
  int* status;
  uint64_t timeout_ns;
  int tma_drain;  // the partials' tensor map (kernel parameter tmapP) is valid
  // work: blocks (4 x 256 rows of m, pair tile of k; tile of k fastest) of
  // `steps` stages of n each, `units` = blocks x steps stages in all; cluster
  // c of NC takes the stages [c units / NC, (c+1) units / NC) in block order
  int units, steps, tiles_q;
};

// The cluster (of nc) whose share of the right kernel's stages holds stage
// u: cluster c takes [floor(c U / nc), floor((c+1) U / nc)) (U >= nc).
__host__ __device__ inline int64_t seg_owner(int64_t u, int64_t U, int64_t nc) {
  return ((u + 1) * nc + U - 1) / U - 1;
}

// One segment of the persistent right kernel, as seen by one CTA: a block's
// stages [s0, s1) within one cluster's share; z numbers the segments of the
// block (its partial).
struct RightItem {
  int64_t m0, q0, g0;  // first row of A, of the pair's k rows, of this CTA's S rows
  int64_t lbeg, lend;  // range of n
  int nsteps, nchains, z;
};

// The right kernel's accumulator drain through the TMA, as drain_chain_tma:
// accumulator j (0, 1) holds rows m0 + 128 j + lane of the warp's TMEM lane
// quarter and the pair's k rows q0 + c in its columns.
__device__ __noinline__ bool drain_right_tma(uint32_t tmem, int quarter, int colset,
                                             uint32_t stage_u32, float* stage,
                                             const CUtensorMap* pmap, int nq, int64_t m0,
                                             int64_t q0, int z, bool first, uint32_t acc_full,
                                             uint32_t lead_acc_empty, int c0, const Abort ab) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) bulk_wait<0>();
  const bool ok = mbar_wait(acc_full, c0 & 1, ab, 0x34, c0);
  if (!__all_sync(0xffffffffu, ok)) return false;  // tcgen05.ld below is warp-collective
  tc_fence_after();
  const int nchunk = (nq + 31) / 32;
  const uint32_t sw = static_cast<uint32_t>(lane) & 7u;
  int nb = 0;
  for (int t = colset; t < 2 * nchunk; t += 2, ++nb) {
    const int j = t / nchunk;
    const int ci = t - j * nchunk;
    uint32_t v[32];
    tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                  static_cast<uint32_t>(j * nq + ci * 32),
              v);
    tmem_ld_wait();
    const uint32_t b = static_cast<uint32_t>(nb & 1);
    if (nb >= 2) {
      if (lane == 0) bulk_wait_read<1>();
      __syncwarp();
    }
    float* row = stage + b * (DRAIN_TILE / 4) + lane * 32;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(row + ((static_cast<uint32_t>(q) ^ sw) << 2)) =
          make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                      __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
    fence_proxy_async_smem();  // the tile is read by the TMA
    __syncwarp();
    if (lane == 0) {
      const int32_t x = static_cast<int32_t>(q0 + ci * 32);
      const int32_t y = static_cast<int32_t>(m0 + j * 128 + quarter * 32);
      const uint32_t src = stage_u32 + b * DRAIN_TILE;
      if (first)
        tma_store_3d(pmap, src, x, y, z);
      else
        tma_reduce_add_3d(pmap, src, x, y, z);
      bulk_commit();
    }
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive_cluster(lead_acc_empty);
  return true;
}

template <int DIST>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_sketch_bf16x2_right(const __grid_constant__ CUtensorMap tmapA,
                          const __grid_constant__ CUtensorMap tmapP, const TcRightParams p) {
  using C = CfgR;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + C::OFF_BAR;
  // full_b: the slot's FP32 A tile has landed; full_o (even CTA): both CTAs'
  // operands of the stage are ready; empty_o: both pairs' MMAs have read
  // what this CTA wrote into the slot (here and, S rows, in its partner);
  // s_recv: the S rows the partner CTA copies into the slot have landed
  auto full_b = [&](int i) { return bar0 + 8u * i; };
  auto full_o = [&](int i) { return bar0 + 8u * (C::NS + i); };
  auto empty_o = [&](int i) { return bar0 + 8u * (2 * C::NS + i); };
  auto s_recv = [&](int i) { return bar0 + 8u * (3 * C::NS + i); };
  const uint32_t acc_full = bar0 + 8u * (4 * C::NS);
  const uint32_t acc_empty = acc_full + 8u;
  const uint32_t drain_bar = acc_full + 16u;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::OFF_MISC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // a cluster holds two CTA pairs (cluster ranks 0-1 and 2-3) with the same
  // k rows and the same range of n on consecutive rows of m; the two CTAs of
  // equal rank in the two pairs hold the same rows of the S tile, and each
  // generates half of them and copies that half into its partner
  const uint32_t cr = cluster_ctarank();
  const uint32_t rank = cr & 1u;  // 0 = even CTA of the pair (MMA issuer)
  const uint32_t pairi = cr >> 1;
  const uint32_t lead_rank = cr & ~1u;          // the pair's even CTA
  const uint32_t partner = cr ^ 2u;             // same rank, other pair
  const uint32_t partner_lead = partner & ~1u;  // the other pair's even CTA
  const bool leader = rank == 0;
  const int nq = p.nq;
  const int gh = nq / 2;                                       // S rows this CTA holds
  const int gq = gh / 2;                                       // ... and generates
  const int gbase = static_cast<int>(pairi) * gq;              // from this row of them
  // Persistent: the stages of all blocks (1024 rows of m x a pair tile of k
  // rows, each `steps` stages of n long) are laid end to end, and cluster c
  // of the NC in the grid takes an equal contiguous share of them, every CTA
  // of the cluster the same; a share is one or a few segments, one per block
  // it touches, each summed into the partial of its place in the block.  Ring
  // slots, barrier phases and accumulation chains are counted across
  // segments, so the next segment's copies and S tiles are under way while
  // the last chain drains.
  const int cl = static_cast<int>(blockIdx.x >> 2);
  const int ncl = static_cast<int>(gridDim.x >> 2);
  const int ubeg = static_cast<int>(static_cast<int64_t>(cl) * p.units / ncl);
  const int uend = static_cast<int>(static_cast<int64_t>(cl + 1) * p.units / ncl);
  auto item = [&](int u) {
    RightItem it;
    const int blk = u / p.steps;
    const int s0 = u - blk * p.steps;
    const int s1 = min(p.steps, s0 + (uend - u));
    it.z = static_cast<int>(cl - seg_owner(static_cast<int64_t>(blk) * p.steps, p.units, ncl));
    const int64_t qt = blk % p.tiles_q;
    const int64_t mb = blk / p.tiles_q;
    it.m0 = (mb * 4 + cr) * C::ROWS;  // this CTA's rows of A
    it.q0 = qt * nq;                  // the pair's k rows
    it.g0 = it.q0 + static_cast<int64_t>(rank) * gh;  // this CTA's S rows
    it.lbeg = static_cast<int64_t>(s0) * BK;
    it.lend = min(p.L, static_cast<int64_t>(s1) * BK);
    it.nsteps = s1 - s0;
    it.nchains = (it.nsteps + CHAIN - 1) / CHAIN;
    return it;
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NS; ++i) {
      mbar_init(full_b(i), 1);
      mbar_init(full_o(i), C::GROUP_WARPS * 2);  // one worker group of each CTA of the pair
      mbar_init(empty_o(i), 2);  // the MMAs of both pairs read what this CTA wrote
      mbar_init(s_recv(i), 1);   // the receiving group's expect-tx, plus the copy's bytes
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
  const uint32_t lead_full_o = mapa_shared(full_o(0), lead_rank);
  const uint32_t partner_s_recv = mapa_shared(s_recv(0), partner);
  const uint32_t partner_s = mapa_shared(sbase + C::OFF_S, partner);
  const uint32_t lead_acc_empty = mapa_shared(acc_empty, lead_rank);
  const uint16_t pair_mask = static_cast<uint16_t>(3u << (2u * pairi));

  if (warp == WARP_TMA) {
    if (lane == 0) {
      int issued = 0, g = 0;
      bool stop = false;
      for (int u = ubeg; u < uend && !stop;) {
        const RightItem it = item(u);
        u += it.nsteps;
        for (int s = 0; s < it.nsteps; ++s, ++g) {
          const int so = g % C::NS;
          // both pairs' MMAs have read the slot's previous stage
          if (g >= C::NS && !mbar_wait(empty_o(so), ((g / C::NS) & 1) ^ 1, ab, 0x13, g)) {
            stop = true;
            break;
          }
          mbar_arrive_expect_tx(full_b(so), C::OPA);
          tma_load_2d(sbase + C::OFF_A + so * C::OPA, &tmapA,
                      static_cast<int32_t>(it.lbeg + static_cast<int64_t>(s) * BK),
                      static_cast<int32_t>(it.m0), full_b(so));
          issued = g + 1;
        }
      }
      if (*abort_flag) {
        for (int s = max(0, issued - C::NS); s < issued; ++s)
          drain_wait(full_b(s % C::NS), (s / C::NS) & 1, 100000000ull);
      }
    }
  } else if (warp == WARP_MMA) {
    if (lane == 0 && leader) {
      const uint32_t idesc = idesc_bf16_f32(256u, static_cast<uint32_t>(nq));
      // The single issuing thread's bookkeeping per stage bounds this kernel
      // (it issues 4 MMAs per 512 tensor cycles), so the slot, phase and
      // chain are counted, not divided, and every operand descriptor is a
      // base descriptor plus offset / 16 in its low word (exact: all offsets
      // are multiples of 16 B and every operand lies below 256 KB).
      const uint64_t a_base = smem_desc(sbase + C::OFF_A, LBO, C::GROUP_A);
      const uint64_t b_base = smem_desc(sbase + C::OFF_S, LBO, SBO);
      const uint32_t a_lo = static_cast<uint32_t>(a_base);
      const uint64_t a_hi = a_base & 0xFFFFFFFF00000000ull;
      const uint32_t b_lo = static_cast<uint32_t>(b_base);
      const uint64_t b_hi = b_base & 0xFFFFFFFF00000000ull;
      int so = 0, chain_no = 0, g = 0;
      uint32_t ph = 0;
      bool stop = false;
      for (int u = ubeg; u < uend && !stop;) {
      const int nsteps = item(u).nsteps;
      u += nsteps;
      int in_chain = 0;
      for (int s = 0; s < nsteps; ++s, ++g) {
        const bool chain_start = in_chain == 0;
        // a chain starts once the epilogue has read the previous one
        if (chain_start && chain_no > 0 &&
            !mbar_wait(acc_empty, (chain_no - 1) & 1, ab, 0x25, g)) {
          stop = true;
          break;
        }
        if (!mbar_wait(full_o(so), ph, ab, 0x22, g)) {
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t a_slot = a_lo + static_cast<uint32_t>(so) * (C::OPA >> 4);
        const uint64_t bdesc = b_hi | (b_lo + static_cast<uint32_t>(so) * (C::OPS >> 4));
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          // hi (pass 0) or lo (pass 1) of accumulator j: 8-row groups 512 B apart
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const uint64_t adesc =
                a_hi | (a_slot + ((static_cast<uint32_t>(pass) * 256u +
                                   static_cast<uint32_t>(j) * C::ACC_A) >> 4));
            mma_bf16_pair(tmem + static_cast<uint32_t>(j * nq), adesc, bdesc, idesc,
                          (!chain_start || pass > 0) ? 1u : 0u);
          }
        }
        mma_commit_pair_mask(empty_o(so), 0xF);  // all four CTAs wrote into the slot
        if (in_chain == CHAIN - 1 || s == nsteps - 1) {  // the chain ends
          mma_commit_pair_mask(acc_full, pair_mask);
          in_chain = 0;
          ++chain_no;
        } else {
          ++in_chain;
        }
        if (++so == C::NS) {
          so = 0;
          ph ^= 1u;
        }
      }
      }
      mma_commit_pair(drain_bar);
      drain_wait(drain_bar, 0, 200000000ull);
    }
  } else if (warp < WARP_WORK0) {
    // ---- epilogue: accumulator j holds rows m0 + 128 j + lane, columns q0 + c ----
    // A warp reads 32 accumulator rows (its TMEM lane quarter) x 32 columns
    // and writes them through a transpose tile, so that every global store /
    // reduction instruction covers whole 128-byte rows, 4 of them, instead of
    // 16 bytes of 32 rows (an eighth of the memory requests: the drain of a
    // chain stalls the MMA issuer, which waits for the whole TMEM).
    const int quarter = warp & 3;
    const int colset = (warp - WARP_EPI0) >> 2;
    const bool vec_ok = (p.Q % 4) == 0;
    const int nchunk = (nq + 31) / 32;
    float* tile = reinterpret_cast<float*>(smem + C::OFF_EPI + (warp - WARP_EPI0) * C::EPI_BYTES);
    const int rsub = lane >> 3;       // row within a group of 4 (read side)
    const int csub = (lane & 7) * 4;  // first of 4 columns (read side)
    int gc = 0;  // chains drained so far (all segments)
    bool stop = false;
    for (int u = ubeg; u < uend && !stop;) {
    const RightItem it = item(u);
    u += it.nsteps;
    const int64_t m0 = it.m0, q0 = it.q0;
    for (int c0 = 0; c0 < it.nchains; ++c0, ++gc) {
      if (p.tma_drain) {  // through the TMA (partial rows of whole 16-byte units)
        if (!drain_right_tma(tmem, quarter, colset, smem_u32(tile), tile, &tmapP, nq, m0, q0,
                             it.z, c0 == 0, acc_full, lead_acc_empty, gc, ab)) {
          stop = true;
          break;
        }
        continue;
      }
      const bool ok = mbar_wait(acc_full, gc & 1, ab, 0x34, gc);
      if (!__all_sync(0xffffffffu, ok)) {
        stop = true;
        break;
      }
      tc_fence_after();
      for (int t = colset; t < 2 * nchunk; t += 2) {
        const int j = t / nchunk;
        const int ci = t - j * nchunk;
        uint32_t v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                      static_cast<uint32_t>(j * nq + ci * 32),
                  v);
        tmem_ld_wait();
        const int64_t grow0 = m0 + j * 128 + quarter * 32;  // the warp's first row of m
        // lane = accumulator row: its 32 columns into the tile
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(tile + lane * C::EPI_PITCH_R + 4 * q) =
              make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                          __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
        __syncwarp();
        const int c = ci * 32 + csub;  // column of the pair's k rows
        const int64_t col = q0 + c;
#pragma unroll
        for (int pass = 0; pass < 8; ++pass) {
          const int rr = 4 * pass + rsub;
          const int64_t gm = grow0 + rr;
          const float4 a = *reinterpret_cast<const float4*>(tile + rr * C::EPI_PITCH_R + csub);
          if (gm < p.P && c < nq) {
            float* d = p.part + (static_cast<int64_t>(it.z) * p.P + gm) * p.Q + col;
            if (vec_ok && col + 4 <= p.Q) {
              if (c0 == 0)
                *reinterpret_cast<float4*>(d) = a;
              else
                red_add_v4(d, a.x, a.y, a.z, a.w);
            } else {
              const float vv[4] = {a.x, a.y, a.z, a.w};
              for (int u = 0; u < 4; ++u) {
                if (col + u < p.Q && c + u < nq) {
                  if (c0 == 0)
                    d[u] = vv[u];
                  else
                    red_add(d + u, vv[u]);
                }
              }
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_acc_empty);
    }
    }
    if (p.tma_drain && lane == 0) bulk_wait<0>();  // the last copies have completed
  } else {
    // ---- workers: this CTA's half of the S tile, and its 256 rows of A ----
    const int grp = (warp - WARP_WORK0) / C::GROUP_WARPS;
    const int wt = threadIdx.x - 32 * WARP_WORK0 - grp * C::GROUP_THREADS;
    static_assert(C::GROUP_WARPS == 4, "16 generated rows per warp cover gq <= 64");
    const int wg = wt >> 5;       // warp of the group
    const bool gfirst = wg == 0;  // registers the expected bytes and waits for them
    // warp wg generates rows 16 wg .. 16 wg + 15 of this CTA's generated rows
    // (whole 8-row groups: 256 contiguous bytes each in the K-major layout)
    // and copies them into the partner itself, so no barrier spans the group
    const int wrows = max(0, min(16, gq - 16 * wg));
    const uint32_t w_off = static_cast<uint32_t>(gbase + 16 * wg) * 32u;
    const uint32_t w_bytes = static_cast<uint32_t>(wrows) * 32u;
    const uint32_t s_bytes = static_cast<uint32_t>(gq) * 32u;  // from all four partner warps
    uint4 words = make_uint4(0u, 0u, 0u, 0u);
    int pend = -1;  // a stage whose copy into this CTA was expected, not yet waited for
    int g = 0;      // stages of the earlier segments
    bool stop = false;
    for (int u = ubeg; u < uend && !stop;) {
    const RightItem it = item(u);
    u += it.nsteps;
    const int64_t g0 = it.g0, lend = it.lend;
    uint32_t cached_blk = 0xffffffffu;  // Philox words belong to one segment's rows
    // this group's stages of the segment: g_item + s = grp (mod NGROUPS)
    const int g_item = g;
    for (int s = ((grp - g_item) % C::NGROUPS + C::NGROUPS) % C::NGROUPS; s < it.nsteps;
         s += C::NGROUPS) {
      g = g_item + s;
      const int so = g % C::NS;
      // both pairs' MMAs have read what this CTA wrote into slot `so` (here
      // and in its partner) last time
      bool ok = g < C::NS || mbar_wait(empty_o(so), ((g / C::NS) & 1) ^ 1, ab, 0x43, g);
      if (!__all_sync(0xffffffffu, ok)) {
        stop = true;
        break;
      }
      uint8_t* sdst = smem + C::OFF_S + so * C::OPS;
      // the partner's half of this CTA's S rows will land here
      if (gfirst) {
        if (lane == 0) mbar_arrive_expect_tx(s_recv(so), s_bytes);
        pend = g;
      }
      const int64_t cbase = it.lbeg + static_cast<int64_t>(s) * BK;
      if (DIST == kRademacher) {
        // a lane: one row (16 wg + lane % 16) and one 8-column half (lane / 16)
        if ((lane & 15) < wrows) {
          const uint32_t r = static_cast<uint32_t>(gbase + 16 * wg + (lane & 15));
          const uint32_t hh = static_cast<uint32_t>(lane >> 4);
          const int64_t grow = g0 + r;
          const int64_t c0 = cbase + 8 * hh;
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (grow < p.Q && c0 < lend) {
            const uint32_t c = static_cast<uint32_t>(c0);
            const uint32_t blk = c >> 7;
            if (blk != cached_blk) {
              words = rademacher_bits(p.rk, static_cast<uint32_t>(grow), blk, 0u);
              cached_blk = blk;
            }
            const uint32_t wsel = (c >> 5) & 3u;
            const uint4 wv = words;
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
        // a lane owns quad qd = lane / 8 of rows 16 wg + 8 it + lane % 8 (the 16
        // lanes of a store phase write 8 rows x 16 B: every bank once)
        const uint32_t qd = (static_cast<uint32_t>(lane) >> 3) & 3u;
        const bool cv = cbase + 4 * qd < lend;
        const uint32_t j = static_cast<uint32_t>(cbase >> 2) + qd;  // Philox block
#pragma unroll
        for (int it = 0; it < 2; ++it) {
          const int rr = 8 * it + (lane & 7);
          if (rr >= wrows) continue;
          const uint32_t r = static_cast<uint32_t>(gbase + 16 * wg + rr);
          const int64_t grow = g0 + r;
          uint2 v = make_uint2(0u, 0u);
          if (grow < p.Q && cv) {
            const float4 a = DIST == kUniform
                                 ? uniform4(p.rk, static_cast<uint32_t>(grow), j, 0u)
                                 : gaussian4(p.rk, static_cast<uint32_t>(grow), j, 0u);
            v = make_uint2(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w));
          }
          const uint32_t off = kmaj_off(r, qd >> 1) + (qd & 1u) * 8u;
          *reinterpret_cast<uint2*>(sdst + off) = v;
        }
      }
      // this warp's rows are written: copy them into the partner (async
      // proxy, completing on its s_recv barrier)
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0 && w_bytes != 0)
        bulk_copy_to_cluster(partner_s + static_cast<uint32_t>(so) * C::OPS + w_off,
                             smem_u32(sdst) + w_off, w_bytes, partner_s_recv + 8u * so);
      ok = mbar_wait(full_b(so), (g / C::NS) & 1, ab, 0x40, g);
      if (!__all_sync(0xffffffffu, ok)) {
        stop = true;
        break;
      }
      // split the FP32 A tile in place, two 8-row groups (512 bytes each) per
      // warp at a time: lane = (group lane / 16, row r = lane % 8, columns
      // 8 h .. 8 h + 7 with h = (lane / 8) % 2).  The TMA lands each 64-byte
      // row with the 64-byte swizzle (16-byte unit u of row r at
      // u ^ ((r / 2) mod 4)), so the 8 lanes of a load phase read 8 different
      // bank groups; the row's hi core-matrix row (8 columns, 16 bytes)
      // replaces bytes 128 h + 16 r of the group, its lo row 256 bytes
      // further, so the 8 lanes of a store phase write 128 contiguous bytes
      {
        uint8_t* slot = smem + C::OFF_A + so * C::OPA;
        const uint32_t r = static_cast<uint32_t>(lane) & 7u;
        const uint32_t h = (static_cast<uint32_t>(lane) >> 3) & 1u;
        const uint32_t sw = (r >> 1) & 3u;
        const uint32_t ld0 = r * 64u + (((2u * h) ^ sw) << 4);
        const uint32_t ld1 = r * 64u + (((2u * h + 1u) ^ sw) << 4);
        const uint32_t dst = h * 128u + r * 16u;
#pragma unroll 2
        for (int gi = 2 * wg + (lane >> 4); gi < C::ROWS / 8; gi += 2 * C::GROUP_WARPS) {
          uint8_t* grp8 = slot + gi * C::GROUP_A;
          const float4 x = *reinterpret_cast<const float4*>(grp8 + ld0);
          const float4 y = *reinterpret_cast<const float4*>(grp8 + ld1);
          __syncwarp();  // the warp's groups have been read
          const uint32_t h0 = pack_bf16x2(x.x, x.y), h1 = pack_bf16x2(x.z, x.w);
          const uint32_t h2 = pack_bf16x2(y.x, y.y), h3 = pack_bf16x2(y.z, y.w);
          // a - hi of two elements in one packed FMA (the product by -1 is
          // exact, so each component is the rounded difference)
          const float2 l0 = __ffma2_rn(f2(__uint_as_float(h0 << 16), __uint_as_float(h0 & 0xffff0000u)),
                                       f2(-1.0f, -1.0f), f2(x.x, x.y));
          const float2 l1 = __ffma2_rn(f2(__uint_as_float(h1 << 16), __uint_as_float(h1 & 0xffff0000u)),
                                       f2(-1.0f, -1.0f), f2(x.z, x.w));
          const float2 l2 = __ffma2_rn(f2(__uint_as_float(h2 << 16), __uint_as_float(h2 & 0xffff0000u)),
                                       f2(-1.0f, -1.0f), f2(y.x, y.y));
          const float2 l3 = __ffma2_rn(f2(__uint_as_float(h3 << 16), __uint_as_float(h3 & 0xffff0000u)),
                                       f2(-1.0f, -1.0f), f2(y.z, y.w));
          *reinterpret_cast<uint4*>(grp8 + dst) = make_uint4(h0, h1, h2, h3);
          *reinterpret_cast<uint4*>(grp8 + 256u + dst) =
              make_uint4(pack_bf16x2(l0.x, l0.y), pack_bf16x2(l1.x, l1.y),
                         pack_bf16x2(l2.x, l2.y), pack_bf16x2(l3.x, l3.y));
        }
      }
      // the S half and the A operands are in this CTA's own shared memory;
      // the group's first warp certifies the partner's rows too
      fence_proxy_async_smem();
      ok = !gfirst || mbar_wait(s_recv(so), (g / C::NS) & 1, ab, 0x46, g);
      if (!__all_sync(0xffffffffu, ok)) {
        stop = true;
        break;
      }
      pend = -1;
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_full_o + 8u * so);
    }
    g = g_item + it.nsteps;
    }
    // leaving early: let a copy the partner may still be sending land first
    if (gfirst && pend >= 0 && lane == 0)
      drain_wait(s_recv(pend % C::NS), (pend / C::NS) & 1, 100000000ull);
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
// FP8 form of the right sketch: Y[m x k] = s diag(2^e) A_q S_q^T, A_q the E4M3
// codes of A with one power-of-two scale 2^e_i per row, S_q = E4M3(g).
//
// Stages of 128 columns of n.  TMA brings this CTA's 256 rows of A_q (rows of
// 128 B, 128-byte swizzle); the workers generate this CTA's half of the E4M3
// S tile (K-major, no swizzle); per stage the even CTA issues 4 K steps x 2
// accumulators of tcgen05.mma kind::f8f6f4 (M = 256 over the pair, N = nq,
// K = 32).  The epilogue multiplies each row by its 2^e (exact) before adding
// the chain into the partial.  Roles, chains and bounded waits are those of
// the BF16 right kernel.
// ---------------------------------------------------------------------------
constexpr int QK = 128;     // contracted columns (bytes of A_q) per FP8 stage
constexpr int QCHAIN = 32;  // FP8 stages per accumulation chain (128 K steps)

struct CfgQ {
  static constexpr int ROWS = 256;  // rows of A per CTA (two 128-row accumulators)
  static constexpr int NGROUPS = 4;
  static constexpr int GROUP_WARPS = NUM_WORK_WARPS / NGROUPS;
  static constexpr int GROUP_THREADS = 32 * GROUP_WARPS;
  static constexpr int NSO = 4;
  static constexpr uint32_t OPA = ROWS * QK;  // 32 KB of A_q
  static constexpr uint32_t OPS = 128 * QK;   // 16 KB: this CTA's half of the S tile
  static constexpr uint32_t OFF_A = 0;
  static constexpr uint32_t OFF_S = OFF_A + NSO * OPA;
  static constexpr uint32_t OFF_EPI = OFF_S + NSO * OPS;  // epilogue transpose tiles
  static constexpr uint32_t OFF_BAR = OFF_EPI + NUM_EPI_WARPS * EPI_TILE;
  // per slot: A landed, operands ready, slot read by both pairs' MMAs, S rows
  // received from the partner CTA; then the accumulator and drain barriers
  static constexpr uint32_t NUM_BARS = 4 * NSO + 3;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NUM_BARS * 8;
  static constexpr uint32_t SMEM = OFF_MISC + 16 + 1024;
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
  static_assert(NGROUPS <= NSO, "worker groups vs ring depth");
};

// E4M3 S tile: [row/8][16-column block][row%8][16 B] -- K-major core matrices
// with 128 B between column blocks (LBO) and 1024 B between 8-row groups (SBO).
__device__ __forceinline__ uint32_t q8_off(uint32_t row, uint32_t col) {
  return (row >> 3) * 1024u + (col >> 4) * 128u + (row & 7u) * 16u + (col & 15u);
}

// Four consecutive +-1 entries (bits b0..b3 of x, set = -1) as E4M3 bytes:
// +1 = 0x38, -1 = 0xB8.  The multiply spreads bit i to bit 8i (no carries).
__device__ __forceinline__ uint32_t rad4_e4m3(uint32_t x) {
  return (((x & 0xFu) * 0x00204081u) & 0x01010101u) << 7 | 0x38383838u;
}

__device__ __forceinline__ uint32_t e4m3x4(float4 a) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a.x, a.y), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(a.z, a.w), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

struct TcRightQParams {
  float* part;          // partials [splits][P][Q]
  const int32_t* exps;  // row exponents of A_q
  int64_t P, Q, L;      // P = m, Q = k, L = n
  int64_t chunk;        // columns per split (multiple of QK)
  int nq;               // N of the MMA: k rows per pair tile (multiple of 16, <= 256)
  int tmem_cols;        // power of two >= 2 * nq
  PhiloxRoundKeys rk;
  int* status;
  uint64_t timeout_ns;
};

template <int DIST>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_sketch_e4m3_right(const __grid_constant__ CUtensorMap tmapA, const TcRightQParams p) {
  using C = CfgQ;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + C::OFF_BAR;
  auto full_a = [&](int i) { return bar0 + 8u * i; };
  auto full_o = [&](int i) { return bar0 + 8u * (C::NSO + i); };
  auto empty_o = [&](int i) { return bar0 + 8u * (2 * C::NSO + i); };
  auto s_recv = [&](int i) { return bar0 + 8u * (3 * C::NSO + i); };
  const uint32_t acc_full = bar0 + 8u * (4 * C::NSO);
  const uint32_t acc_empty = acc_full + 8u;
  const uint32_t drain_bar = acc_full + 16u;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::OFF_MISC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // a cluster holds two CTA pairs (cluster ranks 0-1 and 2-3) with the same
  // k rows and the same range of n on consecutive rows of m; the two CTAs of
  // equal rank hold the same rows of the S tile, and each generates half of
  // them and copies that half into its partner (as in the BF16 right sketch)
  const uint32_t cr = cluster_ctarank();
  const uint32_t rank = cr & 1u;  // 0 = even CTA of the pair (MMA issuer)
  const uint32_t pairi = cr >> 1;
  const uint32_t lead_rank = cr & ~1u;  // the pair's even CTA
  const uint32_t partner = cr ^ 2u;     // same rank, other pair
  const bool leader = rank == 0;
  const int nq = p.nq;
  const int gh = nq / 2;                          // S rows this CTA holds
  const int gq = gh / 2;                          // ... and generates (whole 8-row groups)
  const int gbase = static_cast<int>(pairi) * gq; // from this row of them
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * C::ROWS;  // this CTA's rows of A
  const int64_t q0 = static_cast<int64_t>(blockIdx.y) * nq;       // the pair's k rows
  const int64_t g0 = q0 + static_cast<int64_t>(rank) * gh;        // this CTA's S rows
  const int64_t lbeg = static_cast<int64_t>(blockIdx.z) * p.chunk;
  const int64_t lend = min(p.L, lbeg + p.chunk);
  const int nsteps = static_cast<int>((lend - lbeg + QK - 1) / QK);
  const int nchains = (nsteps + QCHAIN - 1) / QCHAIN;

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NSO; ++i) {
      mbar_init(full_a(i), 1);
      mbar_init(full_o(i), C::GROUP_WARPS * 2);
      mbar_init(empty_o(i), 2);  // the MMAs of both pairs read what this CTA wrote
      mbar_init(s_recv(i), 1);   // the receiving group's expect-tx, plus the copy's bytes
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
  const uint32_t lead_full_o = mapa_shared(full_o(0), lead_rank);
  const uint32_t lead_acc_empty = mapa_shared(acc_empty, lead_rank);
  const uint32_t partner_s_recv = mapa_shared(s_recv(0), partner);
  const uint32_t partner_s = mapa_shared(sbase + C::OFF_S, partner);
  const uint16_t pair_mask = static_cast<uint16_t>(3u << (2u * pairi));

  if (warp == WARP_TMA) {
    if (lane == 0) {
      int issued = 0;
      for (int s = 0; s < nsteps; ++s) {
        const int so = s % C::NSO;
        if (s >= C::NSO && !mbar_wait(empty_o(so), ((s / C::NSO) & 1) ^ 1, ab, 0x13, s)) break;
        mbar_arrive_expect_tx(full_a(so), C::OPA);
        tma_load_2d(sbase + C::OFF_A + so * C::OPA, &tmapA,
                    static_cast<int32_t>(lbeg + static_cast<int64_t>(s) * QK),
                    static_cast<int32_t>(m0), full_a(so));
        issued = s + 1;
      }
      if (*abort_flag) {
        for (int s = max(0, issued - C::NSO); s < issued; ++s)
          drain_wait(full_a(s % C::NSO), (s / C::NSO) & 1, 100000000ull);
      }
    }
  } else if (warp == WARP_MMA) {
    if (lane == 0 && leader) {
      const uint32_t idesc = idesc_e4m3_f32(256u, static_cast<uint32_t>(nq));
      for (int s = 0; s < nsteps; ++s) {
        const int so = s % C::NSO;
        const int in_chain = s % QCHAIN;
        if (s > 0 && in_chain == 0 &&
            !mbar_wait(acc_empty, ((s / QCHAIN) - 1) & 1, ab, 0x25, s))
          break;
        if (!mbar_wait(full_o(so), (s / C::NSO) & 1, ab, 0x22, s)) break;
        tc_fence_after();
#pragma unroll
        for (int ks = 0; ks < QK / 32; ++ks) {
          const uint64_t bdesc =
              smem_desc(sbase + C::OFF_S + so * C::OPS + static_cast<uint32_t>(ks) * 256u, 128u,
                        1024u);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const uint64_t adesc = smem_desc_sw128(
                sbase + C::OFF_A + so * C::OPA + static_cast<uint32_t>(j) * (C::OPA / 2) +
                    static_cast<uint32_t>(ks) * 32u,
                16u, 1024u);
            mma_e4m3_pair(tmem + static_cast<uint32_t>(j * nq), adesc, bdesc, idesc,
                          (in_chain > 0 || ks > 0) ? 1u : 0u);
          }
        }
        mma_commit_pair_mask(empty_o(so), 0xF);  // all four CTAs wrote into the slot
        if (in_chain == QCHAIN - 1 || s == nsteps - 1) mma_commit_pair_mask(acc_full, pair_mask);
      }
      mma_commit_pair(drain_bar);
      drain_wait(drain_bar, 0, 200000000ull);
    }
  } else if (warp < WARP_WORK0) {
    // ---- epilogue: accumulator j holds rows m0 + 128 j + lane, columns q0 + c ----
    // Each row is scaled by its 2^e as it is read from TMEM, then written
    // through a per-warp transpose tile in 64-byte pieces of 8 rows (as in
    // the BF16 right sketch).
    const int quarter = warp & 3;
    const int colset = (warp - WARP_EPI0) >> 2;
    const bool vec_ok = (p.Q % 4) == 0;
    const int nchunk = (nq + 31) / 32;
    float* tile = reinterpret_cast<float*>(smem + C::OFF_EPI + (warp - WARP_EPI0) * EPI_TILE);
    const int rsub = lane >> 2;       // row within a group of 8 (read side)
    const int csub = (lane & 3) * 4;  // first of 4 columns (read side)
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
        const int64_t grow0 = m0 + j * 128 + quarter * 32;  // the warp's first row of m
        const int64_t gl = grow0 + lane;                     // this lane's row (write side)
        const int e = gl < p.P ? p.exps[gl] : 0;  // the row's scale 2^e: an exact multiply
#pragma unroll
        for (int half = 0; half < 2; ++half) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4*>(tile + lane * EPI_PITCH + 4 * q) =
                make_float4(ldexpf(__uint_as_float(v[16 * half + 4 * q]), e),
                            ldexpf(__uint_as_float(v[16 * half + 4 * q + 1]), e),
                            ldexpf(__uint_as_float(v[16 * half + 4 * q + 2]), e),
                            ldexpf(__uint_as_float(v[16 * half + 4 * q + 3]), e));
          __syncwarp();
          const int c = ci * 32 + 16 * half + csub;
          const int64_t col = q0 + c;
#pragma unroll
          for (int pass = 0; pass < 4; ++pass) {
            const int rr = 8 * pass + rsub;
            const int64_t gm = grow0 + rr;
            const float4 a = *reinterpret_cast<const float4*>(tile + rr * EPI_PITCH + csub);
            if (gm < p.P && c < nq) {
              float* d = p.part + (static_cast<int64_t>(blockIdx.z) * p.P + gm) * p.Q + col;
              if (vec_ok && col + 4 <= p.Q) {
                if (c0 == 0)
                  *reinterpret_cast<float4*>(d) = a;
                else
                  red_add_v4(d, a.x, a.y, a.z, a.w);
              } else {
                const float vv[4] = {a.x, a.y, a.z, a.w};
                for (int u = 0; u < 4; ++u) {
                  if (col + u < p.Q && c + u < nq) {
                    if (c0 == 0)
                      d[u] = vv[u];
                    else
                      red_add(d + u, vv[u]);
                  }
                }
              }
            }
          }
          __syncwarp();
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_acc_empty);
    }
  } else {
    // ---- workers: this CTA's half of the E4M3 S tile [gh x 128] ----
    // Each warp generates whole 8-row groups (1024 contiguous bytes each in
    // the tile layout) of this CTA's generated rows and copies each into the
    // partner itself, so no barrier spans the group.
    const int grp = (warp - WARP_WORK0) / C::GROUP_WARPS;
    const int wt = threadIdx.x - 32 * WARP_WORK0 - grp * C::GROUP_THREADS;
    const int wg = wt >> 5;       // warp of the group
    const bool gfirst = wg == 0;  // registers the expected bytes and waits for them
    const uint32_t s_bytes = static_cast<uint32_t>(gq) * QK;  // from all four partner warps
    const int ngroups8 = gq / 8;
    int pend = -1;  // a stage whose copy into this CTA was expected, not yet waited for
    for (int s = grp; s < nsteps; s += C::NGROUPS) {
      const int so = s % C::NSO;
      // both pairs' MMAs have read what this CTA wrote into slot `so` (here
      // and in its partner) last time
      bool ok = s < C::NSO || mbar_wait(empty_o(so), ((s / C::NSO) & 1) ^ 1, ab, 0x43, s);
      if (!__all_sync(0xffffffffu, ok)) break;
      uint8_t* sdst = smem + C::OFF_S + so * C::OPS;
      if (gfirst) {  // the partner's half of this CTA's S rows will land here
        if (lane == 0) mbar_arrive_expect_tx(s_recv(so), s_bytes);
        pend = s;
      }
      const int64_t cbase = lbeg + static_cast<int64_t>(s) * QK;  // a multiple of 128
      for (int rg = wg; rg < ngroups8; rg += C::GROUP_WARPS) {
        const uint32_t r8 = static_cast<uint32_t>(gbase + 8 * rg);  // first row of the group
        if (DIST == kRademacher) {
          // a lane: one row (lane % 8) and one quarter of the stage's 128
          // columns (lane / 8); one Philox call covers the row's 128 columns
          const uint32_t r = r8 + (static_cast<uint32_t>(lane) & 7u);
          const uint32_t qc = static_cast<uint32_t>(lane) >> 3;
          const int64_t grow = g0 + r;
          uint4 w = make_uint4(0u, 0u, 0u, 0u);
          int64_t nv = 0;
          if (grow < p.Q && cbase < lend) {
            w = rademacher_bits(p.rk, static_cast<uint32_t>(grow),
                                static_cast<uint32_t>(cbase >> 7), 0u);
            nv = min(lend - cbase, static_cast<int64_t>(QK));
          }
          const uint32_t word = qc == 0 ? w.x : qc == 1 ? w.y : qc == 2 ? w.z : w.w;
#pragma unroll
          for (int b2 = 0; b2 < 2; ++b2) {  // the quarter's two 16-column blocks
            const uint32_t bits = word >> (16 * b2);
            const int b = 2 * static_cast<int>(qc) + b2;
            uint32_t q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              q[u] = rad4_e4m3(bits >> (4 * u));
              const int64_t c = 16 * b + 4 * u;  // columns past the split are zero
              if (c + 4 > nv) {
                uint32_t keep = 0u;
                for (int e = 0; e < 4; ++e)
                  if (c + e < nv) keep |= 0xFFu << (8 * e);
                q[u] &= keep;
              }
            }
            *reinterpret_cast<uint4*>(sdst + q8_off(r, 16u * b)) =
                make_uint4(q[0], q[1], q[2], q[3]);
          }
        } else {
          // 256 tasks of 4 entries: lane l takes row l / 4 and quad l % 4 of
          // each of the 8 16-column blocks (a warp's 4-byte stores of a block
          // fill its 128 contiguous bytes)
          const uint32_t r = r8 + (static_cast<uint32_t>(lane) >> 2);
          const int64_t grow = g0 + r;
#pragma unroll 2
          for (int b = 0; b < 8; ++b) {
            const uint32_t c = static_cast<uint32_t>(b) * 16u + (static_cast<uint32_t>(lane) & 3u) * 4u;
            const int64_t cc = cbase + c;
            uint32_t q = 0u;
            if (grow < p.Q && cc < lend) {
              const float4 a = DIST == kUniform
                                   ? uniform4(p.rk, static_cast<uint32_t>(grow),
                                              static_cast<uint32_t>(cc >> 2), 0u)
                                   : gaussian4(p.rk, static_cast<uint32_t>(grow),
                                               static_cast<uint32_t>(cc >> 2), 0u);
              q = e4m3x4(a);
            }
            *reinterpret_cast<uint32_t*>(sdst + q8_off(r, c)) = q;
          }
        }
        // the group's rows are written: copy them into the partner (async
        // proxy, completing on its s_recv barrier)
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0)
          bulk_copy_to_cluster(partner_s + static_cast<uint32_t>(so) * C::OPS + r8 * 128u,
                               smem_u32(sdst) + r8 * 128u, 1024u, partner_s_recv + 8u * so);
      }
      ok = mbar_wait(full_a(so), (s / C::NSO) & 1, ab, 0x40, s);
      if (!__all_sync(0xffffffffu, ok)) break;
      // this CTA's own rows are fenced above; the group's first warp
      // certifies the partner's rows too
      ok = !gfirst || mbar_wait(s_recv(so), (s / C::NSO) & 1, ab, 0x46, s);
      if (!__all_sync(0xffffffffu, ok)) break;
      pend = -1;
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_full_o + 8u * so);
    }
    // leaving early: let a copy the partner may still be sending land first
    if (gfirst && pend >= 0 && lane == 0)
      drain_wait(s_recv(pend % C::NSO), (pend / C::NSO) & 1, 100000000ull);
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

// Row exponent of a row with max |a| = amax: the smallest e with
// amax <= 448 * 2^e (0 for a zero row or one holding Inf).  448 = 1.75 * 2^8,
// so from ilogb(amax) - 8 at most one step is needed either way.
__device__ __forceinline__ int e4m3_row_exponent(float amax) {
  int e = 0;
  if (amax > 0.0f && amax <= 3.4028235e38f) {
    e = ilogbf(amax) - 8;
    for (int it = 0; it < 4 && ldexpf(amax, -e) > 448.0f; ++it) ++e;
    for (int it = 0; it < 4 && ldexpf(amax, 1 - e) <= 448.0f; ++it) --e;
  }
  return e;
}

// Quantize rows of A holding a whole row in registers: one 256-thread block
// per row, VPT float4 per thread (n <= 1024 * VPT), rows 16-byte aligned; one
// read of A, codes written once.
template <int VPT>
__global__ void __launch_bounds__(256)
    k_quantize_rows_e4m3_regs(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                              uint8_t* __restrict__ Aq, int64_t ldq, int32_t* __restrict__ exps) {
  __shared__ float wmax[8];
  const int tid = threadIdx.x;
  const int64_t nv = n / 4;  // whole float4 groups; the tail (n % 4) is read per element
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
    const float* a = A + r * lda;
    float4 v[VPT];
    float amax = 0.0f;
#pragma unroll
    for (int i = 0; i < VPT; ++i) {
      const int64_t g = tid + 256 * i;  // float4 index
      if (g < nv) {
        v[i] = __ldcs(reinterpret_cast<const float4*>(a) + g);
      } else {
        v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t c = 4 * g;
        if (c < n) {  // the ragged tail
          v[i].x = a[c];
          if (c + 1 < n) v[i].y = a[c + 1];
          if (c + 2 < n) v[i].z = a[c + 2];
        }
      }
      amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[i].x), fabsf(v[i].y)),
                               fmaxf(fabsf(v[i].z), fabsf(v[i].w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) wmax[tid >> 5] = amax;
    __syncthreads();
    amax = wmax[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) amax = fmaxf(amax, wmax[w]);
    __syncthreads();  // wmax is rewritten by the next row
    const int e = e4m3_row_exponent(amax);
    if (tid == 0) exps[r] = e;
    uint32_t* q = reinterpret_cast<uint32_t*>(Aq + r * ldq);
#pragma unroll
    for (int i = 0; i < VPT; ++i) {
      const int64_t g = tid + 256 * i;
      if (4 * g < ldq)
        q[g] = e4m3x4(make_float4(ldexpf(v[i].x, -e), ldexpf(v[i].y, -e), ldexpf(v[i].z, -e),
                                  ldexpf(v[i].w, -e)));
    }
  }
}

// Quantize rows of A: one warp per row finds max |a| (exact), the row
// exponent e (the smallest with max |a| <= 448 * 2^e) and writes the codes
// RNE_e4m3(a * 2^-e), zero-padded to ldq columns.  VEC: rows 16-byte aligned.
template <bool VEC>
__global__ void __launch_bounds__(256)
    k_quantize_rows_e4m3(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                         uint8_t* __restrict__ Aq, int64_t ldq, int32_t* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * 8;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); r < m;
       r += warps) {
    const float* a = A + r * lda;
    float amax = 0.0f;
    if (VEC) {
      int64_t c = 4 * lane;
      for (; c + 4 <= n; c += 128) {
        const float4 v = *reinterpret_cast<const float4*>(a + c);
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
      for (int64_t t = n / 4 * 4 + lane; t < n; t += 32) amax = fmaxf(amax, fabsf(a[t]));
    } else {
      for (int64_t c = lane; c < n; c += 32) amax = fmaxf(amax, fabsf(a[c]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const int e = e4m3_row_exponent(amax);
    if (lane == 0) exps[r] = e;
    uint8_t* q = Aq + r * ldq;
    for (int64_t c = 16 * lane; c < ldq; c += 512) {  // 16 codes per lane
      float x[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) x[u] = c + u < n ? ldexpf(a[c + u], -e) : 0.0f;
      uint32_t w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        w[u] = e4m3x4(make_float4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]));
      *reinterpret_cast<uint4*>(q + c) = make_uint4(w[0], w[1], w[2], w[3]);
    }
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

template <int DIST, bool PAIR, bool NARROW = false, bool EC = false>
cudaError_t set_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_sketch_bf16x2_left<DIST, PAIR, NARROW, EC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg<PAIR, NARROW>::SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

// cluster_x: CTAs per cluster along x (a CTA pair must be adjacent in x; the
// BF16 right sketch runs clusters of two pairs)
template <bool PAIR>
void fill_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr, dim3 grid, cudaStream_t st,
                 unsigned cluster_x = PAIR ? 2 : 1) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = grid;
  cfg->blockDim = dim3(NTHREADS, 1, 1);
  cfg->dynamicSmemBytes = Cfg<PAIR>::SMEM;
  cfg->stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster_x;
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
                int box_cols, int box_rows,
                CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_NONE) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return false;
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstride,
             box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Geometry of one left problem.
struct LeftPlan {
  bool pair;
  int nt;
  int64_t tiles_p, tiles_q;  // tiles_p counts pair tiles (256 rows) when pair
  int splits;
  int64_t chunk;
  int64_t steps;             // stages of one item
};

// max_nt: the widest output tile (512 columns, two MMA instructions per K
// step; or 256, one instruction, more tiles along n).
LeftPlan left_geometry(const GemmShape& s, bool pair, int max_nt = NT_MAX) {
  LeftPlan pl;
  pl.pair = pair;
  // every CTA holds whole 64-column chunks of the split A
  const int64_t gran = pair ? 2 * HCHUNK : HCHUNK;
  pl.nt = s.Q > 256 && max_nt > 256 ? 512 : static_cast<int>(std::min<int64_t>((s.Q + gran - 1) / gran * gran, 256));
  pl.tiles_q = (s.Q + pl.nt - 1) / pl.nt;
  pl.tiles_p = (s.P + (pair ? 2 * BM : BM) - 1) / (pair ? 2 * BM : BM);
  pl.splits = 1;
  pl.chunk = (s.L + LK - 1) / LK * LK;
  pl.steps = pl.chunk / LK;
  return pl;
}

void set_splits(LeftPlan* pl, const GemmShape& s, int64_t splits) {
  if (splits < 1) splits = 1;
  int64_t chunk = (s.L + splits - 1) / splits;
  chunk = (chunk + LK - 1) / LK * LK;
  pl->chunk = chunk;
  pl->splits = static_cast<int>((s.L + chunk - 1) / chunk);
  pl->steps = chunk / LK;
}

// A single sketch: pairs when the output has at least two 128-row tiles;
// splits that fill whole waves of the resident units.
LeftPlan plan_left(const GemmShape& s) {
  const int64_t tp = (s.P + BM - 1) / BM;
  const int64_t ps = tp >= 2 ? pair_slots() : -1;
  LeftPlan pl = left_geometry(s, ps > 0);
  const int64_t units = pl.pair ? ps / 2 : num_sms_tc();
  const int64_t tiles = pl.tiles_p * pl.tiles_q;
  const int64_t steps_total = (s.L + LK - 1) / LK;
  int64_t smax = steps_total / 4;  // at least 128 rows per split
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

// Whether a problem on pairs splits its FP32 A inside the sketch kernel.
// Rademacher: always (the workers do it; their sign bits leave them idle).
// Gaussian and uniform: the epilogue warps do it, once per 256-row pair tile
// of k that reads the A tile, while the split pass splits it once; on the
// 2^20 x 512, k = 2048 sketch (8 pair tiles) the in-kernel split cost 0.9 ms
// of issue slots against the split pass's 0.65 ms, so only problems with at
// most 4 pair tiles of k (k <= 1024) split A in the kernel.
constexpr int64_t kInlineSplitMaxTiles = 4;
bool inline_split(int dist, const LeftPlan& pl) {
  return pl.pair && (dist == kRademacher || pl.tiles_p <= kInlineSplitMaxTiles);
}

// Split pass of one sketch (A rows 16-byte aligned, lda a multiple of 4).
cudaError_t split_launch_one(const float* A, int64_t lda, int64_t m, int64_t n, void* H,
                             cudaStream_t st) {
  SplitDesc d;
  d.A = A;
  d.lda = lda;
  d.H = static_cast<__nv_bfloat16*>(H);
  d.ldh = (n + HCHUNK - 1) / HCHUNK * HCHUNK;
  d.part = m * d.ldh;
  d.m = m;
  d.n = n;
  const int64_t total = m * (d.ldh / 8);
  const int64_t blocks = std::min<int64_t>((total + 255) / 256,
                                           static_cast<int64_t>(num_sms_tc()) * 16);
  k_split_bf16x2_one<<<static_cast<unsigned>(blocks), 256, 0, st>>>(d);
  count_launches(1);
  return cudaGetLastError();
}

// Host image of a work list: problems (128-byte aligned), items, per-unit
// begin offsets, packed into one buffer for a single upload.
struct HostSched {
  std::vector<LeftProblem> probs;
  std::vector<LeftItem> items;
  int64_t units = 0;  // pairs (or CTAs) to launch
  size_t off_items = 0, off_claim = 0, bytes = 0;
  std::vector<uint8_t> blob;
};

// Items of every problem, longest (estimated) first; the kernel hands them
// out in this order to whichever pair is free.  A stage costs about its
// output columns plus a fixed 256 (generation, barriers), plus 640 for
// Gaussian and uniform S (Box-Muller); launches use at most `max_units`
// pairs (or CTAs).
void build_items(const std::vector<LeftPlan>& plans, const std::vector<int>& dists,
                 int64_t max_units, HostSched* hs) {
  struct Cand {
    LeftItem it;
    double cost;
  };
  std::vector<Cand> cands;
  for (size_t pi = 0; pi < plans.size(); ++pi) {
    const LeftPlan& pl = plans[pi];
    const double gen = dists[pi] == kRademacher ? 0.0 : 640.0;
    const double cost = static_cast<double>(pl.steps) * (static_cast<double>(pl.nt) + 256.0 + gen);
    for (int64_t z = 0; z < pl.splits; ++z)
      for (int64_t tq = 0; tq < pl.tiles_q; ++tq)
        for (int64_t tp = 0; tp < pl.tiles_p; ++tp)
          cands.push_back({{static_cast<int>(pi), static_cast<int>(tp), static_cast<int>(tq),
                            static_cast<int>(z)},
                           cost});
  }
  std::stable_sort(cands.begin(), cands.end(),
                   [](const Cand& a, const Cand& b) { return a.cost > b.cost; });
  hs->items.clear();
  for (const Cand& c : cands) hs->items.push_back(c.it);
  hs->units = std::max<int64_t>(1, std::min<int64_t>(max_units, cands.size()));
}

void pack_sched(HostSched* hs) {
  const size_t pb = hs->probs.size() * sizeof(LeftProblem);
  hs->off_items = (pb + 255) / 256 * 256;
  const size_t ib = hs->items.size() * sizeof(LeftItem);
  hs->off_claim = (hs->off_items + ib + 255) / 256 * 256;
  hs->bytes = hs->off_claim + 256;
  hs->blob.assign(hs->bytes, 0);
  memcpy(hs->blob.data(), hs->probs.data(), pb);
  memcpy(hs->blob.data() + hs->off_items, hs->items.data(), ib);
}

LeftSched device_sched(const HostSched& hs, void* dbuf, int* status,
                       uint64_t timeout_ns = kDefaultWaitLimitNs, long long stall_stage = -1) {
  LeftSched sc;
  uint8_t* b = static_cast<uint8_t*>(dbuf);
  sc.probs = reinterpret_cast<const LeftProblem*>(b);
  sc.items = reinterpret_cast<const LeftItem*>(b + hs.off_items);
  sc.claim = reinterpret_cast<int*>(b + hs.off_claim);
  sc.nitems = static_cast<int>(hs.items.size());
  sc.status = status;
  sc.timeout_ns = timeout_ns;
  sc.stall_stage = stall_stage;
  sc.rk = round_keys(hs.probs.empty() ? PhiloxKey{0u, 0u} : hs.probs[0].key);
  return sc;
}

template <int DIST, bool PAIR, bool NARROW = false, bool EC = false>
cudaError_t launch_left(const LeftSched& sc, int64_t units, cudaStream_t st) {
  cudaError_t e = set_smem_attr<DIST, PAIR, NARROW, EC>();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(sc.claim, 0, sizeof(int), st);  // the work list starts unclaimed
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<PAIR>(&cfg, attr, dim3(static_cast<unsigned>(units * (PAIR ? 2 : 1)), 1, 1), st);
  cfg.dynamicSmemBytes = Cfg<PAIR, NARROW>::SMEM;
  return cudaLaunchKernelEx(&cfg, k_sketch_bf16x2_left<DIST, PAIR, NARROW, EC>, sc);
}

// ec: Gaussian or uniform sketch on pairs whose A the epilogue warps split
template <bool PAIR>
cudaError_t launch_left_dist(int dist, const LeftSched& sc, int64_t units, cudaStream_t st,
                             bool ec = false) {
  if (dist == kStored) return launch_left<kStored, PAIR>(sc, units, st);
  if (dist == kRademacher) return launch_left<kRademacher, PAIR>(sc, units, st);
  if (dist == kUniform)
    return ec ? launch_left<kUniform, PAIR, false, PAIR>(sc, units, st)
              : launch_left<kUniform, PAIR>(sc, units, st);
  return ec ? launch_left<kGaussian, PAIR, false, PAIR>(sc, units, st)
            : launch_left<kGaussian, PAIR>(sc, units, st);
}

// The split A of an m x n problem as a 4D tensor {64 columns, m rows,
// 64-column chunks, hi/lo}; one box = `cols` columns of 16 rows of both.
bool encode_split_map(CUtensorMap* map, const void* H, int64_t m, int64_t n, int cols) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return false;
  const int64_t ldh = split_ld(n);
  const cuuint64_t gdim[4] = {static_cast<cuuint64_t>(HCHUNK), static_cast<cuuint64_t>(m),
                              static_cast<cuuint64_t>(ldh / HCHUNK), 2};
  const cuuint64_t gstride[3] = {static_cast<cuuint64_t>(ldh) * 2, HCHUNK * 2,
                                 static_cast<cuuint64_t>(m) * static_cast<cuuint64_t>(ldh) * 2};
  const cuuint32_t box[4] = {static_cast<cuuint32_t>(HCHUNK), static_cast<cuuint32_t>(LK),
                             static_cast<cuuint32_t>(cols / HCHUNK), 2};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(H), gdim, gstride, box,
             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A caller-stored BF16 S[k x m] (row stride lds elements) as a 5D tensor
// {8 columns, row % 8, 8-column half of a 16-column slab, row / 8, slab}: one
// box {8, 8, 2, 16, 2} is the S tile of a stage (128 rows x 32 columns) in
// the kernel's K-major no-swizzle operand layout.  k % 8 == 0; rows of S
// beyond k are outside the tensor (zeros); lds >= m rounded up to 16.
bool encode_stored_map(CUtensorMap* map, const void* S, int64_t k, int64_t m, int64_t lds) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return false;
  const cuuint64_t gdim[5] = {8, 8, 2, static_cast<cuuint64_t>(k / 8),
                              static_cast<cuuint64_t>((m + 15) / 16)};
  const cuuint64_t row = static_cast<cuuint64_t>(lds) * 2;
  const cuuint64_t gstride[4] = {row, 16, 8 * row, 32};
  const cuuint32_t box[5] = {8, 8, 2, static_cast<cuuint32_t>(BM / 8), LK / 16};
  const cuuint32_t estride[5] = {1, 1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(S), gdim, gstride, box,
             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Stages per accumulation chain of the left sketch.  The error of the split-A
// product grows linearly with the chain length (full C2 size, chains of
// 2048 / 4096 rows: Rademacher 3.5e-6 / 5.5e-6, Gaussian 5.1e-6 / 9.5e-6), so
// Rademacher sketches drain the accumulator half as often as the others.
int left_chain_stages(int dist) { return dist == kRademacher ? 2 * CHAIN_L : CHAIN_L; }

// FP32 A[m x n] (row stride lda) for the in-place split, as 32-column blocks
// [32 rows][32 floats] with the 128-byte swizzle in shared memory; rows past
// m read as zeros.  With n a multiple of 32, a 3D tensor {32 columns, m rows,
// n / 32 blocks} whose one box holds all `cols` columns of a CTA (blocks past
// n read as zeros); otherwise a 2D tensor {n, m} with one 32 x 32 box per
// block (columns past n read as zeros: a 3D box would read the start of the
// next row there).  One box per stage is the faster (C2 Rademacher 2.60 ms
// against 2.82 ms with 8 boxes).  The TMA needs A 16-byte aligned and lda a
// multiple of 4 (fp32_map_ok).  Returns the conv_inline mode, 0 on failure.
bool fp32_map_ok(const float* A, int64_t lda) {
  return reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % 4 == 0;
}
int encode_fp32_map(CUtensorMap* map, const float* A, int64_t m, int64_t n, int64_t lda,
                    int cols) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return 0;
  if (n % 32 == 0) {
    const cuuint64_t gdim[3] = {32, static_cast<cuuint64_t>(m), static_cast<cuuint64_t>(n / 32)};
    const cuuint64_t gstride[2] = {static_cast<cuuint64_t>(lda) * 4, 128};
    const cuuint32_t box[3] = {32, static_cast<cuuint32_t>(LK), static_cast<cuuint32_t>(cols / 32)};
    const cuuint32_t estride[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(A), gdim, gstride,
               box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS ? 1 : 0;
  }
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(m)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(lda) * 4};
  const cuuint32_t box[2] = {32, static_cast<cuuint32_t>(LK)};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim, gstride, box,
             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS ? 2 : 0;
}

// The FP32 partials [splits][P][ldp] as a 3D tensor {Q, P, splits} with boxes
// of 32 columns x 32 rows and the 128-byte swizzle, for the epilogue's TMA
// drain (drain_chain_tma); false when the rows are not 16-byte multiples or
// the base not 16-byte aligned (the epilogue then writes with red.add).
bool encode_part_map(CUtensorMap* map, const float* part, int64_t P, int64_t Q, int64_t ldp,
                     int splits) {
  if (ldp % 4 != 0 || reinterpret_cast<uintptr_t>(part) % 16 != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return false;
  const cuuint64_t gdim[3] = {static_cast<cuuint64_t>(Q), static_cast<cuuint64_t>(P),
                              static_cast<cuuint64_t>(splits)};
  const cuuint64_t gstride[2] = {static_cast<cuuint64_t>(ldp) * 4,
                                 static_cast<cuuint64_t>(P) * static_cast<cuuint64_t>(ldp) * 4};
  const cuuint32_t box[3] = {32, 32, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(part), gdim, gstride,
             box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A_inline: FP32 A (row stride lda) that the kernel splits in place instead
// of reading the split pass's halves from H (problems on CTA pairs whose A
// passes fp32_map_ok), or null.
bool fill_problem(LeftProblem* pr, const LeftPlan& pl, const GemmShape& s, const void* H,
                  float* part, uint64_t seed, int dist, const float* A_inline = nullptr,
                  int64_t lda = 0, int64_t ldp = 0) {
  memset(pr, 0, sizeof(*pr));
  if (!encode_split_map(&pr->map, H, s.L, s.Q, pl.pair ? pl.nt / 2 : pl.nt)) return false;
  if (A_inline != nullptr) {
    if (!pl.pair) return false;
    pr->conv_inline = encode_fp32_map(&pr->amap, A_inline, s.L, s.Q, lda, pl.nt / 2);
    if (pr->conv_inline == 0) return false;
  }
  pr->part = part;
  pr->P = s.P;
  pr->Q = s.Q;
  pr->L = s.L;
  pr->chunk = pl.chunk;
  pr->nt = pl.nt;
  pr->dist = dist;
  pr->chain = left_chain_stages(dist);
  pr->key = make_key(seed);
  pr->ldp = ldp > 0 ? ldp : s.Q;
  pr->tma_drain = encode_part_map(&pr->pmap, part, s.P, s.Q, pr->ldp, pl.splits) ? 1 : 0;
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

// CTAs of the BF16 right kernel that can be resident at once in clusters of
// two pairs (a cluster must fit in one GPC), or -1.
int64_t quad_slots();

// Right sketch: pairs of CTAs own 512 rows of m and nq <= 256 rows of k,
// `cluster` CTAs (two pairs for the BF16 kernel, one for FP8) are adjacent in
// x; the split count keeps the partials (splits x m x k floats) to a few
// hundred MB.
Plan plan_right(const GemmShape& s, int cluster = 4) {
  Plan pl;
  // k rows per pair tile: a multiple of 32, so that each CTA of a pair holds
  // whole 8-row groups of S in each half it generates and receives
  pl.nt = s.Q > 256 ? 256 : static_cast<int>((s.Q + 31) / 32 * 32);
  pl.tmem_cols = 32;
  while (pl.tmem_cols < 2 * pl.nt) pl.tmem_cols *= 2;
  const int64_t rows = static_cast<int64_t>(cluster) * CfgR::ROWS;  // rows of m per cluster
  pl.tiles_p = (s.P + rows - 1) / rows * cluster;                  // CTAs along m
  pl.tiles_q = (s.Q + pl.nt - 1) / pl.nt;
  int64_t slots = cluster == 4 ? quad_slots() : pair_slots();
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

// FP8 right sketch: the same tiling as the BF16 right sketch (clusters of
// two CTA pairs sharing each generated S tile), splits of whole 128-column
// stages.
Plan plan_right_q(const GemmShape& s) {
  Plan pl = plan_right(s, 4);
  int64_t chunk = (s.L + pl.splits - 1) / pl.splits;
  chunk = (chunk + QK - 1) / QK * QK;
  pl.chunk = chunk;
  pl.splits = static_cast<int>((s.L + chunk - 1) / chunk);
  return pl;
}

cudaError_t set_smem_attr_right_q() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_sketch_e4m3_right<kGaussian>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, CfgQ::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sketch_e4m3_right<kRademacher>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, CfgQ::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sketch_e4m3_right<kUniform>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, CfgQ::SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int DIST>
cudaError_t launch_right_q(const CUtensorMap& map, const TcRightQParams& p, dim3 grid,
                           cudaStream_t st) {
  cudaError_t e = set_smem_attr_right_q();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<true>(&cfg, attr, grid, st, 4);
  cfg.dynamicSmemBytes = CfgQ::SMEM;
  return cudaLaunchKernelEx(&cfg, k_sketch_e4m3_right<DIST>, map, p);
}

// A_q[m x n] (row stride ldq bytes) as a 2D byte tensor; one box = 128 bytes
// of 256 rows, 128-byte swizzle (the K-major operand layout of the kernel).
bool encode_q8_map(CUtensorMap* map, const uint8_t* Aq, int64_t m, int64_t n, int64_t ldq) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) return false;
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(m)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ldq)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(QK), static_cast<cuuint32_t>(CfgQ::ROWS)};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(Aq), gdim, gstride, box,
             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t quad_slots() {
  static int64_t cache = 0;
  if (cache != 0) return cache;
  if (set_smem_attr_right() != cudaSuccess) return cache = -1;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<true>(&cfg, attr, dim3(4, 1, 1), nullptr, 4);
  cfg.dynamicSmemBytes = CfgR::SMEM;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_sketch_bf16x2_right<kGaussian>, &cfg) !=
          cudaSuccess ||
      clusters <= 0) {
    cudaGetLastError();
    return cache = -1;
  }
  return cache = static_cast<int64_t>(clusters) * 4;
}

template <int DIST>
cudaError_t launch_right(const CUtensorMap& map, const CUtensorMap& pmap, const TcRightParams& p,
                         dim3 grid, cudaStream_t st) {
  cudaError_t e = set_smem_attr_right();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config<true>(&cfg, attr, grid, st, 4);
  cfg.dynamicSmemBytes = CfgR::SMEM;
  return cudaLaunchKernelEx(&cfg, k_sketch_bf16x2_right<DIST>, map, pmap, p);
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

int64_t split_ld(int64_t n) { return (n + HCHUNK - 1) / HCHUNK * HCHUNK; }

size_t split_bytes(int64_t m, int64_t n) {
  return (static_cast<size_t>(m) * static_cast<size_t>(split_ld(n)) * 4 + 255) / 256 * 256;
}

cudaError_t split_rows(const float* A, int64_t lds, int64_t m, int64_t n, void* H,
                       cudaStream_t st) {
  SplitDesc d;
  d.A = A;
  d.lda = lds;
  d.H = static_cast<__nv_bfloat16*>(H);
  d.ldh = split_ld(n);
  d.part = m * d.ldh;
  d.m = m;
  d.n = n;
  const int64_t rows_per_block = 256 / 32;
  const int64_t blocks = std::min<int64_t>((m + rows_per_block - 1) / rows_per_block,
                                           static_cast<int64_t>(num_sms_tc()) * 8);
  k_split_rows<<<static_cast<unsigned>(blocks), 256, 0, st>>>(d);
  count_launches(1);
  return cudaGetLastError();
}

// Segments of the persistent BF16 right kernel: blocks of 1024 rows of m x
// a pair tile of k rows, each `steps` stages of n long, laid end to end and
// shared equally by the `ncl` resident clusters of two CTA pairs; zmax is the
// most segments any block is cut into, the number of partials the sketch
// needs (2 for the 65536 x 16384, k = 256 sketch on 36 clusters, against 9
// equal splits of n before).
struct RightSegPlan {
  Plan pl;  // tile geometry (nt, tmem_cols, tiles_p, tiles_q)
  int64_t steps, units, ncl;
  int zmax;
};

RightSegPlan plan_right_seg(const GemmShape& s) {
  RightSegPlan r;
  r.pl = plan_right(s);
  r.steps = (s.L + BK - 1) / BK;
  const int64_t blocks = r.pl.tiles_p / 4 * r.pl.tiles_q;
  r.units = blocks * r.steps;
  const int64_t resident = quad_slots() / 4;
  r.ncl = std::max<int64_t>(1, std::min<int64_t>(r.units, resident));
  r.zmax = 1;
  for (int64_t b = 0; b < blocks; ++b) {
    const int64_t z = seg_owner((b + 1) * r.steps - 1, r.units, r.ncl) -
                      seg_owner(b * r.steps, r.units, r.ncl) + 1;
    r.zmax = static_cast<int>(std::max<int64_t>(r.zmax, z));
  }
  return r;
}

// Y = scale x the sum, in segment order, of the partials of each element's
// block (as many as segments the block was cut into).  CUDA block (x, y)
// takes rows y * 1024 + x, + gridDim.x, ... of block row y; a thread keeps
// its columns (and so its blocks' segment counts) for all of them.
__global__ void __launch_bounds__(256)
    k_reduce_segments(const float* __restrict__ part, int64_t P, int64_t Q, int nq, int tiles_q,
                      int64_t steps, int64_t units, int64_t ncl, float scale,
                      float* __restrict__ Y, int64_t ldy) {
  const int64_t total = P * Q;
  const int64_t mblocks = (P + 4 * CfgR::ROWS - 1) / (4 * CfgR::ROWS);
  for (int64_t mb = blockIdx.y; mb < mblocks; mb += gridDim.y) {
    const int64_t r0 = mb * (4 * CfgR::ROWS);
    const int64_t r1 = min(P, r0 + 4 * CfgR::ROWS);
    for (int64_t c = threadIdx.x; c < Q; c += blockDim.x) {
      const int64_t blk = mb * tiles_q + c / nq;
      const int64_t nseg =
          seg_owner((blk + 1) * steps - 1, units, ncl) - seg_owner(blk * steps, units, ncl) + 1;
      for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const int64_t i = r * Q + c;
        float acc = 0.0f;
        for (int64_t z = 0; z < nseg; ++z) acc = __fadd_rn(acc, part[z * total + i]);
        Y[r * ldy + c] = __fmul_rn(scale, acc);
      }
    }
  }
}

size_t tc_workspace_bytes(const GemmShape& s) {
  if (s.left) {
    const LeftPlan pl = plan_left(s);
    return split_bytes(s.L, s.Q) + static_cast<size_t>(pl.splits) * s.P * s.Q * sizeof(float);
  }
  const RightSegPlan rs = plan_right_seg(s);
  return static_cast<size_t>(rs.zmax) * static_cast<size_t>(s.P) * static_cast<size_t>(s.Q) *
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
  const RightSegPlan rs = plan_right_seg(s);
  const Plan& pl = rs.pl;
  CUtensorMap map;
  // A[m x n]: n innermost; one box = 16 columns of n x 256 rows of m, each
  // 64-byte row with the 64-byte swizzle (the in-place split's lane map)
  if (!encode_map(&map, A, s.P, s.L, lda, BK, CfgR::ROWS, CU_TENSOR_MAP_SWIZZLE_64B))
    return cudaErrorInvalidValue;
  TcRightParams p;
  p.P = s.P;
  p.Q = s.Q;
  p.L = s.L;
  p.nq = pl.nt;
  p.tmem_cols = pl.tmem_cols;
  p.rk = round_keys(make_key(h->seed));
  p.status = h->d_status;
  p.timeout_ns = h->wait_limit_ns;
  const size_t need = static_cast<size_t>(rs.zmax) * s.P * s.Q * sizeof(float);
  if (ws == nullptr || ws_bytes < need) return cudaErrorInvalidValue;
  p.part = static_cast<float*>(ws);
  CUtensorMap pmap;
  memset(&pmap, 0, sizeof(pmap));
  p.tma_drain = encode_part_map(&pmap, p.part, s.P, s.Q, s.Q, rs.zmax) ? 1 : 0;
  // persistent clusters of four CTAs, as many as can be resident, each
  // taking an equal contiguous share of the stages
  if (rs.units > (int64_t(1) << 31) - 1) return cudaErrorInvalidValue;  // 32-bit stage numbers
  p.tiles_q = static_cast<int>(pl.tiles_q);
  p.steps = static_cast<int>(rs.steps);
  p.units = static_cast<int>(rs.units);
  dim3 grid(static_cast<unsigned>(4 * rs.ncl), 1, 1);
  prof_mark(h->prof_start, st);
  cudaError_t e;
  if (h->dist == kRademacher)
    e = launch_right<kRademacher>(map, pmap, p, grid, st);
  else if (h->dist == kUniform)
    e = launch_right<kUniform>(map, pmap, p, grid, st);
  else
    e = launch_right<kGaussian>(map, pmap, p, grid, st);
  prof_mark(h->prof_stop, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  const int64_t mblocks = pl.tiles_p / 4;  // blocks of 1024 rows of m
  const int64_t per = std::max<int64_t>(
      1, std::min<int64_t>(4 * CfgR::ROWS,
                           static_cast<int64_t>(num_sms_tc()) * 16 / std::max<int64_t>(1, mblocks)));
  k_reduce_segments<<<dim3(static_cast<unsigned>(per),
                           static_cast<unsigned>(std::min<int64_t>(mblocks, 65535))),
                      256, 0, st>>>(
      static_cast<const float*>(ws), s.P, s.Q, pl.nt, p.tiles_q, rs.steps, rs.units, rs.ncl,
      h->scale, Y, ldy);
  count_launches(1);
  return cudaGetLastError();
}

int64_t q8_ld(int64_t n) { return (n + 15) / 16 * 16; }

cudaError_t q8_quantize(const float* A, int64_t lda, int64_t m, int64_t n, uint8_t* Aq,
                        int64_t ldq, int32_t* exps, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && lda % 4 == 0;
  if (vec && ldq <= 4096 * 4) {  // a row fits in the registers of one block
    const int64_t blocks = std::min<int64_t>(m, static_cast<int64_t>(num_sms_tc()) * 8);
    const unsigned g = static_cast<unsigned>(blocks);
    if (ldq <= 1024)
      k_quantize_rows_e4m3_regs<1><<<g, 256, 0, st>>>(A, lda, m, n, Aq, ldq, exps);
    else if (ldq <= 4096)
      k_quantize_rows_e4m3_regs<4><<<g, 256, 0, st>>>(A, lda, m, n, Aq, ldq, exps);
    else
      k_quantize_rows_e4m3_regs<16><<<g, 256, 0, st>>>(A, lda, m, n, Aq, ldq, exps);
    count_launches(1);
    return cudaGetLastError();
  }
  const int64_t blocks = std::min<int64_t>((m + 7) / 8, static_cast<int64_t>(num_sms_tc()) * 8);
  if (vec)
    k_quantize_rows_e4m3<true><<<static_cast<unsigned>(blocks), 256, 0, st>>>(A, lda, m, n, Aq,
                                                                              ldq, exps);
  else
    k_quantize_rows_e4m3<false><<<static_cast<unsigned>(blocks), 256, 0, st>>>(A, lda, m, n, Aq,
                                                                               ldq, exps);
  count_launches(1);
  return cudaGetLastError();
}

size_t q8_partial_bytes(const GemmShape& s) {
  const Plan pl = plan_right_q(s);
  return static_cast<size_t>(pl.splits) * static_cast<size_t>(s.P) * static_cast<size_t>(s.Q) *
         sizeof(float);
}

size_t q8_workspace_bytes(const GemmShape& s) {
  const size_t codes = (static_cast<size_t>(s.P) * q8_ld(s.L) + 255) / 256 * 256;
  const size_t exps = (static_cast<size_t>(s.P) * 4 + 255) / 256 * 256;
  return codes + exps + q8_partial_bytes(s);
}

cudaError_t q8_sketch_right_quantized(const sk_sketch* h, const GemmShape& s, const uint8_t* Aq,
                                      const int32_t* exps, int64_t ldq, float* Y, int64_t ldy,
                                      void* part, size_t part_bytes, cudaStream_t st) {
  const Plan pl = plan_right_q(s);
  if (part == nullptr || part_bytes < q8_partial_bytes(s)) return cudaErrorInvalidValue;
  CUtensorMap map;
  if (!encode_q8_map(&map, Aq, s.P, s.L, ldq)) return cudaErrorInvalidValue;
  TcRightQParams p;
  p.part = static_cast<float*>(part);
  p.exps = exps;
  p.P = s.P;
  p.Q = s.Q;
  p.L = s.L;
  p.chunk = pl.chunk;
  p.nq = pl.nt;
  p.tmem_cols = pl.tmem_cols;
  p.rk = round_keys(make_key(h->seed));
  p.status = h->d_status;
  p.timeout_ns = h->wait_limit_ns;
  dim3 grid(static_cast<unsigned>(pl.tiles_p), static_cast<unsigned>(pl.tiles_q),
            static_cast<unsigned>(pl.splits));
  prof_mark(h->prof_start, st);
  cudaError_t e;
  if (h->dist == kRademacher)
    e = launch_right_q<kRademacher>(map, p, grid, st);
  else if (h->dist == kUniform)
    e = launch_right_q<kUniform>(map, p, grid, st);
  else
    e = launch_right_q<kGaussian>(map, p, grid, st);
  prof_mark(h->prof_stop, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return splitk_reduce(static_cast<float*>(part), pl.splits, s.P, s.Q, h->scale, Y, ldy, st);
}

cudaError_t q8_sketch_right(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                            float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (ws == nullptr || ws_bytes < q8_workspace_bytes(s)) return cudaErrorInvalidValue;
  const int64_t ldq = q8_ld(s.L);
  uint8_t* w = static_cast<uint8_t*>(ws);
  uint8_t* Aq = w;
  const size_t codes = (static_cast<size_t>(s.P) * ldq + 255) / 256 * 256;
  int32_t* exps = reinterpret_cast<int32_t*>(w + codes);
  const size_t eb = (static_cast<size_t>(s.P) * 4 + 255) / 256 * 256;
  cudaError_t e = q8_quantize(A, lda, s.P, s.L, Aq, ldq, exps, st);
  if (e != cudaSuccess) return e;
  return q8_sketch_right_quantized(h, s, Aq, exps, ldq, Y, ldy, w + codes + eb,
                                   ws_bytes - codes - eb, st);
}

namespace {

// The BF16 left sketch: split pass, then the persistent kernel generating S
// (S_stored null) or reading the caller's BF16 S (row stride lds).
cudaError_t tc_sketch_left(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                           float* Y, int64_t ldy, void* ws, size_t ws_bytes, const void* S_stored,
                           int64_t lds, cudaStream_t st) {
  const LeftPlan pl = plan_left(s);
  const size_t sb = split_bytes(s.L, s.Q);
  const size_t need = sb + static_cast<size_t>(pl.splits) * s.P * s.Q * sizeof(float);
  if (ws == nullptr || ws_bytes < need) return cudaErrorInvalidValue;
  void* H = ws;
  float* part = reinterpret_cast<float*>(static_cast<uint8_t*>(ws) + sb);
  sk_sketch* hm = const_cast<sk_sketch*>(h);
  // The work list depends only on these; upload it again only when they change.
  const uint64_t key[9] = {reinterpret_cast<uint64_t>(A), static_cast<uint64_t>(s.L),
                           static_cast<uint64_t>(s.Q), static_cast<uint64_t>(lda),
                           reinterpret_cast<uint64_t>(ws), h->seed,
                           static_cast<uint64_t>(h->dist) | (static_cast<uint64_t>(h->k) << 8),
                           reinterpret_cast<uint64_t>(S_stored), static_cast<uint64_t>(lds)};
  const int64_t units = pl.pair ? pair_slots() / 2 : num_sms_tc();
  HostSched hs;
  hs.probs.resize(1);
  // Pair sketches split A inside the kernel where inline_split says so;
  // single CTAs and the stored-S mode read the halves the split pass writes
  const bool conv = S_stored == nullptr && inline_split(h->dist, pl) && fp32_map_ok(A, lda);
  if (!fill_problem(&hs.probs[0], pl, s, H, part, h->seed, h->dist, conv ? A : nullptr, lda))
    return cudaErrorInvalidValue;
  if (S_stored && !encode_stored_map(&hs.probs[0].smap, S_stored, s.P, s.L, lds))
    return cudaErrorInvalidValue;
  build_items(std::vector<LeftPlan>{pl}, std::vector<int>{h->dist}, units, &hs);
  pack_sched(&hs);
  if (memcmp(key, hm->sched_key, sizeof(key)) != 0 || hm->d_sched_bytes < hs.bytes) {
    cudaError_t e = grow_device(&hm->d_sched, &hm->d_sched_bytes, hs.bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(hm->d_sched, hs.blob.data(), hs.bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    memcpy(hm->sched_key, key, sizeof(key));
  }
  const LeftSched sc = device_sched(hs, hm->d_sched, h->d_status, h->wait_limit_ns,
                                    h->stall_stage);
  const int64_t nunits = hs.units;
  // the measurement hook brackets both passes: split of A (unless the kernel
  // splits it), then the sketch
  prof_mark(h->prof_start, st);
  cudaError_t e = conv ? cudaSuccess : split_launch_one(A, lda, s.L, s.Q, H, st);
  if (e != cudaSuccess) return e;
  const int mode = S_stored ? kStored : h->dist;
  e = pl.pair ? launch_left_dist<true>(mode, sc, nunits, st, conv && h->dist != kRademacher)
              : launch_left_dist<false>(mode, sc, nunits, st);
  prof_mark(h->prof_stop, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  // fixed-order sum of the split partials, times 1/sqrt(k), into Y
  return splitk_reduce(part, pl.splits, s.P, s.Q, h->scale, Y, ldy, st);
}

}  // namespace

cudaError_t tc_sketch(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                      float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!s.left) return tc_sketch_right(h, s, A, lda, Y, ldy, ws, ws_bytes, st);
  return tc_sketch_left(h, s, A, lda, Y, ldy, ws, ws_bytes, nullptr, 0, st);
}

cudaError_t tc_sketch_left_stored(const sk_sketch* h, const GemmShape& s, const void* S,
                                  int64_t lds, const float* A, int64_t lda, float* Y,
                                  int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st) {
  return tc_sketch_left(h, s, A, lda, Y, ldy, ws, ws_bytes, S, lds, st);
}

struct PlannedBatch {
  HostSched hs;
  std::vector<ReduceDesc> red;
  std::vector<SplitDesc> splits;   // members whose split pass runs in this batch
  std::vector<int64_t> prefix;     // groups of 8 columns before each of them
  size_t off_red = 0, off_split = 0, off_prefix = 0, bytes = 0;
  size_t ws_bytes = 0;             // arena workspace the members need
  int64_t max_elems = 0;
  int64_t units = 0;
  int launches = 0;                // kernels of one run: split (if any), sketch, reduce
  bool narrow = false;             // launched with the 8-stage narrow ring
  bool econv = false;              // the epilogue warps split some member's A
};

LeftPlan member_plan(const BatchMember& mb, const BatchShape& bs, GemmShape* shape) {
  const int64_t item_stages = mb.item_stages > 0 ? mb.item_stages : bs.item_stages;
  GemmShape s;
  s.left = true;
  s.P = mb.k;
  s.Q = mb.n;
  s.L = mb.m;
  LeftPlan pl = left_geometry(s, true, bs.max_nt);
  const int64_t rows16 = (s.L + 15) / 16;  // item lengths count 16-row units
  set_splits(&pl, s, (rows16 + item_stages - 1) / item_stages);
  if (shape) *shape = s;
  return pl;
}

// Batch members keep their partials in rows of a multiple of 4 columns, so
// that every member drains through the TMA.
int64_t member_ldp(int64_t n) { return (n + 3) / 4 * 4; }

size_t partial_bytes(const LeftPlan& pl, const GemmShape& s) {
  return (static_cast<size_t>(pl.splits) * s.P * member_ldp(s.Q) * sizeof(float) + 255) / 256 *
         256;
}

// Work list of a batch whose arena workspace starts at `arena`; with `arena`
// null only the arena size (`ws_bytes`) is computed.  A member's workspace
// holds its BF16 split of A (split_bytes), then its partials.
bool plan_members(const BatchMember* mbs, size_t count, const BatchShape& bs, uint8_t* arena,
                  PlannedBatch* pb) {
  std::vector<LeftPlan> plans;
  std::vector<GemmShape> shapes;
  std::vector<size_t> ws_off;
  size_t total = 0;
  pb->narrow = bs.narrow;
  for (size_t i = 0; i < count; ++i) {
    GemmShape s;
    plans.push_back(member_plan(mbs[i], bs, &s));
    if (plans.back().nt > 256) pb->narrow = false;  // a wide tile needs the wide ring
    shapes.push_back(s);
    ws_off.push_back(total);  // 256-byte aligned: partials take 16-byte vector stores
    if (mbs[i].ws == nullptr) total += split_bytes(s.L, s.Q) + partial_bytes(plans.back(), s);
  }
  pb->ws_bytes = total;
  if (arena == nullptr) return true;  // sizing pass
  pb->hs = HostSched();
  pb->hs.probs.resize(count);
  pb->econv = false;
  pb->red.clear();
  pb->splits.clear();
  pb->prefix.assign(1, 0);
  pb->max_elems = 0;
  for (size_t i = 0; i < count; ++i) {
    const BatchMember& mb = mbs[i];
    uint8_t* w = mb.ws ? static_cast<uint8_t*>(mb.ws) : arena + ws_off[i];
    float* part = reinterpret_cast<float*>(w + split_bytes(mb.m, mb.n));
    // members split A inside the sketch kernel where inline_split says so
    // (Rademacher: the workers; Gaussian and uniform: the epilogue warps); the
    // others (and members whose split is already made) read the halves
    const bool conv = !mb.split_ready && inline_split(mb.dist, plans[i]) &&
                      fp32_map_ok(mb.A, mb.lda);
    if (conv && mb.dist != kRademacher) pb->econv = true;
    if (!fill_problem(&pb->hs.probs[i], plans[i], shapes[i], w, part, mb.seed, mb.dist,
                      conv ? mb.A : nullptr, mb.lda, member_ldp(mb.n)))
      return false;
    if (!mb.split_ready && !conv) {
      SplitDesc d;
      d.A = mb.A;
      d.lda = mb.lda;
      d.H = reinterpret_cast<__nv_bfloat16*>(w);
      d.ldh = split_ld(mb.n);
      d.part = mb.m * d.ldh;
      d.m = mb.m;
      d.n = mb.n;
      pb->splits.push_back(d);
      pb->prefix.push_back(pb->prefix.back() + d.m * (d.ldh / 8));
    }
    ReduceDesc r;
    r.part = part;
    r.Y = mb.Y;
    r.P = mb.k;
    r.Q = mb.n;
    r.ldp = member_ldp(mb.n);
    r.ldy = mb.ldy;
    r.splits = plans[i].splits;
    r.scale = mb.scale;
    pb->red.push_back(r);
    pb->max_elems = std::max<int64_t>(pb->max_elems, mb.k * mb.n);
  }
  const int64_t slots = pair_slots();
  if (slots <= 0) return false;
  std::vector<int> dists(count);
  for (size_t i = 0; i < count; ++i) dists[i] = mbs[i].dist;
  build_items(plans, dists, slots / 2, &pb->hs);
  pack_sched(&pb->hs);
  pb->units = pb->hs.units;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  pb->off_red = up(pb->hs.bytes);
  pb->off_split = up(pb->off_red + pb->red.size() * sizeof(ReduceDesc));
  pb->off_prefix = up(pb->off_split + pb->splits.size() * sizeof(SplitDesc));
  pb->bytes = pb->off_prefix + pb->prefix.size() * sizeof(int64_t);
  pb->launches = pb->splits.empty() ? 2 : 3;
  return true;
}

// Plan the members twice: once for the size of the arena, once with the
// arena's workspace in place.
cudaError_t plan_into_arena(const BatchMember* mbs, size_t count, const BatchShape& bs,
                            BatchArena* ar, PlannedBatch* pb) {
  if (!plan_members(mbs, count, bs, nullptr, pb)) return cudaErrorInvalidValue;
  const cudaError_t e = grow_device(&ar->ws, &ar->ws_bytes, pb->ws_bytes + 256);
  if (e != cudaSuccess) return e;
  if (!plan_members(mbs, count, bs, static_cast<uint8_t*>(ar->ws), pb))
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

// One host image of everything a run reads: work list, reduce descriptors,
// split descriptors and their prefix sums.
void pack_plan(const PlannedBatch& pb, uint8_t* h) {
  memcpy(h, pb.hs.blob.data(), pb.hs.bytes);
  memcpy(h + pb.off_red, pb.red.data(), pb.red.size() * sizeof(ReduceDesc));
  if (!pb.splits.empty())
    memcpy(h + pb.off_split, pb.splits.data(), pb.splits.size() * sizeof(SplitDesc));
  memcpy(h + pb.off_prefix, pb.prefix.data(), pb.prefix.size() * sizeof(int64_t));
}

// Copy the plan into the arena.  With async_upload the copy goes through the
// arena's pinned staging and is not waited for; otherwise this waits for the
// copy so that the host image may change afterwards.
cudaError_t upload_plan(const PlannedBatch& pb, BatchArena* ar, cudaStream_t st) {
  cudaError_t e = grow_device(&ar->d_buf, &ar->d_bytes, pb.bytes);
  if (e != cudaSuccess) return e;
  if (ar->async_upload) {
    if (ar->h_stage_bytes < pb.bytes) {
      if (ar->h_stage) cudaFreeHost(ar->h_stage);
      ar->h_stage = nullptr;
      ar->h_stage_bytes = 0;
      const size_t want = std::max<size_t>(pb.bytes * 2, 1 << 16);
      e = cudaHostAlloc(&ar->h_stage, want, cudaHostAllocDefault);
      if (e != cudaSuccess) return e;
      ar->h_stage_bytes = want;
    }
    pack_plan(pb, static_cast<uint8_t*>(ar->h_stage));
    return cudaMemcpyAsync(ar->d_buf, ar->h_stage, pb.bytes, cudaMemcpyHostToDevice, st);
  }
  std::vector<uint8_t> img(pb.bytes);
  pack_plan(pb, img.data());
  e = cudaMemcpyAsync(ar->d_buf, img.data(), pb.bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

// The split pass (if any member needs it), the persistent sketch launch and
// the batched reduce of an uploaded plan.  Counts the split and sketch
// launches (the reduce counts itself).
cudaError_t launch_plan(const PlannedBatch& pb, const BatchArena& ar, cudaStream_t st) {
  uint8_t* b = static_cast<uint8_t*>(ar.d_buf);
  if (!pb.splits.empty()) {
    const int64_t blocks = std::min<int64_t>((pb.prefix.back() + 255) / 256,
                                             static_cast<int64_t>(num_sms_tc()) * 16);
    k_split_bf16x2_many<<<static_cast<unsigned>(std::max<int64_t>(blocks, 1)), 256, 0, st>>>(
        reinterpret_cast<const SplitDesc*>(b + pb.off_split),
        reinterpret_cast<const int64_t*>(b + pb.off_prefix), static_cast<int>(pb.splits.size()));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launches(1);
  }
  const LeftSched sc = device_sched(pb.hs, ar.d_buf, ar.d_status);
  const cudaError_t e =
      pb.narrow ? (pb.econv ? launch_left<kMixed, true, true, true>(sc, pb.units, st)
                            : launch_left<kMixed, true, true>(sc, pb.units, st))
                : (pb.econv ? launch_left<kMixed, true, false, true>(sc, pb.units, st)
                            : launch_left<kMixed, true, false>(sc, pb.units, st));
  if (e != cudaSuccess) return e;
  count_launches(1);
  return splitk_reduce_batched(reinterpret_cast<const ReduceDesc*>(b + pb.off_red),
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
  const int64_t rows16 = (s.L + 15) / 16;  // in 16-row units, like every item length
  int64_t splits = (units + tiles - 1) / tiles;
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, rows16 / 64));
  return (rows16 + splits - 1) / splits;
}

size_t batch_member_workspace(const BatchMember& mb, int64_t item_stages) {
  GemmShape s;
  BatchShape bs;
  bs.item_stages = item_stages;
  const LeftPlan pl = member_plan(mb, bs, &s);
  return split_bytes(s.L, s.Q) + partial_bytes(pl, s);
}

cudaError_t batch_launch_members(const BatchMember* mbs, size_t count, int64_t item_stages,
                                 BatchArena* ar, cudaEvent_t ready, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  PlannedBatch pb;
  BatchShape bs;
  bs.item_stages = item_stages;
  cudaError_t e = plan_into_arena(mbs, count, bs, ar, &pb);
  if (e == cudaSuccess) e = upload_plan(pb, ar, st);
  if (e == cudaSuccess && ready) e = cudaStreamWaitEvent(st, ready, 0);
  if (e == cudaSuccess) e = launch_plan(pb, *ar, st);
  return e;
}

}  // namespace sk

// ---------------------------------------------------------------------------
// Batches (see include/sketch.h)
// ---------------------------------------------------------------------------
struct sk_batch {
  std::vector<sk::BatchMember> entries;
  int device = 0;
  sk::BatchShape shape;     // item length, tile width and ring of the next plan
  bool chosen = false;      // shape set by sk_batch_tune or sk_batch_set_config
  bool planned = false;
  sk::BatchArena arena;     // work list, reduce descriptors, partials, status
  sk::PlannedBatch plan;
  cudaGraphExec_t graph = nullptr;
};

namespace {


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

// A tuned shape as one integer of the cache file: item stages in the low 20
// bits, bit 20 = 256-column tiles, bit 21 = narrow ring.
int64_t encode_shape(const sk::BatchShape& bs) {
  return bs.item_stages | (bs.max_nt <= 256 ? (int64_t(1) << 20) : 0) |
         (bs.narrow ? (int64_t(1) << 21) : 0);
}

bool decode_shape(int64_t v, sk::BatchShape* bs) {
  const int64_t stages = v & ((int64_t(1) << 20) - 1);
  if (stages <= 0 || (v >> 22) != 0) return false;
  bs->item_stages = stages;
  bs->max_nt = (v >> 20) & 1 ? 256 : 512;
  bs->narrow = ((v >> 21) & 1) != 0;
  return true;
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

// Plan every member with items of about `bs.item_stages` stages of 16 rows.
sk_status batch_plan(sk_batch* b, const sk::BatchShape& bs, cudaStream_t st) {
  cudaError_t e = sk::plan_into_arena(b->entries.data(), b->entries.size(), bs, &b->arena,
                                      &b->plan);
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
    return to_status(batch_launch(b, st));  // launch_plan counted its kernels
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
  if (e == cudaSuccess) sk::count_launches(b->plan.launches);  // split, sketch, reduce
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
  sk::BatchMember e{h->seed, h->dist, h->k, h->scale, A, m, n, lda, Y, ldy, nullptr, 0, false};
  b->entries.push_back(e);
  batch_invalidate(b);
  return SK_OK;
}

sk_status sk_batch_run(sk_batch_handle b, void* stream) {
  if (!b || b->entries.empty()) return SK_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!b->planned) {
    sk::BatchShape bs = b->shape;
    if (!b->chosen && !decode_shape(cache_lookup(batch_signature(b)), &bs)) bs = sk::BatchShape();
    const sk_status ps = batch_plan(b, bs, st);
    if (ps != SK_OK) return ps;
  }
  return batch_run_once(b, st, true);
}

sk_status sk_batch_tune(sk_batch_handle b, void* stream, int64_t* chosen) {
  if (!b || b->entries.empty()) return SK_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // tile width x operand ring x item length; the 512-column tiles only when
  // some member is wider than 256 columns
  bool wide = false;
  for (const auto& e : b->entries) wide = wide || e.n > 256;
  std::vector<sk::BatchShape> cands;
  const int64_t lens[] = {128, 256, 512, 1024, 2048, 4096};
  for (int variant = wide ? 0 : 1; variant < 3; ++variant) {
    for (int64_t t : lens) {
      sk::BatchShape bs;
      bs.item_stages = t;
      bs.max_nt = variant == 0 ? 512 : 256;
      bs.narrow = variant == 2;
      cands.push_back(bs);
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return to_status(cudaGetLastError());
  float best_ms = 1e30f;
  sk::BatchShape best;
  sk_status rs = SK_OK;
  for (const auto& bs : cands) {
    batch_invalidate(b);
    rs = batch_plan(b, bs, st);
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
      best = bs;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_invalidate(b);
  if (rs != SK_OK) return rs;
  b->shape = best;
  b->chosen = true;
  cache_store(batch_signature(b), encode_shape(best));
  if (chosen) *chosen = best.item_stages;
  return SK_OK;
}

sk_status sk_batch_set_config(sk_batch_handle b, int64_t item_stages, int32_t tile_cols,
                              int32_t ring_stages) {
  if (!b || item_stages < 1 || item_stages >= (int64_t(1) << 20)) return SK_EINVAL;
  if (tile_cols != 256 && tile_cols != 512) return SK_EINVAL;
  if (ring_stages != 4 && ring_stages != 8) return SK_EINVAL;
  if (ring_stages == 8 && tile_cols != 256) return SK_EINVAL;
  batch_invalidate(b);
  b->shape.item_stages = item_stages;
  b->shape.max_nt = tile_cols;
  b->shape.narrow = ring_stages == 8;
  b->chosen = true;
  return SK_OK;
}

sk_status sk_batch_config(sk_batch_handle b, int64_t* item_stages, int32_t* tile_cols,
                          int32_t* ring_stages) {
  if (!b) return SK_EINVAL;
  sk::BatchShape bs = b->shape;
  if (!b->chosen && !decode_shape(cache_lookup(batch_signature(b)), &bs)) bs = sk::BatchShape();
  if (item_stages) *item_stages = bs.item_stages;
  if (tile_cols) *tile_cols = bs.max_nt;
  if (ring_stages) *ring_stages = bs.narrow ? 8 : 4;
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

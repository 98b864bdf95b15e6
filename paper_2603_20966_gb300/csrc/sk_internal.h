// sk_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sketch.h"

struct sk_sketch {
  uint64_t seed;
  int dist;
  int64_t k;
  int prec;
  float scale;          // fl32(1/sqrt(k))
  int device;
  int* d_status;        // device status word (sk_status values), 0 = OK
  void* ws;             // split-K partials (owned or lent)
  size_t ws_bytes;
  bool ws_owned;
  float* stage_A;       // device staging for the _host entry points
  size_t stage_A_bytes;
  float* stage_Y;
  size_t stage_Y_bytes;
  cudaEvent_t prof_start;  // optional measurement hook (caller-owned events)
  cudaEvent_t prof_stop;
  void* d_sched;           // device copy of the tensor-core work list (problem + items)
  size_t d_sched_bytes;
  uint64_t sched_key[9];   // what the uploaded work list was built for
  uint64_t wait_limit_ns;  // limit of every bounded device wait (sk_debug_set_wait)
  int64_t stall_stage;     // injected stall of the tests (sk_debug_set_wait), or -1
};

namespace sk {
// Limit of a bounded device wait unless a test shortens it: far beyond any
// healthy stage, short enough that a stuck kernel returns within seconds.
constexpr uint64_t kDefaultWaitLimitNs = 2000000000ull;
}  // namespace sk

namespace sk {

// Count one kernel launch (sk_launch_count).
void count_launches(uint64_t n);

// sk_status of a CUDA error; remembers it for sk_last_cuda_error.
sk_status status_from_cuda(cudaError_t e);

// Record the handle's measurement-hook event, if any, on `st`.
inline void prof_mark(cudaEvent_t ev, cudaStream_t st) {
  if (ev) cudaEventRecord(ev, st);
}

// Problem of one fused launch: D[P x Q] = sum_l X(p, l) W(l, q) with one
// operand generated.  LEFT: X = g (P = k), W = A (Q = n), L = m.
// RIGHT: X = A (P = m), W = g^T (Q = k), L = n.
struct GemmShape {
  bool left;
  int64_t P, Q, L;
};

// ---- FP32 SIMT form (sk_simt.cu) ----
size_t simt_workspace_bytes(const GemmShape& s);
cudaError_t simt_sketch(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                        float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st);
cudaError_t materialize(const sk_sketch* h, int64_t row0, int64_t col0, int64_t rows,
                        int64_t cols, int fmt, int scaled, void* out, int64_t ld,
                        cudaStream_t st);
// fixed-order reduction of split partials: Y[p*ldy+q] = scale * sum_z part[z][p][q]
cudaError_t splitk_reduce(const float* part, int splits, int64_t P, int64_t Q, float scale,
                          float* Y, int64_t ldy, cudaStream_t st);

// fixed-order reduction of many problems in one launch
struct ReduceDesc {
  const float* part;
  float* Y;
  int64_t P, Q, ldy;
  int64_t ldp;  // partial row stride (>= Q): part[(z P + r) ldp + c]
  int splits;
  float scale;
};
cudaError_t splitk_reduce_batched(const ReduceDesc* d_desc, int nprob, int64_t max_elems,
                                  cudaStream_t st);

// ---- batches of left sketches on the tensor cores (sk_tc.cu) ----
struct BatchMember {
  uint64_t seed;
  int dist;
  int64_t k;
  float scale;
  const float* A;
  int64_t m, n, lda;
  float* Y;
  int64_t ldy;
  // own workspace of batch_member_workspace bytes (the BF16 split of A, then
  // the split partials), or null for one from the arena
  void* ws = nullptr;
  int64_t item_stages = 0;   // own work-item length in stages of 16 rows, or 0
  bool split_ready = false;  // ws already holds the BF16 split of A (A is not read)
};
// Decomposition of a batch: item length (16-row units of m), widest output
// tile (512 or 256 columns) and operand ring (the 8-stage narrow ring applies
// only when every tile has at most 256 columns).
struct BatchShape {
  int64_t item_stages = 512;
  int max_nt = 512;
  bool narrow = false;
};
// Device buffers one batch launch uses; grown on demand, owned by the caller.
struct BatchArena {
  void* d_buf = nullptr;  // work list + reduce descriptors
  size_t d_bytes = 0;
  void* ws = nullptr;     // workspaces of the members without their own
  size_t ws_bytes = 0;
  int* d_status = nullptr;
  // pinned staging of the work list: when set, uploads do not synchronise
  // (the caller guarantees the previous launch from this arena has finished)
  bool async_upload = false;
  void* h_stage = nullptr;
  size_t h_stage_bytes = 0;
};
// Work-item length (stages of 16 rows) that spreads one left sketch over all
// CTA pairs of the GPU when it runs alone (items of at least 64 stages); a
// function of the shape only.
int64_t spread_item_stages(const BatchMember& mb);
// Bytes of workspace a member needs with items of `item_stages` stages.
size_t batch_member_workspace(const BatchMember& mb, int64_t item_stages);
// The BF16 split of a left sketch's A[m x n] at the start of its workspace:
// hi rows of split_ld(n) elements, then lo rows (split_bytes in total).
int64_t split_ld(int64_t n);
size_t split_bytes(int64_t m, int64_t n);
// Write the split of A (any alignment, row stride lds; a device address) into
// `H` on `st` (one kernel launch).
cudaError_t split_rows(const float* A, int64_t lds, int64_t m, int64_t n, void* H,
                       cudaStream_t st);
// Plan the members (items of about `item_stages` stages), upload the work
// list into `arena` on `st` (synchronising `st`), make `st` wait for
// `ready` (may be null) and launch the persistent sketch kernel and the
// batched reduction on `st`.
cudaError_t batch_launch_members(const BatchMember* mbs, size_t count, int64_t item_stages,
                                 BatchArena* arena, cudaEvent_t ready, cudaStream_t st);

// ---- BF16 split-A tensor-core form (sk_tc.cu) ----
size_t tc_workspace_bytes(const GemmShape& s);
sk_status tc_check(const GemmShape& s, const float* A, int64_t lda, const float* Y, int64_t ldy);
cudaError_t tc_sketch(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                      float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st);
// the same left sketch reading a caller-stored BF16 S[k x m] (row stride lds)
cudaError_t tc_sketch_left_stored(const sk_sketch* h, const GemmShape& s, const void* S,
                                  int64_t lds, const float* A, int64_t lda, float* Y,
                                  int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st);

// ---- FP8 (E4M3) form of the right sketch (sk_tc.cu) ----
int64_t q8_ld(int64_t n);  // row stride (bytes) of the codes of an n-column A
cudaError_t q8_quantize(const float* A, int64_t lda, int64_t m, int64_t n, uint8_t* Aq,
                        int64_t ldq, int32_t* exps, cudaStream_t st);
size_t q8_partial_bytes(const GemmShape& s);
// codes + row exponents + partials of an apply call that quantizes A itself
size_t q8_workspace_bytes(const GemmShape& s);
cudaError_t q8_sketch_right_quantized(const sk_sketch* h, const GemmShape& s, const uint8_t* Aq,
                                      const int32_t* exps, int64_t ldq, float* Y, int64_t ldy,
                                      void* part, size_t part_bytes, cudaStream_t st);
cudaError_t q8_sketch_right(const sk_sketch* h, const GemmShape& s, const float* A, int64_t lda,
                            float* Y, int64_t ldy, void* ws, size_t ws_bytes, cudaStream_t st);

}  // namespace sk

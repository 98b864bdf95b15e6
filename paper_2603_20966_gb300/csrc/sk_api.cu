// sk_api.cu -- the C ABI declared in include/sketch.h: argument checking,
// scratch management and dispatch to the kernels of each arithmetic form.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "sk_internal.h"

using sk::GemmShape;

namespace sk {
static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace sk

namespace {
thread_local cudaError_t g_last_cuda_error = cudaSuccess;
}  // namespace

sk_status sk::status_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SK_OK;
  g_last_cuda_error = e;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
}

namespace {

constexpr int64_t kMaxIndex = 4294967296LL;  // generator indices are 32-bit

sk_status from_cuda(cudaError_t e) { return sk::status_from_cuda(e); }

bool valid_dist(int d) { return d == SK_GAUSSIAN || d == SK_RADEMACHER || d == SK_UNIFORM; }
bool valid_prec(int p) { return p == SK_FP32 || p == SK_BF16X2 || p == SK_FP8E4M3; }

size_t workspace_for(const sk_sketch* h, const GemmShape& s) {
  if (h->prec == SK_FP32) return sk::simt_workspace_bytes(s);
  if (h->prec == SK_FP8E4M3) return s.left ? 0 : sk::q8_workspace_bytes(s);
  return sk::tc_workspace_bytes(s);
}

// Make sure the handle has at least `need` bytes of scratch.
sk_status ensure_workspace(sk_sketch* h, size_t need) {
  if (need == 0 || h->ws_bytes >= need) return SK_OK;
  if (!h->ws_owned && h->ws != nullptr) return SK_EINVAL;  // lent buffer too small
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  h->ws_owned = true;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SK_ENOMEM;
  }
  h->ws = p;
  h->ws_bytes = need;
  return SK_OK;
}

sk_status check_apply(const sk_sketch* h, const float* A, int64_t m, int64_t n, int64_t lda,
                      const float* Y, int64_t ldy, bool left) {
  if (!h || !A || !Y) return SK_EINVAL;
  if (m <= 0 || n <= 0 || lda < n) return SK_EINVAL;
  if (left) {
    if (m >= kMaxIndex || ldy < n) return SK_EINVAL;
  } else {
    if (n >= kMaxIndex || ldy < h->k) return SK_EINVAL;
  }
  return SK_OK;
}

sk_status apply(sk_sketch* h, const float* A, int64_t m, int64_t n, int64_t lda, float* Y,
                int64_t ldy, void* stream, bool left) {
  sk_status st = check_apply(h, A, m, n, lda, Y, ldy, left);
  if (st != SK_OK) return st;
  GemmShape s;
  s.left = left;
  if (left) {
    s.P = h->k; s.Q = n; s.L = m;
  } else {
    s.P = m; s.Q = h->k; s.L = n;
  }
  if (h->prec == SK_FP8E4M3 && left) return SK_EUNSUPPORTED;  // FP8: right sketch only
  if (h->prec == SK_BF16X2) {
    st = sk::tc_check(s, A, lda, Y, ldy);
    if (st != SK_OK) return st;
  }
  if (h->prec == SK_FP8E4M3 && ((reinterpret_cast<uintptr_t>(Y) & 15u) || ldy % 4 != 0))
    return SK_EINVAL;
  st = ensure_workspace(h, workspace_for(h, s));
  if (st != SK_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (h->prec == SK_FP32)
    e = sk::simt_sketch(h, s, A, lda, Y, ldy, h->ws, h->ws_bytes, cs);
  else if (h->prec == SK_FP8E4M3)
    e = sk::q8_sketch_right(h, s, A, lda, Y, ldy, h->ws, h->ws_bytes, cs);
  else
    e = sk::tc_sketch(h, s, A, lda, Y, ldy, h->ws, h->ws_bytes, cs);
  return from_cuda(e);
}

sk_status grow(float** buf, size_t* have, size_t need) {
  if (*have >= need) return SK_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(buf), need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return SK_ENOMEM;
  }
  *have = need;
  return SK_OK;
}

sk_status apply_host(sk_sketch* h, const float* A, int64_t m, int64_t n, int64_t lda, float* Y,
                     int64_t ldy, void* stream, bool left) {
  sk_status st = check_apply(h, A, m, n, lda, Y, ldy, left);
  if (st != SK_OK) return st;
  const int64_t yr = left ? h->k : m;
  const int64_t yc = left ? n : h->k;
  // staging rows padded to a multiple of 4 floats (16-byte rows for TMA)
  const int64_t lda_d = (n + 3) / 4 * 4;
  const int64_t ldy_d = (yc + 3) / 4 * 4;
  st = grow(&h->stage_A, &h->stage_A_bytes, (size_t)m * (size_t)lda_d * sizeof(float));
  if (st != SK_OK) return st;
  st = grow(&h->stage_Y, &h->stage_Y_bytes, (size_t)yr * (size_t)ldy_d * sizeof(float));
  if (st != SK_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  // rows without padding on either side (leading dimension = row length, a
  // multiple of 4) move as one linear copy of exactly the matrix's bytes
  cudaError_t e =
      lda == n && lda_d == n
          ? cudaMemcpyAsync(h->stage_A, A, (size_t)m * (size_t)lda * sizeof(float),
                            cudaMemcpyHostToDevice, cs)
          : cudaMemcpy2DAsync(h->stage_A, lda_d * sizeof(float), A, lda * sizeof(float),
                              n * sizeof(float), m, cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return from_cuda(e);
  st = apply(h, h->stage_A, m, n, lda_d, h->stage_Y, ldy_d, stream, left);
  if (st != SK_OK) return st;
  e = ldy == yc && ldy_d == yc
          ? cudaMemcpyAsync(Y, h->stage_Y, (size_t)yr * (size_t)ldy * sizeof(float),
                            cudaMemcpyDeviceToHost, cs)
          : cudaMemcpy2DAsync(Y, ldy * sizeof(float), h->stage_Y, ldy_d * sizeof(float),
                              yc * sizeof(float), yr, cudaMemcpyDeviceToHost, cs);
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(cudaStreamSynchronize(cs));
}

}  // namespace

extern "C" {

sk_status sk_create(uint64_t seed, int dist, int64_t k, sk_handle* out) {
  if (!out || !valid_dist(dist) || k < 1 || k > (1LL << 31)) return SK_EINVAL;
  *out = nullptr;
  sk_sketch* h = new (std::nothrow) sk_sketch;
  if (!h) return SK_ENOMEM;
  memset(h, 0, sizeof(*h));
  h->seed = seed;
  h->dist = dist;
  h->k = k;
  h->prec = SK_FP32;
  h->scale = 1.0f / sqrtf((float)k);  // both operations IEEE round-to-nearest
  h->wait_limit_ns = sk::kDefaultWaitLimitNs;
  h->stall_stage = -1;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->d_status), sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int) * 4);
  if (e != cudaSuccess) {
    if (h->d_status) cudaFree(h->d_status);
    delete h;
    return from_cuda(e);
  }
  *out = h;
  return SK_OK;
}

sk_status sk_set_precision(sk_handle h, int precision) {
  if (!h || !valid_prec(precision)) return SK_EINVAL;
  h->prec = precision;
  return SK_OK;
}

sk_status sk_get_info(sk_handle h, uint64_t* seed, int* dist, int64_t* k, int* precision,
                      float* scale) {
  if (!h) return SK_EINVAL;
  if (seed) *seed = h->seed;
  if (dist) *dist = h->dist;
  if (k) *k = h->k;
  if (precision) *precision = h->prec;
  if (scale) *scale = h->scale;
  return SK_OK;
}

sk_status sk_apply_left(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda, float* Y,
                        int64_t ldy, void* stream) {
  return apply(h, A, m, n, lda, Y, ldy, stream, true);
}

sk_status sk_apply_right(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda,
                         float* Y, int64_t ldy, void* stream) {
  return apply(h, A, m, n, lda, Y, ldy, stream, false);
}

sk_status sk_apply_left_host(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda,
                             float* Y, int64_t ldy, void* stream) {
  return apply_host(h, A, m, n, lda, Y, ldy, stream, true);
}

sk_status sk_apply_right_host(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda,
                              float* Y, int64_t ldy, void* stream) {
  return apply_host(h, A, m, n, lda, Y, ldy, stream, false);
}

sk_status sk_materialize(sk_handle h, int64_t row0, int64_t col0, int64_t rows, int64_t cols,
                         int fmt, int scaled, void* out, int64_t ld, void* stream) {
  if (!h || !out || rows <= 0 || cols <= 0 || row0 < 0 || col0 < 0 || ld < cols) return SK_EINVAL;
  if (!valid_prec(fmt) || (scaled && fmt != SK_FP32)) return SK_EINVAL;
  if (row0 + rows > kMaxIndex || col0 + cols > kMaxIndex) return SK_EINVAL;
  return from_cuda(sk::materialize(h, row0, col0, rows, cols, fmt, scaled, out, ld,
                                   static_cast<cudaStream_t>(stream)));
}

sk_status sk_nystrom(sk_handle h, const float* A, int64_t n, int64_t lda, float* B, int64_t ldb,
                     float* C, int64_t ldc, void* stream) {
  if (!h || !A || !B || !C || n <= 0 || lda < n || ldb < h->k || ldc < h->k) return SK_EINVAL;
  if (h->prec == SK_FP8E4M3) return SK_EUNSUPPORTED;  // the second product is a left sketch
  // B[n x k] = A Omega (right sketch), then C[k x k] = Omega^T B = S B (left
  // sketch of B): the same S, regenerated by both kernels
  const sk_status st = apply(h, A, n, n, lda, B, ldb, stream, false);
  if (st != SK_OK) return st;
  return apply(h, B, n, h->k, ldb, C, ldc, stream, true);
}

sk_status sk_apply_left_stored(sk_handle h, const void* S, int64_t lds, const float* A,
                              int64_t m, int64_t n, int64_t lda, float* Y, int64_t ldy,
                              void* stream) {
  sk_status st = check_apply(h, A, m, n, lda, Y, ldy, true);
  if (st != SK_OK) return st;
  if (h->prec != SK_BF16X2) return SK_EUNSUPPORTED;
  if (!S || h->k % 8 != 0 || lds % 8 != 0 || lds < (m + 15) / 16 * 16 ||
      (reinterpret_cast<uintptr_t>(S) & 15u))
    return SK_EINVAL;
  GemmShape s;
  s.left = true;
  s.P = h->k;
  s.Q = n;
  s.L = m;
  st = sk::tc_check(s, A, lda, Y, ldy);
  if (st != SK_OK) return st;
  st = ensure_workspace(h, workspace_for(h, s));
  if (st != SK_OK) return st;
  return from_cuda(sk::tc_sketch_left_stored(h, s, S, lds, A, lda, Y, ldy, h->ws, h->ws_bytes,
                                             static_cast<cudaStream_t>(stream)));
}

sk_status sk_quantize_e4m3(const float* A, int64_t m, int64_t n, int64_t lda, uint8_t* Aq,
                           int64_t ldq, int32_t* row_exp, void* stream) {
  if (!A || !Aq || !row_exp || m <= 0 || n <= 0 || lda < n || ldq < n || ldq % 16 != 0)
    return SK_EINVAL;
  if (reinterpret_cast<uintptr_t>(Aq) & 15u) return SK_EINVAL;
  return from_cuda(sk::q8_quantize(A, lda, m, n, Aq, ldq, row_exp,
                                   static_cast<cudaStream_t>(stream)));
}

sk_status sk_apply_right_e4m3(sk_handle h, const uint8_t* Aq, const int32_t* row_exp, int64_t m,
                              int64_t n, int64_t ldq, float* Y, int64_t ldy, void* stream) {
  if (!h || !Aq || !row_exp || !Y || m <= 0 || n <= 0 || ldq < n || ldq % 16 != 0 ||
      ldy < h->k)
    return SK_EINVAL;
  if ((reinterpret_cast<uintptr_t>(Aq) & 15u) || (reinterpret_cast<uintptr_t>(Y) & 15u) ||
      ldy % 4 != 0)
    return SK_EINVAL;
  if (n >= kMaxIndex || m >= (1LL << 31)) return SK_EINVAL;
  GemmShape s;
  s.left = false;
  s.P = m;
  s.Q = h->k;
  s.L = n;
  const sk_status st = ensure_workspace(h, sk::q8_partial_bytes(s));
  if (st != SK_OK) return st;
  return from_cuda(sk::q8_sketch_right_quantized(h, s, Aq, row_exp, ldq, Y, ldy, h->ws,
                                                 h->ws_bytes, static_cast<cudaStream_t>(stream)));
}

sk_status sk_workspace_size(sk_handle h, int side, int64_t m, int64_t n, size_t* bytes) {
  if (!h || !bytes || (side != 0 && side != 1) || m <= 0 || n <= 0) return SK_EINVAL;
  GemmShape s;
  s.left = side == 0;
  if (s.left) {
    s.P = h->k; s.Q = n; s.L = m;
  } else {
    s.P = m; s.Q = h->k; s.L = n;
  }
  *bytes = workspace_for(h, s);
  return SK_OK;
}

sk_status sk_set_workspace(sk_handle h, void* ptr, size_t bytes) {
  if (!h) return SK_EINVAL;
  if (ptr && (reinterpret_cast<uintptr_t>(ptr) & 15u)) return SK_EINVAL;
  if (h->ws_owned && h->ws) cudaFree(h->ws);
  h->ws = ptr;
  h->ws_bytes = ptr ? bytes : 0;
  h->ws_owned = false;
  return SK_OK;
}

sk_status sk_stream_status(sk_handle h, void* stream) {
  if (!h) return SK_EINVAL;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return from_cuda(e);
  int word = 0;
  e = cudaMemcpy(&word, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  if (word != 0) {
    e = cudaMemset(h->d_status, 0, sizeof(int) * 4);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return static_cast<sk_status>(word);
}

sk_status sk_debug_status(sk_handle h, void* stream, int32_t out[4]) {
  if (!h || !out) return SK_EINVAL;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaMemcpy(out, h->d_status, sizeof(int) * 4, cudaMemcpyDeviceToHost);
  return from_cuda(e);
}

sk_status sk_debug_set_wait(sk_handle h, uint64_t limit_ns, int64_t stall_stage) {
  if (!h) return SK_EINVAL;
  if (limit_ns != 0 && limit_ns < 1000000ull) return SK_EINVAL;  // at least 1 ms
  h->wait_limit_ns = limit_ns ? limit_ns : sk::kDefaultWaitLimitNs;
  h->stall_stage = stall_stage < 0 ? -1 : stall_stage;
  return SK_OK;
}

sk_status sk_destroy(sk_handle h) {
  if (!h) return SK_EINVAL;
  if (h->ws_owned && h->ws) cudaFree(h->ws);
  if (h->stage_A) cudaFree(h->stage_A);
  if (h->stage_Y) cudaFree(h->stage_Y);
  if (h->d_sched) cudaFree(h->d_sched);
  if (h->d_status) cudaFree(h->d_status);
  delete h;
  return SK_OK;
}

sk_status sk_profile_events(sk_handle h, void* start_event, void* stop_event) {
  if (!h || ((start_event == nullptr) != (stop_event == nullptr))) return SK_EINVAL;
  h->prof_start = static_cast<cudaEvent_t>(start_event);
  h->prof_stop = static_cast<cudaEvent_t>(stop_event);
  return SK_OK;
}

uint64_t sk_launch_count(void) { return sk::g_launches.load(std::memory_order_relaxed); }

const char* sk_status_string(int status) {
  switch (status) {
    case SK_OK: return "SK_OK";
    case SK_EINVAL: return "SK_EINVAL: invalid argument";
    case SK_ENOMEM: return "SK_ENOMEM: out of memory";
    case SK_ECUDA: return "SK_ECUDA: CUDA call failed";
    case SK_ETIMEOUT: return "SK_ETIMEOUT: bounded device wait gave up";
    case SK_EBUDGET: return "SK_EBUDGET: request exceeds the memory budget";
    case SK_EUNSUPPORTED: return "SK_EUNSUPPORTED: combination not implemented";
    case SK_EBUSY: return "SK_EBUSY: not ready";
    case SK_ECANCELLED: return "SK_ECANCELLED: request cancelled";
    default: return "unknown sk_status";
  }
}

const char* sk_last_cuda_error(void) {
  return g_last_cuda_error == cudaSuccess ? "no error" : cudaGetErrorString(g_last_cuda_error);
}

int sk_version(void) { return 100; }

}  // extern "C"

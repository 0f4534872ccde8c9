// sr_common.cuh -- internal definitions shared by the libsr translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sr.h"

// ---------------------------------------------------------------- context
struct sr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  // growable device workspace (scratch for partial sums, queues, stacks)
  char *ws = nullptr;
  size_t ws_bytes = 0;
  // small permanent device block: [0] latched error word, [1..] spare
  unsigned *dev_words = nullptr;
  char msg[512] = {0};
  uint64_t launches = 0;  // kernels launched by this context
  int tile_cases = 0;     // cases per evaluation work item (0: automatic)
  int eval_ctas = 0;      // CTAs per SM of the single-problem evaluation (0: automatic, 4, 5)
  int batched_ctas = 0;   // CTAs per SM of the batched evaluation (0: automatic = 4, 3, 4, 5)
  int xform = 1;          // variable transforms of the evaluation: 0 never, 1 automatic, 2 always
  const uint64_t *gen_dev = nullptr;  // device generation counter for selection / variation
  const int32_t *abort_flag = nullptr;  // sr_set_abort_flag (device, or NULL)
};

namespace sr {

constexpr unsigned FULL = 0xffffffffu;

// token encoding (uint8), see sr.h
constexpr int TOK_ADD = 0, TOK_SUB = 1, TOK_MUL = 2, TOK_DIV = 3;
constexpr int TOK_SIN = 4, TOK_COS = 5, TOK_EXP = 6, TOK_LOG = 7, TOK_SQRT = 8,
              TOK_SQ = 9;
// the rest of the operator set of Table 1
constexpr int TOK_INV = 10, TOK_TAN = 11, TOK_ASIN = 12, TOK_ACOS = 13, TOK_ATAN = 14,
              TOK_TANH = 15;
constexpr int UNARY_BASE = 6, UNARY_ALL = 12;  // operator sets of the generators
constexpr int TOK_VAR0 = 16, TOK_CONST0 = 32, TOK_NSLOTS = 16;

// token classes used by the decoders
constexpr int CLS_VAR = 0, CLS_CONST = 1, CLS_UNARY = 2, CLS_BINARY = 3,
              CLS_BAD = 4;

__host__ __device__ __forceinline__ int tok_class(int v) {
  if (v <= TOK_DIV) return CLS_BINARY;
  if (v <= TOK_TANH) return CLS_UNARY;
  if (v >= TOK_VAR0 && v < TOK_VAR0 + TOK_NSLOTS) return CLS_VAR;
  if (v >= TOK_CONST0 && v < TOK_CONST0 + TOK_NSLOTS) return CLS_CONST;
  return CLS_BAD;
}
__host__ __device__ __forceinline__ int cls_effect(int c) {
  return c == CLS_BINARY ? -1 : (c <= CLS_CONST ? 1 : 0);
}

// device error word bits (latched; reported and cleared by sr_sync)
constexpr unsigned ERR_TIMEOUT = 1u;
constexpr unsigned ERR_ABORTED = 2u;

// The next work item of a persistent warp (lane 0 draws it from the atomic
// counter q and the warp shares it), or `total` (no more items) when the
// abort flag is set; then the abort is latched in the error word.  Only
// lane 0 touches memory.
__device__ __forceinline__ long long next_item(unsigned long long *q, long long total, const int32_t *abort_flag,
                                               unsigned *err_word, int lane) {
  long long item = 0;
  if (lane == 0) {
    if (abort_flag && *reinterpret_cast<const volatile int32_t *>(abort_flag) != 0) {
      atomicOr(err_word, ERR_ABORTED);
      item = total;
    } else {
      item = (long long)atomicAdd(q, 1ull);
    }
  }
  return __shfl_sync(FULL, item, 0);
}

// status helpers (sr_ctx.cu)
sr_status fail(sr_ctx *ctx, sr_status s, const char *fmt, ...);
sr_status cuda_fail(sr_ctx *ctx, cudaError_t e, const char *what);
// grow the workspace to at least `bytes` (refused during stream capture)
sr_status ensure_workspace(sr_ctx *ctx, size_t bytes);
bool stream_capturing(sr_ctx *ctx);
// Let `kernel` use up to 227 KB of dynamic shared memory on the context's
// device.  Function attributes belong to a device; this sets each (kernel,
// device) pair once per process (thread-safe).
sr_status allow_dynamic_smem(sr_ctx *ctx, const void *kernel);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// sequential carving of the workspace
struct Carver {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  }
};

}  // namespace sr

#define SR_CHECK_CUDA(ctx, call)                                  \
  do {                                                            \
    cudaError_t _e = (call);                                      \
    if (_e != cudaSuccess) return ::sr::cuda_fail(ctx, _e, #call); \
  } while (0)

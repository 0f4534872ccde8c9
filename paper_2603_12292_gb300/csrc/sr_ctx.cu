// sr_ctx.cu -- context lifetime, workspace, status reporting.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <utility>
#include <vector>

#include "sr_common.cuh"

namespace sr {

sr_status fail(sr_ctx *ctx, sr_status s, const char *fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->msg, sizeof(ctx->msg), fmt, ap);
    va_end(ap);
  }
  return s;
}

sr_status cuda_fail(sr_ctx *ctx, cudaError_t e, const char *what) {
  return fail(ctx, SR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool stream_capturing(sr_ctx *ctx) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &st) != cudaSuccess) return false;
  return st != cudaStreamCaptureStatusNone;
}

sr_status allow_dynamic_smem(sr_ctx *ctx, const void *kernel) {
  static std::mutex mu;
  static std::vector<std::pair<const void *, int>> done;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto &d : done)
    if (d.first == kernel && d.second == ctx->device) return SR_OK;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
  done.emplace_back(kernel, ctx->device);
  return SR_OK;
}

sr_status ensure_workspace(sr_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return SR_OK;
  if (stream_capturing(ctx))
    return fail(ctx, SR_ENOMEM,
                "workspace of %zu bytes needed during stream capture (have %zu); "
                "call sr_reserve before capturing",
                bytes, ctx->ws_bytes);
  // the old workspace may still be read by queued work on this stream
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  size_t want = align_up(bytes + bytes / 4, 1 << 20);
  e = cudaMalloc((void **)&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SR_ENOMEM, "cudaMalloc(%zu) for the workspace: %s", want,
                cudaGetErrorString(e));
  }
  ctx->ws_bytes = want;
  return SR_OK;
}

}  // namespace sr

extern "C" {

sr_status sr_create(sr_ctx **out, int device, void *cuda_stream) {
  if (!out) return SR_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SR_EINVAL;
  }
  sr_ctx *ctx = new sr_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->dev_words, 256);
  if (e == cudaSuccess) e = cudaMemset(ctx->dev_words, 0, 256);
  if (e != cudaSuccess) {
    delete ctx;
    return SR_ECUDA;
  }
  *out = ctx;
  return SR_OK;
}

sr_status sr_destroy(sr_ctx *ctx) {
  if (!ctx) return SR_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->dev_words) cudaFree(ctx->dev_words);
  delete ctx;
  return SR_OK;
}

sr_status sr_set_stream(sr_ctx *ctx, void *cuda_stream) {
  if (!ctx) return SR_EINVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return SR_OK;
}

const char *sr_status_string(sr_status s) {
  switch (s) {
    case SR_OK: return "ok";
    case SR_EINVAL: return "invalid argument";
    case SR_ECUDA: return "CUDA error";
    case SR_ETIMEOUT: return "device wait timed out";
    case SR_EPROGRAM: return "invalid program";
    case SR_ENOMEM: return "out of workspace memory";
    case SR_EABORTED: return "aborted by the abort flag";
  }
  return "unknown status";
}

const char *sr_last_error(const sr_ctx *ctx) { return ctx ? ctx->msg : ""; }

uint64_t sr_kernel_launches(const sr_ctx *ctx) { return ctx ? ctx->launches : 0; }

sr_status sr_sync(sr_ctx *ctx) {
  if (!ctx) return SR_EINVAL;
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  SR_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  unsigned word = 0;
  SR_CHECK_CUDA(ctx, cudaMemcpy(&word, ctx->dev_words, sizeof(word), cudaMemcpyDeviceToHost));
  if (word) {
    SR_CHECK_CUDA(ctx, cudaMemset(ctx->dev_words, 0, sizeof(word)));
    if (word & sr::ERR_ABORTED)
      return sr::fail(ctx, SR_EABORTED, "the abort flag stopped a call: its outputs are undefined (error word 0x%x)",
                      word);
    if (word & sr::ERR_TIMEOUT)
      return sr::fail(ctx, SR_ETIMEOUT, "a bounded device wait gave up (error word 0x%x)", word);
  }
  return SR_OK;
}

sr_status sr_set_abort_flag(sr_ctx *ctx, const int32_t *flag) {
  if (!ctx) return SR_EINVAL;
  ctx->abort_flag = flag;
  return SR_OK;
}

}  // extern "C"

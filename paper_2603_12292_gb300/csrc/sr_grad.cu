// sr_grad.cu -- reverse-mode derivative of the interpreter (dMSE/dconst) and
// the Adam update of the constants.
//
// Layout: a work item is (case chunk, program), handed to one warp by an
// atomic counter, as for evaluation.  Lane 0 decodes the program into
// shared memory: per token its operator and, for a binary operator, the
// token that produced its left operand (the right operand is always the
// token just before).  Each lane then takes one case at a time:
//   forward  -- every token's output goes to a per-lane tape in shared
//               memory, tape[t][lane] (conflict-free), operands read back
//               from the tape;
//   reverse  -- tokens from last to first with the current adjoint in a
//               register and a per-lane adjoint stack for pending left
//               subtrees: a binary op pushes adj * d/da and continues into
//               its right operand with adj * d/db; a unary op multiplies
//               by its derivative; a constant terminal adds adj into its
//               slot's gradient; after any terminal the next adjoint is
//               popped.  No tape leaves the chip: the forward pass is
//               recomputed instead of stored.
// Sums: per lane FP32 compensated (Kahan) over the item's cases, FP64 across
// lanes (shuffles) and chunks (fixed-order finalize).
#include <math.h>

#include "sr_common.cuh"

namespace sr {
namespace {

constexpr int GWARPS = 4;         // warps per CTA
constexpr int GSTRIDE = 32;       // doubles per partial record: [0] sum e^2, [1 + k] sum e dyhat/dc_k
constexpr int TARGET_ITEMS_PER_WARP = 8;

// decoded token: bits 0..7 class/op, 8..15 operand index, 16..31 left operand token
enum GOp : uint32_t { G_VAR = 0, G_CONST, G_ADD, G_SUB, G_MUL, G_DIV, G_SIN, G_COS, G_EXP, G_LOG,
                      G_SQRT, G_SQ };

struct GradParams {
  const uint8_t *programs;
  const int32_t *lengths;
  const float *consts;
  int P, Lmax, K;
  const float *X;
  const float *y;
  int nvars, N;
  long long ldx;
  int chunk, nchunks;
  long long total_items;
  double *partials;   // [P * nchunks][GSTRIDE]
  int32_t *flags;     // [P]
  unsigned long long *queue;
  int warp_bytes;
  int adj_slots;
};

__host__ __device__ inline int grad_warp_bytes(int Lmax) {
  const int adj_slots = (Lmax + 1) / 2 + 1;
  // tape [Lmax][32] | adjoint stack [adj_slots][32] | gradient sums and
  // compensations [2][16][32] | code [Lmax] | constants [16]
  return Lmax * 128 + adj_slots * 128 + 2 * 16 * 128 + ((Lmax * 4 + 15) / 16) * 16 + 64;
}

__device__ __forceinline__ float op_div(float a, float b) {
  return fabsf(b) < 1e-3f ? 1.0f : a / b;
}
__device__ __forceinline__ float op_log(float x) { return fabsf(x) < 1e-3f ? 0.0f : logf(fabsf(x)); }
__device__ __forceinline__ float op_exp(float x) {
  x = x > 80.0f ? 80.0f : (x < -80.0f ? -80.0f : x);
  return expf(x);
}

struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float yv = x - c;
    const float t = s + yv;
    c = (t - s) - yv;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Serial decode by the calling lane: validation flags (same rules as the
// evaluation path), operator codes and left-operand tokens.  `last` is
// scratch of (Lmax + 2) ints.
__device__ int decode_serial(const uint8_t *__restrict__ tok, int L, int Lmax, int nvars, int K,
                             uint32_t *code, int *last) {
  if (L < 1 || L > Lmax) return SR_PF_BAD_LENGTH;
  int flags = 0, depth = 0;
  for (int t = 0; t < L; ++t) {
    const int v = tok[t];
    const int cls = tok_class(v);
    uint32_t op = 0, arg = 0, left = 0;
    if (cls == CLS_VAR) {
      op = G_VAR;
      arg = (uint32_t)(v - TOK_VAR0);
      if ((int)arg >= nvars) flags |= SR_PF_BAD_VAR;
    } else if (cls == CLS_CONST) {
      op = G_CONST;
      arg = (uint32_t)(v - TOK_CONST0);
      if ((int)arg >= K) flags |= SR_PF_BAD_CONST;
    } else if (cls == CLS_UNARY) {
      op = G_SIN + (uint32_t)(v - TOK_SIN);
    } else if (cls == CLS_BINARY) {
      op = G_ADD + (uint32_t)v;
    } else {
      flags |= SR_PF_BAD_TOKEN;
    }
    depth += cls_effect(cls);
    if (depth < 1) flags |= SR_PF_UNDERFLOW;
    if (cls == CLS_BINARY && depth >= 1 && depth <= Lmax) left = (uint32_t)last[depth];
    if (depth >= 0 && depth <= Lmax + 1) last[depth] = t;
    code[t] = op | (arg << 8) | (left << 16);
  }
  if (depth != 1) flags |= SR_PF_BAD_FINAL;
  return flags;
}

__global__ void __launch_bounds__(GWARPS * 32) grad_kernel(GradParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *wb = smem + (size_t)warp * p.warp_bytes;
  float *tape = reinterpret_cast<float *>(wb);                          // [Lmax][32]
  float *astk = tape + (size_t)p.Lmax * 32;                             // [adj_slots][32]
  float *gs = astk + (size_t)p.adj_slots * 32;                          // [16][32]
  float *gc = gs + 16 * 32;                                             // [16][32]
  uint32_t *code = reinterpret_cast<uint32_t *>(gc + 16 * 32);          // [Lmax]
  float *cv = reinterpret_cast<float *>(code + ((p.Lmax * 4 + 15) / 16) * 4);  // [16]
  // `last` for the serial decode reuses this lane's adjoint-stack column
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(p.queue, 1ull);
    item = __shfl_sync(FULL, item, 0);
    if ((long long)item >= p.total_items) break;
    const int c = (int)(item / (unsigned long long)p.P);
    const int prog = (int)(item % (unsigned long long)p.P);
    const int L = p.lengths[prog];
    __syncwarp();
    int flags = 0;
    if (lane == 0) {
      // astk (adj_slots * 32 ints) is free here and larger than Lmax + 2
      flags = decode_serial(p.programs + (size_t)prog * p.Lmax, L, p.Lmax, p.nvars, p.K, code,
                            reinterpret_cast<int *>(astk));
      if (c == 0) p.flags[prog] = flags;
    }
    flags = __shfl_sync(FULL, flags, 0);
    double *rec = p.partials + ((size_t)prog * p.nchunks + c) * GSTRIDE;
    if (flags) continue;
    if (lane < p.K) cv[lane] = p.consts[(size_t)prog * p.K + lane];
    for (int k = 0; k < p.K; ++k) {
      gs[k * 32 + lane] = 0.f;
      gc[k * 32 + lane] = 0.f;
    }
    __syncwarp();

    const int cbeg = c * p.chunk, cend = min(p.N, cbeg + p.chunk);
    Kahan se;
    for (int i = cbeg + lane; i < cend; i += 32) {
      // forward: tape[t] = output of token t
      for (int t = 0; t < L; ++t) {
        const uint32_t w = code[t];
        const int arg = (w >> 8) & 0xff;
        float r;
        switch (w & 0xff) {
          case G_VAR: r = __ldg(p.X + arg * p.ldx + i); break;
          case G_CONST: r = cv[arg]; break;
          case G_ADD: r = tape[(w >> 16) * 32 + lane] + tape[(t - 1) * 32 + lane]; break;
          case G_SUB: r = tape[(w >> 16) * 32 + lane] - tape[(t - 1) * 32 + lane]; break;
          case G_MUL: r = tape[(w >> 16) * 32 + lane] * tape[(t - 1) * 32 + lane]; break;
          case G_DIV: r = op_div(tape[(w >> 16) * 32 + lane], tape[(t - 1) * 32 + lane]); break;
          case G_SIN: r = sinf(tape[(t - 1) * 32 + lane]); break;
          case G_COS: r = cosf(tape[(t - 1) * 32 + lane]); break;
          case G_EXP: r = op_exp(tape[(t - 1) * 32 + lane]); break;
          case G_LOG: r = op_log(tape[(t - 1) * 32 + lane]); break;
          case G_SQRT: r = sqrtf(fabsf(tape[(t - 1) * 32 + lane])); break;
          default: { const float x = tape[(t - 1) * 32 + lane]; r = x * x; } break;
        }
        tape[t * 32 + lane] = r;
      }
      const float e = tape[(L - 1) * 32 + lane] - __ldg(p.y + i);
      se.add(e * e);
      // reverse sweep
      float adj = e;
      int sp = 0;
      for (int t = L - 1; t >= 0; --t) {
        const uint32_t w = code[t];
        const int op = w & 0xff;
        if (op == G_VAR || op == G_CONST) {
          if (op == G_CONST) {
            const int k = (w >> 8) & 0xff;
            // compensated per-lane accumulation of this constant's gradient
            const float yv = adj - gc[k * 32 + lane];
            const float s0 = gs[k * 32 + lane];
            const float tt = s0 + yv;
            gc[k * 32 + lane] = (tt - s0) - yv;
            gs[k * 32 + lane] = tt;
          }
          if (sp > 0) adj = astk[(--sp) * 32 + lane];
          continue;
        }
        const float out = tape[t * 32 + lane];
        const float b = tape[(t - 1) * 32 + lane];  // right operand, or the unary argument
        switch (op) {
          case G_ADD: astk[(sp++) * 32 + lane] = adj; break;
          case G_SUB: astk[(sp++) * 32 + lane] = adj; adj = -adj; break;
          case G_MUL: {
            const float a = tape[(w >> 16) * 32 + lane];
            astk[(sp++) * 32 + lane] = adj * b;
            adj = adj * a;
          } break;
          case G_DIV: {
            if (fabsf(b) < 1e-3f) {
              astk[(sp++) * 32 + lane] = 0.f;
              adj = 0.f;
            } else {
              astk[(sp++) * 32 + lane] = adj / b;
              adj = -adj * out / b;
            }
          } break;
          case G_SIN: adj = adj * cosf(b); break;
          case G_COS: adj = -adj * sinf(b); break;
          case G_EXP: adj = (b > 80.0f || b < -80.0f) ? 0.f : adj * out; break;
          case G_LOG: adj = fabsf(b) < 1e-3f ? 0.f : adj / b; break;
          case G_SQRT: adj = b == 0.0f ? 0.f : (b > 0.0f ? adj * 0.5f / out : -adj * 0.5f / out); break;
          default: adj = adj * 2.0f * b; break;
        }
      }
    }
    const double sv = warp_sum(se.value());
    if (lane == 0) rec[0] = sv;
    for (int k = 0; k < p.K; ++k) {
      const double g = warp_sum((double)gs[k * 32 + lane] - (double)gc[k * 32 + lane]);
      if (lane == 0) rec[1 + k] = g;
    }
  }
}

struct GradFinal {
  const double *partials;
  const int32_t *flags;
  int P, N, K, nchunks;
  double *mse, *dconst;
};

__global__ void grad_finalize_kernel(GradFinal f) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= f.P) return;
  if (f.flags[p]) {
    f.mse[p] = __longlong_as_double(0x7ff0000000000000ll);
    for (int k = 0; k < f.K; ++k) f.dconst[(size_t)p * f.K + k] = 0.0;
    return;
  }
  const double *rec = f.partials + (size_t)p * f.nchunks * GSTRIDE;
  double se = 0.0;
  for (int c = 0; c < f.nchunks; ++c) se += rec[c * GSTRIDE];
  f.mse[p] = isfinite(se) ? se / (double)f.N : __longlong_as_double(0x7ff0000000000000ll);
  for (int k = 0; k < f.K; ++k) {
    double g = 0.0;
    for (int c = 0; c < f.nchunks; ++c) g += rec[c * GSTRIDE + 1 + k];
    f.dconst[(size_t)p * f.K + k] = 2.0 * g / (double)f.N;
  }
}

// Adam, FP64 moments, every operation rounded on its own in the written order
__global__ void adam_kernel(float *c, const double *__restrict__ g, double *m, double *v, int n,
                            double lr, double b1, double b2, double eps, double bc1, double bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gi = g[i];
  if (!isfinite(gi)) return;
  const double mi = __dadd_rn(__dmul_rn(b1, m[i]), __dmul_rn(__dsub_rn(1.0, b1), gi));
  const double vi = __dadd_rn(__dmul_rn(b2, v[i]), __dmul_rn(__dmul_rn(__dsub_rn(1.0, b2), gi), gi));
  m[i] = mi;
  v[i] = vi;
  const double mh = __ddiv_rn(mi, bc1), vh = __ddiv_rn(vi, bc2);
  const double step = __ddiv_rn(__dmul_rn(lr, mh), __dadd_rn(__dsqrt_rn(vh), eps));
  c[i] = __double2float_rn(__dsub_rn((double)c[i], step));
}

}  // namespace
}  // namespace sr

extern "C" {

sr_status sr_eval_grad(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths,
                       const float *consts, int P, int Lmax, int K, const float *X, const float *y,
                       int nvars, int N, int ldx, double *mse, double *dconst, int32_t *prog_flags) {
  using namespace sr;
  if (!ctx) return SR_EINVAL;
  if (P < 0 || Lmax < 1 || Lmax > SR_MAX_LMAX || K < 1 || K > SR_MAX_CONSTS || nvars < 1 ||
      nvars > SR_MAX_VARS || N < 1 || ldx < N)
    return fail(ctx, SR_EINVAL, "bad sr_eval_grad shape");
  if (P == 0) return SR_OK;
  if (!programs || !lengths || !consts || !X || !y || !mse || !dconst)
    return fail(ctx, SR_EINVAL, "NULL pointer");
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  const int warp_bytes = grad_warp_bytes(Lmax);
  const int smem = GWARPS * warp_bytes;
  static int configured = 0;
  if (!configured) {
    SR_CHECK_CUDA(ctx, cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            227 * 1024));
    configured = 1;
  }
  int nb = 0;
  SR_CHECK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, grad_kernel, GWARPS * 32, smem));
  if (nb < 1) return fail(ctx, SR_EINVAL, "Lmax %d too large for the gradient tape", Lmax);
  const int grid = nb * ctx->num_sms;
  const long long warps = (long long)grid * GWARPS;
  int nch = (int)((warps * TARGET_ITEMS_PER_WARP + P - 1) / P);
  const int max_chunks = (N + 1023) / 1024;
  nch = nch < 1 ? 1 : (nch > max_chunks ? max_chunks : nch);
  int chunk = (N + nch - 1) / nch;
  chunk = (chunk + 31) / 32 * 32;
  const int nchunks = (N + chunk - 1) / chunk;
  const long long items = (long long)P * nchunks;
  Carver cv;
  const size_t off_q = cv.take(256), off_f = cv.take((size_t)P * 4),
               off_p = cv.take((size_t)items * GSTRIDE * 8);
  sr_status st = ensure_workspace(ctx, cv.off);
  if (st != SR_OK) return st;
  GradParams gp;
  gp.programs = programs;
  gp.lengths = lengths;
  gp.consts = consts;
  gp.P = P;
  gp.Lmax = Lmax;
  gp.K = K;
  gp.X = X;
  gp.y = y;
  gp.nvars = nvars;
  gp.N = N;
  gp.ldx = ldx;
  gp.chunk = chunk;
  gp.nchunks = nchunks;
  gp.total_items = items;
  gp.partials = reinterpret_cast<double *>(ctx->ws + off_p);
  gp.flags = prog_flags ? prog_flags : reinterpret_cast<int32_t *>(ctx->ws + off_f);
  gp.queue = reinterpret_cast<unsigned long long *>(ctx->ws + off_q);
  gp.warp_bytes = warp_bytes;
  gp.adj_slots = (Lmax + 1) / 2 + 1;
  SR_CHECK_CUDA(ctx, cudaMemsetAsync(gp.queue, 0, 8, ctx->stream));
  grad_kernel<<<grid, GWARPS * 32, smem, ctx->stream>>>(gp);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  GradFinal gf{gp.partials, gp.flags, P, N, K, nchunks, mse, dconst};
  grad_finalize_kernel<<<(P + 255) / 256, 256, 0, ctx->stream>>>(gf);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 2;
  return SR_OK;
}

sr_status sr_adam_step(sr_ctx *ctx, float *consts, const double *grad, double *m, double *v, int n,
                       int t, const sr_adam_cfg *cfg) {
  using namespace sr;
  if (!ctx || !cfg) return SR_EINVAL;
  if (n < 0 || t < 1) return fail(ctx, SR_EINVAL, "n < 0 or t < 1");
  if (n == 0) return SR_OK;
  if (!consts || !grad || !m || !v) return fail(ctx, SR_EINVAL, "NULL pointer");
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  // bias corrections on the host: products of t factors, in order
  double p1 = 1.0, p2 = 1.0;
  for (int s = 0; s < t; ++s) {
    p1 *= cfg->beta1;
    p2 *= cfg->beta2;
  }
  adam_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(consts, grad, m, v, n, cfg->lr, cfg->beta1,
                                                         cfg->beta2, cfg->eps, 1.0 - p1, 1.0 - p2);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 1;
  return SR_OK;
}

}  // extern "C"

// sr_eval.cu -- population evaluation: the postfix interpreter with fused
// MSE / 1 - r^2 reductions (sr_eval) and the raw program outputs (sr_predict).
//
// Paper: all genomes of a generation go to the GPU together, each runs a
// batch of fitness cases and one aggregate per genome comes back (Sec.
// 2.1.2); genomes are RPN programs (Sec. 2.1.4); correlation fitness is r of
// Eq. 1, scored here as 1 - r^2 (Sec. 2.1.5).
//
// Layout on the device
//   - A work item is (case chunk c, program p).  Items are handed out
//     chunk-major by an atomic counter to single warps of a persistent grid,
//     so warps running at the same time read the same X columns (L1/L2 hits)
//     and short and long programs balance out dynamically.
//   - A warp decodes its program once per item (warp-parallel scan of the
//     stack effects: validation, stack slots, max depth) into shared memory,
//     then interprets it with lanes over cases, 4 cases per lane (one float4
//     of each X row), 128 cases per step.  The op stream is warp-uniform:
//     no divergence.
//   - Top of stack lives in registers; the rest of the stack in per-warp
//     shared memory slots [slot][lane] (conflict-free float4), or in global
//     scratch for programs deeper than the shared slots.
//   - A terminal followed by a binary op is fused into one instruction
//     "top = top op terminal" (no push, no pop).
//   - Per lane, FP32 Kahan-compensated sums over the item's cases; then FP64
//     warp reduction; one FP64 partial per (program, chunk); a finalize
//     kernel merges the chunks of each program in a fixed order.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "sr_common.cuh"

namespace sr {
namespace {

constexpr int WARPS = 8;        // warps per CTA
constexpr int STEP = 128;       // cases per warp step (32 lanes x float4)
constexpr int DSM = 16;         // stack slots below the top kept in shared memory
constexpr int PSTRIDE = 8;      // doubles per partial record
constexpr int TARGET_ITEMS_PER_WARP = 8;

enum Mode { MODE_PREDICT = 0, MODE_MSE = 1, MODE_CORR = 2, MODE_BOTH = 3 };

// decoded instruction: bits 0..7 opcode, 8..15 operand index, 16..31 slot
enum Op : uint32_t {
  OP_LDV = 0,   // top = x_j                      (first token, empty stack)
  OP_LDC,       // top = c_k
  OP_PUSHV,     // stack[slot] = top; top = x_j
  OP_PUSHC,     // stack[slot] = top; top = c_k
  OP_ADD,       // top = stack[slot] op top
  OP_SUB,
  OP_MUL,
  OP_DIV,
  OP_SIN,       // top = f(top)
  OP_COS,
  OP_EXP,
  OP_LOG,
  OP_SQRT,
  OP_SQ,
  OP_VADD,      // top = top op x_j   (terminal fused with the binary op after it)
  OP_VSUB,
  OP_VMUL,
  OP_VDIV,
  OP_CADD,      // top = top op c_k
  OP_CSUB,
  OP_CMUL,
  OP_CDIV,
};

struct EvalParams {
  const uint8_t *programs;
  const int32_t *lengths;
  const float *consts;
  int P, Lmax, K;
  const float *X;
  const float *y;
  const float *yc;         // centred target (1 - r^2 only), padded with zeros
  int nvars, N;
  long long ldx;
  int chunk, nchunks;
  long long total_items;
  double *partials;        // [P * nchunks][PSTRIDE]
  int32_t *flags;          // [P]
  unsigned long long *queue;
  float *yhat;             // predict: [P][ldy]
  long long ldy;
  float4 *deep_stack;      // per warp: deep_slots * 32 float4
  int deep_slots;
  int warp_bytes;          // shared memory per warp
};

__host__ __device__ inline int warp_smem_bytes(int Lmax) {
  // stack slots | 16 constants | decoded code
  return DSM * 32 * 16 + 64 + ((Lmax * 4 + 15) / 16) * 16;
}

// ---------------------------------------------------------------- operators
__device__ __forceinline__ float op_div(float a, float b) {
  // |b| < 1e-3f in FP32 is exactly "|b| <= 1e-3" for FP32 values of b
  return fabsf(b) < 1e-3f ? 1.0f : a / b;
}
__device__ __forceinline__ float op_log(float x) {
  return fabsf(x) < 1e-3f ? 0.0f : logf(fabsf(x));
}
__device__ __forceinline__ float op_exp(float x) {
  x = x > 80.0f ? 80.0f : (x < -80.0f ? -80.0f : x);  // NaN passes through
  return expf(x);
}

#define MAP4(f, v) make_float4(f((v).x), f((v).y), f((v).z), f((v).w))
#define ZIP4(f, a, b) make_float4(f((a).x, (b).x), f((a).y, (b).y), f((a).z, (b).z), f((a).w, (b).w))

__device__ __forceinline__ float f_add(float a, float b) { return a + b; }
__device__ __forceinline__ float f_sub(float a, float b) { return a - b; }
__device__ __forceinline__ float f_mul(float a, float b) { return a * b; }
__device__ __forceinline__ float f_sqrt(float x) { return sqrtf(fabsf(x)); }
__device__ __forceinline__ float f_sq(float x) { return x * x; }

__device__ __forceinline__ float4 splat(float c) { return make_float4(c, c, c, c); }
__device__ __forceinline__ float4 ldx4(const float *p) {
  return __ldg(reinterpret_cast<const float4 *>(p));
}

// ---------------------------------------------------------------- decode
struct Decoded {
  int n;      // instructions
  int maxd;   // largest stack depth
  int flags;  // SR_PF_* bits
};

// Warp-cooperative validation and decoding of one program into `code`.
__device__ Decoded decode_program(const uint8_t *__restrict__ tok, int L, int Lmax,
                                  int nvars, int K, uint32_t *code, int lane) {
  Decoded d{0, 0, 0};
  if (L < 1 || L > Lmax) {
    d.flags = SR_PF_BAD_LENGTH;
    return d;
  }
  int depth = 0, maxd = 0, n = 0, flags = 0;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int base = 0; base < L; base += 32) {
    const int t = base + lane;
    const bool act = t < L;
    const int v = act ? tok[t] : 255;
    const int vprev = (act && t > 0) ? tok[t - 1] : 255;
    const int vnext = (act && t + 1 < L) ? tok[t + 1] : 255;
    const int cls = tok_class(v);
    const int eff = act ? cls_effect(cls) : 0;
    if (act) {
      if (cls == CLS_BAD) flags |= SR_PF_BAD_TOKEN;
      if (cls == CLS_VAR && v - TOK_VAR0 >= nvars) flags |= SR_PF_BAD_VAR;
      if (cls == CLS_CONST && v - TOK_CONST0 >= K) flags |= SR_PF_BAD_CONST;
    }
    int s = eff;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += u;
    }
    const int after = depth + s;
    const int before = after - eff;
    if (act && after < 1) flags |= SR_PF_UNDERFLOW;
    maxd = max(maxd, __reduce_max_sync(FULL, act ? after : 0));
    const int cn = tok_class(vnext), cp = tok_class(vprev);
    const bool term = cls == CLS_VAR || cls == CLS_CONST;
    const bool head = act && term && cn == CLS_BINARY;
    const bool absorbed = act && cls == CLS_BINARY && (cp == CLS_VAR || cp == CLS_CONST);
    const bool emit = act && !absorbed;
    uint32_t ins = 0;
    if (term) {
      const uint32_t arg = cls == CLS_VAR ? (uint32_t)(v - TOK_VAR0) : (uint32_t)(v - TOK_CONST0);
      if (head) {
        ins = (uint32_t)((cls == CLS_VAR ? OP_VADD : OP_CADD) + vnext) | (arg << 8);
      } else if (before == 0) {
        ins = (uint32_t)(cls == CLS_VAR ? OP_LDV : OP_LDC) | (arg << 8);
      } else {
        ins = (uint32_t)(cls == CLS_VAR ? OP_PUSHV : OP_PUSHC) | (arg << 8) |
              ((uint32_t)(before - 1) << 16);
      }
    } else if (cls == CLS_UNARY) {
      ins = (uint32_t)(OP_SIN + (v - TOK_SIN));
    } else if (cls == CLS_BINARY) {
      ins = (uint32_t)(OP_ADD + v) | ((uint32_t)max(before - 2, 0) << 16);
    }
    const unsigned bal = __ballot_sync(FULL, emit);
    if (emit) code[n + __popc(bal & lt_mask)] = ins;
    n += __popc(bal);
    depth = __shfl_sync(FULL, after, 31);
  }
  flags = __reduce_or_sync(FULL, flags);
  if (depth != 1) flags |= SR_PF_BAD_FINAL;
  d.n = n;
  d.maxd = maxd;
  d.flags = flags;
  return d;
}

// ---------------------------------------------------------------- interpreter
// Runs the decoded program for this lane's 4 cases starting at c0.
// `stk` points at this lane's slot-0 entry; slot s is stk[32 * s].
__device__ __forceinline__ float4 interpret(const uint32_t *__restrict__ code, int n,
                                            const float *__restrict__ cv, float4 *stk,
                                            const float *__restrict__ X, long long ldx, int c0) {
  float4 T = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int ip = 0; ip < n; ++ip) {
    const uint32_t w = code[ip];
    const int arg = (w >> 8) & 0xff;
    float4 *sp = stk + 32 * (int)(w >> 16);
    switch (w & 0xff) {
      case OP_LDV: T = ldx4(X + arg * ldx + c0); break;
      case OP_LDC: T = splat(cv[arg]); break;
      case OP_PUSHV: *sp = T; T = ldx4(X + arg * ldx + c0); break;
      case OP_PUSHC: *sp = T; T = splat(cv[arg]); break;
      case OP_ADD: { float4 a = *sp; T = ZIP4(f_add, a, T); } break;
      case OP_SUB: { float4 a = *sp; T = ZIP4(f_sub, a, T); } break;
      case OP_MUL: { float4 a = *sp; T = ZIP4(f_mul, a, T); } break;
      case OP_DIV: { float4 a = *sp; T = ZIP4(op_div, a, T); } break;
      case OP_SIN: T = MAP4(sinf, T); break;
      case OP_COS: T = MAP4(cosf, T); break;
      case OP_EXP: T = MAP4(op_exp, T); break;
      case OP_LOG: T = MAP4(op_log, T); break;
      case OP_SQRT: T = MAP4(f_sqrt, T); break;
      case OP_SQ: T = MAP4(f_sq, T); break;
      case OP_VADD: { float4 v = ldx4(X + arg * ldx + c0); T = ZIP4(f_add, T, v); } break;
      case OP_VSUB: { float4 v = ldx4(X + arg * ldx + c0); T = ZIP4(f_sub, T, v); } break;
      case OP_VMUL: { float4 v = ldx4(X + arg * ldx + c0); T = ZIP4(f_mul, T, v); } break;
      case OP_VDIV: { float4 v = ldx4(X + arg * ldx + c0); T = ZIP4(op_div, T, v); } break;
      case OP_CADD: { float4 v = splat(cv[arg]); T = ZIP4(f_add, T, v); } break;
      case OP_CSUB: { float4 v = splat(cv[arg]); T = ZIP4(f_sub, T, v); } break;
      case OP_CMUL: { float4 v = splat(cv[arg]); T = ZIP4(f_mul, T, v); } break;
      case OP_CDIV: { float4 v = splat(cv[arg]); T = ZIP4(op_div, T, v); } break;
      default: break;
    }
  }
  return T;
}

// ---------------------------------------------------------------- reductions
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

__device__ __forceinline__ float sel(bool ok, float v) { return ok ? v : 0.0f; }

__device__ __forceinline__ float4 load_y4(const float *__restrict__ y, int c0, int N) {
  if (c0 + 3 < N) return __ldg(reinterpret_cast<const float4 *>(y + c0));
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c0 < N) r.x = y[c0];
  if (c0 + 1 < N) r.y = y[c0 + 1];
  if (c0 + 2 < N) r.z = y[c0 + 2];
  return r;
}

// ---------------------------------------------------------------- one work item
struct WarpSmem {
  float4 *stk_s;    // shared stack slots, [DSM][32] float4
  float *cvals;     // the program's constants
  uint32_t *code;   // decoded instructions
  float4 *stk_g;    // this warp's global stack slots for deep programs
};

__device__ __forceinline__ WarpSmem warp_smem(unsigned char *smem, int warp, int warp_bytes,
                                              float4 *deep_stack, int deep_slots) {
  unsigned char *wbase = smem + (size_t)warp * warp_bytes;
  WarpSmem w;
  w.stk_s = reinterpret_cast<float4 *>(wbase);
  w.cvals = reinterpret_cast<float *>(wbase + DSM * 32 * 16);
  w.code = reinterpret_cast<uint32_t *>(wbase + DSM * 32 * 16 + 64);
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
  w.stk_g = deep_stack ? deep_stack + (size_t)gw * deep_slots * 32 : nullptr;
  return w;
}

// Evaluates program `prog` of problem p on case chunk `c` with the calling
// warp.  MODE_BOTH accumulates the sums selected by `want` (bit 0: squared
// error, bit 1: correlation moments); the other modes ignore `want`.
template <int MODE>
__device__ __forceinline__ void eval_item(const EvalParams &p, int c, int prog, const WarpSmem &w,
                                          int lane, int want) {
  const bool do_mse = MODE == MODE_MSE || (MODE == MODE_BOTH && (want & 1));
  const bool do_corr = MODE == MODE_CORR || (MODE == MODE_BOTH && (want & 2));
  __syncwarp();  // the previous item is done reading code/cvals
  const Decoded dec = decode_program(p.programs + (size_t)prog * p.Lmax, p.lengths[prog], p.Lmax,
                                     p.nvars, p.K, w.code, lane);
  if (lane == 0 && c == 0) p.flags[prog] = dec.flags;
  const int cbeg = c * p.chunk;
  const int cend = min(p.N, cbeg + p.chunk);

  if (dec.flags) {
    if (MODE == MODE_PREDICT) {
      float *row = p.yhat + (size_t)prog * p.ldy;
      for (int i = cbeg + lane; i < cend; i += 32) row[i] = __int_as_float(0x7fc00000);
    }
    return;
  }
  if (lane < p.K) w.cvals[lane] = p.consts[(size_t)prog * p.K + lane];
  __syncwarp();

  float4 *stk = (dec.maxd - 1 <= DSM) ? w.stk_s + lane : w.stk_g + lane;
  const int last_group = (cend - 1) & ~3;

  Kahan se, s1, s2, s3;
  float shift = 0.f;
  for (int base = cbeg; base < cend; base += STEP) {
    const int c0 = base + 4 * lane;
    const int cl = c0 < cend ? c0 : last_group;  // clamped, always readable
    const float4 T = interpret(w.code, dec.n, w.cvals, stk, p.X, p.ldx, cl);
    const bool v0 = c0 < cend, v1 = c0 + 1 < cend, v2 = c0 + 2 < cend, v3 = c0 + 3 < cend;
    if (MODE == MODE_PREDICT) {
      float *row = p.yhat + (size_t)prog * p.ldy;
      if (v0) row[c0] = T.x;
      if (v1) row[c0 + 1] = T.y;
      if (v2) row[c0 + 2] = T.z;
      if (v3) row[c0 + 3] = T.w;
    }
    if (do_mse) {
      const float4 yv = load_y4(p.y, cl, p.N);
      const float e0 = sel(v0, T.x - yv.x), e1 = sel(v1, T.y - yv.y);
      const float e2 = sel(v2, T.z - yv.z), e3 = sel(v3, T.w - yv.w);
      se.add((e0 * e0 + e1 * e1) + (e2 * e2 + e3 * e3));
    }
    if (do_corr) {
      if (base == cbeg) shift = __shfl_sync(FULL, T.x, 0);
      const float4 yv = ldx4(p.yc + cl);
      const float d0 = sel(v0, T.x - shift), d1 = sel(v1, T.y - shift);
      const float d2 = sel(v2, T.z - shift), d3 = sel(v3, T.w - shift);
      s1.add((d0 + d1) + (d2 + d3));
      s2.add((d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3));
      s3.add((d0 * yv.x + d1 * yv.y) + (d2 * yv.z + d3 * yv.w));
    }
  }
  if (MODE != MODE_PREDICT) {
    double *rec = p.partials + ((size_t)prog * p.nchunks + c) * PSTRIDE;
    if (do_mse) {
      const double v = warp_sum(se.value());
      if (lane == 0) rec[0] = v;
    }
    if (do_corr) {
      const double a = warp_sum(s1.value());
      const double b = warp_sum(s2.value());
      const double d = warp_sum(s3.value());
      if (lane == 0) {
        rec[1] = (double)shift;
        rec[2] = a;
        rec[3] = b;
        rec[4] = d;
      }
    }
  }
}

// ---------------------------------------------------------------- single problem
template <int MODE>
__global__ void __launch_bounds__(WARPS * 32) eval_kernel(EvalParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpSmem w = warp_smem(smem, warp, p.warp_bytes, p.deep_stack, p.deep_slots);
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(p.queue, 1ull);
    item = __shfl_sync(FULL, item, 0);
    if ((long long)item >= p.total_items) break;
    const int c = (int)(item / (unsigned long long)p.P);
    const int prog = (int)(item % (unsigned long long)p.P);
    eval_item<MODE>(p, c, prog, w, lane, 3);
  }
}

// ---------------------------------------------------------------- many problems, one launch
constexpr int MAX_BATCH = 64;

struct BatchProblem {
  const uint8_t *programs;
  const int32_t *lengths;
  const float *consts;
  const float *X;
  const float *y;
  float *yc;           // centred target (1 - r^2), padded
  double *partials;    // [P * nchunks][PSTRIDE]
  int32_t *flags;      // [P]
  double *fitness;     // [P] or [2][P]
  double *ychunk;      // [nchunks][2]
  double *stats;       // [8]
  long long ldx;
  long long item_begin;  // first work item of this problem in the launch
  int P, Lmax, K, nvars, N, chunk, nchunks;
  int mode;            // MODE_MSE, MODE_CORR or MODE_BOTH
  int corr_chunk_begin;  // first block of this problem in the batched centring launch (-1: none)
};

struct BatchParams {
  BatchProblem prob[MAX_BATCH];
  int nprob;
  int corr_list[MAX_BATCH];  // problems that need the centred target, in order
  int ncorr;
  long long total_items;
  unsigned long long *queue;
  float4 *deep_stack;
  int deep_slots;
  int warp_bytes;
};

// Work items of every problem come from one atomic counter: problem q owns
// items [item_begin_q, item_begin_q + P_q * nchunks_q), chunk-major inside.
__global__ void __launch_bounds__(WARPS * 32) eval_batched_kernel(const __grid_constant__ BatchParams b) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpSmem w = warp_smem(smem, warp, b.warp_bytes, b.deep_stack, b.deep_slots);
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(b.queue, 1ull);
    item = __shfl_sync(FULL, item, 0);
    if ((long long)item >= b.total_items) break;
    int lo = 0, hi = b.nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.prob[mid].item_begin <= (long long)item) lo = mid;
      else hi = mid - 1;
    }
    const BatchProblem &q = b.prob[lo];
    EvalParams p;
    p.programs = q.programs;
    p.lengths = q.lengths;
    p.consts = q.consts;
    p.P = q.P;
    p.Lmax = q.Lmax;
    p.K = q.K;
    p.X = q.X;
    p.y = q.y;
    p.yc = q.yc;
    p.nvars = q.nvars;
    p.N = q.N;
    p.ldx = q.ldx;
    p.chunk = q.chunk;
    p.nchunks = q.nchunks;
    p.partials = q.partials;
    p.flags = q.flags;
    const long long local = (long long)item - q.item_begin;
    const int c = (int)(local / q.P);
    const int prog = (int)(local % q.P);
    const int want = q.mode == MODE_MSE ? 1 : (q.mode == MODE_CORR ? 2 : 3);
    eval_item<MODE_BOTH>(p, c, prog, w, lane, want);
  }
}

// ---------------------------------------------------------------- target prep (1 - r^2)
constexpr int PREP_THREADS = 512;

__device__ double block_sum(double v, double *red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;  // valid in thread 0
}

// ybar = sum(y) / N in FP64 (one block, fixed order)
__global__ void __launch_bounds__(PREP_THREADS) ymean_kernel(const float *__restrict__ y, int N,
                                                             double *stats) {
  __shared__ double red[PREP_THREADS / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += (double)y[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) stats[0] = s / (double)N;
}

// yc = fl32(y - ybar) per chunk, with its FP64 sum and sum of squares
__global__ void __launch_bounds__(PREP_THREADS) ycenter_kernel(const float *__restrict__ y, int N,
                                                               int chunk, int padded,
                                                               const double *stats, float *yc,
                                                               double *ychunk) {
  __shared__ double red[PREP_THREADS / 32];
  const double ybar = stats[0];
  const int beg = blockIdx.x * chunk, end = min(N, beg + chunk);
  double a = 0.0, b = 0.0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const float v = (float)((double)y[i] - ybar);
    yc[i] = v;
    a += (double)v;
    b += (double)v * (double)v;
  }
  if (blockIdx.x == gridDim.x - 1)
    for (int i = N + threadIdx.x; i < padded; i += blockDim.x) yc[i] = 0.0f;
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    ychunk[2 * blockIdx.x] = a;
    ychunk[2 * blockIdx.x + 1] = b;
  }
}

// ---------------------------------------------------------------- finalize
struct FinalParams {
  const double *partials;
  const int32_t *flags;
  const double *ychunk;
  int P, N, chunk, nchunks;
  double *fitness;  // [P] or [2][P]
};

// 1 - r^2 of one program from its chunk records.
// chunk c: n_c cases, shift s_c, S1 = sum d, S2 = sum d^2, S3 = sum d yc with
// d = yhat - s_c.  Chunk mean m_c = s_c + S1/n_c, chunk M2 = S2 - S1^2/n_c;
// merged (Chan et al.): Shh = sum M2_c + n_c (m_c - m)^2.
// sum yhat*yc = sum (S3_c + s_c Yc_c); Shy = that - m * Y1; Syy = Y2 - Y1^2/N.
__device__ double corr_fitness(const double *rec, const double *ychunk, int Nc, int chunk,
                               int nchunks) {
  const double N = (double)Nc;
  double y1 = 0.0, y2 = 0.0, tot = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    y1 += ychunk[2 * c];
    y2 += ychunk[2 * c + 1];
    const double nc = (double)min(chunk, Nc - c * chunk);
    tot += nc * rec[c * PSTRIDE + 1] + rec[c * PSTRIDE + 2];
  }
  const double m = tot / N;
  double shh = 0.0, g = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const double nc = (double)min(chunk, Nc - c * chunk);
    const double s = rec[c * PSTRIDE + 1], a = rec[c * PSTRIDE + 2];
    const double b = rec[c * PSTRIDE + 3], d = rec[c * PSTRIDE + 4];
    const double mc = s + a / nc;
    shh += (b - a * a / nc) + nc * (mc - m) * (mc - m);
    g += d + s * ychunk[2 * c];
  }
  const double shy = g - m * y1;
  const double syy = y2 - y1 * y1 / N;
  double fit = 1.0;
  if (isfinite(shh) && isfinite(shy) && isfinite(syy) && shh > 0.0 && syy > 0.0 && Nc >= 2) {
    const double r2 = (shy * shy) / (syy * shh);
    fit = 1.0 - r2;
    fit = fit < 0.0 ? 0.0 : (fit > 1.0 ? 1.0 : fit);
  }
  return fit;
}

template <int MODE>
__global__ void finalize_kernel(FinalParams f) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= f.P) return;
  const double INF = __longlong_as_double(0x7ff0000000000000ll);
  double *mse_out = f.fitness;
  double *corr_out = MODE == MODE_BOTH ? f.fitness + f.P : f.fitness;
  if (f.flags[p]) {
    if (MODE == MODE_MSE || MODE == MODE_BOTH) mse_out[p] = INF;
    if (MODE == MODE_CORR || MODE == MODE_BOTH) corr_out[p] = INF;
    return;
  }
  const double *rec = f.partials + (size_t)p * f.nchunks * PSTRIDE;
  const double N = (double)f.N;
  if (MODE == MODE_MSE || MODE == MODE_BOTH) {
    double se = 0.0;
    for (int c = 0; c < f.nchunks; ++c) se += rec[c * PSTRIDE];
    mse_out[p] = isfinite(se) ? se / N : INF;
  }
  if (MODE == MODE_CORR || MODE == MODE_BOTH)
    corr_out[p] = corr_fitness(rec, f.ychunk, f.N, f.chunk, f.nchunks);
}

// ---------------------------------------------------------------- batched prep / finalize
// one block per problem that needs the centred target: its FP64 mean
__global__ void __launch_bounds__(PREP_THREADS) ymean_batched_kernel(const __grid_constant__ BatchParams b) {
  __shared__ double red[PREP_THREADS / 32];
  const BatchProblem &q = b.prob[b.corr_list[blockIdx.x]];
  double s = 0.0;
  for (int i = threadIdx.x; i < q.N; i += blockDim.x) s += (double)q.y[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) q.stats[0] = s / (double)q.N;
}

// one block per (problem, chunk): centred target and its chunk sums
__global__ void __launch_bounds__(PREP_THREADS) ycenter_batched_kernel(const __grid_constant__ BatchParams b) {
  __shared__ double red[PREP_THREADS / 32];
  int r = 0;
  while (r + 1 < b.ncorr && b.prob[b.corr_list[r + 1]].corr_chunk_begin <= (int)blockIdx.x) ++r;
  const BatchProblem &q = b.prob[b.corr_list[r]];
  const int c = (int)blockIdx.x - q.corr_chunk_begin;
  const double ybar = q.stats[0];
  const int beg = c * q.chunk, end = min(q.N, beg + q.chunk);
  double a = 0.0, bb = 0.0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const float v = (float)((double)q.y[i] - ybar);
    q.yc[i] = v;
    a += (double)v;
    bb += (double)v * (double)v;
  }
  if (c == q.nchunks - 1) {
    const int padded = (q.N + STEP - 1) / STEP * STEP;
    for (int i = q.N + threadIdx.x; i < padded; i += blockDim.x) q.yc[i] = 0.0f;
  }
  a = block_sum(a, red);
  bb = block_sum(bb, red);
  if (threadIdx.x == 0) {
    q.ychunk[2 * c] = a;
    q.ychunk[2 * c + 1] = bb;
  }
}

// one block per problem, threads over its programs
__global__ void finalize_batched_kernel(const __grid_constant__ BatchParams b) {
  const BatchProblem &q = b.prob[blockIdx.x];
  FinalParams f{q.partials, q.flags, q.ychunk, q.P, q.N, q.chunk, q.nchunks, q.fitness};
  for (int p0 = 0; p0 < q.P; p0 += blockDim.x) {
    const int p = p0 + threadIdx.x;
    if (p >= q.P) break;
    const double INF = __longlong_as_double(0x7ff0000000000000ll);
    double *mse_out = f.fitness;
    double *corr_out = q.mode == MODE_BOTH ? f.fitness + f.P : f.fitness;
    if (f.flags[p]) {
      if (q.mode != MODE_CORR) mse_out[p] = INF;
      if (q.mode != MODE_MSE) corr_out[p] = INF;
      continue;
    }
    const double *rec = f.partials + (size_t)p * f.nchunks * PSTRIDE;
    const double N = (double)f.N;
    if (q.mode != MODE_CORR) {
      double se = 0.0;
      for (int c = 0; c < f.nchunks; ++c) se += rec[c * PSTRIDE];
      mse_out[p] = isfinite(se) ? se / N : INF;
    }
    if (q.mode != MODE_MSE) corr_out[p] = corr_fitness(rec, f.ychunk, f.N, f.chunk, f.nchunks);
  }
}

// ---------------------------------------------------------------- host side
template <int MODE>
sr_status occupancy_grid(sr_ctx *ctx, int smem, int *grid) {
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(eval_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(eval_kernel)");
    configured = 1;
  }
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_kernel<MODE>, WARPS * 32, smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (nb < 1) return fail(ctx, SR_EINVAL, "Lmax too large for shared memory");
  *grid = nb * ctx->num_sms;
  return SR_OK;
}

sr_status grid_for(sr_ctx *ctx, int mode, int smem, int *grid) {
  switch (mode) {
    case MODE_PREDICT: return occupancy_grid<MODE_PREDICT>(ctx, smem, grid);
    case MODE_MSE: return occupancy_grid<MODE_MSE>(ctx, smem, grid);
    case MODE_CORR: return occupancy_grid<MODE_CORR>(ctx, smem, grid);
    default: return occupancy_grid<MODE_BOTH>(ctx, smem, grid);
  }
}

struct Plan {
  int grid, smem, chunk, nchunks, deep_slots;
  long long items;
  size_t off_queue, off_flags, off_part, off_yc, off_ych, off_stats, off_deep, bytes;
};

sr_status make_plan(sr_ctx *ctx, int mode, int P, int Lmax, int N, Plan *pl) {
  pl->smem = WARPS * warp_smem_bytes(Lmax);
  sr_status st = grid_for(ctx, mode, pl->smem, &pl->grid);
  if (st != SR_OK) return st;
  const long long warps = (long long)pl->grid * WARPS;
  const long long want = warps * TARGET_ITEMS_PER_WARP;
  int nch = (int)((want + P - 1) / (P > 0 ? P : 1));
  const int max_chunks = (N + 1023) / 1024;
  nch = nch < 1 ? 1 : (nch > max_chunks ? max_chunks : nch);
  int chunk = (N + nch - 1) / nch;
  if (ctx->tile_cases > 0) chunk = ctx->tile_cases;  // autotuned cases per work item
  chunk = (chunk + STEP - 1) / STEP * STEP;
  pl->chunk = chunk;
  pl->nchunks = (N + chunk - 1) / chunk;
  pl->items = (long long)P * pl->nchunks;
  const int max_depth = (Lmax + 1) / 2;
  pl->deep_slots = max_depth - 1 > DSM ? max_depth - 1 : 0;
  Carver cv;
  pl->off_queue = cv.take(256);
  pl->off_flags = cv.take((size_t)P * 4);
  pl->off_part = cv.take((size_t)pl->items * PSTRIDE * 8);
  const size_t padded = align_up((size_t)N, STEP);
  pl->off_yc = cv.take(padded * 4);
  pl->off_ych = cv.take((size_t)pl->nchunks * 16);
  pl->off_stats = cv.take(64);
  pl->off_deep = cv.take((size_t)warps * pl->deep_slots * 32 * 16);
  pl->bytes = cv.off;
  return SR_OK;
}

sr_status check_common(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths,
                       const float *consts, int P, int Lmax, int K, const float *X, int nvars,
                       int N, int ldx) {
  if (!ctx) return SR_EINVAL;
  if (P < 0) return fail(ctx, SR_EINVAL, "P < 0");
  if (Lmax < 1 || Lmax > SR_MAX_LMAX) return fail(ctx, SR_EINVAL, "Lmax %d outside [1, %d]", Lmax, SR_MAX_LMAX);
  if (K < 0 || K > SR_MAX_CONSTS) return fail(ctx, SR_EINVAL, "K %d outside [0, %d]", K, SR_MAX_CONSTS);
  if (nvars < 1 || nvars > SR_MAX_VARS) return fail(ctx, SR_EINVAL, "nvars %d outside [1, %d]", nvars, SR_MAX_VARS);
  if (N < 1) return fail(ctx, SR_EINVAL, "N must be >= 1");
  if (ldx < N || ldx % 4) return fail(ctx, SR_EINVAL, "ldx %d must be >= N and a multiple of 4", ldx);
  if (P > 0 && (!programs || !lengths || (K > 0 && !consts) || !X))
    return fail(ctx, SR_EINVAL, "NULL input pointer");
  if (((uintptr_t)X) & 15) return fail(ctx, SR_EINVAL, "X must be 16-byte aligned");
  return SR_OK;
}

sr_status launch_eval(sr_ctx *ctx, int mode, const uint8_t *programs, const int32_t *lengths,
                      const float *consts, int P, int Lmax, int K, const float *X, const float *y,
                      int nvars, int N, int ldx, double *fitness, int32_t *prog_flags, float *yhat,
                      int ldy) {
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  Plan pl;
  sr_status st = make_plan(ctx, mode, P, Lmax, N, &pl);
  if (st != SR_OK) return st;
  st = ensure_workspace(ctx, pl.bytes);
  if (st != SR_OK) return st;
  char *ws = ctx->ws;
  cudaStream_t s = ctx->stream;

  EvalParams ep;
  ep.programs = programs;
  ep.lengths = lengths;
  ep.consts = consts;
  ep.P = P;
  ep.Lmax = Lmax;
  ep.K = K;
  ep.X = X;
  ep.y = y;
  ep.yc = reinterpret_cast<const float *>(ws + pl.off_yc);
  ep.nvars = nvars;
  ep.N = N;
  ep.ldx = ldx;
  ep.chunk = pl.chunk;
  ep.nchunks = pl.nchunks;
  ep.total_items = pl.items;
  ep.partials = reinterpret_cast<double *>(ws + pl.off_part);
  ep.flags = prog_flags ? prog_flags : reinterpret_cast<int32_t *>(ws + pl.off_flags);
  ep.queue = reinterpret_cast<unsigned long long *>(ws + pl.off_queue);
  ep.yhat = yhat;
  ep.ldy = ldy;
  ep.deep_stack = pl.deep_slots ? reinterpret_cast<float4 *>(ws + pl.off_deep) : nullptr;
  ep.deep_slots = pl.deep_slots;
  ep.warp_bytes = warp_smem_bytes(Lmax);

  SR_CHECK_CUDA(ctx, cudaMemsetAsync(ep.queue, 0, sizeof(unsigned long long), s));
  double *ych = reinterpret_cast<double *>(ws + pl.off_ych);
  if (mode == MODE_CORR || mode == MODE_BOTH) {
    double *stats = reinterpret_cast<double *>(ws + pl.off_stats);
    ymean_kernel<<<1, PREP_THREADS, 0, s>>>(y, N, stats);
    ycenter_kernel<<<pl.nchunks, PREP_THREADS, 0, s>>>(y, N, pl.chunk, (int)align_up(N, STEP), stats,
                                                      const_cast<float *>(ep.yc), ych);
    ctx->launches += 2;
  }
  switch (mode) {
    case MODE_PREDICT: eval_kernel<MODE_PREDICT><<<pl.grid, WARPS * 32, pl.smem, s>>>(ep); break;
    case MODE_MSE: eval_kernel<MODE_MSE><<<pl.grid, WARPS * 32, pl.smem, s>>>(ep); break;
    case MODE_CORR: eval_kernel<MODE_CORR><<<pl.grid, WARPS * 32, pl.smem, s>>>(ep); break;
    default: eval_kernel<MODE_BOTH><<<pl.grid, WARPS * 32, pl.smem, s>>>(ep); break;
  }
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 1;
  if (mode != MODE_PREDICT) {
    FinalParams fp{ep.partials, ep.flags, ych, P, N, pl.chunk, pl.nchunks, fitness};
    const int nb = (P + 255) / 256;
    switch (mode) {
      case MODE_MSE: finalize_kernel<MODE_MSE><<<nb, 256, 0, s>>>(fp); break;
      case MODE_CORR: finalize_kernel<MODE_CORR><<<nb, 256, 0, s>>>(fp); break;
      default: finalize_kernel<MODE_BOTH><<<nb, 256, 0, s>>>(fp); break;
    }
    SR_CHECK_CUDA(ctx, cudaGetLastError());
    ctx->launches += 1;
  }
  return SR_OK;
}

// ---------------------------------------------------------------- batched host side
struct BatchPlan {
  int grid, smem, deep_slots, maxL;
};

sr_status batched_grid(sr_ctx *ctx, int smem, int *grid) {
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(eval_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(eval_batched_kernel)");
    configured = 1;
  }
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_batched_kernel, WARPS * 32, smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (nb < 1) return fail(ctx, SR_EINVAL, "Lmax too large for shared memory");
  *grid = nb * ctx->num_sms;
  return SR_OK;
}

int mode_of(sr_fitness_kind k) {
  return k == SR_MSE ? MODE_MSE : (k == SR_CORR ? MODE_CORR : MODE_BOTH);
}

sr_status launch_batched(sr_ctx *ctx, const sr_problem *pr, int nprob) {
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  int maxL = 1;
  double work = 0.0;
  for (int i = 0; i < nprob; ++i) {
    const sr_problem &q = pr[i];
    sr_status st = check_common(ctx, q.programs, q.lengths, q.consts, q.P, q.Lmax, q.K, q.X, q.nvars,
                                q.N, q.ldx);
    if (st != SR_OK) return fail(ctx, st, "problem %d: %s", i, ctx->msg);
    if (q.kind != SR_MSE && q.kind != SR_CORR && q.kind != SR_MSE_CORR)
      return fail(ctx, SR_EINVAL, "problem %d: unknown fitness kind", i);
    if (q.P > 0 && (!q.y || !q.fitness || (((uintptr_t)q.y) & 15)))
      return fail(ctx, SR_EINVAL, "problem %d: y NULL or not 16-byte aligned, or fitness NULL", i);
    if (q.cases_per_tile < 0) return fail(ctx, SR_EINVAL, "problem %d: cases_per_tile < 0", i);
    maxL = q.Lmax > maxL ? q.Lmax : maxL;
    work += (double)q.P * (double)q.N;
  }
  BatchPlan bp;
  bp.maxL = maxL;
  bp.smem = WARPS * warp_smem_bytes(maxL);
  sr_status st = batched_grid(ctx, bp.smem, &bp.grid);
  if (st != SR_OK) return st;
  const long long warps = (long long)bp.grid * WARPS;
  const double want = (double)warps * TARGET_ITEMS_PER_WARP;
  const int max_depth = (maxL + 1) / 2;
  bp.deep_slots = max_depth - 1 > DSM ? max_depth - 1 : 0;

  // chunking per problem: items in proportion to its share of the work
  std::vector<int> chunk(nprob), nch(nprob), order;
  for (int i = 0; i < nprob; ++i) {
    const sr_problem &q = pr[i];
    if (q.P == 0) continue;
    int c;
    if (q.cases_per_tile > 0) {
      c = q.cases_per_tile;
    } else {
      const double share = want * ((double)q.P * (double)q.N) / (work > 0 ? work : 1.0);
      int n = (int)ceil(share / q.P);
      const int max_chunks = (q.N + 1023) / 1024;
      n = n < 1 ? 1 : (n > max_chunks ? max_chunks : n);
      c = (q.N + n - 1) / n;
    }
    c = (c + STEP - 1) / STEP * STEP;
    chunk[i] = c;
    nch[i] = (q.N + c - 1) / c;
    order.push_back(i);
  }
  // longest items first (cases per item x longest program), so the tail of
  // the launch is made of short items
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)chunk[a] * pr[a].Lmax > (double)chunk[b] * pr[b].Lmax;
  });

  // workspace: the largest group decides (all groups reuse it in turn)
  auto group_bytes = [&](size_t g0, size_t g1, BatchParams *bpar) -> size_t {
    Carver cv;
    const size_t off_q = cv.take(256);
    const size_t off_deep = cv.take((size_t)warps * bp.deep_slots * 32 * 16);
    long long items = 0;
    int corr_chunks = 0, ncorr = 0;
    for (size_t g = g0; g < g1; ++g) {
      const int i = order[g];
      const sr_problem &q = pr[i];
      const int mode = mode_of(q.kind);
      const size_t off_f = q.prog_flags ? 0 : cv.take((size_t)q.P * 4);
      const size_t off_p = cv.take((size_t)q.P * nch[i] * PSTRIDE * 8);
      size_t off_yc = 0, off_ych = 0, off_st = 0;
      const bool corr = mode != MODE_MSE;
      if (corr) {
        off_yc = cv.take(align_up((size_t)q.N, STEP) * 4);
        off_ych = cv.take((size_t)nch[i] * 16);
        off_st = cv.take(64);
      }
      if (bpar) {
        BatchProblem &b = bpar->prob[g - g0];
        char *ws = ctx->ws;
        b.programs = q.programs;
        b.lengths = q.lengths;
        b.consts = q.consts;
        b.X = q.X;
        b.y = q.y;
        b.yc = corr ? reinterpret_cast<float *>(ws + off_yc) : nullptr;
        b.partials = reinterpret_cast<double *>(ws + off_p);
        b.flags = q.prog_flags ? q.prog_flags : reinterpret_cast<int32_t *>(ws + off_f);
        b.fitness = q.fitness;
        b.ychunk = corr ? reinterpret_cast<double *>(ws + off_ych) : nullptr;
        b.stats = corr ? reinterpret_cast<double *>(ws + off_st) : nullptr;
        b.ldx = q.ldx;
        b.item_begin = items;
        b.P = q.P;
        b.Lmax = q.Lmax;
        b.K = q.K;
        b.nvars = q.nvars;
        b.N = q.N;
        b.chunk = chunk[i];
        b.nchunks = nch[i];
        b.mode = mode;
        b.corr_chunk_begin = corr ? corr_chunks : -1;
        if (corr) bpar->corr_list[ncorr] = (int)(g - g0);
      }
      items += (long long)q.P * nch[i];
      if (corr) {
        corr_chunks += nch[i];
        ++ncorr;
      }
    }
    if (bpar) {
      bpar->nprob = (int)(g1 - g0);
      bpar->ncorr = ncorr;
      bpar->total_items = items;
      bpar->queue = reinterpret_cast<unsigned long long *>(ctx->ws + off_q);
      bpar->deep_stack = bp.deep_slots ? reinterpret_cast<float4 *>(ctx->ws + off_deep) : nullptr;
      bpar->deep_slots = bp.deep_slots;
      bpar->warp_bytes = warp_smem_bytes(maxL);
    }
    return cv.off;
  };
  size_t need = 0;
  for (size_t g0 = 0; g0 < order.size(); g0 += MAX_BATCH) {
    const size_t g1 = std::min(order.size(), g0 + MAX_BATCH);
    need = std::max(need, group_bytes(g0, g1, nullptr));
  }
  if (order.empty()) return SR_OK;
  st = ensure_workspace(ctx, need);
  if (st != SR_OK) return st;

  cudaStream_t s = ctx->stream;
  for (size_t g0 = 0; g0 < order.size(); g0 += MAX_BATCH) {
    const size_t g1 = std::min(order.size(), g0 + MAX_BATCH);
    BatchParams b;
    group_bytes(g0, g1, &b);
    int corr_blocks = 0;
    for (int r = 0; r < b.ncorr; ++r) corr_blocks += b.prob[b.corr_list[r]].nchunks;
    SR_CHECK_CUDA(ctx, cudaMemsetAsync(b.queue, 0, sizeof(unsigned long long), s));
    if (b.ncorr > 0) {
      ymean_batched_kernel<<<b.ncorr, PREP_THREADS, 0, s>>>(b);
      ycenter_batched_kernel<<<corr_blocks, PREP_THREADS, 0, s>>>(b);
      ctx->launches += 2;
    }
    eval_batched_kernel<<<bp.grid, WARPS * 32, bp.smem, s>>>(b);
    finalize_batched_kernel<<<b.nprob, 256, 0, s>>>(b);
    SR_CHECK_CUDA(ctx, cudaGetLastError());
    ctx->launches += 2;
  }
  return SR_OK;
}

}  // namespace
}  // namespace sr

extern "C" {

sr_status sr_eval(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths, const float *consts,
                  int P, int Lmax, int K, const float *X, const float *y, int nvars, int N, int ldx,
                  sr_fitness_kind kind, double *fitness, int32_t *prog_flags) {
  using namespace sr;
  sr_status st = check_common(ctx, programs, lengths, consts, P, Lmax, K, X, nvars, N, ldx);
  if (st != SR_OK) return st;
  if (kind != SR_MSE && kind != SR_CORR && kind != SR_MSE_CORR)
    return fail(ctx, SR_EINVAL, "unknown fitness kind %d", (int)kind);
  if (P == 0) return SR_OK;
  if (!y || !fitness) return fail(ctx, SR_EINVAL, "NULL y or fitness");
  if (((uintptr_t)y) & 15) return fail(ctx, SR_EINVAL, "y must be 16-byte aligned");
  const int mode = kind == SR_MSE ? MODE_MSE : (kind == SR_CORR ? MODE_CORR : MODE_BOTH);
  return launch_eval(ctx, mode, programs, lengths, consts, P, Lmax, K, X, y, nvars, N, ldx,
                     fitness, prog_flags, nullptr, 0);
}

sr_status sr_predict(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths,
                     const float *consts, int P, int Lmax, int K, const float *X, int nvars, int N,
                     int ldx, float *yhat, int ldy, int32_t *prog_flags) {
  using namespace sr;
  sr_status st = check_common(ctx, programs, lengths, consts, P, Lmax, K, X, nvars, N, ldx);
  if (st != SR_OK) return st;
  if (P == 0) return SR_OK;
  if (!yhat || ldy < N) return fail(ctx, SR_EINVAL, "yhat NULL or ldy < N");
  return launch_eval(ctx, MODE_PREDICT, programs, lengths, consts, P, Lmax, K, X, nullptr, nvars,
                     N, ldx, nullptr, prog_flags, yhat, ldy);
}

sr_status sr_eval_batched(sr_ctx *ctx, const sr_problem *problems, int nprob) {
  using namespace sr;
  if (!ctx) return SR_EINVAL;
  if (nprob < 0 || (nprob > 0 && !problems)) return fail(ctx, SR_EINVAL, "bad problem list");
  if (nprob == 0) return SR_OK;
  return launch_batched(ctx, problems, nprob);
}

sr_status sr_set_tile(sr_ctx *ctx, int cases_per_tile) {
  if (!ctx || cases_per_tile < 0) return SR_EINVAL;
  ctx->tile_cases = cases_per_tile;
  return SR_OK;
}

sr_status sr_reserve(sr_ctx *ctx, int P, int Lmax, int N) {
  using namespace sr;
  if (!ctx || P < 0 || Lmax < 1 || Lmax > SR_MAX_LMAX || N < 1) return SR_EINVAL;
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t need = 0;
  for (int mode = 0; mode < 4; ++mode) {
    Plan pl;
    sr_status st = make_plan(ctx, mode, P, Lmax, N, &pl);
    if (st != SR_OK) return st;
    need = pl.bytes > need ? pl.bytes : need;
  }
  return ensure_workspace(ctx, need);
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free evaluation
// sr_eval_noalloc: the same kernels as sr_eval, with every byte of scratch
// taken from one file-scope device array instead of a context workspace.
#include <mutex>

namespace sr {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;  // 16 MiB, held per device until exit
constexpr int NOALLOC_MAX_DEVICES = 64;

__device__ __align__(256) char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mutex;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES];  // device address of the array, per device

// Looks up the device address of the scratch array on the current device
// (once per device; the host-side symbol is not a device address).
sr_status noalloc_scratch(int dev, void **out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SR_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SR_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return SR_OK;
}

}  // namespace
}  // namespace sr

extern "C" sr_status sr_eval_noalloc(void *cuda_stream, const uint8_t *programs,
                                     const int32_t *lengths, const float *consts, int P, int Lmax,
                                     int K, const float *X, const float *y, int nvars, int N,
                                     int ldx, sr_fitness_kind kind, double *fitness,
                                     int32_t *prog_flags) {
  using namespace sr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SR_ECUDA;
  }
  // a context on the stack: nothing is allocated for it, and its workspace
  // is the static array, so the workspace never needs to grow
  sr_ctx local;
  local.device = dev;
  local.stream = (cudaStream_t)cuda_stream;
  if (cudaDeviceGetAttribute(&local.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SR_ECUDA;
  }
  sr_status st = check_common(&local, programs, lengths, consts, P, Lmax, K, X, nvars, N, ldx);
  if (st != SR_OK) return st;
  if (kind != SR_MSE && kind != SR_CORR && kind != SR_MSE_CORR) return SR_EINVAL;
  if (P == 0) return SR_OK;
  if (!y || !fitness || (((uintptr_t)y) & 15)) return SR_EINVAL;
  const int mode = kind == SR_MSE ? MODE_MSE : (kind == SR_CORR ? MODE_CORR : MODE_BOTH);
  // fit the plan into the array: fewer SMs' worth of persistent CTAs means
  // fewer per-warp stacks and partial records
  Plan pl;
  for (;;) {
    st = make_plan(&local, mode, P, Lmax, N, &pl);
    if (st != SR_OK) return st;
    if (pl.bytes <= NOALLOC_SCRATCH_BYTES) break;
    if (local.num_sms == 1) return SR_ENOMEM;  // does not fit even on one SM
    local.num_sms = local.num_sms / 2 > 0 ? local.num_sms / 2 : 1;
  }
  void *scratch = nullptr;
  st = noalloc_scratch(dev, &scratch);
  if (st != SR_OK) return st;
  local.ws = static_cast<char *>(scratch);
  local.ws_bytes = NOALLOC_SCRATCH_BYTES;
  return launch_eval(&local, mode, programs, lengths, consts, P, Lmax, K, X, y, nvars, N, ldx,
                     fitness, prog_flags, nullptr, 0);
}

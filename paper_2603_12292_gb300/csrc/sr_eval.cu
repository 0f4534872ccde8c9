// sr_eval.cu -- population evaluation: the postfix interpreter with fused
// MSE / 1 - r^2 reductions (sr_eval, sr_eval_batched) and the raw program
// outputs (sr_predict).
//
// Paper: all genomes of a generation go to the GPU together, each runs a
// batch of fitness cases and one aggregate per genome comes back (Sec.
// 2.1.2); genomes are RPN programs (Sec. 2.1.4); correlation fitness is r of
// Eq. 1, scored here as 1 - r^2 (Sec. 2.1.5).
//
// Design on the device
//   1. Decode pre-pass, a warp per program (lane 0 walks the tree in shared
//      memory): validation, then the expression tree is rescheduled
//      Sethi-Ullman style -- at every binary node the child that needs more
//      stack is evaluated first (a reversed opcode keeps a - b and a / b
//      exact when the right child goes first).  The stack depth of any
//      program is then at most floor(log2(leaves)) + 1 (9 for 512 tokens), so
//      floor(log2((Lmax + 1) / 2)) slots always suffice; most programs need
//      far fewer, so the main passes give each warp only what fits 4 or 5
//      CTAs per SM and the rare deeper programs run in a third pass.
//      A terminal evaluated second is fused into its binary operator
//      ("top = top op x_j"), and every operand is resolved here (constant
//      value, X row offset, stack-slot byte offset): the interpreter does no
//      per-token address or index arithmetic.  Values are bit-identical to
//      plain left-to-right evaluation (same operation on the same operands).
//   2. Evaluation, persistent grid: a work item is (case chunk, program),
//      handed out chunk-major by one atomic counter to single warps, so
//      warps running together share X columns in L1/L2 and uneven program
//      lengths balance out.  The warp copies the program's code into shared
//      memory and interprets it with lanes over cases, 8 cases per lane (two
//      float4 per operand), 256 cases per step; the op stream is
//      warp-uniform (no divergence).  Top of stack in registers, the slots
//      below in shared memory [slot][half][lane] (conflict-free float4).
//   3. Per lane, FP32 Kahan-compensated sums over the item's cases; FP64 warp
//      reduction; one FP64 partial per (program, chunk); a finalize kernel
//      merges the chunks of each program (a warp per program, fixed order).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "sr_common.cuh"
#include "sr_interp.cuh"

namespace sr {
namespace {

constexpr int WARPS = 8;        // warps per CTA (measured best of 4, 8, 16 warps per CTA)
constexpr int CPL = 8;          // cases per lane per dispatched instruction (two float4)
constexpr int STEP = 32 * CPL;  // cases per warp step
constexpr int SLOT_BYTES = 32 * CPL * 4;  // one stack slot of a warp: [2][32 lanes] float4
constexpr int PSTRIDE = 8;      // doubles per partial record
// Calls of at least this many cases and programs read the unary transforms
// of the variables from a table (sr_set_transforms' automatic mode); below
// that the table's launch and copy cost more than the few programs sharing
// each row save.
constexpr int XFORM_MIN_N = 16384, XFORM_MIN_P = 64;
// The compositions u(v(x_j)) join the table while it stays within this size
// (a call), and while a batch's tables with them stay within the second.
constexpr long long XFORM2_MAX_BYTES = 2ll << 30, XFORM2_BATCH_BYTES = 16ll << 30;
// A work item's slice of the table (its rows over the item's cases) is kept
// within this size when the library picks the cases per item, so that the
// items running at one time share a part of the table that stays in L2:
// on 262,144 programs x 10^6 cases, one item per program read the 520 MB
// table from DRAM, 3,961 GPop/s; 64k cases per item 4,236.
constexpr long long XFORM_SLICE_BYTES = 32ll << 20;
constexpr int TARGET_ITEMS_PER_WARP = 16;  // balances the launch tail; measured best of 8 to 28 at 4,096 x 100k
// Occupancy variants of the evaluation kernel: MINB CTAs of WARPS warps per
// SM.  Shared memory per CTA that leaves room for MINB of them (228 KB per
// SM, 1 KB of it reserved per CTA); the registers are bounded to match
// (5 CTAs: 48 registers).  Measured on 4,096 programs x 100,000 cases
// (Lmax 128): 5 CTAs with 4 stack slots 2,579 -> 2,649 GPop/s, Table 1
// operators 1,432 -> 1,592; at Lmax 256 the 48-register bound costs more than
// it gives (2,810 -> 2,625), so there it stays at 4 CTAs.
// (228 KB / MINB - 1 KB, rounded down to 512 bytes: 3 -> 76,800, 4 -> 57,344,
// 5 -> 45,568)
__host__ __device__ constexpr int smem_target(int minb) { return (233472 / minb - 1024) / 512 * 512; }

enum Mode { MODE_PREDICT = 0, MODE_MSE = 1, MODE_CORR = 2, MODE_BOTH = 3, MODE_R4 = 4, MODE_P2P = 5 };

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
  uint2 *code;             // [P][Lmax] decoded instructions
  int32_t *ncode;          // [P]
  // [0] work counter, [1] work counter of the EXT pass, [2] EXT programs,
  // [3] work counter of the deep pass, [4] deep programs
  unsigned long long *queue;
  float *yhat;             // predict: [P][ldy]
  long long ldy;
  int warp_bytes;          // shared memory per warp
  int slots;               // stack slots per warp
  int deep;                // 1: this launch is the pass of the NCODE_DEEP programs
  int score_M;             // Beagle scores: the maximum score per case
  const int32_t *abort;    // sr_set_abort_flag (or NULL)
  unsigned *err;           // the context's latched error word
  int xform = 0;           // >= 1: X is the variable table of this depth (DecodeArgs::xform)
  uint8_t *xneed = nullptr;  // the transforms some program reads
};

__host__ __device__ inline int code_smem_bytes(int Lmax) { return ((Lmax * 8 + 15) / 16) * 16; }

__host__ __device__ inline int warp_smem_bytes(int slots, int Lmax) {
  // stack slots | decoded code (8 bytes per token)
  return slots * SLOT_BYTES + code_smem_bytes(Lmax);
}

// Stack slots of the main evaluation passes: as many as fit smem_target(minb),
// at most slots_for(Lmax) and at least min(slots_for(Lmax), 4).  Programs of
// up to 256 tokens, random or evolved, rarely need more than 4 (Sethi-Ullman
// order) while slots_for(256) = 7 would leave room for only 3 CTAs per SM;
// the few that need more than the main passes give (NCODE_DEEP) run in a
// third pass with slots_for(Lmax) slots.
__host__ __device__ inline int shallow_slots(int Lmax, int minb) {
  const int full = slots_for(Lmax), lo = full < 4 ? full : 4;
  const int s = (smem_target(minb) / WARPS - code_smem_bytes(Lmax)) / SLOT_BYTES;
  return s < lo ? lo : (s > full ? full : s);
}

// 5 CTAs per SM where they fit with at least min(slots_for(Lmax), 4) slots
// (Lmax <= 200), else 4.
inline int minb_for(int Lmax) {
  return WARPS * warp_smem_bytes(shallow_slots(Lmax, 5), Lmax) <= smem_target(5) ? 5 : 4;
}
// The evaluation's CTAs per SM: the tuned choice where it fits, else the
// automatic one
inline int eval_minb(int Lmax, int tuned) {
  if (tuned == 5) return minb_for(Lmax);
  if (tuned == 4) return 4;
  return minb_for(Lmax);
}

// ---------------------------------------------------------------- operators
#define MAP4(f, v) make_float4(f((v).x), f((v).y), f((v).z), f((v).w))
#define ZIP4(f, a, b) make_float4(f((a).x, (b).x), f((a).y, (b).y), f((a).z, (b).z), f((a).w, (b).w))

__device__ __forceinline__ float f_add(float a, float b) { return a + b; }
__device__ __forceinline__ float f_sub(float a, float b) { return a - b; }
__device__ __forceinline__ float f_mul(float a, float b) { return a * b; }
__device__ __forceinline__ float f_sq(float x) { return x * x; }

__device__ __forceinline__ float4 splat(float c) { return make_float4(c, c, c, c); }
__device__ __forceinline__ float4 ldx4(const float *p) {
  return __ldg(reinterpret_cast<const float4 *>(p));
}

// ---------------------------------------------------------------- decode pre-pass
// cap_slots: programs that need more get NCODE_DEEP, counted in deep_count
__device__ __forceinline__ DecodeArgs decode_args(const EvalParams &p, int cap_slots,
                                                  unsigned long long *deep_count) {
  DecodeArgs a;
  a.programs = p.programs;
  a.lengths = p.lengths;
  a.consts = p.consts;
  a.Lmax = p.Lmax;
  a.K = p.K;
  a.nvars = p.nvars;
  a.ldx = p.ldx;
  a.slot_bytes = SLOT_BYTES;
  a.code = p.code;
  a.ncode = p.ncode;
  a.flags = p.flags;
  a.ext_count = p.queue ? p.queue + 2 : nullptr;
  a.max_slots = slots_for(p.Lmax);
  a.cap_slots = cap_slots;
  a.deep_count = deep_count;
  a.fold = 1;  // constant-only subtrees are evaluated once, in the decoder
  a.adj_info = 0;
  a.xform = p.xform;
  a.xneed = p.xneed;
  return a;
}

// one warp per program, scratch in shared memory (decode_warp)
__global__ void decode_kernel(EvalParams p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  decode_warp(decode_args(p, p.slots, p.queue + 4), p.P, dsm);
}

// The variable table of an evaluation with transforms (DecodeArgs::xform):
// row j < nvars is x_j, row xform_row(nvars, u, j) is u(x_j) and row
// xform_row2(nvars, u, v, j) is u(v(x_j)), for the rows some program reads
// (xneed, marked by the decoder), by the interpreter's own FP32 functions
// (fold_op), so a program reads the bits its own per-case evaluation would
// give.  Blocks: (case group of XF_THREADS * 4 cases, row).
constexpr int XF_THREADS = 256;
__global__ void __launch_bounds__(XF_THREADS)
    xform_kernel(const float *__restrict__ X, long long ldx, int nvars, int N, int ldxt,
                 const uint8_t *__restrict__ xneed, float *__restrict__ xt) {
  const int r = blockIdx.y;
  if (r >= nvars && !xneed[r - nvars]) return;
  const int c = (blockIdx.x * XF_THREADS + threadIdx.x) * 4;
  if (c >= N) return;  // c + 3 < ldx and < ldxt: both are multiples of 4 and >= N
  const int r2 = nvars * (1 + UNARY_ALL);  // first composition row
  int u = -1, v = -1, j = r;
  if (r >= r2) {
    const int k = (r - r2) / nvars;
    j = (r - r2) % nvars;
    u = TOK_SIN + k / XFORM_BASE;
    v = TOK_SIN + k % XFORM_BASE;
  } else if (r >= nvars) {
    u = TOK_SIN + (r - nvars) / nvars;
    j = (r - nvars) % nvars;
  }
  float4 x = ldx4(X + (size_t)j * ldx + c);
  if (v >= 0)
    x = make_float4(fold_op(v, x.x, 0.f), fold_op(v, x.y, 0.f), fold_op(v, x.z, 0.f), fold_op(v, x.w, 0.f));
  if (u >= 0)
    x = make_float4(fold_op(u, x.x, 0.f), fold_op(u, x.y, 0.f), fold_op(u, x.z, 0.f), fold_op(u, x.w, 0.f));
  *reinterpret_cast<float4 *>(xt + (size_t)r * ldxt + c) = x;
}

// ---------------------------------------------------------------- interpreter
// CPL = 8 cases per lane: the value on top of the stack is two float4 (a: the
// lane's cases 0-3, b: cases 4-7); a stack slot holds the same for every
// lane as [slot][half][lane] float4, so each 128-bit access of a warp covers
// 512 contiguous bytes (no bank conflicts).
struct V8 {
  float4 a, b;
};

__device__ __forceinline__ V8 splat8(float c) {
  V8 r;
  r.a = splat(c);
  r.b = r.a;
  return r;
}
#define MAP8(f, v) V8{MAP4(f, (v).a), MAP4(f, (v).b)}
#define ZIP8(f, p, q) V8{ZIP4(f, (p).a, (q).a), ZIP4(f, (p).b, (q).b)}

__device__ __forceinline__ V8 ld8(const char *stk, uint32_t off) {
  V8 r;
  r.a = *reinterpret_cast<const float4 *>(stk + off);
  r.b = *reinterpret_cast<const float4 *>(stk + off + 32 * 16);
  return r;
}
__device__ __forceinline__ void st8(char *stk, uint32_t off, const V8 &v) {
  *reinterpret_cast<float4 *>(stk + off) = v.a;
  *reinterpret_cast<float4 *>(stk + off + 32 * 16) = v.b;
}
__device__ __forceinline__ V8 ldX8(const float *xa, const float *xb, uint32_t off) {
  return V8{ldx4(xa + off), ldx4(xb + off)};
}

#ifndef SR_MATH_UNROLL
#define SR_MATH_UNROLL 8
#endif
constexpr int MATH_UNROLL = SR_MATH_UNROLL;
// The costly operators (the FP32 math library routines and the quotient)
// live out of line, one copy each, so the interpreter's dispatch loop stays
// small enough for the instruction cache; inside, SR_MATH_UNROLL values are
// in flight at a time.  Measured on the 4096 x 100,000 mixed population:
// everything inlined ~1,450 GPop/s, out of line with 4 in flight ~1,530,
// with 8 in flight ~2,200.
struct FSin { __device__ __forceinline__ float operator()(float x) const { return f_sin(x); } };
struct FCos { __device__ __forceinline__ float operator()(float x) const { return f_cos(x); } };
struct FExp { __device__ __forceinline__ float operator()(float x) const { return op_exp(x); } };
struct FLog { __device__ __forceinline__ float operator()(float x) const { return op_log(x); } };
struct FSqrt { __device__ __forceinline__ float operator()(float x) const { return f_sqrt(x); } };
struct FInv { __device__ __forceinline__ float operator()(float x) const { return op_inv(x); } };
struct FTan { __device__ __forceinline__ float operator()(float x) const { return f_tan(x); } };
struct FAsin { __device__ __forceinline__ float operator()(float x) const { return f_asin(x); } };
struct FAcos { __device__ __forceinline__ float operator()(float x) const { return f_acos(x); } };
struct FAtan { __device__ __forceinline__ float operator()(float x) const { return f_atan(x); } };
struct FTanh { __device__ __forceinline__ float operator()(float x) const { return f_tanh(x); } };

template <typename F>
__device__ __forceinline__ V8 map8_unrolled(V8 v, F f) {
  float t[8] = {v.a.x, v.a.y, v.a.z, v.a.w, v.b.x, v.b.y, v.b.z, v.b.w};
#pragma unroll MATH_UNROLL
  for (int i = 0; i < 8; ++i) t[i] = f(t[i]);
  return V8{make_float4(t[0], t[1], t[2], t[3]), make_float4(t[4], t[5], t[6], t[7])};
}
__device__ __noinline__ V8 sin8(V8 v) { return map8_unrolled(v, FSin()); }
__device__ __noinline__ V8 cos8(V8 v) { return map8_unrolled(v, FCos()); }
__device__ __noinline__ V8 exp8(V8 v) { return map8_unrolled(v, FExp()); }
__device__ __noinline__ V8 log8(V8 v) { return map8_unrolled(v, FLog()); }
__device__ __noinline__ V8 sqrt8(V8 v) { return map8_unrolled(v, FSqrt()); }
// The EXT instantiation of the interpreter (programs that use 1/x, tan, asin,
// acos, atan, tanh) runs twelve library routines: unrolled 8-wide they no
// longer fit the instruction cache (ncu: 26 cycles per issue stalled on
// instruction fetch, 23 % of issue slots used).  There the extended routines
// run four cases at a time and the base ones two.  On a Table 1 population
// (GPop/s, at 5 CTAs per SM): extended one at a time 1,600, two 1,708, four
// 1,756, eight 1,383; base four at a time with extended four 1,309: the
// instruction cache decides.  The base instantiation keeps its 8-wide copies
// (4-wide: 2,662 -> 1,930 on base populations).
template <typename F>
__device__ __forceinline__ V8 map8_small(V8 v, F f) {
  float t[8] = {v.a.x, v.a.y, v.a.z, v.a.w, v.b.x, v.b.y, v.b.z, v.b.w};
#pragma unroll 4
  for (int i = 0; i < 8; ++i) t[i] = f(t[i]);
  return V8{make_float4(t[0], t[1], t[2], t[3]), make_float4(t[4], t[5], t[6], t[7])};
}
template <typename F>
__device__ __forceinline__ V8 map8_base_small(V8 v, F f) {  // 2 in flight
  float t[8] = {v.a.x, v.a.y, v.a.z, v.a.w, v.b.x, v.b.y, v.b.z, v.b.w};
#pragma unroll 2
  for (int i = 0; i < 8; ++i) t[i] = f(t[i]);
  return V8{make_float4(t[0], t[1], t[2], t[3]), make_float4(t[4], t[5], t[6], t[7])};
}
__device__ __noinline__ V8 sin8s(V8 v) { return map8_base_small(v, FSin()); }
__device__ __noinline__ V8 cos8s(V8 v) { return map8_base_small(v, FCos()); }
__device__ __noinline__ V8 exp8s(V8 v) { return map8_base_small(v, FExp()); }
__device__ __noinline__ V8 log8s(V8 v) { return map8_base_small(v, FLog()); }
__device__ __noinline__ V8 sqrt8s(V8 v) { return map8_base_small(v, FSqrt()); }
__device__ __noinline__ V8 div8s(V8 a, V8 b) {
  float x[8] = {a.a.x, a.a.y, a.a.z, a.a.w, a.b.x, a.b.y, a.b.z, a.b.w};
  const float y[8] = {b.a.x, b.a.y, b.a.z, b.a.w, b.b.x, b.b.y, b.b.z, b.b.w};
#pragma unroll 2
  for (int i = 0; i < 8; ++i) x[i] = op_div(x[i], y[i]);
  return V8{make_float4(x[0], x[1], x[2], x[3]), make_float4(x[4], x[5], x[6], x[7])};
}
__device__ __noinline__ V8 ext8(uint32_t op, V8 v) {
  switch (op) {
    case OP_INV: return map8_small(v, FInv());
    case OP_TAN: return map8_small(v, FTan());
    case OP_ASIN: return map8_small(v, FAsin());
    case OP_ACOS: return map8_small(v, FAcos());
    case OP_ATAN: return map8_small(v, FAtan());
    default: return map8_small(v, FTanh());
  }
}
__device__ __noinline__ V8 div8(V8 a, V8 b) {
  float x[8] = {a.a.x, a.a.y, a.a.z, a.a.w, a.b.x, a.b.y, a.b.z, a.b.w};
  const float y[8] = {b.a.x, b.a.y, b.a.z, b.a.w, b.b.x, b.b.y, b.b.z, b.b.w};
#pragma unroll MATH_UNROLL
  for (int i = 0; i < 8; ++i) x[i] = op_div(x[i], y[i]);
  return V8{make_float4(x[0], x[1], x[2], x[3]), make_float4(x[4], x[5], x[6], x[7])};
}
#define SIN8(v) sin8(v)
#define COS8(v) cos8(v)
#define EXP8(v) exp8(v)
#define LOG8(v) log8(v)
#define SQRT8(v) sqrt8(v)
#define DIV8(p, q) div8(p, q)
#define EXT8(op, v) ext8(op, v)

// Runs the decoded program for this lane's 8 cases.  xa / xb point at the
// lane's first and second case group in row 0 of X; `stk` at this lane's
// entry of stack slot 0 in shared memory.
// EXT: the copy of the loop that also runs 1/x, tan, asin, acos, atan, tanh
template <bool EXT>
__device__ __forceinline__ V8 interpret(const uint2 *__restrict__ code, int n, char *stk,
                                        const float *__restrict__ xa, const float *__restrict__ xb) {
  V8 T = splat8(0.f);
  for (int ip = 0; ip < n; ++ip) {
    const uint2 w = code[ip];
    const uint32_t off = ins_off(w);
    switch (ins_op(w)) {
      case OP_LDV: T = ldX8(xa, xb, w.y); break;
      case OP_LDC: T = splat8(__uint_as_float(w.y)); break;
      case OP_PUSHV: st8(stk, off, T); T = ldX8(xa, xb, w.y); break;
      case OP_PUSHC: st8(stk, off, T); T = splat8(__uint_as_float(w.y)); break;
      case OP_ADD: { const V8 a = ld8(stk, off); T = ZIP8(f_add, a, T); } break;
      case OP_SUB: { const V8 a = ld8(stk, off); T = ZIP8(f_sub, a, T); } break;
      case OP_MUL: { const V8 a = ld8(stk, off); T = ZIP8(f_mul, a, T); } break;
      case OP_DIV: { const V8 a = ld8(stk, off); T = EXT ? div8s(a, T) : DIV8(a, T); } break;
      case OP_RSUB: { const V8 b = ld8(stk, off); T = ZIP8(f_sub, T, b); } break;
      case OP_RDIV: { const V8 b = ld8(stk, off); T = EXT ? div8s(T, b) : DIV8(T, b); } break;
      case OP_SIN: T = EXT ? sin8s(T) : SIN8(T); break;
      case OP_COS: T = EXT ? cos8s(T) : COS8(T); break;
      case OP_EXP: T = EXT ? exp8s(T) : EXP8(T); break;
      case OP_LOG: T = EXT ? log8s(T) : LOG8(T); break;
      case OP_SQRT: T = EXT ? sqrt8s(T) : SQRT8(T); break;
      case OP_SQ: T = MAP8(f_sq, T); break;
      case OP_INV:
      case OP_TAN:
      case OP_ASIN:
      case OP_ACOS:
      case OP_ATAN:
      case OP_TANH:
        if (EXT) T = EXT8(ins_op(w), T);
        break;
      case OP_VADD: { const V8 v = ldX8(xa, xb, w.y); T = ZIP8(f_add, T, v); } break;
      case OP_VSUB: { const V8 v = ldX8(xa, xb, w.y); T = ZIP8(f_sub, T, v); } break;
      case OP_VMUL: { const V8 v = ldX8(xa, xb, w.y); T = ZIP8(f_mul, T, v); } break;
      case OP_VDIV: { const V8 v = ldX8(xa, xb, w.y); T = EXT ? div8s(T, v) : DIV8(T, v); } break;
      case OP_VRSUB: { const V8 v = ldX8(xa, xb, w.y); T = ZIP8(f_sub, v, T); } break;
      case OP_VRDIV: { const V8 v = ldX8(xa, xb, w.y); T = EXT ? div8s(v, T) : DIV8(v, T); } break;
      case OP_CADD: { const V8 v = splat8(__uint_as_float(w.y)); T = ZIP8(f_add, T, v); } break;
      case OP_CSUB: { const V8 v = splat8(__uint_as_float(w.y)); T = ZIP8(f_sub, T, v); } break;
      case OP_CMUL: { const V8 v = splat8(__uint_as_float(w.y)); T = ZIP8(f_mul, T, v); } break;
      case OP_CDIV: { const V8 v = splat8(__uint_as_float(w.y)); T = EXT ? div8s(T, v) : DIV8(T, v); } break;
      case OP_CRSUB: { const V8 v = splat8(__uint_as_float(w.y)); T = ZIP8(f_sub, v, T); } break;
      case OP_CRDIV: { const V8 v = splat8(__uint_as_float(w.y)); T = EXT ? div8s(v, T) : DIV8(v, T); } break;
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

// Eq. 3 on one case, FP32, every operation rounded on its own (no
// contraction), the result rounded half to even.
__device__ __forceinline__ int p2p_case(float yh, float y, int M, float Mf, float pen) {
  const bool vh = isfinite(yh), vy = isfinite(y);
  if (!(vh && vy)) return (vh || vy) ? -M : M;
  const float a = fabsf(yh), b = fabsf(y);
  const float mx = fmaxf(a, b), mn = fminf(a, b);
  if (mx == 0.0f) return M;
  float v = __fmul_rn(Mf, __fdiv_rn(mn, mx));
  if ((yh < 0.0f && y > 0.0f) || (yh > 0.0f && y < 0.0f)) v = __fsub_rn(v, pen);
  return (int)rintf(v);
}

// Eq. 2 sums over one lane's 8 cases (nvalid of them inside the chunk):
// pairs with both values finite give the moments of the shifted output d
// and the centred target e; one invalid value counts in n1, both in n2.
// Out of line: the copy inside the interpreter loop measured 1.7 % slower.
struct R4Part { float s1, s2, s3, s4, s5; int n1, n2; };
__device__ __noinline__ R4Part r4_part(V8 T, float4 ya, float4 yb, int nvalid, float shift) {
  const float tv[CPL] = {T.a.x, T.a.y, T.a.z, T.a.w, T.b.x, T.b.y, T.b.z, T.b.w};
  const float yv[CPL] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
  float d[CPL], e[CPL];
  int c1 = 0, c2 = 0;
#pragma unroll
  for (int i = 0; i < CPL; ++i) {
    const bool ok = i < nvalid;
    const bool vh = isfinite(tv[i]), vy = isfinite(yv[i]);
    const bool pair = ok && vh && vy;
    c1 += (ok && vh != vy) ? 1 : 0;
    c2 += (ok && !vh && !vy) ? 1 : 0;
    d[i] = pair ? tv[i] - shift : 0.0f;
    e[i] = pair ? yv[i] : 0.0f;
  }
  R4Part r;
  r.s1 = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7]));
  r.s2 = ((d[0] * d[0] + d[1] * d[1]) + (d[2] * d[2] + d[3] * d[3])) +
         ((d[4] * d[4] + d[5] * d[5]) + (d[6] * d[6] + d[7] * d[7]));
  r.s3 = ((d[0] * e[0] + d[1] * e[1]) + (d[2] * e[2] + d[3] * e[3])) +
         ((d[4] * e[4] + d[5] * e[5]) + (d[6] * e[6] + d[7] * e[7]));
  r.s4 = ((e[0] + e[1]) + (e[2] + e[3])) + ((e[4] + e[5]) + (e[6] + e[7]));
  r.s5 = ((e[0] * e[0] + e[1] * e[1]) + (e[2] * e[2] + e[3] * e[3])) +
         ((e[4] * e[4] + e[5] * e[5]) + (e[6] * e[6] + e[7] * e[7]));
  r.n1 = c1;
  r.n2 = c2;
  return r;
}

// ---------------------------------------------------------------- one work item
struct WarpSmem {
  char *stk;        // shared stack slots of this warp, [DSM][2][32] float4
  uint2 *code;      // this warp's copy of the program's code
};

__device__ __forceinline__ WarpSmem warp_smem(unsigned char *smem, int warp, int warp_bytes, int slots) {
  unsigned char *wbase = smem + (size_t)warp * warp_bytes;
  WarpSmem w;
  w.stk = reinterpret_cast<char *>(wbase);
  w.code = reinterpret_cast<uint2 *>(wbase + slots * SLOT_BYTES);
  return w;
}

// Evaluates program `prog` of problem p on case chunk `c` with the calling
// warp.  MODE_BOTH accumulates the sums selected by `want` (bit 0: squared
// error, bit 1: correlation moments); the other modes ignore `want`.
template <int MODE, bool EXT>
__device__ __forceinline__ void eval_item(const EvalParams &p, int c, int prog, const WarpSmem &w,
                                          int lane, int want) {
  const bool do_mse = MODE == MODE_MSE || (MODE == MODE_BOTH && (want & 1));
  const bool do_corr = MODE == MODE_CORR || (MODE == MODE_BOTH && (want & 2));
  const int cbeg = c * p.chunk;
  const int cend = min(p.N, cbeg + p.chunk);
  if (p.flags[prog]) {
    if (MODE == MODE_PREDICT) {
      float *row = p.yhat + (size_t)prog * p.ldy;
      for (int i = cbeg + lane; i < cend; i += 32) row[i] = __int_as_float(0x7fc00000);
    }
    return;
  }
  const int n = ncode_count(p.ncode[prog]);
  __syncwarp();  // the previous item is done reading the code
  const uint2 *src = p.code + (size_t)prog * p.Lmax;
  for (int i = lane; i < n; i += 32) w.code[i] = src[i];
  __syncwarp();

  char *stk = w.stk + lane * 16;
  const int last_group = (cend - 1) & ~(CPL - 1);

  Kahan se, s1, s2, s3, s4, s5;
  float shift = 0.f;
  long long score = 0;
  int c1 = 0, c2 = 0;
  const float Mf = (float)p.score_M, pen = __fdiv_rn(Mf, 11.0f);
  for (int base = cbeg; base < cend; base += STEP) {
    const int c0 = base + CPL * lane;
    const int cl = c0 < cend ? c0 : last_group;           // first 4 cases, always readable
    const int cl4 = cl + 4 < cend ? cl + 4 : cl;          // second 4, or a re-read when none valid
    const V8 T = interpret<EXT>(w.code, n, stk, p.X + cl, p.X + cl4);
    const float tv[CPL] = {T.a.x, T.a.y, T.a.z, T.a.w, T.b.x, T.b.y, T.b.z, T.b.w};
    bool ok[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ok[i] = c0 + i < cend;
    if (MODE == MODE_PREDICT) {
      float *row = p.yhat + (size_t)prog * p.ldy;
#pragma unroll
      for (int i = 0; i < CPL; ++i)
        if (ok[i]) row[c0 + i] = tv[i];
    }
    if (do_mse) {
      const float4 ya = load_y4(p.y, cl, p.N), yb = load_y4(p.y, cl4, p.N);
      const float yv[CPL] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
      float e[CPL];
#pragma unroll
      for (int i = 0; i < CPL; ++i) e[i] = sel(ok[i], tv[i] - yv[i]);
      se.add(((e[0] * e[0] + e[1] * e[1]) + (e[2] * e[2] + e[3] * e[3])) +
             ((e[4] * e[4] + e[5] * e[5]) + (e[6] * e[6] + e[7] * e[7])));
    }
    if (do_corr) {
      if (base == cbeg) shift = __shfl_sync(FULL, T.a.x, 0);
      const float4 ya = ldx4(p.yc + cl), yb = ldx4(p.yc + cl4);
      const float yv[CPL] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
      float d[CPL];
#pragma unroll
      for (int i = 0; i < CPL; ++i) d[i] = sel(ok[i], tv[i] - shift);
      s1.add(((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])));
      s2.add(((d[0] * d[0] + d[1] * d[1]) + (d[2] * d[2] + d[3] * d[3])) +
             ((d[4] * d[4] + d[5] * d[5]) + (d[6] * d[6] + d[7] * d[7])));
      s3.add(((d[0] * yv[0] + d[1] * yv[1]) + (d[2] * yv[2] + d[3] * yv[3])) +
             ((d[4] * yv[4] + d[5] * yv[5]) + (d[6] * yv[6] + d[7] * yv[7])));
    }
    if (MODE == MODE_R4) {
      // pairs: both finite -> moments; one invalid -> c1; both -> c2.  yc
      // holds y - ybar for finite y and NaN for invalid targets.
      if (base == cbeg) {
        const unsigned fin = __ballot_sync(FULL, isfinite(T.a.x));
        shift = fin ? __shfl_sync(FULL, T.a.x, __ffs(fin) - 1) : 0.0f;
      }
      const float4 ya = ldx4(p.yc + cl), yb = ldx4(p.yc + cl4);
      const R4Part q = r4_part(T, ya, yb, cend - c0, shift);
      s1.add(q.s1);
      s2.add(q.s2);
      s3.add(q.s3);
      s4.add(q.s4);
      s5.add(q.s5);
      c1 += q.n1;
      c2 += q.n2;
    }
    if (MODE == MODE_P2P) {
      const float4 ya = load_y4(p.y, cl, p.N), yb = load_y4(p.y, cl4, p.N);
      // one copy of the per-case body: the values rotate through it
      float t0 = T.a.x, t1 = T.a.y, t2 = T.a.z, t3 = T.a.w, t4 = T.b.x, t5 = T.b.y, t6 = T.b.z, t7 = T.b.w;
      float y0 = ya.x, y1 = ya.y, y2 = ya.z, y3 = ya.w, y4 = yb.x, y5 = yb.y, y6 = yb.z, y7 = yb.w;
#pragma unroll 1
      for (int i = 0; i < CPL; ++i) {
        if (c0 + i < cend) {
          const bool vh = isfinite(t0), vy = isfinite(y0);
          c1 += vh != vy ? 1 : 0;
          c2 += (!vh && !vy) ? 1 : 0;
          score += p2p_case(t0, y0, p.score_M, Mf, pen);
        }
        t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = t7;
        y0 = y1; y1 = y2; y2 = y3; y3 = y4; y4 = y5; y5 = y6; y6 = y7;
      }
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
    if (MODE == MODE_R4) {
      // [shift, sum d, sum d^2, sum d e, sum e, sum e^2, c1, c2]
      const double v1 = warp_sum(s1.value()), v2 = warp_sum(s2.value()), v3 = warp_sum(s3.value());
      const double v4 = warp_sum(s4.value()), v5 = warp_sum(s5.value());
      const double n1 = warp_sum((double)c1), n2 = warp_sum((double)c2);
      if (lane == 0) {
        rec[0] = (double)shift;
        rec[1] = v1;
        rec[2] = v2;
        rec[3] = v3;
        rec[4] = v4;
        rec[5] = v5;
        rec[6] = n1;
        rec[7] = n2;
      }
    }
    if (MODE == MODE_P2P) {
      // [sum of the integer scores (exact), c1, c2]
      const double v = warp_sum((double)score);
      const double n1 = warp_sum((double)c1), n2 = warp_sum((double)c2);
      if (lane == 0) {
        rec[0] = v;
        rec[6] = n1;
        rec[7] = n2;
      }
    }
  }
}

// ---------------------------------------------------------------- single problem
// Up to three passes over the work items: EXT = false takes the programs of
// the base operators (and the invalid ones), EXT = true those that use 1/x,
// tan, asin, acos, atan or tanh; it returns at once when the decoder counted
// none.  Keeping the extended operators out of the first kernel keeps its
// loop (and its speed) what it is for the base operators.  Both give each
// warp shallow_slots(Lmax, MINB) stack slots; the programs that need more
// (NCODE_DEEP) run in a third launch of the EXT kernel with deep = 1 and
// slots_for(Lmax) slots, made only when the two differ.
template <int MODE, bool EXT, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) eval_kernel(EvalParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const bool deep = EXT && p.deep;  // the deep pass runs the EXT copy of the loop
  if (deep ? p.queue[4] == 0 : (EXT && p.queue[2] == 0)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpSmem w = warp_smem(smem, warp, p.warp_bytes, p.slots);
  unsigned long long *q = p.queue + (deep ? 3 : (EXT ? 1 : 0));
  for (;;) {
    const long long item = next_item(q, p.total_items, p.abort, p.err, lane);
    if (item >= p.total_items) break;
    const int c = (int)(item / (unsigned long long)p.P);
    const int prog = (int)(item % (unsigned long long)p.P);
    const int nc = p.ncode[prog];
    if (deep ? !ncode_deep(nc) : (nc & (NCODE_EXT | NCODE_DEEP)) != (EXT ? NCODE_EXT : 0)) continue;
    eval_item<MODE, EXT>(p, c, prog, w, lane, 3);
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
  uint2 *code;         // [P][Lmax]
  int32_t *ncode;      // [P]
  double *fitness;     // [P] or [2][P]
  double *ychunk;      // [nchunks][2]
  double *ysum;        // [nchunks][2]: FP64 sum and count of y per chunk
  long long ldx;
  long long item_begin;  // first work item of this problem in the launch
  int prog_begin;        // first program of this problem in the decode launch
  int P, Lmax, K, nvars, N, chunk, nchunks;
  int mode;              // MODE_MSE, MODE_CORR or MODE_BOTH
  int corr_chunk_begin;  // first block of this problem in the batched centring launch (-1: none)
  int xform;             // >= 1: X / ldx are the problem's variable table of this depth (EvalParams::xform)
  uint8_t *xneed;
};

struct BatchParams {
  BatchProblem prob[MAX_BATCH];
  int nprob;
  int corr_list[MAX_BATCH];  // problems that need the centred target, in order
  int ncorr;
  int total_progs;
  long long total_items;
  unsigned long long *queue;  // as EvalParams::queue
  int warp_bytes;
  int slots;
  int maxL;                   // the largest Lmax of the batch
  int deep;                   // as EvalParams::deep
  const int32_t *abort;       // as EvalParams::abort
  unsigned *err;
};

static_assert(sizeof(BatchParams) <= 32764, "the problem table must fit the kernel parameters");

__device__ __forceinline__ EvalParams view(const BatchProblem &q) {
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
  p.code = q.code;
  p.ncode = q.ncode;
  p.xform = q.xform;
  p.xneed = q.xneed;
  return p;
}

// a warp per program of every problem in the batch (shared regions sized
// for the batch's largest Lmax, b.maxL)
__global__ void decode_batched_kernel(const __grid_constant__ BatchParams b) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int warp = threadIdx.x >> 5;
  const int g = blockIdx.x * (blockDim.x >> 5) + warp;
  if (g >= b.total_progs) return;
  int lo = 0, hi = b.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.prob[mid].prog_begin <= g) lo = mid;
    else hi = mid - 1;
  }
  EvalParams p = view(b.prob[lo]);
  p.queue = b.queue;
  decode_warp_one(decode_args(p, b.slots, b.queue + 4), g - b.prob[lo].prog_begin,
                  dsm + (size_t)warp * decode_warp_bytes(b.maxL));
}

// Work items of every problem come from one atomic counter: problem q owns
// items [item_begin_q, item_begin_q + P_q * nchunks_q), chunk-major inside.
// EXT and deep as for eval_kernel (the extended programs of every problem
// in a second launch, the deep ones in a third).
// At most 64 registers, so that 4 CTAs fit an SM (75 unbounded, 3 CTAs):
// 2,608 -> 2,949 GPop/s on the 64-problem batch despite a few spilled values.
template <bool EXT, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) eval_batched_kernel(const __grid_constant__ BatchParams b) {
  extern __shared__ __align__(16) unsigned char smem[];
  const bool deep = EXT && b.deep;
  if (deep ? b.queue[4] == 0 : (EXT && b.queue[2] == 0)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpSmem w = warp_smem(smem, warp, b.warp_bytes, b.slots);
  unsigned long long *qc = b.queue + (deep ? 3 : (EXT ? 1 : 0));
  for (;;) {
    const long long item = next_item(qc, b.total_items, b.abort, b.err, lane);
    if (item >= b.total_items) break;
    int lo = 0, hi = b.nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.prob[mid].item_begin <= (long long)item) lo = mid;
      else hi = mid - 1;
    }
    const BatchProblem &q = b.prob[lo];
    const EvalParams p = view(q);
    const long long local = (long long)item - q.item_begin;
    const int c = (int)(local / q.P);
    const int prog = (int)(local % q.P);
    const int nc = q.ncode[prog];
    if (deep ? !ncode_deep(nc) : (nc & (NCODE_EXT | NCODE_DEEP)) != (EXT ? NCODE_EXT : 0)) continue;
    const int want = q.mode == MODE_MSE ? 1 : (q.mode == MODE_CORR ? 2 : 3);
    eval_item<MODE_BOTH, EXT>(p, c, prog, w, lane, want);
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

// FP64 sum and count of one chunk of y: every value, or (finite_only) the
// finite ones.  ysum [nchunks][2].
__device__ void ysum_chunk(const float *__restrict__ y, int N, int chunk, int c, bool finite_only,
                           double *ysum, double *red) {
  const int beg = c * chunk, end = min(N, beg + chunk);
  double a = 0.0, n = 0.0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const float v = y[i];
    if (!finite_only || isfinite(v)) {
      a += (double)v;
      n += 1.0;
    }
  }
  a = block_sum(a, red);
  n = block_sum(n, red);
  if (threadIdx.x == 0) {
    ysum[2 * c] = a;
    ysum[2 * c + 1] = n;
  }
}

__global__ void __launch_bounds__(PREP_THREADS) ysum_kernel(const float *__restrict__ y, int N, int chunk,
                                                            int finite_only, double *ysum) {
  __shared__ double red[PREP_THREADS / 32];
  ysum_chunk(y, N, chunk, blockIdx.x, finite_only != 0, ysum, red);
}

// ybar = (sum of the chunk sums) / (their count), chunks in order; then
// yc = fl32(y - ybar) on one chunk (NaN at invalid targets when
// nan_invalid) with the chunk's FP64 sum and sum of squares of yc
__device__ void ycenter_chunk(const float *__restrict__ y, int N, int chunk, int nchunks, int c,
                              const double *ysum, bool nan_invalid, float *yc, double *ychunk,
                              double *red) {
  __shared__ double ybar_s;
  if (threadIdx.x == 0) {
    double t = 0.0, n = 0.0;
    for (int k = 0; k < nchunks; ++k) {
      t += ysum[2 * k];
      n += ysum[2 * k + 1];
    }
    ybar_s = n > 0.0 ? t / n : 0.0;
  }
  __syncthreads();
  const double ybar = ybar_s;
  const int beg = c * chunk, end = min(N, beg + chunk);
  double a = 0.0, b = 0.0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const float yi = y[i];
    if (nan_invalid && !isfinite(yi)) {
      yc[i] = __int_as_float(0x7fc00000);
      continue;
    }
    const float v = (float)((double)yi - ybar);
    yc[i] = v;
    a += (double)v;
    b += (double)v * (double)v;
  }
  if (c == nchunks - 1) {
    const int padded = (N + STEP - 1) / STEP * STEP;
    for (int i = N + threadIdx.x; i < padded; i += blockDim.x) yc[i] = 0.0f;
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    ychunk[2 * c] = a;
    ychunk[2 * c + 1] = b;
  }
}

__global__ void __launch_bounds__(PREP_THREADS) ycenter_kernel(const float *__restrict__ y, int N,
                                                               int chunk, int nchunks,
                                                               const double *ysum, int nan_invalid,
                                                               float *yc, double *ychunk) {
  __shared__ double red[PREP_THREADS / 32];
  ycenter_chunk(y, N, chunk, nchunks, blockIdx.x, ysum, nan_invalid != 0, yc, ychunk, red);
}

// ---------------------------------------------------------------- finalize
// The merges below run with a warp per program: lane l takes chunks l,
// l + 32, ...; every sum over chunks is a per-lane sum followed by a fixed
// xor-butterfly reduction (warp_sum), so the result is deterministic and
// the same on every lane.  (A thread per program ran the FP64 chain of all
// chunks serially: 0.7 % of a 4,096 x 100,000 generation.)

// 1 - r^2 of one program from its chunk records.
// chunk c: n_c cases, shift s_c, S1 = sum d, S2 = sum d^2, S3 = sum d yc with
// d = yhat - s_c.  Chunk mean m_c = s_c + S1/n_c, chunk M2 = S2 - S1^2/n_c;
// merged (Chan et al.): Shh = sum M2_c + n_c (m_c - m)^2.
// sum yhat*yc = sum (S3_c + s_c Yc_c); Shy = that - m * Y1; Syy = Y2 - Y1^2/N.
__device__ double corr_fitness(const double *rec, const double *ychunk, int Nc, int chunk,
                               int nchunks, int lane) {
  const double N = (double)Nc;
  double y1 = 0.0, y2 = 0.0, tot = 0.0;
  for (int c = lane; c < nchunks; c += 32) {
    y1 += ychunk[2 * c];
    y2 += ychunk[2 * c + 1];
    const double nc = (double)min(chunk, Nc - c * chunk);
    tot += nc * rec[c * PSTRIDE + 1] + rec[c * PSTRIDE + 2];
  }
  y1 = warp_sum(y1);
  y2 = warp_sum(y2);
  const double m = warp_sum(tot) / N;
  double shh = 0.0, g = 0.0;
  for (int c = lane; c < nchunks; c += 32) {
    const double nc = (double)min(chunk, Nc - c * chunk);
    const double s = rec[c * PSTRIDE + 1], a = rec[c * PSTRIDE + 2];
    const double b = rec[c * PSTRIDE + 3], d = rec[c * PSTRIDE + 4];
    const double mc = s + a / nc;
    shh += (b - a * a / nc) + nc * (mc - m) * (mc - m);
    g += d + s * ychunk[2 * c];
  }
  shh = warp_sum(shh);
  const double shy = warp_sum(g) - m * y1;
  const double syy = y2 - y1 * y1 / N;
  double fit = 1.0;
  if (isfinite(shh) && isfinite(shy) && isfinite(syy) && shh > 0.0 && syy > 0.0 && Nc >= 2) {
    const double r2 = (shy * shy) / (syy * shh);
    fit = 1.0 - r2;
    fit = fit < 0.0 ? 0.0 : (fit > 1.0 ? 1.0 : fit);
  }
  return fit;
}

// Eq. 2 of one program from its chunk records [shift s, S1 = sum d,
// S2 = sum d^2, X = sum d e, E1 = sum e, E2 = sum e^2, c1, c2] over the
// valid pairs (d = yhat - s, e = y - ybar).  Valid pairs of chunk c:
// n_c = cases - c1 - c2.  Shh merges the chunks by Chan et al.; e shares one
// centre, so See = E2 - E1^2 / n; Seh = sum (X_c + s_c E1_c) - m E1.
__device__ double r4_score(const double *rec, int Nc, int chunk, int nchunks, double M, double *c1o,
                           double *c2o, int lane) {
  double c1 = 0.0, c2 = 0.0, n = 0.0, tot = 0.0, e1 = 0.0, e2 = 0.0;
  for (int c = lane; c < nchunks; c += 32) {
    const double *r = rec + c * PSTRIDE;
    const double nv = (double)min(chunk, Nc - c * chunk) - r[6] - r[7];
    c1 += r[6];
    c2 += r[7];
    n += nv;
    tot += r[1] + nv * r[0];
    e1 += r[4];
    e2 += r[5];
  }
  c1 = warp_sum(c1);
  c2 = warp_sum(c2);
  n = warp_sum(n);
  tot = warp_sum(tot);
  e1 = warp_sum(e1);
  e2 = warp_sum(e2);
  double r2 = 0.0;
  if (n >= 2.0) {
    const double m = tot / n;
    double shh = 0.0, seh = 0.0;
    for (int c = lane; c < nchunks; c += 32) {
      const double *r = rec + c * PSTRIDE;
      const double nv = (double)min(chunk, Nc - c * chunk) - r[6] - r[7];
      if (nv <= 0.0) continue;
      const double mc = r[0] + r[1] / nv;
      shh += (r[2] - r[1] * r[1] / nv) + nv * (mc - m) * (mc - m);
      seh += r[3] + r[0] * r[4];
    }
    shh = warp_sum(shh);
    seh = warp_sum(seh) - m * e1;
    const double see = e2 - e1 * e1 / n;
    if (isfinite(shh) && isfinite(seh) && isfinite(see) && shh > 0.0 && see > 0.0) {
      r2 = (seh * seh) / (shh * see);
      r2 = r2 < 0.0 ? 0.0 : (r2 > 1.0 ? 1.0 : r2);
    }
  }
  *c1o = c1;
  *c2o = c2;
  return M * (r2 * r2) * n - M * (c1 - c2);
}

// fitness of program p from its partial records (mode picks the outputs);
// called by all 32 lanes of a warp, lane 0 writes
__device__ void finalize_one(int mode, const double *partials, const int32_t *flags,
                             const double *ychunk, int P, int N, int chunk, int nchunks,
                             double *fitness, int p, int lane, int M = 0, int32_t *counts = nullptr) {
  const double INF = __longlong_as_double(0x7ff0000000000000ll);
  if (mode == MODE_R4 || mode == MODE_P2P) {
    double c1 = 0.0, c2 = 0.0, sc = -INF;
    if (!flags[p]) {
      const double *rec = partials + (size_t)p * nchunks * PSTRIDE;
      if (mode == MODE_R4) {
        sc = r4_score(rec, N, chunk, nchunks, (double)M, &c1, &c2, lane);
      } else {
        sc = 0.0;
        for (int c = lane; c < nchunks; c += 32) {
          sc += rec[c * PSTRIDE];
          c1 += rec[c * PSTRIDE + 6];
          c2 += rec[c * PSTRIDE + 7];
        }
        sc = warp_sum(sc);  // integers below 2^53: exact in any order
        c1 = warp_sum(c1);
        c2 = warp_sum(c2);
      }
    }
    if (lane == 0) {
      fitness[p] = sc;
      if (counts) {
        counts[2 * p] = (int32_t)c1;
        counts[2 * p + 1] = (int32_t)c2;
      }
    }
    return;
  }
  double *mse_out = fitness;
  double *corr_out = mode == MODE_BOTH ? fitness + P : fitness;
  if (flags[p]) {
    if (lane == 0 && mode != MODE_CORR) mse_out[p] = INF;
    if (lane == 0 && mode != MODE_MSE) corr_out[p] = INF;
    return;
  }
  const double *rec = partials + (size_t)p * nchunks * PSTRIDE;
  if (mode != MODE_CORR) {
    double se = 0.0;
    for (int c = lane; c < nchunks; c += 32) se += rec[c * PSTRIDE];
    se = warp_sum(se);
    if (lane == 0) mse_out[p] = isfinite(se) ? se / (double)N : INF;
  }
  if (mode != MODE_MSE) {
    const double f = corr_fitness(rec, ychunk, N, chunk, nchunks, lane);
    if (lane == 0) corr_out[p] = f;
  }
}

struct FinalParams {
  const double *partials;
  const int32_t *flags;
  const double *ychunk;
  int P, N, chunk, nchunks, mode;
  double *fitness;  // [P] or [2][P]
  int M;            // Beagle scores
  int32_t *counts;  // Beagle scores: [P][2] (c1, c2) or NULL
};

// a warp per program, FINAL_WARPS programs per block
constexpr int FINAL_WARPS = 4;

__global__ void finalize_kernel(FinalParams f) {
  const int p = blockIdx.x * FINAL_WARPS + (threadIdx.x >> 5);
  if (p >= f.P) return;
  finalize_one(f.mode, f.partials, f.flags, f.ychunk, f.P, f.N, f.chunk, f.nchunks, f.fitness, p,
               threadIdx.x & 31, f.M, f.counts);
}

// ---------------------------------------------------------------- batched prep / finalize
// one block per (problem, chunk) of the problems that need the centred
// target: the chunk sums of y, then (next launch) the centred target
__device__ __forceinline__ int corr_problem_of_block(const BatchParams &b) {
  int r = 0;
  while (r + 1 < b.ncorr && b.prob[b.corr_list[r + 1]].corr_chunk_begin <= (int)blockIdx.x) ++r;
  return b.corr_list[r];
}

__global__ void __launch_bounds__(PREP_THREADS) ysum_batched_kernel(const __grid_constant__ BatchParams b) {
  __shared__ double red[PREP_THREADS / 32];
  const BatchProblem &q = b.prob[corr_problem_of_block(b)];
  ysum_chunk(q.y, q.N, q.chunk, (int)blockIdx.x - q.corr_chunk_begin, false, q.ysum, red);
}

__global__ void __launch_bounds__(PREP_THREADS) ycenter_batched_kernel(const __grid_constant__ BatchParams b) {
  __shared__ double red[PREP_THREADS / 32];
  const BatchProblem &q = b.prob[corr_problem_of_block(b)];
  ycenter_chunk(q.y, q.N, q.chunk, q.nchunks, (int)blockIdx.x - q.corr_chunk_begin, q.ysum, false, q.yc,
                q.ychunk, red);
}

// blocks (problem, FINAL_WARPS programs of it), a warp per program
__global__ void finalize_batched_kernel(const __grid_constant__ BatchParams b) {
  const BatchProblem &q = b.prob[blockIdx.x];
  for (int p = blockIdx.y * FINAL_WARPS + (threadIdx.x >> 5); p < q.P; p += gridDim.y * FINAL_WARPS)
    finalize_one(q.mode, q.partials, q.flags, q.ychunk, q.P, q.N, q.chunk, q.nchunks, q.fitness, p,
                 threadIdx.x & 31);
}

// ---------------------------------------------------------------- host side
template <int MODE, bool EXT, int MINB>
sr_status occupancy_grid(sr_ctx *ctx, int smem, int *grid) {
  sr_status st = allow_dynamic_smem(ctx, reinterpret_cast<const void *>(eval_kernel<MODE, EXT, MINB>));
  if (st != SR_OK) return st;
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_kernel<MODE, EXT, MINB>, WARPS * 32, smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (nb < 1) return fail(ctx, SR_EINVAL, "Lmax too large for shared memory");
  *grid = nb * ctx->num_sms;
  return SR_OK;
}

template <bool EXT, int MINB>
sr_status grid_for_m(sr_ctx *ctx, int mode, int smem, int *grid) {
  switch (mode) {
    case MODE_PREDICT: return occupancy_grid<MODE_PREDICT, EXT, MINB>(ctx, smem, grid);
    case MODE_MSE: return occupancy_grid<MODE_MSE, EXT, MINB>(ctx, smem, grid);
    case MODE_CORR: return occupancy_grid<MODE_CORR, EXT, MINB>(ctx, smem, grid);
    case MODE_R4: return occupancy_grid<MODE_R4, EXT, MINB>(ctx, smem, grid);
    case MODE_P2P: return occupancy_grid<MODE_P2P, EXT, MINB>(ctx, smem, grid);
    default: return occupancy_grid<MODE_BOTH, EXT, MINB>(ctx, smem, grid);
  }
}

template <bool EXT>
sr_status grid_for_t(sr_ctx *ctx, int mode, int minb, int smem, int *grid) {
  return minb == 5 ? grid_for_m<EXT, 5>(ctx, mode, smem, grid) : grid_for_m<EXT, 4>(ctx, mode, smem, grid);
}

template <bool EXT, int MINB>
void launch_mode_m(int mode, int grid, int smem, cudaStream_t s, const EvalParams &ep) {
  switch (mode) {
    case MODE_PREDICT: eval_kernel<MODE_PREDICT, EXT, MINB><<<grid, WARPS * 32, smem, s>>>(ep); break;
    case MODE_MSE: eval_kernel<MODE_MSE, EXT, MINB><<<grid, WARPS * 32, smem, s>>>(ep); break;
    case MODE_CORR: eval_kernel<MODE_CORR, EXT, MINB><<<grid, WARPS * 32, smem, s>>>(ep); break;
    case MODE_R4: eval_kernel<MODE_R4, EXT, MINB><<<grid, WARPS * 32, smem, s>>>(ep); break;
    case MODE_P2P: eval_kernel<MODE_P2P, EXT, MINB><<<grid, WARPS * 32, smem, s>>>(ep); break;
    default: eval_kernel<MODE_BOTH, EXT, MINB><<<grid, WARPS * 32, smem, s>>>(ep); break;
  }
}

template <bool EXT>
void launch_mode(int mode, int minb, int grid, int smem, cudaStream_t s, const EvalParams &ep) {
  if (minb == 5) launch_mode_m<EXT, 5>(mode, grid, smem, s, ep);
  else launch_mode_m<EXT, 4>(mode, grid, smem, s, ep);
}

struct Plan {
  int minb;       // CTAs per SM of the main passes (eval_kernel's MINB)
  int slots;      // stack slots per warp of the main passes
  int grid, smem, chunk, nchunks;
  int smem_deep;  // shared memory of the deep pass (0: none)
  long long items;
  int xform;      // the variable table's depth (0: none; rows of ldxt floats)
  int ldxt;
  size_t off_queue, off_flags, off_ncode, off_code, off_part, off_yc,
      off_ych, off_ysum, off_xt, off_xneed, bytes;
};

// Whether a call (or a batch's problem) of P programs and N cases over nvars variables reads
// the variable table, and that table's row stride.
// (0: no; 1: u(x_j); 2: also the compositions, where the table stays
// within XFORM2_MAX_BYTES), and that table's row stride.
inline int use_xform(const sr_ctx *ctx, int P, int nvars, int N, int *ldxt) {
  *ldxt = (N + 3) / 4 * 4;
  const bool automatic = ctx->xform == 1 && N >= XFORM_MIN_N && P >= XFORM_MIN_P;
  if (!(ctx->xform == 2 || automatic)) return 0;
  const long long cells2 = (long long)xform_rows(nvars, 2) * *ldxt;
  if (cells2 < 0xFFFFFFFFll && cells2 * 4 <= XFORM2_MAX_BYTES) return 2;
  return (long long)xform_rows(nvars, 1) * *ldxt < 0xFFFFFFFFll ? 1 : 0;
}

sr_status make_plan(sr_ctx *ctx, int mode, int P, int Lmax, int N, Plan *pl, int nvars = 1) {
  pl->minb = eval_minb(Lmax, ctx->eval_ctas);
  pl->slots = shallow_slots(Lmax, pl->minb);
  pl->smem = WARPS * warp_smem_bytes(pl->slots, Lmax);
  pl->smem_deep = slots_for(Lmax) > pl->slots ? WARPS * warp_smem_bytes(slots_for(Lmax), Lmax) : 0;
  sr_status st = grid_for_t<false>(ctx, mode, pl->minb, pl->smem, &pl->grid);
  if (st != SR_OK) return st;
  const long long warps = (long long)pl->grid * WARPS;
  const long long want = warps * TARGET_ITEMS_PER_WARP;
  int nch = (int)((want + P - 1) / (P > 0 ? P : 1));
  // chunks of at least one warp step: a small problem (few programs, few
  // cases) then still spreads over many warps, its items one step each
  const int max_chunks = (N + STEP - 1) / STEP;
  nch = nch < 1 ? 1 : (nch > max_chunks ? max_chunks : nch);
  int chunk = (N + nch - 1) / nch;
  pl->xform = use_xform(ctx, P, nvars, N, &pl->ldxt);
  if (ctx->tile_cases > 0) {
    chunk = ctx->tile_cases;  // autotuned cases per work item
  } else if (pl->xform) {
    const long long cap = XFORM_SLICE_BYTES / (4ll * xform_rows(nvars, pl->xform));
    if (chunk > cap) chunk = (int)(cap > STEP ? cap : STEP);
  }
  chunk = (chunk + STEP - 1) / STEP * STEP;
  pl->chunk = chunk;
  pl->nchunks = (N + chunk - 1) / chunk;
  pl->items = (long long)P * pl->nchunks;
  const size_t tokens = (size_t)P * Lmax;
  Carver cv;
  pl->off_queue = cv.take(256);
  pl->off_flags = cv.take((size_t)P * 4);
  pl->off_ncode = cv.take((size_t)P * 4);
  pl->off_code = cv.take(tokens * 8);
  pl->off_part = cv.take((size_t)pl->items * PSTRIDE * 8);
  pl->off_yc = cv.take(align_up((size_t)N, STEP) * 4);
  pl->off_ych = cv.take((size_t)pl->nchunks * 16);
  pl->off_ysum = cv.take((size_t)pl->nchunks * 16);
  // the variable table: X's rows, then u(x_j) for the 12 unary operators
  // (those some program reads are filled per call); where the call is large
  // enough for it to pay and its row offsets fit the 32-bit operand
  pl->off_xt = pl->off_xneed = 0;
  if (pl->xform) {
    const size_t rows = (size_t)xform_rows(nvars, pl->xform);
    pl->off_xt = cv.take(rows * pl->ldxt * 4);
    pl->off_xneed = cv.take(rows - nvars);
  }
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
  if ((long long)ldx * nvars > 0xFFFFFFFFll)
    return fail(ctx, SR_EINVAL, "X too large: nvars * ldx must stay below 2^32 elements");
  if (P > 0 && (!programs || !lengths || (K > 0 && !consts) || !X))
    return fail(ctx, SR_EINVAL, "NULL input pointer");
  if (((uintptr_t)X) & 15) return fail(ctx, SR_EINVAL, "X must be 16-byte aligned");
  return SR_OK;
}

int mode_of(sr_fitness_kind k) {
  return k == SR_MSE ? MODE_MSE : (k == SR_CORR ? MODE_CORR : MODE_BOTH);
}

sr_status launch_eval(sr_ctx *ctx, int mode, const uint8_t *programs, const int32_t *lengths,
                      const float *consts, int P, int Lmax, int K, const float *X, const float *y,
                      int nvars, int N, int ldx, double *fitness, int32_t *prog_flags, float *yhat,
                      int ldy, int M = 0, int32_t *counts = nullptr) {
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  Plan pl;
  sr_status st = make_plan(ctx, mode, P, Lmax, N, &pl, nvars);
  if (st != SR_OK) return st;
  st = ensure_workspace(ctx, pl.bytes);
  if (st == SR_ENOMEM && pl.xform) {  // no room for the variable table: evaluate without it
    const int mode_x = ctx->xform;
    ctx->xform = 0;
    st = make_plan(ctx, mode, P, Lmax, N, &pl, nvars);
    ctx->xform = mode_x;
    if (st == SR_OK) st = ensure_workspace(ctx, pl.bytes);
  }
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
  ep.code = reinterpret_cast<uint2 *>(ws + pl.off_code);
  ep.ncode = reinterpret_cast<int32_t *>(ws + pl.off_ncode);
  ep.queue = reinterpret_cast<unsigned long long *>(ws + pl.off_queue);
  ep.yhat = yhat;
  ep.ldy = ldy;
  ep.slots = pl.slots;
  ep.warp_bytes = warp_smem_bytes(pl.slots, Lmax);
  ep.deep = 0;
  ep.abort = ctx->abort_flag;
  ep.err = ctx->dev_words;
  ep.score_M = M;
  ep.xform = pl.xform;
  ep.xneed = pl.xform ? reinterpret_cast<uint8_t *>(ws + pl.off_xneed) : nullptr;
  if (pl.xform) {  // the kernels read the variable table; the decoder writes its row offsets
    ep.X = reinterpret_cast<const float *>(ws + pl.off_xt);
    ep.ldx = pl.ldxt;
  }

  int grid_ext = 0, grid_deep = 0;
  st = grid_for_t<true>(ctx, mode, pl.minb, pl.smem, &grid_ext);
  if (st != SR_OK) return st;
  if (pl.smem_deep) {
    st = grid_for_t<true>(ctx, mode, 4, pl.smem_deep, &grid_deep);
    if (st != SR_OK) return st;
  }
  SR_CHECK_CUDA(ctx, cudaMemsetAsync(ep.queue, 0, 5 * sizeof(unsigned long long), s));
  if (pl.xform) SR_CHECK_CUDA(ctx, cudaMemsetAsync(ep.xneed, 0, (size_t)(xform_rows(nvars, pl.xform) - nvars), s));
  // one warp per block spreads the serial per-program decode over the SMs
  st = allow_dynamic_smem(ctx, reinterpret_cast<const void *>(decode_kernel));
  if (st != SR_OK) return st;
  decode_kernel<<<(P + DECODE_WARPS - 1) / DECODE_WARPS, DECODE_WARPS * 32, DECODE_WARPS * decode_warp_bytes(Lmax),
                  s>>>(ep);
  ctx->launches += 1;
  if (pl.xform) {
    const dim3 g((unsigned)((N + XF_THREADS * 4 - 1) / (XF_THREADS * 4)), (unsigned)xform_rows(nvars, pl.xform));
    xform_kernel<<<g, XF_THREADS, 0, s>>>(X, ldx, nvars, N, pl.ldxt, ep.xneed,
                                          reinterpret_cast<float *>(ws + pl.off_xt));
    ctx->launches += 1;
  }
  double *ych = reinterpret_cast<double *>(ws + pl.off_ych);
  if (mode == MODE_CORR || mode == MODE_BOTH || mode == MODE_R4) {
    double *ysum = reinterpret_cast<double *>(ws + pl.off_ysum);
    const int r4 = mode == MODE_R4;
    ysum_kernel<<<pl.nchunks, PREP_THREADS, 0, s>>>(y, N, pl.chunk, r4, ysum);
    ycenter_kernel<<<pl.nchunks, PREP_THREADS, 0, s>>>(y, N, pl.chunk, pl.nchunks, ysum, r4,
                                                      const_cast<float *>(ep.yc), ych);
    ctx->launches += 2;
  }
  launch_mode<false>(mode, pl.minb, pl.grid, pl.smem, s, ep);
  launch_mode<true>(mode, pl.minb, grid_ext, pl.smem, s, ep);
  ctx->launches += 2;
  if (pl.smem_deep) {
    EvalParams ed = ep;
    ed.deep = 1;
    ed.slots = slots_for(Lmax);
    ed.warp_bytes = warp_smem_bytes(ed.slots, Lmax);
    launch_mode<true>(mode, 4, grid_deep, pl.smem_deep, s, ed);
    ctx->launches += 1;
  }
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  if (mode != MODE_PREDICT) {
    FinalParams fp{ep.partials, ep.flags, ych, P, N, pl.chunk, pl.nchunks, mode, fitness, M, counts};
    finalize_kernel<<<(P + FINAL_WARPS - 1) / FINAL_WARPS, FINAL_WARPS * 32, 0, s>>>(fp);
    SR_CHECK_CUDA(ctx, cudaGetLastError());
    ctx->launches += 1;
  }
  return SR_OK;
}

// ---------------------------------------------------------------- batched host side
template <bool EXT, int MINB>
sr_status batched_grid_m(sr_ctx *ctx, int smem, int *grid) {
  sr_status st = allow_dynamic_smem(ctx, reinterpret_cast<const void *>(eval_batched_kernel<EXT, MINB>));
  if (st != SR_OK) return st;
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_batched_kernel<EXT, MINB>, WARPS * 32, smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (nb < 1) return fail(ctx, SR_EINVAL, "Lmax too large for shared memory");
  *grid = nb * ctx->num_sms;
  return SR_OK;
}

template <bool EXT>
sr_status batched_grid(sr_ctx *ctx, int minb, int smem, int *grid) {
  return minb == 3 ? batched_grid_m<EXT, 3>(ctx, smem, grid)
                   : (minb == 5 ? batched_grid_m<EXT, 5>(ctx, smem, grid) : batched_grid_m<EXT, 4>(ctx, smem, grid));
}

template <bool EXT>
void launch_batched_kernel(int minb, int grid, int smem, cudaStream_t s, const BatchParams &b) {
  if (minb == 3) eval_batched_kernel<EXT, 3><<<grid, WARPS * 32, smem, s>>>(b);
  else if (minb == 5) eval_batched_kernel<EXT, 5><<<grid, WARPS * 32, smem, s>>>(b);
  else eval_batched_kernel<EXT, 4><<<grid, WARPS * 32, smem, s>>>(b);
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
  // CTAs per SM of the main passes: 4 unless tuned (3 gives more stack slots
  // and registers, 5 more warps); it must leave room for min(slots_for, 4)
  // stack slots
  int bminb = ctx->batched_ctas ? ctx->batched_ctas : 4;
  if (bminb == 5 && WARPS * warp_smem_bytes(shallow_slots(maxL, 5), maxL) > smem_target(5)) bminb = 4;
  const int bslots = shallow_slots(maxL, bminb);
  const int smem = WARPS * warp_smem_bytes(bslots, maxL);
  const int smem_deep = slots_for(maxL) > bslots ? WARPS * warp_smem_bytes(slots_for(maxL), maxL) : 0;
  int grid = 0, grid_ext = 0, grid_deep = 0;
  sr_status st = batched_grid<false>(ctx, bminb, smem, &grid);
  if (st != SR_OK) return st;
  st = batched_grid<true>(ctx, bminb, smem, &grid_ext);
  if (st != SR_OK) return st;
  if (smem_deep) {
    st = batched_grid<true>(ctx, 4, smem_deep, &grid_deep);
    if (st != SR_OK) return st;
  }
  const long long warps = (long long)grid * WARPS;
  const double want = (double)warps * TARGET_ITEMS_PER_WARP;

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
      const int max_chunks = (q.N + STEP - 1) / STEP;
      n = n < 1 ? 1 : (n > max_chunks ? max_chunks : n);
      c = (q.N + n - 1) / n;
      int ldxt = 0;
      const int xf = use_xform(ctx, q.P, q.nvars, q.N, &ldxt);
      if (xf) {  // as in make_plan: the item's slice of the problem's table
        const long long cap = XFORM_SLICE_BYTES / (4ll * xform_rows(q.nvars, xf));
        if (c > cap) c = (int)(cap > STEP ? cap : STEP);
      }
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
    long long depth2 = 0;  // bytes of the group's tables with compositions
    const size_t off_q = cv.take(256);
    long long items = 0;
    int corr_chunks = 0, ncorr = 0, progs = 0;
    for (size_t g = g0; g < g1; ++g) {
      const int i = order[g];
      const sr_problem &q = pr[i];
      const int mode = mode_of(q.kind);
      const size_t tokens = (size_t)q.P * q.Lmax;
      const size_t off_f = q.prog_flags ? 0 : cv.take((size_t)q.P * 4);
      const size_t off_nc = cv.take((size_t)q.P * 4);
      const size_t off_code = cv.take(tokens * 8);
      const size_t off_p = cv.take((size_t)q.P * nch[i] * PSTRIDE * 8);
      size_t off_yc = 0, off_ych = 0, off_st = 0, off_xt = 0, off_xn = 0;
      const bool corr = mode != MODE_MSE;
      if (corr) {
        off_yc = cv.take(align_up((size_t)q.N, STEP) * 4);
        off_ych = cv.take((size_t)nch[i] * 16);
        off_st = cv.take((size_t)nch[i] * 16);
      }
      int ldxt = 0;
      int xf = use_xform(ctx, q.P, q.nvars, q.N, &ldxt);
      if (xf == 2) {
        const long long b2 = (long long)xform_rows(q.nvars, 2) * ldxt * 4;
        if (depth2 + b2 > XFORM2_BATCH_BYTES) xf = 1;
        else depth2 += b2;
      }
      if (xf) {
        const size_t rows = (size_t)xform_rows(q.nvars, xf);
        off_xt = cv.take(rows * ldxt * 4);
        off_xn = cv.take(rows - q.nvars);
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
        b.code = reinterpret_cast<uint2 *>(ws + off_code);
        b.ncode = reinterpret_cast<int32_t *>(ws + off_nc);
        b.fitness = q.fitness;
        b.ychunk = corr ? reinterpret_cast<double *>(ws + off_ych) : nullptr;
        b.ysum = corr ? reinterpret_cast<double *>(ws + off_st) : nullptr;
        b.ldx = q.ldx;
        b.item_begin = items;
        b.prog_begin = progs;
        b.P = q.P;
        b.Lmax = q.Lmax;
        b.K = q.K;
        b.nvars = q.nvars;
        b.N = q.N;
        b.chunk = chunk[i];
        b.nchunks = nch[i];
        b.mode = mode;
        b.corr_chunk_begin = corr ? corr_chunks : -1;
        b.xform = xf;
        b.xneed = xf ? reinterpret_cast<uint8_t *>(ws + off_xn) : nullptr;
        if (xf) {
          b.X = reinterpret_cast<const float *>(ws + off_xt);
          b.ldx = ldxt;
        }
        if (corr) bpar->corr_list[ncorr] = (int)(g - g0);
      }
      items += (long long)q.P * nch[i];
      progs += q.P;
      if (corr) {
        corr_chunks += nch[i];
        ++ncorr;
      }
    }
    if (bpar) {
      bpar->nprob = (int)(g1 - g0);
      bpar->ncorr = ncorr;
      bpar->total_progs = progs;
      bpar->total_items = items;
      bpar->queue = reinterpret_cast<unsigned long long *>(ctx->ws + off_q);
      bpar->slots = bslots;
      bpar->maxL = maxL;
      bpar->warp_bytes = warp_smem_bytes(bpar->slots, maxL);
      bpar->deep = 0;
      bpar->abort = ctx->abort_flag;
      bpar->err = ctx->dev_words;
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
  // no room for the variable tables: evaluate without them (the context's
  // setting comes back when the call returns)
  struct Restore {
    sr_ctx *c;
    int mode;
    ~Restore() { c->xform = mode; }
  } restore{ctx, ctx->xform};
  if (st == SR_ENOMEM && ctx->xform != 0) {
    ctx->xform = 0;
    need = 0;
    for (size_t g0 = 0; g0 < order.size(); g0 += MAX_BATCH) {
      const size_t g1 = std::min(order.size(), g0 + MAX_BATCH);
      need = std::max(need, group_bytes(g0, g1, nullptr));
    }
    st = ensure_workspace(ctx, need);
  }
  if (st != SR_OK) return st;

  cudaStream_t s = ctx->stream;
  for (size_t g0 = 0; g0 < order.size(); g0 += MAX_BATCH) {
    const size_t g1 = std::min(order.size(), g0 + MAX_BATCH);
    BatchParams b;
    group_bytes(g0, g1, &b);
    int corr_blocks = 0;
    for (int r = 0; r < b.ncorr; ++r) corr_blocks += b.prob[b.corr_list[r]].nchunks;
    SR_CHECK_CUDA(ctx, cudaMemsetAsync(b.queue, 0, 5 * sizeof(unsigned long long), s));
    for (int r = 0; r < b.nprob; ++r)
      if (b.prob[r].xform)
        SR_CHECK_CUDA(ctx, cudaMemsetAsync(b.prob[r].xneed, 0,
                                           (size_t)(xform_rows(b.prob[r].nvars, b.prob[r].xform) - b.prob[r].nvars), s));
    decode_batched_kernel<<<(b.total_progs + DECODE_WARPS - 1) / DECODE_WARPS, DECODE_WARPS * 32,
                            DECODE_WARPS * decode_warp_bytes(maxL), s>>>(b);
    ctx->launches += 1;
    for (size_t g = g0; g < g1; ++g) {  // the variable tables, from the problems' own X
      const BatchProblem &q = b.prob[g - g0];
      if (!q.xform) continue;
      const sr_problem &o = pr[order[g]];
      const dim3 xg((unsigned)((q.N + XF_THREADS * 4 - 1) / (XF_THREADS * 4)), (unsigned)xform_rows(q.nvars, q.xform));
      xform_kernel<<<xg, XF_THREADS, 0, s>>>(o.X, o.ldx, q.nvars, q.N, (int)q.ldx, q.xneed,
                                             const_cast<float *>(q.X));
      ctx->launches += 1;
    }
    if (b.ncorr > 0) {
      ysum_batched_kernel<<<corr_blocks, PREP_THREADS, 0, s>>>(b);
      ycenter_batched_kernel<<<corr_blocks, PREP_THREADS, 0, s>>>(b);
      ctx->launches += 2;
    }
    launch_batched_kernel<false>(bminb, grid, smem, s, b);
    launch_batched_kernel<true>(bminb, grid_ext, smem, s, b);
    ctx->launches += 2;
    if (smem_deep) {
      BatchParams bd = b;
      bd.deep = 1;
      bd.slots = slots_for(maxL);
      bd.warp_bytes = warp_smem_bytes(bd.slots, maxL);
      launch_batched_kernel<true>(4, grid_deep, smem_deep, s, bd);
      ctx->launches += 1;
    }
    int maxP = 1;
    for (int r = 0; r < b.nprob; ++r) maxP = b.prob[r].P > maxP ? b.prob[r].P : maxP;
    const int yblocks = std::min((maxP + FINAL_WARPS - 1) / FINAL_WARPS, 65535);
    finalize_batched_kernel<<<dim3(b.nprob, yblocks), FINAL_WARPS * 32, 0, s>>>(b);
    SR_CHECK_CUDA(ctx, cudaGetLastError());
    ctx->launches += 1;
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
  return launch_eval(ctx, mode_of(kind), programs, lengths, consts, P, Lmax, K, X, y, nvars, N, ldx,
                     fitness, prog_flags, nullptr, 0);
}

sr_status sr_eval_score(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths,
                        const float *consts, int P, int Lmax, int K, const float *X, const float *y,
                        int nvars, int N, int ldx, sr_score_kind kind, int M, double *score,
                        int32_t *pair_counts, int32_t *prog_flags) {
  using namespace sr;
  sr_status st = check_common(ctx, programs, lengths, consts, P, Lmax, K, X, nvars, N, ldx);
  if (st != SR_OK) return st;
  if (kind != SR_SCORE_R4 && kind != SR_SCORE_P2P)
    return fail(ctx, SR_EINVAL, "unknown score kind %d", (int)kind);
  if (M < 1 || M > (1 << 24)) return fail(ctx, SR_EINVAL, "M %d outside [1, 2^24]", M);
  if ((double)M * (double)N > 9007199254740992.0)
    return fail(ctx, SR_EINVAL, "M * N above 2^53: the score sum would not be exact");
  if (P == 0) return SR_OK;
  if (!y || !score) return fail(ctx, SR_EINVAL, "NULL y or score");
  if (((uintptr_t)y) & 15) return fail(ctx, SR_EINVAL, "y must be 16-byte aligned");
  return launch_eval(ctx, kind == SR_SCORE_R4 ? MODE_R4 : MODE_P2P, programs, lengths, consts, P, Lmax, K,
                     X, y, nvars, N, ldx, score, prog_flags, nullptr, 0, M, pair_counts);
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

sr_status sr_set_occupancy(sr_ctx *ctx, int eval_ctas_per_sm, int batched_ctas_per_sm) {
  if (!ctx) return SR_EINVAL;
  if (eval_ctas_per_sm != 0 && eval_ctas_per_sm != 4 && eval_ctas_per_sm != 5)
    return sr::fail(ctx, SR_EINVAL, "eval_ctas_per_sm %d: 0, 4 or 5", eval_ctas_per_sm);
  if (batched_ctas_per_sm != 0 && (batched_ctas_per_sm < 3 || batched_ctas_per_sm > 5))
    return sr::fail(ctx, SR_EINVAL, "batched_ctas_per_sm %d: 0, 3, 4 or 5", batched_ctas_per_sm);
  ctx->eval_ctas = eval_ctas_per_sm;
  ctx->batched_ctas = batched_ctas_per_sm;
  return SR_OK;
}

sr_status sr_set_transforms(sr_ctx *ctx, int mode) {
  if (!ctx) return SR_EINVAL;
  if (mode < 0 || mode > 2) return sr::fail(ctx, SR_EINVAL, "transform mode %d: 0, 1 or 2", mode);
  ctx->xform = mode;
  return SR_OK;
}

sr_status sr_reserve(sr_ctx *ctx, int P, int Lmax, int N) {
  using namespace sr;
  if (!ctx || P < 0 || Lmax < 1 || Lmax > SR_MAX_LMAX || N < 1) return SR_EINVAL;
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  size_t need = 0;
  for (int mode = 0; mode < 4; ++mode) {
    Plan pl;
    for (int nv = 1; nv <= SR_MAX_VARS; ++nv) {  // the table's size depends on the variable count
      sr_status st = make_plan(ctx, mode, P, Lmax, N, &pl, nv);
      if (st != SR_OK) return st;
      need = pl.bytes > need ? pl.bytes : need;
    }
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
  local.xform = 0;  // no variable table: the scratch stays within the terms sr.h lists
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
  const int mode = mode_of(kind);
  // fit the plan into the array: fewer SMs' worth of persistent CTAs means
  // fewer work items and partial records
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

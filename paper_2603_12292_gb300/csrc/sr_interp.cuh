// sr_interp.cuh -- the scheduled instruction stream shared by the evaluation
// kernels (sr_eval.cu) and the adjoint kernel (sr_grad.cu).
//
// A program (RPN, paper Sec. 2.1.4) is decoded once per call by a pre-pass,
// a warp per program (decode_warp): validation, then the expression tree is
// rescheduled Sethi-Ullman style -- at every binary node the child that needs
// more stack is evaluated first, with a reversed opcode keeping a - b and
// a / b exact when the right child goes first.  The number of live values is
// then at most floor(log2(leaves)) + 1: 9 for 512 tokens, so 8 stack slots
// below the top always suffice.  A terminal evaluated second is fused into
// its binary operator ("top = top op x_j").  Values are bit-identical to
// plain left-to-right evaluation: every operator sees the same operands.
#pragma once

#include "sr_common.cuh"

namespace sr {

// stack slots below the top register (see above)
constexpr int DSM = 8;
static_assert(SR_MAX_LMAX <= 512, "8 slots cover programs of up to 512 tokens");

// The slots programs of up to Lmax tokens can need: floor(log2(leaves)) with
// leaves <= (Lmax + 1) / 2.  Kernels size their shared stack by it (6 slots
// for Lmax = 128 instead of 8 -- more warps per SM).
__host__ __device__ inline int slots_for(int Lmax) {
  int leaves = (Lmax + 1) / 2, s = 0;
  while ((2 << s) <= leaves) ++s;
  return s < 1 ? 1 : (s > DSM ? DSM : s);
}

// ---------------------------------------------------------------- operators (FP32)
// The protected quotient.  The quotient itself comes from PTX div.full.f32:
// full range, at most 2 ulp off (subnormal results included) -- within the
// 2-ulp allowance the oracle's enclosure gives every operation.  Computed
// whatever b is and selected, so the vector loops stay branch-free.
// Measured on the paper-shaped population: +12 % over the IEEE quotient,
// whose longer sequence also pushed the interpreter loop out of the
// instruction cache; a redo of the subnormal results by the IEEE quotient
// cost back 11 %.
__device__ __forceinline__ float op_div(float a, float b) {
  float q;
  asm("div.full.f32 %0, %1, %2;" : "=f"(q) : "f"(a), "f"(b));
  // |b| < 1e-3f in FP32 is exactly "|b| <= 1e-3" for FP32 values of b
  return fabsf(b) < 1e-3f ? 1.0f : q;
}
__device__ __forceinline__ float op_log(float x) {
  return fabsf(x) < 1e-3f ? 0.0f : logf(fabsf(x));
}
__device__ __forceinline__ float op_exp(float x) {
  x = x > 80.0f ? 80.0f : (x < -80.0f ? -80.0f : x);  // NaN passes through
  return expf(x);
}
__device__ __forceinline__ float f_sqrt(float x) { return sqrtf(fabsf(x)); }

// sinf / cosf carry a long path for large arguments; keep one out-of-line
// copy of it and let the inlined copies assume a moderate argument (NaN and
// +-inf also take the out-of-line call)
static __device__ __noinline__ float sin_wide(float x) { return sinf(x); }
static __device__ __noinline__ float cos_wide(float x) { return cosf(x); }
__device__ __forceinline__ float f_sin(float x) {
  if (!(fabsf(x) <= 4.0e4f)) return sin_wide(x);
  __builtin_assume(fabsf(x) <= 4.0e4f);
  return sinf(x);
}
__device__ __forceinline__ float f_cos(float x) {
  if (!(fabsf(x) <= 4.0e4f)) return cos_wide(x);
  __builtin_assume(fabsf(x) <= 4.0e4f);
  return cosf(x);
}
static __device__ __noinline__ float tan_wide(float x) { return tanf(x); }
__device__ __forceinline__ float f_tan(float x) {
  if (!(fabsf(x) <= 4.0e4f)) return tan_wide(x);
  __builtin_assume(fabsf(x) <= 4.0e4f);
  return tanf(x);
}
// The rest of Table 1: 1/x protected like division; tan, asin, acos, atan,
// tanh as the FP32 library computes them (asin / acos outside [-1, 1] give
// NaN: a non-real result, which the NaN-aware scores of Eq. 2 / Eq. 3 take
// as an invalid output and MSE / 1 - r^2 as the worst fitness).
__device__ __forceinline__ float op_inv(float x) { return op_div(1.0f, x); }
__device__ __forceinline__ float f_asin(float x) { return asinf(x); }
__device__ __forceinline__ float f_acos(float x) { return acosf(x); }
__device__ __forceinline__ float f_atan(float x) { return atanf(x); }
__device__ __forceinline__ float f_tanh(float x) { return tanhf(x); }


// Instruction (uint2):
//   x bits 0..7   opcode
//   x bits 8..23  byte offset of the stack slot it pushes to / pops from
//   x bits 24..27 constant index k (constant operands only)
//   y             operand: FP32 bits of c_k, or the row offset j * ldx of x_j
enum Op : uint32_t {
  OP_LDV = 0,   // top = x_j                        (stack empty)
  OP_LDC,       // top = c_k
  OP_PUSHV,     // stack[slot] = top; top = x_j
  OP_PUSHC,     // stack[slot] = top; top = c_k
  OP_ADD,       // top = stack[slot] op top         (left operand evaluated first)
  OP_SUB,
  OP_MUL,
  OP_DIV,
  OP_RSUB,      // top = top - stack[slot]          (right operand evaluated first)
  OP_RDIV,      // top = top / stack[slot]
  OP_SIN,       // top = f(top)
  OP_COS,
  OP_EXP,
  OP_LOG,
  OP_SQRT,
  OP_SQ,
  OP_INV,       // 1 / top (protected as /)
  OP_TAN,
  OP_ASIN,
  OP_ACOS,
  OP_ATAN,
  OP_TANH,
  OP_VADD,      // top = top op x_j   (terminal right operand, evaluated second)
  OP_VSUB,
  OP_VMUL,
  OP_VDIV,
  OP_VRSUB,     // top = x_j - top    (terminal left operand, evaluated second)
  OP_VRDIV,     // top = x_j / top
  OP_CADD,      // top = top op c_k
  OP_CSUB,
  OP_CMUL,
  OP_CDIV,
  OP_CRSUB,     // top = c_k - top
  OP_CRDIV,     // top = c_k / top
};

__device__ __forceinline__ uint32_t ins_op(uint2 w) { return w.x & 0xffu; }
__device__ __forceinline__ uint32_t ins_off(uint2 w) { return (w.x >> 8) & 0xffffu; }
__device__ __forceinline__ int ins_k(uint2 w) { return (int)((w.x >> 24) & 0xfu); }

// ncode[p] holds the instruction count in its low 16 bits; NCODE_EXT is set
// when the program uses one of 1/x, tan, asin, acos, atan, tanh, so that
// the kernels can run those programs in a separate copy of their loop and
// keep the loop of the base operators free of the extra call site.
constexpr int NCODE_EXT = 1 << 30;
// NCODE_DEEP is set when the program needs more stack slots than the
// decoder's cap_slots: the evaluation kernels give most programs a few slots
// (more warps fit on an SM) and run the rare deeper ones in a separate pass.
constexpr int NCODE_DEEP = 1 << 29;
__device__ __forceinline__ int ncode_count(int v) { return v & 0xffff; }
__device__ __forceinline__ bool ncode_ext(int v) { return (v & NCODE_EXT) != 0; }
__device__ __forceinline__ bool ncode_deep(int v) { return (v & NCODE_DEEP) != 0; }

struct DecodeArgs {
  const uint8_t *programs;  // [P][Lmax]
  const int32_t *lengths;
  const float *consts;      // [P][K]
  int Lmax, K, nvars;
  long long ldx;
  int slot_bytes;           // bytes between consecutive stack slots of a warp
  uint2 *code;              // [P][Lmax] out
  int32_t *ncode;           // [P] out
  int32_t *flags;           // [P] out
  unsigned long long *ext_count;  // programs with NCODE_EXT are counted here (or NULL)
  int max_slots;            // stack slots the kernel provides (<= DSM)
  int cap_slots;            // programs that need more than this get NCODE_DEEP (<= max_slots)
  unsigned long long *deep_count;  // programs with NCODE_DEEP are counted here (or NULL)
  int fold;                 // 1: fold constant-only subtrees into one constant (evaluation only)
  int adj_info;             // 1: mark what the adjoint sweep needs (INS_NOADJ / INS_SA / INS_TA)
  // >= 1 (evaluation only): a unary operator applied to a variable, u(x_j),
  // reads row xform_row(nvars, u, j) of the variable table instead (the
  // table's first nvars rows are X); with 2, also a base unary operator
  // applied to a base u(x_j), u(v(x_j)), reads row xform_row2(nvars, u, v, j).
  // The decoder marks in xneed[row - nvars] each row some program reads, and
  // a kernel fills those rows before the evaluation.  ldx is then the
  // table's row stride.
  int xform = 0;
  uint8_t *xneed = nullptr;
};

// The variable table of an evaluation with transforms: X's nvars rows, then
// u(x_j) for the twelve unary operators, then (depth 2) u(v(x_j)) for the
// 36 pairs of the six base ones (sin cos exp log sqrt sq).
constexpr int XFORM_BASE = TOK_SQ - TOK_SIN + 1;
__host__ __device__ inline int xform_row(int nvars, int u, int j) { return nvars + (u - TOK_SIN) * nvars + j; }
__host__ __device__ inline int xform_row2(int nvars, int u, int v, int j) {
  return nvars * (1 + UNARY_ALL) + ((u - TOK_SIN) * XFORM_BASE + (v - TOK_SIN)) * nvars + j;
}
__host__ __device__ inline int xform_rows(int nvars, int depth) {
  return nvars * (1 + UNARY_ALL + (depth > 1 ? XFORM_BASE * XFORM_BASE : 0));
}

// Instruction flags for the adjoint kernel (bits 28-30 of x; evaluation
// ignores them).  A constant's derivative flows only through nodes whose
// subtree reads a constant:
//   INS_NOADJ  this operator's subtree reads no constant: the forward pass
//              tapes nothing for it, and the reverse sweep jumps from it to
//              the subtree's first instruction (a variable load, whose
//              reverse restores the outer adjoint); the jump target is in y,
//              or, for an operator fused with a variable (VADD ... VRDIV),
//              in the slot-offset field
//   INS_SA     (binary operator with a stack operand) the operand in the
//              stack slot reads a constant: its adjoint is wanted
//   INS_TA     the operand on top reads a constant: its adjoint is wanted
constexpr uint32_t INS_NOADJ = 1u << 28, INS_SA = 1u << 29, INS_TA = 1u << 30;

__device__ __forceinline__ bool is_term(int v) {
  const int c = tok_class(v);
  return c == CLS_VAR || c == CLS_CONST;
}

__device__ __forceinline__ uint2 with_operand(uint32_t x, int v, const float *crow, long long ldx) {
  if (tok_class(v) == CLS_VAR) return make_uint2(x, (uint32_t)((long long)(v - TOK_VAR0) * ldx));
  const int k = v - TOK_CONST0;
  return make_uint2(x | ((uint32_t)k << 24), __float_as_uint(crow[k]));
}

// The FP32 value of an operator node whose operands are constants, by the
// same functions the interpreter applies to every case, so that a folded
// subtree gives the bits its per-case evaluation gives.  Each operation is
// one function call: nothing is contracted across operations.
static __device__ __noinline__ float fold_op(int v, float a, float b) {
  switch (v) {
    case TOK_ADD: return __fadd_rn(a, b);
    case TOK_SUB: return __fsub_rn(a, b);
    case TOK_MUL: return __fmul_rn(a, b);
    case TOK_DIV: return op_div(a, b);
    case TOK_SIN: return f_sin(a);
    case TOK_COS: return f_cos(a);
    case TOK_EXP: return op_exp(a);
    case TOK_LOG: return op_log(a);
    case TOK_SQRT: return f_sqrt(a);
    case TOK_SQ: return __fmul_rn(a, a);
    case TOK_INV: return op_inv(a);
    case TOK_TAN: return f_tan(a);
    case TOK_ASIN: return f_asin(a);
    case TOK_ACOS: return f_acos(a);
    case TOK_ATAN: return f_atan(a);
    default: return f_tanh(a);
  }
}

constexpr uint8_t NEED_FOLDED = 0x80;  // need[] bit: the subtree reads only constants (folded)
constexpr uint8_t NEED_HASC = 0x40;    // need[] bit: the subtree reads a constant (adjoint info)
constexpr uint8_t NEED_XVAR = 0x20;    // need[] bit: u(x_j), read from the variable table (xform)
constexpr uint8_t NEED_COUNT = 0x1f;   // need[] bits: the stack need itself

// Validation and scheduled decoding of program `prog` (one thread), reading
// its tokens from `tok`, its constants from `crow` and using the scratch rows
// start / need / task (Lmax entries each).
// Flag rules: length outside [1, Lmax]; bad byte; variable / constant index
// out of range; depth (running sum of +1 terminal, 0 unary or bad byte, -1
// binary) below 1 after some token; final depth not 1.
__device__ inline void decode_one(const DecodeArgs &p, int prog, const uint8_t *tok, int16_t *start,
                                  uint8_t *need, int16_t *task, const float *crow, float *fval, int L) {
  int flags = 0;
  if (L < 1 || L > p.Lmax) {
    flags = SR_PF_BAD_LENGTH;
  } else {
    int depth = 0;
    for (int t = 0; t < L; ++t) {
      const int v = tok[t];
      const int cls = tok_class(v);
      if (cls == CLS_BAD) flags |= SR_PF_BAD_TOKEN;
      if (cls == CLS_VAR && v - TOK_VAR0 >= p.nvars) flags |= SR_PF_BAD_VAR;
      if (cls == CLS_CONST && v - TOK_CONST0 >= p.K) flags |= SR_PF_BAD_CONST;
      depth += cls_effect(cls);
      if (depth < 1) flags |= SR_PF_UNDERFLOW;
    }
    if (depth != 1) flags |= SR_PF_BAD_FINAL;
  }
  p.flags[prog] = flags;
  if (flags) {
    p.ncode[prog] = 0;
    return;
  }
  int ext = 0;
  // pass 1, postfix order is bottom-up: subtree starts and stack needs
  // (terminal 1; unary as its child; binary max of the children, +1 on a tie).
  // With p.fold, a subtree that reads only constants is evaluated here, once,
  // and becomes a constant leaf (need 1, NEED_FOLDED, value in fval).
  int sp = 0;
  for (int t = 0; t < L; ++t) {
    const int v = tok[t];
    const int cls = tok_class(v);
    if (cls == CLS_VAR || cls == CLS_CONST) {
      start[t] = (int16_t)t;
      need[t] = 1;
      if (p.fold && cls == CLS_CONST) {
        need[t] = 1 | NEED_FOLDED;
        fval[t] = crow[v - TOK_CONST0];
      }
      if (p.adj_info && cls == CLS_CONST) need[t] |= NEED_HASC;
      task[sp++] = (int16_t)t;
    } else if (cls == CLS_UNARY) {
      const int c = task[sp - 1];
      start[t] = start[c];
      if (need[c] & NEED_FOLDED) {
        need[t] = 1 | NEED_FOLDED;
        fval[t] = fold_op(v, fval[c], 0.0f);
      } else if (p.xform && tok_class(tok[c]) == CLS_VAR) {
        // u(x_j): a leaf reading the transformed variable's row (its index in fval)
        const int j = tok[c] - TOK_VAR0;
        const int row = xform_row(p.nvars, v, j);
        need[t] = 1 | NEED_XVAR;
        reinterpret_cast<int32_t *>(fval)[t] = row;
        p.xneed[row - p.nvars] = 1;
      } else if (p.xform > 1 && (need[c] & NEED_XVAR) && v <= TOK_SQ &&
                 reinterpret_cast<const int32_t *>(fval)[c] < xform_row(p.nvars, TOK_SQ + 1, 0)) {
        // u(v(x_j)) of base operators: the row of the composition
        const int k = reinterpret_cast<const int32_t *>(fval)[c] - p.nvars;
        const int row = xform_row2(p.nvars, v, TOK_SIN + k / p.nvars, k % p.nvars);
        need[t] = 1 | NEED_XVAR;
        reinterpret_cast<int32_t *>(fval)[t] = row;
        p.xneed[row - p.nvars] = 1;
      } else {
        ext |= v > TOK_SQ;
        need[t] = need[c] & (uint8_t)~NEED_XVAR;
      }
      task[sp - 1] = (int16_t)t;
    } else {
      const int b = task[--sp], a = task[sp - 1];
      start[t] = start[a];
      if ((need[a] & need[b]) & NEED_FOLDED) {
        need[t] = 1 | NEED_FOLDED;
        fval[t] = fold_op(v, fval[a], fval[b]);
      } else {
        const int na = need[a] & NEED_COUNT, nb = need[b] & NEED_COUNT;
        need[t] = (uint8_t)((na == nb ? na + 1 : (na > nb ? na : nb)) | ((need[a] | need[b]) & NEED_HASC));
      }
      task[sp - 1] = (int16_t)t;
    }
  }
  // pass 2, emission: depth-first from the root, larger-need child first;
  // work stack entries are node << 2 | phase.  d counts the live values
  // (top included): a terminal pushes the old top into slot d - 1, a binary
  // operator pops slot d - 2.
  uint2 *code = p.code + (size_t)prog * p.Lmax;
  int n = 0, d = 0, used = 0;
  sp = 0;
  task[sp++] = (int16_t)((L - 1) << 2);
  // a leaf's operand: x_j, c_k, or a folded subtree's value (constant index
  // 0: the evaluation kernels read only the value)
  auto operand = [&](uint32_t x, int node) -> uint2 {
    if (need[node] & NEED_FOLDED) return make_uint2(x, __float_as_uint(fval[node]));
    if (need[node] & NEED_XVAR)
      return make_uint2(x, (uint32_t)((long long)reinterpret_cast<const int32_t *>(fval)[node] * p.ldx));
    return with_operand(x, tok[node], crow, p.ldx);
  };
  auto is_leaf = [&](int node) { return is_term(tok[node]) || (need[node] & (NEED_FOLDED | NEED_XVAR)) != 0; };
  // a leaf that reads a row of the variable table: x_j, or u(x_j) with transforms
  auto reads_row = [&](int node) {
    return (need[node] & NEED_XVAR) != 0 || (!(need[node] & NEED_FOLDED) && tok_class(tok[node]) == CLS_VAR);
  };
  // adjoint info: the first instruction of every subtree (fval's storage,
  // unused without folding) and the flags of an operator instruction
  int32_t *first_ins = reinterpret_cast<int32_t *>(fval);
  auto adj = [&](uint2 w, int node, bool fused_var, int slot_op, int top_op) -> uint2 {
    if (!p.adj_info) return w;
    if (!(need[node] & NEED_HASC)) {
      w.x |= INS_NOADJ;
      if (fused_var) w.x = (w.x & ~(0xffffu << 8)) | ((uint32_t)first_ins[node] << 8);
      else w.y = (uint32_t)first_ins[node];
      return w;
    }
    if (slot_op >= 0 && (need[slot_op] & NEED_HASC)) w.x |= INS_SA;
    if (top_op >= 0 && (need[top_op] & NEED_HASC)) w.x |= INS_TA;
    return w;
  };
  while (sp > 0) {
    const int e = task[sp - 1];
    const int node = e >> 2, ph = e & 3;
    const int v = tok[node];
    const int cls = is_leaf(node) ? (reads_row(node) ? CLS_VAR : CLS_CONST) : tok_class(v);
    if (p.adj_info && ph == 0) first_ins[node] = n;
    if (cls == CLS_VAR || cls == CLS_CONST) {
      --sp;
      if (d > p.max_slots) {  // cannot happen for programs of <= Lmax tokens; never write past the slots
        p.flags[prog] = SR_PF_TOO_DEEP;
        p.ncode[prog] = 0;
        return;
      }
      const bool var = cls == CLS_VAR;
      uint32_t op = var ? OP_LDV : OP_LDC;
      if (d > 0) op = (uint32_t)(var ? OP_PUSHV : OP_PUSHC) | ((uint32_t)((d - 1) * p.slot_bytes) << 8);
      used = d > used ? d : used;  // slots 0 .. d - 1 are in use
      code[n++] = operand(op, node);
      ++d;
    } else if (cls == CLS_UNARY) {
      if (ph == 0) {
        task[sp - 1] = (int16_t)(e | 1);
        task[sp++] = (int16_t)((node - 1) << 2);
      } else {
        --sp;
        code[n] = adj(make_uint2((uint32_t)(OP_SIN + (v - TOK_SIN)), 0u), node, false, -1, node - 1);
        ++n;
      }
    } else {
      const int b = node - 1, a = start[b] - 1;
      const bool rev = (need[b] & NEED_COUNT) > (need[a] & NEED_COUNT);
      const int first = rev ? b : a, second = rev ? a : b;
      if (ph == 0) {
        task[sp - 1] = (int16_t)(e | 1);
        task[sp++] = (int16_t)(first << 2);
      } else if (ph == 1 && is_leaf(second)) {
        --sp;
        const bool var = reads_row(second);
        uint32_t op;
        if (rev && v == TOK_SUB) op = var ? OP_VRSUB : OP_CRSUB;
        else if (rev && v == TOK_DIV) op = var ? OP_VRDIV : OP_CRDIV;
        else op = (uint32_t)((var ? OP_VADD : OP_CADD) + v);  // + and * commute exactly
        code[n] = adj(operand(op, second), node, var, -1, first);
        ++n;
      } else if (ph == 1) {
        task[sp - 1] = (int16_t)((e & ~3) | 2);
        task[sp++] = (int16_t)(second << 2);
      } else {
        --sp;
        uint32_t op;
        if (rev && v == TOK_SUB) op = OP_RSUB;
        else if (rev && v == TOK_DIV) op = OP_RDIV;
        else op = (uint32_t)(OP_ADD + v);
        code[n] = adj(make_uint2(op | ((uint32_t)((d - 2) * p.slot_bytes) << 8), 0u), node, false, first, second);
        ++n;
        --d;
      }
    }
  }
  const bool deep = used > p.cap_slots;
  p.ncode[prog] = n | (ext ? NCODE_EXT : 0) | (deep ? NCODE_DEEP : 0);
  if (ext && p.ext_count) atomicAdd(p.ext_count, 1ull);
  if (deep && p.deep_count) atomicAdd(p.deep_count, 1ull);
}

// Decoding by warps in shared memory: one warp per program.  The warp copies
// the program's token row and constants with coalesced loads, then lane 0
// decodes it with its scratch in shared memory.  The tree walk is serial and
// branchy: a lane per program of a 32-program warp serialised the lanes'
// different paths (9 of 32 threads active on average) and left one warp per
// SM; a warp per program spreads the programs over every SM and keeps
// several warps per scheduler to hide the walk's latency.
// Dynamic shared memory per warp: decode_warp_bytes.
// layout: tokens [Lmax + 4] | need [Lmax + 4] | start [Lmax + 2] int16 |
// task [Lmax + 2] int16 | constants [SR_MAX_CONSTS] float (4-byte aligned) |
// folded values [Lmax] float
__host__ __device__ inline int decode_consts_offset(int Lmax) { return (6 * Lmax + 16 + 3) & ~3; }
__host__ __device__ inline int decode_fval_offset(int Lmax) { return decode_consts_offset(Lmax) + SR_MAX_CONSTS * 4; }
__host__ __device__ inline int decode_warp_bytes(int Lmax) {
  return (decode_fval_offset(Lmax) + 4 * Lmax + 15) & ~15;
}
constexpr int DECODE_WARPS = 4;  // warps (programs) per block of the decode kernels

// Program `prog` decoded by the calling warp in its shared region `base`
// (decode_warp_bytes(Lmax) bytes for some Lmax >= p.Lmax).
__device__ inline void decode_warp_one(const DecodeArgs &p, int prog, unsigned char *base) {
  const int lane = threadIdx.x & 31;
  const int Lt = p.Lmax + 4, Ls = p.Lmax + 2;
  uint8_t *toks = base;                                          // [Lt]
  uint8_t *need = base + Lt;                                     // [Lt]
  int16_t *start = reinterpret_cast<int16_t *>(base + 2 * Lt);   // [Ls]
  int16_t *task = start + Ls;                                    // [Ls]
  float *cs = reinterpret_cast<float *>(base + decode_consts_offset(p.Lmax));
  float *fv = reinterpret_cast<float *>(base + decode_fval_offset(p.Lmax));
  const uint8_t *src = p.programs + (size_t)prog * p.Lmax;
  for (int b = lane; b < p.Lmax; b += 32) toks[b] = src[b];
  if (lane < p.K) cs[lane] = p.consts[(size_t)prog * p.K + lane];
  const int L = p.lengths[prog];
  __syncwarp();
  if (lane == 0) decode_one(p, prog, toks, start, need, task, cs, fv, L);
}

__device__ inline void decode_warp(const DecodeArgs &p, int P, unsigned char *smem) {
  const int warp = threadIdx.x >> 5;
  const int prog = blockIdx.x * (blockDim.x >> 5) + warp;
  if (prog >= P) return;
  decode_warp_one(p, prog, smem + (size_t)warp * decode_warp_bytes(p.Lmax));
}

}  // namespace sr

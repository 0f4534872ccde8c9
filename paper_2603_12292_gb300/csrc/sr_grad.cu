// sr_grad.cu -- reverse-mode derivative of the interpreter (dMSE/dconst) and
// the Adam update of the constants.
//
// The adjoint runs over the same scheduled instruction stream as evaluation
// (sr_interp.cuh: Sethi-Ullman order, at most 8 stack slots, fused terminal
// operators).  Work item = (case chunk, program), one warp, 4 cases per lane
// (one float4 per value), 128 cases per step.  Per step:
//   forward  -- the program runs with the top of stack in registers and the
//               slots below in shared memory.  What the reverse sweep needs
//               goes on a LIFO tape: for a unary operator its local
//               derivative, computed here next to the value (cos x with
//               sin x from one sincos, exp x, 1/x, +-1/(2 sqrt|x|), 2x,
//               1 + tan^2 x, ...), so
//               that the reverse step is one multiply; for a product both
//               factors; for a quotient the denominator and the result.  A
//               terminal operand fused into * or / needs no entry (x_j is
//               re-read, c_k is in the instruction).  The tape lives in
//               shared memory when a whole one (Lmax entries) fits there,
//               else in this warp's global scratch: most of it is in L2, its
//               latency hidden by 40 warps per SM.
//   reverse  -- the instructions are walked backwards with the adjoint of
//               the top in registers; a binary operator writes the adjoint
//               of the operand it popped into that operand's stack slot (the
//               values there are dead by then), and the push that produced
//               the operand reads it back; constants add their adjoint into
//               their gradient sum.
// Nothing is kept between an evaluation and this call: the forward pass is
// recomputed.  Sums: per lane FP32 compensated (Kahan) over the item's
// cases, FP64 across lanes (shuffles) and chunks (fixed-order finalize).
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sr_common.cuh"
#include "sr_interp.cuh"

namespace sr {
namespace {

constexpr int GWARPS = 8;                // warps per CTA
#ifndef SR_GRAD_CPL
#define SR_GRAD_CPL 4
#endif
constexpr int GCPL = SR_GRAD_CPL;        // cases per lane (2: one float2, 4: one float4)
static_assert(GCPL == 2 || GCPL == 4, "2 or 4 cases per lane");
constexpr int GSTEP = 32 * GCPL;         // cases per warp step
constexpr int GSLOT = GSTEP * 4;         // bytes of one stack slot / tape entry of a warp
constexpr int GSTRIDE = 32;              // doubles per partial record: [0] sum e^2, [1 + k] sum e dyhat/dc_k
constexpr int GTARGET_ITEMS_PER_WARP = 24;
// Shared-memory budget: GCTAS_PER_SM CTAs of 8 warps per SM, the register
// limit (2 cases per lane: 40 registers, 48 warps; 4: 48 registers, 40
// warps).  Unless a whole tape fits in a warp's share, the tape goes to the
// warp's scratch, which stays mostly in L2.  Measured on 2,048 x 131,072
// (K = 8, L <= 96), 2 cases per lane: 12 warps per SM with a 56-entry shared
// tape 366 GPop/s, 24 -> 579, 32 -> 674, 40 -> 747, 48 -> 791; 48 with the
// tape wholly in the scratch instead of its first 2 entries in shared memory
// (no per-access choice) 831.  4 cases per lane (the dispatch of each
// instruction shared by twice the cases) 980; 8 per lane 371.
constexpr int GCTAS_PER_SM = GCPL == 2 ? 6 : 5;

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
  uint2 *code;        // [P][Lmax] scheduled instructions (slot bytes GSLOT)
  int32_t *ncode;     // [P]
  unsigned long long *queue;
  char *gtape;        // per warp: Lmax entries of GSLOT bytes (tape off chip), else NULL
  const int32_t *abort;  // sr_set_abort_flag (or NULL)
  unsigned *err;         // the context's latched error word
  int warp_bytes;
};

// shared memory of one warp: stack slots [slots_for(Lmax)] | gradient sums
// and compensations [2][K][32] | code [Lmax] | tape [Lmax] (tape on chip only)
__host__ __device__ inline int grad_fixed_bytes(int Lmax, int K) {
  return slots_for(Lmax) * GSLOT + 2 * K * 128 + ((Lmax * 8 + 15) / 16) * 16;
}

__device__ __forceinline__ DecodeArgs grad_decode_args(const GradParams &p) {
  DecodeArgs a;
  a.programs = p.programs;
  a.lengths = p.lengths;
  a.consts = p.consts;
  a.Lmax = p.Lmax;
  a.K = p.K;
  a.nvars = p.nvars;
  a.ldx = p.ldx;
  a.slot_bytes = GSLOT;
  a.code = p.code;
  a.ncode = p.ncode;
  a.flags = p.flags;
  a.ext_count = nullptr;
  a.max_slots = slots_for(p.Lmax);
  a.cap_slots = a.max_slots;  // one pass: no program is deep
  a.deep_count = nullptr;
  a.fold = 0;  // every constant keeps its own slot: its derivative is wanted
  a.adj_info = 1;
  a.xform = 0;  // the adjoint reads X itself
  a.xneed = nullptr;
  return a;
}

__global__ void grad_decode_kernel(GradParams p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  decode_warp(grad_decode_args(p), p.P, dsm);
}

// ---------------------------------------------------------------- per-lane vectors
// VG: this lane's GCPL cases of one value (one float2 or float4 in memory)
struct alignas(GCPL * 4) VG {
  float v[GCPL];
};
__device__ __forceinline__ VG splatg(float c) {
  VG r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) r.v[i] = c;
  return r;
}
#define SR_VG_BINOP(name, expr)                                   \
  __device__ __forceinline__ VG name(VG a, VG b) {                \
    VG r;                                                         \
    _Pragma("unroll") for (int i = 0; i < GCPL; ++i) r.v[i] = expr; \
    return r;                                                     \
  }
SR_VG_BINOP(addg, a.v[i] + b.v[i])
SR_VG_BINOP(subg, a.v[i] - b.v[i])
SR_VG_BINOP(mulg, a.v[i] * b.v[i])
#undef SR_VG_BINOP
__device__ __forceinline__ VG negg(VG a) {
  VG r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) r.v[i] = -a.v[i];
  return r;
}
// a value and its local derivative, from the forward operators below
struct VD {
  VG v, d;
};

// Out-of-line operators (one copy of each long body keeps the interpreter
// loop inside the instruction cache).  fwd_* return the value and the local
// derivative under these conventions at the kinks: a protected fallback, a
// clamped exp and sqrt|x| at 0 have derivative 0.
static __device__ __noinline__ float2 sincos_wide(float x) {
  float s, c;
  sincosf(x, &s, &c);
  return make_float2(s, c);
}
__device__ __forceinline__ float2 f_sincos(float x) {
  if (!(fabsf(x) <= 4.0e4f)) return sincos_wide(x);
  __builtin_assume(fabsf(x) <= 4.0e4f);
  float s, c;
  sincosf(x, &s, &c);
  return make_float2(s, c);
}
__device__ __noinline__ VD fwd_sin(VG x) {
  VD r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) {
    const float2 sc = f_sincos(x.v[i]);
    r.v.v[i] = sc.x;
    r.d.v[i] = sc.y;
  }
  return r;
}
__device__ __noinline__ VD fwd_cos(VG x) {
  VD r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) {
    const float2 sc = f_sincos(x.v[i]);
    r.v.v[i] = sc.y;
    r.d.v[i] = -sc.x;
  }
  return r;
}
__device__ __forceinline__ float d_exp(float x, float v) { return (x > 80.0f || x < -80.0f) ? 0.0f : v; }
__device__ __noinline__ VD fwd_exp(VG x) {
  VD r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) {
    r.v.v[i] = op_exp(x.v[i]);
    r.d.v[i] = d_exp(x.v[i], r.v.v[i]);
  }
  return r;
}
__device__ __forceinline__ float d_log(float x) { return fabsf(x) < 1e-3f ? 0.0f : 1.0f / x; }
__device__ __noinline__ VD fwd_log(VG x) {
  VD r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) {
    r.v.v[i] = op_log(x.v[i]);
    r.d.v[i] = d_log(x.v[i]);
  }
  return r;
}
__device__ __forceinline__ float d_sqrt(float x, float v) { return x == 0.0f ? 0.0f : copysignf(0.5f / v, x); }
__device__ __noinline__ VD fwd_sqrt(VG x) {
  VD r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) {
    r.v.v[i] = f_sqrt(x.v[i]);
    r.d.v[i] = d_sqrt(x.v[i], r.v.v[i]);
  }
  return r;
}
// the rest of Table 1: 1/x (derivative -1/x^2, 0 where the fallback was
// taken), tan (1 + tan^2), asin (1/sqrt(1 - x^2)), acos (-1/sqrt(1 - x^2)),
// atan (1/(1 + x^2)), tanh (sech^2)
__device__ __forceinline__ float d_inv(float x, float v) { return fabsf(x) < 1e-3f ? 0.0f : -(v * v); }
// 1 - x^2 as (1 - x)(1 + x): no cancellation near |x| = 1
__device__ __forceinline__ float d_asin(float x) { return 1.0f / sqrtf((1.0f - x) * (1.0f + x)); }
// sech^2 x = 4e / (1 + e)^2 with e = exp(-2|x|): 1 - tanh^2 would cancel
// to 0 long before the derivative underflows
__device__ __forceinline__ float d_tanh(float x) {
  const float e = expf(-2.0f * fabsf(x));
  const float q = 1.0f + e;
  return 4.0f * e / (q * q);
}
__device__ __forceinline__ float2 fwd_ext1(uint32_t op, float x) {
  switch (op) {
    case OP_INV: {
      const float a = op_inv(x);
      return make_float2(a, d_inv(x, a));
    }
    case OP_TAN: {
      const float a = f_tan(x);
      return make_float2(a, 1.0f + a * a);
    }
    case OP_ASIN: return make_float2(f_asin(x), d_asin(x));
    case OP_ACOS: return make_float2(f_acos(x), -d_asin(x));
    case OP_ATAN: return make_float2(f_atan(x), 1.0f / (1.0f + x * x));
    default: return make_float2(f_tanh(x), d_tanh(x));
  }
}
// one out-of-line entry for all of them keeps the forward switch small
__device__ __noinline__ VD fwd_ext(uint32_t op, VG x) {
  VD r;
#pragma unroll 1
  for (int i = 0; i < GCPL; ++i) {
    const float2 vd = fwd_ext1(op, x.v[i]);
    r.v.v[i] = vd.x;
    r.d.v[i] = vd.y;
  }
  return r;
}
// protected quotient (the interpreter's operator)
__device__ __noinline__ VG pdivg(VG a, VG b) {
  VG r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) r.v[i] = op_div(a.v[i], b.v[i]);
  return r;
}
// adjoint through a protected quotient: a / den, 0 where the fallback was taken
__device__ __forceinline__ float qdiv(float a, float d) { return fabsf(d) < 1e-3f ? 0.0f : a / d; }
__device__ __noinline__ VG qdivg(VG a, VG d) {
  VG r;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) r.v[i] = qdiv(a.v[i], d.v[i]);
  return r;
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

struct GradWarp {
  char *slot;    // this lane's entry of stack slot 0 (shared)
  float *gs;     // gradient sums [K][32] (shared)
  float *gc;     // their compensations [K][32]
  uint2 *code;   // this warp's code (shared)
  char *ts;      // this lane's entry of tape entry 0 (shared; ONCHIP)
  char *tg;      // this lane's entry of tape entry 0 (the warp's global scratch; !ONCHIP)
  int lane;
};

__device__ __forceinline__ VG *slot_at(const GradWarp &w, uint32_t off) {
  return reinterpret_cast<VG *>(w.slot + off);
}
// ONCHIP: the whole tape is in shared memory, else wholly in the scratch
template <bool ONCHIP>
__device__ __forceinline__ VG *tape_at(const GradWarp &w, int i) {
  return reinterpret_cast<VG *>((ONCHIP ? w.ts : w.tg) + (size_t)i * GSLOT);
}
// add this lane's valid cases of v (bit i of okm: case i is inside the
// chunk) into constant k's compensated sum
// (out of line: eight call sites in the reverse sweep; one copy keeps the
// loop inside the instruction cache, measured 962 -> 1,002 GPop/s)
__device__ __noinline__ void gacc(const GradWarp &w, int k, VG v, unsigned okm) {
  float x = 0.0f;
#pragma unroll
  for (int i = 0; i < GCPL; ++i) x += ((okm >> i) & 1u) ? v.v[i] : 0.0f;
  float *s = w.gs + k * 32 + w.lane, *c = w.gc + k * 32 + w.lane;
  const float sv = *s, cv = *c;
  const float yv = x - cv;
  const float t = sv + yv;
  *c = (t - sv) - yv;
  *s = t;
}
__device__ __forceinline__ VG ldxg(const float *xr, uint32_t off) {
  VG r;
  if (GCPL == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(xr + off));
    r.v[0] = q.x;
    r.v[1] = q.y;
    r.v[GCPL > 2 ? 2 : 0] = q.z;
    r.v[GCPL > 3 ? 3 : 1] = q.w;
  } else {
    const float2 q = __ldg(reinterpret_cast<const float2 *>(xr + off));
    r.v[0] = q.x;
    r.v[1] = q.y;
  }
  return r;
}

// One work item: program `prog` on case chunk `c` with the calling warp.
// w's shared regions are laid out for the largest Lmax and K of the launch
// (at least p's).
template <bool ONCHIP>
__device__ __forceinline__ void grad_item(const GradParams &p, int c, int prog, const GradWarp &w, int lane) {
  if (p.flags[prog]) return;
  const int n = ncode_count(p.ncode[prog]);
  __syncwarp();
  const uint2 *src = p.code + (size_t)prog * p.Lmax;
  for (int i = lane; i < n; i += 32) w.code[i] = src[i];
  for (int k = 0; k < p.K; ++k) {
    w.gs[k * 32 + lane] = 0.f;
    w.gc[k * 32 + lane] = 0.f;
  }
  __syncwarp();

  const int cbeg = c * p.chunk, cend = min(p.N, cbeg + p.chunk);
  const int last_group = (cend - 1) & ~(GCPL - 1);
  Kahan se;
  for (int base = cbeg; base < cend; base += GSTEP) {
    const int c0 = base + GCPL * lane;
    unsigned okm = 0;  // bit i: case c0 + i is inside the chunk
#pragma unroll
    for (int i = 0; i < GCPL; ++i) okm |= (c0 + i < cend ? 1u : 0u) << i;
    const float *xr = p.X + (okm ? c0 : last_group);
    int tp = 0;
    auto push = [&](VG v) { *tape_at<ONCHIP>(w, tp++) = v; };
    auto pop = [&]() { return *tape_at<ONCHIP>(w, --tp); };
    // ---- forward
    VG T = splatg(0.f);
    for (int ip = 0; ip < n; ++ip) {
      const uint2 ins = w.code[ip];
      const uint32_t off = ins_off(ins);
      const float cv = __uint_as_float(ins.y);
      switch (ins_op(ins)) {
        case OP_LDV: T = ldxg(xr, ins.y); break;
        case OP_LDC: T = splatg(cv); break;
        case OP_PUSHV: *slot_at(w, off) = T; T = ldxg(xr, ins.y); break;
        case OP_PUSHC: *slot_at(w, off) = T; T = splatg(cv); break;
        case OP_ADD: { const VG a = *slot_at(w, off); T = addg(a, T); } break;
        case OP_SUB: { const VG a = *slot_at(w, off); T = subg(a, T); } break;
        case OP_RSUB: { const VG b = *slot_at(w, off); T = subg(T, b); } break;
        // the tape keeps only what the reverse sweep will use (INS_SA / INS_TA:
        // which operands' adjoints are wanted; INS_NOADJ: none)
        case OP_MUL: {
          const VG a = *slot_at(w, off);
          if (ins.x & INS_TA) push(a);
          if (ins.x & INS_SA) push(T);
          T = mulg(a, T);
        } break;
        case OP_DIV: {
          const VG a = *slot_at(w, off);
          if (ins.x & (INS_SA | INS_TA)) push(T);
          T = pdivg(a, T);
          if (ins.x & INS_TA) push(T);
        } break;
        case OP_RDIV: {
          const VG b = *slot_at(w, off);
          if (ins.x & (INS_SA | INS_TA)) push(b);
          T = pdivg(T, b);
          if (ins.x & INS_SA) push(T);
        } break;
        // a unary operator with no constant below (INS_NOADJ) tapes nothing;
        // its local derivative is computed all the same: one code path per
        // operator keeps the loop inside the instruction cache
        case OP_SIN: { const VD r = fwd_sin(T); if (!(ins.x & INS_NOADJ)) push(r.d); T = r.v; } break;
        case OP_COS: { const VD r = fwd_cos(T); if (!(ins.x & INS_NOADJ)) push(r.d); T = r.v; } break;
        case OP_EXP: { const VD r = fwd_exp(T); if (!(ins.x & INS_NOADJ)) push(r.d); T = r.v; } break;
        case OP_LOG: { const VD r = fwd_log(T); if (!(ins.x & INS_NOADJ)) push(r.d); T = r.v; } break;
        case OP_SQRT: { const VD r = fwd_sqrt(T); if (!(ins.x & INS_NOADJ)) push(r.d); T = r.v; } break;
        case OP_SQ: if (!(ins.x & INS_NOADJ)) push(addg(T, T)); T = mulg(T, T); break;
        case OP_INV:
        case OP_TAN:
        case OP_ASIN:
        case OP_ACOS:
        case OP_ATAN:
        case OP_TANH: { const VD r = fwd_ext(ins_op(ins), T); if (!(ins.x & INS_NOADJ)) push(r.d); T = r.v; } break;
        case OP_VADD: T = addg(T, ldxg(xr, ins.y)); break;
        case OP_VSUB: T = subg(T, ldxg(xr, ins.y)); break;
        case OP_VRSUB: T = subg(ldxg(xr, ins.y), T); break;
        case OP_VMUL: T = mulg(T, ldxg(xr, ins.y)); break;
        case OP_VDIV: T = pdivg(T, ldxg(xr, ins.y)); break;
        case OP_VRDIV:
          if (ins.x & INS_NOADJ) {
            T = pdivg(ldxg(xr, ins.y), T);
          } else {
            push(T);
            T = pdivg(ldxg(xr, ins.y), T);
            push(T);
          }
          break;
        case OP_CADD: T = addg(T, splatg(cv)); break;
        case OP_CSUB: T = subg(T, splatg(cv)); break;
        case OP_CRSUB: T = subg(splatg(cv), T); break;
        case OP_CMUL: push(T); T = mulg(T, splatg(cv)); break;
        case OP_CDIV: T = pdivg(T, splatg(cv)); push(T); break;
        case OP_CRDIV: push(T); T = pdivg(splatg(cv), T); push(T); break;
        default: break;
      }
    }
    // ---- loss and seed: e = yhat - y on valid cases, 0 elsewhere
    VG e;
    float e2 = 0.0f;
#pragma unroll
    for (int i = 0; i < GCPL; ++i) {
      const bool ok = (okm >> i) & 1u;
      e.v[i] = ok ? T.v[i] - __ldg(p.y + c0 + i) : 0.0f;
      e2 += e.v[i] * e.v[i];
    }
    se.add(e2);
    // ---- reverse
    VG aT = e;
    for (int ip = n - 1; ip >= 0; --ip) {
      uint2 ins = w.code[ip];
      if (ins.x & INS_NOADJ) {
        // a subtree without constants: nothing of it is on the tape and no
        // adjoint flows into it; go on from its first instruction (a
        // variable load, whose reverse restores the outer adjoint)
        const uint32_t o = ins_op(ins);
        ip = (o >= OP_VADD && o <= OP_VRDIV) ? (int)ins_off(ins) : (int)ins.y;
        ins = w.code[ip];
      }
      const uint32_t off = ins_off(ins);
      const float cv = __uint_as_float(ins.y);
      const int k = ins_k(ins);
      switch (ins_op(ins)) {
        case OP_LDV: break;
        case OP_LDC: gacc(w, k, aT, okm); break;
        case OP_PUSHV: aT = *slot_at(w, off); break;
        case OP_PUSHC: gacc(w, k, aT, okm); aT = *slot_at(w, off); break;
        case OP_ADD: *slot_at(w, off) = aT; break;
        case OP_SUB: *slot_at(w, off) = aT; aT = negg(aT); break;
        case OP_RSUB: *slot_at(w, off) = negg(aT); break;
        case OP_MUL: {  // T = a t
          const bool sa = ins.x & INS_SA, ta = ins.x & INS_TA;
          const VG t = sa ? pop() : splatg(0.f);
          const VG a = ta ? pop() : splatg(0.f);
          if (sa) *slot_at(w, off) = mulg(aT, t);
          if (ta) aT = mulg(aT, a);
        } break;
        case OP_DIV: {  // T = a / t: dT/da = 1/t, dT/dt = -T/t
          const bool sa = ins.x & INS_SA, ta = ins.x & INS_TA;
          const VG Tn = ta ? pop() : splatg(0.f);
          const VG t = (sa || ta) ? pop() : splatg(1.f);
          const VG q = qdivg(aT, t);
          if (sa) *slot_at(w, off) = q;
          if (ta) aT = negg(mulg(q, Tn));
        } break;
        case OP_RDIV: {  // T = t / b
          const bool sa = ins.x & INS_SA, ta = ins.x & INS_TA;
          const VG Tn = sa ? pop() : splatg(0.f);
          const VG b = (sa || ta) ? pop() : splatg(1.f);
          const VG q = qdivg(aT, b);
          if (sa) *slot_at(w, off) = negg(mulg(q, Tn));
          if (ta) aT = q;
        } break;
        case OP_SIN:
        case OP_COS:
        case OP_EXP:
        case OP_LOG:
        case OP_SQRT:
        case OP_SQ:
        case OP_INV:
        case OP_TAN:
        case OP_ASIN:
        case OP_ACOS:
        case OP_ATAN:
        case OP_TANH: { const VG d = pop(); aT = mulg(aT, d); } break;
        case OP_VADD:
        case OP_VSUB: break;
        case OP_VRSUB: aT = negg(aT); break;
        case OP_VMUL: aT = mulg(aT, ldxg(xr, ins.y)); break;
        case OP_VDIV: aT = qdivg(aT, ldxg(xr, ins.y)); break;
        case OP_VRDIV: {  // T = v / t
          const VG Tn = pop(), t = pop();
          aT = negg(mulg(qdivg(aT, t), Tn));
        } break;
        case OP_CADD: gacc(w, k, aT, okm); break;
        case OP_CSUB: gacc(w, k, negg(aT), okm); break;
        case OP_CRSUB: gacc(w, k, aT, okm); aT = negg(aT); break;
        case OP_CMUL: {  // T = t c
          const VG t = pop();
          gacc(w, k, mulg(aT, t), okm);
          aT = mulg(aT, splatg(cv));
        } break;
        case OP_CDIV: {  // T = t / c: dT/dt = 1/c, dT/dc = -T/c
          const VG Tn = pop();
          const VG q = qdivg(aT, splatg(cv));
          gacc(w, k, negg(mulg(q, Tn)), okm);
          aT = q;
        } break;
        case OP_CRDIV: {  // T = c / t: dT/dc = 1/t, dT/dt = -T/t
          const VG Tn = pop(), t = pop();
          const VG q = qdivg(aT, t);
          gacc(w, k, q, okm);
          aT = negg(mulg(q, Tn));
        } break;
        default: break;
      }
    }
  }
  double *rec = p.partials + ((size_t)prog * p.nchunks + c) * GSTRIDE;
  const double sv = warp_sum(se.value());
  if (lane == 0) rec[0] = sv;
  __syncwarp();
  for (int k = 0; k < p.K; ++k) {
    const double g = warp_sum((double)w.gs[k * 32 + lane] - (double)w.gc[k * 32 + lane]);
    if (lane == 0) rec[1 + k] = g;
  }
}

// Shared memory of a warp, for the largest Lmax (Lw) and K (Kw) of a launch.
__device__ __forceinline__ GradWarp grad_warp(unsigned char *smem, int warp_bytes, int Lw, int Kw, char *gtape,
                                              bool onchip) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *wb = smem + (size_t)warp * warp_bytes;
  GradWarp w;
  w.slot = reinterpret_cast<char *>(wb) + lane * (GCPL * 4);
  const int slot_bytes = slots_for(Lw) * GSLOT;
  w.gs = reinterpret_cast<float *>(wb + slot_bytes);
  w.gc = w.gs + Kw * 32;
  w.code = reinterpret_cast<uint2 *>(wb + slot_bytes + 2 * Kw * 128);
  w.ts = reinterpret_cast<char *>(wb + grad_fixed_bytes(Lw, Kw)) + lane * (GCPL * 4);
  const int gw = blockIdx.x * GWARPS + warp;
  w.tg = onchip ? nullptr : gtape + (size_t)gw * Lw * GSLOT + lane * (GCPL * 4);
  w.lane = lane;
  return w;
}

template <bool ONCHIP>
__global__ void __launch_bounds__(GWARPS * 32, GCTAS_PER_SM) grad_kernel(GradParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const GradWarp w = grad_warp(smem, p.warp_bytes, p.Lmax, p.K, p.gtape, ONCHIP);
  for (;;) {
    const long long item = next_item(p.queue, p.total_items, p.abort, p.err, lane);
    if (item >= p.total_items) break;
    const int c = (int)(item / (unsigned long long)p.P);
    const int prog = (int)(item % (unsigned long long)p.P);
    grad_item<ONCHIP>(p, c, prog, w, lane);
  }
}

// ---------------------------------------------------------------- many problems, one launch
constexpr int MAX_GBATCH = 64;

struct GradBatch {
  GradParams prob[MAX_GBATCH];    // per problem (queue / tape / abort fields unused)
  long long item_begin[MAX_GBATCH];  // first work item of each problem
  int prog_begin[MAX_GBATCH];     // first program of each problem in the decode launch
  double *mse[MAX_GBATCH];
  double *dconst[MAX_GBATCH];
  int nprob, total_progs;
  long long total_items;
  unsigned long long *queue;
  char *gtape;
  const int32_t *abort;
  unsigned *err;
  int warp_bytes, Lw, Kw;         // shared layout: the largest Lmax and K
};

__device__ __forceinline__ int batch_problem(const long long *begin, int nprob, long long x) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// a warp per program of every problem
__global__ void grad_decode_batched_kernel(const __grid_constant__ GradBatch b) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int warp = threadIdx.x >> 5;
  const int g = blockIdx.x * (blockDim.x >> 5) + warp;
  if (g >= b.total_progs) return;
  int q = 0;
  while (q + 1 < b.nprob && b.prog_begin[q + 1] <= g) ++q;
  decode_warp_one(grad_decode_args(b.prob[q]), g - b.prog_begin[q],
                  dsm + (size_t)warp * decode_warp_bytes(b.Lw));
}

// Work items of every problem from one atomic counter, longest items first
// (problems ordered by cases per item x Lmax); problem q owns items
// [item_begin_q, item_begin_q + P_q nchunks_q), chunk-major inside.
template <bool ONCHIP>
__global__ void __launch_bounds__(GWARPS * 32, GCTAS_PER_SM) grad_batched_kernel(const __grid_constant__ GradBatch b) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const GradWarp w = grad_warp(smem, b.warp_bytes, b.Lw, b.Kw, b.gtape, ONCHIP);
  for (;;) {
    const long long item = next_item(b.queue, b.total_items, b.abort, b.err, lane);
    if (item >= b.total_items) break;
    const int q = batch_problem(b.item_begin, b.nprob, item);
    const GradParams &p = b.prob[q];
    const long long local = item - b.item_begin[q];
    grad_item<ONCHIP>(p, (int)(local / p.P), (int)(local % p.P), w, lane);
  }
}

struct GradFinal {
  const double *partials;
  const int32_t *flags;
  int P, N, K, nchunks;
  double *mse, *dconst;
};

__device__ void finalize_grad_one(const GradFinal &f, int p) {
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

__global__ void grad_finalize_kernel(GradFinal f) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < f.P) finalize_grad_one(f, p);
}

// Adam, FP64 moments, every operation rounded on its own in the written order
__device__ __forceinline__ void adam_one(float *c, const double *__restrict__ g, double *m, double *v, int i,
                                         double lr, double b1, double b2, double eps, double bc1, double bc2) {
  const double gi = g[i];
  if (!isfinite(gi)) return;  // leaves c, m, v unchanged
  const double mi = __dadd_rn(__dmul_rn(b1, m[i]), __dmul_rn(__dsub_rn(1.0, b1), gi));
  const double vi = __dadd_rn(__dmul_rn(b2, v[i]), __dmul_rn(__dmul_rn(__dsub_rn(1.0, b2), gi), gi));
  m[i] = mi;
  v[i] = vi;
  const double mh = __ddiv_rn(mi, bc1), vh = __ddiv_rn(vi, bc2);
  const double step = __ddiv_rn(__dmul_rn(lr, mh), __dadd_rn(__dsqrt_rn(vh), eps));
  c[i] = __double2float_rn(__dsub_rn((double)c[i], step));
}

__global__ void adam_kernel(float *c, const double *__restrict__ g, double *m, double *v, int n,
                            double lr, double b1, double b2, double eps, double bc1, double bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) adam_one(c, g, m, v, i, lr, b1, b2, eps, bc1, bc2);
}

// Adam of many constant tables in one launch: blocks (table, 256 entries)
constexpr int MAX_ABATCH = 64;
struct AdamBatch {
  float *c[MAX_ABATCH];
  const double *g[MAX_ABATCH];
  double *m[MAX_ABATCH];
  double *v[MAX_ABATCH];
  int n[MAX_ABATCH];
  int count;
  double lr, b1, b2, eps, bc1, bc2;
};

__global__ void adam_batched_kernel(const __grid_constant__ AdamBatch a) {
  const int q = blockIdx.x;
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < a.n[q]; i += gridDim.y * blockDim.x)
    adam_one(a.c[q], a.g[q], a.m[q], a.v[q], i, a.lr, a.b1, a.b2, a.eps, a.bc1, a.bc2);
}

// blocks (problem, 256 programs of it), a thread per program
__global__ void grad_finalize_batched_kernel(const __grid_constant__ GradBatch b) {
  const GradParams &q = b.prob[blockIdx.x];
  for (int p = blockIdx.y * blockDim.x + threadIdx.x; p < q.P; p += gridDim.y * blockDim.x) {
    GradFinal f{q.partials, q.flags, q.P, q.N, q.K, q.nchunks, b.mse[blockIdx.x], b.dconst[blockIdx.x]};
    finalize_grad_one(f, p);
  }
}

// ---------------------------------------------------------------- host side
// Launch shape of the gradient kernels for the largest Lmax and K of a
// launch: whether the tape fits a warp's share of shared memory, the bytes
// per warp and per block, and the persistent grid.
struct GradShape {
  bool onchip;
  int warp_bytes, smem, grid;
};

sr_status grad_shape_uncached(sr_ctx *ctx, int Lw, int Kw, bool batched, GradShape *g) {
  int sm_bytes = 0, blk_max = 0, blk_reserved = 0;
  SR_CHECK_CUDA(ctx, cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
  SR_CHECK_CUDA(ctx, cudaDeviceGetAttribute(&blk_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  SR_CHECK_CUDA(ctx, cudaDeviceGetAttribute(&blk_reserved, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device));
  // tape entries in shared memory: what is left of a warp's share when
  // GCTAS_PER_SM blocks fill the SM
  const int fixed = grad_fixed_bytes(Lw, Kw);
  const int budget = (sm_bytes / GCTAS_PER_SM - blk_reserved) / GWARPS;
  g->onchip = fixed + Lw * GSLOT <= budget;  // a whole tape fits a warp's share
  g->warp_bytes = fixed + (g->onchip ? Lw * GSLOT : 0);
  g->smem = GWARPS * g->warp_bytes;
  if (g->smem > blk_max) return fail(ctx, SR_EINVAL, "Lmax %d, K %d too large for the gradient kernel", Lw, Kw);
  const void *kern = batched ? (g->onchip ? reinterpret_cast<const void *>(grad_batched_kernel<true>)
                                          : reinterpret_cast<const void *>(grad_batched_kernel<false>))
                             : (g->onchip ? reinterpret_cast<const void *>(grad_kernel<true>)
                                          : reinterpret_cast<const void *>(grad_kernel<false>));
  sr_status st = allow_dynamic_smem(ctx, kern);  // once per (kernel, device): every shape fits
  if (st != SR_OK) return st;
  int nb = 0;
  SR_CHECK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, GWARPS * 32, g->smem));
  if (nb < 1) return fail(ctx, SR_EINVAL, "Lmax %d, K %d too large for the gradient kernel", Lw, Kw);
  g->grid = nb * ctx->num_sms;
  return SR_OK;
}

// grad_shape_uncached, remembered per (device, Lmax, K, kernel): the batched
// call asks it for every problem of a batch
sr_status grad_shape(sr_ctx *ctx, int Lw, int Kw, bool batched, GradShape *g) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int>, std::pair<GradShape, int>> memo;
  const auto key = std::make_tuple(ctx->device, Lw, Kw, batched ? 1 : 0);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = memo.find(key);
    if (it != memo.end()) {
      *g = it->second.first;
      g->grid = it->second.second * ctx->num_sms;  // blocks per SM x this context's SM count
      return SR_OK;
    }
  }
  sr_status st = grad_shape_uncached(ctx, Lw, Kw, batched, g);
  if (st != SR_OK) return st;
  std::lock_guard<std::mutex> lock(mu);
  memo[key] = std::make_pair(*g, g->grid / ctx->num_sms);
  return SR_OK;
}

// cases per work item: about `items` items of this problem, at least one
// 1,024-case block each
int grad_chunk(int N, double items_wanted, int P) {
  int nch = (int)ceil(items_wanted / (P > 0 ? P : 1));
  const int max_chunks = (N + 1023) / 1024;
  nch = nch < 1 ? 1 : (nch > max_chunks ? max_chunks : nch);
  int chunk = (N + nch - 1) / nch;
  return (chunk + GSTEP - 1) / GSTEP * GSTEP;
}

sr_status check_grad(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths, const float *consts, int P,
                     int Lmax, int K, const float *X, const float *y, int nvars, int N, int ldx, const double *mse,
                     const double *dconst) {
  if (P < 0 || Lmax < 1 || Lmax > SR_MAX_LMAX || K < 1 || K > SR_MAX_CONSTS || nvars < 1 ||
      nvars > SR_MAX_VARS || N < 1 || ldx < N || ldx % 4 || (long long)ldx * nvars > 0xFFFFFFFFll)
    return fail(ctx, SR_EINVAL, "bad sr_eval_grad shape");
  if (P == 0) return SR_OK;
  if (!programs || !lengths || !consts || !X || !y || !mse || !dconst)
    return fail(ctx, SR_EINVAL, "NULL pointer");
  if (((uintptr_t)X) & 15) return fail(ctx, SR_EINVAL, "X must be 16-byte aligned");
  return SR_OK;
}

}  // namespace
}  // namespace sr

extern "C" {

sr_status sr_eval_grad(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths,
                       const float *consts, int P, int Lmax, int K, const float *X, const float *y,
                       int nvars, int N, int ldx, double *mse, double *dconst, int32_t *prog_flags) {
  using namespace sr;
  if (!ctx) return SR_EINVAL;
  sr_status st = check_grad(ctx, programs, lengths, consts, P, Lmax, K, X, y, nvars, N, ldx, mse, dconst);
  if (st != SR_OK || P == 0) return st;
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  GradShape gs;
  st = grad_shape(ctx, Lmax, K, false, &gs);
  if (st != SR_OK) return st;
  const long long warps = (long long)gs.grid * GWARPS;
  const int chunk = grad_chunk(N, (double)warps * GTARGET_ITEMS_PER_WARP, P);
  const int nchunks = (N + chunk - 1) / chunk;
  const long long items = (long long)P * nchunks;
  const size_t tokens = (size_t)P * Lmax;
  Carver cv;
  const size_t off_q = cv.take(256), off_f = cv.take((size_t)P * 4), off_nc = cv.take((size_t)P * 4),
               off_code = cv.take(tokens * 8),
               off_p = cv.take((size_t)items * GSTRIDE * 8),
               off_t = cv.take(gs.onchip ? 0 : (size_t)warps * Lmax * GSLOT);
  st = ensure_workspace(ctx, cv.off);
  if (st != SR_OK) return st;
  char *ws = ctx->ws;
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
  gp.partials = reinterpret_cast<double *>(ws + off_p);
  gp.flags = prog_flags ? prog_flags : reinterpret_cast<int32_t *>(ws + off_f);
  gp.code = reinterpret_cast<uint2 *>(ws + off_code);
  gp.ncode = reinterpret_cast<int32_t *>(ws + off_nc);
  gp.queue = reinterpret_cast<unsigned long long *>(ws + off_q);
  gp.gtape = gs.onchip ? nullptr : ws + off_t;
  gp.abort = ctx->abort_flag;
  gp.err = ctx->dev_words;
  gp.warp_bytes = gs.warp_bytes;
  cudaStream_t s = ctx->stream;
  SR_CHECK_CUDA(ctx, cudaMemsetAsync(gp.queue, 0, 8, s));
  st = allow_dynamic_smem(ctx, reinterpret_cast<const void *>(grad_decode_kernel));
  if (st != SR_OK) return st;
  grad_decode_kernel<<<(P + DECODE_WARPS - 1) / DECODE_WARPS, DECODE_WARPS * 32,
                       DECODE_WARPS * decode_warp_bytes(Lmax), s>>>(gp);
  if (gs.onchip) grad_kernel<true><<<gs.grid, GWARPS * 32, gs.smem, s>>>(gp);
  else grad_kernel<false><<<gs.grid, GWARPS * 32, gs.smem, s>>>(gp);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  GradFinal gf{gp.partials, gp.flags, P, N, K, nchunks, mse, dconst};
  grad_finalize_kernel<<<(P + 255) / 256, 256, 0, s>>>(gf);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 3;
  return SR_OK;
}

sr_status sr_eval_grad_batched(sr_ctx *ctx, const sr_grad_problem *pr, int nprob) {
  using namespace sr;
  if (!ctx) return SR_EINVAL;
  if (nprob < 0 || (nprob > 0 && !pr)) return fail(ctx, SR_EINVAL, "bad problem list");
  int Lw = 1, Kw = 1;
  for (int i = 0; i < nprob; ++i) {
    const sr_grad_problem &q = pr[i];
    sr_status st = check_grad(ctx, q.programs, q.lengths, q.consts, q.P, q.Lmax, q.K, q.X, q.y, q.nvars, q.N,
                              q.ldx, q.mse, q.dconst);
    if (st != SR_OK) return fail(ctx, st, "problem %d: %s", i, ctx->msg);
    if (q.P == 0) continue;
    Lw = q.Lmax > Lw ? q.Lmax : Lw;
    Kw = q.K > Kw ? q.K : Kw;
  }
  std::vector<int> order;
  for (int i = 0; i < nprob; ++i)
    if (pr[i].P > 0) order.push_back(i);
  if (order.empty()) return SR_OK;
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  GradShape gs;
  sr_status st = grad_shape(ctx, Lw, Kw, true, &gs);
  if (st != SR_OK) return st;
  const long long warps = (long long)gs.grid * GWARPS;
  // cases per item per problem: the chunking sr_eval_grad would choose for
  // the problem alone (so every problem's sums, and its results, are the
  // same bits as its own call's); the batch shares one grid and one tail
  std::vector<int> chunk(nprob, 0), nch(nprob, 0);
  for (int i : order) {
    const sr_grad_problem &q = pr[i];
    GradShape alone;
    st = grad_shape(ctx, q.Lmax, q.K, false, &alone);
    if (st != SR_OK) return st;
    chunk[i] = grad_chunk(q.N, (double)alone.grid * GWARPS * GTARGET_ITEMS_PER_WARP, q.P);
    nch[i] = (q.N + chunk[i] - 1) / chunk[i];
  }
  // longest items first: the launch's tail is made of short items
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)chunk[a] * pr[a].Lmax > (double)chunk[b] * pr[b].Lmax;
  });
  auto group_bytes = [&](size_t g0, size_t g1, GradBatch *b) -> size_t {
    Carver cv;
    const size_t off_q = cv.take(256);
    const size_t off_t = cv.take(gs.onchip ? 0 : (size_t)warps * Lw * GSLOT);
    long long items = 0;
    int progs = 0;
    for (size_t g = g0; g < g1; ++g) {
      const int i = order[g];
      const sr_grad_problem &q = pr[i];
      const size_t off_f = q.prog_flags ? 0 : cv.take((size_t)q.P * 4);
      const size_t off_nc = cv.take((size_t)q.P * 4);
      const size_t off_code = cv.take((size_t)q.P * q.Lmax * 8);
      const size_t off_p = cv.take((size_t)q.P * nch[i] * GSTRIDE * 8);
      if (b) {
        char *ws = ctx->ws;
        GradParams &p = b->prob[g - g0];
        p.programs = q.programs;
        p.lengths = q.lengths;
        p.consts = q.consts;
        p.P = q.P;
        p.Lmax = q.Lmax;
        p.K = q.K;
        p.X = q.X;
        p.y = q.y;
        p.nvars = q.nvars;
        p.N = q.N;
        p.ldx = q.ldx;
        p.chunk = chunk[i];
        p.nchunks = nch[i];
        p.total_items = (long long)q.P * nch[i];
        p.partials = reinterpret_cast<double *>(ws + off_p);
        p.flags = q.prog_flags ? q.prog_flags : reinterpret_cast<int32_t *>(ws + off_f);
        p.code = reinterpret_cast<uint2 *>(ws + off_code);
        p.ncode = reinterpret_cast<int32_t *>(ws + off_nc);
        p.queue = nullptr;
        p.gtape = nullptr;
        p.abort = nullptr;
        p.err = nullptr;
        p.warp_bytes = gs.warp_bytes;
        b->item_begin[g - g0] = items;
        b->prog_begin[g - g0] = progs;
        b->mse[g - g0] = q.mse;
        b->dconst[g - g0] = q.dconst;
      }
      items += (long long)q.P * nch[i];
      progs += q.P;
    }
    if (b) {
      b->nprob = (int)(g1 - g0);
      b->total_progs = progs;
      b->total_items = items;
      b->queue = reinterpret_cast<unsigned long long *>(ctx->ws + off_q);
      b->gtape = gs.onchip ? nullptr : ctx->ws + off_t;
      b->abort = ctx->abort_flag;
      b->err = ctx->dev_words;
      b->warp_bytes = gs.warp_bytes;
      b->Lw = Lw;
      b->Kw = Kw;
    }
    return cv.off;
  };
  size_t need = 0;
  for (size_t g0 = 0; g0 < order.size(); g0 += MAX_GBATCH)
    need = std::max(need, group_bytes(g0, std::min(order.size(), g0 + MAX_GBATCH), nullptr));
  st = ensure_workspace(ctx, need);
  if (st != SR_OK) return st;
  st = allow_dynamic_smem(ctx, reinterpret_cast<const void *>(grad_decode_batched_kernel));
  if (st != SR_OK) return st;
  cudaStream_t s = ctx->stream;
  for (size_t g0 = 0; g0 < order.size(); g0 += MAX_GBATCH) {
    GradBatch b;
    group_bytes(g0, std::min(order.size(), g0 + MAX_GBATCH), &b);
    SR_CHECK_CUDA(ctx, cudaMemsetAsync(b.queue, 0, 8, s));
    grad_decode_batched_kernel<<<(b.total_progs + DECODE_WARPS - 1) / DECODE_WARPS, DECODE_WARPS * 32,
                                 DECODE_WARPS * decode_warp_bytes(Lw), s>>>(b);
    if (gs.onchip) grad_batched_kernel<true><<<gs.grid, GWARPS * 32, gs.smem, s>>>(b);
    else grad_batched_kernel<false><<<gs.grid, GWARPS * 32, gs.smem, s>>>(b);
    int maxP = 1;
    for (int r = 0; r < b.nprob; ++r) maxP = b.prob[r].P > maxP ? b.prob[r].P : maxP;
    grad_finalize_batched_kernel<<<dim3(b.nprob, std::min((maxP + 255) / 256, 65535)), 256, 0, s>>>(b);
    SR_CHECK_CUDA(ctx, cudaGetLastError());
    ctx->launches += 3;
  }
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

sr_status sr_adam_step_batched(sr_ctx *ctx, const sr_adam_table *tables, int ntables, int t,
                               const sr_adam_cfg *cfg) {
  using namespace sr;
  if (!ctx || !cfg) return SR_EINVAL;
  if (ntables < 0 || (ntables > 0 && !tables) || t < 1) return fail(ctx, SR_EINVAL, "bad table list or t < 1");
  for (int i = 0; i < ntables; ++i) {
    const sr_adam_table &q = tables[i];
    if (q.n < 0) return fail(ctx, SR_EINVAL, "table %d: n < 0", i);
    if (q.n > 0 && (!q.consts || !q.grad || !q.m || !q.v)) return fail(ctx, SR_EINVAL, "table %d: NULL pointer", i);
  }
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  double p1 = 1.0, p2 = 1.0;
  for (int s = 0; s < t; ++s) {
    p1 *= cfg->beta1;
    p2 *= cfg->beta2;
  }
  for (int g0 = 0; g0 < ntables; g0 += MAX_ABATCH) {
    AdamBatch a;
    a.count = 0;
    int maxn = 0;
    for (int i = g0; i < ntables && i < g0 + MAX_ABATCH; ++i) {
      const sr_adam_table &q = tables[i];
      if (q.n == 0) continue;
      a.c[a.count] = q.consts;
      a.g[a.count] = q.grad;
      a.m[a.count] = q.m;
      a.v[a.count] = q.v;
      a.n[a.count] = q.n;
      maxn = q.n > maxn ? q.n : maxn;
      ++a.count;
    }
    if (a.count == 0) continue;
    a.lr = cfg->lr;
    a.b1 = cfg->beta1;
    a.b2 = cfg->beta2;
    a.eps = cfg->eps;
    a.bc1 = 1.0 - p1;
    a.bc2 = 1.0 - p2;
    adam_batched_kernel<<<dim3(a.count, std::min((maxn + 255) / 256, 65535)), 256, 0, ctx->stream>>>(a);
    SR_CHECK_CUDA(ctx, cudaGetLastError());
    ctx->launches += 1;
  }
  return SR_OK;
}

}  // extern "C"

// sr_evolve.cu -- selection and variation on the device: Philox4x32-10,
// k-way tournament, subtree crossover, point / subtree / constant mutation
// and random valid programs.  The paper runs selection, births and mutation
// on the CPU and only evaluation on the GPU (Sec. 2.1.2); here the whole
// generation stays resident.  Every child is a pure function of (seed,
// generation, inputs), so a CPU implementation of the same rules (the
// specification in sr.h) reproduces it bit for bit.
#include <math.h>

#include "sr_common.cuh"

namespace sr {
namespace {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3"
// (SC'11): ten rounds of two 32x32 multiplies with a Weyl-sequence key.
struct Word4 {
  uint32_t v[4];
};

__device__ __forceinline__ Word4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u * c0, h0 = __umulhi(0xD2511F53u, c0);
    const uint32_t m1 = 0xCD9E8D57u * c2, h1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
    c0 = n0;
    c1 = m1;
    c2 = n2;
    c3 = m0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  Word4 w;
  w.v[0] = c0;
  w.v[1] = c1;
  w.v[2] = c2;
  w.v[3] = c3;
  return w;
}

struct Rng {
  uint32_t k0, k1, gen;
  const uint64_t *gen_dev;  // when set, the generation is *gen_dev + gen (read on the device)
  __device__ __forceinline__ Word4 draw(uint32_t d, uint32_t indiv, uint32_t purpose) const {
    return philox(d, indiv, purpose, gen, k0, k1);
  }
  __device__ __forceinline__ Rng resolved() const {
    Rng r = *this;
    if (gen_dev) r.gen = (uint32_t)(*gen_dev + (uint64_t)gen);
    r.gen_dev = nullptr;
    return r;
  }
};

inline Rng make_rng(uint64_t seed, uint64_t gen, const uint64_t *gen_dev = nullptr) {
  Rng r;
  r.k0 = (uint32_t)seed;
  r.k1 = (uint32_t)(seed >> 32);
  r.gen = (uint32_t)gen;
  r.gen_dev = gen_dev;
  return r;
}

// [0, n) by multiply-high (Lemire 2019); [0, 1) from the top 24 bits
__device__ __forceinline__ uint32_t below(uint32_t w, uint32_t n) { return __umulhi(w, n); }
__device__ __forceinline__ float unit24(uint32_t w) {
  return __fmul_rn((float)(w >> 8), 5.9604644775390625e-8f);  // 2^-24, exact
}

constexpr uint32_t PU_TOURN_A = 1, PU_TOURN_B = 2, PU_DECIDE = 3, PU_CROSS = 4, PU_POINT = 5,
                   PU_SUBTREE = 6, PU_SUBGEN = 7, PU_CONSTMUT = 8, PU_INIT = 9, PU_INITC = 10,
                   PU_MICRO_SAMPLE = 11, PU_MICRO_A = 12, PU_MICRO_B = 13;

__device__ __forceinline__ int effect(int v) { return cls_effect(tok_class(v)); }

// token with depth d before it and r tokens left (this one included):
// terminal if d <= r-1, unary if 1 <= d <= r, binary if 2 <= d <= r+1
__device__ __forceinline__ int gen_token(int d, int r, int nvars, int K, int nun, uint32_t w0, uint32_t w1) {
  int allowed[3];
  int na = 0;
  if (d <= r - 1) allowed[na++] = 0;
  if (d >= 1 && d <= r) allowed[na++] = 1;
  if (d >= 2 && d <= r + 1) allowed[na++] = 2;
  const int cls = allowed[below(w0, (uint32_t)na)];
  if (cls == 0) {
    const int q = (int)below(w1, (uint32_t)(nvars + K));
    return q < nvars ? TOK_VAR0 + q : TOK_CONST0 + (q - nvars);
  }
  if (cls == 1) return TOK_SIN + (int)below(w1, (uint32_t)nun);
  return TOK_ADD + (int)below(w1, 4u);
}

// first token of the subtree whose root is `end`
__device__ __forceinline__ int subtree_start(const uint8_t *tok, int end) {
  int acc = 0;
  for (int t = end; t >= 0; --t) {
    acc += effect(tok[t]);
    if (acc == 1) return t;
  }
  return 0;
}

// ---------------------------------------------------------------- kernels
__global__ void philox_kernel(const uint32_t *__restrict__ ctr, uint32_t k0, uint32_t k1,
                              uint32_t *__restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Word4 w = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
  for (int j = 0; j < 4; ++j) out[4 * i + j] = w.v[j];
}

// MAXIMISE = 0: the smallest fitness wins, NaN counting as +inf;
// MAXIMISE = 1: the largest score wins, NaN counting as -inf.
template <int MAXIMISE>
__global__ void tournament_kernel(const double *__restrict__ fitness, int P, int k, Rng rng_in,
                                  int32_t *__restrict__ parents) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * P) return;
  const Rng rng = rng_in.resolved();
  const int i = t >> 1, s = t & 1;
  const double INF = __longlong_as_double(0x7ff0000000000000ll);
  int best = -1;
  double bestf = 0.0;
  Word4 w;
  for (int j = 0; j < k; ++j) {
    if ((j & 3) == 0) w = rng.draw((uint32_t)(j >> 2), (uint32_t)i, s ? PU_TOURN_B : PU_TOURN_A);
    const int cand = (int)below(w.v[j & 3], (uint32_t)P);
    double f = fitness[cand];
    if (isnan(f)) f = MAXIMISE ? -INF : INF;
    const bool better = MAXIMISE ? f > bestf : f < bestf;
    if (best < 0 || better || (f == bestf && cand < best)) {
      best = cand;
      bestf = f;
    }
  }
  parents[t] = best;
}

struct VaryParams {
  const uint8_t *prog_in;
  const int32_t *len_in;
  const float *c_in;
  const int32_t *parents;
  uint8_t *prog_out;
  int32_t *len_out;
  float *c_out;
  int P, Lmax, K, nvars;
  sr_var_cfg cfg;
  Rng rng;
  int P_in;  // parents' population size
};

// One warp per child: the warp copies both parents' token rows into shared
// memory with coalesced loads, lane 0 builds the child there (the steps below
// are serial), and the warp writes the child's row back.  A thread per child
// walked the rows in global memory byte by byte: 18 us for 256 children of
// <= 32 tokens, latency-bound.
constexpr int VARY_WARPS = 4;
__host__ __device__ inline int vary_row_bytes(int Lmax) { return (Lmax + 15) & ~15; }
__device__ int vary_child(VaryParams &p, int i, int ia, int ib, const uint8_t *A, int la, const uint8_t *B,
                          int lb, uint8_t *out);

__global__ void vary_kernel(VaryParams p) {
  extern __shared__ __align__(16) uint8_t vsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * VARY_WARPS + warp;
  if (i >= p.P) return;
  // out-of-range parents and lengths are clamped so that no access leaves
  // the buffers (valid inputs are unaffected)
  const int ia = min(max(p.parents[2 * i], 0), p.P_in - 1);
  const int ib = min(max(p.parents[2 * i + 1], 0), p.P_in - 1);
  const int la = min(max(p.len_in[ia], 1), p.Lmax), lb = min(max(p.len_in[ib], 1), p.Lmax);
  const int R = vary_row_bytes(p.Lmax);
  uint8_t *sA = vsm + (size_t)warp * 3 * R, *sB = sA + R, *out = sB + R;
  {
    const uint8_t *gA = p.prog_in + (size_t)ia * p.Lmax, *gB = p.prog_in + (size_t)ib * p.Lmax;
    for (int t = lane; t < la; t += 32) sA[t] = gA[t];
    for (int t = lane; t < lb; t += 32) sB[t] = gB[t];
  }
  __syncwarp();
  int len = 0;
  if (lane == 0) len = vary_child(p, i, ia, ib, sA, la, sB, lb, out);
  len = __shfl_sync(FULL, len, 0);
  __syncwarp();
  uint8_t *g_out = p.prog_out + (size_t)i * p.Lmax;
  for (int t = lane; t < p.Lmax; t += 32) g_out[t] = t < len ? out[t] : 0;
}

// Builds child i from parents A (row ia, la tokens) and B (row ib) into out
// (shared memory, Lmax bytes); writes its length and constants and returns
// the length.
__device__ int vary_child(VaryParams &p, int i, int ia, int ib, const uint8_t *A, int la, const uint8_t *B,
                          int lb, uint8_t *out) {
  p.rng = p.rng.resolved();
  float c[TOK_NSLOTS];
  for (int k = 0; k < p.K; ++k) c[k] = p.c_in[(size_t)ia * p.K + k];

  const Word4 dw = p.rng.draw(0, (uint32_t)i, PU_DECIDE);
  const float u_cross = unit24(dw.v[0]), u_point = unit24(dw.v[1]);
  const float u_sub = unit24(dw.v[2]), u_const = unit24(dw.v[3]);

  int len = la;
  bool crossed = false;
  if (u_cross < p.cfg.p_cross) {
    const Word4 w = p.rng.draw(0, (uint32_t)i, PU_CROSS);
    const int a = (int)below(w.v[0], (uint32_t)la);
    const int b = (int)below(w.v[1], (uint32_t)lb);
    const int sa = subtree_start(A, a), sb = subtree_start(B, b);
    const int nl = la - (a - sa + 1) + (b - sb + 1);
    if (nl <= p.Lmax) {
      int q = 0;
      uint32_t usedA = 0, usedB = 0;
      for (int t = 0; t < sa; ++t) {
        const int v = A[t];
        out[q++] = (uint8_t)v;
        if (tok_class(v) == CLS_CONST) usedA |= 1u << (v - TOK_CONST0);
      }
      for (int t = sb; t <= b; ++t) {
        const int v = B[t];
        out[q++] = (uint8_t)v;
        if (tok_class(v) == CLS_CONST) usedB |= 1u << (v - TOK_CONST0);
      }
      for (int t = a + 1; t < la; ++t) {
        const int v = A[t];
        out[q++] = (uint8_t)v;
        if (tok_class(v) == CLS_CONST) usedA |= 1u << (v - TOK_CONST0);
      }
      for (int k = 0; k < p.K; ++k)
        if (((usedB >> k) & 1u) && !((usedA >> k) & 1u)) c[k] = p.c_in[(size_t)ib * p.K + k];
      len = nl;
      crossed = true;
    }
  }
  if (!crossed)
    for (int t = 0; t < la; ++t) out[t] = A[t];

  if (u_point < p.cfg.p_point) {
    const Word4 w = p.rng.draw(0, (uint32_t)i, PU_POINT);
    const int t = (int)below(w.v[0], (uint32_t)len);
    const int cls = tok_class(out[t]);
    int v;
    if (cls == CLS_BINARY) {
      v = TOK_ADD + (int)below(w.v[1], 4u);
    } else if (cls == CLS_UNARY) {
      v = TOK_SIN + (int)below(w.v[1], (uint32_t)p.cfg.unary_ops);
    } else {
      const int q = (int)below(w.v[1], (uint32_t)(p.nvars + p.K));
      v = q < p.nvars ? TOK_VAR0 + q : TOK_CONST0 + (q - p.nvars);
    }
    out[t] = (uint8_t)v;
  }

  if (u_sub < p.cfg.p_subtree && p.cfg.max_subtree > 0) {
    const Word4 w = p.rng.draw(0, (uint32_t)i, PU_SUBTREE);
    const int t = (int)below(w.v[0], (uint32_t)len);
    const int n = 1 + (int)below(w.v[1], (uint32_t)p.cfg.max_subtree);
    const int s = subtree_start(out, t);
    const int span = t - s + 1;
    const int nl = len - span + n;
    if (nl <= p.Lmax) {
      // move the tail out[t+1, len) to start at s + n
      if (n > span) {
        for (int j = len - 1; j > t; --j) out[j + (n - span)] = out[j];
      } else if (n < span) {
        for (int j = t + 1; j < len; ++j) out[j - (span - n)] = out[j];
      }
      int d = 0;
      for (int q = 0; q < n; ++q) {
        const Word4 g = p.rng.draw((uint32_t)q, (uint32_t)i, PU_SUBGEN);
        const int v = gen_token(d, n - q, p.nvars, p.K, p.cfg.unary_ops, g.v[0], g.v[1]);
        out[s + q] = (uint8_t)v;
        d += effect(v);
      }
      len = nl;
    }
  }

  if (u_const < p.cfg.p_const && p.K > 0) {
    const Word4 w = p.rng.draw(0, (uint32_t)i, PU_CONSTMUT);
    const int k = (int)below(w.v[0], (uint32_t)p.K);
    const float step = __fmul_rn(__fsub_rn(unit24(w.v[1]), 0.5f), p.cfg.const_delta);
    c[k] = __fadd_rn(c[k], step);
  }

  p.len_out[i] = len;
  for (int k = 0; k < p.K; ++k) p.c_out[(size_t)i * p.K + k] = c[k];
  return len;
}

// ---------------------------------------------------------------- microcosm selection
// Beagle's Monte-Carlo population control (Sec. 2.1.6): a sample of S
// individuals stands in for the whole population; its keep-quantile tau
// estimates the fitness threshold of the best fraction keep.  Keys: fitness,
// NaN as +inf (smaller is better).
__device__ __forceinline__ double micro_key(double f) {
  return isnan(f) ? __longlong_as_double(0x7ff0000000000000ll) : f;
}

constexpr int MICRO_MAX_SAMPLE = 1024;
constexpr int MICRO_ROUNDS = 16;  // 4 candidates per Philox draw: at most 64 per parent

// one block of S threads: draw, sort by rank (S <= 1024, O(S^2) compares),
// tau = the sample's value at rank ceil(keep S) - 1
__global__ void microcosm_sample_kernel(const double *__restrict__ fitness, int P, int S, int kq, Rng rng_in,
                                        double *tau) {
  __shared__ double key[MICRO_MAX_SAMPLE];
  __shared__ int idx[MICRO_MAX_SAMPLE];
  const Rng rng = rng_in.resolved();
  const int j = threadIdx.x;
  if (j < S) {
    const Word4 w = rng.draw((uint32_t)(j >> 2), 0u, PU_MICRO_SAMPLE);
    idx[j] = (int)below(w.v[j & 3], (uint32_t)P);
    key[j] = micro_key(fitness[idx[j]]);
  }
  __syncthreads();
  if (j < S) {
    // rank of sample j: smaller keys first, equal keys by sample position
    int r = 0;
    for (int t = 0; t < S; ++t) r += key[t] < key[j] || (key[t] == key[j] && t < j);
    if (r == kq) *tau = key[j];
  }
}

// thread per (child, parent slot): the first of up to 64 uniform candidates
// whose key is at most tau; if none is, the best candidate drawn (ties to
// the smaller index)
__global__ void microcosm_select_kernel(const double *__restrict__ fitness, int P_in, int P_out, Rng rng_in,
                                        const double *tau_p, int32_t *__restrict__ parents) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * P_out) return;
  const Rng rng = rng_in.resolved();
  const int i = t >> 1, s = t & 1;
  const double tau = *tau_p;
  int best = -1;
  double bestk = 0.0;
  for (int r = 0; r < MICRO_ROUNDS; ++r) {
    const Word4 w = rng.draw((uint32_t)r, (uint32_t)i, s ? PU_MICRO_B : PU_MICRO_A);
    for (int q = 0; q < 4; ++q) {
      const int cand = (int)below(w.v[q], (uint32_t)P_in);
      const double k = micro_key(fitness[cand]);
      if (k <= tau) {
        parents[t] = cand;
        return;
      }
      if (best < 0 || k < bestk || (k == bestk && cand < best)) {
        best = cand;
        bestk = k;
      }
    }
  }
  parents[t] = best;
}

__global__ void random_programs_kernel(uint8_t *prog, int32_t *len, float *c, int P, int Lmin,
                                       int Lmax, int K, int nvars, int nun, float cmin, float cmax,
                                       Rng rng) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const Word4 lw = rng.draw(0, (uint32_t)i, PU_INIT);
  const int L = Lmin + (int)below(lw.v[0], (uint32_t)(Lmax - Lmin + 1));
  uint8_t *out = prog + (size_t)i * Lmax;
  int d = 0;
  for (int t = 0; t < L; ++t) {
    const Word4 w = rng.draw((uint32_t)(1 + t), (uint32_t)i, PU_INIT);
    const int v = gen_token(d, L - t, nvars, K, nun, w.v[0], w.v[1]);
    out[t] = (uint8_t)v;
    d += effect(v);
  }
  for (int t = L; t < Lmax; ++t) out[t] = 0;
  len[i] = L;
  const float span = __fsub_rn(cmax, cmin);
  for (int k = 0; k < K; ++k) {
    const Word4 w = rng.draw((uint32_t)k, (uint32_t)i, PU_INITC);
    c[(size_t)i * K + k] = __fadd_rn(cmin, __fmul_rn(unit24(w.v[0]), span));
  }
}

}  // namespace
}  // namespace sr

extern "C" {

sr_status sr_philox4x32_10(sr_ctx *ctx, const uint32_t *ctr, uint32_t key0, uint32_t key1,
                           uint32_t *out, int n) {
  using namespace sr;
  if (!ctx || n < 0 || (n > 0 && (!ctr || !out))) return fail(ctx, SR_EINVAL, "bad philox arguments");
  if (n == 0) return SR_OK;
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  philox_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctr, key0, key1, out, n);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 1;
  return SR_OK;
}

static sr_status select_tournament(sr_ctx *ctx, const double *fitness, int P, int k, uint64_t seed,
                                   uint64_t gen, int32_t *parents, bool maximise) {
  using namespace sr;
  if (!ctx) return SR_EINVAL;
  if (P < 0 || k < 1 || k > 64) return fail(ctx, SR_EINVAL, "P < 0 or k outside [1, 64]");
  if (P == 0) return SR_OK;
  if (!fitness || !parents) return fail(ctx, SR_EINVAL, "NULL fitness or parents");
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  const Rng rng = make_rng(seed, gen, ctx->gen_dev);
  if (maximise)
    tournament_kernel<1><<<(2 * P + 255) / 256, 256, 0, ctx->stream>>>(fitness, P, k, rng, parents);
  else
    tournament_kernel<0><<<(2 * P + 255) / 256, 256, 0, ctx->stream>>>(fitness, P, k, rng, parents);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 1;
  return SR_OK;
}

sr_status sr_select_tournament(sr_ctx *ctx, const double *fitness, int P, int k, uint64_t seed,
                               uint64_t gen, int32_t *parents) {
  return select_tournament(ctx, fitness, P, k, seed, gen, parents, false);
}

sr_status sr_select_tournament_max(sr_ctx *ctx, const double *score, int P, int k, uint64_t seed,
                                   uint64_t gen, int32_t *parents) {
  return select_tournament(ctx, score, P, k, seed, gen, parents, true);
}

sr_status sr_vary(sr_ctx *ctx, const uint8_t *prog_in, const int32_t *len_in, const float *c_in, int P_in,
                  const int32_t *parents, uint8_t *prog_out, int32_t *len_out, float *c_out, int P,
                  int Lmax, int K, int nvars, const sr_var_cfg *cfg, uint64_t seed, uint64_t gen) {
  using namespace sr;
  if (!ctx || !cfg) return SR_EINVAL;
  if (P > 0 && P_in < 1) return fail(ctx, SR_EINVAL, "P_in must be >= 1 when there are children");
  if (P < 0 || Lmax < 1 || Lmax > SR_MAX_LMAX || K < 0 || K > SR_MAX_CONSTS || nvars < 1 ||
      nvars > SR_MAX_VARS || cfg->max_subtree < 0 || cfg->max_subtree > Lmax ||
      (cfg->unary_ops != UNARY_BASE && cfg->unary_ops != UNARY_ALL))
    return fail(ctx, SR_EINVAL, "bad sr_vary shape or configuration");
  if (P == 0) return SR_OK;
  if (!prog_in || !len_in || !parents || !prog_out || !len_out || (K > 0 && (!c_in || !c_out)))
    return fail(ctx, SR_EINVAL, "NULL pointer");
  if (prog_in == prog_out) return fail(ctx, SR_EINVAL, "prog_out must not alias prog_in");
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  VaryParams vp{prog_in, len_in, c_in, parents, prog_out, len_out, c_out, P, Lmax, K, nvars, *cfg,
                make_rng(seed, gen, ctx->gen_dev), P_in};
  vary_kernel<<<(P + VARY_WARPS - 1) / VARY_WARPS, VARY_WARPS * 32, VARY_WARPS * 3 * vary_row_bytes(Lmax),
                ctx->stream>>>(vp);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 1;
  return SR_OK;
}

sr_status sr_select_microcosm(sr_ctx *ctx, const double *fitness, int P_in, int P_out, int sample,
                              double keep, uint64_t seed, uint64_t gen, int32_t *parents, double *threshold) {
  using namespace sr;
  if (!ctx) return SR_EINVAL;
  if (P_in < 0 || P_out < 0 || sample < 1 || sample > MICRO_MAX_SAMPLE || !(keep > 0.0 && keep <= 1.0))
    return fail(ctx, SR_EINVAL, "bad sr_select_microcosm arguments");
  if (P_out == 0) return SR_OK;
  if (P_in == 0) return fail(ctx, SR_EINVAL, "no parents to select from");
  if (!fitness || !parents) return fail(ctx, SR_EINVAL, "NULL fitness or parents");
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  double *tau = threshold;
  if (!tau) {
    sr_status st = ensure_workspace(ctx, 256);
    if (st != SR_OK) return st;
    tau = reinterpret_cast<double *>(ctx->ws);
  }
  int kq = (int)ceil(keep * (double)sample) - 1;
  kq = kq < 0 ? 0 : (kq >= sample ? sample - 1 : kq);
  const Rng rng = make_rng(seed, gen, ctx->gen_dev);
  microcosm_sample_kernel<<<1, (sample + 31) / 32 * 32, 0, ctx->stream>>>(fitness, P_in, sample, kq, rng, tau);
  microcosm_select_kernel<<<(2 * P_out + 255) / 256, 256, 0, ctx->stream>>>(fitness, P_in, P_out, rng, tau,
                                                                             parents);
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 2;
  return SR_OK;
}

sr_status sr_set_generation_source(sr_ctx *ctx, const uint64_t *gen_dev) {
  if (!ctx) return SR_EINVAL;
  ctx->gen_dev = gen_dev;
  return SR_OK;
}

sr_status sr_random_programs(sr_ctx *ctx, uint8_t *prog, int32_t *len, float *c, int P, int Lmin,
                             int Lmax, int K, int nvars, int unary_ops, float cmin, float cmax,
                             uint64_t seed, uint64_t stream) {
  using namespace sr;
  if (!ctx) return SR_EINVAL;
  if (P < 0 || Lmin < 1 || Lmin > Lmax || Lmax > SR_MAX_LMAX || K < 0 || K > SR_MAX_CONSTS ||
      nvars < 1 || nvars > SR_MAX_VARS || (unary_ops != UNARY_BASE && unary_ops != UNARY_ALL))
    return fail(ctx, SR_EINVAL, "bad sr_random_programs shape");
  if (P == 0) return SR_OK;
  if (!prog || !len || (K > 0 && !c)) return fail(ctx, SR_EINVAL, "NULL pointer");
  SR_CHECK_CUDA(ctx, cudaSetDevice(ctx->device));
  random_programs_kernel<<<(P + 127) / 128, 128, 0, ctx->stream>>>(prog, len, c, P, Lmin, Lmax, K,
                                                                    nvars, unary_ops, cmin, cmax,
                                                                    make_rng(seed, stream));
  SR_CHECK_CUDA(ctx, cudaGetLastError());
  ctx->launches += 1;
  return SR_OK;
}

}  // extern "C"

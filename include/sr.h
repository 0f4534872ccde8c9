/*
 * sr.h -- C ABI of libsr: population evaluation for GP symbolic regression
 * on one GB300 (sm_103a).
 *
 * The paper (arXiv 2603.12292, "GPU-Accelerated Genetic Programming for
 * Symbolic Regression with Beagle Framework") sends all genomes of a
 * generation to the GPU together, asks each to run a batch of fitness cases,
 * and returns one aggregate fitness per genome (Sec. 2.1.2).  Genomes are
 * linear programs in Reverse Polish Notation (Sec. 2.1.4).  This library
 * does that for a whole population in one call and keeps selection and
 * variation on the device too.
 *
 * Conventions shared by every entry point
 *   - Pointers marked "device" are device memory of the context's GPU, owned
 *     by the caller (the library never frees them).  "host" marks host memory.
 *   - Every call is asynchronous on the context's stream and returns before
 *     the work finishes; argument errors are reported synchronously.  Results
 *     are valid after the stream is synchronised (sr_sync does that).
 *   - The context owns one device workspace.  It grows (cudaMalloc) when a
 *     call needs more; growth is refused with SR_ENOMEM while the stream is
 *     being captured into a CUDA graph, so reserve first (sr_reserve).
 *   - No entry point calls the host back or synchronises, except sr_sync.
 *
 * Token format (uint8), one byte per program node:
 *     0 ADD  1 SUB  2 MUL  3 DIV (protected)          binary
 *     4 SIN  5 COS  6 EXP (clamped)  7 LOG (protected) 8 SQRT|.|  9 SQ   unary
 *    10 INV (1/x, protected)  11 TAN  12 ASIN  13 ACOS  14 ATAN  15 TANH  unary
 *     16 + j   variable x_j   (j < nvars <= 16)
 *     32 + k   constant c_k   (k < K <= 16)
 *   any other byte is invalid.  A binary op pops b, then a, and pushes a op b
 *   ("x0 x1 -" computes x0 - x1).  Operator readings (the paper lists the
 *   operators but not their domains):
 *     a DIV b   = a / b      if |b| > 1e-3, else 1 (quotient within 2 ulp)
 *     LOG x     = log|x|     if |x| > 1e-3, else 0
 *     SQRT x    = sqrt(|x|)
 *     EXP x     = exp(min(max(x, -80), 80))
 *     SQ x      = x * x
 *     INV x     = 1 DIV x
 *     TAN, ASIN, ACOS, ATAN, TANH as the FP32 math library computes them;
 *     ASIN / ACOS outside [-1, 1] give NaN (a non-real result, Sec. 2.1.5)
 *   Tokens 0-15 are the operator set of Table 1.  NaN operands propagate
 *   through every operator.  Evaluation is FP32.
 *
 * Program layout: programs [P][Lmax] bytes (row p = program p, bytes past
 * lengths[p] are ignored), lengths [P] int32, consts [P][K] float.
 * Case layout: X [nvars][ldx] float (row j holds variable j for every case;
 * ldx >= N, ldx % 4 == 0, X 16-byte aligned), y [N] float (16-byte aligned).
 */
#ifndef SR_H
#define SR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SR_OK = 0,
  SR_EINVAL = 1,   /* bad argument (nothing was launched)                 */
  SR_ECUDA = 2,    /* a CUDA runtime call failed                          */
  SR_ETIMEOUT = 3, /* a bounded device wait gave up (latched error word)  */
  SR_EPROGRAM = 4, /* reserved: invalid programs are flagged, not errors  */
  SR_ENOMEM = 5,   /* workspace growth failed or was refused in capture   */
  SR_EABORTED = 6  /* the abort flag stopped a call (latched error word)  */
} sr_status;

/* Fitness kinds.  SR_MSE: mean((yhat - y)^2).  SR_CORR: 1 - r^2 with r the
 * Pearson correlation of Eq. 1 between y and yhat (the 1 - r^2 objective of
 * Sec. 2.1.5).  SR_MSE_CORR: both from one pass; fitness is then [2][P]
 * (row 0 MSE, row 1 1 - r^2). */
typedef enum { SR_MSE = 0, SR_CORR = 1, SR_MSE_CORR = 2 } sr_fitness_kind;

/* Program flag bits written to prog_flags (0 = valid).  The depth after a
 * token is the running sum of +1 (terminal, valid or not), 0 (unary op or
 * invalid byte) and -1 (binary op). */
#define SR_PF_BAD_LENGTH 1 /* length outside [1, Lmax]; nothing else checked */
#define SR_PF_BAD_TOKEN 2  /* a byte that is no token                      */
#define SR_PF_BAD_VAR 4    /* variable index >= nvars                       */
#define SR_PF_BAD_CONST 8  /* constant index >= K                           */
#define SR_PF_UNDERFLOW 16 /* depth after some token below 1                */
#define SR_PF_BAD_FINAL 32 /* depth after the last token is not 1           */
#define SR_PF_TOO_DEEP 64  /* evaluation would need more than 9 live values;
                              cannot happen for valid programs of up to
                              SR_MAX_LMAX tokens (reported, never evaluated) */

#define SR_MAX_LMAX 512  /* largest supported Lmax                           */
#define SR_MAX_VARS 16
#define SR_MAX_CONSTS 16

typedef struct sr_ctx sr_ctx;

/* Create a context on `device` issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Errors: SR_EINVAL (out NULL, bad device), SR_ECUDA. */
sr_status sr_create(sr_ctx **out, int device, void *cuda_stream);

/* Release the context and its workspace (synchronises its stream first).
 * NULL is accepted. */
sr_status sr_destroy(sr_ctx *ctx);

/* Change the stream later calls are issued on. */
sr_status sr_set_stream(sr_ctx *ctx, void *cuda_stream);

/* Text of a status code (static storage). */
const char *sr_status_string(sr_status s);

/* Text of the last error this context reported (context-owned storage,
 * overwritten by the next failing call). */
const char *sr_last_error(const sr_ctx *ctx);

/* Grow the workspace now so that sr_eval / sr_predict on up to P programs
 * of up to Lmax tokens and up to N cases need no allocation later (for
 * example inside CUDA-graph capture), the variable table of the transforms
 * (sr_set_transforms) included for up to 16 variables.  Synchronous.
 * Errors: SR_EINVAL, SR_ENOMEM. */
sr_status sr_reserve(sr_ctx *ctx, int P, int Lmax, int N);

/* Number of kernels this context has launched so far (host counter,
 * incremented at every launch the library makes; memsets are not counted). */
uint64_t sr_kernel_launches(const sr_ctx *ctx);

/* Wait for all work on the context's stream and report device-side errors
 * latched since the last sr_sync (SR_EABORTED, SR_ETIMEOUT), else SR_OK.
 * The latched word is cleared. */
sr_status sr_sync(sr_ctx *ctx);

/* Host-side cancellation of long calls.  flag: device int32 owned by the
 * caller, or NULL (the default) for none.  While *flag is nonzero, the warps
 * of sr_eval, sr_eval_score, sr_predict, sr_eval_batched and sr_eval_grad
 * take no further work items: a call that sees the flag ends early, its
 * outputs are undefined, and the next sr_sync returns SR_EABORTED.  The flag
 * is read when a warp takes a work item (uncached), never waited on: setting
 * it from another stream or the host while a call runs stops the call within
 * one work item per warp.  Later calls run normally once the flag is zero.
 * Errors: SR_EINVAL (ctx NULL). */
sr_status sr_set_abort_flag(sr_ctx *ctx, const int32_t *flag);

/*
 * sr_eval -- fitness of every program (Sec. 2.1.2 aggregation; Eq. 1 for
 * SR_CORR).
 *   programs  device uint8 [P][Lmax]      program p's tokens in row p
 *   lengths   device int32 [P]            tokens used in each row
 *   consts    device float [P][K]         c_k of program p (K may be 0: NULL)
 *   P         >= 0 programs (0: nothing is launched)
 *   Lmax      1..SR_MAX_LMAX
 *   K         0..SR_MAX_CONSTS
 *   X         device float [nvars][ldx]   16-byte aligned, ldx % 4 == 0
 *   y         device float [N]            16-byte aligned, finite
 *   nvars     1..SR_MAX_VARS;  N >= 1 cases;  ldx >= N
 *   kind      SR_MSE, SR_CORR or SR_MSE_CORR
 *   fitness   device double [P] ([2][P] for SR_MSE_CORR), written
 *   prog_flags device int32 [P] (SR_PF_* bits) or NULL
 * Per program: FP32 evaluation of every case; per-lane FP32 compensated
 * (Kahan) sums, FP64 across lanes, tiles and the final merge.  MSE =
 * sum (yhat - y)^2 / N.  1 - r^2 uses per-tile shifted moments of yhat
 * merged in FP64 (Chan et al.) against y centred in FP64, clamped to [0, 1].
 * An invalid program scores +inf; a non-finite output (or an FP32 sum that
 * overflows) scores +inf for MSE and 1 for 1 - r^2; so does zero output
 * variance for 1 - r^2.
 * Errors: SR_EINVAL (shapes, alignment, NULL pointers), SR_ENOMEM, SR_ECUDA.
 */
sr_status sr_eval(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths,
                  const float *consts, int P, int Lmax, int K, const float *X,
                  const float *y, int nvars, int N, int ldx,
                  sr_fitness_kind kind, double *fitness, int32_t *prog_flags);

/* Beagle's own scores (Sec. 2.1.5); both are maximised.
 *   SR_SCORE_R4  (Eq. 2) score = M r^4 (N - (c1 + c2)) - M (c1 - c2), with r
 *                the Pearson correlation of Eq. 1 over the valid pairs only.
 *   SR_SCORE_P2P (Eq. 3) score = sum over cases of the point-to-point
 *                fitness: M when max(|yhat|, |y|) = 0; otherwise
 *                round(M min(|yhat|,|y|) / max(|yhat|,|y|)), less M/11
 *                inside the round when yhat y < 0; M when both values are
 *                invalid, -M when exactly one is.
 * A value is invalid when it is not finite (NaN, +inf, -inf).  A pair is
 * valid when both yhat and y are; c1 counts the pairs with exactly one
 * invalid value, c2 those with two. */
typedef enum { SR_SCORE_R4 = 0, SR_SCORE_P2P = 1 } sr_score_kind;

/*
 * sr_eval_score -- Beagle's scores of every program (Eq. 2 or Eq. 3).
 *   y            device float [N], 16-byte aligned; may hold NaN / +-inf
 *                (invalid target values)
 *   kind         SR_SCORE_R4 or SR_SCORE_P2P
 *   M            the maximum score per case, 1 <= M <= 2^24
 *   score        device double [P], written (larger is better)
 *   pair_counts  device int32 [P][2] (c1, c2) or NULL
 *   other arguments as for sr_eval.
 * Arithmetic.  Eq. 3 per case in FP32, each operation rounded on its own:
 * q = min / max, v = M q, v = v - M/11 (M/11 rounded to FP32) when the signs
 * differ, rounded to an integer half to even; the integer scores are summed
 * exactly.  Eq. 2: per-lane FP32 compensated sums over the valid pairs of
 * yhat - s (s: a finite output of the tile) and of y - ybar (ybar: the FP64
 * mean of the finite targets), merged in FP64; r^2 is clamped to [0, 1] and
 * is 0 when fewer than two pairs are valid, either variance is zero, or an
 * FP32 moment sum overflows (outputs beyond ~1e18; as for SR_CORR).
 * An invalid program scores -inf with counts (0, 0).
 * Errors: as sr_eval; SR_EINVAL for an unknown kind or M out of range.
 */
sr_status sr_eval_score(sr_ctx *ctx, const uint8_t *programs, const int32_t *lengths,
                        const float *consts, int P, int Lmax, int K, const float *X,
                        const float *y, int nvars, int N, int ldx, sr_score_kind kind,
                        int M, double *score, int32_t *pair_counts, int32_t *prog_flags);

/* One problem of a batch: its own population, data, kind and outputs. */
typedef struct {
  const uint8_t *programs;  /* device [P][Lmax]                          */
  const int32_t *lengths;   /* device [P]                                */
  const float *consts;      /* device [P][K] (NULL when K == 0)          */
  int P, Lmax, K;
  const float *X;           /* device [nvars][ldx], 16-byte aligned      */
  const float *y;           /* device [N], 16-byte aligned               */
  int nvars, N, ldx;
  sr_fitness_kind kind;
  double *fitness;          /* device [P] ([2][P] for SR_MSE_CORR)       */
  int32_t *prog_flags;      /* device [P] or NULL                        */
  int cases_per_tile;       /* cases per work item; 0 = automatic        */
} sr_problem;

/*
 * sr_eval_batched -- sr_eval of many independent problems (different case
 * counts, variable counts, population sizes, lengths and kinds) in one
 * persistent launch: a single atomic work counter hands out (problem, case
 * chunk, program) items, longest items first, to the warps of one grid.
 * Up to 64 problems share a launch (more are split into groups of 64); the
 * problem table travels in the kernel parameters, so the call can be
 * captured in a CUDA graph once the workspace has grown (call it once, or
 * sr_reserve, before capturing).  Results equal those of sr_eval per
 * problem up to the summation order of the case chunks.
 *   problems  host array of nprob entries (copied during the call)
 * Errors: SR_EINVAL (first bad problem is named in sr_last_error),
 * SR_ENOMEM, SR_ECUDA.
 */
sr_status sr_eval_batched(sr_ctx *ctx, const sr_problem *problems, int nprob);

/* Cases per evaluation work item for later sr_eval / sr_predict calls on
 * this context (rounded up to a multiple of 128); 0 restores the automatic
 * choice (about eight items per resident warp).  Set by the autotuner. */
sr_status sr_set_tile(sr_ctx *ctx, int cases_per_tile);

/* CTAs (of 8 warps) per SM of the persistent evaluation kernels, set by the
 * autotuner.  eval_ctas_per_sm: sr_eval / sr_eval_score / sr_predict, 0
 * (automatic: 5 where Lmax <= 200, else 4), 4 or 5 (5 only where it fits,
 * else 4).  batched_ctas_per_sm: sr_eval_batched, 0 (automatic: 4), 3, 4 or
 * 5.  Fewer CTAs give each warp more stack slots in shared memory (fewer
 * programs in the deep pass) and more registers; more CTAs hide more
 * latency.  Results do not depend on it (per-program sums do not depend on
 * which warp runs an item).  Errors: SR_EINVAL. */
sr_status sr_set_occupancy(sr_ctx *ctx, int eval_ctas_per_sm, int batched_ctas_per_sm);

/* Variable transforms of sr_eval / sr_eval_score / sr_predict /
 * sr_eval_batched on this context.  A unary operator applied directly to a
 * variable, u(x_j), is the same column of values in every program of the
 * population: with transforms the decoder turns it into a read of row
 * u(x_j) of a per-call table (X's rows, then u(x_j) for each of the twelve
 * operators and each variable, then -- where the table stays within 2 GiB,
 * and a batch's tables with them within 16 GiB -- the compositions u(v(x_j))
 * of the six base operators), and one kernel
 * fills the rows some program reads, per call, with the FP32 functions the
 * interpreter applies per case: results are bit for bit those without it,
 * while a program's sin(x3), say, costs a load instead of the library
 * routine.  The paper has no counterpart (an evaluation-side
 * common-subexpression elimination, like the folding of constant-only
 * subtrees).
 *   mode  0 never; 1 automatic (the default): calls (and problems of a
 *         batch) of at least 64 programs and 16,384 cases; 2 always
 * The table adds nvars * 13 * N * 4 bytes to the workspace, nvars * 49 * N
 * * 4 with the compositions (sr_reserve counts the largest for up to 16
 * variables); a call whose table does not fit the workspace when it cannot
 * grow (inside stream capture) runs without it.  Errors: SR_EINVAL. */
sr_status sr_set_transforms(sr_ctx *ctx, int mode);

/*
 * sr_predict -- the output yhat of every program on every case (the value
 * left on the stack, Sec. 2.1.4), FP32.
 *   yhat  device float [P][ldy], ldy >= N; row p, column i = program p on
 *         case i.  Rows of invalid programs are filled with NaN.
 *   other arguments as for sr_eval (no y, no kind).
 * Errors: as sr_eval.
 */
sr_status sr_predict(sr_ctx *ctx, const uint8_t *programs,
                     const int32_t *lengths, const float *consts, int P,
                     int Lmax, int K, const float *X, int nvars, int N, int ldx,
                     float *yhat, int ldy, int32_t *prog_flags);

/* ------------------------------------------------------------------------
 * Selection and variation on the device (the paper does selection, births
 * and mutation on the CPU, Sec. 2.1.2, with no crossover; this library keeps
 * the whole generation on the GPU and adds subtree crossover).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 * (seed low 32 bits, seed high 32 bits), counter = (draw, individual,
 * purpose, generation low 32 bits).  A word w maps to [0, n) as
 * floor(w * n / 2^32) (multiply-high, Lemire 2019) and to [0, 1) as
 * (w >> 8) * 2^-24.  Purposes: 1 tournament for parent A, 2 for parent B,
 * 3 variation decisions, 4 crossover points, 5 point mutation, 6 subtree
 * mutation, 7 generated subtree tokens, 8 constant mutation, 9 random
 * program tokens, 10 random program constants.  Every value below is a pure
 * function of (seed, generation, inputs): results are bit-identical to a CPU
 * implementation of the same rules.
 * ---------------------------------------------------------------------- */

/* Philox4x32-10 on n counters: out[i] = Philox(ctr[i], key).  Device
 * arrays of n x 4 words. */
sr_status sr_philox4x32_10(sr_ctx *ctx, const uint32_t *ctr, uint32_t key0,
                           uint32_t key1, uint32_t *out, int n);

/*
 * sr_select_tournament -- k-way tournament with replacement.  Child slot i
 * (0 <= i < P) gets parents[2i] (purpose 1) and parents[2i+1] (purpose 2):
 * candidate j (0 <= j < k) is word j%4 of Philox(j/4, i, purpose, gen)
 * mapped to [0, P); the smallest fitness wins, NaN counting as +inf and
 * equal fitness going to the smaller index.
 *   fitness  device double [P];  parents  device int32 [P][2], written
 *   1 <= k <= 64.   Errors: SR_EINVAL.
 */
sr_status sr_select_tournament(sr_ctx *ctx, const double *fitness, int P, int k,
                               uint64_t seed, uint64_t gen, int32_t *parents);

/* sr_select_tournament_max -- the same draws; the largest score wins (for
 * the scores of sr_eval_score), NaN counting as -inf and equal scores going
 * to the smaller index. */
sr_status sr_select_tournament_max(sr_ctx *ctx, const double *score, int P, int k,
                                   uint64_t seed, uint64_t gen, int32_t *parents);

/*
 * sr_select_microcosm -- Beagle's Monte-Carlo ("microcosm") selection
 * (Sec. 2.1.6): a small random sample of the population stands in for the
 * whole when ranking it.
 *  1. sample: S individuals, sample j = word j%4 of Philox(j/4, 0, 11, gen)
 *     mapped to [0, P_in); sorted by key (fitness, NaN as +inf; equal keys
 *     by sample position); the threshold tau is the key at rank
 *     max(0, ceil(keep S) - 1): an estimate of the fitness that the best
 *     fraction keep of the whole population reaches.
 *  2. one pass over the P_out child slots: parents[2i + s] (s = 0, 1) is the
 *     first of the candidates word q of Philox(r, i, 12 + s, gen) mapped to
 *     [0, P_in), r = 0..15, q = 0..3, whose key is at most tau; when none of
 *     those 64 is, the one with the smallest key (ties to the smaller index).
 * Smaller fitness is better (MSE, 1 - r^2; negate scores first).
 *   fitness    device double [P_in];   parents  device int32 [P_out][2]
 *   sample     1..1024 (the paper samples 100);  keep in (0, 1]
 *   threshold  device double [1] receiving tau, or NULL
 * P_out may differ from P_in: a population schedule grows or shrinks the
 * population between generations (sr_vary takes both sizes).
 * Errors: SR_EINVAL.
 */
sr_status sr_select_microcosm(sr_ctx *ctx, const double *fitness, int P_in, int P_out, int sample,
                              double keep, uint64_t seed, uint64_t gen, int32_t *parents,
                              double *threshold);

/* Variation parameters (probabilities in [0, 1], FP32). */
typedef struct {
  float p_cross;    /* subtree crossover (else the child starts as parent A) */
  float p_point;    /* point mutation: one token -> another of its arity     */
  float p_subtree;  /* subtree mutation: one subtree -> a random program     */
  float p_const;    /* constant mutation: c_k += (u - 1/2) * const_delta     */
  float const_delta;
  int max_subtree;  /* generated subtrees have 1..max_subtree tokens         */
  int unary_ops;    /* unary operators drawn: 6 (tokens 4-9) or 12 (4-15)  */
} sr_var_cfg;

/*
 * sr_vary -- one child per slot i < P from A = parents[2i], B = parents[2i+1],
 * indices into the parent population of P_in programs (P may differ).
 * Decisions: u_cross, u_point, u_sub, u_const = the four words of
 * Philox(0, i, 3, gen) in [0, 1).
 *  1. crossover when u_cross < p_cross: words 0 and 1 of Philox(0, i, 4, gen)
 *     pick node a in [0, lenA) and b in [0, lenB); with [sa, a] and [sb, b]
 *     the subtrees rooted there (the shortest suffix ending at the node
 *     whose stack effect is +1), the child is A[0,sa) ++ B[sb,b] ++ A(a,lenA)
 *     unless that exceeds Lmax (then the child is A).  Constants start as
 *     A's; slot k takes B's value when k is read inside the inserted B
 *     subtree and nowhere in the kept parts of A.  Otherwise child = A.
 *  2. point mutation when u_point < p_point: Philox(0, i, 5, gen): position
 *     [0, len); binary -> [0,4), unary -> 4 + [0,unary_ops), terminal ->
 *     [0, nvars+K)
 *     (variables first, then constants).
 *  3. subtree mutation when u_sub < p_subtree: Philox(0, i, 6, gen): position
 *     t in [0, len), size n = 1 + [0, max_subtree); the subtree rooted at t
 *     becomes a random program of n tokens whose token q uses
 *     Philox(q, i, 7, gen) (word 0 picks the class among those allowed --
 *     terminal if d <= r-1, unary if 1 <= d <= r, binary if 2 <= d <= r+1,
 *     for depth d and r tokens left -- word 1 the token in the class: binary
 *     [0, 4), unary 4 + [0, unary_ops), terminal as for point mutation); skipped
 *     when the result would exceed Lmax.
 *  4. constant mutation when u_const < p_const and K > 0: Philox(0, i, 8,
 *     gen): slot [0, K), u = word 1 in [0, 1);
 *     c = fl32(c + fl32(fl32(u - 0.5) * const_delta)).
 * Children of valid parents are valid.  Bytes past each child's length are
 * zero.  Parent indices outside [0, P_in) and lengths outside [1, Lmax] are
 * clamped into range (never read out of bounds).
 *   prog_in/len_in/c_in  device, the parent population ([P_in][Lmax], [P_in],
 *                        [P_in][K])
 *   parents              device int32 [P][2], each in [0, P)
 *   prog_out/len_out/c_out device, the children (must not alias the inputs)
 * Errors: SR_EINVAL.
 */
sr_status sr_vary(sr_ctx *ctx, const uint8_t *prog_in, const int32_t *len_in,
                  const float *c_in, int P_in, const int32_t *parents, uint8_t *prog_out,
                  int32_t *len_out, float *c_out, int P, int Lmax, int K,
                  int nvars, const sr_var_cfg *cfg, uint64_t seed,
                  uint64_t gen);

/*
 * sr_set_generation_source -- make later sr_select_tournament and sr_vary
 * calls on this context read the generation from device memory: the
 * generation used is *gen_dev + gen (gen = the call's argument), read when
 * the kernel runs.  This lets a captured CUDA graph advance the generation
 * on every replay (increment *gen_dev inside the graph).  NULL restores the
 * argument-only behaviour.  gen_dev: device uint64, caller-owned.
 */
sr_status sr_set_generation_source(sr_ctx *ctx, const uint64_t *gen_dev);

/*
 * sr_random_programs -- a random valid population: program i has length
 * Lmin + [0, Lmax - Lmin] from word 0 of Philox(0, i, 9, stream), token t from
 * Philox(1 + t, i, 9, stream) (same token rule as generated subtrees), and
 * constant k = fl32(cmin + fl32(u * fl32(cmax - cmin))) with u from word 0 of
 * Philox(k, i, 10, stream).  Rows are zero past their length.
 *   prog device uint8 [P][Lmax], len device int32 [P], c device float [P][K]
 *   1 <= Lmin <= Lmax <= SR_MAX_LMAX;  unary_ops 6 or 12 (as in sr_var_cfg).
 * Errors: SR_EINVAL.
 */
sr_status sr_random_programs(sr_ctx *ctx, uint8_t *prog, int32_t *len, float *c,
                             int P, int Lmin, int Lmax, int K, int nvars, int unary_ops,
                             float cmin, float cmax, uint64_t seed,
                             uint64_t stream);

/* ------------------------------------------------------------------------
 * Constant optimisation: reverse-mode derivative of the interpreter and Adam
 * (Kingma & Ba, 2015).  The paper has no gradient step; it is the
 * differentiation pattern applied to the same evaluation.
 * ---------------------------------------------------------------------- */

/*
 * sr_eval_grad -- MSE of every program and its gradient with respect to the
 * program's constants: dconst[p][k] = (2/N) sum_i (yhat_i - y_i) dyhat_i/dc_k.
 * Per (program, case) the forward pass is recomputed into an on-chip tape
 * (one value per token, shared memory) and swept in reverse with an adjoint
 * stack.  Derivative conventions: a protected fallback branch, a clamped exp
 * and sqrt|x| at x = 0 have derivative 0; d log|x|/dx = 1/x; d sqrt|x|/dx =
 * sign(x) / (2 sqrt|x|).  FP32 per case, FP32 compensated sums per lane,
 * FP64 across lanes and case chunks.
 *   arguments as sr_eval; mse device double [P]; dconst device double
 *   [P][K] (K >= 1).  Invalid programs: mse = +inf, dconst = 0.
 * Errors: SR_EINVAL, SR_ENOMEM, SR_ECUDA.
 */
sr_status sr_eval_grad(sr_ctx *ctx, const uint8_t *programs,
                       const int32_t *lengths, const float *consts, int P,
                       int Lmax, int K, const float *X, const float *y,
                       int nvars, int N, int ldx, double *mse, double *dconst,
                       int32_t *prog_flags);

/* One problem of a batched gradient call: its own population, data and
 * outputs (as the arguments of sr_eval_grad). */
typedef struct {
  const uint8_t *programs;  /* device [P][Lmax]                          */
  const int32_t *lengths;   /* device [P]                                */
  const float *consts;      /* device [P][K], K >= 1                     */
  int P, Lmax, K;
  const float *X;           /* device [nvars][ldx], 16-byte aligned      */
  const float *y;           /* device [N]                                */
  int nvars, N, ldx;
  double *mse;              /* device [P], written                       */
  double *dconst;           /* device [P][K], written                    */
  int32_t *prog_flags;      /* device [P] or NULL                        */
} sr_grad_problem;

/*
 * sr_eval_grad_batched -- sr_eval_grad of many independent problems
 * (different populations, constant counts, lengths, variables and case
 * counts) in one persistent launch: one atomic work counter hands out
 * (problem, case chunk, program) items, longest first, to the warps of one
 * grid, so that many small problems keep the whole GPU busy where a loop of
 * sr_eval_grad calls would launch each on its own.  Up to 64 problems share
 * a launch (more are split into groups of 64).  Each problem is cut into
 * the case chunks sr_eval_grad would use for it alone, so its results are
 * bit for bit those of its own sr_eval_grad call on the same context.
 *   problems  host array of nprob entries (read during the call)
 * Errors: SR_EINVAL (the first bad problem is named in sr_last_error),
 * SR_ENOMEM, SR_ECUDA.
 */
sr_status sr_eval_grad_batched(sr_ctx *ctx, const sr_grad_problem *problems, int nprob);

typedef struct {
  double lr;     /* step size (default 1e-2)  */
  double beta1;  /* default 0.9               */
  double beta2;  /* default 0.999             */
  double eps;    /* default 1e-8              */
} sr_adam_cfg;

/*
 * sr_adam_step -- one Adam update of n FP32 constants with FP64 moments, step
 * number t >= 1:  m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g g;
 * c = fl32(c - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)), each FP64
 * operation rounded in that order (b^t as a product of t factors).  A
 * non-finite g leaves c, m, v unchanged.
 *   consts device float [n] (updated), grad device double [n],
 *   m, v device double [n] (updated).   Errors: SR_EINVAL.
 */
sr_status sr_adam_step(sr_ctx *ctx, float *consts, const double *grad,
                       double *m, double *v, int n, int t,
                       const sr_adam_cfg *cfg);

/* One table of constants updated by sr_adam_step_batched (as the arguments
 * of sr_adam_step). */
typedef struct {
  float *consts;        /* device [n], updated */
  const double *grad;   /* device [n]          */
  double *m, *v;        /* device [n], updated */
  int n;
} sr_adam_table;

/* sr_adam_step_batched -- sr_adam_step on many tables with one step number
 * and configuration, in one launch per 64 tables: the constant update of
 * every problem of a batched gradient (sr_eval_grad_batched).  Each table's
 * result is bit for bit that of sr_adam_step on it.  Errors: SR_EINVAL. */
sr_status sr_adam_step_batched(sr_ctx *ctx, const sr_adam_table *tables, int ntables, int t,
                               const sr_adam_cfg *cfg);

/*
 * sr_eval_noalloc -- sr_eval for callers that cannot allocate device memory.
 * (The paper has no counterpart: this exists for embedding.)  Some host
 * programs may not call cudaMalloc once they are running -- a serving process
 * whose device memory is budgeted and carved up at start-up, a plug-in that
 * lives inside another application's CUDA context, or code that must not
 * trigger the device-wide synchronisation an allocation can cause.  This
 * entry point needs no context and allocates nothing: it computes exactly
 * what sr_eval computes, taking all of its scratch from one static device
 * array of 16 MiB that the library reserves in every GPU that loads it, for
 * the life of the process.
 *   cuda_stream  the cudaStream_t to issue on (NULL = legacy default stream);
 *                it must belong to the calling thread's current device
 *   other arguments and results as for sr_eval.
 * The first call on each device looks up the array's device address (once,
 * with that device current); make that first call before capturing a stream
 * into a CUDA graph.  With CUDA's lazy module loading (the default), the
 * library's device code -- and with it the 16 MiB array -- is loaded on a
 * device by the first libsr call there, whichever it is; that load is the
 * one device allocation this entry point can cause, and only on its first
 * call in a process that has made no other libsr call on that device.  A
 * caller that must not allocate at all makes any libsr call on each device
 * during start-up (or sets CUDA_MODULE_LOADING=EAGER).  The scratch is shared
 * by every call on a device and keeps the previous call's contents (each
 * call clears what it needs cleared), so calls whose work overlaps on the
 * GPU race: issue them on one stream, or order them with events.
 * Scratch of one call, in bytes (each term rounded up to 256):
 *     P * 8 * Lmax            decoded instructions
 *   + P * 64 * nchunks        partial sums per program and case chunk
 *   + P * 8                   per-program flags and instruction counts
 *   + 4 * N (rounded up to 256 cases)   centred target (1 - r^2 only)
 *   + 32 * nchunks + 256      target chunk sums, work counters
 * where nchunks (case chunks per program) is chosen as for sr_eval and is
 * lowered, by shrinking the persistent grid, down to 1 when needed; so a
 * problem fits when P * (8 * Lmax + 72) + 4 * N stays somewhat below 16 MiB
 * (for example P = 8,192 programs of Lmax = 128 with N up to 10^6).
 * Errors: SR_EINVAL as for sr_eval; SR_ENOMEM when the scratch does not fit
 * in 16 MiB even with one case chunk per program -- use sr_eval then;
 * SR_ECUDA.
 */
sr_status sr_eval_noalloc(void *cuda_stream, const uint8_t *programs,
                          const int32_t *lengths, const float *consts, int P,
                          int Lmax, int K, const float *X, const float *y,
                          int nvars, int N, int ldx, sr_fitness_kind kind,
                          double *fitness, int32_t *prog_flags);

#ifdef __cplusplus
}
#endif

#endif /* SR_H */

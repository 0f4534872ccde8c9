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
 *     16 + j   variable x_j   (j < nvars <= 16)
 *     32 + k   constant c_k   (k < K <= 16)
 *   any other byte is invalid.  A binary op pops b, then a, and pushes a op b
 *   ("x0 x1 -" computes x0 - x1).  Operator readings (the paper lists the
 *   operators but not their domains):
 *     a DIV b   = a / b      if |b| > 1e-3, else 1
 *     LOG x     = log|x|     if |x| > 1e-3, else 0
 *     SQRT x    = sqrt(|x|)
 *     EXP x     = exp(min(max(x, -80), 80))
 *     SQ x      = x * x
 *   NaN operands propagate through every operator.  Evaluation is FP32.
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
  SR_ENOMEM = 5    /* workspace growth failed or was refused in capture   */
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
 * example inside CUDA-graph capture).  Synchronous.  Errors: SR_EINVAL,
 * SR_ENOMEM. */
sr_status sr_reserve(sr_ctx *ctx, int P, int Lmax, int N);

/* Number of kernels this context has launched so far (host counter,
 * incremented at every launch the library makes; memsets are not counted). */
uint64_t sr_kernel_launches(const sr_ctx *ctx);

/* Wait for all work on the context's stream and report device-side errors
 * latched since the last sr_sync (SR_ETIMEOUT), else SR_OK. */
sr_status sr_sync(sr_ctx *ctx);

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
 * into a CUDA graph.  The scratch is shared by every call on a device and
 * keeps the previous call's contents (each call clears what it needs
 * cleared), so calls whose work overlaps on the GPU race: issue them on one
 * stream, or order them with events.
 * Errors: SR_EINVAL as for sr_eval; SR_ENOMEM when the problem's scratch
 * (partial sums per program and case chunk, the centred target for 1 - r^2,
 * stack slots for deep programs) does not fit in 16 MiB even with the
 * persistent grid shrunk to one SM -- use sr_eval then; SR_ECUDA.
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

/*
 * sr_oracle.c -- plain, slow, FP64 reference for GP symbolic-regression
 * population evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * it is used by tests/, by __graft_entry__.smoke() and by the cpu_baseline leg
 * of bench.py.  It shares no code, header, table or constant with the CUDA
 * library; every encoding value below is written out here on its own from the
 * documented token format.
 *
 * What it computes (paper: "GPU-Accelerated Genetic Programming for Symbolic
 * Regression with Beagle Framework", arXiv 2603.12292):
 *   - Genomes are linear programs in Reverse Polish Notation evaluated with a
 *     value stack (Sec. 2.1.4, "GPU-Friendly Bespoke Language").
 *   - Every genome is evaluated on every fitness case and the per-case
 *     results are aggregated into one fitness per genome (Sec. 2.1.2).
 *   - Correlation fitness: Pearson r of Eq. 1 between the target y and the
 *     program output, scored as 1 - r^2 (Sec. 2.1.5, the "minimising 1 - r^2"
 *     objective the paper attributes to prior work).
 *   - Point-to-point fitness: mean squared error, mean((yhat - y)^2).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - binary op: b = pop, a = pop, push(a op b)   ("x0 x1 -" is x0 - x1)
 *   - protected division: a / b when |b| > 1e-3, else 1
 *   - protected log: log|x| when |x| > 1e-3, else 0
 *   - sqrt|x|, x*x, exp(clamp(x, -80, 80))
 *   - NaN operands flow through every operator (a NaN never selects the
 *     protected fallback value)
 *   - any non-finite output -> MSE = +inf, 1 - r^2 = 1
 *   - zero output variance, zero target variance or N < 2 -> 1 - r^2 = 1
 *   - an invalid program (see or_validate) gets fitness +inf for both kinds
 *
 * Precision: every arithmetic step is FP64; X, y and constants are FP32
 * values widened to FP64 by the caller (or FP64 values passed directly).
 *
 * Random numbers: Philox4x32-10 written from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",
 * SC'11); integer ranges by the 32x32->64 multiply-high map (Lemire 2019).
 * Selection and variation follow the specification in include/sr.h so that
 * the device kernels can be checked bit for bit.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- token encoding (own copy of the documented uint8 format) ---------- */
enum {
  TK_ADD = 0, TK_SUB = 1, TK_MUL = 2, TK_DIV = 3,
  TK_SIN = 4, TK_COS = 5, TK_EXP = 6, TK_LOG = 7, TK_SQRT = 8, TK_SQ = 9
};
#define TK_VAR0 16
#define TK_CONST0 32
#define TK_NSLOTS 16

/* program flag bits */
#define PF_BAD_LENGTH 1
#define PF_BAD_TOKEN 2
#define PF_BAD_VAR 4
#define PF_BAD_CONST 8
#define PF_UNDERFLOW 16
#define PF_BAD_FINAL 32

/* conditioning flag bits */
#define CF_RANGE 1     /* an intermediate outside the FP32 normal range      */
#define CF_BRANCH 2    /* a branch argument close to its switch point        */
#define CF_FITRANGE 4  /* a fitness term whose FP32 partial sums may overflow */

#define PROTECT_EPS 1e-3
#define EXP_CLAMP 80.0

enum { KIND_MSE = 0, KIND_CORR = 1 };

/* ---- token classes ----------------------------------------------------- */
static int is_binary(int t) { return t >= TK_ADD && t <= TK_DIV; }
static int is_unary(int t) { return t >= TK_SIN && t <= TK_SQ; }
static int is_var(int t) { return t >= TK_VAR0 && t < TK_VAR0 + TK_NSLOTS; }
static int is_const(int t) { return t >= TK_CONST0 && t < TK_CONST0 + TK_NSLOTS; }

/*
 * Validate one program.  Returns the flag bits (0 = valid) and the largest
 * stack depth reached.  The stack depth after each token is the running sum
 * of its effect: +1 for a terminal (variable or constant, in range or not),
 * 0 for a unary op and for an unknown token, -1 for a binary op.
 *   PF_BAD_LENGTH  length outside [1, Lmax] (nothing else is checked)
 *   PF_BAD_TOKEN   a byte that is no token
 *   PF_BAD_VAR     a variable index >= nvars
 *   PF_BAD_CONST   a constant index >= K
 *   PF_UNDERFLOW   the depth after some token is below 1
 *   PF_BAD_FINAL   the depth after the last token is not 1
 */
int or_validate(const uint8_t *tok, int len, int Lmax, int nvars, int K,
                int *max_depth_out) {
  int flags = 0, depth = 0, maxd = 0;
  if (len < 1 || len > Lmax) {
    if (max_depth_out) *max_depth_out = 0;
    return PF_BAD_LENGTH;
  }
  for (int t = 0; t < len; ++t) {
    int v = tok[t];
    if (is_binary(v)) {
      depth -= 1;
    } else if (is_unary(v)) {
      /* no change */
    } else if (is_var(v)) {
      if (v - TK_VAR0 >= nvars) flags |= PF_BAD_VAR;
      depth += 1;
    } else if (is_const(v)) {
      if (v - TK_CONST0 >= K) flags |= PF_BAD_CONST;
      depth += 1;
    } else {
      flags |= PF_BAD_TOKEN;
    }
    if (depth < 1) flags |= PF_UNDERFLOW;
    if (depth > maxd) maxd = depth;
  }
  if (depth != 1) flags |= PF_BAD_FINAL;
  if (max_depth_out) *max_depth_out = maxd;
  return flags;
}

/* or_validate over a whole population ([P][Lmax] bytes, lengths [P]). */
void or_validate_all(const uint8_t *programs, const int32_t *lengths, int P,
                     int Lmax, int nvars, int K, int32_t *flags,
                     int32_t *max_depth) {
  for (int p = 0; p < P; ++p) {
    int md = 0;
    flags[p] = or_validate(programs + (size_t)p * Lmax, lengths[p], Lmax, nvars,
                           K, &md);
    if (max_depth) max_depth[p] = md;
  }
}

/* ---- operators ---------------------------------------------------------- */
static double op_div(double a, double b) {
  if (fabs(b) <= PROTECT_EPS) return 1.0;  /* NaN b fails the test: a/b=NaN */
  return a / b;
}
static double op_log(double x) {
  if (fabs(x) <= PROTECT_EPS) return 0.0;
  return log(fabs(x));
}
static double op_exp(double x) {
  if (x > EXP_CLAMP) x = EXP_CLAMP;
  else if (x < -EXP_CLAMP) x = -EXP_CLAMP;
  return exp(x);
}
static double apply_binary(int t, double a, double b) {
  switch (t) {
    case TK_ADD: return a + b;
    case TK_SUB: return a - b;
    case TK_MUL: return a * b;
    default: return op_div(a, b);
  }
}
static double apply_unary(int t, double x) {
  switch (t) {
    case TK_SIN: return sin(x);
    case TK_COS: return cos(x);
    case TK_EXP: return op_exp(x);
    case TK_LOG: return op_log(x);
    case TK_SQRT: return sqrt(fabs(x));
    default: return x * x;
  }
}

/* ---- perturbation sign for the conditioning report --------------------- */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/*
 * Evaluate one valid program on case i.  When eps != 0 every operator
 * output v is replaced by v * (1 +- eps), the sign drawn from a hash of
 * (trial, token, case): a stochastic-arithmetic estimate of how far rounding
 * at relative size eps can move the result (Vignes' CESTAC idea).  When
 * cond != NULL, range and branch-proximity flags are OR-ed into *cond.
 */
static double eval_case(const uint8_t *tok, int len, const double *c,
                        const double *X, long ldx, long i, double *stack,
                        double eps, int trial, int *cond) {
  int sp = 0;
  for (int t = 0; t < len; ++t) {
    int v = tok[t];
    double r;
    if (is_var(v)) {
      stack[sp++] = X[(long)(v - TK_VAR0) * ldx + i];
      continue;
    }
    if (is_const(v)) {
      stack[sp++] = c[v - TK_CONST0];
      continue;
    }
    if (is_binary(v)) {
      double b = stack[--sp];
      double a = stack[sp - 1];
      r = apply_binary(v, a, b);
      if (cond && v == TK_DIV) {
        double m = fabs(b);
        if (fabs(m - PROTECT_EPS) <= 1e-3 * PROTECT_EPS) *cond |= CF_BRANCH;
      }
      if (eps != 0.0) {
        uint64_t h = splitmix64(((uint64_t)trial << 48) ^ ((uint64_t)t << 32) ^
                                (uint64_t)i);
        r *= (h >> 63) ? (1.0 - eps) : (1.0 + eps);
      }
      stack[sp - 1] = r;
    } else {
      double x = stack[sp - 1];
      r = apply_unary(v, x);
      if (cond) {
        if (v == TK_LOG &&
            fabs(fabs(x) - PROTECT_EPS) <= 1e-3 * PROTECT_EPS)
          *cond |= CF_BRANCH;
        if (v == TK_EXP &&
            fabs(fabs(x) - EXP_CLAMP) <= 1e-3 * EXP_CLAMP)
          *cond |= CF_BRANCH;
      }
      if (eps != 0.0) {
        uint64_t h = splitmix64(((uint64_t)trial << 48) ^ ((uint64_t)t << 32) ^
                                (uint64_t)i);
        r *= (h >> 63) ? (1.0 - eps) : (1.0 + eps);
      }
      stack[sp - 1] = r;
    }
    if (cond) {
      double m = fabs(r);
      if (m > FLT_MAX || (m > 0.0 && m < FLT_MIN)) *cond |= CF_RANGE;
    }
  }
  return stack[0];
}

/*
 * Program output yhat[i] for i < N.  X is [nvars][ldx] (column i of row j is
 * variable j on case i).  The program must be valid.
 */
void or_predict(const uint8_t *tok, int len, const double *c, const double *X,
                long ldx, long N, double *yhat) {
  double *stack = (double *)malloc(sizeof(double) * (size_t)(len + 1));
  for (long i = 0; i < N; ++i)
    yhat[i] = eval_case(tok, len, c, X, ldx, i, stack, 0.0, 0, NULL);
  free(stack);
}

/*
 * Per-case rounding sensitivity of one valid program's output: yhat[i] is
 * the plain FP64 value and sens[i] = max over `trials` of |yhat_trial[i] -
 * yhat[i]|, a trial perturbing every operator output by a relative +-eps.
 * *cflags receives CF_RANGE / CF_BRANCH found on the plain evaluation.
 */
void or_predict_sens(const uint8_t *tok, int len, const double *c,
                     const double *X, long ldx, long N, int trials, double eps,
                     double *yhat, double *sens, int *cflags) {
  double *stack = (double *)malloc(sizeof(double) * (size_t)(len + 1));
  int cf = 0;
  for (long i = 0; i < N; ++i) {
    yhat[i] = eval_case(tok, len, c, X, ldx, i, stack, 0.0, 0, &cf);
    double m = fabs(yhat[i]);
    if (m > FLT_MAX || (m > 0.0 && m < FLT_MIN)) cf |= CF_RANGE;
    double w = 0.0;
    for (int tr = 1; tr <= trials; ++tr) {
      double v = eval_case(tok, len, c, X, ldx, i, stack, eps, tr, NULL);
      double d = fabs(v - yhat[i]);
      if (!(d <= w)) w = d; /* NaN differences propagate as NaN */
    }
    sens[i] = w;
  }
  *cflags = cf;
  free(stack);
}

/* ---- fitness ------------------------------------------------------------- */
/* MSE = (1/N) sum (yhat - y)^2; any non-finite output or sum -> +inf. */
double or_mse(const double *yhat, const double *y, long N) {
  double s = 0.0;
  for (long i = 0; i < N; ++i) {
    if (!isfinite(yhat[i])) return INFINITY;
    double e = yhat[i] - y[i];
    s += e * e;
  }
  if (!isfinite(s) || N < 1) return INFINITY;
  return s / (double)N;
}

/*
 * 1 - r^2 with r from Eq. 1, computed two-pass: the means first, then the
 * centred sums.  Degenerate cases score 1 (see the file header).
 */
double or_corr(const double *yhat, const double *y, long N) {
  if (N < 2) return 1.0;
  double my = 0.0, mh = 0.0;
  for (long i = 0; i < N; ++i) {
    if (!isfinite(yhat[i])) return 1.0;
    my += y[i];
    mh += yhat[i];
  }
  my /= (double)N;
  mh /= (double)N;
  double sxy = 0.0, syy = 0.0, shh = 0.0;
  for (long i = 0; i < N; ++i) {
    double dy = y[i] - my, dh = yhat[i] - mh;
    sxy += dy * dh;
    syy += dy * dy;
    shh += dh * dh;
  }
  if (!isfinite(sxy) || !isfinite(syy) || !isfinite(shh)) return 1.0;
  if (syy == 0.0 || shh == 0.0) return 1.0;
  double r = sxy / sqrt(syy * shh);
  return 1.0 - r * r;
}

static double fitness_of(int kind, const double *yhat, const double *y,
                         long N) {
  return kind == KIND_MSE ? or_mse(yhat, y, N) : or_corr(yhat, y, N);
}

static void widen_consts(const float *src, int K, double *dst) {
  for (int k = 0; k < TK_NSLOTS; ++k) dst[k] = k < K ? (double)src[k] : 0.0;
}

static int thread_count(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/*
 * Whole-population evaluation: fitness[p] and flags[p] for every program.
 * programs is [P][Lmax] bytes, lengths [P], consts [P][K] (FP32, widened).
 */
void or_eval(const uint8_t *programs, const int32_t *lengths,
             const float *consts, int P, int Lmax, int K, const double *X,
             long ldx, const double *y, int nvars, long N, int kind,
             double *fitness, int32_t *flags, int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel num_threads(nt)
  {
    double *yhat = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double c[TK_NSLOTS];
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
      const uint8_t *tok = programs + (size_t)p * Lmax;
      int md;
      int f = or_validate(tok, lengths[p], Lmax, nvars, K, &md);
      if (flags) flags[p] = f;
      if (f) {
        fitness[p] = INFINITY;
        continue;
      }
      widen_consts(consts + (size_t)p * K, K, c);
      or_predict(tok, lengths[p], c, X, ldx, N, yhat);
      fitness[p] = fitness_of(kind, yhat, y, N);
    }
    free(yhat);
  }
}

/*
 * Conditioning report for one valid program (FP32 consts widened).
 *   *sens   = max over trials of |f_trial - f_0|, where a trial perturbs
 *             every operator output by a relative +-eps (0 when f_0 is not
 *             finite, or when the program has no operator)
 *   *cflags = CF_RANGE | CF_BRANCH | CF_FITRANGE as found on the unperturbed
 *             evaluation.  CF_FITRANGE: some per-case fitness term exceeds
 *             FLT_MAX / N, so an FP32 partial sum of such terms may overflow
 *             (MSE: (yhat - y)^2; correlation: d^2 and |d * (y - mean y)|
 *             with d = yhat - yhat[0]).
 *   *f0     = the unperturbed fitness
 */
void or_condition_one(const uint8_t *tok, int len, const double *c,
                      const double *X, long ldx, const double *y, long N,
                      int kind, int trials, double eps, double *yhat,
                      double *stack, double *sens, int *cflags, double *f0) {
  int cf = 0;
  for (long i = 0; i < N; ++i)
    yhat[i] = eval_case(tok, len, c, X, ldx, i, stack, 0.0, 0, &cf);
  for (long i = 0; i < N; ++i) {
    double m = fabs(yhat[i]);
    if (m > FLT_MAX || (m > 0.0 && m < FLT_MIN)) cf |= CF_RANGE;
  }
  double base = fitness_of(kind, yhat, y, N);
  /* fitness-term range */
  double lim = (double)FLT_MAX / (double)(N > 0 ? N : 1);
  if (kind == KIND_MSE) {
    for (long i = 0; i < N; ++i) {
      double e = yhat[i] - y[i];
      if (e * e > lim) cf |= CF_FITRANGE;
    }
  } else if (N > 0) {
    double my = 0.0;
    for (long i = 0; i < N; ++i) my += y[i];
    my /= (double)N;
    for (long i = 0; i < N; ++i) {
      double d = yhat[i] - yhat[0];
      if (d * d > lim || fabs(d * (y[i] - my)) > lim) cf |= CF_FITRANGE;
    }
  }
  double worst = 0.0;
  if (isfinite(base)) {
    for (int tr = 1; tr <= trials; ++tr) {
      for (long i = 0; i < N; ++i)
        yhat[i] = eval_case(tok, len, c, X, ldx, i, stack, eps, tr, NULL);
      double f = fitness_of(kind, yhat, y, N);
      double d = isfinite(f) ? fabs(f - base) : INFINITY;
      if (d > worst) worst = d;
    }
  }
  *sens = worst;
  *cflags = cf;
  *f0 = base;
}

void or_condition(const uint8_t *programs, const int32_t *lengths,
                  const float *consts, int P, int Lmax, int K,
                  const double *X, long ldx, const double *y, int nvars,
                  long N, int kind, int trials, double eps, double *sens,
                  int32_t *cflags, double *f0, int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel num_threads(nt)
  {
    double *yhat = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *stack = (double *)malloc(sizeof(double) * (size_t)(Lmax + 1));
    double c[TK_NSLOTS];
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
      const uint8_t *tok = programs + (size_t)p * Lmax;
      int md;
      if (or_validate(tok, lengths[p], Lmax, nvars, K, &md)) {
        sens[p] = 0.0;
        cflags[p] = 0;
        f0[p] = INFINITY;
        continue;
      }
      widen_consts(consts + (size_t)p * K, K, c);
      int cf;
      or_condition_one(tok, lengths[p], c, X, ldx, y, N, kind, trials, eps,
                       yhat, stack, &sens[p], &cf, &f0[p]);
      cflags[p] = cf;
    }
    free(yhat);
    free(stack);
  }
}

/* ---- gradient of MSE with respect to the constants (forward mode) ------ */
/*
 * Forward-mode (tangent) differentiation: every stack entry carries its
 * value and its derivative with respect to each of the K constants.  This is
 * a different method from the device's reverse sweep, on purpose.
 * Derivative conventions: d|x|/dx = sign(x) (0 at 0); a protected fallback
 * branch and a clamped exp have derivative 0; d sqrt|x| / dx = 0 at x = 0.
 * *kink receives the smallest distance, over all cases, of a branch
 * argument to its switch point (|b| - 1e-3 for division, |x| - 1e-3 for
 * log, |x| for sqrt|x|, |x| - 80 for exp).
 */
void or_grad_one(const uint8_t *tok, int len, const double *c, int K,
                 const double *X, long ldx, const double *y, long N,
                 double *mse_out, double *grad, double *kink) {
  double *val = (double *)malloc(sizeof(double) * (size_t)(len + 1));
  double *tan_ = (double *)malloc(sizeof(double) * (size_t)(len + 1) *
                                  (size_t)(K > 0 ? K : 1));
  double s = 0.0, kmin = INFINITY;
  for (int k = 0; k < K; ++k) grad[k] = 0.0;
  int finite = 1;
  for (long i = 0; i < N; ++i) {
    int sp = 0;
    for (int t = 0; t < len; ++t) {
      int v = tok[t];
      if (is_var(v)) {
        val[sp] = X[(long)(v - TK_VAR0) * ldx + i];
        for (int k = 0; k < K; ++k) tan_[sp * K + k] = 0.0;
        ++sp;
      } else if (is_const(v)) {
        val[sp] = c[v - TK_CONST0];
        for (int k = 0; k < K; ++k)
          tan_[sp * K + k] = (k == v - TK_CONST0) ? 1.0 : 0.0;
        ++sp;
      } else if (is_binary(v)) {
        --sp;
        double a = val[sp - 1], b = val[sp];
        double *ta = &tan_[(sp - 1) * K], *tb = &tan_[sp * K];
        double r, da, db;
        switch (v) {
          case TK_ADD: r = a + b; da = 1.0; db = 1.0; break;
          case TK_SUB: r = a - b; da = 1.0; db = -1.0; break;
          case TK_MUL: r = a * b; da = b; db = a; break;
          default: {
            double m = fabs(b);
            if (fabs(m - PROTECT_EPS) < kmin) kmin = fabs(m - PROTECT_EPS);
            if (m <= PROTECT_EPS) {
              r = 1.0; da = 0.0; db = 0.0;
            } else {
              r = a / b; da = 1.0 / b; db = -a / (b * b);
            }
          }
        }
        for (int k = 0; k < K; ++k) ta[k] = da * ta[k] + db * tb[k];
        val[sp - 1] = r;
      } else {
        double x = val[sp - 1];
        double *tx = &tan_[(sp - 1) * K];
        double r, dx;
        switch (v) {
          case TK_SIN: r = sin(x); dx = cos(x); break;
          case TK_COS: r = cos(x); dx = -sin(x); break;
          case TK_EXP:
            if (fabs(fabs(x) - EXP_CLAMP) < kmin) kmin = fabs(fabs(x) - EXP_CLAMP);
            if (x > EXP_CLAMP || x < -EXP_CLAMP) {
              r = op_exp(x); dx = 0.0;
            } else {
              r = exp(x); dx = r;
            }
            break;
          case TK_LOG:
            if (fabs(fabs(x) - PROTECT_EPS) < kmin)
              kmin = fabs(fabs(x) - PROTECT_EPS);
            if (fabs(x) <= PROTECT_EPS) {
              r = 0.0; dx = 0.0;
            } else {
              r = log(fabs(x)); dx = 1.0 / x;
            }
            break;
          case TK_SQRT:
            if (fabs(x) < kmin) kmin = fabs(x);
            r = sqrt(fabs(x));
            dx = (x == 0.0) ? 0.0 : (x > 0.0 ? 0.5 / r : -0.5 / r);
            break;
          default: r = x * x; dx = 2.0 * x; break;
        }
        for (int k = 0; k < K; ++k) tx[k] = dx * tx[k];
        val[sp - 1] = r;
      }
    }
    double yh = val[0];
    if (!isfinite(yh)) finite = 0;
    double e = yh - y[i];
    s += e * e;
    for (int k = 0; k < K; ++k) grad[k] += 2.0 * e * tan_[k];
  }
  for (int k = 0; k < K; ++k) grad[k] /= (double)N;
  *mse_out = (finite && isfinite(s)) ? s / (double)N : INFINITY;
  if (kink) *kink = kmin;
  free(val);
  free(tan_);
}

/* FP64-constant evaluation of MSE for one program (finite differences). */
double or_mse_fp64_consts(const uint8_t *tok, int len, const double *c,
                          const double *X, long ldx, const double *y, long N) {
  double *yhat = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  or_predict(tok, len, c, X, ldx, N, yhat);
  double f = or_mse(yhat, y, N);
  free(yhat);
  return f;
}

void or_grad(const uint8_t *programs, const int32_t *lengths,
             const float *consts, int P, int Lmax, int K, const double *X,
             long ldx, const double *y, int nvars, long N, double *mse,
             double *grad, double *kink, int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (int p = 0; p < P; ++p) {
    const uint8_t *tok = programs + (size_t)p * Lmax;
    int md;
    double c[TK_NSLOTS];
    if (or_validate(tok, lengths[p], Lmax, nvars, K, &md)) {
      mse[p] = INFINITY;
      for (int k = 0; k < K; ++k) grad[(size_t)p * K + k] = 0.0;
      if (kink) kink[p] = 0.0;
      continue;
    }
    widen_consts(consts + (size_t)p * K, K, c);
    or_grad_one(tok, lengths[p], c, K, X, ldx, y, N, &mse[p],
                grad + (size_t)p * K, kink ? &kink[p] : NULL);
  }
}

/* ---- Adam (Kingma & Ba 2015), FP64 update of FP32 constants ------------ */
/*
 * m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 * mhat = m / (1 - b1^t);  vhat = v / (1 - b2^t);
 * c = fl32(c - lr * mhat / (sqrt(vhat) + eps)), every FP64 operation
 * rounded on its own (the file is built with -ffp-contract=off).
 * A non-finite gradient leaves that constant and its moments unchanged.
 */
void or_adam(float *c, const double *g, double *m, double *v, long n, int t,
             double lr, double b1, double b2, double eps) {
  /* b^t as a product of t factors, in order (no pow: its last bit is
   * library-dependent) */
  double p1 = 1.0, p2 = 1.0;
  for (int s = 0; s < t; ++s) {
    p1 *= b1;
    p2 *= b2;
  }
  double bc1 = 1.0 - p1;
  double bc2 = 1.0 - p2;
  for (long i = 0; i < n; ++i) {
    if (!isfinite(g[i])) continue;
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / bc1, vh = v[i] / bc2;
    c[i] = (float)((double)c[i] - lr * mh / (sqrt(vh) + eps));
  }
}

/* ---- Philox4x32-10 ------------------------------------------------------- */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, x0, &hi0, &lo0);
    mulhilo32(M1, x2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ x1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ x3 ^ k1;
    uint32_t n3 = lo0;
    x0 = n0; x1 = n1; x2 = n2; x3 = n3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* counter = (draw, individual, purpose, generation), key = seed halves */
static void draw4(uint64_t seed, uint32_t draw, uint32_t indiv,
                  uint32_t purpose, uint64_t gen, uint32_t out[4]) {
  uint32_t ctr[4] = {draw, indiv, purpose, (uint32_t)gen};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* [0, n) from one 32-bit word: floor(u * n / 2^32) */
static uint32_t below(uint32_t u, uint32_t n) {
  return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}
/* [0, 1) in FP32 from the top 24 bits: (u >> 8) * 2^-24 (exact) */
static float unit24(uint32_t u) { return (float)(u >> 8) * (1.0f / 16777216.0f); }

/* purposes of the counter's third word */
#define PU_TOURN_A 1
#define PU_TOURN_B 2
#define PU_DECIDE 3
#define PU_CROSS 4
#define PU_POINT 5
#define PU_SUBTREE 6
#define PU_SUBGEN 7
#define PU_CONSTMUT 8
#define PU_INIT 9
#define PU_INITC 10

/* ---- tournament selection ---------------------------------------------- */
/*
 * Child slot i draws k candidates per parent with replacement:
 * candidate j uses word j%4 of Philox(counter = (j/4, i, purpose, gen)),
 * mapped to [0, P).  The smallest fitness wins; NaN counts as +inf; equal
 * fitness goes to the smaller index.  Parent A uses purpose 1, B purpose 2.
 */
void or_tournament(const double *fitness, int P, int k, uint64_t seed,
                   uint64_t gen, int32_t *parents) {
  for (int i = 0; i < P; ++i) {
    for (int s = 0; s < 2; ++s) {
      int best = -1;
      double bestf = 0.0;
      uint32_t w[4];
      for (int j = 0; j < k; ++j) {
        if (j % 4 == 0)
          draw4(seed, (uint32_t)(j / 4), (uint32_t)i,
                s == 0 ? PU_TOURN_A : PU_TOURN_B, gen, w);
        int cand = (int)below(w[j % 4], (uint32_t)P);
        double f = fitness[cand];
        if (isnan(f)) f = INFINITY;
        if (best < 0 || f < bestf || (f == bestf && cand < best)) {
          best = cand;
          bestf = f;
        }
      }
      parents[2 * i + s] = best;
    }
  }
}

/* ---- random program generation ------------------------------------------ */
static int token_effect(int v) {
  if (is_binary(v)) return -1;
  if (is_unary(v)) return 0;
  return 1;
}

/*
 * One token of a random valid program: depth d before the token, r tokens
 * left including this one.  Allowed classes, in the order terminal, unary,
 * binary: terminal if d <= r - 1; unary if 1 <= d <= r; binary if
 * 2 <= d <= r + 1.  Word w0 picks the class among the allowed ones, word w1
 * the token inside the class (terminal: [0, nvars + K), variables first).
 */
static int gen_token(int d, int r, int nvars, int K, uint32_t w0, uint32_t w1) {
  int allowed[3], na = 0;
  if (d <= r - 1) allowed[na++] = 0;
  if (d >= 1 && d <= r) allowed[na++] = 1;
  if (d >= 2 && d <= r + 1) allowed[na++] = 2;
  int cls = allowed[below(w0, (uint32_t)na)];
  if (cls == 0) {
    int q = (int)below(w1, (uint32_t)(nvars + K));
    return q < nvars ? TK_VAR0 + q : TK_CONST0 + (q - nvars);
  }
  if (cls == 1) return TK_SIN + (int)below(w1, 6u);
  return TK_ADD + (int)below(w1, 4u);
}

/*
 * Random population: length L = Lmin + [0, Lmax - Lmin] from word 0 of
 * Philox(0, i, 9, stream); token t from Philox(1 + t, i, 9, stream);
 * constant k = fl32(cmin + fl32(u * fl32(cmax - cmin))) with u from word 0
 * of Philox(k, i, 10, stream).  Bytes past L are zero.
 */
void or_random_programs(uint8_t *prog, int32_t *len, float *c, int P,
                        int Lmin, int Lmax, int K, int nvars, float cmin,
                        float cmax, uint64_t seed, uint64_t stream) {
  volatile float span = cmax - cmin;
  for (int i = 0; i < P; ++i) {
    uint32_t w[4];
    draw4(seed, 0, (uint32_t)i, PU_INIT, stream, w);
    int L = Lmin + (int)below(w[0], (uint32_t)(Lmax - Lmin + 1));
    uint8_t *out = prog + (size_t)i * Lmax;
    memset(out, 0, (size_t)Lmax);
    int d = 0;
    for (int t = 0; t < L; ++t) {
      draw4(seed, (uint32_t)(1 + t), (uint32_t)i, PU_INIT, stream, w);
      int v = gen_token(d, L - t, nvars, K, w[0], w[1]);
      out[t] = (uint8_t)v;
      d += token_effect(v);
    }
    len[i] = L;
    for (int k = 0; k < K; ++k) {
      draw4(seed, (uint32_t)k, (uint32_t)i, PU_INITC, stream, w);
      volatile float prod = unit24(w[0]) * span;
      volatile float val = cmin + prod;
      c[(size_t)i * K + k] = val;
    }
  }
}

/* ---- variation ----------------------------------------------------------- */
/* first index of the subtree whose root is token `end` */
static int subtree_start(const uint8_t *tok, int end) {
  int acc = 0;
  for (int t = end; t >= 0; --t) {
    acc += token_effect(tok[t]);
    if (acc == 1) return t;
  }
  return 0; /* unreachable for a valid program */
}

/*
 * One child per slot i from parents A = parents[2i], B = parents[2i+1].
 * Step 0: u_cross, u_point, u_sub, u_const = unit24 of the four words of
 *         Philox(0, i, 3, gen).
 * Step 1 (crossover, u_cross < p_cross): words of Philox(0, i, 4, gen) pick
 *         node a in A ([0, lenA)) and node b in B ([0, lenB)); the subtrees
 *         rooted there are [sa, a] and [sb, b]; the child is
 *         A[0, sa) ++ B[sb, b] ++ A(a, lenA).  If that is longer than Lmax
 *         the child is A.  Constants: the child starts with A's; slot k
 *         takes B's value when k is read inside the inserted B subtree and
 *         nowhere in the kept parts of A.
 *         Otherwise the child is a copy of A.
 * Step 2 (point, u_point < p_point): Philox(0, i, 5, gen): position
 *         [0, len); the token is replaced by one of the same arity
 *         (binary [0,4), unary [0,6), terminal [0, nvars + K)).
 * Step 3 (subtree, u_sub < p_subtree): Philox(0, i, 6, gen): position t in
 *         [0, len) and size n = 1 + [0, max_subtree); the subtree rooted at
 *         t is replaced by a random program of length n whose token q comes
 *         from Philox(q, i, 7, gen) (see gen_token); skipped when the result
 *         would exceed Lmax.
 * Step 4 (constant, u_const < p_const and K > 0): Philox(0, i, 8, gen): slot
 *         k in [0, K), u = unit24(word 1);
 *         c[k] = fl32(c[k] + fl32(fl32(u - 0.5) * delta)).
 */
void or_vary(const uint8_t *prog_in, const int32_t *len_in, const float *c_in,
             const int32_t *parents, uint8_t *prog_out, int32_t *len_out,
             float *c_out, int P, int Lmax, int K, int nvars, float p_cross,
             float p_point, float p_subtree, float p_const, float delta,
             int max_subtree, uint64_t seed, uint64_t gen) {
  uint8_t *buf = (uint8_t *)malloc((size_t)Lmax + (size_t)max_subtree + 8);
  uint8_t *tmp = (uint8_t *)malloc((size_t)Lmax + (size_t)max_subtree + 8);
  for (int i = 0; i < P; ++i) {
    int ia = parents[2 * i], ib = parents[2 * i + 1];
    const uint8_t *A = prog_in + (size_t)ia * Lmax;
    const uint8_t *B = prog_in + (size_t)ib * Lmax;
    int la = len_in[ia], lb = len_in[ib];
    float c[TK_NSLOTS];
    for (int k = 0; k < K; ++k) c[k] = c_in[(size_t)ia * K + k];
    uint32_t dw[4], w[4];
    draw4(seed, 0, (uint32_t)i, PU_DECIDE, gen, dw);
    float u_cross = unit24(dw[0]), u_point = unit24(dw[1]);
    float u_sub = unit24(dw[2]), u_const = unit24(dw[3]);

    int len = la;
    memcpy(buf, A, (size_t)la);
    if (u_cross < p_cross) {
      draw4(seed, 0, (uint32_t)i, PU_CROSS, gen, w);
      int a = (int)below(w[0], (uint32_t)la);
      int b = (int)below(w[1], (uint32_t)lb);
      int sa = subtree_start(A, a), sb = subtree_start(B, b);
      int nl = la - (a - sa + 1) + (b - sb + 1);
      if (nl <= Lmax) {
        int q = 0;
        for (int t = 0; t < sa; ++t) buf[q++] = A[t];
        for (int t = sb; t <= b; ++t) buf[q++] = B[t];
        for (int t = a + 1; t < la; ++t) buf[q++] = A[t];
        len = nl;
        int usedA[TK_NSLOTS] = {0}, usedB[TK_NSLOTS] = {0};
        for (int t = 0; t < la; ++t)
          if ((t < sa || t > a) && is_const(A[t])) usedA[A[t] - TK_CONST0] = 1;
        for (int t = sb; t <= b; ++t)
          if (is_const(B[t])) usedB[B[t] - TK_CONST0] = 1;
        for (int k = 0; k < K; ++k)
          if (usedB[k] && !usedA[k]) c[k] = c_in[(size_t)ib * K + k];
      }
    }
    if (u_point < p_point) {
      draw4(seed, 0, (uint32_t)i, PU_POINT, gen, w);
      int t = (int)below(w[0], (uint32_t)len);
      int v = buf[t];
      if (is_binary(v)) {
        buf[t] = (uint8_t)(TK_ADD + (int)below(w[1], 4u));
      } else if (is_unary(v)) {
        buf[t] = (uint8_t)(TK_SIN + (int)below(w[1], 6u));
      } else {
        int q = (int)below(w[1], (uint32_t)(nvars + K));
        buf[t] = (uint8_t)(q < nvars ? TK_VAR0 + q : TK_CONST0 + (q - nvars));
      }
    }
    if (u_sub < p_subtree && max_subtree > 0) {
      draw4(seed, 0, (uint32_t)i, PU_SUBTREE, gen, w);
      int t = (int)below(w[0], (uint32_t)len);
      int n = 1 + (int)below(w[1], (uint32_t)max_subtree);
      int s = subtree_start(buf, t);
      int nl = len - (t - s + 1) + n;
      if (nl <= Lmax) {
        int q = 0;
        for (int j = 0; j < s; ++j) tmp[q++] = buf[j];
        int d = 0;
        for (int j = 0; j < n; ++j) {
          uint32_t g[4];
          draw4(seed, (uint32_t)j, (uint32_t)i, PU_SUBGEN, gen, g);
          int v = gen_token(d, n - j, nvars, K, g[0], g[1]);
          tmp[q++] = (uint8_t)v;
          d += token_effect(v);
        }
        for (int j = t + 1; j < len; ++j) tmp[q++] = buf[j];
        memcpy(buf, tmp, (size_t)nl);
        len = nl;
      }
    }
    if (u_const < p_const && K > 0) {
      draw4(seed, 0, (uint32_t)i, PU_CONSTMUT, gen, w);
      int k = (int)below(w[0], (uint32_t)K);
      volatile float centred = unit24(w[1]) - 0.5f;
      volatile float step = centred * delta;
      volatile float nc = c[k] + step;
      c[k] = nc;
    }
    uint8_t *out = prog_out + (size_t)i * Lmax;
    memset(out, 0, (size_t)Lmax);
    memcpy(out, buf, (size_t)len);
    len_out[i] = len;
    for (int k = 0; k < K; ++k) c_out[(size_t)i * K + k] = c[k];
  }
  free(buf);
  free(tmp);
}

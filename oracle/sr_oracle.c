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
 * the device kernels can be checked bit for bit.  The paper prints no values
 * for them (Beagle has no crossover and selects by rank on the CPU), so their
 * parity is unpinned by the paper: tests pin them to invariants (validity,
 * whole-subtree swaps, the tournament rank law) and to the specification.
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
  TK_SIN = 4, TK_COS = 5, TK_EXP = 6, TK_LOG = 7, TK_SQRT = 8, TK_SQ = 9,
  /* the rest of the operator set of Table 1 */
  TK_INV = 10, TK_TAN = 11, TK_ASIN = 12, TK_ACOS = 13, TK_ATAN = 14, TK_TANH = 15
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
#define CF_FITRANGE 4  /* a fitness term whose FP32 partial sums may overflow */
#define CF_BRANCH 8    /* FP32 rounding could flip a protected branch, a clamp
                          or the sign inside sqrt|x| (derivative unbounded)  */
#define CF_NONLIN 16   /* first-order error analysis not trusted: the rigorous
                          enclosure is wider than the linear estimate allows  */

#define PROTECT_EPS 1e-3
#define EXP_CLAMP 80.0

enum { KIND_MSE = 0, KIND_CORR = 1 };

/* ---- token classes ----------------------------------------------------- */
static int is_binary(int t) { return t >= TK_ADD && t <= TK_DIV; }
static int is_unary(int t) { return t >= TK_SIN && t <= TK_TANH; }
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
    case TK_SQ: return x * x;
    /* Table 1's other operators: 1/x protected like division; asin and acos
     * outside [-1, 1] are not real (NaN), as the paper's NaN-aware fitness
     * expects (Sec. 2.1.5) */
    case TK_INV: return op_div(1.0, x);
    case TK_TAN: return tan(x);
    case TK_ASIN: return asin(x);
    case TK_ACOS: return acos(x);
    case TK_ATAN: return atan(x);
    default: return tanh(x);
  }
}

/* Evaluate one valid program on case i (value stack, Sec. 2.1.4). */
static double eval_case(const uint8_t *tok, int len, const double *c,
                        const double *X, long ldx, long i, double *stack) {
  int sp = 0;
  for (int t = 0; t < len; ++t) {
    int v = tok[t];
    if (is_var(v)) {
      stack[sp++] = X[(long)(v - TK_VAR0) * ldx + i];
    } else if (is_const(v)) {
      stack[sp++] = c[v - TK_CONST0];
    } else if (is_binary(v)) {
      double b = stack[--sp];
      double a = stack[sp - 1];
      stack[sp - 1] = apply_binary(v, a, b);
    } else {
      stack[sp - 1] = apply_unary(v, stack[sp - 1]);
    }
  }
  return stack[0];
}

/* ---- interval enclosure of the FP32 evaluation ------------------------- */
/*
 * Every FP32 operator output is within a relative u of the exact operator
 * applied to its FP32 operands (u = 2^-22 covers correctly rounded arithmetic
 * and library functions accurate to 2 ulp; tan, asin, acos, atan and tanh
 * are allowed 4u), plus 2^-148 absolute (2 ulp of the subnormal spacing) for
 * subnormal results.  Inputs and constants are exact.  Evaluating the program
 * on intervals -- each operator's exact range over its operand intervals,
 * widened by that rounding -- therefore encloses the FP32 result of every
 * case, whatever the nonlinearity, clamp or protected branch in between.
 */
typedef struct {
  double lo, hi;
} ival;

#define SUBNORMAL_SLACK 2.802596928649634e-45 /* 2^-148: 2 ulp of the subnormal spacing */

static ival iv(double lo, double hi) {
  ival r = {lo, hi};
  return r;
}
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static ival widen(ival a, double u) {
  a.lo -= u * fabs(a.lo) + SUBNORMAL_SLACK;
  a.hi += u * fabs(a.hi) + SUBNORMAL_SLACK;
  return a;
}
static ival hull(ival a, ival b) { return iv(dmin(a.lo, b.lo), dmax(a.hi, b.hi)); }
static ival iv_mul(ival a, ival b) {
  double p1 = a.lo * b.lo, p2 = a.lo * b.hi, p3 = a.hi * b.lo, p4 = a.hi * b.hi;
  return iv(dmin(dmin(p1, p2), dmin(p3, p4)), dmax(dmax(p1, p2), dmax(p3, p4)));
}
/* a / b for b inside [b1, b2] not containing 0 */
static ival iv_quot(ival a, double b1, double b2) {
  double q1 = a.lo / b1, q2 = a.lo / b2, q3 = a.hi / b1, q4 = a.hi / b2;
  return iv(dmin(dmin(q1, q2), dmin(q3, q4)), dmax(dmax(q1, q2), dmax(q3, q4)));
}
/* protected division: 1 where |b| <= 1e-3, a / b elsewhere */
static ival iv_div(ival a, ival b) {
  int have = 0;
  ival r = iv(0.0, 0.0);
  if (b.lo <= PROTECT_EPS && b.hi >= -PROTECT_EPS) {
    r = iv(1.0, 1.0);
    have = 1;
  }
  if (b.lo < -PROTECT_EPS) {
    ival q = iv_quot(a, b.lo, dmin(b.hi, -PROTECT_EPS));
    r = have ? hull(r, q) : q;
    have = 1;
  }
  if (b.hi > PROTECT_EPS) {
    ival q = iv_quot(a, dmax(b.lo, PROTECT_EPS), b.hi);
    r = have ? hull(r, q) : q;
  }
  return r;
}
/* range of sin over [lo, hi] (cos via a shift of pi/2 in the extremum test) */
static ival iv_trig(ival a, int is_cos) {
  const double two_pi = 6.283185307179586, half_pi = 1.5707963267948966;
  if (!(a.hi - a.lo < two_pi)) return iv(-1.0, 1.0);
  double f1 = is_cos ? cos(a.lo) : sin(a.lo), f2 = is_cos ? cos(a.hi) : sin(a.hi);
  ival r = iv(dmin(f1, f2), dmax(f1, f2));
  /* maxima of sin at pi/2 + 2k pi, of cos at 2k pi; minima half a turn on */
  double pmax = is_cos ? 0.0 : half_pi;
  double k = ceil((a.lo - pmax) / two_pi);
  if (pmax + two_pi * k <= a.hi) r.hi = 1.0;
  k = ceil((a.lo - pmax - 3.141592653589793) / two_pi);
  if (pmax + 3.141592653589793 + two_pi * k <= a.hi) r.lo = -1.0;
  /* the extremum tests are done in FP64 near the endpoints: widen a touch */
  r.lo = dmax(-1.0, r.lo - 1e-15);
  r.hi = dmin(1.0, r.hi + 1e-15);
  return r;
}
/* range of |x| over [lo, hi] */
static ival iv_abs(ival a) {
  if (a.lo <= 0.0 && a.hi >= 0.0) return iv(0.0, dmax(-a.lo, a.hi));
  return iv(dmin(fabs(a.lo), fabs(a.hi)), dmax(fabs(a.lo), fabs(a.hi)));
}
static ival iv_unary(int v, ival a) {
  switch (v) {
    case TK_SIN: return iv_trig(a, 0);
    case TK_COS: return iv_trig(a, 1);
    case TK_EXP: return iv(op_exp(a.lo), op_exp(a.hi)); /* monotone, clamped */
    case TK_LOG: {
      ival m = iv_abs(a);
      int have = 0;
      ival r = iv(0.0, 0.0);
      if (m.lo <= PROTECT_EPS) {
        r = iv(0.0, 0.0);
        have = 1;
      }
      if (m.hi > PROTECT_EPS) {
        ival q = iv(log(dmax(m.lo, PROTECT_EPS)), log(m.hi));
        r = have ? hull(r, q) : q;
      }
      return r;
    }
    case TK_SQRT: {
      ival m = iv_abs(a);
      return iv(sqrt(m.lo), sqrt(m.hi));
    }
    case TK_SQ: {
      ival m = iv_abs(a);
      return iv(m.lo * m.lo, m.hi * m.hi);
    }
    case TK_INV: return iv_div(iv(1.0, 1.0), a);
    case TK_TAN: {
      /* increasing between the poles pi/2 + k pi; a pole inside (or within
       * FP64 reach of an end) makes the range unbounded */
      const double pi = 3.141592653589793, half_pi = 1.5707963267948966;
      double k = ceil((a.lo - half_pi) / pi - 1e-12);
      if (!(a.hi - a.lo < pi) || half_pi + k * pi <= a.hi + 1e-12 * (1.0 + fabs(a.hi)))
        return iv(-INFINITY, INFINITY);
      return iv(tan(a.lo), tan(a.hi));
    }
    case TK_ASIN:
    case TK_ACOS: {
      /* outside [-1, 1] the result may be NaN */
      if (!(a.lo >= -1.0 && a.hi <= 1.0)) return iv(NAN, NAN);
      return v == TK_ASIN ? iv(asin(a.lo), asin(a.hi)) : iv(acos(a.hi), acos(a.lo));
    }
    case TK_ATAN: return iv(atan(a.lo), atan(a.hi));
    default: return iv(tanh(a.lo), tanh(a.hi));
  }
}

/*
 * Interval enclosure of the FP32 output of one valid program on case i.
 * Returns the FP64 value; *lo, *hi receive the enclosure.  *cond gets
 * CF_RANGE when an enclosure reaches beyond the FP32 range (FP32 could
 * overflow to inf) or is not a number (FP32 could produce NaN).
 * Work arrays: val [len + 1], box [len + 1].
 */
static double case_interval(const uint8_t *tok, int len, const double *c,
                            const double *X, long ldx, long i, double u,
                            double *val, ival *box, int *cond, double *lo,
                            double *hi) {
  int sp = 0, cf = 0;
  for (int t = 0; t < len; ++t) {
    int v = tok[t];
    if (is_var(v) || is_const(v)) {
      double x = is_var(v) ? X[(long)(v - TK_VAR0) * ldx + i] : c[v - TK_CONST0];
      val[sp] = x;
      box[sp++] = iv(x, x);
      continue;
    }
    ival r;
    if (is_binary(v)) {
      --sp;
      ival a = box[sp - 1], b = box[sp];
      val[sp - 1] = apply_binary(v, val[sp - 1], val[sp]);
      switch (v) {
        case TK_ADD: r = iv(a.lo + b.lo, a.hi + b.hi); break;
        case TK_SUB: r = iv(a.lo - b.hi, a.hi - b.lo); break;
        case TK_MUL: r = iv_mul(a, b); break;
        default: r = iv_div(a, b); break;
      }
    } else {
      val[sp - 1] = apply_unary(v, val[sp - 1]);
      r = iv_unary(v, box[sp - 1]);
    }
    /* tan and the inverse trigonometric / hyperbolic routines get a wider
     * allowance (8 ulp) than the other library functions */
    r = widen(r, (v >= TK_TAN && v <= TK_TANH) ? 4.0 * u : u);
    if (!(r.lo >= -FLT_MAX && r.hi <= FLT_MAX)) cf |= CF_RANGE; /* also NaN */
    box[sp - 1] = r;
  }
  if (cond) *cond |= cf;
  *lo = box[0].lo;
  *hi = box[0].hi;
  return val[0];
}

/*
 * Program output yhat[i] for i < N.  X is [nvars][ldx] (column i of row j is
 * variable j on case i).  The program must be valid.
 */
void or_predict(const uint8_t *tok, int len, const double *c, const double *X,
                long ldx, long N, double *yhat) {
  double *stack = (double *)malloc(sizeof(double) * (size_t)(len + 1));
  for (long i = 0; i < N; ++i)
    yhat[i] = eval_case(tok, len, c, X, ldx, i, stack);
  free(stack);
}

/*
 * FP64 output of one valid program on cases [0, N), the interval [lo, hi]
 * enclosing its FP32 output on every case (see case_interval), and the
 * conditioning flags of every case.
 */
void or_predict_interval(const uint8_t *tok, int len, const double *c,
                         const double *X, long ldx, long N, double u,
                         double *yhat, double *lo, double *hi,
                         int32_t *cflags) {
  double *val = (double *)malloc(sizeof(double) * (size_t)(len + 1));
  ival *box = (ival *)malloc(sizeof(ival) * (size_t)(len + 1));
  for (long i = 0; i < N; ++i) {
    int cf = 0;
    yhat[i] = case_interval(tok, len, c, X, ldx, i, u, val, box, &cf, &lo[i],
                            &hi[i]);
    cflags[i] = cf;
  }
  free(val);
  free(box);
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
 * Conditioning report for one valid program (FP32 constants widened).
 *   *f0     = the fitness (FP64)
 *   *errb   = bound on how far FP32 evaluation can move the fitness, from
 *             the per-case enclosures [lo_i, hi_i] of the output (0 when f0
 *             is not finite; +inf when not finite):
 *             MSE: the exact range of (1/N) sum (v_i - y_i)^2 over
 *                  v_i in [lo_i, hi_i], each term's interval widened by the
 *                  FP32 subtraction, squaring and summation (4u relative);
 *             1 - r^2 (Eq. 1): with b_i = max(hi_i - yhat_i, yhat_i - lo_i),
 *                  xc_i = yhat_i - mean yhat, yc_i = y_i - mean y and
 *                  d_i = yhat_i - yhat_0 (FP32 moments are taken about a
 *                  shift), Sxy moves by at most A = sum |yc_i| b_i +
 *                  8u sum |d_i yc_i| and Sxx by at most B = 2 sum |xc_i| b_i
 *                  + sum b_i^2 + 8u sum d_i^2, so r^2 stays within
 *                  [(|Sxy| - A)_+^2 / ((Sxx + B) Syy),
 *                   (|Sxy| + A)^2 / ((Sxx - B) Syy)], widened by 4u r^2
 *   *cflags = OR of the case flags, plus CF_FITRANGE when some per-case
 *             fitness term exceeds FLT_MAX / N, so an FP32 partial sum of
 *             such terms may overflow (MSE: e_i^2; correlation: d_i^2 and
 *             |d_i yc_i|), or when the correlation's FP32 products d_i^2,
 *             d_i yc_i are so small that their underflow (each term off by
 *             up to 2^-149) could move the sums by 1e-6 of themselves.
 * Work arrays yhat, lo, hi [N], cfl [N].
 */
/* 1 when the FP32 moment products of 1 - r^2 (d^2 and d yc, d = yhat minus
 * a shift) are tiny enough that rounding them into the subnormal range or
 * to 0 (an absolute error of up to 2^-149 each) could move sum d^2 or
 * sum |d yc| by 1e-6 of themselves: then the device's moments, and with
 * them 1 - r^2, are not determined by the outputs. */
static int fp32_terms_underflow(long N, double D2, double DY) {
  const double floor_err = (double)N * 1.401298464324817e-45 * 1e6;
  return D2 < floor_err || DY < floor_err;
}

void or_condition_one(const uint8_t *tok, int len, const double *c,
                      const double *X, long ldx, const double *y, long N,
                      int kind, double u, double *yhat, double *lo, double *hi,
                      int32_t *cfl, double *errb, int *cflags, double *f0) {
  or_predict_interval(tok, len, c, X, ldx, N, u, yhat, lo, hi, cfl);
  int cf = 0;
  for (long i = 0; i < N; ++i) cf |= cfl[i];
  double base = fitness_of(kind, yhat, y, N);
  double lim = (double)FLT_MAX / (double)(N > 0 ? N : 1);
  double err = 0.0;
  if (kind == KIND_MSE) {
    double smin = 0.0, smax = 0.0;
    for (long i = 0; i < N; ++i) {
      double e = yhat[i] - y[i];
      if (e * e > lim) cf |= CF_FITRANGE;
      double elo = lo[i] - y[i], ehi = hi[i] - y[i];
      double qmax = dmax(elo * elo, ehi * ehi);
      double qmin = (elo <= 0.0 && ehi >= 0.0) ? 0.0 : dmin(elo * elo, ehi * ehi);
      smin += qmin * (1.0 - 4.0 * u);
      smax += qmax * (1.0 + 4.0 * u);
    }
    smin /= (double)N;
    smax /= (double)N;
    err = dmax(smax - base, base - smin);
  } else if (N >= 2) {
    double my = 0.0, mh = 0.0;
    for (long i = 0; i < N; ++i) {
      my += y[i];
      mh += yhat[i];
    }
    my /= (double)N;
    mh /= (double)N;
    double sxy = 0.0, syy = 0.0, sxx = 0.0, A = 0.0, B = 0.0, D2 = 0.0, DY = 0.0;
    for (long i = 0; i < N; ++i) {
      double yc = y[i] - my, xc = yhat[i] - mh, d = yhat[i] - yhat[0];
      double b = dmax(hi[i] - yhat[i], yhat[i] - lo[i]);
      if (d * d > lim || fabs(d * yc) > lim) cf |= CF_FITRANGE;
      sxy += yc * xc;
      syy += yc * yc;
      sxx += xc * xc;
      A += fabs(yc) * b;
      B += 2.0 * fabs(xc) * b + b * b;
      D2 += d * d;
      DY += fabs(d * yc);
    }
    A += 8.0 * u * DY;
    B += 8.0 * u * D2;
    if (fp32_terms_underflow(N, D2, DY)) cf |= CF_FITRANGE;
    if (sxx > 0.0 && syy > 0.0) {
      double r2 = sxy * sxy / (sxx * syy);
      double l = fabs(sxy) - A;
      l = l > 0.0 ? l * l / ((sxx + B) * syy) : 0.0;
      double h = sxx - B > 0.0 ? (fabs(sxy) + A) * (fabs(sxy) + A) / ((sxx - B) * syy)
                               : INFINITY;
      err = dmax(h - r2, r2 - l) + 4.0 * u * r2;
    }
  }
  if (!isfinite(base)) err = 0.0;
  else if (!isfinite(err)) err = INFINITY;
  *errb = err;
  *cflags = cf;
  *f0 = base;
}

void or_condition(const uint8_t *programs, const int32_t *lengths,
                  const float *consts, int P, int Lmax, int K,
                  const double *X, long ldx, const double *y, int nvars,
                  long N, int kind, double u, double *errb, int32_t *cflags,
                  double *f0, int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel num_threads(nt)
  {
    size_t nn = (size_t)(N > 0 ? N : 1);
    double *yhat = (double *)malloc(sizeof(double) * nn * 3);
    int32_t *cfl = (int32_t *)malloc(sizeof(int32_t) * nn);
    double c[TK_NSLOTS];
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
      const uint8_t *tok = programs + (size_t)p * Lmax;
      int md;
      if (or_validate(tok, lengths[p], Lmax, nvars, K, &md)) {
        errb[p] = 0.0;
        cflags[p] = 0;
        f0[p] = INFINITY;
        continue;
      }
      widen_consts(consts + (size_t)p * K, K, c);
      int cf;
      or_condition_one(tok, lengths[p], c, X, ldx, y, N, kind, u, yhat,
                       yhat + nn, yhat + 2 * nn, cfl, &errb[p], &cf, &f0[p]);
      cflags[p] = cf;
    }
    free(yhat);
    free(cfl);
  }
}

/* ---- probabilistic first-order rounding-error bound ---------------------- */
/*
 * A second, tighter certificate of "well-conditioned", next to the rigorous
 * interval bound above.  Model (first-order rounding-error analysis): the
 * FP32 evaluation rounds every operator output once, v -> v (1 + d),
 * |d| <= u_v (u_v = u for + - * / and the base library functions, 4u for
 * tan, asin, acos, atan, tanh; inputs and constants are exact FP32 values).
 * Probabilistic rounding-error analysis (N. J. Higham and T. Mary, "A New
 * Approach to Probabilistic Rounding Error Analysis", SIAM J. Sci. Comput.
 * 41(5), 2019) takes the d as independent and mean-zero; a sum sum_k a_k d_k
 * then stays within lam sqrt(sum_k (a_k u_k)^2) except with probability
 * 2 exp(-lam^2 / 2) (Hoeffding's inequality).  Here:
 *   - every node carries, besides its FP64 value v, the first-order variance
 *     scale s2(v) = sum over the operators j below it of (u_j c_j)^2 with
 *     c_j = v_j dv/dv_j, propagated forward: s2 = sum_children
 *     (dv/dchild)^2 s2(child) + (u_v v)^2;
 *   - and a systematic part w(v), taken at its worst: a share BIAS of every
 *     operator's bound (rounding errors of one operator across the cases are
 *     allowed a common bias of BIAS u_j), plus the second-order term of every
 *     nonlinear operator over the lam-sigma neighbourhood of its operands
 *     (|f''| max / 2 times the squared reach, and the product of the reaches
 *     for a product);
 *   - a branch (protected division, 1/x, log, the exp clamp) whose argument
 *     lies within lam sigma + w of its switch point could go either way in
 *     FP32: the case is flagged CF_BRANCH, as is sqrt|x| within that reach
 *     of 0 (unbounded derivative);
 *   - the expansion is not trusted (CF_NONLIN) where an operand's reach
 *     comes within a tenth of a singular point of the operator (0 for a
 *     divisor, log or sqrt, +-1 for asin / acos, a pole of tan) or exceeds
 *     0.1 in the argument of sin, cos, exp, tan or tanh, or where a value's
 *     reach leaves the FP32 range.
 * On a case flagged CF_BRANCH or CF_NONLIN the expansion is not used: that
 * case's output error is taken at its worst, the half-width of its rigorous
 * FP32 enclosure (case_interval), in the systematic part.
 * A fitness F moves by sum_i g_i dyhat_i, g_i = dF/dyhat_i:
 *     MSE:     g_i = (2/N) e_i,  e_i = yhat_i - y_i
 *     1 - r^2: g_i = -(2 Sxy / (Sxx Syy)) (yc_i - (Sxy / Sxx) xc_i)
 * with the centred sums of Eq. 1 (xc = yhat - mean yhat, yc = y - mean y),
 * so errp = min(lam sqrt(sum_i g_i^2 s2_i), sum_i |g_i| w1_i) + sum_i |g_i| w_i
 * (w1: the linear worst case sum_j u_j |c_ij|, which Hoeffding's bound
 * never needs to exceed), plus the FP32 reduction -- each case's terms
 * (e^2; d^2 and d yc with d = yhat - shift) rounded within 2u and
 * independently of the other cases, the compensated running sums within
 * u / 2 of their terms' magnitudes -- and the fitness's own second-order
 * terms.
 */
#define FO_BIAS 0.0625

/* Local partial derivatives of one operator at FP64 operands (a, and b for
 * binary ones) and result r, under the readings of the file header: the
 * protected fallback, a clamped exp and sqrt|x| at 0 have derivative 0. */
static void op_partials(int v, double a, double b, double r, double *pa, double *pb) {
  *pa = 0.0;
  *pb = 0.0;
  switch (v) {
    case TK_ADD: *pa = 1.0; *pb = 1.0; return;
    case TK_SUB: *pa = 1.0; *pb = -1.0; return;
    case TK_MUL: *pa = b; *pb = a; return;
    case TK_DIV:
      if (fabs(b) > PROTECT_EPS) {
        *pa = 1.0 / b;
        *pb = -r / b;
      }
      return;
    case TK_SIN: *pa = cos(a); return;
    case TK_COS: *pa = -sin(a); return;
    case TK_EXP: *pa = (a > EXP_CLAMP || a < -EXP_CLAMP) ? 0.0 : r; return;
    case TK_LOG: *pa = fabs(a) <= PROTECT_EPS ? 0.0 : 1.0 / a; return;
    case TK_SQRT: *pa = a == 0.0 ? 0.0 : (a > 0.0 ? 0.5 / r : -0.5 / r); return;
    case TK_SQ: *pa = 2.0 * a; return;
    case TK_INV: *pa = fabs(a) <= PROTECT_EPS ? 0.0 : -r * r; return;
    case TK_TAN: *pa = 1.0 + r * r; return;
    case TK_ASIN: *pa = 1.0 / sqrt((1.0 - a) * (1.0 + a)); return;
    case TK_ACOS: *pa = -1.0 / sqrt((1.0 - a) * (1.0 + a)); return;
    case TK_ATAN: *pa = 1.0 / (1.0 + a * a); return;
    default: {
      double ch = cosh(a);
      *pa = 1.0 / (ch * ch);
      return;
    }
  }
}

/* |f''| / 2 of a unary operator, bounded over [x - r, x + r], or -1 when the
 * expansion is not trusted there (see CF_NONLIN above). */
static double unary_curvature(int v, double x, double r, double val) {
  double m;
  switch (v) {
    case TK_SIN:
    case TK_COS: return r <= 0.1 ? 0.5 : -1.0;
    case TK_EXP: return r <= 0.1 ? 0.5 * fabs(val) * exp(r) : -1.0;
    case TK_LOG:
      m = fabs(x) - r;
      return m >= 0.9 * fabs(x) && m > 0.0 ? 0.5 / (m * m) : -1.0;
    case TK_SQRT:
      m = fabs(x) - r;
      return m >= 0.9 * fabs(x) && m > 0.0 ? 0.125 / (m * sqrt(m)) : -1.0;
    case TK_SQ: return 1.0;
    case TK_INV:
      m = fabs(x) - r;
      return m >= 0.9 * fabs(x) && m > 0.0 ? 1.0 / (m * m * m) : -1.0;
    case TK_TAN: {
      double cs = fabs(cos(x)) - r;
      if (!(r <= 0.1 && cs >= 0.9 * fabs(cos(x)) && cs > 0.0)) return -1.0;
      double t = (fabs(sin(x)) + r) / cs; /* |tan| over the reach */
      return t * (1.0 + t * t);
    }
    case TK_ASIN:
    case TK_ACOS:
      m = 1.0 - (fabs(x) + r);
      return m >= 0.9 * (1.0 - fabs(x)) && m > 0.0 ? 0.5 * (fabs(x) + r) / (m * sqrt(m * (2.0 - m))) : -1.0;
    case TK_ATAN: return 0.65; /* |2x / (1 + x^2)^2| <= 3 sqrt(3) / 8 */
    default: return r <= 0.1 ? 0.39 : -1.0; /* |sech^2 tanh| <= 4 / (3 sqrt(3)) */
  }
}

/*
 * First-order analysis of one valid program on case i.  Returns the FP64
 * output; *s2, *w receive its variance scale and systematic part; *cond
 * gets CF_RANGE, CF_BRANCH and CF_NONLIN.  Work arrays (len + 1 entries):
 * val, s2v, wv.
 */
/* how far FP32 rounding can move a node, from its three error measures:
 * the random part at lam sigma (never beyond the linear worst case) plus
 * the systematic part */
static double fo_reach(double lam, double s2, double w1, double w) { return dmin(lam * sqrt(s2), w1) + w; }

/*
 * Tangents for the gradient certificate (optional in case_first_order):
 * per stack entry and constant k, t = dv/dc_k in FP64, a its bound with
 * absolute partials, and ea a first-order bound on how far the tangent of
 * an FP32 evaluation can lie from t because the local partials are taken at
 * FP32 values, each within its reach of the FP64 one:
 *     ea(y) = sum_children |p| ea(child) + dp (a(child) + ea(child)),
 * dp the most the partial p can move while its operands move within their
 * reaches (for f(x): max |f''| over the reach times the reach of x, i.e.
 * twice the curvature term of unary_curvature times that reach; for a * b:
 * the other operand's reach; for a / b, with m the least |b| over its
 * reach: d(1/b) <= r_b / m^2 and d(a/b^2) <= r_a / m^2 + 2 (|a| + r_a) r_b /
 * m^3).  The FP32 rounding of the tangent products themselves is not in ea
 * (a relative error of a few u per operator along each path).  Arrays
 * [(len + 1) K]; where a case is flagged CF_BRANCH or CF_NONLIN, ea is not
 * meaningful.
 */
typedef struct {
  int K;
  double *t, *a, *ea;
} tangents;

static double case_first_order_t(const uint8_t *tok, int len, const double *c, const double *X, long ldx,
                                 long i, double u, double lam, double *val, double *s2v, double *w1v,
                                 double *wv, double *s2, double *w1, double *w, int *cond, const tangents *tg) {
  int sp = 0, cf = 0;
  const int K = tg ? tg->K : 0;
  for (int t = 0; t < len; ++t) {
    int v = tok[t];
    if (is_var(v) || is_const(v)) {
      val[sp] = is_var(v) ? X[(long)(v - TK_VAR0) * ldx + i] : c[v - TK_CONST0];
      s2v[sp] = 0.0;
      w1v[sp] = 0.0;
      wv[sp] = 0.0;
      for (int k = 0; k < K; ++k) {
        tg->t[sp * K + k] = tg->a[sp * K + k] = (is_const(v) && k == v - TK_CONST0) ? 1.0 : 0.0;
        tg->ea[sp * K + k] = 0.0;
      }
      ++sp;
      continue;
    }
    double uv = (v >= TK_TAN && v <= TK_TANH) ? 4.0 * u : u;
    double r, q2, q1, l1;
    if (is_binary(v)) {
      --sp;
      double a = val[sp - 1], b = val[sp];
      double ra = fo_reach(lam, s2v[sp - 1], w1v[sp - 1], wv[sp - 1]);
      double rb = fo_reach(lam, s2v[sp], w1v[sp], wv[sp]);
      r = apply_binary(v, a, b);
      double pa, pb, second = 0.0, dpa = 0.0, dpb = 0.0;
      op_partials(v, a, b, r, &pa, &pb);
      if (v == TK_MUL) {
        second = ra * rb;
        dpa = rb;
        dpb = ra;
      }
      if (v == TK_DIV) {
        double m = fabs(b) - rb;
        if (fabs(fabs(b) - PROTECT_EPS) <= rb) cf |= CF_BRANCH;
        if (!(m >= 0.9 * fabs(b) && m > 0.0)) cf |= CF_NONLIN;
        else if (fabs(b) > PROTECT_EPS) {
          second = (ra * rb + (fabs(a) + ra) * rb * rb / m) / (m * m);
          dpa = rb / (m * m);
          dpb = ra / (m * m) + 2.0 * (fabs(a) + ra) * rb / (m * m * m);
        }
      }
      q2 = pa * pa * s2v[sp - 1] + pb * pb * s2v[sp];
      l1 = fabs(pa) * w1v[sp - 1] + fabs(pb) * w1v[sp];
      q1 = fabs(pa) * wv[sp - 1] + fabs(pb) * wv[sp] + second;
      for (int k = 0; k < K; ++k) {
        double *ta = tg->t + (sp - 1) * K, *tb = tg->t + sp * K;
        double *aa = tg->a + (sp - 1) * K, *ab = tg->a + sp * K;
        double *ea = tg->ea + (sp - 1) * K, *eb = tg->ea + sp * K;
        double e = fabs(pa) * ea[k] + fabs(pb) * eb[k] + dpa * (aa[k] + ea[k]) + dpb * (ab[k] + eb[k]);
        ta[k] = pa * ta[k] + pb * tb[k];
        aa[k] = fabs(pa) * aa[k] + fabs(pb) * ab[k];
        ea[k] = e;
      }
    } else {
      double x = val[sp - 1];
      double rx = fo_reach(lam, s2v[sp - 1], w1v[sp - 1], wv[sp - 1]);
      r = apply_unary(v, x);
      double pa, pb;
      op_partials(v, x, 0.0, r, &pa, &pb);
      if ((v == TK_LOG || v == TK_INV) && fabs(fabs(x) - PROTECT_EPS) <= rx) cf |= CF_BRANCH;
      if (v == TK_EXP && fabs(fabs(x) - EXP_CLAMP) <= rx) cf |= CF_BRANCH;
      if (v == TK_SQRT && fabs(x) <= rx) cf |= CF_BRANCH;
      double k = unary_curvature(v, x, rx, r);
      int flat = (v == TK_LOG || v == TK_INV) && fabs(x) <= PROTECT_EPS; /* the constant fallback */
      if (k < 0.0 && !flat) cf |= CF_NONLIN;
      q2 = pa * pa * s2v[sp - 1];
      l1 = fabs(pa) * w1v[sp - 1];
      q1 = fabs(pa) * wv[sp - 1] + (k > 0.0 && !flat ? k * rx * rx : 0.0);
      /* the partial is 0 on a protected fallback and beyond the exp clamp */
      int flat_p = flat || (v == TK_EXP && (x > EXP_CLAMP || x < -EXP_CLAMP));
      double dp = (k > 0.0 && !flat_p) ? 2.0 * k * rx : 0.0;
      for (int j = 0; j < K; ++j) {
        double *tx = tg->t + (sp - 1) * K, *ax = tg->a + (sp - 1) * K, *ex = tg->ea + (sp - 1) * K;
        ex[j] = fabs(pa) * ex[j] + dp * (ax[j] + ex[j]);
        tx[j] = pa * tx[j];
        ax[j] = fabs(pa) * ax[j];
      }
    }
    val[sp - 1] = r;
    s2v[sp - 1] = q2 + (uv * r) * (uv * r);
    w1v[sp - 1] = l1 + uv * fabs(r);
    wv[sp - 1] = q1 + FO_BIAS * uv * fabs(r);
    /* a reach beyond the FP32 range (or NaN): not trusted, the rigorous
     * enclosure decides (and flags CF_RANGE if it leaves the range too) */
    if (!(fabs(r) + fo_reach(lam, s2v[sp - 1], w1v[sp - 1], wv[sp - 1]) <= FLT_MAX)) cf |= CF_NONLIN;
  }
  *s2 = s2v[0];
  *w1 = w1v[0];
  *w = wv[0];
  *cond |= cf;
  return val[0];
}

static double case_first_order(const uint8_t *tok, int len, const double *c, const double *X, long ldx,
                               long i, double u, double lam, double *val, double *s2v, double *w1v,
                               double *wv, double *s2, double *w1, double *w, int *cond) {
  return case_first_order_t(tok, len, c, X, ldx, i, u, lam, val, s2v, w1v, wv, s2, w1, w, cond, NULL);
}

/* case_first_order and case_interval of one case (*lo, *hi: the rigorous
 * enclosure), with the fallback for untrusted cases: on a case flagged
 * CF_BRANCH or CF_NONLIN the output error is taken at its worst, the
 * half-width of the rigorous enclosure, as systematic part (s2 = w1 = 0).
 * *cond gets the range flags of both analyses.  Work arrays: val
 * [4 (len + 1)], box [len + 1]. */
static double case_analysis(const uint8_t *tok, int len, const double *c, const double *X, long ldx, long i,
                            double u, double lam, double *val, ival *box, double *s2, double *w1, double *w,
                            double *lo, double *hi, int *cond) {
  size_t L = (size_t)len + 1;
  int ci = 0, cr = 0;
  double y0 = case_first_order(tok, len, c, X, ldx, i, u, lam, val, val + L, val + 2 * L, val + 3 * L, s2, w1,
                               w, &ci);
  case_interval(tok, len, c, X, ldx, i, u, val, box, &cr, lo, hi);
  if (ci & (CF_BRANCH | CF_NONLIN)) {
    *s2 = 0.0;
    *w1 = 0.0;
    *w = dmax(*hi - y0, y0 - *lo);
    ci &= ~(CF_BRANCH | CF_NONLIN);
    if (!isfinite(*w)) ci |= CF_RANGE;
  }
  *cond |= ci | cr;
  return y0;
}

/*
 * Both fitness kinds of one valid program with both certificates:
 *   errb[k]  the rigorous bound of or_condition_one for kind k (0 MSE,
 *            1 1 - r^2), from the per-case enclosures
 *   errp[k]  the probabilistic first-order bound (see above), lam standard
 *            units; never above errb[k] by construction of neither, so a
 *            caller takes the smaller
 *   cfl[k]   CF_RANGE (some case's enclosure or reach leaves the FP32 range)
 *            and CF_FITRANGE (kind k's FP32 sums may overflow, or for
 *            1 - r^2 underflow: or_condition_one)
 *   f0[k]    the FP64 fitness
 * For 1 - r^2, when the reach of the outputs moves Sxy or Sxx by more than
 * 1 % of them, r^2 is not expanded: its enclosure over the moved outputs is
 * taken instead (the rigorous bound's formula with the reach as width).
 * Work: yhat, s2, w1, w, lo, hi [N].
 */
void or_condition_fo_one(const uint8_t *tok, int len, const double *c, const double *X, long ldx,
                         const double *y, long N, double u, double lam, double *work, double *errb,
                         double *errp, int32_t *cfl, double *f0) {
  size_t L = (size_t)len + 1, nn = (size_t)(N > 0 ? N : 1);
  double *yh = work, *s2 = work + nn, *w1 = work + 2 * nn, *w = work + 3 * nn;
  double *lo = work + 4 * nn, *hi = work + 5 * nn;
  double *val = (double *)malloc(sizeof(double) * L * 4);
  ival *box = (ival *)malloc(sizeof(ival) * L);
  int cf = 0;
  for (long i = 0; i < N; ++i)
    yh[i] = case_analysis(tok, len, c, X, ldx, i, u, lam, val, box, &s2[i], &w1[i], &w[i], &lo[i], &hi[i], &cf);
  free(val);
  free(box);
  const double lim = (double)FLT_MAX / (double)nn;
  /* ---- MSE */
  {
    double base = or_mse(yh, y, N), rnd = 0.0, lin = 0.0, sys = 0.0, sec = 0.0, smin = 0.0, smax = 0.0;
    double e4 = 0.0;
    int cfk = cf;
    for (long i = 0; i < N; ++i) {
      double e = yh[i] - y[i];
      e4 += e * e * e * e;
      if (e * e > lim) cfk |= CF_FITRANGE;
      double reach = fo_reach(lam, s2[i], w1[i], w[i]);
      rnd += e * e * s2[i];
      lin += fabs(e) * w1[i];
      sys += fabs(e) * w[i];
      sec += reach * reach;
      double elo = lo[i] - y[i], ehi = hi[i] - y[i];
      double qmax = dmax(elo * elo, ehi * ehi);
      double qmin = (elo <= 0.0 && ehi >= 0.0) ? 0.0 : dmin(elo * elo, ehi * ehi);
      smin += qmin * (1.0 - 4.0 * u);
      smax += qmax * (1.0 + 4.0 * u);
    }
    /* the FP32 reduction: each case's term e^2 (the subtraction, the square
     * and its share of an 8-term sum, within 2u of it) rounds independently
     * of the others; the compensated (Kahan) running sums add at most 2
     * FP32 unit roundoffs (u / 2) of the sum of their terms' magnitudes
     * (N. J. Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed.,
     * Sec. 4.3) */
    double red = (lam * 2.0 * u * sqrt(e4)) / (double)N + 0.5 * u * base;
    double ep = (2.0 * (dmin(lam * sqrt(rnd), lin) + sys) + sec) / (double)N + red;
    double eb = dmax(smax / (double)N - base, base - smin / (double)N);
    errb[0] = !isfinite(base) ? 0.0 : (isfinite(eb) ? eb : INFINITY);
    errp[0] = !isfinite(base) ? 0.0 : (isfinite(ep) ? ep : INFINITY);
    cfl[0] = cfk & (CF_RANGE | CF_FITRANGE);
    f0[0] = base;
  }
  /* ---- 1 - r^2 */
  {
    double base = or_corr(yh, y, N), ep = 0.0, eb = 0.0;
    int cfk = cf;
    if (N >= 2) {
      double my = 0.0, mh = 0.0;
      for (long i = 0; i < N; ++i) {
        my += y[i];
        mh += yh[i];
      }
      my /= (double)N;
      mh /= (double)N;
      double sxy = 0.0, syy = 0.0, sxx = 0.0, A = 0.0, B = 0.0, Ab = 0.0, Bb = 0.0, D2 = 0.0, DY = 0.0;
      double D4 = 0.0, DY2 = 0.0, S1 = 0.0, D1 = 0.0;
      for (long i = 0; i < N; ++i) {
        double yc = y[i] - my, xc = yh[i] - mh, d = yh[i] - yh[0];
        D4 += d * d * d * d;
        DY2 += d * d * yc * yc;
        S1 += d;
        D1 += fabs(d);
        double reach = fo_reach(lam, s2[i], w1[i], w[i]);
        double b = dmax(hi[i] - yh[i], yh[i] - lo[i]);
        if (d * d > lim || fabs(d * yc) > lim) cfk |= CF_FITRANGE;
        sxy += yc * xc;
        syy += yc * yc;
        sxx += xc * xc;
        A += fabs(yc) * reach;
        B += 2.0 * fabs(xc) * reach + reach * reach;
        Ab += fabs(yc) * b;
        Bb += 2.0 * fabs(xc) * b + b * b;
        D2 += d * d;
        DY += fabs(d * yc);
      }
      if (fp32_terms_underflow(N, D2, DY)) cfk |= CF_FITRANGE;
      if (sxx > 0.0 && syy > 0.0) {
        double r2 = sxy * sxy / (sxx * syy);
        /* enclosure of r^2 over outputs moved by up to width[i] (A, B) plus
         * the FP32 moment reduction at its worst (8u of its sums) */
#define R2_ENCLOSURE(A_, B_, out)                                                              \
  do {                                                                                          \
    double Ar_ = (A_) + 8.0 * u * DY, Br_ = (B_) + 8.0 * u * D2;                                \
    double l_ = fabs(sxy) - Ar_;                                                                \
    l_ = l_ > 0.0 ? l_ * l_ / ((sxx + Br_) * syy) : 0.0;                                         \
    double h_ = sxx - Br_ > 0.0 ? (fabs(sxy) + Ar_) * (fabs(sxy) + Ar_) / ((sxx - Br_) * syy) : INFINITY; \
    (out) = dmax(h_ - r2, r2 - l_) + 4.0 * u * r2;                                              \
  } while (0)
        R2_ENCLOSURE(Ab, Bb, eb);
        double alpha = 2.0 * sxy / (sxx * syy), beta = sxy / sxx, rnd = 0.0, lin = 0.0, sys = 0.0;
        for (long i = 0; i < N; ++i) {
          double g = alpha * ((y[i] - my) - beta * (yh[i] - mh));
          rnd += g * g * s2[i];
          lin += fabs(g) * w1[i];
          sys += fabs(g) * w[i];
        }
        double ra = fabs(sxy) > 0.0 ? A / fabs(sxy) : INFINITY, rb = B / sxx;
        if (ra <= 1e-2 && rb <= 1e-2) {
          /* the FP32 moment reduction: per case the terms d yc and d^2 (with
           * d = yhat - shift and yc = y - mean y rounded to FP32) are within 2u
           * of exact and round independently of the other cases; the
           * compensated running sums add at most u / 2 of the sum of their
           * terms' magnitudes; Sxx = sum d^2 - (sum d)^2 / N also carries the
           * error of sum d.  The merges and r^2 itself are FP64 (1e-15). */
          double ea = lam * 2.0 * u * sqrt(DY2) + 0.5 * u * DY;
          double es1 = lam * u * sqrt(D2) + 0.5 * u * D1;
          double eb2 = lam * 2.0 * u * sqrt(D4) + 0.5 * u * D2 + 2.0 * fabs(S1) / (double)N * es1;
          double l = fabs(sxy) - ea;
          l = l > 0.0 ? l * l / ((sxx + eb2) * syy) : 0.0;
          double h = sxx - eb2 > 0.0 ? (fabs(sxy) + ea) * (fabs(sxy) + ea) / ((sxx - eb2) * syy) : INFINITY;
          double red = dmax(h - r2, r2 - l) + 1e-15 * r2;
          ep = dmin(lam * sqrt(rnd), lin) + sys + red + 4.0 * r2 * (ra * ra + rb * rb);
        } else {
          /* too far for a linear expansion of r^2 */
          R2_ENCLOSURE(A, B, ep);
        }
#undef R2_ENCLOSURE
      }
    }
    errb[1] = !isfinite(base) ? 0.0 : (isfinite(eb) ? eb : INFINITY);
    errp[1] = !isfinite(base) ? 0.0 : (isfinite(ep) ? ep : INFINITY);
    cfl[1] = cfk & (CF_RANGE | CF_FITRANGE);
    f0[1] = base;
  }
}

/* or_condition_fo_one for every program; outputs [2][P] (row 0 MSE, row 1
 * 1 - r^2).  Invalid programs: bounds 0, flags 0, fitness +inf. */
void or_condition_fo(const uint8_t *programs, const int32_t *lengths, const float *consts, int P,
                     int Lmax, int K, const double *X, long ldx, const double *y, int nvars, long N,
                     double u, double lam, double *errb, double *errp, int32_t *cflags, double *f0,
                     int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel num_threads(nt)
  {
    size_t nn = (size_t)(N > 0 ? N : 1);
    double *work = (double *)malloc(sizeof(double) * nn * 6);
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
      const uint8_t *tok = programs + (size_t)p * Lmax;
      int md;
      double eb[2] = {0.0, 0.0}, ep[2] = {0.0, 0.0}, f[2] = {INFINITY, INFINITY};
      int32_t cf[2] = {0, 0};
      if (!or_validate(tok, lengths[p], Lmax, nvars, K, &md)) {
        double c[TK_NSLOTS];
        widen_consts(consts + (size_t)p * K, K, c);
        or_condition_fo_one(tok, lengths[p], c, X, ldx, y, N, u, lam, work, eb, ep, cf, f);
      }
      for (int k = 0; k < 2; ++k) {
        errb[(size_t)k * P + p] = eb[k];
        errp[(size_t)k * P + p] = ep[k];
        cflags[(size_t)k * P + p] = cf[k];
        f0[(size_t)k * P + p] = f[k];
      }
    }
    free(work);
  }
}

/* Per case of one valid program: output, variance scale s2, linear worst
 * case w1, systematic part w and the case's flags, after the fallback of
 * untrusted cases (raw = 0), or straight from the expansion with the
 * CF_BRANCH / CF_NONLIN flags it raised (raw = 1); for tests. */
void or_first_order_cases(const uint8_t *tok, int len, const double *c, const double *X, long ldx, long N,
                          double u, double lam, int raw, double *yhat, double *s2, double *w1, double *w,
                          int32_t *cflags) {
  size_t L = (size_t)len + 1;
  double *val = (double *)malloc(sizeof(double) * L * 4);
  ival *box = (ival *)malloc(sizeof(ival) * L);
  for (long i = 0; i < N; ++i) {
    int cf = 0;
    double lo, hi;
    yhat[i] = raw ? case_first_order(tok, len, c, X, ldx, i, u, lam, val, val + L, val + 2 * L, val + 3 * L,
                                     &s2[i], &w1[i], &w[i], &cf)
                  : case_analysis(tok, len, c, X, ldx, i, u, lam, val, box, &s2[i], &w1[i], &w[i], &lo, &hi, &cf);
    cflags[i] = cf;
  }
  free(val);
  free(box);
}

/* ---- Beagle's scores (Sec. 2.1.5, Eq. 2 and Eq. 3) ---------------------- */
/*
 * Readings (also in the design notes):
 *   - a value is invalid when it is not finite (NaN, +inf, -inf); a model
 *     output is FP32, so an FP64 output at or beyond the FP32 overflow
 *     threshold (2^128 - 2^103) counts as invalid;
 *   - a pair is valid when both values are; c1 counts pairs with exactly one
 *     invalid value, c2 pairs with two;
 *   - Eq. 3 is decided in FP32 (the precision of the outputs), every
 *     operation rounded on its own, "round" = half to even; the case scores
 *     are integers summed exactly;
 *   - Eq. 2: r is Eq. 1 over the valid pairs (two-pass, FP64); r^2 = 0 when
 *     fewer than two pairs are valid or either sum of squares is 0; r^2 is
 *     at most 1.
 */
#define OVF32 3.4028235677973366e38 /* 2^128 - 2^103: FP32 rounds to inf from here */

static int valid_output(double v) { return !isnan(v) && fabs(v) < OVF32; }

/* Eq. 3 on one case (FP32). */
int or_p2p_case32(float yh, float y, int M) {
  int vh = isfinite(yh), vy = isfinite(y);
  if (!(vh && vy)) return (vh || vy) ? -M : M;
  float a = fabsf(yh), b = fabsf(y);
  float mx = a > b ? a : b, mn = a > b ? b : a;
  if (mx == 0.0f) return M;
  float Mf = (float)M;
  float pen = Mf / 11.0f;
  float v = Mf * (mn / mx);
  if ((yh < 0.0f && y > 0.0f) || (yh > 0.0f && y < 0.0f)) v = v - pen;
  return (int)rintf(v);
}

/* Eq. 3 summed over N cases of FP64 outputs (rounded to FP32) and FP32-valued
 * targets; pair counts in c12[0], c12[1]. */
double or_score_p2p(const double *yhat, const double *y, long N, int M, double *c12) {
  double s = 0.0, c1 = 0.0, c2 = 0.0;
  for (long i = 0; i < N; ++i) {
    float yh = valid_output(yhat[i]) ? (float)yhat[i] : NAN;
    float yt = (float)y[i];
    int vh = isfinite(yh), vy = isfinite(yt);
    c1 += vh != vy;
    c2 += !vh && !vy;
    s += (double)or_p2p_case32(yh, yt, M);
  }
  if (c12) {
    c12[0] = c1;
    c12[1] = c2;
  }
  return s;
}

/* Eq. 2: M r^4 (N - (c1 + c2)) - M (c1 - c2), r over the valid pairs. */
double or_score_r4(const double *yhat, const double *y, long N, int M, double *c12) {
  double c1 = 0.0, c2 = 0.0, n = 0.0, mh = 0.0, my = 0.0;
  for (long i = 0; i < N; ++i) {
    int vh = valid_output(yhat[i]), vy = isfinite(y[i]);
    c1 += vh != vy;
    c2 += !vh && !vy;
    if (vh && vy) {
      n += 1.0;
      mh += yhat[i];
      my += y[i];
    }
  }
  double r2 = 0.0;
  if (n >= 2.0) {
    mh /= n;
    my /= n;
    double sxy = 0.0, syy = 0.0, shh = 0.0;
    for (long i = 0; i < N; ++i) {
      if (!(valid_output(yhat[i]) && isfinite(y[i]))) continue;
      double dy = y[i] - my, dh = yhat[i] - mh;
      sxy += dy * dh;
      syy += dy * dy;
      shh += dh * dh;
    }
    if (isfinite(sxy) && isfinite(syy) && isfinite(shh) && syy > 0.0 && shh > 0.0) {
      r2 = (sxy * sxy) / (syy * shh);
      if (r2 > 1.0) r2 = 1.0;
    }
  }
  if (c12) {
    c12[0] = c1;
    c12[1] = c2;
  }
  return (double)M * (r2 * r2) * n - (double)M * (c1 - c2);
}

/*
 * Whole-population scores (kind 0: Eq. 2, kind 1: Eq. 3).  Invalid programs
 * score -inf with counts (0, 0).  counts [P][2] may be NULL.
 */
void or_eval_score(const uint8_t *programs, const int32_t *lengths, const float *consts, int P,
                   int Lmax, int K, const double *X, long ldx, const double *y, int nvars, long N,
                   int kind, int M, double *score, double *counts, int32_t *flags, int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel num_threads(nt)
  {
    double *yhat = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double c[TK_NSLOTS], c12[2];
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
      const uint8_t *tok = programs + (size_t)p * Lmax;
      int md;
      int f = or_validate(tok, lengths[p], Lmax, nvars, K, &md);
      if (flags) flags[p] = f;
      c12[0] = c12[1] = 0.0;
      if (f) {
        score[p] = -INFINITY;
      } else {
        widen_consts(consts + (size_t)p * K, K, c);
        or_predict(tok, lengths[p], c, X, ldx, N, yhat);
        score[p] = kind == 0 ? or_score_r4(yhat, y, N, M, c12) : or_score_p2p(yhat, y, N, M, c12);
      }
      if (counts) {
        counts[2 * p] = c12[0];
        counts[2 * p + 1] = c12[1];
      }
    }
    free(yhat);
  }
}

/*
 * Range of the Eq. 3 score that any FP32 evaluation can produce.  Per case
 * the FP32 output lies in the enclosure [lo, hi] (case_interval).  With y
 * fixed, min(|v|,|y|) / max(|v|,|y|) is monotone in v between the breakpoints
 * -|y|, 0 and |y|, the sign penalty is constant on each side of 0, and the
 * FP32 operations that follow are monotone; so the case score's extremes over
 * [lo, hi] are among its values at the ends, at the breakpoints inside, and
 * at the nearest nonzero FP32 values on either side of 0.  When the enclosure
 * reaches past the FP32 range, the invalid-output score joins the candidates.
 * *smin, *smax: sums over the cases; returns 1 when some intermediate of some
 * case may leave the FP32 range (the enclosure then does not model FP32
 * overflow inside the program, and the range is not guaranteed).
 */
int or_p2p_range_one(const uint8_t *tok, int len, const double *c, const double *X, long ldx,
                     const double *y, long N, double u, int M, double *smin, double *smax) {
  double *val = (double *)malloc(sizeof(double) * (size_t)(len + 1));
  ival *box = (ival *)malloc(sizeof(ival) * (size_t)(len + 1));
  double tmin = 0.0, tmax = 0.0;
  int any = 0;
  for (long i = 0; i < N; ++i) {
    int cf = 0;
    double lo, hi;
    case_interval(tok, len, c, X, ldx, i, u, val, box, &cf, &lo, &hi);
    any |= cf & CF_RANGE;
    float yt = (float)y[i];
    float cand[8];
    int nc = 0;
    if (!(lo >= -FLT_MAX && hi <= FLT_MAX)) cand[nc++] = NAN;
    double l = lo < -FLT_MAX ? -FLT_MAX : lo, h = hi > FLT_MAX ? FLT_MAX : hi;
    if (l <= h) {
      cand[nc++] = (float)l;
      cand[nc++] = (float)h;
      double ay = fabs((double)yt);
      if (isfinite(ay)) {
        if (-ay >= l && -ay <= h) cand[nc++] = (float)-ay;
        if (ay >= l && ay <= h) cand[nc++] = (float)ay;
      }
      if (l <= 0.0 && h >= 0.0) {
        cand[nc++] = 0.0f;
        if (l < 0.0) cand[nc++] = -FLT_TRUE_MIN;
        if (h > 0.0) cand[nc++] = FLT_TRUE_MIN;
      }
    }
    int mn = 0, mx = 0;
    for (int k = 0; k < nc; ++k) {
      int v = or_p2p_case32(cand[k], yt, M);
      if (k == 0 || v < mn) mn = v;
      if (k == 0 || v > mx) mx = v;
    }
    tmin += mn;
    tmax += mx;
  }
  free(val);
  free(box);
  *smin = tmin;
  *smax = tmax;
  return any;
}

/* or_p2p_range_one for every program (invalid programs: -inf, -inf, 0). */
void or_p2p_range(const uint8_t *programs, const int32_t *lengths, const float *consts, int P,
                  int Lmax, int K, const double *X, long ldx, const double *y, int nvars, long N,
                  double u, int M, double *smin, double *smax, int32_t *range_flag, int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel num_threads(nt)
  {
    double c[TK_NSLOTS];
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
      const uint8_t *tok = programs + (size_t)p * Lmax;
      int md;
      if (or_validate(tok, lengths[p], Lmax, nvars, K, &md)) {
        smin[p] = smax[p] = -INFINITY;
        range_flag[p] = 0;
        continue;
      }
      widen_consts(consts + (size_t)p * K, K, c);
      range_flag[p] = or_p2p_range_one(tok, lengths[p], c, X, ldx, y, N, u, M, &smin[p], &smax[p]);
    }
  }
}

/* ---- gradient of MSE with respect to the constants (forward mode) ------ */
/*
 * Forward-mode (tangent) differentiation: every stack entry carries its
 * value and its derivative with respect to each of the K constants.  This is
 * a different method from the device's reverse sweep, on purpose.
 * Derivative conventions: d|x|/dx = sign(x) (0 at 0); a protected fallback
 * branch and a clamped exp have derivative 0; d sqrt|x| / dx = 0 at x = 0.
 * gabs (optional) receives (2/N) sum_i |e_i| a_ik, where a_ik is the
 * derivative propagated with absolute values (|da| a_a + |db| a_b at every
 * operator): the sum of the magnitudes of all chain-rule path products, which
 * bounds (up to a factor of the operation count times the unit roundoff) the
 * rounding error of any evaluation order of the chain rule -- including one
 * whose contributions cancel exactly in exact arithmetic, as for c / c.
 * *kink receives the smallest distance, over all cases, of a branch
 * argument to its switch point (|b| - 1e-3 for division and 1/x, |x| - 1e-3
 * for log, |x| for sqrt|x|, |x| - 80 for exp) or of an argument to a point
 * where the derivative explodes (|cos x| for tan, 1 - |x| for asin and acos).
 */
void or_grad_one_ex(const uint8_t *tok, int len, const double *c, int K,
                    const double *X, long ldx, const double *y, long N,
                    double *mse_out, double *grad, double *kink, double *gabs,
                    const double *reach, double *gerr) {
  double *val = (double *)malloc(sizeof(double) * (size_t)(len + 1));
  double *tan_ = (double *)malloc(sizeof(double) * (size_t)(len + 1) *
                                  (size_t)(K > 0 ? K : 1));
  double *tab = (double *)malloc(sizeof(double) * (size_t)(len + 1) *
                                 (size_t)(K > 0 ? K : 1));
  double s = 0.0, kmin = INFINITY;
  for (int k = 0; k < K; ++k) grad[k] = 0.0;
  if (gabs)
    for (int k = 0; k < K; ++k) gabs[k] = 0.0;
  if (gerr)
    for (int k = 0; k < K; ++k) gerr[k] = 0.0;
  int finite = 1;
  for (long i = 0; i < N; ++i) {
    int sp = 0;
    for (int t = 0; t < len; ++t) {
      int v = tok[t];
      if (is_var(v)) {
        val[sp] = X[(long)(v - TK_VAR0) * ldx + i];
        for (int k = 0; k < K; ++k) tan_[sp * K + k] = tab[sp * K + k] = 0.0;
        ++sp;
      } else if (is_const(v)) {
        val[sp] = c[v - TK_CONST0];
        for (int k = 0; k < K; ++k)
          tan_[sp * K + k] = tab[sp * K + k] = (k == v - TK_CONST0) ? 1.0 : 0.0;
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
        double *aa = &tab[(sp - 1) * K], *ab = &tab[sp * K];
        for (int k = 0; k < K; ++k) aa[k] = fabs(da) * aa[k] + fabs(db) * ab[k];
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
          case TK_SQ: r = x * x; dx = 2.0 * x; break;
          case TK_INV:
            if (fabs(fabs(x) - PROTECT_EPS) < kmin) kmin = fabs(fabs(x) - PROTECT_EPS);
            if (fabs(x) <= PROTECT_EPS) {
              r = 1.0; dx = 0.0;
            } else {
              r = 1.0 / x; dx = -1.0 / (x * x);
            }
            break;
          case TK_TAN:
            /* the derivative explodes at the poles: distance |cos x| */
            if (fabs(cos(x)) < kmin) kmin = fabs(cos(x));
            r = tan(x); dx = 1.0 + r * r;
            break;
          case TK_ASIN:
          case TK_ACOS:
            /* and at the ends of the domain: distance 1 - |x| */
            if (fabs(1.0 - fabs(x)) < kmin) kmin = fabs(1.0 - fabs(x));
            r = v == TK_ASIN ? asin(x) : acos(x);
            /* 1 - x^2 as (1 - x)(1 + x): exact factors near |x| = 1 */
            dx = (v == TK_ASIN ? 1.0 : -1.0) / sqrt((1.0 - x) * (1.0 + x));
            break;
          case TK_ATAN: r = atan(x); dx = 1.0 / (1.0 + x * x); break;
          default: {
            /* d tanh / dx = sech^2 x, evaluated directly (1 - tanh^2 cancels) */
            double ch = cosh(x);
            r = tanh(x);
            dx = 1.0 / (ch * ch);
            break;
          }
        }
        for (int k = 0; k < K; ++k) tx[k] = dx * tx[k];
        for (int k = 0; k < K; ++k) tab[(sp - 1) * K + k] *= fabs(dx);
        val[sp - 1] = r;
      }
    }
    double yh = val[0];
    if (!isfinite(yh)) finite = 0;
    double e = yh - y[i];
    s += e * e;
    for (int k = 0; k < K; ++k) grad[k] += 2.0 * e * tan_[k];
    if (gabs)
      for (int k = 0; k < K; ++k) gabs[k] += 2.0 * fabs(e) * tab[k];
    if (gerr && reach)
      for (int k = 0; k < K; ++k) gerr[k] += 2.0 * reach[i] * tab[k];
  }
  for (int k = 0; k < K; ++k) grad[k] /= (double)N;
  if (gabs)
    for (int k = 0; k < K; ++k) gabs[k] /= (double)N;
  if (gerr)
    for (int k = 0; k < K; ++k) gerr[k] /= (double)N;
  *mse_out = (finite && isfinite(s)) ? s / (double)N : INFINITY;
  if (kink) *kink = kmin;
  free(val);
  free(tan_);
  free(tab);
}

void or_grad_one(const uint8_t *tok, int len, const double *c, int K, const double *X, long ldx,
                 const double *y, long N, double *mse_out, double *grad, double *kink, double *gabs) {
  or_grad_one_ex(tok, len, c, K, X, ldx, y, N, mse_out, grad, kink, gabs, NULL, NULL);
}

/*
 * or_grad with what a comparison of a device gradient needs, per program:
 *   nbranch  the cases on which FP32 rounding could flip a protected branch,
 *            a clamp or the sign inside sqrt|x| (CF_BRANCH of the first-order
 *            analysis, before its fallback): there the device's derivative
 *            may belong to the other branch, so such a program's gradient is
 *            not comparable;
 *   nnonlin  the cases on which the first-order expansion is not trusted
 *            (CF_NONLIN: an operand's reach comes near a singular point, or
 *            sin / cos / exp / tan / tanh of an argument FP32 moves by more
 *            than 0.1): the device's local derivatives there carry errors
 *            the linear scale gabs does not bound, so such a program's
 *            gradient is not comparable either;
 *   gerr     [P][K] (2/N) sum_i (reach_i a_ik + (|e_i| + reach_i) ea_ik):
 *            how far FP32 evaluation can move the gradient, through e_i
 *            (reach_i: the first-order analysis's bound on the output of
 *            case i, or its rigorous enclosure where the expansion is not
 *            trusted; a_ik the derivative propagated with absolute partials)
 *            and through the local partials, which the device takes at FP32
 *            values (ea_ik: the tangent error bound of case_first_order_t).
 */
void or_grad_cert(const uint8_t *programs, const int32_t *lengths, const float *consts, int P, int Lmax, int K,
                  const double *X, long ldx, const double *y, int nvars, long N, double u, double lam,
                  double *mse, double *grad, double *gabs, double *gerr, int32_t *nbranch, int32_t *nnonlin,
                  int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel num_threads(nt)
  {
    size_t nn = (size_t)(N > 0 ? N : 1);
    double *reach = (double *)malloc(sizeof(double) * nn);
    double *val = (double *)malloc(sizeof(double) * (size_t)(Lmax + 1) * 4);
    ival *box = (ival *)malloc(sizeof(ival) * (size_t)(Lmax + 1));
    size_t nk = (size_t)(Lmax + 1) * (size_t)(K > 0 ? K : 1);
    tangents tg = {K, (double *)malloc(sizeof(double) * nk), (double *)malloc(sizeof(double) * nk),
                   (double *)malloc(sizeof(double) * nk)};
    double *gpart = (double *)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
      const uint8_t *tok = programs + (size_t)p * Lmax;
      int md;
      double c[TK_NSLOTS];
      if (or_validate(tok, lengths[p], Lmax, nvars, K, &md)) {
        mse[p] = INFINITY;
        for (int k = 0; k < K; ++k)
          grad[(size_t)p * K + k] = gabs[(size_t)p * K + k] = gerr[(size_t)p * K + k] = 0.0;
        nbranch[p] = nnonlin[p] = 0;
        continue;
      }
      widen_consts(consts + (size_t)p * K, K, c);
      int len = lengths[p], nb = 0, nl = 0;
      size_t L = (size_t)len + 1;
      for (int k = 0; k < K; ++k) gpart[k] = 0.0;
      for (long i = 0; i < N; ++i) {
        double s2, w1, w, lo, hi;
        int cf = 0;
        double y0 = case_first_order_t(tok, len, c, X, ldx, i, u, lam, val, val + L, val + 2 * L, val + 3 * L,
                                       &s2, &w1, &w, &cf, &tg);
        nb += (cf & CF_BRANCH) != 0;
        nl += (cf & CF_NONLIN) != 0;
        /* the root's tangent error, weighed by |e_i| and its reach */
        double e = fabs(y0 - y[i]);
        int ca = 0;
        case_analysis(tok, len, c, X, ldx, i, u, lam, val, box, &s2, &w1, &w, &lo, &hi, &ca);
        reach[i] = fo_reach(lam, s2, w1, w);
        for (int k = 0; k < K; ++k) gpart[k] += 2.0 * (e + reach[i]) * tg.ea[k];
      }
      nbranch[p] = nb;
      nnonlin[p] = nl;
      or_grad_one_ex(tok, len, c, K, X, ldx, y, N, &mse[p], grad + (size_t)p * K, NULL, gabs + (size_t)p * K,
                     reach, gerr + (size_t)p * K);
      for (int k = 0; k < K; ++k) gerr[(size_t)p * K + k] += gpart[k] / (double)N;
    }
    free(reach);
    free(val);
    free(box);
    free(tg.t);
    free(tg.a);
    free(tg.ea);
    free(gpart);
  }
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
             double *grad, double *kink, double *gabs, int nthreads) {
  int nt = thread_count(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (int p = 0; p < P; ++p) {
    const uint8_t *tok = programs + (size_t)p * Lmax;
    int md;
    double c[TK_NSLOTS];
    if (or_validate(tok, lengths[p], Lmax, nvars, K, &md)) {
      mse[p] = INFINITY;
      for (int k = 0; k < K; ++k) grad[(size_t)p * K + k] = 0.0;
      if (gabs)
        for (int k = 0; k < K; ++k) gabs[(size_t)p * K + k] = 0.0;
      if (kink) kink[p] = 0.0;
      continue;
    }
    widen_consts(consts + (size_t)p * K, K, c);
    or_grad_one(tok, lengths[p], c, K, X, ldx, y, N, &mse[p],
                grad + (size_t)p * K, kink ? &kink[p] : NULL,
                gabs ? gabs + (size_t)p * K : NULL);
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
#define PU_MICRO_SAMPLE 11
#define PU_MICRO_A 12
#define PU_MICRO_B 13

/* ---- tournament selection ---------------------------------------------- */
/*
 * Child slot i draws k candidates per parent with replacement:
 * candidate j uses word j%4 of Philox(counter = (j/4, i, purpose, gen)),
 * mapped to [0, P).  The smallest fitness wins; NaN counts as +inf; equal
 * fitness goes to the smaller index.  Parent A uses purpose 1, B purpose 2.
 */
/* k-way tournament; maximise = 0: the smallest fitness wins (NaN = +inf),
 * maximise = 1: the largest score wins (NaN = -inf); ties to the smaller
 * index in both. */
static void tournament_dir(const double *fitness, int P, int k, uint64_t seed, uint64_t gen,
                           int maximise, int32_t *parents) {
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
        if (isnan(f)) f = maximise ? -INFINITY : INFINITY;
        int better = maximise ? f > bestf : f < bestf;
        if (best < 0 || better || (f == bestf && cand < best)) {
          best = cand;
          bestf = f;
        }
      }
      parents[2 * i + s] = best;
    }
  }
}

void or_tournament(const double *fitness, int P, int k, uint64_t seed,
                   uint64_t gen, int32_t *parents) {
  tournament_dir(fitness, P, k, seed, gen, 0, parents);
}

void or_tournament_max(const double *score, int P, int k, uint64_t seed,
                       uint64_t gen, int32_t *parents) {
  tournament_dir(score, P, k, seed, gen, 1, parents);
}

/*
 * Beagle's Monte-Carlo ("microcosm") selection (Sec. 2.1.6), as specified in
 * include/sr.h: S sampled individuals, sorted by key (fitness, NaN as +inf,
 * equal keys by sample position); tau = the key at rank ceil(keep S) - 1;
 * each parent is the first of up to 64 uniform candidates whose key is at
 * most tau, else the best of them (ties to the smaller index).
 */
static double micro_key(double f) { return isnan(f) ? INFINITY : f; }

typedef struct {
  double key;
  int pos;
} keyed;

static int keyed_cmp(const void *a, const void *b) {
  const keyed *x = (const keyed *)a, *y = (const keyed *)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return (x->pos > y->pos) - (x->pos < y->pos);
}

void or_microcosm(const double *fitness, int P_in, int P_out, int S, double keep, uint64_t seed,
                  uint64_t gen, int32_t *parents, double *tau_out) {
  keyed *smp = (keyed *)malloc(sizeof(keyed) * (size_t)S);
  uint32_t w[4];
  for (int j = 0; j < S; ++j) {
    if (j % 4 == 0) draw4(seed, (uint32_t)(j / 4), 0u, PU_MICRO_SAMPLE, gen, w);
    int idx = (int)below(w[j % 4], (uint32_t)P_in);
    smp[j].key = micro_key(fitness[idx]);
    smp[j].pos = j;
  }
  qsort(smp, (size_t)S, sizeof(keyed), keyed_cmp);
  int kq = (int)ceil(keep * (double)S) - 1;
  kq = kq < 0 ? 0 : (kq >= S ? S - 1 : kq);
  double tau = smp[kq].key;
  free(smp);
  if (tau_out) *tau_out = tau;
  for (int i = 0; i < P_out; ++i) {
    for (int s = 0; s < 2; ++s) {
      int best = -1, chosen = -1;
      double bestk = 0.0;
      for (int r = 0; r < 16 && chosen < 0; ++r) {
        draw4(seed, (uint32_t)r, (uint32_t)i, s == 0 ? PU_MICRO_A : PU_MICRO_B, gen, w);
        for (int q = 0; q < 4; ++q) {
          int cand = (int)below(w[q], (uint32_t)P_in);
          double k = micro_key(fitness[cand]);
          if (k <= tau) {
            chosen = cand;
            break;
          }
          if (best < 0 || k < bestk || (k == bestk && cand < best)) {
            best = cand;
            bestk = k;
          }
        }
      }
      parents[2 * i + s] = chosen >= 0 ? chosen : best;
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
static int gen_token(int d, int r, int nvars, int K, int nun, uint32_t w0, uint32_t w1) {
  int allowed[3], na = 0;
  if (d <= r - 1) allowed[na++] = 0;
  if (d >= 1 && d <= r) allowed[na++] = 1;
  if (d >= 2 && d <= r + 1) allowed[na++] = 2;
  int cls = allowed[below(w0, (uint32_t)na)];
  if (cls == 0) {
    int q = (int)below(w1, (uint32_t)(nvars + K));
    return q < nvars ? TK_VAR0 + q : TK_CONST0 + (q - nvars);
  }
  if (cls == 1) return TK_SIN + (int)below(w1, (uint32_t)nun);
  return TK_ADD + (int)below(w1, 4u);
}

/*
 * Random population: length L = Lmin + [0, Lmax - Lmin] from word 0 of
 * Philox(0, i, 9, stream); token t from Philox(1 + t, i, 9, stream);
 * constant k = fl32(cmin + fl32(u * fl32(cmax - cmin))) with u from word 0
 * of Philox(k, i, 10, stream).  Bytes past L are zero.
 */
void or_random_programs(uint8_t *prog, int32_t *len, float *c, int P,
                        int Lmin, int Lmax, int K, int nvars, int unary_ops,
                        float cmin, float cmax, uint64_t seed, uint64_t stream) {
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
      int v = gen_token(d, L - t, nvars, K, unary_ops, w[0], w[1]);
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
void or_vary(const uint8_t *prog_in, const int32_t *len_in, const float *c_in, int P_in,
             const int32_t *parents, uint8_t *prog_out, int32_t *len_out,
             float *c_out, int P, int Lmax, int K, int nvars, float p_cross,
             float p_point, float p_subtree, float p_const, float delta,
             int max_subtree, int unary_ops, uint64_t seed, uint64_t gen) {
  uint8_t *buf = (uint8_t *)malloc((size_t)Lmax + (size_t)max_subtree + 8);
  uint8_t *tmp = (uint8_t *)malloc((size_t)Lmax + (size_t)max_subtree + 8);
  for (int i = 0; i < P; ++i) {
    int ia = parents[2 * i], ib = parents[2 * i + 1];
    ia = ia < 0 ? 0 : (ia >= P_in ? P_in - 1 : ia);
    ib = ib < 0 ? 0 : (ib >= P_in ? P_in - 1 : ib);
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
        buf[t] = (uint8_t)(TK_SIN + (int)below(w[1], (uint32_t)unary_ops));
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
          int v = gen_token(d, n - j, nvars, K, unary_ops, g[0], g[1]);
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

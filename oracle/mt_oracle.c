/*
 * mt_oracle.c -- ORACLE.  Test infrastructure only.
 *
 * A plain, slow, sequential CPU implementation of the level-line Newton
 * splitting of Mihalache & Vigneron, "How to split a tera-polynomial"
 * (arXiv 2402.06083), used to check the CUDA library.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (each step cites the passage it follows):
 *   - p_0 = 0, p_{k+1} = p_k^2 + c                         (Sec. 1, eq. def:hyp_poly)
 *   - the c-derivative by differentiating that recurrence:
 *     p'_0 = 0, p'_{k+1} = 2 p_k p'_k + 1                    (Sec. 6.3.2, eq. DerParamDyna)
 *   - s_{l,n} = p_{l+n-1} + p_{l-1}                          (eq. polySimple / polyMisSimple)
 *   - q_{l,n} = p_{l+n} - p_l, with multiple roots            (eq. def:mis, Thm fact_mis)
 *   - the real end point of |P| = lambda0 by dichotomy       (Sec. 6.3.1)
 *   - the discrete level line walked sequentially, M points per
 *     turn, each point the Newton-with-target limit           (Prop. computeLevelLine,
 *                                                              eq. auxSequence, Sec. 6.3.1)
 *   - a Newton descent from every (M/c_L)-th point, capped at
 *     max{20, I_N log2 d} steps                              (Algorithm S_par, Sec. 4.2)
 *   - a sorted set with the Chebyshev separation rule and the
 *     conjugate fold near the real axis                      (Sec. 6.1, eq. nsetAsumption)
 *   - count check; on a missing root, double M and c_L       (Sec. 4.1, after Prop.
 *                                                              computeLevelLine)
 *   - exact period / Misiurewicz type of each root           (eq. def:hyp, def:mis,
 *                                                              Thm countingHyp, eq. polyMisSimple)
 *   - q_{l,n}: no descent on q itself.  eq. polySimple, s_{j,n} =
 *     q_{j,n} / q_{j-1,n}, telescoped from q_{0,n} = p_n with s_{1,n} = p_n
 *     (eq. hypCase), gives q_{l,n} = p_n^2 prod_{j=2..l} s_{j,n}, a product
 *     of polynomials with simple roots.  The distinct roots of q are the
 *     union of this oracle's own splits of p_n and of s_{j,n}, j = 2..l,
 *     merged with the Chebyshev rule; a root's multiplicity is the number
 *     of factors (p_n twice) it is a root of, its type the factor's type
 *                                                             (eq. polySimple, eq. hypCase)
 *   - seeds at any external angle: a point of |p_1| = lambda0 lifted
 *     through the nested family p_k -> p_{k+1} (target lambda0^2 at the
 *     doubled phase, then the radius brought back to lambda0), so that a
 *     window of the level line can be walked on its own    (Sec. 4.2)
 *
 * Deliberately different from the GPU design: one sequential walk from the
 * real end point (no lifting, no chunks), qsort + linear scan for the set,
 * binary128 throughout.
 *
 * Precision: binary128 by default (__float128 on x86-64, long double on
 * AArch64, both IEEE quad); binary64 when built with -DORACLE_FP64 (the
 * timed CPU baseline, same algorithm).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0 /* 0 = the oracle; 1..12 plant a known mistake (tests only) */
#endif

#if defined(ORACLE_FP64)
typedef double real;
#define RSQRT(x) sqrt(x)
#define RSIN(x) sin(x)
#define RCOS(x) cos(x)
#define RFLOOR(x) floor(x)
#define RPI 3.14159265358979323846264338327950288
#define R_TOL_WALK 1e-14
#define R_TOL_FINAL 1e-15
#define R_TOL_CLASS 1e-11
#elif defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 real;
#define RSQRT(x) sqrtq(x)
#define RSIN(x) sinq(x)
#define RCOS(x) cosq(x)
#define RFLOOR(x) floorq(x)
#define RPI M_PIq
#define R_TOL_WALK 1e-28Q
#define R_TOL_FINAL 1e-31Q
#define R_TOL_CLASS 1e-22Q
#else
typedef long double real; /* IEEE binary128 on AArch64 Linux */
#define RSQRT(x) sqrtl(x)
#define RSIN(x) sinl(x)
#define RCOS(x) cosl(x)
#define RFLOOR(x) floorl(x)
#define RPI 3.14159265358979323846264338327950288L
#define R_TOL_WALK 1e-28L
#define R_TOL_FINAL 1e-31L
#define R_TOL_CLASS 1e-22L
#endif

typedef struct {
  real re, im;
} cplx;

static cplx cx(real a, real b) {
  cplx z;
  z.re = a;
  z.im = b;
  return z;
}
static cplx cadd(cplx a, cplx b) { return cx(a.re + b.re, a.im + b.im); }
static cplx csub(cplx a, cplx b) { return cx(a.re - b.re, a.im - b.im); }
static cplx cmul(cplx a, cplx b) {
  return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
/* Textbook quotient.  In binary128 the squared modulus never overflows for
   the values met here; in binary64 |b|^2 overflows once |b| > 1e154 (orbits
   that escaped), so both operands are first scaled by the same power of two
   (exact), as the paper does when "simplifying a common large factor"
   (Sec. 6.3.2, remark on the FP80 exponent range). */
static cplx cdiv(cplx a, cplx b) {
#if defined(ORACLE_FP64)
  int e = 0;
  real m = b.re < 0 ? -b.re : b.re;
  real mi = b.im < 0 ? -b.im : b.im;
  if (mi > m) m = mi;
  if (m > 0 && m < HUGE_VAL) {
    frexp(m, &e);
    a = cx(ldexp(a.re, -e), ldexp(a.im, -e));
    b = cx(ldexp(b.re, -e), ldexp(b.im, -e));
  }
#endif
  real den = b.re * b.re + b.im * b.im;
  return cx((a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den);
}
static real cabs_(cplx a) { return RSQRT(a.re * a.re + a.im * a.im); }
static real rabs(real x) { return x < 0 ? -x : x; }
static int cfinite(cplx a) {
  /* x - x is 0 for finite x and NaN for inf/NaN */
  real t = (a.re - a.re) + (a.im - a.im);
  return t == t;
}

/* ------------------------------------------------------------------ */
/* The polynomial family.                                               */
/* kind 0: P = p_n (degree 2^(n-1));  kind 1: P = s_{l,n} = p_{l+n-1} + p_{l-1}
   (degree 2^(l+n-2));  kind 2: P = q_{l,n} = p_{l+n} - p_l (degree 2^(l+n-1)). */
typedef struct {
  int kind, l, n;
  int m;        /* length of the critical orbit that is evaluated */
  long degree;  /* deg P */
} poly;

static int poly_init(poly* P, int kind, int l, int n) {
  if (n < 1 || n > 40) return -1;
  P->kind = kind;
  P->l = l;
  P->n = n;
  if (kind == 0) {
    P->m = n;
    P->degree = 1L << (n - 1);
  } else if (kind == 1) {
    if (l < 1 || l + n > 41) return -1;
    P->m = l + n - 1;
    P->degree = 1L << (l + n - 2);
  } else if (kind == 2) {
    if (l < 1 || l + n > 40) return -1;
    P->m = l + n;
    P->degree = 1L << (l + n - 1);
  } else {
    return -1;
  }
  return 0;
}

/* Critical orbit p_k(c) with its c-derivative, eq. def:hyp_poly differentiated
   in c (the parameter-space form of eq. DerParamDyna). */
static void eval_P(const poly* P, cplx c, cplx* v, cplx* dv) {
  cplx z = cx(0, 0), dz = cx(0, 0);
  cplx zl = cx(0, 0), dzl = cx(0, 0);
#if ORACLE_MUTANT == 3 /* planted mistake: s_{l,n} built with p_l instead of p_{l-1} */
  int lcap = (P->kind == 1) ? P->l : -1;
#else
  int lcap = (P->kind == 1) ? P->l - 1 : -1;
#endif
#if ORACLE_MUTANT == 6 /* planted mistake: q_{l,n} built with p_{l-1} instead of p_l */
  if (P->kind == 2) lcap = P->l - 1;
#else
  if (P->kind == 2) lcap = P->l;
#endif
  if (lcap == 0) { zl = z; dzl = dz; }
  for (int k = 1; k <= P->m; ++k) {
#if ORACLE_MUTANT == 1 /* planted mistake: derivative from p_k instead of p_{k-1} */
    z = cadd(cmul(z, z), c);
    dz = cadd(cmul(cx(2 * z.re, 2 * z.im), dz), cx(1, 0));
#elif ORACLE_MUTANT == 2 /* planted mistake: sign of Im(z)^2 in Re(z^2) */
    cplx two_z = cx(2 * z.re, 2 * z.im);
    dz = cadd(cmul(two_z, dz), cx(1, 0));
    z = cx(z.re * z.re + z.im * z.im + c.re, 2 * z.re * z.im + c.im);
#else
    cplx two_z = cx(2 * z.re, 2 * z.im);
    dz = cadd(cmul(two_z, dz), cx(1, 0)); /* p'_k = 2 p_{k-1} p'_{k-1} + 1 */
    z = cadd(cmul(z, z), c);              /* p_k  = p_{k-1}^2 + c          */
#endif
    if (k == lcap) { zl = z; dzl = dz; }
  }
  if (P->kind == 1) {
    z = cadd(z, zl);
    dz = cadd(dz, dzl);
  } else if (P->kind == 2) { /* q_{l,n} = p_{l+n} - p_l */
    z = csub(z, zl);
    dz = csub(dz, dzl);
  }
  *v = z;
  *dv = dz;
}

/* p_k and p'_k at c (plain hyperbolic polynomial of index k). */
static void eval_pk(int k, cplx c, cplx* v, cplx* dv) {
  cplx z = cx(0, 0), dz = cx(0, 0);
  for (int j = 1; j <= k; ++j) {
    cplx two_z = cx(2 * z.re, 2 * z.im);
    dz = cadd(cmul(two_z, dz), cx(1, 0));
    z = cadd(cmul(z, z), c);
  }
  *v = z;
  *dv = dz;
}

/* ------------------------------------------------------------------ */
/* Real end point of the level line |P| = lambda0 on c > 0 (Sec. 6.3.1:
   "found by dichotomy").  P is increasing on (0, +inf) for the three
   families (every p_k and p'_k grows with c there, and p'_{k+1} >= p'_k for
   q) and P(0) = 0 < lambda0 <= P(lambda0), so [0, lambda0] brackets it. */
static real real_endpoint(const poly* P, real lambda0) {
  real lo = 0, hi = lambda0;
  for (int it = 0; it < 400; ++it) {
    real mid = (lo + hi) / 2;
    if (mid == lo || mid == hi) break;
    cplx v, dv;
    eval_P(P, cx(mid, 0), &v, &dv);
    if (v.re < lambda0) lo = mid; else hi = mid;
  }
  return (lo + hi) / 2;
}

/* Newton map with target zeta: L(P; z0, zeta) = lim N_{P - zeta}^k(z0)
   (Sec. 4.1, definition before Prop. computeLevelLine).  Returns the number
   of Newton steps taken; *ok is 0 if the limit was not reached. */
static int newton_target(const poly* P, cplx* z, cplx zeta, real tol, int cap, int* ok) {
  int it;
  *ok = 0;
  for (it = 0; it < cap;) {
    cplx v, dv;
    eval_P(P, *z, &v, &dv);
    cplx step = cdiv(csub(v, zeta), dv);
    *z = csub(*z, step);
    ++it;
    if (!cfinite(*z)) return it;
    real s = cabs_(step);
    if (s <= tol * (1 + cabs_(*z))) { *ok = 1; return it; }
  }
  return it;
}

static void split_real(real x, double* hi, double* lo);

/* ------------------------------------------------------------------ */
typedef struct {
  long degree;       /* deg P */
  long n_roots;      /* distinct roots found (full conjugate-closed list) */
  long n_real;       /* real roots among them */
  long n_starts;     /* descents started (upper half of the level line) */
  long n_conv;       /* descents that converged */
  long n_repeat;     /* converged descents that hit an already found root */
  long n_diverge;    /* descents stopped by a long jump / non-finite value */
  long n_timeout;    /* descents stopped by the iteration cap */
  long walk_newton;  /* Newton steps spent on the level line */
  long desc_newton;  /* Newton steps spent in descents */
  long walk_fail;    /* level-line points whose Newton limit was not reached */
  int M, cL;         /* points per turn and starts per root finally used */
  int retries;       /* number of (M, c_L) doublings */
  int endpoint_ok;   /* the walk ended on the real axis left of the set */
  long n_mult;       /* roots counted with multiplicity (q_{l,n}; n_roots otherwise) */
} or_stats;

typedef struct {
  cplx z;
  real step; /* size of the last Newton step (the representative rule) */
} cand;

static int cand_cmp(const void* a, const void* b) {
  const cand* x = (const cand*)a;
  const cand* y = (const cand*)b;
  if (x->z.re < y->z.re) return -1;
  if (x->z.re > y->z.re) return 1;
  if (x->z.im < y->z.im) return -1;
  if (x->z.im > y->z.im) return 1;
  return 0;
}

static int cplx_lex_cmp(const void* a, const void* b) {
  const cplx* x = (const cplx*)a;
  const cplx* y = (const cplx*)b;
  /* eq. defLexi: Re first, then Im */
  if (x->re < y->re) return -1;
  if (x->re > y->re) return 1;
  if (x->im < y->im) return -1;
  if (x->im > y->im) return 1;
  return 0;
}

/* One pass of the method with given (M, c_L) over the sub-steps jbeg ..
   jend of the upper half of the level line (external-angle index t =
   j / (M d), t in [0, 1/2]): the walk starts from z0, the point of index
   jbeg, and, when 'descend' is set, a Newton descent runs from every
   (M/c_L)-th point; the folded converged candidates are left in *out.
   With descend = 0 only the starts are recorded (the level line itself). */
static long one_pass(const poly* P, int M, int cL, real lambda0, int cap, long jbeg, long jend,
                     cplx z0, int descend, cand** out, or_stats* st, double* starts_out,
                     long starts_cap) {
  long J = (long)M * P->degree / 2; /* sub-steps from t = 0 to t = 1/2 */
  int every = M / cL;
  long ncap = (jend - jbeg) / every + 2;
  cand* cs = (cand*)malloc(sizeof(cand) * (size_t)ncap);
  long nc = 0, nstart = 0;
  cplx z = z0;
  for (long j = jbeg; j <= jend; ++j) {
    if (j > jbeg) {
      /* target P(z_j) = lambda0 e^{2 i pi j / M}; the phase is reduced mod M
         so that it is exact for every j (Sec. 6.3.1). */
#if ORACLE_MUTANT == 4 /* planted mistake: the walk turns the wrong way */
      real ang = -2 * RPI * (real)(j % M) / (real)M;
#else
      real ang = 2 * RPI * (real)(j % M) / (real)M;
#endif
      cplx zeta = cx(lambda0 * RCOS(ang), lambda0 * RSIN(ang));
      int ok;
      st->walk_newton += newton_target(P, &z, zeta, R_TOL_WALK, 80, &ok);
      if (!ok) st->walk_fail++;
    }
    if (j % every != 0) continue;
    if (starts_out && nstart < starts_cap) {
      split_real(z.re, &starts_out[4 * nstart + 0], &starts_out[4 * nstart + 1]);
      split_real(z.im, &starts_out[4 * nstart + 2], &starts_out[4 * nstart + 3]);
    }
    ++nstart;
    if (!descend) continue;
    /* Newton descent (Algorithm S_par, capped at max{20, I_N log2 d}). */
    cplx w = z;
    real s = 0;
    /* a long-distance jump (Sec. 6.4.1): beyond twice the start radius and
       outside D(0, 4), which holds every root (M lies in D(0,2) u {-2}) */
    real rdiv = 2 * cabs_(z);
    if (rdiv < 4) rdiv = 4;
    int conv = 0, div = 0, it;
    for (it = 0; it < cap; ++it) {
      cplx v, dv;
      eval_P(P, w, &v, &dv);
      cplx step = cdiv(v, dv);
      st->desc_newton++;
      w = csub(w, step);
      if (!cfinite(w) || cabs_(w) > rdiv) { div = 1; break; }
      s = cabs_(step);
      if (s < 1e-12) { conv = 1; break; }
    }
    if (conv) {
      /* finish to the working precision (a few quadratic steps) */
#if ORACLE_MUTANT == 10 /* planted mistake: no finishing steps to the working precision */
      for (int k = 0; k < 0; ++k) {
#else
      for (int k = 0; k < 8 && s > R_TOL_FINAL; ++k) {
#endif
        cplx v, dv;
        eval_P(P, w, &v, &dv);
        cplx step = cdiv(v, dv);
        real s2 = cabs_(step);
        w = csub(w, step);
        st->desc_newton++;
        if (!(s2 < s)) { s = s2; break; }
        s = s2;
      }
#if ORACLE_MUTANT != 5 /* mutant 5 plants a missing conjugate fold */
      if (w.im < 0) w.im = -w.im; /* conjugate fold: the root set is symmetric */
#endif
      cs[nc].z = w;
      cs[nc].step = s;
      ++nc;
      st->n_conv++;
    } else if (div) {
      st->n_diverge++;
    } else {
      st->n_timeout++;
    }
  }
  st->n_starts += nstart;
  if (jbeg == 0 && jend == J) {
    /* the walk must end at the negative real end point, left of M */
    st->endpoint_ok = (rabs(z.im) < 1e-10 && z.re < -1.9) ? 1 : 0;
  }
  *out = cs;
  return nc;
}

/* Sorted set with the Chebyshev separation rule (eq. nsetAsumption): a
   candidate joins an existing point if max(|dRe|, |dIm|) < eps.  Points with
   |Im| < eps/2 are real.  Returns the number of upper-half representatives. */
static long dedup(cand* cs, long nc, real eps, cplx* reps, long* n_repeat) {
#if ORACLE_MUTANT != 8 /* mutant 8 plants a missing real-root rule */
  for (long i = 0; i < nc; ++i)
    if (cs[i].z.im < eps / 2) cs[i].z.im = 0;
#endif
  qsort(cs, (size_t)nc, sizeof(cand), cand_cmp);
  long nr = 0;
  for (long i = 0; i < nc; ++i) {
    int dup = 0;
    for (long j = nr - 1; j >= 0 && cs[i].z.re - reps[j].re < eps; --j) {
      if (rabs(cs[i].z.im - reps[j].im) < eps) { dup = 1; break; }
    }
    if (dup) { (*n_repeat)++; continue; }
    reps[nr++] = cs[i].z;
  }
  return nr;
}

static void split_real(real x, double* hi, double* lo) {
  double h = (double)x;
  *hi = h;
  *lo = (double)(x - (real)h);
}
static real join_real(double hi, double lo) { return (real)hi + (real)lo; }

/* ------------------------------------------------------------------ */
/* Exact type of a root (eq. def:hyp and def:mis).
   kind 0: *a = 0, *b = smallest k | n with p_k(c) = 0.
   kind 1 (root of s_{l,n}): hyperbolic centres of period k | gcd(n, l-1)
   give (*a, *b) = (0, k); otherwise (*a, *b) = (l, k) with k the smallest
   divisor of n such that q_{l,k}(c) = p_{l+k}(c) - p_l(c) = 0.  A value is
   "zero" when its Newton step |f/f'| is below tau. */
static int is_zero_step(cplx v, cplx dv, real tau) {
  real a = cabs_(v), b = cabs_(dv);
  return a <= tau * b;
}
static int gcd_i(int a, int b) {
  while (b) { int t = a % b; a = b; b = t; }
  return a;
}
static int is_zero_q(int j, int k, cplx c, real tau) {
  /* q_{j,k}(c) = p_{j+k}(c) - p_j(c) */
  cplx v1, d1, v2, d2;
  eval_pk(j + k, c, &v1, &d1);
  eval_pk(j, c, &v2, &d2);
  return is_zero_step(csub(v1, v2), csub(d1, d2), tau);
}
static void classify(const poly* P, cplx c, real tau, int* a, int* b) {
  cplx v, dv;
  if (P->kind == 2) {
    /* root of q_{l,n} (Thm fact_mis): Hyp(k) for the smallest k | n with
       p_k(c) = 0; otherwise Mis(j,k): k the smallest divisor of n with
       q_{l,k}(c) = 0, then j the smallest preperiod with q_{j,k}(c) = 0
       (q_{j,k} vanishes on Mis(j0,k0) exactly when j >= j0 and k0 | k) */
    for (int k = 1; k <= P->n; ++k) {
      if (P->n % k) continue;
      eval_pk(k, c, &v, &dv);
      if (is_zero_step(v, dv, tau)) { *a = 0; *b = k; return; }
    }
    for (int k = 1; k <= P->n; ++k) {
      if (P->n % k || !is_zero_q(P->l, k, c, tau)) continue;
      for (int j = 2; j <= P->l; ++j)
        if (is_zero_q(j, k, c, tau)) { *a = j; *b = k; return; }
    }
    *a = -1; *b = -1;
    return;
  }
  if (P->kind == 0) {
#if ORACLE_MUTANT == 9 /* planted mistake: the largest period that vanishes, not the smallest */
    for (int k = P->n; k >= 1; --k) {
#else
    for (int k = 1; k <= P->n; ++k) {
#endif
      if (P->n % k) continue;
      eval_pk(k, c, &v, &dv);
      if (is_zero_step(v, dv, tau)) { *a = 0; *b = k; return; }
    }
    *a = 0; *b = -1;
    return;
  }
  int g = gcd_i(P->n, P->l - 1);
#if ORACLE_MUTANT == 12 /* planted mistake: Mis(l,k) tested before Hyp(k) */
  g = 0;
#endif
  for (int k = 1; k <= g; ++k) {
    if (g % k) continue;
    eval_pk(k, c, &v, &dv);
    if (is_zero_step(v, dv, tau)) { *a = 0; *b = k; return; }
  }
  for (int k = 1; k <= P->n; ++k) {
    if (P->n % k) continue;
    cplx v1, d1, v2, d2;
    eval_pk(P->l + k, c, &v1, &d1);
    eval_pk(P->l, c, &v2, &d2);
    if (is_zero_step(csub(v1, v2), csub(d1, d2), tau)) { *a = P->l; *b = k; return; }
  }
  *a = -1; *b = -1;
}

/* ------------------------------------------------------------------ */
/* Public entry points (ctypes).                                        */

long or_degree(int kind, int l, int n) {
  poly P;
  if (poly_init(&P, kind, l, n)) return -1;
  return P.degree;
}

/* P and P' at c = (re_hi + re_lo) + i (im_hi + im_lo).
   out[0..3] = Re P hi, lo, Im P hi, lo;  out[4..7] = same for P'. */
int or_eval(int kind, int l, int n, const double* c4, double* out8) {
  poly P;
  if (poly_init(&P, kind, l, n)) return -1;
  cplx c = cx(join_real(c4[0], c4[1]), join_real(c4[2], c4[3]));
  cplx v, dv;
  eval_P(&P, c, &v, &dv);
  split_real(v.re, &out8[0], &out8[1]);
  split_real(v.im, &out8[2], &out8[3]);
  split_real(dv.re, &out8[4], &out8[5]);
  split_real(dv.im, &out8[6], &out8[7]);
  return 0;
}

/* p_k and p'_k at c, same layout as or_eval. */
int or_eval_pk(int k, const double* c4, double* out8) {
  cplx c = cx(join_real(c4[0], c4[1]), join_real(c4[2], c4[3]));
  cplx v, dv;
  eval_pk(k, c, &v, &dv);
  split_real(v.re, &out8[0], &out8[1]);
  split_real(v.im, &out8[2], &out8[3]);
  split_real(dv.re, &out8[4], &out8[5]);
  split_real(dv.im, &out8[6], &out8[7]);
  return 0;
}

int or_real_endpoint(int kind, int l, int n, double lambda0, double* out2) {
  poly P;
  if (poly_init(&P, kind, l, n)) return -1;
  split_real(real_endpoint(&P, (real)lambda0), &out2[0], &out2[1]);
  return 0;
}

static int newton_cap(const poly* P, double I_N) {
  double log2d = 0;
  for (long d = P->degree; d > 1; d >>= 1) log2d += 1;
  int cap_steps = (int)ceil(I_N * log2d);
  return cap_steps < 20 ? 20 : cap_steps;
}

/* The split of p_n or s_{l,n} (kinds 0 and 1; q_{l,n} is or_split_q).
   roots: [cap][4] (Re hi, Re lo, Im hi, Im lo), full conjugate-closed list
   sorted by eq. defLexi.  type_a/type_b: per-root type (or NULL).  starts:
   [starts_cap][4] level-line start points of the final pass (Re hi, Re lo,
   Im hi, Im lo), upper half in external-angle order, or NULL.  frac < 1
   walks only the first part of the upper half (a bounded sample; no count
   check, no retries).  Returns the number of roots written, or a negative
   error. */
long or_split(int kind, int l, int n, int M, int cL, double lambda0, double I_N,
              double eps_dup, int max_retries, double frac,
              double* roots, long cap, int* type_a, int* type_b,
              double* starts, long starts_cap, or_stats* st) {
  poly P;
  if (kind == 2 || poly_init(&P, kind, l, n)) return -1;
  if (M < 2 || cL < 1 || M % cL) return -1;
  memset(st, 0, sizeof(*st));
  st->degree = P.degree;
  int cap_steps = newton_cap(&P, I_N);
  real eps = (real)eps_dup;
  long nfull = 0;
  cplx* full = NULL;
  for (int attempt = 0; attempt <= max_retries; ++attempt) {
    or_stats s1;
    memset(&s1, 0, sizeof(s1));
    s1.degree = P.degree;
    cand* cs = NULL;
    if (starts) memset(starts, 0, sizeof(double) * 4 * (size_t)starts_cap);
    long J = (long)M * P.degree / 2;
    long jend = (frac >= 1.0) ? J : (long)(frac * (double)J);
    long nc = one_pass(&P, M, cL, (real)lambda0, cap_steps, 0, jend, cx(real_endpoint(&P, (real)lambda0), 0),
                       1, &cs, &s1, starts, starts_cap);
    cplx* reps = (cplx*)malloc(sizeof(cplx) * (size_t)(nc + 1));
    long nr = dedup(cs, nc, eps, reps, &s1.n_repeat);
    free(cs);
    long nreal = 0;
    for (long i = 0; i < nr; ++i) nreal += (reps[i].im == 0);
    nfull = nreal + 2 * (nr - nreal);
    free(full);
    full = (cplx*)malloc(sizeof(cplx) * (size_t)(nfull + 1));
    long w = 0;
    for (long i = 0; i < nr; ++i) {
      full[w++] = reps[i];
      if (reps[i].im != 0) full[w++] = cx(reps[i].re, -reps[i].im);
    }
    free(reps);
    /* keep the cumulative work counters across retries */
    s1.walk_newton += st->walk_newton;
    s1.desc_newton += st->desc_newton;
    s1.retries = attempt;
    s1.n_roots = nfull;
    s1.n_mult = nfull;
    s1.n_real = nreal;
    s1.M = M;
    s1.cL = cL;
    *st = s1;
    if (frac < 1.0 || nfull >= P.degree) break;
    M *= 2; /* missing roots: a finer level line contains the coarser one */
    cL *= 2;
  }
  qsort(full, (size_t)nfull, sizeof(cplx), cplx_lex_cmp);
  long nout = nfull < cap ? nfull : cap;
  for (long i = 0; i < nout; ++i) {
    split_real(full[i].re, &roots[4 * i + 0], &roots[4 * i + 1]);
    split_real(full[i].im, &roots[4 * i + 2], &roots[4 * i + 3]);
    if (type_a && type_b) classify(&P, full[i], R_TOL_CLASS, &type_a[i], &type_b[i]);
  }
  free(full);
  return nfull;
}

/* The level line alone (kinds 0, 1 and 2): the (c_L/2) d + 1 starts of the
   upper half walked sequentially from the real end point, as in or_split,
   with no descents.  starts: [starts_cap][4].  Returns the number of starts. */
long or_walk(int kind, int l, int n, int M, int cL, double lambda0, double* starts, long starts_cap,
             or_stats* st) {
  poly P;
  if (poly_init(&P, kind, l, n)) return -1;
  if (M < 2 || cL < 1 || M % cL) return -1;
  memset(st, 0, sizeof(*st));
  st->degree = P.degree;
  cand* cs = NULL;
  long J = (long)M * P.degree / 2;
  one_pass(&P, M, cL, (real)lambda0, 0, 0, J, cx(real_endpoint(&P, (real)lambda0), 0), 0, &cs, st,
           starts, starts_cap);
  free(cs);
  st->M = M;
  st->cL = cL;
  return st->n_starts;
}

/* ------------------------------------------------------------------ */
/* A seed at any external angle (Sec. 4.2, the nested family).  The point
   of index j of the level line of p_n with M points per turn has external
   angle t = j / (M 2^(n-1)) and satisfies p_n(z) = lambda0 e^{2 i pi j / M}.
   On |p_k| = lambda0 the same angle has phase 2 pi 2^(k-1) t, the fraction
   j / (M 2^(n-k)) of a turn, reduced exactly (a dyadic fraction).  Level 1:
   p_1(c) = c, so z = lambda0 e^{2 i pi t}.  From level k to k+1: p_{k+1}(z) =
   p_k(z)^2 + z = lambda0^2 e^{i phi} + z with phi the phase of level k+1, so
   Newton with target lambda0^2 e^{i phi} moves z onto |p_{k+1}| = lambda0^2;
   the radius is then brought back to lambda0 at that phase in 'shrink'
   geometric steps, each a Newton-with-target solve from the previous point.
   Returns 0, or the number of solves that did not converge. */
static void unit_phase(long num, long den, real lambda, cplx* out) {
  long r = num % den;
  if (r < 0) r += den;
  real ang = 2 * RPI * ((real)r / (real)den);
  *out = cx(lambda * RCOS(ang), lambda * RSIN(ang));
}

static int lift_seed_pn(int n, int M, long j, real lambda0, int shrink, cplx* z_out, long* steps) {
  poly Pk;
  int fails = 0;
  cplx z;
  /* level 1 */
  unit_phase(j, (long)M << (n - 1), lambda0, &z);
  for (int k = 1; k < n; ++k) {
    poly_init(&Pk, 0, 0, k + 1);
    long den = (long)M << (n - k - 1);
    cplx target;
    int ok;
    unit_phase(j, den, lambda0 * lambda0, &target);
    *steps += newton_target(&Pk, &z, target, R_TOL_WALK, 80, &ok);
    fails += !ok;
    for (int q = 1; q <= shrink; ++q) {
      real e = 2 - (real)q / (real)shrink;
      real r = (real)exp((double)e * log((double)lambda0));
      if (q == shrink) r = lambda0;
      unit_phase(j, den, r, &target);
      *steps += newton_target(&Pk, &z, target, R_TOL_WALK, 80, &ok);
      fails += !ok;
    }
  }
  if (j == 0 || 2 * j == (long)M << (n - 1)) z.im = 0; /* the two real end points */
  *z_out = z;
  return fails;
}

/* The lifted seed of index j (kind 0 only); out4 as or_eval's layout. */
int or_lift_seed(int n, int M, long j, double lambda0, int shrink, double* out4) {
  if (n < 1 || n > 40 || M < 2 || shrink < 1) return -1;
  cplx z;
  long steps = 0;
  int f = lift_seed_pn(n, M, j, (real)lambda0, shrink, &z, &steps);
  split_real(z.re, &out4[0], &out4[1]);
  split_real(z.im, &out4[2], &out4[3]);
  return f;
}

/* One window of the split of p_n: sub-steps jbeg .. jend of the upper half
   (0 <= jbeg < jend <= M 2^(n-1) / 2), walked from the lifted seed of index
   jbeg, a descent from every (M/c_L)-th point, and the window's own root
   set (Chebyshev rule, conjugate fold).  A bounded sample of the whole
   split's work at any place of the line (the timed CPU baseline).  Returns
   the number of distinct upper-half roots found in the window, or a
   negative error; roots4 (NULL or [cap][4]) receives them in (Re, Im)
   order, st the window's counters. */
long or_split_window(int n, int M, int cL, double lambda0, double I_N, double eps_dup, long jbeg, long jend,
                     int shrink, double* roots4, long cap, or_stats* st) {
  poly P;
  if (poly_init(&P, 0, 0, n)) return -1;
  long J = (long)M * P.degree / 2;
  if (M < 2 || cL < 1 || M % cL || jbeg < 0 || jend <= jbeg || jend > J || shrink < 1) return -1;
  memset(st, 0, sizeof(*st));
  st->degree = P.degree;
  cplx z0;
  long steps = 0;
  st->walk_fail += lift_seed_pn(n, M, jbeg, (real)lambda0, shrink, &z0, &steps);
  st->walk_newton += steps;
  cand* cs = NULL;
  long nc = one_pass(&P, M, cL, (real)lambda0, newton_cap(&P, I_N), jbeg, jend, z0, 1, &cs, st, NULL, 0);
  cplx* reps = (cplx*)malloc(sizeof(cplx) * (size_t)(nc + 1));
  long nr = dedup(cs, nc, (real)eps_dup, reps, &st->n_repeat);
  free(cs);
  for (long i = 0; roots4 && i < nr && i < cap; ++i) {
    split_real(reps[i].re, &roots4[4 * i + 0], &roots4[4 * i + 1]);
    split_real(reps[i].im, &roots4[4 * i + 2], &roots4[4 * i + 3]);
  }
  free(reps);
  st->n_roots = nr;
  st->M = M;
  st->cL = cL;
  return nr;
}

/* ------------------------------------------------------------------ */
/* q_{l,n} = p_{l+n} - p_l from the telescoped eq. polySimple:
       q_{l,n} = q_{0,n} prod_{j=1..l} s_{j,n},  q_{0,n} = p_n,  s_{1,n} = p_n
   (eq. hypCase: q_{1,n} = p_n^2), i.e. q_{l,n} = p_n^2 prod_{j=2..l} s_{j,n}.
   Every factor has simple roots (Sec. 2), so the roots of q with their
   multiplicities are the union of the factors' roots, each counted once per
   factor it belongs to (p_n twice).  The factors are split by or_split
   above (each with its own count check and retries); their roots are
   merged with the Chebyshev rule of eq. nsetAsumption at eps_q.  Each
   distinct root takes the type its factor gives it: Hyp(k) -> (0, k) from
   p_n or from s_{j,n}; Mis(j,k) -> (j, k) from s_{j,n}.  Members of one
   cluster whose types differ are counted in *n_conflict. */
typedef struct {
  cplx z;
  int a, b;   /* type: (preperiod, period) */
  int w;      /* multiplicity contributed */
} qent;

static int qent_cmp(const void* x, const void* y) {
  return cplx_lex_cmp(&((const qent*)x)->z, &((const qent*)y)->z);
}

long or_split_q(int l, int n, int M, int cL, double lambda_p, double lambda_s, double IN_p, double IN_s,
                const double* eps_factor, double eps_q, int max_retries, double* roots, long cap, int* pre,
                int* per, int* mult, long* n_conflict, or_stats* st) {
  if (l < 1 || n < 1 || l + n > 40) return -1;
  memset(st, 0, sizeof(*st));
  st->degree = 1L << (l + n - 1);
  /* factor list: p_n with weight 2, then s_{j,n}, j = 2..l, weight 1 */
  int fk[42], fl[42], fw[42], nf = 0;
#if ORACLE_MUTANT == 11 /* planted mistake: p_n counted once (q_{0,n} without s_{1,n}) */
  fk[nf] = 0; fl[nf] = 0; fw[nf] = 1; ++nf;
#else
  fk[nf] = 0; fl[nf] = 0; fw[nf] = 2; ++nf;
#endif
#if ORACLE_MUTANT == 7 /* planted mistake: the product over s_{j,n} taken from j = 1 (s_{1,n} = p_n) */
  fk[nf] = 0; fl[nf] = 0; fw[nf] = 1; ++nf;
#endif
  for (int j = 2; j <= l; ++j) { fk[nf] = 1; fl[nf] = j; fw[nf] = 1; ++nf; }
  long total = 0;
  for (int f = 0; f < nf; ++f) total += (fk[f] == 0) ? (1L << (n - 1)) : (1L << (fl[f] + n - 2));
  qent* e = (qent*)malloc(sizeof(qent) * (size_t)(total + 1));
  long ne = 0;
  for (int f = 0; f < nf; ++f) {
    poly F;
    if (poly_init(&F, fk[f], fl[f], n)) { free(e); return -1; }
    double* r4 = (double*)malloc(sizeof(double) * 4 * (size_t)F.degree);
    int* ta = (int*)malloc(sizeof(int) * (size_t)F.degree);
    int* tb = (int*)malloc(sizeof(int) * (size_t)F.degree);
    or_stats fs;
    /* eps_factor[0] for p_n, eps_factor[j - 1] for s_{j,n} */
    double eps = eps_factor[fk[f] ? fl[f] - 1 : 0];
    long nr = or_split(fk[f], fl[f], n, M, cL, fk[f] ? lambda_s : lambda_p, fk[f] ? IN_s : IN_p, eps,
                       max_retries, 1.0, r4, F.degree, ta, tb, NULL, 0, &fs);
    st->walk_newton += fs.walk_newton;
    st->desc_newton += fs.desc_newton;
    st->n_starts += fs.n_starts;
    st->n_conv += fs.n_conv;
    st->n_repeat += fs.n_repeat;
    st->n_diverge += fs.n_diverge;
    st->n_timeout += fs.n_timeout;
    st->walk_fail += fs.walk_fail;
    if (fs.retries > st->retries) st->retries = fs.retries;
    if (nr > F.degree) nr = F.degree;
    for (long i = 0; i < nr; ++i) {
      e[ne].z = cx(join_real(r4[4 * i], r4[4 * i + 1]), join_real(r4[4 * i + 2], r4[4 * i + 3]));
      e[ne].a = ta[i];
      e[ne].b = tb[i];
      e[ne].w = fw[f];
      ++ne;
    }
    free(r4);
    free(ta);
    free(tb);
  }
  qsort(e, (size_t)ne, sizeof(qent), qent_cmp);
  /* greedy Chebyshev clustering in (Re, Im) order, as dedup() does */
  real eps = (real)eps_q;
  qent* reps = (qent*)malloc(sizeof(qent) * (size_t)(ne + 1));
  long nr = 0, nconf = 0, nmult = 0;
  for (long i = 0; i < ne; ++i) {
    long hit = -1;
    for (long k = nr - 1; k >= 0 && e[i].z.re - reps[k].z.re < eps; --k) {
      if (rabs(e[i].z.im - reps[k].z.im) < eps) { hit = k; break; }
    }
    if (hit < 0) {
      reps[nr++] = e[i];
      continue;
    }
    if (reps[hit].a != e[i].a || reps[hit].b != e[i].b) ++nconf;
    reps[hit].w += e[i].w;
  }
  long nout = nr < cap ? nr : cap;
  long nreal = 0;
  for (long i = 0; i < nr; ++i) {
    nmult += reps[i].w;
    nreal += (reps[i].z.im == 0);
    if (i < nout) {
      split_real(reps[i].z.re, &roots[4 * i + 0], &roots[4 * i + 1]);
      split_real(reps[i].z.im, &roots[4 * i + 2], &roots[4 * i + 3]);
      pre[i] = reps[i].a;
      per[i] = reps[i].b;
      mult[i] = reps[i].w;
    }
  }
  free(e);
  free(reps);
  st->n_roots = nr;
  st->n_real = nreal;
  st->n_mult = nmult;
  st->M = M;
  st->cL = cL;
  *n_conflict = nconf;
  return nr;
}

/* Newton polish of a given point (used to check roots produced elsewhere):
   'steps' Newton steps on P from c; out4 receives the result, *disp the
   distance |result - c|. */
int or_polish(int kind, int l, int n, const double* c4, int steps, double* out4, double* disp) {
  poly P;
  if (poly_init(&P, kind, l, n)) return -1;
  cplx c0 = cx(join_real(c4[0], c4[1]), join_real(c4[2], c4[3]));
  cplx w = c0;
  for (int k = 0; k < steps; ++k) {
    cplx v, dv;
    eval_P(&P, w, &v, &dv);
    w = csub(w, cdiv(v, dv));
    if (!cfinite(w)) return -2;
  }
  split_real(w.re, &out4[0], &out4[1]);
  split_real(w.im, &out4[2], &out4[3]);
  *disp = (double)cabs_(csub(w, c0));
  return 0;
}

/* or_polish over a list: points c4[count][4]; out4[count][4] the polished
   points (or NULL), disp[count] the distances |result - c|, last[count]
   the size of the last Newton step (quadratic convergence leaves it at the
   rounding floor).  A point whose iterate is not finite gets disp = +inf.
   Returns the number of such points. */
long or_polish_many(int kind, int l, int n, const double* c4, long count, int steps, double* out4,
                    double* disp, double* last) {
  poly P;
  if (poly_init(&P, kind, l, n)) return -1;
  long bad = 0;
  for (long i = 0; i < count; ++i) {
    cplx c0 = cx(join_real(c4[4 * i], c4[4 * i + 1]), join_real(c4[4 * i + 2], c4[4 * i + 3]));
    cplx w = c0;
    real s = 0;
    int ok = 1;
    for (int k = 0; k < steps; ++k) {
      cplx v, dv;
      eval_P(&P, w, &v, &dv);
      cplx step = cdiv(v, dv);
      w = csub(w, step);
      s = cabs_(step);
      if (!cfinite(w)) { ok = 0; break; }
    }
    if (!ok) {
      disp[i] = HUGE_VAL;
      last[i] = HUGE_VAL;
      ++bad;
      continue;
    }
    if (out4) {
      split_real(w.re, &out4[4 * i + 0], &out4[4 * i + 1]);
      split_real(w.im, &out4[4 * i + 2], &out4[4 * i + 3]);
    }
    disp[i] = (double)cabs_(csub(w, c0));
    last[i] = (double)s;
  }
  return bad;
}

/* Type of one point (see classify).  tau <= 0 selects the default. */
int or_classify(int kind, int l, int n, const double* c4, double tau, int* a, int* b) {
  poly P;
  if (poly_init(&P, kind, l, n)) return -1;
  cplx c = cx(join_real(c4[0], c4[1]), join_real(c4[2], c4[3]));
  classify(&P, c, tau > 0 ? (real)tau : R_TOL_CLASS, a, b);
  return 0;
}

/* Number of roots of P inside the open disk D(c, r), counted from a root
   list (the plain definition a certification claim is checked against). */
long or_count_in_disk(const double* roots4, long nroots, const double* c4, double r) {
  cplx c = cx(join_real(c4[0], c4[1]), join_real(c4[2], c4[3]));
  long k = 0;
  for (long i = 0; i < nroots; ++i) {
    cplx z = cx(join_real(roots4[4 * i + 0], roots4[4 * i + 1]),
                join_real(roots4[4 * i + 2], roots4[4 * i + 3]));
    if (cabs_(csub(z, c)) < (real)r) ++k;
  }
  return k;
}

int or_precision_bits(void) {
#if defined(ORACLE_FP64)
  return 53;
#else
  return 113;
#endif
}

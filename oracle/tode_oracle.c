/*
 * tode_oracle.c -- plain, slow FP64 CPU oracle for batched adaptive explicit
 * Runge-Kutta 5(4) solving (Dormand-Prince, and Tsitouras as the second
 * pair) with fully independent per-instance solver state.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the package's smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA path: every constant below is written out here independently.
 *
 * What it follows (torchode paper):
 *   - Sec. 3 "Design & Features": every instance of the batch keeps its own
 *     initial condition, integration bounds, step size, tolerances and
 *     accept/reject decisions; nothing couples instances.
 *   - Sec. 3, paragraph "What makes torchode fast?": FSAL/SSAL reuse of stage
 *     values, dense output polynomials evaluated by Horner's rule.
 *   - Sec. 3, paragraph "What slows torchode down?": every instance passes its
 *     own evaluation points at its own pace.
 *   - App. A: dopri5 (Dormand & Prince 1980) with an integral controller;
 *     tsit5 (Tsitouras 2011), which App. A names as also available, as the
 *     second pair, swapped in by tableau only (orc_opts.method).
 *   - App. C "Impact of PID Control": the controller is a filter over the
 *     last error estimates (Soderlind 2002/2003); the PI subset is used here.
 *   - App. A, FEN benchmark: gradients by backpropagation through the solver
 *     (discretize-then-optimize) -> the discrete adjoint of the fixed-mesh map.
 *   - App. A, CNF benchmark ("torchode-joint"): the continuous adjoint
 *     equation of the whole batch solved jointly, one problem of size
 *     2bf + p (the state integrated back, its adjoint, the shared
 *     parameters' adjoint) -> orc_joint_adjoint over the augmented field
 *     ORC_AUGADJ, with the same single-problem solver.
 *   - integration backward in time (t1 < t0): the same method with negative
 *     steps; the controller acts on |h|, evaluation points run from t0 down
 *     to t1 (a reading: the paper only uses forward integration).
 *   - Sec. 4.1 "Batching ODEs": joint ("stacked") solving, the comparison
 *     semantics of the batching experiment -- n problems of size p handed to
 *     this same single-problem solver as one problem of size np (a stacked
 *     field, ORC_STACKED), so that they share step size, error norm and
 *     accept/reject decisions.
 *
 * Readings of passages the paper leaves open (it prints no tableau, norm,
 * controller constants, starting-step rule or interpolant):
 *   - tableau: Dormand & Prince 1980, "A family of embedded Runge-Kutta
 *     formulae", the 5(4) pair with FSAL; for tsit5, the table and the
 *     order-4 continuous extension published by Tsitouras (2011), decimals
 *     as printed there (pinned by the order conditions to their rounding);
 *   - dense output: the 4th-order continuous extension of that pair given by
 *     Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.6, expanded into one
 *     quartic polynomial b_i(theta) per stage and evaluated by Horner's rule;
 *   - error norm: the weighted RMS norm of HNW Sec. II.4, per instance;
 *   - controller: factor = safety * err^-beta1 * err_prev^beta2 *
 *     err_prev2^-beta3, clamped (App. C: a PID controller looks at the last
 *     three error estimates; beta3 = beta2 = 0 is the I controller);
 *   - powers err^-beta: a fixed exp/log procedure (orc_pow) so that every
 *     IEEE machine running it reproduces the controller's step sizes;
 *   - starting step: the heuristic of HNW Sec. II.4 ("starting step size"),
 *     with the probe evaluation taken in the direction of integration (the
 *     paper gives no starting-step rule; the tests pin this one against its
 *     closed form on diagonal linear systems and an exact rational
 *     evaluation on Van der Pol, every branch of it deciding once).
 *
 * Arithmetic: double everywhere, built with -O2 -ffp-contract=off and no
 * fast-math, sums taken left to right in the order written.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <sched.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------ */
/* Dormand-Prince 5(4) tableau (Dormand & Prince 1980; dopri5 in App. A).    */
/* ------------------------------------------------------------------------ */
#define NS 7

static const double DP_C[NS] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};

static const double DP_A[NS][NS] = {
    {0, 0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0}};

/* 5th-order weights: identical to the last stage row (FSAL/SSAL, Sec. 3). */
static const double DP_B[NS] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0,
                                -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
/* embedded 4th-order weights */
static const double DP_BHAT[NS] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                   -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

/* Dense output: b_i(theta) = theta*(q0 + theta*(q1 + theta*(q2 + theta*q3))).
 * These are the expanded coefficients of the HNW Sec. II.6 continuous
 * extension of the pair above, one exact rational each. */
static const double DP_Q[NS][4] = {
    {1.0, -8048581381.0 / 2820520608.0, 8663915743.0 / 2820520608.0,
     -12715105075.0 / 11282082432.0},
    {0.0, 0.0, 0.0, 0.0},
    {0.0, 131558114200.0 / 32700410799.0, -68118460800.0 / 10900136933.0,
     87487479700.0 / 32700410799.0},
    {0.0, -1754552775.0 / 470086768.0, 14199869525.0 / 1410260304.0,
     -10690763975.0 / 1880347072.0},
    {0.0, 127303824393.0 / 49829197408.0, -318862633887.0 / 49829197408.0,
     701980252875.0 / 199316789632.0},
    {0.0, -282668133.0 / 205662961.0, 2019193451.0 / 616988883.0,
     -1453857185.0 / 822651844.0},
    {0.0, 40617522.0 / 29380423.0, -110615467.0 / 29380423.0, 69997945.0 / 29380423.0}};

/* ------------------------------------------------------------------------ */
/* Tsitouras 5(4) pair ("tsit5", named in App. A as available in torchode   */
/* and often recommended over dopri5): Ch. Tsitouras, Runge-Kutta pairs of   */
/* order 5(4) satisfying only the first column simplifying assumption,       */
/* Comput. Math. Appl. 62 (2011), the pair's table and its continuous        */
/* extension of order 4.  The decimals as published; FSAL (a7 = b, b7 = 0).  */
/* ------------------------------------------------------------------------ */
static const double TS_C[NS] = {0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0};

static const double TS_A[NS][NS] = {
    {0, 0, 0, 0, 0, 0, 0},
    {0.161, 0, 0, 0, 0, 0, 0},
    {-0.008480655492356989, 0.335480655492357, 0, 0, 0, 0, 0},
    {2.897153057105493, -6.359448489975075, 4.3622954328695815, 0, 0, 0, 0},
    {5.325864828439257, -11.748883564062828, 7.4955393428898365, -0.09249506636175525, 0, 0, 0},
    {5.86145544294642, -12.92096931784711, 8.159367898576159, -0.071584973281401,
     -0.028269050394068383, 0, 0},
    {0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742, -3.290069515436081,
     2.324710524099774, 0}};

/* error weights: the difference of the 5th- and 4th-order weight rows */
static const double TS_E[NS] = {-0.00178001105222577714, -0.0008164344596567469,
                                0.007880878010261995,    -0.1447110071732629,
                                0.5823571654525552,      -0.45808210592918697,
                                0.015151515151515152};

/* Continuous extension, b_i(theta) = k_i theta^m_i * (product of the listed
 * monic factors): m_1 = 1 with the factors (theta - r) and (theta^2 + p theta
 * + s); m_i = 2 for i >= 2 with one quadratic or two linear factors.  Each
 * factor is given by its coefficients, highest power first. */
typedef struct {
  double k;
  int m;
  int nf;
  int deg[2];
  double f[2][3];
} ts_dense_factored;

static const ts_dense_factored TS_BT[NS] = {
    {-1.0530884977290216, 1, 2, {1, 2},
     {{1.0, -1.3299890189751412, 0.0}, {1.0, -1.4364028541716351, 0.7139816917074209}}},
    {0.1017, 2, 1, {2, 0}, {{1.0, -2.1966568338249754, 1.2949852507374631}, {0, 0, 0}}},
    {2.490627285651252793, 2, 1, {2, 0}, {{1.0, -2.38535645472061657, 1.57803468208092486}, {0, 0, 0}}},
    {-16.54810288924490272, 2, 2, {1, 1}, {{1.0, -1.21712927295533244, 0}, {1.0, -0.61620406037800089, 0}}},
    {47.37952196281928122, 2, 2, {1, 1}, {{1.0, -1.203071208372362603, 0}, {1.0, -0.658047292653547382, 0}}},
    {-34.87065786149660974, 2, 2, {1, 1}, {{1.0, -1.2, 0}, {1.0, -0.666666666666666667, 0}}},
    {2.5, 2, 2, {1, 1}, {{1.0, -1.0, 0}, {1.0, -0.6, 0}}}};

/* One method's coefficients as the solver uses them. */
typedef struct {
  double c[NS];
  double a[NS][NS];
  double b[NS];
  double e[NS];    /* b_i - bhat_i */
  double q[NS][4]; /* b_i(theta) = theta*(q0 + theta*(q1 + theta*(q2 + theta*q3))) */
} rk_tab;

static rk_tab TAB[2];
static pthread_once_t TAB_ONCE = PTHREAD_ONCE_INIT;

/* Multiplies out k theta^m prod(factors) into monomial coefficients
 * (plain polynomial products, lowest power first). */
static void ts_expand(const ts_dense_factored *d, double *out /*[5]: theta^0..theta^4*/) {
  double p[5] = {0, 0, 0, 0, 0};
  p[d->m] = d->k; /* k theta^m */
  int deg = d->m;
  for (int f = 0; f < d->nf; ++f) {
    double r[5] = {0, 0, 0, 0, 0};
    const int df = d->deg[f];
    for (int u = 0; u <= deg; ++u)
      for (int v = 0; v <= df; ++v) r[u + v] = r[u + v] + p[u] * d->f[f][df - v];
    deg += df;
    for (int u = 0; u < 5; ++u) p[u] = r[u];
  }
  for (int u = 0; u < 5; ++u) out[u] = p[u];
}

static void tab_init(void) {
  for (int i = 0; i < NS; ++i) {
    TAB[0].c[i] = DP_C[i];
    TAB[0].b[i] = DP_B[i];
    TAB[0].e[i] = DP_B[i] - DP_BHAT[i];
    for (int j = 0; j < NS; ++j) TAB[0].a[i][j] = DP_A[i][j];
    for (int j = 0; j < 4; ++j) TAB[0].q[i][j] = DP_Q[i][j];
    TAB[1].c[i] = TS_C[i];
    TAB[1].b[i] = TS_A[NS - 1][i];
    TAB[1].e[i] = TS_E[i];
    for (int j = 0; j < NS; ++j) TAB[1].a[i][j] = TS_A[i][j];
    double m[5];
    ts_expand(&TS_BT[i], m); /* m[0] = 0: every b_i(theta) has a factor theta */
    for (int j = 0; j < 4; ++j) TAB[1].q[i][j] = m[j + 1];
  }
}

/* ORC_DOPRI5 = 0, ORC_TSIT5 = 1 */
static const rk_tab *tab_of(int method) {
  pthread_once(&TAB_ONCE, tab_init);
  return &TAB[method == 1 ? 1 : 0];
}

/* For the tests: one method's coefficients (e = b - bhat, q as above). */
void orc_tableau_m(int method, double *c, double *a, double *b, double *e, double *q) {
  const rk_tab *T = tab_of(method);
  for (int i = 0; i < NS; ++i) {
    c[i] = T->c[i];
    b[i] = T->b[i];
    e[i] = T->e[i];
    for (int j = 0; j < NS; ++j) a[i * NS + j] = T->a[i][j];
    for (int j = 0; j < 4; ++j) q[i * 4 + j] = T->q[i][j];
  }
}

/* Lets tests compare these doubles with an exact rational table. */
void orc_tableau(double *c, double *a, double *b, double *bhat, double *q) {
  for (int i = 0; i < NS; ++i) {
    c[i] = DP_C[i];
    b[i] = DP_B[i];
    bhat[i] = DP_BHAT[i];
    for (int j = 0; j < NS; ++j) a[i * NS + j] = DP_A[i][j];
    for (int j = 0; j < 4; ++j) q[i * 4 + j] = DP_Q[i][j];
  }
}

/* ------------------------------------------------------------------------ */
/* Problem description.                                                      */
/* ------------------------------------------------------------------------ */
enum { ORC_VDP = 1, ORC_LINEAR = 2, ORC_MLP = 3, ORC_STACKED = 4, ORC_AUGADJ = 5 };
enum { ST_SUCCESS = 0, ST_MAX_STEPS = 1, ST_DT_UNDERFLOW = 2, ST_NONFINITE = 3,
       ST_INVALID_INPUT = 4, ST_RUNNING = -1 };

#define MLP_MAX_LAYERS 8

typedef struct orc_field_s {
  int kind;
  int D;
  const double *mu;          /* Van der Pol: [B] damping */
  const double *A;           /* linear: [B][D][D] row-major */
  int n_layers;              /* MLP: number of weight matrices */
  const int *widths;         /* MLP: [n_layers+1]; widths[0]=D+1, widths[n_layers]=D */
  const double *const *W;    /* MLP: W[l] is [widths[l+1]][widths[l]] row-major */
  const double *const *bias; /* MLP: bias[l] is [widths[l+1]] */
  /* Stacked: n_inner instances of `inner` concatenated into one problem of
   * size D = n_inner * inner->D (Sec. 4.1: a mini-batch of n problems of
   * size p solved as a single problem of size np); block b of the state is
   * instance b of the inner field. */
  const struct orc_field_s *inner;
  int n_inner;
  /* ORC_AUGADJ: the augmented adjoint system of n_inner instances of the MLP
   * field `inner` (orc_joint_adjoint builds it; scr is its scratch) */
  double *scr;
} orc_field;

typedef struct {
  double rtol, atol;
  const double *rtol_b, *atol_b; /* optional per-instance tolerances [B], NULL = scalar */
  double safety, fac_min, fac_max, beta1, beta2;
  double h0;                     /* > 0: first step given; 0: starting-step heuristic */
  int max_steps;                 /* attempted steps per instance */
  double beta3;                  /* derivative term: exponent of err_prev2 (App. C) */
  int method;                    /* 0 dopri5, 1 tsit5 (App. A) */
} orc_opts;

typedef struct {
  int cap;          /* attempts recorded per instance */
  double *t, *h, *err;
  int32_t *accepted; /* all [B][cap] */
  int32_t *len;      /* [B]: attempts recorded */
} orc_trace;

static int mlp_max_width(const orc_field *F) {
  int m = 0;
  for (int l = 0; l <= F->n_layers; ++l)
    if (F->widths[l] > m) m = F->widths[l];
  return m;
}

/* ------------------------------------------------------------------------ */
/* Vector fields f(t, y) for instance i.                                     */
/* ------------------------------------------------------------------------ */

/* Van der Pol, Eq. 1 written as a first-order system:
 * y1' = y2,  y2' = mu (1 - y1^2) y2 - y1. */
static void f_vdp(double mu, const double *y, double *out) {
  out[0] = y[1];
  out[1] = mu * (1.0 - y[0] * y[0]) * y[1] - y[0];
}

/* y' = A_i y, A_i row-major. */
static void f_linear(const double *A, int D, const double *y, double *out) {
  for (int r = 0; r < D; ++r) {
    double s = 0.0;
    for (int c = 0; c < D; ++c) s = s + A[r * D + c] * y[c];
    out[r] = s;
  }
}

/* MLP field f(t,y) = W_L tanh( ... tanh(W_1 [y; t] + b_1) ... ) + b_L.
 * act (optional) receives the input of every layer: act[l] has widths[l]
 * entries, act[0] = [y; t]; it needs sum(widths) doubles. */
static void f_mlp(const orc_field *F, double t, const double *y, double *out, double *act) {
  const int L = F->n_layers, D = F->D;
  double *a = act; /* act[0] */
  for (int j = 0; j < D; ++j) a[j] = y[j];
  a[D] = t;
  for (int l = 0; l < L; ++l) {
    const int nin = F->widths[l], nout = F->widths[l + 1];
    const double *W = F->W[l], *bv = F->bias[l];
    double *next = (l + 1 < L) ? a + nin : out;
    for (int r = 0; r < nout; ++r) {
      double s = 0.0;
      for (int c = 0; c < nin; ++c) s = s + W[r * nin + c] * a[c];
      s = s + bv[r];
      next[r] = (l + 1 < L) ? tanh(s) : s;
    }
    a = next;
  }
}

typedef struct {
  const orc_field *F;
  int i;        /* instance index */
  double *act;  /* MLP scratch */
  long nfe;     /* evaluations */
} fctx;

static void aug_eval(const orc_field *F, double t, const double *z, double *out);

static void feval(fctx *c, double t, const double *y, double *out) {
  const orc_field *F = c->F;
  c->nfe++;
  if (F->kind == ORC_AUGADJ) {
    aug_eval(F, t, y, out);
  } else if (F->kind == ORC_VDP) {
    f_vdp(F->mu[c->i], y, out);
  } else if (F->kind == ORC_LINEAR) {
    f_linear(F->A + (size_t)c->i * F->D * F->D, F->D, y, out);
  } else if (F->kind == ORC_STACKED) {
    /* the concatenated field: every block evolves by its own instance's f */
    const int d = F->inner->D;
    for (int b = 0; b < F->n_inner; ++b) {
      fctx sub = {F->inner, b, c->act, 0};
      feval(&sub, t, y + (size_t)b * d, out + (size_t)b * d);
    }
  } else {
    f_mlp(F, t, y, out, c->act);
  }
}

/* Exported single evaluation (tests pin the fields with it). */
void orc_field_eval(const orc_field *F, int i, double t, const double *y, double *out) {
  fctx c = {F, i, NULL, 0};
  double *act = NULL;
  const orc_field *M = F->kind == ORC_STACKED ? F->inner : F;
  if (M->kind == ORC_MLP) {
    int tot = 0;
    for (int l = 0; l <= M->n_layers; ++l) tot += M->widths[l];
    act = (double *)malloc(sizeof(double) * tot);
    c.act = act;
  }
  feval(&c, t, y, out);
  free(act);
}

/* ------------------------------------------------------------------------ */
/* Norm, starting step, controller.                                          */
/* ------------------------------------------------------------------------ */

/* Weighted RMS norm of v with weights sc (HNW Sec. II.4), taken per instance
 * (Sec. 3 / Sec. 4.1: never across the batch). */
static double rms(const double *v, const double *sc, int D) {
  double s = 0.0;
  for (int j = 0; j < D; ++j) {
    double q = v[j] / sc[j];
    s = s + q * q;
  }
  return sqrt(s / (double)D);
}

static double dmax(double a, double b) { return (a > b) ? a : b; }
static double dmin(double a, double b) { return (b < a) ? b : a; }

/* x^y for the step-size controller and the starting step, evaluated as
 * exp(y ln x) by a fully specified sequence of IEEE-754 double operations:
 *   ln x: x = 2^e m with m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),
 *         ln m = 2 (s + s^3/3 + ... + s^23/23) (Horner in s^2),
 *         ln x = e ln2_hi + (e ln2_lo + ln m)  (ln 2 split after 32 bits);
 *   exp z: k = floor(z / ln2 + 1/2), r = (z - k ln2_hi) - k ln2_lo,
 *         exp r = sum_{j<=14} r^j / j! (Horner), times 2^k exactly.
 * Platform pow implementations may differ by an ulp, and the embedded error
 * estimate (a difference of nearly equal stage sums) amplifies such a
 * difference about 1e4-fold; with this procedure any IEEE machine that runs
 * the same operations in the same order gets the same bits. */
static const double CTL_LN2_HI = 0x1.62e42fee00000p-1;
static const double CTL_LN2_LO = 0x1.a39ef35793c76p-33;
static const double CTL_INV_LN2 = 0x1.71547652b82fep+0;
static const double CTL_SQRT2 = 0x1.6a09e667f3bcdp+0;

static double ctl_ln(double x) {
  uint64_t u;
  memcpy(&u, &x, 8);
  int e = (int)((u >> 52) & 0x7ff);
  if (e == 0) { /* subnormal: scale by 2^54 exactly */
    x = x * 18014398509481984.0;
    memcpy(&u, &x, 8);
    e = (int)((u >> 52) & 0x7ff) - 54;
  }
  e -= 1023;
  u = (u & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
  double m;
  memcpy(&m, &u, 8);
  if (m > CTL_SQRT2) {
    m = m * 0.5;
    e = e + 1;
  }
  double s = (m - 1.0) / (m + 1.0);
  double w = s * s;
  double p = 1.0 / 23.0;
  p = 1.0 / 21.0 + w * p;
  p = 1.0 / 19.0 + w * p;
  p = 1.0 / 17.0 + w * p;
  p = 1.0 / 15.0 + w * p;
  p = 1.0 / 13.0 + w * p;
  p = 1.0 / 11.0 + w * p;
  p = 1.0 / 9.0 + w * p;
  p = 1.0 / 7.0 + w * p;
  p = 1.0 / 5.0 + w * p;
  p = 1.0 / 3.0 + w * p;
  p = 1.0 + w * p;
  double lnm = 2.0 * (s * p);
  double de = (double)e;
  return de * CTL_LN2_HI + (de * CTL_LN2_LO + lnm);
}

static double ctl_exp(double z) {
  if (z > 700.0) return INFINITY;
  if (z < -700.0) return 0.0;
  double k = floor(z * CTL_INV_LN2 + 0.5);
  double r = (z - k * CTL_LN2_HI) - k * CTL_LN2_LO;
  double p = 1.0 / 87178291200.0;           /* 1/14! */
  p = 1.0 / 6227020800.0 + r * p;           /* 1/13! */
  p = 1.0 / 479001600.0 + r * p;
  p = 1.0 / 39916800.0 + r * p;
  p = 1.0 / 3628800.0 + r * p;
  p = 1.0 / 362880.0 + r * p;
  p = 1.0 / 40320.0 + r * p;
  p = 1.0 / 5040.0 + r * p;
  p = 1.0 / 720.0 + r * p;
  p = 1.0 / 120.0 + r * p;
  p = 1.0 / 24.0 + r * p;
  p = 1.0 / 6.0 + r * p;
  p = 0.5 + r * p;
  p = 1.0 + r * p;
  p = 1.0 + r * p;
  uint64_t b = (uint64_t)((int64_t)k + 1023) << 52;
  double two_k;
  memcpy(&two_k, &b, 8);
  return p * two_k;
}

double orc_pow(double x, double y) {
  if (x != x || y != y || x < 0.0) return NAN;
  if (x == 0.0) return (y > 0.0) ? 0.0 : INFINITY;
  if (isinf(x)) return (y > 0.0) ? INFINITY : 0.0;
  if (x == 1.0 || y == 0.0) return 1.0;
  return ctl_exp(y * ctl_ln(x));
}

/* Starting step size, HNW Sec. II.4 (pinned by the tests, see header).  f0 =
 * f(t0, y0) is supplied and reused as the first step's k1 (FSAL). */
/* Magnitude of the first step; the trial step goes in the direction dir of
 * integration (+1 forward, -1 from t0 down to t1). */
static double starting_step(fctx *c, double t0, double t1, double dir, const double *y0,
                            const double *f0, int D, double rtol, double atol, double *w1,
                            double *w2, double *sc) {
  for (int j = 0; j < D; ++j) sc[j] = atol + rtol * fabs(y0[j]);
  double d0 = rms(y0, sc, D);
  double d1 = rms(f0, sc, D);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * (d0 / d1);
  for (int j = 0; j < D; ++j) w1[j] = y0[j] + (dir * h0) * f0[j];
  feval(c, t0 + dir * h0, w1, w2);
  for (int j = 0; j < D; ++j) w2[j] = w2[j] - f0[j];
  double d2 = rms(w2, sc, D) / h0;
  double m = (d1 > d2) ? d1 : d2;
  double h1 = (m <= 1e-15) ? dmax(1e-6, h0 * 1e-3) : orc_pow(0.01 / m, 1.0 / 5.0);
  double h = dmin(100.0 * h0, h1);
  h = dmin(h, dir * (t1 - t0));
  if (!(h > 0.0 && isfinite(h))) h = dir * (t1 - t0);
  return h;
}

/* ------------------------------------------------------------------------ */
/* One step of the pair T from (t, y) with step h; k[0] holds f(t, y) on    */
/* entry (FSAL).  Fills k[1..6], Y (stage inputs, Y[6] = y1 by SSAL).        */
/* ------------------------------------------------------------------------ */
static void dp_stages(const rk_tab *T, fctx *c, double t, double h, const double *y, int D,
                      double *k /*[7][D]*/, double *Y /*[7][D]*/) {
  for (int j = 0; j < D; ++j) Y[j] = y[j];
  for (int i = 1; i < NS; ++i) {
    double *Yi = Y + i * D;
    for (int j = 0; j < D; ++j) {
      double s = 0.0;
      for (int l = 0; l < i; ++l) s = s + T->a[i][l] * k[l * D + j];
      Yi[j] = y[j] + h * s;
    }
    feval(c, t + T->c[i] * h, Yi, k + i * D);
  }
}

/* Embedded error e = h * sum_i (b_i - bhat_i) k_i, then its weighted RMS norm
 * against sc = atol + rtol * max(|y|, |y1|). */
static double dp_error(const rk_tab *T, double h, const double *y, const double *y1,
                       const double *k, int D, double rtol, double atol, double *e, double *sc) {
  for (int j = 0; j < D; ++j) {
    double s = 0.0;
    for (int i = 0; i < NS; ++i) s = s + T->e[i] * k[i * D + j];
    e[j] = h * s;
    sc[j] = atol + rtol * dmax(fabs(y[j]), fabs(y1[j]));
  }
  return rms(e, sc, D);
}

/* Dense output at theta in [0,1): y + h * sum_i b_i(theta) k_i, each b_i by
 * Horner's rule (Sec. 3, "What makes torchode fast?"). */
static void dp_dense(const rk_tab *T, double theta, double h, const double *y, const double *k,
                     int D, double *out) {
  double bt[NS];
  for (int i = 0; i < NS; ++i) {
    const double *q = T->q[i];
    bt[i] = theta * (q[0] + theta * (q[1] + theta * (q[2] + theta * q[3])));
  }
  for (int j = 0; j < D; ++j) {
    double s = 0.0;
    for (int i = 0; i < NS; ++i) s = s + bt[i] * k[i * D + j];
    out[j] = y[j] + h * s;
  }
}

/* Exported: dense-output weights b_i(theta), for the tests. */
/* d/dt of the dense output y + hs sum_i b_i(theta) k_i with theta = (t -
 * t_n) / hs: sum_i b_i'(theta) k_i, b_i'(theta) = q0 + 2 q1 theta + 3 q2
 * theta^2 + 4 q3 theta^3 from the same quartics (the step's sign cancels). */
static void dp_dense_deriv(const rk_tab *T, double theta, const double *k, int D, double *out) {
  double bd[NS];
  for (int i = 0; i < NS; ++i) {
    const double *q = T->q[i];
    bd[i] = q[0] + theta * (2.0 * q[1] + theta * (3.0 * q[2] + theta * (4.0 * q[3])));
  }
  for (int j = 0; j < D; ++j) {
    double s = 0.0;
    for (int i = 0; i < NS; ++i) s = s + bd[i] * k[i * D + j];
    out[j] = s;
  }
}

static void dense_weights(const rk_tab *T, double theta, double *bt) {
  for (int i = 0; i < NS; ++i) {
    const double *q = T->q[i];
    bt[i] = theta * (q[0] + theta * (q[1] + theta * (q[2] + theta * q[3])));
  }
}
void orc_dense_weights_m(int method, double theta, double *bt) {
  dense_weights(tab_of(method), theta, bt);
}
void orc_dense_weights(double theta, double *bt) { dense_weights(tab_of(0), theta, bt); }

/* ------------------------------------------------------------------------ */
/* Input checks (Sec. 3: per-instance bounds and evaluation points).         */
/* ------------------------------------------------------------------------ */
/* Finite times; evaluation points between t0 and t1 and ordered in the
 * direction of integration (t1 < t0 integrates backward in time). */
static int instance_inputs_valid(double t0, double t1, const double *te, int K) {
  if (!isfinite(t0) || !isfinite(t1)) return 0;
  const double dir = (t1 < t0) ? -1.0 : 1.0;
  for (int q = 0; q < K; ++q) {
    if (!isfinite(te[q]) || dir * te[q] < dir * t0 || dir * te[q] > dir * t1) return 0;
    if (q > 0 && dir * te[q] < dir * te[q - 1]) return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Adaptive solve of one instance (Sec. 3; App. A: dopri5 + I controller).   */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_field *F;
  const orc_opts *O;
  const rk_tab *T; /* the pair (dopri5 or tsit5) */
  int B, K;
  const double *y0, *t0, *t1, *t_eval;
  double *y_eval, *y_final;
  double *yp_eval; /* optional: dy/dt of the dense output at every evaluation point */
  int32_t *n_acc, *n_rej, *n_feval, *status;
  const orc_trace *trace;
  /* replay / adjoint */
  const double *mesh_t, *mesh_h;
  const int32_t *mesh_n;
  int mesh_cap;
  const double *gy_eval, *gy_final;
  double *gy0, *gparam; /* gparam: VdP [B], linear [B][D][D] */
  double *gt0, *gt1;    /* optional: dL/dt0, dL/dt1 [B] */
  double **gW_part, **gb_part; /* MLP per-thread partial sums */
  /* threading */
  int nthreads;
} job;

static void fill_nan(double *p, size_t n) {
  for (size_t j = 0; j < n; ++j) p[j] = NAN;
}

static void solve_one(const job *J, int i, double *work, double *act) {
  const orc_field *F = J->F;
  const orc_opts *O = J->O;
  const int D = F->D, K = J->K;
  const double rtol = O->rtol_b ? O->rtol_b[i] : O->rtol;
  const double atol = O->atol_b ? O->atol_b[i] : O->atol;
  const double t0 = J->t0[i], t1 = J->t1[i];
  const double *te = J->t_eval + (size_t)i * K;
  double *ye = J->y_eval + (size_t)i * K * D;
  double *yp = J->yp_eval ? J->yp_eval + (size_t)i * K * D : NULL;
  double *yf = J->y_final + (size_t)i * D;
  double *y = work, *y1 = y + D, *k = y1 + D, *Y = k + NS * D, *e = Y + NS * D, *sc = e + D,
         *w1 = sc + D, *w2 = w1 + D;
  fctx c = {F, i, act, 0};
  int n_acc = 0, n_rej = 0, st = ST_RUNNING, tr = 0;

  fill_nan(ye, (size_t)K * D);
  if (yp) fill_nan(yp, (size_t)K * D);
  if (!instance_inputs_valid(t0, t1, te, K)) {
    fill_nan(yf, D);
    J->n_acc[i] = J->n_rej[i] = J->n_feval[i] = 0;
    J->status[i] = ST_INVALID_INPUT;
    if (J->trace) J->trace->len[i] = 0;
    return;
  }
  for (int j = 0; j < D; ++j) y[j] = J->y0[(size_t)i * D + j];

  /* evaluation points at t0 take y0 itself */
  int cur = 0;
  while (cur < K && te[cur] == t0) {
    for (int j = 0; j < D; ++j) ye[(size_t)cur * D + j] = y[j];
    cur++;
  }
  if (yp && cur > 0) { /* the derivative at t0 is f(t0, y0) (not counted) */
    fctx c0 = {F, i, act, 0};
    feval(&c0, t0, y, w1);
    for (int q = 0; q < cur; ++q)
      for (int j = 0; j < D; ++j) yp[(size_t)q * D + j] = w1[j];
  }
  if (t1 == t0) {
    for (int j = 0; j < D; ++j) yf[j] = y[j];
    J->n_acc[i] = J->n_rej[i] = J->n_feval[i] = 0;
    J->status[i] = ST_SUCCESS;
    if (J->trace) J->trace->len[i] = 0;
    return;
  }

  /* backward in time when t1 < t0: the same method with negative steps
   * hs = dir * h; h, the controller's quantity, stays positive */
  const double dir = (t1 < t0) ? -1.0 : 1.0;
  double t = t0;
  feval(&c, t, y, k); /* k1 = f(t0, y0) */
  double h = (O->h0 > 0.0) ? O->h0
                           : starting_step(&c, t0, t1, dir, y, k, D, rtol, atol, w1, w2, sc);
  double err_prev = 1.0, err_prev2 = 1.0; /* the last two accepted steps' errors */
  int prev_rejected = 0;

  while (st == ST_RUNNING) {
    int last = 0;
    if (dir * (t + dir * h) >= dir * t1) {
      h = dir * (t1 - t);
      last = 1;
    }
    const double hs = dir * h;
    dp_stages(J->T, &c, t, hs, y, D, k, Y);
    for (int j = 0; j < D; ++j) y1[j] = Y[6 * D + j]; /* SSAL: y1 is the last stage input */
    double err = dp_error(J->T, hs, y, y1, k, D, rtol, atol, e, sc);
    int finite = isfinite(err);
    for (int j = 0; j < D; ++j) finite = finite && isfinite(y1[j]);
    int accept = finite && err <= 1.0;

    if (J->trace && tr < J->trace->cap) {
      size_t o = (size_t)i * J->trace->cap + tr;
      J->trace->t[o] = t;
      J->trace->h[o] = hs;
      J->trace->err[o] = err;
      J->trace->accepted[o] = accept;
      tr++;
    }

    double h_next;
    if (accept) {
      double t_next = last ? t1 : t + hs;
      /* dense output for every evaluation point in (t, t_next] */
      while (cur < K && dir * te[cur] <= dir * t_next) {
        double *o = ye + (size_t)cur * D;
        if (te[cur] == t_next) {
          for (int j = 0; j < D; ++j) o[j] = y1[j];
        } else {
          dp_dense(J->T, (te[cur] - t) / hs, hs, y, k, D, o);
        }
        if (yp) /* the interpolant's derivative; theta = 1 at the step's end */
          dp_dense_deriv(J->T, te[cur] == t_next ? 1.0 : (te[cur] - t) / hs, k, D,
                         yp + (size_t)cur * D);
        cur++;
      }
      /* controller: factor = safety * err^-beta1 * err_prev^beta2 * err_prev2^-beta3 */
      double fac;
      if (err == 0.0) {
        fac = O->fac_max;
      } else {
        fac = O->safety * orc_pow(err, -O->beta1);
        if (O->beta2 != 0.0) fac = fac * orc_pow(err_prev, O->beta2);
        if (O->beta3 != 0.0) fac = fac * orc_pow(err_prev2, -O->beta3);
      }
      fac = dmin(dmax(fac, O->fac_min), O->fac_max);
      if (prev_rejected) fac = dmin(fac, 1.0);
      h_next = h * fac;
      err_prev2 = err_prev;
      err_prev = dmax(err, 1e-4);
      prev_rejected = 0;
      n_acc++;
      t = t_next;
      for (int j = 0; j < D; ++j) {
        y[j] = y1[j];
        k[j] = k[6 * D + j]; /* FSAL */
      }
      if (last) st = ST_SUCCESS;
    } else {
      double fac = finite ? dmin(dmax(O->safety * orc_pow(err, -O->beta1), O->fac_min), 1.0)
                          : O->fac_min;
      h_next = h * fac;
      prev_rejected = 1;
      n_rej++;
    }
    h = h_next;
    if (st == ST_RUNNING) {
      double scale = dmax(fabs(t), fabs(t1));
      if (t + dir * h == t || h < 1e-14 * scale || !(h > 0.0))
        st = finite ? ST_DT_UNDERFLOW : ST_NONFINITE;
      else if (n_acc + n_rej >= O->max_steps)
        st = ST_MAX_STEPS;
    }
  }
  for (int j = 0; j < D; ++j) yf[j] = y[j];
  J->n_acc[i] = n_acc;
  J->n_rej[i] = n_rej;
  J->n_feval[i] = (int32_t)c.nfe;
  J->status[i] = st;
  if (J->trace) J->trace->len[i] = tr;
}

/* ------------------------------------------------------------------------ */
/* Fixed-mesh replay (no controller): the map whose discrete adjoint the     */
/* gradient is.  mesh_t[i][n], mesh_h[i][n] for n < mesh_n[i]; the last step */
/* ends at t1[i].  Also returns every step-start state when ys != NULL.      */
/* ------------------------------------------------------------------------ */
static double mesh_end(const job *J, int i, int n) {
  const int N = J->mesh_n[i];
  return (n + 1 < N) ? J->mesh_t[(size_t)i * J->mesh_cap + n + 1] : J->t1[i];
}

static void replay_one(const job *J, int i, double *work, double *act, double *ys /*[N+1][D]*/) {
  const orc_field *F = J->F;
  const int D = F->D, K = J->K, N = J->mesh_n[i];
  const double t0 = J->t0[i];
  const double dir = (J->t1[i] < t0) ? -1.0 : 1.0; /* mesh steps carry this sign */
  const double *te = J->t_eval + (size_t)i * K;
  double *ye = J->y_eval + (size_t)i * K * D;
  double *yp = J->yp_eval ? J->yp_eval + (size_t)i * K * D : NULL;
  double *y = work, *k = y + D, *Y = k + NS * D;
  fctx c = {F, i, act, 0};
  for (int j = 0; j < D; ++j) y[j] = J->y0[(size_t)i * D + j];
  fill_nan(ye, (size_t)K * D);
  if (yp) fill_nan(yp, (size_t)K * D);
  int cur = 0;
  while (cur < K && te[cur] == t0) {
    for (int j = 0; j < D; ++j) ye[(size_t)cur * D + j] = y[j];
    cur++;
  }
  if (yp && cur > 0) { /* the derivative at t0 is f(t0, y0) */
    feval(&c, t0, y, k);
    for (int q = 0; q < cur; ++q)
      for (int j = 0; j < D; ++j) yp[(size_t)q * D + j] = k[j];
  }
  if (ys)
    for (int j = 0; j < D; ++j) ys[j] = y[j];
  for (int n = 0; n < N; ++n) {
    const double t = J->mesh_t[(size_t)i * J->mesh_cap + n];
    const double h = J->mesh_h[(size_t)i * J->mesh_cap + n];
    const double t_next = mesh_end(J, i, n);
    feval(&c, t, y, k);
    dp_stages(J->T, &c, t, h, y, D, k, Y);
    const double *y1 = Y + 6 * D;
    while (cur < K && dir * te[cur] <= dir * t_next) {
      double *o = ye + (size_t)cur * D;
      if (te[cur] == t_next) {
        for (int j = 0; j < D; ++j) o[j] = y1[j];
      } else {
        dp_dense(J->T, (te[cur] - t) / h, h, y, k, D, o);
      }
      if (yp) /* the interpolant's derivative; theta = 1 at the step's end */
        dp_dense_deriv(J->T, te[cur] == t_next ? 1.0 : (te[cur] - t) / h, k, D,
                       yp + (size_t)cur * D);
      cur++;
    }
    for (int j = 0; j < D; ++j) y[j] = y1[j];
    if (ys)
      for (int j = 0; j < D; ++j) ys[(size_t)(n + 1) * D + j] = y[j];
  }
  for (int j = 0; j < D; ++j) J->y_final[(size_t)i * D + j] = y[j];
}

/* ------------------------------------------------------------------------ */
/* Vector-Jacobian products of the fields: gy += J_f(y)^T v, and the         */
/* parameter cotangents.                                                     */
/* ------------------------------------------------------------------------ */
static void vjp(const job *J, int i, double t, const double *y, const double *v, double *gy,
                double *gparam_i, double *gW, double *gb, double *act, double *dscr,
                double *gt) {
  const orc_field *F = J->F;
  const int D = F->D;
  if (F->kind == ORC_VDP) {
    /* J = [[0, 1], [-2 mu y1 y2 - 1, mu (1 - y1^2)]] */
    const double mu = F->mu[i];
    gy[0] = gy[0] + v[1] * (-2.0 * mu * y[0] * y[1] - 1.0);
    gy[1] = gy[1] + (v[0] + v[1] * (mu * (1.0 - y[0] * y[0])));
    gparam_i[0] = gparam_i[0] + v[1] * ((1.0 - y[0] * y[0]) * y[1]);
  } else if (F->kind == ORC_LINEAR) {
    const double *A = F->A + (size_t)i * D * D;
    for (int cidx = 0; cidx < D; ++cidx) {
      double s = 0.0;
      for (int r = 0; r < D; ++r) s = s + A[r * D + cidx] * v[r];
      gy[cidx] = gy[cidx] + s;
    }
    for (int r = 0; r < D; ++r)
      for (int cidx = 0; cidx < D; ++cidx)
        gparam_i[r * D + cidx] = gparam_i[r * D + cidx] + v[r] * y[cidx];
  } else {
    /* forward pass storing every layer input, then backpropagation */
    const int L = F->n_layers;
    double out_dummy[256];
    double *outp = (D <= 256) ? out_dummy : NULL;
    f_mlp(F, t, y, outp, act);
    int off[MLP_MAX_LAYERS + 1];
    off[0] = 0;
    for (int l = 0; l < L; ++l) off[l + 1] = off[l] + F->widths[l];
    int maxw = mlp_max_width(F);
    double *delta = dscr, *ga = dscr + maxw;
    for (int r = 0; r < D; ++r) delta[r] = v[r];
    size_t woff = 0, boff = 0;
    size_t wstart[MLP_MAX_LAYERS], bstart[MLP_MAX_LAYERS];
    for (int l = 0; l < L; ++l) {
      wstart[l] = woff;
      bstart[l] = boff;
      woff += (size_t)F->widths[l] * F->widths[l + 1];
      boff += F->widths[l + 1];
    }
    for (int l = L - 1; l >= 0; --l) {
      const int nin = F->widths[l], nout = F->widths[l + 1];
      const double *a = act + off[l];
      const double *W = F->W[l];
      double *gWl = gW + wstart[l], *gbl = gb + bstart[l];
      for (int r = 0; r < nout; ++r) {
        gbl[r] = gbl[r] + delta[r];
        for (int cidx = 0; cidx < nin; ++cidx)
          gWl[(size_t)r * nin + cidx] = gWl[(size_t)r * nin + cidx] + delta[r] * a[cidx];
      }
      for (int cidx = 0; cidx < nin; ++cidx) {
        double s = 0.0;
        for (int r = 0; r < nout; ++r) s = s + W[(size_t)r * nin + cidx] * delta[r];
        ga[cidx] = s;
      }
      if (l > 0) {
        for (int cidx = 0; cidx < nin; ++cidx) delta[cidx] = ga[cidx] * (1.0 - a[cidx] * a[cidx]);
      } else {
        for (int r = 0; r < D; ++r) gy[r] = gy[r] + ga[r];
        if (gt) *gt = *gt + ga[D]; /* the t input: df/dt^T v */
      }
    }
  }
}

/* Discrete adjoint of one instance over its fixed mesh (the reverse of
 * replay_one).  For step n with stages Y_i, k_i = f(t_n + c_i h, Y_i):
 *   kbar_i = h b_i ybar_{n+1} + sum_{tau in step} h b_i(theta_tau) ybar_tau
 *   for i = 7..1: g_i = J_f(Y_i)^T kbar_i, kbar_j += h a_ij g_i (j < i)
 *   ybar_n = ybar_{n+1} + sum_tau ybar_tau + sum_i g_i.
 * With gt0 / gt1, also the gradients with respect to the integration bounds
 * of the same frozen map, read this way: every accepted step size but the
 * last and every evaluation point's step are constants, t_n = t0 + sum_{j<n}
 * h_j for n < N, and the last step h_{N-1} = t1 - t_{N-1} absorbs the rest.
 * A step's size enters through y_{n+1} = y_n + h sum b_i k_i, the stage
 * inputs Y_i = y_n + h sum_j a_ij k_j at times t_n + c_i h, and the dense
 * outputs y_n + h sum b_i(theta) k_i with theta = (tau - t_n) / h:
 *   hbar_n = <ybar_{n+1}, sum_i b_i k_i>
 *          + sum_tau <ybar_tau, sum_i (b_i(theta) - theta b_i'(theta)) k_i>
 *          + sum_i <g_i, sum_j a_ij k_j> + sum_i c_i gt_i
 * and its start time through the abscissae and the field's time argument:
 *   tbar_n = -sum_tau <ybar_tau, sum_i b_i'(theta) k_i> + sum_i gt_i,
 * gt_i = (df/dt at stage i)^T kbar_i (0 for autonomous fields).  A point at
 * a step's end counts as theta = 1 of that step, a point at t0 as theta = 0
 * of the first.  Then dL/dt1 = hbar_{N-1} and dL/dt0 = sum_n tbar_n -
 * hbar_{N-1}. */
static void adjoint_one(const job *J, int i, double *work, double *act, double *dscr,
                        double *gW, double *gb) {
  const orc_field *F = J->F;
  const int D = F->D, K = J->K, N = J->mesh_n[i];
  const double t0 = J->t0[i];
  const double dir = (J->t1[i] < t0) ? -1.0 : 1.0; /* mesh steps carry this sign */
  const double *te = J->t_eval + (size_t)i * K;
  const double *gye = J->gy_eval ? J->gy_eval + (size_t)i * K * D : NULL;
  double *ys = (double *)malloc(sizeof(double) * (size_t)(N + 1) * D);
  double *yb = work, *k = yb + D, *Y = k + NS * D, *kb = Y + NS * D, *g = kb + NS * D;
  double *scratch = g + D;
  double *tv = (double *)malloc(sizeof(double) * (size_t)2 * D); /* sum_i w_i k_i, scratch */
  const int want_t = J->gt0 != NULL || J->gt1 != NULL;
  double tbar = 0.0, hbar_last = 0.0;
  double *gp = NULL;
  if (F->kind == ORC_VDP) gp = J->gparam + i;
  if (F->kind == ORC_LINEAR) gp = J->gparam + (size_t)i * D * D;
  if (gp) {
    int np = (F->kind == ORC_VDP) ? 1 : D * D;
    for (int p = 0; p < np; ++p) gp[p] = 0.0;
  }

  /* forward replay to recover the step-start states */
  replay_one(J, i, scratch, act, ys);
  fctx c = {F, i, act, 0};

  for (int j = 0; j < D; ++j) yb[j] = J->gy_final ? J->gy_final[(size_t)i * D + j] : 0.0;
  int cur = K - 1;
  for (int n = N - 1; n >= 0; --n) {
    const double t = J->mesh_t[(size_t)i * J->mesh_cap + n];
    const double h = J->mesh_h[(size_t)i * J->mesh_cap + n];
    const double t_next = mesh_end(J, i, n);
    const double *y = ys + (size_t)n * D;
    feval(&c, t, y, k);
    dp_stages(J->T, &c, t, h, y, D, k, Y);
    const rk_tab *T = J->T;
    double hbar = 0.0;
    if (want_t) { /* <ybar_{n+1}, sum b_i k_i> (dp_stages left k_7 = f(t_{n+1}, y_{n+1})) */
      for (int j = 0; j < D; ++j) {
        double s = 0.0;
        for (int q = 0; q < NS; ++q) s = s + T->b[q] * k[q * D + j];
        hbar = hbar + yb[j] * s;
      }
    }
    /* cotangents of the stage values */
    for (int s = 0; s < NS; ++s)
      for (int j = 0; j < D; ++j) kb[s * D + j] = h * T->b[s] * yb[j];
    while (cur >= 0 && dir * te[cur] > dir * t) {
      if (gye) {
        const double *gq = gye + (size_t)cur * D;
        double bt[NS];
        if (te[cur] == t_next) {
          /* this output is y_{n+1} itself: y_{n+1} = y_n + h sum b_i k_i */
          for (int s = 0; s < NS; ++s) bt[s] = T->b[s];
        } else {
          dense_weights(T, (te[cur] - t) / h, bt);
        }
        for (int s = 0; s < NS; ++s)
          for (int j = 0; j < D; ++j) kb[s * D + j] = kb[s * D + j] + h * bt[s] * gq[j];
        for (int j = 0; j < D; ++j) yb[j] = yb[j] + gq[j];
        if (want_t) {
          const double th = te[cur] == t_next ? 1.0 : (te[cur] - t) / h;
          dp_dense_deriv(T, th, k, D, tv); /* sum_i b_i'(theta) k_i */
          for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int q = 0; q < NS; ++q) s = s + bt[q] * k[q * D + j];
            hbar = hbar + gq[j] * (s - th * tv[j]);
            tbar = tbar - gq[j] * tv[j];
          }
        }
      }
      cur--;
    }
    for (int s = NS - 1; s >= 0; --s) {
      double gts = 0.0;
      for (int j = 0; j < D; ++j) g[j] = 0.0;
      vjp(J, i, t + T->c[s] * h, Y + s * D, kb + s * D, g, gp, gW, gb, act, dscr,
          want_t ? &gts : NULL);
      if (want_t) {
        for (int j = 0; j < D; ++j) {
          double s2 = 0.0;
          for (int l = 0; l < s; ++l) s2 = s2 + T->a[s][l] * k[l * D + j];
          hbar = hbar + g[j] * s2;
        }
        hbar = hbar + T->c[s] * gts;
        tbar = tbar + gts;
      }
      for (int l = 0; l < s; ++l)
        for (int j = 0; j < D; ++j) kb[l * D + j] = kb[l * D + j] + h * T->a[s][l] * g[j];
      for (int j = 0; j < D; ++j) yb[j] = yb[j] + g[j];
    }
    if (n == N - 1) hbar_last = hbar;
  }
  /* evaluation points at t0 are y0 itself (theta = 0 of the first step:
   * the abscissa's derivative is f(t0, y0)) */
  double *f0 = NULL;
  while (cur >= 0) {
    if (gye && te[cur] == t0) {
      for (int j = 0; j < D; ++j) yb[j] = yb[j] + gye[(size_t)cur * D + j];
      if (want_t) {
        if (!f0) {
          f0 = tv + D;
          feval(&c, t0, ys, f0);
        }
        for (int j = 0; j < D; ++j) tbar = tbar - gye[(size_t)cur * D + j] * f0[j];
      }
    }
    cur--;
  }
  for (int j = 0; j < D; ++j) J->gy0[(size_t)i * D + j] = yb[j];
  if (J->gt1) J->gt1[i] = hbar_last;
  if (J->gt0) J->gt0[i] = tbar - hbar_last;
  free(tv);
  free(ys);
}

/* ------------------------------------------------------------------------ */
/* Threading over instances (independent by construction, Sec. 3).          */
/* ------------------------------------------------------------------------ */
enum { MODE_SOLVE = 0, MODE_REPLAY = 1, MODE_ADJOINT = 2 };

typedef struct {
  const job *J;
  int mode, tid, lo, hi;
} worker_arg;

static size_t mlp_params(const orc_field *F, size_t *nb) {
  size_t w = 0, b = 0;
  for (int l = 0; l < F->n_layers; ++l) {
    w += (size_t)F->widths[l] * F->widths[l + 1];
    b += F->widths[l + 1];
  }
  if (nb) *nb = b;
  return w;
}

/* ------------------------------------------------------------------------ */
/* Joint continuous adjoint (App. A, CNF benchmark: the "torchode-joint"    */
/* backward pass, one adjoint equation of size bf + p for the whole batch). */
/* ------------------------------------------------------------------------ */
/* The augmented system of B instances of the MLP field M sharing its
 * parameters theta: z = [y (B x D); a (B x D); abar (P)] with
 *   dy/dt = f(t, y_b),  da_b/dt = -J_f(t, y_b)^T a_b,
 *   dabar/dt = -sum_b (df/dtheta)(t, y_b)^T a_b,
 * abar laid out as the weights then the biases, layer by layer (W[l] row
 * major).  One problem of size 2BD + P. */
static void aug_eval(const orc_field *F, double t, const double *z, double *out) {
  const orc_field *M = F->inner;
  const int B = F->n_inner, D = M->D;
  size_t nb;
  const size_t nw = mlp_params(M, &nb);
  int acts = 0;
  for (int l = 0; l < M->n_layers; ++l) acts += M->widths[l];
  const int maxw = mlp_max_width(M);
  double *act = F->scr, *dscr = act + acts + 8, *gy = dscr + 2 * maxw + 8;
  const double *y = z, *a = z + (size_t)B * D;
  double *oy = out, *oa = out + (size_t)B * D, *ow = out + 2 * (size_t)B * D, *ob = ow + nw;
  for (size_t p = 0; p < nw + nb; ++p) ow[p] = 0.0;
  job Jm;
  memset(&Jm, 0, sizeof(Jm));
  Jm.F = M;
  for (int b = 0; b < B; ++b) {
    const double *yb = y + (size_t)b * D, *ab = a + (size_t)b * D;
    f_mlp(M, t, yb, oy + (size_t)b * D, act);
    for (int j = 0; j < D; ++j) gy[j] = 0.0;
    /* gy = J^T a_b; the parameter cotangents summed into ow, ob in b order */
    vjp(&Jm, 0, t, yb, ab, gy, NULL, ow, ob, act, dscr, NULL);
    for (int j = 0; j < D; ++j) oa[(size_t)b * D + j] = -gy[j];
  }
  for (size_t p = 0; p < nw + nb; ++p) ow[p] = -ow[p];
}

static void *worker(void *p) {
  worker_arg *a = (worker_arg *)p;
  const job *J = a->J;
  const int D = J->F->D;
  int acts = 0, maxw = 8;
  const orc_field *M = J->F->kind == ORC_STACKED ? J->F->inner : J->F;
  if (M->kind == ORC_MLP) {
    for (int l = 0; l <= M->n_layers; ++l) acts += M->widths[l];
    maxw = mlp_max_width(M);
  }
  double *work = (double *)malloc(sizeof(double) * (size_t)(40 * D + 64));
  double *act = (double *)malloc(sizeof(double) * (size_t)(acts + 8));
  double *dscr = (double *)malloc(sizeof(double) * (size_t)(2 * maxw + 8));
  for (int i = a->lo; i < a->hi; ++i) {
    if (a->mode == MODE_SOLVE) solve_one(J, i, work, act);
    else if (a->mode == MODE_REPLAY) replay_one(J, i, work, act, NULL);
    else {
      double *gW = J->gW_part ? J->gW_part[a->tid] : NULL;
      double *gb = J->gb_part ? J->gb_part[a->tid] : NULL;
      adjoint_one(J, i, work, act, dscr, gW, gb);
    }
  }
  free(work);
  free(act);
  free(dscr);
  return NULL;
}

static int default_threads(void) {
  cpu_set_t s;
  if (sched_getaffinity(0, sizeof(s), &s) == 0) return CPU_COUNT(&s);
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

static int run(job *J, int mode, int nthreads) {
  if (nthreads <= 0) nthreads = default_threads();
  if (nthreads > J->B) nthreads = J->B > 0 ? J->B : 1;
  J->nthreads = nthreads;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
  worker_arg *args = (worker_arg *)malloc(sizeof(worker_arg) * nthreads);
  for (int k = 0; k < nthreads; ++k) {
    args[k].J = J;
    args[k].mode = mode;
    args[k].tid = k;
    args[k].lo = (int)((long)J->B * k / nthreads);
    args[k].hi = (int)((long)J->B * (k + 1) / nthreads);
  }
  for (int k = 1; k < nthreads; ++k) pthread_create(&th[k], NULL, worker, &args[k]);
  if (nthreads > 0) worker(&args[0]);
  for (int k = 1; k < nthreads; ++k) pthread_join(th[k], NULL);
  free(th);
  free(args);
  return nthreads;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points.  All arrays are host arrays, instance-major.       */
/* Return value: the number of threads used.                                 */
/* ------------------------------------------------------------------------ */
int orc_solve_yp(const orc_field *F, const orc_opts *O, int B, const double *y0,
                 const double *t0, const double *t1, const double *t_eval, int K,
                 double *y_eval, double *yp_eval, double *y_final, int32_t *n_acc,
                 int32_t *n_rej, int32_t *n_feval, int32_t *status, const orc_trace *trace,
                 int nthreads);
int orc_solve(const orc_field *F, const orc_opts *O, int B, const double *y0, const double *t0,
              const double *t1, const double *t_eval, int K, double *y_eval, double *y_final,
              int32_t *n_acc, int32_t *n_rej, int32_t *n_feval, int32_t *status,
              const orc_trace *trace, int nthreads) {
  return orc_solve_yp(F, O, B, y0, t0, t1, t_eval, K, y_eval, NULL, y_final, n_acc, n_rej,
                      n_feval, status, trace, nthreads);
}
/* orc_solve, plus dy/dt of the dense output at every evaluation point when
 * yp_eval is not NULL ([B][K][D]; NaN where y_eval is). */
int orc_solve_yp(const orc_field *F, const orc_opts *O, int B, const double *y0,
                 const double *t0, const double *t1, const double *t_eval, int K,
                 double *y_eval, double *yp_eval, double *y_final, int32_t *n_acc,
                 int32_t *n_rej, int32_t *n_feval, int32_t *status, const orc_trace *trace,
                 int nthreads) {
  job J;
  memset(&J, 0, sizeof(J));
  J.F = F;
  J.O = O;
  J.T = tab_of(O->method);
  J.B = B;
  J.K = K;
  J.y0 = y0;
  J.t0 = t0;
  J.t1 = t1;
  J.t_eval = t_eval;
  J.y_eval = y_eval;
  J.yp_eval = yp_eval;
  J.y_final = y_final;
  J.n_acc = n_acc;
  J.n_rej = n_rej;
  J.n_feval = n_feval;
  J.status = status;
  J.trace = trace;
  return run(&J, MODE_SOLVE, nthreads);
}

/* The fixed-mesh replay with the pair `method` (0 dopri5, 1 tsit5); yp_eval
 * (optional, [B][K][D]) receives dy/dt of the dense output at the points. */
int orc_replay_yp(int method, const orc_field *F, int B, const double *y0, const double *t0,
                  const double *t1, const double *mesh_t, const double *mesh_h,
                  const int32_t *mesh_n, int mesh_cap, const double *t_eval, int K,
                  double *y_eval, double *yp_eval, double *y_final, int nthreads);
int orc_replay_m(int method, const orc_field *F, int B, const double *y0, const double *t0,
                 const double *t1, const double *mesh_t, const double *mesh_h,
                 const int32_t *mesh_n, int mesh_cap, const double *t_eval, int K,
                 double *y_eval, double *y_final, int nthreads) {
  return orc_replay_yp(method, F, B, y0, t0, t1, mesh_t, mesh_h, mesh_n, mesh_cap, t_eval, K,
                       y_eval, NULL, y_final, nthreads);
}
int orc_replay_yp(int method, const orc_field *F, int B, const double *y0, const double *t0,
                  const double *t1, const double *mesh_t, const double *mesh_h,
                  const int32_t *mesh_n, int mesh_cap, const double *t_eval, int K,
                  double *y_eval, double *yp_eval, double *y_final, int nthreads) {
  job J;
  memset(&J, 0, sizeof(J));
  J.F = F;
  J.T = tab_of(method);
  J.B = B;
  J.K = K;
  J.y0 = y0;
  J.t0 = t0;
  J.t1 = t1;
  J.t_eval = t_eval;
  J.y_eval = y_eval;
  J.yp_eval = yp_eval;
  J.y_final = y_final;
  J.mesh_t = mesh_t;
  J.mesh_h = mesh_h;
  J.mesh_n = mesh_n;
  J.mesh_cap = mesh_cap;
  return run(&J, MODE_REPLAY, nthreads);
}
int orc_replay(const orc_field *F, int B, const double *y0, const double *t0, const double *t1,
               const double *mesh_t, const double *mesh_h, const int32_t *mesh_n, int mesh_cap,
               const double *t_eval, int K, double *y_eval, double *y_final, int nthreads) {
  return orc_replay_m(0, F, B, y0, t0, t1, mesh_t, mesh_h, mesh_n, mesh_cap, t_eval, K, y_eval,
                      y_final, nthreads);
}

/* gparam: VdP [B] (d/dmu), linear [B][D][D] (d/dA); MLP: gW[l], gb[l] summed
 * over the batch (per-thread partials added in thread order). */
int orc_adjoint_tm(int method, const orc_field *F, int B, const double *y0, const double *t0,
                   const double *t1, const double *mesh_t, const double *mesh_h,
                   const int32_t *mesh_n, int mesh_cap, const double *t_eval, int K,
                   const double *gy_eval, const double *gy_final, double *gy0, double *gparam,
                   double *const *gW, double *const *gb, double *gt0, double *gt1,
                   int nthreads);
int orc_adjoint_t(const orc_field *F, int B, const double *y0, const double *t0,
                  const double *t1, const double *mesh_t, const double *mesh_h,
                  const int32_t *mesh_n, int mesh_cap, const double *t_eval, int K,
                  const double *gy_eval, const double *gy_final, double *gy0, double *gparam,
                  double *const *gW, double *const *gb, double *gt0, double *gt1, int nthreads) {
  return orc_adjoint_tm(0, F, B, y0, t0, t1, mesh_t, mesh_h, mesh_n, mesh_cap, t_eval, K,
                        gy_eval, gy_final, gy0, gparam, gW, gb, gt0, gt1, nthreads);
}
int orc_adjoint(const orc_field *F, int B, const double *y0, const double *t0, const double *t1,
                const double *mesh_t, const double *mesh_h, const int32_t *mesh_n, int mesh_cap,
                const double *t_eval, int K, const double *gy_eval, const double *gy_final,
                double *gy0, double *gparam, double *const *gW, double *const *gb,
                int nthreads) {
  return orc_adjoint_t(F, B, y0, t0, t1, mesh_t, mesh_h, mesh_n, mesh_cap, t_eval, K, gy_eval,
                       gy_final, gy0, gparam, gW, gb, NULL, NULL, nthreads);
}
/* orc_adjoint, plus dL/dt0 and dL/dt1 of the frozen map when gt0 / gt1 are
 * not NULL ([B]; see adjoint_one), for the pair `method` (0 dopri5, 1 tsit5). */
int orc_adjoint_tm(int method, const orc_field *F, int B, const double *y0, const double *t0,
                   const double *t1, const double *mesh_t, const double *mesh_h,
                   const int32_t *mesh_n, int mesh_cap, const double *t_eval, int K,
                   const double *gy_eval, const double *gy_final, double *gy0, double *gparam,
                   double *const *gW, double *const *gb, double *gt0, double *gt1,
                   int nthreads) {
  /* the adjoint of a stacked problem is the per-instance adjoint on the
   * shared mesh (every block's Jacobian is its own); call it that way */
  if (F->kind == ORC_STACKED) return -1;
  job J;
  memset(&J, 0, sizeof(J));
  J.F = F;
  J.T = tab_of(method);
  J.B = B;
  J.K = K;
  J.y0 = y0;
  J.t0 = t0;
  J.t1 = t1;
  J.t_eval = t_eval;
  J.mesh_t = mesh_t;
  J.mesh_h = mesh_h;
  J.mesh_n = mesh_n;
  J.mesh_cap = mesh_cap;
  J.gy_eval = gy_eval;
  J.gy_final = gy_final;
  J.gy0 = gy0;
  J.gparam = gparam;
  J.gt0 = gt0;
  J.gt1 = gt1;
  double *ye_dummy = (double *)malloc(sizeof(double) * ((size_t)B * K * F->D + 1));
  double *yf_dummy = (double *)malloc(sizeof(double) * ((size_t)B * F->D + 1));
  J.y_eval = ye_dummy;
  J.y_final = yf_dummy;
  int T = nthreads <= 0 ? default_threads() : nthreads;
  if (T > B) T = B > 0 ? B : 1;
  size_t nb = 0, nw = 0;
  if (F->kind == ORC_MLP) {
    nw = mlp_params(F, &nb);
    J.gW_part = (double **)malloc(sizeof(double *) * T);
    J.gb_part = (double **)malloc(sizeof(double *) * T);
    for (int k = 0; k < T; ++k) {
      J.gW_part[k] = (double *)calloc(nw, sizeof(double));
      J.gb_part[k] = (double *)calloc(nb, sizeof(double));
    }
  }
  int used = run(&J, MODE_ADJOINT, T);
  if (F->kind == ORC_MLP) {
    size_t wo = 0, bo = 0;
    for (int l = 0; l < F->n_layers; ++l) {
      size_t nwl = (size_t)F->widths[l] * F->widths[l + 1], nbl = F->widths[l + 1];
      for (size_t p = 0; p < nwl; ++p) {
        double s = 0.0;
        for (int k = 0; k < used; ++k) s = s + J.gW_part[k][wo + p];
        gW[l][p] = s;
      }
      for (size_t p = 0; p < nbl; ++p) {
        double s = 0.0;
        for (int k = 0; k < used; ++k) s = s + J.gb_part[k][bo + p];
        gb[l][p] = s;
      }
      wo += nwl;
      bo += nbl;
    }
    for (int k = 0; k < T; ++k) {
      free(J.gW_part[k]);
      free(J.gb_part[k]);
    }
    free(J.gW_part);
    free(J.gb_part);
  }
  free(ye_dummy);
  free(yf_dummy);
  return used;
}

/* Joint continuous adjoint of B instances of the MLP field M over a shared
 * time axis (App. A, CNF benchmark): the augmented system of aug_eval
 * integrated backward from t1 to t0 as ONE problem -- one step size, one
 * RMS error norm over all 2BD + P components, one accept/reject decision
 * (the joint semantics of Sec. 4.1), with the pair, controller and
 * starting-step heuristic of orc_solve.  Start: y = y1 (the forward's
 * y(t1)), a = gy_final plus the cotangents of evaluation points at t1,
 * abar = 0.  The integration stops at every evaluation point strictly
 * inside (t0, t1), adds that point's cotangent to a (the loss jumps there),
 * and restarts (a new starting step); points at t0 add to a at the end.
 * Outputs: gy0 = a(t0) (dL/dy0), gW/gb = abar(t0) (dL/dtheta), y0_rec =
 * y(t0) (the state integrated back), stats = {accepted, rejected,
 * augmented-field evaluations, status} over all segments (status: the
 * first failure, else success).  t_eval [K] is shared and ordered from t0
 * to t1 (t0 < t1).  Returns -1 for an invalid call. */
int orc_joint_adjoint(const orc_field *M, const orc_opts *O, int B, const double *y1, double t0,
                      double t1, const double *t_eval, int K, const double *gy_eval,
                      const double *gy_final, double *gy0, double *const *gW, double *const *gb,
                      double *y0_rec, int32_t *stats) {
  if (!M || M->kind != ORC_MLP || B < 1 || !(t0 < t1) || K < 0) return -1;
  for (int k = 0; k < K; ++k)
    if (!(t_eval[k] >= t0 && t_eval[k] <= t1) || (k > 0 && t_eval[k] < t_eval[k - 1])) return -1;
  const int D = M->D;
  size_t nb;
  const size_t nw = mlp_params(M, &nb);
  const size_t BD = (size_t)B * D, N = 2 * BD + nw + nb;
  int acts = 0;
  for (int l = 0; l < M->n_layers; ++l) acts += M->widths[l];
  orc_field A;
  memset(&A, 0, sizeof(A));
  A.kind = ORC_AUGADJ;
  A.D = (int)N;
  A.inner = M;
  A.n_inner = B;
  A.scr = (double *)malloc(sizeof(double) * (size_t)(acts + 3 * mlp_max_width(M) + D + 32));
  double *z = (double *)malloc(sizeof(double) * N), *z2 = (double *)malloc(sizeof(double) * N);
  for (size_t j = 0; j < BD; ++j) {
    z[j] = y1[j];
    z[BD + j] = gy_final ? gy_final[j] : 0.0;
  }
  for (size_t p = 2 * BD; p < N; ++p) z[p] = 0.0;
  orc_opts o = *O;
  o.rtol_b = o.atol_b = NULL;
  /* cotangent of the points at index k added to a */
  int k = K - 1;
  while (k >= 0 && t_eval[k] == t1) {
    if (gy_eval)
      for (int b = 0; b < B; ++b)
        for (int j = 0; j < D; ++j) z[BD + (size_t)b * D + j] += gy_eval[((size_t)b * K + k) * D + j];
    k--;
  }
  int32_t n_acc = 0, n_rej = 0, n_fe = 0, status = ST_SUCCESS;
  double start = t1;
  while (1) {
    const double end = (k >= 0 && t_eval[k] > t0) ? t_eval[k] : t0;
    if (end != start) {
      int32_t na = 0, nr = 0, nf = 0, st = 0;
      orc_solve_yp(&A, &o, 1, z, &start, &end, NULL, 0, NULL, NULL, z2, &na, &nr, &nf, &st, NULL,
                   1);
      n_acc += na;
      n_rej += nr;
      n_fe += nf;
      if (st != ST_SUCCESS) {
        status = st;
        memcpy(z, z2, sizeof(double) * N);
        break;
      }
      memcpy(z, z2, sizeof(double) * N);
    }
    while (k >= 0 && t_eval[k] == end) {
      if (gy_eval)
        for (int b = 0; b < B; ++b)
          for (int j = 0; j < D; ++j)
            z[BD + (size_t)b * D + j] += gy_eval[((size_t)b * K + k) * D + j];
      k--;
    }
    start = end;
    if (end == t0) break;
  }
  for (size_t j = 0; j < BD; ++j) {
    gy0[j] = z[BD + j];
    if (y0_rec) y0_rec[j] = z[j];
  }
  size_t off = 2 * BD;
  for (int l = 0; l < M->n_layers; ++l) {
    const size_t n = (size_t)M->widths[l] * M->widths[l + 1];
    for (size_t q = 0; q < n; ++q) gW[l][q] = z[off + q];
    off += n;
  }
  for (int l = 0; l < M->n_layers; ++l) {
    for (int q = 0; q < M->widths[l + 1]; ++q) gb[l][q] = z[off + q];
    off += M->widths[l + 1];
  }
  stats[0] = n_acc;
  stats[1] = n_rej;
  stats[2] = n_fe;
  stats[3] = status;
  free(A.scr);
  free(z);
  free(z2);
  return 0;
}

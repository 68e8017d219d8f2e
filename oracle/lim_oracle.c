/*
 * lim_oracle.c -- plain CPU oracle of the local autonomous inference machine.
 *
 * TEST INFRASTRUCTURE ONLY (see lim_oracle.h).  Written for readability: every
 * loop follows the paper's definitions in the paper's order, with no blocking,
 * fusion or reordering.  Compile with -ffp-contract=off so that no multiply-add
 * is fused (the binary32 emulation below relies on separately rounded ops).
 */
#define _GNU_SOURCE
#include "lim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_LN2
#define M_LN2 0.69314718055994530942
#endif

/* ------------------------------------------------------------------------- */
/* Philox (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as   */
/* 1, 2, 3", SC'11).  Each round multiplies words 0 and 2 by the round        */
/* multipliers, takes hi/lo halves, and permutes/XORs with the key; the key   */
/* is bumped by the Weyl constants between rounds.  10 rounds.                */
/* ------------------------------------------------------------------------- */
#define PHILOX_M4x32_0 0xD2511F53u
#define PHILOX_M4x32_1 0xCD9E8D57u
#define PHILOX_W32_0 0x9E3779B9u /* floor(2^32 (golden ratio - 1)) */
#define PHILOX_W32_1 0xBB67AE85u /* floor(2^32 (sqrt(3) - 1))      */
#define PHILOX_M4x64_0 0xD2E7470EE14C6C93ull
#define PHILOX_M4x64_1 0xCA5A826395121157ull
#define PHILOX_W64_0 0x9E3779B97F4A7C15ull
#define PHILOX_W64_1 0xBB67AE8584CAA73Bull

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += PHILOX_W32_0;
      k1 += PHILOX_W32_1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M4x32_0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M4x32_1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += PHILOX_W64_0;
      k1 += PHILOX_W64_1;
    }
    unsigned __int128 p0 = (unsigned __int128)PHILOX_M4x64_0 * c0;
    unsigned __int128 p1 = (unsigned __int128)PHILOX_M4x64_1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout shared with the CUDA path by specification (not by code):
 * key = (seed low word, seed high word); counter = (shot, tick, site,
 * point << 4 | stream), stream 0 = noise, 1 = clock rings. */
static void draw(uint64_t seed, uint32_t shot, uint32_t tick, uint32_t site, uint32_t point,
                 uint32_t stream, uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {shot, tick, site, (point << 4) | stream};
  or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------- */
/* Rounding to the storage formats (IEEE 754 round to nearest, ties to even). */
/* The value is scaled by its quantum (a power of two, so exactly), rounded   */
/* to an integer with nearbyint (default mode: ties to even) and scaled back. */
/* ------------------------------------------------------------------------- */
static double round_to_format(double x, int frac_bits, int emin) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  frexp(x, &e); /* |x| in [2^(e-1), 2^e) */
  int ex = e - 1;
  if (ex < emin) ex = emin; /* subnormal range: fixed quantum */
  double quantum = ldexp(1.0, ex - frac_bits);
  return nearbyint(x / quantum) * quantum;
}
/* binary16: 10 fraction bits, smallest normal exponent -14. */
double or_round_f16(double x) {
  double r = round_to_format(x, 10, -14);
  if (fabs(r) > 65504.0) r = copysign(INFINITY, r);
  return r;
}
/* bfloat16: 7 fraction bits, binary32's exponent range. */
double or_round_bf16(double x) { return round_to_format(x, 7, -126); }

static double r32(double x) { return (double)(float)x; }

static double round_half_away(double x) { return x < 0 ? -floor(-x + 0.5) : floor(x + 0.5); }

/* ------------------------------------------------------------------------- */
/* Working arithmetic of one precision mode.                                 */
/* ------------------------------------------------------------------------- */
typedef struct {
  int prec, rule, is_int, is_f32;
  double pi0;      /* prior LLR (working units) */
  double clamp;    /* working units             */
  double alpha;    /* relaxation factor         */
  double alpha_w;  /* alpha as used (binary32 in the float modes) */
  int32_t A;       /* round(alpha*2^15), integer modes */
  double delta;    /* quantisation step         */
  uint64_t ring_thr;
} wk;

static int setup_wk(const or_params *prm, wk *w) {
  memset(w, 0, sizeof(*w));
  w->prec = prm->precision;
  w->rule = prm->rule;
  if (prm->precision < OR_PREC_F64 || prm->precision > OR_PREC_I8) return OR_E_INVAL;
  if (prm->rule != OR_RULE_MINSUM && prm->rule != OR_RULE_SUMPRODUCT) return OR_E_INVAL;
  if (prm->feedback != OR_FB_CHECK_MOVE && prm->feedback != OR_FB_BIT_DISCRETE &&
      prm->feedback != OR_FB_CHECK_MOVE_MULTI)
    return OR_E_INVAL;
  if (!(prm->q > 0.0 && prm->q < 1.0) || !(prm->clamp > 0.0)) return OR_E_INVAL;
  if (prm->sweeps_per_tick < 1 || prm->tick_budget < 0) return OR_E_INVAL;
  w->is_int = (prm->precision == OR_PREC_I16 || prm->precision == OR_PREC_I8);
  w->is_f32 = (prm->precision == OR_PREC_F32 || prm->precision == OR_PREC_F16 ||
               prm->precision == OR_PREC_BF16);
  if (w->is_int && prm->rule != OR_RULE_MINSUM) return OR_E_UNSUPPORTED;
  if (!(prm->tie_rel >= 0.0 && prm->tie_rel <= 0.5)) return OR_E_INVAL;
  if (w->is_int && prm->tie_rel != 0.0) return OR_E_INVAL;
  /* alpha = dt / (K tau): K Euler steps of tau dm/dt = F(m) - m per tick. */
  if (prm->tau > 0.0 && prm->dt_tick > 0.0) {
    w->alpha = prm->dt_tick / (prm->sweeps_per_tick * prm->tau);
  } else {
    w->alpha = 1.0; /* discrete machine: m <- F(m) */
  }
  if (!(w->alpha > 0.0 && w->alpha <= 1.0)) return OR_E_INVAL;
  double pi = log(prm->q / (1.0 - prm->q));
  if (w->is_int) {
    double qmax = (prm->precision == OR_PREC_I16) ? 32767.0 : 127.0;
    if (!(prm->quant_scale > 0.0)) return OR_E_INVAL;
    w->delta = prm->quant_scale;
    w->pi0 = round_half_away(pi / w->delta);
    double cq = round_half_away(prm->clamp / w->delta);
    w->clamp = cq < qmax ? cq : qmax;
    w->A = (int32_t)round_half_away(w->alpha * 32768.0);
    w->alpha_w = w->alpha;
  } else if (w->is_f32) {
    w->pi0 = r32(pi);
    w->clamp = r32(prm->clamp);
    w->alpha_w = r32(w->alpha);
  } else {
    w->pi0 = pi;
    w->clamp = prm->clamp;
    w->alpha_w = w->alpha;
  }
  double rho = prm->ring_prob >= 0.0 ? prm->ring_prob : 1.0 - exp(-prm->dt_tick);
  if (rho >= 1.0) w->ring_thr = 4294967296ull;
  else if (rho <= 0.0) w->ring_thr = 0;
  else w->ring_thr = (uint64_t)floor(rho * 4294967296.0);
  return OR_OK;
}

static double w_add(const wk *w, double a, double b) { return w->is_f32 ? r32(a + b) : a + b; }
static double w_sub(const wk *w, double a, double b) { return w->is_f32 ? r32(a - b) : a - b; }
static double w_mul(const wk *w, double a, double b) { return w->is_f32 ? r32(a * b) : a * b; }

static double w_clamp(const wk *w, double x) {
  if (x > w->clamp) return w->clamp;
  if (x < -w->clamp) return -w->clamp;
  return x;
}

/* Rounding of a freshly computed message to the storage format. */
static double w_store(const wk *w, double x) {
  switch (w->prec) {
    case OR_PREC_F32: return r32(x);
    case OR_PREC_F16: return or_round_f16(x);
    case OR_PREC_BF16: return or_round_bf16(x);
    default: return x; /* F64 and the integer modes are exact here */
  }
}

/* One Euler step of tau dm/dt = F(m) - m with step alpha (Algorithm 1, the
 * continuous-time BP; Sec. S4 discretisation), applied to a message whose new
 * BP value is m_new.  alpha = 1 is the discrete BP map itself. */
static double w_relax(const wk *w, double m_old, double m_new) {
  if (w->alpha == 1.0) return m_new;
  if (w->is_int) {
    /* m + alpha (m' - m) with alpha = A / 2^15, rounded half away from zero: an
     * odd function of (m, m'), so the update keeps the gauge covariance of BP
     * (Proposition of Sec. S2) exactly. */
    double d = m_new - m_old;
    double q = floor((w->A * fabs(d) + 16384.0) / 32768.0);
    return m_old + (d < 0 ? -q : q);
  }
  return w_add(w, m_old, w_mul(w, w->alpha_w, w_sub(w, m_new, m_old)));
}

/* All LLRs are clamped at CLAMP (Sec. S4): the BP value is clamped, relaxed and
 * clamped again, then rounded to the storage format. */
static double w_update(const wk *w, double m_old, double m_raw) {
  return w_store(w, w_clamp(w, w_relax(w, m_old, w_clamp(w, m_raw))));
}

/* Lower end of LocalMove's tie set (Algorithm 1: the argmax, ties broken
 * uniformly): best - tie_rel * max(1, |best|).  In the binary32 modes tie_rel is
 * held as binary32 and the product and the difference are each rounded to
 * binary32, the arithmetic of the beliefs themselves; integer modes tie exactly
 * (setup_wk refuses a nonzero tie_rel there). */
static double tie_floor(const wk *w, double tie_rel, double best) {
  if (w->is_int || tie_rel == 0.0) return best;
  const double a = fabs(best) > 1.0 ? fabs(best) : 1.0;
  if (w->is_f32) return r32(best - r32(r32(tie_rel) * a));
  return best - tie_rel * a;
}

double or_theta(const or_params *prm, int32_t d) {
  wk w;
  if (setup_wk(prm, &w) != OR_OK) return NAN;
  if (d <= 1) return INFINITY;
  /* Evidence(c) >= 1/d_c with Evidence = max_v sigma(L_v)  <=>  max_v L_v >= -log(d_c - 1). */
  double th = -log((double)(d - 1));
  if (w.is_int) return ceil(th / w.delta);
  if (w.is_f32) return r32(th);
  return th;
}

int or_derive(const or_params *prm, or_derived *out) {
  wk w;
  int st = setup_wk(prm, &w);
  if (st != OR_OK) return st;
  out->pi = w.pi0;
  out->clamp = w.clamp;
  out->alpha = w.alpha;
  out->alpha_q = w.A;
  out->ring_thr = w.ring_thr;
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Tanner graph: CSR given; the oracle builds its own CSC (Sec. S1, Tanner    */
/* graph definition: N(c) from the rows of H_X, N(v) from its columns).       */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t n, m, E;
  const int32_t *cptr, *cvar; /* N(c) = cvar[cptr[c] .. cptr[c+1]), edge ids = positions */
  int32_t *vptr;              /* [n+1] */
  int32_t *vchk;              /* [E] check of the j-th edge of v (ascending)  */
  int32_t *vedge;             /* [E] edge id of that edge                     */
} graph;

static void graph_free(graph *g) {
  free(g->vptr); free(g->vchk); free(g->vedge);
}

static int graph_build(const or_code *code, graph *g) {
  memset(g, 0, sizeof(*g));
  if (code->n <= 0 || code->m < 0 || !code->hx_ptr) return OR_E_INVAL;
  g->n = code->n;
  g->m = code->m;
  g->cptr = code->hx_ptr;
  g->cvar = code->hx_col;
  if (code->hx_ptr[0] != 0) return OR_E_INVAL;
  for (int c = 0; c < g->m; c++) {
    if (code->hx_ptr[c + 1] < code->hx_ptr[c]) return OR_E_INVAL;
    for (int e = code->hx_ptr[c]; e < code->hx_ptr[c + 1]; e++) {
      int v = code->hx_col[e];
      if (v < 0 || v >= g->n) return OR_E_INVAL;
      if (e > code->hx_ptr[c] && code->hx_col[e - 1] >= v) return OR_E_INVAL;
    }
  }
  g->E = code->hx_ptr[g->m];
  g->vptr = (int32_t *)calloc((size_t)g->n + 1, sizeof(int32_t));
  g->vchk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
  g->vedge = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
  if (!g->vptr || !g->vchk || !g->vedge) { graph_free(g); return OR_E_NOMEM; }
  for (int e = 0; e < g->E; e++) g->vptr[g->cvar[e] + 1]++;
  for (int v = 0; v < g->n; v++) g->vptr[v + 1] += g->vptr[v];
  int32_t *fill = (int32_t *)calloc((size_t)g->n, sizeof(int32_t));
  if (!fill) { graph_free(g); return OR_E_NOMEM; }
  for (int c = 0; c < g->m; c++) /* rows in increasing c: each N(v) ends up ascending */
    for (int e = g->cptr[c]; e < g->cptr[c + 1]; e++) {
      int v = g->cvar[e];
      int pos = g->vptr[v] + fill[v]++;
      g->vchk[pos] = c;
      g->vedge[pos] = e;
    }
  free(fill);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Check-to-qubit update, Eq. 2:                                             */
/*   m_{c->v} = 2 (-1)^{s_c + d_c} atanh( prod_{w in N(c)\v} tanh(m_{w->c}/2) ) */
/* Sum-product is evaluated in FP64 through the identity                     */
/*   2 atanh(prod tanh(a_w/2)) = phi(sum phi(a_w)) (a_w = |x_w|, signs apart), */
/*   phi(a) = -log tanh(a/2) = log((1+e^-a)/(1-e^-a)),                        */
/* with phi carried in the log domain so that neither tanh(a/2) -> 1 nor     */
/* e^-a -> 0 loses the value (messages up to CLAMP = 1000).                  */
/* Min-sum replaces the magnitude by min_w a_w (same sign rule).             */
/* ------------------------------------------------------------------------- */
/* log(1 - e^-a) for a > 0, accurate at both ends (log1p for small e^-a,
 * expm1 for a near 0). */
static double log1mexp(double a) { return a > M_LN2 ? log1p(-exp(-a)) : log(-expm1(-a)); }
static double phi(double a) { return log1p(exp(-a)) - log1mexp(a); }
static double log_phi(double a) { /* log phi(a), a > 0 */
  if (a > 20.0) return M_LN2 - a; /* phi(a) = 2e^-a (1 + e^-2a/3 + ...), correction < 1e-17 */
  return log(phi(a));
}
static double phi_of_log(double lu) { /* phi(U) with U = exp(lu) */
  if (lu < -36.0) return M_LN2 - lu; /* phi(U) = log(2/U) + O(U^2) */
  return phi(exp(lu));
}

/* x[0..d): incoming qubit->check messages of check c (CSR order); returns the
 * message to position `self`, before relaxation/clamp. */
static double check_out(const wk *w, int rule, int s_c, int d, const double *x, int self) {
  int neg = (s_c + d) & 1;
  int any_zero = 0;
  for (int j = 0; j < d; j++) {
    if (j == self) continue;
    if (x[j] < 0) neg ^= 1; /* sgn(0) = +1 */
    if (x[j] == 0) any_zero = 1;
  }
  double mag;
  if (d == 1) {
    /* Empty product: tanh-product 1, atanh(1) = +inf; a weight-1 check fixes its
     * qubit, and the clamp turns the infinite LLR into +-CLAMP. */
    mag = INFINITY;
  } else if (any_zero) {
    mag = 0.0;
  } else if (rule == OR_RULE_MINSUM) {
    mag = INFINITY;
    for (int j = 0; j < d; j++)
      if (j != self && fabs(x[j]) < mag) mag = fabs(x[j]);
  } else {
    double mx = -INFINITY;
    for (int j = 0; j < d; j++)
      if (j != self) {
        double l = log_phi(fabs(x[j]));
        if (l > mx) mx = l;
      }
    double sum = 0.0;
    for (int j = 0; j < d; j++)
      if (j != self) sum += exp(log_phi(fabs(x[j])) - mx);
    mag = phi_of_log(mx + log(sum));
    if (w->is_f32) mag = r32(mag);
  }
  if (mag == 0.0) return 0.0; /* sgn(0) irrelevant: store +0 */
  return neg ? -mag : mag;
}

/* ------------------------------------------------------------------------- */
/* One Jacobi sweep of Eq. 1-2 from the state (pi, cv, vc) on syndrome s:    */
/* both message families are computed from the previous iterate (Sec. S2,    */
/* steps 1-2), then relaxed and clamped.                                     */
/* ------------------------------------------------------------------------- */
static void sweep(const wk *w, const graph *g, const uint8_t *s, const double *pi,
                  const double *cv, const double *vc, double *cv_new, double *vc_new,
                  double *xbuf) {
  /* Eq. 1: m_{v->c} = pi_v + sum_{c' in N(v)\c} m_{c'->v}, summed in ascending c'. */
  for (int v = 0; v < g->n; v++) {
    for (int j = g->vptr[v]; j < g->vptr[v + 1]; j++) {
      double acc = pi[v];
      for (int jj = g->vptr[v]; jj < g->vptr[v + 1]; jj++)
        if (jj != j) acc = w_add(w, acc, cv[g->vedge[jj]]);
      int e = g->vedge[j];
      vc_new[e] = w_update(w, vc[e], acc);
    }
  }
  /* Eq. 2 for every edge of every check. */
  for (int c = 0; c < g->m; c++) {
    int b = g->cptr[c], d = g->cptr[c + 1] - b;
    for (int j = 0; j < d; j++) xbuf[j] = vc[b + j];
    for (int j = 0; j < d; j++) {
      double raw = check_out(w, w->rule, s[c], d, xbuf, j);
      cv_new[b + j] = w_update(w, cv[b + j], raw);
    }
  }
}

/* Eq. 3 read-out: L_v = pi_v + sum_{c in N(v)} m_{c->v}, ascending c. */
static void readout(const wk *w, const graph *g, const double *pi, const double *cv, double *L) {
  for (int v = 0; v < g->n; v++) {
    double acc = pi[v];
    for (int j = g->vptr[v]; j < g->vptr[v + 1]; j++) acc = w_add(w, acc, cv[g->vedge[j]]);
    L[v] = acc;
  }
}

static int max_check_degree(const graph *g) {
  int dm = 0;
  for (int c = 0; c < g->m; c++)
    if (g->cptr[c + 1] - g->cptr[c] > dm) dm = g->cptr[c + 1] - g->cptr[c];
  return dm;
}

int or_bp_sweeps(const or_code *code, const or_params *prm, const uint8_t *s, const double *pi_in,
                 const double *cv_in, const double *vc_in, double *cv_out, double *vc_out,
                 int32_t ksweeps) {
  wk w;
  int st = setup_wk(prm, &w);
  if (st != OR_OK) return st;
  graph g;
  st = graph_build(code, &g);
  if (st != OR_OK) return st;
  size_t E = (size_t)(g.E > 0 ? g.E : 1);
  double *cv = malloc(E * sizeof(double)), *vc = malloc(E * sizeof(double));
  double *cn = malloc(E * sizeof(double)), *vn = malloc(E * sizeof(double));
  double *pi = malloc((size_t)g.n * sizeof(double));
  double *xb = malloc((size_t)(max_check_degree(&g) + 1) * sizeof(double));
  if (!cv || !vc || !cn || !vn || !pi || !xb) {
    free(cv); free(vc); free(cn); free(vn); free(pi); free(xb); graph_free(&g);
    return OR_E_NOMEM;
  }
  memcpy(cv, cv_in, (size_t)g.E * sizeof(double));
  memcpy(vc, vc_in, (size_t)g.E * sizeof(double));
  for (int v = 0; v < g.n; v++) pi[v] = pi_in ? pi_in[v] : w.pi0;
  for (int k = 0; k < ksweeps; k++) {
    sweep(&w, &g, s, pi, cv, vc, cn, vn, xb);
    double *t = cv; cv = cn; cn = t;
    t = vc; vc = vn; vn = t;
  }
  memcpy(cv_out, cv, (size_t)g.E * sizeof(double));
  memcpy(vc_out, vc, (size_t)g.E * sizeof(double));
  free(cv); free(vc); free(cn); free(vn); free(pi); free(xb);
  graph_free(&g);
  return OR_OK;
}

int or_readout(const or_code *code, const or_params *prm, const double *pi_in, const double *cv,
               double *l_out) {
  wk w;
  int st = setup_wk(prm, &w);
  if (st != OR_OK) return st;
  graph g;
  st = graph_build(code, &g);
  if (st != OR_OK) return st;
  double *pi = malloc((size_t)g.n * sizeof(double));
  if (!pi) { graph_free(&g); return OR_E_NOMEM; }
  for (int v = 0; v < g.n; v++) pi[v] = pi_in ? pi_in[v] : w.pi0;
  readout(&w, &g, pi, cv, l_out);
  free(pi);
  graph_free(&g);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Noise: e_v ~ Bernoulli(p) i.i.d. (code-capacity Z noise, Preliminaries),   */
/* e_v = [u < floor(p 2^32)] with u word (v mod 4) of the Philox block         */
/* (shot, 0, v/4, point<<4|0); syndrome s = H_X e mod 2.                      */
/* ------------------------------------------------------------------------- */
static uint64_t prob_thr(double p) {
  if (p >= 1.0) return 4294967296ull;
  if (p <= 0.0) return 0;
  return (uint64_t)floor(p * 4294967296.0);
}

static void syndrome(const graph *g, const uint8_t *e, uint8_t *s) {
  for (int c = 0; c < g->m; c++) {
    int par = 0;
    for (int j = g->cptr[c]; j < g->cptr[c + 1]; j++) par ^= e[g->cvar[j]];
    s[c] = (uint8_t)par;
  }
}

static void noise(const graph *g, double p, uint64_t seed, uint32_t point, uint32_t shot,
                  uint8_t *e, uint8_t *s) {
  uint64_t thr = prob_thr(p);
  for (int v = 0; v < g->n; v++) {
    uint32_t u[4];
    draw(seed, shot, 0, (uint32_t)v >> 2, point, 0, u);
    e[v] = (uint64_t)u[v & 3] < thr;
  }
  syndrome(g, e, s);
}

int or_noise(const or_code *code, double p, uint64_t seed, uint32_t point, uint32_t shot,
             uint8_t *e_out, uint8_t *s_out) {
  graph g;
  int st = graph_build(code, &g);
  if (st != OR_OK) return st;
  noise(&g, p, seed, point, shot, e_out, s_out);
  graph_free(&g);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* One trajectory.                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
  uint32_t prio; /* ring time inside the tick, as a uniform 32-bit key */
  int32_t c;
  uint32_t pick; /* tie-break word */
} ring_t;

static int ring_cmp(const void *a, const void *b) {
  const ring_t *x = (const ring_t *)a, *y = (const ring_t *)b;
  if (x->prio != y->prio) return x->prio < y->prio ? -1 : 1;
  return x->c < y->c ? -1 : (x->c > y->c);
}

static void flip_qubit(const graph *g, uint8_t *e, uint8_t *s, int v) {
  e[v] ^= 1;
  for (int j = g->vptr[v]; j < g->vptr[v + 1]; j++) s[g->vchk[j]] ^= 1; /* s <- s + H_X 1_v */
}

/* Gauge switch of qubit v (Sec. S2, local rule): prior and every message on v
 * change sign. */
static void gauge_qubit(const graph *g, double *pi, double *cv, double *vc, int v) {
  pi[v] = -pi[v];
  for (int j = g->vptr[v]; j < g->vptr[v + 1]; j++) {
    int e = g->vedge[j];
    cv[e] = -cv[e];
    vc[e] = -vc[e];
  }
}

static int all_zero(const uint8_t *x, int len) {
  for (int i = 0; i < len; i++)
    if (x[i]) return 0;
  return 1;
}

static void log_move(or_trace *tr, int t, int c, int v) {
  if (!tr) return;
  if (tr->moves && tr->n_moves < tr->move_cap) {
    tr->moves[3 * tr->n_moves + 0] = t;
    tr->moves[3 * tr->n_moves + 1] = c;
    tr->moves[3 * tr->n_moves + 2] = v;
  }
  tr->n_moves++;
}

static void snap(or_trace *tr, const graph *g, int t, const uint8_t *e, const uint8_t *s) {
  if (!tr || t > tr->max_ticks) return;
  if (tr->e_hist) memcpy(tr->e_hist + (size_t)t * g->n, e, (size_t)g->n);
  if (tr->s_hist) memcpy(tr->s_hist + (size_t)t * g->m, s, (size_t)g->m);
}

static int run(const or_code *code, const or_params *prm, double p, const uint8_t *e_given,
               uint64_t seed, uint32_t point, uint32_t shot, or_record *rec, or_trace *tr);

uint32_t or_multi_move_set(const double *L, int32_t d, int32_t first) {
  if (d < 1 || d > 32 || first < 0 || first >= d) return 0;
  uint32_t mask = 1u << first;
  /* the other positions by L descending, ties by position (selection order) */
  int order[32], n = 0;
  for (int j = 0; j < d; j++)
    if (j != first) order[n++] = j;
  for (int i = 0; i < n; i++)
    for (int k = i + 1; k < n; k++)
      if (L[order[k]] > L[order[i]] || (L[order[k]] == L[order[i]] && order[k] < order[i])) {
        int t = order[i]; order[i] = order[k]; order[k] = t;
      }
  /* add pairs while they raise the log-likelihood of the set */
  for (int i = 0; i + 1 < n; i += 2) {
    if (!(L[order[i]] + L[order[i + 1]] > 0)) break;
    mask |= (1u << order[i]) | (1u << order[i + 1]);
  }
  return mask;
}

int or_run_shot(const or_code *code, const or_params *prm, double p, uint64_t seed,
                uint32_t point, uint32_t shot, or_record *rec, or_trace *tr) {
  return run(code, prm, p, NULL, seed, point, shot, rec, tr);
}

int or_run_from(const or_code *code, const or_params *prm, const uint8_t *e0, uint64_t seed,
                uint32_t point, uint32_t shot, or_record *rec, or_trace *tr) {
  if (!e0) return OR_E_INVAL;
  return run(code, prm, 0.0, e0, seed, point, shot, rec, tr);
}

static int run(const or_code *code, const or_params *prm, double p, const uint8_t *e_given,
               uint64_t seed, uint32_t point, uint32_t shot, or_record *rec, or_trace *tr) {
  wk w;
  int st = setup_wk(prm, &w);
  if (st != OR_OK) return st;
  graph g;
  st = graph_build(code, &g);
  if (st != OR_OK) return st;
  int n = g.n, m = g.m;
  size_t E = (size_t)(g.E > 0 ? g.E : 1);
  int dmax = max_check_degree(&g);
  uint8_t *e = calloc((size_t)n, 1), *s = calloc((size_t)(m > 0 ? m : 1), 1);
  double *pi = malloc((size_t)n * sizeof(double)), *L = malloc((size_t)n * sizeof(double));
  double *cv = calloc(E, sizeof(double)), *vc = calloc(E, sizeof(double));
  double *cn = calloc(E, sizeof(double)), *vn = calloc(E, sizeof(double));
  double *xb = malloc((size_t)(dmax + 1) * sizeof(double));
  double *theta = malloc((size_t)(dmax + 1) * sizeof(double));
  ring_t *rings = malloc(sizeof(ring_t) * (size_t)(m > 0 ? m : 1));
  uint8_t *flip = calloc((size_t)n, 1);
  if (!e || !s || !pi || !L || !cv || !vc || !cn || !vn || !xb || !theta || !rings || !flip) {
    st = OR_E_NOMEM;
    goto done;
  }
  if (prm->feedback == OR_FB_CHECK_MOVE_MULTI && dmax > 32) { /* move sets are 32-bit masks */
    st = OR_E_UNSUPPORTED;
    goto done;
  }
  if (tr) tr->n_moves = 0;
  for (int d = 0; d <= dmax; d++) theta[d] = or_theta(prm, d);

  /* Initialisation (Algorithm 1; Sec. S2): m = 0, pi_v = log(q/(1-q)). */
  for (int v = 0; v < n; v++) pi[v] = w.pi0;
  if (e_given) {
    for (int v = 0; v < n; v++) e[v] = e_given[v] & 1;
    syndrome(&g, e, s);
  } else {
    noise(&g, p, seed, point, shot, e, s);
  }
  snap(tr, &g, 0, e, s);

  or_record r = {-1, 0, 1, 0, 0, 0};
  if (all_zero(s, m)) {
    r.t_clr = 0;
    r.converged = 1;
  } else {
    for (int t = 1; t <= prm->tick_budget; t++) {
      r.ticks = t;
      /* Read-out from the messages of the previous tick (Eq. 3). */
      readout(&w, &g, pi, cv, L);
      if (tr && tr->l_hist && t <= tr->max_ticks) memcpy(tr->l_hist + (size_t)t * n, L, (size_t)n * sizeof(double));

      if (prm->feedback == OR_FB_CHECK_MOVE || prm->feedback == OR_FB_CHECK_MOVE_MULTI) {
        /* Poisson clocks discretised per tick: each check active at the start of the
         * tick rings with probability rho; ringing checks act in the order of a
         * uniform random ring time (ties by check index). */
        int nr = 0;
        for (int c = 0; c < m; c++) {
          if (!s[c]) continue;
          uint32_t u[4];
          draw(seed, shot, (uint32_t)t, (uint32_t)c, point, 1, u);
          if ((uint64_t)u[0] < w.ring_thr) {
            rings[nr].prio = u[1];
            rings[nr].c = c;
            rings[nr].pick = u[2];
            nr++;
          }
        }
        qsort(rings, (size_t)nr, sizeof(ring_t), ring_cmp);
        for (int i = 0; i < nr; i++) {
          int c = rings[i].c;
          if (!s[c]) continue; /* (i) the check must still be active */
          int b = g.cptr[c], d = g.cptr[c + 1] - b;
          double best = -INFINITY;
          for (int j = 0; j < d; j++)
            if (L[g.cvar[b + j]] > best) best = L[g.cvar[b + j]];
          if (!(best >= theta[d])) continue; /* (ii) Evidence(c) >= 1/d_c */
          /* LocalMove: flip a qubit of argmax_w Pr_BP(e_w|s), ties broken uniformly;
           * the ties are the beliefs >= lo (lo = best when tie_rel = 0). */
          const double lo = tie_floor(&w, prm->tie_rel, best);
          int nt = 0;
          for (int j = 0; j < d; j++)
            if (L[g.cvar[b + j]] >= lo) nt++;
          int pick = (int)(((uint64_t)rings[i].pick * (uint64_t)nt) >> 32);
          int first = -1;
          for (int j = 0; j < d; j++)
            if (L[g.cvar[b + j]] >= lo) {
              if (pick == 0) { first = j; break; }
              pick--;
            }
          uint32_t set = 1u << first;
          if (prm->feedback == OR_FB_CHECK_MOVE_MULTI) {
            double Lc[32];
            for (int j = 0; j < d; j++) Lc[j] = L[g.cvar[b + j]];
            set = or_multi_move_set(Lc, d, first);
          }
          for (int j = 0; j < d; j++) {
            if (!((set >> j) & 1)) continue;
            const int v = g.cvar[b + j];
            flip_qubit(&g, e, s, v);
            r.moves++;
            log_move(tr, t, c, v);
            if (prm->gauge_on_move) {
              gauge_qubit(&g, pi, cv, vc, v);
              L[v] = -L[v];
            }
          }
        }
      } else {
        /* Eq. 3-4: f_v = 1[L_v > 0] for every qubit at once, s <- s + H_X f,
         * then the gauge switch of every flipped qubit. */
        for (int v = 0; v < n; v++) flip[v] = L[v] > 0;
        for (int v = 0; v < n; v++)
          if (flip[v]) {
            flip_qubit(&g, e, s, v);
            gauge_qubit(&g, pi, cv, vc, v);
            r.moves++;
            log_move(tr, t, -1, v);
          }
      }
      snap(tr, &g, t, e, s);

      if (all_zero(s, m)) { /* clearance time */
        r.t_clr = t;
        r.converged = 1;
        break;
      }
      if (t == prm->tick_budget) break; /* budget exhausted: non-convergent */

      for (int k = 0; k < prm->sweeps_per_tick; k++) {
        sweep(&w, &g, s, pi, cv, vc, cn, vn, xb);
        double *tmp = cv; cv = cn; cn = tmp;
        tmp = vc; vc = vn; vn = tmp;
        r.sweeps++;
      }
    }
  }
  /* Fill the remaining trace rows with the final state. */
  if (tr) {
    for (int t = (int)r.ticks + 1; t <= tr->max_ticks; t++) snap(tr, &g, t, e, s);
    if (tr->cv_final) memcpy(tr->cv_final, cv, (size_t)g.E * sizeof(double));
    if (tr->vc_final) memcpy(tr->vc_final, vc, (size_t)g.E * sizeof(double));
    if (tr->pi_final) memcpy(tr->pi_final, pi, (size_t)n * sizeof(double));
    if (tr->e_final) memcpy(tr->e_final, e, (size_t)n);
  }
  /* Decoding criteria (1)-(2): non-convergence is a failure; otherwise the
   * residual e (= e_0 + correction, H_X e = 0) fails iff it anticommutes with
   * an X-logical, i.e. e is not in row(H_Z). */
  if (r.converged) {
    r.failed = 0;
    for (int j = 0; j < code->k; j++) {
      int par = 0;
      for (int v = 0; v < n; v++) par ^= e[v] & code->logicals[(size_t)j * n + v];
      if (par) r.failed = 1;
    }
  } else {
    r.failed = 1;
  }
  *rec = r;
  st = OR_OK;
done:
  free(e); free(s); free(pi); free(L); free(cv); free(vc); free(cn); free(vn);
  free(xb); free(theta); free(rings); free(flip);
  graph_free(&g);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Ordinary BP decoding: fixed syndrome, no gauge, hard decision per iteration. */
/* ------------------------------------------------------------------------- */
int or_bp_decode(const or_code *code, const or_params *prm, double p, uint64_t seed,
                 uint32_t point, uint32_t shot, or_record *rec, uint8_t *ehat_out) {
  if (!rec) return OR_E_INVAL;
  wk w;
  int st = setup_wk(prm, &w);
  if (st != OR_OK) return st;
  graph g;
  st = graph_build(code, &g);
  if (st != OR_OK) return st;
  int n = g.n, m = g.m;
  size_t E = (size_t)(g.E > 0 ? g.E : 1), M = (size_t)(m > 0 ? m : 1);
  int dmax = max_check_degree(&g);
  uint8_t *e0 = calloc((size_t)n, 1), *ehat = calloc((size_t)n, 1);
  uint8_t *s = calloc(M, 1), *s_hat = calloc(M, 1);
  double *pi = malloc((size_t)n * sizeof(double)), *L = malloc((size_t)n * sizeof(double));
  double *cv = calloc(E, sizeof(double)), *vc = calloc(E, sizeof(double));
  double *cn = calloc(E, sizeof(double)), *vn = calloc(E, sizeof(double));
  double *xb = malloc((size_t)(dmax + 1) * sizeof(double));
  if (!e0 || !ehat || !s || !s_hat || !pi || !L || !cv || !vc || !cn || !vn || !xb) {
    st = OR_E_NOMEM;
    goto done;
  }
  for (int v = 0; v < n; v++) pi[v] = w.pi0;
  noise(&g, p, seed, point, shot, e0, s);

  or_record r = {-1, 0, 1, 0, 0, 0};
  if (all_zero(s, m)) {
    r.t_clr = 0;
    r.converged = 1;
  } else {
    for (int i = 1; i <= prm->tick_budget; i++) {
      r.ticks = i;
      readout(&w, &g, pi, cv, L); /* beliefs from the messages after i-1 sweeps */
      for (int v = 0; v < n; v++) {
        uint8_t d = L[v] > 0 ? 1 : (L[v] < 0 ? 0 : ehat[v]);
        if (d != ehat[v]) {
          ehat[v] = d;
          r.moves++;
        }
      }
      syndrome(&g, ehat, s_hat);
      if (memcmp(s_hat, s, (size_t)m) == 0) {
        r.t_clr = i;
        r.converged = 1;
        break;
      }
      if (i == prm->tick_budget) break;
      for (int k = 0; k < prm->sweeps_per_tick; k++) {
        sweep(&w, &g, s, pi, cv, vc, cn, vn, xb);
        double *tmp = cv; cv = cn; cn = tmp;
        tmp = vc; vc = vn; vn = tmp;
        r.sweeps++;
      }
    }
  }
  /* The decoder's output is ehat; the residual e0 + ehat has zero syndrome when
   * converged and fails iff it anticommutes with an X-logical. */
  if (r.converged) {
    r.failed = 0;
    for (int j = 0; j < code->k; j++) {
      int par = 0;
      for (int v = 0; v < n; v++) par ^= (e0[v] ^ ehat[v]) & code->logicals[(size_t)j * n + v];
      if (par) r.failed = 1;
    }
  }
  if (ehat_out) memcpy(ehat_out, ehat, (size_t)n);
  *rec = r;
  st = OR_OK;
done:
  free(e0); free(ehat); free(s); free(s_hat); free(pi); free(L);
  free(cv); free(vc); free(cn); free(vn); free(xb);
  graph_free(&g);
  return st;
}

int or_run_shots(const or_code *code, const or_params *prm, double p, uint64_t seed,
                 uint32_t point, uint32_t shot0, uint32_t nshots, or_record *records) {
  for (uint32_t i = 0; i < nshots; i++) {
    int st = or_run_shot(code, prm, p, seed, point, shot0 + i, &records[i], NULL);
    if (st != OR_OK) return st;
  }
  return OR_OK;
}

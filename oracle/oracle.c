/*
 * oracle.c -- CPU oracle for the next reaction random time algorithm (NRRTA).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code.  It shares no code with the CUDA path.
 *
 * What it computes (Liu & Wang, arXiv:2103.00405):
 *   - propensities a_k = c_k h_k(X), h_k = prod_j binom(X_j, sigma_jk)      (Eq. 1-2)
 *   - internal times T_k(t) = int_0^t a_k ds                                  (Eq. 17-18)
 *   - unit-rate internal-time increments dT = ln(1/r) ~ Exp(1)               (Eq. 24)
 *   - per-channel real waiting time from int a_k ds = dT_k, i.e. for a
 *     constant a_k over the step: dt_k = (P_k - T_k) / a_k                   (Eq. 25)
 *   - the smallest dt_k fires ("first arriving wins")                        (Eq. 26)
 *   - only the fired channel draws a fresh increment; the others keep their
 *     unused internal time                                                   (Eq. 27, Table 2)
 * P_k is the internal time of channel k's next firing (sum of its Exp(1)
 * increments), so P_k - T_k is the remaining internal time of Table 2.
 *
 * Every floating-point operation is one IEEE binary64 operation rounded to
 * nearest; the file must be compiled with -ffp-contract=off and without
 * -ffast-math.  All a_k are recomputed from X after every event (the plain
 * definition; a dependency graph is only a shortcut that gives the same values).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from its published
 * definition.  Draw n of channel k of trajectory g uses counter
 * (n >> 1, lo32(g), k, stream) and key (lo32(seed), hi32(seed)); even n takes
 * output words 0,1 and odd n words 2,3.  The 52 high bits v of (w1:w0) give
 * u = (2v + 1) 2^-53 in (0, 1), and the increment is -ln(u).
 *
 * The logarithm is an integer fixed-point evaluation (fx_log below) rounded
 * once to binary64, so it is exactly reproducible on any machine.  It follows
 * the textbook reduction ln(M 2^E) = (E + q) ln 2 + ln(m), m = M / 2^q in
 * [sqrt(1/2), sqrt(2)), and ln(m) = 2 atanh(s), s = (m - 1)/(m + 1), with the
 * atanh power series 2 s (1 + s^2/3 + s^4/5 + ...).
 *
 * Modes (oracle_run's `mode`):
 *   0  Table 2 in the internal-time form above: every internal time advances at
 *      every event, T_k += a_k dt, and the waiting times (P_k - T_k) / a_k are
 *      recomputed for all channels.
 *   1  the same method in absolute-time ("lazy") form, the Gibson-Bruck next
 *      reaction method with the dependency graph the paper describes (Sec. 5):
 *      each channel keeps the real time s_k of its last update and its absolute
 *      firing time tau_k = s_k + (P_k - T_k) / a_k; an event at tau_mu touches
 *      only mu and the channels that read a species the event changed (their
 *      internal time is first brought up to the event, T_k += a_k (t - s_k), then
 *      a_k and tau_k are recomputed); every other tau_k stays as it is.  In exact
 *      arithmetic both modes give the same path; their roundings differ.
 *   2  Table 3's form ("parallel NRRTA"): each channel keeps its relative waiting
 *      time w_k and the propensity p_k it was computed with; after an event that
 *      took dt, every propensity is recomputed (no dependency graph) and every
 *      other channel's waiting time is rescaled, w_k = (p_k / a_k) (w_k - dt); the
 *      fired channel draws w_mu = E / a_mu; then p_k = a_k (the update Table 3
 *      leaves implicit).  A channel whose propensity drops to 0 keeps its remaining
 *      internal time q_k = p_k (w_k - dt) frozen (w_k = +inf) and resumes with
 *      w_k = q_k / a_k.  Internal times for the likelihood accumulate T_k += a_k dt.
 *      Same path as modes 0 and 1 in exact arithmetic.
 * beta (NULL = constant rates; mode 0 only): time-dependent rates c_k(t) = c_k (1 + beta_k t),
 * beta_k >= 0 (Sec. 6, Eq. 29: the random-time form needs only each channel's own
 * integral).  With A_k = c_k h_k(X) constant between events, channel k's internal time
 * over [t, t + d] grows by A_k I_k(t, d), I_k = d (1 + beta_k t) + beta_k d^2 / 2, and its
 * waiting time solves A_k I_k(t, d) = P_k - T_k:
 *   u = 1 + beta t,  b = A u,  d = 2 R / (b + sqrt(b^2 + 2 A beta R)),  R = P_k - T_k
 * (the root of the quadratic written without cancellation); for beta_k = 0 the operations
 * are exactly those of the constant-rate form.  ln a_mu is taken at the event time,
 * a_mu = A_mu (1 + beta_mu t).
 * enabled (NULL = all): a channel with enabled[k] == 0 is forbidden to fire; its
 * propensity is taken as 0, so its internal time is frozen (Table 2's note on
 * boundary conditions).
 *
 * ORACLE_MUTANT (0 by default) plants one deliberate mistake per value, used only
 * by the mutation test to show that the pins catch such mistakes.
 */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------------ */
/* Philox4x32-10                                                                  */
/* ------------------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) { /* key schedule: add the Weyl constants between rounds */
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ (ORACLE_MUTANT == 14 ? c3 : c1) ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------------ */
/* Fixed-point natural logarithm                                                  */
/* ------------------------------------------------------------------------------ */

/* round(ln 2 * 2^64) */
static const uint64_t LN2_Q64 = 0xB17217F7D1CF79ACull;

static int bitlen64(uint64_t v) {
  int n = 0;
  while (v) { n++; v >>= 1; }
  return n;
}

static int bitlen128(u128 v) {
  int n = 0;
  while (v) { n++; v >>= 1; }
  return n;
}

static uint64_t mulhi64(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * (u128)b) >> 64); }

/* The binary64 value nearest to V * 2^scale (V > 0), ties to even.  The result
 * is known to be a normal number for every call made in this file. */
static double round_to_double(u128 V, int scale) {
  int p = bitlen128(V) - 1; /* V in [2^p, 2^(p+1)) */
  uint64_t mant;
  if (p <= 52) {
    mant = (uint64_t)(V << (52 - p));
  } else {
    int sh = p - 52;
    u128 q = V >> sh;
    u128 rem = V - (q << sh);
    u128 half = (u128)1 << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) q += 1;
    if (q >> 53) { /* rounding carried into a new bit */
      q >>= 1;
      p += 1;
    }
    mant = (uint64_t)q;
  }
  int e2 = p + scale; /* value = mant * 2^(e2 - 52), mant in [2^52, 2^53) */
  uint64_t bits = ((uint64_t)(e2 + 1023) << 52) | (mant & 0x000FFFFFFFFFFFFFull);
  double r;
  memcpy(&r, &bits, sizeof r);
  return r;
}

/* ln(M * 2^E) for an integer 1 <= M < 2^53 and an integer E. */
static double fx_log(uint64_t M, int E) {
  /* reduce: m = M / 2^q in [sqrt(1/2), sqrt(2)) */
  int q = bitlen64(M) - 1;                              /* M / 2^q in [1, 2)          */
  if ((u128)M * M >= ((u128)1 << (2 * q + 1))) q += 1;  /* (M/2^q)^2 >= 2: use m/2    */
  int K = E + q;                                        /* ln(M 2^E) = K ln2 + ln(m)  */
  uint64_t P = (uint64_t)1 << q;
  uint64_t n = M >= P ? M - P : P - M; /* |m - 1| 2^q */
  uint64_t d = M + P;                  /* (m + 1) 2^q */
  int sgn = M > P ? 1 : (M < P ? -1 : 0); /* sign of ln(m) */

  /* L = |ln m| = 2 atanh(|s|), |s| = n / d, held as Lm * 2^Lexp */
  u128 Lm = 0;
  int Lexp = 0;
  if (n != 0) {
    int a = 64 - bitlen64(n), b = 64 - bitlen64(d);   /* leading zero counts */
    uint64_t Nn = n << a, Dn = d << b;                 /* both in [2^63, 2^64) */
    uint64_t Q = (uint64_t)((((u128)Nn) << 63) / Dn);  /* |s| = Q 2^(-63 + b - a)  */
    int sh = a - b - 1;                                /* |s| in Q64 is Q >> sh     */
    uint64_t s64 = sh >= 64 ? 0 : (Q >> sh);
    uint64_t z = mulhi64(s64, s64);                    /* s^2 in Q64 */
    /* F = sum_{i=1..12} z^i / (2i + 1) in Q64, by Horner's rule */
    uint64_t R = 0;
    for (int i = ORACLE_MUTANT == 12 ? 2 : 12; i >= 1; i--) {
      uint64_t ci = (uint64_t)((((u128)1) << 64) / (u128)(2 * i + 1));
      R = ci + mulhi64(z, R);
    }
    uint64_t F = mulhi64(z, R);
    /* L = 2 |s| (1 + F 2^-64) = (Q + Q F 2^-64) 2^(-62 + b - a) */
    Lm = (u128)Q + (u128)mulhi64(Q, F);
    Lexp = -62 + b - a;
  }

  if (K == 0) {
    if (n == 0) return 0.0;
    double r = round_to_double(Lm, Lexp);
    return sgn > 0 ? r : -r;
  }
  /* |K| ln 2 and L in Q64 (128-bit); Lexp + 64 <= 0 always here */
  u128 A = (u128)(uint64_t)(K > 0 ? K : -K) * (u128)LN2_Q64;
  int rs = -(Lexp + 64);
  u128 LQ = n == 0 ? 0 : (rs >= 128 ? 0 : (Lm >> rs));
  if (K > 0) {
    u128 V = sgn >= 0 ? A + LQ : A - LQ; /* K ln2 + sgn L > 0 */
    return round_to_double(V, -64);
  } else {
    u128 V = sgn >= 0 ? A - LQ : A + LQ; /* -(K ln2 + sgn L) > 0 */
    return -round_to_double(V, -64);
  }
}

/* Natural log of a positive finite binary64 value. */
double oracle_rt_log(double x) {
  uint64_t bits;
  memcpy(&bits, &x, sizeof bits);
  int ef = (int)((bits >> 52) & 0x7FF);
  uint64_t frac = bits & 0x000FFFFFFFFFFFFFull;
  if (ef == 0) return fx_log(frac, -1074);           /* subnormal */
  return fx_log(frac | (1ull << 52), ef - 1075);     /* normal    */
}

/* ------------------------------------------------------------------------------ */
/* Random draws                                                                   */
/* ------------------------------------------------------------------------------ */

static void draw_words(uint64_t seed, uint64_t traj, uint32_t k, uint64_t n, uint32_t stream,
                       uint32_t *w0, uint32_t *w1) {
  uint32_t ctr[4] = {(uint32_t)(n >> 1), (uint32_t)traj, k, stream};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  oracle_philox4x32_10(ctr, key, out);
  if (n & 1) { *w0 = out[2]; *w1 = out[3]; }
  else       { *w0 = out[0]; *w1 = out[1]; }
}

/* the odd integer x = 2v + 1 with u = x 2^-53 */
static uint64_t draw_x(uint64_t seed, uint64_t traj, uint32_t k, uint64_t n, uint32_t stream) {
  uint32_t w0, w1;
  draw_words(seed, traj, k, n, stream, &w0, &w1);
  uint64_t v = (((uint64_t)w1 << 32) | w0) >> 12;
  return ORACLE_MUTANT == 13 ? (v | 1) : 2 * v + 1;
}

double oracle_uniform(uint64_t seed, uint64_t traj, uint32_t k, uint64_t n, uint32_t stream) {
  return (double)draw_x(seed, traj, k, n, stream) * 0x1p-53;
}

/* Exp(1) internal-time increment ln(1/u) (Eq. 24) */
double oracle_exp1(uint64_t seed, uint64_t traj, uint32_t k, uint64_t n, uint32_t stream) {
  return -fx_log(draw_x(seed, traj, k, n, stream), -53);
}

/* ------------------------------------------------------------------------------ */
/* Network                                                                        */
/* ------------------------------------------------------------------------------ */

typedef struct {
  int32_t N, M;
  int64_t *rptr; /* reactants of reaction k: rsp/rcoef[rptr[k] .. rptr[k+1]) */
  int32_t *rsp, *rcoef;
  int64_t *vptr; /* net change of reaction k: vsp/vdel[vptr[k] .. vptr[k+1]) */
  int32_t *vsp, *vdel;
  const double *c;
  const uint8_t *enabled; /* NULL: every channel may fire */
  const double *beta;     /* NULL: constant rates; else c_k (1 + beta_k t) */
} onet;

/* Group COO entries by reaction; entries for the same (reaction, species) are summed
 * and zero sums dropped. */
static int group_coo(int32_t M, int64_t nnz, const int32_t *rxn, const int32_t *sp, const int32_t *val,
                     int64_t **ptr_out, int32_t **sp_out, int32_t **val_out) {
  int64_t *ptr = calloc((size_t)M + 1, sizeof *ptr);
  int32_t *osp = malloc(sizeof *osp * (size_t)(nnz > 0 ? nnz : 1));
  int32_t *oval = malloc(sizeof *oval * (size_t)(nnz > 0 ? nnz : 1));
  int64_t *fill = calloc((size_t)M + 1, sizeof *fill);
  if (!ptr || !osp || !oval || !fill) return -1;
  for (int64_t i = 0; i < nnz; i++) ptr[rxn[i] + 1]++;
  for (int32_t k = 0; k < M; k++) ptr[k + 1] += ptr[k];
  for (int64_t i = 0; i < nnz; i++) {
    int32_t k = rxn[i];
    int64_t base = ptr[k];
    int64_t j;
    for (j = 0; j < fill[k]; j++)
      if (osp[base + j] == sp[i]) break;
    if (j < fill[k]) {
      oval[base + j] += val[i];
    } else {
      osp[base + fill[k]] = sp[i];
      oval[base + fill[k]] = val[i];
      fill[k]++;
    }
  }
  /* compact: drop zero sums and the unused tail of each group */
  int64_t w = 0;
  int64_t start = 0;
  for (int32_t k = 0; k < M; k++) {
    int64_t b = start, e = start + fill[k];
    start = ptr[k + 1];
    ptr[k] = w;
    for (int64_t j = b; j < e; j++)
      if (oval[j] != 0) { osp[w] = osp[j]; oval[w] = oval[j]; w++; }
  }
  ptr[M] = w;
  free(fill);
  *ptr_out = ptr; *sp_out = osp; *val_out = oval;
  return 0;
}

static void free_net(onet *g) {
  free(g->rptr); free(g->rsp); free(g->rcoef);
  free(g->vptr); free(g->vsp); free(g->vdel);
}

/* binom(x, s) computed exactly in integers (0 if x < s) */
static int64_t binom(int64_t x, int32_t s) {
  if (x < s) return 0;
  int64_t r = 1;
  for (int32_t i = 0; i < s; i++) r = r * (x - i) / (ORACLE_MUTANT == 1 ? 1 : (i + 1));
  return r;
}

/* a_k = c_k * h_k(X), h_k = prod_j binom(X_j, sigma_jk) (Eq. 1-2) */
static double propensity(const onet *g, int32_t k, const int32_t *X) {
  if (g->enabled && !g->enabled[k]) return 0.0; /* forbidden channel: frozen internal time */
  int64_t h = 1;
  for (int64_t i = g->rptr[k]; i < g->rptr[k + 1]; i++)
    h *= binom(X[g->rsp[ORACLE_MUTANT == 2 ? g->rptr[k] : i]], g->rcoef[i]);
  return g->c[k] * (double)h;
}

/* ------------------------------------------------------------------------------ */
/* Simulation                                                                     */
/* ------------------------------------------------------------------------------ */

enum { ST_TEND = 0, ST_MAX_EVENTS = 1, ST_ABSORBED = 2, ST_OVERFLOW = 3, ST_BAD_X0 = 5 };

/* Waiting time of a channel with base propensity A > 0, rate slope beta and remaining internal
 * time R at time t (Eq. 29 for c(t) = c (1 + beta t)). */
static double tdep_wait(double A, double beta, double R, double t) {
  if (!(R > 0.0)) return 0.0;
  if (beta == 0.0) return R / A;
  double u = 1.0 + (ORACLE_MUTANT == 23 ? 0.0 : beta * t);
  double b = A * u;
  double e = ((2.0 * A) * beta) * R;
  double den = b + sqrt(b * b + e);
  return (2.0 * R) / den;
}

/* int_t^{t+d} (1 + beta s) ds = d (1 + beta t) + beta d^2 / 2 */
static double tdep_integral(double beta, double t, double d) {
  if (beta == 0.0) return d;
  double u = 1.0 + beta * t;
  return d * u + (ORACLE_MUTANT == 22 ? 0.0 : ((beta * d) * d) * 0.5);
}

int64_t oracle_grid_len(double t_end, double sample_dt) {
  if (!(sample_dt > 0.0) || !isfinite(t_end) || t_end < 0.0) return 0;
  return (int64_t)floor(t_end / sample_dt * (1.0 + 1e-12)) + 1;
}

typedef struct {
  const onet *g;
  int32_t mode;
  const int32_t *x0; int per_traj_x0;
  double t_end; int64_t max_events;
  uint64_t seed; uint32_t stream; int64_t traj_offset;
  double sample_dt; int64_t G;
  int32_t *x_final, *grid;
  int64_t *n_events; int32_t *status; double *t_last;
  double *loglik; int32_t *counts; double *t_internal;
  int64_t trace_len; int32_t *trace_mu; double *trace_t;
  int64_t j0, j1;
  int err;
} job_t;

static void run_traj(const job_t *J, int64_t j, double *P, double *T, double *a, int32_t *n, int32_t *X) {
  const onet *g = J->g;
  const int32_t N = g->N, M = g->M;
  const uint64_t gid = (uint64_t)(J->traj_offset + j);
  const int32_t *x0 = J->x0 + (J->per_traj_x0 ? j * (int64_t)N : 0);
  int32_t *grid = J->grid ? J->grid + j * J->G * N : NULL;
  int32_t *trace_mu = J->trace_mu ? J->trace_mu + j * J->trace_len : NULL;
  double *trace_t = J->trace_t ? J->trace_t + j * J->trace_len : NULL;
  for (int64_t i = 0; i < J->trace_len; i++) {
    if (trace_mu) trace_mu[i] = -1;
    if (trace_t) trace_t[i] = 0.0;
  }

  int32_t status = ST_TEND;
  int bad = 0;
  for (int32_t i = 0; i < N; i++) {
    X[i] = x0[i];
    if (x0[i] < 0) bad = 1;
  }
  double t = 0.0, ll = 0.0;
  int64_t ev = 0, gi = 0;

  if (bad) {
    status = ST_BAD_X0;
    for (int32_t k = 0; k < M; k++) { n[k] = 0; T[k] = 0.0; }
  } else {
    /* initialise (Table 2): T_k = 0, P_k = first Exp(1) draw, a_k from X(0) */
    for (int32_t k = 0; k < M; k++) {
      n[k] = 0;
      T[k] = 0.0;
      P[k] = oracle_exp1(J->seed, gid, (uint32_t)k, 0, J->stream);
      a[k] = propensity(g, k, X);
    }
    for (;;) {
      /* waiting time of each channel (Eq. 25) and the first to fire (Eq. 26);
       * ties go to the smallest index */
      double dmin = INFINITY;
      int32_t mu = -1;
      for (int32_t k = 0; k < M; k++) {
        double w;
        if (a[k] == 0.0) {
          w = INFINITY;
        } else if (g->beta) {
          w = tdep_wait(a[k], g->beta[k], P[k] - T[k], t);
        } else {
          double rem = P[k] - (ORACLE_MUTANT == 3 ? 0.0 : T[k]);
          w = rem > 0.0 ? rem / a[k] : 0.0;
        }
        if (ORACLE_MUTANT == 4 ? (w < dmin && mu < 0) : (w < dmin)) { dmin = w; mu = k; }
      }
      if (mu < 0) { status = ST_ABSORBED; break; }
      double tn = t + dmin;
      if (tn > J->t_end) { status = ST_TEND; break; }
      if (ev == J->max_events) { status = ST_MAX_EVENTS; break; }
      int over = 0;
      for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++) {
        int64_t nx = (int64_t)X[g->vsp[i]] + g->vdel[i];
        if (nx > INT32_MAX || nx < 0) over = 1;
      }
      if (over) { status = ST_OVERFLOW; break; }

      /* grid points strictly before the event see the pre-event state */
      if (grid)
        while (gi < J->G && (ORACLE_MUTANT == 10 ? (double)gi * J->sample_dt <= tn + 0.5 * J->sample_dt
                                                    : (double)gi * J->sample_dt < tn)) {
          memcpy(grid + gi * N, X, sizeof(int32_t) * (size_t)N);
          gi++;
        }
      else
        while (gi < J->G && (double)gi * J->sample_dt < tn) gi++;

      double tprev = t;
      t = tn;
      /* every internal time advances by a_k dt (Eq. 17) */
      if (ORACLE_MUTANT == 5) { /* propensities of the post-event state used for the elapsed step */
        for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++) X[g->vsp[i]] += g->vdel[i];
        for (int32_t k = 0; k < M; k++) a[k] = propensity(g, k, X);
        for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++) X[g->vsp[i]] -= g->vdel[i];
      }
      if (g->beta) {
        /* over the step [tprev, t]: int c_k(s) h_k ds = A_k I_k(tprev, dt) */
        for (int32_t k = 0; k < M; k++) T[k] = T[k] + a[k] * tdep_integral(g->beta[k], tprev, dmin);
        if (J->loglik)
          ll = ll + oracle_rt_log(a[mu] * (1.0 + g->beta[mu] * (ORACLE_MUTANT == 24 ? tprev : t)));
      } else {
        for (int32_t k = 0; k < M; k++) T[k] = T[k] + a[k] * (ORACLE_MUTANT == 6 ? t : dmin);
        if (J->loglik) ll = ll + oracle_rt_log(a[mu]);
      }
      /* fire: X += v_mu (Eq. 5) */
      for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++)
        X[g->vsp[i]] += (ORACLE_MUTANT == 7 && g->vdel[i] < 0) ? -g->vdel[i] : g->vdel[i];
      if (trace_mu && ev < J->trace_len) { trace_mu[ev] = mu; trace_t[ev] = t; }
      n[mu] += 1;
      ev += 1;
      /* only the fired channel draws a new increment (Eq. 27) */
      if (ORACLE_MUTANT == 8) P[mu] = oracle_exp1(J->seed, gid, (uint32_t)mu, (uint64_t)n[mu], J->stream);
      else P[mu] = P[mu] + oracle_exp1(J->seed, gid, (uint32_t)mu, (uint64_t)(ORACLE_MUTANT == 9 ? 0 : n[mu]),
                                       J->stream);
      /* propensities from the new state (Eq. 1-2) */
      for (int32_t k = 0; k < M; k++) a[k] = propensity(g, k, X);
    }
  }

  /* remaining grid points: known state if the path ended by t_end or absorption */
  if (grid)
    for (; gi < J->G; gi++)
      for (int32_t i = 0; i < N; i++)
        grid[gi * N + i] = (status == ST_TEND || status == ST_ABSORBED) ? X[i] : -1;

  if (status != ST_BAD_X0 && (status == ST_TEND || status == ST_ABSORBED) && isfinite(J->t_end)) {
    /* internal times at t_end (for the likelihood) */
    double rest = J->t_end - t;
    for (int32_t k = 0; k < M; k++)
      T[k] = T[k] + a[k] * (g->beta ? tdep_integral(g->beta[k], t, rest) : rest);
  }
  if (J->loglik) {
    /* log-likelihood of the path: sum of ln a_mu minus the integrated propensity */
    double sT = 0.0;
    for (int32_t k = 0; k < M; k++) sT = sT + T[k];
    J->loglik[j] = status == ST_BAD_X0 ? NAN : (ORACLE_MUTANT == 11 ? ll + sT : ll - sT);
  }
  if (J->counts) memcpy(J->counts + j * (int64_t)M, n, sizeof(int32_t) * (size_t)M);
  if (J->t_internal) memcpy(J->t_internal + j * (int64_t)M, T, sizeof(double) * (size_t)M);
  if (J->x_final) memcpy(J->x_final + j * (int64_t)N, X, sizeof(int32_t) * (size_t)N);
  if (J->n_events) J->n_events[j] = ev;
  if (J->status) J->status[j] = status;
  if (J->t_last) J->t_last[j] = t;
}

/* Absolute firing time of a channel updated at real time su: su + (P - T) / a
 * (0 remaining internal time gives su), +inf for a = 0 (mode 1). */
static double lazy_tau(double P, double T, double a, double su) {
  if (a == 0.0) return INFINITY;
  double rem = P - T;
  double w = rem > 0.0 ? rem / a : 0.0;
  return ORACLE_MUTANT == 17 ? w : su + w;
}

/* Mode 1: the absolute-time form (see the header).  s[k] is the real time up to
 * which T[k] is accounted, tau[k] the absolute firing time; upd[k] flags the
 * channels an event touches and chg[i] the species it changed. */
static void run_traj_lazy(const job_t *J, int64_t j, double *P, double *T, double *a, int32_t *n, int32_t *X,
                          double *s, double *tau, uint8_t *upd, uint8_t *chg) {
  const onet *g = J->g;
  const int32_t N = g->N, M = g->M;
  const uint64_t gid = (uint64_t)(J->traj_offset + j);
  const int32_t *x0 = J->x0 + (J->per_traj_x0 ? j * (int64_t)N : 0);
  int32_t *grid = J->grid ? J->grid + j * J->G * N : NULL;
  int32_t *trace_mu = J->trace_mu ? J->trace_mu + j * J->trace_len : NULL;
  double *trace_t = J->trace_t ? J->trace_t + j * J->trace_len : NULL;
  for (int64_t i = 0; i < J->trace_len; i++) {
    if (trace_mu) trace_mu[i] = -1;
    if (trace_t) trace_t[i] = 0.0;
  }

  int32_t status = ST_TEND;
  int bad = 0;
  for (int32_t i = 0; i < N; i++) {
    X[i] = x0[i];
    chg[i] = 0;
    if (x0[i] < 0) bad = 1;
  }
  double t = 0.0, ll = 0.0;
  int64_t ev = 0, gi = 0;
  for (int32_t k = 0; k < M; k++) { n[k] = 0; T[k] = 0.0; s[k] = 0.0; a[k] = 0.0; }

  if (bad) {
    status = ST_BAD_X0;
  } else {
    for (int32_t k = 0; k < M; k++) {
      P[k] = oracle_exp1(J->seed, gid, (uint32_t)k, 0, J->stream);
      a[k] = propensity(g, k, X);
      tau[k] = lazy_tau(P[k], T[k], a[k], 0.0);
    }
    for (;;) {
      /* the earliest absolute firing time; ties go to the smallest index */
      double tmin = INFINITY;
      int32_t mu = -1;
      for (int32_t k = 0; k < M; k++)
        if (tau[k] < tmin) { tmin = tau[k]; mu = k; }
      if (mu < 0) { status = ST_ABSORBED; break; }
      double tn = tmin;
      if (tn > J->t_end) { status = ST_TEND; break; }
      if (ev == J->max_events) { status = ST_MAX_EVENTS; break; }
      int over = 0;
      for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++) {
        int64_t nx = (int64_t)X[g->vsp[i]] + g->vdel[i];
        if (nx > INT32_MAX || nx < 0) over = 1;
      }
      if (over) { status = ST_OVERFLOW; break; }
      if (grid)
        while (gi < J->G && (double)gi * J->sample_dt < tn) {
          memcpy(grid + gi * N, X, sizeof(int32_t) * (size_t)N);
          gi++;
        }
      else
        while (gi < J->G && (double)gi * J->sample_dt < tn) gi++;
      t = tn;
      if (J->loglik) ll = ll + oracle_rt_log(a[mu]);
      /* fire: X += v_mu (Eq. 5); the species it changed */
      for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++) {
        X[g->vsp[i]] += g->vdel[i];
        chg[g->vsp[i]] = 1;
      }
      if (trace_mu && ev < J->trace_len) { trace_mu[ev] = mu; trace_t[ev] = t; }
      n[mu] += 1;
      ev += 1;
      /* the channels the event touches: mu, and every channel with a reactant species
       * among the changed ones (the dependency graph, Sec. 5) */
      for (int32_t k = 0; k < M; k++) {
        upd[k] = k == mu;
        for (int64_t i = g->rptr[k]; i < g->rptr[k + 1]; i++)
          if (chg[g->rsp[i]] && !(ORACLE_MUTANT == 16 && i > g->rptr[k])) upd[k] = 1;
      }
      /* their internal times are brought up to the event with the old propensities (Eq. 17) */
      for (int32_t k = 0; k < M; k++)
        if (upd[k]) {
          if (!(ORACLE_MUTANT == 15 && k != mu)) T[k] = T[k] + a[k] * (t - s[k]);
          s[k] = t;
        }
      /* only the fired channel draws a new increment (Eq. 27) */
      P[mu] = P[mu] + oracle_exp1(J->seed, gid, (uint32_t)mu, (uint64_t)n[mu], J->stream);
      /* new propensities (Eq. 1-2) and absolute firing times of the touched channels */
      for (int32_t k = 0; k < M; k++)
        if (upd[k]) {
          a[k] = propensity(g, k, X);
          tau[k] = lazy_tau(P[k], T[k], a[k], t);
        }
      for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++) chg[g->vsp[i]] = 0;
    }
  }

  if (grid)
    for (; gi < J->G; gi++)
      for (int32_t i = 0; i < N; i++)
        grid[gi * N + i] = (status == ST_TEND || status == ST_ABSORBED) ? X[i] : -1;

  if (status != ST_BAD_X0 && ORACLE_MUTANT != 18) {
    /* every channel's internal time up to the end of the run: t_end if the path
     * reached it (or was absorbed before a finite t_end), else the last event */
    double tf = ((status == ST_TEND || status == ST_ABSORBED) && isfinite(J->t_end)) ? J->t_end : t;
    for (int32_t k = 0; k < M; k++) T[k] = T[k] + a[k] * (tf - s[k]);
  }
  if (J->loglik) {
    double sT = 0.0;
    for (int32_t k = 0; k < M; k++) sT = sT + T[k];
    J->loglik[j] = status == ST_BAD_X0 ? NAN : ll - sT;
  }
  if (J->counts) memcpy(J->counts + j * (int64_t)M, n, sizeof(int32_t) * (size_t)M);
  if (J->t_internal) memcpy(J->t_internal + j * (int64_t)M, T, sizeof(double) * (size_t)M);
  if (J->x_final) memcpy(J->x_final + j * (int64_t)N, X, sizeof(int32_t) * (size_t)N);
  if (J->n_events) J->n_events[j] = ev;
  if (J->status) J->status[j] = status;
  if (J->t_last) J->t_last[j] = t;
}

/* Mode 2: Table 3's rescaled form (see the header).  w: relative waiting times, p: the
 * propensities they were computed with, q: frozen remaining internal times. */
static void run_traj_rescaled(const job_t *J, int64_t j, double *w, double *T, double *a, int32_t *n, int32_t *X,
                              double *p, double *q) {
  const onet *g = J->g;
  const int32_t N = g->N, M = g->M;
  const uint64_t gid = (uint64_t)(J->traj_offset + j);
  const int32_t *x0 = J->x0 + (J->per_traj_x0 ? j * (int64_t)N : 0);
  int32_t *grid = J->grid ? J->grid + j * J->G * N : NULL;
  int32_t *trace_mu = J->trace_mu ? J->trace_mu + j * J->trace_len : NULL;
  double *trace_t = J->trace_t ? J->trace_t + j * J->trace_len : NULL;
  for (int64_t i = 0; i < J->trace_len; i++) {
    if (trace_mu) trace_mu[i] = -1;
    if (trace_t) trace_t[i] = 0.0;
  }
  int32_t status = ST_TEND;
  int bad = 0;
  for (int32_t i = 0; i < N; i++) {
    X[i] = x0[i];
    if (x0[i] < 0) bad = 1;
  }
  double t = 0.0, ll = 0.0;
  int64_t ev = 0, gi = 0;
  for (int32_t k = 0; k < M; k++) { n[k] = 0; T[k] = 0.0; a[k] = 0.0; }

  if (bad) {
    status = ST_BAD_X0;
  } else {
    /* initialise (Table 3): a_k, dt_k = ln(1/r_k) / a_k, p_k = a_k */
    for (int32_t k = 0; k < M; k++) {
      double E = oracle_exp1(J->seed, gid, (uint32_t)k, 0, J->stream);
      a[k] = propensity(g, k, X);
      p[k] = a[k];
      if (a[k] > 0.0) { w[k] = E / a[k]; q[k] = 0.0; }
      else { w[k] = INFINITY; q[k] = E; }
    }
    for (;;) {
      /* scan for the smallest waiting time; ties go to the smallest index */
      double dmin = INFINITY;
      int32_t mu = -1;
      for (int32_t k = 0; k < M; k++)
        if (w[k] < dmin) { dmin = w[k]; mu = k; }
      if (mu < 0) { status = ST_ABSORBED; break; }
      double tn = t + dmin;
      if (tn > J->t_end) { status = ST_TEND; break; }
      if (ev == J->max_events) { status = ST_MAX_EVENTS; break; }
      int over = 0;
      for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++) {
        int64_t nx = (int64_t)X[g->vsp[i]] + g->vdel[i];
        if (nx > INT32_MAX || nx < 0) over = 1;
      }
      if (over) { status = ST_OVERFLOW; break; }
      if (grid)
        while (gi < J->G && (double)gi * J->sample_dt < tn) {
          memcpy(grid + gi * N, X, sizeof(int32_t) * (size_t)N);
          gi++;
        }
      else
        while (gi < J->G && (double)gi * J->sample_dt < tn) gi++;
      t = tn;
      for (int32_t k = 0; k < M; k++) T[k] = T[k] + a[k] * dmin;
      if (J->loglik) ll = ll + oracle_rt_log(a[mu]);
      for (int64_t i = g->vptr[mu]; i < g->vptr[mu + 1]; i++) X[g->vsp[i]] += g->vdel[i];
      if (trace_mu && ev < J->trace_len) { trace_mu[ev] = mu; trace_t[ev] = t; }
      n[mu] += 1;
      ev += 1;
      /* recalculate every propensity; rescale every other waiting time; redraw the fired one */
      for (int32_t k = 0; k < M; k++) {
        double an = propensity(g, k, X);
        if (k == mu) {
          double E = oracle_exp1(J->seed, gid, (uint32_t)mu,
                                 (uint64_t)(ORACLE_MUTANT == 20 ? n[mu] - 1 : n[mu]), J->stream);
          if (an > 0.0) w[k] = E / an;
          else { q[k] = E; w[k] = INFINITY; }
        } else if (p[k] > 0.0) {
          double rem = w[k] - dmin;
          if (an > 0.0) w[k] = ORACLE_MUTANT == 19 ? rem : (p[k] / an) * rem;
          else { q[k] = p[k] * rem; w[k] = INFINITY; }
        } else if (an > 0.0) {
          w[k] = (ORACLE_MUTANT == 21 ? 0.0 : q[k]) / an;
        }
        p[k] = an;
        a[k] = an;
      }
    }
  }

  if (grid)
    for (; gi < J->G; gi++)
      for (int32_t i = 0; i < N; i++)
        grid[gi * N + i] = (status == ST_TEND || status == ST_ABSORBED) ? X[i] : -1;
  if (status != ST_BAD_X0 && (status == ST_TEND || status == ST_ABSORBED) && isfinite(J->t_end)) {
    double rest = J->t_end - t;
    for (int32_t k = 0; k < M; k++) T[k] = T[k] + a[k] * rest;
  }
  if (J->loglik) {
    double sT = 0.0;
    for (int32_t k = 0; k < M; k++) sT = sT + T[k];
    J->loglik[j] = status == ST_BAD_X0 ? NAN : ll - sT;
  }
  if (J->counts) memcpy(J->counts + j * (int64_t)M, n, sizeof(int32_t) * (size_t)M);
  if (J->t_internal) memcpy(J->t_internal + j * (int64_t)M, T, sizeof(double) * (size_t)M);
  if (J->x_final) memcpy(J->x_final + j * (int64_t)N, X, sizeof(int32_t) * (size_t)N);
  if (J->n_events) J->n_events[j] = ev;
  if (J->status) J->status[j] = status;
  if (J->t_last) J->t_last[j] = t;
}

static void *worker(void *arg) {
  job_t *J = (job_t *)arg;
  int32_t M = J->g->M, N = J->g->N;
  double *P = malloc(sizeof(double) * (size_t)M), *T = malloc(sizeof(double) * (size_t)M);
  double *a = malloc(sizeof(double) * (size_t)M);
  int32_t *n = malloc(sizeof(int32_t) * (size_t)M), *X = malloc(sizeof(int32_t) * (size_t)N);
  double *s = malloc(sizeof(double) * (size_t)M), *tau = malloc(sizeof(double) * (size_t)M);
  uint8_t *upd = malloc((size_t)M), *chg = malloc((size_t)N);
  if (!P || !T || !a || !n || !X || !s || !tau || !upd || !chg) {
    J->err = -4;
  } else {
    for (int64_t j = J->j0; j < J->j1; j++) {
      if (J->mode == 1) run_traj_lazy(J, j, P, T, a, n, X, s, tau, upd, chg);
      else if (J->mode == 2) run_traj_rescaled(J, j, P, T, a, n, X, s, tau);
      else run_traj(J, j, P, T, a, n, X);
    }
  }
  free(P); free(T); free(a); free(n); free(X); free(s); free(tau); free(upd); free(chg);
  return NULL;
}

/*
 * Run n_traj trajectories (global ids traj_offset + j) of one network in the given
 * mode (0: Table 2 internal-time form, 1: absolute-time form, 2: Table 3's rescaled
 * form; see the header).
 * Output arrays may be NULL.  Returns 0, -1 for invalid arguments, -4 for
 * allocation failure.
 */
int oracle_run(int32_t mode, int32_t N, int32_t M,
               int64_t n_reac_nz, const int32_t *reac_rxn, const int32_t *reac_sp, const int32_t *reac_coef,
               int64_t n_stoi_nz, const int32_t *stoi_rxn, const int32_t *stoi_sp, const int32_t *stoi_delta,
               const double *c, const uint8_t *enabled, const double *beta, const int32_t *x0, int32_t per_traj_x0,
               double t_end, int64_t max_events, uint64_t seed, uint32_t stream,
               int64_t n_traj, int64_t traj_offset, double sample_dt,
               int32_t *x_final, int32_t *grid, int64_t *n_events, int32_t *status, double *t_last,
               double *loglik, int32_t *counts, double *t_internal,
               int64_t trace_len, int32_t *trace_mu, double *trace_t, int32_t n_threads) {
  if (mode < 0 || mode > 2 || N < 1 || M < 1 || n_traj < 0 || max_events < 0 || t_end != t_end) return -1;
  if (beta) {
    if (mode != 0) return -1;
    for (int32_t k = 0; k < M; k++)
      if (!(beta[k] >= 0.0) || !isfinite(beta[k])) return -1;
  }
  for (int64_t i = 0; i < n_reac_nz; i++)
    if (reac_rxn[i] < 0 || reac_rxn[i] >= M || reac_sp[i] < 0 || reac_sp[i] >= N || reac_coef[i] <= 0)
      return -1;
  for (int64_t i = 0; i < n_stoi_nz; i++)
    if (stoi_rxn[i] < 0 || stoi_rxn[i] >= M || stoi_sp[i] < 0 || stoi_sp[i] >= N) return -1;
  onet g;
  g.N = N; g.M = M; g.c = c; g.enabled = enabled; g.beta = beta;
  if (group_coo(M, n_reac_nz, reac_rxn, reac_sp, reac_coef, &g.rptr, &g.rsp, &g.rcoef)) return -4;
  if (group_coo(M, n_stoi_nz, stoi_rxn, stoi_sp, stoi_delta, &g.vptr, &g.vsp, &g.vdel)) return -4;

  int64_t G = grid ? oracle_grid_len(t_end, sample_dt) : 0;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_traj) n_threads = n_traj > 0 ? (int32_t)n_traj : 1;
  job_t *jobs = calloc((size_t)n_threads, sizeof *jobs);
  pthread_t *th = calloc((size_t)n_threads, sizeof *th);
  int rc = 0;
  for (int32_t w = 0; w < n_threads; w++) {
    job_t *J = &jobs[w];
    J->g = &g; J->mode = mode; J->x0 = x0; J->per_traj_x0 = per_traj_x0;
    J->t_end = t_end; J->max_events = max_events; J->seed = seed; J->stream = stream;
    J->traj_offset = traj_offset; J->sample_dt = sample_dt; J->G = G;
    J->x_final = x_final; J->grid = grid; J->n_events = n_events; J->status = status; J->t_last = t_last;
    J->loglik = loglik; J->counts = counts; J->t_internal = t_internal;
    J->trace_len = trace_mu || trace_t ? trace_len : 0; J->trace_mu = trace_mu; J->trace_t = trace_t;
    J->j0 = n_traj * w / n_threads; J->j1 = n_traj * (w + 1) / n_threads;
  }
  if (n_threads == 1) {
    worker(&jobs[0]);
  } else {
    for (int32_t w = 0; w < n_threads; w++) pthread_create(&th[w], NULL, worker, &jobs[w]);
    for (int32_t w = 0; w < n_threads; w++) pthread_join(th[w], NULL);
  }
  for (int32_t w = 0; w < n_threads; w++)
    if (jobs[w].err) rc = jobs[w].err;
  free(jobs); free(th);
  free_net(&g);
  return rc;
}

/*
 * Gradient of sum_j w_j l_j with respect to c:
 *   dl_j/dc_k = n_jk / c_k - int h_k dt = (n_jk - T_jk(t_end)) / c_k,
 * since T_k = c_k int h_k dt for a constant rate.  Summed over j in index order.
 */
void oracle_loglik_backward(int32_t M, int64_t n_traj, const double *grad_ll, const int32_t *counts,
                            const double *t_internal, const double *c, double *grad_c) {
  for (int32_t k = 0; k < M; k++) {
    double s = 0.0;
    for (int64_t j = 0; j < n_traj; j++)
      s = s + grad_ll[j] * (((double)counts[j * M + k] - t_internal[j * M + k]) / c[k]);
    grad_c[k] = s;
  }
}

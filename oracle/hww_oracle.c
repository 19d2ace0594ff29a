/*
 * hww_oracle.c -- plain, slow, FP64 CPU oracle of one time step of the
 * hybrid weight-window (HWW) Monte Carlo method of Shaw & Anistratov
 * (arXiv 2512.19925).
 *
 * TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU-baseline leg
 * of the benchmark may use it; the library never does.  It shares no code
 * with the CUDA path.
 *
 * What each part follows in the paper:
 *   transport physics ............ Sec. 3, Eq. (HO_transport), BCs and IC
 *   weight-window center ......... Sec. 2, Eq. (ww-center); ceiling/floor Eq. (ww-c&f)
 *   split / roulette ............. Sec. 2 (N_d = ceil(w/ww), survival p = w/ww)
 *   track-length tally ........... Sec. 3, Eq. (phi-mc)
 *   time-crossing (census) tally . Sec. 3, Eq. (ct-mc); edge current by linear
 *                                  interpolation of adjacent cell averages
 *   LOSM equations ............... Sec. 3, Eqs. (losm), (theta-scheme),
 *                                  (losm-0), (losm-1), (losm-disc-bc)
 *   semi-implicit HLOSM .......... Sec. 3, Eqs. (losm-1-semi), (losm-disc-bc-semi)
 *   moving-average filter ........ Sec. 4, Eq. (moving_average)
 *   uniform combing .............. Sec. 5.1 (population control)
 *   derivatives .................. not in the paper: likelihood-ratio (score
 *                                  function) tallies of d/d(Sigma_t, c) per
 *                                  region, carried through the games and the
 *                                  comb, and the adjoint of the fully implicit
 *                                  LOSM solve of Sec. 3 (its transpose system)
 * Readings of passages the paper leaves open are listed next to the code
 * that takes them.
 *
 * Floating point: every operation below is a single IEEE-754 double
 * operation in the order written (build with -ffp-contract=off, no
 * -ffast-math); fma() appears only where the numerics contract names it.
 * Tallies are accumulated as 128-bit fixed-point integers, so their value does
 * not depend on the order in which particles are processed.
 */
#include "hww_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Numerics contract                                                        */
/* ------------------------------------------------------------------------ */

enum { OR_VACUUM = 0, OR_REFLECT = 1 };
enum { OR_MODE_HWW = 0, OR_MODE_ANALOG = 1, OR_MODE_LWW = 2 };
enum { OR_SCALE_MEAN_WEIGHT = 0, OR_SCALE_LITERAL = 1 };
#define OR_MAX_UPDATES 16
#define OR_MAX_C 16.0                  /* largest mean number of particles per collision */
#define SECONDARY_EVENT 0x80000000u    /* lineage namespace of a collision's extra particles */
enum {
    K_TL_PHI = 0, K_TL_J, K_TL_F, K_CEN_PHI, K_CEN_J, K_CEN_F, K_BATCH_PHI, K_BOUNDARY,
    K_WW_CENTER, K_CLOSURE_PHI, K_CLOSURE_J, K_CLOSURE_F
};
enum { E_ARG = -1, E_STATE = -2, E_OOM = -3, E_NUMERIC = -6 };

#define MAX_EVENTS_PER_TRACK (1u << 30)
#define MAX_DAUGHTERS (1u << 24)
#define GRAZE_MU 0.01 /* surface-estimator cutoff: 1/|mu| -> 2/GRAZE_MU below it */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplications with a Weyl-sequence key schedule. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on the open interval (0,1): the top 52 bits of the 64-bit word
 * hi:lo, offset by half a unit, scaled by 2^-52.  Exact in double. */
double or_u01(uint32_t lo, uint32_t hi) {
    uint64_t x = ((uint64_t)hi << 32) | lo;
    return ((double)(x >> 12) + 0.5) * 0x1p-52;
}

/* Natural logarithm of a positive normal double (u in (0, 1) here) by
 * table-driven reduction:
 *   u = 2^e m, m in [1, 2); j = the top 7 bits of m's mantissa;
 *   j < 64:  c = 1 + j/128,           IC_j = 1/c rounded,       K_j = 0;
 *   j >= 64: c = (1 + (j+1)/128) / 2, IC_j = (1/c rounded) / 2, K_j = 1;
 *   r = m IC_j - 1 (one fused multiply-add; |r| < 2^-7),
 *   log u = (e + K_j) ln 2 + T_j + log1p(r),  T_j = -log(IC_j 2^K_j),
 * with log1p(r) = r + r^2 (-1/2 + r/3 - ... + r^7/9) by Horner's rule
 * (the next term is below 2^-64 of r) and ln 2 split into a 32-bit head and
 * a tail.  The centers next to 1 are 1 itself (T = 0, r exact), and T and
 * log1p(r) share a sign whenever e + K_j = 0, so nothing cancels; the error
 * stays within 2 ulp.  T_j is log(IC_j 2^K_j) rounded once to double: this
 * file computes it at first use in double-double arithmetic (atanh series),
 * which is accurate to about 2^-100, far inside the rounding.  The device
 * implements the same steps from its own table. */
static const double LN2_HI = 0x1.62e42fee00000p-1;
static const double LN2_LO = 0x1.a39ef35793c76p-33;

typedef struct {
    double hi, lo;
} dd;

static dd dd_two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = {s, e};
    return r;
}
static dd dd_norm(double hi, double lo) {
    double s = hi + lo;
    double e = lo - (s - hi);
    dd r = {s, e};
    return r;
}
static dd dd_add(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    return dd_norm(s.hi, s.lo + (a.lo + b.lo));
}
static dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e = e + (a.hi * b.lo + a.lo * b.hi);
    return dd_norm(p, e);
}
static dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd qb = dd_mul((dd){q1, 0.0}, b);
    dd rem = dd_add(a, (dd){-qb.hi, -qb.lo});
    double q2 = rem.hi / b.hi;
    dd qqb = dd_mul((dd){q2, 0.0}, b);
    rem = dd_add(rem, (dd){-qqb.hi, -qqb.lo});
    double q3 = rem.hi / b.hi;
    dd q = dd_norm(q1, q2);
    return dd_add(q, (dd){q3, 0.0});
}

/* log(y) for y in [1/2, 2] in double-double: 2 atanh(s), s = (y-1)/(y+1) */
static dd dd_log(double y) {
    dd num = {y - 1.0, 0.0}; /* exact (Sterbenz) */
    dd den = dd_two_sum(y, 1.0);
    dd sv = dd_div(num, den);
    dd s2 = dd_mul(sv, sv);
    dd term = sv, sum = sv;
    for (int n = 1; n < 40; ++n) {
        term = dd_mul(term, s2);
        dd t = dd_div(term, (dd){(double)(2 * n + 1), 0.0});
        sum = dd_add(sum, t);
        if (fabs(t.hi) < 0x1p-110 * fabs(sum.hi)) break;
    }
    return dd_add(sum, sum);
}

static double LOG_IC[128], LOG_T[128];
static int log_table_ready = 0;

static void log_table_init(void) {
    for (int j = 0; j < 128; ++j) {
        double ic, y;
        if (j < 64) {
            const double c = 1.0 + (double)j / 128.0;
            ic = 1.0 / c;
            y = ic;
        } else {
            const double c = (1.0 + (double)(j + 1) / 128.0) * 0.5;
            const double inv = 1.0 / c;
            ic = inv * 0.5;
            y = inv;
        }
        LOG_IC[j] = ic;
        /* the normalized double-double's head is the rounding; log 1 = +0 */
        LOG_T[j] = (y == 1.0) ? 0.0 : -dd_log(y).hi;
    }
    log_table_ready = 1;
}

void or_log_table(int32_t j, double* ic, double* t) {
    if (!log_table_ready) log_table_init();
    *ic = LOG_IC[j & 127];
    *t = LOG_T[j & 127];
}

double or_log(double u) {
    if (!log_table_ready) log_table_init();
    uint64_t b;
    memcpy(&b, &u, sizeof b);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const uint64_t mant = b & 0x000fffffffffffffull;
    const uint64_t mb = mant | 0x3ff0000000000000ull; /* m in [1,2) */
    double m;
    memcpy(&m, &mb, sizeof m);
    const int j = (int)(mant >> 45);
    const double r = fma(m, LOG_IC[j], -1.0);
    double q = 1.0 / 9.0;
    q = fma(q, r, -1.0 / 8.0);
    q = fma(q, r, 1.0 / 7.0);
    q = fma(q, r, -1.0 / 6.0);
    q = fma(q, r, 1.0 / 5.0);
    q = fma(q, r, -1.0 / 4.0);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -1.0 / 2.0);
    const double r2 = r * r;
    const double p = fma(r2, q, r);
    const double kd = (double)(e + (j >> 6));
    const double hi = fma(kd, LN2_HI, LOG_T[j]);
    const double lo = fma(kd, LN2_LO, p);
    return hi + lo;
}

/* 128-bit two's-complement accumulator and its conversion to double:
 * values that fit a signed 64-bit integer convert in one rounding,
 * wider values as hi*2^64 + lo (two roundings). */
typedef __int128 i128;

static double conv128(i128 a) {
    if (a >= -(i128)0x7fffffffffffffffLL - 1 && a <= (i128)0x7fffffffffffffffLL)
        return (double)(int64_t)a;
    int64_t hi = (int64_t)(a >> 64);
    uint64_t lo = (uint64_t)a;
    return (double)hi * 0x1p64 + (double)lo;
}

/* exponent E of w_bar (w_bar = m 2^E, m in [1,2)); 0 for w_bar == 0 */
static int wbar_exponent(double wbar) {
    if (!(wbar > 0.0)) return 0;
    int e;
    frexp(wbar, &e);   /* wbar = f 2^e, f in [0.5,1) */
    return e - 1;
}

static int bit_length(int64_t n) {
    int l = 0;
    while (n > 0) { ++l; n >>= 1; }
    return l;
}

/* ------------------------------------------------------------------------ */
/* Problem state                                                            */
/* ------------------------------------------------------------------------ */

#define MAX_DERIV 8 /* 2R scores, R <= 4 regions */

typedef struct {
    double x, mu, tau, w;
    int32_t cell;
    uint32_t id;
    uint64_t lin;
    uint32_t e;
    double S[MAX_DERIV]; /* likelihood-ratio scores: Sigma_t of region r at r, c at R + r */
} or_particle;

typedef struct {
    double x, mu, w;
    int32_t cell;
    uint32_t id;
    uint64_t lin;
    double S[MAX_DERIV];
} or_census;

struct or_problem {
    or_desc d;
    int32_t I;
    double *edges, *dx, *sigt, *inv_sigt, *c, *siga;
    int xs_set, ww_set;
    double rho, eps;
    int32_t mode, scaling;
    int32_t n_updates;                 /* in-step window updates u_ww (Sec. 3, Eq. Hpn) */
    double ww_frac[OR_MAX_UPDATES];    /* their history fractions f_p */
    int64_t N;           /* particles per step = source particles */
    int64_t n;           /* completed steps */
    /* combed bank for the next step (x, mu, cell); weight w_bar each */
    double *bx, *bmu;
    int32_t* bcell;
    int64_t nbank;
    double wbar;
    /* WW arrays for the current step */
    double *ww_c, *ww_hi, *ww_lo;
    double* ww_override;
    int has_override;
    /* fixed-point tallies of the last step (scale 2^(40-E)) */
    i128 *tl_phi, *tl_j, *tl_f, *cen_w, *cen_wmu, *cen_wf, *batch;
    i128 bnd[6];
    int tally_shift;
    /* closure / IC vectors at the end of the last step (paper indexing) */
    double *clo_phi, *clo_J, *clo_F; /* I+2, I+1, I+2 */
    double clo_PL, clo_PR;
    /* LOSM solutions of the last step */
    double *semi_phi, *semi_J, *full_phi, *full_J;
    /* previous-step track-length flux (for lagged windows) */
    double* prev_tl_phi;
    int has_prev_tl;
    int bank_loaded; /* the next step starts from a loaded bank */
    /* derivatives (R regions, 2R parameters) */
    int R;
    int32_t* region;
    double* inv_c;
    double* bS;                        /* N x 2R scores of the combed bank */
    i128 *dtl, *dcen, *dbnd;           /* [2R][I], [3][2R][I], [2R][6] */
    double *dclo_phi, *dclo_J, *dclo_F;          /* derivative closure set at t^n */
    double *dclo_PL, *dclo_PR;                   /* [2R] */
    double *dold_phi, *dold_J, *dold_F;          /* ... at the step start */
    double *last_phi_old, *last_J_old, *last_F_old; /* closure set at the step start */
    double last_PL_old, last_PR_old;
    /* census bank of the last step */
    or_census* census;
    int64_t ncensus;
};

static void* xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

int or_create(const or_desc* d, or_problem** out) {
    if (!d || !out) return E_ARG;
    *out = NULL;
    int32_t I = d->n_cells;
    if (I < 1 || !d->edges || !(d->v > 0) || !(d->dt > 0) || d->particles_per_step < 1 ||
        d->particles_per_step >= (1LL << 30) || (d->theta != 0.5 && d->theta != 1.0) ||
        d->n_var_batches < 1 || d->bc_left < 0 || d->bc_left > 1 || d->bc_right < 0 ||
        d->bc_right > 1 || d->filter < 0 || d->filter > 2 || (d->filter == 1 && d->filter_k < 1) ||
        (d->filter == 2 && d->filter_k < 0) ||
        d->deriv_regions < 0 || 2 * d->deriv_regions > MAX_DERIV)
        return E_ARG;
    for (int32_t i = 0; i < I; ++i)
        if (!(d->edges[i + 1] > d->edges[i])) return E_ARG;
    if (!(d->src_x >= d->edges[0] && d->src_x <= d->edges[I])) return E_ARG;
    or_problem* p = (or_problem*)calloc(1, sizeof *p);
    if (!p) return E_OOM;
    p->d = *d;
    p->I = I;
    p->N = d->particles_per_step;
    p->edges = xcalloc(I + 1, sizeof(double));
    p->dx = xcalloc(I, sizeof(double));
    p->sigt = xcalloc(I, sizeof(double));
    p->inv_sigt = xcalloc(I, sizeof(double));
    p->c = xcalloc(I, sizeof(double));
    p->siga = xcalloc(I, sizeof(double));
    p->ww_c = xcalloc(I, sizeof(double));
    p->ww_hi = xcalloc(I, sizeof(double));
    p->ww_lo = xcalloc(I, sizeof(double));
    p->ww_override = xcalloc(I, sizeof(double));
    p->tl_phi = xcalloc(I, sizeof(i128));
    p->tl_j = xcalloc(I, sizeof(i128));
    p->tl_f = xcalloc(I, sizeof(i128));
    p->cen_w = xcalloc(I, sizeof(i128));
    p->cen_wmu = xcalloc(I, sizeof(i128));
    p->cen_wf = xcalloc(I, sizeof(i128));
    p->batch = xcalloc((size_t)I * d->n_var_batches, sizeof(i128));
    p->clo_phi = xcalloc(I + 2, sizeof(double));
    p->clo_J = xcalloc(I + 1, sizeof(double));
    p->clo_F = xcalloc(I + 2, sizeof(double));
    p->semi_phi = xcalloc(I + 2, sizeof(double));
    p->semi_J = xcalloc(I + 1, sizeof(double));
    p->full_phi = xcalloc(I + 2, sizeof(double));
    p->full_J = xcalloc(I + 1, sizeof(double));
    p->prev_tl_phi = xcalloc(I, sizeof(double));
    if (!p->edges || !p->dx || !p->sigt || !p->inv_sigt || !p->c || !p->siga || !p->ww_c ||
        !p->ww_hi || !p->ww_lo || !p->ww_override || !p->tl_phi || !p->tl_j || !p->tl_f ||
        !p->cen_w || !p->cen_wmu || !p->cen_wf || !p->batch || !p->clo_phi || !p->clo_J ||
        !p->clo_F || !p->semi_phi || !p->semi_J || !p->full_phi || !p->full_J || !p->prev_tl_phi) {
        or_destroy(p);
        return E_OOM;
    }
    p->R = d->deriv_regions;
    p->region = xcalloc(I, sizeof(int32_t));
    p->inv_c = xcalloc(I, sizeof(double));
    p->last_phi_old = xcalloc(I + 2, sizeof(double));
    p->last_J_old = xcalloc(I + 1, sizeof(double));
    p->last_F_old = xcalloc(I + 2, sizeof(double));
    if (p->R > 0) {
        const int P2 = 2 * p->R;
        p->dtl = xcalloc((size_t)P2 * I, sizeof(i128));
        p->dcen = xcalloc((size_t)3 * P2 * I, sizeof(i128));
        p->dbnd = xcalloc((size_t)6 * P2, sizeof(i128));
        p->dclo_PL = xcalloc((size_t)P2, sizeof(double));
        p->dclo_PR = xcalloc((size_t)P2, sizeof(double));
        p->dclo_phi = xcalloc((size_t)P2 * (I + 2), sizeof(double));
        p->dclo_J = xcalloc((size_t)P2 * (I + 1), sizeof(double));
        p->dclo_F = xcalloc((size_t)P2 * (I + 2), sizeof(double));
        p->dold_phi = xcalloc((size_t)P2 * (I + 2), sizeof(double));
        p->dold_J = xcalloc((size_t)P2 * (I + 1), sizeof(double));
        p->dold_F = xcalloc((size_t)P2 * (I + 2), sizeof(double));
        if (!p->dtl || !p->dcen || !p->dbnd || !p->dclo_PL || !p->dclo_PR || !p->dclo_phi || !p->dclo_J || !p->dclo_F || !p->dold_phi || !p->dold_J ||
            !p->dold_F) {
            or_destroy(p);
            return E_OOM;
        }
    }
    if (!p->region || !p->inv_c || !p->last_phi_old || !p->last_J_old || !p->last_F_old) {
        or_destroy(p);
        return E_OOM;
    }
    memcpy(p->edges, d->edges, sizeof(double) * (I + 1));
    p->d.edges = p->edges;
    for (int32_t i = 0; i < I; ++i) p->dx[i] = p->edges[i + 1] - p->edges[i];
    p->wbar = 1.0;
    p->rho = 1.0;
    p->eps = 1e-3;
    *out = p;
    return 0;
}

void or_destroy(or_problem* p) {
    if (!p) return;
    free(p->edges); free(p->dx); free(p->sigt); free(p->inv_sigt); free(p->c); free(p->siga);
    free(p->bx); free(p->bmu); free(p->bcell);
    free(p->ww_c); free(p->ww_hi); free(p->ww_lo); free(p->ww_override);
    free(p->tl_phi); free(p->tl_j); free(p->tl_f); free(p->cen_w); free(p->cen_wmu);
    free(p->cen_wf); free(p->batch);
    free(p->clo_phi); free(p->clo_J); free(p->clo_F);
    free(p->semi_phi); free(p->semi_J); free(p->full_phi); free(p->full_J);
    free(p->prev_tl_phi);
    free(p->census);
    free(p->region); free(p->inv_c); free(p->bS); free(p->dtl); free(p->dcen); free(p->dbnd); free(p->dclo_PL); free(p->dclo_PR);
    free(p->dclo_phi); free(p->dclo_J); free(p->dclo_F);
    free(p->dold_phi); free(p->dold_J); free(p->dold_F);
    free(p->last_phi_old); free(p->last_J_old); free(p->last_F_old);
    free(p);
}

/* c is the mean number of particles a collision emits, (Sigma_s + nu_f
 * Sigma_f) / Sigma_t (Eq. HO_transport): c <= 1 a scattering-absorbing
 * medium, c > 1 a multiplying one (up to OR_MAX_C); Sigma_a of the LOSM
 * equations is Sigma_t (1 - c).  Derivative runs need c <= 1. */
int or_set_cross_sections(or_problem* p, const double* sigma_t, const double* c) {
    if (!p || !sigma_t || !c) return E_ARG;
    for (int32_t i = 0; i < p->I; ++i)
        if (!(sigma_t[i] > 0) || !(c[i] >= 0 && c[i] <= OR_MAX_C) || !isfinite(sigma_t[i]) ||
            (p->R > 0 && c[i] > 1.0))
            return E_ARG;
    for (int32_t i = 0; i < p->I; ++i) {
        p->sigt[i] = sigma_t[i];
        p->inv_sigt[i] = 1.0 / sigma_t[i];
        p->c[i] = c[i];
        p->siga[i] = sigma_t[i] * (1.0 - c[i]); /* Sigma_t - Sigma_s - nu_f Sigma_f */
        p->inv_c[i] = (c[i] > 0.0) ? 1.0 / c[i] : 0.0;
    }
    p->xs_set = 1;
    return 0;
}

int or_set_ww_updates(or_problem* p, int32_t n, const double* fractions) {
    if (!p || n < 0 || n > OR_MAX_UPDATES) return E_ARG;
    for (int32_t k = 0; k < n; ++k) {
        /* default f_p = p / (u + 1) (the fractions the paper uses) */
        const double f = fractions ? fractions[k] : (double)(k + 1) / (double)(n + 1);
        if (!(f > 0.0 && f < 1.0) || (k > 0 && !(f > p->ww_frac[k - 1]))) return E_ARG;
        p->ww_frac[k] = f;
    }
    p->n_updates = n;
    return 0;
}

int or_set_ww_params(or_problem* p, double rho, double eps_min, int32_t mode, int32_t scaling) {
    if (!p || !(rho >= 1.0) || !(eps_min > 0.0 && eps_min <= 1.0) || mode < 0 || mode > 2 ||
        scaling < 0 || scaling > 1)
        return E_ARG;
    p->rho = rho;
    p->eps = eps_min;
    p->mode = mode;
    p->scaling = scaling;
    p->ww_set = 1;
    return 0;
}

int or_set_regions(or_problem* p, const int32_t* region) {
    if (!p || !region) return E_ARG;
    for (int32_t i = 0; i < p->I; ++i)
        if (region[i] < 0 || (p->R > 0 && region[i] >= p->R)) return E_ARG;
    memcpy(p->region, region, sizeof(int32_t) * p->I);
    return 0;
}

int or_set_ww_centers(or_problem* p, const double* centers) {
    if (!p || !centers) return E_ARG;
    for (int32_t i = 0; i < p->I; ++i) {
        if (!(centers[i] > 0)) return E_ARG;
        p->ww_override[i] = centers[i];
    }
    p->has_override = 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Moving-average filter, Eq. (moving_average)                              */
/* Reading: the base shrinks symmetrically near the ends,                   */
/* k_m = min(k, m-1, M-m) for 1-based m, so the window never leaves the     */
/* vector and the end values are kept.                                      */
/* ------------------------------------------------------------------------ */
int or_ma_filter(const double* in, double* out, int32_t m, int32_t k) {
    if (!in || !out || m < 0 || k < 0) return E_ARG;
    for (int32_t j = 1; j <= m; ++j) {
        int32_t kk = k;
        if (j - 1 < kk) kk = j - 1;
        if (m - j < kk) kk = m - j;
        double s = 0.0;
        for (int32_t l = -kk; l <= kk; ++l) s = s + in[j - l - 1];
        out[j - 1] = s / (double)(2 * kk + 1);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Fourier low-pass filter, Eqs. (fft), (ifft) and the cutoff between them   */
/* The DFT of the vector, the modes above the cutoff set to zero, the       */
/* inverse DFT.  Reading: the printed sums run j = 1..M, which puts the     */
/* constant mode at j = M; a low-pass filter keeps the constant mode and    */
/* both signs of every frequency up to kappa, i.e. the modes with           */
/* min(j, M - j) <= kappa (0-based j), which keeps the result real.  The    */
/* angles are reduced exactly, 2 pi ((j m) mod M) / M.                      */
/* ------------------------------------------------------------------------ */
int or_fourier_filter(const double* in, double* out, int32_t M, int32_t kappa) {
    if (!in || !out || M < 0 || kappa < 0) return E_ARG;
    double* Xr = xcalloc(M ? M : 1, sizeof(double));
    double* Xi = xcalloc(M ? M : 1, sizeof(double));
    if (!Xr || !Xi) {
        free(Xr); free(Xi);
        return E_OOM;
    }
    const double two_pi = 6.283185307179586476925286766559;
    for (int32_t j = 0; j < M; ++j) {
        double re = 0.0, im = 0.0;
        for (int32_t m = 0; m < M; ++m) {
            const double ang = two_pi * (double)(((int64_t)j * m) % M) / (double)M;
            re = re + in[m] * cos(ang);
            im = im - in[m] * sin(ang);
        }
        const int32_t f = (j < M - j) ? j : M - j;
        Xr[j] = (f <= kappa) ? re : 0.0;
        Xi[j] = (f <= kappa) ? im : 0.0;
    }
    for (int32_t m = 0; m < M; ++m) {
        double acc = 0.0;
        for (int32_t j = 0; j < M; ++j) {
            const double ang = two_pi * (double)(((int64_t)j * m) % M) / (double)M;
            acc = acc + (Xr[j] * cos(ang) - Xi[j] * sin(ang));
        }
        out[m] = acc / (double)M;
    }
    free(Xr);
    free(Xi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* LOSM solve, Eqs. (losm-0), (losm-1), (losm-disc-bc)                       */
/*                                                                          */
/* Unknowns in interleaved order u = (phi_0, J_0, phi_1, J_1, ..., phi_I,   */
/* J_I, phi_{I+1}); rows: 0 left BC, 2i+1 first-moment equation on the     */
/* half cells around edge x_i (i = 0..I), 2i balance on cell i (i = 1..I), */
/* 2I+2 right BC.  The matrix is tridiagonal in this order and is solved   */
/* by Gaussian elimination with partial pivoting (two rows compete per     */
/* column, one extra super-diagonal of fill).                              */
/*                                                                          */
/* Arrays follow the paper's 1-based cell indexing:                         */
/*   dx, sigma_t, sigma_a, q_*  : length I, entry i-1 is cell i            */
/*   phi_old, F_old, F_new      : length I+2 (boundary, cells 1..I, boundary)*/
/*   J_old, J_new               : length I+1 (edges x_0..x_I)              */
/* Readings:                                                                 */
/*  - the sign of the old-level gradient term in Eq. (losm-1) is taken as   */
/*    (phi_{i+1} - phi_i), the one the continuous theta scheme gives;       */
/*  - Sigma_hat_i averages the two cells that share edge x_i (cells i and   */
/*    i+1), with the boundary edges using the single interior cell, the    */
/*    same pairing as Delta x_hat_i;                                       */
/*  - q_i is the source integrated over cell i (zero for a pulse start);    */
/*  - a reflecting side replaces its BC row by J = 0;                      */
/*  - inflow currents J_L, J_R are zero (vacuum).                          */
/* ------------------------------------------------------------------------ */
/* rows of the interleaved system: sub-diagonal a, diagonal b, super c, rhs r */
static void losm_assemble(int32_t I, const double* dx, const double* sigma_t, const double* sigma_a, double v,
                          double dt, double theta, int32_t bc_left, int32_t bc_right, const double* phi_old,
                          const double* J_old, const double* F_old, const double* F_new, double PL_new,
                          double PR_new, const double* q_old, const double* q_new, double* a, double* b,
                          double* c, double* r) {
    const int32_t n = 2 * I + 3;
    const double vdt = v * dt;
    const double tm1 = theta - 1.0;
    for (int32_t k = 0; k < n; ++k) a[k] = b[k] = c[k] = r[k] = 0.0;
    /* left boundary row */
    if (bc_left == OR_REFLECT) {
        b[0] = 0.0; c[0] = 1.0; r[0] = 0.0;           /* J_0 = 0 */
    } else {
        b[0] = 0.5; c[0] = 1.0; r[0] = PL_new;         /* J_0 + phi_0/2 = P_L */
    }
    for (int32_t i = 0; i <= I; ++i) {
        /* first-moment equation at edge x_i, row 2i+1 */
        double dxl = (i >= 1) ? dx[i - 1] : 0.0;       /* cell i   (Delta x_0 = 0)     */
        double dxr = (i <= I - 1) ? dx[i] : 0.0;       /* cell i+1 (Delta x_{I+1} = 0) */
        double stl = (i >= 1) ? sigma_t[i - 1] : 0.0;
        double str = (i <= I - 1) ? sigma_t[i] : 0.0;
        double dxh = 0.5 * (dxl + dxr);
        double sth = (stl * dxl + str * dxr) / (dxl + dxr);
        int32_t row = 2 * i + 1;
        a[row] = -theta / 3.0;                         /* phi_i     */
        b[row] = dxh / vdt + theta * sth * dxh;        /* J_i       */
        c[row] = theta / 3.0;                          /* phi_{i+1} */
        double old = (phi_old[i + 1] - phi_old[i]) / 3.0 + sth * dxh * J_old[i] - F_old[i + 1] + F_old[i];
        r[row] = dxh / vdt * J_old[i] + theta * (F_new[i + 1] - F_new[i]) + tm1 * old;
    }
    for (int32_t i = 1; i <= I; ++i) {
        /* balance on cell i, row 2i */
        int32_t row = 2 * i;
        double dxi = dx[i - 1];
        a[row] = -theta;                               /* J_{i-1} */
        b[row] = dxi / vdt + theta * sigma_a[i - 1] * dxi;
        c[row] = theta;                                /* J_i     */
        double qn = q_new ? q_new[i - 1] : 0.0;
        double qo = q_old ? q_old[i - 1] : 0.0;
        double old = J_old[i] - J_old[i - 1] + sigma_a[i - 1] * dxi * phi_old[i] - qo;
        r[row] = dxi / vdt * phi_old[i] + theta * qn + tm1 * old;
    }
    /* right boundary row */
    if (bc_right == OR_REFLECT) {
        a[n - 1] = 1.0; b[n - 1] = 0.0; r[n - 1] = 0.0; /* J_I = 0 */
    } else {
        a[n - 1] = 1.0; b[n - 1] = -0.5; r[n - 1] = -PR_new; /* J_I - phi_{I+1}/2 = -P_R */
    }
}

/* Gaussian elimination with partial pivoting on a tridiagonal matrix (two
 * rows compete per column, one extra super-diagonal of fill); solution in r */
static int tri_solve_pivot(int32_t n, double* a, double* b, double* c, double* r) {
    double* f = xcalloc(n, sizeof(double));
    if (!f) return E_OOM;
    for (int32_t k = 0; k < n - 1; ++k) {
        if (fabs(a[k + 1]) > fabs(b[k])) {
            /* swap rows k and k+1 (row k+1 has entries a,b,c in columns k..k+2) */
            double t;
            t = b[k]; b[k] = a[k + 1]; a[k + 1] = t;
            t = c[k]; c[k] = b[k + 1]; b[k + 1] = t;
            t = f[k]; f[k] = c[k + 1]; c[k + 1] = t;
            t = r[k]; r[k] = r[k + 1]; r[k + 1] = t;
        }
        if (b[k] == 0.0) {
            free(f);
            return E_NUMERIC;
        }
        double l = a[k + 1] / b[k];
        a[k + 1] = 0.0;
        b[k + 1] = b[k + 1] - l * c[k];
        c[k + 1] = c[k + 1] - l * f[k];
        r[k + 1] = r[k + 1] - l * r[k];
    }
    if (b[n - 1] == 0.0) {
        free(f);
        return E_NUMERIC;
    }
    r[n - 1] = r[n - 1] / b[n - 1];
    if (n >= 2) r[n - 2] = (r[n - 2] - c[n - 2] * r[n - 1]) / b[n - 2];
    for (int32_t k = n - 3; k >= 0; --k) r[k] = (r[k] - c[k] * r[k + 1] - f[k] * r[k + 2]) / b[k];
    free(f);
    return 0;
}

int or_losm_solve(int32_t I, const double* dx, const double* sigma_t, const double* sigma_a,
                  double v, double dt, double theta, int32_t bc_left, int32_t bc_right,
                  const double* phi_old, const double* J_old, const double* F_old,
                  const double* F_new, double PL_new, double PR_new,
                  const double* q_old, const double* q_new, double* phi_new, double* J_new) {
    if (I < 1 || !dx || !sigma_t || !sigma_a || !phi_old || !J_old || !F_old || !F_new ||
        !phi_new || !J_new)
        return E_ARG;
    int32_t n = 2 * I + 3;
    double* a = xcalloc(n, sizeof(double));
    double* b = xcalloc(n, sizeof(double));
    double* c = xcalloc(n, sizeof(double));
    double* r = xcalloc(n, sizeof(double));
    if (!a || !b || !c || !r) {
        free(a); free(b); free(c); free(r);
        return E_OOM;
    }
    losm_assemble(I, dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, phi_old, J_old, F_old, F_new,
                  PL_new, PR_new, q_old, q_new, a, b, c, r);
    int rc = tri_solve_pivot(n, a, b, c, r);
    if (rc == 0) {
        for (int32_t i = 0; i <= I + 1; ++i) phi_new[i] = r[2 * i];
        for (int32_t i = 0; i <= I; ++i) J_new[i] = r[2 * i + 1];
    }
    free(a); free(b); free(c); free(r);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Uniform comb (Sec. 5.1)                                                   */
/* Census particles in canonical order (source id, then lineage key) occupy */
/* consecutive intervals of their fixed-point weights on [0, W).  Tooth k   */
/* sits at T_k = (k + (2U+1)/2^33) W / N, k = 0..N-1, with U a 32-bit      */
/* uniform word; tooth k becomes particle k of the next step.  The first    */
/* tooth at or after a cumulative weight C is the least k with T_k >= C,    */
/* i.e. ceil((N C 2^33 - (2U+1) W) / (W 2^33)) clamped to [0, N], computed  */
/* exactly in 128-bit integers, so the copy counts sum to exactly N.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t id;
    uint64_t lin;
    int64_t idx;
} or_key;

static int key_cmp(const void* A, const void* B) {
    const or_key* a = (const or_key*)A;
    const or_key* b = (const or_key*)B;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    if (a->lin != b->lin) return a->lin < b->lin ? -1 : 1;
    return 0;
}

static int64_t first_tooth(uint64_t C, uint64_t W, int64_t N, uint32_t U) {
    typedef unsigned __int128 u128;
    const u128 num = ((u128)(uint64_t)N * C) << 33;
    const u128 sub = (u128)(2ull * U + 1ull) * W;
    if (num <= sub) return 0;
    const u128 den = (u128)W << 33;
    const u128 k = (num - sub + den - 1) / den;
    if (k > (u128)N) return N;
    return (int64_t)k;
}

int or_comb(int64_t m, const uint32_t* id, const uint64_t* lin, const uint64_t* wfx, int64_t n,
            uint32_t U, int32_t* src_of_slot) {
    if (m < 0 || n < 0 || !src_of_slot || (m > 0 && (!id || !lin || !wfx))) return E_ARG;
    or_key* k = (or_key*)xcalloc(m, sizeof(or_key));
    if (!k) return E_OOM;
    uint64_t W = 0;
    for (int64_t j = 0; j < m; ++j) {
        k[j].id = id[j];
        k[j].lin = lin[j];
        k[j].idx = j;
        W += wfx[j];
    }
    qsort(k, (size_t)m, sizeof(or_key), key_cmp);
    for (int64_t s = 0; s < n; ++s) src_of_slot[s] = -1;
    if (W == 0) {
        free(k);
        return 0;
    }
    uint64_t C = 0;
    for (int64_t j = 0; j < m; ++j) {
        int64_t k0 = first_tooth(C, W, n, U);
        C += wfx[k[j].idx];
        int64_t k1 = first_tooth(C, W, n, U);
        for (int64_t s = k0; s < k1; ++s) src_of_slot[s] = (int32_t)k[j].idx;
    }
    free(k);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One time step                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    or_particle* v;
    int64_t n, cap;
} pstack;

static int ps_push(pstack* s, const or_particle* q) {
    if (s->n == s->cap) {
        int64_t nc = s->cap ? 2 * s->cap : 1024;
        or_particle* nv = (or_particle*)realloc(s->v, sizeof(or_particle) * nc);
        if (!nv) return E_OOM;
        s->v = nv;
        s->cap = nc;
    }
    s->v[s->n++] = *q;
    return 0;
}

typedef struct {
    or_census* v;
    int64_t n, cap;
} cbank;

static int cb_push(cbank* s, const or_census* q) {
    if (s->n == s->cap) {
        int64_t nc = s->cap ? 2 * s->cap : 1024;
        or_census* nv = (or_census*)realloc(s->v, sizeof(or_census) * nc);
        if (!nv) return E_OOM;
        s->v = nv;
        s->cap = nc;
    }
    s->v[s->n++] = *q;
    return 0;
}

static void philox_event(const or_particle* q, uint32_t word, const uint32_t key[2], uint32_t r[4]) {
    uint32_t ctr[4] = {q->id, (uint32_t)q->lin, (uint32_t)(q->lin >> 32), word};
    or_philox4x32_10(ctr, key, r);
}

/* lineage key of daughter j of a split at event e: Philox of (lin, e, j)
 * under a fixed key */
static uint64_t lineage_hash(uint64_t lin, uint32_t e, uint32_t j) {
    uint32_t ctr[4] = {(uint32_t)lin, (uint32_t)(lin >> 32), e, j};
    uint32_t key[2] = {0x4C494E45u, 0x41474521u};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    return ((uint64_t)r[1] << 32) | r[0];
}

/* round-to-nearest-even of x * 2^s to a signed 64-bit integer */
static int64_t to_fixed(double x, int s) { return llrint(ldexp(x, s)); }

/* Closure and initial-condition vectors from the census (time-crossing)
 * tallies, Eq. (ct-mc).  Readings: phi_0, phi_{I+1}, F_0, F_{I+1} copy the
 * adjacent cell; interior edge currents interpolate the two adjacent cell
 * averages linearly in space; the boundary edge current follows the BC
 * relation (0 on a reflecting side); the MA filter, when on, acts on the
 * cell vectors of phi and F and on the edge vector of J. */
static void build_closure_set(const or_problem* p, const double* cphi, const double* cJ, const double* cF,
                              double PL, double PR, double* ophi, double* oJ, double* oF, double* oPL,
                              double* oPR) {
    int32_t I = p->I;
    double* tmp = xcalloc(I + 1, sizeof(double));
    double* tmp2 = xcalloc(I + 1, sizeof(double));
    for (int32_t i = 1; i <= I; ++i) {
        ophi[i] = cphi[i - 1];
        oF[i] = cF[i - 1];
    }
    for (int32_t i = 1; i <= I - 1; ++i) {
        double dl = p->dx[i - 1], dr = p->dx[i];
        oJ[i] = (cJ[i - 1] * dr + cJ[i] * dl) / (dl + dr);
    }
    ophi[0] = ophi[1];
    ophi[I + 1] = ophi[I];
    oF[0] = oF[1];
    oF[I + 1] = oF[I];
    oJ[0] = (p->d.bc_left == OR_REFLECT) ? 0.0 : (-0.5 * ophi[0] + PL);
    oJ[I] = (p->d.bc_right == OR_REFLECT) ? 0.0 : (0.5 * ophi[I + 1] - PR);
    if (oPL) *oPL = (p->d.bc_left == OR_REFLECT) ? 0.0 : PL;
    if (oPR) *oPR = (p->d.bc_right == OR_REFLECT) ? 0.0 : PR;
    if (p->d.filter == 1 || p->d.filter == 2) {
        int (*filt)(const double*, double*, int32_t, int32_t) = (p->d.filter == 1) ? or_ma_filter : or_fourier_filter;
        filt(ophi + 1, tmp, I, p->d.filter_k);
        memcpy(ophi + 1, tmp, sizeof(double) * I);
        filt(oF + 1, tmp, I, p->d.filter_k);
        memcpy(oF + 1, tmp, sizeof(double) * I);
        filt(oJ, tmp2, I + 1, p->d.filter_k);
        memcpy(oJ, tmp2, sizeof(double) * (I + 1));
        /* the ghost values copy the filtered end cells (the MA filter keeps
         * the end values, so for it nothing changes); the edge currents,
         * boundary edges included, are the filtered ones */
        ophi[0] = ophi[1];
        ophi[I + 1] = ophi[I];
        oF[0] = oF[1];
        oF[I + 1] = oF[I];
    }
    free(tmp);
    free(tmp2);
}

int or_build_closures(const or_problem* p, const double* cphi, const double* cJ, const double* cF,
                      double PL, double PR, double* phi, double* J, double* F, double* P) {
    if (!p || !cphi || !cJ || !cF || !phi || !J || !F || !P) return E_ARG;
    build_closure_set(p, cphi, cJ, cF, PL, PR, phi, J, F, &P[0], &P[1]);
    return 0;
}

static void build_closures(or_problem* p, const double* cphi, const double* cJ, const double* cF,
                           double PL, double PR) {
    build_closure_set(p, cphi, cJ, cF, PL, PR, p->clo_phi, p->clo_J, p->clo_F, &p->clo_PL, &p->clo_PR);
}

/* Exact moments of the unit isotropic plane pulse at t = 0 (step-1 IC).
 * Reading: the pulse goes to the cell containing src_x, split evenly when
 * src_x is an interior edge; on a domain end it belongs to the end cell.
 * phi = v * density; J = F = P = 0 for an isotropic pulse. */
static void source_moments(or_problem* p) {
    int32_t I = p->I;
    for (int32_t i = 0; i <= I + 1; ++i) p->clo_phi[i] = 0.0;
    for (int32_t i = 0; i <= I; ++i) p->clo_J[i] = 0.0;
    for (int32_t i = 0; i <= I + 1; ++i) p->clo_F[i] = 0.0;
    p->clo_PL = p->clo_PR = 0.0;
    double xs = p->d.src_x, v = p->d.v;
    int32_t edge = -1;
    for (int32_t i = 0; i <= I; ++i)
        if (p->edges[i] == xs) edge = i;
    if (edge == 0) {
        p->clo_phi[1] = v / p->dx[0];
    } else if (edge == I) {
        p->clo_phi[I] = v / p->dx[I - 1];
    } else if (edge > 0) {
        p->clo_phi[edge] = 0.5 * v / p->dx[edge - 1];
        p->clo_phi[edge + 1] = 0.5 * v / p->dx[edge];
    } else {
        for (int32_t i = 0; i < I; ++i)
            if (xs > p->edges[i] && xs < p->edges[i + 1]) p->clo_phi[i + 1] = v / p->dx[i];
    }
    p->clo_phi[0] = p->clo_phi[1];
    p->clo_phi[I + 1] = p->clo_phi[I];
}

/* Window centers are rounded to 20 significant bits (round half up on the
 * bit pattern) before use.  Reading: the center only places the window to
 * within a factor rho, so this changes nothing in the method, but it makes
 * the windows identical for two algebraically equivalent LOSM solvers whose
 * solutions differ in the last bits (a survivor of roulette takes the
 * center as its weight, so the last bits would otherwise reach the
 * tallies). */
static double quantize_center(double c) {
    uint64_t b;
    memcpy(&b, &c, sizeof b);
    b = (b + (1ull << 31)) & ~((1ull << 32) - 1ull);
    memcpy(&c, &b, sizeof c);
    return c;
}

/* WW centers, Eq. (ww-center), from a cell vector phi_tilde (length I):
 * phi_tilde clamped at 0 (a CN solution can undershoot ahead of a front),
 * normalised by its maximum, floored by eps, scaled by w_bar
 * (MEAN_WEIGHT) or 1 (LITERAL); ceiling rho*center, floor center/rho,
 * Eq. (ww-c&f). */
static void ww_from_flux(or_problem* p, const double* phit) {
    int32_t I = p->I;
    double mx = 0.0;
    for (int32_t i = 0; i < I; ++i) {
        double f = phit[i] > 0.0 ? phit[i] : 0.0;
        if (f > mx) mx = f;
    }
    double scale = (p->scaling == OR_SCALE_MEAN_WEIGHT) ? p->wbar : 1.0;
    for (int32_t i = 0; i < I; ++i) {
        double f = phit[i] > 0.0 ? phit[i] : 0.0;
        double ratio = (mx > 0.0) ? f / mx : 1.0;
        double b = ratio * (1.0 - p->eps) + p->eps;
        double ctr = quantize_center(scale * b);
        p->ww_c[i] = ctr;
        p->ww_hi[i] = ctr * p->rho;
        p->ww_lo[i] = ctr / p->rho;
    }
}

/* locate the birth cell of src_x for direction mu.  Reading: x_{k} <= x <
 * x_{k+1}, except on an interior edge with mu < 0, where the left cell is
 * taken; on a domain end the end cell. */
static int32_t birth_cell(const or_problem* p, double x, double mu) {
    int32_t I = p->I;
    if (x <= p->edges[0]) return 0;
    if (x >= p->edges[I]) return I - 1;
    for (int32_t i = 0; i < I; ++i) {
        if (x == p->edges[i] && i > 0) return mu < 0.0 ? i - 1 : i;
        if (x > p->edges[i] && x < p->edges[i + 1]) return i;
    }
    return I - 1;
}

/* windows of an in-step update: closures from the census and boundary
 * tallies of the histories so far (normalised by their number Hp), the fully
 * implicit HLOSM solution with them as the new level, centers from it */
static int update_windows(or_problem* p, int64_t Hp, const double* phi_old, const double* J_old,
                          const double* F_old, int S) {
    const int32_t I = p->I;
    const double v = p->d.v;
    double* cphi = xcalloc(I, sizeof(double));
    double* cJ = xcalloc(I, sizeof(double));
    double* cF = xcalloc(I, sizeof(double));
    double* tphi = xcalloc(I + 2, sizeof(double));
    double* tJ = xcalloc(I + 1, sizeof(double));
    double* tF = xcalloc(I + 2, sizeof(double));
    double* uphi = xcalloc(I + 2, sizeof(double));
    double* uJ = xcalloc(I + 1, sizeof(double));
    int rc = E_OOM;
    if (cphi && cJ && cF && tphi && tJ && tF && uphi && uJ) {
        for (int32_t i = 0; i < I; ++i) {
            const double den = (double)Hp * p->dx[i];
            cphi[i] = (v * ldexp(conv128(p->cen_w[i]), -S)) / den;
            cJ[i] = (v * ldexp(conv128(p->cen_wmu[i]), -S)) / den;
            cF[i] = (v * ldexp(conv128(p->cen_wf[i]), -S)) / den;
        }
        const double PL = ldexp(conv128(p->bnd[2]), -S) / ((double)Hp * p->d.dt);
        const double PR = ldexp(conv128(p->bnd[5]), -S) / ((double)Hp * p->d.dt);
        double tPL = 0.0, tPR = 0.0;
        build_closure_set(p, cphi, cJ, cF, PL, PR, tphi, tJ, tF, &tPL, &tPR);
        rc = or_losm_solve(I, p->dx, p->sigt, p->siga, v, p->d.dt, p->d.theta, p->d.bc_left, p->d.bc_right,
                           phi_old, J_old, F_old, tF, tPL, tPR, NULL, NULL, uphi, uJ);
        if (rc == 0) ww_from_flux(p, uphi + 1);
    }
    free(cphi); free(cJ); free(cF); free(tphi); free(tJ); free(tF); free(uphi); free(uJ);
    return rc;
}

int or_run_step(or_problem* p, or_stats* st) {
    if (!p) return E_ARG;
    if (!p->xs_set || !p->ww_set) return E_STATE;
    const int32_t I = p->I;
    const int32_t B = p->d.n_var_batches;
    const int64_t N = p->N;
    const int64_t n = p->n + 1;
    const double v = p->d.v;
    const double tau0 = v * p->d.dt;
    or_stats s;
    memset(&s, 0, sizeof s);

    /* 1. ICs and lagged closures: exact pulse moments for n = 1, else the
     *    closure vectors built at the end of step n-1. */
    if (n == 1) source_moments(p);
    double* phi_old = xcalloc(I + 2, sizeof(double));
    double* J_old = xcalloc(I + 1, sizeof(double));
    double* F_old = xcalloc(I + 2, sizeof(double));
    memcpy(phi_old, p->clo_phi, sizeof(double) * (I + 2));
    memcpy(J_old, p->clo_J, sizeof(double) * (I + 1));
    memcpy(F_old, p->clo_F, sizeof(double) * (I + 2));
    double PL_old = p->clo_PL, PR_old = p->clo_PR;
    memcpy(p->last_phi_old, phi_old, sizeof(double) * (I + 2));
    memcpy(p->last_J_old, J_old, sizeof(double) * (I + 1));
    memcpy(p->last_F_old, F_old, sizeof(double) * (I + 2));
    p->last_PL_old = PL_old;
    p->last_PR_old = PR_old;
    const int R = p->R, P2 = 2 * p->R;
    if (R > 0) {
        /* derivative closures of the step start: those built at the end of the
         * previous step (zero for the exact pulse moments of step 1) */
        if (n == 1) {
            memset(p->dclo_phi, 0, sizeof(double) * P2 * (I + 2));
            memset(p->dclo_J, 0, sizeof(double) * P2 * (I + 1));
            memset(p->dclo_F, 0, sizeof(double) * P2 * (I + 2));
        }
        memcpy(p->dold_phi, p->dclo_phi, sizeof(double) * P2 * (I + 2));
        memcpy(p->dold_J, p->dclo_J, sizeof(double) * P2 * (I + 1));
        memcpy(p->dold_F, p->dclo_F, sizeof(double) * P2 * (I + 2));
    }

    /* 2. semi-implicit HLOSM, Eqs. (losm-0), (losm-1-semi), (losm-disc-bc-semi):
     *    the new-level closure is the lagged one. */
    int rc = or_losm_solve(I, p->dx, p->sigt, p->siga, v, p->d.dt, p->d.theta, p->d.bc_left,
                           p->d.bc_right, phi_old, J_old, F_old, F_old, PL_old, PR_old, NULL, NULL,
                           p->semi_phi, p->semi_J);
    if (rc) goto fail;

    /* 3. weight windows */
    int ww_on = 0;
    const int override_step = p->has_override;
    if (p->has_override) {
        for (int32_t i = 0; i < I; ++i) {
            double ctr = quantize_center(p->ww_override[i]);
            p->ww_c[i] = ctr;
            p->ww_hi[i] = ctr * p->rho;
            p->ww_lo[i] = ctr / p->rho;
        }
        p->has_override = 0;
        ww_on = 1;
    } else if (p->mode == OR_MODE_HWW) {
        ww_from_flux(p, p->semi_phi + 1);
        ww_on = 1;
    } else if (p->mode == OR_MODE_LWW && p->has_prev_tl) {
        ww_from_flux(p, p->prev_tl_phi);
        ww_on = 1;
    }

    /* 4. tracking */
    const int E = wbar_exponent(p->wbar);
    const int S = 40 - E;                       /* tally fixed-point shift */
    p->tally_shift = S;
    const int Sc = 59 - E - bit_length(N);      /* comb weight shift */
    const uint32_t key[2] = {(uint32_t)p->d.seed, (uint32_t)(p->d.seed >> 32) ^ (uint32_t)n};
    for (int32_t i = 0; i < I; ++i) {
        p->tl_phi[i] = p->tl_j[i] = p->tl_f[i] = 0;
        p->cen_w[i] = p->cen_wmu[i] = p->cen_wf[i] = 0;
    }
    for (int64_t i = 0; i < (int64_t)I * B; ++i) p->batch[i] = 0;
    for (int j = 0; j < 6; ++j) p->bnd[j] = 0;
    if (R > 0) {
        for (int64_t i = 0; i < (int64_t)P2 * I; ++i) p->dtl[i] = 0;
        for (int64_t i = 0; i < (int64_t)3 * P2 * I; ++i) p->dcen[i] = 0;
        for (int64_t i = 0; i < (int64_t)6 * P2; ++i) p->dbnd[i] = 0;
    }

    pstack stack = {0};
    cbank census = {0};
    const int birth = (n == 1 && !p->bank_loaded);
    p->bank_loaded = 0;
    int64_t nstart = birth ? N : p->nbank;
    s.n_start = nstart;
    /* In-step window updates (Sec. 3, Eq. Hpn): the start bank is tracked in
     * u_ww + 1 chunks of source ids, [H_{p-1}, H_p) with H_p = floor(f_p H);
     * after each of the first u_ww chunks (all their descendants done) the
     * windows are re-derived from the fully implicit HLOSM solution whose
     * new-level closures come from the histories so far, normalised per
     * history (H_p).  Only HLOSM windows are updated (not an override, not
     * the lagged or analog modes). */
    const int nupd = (ww_on && p->mode == OR_MODE_HWW && !override_step) ? p->n_updates : 0;
    for (int chunk = 0; chunk <= nupd; ++chunk) {
        const int64_t lo = (chunk == 0) ? 0 : (int64_t)(p->ww_frac[chunk - 1] * (double)nstart);
        const int64_t hi = (chunk == nupd) ? nstart : (int64_t)(p->ww_frac[chunk] * (double)nstart);
        for (int64_t k = hi - 1; k >= lo; --k) {
            or_particle q;
            q.id = (uint32_t)k;
            q.lin = 0;
            for (int j = 0; j < MAX_DERIV; ++j) q.S[j] = 0.0;
            q.e = 0;
            q.tau = tau0;
            q.w = p->wbar;
            if (birth) {
                uint32_t ctr[4] = {(uint32_t)k, 0u, 0u, 0xFFFFFFFFu}, r[4];
                or_philox4x32_10(ctr, key, r);
                q.mu = 2.0 * or_u01(r[0], r[1]) - 1.0;
                q.x = p->d.src_x;
                if (q.x <= p->edges[0] && q.mu < 0.0 && p->d.bc_left == OR_REFLECT) q.mu = -q.mu;
                if (q.x >= p->edges[I] && q.mu > 0.0 && p->d.bc_right == OR_REFLECT) q.mu = -q.mu;
                q.cell = birth_cell(p, q.x, q.mu);
            } else {
                q.x = p->bx[k];
                q.mu = p->bmu[k];
                q.cell = p->bcell[k];
                if (R > 0 && p->bS)
                    for (int j = 0; j < P2; ++j) q.S[j] = p->bS[k * P2 + j];
            }
            if (ps_push(&stack, &q)) { rc = E_OOM; goto fail_track; }
        }

        while (stack.n > 0) {
            or_particle q = stack.v[--stack.n];
            for (;;) {
                if (q.e >= MAX_EVENTS_PER_TRACK) { s.error = E_NUMERIC; break; }
                uint32_t r[4];
                philox_event(&q, 2u * q.e, key, r);
                const double uf = or_u01(r[0], r[1]);
                const double uc = or_u01(r[2], r[3]);
                const int32_t k = q.cell;
                const double inv_mu = 1.0 / q.mu;
                const double dcoll = (-or_log(uf)) * p->inv_sigt[k];
                const double xe = (q.mu > 0.0) ? p->edges[k + 1] : p->edges[k];
                const double dedge = (xe - q.x) * inv_mu;
                const double dcens = q.tau;
                int ev; /* 0 census, 1 crossing, 2 collision */
                double l;
                if (dcens <= dedge && dcens <= dcoll) { ev = 0; l = dcens; }
                else if (dedge <= dcoll) { ev = 1; l = dedge; }
                else { ev = 2; l = dcoll; }
                /* track-length tallies, Eq. (phi-mc) */
                const double wl = q.w * l;
                const double wlmu = wl * q.mu;
                const double wlf = wl * (1.0 / 3.0 - q.mu * q.mu);
                p->tl_phi[k] += to_fixed(wl, S);
                p->tl_j[k] += to_fixed(wlmu, S);
                p->tl_f[k] += to_fixed(wlf, S);
                p->batch[(int64_t)(((uint64_t)q.id * (uint64_t)B) / (uint64_t)N) * I + k] += to_fixed(wl, S);
                if (R > 0) {
                    /* likelihood-ratio scores: the flight of length l in region r
                     * contributes -l to the Sigma_t score, a collision 1/Sigma_t;
                     * the derivative tally of this segment is w l S */
                    const int r = p->region[k];
                    q.S[r] = q.S[r] - l;
                    if (ev == 2) q.S[r] = q.S[r] + p->inv_sigt[k];
                    for (int j = 0; j < P2; ++j) p->dtl[(int64_t)j * I + k] += to_fixed(wl * q.S[j], S);
                }
                s.segments++;
                /* move */
                if (ev == 1) {
                    q.x = xe;
                } else {
                    double xn = q.x + q.mu * l;
                    if (xn < p->edges[k]) xn = p->edges[k];
                    if (xn > p->edges[k + 1]) xn = p->edges[k + 1];
                    q.x = xn;
                }
                q.tau = (ev == 0) ? 0.0 : q.tau - l;
                const uint32_t e_ev = q.e;
                q.e = q.e + 1;
                if (ev == 0) {
                    /* census: time-crossing tallies, Eq. (ct-mc) */
                    const double wmu = q.w * q.mu;
                    const double wf = q.w * (1.0 / 3.0 - q.mu * q.mu);
                    p->cen_w[k] += to_fixed(q.w, S);
                    p->cen_wmu[k] += to_fixed(wmu, S);
                    p->cen_wf[k] += to_fixed(wf, S);
                    for (int j = 0; j < P2; ++j) {
                        p->dcen[((int64_t)0 * P2 + j) * I + k] += to_fixed(q.w * q.S[j], S);
                        p->dcen[((int64_t)1 * P2 + j) * I + k] += to_fixed(wmu * q.S[j], S);
                        p->dcen[((int64_t)2 * P2 + j) * I + k] += to_fixed(wf * q.S[j], S);
                    }
                    or_census cq;
                    cq.x = q.x;
                    cq.mu = q.mu;
                    cq.w = q.w;
                    cq.cell = q.cell;
                    cq.id = q.id;
                    cq.lin = q.lin;
                    memcpy(cq.S, q.S, sizeof cq.S);
                    if (cb_push(&census, &cq)) { rc = E_OOM; goto fail_track; }
                    s.census++;
                    if (q.e > (uint32_t)s.max_events) s.max_events = q.e;
                    break;
                }
                int need_ww = 0;
                int have_r2 = 0;
                uint32_t r2[4];
                if (ev == 1) {
                    s.crossings++;
                    const int32_t nk = (q.mu > 0.0) ? k + 1 : k - 1;
                    if (nk < 0 || nk >= I) {
                        const int side = (nk < 0) ? 0 : 1;
                        const int32_t bc = side ? p->d.bc_right : p->d.bc_left;
                        const double amu = fabs(q.mu);
                        const double ia = (amu < GRAZE_MU) ? 2.0 / GRAZE_MU : 1.0 / amu;
                        if (bc == OR_VACUUM) {
                            /* surface estimators for the boundary closures:
                             * phi_b ~ w/|mu|, F_b ~ w(1/3-mu^2)/|mu|, P_b ~ w(1/2-|mu|)/|mu| */
                            const double wi = q.w * ia;
                            p->bnd[3 * side + 0] += to_fixed(wi, S);
                            p->bnd[3 * side + 1] += to_fixed(wi * (1.0 / 3.0 - q.mu * q.mu), S);
                            p->bnd[3 * side + 2] += to_fixed(wi * (0.5 - amu), S);
                            for (int j = 0; j < P2; ++j) {
                                p->dbnd[6 * j + 3 * side + 0] += to_fixed(wi * q.S[j], S);
                                p->dbnd[6 * j + 3 * side + 1] += to_fixed(wi * (1.0 / 3.0 - q.mu * q.mu) * q.S[j], S);
                                p->dbnd[6 * j + 3 * side + 2] += to_fixed(wi * (0.5 - amu) * q.S[j], S);
                            }
                            s.leaked++;
                            if (q.e > (uint32_t)s.max_events) s.max_events = q.e;
                            break;
                        }
                        q.mu = -q.mu; /* specular reflection, stays in cell k */
                        s.reflections++;
                    } else {
                        q.cell = nk;
                    }
                    need_ww = 1;
                } else {
                    s.collisions++;
                    /* the collision emits floor(c) + [u_c < c - floor(c)] particles
                     * (mean c); none: absorbed */
                    const double cfl = floor(p->c[k]);
                    const uint32_t nsec = (uint32_t)cfl + ((uc < p->c[k] - cfl) ? 1u : 0u);
                    if (nsec == 0) {
                        s.absorbed++;
                        if (q.e > (uint32_t)s.max_events) s.max_events = q.e;
                        break;
                    }
                    philox_event(&q, 2u * e_ev + 1u, key, r2);
                    have_r2 = 1;
                    q.mu = 2.0 * or_u01(r2[0], r2[1]) - 1.0;
                    s.scatters++;
                    if (R > 0) q.S[R + p->region[k]] = q.S[R + p->region[k]] + p->inv_c[k]; /* scatter, prob c */
                    /* the other emitted particles (a multiplying medium): each with
                     * its own lineage in the secondaries' namespace and its own
                     * isotropic direction; the track continues as the first */
                    if (nsec > 1) {
                        s.daughters += nsec - 1;
                        for (uint32_t j = nsec - 1; j >= 1; --j) {
                            or_particle dq = q;
                            dq.lin = lineage_hash(q.lin, e_ev | SECONDARY_EVENT, j);
                            dq.e = 0;
                            uint32_t ctr[4] = {dq.id, (uint32_t)dq.lin, (uint32_t)(dq.lin >> 32), 0xFFFFFFFEu}, rr[4];
                            or_philox4x32_10(ctr, key, rr);
                            dq.mu = 2.0 * or_u01(rr[0], rr[1]) - 1.0;
                            if (ps_push(&stack, &dq)) { rc = E_OOM; goto fail_track; }
                        }
                    }
                    need_ww = 1;
                }
                if (need_ww && ww_on) {
                    const int32_t kc = q.cell;
                    if (q.w > p->ww_hi[kc]) {
                        const double ratio = q.w / p->ww_c[kc];
                        const double ndd = ceil(ratio);
                        if (ndd > (double)MAX_DAUGHTERS) { s.error = E_NUMERIC; break; }
                        const uint32_t nd = (uint32_t)ndd;
                        const double wd = q.w / (double)nd;
                        s.split_events++;
                        s.daughters += nd - 1;
                        for (uint32_t j = nd - 1; j >= 1; --j) {
                            or_particle dq = q;
                            dq.w = wd;
                            dq.lin = lineage_hash(q.lin, e_ev, j);
                            dq.e = 0;
                            if (ps_push(&stack, &dq)) { rc = E_OOM; goto fail_track; }
                        }
                        q.w = wd;
                        q.lin = lineage_hash(q.lin, e_ev, 0);
                        q.e = 0;
                    } else if (q.w < p->ww_lo[kc]) {
                        if (!have_r2) philox_event(&q, 2u * e_ev + 1u, key, r2);
                        const double ur = or_u01(r2[2], r2[3]);
                        const double ps = q.w / p->ww_c[kc];
                        if (ur < ps) {
                            q.w = p->ww_c[kc];
                            s.roulette_survivals++;
                        } else {
                            s.roulette_kills++;
                            if (q.e > (uint32_t)s.max_events) s.max_events = q.e;
                            break;
                        }
                    }
                }
            }
        }
        if (chunk < nupd && hi > 0) {
            rc = update_windows(p, hi, phi_old, J_old, F_old, S);
            if (rc) goto fail_track;
        }
    }
    free(stack.v);
    stack.v = NULL;

    /* 5. normalised census tallies -> closures at t^n -> fully implicit HLOSM */
    {
        double* cphi = xcalloc(I, sizeof(double));
        double* cJ = xcalloc(I, sizeof(double));
        double* cF = xcalloc(I, sizeof(double));
        for (int32_t i = 0; i < I; ++i) {
            const double den = (double)N * p->dx[i];
            cphi[i] = (v * ldexp(conv128(p->cen_w[i]), -S)) / den;
            cJ[i] = (v * ldexp(conv128(p->cen_wmu[i]), -S)) / den;
            cF[i] = (v * ldexp(conv128(p->cen_wf[i]), -S)) / den;
        }
        const double PL = ldexp(conv128(p->bnd[2]), -S) / ((double)N * p->d.dt);
        const double PR = ldexp(conv128(p->bnd[5]), -S) / ((double)N * p->d.dt);
        build_closures(p, cphi, cJ, cF, PL, PR);
        for (int j = 0; j < P2; ++j) {
            /* derivative closures: the same linear map applied to the census
             * and boundary derivative tallies */
            for (int32_t i = 0; i < I; ++i) {
                const double den = (double)N * p->dx[i];
                cphi[i] = (v * ldexp(conv128(p->dcen[((int64_t)0 * P2 + j) * I + i]), -S)) / den;
                cJ[i] = (v * ldexp(conv128(p->dcen[((int64_t)1 * P2 + j) * I + i]), -S)) / den;
                cF[i] = (v * ldexp(conv128(p->dcen[((int64_t)2 * P2 + j) * I + i]), -S)) / den;
            }
            const double dPL = ldexp(conv128(p->dbnd[6 * j + 2]), -S) / ((double)N * p->d.dt);
            const double dPR = ldexp(conv128(p->dbnd[6 * j + 5]), -S) / ((double)N * p->d.dt);
            build_closure_set(p, cphi, cJ, cF, dPL, dPR, p->dclo_phi + (int64_t)j * (I + 2),
                              p->dclo_J + (int64_t)j * (I + 1), p->dclo_F + (int64_t)j * (I + 2), &p->dclo_PL[j],
                              &p->dclo_PR[j]);
        }
        free(cphi); free(cJ); free(cF);
        rc = or_losm_solve(I, p->dx, p->sigt, p->siga, v, p->d.dt, p->d.theta, p->d.bc_left,
                           p->d.bc_right, phi_old, J_old, F_old, p->clo_F, p->clo_PL, p->clo_PR,
                           NULL, NULL, p->full_phi, p->full_J);
        if (rc) goto fail_track;
        for (int32_t i = 0; i < I; ++i)
            p->prev_tl_phi[i] = ldexp(conv128(p->tl_phi[i]), -S) / (((double)N * p->dx[i]) * p->d.dt);
        p->has_prev_tl = 1;
    }

    /* 6. uniform comb to N */
    {
        const int64_t m = census.n;
        uint32_t* ids = xcalloc(m, sizeof(uint32_t));
        uint64_t* lins = xcalloc(m, sizeof(uint64_t));
        uint64_t* wfx = xcalloc(m, sizeof(uint64_t));
        int32_t* src = xcalloc(N, sizeof(int32_t));
        uint64_t W = 0;
        for (int64_t j = 0; j < m; ++j) {
            ids[j] = census.v[j].id;
            lins[j] = census.v[j].lin;
            wfx[j] = (uint64_t)to_fixed(census.v[j].w, Sc);
            W += wfx[j];
        }
        /* lineage collisions: equal (id, lineage) pairs */
        {
            or_key* kk = xcalloc(m, sizeof(or_key));
            for (int64_t j = 0; j < m; ++j) { kk[j].id = ids[j]; kk[j].lin = lins[j]; kk[j].idx = j; }
            qsort(kk, (size_t)m, sizeof(or_key), key_cmp);
            for (int64_t j = 1; j < m; ++j)
                if (kk[j].id == kk[j - 1].id && kk[j].lin == kk[j - 1].lin) s.lineage_collisions++;
            free(kk);
        }
        uint32_t cctr[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xC0B0u}, r[4];
        or_philox4x32_10(cctr, key, r);
        or_comb(m, ids, lins, wfx, N, r[1], src);
        free(p->bx); free(p->bmu); free(p->bcell);
        p->bx = xcalloc(N, sizeof(double));
        p->bmu = xcalloc(N, sizeof(double));
        p->bcell = xcalloc(N, sizeof(int32_t));
        if (R > 0) {
            free(p->bS);
            p->bS = xcalloc((size_t)N * P2, sizeof(double));
        }
        if (W == 0) {
            p->nbank = 0;
            p->wbar = 0.0;
        } else {
            for (int64_t k = 0; k < N; ++k) {
                const or_census* cq = &census.v[src[k]];
                p->bx[k] = cq->x;
                p->bmu[k] = cq->mu;
                p->bcell[k] = cq->cell;
                for (int j = 0; j < P2; ++j) p->bS[k * P2 + j] = cq->S[j];
            }
            p->nbank = N;
            p->wbar = ldexp((double)W, -Sc) / (double)N;
        }
        s.n_next = p->nbank;
        s.w_bar_next = p->wbar;
        free(ids); free(lins); free(wfx); free(src);
    }
    free(p->census);
    p->census = census.v;
    p->ncensus = census.n;
    free(phi_old); free(J_old); free(F_old);
    p->n = n;
    if (st) *st = s;
    return s.error;

fail_track:
    free(stack.v);
    free(census.v);
fail:
    free(phi_old); free(J_old); free(F_old);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Read-out                                                                 */
/* ------------------------------------------------------------------------ */

int or_get_tallies(const or_problem* p, int32_t kind, double* out, int64_t n) {
    if (!p || !out) return E_ARG;
    const int32_t I = p->I, B = p->d.n_var_batches;
    const int64_t N = p->N;
    const int S = p->tally_shift;
    const double v = p->d.v, dt = p->d.dt;
    switch (kind) {
    case K_TL_PHI: case K_TL_J: case K_TL_F: {
        if (n < I) return E_ARG;
        const i128* a = kind == K_TL_PHI ? p->tl_phi : kind == K_TL_J ? p->tl_j : p->tl_f;
        for (int32_t i = 0; i < I; ++i) out[i] = ldexp(conv128(a[i]), -S) / (((double)N * p->dx[i]) * dt);
        return 0;
    }
    case K_CEN_PHI: case K_CEN_J: case K_CEN_F: {
        if (n < I) return E_ARG;
        const i128* a = kind == K_CEN_PHI ? p->cen_w : kind == K_CEN_J ? p->cen_wmu : p->cen_wf;
        for (int32_t i = 0; i < I; ++i) out[i] = (v * ldexp(conv128(a[i]), -S)) / ((double)N * p->dx[i]);
        return 0;
    }
    case K_BATCH_PHI: {
        if (n < (int64_t)I * B) return E_ARG;
        for (int32_t b = 0; b < B; ++b) {
            /* ids with floor(id B / N) == b: ceil(b N / B) .. ceil((b+1) N / B) - 1 */
            const int64_t nb = ((b + 1) * N + B - 1) / B - (b * N + B - 1) / B;
            for (int32_t i = 0; i < I; ++i)
                out[(int64_t)b * I + i] =
                    nb ? ldexp(conv128(p->batch[(int64_t)b * I + i]), -S) / (((double)nb * p->dx[i]) * dt)
                       : 0.0;
        }
        return 0;
    }
    case K_BOUNDARY: {
        if (n < 6) return E_ARG;
        for (int j = 0; j < 6; ++j) out[j] = ldexp(conv128(p->bnd[j]), -S) / ((double)N * dt);
        return 0;
    }
    case K_WW_CENTER:
        if (n < I) return E_ARG;
        memcpy(out, p->ww_c, sizeof(double) * I);
        return 0;
    case K_CLOSURE_PHI:
        if (n < I + 2) return E_ARG;
        memcpy(out, p->clo_phi, sizeof(double) * (I + 2));
        return 0;
    case K_CLOSURE_J:
        if (n < I + 1) return E_ARG;
        memcpy(out, p->clo_J, sizeof(double) * (I + 1));
        return 0;
    case K_CLOSURE_F:
        if (n < I + 2) return E_ARG;
        memcpy(out, p->clo_F, sizeof(double) * (I + 2));
        return 0;
    default:
        return E_ARG;
    }
}

int or_get_tallies_raw(const or_problem* p, int32_t kind, int64_t* out, int64_t n) {
    if (!p || !out) return E_ARG;
    const int32_t I = p->I, B = p->d.n_var_batches;
    const i128* a = NULL;
    int64_t len = I;
    switch (kind) {
    case K_TL_PHI: a = p->tl_phi; break;
    case K_TL_J: a = p->tl_j; break;
    case K_TL_F: a = p->tl_f; break;
    case K_CEN_PHI: a = p->cen_w; break;
    case K_CEN_J: a = p->cen_wmu; break;
    case K_CEN_F: a = p->cen_wf; break;
    case K_BATCH_PHI: a = p->batch; len = (int64_t)I * B; break;
    case K_BOUNDARY: a = p->bnd; len = 6; break;
    default: return E_ARG;
    }
    if (n < 2 * len) return E_ARG;
    for (int64_t i = 0; i < len; ++i) {
        out[2 * i] = (int64_t)(uint64_t)a[i];
        out[2 * i + 1] = (int64_t)(a[i] >> 64);
    }
    return 0;
}

int or_get_losm_solution(const or_problem* p, int32_t which, double* phi, double* J) {
    if (!p || !phi || !J || which < 0 || which > 1) return E_ARG;
    memcpy(phi, which == 0 ? p->semi_phi : p->full_phi, sizeof(double) * (p->I + 2));
    memcpy(J, which == 0 ? p->semi_J : p->full_J, sizeof(double) * (p->I + 1));
    return 0;
}

int or_get_ww(const or_problem* p, double* center, double* ceil_, double* floor_) {
    if (!p) return E_ARG;
    if (center) memcpy(center, p->ww_c, sizeof(double) * p->I);
    if (ceil_) memcpy(ceil_, p->ww_hi, sizeof(double) * p->I);
    if (floor_) memcpy(floor_, p->ww_lo, sizeof(double) * p->I);
    return 0;
}

int or_set_bank(or_problem* p, const double* x, const double* mu, const int32_t* cell, int64_t n, double wbar) {
    if (!p || n < 0 || n > p->N || (n > 0 && (!x || !mu || !cell)) || !(wbar > 0.0)) return E_ARG;
    for (int64_t k = 0; k < n; ++k)
        if (cell[k] < 0 || cell[k] >= p->I || !(mu[k] != 0.0) || !(mu[k] >= -1.0 && mu[k] <= 1.0)) return E_ARG;
    free(p->bx); free(p->bmu); free(p->bcell);
    p->bx = xcalloc(n, sizeof(double));
    p->bmu = xcalloc(n, sizeof(double));
    p->bcell = xcalloc(n, sizeof(int32_t));
    if (!p->bx || !p->bmu || !p->bcell) return E_OOM;
    memcpy(p->bx, x, sizeof(double) * n);
    memcpy(p->bmu, mu, sizeof(double) * n);
    memcpy(p->bcell, cell, sizeof(int32_t) * n);
    p->nbank = n;
    p->wbar = wbar;
    p->bank_loaded = 1;
    if (p->R > 0) {
        free(p->bS);
        p->bS = xcalloc((size_t)(n ? n : 1) * 2 * p->R, sizeof(double));
    }
    return 0;
}

int or_get_census(const or_problem* p, double* x, double* mu, double* w, int32_t* cell, uint32_t* id,
                  uint64_t* lin, int64_t cap, int64_t* n) {
    if (!p || !n) return E_ARG;
    *n = p->ncensus;
    if (cap == 0) return 0;
    if (cap < p->ncensus) return E_ARG;
    for (int64_t j = 0; j < p->ncensus; ++j) {
        const or_census* c = &p->census[j];
        if (x) x[j] = c->x;
        if (mu) mu[j] = c->mu;
        if (w) w[j] = c->w;
        if (cell) cell[j] = c->cell;
        if (id) id[j] = c->id;
        if (lin) lin[j] = c->lin;
    }
    return 0;
}

int or_get_bank(const or_problem* p, double* x, double* mu, int32_t* cell, int64_t cap, int64_t* n) {
    if (!p || !n) return E_ARG;
    *n = p->nbank;
    if (cap < p->nbank) return p->nbank ? E_ARG : 0;
    for (int64_t k = 0; k < p->nbank; ++k) {
        if (x) x[k] = p->bx[k];
        if (mu) mu[k] = p->bmu[k];
        if (cell) cell[k] = p->bcell[k];
    }
    return 0;
}

int or_set_bank_scores(or_problem* p, const double* S) {
    if (!p || p->R < 1) return E_ARG;
    const int P2 = 2 * p->R;
    free(p->bS);
    p->bS = xcalloc((size_t)(p->nbank ? p->nbank : 1) * P2, sizeof(double));
    if (!p->bS) return E_OOM;
    if (S) memcpy(p->bS, S, sizeof(double) * p->nbank * P2);
    return 0;
}

int or_get_deriv_tallies(const or_problem* p, int32_t which, double* out, int64_t n) {
    if (!p || !out || p->R < 1 || which < 0 || which > 4) return E_ARG;
    const int32_t I = p->I;
    const int P2 = 2 * p->R;
    const int S = p->tally_shift;
    const int64_t N = p->N;
    if (which == 4) {
        if (n < (int64_t)P2 * 6) return E_ARG;
        for (int64_t k = 0; k < (int64_t)P2 * 6; ++k) out[k] = ldexp(conv128(p->dbnd[k]), -S) / ((double)N * p->d.dt);
        return 0;
    }
    if (n < (int64_t)P2 * I) return E_ARG;
    for (int j = 0; j < P2; ++j)
        for (int32_t i = 0; i < I; ++i) {
            double val;
            if (which == 0) {
                val = ldexp(conv128(p->dtl[(int64_t)j * I + i]), -S) / (((double)N * p->dx[i]) * p->d.dt);
            } else {
                const i128 a = p->dcen[((int64_t)(which - 1) * P2 + j) * I + i];
                val = (p->d.v * ldexp(conv128(a), -S)) / ((double)N * p->dx[i]);
            }
            out[(int64_t)j * I + i] = val;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the LOSM solve (differentiation of the HLOSM step)            */
/*                                                                          */
/* The solve is A(Sigma) u = b(Sigma, data), with data = (phi_old, J_old,   */
/* F_old, F_new, P_L, P_R) entering b linearly.  For a scalar g . u the    */
/* change along a direction (dSigma_t, dSigma_a, d data) is                */
/*   g . du = lambda . ( b(Sigma, d data) + db/dSigma - dA/dSigma u ),     */
/* with A^T lambda = g.  Sigma_t enters only the first-moment rows, through */
/* Sigma_hat at the edges, and Sigma_a only the balance rows.               */
/* ------------------------------------------------------------------------ */
int or_losm_adjoint(int32_t I, const double* dx, const double* sigma_t, const double* sigma_a, double v,
                    double dt, double theta, int32_t bc_left, int32_t bc_right, const double* g_phi,
                    const double* g_J, double* lam) {
    if (I < 1 || !dx || !sigma_t || !sigma_a || !g_phi || !g_J || !lam) return E_ARG;
    const int32_t n = 2 * I + 3;
    double* a = xcalloc(n, sizeof(double));
    double* b = xcalloc(n, sizeof(double));
    double* c = xcalloc(n, sizeof(double));
    double* r = xcalloc(n, sizeof(double));
    double* z = xcalloc(I + 2, sizeof(double));
    double* at = xcalloc(n, sizeof(double));
    double* ct = xcalloc(n, sizeof(double));
    int rc = E_OOM;
    if (a && b && c && r && z && at && ct) {
        /* the matrix does not depend on the data: assemble with zero data */
        losm_assemble(I, dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, z, z, z, z, 0.0, 0.0, NULL,
                      NULL, a, b, c, r);
        /* transpose: (A^T)[k][k-1] = A[k-1][k] = c[k-1], (A^T)[k][k+1] = A[k+1][k] = a[k+1] */
        for (int32_t k = 0; k < n; ++k) {
            at[k] = (k >= 1) ? c[k - 1] : 0.0;
            ct[k] = (k + 1 < n) ? a[k + 1] : 0.0;
        }
        for (int32_t i = 0; i <= I + 1; ++i) lam[2 * i] = g_phi[i];
        for (int32_t i = 0; i <= I; ++i) lam[2 * i + 1] = g_J[i];
        rc = tri_solve_pivot(n, at, b, ct, lam);
    }
    free(a); free(b); free(c); free(r); free(z); free(at); free(ct);
    return rc;
}

int or_losm_directional(int32_t I, const double* dx, const double* sigma_t, const double* sigma_a, double v,
                        double dt, double theta, int32_t bc_left, int32_t bc_right, const double* lam,
                        const double* phi_old, const double* J_old, const double* phi_new, const double* J_new,
                        const double* dsigma_t, const double* dsigma_a, const double* dphi_old,
                        const double* dJ_old, const double* dF_old, const double* dF_new, double dPL,
                        double dPR, double* out) {
    if (I < 1 || !dx || !sigma_t || !sigma_a || !lam || !phi_old || !J_old || !phi_new || !J_new ||
        !dsigma_t || !dsigma_a || !dphi_old || !dJ_old || !dF_old || !dF_new || !out)
        return E_ARG;
    const int32_t n = 2 * I + 3;
    double* a = xcalloc(n, sizeof(double));
    double* b = xcalloc(n, sizeof(double));
    double* c = xcalloc(n, sizeof(double));
    double* r = xcalloc(n, sizeof(double));
    if (!a || !b || !c || !r) {
        free(a); free(b); free(c); free(r);
        return E_OOM;
    }
    /* data part: the right-hand side assembled from the data's change */
    losm_assemble(I, dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, dphi_old, dJ_old, dF_old, dF_new,
                  dPL, dPR, NULL, NULL, a, b, c, r);
    double acc = 0.0;
    for (int32_t k = 0; k < n; ++k) acc += lam[k] * r[k];
    /* cross-section part, first-moment rows: (theta-1) dSigma_hat dxh J_old
     * on the right, theta dSigma_hat dxh J_new moved from the left */
    const double tm1 = theta - 1.0;
    for (int32_t i = 0; i <= I; ++i) {
        const double dxl = (i >= 1) ? dx[i - 1] : 0.0;
        const double dxr = (i <= I - 1) ? dx[i] : 0.0;
        const double dsl = (i >= 1) ? dsigma_t[i - 1] : 0.0;
        const double dsr = (i <= I - 1) ? dsigma_t[i] : 0.0;
        const double dsh = (dsl * dxl + dsr * dxr) / (dxl + dxr);
        const double dxh = 0.5 * (dxl + dxr);
        acc += lam[2 * i + 1] * (tm1 * dsh * dxh * J_old[i] - theta * dsh * dxh * J_new[i]);
    }
    /* balance rows: (theta-1) dSigma_a dx phi_old and theta dSigma_a dx phi_new */
    for (int32_t i = 1; i <= I; ++i) {
        const double dsa = dsigma_a[i - 1];
        const double dxi = dx[i - 1];
        acc += lam[2 * i] * (tm1 * dsa * dxi * phi_old[i] - theta * dsa * dxi * phi_new[i]);
    }
    *out = acc;
    free(a); free(b); free(c); free(r);
    return 0;
}

/* g . d(full HLOSM solution of the last step)/d(theta_j): the direction of
 * theta_j is dSigma_t = 1 on region j (j < R) or 0, dSigma_a = (1 - c) on
 * region j (Sigma_a = Sigma_t (1 - c)) or -Sigma_t on region j - R (j >= R),
 * and the data's change is the derivative closures of the step. */
int or_losm_vjp(const or_problem* p, const double* g_phi, const double* g_J, double* grad) {
    if (!p || !g_phi || !g_J || !grad || p->R < 1 || p->n < 1) return E_ARG;
    const int32_t I = p->I, n = 2 * I + 3;
    const int R = p->R, P2 = 2 * R;
    double* lam = xcalloc(n, sizeof(double));
    double* dst = xcalloc(I, sizeof(double));
    double* dsa = xcalloc(I, sizeof(double));
    int rc = E_OOM;
    if (lam && dst && dsa)
        rc = or_losm_adjoint(I, p->dx, p->sigt, p->siga, p->d.v, p->d.dt, p->d.theta, p->d.bc_left,
                             p->d.bc_right, g_phi, g_J, lam);
    for (int j = 0; j < P2 && rc == 0; ++j) {
        const int is_sigma = j < R;
        const int g = is_sigma ? j : j - R;
        for (int32_t i = 0; i < I; ++i) {
            const int in = p->region[i] == g;
            dst[i] = (is_sigma && in) ? 1.0 : 0.0;
            dsa[i] = in ? (is_sigma ? 1.0 - p->c[i] : -p->sigt[i]) : 0.0;
        }
        rc = or_losm_directional(I, p->dx, p->sigt, p->siga, p->d.v, p->d.dt, p->d.theta, p->d.bc_left,
                                 p->d.bc_right, lam, p->last_phi_old, p->last_J_old, p->full_phi, p->full_J,
                                 dst, dsa, p->dold_phi + (int64_t)j * (I + 2), p->dold_J + (int64_t)j * (I + 1),
                                 p->dold_F + (int64_t)j * (I + 2), p->dclo_F + (int64_t)j * (I + 2),
                                 p->dclo_PL[j], p->dclo_PR[j], &grad[j]);
    }
    free(lam); free(dst); free(dsa);
    return rc;
}

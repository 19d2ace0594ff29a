/*
 * hww_oracle.h -- plain FP64 CPU oracle of the hybrid weight-window (HWW)
 * time-dependent Monte Carlo step (Shaw & Anistratov, arXiv 2512.19925).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA path; the only thing both sides agree on is the written numerics
 * contract (Philox4x32-10 keyed as documented, the 52-bit uniform map, the
 * table-driven logarithm, the fixed-point tally format and the event rules),
 * which each side implements on its own.
 *
 * Every function returns 0 on success and a negative code on error.
 */
#ifndef HWW_ORACLE_H
#define HWW_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_problem or_problem;

typedef struct {
    int32_t n_cells;
    const double* edges;          /* n_cells+1, strictly increasing */
    double v, dt;
    int32_t bc_left, bc_right;    /* 0 vacuum, 1 reflecting */
    double src_x;                 /* unit isotropic plane pulse at t = 0 */
    int64_t particles_per_step;  /* 1 <= N < 2^30 */
    uint64_t seed;
    double theta;                 /* 0.5 Crank-Nicolson, 1.0 backward Euler */
    int32_t filter, filter_k;     /* 0 none, 1 moving average of base k, 2 Fourier low-pass
                                     with cutoff k */
    int32_t n_var_batches;        /* B for the batch-mean variance tally */
    int32_t deriv_regions;        /* R > 0: likelihood-ratio derivative tallies for
                                     (Sigma_t, c) of R regions (R <= 4) */
} or_desc;

typedef struct {
    int64_t n_start, segments, collisions, crossings, reflections;
    int64_t leaked, absorbed, scatters, split_events, daughters;
    int64_t roulette_kills, roulette_survivals, census, lineage_collisions;
    int64_t max_events, n_next;
    double w_bar_next;
    int32_t error;
} or_stats;

/* problem life cycle (mirrors the C ABI verbs of the library) */
int or_create(const or_desc* d, or_problem** out);
int or_set_cross_sections(or_problem* p, const double* sigma_t, const double* c);
int or_set_ww_params(or_problem* p, double rho, double eps_min, int32_t mode, int32_t center_scaling);
int or_set_regions(or_problem* p, const int32_t* region); /* region of each cell, 0..R-1 */
/* in-step window updates: n <= 16 updates after the fractions f_1 < ... < f_n
 * in (0,1) of the step's histories (NULL: f_p = p/(n+1)); n = 0 turns them off */
int or_set_ww_updates(or_problem* p, int32_t n, const double* fractions);
int or_set_ww_centers(or_problem* p, const double* centers); /* override for the next step only */
int or_run_step(or_problem* p, or_stats* st);
int or_get_tallies(const or_problem* p, int32_t kind, double* out, int64_t n);
int or_get_tallies_raw(const or_problem* p, int32_t kind, int64_t* out, int64_t n);
int or_get_losm_solution(const or_problem* p, int32_t which, double* phi, double* J);
/* derivative tallies of the last step, [2R][I]: parameter j < R is Sigma_t of
 * region j, j >= R is c of region j - R; which: 0 track-length phi, 1 census
 * phi, 2 census J, 3 census F, 4 boundary ([2R][6]) (normalised like the
 * tallies) */
int or_get_deriv_tallies(const or_problem* p, int32_t which, double* out, int64_t n);
/* vector-Jacobian product of the last step's fully implicit HLOSM solution:
 * grad[j] = g_phi . dphi/dtheta_j + g_J . dJ/dtheta_j (2R values) */
int or_losm_vjp(const or_problem* p, const double* g_phi, const double* g_J, double* grad);
/* adjoint of a LOSM solve: lambda (2I+3, interleaved phi_0, J_0, phi_1, ...)
 * with A^T lambda = (g_phi, g_J) interleaved */
int or_losm_adjoint(int32_t I, const double* dx, const double* sigma_t, const double* sigma_a, double v,
                    double dt, double theta, int32_t bc_left, int32_t bc_right, const double* g_phi,
                    const double* g_J, double* lam);
/* g . du of a LOSM solve along a change of the cross sections and of the
 * data, given lambda, the data's old vectors and the solution u */
int or_losm_directional(int32_t I, const double* dx, const double* sigma_t, const double* sigma_a, double v,
                        double dt, double theta, int32_t bc_left, int32_t bc_right, const double* lam,
                        const double* phi_old, const double* J_old, const double* phi_new, const double* J_new,
                        const double* dsigma_t, const double* dsigma_a, const double* dphi_old,
                        const double* dJ_old, const double* dF_old, const double* dF_new, double dPL,
                        double dPR, double* out);
int or_get_ww(const or_problem* p, double* center, double* ceil_, double* floor_);
int or_get_bank(const or_problem* p, double* x, double* mu, int32_t* cell, int64_t cap, int64_t* n);
/* replace the start bank of the next step: n particles with ids 0..n-1,
 * weight w_bar each (also before the first step, instead of the pulse) */
int or_set_bank(or_problem* p, const double* x, const double* mu, const int32_t* cell, int64_t n, double wbar);
/* with derivatives: the scores of the loaded bank (n x 2R, may be NULL = 0) */
int or_set_bank_scores(or_problem* p, const double* S);
int or_get_census(const or_problem* p, double* x, double* mu, double* w, int32_t* cell, uint32_t* id,
                  uint64_t* lin, int64_t cap, int64_t* n);
void or_destroy(or_problem* p);

/* building blocks, exported so that each can be pinned on its own */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01(uint32_t lo, uint32_t hi);
double or_log(double u);
/* entry j of the logarithm's reduction table: 1/c_j rounded (halved for
 * j >= 64) and T_j = -log(IC_j 2^K_j) rounded */
void or_log_table(int32_t j, double* ic, double* t);
int or_fourier_filter(const double* in, double* out, int32_t m, int32_t kappa);
int or_ma_filter(const double* in, double* out, int32_t m, int32_t k);
int or_losm_solve(int32_t n_cells, const double* dx, const double* sigma_t, const double* sigma_a,
                  double v, double dt, double theta, int32_t bc_left, int32_t bc_right,
                  const double* phi_old, const double* J_old, const double* F_old,
                  const double* F_new, double PL_new, double PR_new,
                  const double* q_old, const double* q_new,
                  double* phi_new, double* J_new);
int or_comb(int64_t m, const uint32_t* id, const uint64_t* lin, const uint64_t* wfx,
            int64_t n, uint32_t U, int32_t* src_of_slot);
/* the closure and initial-condition vectors at a time layer (Eq. ct-mc, Eq.
 * losm-disc-bc) that a step forms from its normalised census moments
 * cphi, cJ, cF (I cell averages each) and its boundary closures PL, PR, on
 * p's mesh, boundary conditions and filter: phi (I+2), J (I+1), F (I+2) and
 * the boundary closures (PL, PR) the HLOSM solve takes */
int or_build_closures(const or_problem* p, const double* cphi, const double* cJ, const double* cF,
                      double PL, double PR, double* phi, double* J, double* F, double* P);

#ifdef __cplusplus
}
#endif
#endif

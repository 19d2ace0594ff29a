/*
 * hww.h -- C ABI of the GB300 (sm_103a) library for one time step of the
 * hybrid weight-window (HWW) time-dependent Monte Carlo method of
 * Shaw & Anistratov, "Hybrid weight windows for time-dependent Monte Carlo
 * transport" (arXiv 2512.19925).
 *
 * The method (paper Secs. 2-4): one-speed particles with isotropic
 * scattering move through a 1D slab (Eq. HO_transport).  Each time step
 *   1. solves the semi-implicit hybrid low-order second-moment (HLOSM)
 *      equations (Eqs. losm-0, losm-1-semi, losm-disc-bc-semi) with the
 *      closures of the previous step to obtain weight-window (WW) centers
 *      (Eq. ww-center) with ceiling and floor (Eq. ww-c&f);
 *   2. tracks the particle bank (collision, cell-crossing and census
 *      events), splitting and rouletting against the windows (Sec. 2),
 *      accumulating track-length tallies (Eq. phi-mc) and census
 *      (time-crossing) tallies (Eq. ct-mc);
 *   3. builds the closures F, P_L, P_R and the initial conditions of the
 *      next step from the census tallies, optionally filtered by a moving
 *      average (Sec. 4, Eq. moving_average), and solves the fully implicit
 *      HLOSM equations (Eqs. losm-0, losm-1, losm-disc-bc);
 *   4. combs the census bank back to N particles (uniform combing, Sec. 5.1).
 *
 * Conventions for every entry point:
 *   - All functions return an hww_status; nothing throws across the ABI.
 *   - Input arrays are caller-owned and copied before the call returns.
 *   - Output arrays are caller-allocated.  When an `on_device` argument is 1
 *     the pointer is a CUDA device pointer on the problem's device (for
 *     instance a torch tensor's data_ptr()); when 0 it is host memory.
 *   - Work is enqueued on the CUDA stream given at creation (0 = the legacy
 *     default stream).  Calls that return data to host memory, and
 *     run_step with a non-NULL stats pointer, synchronize that stream;
 *     run_step itself waits once per step for its tracking stage (below).
 *   - A problem must be used from one host thread at a time.
 *   - Device memory is allocated by create_problem (stream-ordered
 *     allocation on the problem's stream) and released by destroy_problem.
 *   - Array layouts: cells are 0-based (cell k spans [edges[k],
 *     edges[k+1]]); the LOSM vectors use the paper's layout: phi has I+2
 *     entries (x_0 boundary value, cells 1..I, x_I boundary value) and J has
 *     I+1 entries (edges x_0..x_I).
 */
#ifndef HWW_H
#define HWW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hww_problem hww_problem; /* opaque, library-owned */
typedef struct hww_batch hww_batch;     /* opaque, library-owned */

typedef enum {
    HWW_OK = 0,
    HWW_ERR_ARG = 1,           /* an argument is out of range or NULL */
    HWW_ERR_STATE = 2,         /* a verb was called out of order */
    HWW_ERR_OOM = 3,           /* device or host allocation failed */
    HWW_ERR_BANK_OVERFLOW = 4, /* a particle bank or queue filled up; the step is invalid */
    HWW_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    HWW_ERR_NUMERIC = 6,       /* a numeric guard fired (split count, event count, LOSM pivot) */
    HWW_ERR_CUDA = 7,          /* a CUDA runtime call failed */
    HWW_ERR_NO_DEVICE = 8      /* no usable CUDA device */
} hww_status;

enum { HWW_BC_VACUUM = 0, HWW_BC_REFLECT = 1 };
enum { HWW_FP64 = 0, HWW_FP32_TRACK = 1 };
/* FP32 tracking kernels (hww_set_tracking) */
enum { HWW_TRACK_WARP = 0, HWW_TRACK_EVENT = 1, HWW_TRACK_AUTO = 2 };
enum { HWW_FILTER_NONE = 0, HWW_FILTER_MA = 1, HWW_FILTER_FOURIER = 2 };
/* window modes: HLOSM centers (the paper's method), analog (no windows),
 * lagged (centers from the previous step's track-length flux) */
enum { HWW_MODE_HWW = 0, HWW_MODE_ANALOG = 1, HWW_MODE_LWW = 2 };
/* center scaling: multiply Eq. (ww-center) by the mean particle weight after
 * the previous comb, or use it literally */
enum { HWW_SCALE_MEAN_WEIGHT = 0, HWW_SCALE_LITERAL = 1 };
/* get_tallies kinds; all are normalised per source particle */
enum {
    HWW_TL_PHI = 0,      /* <phi>_i^n, Eq. (phi-mc)                       [I]   */
    HWW_TL_J = 1,        /* track-length current, same normalisation      [I]   */
    HWW_TL_F = 2,        /* track-length (1/3 - mu^2) moment              [I]   */
    HWW_CENSUS_PHI = 3,  /* [[phi]]_i^n, Eq. (ct-mc)                       [I]   */
    HWW_CENSUS_J = 4,    /* census current                                [I]   */
    HWW_CENSUS_F = 5,    /* census closure F_i^n, Eq. (F)                  [I]   */
    HWW_BATCH_PHI = 6,   /* <phi> per variance batch b = floor(id B / N)   [B*I] */
    HWW_BOUNDARY = 7,    /* phi_L, F_L, P_L, phi_R, F_R, P_R time averages [6]   */
    HWW_WW_CENTER = 8,   /* window centers used in the step               [I]   */
    HWW_CLOSURE_PHI = 9, /* IC / closure vectors built at t^n            [I+2] */
    HWW_CLOSURE_J = 10,  /*                                               [I+1] */
    HWW_CLOSURE_F = 11   /*                                               [I+2] */
};
enum { HWW_LOSM_SEMI = 0, HWW_LOSM_FULL = 1 };

typedef struct {
    int32_t n_cells;          /* I >= 1 */
    const double* edges;      /* I+1 strictly increasing positions (host) */
    double v;                 /* particle speed > 0 */
    double dt;                /* time step > 0 */
    int32_t bc_left, bc_right;/* HWW_BC_VACUUM | HWW_BC_REFLECT */
    double src_x;             /* unit isotropic plane pulse at t = 0, in [edges[0], edges[I]] */
    int64_t particles_per_step; /* N, 1 <= N < 2^30 */
    uint64_t seed;            /* Philox key (with the step index) */
    int32_t precision;        /* HWW_FP64 | HWW_FP32_TRACK */
    double theta;             /* 0.5 Crank-Nicolson | 1.0 backward Euler */
    int32_t filter, filter_k; /* HWW_FILTER_NONE | HWW_FILTER_MA with base k >= 1 (Eq. moving_average) |
                                 HWW_FILTER_FOURIER with cutoff k >= 0 (Eqs. fft, ifft): the modes of
                                 frequency min(j, M - j) <= k kept */
    int32_t n_var_batches;    /* B >= 1 batches for the batch-mean variance tally */
    int32_t deriv_regions;    /* 0, or 1 <= R <= 4 regions for derivative tallies (FP64 only; the
                                 tracking needs (7 + 2R) I 8 bytes of shared memory per block,
                                 at most 227 KB) */
    int64_t bank_capacity;    /* census slots; each record queue gets half; 0 = 4 N census, 2 N per queue */
    void* cuda_stream;        /* cudaStream_t; NULL = legacy default stream */
    int32_t device;           /* CUDA device ordinal */
} hww_problem_desc;

typedef struct {
    int64_t n_start, segments, collisions, crossings, reflections;
    int64_t leaked, absorbed, scatters, split_events, daughters;
    int64_t roulette_kills, roulette_survivals, census, lineage_collisions;
    int64_t max_events, n_next;
    double w_bar_next;  /* weight of each combed particle for the next step */
    int32_t waves;      /* tracking launches the step needed */
    int32_t status;     /* hww_status of the step */
} hww_step_stats;

/* Create a problem from the description (paper Sec. 3 problem statement:
 * slab [x_0, x_I], cells of Eq. losm-disc, pulse initial condition).
 * Errors: HWW_ERR_ARG for an invalid field, HWW_ERR_NO_DEVICE, HWW_ERR_OOM,
 * HWW_ERR_CUDA.  On error *out is NULL. */
hww_status create_problem(const hww_problem_desc* desc, hww_problem** out);

/* Per-cell total cross section Sigma_t > 0 and the mean number of particles
 * a collision emits, c = (Sigma_s + nu_f Sigma_f) / Sigma_t, 0 <= c <= 16
 * (Eq. HO_transport): c <= 1 scattering and absorption, c > 1 a multiplying
 * medium, where a collision emits floor(c) + [u < c - floor(c)] particles,
 * the extra ones with their own isotropic directions.  Derivative runs need
 * c <= 1.  `region` (nullable)
 * maps each cell to a region 0..R-1 for the derivative tallies.  Host arrays
 * of length I.  May be called again between steps.  Refactors the LOSM
 * matrix and synchronizes.  Errors: HWW_ERR_ARG for a NULL array, Sigma_t
 * not finite and > 0, c outside [0, 16] (or above 1 in a derivative run) or
 * a region out of range (nothing is changed); HWW_ERR_NUMERIC when the LOSM
 * factorization meets a zero pivot. */
hww_status set_cross_sections(hww_problem* p, const double* sigma_t, const double* c,
                              const int32_t* region);

/* Window width rho >= 1 (ceiling rho*ww, floor ww/rho, Eq. ww-c&f), minimum
 * center 0 < eps_min <= 1 (Eq. ww-center), mode HWW_MODE_*, center scaling
 * HWW_SCALE_*.  HWW_ERR_ARG for a value out of range. */
hww_status set_ww_params(hww_problem* p, double rho, double eps_min, int32_t mode,
                         int32_t center_scaling);

/* Replace the window centers of the next step only (I host values > 0);
 * ceiling and floor follow from rho.  Used to run both implementations
 * from identical windows.  HWW_ERR_ARG for a center that is not finite and
 * positive. */
hww_status set_ww_centers(hww_problem* p, const double* centers);

/* In-step window updates (Sec. 3, Eq. Hpn): during a step whose windows
 * come from the HLOSM solution (HWW mode, no set_ww_centers override), the
 * start bank is tracked in n + 1 chunks of source ids [H_{p-1}, H_p),
 * H_p = floor(f_p H) of the step's H start particles; after each of the
 * first n chunks (all their descendants tracked) the windows are re-derived
 * from the fully implicit HLOSM solution closed with the census and boundary
 * tallies of the histories so far (normalised per history).  n <= 16;
 * fractions strictly increasing in (0, 1), NULL for f_p = p / (n + 1);
 * n = 0 turns the updates off (HWW_ERR_ARG for invalid fractions).  Not
 * supported for batch members (run_batch_step returns HWW_ERR_STATE). */
hww_status set_ww_updates(hww_problem* p, int32_t n, const double* fractions);

/* Advance the problem by one time step (steps 1-4 above).  The host waits
 * once, after the tracking stage, for its overflow flag: a census bank or
 * record queue that filled up leaves the start bank and the closures as they
 * were, and the step is tracked again with larger buffers (each at least
 * doubled, at most 12 times), bit-identical to a run that had the room from
 * the start.  The rest of the step (closures, HLOSM, comb) is enqueued on
 * the problem's stream without waiting, unless `stats` is non-NULL, in which
 * case the stream is synchronized and the counts of the step are returned.
 * HWW_ERR_STATE before set_cross_sections and set_ww_params.  An overflow
 * that outlasts the regrowths, or a numeric guard, makes this or the next
 * synchronizing call return the error; the step's results are then
 * invalid. */
hww_status run_step(hww_problem* p, hww_step_stats* stats);

/* Copy tally `kind` (HWW_* kinds above) of the last completed step into
 * `out` (capacity n doubles; host or device per on_device).  Values are
 * normalised per source particle: track-length kinds by N dx_i dt, census
 * kinds by N dx_i / v, boundary kinds by N dt. */
hww_status get_tallies(const hww_problem* p, int32_t kind, double* out, int64_t n,
                       int32_t on_device);

/* Raw 128-bit fixed-point accumulators of a tally kind 0..7 as (lo, hi)
 * int64 pairs (2 n values), for bit-exact comparisons.  Host memory. */
hww_status get_tallies_raw(const hww_problem* p, int32_t kind, int64_t* out, int64_t n);

/* Copy the HLOSM solution of the last step: HWW_LOSM_SEMI (the one that set
 * the windows, Eq. losm-disc-semi) or HWW_LOSM_FULL (end of step, Eq.
 * losm-disc).  phi has I+2 entries and J has I+1. */
hww_status get_losm_solution(const hww_problem* p, int32_t which, double* phi, double* J,
                             int32_t on_device);

/* ------------------------------------------------------------------------
 * Derivatives (not in the paper).  With deriv_regions = R > 0 the step also
 * estimates the derivatives of its tallies with respect to the 2R parameters
 * theta_j: j < R is Sigma_t of region j, j = R + r is c of region r (Sigma_s =
 * c Sigma_t, so Sigma_a = (1 - c) Sigma_t moves with both).  Estimator:
 * likelihood-ratio scores carried by every particle (a flight of length l
 * adds -l, a collision 1/Sigma_t, a scatter 1/c to the scores of the cell's
 * region), inherited by daughters, roulette survivors and comb copies; the
 * windows' centers count as constants (the games are unbiased for any
 * centers).  The c derivative needs c > 0 in the region.
 * ------------------------------------------------------------------------ */

/* Derivative tallies of the last step, normalised like the tallies:
 * which 0 track-length phi, 1 census phi, 2 census J, 3 census F (each
 * [2R][I], row j = d/dtheta_j), 4 boundary ([2R][6], the HWW_BOUNDARY
 * layout).  n is the capacity of out in doubles.  HWW_ERR_STATE without
 * derivatives or before the first step. */
hww_status get_deriv_tallies(const hww_problem* p, int32_t which, double* out, int64_t n, int32_t on_device);

/* Doubles of the state block that losm_vjp needs for one step. */
hww_status vjp_state_size(const hww_problem* p, int64_t* n);

/* Save the last step's state block (the step's closures at both levels, its
 * derivative closures, its fully implicit solution and its normalised
 * derivative track-length tally) into `state` (n doubles, host or device
 * memory by on_device), so that the adjoint of that step can run after later
 * steps. */
hww_status save_vjp_state(hww_problem* p, double* state, int64_t n, int32_t on_device);

/* Vector-Jacobian product of one step:
 *   grad[j] = g_mc . d<phi>/dtheta_j + g_phi . dphi_H/dtheta_j + g_J . dJ_H/dtheta_j
 * with <phi> the step's track-length flux (I), (phi_H, J_H) its fully
 * implicit HLOSM solution (I+2, I+1; Eqs. losm-0, losm-1, losm-disc-bc).
 * The HLOSM part is the adjoint of the solve: lambda = A^{-T} g by a
 * transposed Thomas sweep, contracted with the derivative closures and with
 * dA/dtheta, db/dtheta (recomputed per call, nothing stored but the state
 * block).  state: NULL for the last step, else a block from save_vjp_state of
 * this problem under its current cross sections (HWW_ERR_STATE otherwise).
 * g_mc, g_phi, g_J may be NULL (zero).  All vectors and grad (2R) are host or
 * device memory by on_device. */
hww_status losm_vjp(hww_problem* p, const double* state, const double* g_mc, const double* g_phi,
                    const double* g_J, double* grad, int32_t on_device);

/* Copy the combed bank that will start the next step (positions, directions,
 * cells; each particle carries weight stats.w_bar_next).  Host arrays of
 * capacity cap; *n receives the bank size (call with cap = 0 to query). */
hww_status get_bank(const hww_problem* p, double* x, double* mu, int32_t* cell, int64_t cap,
                    int64_t* n);

/* Replace the start bank of the next step (a checkpoint restart, or a
 * comparison from a known state): n <= N particles at positions x (inside
 * their cells), directions mu (nonzero, |mu| <= 1) and cells, each of weight
 * w_bar > 0, taking source ids 0..n-1.  Host arrays.  Synchronous.  The
 * next step starts from this bank instead of the pulse or the last comb. */
hww_status set_bank(hww_problem* p, const double* x, const double* mu, const int32_t* cell, int64_t n,
                    double w_bar);

/* Copy the census bank of the last step (the particles that reached t^n,
 * before combing): positions, directions, weights, cells, source ids and
 * lineage keys, in the device's storage order.  Host arrays of capacity
 * cap (any pointer may be NULL); *n receives the census size (cap = 0
 * queries it).  Used to check individual histories. */
hww_status get_census(const hww_problem* p, double* x, double* mu, double* w, int32_t* cell,
                      uint32_t* id, uint64_t* lin, int64_t cap, int64_t* n);

/* ---------------------------------------------------------------------
 * Batches: many independent problems stepped together on one GPU (problems
 * of uneven size and window settings).  Each member is an ordinary problem
 * (configure it with set_cross_sections / set_ww_params and read it with
 * the get_* calls through batch_problem).  A batch step runs, on the
 * batch's stream:
 *   - one CUDA graph with the pre-tracking stage of every member (step
 *     scalars, semi-implicit HLOSM, windows) as parallel branches;
 *   - per tracking wave, one persistent launch over all members: blocks
 *     pop tiles (member, id range) from a device counter, so members of
 *     very different sizes share the GPU without a launch per member;
 *   - one CUDA graph with the post-tracking stage of every member
 *     (closures, fully implicit HLOSM, comb).
 * Results are bit-identical to stepping each member alone: the tile size
 * and the event budget change only the order of integer tally additions.
 * The graphs are recorded on the first step; changing a member's window
 * mode or scaling afterwards is not supported.
 * ------------------------------------------------------------------- */
typedef struct {
    int64_t problems, segments, census, daughters, roulette_kills, absorbed, leaked;
    int32_t waves;
    int32_t status;   /* worst hww_status over the members */
    int32_t member_replays;  /* members tracked again on their own after an overflow, this step */
    int32_t member_grows;    /* members whose buffers grew ahead of demand after this step */
} hww_batch_stats;

/* Create n problems (n <= 1024) from descs (all with the same precision and
 * no derivative tallies; their cuda_stream and device fields are ignored).
 * Work is enqueued on `cuda_stream` of `device`. */
hww_status create_batch(const hww_problem_desc* descs, int32_t n, void* cuda_stream, int32_t device,
                        hww_batch** out);
/* Member i of the batch (owned by the batch; do not destroy it). */
hww_status batch_problem(hww_batch* b, int32_t i, hww_problem** out);
/* Tile size in particles (>= 256) and events per track before requeueing
 * (>= 1) of the batched tracking launches; results do not depend on them. */
hww_status batch_set_tuning(hww_batch* b, int32_t tile, int32_t emax);
/* Advance every member by one time step; stats (nullable) synchronizes.
 * As in run_step the host waits for the tracking waves.  A member whose
 * census bank or record queue overflowed gets larger buffers and is tracked
 * again on its own through the single-problem path (same result as a batch
 * that had the room; after 12 regrowths its status reports the overflow);
 * the other members' tracking stands.  A member whose census or record
 * count came within 60% of its capacity gets at least twice the capacity
 * after the step's comb.  HWW_ERR_STATE when a member lacks cross sections or
 * window parameters, or has in-step window updates. */
hww_status run_batch_step(hww_batch* b, hww_batch_stats* stats);
/* Counts of member i's last step (synchronizes). */
hww_status batch_member_stats(hww_batch* b, int32_t i, hww_step_stats* stats);
void destroy_batch(hww_batch* b);

/* Launch accounting of a problem since creation or the last reset: kernels
 * the library launched, tracking-kernel launches (of which event_launches
 * ran the event loop), the particles the event loop's blocks spilled (a
 * pass's outputs beyond the block's ring wait in the block's slice of the
 * record queue that wave 0 leaves idle, and the block tracks them itself;
 * what the slice cannot hold goes to the record queue and a further wave),
 * and (when timing is on) the device time of the tracking launches measured
 * with CUDA events on the problem's stream. */
typedef struct {
    int64_t kernel_launches;
    int64_t track_launches;
    double track_ms;
    int64_t steps;
    int64_t census_capacity, queue_capacity;
    int64_t event_launches;
    int64_t spilled;
} hww_counters;

/* The kernel that tracks an FP32 problem's start-bank particles (the events
 * of Sec. 2 and the tallies of Eq. phi-mc):
 *   HWW_TRACK_WARP  a warp-synchronous history loop: each lane follows one
 *                   track event by event and takes new work (daughters from
 *                   its warp's stack, start particles) when its track ends;
 *   HWW_TRACK_EVENT an event-based loop: blocks of 256 threads (up to four per
 *                   SM) each keep a ring of live particles in shared memory and
 *                   advance all of them by one event per pass, appending
 *                   survivors and daughters after a block-wide scan (what
 *                   the ring cannot hold waits in the block's spill in
 *                   global memory);
 *   HWW_TRACK_AUTO  the event loop where the mesh leaves room for its rings,
 *                   the warp loop otherwise (the default; FP64 problems track
 *                   with their own loop).
 * Both loops draw the same random numbers and do the same arithmetic, so a
 * step gives bit-identical tallies, census and next start bank with either;
 * the record waves (what the spills cannot hold, daughters of splits into
 * more particles than a ring holds, multiplying collisions' extra particles)
 * always run the warp loop.  HWW_ERR_ARG for an unknown kind, for
 * HWW_TRACK_EVENT or HWW_TRACK_AUTO on an FP64 problem, for HWW_TRACK_EVENT
 * on a mesh whose tallies (24 I bytes) leave even one block per SM less than
 * 24 KB of ring.  Applies from the next step. */
hww_status hww_set_tracking(hww_problem* p, int32_t kind);
/* Turn CUDA-event timing of the tracking launches on (1) or off (0). */
hww_status hww_set_timing(hww_problem* p, int32_t enable);
hww_status hww_get_counters(const hww_problem* p, hww_counters* out);
hww_status hww_reset_counters(hww_problem* p);

/* Release the problem and its device memory (NULL is allowed). */
void destroy_problem(hww_problem* p);

/* Static text for a status code. */
const char* hww_status_string(hww_status s);

/* Text of the last CUDA runtime error the library saw on this host thread
 * (name, message and the place it was caught), for HWW_ERR_CUDA diagnosis. */
const char* hww_last_error_string(void);

/* Solve one LOSM system (Eqs. losm-0, losm-1, losm-disc-bc) on the device
 * for given inputs, with the library's solver.  Host arrays in the paper's
 * layout (dx, sigma_t, sigma_a, q_old, q_new: I cells, q cell-integrated and
 * nullable; phi_old, F_old, F_new, phi_new: I+2; J_old, J_new: I+1).
 * Synchronous.  Used to check the device solver on its own. */
hww_status hww_losm_solve(int32_t n_cells, const double* dx, const double* sigma_t,
                          const double* sigma_a, double v, double dt, double theta,
                          int32_t bc_left, int32_t bc_right, const double* phi_old,
                          const double* J_old, const double* F_old, const double* F_new,
                          double PL_new, double PR_new, const double* q_old, const double* q_new,
                          double* phi_new, double* J_new);

/* The same LOSM solve as hww_losm_solve, for callers that cannot let the
 * library allocate device memory: an application whose device memory is
 * handed out up front by its own pool, a latency-critical loop in which
 * cudaMalloc / cudaFree would synchronize the device, or a process whose
 * policy forbids new device allocations after start-up.  The paper has no
 * counterpart; this is a service of the library.
 *
 * Arguments, layouts and results are those of hww_losm_solve (host arrays,
 * synchronous, on the current device).  Instead of allocating, the call
 * stages everything in a fixed device array compiled into the library,
 * sized for n_cells <= HWW_NOALLOC_MAX_CELLS (about 0.8 MB, held on every
 * GPU that loads the library until the process exits); larger n_cells
 * return HWW_ERR_ARG.  Every call looks up that array's device address
 * on the current device (so the address is never stale, for instance
 * after a context reset); make the first call on a device before any
 * stream capture.  The call uses no cudaMalloc, cudaFree or other
 * allocating routine.  A CUDA error is recorded for
 * hww_last_error_string, as hww_losm_solve does.  All calls on a device share the array, which keeps
 * the previous call's contents (the call clears what must start at zero),
 * so calls that overlap on the GPU, for instance from two host threads at
 * the same time, race. */
#define HWW_NOALLOC_MAX_CELLS 4096
hww_status hww_losm_solve_noalloc(int32_t n_cells, const double* dx, const double* sigma_t,
                                  const double* sigma_a, double v, double dt, double theta,
                                  int32_t bc_left, int32_t bc_right, const double* phi_old,
                                  const double* J_old, const double* F_old, const double* F_new,
                                  double PL_new, double PR_new, const double* q_old,
                                  const double* q_new, double* phi_new, double* J_new);

/* The current device's FP64 fused multiply-add rate in floating-point
 * operations per second (two per DFMA), measured by the library's own loop:
 * 8 independent DFMA chains per thread, `iters` iterations, 8 blocks of 256
 * threads per SM, timed with CUDA events after a short warm-up.  The paper
 * has no counterpart: it is the denominator of the FP64 path's ALU
 * roofline.  Synchronous; allocates one double. */
hww_status hww_dfma_rate(int64_t iters, double* flops_per_s);

/* Philox4x32-10 of n consecutive counters {c0 + i, c1, c2, c3} under key
 * (k0, k1), computed by the library's device generator; out holds 4 n
 * words (host).  Synchronous.  Used to check the generator. */
hww_status hww_philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                            uint32_t k1, int64_t n, uint32_t* out);

#ifdef __cplusplus
}
#endif
#endif /* HWW_H */

// losm_kernels.cuh -- argument blocks of the closure, LOSM and window stages.
#pragma once
#include "hww_internal.cuh"

namespace hww {

// constant part of the discrete LOSM system of one problem
struct LosmMat {
    int I;
    double theta;
    int bc_l, bc_r;
    double* eJ;      // [I+1] dxhat_i / (v dt)
    double* eS;      // [I+1] Sigma_hat_i dxhat_i
    double* invd;    // [I+1] 1 / d_i
    double* g;       // [I+1] theta / (3 d_i)
    double* cP;      // [I]   dx_i / (v dt)
    double* cA;      // [I]   Sigma_a,i dx_i
    double* cB;      // [I]   dx_i / (v dt) + theta Sigma_a,i dx_i
    double* inv_den; // [I+2] Thomas pivots, inverted
    double* vf;      // [I+2] -A_r / den_r
    double* cp;      // [I+2] C_r / den_r
    double* nA;      // [I+2] -A_r, for the transposed solve (nullable)
};

// right-hand-side inputs of one solve (paper layout).  With `sd` set, the
// vectors come from the two closure sets by the device's parity: the old
// level is set `cur`; the new-level closure is set `cur` again for the
// semi-implicit solve (full = 0) and set 1-cur for the fully implicit one.
// Without `sd`, the explicit pointers and values are used.
struct LosmRhsIn {
    const StepDev* sd;
    int full;
    const double* set_phi[2];
    const double* set_J[2];
    const double* set_F[2];
    const double* set_P[2];
    const double* phi_old;  // I+2
    const double* J_old;    // I+1
    const double* F_old;    // I+2
    const double* F_new;    // I+2
    const double* P_new;    // device [2] or NULL (then PL, PR)
    double PL, PR;
    const double* q_old;    // I or NULL
    const double* q_new;    // I or NULL
};

struct LosmWork {
    double* u;    // I+2
    double* mom;  // I+1
    double* y;    // I+2
};

struct WwArgs {
    int I;
    int scaling;  // 0 mean weight, 1 literal
    double eps, rho;
    const StepDev* sd;       // ww_src picks the source: 1 HLOSM, 2 previous flux, 3 override
    const double* phit_hlosm;
    const double* phit_prev;
    const double* mx_hlosm;
    const double* mx_prev;
    const double* override_c;
    double *ww_c, *ww_hi, *ww_lo;
    double2* ww_hl;  // (ceiling, floor) packed for the tracking kernels
};

struct ClosureArgs {
    int I;
    const StepDev* sd;
    double v, dt;
    long long N;
    int bc_l, bc_r;
    int filter_k;                  // MA base (0: no MA filter)
    int fourier, kappa;            // Fourier low-pass with cutoff kappa instead
    const double* dx;
    const Acc128* cent;
    const Acc128* tl;
    const Acc128* bnd;
    double *rphi, *rJ, *rF;        // unfiltered: I, I+1, I
    double *set_phi[2], *set_J[2], *set_F[2], *set_P[2];  // closure sets; t^n goes to 1-cur
    double* prev_tl;               // I (written when tl is set)
    // several closure sets at once (the derivative closures, one per
    // parameter; blockIdx.y picks the set): consecutive sets are 3I
    // accumulators apart in cent, 6 in bnd, I+1 in the scratch vectors and
    // I+2 / I+1 / I+2 / 2 in the phi / J / F / P sets
    int nsets;
};

// adjoint of the fully implicit solve of the last step (transpose Thomas)
// contracted with the parameter directions; the step's vectors come from a
// state block laid out by vjp_state_offsets
struct VjpArgs {
    LosmMat m;
    const double* dx;
    const double* sigt;
    const double* c;
    const int32_t* region;
    int R, P2;
    const double* state;
    const double* g_mc;   // I or NULL
    const double* g_phi;  // I+2
    const double* g_J;    // I+1
    double* psi;          // work: I+2 (even unknowns of lambda)
    double* z;            // work: I+2
    double* grad;         // P2
};

// doubles of a state block and the offsets of its parts
struct VjpLayout {
    long long phi_old, J_old, phi_new, J_new, dtl, dphi_old, dJ_old, dF_old, dF_new, dP_new, total;
};
__host__ __device__ inline VjpLayout vjp_layout(int I, int P2) {
    VjpLayout L;
    long long o = 4;  // header: I, P2, cross-section version, spare
    L.phi_old = o; o += I + 2;
    L.J_old = o; o += I + 1;
    L.phi_new = o; o += I + 2;
    L.J_new = o; o += I + 1;
    L.dtl = o; o += (long long)P2 * I;
    L.dphi_old = o; o += (long long)P2 * (I + 2);
    L.dJ_old = o; o += (long long)P2 * (I + 1);
    L.dF_old = o; o += (long long)P2 * (I + 2);
    L.dF_new = o; o += (long long)P2 * (I + 2);
    L.dP_new = o; o += (long long)P2 * 2;
    L.total = o;
    return L;
}

void launch_losm_setup(const LosmMat& m, const double* dx, const double* sigt, const double* siga, double v,
                       double dt, double theta, int bc_l, int bc_r, unsigned* err, cudaStream_t s);
int launch_losm_solve(const LosmMat& m, const LosmRhsIn& in, const LosmWork& w, double* phi, double* J,
                      double* mx, cudaStream_t s);
// A standalone LOSM solve from host vectors (hww_losm_solve and its
// no-allocation variant): the cell arrays, the old and new vectors, the
// factorized matrix, the work vectors and an error word are carved from one
// device block of losm_staged_doubles(I) doubles at `base`; the inputs are
// copied in, the solve runs on the default stream, and phi (I+2), J (I+1) are
// copied back.  Synchronous.  Returns the first CUDA error; *numeric is set
// when the solver's guard fired.
constexpr size_t losm_staged_doubles(size_t I) { return 24 * I + 26; }
cudaError_t losm_solve_staged(double* base, int I, const double* dx, const double* sigma_t, const double* sigma_a,
                              double v, double dt, double theta, int bc_left, int bc_right, const double* phi_old,
                              const double* J_old, const double* F_old, const double* F_new, double PL_new,
                              double PR_new, const double* q_old, const double* q_new, double* phi_new,
                              double* J_new, bool* numeric);
int launch_ww_centers(const WwArgs& a, int lagged, cudaStream_t s);
void launch_step_scalars(StepDev* sd, int nbits, unsigned long long seed, int mode, unsigned long long* stats,
                         cudaStream_t s);
int launch_closures(const ClosureArgs& a, cudaStream_t s);
int fourier_filter_smem_optin(size_t smem);
int launch_losm_vjp(const VjpArgs& a, cudaStream_t s);

}  // namespace hww

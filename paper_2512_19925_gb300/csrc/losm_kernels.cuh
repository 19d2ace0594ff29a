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
};

// right-hand-side inputs of one solve (paper layout)
struct LosmRhsIn {
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
    int source;   // 1 HLOSM solution, 2 previous track-length flux, 3 override
    int scaling;  // 0 mean weight, 1 literal
    double eps, rho;
    const StepDev* sd;
    const double* phit;
    const double* mx_ptr;
    const double* override_c;
    double *ww_c, *ww_hi, *ww_lo;
};

struct ClosureArgs {
    int I;
    const StepDev* sd;
    double v, dt;
    long long N;
    int bc_l, bc_r;
    int filter_k;
    const double* dx;
    const Acc128* cent;
    const Acc128* tl;
    const Acc128* bnd;
    double *rphi, *rJ, *rF;        // unfiltered: I, I+1, I
    double *nphi, *nJ, *nF, *nP;   // closure set at t^n: I+2, I+1, I+2, 2
    double* prev_tl;               // I
};

void launch_losm_setup(const LosmMat& m, const double* dx, const double* sigt, const double* siga, double v,
                       double dt, double theta, int bc_l, int bc_r, unsigned* err, cudaStream_t s);
int launch_losm_solve(const LosmMat& m, const LosmRhsIn& in, const LosmWork& w, double* phi, double* J,
                      double* mx, cudaStream_t s);
int launch_ww_centers(const WwArgs& a, cudaStream_t s);
void launch_step_scalars(StepDev* sd, int nbits, uint32_t k0, uint32_t k1, unsigned long long* stats,
                         cudaStream_t s);
int launch_closures(const ClosureArgs& a, cudaStream_t s);

}  // namespace hww

// step_kernels.cuh -- argument blocks of the stages around the tracking kernel.
#pragma once
#include "hww_internal.cuh"

namespace hww {

// inputs of one LOSM solve (paper layout: phi and F of length I+2, J of I+1,
// cell arrays of length I, q cell-integrated and nullable)
struct LosmIn {
    int I;
    const double* dx;
    const double* sigt;
    const double* siga;
    double v, dt, theta;
    int bc_l, bc_r;
    const double* phi_old;
    const double* J_old;
    const double* F_old;
    const double* F_new;
    double PL, PR;
    const double* q_old;
    const double* q_new;
};

struct PreArgs {
    StepDev* sd;
    int nbits;          // bit length of N
    uint32_t k0, k1;    // Philox key of the step
    LosmIn losm;        // semi-implicit solve (F_new = F_old)
    const double* P_old;  // device [2]: P_L, P_R of the previous step
    double* semi_phi;
    double* semi_J;
    double *w_d, *w_m, *w_c, *w_r;
    unsigned* err;
    int ww_source;      // 0 none, 1 semi-implicit HLOSM, 2 previous track-length flux, 3 override
    int scaling;        // 0 mean weight, 1 literal
    double eps, rho;
    const double* prev_tl;
    const double* ww_override;
    double *ww_c, *ww_hi, *ww_lo;
    unsigned long long* stats;
};

struct PostArgs {
    int I;
    const StepDev* sd;
    double v, dt;
    long long N;
    int bc_l, bc_r;
    int filter_k;       // 0 = no filter
    const double* dx;
    const Acc128* cent;
    const Acc128* tl;
    const Acc128* bnd;
    double *nphi, *nJ, *nF, *nP;  // closure set at t^n being built
    double* cJ;
    double* tmp;
    double* prev_tl;
    double *ophi, *oJ, *oF, *oP;  // closure set of the step start
    LosmIn losm;                  // full solve; old-level vectors = o*
    double* full_phi;
    double* full_J;
    double *w_d, *w_m, *w_c, *w_r;
    unsigned* err;
};

struct ScanArgs {
    const uint32_t* cnt;
    const unsigned long long* w;
    long long n;
    unsigned long long* tile_c;
    unsigned long long* tile_w;
    unsigned long long* out_c;  // n+1 entries
    unsigned long long* out_w;  // n+1 entries
};

template <class Real>
struct CombArgs {
    StepDev* sd;
    long long N;
    const unsigned long long* ncensus_ptr;
    long long cen_cap;
    const Real* cx;
    const Real* cmu;
    const double* cw;
    const int32_t* ccell;
    const uint32_t* cid;
    const uint64_t* clin;
    const uint32_t* gcnt;
    const unsigned long long* goff;
    const unsigned long long* goff_w;
    uint32_t* gcur;
    uint32_t* member;
    Real* bx;
    Real* bmu;
    int32_t* bcell;
    unsigned long long* stats;
    unsigned* err;
};

void launch_prestep(const PreArgs& a, cudaStream_t s);
void launch_poststep(const PostArgs& a, cudaStream_t s);
void launch_group_scan(const ScanArgs& a, cudaStream_t s);
long long group_scan_tiles(long long n);
template <class Real>
void launch_comb(const CombArgs<Real>& a, int grid, cudaStream_t s);
void launch_losm_only(const LosmIn& in, double* phi, double* J, double* work, unsigned* err,
                      cudaStream_t s);
void launch_philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                         long long n, uint32_t* out, cudaStream_t s);

int track_smem_optin_fp64(size_t smem);
int track_smem_optin_fp32(size_t smem);
int track_blocks_per_sm_fp64(int block, size_t smem);
int track_blocks_per_sm_fp32(int block, size_t smem);

}  // namespace hww

// noalloc.cu -- a LOSM-solve entry point that allocates no memory.
//
// hww_losm_solve stages its inputs, the factorized matrix and its work
// vectors in device memory it obtains with cudaMalloc.  Some callers cannot
// let a library do that: an application whose device memory is handed out
// up front by its own pool (a later cudaMalloc fails or fragments the pool),
// a latency-critical loop in which cudaMalloc / cudaFree would synchronize
// the device, or a host process whose policy forbids new device allocations
// after start-up.  hww_losm_solve_noalloc gives them the same solve with its
// scratch in a fixed device array that is part of the loaded library.
//
// The array has room for HWW_NOALLOC_MAX_CELLS cells (about 0.8 MB); every
// GPU that loads the library holds it until the process exits.  Its device
// address is looked up once per device, on the first call made with that
// device current.  All calls on a device share the array, so calls that
// overlap on the GPU (for instance from two host threads at once) race.
#include <cmath>
#include <mutex>

#include "../../include/hww.h"
#include "losm_kernels.cuh"

using namespace hww;

namespace {

// doubles the solve needs for I cells: inputs 5 I + 3 (I+2) + (I+1),
// outputs (I+2) + (I+1), matrix 4 (I+1) + 3 I + 3 (I+2), work 2 (I+2) + (I+1),
// and one word for the error flags
constexpr size_t scratch_doubles(size_t I) { return 24 * I + 26; }
constexpr size_t SCRATCH_DOUBLES = scratch_doubles(HWW_NOALLOC_MAX_CELLS);
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_losm_scratch[SCRATCH_DOUBLES];

double* g_scratch_addr[MAX_DEVICES] = {};
std::mutex g_setup_mutex;

// device address of the scratch array on the current device (looked up on
// the first call per device)
hww_status scratch_on_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HWW_ERR_NO_DEVICE;
    if (dev < 0 || dev >= MAX_DEVICES) return HWW_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_losm_scratch);
        if (e != cudaSuccess || !p) return HWW_ERR_CUDA;
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return HWW_OK;
}

}  // namespace

extern "C" hww_status hww_losm_solve_noalloc(int32_t I, const double* dx, const double* sigma_t,
                                             const double* sigma_a, double v, double dt, double theta,
                                             int32_t bc_left, int32_t bc_right, const double* phi_old,
                                             const double* J_old, const double* F_old, const double* F_new,
                                             double PL_new, double PR_new, const double* q_old,
                                             const double* q_new, double* phi_new, double* J_new) {
    if (I < 1 || !dx || !sigma_t || !sigma_a || !phi_old || !J_old || !F_old || !F_new || !phi_new || !J_new ||
        !(v > 0) || !(dt > 0) || (theta != 0.5 && theta != 1.0) || bc_left < 0 || bc_left > 1 || bc_right < 0 ||
        bc_right > 1)
        return HWW_ERR_ARG;
    if (I > HWW_NOALLOC_MAX_CELLS) return HWW_ERR_ARG;  // larger than the fixed scratch array
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return HWW_ERR_NO_DEVICE;
    double* q = nullptr;
    hww_status st = scratch_on_current_device(&q);
    if (st) return st;
    auto take = [&](size_t k) {
        double* r = q;
        q += k;
        return r;
    };
    const size_t n2 = I + 2, n1 = I + 1;
    double* d_dx = take(I);
    double* d_st = take(I);
    double* d_sa = take(I);
    double* d_qo = take(I);
    double* d_qn = take(I);
    double* d_po = take(n2);
    double* d_Fo = take(n2);
    double* d_Fn = take(n2);
    double* d_Jo = take(n1);
    double* d_pn = take(n2);
    double* d_Jn = take(n1);
    LosmMat m{};
    m.I = I;
    m.theta = theta;
    m.bc_l = bc_left;
    m.bc_r = bc_right;
    m.eJ = take(n1);
    m.eS = take(n1);
    m.invd = take(n1);
    m.g = take(n1);
    m.cP = take(I);
    m.cA = take(I);
    m.cB = take(I);
    m.inv_den = take(n2);
    m.vf = take(n2);
    m.cp = take(n2);
    LosmWork w{};
    w.u = take(n2);
    w.y = take(n2);
    w.mom = take(n1);
    unsigned* d_err = (unsigned*)take(1);

    cudaError_t e = cudaSuccess;
    auto up = [&](double* dst, const double* src, size_t cnt) {
        if (e == cudaSuccess && src) e = cudaMemcpy(dst, src, cnt * sizeof(double), cudaMemcpyHostToDevice);
    };
    up(d_dx, dx, I);
    up(d_st, sigma_t, I);
    up(d_sa, sigma_a, I);
    up(d_qo, q_old, I);
    up(d_qn, q_new, I);
    up(d_po, phi_old, n2);
    up(d_Fo, F_old, n2);
    up(d_Fn, F_new, n2);
    up(d_Jo, J_old, n1);
    // the array keeps the previous call's contents: the error word starts at 0
    if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        launch_losm_setup(m, d_dx, d_st, d_sa, v, dt, theta, bc_left, bc_right, d_err, 0);
        LosmRhsIn in{};
        in.phi_old = d_po;
        in.J_old = d_Jo;
        in.F_old = d_Fo;
        in.F_new = d_Fn;
        in.P_new = nullptr;
        in.PL = PL_new;
        in.PR = PR_new;
        in.q_old = q_old ? d_qo : nullptr;
        in.q_new = q_new ? d_qn : nullptr;
        launch_losm_solve(m, in, w, d_pn, d_Jn, nullptr, 0);
        e = cudaGetLastError();
    }
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(phi_new, d_pn, n2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(J_new, d_Jn, n1 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return (e == cudaErrorMemoryAllocation) ? HWW_ERR_OOM : HWW_ERR_CUDA;
    return herr ? HWW_ERR_NUMERIC : HWW_OK;
}

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
// address is looked up on every call, with the calling thread's device
// current (a lookup costs little, and an address cached across a context
// reset would be stale).  All calls on a device share the array, so calls
// that overlap on the GPU (for instance from two host threads at once) race.
#include <cmath>

#include "../../include/hww.h"
#include "hww_internal.cuh"
#include "losm_kernels.cuh"

using namespace hww;

namespace {

constexpr size_t SCRATCH_DOUBLES = losm_staged_doubles(HWW_NOALLOC_MAX_CELLS);

static __device__ __align__(256) double g_losm_scratch[SCRATCH_DOUBLES];
static_assert(sizeof(g_losm_scratch) >= losm_staged_doubles(HWW_NOALLOC_MAX_CELLS) * sizeof(double),
              "the fixed scratch array must hold the solve's staging block at the largest size");

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
    // the array's address on the current device (a host-side name is not a
    // device address)
    void* base = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&base, g_losm_scratch);
    if (e != cudaSuccess) return record_cuda_error(e);
    if (!base) return HWW_ERR_CUDA;
    bool numeric = false;
    e = losm_solve_staged((double*)base, I, dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, phi_old, J_old,
                          F_old, F_new, PL_new, PR_new, q_old, q_new, phi_new, J_new, &numeric);
    if (e != cudaSuccess) return record_cuda_error(e);
    return numeric ? HWW_ERR_NUMERIC : HWW_OK;
}

// step.cu -- the O(I) and O(N) stages around the tracking kernel:
//   prestep   step scalars, semi-implicit HLOSM solve (Eqs. losm-0,
//             losm-1-semi, losm-disc-bc-semi) and window centers (Eq.
//             ww-center, Eq. ww-c&f);
//   poststep  census tallies -> closures and initial conditions (Eq. ct-mc,
//             linear edge-current interpolation, moving-average filter Eq.
//             moving_average) and the fully implicit HLOSM solve (Eqs.
//             losm-0, losm-1, losm-disc-bc);
//   comb      uniform combing of the census bank back to N (Sec. 5.1):
//             canonical order by (source id, lineage key) via per-id groups,
//             exact fixed-point cumulative weights, teeth (k + u) W / N.
// Built with contraction off so that the closure arithmetic and the comb
// positions are the single IEEE operations written.
#include "hww_internal.cuh"
#include "step_kernels.cuh"

namespace hww {
namespace {

__device__ __forceinline__ int wbar_exponent(double wbar) {
    if (!(wbar > 0.0)) return 0;
    int e;
    frexp(wbar, &e);
    return e - 1;
}

// ---------------------------------------------------------------------------
// LOSM solver.  The interleaved system of Eqs. (losm-0), (losm-1),
// (losm-disc-bc) is reduced to a tridiagonal system in phi alone: each
// first-moment row gives J_i = m_i/d_i + g_i (phi_i - phi_{i+1}) with
// g_i = theta / (3 d_i), which substituted into the balance rows and the
// boundary rows leaves a diagonally dominant tridiagonal system of size I+2,
// solved by the Thomas algorithm; J then follows from the same relation.
// Assembly terms are formed exactly as the interleaved rows are.
// ---------------------------------------------------------------------------
__device__ void losm_solve_serial(const LosmIn in, double* phi_new, double* J_new, double* w_d,
                                  double* w_m, double* w_c, double* w_r, unsigned* err) {
    const int I = in.I;
    const double vdt = in.v * in.dt;
    const double th = in.theta;
    const double tm1 = th - 1.0;
    // first-moment rows: d_i (diagonal), m_i (right-hand side)
    for (int i = 0; i <= I; ++i) {
        const double dxl = (i >= 1) ? in.dx[i - 1] : 0.0;
        const double dxr = (i <= I - 1) ? in.dx[i] : 0.0;
        const double stl = (i >= 1) ? in.sigt[i - 1] : 0.0;
        const double str = (i <= I - 1) ? in.sigt[i] : 0.0;
        const double dxh = 0.5 * (dxl + dxr);
        const double sth = (stl * dxl + str * dxr) / (dxl + dxr);
        const double d = dxh / vdt + th * sth * dxh;
        const double old = (in.phi_old[i + 1] - in.phi_old[i]) / 3.0 + sth * dxh * in.J_old[i] -
                           in.F_old[i + 1] + in.F_old[i];
        const double m = dxh / vdt * in.J_old[i] + th * (in.F_new[i + 1] - in.F_new[i]) + tm1 * old;
        w_d[i] = d;
        w_m[i] = m;
    }
    // Thomas forward sweep over rows 0..I+1 (c' in w_c, r' in w_r)
    double cprev = 0.0, rprev = 0.0;
    for (int i = 0; i <= I + 1; ++i) {
        double A, B, C, R;
        if (i == 0) {
            const double g = th / (3.0 * w_d[0]);
            A = 0.0;
            C = -g;
            if (in.bc_l == 1) {
                B = g;
                R = -w_m[0] / w_d[0];
            } else {
                B = 0.5 + g;
                R = in.PL - w_m[0] / w_d[0];
            }
        } else if (i == I + 1) {
            const double g = th / (3.0 * w_d[I]);
            A = -g;
            C = 0.0;
            if (in.bc_r == 1) {
                B = g;
                R = w_m[I] / w_d[I];
            } else {
                B = g + 0.5;
                R = in.PR + w_m[I] / w_d[I];
            }
        } else {
            const double dxi = in.dx[i - 1];
            const double gl = th / (3.0 * w_d[i - 1]);
            const double gr = th / (3.0 * w_d[i]);
            const double b = dxi / vdt + th * in.siga[i - 1] * dxi;
            const double qn = in.q_new ? in.q_new[i - 1] : 0.0;
            const double qo = in.q_old ? in.q_old[i - 1] : 0.0;
            const double oldb = in.J_old[i] - in.J_old[i - 1] + in.siga[i - 1] * dxi * in.phi_old[i] - qo;
            const double r = dxi / vdt * in.phi_old[i] + th * qn + tm1 * oldb;
            A = -th * gl;
            C = -th * gr;
            B = b + th * gl + th * gr;
            R = r + th * w_m[i - 1] / w_d[i - 1] - th * w_m[i] / w_d[i];
        }
        const double den = B - A * cprev;
        if (den == 0.0 || !isfinite(den)) {
            atomicOr(err, ERR_LOSM);
            return;
        }
        const double inv = 1.0 / den;
        cprev = C * inv;
        rprev = (R - A * rprev) * inv;
        w_c[i] = cprev;
        w_r[i] = rprev;
    }
    phi_new[I + 1] = w_r[I + 1];
    for (int i = I; i >= 0; --i) phi_new[i] = w_r[i] - w_c[i] * phi_new[i + 1];
    for (int i = 0; i <= I; ++i) {
        const double g = th / (3.0 * w_d[i]);
        J_new[i] = w_m[i] / w_d[i] + g * (phi_new[i] - phi_new[i + 1]);
    }
}

// window centers from a cell vector (Eq. ww-center with the clamp at 0)
__device__ void ww_centers(const double* phit, int I, double scale, double eps, double rho,
                           double* ww_c, double* ww_hi, double* ww_lo, double* red) {
    double mx = 0.0;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const double f = phit[i] > 0.0 ? phit[i] : 0.0;
        mx = fmax(mx, f);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    mx = red[0];
    __syncthreads();
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const double f = phit[i] > 0.0 ? phit[i] : 0.0;
        const double ratio = (mx > 0.0) ? f / mx : 1.0;
        const double b = ratio * (1.0 - eps) + eps;
        const double ctr = scale * b;
        ww_c[i] = ctr;
        ww_hi[i] = ctr * rho;
        ww_lo[i] = ctr / rho;
    }
}

__global__ void prestep_kernel(PreArgs a) {
    __shared__ double red[256];
    StepDev* sd = a.sd;
    if (threadIdx.x == 0) {
        const int E = wbar_exponent(sd->wbar);
        sd->S = 40 - E;
        sd->Sc = 59 - E - a.nbits;
        sd->tscale = pow2(sd->S);
        sd->cscale = pow2(sd->Sc);
        uint32_t r[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xC0B0u};
        philox4x32_10(r, a.k0, a.k1);
        sd->u_comb = u01(r[0], r[1]);
        a.stats[ST_NSTART] = sd->nbank;
        LosmIn in = a.losm;
        in.PL = a.P_old[0];
        in.PR = a.P_old[1];
        losm_solve_serial(in, a.semi_phi, a.semi_J, a.w_d, a.w_m, a.w_c, a.w_r, a.err);
    }
    __syncthreads();
    const double scale = (a.scaling == 0) ? sd->wbar : 1.0;
    if (a.ww_source == 1) {
        ww_centers(a.semi_phi + 1, a.losm.I, scale, a.eps, a.rho, a.ww_c, a.ww_hi, a.ww_lo, red);
    } else if (a.ww_source == 2) {
        ww_centers(a.prev_tl, a.losm.I, scale, a.eps, a.rho, a.ww_c, a.ww_hi, a.ww_lo, red);
    } else if (a.ww_source == 3) {
        for (int i = threadIdx.x; i < a.losm.I; i += blockDim.x) {
            const double ctr = a.ww_override[i];
            a.ww_c[i] = ctr;
            a.ww_hi[i] = ctr * a.rho;
            a.ww_lo[i] = ctr / a.rho;
        }
    }
}

// moving average with the symmetric shrink at the ends; the sum runs over
// the window from its right end to its left end
__device__ void ma_filter_dev(const double* in, double* out, int m, int k) {
    for (int j = 1 + threadIdx.x; j <= m; j += blockDim.x) {
        int kk = k;
        if (j - 1 < kk) kk = j - 1;
        if (m - j < kk) kk = m - j;
        double s = 0.0;
        for (int l = -kk; l <= kk; ++l) s = s + in[j - l - 1];
        out[j - 1] = s / (double)(2 * kk + 1);
    }
}

__global__ void poststep_kernel(PostArgs a) {
    const int I = a.I;
    const StepDev* sd = a.sd;
    const double isc = pow2(-sd->S);
    const double v = a.v;
    const double N = (double)a.N;
    // normalised census tallies (cell vectors, 0-based) into the new closure
    // vectors (paper layout)
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const double den = N * a.dx[i];
        a.nphi[i + 1] = (v * (acc_to_double(a.cent[i]) * isc)) / den;
        a.nF[i + 1] = (v * (acc_to_double(a.cent[2 * I + i]) * isc)) / den;
        a.cJ[i] = (v * (acc_to_double(a.cent[I + i]) * isc)) / den;
        a.prev_tl[i] = (acc_to_double(a.tl[i]) * isc) / ((N * a.dx[i]) * a.dt);
    }
    __syncthreads();
    const double PL = (a.bc_l == 1) ? 0.0 : (acc_to_double(a.bnd[2]) * isc) / (N * a.dt);
    const double PR = (a.bc_r == 1) ? 0.0 : (acc_to_double(a.bnd[5]) * isc) / (N * a.dt);
    for (int i = 1 + threadIdx.x; i <= I - 1; i += blockDim.x) {
        const double dl = a.dx[i - 1], dr = a.dx[i];
        a.nJ[i] = (a.cJ[i - 1] * dr + a.cJ[i] * dl) / (dl + dr);
    }
    if (threadIdx.x == 0) {
        a.nphi[0] = a.nphi[1];
        a.nphi[I + 1] = a.nphi[I];
        a.nF[0] = a.nF[1];
        a.nF[I + 1] = a.nF[I];
        a.nJ[0] = (a.bc_l == 1) ? 0.0 : (-0.5 * a.nphi[0] + PL);
        a.nJ[I] = (a.bc_r == 1) ? 0.0 : (0.5 * a.nphi[I + 1] - PR);
        a.nP[0] = PL;
        a.nP[1] = PR;
    }
    __syncthreads();
    if (a.filter_k > 0) {
        ma_filter_dev(a.nphi + 1, a.tmp, I, a.filter_k);
        __syncthreads();
        for (int i = threadIdx.x; i < I; i += blockDim.x) a.nphi[i + 1] = a.tmp[i];
        __syncthreads();
        ma_filter_dev(a.nF + 1, a.tmp, I, a.filter_k);
        __syncthreads();
        for (int i = threadIdx.x; i < I; i += blockDim.x) a.nF[i + 1] = a.tmp[i];
        __syncthreads();
        ma_filter_dev(a.nJ, a.tmp, I + 1, a.filter_k);
        __syncthreads();
        for (int i = threadIdx.x; i <= I; i += blockDim.x) a.nJ[i] = a.tmp[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        LosmIn in = a.losm;  // old-level vectors are the closure set of the step start
        in.F_new = a.nF;
        in.PL = a.nP[0];
        in.PR = a.nP[1];
        losm_solve_serial(in, a.full_phi, a.full_J, a.w_d, a.w_m, a.w_c, a.w_r, a.err);
    }
}

// copy the new closure set over the old one (next step's initial conditions)
__global__ void closure_commit_kernel(PostArgs a) {
    const int I = a.I;
    for (int i = threadIdx.x; i < I + 2; i += blockDim.x) {
        a.ophi[i] = a.nphi[i];
        a.oF[i] = a.nF[i];
    }
    for (int i = threadIdx.x; i < I + 1; i += blockDim.x) a.oJ[i] = a.nJ[i];
    if (threadIdx.x < 2) a.oP[threadIdx.x] = a.nP[threadIdx.x];
}

// ---------------------------------------------------------------------------
// Exclusive scan of (count, weight) pairs over the N source ids, in three
// passes: tile sums, scan of tile sums, tile rescan with the tile offset.
// ---------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

struct Pair {
    unsigned long long c, w;
};

__device__ __forceinline__ Pair padd(Pair a, Pair b) { return Pair{a.c + b.c, a.w + b.w}; }

// block-wide exclusive scan; returns the block total
__device__ Pair block_exclusive_scan(Pair& x) {
    __shared__ unsigned long long sc[SCAN_BLOCK / 32], sw[SCAN_BLOCK / 32];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    Pair inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long c = __shfl_up_sync(0xffffffffu, inc.c, o);
        const unsigned long long w = __shfl_up_sync(0xffffffffu, inc.w, o);
        if ((int)lane >= o) {
            inc.c += c;
            inc.w += w;
        }
    }
    if (lane == 31) {
        sc[warp] = inc.c;
        sw[warp] = inc.w;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = SCAN_BLOCK / 32;
        unsigned long long c = (lane < (unsigned)nw) ? sc[lane] : 0ull;
        unsigned long long w = (lane < (unsigned)nw) ? sw[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long c2 = __shfl_up_sync(0xffffffffu, c, o);
            const unsigned long long w2 = __shfl_up_sync(0xffffffffu, w, o);
            if ((int)lane >= o) {
                c += c2;
                w += w2;
            }
        }
        if (lane < (unsigned)nw) {
            sc[lane] = c;
            sw[lane] = w;
        }
    }
    __syncthreads();
    const Pair tot{sc[SCAN_BLOCK / 32 - 1], sw[SCAN_BLOCK / 32 - 1]};
    const Pair before = (warp > 0) ? Pair{sc[warp - 1], sw[warp - 1]} : Pair{0ull, 0ull};
    x = Pair{before.c + inc.c - x.c, before.w + inc.w - x.w};
    __syncthreads();
    return tot;
}

__device__ __forceinline__ Pair load_pair(const uint32_t* cnt, const unsigned long long* w, long long i,
                                          long long n) {
    if (i < n) return Pair{cnt[i], w[i]};
    return Pair{0ull, 0ull};
}

__global__ void __launch_bounds__(SCAN_BLOCK) scan_tiles_kernel(ScanArgs a) {
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    Pair s{0ull, 0ull};
    for (int k = 0; k < SCAN_ITEMS; ++k)
        s = padd(s, load_pair(a.cnt, a.w, base + (long long)threadIdx.x * SCAN_ITEMS + k, a.n));
    const Pair tot = block_exclusive_scan(s);
    if (threadIdx.x == 0) {
        a.tile_c[blockIdx.x] = tot.c;
        a.tile_w[blockIdx.x] = tot.w;
    }
}

__global__ void __launch_bounds__(SCAN_BLOCK) scan_tile_sums_kernel(ScanArgs a, long long ntiles) {
    Pair carry{0ull, 0ull};
    for (long long b = 0; b < ntiles; b += SCAN_BLOCK) {
        const long long i = b + threadIdx.x;
        Pair x = (i < ntiles) ? Pair{a.tile_c[i], a.tile_w[i]} : Pair{0ull, 0ull};
        const Pair tot = block_exclusive_scan(x);
        if (i < ntiles) {
            a.tile_c[i] = carry.c + x.c;
            a.tile_w[i] = carry.w + x.w;
        }
        carry = padd(carry, tot);
    }
    if (threadIdx.x == 0) {
        a.out_c[a.n] = carry.c;
        a.out_w[a.n] = carry.w;
    }
}

__global__ void __launch_bounds__(SCAN_BLOCK) scan_apply_kernel(ScanArgs a) {
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    Pair v[SCAN_ITEMS];
    Pair s{0ull, 0ull};
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = load_pair(a.cnt, a.w, base + (long long)threadIdx.x * SCAN_ITEMS + k, a.n);
        s = padd(s, v[k]);
    }
    block_exclusive_scan(s);
    Pair run{a.tile_c[blockIdx.x] + s.c, a.tile_w[blockIdx.x] + s.w};
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const long long i = base + (long long)threadIdx.x * SCAN_ITEMS + k;
        if (i < a.n) {
            a.out_c[i] = run.c;
            a.out_w[i] = run.w;
        }
        run = padd(run, v[k]);
    }
}

// ---------------------------------------------------------------------------
// Comb
// ---------------------------------------------------------------------------
template <class Real>
__global__ void comb_scatter_kernel(CombArgs<Real> a) {
    const long long m = (long long)*a.ncensus_ptr;
    const long long mm = m < a.cen_cap ? m : a.cen_cap;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < mm;
         j += (long long)gridDim.x * blockDim.x) {
        const uint32_t id = a.cid[j];
        const unsigned long long slot = a.goff[id] + atomicAdd(&a.gcur[id], 1u);
        a.member[slot] = (uint32_t)j;
    }
}

__device__ __forceinline__ long long first_tooth(unsigned long long C, unsigned long long W,
                                                 long long N, double u) {
    if (C == W) return N;
    const double q = ((double)N * (double)C) / (double)W - u;
    const double k = ceil(q);
    if (k < 0.0) return 0;
    if (k > (double)N) return N;
    return (long long)k;
}

template <class Real>
__global__ void comb_write_kernel(CombArgs<Real> a) {
    const long long m = (long long)*a.ncensus_ptr;
    const long long mm = m < a.cen_cap ? m : a.cen_cap;
    const unsigned long long W = a.goff_w[a.N];
    const double cscale = a.sd->cscale;
    const double u = a.sd->u_comb;
    unsigned long long coll = 0;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < mm;
         j += (long long)gridDim.x * blockDim.x) {
        const uint32_t id = a.cid[j];
        const uint32_t g = a.gcnt[id];
        unsigned long long C0 = a.goff_w[id];
        const unsigned long long wj = (unsigned long long)to_fixed(a.cw[j], cscale);
        if (g > 1) {
            const unsigned long long base = a.goff[id];
            const uint64_t lj = a.clin[j];
            for (uint32_t t = 0; t < g; ++t) {
                const uint32_t jj = a.member[base + t];
                if ((long long)jj == j) continue;
                const uint64_t lm = a.clin[jj];
                if (lm < lj || (lm == lj && (long long)jj < j)) {
                    C0 += (unsigned long long)to_fixed(a.cw[jj], cscale);
                    if (lm == lj) ++coll;
                }
            }
        }
        const long long k0 = first_tooth(C0, W, a.N, u);
        const long long k1 = first_tooth(C0 + wj, W, a.N, u);
        const Real x = a.cx[j];
        const Real mu = a.cmu[j];
        const int32_t cell = a.ccell[j];
        for (long long k = k0; k < k1; ++k) {
            a.bx[k] = x;
            a.bmu[k] = mu;
            a.bcell[k] = cell;
        }
    }
    if (coll) atomicAdd(&a.stats[ST_LINEAGE], coll);
}

__global__ void comb_finalize_kernel(StepDev* sd, const unsigned long long* goff_w,
                                     const unsigned long long* ncensus_ptr, long long N, long long cen_cap,
                                     unsigned* err) {
    const unsigned long long W = goff_w[N];
    const unsigned long long m = *ncensus_ptr;
    sd->ncensus = m;
    sd->W = W;
    if (m > (unsigned long long)cen_cap) atomicOr(err, ERR_CENSUS_OVERFLOW);
    if (W == 0) {
        sd->nbank = 0;
        sd->wbar = 0.0;
    } else {
        sd->nbank = (unsigned long long)N;
        sd->wbar = (((double)W) * pow2(-sd->Sc)) / (double)N;
    }
}

}  // namespace

void launch_prestep(const PreArgs& a, cudaStream_t s) { prestep_kernel<<<1, 256, 0, s>>>(a); }

void launch_poststep(const PostArgs& a, cudaStream_t s) {
    poststep_kernel<<<1, 256, 0, s>>>(a);
    closure_commit_kernel<<<1, 256, 0, s>>>(a);
}

void launch_group_scan(const ScanArgs& a, cudaStream_t s) {
    const long long ntiles = (a.n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles > 0) scan_tiles_kernel<<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(a);
    scan_tile_sums_kernel<<<1, SCAN_BLOCK, 0, s>>>(a, ntiles);
    if (ntiles > 0) scan_apply_kernel<<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(a);
}

long long group_scan_tiles(long long n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

template <class Real>
void launch_comb(const CombArgs<Real>& a, int grid, cudaStream_t s) {
    comb_scatter_kernel<Real><<<grid, 256, 0, s>>>(a);
    comb_write_kernel<Real><<<grid, 256, 0, s>>>(a);
    comb_finalize_kernel<<<1, 1, 0, s>>>(a.sd, a.goff_w, a.ncensus_ptr, a.N, a.cen_cap, a.err);
}

template void launch_comb<double>(const CombArgs<double>&, int, cudaStream_t);
template void launch_comb<float>(const CombArgs<float>&, int, cudaStream_t);

// standalone LOSM solve for checking the solver
__global__ void losm_only_kernel(LosmIn in, double* phi, double* J, double* w_d, double* w_m,
                                 double* w_c, double* w_r, unsigned* err) {
    if (threadIdx.x == 0) losm_solve_serial(in, phi, J, w_d, w_m, w_c, w_r, err);
}

void launch_losm_only(const LosmIn& in, double* phi, double* J, double* work, unsigned* err,
                      cudaStream_t s) {
    const int n = in.I + 2;
    losm_only_kernel<<<1, 32, 0, s>>>(in, phi, J, work, work + n, work + 2 * n, work + 3 * n, err);
}

__global__ void philox_block_kernel(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                    uint32_t k1, long long n, uint32_t* out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        uint32_t r[4] = {c0 + (uint32_t)i, c1, c2, c3};
        philox4x32_10(r, k0, k1);
        out[4 * i + 0] = r[0];
        out[4 * i + 1] = r[1];
        out[4 * i + 2] = r[2];
        out[4 * i + 3] = r[3];
    }
}

void launch_philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                         long long n, uint32_t* out, cudaStream_t s) {
    const long long blocks = (n + 255) / 256;
    philox_block_kernel<<<(unsigned)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), 256, 0, s>>>(
        c0, c1, c2, c3, k0, k1, n, out);
}

}  // namespace hww

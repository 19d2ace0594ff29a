// losm.cu -- closures, moving-average filter, HLOSM solves and window
// centers, laid out for GB300's FP64 units (few per SM, long latency):
// every FP64 stage is spread over many threads and blocks, and the only
// inherently sequential part, the tridiagonal substitution, runs as two
// chunked affine scans.
//
// The discrete LOSM equations (Eqs. losm-0, losm-1, losm-disc-bc and their
// semi-implicit form, Eqs. losm-1-semi, losm-disc-bc-semi) share one matrix:
// it depends on the cross sections, dt, v and theta only.  Eliminating J with
// the first-moment rows, J_i = m_i/d_i + g_i (phi_i - phi_{i+1}),
// g_i = theta / (3 d_i), leaves a diagonally dominant tridiagonal system in
// phi of size I+2.  Its Thomas factorization (pivots and multipliers) is
// computed once per cross-section set; a solve then needs
//   1. the right-hand side (m_i on edges, R_r on rows), pure multiply-adds;
//   2. forward substitution y_r = R_r/den_r - (A_r/den_r) y_{r-1} and back
//      substitution phi_r = y_r - c'_r phi_{r+1}, both first-order linear
//      recurrences evaluated by a chunked scan of affine maps.
// Built with contraction off.
#include "hww_internal.cuh"
#include "losm_kernels.cuh"

namespace hww {
namespace {

constexpr int SCAN_T = 256;  // threads of the substitution kernel

// ---------------------------------------------------------------------------
// setup: constant coefficients and the factorization
// ---------------------------------------------------------------------------
__global__ void losm_coef_kernel(LosmMat m, const double* dx, const double* sigt, const double* siga, double v,
                                 double dt, double theta) {
    const int I = m.I;
    const double vdt = v * dt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= I; i += gridDim.x * blockDim.x) {
        const double dxl = (i >= 1) ? dx[i - 1] : 0.0;
        const double dxr = (i <= I - 1) ? dx[i] : 0.0;
        const double stl = (i >= 1) ? sigt[i - 1] : 0.0;
        const double str = (i <= I - 1) ? sigt[i] : 0.0;
        const double dxh = 0.5 * (dxl + dxr);
        const double sth = (stl * dxl + str * dxr) / (dxl + dxr);
        const double d = dxh / vdt + theta * sth * dxh;
        m.eJ[i] = dxh / vdt;
        m.eS[i] = sth * dxh;
        m.invd[i] = 1.0 / d;
        m.g[i] = theta / (3.0 * d);
        if (i < I) {
            m.cP[i] = dx[i] / vdt;
            m.cA[i] = siga[i] * dx[i];
            m.cB[i] = dx[i] / vdt + theta * siga[i] * dx[i];
        }
    }
}

// Thomas factorization of the eliminated matrix (rows 0..I+1), run once per
// cross-section set.  The pivot recurrence den_r = B_r - A_r C_{r-1} / den_{r-1}
// is a linear-fractional map of den_{r-1}, x -> (B_r x - A_r C_{r-1}) / x, i.e.
// the 2x2 matrix [[B_r, -A_r C_{r-1}], [1, 0]] acting on x = p/q.  Each thread
// composes the maps of its chunk of rows (rescaled: only the ratio p/q
// matters), a block scan composes the chunks, and each thread then runs the
// exact recurrence over its chunk from the pivot entering it.
__device__ __forceinline__ void factor_row(const LosmMat& m, int r, double theta, int bc_l, int bc_r, double& A,
                                           double& B, double& C) {
    const int I = m.I;
    if (r == 0) {
        A = 0.0;
        C = -m.g[0];
        B = (bc_l == 1) ? m.g[0] : 0.5 + m.g[0];
    } else if (r == I + 1) {
        A = -m.g[I];
        C = 0.0;
        B = (bc_r == 1) ? m.g[I] : m.g[I] + 0.5;
    } else {
        A = -theta * m.g[r - 1];
        C = -theta * m.g[r];
        B = m.cB[r - 1] + theta * m.g[r - 1] + theta * m.g[r];
    }
}

struct Mob {
    double a, b, c, d;  // [[a, b], [c, d]]
};

// g after f (the product g f), rescaled by its largest entry
__device__ __forceinline__ Mob mob_then(Mob f, Mob g) {
    Mob h{g.a * f.a + g.b * f.c, g.a * f.b + g.b * f.d, g.c * f.a + g.d * f.c, g.c * f.b + g.d * f.d};
    const double s = fmax(fmax(fabs(h.a), fabs(h.b)), fmax(fabs(h.c), fabs(h.d)));
    if (s > 0.0 && isfinite(s)) {
        const double inv = 1.0 / s;
        h.a *= inv;
        h.b *= inv;
        h.c *= inv;
        h.d *= inv;
    }
    return h;
}

__global__ void __launch_bounds__(SCAN_T) losm_factor_kernel(LosmMat m, double theta, int bc_l, int bc_r,
                                                             unsigned* err) {
    __shared__ Mob sh[SCAN_T];
    const int n = m.I + 2;
    const int L = (n + SCAN_T - 1) / SCAN_T;
    const int r0 = threadIdx.x * L, r1 = min(n, r0 + L);
    // the chunk's composite map
    Mob f{1.0, 0.0, 0.0, 1.0};
    double A, B, C, Cprev = 0.0;
    if (r0 > 0 && r0 < n) {
        double A0, B0;
        factor_row(m, r0 - 1, theta, bc_l, bc_r, A0, B0, Cprev);
    }
    for (int r = r0; r < r1; ++r) {
        factor_row(m, r, theta, bc_l, bc_r, A, B, C);
        f = mob_then(f, Mob{B, -A * Cprev, 1.0, 0.0});
        Cprev = C;
    }
    // inclusive scan of the chunk maps (Hillis-Steele)
    sh[threadIdx.x] = f;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {
        Mob y = f;
        if ((int)threadIdx.x >= o) y = mob_then(sh[threadIdx.x - o], f);
        __syncthreads();
        sh[threadIdx.x] = y;
        f = y;
        __syncthreads();
    }
    // the pivot entering the chunk: the maps of all earlier chunks applied
    // to any start (row 0 ignores its predecessor)
    double cprev = 0.0;
    if (threadIdx.x > 0 && r0 < n) {
        const Mob e = sh[threadIdx.x - 1];
        const double p = e.a + e.b, q = e.c + e.d;
        double A0, B0, Cm;
        factor_row(m, r0 - 1, theta, bc_l, bc_r, A0, B0, Cm);
        cprev = Cm * (q / p);
    }
    for (int r = r0; r < r1; ++r) {
        factor_row(m, r, theta, bc_l, bc_r, A, B, C);
        const double den = B - A * cprev;
        if (den == 0.0 || !isfinite(den)) {
            atomicOr(err, ERR_LOSM);
            return;
        }
        const double inv = 1.0 / den;
        cprev = C * inv;
        m.inv_den[r] = inv;
        m.vf[r] = -A * inv;
        m.cp[r] = cprev;
        if (m.nA) m.nA[r] = -A;
    }
}

// ---------------------------------------------------------------------------
// right-hand side
// ---------------------------------------------------------------------------
struct RhsPtrs {
    const double *phi_old, *J_old, *F_old, *F_new, *P_new;
};

__device__ __forceinline__ RhsPtrs resolve(const LosmRhsIn& in) {
    RhsPtrs r;
    if (in.sd) {
        const int c = in.sd->cur;
        r.phi_old = in.set_phi[c];
        r.J_old = in.set_J[c];
        r.F_old = in.set_F[c];
        r.F_new = in.full ? in.set_F[1 - c] : in.set_F[c];
        r.P_new = in.full ? in.set_P[1 - c] : in.set_P[c];
    } else {
        r.phi_old = in.phi_old;
        r.J_old = in.J_old;
        r.F_old = in.F_old;
        r.F_new = in.F_new;
        r.P_new = in.P_new;
    }
    return r;
}

__device__ __forceinline__ double moment_rhs(const LosmMat& m, const RhsPtrs& in, int i) {
    const double th = m.theta, tm1 = th - 1.0;
    const double old = (in.phi_old[i + 1] - in.phi_old[i]) * (1.0 / 3.0) + m.eS[i] * in.J_old[i] -
                       in.F_old[i + 1] + in.F_old[i];
    return m.eJ[i] * in.J_old[i] + th * (in.F_new[i + 1] - in.F_new[i]) + tm1 * old;
}

__global__ void losm_rhs_kernel(LosmMat m, LosmRhsIn rin, double* u, double* mom) {
    const int I = m.I;
    const double th = m.theta, tm1 = th - 1.0;
    const RhsPtrs in = resolve(rin);
    const double PL = in.P_new ? in.P_new[0] : rin.PL;
    const double PR = in.P_new ? in.P_new[1] : rin.PR;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r <= I + 1; r += gridDim.x * blockDim.x) {
        double R;
        if (r == 0) {
            const double m0 = moment_rhs(m, in, 0);
            mom[0] = m0;
            R = (m.bc_l == 1) ? -m0 * m.invd[0] : PL - m0 * m.invd[0];
        } else if (r == I + 1) {
            const double mI = moment_rhs(m, in, I);
            R = (m.bc_r == 1) ? mI * m.invd[I] : PR + mI * m.invd[I];
        } else {
            const double ml = moment_rhs(m, in, r - 1);
            const double mr = moment_rhs(m, in, r);
            mom[r] = mr;
            const double qn = rin.q_new ? rin.q_new[r - 1] : 0.0;
            const double qo = rin.q_old ? rin.q_old[r - 1] : 0.0;
            const double oldb = in.J_old[r] - in.J_old[r - 1] + m.cA[r - 1] * in.phi_old[r] - qo;
            const double rr = m.cP[r - 1] * in.phi_old[r] + th * qn + tm1 * oldb;
            R = rr + th * ml * m.invd[r - 1] - th * mr * m.invd[r];
        }
        u[r] = R * m.inv_den[r];
    }
}

// ---------------------------------------------------------------------------
// substitution: y_r = u_r + vf_r y_{r-1} (forward), phi_r = y_r - cp_r phi_{r+1}
// (backward), by chunked scans of affine maps x -> a + b x
// ---------------------------------------------------------------------------
struct Aff {
    double a, b;
};

// compose: apply f first, then g
__device__ __forceinline__ Aff compose(Aff f, Aff g) { return Aff{g.a + g.b * f.a, g.b * f.b}; }

// inclusive scan of one affine map per thread (Hillis-Steele in shared memory)
__device__ Aff block_scan_aff(Aff x, Aff* sh) {
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {
        Aff y = x;
        if ((int)threadIdx.x >= o) y = compose(sh[threadIdx.x - o], x);
        __syncthreads();
        sh[threadIdx.x] = y;
        x = y;
        __syncthreads();
    }
    return x;
}

__global__ void __launch_bounds__(SCAN_T) losm_scan_kernel(LosmMat m, const double* u, const double* mom,
                                                           double* y, double* phi, double* J, double* red_max,
                                                           int want_max) {
    __shared__ Aff sh[SCAN_T];
    __shared__ double smax[SCAN_T];
    const int n = m.I + 2;
    const int L = (n + SCAN_T - 1) / SCAN_T;
    const int r0 = threadIdx.x * L;
    const int r1 = min(n, r0 + L);
    // forward: y_r = u_r + vf_r y_{r-1}
    Aff f{0.0, 1.0};
    for (int r = r0; r < r1; ++r) f = compose(f, Aff{u[r], m.vf[r]});
    Aff inc = block_scan_aff(f, sh);
    Aff exc = (threadIdx.x > 0) ? sh[threadIdx.x - 1] : Aff{0.0, 1.0};
    (void)inc;
    double yy = exc.a;  // y_{r0-1} with y_{-1} = 0
    for (int r = r0; r < r1; ++r) {
        yy = u[r] + m.vf[r] * yy;
        y[r] = yy;
    }
    __syncthreads();
    // backward over the reversed order: phi_r = y_r - cp_r phi_{r+1}; thread t
    // takes the chunk of reversed position t
    const int q0 = threadIdx.x * L;
    const int q1 = min(n, q0 + L);
    Aff g{0.0, 1.0};
    for (int q = q0; q < q1; ++q) {
        const int r = n - 1 - q;
        g = compose(g, Aff{y[r], -m.cp[r]});
    }
    block_scan_aff(g, sh);
    Aff gexc = (threadIdx.x > 0) ? sh[threadIdx.x - 1] : Aff{0.0, 1.0};
    double pp = gexc.a;  // phi_{r+1} of the first row of this chunk, phi_{n} = 0
    for (int q = q0; q < q1; ++q) {
        const int r = n - 1 - q;
        pp = y[r] - m.cp[r] * pp;
        phi[r] = pp;
    }
    __syncthreads();
    // J on edges and the maximum of the clamped cell flux
    double mx = 0.0;
    for (int i = threadIdx.x; i <= m.I; i += SCAN_T) {
        J[i] = mom[i] * m.invd[i] + m.g[i] * (phi[i] - phi[i + 1]);
        if (i >= 1) mx = fmax(mx, phi[i] > 0.0 ? phi[i] : 0.0);
    }
    if (want_max) {
        smax[threadIdx.x] = mx;
        __syncthreads();
        for (int s = SCAN_T / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
            __syncthreads();
        }
        if (threadIdx.x == 0) *red_max = smax[0];
    }
}

// ---------------------------------------------------------------------------
// window centers, Eq. (ww-center) with the clamp at 0 and Eq. (ww-c&f).
// Centers are rounded to 20 significant bits (half up on the bit pattern):
// the window only needs the center to within a factor rho, and the rounding
// keeps the windows independent of last-bit differences between equivalent
// LOSM solvers (a roulette survivor takes the center as its weight).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double quantize_center(double c) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(c);
    return __longlong_as_double((long long)((b + (1ull << 31)) & ~((1ull << 32) - 1ull)));
}

__global__ void ww_centers_kernel(WwArgs a) {
    const int source = a.sd->ww_src;
    if (source == 0) return;
    const double mx = (source == 2) ? *a.mx_prev : *a.mx_hlosm;
    const double* phit = (source == 2) ? a.phit_prev : a.phit_hlosm;
    const double scale = (a.scaling == 0) ? a.sd->wbar : 1.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.I; i += gridDim.x * blockDim.x) {
        double ctr;
        if (source == 3) {
            ctr = a.override_c[i];
        } else {
            const double f = phit[i] > 0.0 ? phit[i] : 0.0;
            const double ratio = (mx > 0.0) ? f / mx : 1.0;
            const double b = ratio * (1.0 - a.eps) + a.eps;
            ctr = scale * b;
        }
        ctr = quantize_center(ctr);
        const double hi = ctr * a.rho, lo = ctr / a.rho;
        a.ww_c[i] = ctr;
        a.ww_hi[i] = hi;
        a.ww_lo[i] = lo;
        a.ww_hl[i] = make_double2(hi, lo);
    }
}

// maximum of a clamped cell vector (lagged windows take the previous step's
// track-length flux)
__global__ void vec_max_kernel(const double* x, int n, double* out) {
    __shared__ double s[256];
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, x[i] > 0.0 ? x[i] : 0.0);
    s[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// step scalars: Philox key, tally and comb fixed-point scales, comb offset,
// birth flag and the window source of the step
__global__ void step_scalars_kernel(StepDev* sd, int nbits, unsigned long long seed, int mode,
                                    unsigned long long* stats) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long n = sd->step + 1;
    sd->k0 = (uint32_t)seed;
    sd->k1 = (uint32_t)(seed >> 32) ^ (uint32_t)n;
    int E = 0;
    if (sd->wbar > 0.0) {
        int e;
        frexp(sd->wbar, &e);
        E = e - 1;
    }
    sd->S = 40 - E;
    sd->Sc = 59 - E - nbits;
    sd->tscale = pow2(sd->S);
    sd->cscale = pow2(sd->Sc);
    sd->Wbar = to_fixed(sd->wbar, sd->tscale);
    uint32_t r[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xC0B0u};
    philox4x32_10(r, sd->k0, sd->k1);
    sd->U_comb = r[1];
    sd->birth = (sd->step == 0 && !sd->bank_loaded) ? 1 : 0;
    const int src = sd->override_c ? 3 : (mode == 0) ? 1 : (mode == 2 && sd->has_prev) ? 2 : 0;
    sd->ww_src = src;
    sd->ww_on = src != 0;
    stats[ST_NSTART] = sd->nbank;
}

// ---------------------------------------------------------------------------
// closures from the census tallies (Eq. ct-mc), then the filter
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cen_val(const ClosureArgs& a, int q, int i, double isc) {
    return (a.v * (acc_to_double(a.cent[q * a.I + i]) * isc)) / ((double)a.N * a.dx[i]);
}

// offsets of closure set blockIdx.y (see ClosureArgs)
__device__ __forceinline__ ClosureArgs closure_set(const ClosureArgs& in) {
    ClosureArgs a = in;
    const long long y = blockIdx.y, I = a.I;
    if (y == 0) return a;
    a.cent += y * 3 * I;
    a.bnd += y * 6;
    a.rphi += y * (I + 1);
    a.rJ += y * (I + 1);
    a.rF += y * (I + 1);
    for (int k = 0; k < 2; ++k) {
        a.set_phi[k] += y * (I + 2);
        a.set_J[k] += y * (I + 1);
        a.set_F[k] += y * (I + 2);
        a.set_P[k] += y * 2;
    }
    return a;
}

__global__ void closure_kernel(ClosureArgs a_in) {
    const ClosureArgs a = closure_set(a_in);
    const int I = a.I;
    double* nP = a.set_P[1 - a.sd->cur];
    const double isc = pow2(-a.sd->S);
    const double PL = (a.bc_l == 1) ? 0.0 : (acc_to_double(a.bnd[2]) * isc) / ((double)a.N * a.dt);
    const double PR = (a.bc_r == 1) ? 0.0 : (acc_to_double(a.bnd[5]) * isc) / ((double)a.N * a.dt);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= I; i += gridDim.x * blockDim.x) {
        if (i < I) {
            a.rphi[i] = cen_val(a, 0, i, isc);
            a.rF[i] = cen_val(a, 2, i, isc);
            if (a.tl) a.prev_tl[i] = (acc_to_double(a.tl[i]) * isc) / (((double)a.N * a.dx[i]) * a.dt);
        }
        double J;
        if (i == 0) {
            J = (a.bc_l == 1) ? 0.0 : (-0.5 * cen_val(a, 0, 0, isc) + PL);
        } else if (i == I) {
            J = (a.bc_r == 1) ? 0.0 : (0.5 * cen_val(a, 0, I - 1, isc) - PR);
        } else {
            const double dl = a.dx[i - 1], dr = a.dx[i];
            J = (cen_val(a, 1, i - 1, isc) * dr + cen_val(a, 1, i, isc) * dl) / (dl + dr);
        }
        a.rJ[i] = J;
        if (i == 0) {
            nP[0] = PL;
            nP[1] = PR;
        }
    }
}

// moving average with the symmetric shrink at the ends (k = 0: copy); the
// window sum runs from its right end to its left end
__device__ __forceinline__ double ma_at(const double* in, int m, int j, int k) {
    int kk = k;
    if (j - 1 < kk) kk = j - 1;
    if (m - j < kk) kk = m - j;
    double s = 0.0;
    for (int l = -kk; l <= kk; ++l) s = s + in[j - l - 1];
    return s / (double)(2 * kk + 1);
}

__global__ void filter_kernel(ClosureArgs a_in) {
    const ClosureArgs a = closure_set(a_in);
    const int I = a.I, k = a.filter_k;
    const int c1 = 1 - a.sd->cur;
    double* nphi = a.set_phi[c1];
    double* nJ = a.set_J[c1];
    double* nF = a.set_F[c1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= I + 1; i += gridDim.x * blockDim.x) {
        if (i >= 1 && i <= I) {
            nphi[i] = k ? ma_at(a.rphi, I, i, k) : a.rphi[i - 1];
            nF[i] = k ? ma_at(a.rF, I, i, k) : a.rF[i - 1];
        }
        if (i <= I) nJ[i] = k ? ma_at(a.rJ, I + 1, i + 1, k) : a.rJ[i];
        if (i == 0) {
            // end values are kept by the filter, so the boundary copies use them
            nphi[0] = a.rphi[0];
            nF[0] = a.rF[0];
        }
        if (i == I + 1) {
            nphi[I + 1] = a.rphi[I - 1];
            nF[I + 1] = a.rF[I - 1];
        }
    }
}

// ---------------------------------------------------------------------------
// adjoint of the fully implicit solve (differentiation; not in the paper)
//
// lambda = A^{-T} g for the interleaved system A u = b, u = (phi_0, J_0,
// phi_1, ..., J_I, phi_{I+1}).  Eliminating the J-rows of A^T (one per edge,
// diagonal d_i) leaves, for the multipliers psi of the phi-rows, the
// transpose M^T of the eliminated matrix M = L U that the forward solve
// factorized (with the sign of the last row's multiplier flipped, because
// the forward solve negates that row):
//   M^T psi' = h,  h_r = g_phi,r - g_{r-1} g_J,r-1 + g_r g_J,r,
//   psi_r = psi'_r (r <= I), psi_{I+1} = -psi'_{I+1},
//   chi_i = (g_J,i - alpha_i psi_i - beta_i psi_{i+1}) / d_i,
// alpha_0 = 1 (the left boundary row), alpha_i = theta; beta_I = 1 (the right
// boundary row), beta_i = -theta.  M^T = U^T L^T turns into two first-order
// recurrences, evaluated by the same chunked affine scans as the forward
// solve:  z_r = h_r - c'_{r-1} z_{r-1},  psi'_r = (z_r + (-A_{r+1}) psi'_{r+1}) / den_r.
// The parameter gradients contract lambda with the right-hand side of the
// step's derivative data (old closures, new F and boundary closures) and with
// the explicit dependence of A and b on Sigma_t (through Sigma_hat at the
// edges) and on Sigma_a = Sigma_t (1 - c) (balance rows).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double vjp_block_sum(double x, double* sh) {
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = SCAN_T / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_T) losm_vjp_kernel(VjpArgs a) {
    __shared__ Aff sh[SCAN_T];
    __shared__ double sred[SCAN_T];
    const LosmMat& m = a.m;
    const int I = m.I, n = I + 2;
    const double th = m.theta, tm1 = th - 1.0;
    const VjpLayout L = vjp_layout(I, a.P2);
    const double* st = a.state;
    // h
    for (int r = threadIdx.x; r < n; r += SCAN_T) {
        double h = a.g_phi[r];
        if (r >= 1) h = h - m.g[r - 1] * a.g_J[r - 1];
        if (r <= I) h = h + m.g[r] * a.g_J[r];
        a.z[r] = h;
    }
    __syncthreads();
    const int Lc = (n + SCAN_T - 1) / SCAN_T;
    // forward: z_r = h_r - cp_{r-1} z_{r-1}
    {
        const int r0 = threadIdx.x * Lc, r1 = min(n, r0 + Lc);
        Aff f{0.0, 1.0};
        for (int r = r0; r < r1; ++r) f = compose(f, Aff{a.z[r], r ? -m.cp[r - 1] : 0.0});
        block_scan_aff(f, sh);
        const Aff exc = (threadIdx.x > 0) ? sh[threadIdx.x - 1] : Aff{0.0, 1.0};
        double zz = exc.a;
        for (int r = r0; r < r1; ++r) {
            zz = a.z[r] + (r ? -m.cp[r - 1] : 0.0) * zz;
            a.z[r] = zz;
        }
    }
    __syncthreads();
    // backward: psi'_r = inv_den_r z_r + inv_den_r (-A_{r+1}) psi'_{r+1}
    {
        const int q0 = threadIdx.x * Lc, q1 = min(n, q0 + Lc);
        Aff g{0.0, 1.0};
        for (int q = q0; q < q1; ++q) {
            const int r = n - 1 - q;
            const double nb = (r + 1 < n) ? m.inv_den[r] * m.nA[r + 1] : 0.0;
            g = compose(g, Aff{m.inv_den[r] * a.z[r], nb});
        }
        block_scan_aff(g, sh);
        const Aff gexc = (threadIdx.x > 0) ? sh[threadIdx.x - 1] : Aff{0.0, 1.0};
        double pp = gexc.a;
        for (int q = q0; q < q1; ++q) {
            const int r = n - 1 - q;
            const double nb = (r + 1 < n) ? m.inv_den[r] * m.nA[r + 1] : 0.0;
            pp = m.inv_den[r] * a.z[r] + nb * pp;
            a.psi[r] = (r == n - 1) ? -pp : pp;
        }
    }
    __syncthreads();
    // contractions, one parameter at a time
    const double* phi_old = st + L.phi_old;
    const double* J_old = st + L.J_old;
    const double* phi_new = st + L.phi_new;
    const double* J_new = st + L.J_new;
    for (int j = 0; j < a.P2; ++j) {
        const bool is_sigma = j < a.R;
        const int gr = is_sigma ? j : j - a.R;
        RhsPtrs d;
        d.phi_old = st + L.dphi_old + (long long)j * (I + 2);
        d.J_old = st + L.dJ_old + (long long)j * (I + 1);
        d.F_old = st + L.dF_old + (long long)j * (I + 2);
        d.F_new = st + L.dF_new + (long long)j * (I + 2);
        const double dPL = st[L.dP_new + 2 * j], dPR = st[L.dP_new + 2 * j + 1];
        double acc = 0.0;
        // first-moment rows (lambda_{2i+1} = chi_i)
        for (int i = threadIdx.x; i <= I; i += SCAN_T) {
            const double al = (i == 0) ? 1.0 : th;
            const double be = (i == I) ? 1.0 : -th;
            const double chi = (a.g_J[i] - al * a.psi[i] - be * a.psi[i + 1]) * m.invd[i];
            double rhs = moment_rhs(m, d, i);
            const double dxl = (i >= 1) ? a.dx[i - 1] : 0.0;
            const double dxr = (i <= I - 1) ? a.dx[i] : 0.0;
            const double dsl = (is_sigma && i >= 1 && a.region[i - 1] == gr) ? 1.0 : 0.0;
            const double dsr = (is_sigma && i <= I - 1 && a.region[i] == gr) ? 1.0 : 0.0;
            const double dES = 0.5 * (dsl * dxl + dsr * dxr);  // d(Sigma_hat dxhat)
            rhs = rhs + tm1 * dES * J_old[i] - th * dES * J_new[i];
            acc = acc + chi * rhs;
        }
        // balance rows (lambda_{2r} = psi_r), r = 1..I
        for (int r = threadIdx.x + 1; r <= I; r += SCAN_T) {
            const double oldb = d.J_old[r] - d.J_old[r - 1] + m.cA[r - 1] * d.phi_old[r];
            double rhs = m.cP[r - 1] * d.phi_old[r] + tm1 * oldb;
            if (a.region[r - 1] == gr) {
                const double dsa = is_sigma ? 1.0 - a.c[r - 1] : -a.sigt[r - 1];
                const double dxi = a.dx[r - 1];
                rhs = rhs + tm1 * dsa * dxi * phi_old[r] - th * dsa * dxi * phi_new[r];
            }
            acc = acc + a.psi[r] * rhs;
        }
        // boundary rows (natural form: P_L on the left, -P_R on the right)
        if (threadIdx.x == 0) {
            if (m.bc_l != 1) acc = acc + a.psi[0] * dPL;
            if (m.bc_r != 1) acc = acc - a.psi[I + 1] * dPR;
        }
        // Monte Carlo flux part
        if (a.g_mc) {
            const double* dtl = st + L.dtl + (long long)j * I;
            for (int i = threadIdx.x; i < I; i += SCAN_T) acc = acc + dtl[i] * a.g_mc[i];
        }
        const double tot = vjp_block_sum(acc, sred);
        if (threadIdx.x == 0) a.grad[j] = tot;
    }
}

// Fourier low-pass (Eqs. fft, ifft and the cutoff): the modes of frequency
// f <= kappa of a real vector x of length M, X_f = sum_m x_m e^{-2 pi i f m / M},
// give the filtered x~_m = (X_0 + 2 sum_{0<f<M/2} Re(X_f e^{2 pi i f m / M})
// [+ X_{M/2} e^{i pi m} when kappa reaches M/2]) / M.  Angles are reduced
// exactly: sincospi(2 ((f m) mod M) / M).  One block per vector (blockIdx.x:
// 0 phi on cells, 1 F on cells, 2 J on edges) and closure set (blockIdx.y);
// the block writes the filtered vector and, for phi and F, the ghost values.
__global__ void fourier_filter_kernel(ClosureArgs a_in) {
    extern __shared__ double fsh[];  // x (M), then Xr, Xi (kappa' + 1 each)
    const ClosureArgs a = closure_set(a_in);
    const int I = a.I;
    const int c1 = 1 - a.sd->cur;
    const int which = blockIdx.x;
    const int M = (which == 2) ? I + 1 : I;
    const double* in = (which == 0) ? a.rphi : (which == 1) ? a.rF : a.rJ;
    double* out = (which == 0) ? a.set_phi[c1] + 1 : (which == 1) ? a.set_F[c1] + 1 : a.set_J[c1];
    const int kp = min(a.kappa, M / 2);
    double* x = fsh;
    double* Xr = fsh + M;
    double* Xi = Xr + (kp + 1);
    for (int m = threadIdx.x; m < M; m += blockDim.x) x[m] = in[m];
    __syncthreads();
    for (int f = threadIdx.x; f <= kp; f += blockDim.x) {
        double re = 0.0, im = 0.0;
        long long fm = 0;  // (f m) mod M
        for (int m = 0; m < M; ++m) {
            double sn, cs;
            sincospi(2.0 * (double)fm / (double)M, &sn, &cs);
            re = re + x[m] * cs;
            im = im - x[m] * sn;
            fm += f;
            if (fm >= M) fm -= M;
        }
        Xr[f] = re;
        Xi[f] = im;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        double acc = Xr[0];
        for (int f = 1; f <= kp; ++f) {
            const long long fm = ((long long)f * m) % M;
            double sn, cs;
            sincospi(2.0 * (double)fm / (double)M, &sn, &cs);
            const double t = Xr[f] * cs - Xi[f] * sn;
            acc = acc + ((2 * f == M) ? t : 2.0 * t);
        }
        out[m] = acc / (double)M;
    }
    if (which < 2) {
        __syncthreads();
        if (threadIdx.x == 0) {
            out[-1] = out[0];     // ghost values copy the filtered end cells
            out[M] = out[M - 1];
        }
    }
}

int small_grid(int n) {
    const int b = (n + 127) / 128;
    return b < 1 ? 1 : (b > 64 ? 64 : b);
}

}  // namespace

void launch_losm_setup(const LosmMat& m, const double* dx, const double* sigt, const double* siga, double v,
                       double dt, double theta, int bc_l, int bc_r, unsigned* err, cudaStream_t s) {
    losm_coef_kernel<<<small_grid(m.I + 1), 128, 0, s>>>(m, dx, sigt, siga, v, dt, theta);
    losm_factor_kernel<<<1, SCAN_T, 0, s>>>(m, theta, bc_l, bc_r, err);
}

int launch_losm_solve(const LosmMat& m, const LosmRhsIn& in, const LosmWork& w, double* phi, double* J,
                      double* mx, cudaStream_t s) {
    losm_rhs_kernel<<<small_grid(m.I + 2), 128, 0, s>>>(m, in, w.u, w.mom);
    losm_scan_kernel<<<1, SCAN_T, 0, s>>>(m, w.u, w.mom, w.y, phi, J, mx, mx != nullptr);
    return 2;
}

int launch_ww_centers(const WwArgs& a, int lagged, cudaStream_t s) {
    int n = 0;
    if (lagged) {
        vec_max_kernel<<<1, 256, 0, s>>>(a.phit_prev, a.I, (double*)a.mx_prev);
        ++n;
    }
    ww_centers_kernel<<<small_grid(a.I), 128, 0, s>>>(a);
    return n + 1;
}

void launch_step_scalars(StepDev* sd, int nbits, unsigned long long seed, int mode, unsigned long long* stats,
                         cudaStream_t s) {
    step_scalars_kernel<<<1, 32, 0, s>>>(sd, nbits, seed, mode, stats);
}

int launch_closures(const ClosureArgs& a, cudaStream_t s) {
    const unsigned ny = a.nsets > 1 ? (unsigned)a.nsets : 1u;
    closure_kernel<<<dim3(small_grid(a.I + 1), ny), 128, 0, s>>>(a);
    if (a.fourier) {
        const int kp = a.kappa < (a.I + 1) / 2 ? a.kappa : (a.I + 1) / 2;
        const size_t smem = sizeof(double) * ((size_t)a.I + 1 + 2 * ((size_t)kp + 1));
        fourier_filter_kernel<<<dim3(3, ny), 256, smem, s>>>(a);
    } else {
        filter_kernel<<<dim3(small_grid(a.I + 2), ny), 128, 0, s>>>(a);
    }
    return 2;
}

int fourier_filter_smem_optin(size_t smem) {
    return (int)cudaFuncSetAttribute(fourier_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int launch_losm_vjp(const VjpArgs& a, cudaStream_t s) {
    losm_vjp_kernel<<<1, SCAN_T, 0, s>>>(a);
    return 1;
}

cudaError_t losm_solve_staged(double* base, int I, const double* dx, const double* sigma_t, const double* sigma_a,
                              double v, double dt, double theta, int bc_left, int bc_right, const double* phi_old,
                              const double* J_old, const double* F_old, const double* F_new, double PL_new,
                              double PR_new, const double* q_old, const double* q_new, double* phi_new,
                              double* J_new, bool* numeric) {
    *numeric = false;
    double* q = base;
    auto take = [&](size_t k) {
        double* r = q;
        q += k;
        return r;
    };
    const size_t n2 = (size_t)I + 2, n1 = (size_t)I + 1;
    double* d_dx = take(I);
    double* d_st = take(I);
    double* d_sa = take(I);
    double* d_qo = take(I);
    double* d_qn = take(I);
    double* d_po = take(n2);
    double* d_Fo = take(n2);
    double* d_Fn = take(n2);
    double* d_pn = take(n2);
    double* d_Jo = take(n1);
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
    // the block may hold an earlier call's contents: the error word starts at 0
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
    // the carving above must stay within the block the callers size
    if (e == cudaSuccess && (size_t)(q - base) != losm_staged_doubles(I)) e = cudaErrorInvalidValue;
    *numeric = herr != 0;
    return e;
}

}  // namespace hww

// track_fp32.cu -- FP32-tracking variant of the event loop.
//
// Same events, rules and random streams as the FP64 kernel (the uniforms are
// the top 23 bits of the same Philox words), but the geometry runs in FP32:
// a track keeps its cell index and an FP32 offset from the cell's left edge,
// an FP32 direction, an FP32 distance to census and FP32 flight distances.
// Weights, the window tests, every tally contribution and all downstream
// steps (closures, filter, LOSM solves, comb) stay in FP64, the steps whose
// accuracy the estimators rest on.
#include "track_common.cuh"

namespace hww {
namespace {

struct P32 {
    float xo, mu, inv_mu, tau;
    double w;
    int cell;
    uint32_t id;
    uint64_t lin;
    uint32_t e;
};

__device__ __forceinline__ void push_record(const TrackArgs<float>& a, const P32& q, double w,
                                            uint32_t e, uint32_t jstart, uint32_t jcount,
                                            unsigned long long slot) {
    if ((long long)slot >= a.rout.cap) {
        atomicOr(a.err, ERR_QUEUE_OVERFLOW);
        return;
    }
    a.rout.x[slot] = q.xo;
    a.rout.mu[slot] = q.mu;
    a.rout.tau[slot] = q.tau;
    a.rout.w[slot] = w;
    a.rout.cell[slot] = q.cell;
    a.rout.id[slot] = q.id;
    a.rout.lin[slot] = q.lin;
    a.rout.e[slot] = e;
    a.rout.jstart[slot] = jstart;
    a.rout.jcount[slot] = jcount;
}

__device__ void run_track(const TrackArgs<float>& a, P32 q, long long* s_tl, long long* s_cen,
                          Counters& cnt, double tscale, double cscale) {
    const int I = a.I;
    int evs = 0;
    for (;;) {
        if (evs == a.emax) {
            push_record(a, q, q.w, q.e, 0u, 0u, atomicAdd(a.rout.count, 1ull));
            return;
        }
        if (q.e >= MAX_EVENTS) {
            atomicOr(a.err, ERR_EVENTS);
            return;
        }
        uint32_t r[4] = {q.id, (uint32_t)q.lin, (uint32_t)(q.lin >> 32), 2u * q.e};
        philox4x32_10(r, a.k0, a.k1);
        const float uf = u01f(r[1]);
        const float uc = u01f(r[3]);
        const int k = q.cell;
        const float dxk = a.dxf[k];
        const float dcoll = -logf(uf) * a.inv_sigt_f[k];
        const float dedge = ((q.mu > 0.0f) ? (dxk - q.xo) : -q.xo) * q.inv_mu;
        const float dcens = q.tau;
        int ev;
        float l;
        if (dcens <= dedge && dcens <= dcoll) {
            ev = 0;
            l = dcens;
        } else if (dedge <= dcoll) {
            ev = 1;
            l = dedge;
        } else {
            ev = 2;
            l = dcoll;
        }
        const double wl = q.w * (double)l;
        const long long fphi = to_fixed(wl, tscale);
        sadd(&s_tl[k], fphi);
        sadd(&s_tl[I + k], to_fixed(wl * (double)q.mu, tscale));
        sadd(&s_tl[2 * I + k], to_fixed(wl * (double)(1.0f / 3.0f - q.mu * q.mu), tscale));
        add128(&a.batch[(long long)(q.id % (uint32_t)a.B) * I + k], fphi);
        cnt.v[ST_SEGMENTS]++;
        if (ev != 1) {
            float xn = fmaf(q.mu, l, q.xo);
            xn = fminf(fmaxf(xn, 0.0f), dxk);
            q.xo = xn;
        }
        q.tau = (ev == 0) ? 0.0f : q.tau - l;
        const uint32_t e_ev = q.e;
        q.e = q.e + 1;
        ++evs;
        if (ev == 0) {
            const double wmu = q.w * (double)q.mu;
            const double wf = q.w * (double)(1.0f / 3.0f - q.mu * q.mu);
            sadd(&s_cen[k], to_fixed(q.w, tscale));
            sadd(&s_cen[I + k], to_fixed(wmu, tscale));
            sadd(&s_cen[2 * I + k], to_fixed(wf, tscale));
            const unsigned long long slot = warp_reserve(a.cen.count);
            if ((long long)slot < a.cen.cap) {
                a.cen.x[slot] = q.xo;
                a.cen.mu[slot] = q.mu;
                a.cen.w[slot] = q.w;
                a.cen.cell[slot] = q.cell;
                a.cen.id[slot] = q.id;
                a.cen.lin[slot] = q.lin;
                atomicAdd(&a.gcnt[q.id], 1u);
                atomicAdd(&a.gw[q.id], (unsigned long long)to_fixed(q.w, cscale));
            } else {
                atomicOr(a.err, ERR_CENSUS_OVERFLOW);
            }
            cnt.v[ST_CENSUS]++;
            cnt.v[ST_MAX_EVENTS] = max(cnt.v[ST_MAX_EVENTS], q.e);
            return;
        }
        bool have_r2 = false;
        uint32_t r2[4];
        if (ev == 1) {
            cnt.v[ST_CROSSINGS]++;
            const int nk = (q.mu > 0.0f) ? k + 1 : k - 1;
            if (nk < 0 || nk >= I) {
                const int side = (nk < 0) ? 0 : 1;
                const int bc = side ? a.bc_r : a.bc_l;
                if (bc == 0) {
                    const double amu = fabs((double)q.mu);
                    const double ia = (amu < GRAZE_MU) ? 2.0 / GRAZE_MU : 1.0 / amu;
                    const double wi = q.w * ia;
                    const double m2 = (double)q.mu * (double)q.mu;
                    add128(&a.bnd[3 * side + 0], to_fixed(wi, tscale));
                    add128(&a.bnd[3 * side + 1], to_fixed(wi * (1.0 / 3.0 - m2), tscale));
                    add128(&a.bnd[3 * side + 2], to_fixed(wi * (0.5 - amu), tscale));
                    cnt.v[ST_LEAKED]++;
                    cnt.v[ST_MAX_EVENTS] = max(cnt.v[ST_MAX_EVENTS], q.e);
                    return;
                }
                q.mu = -q.mu;
                q.inv_mu = -q.inv_mu;
                q.xo = side ? dxk : 0.0f;
                cnt.v[ST_REFLECTIONS]++;
            } else {
                q.cell = nk;
                q.xo = (q.mu > 0.0f) ? 0.0f : a.dxf[nk];
            }
        } else {
            cnt.v[ST_COLLISIONS]++;
            if ((double)uc >= a.c[k]) {
                cnt.v[ST_ABSORBED]++;
                cnt.v[ST_MAX_EVENTS] = max(cnt.v[ST_MAX_EVENTS], q.e);
                return;
            }
            r2[0] = q.id;
            r2[1] = (uint32_t)q.lin;
            r2[2] = (uint32_t)(q.lin >> 32);
            r2[3] = 2u * e_ev + 1u;
            philox4x32_10(r2, a.k0, a.k1);
            have_r2 = true;
            q.mu = 2.0f * u01f(r2[1]) - 1.0f;
            q.inv_mu = 1.0f / q.mu;
            cnt.v[ST_SCATTERS]++;
        }
        if (a.ww_on) {
            const int kc = q.cell;
            const double hi = a.ww_hi[kc];
            const double lo = a.ww_lo[kc];
            if (q.w > hi) {
                const double ctr = a.ww_c[kc];
                const double ndd = ceil(q.w / ctr);
                if (ndd > (double)MAX_DAUGHTERS) {
                    atomicOr(a.err, ERR_DAUGHTERS);
                    return;
                }
                const uint32_t nd = (uint32_t)ndd;
                const double wd = q.w / (double)nd;
                cnt.v[ST_SPLIT_EVENTS]++;
                cnt.v[ST_DAUGHTERS] += nd - 1;
                const uint32_t nch = (nd - 1 + SPLIT_CHUNK - 1) / SPLIT_CHUNK;
                const unsigned long long base = atomicAdd(a.rout.count, (unsigned long long)nch);
                for (uint32_t ch = 0; ch < nch; ++ch) {
                    const uint32_t j0 = 1 + ch * SPLIT_CHUNK;
                    const uint32_t jc = min((uint32_t)SPLIT_CHUNK, nd - j0);
                    push_record(a, q, wd, e_ev, j0, jc, base + ch);
                }
                q.w = wd;
                q.lin = lineage_hash(q.lin, e_ev, 0);
                q.e = 0;
            } else if (q.w < lo) {
                if (!have_r2) {
                    r2[0] = q.id;
                    r2[1] = (uint32_t)q.lin;
                    r2[2] = (uint32_t)(q.lin >> 32);
                    r2[3] = 2u * e_ev + 1u;
                    philox4x32_10(r2, a.k0, a.k1);
                }
                const double ctr = a.ww_c[kc];
                const double ur = u01(r2[2], r2[3]);
                const double ps = q.w / ctr;
                if (ur < ps) {
                    q.w = ctr;
                    cnt.v[ST_RSURVIVE]++;
                } else {
                    cnt.v[ST_RKILLS]++;
                    cnt.v[ST_MAX_EVENTS] = max(cnt.v[ST_MAX_EVENTS], q.e);
                    return;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) track32_kernel(TrackArgs<float> a) {
    extern __shared__ long long sm[];
    const int I = a.I;
    long long* s_tl = sm;
    long long* s_cen = sm + 3 * I;
    for (int i = threadIdx.x; i < 6 * I; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    Counters cnt;
    cnt.zero();
    const double tscale = a.sd->tscale;
    const double cscale = a.sd->cscale;
    const double wbar = a.sd->wbar;
    const float tau0 = (float)a.tau0;
    const long long n_in = a.from_bank ? (long long)a.sd->nbank : (long long)*a.rin.count;
    const long long n_use = (!a.from_bank && n_in > a.rin.cap) ? a.rin.cap : n_in;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_use; i += stride) {
        P32 p;
        uint32_t jstart = 0, jcount = 0;
        if (a.from_bank) {
            p.id = (uint32_t)i;
            p.lin = 0;
            p.e = 0;
            p.tau = tau0;
            p.w = wbar;
            if (a.birth) {
                uint32_t r[4] = {(uint32_t)i, 0u, 0u, 0xFFFFFFFFu};
                philox4x32_10(r, a.k0, a.k1);
                p.mu = 2.0f * u01f(r[1]) - 1.0f;
                const double x = a.src_x;
                if (x <= a.edges[0] && p.mu < 0.0f && a.bc_l == 1) p.mu = -p.mu;
                if (x >= a.edges[I] && p.mu > 0.0f && a.bc_r == 1) p.mu = -p.mu;
                p.cell = (p.mu < 0.0f) ? a.birth_cell_neg : a.birth_cell_pos;
                p.xo = (float)(x - a.edges[p.cell]);
            } else {
                p.xo = a.bx[i];
                p.mu = a.bmu[i];
                p.cell = a.bcell[i];
            }
        } else {
            p.xo = a.rin.x[i];
            p.mu = a.rin.mu[i];
            p.tau = a.rin.tau[i];
            p.w = a.rin.w[i];
            p.cell = a.rin.cell[i];
            p.id = a.rin.id[i];
            p.lin = a.rin.lin[i];
            p.e = a.rin.e[i];
            jstart = a.rin.jstart[i];
            jcount = a.rin.jcount[i];
        }
        const uint32_t ntracks = jcount ? jcount : 1u;
        for (uint32_t t = 0; t < ntracks; ++t) {
            P32 q = p;
            if (jcount) {
                q.lin = lineage_hash(p.lin, p.e, jstart + t);
                q.e = 0;
            }
            q.inv_mu = 1.0f / q.mu;
            run_track(a, q, s_tl, s_cen, cnt, tscale, cscale);
        }
    }
    __syncthreads();
    flush_tallies(sm, I, a.tl, a.cent);
    flush_counters(cnt, a.stats);
}

}  // namespace

void launch_track_fp32(const TrackArgs<float>& a, int grid, int block, size_t smem, cudaStream_t s) {
    track32_kernel<<<grid, block, smem, s>>>(a);
}

int track_smem_optin_fp32(size_t smem) {
    return (int)cudaFuncSetAttribute(track32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
}

int track_blocks_per_sm_fp32(int block, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, track32_kernel, block, smem);
    return n;
}

}  // namespace hww

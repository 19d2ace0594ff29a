// api.cu -- the C ABI (include/hww.h) and the host-side step orchestration.
//
// A time step is a fixed sequence of stream-ordered launches:
//   clear accumulators -> prestep (semi-implicit HLOSM, windows) ->
//   tracking wave 0 over the start bank -> tracking waves over the record
//   queue until it is empty -> poststep (closures, fully implicit HLOSM) ->
//   comb (group scan, member scatter, tooth writes, next-step scalars).
// Only the queue-empty test between waves reads a device counter back.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <climits>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/hww.h"
#include "hww_internal.cuh"
#include "losm_kernels.cuh"
#include "step_kernels.cuh"

using namespace hww;

namespace {

constexpr int TRACK_BLOCK = TRACK_THREADS;
constexpr int MAX_CELLS = 4000;
constexpr int MAX_WAVES = 100000;
constexpr int MAX_REGROW = 12;

template <class Real>
struct Banks {
    BankRec<Real>* bank = nullptr;  // start bank
    RecQ<Real> q[2] = {};
    CenQ<Real> cen = {};
};

}  // namespace

struct hww_problem {
    hww_problem_desc d{};
    int I = 0, B = 0;
    long long N = 0;
    int fp32 = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int nsm = 0;
    long long cen_cap = 0, q_cap = 0;
    std::vector<double> edges, dx;
    std::vector<void*> allocs;       // freed at destroy
    std::vector<void*> bank_allocs;  // census bank, record queues, comb members: regrown on overflow
    // mesh and cross sections
    double *d_edges = nullptr, *d_dx = nullptr, *d_sigt = nullptr, *d_inv_sigt = nullptr, *d_c = nullptr,
           *d_siga = nullptr;
    float4* d_cellf = nullptr;
    double2* d_ww_hl = nullptr;
    int32_t* d_region = nullptr;
    double *ww_c = nullptr, *ww_hi = nullptr, *ww_lo = nullptr, *ww_override = nullptr;
    Banks<double> b64;
    Banks<float> b32;
    // per-step accumulators (one clear)
    void* acc = nullptr;
    size_t acc_bytes = 0;
    Acc128 *tl = nullptr, *cent = nullptr, *batch = nullptr, *bnd = nullptr;
    unsigned long long* stats = nullptr;
    unsigned long long* counts = nullptr;  // [0] census, [1] q0, [2] q1, [3..8] comb group list lengths
    // comb groups (one clear)
    void* grp = nullptr;
    size_t grp_bytes = 0;
    unsigned long long* gw = nullptr;
    uint32_t *gcnt = nullptr, *gcur = nullptr;
    GroupRec* gro = nullptr;  // [N+1] census group records from the scan
    unsigned long long *tile_c = nullptr, *tile_w = nullptr;
    MemberRec* member = nullptr;
    unsigned long long* cpre = nullptr;    // comb prefix C0 of every census particle (census-sized)
    GroupRec* glist = nullptr;             // records of the comb groups of 2+ members by size class (census-sized)
    // closures and LOSM
    // two closure sets (phi I+2, J I+1, F I+2, P 2): `cur` holds the
    // initial conditions of the next step, the other is built at t^n
    double *cl_phi[2] = {}, *cl_J[2] = {}, *cl_F[2] = {}, *cl_P[2] = {};
    int cur = 0;
    double *rphi = nullptr, *rJ = nullptr, *rF = nullptr, *mx = nullptr;  // mx: [0] HLOSM, [1] lagged
    double *prev_tl = nullptr, *semi_phi = nullptr, *semi_J = nullptr, *full_phi = nullptr,
           *full_J = nullptr, *norm = nullptr;
    LosmMat mat{};
    LosmWork work{};
    StepDev* sd = nullptr;
    unsigned* err = nullptr;
    // pinned: after each tracking wave the record count, the census count,
    // the error word (its low 32 bits) and the spill count, read with one
    // synchronize
    unsigned long long* h_count = nullptr;
    unsigned long long* d_count = nullptr;  // the device's view of h_count (mapped)
    unsigned long long* spill_n = nullptr;  // device: particles the event loop spilled since the last reset
    StatsExport* h_stats = nullptr;          // pinned, mapped: a step's statistics read back
    StatsExport* d_stats = nullptr;
    // host state
    int xs_set = 0, ww_set = 0;
    double rho = 1.0, eps = 1e-3;
    int mode = 0, scaling = 0;
    long long steps = 0;
    int birth_pos = 0, birth_neg = 0;
    int track_grid = 0;
    size_t track_smem = 0;
    int last_waves = 0;
    int emax = 64;         // events per track before it is requeued
    int n_updates = 0;                 // in-step window updates (Sec. 3, Eq. Hpn)
    double ww_frac[MAX_UPDATES] = {};  // their history fractions
    // likelihood-ratio derivatives (P2 = 2R parameters; 0: off)
    int R = 0, P2 = 0;
    double* d_inv_c = nullptr;                 // I, 1/c (0 where c = 0)
    double* bS = nullptr;                      // [P2][N] start-bank scores
    Acc128 *dtl = nullptr, *dcen = nullptr, *dbnd = nullptr;  // in the accumulator block
    double *dcl_phi[2] = {}, *dcl_J[2] = {}, *dcl_F[2] = {}, *dcl_P[2] = {};  // derivative closure sets
    double *drphi = nullptr, *drJ = nullptr, *drF = nullptr;  // [P2][I+1] scratch
    double* vjp_state = nullptr;               // state block of the last step
    double* vjp_work = nullptr;                // psi, z, g_mc, g_phi, g_J, grad
    unsigned long long xs_version = 0;         // bumped by set_cross_sections
    long long q_peak = 0;  // largest record count a wave produced in the last pass
    // launch accounting
    int timing = 0;
    int track_kind = HWW_TRACK_WARP;  // FP32 wave-0 tracking kernel (hww_set_tracking)
    EvShape ev{0, 0};                 // the event kernel's blocks per SM and ring capacity
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    long long kernel_launches = 0, track_launches = 0, event_launches = 0;
    long long spilled = 0;  // spill_n as of the last tracking wave's synchronize
    double track_ms = 0.0;
};

namespace {

thread_local cudaError_t g_last_cuda_error = cudaSuccess;
thread_local int g_last_cuda_line = 0;

hww_status cuda_status_at(cudaError_t e, int line) {
    if (e == cudaSuccess) return HWW_OK;
    g_last_cuda_error = e;
    g_last_cuda_line = line;
    if (e == cudaErrorMemoryAllocation) return HWW_ERR_OOM;
    return HWW_ERR_CUDA;
}

hww_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return HWW_OK;
    g_last_cuda_error = e;
    if (e == cudaErrorMemoryAllocation) return HWW_ERR_OOM;
    return HWW_ERR_CUDA;
}

}  // namespace

// a CUDA error of another translation unit, recorded for hww_last_error_string
hww_status hww::record_cuda_error(cudaError_t e) { return cuda_status(e); }

namespace {

#define HWW_CK(call)                                              \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_status_at(e_, __LINE__); \
    } while (0)

template <class T>
hww_status dalloc(hww_problem* p, T** ptr, size_t count, bool bank = false) {
    void* v = nullptr;
    const size_t bytes = (count ? count : 1) * sizeof(T);
    cudaError_t e = cudaMallocAsync(&v, bytes, p->stream);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return cuda_status(e);
    }
    (bank ? p->bank_allocs : p->allocs).push_back(v);
    *ptr = (T*)v;
    return HWW_OK;
}

int bit_length(long long n) {
    int l = 0;
    while (n > 0) {
        ++l;
        n >>= 1;
    }
    return l;
}

// birth cell of the pulse: x_k <= x < x_{k+1}, the left cell on an interior
// edge for mu < 0, the end cell on a domain end
int birth_cell(const std::vector<double>& e, int I, double x, double mu) {
    if (x <= e[0]) return 0;
    if (x >= e[I]) return I - 1;
    for (int i = 0; i < I; ++i) {
        if (x == e[i] && i > 0) return mu < 0.0 ? i - 1 : i;
        if (x > e[i] && x < e[i + 1]) return i;
    }
    return I - 1;
}

// exact moments of the unit isotropic pulse at t = 0 (step-1 initial condition)
void source_moments(const hww_problem* p, std::vector<double>& phi) {
    const int I = p->I;
    phi.assign(I + 2, 0.0);
    const double xs = p->d.src_x, v = p->d.v;
    int edge = -1;
    for (int i = 0; i <= I; ++i)
        if (p->edges[i] == xs) edge = i;
    if (edge == 0) {
        phi[1] = v / p->dx[0];
    } else if (edge == I) {
        phi[I] = v / p->dx[I - 1];
    } else if (edge > 0) {
        phi[edge] = 0.5 * v / p->dx[edge - 1];
        phi[edge + 1] = 0.5 * v / p->dx[edge];
    } else {
        for (int i = 0; i < I; ++i)
            if (xs > p->edges[i] && xs < p->edges[i + 1]) phi[i + 1] = v / p->dx[i];
    }
    phi[0] = phi[1];
    phi[I + 1] = phi[I];
}

template <class Real>
hww_status alloc_start_bank(hww_problem* p, Banks<Real>& b) {
    hww_status s;
    const long long N = p->N;
    if ((s = dalloc(p, &b.bank, N))) return s;
    return HWW_OK;
}

// comb group lists (COMB_LIST_MIN gives each list's bound) laid out one
// after the other for a census capacity C
void glist_offsets(long long C, long long off[COMB_LISTS]) {
    long long o = 0;
    for (int k = 0; k < COMB_LISTS; ++k) {
        off[k] = o;
        o += C / COMB_LIST_MIN[k] + 1;
    }
}
size_t glist_len(long long C) {
    long long off[COMB_LISTS];
    glist_offsets(C, off);
    return (size_t)(off[COMB_LISTS - 1] + C / COMB_LIST_MIN[COMB_LISTS - 1] + 1);
}

// census bank, both record queues and the comb member list, sized by the
// current capacities
template <class Real>
hww_status alloc_banks(hww_problem* p, Banks<Real>& b) {
    hww_status s;
    const long long C = p->cen_cap, Q = p->q_cap;
    if ((s = dalloc(p, &b.cen.x, C, true)) || (s = dalloc(p, &b.cen.mu, C, true)) ||
        (s = dalloc(p, &b.cen.w, C, true)) || (s = dalloc(p, &b.cen.cell, C, true)) ||
        (s = dalloc(p, &b.cen.id, C, true)) || (s = dalloc(p, &b.cen.lw, C, true)) ||
        (sizeof(Real) == sizeof(double) && (s = dalloc(p, &b.cen.imu, C, true))) ||
        (s = dalloc(p, &p->member, C, true)) ||
        (s = dalloc(p, &p->cpre, C, true)) || (s = dalloc(p, &p->glist, glist_len(C), true)))
        return s;
    b.cen.cap = C;
    b.cen.count = p->counts + 0;
    for (int k = 0; k < 2; ++k) {
        RecQ<Real>& q = b.q[k];
        if ((s = dalloc(p, &q.x, Q, true)) || (s = dalloc(p, &q.mu, Q, true)) || (s = dalloc(p, &q.tau, Q, true)) ||
            (s = dalloc(p, &q.w, Q, true)) || (s = dalloc(p, &q.cell, Q, true)) || (s = dalloc(p, &q.id, Q, true)) ||
            (s = dalloc(p, &q.lin, Q, true)) || (s = dalloc(p, &q.e, Q, true)) ||
            (s = dalloc(p, &q.jstart, Q, true)) || (s = dalloc(p, &q.jcount, Q, true)))
            return s;
        q.cap = Q;
        q.count = p->counts + 1 + k;
        if (p->P2 > 0 && (s = dalloc(p, &q.S, (size_t)p->P2 * Q, true))) return s;
    }
    if (p->P2 > 0 && (s = dalloc(p, &b.cen.S, (size_t)p->P2 * C, true))) return s;
    return HWW_OK;
}

void free_banks(hww_problem* p) {
    for (void* v : p->bank_allocs) cudaFreeAsync(v, p->stream);
    p->bank_allocs.clear();
}

// grow the census and queue capacities to at least twice their size and at
// least 5/4 of the demand the failed pass saw (the start bank is kept)
// adjoint work vectors: psi (I+2), z (I+2), g_mc (I), g_phi (I+2), g_J (I+1),
// grad (P2)
size_t vjp_work_doubles(int I, int P2) { return 5 * (size_t)I + 7 + (size_t)P2; }

// scores of the start bank, derivative closure sets and their scratch, and
// the adjoint's state block and work vectors
hww_status alloc_deriv(hww_problem* p) {
    const size_t I = (size_t)p->I, P2 = (size_t)p->P2;
    const VjpLayout L = vjp_layout(p->I, p->P2);
    hww_status s;
    if ((s = dalloc(p, &p->d_inv_c, I)) || (s = dalloc(p, &p->bS, P2 * (size_t)p->N)) ||
        (s = dalloc(p, &p->drphi, P2 * (I + 1))) || (s = dalloc(p, &p->drJ, P2 * (I + 1))) ||
        (s = dalloc(p, &p->drF, P2 * (I + 1))) || (s = dalloc(p, &p->vjp_state, (size_t)L.total)) ||
        (s = dalloc(p, &p->vjp_work, vjp_work_doubles(p->I, p->P2))))
        return s;
    for (int k = 0; k < 2; ++k)
        if ((s = dalloc(p, &p->dcl_phi[k], P2 * (I + 2))) || (s = dalloc(p, &p->dcl_J[k], P2 * (I + 1))) ||
            (s = dalloc(p, &p->dcl_F[k], P2 * (I + 2))) || (s = dalloc(p, &p->dcl_P[k], P2 * 2)))
            return s;
    return HWW_OK;
}

hww_status regrow_banks(hww_problem* p, long long cen_need, long long q_need) {
    HWW_CK(cudaStreamSynchronize(p->stream));
    free_banks(p);
    p->cen_cap = std::max(2 * p->cen_cap, cen_need + cen_need / 4);
    p->q_cap = std::max(2 * p->q_cap, q_need + q_need / 4);
    hww_status s = p->fp32 ? alloc_banks(p, p->b32) : alloc_banks(p, p->b64);
    if (s == HWW_OK) HWW_CK(cudaStreamSynchronize(p->stream));
    return s;
}

template <class Real>
TrackArgs<Real> base_track_args(hww_problem* p, const Banks<Real>& b) {
    TrackArgs<Real> a{};
    a.I = p->I;
    a.B = p->B;
    a.N = p->N;
    a.batch_m = p->N > 0 ? ~0ull / (unsigned long long)p->N : 0ull;
    a.comb_shift = bit_length(p->N) - 19;  // S - Sc = (40 - E) - (59 - E - bitlen N)
    a.emax = p->emax;
    a.bc_l = p->d.bc_left;
    a.bc_r = p->d.bc_right;
    a.birth_cell_pos = p->birth_pos;
    a.birth_cell_neg = p->birth_neg;
    a.tau0 = p->d.v * p->d.dt;
    a.tau0f = (float)a.tau0;
    a.src_x = p->d.src_x;
    a.edges = p->d_edges;
    a.inv_sigt = p->d_inv_sigt;
    a.c = p->d_c;
    a.cellf = p->d_cellf;
    a.ww_hl = p->d_ww_hl;
    a.ww_c = p->ww_c;
    a.ww_hi = p->ww_hi;
    a.ww_lo = p->ww_lo;
    a.sd = p->sd;
    a.bank = b.bank;
    a.cen = b.cen;
    a.gcnt = p->gcnt;
    a.gw = p->gw;
    a.tl = p->tl;
    a.cent = p->cent;
    a.batch = p->batch;
    a.bnd = p->bnd;
    a.stats = p->stats;
    a.err = p->err;
    a.spilled = p->spill_n;
    a.R = p->R;
    a.P2 = p->P2;
    a.region = p->d_region;
    a.inv_c = p->d_inv_c;
    a.bS = p->bS;
    a.bank_lo = 0;
    a.bank_hi = LLONG_MAX;
    a.dtl = p->dtl;
    a.dcen = p->dcen;
    a.dbnd = p->dbnd;
    return a;
}

void launch_track(hww_problem* p, const TrackArgs<double>& a) {
    if (p->timing) cudaEventRecord(p->ev_a, p->stream);
    launch_track_fp64(a, p->track_grid, TRACK_BLOCK, p->track_smem, p->stream);
    if (p->timing) cudaEventRecord(p->ev_b, p->stream);
    ++p->kernel_launches;
    ++p->track_launches;
}
void launch_track(hww_problem* p, const TrackArgs<float>& a) {
    if (p->timing) cudaEventRecord(p->ev_a, p->stream);
    const bool ev = a.from_bank && p->ev.blocks_per_sm > 0 &&
                    (p->track_kind == HWW_TRACK_EVENT || p->track_kind == HWW_TRACK_AUTO);
    if (ev) {
        launch_track_fp32_event(a, p->nsm, p->ev, p->stream);
        ++p->event_launches;
    } else {
        launch_track_fp32(a, p->track_grid, TRACK_BLOCK, p->track_smem, p->stream);
    }
    if (p->timing) cudaEventRecord(p->ev_b, p->stream);
    ++p->kernel_launches;
    ++p->track_launches;
}

// after a synchronize: add the last tracking launch's device time
void account_track_time(hww_problem* p) {
    if (!p->timing) return;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev_a, p->ev_b) == cudaSuccess) p->track_ms += ms;
}

// the host's view of a step's end: counters, step state and error word,
// written by one small kernel into pinned mapped host memory (one launch and
// one synchronize instead of small copies into pageable memory)
__global__ void export_stats_kernel(const unsigned long long* stats, const StepDev* sd, const unsigned* err,
                                    StatsExport* out) {
    const int t = threadIdx.x;
    if (t < ST_COUNT) out->stats[t] = stats[t];
    if (t == 0) {
        out->sd = *sd;
        out->err = *err;
    }
}

// after a tracking wave: the record count of its output queue, the census
// count, the error word and the spill count, into the mapped h_count
__global__ void export_wave_kernel(const unsigned long long* qcount, const unsigned long long* ncen,
                                   const unsigned* err, const unsigned long long* spilled,
                                   unsigned long long* out) {
    out[0] = *qcount;
    out[1] = *ncen;
    out[2] = *err;
    out[3] = *spilled;
}

// the tracking waves of start-bank items [lo, hi): wave 0 from the bank,
// then record waves until no record is left
template <class Real>
hww_status track_waves(hww_problem* p, Banks<Real>& b, long long lo = 0, long long hi = LLONG_MAX) {
    TrackArgs<Real> a = base_track_args(p, b);
    a.from_bank = 1;
    a.bank_lo = lo;
    a.bank_hi = hi;
    a.rin = b.q[1];
    a.rout = b.q[0];
    if (lo > 0) HWW_CK(cudaMemsetAsync(b.q[0].count, 0, sizeof(unsigned long long), p->stream));
    launch_track(p, a);
    HWW_CK(cudaGetLastError());
    int cur = 0, waves = 1;
    for (;;) {
        export_wave_kernel<<<1, 1, 0, p->stream>>>(b.q[cur].count, p->counts, p->err, p->spill_n, p->d_count);
        HWW_CK(cudaGetLastError());
        HWW_CK(cudaStreamSynchronize(p->stream));
        account_track_time(p);
        p->spilled = (long long)p->h_count[3];
        p->q_peak = std::max(p->q_peak, (long long)*p->h_count);
        if (*p->h_count == 0) break;
        if (waves >= MAX_WAVES) {
            p->last_waves = waves;
            return HWW_ERR_TIMEOUT;
        }
        const int other = 1 - cur;
        HWW_CK(cudaMemsetAsync(b.q[other].count, 0, sizeof(unsigned long long), p->stream));
        a.from_bank = 0;
        a.rin = b.q[cur];
        a.rout = b.q[other];
        launch_track(p, a);
        HWW_CK(cudaGetLastError());
        cur = other;
        ++waves;
    }
    p->last_waves = waves;
    return HWW_OK;
}

// blocks of the comb kernels (grid-stride loops, so any size is correct):
// about one 256-thread block per 1024 expected census particles (twice the
// start bank), at most 8 per SM.  A small problem's comb then leaves the
// GPU to the other members of a batch, whose stages run as parallel graph
// branches, instead of occupying every SM with near-empty blocks.
int comb_grid(const hww_problem* p) {
    const long long want = (2 * p->N + 1023) / 1024;
    return (int)std::max(1LL, std::min<long long>(want, 8LL * p->nsm));
}

template <class Real>
CombArgs<Real> comb_args(hww_problem* p, Banks<Real>& b) {
    CombArgs<Real> c{};
    c.sd = p->sd;
    c.N = p->N;
    c.ncensus_ptr = p->counts + 0;
    c.cen_cap = p->cen_cap;
    c.cx = b.cen.x;
    c.cmu = b.cen.mu;
    c.cw = b.cen.w;
    c.ccell = b.cen.cell;
    c.cid = b.cen.id;
    c.clw = b.cen.lw;
    c.cimu = b.cen.imu;
    c.gcnt = p->gcnt;
    c.gro = p->gro;
    c.gcur = p->gcur;
    c.member = p->member;
    c.cpre = p->cpre;
    c.glist = p->glist;
    glist_offsets(p->cen_cap, c.glist_off);
    c.glist_n = p->counts + 3;
    c.bank = b.bank;
    c.stats = p->stats;
    c.err = p->err;
    c.I = p->I;
    c.cent = p->cent;
    c.P2 = p->P2;
    c.cS = b.cen.S;
    c.dcen = p->dcen;
    c.bS = p->bS;
    return c;
}

// the comb up to the copies, with the census tallies (Eq. ct-mc): group
// scan, member lists, in-group prefixes, teeth and copies
template <class Real>
hww_status comb_step(hww_problem* p, Banks<Real>& b) {
    ScanArgs s{};
    s.cnt = p->gcnt;
    s.w = p->gw;
    s.n = p->N;
    s.tile_c = p->tile_c;
    s.tile_w = p->tile_w;
    s.out = p->gro;
    s.glist = p->glist;
    glist_offsets(p->cen_cap, s.glist_off);
    s.glist_n = p->counts + 3;
    launch_group_scan(s, p->stream);
    HWW_CK(cudaGetLastError());
    p->kernel_launches += (group_scan_tiles(p->N) > 0) ? 3 : 1;
    launch_comb(comb_args(p, b), comb_grid(p), p->stream);
    HWW_CK(cudaGetLastError());
    p->kernel_launches += 5 + (p->P2 > 0 ? 1 : 0);
    return HWW_OK;
}

// the comb's last kernel: next start-bank size and weight, step-state advance
template <class Real>
hww_status comb_finalize(hww_problem* p, Banks<Real>& b) {
    launch_comb_finalize(comb_args(p, b), p->stream);
    HWW_CK(cudaGetLastError());
    ++p->kernel_launches;
    return HWW_OK;
}

hww_status err_to_status(unsigned e) {
    if (e & (ERR_CENSUS_OVERFLOW | ERR_QUEUE_OVERFLOW)) return HWW_ERR_BANK_OVERFLOW;
    if (e) return HWW_ERR_NUMERIC;
    return HWW_OK;
}

__global__ void normalize_kernel(int kind, const Acc128* a, int n, int I, int B, long long N, const double* dx,
                                 double v, double dt, const StepDev* sd, double* out) {
    const double isc = pow2(-sd->S);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double val = acc_to_double(a[i]) * isc;
        double r;
        if (kind <= HWW_TL_F) {
            r = val / (((double)N * dx[i]) * dt);
        } else if (kind <= HWW_CENSUS_F) {
            r = (v * val) / ((double)N * dx[i]);
        } else if (kind == HWW_BATCH_PHI) {
            const int b = i / I, k = i % I;
            const long long nb = ((b + 1) * N + B - 1) / B - (b * N + B - 1) / B;
            r = nb ? val / (((double)nb * dx[k]) * dt) : 0.0;
        } else {
            r = val / ((double)N * dt);
        }
        out[i] = r;
    }
}

template <class Real>
__global__ void bank_to_x_kernel(const Real* bx, const int32_t* bcell, const double* edges, long long n,
                                 double* out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (sizeof(Real) == sizeof(float)) {
            // offset from the cell's left edge; the FP32 cell width may round
            // above the FP64 one, so the position is clamped into the cell
            const int c = bcell[i];
            out[i] = fmin(fmax(edges[c] + (double)bx[i], edges[c]), edges[c + 1]);
        } else
            out[i] = (double)bx[i];
    }
}

// one field of the start-bank records as doubles: 0 position, 1 direction,
// 2 cell (an int32 copy, into out as raw words)
template <class Real>
__global__ void bank_field_kernel(const BankRec<Real>* bank, const double* edges, long long n, int field,
                                  double* out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const BankRec<Real> r = bank[i];
        if (field == 0) {
            if (sizeof(Real) == sizeof(float)) {
                const int c = r.cell;
                out[i] = fmin(fmax(edges[c] + (double)r.x, edges[c]), edges[c + 1]);
            } else {
                out[i] = (double)r.x;
            }
        } else if (field == 1) {
            out[i] = (double)r.mu;
        } else {
            ((int32_t*)out)[i] = r.cell;
        }
    }
}

template <class Real>
__global__ void to_double_kernel(const Real* in, long long n, double* out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

hww_status copy_out(const hww_problem* p, double* out, const double* src, size_t n, int on_device) {
    HWW_CK(cudaMemcpyAsync(out, src, n * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
    if (!on_device) HWW_CK(cudaStreamSynchronize(p->stream));
    return HWW_OK;
}


// normalised derivative tallies: which 0 track length [P2][I], 1..3 census
// phi, J, F [P2][I], 4 boundary [P2][6]; the same scalings as the tallies
__global__ void deriv_normalize_kernel(int which, int P2, int I, long long N, const double* dx, double v, double dt,
                                       const StepDev* sd, const Acc128* dtl, const Acc128* dcen,
                                       const Acc128* dbnd, double* out) {
    const double isc = pow2(-sd->S);
    const int n = (which == 4) ? 6 * P2 : P2 * I;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        if (which == 4) {
            out[t] = (acc_to_double(dbnd[t]) * isc) / ((double)N * dt);
            continue;
        }
        const int j = t / I, i = t % I;
        if (which == 0) {
            out[t] = (acc_to_double(dtl[t]) * isc) / (((double)N * dx[i]) * dt);
        } else {
            const Acc128 a = dcen[(long long)j * 3 * I + (long long)(which - 1) * I + i];
            out[t] = (v * (acc_to_double(a) * isc)) / ((double)N * dx[i]);
        }
    }
}

void launch_deriv_normalize(const hww_problem* p, int which, double* out) {
    const int n = (which == 4) ? 6 * p->P2 : p->P2 * p->I;
    const int grid = std::max(1, std::min(64, (n + 255) / 256));
    deriv_normalize_kernel<<<grid, 256, 0, p->stream>>>(which, p->P2, p->I, p->N, p->d_dx, p->d.v, p->d.dt, p->sd,
                                                         p->dtl, p->dcen, p->dbnd, out);
}

// the adjoint's state block of the last step (device, p->vjp_state)
hww_status fill_vjp_state(hww_problem* p) {
    const int I = p->I, P2 = p->P2;
    const VjpLayout L = vjp_layout(I, P2);
    const int nw = p->cur, od = 1 - p->cur;  // after a step: set `cur` was built at t^n
    double* st = p->vjp_state;
    const double hdr[4] = {(double)I, (double)P2, (double)p->xs_version, (double)p->steps};
    auto d2d = [&](double* dst, const double* src, size_t n) {
        return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream);
    };
    HWW_CK(cudaMemcpyAsync(st, hdr, sizeof(hdr), cudaMemcpyHostToDevice, p->stream));
    HWW_CK(d2d(st + L.phi_old, p->cl_phi[od], I + 2));
    HWW_CK(d2d(st + L.J_old, p->cl_J[od], I + 1));
    HWW_CK(d2d(st + L.phi_new, p->full_phi, I + 2));
    HWW_CK(d2d(st + L.J_new, p->full_J, I + 1));
    launch_deriv_normalize(p, 0, st + L.dtl);
    HWW_CK(cudaGetLastError());
    HWW_CK(d2d(st + L.dphi_old, p->dcl_phi[od], (size_t)P2 * (I + 2)));
    HWW_CK(d2d(st + L.dJ_old, p->dcl_J[od], (size_t)P2 * (I + 1)));
    HWW_CK(d2d(st + L.dF_old, p->dcl_F[od], (size_t)P2 * (I + 2)));
    HWW_CK(d2d(st + L.dF_new, p->dcl_F[nw], (size_t)P2 * (I + 2)));
    HWW_CK(d2d(st + L.dP_new, p->dcl_P[nw], (size_t)P2 * 2));
    // the header is read back from pageable memory: wait before it goes
    HWW_CK(cudaStreamSynchronize(p->stream));
    return HWW_OK;
}

// Stages of one time step.  Every launch parameter below is fixed for the
// life of the problem (the per-step values live in StepDev), so the stages
// can also be recorded into CUDA graphs (see the batch engine).
LosmRhsIn semi_rhs(const hww_problem* p) {
    LosmRhsIn in{};
    in.sd = p->sd;
    in.full = 0;
    for (int k = 0; k < 2; ++k) {
        in.set_phi[k] = p->cl_phi[k];
        in.set_J[k] = p->cl_J[k];
        in.set_F[k] = p->cl_F[k];
        in.set_P[k] = p->cl_P[k];
    }
    return in;
}

// clear the step's accumulators; step scalars; semi-implicit HLOSM with the
// lagged closure (Eqs. losm-0, losm-1-semi, losm-disc-bc-semi); windows
hww_status stage_pre(hww_problem* p) {
    HWW_CK(cudaMemsetAsync(p->acc, 0, p->acc_bytes, p->stream));
    HWW_CK(cudaMemsetAsync(p->grp, 0, p->grp_bytes, p->stream));
    launch_step_scalars(p->sd, bit_length(p->N), p->d.seed, p->mode, p->stats, p->stream);
    p->kernel_launches += 1 + launch_losm_solve(p->mat, semi_rhs(p), p->work, p->semi_phi, p->semi_J, p->mx,
                                                p->stream);
    WwArgs wa{};
    wa.I = p->I;
    wa.scaling = p->scaling;
    wa.eps = p->eps;
    wa.rho = p->rho;
    wa.sd = p->sd;
    wa.phit_hlosm = p->semi_phi + 1;
    wa.phit_prev = p->prev_tl;
    wa.mx_hlosm = p->mx;
    wa.mx_prev = p->mx + 1;
    wa.override_c = p->ww_override;
    wa.ww_c = p->ww_c;
    wa.ww_hi = p->ww_hi;
    wa.ww_lo = p->ww_lo;
    wa.ww_hl = p->d_ww_hl;
    p->kernel_launches += launch_ww_centers(wa, p->mode == HWW_MODE_LWW, p->stream);
    HWW_CK(cudaGetLastError());
    return HWW_OK;
}

// the comb with the census tallies (Eq. ct-mc; the comb does not depend on
// the closures), closures and initial conditions at t^n, the fully implicit
// HLOSM (Eqs. losm-0, losm-1, losm-disc-bc), and the step-state advance
hww_status stage_post(hww_problem* p) {
    launch_tl_phi(p->tl, p->batch, p->B, p->I, p->stream);
    ++p->kernel_launches;
    if (p->n_updates > 0)  // an in-step update left partial census tallies
        HWW_CK(cudaMemsetAsync(p->cent, 0, sizeof(Acc128) * 3 * (size_t)p->I, p->stream));
    hww_status st = p->fp32 ? comb_step(p, p->b32) : comb_step(p, p->b64);
    if (st) return st;
    ClosureArgs ca{};
    ca.I = p->I;
    ca.sd = p->sd;
    ca.v = p->d.v;
    ca.dt = p->d.dt;
    ca.N = p->N;
    ca.bc_l = p->d.bc_left;
    ca.bc_r = p->d.bc_right;
    ca.filter_k = p->d.filter == HWW_FILTER_MA ? p->d.filter_k : 0;
    ca.fourier = p->d.filter == HWW_FILTER_FOURIER;
    ca.kappa = p->d.filter_k;
    ca.dx = p->d_dx;
    ca.cent = p->cent;
    ca.tl = p->tl;
    ca.bnd = p->bnd;
    ca.rphi = p->rphi;
    ca.rJ = p->rJ;
    ca.rF = p->rF;
    for (int k = 0; k < 2; ++k) {
        ca.set_phi[k] = p->cl_phi[k];
        ca.set_J[k] = p->cl_J[k];
        ca.set_F[k] = p->cl_F[k];
        ca.set_P[k] = p->cl_P[k];
    }
    ca.prev_tl = p->prev_tl;
    ca.nsets = 1;
    p->kernel_launches += launch_closures(ca, p->stream);
    if (p->P2 > 0) {
        // derivative closures: the same linear map on the derivative census
        // and boundary tallies, one set per parameter
        ClosureArgs dc = ca;
        dc.cent = p->dcen;
        dc.bnd = p->dbnd;
        dc.tl = nullptr;
        dc.rphi = p->drphi;
        dc.rJ = p->drJ;
        dc.rF = p->drF;
        for (int k = 0; k < 2; ++k) {
            dc.set_phi[k] = p->dcl_phi[k];
            dc.set_J[k] = p->dcl_J[k];
            dc.set_F[k] = p->dcl_F[k];
            dc.set_P[k] = p->dcl_P[k];
        }
        dc.nsets = p->P2;
        p->kernel_launches += launch_closures(dc, p->stream);
    }
    LosmRhsIn full = semi_rhs(p);
    full.full = 1;
    p->kernel_launches += launch_losm_solve(p->mat, full, p->work, p->full_phi, p->full_J, nullptr, p->stream);
    HWW_CK(cudaGetLastError());
    return p->fp32 ? comb_finalize(p, p->b32) : comb_finalize(p, p->b64);
}

double bits_to_double(unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
}

// step statistics from the raw counters, the start-bank size and weight of
// the next step and the device error word
void fill_stats(const unsigned long long* h, unsigned long long nbank, double wbar, unsigned e, int waves,
                hww_step_stats* st) {
    std::memset(st, 0, sizeof(*st));
    st->segments = (int64_t)h[ST_SEGMENTS];
    st->collisions = (int64_t)h[ST_COLLISIONS];
    st->crossings = (int64_t)h[ST_CROSSINGS];
    st->reflections = (int64_t)h[ST_REFLECTIONS];
    st->leaked = (int64_t)h[ST_LEAKED];
    st->absorbed = (int64_t)h[ST_ABSORBED];
    st->scatters = (int64_t)h[ST_SCATTERS];
    st->split_events = (int64_t)h[ST_SPLIT_EVENTS];
    st->daughters = (int64_t)h[ST_DAUGHTERS];
    st->roulette_kills = (int64_t)h[ST_RKILLS];
    st->roulette_survivals = (int64_t)h[ST_RSURVIVE];
    st->census = (int64_t)h[ST_CENSUS];
    st->lineage_collisions = (int64_t)h[ST_LINEAGE];
    st->max_events = (int64_t)h[ST_MAX_EVENTS];
    st->n_next = (int64_t)nbank;
    st->n_start = (int64_t)h[ST_NSTART];
    st->w_bar_next = wbar;
    st->waves = waves;
    st->status = err_to_status(e);
}

// windows of an in-step update (Sec. 3, Eq. Hpn): closures from the census
// and boundary tallies of the first Hp histories (normalised by Hp), the
// fully implicit HLOSM solution with them as the new level, centers from it
hww_status update_windows(hww_problem* p, long long Hp) {
    // the census tallies of the histories so far (the comb forms the step's
    // own at its end)
    HWW_CK(cudaMemsetAsync(p->cent, 0, sizeof(Acc128) * 3 * (size_t)p->I, p->stream));
    if (p->fp32)
        launch_census_tallies(comb_args(p, p->b32), 2 * p->nsm, p->stream);
    else
        launch_census_tallies(comb_args(p, p->b64), 2 * p->nsm, p->stream);
    ++p->kernel_launches;
    ClosureArgs ca{};
    ca.I = p->I;
    ca.sd = p->sd;
    ca.v = p->d.v;
    ca.dt = p->d.dt;
    ca.N = Hp;
    ca.bc_l = p->d.bc_left;
    ca.bc_r = p->d.bc_right;
    ca.filter_k = p->d.filter == HWW_FILTER_MA ? p->d.filter_k : 0;
    ca.fourier = p->d.filter == HWW_FILTER_FOURIER;
    ca.kappa = p->d.filter_k;
    ca.dx = p->d_dx;
    ca.cent = p->cent;
    ca.tl = nullptr;
    ca.bnd = p->bnd;
    ca.rphi = p->rphi;
    ca.rJ = p->rJ;
    ca.rF = p->rF;
    for (int k = 0; k < 2; ++k) {
        ca.set_phi[k] = p->cl_phi[k];
        ca.set_J[k] = p->cl_J[k];
        ca.set_F[k] = p->cl_F[k];
        ca.set_P[k] = p->cl_P[k];
    }
    ca.prev_tl = p->prev_tl;
    ca.nsets = 1;
    p->kernel_launches += launch_closures(ca, p->stream);
    LosmRhsIn full = semi_rhs(p);
    full.full = 1;
    p->kernel_launches += launch_losm_solve(p->mat, full, p->work, p->full_phi, p->full_J, p->mx, p->stream);
    WwArgs wa{};
    wa.I = p->I;
    wa.scaling = p->scaling;
    wa.eps = p->eps;
    wa.rho = p->rho;
    wa.sd = p->sd;
    wa.phit_hlosm = p->full_phi + 1;
    wa.phit_prev = p->prev_tl;
    wa.mx_hlosm = p->mx;
    wa.mx_prev = p->mx + 1;
    wa.override_c = p->ww_override;
    wa.ww_c = p->ww_c;
    wa.ww_hi = p->ww_hi;
    wa.ww_lo = p->ww_lo;
    wa.ww_hl = p->d_ww_hl;
    p->kernel_launches += launch_ww_centers(wa, 0, p->stream);
    HWW_CK(cudaGetLastError());
    return HWW_OK;
}

// the tracking of one step: in u_ww + 1 chunks of source ids when in-step
// window updates are on and the step's windows come from the HLOSM solution
template <class Real>
hww_status track_step(hww_problem* p, Banks<Real>& b) {
    if (p->n_updates == 0 || p->mode != HWW_MODE_HWW) return track_waves(p, b);
    StepDev sdh;
    HWW_CK(cudaMemcpyAsync(&sdh, p->sd, sizeof(StepDev), cudaMemcpyDeviceToHost, p->stream));
    HWW_CK(cudaStreamSynchronize(p->stream));
    if (sdh.ww_src != 1) return track_waves(p, b);  // an override step: no updates
    const long long H = (long long)sdh.nbank;
    const int u = p->n_updates;
    int waves = 0;
    for (int c = 0; c <= u; ++c) {
        const long long lo = (c == 0) ? 0 : (long long)(p->ww_frac[c - 1] * (double)H);
        const long long hi = (c == u) ? H : (long long)(p->ww_frac[c] * (double)H);
        const hww_status s = track_waves(p, b, lo, hi);
        if (s) return s;
        waves += p->last_waves;
        if (c < u && hi > 0) {
            const hww_status s2 = update_windows(p, hi);
            if (s2) return s2;
        }
    }
    p->last_waves = waves;
    return HWW_OK;
}

// The tracking of a step, replayed from its start with larger buffers when a
// census bank or record queue overflowed (the start bank and the closure
// vectors are untouched until the post stage, so a replay is bit-identical
// to a run that had the room from the beginning).  After MAX_REGROW regrowths
// the step goes on with the overflow flagged in its status.
hww_status track_with_regrow(hww_problem* p) {
    for (int attempt = 0;; ++attempt) {
        hww_status s = stage_pre(p);
        if (s) return s;
        p->q_peak = 0;
        s = p->fp32 ? track_step(p, p->b32) : track_step(p, p->b64);
        if (s) return s;
        // the step's tracking ends with a wave; its synchronize read the
        // census count and the error word
        const unsigned e = (unsigned)p->h_count[2];
        const unsigned long long ncen = p->h_count[1];
        if (!(e & (ERR_CENSUS_OVERFLOW | ERR_QUEUE_OVERFLOW)) || attempt >= MAX_REGROW) return HWW_OK;
        s = regrow_banks(p, (long long)ncen, p->q_peak);
        if (s) return s;
        const unsigned keep = e & ~(unsigned)(ERR_CENSUS_OVERFLOW | ERR_QUEUE_OVERFLOW);
        HWW_CK(cudaMemcpyAsync(p->err, &keep, sizeof(unsigned), cudaMemcpyHostToDevice, p->stream));
        HWW_CK(cudaStreamSynchronize(p->stream));
    }
}

hww_status read_stats(hww_problem* p, hww_step_stats* st) {
    export_stats_kernel<<<1, 32, 0, p->stream>>>(p->stats, p->sd, p->err, p->d_stats);
    HWW_CK(cudaGetLastError());
    HWW_CK(cudaStreamSynchronize(p->stream));
    const StatsExport& x = *p->h_stats;
    const unsigned e = x.err;
    fill_stats(x.stats, x.sd.nbank, x.sd.wbar, e, p->last_waves, st);
    if (e) HWW_CK(cudaMemsetAsync(p->err, 0, sizeof(unsigned), p->stream));
    return (hww_status)st->status;
}

}  // namespace

extern "C" {

const char* hww_last_error_string(void) {
    static thread_local char buf[256];
    std::snprintf(buf, sizeof buf, "%s (%s) at api.cu:%d", cudaGetErrorName(g_last_cuda_error),
                  cudaGetErrorString(g_last_cuda_error), g_last_cuda_line);
    return buf;
}

const char* hww_status_string(hww_status s) {
    switch (s) {
    case HWW_OK: return "ok";
    case HWW_ERR_ARG: return "invalid argument";
    case HWW_ERR_STATE: return "call out of order";
    case HWW_ERR_OOM: return "out of memory";
    case HWW_ERR_BANK_OVERFLOW: return "particle bank or queue overflow";
    case HWW_ERR_TIMEOUT: return "bounded wait gave up";
    case HWW_ERR_NUMERIC: return "numeric guard fired";
    case HWW_ERR_CUDA: return "CUDA runtime error";
    case HWW_ERR_NO_DEVICE: return "no CUDA device";
    }
    return "unknown status";
}

void destroy_problem(hww_problem* p) {
    if (!p) return;
    cudaSetDevice(p->device);
    for (void* v : p->allocs) cudaFreeAsync(v, p->stream);
    free_banks(p);
    cudaStreamSynchronize(p->stream);
    if (p->h_count) cudaFreeHost(p->h_count);
    if (p->h_stats) cudaFreeHost(p->h_stats);
    if (p->ev_a) cudaEventDestroy(p->ev_a);
    if (p->ev_b) cudaEventDestroy(p->ev_b);
    delete p;
}

hww_status create_problem(const hww_problem_desc* d, hww_problem** out) {
    if (!out) return HWW_ERR_ARG;
    *out = nullptr;
    if (!d || !d->edges) return HWW_ERR_ARG;
    const int I = d->n_cells;
    if (I < 1 || I > MAX_CELLS || !(d->v > 0) || !(d->dt > 0) || !std::isfinite(d->v * d->dt) ||
        d->particles_per_step < 1 || d->particles_per_step >= (1LL << 30) ||
        (d->theta != 0.5 && d->theta != 1.0) || d->n_var_batches < 1 || d->n_var_batches > 64 ||
        d->bc_left < 0 || d->bc_left > 1 || d->bc_right < 0 || d->bc_right > 1 || d->filter < 0 ||
        d->filter > 2 || (d->filter == 1 && d->filter_k < 1) || (d->filter == 2 && d->filter_k < 0) ||
        d->precision < 0 || d->precision > 1 ||
        d->deriv_regions < 0 || d->deriv_regions > MAX_SCORES / 2 ||
        (d->deriv_regions > 0 && d->precision != HWW_FP64) || d->bank_capacity < 0)
        return HWW_ERR_ARG;
    for (int i = 0; i < I; ++i)
        if (!(d->edges[i + 1] > d->edges[i]) || !std::isfinite(d->edges[i + 1])) return HWW_ERR_ARG;
    if (!(d->src_x >= d->edges[0] && d->src_x <= d->edges[I])) return HWW_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return HWW_ERR_NO_DEVICE;
    if (d->device < 0 || d->device >= ndev) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(d->device));

    hww_problem* p = new (std::nothrow) hww_problem();
    if (!p) return HWW_ERR_OOM;
    p->d = *d;
    p->d.edges = nullptr;
    p->I = I;
    p->B = d->n_var_batches;
    p->N = d->particles_per_step;
    p->fp32 = d->precision == HWW_FP32_TRACK;
    p->R = d->deriv_regions;
    p->P2 = 2 * p->R;
    p->stream = (cudaStream_t)d->cuda_stream;
    p->device = d->device;
    p->edges.assign(d->edges, d->edges + I + 1);
    p->dx.resize(I);
    for (int i = 0; i < I; ++i) p->dx[i] = p->edges[i + 1] - p->edges[i];
    p->cen_cap = d->bank_capacity ? d->bank_capacity : 4 * p->N;
    p->q_cap = d->bank_capacity ? d->bank_capacity / 2 + 1 : 2 * p->N;
    cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);
    p->birth_pos = birth_cell(p->edges, I, d->src_x, 1.0);
    p->birth_neg = birth_cell(p->edges, I, d->src_x, -1.0);

    hww_status s = HWW_OK;
    const int B = p->B;
    const size_t P2 = (size_t)p->P2;
    const size_t acc_main = sizeof(Acc128) * (6 * (size_t)I + (size_t)B * I + 6) +
                            sizeof(unsigned long long) * (ST_COUNT + 3 + COMB_LISTS);
    // derivative accumulators after the main block (16-byte aligned)
    const size_t acc_off = (acc_main + 15) / 16 * 16;
    p->acc_bytes = acc_off + sizeof(Acc128) * (P2 * I + 3 * P2 * I + 6 * P2);
    p->grp_bytes = (sizeof(unsigned long long) + 2 * sizeof(uint32_t)) * (size_t)p->N;
    const long long ntiles = group_scan_tiles(p->N);
    if ((s = dalloc(p, (char**)&p->acc, p->acc_bytes)) || (s = dalloc(p, (char**)&p->grp, p->grp_bytes)) ||
        (s = dalloc(p, &p->d_edges, I + 1)) || (s = dalloc(p, &p->d_dx, I)) || (s = dalloc(p, &p->d_sigt, I)) ||
        (s = dalloc(p, &p->d_inv_sigt, I)) || (s = dalloc(p, &p->d_c, I)) || (s = dalloc(p, &p->d_siga, I)) ||
        (s = dalloc(p, &p->d_region, I)) ||
        (s = dalloc(p, &p->ww_c, I)) || (s = dalloc(p, &p->ww_hi, I)) || (s = dalloc(p, &p->ww_lo, I)) ||
        (s = dalloc(p, &p->ww_override, I)) || (s = dalloc(p, &p->d_cellf, I)) || (s = dalloc(p, &p->d_ww_hl, I)) || (s = dalloc(p, &p->gro, p->N + 1)) ||
        (s = dalloc(p, &p->tile_c, ntiles + 1)) ||
        (s = dalloc(p, &p->tile_w, ntiles + 1)) ||
        (s = dalloc(p, &p->cl_phi[0], I + 2)) || (s = dalloc(p, &p->cl_J[0], I + 1)) ||
        (s = dalloc(p, &p->cl_F[0], I + 2)) || (s = dalloc(p, &p->cl_P[0], 2)) ||
        (s = dalloc(p, &p->cl_phi[1], I + 2)) || (s = dalloc(p, &p->cl_J[1], I + 1)) ||
        (s = dalloc(p, &p->cl_F[1], I + 2)) || (s = dalloc(p, &p->cl_P[1], 2)) || (s = dalloc(p, &p->rphi, I)) ||
        (s = dalloc(p, &p->rJ, I + 1)) || (s = dalloc(p, &p->rF, I)) || (s = dalloc(p, &p->mx, 2)) ||
        (s = dalloc(p, &p->prev_tl, I)) || (s = dalloc(p, &p->semi_phi, I + 2)) ||
        (s = dalloc(p, &p->semi_J, I + 1)) || (s = dalloc(p, &p->full_phi, I + 2)) ||
        (s = dalloc(p, &p->full_J, I + 1)) || (s = dalloc(p, &p->work.u, I + 2)) ||
        (s = dalloc(p, &p->work.mom, I + 1)) || (s = dalloc(p, &p->work.y, I + 2)) ||
        (s = dalloc(p, &p->mat.eJ, I + 1)) || (s = dalloc(p, &p->mat.eS, I + 1)) ||
        (s = dalloc(p, &p->mat.invd, I + 1)) || (s = dalloc(p, &p->mat.g, I + 1)) ||
        (s = dalloc(p, &p->mat.cP, I)) || (s = dalloc(p, &p->mat.cA, I)) || (s = dalloc(p, &p->mat.cB, I)) ||
        (s = dalloc(p, &p->mat.inv_den, I + 2)) || (s = dalloc(p, &p->mat.vf, I + 2)) ||
        (s = dalloc(p, &p->mat.cp, I + 2)) || (s = dalloc(p, &p->mat.nA, I + 2)) ||
        (s = dalloc(p, &p->norm, (size_t)B * I + 6 * (size_t)I + 8)) || (s = dalloc(p, &p->sd, 1)) ||
        (s = dalloc(p, &p->err, 1)) || (s = dalloc(p, &p->spill_n, 1))) {
        destroy_problem(p);
        return s;
    }
    char* acc = (char*)p->acc;
    p->tl = (Acc128*)acc;
    p->cent = p->tl + 3 * I;
    p->batch = p->cent + 3 * I;
    p->bnd = p->batch + (size_t)B * I;
    p->stats = (unsigned long long*)(p->bnd + 6);
    p->counts = p->stats + ST_COUNT;
    if (p->P2 > 0) {
        p->dtl = (Acc128*)(acc + acc_off);
        p->dcen = p->dtl + P2 * I;
        p->dbnd = p->dcen + 3 * P2 * I;
    }
    p->gw = (unsigned long long*)p->grp;
    p->gcnt = (uint32_t*)(p->gw + p->N);
    p->gcur = p->gcnt + p->N;
    s = p->fp32 ? alloc_start_bank(p, p->b32) : alloc_start_bank(p, p->b64);
    if (s == HWW_OK) s = p->fp32 ? alloc_banks(p, p->b32) : alloc_banks(p, p->b64);
    if (s == HWW_OK && p->P2 > 0) s = alloc_deriv(p);
    if (s) {
        destroy_problem(p);
        return s;
    }
    if (cudaHostAlloc(&p->h_count, 4 * sizeof(unsigned long long), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&p->d_count, p->h_count, 0) != cudaSuccess ||
        cudaHostAlloc(&p->h_stats, sizeof(StatsExport), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&p->d_stats, p->h_stats, 0) != cudaSuccess) {
        destroy_problem(p);
        return HWW_ERR_OOM;
    }
    // mesh, initial condition and step scalars
    std::vector<double> phi0;
    source_moments(p, phi0);
    std::vector<double> zeros(I + 2, 0.0);
    StepDev sd{};
    sd.wbar = 1.0;
    sd.nbank = (unsigned long long)p->N;
    cudaError_t e = cudaSuccess;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, p->stream);
    };
    up(p->d_edges, p->edges.data(), sizeof(double) * (I + 1));
    up(p->d_dx, p->dx.data(), sizeof(double) * I);
    up(p->cl_phi[0], phi0.data(), sizeof(double) * (I + 2));
    up(p->cl_J[0], zeros.data(), sizeof(double) * (I + 1));
    up(p->cl_F[0], zeros.data(), sizeof(double) * (I + 2));
    up(p->cl_P[0], zeros.data(), sizeof(double) * 2);
    if (p->P2 > 0) {
        // derivative closures of the exact pulse moments, and the scores of
        // the first start bank: zero
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaMemsetAsync(p->dcl_phi[k], 0, sizeof(double) * P2 * (I + 2), p->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->dcl_J[k], 0, sizeof(double) * P2 * (I + 1), p->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->dcl_F[k], 0, sizeof(double) * P2 * (I + 2), p->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->dcl_P[k], 0, sizeof(double) * P2 * 2, p->stream);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(p->bS, 0, sizeof(double) * P2 * p->N, p->stream);
    }
    p->mat.I = I;
    p->mat.theta = d->theta;
    p->mat.bc_l = d->bc_left;
    p->mat.bc_r = d->bc_right;
    up(p->sd, &sd, sizeof(StepDev));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->err, 0, sizeof(unsigned), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->spill_n, 0, sizeof(unsigned long long), p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        destroy_problem(p);
        return cuda_status(e);
    }
    // tracking launch shape: persistent grid of resident blocks
    p->track_smem = sizeof(long long) * ((p->fp32 ? TALLY_ROWS_FP32 : TALLY_ROWS) + P2) * (size_t)I;
    // the dynamic shared memory limits are set whatever the sizes: a kernel's
    // static shared memory counts against the default 48 KB as well
    const size_t cen_smem = sizeof(long long) * 3 * (size_t)I;
    if ((p->fp32 ? track_smem_optin_fp32(p->track_smem) : track_smem_optin_fp64(p->track_smem, p->P2 > 0)) != 0 ||
        (p->fp32 ? comb_write_smem_optin<float>(cen_smem) : comb_write_smem_optin<double>(cen_smem)) != 0 ||
        (p->fp32 ? census_tally_smem_optin<float>(cen_smem) : census_tally_smem_optin<double>(cen_smem)) != 0 ||
        (P2 > 0 && (p->fp32 ? deriv_census_smem_optin<float>(P2, I) : deriv_census_smem_optin<double>(P2, I)) != 0)) {
        destroy_problem(p);
        return HWW_ERR_CUDA;
    }
    if (d->filter == HWW_FILTER_FOURIER) {
        const long long kp = std::min<long long>(d->filter_k, (I + 1) / 2);
        if (fourier_filter_smem_optin(sizeof(double) * ((size_t)I + 1 + 2 * ((size_t)kp + 1))) != 0) {
            destroy_problem(p);
            return HWW_ERR_CUDA;
        }
    }
    int per_sm = p->fp32 ? track_blocks_per_sm_fp32(TRACK_BLOCK, p->track_smem)
                         : track_blocks_per_sm_fp64(TRACK_BLOCK, p->track_smem, p->P2 > 0);
    if (per_sm < 1) per_sm = 1;
    p->track_grid = p->nsm * per_sm;
    // FP32 problems track wave 0 with the event kernel where its rings fit
    // the mesh (measured as fast as or faster than the warp loop on every
    // step of the slab and shield workloads, its record waves included)
    if (p->fp32) {
        const EvShape sh = ev_shape(I);
        if (sh.blocks_per_sm > 0 && track_event_smem_optin_fp32(I, sh.cap) == 0) {
            p->ev = sh;
            p->track_kind = HWW_TRACK_AUTO;
        }
    }
    *out = p;
    return HWW_OK;
}

hww_status set_cross_sections(hww_problem* p, const double* sigma_t, const double* c, const int32_t* region) {
    if (!p || !sigma_t || !c) return HWW_ERR_ARG;
    const int I = p->I;
    for (int i = 0; i < I; ++i) {
        if (!(sigma_t[i] > 0) || !std::isfinite(sigma_t[i]) || !(c[i] >= 0 && c[i] <= MAX_C) ||
            (p->P2 > 0 && c[i] > 1.0))
            return HWW_ERR_ARG;
        if (region && (region[i] < 0 || (p->d.deriv_regions > 0 && region[i] >= p->d.deriv_regions)))
            return HWW_ERR_ARG;
    }
    HWW_CK(cudaSetDevice(p->device));
    std::vector<double> st(sigma_t, sigma_t + I), inv(I), cc(c, c + I), sa(I);
    std::vector<float> invf(I);
    std::vector<float4> cellf(I);
    std::vector<int32_t> reg(I, 0);
    for (int i = 0; i < I; ++i) {
        inv[i] = 1.0 / st[i];
        invf[i] = (float)(1.0 / st[i]);
        sa[i] = st[i] * (1.0 - cc[i]);
        cellf[i] = make_float4((float)p->dx[i], invf[i], (float)cc[i], 0.0f);
        if (region) reg[i] = region[i];
    }
    HWW_CK(cudaMemcpyAsync(p->d_cellf, cellf.data(), sizeof(float4) * I, cudaMemcpyHostToDevice, p->stream));
    HWW_CK(cudaMemcpyAsync(p->d_sigt, st.data(), sizeof(double) * I, cudaMemcpyHostToDevice, p->stream));
    HWW_CK(cudaMemcpyAsync(p->d_inv_sigt, inv.data(), sizeof(double) * I, cudaMemcpyHostToDevice, p->stream));
    HWW_CK(cudaMemcpyAsync(p->d_c, cc.data(), sizeof(double) * I, cudaMemcpyHostToDevice, p->stream));
    HWW_CK(cudaMemcpyAsync(p->d_siga, sa.data(), sizeof(double) * I, cudaMemcpyHostToDevice, p->stream));
    HWW_CK(cudaMemcpyAsync(p->d_region, reg.data(), sizeof(int32_t) * I, cudaMemcpyHostToDevice, p->stream));
    std::vector<double> ic(I);
    if (p->P2 > 0) {
        for (int i = 0; i < I; ++i) ic[i] = (cc[i] > 0.0) ? 1.0 / cc[i] : 0.0;
        HWW_CK(cudaMemcpyAsync(p->d_inv_c, ic.data(), sizeof(double) * I, cudaMemcpyHostToDevice, p->stream));
    }
    // the LOSM matrix depends on the cross sections: refactor it
    launch_losm_setup(p->mat, p->d_dx, p->d_sigt, p->d_siga, p->d.v, p->d.dt, p->d.theta, p->d.bc_left,
                      p->d.bc_right, p->err, p->stream);
    HWW_CK(cudaGetLastError());
    p->kernel_launches += 2;
    unsigned e = 0;
    HWW_CK(cudaMemcpyAsync(&e, p->err, sizeof(unsigned), cudaMemcpyDeviceToHost, p->stream));
    HWW_CK(cudaStreamSynchronize(p->stream));
    if (e & ERR_LOSM) return HWW_ERR_NUMERIC;
    p->xs_set = 1;
    ++p->xs_version;
    return HWW_OK;
}

hww_status set_ww_params(hww_problem* p, double rho, double eps_min, int32_t mode, int32_t scaling) {
    if (!p || !(rho >= 1.0) || !std::isfinite(rho) || !(eps_min > 0.0 && eps_min <= 1.0) || mode < 0 ||
        mode > 2 || scaling < 0 || scaling > 1)
        return HWW_ERR_ARG;
    p->rho = rho;
    p->eps = eps_min;
    p->mode = mode;
    p->scaling = scaling;
    p->ww_set = 1;
    return HWW_OK;
}

hww_status set_ww_centers(hww_problem* p, const double* centers) {
    if (!p || !centers) return HWW_ERR_ARG;
    for (int i = 0; i < p->I; ++i)
        if (!(centers[i] > 0) || !std::isfinite(centers[i])) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(p->device));
    HWW_CK(cudaMemcpyAsync(p->ww_override, centers, sizeof(double) * p->I, cudaMemcpyHostToDevice, p->stream));
    const int one = 1;
    HWW_CK(cudaMemcpyAsync(&p->sd->override_c, &one, sizeof(int), cudaMemcpyHostToDevice, p->stream));
    HWW_CK(cudaStreamSynchronize(p->stream));
    return HWW_OK;
}

hww_status set_ww_updates(hww_problem* p, int32_t n, const double* fractions) {
    if (!p || n < 0 || n > MAX_UPDATES) return HWW_ERR_ARG;
    double f[MAX_UPDATES];
    for (int k = 0; k < n; ++k) {
        // default f_p = p / (u + 1) (the fractions the paper uses)
        f[k] = fractions ? fractions[k] : (double)(k + 1) / (double)(n + 1);
        if (!(f[k] > 0.0 && f[k] < 1.0) || (k > 0 && !(f[k] > f[k - 1]))) return HWW_ERR_ARG;
    }
    for (int k = 0; k < n; ++k) p->ww_frac[k] = f[k];
    p->n_updates = n;
    return HWW_OK;
}

hww_status run_step(hww_problem* p, hww_step_stats* st) {
    if (!p) return HWW_ERR_ARG;
    if (!p->xs_set || !p->ww_set) return HWW_ERR_STATE;
    HWW_CK(cudaSetDevice(p->device));
    // Tracking (replayed from the step's start with larger buffers on an
    // overflow)
    hww_status s = track_with_regrow(p);
    if (s) return s;
    s = stage_post(p);
    if (s) return s;
    p->cur ^= 1;
    p->steps += 1;
    return st ? read_stats(p, st) : HWW_OK;
}

hww_status get_tallies(const hww_problem* p, int32_t kind, double* out, int64_t n, int32_t on_device) {
    if (!p || !out || kind < 0 || kind > HWW_CLOSURE_F) return HWW_ERR_ARG;
    if (p->steps < 1) return HWW_ERR_STATE;
    HWW_CK(cudaSetDevice(p->device));
    const int I = p->I, B = p->B;
    const Acc128* src = nullptr;
    int len = I;
    switch (kind) {
    case HWW_TL_PHI: src = p->tl; break;
    case HWW_TL_J: src = p->tl + I; break;
    case HWW_TL_F: src = p->tl + 2 * I; break;
    case HWW_CENSUS_PHI: src = p->cent; break;
    case HWW_CENSUS_J: src = p->cent + I; break;
    case HWW_CENSUS_F: src = p->cent + 2 * I; break;
    case HWW_BATCH_PHI: src = p->batch; len = B * I; break;
    case HWW_BOUNDARY: src = p->bnd; len = 6; break;
    case HWW_WW_CENTER: return n < I ? HWW_ERR_ARG : copy_out(p, out, p->ww_c, I, on_device);
    case HWW_CLOSURE_PHI: return n < I + 2 ? HWW_ERR_ARG : copy_out(p, out, p->cl_phi[p->cur], I + 2, on_device);
    case HWW_CLOSURE_J: return n < I + 1 ? HWW_ERR_ARG : copy_out(p, out, p->cl_J[p->cur], I + 1, on_device);
    case HWW_CLOSURE_F: return n < I + 2 ? HWW_ERR_ARG : copy_out(p, out, p->cl_F[p->cur], I + 2, on_device);
    }
    if (n < len) return HWW_ERR_ARG;
    normalize_kernel<<<(len + 255) / 256, 256, 0, p->stream>>>(kind, src, len, I, B, p->N, p->d_dx, p->d.v,
                                                                p->d.dt, p->sd, p->norm);
    HWW_CK(cudaGetLastError());
    return copy_out(p, out, p->norm, len, on_device);
}

hww_status get_tallies_raw(const hww_problem* p, int32_t kind, int64_t* out, int64_t n) {
    if (!p || !out || kind < 0 || kind > HWW_BOUNDARY) return HWW_ERR_ARG;
    if (p->steps < 1) return HWW_ERR_STATE;
    HWW_CK(cudaSetDevice(p->device));
    const int I = p->I, B = p->B;
    const Acc128* src = nullptr;
    long long len = I;
    switch (kind) {
    case HWW_TL_PHI: src = p->tl; break;
    case HWW_TL_J: src = p->tl + I; break;
    case HWW_TL_F: src = p->tl + 2 * I; break;
    case HWW_CENSUS_PHI: src = p->cent; break;
    case HWW_CENSUS_J: src = p->cent + I; break;
    case HWW_CENSUS_F: src = p->cent + 2 * I; break;
    case HWW_BATCH_PHI: src = p->batch; len = (long long)B * I; break;
    case HWW_BOUNDARY: src = p->bnd; len = 6; break;
    }
    if (n < 2 * len) return HWW_ERR_ARG;
    // the device keeps split sums; report the exact 128-bit values
    std::vector<Acc128> h(len);
    HWW_CK(cudaMemcpyAsync(h.data(), src, sizeof(Acc128) * len, cudaMemcpyDeviceToHost, p->stream));
    HWW_CK(cudaStreamSynchronize(p->stream));
    for (long long i = 0; i < len; ++i) {
        const I128 v = acc_value(h[i]);
        out[2 * i] = (int64_t)v.lo;
        out[2 * i + 1] = (int64_t)v.hi;
    }
    return HWW_OK;
}

hww_status get_losm_solution(const hww_problem* p, int32_t which, double* phi, double* J, int32_t on_device) {
    if (!p || !phi || !J || which < 0 || which > 1) return HWW_ERR_ARG;
    if (p->steps < 1) return HWW_ERR_STATE;
    HWW_CK(cudaSetDevice(p->device));
    hww_status s = copy_out(p, phi, which ? p->full_phi : p->semi_phi, p->I + 2, on_device);
    if (s) return s;
    return copy_out(p, J, which ? p->full_J : p->semi_J, p->I + 1, on_device);
}

hww_status get_deriv_tallies(const hww_problem* p, int32_t which, double* out, int64_t n, int32_t on_device) {
    if (!p || !out || which < 0 || which > 4) return HWW_ERR_ARG;
    if (p->P2 < 1 || p->steps < 1) return HWW_ERR_STATE;
    const int64_t need = (which == 4) ? 6LL * p->P2 : (int64_t)p->P2 * p->I;
    if (n < need) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(p->device));
    // host output: staged through the adjoint's state block (larger than
    // [P2][I]; it is refilled whenever the adjoint runs on the last step)
    double* dst = on_device ? out : p->vjp_state;
    launch_deriv_normalize(p, which, dst);
    HWW_CK(cudaGetLastError());
    if (!on_device) {
        HWW_CK(cudaMemcpyAsync(out, dst, sizeof(double) * need, cudaMemcpyDeviceToHost, p->stream));
        HWW_CK(cudaStreamSynchronize(p->stream));
    }
    return HWW_OK;
}

hww_status vjp_state_size(const hww_problem* p, int64_t* n) {
    if (!p || !n) return HWW_ERR_ARG;
    if (p->P2 < 1) return HWW_ERR_STATE;
    *n = vjp_layout(p->I, p->P2).total;
    return HWW_OK;
}

hww_status save_vjp_state(hww_problem* p, double* state, int64_t n, int32_t on_device) {
    if (!p || !state) return HWW_ERR_ARG;
    if (p->P2 < 1 || p->steps < 1) return HWW_ERR_STATE;
    const VjpLayout L = vjp_layout(p->I, p->P2);
    if (n < L.total) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(p->device));
    hww_status s = fill_vjp_state(p);
    if (s) return s;
    HWW_CK(cudaMemcpyAsync(state, p->vjp_state, sizeof(double) * L.total,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
    if (!on_device) HWW_CK(cudaStreamSynchronize(p->stream));
    return HWW_OK;
}

hww_status losm_vjp(hww_problem* p, const double* state, const double* g_mc, const double* g_phi,
                    const double* g_J, double* grad, int32_t on_device) {
    if (!p || !grad) return HWW_ERR_ARG;
    if (p->P2 < 1 || p->steps < 1) return HWW_ERR_STATE;
    HWW_CK(cudaSetDevice(p->device));
    const int I = p->I, P2 = p->P2;
    const VjpLayout L = vjp_layout(I, P2);
    const double* st = p->vjp_state;
    hww_status s = HWW_OK;
    if (!state) {
        if ((s = fill_vjp_state(p))) return s;
    } else {
        double hdr[4];
        if (on_device) {
            HWW_CK(cudaMemcpyAsync(hdr, state, sizeof(hdr), cudaMemcpyDeviceToHost, p->stream));
            HWW_CK(cudaStreamSynchronize(p->stream));
            st = state;
        } else {
            std::memcpy(hdr, state, sizeof(hdr));
            HWW_CK(cudaMemcpyAsync(p->vjp_state, state, sizeof(double) * L.total, cudaMemcpyHostToDevice,
                                   p->stream));
        }
        // the state must come from this problem, with its current cross sections
        if (hdr[0] != (double)I || hdr[1] != (double)P2) return HWW_ERR_ARG;
        if (hdr[2] != (double)p->xs_version) return HWW_ERR_STATE;
    }
    double* w = p->vjp_work;  // laid out as vjp_work_doubles counts
    double *psi = w, *z = w + (I + 2), *wmc = w + 2 * (I + 2), *wphi = wmc + I, *wJ = wphi + (I + 2),
           *wgrad = wJ + (I + 1);
    VjpArgs a{};
    a.m = p->mat;
    a.dx = p->d_dx;
    a.sigt = p->d_sigt;
    a.c = p->d_c;
    a.region = p->d_region;
    a.R = p->R;
    a.P2 = P2;
    a.state = st;
    a.psi = psi;
    a.z = z;
    // upstream vectors: used in place on the device, else staged; NULL is zero
    cudaError_t e = cudaSuccess;
    auto stage = [&](const double* src, double* dst, size_t n) -> const double* {
        if (!src) {
            if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, n * sizeof(double), p->stream);
            return dst;
        }
        if (on_device) return src;
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, p->stream);
        return dst;
    };
    a.g_mc = g_mc ? stage(g_mc, wmc, I) : nullptr;
    a.g_phi = stage(g_phi, wphi, I + 2);
    a.g_J = stage(g_J, wJ, I + 1);
    HWW_CK(e);
    a.grad = on_device ? grad : wgrad;
    HWW_CK(cudaPeekAtLastError());
    p->kernel_launches += launch_losm_vjp(a, p->stream);
    HWW_CK(cudaGetLastError());
    if (!on_device) {
        HWW_CK(cudaMemcpyAsync(grad, wgrad, sizeof(double) * P2, cudaMemcpyDeviceToHost, p->stream));
        HWW_CK(cudaStreamSynchronize(p->stream));
    }
    return HWW_OK;
}

hww_status get_bank(const hww_problem* p, double* x, double* mu, int32_t* cell, int64_t cap, int64_t* n) {
    if (!p || !n) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(p->device));
    StepDev sdh;
    HWW_CK(cudaMemcpyAsync(&sdh, p->sd, sizeof(StepDev), cudaMemcpyDeviceToHost, p->stream));
    HWW_CK(cudaStreamSynchronize(p->stream));
    const long long m = (p->steps < 1) ? 0 : (long long)sdh.nbank;
    *n = m;
    if (cap == 0 || m == 0) return HWW_OK;
    if (cap < m) return HWW_ERR_ARG;
    double* tmp = nullptr;
    HWW_CK(cudaMallocAsync(&tmp, sizeof(double) * m, p->stream));
    cudaError_t e = cudaSuccess;
    const int grid = p->nsm * 4;
    auto field = [&](int f) {
        if (p->fp32)
            bank_field_kernel<float><<<grid, 256, 0, p->stream>>>(p->b32.bank, p->d_edges, m, f, tmp);
        else
            bank_field_kernel<double><<<grid, 256, 0, p->stream>>>(p->b64.bank, p->d_edges, m, f, tmp);
    };
    if (x) {
        field(0);
        e = cudaMemcpyAsync(x, tmp, sizeof(double) * m, cudaMemcpyDeviceToHost, p->stream);
    }
    if (mu && e == cudaSuccess) {  // stream order: after the copy of x
        field(1);
        e = cudaMemcpyAsync(mu, tmp, sizeof(double) * m, cudaMemcpyDeviceToHost, p->stream);
    }
    if (cell && e == cudaSuccess) {
        field(2);
        e = cudaMemcpyAsync(cell, tmp, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, p->stream);
    }
    cudaFreeAsync(tmp, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return cuda_status(e);
}

hww_status hww_set_tracking(hww_problem* p, int32_t kind) {
    if (!p || (kind != HWW_TRACK_WARP && kind != HWW_TRACK_EVENT && kind != HWW_TRACK_AUTO)) return HWW_ERR_ARG;
    if (kind != HWW_TRACK_WARP) {
        if (!p->fp32) return HWW_ERR_ARG;
        HWW_CK(cudaSetDevice(p->device));
        const EvShape sh = ev_shape(p->I);
        if (sh.blocks_per_sm == 0) {
            if (kind == HWW_TRACK_EVENT) return HWW_ERR_ARG;
            p->ev = sh;  // HWW_TRACK_AUTO: the warp loop
        } else {
            if (track_event_smem_optin_fp32(p->I, sh.cap) != 0) return HWW_ERR_CUDA;
            p->ev = sh;
        }
    }
    p->track_kind = kind;
    return HWW_OK;
}

hww_status hww_set_timing(hww_problem* p, int32_t enable) {
    if (!p || enable < 0 || enable > 1) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(p->device));
    if (enable && !p->ev_a) {
        HWW_CK(cudaEventCreate(&p->ev_a));
        HWW_CK(cudaEventCreate(&p->ev_b));
    }
    p->timing = enable;
    return HWW_OK;
}

hww_status hww_get_counters(const hww_problem* p, hww_counters* out) {
    if (!p || !out) return HWW_ERR_ARG;
    out->kernel_launches = p->kernel_launches;
    out->track_launches = p->track_launches;
    out->event_launches = p->event_launches;
    out->spilled = p->spilled;
    out->track_ms = p->track_ms;
    out->steps = p->steps;
    out->census_capacity = p->cen_cap;
    out->queue_capacity = p->q_cap;
    return HWW_OK;
}

hww_status hww_reset_counters(hww_problem* p) {
    if (!p) return HWW_ERR_ARG;
    p->kernel_launches = 0;
    p->track_launches = 0;
    p->event_launches = 0;
    p->spilled = 0;
    p->track_ms = 0.0;
    HWW_CK(cudaSetDevice(p->device));
    HWW_CK(cudaMemsetAsync(p->spill_n, 0, sizeof(unsigned long long), p->stream));
    return HWW_OK;
}

hww_status set_bank(hww_problem* p, const double* x, const double* mu, const int32_t* cell, int64_t n,
                    double w_bar) {
    if (!p || n < 0 || n > p->N || (n > 0 && (!x || !mu || !cell)) || !(w_bar > 0.0) || !std::isfinite(w_bar))
        return HWW_ERR_ARG;
    for (int64_t k = 0; k < n; ++k) {
        const int c = cell[k];
        if (c < 0 || c >= p->I || !(mu[k] != 0.0) || !(mu[k] >= -1.0 && mu[k] <= 1.0) ||
            !(x[k] >= p->edges[c] && x[k] <= p->edges[c + 1]))
            return HWW_ERR_ARG;
    }
    HWW_CK(cudaSetDevice(p->device));
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        if (p->fp32) {
            std::vector<BankRec<float>> r(n);
            for (int64_t k = 0; k < n; ++k) {
                r[k].x = (float)(x[k] - p->edges[cell[k]]);
                r[k].mu = (float)mu[k];
                r[k].cell = cell[k];
                r[k].pad = 0;
            }
            e = cudaMemcpy(p->b32.bank, r.data(), sizeof(BankRec<float>) * n, cudaMemcpyHostToDevice);
        } else {
            std::vector<BankRec<double>> r(n);
            for (int64_t k = 0; k < n; ++k) {
                r[k] = BankRec<double>{};
                r[k].x = x[k];
                r[k].mu = mu[k];
                r[k].imu = 1.0 / mu[k];
                r[k].cell = cell[k];
            }
            e = cudaMemcpy(p->b64.bank, r.data(), sizeof(BankRec<double>) * n, cudaMemcpyHostToDevice);
        }
    }
    StepDev sdh;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sdh, p->sd, sizeof(StepDev), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (p->P2 > 0 && n > 0)  // a loaded bank starts with zero scores
        HWW_CK(cudaMemsetAsync(p->bS, 0, sizeof(double) * (size_t)p->P2 * p->N, p->stream));
    sdh.nbank = (unsigned long long)n;
    sdh.wbar = w_bar;
    sdh.bank_loaded = 1;
    HWW_CK(cudaMemcpyAsync(p->sd, &sdh, sizeof(StepDev), cudaMemcpyHostToDevice, p->stream));
    HWW_CK(cudaStreamSynchronize(p->stream));
    return HWW_OK;
}

hww_status get_census(const hww_problem* p, double* x, double* mu, double* w, int32_t* cell, uint32_t* id,
                      uint64_t* lin, int64_t cap, int64_t* n) {
    if (!p || !n) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(p->device));
    StepDev sdh;
    HWW_CK(cudaMemcpyAsync(&sdh, p->sd, sizeof(StepDev), cudaMemcpyDeviceToHost, p->stream));
    HWW_CK(cudaStreamSynchronize(p->stream));
    long long m = (p->steps < 1) ? 0 : (long long)sdh.ncensus;
    if (m > p->cen_cap) m = p->cen_cap;
    *n = m;
    if (cap == 0 || m == 0) return HWW_OK;
    if (cap < m) return HWW_ERR_ARG;
    double* tmp = nullptr;
    HWW_CK(cudaMallocAsync(&tmp, sizeof(double) * m, p->stream));
    cudaError_t e = cudaSuccess;
    const int grid = p->nsm * 4;
    if (x) {
        if (p->fp32)
            bank_to_x_kernel<float><<<grid, 256, 0, p->stream>>>(p->b32.cen.x, p->b32.cen.cell, p->d_edges, m, tmp);
        else
            bank_to_x_kernel<double><<<grid, 256, 0, p->stream>>>(p->b64.cen.x, p->b64.cen.cell, p->d_edges, m, tmp);
        e = cudaMemcpyAsync(x, tmp, sizeof(double) * m, cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    }
    if (mu && e == cudaSuccess) {
        if (p->fp32)
            to_double_kernel<float><<<grid, 256, 0, p->stream>>>(p->b32.cen.mu, m, tmp);
        else
            to_double_kernel<double><<<grid, 256, 0, p->stream>>>(p->b64.cen.mu, m, tmp);
        e = cudaMemcpyAsync(mu, tmp, sizeof(double) * m, cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    }
    if (w && e == cudaSuccess)
        e = cudaMemcpyAsync(w, p->fp32 ? p->b32.cen.w : p->b64.cen.w, sizeof(double) * m, cudaMemcpyDeviceToHost,
                            p->stream);
    if (cell && e == cudaSuccess)
        e = cudaMemcpyAsync(cell, p->fp32 ? p->b32.cen.cell : p->b64.cen.cell, sizeof(int32_t) * m,
                            cudaMemcpyDeviceToHost, p->stream);
    if (id && e == cudaSuccess)
        e = cudaMemcpyAsync(id, p->fp32 ? p->b32.cen.id : p->b64.cen.id, sizeof(uint32_t) * m,
                            cudaMemcpyDeviceToHost, p->stream);
    if (lin && e == cudaSuccess)
        e = cudaMemcpy2DAsync(lin, sizeof(uint64_t), p->fp32 ? (const void*)p->b32.cen.lw : (const void*)p->b64.cen.lw,
                              sizeof(LinW), sizeof(uint64_t), (size_t)m, cudaMemcpyDeviceToHost, p->stream);
    cudaFreeAsync(tmp, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return cuda_status(e);
}

hww_status hww_losm_solve(int32_t I, const double* dx, const double* sigma_t, const double* sigma_a, double v,
                          double dt, double theta, int32_t bc_left, int32_t bc_right, const double* phi_old,
                          const double* J_old, const double* F_old, const double* F_new, double PL_new,
                          double PR_new, const double* q_old, const double* q_new, double* phi_new,
                          double* J_new) {
    if (I < 1 || !dx || !sigma_t || !sigma_a || !phi_old || !J_old || !F_old || !F_new || !phi_new || !J_new ||
        !(v > 0) || !(dt > 0) || (theta != 0.5 && theta != 1.0) || bc_left < 0 || bc_left > 1 || bc_right < 0 ||
        bc_right > 1)
        return HWW_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return HWW_ERR_NO_DEVICE;
    double* buf = nullptr;
    HWW_CK(cudaMalloc(&buf, losm_staged_doubles((size_t)I) * sizeof(double)));
    bool numeric = false;
    const cudaError_t e = losm_solve_staged(buf, I, dx, sigma_t, sigma_a, v, dt, theta, bc_left, bc_right, phi_old,
                                            J_old, F_old, F_new, PL_new, PR_new, q_old, q_new, phi_new, J_new,
                                            &numeric);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_status(e);
    return numeric ? HWW_ERR_NUMERIC : HWW_OK;
}

hww_status hww_philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                            int64_t n, uint32_t* out) {
    if (n < 0 || (n > 0 && !out) || n > (1LL << 28)) return HWW_ERR_ARG;
    if (n == 0) return HWW_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return HWW_ERR_NO_DEVICE;
    uint32_t* d = nullptr;
    HWW_CK(cudaMalloc(&d, sizeof(uint32_t) * 4 * n));
    launch_philox_block(c0, c1, c2, c3, k0, k1, n, d, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
struct hww_batch {
    int P = 0, device = 0, fp32 = 0;
    cudaStream_t user = nullptr;   // the caller's stream
    cudaStream_t stream = nullptr; // the batch's own stream (graphs are captured and run on it)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<hww_problem*> m;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t pre = nullptr, post = nullptr;
    int tile = 4096, emax = 64;
    int grid = 0;
    size_t smem = 0;
    void* d_args[3] = {};          // TrackArgs per member: wave 0, odd waves, even waves
    long long* d_tile_off = nullptr;
    unsigned long long* d_head = nullptr;
    unsigned long long* d_total = nullptr;
    unsigned* d_errs = nullptr;
    unsigned long long* d_qpeak = nullptr;  // per member: largest record count of a wave
    unsigned long long* d_ncen = nullptr;   // per member: census count after the last wave
    unsigned long long* h_ncen = nullptr;   // pinned
    unsigned long long* h_total = nullptr;  // pinned
    unsigned* h_errs = nullptr;             // pinned
    unsigned long long* h_qpeak = nullptr;  // pinned
    // every member's step statistics gathered by one kernel: per member
    // ST_COUNT counters, start-bank size, weight bits, error word
    unsigned long long* d_gather = nullptr;
    unsigned long long* h_gather = nullptr;  // pinned
    int gathered = 0;                        // h_gather holds the last step
    int last_waves = 0;
    int step_replays = 0;                    // members tracked again alone after an overflow (last step)
    int step_grows = 0;                      // members grown ahead of demand (last step)
};

namespace {

template <class Real>
__global__ void batch_plan_kernel(const TrackArgs<Real>* args, int P, int tile, long long* tile_off,
                                  unsigned long long* head) {
    __shared__ long long cnt[1024];
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const TrackArgs<Real>& a = args[p];
        const long long n_in = a.from_bank ? (long long)a.sd->nbank : (long long)*a.rin.count;
        const long long n_use = (!a.from_bank && n_in > a.rin.cap) ? a.rin.cap : n_in;
        cnt[p] = (n_use + tile - 1) / tile;
        if (!a.from_bank) *a.rout.count = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int p = 0; p < P; ++p) {
            tile_off[p] = acc;
            acc += cnt[p];
        }
        tile_off[P] = acc;
        *head = 0;
    }
}

template <class Real>
__global__ void batch_total_kernel(const TrackArgs<Real>* args, int P, unsigned long long* total, unsigned* errs,
                                   unsigned long long* qpeak, unsigned long long* ncen) {
    __shared__ unsigned long long s[256];
    unsigned long long acc = 0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const unsigned long long c = *args[p].rout.count;
        acc += c;
        errs[p] = *args[p].err;
        if (c > qpeak[p]) qpeak[p] = c;
        ncen[p] = *args[p].cen.count;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s[0];
}

constexpr int GATHER = ST_COUNT + 3;

// gather the members' statistics of the step and clear their error words
// (each step reports its errors once, as read_stats does)
template <class Real>
__global__ void batch_gather_kernel(const TrackArgs<Real>* args, int P, unsigned long long* out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P * GATHER; t += gridDim.x * blockDim.x) {
        const int p = t / GATHER, k = t % GATHER;
        const TrackArgs<Real>& a = args[p];
        unsigned long long v;
        if (k < ST_COUNT)
            v = a.stats[k];
        else if (k == ST_COUNT)
            v = a.sd->nbank;
        else if (k == ST_COUNT + 1)
            v = (unsigned long long)__double_as_longlong(a.sd->wbar);
        else {
            v = *a.err;  // read and cleared by this thread only
            *a.err = 0;
        }
        out[t] = v;
    }
}

template <class Real>
Banks<Real>& banks_of(hww_problem* p);
template <>
Banks<double>& banks_of<double>(hww_problem* p) { return p->b64; }
template <>
Banks<float>& banks_of<float>(hww_problem* p) { return p->b32; }

// per-member tracking arguments of wave 0, odd and even waves
template <class Real>
hww_status upload_batch_args(hww_batch* b) {
    std::vector<TrackArgs<Real>> a[3];
    for (int k = 0; k < 3; ++k) a[k].resize(b->P);
    for (int i = 0; i < b->P; ++i) {
        hww_problem* p = b->m[i];
        p->emax = b->emax;
        Banks<Real>& bk = banks_of<Real>(p);
        TrackArgs<Real> t = base_track_args(p, bk);
        a[0][i] = t;
        a[0][i].from_bank = 1;
        a[0][i].rin = bk.q[1];
        a[0][i].rout = bk.q[0];
        a[1][i] = t;
        a[1][i].from_bank = 0;
        a[1][i].rin = bk.q[0];
        a[1][i].rout = bk.q[1];
        a[2][i] = t;
        a[2][i].from_bank = 0;
        a[2][i].rin = bk.q[1];
        a[2][i].rout = bk.q[0];
    }
    for (int k = 0; k < 3; ++k)
        HWW_CK(cudaMemcpyAsync(b->d_args[k], a[k].data(), sizeof(TrackArgs<Real>) * b->P, cudaMemcpyHostToDevice,
                               b->stream));
    HWW_CK(cudaStreamSynchronize(b->stream));
    return HWW_OK;
}

hww_status upload_batch_args(hww_batch* b) {
    return b->fp32 ? upload_batch_args<float>(b) : upload_batch_args<double>(b);
}

// record one stage of every member as parallel branches of a graph
hww_status capture_stage(hww_batch* b, int pre, cudaGraphExec_t* exec) {
    if (*exec) {
        cudaGraphExecDestroy(*exec);
        *exec = nullptr;
    }
    HWW_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaEventRecord(b->fork, b->stream);
    for (cudaStream_t s : b->pool) cudaStreamWaitEvent(s, b->fork, 0);
    hww_status st = HWW_OK;
    for (hww_problem* p : b->m) {
        st = pre ? stage_pre(p) : stage_post(p);
        if (st) break;
    }
    for (size_t k = 0; k < b->pool.size(); ++k) {
        cudaEventRecord(b->join[k], b->pool[k]);
        cudaStreamWaitEvent(b->stream, b->join[k], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (st || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st ? st : cuda_status(e);
    }
    const cudaError_t e2 = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return cuda_status(e2);
}

template <class Real>
hww_status batch_waves(hww_batch* b) {
    int waves = 0;
    HWW_CK(cudaMemsetAsync(b->d_qpeak, 0, sizeof(unsigned long long) * b->P, b->stream));
    for (int wave = 0;; ++wave) {
        const int k = (wave == 0) ? 0 : (wave % 2 == 1 ? 1 : 2);
        const TrackArgs<Real>* args = (const TrackArgs<Real>*)b->d_args[k];
        batch_plan_kernel<Real><<<1, 256, 0, b->stream>>>(args, b->P, b->tile, b->d_tile_off, b->d_head);
        BatchPlan plan{b->d_tile_off, b->P, b->tile, b->d_head};
        if (b->fp32)
            launch_track_batch_fp32((const TrackArgs<float>*)args, plan, b->grid, TRACK_BLOCK, b->smem, b->stream);
        else
            launch_track_batch_fp64((const TrackArgs<double>*)args, plan, b->grid, TRACK_BLOCK, b->smem, b->stream);
        batch_total_kernel<Real><<<1, 256, 0, b->stream>>>(args, b->P, b->d_total, b->d_errs, b->d_qpeak,
                                                           b->d_ncen);
        HWW_CK(cudaGetLastError());
        ++waves;
        HWW_CK(cudaMemcpyAsync(b->h_total, b->d_total, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               b->stream));
        HWW_CK(cudaStreamSynchronize(b->stream));
        if (*b->h_total == 0) break;
        if (waves >= MAX_WAVES) return HWW_ERR_TIMEOUT;
    }
    b->last_waves = waves;
    return HWW_OK;
}

}  // namespace

extern "C" {

void destroy_batch(hww_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->pre) cudaGraphExecDestroy(b->pre);
    if (b->post) cudaGraphExecDestroy(b->post);
    for (hww_problem* p : b->m) destroy_problem(p);
    for (int k = 0; k < 3; ++k)
        if (b->d_args[k]) cudaFree(b->d_args[k]);
    if (b->d_tile_off) cudaFree(b->d_tile_off);
    if (b->d_head) cudaFree(b->d_head);
    if (b->d_total) cudaFree(b->d_total);
    if (b->d_errs) cudaFree(b->d_errs);
    if (b->d_qpeak) cudaFree(b->d_qpeak);
    if (b->d_ncen) cudaFree(b->d_ncen);
    if (b->h_ncen) cudaFreeHost(b->h_ncen);
    if (b->d_gather) cudaFree(b->d_gather);
    if (b->h_gather) cudaFreeHost(b->h_gather);
    if (b->h_qpeak) cudaFreeHost(b->h_qpeak);
    if (b->h_total) cudaFreeHost(b->h_total);
    if (b->h_errs) cudaFreeHost(b->h_errs);
    for (cudaStream_t s : b->pool) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

hww_status create_batch(const hww_problem_desc* descs, int32_t n, void* cuda_stream, int32_t device,
                        hww_batch** out) {
    if (!out) return HWW_ERR_ARG;
    *out = nullptr;
    if (!descs || n < 1 || n > 1024) return HWW_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (descs[i].precision != descs[0].precision || descs[i].deriv_regions != 0) return HWW_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return HWW_ERR_NO_DEVICE;
    if (device < 0 || device >= ndev) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(device));
    hww_batch* b = new (std::nothrow) hww_batch();
    if (!b) return HWW_ERR_OOM;
    b->P = n;
    b->device = device;
    b->fp32 = descs[0].precision == HWW_FP32_TRACK;
    b->user = (cudaStream_t)cuda_stream;
    const int K = std::min(n, 32);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->pool.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(ev);
    }
    if (e != cudaSuccess) {
        destroy_batch(b);
        return cuda_status(e);
    }
    int Imax = 0;
    for (int i = 0; i < n; ++i) {
        hww_problem_desc d = descs[i];
        d.cuda_stream = (void*)b->pool[i % K];
        d.device = device;
        hww_problem* p = nullptr;
        const hww_status s = create_problem(&d, &p);
        if (s) {
            destroy_batch(b);
            return s;
        }
        b->m.push_back(p);
        Imax = std::max(Imax, p->I);
    }
    b->smem = sizeof(long long) * (b->fp32 ? TALLY_ROWS_FP32 : TALLY_ROWS) * (size_t)Imax;
    if (track_batch_smem_optin(b->fp32, b->smem) != 0) {  // static shared memory counts too
        destroy_batch(b);
        return HWW_ERR_CUDA;
    }
    int per_sm = track_batch_blocks_per_sm(b->fp32, TRACK_BLOCK, b->smem);
    if (per_sm < 1) per_sm = 1;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    b->grid = nsm * per_sm;
    const size_t asz = b->fp32 ? sizeof(TrackArgs<float>) : sizeof(TrackArgs<double>);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&b->d_args[k], asz * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tile_off, sizeof(long long) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_head, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_total, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_errs, sizeof(unsigned) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_qpeak, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_qpeak, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ncen, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_ncen, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_gather, sizeof(unsigned long long) * GATHER * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_gather, sizeof(unsigned long long) * GATHER * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_total, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_errs, sizeof(unsigned) * n);
    if (e != cudaSuccess) {
        destroy_batch(b);
        return cuda_status(e);
    }
    const hww_status s = upload_batch_args(b);
    if (s) {
        destroy_batch(b);
        return s;
    }
    *out = b;
    return HWW_OK;
}

hww_status batch_problem(hww_batch* b, int32_t i, hww_problem** out) {
    if (!b || !out || i < 0 || i >= b->P) return HWW_ERR_ARG;
    *out = b->m[i];
    return HWW_OK;
}

hww_status batch_set_tuning(hww_batch* b, int32_t tile, int32_t emax) {
    if (!b || tile < 256 || emax < 1) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(b->device));
    b->tile = tile;
    b->emax = emax;
    return upload_batch_args(b);
}

hww_status run_batch_step(hww_batch* b, hww_batch_stats* stats) {
    if (!b) return HWW_ERR_ARG;
    for (hww_problem* p : b->m)
        if (!p->xs_set || !p->ww_set || p->n_updates > 0) return HWW_ERR_STATE;
    HWW_CK(cudaSetDevice(b->device));
    // order the batch's own stream after the caller's work
    HWW_CK(cudaEventRecord(b->ev_in, b->user));
    HWW_CK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    hww_status s = HWW_OK;
    if (!b->pre && (s = capture_stage(b, 1, &b->pre))) return s;
    if (!b->post && (s = capture_stage(b, 0, &b->post))) return s;
    HWW_CK(cudaGraphLaunch(b->pre, b->stream));
    s = b->fp32 ? batch_waves<float>(b) : batch_waves<double>(b);
    if (s) return s;
    HWW_CK(cudaMemcpyAsync(b->h_errs, b->d_errs, sizeof(unsigned) * b->P, cudaMemcpyDeviceToHost, b->stream));
    HWW_CK(cudaMemcpyAsync(b->h_qpeak, b->d_qpeak, sizeof(unsigned long long) * b->P, cudaMemcpyDeviceToHost,
                           b->stream));
    HWW_CK(cudaMemcpyAsync(b->h_ncen, b->d_ncen, sizeof(unsigned long long) * b->P, cudaMemcpyDeviceToHost,
                           b->stream));
    HWW_CK(cudaStreamSynchronize(b->stream));
    // A member whose census bank or record queue overflowed is tracked again
    // on its own, through the single-problem path (same per-track arithmetic,
    // so the same result as a batch that had the room); the other members'
    // tracking stands.  Members that came near their capacities grow after
    // the comb (which still reads this step's census bank).
    bool rebuilt = false;
    std::vector<int> grow;
    b->step_replays = 0;
    b->step_grows = 0;
    for (int i = 0; i < b->P; ++i) {
        hww_problem* p = b->m[i];
        const unsigned e = b->h_errs[i];
        if (e & (ERR_CENSUS_OVERFLOW | ERR_QUEUE_OVERFLOW)) {
            s = regrow_banks(p, (long long)b->h_ncen[i], (long long)b->h_qpeak[i]);
            if (s) return s;
            const unsigned keep = e & ~(unsigned)(ERR_CENSUS_OVERFLOW | ERR_QUEUE_OVERFLOW);
            HWW_CK(cudaMemcpy(p->err, &keep, sizeof(unsigned), cudaMemcpyHostToDevice));
            s = track_with_regrow(p);
            if (s) return s;
            ++b->step_replays;
            rebuilt = true;
        } else if ((long long)b->h_ncen[i] * 5 > p->cen_cap * 3 || (long long)b->h_qpeak[i] * 5 > p->q_cap * 3) {
            grow.push_back(i);
        }
    }
    // the comb and the tracking arguments refer to the regrown buffers
    if (rebuilt && ((s = upload_batch_args(b)) || (s = capture_stage(b, 0, &b->post)))) return s;
    HWW_CK(cudaGraphLaunch(b->post, b->stream));
    if (!grow.empty()) {
        // twice the capacity (at least) for the members that came within 60%
        // of it, once the comb has read their census banks
        HWW_CK(cudaStreamSynchronize(b->stream));
        for (int i : grow) {
            s = regrow_banks(b->m[i], (long long)b->h_ncen[i], (long long)b->h_qpeak[i]);
            if (s) return s;
            ++b->step_grows;
        }
        if ((s = upload_batch_args(b)) || (s = capture_stage(b, 0, &b->post))) return s;
    }
    // and the caller's stream after the batch step
    HWW_CK(cudaEventRecord(b->ev_out, b->stream));
    HWW_CK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    for (hww_problem* p : b->m) {
        p->cur ^= 1;
        p->steps += 1;
        p->last_waves = b->last_waves;
    }
    b->gathered = 0;
    if (!stats) return HWW_OK;
    // one gather kernel and one copy for all members' statistics
    if (b->fp32)
        batch_gather_kernel<float><<<(b->P * GATHER + 255) / 256, 256, 0, b->stream>>>(
            (const TrackArgs<float>*)b->d_args[0], b->P, b->d_gather);
    else
        batch_gather_kernel<double><<<(b->P * GATHER + 255) / 256, 256, 0, b->stream>>>(
            (const TrackArgs<double>*)b->d_args[0], b->P, b->d_gather);
    HWW_CK(cudaGetLastError());
    HWW_CK(cudaMemcpyAsync(b->h_gather, b->d_gather, sizeof(unsigned long long) * GATHER * b->P,
                           cudaMemcpyDeviceToHost, b->stream));
    HWW_CK(cudaStreamSynchronize(b->stream));
    b->gathered = 1;
    std::memset(stats, 0, sizeof(*stats));
    stats->problems = b->P;
    stats->waves = b->last_waves;
    stats->member_replays = b->step_replays;
    stats->member_grows = b->step_grows;
    for (int i = 0; i < b->P; ++i) {
        const unsigned long long* g = b->h_gather + (size_t)i * GATHER;
        hww_step_stats ms;
        fill_stats(g, g[ST_COUNT], bits_to_double(g[ST_COUNT + 1]), (unsigned)g[ST_COUNT + 2],
                   b->last_waves, &ms);
        const hww_status r = (hww_status)ms.status;
        stats->segments += ms.segments;
        stats->census += ms.census;
        stats->daughters += ms.daughters;
        stats->roulette_kills += ms.roulette_kills;
        stats->absorbed += ms.absorbed;
        stats->leaked += ms.leaked;
        if (r && !stats->status) stats->status = r;
    }
    return (hww_status)stats->status;
}

hww_status batch_member_stats(hww_batch* b, int32_t i, hww_step_stats* stats) {
    if (!b || !stats || i < 0 || i >= b->P) return HWW_ERR_ARG;
    HWW_CK(cudaSetDevice(b->device));
    HWW_CK(cudaStreamSynchronize(b->stream));
    if (b->gathered) {
        // the statistics gathered at the end of the step (errors already reported there)
        const unsigned long long* g = b->h_gather + (size_t)i * GATHER;
        fill_stats(g, g[ST_COUNT], bits_to_double(g[ST_COUNT + 1]), (unsigned)g[ST_COUNT + 2],
                   b->last_waves, stats);
        return (hww_status)stats->status;
    }
    return read_stats(b->m[i], stats);
}

}  // extern "C"

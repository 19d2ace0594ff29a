// track_fp64.cu -- FP64 tracking kernel: one event-loop pass over a set of
// tracks of one time step (paper Secs. 2-3).
//
// Built with contraction off (-fmad=false): every floating-point operation
// is the single IEEE double operation written, so a track takes exactly the
// events, splits and roulette outcomes the numerics contract defines.
//
// Per event (Eq. HO_transport physics, one speed, isotropic scattering):
//   flight   d_coll = -log(u_f) / Sigma_t   (as  -log(u_f) * (1/Sigma_t))
//   edge     d_edge = (x_edge - x) / mu     (as  (x_edge - x) * (1/mu))
//   census   d_cens = tau, the distance left to t^n
//   the smallest wins, ties in the order census, crossing, collision;
//   track-length tallies of w l, w l mu, w l (1/3 - mu^2) (Eq. phi-mc) and the
//   batch tally w l in batch id mod B;
//   census: time-crossing tallies w, w mu, w (1/3 - mu^2) (Eq. ct-mc) and the
//   comb group of the source id;
//   crossing: next cell, leak through a vacuum side (surface estimators for
//   the boundary closures P_L, P_R), specular reflection on a reflecting side;
//   collision: absorption with probability 1 - c, else a new direction;
//   after a scatter, a cell entry or a reflection the weight window of the
//   cell applies (Sec. 2): split into ceil(w/ww) equal daughters above the
//   ceiling, roulette with survival w/ww below the floor.
// A thread keeps daughter 0 of a split in registers and queues the others
// as chunk records; after `emax` events a live track is queued as a
// continuation record, so long histories are rebalanced between launches.
// The event loop is flattened: a lane whose track ends loads its next track
// while the other lanes take their next event.
//
// Derivative runs (a separate instantiation, DERIV = true) also carry the
// likelihood-ratio scores of (Sigma_t, c) per region: a flight of length l in
// region r adds -l to the Sigma_t score of r and a collision 1/Sigma_t; a
// scatter adds 1/c to the c score of r (an absorption ends the history, so its
// score never reaches a tally).  Each tally gets w l S_j (track length), w S_j,
// w mu S_j, w (1/3 - mu^2) S_j (census) and the surface terms times S_j, with
// the scores after the segment's own flight term.  Daughters, roulette
// survivors, records and census particles keep the scores; the games' own
// probabilities do not depend on the parameters (their centers are held
// fixed), so they add nothing.
#include "track_common.cuh"

namespace hww {
namespace {

struct P64 {
    double x, mu, inv_mu, tau, w;
    int cell;
    uint32_t id;
    uint64_t lin;
    uint32_t e;
};

// The pending parent of a lane (the record whose daughters it expands) and
// its scores, in shared memory, one column per thread: written at a split,
// read once per daughter; registers are what limits the resident warps (the
// derivative loop spilled with the parent in registers).
template <bool DERIV>
struct PendingParent64 {
    double x[TRACK_THREADS], mu[TRACK_THREADS], imu[TRACK_THREADS], tau[TRACK_THREADS], w[TRACK_THREADS];
    int cell[TRACK_THREADS];
    uint32_t id[TRACK_THREADS], e[TRACK_THREADS];
    uint64_t lin[TRACK_THREADS];
    double S[DERIV ? MAX_SCORES : 1][TRACK_THREADS];
    __device__ __forceinline__ void store(int t, const P64& q, const double* sc) {
        x[t] = q.x;
        mu[t] = q.mu;
        imu[t] = q.inv_mu;
        tau[t] = q.tau;
        w[t] = q.w;
        cell[t] = q.cell;
        id[t] = q.id;
        e[t] = q.e;
        lin[t] = q.lin;
        if constexpr (DERIV) {
#pragma unroll
            for (int j = 0; j < MAX_SCORES; ++j) S[j][t] = sc[j];
        }
    }
    __device__ __forceinline__ void load(int t, P64& q, double* sc) const {
        q.x = x[t];
        q.mu = mu[t];
        q.inv_mu = imu[t];
        q.tau = tau[t];
        q.w = w[t];
        q.cell = cell[t];
        q.id = id[t];
        q.e = e[t];
        q.lin = lin[t];
        if constexpr (DERIV) {
#pragma unroll
            for (int j = 0; j < MAX_SCORES; ++j) sc[j] = S[j][t];
        }
    }
};

template <bool DERIV>
__device__ __forceinline__ void push_record(const TrackArgs<double>& a, const P64& q, const double* S, double w,
                                            uint32_t e, uint32_t jstart, uint32_t jcount,
                                            unsigned long long slot) {
    if ((long long)slot >= a.rout.cap) {
        atomicOr(a.err, ERR_QUEUE_OVERFLOW);
        return;
    }
    if constexpr (DERIV) {
#pragma unroll
        for (int j = 0; j < MAX_SCORES; ++j)
            if (j < a.P2) a.rout.S[(long long)j * a.rout.cap + (long long)slot] = S[j];
    }
    a.rout.x[slot] = q.x;
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

// The event loop over items [item, item_end): with the given stride, or, when
// s_next is a block-shared counter, item + the next value of that counter
// (lanes busy with many daughters then take fewer items); b_blk is the
// variance batch whose row is kept in shared memory (-1: none).
// In derivative runs the shared row block after the batch row holds the
// derivative track-length tallies [P2][I].
template <bool DERIV, uint32_t LOCAL_MAX>
__device__ __forceinline__ void run_items(const TrackArgs<double>& a, long long item, const long long item_end,
                                          const long long stride, unsigned* s_next, const int b_blk, long long* sm,
                                          Counters& cnt, PendingParent64<DERIV>* pp) {
    const int I = a.I;
    const int t = threadIdx.x;
    long long* s_tl = sm;
    long long* s_bat = sm + 3 * I;                // batch row of the current id range
    long long* s_dtl = sm + TALLY_ROWS * I;       // derivative runs: [P2][I]
    const int R = a.R, P2 = a.P2;
    double S[DERIV ? MAX_SCORES : 1];     // scores of the current track
    const int S_t = a.sd->S;  // tscale = 2^S_t
    const double wbar = a.sd->wbar;
    const uint32_t k0 = a.sd->k0, k1 = a.sd->k1;
    const int birth = a.sd->birth, ww_on = a.sd->ww_on;
    
    // flattened event loop: a lane whose track ends loads its next one while
    // the other lanes take their next event
    P64 q;
    uint32_t jnext = 0, jend = 0;
    bool fresh = false;  // the record being expanded holds a collision's extra particles
    bool have = false;
    int evs = 0;
    int qb = 0;  // variance batch of the current track's source id
    for (;;) {
        if (!have) {
            if (jnext < jend) {
                pp->load(t, q, S);
                q.lin = lineage_hash(q.lin, q.e, jnext);
                q.e = 0;
                ++jnext;
                if (fresh) {  // its own isotropic direction
                    uint32_t rr[4] = {q.id, (uint32_t)q.lin, (uint32_t)(q.lin >> 32), 0xFFFFFFFEu};
                    philox4x32_10(rr, k0, k1);
                    q.mu = 2.0 * u01(rr[0], rr[1]) - 1.0;
                    q.inv_mu = 1.0 / q.mu;
                }  // else the parent's direction and its reciprocal
            } else {
                long long i;
                if (s_next) {
                    i = item + (long long)warp_reserve(s_next);
                } else {
                    i = item;
                    item += stride;
                }
                if (i >= item_end) break;
                if (a.from_bank) {
                    q.id = (uint32_t)i;
                    q.lin = 0;
                    q.e = 0;
                    q.tau = a.tau0;
                    q.w = wbar;
                    if constexpr (DERIV) {
#pragma unroll
                        for (int j = 0; j < MAX_SCORES; ++j)
                            S[j] = (!birth && j < P2) ? a.bS[(long long)j * a.N + i] : 0.0;
                    }
                    if (birth) {
                        uint32_t r[4] = {(uint32_t)i, 0u, 0u, 0xFFFFFFFFu};
                        philox4x32_10(r, k0, k1);
                        q.mu = 2.0 * u01(r[0], r[1]) - 1.0;
                        q.x = a.src_x;
                        if (q.x <= a.edges[0] && q.mu < 0.0 && a.bc_l == 1) q.mu = -q.mu;
                        if (q.x >= a.edges[I] && q.mu > 0.0 && a.bc_r == 1) q.mu = -q.mu;
                        q.cell = (q.mu < 0.0) ? a.birth_cell_neg : a.birth_cell_pos;
                        q.inv_mu = 1.0 / q.mu;
                    } else {
                        const BankRec<double> r = a.bank[i];
                        q.x = r.x;
                        q.mu = r.mu;
                        q.inv_mu = r.imu;
                        q.cell = r.cell;
                    }
                } else {
                    q.x = a.rin.x[i];
                    q.mu = a.rin.mu[i];
                    q.inv_mu = 1.0 / q.mu;
                    q.tau = a.rin.tau[i];
                    q.w = a.rin.w[i];
                    q.cell = a.rin.cell[i];
                    q.id = a.rin.id[i];
                    q.lin = a.rin.lin[i];
                    q.e = a.rin.e[i];
                    if constexpr (DERIV) {
#pragma unroll
                        for (int j = 0; j < MAX_SCORES; ++j)
                            S[j] = (j < P2) ? a.rin.S[(long long)j * a.rin.cap + i] : 0.0;
                    }
                    const uint32_t jc = a.rin.jcount[i];
                    if (jc) {
                        pp->store(t, q, S);
                        const uint32_t js = a.rin.jstart[i];
                        fresh = (js & FRESH_DIRECTION) != 0;
                        jnext = js & ~FRESH_DIRECTION;
                        jend = jnext + jc;
                        q.lin = lineage_hash(q.lin, q.e, jnext);
                        q.e = 0;
                        ++jnext;
                        if (fresh) {  // its own isotropic direction
                            uint32_t rr[4] = {q.id, (uint32_t)q.lin, (uint32_t)(q.lin >> 32), 0xFFFFFFFEu};
                            philox4x32_10(rr, k0, k1);
                            q.mu = 2.0 * u01(rr[0], rr[1]) - 1.0;
                            q.inv_mu = 1.0 / q.mu;
                        }
                    }
                }
            }
            have = true;
            evs = 0;
            qb = batch_of(q.id, a.B, a.N, a.batch_m);
        }
        // ---- one event ----
        if (evs == a.emax) {
            push_record<DERIV>(a, q, S, q.w, q.e, 0u, 0u, warp_reserve(a.rout.count));
            have = false;
            continue;
        }
        if (q.e >= MAX_EVENTS) {
            atomicOr(a.err, ERR_EVENTS);
            have = false;
            continue;
        }
        uint32_t r[4] = {q.id, (uint32_t)q.lin, (uint32_t)(q.lin >> 32), 2u * q.e};
        philox4x32_10(r, k0, k1);
        const double uf = u01(r[0], r[1]);
        const double uc = u01(r[2], r[3]);
        const int k = q.cell;
        const double dcoll = (-hw_log(uf)) * a.inv_sigt[k];
        const double xl = a.edges[k], xr = a.edges[k + 1];
        const double xe = (q.mu > 0.0) ? xr : xl;
        const double dedge = (xe - q.x) * q.inv_mu;
        const double dcens = q.tau;
        int ev;
        double l;
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
        // track-length tallies
        const double wl = q.w * l;
        const double wlmu = wl * q.mu;
        const double wlf = wl * (1.0 / 3.0 - q.mu * q.mu);
        {
            // one shared atomic per lane and word; the flux to the batch row
            // only (see the FP32 loop)
            const int b = qb;
            const long long c0 = fixed_bits(wl, S_t);
            sadd(&s_tl[I + k], fixed_bits(wlmu, S_t));
            sadd(&s_tl[2 * I + k], fixed_bits(wlf, S_t));
            if (b == b_blk)
                sadd(&s_bat[k], c0);
            else
                add128(&a.batch[(long long)b * I + k], c0);
        }
        if constexpr (DERIV) {
            // scores after this segment's flight, then w l S_j per parameter
            const int rg = a.region[k];
#pragma unroll
            for (int j = 0; j < MAX_SCORES; ++j) {
                if (j == rg) {
                    S[j] = S[j] - l;
                    if (ev == 2) S[j] = S[j] + a.inv_sigt[k];
                }
            }
#pragma unroll
            for (int j = 0; j < MAX_SCORES; ++j)
                if (j < P2) sadd(&s_dtl[j * I + k], fixed_bits(wl * S[j], S_t));
        }
        // move
        if (ev == 1) {
            q.x = xe;
        } else {
            double xn = q.x + q.mu * l;
            if (xn < xl) xn = xl;
            if (xn > xr) xn = xr;
            q.x = xn;
        }
        q.tau = (ev == 0) ? 0.0 : q.tau - l;
        const uint32_t e_ev = q.e;
        q.e = q.e + 1;
        ++evs;
        if (ev == 0) {
            // census: the bank record (its tallies, and a derivative run's
            // census derivative tallies, come from the comb's census pass)
            const unsigned long long slot = warp_reserve(a.cen.count);
            if ((long long)slot < a.cen.cap) {
                if constexpr (DERIV) {
#pragma unroll
                    for (int j = 0; j < MAX_SCORES; ++j)
                        if (j < P2) a.cen.S[(long long)j * a.cen.cap + (long long)slot] = S[j];
                }
                a.cen.x[slot] = q.x;
                a.cen.mu[slot] = q.mu;
                a.cen.w[slot] = q.w;
                a.cen.cell[slot] = q.cell;
                a.cen.id[slot] = q.id;

                const unsigned long long wfx = (unsigned long long)fixed_bits(q.w, a.sd->Sc);
                a.cen.lw[slot] = LinW{q.lin, wfx};
                a.cen.imu[slot] = q.inv_mu;
                atomicAdd(&a.gcnt[q.id], 1u);
                atomicAdd(&a.gw[q.id], wfx);
            } else {
                atomicOr(a.err, ERR_CENSUS_OVERFLOW);
            }
            cnt.v[ST_CENSUS]++;
            cnt.v[ST_MAX_EVENTS] = max(cnt.v[ST_MAX_EVENTS], q.e);
            have = false;
            continue;
        }
        bool have_r2 = false;
        uint32_t r2[4];
        if (ev == 1) {
            cnt.v[ST_CROSSINGS]++;
            const int nk = (q.mu > 0.0) ? k + 1 : k - 1;
            if (nk < 0 || nk >= I) {
                const int side = (nk < 0) ? 0 : 1;
                const int bc = side ? a.bc_r : a.bc_l;
                if (bc == 0) {
                    const double amu = fabs(q.mu);
                    const double ia = (amu < GRAZE_MU) ? 2.0 / GRAZE_MU : 1.0 / amu;
                    const double wi = q.w * ia;
                    add128(&a.bnd[3 * side + 0], fixed_bits(wi, S_t));
                    add128(&a.bnd[3 * side + 1], fixed_bits(wi * (1.0 / 3.0 - q.mu * q.mu), S_t));
                    add128(&a.bnd[3 * side + 2], fixed_bits(wi * (0.5 - amu), S_t));
                    if constexpr (DERIV) {
#pragma unroll
                        for (int j = 0; j < MAX_SCORES; ++j) {
                            if (j < P2) {
                                Acc128* d = a.dbnd + 6 * j + 3 * side;
                                add128(&d[0], fixed_bits(wi * S[j], S_t));
                                add128(&d[1], fixed_bits(wi * (1.0 / 3.0 - q.mu * q.mu) * S[j], S_t));
                                add128(&d[2], fixed_bits(wi * (0.5 - amu) * S[j], S_t));
                            }
                        }
                    }
                    cnt.v[ST_LEAKED]++;
                    cnt.v[ST_MAX_EVENTS] = max(cnt.v[ST_MAX_EVENTS], q.e);
                    have = false;
                    continue;
                }
                q.mu = -q.mu;
                q.inv_mu = -q.inv_mu;
                cnt.v[ST_REFLECTIONS]++;
            } else {
                q.cell = nk;
            }
        } else {
            cnt.v[ST_COLLISIONS]++;
            // the collision emits floor(c) + [u_c < c - floor(c)] particles (mean c)
            const double cc = a.c[k];
            const double cfl = floor(cc);
            const uint32_t nsec = (uint32_t)cfl + ((uc < cc - cfl) ? 1u : 0u);
            if (nsec == 0) {
                cnt.v[ST_ABSORBED]++;
                cnt.v[ST_MAX_EVENTS] = max(cnt.v[ST_MAX_EVENTS], q.e);
                have = false;
                continue;
            }
            r2[0] = q.id;
            r2[1] = (uint32_t)q.lin;
            r2[2] = (uint32_t)(q.lin >> 32);
            r2[3] = 2u * e_ev + 1u;
            philox4x32_10(r2, k0, k1);
            have_r2 = true;
            q.mu = 2.0 * u01(r2[0], r2[1]) - 1.0;
            q.inv_mu = 1.0 / q.mu;
            if (nsec > 1) {
                // the other emitted particles: daughters that take their own
                // lineages and isotropic directions, expanded by this lane
                // after the current track, or queued as records when it is
                // already expanding a parent
                const uint32_t nx = nsec - 1;
                uint32_t jr = 1;  // the first daughter that goes to the record queue
                if (LOCAL_MAX > 0 && jnext >= jend) {
                    P64 b = q;
                    b.e = e_ev | SECONDARY_EVENT;
                    pp->store(t, b, S);
                    fresh = true;
                    jnext = 1;
                    jend = min(nsec, 1u + LOCAL_MAX);
                    jr = jend;
                }
                if (jr < nsec) {
                    const uint32_t nch = (nsec - jr + SPLIT_CHUNK - 1) / SPLIT_CHUNK;
                    const unsigned long long b0 = warp_reserve_n(a.rout.count, nch);
                    for (uint32_t ch = 0; ch < nch; ++ch) {
                        const uint32_t j0 = jr + ch * SPLIT_CHUNK;
                        const uint32_t jc = min((uint32_t)SPLIT_CHUNK, nsec - j0);
                        push_record<DERIV>(a, q, S, q.w, e_ev | SECONDARY_EVENT, j0 | FRESH_DIRECTION, jc,
                                           b0 + ch);
                    }
                }
                cnt.v[ST_DAUGHTERS] += nx;
            }
            if constexpr (DERIV) {
                const int jc = R + a.region[k];
#pragma unroll
                for (int j = 0; j < MAX_SCORES; ++j)
                    if (j == jc) S[j] = S[j] + a.inv_c[k];
            }
        }
        if (ww_on) {
            const int kc = q.cell;
            const double hi = a.ww_hi[kc];
            const double lo = a.ww_lo[kc];
            if (q.w > hi) {
                const double ctr = a.ww_c[kc];
                const double ndd = ceil(q.w / ctr);
                if (ndd > (double)MAX_DAUGHTERS) {
                    atomicOr(a.err, ERR_DAUGHTERS);
                    have = false;
                    continue;
                }
                const uint32_t nd = (uint32_t)ndd;
                const double wd = q.w / (double)nd;
                cnt.v[ST_SPLIT_EVENTS]++;
                cnt.v[ST_DAUGHTERS] += nd - 1;
                uint32_t jr = 1;  // the first daughter that goes to the record queue
                if (LOCAL_MAX > 0 && jnext >= jend) {
                    // up to LOCAL_MAX daughters follow the current track on
                    // this lane (same block, so their batch row stays in
                    // shared memory); the bound keeps a large split from
                    // holding one lane while the rest of its block waits
                    P64 b = q;
                    b.w = wd;
                    b.e = e_ev;
                    pp->store(t, b, S);
                    fresh = false;
                    jnext = 1;
                    jend = min(nd, 1u + LOCAL_MAX);
                    jr = jend;
                }
                if (jr < nd) {
                    const uint32_t nch = (nd - jr + SPLIT_CHUNK - 1) / SPLIT_CHUNK;
                    const unsigned long long b0 = warp_reserve_n(a.rout.count, nch);
                    for (uint32_t ch = 0; ch < nch; ++ch) {
                        const uint32_t j0 = jr + ch * SPLIT_CHUNK;
                        const uint32_t jc = min((uint32_t)SPLIT_CHUNK, nd - j0);
                        push_record<DERIV>(a, q, S, wd, e_ev, j0, jc, b0 + ch);
                    }
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
                    philox4x32_10(r2, k0, k1);
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
                    have = false;
                    continue;
                }
            }
        }
    }
}

template <bool DERIV>
// Two resident blocks of 256 threads per SM: the event loop wants about 120
// registers; at three blocks it spills to local memory, whose traffic (the
// L1 left beside the shared tallies hits ~20% of it) costs more time than
// the extra warps hide.
__global__ void __launch_bounds__(TRACK_THREADS, 2) track64_kernel(TrackArgs<double> a) {
    extern __shared__ long long sm[];
    __shared__ unsigned s_next;
    __shared__ PendingParent64<DERIV> s_pp;
    const int I = a.I;
    if (threadIdx.x == 0) s_next = 0;
    const int rows = DERIV ? TALLY_ROWS + a.P2 : TALLY_ROWS;
    for (int i = threadIdx.x; i < rows * I; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    Counters cnt;
    cnt.zero();
    const long long n_in = a.from_bank ? (long long)a.sd->nbank : (long long)*a.rin.count;
    const long long n_use = (!a.from_bank && n_in > a.rin.cap) ? a.rin.cap : n_in;
    // wave 0: each block takes a contiguous id range of [bank_lo, bank_hi), so
    // nearly all of its segments fall in one variance batch (kept in shared
    // memory), and its lanes take the range's items from a shared counter
    // (splits leave the daughters with the splitting lane, so lanes carry
    // uneven work); record waves: grid-stride over the records.  More,
    // smaller ranges balance the blocks better but cost more tally flushes;
    // one range per resident block measured fastest.
    long long stride, item, item_end;
    unsigned* dyn = nullptr;
    int b_blk = -1;
    if (a.from_bank) {
        const long long lo = a.bank_lo;
        const long long hi = min(n_use, a.bank_hi);
        const long long len = hi > lo ? hi - lo : 0;
        const long long chunk = (len + gridDim.x - 1) / gridDim.x;
        const long long first = lo + (long long)blockIdx.x * chunk;
        item = first;
        item_end = min(hi, first + chunk);
        stride = 0;
        dyn = &s_next;
        if (first < hi) b_blk = batch_of((uint32_t)first, a.B, a.N, a.batch_m);
    } else {
        item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        item_end = n_use;
        stride = (long long)gridDim.x * blockDim.x;
    }
    run_items<DERIV, LOCAL_DAUGHTERS>(a, item, item_end, stride, dyn, b_blk, sm, cnt, &s_pp);
    __syncthreads();
    flush_tallies(sm, I, a.tl);
    if constexpr (DERIV) {
        for (int i = threadIdx.x; i < a.P2 * I; i += blockDim.x)
            if (sm[TALLY_ROWS * I + i] != 0) add128(&a.dtl[i], sm[TALLY_ROWS * I + i]);
    }
    if (b_blk >= 0)
        for (int i = threadIdx.x; i < I; i += blockDim.x)
            if (sm[3 * I + i] != 0) add128(&a.batch[(long long)b_blk * I + i], sm[3 * I + i]);
    flush_counters(cnt, a.stats);
}

// Persistent batched variant: blocks pop tiles (problem, id range) from a
// device counter; the block-private tallies are flushed when a block moves
// to another problem, the batch row after every tile.
__global__ void __launch_bounds__(TRACK_THREADS, 2) track64_kernel_batch(const TrackArgs<double>* args, BatchPlan plan) {
    extern __shared__ long long sm[];
    __shared__ TrackArgs<double> A;
    __shared__ long long s_t;
    __shared__ int s_p;
    __shared__ unsigned s_next;
    __shared__ PendingParent64<false> s_pp;
    Counters cnt;
    cnt.zero();
    const long long total = plan.tile_off[plan.P];
    int cur = -1, Ic = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = (long long)atomicAdd(plan.head, 1ull);
            int p = -1;
            if (t < total) {
                int lo = 0, hi = plan.P - 1;  // largest p with tile_off[p] <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (plan.tile_off[mid] <= t) lo = mid; else hi = mid - 1;
                }
                p = lo;
            }
            s_t = t;
            s_p = p;
            s_next = 0;
        }
        __syncthreads();
        const long long t = s_t;
        const int p = s_p;
        if (p < 0 || p != cur) {  // a problem switch, or no tile left (also on the first pop)
            if (cur >= 0) {
                flush_tallies(sm, Ic, A.tl);
                flush_counters(cnt, A.stats);
                cnt.zero();
                __syncthreads();
            }
            if (p < 0) break;
            if (threadIdx.x == 0) A = args[p];
            __syncthreads();
            cur = p;
            Ic = A.I;
            for (int i = threadIdx.x; i < TALLY_ROWS * Ic; i += blockDim.x) sm[i] = 0;
            __syncthreads();
        }
        const long long n_in = A.from_bank ? (long long)A.sd->nbank : (long long)*A.rin.count;
        const long long n_use = (!A.from_bank && n_in > A.rin.cap) ? A.rin.cap : n_in;
        const long long i0 = (t - plan.tile_off[p]) * (long long)plan.tile;
        const long long i1 = min(n_use, i0 + (long long)plan.tile);
        const int b_tile = (A.from_bank && i0 < n_use) ? batch_of((uint32_t)i0, A.B, A.N, A.batch_m) : -1;
        run_items<false, 0>(A, i0, i1, 0, &s_next, b_tile, sm, cnt, &s_pp);
        __syncthreads();
        if (b_tile >= 0)
            for (int i = threadIdx.x; i < Ic; i += blockDim.x) {
                const long long v = sm[3 * Ic + i];
                if (v != 0) {
                    add128(&A.batch[(long long)b_tile * Ic + i], v);
                    sm[3 * Ic + i] = 0;
                }
            }
        __syncthreads();
    }
}

}  // namespace

void launch_track_fp64(const TrackArgs<double>& a, int grid, int block, size_t smem, cudaStream_t s) {
    if (a.P2 > 0)
        track64_kernel<true><<<grid, block, smem, s>>>(a);
    else
        track64_kernel<false><<<grid, block, smem, s>>>(a);
}

int track_smem_optin_fp64(size_t smem, int deriv) {
    return deriv ? raise_smem_limit((const void*)track64_kernel<true>, smem)
                 : raise_smem_limit((const void*)track64_kernel<false>, smem);
}

int track_blocks_per_sm_fp64(int block, size_t smem, int deriv) {
    int n = 0;
    if (deriv)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, track64_kernel<true>, block, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, track64_kernel<false>, block, smem);
    return n;
}

void launch_track_batch_fp64(const TrackArgs<double>* args, const BatchPlan& plan, int grid, int block, size_t smem,
                             cudaStream_t s) {
    track64_kernel_batch<<<grid, block, smem, s>>>(args, plan);
}

int track_batch_smem_optin_fp64(size_t smem) {
    return raise_smem_limit((const void*)track64_kernel_batch, smem);
}

int track_batch_blocks_per_sm_fp64(int block, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, track64_kernel_batch, block, smem);
    return n;
}

}  // namespace hww

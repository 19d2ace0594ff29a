// track_fp32.cu -- FP32-tracking variant of the event loop.
//
// Same events, rules and random streams as the FP64 kernel (the uniforms are
// the top 23 bits of the same Philox words), but the geometry runs in FP32:
// a track keeps its cell index and an FP32 offset from the cell's left edge,
// an FP32 direction, an FP32 distance to census and FP32 flight distances.
// Weights stay FP64 (the window tests compare their bit patterns, and the
// split count and survival test use an FP32 ratio and a product in place of
// FP64 divides); tally contributions are formed in
// exact integer arithmetic from a fixed-point copy of the weight,
//     round(W * f),   W = round(w 2^S) (64-bit),  f = l, l mu, l (1/3 - mu^2) (FP32),
// i.e. the exact product of the 64-bit weight and the 24-bit mantissa of f,
// rounded once (half up) at the tally scale.  The FP64 pipe, of which GB300
// has little, is left to rare events (splits, roulette, leaks, census).
//
// The event loop is flattened: a lane whose track ends (census, absorption,
// leak, roulette kill, event budget) loads its next track in the same loop
// iteration the other lanes spend on their next event, so a warp stays full
// until the work runs out.
#include "track_common.cuh"

namespace hww {
namespace {

struct P32 {
    float xo, mu, inv_mu, tau;
    double w;
    long long W;  // w 2^S rounded
    int cell;
    uint32_t id;
    uint64_t lin;
    uint32_t e;
};

// The pending parent of a lane (the record whose daughters it expands), kept
// in shared memory, one column per thread: it is written at a split and read
// once per daughter, and registers are what limits the resident warps.
struct PendingParent {
    float xo[TRACK_THREADS], mu[TRACK_THREADS], tau[TRACK_THREADS];
    double w[TRACK_THREADS];
    long long W[TRACK_THREADS];
    int cell[TRACK_THREADS];
    uint32_t id[TRACK_THREADS], e[TRACK_THREADS];
    uint64_t lin[TRACK_THREADS];
    __device__ __forceinline__ void store(int t, const P32& q) {
        xo[t] = q.xo;
        mu[t] = q.mu;
        tau[t] = q.tau;
        w[t] = q.w;
        W[t] = q.W;
        cell[t] = q.cell;
        id[t] = q.id;
        e[t] = q.e;
        lin[t] = q.lin;
    }
    __device__ __forceinline__ void load(int t, P32& q) const {
        q.xo = xo[t];
        q.mu = mu[t];
        q.tau = tau[t];
        q.w = w[t];
        q.W = W[t];
        q.cell = cell[t];
        q.id = id[t];
        q.e = e[t];
        q.lin = lin[t];
    }
};

// The comb-scale weight of a census particle from its tally-scale weight W:
// W 2^(Sc - S), rounded to nearest (ties to even) when Sc < S; integer
// arithmetic, so the common census event uses no FP64 instruction (the FP64
// path rounds w 2^Sc directly; the two can differ in the last bit)
__device__ __forceinline__ unsigned long long comb_weight(long long W, int shift) {
    const unsigned long long u = (unsigned long long)W;
    if (shift <= 0) return u << (-shift);
    const unsigned long long q = u >> shift, r = u & ((1ull << shift) - 1ull), h = 1ull << (shift - 1);
    return q + ((r > h || (r == h && (q & 1ull))) ? 1ull : 0ull);
}

// positive doubles order like their bit patterns
__device__ __forceinline__ bool dgt(double a, double b) { return __double_as_longlong(a) > __double_as_longlong(b); }

__device__ __forceinline__ void push_record(const TrackArgs<float>& a, const P32& q, double w, uint32_t e,
                                            uint32_t jstart, uint32_t jcount, unsigned long long slot) {
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

// The event loop over items [item, item_end): with the given stride, or, when
// s_next is a block-shared counter, item + the next value of that counter
// (lanes busy with many daughters then take fewer items); b_blk is the
// variance batch whose row is kept in shared memory (-1: none).
template <uint32_t LOCAL_MAX>
__device__ __forceinline__ void run_items(const TrackArgs<float>& a, long long item, const long long item_end,
                                          const long long stride, unsigned* s_next, const int b_blk, long long* sm,
                                          Counters& cnt, PendingParent* pp) {
    const int I = a.I;
    long long* s_tl = sm;
    long long* s_bat = sm + 3 * I;  // batch row of the current id range
    // the step scalars needed only at rare events are read where they are
    // used (registers are what limits the resident warps)
    const uint32_t k0 = a.sd->k0, k1 = a.sd->k1;
    const int ww_on = a.sd->ww_on;
    const int t = threadIdx.x;

    P32 q;
    uint32_t jnext = 0, jend = 0;
    bool fresh = false;  // the pending parent's daughters are a collision's extra particles
    bool have = false;
    int evs = 0;
    int qb = 0;  // variance batch of the current track's source id
    for (;;) {
        if (!have) {
            if (jnext < jend) {
                pp->load(t, q);
                q.lin = lineage_hash(q.lin, q.e, jnext);
                q.e = 0;
                ++jnext;
                if (fresh) {  // its own isotropic direction
                    uint32_t rr[4] = {q.id, (uint32_t)q.lin, (uint32_t)(q.lin >> 32), 0xFFFFFFFEu};
                    philox4x32_10(rr, k0, k1);
                    q.mu = 2.0f * u01f(rr[1]) - 1.0f;
                }
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
                    q.tau = a.tau0f;
                    q.w = a.sd->wbar;
                    q.W = a.sd->Wbar;
                    if (a.sd->birth) {
                        uint32_t r[4] = {(uint32_t)i, 0u, 0u, 0xFFFFFFFFu};
                        philox4x32_10(r, k0, k1);
                        q.mu = 2.0f * u01f(r[1]) - 1.0f;
                        const double x = a.src_x;
                        if (x <= a.edges[0] && q.mu < 0.0f && a.bc_l == 1) q.mu = -q.mu;
                        if (x >= a.edges[I] && q.mu > 0.0f && a.bc_r == 1) q.mu = -q.mu;
                        q.cell = (q.mu < 0.0f) ? a.birth_cell_neg : a.birth_cell_pos;
                        q.xo = (float)(x - a.edges[q.cell]);
                    } else {
                        const BankRec<float> r = a.bank[i];
                        q.xo = r.x;
                        q.mu = r.mu;
                        q.cell = r.cell;
                    }
                } else {
                    q.xo = a.rin.x[i];
                    q.mu = a.rin.mu[i];
                    q.tau = a.rin.tau[i];
                    q.w = a.rin.w[i];
                    q.W = to_fixed(q.w, a.sd->tscale);
                    q.cell = a.rin.cell[i];
                    q.id = a.rin.id[i];
                    q.lin = a.rin.lin[i];
                    q.e = a.rin.e[i];
                    const uint32_t jc = a.rin.jcount[i];
                    if (jc) {
                        pp->store(t, q);
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
                            q.mu = 2.0f * u01f(rr[1]) - 1.0f;
                        }
                    }
                }
            }
            q.inv_mu = __frcp_rn(q.mu);  // the correctly rounded 1/mu
            have = true;
            evs = 0;
            qb = batch_of(q.id, a.B, a.N, a.batch_m);
        }
        // ---- one event ----
        if (evs == a.emax) {
            push_record(a, q, q.w, q.e, 0u, 0u, warp_reserve(a.rout.count));
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
        const float uf = u01f(r[1]);
        const float uc = u01f(r[3]);
        const int k = q.cell;
        const float4 cf = __ldg(&a.cellf[k]);  // width, 1/Sigma_t, c
        const float dxk = cf.x;
        const float dcoll = -logf(uf) * cf.y;
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
        const float m2 = q.mu * q.mu;
        const float f3 = 1.0f / 3.0f - m2;
        {
            // one shared atomic per lane and word: merging the lanes of a
            // warp that share a cell first (match + shuffle tree) measured
            // slower than the atomics it saves.  The flux goes to the
            // variance-batch row only: the flux tally is the sum of the batch
            // rows, formed after the tracking (one atomic fewer per segment)
            const int b = qb;
            const long long c0 = fx_mul(q.W, l);
            sadd(&s_tl[I + k], fx_mul(q.W, l * q.mu));
            sadd(&s_tl[2 * I + k], fx_mul(q.W, l * f3));
            if (b == b_blk)
                sadd(&s_bat[k], c0);
            else
                add128(&a.batch[(long long)b * I + k], c0);
        }
        if (ev != 1) q.xo = fminf(fmaxf(fmaf(q.mu, l, q.xo), 0.0f), dxk);
        q.tau = (ev == 0) ? 0.0f : q.tau - l;
        const uint32_t e_ev = q.e;
        q.e = q.e + 1;
        ++evs;
        if (ev == 0) {
            // census: the bank record (its tallies come from the census pass)
            const unsigned long long slot = warp_reserve(a.cen.count);
            if ((long long)slot < a.cen.cap) {
                a.cen.x[slot] = q.xo;
                a.cen.mu[slot] = q.mu;
                a.cen.w[slot] = q.w;
                a.cen.cell[slot] = q.cell;
                a.cen.id[slot] = q.id;

                const unsigned long long wfx = comb_weight(q.W, a.comb_shift);
                a.cen.lw[slot] = LinW{q.lin, wfx};
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
            const int nk = (q.mu > 0.0f) ? k + 1 : k - 1;
            if (nk < 0 || nk >= I) {
                const int side = (nk < 0) ? 0 : 1;
                const int bc = side ? a.bc_r : a.bc_l;
                if (bc == 0) {
                    const double amu = fabs((double)q.mu);
                    const double ia = (amu < GRAZE_MU) ? 2.0 / GRAZE_MU : 1.0 / amu;
                    const double wi = q.w * ia;
                    const double dm2 = (double)q.mu * (double)q.mu;
                    add128(&a.bnd[3 * side + 0], to_fixed(wi, a.sd->tscale));
                    add128(&a.bnd[3 * side + 1], to_fixed(wi * (1.0 / 3.0 - dm2), a.sd->tscale));
                    add128(&a.bnd[3 * side + 2], to_fixed(wi * (0.5 - amu), a.sd->tscale));
                    cnt.v[ST_LEAKED]++;
                    cnt.v[ST_MAX_EVENTS] = max(cnt.v[ST_MAX_EVENTS], q.e);
                    have = false;
                    continue;
                }
                q.mu = -q.mu;
                q.inv_mu = -q.inv_mu;
                q.xo = side ? dxk : 0.0f;
                cnt.v[ST_REFLECTIONS]++;
            } else {
                q.cell = nk;
                q.xo = (q.mu > 0.0f) ? 0.0f : __ldg(&a.cellf[nk]).x;
            }
        } else {
            cnt.v[ST_COLLISIONS]++;
            // the collision emits floor(c) + [u_c < c - floor(c)] particles (mean c)
            const float cfl = floorf(cf.z);
            const uint32_t nsec = (uint32_t)cfl + ((uc < cf.z - cfl) ? 1u : 0u);
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
            q.mu = 2.0f * u01f(r2[1]) - 1.0f;
            q.inv_mu = __frcp_rn(q.mu);
            if (nsec > 1) {
                // the other emitted particles: daughters that take their own
                // lineages and isotropic directions, expanded by this lane
                // after the current track, or queued as records when it is
                // already expanding a parent
                const uint32_t nx = nsec - 1;
                uint32_t jr = 1;  // the first daughter that goes to the record queue
                if (LOCAL_MAX > 0 && jnext >= jend) {
                    P32 b = q;
                    b.e = e_ev | SECONDARY_EVENT;
                    pp->store(t, b);
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
                        push_record(a, q, q.w, e_ev | SECONDARY_EVENT, j0 | FRESH_DIRECTION, jc, b0 + ch);
                    }
                }
                cnt.v[ST_DAUGHTERS] += nx;
            }
        }
        if (ww_on) {
            const int kc = q.cell;
            const double2 hl = __ldg(&a.ww_hl[kc]);  // ceiling, floor
            if (dgt(q.w, hl.x)) {
                const double ctr = a.ww_c[kc];
                // split count from an FP32 ratio (the FP32 path's own rounding)
                const float ndf = ceilf((float)q.w / (float)ctr);
                const double ndd = (double)fmaxf(ndf, 2.0f);
                if (ndd > (double)MAX_DAUGHTERS) {
                    atomicOr(a.err, ERR_DAUGHTERS);
                    have = false;
                    continue;
                }
                const uint32_t nd = (uint32_t)ndd;
                const double wd = q.w / (double)nd;
                const long long Wd = to_fixed(wd, a.sd->tscale);
                cnt.v[ST_SPLIT_EVENTS]++;
                cnt.v[ST_DAUGHTERS] += nd - 1;
                uint32_t jr = 1;  // the first daughter that goes to the record queue
                if (LOCAL_MAX > 0 && jnext >= jend) {
                    // up to LOCAL_MAX daughters follow the current track on
                    // this lane (same block, so their batch row stays in
                    // shared memory); the bound keeps a large split from
                    // holding one lane while the rest of its block waits
                    P32 b = q;
                    b.w = wd;
                    b.W = Wd;
                    b.e = e_ev;
                    pp->store(t, b);
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
                        push_record(a, q, wd, e_ev, j0, jc, b0 + ch);
                    }
                }
                q.w = wd;
                q.W = Wd;
                q.lin = lineage_hash(q.lin, e_ev, 0);
                q.e = 0;
            } else if (dgt(hl.y, q.w)) {
                if (!have_r2) {
                    r2[0] = q.id;
                    r2[1] = (uint32_t)q.lin;
                    r2[2] = (uint32_t)(q.lin >> 32);
                    r2[3] = 2u * e_ev + 1u;
                    philox4x32_10(r2, k0, k1);
                }
                const double ctr = a.ww_c[kc];
                // survive iff u < w / ww, tested as u ww < w (no divide)
                const double ur = u01(r2[2], r2[3]);
                if (ur * ctr < q.w) {
                    q.w = ctr;
                    q.W = to_fixed(ctr, a.sd->tscale);
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

// Two resident blocks of 256 threads per SM: the event loop wants about 120
// registers; at three blocks it spills to local memory, whose traffic (the
// L1 left beside the shared tallies hits ~20% of it) costs more time than
// the extra warps hide.
__global__ void __launch_bounds__(TRACK_THREADS, 2) track32_kernel(TrackArgs<float> a) {
    extern __shared__ long long sm[];
    __shared__ unsigned s_next;
    __shared__ PendingParent s_pp;
    const int I = a.I;
    if (threadIdx.x == 0) s_next = 0;
    for (int i = threadIdx.x; i < TALLY_ROWS * I; i += blockDim.x) sm[i] = 0;
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
    run_items<LOCAL_DAUGHTERS>(a, item, item_end, stride, dyn, b_blk, sm, cnt, &s_pp);
    __syncthreads();
    flush_tallies(sm, I, a.tl);
    if (b_blk >= 0)
        for (int i = threadIdx.x; i < I; i += blockDim.x)
            if (sm[3 * I + i] != 0) add128(&a.batch[(long long)b_blk * I + i], sm[3 * I + i]);
    flush_counters(cnt, a.stats);
}

// Persistent batched variant: blocks pop tiles (problem, id range) from a
// device counter; the block-private tallies are flushed when a block moves
// to another problem, the batch row after every tile.
__global__ void __launch_bounds__(TRACK_THREADS, 2) track32_kernel_batch(const TrackArgs<float>* args,
                                                                         BatchPlan plan) {
    extern __shared__ long long sm[];
    __shared__ PendingParent s_pp;
    __shared__ TrackArgs<float> A;
    __shared__ long long s_t;
    __shared__ int s_p;
    __shared__ unsigned s_next;
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
        run_items<0>(A, i0, i1, 0, &s_next, b_tile, sm, cnt, &s_pp);
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

void launch_track_fp32(const TrackArgs<float>& a, int grid, int block, size_t smem, cudaStream_t s) {
    track32_kernel<<<grid, block, smem, s>>>(a);
}

int track_smem_optin_fp32(size_t smem) {
    return raise_smem_limit((const void*)track32_kernel, smem);
}

int track_blocks_per_sm_fp32(int block, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, track32_kernel, block, smem);
    return n;
}

void launch_track_batch_fp32(const TrackArgs<float>* args, const BatchPlan& plan, int grid, int block, size_t smem,
                             cudaStream_t s) {
    track32_kernel_batch<<<grid, block, smem, s>>>(args, plan);
}

int track_batch_smem_optin_fp32(size_t smem) {
    return raise_smem_limit((const void*)track32_kernel_batch, smem);
}

int track_batch_blocks_per_sm_fp32(int block, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, track32_kernel_batch, block, smem);
    return n;
}

}  // namespace hww

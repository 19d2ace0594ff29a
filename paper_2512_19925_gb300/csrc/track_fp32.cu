// track_fp32.cu -- FP32-tracking variant of the event loop.
//
// Same events, rules and random streams as the FP64 kernel (the uniforms are
// the top 23 bits of the same Philox words), but the geometry runs in FP32:
// a track keeps its cell index and an FP32 offset from the cell's left edge,
// an FP32 direction, an FP32 distance to census and FP32 flight distances
// (-ln u from the hardware base-2 logarithm).
// Weights stay FP64 (the window tests compare their bit patterns, and the
// split count and survival test use an FP32 ratio and a product in place of
// FP64 divides); tally contributions are formed in exact integer arithmetic
// from an FP32 copy of the weight at the tally scale,
//     round(a * f),   a = fl32(w 2^S),  f = l, l mu, l (1/3 - mu^2) (FP32),
// i.e. the exact 48-bit product of two 24-bit significands (one wide integer
// multiply), rounded once (half up) at the tally scale.  The FP64 pipe, of
// which GB300 has little, is left to rare events (weight changes, leaks,
// census).
//
// Both the single-problem kernel and the persistent batched kernel (one
// tile of one problem at a time) run a warp-synchronous loop (run_warp): the
// lanes of a warp take their events together and share a daughter stack, so
// the daughters of a split spread over the warp's idle lanes.
#include <algorithm>

#include "track_common.cuh"

namespace hww {
namespace {

struct P32 {
    float xo, mu, inv_mu, tau;
    double w;
    float tw;     // tally weight: w 2^S rounded to FP32
    int cell;
    uint32_t id;
    uint64_t lin;
    uint32_t e;
};

// The comb-scale weight of a census particle from its fixed-point weight
// W = round(w 2^S): W 2^(Sc - S), rounded to nearest (ties to even) when
// Sc < S (the FP64 path rounds w 2^Sc directly; the two can differ in the
// last bit)
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

// ---------------------------------------------------------------------------
// The event loop, warp-synchronous.
//
// All 32 lanes of a warp iterate together until the warp has no work left.
// Each iteration hands work to the lanes without a track (deriving the
// lineage keys of the daughters it hands out), draws the Philox blocks of
// every lane at one site, takes one event of every live track (or one
// direction-sampling step of a new track), stages the iteration's census
// particles and sums its counts.  Work comes, in this order, from the warp's daughter
// stack in shared memory (a split leaves its daughters there, so they spread
// over the warp's idle lanes instead of queueing behind one lane), then from
// the block's range of start-bank items (prefetched 32 at a time into shared
// memory with asynchronous copies, so that a new track does not wait for
// HBM) or records.  Census particles are staged per warp in shared memory and
// written out 32 at a time with one slot reservation on the census counter
// (one global atomic per 32 census particles instead of one per iteration,
// and 128-byte stores).  Counts are summed over the warp (each lane holds one
// counter), so they take no per-lane registers.  A split whose warp stack is
// full, and a track past its event budget, go to the record queue.
constexpr int WARPS = TRACK_THREADS / 32;
constexpr int WSTACK = 32;  // daughter-stack entries per warp
constexpr int KSTACK = 64;  // lineage keys per warp, for the daughters of stack entries
constexpr uint16_t NO_KEYS = 0xFFFFu;
// Splits are queued per warp and processed (split count, daughter weight,
// stack push) by the whole warp once SPLIT_BATCH of them wait, or when lanes
// run out of other work: the split's arithmetic (two divisions and a
// fixed-point rounding in FP64) then runs for many lanes at once instead of
// for the one or two lanes that split in a typical iteration.
constexpr unsigned SPLIT_BATCH = 16;
constexpr int ROWS32 = TALLY_ROWS_FP32;

struct WarpShared {
    // daughter stack
    float xo[WARPS][WSTACK], mu[WARPS][WSTACK], tau[WARPS][WSTACK];
    double w[WARPS][WSTACK];
    float tw[WARPS][WSTACK];
    int cell[WARPS][WSTACK];
    uint32_t id[WARPS][WSTACK], e[WARPS][WSTACK];
    uint64_t lin[WARPS][WSTACK];
    uint32_t jn[WARPS][WSTACK];  // next daughter to hand out (FRESH_DIRECTION: own isotropic directions)
    uint32_t je[WARPS][WSTACK];  // one past the last daughter
    uint16_t kb[WARPS][WSTACK];  // daughter j's lineage key is key[kb + j] (NO_KEYS: derived when taken)
    int top[WARPS];              // entries in use (only atomics while tracks run)
    // lineage keys of the daughters of stack entries, a stack beside the
    // entries': an entry's keys lie above those of the entries below it, and
    // its last daughter taken frees them
    uint64_t key[WARPS][KSTACK];
    int ktop[WARPS];
    // census staging
    float cx[WARPS][32], cmu[WARPS][32];
    double cw[WARPS][32];
    int ccell[WARPS][32];
    uint32_t cid[WARPS][32];
    LinW clw[WARPS][32];
    // split queue: parents whose split is pending (state before the split,
    // the event index of the split)
    float sx[WARPS][32], smu[WARPS][32], stau[WARPS][32];
    double sw[WARPS][32];
    int scell[WARPS][32];
    uint32_t sid[WARPS][32], se[WARPS][32];
    uint64_t slin[WARPS][32];
    // start-bank records of the next items, two slots of 32: slot s holds
    // items item0 + rb[s] .. + rn[s]; items are handed out from slot rcs
    // starting at rpos
    BankRec<float> ring[WARPS][2][32];
    unsigned rb[WARPS][2];
    int rn[WARPS][2], rcs[WARPS], rpos[WARPS];
};

// event outcome bits of one lane in one iteration (summed over the warp)
enum EvBit : unsigned {
    EB_CENSUS = 0, EB_CROSS, EB_COLL, EB_REFL, EB_LEAK, EB_ABS, EB_SPLIT, EB_RKILL, EB_RSURV, EB_COUNT
};
// the counter each lane of a warp holds
__device__ __constant__ const int kLaneStat[EB_COUNT] = {ST_CENSUS, ST_CROSSINGS, ST_COLLISIONS, ST_REFLECTIONS,
                                                         ST_LEAKED, ST_ABSORBED, ST_SPLIT_EVENTS, ST_RKILLS,
                                                         ST_RSURVIVE};
constexpr int LANE_DAUGHTERS = EB_COUNT;  // lane holding the daughter count
constexpr int LANE_MAXEV = EB_COUNT + 1;  // lane holding the largest event count

// push a parent whose daughters [jn, je) are to be handed out (jn may carry
// FRESH_DIRECTION), with their lineage keys at key[kb + j] or NO_KEYS; false
// when the warp's stack is full
__device__ __forceinline__ bool stack_push(WarpShared& ws, int wp, const P32& b, uint32_t jn, uint32_t je,
                                           uint16_t kb) {
    const int slot = (int)warp_reserve((unsigned*)&ws.top[wp]);
    if (slot >= WSTACK) {
        atomicSub((unsigned*)&ws.top[wp], 1u);
        return false;
    }
    ws.xo[wp][slot] = b.xo;
    ws.mu[wp][slot] = b.mu;
    ws.tau[wp][slot] = b.tau;
    ws.w[wp][slot] = b.w;
    ws.tw[wp][slot] = b.tw;
    ws.cell[wp][slot] = b.cell;
    ws.id[wp][slot] = b.id;
    ws.e[wp][slot] = b.e;
    ws.lin[wp][slot] = b.lin;
    ws.jn[wp][slot] = jn;
    ws.je[wp][slot] = je;
    ws.kb[wp][slot] = kb;
    return true;
}

// daughters j0.. of a parent as chunk records of the record queue
__device__ __forceinline__ void queue_daughters(const TrackArgs<float>& a, const P32& b, uint32_t j0, uint32_t nd,
                                                uint32_t fresh) {
    const uint32_t nch = (nd - j0 + SPLIT_CHUNK - 1) / SPLIT_CHUNK;
    const unsigned long long b0 = warp_reserve_n(a.rout.count, nch);
    for (uint32_t ch = 0; ch < nch; ++ch) {
        const uint32_t js = j0 + ch * SPLIT_CHUNK;
        const uint32_t jc = min((uint32_t)SPLIT_CHUNK, nd - js);
        push_record(a, b, b.w, b.e, js | fresh, jc, b0 + ch);
    }
}

// Two Philox4x32-10 blocks side by side, round by round (two independent
// dependency chains): block r under the per-lane key (ka0, ka1), block s under
// the step's key (k0, k1).
__device__ __forceinline__ void philox_pair(uint32_t r[4], uint32_t s[4], uint32_t ka0, uint32_t ka1, uint32_t k0,
                                            uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * r[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * r[2];
        const uint64_t q0 = (uint64_t)0xD2511F53u * s[0];
        const uint64_t q1 = (uint64_t)0xCD9E8D57u * s[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ r[1] ^ ka0, n2 = (uint32_t)(p0 >> 32) ^ r[3] ^ ka1;
        const uint32_t m0 = (uint32_t)(q1 >> 32) ^ s[1] ^ k0, m2 = (uint32_t)(q0 >> 32) ^ s[3] ^ k1;
        r[0] = n0;
        r[1] = (uint32_t)p1;
        r[2] = n2;
        r[3] = (uint32_t)p0;
        s[0] = m0;
        s[1] = (uint32_t)q1;
        s[2] = m2;
        s[3] = (uint32_t)q0;
        ka0 += 0x9E3779B9u;
        ka1 += 0xBB67AE85u;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// What a lane's track needs next.  The daughters of a split get their
// lineage keys when the split is processed (key stack); a daughter taken
// without one (a multiplying collision's extra particle, a chunk record, a
// split whose keys did not fit) is in M_LINEAGE and gets its key right after
// the refill, from one Philox block the warp draws for all such lanes at
// once, and goes on to its first event in the same iteration.  The other setup steps take the lane's
// iteration with the event's Philox blocks: an extra particle of a
// multiplying collision draws its own direction (M_DIRECTION), a pulse
// particle its birth direction (M_BIRTH).
enum LaneMode : int { M_EVENT = 0, M_LINEAGE = 1, M_DIRECTION = 2, M_BIRTH = 3 };

// 32-bit halves of a block-private 64-bit accumulator kept as two word
// arrays (low words, then high words, of a row of I): exact modulo 2^64
__device__ __forceinline__ void sadd_split(unsigned* lo, unsigned* hi, long long v) {
    const unsigned vl = (unsigned)(unsigned long long)v;
    const unsigned old = atomicAdd(lo, vl);
    const unsigned vh = (unsigned)((unsigned long long)v >> 32) + ((old + vl < old) ? 1u : 0u);
    if (vh) atomicAdd(hi, vh);
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// start-bank records [i0, i0 + n) into a ring slot (lane l copies record l),
// one commit group per call
__device__ __forceinline__ void ring_fetch(BankRec<float>* slot, const BankRec<float>* bank, long long i0, int n,
                                           unsigned lane) {
    if ((int)lane < n)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(slot + lane)),
                     "l"(bank + i0 + lane));
    asm volatile("cp.async.commit_group;\n" ::);
}

__device__ __forceinline__ void ring_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// the warp's staged census particles [0, n) to the census bank: one slot
// reservation, then each lane writes one particle (and its comb group sums)
__device__ __forceinline__ void census_flush(const TrackArgs<float>& a, WarpShared& ws, int wp, unsigned n,
                                             unsigned lane) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.cen.count, (unsigned long long)n);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lane < n) {
        const unsigned long long slot = base + lane;
        if ((long long)slot < a.cen.cap) {
            const uint32_t id = ws.cid[wp][lane];
            const LinW lw = ws.clw[wp][lane];
            a.cen.x[slot] = ws.cx[wp][lane];
            a.cen.mu[slot] = ws.cmu[wp][lane];
            a.cen.w[slot] = ws.cw[wp][lane];
            a.cen.cell[slot] = ws.ccell[wp][lane];
            a.cen.id[slot] = id;
            a.cen.lw[slot] = lw;
            atomicAdd(&a.gcnt[id], 1u);
            atomicAdd(&a.gw[id], lw.wfx);
        } else {
            atomicOr(a.err, ERR_CENSUS_OVERFLOW);
        }
    }
    __syncwarp();
}

// A split's daughter count ceil(w / ww), at least 2, from the FP32 ratio of
// the FP32 roundings of w and ww (the FP32 path's own rounding; the
// roundings are formed from the bits, so no FP64 instruction runs); 0, with
// the error flag set, above MAX_DAUGHTERS.
__device__ __forceinline__ uint32_t split_count(const TrackArgs<float>& a, double w, double ctr) {
    const float ndf = fmaxf(ceilf(fl32_scaled(w, 0) / fl32_scaled(ctr, 0)), 2.0f);
    if (!(ndf <= (float)MAX_DAUGHTERS)) {
        atomicOr(a.err, ERR_DAUGHTERS);
        return 0u;
    }
    return (uint32_t)ndf;
}

// 1/nd rounded to FP64 for nd = 1..64 (entry 0 unused), by the compiler
__device__ const double kInvNd[65] = {
    0.0,
    1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8,
    1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16,
    1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24,
    1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32,
    1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39, 1.0 / 40,
    1.0 / 41, 1.0 / 42, 1.0 / 43, 1.0 / 44, 1.0 / 45, 1.0 / 46, 1.0 / 47, 1.0 / 48,
    1.0 / 49, 1.0 / 50, 1.0 / 51, 1.0 / 52, 1.0 / 53, 1.0 / 54, 1.0 / 55, 1.0 / 56,
    1.0 / 57, 1.0 / 58, 1.0 / 59, 1.0 / 60, 1.0 / 61, 1.0 / 62, 1.0 / 63, 1.0 / 64};

// the weight of each daughter of a split into nd: w times fl64(1/nd), one
// FP64 multiply (the FP32 path's rule; an FP64 division is about ten
// instructions on GB300's narrow FP64 pipe)
__device__ __forceinline__ double daughter_weight(double w, uint32_t nd) {
    return w * (nd <= 64u ? kInvNd[nd] : 1.0 / (double)nd);
}

// The warp's queued splits [0, n), one per lane: the split count, the
// daughters' weight, the daughters' lineage keys (into the warp's key stack,
// consecutive in lane order, when it has room for all of them: the warp
// draws them round by round, daughter j of every split in round j) and the
// parent pushed to the daughter stack with its daughters 0..nd-1 (or queued
// as records when the stack is full); returns the daughters created beyond
// the parents (this lane's share).  Whole warp, converged.
__device__ __noinline__ uint32_t process_splits(const TrackArgs<float>& a, WarpShared& ws, int wp, unsigned n,
                                                   unsigned lane, int S) {
    P32 b;
    uint32_t nd = 0;
    if (lane < n) {
        b.xo = ws.sx[wp][lane];
        b.mu = ws.smu[wp][lane];
        b.tau = ws.stau[wp][lane];
        b.cell = ws.scell[wp][lane];
        b.id = ws.sid[wp][lane];
        b.e = ws.se[wp][lane];
        b.lin = ws.slin[wp][lane];
        const double w = ws.sw[wp][lane];
        nd = split_count(a, w, a.ww_c[b.cell]);
        if (nd) {
            b.w = daughter_weight(w, nd);
            b.tw = tally_weight_bits(b.w, S);
        }
    }
    uint32_t incl = nd;  // daughters of lanes 0..lane
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const int kt = ws.ktop[wp];
    const bool keyed = total <= (uint32_t)(KSTACK - kt);  // uniform over the warp
    const uint32_t kb = (uint32_t)kt + incl - nd;
    if (keyed) {
        const uint32_t rounds = __reduce_max_sync(0xffffffffu, nd);
        for (uint32_t j = 0; j < rounds; ++j)
            if (j < nd) ws.key[wp][kb + j] = lineage_hash(b.lin, b.e, j);
    }
    bool kept = false;  // pushed with its keys
    if (nd) {
        if (stack_push(ws, wp, b, 0u, nd, keyed ? (uint16_t)kb : NO_KEYS))
            kept = keyed;
        else
            queue_daughters(a, b, 0u, nd, 0u);
    }
    // the key stack ends after the keys of the last parent that kept them
    // (the keys of parents that went to the record queue are dropped)
    const uint32_t kend = __reduce_max_sync(0xffffffffu, kept ? kb + nd : 0u);
    __syncwarp();
    if (lane == 0 && keyed) ws.ktop[wp] = max(kt, (int)kend);
    __syncwarp();
    return nd ? nd - 1 : 0u;
}

// Hands daughters from the warp's stack (top entry first) to the lanes in
// `need` until the stack is empty or each of them has one.  A daughter whose
// lineage key was drawn with its split starts with its first event; the
// others take the lineage step.  An entry's last daughter taken frees its
// keys.  Whole warp, converged.
__device__ __forceinline__ void pop_daughters(WarpShared& ws, int wp, unsigned& need, unsigned lane, unsigned lt,
                                              P32& q, uint32_t& jd, bool& fresh, int& mode, bool& have, bool& got) {
    while (need) {
        const int top = *(volatile int*)&ws.top[wp];
        if (top <= 0) break;
        const int t = top - 1;
        const uint32_t jn0 = ws.jn[wp][t], je = ws.je[wp][t];
        const uint16_t kbt = ws.kb[wp][t];
        const uint32_t fr = jn0 & FRESH_DIRECTION, jn = jn0 & ~FRESH_DIRECTION;
        const uint32_t left = je - jn;
        const uint32_t take = min((uint32_t)__popc(need), left);
        const uint32_t rank = __popc(need & lt);
        const bool mine = ((need >> lane) & 1u) && rank < take;
        if (mine) {
            q.xo = ws.xo[wp][t];
            q.mu = ws.mu[wp][t];
            q.tau = ws.tau[wp][t];
            q.w = ws.w[wp][t];
            q.tw = ws.tw[wp][t];
            q.cell = ws.cell[wp][t];
            q.id = ws.id[wp][t];
            jd = jn + rank;
            fresh = fr != 0;
            if (kbt != NO_KEYS) {
                q.lin = ws.key[wp][kbt + jd];
                q.e = 0;
                mode = fresh ? M_DIRECTION : M_EVENT;
            } else {
                q.lin = ws.lin[wp][t];
                q.e = ws.e[wp][t];
                mode = M_LINEAGE;
            }
            have = true;
            got = true;
        }
        __syncwarp();
        if (lane == 0) {
            if (take == left) {
                ws.top[wp] = t;
                if (kbt != NO_KEYS) ws.ktop[wp] = kbt;
            } else {
                ws.jn[wp][t] = (jn + take) | fr;
            }
        }
        need &= ~__ballot_sync(0xffffffffu, mine);
        __syncwarp();
    }
}

struct BlockScalars {
    double wbar, tscale;
    float twbar;  // the start weight's tally weight
    int S;        // the tally scale's exponent
};

// One event of a live track: the flight to the nearest of census, the
// cell edge and a collision, its track-length tallies (block-private J, F
// and batch-row words; another batch's row and the leak tallies in global
// memory), the move and the outcome, with the window test after a crossing
// or a scatter.  Sets the outcome bits in eb; a track that ended (census,
// leak, absorption, roulette kill) or splits gets have = false (a split
// keeps e = the split's event index, the key of its daughters' lineages,
// and the caller places its daughters), e_end the event count of an ended
// track.  The extra particles of a multiplying collision go to
// emit_secondaries(state at the collision, n) (daughters 1..n-1).
template <class EmitSecondaries>
__device__ __forceinline__ void take_event(const TrackArgs<float>& a, const BlockScalars& bs, const int ww_on,
                                           unsigned* tl32, const int qb, const int b_blk, const uint32_t r[4],
                                           const uint32_t r2[4], P32& q, bool& have, unsigned& eb,
                                           uint32_t& e_end, EmitSecondaries&& emit_secondaries) {
    const int I = a.I;
    unsigned* sJl = tl32;
    unsigned* sJh = tl32 + I;
    unsigned* sFl = tl32 + 2 * I;
    unsigned* sFh = tl32 + 3 * I;
    unsigned* sBl = tl32 + 4 * I;
    unsigned* sBh = tl32 + 5 * I;
    const float uf = u01f(r[1]);
    const float uc = u01f(r[3]);
    const int k = q.cell;
    const float4 cf = __ldg(&a.cellf[k]);  // width, 1/Sigma_t, c
    const float dxk = cf.x;
    // the hardware base-2 logarithm times ln 2: within 2^-21.41 absolute for
    // u in [1/2, 1) and 3 ulp below (the CUDA intrinsic's stated bounds)
    const float dcoll = -__logf(uf) * cf.y;
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
    const float f3 = 1.0f / 3.0f - q.mu * q.mu;
    {
        const long long c0 = fx_mul24(q.tw, l);
        sadd_split(&sJl[k], &sJh[k], fx_mul24(q.tw, l * q.mu));
        sadd_split(&sFl[k], &sFh[k], fx_mul24(q.tw, l * f3));
        if (qb == b_blk)
            sadd_split(&sBl[k], &sBh[k], c0);
        else
            add128(&a.batch[(long long)qb * I + k], c0);
    }
    if (ev != 1) q.xo = fminf(fmaxf(fmaf(q.mu, l, q.xo), 0.0f), dxk);
    q.tau = (ev == 0) ? 0.0f : q.tau - l;
    const uint32_t e_ev = q.e;
    q.e = q.e + 1;
    bool ww = false;
    if (ev == 0) {
        // census: staged below (its tallies come from the census pass)
        eb |= 1u << EB_CENSUS;
        e_end = q.e;
        have = false;
    } else if (ev == 1) {
        eb |= 1u << EB_CROSS;
        const int nk = (q.mu > 0.0f) ? k + 1 : k - 1;
        if (nk < 0 || nk >= I) {
            const int side = (nk < 0) ? 0 : 1;
            const int bc = side ? a.bc_r : a.bc_l;
            if (bc == 0) {
                const double amu = fabs((double)q.mu);
                const double ia = (amu < GRAZE_MU) ? 2.0 / GRAZE_MU : 1.0 / amu;
                const double wi = q.w * ia;
                const double dm2 = (double)q.mu * (double)q.mu;
                add128(&a.bnd[3 * side + 0], to_fixed(wi, bs.tscale));
                add128(&a.bnd[3 * side + 1], to_fixed(wi * (1.0 / 3.0 - dm2), bs.tscale));
                add128(&a.bnd[3 * side + 2], to_fixed(wi * (0.5 - amu), bs.tscale));
                eb |= 1u << EB_LEAK;
                e_end = q.e;
                have = false;
            } else {
                q.mu = -q.mu;
                q.inv_mu = -q.inv_mu;
                q.xo = side ? dxk : 0.0f;
                eb |= 1u << EB_REFL;
                ww = true;
            }
        } else {
            q.cell = nk;
            q.xo = (q.mu > 0.0f) ? 0.0f : __ldg(&a.cellf[nk]).x;
            ww = true;
        }
    } else {
        eb |= 1u << EB_COLL;
        // the collision emits floor(c) + [u_c < c - floor(c)] particles (mean c)
        const float cfl = floorf(cf.z);
        const uint32_t nsec = (uint32_t)cfl + ((uc < cf.z - cfl) ? 1u : 0u);
        if (nsec == 0) {
            eb |= 1u << EB_ABS;
            e_end = q.e;
            have = false;
        } else {
            q.mu = 2.0f * u01f(r2[1]) - 1.0f;
            q.inv_mu = __frcp_rn(q.mu);
            if (nsec > 1) {
                // the other emitted particles: daughters with their
                // own lineages and isotropic directions
                P32 b = q;
                b.e = e_ev | SECONDARY_EVENT;
                emit_secondaries(b, nsec);
            }
            ww = true;
        }
    }
    if (ww && ww_on) {
        const int kc = q.cell;
        const double2 hl = __ldg(&a.ww_hl[kc]);  // ceiling, floor
        if (dgt(q.w, hl.x)) {
            // a split: the caller places the daughters
            eb |= 1u << EB_SPLIT;
            q.e = e_ev;
            have = false;
        } else if (dgt(hl.y, q.w)) {
            const double ctr = a.ww_c[kc];
            // survive iff u < w / ww, tested as u ww < w (no divide)
            const double ur = u01(r2[2], r2[3]);
            if (ur * ctr < q.w) {
                q.w = ctr;
                q.tw = tally_weight_bits(ctr, bs.S);
                eb |= 1u << EB_RSURV;
            } else {
                eb |= 1u << EB_RKILL;
                e_end = q.e;
                have = false;
            }
        }
    }
}

// Items [item0, item_end) of the block, from a block-shared counter; wave 0
// items are start-bank particles, later waves' items records.
__device__ __forceinline__ void run_warp(const TrackArgs<float>& a, const long long item0, const long long item_end,
                                         unsigned* s_next, const int b_blk, const uint32_t b_end, unsigned* tl32,
                                         WarpShared& ws, const BlockScalars& bs, unsigned long long* s_stats) {
    const int I = a.I;
    const uint32_t k0 = a.sd->k0, k1 = a.sd->k1;
    const int ww_on = a.sd->ww_on;
    const int birth = a.sd->birth;
    const bool ring_on = a.from_bank && !birth;  // start-bank records prefetched
    const unsigned lane = lane_id();
    const int wp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;

    if (ring_on) {
        unsigned b = 0;
        if (lane == 0) b = atomicAdd(s_next, 64u);
        b = __shfl_sync(0xffffffffu, b, 0);
        const int n0 = (int)max(0LL, min(32LL, item_end - (item0 + (long long)b)));
        const int n1 = (int)max(0LL, min(32LL, item_end - (item0 + (long long)b + 32)));
        ring_fetch(ws.ring[wp][0], a.bank, item0 + (long long)b, n0, lane);
        ring_fetch(ws.ring[wp][1], a.bank, item0 + (long long)b + 32, n1, lane);
        if (lane == 0) {
            ws.rb[wp][0] = b;
            ws.rb[wp][1] = b + 32u;
            ws.rn[wp][0] = n0;
            ws.rn[wp][1] = n1;
            ws.rcs[wp] = 0;
            ws.rpos[wp] = 0;
        }
        asm volatile("cp.async.wait_group 1;\n" ::);
        __syncwarp();
    }

    P32 q;
    bool have = false;
    int mode = M_EVENT;
    uint32_t jd = 0;     // M_LINEAGE: the daughter index hashed into the lineage
    bool fresh = false;  // M_LINEAGE: then draw an own direction
    bool items_left = true;
    int evs = 0;
    int qb = 0;
    unsigned cfill = 0;            // staged census particles of the warp
    unsigned sqn = 0;              // queued splits of the warp
    unsigned long long mycnt = 0;  // lane k < EB_COUNT: counter kLaneStat[k]; then daughters, max events
    for (;;) {
        uint32_t nadd = 0;    // daughters created in this iteration (this lane's share)
        // ---- refill: daughters from the warp's stack, then new items ----
        unsigned need = __ballot_sync(0xffffffffu, !have);
        bool got = false;  // this lane took a new track this iteration
        pop_daughters(ws, wp, need, lane, lt, q, jd, fresh, mode, have, got);
        if (need && ring_on) {
            // prefetched start-bank records; when the current slot runs out,
            // the other (already fetched) slot takes over and the emptied one
            // fetches the next 32 items
            int cs = ws.rcs[wp], cpos = ws.rpos[wp];
            while (need) {
                const int avail = ws.rn[wp][cs] - cpos;
                if (avail <= 0) {
                    if (ws.rn[wp][cs ^ 1] == 0) break;  // no items left
                    ring_wait_all();
                    __syncwarp();
                    unsigned b = 0;
                    if (lane == 0) b = atomicAdd(s_next, 32u);
                    b = __shfl_sync(0xffffffffu, b, 0);
                    const int nn = (int)max(0LL, min(32LL, item_end - (item0 + (long long)b)));
                    ring_fetch(ws.ring[wp][cs], a.bank, item0 + (long long)b, nn, lane);
                    __syncwarp();
                    if (lane == 0) {
                        ws.rb[wp][cs] = b;
                        ws.rn[wp][cs] = nn;
                    }
                    __syncwarp();
                    cs ^= 1;
                    cpos = 0;
                    continue;
                }
                const unsigned take = min((unsigned)__popc(need), (unsigned)avail);
                const unsigned rank = __popc(need & lt);
                const bool mine = ((need >> lane) & 1u) && rank < take;
                if (mine) {
                    const BankRec<float> r = ws.ring[wp][cs][cpos + (int)rank];
                    q.id = (uint32_t)(item0 + (long long)ws.rb[wp][cs] + cpos + (long long)rank);
                    q.lin = 0;
                    q.e = 0;
                    q.tau = a.tau0f;
                    q.w = bs.wbar;
                    q.tw = bs.twbar;
                    q.xo = r.x;
                    q.mu = r.mu;
                    q.cell = r.cell;
                    mode = M_EVENT;
                    have = true;
                    got = true;
                }
                cpos += (int)take;
                need &= ~__ballot_sync(0xffffffffu, mine);
            }
            __syncwarp();
            if (lane == 0) {
                ws.rcs[wp] = cs;
                ws.rpos[wp] = cpos;
            }
        } else if (need && items_left) {
            const unsigned k = __popc(need);
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(s_next, k);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (item0 + (long long)base + k >= item_end) items_left = false;
            const long long i = item0 + (long long)base + (long long)__popc(need & lt);
            const bool took = ((need >> lane) & 1u) && i < item_end;
            if (took) {
                mode = M_EVENT;
                if (a.from_bank) {  // the pulse (step 1)
                    q.id = (uint32_t)i;
                    q.lin = 0;
                    q.e = 0;
                    q.tau = a.tau0f;
                    q.w = bs.wbar;
                    q.tw = bs.twbar;
                    mode = M_BIRTH;
                } else {
                    q.xo = a.rin.x[i];
                    q.mu = a.rin.mu[i];
                    q.tau = a.rin.tau[i];
                    q.w = a.rin.w[i];
                    q.tw = tally_weight_bits(q.w, bs.S);
                    q.cell = a.rin.cell[i];
                    q.id = a.rin.id[i];
                    q.lin = a.rin.lin[i];
                    q.e = a.rin.e[i];
                    const uint32_t jc = a.rin.jcount[i];
                    if (jc) {
                        // a chunk of daughters: this lane takes the first, the
                        // rest go to the warp's stack (or back to the queue)
                        const uint32_t js = a.rin.jstart[i];
                        const uint32_t j0 = js & ~FRESH_DIRECTION;
                        if (jc > 1 && !stack_push(ws, wp, q, js + 1u, j0 + jc, NO_KEYS))
                            queue_daughters(a, q, j0 + 1u, j0 + jc, js & FRESH_DIRECTION);
                        jd = j0;
                        fresh = (js & FRESH_DIRECTION) != 0;
                        mode = M_LINEAGE;
                    }
                }
                have = true;
                got = true;
            }
            need &= ~__ballot_sync(0xffffffffu, took);
        }
        if (need && sqn) {
            // lanes still without work: the queued splits' daughters
            nadd += process_splits(a, ws, wp, sqn, lane, bs.S);
            sqn = 0;
            pop_daughters(ws, wp, need, lane, lt, q, jd, fresh, mode, have, got);
        }
        if (got) {
            evs = 0;
            // the block's range lies in batch b_blk up to id b_end (at most
            // a few ids of a range reach the next batch)
            qb = (q.id >= (uint32_t)item0 && q.id < b_end) ? b_blk : batch_of(q.id, a.B, a.N, a.batch_m);
            if (mode == M_EVENT) q.inv_mu = __frcp_rn(q.mu);  // the correctly rounded 1/mu
        }
        if (!__any_sync(0xffffffffu, have)) {
            if (!sqn) break;
            continue;  // the queued splits go to the lanes at the next refill
        }
        // ---- daughters taken in this refill without a lineage key: their
        // keys (one Philox block for the warp), so that they take their
        // first event now ----
        if (__any_sync(0xffffffffu, have && mode == M_LINEAGE)) {
            const uint64_t nl = lineage_hash(q.lin, q.e, jd);
            if (have && mode == M_LINEAGE) {
                q.lin = nl;
                q.e = 0;
                mode = fresh ? M_DIRECTION : M_EVENT;
                if (mode == M_EVENT) q.inv_mu = __frcp_rn(q.mu);
            }
        }

        unsigned eb = 0;      // outcome bits
        uint32_t e_end = 0;   // event count of a track that ended
        if (have && mode == M_EVENT) {
            if (evs == a.emax) {  // past the event budget: a continuation record
                push_record(a, q, q.w, q.e, 0u, 0u, warp_reserve(a.rout.count));
                have = false;
            } else if (q.e >= MAX_EVENTS) {
                atomicOr(a.err, ERR_EVENTS);
                have = false;
            }
        }
        // ---- the iteration's Philox blocks, all lanes at once ----
        uint32_t r[4], r2[4];
        if (mode == M_EVENT) {
            r[0] = q.id;
            r[1] = (uint32_t)q.lin;
            r[2] = (uint32_t)(q.lin >> 32);
            r[3] = 2u * q.e;
        } else if (mode == M_DIRECTION) {
            r[0] = q.id;
            r[1] = (uint32_t)q.lin;
            r[2] = (uint32_t)(q.lin >> 32);
            r[3] = 0xFFFFFFFEu;
        } else {
            r[0] = q.id;
            r[1] = 0u;
            r[2] = 0u;
            r[3] = 0xFFFFFFFFu;
        }
        r2[0] = q.id;
        r2[1] = (uint32_t)q.lin;
        r2[2] = (uint32_t)(q.lin >> 32);
        r2[3] = 2u * q.e + 1u;
        philox_pair(r, r2, k0, k1, k0, k1);

        if (have && mode != M_EVENT) {
            // ---- a setup step of a new track ----
            if (mode == M_DIRECTION) {
                q.mu = 2.0f * u01f(r[1]) - 1.0f;
                mode = M_EVENT;
            } else {  // the pulse: isotropic birth direction, mirrored into a reflecting wall's side
                q.mu = 2.0f * u01f(r[1]) - 1.0f;
                const double x = a.src_x;
                if (x <= a.edges[0] && q.mu < 0.0f && a.bc_l == 1) q.mu = -q.mu;
                if (x >= a.edges[I] && q.mu > 0.0f && a.bc_r == 1) q.mu = -q.mu;
                q.cell = (q.mu < 0.0f) ? a.birth_cell_neg : a.birth_cell_pos;
                q.xo = (float)(x - a.edges[q.cell]);
                mode = M_EVENT;
            }
            if (mode == M_EVENT) q.inv_mu = __frcp_rn(q.mu);
        } else if (have) {
            // ---- one event ----
            ++evs;
            take_event(a, bs, ww_on, tl32, qb, b_blk, r, r2, q, have, eb, e_end, [&](const P32& b, uint32_t nsec) {
                if (!stack_push(ws, wp, b, 1u | FRESH_DIRECTION, nsec, NO_KEYS))
                    queue_daughters(a, b, 1u, nsec, FRESH_DIRECTION);
                nadd += nsec - 1;
            });
        }
        __syncwarp();
        // ---- splits of the iteration: queued, processed a batch at a time ----
        {
            const unsigned sm_ = __ballot_sync(0xffffffffu, (eb >> EB_SPLIT) & 1u);
            const unsigned ns = __popc(sm_);
            if (ns) {
                if (sqn + ns > 32u) {
                    nadd += process_splits(a, ws, wp, sqn, lane, bs.S);
                    sqn = 0;
                }
                if ((sm_ >> lane) & 1u) {
                    const unsigned pos = sqn + __popc(sm_ & lt);
                    ws.sx[wp][pos] = q.xo;
                    ws.smu[wp][pos] = q.mu;
                    ws.stau[wp][pos] = q.tau;
                    ws.sw[wp][pos] = q.w;
                    ws.scell[wp][pos] = q.cell;
                    ws.sid[wp][pos] = q.id;
                    ws.se[wp][pos] = q.e;
                    ws.slin[wp][pos] = q.lin;
                }
                sqn += ns;
                __syncwarp();
                if (sqn >= SPLIT_BATCH) {
                    nadd += process_splits(a, ws, wp, sqn, lane, bs.S);
                    sqn = 0;
                }
            }
        }
        // ---- census particles of the iteration: staged, written 32 at a time ----
        {
            const unsigned cm = __ballot_sync(0xffffffffu, (eb >> EB_CENSUS) & 1u);
            const unsigned nc = __popc(cm);
            if (nc) {
                if (cfill + nc > 32u) {
                    census_flush(a, ws, wp, cfill, lane);
                    cfill = 0;
                }
                if ((cm >> lane) & 1u) {
                    const unsigned pos = cfill + __popc(cm & lt);
                    ws.cx[wp][pos] = q.xo;
                    ws.cmu[wp][pos] = q.mu;
                    ws.cw[wp][pos] = q.w;
                    ws.ccell[wp][pos] = q.cell;
                    ws.cid[wp][pos] = q.id;
                    ws.clw[wp][pos] = LinW{q.lin, comb_weight(fixed_bits(q.w, bs.S), a.comb_shift)};
                }
                cfill += nc;
                __syncwarp();
            }
        }
        // ---- the iteration's counts, summed over the warp ----
        {
            // bit k of the outcome goes to bit 6k of a word (five 6-bit fields
            // per word: a field sums at most 32 lanes); a multiply places
            // non-overlapping 5-bit copies 5 bits apart, so bit k of copy k
            // lands at 6k
            const unsigned wlo = ((eb & 0x1Fu) * 0x108421u) & 0x1041041u;
            const unsigned whi = (((eb >> 5) & 0xFu) * 0x8421u) & 0x41041u;
            const unsigned slo = __reduce_add_sync(0xffffffffu, wlo);
            const unsigned shi = __reduce_add_sync(0xffffffffu, whi);
            const unsigned sd = __reduce_add_sync(0xffffffffu, nadd);
            const unsigned smax = __reduce_max_sync(0xffffffffu, e_end);
            const unsigned f = ((lane < 5u ? slo : shi) >> (6u * (lane < 5u ? lane : lane - 5u))) & 63u;
            const unsigned add = lane < (unsigned)EB_COUNT ? f : (lane == (unsigned)LANE_DAUGHTERS ? sd : 0u);
            mycnt += add;
            if (lane == (unsigned)LANE_MAXEV) mycnt = max(mycnt, (unsigned long long)smax);
        }
    }
    if (cfill) census_flush(a, ws, wp, cfill, lane);
    if (ring_on) ring_wait_all();  // no copy outlives the block
    // the warp's counts into the block's
    if (lane < (unsigned)EB_COUNT) {
        if (mycnt) atomicAdd(&s_stats[kLaneStat[lane]], mycnt);
    } else if (lane == (unsigned)LANE_DAUGHTERS) {
        if (mycnt) atomicAdd(&s_stats[ST_DAUGHTERS], mycnt);
    } else if (lane == (unsigned)LANE_MAXEV) {
        if (mycnt) atomicMax(&s_stats[ST_MAX_EVENTS], mycnt);
    }
}

// the block-private J and F rows (32-bit halves) into the global 128-bit
// tallies
__device__ __forceinline__ void flush_jf(const unsigned* tl32, int I, Acc128* tl) {
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const long long vJ = (long long)(((unsigned long long)tl32[I + i] << 32) | tl32[i]);
        const long long vF = (long long)(((unsigned long long)tl32[3 * I + i] << 32) | tl32[2 * I + i]);
        if (vJ != 0) add128(&tl[I + i], vJ);
        if (vF != 0) add128(&tl[2 * I + i], vF);
    }
}

// the block-private batch row into the global batch tally of batch b (and
// cleared when `clear`)
__device__ __forceinline__ void flush_batch_row(unsigned* tl32, int I, Acc128* batch, int b, bool clear) {
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const long long vB = (long long)(((unsigned long long)tl32[5 * I + i] << 32) | tl32[4 * I + i]);
        if (vB != 0) add128(&batch[(long long)b * I + i], vB);
        if (clear) {
            tl32[4 * I + i] = 0;
            tl32[5 * I + i] = 0;
        }
    }
}

// the block's counts into the problem's (segments and scatters follow from
// the event counts); a barrier first and last
__device__ __forceinline__ void flush_block_stats(unsigned long long* s_stats, unsigned long long* stats) {
    __syncthreads();
    if (threadIdx.x == 0) {
        s_stats[ST_SEGMENTS] = s_stats[ST_CENSUS] + s_stats[ST_CROSSINGS] + s_stats[ST_COLLISIONS];
        s_stats[ST_SCATTERS] = s_stats[ST_COLLISIONS] - s_stats[ST_ABSORBED];
    }
    __syncthreads();
    if (threadIdx.x < ST_COUNT && s_stats[threadIdx.x]) {
        if (threadIdx.x == ST_MAX_EVENTS)
            atomicMax(&stats[ST_MAX_EVENTS], s_stats[threadIdx.x]);
        else
            atomicAdd(&stats[threadIdx.x], s_stats[threadIdx.x]);
    }
    __syncthreads();
}

// Three resident blocks of 256 threads per SM (85 registers): measured at the
// workload, four blocks (64 registers) executed 4.5% more instructions
// (register pressure) and ran 7% slower, two blocks (128 registers) 11% fewer
// instructions but too few warps to hide the loop's latencies (5% slower).
__global__ void __launch_bounds__(TRACK_THREADS, 3) track32_kernel(TrackArgs<float> a) {
    extern __shared__ long long sm[];  // ROWS32 rows of I 64-bit words, as 32-bit halves
    __shared__ unsigned s_next;
    __shared__ WarpShared s_ws;
    __shared__ unsigned long long s_stats[ST_COUNT];
    __shared__ BlockScalars s_bs;
    const int I = a.I;
    unsigned* tl32 = reinterpret_cast<unsigned*>(sm);
    if (threadIdx.x == 0) {
        s_next = 0;
        s_bs.wbar = a.sd->wbar;
        s_bs.tscale = a.sd->tscale;
        s_bs.twbar = tally_weight_bits(a.sd->wbar, a.sd->S);
        s_bs.S = a.sd->S;
    }
    if (threadIdx.x < WARPS) {
        s_ws.top[threadIdx.x] = 0;
        s_ws.ktop[threadIdx.x] = 0;
    }
    if (threadIdx.x < ST_COUNT) s_stats[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < 2 * ROWS32 * I; i += blockDim.x) tl32[i] = 0;
    __syncthreads();
    const long long n_in = a.from_bank ? (long long)a.sd->nbank : (long long)*a.rin.count;
    const long long n_use = (!a.from_bank && n_in > a.rin.cap) ? a.rin.cap : n_in;
    // each block takes a contiguous range: of [bank_lo, bank_hi) in wave 0,
    // so that nearly all of its segments fall in one variance batch (kept in
    // shared memory), or of the record queue in later waves
    const long long lo = a.from_bank ? a.bank_lo : 0;
    const long long hi = a.from_bank ? min(n_use, a.bank_hi) : n_use;
    const long long len = hi > lo ? hi - lo : 0;
    const long long chunk = (len + gridDim.x - 1) / gridDim.x;
    const long long first = lo + (long long)blockIdx.x * chunk;
    const long long last = min(hi, first + chunk);
    int b_blk = -1;
    uint32_t b_end = 0;  // first id past batch b_blk (0: none of the range)
    if (a.from_bank && first < hi) {
        b_blk = batch_of((uint32_t)first, a.B, a.N, a.batch_m);
        // ids with floor(id B / N) == b_blk end at ceil((b_blk + 1) N / B)
        b_end = (uint32_t)min((long long)UINT32_MAX, ((long long)(b_blk + 1) * a.N + a.B - 1) / a.B);
    }
    const BlockScalars bs = s_bs;
    run_warp(a, first, last, &s_next, b_blk, b_end, tl32, s_ws, bs, s_stats);
    __syncthreads();
    // block-private tallies into the global ones (J, F; the batch row)
    flush_jf(tl32, I, a.tl);
    if (b_blk >= 0) flush_batch_row(tl32, I, a.batch, b_blk, false);
    flush_block_stats(s_stats, a.stats);
}

// Persistent batched variant: blocks pop tiles (problem, id range) from a
// device counter and run the warp-synchronous loop over each tile's items;
// the block-private tallies and counts are flushed when a block moves to
// another problem, the batch row after every tile.  A warp leaves a tile
// only with its daughter stack empty, so the tile's barrier waits for no
// queued work.
__global__ void __launch_bounds__(TRACK_THREADS, 2) track32_kernel_batch(const TrackArgs<float>* args,
                                                                         BatchPlan plan) {
    extern __shared__ long long sm[];  // ROWS32 rows of Imax 64-bit words, as 32-bit halves
    __shared__ WarpShared s_ws;
    __shared__ TrackArgs<float> A;
    __shared__ BlockScalars s_bs;
    __shared__ unsigned long long s_stats[ST_COUNT];
    __shared__ long long s_t;
    __shared__ int s_p;
    __shared__ unsigned s_next;
    unsigned* tl32 = reinterpret_cast<unsigned*>(sm);
    if (threadIdx.x < WARPS) {
        s_ws.top[threadIdx.x] = 0;
        s_ws.ktop[threadIdx.x] = 0;
    }
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
                flush_jf(tl32, Ic, A.tl);
                flush_block_stats(s_stats, A.stats);
            }
            if (p < 0) break;
            if (threadIdx.x == 0) A = args[p];
            __syncthreads();
            if (threadIdx.x == 0) {
                s_bs.wbar = A.sd->wbar;
                s_bs.tscale = A.sd->tscale;
                s_bs.twbar = tally_weight_bits(A.sd->wbar, A.sd->S);
                s_bs.S = A.sd->S;
            }
            if (threadIdx.x < ST_COUNT) s_stats[threadIdx.x] = 0;
            cur = p;
            Ic = A.I;
            for (int i = threadIdx.x; i < 2 * ROWS32 * Ic; i += blockDim.x) tl32[i] = 0;
            __syncthreads();
        }
        const long long n_in = A.from_bank ? (long long)A.sd->nbank : (long long)*A.rin.count;
        const long long n_use = (!A.from_bank && n_in > A.rin.cap) ? A.rin.cap : n_in;
        const long long i0 = (t - plan.tile_off[p]) * (long long)plan.tile;
        const long long i1 = min(n_use, i0 + (long long)plan.tile);
        int b_tile = -1;
        uint32_t b_end = 0;
        if (A.from_bank && i0 < n_use) {
            b_tile = batch_of((uint32_t)i0, A.B, A.N, A.batch_m);
            b_end = (uint32_t)min((long long)UINT32_MAX, ((long long)(b_tile + 1) * A.N + A.B - 1) / A.B);
        }
        const BlockScalars bs = s_bs;
        run_warp(A, i0, i1, &s_next, b_tile, b_end, tl32, s_ws, bs, s_stats);
        __syncthreads();
        if (b_tile >= 0) flush_batch_row(tl32, Ic, A.batch, b_tile, true);
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------
// Event-based variant of wave 0 (start-bank particles).
//
// Each block of EV_THREADS threads keeps its live particles in a ring in
// shared memory and advances them one event per pass: thread t takes the
// t-th particle from the ring's head, draws its Philox blocks, takes its
// event and tallies the flight (take_event, the warp loop's arithmetic, so
// both kernels give the same tallies, census and records bit for bit).  A
// block-wide exclusive scan of the threads' output counts then appends the
// survivors and the daughters of splits at the ring's tail and gives the
// pass's census particles consecutive census slots (one reservation per
// pass); the daughters are made by their whole warp, daughter 32 r + l of
// the warp's splits by lane l in round r (parent found by a binary search
// over the warp's prefix of daughter counts, its state taken by shuffles,
// its lineage key drawn by the lane).  Fresh particles from the block's
// contiguous range of the start bank keep at least one pass of work in the
// ring.  Outputs beyond the ring's room wait in the block's spill, a FIFO in
// the block's own slice of the record queue that wave 0 leaves idle (it reads
// no records); the refill drains the spill before it takes fresh particles,
// so a block tracks its own overflow.  Only what the slice cannot hold, the
// daughters of a split into more particles than a ring holds, and the extra
// particles of a multiplying collision go to the record queue (the warp loop
// takes them in the next wave).  Every event of a pass is one SIMT lane's
// work, so lanes idle only at divergent outcomes and in a block's last
// passes; the price is the ring's shared-memory traffic (48 bytes read and
// written per event) and three block barriers per pass, which the SM's other
// blocks hide (small blocks, several per SM: a barrier waits for fewer
// warps).
// ---------------------------------------------------------------------------
constexpr int EV_THREADS = 256;
constexpr int EV_WARPS = EV_THREADS / 32;
// up to four blocks per SM (registers are budgeted for four); fewer where a
// large mesh's tallies leave four blocks less than two passes of ring
constexpr int EV_MAX_BLOCKS_PER_SM = 4;
constexpr int EV_REC_BYTES = 48;  // ring bytes per particle

// the ring's field arrays over a runtime capacity (the shared memory the
// tallies leave), 8-byte fields first
struct EvRing {
    double* w;
    uint64_t* lin;
    float *x, *mu, *imu, *tau, *tw;
    int* cell;
    uint32_t *id, *e;
    __device__ EvRing(void* base, int cap) {
        char* b = reinterpret_cast<char*>(base);
        w = reinterpret_cast<double*>(b);
        lin = reinterpret_cast<uint64_t*>(b + 8 * (size_t)cap);
        x = reinterpret_cast<float*>(b + 16 * (size_t)cap);
        mu = x + cap;
        imu = mu + cap;
        tau = imu + cap;
        tw = tau + cap;
        cell = reinterpret_cast<int*>(tw + cap);
        id = reinterpret_cast<uint32_t*>(cell + cap);
        e = id + cap;
    }
    __device__ __forceinline__ void put(int s, const P32& q) const {
        w[s] = q.w;
        lin[s] = q.lin;
        x[s] = q.xo;
        mu[s] = q.mu;
        imu[s] = q.inv_mu;
        tau[s] = q.tau;
        tw[s] = q.tw;
        cell[s] = q.cell;
        id[s] = q.id;
        e[s] = q.e;
    }
    __device__ __forceinline__ void get(int s, P32& q) const {
        q.w = w[s];
        q.lin = lin[s];
        q.xo = x[s];
        q.mu = mu[s];
        q.inv_mu = imu[s];
        q.tau = tau[s];
        q.tw = tw[s];
        q.cell = cell[s];
        q.id = id[s];
        q.e = e[s];
    }
};

// start particle i (of the bank, or of the pulse at birth)
__device__ __forceinline__ void ev_start(const TrackArgs<float>& a, const BlockScalars& bs, int birth, uint32_t k0,
                                         uint32_t k1, long long i, P32& q) {
    q.id = (uint32_t)i;
    q.lin = 0;
    q.e = 0;
    q.tau = a.tau0f;
    q.w = bs.wbar;
    q.tw = bs.twbar;
    if (birth) {
        // the pulse: isotropic birth direction, mirrored into a reflecting wall's side
        uint32_t r[4] = {q.id, 0u, 0u, 0xFFFFFFFFu};
        philox4x32_10(r, k0, k1);
        q.mu = 2.0f * u01f(r[1]) - 1.0f;
        const double x = a.src_x;
        if (x <= a.edges[0] && q.mu < 0.0f && a.bc_l == 1) q.mu = -q.mu;
        if (x >= a.edges[a.I] && q.mu > 0.0f && a.bc_r == 1) q.mu = -q.mu;
        q.cell = (q.mu < 0.0f) ? a.birth_cell_neg : a.birth_cell_pos;
        q.xo = (float)(x - a.edges[q.cell]);
    } else {
        const BankRec<float> r = a.bank[i];
        q.xo = r.x;
        q.mu = r.mu;
        q.cell = r.cell;
    }
    q.inv_mu = __frcp_rn(q.mu);  // the correctly rounded 1/mu
}

__device__ __forceinline__ int ring_slot(int s, int cap) { return s >= cap ? s - cap : s; }

// a spilled particle in slot i of the idle record queue, every field of the
// ring's copy kept (1/mu and the tally weight in the chunk words, which a
// spilled particle does not use)
__device__ __forceinline__ void spill_put(const RecQ<float>& s, long long i, const P32& q) {
    s.x[i] = q.xo;
    s.mu[i] = q.mu;
    s.tau[i] = q.tau;
    s.w[i] = q.w;
    s.cell[i] = q.cell;
    s.id[i] = q.id;
    s.lin[i] = q.lin;
    s.e[i] = q.e;
    s.jstart[i] = __float_as_uint(q.inv_mu);
    s.jcount[i] = __float_as_uint(q.tw);
}

__device__ __forceinline__ void spill_get(const RecQ<float>& s, long long i, P32& q) {
    q.xo = s.x[i];
    q.mu = s.mu[i];
    q.tau = s.tau[i];
    q.w = s.w[i];
    q.cell = s.cell[i];
    q.id = s.id[i];
    q.lin = s.lin[i];
    q.e = s.e[i];
    q.inv_mu = __uint_as_float(s.jstart[i]);
    q.tw = __uint_as_float(s.jcount[i]);
}

__global__ void __launch_bounds__(EV_THREADS, EV_MAX_BLOCKS_PER_SM) track32_event_kernel(TrackArgs<float> a, int cap) {
    extern __shared__ long long sm[];
    __shared__ unsigned long long s_stats[ST_COUNT];
    __shared__ BlockScalars s_bs;
    __shared__ unsigned s_wsum[EV_WARPS];   // per-warp output words, then their exclusive prefixes
    __shared__ unsigned s_total;            // the pass's output word: outputs << 11 | census
    __shared__ unsigned long long s_cbase;  // the pass's first census slot
    const int I = a.I;
    unsigned* tl32 = reinterpret_cast<unsigned*>(sm);
    const EvRing R(sm + (size_t)ROWS32 * I, cap);
    const unsigned t = threadIdx.x, lane = t & 31u, wid = t >> 5;
    if (t == 0) {
        s_bs.wbar = a.sd->wbar;
        s_bs.tscale = a.sd->tscale;
        s_bs.twbar = tally_weight_bits(a.sd->wbar, a.sd->S);
        s_bs.S = a.sd->S;
    }
    if (t < ST_COUNT) s_stats[t] = 0;
    for (int i = t; i < 2 * ROWS32 * I; i += EV_THREADS) tl32[i] = 0;
    const uint32_t k0 = a.sd->k0, k1 = a.sd->k1;
    const int ww_on = a.sd->ww_on;
    const int birth = a.sd->birth;
    // the block's contiguous range of [bank_lo, min(bank_hi, size)), as in
    // the warp-loop kernel, so that nearly all its flights fall in one
    // variance batch (kept in shared memory)
    const long long n_in = (long long)a.sd->nbank;
    const long long lo = a.bank_lo, hi = min(n_in, a.bank_hi);
    const long long len = hi > lo ? hi - lo : 0;
    const long long chunk = (len + gridDim.x - 1) / gridDim.x;
    const long long first = lo + (long long)blockIdx.x * chunk;
    const long long last = min(hi, first + chunk);
    int b_blk = -1;
    uint32_t b_end = 0;
    if (first < hi) {
        b_blk = batch_of((uint32_t)first, a.B, a.N, a.batch_m);
        b_end = (uint32_t)min((long long)UINT32_MAX, ((long long)(b_blk + 1) * a.N + a.B - 1) / a.B);
    }
    __syncthreads();
    const BlockScalars bs = s_bs;
    // ring state, the same in every thread: particles [head, head + count)
    long long next = first;  // the next start particle of the range
    int head = 0, count = 0;
    // spill state, the same in every thread: particles in slots [sp_h,
    // sp_h + sp_n) (mod SC) of the block's slice; the first sp_rdy of them
    // were written before the last pass's barriers, so any thread may read
    // them (a pass's own spills become readable one pass later)
    const int SC = (int)min(a.rin.cap / (long long)gridDim.x, (long long)(INT_MAX / 2));
    const long long sbase = (long long)blockIdx.x * SC;
    int sp_h = 0, sp_n = 0, sp_rdy = 0;
    long long sp_total = 0;  // particles the block spilled
    unsigned long long mycnt = 0;  // lane k < EB_COUNT: counter kLaneStat[k]; then daughters, max events
    for (;;) {
        // ---- keep a pass of work in the ring: spilled particles first ----
        const int want = max(0, min(EV_THREADS - count, cap - count));
        const int fs = min(want, sp_rdy);
        const int add = (int)max(0LL, min((long long)(want - fs), last - next));
        if ((int)t < fs) {
            P32 q;
            const int sl = sp_h + (int)t;
            spill_get(a.rin, sbase + (sl >= SC ? sl - SC : sl), q);
            R.put(ring_slot(head + count + (int)t, cap), q);
        } else if ((int)t < fs + add) {
            P32 q;
            ev_start(a, bs, birth, k0, k1, next + ((int)t - fs), q);
            R.put(ring_slot(head + count + (int)t, cap), q);
        }
        sp_h += fs;
        if (sp_h >= SC) sp_h -= SC;
        sp_n -= fs;
        sp_rdy -= fs;
        next += add;
        count += fs + add;
        // an empty ring after the refill means an empty spill too: a pass
        // that spilled left the ring full
        if (count == 0) break;
        __syncthreads();
        // ---- the t-th particle from the head: one event ----
        const int m = min(count, EV_THREADS);
        P32 q;
        bool have = (int)t < m;
        if (have) {
            R.get(ring_slot(head + (int)t, cap), q);
            if (q.e >= MAX_EVENTS) {
                atomicOr(a.err, ERR_EVENTS);
                have = false;
            }
        } else {
            q.id = 0;
            q.lin = 0;
            q.e = 0;
        }
        uint32_t r[4] = {q.id, (uint32_t)q.lin, (uint32_t)(q.lin >> 32), 2u * q.e};
        uint32_t r2[4] = {q.id, (uint32_t)q.lin, (uint32_t)(q.lin >> 32), 2u * q.e + 1u};
        philox_pair(r, r2, k0, k1, k0, k1);
        unsigned eb = 0;
        uint32_t e_end = 0, nadd = 0, nd = 0;
        if (have) {
            const int qb = (q.id >= (uint32_t)first && q.id < b_end) ? b_blk : batch_of(q.id, a.B, a.N, a.batch_m);
            take_event(a, bs, ww_on, tl32, qb, b_blk, r, r2, q, have, eb, e_end, [&](const P32& b, uint32_t nsec) {
                queue_daughters(a, b, 1u, nsec, FRESH_DIRECTION);
                nadd += nsec - 1;
            });
            if ((eb >> EB_SPLIT) & 1u) {
                nd = split_count(a, q.w, a.ww_c[q.cell]);
                if (nd) nadd += nd - 1;
            }
        }
        // ---- outputs (a survivor, or a split's daughters) and census: slots ----
        const uint32_t nout = have ? 1u : nd;
        const unsigned cen = (eb >> EB_CENSUS) & 1u;
        // a lane reserves at most cap outputs in the scan word (EV_THREADS x
        // cap < 2^21 outputs); a split into more daughters (up to
        // MAX_DAUGHTERS) sends the rest to the record queue
        const unsigned v = (min(nout, (uint32_t)cap) << 11) | cen;
        unsigned incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const unsigned x = lane < (unsigned)EV_WARPS ? s_wsum[lane] : 0u;
            unsigned xi = x;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, xi, o);
                if ((int)lane >= o) xi += y;
            }
            if (lane < (unsigned)EV_WARPS) s_wsum[lane] = xi - x;
            if (lane == (unsigned)EV_WARPS - 1) {
                s_total = xi;
                const unsigned nc = xi & 0x7FFu;
                s_cbase = nc ? atomicAdd(a.cen.count, (unsigned long long)nc) : 0ull;
            }
        }
        __syncthreads();
        const unsigned off = s_wsum[wid] + incl - v;
        const unsigned tot = s_total;
        // the pass's inputs are free now: outputs go at the ring's tail,
        // into the room the particles not taken leave, then to the spill's
        // free slots, then to the record queue
        const int tail = ring_slot(head + count, cap);
        const int room = cap - (count - m);
        const int sp_room = SC - sp_n;
        const auto place = [&](const P32& x, unsigned long long o) {
            if (o < (unsigned long long)room) {
                R.put(ring_slot(tail + (int)o, cap), x);
            } else if (o - (unsigned long long)room < (unsigned long long)sp_room) {
                const int sl = sp_h + sp_n + (int)(o - (unsigned long long)room);
                spill_put(a.rin, sbase + (sl >= SC ? sl - SC : sl), x);
            } else {
                push_record(a, x, x.w, x.e, 0u, 0u, warp_reserve(a.rout.count));
            }
        };
        if (cen) {
            const unsigned long long slot = s_cbase + (off & 0x7FFu);
            if ((long long)slot < a.cen.cap) {
                const unsigned long long wfx = comb_weight(fixed_bits(q.w, bs.S), a.comb_shift);
                a.cen.x[slot] = q.xo;
                a.cen.mu[slot] = q.mu;
                a.cen.w[slot] = q.w;
                a.cen.cell[slot] = q.cell;
                a.cen.id[slot] = q.id;
                a.cen.lw[slot] = LinW{q.lin, wfx};
                atomicAdd(&a.gcnt[q.id], 1u);
                atomicAdd(&a.gw[q.id], wfx);
            } else {
                atomicOr(a.err, ERR_CENSUS_OVERFLOW);
            }
        }
        const unsigned o0 = off >> 11;
        if (have) place(q, o0);
        // the warp's daughters, round by round over all its lanes
        uint32_t dincl = nd;  // daughters of lanes 0..lane
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, dincl, o);
            if ((int)lane >= o) dincl += y;
        }
        const uint32_t dtot = __shfl_sync(0xffffffffu, dincl, 31);
        if (dtot) {
            double wd = 0.0;
            float twd = 0.0f;
            if (nd) {
                wd = daughter_weight(q.w, nd);
                twd = tally_weight_bits(wd, bs.S);
            }
            for (uint32_t g0 = 0; g0 < dtot; g0 += 32) {
                const uint32_t g = g0 + lane;
                // parent: the number of lanes whose daughters all come before g
                int pl = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t c = __shfl_sync(0xffffffffu, dincl, pl + step - 1);
                    if (c <= g) pl += step;
                }
                pl = min(pl, 31);
                P32 d;
                d.xo = __shfl_sync(0xffffffffu, q.xo, pl);
                d.mu = __shfl_sync(0xffffffffu, q.mu, pl);
                d.inv_mu = __shfl_sync(0xffffffffu, q.inv_mu, pl);
                d.tau = __shfl_sync(0xffffffffu, q.tau, pl);
                d.cell = __shfl_sync(0xffffffffu, q.cell, pl);
                d.id = __shfl_sync(0xffffffffu, q.id, pl);
                const uint64_t plin = __shfl_sync(0xffffffffu, q.lin, pl);
                const uint32_t pe = __shfl_sync(0xffffffffu, q.e, pl);
                d.w = __shfl_sync(0xffffffffu, wd, pl);
                d.tw = __shfl_sync(0xffffffffu, twd, pl);
                const uint32_t pbase = __shfl_sync(0xffffffffu, dincl - nd, pl);  // warp prefix of the parent
                const unsigned po = __shfl_sync(0xffffffffu, o0, pl);            // the parent's first slot
                if (g < dtot) {
                    const uint32_t j = g - pbase;
                    d.lin = lineage_hash(plin, pe, j);
                    d.e = 0;
                    // the parent's scan word reserved at most cap outputs;
                    // its daughters past them have no slot of their own
                    if (j < (uint32_t)cap)
                        place(d, (unsigned long long)po + j);
                    else
                        push_record(a, d, d.w, 0u, 0u, 0u, warp_reserve(a.rout.count));
                }
            }
        }
        // ---- the pass's counts, summed over the warp ----
        {
            const unsigned wlo = ((eb & 0x1Fu) * 0x108421u) & 0x1041041u;
            const unsigned whi = (((eb >> 5) & 0xFu) * 0x8421u) & 0x41041u;
            const unsigned slo = __reduce_add_sync(0xffffffffu, wlo);
            const unsigned shi = __reduce_add_sync(0xffffffffu, whi);
            const unsigned sd = __reduce_add_sync(0xffffffffu, nadd);
            const unsigned smax = __reduce_max_sync(0xffffffffu, e_end);
            const unsigned f = ((lane < 5u ? slo : shi) >> (6u * (lane < 5u ? lane : lane - 5u))) & 63u;
            const unsigned cadd = lane < (unsigned)EB_COUNT ? f : (lane == (unsigned)LANE_DAUGHTERS ? sd : 0u);
            mycnt += cadd;
            if (lane == (unsigned)LANE_MAXEV) mycnt = max(mycnt, (unsigned long long)smax);
        }
        // the next pass's refill barrier orders the ring's writes before its
        // reads; the spill's writes wait one more pass (sp_rdy)
        const int nput = (int)(tot >> 11);
        head = ring_slot(head + m, cap);
        count = count - m + min(nput, room);
        const int nsp = min(max(0, nput - room), sp_room);
        sp_rdy = sp_n;
        sp_n += nsp;
        sp_total += nsp;
    }
    // the warp's counts into the block's
    if (lane < (unsigned)EB_COUNT) {
        if (mycnt) atomicAdd(&s_stats[kLaneStat[lane]], mycnt);
    } else if (lane == (unsigned)LANE_DAUGHTERS) {
        if (mycnt) atomicAdd(&s_stats[ST_DAUGHTERS], mycnt);
    } else if (lane == (unsigned)LANE_MAXEV) {
        if (mycnt) atomicMax(&s_stats[ST_MAX_EVENTS], mycnt);
    }
    if (t == 0 && sp_total && a.spilled) atomicAdd(a.spilled, (unsigned long long)sp_total);
    __syncthreads();
    flush_jf(tl32, I, a.tl);
    if (b_blk >= 0) flush_batch_row(tl32, I, a.batch, b_blk, false);
    flush_block_stats(s_stats, a.stats);
}

}  // namespace

void launch_track_fp32(const TrackArgs<float>& a, int grid, int block, size_t smem, cudaStream_t s) {
    track32_kernel<<<grid, block, smem, s>>>(a);
}

// the event kernel's launch shape for a mesh of I cells on the current
// device: the most blocks per SM (4, 3, 2, 1) whose share of the SM's shared
// memory, less the tallies, holds at least two passes of ring, and that ring
// in whole warps of particles; blocks 0 when even one block per SM does not
EvShape ev_shape(int I) {
    int dev = 0, per_sm = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const long long static_bytes = 1024 + 2048;  // the kernel's own variables and the per-block reserve, rounded up
    const long long tallies = (long long)sizeof(long long) * ROWS32 * I;
    for (int bps = EV_MAX_BLOCKS_PER_SM; bps >= 1; --bps) {
        const long long budget = std::min<long long>(optin, per_sm / bps - static_bytes);
        long long cap = (budget - tallies) / EV_REC_BYTES;
        cap = cap / 32 * 32;
        // the pass's scan word holds EV_THREADS x cap outputs in 21 bits
        if (cap >= 2 * EV_THREADS) return EvShape{bps, (int)std::min<long long>(cap, (1 << 21) / EV_THREADS - 32)};
    }
    return EvShape{0, 0};
}

size_t track_event_smem_fp32(int I, int cap) {
    return sizeof(long long) * (size_t)ROWS32 * (size_t)I + (size_t)EV_REC_BYTES * (size_t)cap;
}

void launch_track_fp32_event(const TrackArgs<float>& a, int nsm, const EvShape& shape, cudaStream_t s) {
    track32_event_kernel<<<nsm * shape.blocks_per_sm, EV_THREADS, track_event_smem_fp32(a.I, shape.cap), s>>>(
        a, shape.cap);
}

int track_event_smem_optin_fp32(int I, int cap) {
    return raise_smem_limit((const void*)track32_event_kernel, track_event_smem_fp32(I, cap));
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

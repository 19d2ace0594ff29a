// step.cu -- the O(N) stage after tracking:
//   comb      uniform combing of the census bank back to N (Sec. 5.1):
//             canonical order by (source id, lineage key) via per-id groups,
//             exact fixed-point cumulative weights, teeth (k + (2U+1)/2^33) W / N
//             decided in integers.
// Built with contraction off so that the comb positions are the single IEEE
// operations written.
#include <algorithm>

#include "hww_internal.cuh"
#include "step_kernels.cuh"
#include "track_common.cuh"

namespace hww {
namespace {

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
    if (threadIdx.x == 0) a.out[a.n] = GroupRec{carry.w, (uint32_t)carry.c, 0u};
}

// size classes of the comb's group lists (step_kernels.cuh): pairs, groups
// of 3-4, 5-8, 9-16, 17-32 members (warp segments), 33..MID_MAX (a warp per
// group), more (a block per group)
constexpr int MID_CLASS = 5;
constexpr int BIG_CLASS = 6;
constexpr int MID_MAX = 256;
static_assert(COMB_LISTS == BIG_CLASS + 1, "one list per size class");

__device__ __forceinline__ int size_class(uint32_t g) {
    return g == 2 ? 0 : g <= 4 ? 1 : g <= 8 ? 2 : g <= 16 ? 3 : g <= 32 ? 4 : g <= (uint32_t)MID_MAX ? MID_CLASS
                                                                                                   : BIG_CLASS;
}

// The scan's last pass: each tile's records (staged in shared memory, so
// that they are written coalesced), and the records of its groups of two or
// more members appended to their size class's list (the group passes read
// them there, without a gather by source id).  A thread's per-class counts
// are 16-bit fields of two words (classes 0-3, 4-6; a tile has at most 2048
// groups), scanned over the block, so each class takes one global
// reservation per tile.
__global__ void __launch_bounds__(SCAN_BLOCK) scan_apply_kernel(ScanArgs a) {
    __shared__ GroupRec s_out[SCAN_TILE];
    __shared__ unsigned long long s_wa[SCAN_BLOCK / 32], s_wb[SCAN_BLOCK / 32];
    __shared__ unsigned long long s_gbase[COMB_LISTS];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    Pair v[SCAN_ITEMS];
    Pair s{0ull, 0ull};
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = load_pair(a.cnt, a.w, base + (long long)t * SCAN_ITEMS + k, a.n);
        s = padd(s, v[k]);
    }
    block_exclusive_scan(s);
    Pair run{a.tile_c[blockIdx.x] + s.c, a.tile_w[blockIdx.x] + s.w};
    int kc[SCAN_ITEMS];
    unsigned long long A = 0, B = 0;  // this thread's groups per class, 16-bit fields
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        s_out[t * SCAN_ITEMS + k] = GroupRec{run.w, (uint32_t)run.c, (uint32_t)v[k].c};
        run = padd(run, v[k]);
        kc[k] = v[k].c >= 2 ? size_class((uint32_t)v[k].c) : -1;
        if (kc[k] >= 4)
            B += 1ull << (16 * (kc[k] - 4));
        else if (kc[k] >= 0)
            A += 1ull << (16 * kc[k]);
    }
    unsigned long long ia = A, ib = B;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long ya = __shfl_up_sync(0xffffffffu, ia, o);
        const unsigned long long yb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ya;
            ib += yb;
        }
    }
    if (lane == 31) {
        s_wa[wp] = ia;
        s_wb[wp] = ib;
    }
    __syncthreads();
    if (wp == 0) {
        constexpr int NW = SCAN_BLOCK / 32;
        const unsigned long long xa = lane < NW ? s_wa[lane] : 0ull, xb = lane < NW ? s_wb[lane] : 0ull;
        unsigned long long ja = xa, jb = xb;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long ya = __shfl_up_sync(0xffffffffu, ja, o);
            const unsigned long long yb = __shfl_up_sync(0xffffffffu, jb, o);
            if (lane >= o) {
                ja += ya;
                jb += yb;
            }
        }
        if (lane < NW) {
            s_wa[lane] = ja - xa;
            s_wb[lane] = jb - xb;
        }
        if (lane == NW - 1) {
            for (int c = 0; c < COMB_LISTS; ++c) {
                const unsigned long long n = ((c < 4 ? ja : jb) >> (16 * (c & 3))) & 0xFFFFull;
                s_gbase[c] = n ? atomicAdd(&a.glist_n[c], n) : 0ull;
            }
        }
    }
    __syncthreads();
    for (int i = t; i < SCAN_TILE; i += SCAN_BLOCK)
        if (base + i < a.n) a.out[base + i] = s_out[i];
    unsigned long long ea = s_wa[wp] + ia - A, eb = s_wb[wp] + ib - B;  // groups before this thread's
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int c = kc[k];
        if (c < 0) continue;
        unsigned long long& e = c < 4 ? ea : eb;
        const unsigned long long pos = s_gbase[c] + ((e >> (16 * (c & 3))) & 0xFFFFull);
        a.glist[a.glist_off[c] + pos] = s_out[t * SCAN_ITEMS + k];
        e += 1ull << (16 * (c & 3));
    }
}

// ---------------------------------------------------------------------------
// Comb
//
// The census particles of one source id form a group (its record from the
// scan: member count, start in the member list, fixed-point weight offset).
// Within a group the canonical order is (lineage key, census slot).  Census
// particle j owns the teeth in [C0_j, C0_j + w_j), C0_j = the group's weight
// offset plus the weights of the group members before it.  Most groups have
// one member: its C0 is set by the scatter pass, which lists only the members
// of larger groups (each with its key and weight, so that the group passes
// read their members contiguously); the scan's last pass lists the groups by
// size class, and their prefixes are found once per group: groups of up to
// 32 by a warp segment of 2 to 32 lanes (a rank count over shuffles), larger
// groups by a warp (up to 256 members)
// or a block with bucket lists: the lineage keys are uniform hashes, so
// bucketing members by the top bits of the key into at least as many buckets
// as members leaves about one member per bucket, the buckets are in key
// order, and a member's prefix is the scan of the bucket weights before its
// bucket plus the weights of the smaller keys in its own bucket's list.
// The copies are then written in census order, reading the census bank and
// the stored prefixes coalesced.
// ---------------------------------------------------------------------------
constexpr int MID_WARPS = 4;   // warps (groups in flight) per block of the warp-per-group kernel
constexpr int BIG_CAP = 4096;  // members a block keeps in shared memory
constexpr int BIG_T = 256;
template <class Real>
__global__ void comb_scatter_kernel(CombArgs<Real> a) {
    const long long m = (long long)*a.ncensus_ptr;
    const long long mm = m < a.cen_cap ? m : a.cen_cap;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < mm;
         j += (long long)gridDim.x * blockDim.x) {
        const uint32_t id = a.cid[j];
        const GroupRec g = a.gro[id];
        if (g.cnt == 1) {
            a.cpre[j] = g.offw;
            continue;
        }
        const unsigned long long slot = (unsigned long long)g.off + atomicAdd(&a.gcur[id], 1u);
        const LinW x = a.clw[j];
        MemberRec r;
        r.lin = x.lin;
        r.wfx = x.wfx;
        r.j = (uint32_t)j;
        r.pad[0] = r.pad[1] = r.pad[2] = 0u;
        a.member[slot] = r;
    }
}

__device__ __forceinline__ bool key_less(uint64_t la, uint32_t ja, uint64_t lb, uint32_t jb) {
    return la < lb || (la == lb && ja < jb);
}

// warp segments of S lanes, one group of at most S members per segment:
// lane i holds member i; its prefix is the weight of the segment's members
// with a smaller (lineage, slot) key, gathered by S shuffles.  One call
// handles the 32/S groups [e0, e0 + 32/S) of a class list (the whole warp,
// converged).
template <class Real, int S>
__device__ __forceinline__ void seg_groups(const CombArgs<Real>& a, const GroupRec* list, unsigned long long n,
                                           unsigned long long e0, unsigned long long& coll) {
    const int lane = threadIdx.x & 31, seg = lane / S, li = lane % S;
    const unsigned long long e = e0 + seg;
    uint32_t g = 0;
    unsigned long long base = 0, C = 0;
    if (e < n) {
        const GroupRec G = list[e];
        g = G.cnt;
        base = G.off;
        C = G.offw;
    }
    uint64_t lin = ~0ull;
    uint32_t jj = 0xFFFFFFFFu;
    unsigned long long w = 0;
    if ((uint32_t)li < g) {
        const MemberRec x = a.member[base + li];
        jj = x.j;
        lin = x.lin;
        w = x.wfx;
    }
    unsigned long long C0 = 0;
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const uint64_t lt = __shfl_sync(0xffffffffu, lin, t, S);
        const uint32_t jt = __shfl_sync(0xffffffffu, jj, t, S);
        const unsigned long long wt = __shfl_sync(0xffffffffu, w, t, S);
        if (key_less(lt, jt, lin, jj)) {
            C0 += wt;
            if (lt == lin && (uint32_t)t < g && (uint32_t)li < g) ++coll;
        }
    }
    if ((uint32_t)li < g) a.cpre[jj] = C + C0;
}

// the five warp-segment classes (pairs, 3-4, 5-8, 9-16, 17-32 members) in
// one launch: warp task t takes the next 32/S groups of its class's list
template <class Real>
__global__ void comb_seg_kernel(CombArgs<Real> a) {
    const unsigned long long n0 = a.glist_n[0], n1 = a.glist_n[1], n2 = a.glist_n[2], n3 = a.glist_n[3],
                             n4 = a.glist_n[4];
    const unsigned long long t1 = (n0 + 15) / 16, t2 = t1 + (n1 + 7) / 8, t3 = t2 + (n2 + 3) / 4,
                             t4 = t3 + (n3 + 1) / 2, t5 = t4 + n4;
    const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarp = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long coll = 0;
    for (unsigned long long t = warp; t < t5; t += nwarp) {  // warp-uniform branches
        if (t < t1)
            seg_groups<Real, 2>(a, a.glist + a.glist_off[0], n0, t * 16, coll);
        else if (t < t2)
            seg_groups<Real, 4>(a, a.glist + a.glist_off[1], n1, (t - t1) * 8, coll);
        else if (t < t3)
            seg_groups<Real, 8>(a, a.glist + a.glist_off[2], n2, (t - t2) * 4, coll);
        else if (t < t4)
            seg_groups<Real, 16>(a, a.glist + a.glist_off[3], n3, (t - t3) * 2, coll);
        else
            seg_groups<Real, 32>(a, a.glist + a.glist_off[4], n4, t - t4, coll);
    }
    if (coll) atomicAdd(&a.stats[ST_LINEAGE], coll);
}

// Bucket lists of one group held in shared memory: member i's key, weight
// and census slot, the first member of each bucket's list (-1: empty) and
// the next member of the same bucket.
struct BucketView {
    uint64_t* lin;
    unsigned long long* w;
    uint32_t* j;
    int* next;
    int* head;
};

// member i of a group into its bucket's list (bucket = the top bits of the
// lineage key, `sh` = 64 - log2(buckets))
__device__ __forceinline__ void bucket_insert(const BucketView& B, const MemberRec& m, int i, int sh) {
    B.lin[i] = m.lin;
    B.w[i] = m.wfx;
    B.j[i] = m.j;
    const int b = (int)(m.lin >> sh);
    B.next[i] = atomicExch(&B.head[b], i);
}

// total weight of buckets [b0, b1)
__device__ __forceinline__ unsigned long long bucket_sum(const BucketView& B, int b0, int b1) {
    unsigned long long t = 0;
    for (int b = b0; b < b1; ++b)
        for (int k = B.head[b]; k >= 0; k = B.next[k]) t += B.w[k];
    return t;
}

// the prefixes of the members of buckets [b0, b1), `run` the weight before
// bucket b0: the bucket's run plus the weights of the members of the same
// bucket with a smaller (lineage, slot) key; counts members with an equal
// lineage before each member (hash collisions) into coll
template <class Real>
__device__ __forceinline__ void bucket_prefixes(const CombArgs<Real>& a, const BucketView& B, int b0, int b1,
                                                unsigned long long run, unsigned long long& coll) {
    for (int b = b0; b < b1; ++b) {
        unsigned long long bsum = 0;
        for (int k = B.head[b]; k >= 0; k = B.next[k]) {
            const uint64_t lk = B.lin[k];
            const uint32_t jk = B.j[k];
            unsigned long long pre = run;
            for (int u = B.head[b]; u >= 0; u = B.next[u]) {
                if (key_less(B.lin[u], B.j[u], lk, jk)) {
                    pre += B.w[u];
                    if (B.lin[u] == lk) ++coll;
                }
            }
            a.cpre[jk] = pre;
            bsum += B.w[k];
        }
        run += bsum;
    }
}

// the number of buckets for g members: a power of two >= g, at least `lo`;
// returns log2 of it
__device__ __forceinline__ int bucket_bits(uint32_t g, int lo_bits) {
    int bits = lo_bits;
    while ((1u << bits) < g) ++bits;
    return bits;
}

// one warp per group of 33..MID_MAX members: bucket lists in the warp's
// share of shared memory (at least 32 buckets, a lane owns nb / 32
// consecutive ones), a shuffle scan of the lanes' bucket weights
template <class Real>
__global__ void __launch_bounds__(32 * MID_WARPS) comb_mid_kernel(CombArgs<Real> a) {
    __shared__ uint64_t s_lin[MID_WARPS][MID_MAX];
    __shared__ unsigned long long s_w[MID_WARPS][MID_MAX];
    __shared__ uint32_t s_j[MID_WARPS][MID_MAX];
    __shared__ int s_next[MID_WARPS][MID_MAX];
    __shared__ int s_head[MID_WARPS][MID_MAX];
    const unsigned long long n = a.glist_n[MID_CLASS];
    const GroupRec* list = a.glist + a.glist_off[MID_CLASS];
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const BucketView B{s_lin[wp], s_w[wp], s_j[wp], s_next[wp], s_head[wp]};
    unsigned long long coll = 0;
    for (unsigned long long e = (unsigned long long)blockIdx.x * MID_WARPS + wp; e < n;
         e += (unsigned long long)gridDim.x * MID_WARPS) {  // warp-uniform
        const GroupRec G = list[e];
        const int g = (int)G.cnt;
        const int bits = bucket_bits(G.cnt, 5);
        const int nb = 1 << bits, per = nb >> 5;
        for (int b = lane; b < nb; b += 32) B.head[b] = -1;
        __syncwarp();
        for (int i = lane; i < g; i += 32) bucket_insert(B, a.member[G.off + i], i, 64 - bits);
        __syncwarp();
        const int b0 = lane * per;
        const unsigned long long lsum = bucket_sum(B, b0, b0 + per);
        unsigned long long inc = lsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        bucket_prefixes(a, B, b0, b0 + per, G.offw + (inc - lsum), coll);
        __syncwarp();
    }
    if (coll) atomicAdd(&a.stats[ST_LINEAGE], coll);
}

// dynamic shared memory of the block-per-group kernel: keys, weights, slots,
// list links and bucket heads of BIG_CAP members
constexpr size_t BIG_SMEM = (size_t)BIG_CAP * (8 + 8 + 4 + 4 + 4);

// one block per group of more than MID_MAX members: bucket lists in shared
// memory (a thread owns nb / BIG_T consecutive buckets, at least one), a
// block scan of the threads' bucket weights; groups beyond BIG_CAP members
// take the rank count with the block's threads
template <class Real>
__global__ void __launch_bounds__(BIG_T) comb_big_kernel(CombArgs<Real> a) {
    extern __shared__ unsigned long long s_big[];
    __shared__ unsigned long long s_wsum[BIG_T / 32];
    const BucketView B{reinterpret_cast<uint64_t*>(s_big), s_big + BIG_CAP,
                       reinterpret_cast<uint32_t*>(s_big + 2 * BIG_CAP),
                       reinterpret_cast<int*>(s_big + 2 * BIG_CAP) + BIG_CAP,
                       reinterpret_cast<int*>(s_big + 2 * BIG_CAP) + 2 * BIG_CAP};
    const unsigned long long nbig = a.glist_n[BIG_CLASS];
    const GroupRec* list = a.glist + a.glist_off[BIG_CLASS];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    unsigned long long coll = 0;
    for (unsigned long long e = blockIdx.x; e < nbig; e += gridDim.x) {
        const GroupRec G = list[e];
        const uint32_t g = G.cnt;
        const unsigned long long base = G.off;
        const unsigned long long C = G.offw;
        if (g > (uint32_t)BIG_CAP) {
            for (uint32_t t = threadIdx.x; t < g; t += blockDim.x) {
                const MemberRec mt = a.member[base + t];
                unsigned long long C0 = C;
                for (uint32_t u = 0; u < g; ++u) {
                    const MemberRec mu = a.member[base + u];
                    if (key_less(mu.lin, mu.j, mt.lin, mt.j)) {
                        C0 += mu.wfx;
                        if (mu.lin == mt.lin) ++coll;
                    }
                }
                a.cpre[mt.j] = C0;
            }
            continue;
        }
        const int bits = bucket_bits(g, 8);  // at least BIG_T buckets
        const int nb = 1 << bits, per = nb / BIG_T;
        for (int b = threadIdx.x; b < nb; b += BIG_T) B.head[b] = -1;
        __syncthreads();
        for (int i = threadIdx.x; i < (int)g; i += BIG_T) bucket_insert(B, a.member[base + i], i, 64 - bits);
        __syncthreads();
        const int b0 = threadIdx.x * per;
        const unsigned long long tsum = bucket_sum(B, b0, b0 + per);
        unsigned long long inc = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_wsum[wp] = inc;
        __syncthreads();
        unsigned long long wbase = 0;
        for (int k = 0; k < wp; ++k) wbase += s_wsum[k];
        bucket_prefixes(a, B, b0, b0 + per, C + wbase + (inc - tsum), coll);
        __syncthreads();
    }
    if (coll) atomicAdd(&a.stats[ST_LINEAGE], coll);
}

// T_k >= C for tooth k at T_k = (k + (2U+1)/2^33) W / N, decided exactly:
// (k 2^33 + 2U + 1) W >= N C 2^33 in 128-bit integers; the right-hand side
// (rh, rl) depends on C only and is formed once per search
__device__ __forceinline__ bool tooth_at_or_after(long long k, unsigned long long W, unsigned U,
                                                  unsigned long long rh, unsigned long long rl) {
    const unsigned long long a = ((unsigned long long)k << 33) + 2ull * U + 1ull;
    const unsigned long long lh = __umul64hi(a, W), ll = a * W;
    return (lh > rh) || (lh == rh && ll >= rl);
}

// the scale of the tooth estimate: W reduced to its top 32 bits (shift sh)
// and R = floor(N 2^32 / W_r), computed once per thread
struct ToothScale {
    int sh;
    unsigned long long R;
};
__device__ __forceinline__ ToothScale tooth_scale(unsigned long long W, long long N) {
    ToothScale t;
    t.sh = max(0, 64 - __clzll((long long)W) - 32);
    const unsigned long long Wr = W >> t.sh;
    t.R = Wr ? (((unsigned long long)N << 32) / Wr) : 0ull;
    return t;
}

// least k in [0, N] with T_k >= C: the estimate (C_r R) / 2^32 from the top
// 32 bits of C and W is within two of the answer; exact steps finish it
__device__ __forceinline__ long long first_tooth(unsigned long long C, unsigned long long W, long long N,
                                                 unsigned U, const ToothScale& ts) {
    const unsigned long long Cr = C >> ts.sh;
    long long k = (long long)((Cr * ts.R) >> 32);
    if (k > N) k = N;
    const unsigned long long th = __umul64hi((unsigned long long)N, C), tl = (unsigned long long)N * C;
    const unsigned long long rh = (th << 33) | (tl >> 31), rl = tl << 33;  // N C 2^33
    for (int it = 0; it < 64 && k > 0 && tooth_at_or_after(k - 1, W, U, rh, rl); ++it) --k;
    for (int it = 0; it < 64 && k < N && !tooth_at_or_after(k, W, U, rh, rl); ++it) ++k;
    return k;
}

// census (time-crossing) tally contributions of one census particle, formed
// exactly as the precision's event loop forms them at a census event:
// FP64 round(x 2^S) of the FP64 products w, w mu, w (1/3 - mu^2); FP32 the
// fixed-point weight W = round(w 2^S) and, from the FP32 tally weight
// a = fl32(w 2^S), round(a mu) and round(a (1/3 - mu^2)) (the event loop's
// rule for its track-length contributions)
__device__ __forceinline__ void census_terms(double w, double mu, double tscale, int, long long& c0, long long& c1,
                                             long long& c2) {
    c0 = to_fixed(w, tscale);
    c1 = to_fixed(w * mu, tscale);
    c2 = to_fixed(w * (1.0 / 3.0 - mu * mu), tscale);
}
__device__ __forceinline__ void census_terms(double w, float mu, double, int S, long long& c0, long long& c1,
                                             long long& c2) {
    // the same roundings from the bits of w (no FP64 instruction)
    c0 = fixed_bits(w, S);
    const float a = tally_weight_bits(w, S);
    c1 = fx_mul24(a, mu);
    c2 = fx_mul24(a, 1.0f / 3.0f - mu * mu);
}

// census tallies alone (Eq. ct-mc) of the census bank so far: the closures
// of an in-step window update need them before the comb
template <class Real>
__global__ void census_tally_kernel(CombArgs<Real> a) {
    extern __shared__ long long s_cen[];  // 3 I
    const int I = a.I;
    for (int i = threadIdx.x; i < 3 * I; i += blockDim.x) s_cen[i] = 0;
    __syncthreads();
    const long long m = (long long)*a.ncensus_ptr;
    const long long mm = m < a.cen_cap ? m : a.cen_cap;
    const double tscale = a.sd->tscale;
    const int S = a.sd->S;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < mm;
         j += (long long)gridDim.x * blockDim.x) {
        const int k = a.ccell[j];
        long long c0, c1, c2;
        census_terms(a.cw[j], a.cmu[j], tscale, S, c0, c1, c2);
        sadd(&s_cen[k], c0);
        sadd(&s_cen[I + k], c1);
        sadd(&s_cen[2 * I + k], c2);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * I; i += blockDim.x)
        if (s_cen[i] != 0) add128(&a.cent[i], s_cen[i]);
}

// census derivative tallies of a derivative run: w S_q, w mu S_q and
// w (1/3 - mu^2) S_q of each census particle, the FP64 products of the
// numerics contract rounded at the tally scale.  Score q is the grid's
// y index; each block keeps its plane (3 I words) in shared memory and
// flushes it once (a global atomic per census particle and word had the
// atomic units serialize on the few hundred cells).
template <class Real>
__global__ void deriv_census_kernel(CombArgs<Real> a) {
    extern __shared__ long long s_d[];  // 3 I
    const int I = a.I;
    const int q = blockIdx.y;
    for (int i = threadIdx.x; i < 3 * I; i += blockDim.x) s_d[i] = 0;
    __syncthreads();
    const long long m = (long long)*a.ncensus_ptr;
    const long long mm = m < a.cen_cap ? m : a.cen_cap;
    const int S = a.sd->S;
    const double* sc = a.cS + (long long)q * a.cen_cap;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < mm;
         j += (long long)gridDim.x * blockDim.x) {
        const double w = a.cw[j];
        const double mu = (double)a.cmu[j];
        const int k = a.ccell[j];
        const double sq = sc[j];
        const double wmu = w * mu;
        const double wf = w * (1.0 / 3.0 - mu * mu);
        sadd(&s_d[k], fixed_bits(w * sq, S));
        sadd(&s_d[I + k], fixed_bits(wmu * sq, S));
        sadd(&s_d[2 * I + k], fixed_bits(wf * sq, S));
    }
    __syncthreads();
    Acc128* d = a.dcen + (long long)q * 3 * I;
    for (int i = threadIdx.x; i < 3 * I; i += blockDim.x)
        if (s_d[i] != 0) add128(&d[i], s_d[i]);
}

// The same tallies for all scores in one pass over the census bank, when
// their planes (3 P2 I words) fit one block's shared memory: one block of
// 1024 threads per SM, the census particle's w mu and w (1/3 - mu^2) formed
// once for all scores.
constexpr size_t DERIV_ALL_SMEM_MAX = 200 * 1024;

template <class Real>
__global__ void __launch_bounds__(1024) deriv_census_all_kernel(CombArgs<Real> a) {
    extern __shared__ long long s_d[];  // [P2][3][I]
    const int I = a.I, P2 = a.P2;
    for (int i = threadIdx.x; i < 3 * P2 * I; i += blockDim.x) s_d[i] = 0;
    __syncthreads();
    const long long m = (long long)*a.ncensus_ptr;
    const long long mm = m < a.cen_cap ? m : a.cen_cap;
    const int S = a.sd->S;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < mm;
         j += (long long)gridDim.x * blockDim.x) {
        const double w = a.cw[j];
        const double mu = (double)a.cmu[j];
        const int k = a.ccell[j];
        const double wmu = w * mu;
        const double wf = w * (1.0 / 3.0 - mu * mu);
        for (int q = 0; q < P2; ++q) {
            const double sq = a.cS[(long long)q * a.cen_cap + j];
            long long* d = s_d + (long long)q * 3 * I;
            sadd(&d[k], fixed_bits(w * sq, S));
            sadd(&d[I + k], fixed_bits(wmu * sq, S));
            sadd(&d[2 * I + k], fixed_bits(wf * sq, S));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * P2 * I; i += blockDim.x)
        if (s_d[i] != 0) add128(&a.dcen[i], s_d[i]);
}

// census order: each census particle's census tallies (Eq. ct-mc; block-
// private in shared memory), its teeth and its copies
template <class Real>
__global__ void comb_write_kernel(CombArgs<Real> a) {
    extern __shared__ long long s_cen[];  // 3 I
    const int I = a.I;
    for (int i = threadIdx.x; i < 3 * I; i += blockDim.x) s_cen[i] = 0;
    __syncthreads();
    const long long m = (long long)*a.ncensus_ptr;
    const long long mm = m < a.cen_cap ? m : a.cen_cap;
    const unsigned long long W = a.gro[a.N].offw;
    const unsigned U = a.sd->U_comb;
    const double tscale = a.sd->tscale;
    const int S = a.sd->S;
    const ToothScale ts = tooth_scale(W, a.N);
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < mm;
         j += (long long)gridDim.x * blockDim.x) {
        {
            // census order scatters the cells over a warp: one shared atomic
            // per lane and word (a warp aggregation would rarely merge lanes)
            const int k = a.ccell[j];
            long long c0, c1, c2;
            census_terms(a.cw[j], a.cmu[j], tscale, S, c0, c1, c2);
            sadd(&s_cen[k], c0);
            sadd(&s_cen[I + k], c1);
            sadd(&s_cen[2 * I + k], c2);
        }
        const unsigned long long C0 = a.cpre[j];
        const unsigned long long wj = a.clw[j].wfx;
        const long long k0 = first_tooth(C0, W, a.N, U, ts);
        const long long k1 = first_tooth(C0 + wj, W, a.N, U, ts);
        if (k1 <= k0) continue;
        const Real x = a.cx[j];
        const Real mu = a.cmu[j];
        const int32_t cell = a.ccell[j];
        BankRec<Real> rec{};
        rec.x = x;
        rec.mu = mu;
        rec.cell = cell;
        if constexpr (sizeof(Real) == sizeof(double)) rec.imu = a.cimu[j];
        for (long long k = k0; k < k1; ++k) a.bank[k] = rec;
        // derivative runs: every copy keeps the scores of its source
        for (int q = 0; q < a.P2; ++q) {
            const double sq = a.cS[(long long)q * a.cen_cap + j];
            for (long long k = k0; k < k1; ++k) a.bS[(long long)q * a.N + k] = sq;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * I; i += blockDim.x)
        if (s_cen[i] != 0) add128(&a.cent[i], s_cen[i]);
}

// the track-length flux tally as the sum of its variance-batch rows (the
// tracking adds each segment's flux to its batch row only): split
// accumulators add word by word, so the words equal those a direct
// accumulation would hold
__global__ void tl_phi_kernel(Acc128* tl, const Acc128* batch, int B, int I) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I; i += gridDim.x * blockDim.x) {
        unsigned long long lo = 0;
        long long hi = 0;
        for (int b = 0; b < B; ++b) {
            const Acc128 v = batch[(long long)b * I + i];
            lo += v.lo;
            hi += v.hi;
        }
        tl[i] = Acc128{lo, hi};
    }
}

__global__ void comb_finalize_kernel(StepDev* sd, const GroupRec* gro, const unsigned long long* ncensus_ptr,
                                     long long N, long long cen_cap, unsigned* err) {
    const unsigned long long W = gro[N].offw;
    const unsigned long long m = *ncensus_ptr;
    sd->ncensus = m;
    sd->W = W;
    // the step is complete: advance the device-side step state
    sd->step += 1;
    sd->cur ^= 1;
    sd->override_c = 0;
    sd->bank_loaded = 0;
    sd->has_prev = 1;
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

void launch_tl_phi(Acc128* tl, const Acc128* batch, int B, int I, cudaStream_t s) {
    tl_phi_kernel<<<(I + 255) / 256, 256, 0, s>>>(tl, batch, B, I);
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
    comb_seg_kernel<Real><<<grid, 256, 0, s>>>(a);
    comb_mid_kernel<Real><<<grid, 32 * MID_WARPS, 0, s>>>(a);
    comb_big_kernel<Real><<<grid, BIG_T, BIG_SMEM, s>>>(a);
    comb_write_kernel<Real><<<grid, 256, sizeof(long long) * 3 * (size_t)a.I, s>>>(a);
    if (a.P2 > 0) {  // about one block per SM (and score): few plane flushes
        const size_t all = sizeof(long long) * 3 * (size_t)a.P2 * (size_t)a.I;
        if (all <= DERIV_ALL_SMEM_MAX)
            deriv_census_all_kernel<Real><<<(unsigned)std::max(1, grid / 8), 1024, all, s>>>(a);
        else
            deriv_census_kernel<Real><<<dim3((unsigned)std::max(1, grid / 8), (unsigned)a.P2), 256,
                                        sizeof(long long) * 3 * (size_t)a.I, s>>>(a);
    }
}

template <class Real>
void launch_census_tallies(const CombArgs<Real>& a, int grid, cudaStream_t s) {
    census_tally_kernel<Real><<<grid, 256, sizeof(long long) * 3 * (size_t)a.I, s>>>(a);
}

template <class Real>
int census_tally_smem_optin(size_t smem) {
    return raise_smem_limit((const void*)census_tally_kernel<Real>, smem);
}

template <class Real>
void launch_comb_finalize(const CombArgs<Real>& a, cudaStream_t s) {
    comb_finalize_kernel<<<1, 1, 0, s>>>(a.sd, a.gro, a.ncensus_ptr, a.N, a.cen_cap, a.err);
}

template <class Real>
int comb_write_smem_optin(size_t smem) {
    int e = raise_smem_limit((const void*)comb_write_kernel<Real>, smem);
    if (!e) e = raise_smem_limit((const void*)deriv_census_kernel<Real>, smem);
    // the block-per-group pass's lists have a fixed size
    return e ? e : raise_smem_limit((const void*)comb_big_kernel<Real>, BIG_SMEM);
}

// the all-scores census derivative pass: its planes, when they fit
template <class Real>
int deriv_census_smem_optin(int P2, int I) {
    const size_t all = sizeof(long long) * 3 * (size_t)P2 * (size_t)I;
    return (all <= DERIV_ALL_SMEM_MAX) ? raise_smem_limit((const void*)deriv_census_all_kernel<Real>, all) : 0;
}
template int deriv_census_smem_optin<double>(int, int);
template int deriv_census_smem_optin<float>(int, int);

template void launch_comb<double>(const CombArgs<double>&, int, cudaStream_t);
template void launch_comb<float>(const CombArgs<float>&, int, cudaStream_t);
template void launch_comb_finalize<double>(const CombArgs<double>&, cudaStream_t);
template void launch_comb_finalize<float>(const CombArgs<float>&, cudaStream_t);
template int comb_write_smem_optin<double>(size_t);
template int comb_write_smem_optin<float>(size_t);
template void launch_census_tallies<double>(const CombArgs<double>&, int, cudaStream_t);
template void launch_census_tallies<float>(const CombArgs<float>&, int, cudaStream_t);
template int census_tally_smem_optin<double>(size_t);
template int census_tally_smem_optin<float>(size_t);

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

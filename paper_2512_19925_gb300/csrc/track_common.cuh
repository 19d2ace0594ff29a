// track_common.cuh -- pieces shared by the FP64 and FP32 tracking kernels:
// warp-aggregated slot reservation, per-block counters and the flush of the
// block-private fixed-point tallies.
#pragma once
#include <map>
#include <mutex>
#include <utility>

#include "hww_internal.cuh"

namespace hww {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Daughters of a split (or extra particles of a multiplying collision) that
// the single-problem kernels track on the splitting lane, after its current
// track, when the lane holds no other pending parent; the rest go to the
// record queue in chunks.  The persistent batched kernels, which end every
// tile with a block barrier, queue them all (a lane with pending daughters
// would hold its block at the barrier).
constexpr uint32_t LOCAL_DAUGHTERS = 32;

// One slot per calling lane; one atomic per group of converged lanes (a
// global counter, or a block's shared one).
template <class T>
__device__ __forceinline__ T warp_reserve(T* cnt) {
    const unsigned mask = __activemask();
    const int leader = __ffs(mask) - 1;
    const unsigned lane = lane_id();
    T base = 0;
    if ((int)lane == leader) base = atomicAdd(cnt, (T)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + (T)__popc(mask & ((1u << lane) - 1u));
}

// n consecutive slots per calling lane: lanes asking for the same n share
// one atomic (a split of up to 8 daughters asks for one record, so nearly
// all splitting lanes of a warp do); the counter is global and hot, so
// fewer atomics on it matter more than the match.
__device__ __forceinline__ unsigned long long warp_reserve_n(unsigned long long* cnt, unsigned n) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, n);
    const int leader = __ffs(peers) - 1;
    const unsigned lane = lane_id();
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(cnt, (unsigned long long)n * (unsigned long long)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + (unsigned long long)n * (unsigned long long)__popc(peers & ((1u << lane) - 1u));
}

// variance batch of a source id: contiguous id ranges, b = floor(id B / N),
// without a division: q = (x m) / 2^64 with m = floor((2^64 - 1) / N) (from
// the host) is floor(x / N) or one less (x = id B < 2^37), and one
// comparison decides
__device__ __forceinline__ int batch_of(uint32_t id, int B, long long N, unsigned long long m) {
    const unsigned long long x = (unsigned long long)id * (unsigned long long)B;
    unsigned long long q = __umul64hi(x, m);
    if ((q + 1) * (unsigned long long)N <= x) ++q;
    return (int)q;
}

// Add v to a 64-bit block-private accumulator in shared memory, exactly
// (modulo 2^64): shared memory has native 32-bit atomic adds but no 64-bit
// one (a 64-bit add is a compare-and-swap loop, retried under contention), so
// the low word is added with a returned old value, and the high word gets the
// high half of v plus the carry out of the low word.
__device__ __forceinline__ void sadd(long long* s, long long v) {
    unsigned* w = reinterpret_cast<unsigned*>(s);
    const unsigned lo = (unsigned)(unsigned long long)v;
    const unsigned old = atomicAdd(w, lo);
    const unsigned hi = (unsigned)((unsigned long long)v >> 32) + ((old + lo < old) ? 1u : 0u);
    if (hi) atomicAdd(w + 1, hi);
}

struct Counters {
    unsigned v[ST_COUNT];
    __device__ void zero() {
#pragma unroll
        for (int i = 0; i < ST_COUNT; ++i) v[i] = 0;
    }
};

// block reduction of the per-thread counters into the global 64-bit stats;
// segments and scatters are not counted in the event loops but follow from
// the event counts (every segment ends in a census, a crossing or a
// collision; a collision that emits a particle is a scatter)
__device__ __forceinline__ void flush_counters(Counters& c, unsigned long long* stats) {
    c.v[ST_SEGMENTS] = c.v[ST_CENSUS] + c.v[ST_CROSSINGS] + c.v[ST_COLLISIONS];
    c.v[ST_SCATTERS] = c.v[ST_COLLISIONS] - c.v[ST_ABSORBED];
    __shared__ unsigned long long red[ST_COUNT];
    if (threadIdx.x < ST_COUNT) red[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ST_COUNT; ++i) {
        unsigned x = c.v[i];
        if (i == ST_MAX_EVENTS) {
            for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
            if (lane_id() == 0 && x) atomicMax(&red[i], (unsigned long long)x);
        } else {
            unsigned long long y = x;
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if (lane_id() == 0 && y) atomicAdd(&red[i], y);
        }
    }
    __syncthreads();
    if (threadIdx.x < ST_COUNT && red[threadIdx.x]) {
        if (threadIdx.x == ST_MAX_EVENTS)
            atomicMax(&stats[ST_MAX_EVENTS], red[threadIdx.x]);
        else
            atomicAdd(&stats[threadIdx.x], red[threadIdx.x]);
    }
}

// block-private track-length tallies (3 I signed 64-bit) into the global
// 128-bit ones
__device__ __forceinline__ void flush_tallies(const long long* sm, int I, Acc128* tl) {
    for (int i = threadIdx.x; i < 3 * I; i += blockDim.x) {
        const long long v = sm[i];
        if (v != 0) add128(&tl[i], v);
    }
}


// The dynamic shared memory limit is a process-wide attribute of a kernel on
// a device: it is only ever raised, so that creating a problem with fewer
// cells does not lower the limit that an existing problem launches with.
inline int raise_smem_limit(const void* fn, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> lim;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> g(mu);
    size_t& l = lim[std::make_pair(fn, dev)];
    if (smem <= l) return 0;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) l = smem;
    return (int)e;
}

}  // namespace hww

// step.cu -- the O(N) stage after tracking:
//   comb      uniform combing of the census bank back to N (Sec. 5.1):
//             canonical order by (source id, lineage key) via per-id groups,
//             exact fixed-point cumulative weights, teeth (k + u) W / N.
// Built with contraction off so that the comb positions are the single IEEE
// operations written.
#include "hww_internal.cuh"
#include "step_kernels.cuh"

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

// T_k >= C for tooth k at T_k = (k + (2U+1)/2^33) W / N, decided exactly:
// (k 2^33 + 2U + 1) W >= N C 2^33 in 128-bit integers
__device__ __forceinline__ bool tooth_at_or_after(long long k, unsigned long long C, unsigned long long W,
                                                  long long N, unsigned U) {
    const unsigned long long a = ((unsigned long long)k << 33) + 2ull * U + 1ull;
    const unsigned long long lh = __umul64hi(a, W), ll = a * W;
    const unsigned long long th = __umul64hi((unsigned long long)N, C), tl = (unsigned long long)N * C;
    const unsigned long long rh = (th << 33) | (tl >> 31), rl = tl << 33;
    return (lh > rh) || (lh == rh && ll >= rl);
}

// least k in [0, N] with T_k >= C: an integer estimate from the top 32 bits
// of W and C, then exact steps (the estimate is within two of the answer)
__device__ __forceinline__ long long first_tooth(unsigned long long C, unsigned long long W, long long N,
                                                 unsigned U) {
    const int sh = max(0, 64 - __clzll((long long)W) - 32);
    const unsigned long long Wr = W >> sh, Cr = C >> sh;
    long long k = Wr ? (long long)((Cr * (unsigned long long)N) / Wr) : 0;
    if (k > N) k = N;
    for (int it = 0; it < 64 && k > 0 && tooth_at_or_after(k - 1, C, W, N, U); ++it) --k;
    for (int it = 0; it < 64 && k < N && !tooth_at_or_after(k, C, W, N, U); ++it) ++k;
    return k;
}

template <class Real>
__global__ void comb_write_kernel(CombArgs<Real> a) {
    const long long m = (long long)*a.ncensus_ptr;
    const long long mm = m < a.cen_cap ? m : a.cen_cap;
    const unsigned long long W = a.goff_w[a.N];
    const double cscale = a.sd->cscale;
    const unsigned U = a.sd->U_comb;
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
        const long long k0 = first_tooth(C0, W, a.N, U);
        const long long k1 = first_tooth(C0 + wj, W, a.N, U);
        const Real x = a.cx[j];
        const Real mu = a.cmu[j];
        const int32_t cell = a.ccell[j];
        for (long long k = k0; k < k1; ++k) {
            a.bx[k] = x;
            a.bmu[k] = mu;
            a.bcell[k] = cell;
        }
        // derivative runs: every copy keeps the scores of its source
        for (int q = 0; q < a.P2; ++q) {
            const double sq = a.cS[(long long)q * a.cen_cap + j];
            for (long long k = k0; k < k1; ++k) a.bS[(long long)q * a.N + k] = sq;
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

// hww_internal.cuh -- data layout shared by the library's translation units.
//
// Device memory of one problem (all SoA, one GPU):
//   start bank   x | mu | cell           N particles; weight w_bar each, tau = v dt,
//                                        id = slot, lineage 0, event 0 (implicit)
//   record queue x mu tau w cell id lin e jstart jcount   (two, ping-pong)
//                a record is either one live track (jcount == 0) or up to
//                SPLIT_CHUNK daughters j in [jstart, jstart+jcount) of a split
//   census bank  x mu w cell id lin     particles that reached t^n
//   comb groups  count / fixed-point weight per source id, their exclusive
//                scans, and the census indices grouped by id
//   tallies      128-bit fixed-point accumulators (Acc128)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hww.h"
#include "hww_device.cuh"

namespace hww {

constexpr int SPLIT_CHUNK = 8;
constexpr int TRACK_THREADS = 256;  // threads per tracking block
// A record's jstart carries FRESH_DIRECTION for the extra particles of a
// multiplying collision: each daughter then samples its own isotropic
// direction.  Their lineages hash the event with SECONDARY_EVENT set.
constexpr uint32_t FRESH_DIRECTION = 0x80000000u;
constexpr uint32_t SECONDARY_EVENT = 0x80000000u;
constexpr double MAX_C = 16.0;  // largest mean number of particles per collision
constexpr uint32_t MAX_DAUGHTERS = 1u << 24;
constexpr uint32_t MAX_EVENTS = 1u << 30;
constexpr double GRAZE_MU = 0.01;
constexpr int MAX_SCORES = 8;
constexpr int MAX_UPDATES = 16;  // in-step window updates per step  // likelihood-ratio scores per particle: (Sigma_t, c) of up to 4 regions

enum ErrBits : unsigned {
    ERR_CENSUS_OVERFLOW = 1u,
    ERR_QUEUE_OVERFLOW = 2u,
    ERR_DAUGHTERS = 4u,
    ERR_EVENTS = 8u,
    ERR_LOSM = 16u,
    ERR_COMB = 32u,
};

enum StatIdx {
    ST_SEGMENTS = 0, ST_COLLISIONS, ST_CROSSINGS, ST_REFLECTIONS, ST_LEAKED, ST_ABSORBED,
    ST_SCATTERS, ST_SPLIT_EVENTS, ST_DAUGHTERS, ST_RKILLS, ST_RSURVIVE, ST_CENSUS,
    ST_LINEAGE, ST_MAX_EVENTS, ST_NSTART, ST_COUNT
};

// per-step state that lives on the device, so that no stage of a step needs
// a parameter from the host (the stages can be captured once into graphs)
struct StepDev {
    double wbar;     // weight of each start-bank particle
    double tscale;   // 2^S, tally fixed-point scale
    double cscale;   // 2^Sc, comb weight fixed-point scale
    long long Wbar;  // wbar at the tally scale, round(wbar 2^S)
    int S, Sc;
    unsigned U_comb; // comb offset word: teeth at (k + (2U+1)/2^33) W / N
    unsigned k0, k1; // Philox key of the step: (seed_lo, seed_hi ^ n)
    int cur;         // closure set holding the initial conditions of the step
    int birth;       // the step starts from the pulse
    int bank_loaded; // set_bank was called since the last step
    int override_c;  // set_ww_centers was called since the last step
    int has_prev;    // a previous step exists (lagged windows)
    int ww_src;      // 0 none, 1 HLOSM, 2 previous track-length flux, 3 override
    int ww_on;
    unsigned long long step;       // completed steps
    unsigned long long nbank;      // start-bank size
    unsigned long long W;          // total census weight (fixed point)
    unsigned long long ncensus;    // census bank size of the step
};

// a step's statistics as the host reads them back: the counters, the step
// state and the error word
struct StatsExport {
    unsigned long long stats[ST_COUNT];
    StepDev sd;
    unsigned err;
};

// one start-bank particle (position, direction, cell) in one aligned record,
// so that a comb copy is one scattered store and a bank read one load:
// 16 bytes for the FP32 path (cell-local offset), 32 for FP64
template <class Real>
struct BankRec;
template <>
struct __align__(16) BankRec<float> {
    float x, mu;
    int32_t cell, pad;
};
template <>
struct __align__(32) BankRec<double> {
    double x, mu;
    double imu;  // 1/mu, carried so that a track start needs no FP64 divide
    int32_t cell, pad;
};

// a census particle's comb key and weight, read together by the comb
struct __align__(16) LinW {
    uint64_t lin;              // lineage key
    unsigned long long wfx;    // weight in fixed point at the comb scale 2^Sc
};

template <class Real>
struct RecQ {
    Real* x;
    Real* mu;
    Real* tau;
    double* w;
    int32_t* cell;
    uint32_t* id;
    uint64_t* lin;
    uint32_t* e;
    uint32_t* jstart;
    uint32_t* jcount;
    double* S;  // [P2][cap] scores (derivative runs only)
    unsigned long long* count;
    long long cap;
};

template <class Real>
struct CenQ {
    Real* x;
    Real* mu;
    double* w;
    int32_t* cell;
    uint32_t* id;
    LinW* lw;  // lineage key and weight at the comb scale 2^Sc, one 16-byte word
    Real* imu; // 1/mu of the FP64 path (its next start bank carries it); unused in FP32
    double* S;  // [P2][cap] scores (derivative runs only)
    unsigned long long* count;
    long long cap;
};

template <class Real>
struct TrackArgs {
    int I, B, emax;
    long long N;      // source particles per step (variance batches)
    unsigned long long batch_m;  // floor((2^64 - 1) / N): the variance-batch divisor
    int from_bank;
    long long bank_lo, bank_hi;  // wave 0 takes start-bank items [bank_lo, min(bank_hi, size))
    int bc_l, bc_r;
    int birth_cell_pos, birth_cell_neg;
    double tau0;      // v dt
    float tau0f;      // v dt rounded to FP32 (the FP32 path's distance to census at a step start)
    int comb_shift;   // S - Sc: the tally-scale weight shifted right by this is the comb-scale weight
    double src_x;
    const double* edges;
    const double* inv_sigt;
    const double* c;
    const float4* cellf;     // FP32 (width, 1/Sigma_t, c, 0) per cell, one load
    const double2* ww_hl;    // (ceiling, floor) per cell, one load
    const double* ww_c;
    const double* ww_hi;
    const double* ww_lo;
    const StepDev* sd;
    const BankRec<Real>* bank;  // start bank
    RecQ<Real> rin, rout;
    CenQ<Real> cen;
    uint32_t* gcnt;
    unsigned long long* gw;
    Acc128* tl;     // 3 I
    Acc128* cent;   // 3 I
    Acc128* batch;  // B I
    Acc128* bnd;    // 6
    unsigned long long* stats;
    unsigned* err;
    unsigned long long* spilled;  // running count of the particles the event loop spilled (null: not kept)
    // likelihood-ratio derivatives (P2 = 2R > 0): score j < R is that of
    // Sigma_t of region j, R + r that of c of region r
    int R, P2;
    const int32_t* region;  // I
    const double* inv_c;    // I, 1/c (scatter score)
    const double* bS;       // [P2][N] scores of the start bank
    Acc128* dtl;            // [P2][I]
    Acc128* dcen;           // [P2][3][I]
    Acc128* dbnd;           // [P2][6]
};

// work plan of one batched tracking launch: problem p owns tiles
// [tile_off[p], tile_off[p+1]) of `tile` items each; blocks pop tiles from
// the counter `head`
struct BatchPlan {
    const long long* tile_off;  // P+1
    int P;
    int tile;
    unsigned long long* head;
};

// the status of a CUDA error, recorded for hww_last_error_string (defined with
// the C ABI)
hww_status record_cuda_error(cudaError_t e);

// kernels implemented in the tracking translation units
void launch_track_fp64(const TrackArgs<double>& a, int grid, int block, size_t smem, cudaStream_t s);
void launch_track_fp32(const TrackArgs<float>& a, int grid, int block, size_t smem, cudaStream_t s);
// the event-based FP32 kernel of wave 0 (start-bank particles): blocks of
// 256 threads, up to four per SM, each with its tallies and a ring of `cap`
// particles in dynamic shared memory; ev_shape gives blocks per SM and the
// ring for a mesh of I cells on the current device (blocks 0: the mesh leaves
// no room)
struct EvShape {
    int blocks_per_sm;
    int cap;
};
EvShape ev_shape(int I);
size_t track_event_smem_fp32(int I, int cap);
int track_event_smem_optin_fp32(int I, int cap);
void launch_track_fp32_event(const TrackArgs<float>& a, int nsm, const EvShape& shape, cudaStream_t s);
void launch_track_batch_fp64(const TrackArgs<double>* args, const BatchPlan& plan, int grid, int block, size_t smem,
                             cudaStream_t s);
void launch_track_batch_fp32(const TrackArgs<float>* args, const BatchPlan& plan, int grid, int block, size_t smem,
                             cudaStream_t s);
// Rows of the tracking kernels' block-private 64-bit tallies in shared
// memory, each I long: track-length phi, J, F, then the batch row of the
// block's current id range; derivative runs append their [2R][I]
// track-length rows.
constexpr int TALLY_ROWS = 4;
// Rows of the single-problem FP32 kernel's block-private tallies: J, F and the
// batch row of the block's id range (the flux tally is the sum of the batch
// rows); each row is I low words then I high words (32-bit), so that the
// low-word atomics of a warp spread over all 32 banks.
constexpr int TALLY_ROWS_FP32 = 3;

int track_batch_smem_optin_fp32(size_t smem);
int track_batch_smem_optin_fp64(size_t smem);
int track_batch_blocks_per_sm_fp32(int block, size_t smem);
int track_batch_blocks_per_sm_fp64(int block, size_t smem);
inline int track_batch_smem_optin(int fp32, size_t smem) {
    return fp32 ? track_batch_smem_optin_fp32(smem) : track_batch_smem_optin_fp64(smem);
}
inline int track_batch_blocks_per_sm(int fp32, int block, size_t smem) {
    return fp32 ? track_batch_blocks_per_sm_fp32(block, smem) : track_batch_blocks_per_sm_fp64(block, smem);
}

}  // namespace hww

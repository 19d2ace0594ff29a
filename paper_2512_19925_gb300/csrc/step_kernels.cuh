// step_kernels.cuh -- argument blocks of the stages around the tracking kernel.
#pragma once
#include "hww_internal.cuh"

namespace hww {

// One source id's census group after the scan, read with one 16-byte load:
// exclusive prefix of the group weights (comb scale) and of the member
// counts over the ids before it, and its own member count.  Census slots are
// 32-bit (member lists hold them as such), so are the counts.
struct __align__(16) GroupRec {
    unsigned long long offw;
    uint32_t off;
    uint32_t cnt;
};

// One census particle in its group's member list: its lineage key and comb
// weight (copied from the census bank by the scatter pass, so that the
// passes over groups read their members contiguously instead of gathering
// them) and its census slot, in one 32-byte sector.
struct __align__(32) MemberRec {
    uint64_t lin;
    unsigned long long wfx;
    uint32_t j;
    uint32_t pad[3];
};

// lists of comb groups of 2+ members by size: 2, 3-4, 5-8, 9-16, 17-32 (warp
// segments), 33-256 (a warp per group), more (a block per group); a list
// whose groups have at least COMB_LIST_MIN[k] members holds at most
// census / COMB_LIST_MIN[k] of them
constexpr int COMB_LISTS = 7;
constexpr long long COMB_LIST_MIN[COMB_LISTS] = {2, 3, 5, 9, 17, 33, 257};

struct ScanArgs {
    const uint32_t* cnt;
    const unsigned long long* w;
    long long n;
    unsigned long long* tile_c;
    unsigned long long* tile_w;
    GroupRec* out;  // n+1 entries; entry n holds the totals
    // the group lists by size class (group records), filled by the scan's last pass
    GroupRec* glist;
    long long glist_off[COMB_LISTS];
    unsigned long long* glist_n;  // [COMB_LISTS] list lengths (cleared with the step's accumulators)
};

template <class Real>
struct CombArgs {
    StepDev* sd;
    long long N;
    const unsigned long long* ncensus_ptr;
    long long cen_cap;
    const Real* cx;
    const Real* cmu;
    const double* cw;
    const int32_t* ccell;
    const uint32_t* cid;
    const LinW* clw;  // [cen_cap] lineage keys and comb weights
    const Real* cimu; // [cen_cap] 1/mu (FP64 path)
    const uint32_t* gcnt;
    const GroupRec* gro;  // [N+1] group records (entry N: totals)
    uint32_t* gcur;
    MemberRec* member;
    BankRec<Real>* bank;  // next start bank
    unsigned long long* stats;
    unsigned* err;
    unsigned long long* cpre;        // [cen_cap] comb prefix C0 of every census particle
    const GroupRec* glist;           // records of the groups of 2+ members, by size class (COMB_LISTS lists)
    long long glist_off[COMB_LISTS]; // start of each class's list in glist
    unsigned long long* glist_n;     // [COMB_LISTS] list lengths (cleared with the step's accumulators)
    int I;             // cells (census tallies)
    Acc128* cent;      // census tallies 3 I
    int P2;            // scores per particle (0: none)
    const double* cS;  // [P2][cen_cap] census scores
    Acc128* dcen;      // [P2][3][I] census derivative tallies (derivative runs)
    double* bS;        // [P2][N] start-bank scores
};

void launch_group_scan(const ScanArgs& a, cudaStream_t s);
// track-length flux tally = sum of its variance-batch rows
void launch_tl_phi(Acc128* tl, const Acc128* batch, int B, int I, cudaStream_t s);
long long group_scan_tiles(long long n);
// the comb up to the copies (group scan excluded), with the census tallies;
// the finalize step (which advances the step state) runs separately, last
template <class Real>
void launch_comb(const CombArgs<Real>& a, int grid, cudaStream_t s);
template <class Real>
void launch_comb_finalize(const CombArgs<Real>& a, cudaStream_t s);
// raises the comb passes' dynamic shared memory limits (census tallies of
// `smem` bytes, the large groups' bucket lists)
template <class Real>
int comb_write_smem_optin(size_t smem);
template <class Real>
int deriv_census_smem_optin(int P2, int I);
// census tallies of the census bank so far, into the (cleared) tallies
template <class Real>
void launch_census_tallies(const CombArgs<Real>& a, int grid, cudaStream_t s);
template <class Real>
int census_tally_smem_optin(size_t smem);
void launch_philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                         long long n, uint32_t* out, cudaStream_t s);

int track_smem_optin_fp64(size_t smem, int deriv);
int track_smem_optin_fp32(size_t smem);
int track_blocks_per_sm_fp64(int block, size_t smem, int deriv);
int track_blocks_per_sm_fp32(int block, size_t smem);

}  // namespace hww

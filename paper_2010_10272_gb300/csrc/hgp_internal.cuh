// Internal device-side layout of libhgp.  Not part of the public ABI (include/hgp.h).
//
// HBM layout of one handle (n vertices, m nets, P pins, k blocks):
//   net_off[m+1], pins[P]        net -> pins CSR, int32 (Sec. 2 / Sec. 3.2 adjacency arrays)
//   vtx_off[n+1], inc[P]         vertex -> incident nets CSR I(v), int32 (bit 31: wide net)
//   vw[n]                        vertex weights c(v) (absent for unit weights)
//   part[n]                      Pi as uint8 (k <= 64)
//   phi                          Phi(e, i), row-major [m][k], entries of 1, 2 or 4 bytes packed
//                                into 32-bit words; nets larger than the entry can count keep
//                                int32 rows in phi_wide[n_wide][k] (Sec. 5.1 pin-count table)
//   rec[m]                       per-net hot record read by the gain step: Lambda(e) bitset,
//                                S1(e) = {i : Phi(e,i) = 1} bitset, omega(e), move stamp
//   bw[k], obj                   block weights c(V_i) and the (lambda-1) objective, int64
// plus per-sub-round scratch (candidate slots, approval histograms, tie prefix sums).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hgp.h"

namespace hgp {

constexpr int kRange = 256;              // consecutive vertices handled by one warp
constexpr int kWarps = 8;                // warps per tile CTA
constexpr int kRvSlotBytes = 32;         // one slot of the revert variant's hash table
constexpr int kWqPerRow = 128;           // work counters per stats row: 64 sub-rounds x 2 kernels
constexpr int kTile = kRange * kWarps;   // vertices per tile (one CTA)
constexpr int kThreads = 32 * kWarps;
constexpr int kBins = 4096;              // approval histogram bins (gains 1..4094 exact)
constexpr int kNever = -2;               // move-stamp round meaning "never moved"
constexpr uint32_t kWideFlag = 0x80000000u;
// inc[] entries carry the net id in bits 0..30 and, in bit 31, whether the net's Phi row lives
// in the wide table (so the apply step knows it without reading the net's record first)
constexpr int32_t kNetMask = 0x7fffffff;

// Per-net record for k <= 32, 16 bytes (two per 32-byte sector).
struct __align__(16) Rec16 {
    uint32_t s1;    // bit i set iff Phi(e,i) == 1
    int32_t w;      // omega(e) in bits 0..30, bit 31 = row lives in the wide table
    int32_t mv;     // move stamp: (last round with a pin move) * 2 + (moved in the round before)
    uint32_t lam;   // Lambda(e): bit i set iff Phi(e,i) > 0
};

// Per-net record for k <= 64, 32 bytes (one sector).  The first half is what the eligibility /
// b(u) pass needs, the second half what the connectivity pass needs.
struct __align__(16) Rec32 {
    uint64_t s1;
    int32_t w;
    int32_t mv;
    uint64_t lam;
    int32_t w2;     // copy of w
    int32_t pad;
};

// Approval state of one target block for the current sub-round.
struct Sel {
    int32_t mode;   // 0: approve every candidate; 1: threshold; 2: threshold inside the
                    //    overflow bin, being resolved digit by digit
    int32_t level;  // next refinement level for mode 2
    int64_t g;      // threshold gain (mode 1) / digit prefix (mode 2)
    int64_t rem;    // weight budget left for candidates with gain == g (mode 1) or with the
                    // current digit prefix (mode 2)
};

enum { SEL_ALL = 0, SEL_THRESH = 1, SEL_REFINE = 2 };
enum { ST_OBJ = 0, ST_CAND = 1, ST_APPR = 2, ST_ELIG = 3, ST_MAXW = 4, ST_MOVED = 5, ST_REV = 6, ST_N = 7 };
enum { ERR_INVALID = 1, ERR_UNSUPPORTED = 2, ERR_TABLE = 4 };

struct Dev {
    int32_t n, m, k, P;
    int32_t S;
    int32_t phi_w;          // 1, 2 or 4
    int32_t n_ranges, n_tiles;
    int64_t lmax;
    const int32_t *net_off;
    const int32_t *pins;
    const int32_t *vtx_off;
    const int32_t *inc;
    const int32_t *vw;      // nullptr: unit weights
    const int32_t *nw;      // net weights as given (nullptr: unit)
    uint8_t *part;
    uint32_t *phi;
    int32_t *phi_wide;
    const int32_t *widx;    // [m] row index in phi_wide (valid where the wide flag is set)
    const int32_t *net_perm;  // [m] internal id of input net e (nullptr: input order kept);
                              // every per-net array above is in internal order
    void *rec;              // Rec16[m] (k <= 32) or Rec32[m]
    int64_t *bw;
    int64_t *obj;
    // scratch
    uint8_t *sub_list;      // [n_ranges * kRange] local vertex offsets grouped by sub-round
    uint16_t *sub_start;    // [n_ranges * (S + 1)]
    uint64_t *cand;         // [n_ranges * kRange] (gain << 32 | local << 8 | target)
    int32_t *cand_cnt;      // [n_ranges]
    int64_t *tot;           // [k] candidate weight per target block
    unsigned long long *hist;  // [k * kBins]
    Sel *sel;               // [k]
    int64_t *tie;           // [k * n_tiles]
    int64_t *stats;         // [rounds * ST_N]
    int32_t *wq;            // [rounds * kWqPerRow] work counters of the single-instance persistent
                            // kernels (nullptr in batches: static assignment)
    int32_t *err;
    uint64_t seed;          // sub-round hash seed
    int32_t variant;        // bit 0: zero-gain balance moves; bit 1: revert negative moves
    int32_t pad0;
    int32_t *rs;            // round state on the device: rs[0] = next round r, rs[1] = 0 while
                            // every vertex is eligible (first round), 1 afterwards
    // revert variant only (nullptr otherwise)
    uint8_t *rv_src;        // [n_ranges * kRange] per candidate slot: block an approved move left,
                            // | 0x80 when it is to be undone; 0xFF when not approved
    void *rv_tab;           // hash table of (net, block) order statistics of the sub-round's moves
    int64_t rv_cap;         // its capacity in slots (a power of two >= 2 P)
    unsigned long long *rv_cnt;  // [2] incidences of the vertices moved in the current sub-round,
                                 // and those of them on nets with several movers
    int32_t *rv_net;        // [m] movers of each net in the current sub-round
};

__device__ __forceinline__ int lam_bits_ctz(uint32_t x) { return __ffs(x) - 1; }
__device__ __forceinline__ int lam_bits_ctz(uint64_t x) { return __ffsll((long long)x) - 1; }
__device__ __forceinline__ int lam_popc(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int lam_popc(uint64_t x) { return __popcll(x); }

// Adds delta (+1 or -1) to Phi(e, i) and returns the value before the update.  Narrow
// entries are updated with one 32-bit atomic on the word that holds them; this is exact
// because every intermediate value of an entry stays in [0, |e|] (decrements of Phi(e,i)
// in one sub-round come from distinct pins that were in block i at its start), so no
// borrow or carry crosses into a neighbouring entry.
__device__ __forceinline__ int32_t phi_add(const Dev &d, int32_t e, int32_t i, int32_t delta,
                                           bool wide, int32_t wrow)
{
    if (wide) return atomicAdd(&d.phi_wide[(int64_t)wrow * d.k + i], delta);
    const int64_t x = (int64_t)e * d.k + i;
    if (d.phi_w == 4) return atomicAdd(reinterpret_cast<int *>(d.phi) + x, delta);
    if (d.phi_w == 2) {
        const uint32_t sh = (uint32_t)(x & 1) * 16u;
        const uint32_t old = atomicAdd(&d.phi[x >> 1], (uint32_t)delta << sh);
        return (int32_t)((old >> sh) & 0xFFFFu);
    }
    const uint32_t sh = (uint32_t)(x & 3) * 8u;
    const uint32_t old = atomicAdd(&d.phi[x >> 2], (uint32_t)delta << sh);
    return (int32_t)((old >> sh) & 0xFFu);
}

__device__ __forceinline__ int32_t phi_get(const Dev &d, int32_t e, int32_t i, bool wide,
                                           int32_t wrow)
{
    if (wide) return d.phi_wide[(int64_t)wrow * d.k + i];
    const int64_t x = (int64_t)e * d.k + i;
    if (d.phi_w == 4) return reinterpret_cast<const int *>(d.phi)[x];
    if (d.phi_w == 2) return reinterpret_cast<const uint16_t *>(d.phi)[x];
    return reinterpret_cast<const uint8_t *>(d.phi)[x];
}

__device__ __forceinline__ void phi_set(const Dev &d, int32_t e, int32_t i, int32_t v, bool wide,
                                        int32_t wrow)
{
    if (wide) { d.phi_wide[(int64_t)wrow * d.k + i] = v; return; }
    const int64_t x = (int64_t)e * d.k + i;
    if (d.phi_w == 4) reinterpret_cast<int *>(d.phi)[x] = v;
    else if (d.phi_w == 2) reinterpret_cast<uint16_t *>(d.phi)[x] = (uint16_t)v;
    else reinterpret_cast<uint8_t *>(d.phi)[x] = (uint8_t)v;
}

// Eligibility test of Sec. 6 ("u and its neighbours"): did net e have a pin moved in
// round r-1?  The stamp keeps the last round with a move and whether the round before it
// had one too, so writes during round r do not hide round r-1.
__device__ __forceinline__ bool moved_in_prev_round(int32_t mv, int32_t r)
{
    const int32_t last = mv >> 1;
    return last == r - 1 || (last == r && (mv & 1));
}

// Stamp net e as moved in round r.  Every writer of round r computes the same value from
// the pre-round stamp, and a writer that already sees round r leaves it alone, so plain
// stores suffice.
__device__ __forceinline__ void stamp_moved(int32_t *mv_ptr, int32_t r)
{
    const int32_t v = *reinterpret_cast<volatile int32_t *>(mv_ptr);
    const int32_t last = v >> 1;
    if (last != r) *mv_ptr = (r << 1) | (last == r - 1 ? 1 : 0);
}

__device__ __forceinline__ uint64_t splitmix64_output(uint64_t z)
{
    // SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014)
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- host-side helpers
struct Handle;
cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int64_t count, int32_t *block_sums,
                            cudaStream_t st);
int64_t scan_scratch_elems(int64_t count);

}  // namespace hgp

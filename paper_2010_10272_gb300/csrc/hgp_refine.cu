// libhgp: synchronous label-propagation rounds (Sec. 6) on the device.
//
// One round r = round_prep, then for each sub-round s: gain -> approval -> apply, then
// round_end.  Kernels and what they compute:
//
//   k_round_prep   splitmix64(seed ^ (r << 32 | u)) mod S for every vertex, and per warp range
//                  of 256 vertices a list of its vertices grouped by sub-round (id order kept).
//   k_gain         for each active vertex u (a = Pi(u)), against the frozen state:
//                  W = omega(I(u)), b(u) = omega({e : Phi(e,a) = 1}) (Sec. 5), eligibility
//                  (a net of u moved in round r-1, Sec. 6), and the best target
//                  t = argmax_{i != a, feasible} g_i(u), g_i(u) = b(u) - p_i(u)
//                    = b(u) + omega({e in I(u) : i in Lambda(e)}) - W,
//                  ties to the smaller block; only blocks in the union of Lambda(e) over the
//                  nets with Phi(e,a) = 1 can have positive gain (g_i <= omega of those nets
//                  that contain i), so only those are evaluated.
//   k_hist/k_select   per target block t whose candidates do not all fit (w(t) + sum c > L_max):
//                  histogram of candidate weight by gain, scanned from the highest gain to
//                  find the threshold gain G_t and the budget left for candidates with
//                  gain == G_t (approval order (gain desc, id asc), inclusive prefix sums).
//   k_tie_sum/k_tie_scan   per tile weight of the gain == G_t candidates, exclusive prefix over
//                  tiles (tiles are in vertex-id order), so ties are approved in id order.
//   k_apply        applies every approved move: Pi(u) = t, block weights, Phi(e,a)--,
//                  Phi(e,t)++ with integer atomics, and Lambda(e), S1(e) and the objective
//                  from the atomics' old values (each step of a pin count across 0/1/2 toggles
//                  the matching bit, so the final bits are right whatever the order).
//   k_round_end    per-round objective and heaviest block; advances the device round state.
//
// Every kernel takes the instance state as `const Dev *devs` in device memory and a list of
// work items.  A single-handle launch passes items == nullptr: item i is the handle's own
// range / tile / block i.  A batch launch passes (instance, local index) pairs covering many
// handles at once, so one launch per phase refines a whole batch.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "hgp_host.cuh"

using namespace hgp;

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// instance and local index of work item i
__device__ __forceinline__ const Dev &item_of(const Dev *devs, const int2 *items, int32_t i, int32_t &local)
{
    if (items) {
        const int2 it = items[i];
        local = it.y;
        return devs[it.x];
    }
    local = i;
    return devs[0];
}

__device__ __forceinline__ int32_t item_count(const Dev *devs, const int2 *items, int32_t n_items, int kind)
{
    if (items) return n_items;
    return kind == 0 ? devs[0].n_ranges : (kind == 1 ? devs[0].n_tiles : devs[0].k);
}

// ------------------------------------------------------------------ round preparation
// warp per range item
// r_ovr >= 0: hash with that round number instead of the device round state (rebalancing)
__global__ void __launch_bounds__(kThreads) k_round_prep(const Dev *devs, const int2 *items, int32_t n_items,
                                                         int32_t r_ovr = -1)
{
    __shared__ uint8_t subs[kWarps][kRange];
    __shared__ int32_t cnt[kWarps][65];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t item = blockIdx.x * kWarps + wid;
    if (item >= item_count(devs, items, n_items, 0)) return;
    int32_t range;
    const Dev d = item_of(devs, items, item, range);
    const int32_t r = r_ovr >= 0 ? r_ovr : d.rs[0];
    const uint64_t seed = d.seed;
    const int32_t base = range * kRange;
    const int32_t nv = min(kRange, d.n - base);
    const int32_t S = d.S;
    const bool pow2 = (S & (S - 1)) == 0;
    for (int i = lane; i <= S; i += 32) cnt[wid][i] = 0;
    __syncwarp();
    for (int c = 0; c < kRange / 32; ++c) {
        const int idx = c * 32 + lane;
        if (idx < nv) {
            const uint32_t u = (uint32_t)(base + idx);
            const uint64_t z = splitmix64_output(seed ^ (((uint64_t)(uint32_t)r << 32) | u));
            const int sv = pow2 ? (int)(z & (uint64_t)(S - 1)) : (int)(z % (uint64_t)S);
            subs[wid][idx] = (uint8_t)sv;
            atomicAdd(&cnt[wid][sv], 1);
        }
    }
    __syncwarp();
    uint16_t *ss = d.sub_start + (int64_t)range * (S + 1);
    if (lane == 0) {
        int32_t run = 0;
        for (int i = 0; i < S; ++i) {
            const int32_t c = cnt[wid][i];
            cnt[wid][i] = run;
            ss[i] = (uint16_t)run;
            run += c;
        }
        ss[S] = (uint16_t)run;
    }
    __syncwarp();
    uint8_t *list = d.sub_list + (int64_t)range * kRange;
    for (int c = 0; c < kRange / 32; ++c) {
        const int idx = c * 32 + lane;
        const bool act = idx < nv;
        const unsigned mask = __ballot_sync(kFull, act);
        if (act) {
            const int sv = subs[wid][idx];
            const unsigned peers = __match_any_sync(mask, sv);
            const int pos = cnt[wid][sv] + __popc(peers & lanemask_lt());
            list[pos] = (uint8_t)idx;
            __syncwarp(mask);
            if (lane == __ffs(peers) - 1) cnt[wid][sv] += __popc(peers);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ gain + best target
template <typename Rec> struct RecIO;

template <> struct RecIO<Rec16> {
    typedef uint32_t Lam;
    // eligibility/b pass: s1, w, mv, and lam (same 16 bytes)
    __device__ static void load_a(const Rec16 *r, Lam &s1, int32_t &w, int32_t &mv, Lam &lam, bool &has_lam)
    {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(r));
        s1 = q.x; w = (int32_t)q.y; mv = (int32_t)q.z; lam = q.w; has_lam = true;
    }
    __device__ static Lam load_lam(const Rec16 *r) { return __ldg(&r->lam); }
    __device__ static void load_full(const Rec16 *r, Lam &s1, int32_t &w, int32_t &mv, Lam &lam)
    {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(r));
        s1 = q.x; w = (int32_t)q.y; mv = (int32_t)q.z; lam = q.w;
    }
    __device__ static void load_b(const Rec16 *r, Lam &lam, int32_t &w)
    {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(r));
        lam = q.w; w = (int32_t)q.y;
    }
};

template <> struct RecIO<Rec32> {
    typedef uint64_t Lam;
    __device__ static void load_a(const Rec32 *r, Lam &s1, int32_t &w, int32_t &mv, Lam &lam, bool &has_lam)
    {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(r));
        s1 = (uint64_t)q.x | ((uint64_t)q.y << 32); w = (int32_t)q.z; mv = (int32_t)q.w;
        lam = 0; has_lam = false;
    }
    __device__ static void load_full(const Rec32 *r, Lam &s1, int32_t &w, int32_t &mv, Lam &lam)
    {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(r));
        const uint2 l = __ldg(reinterpret_cast<const uint2 *>(&r->lam));
        s1 = (uint64_t)q.x | ((uint64_t)q.y << 32); w = (int32_t)q.z; mv = (int32_t)q.w;
        lam = (uint64_t)l.x | ((uint64_t)l.y << 32);
    }
    __device__ static Lam load_lam(const Rec32 *r)
    {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(&r->lam));
        return (uint64_t)q.x | ((uint64_t)q.y << 32);
    }
    __device__ static void load_b(const Rec32 *r, Lam &lam, int32_t &w)
    {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(&r->lam));
        lam = (uint64_t)q.x | ((uint64_t)q.y << 32); w = (int32_t)q.z;
    }
};

template <typename Lam> __device__ __forceinline__ uint32_t lo32(Lam x) { return (uint32_t)x; }
template <typename Lam> __device__ __forceinline__ uint32_t hi32(Lam x)
{
    return sizeof(Lam) == 8 ? (uint32_t)((uint64_t)x >> 32) : 0u;
}

constexpr int kCache = 256;   // incidences per chunk whose (Lambda, omega) stay in shared memory

template <typename Lam>
struct alignas(16) GainWarp {
    Lam lamc[kCache];            // Lambda(e) of the chunk's incidences, in flattened order
    int32_t wc[kCache];          // omega(e)
    unsigned long long T[32];
    unsigned long long A2[32];   // AND of Lambda(e) over nets with Phi(e,a) >= 2 (balance moves)
    int32_t W[32], b[32], jb[32], a[32], elig[32];
    int32_t off[33];
};
static_assert(sizeof(GainWarp<uint32_t>) % 16 == 0 && sizeof(GainWarp<uint64_t>) % 16 == 0, "GainWarp alignment");
static_assert(offsetof(GainWarp<uint32_t>, T) % 8 == 0 && offsetof(GainWarp<uint64_t>, T) % 8 == 0, "GainWarp alignment");

__device__ __forceinline__ int slot_of(const int32_t *off, int32_t i)
{
    int v = 0;
#pragma unroll
    for (int st = 16; st; st >>= 1)
        if (off[v + st] <= i) v += st;
    return v;
}

// Connectivity of one vertex to every block of T, held as NP bit planes (bit t of plane p is
// bit p of conn_t), accumulated with a ripple-carry adder on whole bitsets: adding omega(e) to
// every block of Lambda(e) & T costs O(NP) word operations, whatever the number of blocks.
// Returns the block of T with the largest conn_t (smallest id among equals) and its value.
// Requires conn_t <= W(u) < 2^NP.
template <typename Lam, typename Rec, int NP, bool UNIT>
__device__ __forceinline__ void bitsliced_best(const GainWarp<Lam> &g, const Rec *recs, const int32_t *inc,
                                               int32_t i_begin, int32_t i_end, int32_t jb, int32_t off,
                                               Lam T, int &t_out, int32_t &conn_out, int32_t eq_value,
                                               Lam &eq_out)
{
    Lam c[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) c[p] = 0;
    for (int32_t i = i_begin; i < i_end; ++i) {
        Lam lam;
        int32_t w;
        if (i < kCache) {
            lam = g.lamc[i];
            w = g.wc[i];
        } else {
            RecIO<Rec>::load_b(recs + (__ldg(&inc[jb + (i - off)]) & kNetMask), lam, w);
            w &= 0x7fffffff;
        }
        const Lam x = lam & T;
        if (UNIT) {
            Lam carry = x;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const Lam t = c[p] & carry;
                c[p] ^= carry;
                carry = t;
            }
        } else {
            Lam carry = 0;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const Lam ad = ((w >> p) & 1) ? x : (Lam)0;
                const Lam cp = c[p];
                c[p] = cp ^ ad ^ carry;
                carry = (cp & ad) | (carry & (cp ^ ad));
            }
        }
    }
    Lam C = T;
#pragma unroll
    for (int p = NP - 1; p >= 0; --p) {
        const Lam m = C & c[p];
        C = m ? m : C;
    }
    const int t = lam_bits_ctz(C);
    int32_t v = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) v |= (int32_t)((c[p] >> t) & 1) << p;
    t_out = t;
    conn_out = v;
    // blocks of T whose conn equals eq_value (eq_value < 0: none)
    Lam eq = eq_value >= 0 && (eq_value >> NP) == 0 ? T : (Lam)0;
#pragma unroll
    for (int p = 0; p < NP; ++p) eq &= ((eq_value >> p) & 1) ? c[p] : ~c[p];
    eq_out = eq;
}

template <typename Lam, typename Rec, bool UNIT>
__device__ __forceinline__ void best_by_planes(int np, const GainWarp<Lam> &g, const Rec *recs,
                                               const int32_t *inc, int32_t ib, int32_t ie, int32_t jb,
                                               int32_t off, Lam T, int &t, int32_t &conn, int32_t eqv, Lam &eq)
{
    if (np <= 4) bitsliced_best<Lam, Rec, 4, UNIT>(g, recs, inc, ib, ie, jb, off, T, t, conn, eqv, eq);
    else if (np <= 6) bitsliced_best<Lam, Rec, 6, UNIT>(g, recs, inc, ib, ie, jb, off, T, t, conn, eqv, eq);
    else if (np <= 8) bitsliced_best<Lam, Rec, 8, UNIT>(g, recs, inc, ib, ie, jb, off, T, t, conn, eqv, eq);
    else bitsliced_best<Lam, Rec, 11, UNIT>(g, recs, inc, ib, ie, jb, off, T, t, conn, eqv, eq);
}

constexpr int32_t kPlaneMaxW = 2047;   // W(u) up to this uses bit planes (NP <= 11)

// Per-warp state of the gain step that depends on the instance.
template <typename Lam>
struct GainInst {
    Lam feas1;           // blocks with room for a unit-weight vertex
    int32_t r;           // round number
    int32_t all_elig;    // first round: every vertex eligible
};

// Rebalancing pass settings (RB instances of the gain step).
struct RbArgs {
    int32_t r;       // round number of the sub-round hash for this pass
    int32_t phase;   // 1: gain >= 0 only; 2: any gain
    int32_t off;     // added to the gain to make the approval priority non-negative
};

// One range item of the gain step (see k_gain); returns the number of candidates written.
// RB: a rebalancing pass (Sec. 8): only vertices of overloaded blocks take part, their target
// is the block with room of highest gain (any sign), and the candidate records its source
// block (bits 16..23) and the priority gain + off; the per-block totals are by source block.
template <typename Rec, bool RB>
__device__ __forceinline__ int32_t gain_range(const Dev &d, int32_t range, int32_t s, GainWarp<typename RecIO<Rec>::Lam> &g,
                                              const long long *slack, unsigned long long *tot,
                                              const GainInst<typename RecIO<Rec>::Lam> &gi, int32_t &nel,
                                              const RbArgs &rb)
{
    typedef typename RecIO<Rec>::Lam Lam;
    constexpr bool kWide = sizeof(Lam) == 8;
    const int lane = threadIdx.x & 31;
    const Lam feas1 = gi.feas1;
    const int32_t r = gi.r, all_elig = gi.all_elig;
    const bool balance = !RB && (d.variant & 1) != 0;
        const Rec *recs = reinterpret_cast<const Rec *>(d.rec);
        const bool unit = d.nw == nullptr;
        const int32_t rbase = range * kRange;
        int32_t beg = 0, cnt = 0;
        if (s < d.S) {
            const uint16_t *ss = d.sub_start + (int64_t)range * (d.S + 1);
            beg = ss[s];
            cnt = (int32_t)ss[s + 1] - beg;
        }
        const uint8_t *list = d.sub_list + (int64_t)range * kRange + beg;
        uint64_t *out = d.cand + (int64_t)range * kRange;
        int32_t nout = 0;
        nel = 0;
        for (int32_t c0 = 0; c0 < cnt; c0 += 32) {
            const int32_t idx = c0 + lane;
            const bool valid = idx < cnt;
            int32_t ul = 0, cu = 1, deg = 0, jb = 0, a = 0;
            if (valid) {
                ul = list[idx];
                const int32_t u = rbase + ul;
                a = d.part[u];
                cu = d.vw ? d.vw[u] : 1;
                jb = d.vtx_off[u];
                deg = d.vtx_off[u + 1] - jb;
                if (RB && slack[a] >= 0) deg = 0;   // not in an overloaded block: no work
            }
            g.a[lane] = a;
            g.jb[lane] = jb;
            g.W[lane] = 0;
            g.b[lane] = 0;
            g.T[lane] = 0;
            g.A2[lane] = ~0ull;
            g.elig[lane] = RB ? (valid && slack[a] < 0) : all_elig;
            int32_t incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int32_t total = __shfl_sync(kFull, incl, 31);
            const int32_t my_off = incl - deg;
            g.off[lane] = my_off;
            if (lane == 31) g.off[32] = total;
            __syncwarp();
            // ---- pass A over the flattened incidences
            for (int32_t i0 = 0; i0 < total; i0 += 64) {
                const int32_t i1 = i0 + lane, i2 = i0 + 32 + lane;
                int v1 = 0, v2 = 0, e1 = 0, e2 = 0;
                if (i1 < total) {
                    v1 = slot_of(g.off, i1);
                    e1 = __ldg(&d.inc[g.jb[v1] + (i1 - g.off[v1])]) & kNetMask;
                }
                if (i2 < total) {
                    v2 = slot_of(g.off, i2);
                    e2 = __ldg(&d.inc[g.jb[v2] + (i2 - g.off[v2])]) & kNetMask;
                }
                Lam s11 = 0, lam1 = 0, s12 = 0, lam2 = 0;
                int32_t w1 = 0, mv1 = 0, w2 = 0, mv2 = 0;
                if (i1 < total) RecIO<Rec>::load_full(recs + e1, s11, w1, mv1, lam1);
                if (i2 < total) RecIO<Rec>::load_full(recs + e2, s12, w2, mv2, lam2);
                if (i1 < total) {
                    w1 &= 0x7fffffff;
                    if (i1 < kCache) { g.lamc[i1] = lam1; g.wc[i1] = w1; }
                    atomicAdd(&g.W[v1], w1);
                    if ((s11 >> g.a[v1]) & 1) {
                        atomicAdd(&g.b[v1], w1);
                        atomicOr(&g.T[v1], (unsigned long long)lam1);
                    } else if (balance) {
                        atomicAnd(&g.A2[v1], (unsigned long long)lam1);
                    }
                    if (!RB && moved_in_prev_round(mv1, r)) g.elig[v1] = 1;
                }
                if (i2 < total) {
                    w2 &= 0x7fffffff;
                    if (i2 < kCache) { g.lamc[i2] = lam2; g.wc[i2] = w2; }
                    atomicAdd(&g.W[v2], w2);
                    if ((s12 >> g.a[v2]) & 1) {
                        atomicAdd(&g.b[v2], w2);
                        atomicOr(&g.T[v2], (unsigned long long)lam2);
                    } else if (balance) {
                        atomicAnd(&g.A2[v2], (unsigned long long)lam2);
                    }
                    if (!RB && moved_in_prev_round(mv2, r)) g.elig[v2] = 1;
                }
            }
            __syncwarp();
            // ---- per vertex: eligibility, candidate blocks, best block
            const int32_t W = g.W[lane], b = g.b[lane];
            const bool elig = valid && g.elig[lane] != 0;
            const Lam kall = d.k >= (int)(8 * sizeof(Lam)) ? ~(Lam)0 : (((Lam)1 << d.k) - 1);
            Lam T = elig ? (RB ? kall : (Lam)g.T[lane]) : (Lam)0;
            T &= ~((Lam)1 << a);
            const Lam T_all = T;   // before the room filter (balance moves need it)
            if (d.vw) {
                for (Lam x = T; x; x &= x - 1) {
                    const int t = lam_bits_ctz(x);
                    if (slack[t] < cu) T &= ~((Lam)1 << t);
                }
            } else {
                T &= feas1;
            }
            const bool plane_path = T != 0 && W <= kPlaneMaxW;
            const bool coop_path = T != 0 && W > kPlaneMaxW;
            int32_t t_best = -1, g_best = 0;
            const int32_t bw_ = b - W;
            const unsigned wmax = __reduce_max_sync(kFull, plane_path ? (unsigned)W : 0u);
            Lam zero_in = 0;   // blocks of T with gain exactly 0 (balance moves)
            if (plane_path) {
                const int np = 32 - __clz((int)wmax);   // 2^np > wmax >= conn_t
                int t;
                int32_t conn;
                const int32_t eqv = balance ? W - b : -1;
                if (unit) best_by_planes<Lam, Rec, true>(np, g, recs, d.inc, my_off, my_off + deg, jb, my_off, T, t, conn, eqv, zero_in);
                else best_by_planes<Lam, Rec, false>(np, g, recs, d.inc, my_off, my_off + deg, jb, my_off, T, t, conn, eqv, zero_in);
                const int32_t gg = bw_ + conn;
                if (RB ? (rb.phase == 2 || gg >= 0) : gg > 0) {
                    t_best = t;
                    g_best = gg;
                }
            }
            // ---- warp-cooperative pass for vertices with large incident net weight
            unsigned hm = __ballot_sync(kFull, coop_path);
            while (hm) {
                const int src = __ffs(hm) - 1;
                hm &= hm - 1;
                const int32_t hjb = __shfl_sync(kFull, jb, src), hje = hjb + __shfl_sync(kFull, deg, src);
                const int32_t hbw = __shfl_sync(kFull, bw_, src);
                const uint32_t Tlo = __shfl_sync(kFull, lo32(T), src);
                const uint32_t Thi = kWide ? __shfl_sync(kFull, hi32(T), src) : 0u;
                int32_t acc0 = 0, acc1 = 0;
                for (int32_t j0 = hjb; j0 < hje; j0 += 32) {
                    const int32_t j = j0 + lane;
                    Lam lam = 0;
                    int32_t w = 0;
                    if (j < hje) {
                        RecIO<Rec>::load_b(recs + (__ldg(&d.inc[j]) & kNetMask), lam, w);
                        w &= 0x7fffffff;
                    }
                    const int nn = min(32, hje - j0);
                    const uint32_t llo = lo32(lam), lhi = hi32(lam);
                    for (int q = 0; q < nn; ++q) {
                        const uint32_t bl = __shfl_sync(kFull, llo, q);
                        const int32_t wi = __shfl_sync(kFull, w, q);
                        acc0 += ((bl >> lane) & 1) ? wi : 0;
                        if (kWide) {
                            const uint32_t bh = __shfl_sync(kFull, lhi, q);
                            acc1 += ((bh >> lane) & 1) ? wi : 0;
                        }
                    }
                }
                // key = gain << 8 | (255 - block): the larger key is the higher gain, then the
                // smaller block (RB: the gain's sign bit flipped, so negative gains order too)
                unsigned long long key = 0;
                if ((Tlo >> lane) & 1) {
                    const int32_t gg = hbw + acc0;
                    if (RB ? (rb.phase == 2 || gg >= 0) : gg > 0)
                        key = ((unsigned long long)((uint32_t)gg ^ (RB ? 0x80000000u : 0u)) << 8) | (unsigned long long)(255 - lane);
                }
                if (kWide && ((Thi >> lane) & 1)) {
                    const int32_t gg = hbw + acc1;
                    if (RB ? (rb.phase == 2 || gg >= 0) : gg > 0) {
                        const unsigned long long k2 = ((unsigned long long)((uint32_t)gg ^ (RB ? 0x80000000u : 0u)) << 8) | (unsigned long long)(255 - (lane + 32));
                        key = k2 > key ? k2 : key;
                    }
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(kFull, key, o);
                    key = y > key ? y : key;
                }
                if (lane == src && key) {
                    t_best = 255 - (int)(key & 0xFF);
                    g_best = (int32_t)((uint32_t)(key >> 8) ^ (RB ? 0x80000000u : 0u));
                }
                if (balance) {
                    // zero-gain blocks of T among the ones this lane owns
                    const unsigned zlo = __ballot_sync(kFull, ((Tlo >> lane) & 1) && hbw + acc0 == 0);
                    const unsigned zhi = __ballot_sync(kFull, kWide && ((Thi >> lane) & 1) && hbw + acc1 == 0);
                    if (lane == src) zero_in = kWide ? (Lam)((uint64_t)zlo | ((uint64_t)zhi << 32)) : (Lam)zlo;
                }
            }
            if (balance && valid && elig && t_best < 0) {
                // zero-gain moves that improve the balance (Sec. 6): blocks of T with gain 0, and
                // blocks outside T that lie in every net where u is not alone (their gain is
                // b - p_t = 0 exactly then); room and w(t) + c(u) < w(a); lightest block first
                const Lam kmask = d.k >= (int)(8 * sizeof(Lam)) ? ~(Lam)0 : (((Lam)1 << d.k) - 1);
                Lam z = (zero_in | ((Lam)g.A2[lane] & ~T_all & ~((Lam)1 << a))) & kmask;
                const long long wa = d.lmax - slack[a];
                long long best_w = 0;
                for (Lam x = z; x; x &= x - 1) {
                    const int t = lam_bits_ctz(x);
                    const long long wt = d.lmax - slack[t];
                    if (slack[t] < cu || wt + cu >= wa) continue;
                    if (t_best < 0 || wt < best_w) {
                        t_best = t;
                        best_w = wt;
                    }
                }
                g_best = 0;
            }
            nel += __popc(__ballot_sync(kFull, elig));
            const unsigned cm = __ballot_sync(kFull, t_best >= 0);
            if (t_best >= 0) {
                const int pos = nout + __popc(cm & lanemask_lt());
                if (RB) {
                    out[pos] = ((uint64_t)(uint32_t)(g_best + rb.off) << 32) | ((uint32_t)a << 16) |
                               ((uint32_t)ul << 8) | (uint32_t)t_best;
                    atomicAdd(&tot[a], (unsigned long long)cu);
                } else {
                    out[pos] = ((uint64_t)(uint32_t)g_best << 32) | ((uint32_t)ul << 8) | (uint32_t)t_best;
                    atomicAdd(&tot[t_best], (unsigned long long)cu);
                }
            }
            if (!RB && t_best >= 0) {
                // level-0 histogram of the approval step: candidate weight by target block and
                // gain bin (no return value: a reduction in L2)
                const int bin = g_best < kBins - 1 ? g_best : kBins - 1;
                atomicAdd(&d.hist[(int64_t)t_best * kBins + bin], (unsigned long long)cu);
            }
            nout += __popc(cm);
            __syncwarp();
        }
        return nout;
}

template <typename Rec>
__device__ __forceinline__ void gain_refresh(const Dev &d, long long *slack, GainInst<typename RecIO<Rec>::Lam> &gi)
{
    typedef typename RecIO<Rec>::Lam Lam;
    const int lane = threadIdx.x & 31;
    for (int t = lane; t < 64; t += 32) slack[t] = t < d.k ? d.lmax - d.bw[t] : -1;
    __syncwarp();
    const unsigned lo = __ballot_sync(kFull, slack[lane] >= 1);
    const unsigned hi = __ballot_sync(kFull, slack[lane + 32] >= 1);
    if (sizeof(Lam) == 8) gi.feas1 = (Lam)((uint64_t)lo | ((uint64_t)hi << 32));
    else gi.feas1 = (Lam)lo;
    gi.r = d.rs[0];
    gi.all_elig = d.rs[1] == 0;
}

// Dynamic work distribution of the single-instance persistent kernels: a warp takes its next
// range item from a per-launch device counter (zeroed before the launch), so the last items go
// to whichever warps are free instead of a fixed stride.
__device__ __forceinline__ int32_t take_item(int32_t *counter)
{
    int32_t it = 0;
    if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1);
    return __shfl_sync(kFull, it, 0);
}

// the counter increment is issued by lane 0 before the current item is processed; its result
// is only read (broadcast) when the item is done, so the round trip overlaps the work
__device__ __forceinline__ int32_t take_item_early(int32_t *counter)
{
    int32_t it = 0;
    if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1);
    return it;
}

// copies devs[inst] into a warp's shared slot
__device__ __forceinline__ void load_dev(Dev &dst, const Dev *src)
{
    const int lane = threadIdx.x & 31;
    const uint32_t *a = reinterpret_cast<const uint32_t *>(src);
    uint32_t *b = reinterpret_cast<uint32_t *>(&dst);
    for (int i = lane; i < (int)(sizeof(Dev) / 4); i += 32) b[i] = a[i];
    __syncwarp();
}

// Persistent: each warp walks range items with a grid stride and takes the vertices of
// sub-round s of a range 32 at a time (one slot per lane).
//   pass A  flattened over the chunk's incidences (every record gather issued at once): W,
//           b(u) (Sec. 5), eligibility (Sec. 6) and T = union of Lambda(e) over the nets with
//           Phi(e,a) = 1, minus a and the blocks without room for c(u); (Lambda, omega) of each
//           incidence is kept in shared memory.  Only blocks in T can have a positive gain,
//           since g_t <= omega({e : Phi(e,a) = 1, t in Lambda(e)}).
//   pass B  per vertex, conn_t = omega({e in I(u) : t in Lambda(e)}) for all t in T at once in
//           bit planes, and the arg-max of g_t = b(u) - W + conn_t.
// A vertex whose incident net weights exceed kPlaneMaxW uses a warp-cooperative pass instead.
// B = false: one instance, d0 (parameter space), items are its ranges; B = true: a batch,
// items name (instance, range) and each warp copies its item's instance into shared memory.
template <typename Rec, bool B, bool RB = false>
__global__ void __launch_bounds__(kThreads, 4) k_gain(const Dev d0, const Dev *devs, const int2 *items,
                                                      int32_t n_items, int32_t s, int32_t rr, RbArgs rb = RbArgs{0, 0, 0})
{
    typedef typename RecIO<Rec>::Lam Lam;
    __shared__ GainWarp<Lam> ws[kWarps];
    __shared__ long long slack_w[kWarps][64];
    __shared__ unsigned long long tot_w[kWarps][64];
    __shared__ Dev dsm[B ? kWarps : 1];
    __shared__ unsigned long long cnt_s[2];
    __shared__ int warps_done;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    tot_w[wid][lane] = 0;
    tot_w[wid][lane + 32] = 0;
    if (tid == 0) { cnt_s[0] = 0; cnt_s[1] = 0; warps_done = 0; }
    __syncthreads();   // before any warp can add into another warp's slots (at its end)
    GainInst<Lam> gi;
    int32_t nelig = 0, ncand = 0;
    int inst_prev = -1;
    const int32_t n_it = B ? n_items : d0.n_ranges;
    int32_t *wq = d0.wq + ((int64_t)rr * 64 + s) * 2;
    int32_t next_raw = 0;
    for (int32_t item = take_item(wq); item < n_it; item = __shfl_sync(kFull, next_raw, 0)) {
        next_raw = take_item_early(wq);
        if (B) {
            const int2 it = items[item];
            if (it.x != inst_prev) {
                load_dev(dsm[wid], devs + it.x);
                gain_refresh<Rec>(dsm[wid], slack_w[wid], gi);
                inst_prev = it.x;
            }
            const Dev &d = dsm[wid];
            int32_t nel = 0;
            const int32_t nout = gain_range<Rec, false>(d, it.y, s, ws[wid], slack_w[wid], tot_w[wid], gi, nel, rb);
            if (lane == 0) d.cand_cnt[it.y] = nout;
            // flush this item's totals into its own instance
            unsigned long long *row = reinterpret_cast<unsigned long long *>(d.stats + (int64_t)rr * ST_N);
            for (int t = lane; t < 64; t += 32) {
                const unsigned long long v = tot_w[wid][t];
                if (v) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&d.tot[t]), v);
                    tot_w[wid][t] = 0;
                }
            }
            if (lane == 0) {
                if (nel) atomicAdd(row + ST_ELIG, (unsigned long long)nel);
                if (nout) atomicAdd(row + ST_CAND, (unsigned long long)nout);
            }
            __syncwarp();
        } else {
            if (inst_prev < 0) {
                gain_refresh<Rec>(d0, slack_w[wid], gi);
                if (RB) gi.r = rb.r;
                inst_prev = 0;
            }
            int32_t nel = 0;
            const int32_t nout = gain_range<Rec, RB>(d0, item, s, ws[wid], slack_w[wid], tot_w[wid], gi, nel, rb);
            if (lane == 0) d0.cand_cnt[item] = nout;
            nelig += nel;
            ncand += nout;
        }
    }
    if (!B) {
        // one instance: the warps add their partial sums into warp 0's slots as they finish and
        // the last warp of the CTA flushes them with one atomic per block (no barrier, so warps
        // that finish early do not wait for the slowest one)
        if (wid != 0) {
            for (int t = lane; t < 64; t += 32)
                if (tot_w[wid][t]) atomicAdd(&tot_w[0][t], tot_w[wid][t]);
        }
        if (lane == 0) {
            if (nelig) atomicAdd(&cnt_s[0], (unsigned long long)nelig);
            if (ncand) atomicAdd(&cnt_s[1], (unsigned long long)ncand);
        }
        __threadfence_block();
        __syncwarp();
        int last = 0;
        if (lane == 0) last = atomicAdd(&warps_done, 1) == kWarps - 1;
        last = __shfl_sync(kFull, last, 0);
        if (last) {
            __threadfence_block();
            for (int t = lane; t < 64 && t < d0.k; t += 32) {
                const unsigned long long v = atomicAdd(&tot_w[0][t], 0ull);
                if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&d0.tot[t]), v);
            }
            if (lane == 0) {
                unsigned long long *row = reinterpret_cast<unsigned long long *>(d0.stats + (int64_t)rr * ST_N);
                const unsigned long long c0 = atomicAdd(&cnt_s[0], 0ull), c1 = atomicAdd(&cnt_s[1], 0ull);
                if (c0) atomicAdd(row + ST_ELIG, c0);
                if (c1) atomicAdd(row + ST_CAND, c1);
            }
        }
    }
}

// ------------------------------------------------------------------ approval
__device__ __forceinline__ void decode(uint64_t c, int &t, int32_t &g, int &ul)
{
    t = (int)(c & 0xFF);
    ul = (int)((c >> 8) & 0xFF);
    g = (int32_t)(c >> 32);
}

// Which block an approval stage groups a candidate by, and which candidates take part:
//   KEY_T   LP: by target block, all candidates, inclusive prefix <= L_max - w(t);
//   KEY_A   rebalancing, source side: by source block (bits 16..23), all candidates, a
//           candidate passes while the weight before it is <= w(a) - L_max - 1 (exclusive);
//   KEY_TS  rebalancing, target side: by target block, only candidates marked by KEY_A
//           (bit 24), inclusive prefix <= L_max - w(t).
enum { KEY_T = 0, KEY_A = 1, KEY_TS = 2 };
constexpr uint64_t kSelBit = 1ull << 24;

template <int KEY>
__device__ __forceinline__ bool decode_key(uint64_t c, int &key, int &t, int32_t &g, int &ul)
{
    decode(c, t, g, ul);
    key = KEY == KEY_A ? (int)((c >> 16) & 0xFF) : t;
    return KEY != KEY_TS || (c & kSelBit) != 0;
}

// capacity of a key block for the stage (the weight its passing candidates may add up to)
template <int KEY>
__device__ __forceinline__ long long stage_cap(const Dev &d, int key)
{
    return KEY == KEY_A ? (long long)d.bw[key] - d.lmax - 1 : (long long)d.lmax - d.bw[key];
}

// digit of the overflow-bin refinement at `level` (1..3) for value v = g - (kBins - 1),
// and whether v matches the prefix resolved so far
__device__ __forceinline__ int refine_digit(int32_t v, int level, int64_t prefix, bool &match)
{
    if (level == 1) { match = true; return v >> 20; }
    if (level == 2) { match = (v >> 20) == prefix; return (v >> 10) & 1023; }
    match = (v >> 10) == prefix;
    return v & 1023;
}

// warp per range item: histogram of candidate weight by gain for saturated key blocks
template <int KEY = KEY_T>
__global__ void __launch_bounds__(kThreads) k_hist(const Dev *devs, const int2 *items, int32_t n_items, int level)
{
    __shared__ int active[kWarps][64];
    __shared__ long long prefix[kWarps][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t item = blockIdx.x * kWarps + wid;
    if (item >= item_count(devs, items, n_items, 0)) return;
    int32_t range;
    const Dev d = item_of(devs, items, item, range);
    int a_any = 0;
    for (int t = lane; t < 64; t += 32) {
        int a = 0;
        if (t < d.k) {
            if (level == 0) {
                a = d.tot[t] > 0 && d.tot[t] > stage_cap<KEY>(d, t);
            } else {
                const Sel sl = d.sel[t];
                a = sl.mode == SEL_REFINE && sl.level == level;
                prefix[wid][t] = sl.g;
            }
        }
        active[wid][t] = a;
        a_any |= a;
    }
    if (!__any_sync(kFull, a_any)) return;
    __syncwarp();
    const int32_t n = d.cand_cnt[range];
    const uint64_t *cand = d.cand + (int64_t)range * kRange;
    for (int i = lane; i < n; i += 32) {
        int t, ul, key;
        int32_t g;
        if (!decode_key<KEY>(cand[i], key, t, g, ul) || !active[wid][key]) continue;
        t = key;
        const unsigned long long c = d.vw ? (unsigned long long)d.vw[range * kRange + ul] : 1ull;
        int bin;
        if (level == 0) {
            bin = g < kBins - 1 ? g : kBins - 1;
        } else {
            if (g < kBins - 1) continue;
            bool match;
            bin = refine_digit(g - (kBins - 1), level, prefix[wid][t], match);
            if (!match) continue;
        }
        atomicAdd(&d.hist[(int64_t)t * kBins + bin], c);
    }
}

// block-wide exclusive scan of 64-bit values (kThreads threads)
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long *wt)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long t = lane < (int)(blockDim.x >> 5) ? wt[lane] : 0;
        unsigned long long s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        wt[lane] = s - t;
    }
    __syncthreads();
    const unsigned long long r = wt[wid] + x - v;
    __syncthreads();
    return r;
}

// one CTA per block item (instance, t): threshold of the (gain desc, id asc) prefix that fits
template <int KEY = KEY_T>
__global__ void __launch_bounds__(kThreads) k_select(const Dev *devs, const int2 *items, int32_t n_items, int level)
{
    __shared__ unsigned long long wt[32];
    __shared__ int found_bin;
    __shared__ long long found_before;
    const int tid = threadIdx.x;
    if ((int32_t)blockIdx.x >= item_count(devs, items, n_items, 2)) return;
    int32_t t;
    const Dev d = item_of(devs, items, blockIdx.x, t);
    Sel sl = d.sel[t];
    long long cap;
    int nbins;
    if (level == 0) {
        const long long tot = d.tot[t];
        cap = stage_cap<KEY>(d, t);
        if (tot == 0 || tot <= cap) {
            if (KEY == KEY_T) {
                // the gain step filled the level-0 row of every target block
                unsigned long long *row0 = d.hist + (int64_t)t * kBins;
                if (tot)
                    for (int b = tid; b < kBins; b += kThreads) row0[b] = 0;
            }
            if (tid == 0) {
                Sel o;
                o.mode = SEL_ALL; o.level = 0; o.g = 0; o.rem = 0;
                d.sel[t] = o;
                d.tot[t] = 0;
            }
            return;
        }
        nbins = kBins;
    } else {
        if (sl.mode != SEL_REFINE || sl.level != level) return;
        cap = sl.rem;
        nbins = level == 1 ? 2048 : 1024;
    }
    unsigned long long *row = d.hist + (int64_t)t * kBins;
    // thread i owns bins [nbins - per*(i+1), nbins - per*i), visited from high to low
    const int per = nbins / kThreads;
    const int hi = nbins - per * tid;
    unsigned long long sum = 0;
    for (int b = hi - 1; b >= hi - per; --b) sum += row[b];
    if (tid == 0) { found_bin = -1; found_before = 0; }
    const unsigned long long before = block_scan_u64(sum, wt);
    if ((long long)before <= cap && (long long)(before + sum) > cap) {
        unsigned long long c = before;
        for (int b = hi - 1; b >= hi - per; --b) {
            if ((long long)(c + row[b]) > cap) {
                found_bin = b;
                found_before = (long long)c;
                break;
            }
            c += row[b];
        }
    }
    __syncthreads();
    for (int b = tid; b < nbins; b += kThreads) row[b] = 0;
    if (tid == 0) {
        const int fb = found_bin;
        const long long rem = cap - found_before;
        Sel o;
        if (level == 0) {
            d.tot[t] = 0;
            if (fb < kBins - 1) {
                o.mode = SEL_THRESH; o.level = 0; o.g = fb; o.rem = rem;
            } else {
                o.mode = SEL_REFINE; o.level = 1; o.g = 0; o.rem = rem;
            }
        } else {
            const long long p = level == 1 ? fb : (sl.g << 10) | fb;
            if (level == 3) {
                o.mode = SEL_THRESH; o.level = 0; o.g = (kBins - 1) + p; o.rem = rem;
            } else {
                o.mode = SEL_REFINE; o.level = level + 1; o.g = p; o.rem = rem;
            }
        }
        d.sel[t] = o;
    }
}

// one CTA per tile item (instance, tile of 8 ranges): weight of the candidates at their
// block's threshold gain, per block
template <int KEY = KEY_T>
__global__ void __launch_bounds__(kThreads) k_tie_sum(const Dev *devs, const int2 *items, int32_t n_items)
{
    __shared__ int thr[64];
    __shared__ int32_t gthr[64];
    __shared__ unsigned long long ts[64];
    __shared__ int any;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if ((int32_t)blockIdx.x >= item_count(devs, items, n_items, 1)) return;
    int32_t tile;
    const Dev d = item_of(devs, items, blockIdx.x, tile);
    if (tid == 0) any = 0;
    __syncthreads();
    if (tid < 64) {
        ts[tid] = 0;
        int a = 0;
        if (tid < d.k) {
            const Sel sl = d.sel[tid];
            a = sl.mode == SEL_THRESH;
            gthr[tid] = (int32_t)sl.g;
        }
        thr[tid] = a;
        if (a) any = 1;
    }
    __syncthreads();
    if (!any) return;
    const int32_t range = tile * kWarps + wid;
    if (range < d.n_ranges) {
        const int32_t n = d.cand_cnt[range];
        const uint64_t *cand = d.cand + (int64_t)range * kRange;
        for (int i = lane; i < n; i += 32) {
            int t, ul, key;
            int32_t g;
            if (decode_key<KEY>(cand[i], key, t, g, ul) && thr[key] && g == gthr[key])
                atomicAdd(&ts[key], d.vw ? (unsigned long long)d.vw[range * kRange + ul] : 1ull);
        }
    }
    __syncthreads();
    if (tid < d.k && thr[tid]) d.tie[(int64_t)tid * d.n_tiles + tile] = (int64_t)ts[tid];
}

// one CTA per block item: exclusive prefix of the tie weights over the tiles, in tile order
__global__ void __launch_bounds__(1024) k_tie_scan(const Dev *devs, const int2 *items, int32_t n_items)
{
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long carry;
    if ((int32_t)blockIdx.x >= item_count(devs, items, n_items, 2)) return;
    int32_t t;
    const Dev d = item_of(devs, items, blockIdx.x, t);
    if (d.sel[t].mode != SEL_THRESH) return;
    int64_t *row = d.tie + (int64_t)t * d.n_tiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < d.n_tiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const unsigned long long v = i < d.n_tiles ? (unsigned long long)row[i] : 0;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wt[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const unsigned long long tt = wt[lane];
            unsigned long long s = tt;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += y;
            }
            wt[lane] = s - tt;
        }
        __syncthreads();
        const unsigned long long ex = carry + wt[wid] + x - v;
        if (i < d.n_tiles) row[i] = (int64_t)ex;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = ex + v;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ apply
constexpr uint8_t kRvNone = 0xFF, kRvBack = 0x80;   // revert variant: per candidate slot marks

struct alignas(16) ApplyWarp {
    int32_t off[33];
    int32_t jb[32];
    int32_t a[32];
    int32_t t[32];
};

// Applies up to kPins moved pins per lane (vertex moved a -> t, incident net e): Phi(e,a)--,
// Phi(e,t)++, and from the old values the Lambda / S1 bit flips and the objective change
// (Sec. 2: a pin count that steps 1 -> 0 removes the block from Lambda(e), 0 -> 1 adds it,
// each changing (lambda-1) by one; a step into or out of the value 1 flips the S1 bit), then
// stamps e as moved in round r.  Every load and atomic of the kPins pins is issued before any
// result is used, so their latencies overlap.
constexpr int kPins = 4;

// RVC (LP apply with the revert variant on): also counts the movers of every net (d.rv_net)
// and, in `shared`, the moved incidences on nets with several movers (a second mover adds its
// own incidence and the first one's, later movers their own).
template <typename Rec, bool STAMP = true, bool RVC = false>
__device__ __forceinline__ long long apply_pins(const Dev &d, Rec *recs, const ApplyWarp &w_,
                                                int32_t i0, int32_t total, int32_t r, int32_t *shared = nullptr)
{
    typedef typename RecIO<Rec>::Lam Lam;
    int32_t e[kPins], a[kPins], t[kPins], oa[kPins], ot[kPins], w[kPins], mv[kPins];
    bool ok[kPins];
#pragma unroll
    for (int q = 0; q < kPins; ++q) {
        const int32_t i = i0 + q * 32;
        ok[q] = i < total;
        e[q] = 0; a[q] = 0; t[q] = 0;
        if (ok[q]) {
            const int v = slot_of(w_.off, i);
            a[q] = w_.a[v];
            t[q] = w_.t[v];
            e[q] = d.inc[w_.jb[v] + (i - w_.off[v])];
        }
    }
#pragma unroll
    for (int q = 0; q < kPins; ++q) {
        if (!ok[q]) continue;
        const bool wide = e[q] < 0;
        const int32_t ee = e[q] & kNetMask;
        const int32_t wrow = wide ? d.widx[ee] : 0;
        Rec *rc = recs + ee;
        mv[q] = STAMP ? __ldcg(&rc->mv) : 0;
        w[q] = __ldg(&rc->w) & 0x7fffffff;
        oa[q] = phi_add(d, ee, a[q], -1, wide, wrow);
        ot[q] = phi_add(d, ee, t[q], +1, wide, wrow);
        if (RVC && d.rv_net) {
            const int32_t before = atomicAdd(&d.rv_net[ee], 1);
            *shared += before == 1 ? 2 : (before >= 2 ? 1 : 0);
        }
    }
    long long dobj = 0;
#pragma unroll
    for (int q = 0; q < kPins; ++q) {
        if (!ok[q]) continue;
        Rec *rc = recs + (e[q] & kNetMask);
        const Lam ba = (Lam)1 << a[q], bt = (Lam)1 << t[q];
        const Lam lx = (oa[q] == 1 ? ba : (Lam)0) | (ot[q] == 0 ? bt : (Lam)0);
        const Lam sx = ((oa[q] == 1 || oa[q] == 2) ? ba : (Lam)0) | ((ot[q] == 0 || ot[q] == 1) ? bt : (Lam)0);
        if (sizeof(Lam) == 8) {
            if (lx) atomicXor(reinterpret_cast<unsigned long long *>(&rc->lam), (unsigned long long)lx);
            if (sx) atomicXor(reinterpret_cast<unsigned long long *>(&rc->s1), (unsigned long long)sx);
        } else {
            if (lx) atomicXor(reinterpret_cast<unsigned int *>(&rc->lam), (unsigned int)lx);
            if (sx) atomicXor(reinterpret_cast<unsigned int *>(&rc->s1), (unsigned int)sx);
        }
        // stamp: every writer of round r derives the same value from the pre-round stamp,
        // and one that already sees round r leaves it alone
        if (STAMP) {
            const int32_t last = mv[q] >> 1;
            if (last != r) rc->mv = (r << 1) | (last == r - 1 ? 1 : 0);
        }
        dobj += (long long)(ot[q] == 0 ? w[q] : 0) - (long long)(oa[q] == 1 ? w[q] : 0);
    }
    return dobj;
}

// Per-warp approval state of one instance.
struct ApplyInst {
    int mode[64];
    int32_t gthr[64];
    long long rem[64];
};

__device__ __forceinline__ bool apply_refresh(const Dev &d, ApplyInst &ai, int32_t &r)
{
    const int lane = threadIdx.x & 31;
    int thr_any = 0;
    for (int t = lane; t < 64; t += 32) {
        int md = SEL_ALL;
        if (t < d.k) {
            const Sel sl = d.sel[t];
            md = sl.mode;
            ai.gthr[t] = (int32_t)sl.g;
            ai.rem[t] = sl.rem;
        }
        ai.mode[t] = md;
        thr_any |= md == SEL_THRESH;
    }
    r = d.rs[0];
    __syncwarp();
    return __any_sync(kFull, thr_any) != 0;
}

// The id-ordered tie prefix of a range: per key block at its threshold gain, the weight of
// the passing candidates at the threshold in the earlier ranges of the tile (the tile's
// exclusive prefix plus the earlier ranges of the same tile).  Only needed, and only built,
// when the range holds such a candidate; returns whether it does.
template <int KEY>
__device__ __forceinline__ bool range_tie_prefix(const Dev &d, int32_t range, bool any_thr, const ApplyInst &ai,
                                                 unsigned long long *run, const uint64_t *cand, int32_t ncand)
{
    const int lane = threadIdx.x & 31;
    const int *mode = ai.mode;
    const int32_t *gthr = ai.gthr;
    bool has_tie = false;
    if (any_thr) {
        bool tie = false;
        for (int i = lane; i < ncand; i += 32) {
            int t, ul, key;
            int32_t g;
            const bool in = decode_key<KEY>(cand[i], key, t, g, ul);
            tie = tie || (in && mode[key] == SEL_THRESH && g == gthr[key]);
        }
        has_tie = __any_sync(kFull, tie) != 0;
    }
    if (has_tie) {
        const int32_t tile = range / kWarps;
        for (int t = lane; t < 64; t += 32)
            run[t] = (t < d.k && mode[t] == SEL_THRESH)
                         ? (unsigned long long)d.tie[(int64_t)t * d.n_tiles + tile] : 0ull;
        __syncwarp();
        for (int32_t pr = tile * kWarps; pr < range; ++pr) {
            const int32_t n2 = d.cand_cnt[pr];
            const uint64_t *c2 = d.cand + (int64_t)pr * kRange;
            for (int i = lane; i < n2; i += 32) {
                int t, ul, key;
                int32_t g;
                if (decode_key<KEY>(c2[i], key, t, g, ul) && mode[key] == SEL_THRESH && g == gthr[key])
                    atomicAdd(&run[key], d.vw ? (unsigned long long)d.vw[pr * kRange + ul] : 1ull);
            }
        }
        __syncwarp();
    }
    return has_tie;
}

// Approval of the candidate in this lane's slot of a 32-candidate chunk: above its key
// block's threshold gain, or at it and within the block's remainder in id order (KEY_A:
// the weight before it; otherwise: including its own weight).
template <int KEY>
__device__ __forceinline__ bool approve_slot(const Dev &d, int32_t range, const uint64_t *cand, int32_t ncand,
                                             int idx, const ApplyInst &ai, unsigned long long *run, int &t,
                                             int &key, int32_t &g, int &ul, unsigned long long &cw)
{
    const int lane = threadIdx.x & 31;
    bool appr = false, tie = false;
    t = 0; key = 0; g = 0; ul = 0; cw = 1;
    if (idx < ncand) {
        const bool in = decode_key<KEY>(cand[idx], key, t, g, ul);
        if (d.vw) cw = (unsigned long long)d.vw[range * kRange + ul];
        const int md = ai.mode[key];
        if (in) {
            if (md == SEL_ALL || g > ai.gthr[key]) appr = true;
            else if (g == ai.gthr[key]) tie = true;
        }
    }
    unsigned tm = __ballot_sync(kFull, tie);
    while (tm) {
        const int l = __ffs(tm) - 1;
        tm &= tm - 1;
        if (lane == l) {
            appr = (long long)(run[key] + (KEY == KEY_A ? 0ull : cw)) <= ai.rem[key];
            run[key] += cw;
        }
        __syncwarp();
    }
    return appr;
}

// One range item of the apply step (see k_apply).  KEY_T: LP (stamps the nets, records the
// revert variant's source blocks); KEY_TS: rebalancing (no stamps).
template <typename Rec, int KEY>
__device__ __forceinline__ void apply_range(const Dev &d, int32_t range, int32_t r, bool any_thr,
                                            const ApplyInst &ai, unsigned long long *run,
                                            unsigned long long *bwd, ApplyWarp &w_, long long &idobj,
                                            int32_t &iappr, int32_t &ipins, int32_t &ishared)
{
    const int lane = threadIdx.x & 31;
    Rec *recs = reinterpret_cast<Rec *>(d.rec);
    const int32_t ncand = d.cand_cnt[range];
    if (ncand == 0) return;
    const uint64_t *cand = d.cand + (int64_t)range * kRange;
    range_tie_prefix<KEY>(d, range, any_thr, ai, run, cand, ncand);
    for (int32_t c0 = 0; c0 < ncand; c0 += 32) {
        const int idx = c0 + lane;
        int t, key, ul;
        int32_t g;
        unsigned long long cw;
        const bool appr = approve_slot<KEY>(d, range, cand, ncand, idx, ai, run, t, key, g, ul, cw);
        int32_t deg = 0, jb = 0, a = 0;
        if (appr) {
            const int32_t u = range * kRange + ul;
            a = d.part[u];
            d.part[u] = (uint8_t)t;
            atomicAdd(&bwd[a], (unsigned long long)(-(long long)cw));
            atomicAdd(&bwd[t], cw);
            jb = d.vtx_off[u];
            deg = d.vtx_off[u + 1] - jb;
            ++iappr;
            ipins += deg;
        }
        if (KEY == KEY_T && d.rv_src && idx < ncand) d.rv_src[(int64_t)range * kRange + idx] = appr ? (uint8_t)a : kRvNone;
        int32_t incl = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t total = __shfl_sync(kFull, incl, 31);
        w_.off[lane] = incl - deg;
        w_.jb[lane] = jb;
        w_.a[lane] = a;
        w_.t[lane] = t;
        if (lane == 31) w_.off[32] = total;
        __syncwarp();
        for (int32_t i0 = 0; i0 < total; i0 += 32 * kPins)
            idobj += apply_pins<Rec, KEY == KEY_T, KEY == KEY_T>(d, recs, w_, i0 + lane, total, r, &ishared);
        __syncwarp();
    }
}

// Persistent: each warp walks range items with a grid stride.  For each 32 candidates of a
// range it decides approval (ties at a block's threshold gain in vertex-id order: the warp
// starts from the tile's exclusive tie prefix and adds the ties of the earlier ranges of the
// same tile itself, so warps never wait for each other), then applies the approved moves
// over their incidences flattened across the lanes, so all atomics are in flight at once.
// B as for k_gain.
template <typename Rec, bool B, int KEY = KEY_T>
__global__ void __launch_bounds__(kThreads, 4) k_apply(const Dev d0, const Dev *devs, const int2 *items,
                                                       int32_t n_items, int32_t rr, int32_t sub)
{
    __shared__ ApplyInst ai_w[kWarps];
    __shared__ unsigned long long run[kWarps][64];
    __shared__ unsigned long long bwd_w[kWarps][64];
    __shared__ ApplyWarp aw[kWarps];
    __shared__ Dev dsm[B ? kWarps : 1];
    __shared__ unsigned long long objd, napp, mpins;
    __shared__ int warps_done;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    bwd_w[wid][lane] = 0;
    bwd_w[wid][lane + 32] = 0;
    if (tid == 0) { objd = 0; napp = 0; mpins = 0; warps_done = 0; }
    __syncthreads();   // before any warp can add into another warp's slots (at its end)
    long long dobj = 0;
    int32_t nappr = 0, npins = 0, r = 0, nshared = 0;
    int inst_prev = -1;
    bool any_thr = false;
    const int32_t n_it = B ? n_items : d0.n_ranges;
    // static assignment: the 8 warps of a CTA take the 8 ranges of one tile, whose candidates
    // the tie prefixes read (measured faster here than the gain step's dynamic distribution)
    (void)sub;
    for (int32_t item = blockIdx.x * kWarps + wid; item < n_it; item += gridDim.x * kWarps) {
        long long idobj = 0;
        int32_t iappr = 0, ipins = 0, ishared = 0;
        if (B) {
            const int2 it = items[item];
            if (it.x != inst_prev) {
                load_dev(dsm[wid], devs + it.x);
                any_thr = apply_refresh(dsm[wid], ai_w[wid], r);
                inst_prev = it.x;
            }
            const Dev &d = dsm[wid];
            apply_range<Rec, KEY>(d, it.y, r, any_thr, ai_w[wid], run[wid], bwd_w[wid], aw[wid], idobj, iappr, ipins,
                                  ishared);
            for (int o = 16; o; o >>= 1) {
                idobj += __shfl_xor_sync(kFull, idobj, o);
                iappr += __shfl_xor_sync(kFull, iappr, o);
                ipins += __shfl_xor_sync(kFull, ipins, o);
            }
            __syncwarp();
            for (int t = lane; t < 64; t += 32) {
                const unsigned long long v = bwd_w[wid][t];
                if (v) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&d.bw[t]), v);
                    bwd_w[wid][t] = 0;
                }
            }
            if (lane == 0) {
                unsigned long long *row = reinterpret_cast<unsigned long long *>(d.stats + (int64_t)rr * ST_N);
                if (idobj) atomicAdd(reinterpret_cast<unsigned long long *>(d.obj), (unsigned long long)idobj);
                if (iappr) atomicAdd(row + ST_APPR, (unsigned long long)iappr);
                if (ipins) atomicAdd(row + ST_MOVED, (unsigned long long)ipins);
                if (KEY == KEY_T && ipins && d.rv_cnt) atomicAdd(d.rv_cnt, (unsigned long long)ipins);
            }
            __syncwarp();
        } else {
            if (inst_prev < 0) {
                any_thr = apply_refresh(d0, ai_w[wid], r);
                inst_prev = 0;
            }
            apply_range<Rec, KEY>(d0, item, r, any_thr, ai_w[wid], run[wid], bwd_w[wid], aw[wid], idobj, iappr, ipins,
                                  ishared);
            dobj += idobj;
            nappr += iappr;
            npins += ipins;
            nshared += ishared;
        }
    }
    if (!B && KEY == KEY_T && d0.rv_cnt) {
        // revert variant: moved incidences on nets with several movers (sizes the order-statistics table)
        nshared = __reduce_add_sync(kFull, nshared);
        if (lane == 0 && nshared) atomicAdd(d0.rv_cnt + 1, (unsigned long long)nshared);
    }
    if (!B) {
        // as in k_gain: partial sums into warp 0's slots, the last warp to finish flushes
        for (int o = 16; o; o >>= 1) {
            dobj += __shfl_xor_sync(kFull, dobj, o);
            nappr += __shfl_xor_sync(kFull, nappr, o);
            npins += __shfl_xor_sync(kFull, npins, o);
        }
        if (wid != 0) {
            for (int t = lane; t < 64; t += 32)
                if (bwd_w[wid][t]) atomicAdd(&bwd_w[0][t], bwd_w[wid][t]);
        }
        if (lane == 0) {
            if (dobj) atomicAdd(&objd, (unsigned long long)dobj);
            if (nappr) atomicAdd(&napp, (unsigned long long)nappr);
            if (npins) atomicAdd(&mpins, (unsigned long long)npins);
        }
        __threadfence_block();
        __syncwarp();
        int last = 0;
        if (lane == 0) last = atomicAdd(&warps_done, 1) == kWarps - 1;
        last = __shfl_sync(kFull, last, 0);
        if (last) {
            __threadfence_block();
            for (int t = lane; t < 64 && t < d0.k; t += 32) {
                const unsigned long long v = atomicAdd(&bwd_w[0][t], 0ull);
                if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&d0.bw[t]), v);
            }
            if (lane == 0) {
                unsigned long long *row = reinterpret_cast<unsigned long long *>(d0.stats + (int64_t)rr * ST_N);
                const unsigned long long o1 = atomicAdd(&objd, 0ull), a1 = atomicAdd(&napp, 0ull),
                                         p1 = atomicAdd(&mpins, 0ull);
                if (o1) atomicAdd(reinterpret_cast<unsigned long long *>(d0.obj), o1);
                if (a1) atomicAdd(row + ST_APPR, a1);
                if (p1) atomicAdd(row + ST_MOVED, p1);
                if (KEY == KEY_T && p1 && d0.rv_cnt) atomicAdd(d0.rv_cnt, p1);
            }
        }
    }
}

// ------------------------------------------------------------------ revert variant
// Attributed gains (Sec. 5.2) of a sub-round's approved moves, with every net seeing its moves
// in ascending vertex id: the gain of u (a -> b) if the moves of smaller ids had been made
// first.  Lemma 1 (Sec. 5.4) gives it from order statistics of the moves that touch (e, i),
// with the vertex id as the position in the sequence:
//     +omega(e)  iff  Psi(e, a) = 0, u = max out(e, a), min in(e, a) > u
//     -omega(e)  iff  Psi(e, b) = 0, u = min in(e, b),  max out(e, b) < u
// where Psi(e, i) is the number of pins of e that were in block i at the start of the sub-round
// and stayed: Phi(e, i) after the moves minus |in(e, i)|.  Most touched nets have one mover in
// a sub-round; for them the two conditions reduce to Phi(e, a) = 0 and Phi(e, b) = 1 after the
// move.  The apply step counts the movers of every net and the moved incidences of nets with
// several movers; INSERT records max out, min in and |in| of those nets' (e, i) in an
// open-addressing table sized to that count, EVAL sums the terms per move and marks the moves
// whose sum is negative, and the revert step moves those back (Sec. 6).  Balance holds after it: each block's approval was
// checked against its weight at the start of the sub-round, without credit for departures.
struct alignas(16) RvSlot {
    unsigned long long key;   // e * 64 + i, kRvEmpty when free
    int32_t max_out;          // largest id of a mover that left block i (a pin of e), -1 if none
    int32_t min_in;           // smallest id of a mover that entered block i, INT32_MAX if none
    int32_t n_in;             // number of movers that entered block i
    int32_t pad[3];
};
static_assert(sizeof(RvSlot) == kRvSlotBytes, "revert table slot size");
constexpr unsigned long long kRvEmpty = ~0ull;

// slots in use this sub-round: a power of two >= 4 x moved incidences of shared nets (>= 2 x
// keys), at most the capacity (>= 2 P >= keys, so a free slot always exists)
__device__ __forceinline__ uint64_t rv_slots(const Dev &d)
{
    const uint64_t need = 4ull * __ldcg(d.rv_cnt + 1);
    uint64_t c = 1024;
    while (c < need && c < (uint64_t)d.rv_cap) c <<= 1;
    return c;
}

// find (or insert) key by linear probing; at most `mask + 1` probes
__device__ __forceinline__ RvSlot *rv_find(RvSlot *tab, uint64_t mask, unsigned long long key, bool insert)
{
    uint64_t p = splitmix64_output(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        RvSlot *sl = tab + p;
        unsigned long long cur = __ldcg(&sl->key);
        if (cur == key) return sl;
        if (cur == kRvEmpty) {
            if (!insert) return nullptr;
            cur = atomicCAS(&sl->key, kRvEmpty, key);
            if (cur == kRvEmpty || cur == key) return sl;
        }
        p = (p + 1) & mask;
    }
    return nullptr;
}

__global__ void k_rv_clear(const Dev d)
{
    const uint64_t n = rv_slots(d);
    RvSlot *tab = reinterpret_cast<RvSlot *>(d.rv_tab);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        RvSlot sl;
        sl.key = kRvEmpty;
        sl.max_out = -1;
        sl.min_in = 0x7fffffff;
        sl.n_in = 0;
        sl.pad[0] = sl.pad[1] = sl.pad[2] = 0;
        tab[i] = sl;
    }
}

struct alignas(16) RvWarp {
    ApplyWarp w;
    int32_t u[32];
    int32_t g[32];
};

enum { RV_INSERT = 0, RV_EVAL = 1 };

// Warp per range: the approved movers of each 32 candidates, their incidences flattened over
// the lanes, one of the passes above per launch.
template <typename Rec, int PASS>
__global__ void __launch_bounds__(kThreads) k_rv_pass(const Dev d)
{
    __shared__ RvWarp rw_[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t range = blockIdx.x * kWarps + wid;
    if (range >= d.n_ranges) return;
    const int32_t ncand = d.cand_cnt[range];
    if (ncand == 0) return;
    RvWarp &rw = rw_[wid];
    const uint64_t mask = (PASS == RV_INSERT || PASS == RV_EVAL) ? rv_slots(d) - 1 : 0;
    RvSlot *tab = reinterpret_cast<RvSlot *>(d.rv_tab);
    const Rec *recs = reinterpret_cast<const Rec *>(d.rec);
    const uint64_t *cand = d.cand + (int64_t)range * kRange;
    uint8_t *src = d.rv_src + (int64_t)range * kRange;
    bool lost = false;
    for (int32_t c0 = 0; c0 < ncand; c0 += 32) {
        const int idx = c0 + lane;
        int32_t deg = 0, jb = 0, u = 0;
        int t = 0, a = 0;
        const uint8_t sa = idx < ncand ? src[idx] : kRvNone;
        if (sa != kRvNone) {
            int ul;
            int32_t g;
            decode(cand[idx], t, g, ul);
            u = range * kRange + ul;
            a = sa;
            jb = d.vtx_off[u];
            deg = d.vtx_off[u + 1] - jb;
        }
        int32_t incl = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t total = __shfl_sync(kFull, incl, 31);
        rw.w.off[lane] = incl - deg;
        rw.w.jb[lane] = jb;
        rw.w.a[lane] = a;
        rw.w.t[lane] = t;
        rw.u[lane] = u;
        rw.g[lane] = 0;
        if (lane == 31) rw.w.off[32] = total;
        __syncwarp();
        for (int32_t i = lane; i < total; i += 32) {
            const int v = slot_of(rw.w.off, i);
            const int32_t e = d.inc[rw.w.jb[v] + (i - rw.w.off[v])];
            const int32_t ee = e & kNetMask;
            const int32_t movers = __ldcg(&d.rv_net[ee]);
            const int32_t av = rw.w.a[v], bv = rw.w.t[v], uv = rw.u[v];
            if (PASS == RV_INSERT) {
                if (movers < 2) continue;
                RvSlot *s_a = rv_find(tab, mask, (unsigned long long)ee * 64 + av, true);
                RvSlot *s_b = rv_find(tab, mask, (unsigned long long)ee * 64 + bv, true);
                if (!s_a || !s_b) {
                    lost = true;
                    continue;
                }
                atomicMax(&s_a->max_out, uv);
                atomicMin(&s_b->min_in, uv);
                atomicAdd(&s_b->n_in, 1);
            } else {
                const bool wide = e < 0;
                const int32_t wrow = wide ? d.widx[ee] : 0;
                const int32_t pa = phi_get(d, ee, av, wide, wrow), pb = phi_get(d, ee, bv, wide, wrow);
                const int32_t w = __ldg(&recs[ee].w) & 0x7fffffff;
                int32_t g = 0;
                if (movers < 2) {
                    // the only mover of e: Phi(e, a) went 1 -> 0, or Phi(e, b) went 0 -> 1
                    if (pa == 0) g += w;
                    if (pb == 1) g -= w;
                } else {
                    const RvSlot *s_a = rv_find(tab, mask, (unsigned long long)ee * 64 + av, false);
                    const RvSlot *s_b = rv_find(tab, mask, (unsigned long long)ee * 64 + bv, false);
                    if (!s_a || !s_b) {
                        lost = true;
                        continue;
                    }
                    if (pa == s_a->n_in && s_a->max_out == uv && s_a->min_in > uv) g += w;
                    if (pb == s_b->n_in && s_b->min_in == uv && s_b->max_out < uv) g -= w;
                }
                if (g) atomicAdd(&rw.g[v], g);
            }
        }
        __syncwarp();
        if (PASS == RV_EVAL && sa != kRvNone && rw.g[lane] < 0) src[idx] = (uint8_t)(sa | kRvBack);
        __syncwarp();
    }
    if (lost) atomicOr(d.err, ERR_TABLE);
}

// Warp per range: the marked moves go back to their source blocks (Phi, Lambda, S1, block
// weights, objective as in the apply step; the nets keep their round-r stamps).  Resets the
// sub-round's moved-incidence count for the next sub-round.
template <typename Rec>
__global__ void __launch_bounds__(kThreads) k_rv_revert(const Dev d, int32_t rr)
{
    __shared__ ApplyWarp aw[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t range = blockIdx.x * kWarps + wid;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.rv_cnt[0] = 0;
        d.rv_cnt[1] = 0;
    }
    if (range >= d.n_ranges) return;
    const int32_t ncand = d.cand_cnt[range];
    if (ncand == 0) return;
    const uint8_t *src = d.rv_src + (int64_t)range * kRange;
    const uint64_t *cand = d.cand + (int64_t)range * kRange;
    Rec *recs = reinterpret_cast<Rec *>(d.rec);
    const int32_t r = d.rs[0];
    long long dobj = 0;
    int32_t nrev = 0;
    for (int32_t c0 = 0; c0 < ncand; c0 += 32) {
        const int idx = c0 + lane;
        const uint8_t sa = idx < ncand ? src[idx] : kRvNone;
        const bool back = sa != kRvNone && (sa & kRvBack);
        if (!__any_sync(kFull, back)) continue;
        int32_t deg = 0, jb = 0;
        int t = 0, a = 0;
        if (back) {
            int ul;
            int32_t g;
            decode(cand[idx], t, g, ul);
            const int32_t u = range * kRange + ul;
            a = sa & 0x3F;
            d.part[u] = (uint8_t)a;
            const long long cw = d.vw ? d.vw[u] : 1;
            atomicAdd(reinterpret_cast<unsigned long long *>(&d.bw[t]), (unsigned long long)(-cw));
            atomicAdd(reinterpret_cast<unsigned long long *>(&d.bw[a]), (unsigned long long)cw);
            jb = d.vtx_off[u];
            deg = d.vtx_off[u + 1] - jb;
            ++nrev;
        }
        int32_t incl = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t total = __shfl_sync(kFull, incl, 31);
        aw[wid].off[lane] = incl - deg;
        aw[wid].jb[lane] = jb;
        aw[wid].a[lane] = t;     // the move back leaves the target block ...
        aw[wid].t[lane] = a;     // ... for the source block
        if (lane == 31) aw[wid].off[32] = total;
        __syncwarp();
        for (int32_t i0 = 0; i0 < total; i0 += 32 * kPins)
            dobj += apply_pins<Rec>(d, recs, aw[wid], i0 + lane, total, r);
        __syncwarp();
    }
    for (int o = 16; o; o >>= 1) {
        dobj += __shfl_xor_sync(kFull, dobj, o);
        nrev += __shfl_xor_sync(kFull, nrev, o);
    }
    if (lane == 0) {
        if (dobj) atomicAdd(reinterpret_cast<unsigned long long *>(d.obj), (unsigned long long)dobj);
        if (nrev) atomicAdd(reinterpret_cast<unsigned long long *>(d.stats + (int64_t)rr * ST_N + ST_REV),
                            (unsigned long long)nrev);
    }
}

// Pi of one handle widened to int32 (batch partition read-back)
__global__ void k_part_widen(const uint8_t *part, int32_t n, int32_t *out)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = part[v];
}

// thread per instance: per-round objective and heaviest block; advance the round state
__global__ void k_round_end(const Dev *devs, int32_t n_inst, int32_t rr, int32_t advance = 1)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    const Dev d = devs[i];
    unsigned long long *row = reinterpret_cast<unsigned long long *>(d.stats + (int64_t)rr * ST_N);
    long long mx = 0;
    for (int t = 0; t < d.k; ++t) mx = d.bw[t] > mx ? d.bw[t] : mx;
    row[ST_OBJ] = (unsigned long long)*d.obj;
    row[ST_MAXW] = (unsigned long long)mx;
    if (advance) {
        d.rs[0] += 1;
        d.rs[1] = 1;
    }
}

// Rebalancing, source side (KEY_A): persistent, a warp per range item with a grid stride (the
// per-block thresholds are read once per warp); marks the candidates that may leave their block
// (bit 24) and adds their weights to the per-target totals of the target-side stage.
__global__ void __launch_bounds__(kThreads) k_rb_mark(const Dev d)
{
    __shared__ ApplyInst ai_w[kWarps];
    __shared__ unsigned long long run_w[kWarps][64];
    __shared__ unsigned long long tot_w[kWarps][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t r;
    const bool any_thr = apply_refresh(d, ai_w[wid], r);
    tot_w[wid][lane] = 0;
    tot_w[wid][lane + 32] = 0;
    __syncwarp();
    for (int32_t range = blockIdx.x * kWarps + wid; range < d.n_ranges; range += gridDim.x * kWarps) {
        const int32_t ncand = d.cand_cnt[range];
        if (ncand == 0) continue;
        uint64_t *cand = d.cand + (int64_t)range * kRange;
        range_tie_prefix<KEY_A>(d, range, any_thr, ai_w[wid], run_w[wid], cand, ncand);
        for (int32_t c0 = 0; c0 < ncand; c0 += 32) {
            const int idx = c0 + lane;
            int t, key, ul;
            int32_t g;
            unsigned long long cw;
            const bool sel = approve_slot<KEY_A>(d, range, cand, ncand, idx, ai_w[wid], run_w[wid], t, key, g, ul, cw);
            if (sel) {
                cand[idx] |= kSelBit;
                atomicAdd(&tot_w[wid][t], cw);
            }
        }
        __syncwarp();
    }
    __syncwarp();
    for (int t = lane; t < 64 && t < d.k; t += 32)
        if (tot_w[wid][t]) atomicAdd(reinterpret_cast<unsigned long long *>(&d.tot[t]), tot_w[wid][t]);
}

__global__ void k_expand_candidates(const Dev *devs, int32_t *target, int64_t *gain)
{
    const Dev d = devs[0];
    const int lane = threadIdx.x & 31;
    const int32_t range = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (range >= d.n_ranges) return;
    const int32_t n = d.cand_cnt[range];
    for (int i = lane; i < n; i += 32) {
        int t, ul;
        int32_t g;
        decode(d.cand[(int64_t)range * kRange + i], t, g, ul);
        target[range * kRange + ul] = t;
        gain[range * kRange + ul] = g;
    }
}

// ------------------------------------------------------------------ launch plans (host)
// A set of instances with one record type, launched together: one instance with its own
// ranges (items == nullptr), or a batch group with explicit (instance, local index) items.
struct Plan {
    Dev d0{};                     // single instance: its state by value (kernel parameter)
    const Dev *devs = nullptr;
    const int2 *ranges = nullptr, *tiles = nullptr, *blocks = nullptr;
    int32_t n_ranges = 0, n_tiles = 0, n_blocks = 0, n_inst = 0;
    int32_t S_max = 0;
    bool levels = false;   // some instance can have gains >= kBins - 1
    bool rec32 = false;
    bool revert = false;   // revert variant (single instance only)
    int grid_gain = 0, grid_apply = 0;
    cudaStream_t st = nullptr;
    int64_t *launches = nullptr;
    hgp_handle *prof = nullptr;   // per-phase event timing (single-instance launches only)
};

template <typename K>
int persistent_grid(int device, K kernel, int32_t n_ranges)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
    (void)cudaGetLastError();
    int64_t g = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (n_ranges + kWarps - 1) / kWarps;
    if (g > need) g = need;
    return (int)(g < 1 ? 1 : g);
}

void set_grids(Plan &p, int device)
{
    const bool b = p.ranges != nullptr;
    if (p.rec32) {
        p.grid_gain = persistent_grid(device, b ? k_gain<Rec32, true> : k_gain<Rec32, false>, p.n_ranges);
        p.grid_apply = persistent_grid(device, b ? k_apply<Rec32, true> : k_apply<Rec32, false>, p.n_ranges);
    } else {
        p.grid_gain = persistent_grid(device, b ? k_gain<Rec16, true> : k_gain<Rec16, false>, p.n_ranges);
        p.grid_apply = persistent_grid(device, b ? k_apply<Rec16, true> : k_apply<Rec16, false>, p.n_ranges);
    }
}

// Per-phase event timing (profiling mode): a pair of events around each phase instance.
enum { PH_PREP = 0, PH_GAIN = 1, PH_APPROVE = 2, PH_APPLY = 3, PH_END = 4, PH_REVERT = 5 };

cudaError_t phase_begin(hgp_handle *h)
{
    if (!h || !h->profiling) return cudaSuccess;
    if (h->events_used + 2 > h->n_events) {
        // grow the pool (existing events stay valid; pending pairs are kept)
        const int32_t cap = h->n_events ? h->n_events * 2 : 256;
        cudaEvent_t *ev = new (std::nothrow) cudaEvent_t[cap];
        int32_t *ph = new (std::nothrow) int32_t[cap / 2];
        int32_t *ct = new (std::nothrow) int32_t[cap / 2];
        if (!ev || !ph || !ct) {
            delete[] ev; delete[] ph; delete[] ct;
            return cudaErrorMemoryAllocation;
        }
        for (int32_t i = 0; i < h->n_events; ++i) ev[i] = h->events[i];
        for (int32_t i = 0; i < h->n_events / 2; ++i) { ph[i] = h->event_phase[i]; ct[i] = h->event_count[i]; }
        for (int32_t i = h->n_events; i < cap; ++i) {
            cudaError_t e = cudaEventCreate(&ev[i]);
            if (e != cudaSuccess) {
                for (int32_t j = h->n_events; j < i; ++j) cudaEventDestroy(ev[j]);
                delete[] ev; delete[] ph; delete[] ct;
                return e;
            }
        }
        delete[] h->events; delete[] h->event_phase; delete[] h->event_count;
        h->events = ev; h->event_phase = ph; h->event_count = ct;
        h->n_events = cap;
    }
    return cudaEventRecord(h->events[h->events_used], h->stream);
}

cudaError_t phase_end(hgp_handle *h, int phase, int32_t launches)
{
    if (!h || !h->profiling) return cudaSuccess;
    cudaError_t e = cudaEventRecord(h->events[h->events_used + 1], h->stream);
    h->event_phase[h->events_used / 2] = phase;
    h->event_count[h->events_used / 2] = launches;
    h->events_used += 2;
    return e;
}

cudaError_t collect_profile(hgp_handle *h)
{
    if (!h->profiling || h->events_used == 0) return cudaSuccess;
    cudaError_t e = stream_wait(h->stream);
    for (int32_t i = 0; i + 1 < h->events_used && e == cudaSuccess; i += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->events[i], h->events[i + 1]);
        h->prof_ms[h->event_phase[i / 2]] += ms;
        h->prof_launches[h->event_phase[i / 2]] += h->event_count[i / 2];
    }
    h->events_used = 0;
    return e;
}

unsigned warp_grid(int32_t n_items) { return (unsigned)((n_items + kWarps - 1) / kWarps); }

cudaError_t launch_gain(const Plan &p, int32_t s, int32_t rr)
{
    const bool b = p.ranges != nullptr;
    if (p.rec32 && b) k_gain<Rec32, true><<<p.grid_gain, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, s, rr);
    else if (p.rec32) k_gain<Rec32, false><<<p.grid_gain, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, s, rr);
    else if (b) k_gain<Rec16, true><<<p.grid_gain, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, s, rr);
    else k_gain<Rec16, false><<<p.grid_gain, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, s, rr);
    *p.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_prep(const Plan &p)
{
    k_round_prep<<<warp_grid(p.n_ranges), kThreads, 0, p.st>>>(p.devs, p.ranges, p.n_ranges);
    *p.launches += 1;
    return cudaGetLastError();
}

// one round: sub-round lists, then per sub-round gain -> approval -> apply, then round end
cudaError_t launch_round(const Plan &p, int32_t rr)
{
    cudaError_t e = phase_begin(p.prof);
    if (e == cudaSuccess) e = launch_prep(p);
    if (e == cudaSuccess) e = phase_end(p.prof, PH_PREP, 1);
    for (int32_t s = 0; s < p.S_max && e == cudaSuccess; ++s) {
        e = phase_begin(p.prof);
        if (e == cudaSuccess) e = launch_gain(p, s, rr);
        if (e == cudaSuccess) e = phase_end(p.prof, PH_GAIN, 1);
        if (e == cudaSuccess) e = phase_begin(p.prof);
        if (e != cudaSuccess) break;
        int32_t n = 0;
        // the level-0 histogram was filled by the gain step
        k_select<<<p.n_blocks, kThreads, 0, p.st>>>(p.devs, p.blocks, p.n_blocks, 0);
        n += 1;
        if (p.levels) {
            for (int level = 1; level <= 3; ++level) {
                k_hist<<<warp_grid(p.n_ranges), kThreads, 0, p.st>>>(p.devs, p.ranges, p.n_ranges, level);
                k_select<<<p.n_blocks, kThreads, 0, p.st>>>(p.devs, p.blocks, p.n_blocks, level);
                n += 2;
            }
        }
        k_tie_sum<<<p.n_tiles, kThreads, 0, p.st>>>(p.devs, p.tiles, p.n_tiles);
        k_tie_scan<<<p.n_blocks, 1024, 0, p.st>>>(p.devs, p.blocks, p.n_blocks);
        n += 2;
        *p.launches += n;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = phase_end(p.prof, PH_APPROVE, n);
        if (e == cudaSuccess) e = phase_begin(p.prof);
        if (e != cudaSuccess) break;
        const bool b = p.ranges != nullptr;
        if (p.revert) e = cudaMemsetAsync(p.d0.rv_net, 0, sizeof(int32_t) * (size_t)p.d0.m, p.st);
        if (e != cudaSuccess) break;
        if (p.rec32 && b) k_apply<Rec32, true><<<p.grid_apply, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, rr, s);
        else if (p.rec32) k_apply<Rec32, false><<<p.grid_apply, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, rr, s);
        else if (b) k_apply<Rec16, true><<<p.grid_apply, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, rr, s);
        else k_apply<Rec16, false><<<p.grid_apply, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, rr, s);
        *p.launches += 1;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = phase_end(p.prof, PH_APPLY, 1);
        if (p.revert && e == cudaSuccess) e = phase_begin(p.prof);
        if (e == cudaSuccess && p.revert) {
            const unsigned g = warp_grid(p.n_ranges);
            // the apply step counted the movers of every net and the shared incidences
            k_rv_clear<<<p.grid_apply * 4, kThreads, 0, p.st>>>(p.d0);
            if (p.rec32) {
                k_rv_pass<Rec32, RV_INSERT><<<g, kThreads, 0, p.st>>>(p.d0);
                k_rv_pass<Rec32, RV_EVAL><<<g, kThreads, 0, p.st>>>(p.d0);
                k_rv_revert<Rec32><<<g, kThreads, 0, p.st>>>(p.d0, rr);
            } else {
                k_rv_pass<Rec16, RV_INSERT><<<g, kThreads, 0, p.st>>>(p.d0);
                k_rv_pass<Rec16, RV_EVAL><<<g, kThreads, 0, p.st>>>(p.d0);
                k_rv_revert<Rec16><<<g, kThreads, 0, p.st>>>(p.d0, rr);
            }
            *p.launches += 4;
            e = cudaGetLastError();
            if (e == cudaSuccess) e = phase_end(p.prof, PH_REVERT, 4);
        }
    }
    if (e == cudaSuccess) e = phase_begin(p.prof);
    if (e == cudaSuccess) {
        k_round_end<<<(p.n_inst + 127) / 128, 128, 0, p.st>>>(p.devs, p.n_inst, rr);
        *p.launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = phase_end(p.prof, PH_END, 1);
    return e;
}

// the handle's instance state as a device-resident Dev (re-uploaded when it changed)
cudaError_t sync_dev(hgp_handle *h)
{
    if (!h->d_dev) {
        h->d_dev = static_cast<Dev *>(arena_take(h, sizeof(Dev)));
        if (!h->d_dev) {
            cudaError_t e = dev_alloc(reinterpret_cast<void **>(&h->d_dev), sizeof(Dev), h->stream);
            if (e != cudaSuccess) return e;
        }
        h->dev_dirty = true;
    }
    if (!h->dev_dirty) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(h->d_dev, &h->d, sizeof(Dev), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = stream_wait(h->stream);
    if (e == cudaSuccess) h->dev_dirty = false;
    return e;
}

// persistent grid of ctas_per_sm CTAs per SM (at most one warp per range item), or `fallback`
int grid_override(int device, int ctas_per_sm, int fallback, int32_t n_ranges)
{
    if (ctas_per_sm <= 0) return fallback;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int64_t g = (int64_t)sms * ctas_per_sm;
    const int64_t need = (n_ranges + kWarps - 1) / kWarps;
    if (g > need) g = need;
    return (int)(g < 1 ? 1 : g);
}

Plan single_plan(hgp_handle *h)
{
    Plan p;
    p.d0 = h->d;
    p.devs = h->d_dev;
    p.n_ranges = h->d.n_ranges;
    p.n_tiles = h->d.n_tiles;
    p.n_blocks = h->d.k;
    p.n_inst = 1;
    p.S_max = h->d.S;
    p.levels = h->max_vertex_netweight >= kBins - 1;
    p.rec32 = h->d.k > 32;
    p.revert = h->d.rv_src != nullptr;
    if (!h->grid_gain) {
        Plan q = p;
        set_grids(q, h->device);
        h->grid_gain = grid_override(h->device, h->gain_ctas, q.grid_gain, p.n_ranges);
        h->grid_apply = grid_override(h->device, h->apply_ctas, q.grid_apply, p.n_ranges);
    }
    p.grid_gain = h->grid_gain;
    p.grid_apply = h->grid_apply;
    p.st = h->stream;
    p.launches = &h->launches;
    p.prof = h->profiling ? h : nullptr;
    return p;
}

cudaError_t enqueue_rounds(const Plan &p, int64_t *stats, int32_t rounds)
{
    cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(int64_t) * ST_N * (size_t)rounds, p.st);
    if (e == cudaSuccess && p.d0.wq) e = cudaMemsetAsync(p.d0.wq, 0, sizeof(int32_t) * kWqPerRow * (size_t)rounds, p.st);
    for (int32_t rr = 0; rr < rounds && e == cudaSuccess; ++rr) e = launch_round(p, rr);
    return e;
}

}  // namespace

namespace hgp {

int ensure_stats(hgp_handle *h, int32_t rounds)
{
    if (rounds <= h->stats_cap) return HGP_OK;
    int32_t cap = h->stats_cap ? h->stats_cap : 16;
    while (cap < rounds) cap *= 2;
    int64_t *dev = nullptr, *host = nullptr;
    // stats rows, then the work counters of the persistent kernels: 64 sub-rounds x (gain, apply)
    // per row
    const size_t bytes = sizeof(int64_t) * ST_N * (size_t)cap + sizeof(int32_t) * kWqPerRow * (size_t)cap;
    cudaError_t e = cudaSuccess;
    dev = static_cast<int64_t *>(arena_take(h, bytes));
    if (!dev) e = dev_alloc(reinterpret_cast<void **>(&dev), bytes, h->stream);
    if (e == cudaSuccess) {
        host = static_cast<int64_t *>(malloc(sizeof(int64_t) * ST_N * (size_t)cap));
        if (!host) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (!in_arena(h, dev)) dev_free(dev, h->stream);
        return status_of(e);
    }
    if (h->d.stats && !in_arena(h, h->d.stats)) dev_free(h->d.stats, h->stream);
    free(h->h_stats);
    h->d.stats = dev;
    h->d.wq = reinterpret_cast<int32_t *>(dev + (size_t)ST_N * cap);
    h->h_stats = host;
    h->stats_cap = cap;
    h->dev_dirty = true;
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        h->graph_rounds = 0;
    }
    return HGP_OK;
}

static int copy_stats_out(hgp_handle *h, int32_t rounds, hgp_round_stats *stats)
{
    cudaError_t e = cudaMemcpyAsync(h->h_stats, h->d.stats, sizeof(int64_t) * ST_N * (size_t)rounds,
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = stream_wait(h->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    if (stats) {
        for (int32_t rr = 0; rr < rounds; ++rr) {
            const int64_t *row = h->h_stats + (int64_t)rr * ST_N;
            stats[rr].objective = row[ST_OBJ];
            stats[rr].candidates = row[ST_CAND];
            stats[rr].approved = row[ST_APPR];
            stats[rr].eligible = row[ST_ELIG];
            stats[rr].max_block_weight = row[ST_MAXW];
            stats[rr].moved_pins = row[ST_MOVED];
            stats[rr].reverted = row[ST_REV];
        }
    }
    return HGP_OK;
}

int refine_rounds(hgp_handle *h, int32_t rounds, hgp_round_stats *stats)
{
    if (rounds == 0) return HGP_OK;
    if (h->next_round + rounds >= ((int64_t)1 << 30)) return HGP_ERR_UNSUPPORTED;
    int rc = ensure_stats(h, rounds);
    if (rc != HGP_OK) return rc;
    cudaError_t e = sync_dev(h);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    Plan p = single_plan(h);
    const bool use_graph = h->graph && !h->profiling;
    if (use_graph) {
        if (!h->graph_exec || h->graph_rounds != rounds) {
            if (h->graph_exec) {
                cudaGraphExecDestroy(h->graph_exec);
                h->graph_exec = nullptr;
            }
            // the captured launches are counted at replay, not at capture
            int64_t scratch = 0;
            Plan q = p;
            q.launches = &scratch;
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e2 = enqueue_rounds(q, h->d.stats, rounds);
                e = cudaStreamEndCapture(h->stream, &graph);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e == cudaSuccess) {
                h->graph_rounds = rounds;
                h->graph_launches = scratch;
            }
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(h->graph_exec, h->stream);
        if (e == cudaSuccess) h->launches += h->graph_launches;
    } else {
        e = enqueue_rounds(p, h->d.stats, rounds);
        if (e == cudaSuccess) e = collect_profile(h);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    h->next_round += rounds;
    h->all_eligible = false;
    if (h->debug & 16) {
        // fault injection (tests): the maintained objective loses one unit, as if an update
        // had been dropped; written from the host after the rounds, so no kernel is involved
        int64_t obj = 0;
        e = cudaMemcpyAsync(&obj, h->d.obj, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = stream_wait(h->stream);
        obj -= 1;
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.obj, &obj, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = stream_wait(h->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return status_of(e);
        }
    }
    if (stats || (h->debug & 1)) {
        rc = copy_stats_out(h, rounds, stats);
        if (rc != HGP_OK) return rc;
    }
    if (h->debug & 1) {
        int64_t *tmp = nullptr;
        int64_t from_phi = 0, maintained = 0;
        e = dev_alloc(reinterpret_cast<void **>(&tmp), sizeof(int64_t), h->stream);
        if (e == cudaSuccess) e = objective_from_phi(h, tmp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&from_phi, tmp, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&maintained, h->d.obj, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream);
        if (tmp) pool_free(tmp, h->stream);
        if (e == cudaSuccess) e = stream_wait(h->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return status_of(e);
        }
        if (from_phi != maintained) return HGP_ERR_INTERNAL;
    }
    return HGP_OK;
}

int debug_candidates(hgp_handle *h, int32_t s, int32_t *target, int64_t *gain)
{
    const int rc = ensure_stats(h, 1);
    if (rc != HGP_OK) return rc;
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    cudaError_t e = sync_dev(h);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    Plan p = single_plan(h);
    int32_t *t_d = nullptr;
    int64_t *g_d = nullptr;
    e = dev_alloc(reinterpret_cast<void **>(&t_d), sizeof(int32_t) * (size_t)d.n, st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&g_d), sizeof(int64_t) * (size_t)d.n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(t_d, 0xFF, sizeof(int32_t) * (size_t)d.n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_d, 0, sizeof(int64_t) * (size_t)d.n, st);
    // the stats row written here is scratch: refine() clears the stats before use
    if (e == cudaSuccess) e = launch_prep(p);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.wq, 0, sizeof(int32_t) * kWqPerRow, st);
    if (e == cudaSuccess) e = launch_gain(p, s, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.tot, 0, sizeof(int64_t) * 64, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.hist, 0, sizeof(unsigned long long) * (size_t)d.k * kBins, st);
    if (e == cudaSuccess) {
        k_expand_candidates<<<(d.n_ranges * 32 + 255) / 256, 256, 0, st>>>(h->d_dev, t_d, g_d);
        h->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(target, t_d, sizeof(int32_t) * (size_t)d.n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gain, g_d, sizeof(int64_t) * (size_t)d.n, cudaMemcpyDeviceToHost, st);
    if (t_d) pool_free(t_d, st);
    if (g_d) pool_free(g_d, st);
    if (e == cudaSuccess) e = stream_wait(st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    return HGP_OK;
}

}  // namespace hgp

// ================================================================== launch shape
extern "C" int hgp_set_launch_shape(hgp_handle *h, int32_t gain_ctas_per_sm, int32_t apply_ctas_per_sm)
{
    if (!h || gain_ctas_per_sm < 0 || apply_ctas_per_sm < 0) return HGP_ERR_INVALID;
    settle(h);
    const cudaError_t e = stream_wait(h->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    h->gain_ctas = gain_ctas_per_sm;
    h->apply_ctas = apply_ctas_per_sm;
    h->grid_gain = 0;   // recomputed at the next launch
    h->grid_apply = 0;
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        h->graph_rounds = 0;
    }
    return HGP_OK;
}

// ================================================================== rebalancing (Sec. 8)
namespace {

// one approval stage over all candidates of the sub-round, grouped by KEY
template <int KEY>
int64_t launch_stage(const Plan &p, bool levels)
{
    int64_t n = 0;
    k_hist<KEY><<<warp_grid(p.n_ranges), kThreads, 0, p.st>>>(p.devs, p.ranges, p.n_ranges, 0);
    k_select<KEY><<<p.n_blocks, kThreads, 0, p.st>>>(p.devs, p.blocks, p.n_blocks, 0);
    n += 2;
    if (levels) {
        for (int level = 1; level <= 3; ++level) {
            k_hist<KEY><<<warp_grid(p.n_ranges), kThreads, 0, p.st>>>(p.devs, p.ranges, p.n_ranges, level);
            k_select<KEY><<<p.n_blocks, kThreads, 0, p.st>>>(p.devs, p.blocks, p.n_blocks, level);
            n += 2;
        }
    }
    k_tie_sum<KEY><<<p.n_tiles, kThreads, 0, p.st>>>(p.devs, p.tiles, p.n_tiles);
    k_tie_scan<<<p.n_blocks, 1024, 0, p.st>>>(p.devs, p.blocks, p.n_blocks);
    return n + 2;
}

// one rebalancing pass: S sub-rounds of gain (vertices of overloaded blocks), source-side
// selection, target-side approval and apply, then the pass's objective and heaviest block
template <typename Rec>
cudaError_t launch_rebalance_pass(const Plan &p, int32_t pass, RbArgs rb, bool levels)
{
    k_round_prep<<<warp_grid(p.n_ranges), kThreads, 0, p.st>>>(p.devs, p.ranges, p.n_ranges, rb.r);
    *p.launches += 1;
    for (int32_t s = 0; s < p.S_max; ++s) {
        k_gain<Rec, false, true><<<p.grid_gain, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, s, pass, rb);
        *p.launches += 1;
        *p.launches += launch_stage<KEY_A>(p, levels);
        k_rb_mark<<<p.grid_apply, kThreads, 0, p.st>>>(p.d0);
        *p.launches += 1;
        *p.launches += launch_stage<KEY_TS>(p, levels);
        k_apply<Rec, false, KEY_TS><<<p.grid_apply, kThreads, 0, p.st>>>(p.d0, p.devs, p.ranges, p.n_ranges, pass, s);
        *p.launches += 1;
    }
    k_round_end<<<1, 128, 0, p.st>>>(p.devs, 1, pass, 0);
    *p.launches += 1;
    return cudaGetLastError();
}

}  // namespace

extern "C" int hgp_rebalance(hgp_handle *h, int32_t max_passes, hgp_round_stats *stats, int32_t *phases,
                             int32_t *num_passes)
{
    if (!h || max_passes < 0) return HGP_ERR_INVALID;
    settle(h);
    if (num_passes) *num_passes = 0;
    if (max_passes == 0) return HGP_OK;
    // phase-2 priorities are gain + W_max in [0, 2 W_max]; they must fit the 31-bit gain field
    const int64_t off = h->max_vertex_netweight;
    if (2 * off >= ((int64_t)1 << 31)) return HGP_ERR_UNSUPPORTED;
    int rc = ensure_stats(h, max_passes);
    if (rc != HGP_OK) return rc;
    cudaError_t e = sync_dev(h);
    const cudaStream_t st = h->stream;
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d.stats, 0, sizeof(int64_t) * ST_N * (size_t)max_passes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d.wq, 0, sizeof(int32_t) * kWqPerRow * (size_t)max_passes, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    Plan p = single_plan(h);
    p.prof = nullptr;
    std::vector<int32_t> ph;
    int32_t phase = 1, pass = 0;
    while (pass < max_passes && e == cudaSuccess) {
        int64_t bw[64];
        e = cudaMemcpyAsync(bw, h->d.bw, sizeof(int64_t) * (size_t)h->d.k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = stream_wait(st);
        if (e != cudaSuccess) break;
        int64_t heaviest = 0;
        for (int i = 0; i < h->d.k; ++i) heaviest = bw[i] > heaviest ? bw[i] : heaviest;
        if (heaviest <= h->d.lmax) break;
        RbArgs rb;
        rb.r = (1 << 30) + pass;
        rb.phase = phase;
        rb.off = phase == 2 ? (int32_t)off : 0;
        const bool levels = (phase == 2 ? 2 * off : off) >= kBins - 1;
        e = p.rec32 ? launch_rebalance_pass<Rec32>(p, pass, rb, levels)
                    : launch_rebalance_pass<Rec16>(p, pass, rb, levels);
        int64_t appr = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&appr, h->d.stats + (int64_t)pass * ST_N + ST_APPR, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = stream_wait(st);
        if (e != cudaSuccess) break;
        ph.push_back(phase);
        ++pass;
        if (phase == 1) phase = 2;
        else if (appr == 0) break;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    if (pass > 0 && stats) {
        rc = copy_stats_out(h, pass, stats);
        if (rc != HGP_OK) return rc;
    }
    if (phases)
        for (int32_t i = 0; i < pass; ++i) phases[i] = ph[i];
    if (num_passes) *num_passes = pass;
    return HGP_OK;
}

// ================================================================== batch of handles
struct hgp_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int32_t use_graph = 1;
    int32_t gain_ctas = 0, apply_ctas = 0;     // per-SM CTA overrides (0 = occupancy)
    std::vector<hgp_handle *> hs;
    // the members' streams other than the batch's: a call waits (on the device) for their
    // pending work through events[i], and records its end on each such member's own event
    std::vector<cudaStream_t> member_streams;
    std::vector<cudaEvent_t> events;
    int32_t last_rounds = 0;                    // round count of the last hgp_batch_refine
    cudaEvent_t ev_end = nullptr;               // recorded at the end of each hgp_batch_refine
    cudaStream_t aux = nullptr;                 // statistics read-back of a call, after ev_end only
    struct Group {
        Plan plan;
        std::vector<int32_t> members;           // indices into hs
        Dev *d_devs = nullptr;
        int2 *d_items = nullptr;                // ranges, then tiles, then blocks
        int32_t *d_wq = nullptr;                // gain-step work counters [stats_cap * kWqPerRow]
    } g[2];
    int64_t *d_stats = nullptr;
    int64_t *h_stats = nullptr;
    int32_t stats_cap = 0;
    cudaGraphExec_t exec = nullptr;
    int32_t graph_rounds = 0;
    int64_t graph_launches = 0;
    int64_t launches = 0;
};

namespace {

void free_groups(hgp_batch *b)
{
    for (auto &gr : b->g) {
        dev_free(gr.d_devs, b->stream);
        dev_free(gr.d_items, b->stream);
        dev_free(gr.d_wq, b->stream);
        gr.d_devs = nullptr;
        gr.d_items = nullptr;
        gr.d_wq = nullptr;
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_rounds = 0;
}

// (re)builds the per-group device arrays for a stats capacity of `cap` rounds
int build_groups(hgp_batch *b, int32_t cap)
{
    free_groups(b);
    const int32_t count = (int32_t)b->hs.size();
    dev_free(b->d_stats, b->stream);
    free(b->h_stats);
    b->d_stats = nullptr;
    b->h_stats = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&b->d_stats), sizeof(int64_t) * ST_N * (size_t)cap * count,
                              b->stream);
    if (e == cudaSuccess) {
        b->h_stats = static_cast<int64_t *>(malloc(sizeof(int64_t) * ST_N * (size_t)cap * count));
        if (!b->h_stats) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    b->stats_cap = cap;
    for (int gi = 0; gi < 2; ++gi) {
        auto &gr = b->g[gi];
        gr.members.clear();
        for (int32_t i = 0; i < count; ++i)
            if ((b->hs[i]->d.k > 32) == (gi == 1)) gr.members.push_back(i);
        gr.plan = Plan();
        if (gr.members.empty()) continue;
        std::vector<Dev> devs;
        std::vector<int2> ranges, tiles, blocks;
        int32_t S_max = 0;
        bool levels = false;
        for (size_t j = 0; j < gr.members.size(); ++j) {
            const hgp_handle *h = b->hs[gr.members[j]];
            Dev d = h->d;
            d.stats = b->d_stats + (int64_t)gr.members[j] * cap * ST_N;
            devs.push_back(d);
            for (int32_t r = 0; r < d.n_ranges; ++r) ranges.push_back(make_int2((int)j, r));
            for (int32_t t = 0; t < d.n_tiles; ++t) tiles.push_back(make_int2((int)j, t));
            for (int32_t t = 0; t < d.k; ++t) blocks.push_back(make_int2((int)j, t));
            S_max = d.S > S_max ? d.S : S_max;
            levels = levels || h->max_vertex_netweight >= kBins - 1;
        }
        const size_t n_items = ranges.size() + tiles.size() + blocks.size();
        e = dev_alloc(reinterpret_cast<void **>(&gr.d_devs), sizeof(Dev) * devs.size(), b->stream);
        if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&gr.d_items), sizeof(int2) * n_items, b->stream);
        if (e == cudaSuccess)
            e = dev_alloc(reinterpret_cast<void **>(&gr.d_wq), sizeof(int32_t) * kWqPerRow * (size_t)cap, b->stream);
        std::vector<int2> all;
        all.reserve(n_items);
        all.insert(all.end(), ranges.begin(), ranges.end());
        all.insert(all.end(), tiles.begin(), tiles.end());
        all.insert(all.end(), blocks.begin(), blocks.end());
        // pageable sources: each call returns once its source has been staged
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(gr.d_devs, devs.data(), sizeof(Dev) * devs.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(gr.d_items, all.data(), sizeof(int2) * n_items, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return status_of(e);
        }
        Plan &p = gr.plan;
        p.d0.wq = gr.d_wq;   // the batch kernels read only the work counters from d0
        p.devs = gr.d_devs;
        p.ranges = gr.d_items;
        p.tiles = gr.d_items + ranges.size();
        p.blocks = gr.d_items + ranges.size() + tiles.size();
        p.n_ranges = (int32_t)ranges.size();
        p.n_tiles = (int32_t)tiles.size();
        p.n_blocks = (int32_t)blocks.size();
        p.n_inst = (int32_t)devs.size();
        p.S_max = S_max;
        p.levels = levels;
        p.rec32 = gi == 1;
        set_grids(p, b->device);
        p.grid_gain = grid_override(b->device, b->gain_ctas, p.grid_gain, p.n_ranges);
        p.grid_apply = grid_override(b->device, b->apply_ctas, p.grid_apply, p.n_ranges);
        p.st = b->stream;
        p.launches = &b->launches;
    }
    return HGP_OK;
}

cudaError_t enqueue_batch(hgp_batch *b, int32_t rounds, int64_t *launch_counter)
{
    const int32_t count = (int32_t)b->hs.size();
    cudaError_t e = cudaMemsetAsync(b->d_stats, 0, sizeof(int64_t) * ST_N * (size_t)b->stats_cap * count, b->stream);
    for (int32_t rr = 0; rr < rounds && e == cudaSuccess; ++rr)
        for (auto &gr : b->g) {
            if (gr.members.empty() || e != cudaSuccess) continue;
            Plan p = gr.plan;
            p.launches = launch_counter;
            if (rr == 0) e = cudaMemsetAsync(p.d0.wq, 0, sizeof(int32_t) * kWqPerRow * (size_t)rounds, b->stream);
            if (e == cudaSuccess) e = launch_round(p, rr);
        }
    return e;
}

}  // namespace

// waits for the batch's stream and unpacks the per-member statistics of its last call
static int batch_stats_unpack(hgp_batch *b, int32_t rounds, hgp_round_stats *stats)
{
    const int32_t count = (int32_t)b->hs.size();
    for (int32_t i = 0; i < count; ++i)
        for (int32_t rr = 0; rr < rounds; ++rr) {
            const int64_t *row = b->h_stats + ((int64_t)i * b->stats_cap + rr) * ST_N;
            hgp_round_stats &o = stats[(int64_t)i * rounds + rr];
            o.objective = row[ST_OBJ];
            o.candidates = row[ST_CAND];
            o.approved = row[ST_APPR];
            o.eligible = row[ST_ELIG];
            o.max_block_weight = row[ST_MAXW];
            o.moved_pins = row[ST_MOVED];
            o.reverted = row[ST_REV];
        }
    return HGP_OK;
}

static int batch_stats_out(hgp_batch *b, int32_t rounds, hgp_round_stats *stats)
{
    const int32_t count = (int32_t)b->hs.size();
    cudaError_t e = cudaMemcpyAsync(b->h_stats, b->d_stats, sizeof(int64_t) * ST_N * (size_t)b->stats_cap * count,
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = stream_wait(b->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    return batch_stats_unpack(b, rounds, stats);
}

extern "C" {

void hgp_batch_default_options(hgp_batch_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->graph = 1;
}

int hgp_batch_create(hgp_handle *const *handles, int32_t count, const hgp_batch_options *opt, hgp_batch **out)
{
    if (!out) return HGP_ERR_INVALID;
    *out = nullptr;
    if (!handles || count < 1) return HGP_ERR_INVALID;
    hgp_batch_options o;
    hgp_batch_default_options(&o);
    if (opt) o = *opt;
    int dev = 0;
    cudaGetDevice(&dev);
    for (int32_t i = 0; i < count; ++i) {
        if (!handles[i] || handles[i]->device != dev) return HGP_ERR_INVALID;
        if (handles[i]->d.rv_src) return HGP_ERR_UNSUPPORTED;   // revert variant: single instances only
        for (int32_t j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return HGP_ERR_INVALID;
    }
    hgp_batch *b = new (std::nothrow) hgp_batch();
    if (!b) return HGP_ERR_OOM;
    b->device = dev;
    b->use_graph = o.graph;
    b->gain_ctas = o.gain_ctas_per_sm;
    b->apply_ctas = o.apply_ctas_per_sm;
    b->hs.assign(handles, handles + count);
    if (o.cuda_stream) {
        b->stream = (cudaStream_t)o.cuda_stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        delete b;
        return HGP_ERR_CUDA;
    } else {
        b->own_stream = true;
    }
    for (hgp_handle *h : b->hs) {
        if (h->stream == b->stream) continue;
        bool seen = false;
        for (cudaStream_t s2 : b->member_streams) seen = seen || s2 == h->stream;
        if (!seen) b->member_streams.push_back(h->stream);
    }
    for (size_t i = 0; i < b->member_streams.size(); ++i) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            hgp_batch_destroy(b);
            return HGP_ERR_CUDA;
        }
        b->events.push_back(ev);
    }
    for (hgp_handle *h : b->hs)
        if (h->stream != b->stream && !h->ev_batch &&
            cudaEventCreateWithFlags(&h->ev_batch, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            h->ev_batch = nullptr;
            hgp_batch_destroy(b);
            return HGP_ERR_CUDA;
        }
    if (cudaEventCreateWithFlags(&b->ev_end, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        b->ev_end = nullptr;
        hgp_batch_destroy(b);
        return HGP_ERR_CUDA;
    }
    const int rc = build_groups(b, 8);
    if (rc != HGP_OK) {
        hgp_batch_destroy(b);
        return rc;
    }
    *out = b;
    return HGP_OK;
}

int hgp_batch_refine(hgp_batch *b, int32_t rounds, hgp_round_stats *stats)
{
    if (!b || rounds < 0) return HGP_ERR_INVALID;
    if (rounds == 0) return HGP_OK;
    for (hgp_handle *h : b->hs)
        if (h->next_round + rounds >= ((int64_t)1 << 30)) return HGP_ERR_UNSUPPORTED;
    // the batch reads the handles' state on its own stream: after their streams' pending work,
    // and after the last call of another batch that refined them (on another stream)
    for (size_t i = 0; i < b->member_streams.size(); ++i) {
        cudaError_t e = cudaEventRecord(b->events[i], b->member_streams[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->events[i], 0);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return status_of(e);
        }
    }
    for (hgp_handle *h : b->hs) {
        if (!h->after_batch) continue;
        const cudaError_t e = cudaStreamWaitEvent(b->stream, h->ev_batch, 0);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return status_of(e);
        }
    }
    if (rounds > b->stats_cap) {
        int32_t cap = b->stats_cap;
        while (cap < rounds) cap *= 2;
        const int rc = build_groups(b, cap);
        if (rc != HGP_OK) return rc;
    }
    cudaError_t e = cudaSuccess;
    if (b->use_graph) {
        if (!b->exec || b->graph_rounds != rounds) {
            if (b->exec) {
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
            int64_t scratch = 0;
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e2 = enqueue_batch(b, rounds, &scratch);
                e = cudaStreamEndCapture(b->stream, &graph);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e == cudaSuccess) {
                b->graph_rounds = rounds;
                b->graph_launches = scratch;
            }
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
        if (e == cudaSuccess) b->launches += b->graph_launches;
    } else {
        e = enqueue_batch(b, rounds, &b->launches);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    for (hgp_handle *h : b->hs) {
        h->next_round += rounds;
        h->all_eligible = false;
    }
    b->last_rounds = rounds;
    e = cudaEventRecord(b->ev_end, b->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    // later work on the members' own streams (read-backs, releases) must come after this call:
    // the call's end is recorded on each such member's event, which its next entry point waits on
    for (hgp_handle *h : b->hs) {
        if (h->stream == b->stream) continue;
        e = cudaEventRecord(h->ev_batch, b->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return status_of(e);
        }
        h->after_batch = true;
    }
    if (stats) return batch_stats_out(b, rounds, stats);
    return HGP_OK;
}

int hgp_batch_get_stats(hgp_batch *b, int32_t rounds, hgp_round_stats *stats)
{
    if (!b || !stats || rounds < 1 || rounds != b->last_rounds) return HGP_ERR_INVALID;
    // waits for the last call only, not for work queued on the batch's stream after it (the
    // next tick of a pipelined caller): the copy runs on a private stream after ev_end
    cudaError_t e = cudaSuccess;
    if (!b->aux) {
        e = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking);
        if (e != cudaSuccess) b->aux = nullptr;
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->aux, b->ev_end, 0);
    if (e == cudaSuccess) {
        const int32_t count = (int32_t)b->hs.size();
        e = cudaMemcpyAsync(b->h_stats, b->d_stats, sizeof(int64_t) * ST_N * (size_t)b->stats_cap * count,
                            cudaMemcpyDeviceToHost, b->aux);
    }
    if (e == cudaSuccess) e = stream_wait(b->aux);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    return batch_stats_unpack(b, rounds, stats);
}

static std::mutex g_stage_mu;       // page-locked staging of hgp_batch_get_partitions
static void *g_stage = nullptr;
static size_t g_stage_cap = 0;

int hgp_batch_get_partitions(hgp_batch *b, const int32_t *members, int32_t count, int32_t *out)
{
    if (!b || count < 0 || (count > 0 && (!members || !out))) return HGP_ERR_INVALID;
    int64_t total = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (members[i] < 0 || members[i] >= (int32_t)b->hs.size()) return HGP_ERR_INVALID;
        total += b->hs[members[i]]->d.n;
    }
    if (total == 0) return HGP_OK;
    // after the batch's last call only (work queued on its stream later is not waited for)
    cudaError_t e = cudaSuccess;
    if (!b->aux) {
        e = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking);
        if (e != cudaSuccess) b->aux = nullptr;
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->aux, b->ev_end, 0);
    int32_t *stage = nullptr;
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&stage), sizeof(int32_t) * (size_t)total, b->aux);
    int64_t off = 0;
    for (int32_t i = 0; i < count && e == cudaSuccess; ++i) {
        const Dev &d = b->hs[members[i]]->d;
        const int grid = (int)std::min<int64_t>((d.n + 255) / 256, 152 * 8);
        k_part_widen<<<grid, 256, 0, b->aux>>>(d.part, d.n, stage + off);
        e = cudaGetLastError();
        off += d.n;
        b->launches++;
    }
    // through a page-locked staging buffer of the library (grown when needed), so the copy runs
    // at the link's rate whatever memory `out` is
    const size_t bytes = sizeof(int32_t) * (size_t)total;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (e == cudaSuccess && g_stage_cap < bytes) {
        if (g_stage) cudaFreeHost(g_stage);
        g_stage = nullptr;
        g_stage_cap = 0;
        const size_t cap = std::max(bytes, (size_t)16 << 20);
        e = cudaMallocHost(&g_stage, cap);
        if (e == cudaSuccess) g_stage_cap = cap;
        else g_stage = nullptr;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_stage, stage, bytes, cudaMemcpyDeviceToHost, b->aux);
    if (stage) dev_free(stage, b->aux);
    if (e == cudaSuccess) e = stream_wait(b->aux);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    memcpy(out, g_stage, bytes);
    return HGP_OK;
}

int hgp_batch_query(hgp_batch *b, int32_t *done)
{
    if (!b || !done) return HGP_ERR_INVALID;
    const cudaError_t e = cudaEventQuery(b->ev_end);
    if (e == cudaErrorNotReady) {
        (void)cudaGetLastError();
        *done = 0;
        return HGP_OK;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    *done = 1;
    return HGP_OK;
}

int hgp_batch_synchronize(hgp_batch *b)
{
    if (!b) return HGP_ERR_INVALID;
    const cudaError_t e = stream_wait(b->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    return HGP_OK;
}

int hgp_batch_get_launch_count(hgp_batch *b, int64_t *out)
{
    if (!b || !out) return HGP_ERR_INVALID;
    *out = b->launches;
    return HGP_OK;
}

void hgp_batch_destroy(hgp_batch *b)
{
    if (!b) return;
    free_groups(b);   // touches no member handle: members may already be destroyed
    dev_free(b->d_stats, b->stream);
    free(b->h_stats);
    for (cudaEvent_t ev : b->events) cudaEventDestroy(ev);
    if (b->ev_end) cudaEventDestroy(b->ev_end);
    if (b->aux) cudaStreamDestroy(b->aux);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    (void)cudaGetLastError();
    delete b;
}

int hgp_set_profiling(hgp_handle *h, int32_t enable)
{
    if (!h) return HGP_ERR_INVALID;
    h->profiling = enable != 0;
    h->events_used = 0;
    for (int i = 0; i < HGP_PHASES; ++i) {
        h->prof_ms[i] = 0.0;
        h->prof_launches[i] = 0;
    }
    return HGP_OK;
}

int hgp_get_profile(hgp_handle *h, hgp_profile *out)
{
    if (!h || !out) return HGP_ERR_INVALID;
    for (int i = 0; i < HGP_PHASES; ++i) {
        out->ms[i] = h->prof_ms[i];
        out->launches[i] = h->prof_launches[i];
    }
    return HGP_OK;
}

int hgp_get_launch_count(hgp_handle *h, int64_t *out)
{
    if (!h || !out) return HGP_ERR_INVALID;
    *out = h->launches;
    return HGP_OK;
}

}  // extern "C"

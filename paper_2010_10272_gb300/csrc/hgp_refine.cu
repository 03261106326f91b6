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
//   k_round_end    per-round objective and heaviest block.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <new>

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

// ------------------------------------------------------------------ round preparation
__global__ void __launch_bounds__(kThreads) k_round_prep(Dev d, int32_t r, uint64_t seed)
{
    __shared__ uint8_t subs[kWarps][kRange];
    __shared__ int32_t cnt[kWarps][65];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t range = blockIdx.x * kWarps + wid;
    if (range >= d.n_ranges) return;
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
                                               Lam T, int &t_out, int32_t &conn_out)
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
}

template <typename Lam, typename Rec, bool UNIT>
__device__ __forceinline__ void best_by_planes(int np, const GainWarp<Lam> &g, const Rec *recs,
                                               const int32_t *inc, int32_t ib, int32_t ie, int32_t jb,
                                               int32_t off, Lam T, int &t, int32_t &conn)
{
    if (np <= 4) bitsliced_best<Lam, Rec, 4, UNIT>(g, recs, inc, ib, ie, jb, off, T, t, conn);
    else if (np <= 6) bitsliced_best<Lam, Rec, 6, UNIT>(g, recs, inc, ib, ie, jb, off, T, t, conn);
    else if (np <= 8) bitsliced_best<Lam, Rec, 8, UNIT>(g, recs, inc, ib, ie, jb, off, T, t, conn);
    else bitsliced_best<Lam, Rec, 11, UNIT>(g, recs, inc, ib, ie, jb, off, T, t, conn);
}

constexpr int32_t kPlaneMaxW = 2047;   // W(u) up to this uses bit planes (NP <= 11)

// Persistent: each warp walks warp ranges with a grid stride and takes the vertices of
// sub-round s of a range 32 at a time (one slot per lane).
//   pass A  flattened over the chunk's incidences (every record gather issued at once): W,
//           b(u) (Sec. 5), eligibility (Sec. 6) and T = union of Lambda(e) over the nets with
//           Phi(e,a) = 1, minus a and the blocks without room for c(u); (Lambda, omega) of each
//           incidence is kept in shared memory.  Only blocks in T can have a positive gain,
//           since g_t <= omega({e : Phi(e,a) = 1, t in Lambda(e)}).
//   pass B  per vertex, conn_t = omega({e in I(u) : t in Lambda(e)}) for all t in T at once in
//           bit planes, and the arg-max of g_t = b(u) - W + conn_t.
// A vertex whose incident net weights exceed kPlaneMaxW uses a warp-cooperative pass instead.
template <typename Rec>
__global__ void __launch_bounds__(kThreads, 4) k_gain(Dev d, int32_t r, int32_t s, int32_t all_elig,
                                                      unsigned long long *st_row)
{
    typedef typename RecIO<Rec>::Lam Lam;
    constexpr bool kWide = sizeof(Lam) == 8;
    __shared__ GainWarp<Lam> ws[kWarps];
    __shared__ long long slack[64];
    __shared__ unsigned long long tot_s[64];
    __shared__ unsigned long long cnt_s[2];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid < 64) {
        tot_s[tid] = 0;
        slack[tid] = tid < d.k ? d.lmax - d.bw[tid] : -1;
    }
    if (tid < 2) cnt_s[tid] = 0;
    __syncthreads();
    Lam feas1;
    {
        const unsigned lo = __ballot_sync(kFull, slack[lane] >= 1);
        const unsigned hi = __ballot_sync(kFull, slack[lane + 32] >= 1);
        if (kWide) feas1 = (Lam)((uint64_t)lo | ((uint64_t)hi << 32));
        else feas1 = (Lam)lo;
    }
    GainWarp<Lam> &g = ws[wid];
    const Rec *recs = reinterpret_cast<const Rec *>(d.rec);
    const bool unit = d.nw == nullptr;
    int32_t nelig = 0, ncand = 0;
    for (int32_t range = blockIdx.x * kWarps + wid; range < d.n_ranges; range += gridDim.x * kWarps) {
        const int32_t rbase = range * kRange;
        const uint16_t *ss = d.sub_start + (int64_t)range * (d.S + 1);
        const int32_t beg = ss[s], cnt = (int32_t)ss[s + 1] - beg;
        const uint8_t *list = d.sub_list + (int64_t)range * kRange + beg;
        uint64_t *out = d.cand + (int64_t)range * kRange;
        int32_t nout = 0;
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
            }
            g.a[lane] = a;
            g.jb[lane] = jb;
            g.W[lane] = 0;
            g.b[lane] = 0;
            g.T[lane] = 0;
            g.elig[lane] = all_elig;
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
                    }
                    if (moved_in_prev_round(mv1, r)) g.elig[v1] = 1;
                }
                if (i2 < total) {
                    w2 &= 0x7fffffff;
                    if (i2 < kCache) { g.lamc[i2] = lam2; g.wc[i2] = w2; }
                    atomicAdd(&g.W[v2], w2);
                    if ((s12 >> g.a[v2]) & 1) {
                        atomicAdd(&g.b[v2], w2);
                        atomicOr(&g.T[v2], (unsigned long long)lam2);
                    }
                    if (moved_in_prev_round(mv2, r)) g.elig[v2] = 1;
                }
            }
            __syncwarp();
            // ---- per vertex: eligibility, candidate blocks, best block
            const int32_t W = g.W[lane], b = g.b[lane];
            const bool elig = valid && g.elig[lane] != 0;
            Lam T = elig ? (Lam)g.T[lane] : (Lam)0;
            T &= ~((Lam)1 << a);
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
            if (plane_path) {
                const int np = 32 - __clz((int)wmax);   // 2^np > wmax >= conn_t
                int t;
                int32_t conn;
                if (unit) best_by_planes<Lam, Rec, true>(np, g, recs, d.inc, my_off, my_off + deg, jb, my_off, T, t, conn);
                else best_by_planes<Lam, Rec, false>(np, g, recs, d.inc, my_off, my_off + deg, jb, my_off, T, t, conn);
                const int32_t gg = bw_ + conn;
                if (gg > 0) {
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
                // smaller block
                unsigned long long key = 0;
                if ((Tlo >> lane) & 1) {
                    const int32_t gg = hbw + acc0;
                    if (gg > 0) key = ((unsigned long long)(uint32_t)gg << 8) | (unsigned long long)(255 - lane);
                }
                if (kWide && ((Thi >> lane) & 1)) {
                    const int32_t gg = hbw + acc1;
                    if (gg > 0) {
                        const unsigned long long k2 = ((unsigned long long)(uint32_t)gg << 8) | (unsigned long long)(255 - (lane + 32));
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
                    g_best = (int32_t)(key >> 8);
                }
            }
            nelig += __popc(__ballot_sync(kFull, elig));
            const unsigned cm = __ballot_sync(kFull, t_best >= 0);
            if (t_best >= 0) {
                const int pos = nout + __popc(cm & lanemask_lt());
                out[pos] = ((uint64_t)(uint32_t)g_best << 32) | ((uint32_t)ul << 8) | (uint32_t)t_best;
                atomicAdd(&tot_s[t_best], (unsigned long long)cu);
            }
            nout += __popc(cm);
            __syncwarp();
        }
        if (lane == 0) d.cand_cnt[range] = nout;
        ncand += nout;
    }
    if (lane == 0) {
        if (nelig) atomicAdd(&cnt_s[0], (unsigned long long)nelig);
        if (ncand) atomicAdd(&cnt_s[1], (unsigned long long)ncand);
    }
    __syncthreads();
    if (tid < d.k && tot_s[tid]) atomicAdd(reinterpret_cast<unsigned long long *>(&d.tot[tid]), tot_s[tid]);
    if (tid == 0) {
        if (cnt_s[0]) atomicAdd(st_row + ST_ELIG, cnt_s[0]);
        if (cnt_s[1]) atomicAdd(st_row + ST_CAND, cnt_s[1]);
    }
}

// ------------------------------------------------------------------ approval
__device__ __forceinline__ void decode(uint64_t c, int &t, int32_t &g, int &ul)
{
    t = (int)(c & 0xFF);
    ul = (int)((c >> 8) & 0xFF);
    g = (int32_t)(c >> 32);
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

__global__ void __launch_bounds__(kThreads) k_hist(Dev d, int level)
{
    __shared__ int active[64];
    __shared__ long long prefix[64];
    __shared__ int any;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) any = 0;
    __syncthreads();
    if (tid < 64) {
        int a = 0;
        if (tid < d.k) {
            if (level == 0) {
                a = d.bw[tid] + d.tot[tid] > d.lmax;
            } else {
                const Sel sl = d.sel[tid];
                a = sl.mode == SEL_REFINE && sl.level == level;
                prefix[tid] = sl.g;
            }
        }
        active[tid] = a;
        if (a) any = 1;
    }
    __syncthreads();
    if (!any) return;
    const int32_t range = blockIdx.x * kWarps + wid;
    if (range >= d.n_ranges) return;
    const int32_t n = d.cand_cnt[range];
    const uint64_t *cand = d.cand + (int64_t)range * kRange;
    for (int i = lane; i < n; i += 32) {
        int t, ul;
        int32_t g;
        decode(cand[i], t, g, ul);
        if (!active[t]) continue;
        const unsigned long long c = d.vw ? (unsigned long long)d.vw[range * kRange + ul] : 1ull;
        int bin;
        if (level == 0) {
            bin = g < kBins - 1 ? g : kBins - 1;
        } else {
            if (g < kBins - 1) continue;
            bool match;
            bin = refine_digit(g - (kBins - 1), level, prefix[t], match);
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

// one CTA per block t: threshold of the (gain desc, id asc) prefix that fits
__global__ void __launch_bounds__(kThreads) k_select(Dev d, int level)
{
    __shared__ unsigned long long wt[32];
    __shared__ int found_bin;
    __shared__ long long found_before;
    const int t = blockIdx.x, tid = threadIdx.x;
    Sel sl = d.sel[t];
    long long cap;
    int nbins;
    if (level == 0) {
        const long long tot = d.tot[t];
        cap = d.lmax - d.bw[t];
        if (d.bw[t] + tot <= d.lmax) {
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
    if (tid == 0) found_bin = -1;
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

__global__ void __launch_bounds__(kThreads) k_tie_sum(Dev d)
{
    __shared__ int thr[64];
    __shared__ int32_t gthr[64];
    __shared__ unsigned long long ts[64];
    __shared__ int any;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
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
    const int32_t range = blockIdx.x * kWarps + wid;
    if (range < d.n_ranges) {
        const int32_t n = d.cand_cnt[range];
        const uint64_t *cand = d.cand + (int64_t)range * kRange;
        for (int i = lane; i < n; i += 32) {
            int t, ul;
            int32_t g;
            decode(cand[i], t, g, ul);
            if (thr[t] && g == gthr[t])
                atomicAdd(&ts[t], d.vw ? (unsigned long long)d.vw[range * kRange + ul] : 1ull);
        }
    }
    __syncthreads();
    if (tid < d.k && thr[tid]) d.tie[(int64_t)tid * d.n_tiles + blockIdx.x] = (int64_t)ts[tid];
}

__global__ void __launch_bounds__(1024) k_tie_scan(Dev d)
{
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long carry;
    const int t = blockIdx.x;
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

template <typename Rec>
__device__ __forceinline__ long long apply_pins(const Dev &d, Rec *recs, const ApplyWarp &w_,
                                                int32_t i0, int32_t total, int32_t r)
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
        mv[q] = __ldcg(&rc->mv);
        w[q] = __ldg(&rc->w) & 0x7fffffff;
        oa[q] = phi_add(d, ee, a[q], -1, wide, wrow);
        ot[q] = phi_add(d, ee, t[q], +1, wide, wrow);
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
        const int32_t last = mv[q] >> 1;
        if (last != r) rc->mv = (r << 1) | (last == r - 1 ? 1 : 0);
        dobj += (long long)(ot[q] == 0 ? w[q] : 0) - (long long)(oa[q] == 1 ? w[q] : 0);
    }
    return dobj;
}

// Persistent: each warp walks warp ranges with a grid stride.  For each 32 candidates of a
// range it decides approval (ties at a block's threshold gain in vertex-id order: the warp
// starts from the tile's exclusive tie prefix and adds the ties of the earlier ranges of the
// same tile itself, so warps never wait for each other), then applies the approved moves
// over their incidences flattened across the lanes, so all atomics are in flight at once.
template <typename Rec>
__global__ void __launch_bounds__(kThreads, 4) k_apply(Dev d, int32_t r, unsigned long long *st_row)
{
    __shared__ int mode[64];
    __shared__ int32_t gthr[64];
    __shared__ long long rem[64];
    __shared__ unsigned long long run[kWarps][64];
    __shared__ unsigned long long bwd[64];
    __shared__ ApplyWarp aw[kWarps];
    __shared__ unsigned long long objd, napp, mpins;
    __shared__ int any_thr;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) { objd = 0; napp = 0; mpins = 0; any_thr = 0; }
    __syncthreads();
    if (tid < 64) {
        int md = SEL_ALL;
        if (tid < d.k) {
            const Sel sl = d.sel[tid];
            md = sl.mode;
            gthr[tid] = (int32_t)sl.g;
            rem[tid] = sl.rem;
        }
        mode[tid] = md;
        bwd[tid] = 0;
        if (md == SEL_THRESH) any_thr = 1;
    }
    __syncthreads();
    Rec *recs = reinterpret_cast<Rec *>(d.rec);
    ApplyWarp &w_ = aw[wid];
    long long dobj = 0;
    int32_t nappr = 0, npins = 0;
    for (int32_t range = blockIdx.x * kWarps + wid; range < d.n_ranges; range += gridDim.x * kWarps) {
        const int32_t ncand = d.cand_cnt[range];
        if (ncand == 0) continue;
        const uint64_t *cand = d.cand + (int64_t)range * kRange;
        if (any_thr) {
            const int32_t tile = range / kWarps;
            for (int t = lane; t < 64; t += 32)
                run[wid][t] = (t < d.k && mode[t] == SEL_THRESH)
                                  ? (unsigned long long)d.tie[(int64_t)t * d.n_tiles + tile] : 0ull;
            __syncwarp();
            for (int32_t pr = tile * kWarps; pr < range; ++pr) {
                const int32_t n2 = d.cand_cnt[pr];
                const uint64_t *c2 = d.cand + (int64_t)pr * kRange;
                for (int i = lane; i < n2; i += 32) {
                    int t, ul;
                    int32_t g;
                    decode(c2[i], t, g, ul);
                    if (mode[t] == SEL_THRESH && g == gthr[t])
                        atomicAdd(&run[wid][t], d.vw ? (unsigned long long)d.vw[pr * kRange + ul] : 1ull);
                }
            }
            __syncwarp();
        }
        for (int32_t c0 = 0; c0 < ncand; c0 += 32) {
            const int idx = c0 + lane;
            int t = 0, ul = 0;
            int32_t g = 0;
            unsigned long long cw = 1;
            bool appr = false, tie = false;
            if (idx < ncand) {
                decode(cand[idx], t, g, ul);
                if (d.vw) cw = (unsigned long long)d.vw[range * kRange + ul];
                const int md = mode[t];
                if (md == SEL_ALL || g > gthr[t]) appr = true;
                else if (g == gthr[t]) tie = true;
            }
            // ties in id order: exclusive prefix so far + own weight must fit the budget
            unsigned tm = __ballot_sync(kFull, tie);
            while (tm) {
                const int l = __ffs(tm) - 1;
                tm &= tm - 1;
                if (lane == l) {
                    appr = (long long)(run[wid][t] + cw) <= rem[t];
                    run[wid][t] += cw;
                }
                __syncwarp();
            }
            int32_t deg = 0, jb = 0, a = 0;
            if (appr) {
                const int32_t u = range * kRange + ul;
                a = d.part[u];
                d.part[u] = (uint8_t)t;
                atomicAdd(&bwd[a], (unsigned long long)(-(long long)cw));
                atomicAdd(&bwd[t], cw);
                jb = d.vtx_off[u];
                deg = d.vtx_off[u + 1] - jb;
                ++nappr;
                npins += deg;
            }
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
                dobj += apply_pins<Rec>(d, recs, w_, i0 + lane, total, r);
            __syncwarp();
        }
    }
    for (int o = 16; o; o >>= 1) {
        dobj += __shfl_xor_sync(kFull, dobj, o);
        nappr += __shfl_xor_sync(kFull, nappr, o);
        npins += __shfl_xor_sync(kFull, npins, o);
    }
    if (lane == 0) {
        if (dobj) atomicAdd(&objd, (unsigned long long)dobj);
        if (nappr) atomicAdd(&napp, (unsigned long long)nappr);
        if (npins) atomicAdd(&mpins, (unsigned long long)npins);
    }
    __syncthreads();
    if (tid < d.k && bwd[tid]) atomicAdd(reinterpret_cast<unsigned long long *>(&d.bw[tid]), bwd[tid]);
    if (tid == 0) {
        if (objd) atomicAdd(reinterpret_cast<unsigned long long *>(d.obj), objd);
        if (napp) atomicAdd(st_row + ST_APPR, napp);
        if (mpins) atomicAdd(st_row + ST_MOVED, mpins);
    }
}

__global__ void k_round_end(Dev d, unsigned long long *st_row)
{
    if (threadIdx.x == 0) {
        long long mx = 0;
        for (int i = 0; i < d.k; ++i) mx = d.bw[i] > mx ? d.bw[i] : mx;
        st_row[ST_OBJ] = (unsigned long long)*d.obj;
        st_row[ST_MAXW] = (unsigned long long)mx;
    }
}

__global__ void k_expand_candidates(Dev d, int32_t *target, int64_t *gain)
{
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

// ------------------------------------------------------------------ host side
// Persistent grid: as many CTAs as fit on the device at once, never more than the work.
template <typename K>
int persistent_grid(hgp_handle *h, K kernel)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
    (void)cudaGetLastError();
    int64_t g = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (h->d.n_ranges + kWarps - 1) / kWarps;
    if (g > need) g = need;
    return (int)(g < 1 ? 1 : g);
}

template <typename Rec>
cudaError_t launch_gain(hgp_handle *h, int32_t r, int32_t s, bool all_elig, unsigned long long *st_row)
{
    if (!h->grid_gain) h->grid_gain = persistent_grid(h, k_gain<Rec>);
    k_gain<Rec><<<h->grid_gain, kThreads, 0, h->stream>>>(h->d, r, s, all_elig ? 1 : 0, st_row);
    h->launches++;
    return cudaGetLastError();
}

template <typename Rec>
cudaError_t launch_apply(hgp_handle *h, int32_t r, unsigned long long *st_row)
{
    if (!h->grid_apply) h->grid_apply = persistent_grid(h, k_apply<Rec>);
    k_apply<Rec><<<h->grid_apply, kThreads, 0, h->stream>>>(h->d, r, st_row);
    h->launches++;
    return cudaGetLastError();
}

// Per-phase event timing (profiling mode): a pair of events around each phase instance.
enum { PH_PREP = 0, PH_GAIN = 1, PH_APPROVE = 2, PH_APPLY = 3, PH_END = 4 };

cudaError_t phase_begin(hgp_handle *h)
{
    if (!h->profiling) return cudaSuccess;
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
    if (!h->profiling) return cudaSuccess;
    cudaError_t e = cudaEventRecord(h->events[h->events_used + 1], h->stream);
    h->event_phase[h->events_used / 2] = phase;
    h->event_count[h->events_used / 2] = launches;
    h->events_used += 2;
    return e;
}

cudaError_t collect_profile(hgp_handle *h)
{
    if (!h->profiling || h->events_used == 0) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    for (int32_t i = 0; i + 1 < h->events_used && e == cudaSuccess; i += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->events[i], h->events[i + 1]);
        h->prof_ms[h->event_phase[i / 2]] += ms;
        h->prof_launches[h->event_phase[i / 2]] += h->event_count[i / 2];
    }
    h->events_used = 0;
    return e;
}

cudaError_t launch_subround(hgp_handle *h, int32_t r, int32_t s, bool all_elig, unsigned long long *st_row)
{
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    cudaError_t e = phase_begin(h);
    if (e == cudaSuccess)
        e = d.k <= 32 ? launch_gain<Rec16>(h, r, s, all_elig, st_row) : launch_gain<Rec32>(h, r, s, all_elig, st_row);
    if (e == cudaSuccess) e = phase_end(h, PH_GAIN, 1);
    if (e != cudaSuccess) return e;
    e = phase_begin(h);
    if (e != cudaSuccess) return e;
    int32_t n = 0;
    k_hist<<<d.n_tiles, kThreads, 0, st>>>(d, 0);
    k_select<<<d.k, kThreads, 0, st>>>(d, 0);
    n += 2;
    if (h->max_vertex_netweight >= kBins - 1) {
        for (int level = 1; level <= 3; ++level) {
            k_hist<<<d.n_tiles, kThreads, 0, st>>>(d, level);
            k_select<<<d.k, kThreads, 0, st>>>(d, level);
            n += 2;
        }
    }
    k_tie_sum<<<d.n_tiles, kThreads, 0, st>>>(d);
    k_tie_scan<<<d.k, 1024, 0, st>>>(d);
    n += 2;
    h->launches += n;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = phase_end(h, PH_APPROVE, n);
    if (e == cudaSuccess) e = phase_begin(h);
    if (e != cudaSuccess) return e;
    e = d.k <= 32 ? launch_apply<Rec16>(h, r, st_row) : launch_apply<Rec32>(h, r, st_row);
    if (e == cudaSuccess) e = phase_end(h, PH_APPLY, 1);
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
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&dev), sizeof(int64_t) * ST_N * (size_t)cap);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&host), sizeof(int64_t) * ST_N * (size_t)cap);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (dev) cudaFree(dev);
        return status_of(e);
    }
    if (h->d.stats || h->h_stats) cudaStreamSynchronize(h->stream);
    if (h->d.stats) cudaFree(h->d.stats);
    if (h->h_stats) cudaFreeHost(h->h_stats);
    h->d.stats = dev;
    h->h_stats = host;
    h->stats_cap = cap;
    return HGP_OK;
}

int refine_rounds(hgp_handle *h, int32_t rounds, hgp_round_stats *stats)
{
    if (rounds == 0) return HGP_OK;
    if (h->next_round + rounds >= ((int64_t)1 << 30)) return HGP_ERR_UNSUPPORTED;
    int rc = ensure_stats(h, rounds);
    if (rc != HGP_OK) return rc;
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    cudaError_t e = cudaMemsetAsync(d.stats, 0, sizeof(int64_t) * ST_N * (size_t)rounds, st);
    for (int32_t rr = 0; rr < rounds && e == cudaSuccess; ++rr) {
        const int32_t r = (int32_t)(h->next_round + rr);
        unsigned long long *row = reinterpret_cast<unsigned long long *>(d.stats + (int64_t)rr * ST_N);
        e = phase_begin(h);
        if (e != cudaSuccess) break;
        k_round_prep<<<d.n_tiles, kThreads, 0, st>>>(d, r, h->seed);
        h->launches++;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = phase_end(h, PH_PREP, 1);
        for (int32_t s = 0; s < d.S && e == cudaSuccess; ++s)
            e = launch_subround(h, r, s, h->all_eligible && rr == 0, row);
        if (e == cudaSuccess) e = phase_begin(h);
        if (e == cudaSuccess) {
            k_round_end<<<1, 32, 0, st>>>(d, row);
            h->launches++;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = phase_end(h, PH_END, 1);
    }
    if (e == cudaSuccess) e = collect_profile(h);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    h->next_round += rounds;
    h->all_eligible = false;
    if (stats || (h->debug & 1)) {
        e = cudaMemcpyAsync(h->h_stats, d.stats, sizeof(int64_t) * ST_N * (size_t)rounds, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
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
            }
        }
    }
    if (h->debug & 1) {
        int64_t *tmp = nullptr;
        int64_t from_phi = 0, maintained = 0;
        e = cudaMallocAsync(reinterpret_cast<void **>(&tmp), sizeof(int64_t), st);
        if (e == cudaSuccess) e = objective_from_phi(h, tmp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&from_phi, tmp, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&maintained, d.obj, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (tmp) cudaFreeAsync(tmp, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
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
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    const int32_t r = (int32_t)h->next_round;
    int32_t *t_d = nullptr;
    int64_t *g_d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&t_d), sizeof(int32_t) * (size_t)d.n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&g_d), sizeof(int64_t) * (size_t)d.n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(t_d, 0xFF, sizeof(int32_t) * (size_t)d.n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_d, 0, sizeof(int64_t) * (size_t)d.n, st);
    if (e == cudaSuccess) {
        k_round_prep<<<d.n_tiles, kThreads, 0, st>>>(d, r, h->seed);
        h->launches++;
        e = cudaGetLastError();
    }
    // the stats row written here is scratch: refine() clears the stats before use
    unsigned long long *row = reinterpret_cast<unsigned long long *>(d.stats);
    if (e == cudaSuccess)
        e = d.k <= 32 ? launch_gain<Rec16>(h, r, s, h->all_eligible, row) : launch_gain<Rec32>(h, r, s, h->all_eligible, row);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.tot, 0, sizeof(int64_t) * 64, st);
    if (e == cudaSuccess) {
        k_expand_candidates<<<(d.n_ranges * 32 + 255) / 256, 256, 0, st>>>(d, t_d, g_d);
        h->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(target, t_d, sizeof(int32_t) * (size_t)d.n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gain, g_d, sizeof(int64_t) * (size_t)d.n, cudaMemcpyDeviceToHost, st);
    if (t_d) cudaFreeAsync(t_d, st);
    if (g_d) cudaFreeAsync(g_d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    return HGP_OK;
}

}  // namespace hgp

extern "C" {

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

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
#include <stdint.h>
#include <string.h>

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

template <typename Rec>
__global__ void __launch_bounds__(kThreads) k_gain(Dev d, int32_t r, int32_t s, int32_t all_elig,
                                                   unsigned long long *st_row)
{
    typedef typename RecIO<Rec>::Lam Lam;
    extern __shared__ int32_t acc[];   // [k][kThreads]: per-thread connectivity accumulators
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
        if (sizeof(Lam) == 8) feas1 = (Lam)((uint64_t)lo | ((uint64_t)hi << 32));
        else feas1 = (Lam)lo;
    }
    const Rec *recs = reinterpret_cast<const Rec *>(d.rec);
    const int32_t range = blockIdx.x * kWarps + wid;
    if (range < d.n_ranges) {
        const int32_t base = range * kRange;
        const uint16_t *ss = d.sub_start + (int64_t)range * (d.S + 1);
        const int32_t beg = ss[s], cnt = (int32_t)ss[s + 1] - beg;
        const uint8_t *list = d.sub_list + (int64_t)range * kRange + beg;
        uint64_t *out = d.cand + (int64_t)range * kRange;
        int32_t nout = 0, nelig = 0;
        for (int32_t c0 = 0; c0 < cnt; c0 += 32) {
            const int32_t idx = c0 + lane;
            int32_t t_best = -1, g_best = 0, cu = 1, ul = 0;
            bool elig = false;
            if (idx < cnt) {
                ul = list[idx];
                const int32_t u = base + ul;
                const int a = d.part[u];
                cu = d.vw ? d.vw[u] : 1;
                const int32_t jb = d.vtx_off[u], je = d.vtx_off[u + 1];
                int32_t W = 0, b = 0;
                Lam T = 0;
                elig = all_elig != 0;
                // pass A: W, b(u), eligibility, candidate blocks
                for (int32_t j = jb; j < je; ++j) {
                    const int32_t e = __ldg(&d.inc[j]);
                    Lam s1, lam;
                    int32_t w, mv;
                    bool has_lam;
                    RecIO<Rec>::load_a(recs + e, s1, w, mv, lam, has_lam);
                    w &= 0x7fffffff;
                    W += w;
                    if ((s1 >> a) & 1) {
                        b += w;
                        T |= has_lam ? lam : RecIO<Rec>::load_lam(recs + e);
                    }
                    elig = elig || moved_in_prev_round(mv, r);
                }
                if (elig) {
                    T &= ~((Lam)1 << a);
                    if (d.vw) {
                        for (Lam x = T; x; x &= x - 1) {
                            const int t = lam_bits_ctz(x);
                            if (slack[t] < cu) T &= ~((Lam)1 << t);
                        }
                    } else {
                        T &= feas1;
                    }
                }
                if (elig && T) {
                    // pass B: conn_t = omega({e in I(u) : t in Lambda(e)}) for t in T; a net
                    // covering more than half of T is counted as base minus its complement
                    const int nT = lam_popc(T);
                    for (Lam x = T; x; x &= x - 1) acc[lam_bits_ctz(x) * kThreads + tid] = 0;
                    int32_t cbase = 0;
                    for (int32_t j = jb; j < je; ++j) {
                        const int32_t e = __ldg(&d.inc[j]);
                        Lam lam;
                        int32_t w;
                        RecIO<Rec>::load_b(recs + e, lam, w);
                        w &= 0x7fffffff;
                        const Lam in = lam & T;
                        if (2 * lam_popc(in) <= nT) {
                            for (Lam x = in; x; x &= x - 1) acc[lam_bits_ctz(x) * kThreads + tid] += w;
                        } else {
                            cbase += w;
                            for (Lam x = T & ~lam; x; x &= x - 1) acc[lam_bits_ctz(x) * kThreads + tid] -= w;
                        }
                    }
                    const int32_t bw_ = b - W;
                    for (Lam x = T; x; x &= x - 1) {
                        const int t = lam_bits_ctz(x);
                        const int32_t g = bw_ + (cbase + acc[t * kThreads + tid]);
                        if (g > g_best) {
                            g_best = g;
                            t_best = t;
                        }
                    }
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
        }
        if (lane == 0) {
            d.cand_cnt[range] = nout;
            atomicAdd(&cnt_s[0], (unsigned long long)nelig);
            atomicAdd(&cnt_s[1], (unsigned long long)nout);
        }
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
template <typename Rec>
__global__ void __launch_bounds__(kThreads) k_apply(Dev d, int32_t r, unsigned long long *st_row)
{
    typedef typename RecIO<Rec>::Lam Lam;
    __shared__ int mode[64];
    __shared__ int32_t gthr[64];
    __shared__ long long rem[64];
    __shared__ unsigned long long wtie[kWarps][64];
    __shared__ unsigned long long run[kWarps][64];
    __shared__ unsigned long long bwd[64];
    __shared__ unsigned long long objd, napp;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int tile = blockIdx.x;
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
    }
    for (int i = tid; i < kWarps * 64; i += kThreads) (&wtie[0][0])[i] = 0;
    if (tid == 0) { objd = 0; napp = 0; }
    __syncthreads();
    const int32_t range = tile * kWarps + wid;
    const int32_t ncand = range < d.n_ranges ? d.cand_cnt[range] : 0;
    const uint64_t *cand = d.cand + (int64_t)range * kRange;
    // pass 1: tie weight per block in this warp's range
    for (int i = lane; i < ncand; i += 32) {
        int t, ul;
        int32_t g;
        decode(cand[i], t, g, ul);
        if (mode[t] == SEL_THRESH && g == gthr[t])
            atomicAdd(&wtie[wid][t], d.vw ? (unsigned long long)d.vw[range * kRange + ul] : 1ull);
    }
    __syncthreads();
    for (int t = lane; t < d.k; t += 32) {
        unsigned long long s = 0;
        if (mode[t] == SEL_THRESH) {
            s = (unsigned long long)d.tie[(int64_t)t * d.n_tiles + tile];
            for (int w = 0; w < wid; ++w) s += wtie[w][t];
        }
        run[wid][t] = s;
    }
    __syncwarp();
    Rec *recs = reinterpret_cast<Rec *>(d.rec);
    long long dobj = 0;
    int32_t nappr = 0;
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
        if (appr) {
            const int32_t u = range * kRange + ul;
            const int a = d.part[u];
            d.part[u] = (uint8_t)t;
            atomicAdd(&bwd[a], (unsigned long long)(-(long long)cw));
            atomicAdd(&bwd[t], cw);
            const Lam ba = (Lam)1 << a, bt = (Lam)1 << t;
            const int32_t jb = d.vtx_off[u], je = d.vtx_off[u + 1];
            for (int32_t j = jb; j < je; ++j) {
                const int32_t e = d.inc[j];
                Rec *rc = recs + e;
                const int32_t wf = rc->w;
                const int32_t w = wf & 0x7fffffff;
                const bool wide = wf < 0;
                const int32_t wrow = wide ? d.widx[e] : 0;
                const int32_t oa = phi_add(d, e, a, -1, wide, wrow);
                const int32_t ot = phi_add(d, e, t, +1, wide, wrow);
                const Lam lx = (oa == 1 ? ba : (Lam)0) | (ot == 0 ? bt : (Lam)0);
                const Lam sx = ((oa == 1 || oa == 2) ? ba : (Lam)0) | ((ot == 0 || ot == 1) ? bt : (Lam)0);
                if (sizeof(Lam) == 8) {
                    if (lx) atomicXor(reinterpret_cast<unsigned long long *>(&rc->lam), (unsigned long long)lx);
                    if (sx) atomicXor(reinterpret_cast<unsigned long long *>(&rc->s1), (unsigned long long)sx);
                } else {
                    if (lx) atomicXor(reinterpret_cast<unsigned int *>(&rc->lam), (unsigned int)lx);
                    if (sx) atomicXor(reinterpret_cast<unsigned int *>(&rc->s1), (unsigned int)sx);
                }
                dobj += (ot == 0 ? w : 0) - (oa == 1 ? w : 0);
                stamp_moved(&rc->mv, r);
            }
            ++nappr;
        }
    }
    for (int o = 16; o; o >>= 1) {
        dobj += __shfl_xor_sync(kFull, dobj, o);
        nappr += __shfl_xor_sync(kFull, nappr, o);
    }
    if (lane == 0) {
        if (dobj) atomicAdd(&objd, (unsigned long long)dobj);
        if (nappr) atomicAdd(&napp, (unsigned long long)nappr);
    }
    __syncthreads();
    if (tid < d.k && bwd[tid]) atomicAdd(reinterpret_cast<unsigned long long *>(&d.bw[tid]), bwd[tid]);
    if (tid == 0) {
        if (objd) atomicAdd(reinterpret_cast<unsigned long long *>(d.obj), objd);
        if (napp) atomicAdd(st_row + ST_APPR, napp);
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
template <typename Rec>
cudaError_t set_gain_smem(int k)
{
    static int done[2] = {0, 0};
    const int slot = sizeof(Rec) == 16 ? 0 : 1;
    (void)k;
    if (done[slot]) return cudaSuccess;
    const int bytes = (sizeof(Rec) == 16 ? 32 : 64) * kThreads * (int)sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(k_gain<Rec>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[slot] = 1;
    return e;
}

template <typename Rec>
cudaError_t launch_gain(hgp_handle *h, int32_t r, int32_t s, bool all_elig, unsigned long long *st_row)
{
    cudaError_t e = set_gain_smem<Rec>(h->d.k);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)h->d.k * kThreads * sizeof(int32_t);
    k_gain<Rec><<<h->d.n_tiles, kThreads, smem, h->stream>>>(h->d, r, s, all_elig ? 1 : 0, st_row);
    return cudaGetLastError();
}

cudaError_t launch_subround(hgp_handle *h, int32_t r, int32_t s, bool all_elig, unsigned long long *st_row)
{
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    cudaError_t e = d.k <= 32 ? launch_gain<Rec16>(h, r, s, all_elig, st_row)
                              : launch_gain<Rec32>(h, r, s, all_elig, st_row);
    if (e != cudaSuccess) return e;
    k_hist<<<d.n_tiles, kThreads, 0, st>>>(d, 0);
    k_select<<<d.k, kThreads, 0, st>>>(d, 0);
    if (h->max_vertex_netweight >= kBins - 1) {
        for (int level = 1; level <= 3; ++level) {
            k_hist<<<d.n_tiles, kThreads, 0, st>>>(d, level);
            k_select<<<d.k, kThreads, 0, st>>>(d, level);
        }
    }
    k_tie_sum<<<d.n_tiles, kThreads, 0, st>>>(d);
    k_tie_scan<<<d.k, 1024, 0, st>>>(d);
    if (d.k <= 32) k_apply<Rec16><<<d.n_tiles, kThreads, 0, st>>>(d, r, st_row);
    else k_apply<Rec32><<<d.n_tiles, kThreads, 0, st>>>(d, r, st_row);
    return cudaGetLastError();
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
        k_round_prep<<<d.n_tiles, kThreads, 0, st>>>(d, r, h->seed);
        e = cudaGetLastError();
        for (int32_t s = 0; s < d.S && e == cudaSuccess; ++s)
            e = launch_subround(h, r, s, h->all_eligible && rr == 0, row);
        if (e == cudaSuccess) {
            k_round_end<<<1, 32, 0, st>>>(d, row);
            e = cudaGetLastError();
        }
    }
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
        e = cudaGetLastError();
    }
    // the stats row written here is scratch: refine() clears the stats before use
    unsigned long long *row = reinterpret_cast<unsigned long long *>(d.stats);
    if (e == cudaSuccess)
        e = d.k <= 32 ? launch_gain<Rec16>(h, r, s, h->all_eligible, row) : launch_gain<Rec32>(h, r, s, h->all_eligible, row);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.tot, 0, sizeof(int64_t) * 64, st);
    if (e == cudaSuccess) {
        k_expand_candidates<<<(d.n_ranges * 32 + 255) / 256, 256, 0, st>>>(d, t_d, g_d);
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

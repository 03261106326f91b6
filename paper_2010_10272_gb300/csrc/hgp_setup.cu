// libhgp: creation, validation, CSR transpose, state initialisation and getters.
//
// Setup builds, on the device, everything the refinement rounds read:
//   * the vertex -> incident nets CSR I(v) from the net -> pins CSR (Sec. 2; the paper
//     builds the same two adjacency arrays with prefix sums, Sec. 3.2);
//   * Phi(e, i) from the partition (Sec. 2 / Sec. 5.1), Lambda(e), S1(e) and omega(e) in the
//     per-net record, the block weights and the (lambda-1) objective (Sec. 2).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>

#include "hgp_host.cuh"

using namespace hgp;

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ prefix sums (int32)
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *warp_tot, int32_t *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        int32_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        warp_tot[lane] = s - t;
        if (lane == 31) *total = s;
    }
    __syncthreads();
    const int32_t r = warp_tot[wid] + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const int32_t *in, int64_t count, int32_t *sums)
{
    __shared__ int32_t wt[32];
    __shared__ int32_t tot;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < count) s += in[base + i];
    block_exclusive_scan(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int32_t *sums, int64_t nb)
{
    __shared__ int32_t wt[32];
    __shared__ int32_t tot;
    int32_t carry = 0;
    for (int64_t b = 0; b < nb; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        const int32_t v = i < nb ? sums[i] : 0;
        const int32_t ex = block_exclusive_scan(v, wt, &tot);
        if (i < nb) sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_final(const int32_t *in, int32_t *out, int64_t count, const int32_t *sums)
{
    __shared__ int32_t wt[32];
    __shared__ int32_t tot;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < count ? in[base + i] : 0;
        s += v[i];
    }
    int32_t run = sums[blockIdx.x] + block_exclusive_scan(s, wt, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < count) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = sums[blockIdx.x] + tot;
}

// ------------------------------------------------------------------ validation
// warp per net: pins in range and strictly increasing; largest net size
// Warp-wide: the pins of nets e0 .. e0 + 31 (clipped to e_hi) are contiguous; off33 receives
// their exclusive offsets inside that run (off33[32] = its length) and the run's first pin index
// is returned.  Lanes then walk the run flattened, one pin each, with pin_net to find the net.
__device__ __forceinline__ int32_t net_group(const int32_t *off, int64_t e0, int64_t e_hi, int32_t *off33,
                                             int32_t &sz_lane)
{
    const int lane = threadIdx.x & 31;
    const int64_t e = e0 + lane;
    sz_lane = e < e_hi ? off[e + 1] - off[e] : 0;
    int32_t incl = sz_lane;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    off33[lane] = incl - sz_lane;
    if (lane == 31) off33[32] = incl;
    __syncwarp();
    return off[e0];
}

// slot of the net holding run position i: the largest s with off33[s] <= i (empty nets skipped)
__device__ __forceinline__ int pin_net(const int32_t *off33, int32_t i)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1)
        if (off33[lo + step] <= i) lo += step;
    return lo;
}

// pins in [0, n) and strictly increasing inside every net; the largest net size.  Runs after
// k_check_inputs and does nothing if that found an error.  A warp walks 32 nets' pins at once,
// coalesced.
__global__ void __launch_bounds__(256) k_check_pins(const int32_t *off, const int32_t *pins, int32_t m, int32_t n,
                                                    int32_t *err, int32_t *max_size)
{
    __shared__ int32_t off33_w[8][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *off33 = off33_w[wid];
    // the offsets may only be trusted when the checks before found nothing (they ran to
    // completion earlier on the same stream, so their flag is final)
    if (*reinterpret_cast<volatile int32_t *>(err) & ERR_INVALID) return;
    const int64_t warps = (int64_t)gridDim.x * 8;
    int32_t local_max = 0;
    bool bad = false;
    for (int64_t e0 = ((int64_t)blockIdx.x * 8 + wid) * 32; e0 < m; e0 += warps * 32) {
        int32_t sz;
        const int32_t base = net_group(off, e0, m, off33, sz);
        local_max = max(local_max, sz);
        const int32_t total = off33[32];
        for (int32_t i0 = lane; i0 < total; i0 += 128) {   // four pins (and predecessors) per lane
            int32_t vq[4], pq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t i = i0 + 32 * q;
                vq[q] = i < total ? pins[base + i] : 0;
                pq[q] = i < total && i > 0 ? pins[base + i - 1] : -1;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t i = i0 + 32 * q;
                if (i >= total) continue;
                if (vq[q] < 0 || vq[q] >= n) bad = true;
                if (i > off33[pin_net(off33, i)] && pq[q] >= vq[q]) bad = true;
            }
        }
        __syncwarp();
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(err, ERR_INVALID);
    for (int o = 16; o; o >>= 1) local_max = max(local_max, __shfl_xor_sync(kFull, local_max, o));
    if (lane == 0) atomicMax(max_size, local_max);
}

// ------------------------------------------------------------------ internal net order
// Nets are relabelled by size class, the largest class first and by input id inside a class.
// On skewed instances a few large nets take most record gathers (each incidence reads its net's
// record); stored first, their records and Phi rows share L2 lines and stay resident there.
// Gains, objective and every move are sums over nets, so results do not depend on the order.
constexpr int kNrRanks = 32;        // rank 0: the largest size class (2^30 pins and up)
constexpr int kNrThreads = 256;

__device__ __forceinline__ int nr_rank(int32_t size)
{
    return size <= 1 ? kNrRanks - 1 : __clz(size);   // sizes [2^c, 2^(c+1)) -> 31 - c
}

// per CTA (a contiguous chunk of per_cta nets): nets per rank, written rank-major so that one
// exclusive scan yields every (rank, CTA) base position
__global__ void __launch_bounds__(kNrThreads) k_nr_count(const int32_t *off, int32_t m, int32_t per_cta,
                                                         int32_t *cnt)
{
    __shared__ int32_t c[kNrRanks];
    if (threadIdx.x < kNrRanks) c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t lo = (int64_t)blockIdx.x * per_cta;
    const int64_t hi = min((int64_t)m, lo + per_cta);
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) atomicAdd(&c[nr_rank(off[e + 1] - off[e])], 1);
    __syncthreads();
    if (threadIdx.x < kNrRanks) cnt[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = c[threadIdx.x];
}

// same chunks: internal id of every net (stable inside a rank) and the sizes in internal order
__global__ void __launch_bounds__(kNrThreads) k_nr_place(const int32_t *off, int32_t m, int32_t per_cta,
                                                         const int32_t *base, int32_t *perm, int32_t *size_int)
{
    constexpr int W = kNrThreads / 32;
    __shared__ int32_t run[kNrRanks];
    __shared__ int32_t wc[W][kNrRanks];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < kNrRanks) run[threadIdx.x] = base[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
    const int64_t lo = (int64_t)blockIdx.x * per_cta;
    const int64_t hi = min((int64_t)m, lo + per_cta);
    for (int64_t c0 = lo; c0 < hi; c0 += kNrThreads) {
        for (int i = threadIdx.x; i < W * kNrRanks; i += kNrThreads) (&wc[0][0])[i] = 0;
        __syncthreads();
        const int64_t e = c0 + threadIdx.x;
        const bool valid = e < hi;
        const int32_t size = valid ? off[e + 1] - off[e] : 0;
        const int rk = valid ? nr_rank(size) : kNrRanks;
        const unsigned peers = __match_any_sync(kFull, rk);
        const int below = __popc(peers & ((1u << lane) - 1));
        if (valid && below == 0) wc[wid][rk] = __popc(peers);
        __syncthreads();
        if (valid) {
            int32_t pos = run[rk] + below;
            for (int w = 0; w < wid; ++w) pos += wc[w][rk];
            perm[e] = pos;
            size_int[pos] = size;
        }
        __syncthreads();
        if (threadIdx.x < kNrRanks) {
            int32_t t = 0;
            for (int w = 0; w < W; ++w) t += wc[w][threadIdx.x];
            run[threadIdx.x] += t;
        }
        __syncthreads();
    }
}

// pins (and net weights) into internal order; a warp copies the pins of 32 consecutive input
// nets, reading them as one coalesced run
__global__ void __launch_bounds__(256) k_nr_pins(const int32_t *off, const int32_t *pins, const int32_t *nw,
                                                 int32_t m, const int32_t *perm, const int32_t *off_int,
                                                 int32_t *pins_int, int32_t *nw_int)
{
    __shared__ int32_t off33_w[8][33];
    __shared__ int32_t dst_w[8][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *off33 = off33_w[wid];
    const int64_t warps = (int64_t)gridDim.x * 8;
    for (int64_t e0 = ((int64_t)blockIdx.x * 8 + wid) * 32; e0 < m; e0 += warps * 32) {
        int32_t sz;
        const int32_t src = net_group(off, e0, m, off33, sz);
        const int64_t e = e0 + lane;
        if (e < m) {
            const int32_t q = perm[e];
            dst_w[wid][lane] = off_int[q];
            if (nw) nw_int[q] = nw[e];
        }
        __syncwarp();
        const int32_t total = off33[32];
        for (int32_t i0 = lane; i0 < total; i0 += 128) {   // four loads in flight per lane
            int32_t vq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) vq[q] = i0 + 32 * q < total ? pins[src + i0 + 32 * q] : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t i = i0 + 32 * q;
                if (i >= total) continue;
                const int sl = pin_net(off33, i);
                pins_int[dst_w[wid][sl] + (i - off33[sl])] = vq[q];
            }
        }
        __syncwarp();
    }
}

__global__ void k_check_vertices(const int32_t *vw, const int32_t *part_in, int32_t n, int32_t k,
                                 int32_t *err)
{
    bool bad = false;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (vw && vw[v] < 1) bad = true;
        if (part_in) {
            const int32_t p = part_in[v];
            if (p < 0 || p >= k) bad = true;
        }
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_INVALID);
}

// Creation queues its kernels behind the input checks without waiting for their verdict (for
// instances whose net sizes the host reads itself, see create_impl): every kernel that indexes
// by a pin, a vertex id or a block then returns at once when the checks flagged the input, and
// the creation reports HGP_ERR_INVALID at its one read-back.  guard: the creation's error flag,
// or nullptr outside creation.
__device__ __forceinline__ bool input_invalid(const int32_t *guard)
{
    return guard && (*reinterpret_cast<const volatile int32_t *>(guard) & ERR_INVALID) != 0;
}

// The creation's checks of the offsets (converted to int32 on the way), the net and vertex
// weights and the partition in one launch; the valid partition entries are stored as the 1-byte
// Pi at the same time.
__global__ void k_check_inputs(const int64_t *off64, int32_t *off32, int32_t m, int64_t P, const int32_t *nw,
                               const int32_t *vw, const int32_t *part_in, int32_t n, int32_t k, uint8_t *part,
                               int32_t *err)
{
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t e = t0; e <= m; e += stride) {
        const int64_t a = off64[e];
        if ((e == 0 && a != 0) || (e == m && a != P) || a < 0 || a > P) bad = true;
        if (e < m && off64[e + 1] < a) bad = true;
        if (e < m && nw && nw[e] < 1) bad = true;
        off32[e] = (int32_t)(a < 0 ? 0 : (a > P ? P : a));
    }
    for (int64_t v = t0; v < n; v += stride) {
        if (vw && vw[v] < 1) bad = true;
        const int32_t p = part_in[v];
        if (p < 0 || p >= k) bad = true;
        else part[v] = (uint8_t)p;
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_INVALID);
}

// ------------------------------------------------------------------ per-vertex net weight
// W(u) = sum of incident net weights must stay below 2^31 (int32 gain arithmetic)
__global__ void k_vertex_netweight(const int32_t *vtx_off, const int32_t *inc, const int32_t *nw,
                                   int32_t n, int32_t *err, unsigned long long *max_w)
{
    if (input_invalid(err)) return;
    unsigned long long local = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (int32_t j = vtx_off[v]; j < vtx_off[v + 1]; ++j) s += nw ? nw[inc[j] & kNetMask] : 1;
        if (s >= (int64_t)1 << 31) atomicOr(err, ERR_UNSUPPORTED);
        local = max(local, (unsigned long long)s);
    }
    for (int o = 16; o; o >>= 1) local = max(local, __shfl_xor_sync(kFull, local, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_w, local);
}

// ------------------------------------------------------------------ transpose (net -> vertex)
// Direct form, for instances whose vertex counters fit in L2: degrees by atomic increments,
// an exclusive scan into vtx_off, then every pin takes the next slot of its vertex (warp per
// net) and stores the net id with the wide flag.
constexpr int32_t kTpDirectMaxN = 1 << 21;
// nets are stored in internal (size class) order from this many nets on, when the largest net
// has at least kReorderSkew times the average size: below that count their records fit in L2
// whatever the order, and without large nets no small set of records takes most gathers (on
// near-uniform sizes the relabelling only adds creation time)
constexpr int32_t kReorderMinNets = 1 << 20;
constexpr int64_t kReorderSkew = 8;
// host inputs with fewer nets than this: the host reads the net sizes (see create_impl)
constexpr int32_t kHostSizesMaxNets = 1 << 20;
// in internal order, nets of at least this many pins (a prefix) get their own CTAs at creation
// and initialisation (a power of two: size classes are powers of two)
constexpr int32_t kBigNet = 256;

__global__ void k_degrees(const int32_t *pins, int64_t P, int32_t *deg, const int32_t *guard)
{
    if (input_invalid(guard)) return;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[pins[j]], 1);
}

__global__ void k_scatter(const int32_t *off, const int32_t *pins, int32_t m, int32_t narrow_max, int32_t *fill,
                          int32_t *inc, const int32_t *guard)
{
    if (input_invalid(guard)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < m; e += warps) {
        const int32_t b = off[e], end = off[e + 1];
        const int32_t ef = (int32_t)((uint32_t)e | (end - b > narrow_max ? kWideFlag : 0u));
        for (int32_t j = b + lane; j < end; j += 32) {
            const int32_t pos = atomicAdd(&fill[pins[j]], 1);
            inc[pos] = ef;
        }
    }
}

// Bucketed form, for large instances:
// vertices are grouped into buckets of 2^bshift consecutive ids (at most
// kTpMaxBuckets buckets).  k_tp_hist counts the pins per bucket; k_tp_scatter writes every pin
// as a (vertex, net | wide flag) pair into its bucket's region, reserving one range per (CTA,
// bucket) with a single global atomic; k_tp_place, a CTA per bucket, counts the degrees of its
// vertices, scans them into vtx_off and places the nets into inc.  Every step but the pair
// scatter stays inside one bucket's few hundred KB, so the random accesses hit L2.
constexpr int kTpMaxBuckets = 4096;
constexpr int kTpShift = 14;             // 16384 vertices per bucket, unless that gives too few
constexpr int kTpMinShift = 8;           // buckets for the GPU (small instances) or too many
constexpr int kTpSmemShift = 14;         // buckets up to this size count in shared memory
// nets per scatter CTA, at most (fewer when the instance has few nets): each CTA's walk over its
// nets is a chain of dependent loads, so many short walks beat few long ones even though every
// CTA reserves a range in every bucket (power-law creation: 16384 -> 30.1 ms, 4096 -> 25.1 ms,
// 2048 -> 23.3 ms, 512 -> 23.1 ms)
constexpr int kTpNetsPerCta = 2048;
constexpr int kTpMinCtas = 608;          // target CTAs per launch (4 per SM)

__global__ void __launch_bounds__(256) k_tp_hist(const int32_t *pins, int64_t P, int bshift, int32_t nb,
                                                 int32_t *bucket_cnt, const int32_t *guard)
{
    if (input_invalid(guard)) return;
    __shared__ int32_t h[kTpMaxBuckets];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P; j += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[pins[j] >> bshift], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (h[i]) atomicAdd(&bucket_cnt[i], h[i]);
}

// CTA per per_cta nets; pass 0 counts its pins per bucket, then one range per bucket is
// reserved, pass 1 writes the pairs.  A warp walks the pins of 32 nets at once (coalesced).
__global__ void __launch_bounds__(256) k_tp_scatter(const int32_t *off, const int32_t *pins, int32_t m,
                                                    int32_t e_begin, int bshift, int32_t nb, int32_t narrow_max,
                                                    int32_t per_cta, int32_t *bucket_cur, unsigned long long *pairs,
                                                    const int32_t *guard)
{
    if (input_invalid(guard)) return;
    __shared__ int32_t cur[kTpMaxBuckets];
    __shared__ int32_t off33_w[8][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *off33 = off33_w[wid];
    const int64_t e_lo = e_begin + (int64_t)blockIdx.x * per_cta;
    const int64_t e_hi = min((int64_t)m, e_lo + per_cta);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) cur[i] = 0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t e0 = e_lo + 32 * wid; e0 < e_hi; e0 += 32 * 8) {
            int32_t sz;
            const int32_t base = net_group(off, e0, e_hi, off33, sz);
            const int32_t total = off33[32];
            // four pins per lane are loaded before any is used (their latencies overlap)
            for (int32_t i0 = lane; i0 < total; i0 += 128) {
                int32_t vq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) vq[q] = i0 + 32 * q < total ? pins[base + i0 + 32 * q] : -1;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (vq[q] < 0) continue;
                    const int32_t i = i0 + 32 * q, v = vq[q];
                    const int32_t pos = atomicAdd(&cur[v >> bshift], 1);
                    if (pass == 1) {
                        const int sl = pin_net(off33, i);
                        const uint32_t ef = (uint32_t)(e0 + sl) | (off33[sl + 1] - off33[sl] > narrow_max ? kWideFlag : 0u);
                        pairs[pos] = ((unsigned long long)(uint32_t)v << 32) | ef;
                    }
                }
            }
            __syncwarp();
        }
        __syncthreads();
        if (pass == 0) {
            for (int i = threadIdx.x; i < nb; i += blockDim.x) {
                const int32_t c = cur[i];
                cur[i] = c ? atomicAdd(&bucket_cur[i], c) : 0;
            }
            __syncthreads();
        }
    }
}

// The pins of the large-net prefix [0, m_big) of the internal order (nets of at least kBigNet
// pins), split into chunks of kTpBigChunk pins, one CTA each, so that no CTA takes many large
// nets.  A chunk overlaps at most kTpBigChunk / kBigNet + 2 nets, whose offsets are staged in
// shared memory.  Same two passes as k_tp_scatter.
constexpr int kTpBigChunk = 8192;
constexpr int kTpBigWin = kTpBigChunk / kBigNet + 3;   // offsets of the nets a chunk overlaps, + 1

__global__ void __launch_bounds__(256) k_tp_scatter_big(const int32_t *off, const int32_t *pins, int32_t m_big,
                                                        int bshift, int32_t nb, int32_t narrow_max,
                                                        int32_t *bucket_cur, unsigned long long *pairs,
                                                        const int32_t *guard)
{
    if (input_invalid(guard)) return;
    __shared__ int32_t cur[kTpMaxBuckets];
    __shared__ int32_t win[kTpBigWin];
    __shared__ int32_t first;
    const int32_t p_end = off[m_big];
    const int32_t p0 = blockIdx.x * kTpBigChunk;
    const int32_t p1 = min(p_end, p0 + kTpBigChunk);
    if (threadIdx.x == 0) {   // the net holding pin p0: the largest e < m_big with off[e] <= p0
        int32_t lo = 0, hi = m_big - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= p0) lo = mid;
            else hi = mid - 1;
        }
        first = lo;
    }
    for (int i = threadIdx.x; i < nb; i += blockDim.x) cur[i] = 0;
    __syncthreads();
    const int32_t e_f = first;
    for (int i = threadIdx.x; i < kTpBigWin; i += blockDim.x) win[i] = off[min(m_big, e_f + i)];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int32_t j = p0 + threadIdx.x; j < p1; j += blockDim.x) {
            const int32_t v = pins[j];
            const int32_t pos = atomicAdd(&cur[v >> bshift], 1);
            if (pass == 1) {
                int sl = 0;   // the largest slot with win[sl] <= j
#pragma unroll
                for (int step = 32; step; step >>= 1)
                    if (sl + step < kTpBigWin && win[sl + step] <= j) sl += step;
                const uint32_t ef = (uint32_t)(e_f + sl) | (win[sl + 1] - win[sl] > narrow_max ? kWideFlag : 0u);
                pairs[pos] = ((unsigned long long)(uint32_t)v << 32) | ef;
            }
        }
        __syncthreads();
        if (pass == 0) {
            for (int i = threadIdx.x; i < nb; i += blockDim.x) {
                const int32_t c = cur[i];
                cur[i] = c ? atomicAdd(&bucket_cur[i], c) : 0;
            }
            __syncthreads();
        }
    }
}

// CTA per bucket: degrees, their exclusive prefix (from the bucket's first pair position) into
// vtx_off, then the nets of the bucket's pairs into inc.  SMEM: the bucket's counters live in
// shared memory (buckets of at most 2^kTpSmemShift vertices); otherwise in cursor (zeroed
// int32[n], global).
constexpr int kTpPlaceBatch = 8;

template <bool SMEM>
__global__ void __launch_bounds__(1024) k_tp_place(const unsigned long long *pairs, const int32_t *bucket_off,
                                                   int bshift, int32_t n, int32_t nb, int32_t *cursor,
                                                   int32_t *vtx_off, int32_t *inc, const int32_t *guard)
{
    if (input_invalid(guard)) return;
    __shared__ int32_t wt[32];
    __shared__ int32_t tot;
    extern __shared__ int32_t sc[];
    const int32_t bkt = blockIdx.x;
    const int64_t v0 = (int64_t)bkt << bshift;
    const int64_t v1 = min((int64_t)n, v0 + ((int64_t)1 << bshift));
    const int32_t p0 = bucket_off[bkt], p1 = bucket_off[bkt + 1];
    int32_t *cnt = SMEM ? sc : cursor + v0;          // indexed by v - v0
    if (SMEM)
        for (int64_t i = threadIdx.x; i < v1 - v0; i += blockDim.x) sc[i] = 0;
    __syncthreads();
    // kTpPlaceBatch pairs per thread are loaded before any is used (the loads' latencies overlap)
    const int32_t step = (int32_t)blockDim.x * kTpPlaceBatch;
    for (int32_t i0 = p0 + threadIdx.x; i0 < p1; i0 += step) {
        unsigned long long pr[kTpPlaceBatch];
#pragma unroll
        for (int q = 0; q < kTpPlaceBatch; ++q) {
            const int32_t i = i0 + q * (int32_t)blockDim.x;
            pr[q] = i < p1 ? pairs[i] : ~0ull;            // read again below: keep in L2
        }
#pragma unroll
        for (int q = 0; q < kTpPlaceBatch; ++q)
            if (pr[q] != ~0ull) atomicAdd(&cnt[(int32_t)(pr[q] >> 32) - v0], 1);
    }
    __syncthreads();
    int32_t carry = p0;
    for (int64_t base = v0; base < v1; base += blockDim.x) {
        const int64_t v = base + threadIdx.x;
        const int32_t dv = v < v1 ? (SMEM ? sc[v - v0] : __ldcg(&cnt[v - v0])) : 0;
        const int32_t ex = block_exclusive_scan(dv, wt, &tot);
        if (v < v1) {
            vtx_off[v] = carry + ex;
            cnt[v - v0] = carry + ex;
        }
        carry += tot;
    }
    if (bkt == nb - 1 && threadIdx.x == 0) vtx_off[n] = p1;
    __syncthreads();
    for (int32_t i0 = p0 + threadIdx.x; i0 < p1; i0 += step) {
        unsigned long long pr[kTpPlaceBatch];
#pragma unroll
        for (int q = 0; q < kTpPlaceBatch; ++q) {
            const int32_t i = i0 + q * (int32_t)blockDim.x;
            pr[q] = i < p1 ? __ldcs(&pairs[i]) : ~0ull;
        }
#pragma unroll
        for (int q = 0; q < kTpPlaceBatch; ++q) {
            if (pr[q] == ~0ull) continue;
            const int32_t pos = atomicAdd(&cnt[(int32_t)(pr[q] >> 32) - v0], 1);
            inc[pos] = (int32_t)(uint32_t)pr[q];
        }
    }
}

__global__ void k_wide_flags(const int32_t *off, int32_t m, int32_t narrow_max, int32_t *flags)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        flags[e] = (off[e + 1] - off[e]) > narrow_max ? 1 : 0;
}

// ------------------------------------------------------------------ state initialisation
__global__ void k_copy_part(const int32_t *in, uint8_t *part, int32_t n)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        part[v] = (uint8_t)in[v];
}

__global__ void k_block_weights(Dev d, const int32_t *guard)
{
    if (input_invalid(guard)) return;
    __shared__ unsigned long long w[64];
    if (threadIdx.x < 64) w[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < d.n;
         v += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&w[d.part[v]], (unsigned long long)(d.vw ? d.vw[v] : 1));
    __syncthreads();
    if (threadIdx.x < d.k && w[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(&d.bw[threadIdx.x]), w[threadIdx.x]);
}

// Counts Phi(e, .) from the partition, writes the Phi rows, the records (Lambda, S1, omega,
// stamp) and adds (lambda(e) - 1) * omega(e) to the objective.  A warp takes 32 consecutive nets,
// one per lane: a net of at most kSmallNet pins is counted by its lane in registers; larger nets
// are then counted by the whole warp, one at a time, with shared-memory counters.  The 32 Phi
// rows are assembled in shared memory and written as one contiguous block (coalesced, and no
// separate zeroing of the table); the rows of nets in the wide table stay zero there.
constexpr int kSmallNet = 8;
constexpr int kInitWarps = 8;

template <typename Rec>
__device__ __forceinline__ void write_record(const Dev &d, int64_t e, uint64_t lam, uint64_t s1, int32_t wf)
{
    Rec *rec = reinterpret_cast<Rec *>(d.rec) + e;
    if constexpr (sizeof(Rec) == 16) {
        Rec r;
        r.s1 = (uint32_t)s1;
        r.w = wf;
        r.mv = kNever * 2;
        r.lam = (uint32_t)lam;
        *rec = r;
    } else {
        Rec r;
        r.s1 = s1;
        r.w = wf;
        r.mv = kNever * 2;
        r.lam = lam;
        r.w2 = wf;
        r.pad = 0;
        *rec = r;
    }
}

// entry i of the staged row block (rows of `wb` bytes per net, entries of `w` bytes)
__device__ __forceinline__ void stage_set(uint8_t *blk, int row, int i, int w, int wb, int32_t v)
{
    uint8_t *p = blk + row * wb + i * w;
    if (w == 1) *p = (uint8_t)v;
    else if (w == 2) *reinterpret_cast<uint16_t *>(p) = (uint16_t)v;
    else *reinterpret_cast<int32_t *>(p) = v;
}

template <typename Rec>
__global__ void __launch_bounds__(kInitWarps * 32) k_init_nets(Dev d, int32_t e_begin, const int32_t *guard)
{
    if (input_invalid(guard)) return;
    __shared__ int32_t cnt[kInitWarps][64];
    __shared__ long long part_obj[kInitWarps];
    extern __shared__ __align__(16) uint32_t stage_dyn[];   // kInitWarps blocks of 32 rows
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * kInitWarps;
    const int32_t narrow_max = d.phi_w == 1 ? 255 : (d.phi_w == 2 ? 65535 : 0x7fffffff);
    const int w = d.phi_w, wb = d.k * d.phi_w;       // bytes per entry / per row
    const int blk_words = (32 * wb + 15) / 16 * 4;   // one warp's block, 16-byte multiple
    uint32_t *stage_w = stage_dyn + wid * blk_words;
    uint8_t *stage = reinterpret_cast<uint8_t *>(stage_w);
    long long obj = 0;
    for (int64_t e0 = e_begin + ((int64_t)blockIdx.x * kInitWarps + wid) * 32; e0 < d.m; e0 += warps * 32) {
        const int32_t rows = (int32_t)min((int64_t)32, (int64_t)d.m - e0);
        for (int i = lane; i < blk_words; i += 32) stage_w[i] = 0;
        __syncwarp();
        const int64_t e = e0 + lane;
        int32_t b = 0, size = 0;
        if (e < d.m) {
            b = d.net_off[e];
            size = d.net_off[e + 1] - b;
        }
        const bool small = e < d.m && size <= kSmallNet;
        if (small) {
            int32_t blk[kSmallNet], c[kSmallNet];
            int nd = 0;
#pragma unroll
            for (int i = 0; i < kSmallNet; ++i) {
                blk[i] = -1;
                c[i] = 0;
            }
#pragma unroll
            for (int i = 0; i < kSmallNet; ++i) {
                if (i < size) {
                    const int bk = d.part[d.pins[b + i]];
                    bool found = false;
#pragma unroll
                    for (int j = 0; j < kSmallNet; ++j) {
                        if (blk[j] == bk) { ++c[j]; found = true; }
                    }
                    if (!found) {
#pragma unroll
                        for (int j = 0; j < kSmallNet; ++j)
                            if (j == nd) { blk[j] = bk; c[j] = 1; }
                        ++nd;
                    }
                }
            }
            uint64_t lam = 0, s1 = 0;
#pragma unroll
            for (int j = 0; j < kSmallNet; ++j) {
                if (j < nd) {
                    lam |= 1ull << blk[j];
                    if (c[j] == 1) s1 |= 1ull << blk[j];
                    stage_set(stage, lane, blk[j], w, wb, c[j]);
                }
            }
            const int32_t wv = d.nw ? d.nw[e] : 1;
            write_record<Rec>(d, e, lam, s1, wv);
            if (nd > 0) obj += (long long)(nd - 1) * wv;
        }
        // larger nets: the whole warp on one net at a time
        unsigned big = __ballot_sync(kFull, e < d.m && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t ee = e0 + src;
            const int32_t bb = __shfl_sync(kFull, b, src), sz = __shfl_sync(kFull, size, src);
            cnt[wid][lane] = 0;
            cnt[wid][lane + 32] = 0;
            __syncwarp();
            for (int32_t base = bb; base < bb + sz; base += 32) {
                const int32_t j = base + lane;
                const bool act = j < bb + sz;
                const unsigned mask = __ballot_sync(kFull, act);
                if (act) {
                    const int blk = d.part[d.pins[j]];
                    const unsigned peers = __match_any_sync(mask, blk);
                    if (lane == __ffs(peers) - 1) cnt[wid][blk] += __popc(peers);
                }
                __syncwarp();
            }
            const int32_t wv = d.nw ? d.nw[ee] : 1;
            const bool wide = d.widx != nullptr && sz > narrow_max;
            const int32_t wrow = wide ? d.widx[ee] : 0;
            for (int i = lane; i < d.k; i += 32) {
                if (wide) d.phi_wide[(int64_t)wrow * d.k + i] = cnt[wid][i];
                else stage_set(stage, src, i, w, wb, cnt[wid][i]);
            }
            const unsigned lo_lam = __ballot_sync(kFull, lane < d.k && cnt[wid][lane] > 0);
            const unsigned lo_s1 = __ballot_sync(kFull, lane < d.k && cnt[wid][lane] == 1);
            const unsigned hi_lam = __ballot_sync(kFull, lane + 32 < d.k && cnt[wid][lane + 32] > 0);
            const unsigned hi_s1 = __ballot_sync(kFull, lane + 32 < d.k && cnt[wid][lane + 32] == 1);
            if (lane == 0) {
                const int32_t wf = wv | (wide ? (int32_t)kWideFlag : 0);
                write_record<Rec>(d, ee, (uint64_t)lo_lam | ((uint64_t)hi_lam << 32),
                                  (uint64_t)lo_s1 | ((uint64_t)hi_s1 << 32), wf);
                const int lambda = __popc(lo_lam) + __popc(hi_lam);
                if (lambda > 0) obj += (long long)(lambda - 1) * wv;
            }
            __syncwarp();
        }
        __syncwarp();
        // the block of rows e0 .. e0 + rows - 1 starts at byte e0 * wb of the table
        const int64_t byte0 = e0 * (int64_t)wb;
        uint8_t *dst = reinterpret_cast<uint8_t *>(d.phi) + byte0;
        if ((byte0 & 15) == 0 && (rows * wb) % 16 == 0) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(stage_w);
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            for (int i = lane; i < rows * wb / 16; i += 32) d4[i] = s4[i];
        } else {
            // byte-exact tail (the table's rows need not be 16-byte multiples for small k)
            for (int i = lane; i < rows * wb; i += 32) dst[i] = stage[i];
        }
        __syncwarp();
    }
    for (int o = 16; o; o >>= 1) obj += __shfl_xor_sync(kFull, obj, o);
    if (lane == 0) part_obj[wid] = obj;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int i = 0; i < kInitWarps; ++i) s += part_obj[i];
        if (s) atomicAdd(reinterpret_cast<unsigned long long *>(d.obj), (unsigned long long)s);
    }
}

// The nets of at least kBigNet pins, stored first in internal order (the prefix [0, m_big),
// rounded up to whole 32-net groups), one CTA per net: k_init_nets would give all of them to
// the first few warps.  Same results as k_init_nets for these nets (the narrow row of a net in
// the wide table is written as zeros).
template <typename Rec>
__global__ void __launch_bounds__(256) k_init_big(Dev d, int32_t m_big, const int32_t *guard)
{
    if (input_invalid(guard)) return;
    __shared__ int32_t cnt[64];
    const int lane = threadIdx.x & 31;
    const int32_t narrow_max = d.phi_w == 1 ? 255 : (d.phi_w == 2 ? 65535 : 0x7fffffff);
    const int w = d.phi_w, wb = d.k * d.phi_w;
    long long obj = 0;
    for (int64_t e = blockIdx.x; e < m_big; e += gridDim.x) {
        if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
        __syncthreads();
        const int32_t b = d.net_off[e], sz = d.net_off[e + 1] - b;
        for (int32_t j0 = 0; j0 < sz; j0 += blockDim.x) {
            const int32_t j = j0 + threadIdx.x;
            const bool act = j < sz;
            const unsigned mask = __ballot_sync(kFull, act);
            if (act) {
                const int blk = d.part[d.pins[b + j]];
                const unsigned peers = __match_any_sync(mask, blk);
                if (lane == __ffs(peers) - 1) atomicAdd(&cnt[blk], (int)__popc(peers));
            }
        }
        __syncthreads();
        const bool wide = d.widx != nullptr && sz > narrow_max;
        uint8_t *row = reinterpret_cast<uint8_t *>(d.phi) + e * (int64_t)wb;
        for (int i = threadIdx.x; i < d.k; i += blockDim.x) {
            stage_set(row, 0, i, w, wb, wide ? 0 : cnt[i]);
            if (wide) d.phi_wide[(int64_t)d.widx[e] * d.k + i] = cnt[i];
        }
        if (threadIdx.x < 32) {
            const unsigned lo_lam = __ballot_sync(kFull, lane < d.k && cnt[lane] > 0);
            const unsigned lo_s1 = __ballot_sync(kFull, lane < d.k && cnt[lane] == 1);
            const unsigned hi_lam = __ballot_sync(kFull, lane + 32 < d.k && cnt[lane + 32] > 0);
            const unsigned hi_s1 = __ballot_sync(kFull, lane + 32 < d.k && cnt[lane + 32] == 1);
            if (lane == 0) {
                const int32_t wv = d.nw ? d.nw[e] : 1;
                write_record<Rec>(d, e, (uint64_t)lo_lam | ((uint64_t)hi_lam << 32),
                                  (uint64_t)lo_s1 | ((uint64_t)hi_s1 << 32), wv | (wide ? (int32_t)kWideFlag : 0));
                const int lambda = __popc(lo_lam) + __popc(hi_lam);
                if (lambda > 0) obj += (long long)(lambda - 1) * wv;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && obj) atomicAdd(reinterpret_cast<unsigned long long *>(d.obj), (unsigned long long)obj);
}

// ------------------------------------------------------------------ getters
__global__ void k_obj_from_phi(Dev d, unsigned long long *out)
{
    long long s = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t size = d.net_off[e + 1] - d.net_off[e];
        const bool wide = d.widx != nullptr && size > (d.phi_w == 1 ? 255 : (d.phi_w == 2 ? 65535 : 0x7fffffff));
        const int32_t wrow = wide ? d.widx[e] : 0;
        int lambda = 0;
        for (int i = 0; i < d.k; ++i) lambda += phi_get(d, (int32_t)e, i, wide, wrow) > 0;
        if (lambda > 0) s += (long long)(lambda - 1) * (d.nw ? d.nw[e] : 1);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, (unsigned long long)s);
}

// the per-net getters and the checkpoint take nets in input order
__device__ __forceinline__ int32_t internal_net(const Dev &d, int32_t e)
{
    return d.net_perm ? d.net_perm[e] : e;
}

__global__ void k_widen_phi(Dev d, int32_t *out)
{
    const int64_t total = (int64_t)d.m * d.k;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = internal_net(d, (int32_t)(x / d.k)), i = (int32_t)(x % d.k);
        const int32_t size = d.net_off[e + 1] - d.net_off[e];
        const bool wide = d.widx != nullptr && size > (d.phi_w == 1 ? 255 : (d.phi_w == 2 ? 65535 : 0x7fffffff));
        out[x] = phi_get(d, e, i, wide, wide ? d.widx[e] : 0);
    }
}

template <typename Rec>
__global__ void k_get_lambda(Dev d, uint64_t *out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.m;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (uint64_t)reinterpret_cast<const Rec *>(d.rec)[internal_net(d, (int32_t)e)].lam;
}

// move stamps of the records
template <typename Rec>
__global__ void k_export_moved(Dev d, int32_t r, int32_t first, uint8_t *out)
{
    const Rec *recs = reinterpret_cast<const Rec *>(d.rec);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.m;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (!first && moved_in_prev_round(recs[internal_net(d, (int32_t)e)].mv, r)) ? 1 : 0;
}

template <typename Rec>
__global__ void k_import_moved(Dev d, int32_t r, const uint8_t *flags)
{
    Rec *recs = reinterpret_cast<Rec *>(d.rec);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.m;
         e += (int64_t)gridDim.x * blockDim.x)
        if (flags[e]) recs[internal_net(d, (int32_t)e)].mv = (r - 1) * 2;   // last move in round r-1
}

__global__ void k_set_round_state(int32_t *rs, int32_t r, int32_t started)
{
    if (threadIdx.x == 0) {
        rs[0] = r;
        rs[1] = started;
    }
}

__global__ void k_part_to_i32(const uint8_t *part, int32_t *out, int32_t n)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        out[v] = part[v];
}

// ------------------------------------------------------------------ host helpers
int grid_for(int64_t work, int threads, int cap = 152 * 32)
{
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

namespace hgp {

static constexpr int kMaxPoolDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[kMaxPoolDevices];

static std::atomic<cudaMemPool_t> g_pool_ready[kMaxPoolDevices];   // set once created

// the library's pool on the current device, created on first use
cudaError_t library_pool(cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    if (cudaMemPool_t ready = g_pool_ready[dev].load(std::memory_order_acquire)) {
        *out = ready;
        return cudaSuccess;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e != cudaSuccess) {
            g_pool[dev] = nullptr;
            return e;
        }
        g_pool_ready[dev].store(g_pool[dev], std::memory_order_release);
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

static std::atomic<int> g_blocking_waits{0};

// a blocking-sync event per thread and device, destroyed when the thread ends
struct WaitEvents {
    cudaEvent_t ev[kMaxPoolDevices] = {};
    ~WaitEvents()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        (void)cudaGetLastError();
    }
};
static thread_local WaitEvents t_wait;

cudaError_t stream_wait(cudaStream_t st)
{
    if (!g_blocking_waits.load(std::memory_order_relaxed)) return cudaStreamSynchronize(st);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    cudaEvent_t &ev = t_wait.ev[dev];
    if (!ev) {
        e = cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming);
        if (e != cudaSuccess) {
            ev = nullptr;
            return e;
        }
    }
    e = cudaEventRecord(ev, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev);
    return e;
}

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = library_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
    }
    return e;
}

void dev_free(void *p, cudaStream_t st)
{
    if (p && pool_free(p, st) != cudaSuccess) (void)cudaGetLastError();
}

}  // namespace hgp

namespace {

template <typename T>
cudaError_t dalloc(hgp_handle *h, T **p, int64_t count)
{
    *p = nullptr;
    if (count < 1) count = 1;
    if (void *a = arena_take(h, (size_t)count * sizeof(T))) {
        *p = reinterpret_cast<T *>(a);
        return cudaSuccess;
    }
    if (h->n_allocs >= hgp_handle::kMaxAllocs) return cudaErrorMemoryAllocation;
    void *q = nullptr;
    cudaError_t e = dev_alloc(&q, (size_t)count * sizeof(T), h->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e;
    }
    h->allocs[h->n_allocs++] = q;
    *p = reinterpret_cast<T *>(q);
    return cudaSuccess;
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) {                   \
            (void)cudaGetLastError();              \
            return status_of(_e);                  \
        }                                          \
    } while (0)

// guard: the creation's error flag while creating (kernels skip flagged input), else nullptr
int init_state(hgp_handle *h, const int32_t *guard)
{
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    CK(cudaMemsetAsync(d.bw, 0, sizeof(int64_t) * d.k, st));
    CK(cudaMemsetAsync(d.obj, 0, sizeof(int64_t), st));
    // round 0, every vertex eligible
    CK(cudaMemsetAsync(d.rs, 0, 2 * sizeof(int32_t), st));
    // the net kernel writes every narrow Phi row (zeros included); the wide table's rows are
    // written by their nets, but a row of a net with zero pins in range stays as zeroed here
    if (d.phi_wide && h->n_wide > 0) CK(cudaMemsetAsync(d.phi_wide, 0, sizeof(int32_t) * (size_t)h->n_wide * d.k, st));
    k_block_weights<<<grid_for(d.n, 256), 256, 0, st>>>(d, guard); h->launches++;
    CK(cudaGetLastError());
    const int32_t e_begin = h->m_big32;
    if (e_begin > 0) {
        const int gb = e_begin < 152 * 16 ? e_begin : 152 * 16;
        if (d.k <= 32) k_init_big<Rec16><<<gb, 256, 0, st>>>(d, e_begin, guard);
        else k_init_big<Rec32><<<gb, 256, 0, st>>>(d, e_begin, guard);
        h->launches++;
    }
    if (d.m > e_begin) {
        const int g = grid_for(((int64_t)d.m - e_begin + 31) / 32 * 32, kInitWarps * 32, 152 * 16);
        auto init_smem = [](int k, int w) { return kInitWarps * (32 * k * w + 15) / 16 * 16; };
        const int smem = init_smem(d.k, d.phi_w);
        // the attribute is the kernel's largest need over every k and entry width (the same
        // value from every caller), so concurrent creations cannot lower it under each other
        if (d.k <= 32) {
            cudaFuncSetAttribute(k_init_nets<Rec16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 init_smem(32, 4));
            k_init_nets<Rec16><<<g, kInitWarps * 32, smem, st>>>(d, e_begin, guard); h->launches++;
        } else {
            cudaFuncSetAttribute(k_init_nets<Rec32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 init_smem(64, 4));
            k_init_nets<Rec32><<<g, kInitWarps * 32, smem, st>>>(d, e_begin, guard); h->launches++;
        }
    }
    CK(cudaGetLastError());
    h->next_round = 0;
    h->all_eligible = true;
    return HGP_OK;
}

// Device bytes of every buffer create_impl (and the first refine) allocates for a handle made
// from host inputs of fewer than kHostSizesMaxNets nets, each rounded up to 256 bytes: the arena
// those buffers are carved from.  It covers the direct transpose in input net order without
// wide nets; buffers of any other path (or beyond a miscount) come from the pool instead.
size_t small_handle_bytes(int32_t n, int32_t m, int64_t P, int32_t k, const hgp_options &o, int32_t max_size,
                          bool has_vw, bool has_nw)
{
    auto A = [](int64_t bytes) -> size_t { return (size_t)((bytes < 1 ? 1 : bytes) + 255) / 256 * 256; };
    const int64_t n_ranges = (n + kRange - 1) / kRange, n_tiles = (n_ranges + kWarps - 1) / kWarps;
    const int64_t S = o.subrounds, nm = n > m ? n : m;
    const int w = o.phi_width ? o.phi_width : (max_size <= 255 ? 1 : 2);
    const int64_t nr_ctas = m > 0 ? std::min<int64_t>((m + 2047) / 2048, 1216) : 0;
    const int64_t scan_count = std::max<int64_t>(nm + 1, kNrRanks * nr_ctas + 1);
    const int64_t nb = (scan_count + kScanChunk - 1) / kScanChunk;
    size_t b = 0;
    b += A(8 * (m + 1)) + A(4 * (m + 1)) + A(4 * P) + A(4 * (int64_t)n) + A(4 * 8);   // inputs, flags
    if (has_vw) b += A(4 * (int64_t)n);
    if (has_nw) b += A(4 * (int64_t)m);
    b += A(4 * (nb + 1)) + A(4 * (nm + 1));                                          // scan scratch
    b += A(4 * ((int64_t)n + 1)) + A(4 * P);                                         // vtx_off, inc
    b += A(n) + A(4 * (((int64_t)m * k * w + 3) / 4)) + A((int64_t)m * (k <= 32 ? 16 : 32)) + A(8 * (2 * 64 + 8));
    b += A(n_ranges * kRange) + A(2 * n_ranges * (S + 1)) + A(8 * n_ranges * kRange) + A(4 * n_ranges);
    b += A(8 * 64) + A(8 * (int64_t)k * kBins) + A((int64_t)sizeof(Sel) * 64) + A(8 * (int64_t)k * n_tiles);
    if (o.revert_negative) {
        int64_t cap = 1024;
        while (cap < 2 * P) cap <<= 1;
        b += A(n_ranges * kRange) + A(16) + A(4 * (int64_t)m) + A(cap * kRvSlotBytes);
    }
    b += A(16);                                                                     // round state
    b += A(8 * ST_N * 16 + 4 * kWqPerRow * 16);                                      // statistics
    b += A(sizeof(Dev));                                                            // device Dev
    return b;
}

int create_impl(int32_t n, int32_t m, const int64_t *net_offsets, const int32_t *pins,
                const int32_t *vertex_w, const int32_t *net_w, int32_t k, double eps,
                const int32_t *initial_part, const hgp_options *opt, hgp_handle **out, bool on_device)
{
    if (!out) return HGP_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || m < 0 || !net_offsets || !initial_part || (m > 0 && !pins)) return HGP_ERR_INVALID;
    if (k < 2 || !(eps > 0.0 && eps < 1.0)) return HGP_ERR_INVALID;
    if (k > 64) return HGP_ERR_UNSUPPORTED;
    hgp_options o;
    hgp_default_options(&o);
    if (opt) o = *opt;
    if (o.subrounds == 0) o.subrounds = 4;
    if (o.subrounds < 0) return HGP_ERR_INVALID;
    if (o.subrounds > 64) return HGP_ERR_UNSUPPORTED;
    if (o.phi_width != 0 && o.phi_width != 1 && o.phi_width != 2 && o.phi_width != 4) return HGP_ERR_INVALID;

    int64_t P = 0;
    if (on_device) {
        if (cudaMemcpy(&P, net_offsets + m, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
            (void)cudaGetLastError();
            return HGP_ERR_INVALID;
        }
    } else {
        P = net_offsets[m];
    }
    if (P < 0) return HGP_ERR_INVALID;
    if (P >= ((int64_t)1 << 31)) return HGP_ERR_UNSUPPORTED;

    hgp_handle *h = new (std::nothrow) hgp_handle();
    if (!h) return HGP_ERR_OOM;
    int rc = HGP_OK;
    auto fail = [&](int code) {
        hgp_destroy(h);
        return code;
    };
    Dev &d = h->d;
    cudaGetDevice(&h->device);
    auto release = [&](void *ptr) {   // frees one of the handle's allocations before the end
        if (in_arena(h, ptr)) return;
        for (int i = 0; i < h->n_allocs; ++i)
            if (h->allocs[i] == ptr) {
                dev_free(h->allocs[i], h->stream);
                h->allocs[i] = nullptr;
            }
    };
    if (o.cuda_stream) {
        h->stream = (cudaStream_t)o.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(HGP_ERR_CUDA);
        }
        h->own_stream = true;
    }
    cudaStream_t st = h->stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    h->seed = o.seed;
    h->debug = o.debug;
    if (o.gain_ctas_per_sm < 0 || o.apply_ctas_per_sm < 0) return fail(HGP_ERR_INVALID);
    h->gain_ctas = o.gain_ctas_per_sm;
    h->apply_ctas = o.apply_ctas_per_sm;
    h->graph = o.graph;
    d.n = n;
    d.m = m;
    d.k = k;
    d.P = (int32_t)P;
    d.S = o.subrounds;
    d.n_ranges = (n + kRange - 1) / kRange;
    d.n_tiles = (d.n_ranges + kWarps - 1) / kWarps;

#define CKF(call)                                  \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) {                   \
            (void)cudaGetLastError();              \
            return fail(status_of(_e));            \
        }                                          \
    } while (0)

    // ---- small host inputs: the host checks the offsets and finds the largest net itself
    // (cheaper than a round trip to the device, which waits behind other work on a busy GPU), so
    // the creation is queued to its end without waiting for the device checks: the kernels after
    // them skip flagged input (guard) and the verdict comes with the final read-back.  Their
    // buffers are carved from one allocation (the arena), sized here.
    const bool host_sizes = !on_device && m < kHostSizesMaxNets;
    int32_t max_size = 0;
    if (host_sizes) {
        if (net_offsets[0] != 0) return fail(HGP_ERR_INVALID);
        // branch-free smallest and largest size (vectorisable); offsets checked afterwards
        int64_t lo = 0, hi = 0;
        for (int32_t e = 0; e < m; ++e) {
            const int64_t sz = net_offsets[e + 1] - net_offsets[e];
            lo = sz < lo ? sz : lo;
            hi = sz > hi ? sz : hi;
        }
        if (lo < 0) return fail(HGP_ERR_INVALID);   // then every size is at most P < 2^31
        max_size = (int32_t)hi;
        const size_t bytes = small_handle_bytes(n, m, P, k, o, max_size, vertex_w != nullptr, net_w != nullptr);
        void *a = nullptr;
        if (dev_alloc(&a, bytes, st) == cudaSuccess) {   // else every buffer comes from the pool
            h->allocs[h->n_allocs++] = a;
            h->arena = static_cast<char *>(a);
            h->arena_size = bytes;
        }
    }

    // ---- inputs
    int64_t *off64 = nullptr;
    int32_t *part_in = nullptr, *tmp = nullptr, *misc32 = nullptr;
    int32_t *net_off = nullptr, *pins_d = nullptr, *vw_d = nullptr, *nw_d = nullptr;
    CKF(dalloc(h, &off64, (int64_t)m + 1));
    CKF(dalloc(h, &net_off, (int64_t)m + 1));
    CKF(dalloc(h, &pins_d, P));
    CKF(dalloc(h, &part_in, n));
    CKF(dalloc(h, &misc32, 8));   // err, max net size
    CKF(cudaMemsetAsync(misc32, 0, 8 * sizeof(int32_t), st));
    d.err = misc32;
    int32_t *max_size_d = misc32 + 1;
    CKF(cudaMemcpyAsync(off64, net_offsets, sizeof(int64_t) * ((size_t)m + 1), kind, st));
    if (P) CKF(cudaMemcpyAsync(pins_d, pins, sizeof(int32_t) * (size_t)P, kind, st));
    CKF(cudaMemcpyAsync(part_in, initial_part, sizeof(int32_t) * (size_t)n, kind, st));
    if (vertex_w) {
        CKF(dalloc(h, &vw_d, n));
        CKF(cudaMemcpyAsync(vw_d, vertex_w, sizeof(int32_t) * (size_t)n, kind, st));
    }
    if (net_w) {
        CKF(dalloc(h, &nw_d, m));
        CKF(cudaMemcpyAsync(nw_d, net_w, sizeof(int32_t) * (size_t)m, kind, st));
    }
    d.net_off = net_off;
    d.pins = pins_d;
    d.vw = vw_d;
    d.nw = nw_d;

    // ---- validation
    uint8_t *part = nullptr;
    CKF(dalloc(h, &part, n));
    k_check_inputs<<<grid_for(std::max<int64_t>((int64_t)m + 1, n), 256), 256, 0, st>>>(
        off64, net_off, m, P, nw_d, vw_d, part_in, n, k, part, d.err); h->launches++;
    CKF(cudaGetLastError());
    int32_t host_err[2] = {0, 0};
    // one read-back for both checks: the pin check does nothing when the offsets were bad
    if (m > 0) {
        k_check_pins<<<grid_for(m, 256), 256, 0, st>>>(net_off, pins_d, m, n, d.err, max_size_d); h->launches++;
        CKF(cudaGetLastError());
    }
    const int32_t *guard = nullptr;
    if (host_sizes) {
        guard = d.err;
    } else {
        CKF(cudaMemcpyAsync(host_err, d.err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CKF(stream_wait(st));
        if (host_err[0] & ERR_INVALID) return fail(HGP_ERR_INVALID);
        max_size = host_err[1];
    }

    // ---- scan scratch (shared by the scans below)
    const int64_t nr_ctas = m > 0 ? (m + 2047) / 2048 < 1216 ? (m + 2047) / 2048 : 1216 : 0;
    const int64_t scan_count = std::max((int64_t)(n > m ? n : m) + 1, kNrRanks * nr_ctas + 1);
    const int64_t nb = (scan_count + kScanChunk - 1) / kScanChunk;
    int32_t *block_sums = nullptr;
    CKF(dalloc(h, &block_sums, nb + 1));
    auto scan = [&](const int32_t *in, int32_t *outp, int64_t count) -> cudaError_t {
        const int64_t blocks = (count + kScanChunk - 1) / kScanChunk;
        const int64_t bl = blocks < 1 ? 1 : blocks;
        k_scan_reduce<<<(unsigned)bl, kScanThreads, 0, st>>>(in, count, block_sums); h->launches++;
        k_scan_sums<<<1, kScanThreads, 0, st>>>(block_sums, bl); h->launches++;
        k_scan_final<<<(unsigned)bl, kScanThreads, 0, st>>>(in, outp, count, block_sums); h->launches++;
        return cudaGetLastError();
    };

    // ---- internal net order (largest size class first); the input-order arrays are released
    CKF(dalloc(h, &tmp, (int64_t)(n > m ? n : m) + 1));
    const int64_t avg_size = m > 0 ? (P + m - 1) / m : 0;
    const bool reorder = m > 0 && !(o.debug & 8) &&
                         ((o.debug & 4) || (m >= kReorderMinNets && max_size >= kReorderSkew * avg_size));
    int32_t p_big = 0;   // pins of the large-net prefix
    if (reorder) {
        const int32_t per_cta = (int32_t)((m + nr_ctas - 1) / nr_ctas);
        const int32_t nslots = (int32_t)(kNrRanks * nr_ctas);
        int32_t *cnt = nullptr, *perm = nullptr, *off_int = nullptr, *pins_int = nullptr, *nw_int = nullptr;
        CKF(dev_alloc(reinterpret_cast<void **>(&cnt), sizeof(int32_t) * (2 * (size_t)nslots + 1), st));
        int32_t *base = cnt + nslots;
        CKF(dalloc(h, &perm, m));
        CKF(dalloc(h, &off_int, (int64_t)m + 1));
        if (P) CKF(dalloc(h, &pins_int, P));
        if (nw_d) CKF(dalloc(h, &nw_int, m));
        k_nr_count<<<(unsigned)nr_ctas, kNrThreads, 0, st>>>(net_off, m, per_cta, cnt); h->launches++;
        CKF(scan(cnt, base, nslots));
        int big_rank = 0;   // first rank of the nets below kBigNet pins
        while (((int64_t)1 << (31 - big_rank)) >= kBigNet) ++big_rank;
        int32_t mb = 0;
        CKF(cudaMemcpyAsync(&mb, base + (int64_t)big_rank * nr_ctas, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CKF(stream_wait(st));
        k_nr_place<<<(unsigned)nr_ctas, kNrThreads, 0, st>>>(net_off, m, per_cta, base, perm, tmp); h->launches++;
        CKF(scan(tmp, off_int, m));   // sizes in internal order -> offsets (off_int[m] = P)
        k_nr_pins<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(net_off, pins_d, nw_d, m, perm, off_int,
                                                                  pins_int, nw_int); h->launches++;
        CKF(cudaGetLastError());
        CKF(pool_free(cnt, st));
        CKF(cudaMemcpyAsync(&p_big, off_int + mb, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CKF(stream_wait(st));
        h->m_big = mb;
        h->m_big32 = (int32_t)std::min((int64_t)m, ((int64_t)mb + 31) / 32 * 32);
        release(net_off);
        release(pins_d);
        if (nw_d) release(nw_d);
        net_off = off_int;
        pins_d = pins_int;
        nw_d = nw_int;
        d.net_off = net_off;
        d.pins = pins_d;
        d.nw = nw_d;
        d.net_perm = perm;
    }

    // ---- Phi width chosen by the largest net: 1 byte if every net fits, else 2 bytes; nets
    // beyond the entry's range keep int32 rows in the wide table
    int w = o.phi_width;
    if (w == 0) w = max_size <= 255 ? 1 : 2;
    d.phi_w = w;
    const int32_t narrow_max = w == 1 ? 255 : (w == 2 ? 65535 : 0x7fffffff);

    // ---- wide nets
    if (max_size > narrow_max) {
        int32_t *widx = nullptr;
        CKF(dalloc(h, &widx, (int64_t)m + 1));
        k_wide_flags<<<grid_for(m, 256), 256, 0, st>>>(net_off, m, narrow_max, tmp); h->launches++;
        CKF(scan(tmp, widx, m));
        int32_t nwide = 0;
        CKF(cudaMemcpyAsync(&nwide, widx + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CKF(stream_wait(st));
        h->n_wide = nwide;
        d.widx = widx;
        int32_t *pw = nullptr;
        CKF(dalloc(h, &pw, (int64_t)nwide * k));
        CKF(cudaMemsetAsync(pw, 0, sizeof(int32_t) * (size_t)nwide * k, st));
        d.phi_wide = pw;
    }

    // ---- vertex -> nets CSR (bucketed transpose; the wide flag goes into inc on the way)
    int32_t *vtx_off = nullptr, *inc = nullptr;
    CKF(dalloc(h, &vtx_off, (int64_t)n + 1));
    CKF(dalloc(h, &inc, P));
    CKF(cudaMemsetAsync(tmp, 0, sizeof(int32_t) * ((size_t)n + 1), st));
    if (P > 0 && n <= kTpDirectMaxN && !(o.debug & 2)) {
        k_degrees<<<grid_for(P, 256), 256, 0, st>>>(pins_d, P, tmp, guard); h->launches++;
        CKF(scan(tmp, vtx_off, n));
        CKF(cudaMemcpyAsync(tmp, vtx_off, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        k_scatter<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(net_off, pins_d, m, narrow_max, tmp, inc, guard);
        h->launches++;
        CKF(cudaGetLastError());
    } else if (P > 0) {
        auto buckets = [&](int sh) { return (((int64_t)n + ((int64_t)1 << sh) - 1) >> sh); };
        int bshift = kTpShift;
        while (bshift > kTpMinShift && buckets(bshift) < kTpMinCtas) --bshift;
        while (buckets(bshift) > kTpMaxBuckets) ++bshift;
        const int32_t nbk = (int32_t)buckets(bshift);
        const int32_t e_begin = h->m_big;   // the large-net prefix goes to k_tp_scatter_big
        const int64_t m_rest = (int64_t)m - e_begin;
        int64_t per_cta = (m_rest + kTpMinCtas - 1) / kTpMinCtas;
        per_cta = per_cta < 512 ? 512 : (per_cta > kTpNetsPerCta ? kTpNetsPerCta : per_cta);
        int32_t *bk = nullptr;           // counts [nbk + 1], offsets [nbk + 1], cursors [nbk]
        unsigned long long *pairs = nullptr;
        CKF(dev_alloc(reinterpret_cast<void **>(&bk), sizeof(int32_t) * (3 * (size_t)nbk + 2), st));
        CKF(dev_alloc(reinterpret_cast<void **>(&pairs), sizeof(unsigned long long) * (size_t)P, st));
        int32_t *bk_cnt = bk, *bk_off = bk + nbk + 1, *bk_cur = bk + 2 * nbk + 2;
        CKF(cudaMemsetAsync(bk_cnt, 0, sizeof(int32_t) * ((size_t)nbk + 1), st));
        k_tp_hist<<<grid_for(P, 256, 152 * 8), 256, 0, st>>>(pins_d, P, bshift, nbk, bk_cnt, guard); h->launches++;
        CKF(scan(bk_cnt, bk_off, nbk));
        CKF(cudaMemcpyAsync(bk_cur, bk_off, sizeof(int32_t) * (size_t)nbk, cudaMemcpyDeviceToDevice, st));
        const int64_t sc = (m_rest + per_cta - 1) / per_cta;
        if (e_begin > 0 && p_big > 0) {
            k_tp_scatter_big<<<(unsigned)((p_big + kTpBigChunk - 1) / kTpBigChunk), 256, 0, st>>>(
                net_off, pins_d, e_begin, bshift, nbk, narrow_max, bk_cur, pairs, guard); h->launches++;
        }
        if (sc > 0) {
            k_tp_scatter<<<(unsigned)sc, 256, 0, st>>>(net_off, pins_d, m, e_begin, bshift, nbk, narrow_max,
                                                       (int32_t)per_cta, bk_cur, pairs, guard); h->launches++;
        }
        if (bshift <= kTpSmemShift) {
            const int smem = (int)(sizeof(int32_t) << bshift);
            cudaFuncSetAttribute(k_tp_place<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(int32_t) << kTpSmemShift));   // largest need, as above
            k_tp_place<true><<<nbk, 1024, smem, st>>>(pairs, bk_off, bshift, n, nbk, tmp, vtx_off, inc, guard);
        } else {
            k_tp_place<false><<<nbk, 1024, 0, st>>>(pairs, bk_off, bshift, n, nbk, tmp, vtx_off, inc, guard);
        }
        h->launches++;
        CKF(cudaGetLastError());
        CKF(pool_free(pairs, st));
        CKF(pool_free(bk, st));
    } else {
        CKF(cudaMemsetAsync(vtx_off, 0, sizeof(int32_t) * ((size_t)n + 1), st));
    }
    d.vtx_off = vtx_off;
    d.inc = inc;

    unsigned long long *maxw_d = reinterpret_cast<unsigned long long *>(misc32 + 2);   // zeroed with misc32
    // the result of this check is read with the block weights at the end (nothing in between
    // depends on it)
    k_vertex_netweight<<<grid_for(n, 256), 256, 0, st>>>(vtx_off, inc, nw_d, n, d.err, maxw_d); h->launches++;
    CKF(cudaGetLastError());

    // ---- state (Pi was stored by the input check)
    d.part = part;
    const int64_t entries = (int64_t)m * k;
    const int64_t words = (entries * w + 3) / 4;
    uint32_t *phi = nullptr;
    CKF(dalloc(h, &phi, words));
    d.phi = phi;   // zeroed by init_state
    const size_t rec_bytes = k <= 32 ? sizeof(Rec16) : sizeof(Rec32);
    uint4 *rec = nullptr;
    CKF(dalloc(h, &rec, (int64_t)m * (int64_t)(rec_bytes / 16)));
    d.rec = rec;
    int64_t *small = nullptr;
    CKF(dalloc(h, &small, 2 * 64 + 8));
    d.bw = small;
    d.obj = small + 64;

    // ---- per-sub-round scratch
    uint8_t *sub_list = nullptr;
    uint16_t *sub_start = nullptr;
    uint64_t *cand = nullptr;
    int32_t *cand_cnt = nullptr;
    int64_t *tot = nullptr, *tie = nullptr;
    unsigned long long *hist = nullptr;
    Sel *sel = nullptr;
    CKF(dalloc(h, &sub_list, (int64_t)d.n_ranges * kRange));
    CKF(dalloc(h, &sub_start, (int64_t)d.n_ranges * (d.S + 1)));
    CKF(dalloc(h, &cand, (int64_t)d.n_ranges * kRange));
    CKF(dalloc(h, &cand_cnt, d.n_ranges));
    CKF(dalloc(h, &tot, 64));
    CKF(dalloc(h, &hist, (int64_t)k * kBins));
    CKF(dalloc(h, &sel, 64));
    CKF(dalloc(h, &tie, (int64_t)k * d.n_tiles));
    CKF(cudaMemsetAsync(tot, 0, sizeof(int64_t) * 64, st));
    CKF(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (size_t)k * kBins, st));
    d.sub_list = sub_list;
    d.sub_start = sub_start;
    d.cand = cand;
    d.cand_cnt = cand_cnt;
    d.tot = tot;
    d.hist = hist;
    d.sel = sel;
    d.tie = tie;
    if (o.revert_negative) {
        // per candidate slot source blocks, and a table with room for the two (net, block)
        // keys of every incidence of a sub-round's movers (at most 2 P keys)
        uint8_t *rv_src = nullptr;
        unsigned long long *rv_cnt = nullptr;
        int64_t cap = 1024;
        while (cap < 2 * (int64_t)P) cap <<= 1;
        int32_t *rv_net = nullptr;
        CKF(dalloc(h, &rv_src, (int64_t)d.n_ranges * kRange));
        CKF(dalloc(h, &rv_cnt, 2));
        CKF(dalloc(h, &rv_net, m));
        CKF(dalloc(h, reinterpret_cast<uint4 **>(&d.rv_tab), cap * kRvSlotBytes / 16));
        CKF(cudaMemsetAsync(rv_cnt, 0, 2 * sizeof(unsigned long long), st));
        d.rv_net = rv_net;
        d.rv_src = rv_src;
        d.rv_cnt = rv_cnt;
        d.rv_cap = cap;
    }
    CKF(dalloc(h, &h->d_round, 4));
    d.rs = h->d_round;
    d.seed = o.seed;
    d.variant = (o.balance_moves ? 1 : 0) | (o.revert_negative ? 2 : 0);

    rc = init_state(h, guard);
    if (rc != HGP_OK) return fail(rc);

    // ---- L_max = floor((1 + eps) * ceil(c(V) / k))  (Sec. 2); the incident-weight check
    int64_t bw[64];
    unsigned long long maxw = 0;
    CKF(cudaMemcpyAsync(bw, d.bw, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, st));
    CKF(cudaMemcpyAsync(host_err, d.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CKF(cudaMemcpyAsync(&maxw, maxw_d, sizeof(maxw), cudaMemcpyDeviceToHost, st));
    CKF(stream_wait(st));
    if (host_err[0] & ERR_INVALID) return fail(HGP_ERR_INVALID);
    if (host_err[0] & ERR_UNSUPPORTED) return fail(HGP_ERR_UNSUPPORTED);
    h->max_vertex_netweight = (int64_t)maxw;
    int64_t total = 0;
    for (int i = 0; i < k; ++i) total += bw[i];
    h->total_weight = total;
    const int64_t avg = (total + k - 1) / k;
    d.lmax = (int64_t)floor((1.0 + eps) * (double)avg);

    // the int64 offsets and the int32 partition copy are no longer needed
    for (int i = 0; i < h->n_allocs; ++i) {
        if (h->allocs[i] && !in_arena(h, h->allocs[i]) &&
            (h->allocs[i] == off64 || h->allocs[i] == part_in || h->allocs[i] == block_sums ||
             h->allocs[i] == tmp)) {
            dev_free(h->allocs[i], st);
            h->allocs[i] = nullptr;
        }
    }
    if (in_arena(h, tmp)) h->scratch_n = tmp;   // max(n, m) + 1 entries, free from here on
    rc = ensure_stats(h, 16);
    if (rc != HGP_OK) return fail(rc);
    // the event a batch records its end on (see settle); made here, on the creating thread
    CKF(cudaEventCreateWithFlags(&h->ev_batch, cudaEventDisableTiming));
    *out = h;
    return HGP_OK;
#undef CKF
}

}  // namespace

// ================================================================== C ABI
extern "C" {

void hgp_default_options(hgp_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->subrounds = 4;
}

int hgp_set_blocking_waits(int32_t on)
{
    hgp::g_blocking_waits.store(on ? 1 : 0, std::memory_order_relaxed);
    return HGP_OK;
}

int hgp_set_pool_retention(int64_t bytes)
{
    if (bytes < 0) return HGP_ERR_INVALID;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = hgp::library_pool(&pool);
    uint64_t v = (uint64_t)bytes;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &v);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    return HGP_OK;
}

const char *hgp_strerror(int code)
{
    switch (code) {
    case HGP_OK: return "ok";
    case HGP_ERR_INVALID: return "invalid argument";
    case HGP_ERR_OOM: return "out of memory";
    case HGP_ERR_UNSUPPORTED: return "unsupported size or parameter";
    case HGP_ERR_CUDA: return "CUDA error";
    case HGP_ERR_TIMEOUT: return "device wait timed out";
    case HGP_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status";
    }
}

int hgp_create(int32_t n, int32_t m, const int64_t *net_offsets, const int32_t *pins,
               const int32_t *vertex_w, const int32_t *net_w, int32_t k, double eps,
               const int32_t *initial_part, const hgp_options *opt, hgp_handle **out)
{
    return create_impl(n, m, net_offsets, pins, vertex_w, net_w, k, eps, initial_part, opt, out, false);
}

int hgp_create_device(int32_t n, int32_t m, const int64_t *net_offsets, const int32_t *pins,
                      const int32_t *vertex_w, const int32_t *net_w, int32_t k, double eps,
                      const int32_t *initial_part, const hgp_options *opt, hgp_handle **out)
{
    return create_impl(n, m, net_offsets, pins, vertex_w, net_w, k, eps, initial_part, opt, out, true);
}

// Releases are queued on the handle's stream behind its pending work (and behind the batch
// work that hgp_batch_refine ordered before it), so the call does not wait for the device.
void hgp_destroy(hgp_handle *h)
{
    if (!h) return;
    settle(h);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    for (int i = 0; i < h->n_allocs; ++i)
        if (h->allocs[i]) dev_free(h->allocs[i], h->stream);
    for (int32_t i = 0; i < h->n_events; ++i) cudaEventDestroy(h->events[i]);
    if (h->ev_batch) cudaEventDestroy(h->ev_batch);
    delete[] h->events;
    delete[] h->event_phase;
    delete[] h->event_count;
    if (h->d.stats && !in_arena(h, h->d.stats)) dev_free(h->d.stats, h->stream);
    if (h->d_dev && !in_arena(h, h->d_dev)) dev_free(h->d_dev, h->stream);
    free(h->h_stats);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    (void)cudaGetLastError();
    delete h;
}

int hgp_set_partition(hgp_handle *h, const int32_t *part, int32_t on_device)
{
    if (!h || !part) return HGP_ERR_INVALID;
    settle(h);
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    int32_t *tmp = h->scratch_n;
    if (!tmp) CK(dev_alloc(reinterpret_cast<void **>(&tmp), sizeof(int32_t) * (size_t)d.n, st));
    int rc = HGP_OK;
    int32_t err = 0;
    cudaError_t e = cudaMemcpyAsync(tmp, part, sizeof(int32_t) * (size_t)d.n,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) {
        k_check_vertices<<<grid_for(d.n, 256), 256, 0, st>>>(nullptr, tmp, d.n, d.k, d.err); h->launches++;
        e = cudaMemcpyAsync(&err, d.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = stream_wait(st);
    if (e == cudaSuccess && (err & ERR_INVALID)) rc = HGP_ERR_INVALID;
    if (e == cudaSuccess && rc == HGP_OK) {
        k_copy_part<<<grid_for(d.n, 256), 256, 0, st>>>(tmp, d.part, d.n); h->launches++;
        e = cudaGetLastError();
    }
    if (tmp != h->scratch_n) pool_free(tmp, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    if (rc != HGP_OK) return rc;
    return init_state(h, nullptr);
}

int hgp_export_state(hgp_handle *h, int32_t *part, uint8_t *moved_nets, int64_t *next_round,
                     int32_t *first_round)
{
    if (!h) return HGP_ERR_INVALID;
    settle(h);
    if (part) {
        const int rc = hgp_get_partition(h, part, 0);
        if (rc != HGP_OK) return rc;
    }
    if (moved_nets && h->d.m > 0) {
        Dev &d = h->d;
        uint8_t *tmp = nullptr;
        CK(dev_alloc(reinterpret_cast<void **>(&tmp), (size_t)d.m, h->stream));
        if (d.k <= 32)
            k_export_moved<Rec16><<<grid_for(d.m, 256), 256, 0, h->stream>>>(d, (int32_t)h->next_round,
                                                                             h->all_eligible ? 1 : 0, tmp);
        else
            k_export_moved<Rec32><<<grid_for(d.m, 256), 256, 0, h->stream>>>(d, (int32_t)h->next_round,
                                                                             h->all_eligible ? 1 : 0, tmp);
        h->launches++;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(moved_nets, tmp, (size_t)d.m, cudaMemcpyDeviceToHost, h->stream);
        pool_free(tmp, h->stream);
        if (e == cudaSuccess) e = stream_wait(h->stream);
        CK(e);
    }
    if (next_round) *next_round = h->next_round;
    if (first_round) *first_round = h->all_eligible ? 1 : 0;
    return HGP_OK;
}

int hgp_import_state(hgp_handle *h, const int32_t *part, const uint8_t *moved_nets,
                     int64_t next_round, int32_t first_round)
{
    if (!h || !part || next_round < 0 || next_round >= ((int64_t)1 << 30)) return HGP_ERR_INVALID;
    settle(h);
    if (!first_round && !moved_nets && h->d.m > 0) return HGP_ERR_INVALID;
    int rc = hgp_set_partition(h, part, 0);
    if (rc != HGP_OK) return rc;
    Dev &d = h->d;
    const int32_t r = (int32_t)next_round;
    if (!first_round && d.m > 0) {
        uint8_t *tmp = nullptr;
        CK(dev_alloc(reinterpret_cast<void **>(&tmp), (size_t)d.m, h->stream));
        cudaError_t e = cudaMemcpyAsync(tmp, moved_nets, (size_t)d.m, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) {
            if (d.k <= 32) k_import_moved<Rec16><<<grid_for(d.m, 256), 256, 0, h->stream>>>(d, r, tmp);
            else k_import_moved<Rec32><<<grid_for(d.m, 256), 256, 0, h->stream>>>(d, r, tmp);
            h->launches++;
            e = cudaGetLastError();
        }
        pool_free(tmp, h->stream);
        if (e == cudaSuccess) e = stream_wait(h->stream);
        CK(e);
    }
    k_set_round_state<<<1, 32, 0, h->stream>>>(d.rs, r, first_round ? 0 : 1);
    h->launches++;
    CK(cudaGetLastError());
    CK(stream_wait(h->stream));
    h->next_round = next_round;
    h->all_eligible = first_round != 0;
    return HGP_OK;
}

int hgp_objective(hgp_handle *h, int64_t *out)
{
    if (!h || !out) return HGP_ERR_INVALID;
    settle(h);
    CK(cudaMemcpyAsync(out, h->d.obj, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    CK(stream_wait(h->stream));
    return HGP_OK;
}

int hgp_objective_from_phi(hgp_handle *h, int64_t *out)
{
    if (!h || !out) return HGP_ERR_INVALID;
    settle(h);
    unsigned long long *tmp = nullptr;
    CK(dev_alloc(reinterpret_cast<void **>(&tmp), sizeof(*tmp), h->stream));
    cudaError_t e = objective_from_phi(h, reinterpret_cast<int64_t *>(tmp));
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream);
    pool_free(tmp, h->stream);
    if (e == cudaSuccess) e = stream_wait(h->stream);
    CK(e);
    return HGP_OK;
}

int hgp_get_partition(hgp_handle *h, int32_t *part, int32_t on_device)
{
    if (!h || !part) return HGP_ERR_INVALID;
    settle(h);
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    if (on_device) {
        k_part_to_i32<<<grid_for(d.n, 256), 256, 0, st>>>(d.part, part, d.n); h->launches++;
        CK(cudaGetLastError());
        CK(stream_wait(st));
        return HGP_OK;
    }
    int32_t *tmp = h->scratch_n;
    if (!tmp) CK(dev_alloc(reinterpret_cast<void **>(&tmp), sizeof(int32_t) * (size_t)d.n, st));
    k_part_to_i32<<<grid_for(d.n, 256), 256, 0, st>>>(d.part, tmp, d.n); h->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(part, tmp, sizeof(int32_t) * (size_t)d.n, cudaMemcpyDeviceToHost, st);
    if (tmp != h->scratch_n) pool_free(tmp, st);
    if (e == cudaSuccess) e = stream_wait(st);
    CK(e);
    return HGP_OK;
}

int hgp_get_block_weights(hgp_handle *h, int64_t *w)
{
    if (!h || !w) return HGP_ERR_INVALID;
    settle(h);
    CK(cudaMemcpyAsync(w, h->d.bw, sizeof(int64_t) * h->d.k, cudaMemcpyDeviceToHost, h->stream));
    CK(stream_wait(h->stream));
    return HGP_OK;
}

int hgp_get_phi(hgp_handle *h, int32_t *phi)
{
    if (!h || !phi) return HGP_ERR_INVALID;
    settle(h);
    Dev &d = h->d;
    const int64_t total = (int64_t)d.m * d.k;
    if (total == 0) return HGP_OK;
    int32_t *tmp = nullptr;
    CK(dev_alloc(reinterpret_cast<void **>(&tmp), sizeof(int32_t) * (size_t)total, h->stream));
    k_widen_phi<<<grid_for(total, 256), 256, 0, h->stream>>>(d, tmp); h->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(phi, tmp, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToHost, h->stream);
    pool_free(tmp, h->stream);
    if (e == cudaSuccess) e = stream_wait(h->stream);
    CK(e);
    return HGP_OK;
}

int hgp_get_lambda(hgp_handle *h, uint64_t *lam)
{
    if (!h || !lam) return HGP_ERR_INVALID;
    settle(h);
    Dev &d = h->d;
    if (d.m == 0) return HGP_OK;
    uint64_t *tmp = nullptr;
    CK(dev_alloc(reinterpret_cast<void **>(&tmp), sizeof(uint64_t) * (size_t)d.m, h->stream));
    if (d.k <= 32) { k_get_lambda<Rec16><<<grid_for(d.m, 256), 256, 0, h->stream>>>(d, tmp); h->launches++; }
    else { k_get_lambda<Rec32><<<grid_for(d.m, 256), 256, 0, h->stream>>>(d, tmp); h->launches++; }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam, tmp, sizeof(uint64_t) * (size_t)d.m, cudaMemcpyDeviceToHost, h->stream);
    pool_free(tmp, h->stream);
    if (e == cudaSuccess) e = stream_wait(h->stream);
    CK(e);
    return HGP_OK;
}

int hgp_get_info(hgp_handle *h, int32_t *n, int32_t *m, int32_t *k, int64_t *pins, int64_t *lmax,
                 int32_t *phi_width, int32_t *wide_nets, int64_t *next_round)
{
    if (!h) return HGP_ERR_INVALID;
    if (n) *n = h->d.n;
    if (m) *m = h->d.m;
    if (k) *k = h->d.k;
    if (pins) *pins = h->d.P;
    if (lmax) *lmax = h->d.lmax;
    if (phi_width) *phi_width = h->d.phi_w;
    if (wide_nets) *wide_nets = h->n_wide;
    if (next_round) *next_round = h->next_round;
    return HGP_OK;
}

int hgp_refine(hgp_handle *h, int32_t rounds, hgp_round_stats *stats)
{
    if (!h || rounds < 0) return HGP_ERR_INVALID;
    settle(h);
    return refine_rounds(h, rounds, stats);
}

int hgp_debug_candidates(hgp_handle *h, int32_t s, int32_t *target, int64_t *gain)
{
    if (!h || !target || !gain || s < 0 || s >= h->d.S) return HGP_ERR_INVALID;
    settle(h);
    return debug_candidates(h, s, target, gain);
}

}  // extern "C"

namespace hgp {

cudaError_t objective_from_phi(hgp_handle *h, int64_t *d_out)
{
    cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(int64_t), h->stream);
    if (e != cudaSuccess) return e;
    k_obj_from_phi<<<grid_for(h->d.m, 256), 256, 0, h->stream>>>(h->d, reinterpret_cast<unsigned long long *>(d_out)); h->launches++;
    return cudaGetLastError();
}

}  // namespace hgp

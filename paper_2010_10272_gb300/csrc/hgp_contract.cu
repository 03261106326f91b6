// libhgp: contraction of a vertex clustering into a coarse hypergraph (paper Sec. 3.2).
//
//   1. used cluster ids flagged and remapped to 0..n'-1 by an exclusive prefix sum;
//   2. coarse vertex weights by atomic adds (checked to fit int32);
//   3. every net's pins mapped to coarse ids, sorted and de-duplicated by size class: a thread
//      per net of at most 8 pins (sorting network in registers), a warp per net of 9..32 (bitonic
//      across the lanes), a CTA per net of 33..2048 (bitonic in shared memory), and for larger
//      nets 2048-pin chunks sorted by separate CTAs and merged pairwise by merge-path tiles
//      spread over the whole grid; the net's fingerprint is taken during the de-duplication;
//   4. nets with fewer than two pins dropped; identical nets found through a 64-bit
//      fingerprint table (key -> smallest net id) and an exact comparison with that net; a
//      net that only shares the fingerprint stays unresolved and takes part in the next round
//      (each round resolves the smallest net of every remaining fingerprint group);
//   5. the representatives (smallest id of each identical group) keep their original order;
//      their weights are the sums over the group; offsets by prefix sums.
// Everything is integer and the output is unique: pins sorted inside each net, nets ordered by
// their smallest original id.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "hgp_host.cuh"

using namespace hgp;

struct hgp_coarse {
    int32_t fine_n = 0, n = 0, m = 0;
    int64_t P = 0;
    int64_t *net_off = nullptr;   // device [m+1]
    int32_t *pins = nullptr;      // device [P]
    int32_t *vw = nullptr;        // device [n]
    int32_t *nw = nullptr;        // device [m]
    int32_t *map = nullptr;       // device [fine_n]
    cudaStream_t stream = nullptr;
    int device = 0;
};

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanTile = 1024;
constexpr int kSortThreads = 256;
constexpr unsigned long long kKeyEmpty = ~0ull;
constexpr int32_t kUnresolved = -2, kDropped = -1;

int grid_of(int64_t work, int threads)
{
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return (int)g;
}

// ---------------------------------------------------------------- device-wide exclusive scan
// out[0..len] = exclusive prefix sums of in[0..len-1] (out[len] = total)
template <typename T>
__global__ void __launch_bounds__(kScanTile) k_scan_tile(const T *in, int64_t len, int64_t *out, int64_t *sums)
{
    __shared__ int64_t wt[32];
    const int64_t i = blockIdx.x * (int64_t)kScanTile + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t v = i < len ? (int64_t)in[i] : 0;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int64_t t = wt[lane];
        int64_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        wt[lane] = s - t;
        if (lane == 31) sums[blockIdx.x] = s;
    }
    __syncthreads();
    if (i <= len) out[i] = wt[wid] + x - v;
}

__global__ void k_scan_add(int64_t *out, int64_t len, const int64_t *block_prefix)
{
    const int64_t i = blockIdx.x * (int64_t)kScanTile + threadIdx.x;
    if (i <= len) out[i] += block_prefix[blockIdx.x];
}

// exclusive scan with the total at out[len]; out has len + 1 entries
template <typename T>
cudaError_t scan_excl(const T *in, int64_t len, int64_t *out, cudaStream_t st)
{
    const int64_t tiles = len / kScanTile + 1;   // covers indices 0..len
    int64_t *sums = nullptr, *pref = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&sums), sizeof(int64_t) * (size_t)tiles, st);
    if (e != cudaSuccess) return e;
    k_scan_tile<T><<<(unsigned)tiles, kScanTile, 0, st>>>(in, len, out, sums);
    e = cudaGetLastError();
    if (e == cudaSuccess && tiles > 1) {
        e = dev_alloc(reinterpret_cast<void **>(&pref), sizeof(int64_t) * (size_t)(tiles + 1), st);
        if (e == cudaSuccess) e = scan_excl<int64_t>(sums, tiles, pref, st);
        if (e == cudaSuccess) {
            k_scan_add<<<(unsigned)tiles, kScanTile, 0, st>>>(out, len, pref);
            e = cudaGetLastError();
        }
        if (pref) pool_free(pref, st);
    }
    pool_free(sums, st);
    return e;
}

// ---------------------------------------------------------------- input checks
// offsets non-decreasing from 0 to P, pins in [0, n), weights >= 1
__global__ void k_ct_check(const int64_t *off, const int32_t *pins, const int32_t *vw, const int32_t *nw,
                           int32_t n, int32_t m, int64_t P, int32_t *err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t e = t; e < m; e += stride) {
        if (off[e] < 0 || off[e] > off[e + 1] || off[e + 1] > P || (e == 0 && off[0] != 0)) atomicOr(err, ERR_INVALID);
        if (nw && nw[e] < 1) atomicOr(err, ERR_INVALID);
    }
    for (int64_t j = t; j < P; j += stride)
        if (pins[j] < 0 || pins[j] >= n) atomicOr(err, ERR_INVALID);
    if (vw)
        for (int64_t u = t; u < n; u += stride)
            if (vw[u] < 1) atomicOr(err, ERR_INVALID);
}

// ---------------------------------------------------------------- clusters and weights
__global__ void k_ct_flag(const int32_t *cluster, int32_t n, int32_t *used, int32_t *err)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cluster[u];
        if (c < 0 || c >= n) atomicOr(err, ERR_INVALID);
        else used[c] = 1;
    }
}

__global__ void k_ct_map(const int32_t *cluster, int32_t n, const int64_t *cid, const int32_t *vw,
                         int32_t *map, unsigned long long *w64)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = (int32_t)cid[cluster[u]];
        map[u] = c;
        atomicAdd(&w64[c], (unsigned long long)(vw ? vw[u] : 1));
    }
}

__global__ void k_ct_narrow(const unsigned long long *w64, int64_t len, int32_t *out, int32_t *err)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long w = w64[i];
        if (w >= (1ull << 31)) atomicOr(err, ERR_UNSUPPORTED);
        out[i] = (int32_t)w;
    }
}

// ---------------------------------------------------------------- per-net sort + dedupe
// Fingerprint of a sorted, de-duplicated pin list: the sum of a 64-bit mix of every pin
// (independent of how the pins are split over threads), mixed with the list's length.
__device__ __forceinline__ unsigned long long pin_mix(int32_t v)
{
    return splitmix64_output(0x6a09e667f3bcc908ull ^ (uint64_t)(uint32_t)v);
}

__device__ __forceinline__ unsigned long long key_final(unsigned long long h, int32_t s)
{
    const unsigned long long k = splitmix64_output(h ^ ((uint64_t)(uint32_t)s << 32));
    return k == kKeyEmpty ? k - 1 : k;
}

// result of one net: its de-duplicated size, and its fingerprint (or dropped, < 2 pins)
__device__ __forceinline__ void net_done(int64_t e, int32_t kept, unsigned long long h, int32_t *size1,
                                         unsigned long long *key, int32_t *rep)
{
    size1[e] = kept;
    if (kept < 2) {
        rep[e] = kDropped;
    } else {
        key[e] = key_final(h, kept);
        rep[e] = kUnresolved;
    }
}

constexpr int kTiny = 8, kMid = 256, kMedium = 2048;
constexpr int kClasses = 4;   // listed classes: 9..32, 33..kMid, kMid+1..kMedium, larger

// thread per net: nets of at most kTiny pins are sorted in registers (an unrolled sorting
// network), de-duplicated and fingerprinted; larger nets go to the lists of the warp-register
// (9..32 pins), warp shared-memory (..kMid), CTA shared-memory (..kMedium) and chunked (larger)
// kernels
__global__ void k_ct_tiny(const int64_t *off, const int32_t *pins, int32_t m, const int32_t *map, int32_t *a,
                          int32_t *size1, unsigned long long *key, int32_t *rep, int32_t *lists, int32_t *counts)
{
    const int lane = threadIdx.x & 31;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x; e0 < m; e0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = e0 + threadIdx.x;
        int cls = -1;
        if (e < m) {
            const int64_t b = off[e];
            const int32_t s = (int32_t)(off[e + 1] - b);
            if (s <= kTiny) {
                int32_t v[kTiny];
#pragma unroll
                for (int i = 0; i < kTiny; ++i) v[i] = i < s ? map[pins[b + i]] : 0x7fffffff;
#pragma unroll
                for (int i = 1; i < kTiny; ++i) {
#pragma unroll
                    for (int j = i; j > 0; --j) {
                        const int32_t lo = min(v[j - 1], v[j]), hi = max(v[j - 1], v[j]);
                        v[j - 1] = lo;
                        v[j] = hi;
                    }
                }
                int32_t kept = 0;
                unsigned long long h = 0;
#pragma unroll
                for (int i = 0; i < kTiny; ++i) {
                    if (i < s && (i == 0 || v[i] != v[i - 1])) {
                        a[b + kept] = v[i];
                        h += pin_mix(v[i]);
                        ++kept;
                    }
                }
                net_done(e, kept, h, size1, key, rep);
            } else {
                cls = s <= 32 ? 0 : (s <= kMid ? 1 : (s <= kMedium ? 2 : 3));
            }
        }
        // warp-aggregated append of the larger nets to their class lists
#pragma unroll
        for (int c = 0; c < kClasses; ++c) {
            const unsigned mk = __ballot_sync(kFull, cls == c);
            if (!mk) continue;
            int32_t base = 0;
            if (lane == __ffs(mk) - 1) base = atomicAdd(&counts[c], __popc(mk));
            base = __shfl_sync(kFull, base, __ffs(mk) - 1);
            if (cls == c) lists[(int64_t)c * m + base + __popc(mk & ((1u << lane) - 1))] = (int32_t)e;
        }
    }
}

// warp per listed net of 9..32 pins: bitonic sort across the lanes, de-duplication, fingerprint
__global__ void k_ct_small(const int64_t *off, const int32_t *pins, const int32_t *map, const int32_t *list,
                           const int32_t *count, int32_t *a, int32_t *size1, unsigned long long *key, int32_t *rep)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int32_t cnt = *count;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < cnt; i += warps) {
        const int64_t e = list[i];
        const int64_t b = off[e];
        const int32_t s = (int32_t)(off[e + 1] - b);
        int32_t v = lane < s ? map[pins[b + lane]] : 0x7fffffff;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int32_t o = __shfl_xor_sync(kFull, v, j);
                const bool up = (lane & k) == 0;            // ascending run of the merge
                const bool low = (lane & j) == 0;           // lower partner of the pair
                v = (low == up) ? min(v, o) : max(v, o);
            }
        }
        const int32_t prev = __shfl_up_sync(kFull, v, 1);
        const bool keep = lane < s && (lane == 0 || v != prev);
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) a[b + __popc(km & ((1u << lane) - 1))] = v;
        unsigned long long h = keep ? pin_mix(v) : 0ull;
        for (int o = 16; o; o >>= 1) h += __shfl_xor_sync(kFull, h, o);
        if (lane == 0) net_done(e, __popc(km), h, size1, key, rep);
    }
}

// warp per listed net of 33..kMid pins: bitonic sort in the warp's shared buffer (padded to a
// power of two), then an order-preserving compaction 32 values at a time, and the fingerprint
__global__ void __launch_bounds__(256) k_ct_mid(const int64_t *off, const int32_t *pins, const int32_t *map,
                                                const int32_t *list, const int32_t *count, int32_t *a,
                                                int32_t *size1, unsigned long long *key, int32_t *rep)
{
    __shared__ int32_t buf_w[8][kMid];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *buf = buf_w[wid];
    const int64_t warps = (int64_t)gridDim.x * 8;
    const int32_t cnt = *count;
    for (int64_t i = (int64_t)blockIdx.x * 8 + wid; i < cnt; i += warps) {
        const int64_t e = list[i];
        const int64_t b = off[e];
        const int32_t s = (int32_t)(off[e + 1] - b);
        int32_t np2 = 64;
        while (np2 < s) np2 <<= 1;
        for (int32_t j = lane; j < np2; j += 32) buf[j] = j < s ? map[pins[b + j]] : 0x7fffffff;
        __syncwarp();
        for (int32_t k = 2; k <= np2; k <<= 1) {
            for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
                for (int32_t x = lane; x < np2; x += 32) {
                    const int32_t y = x ^ jj;
                    if (y > x) {
                        const bool up = (x & k) == 0;
                        const int32_t vx = buf[x], vy = buf[y];
                        if ((vx > vy) == up) { buf[x] = vy; buf[y] = vx; }
                    }
                }
                __syncwarp();
            }
        }
        int32_t kept = 0;
        unsigned long long h = 0;
        for (int32_t c = 0; c < s; c += 32) {
            const int32_t j = c + lane;
            const bool has = j < s;
            const int32_t v = has ? buf[j] : 0;
            const bool keep = has && (j == 0 || v != buf[j - 1]);
            const unsigned km = __ballot_sync(kFull, keep);
            if (keep) {
                a[b + kept + __popc(km & ((1u << lane) - 1))] = v;
                h += pin_mix(v);
            }
            kept += __popc(km);
        }
        for (int o = 16; o; o >>= 1) h += __shfl_xor_sync(kFull, h, o);
        if (lane == 0) net_done(e, kept, h, size1, key, rep);
        __syncwarp();
    }
}

// block-wide: order-preserving compaction of the first of every run of equal values of the
// sorted src[0..s) into dst (dst may equal src), fingerprint of the kept values
__device__ __forceinline__ void compact_runs(const int32_t *src, int32_t *dst, int32_t s, int32_t *wtot,
                                             unsigned long long *hsum, int32_t &kept_out, unsigned long long &h_out)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = blockDim.x >> 5;
    int32_t kept = 0;
    if (tid == 0) *hsum = 0;
    for (int32_t t0 = 0; t0 < s; t0 += blockDim.x) {
        const int32_t j = t0 + tid;
        const bool has = j < s;
        const int32_t v = has ? src[j] : 0;
        const bool keep = has && (j == 0 || v != src[j - 1]);
        const unsigned km = __ballot_sync(kFull, keep);
        if (lane == 0) wtot[wid] = __popc(km);
        __syncthreads();
        int32_t before = kept, tile_total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) before += wtot[w];
            tile_total += wtot[w];
        }
        __syncthreads();   // every thread has read its input and the counts
        if (keep) dst[before + __popc(km & ((1u << lane) - 1))] = v;
        if (km) {
            unsigned long long h = keep ? pin_mix(v) : 0ull;
            for (int o = 16; o; o >>= 1) h += __shfl_xor_sync(kFull, h, o);
            if (lane == 0) atomicAdd(hsum, h);
        }
        kept += tile_total;
        __syncthreads();
    }
    kept_out = kept;
    h_out = *hsum;
}

// CTA per listed net of kMid+1..kMedium pins: bitonic sort of the mapped pins in shared memory
// (padded to a power of two), then compaction into a and the fingerprint
__global__ void __launch_bounds__(kSortThreads) k_ct_medium(const int64_t *off, const int32_t *pins,
                                                            const int32_t *map, const int32_t *list,
                                                            const int32_t *count, int32_t *a, int32_t *size1,
                                                            unsigned long long *key, int32_t *rep)
{
    __shared__ int32_t buf[kMedium];
    __shared__ int32_t wtot[kSortThreads / 32];
    __shared__ unsigned long long hsum;
    const int tid = threadIdx.x;
    const int32_t cnt = *count;
    for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
        const int64_t e = list[i];
        const int64_t b = off[e];
        const int32_t s = (int32_t)(off[e + 1] - b);
        int32_t np2 = 2 * kMid;
        while (np2 < s) np2 <<= 1;
        for (int32_t j = tid; j < np2; j += kSortThreads) buf[j] = j < s ? map[pins[b + j]] : 0x7fffffff;
        __syncthreads();
        for (int32_t k = 2; k <= np2; k <<= 1) {
            for (int32_t j = k >> 1; j > 0; j >>= 1) {
                for (int32_t x = tid; x < np2; x += kSortThreads) {
                    const int32_t y = x ^ j;
                    if (y > x) {
                        const bool up = (x & k) == 0;
                        const int32_t vx = buf[x], vy = buf[y];
                        if ((vx > vy) == up) { buf[x] = vy; buf[y] = vx; }
                    }
                }
                __syncthreads();
            }
        }
        int32_t kept;
        unsigned long long h;
        compact_runs(buf, a + b, s, wtot, &hsum, kept, h);
        if (tid == 0) net_done(e, kept, h, size1, key, rep);
        __syncthreads();
    }
}

// Nets of more than kMedium pins, load-balanced over the grid: every kMedium-pin chunk of every
// such net is sorted by one CTA in shared memory (k_lg_chunk), then runs are merged pairwise,
// each CTA producing kMedium outputs of one merge found by a merge-path search (k_lg_merge), and
// finally one CTA per net de-duplicates and fingerprints it (k_lg_dedupe).
constexpr int kLgThreads = 1024;

// chunk task t -> (list index, chunk) through the exclusive prefix of the chunk counts
__device__ __forceinline__ int32_t find_task(const int64_t *cpre, int32_t nl, int64_t t)
{
    int32_t lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (cpre[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_lg_count(const int64_t *off, const int32_t *list, const int32_t *count, int32_t *chunks,
                           int32_t *max_size)
{
    const int32_t nl = *count;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = list[i];
        const int32_t sz = (int32_t)(off[e + 1] - off[e]);
        chunks[i] = (sz + kMedium - 1) / kMedium;
        atomicMax(max_size, sz);
    }
}

// CTA per large net: a representative's pins, offset and summed weight at its coarse position
__global__ void __launch_bounds__(kLgThreads) k_lg_emit(const int64_t *off, const int32_t *a, const int32_t *size1,
                                                        const int32_t *rep, const int64_t *nid, const int64_t *poff,
                                                        const unsigned long long *w64, const int32_t *list,
                                                        const int32_t *count, int32_t *pins2, int64_t *off2,
                                                        int32_t *nw2, int32_t *err)
{
    const int32_t nl = *count;
    for (int64_t i = blockIdx.x; i < nl; i += gridDim.x) {
        const int64_t e = list[i];
        if (rep[e] != (int32_t)e) continue;
        const int64_t src = off[e], dst = poff[e];
        const int32_t s = size1[e];
        for (int32_t j = threadIdx.x; j < s; j += kLgThreads) pins2[dst + j] = a[src + j];
        if (threadIdx.x == 0) {
            off2[nid[e]] = dst;
            const unsigned long long w = w64[e];
            if (w >= (1ull << 31)) atomicOr(err, ERR_UNSUPPORTED);
            nw2[nid[e]] = (int32_t)w;
        }
    }
}

__global__ void __launch_bounds__(kLgThreads) k_lg_chunk(const int64_t *off, const int32_t *pins, const int32_t *map,
                                                         const int32_t *list, const int32_t *count,
                                                         const int64_t *cpre, int64_t tasks, int32_t *a)
{
    __shared__ int32_t buf[kMedium];
    const int tid = threadIdx.x;
    const int32_t nl = *count;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const int32_t li = find_task(cpre, nl, t);
        const int64_t e = list[li];
        const int64_t b = off[e];
        const int32_t s = (int32_t)(off[e + 1] - b);
        const int32_t c0 = (int32_t)(t - cpre[li]) * kMedium;
        const int32_t len = min(kMedium, s - c0);
        for (int32_t j = tid; j < kMedium; j += kLgThreads) buf[j] = j < len ? map[pins[b + c0 + j]] : 0x7fffffff;
        __syncthreads();
        for (int32_t k = 2; k <= kMedium; k <<= 1) {
            for (int32_t j = k >> 1; j > 0; j >>= 1) {
                for (int32_t x = tid; x < kMedium; x += kLgThreads) {
                    const int32_t y = x ^ j;
                    if (y > x) {
                        const bool up = (x & k) == 0;
                        const int32_t vx = buf[x], vy = buf[y];
                        if ((vx > vy) == up) { buf[x] = vy; buf[y] = vx; }
                    }
                }
                __syncthreads();
            }
        }
        for (int32_t j = tid; j < len; j += kLgThreads) a[b + c0 + j] = buf[j];
        __syncthreads();
    }
}

// merge path: number of elements taken from A among the first d outputs of merge(A, B)
__device__ __forceinline__ int32_t merge_split(const int32_t *A, int32_t na, const int32_t *B, int32_t nb, int32_t d)
{
    int32_t lo = max(0, d - nb), hi = min(d, na);
    while (lo < hi) {
        const int32_t i = (lo + hi) >> 1;          // candidate count from A
        if (A[i] <= B[d - 1 - i]) lo = i + 1;     // A[i] comes before B[d-1-i]: take more from A
        else hi = i;
    }
    return lo;
}

// one merge pass over all large nets: runs of width w (sorted) of src are merged pairwise into
// dst; task t = output tile of kMedium elements of one net (same task numbering as the chunks)
__global__ void __launch_bounds__(kLgThreads) k_lg_merge(const int64_t *off, const int32_t *list, const int32_t *count,
                                                         const int64_t *cpre, int64_t tasks, const int32_t *src,
                                                         int32_t *dst, int32_t w)
{
    const int tid = threadIdx.x;
    const int32_t nl = *count;
    constexpr int kPer = kMedium / kLgThreads;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const int32_t li = find_task(cpre, nl, t);
        const int64_t e = list[li];
        const int64_t b = off[e];
        const int32_t s = (int32_t)(off[e + 1] - b);
        const int32_t o0 = (int32_t)(t - cpre[li]) * kMedium + tid * kPer;   // this thread's outputs
        if (o0 >= s) continue;
        const int32_t base = (o0 / (2 * w)) * (2 * w);
        const int32_t na = min(w, s - base), nb = max(0, min(w, s - base - w));
        const int32_t *A = src + b + base, *B = A + na;
        int32_t i = merge_split(A, na, B, nb, o0 - base);
        int32_t j = o0 - base - i;
        int32_t *out = dst + b + o0;
        const int32_t cnt = min(kPer, s - o0);
        for (int q = 0; q < cnt; ++q) {
            const bool takeA = j >= nb || (i < na && A[i] <= B[j]);
            out[q] = takeA ? A[i++] : B[j++];
        }
    }
}

// CTA per large net: compaction of the first of every run into a, and the fingerprint
__global__ void __launch_bounds__(kLgThreads) k_lg_dedupe(const int64_t *off, const int32_t *list, const int32_t *count,
                                                          const int32_t *src, int32_t *a, int32_t *size1,
                                                          unsigned long long *key, int32_t *rep)
{
    __shared__ int32_t wtot[kLgThreads / 32];
    __shared__ unsigned long long hsum;
    const int32_t nl = *count;
    for (int64_t i = blockIdx.x; i < nl; i += gridDim.x) {
        const int64_t e = list[i];
        const int64_t b = off[e];
        const int32_t s = (int32_t)(off[e + 1] - b);
        int32_t kept;
        unsigned long long h;
        compact_runs(src + b, a + b, s, wtot, &hsum, kept, h);
        if (threadIdx.x == 0) net_done(e, kept, h, size1, key, rep);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- identical nets
struct KeySlot {
    unsigned long long key;
    int32_t min_id;
    int32_t pad;
};

__global__ void k_ct_table_clear(KeySlot *tab, int64_t size)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < size; i += (int64_t)gridDim.x * blockDim.x) {
        tab[i].key = kKeyEmpty;
        tab[i].min_id = 0x7fffffff;
    }
}

__device__ __forceinline__ KeySlot *key_find(KeySlot *tab, uint64_t mask, unsigned long long key, bool insert)
{
    uint64_t p = splitmix64_output(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        KeySlot *sl = tab + p;
        unsigned long long cur = __ldcg(&sl->key);
        if (cur == key) return sl;
        if (cur == kKeyEmpty) {
            if (!insert) return nullptr;
            cur = atomicCAS(&sl->key, kKeyEmpty, key);
            if (cur == kKeyEmpty || cur == key) return sl;
        }
        p = (p + 1) & mask;
    }
    return nullptr;
}

// thread per unresolved net: its fingerprint's smallest unresolved net id
__global__ void k_ct_insert(const unsigned long long *key, const int32_t *rep, int32_t m, KeySlot *tab,
                            uint64_t mask, int32_t *err)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        if (rep[e] != kUnresolved) continue;
        KeySlot *sl = key_find(tab, mask, key[e], true);
        if (!sl) { atomicOr(err, ERR_INVALID); continue; }
        atomicMin(&sl->min_id, (int32_t)e);
    }
}

// 32 nets per warp, one per lane: an unresolved net whose fingerprint's smallest net is itself
// is resolved to itself; the others compare their pin lists with that net, the whole warp on
// one net at a time, and are resolved to it if equal, else stay unresolved for the next round
__global__ void k_ct_resolve(const int64_t *off, const int32_t *a, const int32_t *size1,
                             const unsigned long long *key, int32_t *rep, int32_t m, const KeySlot *tab,
                             uint64_t mask, int32_t *left)
{
    const int lane = threadIdx.x & 31;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x; e0 < m; e0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = e0 + threadIdx.x;
        int32_t r = -1;
        bool todo = false;
        if (e < m && rep[e] == kUnresolved) {
            const KeySlot *sl = key_find(const_cast<KeySlot *>(tab), mask, key[e], false);
            r = sl ? sl->min_id : (int32_t)e;
            if (r == (int32_t)e) rep[e] = (int32_t)e;
            else todo = true;
        }
        unsigned tm = __ballot_sync(kFull, todo);
        int32_t nleft = 0;
        while (tm) {
            const int src = __ffs(tm) - 1;
            tm &= tm - 1;
            const int64_t ee = __shfl_sync(kFull, e, src);
            const int32_t rr = __shfl_sync(kFull, r, src);
            const int32_t se = size1[ee];
            bool eq = size1[rr] == se;
            if (eq) {
                const int32_t *pe = a + off[ee], *pr = a + off[rr];
                for (int32_t j = lane; j < se; j += 32) eq = eq && pe[j] == pr[j];
                eq = __all_sync(kFull, eq);
            }
            if (lane == src) {
                if (eq) rep[ee] = rr;
                else ++nleft;
            }
        }
        nleft = __reduce_add_sync(kFull, nleft);
        if (lane == 0 && nleft) atomicAdd(left, nleft);
    }
}

// thread per net: representative flags and sizes for the prefix sums, group weights
__global__ void k_ct_groups(const int32_t *rep, const int32_t *size1, const int32_t *nw, int32_t m,
                            int32_t *is_rep, int32_t *rep_size, unsigned long long *w64)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = rep[e];
        const bool self = r == (int32_t)e;
        is_rep[e] = self;
        rep_size[e] = self ? size1[e] : 0;
        if (r >= 0) atomicAdd(&w64[r], (unsigned long long)(nw ? nw[e] : 1));
    }
}

__device__ __forceinline__ int slot_in(const int32_t *off33, int32_t i)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1)
        if (off33[lo + step] <= i) lo += step;
    return lo;
}

// 32 nets per warp, one per lane: the representatives' pins are copied to their coarse
// positions over the warp's flattened pin range (every lane copies a pin per step), and each
// representative's offset and summed weight are written by its lane
__global__ void k_ct_emit(const int64_t *off, const int32_t *a, const int32_t *size1, const int32_t *rep,
                          const int64_t *nid, const int64_t *poff, const unsigned long long *w64, int32_t m,
                          int32_t *pins2, int64_t *off2, int32_t *nw2, int32_t *err)
{
    __shared__ int32_t off33_w[8][33];
    __shared__ int64_t src_w[8][32], dst_w[8][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *off33 = off33_w[wid];
    for (int64_t e0 = (blockIdx.x * (int64_t)blockDim.x) ; e0 < m; e0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = e0 + threadIdx.x;
        int32_t s = 0;
        if (e < m && rep[e] == (int32_t)e && off[e + 1] - off[e] <= kMedium) {   // larger: k_lg_emit
            s = size1[e];
            src_w[wid][lane] = off[e];
            dst_w[wid][lane] = poff[e];
            off2[nid[e]] = poff[e];
            const unsigned long long w = w64[e];
            if (w >= (1ull << 31)) atomicOr(err, ERR_UNSUPPORTED);
            nw2[nid[e]] = (int32_t)w;
        }
        int32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        off33[lane] = incl - s;
        if (lane == 31) off33[32] = incl;
        __syncwarp();
        const int32_t total = off33[32];
        for (int32_t i = lane; i < total; i += 32) {
            const int v = slot_in(off33, i);
            const int32_t k = i - off33[v];
            pins2[dst_w[wid][v] + k] = a[src_w[wid][v] + k];
        }
        __syncwarp();
    }
}

__global__ void k_ct_project(const int32_t *map, int32_t n, const int32_t *coarse_part, int32_t *fine_part)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        fine_part[u] = coarse_part[map[u]];
}

void coarse_free(hgp_coarse *c)
{
    if (!c) return;
    if (c->net_off) cudaFree(c->net_off);
    if (c->pins) cudaFree(c->pins);
    if (c->vw) cudaFree(c->vw);
    if (c->nw) cudaFree(c->nw);
    if (c->map) cudaFree(c->map);
    delete c;
}

}  // namespace

#define CT(x)                                   \
    do {                                        \
        e = (x);                                \
        if (e != cudaSuccess) goto done;        \
    } while (0)

extern "C" int hgp_contract(int32_t n, int32_t m, const int64_t *net_off, const int32_t *pins,
                            const int32_t *vertex_w, const int32_t *net_w, const int32_t *cluster,
                            void *cuda_stream, hgp_coarse **out)
{
    if (!out) return HGP_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || m < 0 || !net_off || !cluster || (m > 0 && !pins)) return HGP_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    hgp_coarse *c = new (std::nothrow) hgp_coarse;
    if (!c) return HGP_ERR_OOM;
    c->fine_n = n;
    c->stream = st;
    cudaGetDevice(&c->device);
    cudaError_t e = cudaSuccess;
    int rc = HGP_OK;
    int32_t *err = nullptr, *used = nullptr, *a = nullptr, *b = nullptr, *size1 = nullptr, *rep = nullptr;
    int32_t *is_rep = nullptr, *rep_size = nullptr, *left = nullptr, *lists = nullptr, *counts = nullptr;
    void *lg_scratch[2] = {nullptr, nullptr};
    int32_t n_large = 0;
    int sms = 1;
    int64_t *cid = nullptr, *nid = nullptr, *poff = nullptr;
    unsigned long long *w64 = nullptr, *key = nullptr, *nw64 = nullptr;
    KeySlot *tab = nullptr;
    int64_t P = 0, n2 = 0, m2 = 0, P2 = 0;
    int32_t herr = 0;
    const int64_t mm = m > 0 ? m : 1;
    CT(cudaMemcpyAsync(&P, net_off + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CT(stream_wait(st));
    if (P < 0 || (m == 0 && P != 0)) { rc = HGP_ERR_INVALID; goto done; }
    if (P >= ((int64_t)1 << 31)) { rc = HGP_ERR_UNSUPPORTED; goto done; }
    CT(dev_alloc(reinterpret_cast<void **>(&err), sizeof(int32_t) * 2, st));
    CT(cudaMemsetAsync(err, 0, sizeof(int32_t) * 2, st));
    left = err + 1;
    k_ct_check<<<grid_of(P > n ? P : n, 256), 256, 0, st>>>(net_off, pins, vertex_w, net_w, n, m, P, err);
    CT(cudaGetLastError());
    CT(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CT(stream_wait(st));
    if (herr) { rc = HGP_ERR_INVALID; goto done; }
    // (1) remap the used cluster ids
    CT(dev_alloc(reinterpret_cast<void **>(&used), sizeof(int32_t) * (size_t)n, st));
    CT(dev_alloc(reinterpret_cast<void **>(&cid), sizeof(int64_t) * ((size_t)n + 1), st));
    CT(cudaMemsetAsync(used, 0, sizeof(int32_t) * (size_t)n, st));
    k_ct_flag<<<grid_of(n, 256), 256, 0, st>>>(cluster, n, used, err);
    CT(cudaGetLastError());
    CT(scan_excl<int32_t>(used, n, cid, st));
    CT(cudaMemcpyAsync(&n2, cid + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CT(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CT(stream_wait(st));
    if (herr) { rc = HGP_ERR_INVALID; goto done; }
    c->n = (int32_t)n2;
    // (2) map and cluster weights
    CT(cudaMalloc(reinterpret_cast<void **>(&c->map), sizeof(int32_t) * (size_t)n));
    CT(cudaMalloc(reinterpret_cast<void **>(&c->vw), sizeof(int32_t) * (size_t)n2));
    CT(dev_alloc(reinterpret_cast<void **>(&w64), sizeof(unsigned long long) * (size_t)(n > mm ? n : mm), st));
    CT(cudaMemsetAsync(w64, 0, sizeof(unsigned long long) * (size_t)n2, st));
    k_ct_map<<<grid_of(n, 256), 256, 0, st>>>(cluster, n, cid, vertex_w, c->map, w64);
    k_ct_narrow<<<grid_of(n2, 256), 256, 0, st>>>(w64, n2, c->vw, err);
    CT(cudaGetLastError());
    // (3) per-net sort + dedupe
    CT(dev_alloc(reinterpret_cast<void **>(&a), sizeof(int32_t) * (size_t)(P > 0 ? P : 1), st));
    CT(dev_alloc(reinterpret_cast<void **>(&b), sizeof(int32_t) * (size_t)(P > 0 ? P : 1), st));
    CT(dev_alloc(reinterpret_cast<void **>(&size1), sizeof(int32_t) * (size_t)mm, st));
    CT(dev_alloc(reinterpret_cast<void **>(&key), sizeof(unsigned long long) * (size_t)mm, st));
    CT(dev_alloc(reinterpret_cast<void **>(&rep), sizeof(int32_t) * (size_t)mm, st));
    CT(dev_alloc(reinterpret_cast<void **>(&lists), sizeof(int32_t) * kClasses * (size_t)mm + 32, st));
    counts = lists + kClasses * mm;
    CT(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (kClasses + 1), st));
    if (m > 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        k_ct_tiny<<<grid_of(m, 256), 256, 0, st>>>(net_off, pins, m, c->map, a, size1, key, rep, lists, counts);
        k_ct_small<<<sms * 8, 256, 0, st>>>(net_off, pins, c->map, lists, counts, a, size1, key, rep);
        k_ct_mid<<<sms * 8, 256, 0, st>>>(net_off, pins, c->map, lists + mm, counts + 1, a, size1, key, rep);
        k_ct_medium<<<sms * 8, kSortThreads, 0, st>>>(net_off, pins, c->map, lists + 2 * mm, counts + 2, a, size1, key, rep);
        CT(cudaGetLastError());
        // nets of more than kMedium pins: chunk sorts, merge passes, de-duplication
        int32_t hcnt[kClasses] = {0, 0, 0, 0};
        CT(cudaMemcpyAsync(hcnt, counts, sizeof(int32_t) * kClasses, cudaMemcpyDeviceToHost, st));
        CT(stream_wait(st));
        n_large = hcnt[3];
        if (n_large > 0) {
            int32_t *chunks = nullptr;
            int64_t *cpre = nullptr;
            CT(dev_alloc(reinterpret_cast<void **>(&chunks), sizeof(int32_t) * ((size_t)n_large + 1), st));
            CT(dev_alloc(reinterpret_cast<void **>(&cpre), sizeof(int64_t) * ((size_t)n_large + 1), st));
            lg_scratch[0] = chunks;
            lg_scratch[1] = cpre;
            CT(cudaMemsetAsync(counts + kClasses, 0, sizeof(int32_t), st));
            k_lg_count<<<grid_of(n_large, 256), 256, 0, st>>>(net_off, lists + 3 * mm, counts + 3, chunks, counts + kClasses);
            CT(cudaGetLastError());
            CT(scan_excl<int32_t>(chunks, n_large, cpre, st));
            int64_t tasks = 0;
            int32_t max_size = 0;
            CT(cudaMemcpyAsync(&tasks, cpre + n_large, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            CT(cudaMemcpyAsync(&max_size, counts + kClasses, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CT(stream_wait(st));
            const int g = (int)(tasks < (int64_t)sms * 2 ? tasks : (int64_t)sms * 2);
            k_lg_chunk<<<g, kLgThreads, 0, st>>>(net_off, pins, c->map, lists + 3 * mm, counts + 3, cpre, tasks, a);
            int32_t *src = a, *dst = b;
            for (int64_t w = kMedium; w < max_size; w *= 2) {
                k_lg_merge<<<g, kLgThreads, 0, st>>>(net_off, lists + 3 * mm, counts + 3, cpre, tasks, src, dst, (int32_t)w);
                int32_t *t = src; src = dst; dst = t;
            }
            k_lg_dedupe<<<n_large < sms * 2 ? n_large : sms * 2, kLgThreads, 0, st>>>(net_off, lists + 3 * mm, counts + 3,
                                                                                     src, a, size1, key, rep);
            CT(cudaGetLastError());
        }
    }
    // (4) identical nets
    if (m > 0) {
        uint64_t size = 1024;
        while (size < 2 * (uint64_t)m) size <<= 1;
        CT(dev_alloc(reinterpret_cast<void **>(&tab), sizeof(KeySlot) * size, st));
        for (int round = 0;; ++round) {
            if (round >= 4096) { rc = HGP_ERR_INTERNAL; goto done; }
            int32_t hleft = 0;
            CT(cudaMemsetAsync(left, 0, sizeof(int32_t), st));
            k_ct_table_clear<<<grid_of((int64_t)size, 256), 256, 0, st>>>(tab, (int64_t)size);
            k_ct_insert<<<grid_of(m, 256), 256, 0, st>>>(key, rep, m, tab, size - 1, err);
            k_ct_resolve<<<grid_of(m, 256), 256, 0, st>>>(net_off, a, size1, key, rep, m, tab, size - 1, left);
            CT(cudaGetLastError());
            CT(cudaMemcpyAsync(&hleft, left, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CT(stream_wait(st));
            if (hleft == 0) break;
        }
    }
    // (5) representatives in original order, their weights and offsets
    CT(dev_alloc(reinterpret_cast<void **>(&is_rep), sizeof(int32_t) * (size_t)mm, st));
    CT(dev_alloc(reinterpret_cast<void **>(&rep_size), sizeof(int32_t) * (size_t)mm, st));
    CT(dev_alloc(reinterpret_cast<void **>(&nid), sizeof(int64_t) * ((size_t)m + 1), st));
    CT(dev_alloc(reinterpret_cast<void **>(&poff), sizeof(int64_t) * ((size_t)m + 1), st));
    CT(dev_alloc(reinterpret_cast<void **>(&nw64), sizeof(unsigned long long) * (size_t)mm, st));
    CT(cudaMemsetAsync(nw64, 0, sizeof(unsigned long long) * (size_t)mm, st));
    if (m > 0) {
        k_ct_groups<<<grid_of(m, 256), 256, 0, st>>>(rep, size1, net_w, m, is_rep, rep_size, nw64);
        CT(cudaGetLastError());
    }
    CT(scan_excl<int32_t>(is_rep, m, nid, st));
    CT(scan_excl<int32_t>(rep_size, m, poff, st));
    CT(cudaMemcpyAsync(&m2, nid + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CT(cudaMemcpyAsync(&P2, poff + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CT(stream_wait(st));
    c->m = (int32_t)m2;
    c->P = P2;
    CT(cudaMalloc(reinterpret_cast<void **>(&c->net_off), sizeof(int64_t) * ((size_t)m2 + 1)));
    CT(cudaMalloc(reinterpret_cast<void **>(&c->pins), sizeof(int32_t) * (size_t)(P2 > 0 ? P2 : 1)));
    CT(cudaMalloc(reinterpret_cast<void **>(&c->nw), sizeof(int32_t) * (size_t)(m2 > 0 ? m2 : 1)));
    CT(cudaMemcpyAsync(c->net_off + m2, &P2, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (m > 0) {
        if (n_large > 0)
            k_lg_emit<<<n_large < sms * 2 ? n_large : sms * 2, kLgThreads, 0, st>>>(net_off, a, size1, rep, nid, poff, nw64,
                                                                                   lists + 3 * mm, counts + 3, c->pins,
                                                                                   c->net_off, c->nw, err);
        k_ct_emit<<<grid_of(m, 256), 256, 0, st>>>(net_off, a, size1, rep, nid, poff, nw64, m,
                                                                 c->pins, c->net_off, c->nw, err);
        CT(cudaGetLastError());
    }
    CT(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CT(stream_wait(st));
    if (herr & ERR_UNSUPPORTED) rc = HGP_ERR_UNSUPPORTED;
    else if (herr) rc = HGP_ERR_INTERNAL;
done:
    if (err) pool_free(err, st);
    if (used) pool_free(used, st);
    if (cid) pool_free(cid, st);
    if (w64) pool_free(w64, st);
    if (a) pool_free(a, st);
    if (b) pool_free(b, st);
    if (size1) pool_free(size1, st);
    if (key) pool_free(key, st);
    if (rep) pool_free(rep, st);
    if (tab) pool_free(tab, st);
    if (lists) pool_free(lists, st);
    for (void *q : lg_scratch)
        if (q) pool_free(q, st);
    if (is_rep) pool_free(is_rep, st);
    if (rep_size) pool_free(rep_size, st);
    if (nid) pool_free(nid, st);
    if (poff) pool_free(poff, st);
    if (nw64) pool_free(nw64, st);
    {
        const cudaError_t e2 = stream_wait(st);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        rc = status_of(e);
    }
    if (rc != HGP_OK) {
        coarse_free(c);
        return rc;
    }
    *out = c;
    return HGP_OK;
}

extern "C" int hgp_coarse_get_sizes(const hgp_coarse *c, int32_t *n, int32_t *m, int64_t *num_pins)
{
    if (!c || !n || !m || !num_pins) return HGP_ERR_INVALID;
    *n = c->n;
    *m = c->m;
    *num_pins = c->P;
    return HGP_OK;
}

extern "C" int hgp_coarse_get_device_arrays(const hgp_coarse *c, const int64_t **net_off, const int32_t **pins,
                                            const int32_t **vertex_w, const int32_t **net_w, const int32_t **map)
{
    if (!c) return HGP_ERR_INVALID;
    if (net_off) *net_off = c->net_off;
    if (pins) *pins = c->pins;
    if (vertex_w) *vertex_w = c->vw;
    if (net_w) *net_w = c->nw;
    if (map) *map = c->map;
    return HGP_OK;
}

extern "C" int hgp_coarse_copy_to_host(const hgp_coarse *c, int64_t *net_off, int32_t *pins, int32_t *vertex_w,
                                       int32_t *net_w, int32_t *map)
{
    if (!c) return HGP_ERR_INVALID;
    cudaError_t e = cudaSuccess;
    if (net_off) e = cudaMemcpyAsync(net_off, c->net_off, sizeof(int64_t) * ((size_t)c->m + 1), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && pins && c->P > 0)
        e = cudaMemcpyAsync(pins, c->pins, sizeof(int32_t) * (size_t)c->P, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && vertex_w)
        e = cudaMemcpyAsync(vertex_w, c->vw, sizeof(int32_t) * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && net_w && c->m > 0)
        e = cudaMemcpyAsync(net_w, c->nw, sizeof(int32_t) * (size_t)c->m, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && map)
        e = cudaMemcpyAsync(map, c->map, sizeof(int32_t) * (size_t)c->fine_n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = stream_wait(c->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    return HGP_OK;
}

extern "C" int hgp_coarse_project(const hgp_coarse *c, const int32_t *coarse_part, int32_t *fine_part)
{
    if (!c || !coarse_part || !fine_part) return HGP_ERR_INVALID;
    k_ct_project<<<grid_of(c->fine_n, 256), 256, 0, c->stream>>>(c->map, c->fine_n, coarse_part, fine_part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = stream_wait(c->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    return HGP_OK;
}

extern "C" void hgp_coarse_destroy(hgp_coarse *c)
{
    if (c) stream_wait(c->stream);
    coarse_free(c);
}

// libhgp: the gain step (best target and gain per vertex) without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need this computation:
// code that runs while the application's own allocator owns the whole device (frameworks that
// reserve HBM up front and forbid other allocations), code inside host callbacks or other
// contexts where cudaMalloc is not permitted, and latency-critical paths that must not block
// on the allocator.  hgp_candidates_noalloc serves them: it takes every input and output as a
// caller-owned device buffer and keeps its only scratch (per-net records and block weights)
// in a fixed file-scope device array.
//
// The scratch array has room for kNoAllocMaxNets nets.  Every GPU that loads the library holds
// it until the process exits.  Its device address is looked up once per device, on the first
// call made with that device current; that first call should therefore come before any
// stream capture.  No call may be made while its stream is being captured (it reads the
// validation result back and synchronises the stream); such a call returns HGP_ERR_INVALID.
// All calls share the array and it keeps the last call's contents, so calls whose work
// overlaps on the GPU (on different streams, or from several host threads) race.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "hgp_internal.cuh"

using namespace hgp;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int32_t kNoAllocMaxNets = 1 << 18;
constexpr int kMaxDevices = 64;

// scratch layout (bytes): [0, 512) block weights int64[64]; [512, 520) error flags;
// [1024, ...) one 32-byte record per net
struct __align__(16) NaRec {
    uint64_t s1;     // bit i: Phi(e,i) == 1
    uint64_t lam;    // bit i: Phi(e,i) > 0
    int32_t w;       // omega(e)
    int32_t pad[3];
};
constexpr size_t kRecOffset = 1024;
constexpr size_t kScratchBytes = kRecOffset + (size_t)kNoAllocMaxNets * sizeof(NaRec);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices];

int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return HGP_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return HGP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return HGP_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return HGP_OK;
}

__global__ void k_na_clear(int64_t *bw, int32_t *err)
{
    if (threadIdx.x < 64) bw[threadIdx.x] = 0;
    if (threadIdx.x == 0) err[0] = 0;
}

// input checks (every index the later kernels use must be in range)
__global__ void k_na_check(int32_t n, int32_t m, const int32_t *net_off, const int32_t *pins,
                           const int32_t *vtx_off, const int32_t *inc, const int32_t *vw,
                           const int32_t *nw, const int32_t *part, int32_t k, int32_t P, int32_t *err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t e = i0; e <= m; e += stride) {
        const int32_t a = net_off[e];
        if ((e == 0 && a != 0) || (e == m && a != P) || (e < m && net_off[e + 1] < a)) bad = true;
        if (e < m && nw && nw[e] < 1) bad = true;
    }
    for (int64_t v = i0; v <= n; v += stride) {
        const int32_t a = vtx_off[v];
        if ((v == 0 && a != 0) || (v == n && a != P) || (v < n && vtx_off[v + 1] < a)) bad = true;
        if (v < n) {
            if (part[v] < 0 || part[v] >= k) bad = true;
            if (vw && vw[v] < 1) bad = true;
        }
    }
    for (int64_t j = i0; j < P; j += stride)
        if (pins[j] < 0 || pins[j] >= n || inc[j] < 0 || inc[j] >= m) bad = true;
    if (bad) atomicOr(err, 1);
}

// Order checks, warp per list (run after k_na_check has passed, so every index is in range):
// pins strictly increasing inside each net (this also excludes a pin listed twice), and net
// ids strictly increasing inside each vertex's list.
__global__ void k_na_check_order(int32_t n, int32_t m, const int32_t *net_off, const int32_t *pins,
                                 const int32_t *vtx_off, const int32_t *inc, int32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    bool bad = false;
    for (int64_t e = w0; e < m; e += warps)
        for (int32_t j = net_off[e] + 1 + lane; j < net_off[e + 1]; j += 32)
            if (pins[j] <= pins[j - 1]) bad = true;
    for (int64_t v = w0; v < n; v += warps)
        for (int32_t j = vtx_off[v] + 1 + lane; j < vtx_off[v + 1]; j += 32)
            if (inc[j] <= inc[j - 1]) bad = true;
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(err, 1);
}

// Transpose check, thread per incidence (after the order checks): vertex v's list may name net
// e only if v is a pin of e (binary search in the sorted pin list).  With distinct entries per
// list and P entries in total, the two CSRs then describe exactly the same incidences.
__global__ void k_na_check_transpose(int32_t n, const int32_t *net_off, const int32_t *pins,
                                     const int32_t *vtx_off, const int32_t *inc, int32_t *err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        for (int32_t j = vtx_off[v]; j < vtx_off[v + 1]; ++j) {
            const int32_t e = inc[j];
            int32_t lo = net_off[e], hi = net_off[e + 1];
            while (lo < hi) {
                const int32_t mid = lo + ((hi - lo) >> 1);
                if (pins[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= net_off[e + 1] || pins[lo] != (int32_t)v) bad = true;
        }
    }
    if (bad) atomicOr(err, 1);
}

__global__ void k_na_block_weights(int32_t n, const int32_t *part, const int32_t *vw, int64_t *bw)
{
    __shared__ unsigned long long w[64];
    if (threadIdx.x < 64) w[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&w[part[v]], (unsigned long long)(vw ? vw[v] : 1));
    __syncthreads();
    if (threadIdx.x < 64 && w[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(&bw[threadIdx.x]), w[threadIdx.x]);
}

// warp per net: Phi(e, .) counted from the partition -> Lambda(e), S1(e), omega(e)
__global__ void k_na_records(int32_t m, const int32_t *net_off, const int32_t *pins,
                             const int32_t *part, const int32_t *nw, NaRec *recs)
{
    __shared__ int32_t cnt[8][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t e = (int64_t)blockIdx.x * 8 + wid; e < m; e += (int64_t)gridDim.x * 8) {
        cnt[wid][lane] = 0;
        cnt[wid][lane + 32] = 0;
        __syncwarp();
        const int32_t b = net_off[e], end = net_off[e + 1];
        for (int32_t base = b; base < end; base += 32) {
            const int32_t j = base + lane;
            const bool act = j < end;
            const unsigned mask = __ballot_sync(kFull, act);
            if (act) {
                const int blk = part[pins[j]];
                const unsigned peers = __match_any_sync(mask, blk);
                if (lane == __ffs(peers) - 1) cnt[wid][blk] += __popc(peers);
            }
            __syncwarp();
        }
        const unsigned lo_l = __ballot_sync(kFull, cnt[wid][lane] > 0);
        const unsigned hi_l = __ballot_sync(kFull, cnt[wid][lane + 32] > 0);
        const unsigned lo_1 = __ballot_sync(kFull, cnt[wid][lane] == 1);
        const unsigned hi_1 = __ballot_sync(kFull, cnt[wid][lane + 32] == 1);
        if (lane == 0) {
            NaRec r;
            r.s1 = (uint64_t)lo_1 | ((uint64_t)hi_1 << 32);
            r.lam = (uint64_t)lo_l | ((uint64_t)hi_l << 32);
            r.w = nw ? nw[e] : 1;
            r.pad[0] = r.pad[1] = r.pad[2] = 0;
            recs[e] = r;
        }
        __syncwarp();
    }
}

// thread per vertex: the gain step of round 0 (every vertex eligible) for sub-round s, as in
// the refinement rounds: T = blocks of Lambda(e) over nets with Phi(e,a) = 1, minus a and the
// blocks without room; best t in T by g_t = b(u) - W + omega({e : t in Lambda(e)}), smallest
// block on ties; no candidate unless the gain is positive.
__global__ void k_na_candidates(int32_t n, int32_t k, double eps, const int32_t *vtx_off,
                                const int32_t *inc, const NaRec *recs, const int32_t *part,
                                const int32_t *vw, const int64_t *bw, int32_t S, uint64_t seed,
                                int32_t s, int32_t *target, int64_t *gain)
{
    __shared__ long long slack[64];
    if (threadIdx.x < 64) slack[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long total = 0;
        for (int i = 0; i < k; ++i) total += bw[i];
        const long long avg = (total + k - 1) / k;
        const long long lmax = (long long)floor((1.0 + eps) * (double)avg);
        for (int i = 0; i < 64; ++i) slack[i] = i < k ? lmax - bw[i] : -1;
    }
    __syncthreads();
    for (int64_t uu = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; uu < n;
         uu += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = (int32_t)uu;
        int32_t t_best = -1;
        int64_t g_best = 0;
        const uint64_t z = splitmix64_output(seed ^ (uint64_t)(uint32_t)u);
        if ((int32_t)(z % (uint64_t)S) == s) {
            const int a = part[u];
            const int32_t cu = vw ? vw[u] : 1;
            const int32_t jb = vtx_off[u], je = vtx_off[u + 1];
            int64_t W = 0, b = 0;
            uint64_t T = 0;
            for (int32_t j = jb; j < je; ++j) {
                const NaRec &r = recs[inc[j]];
                W += r.w;
                if ((r.s1 >> a) & 1) {
                    b += r.w;
                    T |= r.lam;
                }
            }
            T &= ~(1ull << a);
            for (uint64_t x = T; x; x &= x - 1) {
                const int t = __ffsll((long long)x) - 1;
                if (slack[t] < cu) T &= ~(1ull << t);
            }
            // one pass over the nets per candidate block (registers only)
            for (uint64_t x = T; x; x &= x - 1) {
                const int t = __ffsll((long long)x) - 1;
                int64_t conn = 0;
                for (int32_t j = jb; j < je; ++j) {
                    const NaRec &r = recs[inc[j]];
                    if ((r.lam >> t) & 1) conn += r.w;
                }
                const int64_t g = b - W + conn;
                if (g > g_best) {
                    g_best = g;
                    t_best = t;
                }
            }
        }
        target[u] = t_best;
        gain[u] = g_best;
    }
}

}  // namespace

extern "C" int hgp_candidates_noalloc(int32_t n, int32_t m, const int32_t *net_offsets,
                                      const int32_t *pins, const int32_t *vtx_offsets,
                                      const int32_t *inc_nets, const int32_t *vertex_w,
                                      const int32_t *net_w, int32_t k, double eps,
                                      const int32_t *part, int32_t subrounds, uint64_t seed,
                                      int32_t s, int32_t *target, int64_t *gain, void *cuda_stream)
{
    if (n < 1 || m < 0 || !net_offsets || !vtx_offsets || !part || !target || !gain)
        return HGP_ERR_INVALID;
    if (k < 2 || !(eps > 0.0 && eps < 1.0) || subrounds < 1 || s < 0 || s >= subrounds)
        return HGP_ERR_INVALID;
    if (k > 64 || subrounds > 64 || m > kNoAllocMaxNets) return HGP_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the call reads sizes and the validation result back to the host and synchronises its
    // stream, which a stream capture forbids
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        (void)cudaGetLastError();
        return HGP_ERR_INVALID;
    }
    if (cap != cudaStreamCaptureStatusNone) return HGP_ERR_INVALID;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != HGP_OK) return rc;
    unsigned char *sc = reinterpret_cast<unsigned char *>(base);
    int64_t *bw = reinterpret_cast<int64_t *>(sc);
    int32_t *err = reinterpret_cast<int32_t *>(sc + 512);
    NaRec *recs = reinterpret_cast<NaRec *>(sc + kRecOffset);

    int32_t P = 0;
    cudaError_t e = cudaMemcpyAsync(&P, net_offsets + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return HGP_ERR_CUDA;
    }
    if (P < 0) return HGP_ERR_INVALID;
    if (P > 0 && (!pins || !inc_nets)) return HGP_ERR_INVALID;

    // block weights start from zero and the error flag is cleared on every call
    k_na_clear<<<1, 64, 0, st>>>(bw, err);
    k_na_check<<<152 * 4, 256, 0, st>>>(n, m, net_offsets, pins, vtx_offsets, inc_nets, vertex_w,
                                        net_w, part, k, P, err);
    int32_t bad = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return HGP_ERR_CUDA;
    }
    if (bad) return HGP_ERR_INVALID;
    // every index is in range now: the order and transpose checks may follow them
    if (P > 0) {
        k_na_check_order<<<152 * 8, 256, 0, st>>>(n, m, net_offsets, pins, vtx_offsets, inc_nets, err);
        k_na_check_transpose<<<152 * 4, 256, 0, st>>>(n, net_offsets, pins, vtx_offsets, inc_nets, err);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return HGP_ERR_CUDA;
    }
    if (bad) return HGP_ERR_INVALID;

    k_na_block_weights<<<152 * 4, 256, 0, st>>>(n, part, vertex_w, bw);
    if (m > 0) k_na_records<<<152 * 8, 256, 0, st>>>(m, net_offsets, pins, part, net_w, recs);
    const int64_t blocks = ((int64_t)n + 255) / 256;
    k_na_candidates<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(
        n, k, eps, vtx_offsets, inc_nets, recs, part, vertex_w, bw, subrounds, seed, s, target, gain);
    e = cudaGetLastError();
    if (e != cudaSuccess) return HGP_ERR_CUDA;
    return HGP_OK;
}

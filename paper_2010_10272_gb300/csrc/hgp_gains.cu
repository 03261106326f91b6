// libhgp: exact gains of a move sequence in parallel (paper Sec. 5.4, Lemma 1).
//
// For moves m_1..m_t (vertex u_j from block a_j to b_j, every vertex at most once), the gain of
// m_j if m_1..m_{j-1} were performed first is
//     omega({e in I(u_j) : Phi_j(e, a_j) = 1}) - omega({e in I(u_j) : Phi_j(e, b_j) = 0}),
// with Phi_j the pin counts before m_j.  Lemma 1 turns both conditions into order statistics
// of the moves touching (e, i):
//     Phi_j(e, a) = 1  <=>  Psi(e, a) = 0, j = max out(e, a), min in(e, a) > j
//     Phi_j(e, b) = 0  <=>  Psi(e, b) = 0, j = min in(e, b),  max out(e, b) < j
// where out / in are the moves of a pin of e out of / into the block and
// Psi(e, i) = Phi_1(e, i) - |out(e, i)|.  Pass 1 records, per touched (e, i), max out, min in
// and |out| with atomics; pass 2 evaluates the conditions per move.  The (e, i) entries live in
// an open-addressing hash table sized to the moves (the paper's dense table is O(|E| k)).
#include <cuda_runtime.h>
#include <stdint.h>

#include "hgp_host.cuh"

using namespace hgp;

namespace {

constexpr unsigned long long kEmpty = ~0ull;

struct Slot {
    unsigned long long key;   // e * 64 + i, kEmpty when free
    int32_t max_out;          // largest index of a move out of block i with a pin of e, -1 if none
    int32_t min_in;           // smallest index of a move into block i, INT32_MAX if none
    int32_t n_out;            // |out(e, i)|
    int32_t pad;
};

__device__ __forceinline__ uint64_t slot_hash(uint64_t key) { return splitmix64_output(key); }

// find or insert (linear probing; the table is at most half full, so a free slot exists)
__device__ __forceinline__ Slot *find_slot(Slot *table, uint64_t mask, unsigned long long key, bool insert)
{
    uint64_t p = slot_hash(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        Slot *s = table + p;
        unsigned long long cur = s->key;
        if (cur == key) return s;
        if (cur == kEmpty) {
            if (!insert) return nullptr;
            cur = atomicCAS(&s->key, kEmpty, key);
            if (cur == kEmpty || cur == key) return s;
        }
        p = (p + 1) & mask;
    }
    return nullptr;
}

__global__ void k_eg_init(Slot *table, uint64_t size)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < size;
         i += (uint64_t)gridDim.x * blockDim.x) {
        Slot s;
        s.key = kEmpty;
        s.max_out = -1;
        s.min_in = 0x7fffffff;
        s.n_out = 0;
        s.pad = 0;
        table[i] = s;
    }
}

// validation: vertex in range, moved once, from = Pi(u), to in range and different
__global__ void k_eg_check(Dev d, const int32_t *moves, int32_t count, int32_t *seen, int32_t *err)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = moves[3 * j], a = moves[3 * j + 1], b = moves[3 * j + 2];
        bool bad = u < 0 || u >= d.n || b < 0 || b >= d.k || a == b;
        if (!bad) bad = d.part[u] != a || atomicExch(&seen[u], 1) != 0;
        if (bad) atomicOr(err, 1);
    }
}

// warp per move: record out / in order statistics of every (net, block) the move touches
__global__ void k_eg_pass1(Dev d, const int32_t *moves, int32_t count, Slot *table, uint64_t mask, int32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < count; j += warps) {
        const int32_t u = moves[3 * j], a = moves[3 * j + 1], b = moves[3 * j + 2];
        for (int32_t x = d.vtx_off[u] + lane; x < d.vtx_off[u + 1]; x += 32) {
            const unsigned long long e = (unsigned long long)(d.inc[x] & kNetMask);
            Slot *sa = find_slot(table, mask, e * 64 + a, true);
            Slot *sb = find_slot(table, mask, e * 64 + b, true);
            if (!sa || !sb) {
                atomicOr(err, 2);
                continue;
            }
            atomicMax(&sa->max_out, (int32_t)j);
            atomicAdd(&sa->n_out, 1);
            atomicMin(&sb->min_in, (int32_t)j);
        }
    }
}

// warp per move: exact gain from Lemma 1
__global__ void k_eg_pass2(Dev d, const int32_t *moves, int32_t count, Slot *table, uint64_t mask, int64_t *gains)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const Rec16 *r16 = reinterpret_cast<const Rec16 *>(d.rec);
    const Rec32 *r32 = reinterpret_cast<const Rec32 *>(d.rec);
    for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < count; j += warps) {
        const int32_t u = moves[3 * j], a = moves[3 * j + 1], b = moves[3 * j + 2];
        long long g = 0;
        for (int32_t x = d.vtx_off[u] + lane; x < d.vtx_off[u + 1]; x += 32) {
            const int32_t eraw = d.inc[x];
            const int32_t e = eraw & kNetMask;
            const bool wide = eraw < 0;
            const int32_t wrow = wide ? d.widx[e] : 0;
            const int32_t w = (d.k <= 32 ? r16[e].w : r32[e].w) & 0x7fffffff;
            const Slot *sa = find_slot(table, mask, (unsigned long long)e * 64 + a, false);
            const Slot *sb = find_slot(table, mask, (unsigned long long)e * 64 + b, false);
            if (sa && sa->n_out == phi_get(d, e, a, wide, wrow) && sa->max_out == j && sa->min_in > j) g += w;
            if (sb && sb->n_out == phi_get(d, e, b, wide, wrow) && sb->min_in == j && sb->max_out < j) g -= w;
        }
        for (int o = 16; o; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0) gains[j] = g;
    }
}

int grid_of(int64_t work, int threads)
{
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

}  // namespace

// sum of the degrees of the moved vertices (each contributes 2 keys per incident net)
__global__ void k_eg_degsum(Dev d, const int32_t *moves, int32_t count, unsigned long long *out)
{
    unsigned long long s = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = moves[3 * j];
        if (u >= 0 && u < d.n) s += (unsigned long long)(d.vtx_off[u + 1] - d.vtx_off[u]);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

extern "C" int hgp_exact_gains(hgp_handle *h, int32_t count, const int32_t *moves, int64_t *gains)
{
    if (!h || count < 0 || (count > 0 && (!moves || !gains))) return HGP_ERR_INVALID;
    settle(h);
    if (count == 0) return HGP_OK;
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    int32_t *mv = nullptr, *seen = nullptr, *err = nullptr;
    unsigned long long *degsum = nullptr;
    Slot *table = nullptr;
    int64_t *g_d = nullptr;
    int32_t herr = 0;
    unsigned long long hdeg = 0;
    int rc = HGP_OK;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&mv), sizeof(int32_t) * 3 * (size_t)count, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mv, moves, sizeof(int32_t) * 3 * (size_t)count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&seen), sizeof(int32_t) * ((size_t)d.n + 1), st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&err), sizeof(int32_t), st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&degsum), sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(seen, 0, sizeof(int32_t) * ((size_t)d.n + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(degsum, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        k_eg_check<<<grid_of(count, 256), 256, 0, st>>>(d, mv, count, seen, err);
        k_eg_degsum<<<grid_of(count, 256), 256, 0, st>>>(d, mv, count, degsum);
        h->launches += 2;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hdeg, degsum, sizeof(hdeg), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = stream_wait(st);
    if (e == cudaSuccess && herr) rc = HGP_ERR_INVALID;
    // at most 2 keys per incident net of a moved vertex; keep the table at most half full
    uint64_t size = 64;
    while (size < 4 * (uint64_t)hdeg) size <<= 1;
    if (e == cudaSuccess && rc == HGP_OK) e = dev_alloc(reinterpret_cast<void **>(&table), sizeof(Slot) * size, st);
    if (e == cudaSuccess && rc == HGP_OK) e = dev_alloc(reinterpret_cast<void **>(&g_d), sizeof(int64_t) * (size_t)count, st);
    if (e == cudaSuccess && rc == HGP_OK) {
        k_eg_init<<<grid_of((int64_t)size, 256), 256, 0, st>>>(table, size);
        k_eg_pass1<<<grid_of((int64_t)count * 32, 256), 256, 0, st>>>(d, mv, count, table, size - 1, err);
        k_eg_pass2<<<grid_of((int64_t)count * 32, 256), 256, 0, st>>>(d, mv, count, table, size - 1, g_d);
        h->launches += 3;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && rc == HGP_OK) e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rc == HGP_OK) e = cudaMemcpyAsync(gains, g_d, sizeof(int64_t) * (size_t)count, cudaMemcpyDeviceToHost, st);
    if (mv) pool_free(mv, st);
    if (seen) pool_free(seen, st);
    if (err) pool_free(err, st);
    if (degsum) pool_free(degsum, st);
    if (table) pool_free(table, st);
    if (g_d) pool_free(g_d, st);
    const cudaError_t e2 = stream_wait(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return status_of(e);
    }
    if (rc == HGP_OK && herr) rc = HGP_ERR_INTERNAL;
    return rc;
}

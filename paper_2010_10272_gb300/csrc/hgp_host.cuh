// Host-side handle of libhgp (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hgp_internal.cuh"

struct hgp_handle {
    hgp::Dev d{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t seed = 0;
    int32_t debug = 0;
    int32_t graph = 0;
    int64_t next_round = 0;       // global round counter r
    bool all_eligible = true;     // first round after creation / set_partition
    int32_t n_wide = 0;
    int32_t m_big = 0;            // internal order: nets [0, m_big) have at least kBigNet pins
    int32_t m_big32 = 0;          // m_big rounded up to whole 32-net groups (at most m)
    int64_t max_vertex_netweight = 0;   // max_u sum_{e in I(u)} omega(e)
    int64_t total_weight = 0;
    int32_t stats_cap = 0;
    int64_t *h_stats = nullptr;   // host copy of the stats buffer
    // memory owned by the handle
    static constexpr int kMaxAllocs = 64;
    void *allocs[kMaxAllocs] = {};
    int n_allocs = 0;
    // one allocation (also in allocs) that small handles' buffers are carved from, so that a
    // creation makes one pool call instead of ~25 (pool calls from many threads contend)
    char *arena = nullptr;
    size_t arena_size = 0, arena_used = 0;
    int32_t *scratch_n = nullptr;  // int32[n] in the arena (the creation's scan scratch), reused by
                                   // partition uploads and read-backs; nullptr without an arena
    // CUDA-graph cache: one refine() of `graph_rounds` rounds
    cudaGraphExec_t graph_exec = nullptr;
    int32_t graph_rounds = 0;
    int32_t *d_round = nullptr;   // device round state (Dev::rs)
    hgp::Dev *d_dev = nullptr;    // device copy of d, read by the kernels
    bool dev_dirty = true;        // d changed since the last upload
    int64_t graph_launches = 0;   // kernels in one replay of graph_exec
    // kernel launches since creation, and per-phase event timing
    int64_t launches = 0;
    int grid_gain = 0;            // persistent grid sizes (CTAs), set at first launch
    int grid_apply = 0;
    int32_t gain_ctas = 0;        // per-SM CTA overrides of those grids (0: occupancy)
    int32_t apply_ctas = 0;
    bool profiling = false;
    double prof_ms[HGP_PHASES] = {};
    int64_t prof_launches[HGP_PHASES] = {};
    cudaEvent_t *events = nullptr;  // pool, 2 per timed phase instance
    int32_t n_events = 0;
    int32_t events_used = 0;
    int32_t *event_phase = nullptr; // phase of each event pair
    int32_t *event_count = nullptr; // kernel launches inside each event pair
    // the end of the last batch call that refined this handle from another stream, which later
    // work on the handle's own stream must follow (recorded by the batch, owned by the handle;
    // see settle())
    cudaEvent_t ev_batch = nullptr;
    bool after_batch = false;
};

namespace hgp {

inline int status_of(cudaError_t e)
{
    if (e == cudaSuccess) return HGP_OK;
    if (e == cudaErrorMemoryAllocation) return HGP_ERR_OOM;
    return HGP_ERR_CUDA;
}

// Device memory of handles and batches comes from a library-owned stream-ordered memory pool
// of the current device (cudaMallocFromPoolAsync / cudaFreeAsync on the owner's stream), so
// creating or destroying a handle never implies a device-wide synchronisation and can overlap
// with kernels of other handles (the serving loop relies on this).  Freed memory goes back to
// the system at the next synchronisation unless hgp_set_pool_retention keeps some of it.
cudaError_t library_pool(cudaMemPool_t *out);
// Waits on the host for the work queued on st: spinning in cudaStreamSynchronize, or, after
// hgp_set_blocking_waits(1), sleeping on a blocking-sync event recorded on st.
cudaError_t stream_wait(cudaStream_t st);
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);
// the same for temporaries whose release status the caller checks
inline cudaError_t pool_free(void *p, cudaStream_t st) { return p ? cudaFreeAsync(p, st) : cudaSuccess; }

// Carves `bytes` (rounded up to 256) from the handle's arena; nullptr when it has no room left.
inline void *arena_take(hgp_handle *h, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (!h->arena || h->arena_used + bytes > h->arena_size) return nullptr;
    void *p = h->arena + h->arena_used;
    h->arena_used += bytes;
    return p;
}

inline bool in_arena(const hgp_handle *h, const void *p)
{
    const char *c = static_cast<const char *>(p);
    return h->arena && c >= h->arena && c < h->arena + h->arena_size;
}

// Orders the handle's stream after the last batch call that refined the handle from another
// stream.  Every entry point that queues work on, or reads from, the handle calls it first, so
// a batch call itself never makes the handle's stream wait (work queued there meanwhile, such
// as creating other handles, is not held back by the batch).
inline void settle(hgp_handle *h)
{
    if (h->after_batch) {
        if (cudaStreamWaitEvent(h->stream, h->ev_batch, 0) != cudaSuccess) (void)cudaGetLastError();
        h->after_batch = false;
    }
}

// refine-side entry points used by the C ABI layer (hgp_refine.cu)
int refine_rounds(hgp_handle *h, int32_t rounds, hgp_round_stats *stats);
int debug_candidates(hgp_handle *h, int32_t s, int32_t *target, int64_t *gain);
int ensure_stats(hgp_handle *h, int32_t rounds);
cudaError_t objective_from_phi(hgp_handle *h, int64_t *d_out);

}  // namespace hgp

// libhgp: measurement of the device's random-gather and random-atomic rates.
//
// The gain and apply steps are bound by random accesses to per-net data (one record per
// incidence, Phi entries per moved pin), not by streaming bandwidth: on an array much larger
// than L2, a random 8-, 16- or 32-byte gather costs about the same.  hgp_probe_gather times
// such gathers so that a kernel's gathers per second can be compared with what the memory
// system delivers.  The paper has no counterpart; this is a measurement helper.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hgp_internal.cuh"

using namespace hgp;

namespace {

// each thread gathers `per_thread` records of 32 bytes at pseudo-random indices in [0, count)
__global__ void k_probe_gather(const uint4 *__restrict__ rec, int64_t count, int64_t n_gathers, uint32_t *out)
{
    uint32_t acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_gathers;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = (int64_t)(splitmix64_output((uint64_t)i) % (uint64_t)count);
        const uint4 a = __ldg(rec + 2 * idx), b = __ldg(rec + 2 * idx + 1);
        acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// each thread adds 1 at pseudo-random 32-bit words in [0, count) with atomics whose old value
// it consumes (the form of the apply step's pin-count updates)
__global__ void k_probe_atomic(uint32_t *__restrict__ words, int64_t count, int64_t n_ops, uint32_t *out)
{
    uint32_t acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_ops;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = (int64_t)(splitmix64_output((uint64_t)i ^ 0x5bd1e995ull) % (uint64_t)count);
        acc ^= atomicAdd(words + idx, 1u);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

enum { PROBE_GATHER = 0, PROBE_ATOMIC = 1 };

int probe(int kind, int64_t array_bytes, int64_t n_ops, double *ms_out, double *ops_per_s)
{
    if (array_bytes < 64 || n_ops < 1 || !ms_out || !ops_per_s) return HGP_ERR_INVALID;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (sms > 0 ? sms : 1) * 8, block = 256;
    void *buf = nullptr;
    uint32_t *out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st = nullptr;
    const int64_t count = array_bytes / 32;
    cudaError_t e = cudaMalloc(&buf, (size_t)count * 32);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&out), sizeof(uint32_t) * grid * block);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 1, (size_t)count * 32, st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a, st);
        if (kind == PROBE_GATHER)
            k_probe_gather<<<grid, block, 0, st>>>(reinterpret_cast<const uint4 *>(buf), count, n_ops, out);
        else
            k_probe_atomic<<<grid, block, 0, st>>>(reinterpret_cast<uint32_t *>(buf), count * 8, n_ops, out);
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    if (buf) cudaFree(buf);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? HGP_ERR_OOM : HGP_ERR_CUDA;
    }
    *ms_out = best;
    *ops_per_s = (double)n_ops / (best / 1e3);
    return HGP_OK;
}

}  // namespace

extern "C" int hgp_probe_atomic(int64_t array_bytes, int64_t n_atomics, double *ms_out, double *atomics_per_s)
{
    return probe(PROBE_ATOMIC, array_bytes, n_atomics, ms_out, atomics_per_s);
}

extern "C" int hgp_probe_gather(int64_t array_bytes, int64_t n_gathers, double *ms_out,
                                double *gathers_per_s)
{
    return probe(PROBE_GATHER, array_bytes, n_gathers, ms_out, gathers_per_s);
}

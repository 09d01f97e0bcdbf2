// Allocation-free argmax (hbx_argmax_noalloc in include/hbx.h).
//
// The selection's argmax kernel keeps its per-block partial maxima and its
// finish counter in device memory that the library allocates.  Some callers
// cannot allocate device memory at the point where they need the argmax: a
// service that reserves all of its GPU memory up front and must run within that
// fixed budget, or code that runs inside a memory allocator's own hook (a
// framework's caching allocator), where allocating again would re-enter that
// allocator.  This variant takes its scratch from a file-scope static device
// array instead, so a call allocates nothing.
//
// The array exists once per device that loads the library and lives until the
// process exits.  Every call on a device shares it and leaves the last call's
// contents behind; the finish counter is cleared before each launch.  Calls
// whose launches overlap on the GPU (for example on two streams at once) race
// on the shared array, so a caller must order them (one stream, or events).
//
// CUDA loads a module's device code lazily, on first use, and that load itself
// reserves device memory.  The first call on each device therefore loads this
// kernel explicitly and looks up the array's address; a caller makes that call
// (or the set-up-only call with null pointers and n = 0) before reserving its
// memory budget, and every later call allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "hbx.h"

namespace hbx {

constexpr uint32_t NA_THREADS = 256;
constexpr uint32_t NA_PER_THREAD = 16;  // counts read by one thread
constexpr uint32_t NA_MAX_BLOCKS = 4096;
static_assert((uint64_t)NA_THREADS * NA_PER_THREAD * NA_MAX_BLOCKS == HBX_ARGMAX_NOALLOC_MAX,
              "maximum size of the allocation-free argmax");

struct NoAllocScratch {
    unsigned long long partial[NA_MAX_BLOCKS];  // per-block (count, id) keys
    unsigned int ticket;                        // blocks finished
};

// 32 KB of scratch in the module's static device memory.
static __device__ __align__(256) NoAllocScratch g_argmax_scratch;

// key = (count with its sign bit flipped) << 32 | (2^32 - 1 - id): the largest
// key is the largest count, lowest id on ties, for any int32 counts.
__global__ void __launch_bounds__(NA_THREADS) argmax_noalloc_kernel(const int32_t* __restrict__ cnt, uint32_t n,
                                                                    uint32_t* __restrict__ out,
                                                                    NoAllocScratch* scr) {
    __shared__ unsigned long long s_w[NA_THREADS / 32];
    __shared__ bool s_last;
    const uint32_t base = blockIdx.x * NA_THREADS * NA_PER_THREAD + threadIdx.x;
    unsigned long long best = 0;
#pragma unroll
    for (uint32_t i = 0; i < NA_PER_THREAD; i++) {
        const uint32_t v = base + i * NA_THREADS;
        if (v < n) {
            const unsigned long long key =
                ((unsigned long long)((uint32_t)__ldg(cnt + v) ^ 0x80000000u) << 32) | (0xFFFFFFFFu - v);
            best = key > best ? key : best;
        }
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int w = 0; w < NA_THREADS / 32; w++) m = s_w[w] > m ? s_w[w] : m;
        scr->partial[blockIdx.x] = m;
        __threadfence();
        s_last = atomicAdd(&scr->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long m = 0;
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += NA_THREADS) {
        const unsigned long long y = __ldcg(scr->partial + b);
        m = y > m ? y : m;
    }
    m = warp_max_u64(m);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long r = 0;
        for (int w = 0; w < NA_THREADS / 32; w++) r = s_w[w] > r ? s_w[w] : r;
        *out = 0xFFFFFFFFu - (uint32_t)r;
        scr->ticket = 0;
    }
}

// Host-side address of the scratch array on each device, looked up once per
// device with that device current.  (The array's name in host code is only a
// host-side stand-in, not a device address.)
static std::mutex g_mu;
static NoAllocScratch* g_scratch_ptr[64];
static bool g_ready[64];

static int scratch_for_current_device(NoAllocScratch** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return HBX_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ready[dev]) {
        // load the module on this device now (lazy loading would do it at the
        // first launch), then resolve the array's device address
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, argmax_noalloc_kernel) != cudaSuccess) {
            cudaGetLastError();
            return HBX_ERR_CUDA;
        }
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_argmax_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return HBX_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
        g_ready[dev] = true;
    }
    *out = g_scratch_ptr[dev];
    return HBX_OK;
}

}  // namespace hbx

extern "C" int hbx_argmax_noalloc(const int32_t* d_counts, uint32_t n, uint32_t* d_out, void* cuda_stream) {
    using namespace hbx;
    const bool setup_only = !d_counts && !d_out && n == 0;
    if (!setup_only && (!d_counts || !d_out || n == 0 || (uint64_t)n > HBX_ARGMAX_NOALLOC_MAX))
        return HBX_ERR_INVALID_ARG;
    NoAllocScratch* scr = nullptr;
    const int r = scratch_for_current_device(&scr);
    if (r != HBX_OK || setup_only) return r;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // The last block of every finished launch sets the counter back to 0; this
    // clear guards against a launch that never finished (an aborted context or
    // a launch error), which would leave it non-zero.
    if (cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return HBX_ERR_CUDA;
    }
    const uint32_t per_block = NA_THREADS * NA_PER_THREAD;
    const uint32_t blocks = (n + per_block - 1) / per_block;
    argmax_noalloc_kernel<<<blocks, NA_THREADS, 0, s>>>(d_counts, n, d_out, scr);
    if (cudaGetLastError() != cudaSuccess) return HBX_ERR_CUDA;
    return HBX_OK;
}

// noalloc.cu -- the truncation threshold of the spectral initialisation,
// computed without allocating device memory.
//
// lrccs_init computes gamma = trunc * sum|y|^2 / count with k_energy, whose
// per-block partial sums and completion counter live in context buffers that
// lrccs_create allocates.  This file provides the same reduction for callers
// that must not allocate: its scratch is a fixed-size array at file scope in
// device memory, present on every device that loads the library.

#include "common.cuh"
#include "internal.h"
#include "lrccs.h"

#define NA_THREADS 256
#define NA_ENTRIES_PER_BLOCK 65536
#define NA_MAX_BLOCKS 4096   // LRCCS_NOALLOC_MAX_ENTRIES / NA_ENTRIES_PER_BLOCK

static_assert((int64_t)NA_MAX_BLOCKS * NA_ENTRIES_PER_BLOCK == LRCCS_NOALLOC_MAX_ENTRIES,
              "scratch size and the documented maximum must agree");

// Per-block FP64 partial sums, then the completion counter of the grid
// reduction.  32 KiB + 256 B, held by each device until the process exits.
struct na_scratch {
    double part[NA_MAX_BLOCKS];
    unsigned int counter;
    unsigned int pad[63];
};
static __device__ __align__(256) na_scratch g_na_scratch;

// |y|^2 in FP64 without contraction, as in the context path, so that the
// threshold is the same value lrccs_init computes up to summation order.
static __device__ __forceinline__ double na_abs2(float2 v) {
    return __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y));
}

__global__ void __launch_bounds__(NA_THREADS) k_energy_noalloc(const float2 *__restrict__ y, int64_t count,
                                                               double trunc, na_scratch *scr, double *gamma) {
    __shared__ double s_red[NA_THREADS / 32];
    const int64_t i0 = (int64_t)blockIdx.x * NA_ENTRIES_PER_BLOCK;
    const int64_t i1 = min(count, i0 + NA_ENTRIES_PER_BLOCK);
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += NA_THREADS) acc += na_abs2(y[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) b += s_red[w];
        scr->part[blockIdx.x] = b;
    }
    if (last_block_arrive(&scr->counter) && threadIdx.x == 0) {
        double e = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) e += __ldcg(scr->part + b);
        *gamma = trunc * e / (double)count;
    }
}


extern "C" lrccs_status lrccs_trunc_threshold_noalloc(const void *d_y, int64_t count, double trunc_factor,
                                                      double *d_gamma, void *cuda_stream) {
    if (!d_y || !d_gamma) {
        set_err(nullptr, "lrccs_trunc_threshold_noalloc: d_y and d_gamma must be device pointers");
        return LRCCS_E_INVALID;
    }
    if (count < 1 || count > LRCCS_NOALLOC_MAX_ENTRIES) {
        set_err(nullptr, "lrccs_trunc_threshold_noalloc: count = %lld outside [1, %lld] (the fixed scratch "
                         "holds one partial sum per %d entries, %d at most)",
                (long long)count, (long long)LRCCS_NOALLOC_MAX_ENTRIES, NA_ENTRIES_PER_BLOCK, NA_MAX_BLOCKS);
        return LRCCS_E_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        set_err(nullptr, "lrccs_trunc_threshold_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return LRCCS_E_CUDA;
    }
    // the device address of the array in the current context, resolved on
    // every call (no allocation; stays right after a context is recreated)
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
        set_err(nullptr, "lrccs_trunc_threshold_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return LRCCS_E_CUDA;
    }
    na_scratch *scr = (na_scratch *)p;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // The counter must start at zero; the partial sums are overwritten.
    e = cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) {
        set_err(nullptr, "lrccs_trunc_threshold_noalloc: %s", cudaGetErrorString(e));
        return LRCCS_E_CUDA;
    }
    const unsigned blocks = (unsigned)((count + NA_ENTRIES_PER_BLOCK - 1) / NA_ENTRIES_PER_BLOCK);
    k_energy_noalloc<<<blocks, NA_THREADS, 0, s>>>((const float2 *)d_y, count, trunc_factor, scr, d_gamma);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_err(nullptr, "lrccs_trunc_threshold_noalloc: launch failed: %s", cudaGetErrorString(e));
        return LRCCS_E_CUDA;
    }
    return LRCCS_OK;
}

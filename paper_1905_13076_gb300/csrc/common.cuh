// Device helpers shared by the kernels: bounded grid barrier, deterministic
// cross-block reduction, L2-coherent loads, complex arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "args.h"

namespace pppc {

// A grid barrier gives up after this long (ns of %globaltimer) and reports
// DEV_ERR_TIMEOUT; no phase of any kernel legitimately takes longer.
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;

// Lets kernel fn take all the dynamic shared memory a block may opt into.
// The limit is a property of the function shared by every handle, so it is
// set once to the device maximum rather than to one launch's size (a later,
// smaller setting would make an earlier handle's launches fail).
inline cudaError_t allow_max_dynamic_smem(const void* fn) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
    return *reinterpret_cast<const volatile unsigned int*>(p);
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

// Loads of data written by other blocks earlier in the same launch go through
// L2 only (ld.global.cg): the per-SM L1 is not coherent across SMs.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg2(const double* p) { return __ldcg(reinterpret_cast<const double2*>(p)); }
__device__ __forceinline__ float2 ldcg2(const float* p) { return __ldcg(reinterpret_cast<const float2*>(p)); }

// Loads of another block's rows after a grid barrier.  The barrier's
// acquire (thread 0) followed by __syncthreads orders them after the other
// blocks' writes, so they may be served by L1.
__device__ __forceinline__ double2 gld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ float2 gld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

template <typename T> struct vec2_t;
template <> struct vec2_t<double> { using type = double2; };
template <> struct vec2_t<float> { using type = float2; };

template <typename T>
__device__ __forceinline__ typename vec2_t<T>::type ld2(const T* p) {
    return *reinterpret_cast<const typename vec2_t<T>::type*>(p);
}
template <typename T>
__device__ __forceinline__ void st2(T* p, T a, T b) {
    typename vec2_t<T>::type v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<typename vec2_t<T>::type*>(p) = v;
}

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Spin until pred() holds; gives up after kBarrierTimeoutNs, setting
// DEV_ERR_TIMEOUT.  Returns false on timeout.
template <typename Pred>
__device__ __forceinline__ bool spin_until(Pred pred, int* status) {
    unsigned long long t0 = 0;
    unsigned int spins = 0;
    while (!pred()) {
        if ((++spins & 1023u) == 0u) {
            const unsigned long long t = global_ns();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > kBarrierTimeoutNs) {
                set_status(status, DEV_ERR_TIMEOUT);
                return false;
            }
        }
    }
    return true;
}

// Barrier over a team of nblk blocks (the whole grid, or the blocks of one
// batch member), bid = this block's index in the team, with one atomic per
// block: block 0 adds 2^31 - (nblk - 1), every other block adds 1, so the
// counter grows by exactly 2^31 per round and its top bit flips when the last
// block arrives; each block waits for that flip relative to the value it
// saw.  Returns false if the wait timed out here or in another block (the
// caller then returns).
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, int* status, int bid, int nblk) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int add = bid == 0 ? 0x80000000u - (unsigned int)(nblk - 1) : 1u;
        __threadfence();
        const unsigned int old = atomicAdd(&bar->flip, add);
        int ok = spin_until([&] { return ((ld_acquire_u32(&bar->flip) ^ old) & 0x80000000u) != 0u; }, status);
        __threadfence();
        if (ld_volatile_i32(status) == DEV_ERR_TIMEOUT) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, int* status) {
    return grid_sync(bar, status, blockIdx.x, gridDim.x);
}

// Cross-block reduction without a serial last block.  Each of the nb blocks
// of a team writes its partial sums block-major, part[b * nvals + o]; after
// one grid_sync every
// block reduces all of them itself, in one fixed order, into shared memory.
// All blocks therefore hold bitwise-identical sums and take identical
// decisions.  Thread t sums the partials of output t % nvals over the blocks
// b = t / nvals, t / nvals + chunks, ... (chunks = blockDim / nvals), then the
// chunk results are added in chunk order (tmp[blockDim] holds them).  The caller alternates between two partial buffers so that
// writing the next partials never overtakes a slower block still reading.
template <typename RT>
__device__ __forceinline__ void block_reduce_all(const RT* part, int nvals, RT* sums, RT* tmp, int nb) {
    const int t = threadIdx.x;
    if (nvals >= (int)blockDim.x) {  // more values than threads: one thread per value
        for (int o = t; o < nvals; o += blockDim.x) {
            RT acc = 0;
            for (int b = 0; b < nb; ++b) acc += __ldcg(part + (size_t)b * nvals + o);
            sums[o] = acc;
        }
        __syncthreads();
        return;
    }
    const int chunks = blockDim.x / nvals;
    if (t < chunks * nvals) {
        const int o = t % nvals, c = t / nvals;
        RT acc = 0;
        // 16 independent loads in flight per round
        for (int base = c; base < nb; base += 16 * chunks) {
            RT v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int b = base + k * chunks;
                v[k] = b < nb ? __ldcg(part + (size_t)b * nvals + o) : (RT)0;
            }
#pragma unroll
            for (int w = 8; w > 0; w >>= 1)
#pragma unroll
                for (int k = 0; k < w; ++k) v[k] += v[k + w];
            acc += v[0];
        }
        tmp[t] = acc;
    }
    __syncthreads();
    for (int o = t; o < nvals; o += blockDim.x) {
        RT acc = 0;
        for (int c = 0; c < chunks; ++c) acc += tmp[c * nvals + o];
        sums[o] = acc;
    }
    __syncthreads();
}

// ---- complex helpers (value type double2 / float2 as re, im) -------------
struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    } else {
        double r = b.re / b.im, d = b.im + b.re * r;
        return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
    }
}
__device__ __forceinline__ double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }

}  // namespace pppc

// Device helpers shared by the kernels: bounded grid barrier with a
// deterministic cross-block reduction, L2-coherent loads, complex arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "args.h"

namespace pppc {

// A grid barrier gives up after this long (ns of %globaltimer) and reports
// DEV_ERR_TIMEOUT; no phase of any kernel legitimately takes longer.
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;

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

// Arrive at the barrier and wait for all blocks.  Returns false if the wait
// timed out here or in another block (the caller then returns).
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int g = ld_volatile_u32(&bar->gen);
        __threadfence();
        unsigned int arrived = atomicAdd(&bar->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            unsigned long long t0 = global_ns();
            unsigned int spins = 0;
            while (ld_volatile_u32(&bar->gen) == g) {
                if ((++spins & 255u) == 0u && global_ns() - t0 > kBarrierTimeoutNs) {
                    set_status(status, DEV_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            __threadfence();
        }
        if (ld_volatile_i32(status) == DEV_ERR_TIMEOUT) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Barrier whose last arriving block sums the per-block partials
// part[b * nvals + o] over b = 0..gridDim.x-1 in ascending order (a fixed
// order, so results are bitwise reproducible) into sums[o] before releasing
// the others.  Every block must have written its partials before calling.
__device__ __forceinline__ bool grid_sync_reduce(GridBarrier* bar, int* status, const double* part,
                                                 double* sums, int nvals) {
    __shared__ int s_last, s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        unsigned int g = ld_volatile_u32(&bar->gen);
        __threadfence();
        unsigned int arrived = atomicAdd(&bar->count, 1u);
        s_last = (arrived == gridDim.x - 1);
        if (!s_last) {
            unsigned long long t0 = global_ns();
            unsigned int spins = 0;
            while (ld_volatile_u32(&bar->gen) == g) {
                if ((++spins & 255u) == 0u && global_ns() - t0 > kBarrierTimeoutNs) {
                    set_status(status, DEV_ERR_TIMEOUT);
                    s_ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            __threadfence();
        }
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const int nb = gridDim.x;
        for (int o = threadIdx.x; o < nvals; o += blockDim.x) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int b = 0;
            for (; b + 4 <= nb; b += 4) {
                a0 += __ldcg(part + (size_t)(b + 0) * nvals + o);
                a1 += __ldcg(part + (size_t)(b + 1) * nvals + o);
                a2 += __ldcg(part + (size_t)(b + 2) * nvals + o);
                a3 += __ldcg(part + (size_t)(b + 3) * nvals + o);
            }
            for (; b < nb; ++b) a0 += __ldcg(part + (size_t)b * nvals + o);
            sums[o] = (a0 + a1) + (a2 + a3);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && ld_volatile_i32(status) == DEV_ERR_TIMEOUT) s_ok = 0;
    __syncthreads();
    return s_ok != 0;
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

// Lane-vector helpers shared by the fine sweep and the harmonic solves:
// V adjacent lanes of one row as one vector access, and the fixed-order
// in-block reduction over the row groups of each lane.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace pppc {

// Rows with more nonzeros are multiplied by the whole block (see long_rows).
constexpr int kLongRow = 32;

// V adjacent lanes of one row, loaded and stored as one vector access.
template <typename T, int V>
struct Lanes {
    T v[V];
};
template <typename T, int V>
__device__ __forceinline__ Lanes<T, V> ldv(const T* p) {
    Lanes<T, V> r;
    if constexpr (sizeof(T) * V == 16 && sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else {
#pragma unroll
        for (int h = 0; h < V; h += 2) {
            const auto q = *reinterpret_cast<const typename vec2_t<T>::type*>(p + h);
            r.v[h] = q.x;
            r.v[h + 1] = q.y;
        }
    }
    return r;
}
template <typename T, int V>
__device__ __forceinline__ void stv(T* p, const Lanes<T, V>& x) {
    if constexpr (sizeof(T) * V == 16 && sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
    } else {
#pragma unroll
        for (int h = 0; h < V; h += 2) st2<T>(p + h, x.v[h], x.v[h + 1]);
    }
}

// Slots of the in-block reduction scratch per value and lane: one per warp
// when the row groups of a warp can be combined by shuffles, else one per
// row group.
__host__ __device__ inline int red_slots(int G, int threads) {
    return (G < 32 && (32 % G) == 0) || G == 32 ? threads / 32 : threads / G;
}

// Fixed-order in-block reduction over the row groups of each lane, written as
// this block's partials out[v * NB + lane].  When a
// warp holds several row groups (G < 32 threads per row) they are first
// combined with a fixed shuffle tree; the per-warp results are then summed in
// warp order by one thread per (value, lane).  s_red must hold
// NVP * (blockDim/32) * NB values (NVP * blockDim/G in the general case).
template <typename RT, int V, int NVP>
__device__ __forceinline__ void block_partials(RT* s_red, int G, int NB, int l0, RT (&v)[NVP][V], RT* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (G < 32 && (32 % G) == 0) {
#pragma unroll
        for (int q = 0; q < NVP; ++q)
#pragma unroll
            for (int h = 0; h < V; ++h)
                for (int off = 16; off >= G; off >>= 1) v[q][h] += __shfl_xor_sync(0xffffffffu, v[q][h], off);
        if (lane < G)
#pragma unroll
            for (int q = 0; q < NVP; ++q)
#pragma unroll
                for (int h = 0; h < V; ++h) s_red[(q * nwarps + warp) * NB + l0 + h] = v[q][h];
        __syncthreads();
        for (int o = threadIdx.x; o < NVP * NB; o += blockDim.x) {
            const int q = o / NB, l = o - q * NB;
            RT acc = 0;
            for (int t = 0; t < nwarps; ++t) acc += s_red[(q * nwarps + t) * NB + l];
            out[o] = acc;
        }
        return;
    }
    // general case: one slot per row group, pairwise tree
    const int RB = blockDim.x / G, rb = threadIdx.x / G;
#pragma unroll
    for (int q = 0; q < NVP; ++q)
#pragma unroll
        for (int h = 0; h < V; ++h) s_red[(q * RB + rb) * NB + l0 + h] = v[q][h];
    __syncthreads();
    for (int n = RB; n > 1;) {
        const int half = (n + 1) >> 1, cnt = (n - half) * NB;
        for (int idx = threadIdx.x; idx < NVP * cnt; idx += blockDim.x) {
            const int q = idx / cnt, rem = idx - q * cnt;
            const int t = rem / NB, l = rem - t * NB;
            s_red[(q * RB + t) * NB + l] += s_red[(q * RB + t + half) * NB + l];
        }
        __syncthreads();
        n = half;
    }
    for (int o = threadIdx.x; o < NVP * NB; o += blockDim.x) {
        const int q = o / NB, l = o - q * NB;
        out[o] = s_red[(q * RB) * NB + l];
    }
}

}  // namespace pppc

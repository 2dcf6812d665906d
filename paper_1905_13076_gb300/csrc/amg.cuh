// Device side of the multigrid preconditioner (setup in amg_host.cpp), used
// by the fine PCG (fine.cu, precond = 2) and by the harmonic solves
// (coarse.cu).  Every function is called by all threads of all blocks of a
// team; the team's grid barrier separates steps that read other blocks' rows.
#pragma once
#include <cuda_runtime.h>

#include "args.h"
#include "common.cuh"
#include "lanes.cuh"

namespace pppc {

// What a V-cycle needs from its caller: the team's lanes (row stride of all
// its vectors), levels, coarsest sweeps, workspace, the fine level's
// per-lane special-row values, the team barrier and status word, the long
// rows of each block's own fine rows, and the block's rows of every coarse
// level.
struct AmgCtx {
    int NB, levels, sweeps;
    void* ws;
    const void* J;
    GridBarrier* bar;
    int* status;
    const int* long_start;
    const int* long_rows;
    const int2* rng;   // [levels] this block's rows [x, y) of every coarse level (amg_block_ranges)
};

// ---- multigrid preconditioner (precond = 2) -------------------------------
// z = B r with B one V-cycle over the levels of amg_host.cpp: l1-Jacobi
// smoothing (y = D_l1^-1 b, D_l1 = diag(sum_j |a_ij|), which converges for
// every SPD matrix), R_l = P_l^T, Galerkin coarse matrices of the lane's own
// Jacobian and amg_sweeps l1-Jacobi sweeps on the coarsest level; with the
// same smoother before and after the coarse correction, B is symmetric
// positive definite for every lane.  All vectors are [row][NB] in the
// team's workspace; team barriers separate the steps that read other
// blocks' rows.

// acc += sum_k w[k] x[idx[k]] over k = kb, kb + S, kb + 2S, ... < ke (S = 1:
// the whole row) for this thread's V lanes, with shared scalar weights; four
// gathers are issued before any is consumed (the rows of the coarse levels
// and of R are long, and a gather that waits for its index and then its
// vector would serialise on memory latency), and the last 1-3 entries form
// one more such group (a 7-entry fine row takes two rounds of loads, not
// four); its unused places reload the group's first entry.
template <typename T, int V>
__device__ __forceinline__ void gather_shared(T (&acc)[V], int kb, int ke, const int* __restrict__ idx,
                                              const T* __restrict__ w, const T* x, int NB, int l0, int S = 1) {
    int k = kb;
    for (; k + 3 * S < ke; k += 4 * S) {
        const int i0 = idx[k], i1 = idx[k + S], i2 = idx[k + 2 * S], i3 = idx[k + 3 * S];
        const T w0 = w[k], w1 = w[k + S], w2 = w[k + 2 * S], w3 = w[k + 3 * S];
        const Lanes<T, V> x0 = ldv<T, V>(x + (size_t)i0 * NB + l0);
        const Lanes<T, V> x1 = ldv<T, V>(x + (size_t)i1 * NB + l0);
        const Lanes<T, V> x2 = ldv<T, V>(x + (size_t)i2 * NB + l0);
        const Lanes<T, V> x3 = ldv<T, V>(x + (size_t)i3 * NB + l0);
#pragma unroll
        for (int h = 0; h < V; ++h) acc[h] += (w0 * x0.v[h] + w1 * x1.v[h]) + (w2 * x2.v[h] + w3 * x3.v[h]);
    }
    if (k < ke) {
        const bool h1 = k + S < ke, h2 = k + 2 * S < ke;
        const int k1 = h1 ? k + S : k, k2 = h2 ? k + 2 * S : k;
        const int i0 = idx[k], i1 = idx[k1], i2 = idx[k2];
        const T w0 = w[k], w1 = w[k1], w2 = w[k2];
        const Lanes<T, V> x0 = ldv<T, V>(x + (size_t)i0 * NB + l0);
        const Lanes<T, V> x1 = ldv<T, V>(x + (size_t)i1 * NB + l0);
        const Lanes<T, V> x2 = ldv<T, V>(x + (size_t)i2 * NB + l0);
#pragma unroll
        for (int h = 0; h < V; ++h) {
            T t = w0 * x0.v[h];
            if (h1) t += w1 * x1.v[h];
            if (h2) t += w2 * x2.v[h];
            acc[h] += t;
        }
    }
}

// Same with per-lane weights wl[(s0 + k - kb) NB + l0 ..] (a special row's slots).
template <typename T, int V>
__device__ __forceinline__ void gather_lanes(T (&acc)[V], int kb, int ke, const int* __restrict__ idx, const T* wl,
                                             int s0, const T* x, int NB, int l0, int S = 1) {
    const T* wr = wl + (size_t)(s0 - kb) * NB + l0;
    int k = kb;
    for (; k + 3 * S < ke; k += 4 * S) {
        const int i0 = idx[k], i1 = idx[k + S], i2 = idx[k + 2 * S], i3 = idx[k + 3 * S];
        const Lanes<T, V> w0 = ldv<T, V>(wr + (size_t)k * NB);
        const Lanes<T, V> w1 = ldv<T, V>(wr + (size_t)(k + S) * NB);
        const Lanes<T, V> w2 = ldv<T, V>(wr + (size_t)(k + 2 * S) * NB);
        const Lanes<T, V> w3 = ldv<T, V>(wr + (size_t)(k + 3 * S) * NB);
        const Lanes<T, V> x0 = ldv<T, V>(x + (size_t)i0 * NB + l0);
        const Lanes<T, V> x1 = ldv<T, V>(x + (size_t)i1 * NB + l0);
        const Lanes<T, V> x2 = ldv<T, V>(x + (size_t)i2 * NB + l0);
        const Lanes<T, V> x3 = ldv<T, V>(x + (size_t)i3 * NB + l0);
#pragma unroll
        for (int h = 0; h < V; ++h)
            acc[h] += (w0.v[h] * x0.v[h] + w1.v[h] * x1.v[h]) + (w2.v[h] * x2.v[h] + w3.v[h] * x3.v[h]);
    }
    if (k < ke) {
        const bool h1 = k + S < ke, h2 = k + 2 * S < ke;
        const int k1 = h1 ? k + S : k, k2 = h2 ? k + 2 * S : k;
        const int i0 = idx[k], i1 = idx[k1], i2 = idx[k2];
        const Lanes<T, V> w0 = ldv<T, V>(wr + (size_t)k * NB);
        const Lanes<T, V> w1 = ldv<T, V>(wr + (size_t)k1 * NB);
        const Lanes<T, V> w2 = ldv<T, V>(wr + (size_t)k2 * NB);
        const Lanes<T, V> x0 = ldv<T, V>(x + (size_t)i0 * NB + l0);
        const Lanes<T, V> x1 = ldv<T, V>(x + (size_t)i1 * NB + l0);
        const Lanes<T, V> x2 = ldv<T, V>(x + (size_t)i2 * NB + l0);
#pragma unroll
        for (int h = 0; h < V; ++h) {
            T t = w0.v[h] * x0.v[h];
            if (h1) t += w1.v[h] * x1.v[h];
            if (h2) t += w2.v[h] * x2.v[h];
            acc[h] += t;
        }
    }
}

// Row groups per row on a coarse level: a block owns `rows` rows and RB row
// groups of G threads.  When the rows are few against RB (the deep levels,
// where a row is long and most groups would idle), S groups of one warp
// share a row, each summing every S-th entry, and combine with shuffles.  S
// is a power of two with S G dividing 32 (G must divide 32: otherwise 1).
// Each doubling is taken only if it shortens the longest queue of row
// shares, ceil(rows / (RB / S)) / S, by 10% or more: with many rows per
// group the ceilings differ by a row at most, and a split row pays its
// per-row loads and the shuffles S times.
__device__ __forceinline__ int row_split(int rows, int RB, int G) {
    if (G <= 0 || 32 % G != 0 || rows <= 0) return 1;
    int best = 1;
    long long best_q = (rows + RB - 1) / RB;
    for (int S = 2; S * G <= 32 && RB % S == 0; S <<= 1) {
        const int segs = RB / S;
        const long long q = (rows + segs - 1) / segs;
        if (10 * q * best > 9 * best_q * S) break;
        best = S;
        best_q = q;
    }
    return best;
}

// acc summed over the S row groups of this thread's segment (xor butterfly
// over lane offsets G, 2G, ..., within one warp); every lane ends with the
// row's sum.
template <typename T, int V>
__device__ __forceinline__ void segment_sum(T (&acc)[V], int S, int G) {
    if (S == 1) return;
    const int width = S * G;
    const int lane = threadIdx.x & 31;
    const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u) << (lane & ~(width - 1));
    for (int o = G; o < width; o <<= 1)
#pragma unroll
        for (int h = 0; h < V; ++h) acc[h] += __shfl_xor_sync(mask, acc[h], o);
}

// First row r in [0, n] with cost[r] >= target (cost strictly increasing).
__device__ __forceinline__ int cost_bound(const long long* cost, int n, long long target) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cost[mid] < target)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Rows of every coarse level owned by block bid of a team of nblk: equal
// shares of the level's work (its prefix AmgLevel::cost), so that the long
// rows around a mesh's high-degree nodes, which the aggregation numbers
// first, do not all fall to one block.  Consecutive blocks' ranges tile
// [0, n).  Called once per launch by all threads of the block (ends with a
// block barrier); rng[0] is unused.
__device__ __forceinline__ void amg_block_ranges(const AmgLevel* lvl, int levels, int bid, int nblk, int2* rng) {
    const int t = threadIdx.x;
    if (t < 2 * levels) {
        const int l = t >> 1, side = t & 1;
        int v = 0;
        if (l >= 1) {
            const AmgLevel& lv = lvl[l];
            v = cost_bound(lv.cost, lv.n, lv.cost[lv.n] * (bid + side) / nblk);
        }
        if (side)
            rng[l].y = v;
        else
            rng[l].x = v;
    }
    __syncthreads();
}

// 1 / D_l1 of row i of a level for this thread's lanes (per lane on special rows).
template <typename T, int V>
__device__ __forceinline__ Lanes<T, V> inv_l1(const AmgLevel& lv, const T* l1sp, int i, int NB, int l0) {
    Lanes<T, V> d;
    const int sp = lv.sp_index[i];
    if (sp >= 0) {
        d = ldv<T, V>(l1sp + (size_t)sp * NB + l0);
#pragma unroll
        for (int h = 0; h < V; ++h) d.v[h] = (T)1 / d.v[h];
    } else {
        const T v = (T)1 / static_cast<const T*>(lv.l1)[i];
#pragma unroll
        for (int h = 0; h < V; ++h) d.v[h] = v;
    }
    return d;
}

// Every lane's coarse matrices from its fine Jacobian (a.J, just assembled):
// per level, slot e = slot_base[e] + sum cw * (finer slots), then the l1
// norms of the special rows.  Called by all blocks of the team after a
// barrier that made the Jacobian visible; ends without a barrier (the
// values are read only after the V-cycle's first barriers).
template <typename T, int V>
__device__ bool amg_coarse_values(const AmgCtx& a, const AmgLevel* lvl, int bid, int nblk) {
    const int NB = a.NB, G = NB / V;
    T* ws = static_cast<T*>(a.ws);
    const long long gthreads = (long long)nblk * blockDim.x;
    for (int l = 1; l < a.levels; ++l) {
        const AmgLevel& lv = lvl[l];
        const T* src = l == 1 ? static_cast<const T*>(a.J) : ws + lvl[l - 1].off_slot * NB;
        T* dst = ws + lv.off_slot * NB;
        const T* base = static_cast<const T*>(lv.slot_base);
        const T* cw = static_cast<const T*>(lv.cw);
        const long long items = (long long)lv.n_slots * G;
        for (long long it = bid * (long long)blockDim.x + threadIdx.x; it < items; it += gthreads) {
            const int e = (int)(it / G), lg = (int)(it % G) * V;
            Lanes<T, V> acc;
#pragma unroll
            for (int h = 0; h < V; ++h) acc.v[h] = base[e];
            T sum[V];
#pragma unroll
            for (int h = 0; h < V; ++h) sum[h] = (T)0;
            gather_shared<T, V>(sum, lv.cptr[e], lv.cptr[e + 1], lv.csrc, cw, src, NB, lg);
#pragma unroll
            for (int h = 0; h < V; ++h) acc.v[h] += sum[h];
            stv<T, V>(dst + (size_t)e * NB + lg, acc);
        }
        if (!grid_sync(a.bar, a.status, bid, nblk)) return false;
        T* l1sp = ws + lv.off_l1 * NB;
        const long long ritems = (long long)lv.n_sp * G;
        for (long long it = bid * (long long)blockDim.x + threadIdx.x; it < ritems; it += gthreads) {
            const int isp = (int)(it / G), lg = (int)(it % G) * V;
            const int row = lv.sp_rows[isp];
            const int s0 = lv.row_slot[row], kb = lv.rowptr[row], ke = lv.rowptr[row + 1];
            Lanes<T, V> acc;
#pragma unroll
            for (int h = 0; h < V; ++h) acc.v[h] = (T)0;
            for (int k = kb; k < ke; ++k) {
                const Lanes<T, V> v = ldv<T, V>(dst + (size_t)(s0 + k - kb) * NB + lg);
#pragma unroll
                for (int h = 0; h < V; ++h) acc.v[h] += v.v[h] < (T)0 ? -v.v[h] : v.v[h];
            }
            stv<T, V>(l1sp + (size_t)isp * NB + lg, acc);
        }
    }
    return true;
}

// Fine level, the block's own rows: out = b - J x (mode 0) or
// x + (b - J x) / D_l1 (mode 1); long rows are summed by the whole block.
template <typename T, int V>
__device__ __noinline__ void amg_fine_resid(const AmgCtx& a, const MeshDev& m, const AmgLevel& lv0, const T* KlinT,
                                            const T* J, const T* l1sp, int mode, const T* x, const T* b, T* out,
                                            int re, int row0, int RB, int rb, int l0, int G, T* s_red, T* s_tmp,
                                            int bid) {
    const int NB = a.NB;
    for (int i = row0; i < re; i += RB) {
        const int kb = m.rowptr[i], ke = m.rowptr[i + 1];
        if (ke - kb > kLongRow) continue;
        const int slot0 = m.row_slot[i];
        T acc[V];
#pragma unroll
        for (int h = 0; h < V; ++h) acc[h] = 0;
        if (slot0 < 0)
            gather_shared<T, V>(acc, kb, ke, m.col, KlinT, x, NB, l0);
        else
            gather_lanes<T, V>(acc, kb, ke, m.col, J, slot0, x, NB, l0);
        const size_t o = (size_t)i * NB + l0;
        const Lanes<T, V> bi = ldv<T, V>(b + o);
        Lanes<T, V> res;
        if (mode == 0) {
#pragma unroll
            for (int h = 0; h < V; ++h) res.v[h] = bi.v[h] - acc[h];
        } else {
            const Lanes<T, V> xi = ldv<T, V>(x + o);
            const Lanes<T, V> d = inv_l1<T, V>(lv0, l1sp, i, NB, l0);
#pragma unroll
            for (int h = 0; h < V; ++h) res.v[h] = xi.v[h] + (bi.v[h] - acc[h]) * d.v[h];
        }
        stv<T, V>(out + o, res);
    }
    for (int lr = a.long_start[bid]; lr < a.long_start[bid + 1]; ++lr) {
        const int i = a.long_rows[lr];
        const int kb = m.rowptr[i], ke = m.rowptr[i + 1], slot0 = m.row_slot[i];
        T vv[1][V];
#pragma unroll
        for (int h = 0; h < V; ++h) vv[0][h] = 0;
        for (int kk = kb + rb; kk < ke; kk += RB) {
            const Lanes<T, V> xj = ldv<T, V>(x + (size_t)m.col[kk] * NB + l0);
            if (slot0 < 0) {
                const T kv = KlinT[kk];
#pragma unroll
                for (int h = 0; h < V; ++h) vv[0][h] += kv * xj.v[h];
            } else {
                const Lanes<T, V> jv = ldv<T, V>(J + (size_t)(slot0 + kk - kb) * NB + l0);
#pragma unroll
                for (int h = 0; h < V; ++h) vv[0][h] += jv.v[h] * xj.v[h];
            }
        }
        block_partials<T, V, 1>(s_red, G, NB, l0, vv, s_tmp);
        __syncthreads();
        if (rb == 0) {
            const size_t o = (size_t)i * NB + l0;
            const Lanes<T, V> bi = ldv<T, V>(b + o);
            Lanes<T, V> res;
            if (mode == 0) {
#pragma unroll
                for (int h = 0; h < V; ++h) res.v[h] = bi.v[h] - s_tmp[l0 + h];
            } else {
                const Lanes<T, V> xi = ldv<T, V>(x + o);
                const Lanes<T, V> d = inv_l1<T, V>(lv0, l1sp, i, NB, l0);
#pragma unroll
                for (int h = 0; h < V; ++h) res.v[h] = xi.v[h] + (bi.v[h] - s_tmp[l0 + h]) * d.v[h];
            }
            stv<T, V>(out + o, res);
        }
        __syncthreads();
    }
}

// Coarse level l >= 1, rows [lo, hi): out = b - A_l x (mode 0) or
// x + (b - A_l x) / D_l1 (mode 1).
template <typename T, int V>
__device__ __noinline__ void amg_coarse_resid(const AmgLevel& lv, const T* slots, const T* l1sp, int mode, const T* x,
                                              const T* b, T* out, int lo, int hi, int RB, int rb, int l0, int NB) {
    const T* val = static_cast<const T*>(lv.val);
    const int G = NB / V, S = row_split(hi - lo, RB, G), seg = rb / S, sub = rb - seg * S, NS = RB / S;
    for (int c = lo + seg; c < hi; c += NS) {
        const int kb = lv.rowptr[c], ke = lv.rowptr[c + 1], s0 = lv.row_slot[c];
        T acc[V];
#pragma unroll
        for (int h = 0; h < V; ++h) acc[h] = 0;
        if (S == 1) {   // the whole row: the stride folds away
            if (s0 < 0)
                gather_shared<T, V>(acc, kb, ke, lv.col, val, x, NB, l0);
            else
                gather_lanes<T, V>(acc, kb, ke, lv.col, slots, s0, x, NB, l0);
        } else {
            if (s0 < 0)
                gather_shared<T, V>(acc, kb + sub, ke, lv.col, val, x, NB, l0, S);
            else
                gather_lanes<T, V>(acc, kb + sub, ke, lv.col, slots + (size_t)sub * NB, s0, x, NB, l0, S);
            segment_sum<T, V>(acc, S, G);
        }
        if (sub != 0) continue;
        const size_t o = (size_t)c * NB + l0;
        const Lanes<T, V> bi = ldv<T, V>(b + o);
        Lanes<T, V> res;
        if (mode == 0) {
#pragma unroll
            for (int h = 0; h < V; ++h) res.v[h] = bi.v[h] - acc[h];
        } else {
            const Lanes<T, V> xi = ldv<T, V>(x + o);
            const Lanes<T, V> d = inv_l1<T, V>(lv, l1sp, c, NB, l0);
#pragma unroll
            for (int h = 0; h < V; ++h) res.v[h] = xi.v[h] + (bi.v[h] - acc[h]) * d.v[h];
        }
        stv<T, V>(out + o, res);
    }
}

// Level l >= 1, rows [lo, hi): b = R_l q (q of level l - 1), y = b / D_l1.
template <typename T, int V>
__device__ __noinline__ void amg_restrict(const AmgLevel& lv, const T* q, T* b, T* y, const T* l1sp, int lo, int hi,
                                          int RB, int rb, int l0, int NB) {
    const T* Rv = static_cast<const T*>(lv.Rval);
    const int G = NB / V, S = row_split(hi - lo, RB, G), seg = rb / S, sub = rb - seg * S, NS = RB / S;
    for (int c = lo + seg; c < hi; c += NS) {
        T acc[V];
#pragma unroll
        for (int h = 0; h < V; ++h) acc[h] = 0;
        if (S == 1) {
            gather_shared<T, V>(acc, lv.Rptr[c], lv.Rptr[c + 1], lv.Rcol, Rv, q, NB, l0);
        } else {
            gather_shared<T, V>(acc, lv.Rptr[c] + sub, lv.Rptr[c + 1], lv.Rcol, Rv, q, NB, l0, S);
            segment_sum<T, V>(acc, S, G);
        }
        if (sub != 0) continue;
        const size_t o = (size_t)c * NB + l0;
        const Lanes<T, V> d = inv_l1<T, V>(lv, l1sp, c, NB, l0);
        Lanes<T, V> bv, yv;
#pragma unroll
        for (int h = 0; h < V; ++h) {
            bv.v[h] = acc[h];
            yv.v[h] = acc[h] * d.v[h];
        }
        stv<T, V>(b + o, bv);
        stv<T, V>(y + o, yv);
    }
}

// y += P xc on the rows first, first + RB, ... < hi of the finer level, with
// P = P_{l+1} held by the coarser level's descriptor lc.
template <typename T, int V>
__device__ __noinline__ void amg_prolong(const AmgLevel& lc, const T* xc, T* y, int first, int hi, int RB, int l0,
                                         int NB) {
    const T* Pv = static_cast<const T*>(lc.Pval);
    for (int i = first; i < hi; i += RB) {
        const size_t o = (size_t)i * NB + l0;
        Lanes<T, V> yi = ldv<T, V>(y + o);
        T acc[V];
#pragma unroll
        for (int h = 0; h < V; ++h) acc[h] = 0;
        gather_shared<T, V>(acc, lc.Pptr[i], lc.Pptr[i + 1], lc.Pcol, Pv, xc, NB, l0);
#pragma unroll
        for (int h = 0; h < V; ++h) yi.v[h] += acc[h];
        stv<T, V>(y + o, yi);
    }
}

// z = B r, one V-cycle (see above), on the team's rows: the block's own fine
// rows [rs, re) and its share a.rng of every coarse level.  Every thread of
// the block must belong to a row group (blockDim a multiple of G = NB / V):
// a thread with rb >= RB would repeat another group's rows, and the
// prolongation's y += P x would then add twice.  r must be final on
// the block's own rows; z is final on them at return (the caller's barrier
// publishes it).  Returns false if a team barrier timed out.
template <typename T, int V>
__device__ bool amg_vcycle(const AmgCtx& a, const MeshDev& m, const AmgLevel* lvl, const T* KlinT, const T* J,
                           const T* r, T* z, int bid, int nblk, int re, int row0, int RB, int rb, int l0, int G,
                           T* s_red, T* s_tmp) {
    const int NB = a.NB, L = a.levels;
    T* ws = static_cast<T*>(a.ws);
    auto at = [&](long long off) { return ws + off * NB; };
#define AMG_SYNC \
    if (!grid_sync(a.bar, a.status, bid, nblk)) return false
    const AmgLevel& f = lvl[0];
    T* y0 = at(f.off_y);
    const T* l1f = at(f.off_l1);
    // down: fine level, y0 = r / D_l1, q0 = r - J y0 (kept in z)
    for (int i = row0; i < re; i += RB) {
        const size_t o = (size_t)i * NB + l0;
        const Lanes<T, V> ri = ldv<T, V>(r + o);
        const Lanes<T, V> d = inv_l1<T, V>(f, l1f, i, NB, l0);
        Lanes<T, V> yv;
#pragma unroll
        for (int h = 0; h < V; ++h) yv.v[h] = ri.v[h] * d.v[h];
        stv<T, V>(y0 + o, yv);
    }
    AMG_SYNC;
    amg_fine_resid<T, V>(a, m, f, KlinT, J, l1f, 0, y0, r, z, re, row0, RB, rb, l0, G, s_red, s_tmp, bid);
    AMG_SYNC;
    const T* qprev = z;
    int lo = 0, hi = 0;
    for (int l = 1; l < L - 1; ++l) {
        const AmgLevel& lv = lvl[l];
        lo = a.rng[l].x;
        hi = a.rng[l].y;
        amg_restrict<T, V>(lv, qprev, at(lv.off_b), at(lv.off_y), at(lv.off_l1), lo, hi, RB, rb, l0, NB);
        AMG_SYNC;
        amg_coarse_resid<T, V>(lv, at(lv.off_slot), at(lv.off_l1), 0, at(lv.off_y), at(lv.off_b), at(lv.off_q), lo, hi,
                               RB, rb, l0, NB);
        AMG_SYNC;
        qprev = at(lv.off_q);
    }
    // coarsest level: amg_sweeps l1-Jacobi sweeps from zero
    const AmgLevel& lc = lvl[L - 1];
    lo = a.rng[L - 1].x;
    hi = a.rng[L - 1].y;
    T* cur = at(lc.off_y);
    T* nxt = at(lc.off_q);
    amg_restrict<T, V>(lc, qprev, at(lc.off_b), cur, at(lc.off_l1), lo, hi, RB, rb, l0, NB);
    for (int sw = 1; sw < a.sweeps; ++sw) {
        AMG_SYNC;
        amg_coarse_resid<T, V>(lc, at(lc.off_slot), at(lc.off_l1), 1, cur, at(lc.off_b), nxt, lo, hi, RB, rb, l0, NB);
        T* t = cur;
        cur = nxt;
        nxt = t;
    }
    const T* xc = cur;
    // up: y_l += P_{l+1} x_{l+1}, then x_l = y_l + (b_l - A_l y_l) / D_l1 (kept in q_l)
    for (int l = L - 2; l >= 1; --l) {
        const AmgLevel& lv = lvl[l];
        lo = a.rng[l].x;
        hi = a.rng[l].y;
        AMG_SYNC;
        amg_prolong<T, V>(lvl[l + 1], xc, at(lv.off_y), lo + rb, hi, RB, l0, NB);
        AMG_SYNC;
        amg_coarse_resid<T, V>(lv, at(lv.off_slot), at(lv.off_l1), 1, at(lv.off_y), at(lv.off_b), at(lv.off_q), lo, hi,
                               RB, rb, l0, NB);
        xc = at(lv.off_q);
    }
    AMG_SYNC;
    amg_prolong<T, V>(lvl[1], xc, y0, row0, re, RB, l0, NB);
    AMG_SYNC;
    amg_fine_resid<T, V>(a, m, f, KlinT, J, l1f, 1, y0, r, z, re, row0, RB, rb, l0, G, s_red, s_tmp, bid);
#undef AMG_SYNC
    return true;
}

}  // namespace pppc

// Coarse part of one PP-PC iteration (Sec. 2, Eq. 4 with the implicit-Euler
// coarse step of Eq. 8; the block-cyclic system of Eqs. 9-10 solved by the
// multi-harmonic method of Sec. 3, Eqs. 11-14).
//
// With G linear in its argument (coarse stiffness Kbar frozen within the
// iteration), subtracting Eq. 9 at U^k from Eq. 9 at U^{k+1} gives, for the
// update D_n = U_n^{k+1} - U_n^k and the jumps d_n = F_n(U_{n-1}^k) - U_n^k,
//     Q D_n - C D_{n-1} = Q d_n   (n cyclic),   C = M/dT,  Q = C + Kbar,
// where the source terms f(T_n) cancel.  The DFT along n (forward sign
// exp(-i 2 pi p n / N), unnormalised; inverse with 1/N) turns it into one
// independent shifted system per harmonic p:
//     (Kbar + (1 - z_p) C) Dhat_p = Q dhat_p,   z_p = exp(-i 2 pi p / N).
// Writing Dhat_p = dhat_p + W_p,
//     (Kbar + (1 - z_p) C) W_p = z_p C dhat_p = DFT_p[ C d_{n-1} ],
// whose right-hand side lives only on rows of the conductive region.  Then
//     U_n^{k+1} = U_n^k + d_n + w_n = F_n(U_{n-1}^k) + w_n,  w = IDFT(W).
// For real data only p = 0..N/2 are solved (Hermitian symmetry); each system
// is complex symmetric and is solved by Jacobi-preconditioned COCG (the
// conjugate-orthogonal CG), all harmonics in one cooperative launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "amg.cuh"
#include "common.cuh"
#include "kernels.h"

namespace pppc {
namespace {

inline int grid_for(long long n, int threads, int cap = 65535) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// ---------------------------------------------------------------- jumps --
constexpr int kJumpBlocks = 512;

__global__ void jumps_kernel(int ndof, int N, int NB, const double* U, const double* F, double* d,
                             double* part) {
    __shared__ double red[2][256];
    double dd = 0.0, ff = 0.0;
    const long long total = (long long)ndof * NB;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(it % NB);
        const long long i = it / NB;
        double v = 0.0;
        if (n < N) {
            const double f = F[i * NB + (n + N - 1) % N];
            v = f - U[it];
            ff += f * f;
        }
        d[it] = v;
        dd += v * v;
    }
    red[0][threadIdx.x] = dd;
    red[1][threadIdx.x] = ff;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = red[0][0];
        part[2 * blockIdx.x + 1] = red[1][0];
    }
}

// sums[v] = sum over the nblocks partial pairs part[2 b + v], v = 0, 1: each
// of 256 threads adds a strided share of the partials, then a fixed-order
// tree in shared memory (deterministic, like every reduction here).
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) sum_pairs_kernel(int nblocks, const double* part, double* sums) {
    __shared__ double red[2][kSumThreads];
    const int t = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int q = t; q < nblocks; q += kSumThreads) {
        a += part[2 * q];
        b += part[2 * q + 1];
    }
    red[0][t] = a;
    red[1][t] = b;
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if (t < w) {
            red[0][t] += red[0][t + w];
            red[1][t] += red[1][t + w];
        }
        __syncthreads();
    }
    if (t < 2) sums[t] = red[t][0];
}

// ------------------------------------------------- coarse linearisation --
// Kbar on the special rows: K_lin plus the nonlinear stiffness frozen as
//   lin 0: (1/N) sum_n dK(U)U/dU at U_n   (c1 ab + c2 s_a s_b)
//   lin 1: (1/N) sum_n K(U_n)             (c1 ab)
//   lin 2: dK(U)U/dU at U = 0             (|e| (k1 + k3) ab)
__global__ void kbar_kernel(MeshDev m, int N, int NB, int lin, const double* E, double* Kbar) {
    const size_t P = (size_t)m.n_nl * NB;
    for (int sl = blockIdx.x * blockDim.x + threadIdx.x; sl < m.n_slots; sl += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int c = m.nlc_ptr[sl]; c < m.nlc_ptr[sl + 1]; ++c) {
            const int pk = m.nlc[c];
            const int q = pk / 9, ia = (pk / 3) % 3, ib = pk % 3;
            const double ab = m.nlc_ab[c];
            if (lin == 2) {
                v += m.nl_geom[8 * (size_t)q] * (m.nl_k[4 * (size_t)q] + m.nl_k[4 * (size_t)q + 2]) * ab;
                continue;
            }
            double sc = 0.0;
            for (int n = 0; n < N; ++n) {
                const size_t o = (size_t)q * NB + n;
                double t = E[o] * ab;
                if (lin == 0) t += E[P + o] * E[(2 + ia) * P + o] * E[(2 + ib) * P + o];
                sc += t;
            }
            v += sc / (double)N;
        }
        Kbar[sl] = m.Klin[m.slot_k[sl]] + v;
    }
}

// ------------------------------------------------ right-hand side + DFT --
// y = C d on the special rows (all lanes), then b_p = sum_n y_{n-1} z_p^n.
__global__ void cd_kernel(MeshDev m, int NB, double inv_dT, const double* d, double* y) {
    const long long total = (long long)m.n_sp * NB;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int sp = (int)(it / NB), n = (int)(it % NB);
        const int i = m.sp_rows[sp];
        const int kb = m.rowptr[i], ke = m.rowptr[i + 1], slot0 = m.row_slot[i];
        double v = 0.0;
        for (int k = kb; k < ke; ++k) v += m.Mslot[slot0 + (k - kb)] * d[(size_t)m.col[k] * NB + n];
        y[it] = v * inv_dT;
    }
}

__global__ void dft_rhs_kernel(int n_sp, int N, int NB, int H, const double* y, const double* tw,
                               double* b) {
    const long long total = (long long)n_sp * H;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int sp = (int)(it / H), p = (int)(it % H);
        const double* ys = y + (size_t)sp * NB;
        double re = 0.0, im = 0.0;
        int k = 0;  // (p * n) mod N
        for (int n = 0; n < N; ++n) {
            const double v = ys[(n + N - 1) % N];
            re += v * tw[2 * k];
            im += v * tw[2 * k + 1];
            k += p;
            if (k >= N) k -= N;
        }
        b[2 * it] = re;
        b[2 * it + 1] = im;
    }
}

// ----------------------------------------------------- COCG, all p at once --
template <typename T> struct cvec;
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<float> { using type = float2; };

template <typename T>
__device__ __forceinline__ cplx ldc(const T* p) {
    const auto v = *reinterpret_cast<const typename cvec<T>::type*>(p);
    return {(double)v.x, (double)v.y};
}
template <typename T>
__device__ __forceinline__ void stc(T* p, cplx v) {
    typename cvec<T>::type o;
    o.x = (T)v.re;
    o.y = (T)v.im;
    *reinterpret_cast<typename cvec<T>::type*>(p) = o;
}

constexpr int CNV = 5;  // per lane: |r|^2, (r,z) re/im, (z,w) re/im

// |1 - z_p| for harmonic p (tw[2p] = cos, tw[2p+1] = -sin of 2 pi p / N)
__device__ __forceinline__ double shift_abs(const double* tw, int p) {
    const double re = 1.0 - tw[2 * p], im = -tw[2 * p + 1];
    return sqrt(re * re + im * im);
}

// Multigrid set-up of one harmonic solve: the special rows' values of S_p
// and their l1 norms (two lanes per harmonic), then every harmonic's coarse
// matrices.  Called by all blocks after a barrier.
template <typename P>
__device__ bool cocg_amg_setup(const CocgArgs& a, const AmgLevel* lvl, int bid, int nblk) {
    const MeshDev& m = a.mesh;
    const int H = a.H, NB = 2 * H;
    P* J = static_cast<P*>(a.amg_J);
    P* l1sp = static_cast<P*>(a.amg_ws) + lvl[0].off_l1 * NB;
    const long long items = (long long)m.n_sp * H;
    for (long long it = bid * (long long)blockDim.x + threadIdx.x; it < items; it += (long long)nblk * blockDim.x) {
        const int sp = (int)(it / H), p = (int)(it % H);
        const int i = m.sp_rows[sp], kb = m.rowptr[i], ke = m.rowptr[i + 1], s0 = m.row_slot[i];
        const double c = shift_abs(a.tw, p) * a.inv_dT;
        P l1 = 0;
        for (int k = kb; k < ke; ++k) {
            const int sl = s0 + (k - kb);
            const P v = (P)(a.Kbar[sl] + c * m.Mslot[sl]);
            J[(size_t)sl * NB + 2 * p] = v;
            J[(size_t)sl * NB + 2 * p + 1] = v;
            l1 += v < (P)0 ? -v : v;
        }
        l1sp[(size_t)sp * NB + 2 * p] = l1;
        l1sp[(size_t)sp * NB + 2 * p + 1] = l1;
    }
    if (!grid_sync(a.bar, a.status, bid, nblk)) return false;
    const AmgCtx ctx{NB,           a.amg_levels, a.amg_sweeps, a.amg_ws, a.amg_J, a.bar, a.status,
                     a.long_start, a.long_rows,  nullptr};
    return amg_coarse_values<P, 2>(ctx, lvl, bid, nblk);
}

// z = B r on the block's contiguous rows: r (FP64, final on every row: the
// caller's barrier) converted to P, one V-cycle, z converted back.  The
// caller's barrier publishes z.  The V-cycle needs blockDim to be a multiple
// of H (cocg_config's single-instance launches are; the batched launch's
// 512-thread blocks are not, and its members' solves take no multigrid
// arguments: cocg_args).
template <typename T, typename P>
__device__ bool cocg_amg_apply(const CocgArgs& a, const AmgLevel* lvl, const int2* rng, const T* r, T* z, int bid,
                               int nblk, int RB, int rb, int pl, double* s_red, double* s_tmp) {
    const MeshDev& m = a.mesh;
    const int H = a.H, NB = 2 * H;
    const int rs = a.row_start[bid], re = a.row_start[bid + 1];
    const int l0 = 2 * pl;
    P* rp = static_cast<P*>(a.amg_r);
    P* zp = static_cast<P*>(a.amg_z);
    if (rb < RB)
        for (int i = rs + rb; i < re; i += RB) {
            const size_t o = (size_t)i * NB + l0;
            rp[o] = (P)r[o];
            rp[o + 1] = (P)r[o + 1];
        }
    const AmgCtx ctx{NB,           a.amg_levels, a.amg_sweeps, a.amg_ws, a.amg_J, a.bar, a.status,
                     a.long_start, a.long_rows,  rng};
    if (!amg_vcycle<P, 2>(ctx, m, lvl, static_cast<const P*>(a.klinP), static_cast<const P*>(a.amg_J), rp, zp, bid,
                          nblk, re, rs + rb, RB, rb, l0, H, reinterpret_cast<P*>(s_red), reinterpret_cast<P*>(s_tmp)))
        return false;
    if (rb < RB)
        for (int i = rs + rb; i < re; i += RB) {
            const size_t o = (size_t)i * NB + l0;
            z[o] = (T)zp[o];
            z[o + 1] = (T)zp[o + 1];
        }
    return true;
}

// The whole solve for one team of nblk blocks (bid = this block's place in
// it): the grid of a single-instance launch, or one member's share of a
// batched launch.  Threads beyond the last whole row group (blockDim not a
// multiple of H) take no rows.
template <typename T>
__device__ __forceinline__ void cocg_body(const CocgArgs& a, const int bid, const int nblk) {
    extern __shared__ double smem[];
    const MeshDev m = a.mesh;
    const int H = a.H;
    const int tid = threadIdx.x, pl = tid % H, rb = tid / H, RB = blockDim.x / H;
    double* s_stop = smem;                 // [H]
    double* s_gold = s_stop + H;           // [2H]
    double* s_aold = s_gold + 2 * H;       // [2H]
    double* s_alpha = s_aold + 2 * H;      // [2H]
    double* s_beta = s_alpha + 2 * H;      // [2H]
    double* s_red = s_beta + 2 * H;        // [CNV][RB][H]
    double* s_sums = s_red + CNV * RB * H; // [CNV][H], identical in every block
    double* s_tmp = s_sums + CNV * H;      // [blockDim]
    int* s_act = reinterpret_cast<int*>(s_tmp + blockDim.x);
    __shared__ int s_err;
    double* part_buf[2] = {a.part, a.part + (size_t)nblk * CNV * H};
    int parity = 0;

    T* x = static_cast<T*>(a.x);
    T* r = static_cast<T*>(a.r);
    T* z = static_cast<T*>(a.z);
    T* w = static_cast<T*>(a.w);
    T* p = static_cast<T*>(a.p);
    T* s = static_cast<T*>(a.s);
    T* invd = static_cast<T*>(a.invd_sp);
    const bool in_group = rb < RB;
    const int rstride = nblk * RB;
    const int row0 = in_group ? bid * RB + rb : m.ndof;
    // shift c_p = 1 - z_p of this thread's harmonic
    const cplx cp = {1.0 - a.tw[2 * pl], -a.tw[2 * pl + 1]};
    long long iters = 0;
    if (tid == 0) s_err = 0;
    if (a.team_ns && bid == 0 && tid == 0) a.team_ns[0] = global_ns();
    // multigrid preconditioner: level descriptors in shared memory
    __shared__ AmgLevel s_amg[kAmgMaxLevels];
    const bool amg = a.amg != nullptr;
    if (amg) {
        const int words = a.amg_levels * (int)(sizeof(AmgLevel) / sizeof(int));
        const int* src = reinterpret_cast<const int*>(a.amg);
        int* dst = reinterpret_cast<int*>(s_amg);
        for (int q = tid; q < words; q += blockDim.x) dst[q] = src[q];
        __syncthreads();
    }
    __shared__ int2 s_rng[kAmgMaxLevels];
    if (amg) amg_block_ranges(s_amg, a.amg_levels, bid, nblk, s_rng);
    // z = B r with the multigrid V-cycle (after a barrier that made r final)
    auto precondition = [&]() -> bool {
        return a.amg_fp32 ? cocg_amg_apply<T, float>(a, s_amg, s_rng, r, z, bid, nblk, RB, rb, pl, s_red, s_tmp)
                          : cocg_amg_apply<T, double>(a, s_amg, s_rng, r, z, bid, nblk, RB, rb, pl, s_red, s_tmp);
    };

    // init: x = p = s = 0, r = b, z = D^-1 r
    for (int i = row0; i < m.ndof; i += rstride) {
        const size_t o = 2 * ((size_t)i * H + pl);
        const int sp = m.sp_index[i];
        cplx rv = {0.0, 0.0}, iv;
        if (sp >= 0) {
            rv = {a.b[2 * ((size_t)sp * H + pl)], a.b[2 * ((size_t)sp * H + pl) + 1]};
            const int sl = m.row_slot[i] + (m.diag_k[i] - m.rowptr[i]);
            const cplx dg = {a.Kbar[sl] + cp.re * m.Mslot[sl] * a.inv_dT, cp.im * m.Mslot[sl] * a.inv_dT};
            iv = cdiv({1.0, 0.0}, dg);
            stc<T>(invd + 2 * ((size_t)sp * H + pl), iv);
        } else {
            iv = {m.invdiag_lin[i], 0.0};
        }
        stc<T>(x + o, {0.0, 0.0});
        stc<T>(p + o, {0.0, 0.0});
        stc<T>(s + o, {0.0, 0.0});
        stc<T>(r + o, rv);
        stc<T>(z + o, cmul(iv, rv));
    }
    if (!grid_sync(a.bar, a.status, bid, nblk)) return;
    if (amg) {
        const bool ok = a.amg_fp32 ? cocg_amg_setup<float>(a, s_amg, bid, nblk)
                                   : cocg_amg_setup<double>(a, s_amg, bid, nblk);
        if (!ok || !precondition()) return;
        if (!grid_sync(a.bar, a.status, bid, nblk)) return;
    }

    for (int k = 0;; ++k) {
        double acc[CNV] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = row0; i < m.ndof; i += rstride) {
            const int kb = m.rowptr[i], ke = m.rowptr[i + 1], slot0 = m.row_slot[i];
            cplx wv = {0.0, 0.0};
            if (slot0 < 0) {
                // four gathers in flight: a block serves few rows per pass,
                // so each thread's chain of loads sets the pace
                int kk = kb;
                for (; kk + 3 < ke; kk += 4) {
                    const int c0 = m.col[kk], c1 = m.col[kk + 1], c2 = m.col[kk + 2], c3 = m.col[kk + 3];
                    const double k0 = m.Klin[kk], k1 = m.Klin[kk + 1], k2 = m.Klin[kk + 2], k3 = m.Klin[kk + 3];
                    const cplx z0 = ldc<T>(z + 2 * ((size_t)c0 * H + pl));
                    const cplx z1 = ldc<T>(z + 2 * ((size_t)c1 * H + pl));
                    const cplx z2 = ldc<T>(z + 2 * ((size_t)c2 * H + pl));
                    const cplx z3 = ldc<T>(z + 2 * ((size_t)c3 * H + pl));
                    wv.re += (k0 * z0.re + k1 * z1.re) + (k2 * z2.re + k3 * z3.re);
                    wv.im += (k0 * z0.im + k1 * z1.im) + (k2 * z2.im + k3 * z3.im);
                }
                if (kk < ke) {   // the last 1-3 entries as one more group
                    const int nr = ke - kk;
                    const int k1 = nr > 1 ? kk + 1 : kk, k2 = nr > 2 ? kk + 2 : kk;
                    const int c0 = m.col[kk], c1 = m.col[k1], c2 = m.col[k2];
                    const double q0 = m.Klin[kk], q1 = m.Klin[k1], q2 = m.Klin[k2];
                    const cplx z0 = ldc<T>(z + 2 * ((size_t)c0 * H + pl));
                    const cplx z1 = ldc<T>(z + 2 * ((size_t)c1 * H + pl));
                    const cplx z2 = ldc<T>(z + 2 * ((size_t)c2 * H + pl));
                    double tr = q0 * z0.re, ti = q0 * z0.im;
                    if (nr > 1) {
                        tr += q1 * z1.re;
                        ti += q1 * z1.im;
                    }
                    if (nr > 2) {
                        tr += q2 * z2.re;
                        ti += q2 * z2.im;
                    }
                    wv.re += tr;
                    wv.im += ti;
                }
            } else {
                int kk = kb;
                for (; kk + 1 < ke; kk += 2) {
                    const int sl = slot0 + (kk - kb);
                    const cplx z0 = ldc<T>(z + 2 * ((size_t)m.col[kk] * H + pl));
                    const cplx z1 = ldc<T>(z + 2 * ((size_t)m.col[kk + 1] * H + pl));
                    const double m0 = m.Mslot[sl] * a.inv_dT, m1 = m.Mslot[sl + 1] * a.inv_dT;
                    const cplx a0 = {a.Kbar[sl] + cp.re * m0, cp.im * m0};
                    const cplx a1 = {a.Kbar[sl + 1] + cp.re * m1, cp.im * m1};
                    wv = cadd(wv, cadd(cmul(a0, z0), cmul(a1, z1)));
                }
                for (; kk < ke; ++kk) {
                    const int sl = slot0 + (kk - kb);
                    const double mv = m.Mslot[sl] * a.inv_dT;
                    const cplx av = {a.Kbar[sl] + cp.re * mv, cp.im * mv};
                    wv = cadd(wv, cmul(av, ldc<T>(z + 2 * ((size_t)m.col[kk] * H + pl))));
                }
            }
            const size_t o = 2 * ((size_t)i * H + pl);
            stc<T>(w + o, wv);
            const cplx wr = ldc<T>(w + o);   // the stored (rounded) w
            const cplx ri = ldc<T>(r + o);
            const cplx zi = ldc<T>(z + o);
            acc[0] += cabs2(ri);
            const cplx rz = cmul(ri, zi), zw = cmul(zi, wr);
            acc[1] += rz.re;
            acc[2] += rz.im;
            acc[3] += zw.re;
            acc[4] += zw.im;
        }
#pragma unroll
        for (int q = 0; q < CNV; ++q)
            if (in_group) s_red[(q * RB + rb) * H + pl] = acc[q];
        __syncthreads();
        double* out = part_buf[parity] + (size_t)bid * CNV * H;
        for (int o = tid; o < CNV * H; o += blockDim.x) {
            const int q = o / H, l = o - q * H;
            double sum = 0.0;
            for (int t = 0; t < RB; ++t) sum += s_red[(q * RB + t) * H + l];
            out[o] = sum;
        }
        if (!grid_sync(a.bar, a.status, bid, nblk)) return;
        block_reduce_all<double>(part_buf[parity], CNV * H, s_sums, s_tmp, nblk);
        parity ^= 1;

        int act = 0;
        // stop test: ||r_p||^2 <= tol^2 max(||b_p||^2, sum_q ||b_q||^2 / H).
        // A harmonic that carries at least an average share of the right-hand
        // side is solved to tol relative to its own; one whose right-hand
        // side is far smaller (the even harmonics of a half-wave symmetric
        // excitation hold only rounding noise) stops at tol times the
        // average, where it no longer matters: sum_p ||r_p||^2 <= 2 tol^2
        // sum_p ||b_p||^2 either way
        double share = 0.0;
        if (k == 0) {
            for (int q = 0; q < H; ++q) share += s_sums[q];
            share /= H;
        }
        for (int l = tid; l < H; l += blockDim.x) {
            const double rho = s_sums[l];
            const cplx gam = {s_sums[H + l], s_sums[2 * H + l]};
            const cplx del = {s_sums[3 * H + l], s_sums[4 * H + l]};
            if (k == 0) {
                s_stop[l] = a.tol * a.tol * fmax(rho, share);
                s_act[l] = rho > 0.0;
            }
            int on = 0;
            cplx al = {0.0, 0.0}, be = {0.0, 0.0};
            if (s_act[l]) {
                if (!isfinite(rho) || !isfinite(gam.re) || !isfinite(gam.im) || !isfinite(del.re) ||
                    !isfinite(del.im)) {
                    set_status(a.status, DEV_ERR_NAN);
                    s_err = 1;
                } else if (rho <= s_stop[l]) {
                    s_act[l] = 0;
                } else if (k >= a.max_it) {
                    set_status(a.status, DEV_ERR_LINEAR);
                    s_err = 1;
                } else {
                    cplx den = del;
                    if (k > 0) {
                        be = cdiv(gam, {s_gold[2 * l], s_gold[2 * l + 1]});
                        den = csub(del, cdiv(cmul(be, gam), {s_aold[2 * l], s_aold[2 * l + 1]}));
                    }
                    if (!(cabs2(den) > 0.0) || !(cabs2(gam) > 0.0)) {
                        set_status(a.status, DEV_ERR_BREAKDOWN);
                        s_err = 1;
                    } else {
                        al = cdiv(gam, den);
                        s_gold[2 * l] = gam.re;
                        s_gold[2 * l + 1] = gam.im;
                        s_aold[2 * l] = al.re;
                        s_aold[2 * l + 1] = al.im;
                        on = 1;
                    }
                }
            }
            s_alpha[2 * l] = al.re;
            s_alpha[2 * l + 1] = al.im;
            s_beta[2 * l] = be.re;
            s_beta[2 * l + 1] = be.im;
            act |= on;
        }
        const int any = __syncthreads_or(act);
        if (s_err) return;
        if (!any) break;
        ++iters;

        const cplx al = {s_alpha[2 * pl], s_alpha[2 * pl + 1]};
        const cplx be = {s_beta[2 * pl], s_beta[2 * pl + 1]};
        for (int i = row0; i < m.ndof; i += rstride) {
            const size_t o = 2 * ((size_t)i * H + pl);
            const cplx pv = cadd(ldc<T>(z + o), cmul(be, ldc<T>(p + o)));
            const cplx sv = cadd(ldc<T>(w + o), cmul(be, ldc<T>(s + o)));
            const cplx xv = cadd(ldc<T>(x + o), cmul(al, pv));
            const cplx rv = csub(ldc<T>(r + o), cmul(al, sv));
            stc<T>(p + o, pv);
            stc<T>(s + o, sv);
            stc<T>(x + o, xv);
            stc<T>(r + o, rv);
            if (!amg) {
                const int sp = m.sp_index[i];
                const cplx iv = sp >= 0 ? ldc<T>(invd + 2 * ((size_t)sp * H + pl)) : cplx{m.invdiag_lin[i], 0.0};
                stc<T>(z + o, cmul(iv, rv));
            }
        }
        if (amg) {
            if (!grid_sync(a.bar, a.status, bid, nblk)) return;
            if (!precondition()) return;
        }
        if (!grid_sync(a.bar, a.status, bid, nblk)) return;
    }
    if (bid == 0 && tid == 0) {
        a.counters[2] += iters;
        if (a.team_ns) a.team_ns[1] = global_ns();
    }
}

// Single-instance launches: one block of up to kCocgThreads threads per SM
// (H x floor(kCocgThreads / H) of them), so that a block serves as many rows
// per pass as the register budget allows.
constexpr int kCocgThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kCocgThreads) cocg_kernel(const CocgArgs a) {
    cocg_body<T>(a, blockIdx.x, gridDim.x);
}

// Batched launch of 512-thread blocks: block b serves member map[b].x as
// block map[b].y of a team of map[b].z blocks (map[b].x < 0: idle).
template <typename T>
__global__ void __launch_bounds__(512) cocg_batch_kernel(const CocgArgs* args, const int4* map) {
    __shared__ CocgArgs s_a;
    const int4 mb = map[blockIdx.x];
    if (mb.x < 0) return;
    static_assert(sizeof(CocgArgs) % sizeof(int) == 0, "CocgArgs copied as words");
    const int* src = reinterpret_cast<const int*>(args + mb.x);
    int* dst = reinterpret_cast<int*>(&s_a);
    for (int q = threadIdx.x; q < (int)(sizeof(CocgArgs) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    cocg_body<T>(s_a, mb.y, mb.z);
}

size_t cocg_smem(int H, int threads) {
    const int RB = threads / H;
    return (size_t)(9 * H + CNV * RB * H + CNV * H + threads) * sizeof(double) + H * sizeof(int);
}

// ------------------------------------------------ PP-IC coarse sweep --
// PP-IC (Eq. 5) relaxes periodicity to U_0^{k+1} = U_N^k and sweeps the
// coarse propagator forward: with G linear within the iteration,
//   D_0 = U_N^k - U_0^k,   D_n = (F_n - U_n^k) + Q^{-1} C D_{n-1},  n = 1..N,
// and U_n^{k+1} = U_n^k + D_n (U_N^k being the stored end-of-period value).
__global__ void ppic_start_kernel(int ndof, int NB, const double* U, const double* UN, double* dcur,
                                  double* Unew) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += gridDim.x * blockDim.x) {
        const double d0 = UN[i] - U[(size_t)i * NB];
        dcur[i] = d0;
        Unew[(size_t)i * NB] = U[(size_t)i * NB] + d0;
    }
}

// b = C v on the special rows, as a one-harmonic complex right-hand side
__global__ void ppic_rhs_kernel(MeshDev m, double inv_dT, const double* v, double* b) {
    for (int sp = blockIdx.x * blockDim.x + threadIdx.x; sp < m.n_sp; sp += gridDim.x * blockDim.x) {
        const int i = m.sp_rows[sp];
        const int kb = m.rowptr[i], ke = m.rowptr[i + 1], slot0 = m.row_slot[i];
        double acc = 0.0;
        for (int k = kb; k < ke; ++k) acc += m.Mslot[slot0 + (k - kb)] * v[m.col[k]];
        b[2 * (size_t)sp] = acc * inv_dT;
        b[2 * (size_t)sp + 1] = 0.0;
    }
}

// D_n = (F_n - U_n) + Re x;  U_n^{k+1} = U_n + D_n (n < N) or U_N^{k+1} = U_N + D_N
__global__ void ppic_step_kernel(int ndof, int N, int NB, int n, const double* F, const double* U, const double* UN,
                                 const double* x, double* dcur, double* Unew, double* UNnew) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += gridDim.x * blockDim.x) {
        const double Un = n < N ? U[(size_t)i * NB + n] : UN[i];
        const double dn = (F[(size_t)i * NB + (n - 1)] - Un) + x[2 * (size_t)i];
        dcur[i] = dn;
        if (n < N)
            Unew[(size_t)i * NB + n] = Un + dn;
        else
            UNnew[i] = Un + dn;
    }
}

__global__ void zero_pad_lanes_kernel(int ndof, int N, int NB, double* U) {
    const long long total = (long long)ndof * (NB - N);
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const long long i = it / (NB - N);
        U[i * NB + N + (it % (NB - N))] = 0.0;
    }
}

// ------------------------------------------------ inverse DFT + update --
// U_n^{k+1} = F_n(U_{n-1}^k) + (1/N) sum_{p in P} W_p exp(i 2 pi p n / N),
// the sum taken over the Hermitian spectrum from p = 0..N/2.
template <typename T>
__global__ void idft_update_kernel(int ndof, int N, int NB, int H, const T* W, const double* F,
                                   const double* tw, double* Unew) {
    const long long total = (long long)ndof * NB;
    const double invN = 1.0 / (double)N;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(it % NB);
        const long long i = it / NB;
        if (n >= N) {
            Unew[it] = 0.0;
            continue;
        }
        const T* Wi = W + 2 * (size_t)i * H;
        double acc = (double)Wi[0] + ((n & 1) ? -(double)Wi[2 * (N / 2)] : (double)Wi[2 * (N / 2)]);
        double mid = 0.0;
        int k = n;  // (p * n) mod N for p = 1
        for (int p = 1; p < N / 2; ++p) {
            mid += (double)Wi[2 * p] * tw[2 * k] + (double)Wi[2 * p + 1] * tw[2 * k + 1];
            k += n;
            if (k >= N) k -= N;
        }
        acc += 2.0 * mid;
        Unew[it] = F[i * NB + (n + N - 1) % N] + acc * invN;
    }
}

// ------------------------------------------------ layout conversion --
__global__ void state_to_lanes_kernel(int ndof, int n_nodes, int N, int NB, const int* node_of_dof,
                                      const double* ext, double* lanes) {
    const long long total = (long long)ndof * NB;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(it % NB);
        const long long i = it / NB;
        lanes[it] = n < N ? ext[(size_t)n * n_nodes + node_of_dof[i]] : 0.0;
    }
}

__global__ void lanes_to_state_kernel(int n_nodes, int N, int NB, const int* dof_of_node,
                                      const double* lanes, double* ext) {
    const long long total = (long long)n_nodes * N;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int node = (int)(it % n_nodes);
        const int n = (int)(it / n_nodes);
        const int d = dof_of_node[node];
        ext[it] = d >= 0 ? lanes[(size_t)d * NB + n] : 0.0;
    }
}

}  // namespace

namespace {

// Last kernels of a captured PP-PC iteration: U = Unext unless an error was
// flagged or the jumps met tol_commit (rel_res <= tol_commit keeps U^k, the
// iterate that passed); then the control block for the host.
__global__ void commit_kernel(long long total, const int* status, const double* jsums, const double* tol_commit,
                              const double* Unext, double* U) {
    if (*status != 0) return;
    const double dd = jsums[0], ff = jsums[1];
    const double rr = ff > 0.0 ? sqrt(dd / ff) : (dd > 0.0 ? INFINITY : 0.0);
    if (!(rr > *tol_commit)) return;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x)
        U[it] = Unext[it];
}

__global__ void iter_ctl_kernel(const int* status, const double* jsums, const long long* counters, IterCtl* out) {
    const int t = threadIdx.x;
    if (t == 0) {
        out->status = *status;
        out->jsums[0] = jsums[0];
        out->jsums[1] = jsums[1];
    }
    if (t < kCounters) out->counters[t] = counters[t];
}

}  // namespace

void launch_commit(long long total, const int* status, const double* jsums, const double* tol_commit,
                   const double* Unext, double* U, const long long* counters, IterCtl* ctl, cudaStream_t st) {
    commit_kernel<<<grid_for(total, 256, 152 * 8), 256, 0, st>>>(total, status, jsums, tol_commit, Unext, U);
    iter_ctl_kernel<<<1, 32, 0, st>>>(status, jsums, counters, ctl);
}

void launch_jumps(int ndof, int N, int NB, const double* U, const double* F, double* d, double* part,
                  double* sums, cudaStream_t st) {
    jumps_kernel<<<kJumpBlocks, 256, 0, st>>>(ndof, N, NB, U, F, d, part);
    sum_pairs_kernel<<<1, kSumThreads, 0, st>>>(kJumpBlocks, part, sums);
}

void launch_kbar(const MeshDev& m, int N, int NB, int lin, const double* elem, double* Kbar,
                 cudaStream_t st) {
    if (m.n_slots == 0) return;
    kbar_kernel<<<grid_for(m.n_slots, 128), 128, 0, st>>>(m, N, NB, lin, elem, Kbar);
}

void launch_coarse_rhs(const MeshDev& m, int N, int NB, int H, double inv_dT, const double* d,
                       const double* tw, double* y, double* b, cudaStream_t st) {
    if (m.n_sp == 0) return;
    cd_kernel<<<grid_for((long long)m.n_sp * NB, 256), 256, 0, st>>>(m, NB, inv_dT, d, y);
    dft_rhs_kernel<<<grid_for((long long)m.n_sp * H, 256), 256, 0, st>>>(m.n_sp, N, NB, H, y, tw, b);
}

cudaError_t cocg_config(bool fp32, int H, LaunchCfg* cfg) {
    if (H < 1 || H > 512) return cudaErrorInvalidValue;
    const int threads = H * (kCocgThreads / H);
    const size_t smem = cocg_smem(H, threads);
    const void* fn = fp32 ? (const void*)cocg_kernel<float> : (const void*)cocg_kernel<double>;
    cudaError_t e = allow_max_dynamic_smem(fn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // one block per SM: every block reads all blocks' partials in each reduction
    cfg->blocks = sms;
    cfg->threads = threads;
    cfg->smem = smem;
    return cudaSuccess;
}

cudaError_t launch_cocg(const CocgArgs& a, bool fp32, const LaunchCfg& cfg, cudaStream_t st) {
    // cudaLaunchKernelEx with the cooperative attribute: capturable in a graph
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(cfg.blocks);
    lc.blockDim = dim3(cfg.threads);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (fp32) return cudaLaunchKernelEx(&lc, cocg_kernel<float>, a);
    return cudaLaunchKernelEx(&lc, cocg_kernel<double>, a);
}

size_t cocg_smem_bytes(int H, int threads) { return cocg_smem(H, threads); }

cudaError_t cocg_batch_prepare(size_t* static_smem) {
    const void* fn = (const void*)cocg_batch_kernel<double>;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (static_smem) *static_smem = fa.sharedSizeBytes;
    return allow_max_dynamic_smem(fn);
}

cudaError_t launch_cocg_batch(const CocgArgs* args, const int4* map, int blocks, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cocg_batch_kernel<double>, args, map);
}

void launch_ppic_start(int ndof, int NB, const double* U, const double* UN, double* dcur, double* Unew,
                       cudaStream_t st) {
    ppic_start_kernel<<<grid_for(ndof, 256), 256, 0, st>>>(ndof, NB, U, UN, dcur, Unew);
}

void launch_ppic_rhs(const MeshDev& m, double inv_dT, const double* v, double* b, cudaStream_t st) {
    if (m.n_sp == 0) return;
    ppic_rhs_kernel<<<grid_for(m.n_sp, 256), 256, 0, st>>>(m, inv_dT, v, b);
}

void launch_ppic_step(int ndof, int N, int NB, int n, const double* F, const double* U, const double* UN,
                      const double* x, double* dcur, double* Unew, double* UNnew, cudaStream_t st) {
    ppic_step_kernel<<<grid_for(ndof, 256), 256, 0, st>>>(ndof, N, NB, n, F, U, UN, x, dcur, Unew, UNnew);
}

void launch_zero_pad_lanes(int ndof, int N, int NB, double* U, cudaStream_t st) {
    if (NB == N) return;
    zero_pad_lanes_kernel<<<grid_for((long long)ndof * (NB - N), 256), 256, 0, st>>>(ndof, N, NB, U);
}

void launch_idft_update(int ndof, int N, int NB, int H, bool fp32, const void* W, const double* F,
                        const double* tw, double* Unew, cudaStream_t st) {
    const int g = grid_for((long long)ndof * NB, 256);
    if (fp32)
        idft_update_kernel<float><<<g, 256, 0, st>>>(ndof, N, NB, H, (const float*)W, F, tw, Unew);
    else
        idft_update_kernel<double><<<g, 256, 0, st>>>(ndof, N, NB, H, (const double*)W, F, tw, Unew);
}

void launch_state_to_lanes(int ndof, int n_nodes, int N, int NB, const int* node_of_dof,
                           const double* ext, double* lanes, cudaStream_t st) {
    state_to_lanes_kernel<<<grid_for((long long)ndof * NB, 256), 256, 0, st>>>(ndof, n_nodes, N, NB,
                                                                               node_of_dof, ext, lanes);
}

void launch_lanes_to_state(int ndof, int n_nodes, int N, int NB, const int* dof_of_node,
                           const double* lanes, double* ext, cudaStream_t st) {
    (void)ndof;
    lanes_to_state_kernel<<<grid_for((long long)n_nodes * N, 256), 256, 0, st>>>(n_nodes, N, NB,
                                                                                 dof_of_node, lanes, ext);
}

}  // namespace pppc

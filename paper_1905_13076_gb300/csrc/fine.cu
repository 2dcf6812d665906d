// Batched fine propagators F_n of PP-PC (Sec. 2, Eqs. 2-3).
//
// All N subintervals march at once: lane n of every vector is subinterval
// n+1, started from U_n at T_n.  Each implicit-Euler step of size dt solves
//     R(u) = (M/dt)(u - u_prev) + K(u) u - I(t) g = 0
// by Newton's method; each Newton correction solves J du = -R with
// preconditioned conjugate gradients.  J = K_lin + M/dt + J_nl(u) is SPD; only
// rows touching the nonlinear sheath (the "special" rows) differ per lane, so
// their values are stored per lane and all other rows share one FP64 array.
//
// One cooperative launch runs the whole sweep (all steps, Newton iterations
// and PCG iterations); device-side grid barriers separate the phases, and all
// loop decisions are taken identically by every block from the same reduced
// per-lane scalars.  Lanes that have converged are frozen (step length 0)
// while the others continue.  PCG uses the single-reduction form of
// Chronopoulos and Gear: per iteration one SpMV w = J z, one fused reduction
// of (r,r), (r,z), (z,w), and the updates p = z + b p, s = w + b s,
// x += a p, r -= a s, z = D^-1 r, all in the PCG precision T (FP32 in the
// mixed path, with per-thread FP32 accumulation); u += x in FP64 once the
// solve is done, so the Newton residual refines the FP32 solves.  Each
// solve stops at the Eisenstat-Walker forcing term, and each step's Newton
// iteration may start from the linear extrapolation of the last two steps.
//
// Layout: vectors are [ndof][NB] (lane fastest, NB = N rounded up to the
// lane-vector width V: 4 FP32 or 2 FP64 lanes, one 16-byte access).  Each
// block owns a contiguous range of rows (balanced by nonzeros on the host)
// and a thread owns V adjacent lanes of fixed rows for the whole launch, so
// row-local data is only touched by its owner; other rows' data is read only
// after a grid barrier.
//
// Options carried by FineArgs:
// - preconditioner: Jacobi, or the tridiagonal part of every a.tri
//   consecutive rows factorised per lane (tri_factor / tri_solve);
// - Newton start: u^m, linear or quadratic extrapolation; lanes whose
//   residual does not drop backtrack (apply_steps);
// - a record of every fine level (traj_out), and an adjoint mode in which
//   each lane runs the periodic adjoint of its subinterval backwards over
//   that record (adjoint_rows);
// - teams: fine_sweep_body runs on any team of blocks, the whole grid
//   (fine_sweep_kernel) or one batch member's share (fine_batch_kernel).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "amg.cuh"
#include "common.cuh"
#include "kernels.h"
#include "lanes.cuh"

namespace pppc {

// Element data of nonlinear element q, lane `lane`, from the state u:
//   grad A = sum_a u_a grad N_a,  b = |grad A|^2,  bc = min(b, cap),
//   nu = k1 exp(k2 bc) (1 + k2 (b - bc)) + k3,  dnu/db = k1 k2 exp(k2 bc)
//   (the Brauer law, continued past the cap by its tangent in b),
//   c1 = |e| nu,  c2 = 2 |e| dnu/db,  s_a = grad N_a . grad A.
__device__ __forceinline__ void elem_compute(const MeshDev& m, int NB, const double* u, double* elem,
                                             int q, int lane) {
    const int* dofs = m.nl_dofs + 3 * (size_t)q;
    const double* G = m.nl_geom + 8 * (size_t)q;
    const double* K = m.nl_k + 4 * (size_t)q;
    double ua[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int d = dofs[a];
        ua[a] = d < 0 ? 0.0 : u[(size_t)d * NB + lane];
    }
    // grad A from vertex differences (sum_a grad N_a = 0): rounding stays
    // proportional to the differences of u, not to u
    const double d1 = ua[1] - ua[0], d2 = ua[2] - ua[0];
    const double gx = d1 * G[3] + d2 * G[5];
    const double gy = d1 * G[4] + d2 * G[6];
    const double b = gx * gx + gy * gy;
    const double bc = fmin(b, K[3]);
    const double ex = exp(K[1] * bc);
    const double nu = K[0] * ex * (1.0 + K[1] * (b - bc)) + K[2];
    const double dnu = K[0] * K[1] * ex;
    const size_t P = (size_t)m.n_nl * NB;
    const size_t o = (size_t)q * NB + lane;
    elem[o] = G[0] * nu;
    elem[P + o] = 2.0 * G[0] * dnu;
#pragma unroll
    for (int a = 0; a < 3; ++a) elem[(2 + a) * P + o] = G[1 + 2 * a] * gx + G[2 + 2 * a] * gy;
}

namespace {

__global__ void elem_data_kernel(MeshDev m, int NB, const double* u, double* elem) {
    const long long total = (long long)m.n_nl * NB;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x)
        elem_compute(m, NB, u, elem, (int)(it / NB), (int)(it % NB));
}

constexpr int NV = 3;  // reduced values per lane: (r,r), (r,z), (z,w)
constexpr double kPi = 3.141592653589793;
// Newton also stops when ||R|| no longer halves (kStagnation) while within
// kFloorMult of the tolerance: the residual has reached its rounding floor.
constexpr double kStagnation = 0.5;
constexpr double kFloorMult = 100.0;
// FP32 Jacobian (mixed path): a nonlinear element whose reluctivity exceeds
// this has its whole Jacobian contribution scaled by kNuCapFp32 / nu, which
// keeps J symmetric positive definite and the FP32 PCG within range.  The
// Brauer steel passes it near |B| = 3.2 T, above any converged state of the
// cable workloads; a cold start at full current can overshoot to ~10 T, where
// nu exceeds the FP32 range.  The residual stays exact FP64, so converged
// states do not depend on the cap, and Newton is exact once no element is
// above it.
constexpr double kNuCapFp32 = 1e10;
// Smallest fraction of a Newton step that backtracking tries before the
// lane reports failure (20 halvings).
constexpr double kMinStep = 1.0 / 1048576.0;


// Residual R(u) of the implicit-Euler step on this thread's rows and lanes,
// the per-lane Jacobian values of the special rows, r = -R, z = D^-1 r and
// x = 0.  Accumulates sum R^2 and (r,z) per lane into accR / accz.  Kept out
// of line: it runs once per Newton iteration, and its register demand
// (FP64 state and element data) must not constrain the PCG loops.
template <typename T, int V>
__device__ __noinline__ void residual_rows(const FineArgs& a, const MeshDev& m, int row0, int re, int RB, int l0,
                                           const double* s_I, double* accR, T* accz, T* xB, size_t vo, T* l1sp) {
    const int NB = a.NB, LD = a.ld;
    const size_t P = (size_t)m.n_nl * LD;
    const double* u = a.u + a.lane0;
    const double* uprev = a.uprev + a.lane0;
    const double* E = a.elem + a.lane0;
    T* r = static_cast<T*>(a.r);
    T* z = static_cast<T*>(a.z);
    T* J = static_cast<T*>(a.J);
    T* invd = static_cast<T*>(a.invd_sp);
    const T* invdiag_linT = std::is_same<T, float>::value ? reinterpret_cast<const T*>(m.invdiag_lin32)
                                                          : reinterpret_cast<const T*>(m.invdiag_lin);
    for (int i = row0; i < re; i += RB) {
                const int kb = m.rowptr[i], ke = m.rowptr[i + 1];
                const int slot0 = m.row_slot[i];
                const size_t o = (size_t)i * NB + l0;    // team vectors
                const size_t os = (size_t)i * LD + l0;   // state vectors
                // K_lin u in difference form: sum_{j != i} K_ij (u_j - u_i) + dlin_i u_i
                const Lanes<double, V> ui = ldv<double, V>(u + os);
                const double dl = m.dlin[i];
                double acc[V];
#pragma unroll
                for (int h = 0; h < V; ++h) acc[h] = dl * ui.v[h];
                Lanes<T, V> iv;
                if (slot0 < 0) {
                    for (int k = kb; k < ke; ++k) {
                        const int j = m.col[k];
                        if (j == i) continue;
                        const double kv = m.Klin[k];
                        const Lanes<double, V> uj = ldv<double, V>(u + (size_t)j * LD + l0);
#pragma unroll
                        for (int h = 0; h < V; ++h) acc[h] += kv * (uj.v[h] - ui.v[h]);
                    }
                    const T d = invdiag_linT[i];
#pragma unroll
                    for (int h = 0; h < V; ++h) iv.v[h] = d;
                } else {
                    double dg[V];
                    T l1acc[V];
#pragma unroll
                    for (int h = 0; h < V; ++h) l1acc[h] = (T)0;
                    for (int k = kb; k < ke; ++k) {
                        const int sl = slot0 + (k - kb);
                        const int j = m.col[k];
                        const double kv = m.Klin[k];
                        const double mv = m.Mslot[sl] * a.inv_dt;
                        const Lanes<double, V> uj = ldv<double, V>(u + (size_t)j * LD + l0);
                        const Lanes<double, V> upj = ldv<double, V>(uprev + (size_t)j * LD + l0);
                        const double kl = (j == i) ? 0.0 : kv;
                        double Jv[V];
#pragma unroll
                        for (int h = 0; h < V; ++h) {
                            acc[h] += kl * (uj.v[h] - ui.v[h]) + mv * (uj.v[h] - upj.v[h]);
                            Jv[h] = kv + mv;
                        }
                        for (int c = m.nlc_ptr[sl]; c < m.nlc_ptr[sl + 1]; ++c) {
                            const int pk = m.nlc[c];
                            const int q = pk / 9, ia = (pk / 3) % 3, ib = pk % 3;
                            const double ab = m.nlc_ab[c];
                            // area * cap: c1 = area * nu above it marks a capped element
                            const double c1cap = std::is_same<T, float>::value ? kNuCapFp32 * m.nl_geom[8 * (size_t)q]
                                                                              : 0.0;
                            const size_t eo = (size_t)q * LD + l0;
                            const Lanes<double, V> c1 = ldv<double, V>(E + eo);
                            const Lanes<double, V> c2 = ldv<double, V>(E + P + eo);
                            const Lanes<double, V> sa = ldv<double, V>(E + (2 + ia) * P + eo);
                            const Lanes<double, V> sb = ldv<double, V>(E + (2 + ib) * P + eo);
#pragma unroll
                            for (int h = 0; h < V; ++h) {
                                const double jc = c1.v[h] * ab + c2.v[h] * sa.v[h] * sb.v[h];
                                if constexpr (std::is_same<T, float>::value)
                                    Jv[h] += c1.v[h] > c1cap ? jc * (c1cap / c1.v[h]) : jc;
                                else
                                    Jv[h] += jc;
                                if (j == i) acc[h] += c1.v[h] * sa.v[h];
                            }
                        }
                        Lanes<T, V> jt;
#pragma unroll
                        for (int h = 0; h < V; ++h) {
                            jt.v[h] = (T)Jv[h];
                            l1acc[h] += jt.v[h] < (T)0 ? -jt.v[h] : jt.v[h];
                        }
                        stv<T, V>(J + (size_t)sl * NB + l0, jt);
                        if (j == i)
#pragma unroll
                            for (int h = 0; h < V; ++h) dg[h] = Jv[h];
                    }
#pragma unroll
                    for (int h = 0; h < V; ++h) iv.v[h] = (T)(1.0 / dg[h]);
                    stv<T, V>(invd + (size_t)m.sp_index[i] * NB + l0, iv);
                    if (l1sp) {
                        Lanes<T, V> lv;
#pragma unroll
                        for (int h = 0; h < V; ++h) lv.v[h] = l1acc[h];
                        stv<T, V>(l1sp + (size_t)m.sp_index[i] * NB + l0, lv);
                    }
                }
                const double gi = m.g[i];
                Lanes<T, V> rv, zv, zero;
#pragma unroll
                for (int h = 0; h < V; ++h) {
                    const double R = acc[h] - s_I[l0 + h] * gi;
                    rv.v[h] = (T)(-R);
                    zv.v[h] = rv.v[h] * iv.v[h];
                    zero.v[h] = (T)0;
                    accR[h] += R * R;
                    accz[h] += rv.v[h] * zv.v[h];
                }
                stv<T, V>(r + o, rv);
                stv<T, V>(z + o, zv);
                stv<T, V>(xB + (o - vo), zero);
            }
}

// Periodic adjoint (backwards in time) on this thread's rows and lanes at
// level j of each lane's subinterval (global step m = lane * n_fine + j):
//   R(lam) = (M/dt)(lam - lam_next) + J_m lam - g_m,
//   g_m = g_scale M (du^m - du^{m+1}),   du^m = u^m - u^{m-1},
// J_m = d(K(u)u)/du at the forward state u^m (element data in a.elem were
// computed from it), lam in a.u, lam_next = lam_{m+1} in a.uprev; at j =
// n_fine, du^{m+1} is the next lane's first step.  Writes the per-lane
// Jacobian values of the special rows, r = -R, z = D^-1 r, x = 0, and
// accumulates sum R^2, (r,z) and sum b^2 of the right-hand side
// b = (M/dt) lam_next + g_m.  Out of line like residual_rows.
template <typename T, int V>
__device__ __noinline__ void adjoint_rows(const FineArgs& a, const MeshDev& m, int row0, int re, int RB, int l0, int j,
                                          double* accR, T* accz, double* accb, T* xB, size_t vo, T* l1sp) {
    const int NB = a.NB, N = a.N, LD = a.ld;
    const size_t P = (size_t)m.n_nl * LD;
    const size_t lv = (size_t)m.ndof * LD;
    const double* lam = a.u + a.lane0;
    const double* lnext = a.uprev + a.lane0;
    const double* E = a.elem + a.lane0;
    const double* um = a.traj + a.lane0 + (size_t)j * lv;
    const double* ump = um - lv;
    const bool last = j == a.n_fine;   // du^{m+1} from the next lane's levels 0, 1
    T* r = static_cast<T*>(a.r);
    T* z = static_cast<T*>(a.z);
    T* J = static_cast<T*>(a.J);
    T* invd = static_cast<T*>(a.invd_sp);
    const T* invdiag_linT = std::is_same<T, float>::value ? reinterpret_cast<const T*>(m.invdiag_lin32)
                                                          : reinterpret_cast<const T*>(m.invdiag_lin);
    for (int i = row0; i < re; i += RB) {
        const int kb = m.rowptr[i], ke = m.rowptr[i + 1];
        const int slot0 = m.row_slot[i];
        const size_t o = (size_t)i * NB + l0;   // team vectors
        double acc[V], bb[V];
#pragma unroll
        for (int h = 0; h < V; ++h) acc[h] = bb[h] = 0.0;
        Lanes<T, V> iv;
        if (slot0 < 0) {
            for (int k = kb; k < ke; ++k) {
                const double kv = m.Klin[k];
                const Lanes<double, V> lj = ldv<double, V>(lam + (size_t)m.col[k] * LD + l0);
#pragma unroll
                for (int h = 0; h < V; ++h) acc[h] += kv * lj.v[h];
            }
            const T d = invdiag_linT[i];
#pragma unroll
            for (int h = 0; h < V; ++h) iv.v[h] = d;
        } else {
            double dg[V];
            T l1acc[V];
#pragma unroll
            for (int h = 0; h < V; ++h) l1acc[h] = (T)0;
            for (int k = kb; k < ke; ++k) {
                const int sl = slot0 + (k - kb);
                const int jc = m.col[k];
                const size_t oc = (size_t)jc * LD + l0;   // state vectors
                const double kv = m.Klin[k];
                const double ms = m.Mslot[sl];
                const double mv = ms * a.inv_dt;
                const Lanes<double, V> lj = ldv<double, V>(lam + oc);
                const Lanes<double, V> lnj = ldv<double, V>(lnext + oc);
                double dd[V];   // du^m - du^{m+1} at node jc
                if (ms != 0.0) {
                    const Lanes<double, V> u0 = ldv<double, V>(um + oc);
                    const Lanes<double, V> u1 = ldv<double, V>(ump + oc);
                    if (!last) {
                        const Lanes<double, V> u2 = ldv<double, V>(um + lv + oc);
#pragma unroll
                        for (int h = 0; h < V; ++h) dd[h] = (u0.v[h] - u1.v[h]) - (u2.v[h] - u0.v[h]);
                    } else {
#pragma unroll
                        for (int h = 0; h < V; ++h) {
                            const int ln = (a.lane0 + l0 + h + 1) % N;   // the next subinterval
                            const size_t on = (size_t)jc * LD + ln;
                            dd[h] = (u0.v[h] - u1.v[h]) - (a.traj[lv + on] - a.traj[on]);
                        }
                    }
                } else {
#pragma unroll
                    for (int h = 0; h < V; ++h) dd[h] = 0.0;
                }
                double Jv[V];
#pragma unroll
                for (int h = 0; h < V; ++h) Jv[h] = kv + mv;
                for (int c = m.nlc_ptr[sl]; c < m.nlc_ptr[sl + 1]; ++c) {
                    const int pk = m.nlc[c];
                    const int q = pk / 9, ia = (pk / 3) % 3, ib = pk % 3;
                    const double ab = m.nlc_ab[c];
                    const double c1cap = std::is_same<T, float>::value ? kNuCapFp32 * m.nl_geom[8 * (size_t)q] : 0.0;
                    const size_t eo = (size_t)q * LD + l0;
                    const Lanes<double, V> c1 = ldv<double, V>(E + eo);
                    const Lanes<double, V> c2 = ldv<double, V>(E + P + eo);
                    const Lanes<double, V> sa = ldv<double, V>(E + (2 + ia) * P + eo);
                    const Lanes<double, V> sb = ldv<double, V>(E + (2 + ib) * P + eo);
#pragma unroll
                    for (int h = 0; h < V; ++h) {
                        const double jc2 = c1.v[h] * ab + c2.v[h] * sa.v[h] * sb.v[h];
                        if constexpr (std::is_same<T, float>::value)
                            Jv[h] += c1.v[h] > c1cap ? jc2 * (c1cap / c1.v[h]) : jc2;
                        else
                            Jv[h] += jc2;
                    }
                }
                Lanes<T, V> jt;
#pragma unroll
                for (int h = 0; h < V; ++h) {
                    const double rhs = mv * lnj.v[h] + a.g_scale * ms * dd[h];
                    acc[h] += Jv[h] * lj.v[h] - rhs;
                    bb[h] += rhs;
                    jt.v[h] = (T)Jv[h];
                    l1acc[h] += jt.v[h] < (T)0 ? -jt.v[h] : jt.v[h];
                }
                stv<T, V>(J + (size_t)sl * NB + l0, jt);
                if (jc == i)
#pragma unroll
                    for (int h = 0; h < V; ++h) dg[h] = Jv[h];
            }
#pragma unroll
            for (int h = 0; h < V; ++h) iv.v[h] = (T)(1.0 / dg[h]);
            stv<T, V>(invd + (size_t)m.sp_index[i] * NB + l0, iv);
            if (l1sp) {
                Lanes<T, V> lv;
#pragma unroll
                for (int h = 0; h < V; ++h) lv.v[h] = l1acc[h];
                stv<T, V>(l1sp + (size_t)m.sp_index[i] * NB + l0, lv);
            }
        }
        Lanes<T, V> rv, zv, zero;
#pragma unroll
        for (int h = 0; h < V; ++h) {
            rv.v[h] = (T)(-acc[h]);
            zv.v[h] = rv.v[h] * iv.v[h];
            zero.v[h] = (T)0;
            accR[h] += acc[h] * acc[h];
            accz[h] += rv.v[h] * zv.v[h];
            accb[h] += bb[h] * bb[h];
        }
        stv<T, V>(r + o, rv);
        stv<T, V>(z + o, zv);
        stv<T, V>(xB + (o - vo), zero);
    }
}

// Matrix entry (i, k) of the Newton matrix for this thread's lanes, given
// its CSR index kk: per lane on special rows (J), shared K_lin elsewhere.
template <typename T, int V>
__device__ __forceinline__ Lanes<T, V> entry(const MeshDev& m, const T* KlinT, const T* J, int i, int kk, int NB,
                                           int l0) {
    const int slot0 = m.row_slot[i];
    if (slot0 >= 0) return ldv<T, V>(J + (size_t)(slot0 + kk - m.rowptr[i]) * NB + l0);
    Lanes<T, V> v;
    const T k = KlinT[kk];
#pragma unroll
    for (int h = 0; h < V; ++h) v.v[h] = k;
    return v;
}

// Tridiagonal-chunk preconditioner.  The own rows [rs, re) are cut into
// chunks of a.tri consecutive rows, chunk q handled by row group q mod RB.
// Each chunk's tridiagonal part T_c of the Newton matrix (diagonal and the
// (i, i-1) / (i-1, i) couplings; row order follows the mesh's strongest
// couplings, along the rings of a polar mesh) is factorised per lane as
// L D L^T (multipliers tri_m, inverse pivots tri_ie, FP64 arithmetic), and
// z = T_c^-1 r replaces the Jacobi z = D^-1 r.  tri_factor factorises and
// applies it to the r of the residual phase (z, and (r, z) into accz);
// tri_update is the PCG vector update with z from the chunk solves.
template <typename T, int V>
__device__ __noinline__ void tri_factor(const FineArgs& a, const MeshDev& m, int rs, int re, int RB, int rb, int l0,
                                        T* accz) {
    const int NB = a.NB, c = a.tri;
    const T* KlinT = std::is_same<T, float>::value ? reinterpret_cast<const T*>(m.Klin32)
                                                   : reinterpret_cast<const T*>(m.Klin);
    const T* J = static_cast<const T*>(a.J);
    const T* r = static_cast<const T*>(a.r);
    T* z = static_cast<T*>(a.z);
    T* tm = static_cast<T*>(a.tri_m);
    T* tie = static_cast<T*>(a.tri_ie);
    for (int k0 = rs + rb * c; k0 < re; k0 += RB * c) {
        const int k1 = min(k0 + c, re) - 1;
        double e[V], y[V];
        for (int k = k0; k <= k1; ++k) {
            const size_t o = (size_t)k * NB + l0;
            const Lanes<T, V> d = entry<T, V>(m, KlinT, J, k, m.diag_k[k], NB, l0);
            const Lanes<T, V> rk = ldv<T, V>(r + o);
            const int lk = a.tri_low[k];
            Lanes<T, V> mk, ie, yk;
            if (k > k0 && lk >= 0) {
                const Lanes<T, V> l = entry<T, V>(m, KlinT, J, k, lk, NB, l0);
#pragma unroll
                for (int h = 0; h < V; ++h) {
                    const double mu = (double)l.v[h] / e[h];
                    e[h] = (double)d.v[h] - mu * (double)l.v[h];
                    y[h] = (double)rk.v[h] - mu * y[h];
                    mk.v[h] = (T)mu;
                }
            } else {
#pragma unroll
                for (int h = 0; h < V; ++h) {
                    e[h] = (double)d.v[h];
                    y[h] = (double)rk.v[h];
                    mk.v[h] = (T)0;
                }
            }
#pragma unroll
            for (int h = 0; h < V; ++h) {
                ie.v[h] = (T)(1.0 / e[h]);
                yk.v[h] = (T)y[h];
            }
            stv<T, V>(tm + o, mk);
            stv<T, V>(tie + o, ie);
            stv<T, V>(z + o, yk);   // forward-substituted y, replaced below
        }
        Lanes<T, V> zn;
        for (int k = k1; k >= k0; --k) {
            const size_t o = (size_t)k * NB + l0;
            const Lanes<T, V> yk = ldv<T, V>(z + o);
            const Lanes<T, V> ie = ldv<T, V>(tie + o);
            const Lanes<T, V> rk = ldv<T, V>(r + o);
            Lanes<T, V> mn;
            if (k < k1) mn = ldv<T, V>(tm + o + NB);
            Lanes<T, V> zk;
#pragma unroll
            for (int h = 0; h < V; ++h) {
                zk.v[h] = yk.v[h] * ie.v[h] - (k < k1 ? mn.v[h] * zn.v[h] : (T)0);
                accz[h] += rk.v[h] * zk.v[h];
            }
            stv<T, V>(z + o, zk);
            zn = zk;
        }
    }
}

// z = T_c^-1 r on this row group's chunks with the stored factorisation
// (after the PCG update of r by all threads and a __syncthreads).  Chunks
// have kTri rows: all of a chunk's loads are issued first, then the forward
// and back substitution run in registers (rows past the block's end act as
// zero rows).
constexpr int kTri = 4;
template <typename T, int V>
__device__ __noinline__ void tri_solve(const FineArgs& a, int rs, int re, int RB, int rb, int l0) {
    const int NB = a.NB;
    const T* r = static_cast<const T*>(a.r);
    T* z = static_cast<T*>(a.z);
    const T* tm = static_cast<const T*>(a.tri_m);
    const T* tie = static_cast<const T*>(a.tri_ie);
    for (int k0 = rs + rb * kTri; k0 < re; k0 += RB * kTri) {
        Lanes<T, V> rv[kTri], mv[kTri], iv[kTri];
#pragma unroll
        for (int q = 0; q < kTri; ++q) {
            if (k0 + q < re) {
                const size_t o = (size_t)(k0 + q) * NB + l0;
                rv[q] = ldv<T, V>(r + o);
                mv[q] = ldv<T, V>(tm + o);
                iv[q] = ldv<T, V>(tie + o);
            } else {
#pragma unroll
                for (int h = 0; h < V; ++h) rv[q].v[h] = mv[q].v[h] = iv[q].v[h] = (T)0;
            }
        }
        // forward: y_q = r_q - m_q y_{q-1} (m_0 is 0), in place in rv
#pragma unroll
        for (int q = 1; q < kTri; ++q)
#pragma unroll
            for (int h = 0; h < V; ++h) rv[q].v[h] -= mv[q].v[h] * rv[q - 1].v[h];
        // back: z_q = y_q / e_q - m_{q+1} z_{q+1}, in place in rv
#pragma unroll
        for (int h = 0; h < V; ++h) rv[kTri - 1].v[h] *= iv[kTri - 1].v[h];
#pragma unroll
        for (int q = kTri - 2; q >= 0; --q)
#pragma unroll
            for (int h = 0; h < V; ++h) rv[q].v[h] = rv[q].v[h] * iv[q].v[h] - mv[q + 1].v[h] * rv[q + 1].v[h];
#pragma unroll
        for (int q = 0; q < kTri; ++q)
            if (k0 + q < re) stv<T, V>(z + (size_t)(k0 + q) * NB + l0, rv[q]);
    }
}

// On this thread's rows and lanes: u += x and dx = x for lanes that took a
// Newton step (coef 1), u += coef * dx for lanes that backtrack (coef < 0),
// nothing for the others.  Out of line for the same reason as residual_rows.
template <typename T, int V>
__device__ __noinline__ void apply_steps(double* u, int LD, const T* xB, size_t vo, T* dx, const double* s_coef,
                                         int row0, int re, int RB, int l0, int NB) {
    double cf[V];
    bool step = false, keep = false, back = false;
#pragma unroll
    for (int h = 0; h < V; ++h) {
        cf[h] = s_coef[l0 + h];
        step |= cf[h] == 1.0;
        keep |= cf[h] != 1.0;
        back |= cf[h] < 0.0;
    }
    if (!step && !back) return;
    for (int i = row0; i < re; i += RB) {
        const size_t o = (size_t)i * NB + l0;
        const size_t os = (size_t)i * LD + l0;
        const Lanes<T, V> xi = ldv<T, V>(xB + (o - vo));
        Lanes<double, V> ui = ldv<double, V>(u + os);
        Lanes<T, V> di;
        if (back || keep) di = ldv<T, V>(dx + o);
#pragma unroll
        for (int h = 0; h < V; ++h) {
            if (cf[h] == 1.0) {
                ui.v[h] += (double)xi.v[h];
                di.v[h] = xi.v[h];
            } else if (cf[h] < 0.0) {
                ui.v[h] += cf[h] * (double)di.v[h];
            }
        }
        stv<double, V>(u + os, ui);
        if (step) stv<T, V>(dx + o, di);
    }
}

// The whole sweep for one team of nblk blocks (bid = this block's place in
// it): the grid of a single-instance launch, or one member's share of a
// batched launch.
template <typename T>
__device__ __forceinline__ void fine_sweep_body(const FineArgs& a, const int bid, const int nblk) {
    constexpr int V = sizeof(T) == 4 ? 4 : 2;   // lanes per thread: one 16-byte access
    using RT = T;                               // reductions run in the PCG precision
    extern __shared__ double smem[];
    const MeshDev& m = a.mesh;
    const int NB = a.NB, G = NB / V, LD = a.ld, lane0 = a.lane0;
    const int tid = threadIdx.x, g = tid % G, rb = tid / G, RB = blockDim.x / G;
    const int l0 = V * g;
    double* s_I = smem;            // current I(t) of each lane at the new time level
    double* s_stop = s_I + NB;     // PCG stop threshold on (r,r)
    double* s_gold = s_stop + NB;  // previous (r,z)
    double* s_aold = s_gold + NB;  // previous step length
    double* s_alpha = s_aold + NB;
    double* s_beta = s_alpha + NB;
    double* s_rprev = s_beta + NB; // ||R|| at the previous Newton test
    double* s_eta = s_rprev + NB;  // previous forcing term
    double* s_coef = s_eta + NB;   // this Newton iteration's update u += coef * (x or dx), see below
    double* s_lam = s_coef + NB;   // fraction of the last Newton step dx now applied
    RT* s_red = reinterpret_cast<RT*>(s_lam + NB);   // [NV][red_slots(G)][NB]
    RT* s_sums = s_red + NV * red_slots(G, blockDim.x) * NB;  // [NV][NB], identical in every block
    RT* s_tmp = s_sums + NV * NB;                     // [blockDim]
    int* s_newton = reinterpret_cast<int*>(s_tmp + blockDim.x);
    int* s_pcg = s_newton + NB;
    int* s_nacc = s_pcg + NB;      // accepted Newton steps of the current time step
    int* s_lit = s_nacc + NB;      // PCG iterations each lane needed during this launch
    __shared__ int s_err;
    RT* part_buf[2] = {static_cast<RT*>(a.part), static_cast<RT*>(a.part) + (size_t)nblk * NV * NB};
    int parity = 0;

    // the vectors never alias one another
    T* __restrict__ r = static_cast<T*>(a.r);
    T* __restrict__ z = static_cast<T*>(a.z);
    T* w = static_cast<T*>(a.w);
    T* p = static_cast<T*>(a.p);
    T* s = static_cast<T*>(a.s);
    T* __restrict__ J = static_cast<T*>(a.J);
    T* __restrict__ invd = static_cast<T*>(a.invd_sp);
    const T* KlinT = std::is_same<T, float>::value ? reinterpret_cast<const T*>(m.Klin32)
                                                   : reinterpret_cast<const T*>(m.Klin);
    const T* invdiag_linT = std::is_same<T, float>::value ? reinterpret_cast<const T*>(m.invdiag_lin32)
                                                          : reinterpret_cast<const T*>(m.invdiag_lin);
    // state vectors from this team's first lane on, row stride LD
    double* u = a.u + lane0;
    double* uprev = a.uprev + lane0;
    double* uprev2 = a.uprev2 ? a.uprev2 + lane0 : nullptr;
    double* traj_out = a.traj_out ? a.traj_out + lane0 : nullptr;
    // this block owns the contiguous rows [rs, re)
    const int rs = a.row_start[bid], re = a.row_start[bid + 1];
    // p, s, x, w are only touched by their owning block: when a.vec_rows > 0
    // they live in shared memory (indexed from row rs), else in global memory
    T* __restrict__ pB = p;
    T* __restrict__ sB = s;
    T* __restrict__ xB = static_cast<T*>(a.x);
    T* __restrict__ wB = w;
    size_t vo = 0;   // row offset of the shared-memory vectors (0: global vectors)
    size_t wo = 0;
    if (a.vec_rows > 0) {
        T* sv = reinterpret_cast<T*>(
            (reinterpret_cast<uintptr_t>(s_lit + NB) + 15) & ~static_cast<uintptr_t>(15));
        const size_t len = (size_t)a.vec_rows * NB;
        pB = sv;
        sB = sv + len;
        xB = sv + 2 * len;
        vo = (size_t)rs * NB;
        if (a.vec_w) {
            wB = sv + 3 * len;
            wo = vo;
        }
        for (size_t q = tid; q < 2 * len; q += blockDim.x) sv[q] = (T)0;   // p = s = 0
    }
    const int row0 = rs + rb;
    const double tol_abs = a.tol_abs_dev ? *a.tol_abs_dev : a.tol_abs;
    // multigrid levels (precond = 2), copied to shared memory
    __shared__ AmgLevel s_amg[kAmgMaxLevels];
    const bool amg = a.amg != nullptr;
    if (amg) {
        static_assert(sizeof(AmgLevel) % sizeof(int) == 0, "AmgLevel copied as words");
        const int words = a.amg_levels * (int)(sizeof(AmgLevel) / sizeof(int));
        const int* src = reinterpret_cast<const int*>(a.amg);
        int* dst = reinterpret_cast<int*>(s_amg);
        for (int q = tid; q < words; q += blockDim.x) dst[q] = src[q];
        __syncthreads();
    }
    __shared__ int2 s_rng[kAmgMaxLevels];
    if (amg) amg_block_ranges(s_amg, a.amg_levels, bid, nblk, s_rng);
    T* l1f = amg ? static_cast<T*>(a.amg_ws) + s_amg[0].off_l1 * NB : nullptr;
    const AmgCtx actx{NB,           a.amg_levels, a.amg_sweeps,  a.amg_ws, a.J, a.bar, a.status,
                      a.long_start, a.long_rows,  s_rng};
    const long long n_elem_items = (long long)m.n_nl * NB;
    const long long gthreads = (long long)nblk * blockDim.x;
    // iteration counts, kept by thread 0: newton tests, pcg iterations, pcg
    // iterations since the last Newton test, rounds with a backtracking lane
    __shared__ long long s_cnt[4];
    if (tid == 0) s_cnt[0] = s_cnt[1] = s_cnt[2] = s_cnt[3] = 0;
    if (tid == 0) s_err = 0;
    for (int l = tid; l < NB; l += blockDim.x) s_lit[l] = 0;
    if (a.team_ns && bid == 0 && tid == 0) a.team_ns[0] = global_ns();

    for (int step = 0; step < a.n_fine; ++step) {
        for (int l = tid; l < NB; l += blockDim.x) {
            double I = 0.0;
            const int lg = lane0 + l;   // the problem's lane = subinterval lg + 1
            if (lg < a.N) {
                const double t = (double)((long long)lg * a.n_total + a.level0 + step + 1) * a.dt;
                for (int h = 0; h < a.src.n_harm; ++h)
                    I += a.src.amp[h] * sin(2.0 * kPi * a.src.freq[h] * t + a.src.phase[h]);
            }
            s_I[l] = I;
            s_newton[l] = (lg < a.N);
            s_nacc[l] = 0;
            s_lam[l] = 1.0;
        }
        // u_prev = u^m on own rows; Newton starts from u^m, or from the linear
        // extrapolation 2 u^m - u^{m-1} once a previous step exists.  In the
        // adjoint, u is lambda, u_prev = lambda_{m+1}, and level j counts down.
        const int j = a.adjoint ? a.n_fine - step : step;
        const bool extrap = !a.adjoint && a.predictor && step > 0;
        const bool quad = a.predictor == 2 && !a.adjoint;   // keeps u^{m-2} in uprev2
        for (int i = row0; i < re; i += RB) {
            const size_t o = (size_t)i * LD + l0;
            const Lanes<double, V> um = ldv<double, V>(u + o);
            if (traj_out && step == 0) stv<double, V>(traj_out + o, um);
            if (extrap || quad) {
                const Lanes<double, V> uo = ldv<double, V>(uprev + o);
                if (extrap) {
                    Lanes<double, V> un;
                    if (quad && step > 1) {
                        const Lanes<double, V> uo2 = ldv<double, V>(uprev2 + o);
#pragma unroll
                        for (int h = 0; h < V; ++h) un.v[h] = 3.0 * (um.v[h] - uo.v[h]) + uo2.v[h];
                    } else {
#pragma unroll
                        for (int h = 0; h < V; ++h) un.v[h] = um.v[h] + (um.v[h] - uo.v[h]);
                    }
                    stv<double, V>(u + o, un);
                }
                if (quad) stv<double, V>(uprev2 + o, uo);
            }
            stv<double, V>(uprev + o, um);
        }
        if (extrap && !grid_sync(a.bar, a.status, bid, nblk)) return;
        {
            // element data of the state the Jacobian is taken at: the Newton
            // iterate, or in the adjoint the forward state u^m (fixed for the level)
            const double* eu = a.adjoint ? a.traj + (size_t)j * m.ndof * LD : a.u;
            for (long long it = bid * (long long)blockDim.x + tid; it < n_elem_items; it += gthreads)
                elem_compute(m, LD, eu, a.elem, (int)(it / NB), lane0 + (int)(it % NB));
        }
        if (!grid_sync(a.bar, a.status, bid, nblk)) return;

        for (int nit = 0;; ++nit) {
            // ---- residual R(u), per-lane Jacobian of special rows, r = -R, z = D^-1 r, x = 0
            double accR[V], accb[V];
            T accz[V];
#pragma unroll
            for (int h = 0; h < V; ++h) {
                accR[h] = accb[h] = 0.0;
                accz[h] = 0;
            }
            if (a.adjoint)
                adjoint_rows<T, V>(a, m, row0, re, RB, l0, j, accR, accz, accb, xB, vo, l1f);
            else
                residual_rows<T, V>(a, m, row0, re, RB, l0, s_I, accR, accz, xB, vo, l1f);
            if (amg) {
                // every lane's coarse matrices from its Jacobian at the step's
                // first Newton iteration (the later iterations of the step keep
                // them: Galerkin products of an SPD Jacobian stay SPD, and the
                // fine level smooths with the current Jacobian), then z = B r
                if (!grid_sync(a.bar, a.status, bid, nblk)) return;
                if (nit == 0 && !amg_coarse_values<T, V>(actx, s_amg, bid, nblk)) return;
                if (!amg_vcycle<T, V>(actx, m, s_amg, KlinT, J, r, z, bid, nblk, re, row0, RB, rb, l0, G, s_red, s_tmp))
                    return;
            } else if (a.tri > 0) {
                // the chunk preconditioner replaces z = D^-1 r (r of other threads' rows: sync)
                __syncthreads();
#pragma unroll
                for (int h = 0; h < V; ++h) accz[h] = 0;
                tri_factor<T, V>(a, m, rs, re, RB, rb, l0, accz);
            }
            {
                RT v[NV][V];
#pragma unroll
                for (int h = 0; h < V; ++h) {
                    v[0][h] = (RT)accR[h];
                    v[1][h] = accz[h];
                    v[2][h] = (RT)accb[h];
                }
                block_partials<RT, V, NV>(s_red, G, NB, l0, v, part_buf[parity] + (size_t)bid * NV * NB);
            }
            if (!grid_sync(a.bar, a.status, bid, nblk)) return;
            block_reduce_all<RT>(part_buf[parity], NV * NB, s_sums, s_tmp, nblk);
            parity ^= 1;

            // ---- Newton test per lane; PCG forcing term per lane.  A lane
            // whose FP64 residual did not drop (or is not finite) after a step
            // backtracks: the step is halved (u -= lam/2 dx) and tested again.
            int act = 0, bt = 0;
            for (int l = tid; l < NB; l += blockDim.x) {
                int al = 0;
                double coef = 0.0;
                if (s_newton[l]) {
                    const double rr = (double)s_sums[l];
                    const double Rn = sqrt(rr);
                    const bool fin = isfinite(Rn);
                    // the adjoint's residual is linear: its tolerance is relative to ||b||
                    const double tol = a.adjoint ? a.tol_rel * sqrt((double)s_sums[2 * NB + l]) : tol_abs;
                    if (fin && (Rn <= tol || (nit > 0 && Rn <= kFloorMult * tol && Rn >= kStagnation * s_rprev[l]))) {
                        // converged, or stalled at the rounding floor just above the tolerance
                        s_newton[l] = 0;
                    } else if (nit > 0 && (!fin || Rn > (1.0 - 1e-4 * s_lam[l]) * s_rprev[l])) {
                        if (s_lam[l] <= kMinStep) {
                            set_status(a.status, fin ? DEV_ERR_NEWTON : DEV_ERR_NAN);
                            s_err = 1;
                        } else {
                            coef = -0.5 * s_lam[l];
                            s_lam[l] *= 0.5;
                            bt = 1;
                        }
                    } else if (!fin) {
                        set_status(a.status, DEV_ERR_NAN);
                        s_err = 1;
                    } else if (s_nacc[l] >= a.max_newton) {
                        set_status(a.status, DEV_ERR_NEWTON);
                        s_err = 1;
                    } else {
                        // Eisenstat-Walker forcing: eta = 0.9 (|R_k| / |R_k-1|)^2, kept from
                        // dropping faster than 0.9 eta_{k-1}^2, within [tol_lin, 0.1],
                        // and never tighter than needed to reach the Newton tolerance
                        double eta = a.eta0;
                        if (nit > 0) {
                            const double q = Rn / s_rprev[l];
                            eta = 0.9 * q * q;
                            const double safe = 0.9 * s_eta[l] * s_eta[l];
                            if (safe > 0.1) eta = fmax(eta, safe);
                        }
                        eta = fmin(fmax(eta, a.tol_lin), 0.1);
                        eta = fmax(eta, fmin(0.1, 0.1 * tol / Rn));
                        s_eta[l] = eta;
                        // PCG stops once ||r||_2 (the Newton residual's norm) has dropped by eta
                        s_stop[l] = eta * eta * rr;
                        s_rprev[l] = Rn;
                        s_lam[l] = 1.0;
                        s_nacc[l] += 1;
                        coef = 1.0;
                        al = 1;
                    }
                }
                s_pcg[l] = al;
                s_coef[l] = coef;
                act |= al | bt;
            }
            if (__syncthreads_or(bt) && tid == 0) ++s_cnt[3];
            const int any_newton = __syncthreads_or(act);
            if (a.trace && bid == 0 && tid == 0) {
                double rmax = 0.0;
                int nact = 0;
                for (int l = 0; l < a.N; ++l) {
                    rmax = fmax(rmax, sqrt((double)s_sums[l]));
                    nact += s_pcg[l];
                }
                const int rec = atomicAdd(a.trace_len, 1);
                if (rec < a.trace_cap) {
                    double* t = a.trace + (size_t)rec * kTraceFields;
                    t[0] = step;
                    t[1] = nit;
                    t[2] = rmax;
                    t[3] = nact;
                    t[4] = (double)s_cnt[2];
                }
            }
            if (tid == 0) s_cnt[2] = 0;
            if (s_err) return;
            if (!any_newton) break;
            if (tid == 0) ++s_cnt[0];

            // ---- PCG on J x = -R
            for (int k = 0;; ++k) {
                T rr[V], rz[V], zw[V];
#pragma unroll
                for (int h = 0; h < V; ++h) rr[h] = rz[h] = zw[h] = 0;
                // rows longer than kLongRow are left to the whole block below
                for (int i = row0; i < re; i += RB) {
                    const int kb = m.rowptr[i], ke = m.rowptr[i + 1];
                    if (ke - kb > kLongRow) continue;
                    const int slot0 = m.row_slot[i];
                    T wv[V];
#pragma unroll
                    for (int h = 0; h < V; ++h) wv[h] = 0;
                    if (slot0 < 0)
                        gather_shared<T, V>(wv, kb, ke, m.col, KlinT, z, NB, l0);
                    else
                        gather_lanes<T, V>(wv, kb, ke, m.col, J, slot0, z, NB, l0);
                    const size_t o = (size_t)i * NB + l0;
                    Lanes<T, V> wl;
#pragma unroll
                    for (int h = 0; h < V; ++h) wl.v[h] = wv[h];
                    stv<T, V>(wB + (o - wo), wl);
                    const Lanes<T, V> ri = ldv<T, V>(r + o);
                    const Lanes<T, V> zi = ldv<T, V>(z + o);
#pragma unroll
                    for (int h = 0; h < V; ++h) {
                        rr[h] += ri.v[h] * ri.v[h];
                        rz[h] += ri.v[h] * zi.v[h];
                        zw[h] += zi.v[h] * wv[h];
                    }
                }
                // long rows (e.g. the centre node of a polar mesh): every row group
                // takes a strided share of the nonzeros, then a fixed-order sum
                for (int lr = a.long_start[bid]; lr < a.long_start[bid + 1]; ++lr) {
                    const int i = a.long_rows[lr];
                    const int kb = m.rowptr[i], ke = m.rowptr[i + 1], slot0 = m.row_slot[i];
                    T wp[V];
#pragma unroll
                    for (int h = 0; h < V; ++h) wp[h] = 0;
                    for (int kk = kb + rb; kk < ke; kk += RB) {
                        const Lanes<T, V> zj = ldv<T, V>(z + (size_t)m.col[kk] * NB + l0);
                        if (slot0 < 0) {
                            const T kv = KlinT[kk];
#pragma unroll
                            for (int h = 0; h < V; ++h) wp[h] += kv * zj.v[h];
                        } else {
                            const Lanes<T, V> jv = ldv<T, V>(J + (size_t)(slot0 + kk - kb) * NB + l0);
#pragma unroll
                            for (int h = 0; h < V; ++h) wp[h] += jv.v[h] * zj.v[h];
                        }
                    }
                    // combine the row groups: shuffle within a warp, then warps in order
                    {
                        RT vv[1][V];
#pragma unroll
                        for (int h = 0; h < V; ++h) vv[0][h] = wp[h];
                        block_partials<RT, V, 1>(s_red, G, NB, l0, vv, s_tmp);
                    }
                    __syncthreads();
                    if (rb == 0) {
                        const size_t o = (size_t)i * NB + l0;
                        T wv[V];
#pragma unroll
                        for (int h = 0; h < V; ++h) wv[h] = s_tmp[l0 + h];
                        Lanes<T, V> wl;
#pragma unroll
                        for (int h = 0; h < V; ++h) wl.v[h] = wv[h];
                        stv<T, V>(wB + (o - wo), wl);
                        const Lanes<T, V> ri = ldv<T, V>(r + o);
                        const Lanes<T, V> zi = ldv<T, V>(z + o);
#pragma unroll
                        for (int h = 0; h < V; ++h) {
                            rr[h] += ri.v[h] * ri.v[h];
                            rz[h] += ri.v[h] * zi.v[h];
                            zw[h] += zi.v[h] * wv[h];
                        }
                    }
                    __syncthreads();
                }
                {
                    RT v[NV][V];
#pragma unroll
                    for (int h = 0; h < V; ++h) {
                        v[0][h] = rr[h];
                        v[1][h] = rz[h];
                        v[2][h] = zw[h];
                    }
                    block_partials<RT, V, NV>(s_red, G, NB, l0, v, part_buf[parity] + (size_t)bid * NV * NB);
                }
                if (!grid_sync(a.bar, a.status, bid, nblk)) return;
                block_reduce_all<RT>(part_buf[parity], NV * NB, s_sums, s_tmp, nblk);
                parity ^= 1;

                int act2 = 0;
                for (int l = tid; l < NB; l += blockDim.x) {
                    double al = 0.0, be = 0.0;
                    int on = 0;
                    if (s_pcg[l]) {
                        const double rho = (double)s_sums[l];
                        const double gam = (double)s_sums[NB + l];
                        const double del = (double)s_sums[2 * NB + l];
                        if (!isfinite(rho) || !isfinite(gam) || !isfinite(del)) {
                            set_status(a.status, DEV_ERR_NAN);
                            s_err = 1;
                        } else if (rho <= s_stop[l]) {
                            s_pcg[l] = 0;
                        } else if (k >= a.max_lin) {
                            set_status(a.status, DEV_ERR_LINEAR);
                            s_err = 1;
                        } else {
                            // scalar recurrences in the PCG precision
                            const T gg = (T)gam, d = (T)del;
                            const T b = (k == 0) ? (T)0 : gg / (T)s_gold[l];
                            const T den = (k == 0) ? d : d - b * gg / (T)s_aold[l];
                            if (!(den > (T)0) || !(gg > (T)0)) {
                                set_status(a.status, DEV_ERR_BREAKDOWN);
                                s_err = 1;
                            } else {
                                al = (double)(gg / den);
                                be = (double)b;
                                s_gold[l] = (double)gg;
                                s_aold[l] = al;
                                on = 1;
                                if (bid == 0) ++s_lit[l];
                            }
                        }
                    }
                    s_alpha[l] = on ? al : 0.0;
                    s_beta[l] = on ? be : 0.0;
                    act2 |= on;
                }
                const int any_pcg = __syncthreads_or(act2);
                if (s_err) return;
                if (!any_pcg) break;
                if (tid == 0) {
                    ++s_cnt[1];
                    ++s_cnt[2];
                }

                const bool tri = a.tri > 0;
                T alv[V], bev[V];
#pragma unroll
                for (int h = 0; h < V; ++h) {
                    alv[h] = (T)s_alpha[l0 + h];
                    bev[h] = (T)s_beta[l0 + h];
                }
#pragma unroll 2
                for (int i = row0; i < re; i += RB) {
                    const size_t o = (size_t)i * NB + l0;
                    const size_t ov = o - vo;
                    const Lanes<T, V> zi = ldv<T, V>(z + o);
                    const Lanes<T, V> wi = ldv<T, V>(wB + (o - wo));
                    const Lanes<T, V> pi = ldv<T, V>(pB + ov);
                    const Lanes<T, V> si = ldv<T, V>(sB + ov);
                    const Lanes<T, V> ri = ldv<T, V>(r + o);
                    const Lanes<T, V> xi = ldv<T, V>(xB + ov);
                    Lanes<T, V> pn, sn, rn, xn;
#pragma unroll
                    for (int h = 0; h < V; ++h) {
                        // first iteration: p = z, s = w (whatever p and s held before)
                        pn.v[h] = k == 0 ? zi.v[h] : zi.v[h] + bev[h] * pi.v[h];
                        sn.v[h] = k == 0 ? wi.v[h] : wi.v[h] + bev[h] * si.v[h];
                        rn.v[h] = ri.v[h] - alv[h] * sn.v[h];
                        xn.v[h] = xi.v[h] + alv[h] * pn.v[h];
                    }
                    stv<T, V>(pB + ov, pn);
                    stv<T, V>(sB + ov, sn);
                    stv<T, V>(r + o, rn);
                    stv<T, V>(xB + ov, xn);
                    if (!tri && !amg) {
                        // Jacobi: z = D^-1 r
                        Lanes<T, V> ivl, zn;
                        const int sp = m.sp_index[i];
                        if (sp < 0) {
                            const T d = invdiag_linT[i];
#pragma unroll
                            for (int h = 0; h < V; ++h) ivl.v[h] = d;
                        } else {
                            ivl = ldv<T, V>(invd + (size_t)sp * NB + l0);
                        }
#pragma unroll
                        for (int h = 0; h < V; ++h) zn.v[h] = rn.v[h] * ivl.v[h];
                        stv<T, V>(z + o, zn);
                    }
                }
                if (tri) {
                    __syncthreads();   // the chunks' r were updated by other row groups
                    tri_solve<T, V>(a, rs, re, RB, rb, l0);
                } else if (amg) {
                    if (!amg_vcycle<T, V>(actx, m, s_amg, KlinT, J, r, z, bid, nblk, re, row0, RB, rb, l0, G, s_red,
                                          s_tmp))
                        return;
                }
                if (!grid_sync(a.bar, a.status, bid, nblk)) return;
            }
            // ---- own rows: apply this iteration's steps, then element data at the new u
            apply_steps<T, V>(u, LD, xB, vo, static_cast<T*>(a.dx), s_eta + NB, row0, re, RB, l0, NB);
            if (!grid_sync(a.bar, a.status, bid, nblk)) return;
            if (!a.adjoint) {
                for (long long it = bid * (long long)blockDim.x + tid; it < n_elem_items; it += gthreads)
                    elem_compute(m, LD, a.u, a.elem, (int)(it / NB), lane0 + (int)(it % NB));
                if (!grid_sync(a.bar, a.status, bid, nblk)) return;
            }
        }
        // ---- record the level just solved (own rows)
        double* rec = a.adjoint ? (a.lam_out ? a.lam_out + lane0 + (size_t)(j - 1) * m.ndof * LD : nullptr)
                                : (traj_out ? traj_out + (size_t)(step + 1) * m.ndof * LD : nullptr);
        if (rec)
            for (int i = row0; i < re; i += RB) {
                const size_t o = (size_t)i * LD + l0;
                stv<double, V>(rec + o, ldv<double, V>(u + o));
            }
    }
    if (bid == 0 && tid == 0) {
        // per team: rounds are this team's lockstep rounds; the last team to
        // finish adds the maxima over teams (the launch's critical path)
        long long useful = 0;
        for (int l = 0; l < NB; ++l) useful += s_lit[l];
        atomicMax(&a.sweep_max[0], s_cnt[0]);
        atomicMax(&a.sweep_max[1], s_cnt[1]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.counters[kCntBacktrack]), (unsigned long long)s_cnt[3]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.counters[kCntPcgLaneRounds]),
                  (unsigned long long)(s_cnt[1] * NB));
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.counters[kCntPcgLaneIters]), (unsigned long long)useful);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.counters[kCntNewtonLaneRounds]),
                  (unsigned long long)(s_cnt[0] * NB));
        __threadfence();
        if (atomicAdd(a.teams_done, 1u) == (unsigned int)a.n_teams - 1u) {
            __threadfence();
            a.counters[kCntNewton] += atomicAdd(reinterpret_cast<unsigned long long*>(&a.sweep_max[0]), 0ull);
            a.counters[kCntPcg] += atomicAdd(reinterpret_cast<unsigned long long*>(&a.sweep_max[1]), 0ull);
        }
        if (a.team_ns) a.team_ns[1] = global_ns();
    }
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) fine_sweep_kernel(const FineArgs a) {
    fine_sweep_body<T>(a, blockIdx.x, gridDim.x);
}

// Batched launch: block b serves member map[b].x as block map[b].y of a team
// of map[b].z blocks (map[b].x < 0: idle).  The member's arguments are
// copied to shared memory once.
template <typename T>
__global__ void __launch_bounds__(1024, 1) fine_batch_kernel(const FineArgs* args, const int4* map) {
    __shared__ FineArgs s_a;
    const int4 mb = map[blockIdx.x];
    if (mb.x < 0) return;
    static_assert(sizeof(FineArgs) % sizeof(int) == 0, "FineArgs copied as words");
    const int* src = reinterpret_cast<const int*>(args + mb.x);
    int* dst = reinterpret_cast<int*>(&s_a);
    for (int q = threadIdx.x; q < (int)(sizeof(FineArgs) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    fine_sweep_body<T>(s_a, mb.y, mb.z);
}


}  // namespace

size_t fine_smem(bool fp32, int NB, int threads, int vec_rows, int vec_count) {
    const int V = fp32 ? 4 : 2;
    const int slots = red_slots(NB / V, threads);
    const size_t rt = fp32 ? sizeof(float) : sizeof(double);
    size_t b = (size_t)10 * NB * sizeof(double) + (size_t)(NV * slots * NB + NV * NB + threads) * rt +
               4 * NB * sizeof(int);
    if (vec_rows > 0) b += 16 + (size_t)vec_count * vec_rows * NB * rt;
    return b;
}

cudaError_t fine_config(bool fp32, int NB, int vec_rows, int vec_count, LaunchCfg* cfg) {
    const int V = fp32 ? 4 : 2;
    const int G = NB / V;
    if (G < 1 || G > 512 || NB % V != 0) return cudaErrorInvalidValue;
    const int threads = G * (1024 / G);
    const size_t smem = fine_smem(fp32, NB, threads, vec_rows, vec_count);
    const void* fn = fp32 ? (const void*)fine_sweep_kernel<float> : (const void*)fine_sweep_kernel<double>;
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

cudaError_t launch_fine_sweep(const FineArgs& a, bool fp32, const LaunchCfg& cfg, cudaStream_t st) {
    void* args[] = {const_cast<FineArgs*>(&a)};
    const void* fn = fp32 ? (const void*)fine_sweep_kernel<float> : (const void*)fine_sweep_kernel<double>;
    return cudaLaunchCooperativeKernel(fn, dim3(cfg.blocks), dim3(cfg.threads), args, cfg.smem, st);
}

cudaError_t fine_batch_prepare(bool fp32, size_t* static_smem) {
    const void* fn = fp32 ? (const void*)fine_batch_kernel<float> : (const void*)fine_batch_kernel<double>;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (static_smem) *static_smem = fa.sharedSizeBytes;
    return allow_max_dynamic_smem(fn);
}

cudaError_t launch_fine_batch(const FineArgs* args, const int4* map, bool fp32, int blocks, size_t smem,
                              cudaStream_t st) {
    // cudaLaunchKernelEx with the cooperative attribute: capturable in a graph
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (fp32) return cudaLaunchKernelEx(&cfg, fine_batch_kernel<float>, args, map);
    return cudaLaunchKernelEx(&cfg, fine_batch_kernel<double>, args, map);
}

void launch_elem_data(const MeshDev& m, int NB, const double* u, double* elem, cudaStream_t st) {
    const long long total = (long long)m.n_nl * NB;
    if (total == 0) return;
    long long b = (total + 255) / 256;
    if (b > 65535) b = 65535;
    elem_data_kernel<<<(int)b, 256, 0, st>>>(m, NB, u, elem);
}

}  // namespace pppc

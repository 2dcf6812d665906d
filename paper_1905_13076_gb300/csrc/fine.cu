// Batched fine propagators F_n of PP-PC (Sec. 2, Eqs. 2-3).
//
// All N subintervals march at once: lane n of every vector is subinterval
// n+1, started from U_n at T_n.  Each implicit-Euler step of size dt solves
//     R(u) = (M/dt)(u - u_prev) + K(u) u - I(t) g = 0
// by Newton's method; each Newton correction solves J du = -R with Jacobi-
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
// Layout: vectors are [ndof][NB] (lane fastest); a thread owns 2 adjacent
// lanes of fixed rows for the whole launch, so row-local data is only ever
// touched by its owner; other rows' data is read only after a grid barrier.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace pppc {

// Element data of nonlinear element q, lane `lane`, from the state u:
//   grad A = sum_a u_a grad N_a,  b = |grad A|^2,
//   nu = k1 exp(k2 b) + k3,  dnu/db = k1 k2 exp(k2 b),
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
    const double ex = exp(K[1] * b);
    const double nu = K[0] * ex + K[2];
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

// Fixed-order in-block sum over the row slots of each lane, written as this
// block's partials part[blockIdx.x * NV * NB + v * NB + lane].
template <typename RT>
__device__ __forceinline__ void block_partials(RT* s_red, int RB, int NB, int rb, int l0, const RT (&v)[NV][2],
                                               RT* part) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        s_red[(q * RB + rb) * NB + l0] = v[q][0];
        s_red[(q * RB + rb) * NB + l0 + 1] = v[q][1];
    }
    __syncthreads();
    // fixed pairwise tree over the row slots: fold the upper half onto the lower
    for (int n = RB; n > 1;) {
        const int half = (n + 1) >> 1, cnt = (n - half) * NB;
        for (int idx = threadIdx.x; idx < NV * cnt; idx += blockDim.x) {
            const int q = idx / cnt, rem = idx - q * cnt;
            const int t = rem / NB, l = rem - t * NB;
            s_red[(q * RB + t) * NB + l] += s_red[(q * RB + t + half) * NB + l];
        }
        __syncthreads();
        n = half;
    }
    RT* out = part + (size_t)blockIdx.x * NV * NB;
    for (int o = threadIdx.x; o < NV * NB; o += blockDim.x) {
        const int q = o / NB, l = o - q * NB;
        out[o] = s_red[(q * RB) * NB + l];
    }
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) fine_sweep_kernel(const FineArgs a) {
    extern __shared__ double smem[];
    const MeshDev m = a.mesh;
    const int NB = a.NB, G = NB >> 1;
    const int tid = threadIdx.x, g = tid % G, rb = tid / G, RB = blockDim.x / G;
    const int l0 = 2 * g;
    double* s_I = smem;            // current I(t) of each lane at the new time level
    double* s_stop = s_I + NB;     // PCG stop threshold on (r,r)
    double* s_gold = s_stop + NB;  // previous (r,z)
    double* s_aold = s_gold + NB;  // previous step length
    double* s_alpha = s_aold + NB;
    double* s_beta = s_alpha + NB;
    double* s_rprev = s_beta + NB; // ||R|| at the previous Newton test
    double* s_eta = s_rprev + NB;  // previous forcing term
    // reductions run in the PCG precision: FP32 sums in the mixed path
    using RT = T;
    RT* s_red = reinterpret_cast<RT*>(s_eta + NB);   // [NV][RB][NB]
    RT* s_sums = s_red + NV * RB * NB;                // [NV][NB], identical in every block
    RT* s_tmp = s_sums + NV * NB;                     // [blockDim]
    int* s_newton = reinterpret_cast<int*>(s_tmp + blockDim.x);
    int* s_pcg = s_newton + NB;
    __shared__ int s_err;
    RT* part_buf[2] = {static_cast<RT*>(a.part), static_cast<RT*>(a.part) + (size_t)gridDim.x * NV * NB};
    int parity = 0;

    T* r = static_cast<T*>(a.r);
    T* z = static_cast<T*>(a.z);
    T* w = static_cast<T*>(a.w);
    T* p = static_cast<T*>(a.p);
    T* s = static_cast<T*>(a.s);
    T* x = static_cast<T*>(a.x);
    T* J = static_cast<T*>(a.J);
    T* invd = static_cast<T*>(a.invd_sp);
    const T* KlinT = std::is_same<T, float>::value ? reinterpret_cast<const T*>(m.Klin32)
                                                   : reinterpret_cast<const T*>(m.Klin);
    const T* invdiag_linT = std::is_same<T, float>::value ? reinterpret_cast<const T*>(m.invdiag_lin32)
                                                          : reinterpret_cast<const T*>(m.invdiag_lin);
    double* u = a.u;
    double* uprev = a.uprev;
    const double* E = a.elem;
    const size_t P = (size_t)m.n_nl * NB;
    const int rstride = gridDim.x * RB;
    const int row0 = blockIdx.x * RB + rb;
    const long long n_elem_items = (long long)m.n_nl * NB;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    long long newton_total = 0, pcg_total = 0, pcg_since = 0;
    if (tid == 0) s_err = 0;

    for (int step = 0; step < a.n_fine; ++step) {
        for (int l = tid; l < NB; l += blockDim.x) {
            double I = 0.0;
            if (l < a.N) {
                const double t = (double)((long long)l * a.n_fine + step + 1) * a.dt;
                for (int h = 0; h < a.src.n_harm; ++h)
                    I += a.src.amp[h] * sin(2.0 * kPi * a.src.freq[h] * t + a.src.phase[h]);
            }
            s_I[l] = I;
            s_newton[l] = (l < a.N);
        }
        // u_prev = u^m on own rows; Newton starts from u^m, or from the linear
        // extrapolation 2 u^m - u^{m-1} once a previous step exists
        const bool extrap = a.predictor && step > 0;
        for (int i = row0; i < m.ndof; i += rstride) {
            const size_t o = (size_t)i * NB + l0;
            const double2 um = *reinterpret_cast<const double2*>(u + o);
            if (extrap) {
                const double2 uo = *reinterpret_cast<const double2*>(uprev + o);
                st2<double>(u + o, um.x + (um.x - uo.x), um.y + (um.y - uo.y));
            }
            st2<double>(uprev + o, um.x, um.y);
        }
        if (extrap && !grid_sync(a.bar, a.status)) return;
        for (long long it = blockIdx.x * (long long)blockDim.x + tid; it < n_elem_items; it += gthreads)
            elem_compute(m, NB, u, a.elem, (int)(it / NB), (int)(it % NB));
        if (!grid_sync(a.bar, a.status)) return;

        for (int nit = 0;; ++nit) {
            // ---- residual R(u), per-lane Jacobian of special rows, r = -R, z = D^-1 r, x = 0
            double accR0 = 0.0, accR1 = 0.0;
            T accz0 = 0, accz1 = 0;
            for (int i = row0; i < m.ndof; i += rstride) {
                const int kb = m.rowptr[i], ke = m.rowptr[i + 1];
                const int slot0 = m.row_slot[i];
                // K_lin u in difference form: sum_{j != i} K_ij (u_j - u_i) + dlin_i u_i
                const double2 ui = *reinterpret_cast<const double2*>(u + (size_t)i * NB + l0);
                const double dl = m.dlin[i];
                double a0 = dl * ui.x, a1 = dl * ui.y;
                T iv0, iv1;
                if (slot0 < 0) {
                    for (int k = kb; k < ke; ++k) {
                        const int j = m.col[k];
                        if (j == i) continue;
                        const double kv = m.Klin[k];
                        const double2 uj = gld2(u + (size_t)j * NB + l0);
                        a0 += kv * (uj.x - ui.x);
                        a1 += kv * (uj.y - ui.y);
                    }
                    iv0 = iv1 = invdiag_linT[i];
                } else {
                    double d0 = 1.0, d1 = 1.0;
                    for (int k = kb; k < ke; ++k) {
                        const int sl = slot0 + (k - kb);
                        const int j = m.col[k];
                        const double kv = m.Klin[k];
                        const double mv = m.Mslot[sl] * a.inv_dt;
                        const double2 uj = gld2(u + (size_t)j * NB + l0);
                        const double2 upj = gld2(uprev + (size_t)j * NB + l0);
                        const double kl = (j == i) ? 0.0 : kv;
                        a0 += kl * (uj.x - ui.x) + mv * (uj.x - upj.x);
                        a1 += kl * (uj.y - ui.y) + mv * (uj.y - upj.y);
                        double J0 = kv + mv, J1 = kv + mv;
                        for (int c = m.nlc_ptr[sl]; c < m.nlc_ptr[sl + 1]; ++c) {
                            const int pk = m.nlc[c];
                            const int q = pk / 9, ia = (pk / 3) % 3, ib = pk % 3;
                            const double ab = m.nlc_ab[c];
                            const size_t o = (size_t)q * NB + l0;
                            const double2 c1 = gld2(E + o);
                            const double2 c2 = gld2(E + P + o);
                            const double2 sa = gld2(E + (2 + ia) * P + o);
                            const double2 sb = gld2(E + (2 + ib) * P + o);
                            J0 += c1.x * ab + c2.x * sa.x * sb.x;
                            J1 += c1.y * ab + c2.y * sa.y * sb.y;
                            if (j == i) {
                                a0 += c1.x * sa.x;
                                a1 += c1.y * sa.y;
                            }
                        }
                        st2<T>(J + (size_t)sl * NB + l0, (T)J0, (T)J1);
                        if (j == i) {
                            d0 = J0;
                            d1 = J1;
                        }
                    }
                    iv0 = (T)(1.0 / d0);
                    iv1 = (T)(1.0 / d1);
                    st2<T>(invd + (size_t)m.sp_index[i] * NB + l0, iv0, iv1);
                }
                const double gi = m.g[i];
                const double R0 = a0 - s_I[l0] * gi, R1 = a1 - s_I[l0 + 1] * gi;
                const T r0 = (T)(-R0), r1 = (T)(-R1);
                const T z0 = r0 * iv0, z1 = r1 * iv1;
                const size_t o = (size_t)i * NB + l0;
                st2<T>(r + o, r0, r1);
                st2<T>(z + o, z0, z1);
                st2<T>(x + o, (T)0, (T)0);
                accR0 += R0 * R0;
                accR1 += R1 * R1;
                accz0 += r0 * z0;
                accz1 += r1 * z1;
            }
            {
                const RT v[NV][2] = {{(RT)accR0, (RT)accR1}, {(RT)accz0, (RT)accz1}, {(RT)0, (RT)0}};
                block_partials<RT>(s_red, RB, NB, rb, l0, v, part_buf[parity]);
            }
            if (!grid_sync(a.bar, a.status)) return;
            block_reduce_all<RT>(part_buf[parity], NV * NB, s_sums, s_tmp);
            parity ^= 1;

            // ---- Newton test per lane; PCG forcing term per lane
            int act = 0;
            for (int l = tid; l < NB; l += blockDim.x) {
                int al = 0;
                if (s_newton[l]) {
                    const double rr = (double)s_sums[l];
                    const double Rn = sqrt(rr);
                    if (!isfinite(Rn)) {
                        set_status(a.status, DEV_ERR_NAN);
                        s_err = 1;
                    } else if (Rn <= a.tol_abs ||
                               (nit > 0 && Rn <= kFloorMult * a.tol_abs && Rn >= kStagnation * s_rprev[l])) {
                        // converged, or stalled at the rounding floor just above the tolerance
                        s_newton[l] = 0;
                    } else if (nit >= a.max_newton) {
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
                        eta = fmax(eta, fmin(0.1, 0.1 * a.tol_abs / Rn));
                        s_eta[l] = eta;
                        s_stop[l] = eta * eta * rr;
                        s_rprev[l] = Rn;
                        al = 1;
                    }
                }
                s_pcg[l] = al;
                act |= al;
            }
            const int any_newton = __syncthreads_or(act);
            if (a.trace && blockIdx.x == 0 && tid == 0) {
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
                    t[4] = (double)pcg_since;
                }
            }
            pcg_since = 0;
            if (s_err) return;
            if (!any_newton) break;
            ++newton_total;

            // ---- PCG on J x = -R
            for (int k = 0;; ++k) {
                T rr0 = 0, rr1 = 0, rz0 = 0, rz1 = 0, zw0 = 0, zw1 = 0;
                for (int i = row0; i < m.ndof; i += rstride) {
                    const int kb = m.rowptr[i], ke = m.rowptr[i + 1];
                    const int slot0 = m.row_slot[i];
                    T w0 = 0, w1 = 0;
                    if (slot0 < 0) {
                        for (int kk = kb; kk < ke; ++kk) {
                            const T kv = KlinT[kk];
                            const auto zj = gld2(z + (size_t)m.col[kk] * NB + l0);
                            w0 += kv * zj.x;
                            w1 += kv * zj.y;
                        }
                    } else {
                        for (int kk = kb; kk < ke; ++kk) {
                            const auto jv = ld2<T>(J + (size_t)(slot0 + kk - kb) * NB + l0);
                            const auto zj = gld2(z + (size_t)m.col[kk] * NB + l0);
                            w0 += jv.x * zj.x;
                            w1 += jv.y * zj.y;
                        }
                    }
                    const size_t o = (size_t)i * NB + l0;
                    st2<T>(w + o, w0, w1);
                    const auto ri = ld2<T>(r + o);
                    const auto zi = ld2<T>(z + o);
                    rr0 += ri.x * ri.x;
                    rr1 += ri.y * ri.y;
                    rz0 += ri.x * zi.x;
                    rz1 += ri.y * zi.y;
                    zw0 += zi.x * w0;
                    zw1 += zi.y * w1;
                }
                {
                    const RT v[NV][2] = {{rr0, rr1}, {rz0, rz1}, {zw0, zw1}};
                    block_partials<RT>(s_red, RB, NB, rb, l0, v, part_buf[parity]);
                }
                if (!grid_sync(a.bar, a.status)) return;
                block_reduce_all<RT>(part_buf[parity], NV * NB, s_sums, s_tmp);
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
                            const T g = (T)gam, d = (T)del;
                            const T b = (k == 0) ? (T)0 : g / (T)s_gold[l];
                            const T den = (k == 0) ? d : d - b * g / (T)s_aold[l];
                            if (!(den > (T)0) || !(g > (T)0)) {
                                set_status(a.status, DEV_ERR_BREAKDOWN);
                                s_err = 1;
                            } else {
                                al = (double)(g / den);
                                be = (double)b;
                                s_gold[l] = (double)g;
                                s_aold[l] = al;
                                on = 1;
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
                ++pcg_total;
                ++pcg_since;

                const T al0 = (T)s_alpha[l0], al1 = (T)s_alpha[l0 + 1];
                const T be0 = (T)s_beta[l0], be1 = (T)s_beta[l0 + 1];
                for (int i = row0; i < m.ndof; i += rstride) {
                    const size_t o = (size_t)i * NB + l0;
                    const auto zi = ld2<T>(z + o);
                    const auto wi = ld2<T>(w + o);
                    const auto pi = ld2<T>(p + o);
                    const auto si = ld2<T>(s + o);
                    const auto ri = ld2<T>(r + o);
                    const auto xi = ld2<T>(x + o);
                    const T p0 = zi.x + be0 * pi.x, p1 = zi.y + be1 * pi.y;
                    const T s0 = wi.x + be0 * si.x, s1 = wi.y + be1 * si.y;
                    const T r0 = ri.x - al0 * s0, r1 = ri.y - al1 * s1;
                    T iv0, iv1;
                    const int sp = m.sp_index[i];
                    if (sp < 0) {
                        iv0 = iv1 = invdiag_linT[i];
                    } else {
                        const auto ivv = ld2<T>(invd + (size_t)sp * NB + l0);
                        iv0 = ivv.x;
                        iv1 = ivv.y;
                    }
                    st2<T>(p + o, p0, p1);
                    st2<T>(s + o, s0, s1);
                    st2<T>(r + o, r0, r1);
                    st2<T>(z + o, r0 * iv0, r1 * iv1);
                    st2<T>(x + o, xi.x + al0 * p0, xi.y + al1 * p1);
                }
                if (!grid_sync(a.bar, a.status)) return;
            }
            // ---- u += x on own rows, then element data at the corrected state
            for (int i = row0; i < m.ndof; i += rstride) {
                const size_t o = (size_t)i * NB + l0;
                const auto xi = ld2<T>(x + o);
                const double2 ui = *reinterpret_cast<const double2*>(u + o);
                st2<double>(u + o, ui.x + (double)xi.x, ui.y + (double)xi.y);
            }
            if (!grid_sync(a.bar, a.status)) return;
            for (long long it = blockIdx.x * (long long)blockDim.x + tid; it < n_elem_items; it += gthreads)
                elem_compute(m, NB, u, a.elem, (int)(it / NB), (int)(it % NB));
            if (!grid_sync(a.bar, a.status)) return;
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        a.counters[0] += newton_total;
        a.counters[1] += pcg_total;
    }
}

size_t fine_smem(bool fp32, int NB, int threads) {
    const int RB = threads / (NB / 2);
    const size_t rt = fp32 ? sizeof(float) : sizeof(double);
    return (size_t)8 * NB * sizeof(double) + (size_t)(NV * RB * NB + NV * NB + threads) * rt + 2 * NB * sizeof(int);
}

}  // namespace

cudaError_t fine_config(bool fp32, int NB, LaunchCfg* cfg) {
    const int G = NB / 2;
    if (G < 1 || G > 512) return cudaErrorInvalidValue;
    const int threads = G * (1024 / G);
    const size_t smem = fine_smem(fp32, NB, threads);
    const void* fn = fp32 ? (const void*)fine_sweep_kernel<float> : (const void*)fine_sweep_kernel<double>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

void launch_elem_data(const MeshDev& m, int NB, const double* u, double* elem, cudaStream_t st) {
    const long long total = (long long)m.n_nl * NB;
    if (total == 0) return;
    long long b = (total + 255) / 256;
    if (b > 65535) b = 65535;
    elem_data_kernel<<<(int)b, 256, 0, st>>>(m, NB, u, elem);
}

}  // namespace pppc

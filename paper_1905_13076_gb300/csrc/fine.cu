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
// u += a p, r -= a s, z = D^-1 r.
//
// Layout: vectors are [ndof][NB] (lane fastest); a thread owns 2 adjacent
// lanes of fixed rows for the whole launch, so row-local data is only ever
// touched by its owner and loads of other rows' data go through L2.
#include <cuda_runtime.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace pppc {

// Element data of nonlinear element q, lane `lane`, from the state u:
//   grad A = sum_a u_a grad N_a,  b = |grad A|^2,
//   nu = k1 exp(k2 b) + k3,  dnu/db = k1 k2 exp(k2 b),
//   c1 = |e| nu,  c2 = 2 |e| dnu/db,  s_a = grad N_a . grad A.
__device__ __forceinline__ void elem_compute(const MeshDev& m, int NB, const double* u, double* elem,
                                             int q, int lane, bool coherent) {
    const int* dofs = m.nl_dofs + 3 * (size_t)q;
    const double* G = m.nl_geom + 8 * (size_t)q;
    const double* K = m.nl_k + 4 * (size_t)q;
    double ua[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int d = dofs[a];
        ua[a] = d < 0 ? 0.0 : (coherent ? __ldcg(u + (size_t)d * NB + lane) : u[(size_t)d * NB + lane]);
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
        elem_compute(m, NB, u, elem, (int)(it / NB), (int)(it % NB), false);
}

constexpr int NV = 3;  // reduced values per lane: (r,r), (r,z), (z,w)
constexpr double kPi = 3.141592653589793;
// Newton also stops when ||R|| no longer halves (kStagnation) while within
// kFloorMult of the tolerance: the residual has reached its rounding floor.
constexpr double kStagnation = 0.5;
constexpr double kFloorMult = 100.0;

// Fixed-order in-block sum over the row slots of each lane, written as this
// block's partials part[blockIdx.x][v][lane].
__device__ __forceinline__ void block_partials(double* s_red, int RB, int NB, int rb, int l0,
                                               const double (&v)[NV][2], double* part) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        s_red[(q * RB + rb) * NB + l0] = v[q][0];
        s_red[(q * RB + rb) * NB + l0 + 1] = v[q][1];
    }
    __syncthreads();
    double* out = part + (size_t)blockIdx.x * NV * NB;
    for (int o = threadIdx.x; o < NV * NB; o += blockDim.x) {
        const int q = o / NB, l = o - q * NB;
        double s = 0.0;
        for (int t = 0; t < RB; ++t) s += s_red[(q * RB + t) * NB + l];
        out[o] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(512) fine_sweep_kernel(const FineArgs a) {
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
    double* s_red = s_rprev + NB;  // [NV][RB][NB]
    int* s_newton = reinterpret_cast<int*>(s_red + NV * RB * NB);
    int* s_pcg = s_newton + NB;
    __shared__ int s_err;

    T* r = static_cast<T*>(a.r);
    T* z = static_cast<T*>(a.z);
    T* w = static_cast<T*>(a.w);
    T* p = static_cast<T*>(a.p);
    T* s = static_cast<T*>(a.s);
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
        // u_prev = u on own rows; element data at u
        for (int i = row0; i < m.ndof; i += rstride)
            st2<double>(uprev + (size_t)i * NB + l0, u[(size_t)i * NB + l0], u[(size_t)i * NB + l0 + 1]);
        for (long long it = blockIdx.x * (long long)blockDim.x + tid; it < n_elem_items; it += gthreads)
            elem_compute(m, NB, u, a.elem, (int)(it / NB), (int)(it % NB), true);
        if (!grid_sync(a.bar, a.status)) return;

        for (int nit = 0;; ++nit) {
            // ---- residual R(u), per-lane Jacobian of special rows, r = -R, z = D^-1 r
            double acc[NV][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
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
                        const double2 uj = ldcg2(u + (size_t)j * NB + l0);
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
                        const double2 uj = ldcg2(u + (size_t)j * NB + l0);
                        const double2 upj = ldcg2(uprev + (size_t)j * NB + l0);
                        const double kl = (j == i) ? 0.0 : kv;
                        a0 += kl * (uj.x - ui.x) + mv * (uj.x - upj.x);
                        a1 += kl * (uj.y - ui.y) + mv * (uj.y - upj.y);
                        double J0 = kv + mv, J1 = kv + mv;
                        for (int c = m.nlc_ptr[sl]; c < m.nlc_ptr[sl + 1]; ++c) {
                            const int pk = m.nlc[c];
                            const int q = pk / 9, ia = (pk / 3) % 3, ib = pk % 3;
                            const double ab = m.nlc_ab[c];
                            const size_t o = (size_t)q * NB + l0;
                            const double2 c1 = ldcg2(E + o);
                            const double2 c2 = ldcg2(E + P + o);
                            const double2 sa = ldcg2(E + (2 + ia) * P + o);
                            const double2 sb = ldcg2(E + (2 + ib) * P + o);
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
                st2<T>(r + (size_t)i * NB + l0, r0, r1);
                st2<T>(z + (size_t)i * NB + l0, z0, z1);
                acc[0][0] += R0 * R0;
                acc[0][1] += R1 * R1;
                acc[1][0] += (double)r0 * (double)z0;
                acc[1][1] += (double)r1 * (double)z1;
            }
            block_partials(s_red, RB, NB, rb, l0, acc, a.part);
            if (!grid_sync_reduce(a.bar, a.status, a.part, a.sums, NV * NB)) return;

            // ---- Newton test per lane; PCG tolerance per lane
            int act = 0;
            for (int l = tid; l < NB; l += blockDim.x) {
                int al = 0;
                if (s_newton[l]) {
                    const double rr = __ldcg(a.sums + l);
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
                        double eta = fmax(a.tol_lin, 0.1 * a.tol_abs / Rn);
                        eta = fmin(eta, 0.1);
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
                    rmax = fmax(rmax, sqrt(__ldcg(a.sums + l)));
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

            // ---- PCG on J du = -R (du accumulated directly into u)
            for (int k = 0;; ++k) {
                double acc2[NV][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
                for (int i = row0; i < m.ndof; i += rstride) {
                    const int kb = m.rowptr[i], ke = m.rowptr[i + 1];
                    const int slot0 = m.row_slot[i];
                    T w0 = 0, w1 = 0;
                    if (slot0 < 0) {
                        for (int kk = kb; kk < ke; ++kk) {
                            const T kv = KlinT[kk];
                            const auto zj = ldcg2(z + (size_t)m.col[kk] * NB + l0);
                            w0 += kv * zj.x;
                            w1 += kv * zj.y;
                        }
                    } else {
                        for (int kk = kb; kk < ke; ++kk) {
                            const auto jv = ld2<T>(J + (size_t)(slot0 + kk - kb) * NB + l0);
                            const auto zj = ldcg2(z + (size_t)m.col[kk] * NB + l0);
                            w0 += jv.x * zj.x;
                            w1 += jv.y * zj.y;
                        }
                    }
                    st2<T>(w + (size_t)i * NB + l0, w0, w1);
                    const auto ri = ld2<T>(r + (size_t)i * NB + l0);
                    const auto zi = ld2<T>(z + (size_t)i * NB + l0);
                    acc2[0][0] += (double)ri.x * ri.x;
                    acc2[0][1] += (double)ri.y * ri.y;
                    acc2[1][0] += (double)ri.x * zi.x;
                    acc2[1][1] += (double)ri.y * zi.y;
                    acc2[2][0] += (double)zi.x * w0;
                    acc2[2][1] += (double)zi.y * w1;
                }
                block_partials(s_red, RB, NB, rb, l0, acc2, a.part);
                if (!grid_sync_reduce(a.bar, a.status, a.part, a.sums, NV * NB)) return;

                int act2 = 0;
                for (int l = tid; l < NB; l += blockDim.x) {
                    double al = 0.0, be = 0.0;
                    int on = 0;
                    if (s_pcg[l]) {
                        const double rho = __ldcg(a.sums + l);
                        const double gam = __ldcg(a.sums + NB + l);
                        const double del = __ldcg(a.sums + 2 * NB + l);
                        if (!isfinite(rho) || !isfinite(gam) || !isfinite(del)) {
                            set_status(a.status, DEV_ERR_NAN);
                            s_err = 1;
                        } else if (rho <= s_stop[l]) {
                            s_pcg[l] = 0;
                        } else if (k >= a.max_lin) {
                            set_status(a.status, DEV_ERR_LINEAR);
                            s_err = 1;
                        } else {
                            be = (k == 0) ? 0.0 : gam / s_gold[l];
                            const double den = (k == 0) ? del : del - be * gam / s_aold[l];
                            if (!(den > 0.0) || !(gam > 0.0)) {
                                set_status(a.status, DEV_ERR_BREAKDOWN);
                                s_err = 1;
                            } else {
                                al = gam / den;
                                s_gold[l] = gam;
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

                const double al0 = s_alpha[l0], al1 = s_alpha[l0 + 1];
                const double be0 = s_beta[l0], be1 = s_beta[l0 + 1];
                for (int i = row0; i < m.ndof; i += rstride) {
                    const size_t o = (size_t)i * NB + l0;
                    const auto zi = ld2<T>(z + o);
                    const auto wi = ld2<T>(w + o);
                    const auto pi = ld2<T>(p + o);
                    const auto si = ld2<T>(s + o);
                    const auto ri = ld2<T>(r + o);
                    const T p0 = zi.x + (T)be0 * pi.x, p1 = zi.y + (T)be1 * pi.y;
                    const T s0 = wi.x + (T)be0 * si.x, s1 = wi.y + (T)be1 * si.y;
                    const T r0 = ri.x - (T)al0 * s0, r1 = ri.y - (T)al1 * s1;
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
                    const double2 ui = *reinterpret_cast<const double2*>(u + o);
                    st2<double>(u + o, ui.x + al0 * (double)p0, ui.y + al1 * (double)p1);
                }
                if (!grid_sync(a.bar, a.status)) return;
            }
            // element data at the corrected state
            for (long long it = blockIdx.x * (long long)blockDim.x + tid; it < n_elem_items; it += gthreads)
                elem_compute(m, NB, u, a.elem, (int)(it / NB), (int)(it % NB), true);
            if (!grid_sync(a.bar, a.status)) return;
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        a.counters[0] += newton_total;
        a.counters[1] += pcg_total;
    }
}

size_t fine_smem(int NB, int threads) {
    const int RB = threads / (NB / 2);
    return (size_t)(7 * NB + NV * RB * NB) * sizeof(double) + 2 * NB * sizeof(int);
}

}  // namespace

cudaError_t fine_config(bool fp32, int NB, LaunchCfg* cfg) {
    const int G = NB / 2;
    if (G < 1 || G > 512) return cudaErrorInvalidValue;
    const int threads = G * (512 / G);
    const size_t smem = fine_smem(NB, threads);
    const void* fn = fp32 ? (const void*)fine_sweep_kernel<float> : (const void*)fine_sweep_kernel<double>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cfg->blocks = sms * per_sm;
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

// Periodic adjoint of the period-averaged eddy-current loss (pppc_adjoint).
//
// The adjoint recurrence
//     (M/dt + J_m) lam_m = (M/dt) lam_{m+1} + g_m,   cyclic in m,
// runs backwards in time.  With the coarse points Lam_n = lam at the first
// level of subinterval n+1, the fine propagator of subinterval n maps
// Lam_{n+1} to Lam_n, and PP-PC with the multi-harmonic coarse solve applies
// unchanged once the lane order is reversed: in A'[j] = Lam_{(N-j) mod N} the
// backward cyclic system is the forward one, Q W_j - C W_{j-1} = C d_{j-1},
// so jumps, the DFT right-hand side, the batched COCG and the inverse DFT +
// update are the forward kernels.  The fine sweep works in natural lane
// order (lane s runs subinterval s backwards over the forward trajectory of
// lane s), so its input is rev(A') and its result is reversed back.
//
// Gradient (after convergence, from the last sweep's lambda at every level):
//   dP/dsigma_r = P_r / sigma_r - sum_m lam_m^T (M_r / sigma_r) du^m / dt
//   dP/dk_i     = - sum_m lam_m^T d(K(u^m) u^m) / dk_i
// summed over the nonlinear elements of region r, all lanes and levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/pppc.h"
#include "args.h"
#include "handle.h"
#include "kernels.h"

using namespace pppc;
using namespace pppc::detail;

namespace {

constexpr int kGradBlocks = 512;
constexpr int kGradValues = 6;   // P_all, P_r, S_sigma, G_k1, G_k2, G_k3

__global__ void lanes_reverse_kernel(int ndof, int N, int NB, const double* in, double* out) {
    const long long total = (long long)ndof * NB;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(it % NB);
        const long long i = it / NB;
        out[it] = l < N ? in[i * NB + (N - 1 - l)] : 0.0;
    }
}

struct GradArgs {
    MeshDev m;
    int N, NB, nf;
    double dt, T, sigma_r;
    const double* traj;          // [nf+1][ndof][NB] forward levels
    const double* lam;           // [nf][ndof][NB] lambda at levels 1..nf
    const unsigned char* sel;    // [n_nl] 1: element of region r
    double* part;                // [gridDim][kGradValues]
};

__device__ __forceinline__ double node(const double* lvl, int d, int NB, int s) {
    return d < 0 ? 0.0 : lvl[(size_t)d * NB + s];
}

__global__ void adjoint_grad_kernel(const GradArgs g) {
    const MeshDev& m = g.m;
    const size_t lv = (size_t)m.ndof * g.NB;
    double acc[kGradValues] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    // region r's nonlinear elements x lanes x levels
    const long long ne = (long long)m.n_nl * g.nf * g.N;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < ne; it += stride) {
        const int s = (int)(it % g.N);
        const long long rest = it / g.N;
        const int j = 1 + (int)(rest % g.nf);
        const int q = (int)(rest / g.nf);
        if (!g.sel[q]) continue;
        const int* dofs = m.nl_dofs + 3 * (size_t)q;
        const double* G = m.nl_geom + 8 * (size_t)q;
        const double* K = m.nl_k + 4 * (size_t)q;
        const double* u1 = g.traj + (size_t)j * lv;
        const double* u0 = u1 - lv;
        const double* la = g.lam + (size_t)(j - 1) * lv;
        double ua[3], du[3], lm[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ua[a] = node(u1, dofs[a], g.NB, s);
            du[a] = ua[a] - node(u0, dofs[a], g.NB, s);
            lm[a] = node(la, dofs[a], g.NB, s);
        }
        // grad A and grad lambda from vertex differences (grad N_0 = -grad N_1 - grad N_2)
        const double gx = (ua[1] - ua[0]) * G[3] + (ua[2] - ua[0]) * G[5];
        const double gy = (ua[1] - ua[0]) * G[4] + (ua[2] - ua[0]) * G[6];
        const double lx = (lm[1] - lm[0]) * G[3] + (lm[2] - lm[0]) * G[5];
        const double ly = (lm[1] - lm[0]) * G[4] + (lm[2] - lm[0]) * G[6];
        const double b = gx * gx + gy * gy;
        const double bc = fmin(b, K[3]);
        const double over = b - bc;
        const double ex = exp(K[1] * bc);
        const double w = G[0] * (lx * gx + ly * gy);
        acc[3] += ex * (1.0 + K[1] * over) * w;                                   // dnu/dk1
        acc[4] += K[0] * ex * (bc * (1.0 + K[1] * over) + over) * w;             // dnu/dk2
        acc[5] += w;                                                              // dnu/dk3
        // consistent mass of the element / sigma: |e| (1 + delta_ab) / 12
        const double sl = lm[0] + lm[1] + lm[2], sd = du[0] + du[1] + du[2];
        const double sld = lm[0] * du[0] + lm[1] * du[1] + lm[2] * du[2];
        const double sdd = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
        acc[2] += G[0] / 12.0 * (sld + sl * sd) / g.dt;
        acc[1] += g.sigma_r * G[0] / 12.0 * (sdd + sd * sd) / (g.T * g.dt);
    }
    // all conducting rows: P = (1/T) sum_m du^T M du / dt
    const long long nr = (long long)m.n_sp * g.nf * g.N;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < nr; it += stride) {
        const int s = (int)(it % g.N);
        const long long rest = it / g.N;
        const int j = 1 + (int)(rest % g.nf);
        const int sp = (int)(rest / g.nf);
        const int i = m.sp_rows[sp];
        const double* u1 = g.traj + (size_t)j * lv;
        const double* u0 = u1 - lv;
        const int kb = m.rowptr[i], ke = m.rowptr[i + 1], slot0 = m.row_slot[i];
        double mdu = 0.0;
        for (int k = kb; k < ke; ++k) {
            const size_t oc = (size_t)m.col[k] * g.NB + s;
            mdu += m.Mslot[slot0 + (k - kb)] * (u1[oc] - u0[oc]);
        }
        const size_t oi = (size_t)i * g.NB + s;
        acc[0] += (u1[oi] - u0[oi]) * mdu / (g.T * g.dt);
    }
    __shared__ double red[kGradValues][256];
#pragma unroll
    for (int v = 0; v < kGradValues; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int v = 0; v < kGradValues; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < kGradValues) g.part[(size_t)blockIdx.x * kGradValues + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void grad_sum_kernel(int nblocks, const double* part, double* out) {
    if (threadIdx.x < kGradValues) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * kGradValues + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

int grid_of(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::max(1LL, std::min(b, 65535LL));
}

pppc_status take(pppc_handle* h, double** p, size_t n) {
    void* ptr = nullptr;
    if (h->cfg.alloc) {
        ptr = h->cfg.alloc(n * sizeof(double), h->cfg.alloc_ctx);
    } else if (cudaMalloc(&ptr, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (!ptr) return fail(h, PPPC_ERR_NOMEM, "adjoint workspace allocation failed");
    h->allocs.push_back(ptr);
    *p = static_cast<double*>(ptr);
    return PPPC_OK;
}

pppc_status run_sweep(pppc_handle* h, const FineArgs& a, const char* where) {
    TRY(stage_reset(h));
    CK(cudaEventRecord(h->ev[0], h->st));
    CK(launch_fine_sweep(a, h->fp32, h->fine_cfg, h->st));
    h->stats.launches += 1;
    CK(cudaEventRecord(h->ev[1], h->st));
    TRY(device_status(h, where));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
    h->stats.fine_ms += ms;
    return PPPC_OK;
}

}  // namespace

extern "C" pppc_status pppc_adjoint(pppc_handle* h, int32_t region, double tol, int32_t kmax,
                                    pppc_adjoint_result* out) {
    if (!h) return PPPC_ERR_INVALID_ARG;
    TRY(stage_ready(h));
    if (!out || !(tol > 0.0) || kmax < 0) return fail(h, PPPC_ERR_INVALID_ARG, "out NULL, tol <= 0 or kmax < 0");
    if (h->cfg.method != PPPC_METHOD_PPPC) return fail(h, PPPC_ERR_UNSUPPORTED, "pppc_adjoint: PP-PC handles only");
    if (region < 0 || region >= (int)h->region_kind.size() || !(h->region_kind[region] & ELEM_NONLINEAR) ||
        !(h->region_sigma[region] > 0.0))
        return fail(h, PPPC_ERR_INVALID_ARG, "region must be nonlinear (Brauer) and conducting");
    const HostMesh& hm = h->hm;
    const int ndof = hm.ndof, N = h->N, NB = h->NB, nf = h->cfg.n_fine;
    const size_t LV = (size_t)ndof * NB;
    if (!h->traj) {
        TRY(take(h, &h->traj, (size_t)(nf + 1) * LV));
        TRY(take(h, &h->lam, (size_t)nf * LV));
        TRY(take(h, &h->adjA, LV));
        TRY(take(h, &h->adjB, LV));
        TRY(take(h, &h->adjF, LV));
        TRY(take(h, &h->gpart, (size_t)kGradBlocks * kGradValues));
        TRY(take(h, &h->gout, kGradValues));
        double* sel = nullptr;
        TRY(take(h, &sel, (std::max(hm.n_nl, 1) + 7) / 8));
        h->nl_sel = reinterpret_cast<unsigned char*>(sel);
    }
    std::vector<unsigned char> sel(std::max(hm.n_nl, 1), 0);
    for (int q = 0; q < hm.n_nl; ++q) sel[q] = h->nl_region[q] == region;
    CK(cudaMemcpyAsync(h->nl_sel, sel.data(), sel.size(), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(h->counters, 0, kCounters * sizeof(long long), h->st));
    h->stats = pppc_stats{};

    // ---- forward trajectory of the handle's state (levels 0..nf of every lane)
    CK(cudaMemcpyAsync(h->F, h->U, LV * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    FineArgs fa = fine_args(h, h->F);
    fa.traj_out = h->traj;
    TRY(run_sweep(h, fa, "forward trajectory"));
    double fwd_rr = 0.0;
    TRY(stage_jumps(h, h->U, h->F, &fwd_rr));
    out->forward_rel_res = fwd_rr;
    if (!(fwd_rr <= 1e-6))
        return fail(h, PPPC_ERR_STATE, "pppc_adjoint: the state is not periodic (rel_res " + std::to_string(fwd_rr) +
                                           "); solve it first");

    // ---- Kbar of the forward state, fixed for the whole adjoint solve
    TRY(stage_kbar(h, h->U));

    // ---- adjoint PP-PC in reversed lane order
    FineArgs aa = fine_args(h, h->adjB);
    aa.adjoint = 1;
    aa.traj = h->traj;
    aa.lam_out = h->lam;
    aa.predictor = 0;
    aa.tol_rel = h->cfg.tol_newton;
    aa.g_scale = 2.0 / (h->cfg.T * h->dt);
    CK(cudaMemsetAsync(h->adjA, 0, LV * sizeof(double), h->st));
    const int gb = grid_of((long long)LV);
    double rr = INFINITY;
    int k = 0;
    for (;; ++k) {
        lanes_reverse_kernel<<<gb, 256, 0, h->st>>>(ndof, N, NB, h->adjA, h->adjB);
        CK(cudaGetLastError());
        TRY(run_sweep(h, aa, "adjoint propagators"));
        lanes_reverse_kernel<<<gb, 256, 0, h->st>>>(ndof, N, NB, h->adjB, h->adjF);
        h->stats.launches += 2;
        TRY(stage_jumps(h, h->adjA, h->adjF, &rr));
        if (rr <= tol || k >= kmax) break;
        TRY(stage_correct(h, h->adjF, h->adjB));
        std::swap(h->adjA, h->adjB);
        aa.u = h->adjB;
    }
    out->iterations = k;
    out->rel_res = rr;

    // ---- loss and gradient from the last sweep's lambda levels
    GradArgs g{};
    g.m = h->md;
    g.N = N;
    g.NB = NB;
    g.nf = nf;
    g.dt = h->dt;
    g.T = h->cfg.T;
    g.sigma_r = h->region_sigma[region];
    g.traj = h->traj;
    g.lam = h->lam;
    g.sel = h->nl_sel;
    g.part = h->gpart;
    adjoint_grad_kernel<<<kGradBlocks, 256, 0, h->st>>>(g);
    grad_sum_kernel<<<1, 32, 0, h->st>>>(kGradBlocks, h->gpart, h->gout);
    h->stats.launches += 2;
    CK(cudaGetLastError());
    double v[kGradValues];
    CK(cudaMemcpyAsync(v, h->gout, sizeof v, cudaMemcpyDeviceToHost, h->st));
    long long c[kCounters];
    CK(cudaMemcpyAsync(c, h->counters, sizeof c, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->stats.newton_iters = c[kCntNewton];
    h->stats.pcg_iters = c[kCntPcg];
    h->stats.cocg_iters = c[kCntCocg];
    h->stats.backtracks = c[kCntBacktrack];
    h->stats.pcg_lane_rounds = c[kCntPcgLaneRounds];
    h->stats.pcg_lane_iters = c[kCntPcgLaneIters];
    h->stats.newton_lane_rounds = c[kCntNewtonLaneRounds];
    h->stats.pppc_iters = k;
    h->stats.rel_res = rr;
    const double s = h->region_sigma[region];
    out->loss = v[0];
    out->grad[0] = v[1] / s - v[2];
    out->grad[1] = -v[3];
    out->grad[2] = -v[4];
    out->grad[3] = -v[5];
    if (!(rr <= tol))
        return fail(h, PPPC_ERR_NOT_CONVERGED, "adjoint rel_res " + std::to_string(rr) + " > tol after " +
                                                   std::to_string(kmax) + " updates");
    return PPPC_OK;
}

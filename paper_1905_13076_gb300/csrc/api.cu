// C ABI of the library (include/pppc.h): handle, mesh upload, and the PP-PC
// driver that sequences the kernels of one iteration (Sec. 2, Eq. 4; Sec. 3).
// There is no CPU fallback: every floating-point step of the method runs in
// the kernels of setup.cu, fine.cu and coarse.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pppc.h"
#include "amg_host.h"
#include "args.h"
#include "handle.h"
#include "kernels.h"
#include "mesh_host.h"

using namespace pppc;
using namespace pppc::detail;

namespace {
thread_local std::string g_create_error;
// Smallest relative residual asked of an FP32 PCG/COCG solve (mixed precision):
// with the Jacobian rounded to FP32 a solve cannot contract the FP64 Newton
// residual by much more than ~1e-3, so tighter solves only burn iterations.
constexpr double kFp32KrylovFloor = 1e-4;
// Inexact PP-PC schedule: Newton tolerance min(kNewtonLoose, kNewtonFactor *
// rel_res of the previous iterate), never below pppc_config.tol_newton.
constexpr double kNewtonLoose = 1e-6;
// Rows per tridiagonal chunk of the fine PCG preconditioner (pppc_config.precond
// = 1); the kernel's chunk solve is specialised for it (kTri in fine.cu).
constexpr int kTriChunk = 4;
constexpr double kNewtonFactor = 1e-3;
// l1-Jacobi sweeps on the coarsest multigrid level
constexpr int kAmgCoarsestSweeps = 2;
}


namespace {

const char* kStatusNames[] = {"PPPC_OK",
                              "PPPC_ERR_INVALID_ARG",
                              "PPPC_ERR_CUDA",
                              "PPPC_ERR_STATE",
                              "PPPC_ERR_NEWTON",
                              "PPPC_ERR_LINEAR",
                              "PPPC_ERR_BREAKDOWN",
                              "PPPC_ERR_NAN",
                              "PPPC_ERR_TIMEOUT",
                              "PPPC_ERR_NOT_CONVERGED",
                              "PPPC_ERR_UNSUPPORTED",
                              "PPPC_ERR_NOMEM"};

}  // namespace

pppc_status pppc::detail::fail(pppc_handle* h, pppc_status s, const std::string& msg) {
    h->err = msg;
    return s;
}

namespace {

void* dev_alloc(pppc_handle* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* ptr = nullptr;
    if (h->cfg.alloc) {
        ptr = h->cfg.alloc(bytes, h->cfg.alloc_ctx);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) h->allocs.push_back(ptr);
    return ptr;
}

void free_all(pppc_handle* h) {
    if (h->st) cudaStreamSynchronize(h->st);
    if (h->gst) cudaStreamSynchronize(h->gst);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->graph_dirty = true;
    h->d_ctl_in = nullptr;   // freed with the other workspace below
    h->d_ctl = nullptr;
    h->d_graph_args = nullptr;
    h->d_graph_map = nullptr;
    for (void* ptr : h->allocs) {
        if (h->cfg.free_fn)
            h->cfg.free_fn(ptr, h->cfg.alloc_ctx);
        else
            cudaFree(ptr);
    }
    h->allocs.clear();
    h->row_tables.clear();
    h->plan = pppc_fine_plan{};
    h->has_mesh = false;
}

template <typename T>
pppc_status alloc_n(pppc_handle* h, T** out, size_t n) {
    *out = static_cast<T*>(dev_alloc(h, n * sizeof(T)));
    if (!*out) return fail(h, PPPC_ERR_NOMEM, "device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed");
    return PPPC_OK;
}

template <typename T>
pppc_status upload(pppc_handle* h, T** out, const std::vector<T>& v) {
    TRY(alloc_n(h, out, v.size()));
    if (!v.empty()) CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->st));
    return PPPC_OK;
}

}  // namespace

pppc_status pppc::detail::device_status(pppc_handle* h, const char* where) {
    CK(cudaStreamSynchronize(h->st));
    int code = 0;
    CK(cudaMemcpy(&code, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (code == 0) return PPPC_OK;
    std::string w(where);
    switch (code) {
        case DEV_ERR_NEWTON: return fail(h, PPPC_ERR_NEWTON, w + ": Newton iteration cap reached");
        case DEV_ERR_LINEAR: return fail(h, PPPC_ERR_LINEAR, w + ": linear-solver iteration cap reached");
        case DEV_ERR_BREAKDOWN: return fail(h, PPPC_ERR_BREAKDOWN, w + ": Krylov breakdown");
        case DEV_ERR_NAN: return fail(h, PPPC_ERR_NAN, w + ": non-finite residual");
        case DEV_ERR_TIMEOUT: return fail(h, PPPC_ERR_TIMEOUT, w + ": grid barrier timed out");
        case DEV_ERR_GEOMETRY: return fail(h, PPPC_ERR_INVALID_ARG, w + ": zero-area or non-finite triangle");
        default: return fail(h, PPPC_ERR_CUDA, w + ": unknown device status " + std::to_string(code));
    }
}

namespace {

pppc_status reset_control(pppc_handle* h) {
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
    CK(cudaMemsetAsync(h->bar, 0, kMaxTeams * sizeof(GridBarrier), h->st));
    CK(reset_team_ctl(h, h->st));
    return PPPC_OK;
}

pppc_status need_ready(pppc_handle* h) {
    if (!h) return PPPC_ERR_INVALID_ARG;
    if (!h->has_mesh) return fail(h, PPPC_ERR_STATE, "pppc_set_mesh has not been called");
    if (!h->has_source) return fail(h, PPPC_ERR_STATE, "pppc_set_source has not been called");
    return PPPC_OK;
}

// ---- lane teams of the fine sweep ------------------------------------------
//
// The N lanes (subintervals) of a sweep are independent: they share only the
// mesh.  A plan splits them into teams of `lanes` lanes; each team runs the
// whole sweep on its own share of the SMs, with its own grid barrier and
// reductions and its own [row][lanes] PCG vectors, and never waits for
// another team.  Fewer lanes per team means fewer rows' worth of blocks per
// barrier, a smaller SpMV gather window (lanes x 4 bytes per row) and less
// lockstep (a team stops when its own lanes have converged); more lanes per
// team means wider rows per thread group and more blocks per reduction.
// Which wins depends on the mesh and N, so the choice is measured.

// Fine levels each candidate marches when the plan is tuned.
constexpr int kTuneLevels = 1;
constexpr int kMaxCandidates = 16;

// Lanes per team chosen by the tuner, by size bucket: precision, padded
// lanes, preconditioner and floor(log2(ndof)).  Shared by every handle of
// the process, so a bucket is timed once.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tuned;

std::tuple<int, int, int, int, int> tune_key(const pppc_handle* h) {
    int lg = 0;
    while ((2LL << lg) <= h->hm.ndof) ++lg;
    return {h->fp32 ? 1 : 0, h->NB, h->cfg.precond, lg, h->sms};
}

// Lanes per team that a plan may use: V 2^i (V = 4 FP32 / 2 FP64 lanes per
// thread) dividing NB, with at most one team per SM.
std::vector<int> team_candidates(const pppc_handle* h) {
    const int V = h->fp32 ? 4 : 2;
    std::vector<int> c;
    for (int lanes = V; lanes <= h->NB && (int)c.size() < kMaxCandidates; lanes *= 2)
        if (h->NB % lanes == 0 && h->NB / lanes <= std::min(h->sms, kMaxTeams)) c.push_back(lanes);
    return c;
}

}  // namespace

pppc_status pppc::detail::row_tables_for(pppc_handle* h, int blocks, const pppc_row_tables** out) {
    auto it = h->row_tables.find(blocks);
    if (it == h->row_tables.end()) {
        std::vector<int> rs, ls, lr;
        pppc_row_tables t;
        partition_rows(h->hm, blocks, rs, ls, lr, &t.rows_max);
        TRY(upload(h, &t.rs, rs));
        TRY(upload(h, &t.ls, ls));
        TRY(upload(h, &t.lr, lr));
        it = h->row_tables.emplace(blocks, t).first;
    }
    *out = &it->second;
    return PPPC_OK;
}

namespace {

// Teams of `lanes` lanes, the SMs split as evenly as the team count allows.
pppc_status make_plan(pppc_handle* h, int lanes, pppc_fine_plan* p) {
    pppc_fine_plan q;
    q.lanes = lanes;
    q.teams = h->NB / lanes;
    q.blocks.assign(q.teams, h->sms / q.teams);
    for (int t = 0; t < h->sms % q.teams; ++t) ++q.blocks[t];
    const size_t budget = h->smem_optin - h->fine_static_smem - 1024;
    for (int t = 0; t < q.teams; ++t) {
        const pppc_row_tables* rt = nullptr;
        TRY(row_tables_for(h, q.blocks[t], &rt));
        int vr = 0, vw = 0;
        choose_vec_rows(h->fp32, lanes, rt->rows_max, budget, &vr, &vw);
        q.smem = std::max(q.smem, fine_smem(h->fp32, lanes, 1024, vr, vw ? 4 : 3));
    }
    *p = q;
    return PPPC_OK;
}

// The sweep `base` (one team over all lanes) as the teams of plan p, and
// the block -> (team, block in team, team size) map.
void team_tables(pppc_handle* h, const pppc_fine_plan& p, const FineArgs& base, std::vector<FineArgs>& args,
                 std::vector<int4>& map) {
    args.assign(p.teams, FineArgs{});
    map.assign(h->sms, make_int4(-1, 0, 0, 0));
    size_t part_off = 0;
    int first = 0;
    for (int t = 0; t < p.teams; ++t) {
        const int nb = p.blocks[t];
        args[t] = team_args(h, p.lanes, t, p.teams, nb, base, &part_off);
        for (int k = 0; k < nb; ++k) map[first + k] = make_int4(t, k, nb, 0);
        first += nb;
    }
}

// Launch the sweep `base` as the teams of plan p.
pppc_status launch_plan(pppc_handle* h, const pppc_fine_plan& p, const FineArgs& base) {
    std::vector<FineArgs> args;
    std::vector<int4> map;
    team_tables(h, p, base, args, map);
    CK(cudaMemcpyAsync(h->d_team_args, args.data(), args.size() * sizeof(FineArgs), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->d_team_map, map.data(), map.size() * sizeof(int4), cudaMemcpyHostToDevice, h->st));
    CK(launch_fine_batch(h->d_team_args, h->d_team_map, h->fp32, h->sms, p.smem, h->st));
    h->stats.launches += 1;
    return PPPC_OK;
}

// The plan of h: fixed by cfg.lane_team, or (lane_team = 0) the bucket's
// tuned choice, timing every candidate on the first kTuneLevels levels of
// this sweep (from Uin, into Fout) when the bucket has none yet.
pppc_status choose_plan(pppc_handle* h, const double* Uin, double* Fout) {
    if (h->plan.lanes != 0) return PPPC_OK;
    const std::vector<int> cand = team_candidates(h);
    int lanes = -1;
    if (h->cfg.lane_team > 0) {
        lanes = h->cfg.lane_team;
    } else if (h->cfg.lane_team == 0 && !cand.empty()) {
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tuned.find(tune_key(h));
            if (it != g_tuned.end()) lanes = it->second;
        }
        if (lanes < 0) {
            const size_t lane_bytes = (size_t)h->hm.ndof * h->NB * sizeof(double);
            double best = INFINITY;
            for (size_t c = 0; c < cand.size(); ++c) {
                pppc_fine_plan q;
                TRY(make_plan(h, cand[c], &q));
                CK(cudaMemcpyAsync(Fout, Uin, lane_bytes, cudaMemcpyDeviceToDevice, h->st));
                TRY(reset_control(h));
                FineArgs a = fine_args(h, Fout);
                a.n_fine = std::min(kTuneLevels, h->cfg.n_fine);
                CK(cudaEventRecord(h->ev[0], h->st));
                TRY(launch_plan(h, q, a));
                CK(cudaEventRecord(h->ev[1], h->st));
                TRY(device_status(h, "fine-sweep tuning"));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
                h->tune_ms[c] = ms;
                if (ms < best) {
                    best = ms;
                    lanes = cand[c];
                }
            }
            // the tuning windows are not part of the call's work
            CK(cudaMemsetAsync(h->counters, 0, kCounters * sizeof(long long), h->st));
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tuned[tune_key(h)] = lanes;
        }
    }
    if (lanes > 0) {
        TRY(make_plan(h, lanes, &h->plan));
    } else {
        h->plan = pppc_fine_plan{};
        h->plan.lanes = -1;   // one team over all lanes, the grid-wide kernel
        h->plan.teams = 1;
    }
    return PPPC_OK;
}

}  // namespace

pppc_status pppc::detail::sweep_lanes(pppc_handle* h, int* lanes) {
    TRY(choose_plan(h, h->U, h->F));
    *lanes = h->plan.lanes > 0 ? h->plan.lanes : h->NB;
    return PPPC_OK;
}

namespace {

// ---- stages of one iteration ----------------------------------------------

// F = fine sweep of the lanes in Uin (F may not alias Uin): all n_fine
// levels, or the window of `count` levels from level `first`.
pppc_status run_fine(pppc_handle* h, const double* Uin, double* Fout, int first = 0, int count = -1) {
    const size_t lane_bytes = (size_t)h->hm.ndof * h->NB * sizeof(double);
    TRY(choose_plan(h, Uin, Fout));
    CK(cudaMemcpyAsync(Fout, Uin, lane_bytes, cudaMemcpyDeviceToDevice, h->st));
    TRY(reset_control(h));
    FineArgs a = fine_args(h, Fout);
    if (count >= 0) {
        a.level0 = first;
        a.n_fine = count;
    }
    const bool one_team = h->plan.lanes < 0 || h->trace_cap > 0;   // the trace records one team's lanes
    if (h->trace_cap > 0) {
        CK(cudaMemsetAsync(h->trace_len, 0, sizeof(int), h->st));
        a.trace = h->trace;
        a.trace_cap = h->trace_cap;
        a.trace_len = h->trace_len;
    }
    CK(cudaEventRecord(h->ev[0], h->st));
    if (one_team) {
        CK(launch_fine_sweep(a, h->fp32, h->fine_cfg, h->st));
        h->stats.launches += 1;
    } else {
        TRY(launch_plan(h, h->plan, a));
    }
    CK(cudaEventRecord(h->ev[1], h->st));
    TRY(device_status(h, "fine propagators"));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
    h->stats.fine_ms += ms;
    return PPPC_OK;
}

}  // namespace

cudaError_t pppc::detail::reset_team_ctl(pppc_handle* h, cudaStream_t st) {
    return cudaMemsetAsync(h->team_ctl, 0, 4 * sizeof(long long), st);
}

FineArgs pppc::detail::fine_args(pppc_handle* h, double* Fout) {
    FineArgs a{};
    a.mesh = h->md;
    a.src = h->src;
    a.N = h->N;
    a.NB = h->NB;
    a.ld = h->NB;
    a.lane0 = 0;
    a.n_teams = 1;
    a.sweep_max = h->team_ctl;
    a.teams_done = reinterpret_cast<unsigned int*>(h->team_ctl + 2);
    a.n_fine = h->cfg.n_fine;
    a.level0 = 0;
    a.n_total = h->cfg.n_fine;
    a.dt = h->dt;
    a.inv_dt = 1.0 / h->dt;
    // inexact PP-PC: looser Newton while the jumps are large (pppc_config.newton_schedule)
    const double tol_newton = h->cfg.newton_schedule && std::isfinite(h->rr_prev)
                                  ? std::max(h->cfg.tol_newton, std::min(kNewtonLoose, kNewtonFactor * h->rr_prev))
                                  : (h->cfg.newton_schedule ? std::max(h->cfg.tol_newton, kNewtonLoose) : h->cfg.tol_newton);
    a.tol_abs = tol_newton * h->gnorm * [&] {
        double s = 0.0;
        for (int j = 0; j < h->src.n_harm; ++j) s += std::fabs(h->src.amp[j]);
        return s;
    }();
    a.tol_lin = h->fp32 ? std::max(h->cfg.tol_lin, kFp32KrylovFloor) : h->cfg.tol_lin;
    a.eta0 = std::max(h->cfg.eta0, a.tol_lin);
    a.predictor = h->cfg.predictor;
    a.x = h->x;
    a.dx = h->dx;
    a.uprev2 = h->uprev2;
    if (h->cfg.precond == 1) {
        a.tri = kTriChunk;
        a.tri_low = h->d_tri_low;
        a.tri_m = h->tri_m;
        a.tri_ie = h->tri_ie;
    }
    if (h->amg_levels > 1) {
        a.amg = h->d_amg;
        a.amg_levels = h->amg_levels;
        a.amg_sweeps = kAmgCoarsestSweeps;
        a.amg_ws = h->amg_ws;
    }
    a.max_newton = h->cfg.max_newton;
    a.max_lin = h->cfg.max_lin;
    a.u = Fout;
    a.uprev = h->uprev;
    a.elem = h->elem;
    a.r = h->r;
    a.z = h->z;
    a.w = h->w;
    a.p = h->p;
    a.s = h->s;
    a.J = h->J;
    a.invd_sp = h->invd;
    a.part = h->part;
    a.row_start = h->d_row_start;
    a.long_start = h->d_long_start;
    a.long_rows = h->d_long_rows;
    a.vec_rows = h->vec_rows;
    a.vec_w = h->vec_w;
    a.bar = h->bar;
    a.status = h->status;
    a.counters = h->counters;
    return a;
}

CocgArgs pppc::detail::cocg_args(pppc_handle* h) {
    CocgArgs c{};
    c.mesh = h->md;
    c.N = h->N;
    c.H = h->H;
    c.inv_dT = 1.0 / h->dT;
    // FP32 Krylov recurrences cannot resolve FP64-level tolerances; an inexact
    // coarse solve only slows PP-PC (its fixed point does not depend on it).
    c.tol = h->coarse_fp32 ? std::max(h->cfg.tol_coarse, kFp32KrylovFloor) : h->cfg.tol_coarse;
    c.max_it = h->cfg.max_coarse;
    c.Kbar = h->Kbar;
    c.tw = h->tw;
    c.b = h->b;
    c.x = h->cx;
    c.r = h->cr;
    c.z = h->cz;
    c.w = h->cw;
    c.p = h->cp;
    c.s = h->cs;
    c.invd_sp = h->cinvd;
    c.part = h->part;
    c.bar = h->bar;
    c.status = h->status;
    c.counters = h->counters;
    return c;
}

void pppc::detail::partition_rows(const HostMesh& hm, int nb, std::vector<int>& rs, std::vector<int>& ls,
                                  std::vector<int>& lrows, int* rows_max) {
    std::vector<double> cum(hm.ndof + 1, 0.0);
    for (int i = 0; i < hm.ndof; ++i) {
        const int nz = hm.rowptr[i + 1] - hm.rowptr[i];
        cum[i + 1] = cum[i] + 2.0 + nz * (hm.row_slot[i] >= 0 ? 2.0 : 1.0) + (nz > 32 ? 400.0 : 0.0);
    }
    rs.assign(nb + 1, hm.ndof);
    rs[0] = 0;
    int i = 0;
    for (int b = 1; b < nb; ++b) {
        const double target = cum[hm.ndof] * b / nb;
        while (i < hm.ndof && cum[i] < target) ++i;
        rs[b] = i;
    }
    *rows_max = 0;
    for (int b = 0; b < nb; ++b) *rows_max = std::max(*rows_max, rs[b + 1] - rs[b]);
    ls.assign(nb + 1, 0);
    lrows.clear();
    for (int b = 0; b < nb; ++b) {
        for (int r = rs[b]; r < rs[b + 1]; ++r)
            if (hm.rowptr[r + 1] - hm.rowptr[r] > 32) lrows.push_back(r);
        ls[b + 1] = (int)lrows.size();
    }
}

double pppc::detail::fine_cost_estimate(const pppc_handle* h) {
    const HostMesh& hm = h->hm;
    double c = 0.0;
    for (int i = 0; i < hm.ndof; ++i) {
        const int nz = hm.rowptr[i + 1] - hm.rowptr[i];
        c += 2.0 + nz * (hm.row_slot[i] >= 0 ? 2.0 : 1.0);
    }
    return c * h->NB * h->cfg.n_fine;
}

FineArgs pppc::detail::team_args(pppc_handle* h, int lanes, int t, int teams, int nb, const FineArgs& base,
                                 size_t* part_off) {
    const size_t ts = h->fp32 ? sizeof(float) : sizeof(double);
    const size_t ndof = h->hm.ndof;
    auto at = [&](void* b, size_t elems) -> void* { return b ? static_cast<char*>(b) + elems * ts : nullptr; };
    const pppc_row_tables& rt = h->row_tables.at(nb);
    FineArgs a = base;
    a.NB = lanes;
    a.lane0 = t * lanes;
    a.ld = h->NB;
    a.n_teams = teams;
    const size_t v = (size_t)t * ndof * lanes;
    a.r = at(h->r, v);
    a.z = at(h->z, v);
    a.w = at(h->w, v);
    a.p = at(h->p, v);
    a.s = at(h->s, v);
    a.x = at(h->x, v);
    a.dx = at(h->dx, v);
    a.tri_m = at(h->tri_m, v);
    a.tri_ie = at(h->tri_ie, v);
    a.J = at(h->J, (size_t)t * h->hm.n_slots * lanes);
    a.invd_sp = at(h->invd, (size_t)t * h->hm.n_sp * lanes);
    a.part = at(h->part, *part_off);
    *part_off += 2 * (size_t)nb * 3 * lanes;   // two buffers of 3 sums per lane and block
    a.amg_ws = at(h->amg_ws, (size_t)t * h->amg_units * lanes);
    a.bar = h->bar + t;
    a.row_start = rt.rs;
    a.long_start = rt.ls;
    a.long_rows = rt.lr;
    const size_t budget = h->smem_optin - h->fine_static_smem - 1024;
    choose_vec_rows(h->fp32, lanes, rt.rows_max, budget, &a.vec_rows, &a.vec_w);
    if (t > 0) {   // the Newton trace records one team's lanes
        a.trace = nullptr;
        a.trace_cap = 0;
        a.trace_len = nullptr;
    }
    return a;
}

void pppc::detail::choose_vec_rows(bool fp32, int NB, int rows_max, size_t budget, int* vec_rows, int* vec_w) {
    const int V = fp32 ? 4 : 2, G = NB / V, threads = G * (1024 / G);
    *vec_rows = 0;
    *vec_w = 0;
    if (fine_smem(fp32, NB, threads, rows_max, 4) <= budget) {
        *vec_rows = rows_max;
        *vec_w = 1;
    } else if (fine_smem(fp32, NB, threads, rows_max, 3) <= budget) {
        *vec_rows = rows_max;
    }
}

namespace {

// jumps d and ||d||^2, ||F||^2 into h->jsums
pppc_status run_jumps(pppc_handle* h, const double* Ul, const double* Fl, double* rel_res) {
    CK(cudaEventRecord(h->ev[2], h->st));
    launch_jumps(h->hm.ndof, h->N, h->NB, Ul, Fl, h->d, h->part, h->jsums, h->st);
    h->stats.launches += 2;
    CK(cudaEventRecord(h->ev[3], h->st));
    CK(cudaGetLastError());
    double js[2];
    CK(cudaMemcpyAsync(js, h->jsums, sizeof js, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const double rr = js[1] > 0.0 ? std::sqrt(js[0] / js[1]) : (js[0] > 0.0 ? INFINITY : 0.0);
    if (rel_res) *rel_res = rr;
    h->stats.rel_res = rr;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]));
    h->stats.coarse_ms += ms;
    if (!std::isfinite(js[0]) || !std::isfinite(js[1])) return fail(h, PPPC_ERR_NAN, "non-finite jump norm");
    return PPPC_OK;
}

// Kbar frozen at the N lanes of `state`.
pppc_status run_kbar(pppc_handle* h, const double* state) {
    const int lin = h->cfg.coarse_lin;
    if (lin != PPPC_COARSE_ZERO_FIELD && h->md.n_nl > 0) {
        launch_elem_data(h->md, h->NB, state, h->elem, h->st);
        h->stats.launches += 1;
    }
    if (h->md.n_slots > 0) {
        launch_kbar(h->md, h->N, h->NB, lin, h->elem, h->Kbar, h->st);
        h->stats.launches += 1;
    }
    CK(cudaGetLastError());
    return PPPC_OK;
}

CocgArgs single_cocg_args(pppc_handle* h);

// Unew = Fl (shifted) + the harmonic correction from the jumps in h->d and
// the current Kbar (Eqs. 11-14 in delta form).
pppc_status run_correct(pppc_handle* h, const double* Fl, double* Unew) {
    if (h->md.n_sp > 0) {
        launch_coarse_rhs(h->md, h->N, h->NB, h->H, 1.0 / h->dT, h->d, h->tw, h->y, h->b, h->st);
        h->stats.launches += 2;
    }
    CK(cudaGetLastError());
    TRY(reset_control(h));
    const CocgArgs c = single_cocg_args(h);
    CK(launch_cocg(c, h->coarse_fp32, h->cocg_cfg, h->st));
    h->stats.launches += 1;
    TRY(device_status(h, "harmonic solves"));
    launch_idft_update(h->hm.ndof, h->N, h->NB, h->H, h->coarse_fp32, h->cx, Fl, h->tw, Unew, h->st);
    h->stats.launches += 1;
    CK(cudaGetLastError());
    return PPPC_OK;
}

// Arguments of h's own harmonic solves: the batched COCG over all harmonics,
// multigrid-preconditioned with precond = 2.
CocgArgs single_cocg_args(pppc_handle* h) {
    CocgArgs c = cocg_args(h);
    if (h->amg_levels > 1) {
        // multigrid-preconditioned harmonic solves (precond = 2)
        c.amg = h->d_amg;
        c.amg_levels = h->amg_levels;
        c.amg_sweeps = kAmgCoarsestSweeps;
        c.amg_fp32 = h->fp32 ? 1 : 0;
        c.amg_ws = h->camg_ws;
        c.amg_J = h->camg_J;
        c.amg_r = h->camg_r;
        c.amg_z = h->camg_z;
        c.klinP = h->fp32 ? static_cast<const void*>(h->md.Klin32) : static_cast<const void*>(h->md.Klin);
        c.row_start = h->d_row_start;
        c.long_start = h->d_long_start;
        c.long_rows = h->d_long_rows;
    }
    return c;
}

// Unew = coarse-corrected state from Ul, Fl and the jumps in h->d.
pppc_status run_coarse_solve(pppc_handle* h, const double* Ul, const double* Fl, double* Unew) {
    CK(cudaEventRecord(h->ev[2], h->st));
    TRY(run_kbar(h, h->cfg.coarse_at == PPPC_COARSE_AT_F ? Fl : Ul));
    TRY(run_correct(h, Fl, Unew));
    CK(cudaEventRecord(h->ev[3], h->st));
    CK(cudaEventSynchronize(h->ev[3]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]));
    h->stats.coarse_ms += ms;
    return PPPC_OK;
}

// PP-IC coarse sweep (Eq. 5): Unew and h->UNnext from Ul, Fl and h->UN.
pppc_status run_ppic_sweep(pppc_handle* h, const double* Ul, const double* Fl, double* Unew) {
    const int lin = h->cfg.coarse_lin;
    CK(cudaEventRecord(h->ev[2], h->st));
    if (lin != PPPC_COARSE_ZERO_FIELD && h->md.n_nl > 0) {
        launch_elem_data(h->md, h->NB, h->cfg.coarse_at == PPPC_COARSE_AT_F ? Fl : Ul, h->elem, h->st);
        h->stats.launches += 1;
    }
    if (h->md.n_slots > 0) {
        launch_kbar(h->md, h->N, h->NB, lin, h->elem, h->Kbar, h->st);
        h->stats.launches += 1;
    }
    const int ndof = h->hm.ndof;
    launch_ppic_start(ndof, h->NB, Ul, h->UN, h->dcur, Unew, h->st);
    h->stats.launches += 1;
    CocgArgs c{};
    c.mesh = h->md;
    c.N = h->N;
    c.H = 1;
    c.inv_dT = 1.0 / h->dT;
    c.tol = h->cfg.tol_coarse;
    c.max_it = h->cfg.max_coarse;
    c.Kbar = h->Kbar;
    c.tw = h->tw_c1;  // shift c = 1: the matrix is Q = Kbar + M/dT
    c.b = h->b;
    c.x = h->cx;
    c.r = h->cr;
    c.z = h->cz;
    c.w = h->cw;
    c.p = h->cp;
    c.s = h->cs;
    c.invd_sp = h->cinvd;
    c.part = h->part;
    c.bar = h->bar;
    c.status = h->status;
    c.counters = h->counters;
    for (int n = 1; n <= h->N; ++n) {
        launch_ppic_rhs(h->md, 1.0 / h->dT, h->dcur, h->b, h->st);
        CK(cudaGetLastError());
        TRY(reset_control(h));
        CK(launch_cocg(c, false, h->cocg1_cfg, h->st));
        h->stats.launches += 2;
        TRY(device_status(h, "PP-IC coarse step"));
        launch_ppic_step(ndof, h->N, h->NB, n, Fl, Ul, h->UN, static_cast<const double*>(h->cx), h->dcur, Unew,
                         h->UNnext, h->st);
        h->stats.launches += 1;
    }
    launch_zero_pad_lanes(ndof, h->N, h->NB, Unew, h->st);
    CK(cudaGetLastError());
    CK(cudaEventRecord(h->ev[3], h->st));
    CK(cudaEventSynchronize(h->ev[3]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]));
    h->stats.coarse_ms += ms;
    return PPPC_OK;
}

pppc_status run_update(pppc_handle* h, const double* Ul, const double* Fl, double* Unew) {
    if (h->cfg.method == PPPC_METHOD_PPIC) return run_ppic_sweep(h, Ul, Fl, Unew);
    return run_coarse_solve(h, Ul, Fl, Unew);
}

void swap_state(pppc_handle* h) {
    std::swap(h->U, h->Unext);
    if (h->cfg.method == PPPC_METHOD_PPIC) std::swap(h->UN, h->UNnext);
    h->graph_dirty = true;   // a captured iteration holds the state's address
}

// ---- one PP-PC iteration as one captured CUDA graph -------------------------

bool graph_eligible(const pppc_handle* h) { return h->cfg.method == PPPC_METHOD_PPPC && h->trace_cap == 0; }

void destroy_graph(pppc_handle* h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->graph_dirty = true;
}

// Capture errors end the capture before returning.
#define GCAP(call)                                                                          \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGraph_t g_ = nullptr;                                                       \
            cudaStreamEndCapture(h->gst, &g_);                                              \
            if (g_) cudaGraphDestroy(g_);                                                   \
            cudaGetLastError();                                                             \
            return fail(h, PPPC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                   \
    } while (0)

// Capture U -> F (fine sweep, the handle's lane-team plan), jumps, Kbar,
// right-hand side + DFT, harmonic solves, inverse DFT + update into Unext,
// the commit of Unext into U and the control block, on the handle's graph
// stream.  The Newton tolerance and the commit threshold are read from
// d_ctl_in, which the graph's first node fills from pinned ctl_in.
pppc_status capture_iteration(pppc_handle* h) {
    destroy_graph(h);
    if (!h->gst) CK(cudaStreamCreateWithFlags(&h->gst, cudaStreamNonBlocking));
    if (!h->gev) CK(cudaEventCreate(&h->gev));
    if (!h->ctl_in) {
        CK(cudaMallocHost(&h->ctl_in, 2 * sizeof(double)));
        CK(cudaMallocHost(&h->ctl_out, sizeof(IterCtl)));
    }
    if (!h->d_ctl_in) {
        TRY(alloc_n(h, &h->d_ctl_in, 2));
        TRY(alloc_n(h, &h->d_ctl, 1));
        TRY(alloc_n(h, &h->d_graph_args, kMaxTeams));
        TRY(alloc_n(h, &h->d_graph_map, (size_t)h->sms));
    }
    FineArgs a = fine_args(h, h->F);
    a.tol_abs_dev = h->d_ctl_in;
    const bool one_team = h->plan.lanes < 0;
    if (!one_team) {
        std::vector<FineArgs> args;
        std::vector<int4> map;
        team_tables(h, h->plan, a, args, map);
        CK(cudaMemcpyAsync(h->d_graph_args, args.data(), args.size() * sizeof(FineArgs), cudaMemcpyHostToDevice,
                           h->st));
        CK(cudaMemcpyAsync(h->d_graph_map, map.data(), map.size() * sizeof(int4), cudaMemcpyHostToDevice, h->st));
    }
    CK(cudaStreamSynchronize(h->st));
    const CocgArgs c = single_cocg_args(h);
    const int ndof = h->hm.ndof, N = h->N, NB = h->NB;
    const size_t lane_bytes = (size_t)ndof * NB * sizeof(double);
    int kernels = 0;
    CK(cudaStreamBeginCapture(h->gst, cudaStreamCaptureModeThreadLocal));
    GCAP(cudaMemcpyAsync(h->d_ctl_in, h->ctl_in, 2 * sizeof(double), cudaMemcpyHostToDevice, h->gst));
    GCAP(cudaMemsetAsync(h->status, 0, sizeof(int), h->gst));
    GCAP(cudaMemsetAsync(h->bar, 0, kMaxTeams * sizeof(GridBarrier), h->gst));
    GCAP(reset_team_ctl(h, h->gst));
    GCAP(cudaMemcpyAsync(h->F, h->U, lane_bytes, cudaMemcpyDeviceToDevice, h->gst));
    GCAP(cudaEventRecordWithFlags(h->ev[0], h->gst, cudaEventRecordExternal));
    if (one_team)
        GCAP(launch_fine_sweep(a, h->fp32, h->fine_cfg, h->gst));
    else
        GCAP(launch_fine_batch(h->d_graph_args, h->d_graph_map, h->fp32, h->sms, h->plan.smem, h->gst));
    kernels += 1;
    GCAP(cudaEventRecordWithFlags(h->ev[1], h->gst, cudaEventRecordExternal));
    launch_jumps(ndof, N, NB, h->U, h->F, h->d, h->part, h->jsums, h->gst);
    kernels += 2;
    const int lin = h->cfg.coarse_lin;
    if (lin != PPPC_COARSE_ZERO_FIELD && h->md.n_nl > 0) {
        launch_elem_data(h->md, NB, h->cfg.coarse_at == PPPC_COARSE_AT_F ? h->F : h->U, h->elem, h->gst);
        kernels += 1;
    }
    if (h->md.n_slots > 0) {
        launch_kbar(h->md, N, NB, lin, h->elem, h->Kbar, h->gst);
        kernels += 1;
    }
    if (h->md.n_sp > 0) {
        launch_coarse_rhs(h->md, N, NB, h->H, 1.0 / h->dT, h->d, h->tw, h->y, h->b, h->gst);
        kernels += 2;
    }
    GCAP(cudaGetLastError());
    GCAP(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), h->gst));   // the harmonic solves' barrier; status kept
    GCAP(launch_cocg(c, h->coarse_fp32, h->cocg_cfg, h->gst));
    launch_idft_update(ndof, N, NB, h->H, h->coarse_fp32, h->cx, h->F, h->tw, h->Unext, h->gst);
    launch_commit((long long)ndof * NB, h->status, h->jsums, h->d_ctl_in + 1, h->Unext, h->U, h->counters, h->d_ctl,
                  h->gst);
    kernels += 4;
    GCAP(cudaGetLastError());
    GCAP(cudaEventRecordWithFlags(h->ev[3], h->gst, cudaEventRecordExternal));
    GCAP(cudaMemcpyAsync(h->ctl_out, h->d_ctl, sizeof(IterCtl), cudaMemcpyDeviceToHost, h->gst));
    cudaGraph_t g = nullptr;
    CK(cudaStreamEndCapture(h->gst, &g));
    const cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    h->graph_kernels = kernels;
    h->graph_dirty = false;
    return PPPC_OK;
}

// One PP-PC iteration through the graph: U^{k+1} replaces U^k unless
// rel_res(U^k) <= tol_commit.  *rr receives rel_res(U^k).  One host sync.
pppc_status run_graph_iteration(pppc_handle* h, double tol_commit, double* rr) {
    TRY(choose_plan(h, h->U, h->F));   // a first sweep tunes the lane split outside any graph
    if (h->graph_dirty || !h->gexec) TRY(capture_iteration(h));
    h->ctl_in[0] = fine_args(h, h->F).tol_abs;   // the inexact schedule's Newton tolerance
    h->ctl_in[1] = tol_commit;
    CK(cudaStreamSynchronize(h->st));          // the caller's work on its stream comes first
    CK(cudaEventRecord(h->ev[2], h->gst));
    CK(cudaGraphLaunch(h->gexec, h->gst));
    CK(cudaEventRecord(h->gev, h->gst));
    CK(cudaStreamSynchronize(h->gst));
    h->stats.launches += h->graph_kernels;
    h->stats.graph_launches += 1;
    // fine and coarse device time from the graph's event nodes; if those
    // cannot be read, the whole launch counts as fine time
    float fms = 0.f, cms = 0.f;
    if (cudaEventElapsedTime(&fms, h->ev[0], h->ev[1]) == cudaSuccess &&
        cudaEventElapsedTime(&cms, h->ev[1], h->ev[3]) == cudaSuccess) {
        h->stats.fine_ms += fms;
        h->stats.coarse_ms += cms;
    } else {
        cudaGetLastError();
        CK(cudaEventElapsedTime(&fms, h->ev[2], h->gev));
        h->stats.fine_ms += fms;
    }
    const IterCtl& o = *h->ctl_out;
    if (o.status != 0) {
        TRY(device_status(h, "PP-PC iteration"));
        return fail(h, PPPC_ERR_CUDA, "PP-PC iteration: device status " + std::to_string(o.status));
    }
    const double dd = o.jsums[0], ff = o.jsums[1];
    if (!std::isfinite(dd) || !std::isfinite(ff)) return fail(h, PPPC_ERR_NAN, "non-finite jump norm");
    *rr = ff > 0.0 ? std::sqrt(dd / ff) : (dd > 0.0 ? INFINITY : 0.0);
    h->stats.rel_res = *rr;
    return PPPC_OK;
}

pppc_status begin_call(pppc_handle* h) {
    CK(cudaMemsetAsync(h->counters, 0, kCounters * sizeof(long long), h->st));
    h->stats = pppc_stats{};
    return PPPC_OK;
}

pppc_status end_call(pppc_handle* h) {
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
    return PPPC_OK;
}

pppc_status stage_in(pppc_handle* h, const double* U, int on_device, double* lanes) {
    const size_t n = (size_t)h->N * h->hm.n_nodes;
    const double* src = U;
    if (!on_device) {
        CK(cudaMemcpyAsync(h->ext, U, n * sizeof(double), cudaMemcpyHostToDevice, h->st));
        src = h->ext;
    }
    launch_state_to_lanes(h->hm.ndof, h->hm.n_nodes, h->N, h->NB, h->d_node_of_dof, src, lanes, h->st);
    h->stats.launches += 1;
    CK(cudaGetLastError());
    return PPPC_OK;
}

pppc_status stage_out(pppc_handle* h, const double* lanes, double* U, int on_device) {
    const size_t n = (size_t)h->N * h->hm.n_nodes;
    double* dst = on_device ? U : h->ext;
    launch_lanes_to_state(h->hm.ndof, h->hm.n_nodes, h->N, h->NB, h->d_dof_of_node, lanes, dst, h->st);
    h->stats.launches += 1;
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(U, h->ext, n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return PPPC_OK;
}

}  // namespace

// Stages of one iteration, for the adjoint driver (adjoint.cu).
pppc_status pppc::detail::stage_ready(pppc_handle* h) { return need_ready(h); }
pppc_status pppc::detail::stage_reset(pppc_handle* h) { return reset_control(h); }
pppc_status pppc::detail::stage_jumps(pppc_handle* h, const double* Ul, const double* Fl, double* rr) {
    return run_jumps(h, Ul, Fl, rr);
}
pppc_status pppc::detail::stage_kbar(pppc_handle* h, const double* state) { return run_kbar(h, state); }
pppc_status pppc::detail::stage_correct(pppc_handle* h, const double* Fl, double* Unew) {
    return run_correct(h, Fl, Unew);
}

namespace {

template <typename T>
pppc_status upload_as(pppc_handle* h, const void** out, const std::vector<double>& v) {
    std::vector<T> c(v.begin(), v.end());
    T* d = nullptr;
    TRY(upload(h, &d, c));
    *out = d;
    return PPPC_OK;
}

// values in the fine PCG's precision
pppc_status upload_values(pppc_handle* h, const void** out, const std::vector<double>& v) {
    return h->fp32 ? upload_as<float>(h, out, v) : upload_as<double>(h, out, v);
}

// Multigrid preconditioner of the fine PCG (precond = 2): the representative
// matrix A0 = J at zero field (K_lin plus the Brauer law's nu(0) = k1 + k3 on
// the nonlinear elements, plus M / dt) is assembled by the device, the
// hierarchy is built on the host (amg_host.cpp) and uploaded in the PCG
// precision with one workspace region per lane team.  A mesh too small to
// coarsen keeps amg_levels = 0 and the sweep falls back to Jacobi.
pppc_status setup_amg(pppc_handle* h) {
    const HostMesh& hm = h->hm;
    h->amg_levels = 0;
    if (hm.n_slots > 0) launch_kbar(h->md, h->N, h->NB, PPPC_COARSE_ZERO_FIELD, h->elem, h->Kbar, h->st);
    CK(cudaGetLastError());
    std::vector<double> klin(hm.nnz), kbar0(hm.n_slots), mslot(hm.n_slots);
    CK(cudaMemcpyAsync(klin.data(), h->md.Klin, hm.nnz * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    if (hm.n_slots > 0) {
        CK(cudaMemcpyAsync(kbar0.data(), h->Kbar, hm.n_slots * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(mslot.data(), h->md.Mslot, hm.n_slots * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    }
    CK(cudaStreamSynchronize(h->st));
    std::vector<double> a0(hm.nnz);
    for (int i = 0; i < hm.ndof; ++i)
        for (int k = hm.rowptr[i]; k < hm.rowptr[i + 1]; ++k) {
            const int sl = hm.row_slot[i] >= 0 ? hm.row_slot[i] + (k - hm.rowptr[i]) : -1;
            a0[k] = sl >= 0 ? kbar0[sl] + mslot[sl] / h->dt : klin[k];
        }
    std::vector<AmgHostLevel> lv;
    std::string err;
    if (!build_amg(hm.ndof, hm.rowptr.data(), hm.col.data(), a0.data(), hm.row_slot.data(), AmgOptions{}, lv, err))
        return fail(h, PPPC_ERR_INVALID_ARG, err);
    if (lv.size() < 2) return PPPC_OK;
    if ((int)lv.size() > kAmgMaxLevels) lv.resize(kAmgMaxLevels);
    std::vector<AmgLevel> dl(lv.size());
    long long units = 0;
    auto take = [&](long long n) {
        const long long o = units;
        units += n;
        return o;
    };
    h->amg_rows.clear();
    for (size_t l = 0; l < lv.size(); ++l) {
        const AmgHostLevel& L = lv[l];
        AmgLevel& d = dl[l];
        d = AmgLevel{};
        d.n = L.n;
        d.n_slots = L.n_slots;
        d.n_sp = L.n_sp;
        d.off_b = d.off_q = d.off_slot = -1;
        h->amg_rows.push_back(L.n);
        TRY(upload_values(h, &d.l1, L.l1));
        if (l == 0) {
            // the fine level's matrix is the lane's Newton matrix itself
            d.off_y = take(L.n);
            d.off_l1 = take(L.n_sp);
            d.sp_index = h->md.sp_index;
            continue;
        }
        d.off_slot = take(L.n_slots);
        d.off_l1 = take(L.n_sp);
        d.off_b = take(L.n);
        d.off_y = take(L.n);
        d.off_q = take(L.n);
        int *rowptr, *col, *row_slot, *sp_index, *sp_rows, *Pptr, *Pcol, *Rptr, *Rcol, *cptr, *csrc;
        TRY(upload(h, &rowptr, L.rowptr));
        TRY(upload(h, &col, L.col));
        TRY(upload(h, &row_slot, L.row_slot));
        TRY(upload(h, &sp_index, L.sp_index));
        TRY(upload(h, &sp_rows, L.sp_rows));
        TRY(upload(h, &Pptr, L.Pptr));
        TRY(upload(h, &Pcol, L.Pcol));
        TRY(upload(h, &Rptr, L.Rptr));
        TRY(upload(h, &Rcol, L.Rcol));
        TRY(upload(h, &cptr, L.cptr));
        TRY(upload(h, &csrc, L.csrc));
        long long* cost;
        TRY(upload(h, &cost, L.cost));
        d.cost = cost;
        d.rowptr = rowptr;
        d.col = col;
        d.row_slot = row_slot;
        d.sp_index = sp_index;
        d.sp_rows = sp_rows;
        d.Pptr = Pptr;
        d.Pcol = Pcol;
        d.Rptr = Rptr;
        d.Rcol = Rcol;
        d.cptr = cptr;
        d.csrc = csrc;
        TRY(upload_values(h, &d.val, L.val));
        TRY(upload_values(h, &d.Pval, L.Pval));
        TRY(upload_values(h, &d.Rval, L.Rval));
        TRY(upload_values(h, &d.slot_base, L.slot_base));
        TRY(upload_values(h, &d.cw, L.cw));
    }
    TRY(upload(h, &h->d_amg, dl));
    const size_t ts = h->fp32 ? sizeof(float) : sizeof(double);
    h->amg_ws = dev_alloc(h, (size_t)units * h->NB * ts);
    if (!h->amg_ws) return fail(h, PPPC_ERR_NOMEM, "multigrid workspace allocation failed");
    CK(cudaMemsetAsync(h->amg_ws, 0, (size_t)units * h->NB * ts, h->st));
    // the harmonic solves' V-cycle: the same levels on 2H lanes (re, im per harmonic)
    const size_t cl = 2 * (size_t)h->H;
    h->camg_ws = dev_alloc(h, (size_t)units * cl * ts);
    h->camg_J = dev_alloc(h, (size_t)std::max(hm.n_slots, 1) * cl * ts);
    h->camg_r = dev_alloc(h, (size_t)hm.ndof * cl * ts);
    h->camg_z = dev_alloc(h, (size_t)hm.ndof * cl * ts);
    if (!h->camg_ws || !h->camg_J || !h->camg_r || !h->camg_z)
        return fail(h, PPPC_ERR_NOMEM, "multigrid workspace allocation failed");
    CK(cudaMemsetAsync(h->camg_ws, 0, (size_t)units * cl * ts, h->st));
    h->amg_units = units;
    h->amg_levels = (int)lv.size();
    return PPPC_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

void pppc_config_default(pppc_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->T = 0.02;
    c->N = 16;
    c->n_fine = 20;
    c->precision = PPPC_FP64;
    c->coarse_lin = PPPC_COARSE_AVG_JACOBIAN;
    c->tol_newton = 1e-10;
    c->max_newton = 30;
    c->tol_lin = 1e-6;
    c->max_lin = 20000;
    c->tol_coarse = 1e-8;
    c->max_coarse = 20000;
    c->eta0 = 1e-2;
    c->predictor = 1;
    c->method = PPPC_METHOD_PPPC;
    c->coarse_at = PPPC_COARSE_AT_U;
}

const char* pppc_status_string(pppc_status s) {
    const int i = (int)s;
    if (i < 0 || i >= (int)(sizeof kStatusNames / sizeof kStatusNames[0])) return "PPPC_ERR_UNKNOWN";
    return kStatusNames[i];
}

const char* pppc_last_error(pppc_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

pppc_status pppc_create(const pppc_config* cfg, pppc_handle** out) {
    if (!out) {
        g_create_error = "out is NULL";
        return PPPC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!cfg) {
        g_create_error = "cfg is NULL";
        return PPPC_ERR_INVALID_ARG;
    }
    const pppc_config& c = *cfg;
    std::string why;
    if (!(c.T > 0.0) || !std::isfinite(c.T)) why = "T must be positive";
    else if (c.N < 2 || c.N > kMaxLanes || (c.N % 2) != 0) why = "N must be even and in [2, 1024]";
    else if (c.n_fine < 1) why = "n_fine must be >= 1";
    else if (c.precision != PPPC_FP64 && c.precision != PPPC_MIXED) why = "unknown precision";
    else if (c.coarse_lin < 0 || c.coarse_lin > 2) why = "unknown coarse_lin";
    else if (!(c.tol_newton > 0.0) || !(c.tol_lin > 0.0) || !(c.tol_coarse > 0.0)) why = "tolerances must be positive";
    else if (!(c.eta0 > 0.0) || !(c.eta0 < 1.0)) why = "eta0 must be in (0, 1)";
    else if (c.method != PPPC_METHOD_PPPC && c.method != PPPC_METHOD_PPIC) why = "unknown method";
    else if (c.coarse_at != PPPC_COARSE_AT_U && c.coarse_at != PPPC_COARSE_AT_F) why = "unknown coarse_at";
    else if (c.newton_schedule != 0 && c.newton_schedule != 1) why = "newton_schedule must be 0 or 1";
    else if (c.precond < 0 || c.precond > 2) why = "precond must be 0, 1 or 2";
    else if (c.predictor < 0 || c.predictor > 2) why = "predictor must be 0, 1 or 2";
    else if (c.max_newton < 1 || c.max_lin < 1 || c.max_coarse < 1) why = "iteration caps must be >= 1";
    else if (c.lane_team < -1) why = "lane_team must be -1, 0 or a lane count";
    else if ((c.alloc == nullptr) != (c.free_fn == nullptr)) why = "alloc and free_fn must be given together";
    if (!why.empty()) {
        g_create_error = why;
        return PPPC_ERR_INVALID_ARG;
    }
    pppc_handle* h = new pppc_handle();
    h->cfg = c;
    h->st = static_cast<cudaStream_t>(c.stream);
    h->N = c.N;
    // lanes padded to the fine kernel's lane-vector width (4 FP32 / 2 FP64)
    h->NB = c.precision == PPPC_MIXED ? (c.N + 3) / 4 * 4 : c.N;
    h->H = c.N / 2 + 1;
    h->dT = c.T / c.N;
    h->dt = c.T / ((double)c.N * c.n_fine);
    h->fp32 = c.precision == PPPC_MIXED;
    *out = h;
    return PPPC_OK;
}

void pppc_destroy(pppc_handle* h) {
    if (!h) return;
    free_all(h);
    if (h->gst) cudaStreamDestroy(h->gst);
    if (h->gev) cudaEventDestroy(h->gev);
    if (h->ctl_in) cudaFreeHost(h->ctl_in);
    if (h->ctl_out) cudaFreeHost(h->ctl_out);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

int32_t pppc_ndof(pppc_handle* h) { return (h && h->has_mesh) ? h->hm.ndof : 0; }

pppc_status pppc_set_mesh(pppc_handle* h, int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri,
                          const int32_t* region, const uint8_t* dirichlet, int32_t n_regions,
                          const pppc_material* mat) {
    if (!h) return PPPC_ERR_INVALID_ARG;
    if (!xy || !tri || !region || !dirichlet || !mat || n_regions < 1)
        return fail(h, PPPC_ERR_INVALID_ARG, "null array or n_regions < 1");
    std::vector<int> kinds(n_regions, 0);
    std::vector<double> mtab((size_t)n_regions * 8, 0.0);
    for (int r = 0; r < n_regions; ++r) {
        const pppc_material& q = mat[r];
        if (!(q.sigma >= 0.0) || !std::isfinite(q.sigma))
            return fail(h, PPPC_ERR_INVALID_ARG, "region " + std::to_string(r) + ": sigma must be >= 0");
        if (q.nu_model == PPPC_NU_LINEAR) {
            if (!(q.nu > 0.0) || !std::isfinite(q.nu))
                return fail(h, PPPC_ERR_INVALID_ARG, "region " + std::to_string(r) + ": nu must be > 0");
        } else if (q.nu_model == PPPC_NU_BRAUER) {
            if (!(q.k1 > 0.0) || !(q.k2 >= 0.0) || !(q.k3 > 0.0) || !std::isfinite(q.k1) || !std::isfinite(q.k2) ||
                !std::isfinite(q.k3))
                return fail(h, PPPC_ERR_INVALID_ARG,
                            "region " + std::to_string(r) + ": Brauer needs k1 > 0, k2 >= 0, k3 > 0");
            if (!(q.bmax >= 0.0) || !std::isfinite(q.bmax))
                return fail(h, PPPC_ERR_INVALID_ARG, "region " + std::to_string(r) + ": bmax must be >= 0");
            kinds[r] |= ELEM_NONLINEAR;
        } else {
            return fail(h, PPPC_ERR_INVALID_ARG, "region " + std::to_string(r) + ": unknown nu_model");
        }
        if (q.sigma > 0.0) kinds[r] |= ELEM_CONDUCTIVE;
        if (q.is_source) kinds[r] |= ELEM_SOURCE;
        double* m = &mtab[(size_t)r * 8];
        m[0] = q.sigma;
        m[1] = (double)q.nu_model;
        m[2] = q.nu;
        m[3] = q.k1;
        m[4] = q.k2;
        m[5] = q.k3;
        m[6] = q.is_source ? 1.0 : 0.0;
        m[7] = q.bmax > 0.0 ? q.bmax * q.bmax : INFINITY;   // cap on b = |B|^2
    }
    // host-side validation and preprocessing first: an invalid mesh is
    // refused before any device work and leaves the previous mesh in place
    std::string err;
    HostMesh hm_new;
    if (!build_host_mesh(n_nodes, n_tri, tri, region, dirichlet, n_regions, kinds.data(), hm_new, err))
        return fail(h, PPPC_ERR_INVALID_ARG, err);
    {
        bool any_source = false;
        for (int e = 0; e < n_tri && !any_source; ++e) any_source = (hm_new.elem_kind[e] & ELEM_SOURCE) != 0;
        if (!any_source) return fail(h, PPPC_ERR_INVALID_ARG, "no triangle lies in a source region");
    }
    free_all(h);
    h->has_source = false;
    h->trace_cap = 0;
    for (auto& e : h->ev)
        if (!e) CK(cudaEventCreate(&e));
    h->hm = std::move(hm_new);
    HostMesh& hm = h->hm;
    h->traj = h->lam = h->adjA = h->adjB = h->adjF = h->gpart = h->gout = nullptr;
    h->nl_sel = nullptr;
    h->nl_region.resize(hm.n_nl);
    for (int q = 0; q < hm.n_nl; ++q) h->nl_region[q] = region[hm.nl_elems[q]];
    h->region_sigma.resize(n_regions);
    h->region_kind = kinds;
    for (int r = 0; r < n_regions; ++r) h->region_sigma[r] = mat[r].sigma;

    // uploads
    std::vector<double> vxy(xy, xy + 2 * (size_t)n_nodes);
    std::vector<int> vtri(tri, tri + 3 * (size_t)n_tri), vreg(region, region + n_tri);
    double* d_xy;
    int *d_tri, *d_reg, *d_contrib_ptr, *d_contrib, *d_nl_elems, *d_dcoup_ptr, *d_dcoup;
    double *d_mat, *d_geom;
    int *rowptr, *col, *diag_k, *row_slot, *sp_index, *sp_rows, *slot_k, *nl_dofs, *nlc_ptr, *nlc;
    TRY(upload(h, &d_xy, vxy));
    TRY(upload(h, &d_tri, vtri));
    TRY(upload(h, &d_reg, vreg));
    TRY(upload(h, &d_mat, mtab));
    TRY(upload(h, &d_contrib_ptr, hm.contrib_ptr));
    TRY(upload(h, &d_contrib, hm.contrib));
    TRY(upload(h, &d_nl_elems, hm.nl_elems));
    TRY(upload(h, &d_dcoup_ptr, hm.dcoup_ptr));
    TRY(upload(h, &d_dcoup, hm.dcoup));
    TRY(upload(h, &rowptr, hm.rowptr));
    TRY(upload(h, &col, hm.col));
    TRY(upload(h, &diag_k, hm.diag_k));
    TRY(upload(h, &row_slot, hm.row_slot));
    TRY(upload(h, &sp_index, hm.sp_index));
    TRY(upload(h, &sp_rows, hm.sp_rows));
    TRY(upload(h, &slot_k, hm.slot_k));
    TRY(upload(h, &nl_dofs, hm.nl_dofs));
    TRY(upload(h, &nlc_ptr, hm.nlc_ptr));
    TRY(upload(h, &nlc, hm.nlc));
    TRY(upload(h, &h->d_node_of_dof, hm.node_of_dof));
    TRY(upload(h, &h->d_dof_of_node, hm.dof_of_node));
    TRY(alloc_n(h, &d_geom, (size_t)n_tri * 8));
    double *Klin, *invdiag_lin, *Mslot, *g, *dlin, *nl_geom, *nl_k, *nlc_ab;
    float *Klin32, *invdiag_lin32;
    TRY(alloc_n(h, &Klin, hm.nnz));
    TRY(alloc_n(h, &Klin32, hm.nnz));
    TRY(alloc_n(h, &invdiag_lin, hm.ndof));
    TRY(alloc_n(h, &invdiag_lin32, hm.ndof));
    TRY(alloc_n(h, &Mslot, hm.n_slots));
    TRY(alloc_n(h, &g, hm.ndof));
    TRY(alloc_n(h, &dlin, hm.ndof));
    TRY(alloc_n(h, &nl_geom, (size_t)hm.n_nl * 8));
    TRY(alloc_n(h, &nl_k, (size_t)hm.n_nl * 4));
    TRY(alloc_n(h, &nlc_ab, hm.nlc.size()));
    TRY(alloc_n(h, &h->tw, 2 * (size_t)h->N));
    TRY(alloc_n(h, &h->scalars, 2));
    TRY(alloc_n(h, &h->status, 1));
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));

    SetupArgs sa{};
    sa.n_tri = n_tri;
    sa.ndof = hm.ndof;
    sa.nnz = hm.nnz;
    sa.n_slots = hm.n_slots;
    sa.n_nl = hm.n_nl;
    sa.n_nlc = (int)hm.nlc.size();
    sa.n_regions = n_regions;
    sa.N = h->N;
    sa.xy = d_xy;
    sa.tri = d_tri;
    sa.region = d_reg;
    sa.mat = d_mat;
    sa.contrib_ptr = d_contrib_ptr;
    sa.contrib = d_contrib;
    sa.rowptr = rowptr;
    sa.diag_k = diag_k;
    sa.slot_k = slot_k;
    sa.nl_elems = d_nl_elems;
    sa.nlc = nlc;
    sa.dcoup_ptr = d_dcoup_ptr;
    sa.dcoup = d_dcoup;
    sa.dlin = dlin;
    sa.geom = d_geom;
    sa.Klin = Klin;
    sa.Klin32 = Klin32;
    sa.invdiag_lin = invdiag_lin;
    sa.invdiag_lin32 = invdiag_lin32;
    sa.Mslot = Mslot;
    sa.g = g;
    sa.nl_geom = nl_geom;
    sa.nl_k = nl_k;
    sa.nlc_ab = nlc_ab;
    sa.tw = h->tw;
    sa.scalars = h->scalars;
    sa.status = h->status;
    CK(launch_setup(sa, h->st));
    TRY(device_status(h, "pppc_set_mesh"));
    double sc[2];
    CK(cudaMemcpy(sc, h->scalars, sizeof sc, cudaMemcpyDeviceToHost));
    h->src_area = sc[0];
    h->gnorm = sc[1];
    if (!(h->src_area > 0.0)) return fail(h, PPPC_ERR_INVALID_ARG, "source region has zero area");

    MeshDev& m = h->md;
    m.ndof = hm.ndof;
    m.nnz = hm.nnz;
    m.n_slots = hm.n_slots;
    m.n_sp = hm.n_sp;
    m.n_nl = hm.n_nl;
    m.rowptr = rowptr;
    m.col = col;
    m.diag_k = diag_k;
    m.row_slot = row_slot;
    m.sp_index = sp_index;
    m.sp_rows = sp_rows;
    m.slot_k = slot_k;
    m.Klin = Klin;
    m.Klin32 = Klin32;
    m.invdiag_lin = invdiag_lin;
    m.invdiag_lin32 = invdiag_lin32;
    m.Mslot = Mslot;
    m.g = g;
    m.dlin = dlin;
    m.nl_dofs = nl_dofs;
    m.nl_geom = nl_geom;
    m.nl_k = nl_k;
    m.nlc_ptr = nlc_ptr;
    m.nlc = nlc;
    m.nlc_ab = nlc_ab;

    // workspace
    const size_t LV = (size_t)hm.ndof * h->NB;
    const size_t ts = h->fp32 ? sizeof(float) : sizeof(double);
    TRY(alloc_n(h, &h->U, LV));
    TRY(alloc_n(h, &h->Unext, LV));
    TRY(alloc_n(h, &h->F, LV));
    TRY(alloc_n(h, &h->uprev, LV));
    TRY(alloc_n(h, &h->d, LV));
    TRY(alloc_n(h, &h->elem, (size_t)kElemPlanes * hm.n_nl * h->NB));
    void** fv[] = {&h->r, &h->z, &h->w, &h->p, &h->s, &h->x, &h->dx};
    for (void** v : fv) {
        *v = dev_alloc(h, LV * ts);
        if (!*v) return fail(h, PPPC_ERR_NOMEM, "workspace allocation failed");
        CK(cudaMemsetAsync(*v, 0, LV * ts, h->st));
    }
    h->uprev2 = nullptr;
    if (h->cfg.predictor == 2) TRY(alloc_n(h, &h->uprev2, LV));
    if (h->cfg.precond == 1) {
        std::vector<int> low(hm.ndof, -1);
        for (int i = 1; i < hm.ndof; ++i)
            for (int k = hm.rowptr[i]; k < hm.rowptr[i + 1]; ++k)
                if (hm.col[k] == i - 1) low[i] = k;
        TRY(upload(h, &h->d_tri_low, low));
        h->tri_m = dev_alloc(h, LV * ts);
        h->tri_ie = dev_alloc(h, LV * ts);
        if (!h->tri_m || !h->tri_ie) return fail(h, PPPC_ERR_NOMEM, "workspace allocation failed");
    }
    h->J = dev_alloc(h, (size_t)hm.n_slots * h->NB * ts);
    h->invd = dev_alloc(h, (size_t)hm.n_sp * h->NB * ts);
    if (!h->J || !h->invd) return fail(h, PPPC_ERR_NOMEM, "workspace allocation failed");
    const size_t CV = (size_t)hm.ndof * h->H * 2;
    const size_t cts = h->coarse_fp32 ? sizeof(float) : sizeof(double);
    void** cv[] = {&h->cx, &h->cr, &h->cz, &h->cw, &h->cp, &h->cs};
    for (void** v : cv) {
        *v = dev_alloc(h, CV * cts);
        if (!*v) return fail(h, PPPC_ERR_NOMEM, "workspace allocation failed");
    }
    h->cinvd = dev_alloc(h, (size_t)hm.n_sp * h->H * 2 * cts);
    if (!h->cinvd) return fail(h, PPPC_ERR_NOMEM, "workspace allocation failed");
    TRY(alloc_n(h, &h->y, (size_t)hm.n_sp * h->NB));
    TRY(alloc_n(h, &h->b, (size_t)hm.n_sp * h->H * 2));
    TRY(alloc_n(h, &h->Kbar, hm.n_slots));
    {
        // Fine sweep: one block per SM, each owning a contiguous range of rows of
        // about equal cost (nonzeros; per-lane rows count double; long rows,
        // multiplied by the whole block, carry a fixed extra cost).
        int dev = 0, nb = 0, smem_optin = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nb, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        std::vector<int> rs, ls, lrows;
        int rows_max = 0;
        partition_rows(hm, nb, rs, ls, lrows, &rows_max);
        TRY(upload(h, &h->d_row_start, rs));
        TRY(upload(h, &h->d_long_start, ls));
        TRY(upload(h, &h->d_long_rows, lrows));
        // the team kernel's static shared memory bounds the grid-wide kernel's
        // (same body, plus a copy of its arguments)
        CK(fine_batch_prepare(h->fp32, &h->fine_static_smem));
        // keep p, s, x, w in shared memory when a block's rows fit
        choose_vec_rows(h->fp32, h->NB, rows_max, (size_t)smem_optin - h->fine_static_smem - 1024, &h->vec_rows,
                        &h->vec_w);
        CK(fine_config(h->fp32, h->NB, h->vec_rows, h->vec_w ? 4 : 3, &h->fine_cfg));
        if (h->fine_cfg.blocks != nb) return fail(h, PPPC_ERR_CUDA, "fine sweep: one block per SM expected");
        // lane teams (the plan is chosen at the first sweep)
        h->sms = nb;
        h->smem_optin = (size_t)smem_optin;
        h->plan = pppc_fine_plan{};
        std::fill(std::begin(h->tune_ms), std::end(h->tune_ms), 0.0);
        if (h->cfg.lane_team > 0) {
            const std::vector<int> cand = team_candidates(h);
            if (std::find(cand.begin(), cand.end(), h->cfg.lane_team) == cand.end())
                return fail(h, PPPC_ERR_INVALID_ARG,
                            "lane_team must be a lane-vector width times a power of two dividing the padded N");
        }
    }
    CK(cocg_config(h->coarse_fp32, h->H, &h->cocg_cfg));
    // partial sums: two buffers per reduction (fine: T, COCG: FP64) and the jumps' 2 per block
    size_t np = std::max((size_t)2 * h->fine_cfg.blocks * 3 * h->NB, (size_t)2 * h->cocg_cfg.blocks * 5 * h->H);
    np = std::max(np, (size_t)2 * 512);
    TRY(alloc_n(h, &h->part, np));
    TRY(alloc_n(h, &h->jsums, 2));
    TRY(alloc_n(h, &h->bar, kMaxTeams));
    CK(cudaMemsetAsync(h->bar, 0, kMaxTeams * sizeof(GridBarrier), h->st));
    TRY(alloc_n(h, &h->team_ctl, 4));
    TRY(alloc_n(h, &h->d_team_args, kMaxTeams));
    TRY(alloc_n(h, &h->d_team_map, (size_t)h->fine_cfg.blocks));
    TRY(alloc_n(h, &h->counters, kCounters));
    TRY(alloc_n(h, &h->ext, (size_t)h->N * hm.n_nodes));
    CK(cudaMemsetAsync(h->U, 0, LV * sizeof(double), h->st));
    if (h->cfg.method == PPPC_METHOD_PPIC) {
        TRY(alloc_n(h, &h->UN, hm.ndof));
        TRY(alloc_n(h, &h->UNnext, hm.ndof));
        TRY(alloc_n(h, &h->dcur, hm.ndof));
        TRY(alloc_n(h, &h->tw_c1, 2));
        CK(cudaMemsetAsync(h->UN, 0, hm.ndof * sizeof(double), h->st));
        CK(cudaMemsetAsync(h->tw_c1, 0, 2 * sizeof(double), h->st));
        CK(cocg_config(false, 1, &h->cocg1_cfg));
    }
    CK(cudaMemsetAsync(h->counters, 0, kCounters * sizeof(long long), h->st));
    h->amg_levels = 0;
    h->amg_ws = nullptr;
    h->d_amg = nullptr;
    h->camg_ws = h->camg_J = h->camg_r = h->camg_z = nullptr;
    h->amg_rows.clear();
    if (h->cfg.precond == 2) TRY(setup_amg(h));
    CK(cudaStreamSynchronize(h->st));
    h->has_mesh = true;
    return PPPC_OK;
}

pppc_status pppc_set_source(pppc_handle* h, int32_t n_harm, const double* amp, const double* freq,
                            const double* phase) {
    if (!h) return PPPC_ERR_INVALID_ARG;
    if (!h->has_mesh) return fail(h, PPPC_ERR_STATE, "pppc_set_mesh has not been called");
    if (n_harm < 1 || n_harm > kMaxHarm || !amp || !freq)
        return fail(h, PPPC_ERR_INVALID_ARG, "need 1..16 harmonics with amp and freq");
    SourceDev s{};
    s.n_harm = n_harm;
    for (int j = 0; j < n_harm; ++j) {
        const double cyc = freq[j] * h->cfg.T;
        if (!std::isfinite(amp[j]) || !std::isfinite(freq[j]) || std::fabs(cyc - std::round(cyc)) > 1e-9 * std::max(1.0, std::fabs(cyc)))
            return fail(h, PPPC_ERR_INVALID_ARG, "harmonic " + std::to_string(j) + ": freq * T must be an integer");
        s.amp[j] = amp[j];
        s.freq[j] = freq[j];
        s.phase[j] = phase ? phase[j] : 0.0;
    }
    h->src = s;
    h->has_source = true;
    return PPPC_OK;
}

pppc_status pppc_set_state(pppc_handle* h, const double* U, int32_t on_device) {
    if (!h) return PPPC_ERR_INVALID_ARG;
    if (!h->has_mesh) return fail(h, PPPC_ERR_STATE, "pppc_set_mesh has not been called");
    if (!U) return fail(h, PPPC_ERR_INVALID_ARG, "U is NULL");
    TRY(stage_in(h, U, on_device, h->U));
    h->rr_prev = INFINITY;
    if (h->UN)  // PP-IC: the end-of-period state starts at U_0 (lane 0 of the lane layout)
        CK(cudaMemcpy2DAsync(h->UN, sizeof(double), h->U, (size_t)h->NB * sizeof(double), sizeof(double),
                             h->hm.ndof, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    return PPPC_OK;
}

pppc_status pppc_get_state(pppc_handle* h, double* U, int32_t on_device) {
    if (!h) return PPPC_ERR_INVALID_ARG;
    if (!h->has_mesh) return fail(h, PPPC_ERR_STATE, "pppc_set_mesh has not been called");
    if (!U) return fail(h, PPPC_ERR_INVALID_ARG, "U is NULL");
    return stage_out(h, h->U, U, on_device);
}

pppc_status pppc_propagate_fine(pppc_handle* h, const double* U, double* F, int32_t on_device) {
    TRY(need_ready(h));
    if (!U || !F) return fail(h, PPPC_ERR_INVALID_ARG, "U or F is NULL");
    TRY(begin_call(h));
    TRY(stage_in(h, U, on_device, h->Unext));
    TRY(run_fine(h, h->Unext, h->F));
    TRY(end_call(h));
    h->stats.fine_steps = h->cfg.n_fine;
    return stage_out(h, h->F, F, on_device);
}

pppc_status pppc_propagate_fine_window(pppc_handle* h, const double* U, double* F, int32_t first, int32_t count,
                                       int32_t on_device) {
    TRY(need_ready(h));
    if (!U || !F) return fail(h, PPPC_ERR_INVALID_ARG, "U or F is NULL");
    if (first < 0 || count < 1 || (int64_t)first + count > h->cfg.n_fine)
        return fail(h, PPPC_ERR_INVALID_ARG, "window [first, first + count) must lie in [0, n_fine]");
    TRY(begin_call(h));
    TRY(stage_in(h, U, on_device, h->Unext));
    TRY(run_fine(h, h->Unext, h->F, first, count));
    TRY(end_call(h));
    h->stats.fine_steps = count;
    return stage_out(h, h->F, F, on_device);
}

pppc_status pppc_coarse_update(pppc_handle* h, const double* U, const double* F, double* U_new, double* rel_res,
                               int32_t on_device) {
    TRY(need_ready(h));
    if (!U || !F || !U_new) return fail(h, PPPC_ERR_INVALID_ARG, "U, F or U_new is NULL");
    if (h->cfg.method == PPPC_METHOD_PPIC)
        return fail(h, PPPC_ERR_UNSUPPORTED, "pppc_coarse_update: PP-IC needs the end-of-period state");
    TRY(begin_call(h));
    // lanes: Unext <- U, F <- F (h->U, the handle's state, is untouched)
    TRY(stage_in(h, U, on_device, h->Unext));
    TRY(stage_in(h, F, on_device, h->F));
    TRY(run_jumps(h, h->Unext, h->F, rel_res));
    TRY(run_coarse_solve(h, h->Unext, h->F, h->uprev));
    TRY(end_call(h));
    return stage_out(h, h->uprev, U_new, on_device);
}

pppc_status pppc_iterate(pppc_handle* h, double* rel_res) {
    TRY(need_ready(h));
    TRY(begin_call(h));
    if (graph_eligible(h)) {
        double rr = 0.0;
        TRY(run_graph_iteration(h, -1.0, &rr));   // always commit U^{k+1}
        if (rel_res) *rel_res = rr;
        h->rr_prev = rr;
        TRY(end_call(h));
        h->stats.fine_steps = h->cfg.n_fine;
        h->stats.pppc_iters = 1;
        return PPPC_OK;
    }
    TRY(run_fine(h, h->U, h->F));
    TRY(run_jumps(h, h->U, h->F, rel_res));
    h->rr_prev = h->stats.rel_res;
    TRY(run_update(h, h->U, h->F, h->Unext));
    CK(cudaStreamSynchronize(h->st));
    swap_state(h);
    TRY(end_call(h));
    h->stats.fine_steps = h->cfg.n_fine;
    h->stats.pppc_iters = 1;
    return PPPC_OK;
}

pppc_status pppc_solve_periodic(pppc_handle* h, double tol, int32_t kmax, int32_t* iters, double* rel_res) {
    TRY(need_ready(h));
    if (!(tol > 0.0) || kmax < 0) return fail(h, PPPC_ERR_INVALID_ARG, "tol must be > 0 and kmax >= 0");
    TRY(begin_call(h));
    double rr = INFINITY;
    for (int k = 0; graph_eligible(h); ++k) {
        // the update is committed on the device only while rel_res > tol and k < kmax
        TRY(run_graph_iteration(h, k >= kmax ? INFINITY : tol, &rr));
        h->rr_prev = rr;
        h->stats.fine_steps += h->cfg.n_fine;
        if (rr <= tol || k >= kmax) {
            if (iters) *iters = k;
            if (rel_res) *rel_res = rr;
            h->stats.pppc_iters = k;
            TRY(end_call(h));
            h->stats.rel_res = rr;
            if (rr <= tol) return PPPC_OK;
            return fail(h, PPPC_ERR_NOT_CONVERGED,
                        "rel_res " + std::to_string(rr) + " > tol after " + std::to_string(k) + " updates");
        }
    }
    for (int k = 0;; ++k) {
        TRY(run_fine(h, h->U, h->F));
        TRY(run_jumps(h, h->U, h->F, &rr));
        h->rr_prev = rr;
        h->stats.fine_steps += h->cfg.n_fine;
        if (rr <= tol || k >= kmax) {
            if (iters) *iters = k;
            if (rel_res) *rel_res = rr;
            h->stats.pppc_iters = k;
            TRY(end_call(h));
            h->stats.rel_res = rr;
            if (rr <= tol) return PPPC_OK;
            return fail(h, PPPC_ERR_NOT_CONVERGED,
                        "rel_res " + std::to_string(rr) + " > tol after " + std::to_string(k) + " updates");
        }
        TRY(run_update(h, h->U, h->F, h->Unext));
        CK(cudaStreamSynchronize(h->st));
        swap_state(h);
    }
}

pppc_status pppc_set_trace(pppc_handle* h, int32_t cap) {
    if (!h || cap < 0) return h ? fail(h, PPPC_ERR_INVALID_ARG, "cap must be >= 0") : PPPC_ERR_INVALID_ARG;
    if (!h->has_mesh) return fail(h, PPPC_ERR_STATE, "pppc_set_mesh has not been called");
    h->trace_cap = 0;
    if (cap == 0) return PPPC_OK;
    TRY(alloc_n(h, &h->trace, (size_t)cap * kTraceFields));
    TRY(alloc_n(h, &h->trace_len, 1));
    CK(cudaMemsetAsync(h->trace_len, 0, sizeof(int), h->st));
    h->trace_cap = cap;
    return PPPC_OK;
}

pppc_status pppc_get_trace(pppc_handle* h, double* out, int32_t cap, int32_t* n) {
    if (!h || !out || !n || cap < 0) return h ? fail(h, PPPC_ERR_INVALID_ARG, "null argument") : PPPC_ERR_INVALID_ARG;
    if (h->trace_cap == 0) return fail(h, PPPC_ERR_STATE, "tracing is off (pppc_set_trace)");
    int len = 0;
    CK(cudaMemcpyAsync(&len, h->trace_len, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    *n = len;
    const int k = std::min(std::min(len, cap), h->trace_cap);
    if (k > 0) CK(cudaMemcpy(out, h->trace, (size_t)k * kTraceFields * sizeof(double), cudaMemcpyDeviceToHost));
    return PPPC_OK;
}

pppc_status pppc_get_mesh_counts(pppc_handle* h, pppc_mesh_counts* out) {
    if (!h || !out) return PPPC_ERR_INVALID_ARG;
    if (!h->has_mesh) return fail(h, PPPC_ERR_STATE, "pppc_set_mesh has not been called");
    out->ndof = h->hm.ndof;
    out->nnz = h->hm.nnz;
    out->special_rows = h->hm.n_sp;
    out->special_entries = h->hm.n_slots;
    out->nonlinear_elems = h->hm.n_nl;
    return PPPC_OK;
}

pppc_status pppc_get_stats(pppc_handle* h, pppc_stats* out) {
    if (!h || !out) return PPPC_ERR_INVALID_ARG;
    *out = h->stats;
    return PPPC_OK;
}

pppc_status pppc_get_fine_plan(pppc_handle* h, pppc_fine_plan_info* out) {
    if (!h || !out) return PPPC_ERR_INVALID_ARG;
    if (!h->has_mesh) return fail(h, PPPC_ERR_STATE, "pppc_set_mesh has not been called");
    std::memset(out, 0, sizeof *out);
    const pppc_fine_plan& p = h->plan;
    const int V = h->fp32 ? 4 : 2;
    out->lanes_per_team = p.lanes;
    out->teams = p.teams;
    out->threads_per_row = p.lanes > 0 ? p.lanes / V : h->NB / V;
    if (p.lanes > 0) {
        out->blocks_min = *std::min_element(p.blocks.begin(), p.blocks.end());
        out->blocks_max = *std::max_element(p.blocks.begin(), p.blocks.end());
    } else if (p.lanes < 0) {
        out->blocks_min = out->blocks_max = h->fine_cfg.blocks;
    }
    const std::vector<int> cand = team_candidates(h);
    out->n_candidates = (int)cand.size();
    for (size_t c = 0; c < cand.size() && c < 16; ++c) {
        out->candidate_lanes[c] = cand[c];
        out->candidate_ms[c] = h->tune_ms[c];
    }
    out->amg_levels = h->amg_levels;
    for (int l = 0; l < h->amg_levels && l < 10; ++l) out->amg_rows[l] = h->amg_rows[l];
    return PPPC_OK;
}

}  // extern "C"

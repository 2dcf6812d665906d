// Many independent PP-PC problems at once (the batch calls of pppc.h).
//
// Each member is an ordinary handle (mesh, source, state, workspace).  A
// batch iteration is two captured CUDA graphs:
//   fine graph:   U -> F copies, one cooperative launch in which member c's
//                 fine sweep (Eqs. 2-3) runs on a team of fblocks[c] blocks,
//                 every member's jumps (Eq. 4, Eq. 7), a gather of the
//                 per-member control words and one copy of them to the host;
//   coarse graph: every member's K-bar and DFT right-hand side (Eqs. 11-13),
//                 one cooperative launch of all members' harmonic solves
//                 (team of cblocks[c] blocks each), every member's inverse
//                 DFT + update (Eq. 14) written in place into U, and the
//                 control words again.
// Between the two the host decides which members have converged.  Teams are
// sized by a greedy makespan split of the 152 SMs over the members' costs:
// first a model (rows x lanes x fine steps), then, with autotuning, the
// measured team times x team sizes.  Every change of teams or of the active
// set re-partitions the rows and captures both graphs again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pppc.h"
#include "args.h"
#include "handle.h"
#include "kernels.h"

using namespace pppc;
using namespace pppc::detail;

namespace {

thread_local std::string g_batch_create_error;

// Retune only when the re-split is predicted to shorten the launch by this.
constexpr double kRetuneGain = 0.9;
// A member's lane teams each expect at least this many blocks of the batch.
constexpr int kMinTeamBlocks = 8;

// Where member c's control words live, and what is gathered from them.
struct CtlSrc {
    const double* jsums;       // ||d||^2, ||F||^2
    const int* status;
    const long long* counters; // newton, pcg, cocg, backtracks
    const long long* team_ns;  // fine start, end, coarse start, end
};
struct CtlOut {
    double js0, js1;
    long long status;
    long long c[kCounters];   // the member's counters (kCnt*)
    long long t[4];
};

__global__ void gather_ctl_kernel(const CtlSrc* src, int count, CtlOut* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count) return;
    const CtlSrc s = src[c];
    CtlOut o;
    o.js0 = s.jsums[0];
    o.js1 = s.jsums[1];
    o.status = *s.status;
    for (int q = 0; q < kCounters; ++q) o.c[q] = s.counters[q];
    for (int q = 0; q < 4; ++q) o.t[q] = s.team_ns[q];
    out[c] = o;
}

}  // namespace

struct pppc_batch {
    std::vector<pppc_handle*> m;
    int count = 0;
    cudaStream_t user_st = nullptr;   // the members' stream
    cudaStream_t st = nullptr;        // the batch's own stream (graphs cannot capture the legacy stream)
    bool fp32 = false;
    bool autotune = true;
    std::string err;
    int sms = 0;
    size_t smem_optin = 0, fine_static = 0, cocg_static = 0;
    std::vector<void*> allocs;
    // device tables
    FineArgs* d_fargs = nullptr;
    CocgArgs* d_cargs = nullptr;
    int4* d_fmap = nullptr;
    int4* d_cmap = nullptr;
    long long* d_team_ns = nullptr;   // [count][4]
    CtlSrc* d_src = nullptr;
    CtlOut* d_ctl = nullptr;
    CtlOut* h_ctl = nullptr;          // pinned host copy
    // fine launch: every member's lane teams are units of their own
    std::vector<int> lanes, teams, unit_first;   // per member
    std::vector<int> unit_member;                // per unit
    int units = 0;
    long long* d_unit_ns = nullptr;   // [units][2] %globaltimer at a unit's start and end
    long long* h_unit_ns = nullptr;   // pinned copy
    // host state
    std::vector<int> fblocks, cblocks;   // fblocks per unit, cblocks per member
    std::vector<double> fcost, ccost;    // per unit / per member: time x blocks (model units until measured)
    std::vector<char> active;
    size_t fine_smem_launch = 0, cocg_smem_launch = 0;
    cudaGraphExec_t gfine = nullptr, gcoarse = nullptr;
    bool dirty = true;
    int fine_kernels = 0, coarse_kernels = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    pppc_batch_stats stats{};
};

namespace {

pppc_status bfail(pppc_batch* b, pppc_status s, const std::string& msg) {
    b->err = msg;
    return s;
}

#define BCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? PPPC_ERR_NOMEM : PPPC_ERR_CUDA,     \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

#define BTRY(expr)                     \
    do {                               \
        pppc_status s_ = (expr);       \
        if (s_ != PPPC_OK) return s_;  \
    } while (0)

// Batch tables come from the members' allocator (pppc_config.alloc of the
// first member, e.g. PyTorch's caching allocator), else cudaMalloc.
template <typename T>
pppc_status balloc(pppc_batch* b, T** out, size_t n) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    const pppc_config& c = b->m[0]->cfg;
    if (c.alloc) {
        p = c.alloc(bytes, c.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) return bfail(b, PPPC_ERR_NOMEM, "batch table allocation failed");
    b->allocs.push_back(p);
    *out = static_cast<T*>(p);
    return PPPC_OK;
}

// Greedy makespan split: every active member gets one block, then each
// further block goes to the member with the largest cost / blocks (below its
// cap).  Returns the predicted makespan max cost / blocks.
double split_blocks(const std::vector<double>& cost, const std::vector<char>& active, const std::vector<int>& cap,
                    int total, std::vector<int>& blocks) {
    const int n = (int)cost.size();
    blocks.assign(n, 0);
    int used = 0;
    for (int c = 0; c < n; ++c)
        if (active[c]) {
            blocks[c] = 1;
            ++used;
        }
    while (used < total) {
        int best = -1;
        double bv = -1.0;
        for (int c = 0; c < n; ++c)
            if (active[c] && blocks[c] < cap[c] && cost[c] / blocks[c] > bv) {
                bv = cost[c] / blocks[c];
                best = c;
            }
        if (best < 0) break;
        ++blocks[best];
        ++used;
    }
    double mk = 0.0;
    for (int c = 0; c < n; ++c)
        if (active[c]) mk = std::max(mk, cost[c] / blocks[c]);
    return mk;
}

int fine_cap(const pppc_handle* h, int lanes) {
    const int V = h->fp32 ? 4 : 2, RB = 1024 / (lanes / V);
    return std::max(1, h->hm.ndof / (2 * RB));
}

int cocg_cap(const pppc_handle* h) {
    const int RB = std::max(1, 512 / h->H);
    return std::max(1, h->hm.ndof / (2 * RB));
}

int4* team_map(int total, const std::vector<int>& blocks, std::vector<int4>& map) {
    map.assign(total, make_int4(-1, 0, 0, 0));
    int first = 0;
    for (int c = 0; c < (int)blocks.size(); ++c) {
        for (int k = 0; k < blocks[c]; ++k) map[first + k] = make_int4(c, k, blocks[c], 0);
        first += blocks[c];
    }
    return map.data();
}

}  // namespace

namespace {

void destroy_graphs(pppc_batch* b) {
    if (b->gfine) cudaGraphExecDestroy(b->gfine);
    if (b->gcoarse) cudaGraphExecDestroy(b->gcoarse);
    b->gfine = b->gcoarse = nullptr;
}

pppc_status end_capture(pppc_batch* b, cudaGraphExec_t* exec) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamEndCapture(b->st, &g));
    const cudaError_t e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    BCK(e);
    return PPPC_OK;
}

// Capture errors must end the capture before returning.
#define CAP(call)                                                  \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) {                                   \
            cudaGraph_t g_ = nullptr;                              \
            cudaStreamEndCapture(b->st, &g_);                      \
            if (g_) cudaGraphDestroy(g_);                          \
            cudaGetLastError();                                    \
            return bfail(b, PPPC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                          \
    } while (0)

// Partition rows for the current teams, upload every table and capture the
// two graphs for the current active set.
pppc_status rebuild(pppc_batch* b) {
    BCK(cudaStreamSynchronize(b->st));
    destroy_graphs(b);
    const int n = b->count, nu = b->units;
    std::vector<int> fcap(nu), ccap(n);
    std::vector<char> uactive(nu);
    for (int u = 0; u < nu; ++u) {
        const int c = b->unit_member[u];
        fcap[u] = fine_cap(b->m[c], b->lanes[c]);
        uactive[u] = b->active[c];
    }
    for (int c = 0; c < n; ++c) ccap[c] = cocg_cap(b->m[c]);
    split_blocks(b->fcost, uactive, fcap, b->sms, b->fblocks);
    split_blocks(b->ccost, b->active, ccap, b->sms, b->cblocks);

    // fine: one unit per lane team of every active member, each with the row
    // partition of its block count and shared-memory vectors where they fit
    std::vector<FineArgs> fa(nu);
    std::vector<CocgArgs> ca(n);
    b->fine_smem_launch = 0;
    b->cocg_smem_launch = 0;
    for (int c = 0; c < n; ++c) {
        pppc_handle* h = b->m[c];
        ca[c] = cocg_args(h);
        ca[c].team_ns = b->d_team_ns + 4 * (size_t)c + 2;
        const FineArgs base = fine_args(h, h->F);
        size_t part_off = 0;
        for (int t = 0; t < b->teams[c]; ++t) {
            const int u = b->unit_first[c] + t;
            if (!b->active[c]) {
                fa[u] = base;
                continue;
            }
            const pppc_row_tables* rt = nullptr;
            const pppc_status st = row_tables_for(h, b->fblocks[u], &rt);
            if (st != PPPC_OK) return bfail(b, st, "member " + std::to_string(c) + ": " + h->err);
            fa[u] = team_args(h, b->lanes[c], t, b->teams[c], b->fblocks[u], base, &part_off);
            fa[u].team_ns = b->d_unit_ns + 2 * (size_t)u;
            b->fine_smem_launch = std::max(b->fine_smem_launch,
                                           fine_smem(b->fp32, b->lanes[c], 1024, fa[u].vec_rows, fa[u].vec_w ? 4 : 3));
        }
        if (b->active[c]) b->cocg_smem_launch = std::max(b->cocg_smem_launch, cocg_smem_bytes(h->H, 512));
    }
    BCK(cudaMemcpyAsync(b->d_fargs, fa.data(), nu * sizeof(FineArgs), cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemcpyAsync(b->d_cargs, ca.data(), n * sizeof(CocgArgs), cudaMemcpyHostToDevice, b->st));
    std::vector<int4> fmap, cmap;
    team_map(b->sms, b->fblocks, fmap);
    team_map(b->sms, b->cblocks, cmap);
    BCK(cudaMemcpyAsync(b->d_fmap, fmap.data(), fmap.size() * sizeof(int4), cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemcpyAsync(b->d_cmap, cmap.data(), cmap.size() * sizeof(int4), cudaMemcpyHostToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));

    const int gblocks = (n + 127) / 128;
    // ---- fine graph
    b->fine_kernels = 0;
    BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    CAP(cudaMemsetAsync(b->d_team_ns, 0, 4 * (size_t)n * sizeof(long long), b->st));
    CAP(cudaMemsetAsync(b->d_unit_ns, 0, 2 * (size_t)nu * sizeof(long long), b->st));
    for (int c = 0; c < n; ++c) {
        if (!b->active[c]) continue;
        pppc_handle* h = b->m[c];
        CAP(cudaMemcpyAsync(h->F, h->U, (size_t)h->hm.ndof * h->NB * sizeof(double), cudaMemcpyDeviceToDevice,
                            b->st));
        CAP(cudaMemsetAsync(h->status, 0, sizeof(int), b->st));
        CAP(cudaMemsetAsync(h->bar, 0, kMaxTeams * sizeof(GridBarrier), b->st));
        CAP(reset_team_ctl(h, b->st));
    }
    CAP(launch_fine_batch(b->d_fargs, b->d_fmap, b->fp32, b->sms, b->fine_smem_launch, b->st));
    b->fine_kernels += 1;
    for (int c = 0; c < n; ++c) {
        if (!b->active[c]) continue;
        pppc_handle* h = b->m[c];
        launch_jumps(h->hm.ndof, h->N, h->NB, h->U, h->F, h->d, h->part, h->jsums, b->st);
        b->fine_kernels += 2;
    }
    gather_ctl_kernel<<<gblocks, 128, 0, b->st>>>(b->d_src, n, b->d_ctl);
    b->fine_kernels += 1;
    CAP(cudaGetLastError());
    CAP(cudaMemcpyAsync(b->h_ctl, b->d_ctl, n * sizeof(CtlOut), cudaMemcpyDeviceToHost, b->st));
    CAP(cudaMemcpyAsync(b->h_unit_ns, b->d_unit_ns, 2 * (size_t)nu * sizeof(long long), cudaMemcpyDeviceToHost,
                        b->st));
    BTRY(end_capture(b, &b->gfine));

    // ---- coarse graph
    b->coarse_kernels = 0;
    BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    for (int c = 0; c < n; ++c) {
        if (!b->active[c]) continue;
        pppc_handle* h = b->m[c];
        const int lin = h->cfg.coarse_lin;
        if (lin != PPPC_COARSE_ZERO_FIELD && h->md.n_nl > 0) {
            launch_elem_data(h->md, h->NB, h->cfg.coarse_at == PPPC_COARSE_AT_F ? h->F : h->U, h->elem, b->st);
            b->coarse_kernels += 1;
        }
        if (h->md.n_slots > 0) {
            launch_kbar(h->md, h->N, h->NB, lin, h->elem, h->Kbar, b->st);
            b->coarse_kernels += 1;
        }
        if (h->md.n_sp > 0) {
            launch_coarse_rhs(h->md, h->N, h->NB, h->H, 1.0 / h->dT, h->d, h->tw, h->y, h->b, b->st);
            b->coarse_kernels += 2;
        }
        CAP(cudaMemsetAsync(h->status, 0, sizeof(int), b->st));
        CAP(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), b->st));
    }
    CAP(cudaGetLastError());
    CAP(launch_cocg_batch(b->d_cargs, b->d_cmap, b->sms, b->cocg_smem_launch, b->st));
    b->coarse_kernels += 1;
    for (int c = 0; c < n; ++c) {
        if (!b->active[c]) continue;
        pppc_handle* h = b->m[c];
        // in place: the update reads only F and the harmonic solutions
        launch_idft_update(h->hm.ndof, h->N, h->NB, h->H, false, h->cx, h->F, h->tw, h->U, b->st);
        b->coarse_kernels += 1;
    }
    gather_ctl_kernel<<<gblocks, 128, 0, b->st>>>(b->d_src, n, b->d_ctl);
    b->coarse_kernels += 1;
    CAP(cudaGetLastError());
    CAP(cudaMemcpyAsync(b->h_ctl, b->d_ctl, n * sizeof(CtlOut), cudaMemcpyDeviceToHost, b->st));
    BTRY(end_capture(b, &b->gcoarse));
    b->dirty = false;
    return PPPC_OK;
}

// Read member statuses from the gathered control words; on a device error
// return it (device_status maps the code and records the message).
pppc_status check_members(pppc_batch* b, const char* where) {
    for (int c = 0; c < b->count; ++c) {
        if (!b->active[c] || b->h_ctl[c].status == 0) continue;
        pppc_handle* h = b->m[c];
        const pppc_status s = device_status(h, where);
        return bfail(b, s == PPPC_OK ? PPPC_ERR_CUDA : s, "member " + std::to_string(c) + ": " + h->err);
    }
    return PPPC_OK;
}

void update_member_stats(pppc_batch* b) {
    for (int c = 0; c < b->count; ++c) {
        pppc_stats& s = b->m[c]->stats;
        const long long* k = b->h_ctl[c].c;
        s.newton_iters = k[kCntNewton];
        s.pcg_iters = k[kCntPcg];
        s.cocg_iters = k[kCntCocg];
        s.backtracks = k[kCntBacktrack];
        s.pcg_lane_rounds = k[kCntPcgLaneRounds];
        s.pcg_lane_iters = k[kCntPcgLaneIters];
        s.newton_lane_rounds = k[kCntNewtonLaneRounds];
    }
}

// Online tuning: cost = measured team time x team size; re-split when the
// prediction beats the measured makespan by kRetuneGain.
void retune(pppc_batch* b, bool fine) {
    if (!b->autotune) return;
    std::vector<double>& cost = fine ? b->fcost : b->ccost;
    const std::vector<int>& blocks = fine ? b->fblocks : b->cblocks;
    const int items = fine ? b->units : b->count;
    double measured = 0.0;
    std::vector<double> next = cost;
    std::vector<char> act(items);
    for (int i = 0; i < items; ++i) {
        const int c = fine ? b->unit_member[i] : i;
        act[i] = b->active[c];
        if (!act[i] || blocks[i] < 1) continue;
        const long long t0 = fine ? b->h_unit_ns[2 * i] : b->h_ctl[c].t[2];
        const long long t1 = fine ? b->h_unit_ns[2 * i + 1] : b->h_ctl[c].t[3];
        if (t0 <= 0 || t1 < t0) return;   // no complete record: keep the teams
        const double t = (double)(t1 - t0);
        measured = std::max(measured, t);
        next[i] = t * blocks[i];
    }
    std::vector<int> cap(items), trial;
    for (int i = 0; i < items; ++i) {
        const int c = fine ? b->unit_member[i] : i;
        cap[i] = fine ? fine_cap(b->m[c], b->lanes[c]) : cocg_cap(b->m[c]);
    }
    const double predicted = split_blocks(next, act, cap, b->sms, trial);
    cost = next;
    if (predicted < kRetuneGain * measured && trial != blocks) {
        b->dirty = true;
        b->stats.retunes += 1;
    }
}

pppc_status run_graph(pppc_batch* b, bool fine) {
    BCK(cudaEventRecord(b->ev[fine ? 0 : 2], b->st));
    BCK(cudaGraphLaunch(fine ? b->gfine : b->gcoarse, b->st));
    BCK(cudaEventRecord(b->ev[fine ? 1 : 3], b->st));
    BCK(cudaStreamSynchronize(b->st));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, b->ev[fine ? 0 : 2], b->ev[fine ? 1 : 3]));
    (fine ? b->stats.fine_ms : b->stats.coarse_ms) += ms;
    b->stats.graph_launches += 1;
    b->stats.kernel_launches += fine ? b->fine_kernels : b->coarse_kernels;
    return PPPC_OK;
}

pppc_status begin_batch_call(pppc_batch* b) {
    BCK(cudaStreamSynchronize(b->user_st));   // the members' own work (states) comes first
    b->stats = pppc_batch_stats{};
    for (pppc_handle* h : b->m) {
        BCK(cudaMemsetAsync(h->counters, 0, kCounters * sizeof(long long), b->st));
        h->stats = pppc_stats{};
    }
    std::fill(b->active.begin(), b->active.end(), 1);
    b->dirty = true;   // member states may have been swapped by single-handle calls
    return PPPC_OK;
}

// One fine graph: fine sweeps and jumps of the active members; rr[c] = rel_res.
pppc_status fine_half(pppc_batch* b, std::vector<double>& rr) {
    if (b->dirty) BTRY(rebuild(b));
    BTRY(run_graph(b, true));
    BTRY(check_members(b, "fine propagators"));
    for (int c = 0; c < b->count; ++c) {
        if (!b->active[c]) continue;
        const CtlOut& o = b->h_ctl[c];
        if (!std::isfinite(o.js0) || !std::isfinite(o.js1))
            return bfail(b, PPPC_ERR_NAN, "member " + std::to_string(c) + ": non-finite jump norm");
        rr[c] = o.js1 > 0.0 ? std::sqrt(o.js0 / o.js1) : (o.js0 > 0.0 ? INFINITY : 0.0);
        const pppc_handle* h = b->m[c];
        b->stats.fine_dof_steps += (long long)h->N * h->cfg.n_fine * h->hm.ndof;
        b->m[c]->stats.rel_res = rr[c];
        b->m[c]->stats.fine_steps += h->cfg.n_fine;
    }
    update_member_stats(b);
    retune(b, true);
    return PPPC_OK;
}

pppc_status coarse_half(pppc_batch* b) {
    if (b->dirty) BTRY(rebuild(b));
    BTRY(run_graph(b, false));
    BTRY(check_members(b, "harmonic solves"));
    update_member_stats(b);
    for (int c = 0; c < b->count; ++c)
        if (b->active[c]) b->m[c]->stats.pppc_iters += 1;
    retune(b, false);
    return PPPC_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

const char* pppc_batch_last_error(pppc_batch* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

void pppc_batch_destroy(pppc_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    destroy_graphs(b);
    if (b->st) cudaStreamDestroy(b->st);
    for (void* p : b->allocs) {
        const pppc_config& c = b->m[0]->cfg;
        if (c.free_fn)
            c.free_fn(p, c.alloc_ctx);
        else
            cudaFree(p);
    }
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->h_unit_ns) cudaFreeHost(b->h_unit_ns);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

pppc_status pppc_batch_create(pppc_handle* const* members, int32_t count, int32_t autotune, pppc_batch** out) {
    auto reject = [](pppc_status s, const std::string& why) {
        g_batch_create_error = why;
        return s;
    };
    if (!out) return reject(PPPC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!members || count < 1) return reject(PPPC_ERR_INVALID_ARG, "members is NULL or count < 1");
    // argument errors first (NULL or repeated members), then the members' state
    for (int c = 0; c < count; ++c) {
        const std::string who = "member " + std::to_string(c);
        if (!members[c]) return reject(PPPC_ERR_INVALID_ARG, who + " is NULL");
        for (int d = 0; d < c; ++d)
            if (members[d] == members[c])
                return reject(PPPC_ERR_INVALID_ARG, who + " repeats member " + std::to_string(d));
    }
    for (int c = 0; c < count; ++c) {
        const pppc_handle* h = members[c];
        const std::string who = "member " + std::to_string(c);
        if (!h->has_mesh || !h->has_source) return reject(PPPC_ERR_STATE, who + " has no mesh or source");
        if (h->fp32 != members[0]->fp32) return reject(PPPC_ERR_UNSUPPORTED, who + ": precisions differ");
        if (h->st != members[0]->st) return reject(PPPC_ERR_UNSUPPORTED, who + ": streams differ");
        if (h->cfg.method != PPPC_METHOD_PPPC) return reject(PPPC_ERR_UNSUPPORTED, who + ": PP-IC is not batched");
        if (h->cfg.newton_schedule)
            return reject(PPPC_ERR_UNSUPPORTED, who + ": the inexact Newton schedule is not batched");
        const int V = h->fp32 ? 4 : 2, G = h->NB / V;
        if (G < 1 || (G & (G - 1)) != 0 || G > 1024)
            return reject(PPPC_ERR_UNSUPPORTED, who + ": lanes / vector width must be a power of two");
    }
    pppc_batch* b = new pppc_batch();
    b->m.assign(members, members + count);
    b->count = count;
    b->user_st = members[0]->st;
    b->fp32 = members[0]->fp32;
    b->autotune = autotune != 0;
    auto undo = [&](pppc_status s) {
        g_batch_create_error = b->err;
        pppc_batch_destroy(b);
        return s;
    };
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        b->err = "device query failed";
        return undo(PPPC_ERR_CUDA);
    }
    if (count > sms) {
        b->err = "at most one member per SM (" + std::to_string(sms) + ")";
        return undo(PPPC_ERR_UNSUPPORTED);
    }
    b->sms = sms;
    b->smem_optin = (size_t)optin;
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        b->st = nullptr;
        b->err = "stream creation failed";
        return undo(PPPC_ERR_CUDA);
    }
    if (fine_batch_prepare(b->fp32, &b->fine_static) != cudaSuccess ||
        cocg_batch_prepare(&b->cocg_static) != cudaSuccess) {
        cudaGetLastError();
        b->err = "batch kernels unavailable";
        return undo(PPPC_ERR_CUDA);
    }
    pppc_status s = PPPC_OK;
    auto take = [&](pppc_status r) {
        if (s == PPPC_OK) s = r;
    };
    // every member's lane split: its size bucket's tuned choice (the same
    // tuner as a single handle, timed on the member's state if its bucket has
    // none yet); splits are widened while the teams outnumber the SMs
    b->lanes.assign(count, 0);
    b->teams.assign(count, 1);
    for (int c = 0; c < count; ++c) {
        pppc_handle* h = members[c];
        int lanes = 0;
        const pppc_status ls = sweep_lanes(h, &lanes);
        if (ls != PPPC_OK) {
            b->err = "member " + std::to_string(c) + ": " + h->err;
            return undo(ls);
        }
        b->lanes[c] = lanes;
        b->teams[c] = h->NB / lanes;
    }
    // inside a batch a member gets only its share of the SMs (cost model):
    // its split is widened until every team can expect kMinTeamBlocks blocks
    {
        double sum = 0.0;
        for (int c = 0; c < count; ++c) sum += fine_cost_estimate(members[c]);
        for (int c = 0; c < count; ++c) {
            const double share = sms * fine_cost_estimate(members[c]) / sum;
            while (b->teams[c] > 1 && b->teams[c] * kMinTeamBlocks > share) {
                b->lanes[c] *= 2;
                b->teams[c] = members[c]->NB / b->lanes[c];
            }
        }
    }
    for (;;) {
        int total = 0, widest = -1;
        for (int c = 0; c < count; ++c) {
            total += b->teams[c];
            if (b->teams[c] > 1 && (widest < 0 || b->teams[c] > b->teams[widest])) widest = c;
        }
        if (total <= sms) break;
        if (widest < 0) {
            b->err = "more lane teams than SMs";
            return undo(PPPC_ERR_UNSUPPORTED);
        }
        b->lanes[widest] *= 2;
        b->teams[widest] = members[widest]->NB / b->lanes[widest];
    }
    b->unit_first.assign(count, 0);
    b->unit_member.clear();
    for (int c = 0; c < count; ++c) {
        b->unit_first[c] = (int)b->unit_member.size();
        for (int t = 0; t < b->teams[c]; ++t) b->unit_member.push_back(c);
    }
    b->units = (int)b->unit_member.size();
    take(balloc(b, &b->d_fargs, b->units));
    take(balloc(b, &b->d_cargs, count));
    take(balloc(b, &b->d_fmap, sms));
    take(balloc(b, &b->d_cmap, sms));
    take(balloc(b, &b->d_team_ns, 4 * (size_t)count));
    take(balloc(b, &b->d_unit_ns, 2 * (size_t)b->units));
    take(balloc(b, &b->d_src, count));
    take(balloc(b, &b->d_ctl, count));
    if (s != PPPC_OK) return undo(s);
    if (cudaMallocHost(&b->h_unit_ns, 2 * (size_t)b->units * sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        b->h_unit_ns = nullptr;
        b->err = "pinned host allocation failed";
        return undo(PPPC_ERR_NOMEM);
    }
    std::memset(b->h_unit_ns, 0, 2 * (size_t)b->units * sizeof(long long));
    if (cudaMallocHost(&b->h_ctl, count * sizeof(CtlOut)) != cudaSuccess) {
        cudaGetLastError();
        b->h_ctl = nullptr;
        b->err = "pinned host allocation failed";
        return undo(PPPC_ERR_NOMEM);
    }
    std::memset(b->h_ctl, 0, count * sizeof(CtlOut));
    for (auto& e : b->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
            b->err = "event creation failed";
            return undo(PPPC_ERR_CUDA);
        }
    std::vector<CtlSrc> src(count);
    for (int c = 0; c < count; ++c) {
        pppc_handle* h = members[c];
        src[c] = CtlSrc{h->jsums, h->status, h->counters, b->d_team_ns + 4 * (size_t)c};
    }
    if (cudaMemcpy(b->d_src, src.data(), count * sizeof(CtlSrc), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_team_ns, 0, 4 * (size_t)count * sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        b->err = "batch table upload failed";
        return undo(PPPC_ERR_CUDA);
    }
    b->fcost.resize(b->units);
    b->ccost.resize(count);
    for (int u = 0; u < b->units; ++u) {
        const int c = b->unit_member[u];
        b->fcost[u] = fine_cost_estimate(members[c]) / b->teams[c];
    }
    for (int c = 0; c < count; ++c) {
        // COCG: one complex row per harmonic, a few hundred iterations either way
        b->ccost[c] = (double)members[c]->hm.ndof * members[c]->H;
    }
    b->active.assign(count, 1);
    *out = b;
    return PPPC_OK;
}

pppc_status pppc_batch_iterate(pppc_batch* b, double* rel_res) {
    if (!b) return PPPC_ERR_INVALID_ARG;
    BTRY(begin_batch_call(b));
    std::vector<double> rr(b->count, 0.0);
    BTRY(fine_half(b, rr));
    BTRY(coarse_half(b));
    b->stats.iterations = 1;
    if (rel_res) std::copy(rr.begin(), rr.end(), rel_res);
    return PPPC_OK;
}

pppc_status pppc_batch_solve_periodic(pppc_batch* b, double tol, int32_t kmax, int32_t* iters, double* rel_res) {
    if (!b) return PPPC_ERR_INVALID_ARG;
    if (!(tol > 0.0) || kmax < 0) return bfail(b, PPPC_ERR_INVALID_ARG, "tol must be > 0 and kmax >= 0");
    BTRY(begin_batch_call(b));
    std::vector<double> rr(b->count, INFINITY);
    std::vector<int> its(b->count, 0);
    for (int k = 0;; ++k) {
        BTRY(fine_half(b, rr));
        b->stats.iterations = k + 1;
        bool any = false;
        for (int c = 0; c < b->count; ++c) {
            if (!b->active[c]) continue;
            if (rr[c] <= tol || k >= kmax) {
                its[c] = k;
                b->active[c] = 0;
                b->dirty = true;
            } else {
                any = true;
            }
        }
        if (!any) break;
        BTRY(coarse_half(b));
    }
    if (iters) std::copy(its.begin(), its.end(), iters);
    if (rel_res) std::copy(rr.begin(), rr.end(), rel_res);
    int missed = 0;
    for (int c = 0; c < b->count; ++c) missed += !(rr[c] <= tol);
    if (missed > 0)
        return bfail(b, PPPC_ERR_NOT_CONVERGED,
                     std::to_string(missed) + " member(s) above tol after " + std::to_string(kmax) + " updates");
    return PPPC_OK;
}

pppc_status pppc_batch_get_stats(pppc_batch* b, pppc_batch_stats* out) {
    if (!b || !out) return PPPC_ERR_INVALID_ARG;
    *out = b->stats;
    return PPPC_OK;
}

pppc_status pppc_batch_plan(const double* cost, const int32_t* cap, const int32_t* active, int32_t count,
                            int32_t total, int32_t* blocks, double* makespan) {
    if (!cost || !cap || !active || !blocks || count < 1) return PPPC_ERR_INVALID_ARG;
    std::vector<double> c(cost, cost + count);
    std::vector<int> cp(cap, cap + count), out;
    std::vector<char> act(count);
    int n_active = 0;
    for (int i = 0; i < count; ++i) {
        act[i] = active[i] != 0;
        if (act[i] && (!(c[i] > 0.0) || cp[i] < 1)) return PPPC_ERR_INVALID_ARG;
        n_active += act[i];
    }
    if (total < n_active) return PPPC_ERR_INVALID_ARG;
    const double mk = split_blocks(c, act, cp, total, out);
    for (int i = 0; i < count; ++i) blocks[i] = out[i];
    if (makespan) *makespan = mk;
    return PPPC_OK;
}

pppc_status pppc_batch_get_teams(pppc_batch* b, int32_t* fine_blocks, int32_t* cocg_blocks) {
    if (!b) return PPPC_ERR_INVALID_ARG;
    for (int c = 0; c < b->count; ++c) {
        int fb = 0;
        for (int t = 0; t < b->teams[c]; ++t) {
            const int u = b->unit_first[c] + t;
            fb += u < (int)b->fblocks.size() ? b->fblocks[u] : 0;
        }
        if (fine_blocks) fine_blocks[c] = fb;
        if (cocg_blocks) cocg_blocks[c] = c < (int)b->cblocks.size() ? b->cblocks[c] : 0;
    }
    return PPPC_OK;
}

pppc_status pppc_batch_get_lanes(pppc_batch* b, int32_t* lanes_per_team, int32_t* teams) {
    if (!b) return PPPC_ERR_INVALID_ARG;
    for (int c = 0; c < b->count; ++c) {
        if (lanes_per_team) lanes_per_team[c] = b->lanes[c];
        if (teams) teams[c] = b->teams[c];
    }
    return PPPC_OK;
}

}  // extern "C"

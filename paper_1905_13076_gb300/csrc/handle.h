// Internal: the handle behind the C ABI and the helpers that the batched
// driver (batch.cu) shares with the single-instance driver (api.cu).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/pppc.h"
#include "args.h"
#include "kernels.h"
#include "mesh_host.h"

// Row partition of the fine sweep for one team size (blocks), on the device.
struct pppc_row_tables {
    int* rs = nullptr;     // [blocks + 1] first row of each block
    int* ls = nullptr;     // [blocks + 1] ranges of lr per block
    int* lr = nullptr;     // long rows by owning block
    int rows_max = 0;
};

// How the fine sweep of one handle is split into lane teams: `teams` teams of
// `lanes` lanes each, team t on blocks[t] blocks; the per-team kernel
// arguments (rebuilt per sweep) and the block -> (team, block in team, team
// size) map live on the device.
struct pppc_fine_plan {
    int lanes = 0, teams = 0;
    std::vector<int> blocks;
    size_t smem = 0;
};

struct pppc_handle {
    using HostMesh = pppc::HostMesh;
    using MeshDev = pppc::MeshDev;
    using GridBarrier = pppc::GridBarrier;
    using LaunchCfg = pppc::LaunchCfg;
    using SourceDev = pppc::SourceDev;
    pppc_config cfg{};
    cudaStream_t st = nullptr;
    std::string err;
    bool has_mesh = false, has_source = false;
    int N = 0, NB = 0, H = 0;
    double dt = 0.0, dT = 0.0;
    bool fp32 = false;
    HostMesh hm;
    std::vector<void*> allocs;   // everything allocated for the current mesh
    MeshDev md{};
    int* d_node_of_dof = nullptr;
    int* d_dof_of_node = nullptr;
    int* d_row_start = nullptr;     // [fine blocks + 1] rows owned by each block of the fine sweep
    int* d_long_start = nullptr;    // [fine blocks + 1]
    int* d_long_rows = nullptr;     // rows with more than 32 nonzeros, by owning block
    int vec_rows = 0;               // > 0: fine-sweep vectors p, s, x kept in shared memory
    int vec_w = 0;                  // 1: and w
    // lane vectors [ndof][NB]
    double *U = nullptr, *Unext = nullptr, *F = nullptr, *uprev = nullptr, *d = nullptr;
    double* elem = nullptr;
    void *r = nullptr, *z = nullptr, *w = nullptr, *p = nullptr, *s = nullptr, *x = nullptr, *dx = nullptr,
         *J = nullptr, *invd = nullptr;
    // coarse
    double *y = nullptr, *b = nullptr, *Kbar = nullptr, *tw = nullptr;
    void *cx = nullptr, *cr = nullptr, *cz = nullptr, *cw = nullptr, *cp = nullptr, *cs = nullptr, *cinvd = nullptr;
    // reductions and control
    double *part = nullptr, *jsums = nullptr, *scalars = nullptr;
    GridBarrier* bar = nullptr;     // [kMaxTeams]: one per lane team (bar[0] for every other launch)
    int* status = nullptr;
    long long* counters = nullptr;
    long long* team_ctl = nullptr;  // [4]: max over teams of Newton / PCG rounds, teams done (per sweep)
    // lane teams of the fine sweep
    pppc_fine_plan plan;            // the plan in use (lanes == 0: not chosen yet)
    std::map<int, pppc_row_tables> row_tables;   // by team size
    pppc::FineArgs* d_team_args = nullptr;   // [kMaxTeams]
    int4* d_team_map = nullptr;        // [SMs]
    int sms = 0;
    size_t fine_static_smem = 0, smem_optin = 0;
    double tune_ms[16] = {0};          // tuner: time of each candidate (lanes = V * 2^i), 0 if not timed
    // multigrid preconditioner of the fine PCG (precond = 2)
    pppc::AmgLevel* d_amg = nullptr;   // [amg_levels] level descriptors (device)
    int amg_levels = 0;                // 0: none (precond != 2, or the mesh is too small to coarsen)
    long long amg_units = 0;           // workspace per team, in units of the team's lanes
    void* amg_ws = nullptr;            // [amg_units * NB] of T
    std::vector<int> amg_rows;         // rows per level
    // one PP-PC iteration as a captured CUDA graph (PP-PC method, no trace):
    // run on gst; per-iteration inputs {Newton tolerance, commit threshold}
    // from pinned ctl_in, the control block back into pinned ctl_out
    cudaStream_t gst = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t gev = nullptr;         // end of a graph launch (timing fallback)
    bool graph_dirty = true;
    double* ctl_in = nullptr;          // pinned [2]
    double* d_ctl_in = nullptr;        // device [2]
    pppc::IterCtl* ctl_out = nullptr;  // pinned
    pppc::IterCtl* d_ctl = nullptr;    // device
    pppc::FineArgs* d_graph_args = nullptr;   // [kMaxTeams] the graph's own team arguments
    int4* d_graph_map = nullptr;
    int graph_kernels = 0;
    // the same hierarchy preconditioning the harmonic solves: two lanes per harmonic
    void *camg_ws = nullptr, *camg_J = nullptr, *camg_r = nullptr, *camg_z = nullptr;
    double* ext = nullptr;   // [N][n_nodes] staging for host states
    double* trace = nullptr; // Newton trace of the fine sweep (optional)
    int* trace_len = nullptr;
    int trace_cap = 0;
    LaunchCfg fine_cfg, cocg_cfg, cocg1_cfg;
    // PP-IC: end-of-period state U_N (and its next value), sweep increment, shift 1 "twiddle"
    double *UN = nullptr, *UNnext = nullptr, *dcur = nullptr, *tw_c1 = nullptr;
    bool coarse_fp32 = false;       // the harmonic solves run in FP64 in both precisions
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    SourceDev src{};
    double gnorm = 0.0, src_area = 0.0;
    pppc_stats stats{};
    double rr_prev = INFINITY;   // rel_res of the previous iteration (inexact PP-PC schedule)
    int* d_tri_low = nullptr;    // tridiagonal-chunk preconditioner: CSR index of (i, i-1)
    double* uprev2 = nullptr;    // quadratic predictor: u^{m-2}
    void *tri_m = nullptr, *tri_ie = nullptr;
    // per nonlinear element: its region; per region: sigma (for the adjoint)
    std::vector<int> nl_region;
    std::vector<double> region_sigma;
    std::vector<int> region_kind;
    // adjoint workspace (allocated at the first pppc_adjoint)
    double *traj = nullptr, *lam = nullptr, *adjA = nullptr, *adjB = nullptr, *adjF = nullptr;
    double *gpart = nullptr, *gout = nullptr;
    unsigned char* nl_sel = nullptr;
};

namespace pppc {
namespace detail {

// Record msg as h's last error and return s.
pppc_status fail(pppc_handle* h, pppc_status s, const std::string& msg);
// Synchronise h's stream and map h's device status word to a pppc_status.
pppc_status device_status(pppc_handle* h, const char* where);
// Arguments of h's fine sweep writing F into Fout, as one team over all
// lanes with h's own row partition (callers may replace the partition fields).
FineArgs fine_args(pppc_handle* h, double* Fout);
// Zero h's per-sweep team control words (sweep maxima, teams done) on stream st.
cudaError_t reset_team_ctl(pppc_handle* h, cudaStream_t st);
// Arguments of lane team t (lanes lanes from lane t * lanes, one of `teams`)
// of the sweep `base` on nb blocks: its regions of the PCG vectors, partial
// sums (at *part_off, advanced) and multigrid workspace, its barrier and the
// row partition for nb blocks (row_tables_for must have built it).
FineArgs team_args(pppc_handle* h, int lanes, int t, int teams, int nb, const FineArgs& base, size_t* part_off);
// The row partition of h's fine sweep over nb blocks, built on first use.
pppc_status row_tables_for(pppc_handle* h, int nb, const pppc_row_tables** out);
// Lanes per team of h's fine sweep: the handle's plan, chosen (by the tuner
// with pppc_config.lane_team = 0, from the handle's state) if not yet.
pppc_status sweep_lanes(pppc_handle* h, int* lanes);
// Arguments of h's batched harmonic solve (Eq. 13).
CocgArgs cocg_args(pppc_handle* h);
// Stages of one iteration on h's stream: mesh and source present; control
// words reset; jumps d = F - U into h->d with rel_res; Kbar frozen at the
// lanes of `state`; harmonic correction Unew = F (shifted) + IDFT(W).
pppc_status stage_ready(pppc_handle* h);
pppc_status stage_reset(pppc_handle* h);
pppc_status stage_jumps(pppc_handle* h, const double* Ul, const double* Fl, double* rel_res);
pppc_status stage_kbar(pppc_handle* h, const double* state);
pppc_status stage_correct(pppc_handle* h, const double* Fl, double* Unew);
// Contiguous row ranges for nb blocks of about equal cost (nonzeros;
// per-lane rows count double; long rows carry a fixed extra cost): rs[nb+1];
// the long rows grouped by owning block, ls[nb+1] indexing lrows.
void partition_rows(const HostMesh& hm, int nb, std::vector<int>& rs, std::vector<int>& ls,
                    std::vector<int>& lrows, int* rows_max);
// Estimated cost of one fine sweep of h relative to other handles:
// partition cost x lanes x fine steps.
double fine_cost_estimate(const pppc_handle* h);
// Rows of p, s, x (and w) per block that fit in `budget` bytes of dynamic
// shared memory next to the fine kernel's scratch (0: none).
void choose_vec_rows(bool fp32, int NB, int rows_max, size_t budget, int* vec_rows, int* vec_w);

}  // namespace detail
}  // namespace pppc

// Error plumbing of the handle-based calls: a failing CUDA call records its
// text on h and returns PPPC_ERR_CUDA (PPPC_ERR_NOMEM for allocations); a
// failing stage returns its status.  Both expect a pppc_handle* h in scope.
#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(h, e_ == cudaErrorMemoryAllocation ? PPPC_ERR_NOMEM : PPPC_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

#define TRY(expr)                      \
    do {                               \
        pppc_status s_ = (expr);       \
        if (s_ != PPPC_OK) return s_;  \
    } while (0)

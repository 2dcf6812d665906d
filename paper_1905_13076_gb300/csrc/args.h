// Plain-old-data argument blocks shared by the host driver and the kernels.
// All device pointers are owned by the handle (api.cu); kernels never free.
#pragma once
#include <stdint.h>

namespace pppc {

constexpr int kMaxHarm = 16;        // harmonics of the impressed current
constexpr int kMaxLanes = 1024;     // N (subintervals) upper bound

// Device status codes (mirrors pppc_status; 0 = ok).
enum DevStatus : int {
    DEV_OK = 0,
    DEV_ERR_NEWTON = 4,
    DEV_ERR_LINEAR = 5,
    DEV_ERR_BREAKDOWN = 6,
    DEV_ERR_NAN = 7,
    DEV_ERR_TIMEOUT = 8,
    DEV_ERR_GEOMETRY = 100,   // zero-area or non-finite triangle (set_mesh)
};

// Grid-barrier words, zeroed before every cooperative launch.
struct GridBarrier {
    unsigned int flip;   // plain barrier: the top bit flips once all blocks have arrived
    unsigned int count;  // reducing barrier: arrivals so far
    unsigned int gen;    // reducing barrier: released generations
    unsigned int pad;
};

// Sparse structure and constant values of one mesh (Sec. 2, Eq. 1).
// Rows/columns are free nodes ("dofs").  "Special" rows touch a nonlinear or
// conductive element; their matrix values differ per lane (fine Jacobian) or
// per harmonic (coarse systems) and are stored per "slot" = position of an
// entry among the special rows' entries: slot = row_slot[i] + (k - rowptr[i]).
struct MeshDev {
    int ndof, nnz, n_slots, n_sp, n_nl;
    const int* rowptr;     // [ndof+1]
    const int* col;        // [nnz]
    const int* diag_k;     // [ndof] CSR index of the diagonal entry
    const int* row_slot;   // [ndof] first slot of a special row, -1 otherwise
    const int* sp_index;   // [ndof] index among special rows, -1 otherwise
    const int* sp_rows;    // [n_sp] special rows, ascending
    const int* slot_k;     // [n_slots] CSR index of each slot
    const double* Klin;    // [nnz] stiffness of the linear-material elements
    const float* Klin32;   // [nnz] same, FP32 (mixed precision)
    const double* invdiag_lin;   // [ndof] 1 / Klin(diag) (used on non-special rows)
    const float* invdiag_lin32;  // [ndof]
    const double* Mslot;   // [n_slots] conductivity matrix on the special rows
    const double* g;       // [ndof] source shape (sums to 1)
    const double* dlin;    // [ndof] K_lin row sums = -(couplings to Dirichlet nodes)
    // nonlinear (Brauer) elements
    const int* nl_dofs;    // [n_nl*3] vertex dofs, -1 on the Dirichlet boundary
    const double* nl_geom; // [n_nl*8] area, gx0, gy0, gx1, gy1, gx2, gy2, pad
    const double* nl_k;    // [n_nl*4] k1, k2, k3, cap on |B|^2 (infinite: none)
    const int* nlc_ptr;    // [n_slots+1] nonlinear contributions of each slot
    const int* nlc;        // packed e*9 + a*3 + b  (e: nonlinear element index)
    const double* nlc_ab;  // grad N_a . grad N_b of that element
};

struct SourceDev {
    int n_harm;
    double amp[kMaxHarm];
    double freq[kMaxHarm];
    double phase[kMaxHarm];
};

// Per-lane element data of the nonlinear elements (5 planes of n_nl*NB):
// c1 = area*nu, c2 = 2*area*dnu/d(B^2), s_a = grad N_a . grad A  (a = 0,1,2)
constexpr int kElemPlanes = 5;

// One level of the fine PCG's multigrid preconditioner (precond = 2; setup
// in amg_host.cpp).  Level 0 is the fine Newton matrix itself (the mesh's
// CSR, per-lane special rows in FineArgs::J, shared rows K_lin); levels l >= 1
// hold A_l = P_l^T A_{l-1} P_l for every lane: shared values on ordinary
// rows, per-lane slots on special rows, rebuilt per Newton iteration as
// slot_base + sum cw * (finer slots).  Vectors of a team live in its
// workspace FineArgs::amg_ws at offsets given in units of the team's lanes.
constexpr int kAmgMaxLevels = 10;
struct AmgLevel {
    int n, n_slots, n_sp, pad;
    long long off_b, off_y, off_q, off_slot, off_l1;   // workspace offsets (x team lanes); -1 unused
    const int* rowptr;         // l >= 1: pattern of A_l
    const int* col;
    const void* val;           // [nnz] shared values (T)
    const int* row_slot;       // [n] first per-lane slot of a special row, -1 otherwise
    const int* sp_index;       // [n] index among special rows, -1 otherwise
    const int* sp_rows;        // [n_sp]
    const void* l1;            // [n] sum_j |A_l(i, j)| on shared rows (T)
    const int* Pptr;           // l >= 1: P_l, rows of level l - 1
    const int* Pcol;
    const void* Pval;
    const int* Rptr;           // l >= 1: R_l = P_l^T, rows of level l
    const int* Rcol;
    const void* Rval;
    const void* slot_base;     // l >= 1: [n_slots] (T)
    const int* cptr;           // [n_slots + 1]
    const int* csrc;           // slots of level l - 1
    const void* cw;            // (T)
    const long long* cost;     // l >= 1: [n + 1] prefix of the rows' V-cycle work (amg_host.h)
};

// Arguments of the fine sweep of one lane team: the NB lanes lane0 ..
// lane0 + NB - 1 of a problem with N lanes.  The FP64 state vectors (u,
// uprev, uprev2, traj*, lam_out) and the element planes are shared by all
// teams, [row][ld] with ld the problem's padded lane count, and are passed
// un-offset (the kernel adds lane0).  The PCG vectors (r, z, w, p, s, x, dx,
// J, invd_sp, tri_m, tri_ie) and the partial sums are the team's own,
// [row][NB], already offset to the team's region.
struct FineArgs {
    MeshDev mesh;
    SourceDev src;
    int N, NB, n_fine;       // N: the problem's lanes; NB: this team's lanes;
                             // n_fine: implicit-Euler steps this launch marches per lane
    int ld, lane0;           // row stride of the state vectors; first lane of the team
    int level0, n_total;     // first level of that window and levels per subinterval
                             // (lane l's step s ends at t = (l n_total + level0 + s + 1) dt)
    double dt, inv_dt;
    double tol_abs;          // Newton stop on ||R||_2 per lane
    const double* tol_abs_dev; // if not null: read the Newton stop from here at launch (captured graphs)
    double tol_lin;          // smallest PCG forcing term
    int max_newton, max_lin;
    double* u;               // [ndof*NB] Newton state in, F_n out (FP64)
    double* uprev;           // [ndof*NB]
    double* elem;            // [5*n_nl*NB]
    void* r; void* z; void* w; void* p; void* s;   // [ndof*NB] of T
    void* x;                 // [ndof*NB] of T: the Newton correction being solved for
    void* dx;                // [ndof*NB] of T: each lane's last accepted Newton step (for backtracking)
    double eta0;             // PCG forcing term of the first Newton iteration of a step
    int predictor;           // 1: start each step's Newton from 2 u^m - u^{m-1}; 2: 3 u^m - 3 u^{m-1} + u^{m-2}
    double* uprev2;          // predictor 2: [ndof*NB] u^{m-2}
    void* J;                 // [n_slots*NB] of T
    void* invd_sp;           // [n_sp*NB] of T
    void* part;              // [2][gridDim][3 * NB] per-block partial sums of type T
    const int* row_start;    // [gridDim + 1] first row owned by each block
    const int* long_start;   // [gridDim + 1] ranges of long_rows per block
    const int* long_rows;    // rows with more than 32 nonzeros, grouped by owning block
    int vec_rows;            // > 0: p, s, x of each block's rows kept in shared memory
    int vec_w;               // 1: w as well
    GridBarrier* bar;
    int* status;
    long long* counters;     // [kCounters], see kCounter* below (shared by the teams of a sweep)
    long long* sweep_max;    // [2] per launch, zeroed before it: max over teams of Newton / PCG rounds
    unsigned int* teams_done;// per launch, zeroed before it: teams that finished
    int n_teams;             // teams in this launch (the last one adds sweep_max into counters)
    double* trace;           // optional [trace_cap * kTraceFields] Newton records, or null
    int trace_cap;
    int* trace_len;          // records written (may exceed trace_cap; extra ones dropped)
    long long* team_ns;      // optional [2]: %globaltimer at the team's start and end
    // forward: optional record of every fine level; adjoint mode (see fine.cu)
    double* traj_out;        // forward: [n_fine+1][ndof][NB] u at levels 0..n_fine of each lane, or null
    int adjoint;             // 1: each lane runs its subinterval's periodic adjoint backwards
    const double* traj;      // adjoint: the forward trajectory, layout of traj_out
    double* lam_out;         // adjoint: [n_fine][ndof][NB] lambda at levels 1..n_fine, or null
    double tol_rel;          // adjoint: a level is solved when ||R|| <= tol_rel ||b||
    double g_scale;          // adjoint: 2 / (T dt), the loss weight of the adjoint source
    // preconditioner: 0 = Jacobi; c > 0 = tridiagonal blocks of c consecutive rows
    int tri;
    const int* tri_low;      // [ndof] CSR index of entry (i, i-1), -1 if absent
    void* tri_m;             // [ndof*NB] of T: LDL^T multipliers of the chunk factorisation
    void* tri_ie;            // [ndof*NB] of T: inverse pivots
    // multigrid preconditioner (amg != null): levels, l1-Jacobi sweeps on the
    // coarsest level, and this team's workspace (T)
    const AmgLevel* amg;
    int amg_levels, amg_sweeps;
    void* amg_ws;
};

// Device counters of a handle, accumulated over the sweeps of one call.
constexpr int kCounters = 8;
constexpr int kCntNewton = 0;        // Newton rounds (lockstep per team), max over teams, summed over sweeps
constexpr int kCntPcg = 1;           // PCG rounds, same
constexpr int kCntCocg = 2;          // COCG iterations (lockstep over the harmonics)
constexpr int kCntBacktrack = 3;     // Newton rounds in which some lane backtracked, summed over teams
constexpr int kCntPcgLaneRounds = 4; // sum over teams of PCG rounds x team lanes (lane-vectors streamed)
constexpr int kCntPcgLaneIters = 5;  // sum over lanes of the PCG iterations that lane needed
constexpr int kCntNewtonLaneRounds = 6;  // sum over teams of Newton rounds x team lanes
constexpr int kMaxTeams = 256;       // lane teams of one sweep (at most one block each)

// Control block of one captured PP-PC iteration, gathered on the device and
// copied to pinned host memory by the graph's last node.
struct IterCtl {
    long long status;
    double jsums[2];              // ||d||^2, ||F||^2
    long long counters[kCounters];
};

// One record per Newton test of the fine sweep:
// step, Newton iteration, max over lanes of ||R||_2, lanes still iterating,
// PCG iterations of the solve that preceded this test.
constexpr int kTraceFields = 5;

struct CocgArgs {
    MeshDev mesh;
    int N, H;                // H = N/2 + 1 harmonic lanes
    double inv_dT;
    double tol;              // relative tolerance per harmonic
    int max_it;
    const double* Kbar;      // [n_slots] coarse stiffness on special rows
    const double* tw;        // [2*N] exp(-i 2 pi k / N)
    const double* b;         // [n_sp*H*2] right-hand side (nonzero only on special rows)
    void* x; void* r; void* z; void* w; void* p; void* s;  // [ndof*H] complex T
    void* invd_sp;           // [n_sp*H] complex T
    double* part;            // [2][gridDim][5 * H] per-block partial sums
    GridBarrier* bar;
    int* status;
    long long* counters;     // [2] cocg iterations
    long long* team_ns;      // optional [2]: %globaltimer at the team's start and end
    // multigrid preconditioner (amg != null, single-problem launches): for
    // harmonic p the real SPD matrix S_p = Kbar + |1 - z_p| C, its V-cycle
    // (the fine PCG's hierarchy with S_p's Galerkin coarse matrices) applied
    // to the real and imaginary parts alike -- a real symmetric, hence
    // complex-symmetric, preconditioner as COCG requires.  The V-cycle runs in
    // the fine PCG's precision P on two lanes per harmonic ([row][2H] of P).
    const AmgLevel* amg;
    int amg_levels, amg_sweeps, amg_fp32;
    void* amg_ws;            // [units][2H] of P
    void* amg_J;             // [n_slots][2H] of P: S_p on the special rows
    void* amg_r;             // [ndof][2H] of P: r converted for the V-cycle
    void* amg_z;             // [ndof][2H] of P
    const void* klinP;       // K_lin in P
    const int* row_start;    // [gridDim + 1] contiguous rows of each block (the V-cycle's fine rows)
    const int* long_start;
    const int* long_rows;
};

}  // namespace pppc

// Host-side setup of the algebraic multigrid preconditioner of the fine PCG
// (pppc_config.precond = 2).
//
// The fine Newton matrix of every subinterval ("lane") is
//     J = K_lin + M / dt + J_nl(u_lane),
// identical across lanes except on the rows that touch a nonlinear or
// conductive element (the "special" rows, whose values the fine sweep keeps
// per lane).  The hierarchy is smoothed aggregation built once from a
// representative matrix A0 (J at zero field): aggregates, tentative and
// smoothed prolongators P_l and the Galerkin matrices A_l = P_l^T A_{l-1} P_l.
// Each lane's own coarse matrices are then P_l^T J_{l-1} P_l with the fixed
// P_l: they differ from A0's only on "special" coarse rows (those that some
// special finer row prolongs into), and each of their per-lane entries is
// a fixed linear combination of the finer level's per-lane entries,
//     slot_l[e] = slot_base[e] + sum_c cw[c] * slot_{l-1}[csrc[c]],
// which this setup tabulates so that the device rebuilds every lane's
// hierarchy with one gather per level and Newton iteration.
//
// Integer and FP64 host work at pppc_set_mesh time; no GPU.
#pragma once
#include <string>
#include <vector>

namespace pppc {

struct AmgHostLevel {
    int n = 0;                      // rows (= columns) of A_l
    std::vector<int> rowptr, col;   // pattern, columns sorted within a row
    std::vector<double> val;        // A_l of the representative matrix
    std::vector<int> row_slot;      // per-lane slots of a special row start here; -1 otherwise
    std::vector<int> sp_index;      // index among the special rows, -1 otherwise
    std::vector<int> sp_rows;       // the special rows, ascending
    int n_slots = 0, n_sp = 0;
    std::vector<double> l1;         // sum_j |A_l(i, j)| (the l1 smoother's diagonal on shared rows)
    // l >= 1: prolongation P_l (n_{l-1} x n_l) and restriction R_l = P_l^T (n_l x n_{l-1})
    std::vector<int> Pptr, Pcol, Rptr, Rcol;
    std::vector<double> Pval, Rval;
    // l >= 1: per-lane slot e = slot_base[e] + sum_{c in [cptr[e], cptr[e+1])} cw[c] * (slot csrc[c] of level l-1)
    std::vector<double> slot_base;
    std::vector<int> cptr, csrc;
    std::vector<double> cw;
    // l >= 1: [n + 1] prefix sums of each row's work in one V-cycle, so that
    // a team can split the level into equal shares of work:
    // cost(c) = 2 nnz_A(c) (1 + [c special]) + nnz_R(c) + nnz_P(l+1)(c) + 4
    // (two residual passes, which also read per-lane values on a special
    // row; the restriction; the prolongation from level l + 1; per-row
    // loads and stores).  Strictly increasing from cost[0] = 0.
    std::vector<long long> cost;
};

struct AmgOptions {
    double theta = 0.08;      // strength of connection: |a_ij| >= theta sqrt(|a_ii a_jj|)
    int max_levels = 10;      // including the fine level
    int coarse_rows = 400;    // stop coarsening once a level has at most this many rows
    double min_ratio = 0.85;  // stop when a level would keep more than this share of the rows
};

// Builds the hierarchy.  Input: the fine pattern (n rows, rowptr, col sorted
// within rows), the representative values val (symmetric positive definite),
// and the fine special rows (row_slot >= 0, slots of row i contiguous from
// row_slot[i] in column order).  levels[0] describes the fine level (its
// values are A0; the device takes the fine per-lane values from the Jacobian
// itself).  Returns false with a message if the input is malformed.
bool build_amg(int n, const int* rowptr, const int* col, const double* val, const int* row_slot,
               const AmgOptions& opt, std::vector<AmgHostLevel>& levels, std::string& err);

}  // namespace pppc

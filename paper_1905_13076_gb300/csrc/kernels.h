// Launchers of the device kernels, called by the C-ABI driver (api.cu).
#pragma once
#include <cuda_runtime.h>

#include "args.h"

namespace pppc {

// ---- setup.cu: matrices of Eq. 1 from the mesh ---------------------------
struct SetupArgs {
    int n_tri, ndof, nnz, n_slots, n_nl, n_nlc, n_regions, N;
    const double* xy;          // [2*n_nodes]
    const int* tri;            // [3*n_tri]
    const int* region;         // [n_tri]
    const double* mat;         // [n_regions*8] sigma, nu_model, nu, k1, k2, k3, is_source, 0
    const int* contrib_ptr;    // [nnz+1]
    const int* contrib;        // packed tri*9 + a*3 + b
    const int* rowptr;
    const int* diag_k;
    const int* slot_k;
    const int* nl_elems;       // [n_nl]
    const int* nlc;            // packed q*9 + a*3 + b
    const int* dcoup_ptr;      // [ndof+1]
    const int* dcoup;          // packed tri*9 + a*3 + b, vertex b on the Dirichlet boundary
    double* geom;              // [n_tri*8] scratch: area, gx0, gy0, gx1, gy1, gx2, gy2
    double* Klin;
    float* Klin32;
    double* invdiag_lin;
    float* invdiag_lin32;
    double* Mslot;
    double* g;
    double* dlin;
    double* nl_geom;
    double* nl_k;
    double* nlc_ab;
    double* tw;                // [2*N]
    double* scalars;           // [2]: discrete source area, ||g||_2
    int* status;
};
cudaError_t launch_setup(const SetupArgs& a, cudaStream_t st);

// ---- fine.cu: batched fine propagators (Eqs. 2-3) ------------------------
struct LaunchCfg {
    int blocks = 0, threads = 0;
    size_t smem = 0;
};
// vec_rows > 0: each block keeps p, s, x (vec_count 3) or p, s, x, w (4) of up
// to vec_rows rows in shared memory
cudaError_t fine_config(bool fp32, int NB, int vec_rows, int vec_count, LaunchCfg* cfg);
size_t fine_smem(bool fp32, int NB, int threads, int vec_rows, int vec_count);
cudaError_t launch_fine_sweep(const FineArgs& a, bool fp32, const LaunchCfg& cfg, cudaStream_t st);
// Batched fine sweep: `blocks` blocks of 1024 threads; args[] and map[blocks]
// (member, team block, team size, unused) in device memory.
// fine_batch_prepare lifts the dynamic shared-memory limit to the device
// maximum and reports the kernel's static shared memory.
cudaError_t fine_batch_prepare(bool fp32, size_t* static_smem);
cudaError_t launch_fine_batch(const FineArgs* args, const int4* map, bool fp32, int blocks, size_t smem,
                              cudaStream_t st);
// element data (c1, c2, s_a) of the nonlinear elements at the lanes of u
void launch_elem_data(const MeshDev& m, int NB, const double* u, double* elem, cudaStream_t st);

// ---- coarse.cu: jumps, coarse linearisation, DFT, COCG, IDFT + update ----
// d = F(shifted) - U, per-block partial sums of |d|^2 and |F|^2 -> sums[2]
void launch_jumps(int ndof, int N, int NB, const double* U, const double* F, double* d,
                  double* part, double* sums, cudaStream_t st);
void launch_kbar(const MeshDev& m, int N, int NB, int lin, const double* elem, double* Kbar,
                 cudaStream_t st);
void launch_coarse_rhs(const MeshDev& m, int N, int NB, int H, double inv_dT, const double* d,
                       const double* tw, double* y, double* b, cudaStream_t st);
cudaError_t cocg_config(bool fp32, int H, LaunchCfg* cfg);
cudaError_t launch_cocg(const CocgArgs& a, bool fp32, const LaunchCfg& cfg, cudaStream_t st);
size_t cocg_smem_bytes(int H, int threads);   // dynamic shared memory of one COCG block
// Batched FP64 COCG: `blocks` blocks of 512 threads; args[] and map[blocks] as
// for the batched fine sweep.
cudaError_t cocg_batch_prepare(size_t* static_smem);
cudaError_t launch_cocg_batch(const CocgArgs* args, const int4* map, int blocks, size_t smem, cudaStream_t st);
// PP-IC coarse sweep (Eq. 5): start, right-hand side C v, one step n
void launch_ppic_start(int ndof, int NB, const double* U, const double* UN, double* dcur, double* Unew,
                       cudaStream_t st);
void launch_ppic_rhs(const MeshDev& m, double inv_dT, const double* v, double* b, cudaStream_t st);
void launch_ppic_step(int ndof, int N, int NB, int n, const double* F, const double* U, const double* UN,
                      const double* x, double* dcur, double* Unew, double* UNnew, cudaStream_t st);
void launch_zero_pad_lanes(int ndof, int N, int NB, double* U, cudaStream_t st);
void launch_idft_update(int ndof, int N, int NB, int H, bool fp32, const void* W, const double* F,
                        const double* tw, double* Unew, cudaStream_t st);
// End of a captured PP-PC iteration: U = Unext unless *status != 0 or
// rel_res <= *tol_commit, then the control block ctl (status, jump sums, counters).
void launch_commit(long long total, const int* status, const double* jsums, const double* tol_commit,
                   const double* Unext, double* U, const long long* counters, IterCtl* ctl, cudaStream_t st);

// ---- layout conversion between [N][n_nodes] states and [ndof][NB] lanes ----
void launch_state_to_lanes(int ndof, int n_nodes, int N, int NB, const int* node_of_dof,
                           const double* ext, double* lanes, cudaStream_t st);
void launch_lanes_to_state(int ndof, int n_nodes, int N, int NB, const int* dof_of_node,
                           const double* lanes, double* ext, cudaStream_t st);

}  // namespace pppc

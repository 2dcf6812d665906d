// Test-only C entry point around the library's host mesh preprocessing
// (paper_1905_13076_gb300/csrc/mesh_host.cpp), compiled by
// tests/test_host_mesh.py with the host compiler so that the integer
// structures can be compared with the oracle's assembly without a GPU.
#include <cstring>
#include <string>

#include "mesh_host.h"

extern "C" int mesh_pattern(int n_nodes, int n_tri, const int* tri, const int* region, const unsigned char* dirichlet,
                            int n_regions, const int* kinds, int cap, int* ndof, int* nnz, int* node_of_dof,
                            int* rowptr, int* col, int* row_slot, int* n_special, int* n_nl, char* err, int errlen) {
    pppc::HostMesh m;
    std::string e;
    if (!pppc::build_host_mesh(n_nodes, n_tri, tri, region, dirichlet, n_regions, kinds, m, e)) {
        std::strncpy(err, e.c_str(), errlen - 1);
        err[errlen - 1] = 0;
        return 1;
    }
    *ndof = m.ndof;
    *nnz = m.nnz;
    *n_special = m.n_sp;
    *n_nl = m.n_nl;
    if (m.nnz > cap || m.ndof + 1 > cap) return 2;
    for (int i = 0; i < m.ndof; ++i) {
        node_of_dof[i] = m.node_of_dof[i];
        row_slot[i] = m.row_slot[i];
    }
    for (int i = 0; i <= m.ndof; ++i) rowptr[i] = m.rowptr[i];
    for (int k = 0; k < m.nnz; ++k) col[k] = m.col[k];
    return 0;
}

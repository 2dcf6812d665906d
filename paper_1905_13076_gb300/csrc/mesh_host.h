// Host-side integer preprocessing of a triangle mesh for the FE system of
// Eq. 1: dof numbering, CSR pattern, and the element -> matrix-entry maps
// that let the device gather element contributions without atomics.
// No floating-point arithmetic of the method happens here.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace pppc {

enum ElemKind : int { ELEM_NONLINEAR = 1, ELEM_CONDUCTIVE = 2, ELEM_SOURCE = 4 };

struct HostMesh {
    int n_nodes = 0, n_tri = 0, ndof = 0, nnz = 0;
    std::vector<int> dof_of_node;   // -1 on Dirichlet nodes
    std::vector<int> node_of_dof;
    std::vector<int> rowptr, col, diag_k;
    std::vector<int> elem_kind;     // ElemKind bits per triangle
    // all-element contributions of each CSR entry: packed tri*9 + a*3 + b
    std::vector<int> contrib_ptr, contrib;
    // couplings of each free row to Dirichlet nodes: packed tri*9 + a*3 + b
    // with vertex a the row's node and vertex b on the Dirichlet boundary
    std::vector<int> dcoup_ptr, dcoup;
    // special rows: touch a nonlinear or conductive element
    int n_slots = 0, n_sp = 0;
    std::vector<int> row_slot, sp_index, sp_rows, slot_k;
    // nonlinear elements and their contributions per slot: packed q*9 + a*3 + b
    int n_nl = 0;
    std::vector<int> nl_elems, nl_dofs;
    std::vector<int> nlc_ptr, nlc;
};

// Validates indices and builds the maps.  Returns false with a message on
// invalid input.  kinds[r] holds the ElemKind bits of region r.
bool build_host_mesh(int n_nodes, int n_tri, const int32_t* tri, const int32_t* region,
                     const uint8_t* dirichlet, int n_regions, const int* kinds, HostMesh& out,
                     std::string& err);

}  // namespace pppc

// Test-only C entry points around the library's host multigrid setup
// (paper_1905_13076_gb300/csrc/amg_host.cpp), compiled by
// tests/test_host_amg.py with the host compiler, so that the hierarchy can
// be checked against SciPy's Galerkin products without a GPU.
#include <cstring>
#include <string>
#include <vector>

#include "amg_host.h"

namespace {
std::vector<pppc::AmgHostLevel> g_levels;
std::string g_err;

template <typename V>
int copy_out(const V& v, void* out, int cap) {
    if (out && (int)v.size() <= cap) std::memcpy(out, v.data(), v.size() * sizeof(v[0]));
    return (int)v.size();
}
}  // namespace

extern "C" int amg_build(int n, const int* rowptr, const int* col, const double* val, const int* row_slot,
                         int coarse_rows) {
    pppc::AmgOptions opt;
    opt.coarse_rows = coarse_rows;
    if (!pppc::build_amg(n, rowptr, col, val, row_slot, opt, g_levels, g_err)) return -1;
    return (int)g_levels.size();
}

extern "C" const char* amg_error() { return g_err.c_str(); }

// Copies field `name` of level l into out (if it holds cap elements) and
// returns its length; -1 for an unknown name.
extern "C" int amg_field(int l, const char* name, void* out, int cap) {
    const pppc::AmgHostLevel& L = g_levels.at(l);
    const std::string f(name);
    if (f == "rowptr") return copy_out(L.rowptr, out, cap);
    if (f == "col") return copy_out(L.col, out, cap);
    if (f == "val") return copy_out(L.val, out, cap);
    if (f == "row_slot") return copy_out(L.row_slot, out, cap);
    if (f == "sp_index") return copy_out(L.sp_index, out, cap);
    if (f == "l1") return copy_out(L.l1, out, cap);
    if (f == "Pptr") return copy_out(L.Pptr, out, cap);
    if (f == "Pcol") return copy_out(L.Pcol, out, cap);
    if (f == "Pval") return copy_out(L.Pval, out, cap);
    if (f == "Rptr") return copy_out(L.Rptr, out, cap);
    if (f == "Rcol") return copy_out(L.Rcol, out, cap);
    if (f == "Rval") return copy_out(L.Rval, out, cap);
    if (f == "slot_base") return copy_out(L.slot_base, out, cap);
    if (f == "cptr") return copy_out(L.cptr, out, cap);
    if (f == "csrc") return copy_out(L.csrc, out, cap);
    if (f == "cw") return copy_out(L.cw, out, cap);
    if (f == "cost") return copy_out(L.cost, out, cap);
    return -1;
}

// Host-side integer preprocessing of the mesh (see mesh_host.h).
#include "mesh_host.h"

#include <algorithm>
#include <cstdio>
#include <numeric>

namespace pppc {

bool build_host_mesh(int n_nodes, int n_tri, const int32_t* tri, const int32_t* region,
                     const uint8_t* dirichlet, int n_regions, const int* kinds, HostMesh& m,
                     std::string& err) {
    char buf[256];
    if (n_nodes <= 0 || n_tri <= 0) {
        err = "n_nodes and n_tri must be positive";
        return false;
    }
    m = HostMesh();
    m.n_nodes = n_nodes;
    m.n_tri = n_tri;
    m.dof_of_node.assign(n_nodes, -1);
    for (int i = 0; i < n_nodes; ++i) {
        if (dirichlet[i] == 0) {
            m.dof_of_node[i] = m.ndof++;
            m.node_of_dof.push_back(i);
        }
    }
    if (m.ndof == 0) {
        err = "no free node";
        return false;
    }
    m.elem_kind.resize(n_tri);
    for (int e = 0; e < n_tri; ++e) {
        const int r = region[e];
        if (r < 0 || r >= n_regions) {
            snprintf(buf, sizeof buf, "triangle %d: region %d out of range [0,%d)", e, r, n_regions);
            err = buf;
            return false;
        }
        m.elem_kind[e] = kinds[r];
        for (int a = 0; a < 3; ++a) {
            const int v = tri[3 * e + a];
            if (v < 0 || v >= n_nodes) {
                snprintf(buf, sizeof buf, "triangle %d: node %d out of range [0,%d)", e, v, n_nodes);
                err = buf;
                return false;
            }
        }
        if (tri[3 * e] == tri[3 * e + 1] || tri[3 * e] == tri[3 * e + 2] || tri[3 * e + 1] == tri[3 * e + 2]) {
            snprintf(buf, sizeof buf, "triangle %d repeats a node", e);
            err = buf;
            return false;
        }
    }

    // CSR pattern: entry (i, j) for every pair of free vertices sharing a triangle.
    std::vector<std::vector<int>> adj(m.ndof);
    for (int e = 0; e < n_tri; ++e)
        for (int a = 0; a < 3; ++a) {
            const int i = m.dof_of_node[tri[3 * e + a]];
            if (i < 0) continue;
            for (int b = 0; b < 3; ++b) {
                const int j = m.dof_of_node[tri[3 * e + b]];
                if (j >= 0) adj[i].push_back(j);
            }
        }
    m.rowptr.assign(m.ndof + 1, 0);
    for (int i = 0; i < m.ndof; ++i) {
        std::sort(adj[i].begin(), adj[i].end());
        adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
        if (adj[i].empty()) {
            snprintf(buf, sizeof buf, "free node %d belongs to no triangle", m.node_of_dof[i]);
            err = buf;
            return false;
        }
        m.rowptr[i + 1] = m.rowptr[i] + (int)adj[i].size();
    }
    m.nnz = m.rowptr[m.ndof];
    m.col.resize(m.nnz);
    m.diag_k.resize(m.ndof);
    for (int i = 0; i < m.ndof; ++i) {
        std::copy(adj[i].begin(), adj[i].end(), m.col.begin() + m.rowptr[i]);
        m.diag_k[i] = m.rowptr[i] + (int)(std::lower_bound(adj[i].begin(), adj[i].end(), i) - adj[i].begin());
    }
    auto entry = [&](int i, int j) {
        const int* b = m.col.data() + m.rowptr[i];
        const int* e = m.col.data() + m.rowptr[i + 1];
        return (int)(std::lower_bound(b, e, j) - m.col.data());
    };

    // Contributions of every element to every entry (counting sort by entry).
    std::vector<std::pair<int, int>> pairs;
    pairs.reserve((size_t)n_tri * 9);
    std::vector<char> special(m.ndof, 0);
    for (int e = 0; e < n_tri; ++e)
        for (int a = 0; a < 3; ++a) {
            const int i = m.dof_of_node[tri[3 * e + a]];
            if (i < 0) continue;
            if (m.elem_kind[e] & (ELEM_NONLINEAR | ELEM_CONDUCTIVE)) special[i] = 1;
            for (int b = 0; b < 3; ++b) {
                const int j = m.dof_of_node[tri[3 * e + b]];
                if (j < 0) continue;
                pairs.emplace_back(entry(i, j), e * 9 + a * 3 + b);
            }
        }
    m.contrib_ptr.assign(m.nnz + 1, 0);
    for (auto& p : pairs) m.contrib_ptr[p.first + 1]++;
    std::partial_sum(m.contrib_ptr.begin(), m.contrib_ptr.end(), m.contrib_ptr.begin());
    m.contrib.resize(pairs.size());
    {
        std::vector<int> fill(m.contrib_ptr.begin(), m.contrib_ptr.end() - 1);
        for (auto& p : pairs) m.contrib[fill[p.first]++] = p.second;
    }

    // Couplings to Dirichlet nodes (for the difference form of K u).
    {
        std::vector<std::pair<int, int>> dp;
        for (int e = 0; e < n_tri; ++e)
            for (int a = 0; a < 3; ++a) {
                const int i = m.dof_of_node[tri[3 * e + a]];
                if (i < 0) continue;
                for (int b = 0; b < 3; ++b)
                    if (m.dof_of_node[tri[3 * e + b]] < 0) dp.emplace_back(i, e * 9 + a * 3 + b);
            }
        m.dcoup_ptr.assign(m.ndof + 1, 0);
        for (auto& q : dp) m.dcoup_ptr[q.first + 1]++;
        std::partial_sum(m.dcoup_ptr.begin(), m.dcoup_ptr.end(), m.dcoup_ptr.begin());
        m.dcoup.resize(dp.size());
        std::vector<int> fill(m.dcoup_ptr.begin(), m.dcoup_ptr.end() - 1);
        for (auto& q : dp) m.dcoup[fill[q.first]++] = q.second;
    }

    // Special rows and their slots.
    m.row_slot.assign(m.ndof, -1);
    m.sp_index.assign(m.ndof, -1);
    for (int i = 0; i < m.ndof; ++i) {
        if (!special[i]) continue;
        m.row_slot[i] = m.n_slots;
        m.sp_index[i] = m.n_sp++;
        m.sp_rows.push_back(i);
        for (int k = m.rowptr[i]; k < m.rowptr[i + 1]; ++k) m.slot_k.push_back(k);
        m.n_slots += m.rowptr[i + 1] - m.rowptr[i];
    }

    // Nonlinear elements and their contributions per slot.
    std::vector<int> nl_of_elem(n_tri, -1);
    for (int e = 0; e < n_tri; ++e)
        if (m.elem_kind[e] & ELEM_NONLINEAR) {
            nl_of_elem[e] = m.n_nl++;
            m.nl_elems.push_back(e);
            for (int a = 0; a < 3; ++a) m.nl_dofs.push_back(m.dof_of_node[tri[3 * e + a]]);
        }
    m.nlc_ptr.assign(m.n_slots + 1, 0);
    std::vector<std::pair<int, int>> nlp;
    for (int i = 0; i < m.ndof; ++i) {
        if (m.row_slot[i] < 0) continue;
        for (int k = m.rowptr[i]; k < m.rowptr[i + 1]; ++k) {
            const int s = m.row_slot[i] + (k - m.rowptr[i]);
            for (int c = m.contrib_ptr[k]; c < m.contrib_ptr[k + 1]; ++c) {
                const int e = m.contrib[c] / 9;
                if (nl_of_elem[e] >= 0) nlp.emplace_back(s, nl_of_elem[e] * 9 + m.contrib[c] % 9);
            }
        }
    }
    for (auto& p : nlp) m.nlc_ptr[p.first + 1]++;
    std::partial_sum(m.nlc_ptr.begin(), m.nlc_ptr.end(), m.nlc_ptr.begin());
    m.nlc.resize(nlp.size());
    {
        std::vector<int> fill(m.nlc_ptr.begin(), m.nlc_ptr.end() - 1);
        for (auto& p : nlp) m.nlc[fill[p.first]++] = p.second;
    }
    return true;
}

}  // namespace pppc

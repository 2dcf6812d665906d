// Smoothed-aggregation hierarchy for the fine PCG preconditioner (see
// amg_host.h): strength of connection, greedy aggregation, the tentative and
// the Jacobi-smoothed prolongator, Galerkin coarse matrices, and the tables
// that rebuild each lane's coarse matrices from its fine Jacobian.
#include "amg_host.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>

namespace pppc {
namespace {

struct Csr {
    int n = 0, m = 0;   // rows, columns
    std::vector<int> ptr, col;
    std::vector<double> val;
};

Csr transpose(const Csr& A) {
    Csr T;
    T.n = A.m;
    T.m = A.n;
    T.ptr.assign(T.n + 1, 0);
    for (int c : A.col) ++T.ptr[c + 1];
    for (int i = 0; i < T.n; ++i) T.ptr[i + 1] += T.ptr[i];
    T.col.resize(A.col.size());
    T.val.resize(A.val.size());
    std::vector<int> next(T.ptr.begin(), T.ptr.end() - 1);
    for (int i = 0; i < A.n; ++i)
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            const int q = next[A.col[k]]++;
            T.col[q] = i;   // rows visited in order: columns of T come out sorted
            T.val[q] = A.val[k];
        }
    return T;
}

// C = A B (Gustavson, one dense accumulator row; every structural product
// is kept, so the pattern does not depend on cancellation)
Csr multiply(const Csr& A, const Csr& B) {
    Csr C;
    C.n = A.n;
    C.m = B.m;
    C.ptr.assign(A.n + 1, 0);
    std::vector<int> mark(B.m, -1), cols;
    std::vector<double> acc(B.m, 0.0);
    for (int i = 0; i < A.n; ++i) {
        cols.clear();
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            const int j = A.col[k];
            const double a = A.val[k];
            for (int q = B.ptr[j]; q < B.ptr[j + 1]; ++q) {
                const int c = B.col[q];
                if (mark[c] != i) {
                    mark[c] = i;
                    acc[c] = 0.0;
                    cols.push_back(c);
                }
                acc[c] += a * B.val[q];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int c : cols) {
            C.col.push_back(c);
            C.val.push_back(acc[c]);
        }
        C.ptr[i + 1] = (int)C.col.size();
    }
    return C;
}

// Strong neighbours of every row: j != i with |a_ij| >= theta sqrt(|a_ii a_jj|).
void strength(const Csr& A, double theta, std::vector<int>& sptr, std::vector<int>& scol) {
    std::vector<double> d(A.n, 0.0);
    for (int i = 0; i < A.n; ++i)
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (A.col[k] == i) d[i] = std::fabs(A.val[k]);
    sptr.assign(A.n + 1, 0);
    scol.clear();
    for (int i = 0; i < A.n; ++i) {
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            const int j = A.col[k];
            if (j != i && std::fabs(A.val[k]) >= theta * std::sqrt(d[i] * d[j])) scol.push_back(j);
        }
        sptr[i + 1] = (int)scol.size();
    }
}

// Greedy aggregation in row order: (1) a row whose strong neighbours are all
// free starts an aggregate with them; (2) a remaining row joins the
// aggregate of its first strong neighbour placed in (1); (3) what is left
// forms aggregates with its free strong neighbours.  Returns the count.
int aggregate(int n, const std::vector<int>& sptr, const std::vector<int>& scol, std::vector<int>& agg) {
    agg.assign(n, -1);
    int na = 0;
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        bool free_nb = true;
        for (int k = sptr[i]; k < sptr[i + 1] && free_nb; ++k) free_nb = agg[scol[k]] < 0;
        if (!free_nb) continue;
        agg[i] = na;
        for (int k = sptr[i]; k < sptr[i + 1]; ++k) agg[scol[k]] = na;
        ++na;
    }
    const std::vector<int> first = agg;
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        for (int k = sptr[i]; k < sptr[i + 1]; ++k)
            if (first[scol[k]] >= 0) {
                agg[i] = first[scol[k]];
                break;
            }
    }
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        agg[i] = na;
        for (int k = sptr[i]; k < sptr[i + 1]; ++k)
            if (agg[scol[k]] < 0) agg[scol[k]] = na;
        ++na;
    }
    return na;
}

// Largest eigenvalue of D^-1 A by power iteration from a fixed start.
double lambda_max(const Csr& A, const std::vector<double>& dinv) {
    std::vector<double> x(A.n), y(A.n);
    for (int i = 0; i < A.n; ++i) x[i] = 1.0 + (double)((i * 7919) % 17) / 17.0;
    double lam = 1.0;
    for (int it = 0; it < 30; ++it) {
        double ny = 0.0, nx = 0.0;
        for (int i = 0; i < A.n; ++i) {
            double s = 0.0;
            for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
            y[i] = dinv[i] * s;
            ny += y[i] * y[i];
            nx += x[i] * x[i];
        }
        if (!(ny > 0.0)) break;
        lam = std::sqrt(ny / nx);
        const double s = 1.0 / std::sqrt(ny);
        for (int i = 0; i < A.n; ++i) x[i] = y[i] * s;
    }
    return lam;
}

// Fill the per-level bookkeeping of a level whose pattern, values and
// special rows (row_slot) are set: special-row indices and l1 row norms.
void finish_level(AmgHostLevel& L) {
    L.sp_index.assign(L.n, -1);
    L.sp_rows.clear();
    for (int i = 0; i < L.n; ++i)
        if (L.row_slot[i] >= 0) {
            L.sp_index[i] = (int)L.sp_rows.size();
            L.sp_rows.push_back(i);
        }
    L.n_sp = (int)L.sp_rows.size();
    L.l1.assign(L.n, 0.0);
    for (int i = 0; i < L.n; ++i)
        for (int k = L.rowptr[i]; k < L.rowptr[i + 1]; ++k) L.l1[i] += std::fabs(L.val[k]);
}

Csr as_csr(const AmgHostLevel& L) {
    Csr A;
    A.n = A.m = L.n;
    A.ptr = L.rowptr;
    A.col = L.col;
    A.val = L.val;
    return A;
}

// Coarse level c from fine level f with prolongator P: Galerkin values,
// special coarse rows and the per-lane slot tables.
void coarse_level(const AmgHostLevel& f, const Csr& P, const Csr& Ac, AmgHostLevel& c) {
    c.n = Ac.n;
    c.rowptr = Ac.ptr;
    c.col = Ac.col;
    c.val = Ac.val;
    // a coarse row is special if a special fine row prolongs into it
    c.row_slot.assign(c.n, -1);
    std::vector<char> sp(c.n, 0);
    for (int i = 0; i < f.n; ++i)
        if (f.row_slot[i] >= 0)
            for (int k = P.ptr[i]; k < P.ptr[i + 1]; ++k) sp[P.col[k]] = 1;
    int slots = 0;
    for (int a = 0; a < c.n; ++a)
        if (sp[a]) {
            c.row_slot[a] = slots;
            slots += c.rowptr[a + 1] - c.rowptr[a];
        }
    c.n_slots = slots;
    finish_level(c);
    // contributions (coarse slot <- weight * fine slot), counted then filled
    // per coarse slot: for special fine row i, entry (i, j) = fine slot s,
    // P(i, a) and P(j, b) give weight P(i, a) P(j, b) to coarse entry (a, b)
    // coarse row a's slot of column b: a dense map over the columns of the
    // row last loaded (every column looked up lies in that row's pattern,
    // the Galerkin product's, so stale entries of other columns are never
    // read)
    std::vector<int> pos(c.n, 0);
    int loaded = -1;
    auto load_row = [&](int a) {
        if (a == loaded) return;
        for (int k = c.rowptr[a]; k < c.rowptr[a + 1]; ++k) pos[c.col[k]] = c.row_slot[a] + (k - c.rowptr[a]);
        loaded = a;
    };
    std::vector<int64_t> cnt((size_t)slots + 1, 0);
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<int64_t> fillpos;
        if (pass == 1) {
            for (int e = 0; e < slots; ++e) cnt[e + 1] += cnt[e];
            c.csrc.assign((size_t)cnt[slots], 0);
            c.cw.assign((size_t)cnt[slots], 0.0);
            fillpos.assign(cnt.begin(), cnt.end() - 1);
        }
        for (int i = 0; i < f.n; ++i) {
            if (f.row_slot[i] < 0) continue;
            for (int p = P.ptr[i]; p < P.ptr[i + 1]; ++p) {
                const int a = P.col[p];
                const double pa = P.val[p];
                load_row(a);
                for (int k = f.rowptr[i]; k < f.rowptr[i + 1]; ++k) {
                    const int j = f.col[k];
                    const int s = f.row_slot[i] + (k - f.rowptr[i]);
                    for (int q = P.ptr[j]; q < P.ptr[j + 1]; ++q) {
                        const int e = pos[P.col[q]];
                        if (pass == 0) {
                            ++cnt[e + 1];
                        } else {
                            const size_t w = (size_t)fillpos[e]++;
                            c.csrc[w] = s;
                            c.cw[w] = pa * P.val[q];
                        }
                    }
                }
            }
        }
    }
    // per coarse slot: sorted by source slot, duplicates merged, compacted in
    // place.  The fill visits the fine rows and their entries in order, so a
    // slot's contributions arrive sorted whenever the fine level numbers its
    // slots row by row (the mesh and every coarse level do), and one fine
    // slot reaches a coarse slot at most once (P's rows hold distinct
    // columns): such a slot is kept as filled.  Any other is sorted and
    // merged; merging only shrinks, so the write position never passes the
    // read position.
    c.cptr.assign(slots + 1, 0);
    const auto by_src = [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
        return x.first < y.first;
    };
    std::vector<std::pair<int, double>> tmp;
    size_t w = 0;
    for (int e = 0; e < slots; ++e) {
        const size_t b = (size_t)cnt[e], en = (size_t)cnt[e + 1];
        bool increasing = true;
        for (size_t r = b + 1; r < en && increasing; ++r) increasing = c.csrc[r - 1] < c.csrc[r];
        if (increasing) {
            if (w != b)
                for (size_t r = b; r < en; ++r) {
                    c.csrc[w + (r - b)] = c.csrc[r];
                    c.cw[w + (r - b)] = c.cw[r];
                }
            w += en - b;
        } else {
            tmp.clear();
            for (size_t r = b; r < en; ++r) tmp.emplace_back(c.csrc[r], c.cw[r]);
            if (!std::is_sorted(tmp.begin(), tmp.end(), by_src)) std::sort(tmp.begin(), tmp.end(), by_src);
            for (const auto& x : tmp) {
                if (w > (size_t)c.cptr[e] && c.csrc[w - 1] == x.first) {
                    c.cw[w - 1] += x.second;
                } else {
                    c.csrc[w] = x.first;
                    c.cw[w] = x.second;
                    ++w;
                }
            }
        }
        c.cptr[e + 1] = (int)w;
    }
    c.csrc.resize(w);
    c.cw.resize(w);
    // base: the representative Galerkin value minus what the tabulated
    // contributions give at the representative fine values
    std::vector<double> fslot((size_t)f.n_slots, 0.0);
    for (int i = 0; i < f.n; ++i)
        if (f.row_slot[i] >= 0)
            for (int k = f.rowptr[i]; k < f.rowptr[i + 1]; ++k) fslot[f.row_slot[i] + (k - f.rowptr[i])] = f.val[k];
    c.slot_base.assign(slots, 0.0);
    for (int a = 0; a < c.n; ++a) {
        if (c.row_slot[a] < 0) continue;
        for (int k = c.rowptr[a]; k < c.rowptr[a + 1]; ++k) {
            const int e = c.row_slot[a] + (k - c.rowptr[a]);
            double s = 0.0;
            for (int q = c.cptr[e]; q < c.cptr[e + 1]; ++q) s += c.cw[q] * fslot[c.csrc[q]];
            c.slot_base[e] = c.val[k] - s;
        }
    }
}

}  // namespace

bool build_amg(int n, const int* rowptr, const int* col, const double* val, const int* row_slot,
               const AmgOptions& opt, std::vector<AmgHostLevel>& levels, std::string& err) {
    levels.clear();
    if (n < 1 || !rowptr || !col || !val || !row_slot || rowptr[0] != 0) {
        err = "amg: empty or malformed matrix";
        return false;
    }
    AmgHostLevel f;
    f.n = n;
    f.rowptr.assign(rowptr, rowptr + n + 1);
    f.col.assign(col, col + rowptr[n]);
    f.val.assign(val, val + rowptr[n]);
    f.row_slot.assign(row_slot, row_slot + n);
    for (int i = 0; i < n; ++i) {
        if (f.rowptr[i + 1] < f.rowptr[i]) {
            err = "amg: rowptr decreases";
            return false;
        }
        bool diag = false;
        for (int k = f.rowptr[i]; k < f.rowptr[i + 1]; ++k) {
            if (f.col[k] < 0 || f.col[k] >= n || (k > f.rowptr[i] && f.col[k] <= f.col[k - 1])) {
                err = "amg: column out of range or unsorted";
                return false;
            }
            diag |= f.col[k] == i && f.val[k] > 0.0;
        }
        if (!diag) {
            err = "amg: a row has no positive diagonal";
            return false;
        }
        if (row_slot[i] >= 0) f.n_slots = std::max(f.n_slots, row_slot[i] + (f.rowptr[i + 1] - f.rowptr[i]));
    }
    finish_level(f);
    levels.push_back(std::move(f));
    while ((int)levels.size() < opt.max_levels && levels.back().n > opt.coarse_rows) {
        const AmgHostLevel& F = levels.back();
        const Csr A = as_csr(F);
        std::vector<int> sptr, scol, agg;
        strength(A, opt.theta, sptr, scol);
        const int na = aggregate(A.n, sptr, scol, agg);
        if (na < 1 || na > opt.min_ratio * A.n) break;
        Csr Pt;
        Pt.n = A.n;
        Pt.m = na;
        Pt.ptr.resize(A.n + 1);
        Pt.col = agg;
        Pt.val.assign(A.n, 1.0);
        std::iota(Pt.ptr.begin(), Pt.ptr.end(), 0);
        // P = (I - (4/3) / lambda_max(D^-1 A) D^-1 A) P_tent
        std::vector<double> dinv(A.n, 0.0);
        for (int i = 0; i < A.n; ++i)
            for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
                if (A.col[k] == i) dinv[i] = 1.0 / A.val[k];
        const double omega = 4.0 / 3.0 / lambda_max(A, dinv);
        Csr AP = multiply(A, Pt);
        for (int i = 0; i < AP.n; ++i)
            for (int k = AP.ptr[i]; k < AP.ptr[i + 1]; ++k) AP.val[k] *= -omega * dinv[i];
        // P = P_tent + AP (P_tent's one entry per row is merged into the row)
        Csr P;
        P.n = A.n;
        P.m = na;
        P.ptr.assign(A.n + 1, 0);
        for (int i = 0; i < A.n; ++i) {
            bool placed = false;
            for (int k = AP.ptr[i]; k < AP.ptr[i + 1]; ++k) {
                double v = AP.val[k];
                if (AP.col[k] == agg[i]) {
                    v += 1.0;
                    placed = true;
                }
                P.col.push_back(AP.col[k]);
                P.val.push_back(v);
            }
            if (!placed) {   // cannot happen for a positive diagonal, kept for safety
                P.col.push_back(agg[i]);
                P.val.push_back(1.0);
                std::sort(P.col.begin() + P.ptr[i], P.col.end());
            }
            P.ptr[i + 1] = (int)P.col.size();
        }
        const Csr R = transpose(P);
        const Csr Ac = multiply(R, multiply(A, P));
        AmgHostLevel c;
        coarse_level(F, P, Ac, c);
        c.Pptr = P.ptr;
        c.Pcol = P.col;
        c.Pval = P.val;
        c.Rptr = R.ptr;
        c.Rcol = R.col;
        c.Rval = R.val;
        levels.push_back(std::move(c));
    }
    for (size_t l = 1; l < levels.size(); ++l) {
        AmgHostLevel& L = levels[l];
        const AmgHostLevel* next = l + 1 < levels.size() ? &levels[l + 1] : nullptr;
        L.cost.assign(L.n + 1, 0);
        for (int c = 0; c < L.n; ++c) {
            const long long a = L.rowptr[c + 1] - L.rowptr[c];
            long long w = 2 * a * (L.row_slot[c] >= 0 ? 2 : 1) + (L.Rptr[c + 1] - L.Rptr[c]) + 4;
            if (next) w += next->Pptr[c + 1] - next->Pptr[c];
            L.cost[c + 1] = L.cost[c] + w;
        }
    }
    return true;
}

}  // namespace pppc

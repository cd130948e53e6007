// Two-level ORAS (Section 7: a coarse space restores the scalability of the
// one-level method in the number of subdomains), host side: the prolongation
// from a coarser mesh's Whitney space, the pattern and values of the Galerkin
// coarse operator A_c = P^T A P, and the coarse operator as a decomposition
// with one subdomain and one dense front, so that its factorisation and its
// exact solves run on the same batched kernels as the subdomain solves.
//
// Prolongation (midpoint rule of each fine edge's tangential integral of the
// coarse field):  P[e, E] = N_E(m_e) . (x_hi(e) - x_lo(e)),
// N_E a lowest-order Whitney function of the coarse tet that holds the fine
// edge's midpoint m_e: the lowest-numbered tet whose smallest barycentric
// coordinate of m_e is >= -1e-12 (candidates from a grid over the tets'
// bounding boxes); for a midpoint in no tet, the lowest-numbered tet whose
// smallest barycentric coordinate is within 1e-12 of the largest over all
// tets (the affine extension of the least-outside tet's basis).  Ties go to
// the lowest tet number, so rounding cannot change the choice (N_E's normal
// component jumps across coarse faces).  Only the Whitney DOFs of the fine
// mesh get rows (second-order DOFs have no coarse component).
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include "common.h"
#include "model.h"
#include "parallel.h"

namespace mwi {

namespace {

struct TetGeo {
    double G[4][3];   // gradients of the barycentrics
    double c[3];      // centroid
};

TetGeo tet_geo(const Topology& T, int64_t t) {
    TetGeo g;
    const int32_t* v = &T.tv[4 * t];
    double P[4][3];
    for (int k = 0; k < 4; ++k)
        for (int d = 0; d < 3; ++d) P[k][d] = T.xyz[3 * (int64_t)v[k] + d];
    // E columns: P_k - P_0; rows of E^{-1} are the gradients of lambda_1..3
    double E[3][3];
    for (int d = 0; d < 3; ++d)
        for (int k = 0; k < 3; ++k) E[d][k] = P[k + 1][d] - P[0][d];
    const double det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
                       E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                       E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
    const double id = 1.0 / det;
    const double inv[3][3] = {
        {(E[1][1] * E[2][2] - E[1][2] * E[2][1]) * id, (E[0][2] * E[2][1] - E[0][1] * E[2][2]) * id,
         (E[0][1] * E[1][2] - E[0][2] * E[1][1]) * id},
        {(E[1][2] * E[2][0] - E[1][0] * E[2][2]) * id, (E[0][0] * E[2][2] - E[0][2] * E[2][0]) * id,
         (E[0][2] * E[1][0] - E[0][0] * E[1][2]) * id},
        {(E[1][0] * E[2][1] - E[1][1] * E[2][0]) * id, (E[0][1] * E[2][0] - E[0][0] * E[2][1]) * id,
         (E[0][0] * E[1][1] - E[0][1] * E[1][0]) * id}};
    for (int d = 0; d < 3; ++d) {
        g.G[0][d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
        for (int k = 0; k < 3; ++k) g.G[k + 1][d] = inv[k][d];
    }
    for (int d = 0; d < 3; ++d) g.c[d] = (P[0][d] + P[1][d] + P[2][d] + P[3][d]) / 4.0;
    return g;
}

// uniform grid over the coarse tets' bounding boxes (inflated by 1e-9 of the
// domain's extent): the tets that can hold a point are those listed in the
// point's cell
struct TetGrid {
    double lo[3], h;
    int n[3];
    std::vector<int64_t> start;
    std::vector<int32_t> ids;

    void build(const Topology& T) {
        double hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = 1e300;
            hi[d] = -1e300;
        }
        for (int64_t v = 0; v < T.nv; ++v)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], T.xyz[3 * v + d]);
                hi[d] = std::max(hi[d], T.xyz[3 * v + d]);
            }
        const double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
        pad = 1e-9 * ext;
        h = std::max(ext / std::max(1.0, std::cbrt((double)T.nt / 4.0)), 1e-300);
        for (int d = 0; d < 3; ++d) n[d] = std::max(1, (int)std::ceil((hi[d] - lo[d]) / h) + 1);
        std::vector<std::array<int, 6>> box(T.nt);
        std::vector<int64_t> cnt((size_t)n[0] * n[1] * n[2] + 1, 0);
        for (int64_t t = 0; t < T.nt; ++t) {
            double bl[3] = {1e300, 1e300, 1e300}, bh[3] = {-1e300, -1e300, -1e300};
            for (int k = 0; k < 4; ++k)
                for (int d = 0; d < 3; ++d) {
                    const double x = T.xyz[3 * (int64_t)T.tv[4 * t + k] + d];
                    bl[d] = std::min(bl[d], x);
                    bh[d] = std::max(bh[d], x);
                }
            for (int d = 0; d < 3; ++d) {
                box[t][d] = coord(bl[d] - pad, d);
                box[t][3 + d] = coord(bh[d] + pad, d);
            }
            for (int z = box[t][2]; z <= box[t][5]; ++z)
                for (int y = box[t][1]; y <= box[t][4]; ++y)
                    for (int x = box[t][0]; x <= box[t][3]; ++x) cnt[cell(x, y, z) + 1]++;
        }
        for (size_t i = 1; i < cnt.size(); ++i) cnt[i] += cnt[i - 1];
        start = cnt;
        ids.assign(cnt.back(), 0);
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t t = 0; t < T.nt; ++t)
            for (int z = box[t][2]; z <= box[t][5]; ++z)
                for (int y = box[t][1]; y <= box[t][4]; ++y)
                    for (int x = box[t][0]; x <= box[t][3]; ++x) ids[fill[cell(x, y, z)]++] = (int32_t)t;
    }
    double pad = 0;
    int coord(double x, int d) const {
        const double f = std::floor((x - lo[d]) / h);
        return (int)std::min<double>(std::max<double>(f, 0.0), (double)(n[d] - 1));
    }
    int64_t cell(int x, int y, int z) const { return ((int64_t)z * n[1] + y) * n[0] + x; }
    // tets listed in the cell of p (ascending tet number)
    std::pair<const int32_t*, const int32_t*> near(const double* p) const {
        const int64_t c = cell(coord(p[0], 0), coord(p[1], 1), coord(p[2], 2));
        return {ids.data() + start[c], ids.data() + start[c + 1]};
    }
};

// barycentric coordinates of p in tet g: lambda_q is affine with gradient G_q
// and equals 1/4 at the centroid; returns the smallest
double bary(const TetGeo& g, const double* p, double lam[4]) {
    double mn = 1e300;
    for (int q = 0; q < 4; ++q) {
        lam[q] = g.G[q][0] * (p[0] - g.c[0]) + g.G[q][1] * (p[1] - g.c[1]) + g.G[q][2] * (p[2] - g.c[2]) + 0.25;
        mn = std::min(mn, lam[q]);
    }
    return mn;
}

}  // namespace

void build_prolongation(const Topology& F, const Topology& Cz, CoarseHost& out) {
    MWI_REQUIRE(Cz.order == 1, MWI_EINVAL, "the coarse mesh must be of order 1 (Whitney elements)");
    MWI_REQUIRE(Cz.nt >= 1 && Cz.ndof >= 1, MWI_EINVAL, "empty coarse mesh");
    out.n = F.ndof;
    out.nc = Cz.ndof;
    std::vector<TetGeo> geo(Cz.nt);
    parallel_for(Cz.nt, 4096, [&](int64_t t, int) { geo[t] = tet_geo(Cz, t); });
    TetGrid grid;
    grid.build(Cz);
    // per fine edge with a Whitney DOF: six entries (coarse DOF, value), -1 for removed coarse DOFs
    const int64_t ne = F.ne;
    std::vector<int32_t> ecol((size_t)ne * 6, -1);
    std::vector<double> eval((size_t)ne * 6, 0.0);
    const int kEdges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    parallel_for(ne, 256, [&](int64_t e, int) {
        if (F.edge_dof[e] < 0) return;
        const int64_t a = F.edges[2 * e], b = F.edges[2 * e + 1];
        double mid[3], tang[3];
        for (int d = 0; d < 3; ++d) {
            mid[d] = 0.5 * (F.xyz[3 * a + d] + F.xyz[3 * b + d]);
            tang[d] = F.xyz[3 * b + d] - F.xyz[3 * a + d];
        }
        // the lowest-numbered tet that holds the midpoint (smallest barycentric >= -1e-12)
        int64_t pick = -1;
        double L[4] = {0, 0, 0, 0}, lam[4];
        const auto cand = grid.near(mid);
        for (const int32_t* q = cand.first; q != cand.second; ++q)
            if (bary(geo[*q], mid, lam) >= -1e-12) {
                pick = *q;
                std::copy(lam, lam + 4, L);
                break;
            }
        if (pick < 0) {
            // outside the coarse mesh: the lowest-numbered tet whose smallest
            // barycentric is within 1e-12 of the largest over all tets
            std::vector<double> mins(Cz.nt);
            double best = -1e300;
            for (int64_t t = 0; t < Cz.nt; ++t) {
                mins[t] = bary(geo[t], mid, lam);
                best = std::max(best, mins[t]);
            }
            for (int64_t t = 0; t < Cz.nt; ++t)
                if (mins[t] >= best - 1e-12) {
                    pick = t;
                    bary(geo[t], mid, L);
                    break;
                }
        }
        const TetGeo& g = geo[pick];
        for (int j = 0; j < 6; ++j) {
            const int p = kEdges[j][0], q = kEdges[j][1];
            const int32_t cdof = Cz.tet_dofs[6 * (int64_t)pick + j];
            if (cdof < 0) continue;
            double v = 0.0;
            for (int d = 0; d < 3; ++d) v += (L[p] * g.G[q][d] - L[q] * g.G[p][d]) * tang[d];
            ecol[6 * e + j] = cdof;
            eval[6 * e + j] = v;
        }
    });
    // CSR by fine DOF
    std::vector<int64_t> dof_edge(F.ndof, -1);
    for (int64_t e = 0; e < ne; ++e)
        if (F.edge_dof[e] >= 0) dof_edge[F.edge_dof[e]] = e;
    out.P_rp.assign(F.ndof + 1, 0);
    out.P_col.clear();
    out.P_val.clear();
    for (int64_t r = 0; r < F.ndof; ++r) {
        const int64_t e = dof_edge[r];
        if (e >= 0) {
            std::vector<std::pair<int32_t, double>> row;
            for (int j = 0; j < 6; ++j)
                if (ecol[6 * e + j] >= 0) row.emplace_back(ecol[6 * e + j], eval[6 * e + j]);
            std::sort(row.begin(), row.end());
            for (auto& x : row) {
                out.P_col.push_back(x.first);
                out.P_val.push_back(x.second);
            }
        }
        out.P_rp[r + 1] = (int64_t)out.P_col.size();
    }
    // transpose (rows = coarse DOFs, fine DOFs ascending)
    out.PT_rp.assign(out.nc + 1, 0);
    for (int32_t c : out.P_col) out.PT_rp[c + 1]++;
    for (int64_t c = 0; c < out.nc; ++c) out.PT_rp[c + 1] += out.PT_rp[c];
    out.PT_col.assign(out.P_col.size(), 0);
    out.PT_val.assign(out.P_col.size(), 0.0);
    std::vector<int64_t> fill(out.PT_rp.begin(), out.PT_rp.end() - 1);
    for (int64_t r = 0; r < F.ndof; ++r)
        for (int64_t q = out.P_rp[r]; q < out.P_rp[r + 1]; ++q) {
            const int64_t k2 = fill[out.P_col[q]]++;
            out.PT_col[k2] = (int32_t)r;
            out.PT_val[k2] = out.P_val[q];
        }
}

void coarse_pattern(const std::vector<int64_t>& A_rp, const std::vector<int32_t>& A_col, CoarseHost& C) {
    // row E of P^T A P: coarse DOFs F reached from the fine rows e of P^T's row E
    // through A's row e and P's rows
    const int64_t nc = C.nc;
    std::vector<std::vector<int32_t>> rows(nc);
    parallel_for(nc, 16, [&](int64_t E, int) {
        std::vector<int32_t>& row = rows[E];
        for (int64_t q = C.PT_rp[E]; q < C.PT_rp[E + 1]; ++q) {
            const int64_t e = C.PT_col[q];
            for (int64_t s = A_rp[e]; s < A_rp[e + 1]; ++s) {
                const int64_t f = A_col[s];
                for (int64_t t = C.P_rp[f]; t < C.P_rp[f + 1]; ++t) row.push_back(C.P_col[t]);
            }
        }
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
    });
    C.Ac_rp.assign(nc + 1, 0);
    for (int64_t E = 0; E < nc; ++E) C.Ac_rp[E + 1] = C.Ac_rp[E] + (int64_t)rows[E].size();
    C.Ac_col.resize(C.Ac_rp[nc]);
    for (int64_t E = 0; E < nc; ++E) std::copy(rows[E].begin(), rows[E].end(), C.Ac_col.begin() + C.Ac_rp[E]);
}

void coarse_values(const std::vector<int64_t>& A_rp, const std::vector<int32_t>& A_col, const double2* A_val,
                   const CoarseHost& C, std::vector<double2>& out) {
    // row E: sum over fine e of P[e,E] (A P)[e, :], the fine rows in ascending order
    const int64_t nc = C.nc;
    out.assign(C.Ac_col.size(), make_double2(0.0, 0.0));
    parallel_for(nc, 16, [&](int64_t E, int) {
        // position of each coarse column in row E (-1 elsewhere; reset after the row)
        thread_local std::vector<int32_t> pos;
        if ((int64_t)pos.size() < nc) pos.assign(nc, -1);
        for (int64_t q = C.Ac_rp[E]; q < C.Ac_rp[E + 1]; ++q) pos[C.Ac_col[q]] = (int32_t)(q - C.Ac_rp[E]);
        const int64_t base = C.Ac_rp[E];
        for (int64_t q = C.PT_rp[E]; q < C.PT_rp[E + 1]; ++q) {
            const int64_t e = C.PT_col[q];
            const double pe = C.PT_val[q];
            for (int64_t s = A_rp[e]; s < A_rp[e + 1]; ++s) {
                const int64_t f = A_col[s];
                const double2 a = A_val[s];
                for (int64_t t = C.P_rp[f]; t < C.P_rp[f + 1]; ++t) {
                    const double w = pe * C.P_val[t];
                    double2& o = out[base + pos[C.P_col[t]]];
                    o.x += w * a.x;
                    o.y += w * a.y;
                }
            }
        }
        for (int64_t q = C.Ac_rp[E]; q < C.Ac_rp[E + 1]; ++q) pos[C.Ac_col[q]] = -1;
    });
}

void dense_front_decomposition(const CoarseHost& C, Decomposition& D) {
    const int64_t nc = C.nc;
    MWI_REQUIRE(nc <= 16384, MWI_EINVAL, "coarse space too large for one dense front (at most 16384 DOFs)");
    D = Decomposition();
    D.n_sub = 1;
    D.overlap = 0;
    D.sub_off = {0, nc};
    D.loc2glob.resize(nc);
    std::iota(D.loc2glob.begin(), D.loc2glob.end(), 0);
    D.dweight.assign(nc, 1.0);
    D.own_ptr.resize(nc + 1);
    std::iota(D.own_ptr.begin(), D.own_ptr.end(), 0);
    D.own_row.resize(nc);
    std::iota(D.own_row.begin(), D.own_row.end(), 0);
    D.own_w.assign(nc, 1.0);
    Front F;
    F.sub = 0;
    F.start = 0;
    F.p = (int32_t)nc;
    F.u = 0;
    F.parent = -1;
    F.level = 0;
    F.f_off = 0;
    F.sch_off = 0;
    F.u_off = 0;
    F.upd_row = 0;
    D.fronts = {F};
    D.level_ptr = {0, 1};
    D.level_fronts = {0};
    D.n_levels = 1;
    D.child_ptr = {0, 0};
    D.asm_base = {0};
    D.asm_ptr.assign(nc + 1, 0);
    // front assembly: every entry of the lower triangle of A_c into the column-major panel
    D.amap_front_ptr = {0};
    for (int64_t r = 0; r < nc; ++r)
        for (int64_t q = C.Ac_rp[r]; q < C.Ac_rp[r + 1]; ++q) {
            const int64_t c = C.Ac_col[q];
            if (c > r) continue;
            D.amap_slot.push_back(q);
            D.amap_pos.push_back(c * nc + r);
        }
    D.amap_front_ptr.push_back((int64_t)D.amap_slot.size());
    D.ws_entries = nc * nc;
    D.level_sch = {0};
    D.sch_entries[0] = D.sch_entries[1] = 0;
    D.upd_rows = 0;
    D.factor_entries = nc * nc;
    D.factor_flops = 8.0 / 3.0 * (double)nc * nc * nc * 4.0;
    D.max_front = (int32_t)nc;
    D.B.nrows = nc;
}

}  // namespace mwi

// Antenna -> edge map of the right-hand sides and the receiver functionals.
// The waveguide ports of Section 2 (Eq. eqwgj) are read as edge-current
// dipoles, one mesh edge per antenna.  The edge starts at the mesh vertex
// nearest to the antenna's position (lowest vertex id on ties) and is, among
// the edges at that vertex, the one best aligned with the antenna's direction
// (largest cosine; lowest edge id on ties); its sign says whether the
// direction agrees with the edge's orientation (low -> high vertex id).
//
// The nearest vertex comes from a uniform grid of the vertices, searched in
// shells of cells around the position's cell until no unsearched cell can
// hold a vertex as near as the best one: the result is the exhaustive
// search's, in O(cells searched) instead of O(vertices) per antenna.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "common.h"
#include "model.h"

namespace mwi {

void build_vertex_grid(const std::vector<double>& xyz, int64_t nv, VertexGrid& G) {
    double hi[3];
    for (int a = 0; a < 3; ++a) G.lo[a] = hi[a] = nv > 0 ? xyz[a] : 0.0;
    for (int64_t v = 0; v < nv; ++v)
        for (int a = 0; a < 3; ++a) {
            G.lo[a] = std::min(G.lo[a], xyz[3 * v + a]);
            hi[a] = std::max(hi[a], xyz[3 * v + a]);
        }
    double ext[3], diag2 = 0;
    for (int a = 0; a < 3; ++a) {
        ext[a] = hi[a] - G.lo[a];
        diag2 += ext[a] * ext[a];
    }
    // cubic cells of about two vertices each over the box (flat axes get one cell)
    const double floor_ext = 1e-9 * std::max(std::sqrt(diag2), 1e-300);
    double vol = 1;
    int nflat = 0;
    for (int a = 0; a < 3; ++a) {
        if (ext[a] > floor_ext) vol *= ext[a];
        else ++nflat;
    }
    const double cells = std::max<double>(1.0, 0.5 * (double)nv);
    const double h = nflat == 3 ? 1.0 : std::pow(vol / cells, 1.0 / (3 - nflat));
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        G.n[a] = ext[a] > floor_ext ? std::min<int64_t>(1024, std::max<int64_t>(1, (int64_t)std::ceil(ext[a] / h))) : 1;
        G.h[a] = ext[a] > floor_ext ? ext[a] / (double)G.n[a] : 1.0;
        total *= G.n[a];
    }
    std::vector<int64_t> cell(nv);
    G.cell_ptr.assign(total + 1, 0);
    for (int64_t v = 0; v < nv; ++v) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) c[a] = G.cell_of(a, xyz[3 * v + a]);
        cell[v] = (c[2] * G.n[1] + c[1]) * G.n[0] + c[0];
        ++G.cell_ptr[cell[v] + 1];
    }
    for (int64_t c = 0; c < total; ++c) G.cell_ptr[c + 1] += G.cell_ptr[c];
    G.ids.resize(nv);
    std::vector<int64_t> fill(G.cell_ptr.begin(), G.cell_ptr.end() - 1);
    for (int64_t v = 0; v < nv; ++v) G.ids[fill[cell[v]]++] = (int32_t)v;  // ascending id within a cell
    G.margin2 = 1e-18 * diag2;
}

int64_t nearest_vertex(const std::vector<double>& xyz, const VertexGrid& G, const double* p) {
    int64_t ci[3];
    for (int a = 0; a < 3; ++a) ci[a] = G.cell_of(a, p[a]);
    int64_t best_v = -1;
    double best_d = 0;
    const int64_t rmax = std::max(G.n[0], std::max(G.n[1], G.n[2]));
    for (int64_t r = 0; r <= rmax; ++r) {
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::max<int64_t>(0, ci[a] - r);
            hi[a] = std::min<int64_t>(G.n[a] - 1, ci[a] + r);
        }
        auto scan = [&](int64_t x, int64_t y, int64_t z) {
            const int64_t c = (z * G.n[1] + y) * G.n[0] + x;
            for (int64_t q = G.cell_ptr[c]; q < G.cell_ptr[c + 1]; ++q) {
                const int64_t v = G.ids[q];
                double d = 0;
                for (int k = 0; k < 3; ++k) {
                    const double t = xyz[3 * v + k] - p[k];
                    d += t * t;
                }
                if (best_v < 0 || d < best_d || (d == best_d && v < best_v)) {
                    best_v = v;
                    best_d = d;
                }
            }
        };
        // the cells at Chebyshev distance r from the position's cell: whole
        // rows where y or z is on the shell, else the row's two end cells
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y) {
                if (std::llabs(z - ci[2]) == r || std::llabs(y - ci[1]) == r) {
                    for (int64_t x = lo[0]; x <= hi[0]; ++x) scan(x, y, z);
                } else {
                    if (ci[0] - r >= 0) scan(ci[0] - r, y, z);
                    if (r > 0 && ci[0] + r <= G.n[0] - 1) scan(ci[0] + r, y, z);
                }
            }
        // distance from p to the nearest cell not searched yet (none left: done)
        double bound = HUGE_VAL;
        for (int a = 0; a < 3; ++a) {
            if (ci[a] - r - 1 >= 0) bound = std::min(bound, std::max(0.0, p[a] - (G.lo[a] + (double)(ci[a] - r) * G.h[a])));
            if (ci[a] + r + 1 <= G.n[a] - 1)
                bound = std::min(bound, std::max(0.0, G.lo[a] + (double)(ci[a] + r + 1) * G.h[a] - p[a]));
        }
        if (bound == HUGE_VAL) break;
        // a vertex there is at least `bound` away; the margins cover the
        // rounding of the cell assignment and of the squared distances
        if (best_v >= 0 && bound * bound * (1.0 - 1e-9) > best_d + G.margin2) break;
    }
    return best_v;
}

void map_antennas(const Topology& T, const mwi_antenna* a, int n, std::vector<int32_t>& dof,
                  std::vector<double>& sign) {
    dof.resize(n);
    sign.resize(n);
    for (int k = 0; k < n; ++k) {
        const double* pos = a[k].pos;
        const double* dir = a[k].dir;
        MWI_REQUIRE(std::isfinite(pos[0]) && std::isfinite(pos[1]) && std::isfinite(pos[2]), MWI_EINVAL,
                    "antenna position not finite");
        const double dn = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        MWI_REQUIRE(dn > 0 && std::isfinite(dn), MWI_EINVAL, "antenna direction must be non-zero");
        const int64_t best_v = nearest_vertex(T.xyz, T.vgrid, pos);
        MWI_REQUIRE(best_v >= 0, MWI_EINVAL, "mesh has no vertex");
        int32_t best_e = -1;
        double best_c = -2;
        for (int32_t q = T.v2e_ptr[best_v]; q < T.v2e_ptr[best_v + 1]; ++q) {
            const int32_t e = T.v2e[q];
            const int64_t o = T.edges[2 * e] == best_v ? T.edges[2 * e + 1] : T.edges[2 * e];
            double vec[3], nv = 0, dot = 0;
            for (int d = 0; d < 3; ++d) {
                vec[d] = T.xyz[3 * o + d] - T.xyz[3 * best_v + d];
                nv += vec[d] * vec[d];
                dot += vec[d] * dir[d];
            }
            const double c = dot / (std::sqrt(nv) * dn);
            if (c > best_c) { best_c = c; best_e = e; }
        }
        MWI_REQUIRE(best_e >= 0, MWI_EINVAL, "antenna vertex has no edge");
        MWI_REQUIRE(T.edge_dof[best_e] >= 0, MWI_EINVAL, "antenna falls on a PEC edge");
        double t = 0;
        for (int d = 0; d < 3; ++d)
            t += (T.xyz[3 * (int64_t)T.edges[2 * best_e + 1] + d] - T.xyz[3 * (int64_t)T.edges[2 * best_e] + d]) * dir[d];
        dof[k] = T.edge_dof[best_e];
        sign[k] = t > 0 ? 1.0 : -1.0;
    }
}

}  // namespace mwi

// Host-side data model of the library: mesh topology and DOFs, the ORAS
// decomposition with its slot maps, and the multifrontal symbolic structure.
#pragma once

#include <stdint.h>
#include <vector_types.h>

#include <cmath>
#include <vector>

#include "../../include/mwi.h"

namespace mwi {

// Local entities of a tet whose vertices are sorted by global id.
static const int kLocalEdges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int kLocalFaces[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
static const int kOpposite[4] = {3, 2, 1, 0};

enum { TAG_INTERIOR = 0, TAG_PEC = 1, TAG_IMPEDANCE = 2 };
enum { KIND_WHITNEY = 0, KIND_GRAD = 1, KIND_FACE_A = 2, KIND_FACE_B = 3 };

inline int n_local(int order) { return order == 1 ? 6 : 20; }
inline int n_face_local(int order) { return order == 1 ? 3 : 8; }
inline int n_pack(int nl) { return nl * (nl + 1) / 2; }
// packed index of the symmetric pair (i, j)
inline int pack_idx(int i, int j, int nl) {
    if (i > j) { int t = i; i = j; j = t; }
    return i * nl - i * (i - 1) / 2 + (j - i);
}

// Uniform grid of the mesh vertices for nearest-vertex queries (antenna.cpp):
// cells of about two vertices over the bounding box, the vertices of a cell in
// ascending id.
struct VertexGrid {
    double lo[3] = {0, 0, 0}, h[3] = {1, 1, 1};
    int64_t n[3] = {1, 1, 1};
    double margin2 = 0;             // squared-distance slack of the search's stopping test
    std::vector<int64_t> cell_ptr;  // [cells + 1]
    std::vector<int32_t> ids;       // [nv]
    // cell of coordinate x on axis a, clamped to the grid
    int64_t cell_of(int a, double x) const {
        const double t = std::floor((x - lo[a]) / h[a]);
        if (!(t >= 0)) return 0;
        if (t >= (double)(n[a] - 1)) return n[a] - 1;
        return (int64_t)t;
    }
};

struct Topology {
    int order = 1;
    int nl = 6, nlf = 3;
    int64_t nv = 0, nt = 0, ne = 0, nf = 0, ndof = 0;
    std::vector<double> xyz;          // [nv*3]
    std::vector<double> centroid;     // [nt*3] (((v0 + v1) + v2) + v3) / 4 in the caller's vertex order
    std::vector<int32_t> tv;          // [nt*4] vertices sorted by global id
    std::vector<int32_t> edges;       // [ne*2] (low, high), sorted lexicographically
    std::vector<int32_t> tet_edges;   // [nt*6]
    std::vector<int32_t> faces;       // [nf*3] sorted triples, sorted lexicographically
    std::vector<int32_t> tet_faces;   // [nt*4]
    std::vector<int8_t> face_tag;     // [nf]
    std::vector<int32_t> face_tets;   // [nf*2] (-1 for a boundary face's missing side)
    std::vector<int8_t> face_lf;      // [nf*2] local face index in each tet
    std::vector<uint8_t> pec_edge;    // [ne]
    std::vector<uint8_t> pec_face;    // [nf]
    std::vector<int32_t> tet_dofs;    // [nt*nl] internal DOF id or -1
    std::vector<int32_t> face_dofs;   // [nf*nlf] internal DOF id or -1 (face-local order)
    std::vector<int32_t> edge_dof;    // [ne] Whitney DOF of the edge or -1
    std::vector<int32_t> dof_kind;    // [ndof]
    std::vector<int64_t> dof_verts;   // [ndof*3]
    std::vector<double> dof_pos;      // [ndof*3] edge midpoint / face centroid
    std::vector<int32_t> v2e_ptr, v2e;  // vertex -> incident edges (ascending edge id)
    std::vector<int32_t> v2t_ptr, v2t;  // vertex -> incident tets
    std::vector<int32_t> d2t_ptr, d2t;  // DOF -> (tet*nl + local) incidences, ascending tet
    VertexGrid vgrid;                   // the vertices by grid cell
};

void build_topology(Topology& T, const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                    const int32_t* bface_tag, int order);

// antenna.cpp: the vertex grid; the vertex nearest to p (squared distance
// summed over x, y, z in that order, lowest id on ties; -1 for no vertex); the
// edge DOF and sign of every antenna
void build_vertex_grid(const std::vector<double>& xyz, int64_t nv, VertexGrid& G);
int64_t nearest_vertex(const std::vector<double>& xyz, const VertexGrid& G, const double* p);
void map_antennas(const Topology& T, const mwi_antenna* a, int n, std::vector<int32_t>& dof,
                  std::vector<double>& sign);

// A sparse symmetric pattern with the list of element contributions of every
// stored entry ("slot").  A contribution is encoded in an int64:
//   bits 0..15  packed local pair index
//   bits 16..61 entity (tet id, or face-use id)
//   bit 62      1 for a face-use contribution (kFaceFlag)
struct SlotMatrix {
    int64_t nrows = 0;
    std::vector<int64_t> row_ptr;   // [nrows+1]
    std::vector<int32_t> col;       // [nnz]
    std::vector<int64_t> slot_ptr;  // [nnz+1]
    std::vector<int64_t> contrib;   // [ncontrib]
};

static const int64_t kFaceFlag = (int64_t)1 << 62;

// Face uses: an impedance term i k0 sqrt(eps_t) B_f on face f, with t the tet
// whose eps gives the wavenumber.
struct FaceUses {
    std::vector<int32_t> face;
    std::vector<int32_t> tet;
};

struct Front {
    int32_t sub;      // subdomain
    int32_t start;    // first pivot (local ND index)
    int32_t p;        // pivots
    int32_t u;        // update rows (ancestors' DOFs)
    int32_t parent;   // global front id or -1
    int32_t level;    // 0 = root level of its subdomain tree
    int64_t f_off;    // offset of the f x p panel [L11; L21] in the factor store (entries)
    int64_t sch_off;  // offset of the u x u Schur block in its level's transient buffer
    int64_t u_off;    // offset into the concatenated U lists / relative maps
    int64_t upd_row;  // first row of this front's update vector in the solve buffer
};

struct Decomposition {
    int n_sub = 0, overlap = 1, nd_leaf = 64;
    std::vector<int32_t> part;          // [nt]
    std::vector<int64_t> sub_off;       // [n_sub+1] offsets of the concatenated local vectors
    std::vector<int32_t> loc2glob;      // [nloc] global DOF of each local row (ND order)
    std::vector<double> dweight;        // [nloc] D_i weights
    std::vector<int64_t> own_ptr;       // [ndof+1] scatter list: rows with D > 0 per global DOF
    std::vector<int32_t> own_row;       // local rows
    std::vector<double> own_w;          // their weights
    SlotMatrix B;                       // block-diagonal B_i in local ND numbering
    FaceUses B_faces;
    std::vector<int64_t> fu_off;        // [n_sub+1] offsets of each subdomain's face uses in B_faces
    // multifrontal structure
    std::vector<Front> fronts;          // creation order: per subdomain, children before parents
    std::vector<int32_t> level_ptr;     // [n_levels+1] into level_fronts, deepest level first
    std::vector<int32_t> level_fronts;  // front ids grouped by tree depth
    int n_levels = 0;
    std::vector<int32_t> child_ptr, child;  // children of every front
    std::vector<int32_t> urows;         // [sum u] U lists (local ND index)
    // gather form of the update-vector extend-add of the sweeps: for front
    // row t of front s (index asm_base[s] + t), the rows of the children's
    // update vectors that add into it, children ascending
    std::vector<int64_t> asm_base;      // [nfronts] first front-row index of each front
    std::vector<int64_t> asm_ptr;       // [sum f + 1]
    std::vector<int32_t> asm_src;       // [sum u] row in the update buffer
    std::vector<int32_t> urel;          // [sum u] position of U_c[k] in the parent's front
    std::vector<int64_t> amap_slot;     // front assembly: source slot of B
    std::vector<int64_t> amap_pos;      // destination entry in the front workspace
    std::vector<int64_t> amap_front_ptr;  // [nfronts+1]
    int64_t ws_entries = 0;             // factor store entries (sum f * p)
    std::vector<int64_t> level_sch;     // sum u^2 per level (Schur blocks, transient)
    int64_t sch_entries[2] = {0, 0};    // transient Schur buffer size for even / odd levels
    int64_t upd_rows = 0;               // total update-vector rows
    int64_t factor_entries = 0;         // sum f * p
    double factor_flops = 0;            // real flops of the numeric factorisation
    int32_t max_front = 0;
};

// Two-level ORAS (coarse.cpp): the prolongation P from a coarse mesh's
// Whitney space to the fine DOFs (CSR, and its transpose), and the pattern of
// the Galerkin operator A_c = P^T A P.
struct CoarseHost {
    int64_t n = 0, nc = 0;
    std::vector<int64_t> P_rp, PT_rp, Ac_rp;
    std::vector<int32_t> P_col, PT_col, Ac_col;
    std::vector<double> P_val, PT_val;
};
void build_prolongation(const Topology& fine, const Topology& coarse, CoarseHost& out);
void coarse_pattern(const std::vector<int64_t>& A_rp, const std::vector<int32_t>& A_col, CoarseHost& C);
// A_c values in the pattern's order from A's values (A_rp/A_col: A's CSR)
void coarse_values(const std::vector<int64_t>& A_rp, const std::vector<int32_t>& A_col, const double2* A_val,
                   const CoarseHost& C, std::vector<double2>& out);
// A_c as a decomposition with one subdomain and one dense front (amap_slot
// indexes A_c's values)
void dense_front_decomposition(const CoarseHost& C, Decomposition& D);

// Result of the symbolic analysis of one subdomain (local front ids).
struct LocalFront {
    int32_t start, p, u, parent, level;
    int64_t u_off;  // into LocalSymbolic::urows / urel
};
struct LocalSymbolic {
    std::vector<int32_t> nd_order;   // nd_order[k] = natural index of ND position k
    std::vector<LocalFront> fronts;  // children before parents
    std::vector<int32_t> urows, urel;
    double flops = 0;
};

void rcb_partition(const Topology& T, int nparts, std::vector<int32_t>& part);
void build_decomposition(const Topology& T, const int32_t* part_in, int n_sub, int overlap,
                         int nd_leaf, Decomposition& D);
void build_global_slots(const Topology& T, SlotMatrix& A, FaceUses& fu);
// Nested-dissection ordering and multifrontal structure of one subdomain.
// rows_glob: global DOF of each local row (natural order); adj: local graph
// (natural numbering, no self loops).
void symbolic_subdomain(const Topology& T, int nd_leaf, const std::vector<int32_t>& rows_glob,
                        const std::vector<std::vector<int32_t>>& adj, LocalSymbolic& out);

}  // namespace mwi

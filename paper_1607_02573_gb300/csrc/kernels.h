// Declarations of the device-side data structures and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "common.h"

namespace mwi {

// closed-form element integral tables (see assemble.cu)
struct MTerm { double c; int8_t a, b, pad[6]; };
struct KTerm { double c; int8_t k, gp, l, gq, pad[4]; };
struct FTerm { double c; int8_t a, b, d, pad[5]; };

struct ElementTables {
    int nl = 0, npack = 0, nlf = 0, npack_f = 0;
    std::vector<MTerm> m_terms;
    std::vector<double> mv_c;     // per m_term, 4 coefficients of the lambda_w-weighted mass (w = 0..3)
    std::vector<int32_t> m_ptr;
    std::vector<KTerm> k_terms;
    std::vector<int32_t> k_ptr;
    std::vector<FTerm> f_terms;   // 4 local faces x npack_f pairs
    std::vector<int32_t> f_ptr;
};

struct ElementTablesDev {
    int nl = 0, npack = 0, nlf = 0, npack_f = 0;
    DevBuf<MTerm> m_terms;
    DevBuf<double> mv_c;
    DevBuf<int32_t> m_ptr;
    DevBuf<KTerm> k_terms;
    DevBuf<int32_t> k_ptr;
    DevBuf<FTerm> f_terms;
    DevBuf<int32_t> f_ptr;
};

void build_element_tables(int order, ElementTables& tab);

struct SlotMatrixDev {
    int64_t nrows = 0, nnz = 0;
    DevBuf<int32_t> row_ptr;   // int32 row pointers (nnz < 2^31)
    DevBuf<int32_t> col;
    DevBuf<int64_t> slot_ptr;
    DevBuf<int64_t> contrib;
};

void launch_elem_geom(const double* xyz, const int32_t* tv, int64_t nt, const ElementTablesDev& tab,
                      double* K, double* M, cudaStream_t st);
void launch_face_geom(const double* xyz, const int32_t* tv, const int32_t* face_tets, const int8_t* face_lf,
                      int64_t nf, const ElementTablesDev& tab, double* Bf, cudaStream_t st);
void launch_face_coef(const int32_t* fu_tet, int64_t nfu, const double2* eps, double k0, double2* coef,
                      cudaStream_t st);
// Mk (nullable): per-tet complex mass sum_w kappa_w M_t^(w) [nt][npack] of a nodal
// parameter, used in place of eps_t M_t
void launch_slot_fill(const SlotMatrixDev& S, const double* K, const double* M, int npack, const double* Bf,
                      int npack_f, const int32_t* fu_face, const double2* fu_coef, const double2* eps, double k0,
                      double2* out64, float2* out32, cudaStream_t st, const double2* Mk = nullptr);
// vertex-weighted element masses Mv[t][w][pair] = int_t lambda_w N_i . N_j
void launch_elem_vertex_mass(const double* xyz, const int32_t* tv, int64_t nt, const ElementTablesDev& tab,
                             double* Mv, cudaStream_t st);

// ---- multifrontal factorisation and ORAS application (factor.cu, sweep.cu, oras.cu)
// One GEMM tile of the sweeps: the front's geometry and the tile's first row.
struct __align__(16) TileDesc {
    int64_t a_off;     // panel offset in the factor store
    int64_t rowbase;   // local row of the front's first pivot
    int64_t sbase;     // local row of the subdomain's first row
    int64_t upd_row;   // first row of the front's update vector
    int64_t asm_base;  // first gather-table row of the front
    int64_t u_off;     // first entry of the front's update-row list
    int32_t p, f, row0, pad;
};

// GEMM tiles of the sweeps per level, over the p pivot rows (backward product,
// extend-add) and over all f = p + u front rows (forward product).
struct TileLists {
    int tm = 0;
    DevBuf<TileDesc> p_tiles, f_tiles;
    std::vector<int64_t> p_ptr, f_ptr;  // [n_levels+1]
};

struct FrontsDev {
    int64_t nfronts = 0;
    // tensor-core sweeps (sweep_tc.cu): 128-row tiles whose a_off is the
    // front's offset in each tiled copy of the panels (floats), the per-front
    // offsets, the (front, 32-row block) list of the packing kernel, and the
    // floats of one copy (the store holds the forward then the backward copy)
    TileLists tiles128;
    DevBuf<int64_t> t_off;
    DevBuf<int2> pack_blocks;
    int64_t n_pack_blocks = 0, tiled_floats = 0;
    DevBuf<int32_t> start, p, u, parent, sub;
    DevBuf<int64_t> f_off, u_off, upd_row, sch_off;
    DevBuf<int32_t> child_ptr, child;
    DevBuf<int32_t> urows, urel;
    DevBuf<int64_t> asm_base, asm_ptr;   // gather lists of the sweeps' extend-add
    DevBuf<int32_t> asm_src;
    DevBuf<int2> asm2;                   // the same lists as (source, source) per front row, -1 = none
    // extend-add tiles (front, child, first of four child rows), per level and
    // chunk of 65535 fronts: first children, then second children
    DevBuf<int4> ext_tiles;
    std::vector<int64_t> ext_ptr;
    DevBuf<int64_t> amap_front_ptr, amap_slot, amap_pos;
    DevBuf<int32_t> level_fronts;
    std::vector<int32_t> level_ptr;   // host copy
    std::vector<int32_t> level_pmax;  // host: max p per level
    std::vector<int32_t> level_fmax;  // host: max front size per level
    std::vector<int32_t> level_umax;
    DevBuf<int64_t> sub_off;
    DevBuf<int32_t> loc2glob;
    DevBuf<int64_t> own_ptr;
    DevBuf<int32_t> own_row;
    DevBuf<double> own_w;
    // factor store: ws_entries panel entries, then D^{-1} for the nloc local rows
    int64_t nloc = 0, upd_rows = 0, ws_entries = 0;
    int64_t ws_total() const { return ws_entries + nloc; }
    std::vector<int64_t> level_sch;    // host: sum u^2 of each level
    int64_t sch_entries[2] = {0, 0};
    int n_sub = 0;
    TileLists tiles64, tiles32;        // 64-row and 32-row tiles of every level
    std::vector<double> level_pmean, level_fmean;  // host: mean p and f of each level
    DevBuf<int64_t> inv_off;           // per level position: offset of the front's f x p block
    int64_t inv_entries = 0;           // largest sum of f p over a level
};

// Trailing-update tiles (front, tile row, tile column <= row) of every step
// of the blocked factorisation, in the order the factorisation consumes them
// (levels, chunks of 65535 fronts, steps of nb pivot columns); ptr holds the
// ranges.
struct UpdateTiles {
    int nb = 0, tile = 0;
    DevBuf<int4> tiles;
    std::vector<int64_t> ptr;
    // panel-row tiles (front, first row) of 128 rows below each step's diagonal block
    DevBuf<int2> rtiles;
    std::vector<int64_t> rptr;
};
int factor_block_cols(bool fp32);
int factor_tile_rows(bool fp32);

// ws: factor store (panels); sch[2]: transient Schur buffers (even / odd levels)
template <typename C>
void factorize_fronts(const FrontsDev& F, const UpdateTiles& ut, const double2* Bvals, C* ws, C* const sch[2],
                      C* inv_tmp, int* perturbed, cudaStream_t st);

// Complex FP32 sweep engine: tc = 0 CUDA cores, 1 mma.sync 3xTF32, 2 mma.sync
// TF32, 4 tcgen05 TF32 over the tiled panel store wt (err: the kernels'
// bounded-wait error code, 0 = none)
struct SweepCfg {
    int tc = 0;
    const float* wt = nullptr;
    int* err = nullptr;
};

// y = M^{-1} x; scratch: Y, Z [nloc][m], upd [upd_rows][m]
template <typename C>
void oras_apply(const FrontsDev& F, const C* ws, const double2* x, double2* y, int m, C* Y, C* Z, C* upd,
                cudaStream_t st, const float2* x32 = nullptr, float2* y32 = nullptr, const SweepCfg& sc = SweepCfg());

template <typename C>
void multifrontal_solve(const FrontsDev& F, const C* ws, C* Y, C* Z, C* upd, int m, const SweepCfg& sc,
                        cudaStream_t st);
int sweep_tile_rows(bool fp32);
// columns of the ORAS local vectors for m right-hand sides (even for tc 4)
int sweep_ld(int m, int tc);

// tensor-core sweeps (sweep_tc.cu)
int64_t tiled_panel_floats(int p, int f);
// both tiled copies: the forward one at wt, the backward one at wt + bwd_base
void pack_tiled(const int2* blocks, int64_t nblocks, const int64_t* f_off, const int64_t* t_off, const int32_t* P,
                const int32_t* U, const float2* ws, float* wt, int64_t bwd_base, cudaStream_t st);
void sweep_tc_level(bool backward, const TileDesc* tiles, int64_t ntiles, int m, const int32_t* urows,
                    const int2* asm2, const float* wt, const float2* dinv, float2* Y, float2* Z, float2* upd,
                    int* err, cudaStream_t st);

// Allocation-free ORAS application (oras.cu): scratch from a fixed-size
// file-scope device array of kOrasScratchBytes.
static const size_t kOrasScratchBytes = (size_t)32 << 20;
size_t oras_noalloc_bytes(const FrontsDev& F, int64_t n, int m, bool mixed);
void oras_apply_noalloc(const FrontsDev& F, const void* ws, bool mixed, const double2* x, double2* y, int m,
                        int64_t n, cudaStream_t st, const SweepCfg& sc = SweepCfg());

// ---- two-level ORAS (twolevel.cu): prolongation P [n][nc] and its transpose (CSR, real)
struct CoarseDev {
    int64_t n = 0, nc = 0;
    DevBuf<int64_t> P_rp, PT_rp;
    DevBuf<int32_t> P_col, PT_col;
    DevBuf<double> P_val, PT_val;
};
// scratch of one application: coarse vectors ct, cq [nc][m]; fine vectors q, w [n][m]
template <typename C>
struct TwoLevelScratch {
    C *ct = nullptr, *cq = nullptr, *q = nullptr, *w = nullptr;
};
// y = M_ORAS (x - A Q x) + Q x with Q = P A_c^{-1} P^T; coarse_solve(t, c): c = A_c^{-1} t,
// one_level(w, z): z = M_ORAS w; A in CSR with int32 row pointers
template <typename C>
void two_level_apply(const CoarseDev& cd, const C* x, C* y, int m, const TwoLevelScratch<C>& s,
                     const std::function<void(const C*, C*)>& coarse_solve,
                     const std::function<void(const C*, C*)>& one_level, const int32_t* A_rp, const int32_t* A_col,
                     const C* A_val, cudaStream_t st);

// ---- nodal (P1) permittivity parameter (p1.cu)
struct Topology;
void build_p1_stiffness(const Topology& T, std::vector<int32_t>& rp, std::vector<int32_t>& col,
                        std::vector<double>& val);
// eps_t = kappa at the tet's centroid; Mk[t][p] = sum_w kappa_{v_w(t)} Mv[t][w][p]
void launch_p1_centroid(int64_t nt, const int32_t* tv, const double2* kappa, double2* eps, cudaStream_t st);
void launch_p1_mass(int64_t nt, int npack, const int32_t* tv, const double2* kappa, const double* Mv, double2* Mk,
                    cudaStream_t st);
// per (tet, local vertex): conj of k0^2 sum_j lam^T M_t^(w) u + 1/4 of the tet's beta term
void launch_p1_tet_gradient(int order, int64_t nt, int m, const int32_t* tet_dofs, const int32_t* tet_faces,
                            const int8_t* face_tag, const int32_t* face_dofs, const double* Mv, const double* Bf,
                            const double2* eps, double k0, const double2* U, const double2* Lam, double2* out_tw,
                            cudaStream_t st);
// the same for the mixed path and first order, the volume terms in double-float:
// U and Lam as double-float planes ([2][nm] complex pairs), Mvdf the vertex
// masses as double-float pairs [nt][4][21]
void launch_p1_tet_gradient_df(int64_t nt, int m, int64_t nm, const int32_t* tet_dofs, const int32_t* tet_faces,
                               const int8_t* face_tag, const int32_t* face_dofs, const float2* Mvdf,
                               const double* Bf, const double2* eps, double k0, const double2* U, const double2* Lam,
                               const float2* Udf, const float2* Ldf, double2* out_tw, cudaStream_t st);
int p1_gradient_blocks(int64_t nv);
// per vertex: the (tet, vertex) gradients of its tets plus alpha K kappa;
// partial[block] = the block's sum of Re(conj(kappa_v) (K kappa)_v)
void launch_p1_gradient(int64_t nv, const int32_t* v2t_ptr, const int32_t* v2t, const int32_t* tv,
                        const double2* grad_tw, const int32_t* rp, const int32_t* col, const double* val,
                        const double2* kappa, double alpha, double2* out, double* partial, cudaStream_t st);
// number of entries of a complex array with a non-finite part, into *count (device)
void launch_count_nonfinite(int64_t n, const double2* x, int* count, cudaStream_t st);

// ---- Krylov building blocks (krylov.cu)
template <typename C>
void spmm(int64_t n, const int32_t* row_ptr, const int32_t* col, const C* val, const C* x, C* y, int m,
          cudaStream_t st);

// Initial guess from a recycled subspace: x0 = X_rec Y with
// Y = argmin ||B - C Y|| (C = A X_rec; X_rec, C [n][k], k <= 64; B, x0 [n][m],
// m <= 32), FP32 products, FP64 chunk sums, the k x k normal equations by
// Cholesky on the host.  scratch holds recycle_scratch_entries(k, m) entries.
// Returns the number of recycled columns left out as numerically dependent.
constexpr int kRecycleChunks = 1216;
size_t recycle_scratch_entries(int k, int m);
int recycle_initial_guess(int64_t n, int k, int m, const float2* X32, const float2* C32, const float2* B32,
                          float2* x0, double2* scratch, cudaStream_t st);

}  // namespace mwi

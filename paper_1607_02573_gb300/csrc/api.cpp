// The C ABI (include/mwi.h): handle management and the orchestration of the
// hot path -- assemble, batched factorisation, pseudo-block FGMRES + ORAS,
// S-parameters, misfit, adjoint solve and gradient.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>

#include "common.h"
#include "gmres.h"
#include "kernels.h"
#include "model.h"
#include "physics.h"

namespace mwi {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }
std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_device_allocs{0};

static const double kPi = 3.14159265358979323846;
static const double kC0 = 299792458.0;
static const double kMu0 = 4.0e-7 * kPi;

struct DecompEntry {
    int n_sub, overlap, nd_leaf;
    std::vector<int32_t> part_key;  // empty = RCB
    Decomposition D;
    FrontsDev F;
    SlotMatrixDev B;
    DevBuf<int32_t> fu_face, fu_tet;
    UpdateTiles ut[2];               // trailing-update tiles: [0] complex FP32, [1] complex FP64
    std::once_flag ut_once[2];
};

// Two-level ORAS of one problem: the prolongation and the pattern of
// A_c = P^T A P (host), A_c as one dense front with its factors in the
// problem's precision, and the scratch of the coarse solves and corrections.
struct CoarseLevel {
    CoarseHost H;
    Decomposition D;
    FrontsDev F;
    UpdateTiles ut;
    CoarseDev dev;
    std::vector<double2> Aval_h, Ac_h;
    DevBuf<double2> Ac;
    DevBuf<double2> ws64, inv64, sch64[2];
    DevBuf<float2> ws32, inv32, sch32[2];
    DevBuf<double2> Y64, Z64, upd64, ct64, cq64, q64, w64;
    DevBuf<float2> Y32, Z32, upd32, ct32, cq32, q32, w32;
    DevBuf<int> perturbed;
    int n_perturbed = 0;
    double setup_ms = 0;
    size_t bytes() const {
        size_t b = dev.P_rp.bytes() + dev.PT_rp.bytes() + dev.P_col.bytes() + dev.PT_col.bytes() +
                   dev.P_val.bytes() + dev.PT_val.bytes() + Ac.bytes() + ws64.bytes() + inv64.bytes() +
                   ws32.bytes() + inv32.bytes() + Y64.bytes() + Z64.bytes() + upd64.bytes() + ct64.bytes() +
                   cq64.bytes() + q64.bytes() + w64.bytes() + Y32.bytes() + Z32.bytes() + upd32.bytes() +
                   ct32.bytes() + cq32.bytes() + q32.bytes() + w32.bytes() + perturbed.bytes() + ut.tiles.bytes() +
                   ut.rtiles.bytes();
        for (int k = 0; k < 2; ++k) b += sch64[k].bytes() + sch32[k].bytes();
        return b;
    }
};

// The factorisation's trailing-update tiles, in its consumption order: per
// level, per chunk of at most 65535 fronts, per step k of nb pivot columns,
// the lower-triangle tiles of every front of the chunk with k < p.
void build_update_tiles(const Decomposition& D, int nb, int tile, UpdateTiles& ut, cudaStream_t st) {
    std::vector<int4> t;
    std::vector<int2> rt;
    ut.nb = nb;
    ut.tile = tile;
    ut.ptr.assign(1, 0);
    ut.rptr.assign(1, 0);
    for (int l = 0; l < D.n_levels; ++l) {
        const int lo0 = D.level_ptr[l], hi = D.level_ptr[l + 1];
        int pmax = 0;
        for (int q = lo0; q < hi; ++q) pmax = std::max(pmax, D.fronts[D.level_fronts[q]].p);
        for (int lo = lo0; lo < hi; lo += 65535) {
            const int nf = std::min(65535, hi - lo);
            for (int k = 0; k < pmax; k += nb) {
                for (int q = lo; q < lo + nf; ++q) {
                    const int s = D.level_fronts[q];
                    const Front& fr = D.fronts[s];
                    if (k >= fr.p) continue;
                    const int64_t nrem = (int64_t)fr.p + fr.u - k - std::min(nb, fr.p - k);
                    const int T = (int)((nrem + tile - 1) / tile);
                    for (int bi = 0; bi < T; ++bi)
                        for (int bj = 0; bj <= bi; ++bj) t.push_back(make_int4(s, bi, bj, 0));
                    for (int r = k + std::min(nb, fr.p - k); r < fr.p + fr.u; r += 128) rt.push_back(make_int2(s, r));
                }
                ut.ptr.push_back((int64_t)t.size());
                ut.rptr.push_back((int64_t)rt.size());
            }
        }
    }
    if (t.empty()) t.push_back(make_int4(0, 0, 0, 0));
    if (rt.empty()) rt.push_back(make_int2(0, 0));
    ut.tiles.upload(t, st);
    ut.rtiles.upload(rt, st);
    MWI_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
static void up(DevBuf<T>& d, const std::vector<T>& h, cudaStream_t st) { d.upload(h, st); }

}  // namespace mwi

using namespace mwi;

struct mwi_mesh {
    Topology T;
    int refcount = 0;
    cudaStream_t st = nullptr;  // internal stream for setup work
    DevBuf<double> xyz, Kp, Mp, Bf;
    DevBuf<float2> Mdf;  // element masses as double-float pairs (first order, built on first use)
    DevBuf<int32_t> tv, tet_dofs, face_dofs, tet_faces, face_tets;
    DevBuf<int8_t> face_lf, face_tag;
    ElementTablesDev tabs;
    bool have_A = false;
    SlotMatrix A_host;
    SlotMatrixDev A;
    FaceUses A_fu;
    DevBuf<int32_t> A_fu_face, A_fu_tet;
    std::vector<std::shared_ptr<DecompEntry>> cache;
    std::mutex mu;
    // nodal (P1) parameter: vertex -> tets, P1 stiffness, vertex-weighted element
    // masses (built on first use)
    bool have_p1 = false;
    DevBuf<int32_t> v2t_ptr, v2t, p1_rp, p1_col;
    DevBuf<double> p1_val, Mv;
    DevBuf<float2> Mvdf;  // Mv as double-float pairs (first order, built on first mixed use)
};

struct mwi_problem {
    mwi_mesh* mesh = nullptr;
    std::shared_ptr<DecompEntry> dec;
    cudaStream_t st = nullptr;
    mwi_solver_opts opts;
    double freq = 0, k0 = 0;
    DevBuf<double2> eps, A_coef, B_coef, Aval, Bval;
    DevBuf<float2> Aval32;
    DevBuf<double2> ws64, inv64, sch64[2];
    DevBuf<float2> ws32, inv32, sch32[2];
    DevBuf<float> wt;        // tiled, swizzled copy of the c64 panels (tensor-core sweeps)
    DevBuf<int> sweep_err;   // error code of the tensor-core sweeps' bounded waits
    DevBuf<int> perturbed;
    int n_perturbed = 0;
    // solve state
    DevBuf<double2> Y64, Z64, upd64;
    DevBuf<float2> Y32, Z32, upd32;
    Gmres<double2> outer;
    Gmres<float2> inner;
    GmresDF dfk;                         // MIXED: double-float FGMRES
    BlockGmres bgm;                      // true block FGMRES (block_krylov = 1)
    // recycling: columns of the resident forward (0) / adjoint (1) solution usable
    // as the recycled space of the next solve (0 = none)
    int rec_m[2] = {0, 0};
    int rec_dropped = 0;
    DevBuf<double2> rc_scratch, rc_block;
    int reuse_count = 0;  // eps_r updates since the factors were computed
    // nodal parameter (mwi_update_kappa_device): kappa per vertex, the per-tet
    // complex masses sum_w kappa_w M_t^(w) used by the assembly, the (tet,
    // vertex) gradient terms and the penalty's block sums
    bool p1 = false;
    DevBuf<double2> kappa, Mk, grad_tw;
    DevBuf<double> p1_partial;
    std::vector<double> p1_partial_host;
    DevBuf<int> nonfinite;
    DevBuf<float2> Adf, Bdf, Xdf, Rdf;   // double-float planes
    DevBuf<double2> U, Lam, Brhs, R, Bc, Xc;
    DevBuf<float2> v32, x32, r32;
    DevBuf<double> dscratch;
    int m_fwd = 0;
    bool have_fwd = false, have_adj = false;
    std::vector<int32_t> rx_dof, tx_dof;
    std::vector<double> rx_sign, tx_sign;
    std::vector<mwi_antenna> tx_key, rx_key;  // the antennas tx_dof / rx_dof (and their device copies) map
    DevBuf<int32_t> rx_dof_d, tx_dof_d;
    DevBuf<double> rx_sign_d, tx_sign_d;
    DevBuf<double2> cur_d, S_d, Smeas_d, r_d, grad_d;
    DevBuf<double> w_d, J_d;
    std::unique_ptr<CoarseLevel> coarse;  // two-level ORAS (mwi_set_coarse_space)
    int n_rx = 0;
    double setup_ms = 0;
    int inner_total = 0;
    // per-kernel timing (opts.verbose >= 2): event pairs recorded without
    // synchronisation, harvested by mwi_kernel_times
    double t_ms[4] = {0, 0, 0, 0};
    int64_t t_cnt[4] = {0, 0, 0, 0};
    struct EvPair { cudaEvent_t a, b; int slot; };
    std::vector<EvPair> ev_used;
    std::vector<cudaEvent_t> ev_free;
    ~mwi_problem() {
        for (auto& e : ev_used) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
        for (auto e : ev_free) cudaEventDestroy(e);
    }
    // device bytes held by this problem (the mesh and its decomposition are shared)
    size_t device_bytes() const {
        size_t b = eps.bytes() + A_coef.bytes() + B_coef.bytes() + Aval.bytes() + Bval.bytes() + Aval32.bytes() +
                   ws64.bytes() + inv64.bytes() + ws32.bytes() + inv32.bytes() + perturbed.bytes() + Y64.bytes() +
                   Z64.bytes() + upd64.bytes() + Y32.bytes() + Z32.bytes() + upd32.bytes() + outer.bytes() +
                   inner.bytes() + dfk.bytes() + bgm.bytes() + rc_scratch.bytes() + rc_block.bytes() + Adf.bytes() +
                   Bdf.bytes() + Xdf.bytes() + Rdf.bytes() + U.bytes() + Lam.bytes() + Brhs.bytes() + R.bytes() +
                   Bc.bytes() + Xc.bytes() + v32.bytes() + x32.bytes() + r32.bytes() + dscratch.bytes() +
                   rx_dof_d.bytes() + tx_dof_d.bytes() + rx_sign_d.bytes() + tx_sign_d.bytes() + cur_d.bytes() +
                   S_d.bytes() + Smeas_d.bytes() + r_d.bytes() + grad_d.bytes() + w_d.bytes() + J_d.bytes() +
                   kappa.bytes() + Mk.bytes() + grad_tw.bytes() + p1_partial.bytes() + nonfinite.bytes() +
                   wt.bytes() + sweep_err.bytes();
        for (int k = 0; k < 2; ++k) b += sch64[k].bytes() + sch32[k].bytes();
        if (coarse) b += coarse->bytes();
        return b;
    }
};

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

mwi_solver_opts defaults(const mwi_solver_opts* o) {
    mwi_solver_opts d;
    std::memset(&d, 0, sizeof(d));
    if (o) d = *o;
    if (d.rtol <= 0) d.rtol = 1e-6;
    if (d.max_iter <= 0) d.max_iter = 500;
    if (d.restart <= 0) d.restart = 50;
    if (d.n_sub <= 0) d.n_sub = 64;
    if (d.overlap == 0) d.overlap = 1;
    else if (d.overlap < 0) d.overlap = 0;
    if (d.inner_iters <= 0) d.inner_iters = 30;
    if (d.inner_rtol <= 0) d.inner_rtol = 1e-4;
    if (d.nd_leaf <= 0) d.nd_leaf = 128;
    if (d.max_block <= 0) d.max_block = 64;
    if (d.sweep_engine <= 0) d.sweep_engine = 4;
    if (d.block_krylov < 0 || d.block_krylov > 1) throw Error(MWI_EINVAL, "block_krylov must be 0 or 1");
    if (d.recycle < 0 || d.recycle > 1) throw Error(MWI_EINVAL, "recycle must be 0 or 1");
    if (d.factor_reuse < 0) throw Error(MWI_EINVAL, "factor_reuse must be >= 0");
    return d;
}

cudaEvent_t take_event(mwi_problem* P) {
    if (!P->ev_free.empty()) {
        cudaEvent_t e = P->ev_free.back();
        P->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    MWI_CUDA(cudaEventCreate(&e));
    return e;
}

// complex FP32 sweep engine: 0 CUDA cores, 1 tensor cores 3xTF32, 2 tensor cores TF32
int tc_of(const mwi_solver_opts& o) { return o.sweep_engine == 3 ? 0 : o.sweep_engine; }

// the complex FP32 sweeps of this problem: engine, tiled panels and error flag
// of the tensor-core engine
SweepCfg sweep_cfg(const mwi_problem* P) {
    SweepCfg c;
    c.tc = tc_of(P->opts);
    c.wt = P->wt.p;
    c.err = P->sweep_err.p;
    return c;
}

// a tensor-core sweep whose bounded wait expired reports it here (read after a solve)
void check_sweep_error(mwi_problem* P) {
    if (tc_of(P->opts) != 4 || !P->sweep_err.p) return;
    int code = 0;
    MWI_CUDA(cudaMemcpyAsync(&code, P->sweep_err.p, sizeof(int), cudaMemcpyDeviceToHost, P->st));
    MWI_CUDA(cudaStreamSynchronize(P->st));
    if (code) {
        MWI_CUDA(cudaMemsetAsync(P->sweep_err.p, 0, sizeof(int), P->st));
        throw Error(MWI_ETIMEOUT, "tensor-core sweep: a bounded wait expired (role " + std::to_string(code) + ")");
    }
}

// timed region helper: records an event pair around fn when enabled
template <typename Fn>
void timed(mwi_problem* P, int slot, Fn&& fn) {
    if (P->opts.verbose < 2) { fn(); return; }
    cudaEvent_t a = take_event(P), b = take_event(P);
    MWI_CUDA(cudaEventRecord(a, P->st));
    fn();
    MWI_CUDA(cudaEventRecord(b, P->st));
    P->ev_used.push_back({a, b, slot});
}

void harvest_events(mwi_problem* P) {
    if (P->ev_used.empty()) return;
    MWI_CUDA(cudaStreamSynchronize(P->st));
    for (auto& e : P->ev_used) {
        float ms = 0;
        MWI_CUDA(cudaEventElapsedTime(&ms, e.a, e.b));
        P->t_ms[e.slot] += ms;
        P->t_cnt[e.slot] += 1;
        P->ev_free.push_back(e.a);
        P->ev_free.push_back(e.b);
    }
    P->ev_used.clear();
}

// finiteness of a complex device array (host arrays are checked on the host)
void check_finite_device(mwi_problem* P, const double2* x, int64_t n, const char* what) {
    P->nonfinite.ensure(1);
    MWI_CUDA(cudaMemsetAsync(P->nonfinite.p, 0, sizeof(int), P->st));
    launch_count_nonfinite(n, x, P->nonfinite.p, P->st);
    int bad = 0;
    MWI_CUDA(cudaMemcpyAsync(&bad, P->nonfinite.p, sizeof(int), cudaMemcpyDeviceToHost, P->st));
    MWI_CUDA(cudaStreamSynchronize(P->st));
    MWI_REQUIRE(bad == 0, MWI_EINVAL, std::string(what) + " not finite (" + std::to_string(bad) + " entries)");
}

void build_mesh_device(mwi_mesh* M) {
    Topology& T = M->T;
    cudaStream_t st = M->st;
    up(M->xyz, T.xyz, st);
    up(M->tv, T.tv, st);
    up(M->tet_dofs, T.tet_dofs, st);
    up(M->face_dofs, T.face_dofs, st);
    up(M->tet_faces, T.tet_faces, st);
    up(M->face_tets, T.face_tets, st);
    up(M->face_lf, T.face_lf, st);
    up(M->face_tag, T.face_tag, st);
    ElementTables tab;
    build_element_tables(T.order, tab);
    M->tabs.nl = tab.nl;
    M->tabs.npack = tab.npack;
    M->tabs.nlf = tab.nlf;
    M->tabs.npack_f = tab.npack_f;
    up(M->tabs.m_terms, tab.m_terms, st);
    up(M->tabs.mv_c, tab.mv_c, st);
    up(M->tabs.m_ptr, tab.m_ptr, st);
    up(M->tabs.k_terms, tab.k_terms, st);
    up(M->tabs.k_ptr, tab.k_ptr, st);
    up(M->tabs.f_terms, tab.f_terms, st);
    up(M->tabs.f_ptr, tab.f_ptr, st);
    M->Kp.alloc((size_t)T.nt * tab.npack);
    M->Mp.alloc((size_t)T.nt * tab.npack);
    M->Bf.alloc((size_t)T.nf * tab.npack_f);
    launch_elem_geom(M->xyz.p, M->tv.p, T.nt, M->tabs, M->Kp.p, M->Mp.p, st);
    launch_face_geom(M->xyz.p, M->tv.p, M->face_tets.p, M->face_lf.p, T.nf, M->tabs, M->Bf.p, st);
    MWI_CUDA(cudaStreamSynchronize(st));
}

void upload_slots(const SlotMatrix& S, SlotMatrixDev& D, cudaStream_t st) {
    D.nrows = S.nrows;
    D.nnz = (int64_t)S.col.size();
    MWI_REQUIRE(D.nnz < ((int64_t)1 << 31), MWI_EINVAL, "matrix too large for int32 row pointers");
    std::vector<int32_t> rp(S.row_ptr.begin(), S.row_ptr.end());
    D.row_ptr.upload(rp, st);
    D.col.upload(S.col, st);
    D.slot_ptr.upload(S.slot_ptr, st);
    D.contrib.upload(S.contrib, st);
}

void ensure_global(mwi_mesh* M) {
    if (M->have_A) return;
    build_global_slots(M->T, M->A_host, M->A_fu);
    upload_slots(M->A_host, M->A, M->st);
    up(M->A_fu_face, M->A_fu.face, M->st);
    up(M->A_fu_tet, M->A_fu.tet, M->st);
    MWI_CUDA(cudaStreamSynchronize(M->st));
    M->have_A = true;
}

void upload_fronts(const Decomposition& D, FrontsDev& F, cudaStream_t st);

std::shared_ptr<DecompEntry> get_decomp(mwi_mesh* M, const mwi_solver_opts& o) {
    std::vector<int32_t> key;
    if (o.part) key.assign(o.part, o.part + M->T.nt);
    for (auto& e : M->cache)
        if (e->n_sub == o.n_sub && e->overlap == o.overlap && e->nd_leaf == o.nd_leaf && e->part_key == key)
            return e;
    auto E = std::make_shared<DecompEntry>();
    E->n_sub = o.n_sub;
    E->overlap = o.overlap;
    E->nd_leaf = o.nd_leaf;
    E->part_key = key;
    build_decomposition(M->T, o.part, o.n_sub, o.overlap, o.nd_leaf, E->D);
    Decomposition& D = E->D;
    cudaStream_t st = M->st;
    upload_slots(D.B, E->B, st);
    up(E->fu_face, D.B_faces.face, st);
    up(E->fu_tet, D.B_faces.tet, st);
    upload_fronts(D, E->F, st);
    M->cache.push_back(E);
    return E;
}

// the multifrontal structure of a decomposition on the device: fronts, extend-add
// and assembly lists, the sweeps' tile lists and the tiled-panel offsets
void upload_fronts(const Decomposition& D, FrontsDev& F, cudaStream_t st) {
    const size_t nf = D.fronts.size();
    F.nfronts = (int64_t)nf;
    std::vector<int32_t> start(nf), p(nf), u(nf), parent(nf), sub(nf);
    std::vector<int64_t> f_off(nf), u_off(nf), upd_row(nf), sch_off(nf);
    for (size_t k = 0; k < nf; ++k) {
        const Front& fr = D.fronts[k];
        start[k] = fr.start; p[k] = fr.p; u[k] = fr.u; parent[k] = fr.parent; sub[k] = fr.sub;
        f_off[k] = fr.f_off; u_off[k] = fr.u_off; upd_row[k] = fr.upd_row; sch_off[k] = fr.sch_off;
    }
    up(F.start, start, st); up(F.p, p, st); up(F.u, u, st); up(F.parent, parent, st); up(F.sub, sub, st);
    up(F.f_off, f_off, st); up(F.u_off, u_off, st); up(F.upd_row, upd_row, st); up(F.sch_off, sch_off, st);
    up(F.child_ptr, D.child_ptr, st); up(F.child, D.child, st);
    up(F.urows, D.urows, st); up(F.urel, D.urel, st);
    up(F.asm_base, D.asm_base, st); up(F.asm_ptr, D.asm_ptr, st); up(F.asm_src, D.asm_src, st);
    {
        // every front row receives at most one row from each of its (at most two) children
        const int64_t rows = (int64_t)D.asm_ptr.size() - 1;
        std::vector<int2> a2(std::max<int64_t>(1, rows), make_int2(-1, -1));
        for (int64_t r = 0; r < rows; ++r) {
            const int64_t q0 = D.asm_ptr[r], q1 = D.asm_ptr[r + 1];
            MWI_REQUIRE(q1 - q0 <= 2, MWI_EINVAL, "internal: more than two extend-add sources for a front row");
            if (q1 > q0) a2[r].x = D.asm_src[q0];
            if (q1 > q0 + 1) a2[r].y = D.asm_src[q0 + 1];
        }
        up(F.asm2, a2, st);
    }
    {
        std::vector<int4> et;
        F.ext_ptr.assign(1, 0);
        for (int l = 0; l < D.n_levels; ++l)
            for (int lo = D.level_ptr[l]; lo < D.level_ptr[l + 1]; lo += 65535) {
                const int nf = std::min(65535, D.level_ptr[l + 1] - lo);
                for (int ci = 0; ci < 2; ++ci) {
                    for (int q = lo; q < lo + nf; ++q) {
                        const int sid = D.level_fronts[q];
                        if (D.child_ptr[sid] + ci >= D.child_ptr[sid + 1]) continue;
                        const int c = D.child[D.child_ptr[sid] + ci];
                        for (int b = 0; b < D.fronts[c].u; b += 4) et.push_back(make_int4(sid, c, b, 0));
                    }
                    F.ext_ptr.push_back((int64_t)et.size());
                }
            }
        if (et.empty()) et.push_back(make_int4(0, 0, 0, 0));
        up(F.ext_tiles, et, st);
    }
    up(F.amap_front_ptr, D.amap_front_ptr, st); up(F.amap_slot, D.amap_slot, st); up(F.amap_pos, D.amap_pos, st);
    up(F.level_fronts, D.level_fronts, st);
    F.level_ptr = D.level_ptr;
    const int nlev = D.n_levels;
    F.level_pmax.assign(nlev, 0);
    F.level_fmax.assign(nlev, 0);
    F.level_umax.assign(nlev, 0);
    F.level_pmean.assign(nlev, 0.0);
    F.level_fmean.assign(nlev, 0.0);
    for (int l = 0; l < nlev; ++l)
        for (int q = D.level_ptr[l]; q < D.level_ptr[l + 1]; ++q) {
            const Front& fr = D.fronts[D.level_fronts[q]];
            F.level_pmax[l] = std::max(F.level_pmax[l], fr.p);
            F.level_fmax[l] = std::max(F.level_fmax[l], fr.p + fr.u);
            F.level_umax[l] = std::max(F.level_umax[l], fr.u);
            F.level_pmean[l] += fr.p;
            F.level_fmean[l] += fr.p + fr.u;
        }
    for (int l = 0; l < nlev; ++l) {
        const double cnt = std::max(1, D.level_ptr[l + 1] - D.level_ptr[l]);
        F.level_pmean[l] /= cnt;
        F.level_fmean[l] /= cnt;
    }
    up(F.sub_off, D.sub_off, st);
    up(F.loc2glob, D.loc2glob, st);
    up(F.own_ptr, D.own_ptr, st);
    up(F.own_row, D.own_row, st);
    up(F.own_w, D.own_w, st);
    F.nloc = D.sub_off[D.n_sub];
    F.upd_rows = D.upd_rows;
    F.ws_entries = D.ws_entries;
    F.level_sch = D.level_sch;
    F.sch_entries[0] = D.sch_entries[0];
    F.sch_entries[1] = D.sch_entries[1];
    F.n_sub = D.n_sub;
    // GEMM tile lists of the sweeps and per-level offsets of the inverse scratch
    for (int pass = 0; pass < 2; ++pass) {
        TileLists& TL = pass == 0 ? F.tiles64 : F.tiles32;
        TL.tm = sweep_tile_rows(pass == 0);
        std::vector<TileDesc> pt, ft;
        TL.p_ptr.assign(1, 0);
        TL.f_ptr.assign(1, 0);
        for (int l = 0; l < nlev; ++l) {
            for (int q = D.level_ptr[l]; q < D.level_ptr[l + 1]; ++q) {
                const int sid = D.level_fronts[q];
                const Front& fr = D.fronts[sid];
                TileDesc d;
                d.a_off = fr.f_off;
                d.sbase = D.sub_off[fr.sub];
                d.rowbase = d.sbase + fr.start;
                d.upd_row = fr.upd_row;
                d.asm_base = D.asm_base[sid];
                d.u_off = fr.u_off;
                d.p = fr.p;
                d.f = fr.p + fr.u;
                d.pad = 0;
                for (int r = 0; r < fr.p; r += TL.tm) { d.row0 = r; pt.push_back(d); }
                for (int r = 0; r < fr.p + fr.u; r += TL.tm) { d.row0 = r; ft.push_back(d); }
            }
            // heaviest tiles first within a level (longest-processing-time
            // order), so the last wave is not left with the longest tiles;
            // the tiles of one level are independent, so the order is free
            const int tm = TL.tm;
            std::stable_sort(pt.begin() + TL.p_ptr.back(), pt.end(), [](const TileDesc& a, const TileDesc& b) {
                return a.f - a.row0 > b.f - b.row0;
            });
            std::stable_sort(ft.begin() + TL.f_ptr.back(), ft.end(), [tm](const TileDesc& a, const TileDesc& b) {
                return std::min(a.p, a.row0 + tm) > std::min(b.p, b.row0 + tm);
            });
            TL.p_ptr.push_back((int64_t)pt.size());
            TL.f_ptr.push_back((int64_t)ft.size());
        }
        if (pt.empty()) pt.push_back(TileDesc{});
        if (ft.empty()) ft.push_back(TileDesc{});
        TL.p_tiles.upload(pt, st);
        TL.f_tiles.upload(ft, st);
    }
    {
        // tensor-core sweeps: tiled panel offsets, packing blocks, 128-row tiles
        std::vector<int64_t> toff(nf);
        std::vector<int2> pb;
        int64_t acc = 0;
        for (size_t k = 0; k < nf; ++k) {
            const Front& fr = D.fronts[k];
            toff[k] = acc;
            acc += tiled_panel_floats(fr.p, fr.p + fr.u);
            for (int rb = 0; rb < (fr.p + fr.u + 31) / 32; ++rb) pb.push_back(make_int2((int)k, rb));
        }
        F.tiled_floats = std::max<int64_t>(acc, 512);
        F.n_pack_blocks = (int64_t)pb.size();
        if (pb.empty()) pb.push_back(make_int2(0, 0));
        up(F.t_off, toff, st);
        up(F.pack_blocks, pb, st);
        TileLists& TL = F.tiles128;
        TL.tm = 128;
        std::vector<TileDesc> pt, ft;
        TL.p_ptr.assign(1, 0);
        TL.f_ptr.assign(1, 0);
        for (int l = 0; l < nlev; ++l) {
            for (int q = D.level_ptr[l]; q < D.level_ptr[l + 1]; ++q) {
                const int sid = D.level_fronts[q];
                const Front& fr = D.fronts[sid];
                TileDesc d;
                d.a_off = toff[sid];
                d.sbase = D.sub_off[fr.sub];
                d.rowbase = d.sbase + fr.start;
                d.upd_row = fr.upd_row;
                d.asm_base = D.asm_base[sid];
                d.u_off = fr.u_off;
                d.p = fr.p;
                d.f = fr.p + fr.u;
                d.pad = 0;
                for (int r = 0; r < fr.p; r += 128) { d.row0 = r; pt.push_back(d); }
                for (int r = 0; r < fr.p + fr.u; r += 128) { d.row0 = r; ft.push_back(d); }
            }
            // heaviest first (stages per tile): backward by row blocks, forward by pivot atoms
            std::stable_sort(pt.begin() + TL.p_ptr.back(), pt.end(), [](const TileDesc& a, const TileDesc& b) {
                return (a.f + 31) / 32 - a.row0 / 32 > (b.f + 31) / 32 - b.row0 / 32;
            });
            std::stable_sort(ft.begin() + TL.f_ptr.back(), ft.end(), [](const TileDesc& a, const TileDesc& b) {
                return std::min(a.p, a.row0 + 128) > std::min(b.p, b.row0 + 128);
            });
            TL.p_ptr.push_back((int64_t)pt.size());
            TL.f_ptr.push_back((int64_t)ft.size());
        }
        if (pt.empty()) pt.push_back(TileDesc{});
        if (ft.empty()) ft.push_back(TileDesc{});
        TL.p_tiles.upload(pt, st);
        TL.f_tiles.upload(ft, st);
    }
    {
        std::vector<int64_t> io(D.level_fronts.size());
        F.inv_entries = 0;
        for (int l = 0; l < nlev; ++l) {
            int64_t acc = 0;
            for (int q = D.level_ptr[l]; q < D.level_ptr[l + 1]; ++q) {
                io[q] = acc;
                const Front& fr = D.fronts[D.level_fronts[q]];
                acc += (int64_t)fr.p * (fr.p + fr.u);
            }
            F.inv_entries = std::max(F.inv_entries, acc);
        }
        up(F.inv_off, io, st);
    }
    MWI_CUDA(cudaStreamSynchronize(st));
}

// A_c = P^T A P for the problem's current A (Galerkin product on the host
// cores from a copy of A's values), then A_c's factorisation on the device
void coarse_refresh(mwi_problem* P) {
    CoarseLevel& L = *P->coarse;
    mwi_mesh* M = P->mesh;
    cudaStream_t st = P->st;
    const double t0 = now_ms();
    const int64_t nnz = M->A.nnz;
    L.Aval_h.resize(nnz);
    MWI_CUDA(cudaMemcpyAsync(L.Aval_h.data(), P->Aval.p, nnz * sizeof(double2), cudaMemcpyDeviceToHost, st));
    MWI_CUDA(cudaStreamSynchronize(st));
    coarse_values(M->A_host.row_ptr, M->A_host.col, L.Aval_h.data(), L.H, L.Ac_h);
    L.Ac.ensure(L.Ac_h.size());
    MWI_CUDA(cudaMemcpyAsync(L.Ac.p, L.Ac_h.data(), L.Ac_h.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    L.perturbed.ensure(1);
    MWI_CUDA(cudaMemsetAsync(L.perturbed.p, 0, sizeof(int), st));
    if (P->opts.precision != 0) {
        L.ws32.ensure(L.F.ws_total());
        L.inv32.ensure(std::max<int64_t>(1, L.F.inv_entries));
        for (int k = 0; k < 2; ++k) L.sch32[k].ensure(1);
        float2* sch[2] = {L.sch32[0].p, L.sch32[1].p};
        factorize_fronts<float2>(L.F, L.ut, L.Ac.p, L.ws32.p, sch, L.inv32.p, L.perturbed.p, st);
    } else {
        L.ws64.ensure(L.F.ws_total());
        L.inv64.ensure(std::max<int64_t>(1, L.F.inv_entries));
        for (int k = 0; k < 2; ++k) L.sch64[k].ensure(1);
        double2* sch[2] = {L.sch64[0].p, L.sch64[1].p};
        factorize_fronts<double2>(L.F, L.ut, L.Ac.p, L.ws64.p, sch, L.inv64.p, L.perturbed.p, st);
    }
    MWI_CUDA(cudaMemcpyAsync(&L.n_perturbed, L.perturbed.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MWI_CUDA(cudaStreamSynchronize(st));
    L.setup_ms = now_ms() - t0;
}

// the FP32 copy of A used by the mixed two-level correction (the nested path
// assembles it anyway)
void refresh_a32(mwi_problem* P) {
    if (!P->coarse || P->opts.precision != 1) return;
    const int64_t nnz = P->mesh->A.nnz;
    P->Aval32.ensure(nnz);
    convert_c128_to_c64(nnz, P->Aval.p, P->Aval32.p, P->st);
}

void set_coarse(mwi_problem* P, mwi_mesh* Mc) {
    if (!Mc) {
        MWI_CUDA(cudaStreamSynchronize(P->st));
        P->coarse.reset();
        return;
    }
    mwi_mesh* M = P->mesh;
    cudaStream_t st = P->st;
    const double t0 = now_ms();
    std::unique_ptr<CoarseLevel> L(new CoarseLevel());
    build_prolongation(M->T, Mc->T, L->H);
    coarse_pattern(M->A_host.row_ptr, M->A_host.col, L->H);
    dense_front_decomposition(L->H, L->D);
    upload_fronts(L->D, L->F, st);
    CoarseDev& cd = L->dev;
    cd.n = L->H.n;
    cd.nc = L->H.nc;
    up(cd.P_rp, L->H.P_rp, st);
    up(cd.P_col, L->H.P_col, st);
    up(cd.P_val, L->H.P_val, st);
    up(cd.PT_rp, L->H.PT_rp, st);
    up(cd.PT_col, L->H.PT_col, st);
    up(cd.PT_val, L->H.PT_val, st);
    const bool fp32 = P->opts.precision != 0;
    build_update_tiles(L->D, factor_block_cols(fp32), factor_tile_rows(fp32), L->ut, st);
    MWI_CUDA(cudaStreamSynchronize(st));
    P->coarse = std::move(L);
    try {
        coarse_refresh(P);
        refresh_a32(P);
        MWI_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        P->coarse.reset();
        throw;
    }
    P->coarse->setup_ms = now_ms() - t0;
}

// y = M x for the problem's preconditioner: the one-level ORAS (one_level),
// or the deflated two-level ORAS when a coarse space is set
template <typename C>
void precondition(mwi_problem* P, const C* x, C* y, int m, const std::function<void(const C*, C*)>& one_level) {
    if (!P->coarse) {
        one_level(x, y);
        return;
    }
    CoarseLevel& L = *P->coarse;
    mwi_mesh* M = P->mesh;
    cudaStream_t st = P->st;
    const int64_t n = L.dev.n, nc = L.dev.nc;
    TwoLevelScratch<C> s;
    if constexpr (std::is_same<C, float2>::value) {
        L.ct32.ensure(nc * m);
        L.cq32.ensure(nc * m);
        L.q32.ensure(n * m);
        L.w32.ensure(n * m);
        L.Y32.ensure(nc * (m + 1));
        L.Z32.ensure(nc * (m + 1));
        L.upd32.ensure(1);
        s = {L.ct32.p, L.cq32.p, L.q32.p, L.w32.p};
        // exact coarse solve on the FP32 tensor cores (3xTF32 products)
        SweepCfg sc;
        sc.tc = 1;
        auto cs = [&](const float2* t, float2* c) {
            oras_apply<float2>(L.F, L.ws32.p, nullptr, nullptr, m, L.Y32.p, L.Z32.p, L.upd32.p, st, t, c, sc);
        };
        two_level_apply<float2>(L.dev, x, y, m, s, cs, one_level, M->A.row_ptr.p, M->A.col.p, P->Aval32.p, st);
    } else {
        L.ct64.ensure(nc * m);
        L.cq64.ensure(nc * m);
        L.q64.ensure(n * m);
        L.w64.ensure(n * m);
        L.Y64.ensure(nc * m);
        L.Z64.ensure(nc * m);
        L.upd64.ensure(1);
        s = {L.ct64.p, L.cq64.p, L.q64.p, L.w64.p};
        auto cs = [&](const double2* t, double2* c) {
            oras_apply<double2>(L.F, L.ws64.p, t, c, m, L.Y64.p, L.Z64.p, L.upd64.p, st);
        };
        two_level_apply<double2>(L.dev, x, y, m, s, cs, one_level, M->A.row_ptr.p, M->A.col.p, P->Aval.p, st);
    }
}

// assemble A and B_i values for the current eps, then factorise
// assemble A for the current eps_r; with refactor, also the subdomain
// matrices B_i and their factors (otherwise the previous factors stay as the
// ORAS preconditioner)
void numeric_setup(mwi_problem* P, bool refactor = true) {
    mwi_mesh* M = P->mesh;
    const Topology& T = M->T;
    cudaStream_t st = P->st;
    const double t0 = now_ms();
    P->A_coef.ensure(std::max<size_t>(1, M->A_fu.face.size()));
    launch_face_coef(M->A_fu_tet.p, (int64_t)M->A_fu.face.size(), P->eps.p, P->k0, P->A_coef.p, st);
    P->Aval.ensure(M->A.nnz);
    const bool mixed = P->opts.precision != 0;
    const bool nested = P->opts.precision == 2;
    if (nested) P->Aval32.ensure(M->A.nnz);
    const double2* Mk = P->p1 ? P->Mk.p : nullptr;
    launch_slot_fill(M->A, M->Kp.p, M->Mp.p, M->tabs.npack, M->Bf.p, M->tabs.npack_f, M->A_fu_face.p, P->A_coef.p,
                     P->eps.p, P->k0, P->Aval.p, nested ? P->Aval32.p : nullptr, st, Mk);
    if (mixed && !nested) {
        P->Adf.ensure(2 * (size_t)M->A.nnz);
        split_c128(M->A.nnz, P->Aval.p, P->Adf.p, st);
    }
    DecompEntry& E = *P->dec;
    refresh_a32(P);
    if (!refactor) {
        MWI_CUDA(cudaStreamSynchronize(st));
        P->setup_ms = now_ms() - t0;
        return;
    }
    P->B_coef.ensure(std::max<size_t>(1, E.D.B_faces.face.size()));
    launch_face_coef(E.fu_tet.p, (int64_t)E.D.B_faces.face.size(), P->eps.p, P->k0, P->B_coef.p, st);
    P->Bval.ensure(E.B.nnz);
    launch_slot_fill(E.B, M->Kp.p, M->Mp.p, M->tabs.npack, M->Bf.p, M->tabs.npack_f, E.fu_face.p, P->B_coef.p,
                     P->eps.p, P->k0, P->Bval.p, nullptr, st, Mk);
    P->perturbed.ensure(1);
    MWI_CUDA(cudaMemsetAsync(P->perturbed.p, 0, sizeof(int), st));
    if (mixed) {
        P->ws32.ensure(E.F.ws_total());
        P->inv32.ensure(std::max<int64_t>(1, E.F.inv_entries));
        for (int k = 0; k < 2; ++k) P->sch32[k].ensure(std::max<int64_t>(1, E.F.sch_entries[k]));
        float2* sch[2] = {P->sch32[0].p, P->sch32[1].p};
        std::call_once(E.ut_once[0], [&] {
            build_update_tiles(E.D, factor_block_cols(true), factor_tile_rows(true), E.ut[0], st);
        });
        timed(P, 3, [&] {
            factorize_fronts<float2>(E.F, E.ut[0], P->Bval.p, P->ws32.p, sch, P->inv32.p, P->perturbed.p, st);
            if (tc_of(P->opts) == 4) {
                P->wt.ensure(2 * (size_t)E.F.tiled_floats);
                pack_tiled(E.F.pack_blocks.p, E.F.n_pack_blocks, E.F.f_off.p, E.F.t_off.p, E.F.p.p, E.F.u.p,
                           P->ws32.p, P->wt.p, E.F.tiled_floats, st);
            }
        });
        if (tc_of(P->opts) == 4 && !P->sweep_err.p) {
            P->sweep_err.alloc(1);
            MWI_CUDA(cudaMemsetAsync(P->sweep_err.p, 0, sizeof(int), st));
        }
    } else {
        P->ws64.ensure(E.F.ws_total());
        P->inv64.ensure(std::max<int64_t>(1, E.F.inv_entries));
        for (int k = 0; k < 2; ++k) P->sch64[k].ensure(std::max<int64_t>(1, E.F.sch_entries[k]));
        double2* sch[2] = {P->sch64[0].p, P->sch64[1].p};
        std::call_once(E.ut_once[1], [&] {
            build_update_tiles(E.D, factor_block_cols(false), factor_tile_rows(false), E.ut[1], st);
        });
        timed(P, 3, [&] {
            factorize_fronts<double2>(E.F, E.ut[1], P->Bval.p, P->ws64.p, sch, P->inv64.p, P->perturbed.p, st);
        });
    }
    MWI_CUDA(cudaMemcpyAsync(&P->n_perturbed, P->perturbed.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MWI_CUDA(cudaStreamSynchronize(st));
    if (P->coarse) coarse_refresh(P);
    P->setup_ms = now_ms() - t0;
    (void)T;
}

void create_problem(mwi_mesh* M, const double* eps, bool eps_dev, double freq, const mwi_solver_opts* opts,
                    void* stream, mwi_problem_t* out) {
    MWI_REQUIRE(M && out, MWI_EINVAL, "null mesh or output handle");
    MWI_REQUIRE(eps, MWI_EINVAL, "null eps_r");
    MWI_REQUIRE(freq > 0 && std::isfinite(freq), MWI_EINVAL, "frequency must be positive");
    std::unique_ptr<mwi_problem> P(new mwi_problem());
    P->opts = defaults(opts);
    MWI_REQUIRE(P->opts.precision >= 0 && P->opts.precision <= 2, MWI_EINVAL, "precision must be 0, 1 or 2");
    MWI_REQUIRE(P->opts.sweep_engine >= 1 && P->opts.sweep_engine <= 4, MWI_EINVAL, "sweep_engine must be 0..4");
    MWI_REQUIRE(P->opts.n_sub <= M->T.nt, MWI_EINVAL, "more subdomains than tets");
    P->mesh = M;
    P->st = (cudaStream_t)stream;
    P->freq = freq;
    P->k0 = 2.0 * kPi * freq / kC0;
    {
        std::lock_guard<std::mutex> lk(M->mu);
        ensure_global(M);
        P->dec = get_decomp(M, P->opts);
    }
    P->eps.alloc(M->T.nt);
    if (eps_dev) {
        check_finite_device(P.get(), reinterpret_cast<const double2*>(eps), M->T.nt, "eps_r");
        MWI_CUDA(cudaMemcpyAsync(P->eps.p, eps, M->T.nt * sizeof(double2), cudaMemcpyDeviceToDevice, P->st));
    } else {
        for (int64_t t = 0; t < M->T.nt; ++t)
            MWI_REQUIRE(std::isfinite(eps[2 * t]) && std::isfinite(eps[2 * t + 1]), MWI_EINVAL, "eps_r not finite");
        MWI_CUDA(cudaMemcpyAsync(P->eps.p, eps, M->T.nt * sizeof(double2), cudaMemcpyHostToDevice, P->st));
    }
    numeric_setup(P.get());
    M->refcount++;
    *out = P.release();
}

// the same antennas, byte for byte, as the key
bool same_antennas(const std::vector<mwi_antenna>& key, const mwi_antenna* a, int n) {
    return (int64_t)key.size() == n && std::memcmp(key.data(), a, n * sizeof(mwi_antenna)) == 0;
}

// solve A X = B for m columns by FGMRES; returns info
// x0: X holds an initial guess (else the solve starts from zero)
void solve_block(mwi_problem* P, const double2* B, double2* X, int m, mwi_solve_info* info, bool x0 = false);
void solve_block_df(mwi_problem* P, const double2* B, double2* X, int m, mwi_solve_info* info, bool x0);

// The recycled space is the me columns of extra (when not null: the current
// forward solutions, for an adjoint solve) followed by the m columns X holds on
// entry (when prev: the previous system's solution block); on exit X holds,
// for every column of B, the least-residual element of that span (the
// recycled initial guess, in FP32 arithmetic).  m <= 32, m + me <= 64.  The
// projection keeps columns greedily in this order, so the current system's
// solutions come first.
void recycle_guess(mwi_problem* P, const double2* B, double2* X, int m, bool prev, const double2* extra,
                   int me) {
    mwi_mesh* M = P->mesh;
    const int64_t n = M->T.ndof;
    const int64_t nm = n * m;
    const int k = (prev ? m : 0) + (extra ? me : 0);
    const int64_t nk = n * k;
    cudaStream_t st = P->st;
    // the recycled block [X | extra] as one [n][k] FP64 array, then in FP32
    P->rc_block.ensure(nk);
    if (extra) copy_columns(n, me, 0, me, extra, k, 0, P->rc_block.p, st);
    if (prev) copy_columns(n, m, 0, m, X, k, extra ? me : 0, P->rc_block.p, st);
    P->v32.ensure(nk);
    P->x32.ensure(std::max(nk, nm));
    P->r32.ensure(nm);
    P->rc_scratch.ensure(recycle_scratch_entries(k, m));
    convert_c128_to_c64(nk, P->rc_block.p, P->v32.p, st);
    convert_c128_to_c64(nm, B, P->r32.p, st);
    const float2* C32 = nullptr;
    if (P->Adf.p) {
        // C = A X_rec with the double-float matrix; its head plane is C in FP32
        P->Rdf.ensure(2 * (size_t)nk);
        timed(P, 0, [&] { spmm_df(n, M->A.row_ptr.p, M->A.col.p, P->Adf.p, M->A.nnz, P->v32.p, P->Rdf.p, k, st); });
        C32 = P->Rdf.p;
    } else {
        P->R.ensure(nk);
        timed(P, 0, [&] {
            spmm<double2>(n, M->A.row_ptr.p, M->A.col.p, P->Aval.p, P->rc_block.p, P->R.p, k, st);
        });
        convert_c128_to_c64(nk, P->R.p, P->x32.p, st);
        C32 = P->x32.p;
    }
    // x0 is written to x32 after the projection has consumed C (which x32 holds in the FP64-matrix case)
    timed(P, 2, [&] {
        P->rec_dropped = recycle_initial_guess(n, k, m, P->v32.p, C32, P->r32.p, P->x32.p, P->rc_scratch.p, st);
    });
    convert_c64_to_c128(nm, P->x32.p, X, st);
}

// True block FGMRES (one Krylov space for the m columns) with FP64 vectors;
// the preconditioner M64 is the ORAS of the problem's precision
void solve_block_krylov(mwi_problem* P, const OpFnT<double2>& A64, const OpFnT<double2>& M64, const double2* B,
                        double2* X, int m, int restart, double t0, mwi_solve_info* info, bool x0) {
    const int64_t n = P->mesh->T.ndof;
    const int64_t nm = n * m;
    cudaStream_t st = P->st;
    const mwi_solver_opts& o = P->opts;
    BlockGmres& G = P->bgm;
    G.reserve(n, m, restart);
    G.timer = [P](int slot, const std::function<void()>& fn) { timed(P, slot, fn); };
    P->R.ensure(nm);
    std::vector<double2> gram((size_t)m * m);
    auto col_norms = [&](const double2* x, std::vector<double>& out) {
        G.block_dots(x, 1, x, G.small.p, st);
        MWI_CUDA(cudaMemcpyAsync(gram.data(), G.small.p, gram.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        out.resize(m);
        for (int c = 0; c < m; ++c) out[c] = std::sqrt(std::max(gram[(size_t)c * m + c].x, 0.0));
    };
    std::vector<double> bn, rn, tol(m), est(m);
    col_norms(B, bn);
    for (int c = 0; c < m; ++c) tol[c] = o.rtol * bn[c];
    rn = bn;
    auto converged = [&] {
        A64(X, P->R.p);
        residual_c128(nm, B, P->R.p, st);
        col_norms(P->R.p, rn);
        for (int c = 0; c < m; ++c)
            if (bn[c] > 0 && rn[c] > o.rtol * bn[c]) return false;
        return true;
    };
    bool done = false;
    if (x0) {
        done = converged();
    } else {
        MWI_CUDA(cudaMemsetAsync(X, 0, nm * sizeof(double2), st));
        MWI_CUDA(cudaMemcpyAsync(P->R.p, B, nm * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    int total = 0, deflated = 0;
    while (!done) {
        int defl = 0;
        const int used = G.cycle(A64, M64, P->R.p, X, tol, std::min(restart, o.max_iter - total), st, est.data(), &defl);
        total += used;
        deflated += defl;
        done = converged();
        if (done || total >= o.max_iter || used == 0) break;
    }
    int nconv = 0;
    double rmax = 0;
    for (int c = 0; c < m; ++c) {
        const double rel = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
        rmax = std::max(rmax, rel);
        if (rel <= o.rtol) nconv++;
    }
    if (o.verbose) std::fprintf(stderr, "[mwi] block FGMRES: %d steps, %d deflated columns\n", total, deflated);
    if (info) {
        info->iters_max = total;
        info->inner_total = P->inner_total;
        info->n_converged = nconv;
        info->n_perturbed = P->n_perturbed;
        info->resid_max = rmax;
        info->setup_ms = P->setup_ms;
        info->solve_ms = now_ms() - t0;
    }
    if (nconv < m) throw Error(MWI_ENOTCONV, "block FGMRES did not reach rtol on every column");
}

// solve A X = B for m columns in blocks of at most opts.max_block columns
// (Krylov bases scale with the block width); X and B are [n][m].  recycled:
// X holds the solution block of the previous, nearby system, whose span gives
// the initial guess (only when the m columns form one block of at most 32)
void solve_columns(mwi_problem* P, const double2* B, double2* X, int m, mwi_solve_info* info,
                   bool recycled = false, const double2* extra = nullptr) {
    // a shared block Krylov space costs m^2 per row in its Gram-Schmidt: at most 32 columns
    const int mb = P->opts.block_krylov ? std::min(P->opts.max_block, 32) : P->opts.max_block;
    if (m <= mb) {
        const bool x0 = (recycled || extra) && m <= 32;
        if (x0) recycle_guess(P, B, X, m, recycled, extra, m);
        solve_block(P, B, X, m, info, x0);
        return;
    }
    const int64_t n = P->mesh->T.ndof;
    cudaStream_t st = P->st;
    P->Bc.ensure((size_t)n * mb);
    P->Xc.ensure((size_t)n * mb);
    mwi_solve_info tot;
    std::memset(&tot, 0, sizeof(tot));
    bool notconv = false;
    for (int c0 = 0; c0 < m; c0 += mb) {
        const int mc = std::min(mb, m - c0);
        copy_columns(n, m, c0, mc, B, mc, 0, P->Bc.p, st);
        mwi_solve_info ci;
        std::memset(&ci, 0, sizeof(ci));
        try {
            solve_block(P, P->Bc.p, P->Xc.p, mc, &ci);
        } catch (const Error& e) {
            if (e.status != MWI_ENOTCONV) throw;
            notconv = true;
        }
        copy_columns(n, mc, 0, mc, P->Xc.p, m, c0, X, st);
        tot.iters_max = std::max(tot.iters_max, ci.iters_max);
        tot.inner_total += ci.inner_total;
        tot.n_converged += ci.n_converged;
        tot.n_perturbed = ci.n_perturbed;
        tot.resid_max = std::max(tot.resid_max, ci.resid_max);
        tot.setup_ms = ci.setup_ms;
        tot.solve_ms += ci.solve_ms;
    }
    MWI_CUDA(cudaStreamSynchronize(st));
    if (info) *info = tot;
    if (notconv) throw Error(MWI_ENOTCONV, "FGMRES did not reach rtol on every column");
}

void solve_block(mwi_problem* P, const double2* B, double2* X, int m, mwi_solve_info* info, bool x0) {
    mwi_mesh* M = P->mesh;
    const int64_t n = M->T.ndof;
    const int64_t nm = n * m;
    cudaStream_t st = P->st;
    const mwi_solver_opts& o = P->opts;
    const bool mixed = o.precision != 0;
    const bool nested = o.precision == 2;
    const bool block = o.block_krylov != 0;
    if (mixed && !nested && !block) {
        solve_block_df(P, B, X, m, info, x0);
        return;
    }
    DecompEntry& E = *P->dec;
    // with an inner GMRES the outer FGMRES needs few steps: keep its FP64 bases short
    const int restart = std::min(nested ? std::min(o.restart, 12) : o.restart, std::max(1, o.max_iter));
    if (!block) P->outer.reserve(n, m, restart);
    P->R.ensure(nm);
    P->dscratch.ensure(4 * (size_t)m);
    double* b2 = P->dscratch.p;
    double* tol = P->dscratch.p + m;
    double* bnorm = P->dscratch.p + 2 * m;
    double* r2 = P->dscratch.p + 3 * m;
    // local solve buffers
    if (mixed) {
        P->Y32.ensure((size_t)E.F.nloc * (m + 1));
        P->Z32.ensure((size_t)E.F.nloc * (m + 1));
        P->upd32.ensure((size_t)std::max<int64_t>(1, E.F.upd_rows) * (m + 1));
        if (nested) P->inner.reserve(n, m, std::max(1, o.inner_iters));
        P->v32.ensure(nm);
        P->x32.ensure(nm);
    } else {
        P->Y64.ensure((size_t)E.F.nloc * m);
        P->Z64.ensure((size_t)E.F.nloc * m);
        P->upd64.ensure((size_t)std::max<int64_t>(1, E.F.upd_rows) * m);
    }
    auto A64 = [&](const double2* x, double2* y) {
        timed(P, 0, [&] { spmm<double2>(n, M->A.row_ptr.p, M->A.col.p, P->Aval.p, x, y, m, st); });
    };
    auto A32 = [&](const float2* x, float2* y) {
        timed(P, 0, [&] { spmm<float2>(n, M->A.row_ptr.p, M->A.col.p, P->Aval32.p, x, y, m, st); });
    };
    auto M32 = [&](const float2* x, float2* y) {
        timed(P, 1, [&] {
            precondition<float2>(P, x, y, m, [&](const float2* a, float2* b) {
                oras_apply<float2>(E.F, P->ws32.p, nullptr, nullptr, m, P->Y32.p, P->Z32.p, P->upd32.p, st, a, b,
                                   sweep_cfg(P));
            });
        });
    };
    auto M64 = [&](const double2* x, double2* y) {
        if (!mixed) {
            timed(P, 1, [&] {
                precondition<double2>(P, x, y, m, [&](const double2* a, double2* b) {
                    oras_apply<double2>(E.F, P->ws64.p, a, b, m, P->Y64.p, P->Z64.p, P->upd64.p, st);
                });
            });
            return;
        }
        convert_c128_to_c64(nm, x, P->v32.p, st);
        if (!nested) {
            // the complex FP32 ORAS itself is the preconditioner of the FP64 FGMRES
            M32(P->v32.p, P->x32.p);
            convert_c64_to_c128(nm, P->x32.p, y, st);
            return;
        }
        // inner GMRES in complex FP32 on A z = x, preconditioned by the FP32 ORAS
        MWI_CUDA(cudaMemsetAsync(P->x32.p, 0, nm * sizeof(float2), st));
        double* vb2 = P->inner.dvec.p + 5 * m;
        double* tin = P->inner.dvec.p + 6 * m;
        double* vn = P->inner.dvec.p + 7 * m;
        P->inner.column_norms2(P->v32.p, vb2, st);
        tolerances(m, vb2, o.inner_rtol, tin, vn, st);
        int used = 0;
        P->inner.cycle(A32, M32, P->v32.p, P->x32.p, tin, std::max(1, o.inner_iters), st, nullptr, &used);
        P->inner_total += used;
        convert_c64_to_c128(nm, P->x32.p, y, st);
    };

    auto tfn = [P](int slot, const std::function<void()>& fn) { timed(P, slot, fn); };
    P->outer.timer = tfn;
    P->inner.timer = tfn;
    const double t0 = now_ms();
    P->inner_total = 0;
    if (block) {
        solve_block_krylov(P, A64, M64, B, X, m, restart, t0, info, x0);
        return;
    }
    P->outer.column_norms2(B, b2, st);
    tolerances(m, b2, o.rtol, tol, bnorm, st);
    std::vector<double> bn(m), rn(m);
    MWI_CUDA(cudaMemcpyAsync(bn.data(), bnorm, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    // true FP64 residual; true when every column meets rtol
    auto converged = [&] {
        A64(X, P->R.p);
        residual_c128(nm, B, P->R.p, st);
        P->outer.column_norms2(P->R.p, r2, st);
        MWI_CUDA(cudaMemcpyAsync(rn.data(), r2, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < m; ++c)
            if (bn[c] > 0 && std::sqrt(std::max(rn[c], 0.0)) > o.rtol * bn[c]) return false;
        return true;
    };
    bool done = false;
    if (x0) {
        done = converged();
    } else {
        MWI_CUDA(cudaMemsetAsync(X, 0, nm * sizeof(double2), st));
        MWI_CUDA(cudaMemcpyAsync(P->R.p, B, nm * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    int total = 0;
    while (!done) {
        int used = 0;
        P->outer.cycle(A64, M64, P->R.p, X, tol, std::min(restart, o.max_iter - total), st, nullptr, &used);
        total += used;
        done = converged();
        if (total >= o.max_iter || used == 0) break;
    }
    int nconv = 0;
    double rmax = 0;
    for (int c = 0; c < m; ++c) {
        double rel = bn[c] > 0 ? std::sqrt(std::max(rn[c], 0.0)) / bn[c] : 0.0;
        rmax = std::max(rmax, rel);
        if (rel <= o.rtol) nconv++;
    }
    if (info) {
        info->iters_max = total;
        info->inner_total = P->inner_total;
        info->n_converged = nconv;
        info->n_perturbed = P->n_perturbed;
        info->resid_max = rmax;
        info->setup_ms = P->setup_ms;
        info->solve_ms = now_ms() - t0;
    }
    if (nconv < m) throw Error(MWI_ENOTCONV, "FGMRES did not reach rtol on every column");
}

// MIXED: the complex FP32 ORAS preconditions an FGMRES whose basis, residual
// and iterate are double-float planes (FP64-quality results on the FP32 pipes)
void solve_block_df(mwi_problem* P, const double2* B, double2* X, int m, mwi_solve_info* info, bool x0) {
    mwi_mesh* M = P->mesh;
    const int64_t n = M->T.ndof;
    const int64_t nm = n * m;
    const int64_t nnz = M->A.nnz;
    cudaStream_t st = P->st;
    const mwi_solver_opts& o = P->opts;
    DecompEntry& E = *P->dec;
    const int restart = std::min(o.restart, std::max(1, o.max_iter));
    GmresDF& G = P->dfk;
    G.reserve(n, m, restart);
    P->Bdf.ensure(2 * (size_t)nm);
    P->Xdf.ensure(2 * (size_t)nm);
    P->Rdf.ensure(2 * (size_t)nm);
    P->dscratch.ensure(4 * (size_t)m);
    double* b2 = P->dscratch.p;
    double* tol = P->dscratch.p + m;
    double* bnorm = P->dscratch.p + 2 * m;
    double* r2 = P->dscratch.p + 3 * m;
    P->Y32.ensure((size_t)E.F.nloc * (m + 1));
    P->Z32.ensure((size_t)E.F.nloc * (m + 1));
    P->upd32.ensure((size_t)std::max<int64_t>(1, E.F.upd_rows) * (m + 1));
    auto Aop = [&](const float2* z, float2* w) {
        timed(P, 0, [&] { spmm_df(n, M->A.row_ptr.p, M->A.col.p, P->Adf.p, nnz, z, w, m, st); });
    };
    auto Mop = [&](const float2* v, float2* z) {
        timed(P, 1, [&] {
            precondition<float2>(P, v, z, m, [&](const float2* a, float2* b) {
                oras_apply<float2>(E.F, P->ws32.p, nullptr, nullptr, m, P->Y32.p, P->Z32.p, P->upd32.p, st, a, b,
                                   sweep_cfg(P));
            });
        });
    };
    G.timer = [P](int slot, const std::function<void()>& fn) { timed(P, slot, fn); };
    const double t0 = now_ms();
    split_c128(nm, B, P->Bdf.p, st);
    G.norms2(P->Bdf.p, b2, st);
    tolerances(m, b2, o.rtol, tol, bnorm, st);
    std::vector<double> bn(m), rn(m);
    MWI_CUDA(cudaMemcpyAsync(bn.data(), bnorm, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    // true residual in double-float; true when every column meets rtol
    auto converged = [&] {
        timed(P, 0, [&] {
            residual_df(n, M->A.row_ptr.p, M->A.col.p, P->Adf.p, nnz, P->Bdf.p, P->Xdf.p, P->Rdf.p, m, st);
        });
        G.norms2(P->Rdf.p, r2, st);
        MWI_CUDA(cudaMemcpyAsync(rn.data(), r2, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < m; ++c)
            if (bn[c] > 0 && std::sqrt(std::max(rn[c], 0.0)) > o.rtol * bn[c]) return false;
        return true;
    };
    bool done = false;
    if (x0) {
        split_c128(nm, X, P->Xdf.p, st);
        done = converged();
    } else {
        MWI_CUDA(cudaMemsetAsync(P->Xdf.p, 0, 2 * nm * sizeof(float2), st));
        MWI_CUDA(cudaMemcpyAsync(P->Rdf.p, P->Bdf.p, 2 * nm * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    }
    int total = 0;
    while (!done) {
        int used = 0;
        G.cycle(Aop, Mop, P->Rdf.p, P->Xdf.p, tol, std::min(restart, o.max_iter - total), st, &used);
        total += used;
        done = converged();
        if (done || total >= o.max_iter || used == 0) break;
    }
    join_c128(nm, P->Xdf.p, X, st);
    int nconv = 0;
    double rmax = 0;
    for (int c = 0; c < m; ++c) {
        double rel = bn[c] > 0 ? std::sqrt(std::max(rn[c], 0.0)) / bn[c] : 0.0;
        rmax = std::max(rmax, rel);
        if (rel <= o.rtol) nconv++;
    }
    MWI_CUDA(cudaStreamSynchronize(st));
    if (info) {
        info->iters_max = total;
        info->inner_total = 0;
        info->n_converged = nconv;
        info->n_perturbed = P->n_perturbed;
        info->resid_max = rmax;
        info->setup_ms = P->setup_ms;
        info->solve_ms = now_ms() - t0;
    }
    if (nconv < m) throw Error(MWI_ENOTCONV, "FGMRES did not reach rtol on every column");
}

}  // namespace

mwi_solver_opts mwi::solver_defaults(const mwi_solver_opts* o) { return defaults(o); }

extern "C" {

const char* mwi_last_error(void) { return g_last_error.c_str(); }

mwi_status mwi_mesh_create(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt, const int32_t* bface_tag,
                           int32_t order, mwi_mesh_t* out) {
    return guard([&] {
        MWI_REQUIRE(xyz && tet && bface_tag && out, MWI_EINVAL, "null argument");
        std::unique_ptr<mwi_mesh> M(new mwi_mesh());
        build_topology(M->T, xyz, nv, tet, nt, bface_tag, order);
        MWI_CUDA(cudaStreamCreateWithFlags(&M->st, cudaStreamNonBlocking));
        build_mesh_device(M.get());
        *out = M.release();
    });
}

mwi_status mwi_mesh_ndof(mwi_mesh_t mesh, int64_t* ndof) {
    return guard([&] {
        MWI_REQUIRE(mesh && ndof, MWI_EINVAL, "null argument");
        *ndof = mesh->T.ndof;
    });
}

mwi_status mwi_mesh_dof_keys(mwi_mesh_t mesh, int32_t* kind, int64_t* verts) {
    return guard([&] {
        MWI_REQUIRE(mesh, MWI_EINVAL, "null mesh");
        if (kind) std::copy(mesh->T.dof_kind.begin(), mesh->T.dof_kind.end(), kind);
        if (verts) std::copy(mesh->T.dof_verts.begin(), mesh->T.dof_verts.end(), verts);
    });
}

mwi_status mwi_mesh_destroy(mwi_mesh_t mesh) {
    return guard([&] {
        if (!mesh) return;
        MWI_REQUIRE(mesh->refcount == 0, MWI_ESTATE, "mesh is still referenced by a problem");
        if (mesh->st) cudaStreamDestroy(mesh->st);
        delete mesh;
    });
}

mwi_status mwi_assemble(mwi_mesh_t mesh, const double* eps_r, double freq_hz, const mwi_solver_opts* opts,
                        void* cuda_stream, mwi_problem_t* out) {
    return guard([&] { create_problem(mesh, eps_r, false, freq_hz, opts, cuda_stream, out); });
}

mwi_status mwi_assemble_device(mwi_mesh_t mesh, const double* eps_r_dev, double freq_hz,
                               const mwi_solver_opts* opts, void* cuda_stream, mwi_problem_t* out) {
    return guard([&] { create_problem(mesh, eps_r_dev, true, freq_hz, opts, cuda_stream, out); });
}

// reassemble for the current parameter; factor reuse: up to factor_reuse
// consecutive updates keep the factors
static void refresh_operator(mwi_problem_t P) {
    const bool refactor = P->opts.factor_reuse <= 0 || P->reuse_count >= P->opts.factor_reuse;
    numeric_setup(P, refactor);
    P->reuse_count = refactor ? 0 : P->reuse_count + 1;
    P->have_fwd = false;
    P->have_adj = false;
}

static void update_eps(mwi_problem_t P, const double* eps, bool dev) {
    MWI_REQUIRE(P && eps, MWI_EINVAL, "null argument");
    const int64_t nt = P->mesh->T.nt;
    if (!dev)
        for (int64_t t = 0; t < nt; ++t)
            MWI_REQUIRE(std::isfinite(eps[2 * t]) && std::isfinite(eps[2 * t + 1]), MWI_EINVAL, "eps_r not finite");
    else
        check_finite_device(P, reinterpret_cast<const double2*>(eps), nt, "eps_r");
    MWI_CUDA(cudaMemcpyAsync(P->eps.p, eps, nt * sizeof(double2),
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, P->st));
    P->p1 = false;
    refresh_operator(P);
}

mwi_status mwi_update_eps(mwi_problem_t prob, const double* eps_r) {
    return guard([&] { update_eps(prob, eps_r, false); });
}
mwi_status mwi_update_eps_device(mwi_problem_t prob, const double* eps_r_dev) {
    return guard([&] { update_eps(prob, eps_r_dev, true); });
}

mwi_status mwi_forward_solve(mwi_problem_t P, const mwi_antenna* tx, int32_t n_tx, const mwi_antenna* rx,
                             int32_t n_rx, double* S_out, mwi_solve_info* info) {
    mwi_status status = MWI_OK;
    mwi_status g = guard([&] {
        MWI_REQUIRE(P && tx && rx && S_out, MWI_EINVAL, "null argument");
        MWI_REQUIRE(n_tx >= 1 && n_rx >= 1 && n_tx <= 4096 && n_rx <= 4096, MWI_EINVAL, "bad antenna count");
        const Topology& T = P->mesh->T;
        cudaStream_t st = P->st;
        const int m = n_tx;
        const int64_t nm = T.ndof * (int64_t)m;
        // the edge of an antenna depends only on the mesh and the antenna (a
        // nearest-vertex search over the whole mesh): a call with the same
        // antennas as the previous one (every step of an inversion) keeps the
        // map and its device copies
        if (!same_antennas(P->tx_key, tx, n_tx)) {
            P->tx_key.clear();
            map_antennas(T, tx, n_tx, P->tx_dof, P->tx_sign);
            P->tx_dof_d.upload(P->tx_dof, st);
            P->tx_sign_d.upload(P->tx_sign, st);
            std::vector<double2> cur(m);
            for (int j = 0; j < m; ++j) cur[j] = make_double2(tx[j].re_I, tx[j].im_I);
            P->cur_d.upload(cur, st);
            P->tx_key.assign(tx, tx + n_tx);
        }
        if (!same_antennas(P->rx_key, rx, n_rx)) {
            P->rx_key.clear();
            map_antennas(T, rx, n_rx, P->rx_dof, P->rx_sign);
            P->rx_dof_d.upload(P->rx_dof, st);
            P->rx_sign_d.upload(P->rx_sign, st);
            P->rx_key.assign(rx, rx + n_rx);
        }
        P->Brhs.ensure(nm);
        P->U.ensure(nm);
        MWI_CUDA(cudaMemsetAsync(P->Brhs.p, 0, nm * sizeof(double2), st));
        launch_rhs(m, P->tx_dof_d.p, P->tx_sign_d.p, P->cur_d.p, 2.0 * kPi * P->freq * kMu0, P->Brhs.p, st);
        P->m_fwd = m;
        P->n_rx = n_rx;
        const bool rec = P->opts.recycle && P->rec_m[0] == m;
        P->rec_m[0] = 0;
        try {
            solve_columns(P, P->Brhs.p, P->U.p, m, info, rec);
            P->rec_m[0] = m;
        } catch (const Error& e) {
            if (e.status != MWI_ENOTCONV) throw;
            status = MWI_ENOTCONV;
            set_last_error(e.what());
        }
        check_sweep_error(P);
        P->S_d.ensure((size_t)n_rx * m);
        launch_s_extract(n_rx, m, P->rx_dof_d.p, P->rx_sign_d.p, P->U.p, P->S_d.p, st);
        MWI_CUDA(cudaMemcpyAsync(S_out, P->S_d.p, (size_t)n_rx * m * sizeof(double2), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        P->have_fwd = true;
        P->have_adj = false;
    });
    return g != MWI_OK ? g : status;
}

// misfit J and r = S - S_meas (Eq. defJ) for the last forward solve, the
// adjoint sources (Eq. pbadj) and the adjoint solve with the same factors;
// J stays on the device (P->J_d).  MWI_ENOTCONV of the adjoint solve is
// returned in status, not thrown.
static void misfit_and_adjoint(mwi_problem_t P, const double* S_meas, const double* w, bool dev,
                               mwi_solve_info* info, mwi_status& status) {
    MWI_REQUIRE(P->have_fwd, MWI_ESTATE, "misfit_and_gradient needs a prior forward_solve");
    const Topology& T = P->mesh->T;
    cudaStream_t st = P->st;
    const int m = P->m_fwd, n_rx = P->n_rx;
    const int cnt = n_rx * m;
    const int64_t nm = T.ndof * (int64_t)m;
    const auto kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    P->Smeas_d.ensure(cnt);
    P->r_d.ensure(cnt);
    P->J_d.ensure(1);
    MWI_CUDA(cudaMemcpyAsync(P->Smeas_d.p, S_meas, cnt * sizeof(double2), kind, st));
    const double* wd = nullptr;
    if (w) {
        P->w_d.ensure(cnt);
        MWI_CUDA(cudaMemcpyAsync(P->w_d.p, w, cnt * sizeof(double), kind, st));
        wd = P->w_d.p;
    }
    launch_misfit(cnt, P->S_d.p, P->Smeas_d.p, wd, P->r_d.p, P->J_d.p, st);
    P->Brhs.ensure(nm);
    MWI_CUDA(cudaMemsetAsync(P->Brhs.p, 0, nm * sizeof(double2), st));
    launch_adjoint_rhs(n_rx, m, P->rx_dof_d.p, P->rx_sign_d.p, P->r_d.p, wd, P->Brhs.p, st);
    P->Lam.ensure(nm);
    // recycled space of the adjoint solve: the previous adjoint solutions and
    // the current forward solutions (whose span holds the adjoint solution
    // exactly when the receivers are among the transmitters)
    const bool rec = P->opts.recycle && P->rec_m[1] == m;
    const double2* fwd = P->opts.recycle && P->rec_m[0] == m ? P->U.p : nullptr;
    P->rec_m[1] = 0;
    try {
        solve_columns(P, P->Brhs.p, P->Lam.p, m, info, rec, fwd);
        P->rec_m[1] = m;
    } catch (const Error& e) {
        if (e.status != MWI_ENOTCONV) throw;
        status = MWI_ENOTCONV;
        set_last_error(e.what());
    }
    check_sweep_error(P);
}

static mwi_status misfit_grad_impl(mwi_problem_t P, const double* S_meas, const double* w, double* J_out,
                                   double* dJ, mwi_solve_info* info, bool dev) {
    mwi_status status = MWI_OK;
    mwi_status g = guard([&] {
        MWI_REQUIRE(P && S_meas && J_out && dJ, MWI_EINVAL, "null argument");
        MWI_REQUIRE(!P->p1, MWI_ESTATE, "the operator holds a nodal parameter: use "
                                        "mwi_misfit_and_gradient_kappa_device");
        misfit_and_adjoint(P, S_meas, w, dev, info, status);
        const Topology& T = P->mesh->T;
        cudaStream_t st = P->st;
        double2* out = dev ? reinterpret_cast<double2*>(dJ) : nullptr;
        if (!dev) {
            P->grad_d.ensure(T.nt);
            out = P->grad_d.p;
        }
        mwi_mesh* M = P->mesh;
        if (P->opts.precision != 0 && T.order == 1) {
            // mixed: the volume term in double-float (U and Lam split into the
            // solver's double-float scratch planes, free after the adjoint solve)
            const int64_t nm = T.ndof * (int64_t)P->m_fwd;
            {
                // built once per mesh on the mesh's stream and finished before any
                // problem on the mesh (any stream) can see it
                std::lock_guard<std::mutex> lk(M->mu);
                if (!M->Mdf.p) {
                    DevBuf<float2> mdf((size_t)T.nt * 21);
                    launch_split_real(T.nt * 21, M->Mp.p, mdf.p, M->st);
                    MWI_CUDA(cudaStreamSynchronize(M->st));
                    M->Mdf = std::move(mdf);
                }
            }
            P->Xdf.ensure(2 * (size_t)nm);
            P->Rdf.ensure(2 * (size_t)nm);
            split_c128(nm, P->U.p, P->Xdf.p, st);
            split_c128(nm, P->Lam.p, P->Rdf.p, st);
            launch_gradient_df(T.nt, P->m_fwd, nm, M->tet_dofs.p, M->tet_faces.p, M->face_tag.p, M->face_dofs.p,
                               M->Mdf.p, M->Bf.p, P->eps.p, P->k0, P->U.p, P->Lam.p, P->Xdf.p, P->Rdf.p, out, st);
        } else {
            launch_gradient(T.order, T.nt, P->m_fwd, M->tet_dofs.p, M->tet_faces.p, M->face_tag.p, M->face_dofs.p,
                            M->Mp.p, M->Bf.p, P->eps.p, P->k0, P->U.p, P->Lam.p, out, st);
        }
        MWI_CUDA(cudaMemcpyAsync(J_out, P->J_d.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        if (!dev)
            MWI_CUDA(cudaMemcpyAsync(dJ, P->grad_d.p, T.nt * sizeof(double2), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        P->have_adj = true;
    });
    return g != MWI_OK ? g : status;
}

mwi_status mwi_misfit(mwi_problem_t P, const double* S_meas, const double* w, double* J_out) {
    return guard([&] {
        MWI_REQUIRE(P && S_meas && J_out, MWI_EINVAL, "null argument");
        MWI_REQUIRE(P->have_fwd, MWI_ESTATE, "misfit needs a prior forward_solve");
        cudaStream_t st = P->st;
        const int cnt = P->n_rx * P->m_fwd;
        P->Smeas_d.ensure(cnt);
        P->r_d.ensure(cnt);
        P->J_d.ensure(1);
        MWI_CUDA(cudaMemcpyAsync(P->Smeas_d.p, S_meas, cnt * sizeof(double2), cudaMemcpyHostToDevice, st));
        const double* wd = nullptr;
        if (w) {
            P->w_d.ensure(cnt);
            MWI_CUDA(cudaMemcpyAsync(P->w_d.p, w, cnt * sizeof(double), cudaMemcpyHostToDevice, st));
            wd = P->w_d.p;
        }
        launch_misfit(cnt, P->S_d.p, P->Smeas_d.p, wd, P->r_d.p, P->J_d.p, st);
        MWI_CUDA(cudaMemcpyAsync(J_out, P->J_d.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
    });
}

mwi_status mwi_misfit_and_gradient(mwi_problem_t prob, const double* S_meas, const double* w, double* J_out,
                                   double* dJ_deps, mwi_solve_info* info) {
    return misfit_grad_impl(prob, S_meas, w, J_out, dJ_deps, info, false);
}

mwi_status mwi_misfit_and_gradient_device(mwi_problem_t prob, const double* S_meas_dev, const double* w_dev,
                                          double* J_out, double* dJ_deps_dev, mwi_solve_info* info) {
    return misfit_grad_impl(prob, S_meas_dev, w_dev, J_out, dJ_deps_dev, info, true);
}

mwi_status mwi_fields_device(mwi_problem_t P, int32_t which, void** dev_ptr, int64_t* n, int64_t* m) {
    return guard([&] {
        MWI_REQUIRE(P && dev_ptr, MWI_EINVAL, "null argument");
        MWI_REQUIRE(which == 0 || which == 1, MWI_EINVAL, "which must be 0 or 1");
        MWI_REQUIRE(which == 0 ? P->have_fwd : P->have_adj, MWI_ESTATE, "no fields of that kind yet");
        *dev_ptr = which == 0 ? (void*)P->U.p : (void*)P->Lam.p;
        if (n) *n = P->mesh->T.ndof;
        if (m) *m = P->m_fwd;
    });
}

mwi_status mwi_copy_fields(mwi_problem_t P, int32_t which, double* out) {
    return guard([&] {
        MWI_REQUIRE(P && out, MWI_EINVAL, "null argument");
        MWI_REQUIRE(which == 0 || which == 1, MWI_EINVAL, "which must be 0 or 1");
        MWI_REQUIRE(which == 0 ? P->have_fwd : P->have_adj, MWI_ESTATE, "no fields of that kind yet");
        const double2* src = which == 0 ? P->U.p : P->Lam.p;
        MWI_CUDA(cudaMemcpyAsync(out, src, (size_t)P->mesh->T.ndof * P->m_fwd * sizeof(double2),
                                 cudaMemcpyDeviceToHost, P->st));
        MWI_CUDA(cudaStreamSynchronize(P->st));
    });
}

mwi_status mwi_problem_destroy(mwi_problem_t P) {
    return guard([&] {
        if (!P) return;
        if (P->st) cudaStreamSynchronize(P->st);
        P->mesh->refcount--;
        delete P;
    });
}

mwi_status mwi_spmm_device(mwi_problem_t P, const double* x_dev, double* y_dev, int32_t m) {
    return guard([&] {
        MWI_REQUIRE(P && x_dev && y_dev && m >= 1, MWI_EINVAL, "bad argument");
        mwi_mesh* M = P->mesh;
        spmm<double2>(M->T.ndof, M->A.row_ptr.p, M->A.col.p, P->Aval.p, (const double2*)x_dev, (double2*)y_dev, m,
                      P->st);
        MWI_CUDA(cudaStreamSynchronize(P->st));
    });
}

mwi_status mwi_oras_apply_device(mwi_problem_t P, const double* x_dev, double* y_dev, int32_t m) {
    return guard([&] {
        MWI_REQUIRE(P && x_dev && y_dev && m >= 1, MWI_EINVAL, "bad argument");
        DecompEntry& E = *P->dec;
        const int64_t n = P->mesh->T.ndof;
        if (P->opts.precision != 0) {
            P->Y32.ensure((size_t)E.F.nloc * (m + 1));
            P->Z32.ensure((size_t)E.F.nloc * (m + 1));
            P->upd32.ensure((size_t)std::max<int64_t>(1, E.F.upd_rows) * (m + 1));
            P->v32.ensure(n * m);
            P->x32.ensure(n * m);
            convert_c128_to_c64(n * m, (const double2*)x_dev, P->v32.p, P->st);
            precondition<float2>(P, P->v32.p, P->x32.p, m, [&](const float2* a, float2* b) {
                oras_apply<float2>(E.F, P->ws32.p, nullptr, nullptr, m, P->Y32.p, P->Z32.p, P->upd32.p, P->st, a, b,
                                   sweep_cfg(P));
            });
            convert_c64_to_c128(n * m, P->x32.p, (double2*)y_dev, P->st);
        } else {
            P->Y64.ensure((size_t)E.F.nloc * m);
            P->Z64.ensure((size_t)E.F.nloc * m);
            P->upd64.ensure((size_t)std::max<int64_t>(1, E.F.upd_rows) * m);
            precondition<double2>(P, (const double2*)x_dev, (double2*)y_dev, m, [&](const double2* a, double2* b) {
                oras_apply<double2>(E.F, P->ws64.p, a, b, m, P->Y64.p, P->Z64.p, P->upd64.p, P->st);
            });
        }
        MWI_CUDA(cudaStreamSynchronize(P->st));
        check_sweep_error(P);
    });
}

mwi_status mwi_oras_apply_device_noalloc(mwi_problem_t P, const double* x_dev, double* y_dev, int32_t m) {
    return guard([&] {
        MWI_REQUIRE(P && x_dev && y_dev && m >= 1, MWI_EINVAL, "bad argument");
        MWI_REQUIRE(!P->coarse, MWI_EINVAL,
                    "the allocation-free entry point applies the one-level ORAS only; this problem has a coarse space");
        DecompEntry& E = *P->dec;
        const bool mixed = P->opts.precision != 0;
        const void* ws = mixed ? (const void*)P->ws32.p : (const void*)P->ws64.p;
        oras_apply_noalloc(E.F, ws, mixed, (const double2*)x_dev, (double2*)y_dev, m, P->mesh->T.ndof, P->st,
                           sweep_cfg(P));
        MWI_CUDA(cudaStreamSynchronize(P->st));
        check_sweep_error(P);
    });
}

mwi_status mwi_matrix_csr(mwi_problem_t P, int64_t* nnz, int64_t* row_ptr, int32_t* col, double* val) {
    return guard([&] {
        MWI_REQUIRE(P && nnz, MWI_EINVAL, "null argument");
        mwi_mesh* M = P->mesh;
        *nnz = M->A.nnz;
        if (row_ptr) std::copy(M->A_host.row_ptr.begin(), M->A_host.row_ptr.end(), row_ptr);
        if (col) std::copy(M->A_host.col.begin(), M->A_host.col.end(), col);
        if (val) {
            MWI_CUDA(cudaMemcpyAsync(val, P->Aval.p, M->A.nnz * sizeof(double2), cudaMemcpyDeviceToHost, P->st));
            MWI_CUDA(cudaStreamSynchronize(P->st));
        }
    });
}

mwi_status mwi_decomposition(mwi_problem_t P, int32_t* part, int64_t* n_local) {
    return guard([&] {
        MWI_REQUIRE(P, MWI_EINVAL, "null problem");
        const Decomposition& D = P->dec->D;
        if (part) std::copy(D.part.begin(), D.part.end(), part);
        if (n_local)
            for (int i = 0; i < D.n_sub; ++i) n_local[i] = D.sub_off[i + 1] - D.sub_off[i];
    });
}

mwi_status mwi_factor_stats(mwi_problem_t P, int64_t* factor_entries, int64_t* n_fronts, int64_t* max_front,
                            double* factor_flops) {
    return guard([&] {
        MWI_REQUIRE(P, MWI_EINVAL, "null problem");
        const Decomposition& D = P->dec->D;
        if (factor_entries) *factor_entries = D.factor_entries;
        if (n_fronts) *n_fronts = (int64_t)D.fronts.size();
        if (max_front) *max_front = D.max_front;
        if (factor_flops) *factor_flops = D.factor_flops;
    });
}

static void ensure_p1(mwi_mesh* M) {
    std::lock_guard<std::mutex> lk(M->mu);
    if (M->have_p1) return;
    const Topology& T = M->T;
    std::vector<int32_t> rp, col;
    std::vector<double> val;
    build_p1_stiffness(T, rp, col, val);
    up(M->v2t_ptr, T.v2t_ptr, M->st);
    up(M->v2t, T.v2t, M->st);
    up(M->p1_rp, rp, M->st);
    up(M->p1_col, col, M->st);
    up(M->p1_val, val, M->st);
    M->Mv.alloc((size_t)T.nt * 4 * M->tabs.npack);
    launch_elem_vertex_mass(M->xyz.p, M->tv.p, T.nt, M->tabs, M->Mv.p, M->st);
    MWI_CUDA(cudaStreamSynchronize(M->st));
    M->have_p1 = true;
}

mwi_status mwi_update_kappa_device(mwi_problem_t P, const double* kappa_dev) {
    return guard([&] {
        MWI_REQUIRE(P && kappa_dev, MWI_EINVAL, "null argument");
        mwi_mesh* M = P->mesh;
        const Topology& T = M->T;
        ensure_p1(M);
        const double2* k = reinterpret_cast<const double2*>(kappa_dev);
        check_finite_device(P, k, T.nv, "kappa");
        cudaStream_t st = P->st;
        P->kappa.ensure(T.nv);
        MWI_CUDA(cudaMemcpyAsync(P->kappa.p, k, T.nv * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        // beta and the interface wavenumber from the centroid value; the mass term from kappa itself
        launch_p1_centroid(T.nt, M->tv.p, P->kappa.p, P->eps.p, st);
        P->Mk.ensure((size_t)T.nt * M->tabs.npack);
        launch_p1_mass(T.nt, M->tabs.npack, M->tv.p, P->kappa.p, M->Mv.p, P->Mk.p, st);
        P->p1 = true;
        refresh_operator(P);
    });
}

mwi_status mwi_misfit_and_gradient_kappa_device(mwi_problem_t P, const double* S_meas_dev, const double* w_dev,
                                                double alpha, double* J_out, double* R_out,
                                                double* dPhi_dkappa_dev, mwi_solve_info* info) {
    mwi_status status = MWI_OK;
    mwi_status g = guard([&] {
        MWI_REQUIRE(P && S_meas_dev && J_out && dPhi_dkappa_dev, MWI_EINVAL, "null argument");
        MWI_REQUIRE(alpha >= 0.0 && std::isfinite(alpha), MWI_EINVAL, "alpha must be finite and >= 0");
        MWI_REQUIRE(P->p1, MWI_ESTATE, "no nodal parameter: call mwi_update_kappa_device first");
        misfit_and_adjoint(P, S_meas_dev, w_dev, true, info, status);
        mwi_mesh* M = P->mesh;
        const Topology& T = M->T;
        cudaStream_t st = P->st;
        P->grad_tw.ensure((size_t)T.nt * 4);
        if (P->opts.precision != 0 && T.order == 1) {
            // mixed: the volume terms in double-float (U and Lam split into the
            // solver's double-float scratch planes, free after the adjoint solve)
            const int64_t nm = T.ndof * (int64_t)P->m_fwd;
            {
                // built once per mesh on the mesh's stream and finished before any
                // problem on the mesh (any stream) can see it
                std::lock_guard<std::mutex> lk(M->mu);
                if (!M->Mvdf.p) {
                    DevBuf<float2> mv((size_t)T.nt * 4 * 21);
                    launch_split_real(T.nt * 4 * 21, M->Mv.p, mv.p, M->st);
                    MWI_CUDA(cudaStreamSynchronize(M->st));
                    M->Mvdf = std::move(mv);
                }
            }
            P->Xdf.ensure(2 * (size_t)nm);
            P->Rdf.ensure(2 * (size_t)nm);
            split_c128(nm, P->U.p, P->Xdf.p, st);
            split_c128(nm, P->Lam.p, P->Rdf.p, st);
            launch_p1_tet_gradient_df(T.nt, P->m_fwd, nm, M->tet_dofs.p, M->tet_faces.p, M->face_tag.p,
                                      M->face_dofs.p, M->Mvdf.p, M->Bf.p, P->eps.p, P->k0, P->U.p, P->Lam.p,
                                      P->Xdf.p, P->Rdf.p, P->grad_tw.p, st);
        } else {
            launch_p1_tet_gradient(T.order, T.nt, P->m_fwd, M->tet_dofs.p, M->tet_faces.p, M->face_tag.p,
                                   M->face_dofs.p, M->Mv.p, M->Bf.p, P->eps.p, P->k0, P->U.p, P->Lam.p, P->grad_tw.p,
                                   st);
        }
        const int nb = p1_gradient_blocks(T.nv);
        P->p1_partial.ensure(nb);
        P->p1_partial_host.resize(nb);
        launch_p1_gradient(T.nv, M->v2t_ptr.p, M->v2t.p, M->tv.p, P->grad_tw.p, M->p1_rp.p, M->p1_col.p,
                           M->p1_val.p, P->kappa.p, alpha, reinterpret_cast<double2*>(dPhi_dkappa_dev),
                           P->p1_partial.p, st);
        MWI_CUDA(cudaMemcpyAsync(J_out, P->J_d.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaMemcpyAsync(P->p1_partial_host.data(), P->p1_partial.p, nb * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        double sum = 0.0;
        for (int b = 0; b < nb; ++b) sum += P->p1_partial_host[b];
        if (R_out) *R_out = 0.5 * alpha * sum;
        P->have_adj = true;
    });
    return g != MWI_OK ? g : status;
}

mwi_status mwi_normalised_weights(const double* S_empty, int64_t count, double* w_out) {
    return guard([&] {
        MWI_REQUIRE(S_empty && w_out && count >= 0, MWI_EINVAL, "bad argument");
        for (int64_t e = 0; e < count; ++e) {
            const double a = S_empty[2 * e] * S_empty[2 * e] + S_empty[2 * e + 1] * S_empty[2 * e + 1];
            MWI_REQUIRE(a > 0.0 && std::isfinite(a), MWI_EINVAL,
                        "S_empty entry " + std::to_string(e) + " is zero or not finite");
            w_out[e] = 1.0 / a;
        }
    });
}

mwi_status mwi_oras_traffic(mwi_problem_t P, int32_t m, double* bytes) {
    return guard([&] {
        MWI_REQUIRE(P && bytes, MWI_EINVAL, "null argument");
        MWI_REQUIRE(m > 0, MWI_EINVAL, "m must be positive");
        const Decomposition& D = P->dec->D;
        const double e = P->opts.precision == 0 ? 16.0 : 8.0;  // bytes per stored complex entry
        double factor = 0.0, rows = 0.0;
        for (size_t s = 0; s < D.fronts.size(); ++s) {
            const Front& fr = D.fronts[s];
            const double p = fr.p, u = fr.u;
            factor += 2.0 * (p * (p + 1.0) / 2.0 + u * p) + p;  // both sweeps, plus D^-1
            double uc = 0.0;
            for (int32_t q = D.child_ptr[s]; q < D.child_ptr[s + 1]; ++q) uc += D.fronts[D.child[q]].u;
            rows += (p + uc + p + u) + (p + u + p);              // forward, backward
        }
        const double n = (double)P->mesh->T.ndof, nloc = (double)D.sub_off[D.n_sub];
        *bytes = factor * e + (rows + 2.0 * (n + nloc)) * m * e;  // + gather and scatter
    });
}

mwi_status mwi_sweep_levels(mwi_problem_t P, int32_t max_levels, int32_t* n_levels, int64_t* fronts,
                            int64_t* panel_entries, int64_t* update_rows, int64_t* tiles_fwd, int64_t* tiles_bwd) {
    return guard([&] {
        MWI_REQUIRE(P && n_levels && max_levels >= 0, MWI_EINVAL, "bad argument");
        const Decomposition& D = P->dec->D;
        const FrontsDev& F = P->dec->F;
        *n_levels = D.n_levels;
        for (int l = 0; l < std::min<int>(D.n_levels, max_levels); ++l) {
            int64_t e = 0, u = 0;
            for (int q = D.level_ptr[l]; q < D.level_ptr[l + 1]; ++q) {
                const Front& fr = D.fronts[D.level_fronts[q]];
                e += (int64_t)fr.p * (fr.p + fr.u);
                u += fr.u;
            }
            if (fronts) fronts[l] = D.level_ptr[l + 1] - D.level_ptr[l];
            if (panel_entries) panel_entries[l] = e;
            if (update_rows) update_rows[l] = u;
            if (tiles_fwd) tiles_fwd[l] = F.tiles128.f_ptr[l + 1] - F.tiles128.f_ptr[l];
            if (tiles_bwd) tiles_bwd[l] = F.tiles128.p_ptr[l + 1] - F.tiles128.p_ptr[l];
        }
    });
}

mwi_status mwi_recycle_from(mwi_problem_t dst, mwi_problem_t src) {
    return guard([&] {
        MWI_REQUIRE(dst && src && dst != src, MWI_EINVAL, "bad argument");
        MWI_REQUIRE(dst->mesh == src->mesh, MWI_EINVAL, "the problems are on different meshes");
        MWI_REQUIRE(dst->opts.recycle == 1, MWI_ESTATE, "the destination problem was created without recycle = 1");
        MWI_REQUIRE(src->have_fwd, MWI_ESTATE, "the source problem holds no forward solutions");
        const int m = src->m_fwd;
        MWI_REQUIRE(m <= 32, MWI_EINVAL, "recycling takes at most 32 columns");
        const int64_t nm = src->mesh->T.ndof * (int64_t)m;
        // the source's work is complete (calls return after it); order the copy on the destination's stream
        MWI_CUDA(cudaStreamSynchronize(src->st));
        dst->U.ensure(nm);
        MWI_CUDA(cudaMemcpyAsync(dst->U.p, src->U.p, nm * sizeof(double2), cudaMemcpyDeviceToDevice, dst->st));
        dst->rec_m[0] = m;
        dst->rec_m[1] = 0;
        if (src->have_adj) {
            dst->Lam.ensure(nm);
            MWI_CUDA(cudaMemcpyAsync(dst->Lam.p, src->Lam.p, nm * sizeof(double2), cudaMemcpyDeviceToDevice,
                                     dst->st));
            dst->rec_m[1] = m;
        }
        MWI_CUDA(cudaStreamSynchronize(dst->st));
        dst->have_fwd = false;
        dst->have_adj = false;
    });
}

mwi_status mwi_problem_estimate_bytes(mwi_mesh_t M, const mwi_solver_opts* opts, int32_t n_rhs, int64_t* bytes) {
    return guard([&] {
        MWI_REQUIRE(M && bytes && n_rhs >= 1, MWI_EINVAL, "bad argument");
        const mwi_solver_opts o = defaults(opts);
        MWI_REQUIRE(o.precision >= 0 && o.precision <= 2, MWI_EINVAL, "precision must be 0, 1 or 2");
        std::shared_ptr<DecompEntry> E;
        {
            std::lock_guard<std::mutex> lk(M->mu);
            ensure_global(M);
            E = get_decomp(M, o);
        }
        const FrontsDev& F = E->F;
        const double n = (double)M->T.ndof, nt = (double)M->T.nt, nnz = (double)M->A.nnz;
        const double m = std::min(n_rhs, o.max_block), mall = n_rhs;
        const bool mixed = o.precision != 0, nested = o.precision == 2;
        const double fe = mixed ? 8.0 : 16.0;  // bytes of a factor entry
        const double r = o.restart;
        double b = nt * 16 + (double)M->A_fu.face.size() * 16 + nnz * 16 + (double)E->D.B_faces.face.size() * 16 +
                   (double)E->B.nnz * 16;
        b += nested ? nnz * 8 : (mixed ? 2 * nnz * 8 : 0);
        b += ((double)F.ws_total() + (double)F.inv_entries + (double)F.sch_entries[0] + (double)F.sch_entries[1]) * fe;
        if (mixed && o.sweep_engine == 4) b += 2.0 * (double)F.tiled_floats * 4;
        // fields of every column (forward, adjoint, right-hand sides), block copies, residual
        b += 3 * n * mall * 16 + 3 * n * m * 16;
        // local and update vectors of the ORAS application
        b += (2 * (double)F.nloc + (double)F.upd_rows) * (m + 1) * fe + 2 * n * m * 8;
        if (o.block_krylov) b += (r + 2) * n * m * 16 + 2 * n * m * 16;
        else if (o.precision == 1) b += ((r + 1) * 2 + r + 2) * n * m * 8 + 3 * 2 * n * m * 8;
        else if (nested) b += (13 + 12 + 1) * n * m * 16 + (o.inner_iters * 2 + 2) * n * m * 8;
        else b += (2 * r + 2) * n * m * 16;
        if (o.recycle) b += 64 * n * (16 + 8 + 8) + 2 * 64 * n * 8 + n * m * 16;
        // small per-column and reduction arrays
        b += (double)kDotBlocks * (2 * r + 3) * m * 16 + 64.0 * r * r * m + nt * 16;
        *bytes = (int64_t)(1.1 * b) + ((int64_t)16 << 20);
    });
}

mwi_status mwi_problem_device_bytes(mwi_problem_t P, int64_t* bytes) {
    return guard([&] {
        MWI_REQUIRE(P && bytes, MWI_EINVAL, "null argument");
        *bytes = (int64_t)P->device_bytes();
    });
}

mwi_status mwi_kernel_times(mwi_problem_t P, double* ms, int64_t* counts, int32_t reset) {
    return guard([&] {
        MWI_REQUIRE(P, MWI_EINVAL, "null problem");
        harvest_events(P);
        for (int k = 0; k < 4; ++k) {
            if (ms) ms[k] = P->t_ms[k];
            if (counts) counts[k] = P->t_cnt[k];
            if (reset) { P->t_ms[k] = 0; P->t_cnt[k] = 0; }
        }
    });
}

mwi_status mwi_set_coarse_space(mwi_problem_t P, mwi_mesh_t Mc) {
    return guard([&] {
        MWI_REQUIRE(P, MWI_EINVAL, "null problem");
        set_coarse(P, Mc);
    });
}

mwi_status mwi_coarse_info(mwi_problem_t P, int64_t* n_coarse, int64_t* nnz_p, int64_t* nnz_ac, double* setup_ms,
                           int32_t* n_perturbed) {
    return guard([&] {
        MWI_REQUIRE(P, MWI_EINVAL, "null problem");
        const CoarseLevel* L = P->coarse.get();
        if (n_coarse) *n_coarse = L ? L->H.nc : 0;
        if (nnz_p) *nnz_p = L ? (int64_t)L->H.P_col.size() : 0;
        if (nnz_ac) *nnz_ac = L ? (int64_t)L->H.Ac_col.size() : 0;
        if (setup_ms) *setup_ms = L ? L->setup_ms : 0.0;
        if (n_perturbed) *n_perturbed = L ? L->n_perturbed : 0;
    });
}

mwi_status mwi_coarse_operator(mwi_problem_t P, int64_t* p_rp, int32_t* p_col, double* p_val, int64_t* ac_rp,
                               int32_t* ac_col, double* ac_val) {
    return guard([&] {
        MWI_REQUIRE(P, MWI_EINVAL, "null problem");
        MWI_REQUIRE(P->coarse, MWI_ESTATE, "the problem has no coarse space");
        const CoarseHost& H = P->coarse->H;
        if (p_rp) std::copy(H.P_rp.begin(), H.P_rp.end(), p_rp);
        if (p_col) std::copy(H.P_col.begin(), H.P_col.end(), p_col);
        if (p_val) std::copy(H.P_val.begin(), H.P_val.end(), p_val);
        if (ac_rp) std::copy(H.Ac_rp.begin(), H.Ac_rp.end(), ac_rp);
        if (ac_col) std::copy(H.Ac_col.begin(), H.Ac_col.end(), ac_col);
        if (ac_val) {
            const std::vector<double2>& v = P->coarse->Ac_h;
            for (size_t k = 0; k < v.size(); ++k) {
                ac_val[2 * k] = v[k].x;
                ac_val[2 * k + 1] = v[k].y;
            }
        }
    });
}

int64_t mwi_launch_count(void) { return g_launches.load(); }

int64_t mwi_device_alloc_count(void) { return g_device_allocs.load(); }

}  // extern "C"

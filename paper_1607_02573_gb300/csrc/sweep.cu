// Multifrontal forward/backward sweeps of the ORAS local solves as batched
// dense GEMMs (the B_i^{-1} of Eq. ORAS applied to many vectors at once, as
// Section 3 notes for multiple right-hand sides).
//
// Each front's panel holds [L11^{-1}; L21] (partitioned inverse, the
// factorisation replaces L11 by its inverse; D stays on the diagonal), so a
// front's part of L z = w and L^T x = z needs no sequential substitution:
//
//   forward  (deepest level first)
//     assemble:  w_P = Y[P] + children's updates,  w_U = children's updates
//     FWD_P:     y_P = L11^{-1} w_P                       -> Z[P]
//     FWD_U:     w_U = w_U - L21 y_P                      -> update vector of the front
//   backward (root level first)
//     BWD_T:     t_P = D^{-1} y_P - L21^T x_U             -> Z[P]  (x_U: ancestors' final rows)
//     BWD_X:     x_P = L11^{-T} t_P                       -> Y[P]
//
// Every GEMM is tiled over (front, TM-row tile) x (TN columns of the m
// right-hand sides); operand tiles are staged in shared memory with a
// register prefetch of the next k-slab.
#include <algorithm>

#include "common.h"
#include "kernels.h"

namespace mwi {

template <typename C> struct GemmCfg;
template <> struct GemmCfg<float2> { static constexpr int TM = 64, TN = 32, KB = 32; };
template <> struct GemmCfg<double2> { static constexpr int TM = 32, TN = 32, KB = 16; };

template <typename C>
__device__ __forceinline__ C cone() { C r; r.x = 1; r.y = 0; return r; }

struct FrontArgs {
    const int32_t* P;
    const int32_t* U;
    const int32_t* start;
    const int32_t* sub;
    const int64_t* sub_off;
    const int64_t* f_off;
    const int64_t* u_off;
    const int64_t* upd_row;
    const int32_t* urows;
    const int32_t* child_ptr;
    const int32_t* child;
    const int32_t* urel;
    const int64_t* asm_base;
    const int64_t* asm_ptr;
    const int32_t* asm_src;
};

template <typename C, int MODE>
__global__ void __launch_bounds__(256) sweep_gemm_kernel(const int2* __restrict__ tiles, FrontArgs fa,
                                                         const C* __restrict__ ws, C* __restrict__ Y,
                                                         C* __restrict__ Z, C* __restrict__ upd, int m) {
    constexpr int TM = GemmCfg<C>::TM, TN = GemmCfg<C>::TN, KB = GemmCfg<C>::KB;
    constexpr int RM = TM / 16, CN = TN / 16;
    constexpr int AL = TM * KB / 256, BL = KB * TN / 256;
    __shared__ __align__(16) C As[KB][TM + 2];
    __shared__ __align__(16) C Bs[KB][TN + 2];
    const int2 tile = tiles[blockIdx.x];
    const int s = tile.x, row0 = tile.y;
    const int c0 = blockIdx.y * TN;
    const int p = fa.P[s], u = fa.U[s];
    const int64_t f = (int64_t)p + u;
    const C* L = ws + fa.f_off[s];
    const int64_t sbase = fa.sub_off[fa.sub[s]];
    const int64_t rowbase = sbase + fa.start[s];
    const int32_t* ur = fa.urows + fa.u_off[s];
    // output rows and k range
    const int nrows_all = (MODE == 1) ? u : p;
    const int nrows = min(TM, nrows_all - row0);
    int k0, k1;
    if (MODE == 0) { k0 = 0; k1 = min(p, row0 + TM); }
    else if (MODE == 1) { k0 = 0; k1 = p; }
    else if (MODE == 2) { k0 = 0; k1 = u; }
    else { k0 = row0; k1 = p; }
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    auto loadA = [&](int kb, C* areg) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            const int e = tid + 256 * q;
            int i, kk;
            if (MODE <= 1) { i = e % TM; kk = e / TM; }
            else { kk = e % KB; i = e / KB; }
            const int k = kb + kk;
            C a = czero<C>();
            if (i < nrows && k < k1) {
                const int gi = row0 + i;
                if (MODE == 0) {
                    if (k < gi) a = L[(int64_t)k * f + gi];
                    else if (k == gi) a = cone<C>();
                } else if (MODE == 1) {
                    a = L[(int64_t)k * f + p + gi];
                } else if (MODE == 2) {
                    a = L[(int64_t)gi * f + p + k];
                } else {
                    if (k > gi) a = L[(int64_t)gi * f + k];
                    else if (k == gi) a = cone<C>();
                }
            }
            areg[q] = a;
        }
    };
    auto storeA = [&](const C* areg) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            const int e = tid + 256 * q;
            int i, kk;
            if (MODE <= 1) { i = e % TM; kk = e / TM; }
            else { kk = e % KB; i = e / KB; }
            As[kk][i] = areg[q];
        }
    };
    auto loadB = [&](int kb, C* breg) {
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + 256 * q;
            const int c = e % TN, kk = e / TN;
            const int k = kb + kk;
            C b = czero<C>();
            if (k < k1 && c0 + c < m) {
                int64_t row;
                if (MODE == 2) row = sbase + ur[k];
                else row = rowbase + k;
                b = (MODE == 0 || MODE == 2) ? Y[row * m + c0 + c] : Z[row * m + c0 + c];
            }
            breg[q] = b;
        }
    };
    auto storeB = [&](const C* breg) {
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + 256 * q;
            Bs[e / TN][e % TN] = breg[q];
        }
    };

    C acc[RM][CN];
#pragma unroll
    for (int a = 0; a < RM; ++a)
#pragma unroll
        for (int b = 0; b < CN; ++b) acc[a][b] = czero<C>();

    C areg[AL], breg[BL];
    int kb = (k0 / KB) * KB;
    if (kb < k1) {
        loadA(kb, areg);
        loadB(kb, breg);
    }
    for (; kb < k1; kb += KB) {
        __syncthreads();
        storeA(areg);
        storeB(breg);
        __syncthreads();
        if (kb + KB < k1) {
            loadA(kb + KB, areg);
            loadB(kb + KB, breg);
        }
#pragma unroll 8
        for (int kk = 0; kk < KB; ++kk) {
            C av[RM], bv[CN];
#pragma unroll
            for (int a = 0; a < RM; ++a) av[a] = As[kk][ty * RM + a];
#pragma unroll
            for (int b = 0; b < CN; ++b) bv[b] = Bs[kk][tx * CN + b];
#pragma unroll
            for (int a = 0; a < RM; ++a)
#pragma unroll
                for (int b = 0; b < CN; ++b) acc[a][b] = cfma(av[a], bv[b], acc[a][b]);
        }
    }
    // epilogue
#pragma unroll
    for (int a = 0; a < RM; ++a) {
        const int i = ty * RM + a;
        if (i >= nrows) continue;
        const int gi = row0 + i;
#pragma unroll
        for (int b = 0; b < CN; ++b) {
            const int c = c0 + tx * CN + b;
            if (c >= m) continue;
            if (MODE == 0) {
                Z[(rowbase + gi) * m + c] = acc[a][b];
            } else if (MODE == 1) {
                C& d = upd[(fa.upd_row[s] + gi) * m + c];
                d = csub(d, acc[a][b]);
            } else if (MODE == 2) {
                C& z = Z[(rowbase + gi) * m + c];
                z = csub(cmul(z, crecip(L[(int64_t)gi * f + gi])), acc[a][b]);
            } else {
                Y[(rowbase + gi) * m + c] = acc[a][b];
            }
        }
    }
}

// Extend-add of the children's update vectors in gather form, tiled like the
// GEMMs: w_P = Y[P] + children's rows (in place in Y), w_U = children's rows
// (into the front's own update vector).  Every front row sums its sources in
// a fixed order (children ascending), so no atomics are needed.
template <typename C, bool UPART>
__global__ void __launch_bounds__(256) sweep_gather_kernel(const int2* __restrict__ tiles, int tm, FrontArgs fa,
                                                           C* __restrict__ Y, C* __restrict__ upd, int m) {
    const int2 tile = tiles[blockIdx.x];
    const int s = tile.x, row0 = tile.y;
    const int p = fa.P[s], u = fa.U[s];
    const int nrows = min(tm, (UPART ? u : p) - row0);
    const int c = blockIdx.y * 32 + (threadIdx.x & 31);
    if (c >= m) return;
    const int64_t rowbase = fa.sub_off[fa.sub[s]] + fa.start[s];
    const int64_t base = fa.asm_base[s] + (UPART ? p : 0) + row0;
    for (int i = threadIdx.x >> 5; i < nrows; i += 8) {
        const int t = row0 + i;
        C acc = UPART ? czero<C>() : Y[(rowbase + t) * m + c];
        for (int64_t q = fa.asm_ptr[base + i]; q < fa.asm_ptr[base + i + 1]; ++q) {
            const C v = upd[(int64_t)fa.asm_src[q] * m + c];
            acc.x += v.x;
            acc.y += v.y;
        }
        if (UPART) upd[(fa.upd_row[s] + t) * m + c] = acc;
        else Y[(rowbase + t) * m + c] = acc;
    }
}

template <typename C>
static FrontArgs front_args(const FrontsDev& F) {
    FrontArgs a;
    a.P = F.p.p;
    a.U = F.u.p;
    a.start = F.start.p;
    a.sub = F.sub.p;
    a.sub_off = F.sub_off.p;
    a.f_off = F.f_off.p;
    a.u_off = F.u_off.p;
    a.upd_row = F.upd_row.p;
    a.urows = F.urows.p;
    a.child_ptr = F.child_ptr.p;
    a.child = F.child.p;
    a.urel = F.urel.p;
    a.asm_base = F.asm_base.p;
    a.asm_ptr = F.asm_ptr.p;
    a.asm_src = F.asm_src.p;
    return a;
}

template <typename C, int MODE>
static void launch_gemm(const FrontsDev& F, const TileLists& T, int l, const C* ws, C* Y, C* Z, C* upd, int m,
                        cudaStream_t st) {
    const bool upper = MODE == 1;
    const int64_t b = upper ? T.u_ptr[l] : T.p_ptr[l];
    const int64_t e = upper ? T.u_ptr[l + 1] : T.p_ptr[l + 1];
    const int2* tiles = (upper ? T.u_tiles.p : T.p_tiles.p) + b;
    const int tn = GemmCfg<C>::TN;
    for (int64_t off = 0; off < e - b; off += 2147483647LL) {
        const int64_t n = std::min<int64_t>(e - b - off, 2147483647LL);
        if (n <= 0) break;
        dim3 grd((unsigned)n, (unsigned)((m + tn - 1) / tn));
        sweep_gemm_kernel<C, MODE><<<grd, 256, 0, st>>>(tiles + off, front_args<C>(F), ws, Y, Z, upd, m);
        MWI_CHECK_LAUNCH();
    }
}

template <typename C, bool UPART>
static void launch_gather(const FrontsDev& F, const TileLists& T, int l, C* Y, C* upd, int m, cudaStream_t st) {
    const int64_t b = UPART ? T.u_ptr[l] : T.p_ptr[l];
    const int64_t e = UPART ? T.u_ptr[l + 1] : T.p_ptr[l + 1];
    if (e <= b) return;
    const int2* tiles = (UPART ? T.u_tiles.p : T.p_tiles.p) + b;
    dim3 grd((unsigned)(e - b), (unsigned)((m + 31) / 32));
    sweep_gather_kernel<C, UPART><<<grd, 256, 0, st>>>(tiles, T.tm, front_args<C>(F), Y, upd, m);
    MWI_CHECK_LAUNCH();
}

template <typename C>
void sweep_forward_level(const FrontsDev& F, const TileLists& T, int l, const C* ws, C* Y, C* Z, C* upd, int m,
                         cudaStream_t st) {
    launch_gather<C, false>(F, T, l, Y, upd, m, st);
    launch_gather<C, true>(F, T, l, Y, upd, m, st);
    launch_gemm<C, 0>(F, T, l, ws, Y, Z, upd, m, st);
    launch_gemm<C, 1>(F, T, l, ws, Y, Z, upd, m, st);
}

template <typename C>
void sweep_backward_level(const FrontsDev& F, const TileLists& T, int l, const C* ws, C* Y, C* Z, int m,
                          cudaStream_t st) {
    launch_gemm<C, 2>(F, T, l, ws, Y, Z, nullptr, m, st);
    launch_gemm<C, 3>(F, T, l, ws, Y, Z, nullptr, m, st);
}

template <typename C>
const TileLists& tiles_for(const FrontsDev& F);
template <>
const TileLists& tiles_for<float2>(const FrontsDev& F) { return F.tiles64; }
template <>
const TileLists& tiles_for<double2>(const FrontsDev& F) { return F.tiles32; }

template <typename C>
void multifrontal_solve(const FrontsDev& F, const C* ws, C* Y, C* Z, C* upd, int m, cudaStream_t st) {
    const TileLists& T = tiles_for<C>(F);
    const int nlev = (int)F.level_ptr.size() - 1;
    for (int l = 0; l < nlev; ++l) sweep_forward_level<C>(F, T, l, ws, Y, Z, upd, m, st);
    for (int l = nlev - 1; l >= 0; --l) sweep_backward_level<C>(F, T, l, ws, Y, Z, m, st);
}

template void multifrontal_solve<float2>(const FrontsDev&, const float2*, float2*, float2*, float2*, int,
                                         cudaStream_t);
template void multifrontal_solve<double2>(const FrontsDev&, const double2*, double2*, double2*, double2*, int,
                                          cudaStream_t);

int sweep_tile_rows(bool fp32) { return fp32 ? GemmCfg<float2>::TM : GemmCfg<double2>::TM; }

}  // namespace mwi

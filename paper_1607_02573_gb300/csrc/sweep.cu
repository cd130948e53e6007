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

// w_P = Y[P] + children's updates (in place in Y), w_U = children's updates.
template <typename C>
__global__ void __launch_bounds__(256) sweep_assemble_kernel(const int32_t* __restrict__ level_fronts, int lo,
                                                             FrontArgs fa, C* __restrict__ Y, C* __restrict__ upd,
                                                             int m) {
    const int s = level_fronts[lo + blockIdx.x];
    const int p = fa.P[s], u = fa.U[s];
    const int64_t rowbase = fa.sub_off[fa.sub[s]] + fa.start[s];
    C* us = upd + fa.upd_row[s] * m;
    for (int64_t e = threadIdx.x; e < (int64_t)u * m; e += blockDim.x) us[e] = czero<C>();
    __syncthreads();
    for (int q = fa.child_ptr[s]; q < fa.child_ptr[s + 1]; ++q) {
        const int c = fa.child[q];
        const int uc = fa.U[c];
        const int32_t* rel = fa.urel + fa.u_off[c];
        const C* src = upd + fa.upd_row[c] * m;
        for (int64_t e = threadIdx.x; e < (int64_t)uc * m; e += blockDim.x) {
            const int k = (int)(e / m), col = (int)(e - (int64_t)k * m);
            const int t = rel[k];
            const C v = src[e];
            C& d = t < p ? Y[(rowbase + t) * m + col] : us[(int64_t)(t - p) * m + col];
            d.x += v.x;
            d.y += v.y;
        }
        __syncthreads();
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

template <typename C>
void sweep_forward_level(const FrontsDev& F, const TileLists& T, int l, const C* ws, C* Y, C* Z, C* upd, int m,
                         cudaStream_t st) {
    for (int lo = F.level_ptr[l]; lo < F.level_ptr[l + 1]; lo += 65535) {
        const int nf = std::min(65535, F.level_ptr[l + 1] - lo);
        sweep_assemble_kernel<C><<<nf, 256, 0, st>>>(F.level_fronts.p, lo, front_args<C>(F), Y, upd, m);
        MWI_CHECK_LAUNCH();
    }
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

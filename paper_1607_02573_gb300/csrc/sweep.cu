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
#include <type_traits>

#include "common.h"
#include "kernels.h"

namespace mwi {

// tile: TM rows x 32 columns, k-slabs of KB; complex FP32 uses 64-row tiles on
// levels of large fronts and 32-row tiles on levels of small fronts
template <typename C> struct GemmKB;
template <> struct GemmKB<float2> { static constexpr int KB = 32; };
template <> struct GemmKB<double2> { static constexpr int KB = 16; };
static constexpr int kTN = 32;

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

template <typename C, int MODE, int TM>
__global__ void __launch_bounds__(256) sweep_gemm_kernel(const int2* __restrict__ tiles, FrontArgs fa,
                                                         const C* __restrict__ ws, C* __restrict__ Y,
                                                         C* __restrict__ Z, C* __restrict__ upd, int m) {
    constexpr int TN = kTN, KB = GemmKB<C>::KB;
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

// ---------------------------------------------------------------------------
// The same four products on the tensor cores (complex FP32 factors).
// A complex product C = A B is one real product C' = A' B' with
//   A'[i][2k] = Re A(i,k), A'[i][2k+1] = Im A(i,k)      (interleaved storage as is)
//   B'[2k][2n] = Re B, B'[2k+1][2n] = -Im B, B'[2k][2n+1] = Im B, B'[2k+1][2n+1] = Re B
// so C'[i][2n] = Re C(i,n) and C'[i][2n+1] = Im C(i,n).  The real product
// runs as mma.m16n8k8 TF32 with FP32 accumulation; SPLIT = 1 splits every
// operand into a TF32 head and a TF32 tail (x = hi + lo) and accumulates
// hi*hi + hi*lo + lo*hi, which restores about FP32 accuracy.
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int MODE, int TM, int SPLIT>
__global__ void __launch_bounds__(256) sweep_mma_kernel(const int2* __restrict__ tiles, FrontArgs fa,
                                                        const float2* __restrict__ ws, float2* __restrict__ Y,
                                                        float2* __restrict__ Z, float2* __restrict__ upd, int m) {
    typedef float2 C;
    constexpr int KB = 16;              // complex k per slab (32 real)
    constexpr int WR = TM / 16;         // warps along rows
    constexpr int WC = 8 / WR;          // warps along (real) columns
    constexpr int NT = 64 / (8 * WC);   // n8 tiles per warp (64 real columns per block)
    constexpr int AL = TM * KB / 256, BL = KB * 32 / 256;
    __shared__ __align__(16) float As[TM][2 * KB + 4];
    __shared__ __align__(16) float Bs[2 * KB][64 + 8];
    const int2 tile = tiles[blockIdx.x];
    const int s = tile.x, row0 = tile.y;
    const int c0 = blockIdx.y * 32;
    const int p = fa.P[s], u = fa.U[s];
    const int64_t f = (int64_t)p + u;
    const C* L = ws + fa.f_off[s];
    const int64_t sbase = fa.sub_off[fa.sub[s]];
    const int64_t rowbase = sbase + fa.start[s];
    const int32_t* ur = fa.urows + fa.u_off[s];
    const int nrows_all = (MODE == 1) ? u : p;
    const int nrows = min(TM, nrows_all - row0);
    int k0, k1;
    if (MODE == 0) { k0 = 0; k1 = min(p, row0 + TM); }
    else if (MODE == 1) { k0 = 0; k1 = p; }
    else if (MODE == 2) { k0 = 0; k1 = u; }
    else { k0 = row0; k1 = p; }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = warp % WR, wc = warp / WR;
    const int g = lane >> 2, t = lane & 3;

    auto loadA = [&](int kb, C* areg) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            const int e = tid + 256 * q;
            int i, kk;
            if (MODE <= 1) { i = e % TM; kk = e / TM; }
            else { kk = e % KB; i = e / KB; }
            const int k = kb + kk;
            C a = make_float2(0.f, 0.f);
            if (i < nrows && k < k1) {
                const int gi = row0 + i;
                if (MODE == 0) {
                    if (k < gi) a = L[(int64_t)k * f + gi];
                    else if (k == gi) a = make_float2(1.f, 0.f);
                } else if (MODE == 1) {
                    a = L[(int64_t)k * f + p + gi];
                } else if (MODE == 2) {
                    a = L[(int64_t)gi * f + p + k];
                } else {
                    if (k > gi) a = L[(int64_t)gi * f + k];
                    else if (k == gi) a = make_float2(1.f, 0.f);
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
            As[i][2 * kk] = areg[q].x;
            As[i][2 * kk + 1] = areg[q].y;
        }
    };
    auto loadB = [&](int kb, C* breg) {
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + 256 * q;
            const int c = e % 32, kk = e / 32;
            const int k = kb + kk;
            C b = make_float2(0.f, 0.f);
            if (k < k1 && c0 + c < m) {
                const int64_t row = (MODE == 2) ? sbase + ur[k] : rowbase + k;
                b = (MODE == 0 || MODE == 2) ? Y[row * m + c0 + c] : Z[row * m + c0 + c];
            }
            breg[q] = b;
        }
    };
    auto storeB = [&](const C* breg) {
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + 256 * q;
            const int c = e % 32, kk = e / 32;
            Bs[2 * kk][2 * c] = breg[q].x;
            Bs[2 * kk + 1][2 * c] = -breg[q].y;
            Bs[2 * kk][2 * c + 1] = breg[q].y;
            Bs[2 * kk + 1][2 * c + 1] = breg[q].x;
        }
    };

    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;

    C areg[AL], breg[BL];
    int kb = (k0 / KB) * KB;
    if (kb < k1) {
        loadA(kb, areg);
        loadB(kb, breg);
    }
    const int r0 = wr * 16;
    for (; kb < k1; kb += KB) {
        __syncthreads();
        storeA(areg);
        storeB(breg);
        __syncthreads();
        if (kb + KB < k1) {
            loadA(kb + KB, areg);
            loadB(kb + KB, breg);
        }
#pragma unroll
        for (int ks = 0; ks < 2 * KB; ks += 8) {
            const float af[4] = {As[r0 + g][ks + t], As[r0 + g + 8][ks + t], As[r0 + g][ks + t + 4],
                                 As[r0 + g + 8][ks + t + 4]};
            uint32_t ah[4], al[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ah[q] = to_tf32(af[q]);
                if (SPLIT) al[q] = to_tf32(af[q] - __uint_as_float(ah[q]));
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int n0 = wc * (8 * NT) + nt * 8;
                const float bf[2] = {Bs[ks + t][n0 + g], Bs[ks + t + 4][n0 + g]};
                uint32_t bh[2], bl[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    bh[q] = to_tf32(bf[q]);
                    if (SPLIT) bl[q] = to_tf32(bf[q] - __uint_as_float(bh[q]));
                }
                if (SPLIT) {
                    mma_tf32(acc[nt], al, bh);
                    mma_tf32(acc[nt], ah, bl);
                }
                mma_tf32(acc[nt], ah, bh);
            }
        }
    }
    // epilogue: thread holds (row g / g+8, complex column (n0 / 2) + t) as (re, im) pairs
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int cc = c0 + (wc * (8 * NT) + nt * 8) / 2 + t;
        if (cc >= m) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = r0 + g + 8 * h;
            if (i >= nrows) continue;
            const int gi = row0 + i;
            const C v = make_float2(acc[nt][2 * h], acc[nt][2 * h + 1]);
            if (MODE == 0) {
                Z[(rowbase + gi) * m + cc] = v;
            } else if (MODE == 1) {
                C& d = upd[(fa.upd_row[s] + gi) * m + cc];
                d = csub(d, v);
            } else if (MODE == 2) {
                C& z = Z[(rowbase + gi) * m + cc];
                z = csub(cmul(z, crecip(L[(int64_t)gi * f + gi])), v);
            } else {
                Y[(rowbase + gi) * m + cc] = v;
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

template <typename C>
static bool small_tiles(const FrontsDev& F, int l, bool upart) {
    if (sizeof(C) == sizeof(double2)) return true;  // complex FP64 always uses 32-row tiles
    return (upart ? F.level_umean[l] : F.level_pmean[l]) < 40.0;
}

template <typename C, int MODE, int TM>
static void launch_gemm_tm(const FrontsDev& F, const TileLists& T, int l, const C* ws, C* Y, C* Z, C* upd, int m,
                           int tc, cudaStream_t st) {
    const bool upart = MODE == 1;
    const int64_t b = upart ? T.u_ptr[l] : T.p_ptr[l];
    const int64_t e = upart ? T.u_ptr[l + 1] : T.p_ptr[l + 1];
    if (e <= b) return;
    const int2* tiles = (upart ? T.u_tiles.p : T.p_tiles.p) + b;
    dim3 grd((unsigned)(e - b), (unsigned)((m + kTN - 1) / kTN));
    if constexpr (std::is_same<C, float2>::value) {
        if (tc == 1) {
            sweep_mma_kernel<MODE, TM, 1><<<grd, 256, 0, st>>>(tiles, front_args<C>(F), ws, Y, Z, upd, m);
            MWI_CHECK_LAUNCH();
            return;
        }
        if (tc == 2) {
            sweep_mma_kernel<MODE, TM, 0><<<grd, 256, 0, st>>>(tiles, front_args<C>(F), ws, Y, Z, upd, m);
            MWI_CHECK_LAUNCH();
            return;
        }
    }
    sweep_gemm_kernel<C, MODE, TM><<<grd, 256, 0, st>>>(tiles, front_args<C>(F), ws, Y, Z, upd, m);
    MWI_CHECK_LAUNCH();
}

template <typename C, int MODE>
static void launch_gemm(const FrontsDev& F, int l, const C* ws, C* Y, C* Z, C* upd, int m, int tc,
                        cudaStream_t st) {
    if (small_tiles<C>(F, l, MODE == 1)) launch_gemm_tm<C, MODE, 32>(F, F.tiles32, l, ws, Y, Z, upd, m, tc, st);
    else launch_gemm_tm<C, MODE, 64>(F, F.tiles64, l, ws, Y, Z, upd, m, tc, st);
}

template <typename C, bool UPART>
static void launch_gather(const FrontsDev& F, int l, C* Y, C* upd, int m, cudaStream_t st) {
    const TileLists& T = small_tiles<C>(F, l, UPART) ? F.tiles32 : F.tiles64;
    const int64_t b = UPART ? T.u_ptr[l] : T.p_ptr[l];
    const int64_t e = UPART ? T.u_ptr[l + 1] : T.p_ptr[l + 1];
    if (e <= b) return;
    const int2* tiles = (UPART ? T.u_tiles.p : T.p_tiles.p) + b;
    dim3 grd((unsigned)(e - b), (unsigned)((m + 31) / 32));
    sweep_gather_kernel<C, UPART><<<grd, 256, 0, st>>>(tiles, T.tm, front_args<C>(F), Y, upd, m);
    MWI_CHECK_LAUNCH();
}

template <typename C>
void sweep_forward_level(const FrontsDev& F, int l, const C* ws, C* Y, C* Z, C* upd, int m, int tc,
                         cudaStream_t st) {
    launch_gather<C, false>(F, l, Y, upd, m, st);
    launch_gather<C, true>(F, l, Y, upd, m, st);
    launch_gemm<C, 0>(F, l, ws, Y, Z, upd, m, tc, st);
    launch_gemm<C, 1>(F, l, ws, Y, Z, upd, m, tc, st);
}

template <typename C>
void sweep_backward_level(const FrontsDev& F, int l, const C* ws, C* Y, C* Z, int m, int tc, cudaStream_t st) {
    launch_gemm<C, 2>(F, l, ws, Y, Z, nullptr, m, tc, st);
    launch_gemm<C, 3>(F, l, ws, Y, Z, nullptr, m, tc, st);
}

template <typename C>
void multifrontal_solve(const FrontsDev& F, const C* ws, C* Y, C* Z, C* upd, int m, int tc, cudaStream_t st) {
    const int nlev = (int)F.level_ptr.size() - 1;
    for (int l = 0; l < nlev; ++l) sweep_forward_level<C>(F, l, ws, Y, Z, upd, m, tc, st);
    for (int l = nlev - 1; l >= 0; --l) sweep_backward_level<C>(F, l, ws, Y, Z, m, tc, st);
}

template void multifrontal_solve<float2>(const FrontsDev&, const float2*, float2*, float2*, float2*, int, int,
                                         cudaStream_t);
template void multifrontal_solve<double2>(const FrontsDev&, const double2*, double2*, double2*, double2*, int, int,
                                          cudaStream_t);

int sweep_tile_rows(bool large) { return large ? 64 : 32; }

}  // namespace mwi

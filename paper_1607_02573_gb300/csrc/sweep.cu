// Multifrontal forward/backward sweeps of the ORAS local solves as batched
// dense GEMMs (the B_i^{-1} of Eq. ORAS applied to many vectors at once, as
// Section 3 notes for multiple right-hand sides).
//
// After factorisation each front's f x p panel holds the first p columns of
// the inverse of its unit lower block [L11 0; L21 I], i.e. [L11^{-1}; -G]
// with G = L21 L11^{-1}, with a unit diagonal and zeros above it, and D^{-1}
// sits after the panels, indexed by local row (partitioned inverse).  With
// B = L D L^T, a front's part of L z = w and L^T x = D^{-1} z is then one
// dependency-free product per direction:
//
//   forward  (deepest level first)
//     extend-add: w_P = Y[P] + children's update rows          (in place in Y)
//     FWD:        [z_P; w_U] = [L11^{-1}; -G] w_P + [0; children's rows]
//                 Z[P] <- D^{-1} z_P, w_U -> the front's update vector
//   backward (root level first)
//     BWD:        x_P = [L11^{-T}, -G^T] [D^{-1} z_P; x_U]      -> Y[P]
//                 (x_U: the ancestors' final rows, through the update-row list)
//
// since L21 z_P = G w_P and L11^{-T} L21^T = G^T.  The panel is the A operand
// as stored: FWD reads it (rows = front rows), BWD its transpose (rows =
// pivots).  Every product is tiled over (front, TM-row tile) x (32 columns of
// the m right-hand sides); a tile's geometry comes in one descriptor, and the
// loads that do not depend on the product (gather indices, the children's
// rows, D^{-1}, update-row indices) are issued before the k loop, so that a
// tile waits on few dependent memory round trips.
#include <algorithm>
#include <type_traits>

#include "common.h"
#include "kernels.h"

namespace mwi {

enum { kFwd = 0, kBwd = 1 };

template <typename C> struct GemmKB;
template <> struct GemmKB<float2> { static constexpr int KB = 32; };
template <> struct GemmKB<double2> { static constexpr int KB = 16; };
static constexpr int kTN = 32;

// update-row indices of a BWD tile kept in shared memory (larger update sets
// read them from global memory)
static constexpr int kUrCap = 1024;

struct Geom {
    int p, f, row0, nrows, k0, k1;
};

template <int MODE>
__device__ __forceinline__ Geom tile_geom(const TileDesc& d, int tm) {
    Geom g;
    g.p = d.p;
    g.f = d.f;
    g.row0 = d.row0;
    if (MODE == kFwd) {
        // rows gi < p: triangle of L11^{-1} (k <= gi); rows gi >= p: -G (all k < p)
        g.nrows = min(tm, g.f - g.row0);
        g.k0 = 0;
        g.k1 = min(g.p, g.row0 + tm);
    } else {
        // x_P rows: k over the pivots at or after the row, then the update rows
        g.nrows = min(tm, g.p - g.row0);
        g.k0 = g.row0;
        g.k1 = g.f;
    }
    return g;
}

// address of A(gi, k): FWD panel column k, BWD its transpose
template <typename C, int MODE>
__device__ __forceinline__ const C* a_ptr(const C* L, int f, int gi, int k) {
    return MODE == kFwd ? L + (int64_t)k * f + gi : L + (int64_t)gi * f + k;
}

// children's update rows that add into front row gi (fixed order)
template <typename C>
__device__ __forceinline__ C children_sum(const int2* __restrict__ asm2, int64_t row, const C* __restrict__ upd,
                                          int c, int m) {
    const int2 src = asm2[row];
    C acc = czero<C>();
    if (src.x >= 0) acc = upd[(int64_t)src.x * m + c];
    if (src.y >= 0) {
        const C v = upd[(int64_t)src.y * m + c];
        acc.x += v.x;
        acc.y += v.y;
    }
    return acc;
}

// ---------------------------------------------------------------------------
// CUDA-core form (complex FP32 or FP64): 16 x 16 threads, each RM x CN outputs,
// k-slabs staged in shared memory with a register prefetch of the next slab.
template <typename C, int MODE, int TM>
__global__ void __launch_bounds__(256) sweep_gemm_kernel(const TileDesc* __restrict__ tiles,
                                                         const int32_t* __restrict__ urows,
                                                         const int2* __restrict__ asm2, const C* __restrict__ ws,
                                                         const C* __restrict__ dinv, C* __restrict__ Y,
                                                         C* __restrict__ Z, C* __restrict__ upd, int m) {
    constexpr int TN = kTN, KB = GemmKB<C>::KB;
    constexpr int RM = TM / 16, CN = TN / 16;
    constexpr int AL = TM * KB / 256, BL = KB * TN / 256;
    __shared__ __align__(16) C As[KB][TM + 2];
    __shared__ __align__(16) C Bs[KB][TN + 2];
    const TileDesc d = tiles[blockIdx.x];
    const Geom g = tile_geom<MODE>(d, TM);
    const int c0 = blockIdx.y * TN;
    const C* L = ws + d.a_off;
    const int32_t* ur = urows + d.u_off;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    // FWD: rows fastest (panel columns are contiguous); BWD: k fastest
    auto a_index = [&](int e, int& i, int& kk) {
        if (MODE == kFwd) { i = e % TM; kk = e / TM; }
        else { kk = e % KB; i = e / KB; }
    };
    auto loadA = [&](int kb, C* areg) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            int i, kk;
            a_index(tid + 256 * q, i, kk);
            const int k = kb + kk;
            areg[q] = (i < g.nrows && k < g.k1) ? *a_ptr<C, MODE>(L, g.f, g.row0 + i, k) : czero<C>();
        }
    };
    auto storeA = [&](const C* areg) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            int i, kk;
            a_index(tid + 256 * q, i, kk);
            As[kk][i] = areg[q];
        }
    };
    auto loadB = [&](int kb, C* breg) {
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + 256 * q;
            const int c = e % TN, k = kb + e / TN;
            C b = czero<C>();
            if (k < g.k1 && c0 + c < m) {
                if (MODE == kFwd) b = Y[(d.rowbase + k) * m + c0 + c];
                else if (k < g.p) b = Z[(d.rowbase + k) * m + c0 + c];
                else b = Y[(d.sbase + ur[k - g.p]) * m + c0 + c];
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
    int kb = (g.k0 / KB) * KB;
    if (kb < g.k1) {
        loadA(kb, areg);
        loadB(kb, breg);
    }
    for (; kb < g.k1; kb += KB) {
        __syncthreads();
        storeA(areg);
        storeB(breg);
        __syncthreads();
        if (kb + KB < g.k1) {
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
#pragma unroll
    for (int a = 0; a < RM; ++a) {
        const int i = ty * RM + a;
        if (i >= g.nrows) continue;
        const int gi = g.row0 + i;
#pragma unroll
        for (int b = 0; b < CN; ++b) {
            const int c = c0 + tx * CN + b;
            if (c >= m) continue;
            const C v = acc[a][b];
            if (MODE == kBwd) Y[(d.rowbase + gi) * m + c] = v;
            else if (gi < g.p) Z[(d.rowbase + gi) * m + c] = cmul(v, dinv[d.rowbase + gi]);
            else upd[(d.upd_row + gi - g.p) * m + c] = cadd(v, children_sum<C>(asm2, d.asm_base + gi, upd, c, m));
        }
    }
}

// ---------------------------------------------------------------------------
// The same products on the tensor cores (complex FP32 factors).
// A complex product C = A B is one real product C' = A' B' with
//   A'[i][2k] = Re A(i,k), A'[i][2k+1] = Im A(i,k)      (interleaved storage as is)
//   B'[2k][2n] = Re B, B'[2k+1][2n] = -Im B, B'[2k][2n+1] = Im B, B'[2k+1][2n+1] = Re B
// so C'[i][2n] = Re C(i,n) and C'[i][2n+1] = Im C(i,n).  The real product
// runs as mma.m16n8k8 TF32 with FP32 accumulation; operands are rounded to
// TF32 once, when a slab is written to shared memory (one slab in registers
// ahead of the one being multiplied).  SPLIT = 1 also keeps the TF32 tail of
// every operand (x = hi + lo) and accumulates hi*hi + hi*lo + lo*hi, which
// restores about FP32 accuracy.
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
__global__ void __launch_bounds__(256, 4) sweep_mma_kernel(const TileDesc* __restrict__ tiles,
                                                           const int32_t* __restrict__ urows,
                                                           const int2* __restrict__ asm2,
                                                           const float2* __restrict__ ws,
                                                           const float2* __restrict__ dinv, float2* __restrict__ Y,
                                                           float2* __restrict__ Z, float2* __restrict__ upd, int m) {
    typedef float2 C;
    constexpr int KB = SPLIT ? 16 : 32;  // complex k per slab
    constexpr int WR = TM / 16;          // warps along rows
    constexpr int WC = 8 / WR;           // warps along (real) columns
    constexpr int NT = 64 / (8 * WC);    // n8 tiles per warp (64 real columns per block)
    constexpr int AL = TM * KB / 256, BL = KB * 32 / 256;
    constexpr int AP = 2 * KB + 4, BP = 64 + 8;  // padded row lengths (bank spread)
    constexpr int NS = SPLIT ? 2 : 1;            // head, and tail when split
    __shared__ __align__(16) uint32_t As[NS][TM][AP];
    __shared__ __align__(16) uint32_t Bs[NS][2 * KB][BP];
    __shared__ int sur[MODE == kBwd ? kUrCap : 1];
    const TileDesc d = tiles[blockIdx.x];
    const Geom g = tile_geom<MODE>(d, TM);
    const int c0 = blockIdx.y * 32;
    const C* L = ws + d.a_off;
    const int32_t* ur = urows + d.u_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wr = warp % WR, wc = warp / WR;
    const int gq = lane >> 2, t = lane & 3;
    const int r0 = wr * 16;
    const int u = g.f - g.p;
    const bool ur_smem = MODE == kBwd && u <= kUrCap;
    if (MODE == kBwd && ur_smem)
        for (int j = tid; j < u; j += 256) sur[j] = ur[j];

    // loads independent of the product: FWD update rows start from the
    // children's rows, FWD pivot rows fetch their D^{-1}
    float acc[NT][4];
    C dv[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
    if (MODE == kFwd) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = r0 + gq + 8 * h, gi = g.row0 + i;
            if (i >= g.nrows) continue;
            if (gi < g.p) {
                dv[h] = dinv[d.rowbase + gi];
                continue;
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int cc = c0 + (wc * (8 * NT) + nt * 8) / 2 + t;
                if (cc >= m) continue;
                const C v = children_sum<C>(asm2, d.asm_base + gi, upd, cc, m);
                acc[nt][2 * h] = v.x;
                acc[nt][2 * h + 1] = v.y;
            }
        }
    }
    if (MODE == kBwd && ur_smem) __syncthreads();

    // FWD: a warp takes 8 consecutive rows of 4 panel columns (full 32-byte
    // sectors, 2-way bank conflicts on the stores); BWD: k fastest
    auto a_index = [&](int e, int& i, int& kk) {
        if (MODE == kFwd) {
            const int lane_ = e & 31, w = e >> 5;
            constexpr int IG = TM / 8;
            i = 8 * (w % IG) + (lane_ & 7);
            kk = 4 * (w / IG) + (lane_ >> 3);
        } else {
            kk = e % KB;
            i = e / KB;
        }
    };
    auto loadA = [&](int kb, C* areg) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            int i, kk;
            a_index(tid + 256 * q, i, kk);
            const int k = kb + kk;
            areg[q] = (i < g.nrows && k < g.k1) ? *a_ptr<C, MODE>(L, g.f, g.row0 + i, k) : make_float2(0.f, 0.f);
        }
    };
    auto storeA = [&](const C* areg) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            int i, kk;
            a_index(tid + 256 * q, i, kk);
            const uint32_t rh = to_tf32(areg[q].x), ih = to_tf32(areg[q].y);
            As[0][i][2 * kk] = rh;
            As[0][i][2 * kk + 1] = ih;
            if (SPLIT) {
                As[NS - 1][i][2 * kk] = to_tf32(areg[q].x - __uint_as_float(rh));
                As[NS - 1][i][2 * kk + 1] = to_tf32(areg[q].y - __uint_as_float(ih));
            }
        }
    };
    auto loadB = [&](int kb, C* breg) {
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + 256 * q;
            const int c = e % 32, k = kb + e / 32;
            C b = make_float2(0.f, 0.f);
            if (k < g.k1 && c0 + c < m) {
                if (MODE == kFwd) b = Y[(d.rowbase + k) * m + c0 + c];
                else if (k < g.p) b = Z[(d.rowbase + k) * m + c0 + c];
                else b = Y[(d.sbase + (ur_smem ? sur[k - g.p] : ur[k - g.p])) * m + c0 + c];
            }
            breg[q] = b;
        }
    };
    // TF32 rounding is symmetric, so the rounded -Im is the rounded Im with its sign flipped
    auto storeB = [&](const C* breg) {
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + 256 * q;
            const int c = e % 32, kk = e / 32;
            const uint32_t rh = to_tf32(breg[q].x), ih = to_tf32(breg[q].y);
            Bs[0][2 * kk][2 * c] = rh;
            Bs[0][2 * kk + 1][2 * c] = ih ^ 0x80000000u;
            Bs[0][2 * kk][2 * c + 1] = ih;
            Bs[0][2 * kk + 1][2 * c + 1] = rh;
            if (SPLIT) {
                const uint32_t rl = to_tf32(breg[q].x - __uint_as_float(rh));
                const uint32_t il = to_tf32(breg[q].y - __uint_as_float(ih));
                Bs[NS - 1][2 * kk][2 * c] = rl;
                Bs[NS - 1][2 * kk + 1][2 * c] = il ^ 0x80000000u;
                Bs[NS - 1][2 * kk][2 * c + 1] = il;
                Bs[NS - 1][2 * kk + 1][2 * c + 1] = rl;
            }
        }
    };

    C areg[AL], breg[BL];
    int kb = (g.k0 / KB) * KB;
    if (kb < g.k1) {
        loadA(kb, areg);
        loadB(kb, breg);
    }
    for (; kb < g.k1; kb += KB) {
        __syncthreads();
        storeA(areg);
        storeB(breg);
        __syncthreads();
        if (kb + KB < g.k1) {
            loadA(kb + KB, areg);
            loadB(kb + KB, breg);
        }
#pragma unroll
        for (int ks = 0; ks < 2 * KB; ks += 8) {
            uint32_t ah[4], al[4];
            ah[0] = As[0][r0 + gq][ks + t];
            ah[1] = As[0][r0 + gq + 8][ks + t];
            ah[2] = As[0][r0 + gq][ks + t + 4];
            ah[3] = As[0][r0 + gq + 8][ks + t + 4];
            if (SPLIT) {
                al[0] = As[NS - 1][r0 + gq][ks + t];
                al[1] = As[NS - 1][r0 + gq + 8][ks + t];
                al[2] = As[NS - 1][r0 + gq][ks + t + 4];
                al[3] = As[NS - 1][r0 + gq + 8][ks + t + 4];
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int n0 = wc * (8 * NT) + nt * 8;
                const uint32_t bh[2] = {Bs[0][ks + t][n0 + gq], Bs[0][ks + t + 4][n0 + gq]};
                if (SPLIT) {
                    const uint32_t bl[2] = {Bs[NS - 1][ks + t][n0 + gq], Bs[NS - 1][ks + t + 4][n0 + gq]};
                    mma_tf32(acc[nt], al, bh);
                    mma_tf32(acc[nt], ah, bl);
                }
                mma_tf32(acc[nt], ah, bh);
            }
        }
    }
    // epilogue: thread holds (rows gq / gq+8, complex column (n0 / 2) + t) as (re, im) pairs
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int cc = c0 + (wc * (8 * NT) + nt * 8) / 2 + t;
        if (cc >= m) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = r0 + gq + 8 * h;
            if (i >= g.nrows) continue;
            const int gi = g.row0 + i;
            const C v = make_float2(acc[nt][2 * h], acc[nt][2 * h + 1]);
            if (MODE == kBwd) Y[(d.rowbase + gi) * m + cc] = v;
            else if (gi < g.p) Z[(d.rowbase + gi) * m + cc] = cmul(v, dv[h]);
            else upd[(d.upd_row + gi - g.p) * m + cc] = v;
        }
    }
}

// Extend-add of the children's update vectors into the pivot rows, in gather
// form and tiled like the products: w_P = Y[P] + children's rows (in place in
// Y), in a fixed order, so no atomics are needed.  (The update rows are
// gathered by the FWD product itself.)
template <typename C>
__global__ void __launch_bounds__(256) sweep_gather_kernel(const TileDesc* __restrict__ tiles, int tm,
                                                           const int2* __restrict__ asm2, C* __restrict__ Y,
                                                           const C* __restrict__ upd, int m) {
    const TileDesc d = tiles[blockIdx.x];
    const int nrows = min(tm, d.p - d.row0);
    const int c = blockIdx.y * 32 + (threadIdx.x & 31);
    if (c >= m) return;
    for (int i = threadIdx.x >> 5; i < nrows; i += 8) {
        const int2 src = asm2[d.asm_base + d.row0 + i];
        if (src.x < 0) continue;
        C& y = Y[(d.rowbase + d.row0 + i) * m + c];
        C acc = y;
        C v = upd[(int64_t)src.x * m + c];
        acc.x += v.x;
        acc.y += v.y;
        if (src.y >= 0) {
            v = upd[(int64_t)src.y * m + c];
            acc.x += v.x;
            acc.y += v.y;
        }
        y = acc;
    }
}

// 32-row tiles where the level's mean row count is small (FWD: f; BWD and the
// extend-add: p); complex FP64 always uses 32-row tiles
template <typename C>
static bool small_tiles(const FrontsDev& F, int l, bool frows) {
    if (sizeof(C) == sizeof(double2)) return true;
    return (frows ? F.level_fmean[l] : F.level_pmean[l]) < 40.0;
}

template <typename C, int MODE, int TM>
static void launch_gemm_tm(const FrontsDev& F, const TileLists& T, int l, const C* ws, C* Y, C* Z, C* upd, int m,
                           int tc, cudaStream_t st) {
    const bool frows = MODE == kFwd;
    const int64_t b = frows ? T.f_ptr[l] : T.p_ptr[l];
    const int64_t e = frows ? T.f_ptr[l + 1] : T.p_ptr[l + 1];
    if (e <= b) return;
    const TileDesc* tiles = (frows ? T.f_tiles.p : T.p_tiles.p) + b;
    dim3 grd((unsigned)(e - b), (unsigned)((m + kTN - 1) / kTN));
    const C* dinv = ws + F.ws_entries;
    if constexpr (std::is_same<C, float2>::value) {
        if (tc == 1 || tc == 2) {
            if (tc == 1)
                sweep_mma_kernel<MODE, TM, 1><<<grd, 256, 0, st>>>(tiles, F.urows.p, F.asm2.p, ws, dinv, Y, Z, upd, m);
            else
                sweep_mma_kernel<MODE, TM, 0><<<grd, 256, 0, st>>>(tiles, F.urows.p, F.asm2.p, ws, dinv, Y, Z, upd, m);
            MWI_CHECK_LAUNCH();
            return;
        }
    }
    sweep_gemm_kernel<C, MODE, TM><<<grd, 256, 0, st>>>(tiles, F.urows.p, F.asm2.p, ws, dinv, Y, Z, upd, m);
    MWI_CHECK_LAUNCH();
}

template <typename C, int MODE>
static void launch_gemm(const FrontsDev& F, int l, const C* ws, C* Y, C* Z, C* upd, int m, int tc,
                        cudaStream_t st) {
    if (small_tiles<C>(F, l, MODE == kFwd)) launch_gemm_tm<C, MODE, 32>(F, F.tiles32, l, ws, Y, Z, upd, m, tc, st);
    else launch_gemm_tm<C, MODE, 64>(F, F.tiles64, l, ws, Y, Z, upd, m, tc, st);
}

template <typename C>
static void launch_gather(const FrontsDev& F, int l, C* Y, const C* upd, int m, cudaStream_t st) {
    if (l == 0) return;  // the deepest level holds leaves only
    const TileLists& T = small_tiles<C>(F, l, false) ? F.tiles32 : F.tiles64;
    const int64_t b = T.p_ptr[l], e = T.p_ptr[l + 1];
    if (e <= b) return;
    dim3 grd((unsigned)(e - b), (unsigned)((m + 31) / 32));
    sweep_gather_kernel<C><<<grd, 256, 0, st>>>(T.p_tiles.p + b, T.tm, F.asm2.p, Y, upd, m);
    MWI_CHECK_LAUNCH();
}

// one level's product on the fifth-generation tensor cores (sweep_tc.cu)
template <typename C>
static void launch_tc_product(const FrontsDev& F, int l, bool backward, const C* ws, C* Y, C* Z, C* upd, int m,
                              const SweepCfg& sc, cudaStream_t st) {
    if constexpr (std::is_same<C, float2>::value) {
        const TileLists& T = F.tiles128;
        const int64_t b = backward ? T.p_ptr[l] : T.f_ptr[l];
        const int64_t e = backward ? T.p_ptr[l + 1] : T.f_ptr[l + 1];
        sweep_tc_level(backward, (backward ? T.p_tiles.p : T.f_tiles.p) + b, e - b, m, F.urows.p, F.asm2.p,
                       sc.wt + (backward ? F.tiled_floats : 0), ws + F.ws_entries, Y, Z, upd, sc.err, st);
    } else {
        throw Error(MWI_EINVAL, "internal: tensor-core sweeps need complex FP32 factors");
    }
}

template <typename C>
void multifrontal_solve(const FrontsDev& F, const C* ws, C* Y, C* Z, C* upd, int m, const SweepCfg& sc,
                        cudaStream_t st) {
    const int nlev = (int)F.level_ptr.size() - 1;
    // the tcgen05 engine moves right-hand-side rows by 16-byte bulk copies
    // (oras_apply pads the local vectors to an even column count)
    const bool tc5 = sc.tc == 4;
    const int tc = sc.tc;
    MWI_REQUIRE(!tc5 || (sc.wt && sc.err), MWI_EINVAL, "internal: tensor-core sweeps without the tiled panels");
    MWI_REQUIRE(!tc5 || (m % 2) == 0, MWI_EINVAL, "internal: tensor-core sweeps need an even column count");
    for (int l = 0; l < nlev; ++l) {
        launch_gather<C>(F, l, Y, upd, m, st);
        if (tc5) launch_tc_product<C>(F, l, false, ws, Y, Z, upd, m, sc, st);
        else launch_gemm<C, kFwd>(F, l, ws, Y, Z, upd, m, tc, st);
    }
    // backward levels of small fronts (mean pivot count below 40): the TF32
    // mma.sync kernel with 32-row tiles beats the 128-row tcgen05 tiles there
    // (one tile per front either way; the per-tile pipeline set-up of the
    // tcgen05 kernel dominates), so the tcgen05 engine hands those levels to it
    for (int l = nlev - 1; l >= 0; --l) {
        if (tc5 && !small_tiles<C>(F, l, false)) launch_tc_product<C>(F, l, true, ws, Y, Z, upd, m, sc, st);
        else launch_gemm<C, kBwd>(F, l, ws, Y, Z, upd, m, tc5 ? 2 : tc, st);
    }
}

template void multifrontal_solve<float2>(const FrontsDev&, const float2*, float2*, float2*, float2*, int,
                                         const SweepCfg&, cudaStream_t);
template void multifrontal_solve<double2>(const FrontsDev&, const double2*, double2*, double2*, double2*, int,
                                          const SweepCfg&, cudaStream_t);

int sweep_tile_rows(bool large) { return large ? 64 : 32; }

}  // namespace mwi

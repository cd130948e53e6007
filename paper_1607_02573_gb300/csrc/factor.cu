// Batched multifrontal LDL^T factorisation of every subdomain operator B_i
// (the local solves of Eq. ORAS; the paper uses PARDISO/MUMPS per MPI rank,
// here all subdomains are one batch on one GPU).
//
// B_i is complex symmetric (the form of Eq. pbdirectvarf is bilinear), so
// B_i = L D L^T without conjugation.  Pivoting is static: Im(B_i) is positive
// definite for a lossy medium (Im eps < 0), which makes every leading minor
// non-zero; a pivot that is zero or not finite is replaced and counted.
//
// The fronts of one assembly-tree depth are processed together, deepest
// depth first: assemble (entries of B_i, then extend-add of the children's
// Schur complements), then a blocked right-looking partial factorisation of
// the p pivot columns (panel kernel + trailing-update kernel) that leaves the
// Schur complement for the parent.
// A front (dense, f = p + u, lower triangle used) is stored in two pieces:
// its p pivot columns as a column-major f x p panel in the factor store (L
// with unit diagonal implied, D on the diagonal), and its u x u Schur block in
// a transient buffer shared by the fronts of one level (two buffers, even and
// odd levels, since a level's blocks are consumed by the next level).  Once a
// level is factorised, each panel [L11; L21] is replaced by the first p
// columns of the inverse of [L11 0; L21 I], i.e. [L11^{-1}; -L21 L11^{-1}]
// (partitioned inverse) with a unit diagonal, and D^{-1} is stored after the
// panels (indexed by local row), so that each front's part of the ORAS sweeps
// is one dependency-free dense product per direction (sweep.cu).
#include <algorithm>

#include "common.h"
#include "kernels.h"

namespace mwi {

template <typename C> __device__ __forceinline__ C from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

template <typename C>
__global__ void front_assemble_kernel(const int32_t* __restrict__ level_fronts, int lo,
                                      const int64_t* __restrict__ amap_front_ptr,
                                      const int64_t* __restrict__ amap_slot, const int64_t* __restrict__ amap_pos,
                                      const double2* __restrict__ B, C* __restrict__ ws) {
    const int s = level_fronts[lo + blockIdx.x];
    for (int64_t q = amap_front_ptr[s] + threadIdx.x; q < amap_front_ptr[s + 1]; q += blockDim.x)
        ws[amap_pos[q]] = from_d2<C>(B[amap_slot[q]]);
}

// One block per (front, child, four child rows) tile: parent[urel[a], urel[b]]
// += S_c[a, b], a >= b, where S_c is the child's Schur block and the parent
// entry lies in its panel (pivot column) or in its own Schur block.  The first
// and second children of the fronts go in separate launches (they add into the
// same parent entries; the order is fixed, so no atomics are needed).
template <typename C>
__global__ void extend_add_kernel(const int4* __restrict__ tiles, const int32_t* __restrict__ P,
                                  const int32_t* __restrict__ U, const int64_t* __restrict__ f_off,
                                  const int64_t* __restrict__ sch_off, const int64_t* __restrict__ u_off,
                                  const int32_t* __restrict__ urel, C* __restrict__ ws, const C* __restrict__ sch_child,
                                  C* __restrict__ sch_par) {
    const int4 tl = tiles[blockIdx.x];  // (front, child, first child row)
    const int s = tl.x, c = tl.y;
    const int uc = U[c];
    const int b = tl.z + threadIdx.y;
    if (b >= uc) return;
    const int ps = P[s], us = U[s];
    const int64_t fs = (int64_t)ps + us;
    const int32_t* rel = urel + u_off[c];
    const C* src = sch_child + sch_off[c] + (int64_t)b * uc;
    const int rb = rel[b];
    C* dst = rb < ps ? ws + f_off[s] + (int64_t)rb * fs : sch_par + sch_off[s] + (int64_t)(rb - ps) * us - ps;
    for (int a = b + threadIdx.x; a < uc; a += blockDim.x) {
        const C v = src[a];
        C& d = dst[rel[a]];
        d.x += v.x;
        d.y += v.y;
    }
}

template <typename C>
__device__ __forceinline__ bool bad_pivot(C d) {
    typename real_of<C>::type a = d.x * d.x + d.y * d.y;
    return !(a > (typename real_of<C>::type)0) || !isfinite(a);
}

// Panel step k, part 1: the nb x nb diagonal block of every front of the
// level, one warp per front (lane r owns row r): LDL^T in shared memory, then
// M = L^{-T} D^{-1} (upper triangular) by back substitution, lane j taking
// column j.  The factorised block goes back to the panel (L below the
// diagonal, D on it) and M's strictly upper part into the block's upper
// triangle, which the factorisation does not use otherwise (it is cleared when
// the panel is replaced by its partitioned inverse).
template <typename C, int NB>
__global__ void __launch_bounds__(128) panel_diag_kernel(const int32_t* __restrict__ level_fronts, int lo, int nf,
                                                         int k, const int32_t* __restrict__ P,
                                                         const int32_t* __restrict__ U,
                                                         const int64_t* __restrict__ f_off, C* __restrict__ ws,
                                                         int* __restrict__ perturbed) {
    __shared__ C Dgs[4][NB][NB + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * 4 + warp;
    if (q >= nf) return;
    const int s = level_fronts[lo + q];
    const int p = P[s];
    if (k >= p) return;
    const int64_t f = (int64_t)p + U[s];
    const int nb = min(NB, p - k);
    C* F = ws + f_off[s];
    C (*Dg)[NB + 1] = Dgs[warp];
    {
        // every load of the lane in flight before the stores
        C v[NB * NB / 32];
#pragma unroll
        for (int t = 0; t < NB * NB / 32; ++t) {
            const int e = lane + 32 * t, r = e % NB, c = e / NB;
            v[t] = (r < nb && c < nb && r >= c) ? F[(int64_t)(k + c) * f + k + r] : czero<C>();
        }
#pragma unroll
        for (int t = 0; t < NB * NB / 32; ++t) {
            const int e = lane + 32 * t;
            Dg[e % NB][e / NB] = v[t];
        }
    }
    __syncwarp();
    const int r = lane;
    for (int j = 0; j < nb; ++j) {
        C d = Dg[j][j];
        if (bad_pivot(d)) {  // the same value in every lane
            __syncwarp();
            if (r == 0) {
                Dg[j][j] = cmake<C>(1, 0);
                atomicAdd(perturbed, 1);
            }
            d = cmake<C>(1, 0);
        }
        const bool below = r > j && r < nb;
        C ld = czero<C>();
        if (below) {
            const C l = cmul(Dg[r][j], crecip(d));  // l_rj = a_rj / d_j
            Dg[r][j] = l;
            ld = cmul(l, d);
        }
        __syncwarp();
        if (below)
            for (int c = j + 1; c <= r; ++c) Dg[r][c] = csub(Dg[r][c], cmul(ld, Dg[c][j]));
        __syncwarp();
    }
    // column j of M (lane j): y_j = 1, y_r = -sum_{c=r+1..j} L(c, r) y_c for r < j,
    // kept unscaled in the upper triangle, then scaled by 1 / d_j
    if (r < nb) {
        const int j = r;
        for (int i = j - 1; i >= 0; --i) {
            C y = cmake<C>(-Dg[j][i].x, -Dg[j][i].y);
            for (int c = i + 1; c < j; ++c) y = cfms(Dg[c][i], Dg[c][j], y);
            Dg[i][j] = y;
        }
    }
    __syncwarp();
    for (int e = lane; e < nb * nb; e += 32) {
        const int rr = e % nb, c = e / nb;
        C v = Dg[rr][c];
        if (rr < c) v = cmul(v, crecip(Dg[c][c]));
        F[(int64_t)(k + c) * f + k + rr] = v;
    }
}

// Panel step k, part 2: the rows below the diagonal block, L_i = a_i M, one
// thread per row over a tile list (front, first row) of 128-row tiles; M is
// rebuilt from the block (its strictly upper part, and 1 / D on the diagonal)
template <typename C, int NB>
__global__ void __launch_bounds__(128) panel_rows_kernel(const int2* __restrict__ tiles, int k,
                                                         const int32_t* __restrict__ P, const int32_t* __restrict__ U,
                                                         const int64_t* __restrict__ f_off, C* __restrict__ ws) {
    __shared__ C M[NB][NB + 1];
    const int2 tl = tiles[blockIdx.x];
    const int s = tl.x;
    const int p = P[s];
    const int64_t f = (int64_t)p + U[s];
    const int nb = min(NB, p - k);
    C* F = ws + f_off[s];
    {
        // the block's loads in flight before the stores (128 threads)
        C v[NB * NB / 128];
#pragma unroll
        for (int t = 0; t < NB * NB / 128; ++t) {
            const int e = threadIdx.x + 128 * t, r = e % NB, c = e / NB;
            v[t] = (r < nb && c < nb && r <= c) ? F[(int64_t)(k + c) * f + k + r] : czero<C>();
        }
#pragma unroll
        for (int t = 0; t < NB * NB / 128; ++t) {
            const int e = threadIdx.x + 128 * t, r = e % NB, c = e / NB;
            M[r][c] = r == c && r < nb ? crecip(v[t]) : v[t];
        }
    }
    __syncthreads();
    const int64_t i = (int64_t)tl.y + threadIdx.x;
    if (i >= f) return;
    // the row's output accumulates in registers while its entries stream in,
    // eight independent loads at a time
    C acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = czero<C>();
    for (int c0 = 0; c0 < nb; c0 += 8) {
        C a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = c0 + q < nb ? F[(int64_t)(k + c0 + q) * f + i] : czero<C>();
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int j = 0; j < NB; ++j) acc[j] = cfma(a[q], M[min(c0 + q, NB - 1)][j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < nb) F[(int64_t)(k + j) * f + i] = acc[j];
}

// Trailing update of the lower triangle: F[i][c] -= sum_j L[i][j] d_j L[c][j],
// rows/cols in [k + nb, f).  TILE x TILE output tile per block, 256 threads.
// One block per tile (front, bi, bj >= ... bi) of the level's tile list for step k.
template <typename C, int TILE, int NB>
__global__ void __launch_bounds__(256, 4) update_kernel(const int4* __restrict__ tiles, int k,
                                                     const int32_t* __restrict__ P, const int32_t* __restrict__ U,
                                                     const int64_t* __restrict__ f_off,
                                                     const int64_t* __restrict__ sch_off, C* __restrict__ ws,
                                                     C* __restrict__ sch) {
    const int4 tl = tiles[blockIdx.x];
    const int s = tl.x, bi = tl.y, bj = tl.z;
    const int p = P[s];
    if (k >= p) return;
    const int64_t f = (int64_t)p + U[s];
    const int nb = min(NB, p - k);
    const int64_t r0 = k + nb;
    const int64_t nrem = f - r0;
    if ((int64_t)bi * TILE >= nrem) return;
    C* F = ws + f_off[s];
    constexpr int MT = TILE / 16;
    // complex FP32: a thread's rows (and columns) are the pairs 2t, 2t + 1 and
    // 32 + 2t, 32 + 2t + 1, read as 16-byte shared loads (rows padded to an even
    // length so that every pair is 16-byte aligned)
    constexpr bool kPairs = sizeof(C) == sizeof(float2) && MT == 4;
    constexpr int LD = kPairs ? TILE + 2 : TILE + 1;
    __shared__ __align__(16) C As[NB][LD];
    __shared__ __align__(16) C Bs[NB][LD];
    const int tid = threadIdx.x;
    const int64_t rowA = r0 + (int64_t)bi * TILE, rowB = r0 + (int64_t)bj * TILE;
    {
        // every load of the thread in flight before the products and stores
        constexpr int NT = NB * TILE / 256;
        C av[NT], bv[NT], dv[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int e = tid + 256 * t, ii = e % TILE, j = e / TILE;
            av[t] = bv[t] = dv[t] = czero<C>();
            if (j < nb) {
                dv[t] = F[(int64_t)(k + j) * f + k + j];
                if (rowA + ii < f) av[t] = F[(int64_t)(k + j) * f + rowA + ii];
                if (rowB + ii < f) bv[t] = F[(int64_t)(k + j) * f + rowB + ii];
            }
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int e = tid + 256 * t, ii = e % TILE, j = e / TILE;
            As[j][ii] = cmul(av[t], dv[t]);
            Bs[j][ii] = bv[t];
        }
    }
    __syncthreads();
    const int tx = tid % 16, ty = tid / 16;
    // local row of accumulator a (column of b) within the tile
    auto off = [](int t, int a) { return kPairs ? 32 * (a >> 1) + 2 * t + (a & 1) : t + 16 * a; };
    C acc[MT][MT];
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
        for (int b = 0; b < MT; ++b) acc[a][b] = czero<C>();
#pragma unroll 4
    for (int j = 0; j < NB; ++j) {
        C av[MT], bv[MT];
        if constexpr (kPairs) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 pa = *reinterpret_cast<const float4*>(&As[j][32 * h + 2 * tx]);
                const float4 pb = *reinterpret_cast<const float4*>(&Bs[j][32 * h + 2 * ty]);
                av[2 * h] = cmake<C>(pa.x, pa.y);
                av[2 * h + 1] = cmake<C>(pa.z, pa.w);
                bv[2 * h] = cmake<C>(pb.x, pb.y);
                bv[2 * h + 1] = cmake<C>(pb.z, pb.w);
            }
        } else {
#pragma unroll
            for (int a = 0; a < MT; ++a) av[a] = As[j][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < MT; ++b) bv[b] = Bs[j][ty + 16 * b];
        }
#pragma unroll
        for (int a = 0; a < MT; ++a)
#pragma unroll
            for (int b = 0; b < MT; ++b) acc[a][b] = cfma(av[a], bv[b], acc[a][b]);
    }
    const int u = U[s];
    C* S = sch + sch_off[s];
#pragma unroll
    for (int b = 0; b < MT; ++b) {
        const int64_t col = rowB + off(ty, b);
        if (col >= f) continue;
        // pivot columns live in the panel (ld f), the others in the Schur block (ld u)
        C* colp = col < p ? F + col * f : S + (col - p) * u - p;
#pragma unroll
        for (int a = 0; a < MT; ++a) {
            const int64_t row = rowA + off(tx, a);
            if (row < f && row >= col) {
                C& dst = colp[row];
                dst = csub(dst, acc[a][b]);
            }
        }
    }
}

// Partitioned inverse of every front of a level, used by the sweeps.  The
// panel [L11; L21] is the first p columns of the unit lower triangular
// [L11 0; L21 I], whose inverse has first p columns [L11^{-1}; -L21 L11^{-1}].
// Block (front, RC columns c0..) computes those columns for rows >= c0 by
// column-blocked forward substitution (warp-synchronous 32 x 32 triangles on
// the pivot rows, row updates below them, the update rows included), writing
// the strictly lower part to tmp (per front f x p, ld f).
template <typename C, int RC>
__global__ void __launch_bounds__(256) invert_panel_kernel(const int32_t* __restrict__ level_fronts, int lo,
                                                           const int32_t* __restrict__ P,
                                                           const int32_t* __restrict__ U,
                                                           const int64_t* __restrict__ f_off,
                                                           const int64_t* __restrict__ inv_off,
                                                           const C* __restrict__ ws, C* __restrict__ tmp) {
    constexpr int RP = RC + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* w = reinterpret_cast<C*>(smem_raw);
    __shared__ C Ld[32][33];
    const int s = level_fronts[lo + blockIdx.y];
    const int p = P[s];
    const int c0 = blockIdx.x * RC;
    if (c0 >= p) return;
    const int64_t f = (int64_t)p + U[s];
    const C* L = ws + f_off[s];
    C* T = tmp + inv_off[lo + blockIdx.y];
    const int nr = (int)f - c0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < nr * RC; e += 256) {
        const int i = e / RC, r = e - i * RC;
        w[i * RP + r] = (i == r) ? cmake<C>(1, 0) : czero<C>();
    }
    for (int jb = c0; jb < p; jb += 32) {
        const int nb = min(32, p - jb);
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += 256) {
            const int i = e & 31, j = e >> 5;
            Ld[i][j] = (i < nb && j < i) ? L[(int64_t)(jb + j) * f + jb + i] : czero<C>();
        }
        __syncthreads();
        for (int r = warp; r < RC; r += 8) {
            C val = lane < nb ? w[(jb - c0 + lane) * RP + r] : czero<C>();
            for (int j = 0; j < nb; ++j) {
                C x;
                x.x = __shfl_sync(0xffffffffu, val.x, j);
                x.y = __shfl_sync(0xffffffffu, val.y, j);
                val = cfms(Ld[lane][j], x, val);
            }
            if (lane < nb) w[(jb - c0 + lane) * RP + r] = val;
        }
        __syncthreads();
        for (int i = jb + nb + tid; i < (int)f; i += 256) {
            C acc[RC];
#pragma unroll
            for (int r = 0; r < RC; ++r) acc[r] = w[(i - c0) * RP + r];
            // eight panel entries of the row in flight at a time
            for (int j0 = 0; j0 < nb; j0 += 8) {
                C l[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) l[q] = j0 + q < nb ? L[(int64_t)(jb + j0 + q) * f + i] : czero<C>();
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const C* wj = w + (jb + min(j0 + q, nb - 1) - c0) * RP;
#pragma unroll
                    for (int r = 0; r < RC; ++r) acc[r] = cfms(l[q], wj[r], acc[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < RC; ++r) w[(i - c0) * RP + r] = acc[r];
        }
    }
    __syncthreads();
    for (int e = tid; e < nr * RC; e += 256) {
        const int i = e / RC, r = e - i * RC;
        if (c0 + r < p && i > r) T[(int64_t)(c0 + r) * f + c0 + i] = w[i * RP + r];
    }
}

// panel column j <- [L11^{-1}; -L21 L11^{-1}] with a unit diagonal and zeros
// above it (so that the panel is the sweeps' operand as stored), and
// 1 / D_jj into dinv at the pivot's local row
template <typename C>
__global__ void copy_inverse_kernel(const int32_t* __restrict__ level_fronts, int lo, const int32_t* __restrict__ P,
                                    const int32_t* __restrict__ U, const int32_t* __restrict__ start,
                                    const int32_t* __restrict__ sub, const int64_t* __restrict__ sub_off,
                                    const int64_t* __restrict__ f_off, const int64_t* __restrict__ inv_off,
                                    const C* __restrict__ tmp, C* __restrict__ ws, C* __restrict__ dinv) {
    const int s = level_fronts[lo + blockIdx.y];
    const int p = P[s];
    const int j = blockIdx.x;
    if (j >= p) return;
    const int64_t f = (int64_t)p + U[s];
    C* L = ws + f_off[s] + (int64_t)j * f;
    const C* T = tmp + inv_off[lo + blockIdx.y] + (int64_t)j * f;
    const C d = L[j];
    __syncthreads();
    // four loads per thread in flight before their stores
    for (int64_t i0 = 0; i0 < f; i0 += 4 * (int64_t)blockDim.x) {
        C v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t i = i0 + t * (int64_t)blockDim.x + threadIdx.x;
            v[t] = (i < f && i > j) ? T[i] : (i == j ? cmake<C>(1, 0) : czero<C>());
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t i = i0 + t * (int64_t)blockDim.x + threadIdx.x;
            if (i < f) L[i] = v[t];
        }
    }
    if (threadIdx.x == 0) dinv[sub_off[sub[s]] + start[s] + j] = crecip(d);
}

template <typename C> struct FactorCfg;
template <> struct FactorCfg<float2> { static constexpr int NB = 32; static constexpr int TILE = 64; };
template <> struct FactorCfg<double2> { static constexpr int NB = 16; static constexpr int TILE = 32; };

template <typename C, int RC>
static void invert_level_rc(const FrontsDev& F, int l, int lo, int nf, C* ws, C* tmp, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        MWI_CUDA(cudaFuncSetAttribute(invert_panel_kernel<C, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
        attr = true;
    }
    const int pmax = F.level_pmax[l];
    const size_t sm = (size_t)F.level_fmax[l] * (RC + 1) * sizeof(C);
    dim3 grd((pmax + RC - 1) / RC, nf);
    invert_panel_kernel<C, RC><<<grd, 256, sm, st>>>(F.level_fronts.p, lo, F.p.p, F.u.p, F.f_off.p, F.inv_off.p, ws,
                                                     tmp);
    MWI_CHECK_LAUNCH();
    copy_inverse_kernel<C><<<dim3(pmax, nf), 128, 0, st>>>(F.level_fronts.p, lo, F.p.p, F.u.p, F.start.p, F.sub.p,
                                                           F.sub_off.p, F.f_off.p, F.inv_off.p, tmp, ws,
                                                           ws + F.ws_entries);
    MWI_CHECK_LAUNCH();
}

// widest column block whose substitution rows fit in 200 KB of shared memory
template <typename C>
static void invert_level(const FrontsDev& F, int l, int lo, int nf, C* ws, C* tmp, cudaStream_t st) {
    const size_t row = (size_t)F.level_fmax[l] * sizeof(C);
    const size_t lim = 200 * 1024;
    if constexpr (sizeof(C) == sizeof(float2)) {
        if (row * 9 <= lim) {
            invert_level_rc<C, 8>(F, l, lo, nf, ws, tmp, st);
            return;
        }
    }
    if (row * 5 <= lim) invert_level_rc<C, 4>(F, l, lo, nf, ws, tmp, st);
    else if (row * 3 <= lim) invert_level_rc<C, 2>(F, l, lo, nf, ws, tmp, st);
    else if (row * 2 <= lim) invert_level_rc<C, 1>(F, l, lo, nf, ws, tmp, st);
    else throw Error(MWI_EINVAL, "front too large for the shared-memory inversion");
}

template <typename C>
void factorize_fronts(const FrontsDev& F, const UpdateTiles& ut, const double2* Bvals, C* ws, C* const sch[2],
                      C* inv_tmp, int* perturbed, cudaStream_t st) {
    constexpr int NB = FactorCfg<C>::NB, TILE = FactorCfg<C>::TILE;
    MWI_REQUIRE(ut.nb == NB && ut.tile == TILE, MWI_EINVAL, "internal: update tiles built for another blocking");
    MWI_CUDA(cudaMemsetAsync(ws, 0, (size_t)(F.ws_entries + F.nloc) * sizeof(C), st));
    const int nlev = (int)F.level_ptr.size() - 1;
    size_t range = 0, ext = 0;
    for (int l = 0; l < nlev; ++l) {
        const int lo0 = F.level_ptr[l], hi = F.level_ptr[l + 1];
        C* sch_l = sch[l & 1];
        const C* sch_child = sch[(l + 1) & 1];
        if (F.level_sch[l] > 0) MWI_CUDA(cudaMemsetAsync(sch_l, 0, (size_t)F.level_sch[l] * sizeof(C), st));
        for (int lo = lo0; lo < hi; lo += 65535) {
            const int nf = std::min(65535, hi - lo);
            front_assemble_kernel<C><<<nf, 256, 0, st>>>(F.level_fronts.p, lo, F.amap_front_ptr.p, F.amap_slot.p,
                                                         F.amap_pos.p, Bvals, ws);
            MWI_CHECK_LAUNCH();
            for (int ci = 0; ci < 2; ++ci) {
                MWI_REQUIRE(ext + 1 < F.ext_ptr.size(), MWI_EINVAL, "internal: extend-add tile list out of step");
                const int64_t t0 = F.ext_ptr[ext], t1 = F.ext_ptr[ext + 1];
                ++ext;
                if (t1 > t0) {
                    extend_add_kernel<C><<<(unsigned)(t1 - t0), dim3(64, 4), 0, st>>>(
                        F.ext_tiles.p + t0, F.p.p, F.u.p, F.f_off.p, F.sch_off.p, F.u_off.p, F.urel.p, ws, sch_child,
                        sch_l);
                    MWI_CHECK_LAUNCH();
                }
            }
            const int pmax = F.level_pmax[l];
            for (int k = 0; k < pmax; k += NB) {
                panel_diag_kernel<C, NB><<<(nf + 3) / 4, 128, 0, st>>>(F.level_fronts.p, lo, nf, k, F.p.p,
                                                                       F.u.p, F.f_off.p, ws, perturbed);
                MWI_CHECK_LAUNCH();
                {
                    const int64_t r0 = ut.rptr[range], r1 = ut.rptr[range + 1];
                    if (r1 > r0) {
                        panel_rows_kernel<C, NB><<<(unsigned)(r1 - r0), 128, 0, st>>>(ut.rtiles.p + r0, k, F.p.p,
                                                                                     F.u.p, F.f_off.p, ws);
                        MWI_CHECK_LAUNCH();
                    }
                }
                MWI_REQUIRE(range + 1 < ut.ptr.size() && range + 1 < ut.rptr.size(), MWI_EINVAL,
                            "internal: update tile list out of step");
                const int64_t t0 = ut.ptr[range], t1 = ut.ptr[range + 1];
                ++range;
                if (t1 > t0) {
                    update_kernel<C, TILE, NB><<<(unsigned)(t1 - t0), 256, 0, st>>>(
                        ut.tiles.p + t0, k, F.p.p, F.u.p, F.f_off.p, F.sch_off.p, ws, sch_l);
                    MWI_CHECK_LAUNCH();
                }
            }
            invert_level<C>(F, l, lo, nf, ws, inv_tmp, st);
        }
    }
}

template void factorize_fronts<float2>(const FrontsDev&, const UpdateTiles&, const double2*, float2*,
                                       float2* const[2], float2*, int*, cudaStream_t);
template void factorize_fronts<double2>(const FrontsDev&, const UpdateTiles&, const double2*, double2*,
                                        double2* const[2], double2*, int*, cudaStream_t);

int factor_block_cols(bool fp32) { return fp32 ? FactorCfg<float2>::NB : FactorCfg<double2>::NB; }
int factor_tile_rows(bool fp32) { return fp32 ? FactorCfg<float2>::TILE : FactorCfg<double2>::TILE; }

}  // namespace mwi

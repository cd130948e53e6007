// Application of the ORAS preconditioner  y = sum_i R_i^T D_i B_i^{-1} R_i x
// (Eq. ORAS), all subdomains at once:
//   1. gather   Y = R x            (local vectors of all subdomains, ND order)
//   2. forward  L z = Y            front by front, deepest level first; each
//               front assembles its children's update vectors (extend-add) and
//               passes its own update vector to its parent; z_P /= D on exit
//   3. backward L^T Y = z          root level first; each front reads its
//               ancestors' final values through its update-row list
//   4. scatter  y_g = sum_{(i,l) -> g} D_i[l] Y_{i,l}   (fixed order, no atomics)
// Several right-hand sides go through one forward/backward sweep, as the
// paper notes for multiple vectors (Section 3).  Vectors are row-major
// [rows][m]; each block handles one front and a chunk of RC columns.
#include <algorithm>

#include "common.h"
#include "kernels.h"

namespace mwi {

template <typename A, typename B> __device__ __forceinline__ B cvt(A v);
template <> __device__ __forceinline__ double2 cvt<double2, double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<double2, float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 cvt<float2, double2>(float2 v) { return make_double2(v.x, v.y); }

template <typename In, typename C>
__global__ void gather_kernel(int64_t nloc, int m, const int32_t* __restrict__ loc2glob, const In* __restrict__ x,
                              C* __restrict__ Y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nloc * m) return;
    int64_t r = e / m;
    int c = (int)(e - r * m);
    Y[e] = cvt<In, C>(x[(int64_t)loc2glob[r] * m + c]);
}

template <typename C, typename Out>
__global__ void scatter_kernel(int64_t n, int m, const int64_t* __restrict__ own_ptr, const int32_t* __restrict__ own_row,
                               const double* __restrict__ own_w, const C* __restrict__ Y, Out* __restrict__ y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    int64_t g = e / m;
    int c = (int)(e - g * m);
    typedef typename real_of<C>::type R;
    C acc = czero<C>();
    for (int64_t q = own_ptr[g]; q < own_ptr[g + 1]; ++q) {
        C v = Y[(int64_t)own_row[q] * m + c];
        R w = (R)own_w[q];
        acc.x += w * v.x;
        acc.y += w * v.y;
    }
    y[e] = cvt<C, Out>(acc);
}

// Forward sweep of one front for columns [c0, c0 + rc): w holds the front's
// rows (pivots from Y, update rows zero, plus the children's update vectors);
// per block of 32 pivot columns: the unit-lower diagonal triangle is solved by
// one warp per column with shuffles, then every row below the block subtracts
// its block of L times the solved block (one thread per row, all RC columns in
// registers, each L entry read once, coalesced along the column).
template <typename C, int RC>
__global__ void __launch_bounds__(256) forward_kernel(
    const int32_t* __restrict__ level_fronts, int lo, const int32_t* __restrict__ P, const int32_t* __restrict__ U,
    const int32_t* __restrict__ start, const int32_t* __restrict__ sub, const int64_t* __restrict__ sub_off,
    const int64_t* __restrict__ f_off, const int64_t* __restrict__ u_off, const int64_t* __restrict__ upd_row,
    const int32_t* __restrict__ child_ptr, const int32_t* __restrict__ child, const int32_t* __restrict__ urel,
    const C* __restrict__ ws, C* __restrict__ Y, C* __restrict__ upd, int m) {
    constexpr int RP = RC + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* w = reinterpret_cast<C*>(smem_raw);
    __shared__ C Ld[32][33];
    const int s = level_fronts[lo + blockIdx.y];
    const int c0 = blockIdx.x * RC;
    const int rc = min(RC, m - c0);
    const int p = P[s], u = U[s];
    const int f = p + u;
    const int64_t rowbase = sub_off[sub[s]] + start[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < f * RC; e += 256) {
        const int i = e / RC, r = e - i * RC;
        w[i * RP + r] = (i < p && r < rc) ? Y[(rowbase + i) * m + c0 + r] : czero<C>();
    }
    __syncthreads();
    for (int q = child_ptr[s]; q < child_ptr[s + 1]; ++q) {
        const int c = child[q];
        const int uc = U[c];
        const int32_t* rel = urel + u_off[c];
        const C* src = upd + upd_row[c] * m + c0;
        for (int e = tid; e < uc * RC; e += 256) {
            const int k = e / RC, r = e - k * RC;
            if (r < rc) {
                const C v = src[(int64_t)k * m + r];
                C& d = w[rel[k] * RP + r];
                d.x += v.x;
                d.y += v.y;
            }
        }
        __syncthreads();
    }
    const C* L = ws + f_off[s];
    for (int jb = 0; jb < p; jb += 32) {
        const int nb = min(32, p - jb);
        for (int e = tid; e < 32 * 32; e += 256) {
            const int i = e & 31, j = e >> 5;
            Ld[i][j] = (i < nb && j < i) ? L[(int64_t)(jb + j) * f + jb + i] : czero<C>();
        }
        __syncthreads();
        if (warp < RC) {
            C val = lane < nb ? w[(jb + lane) * RP + warp] : czero<C>();
            for (int j = 0; j < nb; ++j) {
                C x;
                x.x = __shfl_sync(0xffffffffu, val.x, j);
                x.y = __shfl_sync(0xffffffffu, val.y, j);
                val = cfms(Ld[lane][j], x, val);
            }
            if (lane < nb) w[(jb + lane) * RP + warp] = val;
        }
        __syncthreads();
        for (int i = jb + nb + tid; i < f; i += 256) {
            C acc[RC];
#pragma unroll
            for (int r = 0; r < RC; ++r) acc[r] = w[i * RP + r];
            const C* Lc = L + (int64_t)jb * f + i;
#pragma unroll 4
            for (int j = 0; j < nb; ++j) {
                const C l = Lc[(int64_t)j * f];
                const C* wj = w + (jb + j) * RP;
#pragma unroll
                for (int r = 0; r < RC; ++r) acc[r] = cfms(l, wj[r], acc[r]);
            }
#pragma unroll
            for (int r = 0; r < RC; ++r) w[i * RP + r] = acc[r];
        }
        __syncthreads();
    }
    for (int e = tid; e < f * RC; e += 256) {
        const int i = e / RC, r = e - i * RC;
        if (r >= rc) continue;
        if (i < p) Y[(rowbase + i) * m + c0 + r] = cmul(w[i * RP + r], crecip(L[(int64_t)i * f + i]));
        else upd[(upd_row[s] + i - p) * m + c0 + r] = w[i * RP + r];
    }
}

// Backward sweep: per block of 32 pivots (last block first), subtract the
// dots of the block's L columns with the already final rows below (warp per
// 4 columns, lanes along the rows, shuffle reduction), then solve the
// transposed unit-lower triangle with one warp per column.
template <typename C, int RC>
__global__ void __launch_bounds__(256) backward_kernel(
    const int32_t* __restrict__ level_fronts, int lo, const int32_t* __restrict__ P, const int32_t* __restrict__ U,
    const int32_t* __restrict__ start, const int32_t* __restrict__ sub, const int64_t* __restrict__ sub_off,
    const int64_t* __restrict__ f_off, const int64_t* __restrict__ u_off, const int32_t* __restrict__ urows,
    const C* __restrict__ ws, C* __restrict__ Y, int m) {
    constexpr int RP = RC + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* w = reinterpret_cast<C*>(smem_raw);
    __shared__ C Ld[32][33];
    const int s = level_fronts[lo + blockIdx.y];
    const int c0 = blockIdx.x * RC;
    const int rc = min(RC, m - c0);
    const int p = P[s], u = U[s];
    const int f = p + u;
    const int64_t sbase = sub_off[sub[s]];
    const int64_t rowbase = sbase + start[s];
    const int32_t* ur = urows + u_off[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < f * RC; e += 256) {
        const int i = e / RC, r = e - i * RC;
        C v = czero<C>();
        if (r < rc) v = i < p ? Y[(rowbase + i) * m + c0 + r] : Y[(sbase + ur[i - p]) * m + c0 + r];
        w[i * RP + r] = v;
    }
    const C* L = ws + f_off[s];
    const int nblk = (p + 31) / 32;
    for (int bk = nblk - 1; bk >= 0; --bk) {
        const int jb = bk * 32, nb = min(32, p - jb), je = jb + nb;
        for (int e = tid; e < 32 * 32; e += 256) {
            const int i = e & 31, j = e >> 5;
            Ld[i][j] = (i < nb && j < i) ? L[(int64_t)(jb + j) * f + jb + i] : czero<C>();
        }
        __syncthreads();
        {
            C acc[4][RC];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int r = 0; r < RC; ++r) acc[q][r] = czero<C>();
            for (int i = je + lane; i < f; i += 32) {
                C x[RC];
#pragma unroll
                for (int r = 0; r < RC; ++r) x[r] = w[i * RP + r];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jj = warp + 8 * q;
                    if (jj < nb) {
                        const C l = L[(int64_t)(jb + jj) * f + i];
#pragma unroll
                        for (int r = 0; r < RC; ++r) acc[q][r] = cfma(l, x[r], acc[q][r]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int r = 0; r < RC; ++r)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        acc[q][r].x += __shfl_xor_sync(0xffffffffu, acc[q][r].x, o);
                        acc[q][r].y += __shfl_xor_sync(0xffffffffu, acc[q][r].y, o);
                    }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int jj = warp + 8 * q;
                if (jj < nb) {
#pragma unroll
                    for (int r = 0; r < RC; ++r)
                        if (lane == r) w[(jb + jj) * RP + r] = csub(w[(jb + jj) * RP + r], acc[q][r]);
                }
            }
        }
        __syncthreads();
        if (warp < RC) {
            C val = lane < nb ? w[(jb + lane) * RP + warp] : czero<C>();
            for (int j = nb - 1; j > 0; --j) {
                C x;
                x.x = __shfl_sync(0xffffffffu, val.x, j);
                x.y = __shfl_sync(0xffffffffu, val.y, j);
                if (lane < j) val = cfms(Ld[j][lane], x, val);
            }
            if (lane < nb) w[(jb + lane) * RP + warp] = val;
        }
        __syncthreads();
    }
    for (int e = tid; e < p * RC; e += 256) {
        const int i = e / RC, r = e - i * RC;
        if (r < rc) Y[(rowbase + i) * m + c0 + r] = w[i * RP + r];
    }
}

template <typename C> struct SweepCfg;
template <> struct SweepCfg<float2> { static constexpr int RCMAX = 8; };
template <> struct SweepCfg<double2> { static constexpr int RCMAX = 4; };

static int choose_rc(int m, int fmax, size_t elt, int rcmax) {
    int rc = rcmax;
    while (rc > 1 && (rc > m || (size_t)fmax * (rc + 1) * elt > 180 * 1024)) rc >>= 1;
    return rc;
}

static const size_t kSweepSmem = 200 * 1024;

template <typename C, int RC>
static void set_attr_rc() {
    static bool done = false;
    if (!done) {
        MWI_CUDA(cudaFuncSetAttribute(forward_kernel<C, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmem));
        MWI_CUDA(cudaFuncSetAttribute(backward_kernel<C, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmem));
        done = true;
    }
}

template <typename C, int RC>
static void sweep_level(const FrontsDev& F, const C* ws, C* Y, C* upd, int m, int l, bool fwd, cudaStream_t st) {
    set_attr_rc<C, RC>();
    const size_t sm = (size_t)F.level_fmax[l] * (RC + 1) * sizeof(C);
    MWI_REQUIRE(sm <= kSweepSmem, MWI_EINVAL, "front too large for the shared-memory solve");
    for (int lo = F.level_ptr[l]; lo < F.level_ptr[l + 1]; lo += 65535) {
        const int nf = std::min(65535, F.level_ptr[l + 1] - lo);
        dim3 grd((m + RC - 1) / RC, nf);
        if (fwd)
            forward_kernel<C, RC><<<grd, 256, sm, st>>>(F.level_fronts.p, lo, F.p.p, F.u.p, F.start.p, F.sub.p,
                                                        F.sub_off.p, F.f_off.p, F.u_off.p, F.upd_row.p,
                                                        F.child_ptr.p, F.child.p, F.urel.p, ws, Y, upd, m);
        else
            backward_kernel<C, RC><<<grd, 256, sm, st>>>(F.level_fronts.p, lo, F.p.p, F.u.p, F.start.p, F.sub.p,
                                                         F.sub_off.p, F.f_off.p, F.u_off.p, F.urows.p, ws, Y, m);
        MWI_CHECK_LAUNCH();
    }
}

template <typename C>
static void sweep(const FrontsDev& F, const C* ws, C* Y, C* upd, int m, int l, bool fwd, cudaStream_t st) {
    const int rc = choose_rc(m, F.level_fmax[l], sizeof(C), SweepCfg<C>::RCMAX);
    switch (rc) {
        case 8: sweep_level<C, 8>(F, ws, Y, upd, m, l, fwd, st); break;
        case 4: sweep_level<C, 4>(F, ws, Y, upd, m, l, fwd, st); break;
        case 2: sweep_level<C, 2>(F, ws, Y, upd, m, l, fwd, st); break;
        default: sweep_level<C, 1>(F, ws, Y, upd, m, l, fwd, st); break;
    }
}

template <typename C, typename In, typename Out>
static void oras_apply_impl(const FrontsDev& F, const C* ws, const In* x, Out* y, int m, C* Y, C* upd,
                            cudaStream_t st) {
    const int th = 256;
    int64_t tot = F.nloc * m;
    gather_kernel<In, C><<<(unsigned)((tot + th - 1) / th), th, 0, st>>>(F.nloc, m, F.loc2glob.p, x, Y);
    MWI_CHECK_LAUNCH();
    const int nlev = (int)F.level_ptr.size() - 1;
    for (int l = 0; l < nlev; ++l) sweep<C>(F, ws, Y, upd, m, l, true, st);
    for (int l = nlev - 1; l >= 0; --l) sweep<C>(F, ws, Y, upd, m, l, false, st);
    // scatter into the global vector (n = own_ptr size - 1)
    const int64_t n = (int64_t)F.own_ptr.n - 1;
    tot = n * m;
    scatter_kernel<C, Out><<<(unsigned)((tot + th - 1) / th), th, 0, st>>>(n, m, F.own_ptr.p, F.own_row.p,
                                                                          F.own_w.p, Y, y);
    MWI_CHECK_LAUNCH();
}

template <typename C>
void oras_apply(const FrontsDev& F, const C* ws, const double2* x, double2* y, int m, C* Y, C* upd,
                cudaStream_t st, const float2* x32, float2* y32) {
    if (x32) oras_apply_impl<C, float2, float2>(F, ws, x32, y32, m, Y, upd, st);
    else oras_apply_impl<C, double2, double2>(F, ws, x, y, m, Y, upd, st);
}

template void oras_apply<float2>(const FrontsDev&, const float2*, const double2*, double2*, int, float2*, float2*,
                                 cudaStream_t, const float2*, float2*);
template void oras_apply<double2>(const FrontsDev&, const double2*, const double2*, double2*, int, double2*,
                                  double2*, cudaStream_t, const float2*, float2*);

}  // namespace mwi

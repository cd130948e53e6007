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

template <typename C>
__global__ void __launch_bounds__(256) forward_kernel(
    const int32_t* __restrict__ level_fronts, int lo, const int32_t* __restrict__ P, const int32_t* __restrict__ U,
    const int32_t* __restrict__ start, const int32_t* __restrict__ sub, const int64_t* __restrict__ sub_off,
    const int64_t* __restrict__ f_off, const int64_t* __restrict__ u_off, const int64_t* __restrict__ upd_row,
    const int32_t* __restrict__ child_ptr, const int32_t* __restrict__ child, const int32_t* __restrict__ urel,
    const C* __restrict__ ws, C* __restrict__ Y, C* __restrict__ upd, int m, int RC) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* w = reinterpret_cast<C*>(smem_raw);
    const int s = level_fronts[lo + blockIdx.y];
    const int c0 = blockIdx.x * RC;
    const int rc = min(RC, m - c0);
    const int p = P[s], u = U[s];
    const int f = p + u;
    const int64_t rowbase = sub_off[sub[s]] + start[s];
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int e = tid; e < f * RC; e += nth) {
        int i = e / RC, r = e - i * RC;
        w[e] = (i < p && r < rc) ? Y[(rowbase + i) * m + c0 + r] : czero<C>();
    }
    __syncthreads();
    for (int q = child_ptr[s]; q < child_ptr[s + 1]; ++q) {
        const int c = child[q];
        const int uc = U[c];
        const int32_t* rel = urel + u_off[c];
        const C* src = upd + upd_row[c] * m + c0;
        for (int e = tid; e < uc * RC; e += nth) {
            int k = e / RC, r = e - k * RC;
            if (r < rc) {
                C v = src[(int64_t)k * m + r];
                C& d = w[rel[k] * RC + r];
                d.x += v.x;
                d.y += v.y;
            }
        }
        __syncthreads();
    }
    const C* L = ws + f_off[s];
    for (int jb = 0; jb < p; jb += 32) {
        const int je = min(jb + 32, p);
        for (int j = jb; j < je - 1; ++j) {
            const int nr = je - j - 1;
            for (int e = tid; e < nr * RC; e += nth) {
                int i = j + 1 + e / RC, r = e % RC;
                w[i * RC + r] = cfms(L[(int64_t)j * f + i], w[j * RC + r], w[i * RC + r]);
            }
            __syncthreads();
        }
        const int nr = f - je;
        for (int e = tid; e < nr * RC; e += nth) {
            int i = je + e / RC, r = e % RC;
            C acc = w[i * RC + r];
            for (int j = jb; j < je; ++j) acc = cfms(L[(int64_t)j * f + i], w[j * RC + r], acc);
            w[i * RC + r] = acc;
        }
        __syncthreads();
    }
    for (int e = tid; e < f * RC; e += nth) {
        int i = e / RC, r = e - i * RC;
        if (r >= rc) continue;
        if (i < p) Y[(rowbase + i) * m + c0 + r] = cmul(w[e], crecip(L[(int64_t)i * f + i]));
        else upd[(upd_row[s] + i - p) * m + c0 + r] = w[e];
    }
}

template <typename C>
__global__ void __launch_bounds__(256) backward_kernel(
    const int32_t* __restrict__ level_fronts, int lo, const int32_t* __restrict__ P, const int32_t* __restrict__ U,
    const int32_t* __restrict__ start, const int32_t* __restrict__ sub, const int64_t* __restrict__ sub_off,
    const int64_t* __restrict__ f_off, const int64_t* __restrict__ u_off, const int32_t* __restrict__ urows,
    const C* __restrict__ ws, C* __restrict__ Y, int m, int RC) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* w = reinterpret_cast<C*>(smem_raw);
    const int s = level_fronts[lo + blockIdx.y];
    const int c0 = blockIdx.x * RC;
    const int rc = min(RC, m - c0);
    const int p = P[s], u = U[s];
    const int f = p + u;
    const int64_t sbase = sub_off[sub[s]];
    const int64_t rowbase = sbase + start[s];
    const int32_t* ur = urows + u_off[s];
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int e = tid; e < f * RC; e += nth) {
        int i = e / RC, r = e - i * RC;
        C v = czero<C>();
        if (r < rc) v = i < p ? Y[(rowbase + i) * m + c0 + r] : Y[(sbase + ur[i - p]) * m + c0 + r];
        w[e] = v;
    }
    __syncthreads();
    const C* L = ws + f_off[s];
    const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const int nblk = (p + 31) / 32;
    for (int bk = nblk - 1; bk >= 0; --bk) {
        const int jb = bk * 32, je = min(jb + 32, p);
        // w[j] -= sum_{i >= je} L[i][j] w[i]   (warp per j, lanes over i)
        for (int j = jb + warp; j < je; j += nwarp) {
            C acc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r] = czero<C>();
            const C* Lc = L + (int64_t)j * f;
            for (int i = je + lane; i < f; i += 32) {
                C l = Lc[i];
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    if (r < RC) acc[r] = cfma(l, w[i * RC + r], acc[r]);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                if (r >= RC) break;
                C a = acc[r];
                for (int o = 16; o > 0; o >>= 1) {
                    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
                    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
                }
                if (lane == 0) w[j * RC + r] = csub(w[j * RC + r], a);
            }
        }
        __syncthreads();
        for (int j = je - 1; j > jb; --j) {
            const int nr = j - jb;
            for (int e = tid; e < nr * RC; e += nth) {
                int i = jb + e / RC, r = e % RC;
                w[i * RC + r] = cfms(L[(int64_t)i * f + j], w[j * RC + r], w[i * RC + r]);
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < p * RC; e += nth) {
        int i = e / RC, r = e - i * RC;
        if (r < rc) Y[(rowbase + i) * m + c0 + r] = w[e];
    }
}

static int choose_rc(int m, int fmax, size_t elt) {
    int rc = 8;
    while (rc > 1 && (rc > m || (size_t)fmax * rc * elt > 160 * 1024)) rc >>= 1;
    return rc;
}

template <typename C>
static void set_smem_attr() {
    static bool done = false;
    if (!done) {
        MWI_CUDA(cudaFuncSetAttribute(forward_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        MWI_CUDA(cudaFuncSetAttribute(backward_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        done = true;
    }
}

template <typename C, typename In, typename Out>
static void oras_apply_impl(const FrontsDev& F, const C* ws, const In* x, Out* y, int m, C* Y, C* upd,
                            cudaStream_t st) {
    set_smem_attr<C>();
    const int th = 256;
    int64_t tot = F.nloc * m;
    gather_kernel<In, C><<<(unsigned)((tot + th - 1) / th), th, 0, st>>>(F.nloc, m, F.loc2glob.p, x, Y);
    MWI_CHECK_LAUNCH();
    const int nlev = (int)F.level_ptr.size() - 1;
    for (int l = 0; l < nlev; ++l) {
        const int rc = choose_rc(m, F.level_fmax[l], sizeof(C));
        MWI_REQUIRE((size_t)F.level_fmax[l] * rc * sizeof(C) <= 200 * 1024, MWI_EINVAL,
                    "front too large for the shared-memory solve");
        const size_t sm = (size_t)F.level_fmax[l] * rc * sizeof(C);
        for (int lo = F.level_ptr[l]; lo < F.level_ptr[l + 1]; lo += 65535) {
            const int nf = std::min(65535, F.level_ptr[l + 1] - lo);
            dim3 grd((m + rc - 1) / rc, nf);
            forward_kernel<C><<<grd, th, sm, st>>>(F.level_fronts.p, lo, F.p.p, F.u.p, F.start.p, F.sub.p,
                                                   F.sub_off.p, F.f_off.p, F.u_off.p, F.upd_row.p, F.child_ptr.p,
                                                   F.child.p, F.urel.p, ws, Y, upd, m, rc);
            MWI_CHECK_LAUNCH();
        }
    }
    for (int l = nlev - 1; l >= 0; --l) {
        const int rc = choose_rc(m, F.level_fmax[l], sizeof(C));
        const size_t sm = (size_t)F.level_fmax[l] * rc * sizeof(C);
        for (int lo = F.level_ptr[l]; lo < F.level_ptr[l + 1]; lo += 65535) {
            const int nf = std::min(65535, F.level_ptr[l + 1] - lo);
            dim3 grd((m + rc - 1) / rc, nf);
            backward_kernel<C><<<grd, th, sm, st>>>(F.level_fronts.p, lo, F.p.p, F.u.p, F.start.p, F.sub.p,
                                                    F.sub_off.p, F.f_off.p, F.u_off.p, F.urows.p, ws, Y, m, rc);
            MWI_CHECK_LAUNCH();
        }
    }
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

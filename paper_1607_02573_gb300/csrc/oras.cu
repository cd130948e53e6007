// Application of the ORAS preconditioner  y = sum_i R_i^T D_i B_i^{-1} R_i x
// (Eq. ORAS), all subdomains at once:
//   1. gather   Y = R x            (local vectors of all subdomains, ND order)
//   2. forward  L z = Y            front by front, deepest level first; each
//               front assembles its children's update vectors (extend-add) and
//               passes its own update vector to its parent
//   3. backward D L^T Y = z        root level first; each front reads its
//               ancestors' final values through its update-row list
//   (both sweeps are batched dense products, see sweep.cu)
//   4. scatter  y_g = sum_{(i,l) -> g} D_i[l] Y_{i,l}   (fixed order, no atomics)
// Several right-hand sides go through one forward/backward sweep, as the
// paper notes for multiple vectors (Section 3).  Vectors are row-major [rows][m].
#include <algorithm>

#include "common.h"
#include "gmres.h"
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

template <typename C, typename In, typename Out>
static void oras_apply_impl(const FrontsDev& F, const C* ws, const In* x, Out* y, int m, C* Y, C* Z, C* upd,
                            cudaStream_t st) {
    const int th = 256;
    int64_t tot = F.nloc * m;
    gather_kernel<In, C><<<(unsigned)((tot + th - 1) / th), th, 0, st>>>(F.nloc, m, F.loc2glob.p, x, Y);
    MWI_CHECK_LAUNCH();
    multifrontal_solve<C>(F, ws, Y, Z, upd, m, st);
    // scatter into the global vector (n = own_ptr size - 1)
    const int64_t n = (int64_t)F.own_ptr.n - 1;
    tot = n * m;
    scatter_kernel<C, Out><<<(unsigned)((tot + th - 1) / th), th, 0, st>>>(n, m, F.own_ptr.p, F.own_row.p,
                                                                          F.own_w.p, Y, y);
    MWI_CHECK_LAUNCH();
}

template <typename C>
void oras_apply(const FrontsDev& F, const C* ws, const double2* x, double2* y, int m, C* Y, C* Z, C* upd,
                cudaStream_t st, const float2* x32, float2* y32) {
    if (x32) oras_apply_impl<C, float2, float2>(F, ws, x32, y32, m, Y, Z, upd, st);
    else oras_apply_impl<C, double2, double2>(F, ws, x, y, m, Y, Z, upd, st);
}

template void oras_apply<float2>(const FrontsDev&, const float2*, const double2*, double2*, int, float2*, float2*,
                                 float2*, cudaStream_t, const float2*, float2*);
template void oras_apply<double2>(const FrontsDev&, const double2*, const double2*, double2*, int, double2*,
                                  double2*, double2*, cudaStream_t, const float2*, float2*);

}  // namespace mwi

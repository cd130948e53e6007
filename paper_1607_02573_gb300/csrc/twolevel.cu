// Two-level ORAS (Section 7: a coarse space restores the scalability of the
// one-level method in the number of subdomains), device side.  Deflated
// combination of the coarse correction and the one-level preconditioner:
//   Q r = P A_c^{-1} P^T r,      M_2 r = M_ORAS (r - A Q r) + Q r.
// P is real (the midpoint rule of the coarse Whitney fields on the fine
// edges), A and A_c are complex symmetric.  The coarse solve is the
// multifrontal solve of A_c's one dense front (factor.cu / sweep.cu).
#include "common.h"
#include "kernels.h"

namespace mwi {

// y[r][c] = sum_q val[q] x[col[q]][c]   (real CSR times a complex block)
template <typename C>
__global__ void spmm_real_kernel(int64_t rows, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const C* __restrict__ x, C* __restrict__ y, int m) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * m) return;
    const int64_t r = e / m;
    const int c = (int)(e - r * m);
    typedef typename real_of<C>::type R;
    C acc = czero<C>();
    for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
        const R w = (R)val[q];
        const C v = x[(int64_t)col[q] * m + c];
        acc.x += w * v.x;
        acc.y += w * v.y;
    }
    y[e] = acc;
}

// out = a - out
template <typename C>
__global__ void rsub_kernel(int64_t count, const C* __restrict__ a, C* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) out[e] = csub<C>(a[e], out[e]);
}

// y += q
template <typename C>
__global__ void add_kernel(int64_t count, const C* __restrict__ q, C* __restrict__ y) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) y[e] = cadd<C>(y[e], q[e]);
}

static unsigned blocks_of(int64_t count, int th) { return (unsigned)((count + th - 1) / th); }

template <typename C>
static void spmm_real(int64_t rows, const int64_t* rp, const int32_t* col, const double* val, const C* x, C* y, int m,
                      cudaStream_t st) {
    if (rows * m == 0) return;
    spmm_real_kernel<C><<<blocks_of(rows * m, 256), 256, 0, st>>>(rows, rp, col, val, x, y, m);
    MWI_CHECK_LAUNCH();
}

template <typename C>
void two_level_apply(const CoarseDev& cd, const C* x, C* y, int m, const TwoLevelScratch<C>& s,
                     const std::function<void(const C*, C*)>& coarse_solve,
                     const std::function<void(const C*, C*)>& one_level, const int32_t* A_rp, const int32_t* A_col,
                     const C* A_val, cudaStream_t st) {
    const int64_t nm = cd.n * (int64_t)m;
    // Q x = P A_c^{-1} P^T x
    spmm_real<C>(cd.nc, cd.PT_rp.p, cd.PT_col.p, cd.PT_val.p, x, s.ct, m, st);
    coarse_solve(s.ct, s.cq);
    spmm_real<C>(cd.n, cd.P_rp.p, cd.P_col.p, cd.P_val.p, s.cq, s.q, m, st);
    // w = x - A Q x
    spmm<C>(cd.n, A_rp, A_col, A_val, s.q, s.w, m, st);
    if (nm) {
        rsub_kernel<C><<<blocks_of(nm, 256), 256, 0, st>>>(nm, x, s.w);
        MWI_CHECK_LAUNCH();
    }
    // y = M_ORAS w + Q x
    one_level(s.w, y);
    if (nm) {
        add_kernel<C><<<blocks_of(nm, 256), 256, 0, st>>>(nm, s.q, y);
        MWI_CHECK_LAUNCH();
    }
}

template void two_level_apply<float2>(const CoarseDev&, const float2*, float2*, int, const TwoLevelScratch<float2>&,
                                      const std::function<void(const float2*, float2*)>&,
                                      const std::function<void(const float2*, float2*)>&, const int32_t*,
                                      const int32_t*, const float2*, cudaStream_t);
template void two_level_apply<double2>(const CoarseDev&, const double2*, double2*, int,
                                       const TwoLevelScratch<double2>&,
                                       const std::function<void(const double2*, double2*)>&,
                                       const std::function<void(const double2*, double2*)>&, const int32_t*,
                                       const int32_t*, const double2*, cudaStream_t);

}  // namespace mwi

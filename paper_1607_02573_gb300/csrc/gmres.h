// Pseudo-block flexible GMRES engine over row-major [n][m] device vectors.
#pragma once

#include <complex>
#include <functional>
#include <vector>

#include "common.h"

namespace mwi {

static const int kDotBlocks = 608;  // 4 x 152 SMs

// y = op(x) on [n][m] device vectors
template <typename C>
using OpFnT = std::function<void(const C*, C*)>;

template <typename C>
struct Gmres {
    typedef OpFnT<C> OpFn;
    int64_t n = 0;
    int m = 0, restart = 0;
    DevBuf<C> V, Z, W;
    DevBuf<double2> H, cs, sn, g, y, h, hacc, partial;
    DevBuf<double> dvec;
    DevBuf<int> ivec;
    // optional timer: runs fn, attributing its device time to a slot
    std::function<void(int, const std::function<void()>&)> timer;

    void reserve(int64_t n, int m, int restart);
    // One flexible GMRES cycle from residual r0 (initial x in x, updated in
    // place): at most max_steps steps; a column stops when its estimated
    // residual <= tol[c] (device array).  Returns steps taken.
    int cycle(const OpFn& A, const OpFn& M, const C* r0, C* x, const double* tol, int max_steps,
              cudaStream_t st, double* resid_host, int* iters_used);
    // out[i][c] = conj(V_i)^T w (i < nvec), plus conj(w)^T w at i = nvec when self = 1;
    // acc[i] += out[i] for i < nvec
    void dots(const C* V, int nvec, int64_t vstride, const C* w, double2* out, double2* acc, cudaStream_t st,
              int self = 0);
    void column_norms2(const C* x, double* out, cudaStream_t st);
    void column_norms2_into(const C* x, double* out, double2* tmp, cudaStream_t st);
    size_t bytes() const {
        return V.bytes() + Z.bytes() + W.bytes() + H.bytes() + cs.bytes() + sn.bytes() + g.bytes() + y.bytes() +
               h.bytes() + hacc.bytes() + partial.bytes() + dvec.bytes() + ivec.bytes();
    }
};

// FGMRES whose FP64-quality vectors (basis V, w, residual, iterate) are
// double-float planes (hi [n][m] float2 followed by lo [n][m] float2) and
// whose preconditioned directions Z are complex FP32 (the preconditioner's
// own output, so stored exactly).  Arnoldi relation, residual and iterate
// carry about 48 significant bits on the FP32 pipes; the Gram-Schmidt
// coefficients are formed from the FP32 heads, with one reduction and one
// fused update pass per step (classical Gram-Schmidt with delayed
// reorthogonalisation).
struct GmresDF {
    // w = A z (z exact in FP32, w double-float planes)
    typedef std::function<void(const float2*, float2*)> OpA;
    // z = M v (v: FP32 head plane of a basis vector, z complex FP32)
    typedef std::function<void(const float2*, float2*)> OpM;
    int64_t n = 0;
    int m = 0, restart = 0;
    DevBuf<float2> V, Z, W;
    DevBuf<float4> hdf, hdf2, scal, ydf;   // double-float coefficients of the fused updates
    DevBuf<float2> invdf;
    DevBuf<double2> H, Hp, cs, sn, g, y, h, partial;
    DevBuf<double> dvec;
    DevBuf<int> ivec;
    std::function<void(int, const std::function<void()>&)> timer;

    void reserve(int64_t n, int m, int restart);
    // one cycle from the double-float residual r0, x (double-float) updated in place
    int cycle(const OpA& A, const OpM& M, const float2* r0, float2* x, const double* tol, int max_steps,
              cudaStream_t st, int* iters_used);
    // ||x_c||^2 from the FP32 head plane
    void norms2(const float2* xh, double* out, cudaStream_t st);
    size_t bytes() const {
        return V.bytes() + Z.bytes() + W.bytes() + hdf.bytes() + hdf2.bytes() + scal.bytes() + ydf.bytes() +
               invdf.bytes() + H.bytes() + Hp.bytes() + cs.bytes() + sn.bytes() + g.bytes() + y.bytes() + h.bytes() +
               partial.bytes() + dvec.bytes() + ivec.bytes();
    }
};

// True block flexible GMRES over complex FP64 [n][m] blocks: one Krylov space
// shared by the m <= 32 columns (block Arnoldi, block classical Gram-Schmidt
// twice, Cholesky QR twice, Givens QR of the block Hessenberg on the host).
struct BlockGmres {
    int64_t n = 0;
    int m = 0, restart = 0;
    DevBuf<double2> V, Z, W, coef, small, partial;
    std::function<void(int, const std::function<void()>&)> timer;

    void reserve(int64_t n, int m, int restart);
    // One cycle from the residual r0 (x updated in place): at most max_steps
    // block steps, stopping when every column's least-squares residual is
    // <= tol[c] (absolute).  resid_est (host, m) gets the last estimates and
    // deflated the number of columns dropped by the Cholesky QRs.  Returns steps.
    int cycle(const OpFnT<double2>& A, const OpFnT<double2>& M, const double2* r0, double2* x,
              const std::vector<double>& tol, int max_steps, cudaStream_t st, double* resid_est, int* deflated);
    void block_dots(const double2* V, int nq, const double2* W, double2* out, cudaStream_t st);
    void block_update(double2* out, const double2* in, int nq, const double2* Cm, double alpha, double beta,
                      cudaStream_t st);
    int chol_qr(double2* X, std::vector<std::complex<double>>& S, cudaStream_t st);
    size_t bytes() const {
        return V.bytes() + Z.bytes() + W.bytes() + coef.bytes() + small.bytes() + partial.bytes();
    }
};

// w = A z with A as double-float planes (hi nnz entries, then lo), z complex FP32
void spmm_df(int64_t n, const int32_t* row_ptr, const int32_t* col, const float2* A, int64_t nnz, const float2* z,
             float2* w, int m, cudaStream_t st);
// r = b - A x, all double-float
void residual_df(int64_t n, const int32_t* row_ptr, const int32_t* col, const float2* A, int64_t nnz, const float2* b,
                 const float2* x, float2* r, int m, cudaStream_t st);
void split_c128(int64_t count, const double2* a, float2* out, cudaStream_t st);
void join_c128(int64_t count, const float2* in, double2* a, cudaStream_t st);

void convert_c128_to_c64(int64_t nm, const double2* a, float2* b, cudaStream_t st);
void convert_c64_to_c128(int64_t nm, const float2* a, double2* b, cudaStream_t st);
void residual_c128(int64_t nm, const double2* b, double2* r, cudaStream_t st);  // r = b - r
void tolerances(int m, const double* b2, double rtol, double* tol, double* bnorm, cudaStream_t st);
// dst[r][dc0 + c] = src[r][sc0 + c] for c < mc (row-major [n][ms] -> [n][md])
void copy_columns(int64_t n, int ms, int sc0, int mc, const double2* src, int md, int dc0, double2* dst,
                  cudaStream_t st);

}  // namespace mwi

// Pseudo-block flexible GMRES engine over row-major [n][m] device vectors.
#pragma once

#include <functional>

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
    int reorth_passes = 0;
};

void convert_c128_to_c64(int64_t nm, const double2* a, float2* b, cudaStream_t st);
void convert_c64_to_c128(int64_t nm, const float2* a, double2* b, cudaStream_t st);
void residual_c128(int64_t nm, const double2* b, double2* r, cudaStream_t st);  // r = b - r
void tolerances(int m, const double* b2, double rtol, double* tol, double* bnorm, cudaStream_t st);
// dst[r][dc0 + c] = src[r][sc0 + c] for c < mc (row-major [n][ms] -> [n][md])
void copy_columns(int64_t n, int ms, int sc0, int mc, const double2* src, int md, int dc0, double2* dst,
                  cudaStream_t st);

}  // namespace mwi

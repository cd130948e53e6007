// Initial guess from a recycled subspace (the Krylov recycling that Section 7
// cites as a way to speed up the sequence of direct problems of an inversion):
// the k columns of X_rec (solutions of a previous, nearby system, and for an
// adjoint solve also the current forward solutions) span the recycled space,
// and every right-hand side starts from its least-residual element
//   x0_c = X_rec y_c,  y_c = argmin || b_c - C y ||,  C = A X_rec,
// i.e. Y = (C^H C)^{-1} C^H B.  An initial guess needs no more than FP32
// accuracy (the solver that follows corrects it to the requested tolerance),
// so the products run in FP32 with FP64 sums across row chunks, and the k x k
// normal equations are solved by Cholesky on the host.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "common.h"
#include "kernels.h"

namespace mwi {

namespace {

constexpr int kRcRows = 8;
constexpr int kRcMaxK = 64;           // recycled columns
constexpr int kRcMaxM = 32;           // right-hand sides
constexpr int kRcPer = kRcMaxK * kRcMaxK / 256;  // products per thread

// partial[chunk][a][b] = sum over the chunk's rows of conj(P[r][a]) Q[r][b],
// P [n][kp], Q [n][kq] row-major
__global__ void __launch_bounds__(256) rc_dots_kernel(const float2* __restrict__ P, int kp,
                                                       const float2* __restrict__ Q, int kq, int64_t n,
                                                       int64_t rows_per_chunk, double2* __restrict__ partial) {
    __shared__ float2 sp[kRcRows][kRcMaxK];
    __shared__ float2 sq[kRcRows][kRcMaxK];
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r1 = r0 + rows_per_chunk < n ? r0 + rows_per_chunk : n;
    const int kk = kp * kq;
    float2 acc[kRcPer];
#pragma unroll
    for (int s = 0; s < kRcPer; ++s) acc[s] = make_float2(0.f, 0.f);
    for (int64_t rb = r0; rb < r1; rb += kRcRows) {
        const int nr = (int)(r1 - rb < kRcRows ? r1 - rb : kRcRows);
        __syncthreads();
        for (int e = threadIdx.x; e < kRcRows * kRcMaxK; e += blockDim.x) {
            const int rr = e / kRcMaxK, c = e % kRcMaxK;
            sp[rr][c] = rr < nr && c < kp ? P[(rb + rr) * kp + c] : make_float2(0.f, 0.f);
            sq[rr][c] = rr < nr && c < kq ? Q[(rb + rr) * kq + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < kRcPer; ++s) {
            const int e = threadIdx.x + 256 * s;
            if (e >= kk) break;
            const int a = e / kq, b = e % kq;
            float2 t = acc[s];
            for (int rr = 0; rr < nr; ++rr) {
                const float2 x = sp[rr][a], y = sq[rr][b];
                t.x += x.x * y.x + x.y * y.y;
                t.y += x.x * y.y - x.y * y.x;
            }
            acc[s] = t;
        }
    }
#pragma unroll
    for (int s = 0; s < kRcPer; ++s) {
        const int e = threadIdx.x + 256 * s;
        if (e < kk) partial[(int64_t)blockIdx.x * kk + e] = make_double2(acc[s].x, acc[s].y);
    }
}

__global__ void rc_reduce_kernel(const double2* __restrict__ partial, int nchunk, int total,
                                 double2* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunk; ++c) {
        const double2 v = partial[(int64_t)c * total + i];
        s.x += v.x;
        s.y += v.y;
    }
    out[i] = s;
}

// out[r][b] = sum_a in[r][a] Y[a][b]  (in [n][k], Y k x m row-major, FP32)
__global__ void __launch_bounds__(256) rc_combine_kernel(const float2* __restrict__ in, int k,
                                                          const float2* __restrict__ Y, int m, int64_t n,
                                                          float2* __restrict__ out) {
    __shared__ float2 ys[kRcMaxK * kRcMaxM];
    __shared__ float2 sx[kRcRows][kRcMaxK];
    for (int e = threadIdx.x; e < k * m; e += blockDim.x) ys[e] = Y[e];
    const int rr = threadIdx.x / kRcMaxM, b = threadIdx.x % kRcMaxM;
    for (int64_t rb = (int64_t)blockIdx.x * kRcRows; rb < n; rb += (int64_t)gridDim.x * kRcRows) {
        const int64_t r = rb + rr;
        __syncthreads();
        for (int e = threadIdx.x; e < kRcRows * k; e += blockDim.x) {
            const int r2 = e / k, c = e % k;
            if (rb + r2 < n) sx[r2][c] = in[(rb + r2) * k + c];
        }
        __syncthreads();
        if (r < n && b < m) {
            float2 acc = make_float2(0.f, 0.f);
            for (int a = 0; a < k; ++a) {
                const float2 x = sx[rr][a], y = ys[a * m + b];
                acc.x += x.x * y.x - x.y * y.y;
                acc.y += x.x * y.y + x.y * y.x;
            }
            out[r * m + b] = acc;
        }
    }
}

typedef std::complex<double> cd;

}  // namespace

size_t recycle_scratch_entries(int k, int m) {
    return (size_t)kRecycleChunks * std::max(k * k, k * m) + (size_t)k * k + (size_t)k * m;
}

int recycle_initial_guess(int64_t n, int k, int m, const float2* X32, const float2* C32, const float2* B32,
                          float2* x0, double2* scratch, cudaStream_t st) {
    MWI_REQUIRE(k >= 1 && k <= kRcMaxK && m >= 1 && m <= kRcMaxM, MWI_EINVAL,
                "recycling takes 1..64 recycled columns and 1..32 right-hand sides");
    const int kk = k * k, km = k * m;
    int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(kRecycleChunks, (n + 255) / 256));
    const int64_t rows = ((n + nchunk - 1) / nchunk + kRcRows - 1) / kRcRows * kRcRows;
    nchunk = (int)((n + rows - 1) / rows);
    double2* part = scratch;
    double2* G = scratch + (size_t)kRecycleChunks * std::max(kk, km);
    double2* CB = G + kk;
    rc_dots_kernel<<<nchunk, 256, 0, st>>>(C32, k, C32, k, n, rows, part);
    MWI_CHECK_LAUNCH();
    rc_reduce_kernel<<<(kk + 255) / 256, 256, 0, st>>>(part, nchunk, kk, G);
    MWI_CHECK_LAUNCH();
    rc_dots_kernel<<<nchunk, 256, 0, st>>>(C32, k, B32, m, n, rows, part);
    MWI_CHECK_LAUNCH();
    rc_reduce_kernel<<<(km + 255) / 256, 256, 0, st>>>(part, nchunk, km, CB);
    MWI_CHECK_LAUNCH();
    std::vector<double2> gh((size_t)kk + km);
    MWI_CUDA(cudaMemcpyAsync(gh.data(), G, gh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    MWI_CUDA(cudaStreamSynchronize(st));
    // Cholesky C^H C = R^H R; a column whose new direction is below 1 % of its
    // norm (the FP32 Gram matrix cannot resolve it) is left out of the span
    std::vector<cd> R((size_t)kk, cd(0.0));
    std::vector<char> live(k, 0);
    int dropped = 0;
    double gmax = 0.0;
    for (int c = 0; c < k; ++c) gmax = std::max(gmax, gh[(size_t)c * k + c].x);
    for (int c = 0; c < k; ++c) {
        const double gcc = gh[(size_t)c * k + c].x;
        double s = gcc;
        for (int q = 0; q < c; ++q) s -= std::norm(R[(size_t)q * k + c]);
        if (!(gcc > 1e-30 * gmax) || !(s > 1e-4 * gcc)) {
            ++dropped;
            continue;
        }
        live[c] = 1;
        const double d = std::sqrt(s);
        R[(size_t)c * k + c] = d;
        for (int b = c + 1; b < k; ++b) {
            cd t(gh[(size_t)c * k + b].x, gh[(size_t)c * k + b].y);
            for (int q = 0; q < c; ++q) t -= std::conj(R[(size_t)q * k + c]) * R[(size_t)q * k + b];
            R[(size_t)c * k + b] = t / d;
        }
    }
    // Y = R^{-1} R^{-H} C^H B over the live columns (dropped rows of Y stay zero)
    std::vector<float2> yh((size_t)km, make_float2(0.f, 0.f));
    for (int b = 0; b < m; ++b) {
        std::vector<cd> z(k, cd(0.0)), y(k, cd(0.0));
        for (int i = 0; i < k; ++i) {
            if (!live[i]) continue;
            const double2 v = gh[(size_t)kk + (size_t)i * m + b];
            cd t(v.x, v.y);
            for (int q = 0; q < i; ++q) t -= std::conj(R[(size_t)q * k + i]) * z[q];
            z[i] = t / R[(size_t)i * k + i];
        }
        for (int i = k - 1; i >= 0; --i) {
            if (!live[i]) continue;
            cd t = z[i];
            for (int q = i + 1; q < k; ++q) t -= R[(size_t)i * k + q] * y[q];
            y[i] = t / R[(size_t)i * k + i];
        }
        for (int i = 0; i < k; ++i) yh[(size_t)i * m + b] = make_float2((float)y[i].real(), (float)y[i].imag());
    }
    float2* Yd = reinterpret_cast<float2*>(part);  // the partial sums are consumed
    MWI_CUDA(cudaMemcpyAsync(Yd, yh.data(), (size_t)km * sizeof(float2), cudaMemcpyHostToDevice, st));
    const int grid = (int)std::min<int64_t>((n + kRcRows - 1) / kRcRows, 152 * 8);
    rc_combine_kernel<<<grid, 256, 0, st>>>(X32, k, Yd, m, n, x0);
    MWI_CHECK_LAUNCH();
    MWI_CUDA(cudaStreamSynchronize(st));  // yh goes out of scope
    return dropped;
}

}  // namespace mwi

// Pseudo-block flexible GMRES building blocks (Section 6: GMRES right-
// preconditioned by ORAS, stopped on the unpreconditioned relative residual;
// Section 6.3: pseudo-block fusion of the operations of several right-hand
// sides).  Every vector is row-major [n][m] (m right-hand sides contiguous), so
// one launch serves all columns, and columns stay independent: each keeps its
// own Hessenberg matrix, Givens rotations and convergence flag.
//
// Orthogonalisation is classical Gram-Schmidt applied twice (CGS2): dots of
// all basis vectors with w in one pass, then one fused update pass.
#include <algorithm>

#include "common.h"
#include "gmres.h"
#include "kernels.h"

namespace mwi {

// ---------------------------------------------------------------- SpMM
// Y = A X: a group of G lanes (G = min(32, pow2 >= m)) per row, lanes over columns.
template <typename C, int G>
__global__ void __launch_bounds__(256) spmm_kernel(int64_t n, const int32_t* __restrict__ rp,
                                                   const int32_t* __restrict__ col, const C* __restrict__ val,
                                                   const C* __restrict__ X, C* __restrict__ Y, int m) {
    const int lane = threadIdx.x % G;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    if (row >= n) return;
    const int b = rp[row], e = rp[row + 1];
    for (int c0 = 0; c0 < m; c0 += G) {
        const int c = c0 + lane;
        if (c >= m) break;
        C acc = czero<C>();
        for (int q = b; q < e; ++q) acc = cfma(val[q], X[(int64_t)col[q] * m + c], acc);
        Y[row * m + c] = acc;
    }
}

template <typename C>
void spmm(int64_t n, const int32_t* row_ptr, const int32_t* col, const C* val, const C* x, C* y, int m,
          cudaStream_t st) {
    const int th = 256;
    if (m >= 32) {
        int64_t blocks = (n * 32 + th - 1) / th;
        spmm_kernel<C, 32><<<(unsigned)blocks, th, 0, st>>>(n, row_ptr, col, val, x, y, m);
    } else if (m >= 8) {
        int64_t blocks = (n * 8 + th - 1) / th;
        spmm_kernel<C, 8><<<(unsigned)blocks, th, 0, st>>>(n, row_ptr, col, val, x, y, m);
    } else {
        int64_t blocks = (n * 4 + th - 1) / th;
        spmm_kernel<C, 4><<<(unsigned)blocks, th, 0, st>>>(n, row_ptr, col, val, x, y, m);
    }
    MWI_CHECK_LAUNCH();
}
template void spmm<double2>(int64_t, const int32_t*, const int32_t*, const double2*, const double2*, double2*, int,
                            cudaStream_t);
template void spmm<float2>(int64_t, const int32_t*, const int32_t*, const float2*, const float2*, float2*, int,
                           cudaStream_t);

// ---------------------------------------------------------------- dots
// partial[b][i][c] = sum over this block's rows of conj(V_i[r][c]) W[r][c].
// Rows are visited four at a time with independent loads, so that enough
// memory requests are in flight to stream V and W at HBM rate.
// With self = 1 the product conj(W) W is appended as vector index nvec.
template <typename C>
__global__ void __launch_bounds__(256) dots_kernel(int64_t n, int m, int nvec_in, const C* __restrict__ V,
                                                   int64_t vstride, const C* __restrict__ W, int self,
                                                   double2* __restrict__ partial) {
    __shared__ double2 red[8][8][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c = blockIdx.y * 32 + tx;
    const int64_t stride = (int64_t)gridDim.x * 8;
    const int nvec = nvec_in + self;
    for (int i0 = 0; i0 < nvec; i0 += 8) {
        const int nq = min(8, nvec - i0);
        C acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = czero<C>();
        if (c < m) {
            int64_t r = blockIdx.x * 8 + ty;
            for (; r + 3 * stride < n; r += 4 * stride) {
                C w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) w[u] = W[(r + u * stride) * m + c];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < nq) {
                        const C* Vq = (i0 + q < nvec_in ? V + (int64_t)(i0 + q) * vstride : W) + c;
                        C v[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) v[u] = Vq[(r + u * stride) * m];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            acc[q].x += v[u].x * w[u].x + v[u].y * w[u].y;
                            acc[q].y += v[u].x * w[u].y - v[u].y * w[u].x;
                        }
                    }
            }
            for (; r < n; r += stride) {
                const C w = W[r * m + c];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < nq) {
                        const C v = (i0 + q < nvec_in ? V + (int64_t)(i0 + q) * vstride : W)[r * m + c];
                        acc[q].x += v.x * w.x + v.y * w.y;
                        acc[q].y += v.x * w.y - v.y * w.x;
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) red[ty][q][tx] = make_double2((double)acc[q].x, (double)acc[q].y);
        __syncthreads();
        // thread (tx, ty) reduces vector q = ty over the 8 row lanes, in a fixed order
        {
            const int q = ty;
            double sx = 0.0, sy = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                sx += red[k][q][tx].x;
                sy += red[k][q][tx].y;
            }
            if (c < m && i0 + q < nvec) partial[((int64_t)blockIdx.x * nvec + i0 + q) * m + c] = make_double2(sx, sy);
        }
        __syncthreads();
    }
}

// h[i][c] = sum_b partial[b][i][c] for i < nvec; hacc[i][c] += h[i][c] for i < nacc
__global__ void dots_reduce_kernel(int nblk, int nvec, int nacc, int m, const double2* __restrict__ partial,
                                   double2* __restrict__ h, double2* __restrict__ hacc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nvec * m) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nblk; ++b) {
        double2 v = partial[(int64_t)b * nvec * m + e];
        s.x += v.x;
        s.y += v.y;
    }
    h[e] = s;
    if (hacc && e < nacc * m) { hacc[e].x += s.x; hacc[e].y += s.y; }
}

// any column whose norm fell below half of its value before the projection
__global__ void reorth_test_kernel(int m, const double2* __restrict__ w0sq, const double* __restrict__ w1sq,
                                   int* __restrict__ flag) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    if (w1sq[c] < 0.5 * w0sq[c].x) atomicOr(flag, 1);
}

// W[r][c] -= sum_i V_i[r][c] h[i][c]
template <typename C>
__global__ void cgs_update_kernel(int64_t n, int m, int nvec, const C* __restrict__ V, int64_t vstride,
                                  const double2* __restrict__ h, C* __restrict__ W) {
    typedef typename real_of<C>::type R;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const int c = (int)(e % m);
    C w = W[e];
    for (int i = 0; i < nvec; ++i) {
        const double2 hh = h[i * m + c];
        C hc;
        hc.x = (R)hh.x;
        hc.y = (R)hh.y;
        w = cfms(V[(int64_t)i * vstride + e], hc, w);
    }
    W[e] = w;
}

// V[r][c] = W[r][c] * s[c]
template <typename C>
__global__ void scale_kernel(int64_t n, int m, const C* __restrict__ W, const double* __restrict__ s,
                             C* __restrict__ V) {
    typedef typename real_of<C>::type R;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const R f = (R)s[e % m];
    C w = W[e];
    w.x *= f;
    w.y *= f;
    V[e] = w;
}

// X[r][c] += sum_i Z_i[r][c] y[i][c]
template <typename C>
__global__ void lincomb_kernel(int64_t n, int m, int nvec, const C* __restrict__ Z, int64_t zstride,
                               const double2* __restrict__ y, C* __restrict__ X) {
    typedef typename real_of<C>::type R;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const int c = (int)(e % m);
    C x = X[e];
    for (int i = 0; i < nvec; ++i) {
        const double2 yy = y[i * m + c];
        C yc;
        yc.x = (R)yy.x;
        yc.y = (R)yy.y;
        x = cfma(Z[(int64_t)i * zstride + e], yc, x);
    }
    X[e] = x;
}

// R = B - R  (R holds A X on entry)
template <typename C>
__global__ void sub_from_kernel(int64_t nm, const C* __restrict__ B, C* __restrict__ R) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    R[e] = csub(B[e], R[e]);
}

template <typename A, typename B>
__global__ void convert_kernel(int64_t nm, const A* __restrict__ a, B* __restrict__ b) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    b[e].x = a[e].x;
    b[e].y = a[e].y;
}

// Per column c: store the Hessenberg column k (h[0..k], hnorm), apply the
// previous rotations, form the new one, update g, decide convergence.
__global__ void arnoldi_kernel(int m, int k, int restart, const double2* __restrict__ h,
                               const double* __restrict__ hnorm2, double2* __restrict__ H,
                               double2* __restrict__ cs, double2* __restrict__ sn, double2* __restrict__ g,
                               int* __restrict__ active, int* __restrict__ kcol, const double* __restrict__ tol,
                               double* __restrict__ resid, double* __restrict__ inv_norm, int* __restrict__ n_active) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    if (!active[c]) { inv_norm[c] = 0.0; return; }
    double2* Hk = H + (int64_t)k * (restart + 1) * m;
    for (int i = 0; i <= k; ++i) Hk[i * m + c] = h[i * m + c];
    const double hn = sqrt(fmax(hnorm2[c], 0.0));
    Hk[(k + 1) * m + c] = make_double2(hn, 0.0);
    for (int i = 0; i < k; ++i) {
        double2 ci = cs[i * m + c], si = sn[i * m + c];
        double2 a = Hk[i * m + c], b = Hk[(i + 1) * m + c];
        Hk[i * m + c] = cadd(cmul(ci, a), cmul(si, b));
        Hk[(i + 1) * m + c] = csub(cmul(cconj(ci), b), cmul(cconj(si), a));
    }
    double2 a = Hk[k * m + c], b = Hk[(k + 1) * m + c];
    double den = sqrt(cabs2(a) + cabs2(b));
    double2 ck, sk;
    if (den > 0.0) { ck = cscale(cconj(a), 1.0 / den); sk = cscale(cconj(b), 1.0 / den); }
    else { ck = make_double2(1.0, 0.0); sk = make_double2(0.0, 0.0); }
    cs[k * m + c] = ck;
    sn[k * m + c] = sk;
    Hk[k * m + c] = make_double2(den, 0.0);
    Hk[(k + 1) * m + c] = make_double2(0.0, 0.0);
    double2 gk = g[k * m + c];
    g[(k + 1) * m + c] = cscale(cmul(cconj(sk), gk), -1.0);
    g[k * m + c] = cmul(ck, gk);
    kcol[c] = k + 1;
    const double rr = sqrt(cabs2(g[(k + 1) * m + c]));
    resid[c] = rr;
    inv_norm[c] = hn > 0.0 ? 1.0 / hn : 0.0;
    if (rr <= tol[c] || hn == 0.0 || !(rr == rr)) active[c] = 0;
    else atomicAdd(n_active, 1);
}

// y = R^{-1} g per column (R = rotated Hessenberg, kcol[c] columns)
__global__ void lsq_kernel(int m, int restart, const double2* __restrict__ H, const double2* __restrict__ g,
                           const int* __restrict__ kcol, double2* __restrict__ y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const int kk = kcol[c];
    for (int i = kk; i < restart; ++i) y[i * m + c] = make_double2(0.0, 0.0);
    for (int i = kk - 1; i >= 0; --i) {
        double2 s = g[i * m + c];
        for (int j = i + 1; j < kk; ++j)
            s = csub(s, cmul(H[((int64_t)j * (restart + 1) + i) * m + c], y[j * m + c]));
        double2 d = H[((int64_t)i * (restart + 1) + i) * m + c];
        y[i * m + c] = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(s, d);
    }
}

// start of a cycle: g = (beta, 0, ...), inv = 1/beta, active = beta > tol
__global__ void cycle_start_kernel(int m, const double* __restrict__ beta2, const double* __restrict__ tol,
                                   int* __restrict__ active, int* __restrict__ kcol, double2* __restrict__ g,
                                   double* __restrict__ inv_norm, double* __restrict__ resid) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const double b = sqrt(fmax(beta2[c], 0.0));
    g[c] = make_double2(b, 0.0);
    kcol[c] = 0;
    resid[c] = b;
    const bool act = b > tol[c];
    active[c] = act ? 1 : 0;
    inv_norm[c] = act ? 1.0 / b : 0.0;
}

__global__ void tol_kernel(int m, const double* __restrict__ b2, double rtol, double* __restrict__ tol,
                           double* __restrict__ bnorm) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const double b = sqrt(fmax(b2[c], 0.0));
    bnorm[c] = b;
    tol[c] = rtol * b;
}

// extract the real part of the diagonal dots (||w_c||^2)
__global__ void real_part_kernel(int m, const double2* __restrict__ h, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    out[c] = h[c].x;
}

// ----------------------------------------------------------------------------
static inline unsigned nblocks(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

template <typename C>
void Gmres<C>::reserve(int64_t n_, int m_, int restart_) {
    n = n_;
    m = m_;
    restart = restart_;
    V.ensure((size_t)(restart + 1) * n * m);
    reorth_passes = 0;
    Z.ensure((size_t)restart * n * m);
    W.ensure((size_t)n * m);
    H.ensure((size_t)restart * (restart + 1) * m);
    cs.ensure((size_t)restart * m);
    sn.ensure((size_t)restart * m);
    g.ensure((size_t)(restart + 1) * m);
    y.ensure((size_t)restart * m);
    h.ensure((size_t)(restart + 2) * m);
    hacc.ensure((size_t)(restart + 1) * m);
    partial.ensure((size_t)kDotBlocks * (restart + 2) * m);
    dvec.ensure((size_t)8 * m);
    ivec.ensure((size_t)4 * m + 4);
}

template <typename C>
void Gmres<C>::dots(const C* Vb, int nvec, int64_t vstride, const C* w, double2* out, double2* acc,
                    cudaStream_t st, int self) {
    dim3 blk(32, 8), grd(kDotBlocks, (m + 31) / 32);
    dots_kernel<C><<<grd, blk, 0, st>>>(n, m, nvec, Vb, vstride, w, self, partial.p);
    MWI_CHECK_LAUNCH();
    const int nt = nvec + self;
    dots_reduce_kernel<<<nblocks((int64_t)nt * m, 128), 128, 0, st>>>(kDotBlocks, nt, nvec, m, partial.p, out, acc);
    MWI_CHECK_LAUNCH();
}

template <typename C>
void Gmres<C>::column_norms2(const C* x, double* out, cudaStream_t st) {
    column_norms2_into(x, out, h.p, st);
}

// ||x_c||^2 with tmp [m] double2 scratch
template <typename C>
void Gmres<C>::column_norms2_into(const C* x, double* out, double2* tmp, cudaStream_t st) {
    dots(x, 0, 0, x, tmp, nullptr, st, 1);
    real_part_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, tmp, out);
    MWI_CHECK_LAUNCH();
}

template <typename C>
int Gmres<C>::cycle(const OpFn& A, const OpFn& M, const C* r0, C* x, const double* tol, int max_steps,
                    cudaStream_t st, double* resid_host, int* iters_used) {
    const int64_t nm = n * m;
    const int64_t vs = nm;
    double* beta2 = dvec.p;            // [m]
    double* inv = dvec.p + m;          // [m]
    double* resid = dvec.p + 2 * m;    // [m]
    double* hn2 = dvec.p + 3 * m;      // [m]
    int* active = ivec.p;
    int* kcol = ivec.p + m;
    int* nact = ivec.p + 4 * m;
    int* flag = ivec.p + 4 * m + 1;
    column_norms2(r0, beta2, st);
    cycle_start_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, beta2, tol, active, kcol, g.p, inv, resid);
    MWI_CHECK_LAUNCH();
    scale_kernel<C><<<nblocks(nm, 256), 256, 0, st>>>(n, m, r0, inv, V.p);
    MWI_CHECK_LAUNCH();
    int k = 0;
    int n_active_host = 1;
    for (; k < max_steps; ++k) {
        C* vk = V.p + (int64_t)k * vs;
        C* zk = Z.p + (int64_t)k * vs;
        M(vk, zk);
        A(zk, W.p);
        // classical Gram-Schmidt with selective reorthogonalisation: the second
        // pass runs when some column lost more than half of its squared norm
        // in the first (the usual twice-is-enough criterion)
        auto ortho = [&] {
            MWI_CUDA(cudaMemsetAsync(hacc.p, 0, (size_t)(k + 1) * m * sizeof(double2), st));
            dots(V.p, k + 1, vs, W.p, h.p, hacc.p, st, 1);
            const double2* w0sq = h.p + (int64_t)(k + 1) * m;
            cgs_update_kernel<C><<<nblocks(nm, 256), 256, 0, st>>>(n, m, k + 1, V.p, vs, h.p, W.p);
            MWI_CHECK_LAUNCH();
            column_norms2_into(W.p, hn2, h.p + (int64_t)(k + 2) * m, st);
            MWI_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
            reorth_test_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, w0sq, hn2, flag);
            MWI_CHECK_LAUNCH();
            int again = 0;
            MWI_CUDA(cudaMemcpyAsync(&again, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
            MWI_CUDA(cudaStreamSynchronize(st));
            if (again) {
                ++reorth_passes;
                dots(V.p, k + 1, vs, W.p, h.p, hacc.p, st, 0);
                cgs_update_kernel<C><<<nblocks(nm, 256), 256, 0, st>>>(n, m, k + 1, V.p, vs, h.p, W.p);
                MWI_CHECK_LAUNCH();
                column_norms2(W.p, hn2, st);
            }
        };
        if (timer) timer(2, ortho);
        else ortho();
        MWI_CUDA(cudaMemsetAsync(nact, 0, sizeof(int), st));
        arnoldi_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, k, restart, hacc.p, hn2, H.p, cs.p, sn.p, g.p, active,
                                                        kcol, tol, resid, inv, nact);
        MWI_CHECK_LAUNCH();
        if (k + 1 < max_steps) {
            scale_kernel<C><<<nblocks(nm, 256), 256, 0, st>>>(n, m, W.p, inv, V.p + (int64_t)(k + 1) * vs);
            MWI_CHECK_LAUNCH();
        }
        MWI_CUDA(cudaMemcpyAsync(&n_active_host, nact, sizeof(int), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        if (n_active_host == 0) { ++k; break; }
    }
    lsq_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, restart, H.p, g.p, kcol, y.p);
    MWI_CHECK_LAUNCH();
    lincomb_kernel<C><<<nblocks(nm, 256), 256, 0, st>>>(n, m, k, Z.p, vs, y.p, x);
    MWI_CHECK_LAUNCH();
    if (resid_host) {
        MWI_CUDA(cudaMemcpyAsync(resid_host, resid, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
    }
    if (iters_used) *iters_used = k;
    return k;
}

template struct Gmres<double2>;
template struct Gmres<float2>;

void convert_c128_to_c64(int64_t nm, const double2* a, float2* b, cudaStream_t st) {
    convert_kernel<double2, float2><<<nblocks(nm, 256), 256, 0, st>>>(nm, a, b);
    MWI_CHECK_LAUNCH();
}
void convert_c64_to_c128(int64_t nm, const float2* a, double2* b, cudaStream_t st) {
    convert_kernel<float2, double2><<<nblocks(nm, 256), 256, 0, st>>>(nm, a, b);
    MWI_CHECK_LAUNCH();
}
void residual_c128(int64_t nm, const double2* b, double2* r, cudaStream_t st) {
    sub_from_kernel<double2><<<nblocks(nm, 256), 256, 0, st>>>(nm, b, r);
    MWI_CHECK_LAUNCH();
}
__global__ void copy_columns_kernel(int64_t n, int ms, int sc0, int mc, const double2* __restrict__ src, int md,
                                    int dc0, double2* __restrict__ dst) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * mc) return;
    const int64_t r = e / mc;
    const int c = (int)(e - r * mc);
    dst[r * md + dc0 + c] = src[r * ms + sc0 + c];
}

void copy_columns(int64_t n, int ms, int sc0, int mc, const double2* src, int md, int dc0, double2* dst,
                  cudaStream_t st) {
    copy_columns_kernel<<<nblocks(n * mc, 256), 256, 0, st>>>(n, ms, sc0, mc, src, md, dc0, dst);
    MWI_CHECK_LAUNCH();
}

void tolerances(int m, const double* b2, double rtol, double* tol, double* bnorm, cudaStream_t st) {
    tol_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, b2, rtol, tol, bnorm);
    MWI_CHECK_LAUNCH();
}

}  // namespace mwi

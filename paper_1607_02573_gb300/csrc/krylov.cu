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
#include "df.h"
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

// h[i][c] = sum_b partial[b][i][c] for i < nvec; hacc[i][c] += h[i][c] for i < nacc;
// hdf (optional) receives h as double-floats (re hi, re lo, im hi, im lo).
// One block per vector index i: 8 warps split the blocks b (b = lane, lane + 8,
// ...), lanes over columns, then a fixed-order sum of the 8 partial sums.
__global__ void __launch_bounds__(256) dots_reduce_kernel(int nblk, int nvec, int nacc, int m,
                                                          const double2* __restrict__ partial,
                                                          double2* __restrict__ h, double2* __restrict__ hacc,
                                                          float4* __restrict__ hdf) {
    __shared__ double2 red[8][32];
    const int i = blockIdx.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int c0 = 0; c0 < m; c0 += 32) {
        const int c = c0 + tx;
        double sx = 0.0, sy = 0.0;
        if (c < m) {
#pragma unroll 4
            for (int b = ty; b < nblk; b += 8) {
                const double2 v = partial[((int64_t)b * nvec + i) * m + c];
                sx += v.x;
                sy += v.y;
            }
        }
        red[ty][tx] = make_double2(sx, sy);
        __syncthreads();
        if (ty == 0 && c < m) {
            double2 s = red[0][tx];
            for (int k = 1; k < 8; ++k) {
                s.x += red[k][tx].x;
                s.y += red[k][tx].y;
            }
            const int e = i * m + c;
            h[e] = s;
            if (hacc && i < nacc) { hacc[e].x += s.x; hacc[e].y += s.y; }
            if (hdf) {
                const float2 a = df_split(s.x), b = df_split(s.y);
                hdf[e] = make_float4(a.x, a.y, b.x, b.y);
            }
        }
        __syncthreads();
    }
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
                               double* __restrict__ resid, double* __restrict__ inv_norm, int* __restrict__ n_active,
                               float2* __restrict__ inv_df) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    if (!active[c]) {
        inv_norm[c] = 0.0;
        if (inv_df) inv_df[c] = make_float2(0.f, 0.f);
        return;
    }
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
    if (inv_df) inv_df[c] = df_split(inv_norm[c]);
    if (rr <= tol[c] || hn == 0.0 || !(rr == rr)) active[c] = 0;
    else atomicAdd(n_active, 1);
}

// y = R^{-1} g per column (R = rotated Hessenberg, kcol[c] columns)
// ydf (optional) receives y as double-floats (re hi, re lo, im hi, im lo)
__global__ void lsq_kernel(int m, int restart, const double2* __restrict__ H, const double2* __restrict__ g,
                           const int* __restrict__ kcol, double2* __restrict__ y, float4* __restrict__ ydf) {
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
    if (ydf)
        for (int i = 0; i < restart; ++i) {
            const double2 v = y[i * m + c];
            const float2 a = df_split(v.x), b = df_split(v.y);
            ydf[i * m + c] = make_float4(a.x, a.y, b.x, b.y);
        }
}

// start of a cycle: g = (beta, 0, ...), inv = 1/beta, active = beta > tol
__global__ void cycle_start_kernel(int m, const double* __restrict__ beta2, const double* __restrict__ tol,
                                   int* __restrict__ active, int* __restrict__ kcol, double2* __restrict__ g,
                                   double* __restrict__ inv_norm, double* __restrict__ resid,
                                   float2* __restrict__ inv_df) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const double b = sqrt(fmax(beta2[c], 0.0));
    g[c] = make_double2(b, 0.0);
    kcol[c] = 0;
    resid[c] = b;
    const bool act = b > tol[c];
    active[c] = act ? 1 : 0;
    inv_norm[c] = act ? 1.0 / b : 0.0;
    if (inv_df) inv_df[c] = df_split(inv_norm[c]);
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


// ---------------------------------------------------------------- double-float vectors
// A double-float [n][m] complex vector is two float2 planes, hi at p and lo at
// p + n m (value = hi + lo per real component).

// W = A Z (Z exact in FP32, RES = false) or W = B - A X (X and B double-float,
// RES = true), A as double-float planes (Ah, Al); G lanes per row over columns
template <int G, bool RES>
__global__ void __launch_bounds__(256) spmm_df_kernel(int64_t n, const int32_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col, const float2* __restrict__ Ah,
                                                      const float2* __restrict__ Al, const float2* __restrict__ Xh,
                                                      const float2* __restrict__ Xl, const float2* __restrict__ Bh,
                                                      const float2* __restrict__ Bl, float2* __restrict__ Wh,
                                                      float2* __restrict__ Wl, int m) {
    const int lane = threadIdx.x % G;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    if (row >= n) return;
    const int b = rp[row], e = rp[row + 1];
    for (int c0 = 0; c0 < m; c0 += G) {
        const int c = c0 + lane;
        if (c >= m) break;
        dfl re = {0.f, 0.f}, im = {0.f, 0.f};
        if constexpr (RES) {
            const float2 bh = Bh[row * m + c], bl = Bl[row * m + c];
            re = dfl{bh.x, bl.x};
            im = dfl{bh.y, bl.y};
        }
        for (int q = b; q < e; ++q) {
            const float2 ah = Ah[q], al = Al[q];
            const int64_t xi = (int64_t)col[q] * m + c;
            const float2 xh = Xh[xi];
            if constexpr (RES) {
                const float2 xl = Xl[xi];
                df_mac(re, -ah.x, -al.x, xh.x, xl.x);
                df_mac(re, ah.y, al.y, xh.y, xl.y);
                df_mac(im, -ah.x, -al.x, xh.y, xl.y);
                df_mac(im, -ah.y, -al.y, xh.x, xl.x);
            } else {
                df_mac1(re, xh.x, ah.x, al.x);
                df_mac1(re, -xh.y, ah.y, al.y);
                df_mac1(im, xh.y, ah.x, al.x);
                df_mac1(im, xh.x, ah.y, al.y);
            }
        }
        re = df_norm(re);
        im = df_norm(im);
        Wh[row * m + c] = make_float2(re.h, im.h);
        Wl[row * m + c] = make_float2(re.l, im.l);
    }
}

// The same product for an even m >= 32 with two adjacent columns per lane (16
// lanes per row, 16-byte loads of the right-hand sides): four independent
// accumulation chains per thread instead of two.  Entries are applied in the
// same ascending order, so the results are the same bit for bit.
template <bool RES>
__global__ void __launch_bounds__(256) spmm_df2_kernel(int64_t n, const int32_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col, const float2* __restrict__ Ah,
                                                       const float2* __restrict__ Al, const float4* __restrict__ Xh,
                                                       const float4* __restrict__ Xl, const float4* __restrict__ Bh,
                                                       const float4* __restrict__ Bl, float4* __restrict__ Wh,
                                                       float4* __restrict__ Wl, int m) {
    const int lane = threadIdx.x & 15;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 4;
    if (row >= n) return;
    const int h = m >> 1;  // column pairs per row
    const int b = rp[row], e = rp[row + 1];
    for (int c0 = 0; c0 < h; c0 += 16) {
        const int c = c0 + lane;
        if (c >= h) break;
        dfl re0 = {0.f, 0.f}, im0 = {0.f, 0.f}, re1 = {0.f, 0.f}, im1 = {0.f, 0.f};
        if constexpr (RES) {
            const float4 bh = Bh[row * h + c], bl = Bl[row * h + c];
            re0 = dfl{bh.x, bl.x};
            im0 = dfl{bh.y, bl.y};
            re1 = dfl{bh.z, bl.z};
            im1 = dfl{bh.w, bl.w};
        }
        for (int q = b; q < e; ++q) {
            const float2 ah = Ah[q], al = Al[q];
            const int64_t xi = (int64_t)col[q] * h + c;
            const float4 xh = Xh[xi];
            if constexpr (RES) {
                const float4 xl = Xl[xi];
                df_mac(re0, -ah.x, -al.x, xh.x, xl.x);
                df_mac(re0, ah.y, al.y, xh.y, xl.y);
                df_mac(im0, -ah.x, -al.x, xh.y, xl.y);
                df_mac(im0, -ah.y, -al.y, xh.x, xl.x);
                df_mac(re1, -ah.x, -al.x, xh.z, xl.z);
                df_mac(re1, ah.y, al.y, xh.w, xl.w);
                df_mac(im1, -ah.x, -al.x, xh.w, xl.w);
                df_mac(im1, -ah.y, -al.y, xh.z, xl.z);
            } else {
                df_mac1(re0, xh.x, ah.x, al.x);
                df_mac1(re0, -xh.y, ah.y, al.y);
                df_mac1(im0, xh.y, ah.x, al.x);
                df_mac1(im0, xh.x, ah.y, al.y);
                df_mac1(re1, xh.z, ah.x, al.x);
                df_mac1(re1, -xh.w, ah.y, al.y);
                df_mac1(im1, xh.w, ah.x, al.x);
                df_mac1(im1, xh.z, ah.y, al.y);
            }
        }
        re0 = df_norm(re0);
        im0 = df_norm(im0);
        re1 = df_norm(re1);
        im1 = df_norm(im1);
        Wh[row * h + c] = make_float4(re0.h, im0.h, re1.h, im1.h);
        Wl[row * h + c] = make_float4(re0.l, im0.l, re1.l, im1.l);
    }
}

// W -= sum_i V_i h_i per column (V_i and W double-float, h double-float
// [nvec][m] as (re hi, re lo, im hi, im lo)); four basis vectors per step so
// that their loads are in flight together
__global__ void __launch_bounds__(256) cgs_update_df_kernel(int64_t nm, int m, int nvec, const float2* __restrict__ V,
                                                            int64_t vstride, const float4* __restrict__ hdf,
                                                            float2* __restrict__ W) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    const int c = (int)(e % m);
    const float2 wh = W[e], wl = W[nm + e];
    dfl re = {wh.x, wl.x}, im = {wh.y, wl.y};
    int i = 0;
    for (; i + 4 <= nvec; i += 4) {
        float2 vh[4], vl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            vh[u] = V[(int64_t)(i + u) * vstride + e];
            vl[u] = V[(int64_t)(i + u) * vstride + nm + e];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 h = hdf[(i + u) * m + c];
            df_mac(re, -vh[u].x, -vl[u].x, h.x, h.y);
            df_mac(re, vh[u].y, vl[u].y, h.z, h.w);
            df_mac(im, -vh[u].x, -vl[u].x, h.z, h.w);
            df_mac(im, -vh[u].y, -vl[u].y, h.x, h.y);
        }
    }
    for (; i < nvec; ++i) {
        const float2 vh = V[(int64_t)i * vstride + e], vl = V[(int64_t)i * vstride + nm + e];
        const float4 h = hdf[i * m + c];
        df_mac(re, -vh.x, -vl.x, h.x, h.y);
        df_mac(re, vh.y, vl.y, h.z, h.w);
        df_mac(im, -vh.x, -vl.x, h.z, h.w);
        df_mac(im, -vh.y, -vl.y, h.x, h.y);
    }
    re = df_norm(re);
    im = df_norm(im);
    W[e] = make_float2(re.h, im.h);
    W[nm + e] = make_float2(re.l, im.l);
}

// V = W s per column (W, V double-float, s double-float [m])
__global__ void scale_df_kernel(int64_t nm, int m, const float2* __restrict__ W, const float2* __restrict__ s,
                                float2* __restrict__ V) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    const float2 f = s[e % m];
    const float2 wh = W[e], wl = W[nm + e];
    const dfl re = df_mul(wh.x, wl.x, f.x, f.y), im = df_mul(wh.y, wl.y, f.x, f.y);
    V[e] = make_float2(re.h, im.h);
    V[nm + e] = make_float2(re.l, im.l);
}

// X += sum_i Z_i y_i per column (Z_i exact in FP32, X double-float, y
// double-float [nvec][m])
__global__ void __launch_bounds__(256) lincomb_df_kernel(int64_t nm, int m, int nvec, const float2* __restrict__ Z,
                                                         int64_t zstride, const float4* __restrict__ ydf,
                                                         float2* __restrict__ X) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    const int c = (int)(e % m);
    const float2 xh = X[e], xl = X[nm + e];
    dfl re = {xh.x, xl.x}, im = {xh.y, xl.y};
    for (int i = 0; i < nvec; ++i) {
        const float2 z = Z[(int64_t)i * zstride + e];
        const float4 y = ydf[i * m + c];
        df_mac1(re, z.x, y.x, y.y);
        df_mac1(re, -z.y, y.z, y.w);
        df_mac1(im, z.x, y.z, y.w);
        df_mac1(im, z.y, y.x, y.y);
    }
    re = df_norm(re);
    im = df_norm(im);
    X[e] = make_float2(re.h, im.h);
    X[nm + e] = make_float2(re.l, im.l);
}

// double-float planes of a c128 array of count entries, and back
__global__ void split_c128_kernel(int64_t count, const double2* __restrict__ a, float2* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    const double2 v = a[e];
    const float2 x = df_split(v.x), y = df_split(v.y);
    out[e] = make_float2(x.x, y.x);
    out[count + e] = make_float2(x.y, y.y);
}

__global__ void join_c128_kernel(int64_t count, const float2* __restrict__ in, double2* __restrict__ a) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    const float2 h = in[e], l = in[count + e];
    a[e] = make_double2(df_join(h.x, l.x), df_join(h.y, l.y));
}


// ---------------------------------------------------------------- DCGS2 Arnoldi (double-float basis)
// Classical Gram-Schmidt with delayed reorthogonalisation (the one-reduction
// DCGS2 Arnoldi of Swirydowicz, Langou, Ananthan, Yang and Thomas, "Low
// synchronization Gram-Schmidt and generalized minimal residual algorithms",
// 2021): step k makes one pass of dot products over the basis for both the
// new vector w = A z_k and the once-orthogonalised v_k, then one fused update
// pass that reorthogonalises v_k into q_k and projects w into the next v_{k+1}.

// partial[b][j][c], j < nq: conj(Q_j) x; nq + j: conj(Q_j) y; 2 nq: conj(x) x;
// 2 nq + 1: conj(x) y; 2 nq + 2: conj(y) y (FP32 heads, FP32 sums per thread,
// FP64 across threads); eight basis vectors per pass over the rows
__global__ void __launch_bounds__(256) dots2_kernel(int64_t n, int m, int nq, const float2* __restrict__ V,
                                                    int64_t vstride, const float2* __restrict__ X,
                                                    const float2* __restrict__ Yv, double2* __restrict__ partial) {
    __shared__ double2 red[8][8][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c = blockIdx.y * 32 + tx;
    const int64_t stride = (int64_t)gridDim.x * 8;
    const int nout = 2 * nq + 3;
    // fixed-order sum over the eight row lanes of the values in red[.][q][tx]
    auto flush = [&](int nv, int j0, int jstride) {
        __syncthreads();
        if (ty < nv && c < m) {
            double sx = 0.0, sy = 0.0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                sx += red[r][ty][tx].x;
                sy += red[r][ty][tx].y;
            }
            partial[((int64_t)blockIdx.x * nout + j0 + ty * jstride) * m + c] = make_double2(sx, sy);
        }
        __syncthreads();
    };
    for (int q0 = 0; q0 < (nq > 0 ? nq : 1); q0 += 8) {
        const int nqc = nq > 0 ? min(8, nq - q0) : 0;
        const bool self = q0 == 0;
        float2 A[8], B[8], G = make_float2(0.f, 0.f), D = G, O = G;
#pragma unroll
        for (int q = 0; q < 8; ++q) A[q] = B[q] = make_float2(0.f, 0.f);
        if (c < m) {
            // two rows per iteration, their loads issued together
            for (int64_t r = blockIdx.x * 8 + ty; r < n; r += 2 * stride) {
                const bool two = r + stride < n;
                const int64_t r2 = two ? r + stride : r;
                const float2 x0 = X[r * m + c], y0 = Yv[r * m + c];
                const float2 x1 = two ? X[r2 * m + c] : make_float2(0.f, 0.f);
                const float2 y1 = two ? Yv[r2 * m + c] : make_float2(0.f, 0.f);
                float2 v0[8], v1[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < nqc) {
                        const float2* Vq = V + (int64_t)(q0 + q) * vstride + c;
                        v0[q] = Vq[r * m];
                        v1[q] = two ? Vq[r2 * m] : make_float2(0.f, 0.f);
                    }
                if (self) {
                    G.x += x0.x * x0.x + x0.y * x0.y + x1.x * x1.x + x1.y * x1.y;
                    D.x += x0.x * y0.x + x0.y * y0.y + x1.x * y1.x + x1.y * y1.y;
                    D.y += x0.x * y0.y - x0.y * y0.x + x1.x * y1.y - x1.y * y1.x;
                    O.x += y0.x * y0.x + y0.y * y0.y + y1.x * y1.x + y1.y * y1.y;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < nqc) {
                        A[q].x += v0[q].x * x0.x + v0[q].y * x0.y + v1[q].x * x1.x + v1[q].y * x1.y;
                        A[q].y += v0[q].x * x0.y - v0[q].y * x0.x + v1[q].x * x1.y - v1[q].y * x1.x;
                        B[q].x += v0[q].x * y0.x + v0[q].y * y0.y + v1[q].x * y1.x + v1[q].y * y1.y;
                        B[q].y += v0[q].x * y0.y - v0[q].y * y0.x + v1[q].x * y1.y - v1[q].y * y1.x;
                    }
            }
        }
        if (nqc > 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) red[ty][q][tx] = make_double2(A[q].x, A[q].y);
            flush(nqc, q0, 1);
#pragma unroll
            for (int q = 0; q < 8; ++q) red[ty][q][tx] = make_double2(B[q].x, B[q].y);
            flush(nqc, nq + q0, 1);
        }
        if (self) {
            red[ty][0][tx] = make_double2(G.x, 0.0);
            red[ty][1][tx] = make_double2(D.x, D.y);
            red[ty][2][tx] = make_double2(O.x, 0.0);
            flush(3, 2 * nq, 1);
        }
    }
}

// Per column: finalise column k-1 of the Hessenberg matrix with v_k's
// reorthogonalisation (coefficients a, norm nu), form column k from w's
// projections (provisional: its last entry rho_k is the Pythagorean norm of
// the projected w, made exact by the next step's correction), test the
// residual estimate with a provisional rotation of column k, and emit the
// double-float coefficients of the fused update.  A column that converges (or
// the last step) keeps column k as it stands: v_{k+1} then closes the basis
// without reorthogonalisation, which leaves the Arnoldi relation exact.
__device__ __forceinline__ double2 conjmul(double2 a, double2 b) { return cmul(cconj(a), b); }

__device__ void finalize_column(int m, int c, int j, int restart, double2* __restrict__ Hj,
                                double2* __restrict__ cs, double2* __restrict__ sn, double2* __restrict__ g) {
    for (int i = 0; i < j; ++i) {
        const double2 ci = cs[i * m + c], si = sn[i * m + c];
        const double2 a = Hj[i * m + c], b = Hj[(i + 1) * m + c];
        Hj[i * m + c] = cadd(cmul(ci, a), cmul(si, b));
        Hj[(i + 1) * m + c] = csub(cmul(cconj(ci), b), cmul(cconj(si), a));
    }
    const double2 a = Hj[j * m + c], b = Hj[(j + 1) * m + c];
    const double den = sqrt(cabs2(a) + cabs2(b));
    double2 cj, sj;
    if (den > 0.0) { cj = cscale(cconj(a), 1.0 / den); sj = cscale(cconj(b), 1.0 / den); }
    else { cj = make_double2(1.0, 0.0); sj = make_double2(0.0, 0.0); }
    cs[j * m + c] = cj;
    sn[j * m + c] = sj;
    Hj[j * m + c] = make_double2(den, 0.0);
    Hj[(j + 1) * m + c] = make_double2(0.0, 0.0);
    const double2 gj = g[j * m + c];
    g[(j + 1) * m + c] = cscale(cmul(cconj(sj), gj), -1.0);
    g[j * m + c] = cmul(cj, gj);
    (void)restart;
}

__device__ __forceinline__ float4 df4(double2 v) {
    const float2 a = df_split(v.x), b = df_split(v.y);
    return make_float4(a.x, a.y, b.x, b.y);
}

__global__ void arnoldi_dcgs_kernel(int m, int k, int restart, int last, const double2* __restrict__ dots,
                                    double2* __restrict__ H, double2* __restrict__ Hp, double2* __restrict__ cs,
                                    double2* __restrict__ sn, double2* __restrict__ g, int* __restrict__ active,
                                    int* __restrict__ kcol, const double* __restrict__ tol,
                                    double* __restrict__ resid, double* __restrict__ rho,
                                    int* __restrict__ n_active, float4* __restrict__ coefQ,
                                    float4* __restrict__ coefW, float4* __restrict__ scal) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const int nq = k, nout = 2 * nq + 3;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!active[c]) {
        for (int i = 0; i < nq; ++i) coefQ[i * m + c] = coefW[i * m + c] = z4;
        scal[c] = scal[m + c] = z4;
        return;
    }
    const double2* a = dots;               // a_i = conj(q_i) v_k
    const double2* b = dots + nq * m;      // b_i = conj(q_i) w
    const double gam = dots[(2 * nq) * m + c].x;
    const double2 del = dots[(2 * nq + 1) * m + c];
    const double om = dots[(2 * nq + 2) * m + c].x;
    double nu = 1.0;
    if (k > 0) {
        double a2 = 0.0;
        for (int i = 0; i < nq; ++i) a2 += cabs2(a[i * m + c]);
        nu = sqrt(fmax(gam - a2, 1e-30 * fmax(gam, 1e-300)));
        // column k-1: v_k = Q a + nu q_k, so h(i, k-1) += rho_{k-1} a_i and h(k, k-1) = rho_{k-1} nu
        const double r1 = rho[c];
        double2* Hc = H + (int64_t)(k - 1) * (restart + 1) * m;
        const double2* Pc = Hp;
        for (int i = 0; i < k; ++i) Hc[i * m + c] = cadd(Pc[i * m + c], cscale(a[i * m + c], r1));
        Hc[k * m + c] = make_double2(r1 * nu, 0.0);
        finalize_column(m, c, k - 1, restart, Hc, cs, sn, g);
    }
    // q_k^H w and the projected w's norm
    double2 ab = make_double2(0.0, 0.0);
    double b2 = 0.0;
    for (int i = 0; i < nq; ++i) {
        ab = cadd(ab, conjmul(a[i * m + c], b[i * m + c]));
        b2 += cabs2(b[i * m + c]);
    }
    const double2 ck = cscale(csub(del, ab), 1.0 / nu);
    const double rk = sqrt(fmax(om - b2 - cabs2(ck), 1e-14 * om));
    // provisional column k: (b_0 .. b_{k-1}, c_k, rho_k)
    for (int i = 0; i < nq; ++i) Hp[i * m + c] = b[i * m + c];
    Hp[k * m + c] = ck;
    Hp[(k + 1) * m + c] = make_double2(rk, 0.0);
    // its rotated entry k (rotations 0..k-1), then the provisional residual
    double2 t = nq > 0 ? b[c] : ck;
    for (int i = 0; i < k; ++i) {
        const double2 nxt = i + 1 < k ? b[(i + 1) * m + c] : ck;
        const double2 ci = cs[i * m + c], si = sn[i * m + c];
        t = csub(cmul(cconj(ci), nxt), cmul(cconj(si), t));
    }
    const double den = sqrt(cabs2(t) + rk * rk);
    const double rr = den > 0.0 ? rk / den * sqrt(cabs2(g[k * m + c])) : 0.0;
    resid[c] = rr;
    rho[c] = rk;
    const bool stop = rr <= tol[c] || !(rr == rr) || rk == 0.0 || last;
    if (stop) {
        double2* Hc = H + (int64_t)k * (restart + 1) * m;
        for (int i = 0; i <= k + 1; ++i) Hc[i * m + c] = Hp[i * m + c];
        finalize_column(m, c, k, restart, Hc, cs, sn, g);
        kcol[c] = k + 1;
        if (!last) active[c] = 0;
        else if (!(rr <= tol[c])) atomicAdd(n_active, 1);
    } else {
        kcol[c] = k;
        atomicAdd(n_active, 1);
    }
    // fused update: q_k = v_k / nu - sum_i q_i a_i / nu;
    // v_{k+1} = w / rho_k - sum_i q_i (b_i - a_i c_k / nu) / rho_k - v_k c_k / (nu rho_k)
    const double inu = 1.0 / nu, irk = 1.0 / rk;
    for (int i = 0; i < nq; ++i) {
        const double2 ai = a[i * m + c];
        coefQ[i * m + c] = df4(cscale(ai, -inu));
        coefW[i * m + c] = df4(cscale(csub(b[i * m + c], cscale(cmul(ai, ck), inu)), -irk));
    }
    scal[c] = df4(make_double2(k > 0 ? inu : 1.0, irk));         // (1 / nu, 1 / rho_k) as reals
    scal[m + c] = df4(cscale(ck, -inu * irk));                     // -c_k / (nu rho_k)
}

// q_k (into V slot k, when k > 0) and v_{k+1} (into V slot k + 1) in one pass
// over the basis: per element, two double-float accumulators over the k basis
// vectors, v_k and w
__global__ void __launch_bounds__(256) dcgs_update_df_kernel(int64_t nm, int m, int k, float2* __restrict__ V,
                                                             int64_t vstride, const float2* __restrict__ W,
                                                             const float4* __restrict__ coefQ,
                                                             const float4* __restrict__ coefW,
                                                             const float4* __restrict__ scal, int write_next) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nm) return;
    const int c = (int)(e % m);
    const float4 s1 = scal[c], s2 = scal[m + c];
    float2* vk = V + (int64_t)k * vstride;
    const float2 vh = vk[e], vl = vk[nm + e], wh = W[e], wl = W[nm + e];
    // q accumulator: v_k / nu; w accumulator: w / rho_k + v_k (-c_k / (nu rho_k))
    dfl qr = df_mul(vh.x, vl.x, s1.x, s1.y), qi = df_mul(vh.y, vl.y, s1.x, s1.y);
    dfl wr = df_mul(wh.x, wl.x, s1.z, s1.w), wi = df_mul(wh.y, wl.y, s1.z, s1.w);
    df_mac(wr, vh.x, vl.x, s2.x, s2.y);
    df_mac(wr, -vh.y, -vl.y, s2.z, s2.w);
    df_mac(wi, vh.x, vl.x, s2.z, s2.w);
    df_mac(wi, vh.y, vl.y, s2.x, s2.y);
    int i = 0;
    for (; i + 2 <= k; i += 2) {
        float2 qh[2], ql[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            qh[u] = V[(int64_t)(i + u) * vstride + e];
            ql[u] = V[(int64_t)(i + u) * vstride + nm + e];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float4 a = coefQ[(i + u) * m + c], b = coefW[(i + u) * m + c];
            df_mac(qr, qh[u].x, ql[u].x, a.x, a.y);
            df_mac(qr, -qh[u].y, -ql[u].y, a.z, a.w);
            df_mac(qi, qh[u].x, ql[u].x, a.z, a.w);
            df_mac(qi, qh[u].y, ql[u].y, a.x, a.y);
            df_mac(wr, qh[u].x, ql[u].x, b.x, b.y);
            df_mac(wr, -qh[u].y, -ql[u].y, b.z, b.w);
            df_mac(wi, qh[u].x, ql[u].x, b.z, b.w);
            df_mac(wi, qh[u].y, ql[u].y, b.x, b.y);
        }
    }
    for (; i < k; ++i) {
        const float2 qh = V[(int64_t)i * vstride + e], ql = V[(int64_t)i * vstride + nm + e];
        const float4 a = coefQ[i * m + c], b = coefW[i * m + c];
        df_mac(qr, qh.x, ql.x, a.x, a.y);
        df_mac(qr, -qh.y, -ql.y, a.z, a.w);
        df_mac(qi, qh.x, ql.x, a.z, a.w);
        df_mac(qi, qh.y, ql.y, a.x, a.y);
        df_mac(wr, qh.x, ql.x, b.x, b.y);
        df_mac(wr, -qh.y, -ql.y, b.z, b.w);
        df_mac(wi, qh.x, ql.x, b.z, b.w);
        df_mac(wi, qh.y, ql.y, b.x, b.y);
    }
    if (k > 0) {
        qr = df_norm(qr);
        qi = df_norm(qi);
        vk[e] = make_float2(qr.h, qi.h);
        vk[nm + e] = make_float2(qr.l, qi.l);
    }
    if (write_next) {
        wr = df_norm(wr);
        wi = df_norm(wi);
        float2* vn = V + (int64_t)(k + 1) * vstride;
        vn[e] = make_float2(wr.h, wi.h);
        vn[nm + e] = make_float2(wr.l, wi.l);
    }
}

// ----------------------------------------------------------------------------
static inline unsigned nblocks(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

template <typename C>
void Gmres<C>::reserve(int64_t n_, int m_, int restart_) {
    n = n_;
    m = m_;
    restart = restart_;
    V.ensure((size_t)(restart + 1) * n * m);
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

// out[i][c] = conj(V_i)^T w for i < nvec (+ conj(w)^T w at nvec when self = 1),
// acc[i] += out[i] for i < nvec, hdf = out as double-floats (optional)
template <typename C>
static void dots_launch(int64_t n, int m, const C* Vb, int nvec, int64_t vstride, const C* w, double2* partial,
                        double2* out, double2* acc, float4* hdf, cudaStream_t st, int self) {
    dim3 blk(32, 8), grd(kDotBlocks, (m + 31) / 32);
    dots_kernel<C><<<grd, blk, 0, st>>>(n, m, nvec, Vb, vstride, w, self, partial);
    MWI_CHECK_LAUNCH();
    const int nt = nvec + self;
    dots_reduce_kernel<<<nt, 256, 0, st>>>(kDotBlocks, nt, nvec, m, partial, out, acc, hdf);
    MWI_CHECK_LAUNCH();
}

template <typename C>
void Gmres<C>::dots(const C* Vb, int nvec, int64_t vstride, const C* w, double2* out, double2* acc,
                    cudaStream_t st, int self) {
    dots_launch<C>(n, m, Vb, nvec, vstride, w, partial.p, out, acc, nullptr, st, self);
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
    column_norms2(r0, beta2, st);
    cycle_start_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, beta2, tol, active, kcol, g.p, inv, resid, nullptr);
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
        // classical Gram-Schmidt applied twice (CGS2)
        auto ortho = [&] {
            MWI_CUDA(cudaMemsetAsync(hacc.p, 0, (size_t)(k + 1) * m * sizeof(double2), st));
            for (int pass = 0; pass < 2; ++pass) {
                dots(V.p, k + 1, vs, W.p, h.p, hacc.p, st, 0);
                cgs_update_kernel<C><<<nblocks(nm, 256), 256, 0, st>>>(n, m, k + 1, V.p, vs, h.p, W.p);
                MWI_CHECK_LAUNCH();
            }
            column_norms2(W.p, hn2, st);
        };
        if (timer) timer(2, ortho);
        else ortho();
        MWI_CUDA(cudaMemsetAsync(nact, 0, sizeof(int), st));
        arnoldi_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, k, restart, hacc.p, hn2, H.p, cs.p, sn.p, g.p, active,
                                                        kcol, tol, resid, inv, nact, nullptr);
        MWI_CHECK_LAUNCH();
        if (k + 1 < max_steps) {
            scale_kernel<C><<<nblocks(nm, 256), 256, 0, st>>>(n, m, W.p, inv, V.p + (int64_t)(k + 1) * vs);
            MWI_CHECK_LAUNCH();
        }
        MWI_CUDA(cudaMemcpyAsync(&n_active_host, nact, sizeof(int), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        if (n_active_host == 0) { ++k; break; }
    }
    lsq_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, restart, H.p, g.p, kcol, y.p, nullptr);
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

// ---------------------------------------------------------------- double-float FGMRES
void GmresDF::reserve(int64_t n_, int m_, int restart_) {
    n = n_;
    m = m_;
    restart = restart_;
    V.ensure((size_t)(restart + 1) * 2 * n * m);
    Z.ensure((size_t)restart * n * m);
    W.ensure((size_t)2 * n * m);
    H.ensure((size_t)restart * (restart + 1) * m);
    cs.ensure((size_t)restart * m);
    sn.ensure((size_t)restart * m);
    g.ensure((size_t)(restart + 1) * m);
    y.ensure((size_t)restart * m);
    h.ensure((size_t)(2 * restart + 3) * m);
    partial.ensure((size_t)kDotBlocks * (2 * restart + 3) * m);
    hdf.ensure((size_t)(restart + 1) * m);
    hdf2.ensure((size_t)(restart + 1) * m);
    scal.ensure((size_t)2 * m);
    Hp.ensure((size_t)(restart + 2) * m);
    ydf.ensure((size_t)restart * m);
    invdf.ensure((size_t)m);
    dvec.ensure((size_t)8 * m);
    ivec.ensure((size_t)4 * m + 4);
}

void GmresDF::norms2(const float2* xh, double* out, cudaStream_t st) {
    dots_launch<float2>(n, m, xh, 0, 0, xh, partial.p, h.p, nullptr, nullptr, st, 1);
    real_part_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, h.p, out);
    MWI_CHECK_LAUNCH();
}

int GmresDF::cycle(const OpA& A, const OpM& M, const float2* r0, float2* x, const double* tol, int max_steps,
                   cudaStream_t st, int* iters_used) {
    const int64_t nm = n * m;
    const int64_t vs = 2 * nm;  // stride of the double-float basis vectors
    double* beta2 = dvec.p;
    double* inv = dvec.p + m;
    double* resid = dvec.p + 2 * m;
    double* rho = dvec.p + 3 * m;
    int* active = ivec.p;
    int* kcol = ivec.p + m;
    int* nact = ivec.p + 4 * m;
    norms2(r0, beta2, st);
    cycle_start_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, beta2, tol, active, kcol, g.p, inv, resid, invdf.p);
    MWI_CHECK_LAUNCH();
    // v_0 = r0 / beta exactly (q_0 = v_0: no reorthogonalisation at step 0)
    scale_df_kernel<<<nblocks(nm, 256), 256, 0, st>>>(nm, m, r0, invdf.p, V.p);
    MWI_CHECK_LAUNCH();
    int k = 0;
    int n_active_host = 1;
    for (; k < max_steps; ++k) {
        float2* vk = V.p + (int64_t)k * vs;
        float2* zk = Z.p + (int64_t)k * nm;
        // the preconditioner sees the FP32 head of v_k (once orthogonalised);
        // z_k is stored exactly
        M(vk, zk);
        A(zk, W.p);
        const int last = k + 1 == max_steps ? 1 : 0;
        auto ortho = [&] {
            // one wave: two resident blocks per SM at this kernel's register use
            const int nblk = kDotBlocks / 2;
            dim3 blk(32, 8), grd(nblk, (m + 31) / 32);
            dots2_kernel<<<grd, blk, 0, st>>>(n, m, k, V.p, vs, vk, W.p, partial.p);
            MWI_CHECK_LAUNCH();
            const int nout = 2 * k + 3;
            dots_reduce_kernel<<<nout, 256, 0, st>>>(nblk, nout, 0, m, partial.p, h.p, nullptr, nullptr);
            MWI_CHECK_LAUNCH();
            MWI_CUDA(cudaMemsetAsync(nact, 0, sizeof(int), st));
            arnoldi_dcgs_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, k, restart, last, h.p, H.p, Hp.p, cs.p, sn.p,
                                                                 g.p, active, kcol, tol, resid, rho, nact, hdf.p,
                                                                 hdf2.p, scal.p);
            MWI_CHECK_LAUNCH();
            dcgs_update_df_kernel<<<nblocks(nm, 256), 256, 0, st>>>(nm, m, k, V.p, vs, W.p, hdf.p, hdf2.p, scal.p,
                                                                    last ? 0 : 1);
            MWI_CHECK_LAUNCH();
        };
        if (timer) timer(2, ortho);
        else ortho();
        MWI_CUDA(cudaMemcpyAsync(&n_active_host, nact, sizeof(int), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        if (n_active_host == 0) { ++k; break; }
    }
    lsq_kernel<<<nblocks(m, 128), 128, 0, st>>>(m, restart, H.p, g.p, kcol, y.p, ydf.p);
    MWI_CHECK_LAUNCH();
    lincomb_df_kernel<<<nblocks(nm, 256), 256, 0, st>>>(nm, m, k, Z.p, nm, ydf.p, x);
    MWI_CHECK_LAUNCH();
    if (iters_used) *iters_used = k;
    return k;
}

void spmm_df(int64_t n, const int32_t* row_ptr, const int32_t* col, const float2* A, int64_t nnz, const float2* x,
             float2* w, int m, cudaStream_t st) {
    const int th = 256;
    const int64_t nm = n * m;
    if (m >= 32 && (m & 1) == 0) {
        spmm_df2_kernel<false><<<(unsigned)((n * 16 + th - 1) / th), th, 0, st>>>(
            n, row_ptr, col, A, A + nnz, reinterpret_cast<const float4*>(x), nullptr, nullptr, nullptr,
            reinterpret_cast<float4*>(w), reinterpret_cast<float4*>(w + nm), m);
        MWI_CHECK_LAUNCH();
        return;
    }
    const int G = m >= 32 ? 32 : (m >= 8 ? 8 : 4);
    const unsigned blocks = (unsigned)((n * G + th - 1) / th);
    if (G == 32)
        spmm_df_kernel<32, false><<<blocks, th, 0, st>>>(n, row_ptr, col, A, A + nnz, x, nullptr, nullptr, nullptr, w,
                                                         w + nm, m);
    else if (G == 8)
        spmm_df_kernel<8, false><<<blocks, th, 0, st>>>(n, row_ptr, col, A, A + nnz, x, nullptr, nullptr, nullptr, w,
                                                        w + nm, m);
    else
        spmm_df_kernel<4, false><<<blocks, th, 0, st>>>(n, row_ptr, col, A, A + nnz, x, nullptr, nullptr, nullptr, w,
                                                        w + nm, m);
    MWI_CHECK_LAUNCH();
}

void residual_df(int64_t n, const int32_t* row_ptr, const int32_t* col, const float2* A, int64_t nnz, const float2* b,
                 const float2* x, float2* r, int m, cudaStream_t st) {
    const int th = 256;
    const int64_t nm = n * m;
    if (m >= 32 && (m & 1) == 0) {
        spmm_df2_kernel<true><<<(unsigned)((n * 16 + th - 1) / th), th, 0, st>>>(
            n, row_ptr, col, A, A + nnz, reinterpret_cast<const float4*>(x), reinterpret_cast<const float4*>(x + nm),
            reinterpret_cast<const float4*>(b), reinterpret_cast<const float4*>(b + nm), reinterpret_cast<float4*>(r),
            reinterpret_cast<float4*>(r + nm), m);
        MWI_CHECK_LAUNCH();
        return;
    }
    const int G = m >= 32 ? 32 : (m >= 8 ? 8 : 4);
    const unsigned blocks = (unsigned)((n * G + th - 1) / th);
    if (G == 32)
        spmm_df_kernel<32, true><<<blocks, th, 0, st>>>(n, row_ptr, col, A, A + nnz, x, x + nm, b, b + nm, r, r + nm,
                                                        m);
    else if (G == 8)
        spmm_df_kernel<8, true><<<blocks, th, 0, st>>>(n, row_ptr, col, A, A + nnz, x, x + nm, b, b + nm, r, r + nm,
                                                       m);
    else
        spmm_df_kernel<4, true><<<blocks, th, 0, st>>>(n, row_ptr, col, A, A + nnz, x, x + nm, b, b + nm, r, r + nm,
                                                       m);
    MWI_CHECK_LAUNCH();
}

void split_c128(int64_t count, const double2* a, float2* out, cudaStream_t st) {
    split_c128_kernel<<<nblocks(count, 256), 256, 0, st>>>(count, a, out);
    MWI_CHECK_LAUNCH();
}

void join_c128(int64_t count, const float2* in, double2* a, cudaStream_t st) {
    join_c128_kernel<<<nblocks(count, 256), 256, 0, st>>>(count, in, a);
    MWI_CHECK_LAUNCH();
}

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

// True block flexible GMRES: one Krylov space shared by the m right-hand
// sides of a block (the block methods named in Section 7 as the next step
// beyond the pseudo-block GMRES of Section 6.3, where each right-hand side
// keeps its own space and only the operations are fused).
//
//   R_0 = V_1 S_0                                   (Cholesky QR, twice)
//   step j: Z_j = M V_j, W = A Z_j
//           H_ij = V_i^H W, W <- W - V_i H_ij, i <= j   (block classical
//           Gram-Schmidt as two GEMM-shaped passes)
//           W = V_{j+1} H_{j+1,j}                   (Cholesky QR, twice)
//   X = X_0 + [Z_1 .. Z_k] Y,  Y = argmin ||E_1 S_0 - Hbar_k Y||_F
//
// Vectors are complex FP64, row-major [n][m] blocks.  The device does the
// block products (deterministic: fixed row chunks, fixed-order reduction);
// the host keeps the small dense parts: the m x m Cholesky factors and the
// QR of the block Hessenberg, updated by Givens rotations column by column,
// whose last m rows give each column's residual norm.
#include <algorithm>
#include <cmath>
#include <complex>

#include "common.h"
#include "gmres.h"

namespace mwi {

namespace {

constexpr int kBkRows = 8;     // rows staged per step in the block kernels
constexpr int kBkMaxM = 32;    // widest block
constexpr int kBkChunks = 1216;  // row chunks of the dot products (8 per SM)

__device__ __forceinline__ double2 zmul_conj_a(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// partial[(chunk * nq + q) * m*m + a*m + b] = sum over the chunk's rows r of
// conj(V_q[r][a]) W[r][b]
__global__ void __launch_bounds__(256) bk_dots_kernel(const double2* __restrict__ V, int64_t vstride, int nq,
                                                       const double2* __restrict__ W, int64_t n, int m,
                                                       int64_t rows_per_chunk, double2* __restrict__ partial) {
    __shared__ double2 sv[kBkRows][kBkMaxM];
    __shared__ double2 sw[kBkRows][kBkMaxM];
    const int q = blockIdx.y;
    const double2* Vq = V + (int64_t)q * vstride;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r1 = min(n, r0 + rows_per_chunk);
    const int mm = m * m;
    double2 acc[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = make_double2(0.0, 0.0);
    for (int64_t rb = r0; rb < r1; rb += kBkRows) {
        const int nr = (int)(r1 - rb < kBkRows ? r1 - rb : kBkRows);
        __syncthreads();
        for (int e = threadIdx.x; e < kBkRows * kBkMaxM; e += blockDim.x) {
            const int rr = e / kBkMaxM, c = e % kBkMaxM;
            const bool ok = rr < nr && c < m;
            sv[rr][c] = ok ? Vq[(rb + rr) * m + c] : make_double2(0.0, 0.0);
            sw[rr][c] = ok ? W[(rb + rr) * m + c] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int e = threadIdx.x + 256 * s;
            if (e >= mm) break;
            const int a = e / m, b = e % m;
            double2 t = acc[s];
            for (int rr = 0; rr < nr; ++rr) {
                const double2 p = zmul_conj_a(sv[rr][a], sw[rr][b]);
                t.x += p.x;
                t.y += p.y;
            }
            acc[s] = t;
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int e = threadIdx.x + 256 * s;
        if (e < mm) partial[((int64_t)blockIdx.x * nq + q) * mm + e] = acc[s];
    }
}

// out[i] = sum over chunks, in chunk order, of partial[chunk * total + i]
__global__ void bk_reduce_kernel(const double2* __restrict__ partial, int nchunk, int total,
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

// out[r][b] = beta out[r][b] + alpha sum_{q < nq} sum_a in_q[r][a] Cm[q m + a][b]
// (Cm row-major, nq m x m, staged in shared memory).  A row is read into
// shared memory before it is written, by the block that owns it, so
// out == in is allowed when nq == 1.
__global__ void __launch_bounds__(256) bk_update_kernel(double2* out, const double2* in, int64_t istride, int nq,
                                                         const double2* __restrict__ Cm, int64_t n, int m,
                                                         double alpha, double beta) {
    extern __shared__ double2 cs[];  // [nq * m * m]
    __shared__ double2 sx[kBkRows][kBkMaxM];
    const int mm = m * m;
    for (int e = threadIdx.x; e < nq * mm; e += blockDim.x) cs[e] = Cm[e];
    const int rr = threadIdx.x / kBkMaxM, b = threadIdx.x % kBkMaxM;
    for (int64_t rb = (int64_t)blockIdx.x * kBkRows; rb < n; rb += (int64_t)gridDim.x * kBkRows) {
        const int64_t r = rb + rr;
        double2 acc = make_double2(0.0, 0.0);
        for (int q = 0; q < nq; ++q) {
            __syncthreads();
            if (r < n && b < m) sx[rr][b] = in[(int64_t)q * istride + r * m + b];
            __syncthreads();
            if (r < n && b < m) {
                const double2* cq = cs + q * mm;
                for (int a = 0; a < m; ++a) {
                    const double2 x = sx[rr][a], c = cq[a * m + b];
                    acc.x += x.x * c.x - x.y * c.y;
                    acc.y += x.x * c.y + x.y * c.x;
                }
            }
        }
        if (r < n && b < m) {
            double2 o = make_double2(alpha * acc.x, alpha * acc.y);
            if (beta != 0.0) {
                const double2 v = out[r * m + b];
                o.x += beta * v.x;
                o.y += beta * v.y;
            }
            out[r * m + b] = o;
        }
    }
}

typedef std::complex<double> cd;

inline cd to_cd(double2 v) { return cd(v.x, v.y); }
inline double2 to_d2(cd v) { return make_double2(v.real(), v.imag()); }

}  // namespace

void BlockGmres::reserve(int64_t n_, int m_, int restart_) {
    MWI_REQUIRE(m_ >= 1 && m_ <= kBkMaxM, MWI_EINVAL, "block GMRES takes 1..32 columns per block");
    n = n_;
    m = m_;
    restart = restart_;
    V.ensure((size_t)(restart + 1) * n * m);
    Z.ensure((size_t)restart * n * m);
    W.ensure((size_t)n * m);
    coef.ensure((size_t)(restart + 1) * m * m);
    small.ensure((size_t)m * m);
    partial.ensure((size_t)kBkChunks * m * m + (size_t)(restart + 1) * m * m * 2);
}

// out (nq m x m, row-major) = [V_0 .. V_{nq-1}]^H W
void BlockGmres::block_dots(const double2* Vb, int nq, const double2* Wb, double2* out, cudaStream_t st) {
    const int mm = m * m;
    int nchunk = std::max(1, std::min<int>(kBkChunks / std::max(1, nq), (int)((n + 255) / 256)));
    const int64_t rows = ((n + nchunk - 1) / nchunk + kBkRows - 1) / kBkRows * kBkRows;
    nchunk = (int)((n + rows - 1) / rows);
    MWI_REQUIRE((size_t)nchunk * nq * mm <= partial.n, MWI_EINVAL, "internal: block dot scratch too small");
    bk_dots_kernel<<<dim3((unsigned)nchunk, (unsigned)nq), 256, 0, st>>>(Vb, n * m, nq, Wb, n, m, rows, partial.p);
    MWI_CHECK_LAUNCH();
    const int total = nq * mm;
    bk_reduce_kernel<<<(total + 255) / 256, 256, 0, st>>>(partial.p, nchunk, total, out);
    MWI_CHECK_LAUNCH();
}

// out = beta out + alpha [In_0 .. In_{nq-1}] Cm, in passes whose coefficients
// fit in 40 KB of shared memory (with the 4 KB row stage, under the 48 KB a
// launch gets without opting in)
void BlockGmres::block_update(double2* out, const double2* in, int nq, const double2* Cm, double alpha, double beta,
                              cudaStream_t st) {
    const int mm = m * m;
    const int per = std::max(1, (int)((40 * 1024) / (mm * sizeof(double2))));
    const int grid = (int)std::min<int64_t>((n + kBkRows - 1) / kBkRows, 152 * 8);
    for (int q0 = 0; q0 < nq; q0 += per) {
        const int nqp = std::min(per, nq - q0);
        MWI_REQUIRE(out != in || nq == 1, MWI_EINVAL, "internal: in-place block update of several blocks");
        bk_update_kernel<<<grid, 256, (size_t)nqp * mm * sizeof(double2), st>>>(
            out, in + (int64_t)q0 * n * m, n * m, nqp, Cm + (int64_t)q0 * mm, n, m, alpha, q0 == 0 ? beta : 1.0);
        MWI_CHECK_LAUNCH();
    }
}

// Cholesky QR of the block X in place, twice: X = Q S with S = S2 S1 upper
// triangular (returned row-major m x m).  A column whose part orthogonal to
// the preceding ones is below 1e-7 of its norm (or that is zero) is deflated:
// its Q column and its row of S are zero.  Returns the number of deflated columns.
int BlockGmres::chol_qr(double2* X, std::vector<std::complex<double>>& S, cudaStream_t st) {
    std::vector<cd> Sacc(m * m, cd(0.0));
    for (int c = 0; c < m; ++c) Sacc[c * m + c] = 1.0;
    int dead = 0;
    std::vector<double2> gh(m * m), sinv_h(m * m);
    for (int pass = 0; pass < 2; ++pass) {
        block_dots(X, 1, X, small.p, st);
        MWI_CUDA(cudaMemcpyAsync(gh.data(), small.p, m * m * sizeof(double2), cudaMemcpyDeviceToHost, st));
        MWI_CUDA(cudaStreamSynchronize(st));
        double gmax = 0.0;
        for (int c = 0; c < m; ++c) gmax = std::max(gmax, gh[c * m + c].x);
        std::vector<cd> R(m * m, cd(0.0)), Ri(m * m, cd(0.0));
        std::vector<char> live(m, 0);
        dead = 0;
        for (int c = 0; c < m; ++c) {
            const double gcc = gh[c * m + c].x;
            double s = gcc;
            for (int k = 0; k < c; ++k) s -= std::norm(R[k * m + c]);
            if (!(gcc > 1e-30 * gmax) || !(s > 1e-14 * gcc)) {
                ++dead;
                continue;
            }
            live[c] = 1;
            const double d = std::sqrt(s);
            R[c * m + c] = d;
            for (int b = c + 1; b < m; ++b) {
                cd t = to_cd(gh[c * m + b]);
                for (int k = 0; k < c; ++k) t -= std::conj(R[k * m + c]) * R[k * m + b];
                R[c * m + b] = t / d;
            }
        }
        // inverse of the upper triangle over the live columns
        for (int c = 0; c < m; ++c) {
            if (!live[c]) continue;
            Ri[c * m + c] = 1.0 / R[c * m + c];
            for (int b = c + 1; b < m; ++b) {
                if (!live[b]) continue;
                cd t = 0.0;
                for (int k = c; k < b; ++k) t += Ri[c * m + k] * R[k * m + b];
                Ri[c * m + b] = -t / R[b * m + b];
            }
        }
        for (int i = 0; i < m * m; ++i) sinv_h[i] = to_d2(Ri[i]);
        MWI_CUDA(cudaMemcpyAsync(small.p, sinv_h.data(), m * m * sizeof(double2), cudaMemcpyHostToDevice, st));
        block_update(X, X, 1, small.p, 1.0, 0.0, st);
        MWI_CUDA(cudaStreamSynchronize(st));  // sinv_h is reused by the next pass
        // S <- R S
        std::vector<cd> T(m * m, cd(0.0));
        for (int a = 0; a < m; ++a)
            for (int k = a; k < m; ++k) {
                if (R[a * m + k] == cd(0.0)) continue;
                for (int b = 0; b < m; ++b) T[a * m + b] += R[a * m + k] * Sacc[k * m + b];
            }
        Sacc.swap(T);
    }
    S = Sacc;
    return dead;
}

int BlockGmres::cycle(const OpFnT<double2>& A, const OpFnT<double2>& M, const double2* r0, double2* x,
                      const std::vector<double>& tol, int max_steps, cudaStream_t st, double* resid_est,
                      int* deflated) {
    const int64_t nm = n * m;
    const int K = std::min(max_steps, restart);
    if (K <= 0) return 0;
    const int ld = (K + 1) * m;  // rows of the Hessenberg and of the right-hand side
    std::vector<cd> H((size_t)ld * K * m, cd(0.0));  // column-major: H[col * ld + row]
    std::vector<cd> G((size_t)ld * m, cd(0.0));      // column-major: G[b * ld + row]
    struct Rot { int p, q; cd c, s; };
    std::vector<Rot> rots;
    int ndef = 0;

    MWI_CUDA(cudaMemcpyAsync(V.p, r0, nm * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    std::vector<cd> S;
    auto ortho = [&](const std::function<void()>& fn) {
        if (timer) timer(2, fn);
        else fn();
    };
    ortho([&] { ndef += chol_qr(V.p, S, st); });
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) G[(size_t)b * ld + a] = S[a * m + b];

    std::vector<double2> ch((size_t)(K + 1) * m * m);
    int steps = 0;
    for (int j = 0; j < K; ++j) {
        double2* Vj = V.p + (int64_t)j * nm;
        double2* Zj = Z.p + (int64_t)j * nm;
        M(Vj, Zj);
        A(Zj, W.p);
        std::vector<cd> hc((size_t)(j + 1) * m * m, cd(0.0));  // (j+1)m x m, row-major
        ortho([&] {
            for (int pass = 0; pass < 2; ++pass) {
                block_dots(V.p, j + 1, W.p, coef.p, st);
                block_update(W.p, V.p, j + 1, coef.p, -1.0, 1.0, st);
                MWI_CUDA(cudaMemcpyAsync(ch.data(), coef.p, (size_t)(j + 1) * m * m * sizeof(double2),
                                         cudaMemcpyDeviceToHost, st));
                MWI_CUDA(cudaStreamSynchronize(st));
                for (size_t i = 0; i < hc.size(); ++i) hc[i] += to_cd(ch[i]);
            }
            ndef += chol_qr(W.p, S, st);
        });
        MWI_CUDA(cudaMemcpyAsync(V.p + (int64_t)(j + 1) * nm, W.p, nm * sizeof(double2), cudaMemcpyDeviceToDevice,
                                 st));
        // new Hessenberg columns j m + c: rows < (j+1) m from the Gram-Schmidt
        // coefficients, rows (j+1) m + a from S
        for (int c = 0; c < m; ++c) {
            const int col = j * m + c;
            cd* h = &H[(size_t)col * ld];
            for (int r = 0; r < (j + 1) * m; ++r) h[r] = hc[(size_t)r * m + c];
            for (int a = 0; a < m; ++a) h[(j + 1) * m + a] = S[a * m + c];
            for (const Rot& R : rots) {
                const cd u = h[R.p], v = h[R.q];
                h[R.p] = R.c * u + R.s * v;
                h[R.q] = -std::conj(R.s) * u + std::conj(R.c) * v;
            }
            // zero rows col+1 .. col+m against the diagonal
            for (int q = col + 1; q <= col + m; ++q) {
                const cd a = h[col], b = h[q];
                const double den = std::sqrt(std::norm(a) + std::norm(b));
                Rot R{col, q, cd(1.0), cd(0.0)};
                if (den > 0.0) {
                    R.c = std::conj(a) / den;
                    R.s = std::conj(b) / den;
                }
                h[col] = R.c * a + R.s * b;
                h[q] = 0.0;
                for (int bb = 0; bb < m; ++bb) {
                    cd* g = &G[(size_t)bb * ld];
                    const cd u = g[R.p], v = g[R.q];
                    g[R.p] = R.c * u + R.s * v;
                    g[R.q] = -std::conj(R.s) * u + std::conj(R.c) * v;
                }
                rots.push_back(R);
            }
        }
        steps = j + 1;
        bool done = true;
        for (int b = 0; b < m; ++b) {
            double s2 = 0.0;
            for (int a = 0; a < m; ++a) s2 += std::norm(G[(size_t)b * ld + (j + 1) * m + a]);
            if (resid_est) resid_est[b] = std::sqrt(s2);
            if (std::sqrt(s2) > tol[b]) done = false;
        }
        if (done) break;
    }
    // back substitution R Y = G[0 : steps m]; a zero diagonal (deflated
    // direction) leaves its unknown at zero
    const int nk = steps * m;
    std::vector<cd> Y((size_t)nk * m, cd(0.0));  // row-major nk x m
    for (int b = 0; b < m; ++b) {
        for (int i = nk - 1; i >= 0; --i) {
            const cd d = H[(size_t)i * ld + i];
            if (std::abs(d) == 0.0) continue;
            cd t = G[(size_t)b * ld + i];
            for (int k = i + 1; k < nk; ++k) t -= H[(size_t)k * ld + i] * Y[(size_t)k * m + b];
            Y[(size_t)i * m + b] = t / d;
        }
    }
    std::vector<double2> yh((size_t)nk * m);
    for (size_t i = 0; i < yh.size(); ++i) yh[i] = to_d2(Y[i]);
    MWI_CUDA(cudaMemcpyAsync(coef.p, yh.data(), yh.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    ortho([&] { block_update(x, Z.p, steps, coef.p, 1.0, 1.0, st); });
    MWI_CUDA(cudaStreamSynchronize(st));  // yh goes out of scope
    if (deflated) *deflated = ndef;
    return steps;
}

}  // namespace mwi

// Right-hand sides, S-parameters, misfit, adjoint source and the per-tet
// gradient (Sections 4 and 5).
//
// RHS of transmitter j (edge-current dipole on edge k_j, sign s_j):
//     b_j = -i omega mu0 I_j s_j e_{k_j}.
// S-parameters with receiver weight q_i = s_i e_{k_i} (|q_i| = 1), Eq. sij:
//     S_ij = conj(s_i u_j[k_i]).
// Misfit, Eq. defJ with weights w:  J = 1/2 sum_ij w_ij |S_ij - S^mes_ij|^2.
// Adjoint source (discrete Eq. pbadj):  g_j = sum_i w_ij r_ij s_i e_{k_i}.
// Gradient (Section 5, DJ = Re int conj(dk) sum_j conj(E_j . F_j) in
// discrete form, plus the boundary term of beta = k0 sqrt(eps_t)):
//     G_t = sum_j lam_{j,t}^T (k0^2 M_t - i k0 / (2 sqrt(eps_t)) B_t) u_{j,t},
//     dJ/dRe(eps_t) + i dJ/dIm(eps_t) = conj(G_t).
#include "common.h"
#include "df.h"
#include "physics.h"

namespace mwi {

__global__ void rhs_kernel(int m, const int32_t* __restrict__ dof, const double* __restrict__ sign,
                           const double2* __restrict__ cur, double omega_mu0, double2* __restrict__ B) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double2 I = cur[j];
    // -i * omega mu0 * I * s
    const double s = sign[j] * omega_mu0;
    B[(int64_t)dof[j] * m + j] = make_double2(I.y * s, -I.x * s);
}

__global__ void s_extract_kernel(int n_rx, int m, const int32_t* __restrict__ dof, const double* __restrict__ sign,
                                 const double2* __restrict__ U, double2* __restrict__ S) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_rx * m) return;
    const int i = e % n_rx, j = e / n_rx;
    const double2 u = U[(int64_t)dof[i] * m + j];
    S[e] = make_double2(sign[i] * u.x, -sign[i] * u.y);
}

// one block: r = S - S_meas, J = 1/2 sum w |r|^2 (fixed reduction order)
__global__ void misfit_kernel(int cnt, const double2* __restrict__ S, const double2* __restrict__ Sm,
                              const double* __restrict__ w, double2* __restrict__ r, double* __restrict__ J) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int e = threadIdx.x; e < cnt; e += 256) {
        double2 d = make_double2(S[e].x - Sm[e].x, S[e].y - Sm[e].y);
        r[e] = d;
        const double we = w ? w[e] : 1.0;
        acc += we * (d.x * d.x + d.y * d.y);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J = 0.5 * red[0];
}

__global__ void adjoint_rhs_kernel(int n_rx, int m, const int32_t* __restrict__ dof, const double* __restrict__ sign,
                                   const double2* __restrict__ r, const double* __restrict__ w,
                                   double2* __restrict__ G) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    for (int i = 0; i < n_rx; ++i) {
        const int e = i + n_rx * j;
        const double we = (w ? w[e] : 1.0) * sign[i];
        double2& g = G[(int64_t)dof[i] * m + j];
        g.x += we * r[e].x;
        g.y += we * r[e].y;
    }
}

template <int NL, int NLF>
__global__ void __launch_bounds__(256) gradient_kernel(
    int64_t nt, int m, const int32_t* __restrict__ tet_dofs, const int32_t* __restrict__ tet_faces,
    const int8_t* __restrict__ face_tag, const int32_t* __restrict__ face_dofs, const double* __restrict__ Mp,
    const double* __restrict__ Bf, const double2* __restrict__ eps, double k0, const double2* __restrict__ U,
    const double2* __restrict__ Lam, double2* __restrict__ out) {
    constexpr int NP = NL * (NL + 1) / 2;
    constexpr int NPF = NLF * (NLF + 1) / 2;
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= nt) return;
    int dofs[NL];
#pragma unroll
    for (int a = 0; a < NL; ++a) dofs[a] = tet_dofs[t * NL + a];
    const double* M = Mp + t * NP;
    // faces owned by this tet that carry the impedance term
    int ff[4], nff = 0;
#pragma unroll
    for (int lf = 0; lf < 4; ++lf) {
        const int f = tet_faces[t * 4 + lf];
        if (face_tag[f] == 2) ff[nff++] = f;
    }
    double vr = 0.0, vi = 0.0;      // volume sum
    double br = 0.0, bi = 0.0;      // boundary sum
    for (int c = lane; c < m; c += 32) {
        double2 u[NL], l[NL];
#pragma unroll
        for (int a = 0; a < NL; ++a) {
            if (dofs[a] >= 0) {
                u[a] = U[(int64_t)dofs[a] * m + c];
                l[a] = Lam[(int64_t)dofs[a] * m + c];
            } else {
                u[a] = make_double2(0.0, 0.0);
                l[a] = make_double2(0.0, 0.0);
            }
        }
#pragma unroll
        for (int a = 0; a < NL; ++a) {
            double2 mu = make_double2(0.0, 0.0);
#pragma unroll
            for (int b = 0; b < NL; ++b) {
                const int ia = a < b ? a : b, ib = a < b ? b : a;
                const double mab = M[ia * NL - ia * (ia - 1) / 2 + (ib - ia)];
                mu.x += mab * u[b].x;
                mu.y += mab * u[b].y;
            }
            vr += l[a].x * mu.x - l[a].y * mu.y;
            vi += l[a].x * mu.y + l[a].y * mu.x;
        }
        for (int q = 0; q < nff; ++q) {
            const int f = ff[q];
            double2 uf[NLF], lf_[NLF];
#pragma unroll
            for (int a = 0; a < NLF; ++a) {
                const int d = face_dofs[(int64_t)f * NLF + a];
                uf[a] = d >= 0 ? U[(int64_t)d * m + c] : make_double2(0.0, 0.0);
                lf_[a] = d >= 0 ? Lam[(int64_t)d * m + c] : make_double2(0.0, 0.0);
            }
            const double* Bp = Bf + (int64_t)f * NPF;
#pragma unroll
            for (int a = 0; a < NLF; ++a) {
                double2 bu = make_double2(0.0, 0.0);
#pragma unroll
                for (int b = 0; b < NLF; ++b) {
                    const int ia = a < b ? a : b, ib = a < b ? b : a;
                    const double bab = Bp[ia * NLF - ia * (ia - 1) / 2 + (ib - ia)];
                    bu.x += bab * uf[b].x;
                    bu.y += bab * uf[b].y;
                }
                br += lf_[a].x * bu.x - lf_[a].y * bu.y;
                bi += lf_[a].x * bu.y + lf_[a].y * bu.x;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
        br += __shfl_xor_sync(0xffffffffu, br, o);
        bi += __shfl_xor_sync(0xffffffffu, bi, o);
    }
    if (lane == 0) {
        double gr = k0 * k0 * vr, gi = k0 * k0 * vi;
        if (nff > 0) {
            // coef = -i k0 / (2 sqrt(eps))
            const double2 e = eps[t];
            const double r = sqrt(e.x * e.x + e.y * e.y);
            double sx = sqrt(0.5 * (r + e.x)), sy = sqrt(0.5 * (r - e.x));
            if (e.y < 0) sy = -sy;
            const double den = 2.0 * (sx * sx + sy * sy);
            // 1/(2 sqrt(eps)) = (sx - i sy) / (2 |sqrt eps|^2);  times -i k0
            const double cr = -k0 * sy / den;
            const double ci = -k0 * sx / den;
            gr += cr * br - ci * bi;
            gi += cr * bi + ci * br;
        }
        out[t] = make_double2(gr, -gi);
    }
}

// The same gradient for the mixed path and first order with the volume term in
// double-float arithmetic on the FP32 pipes (FP64 runs at 1/64 of the FP32
// rate, and the FP64 form of this kernel is bound by it): U and Lam as
// double-float planes (hi at [0, nm), lo at [nm, 2 nm), complex pairs), the
// element masses as double-float pairs Mdf [nt][21] (split once per mesh), the
// sums over the transmitters and across the warp in double-float, one join to
// FP64 per tet.  The boundary term (impedance faces only) stays in FP64.
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    dfl r;
    quick_two_sum(s, e + (a.l + b.l), r.h, r.l);
    return r;
}

__global__ void __launch_bounds__(256, 2) gradient_df_kernel(
    int64_t nt, int m, int64_t nm, const int32_t* __restrict__ tet_dofs, const int32_t* __restrict__ tet_faces,
    const int8_t* __restrict__ face_tag, const int32_t* __restrict__ face_dofs, const float2* __restrict__ Mdf,
    const double* __restrict__ Bf, const double2* __restrict__ eps, double k0, const double2* __restrict__ U,
    const double2* __restrict__ Lam, const float2* __restrict__ Udf, const float2* __restrict__ Ldf,
    double2* __restrict__ out) {
    constexpr int NL = 6, NLF = 3, NP = 21, NPF = 6;
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= nt) return;
    int dofs[NL];
#pragma unroll
    for (int a = 0; a < NL; ++a) dofs[a] = tet_dofs[t * NL + a];
    int ff[4], nff = 0;
#pragma unroll
    for (int lf = 0; lf < 4; ++lf) {
        const int f = tet_faces[t * 4 + lf];
        if (face_tag[f] == 2) ff[nff++] = f;
    }
    const float2* Mt = Mdf + t * NP;
    dfl vr = {0.f, 0.f}, vi = {0.f, 0.f};  // volume sum
    double br = 0.0, bi = 0.0;             // boundary sum
    for (int c = lane; c < m; c += 32) {
        float2 uh[NL], ul[NL], lh[NL], ll[NL];
#pragma unroll
        for (int a = 0; a < NL; ++a) {
            uh[a] = ul[a] = lh[a] = ll[a] = make_float2(0.f, 0.f);
            if (dofs[a] >= 0) {
                const int64_t e = (int64_t)dofs[a] * m + c;
                uh[a] = Udf[e];
                ul[a] = Udf[nm + e];
                lh[a] = Ldf[e];
                ll[a] = Ldf[nm + e];
            }
        }
#pragma unroll
        for (int a = 0; a < NL; ++a) {
            dfl mr = {0.f, 0.f}, mi = {0.f, 0.f};  // (M u)_a
#pragma unroll
            for (int b = 0; b < NL; ++b) {
                const int ia = a < b ? a : b, ib = a < b ? b : a;
                const float2 mab = Mt[ia * NL - ia * (ia - 1) / 2 + (ib - ia)];
                df_mac(mr, mab.x, mab.y, uh[b].x, ul[b].x);
                df_mac(mi, mab.x, mab.y, uh[b].y, ul[b].y);
            }
            mr = df_norm(mr);
            mi = df_norm(mi);
            // v += lam_a (M u)_a
            df_mac(vr, lh[a].x, ll[a].x, mr.h, mr.l);
            df_mac(vr, -lh[a].y, -ll[a].y, mi.h, mi.l);
            df_mac(vi, lh[a].x, ll[a].x, mi.h, mi.l);
            df_mac(vi, lh[a].y, ll[a].y, mr.h, mr.l);
        }
        for (int q = 0; q < nff; ++q) {
            const int f = ff[q];
            double2 uf[NLF], lf_[NLF];
#pragma unroll
            for (int a = 0; a < NLF; ++a) {
                const int d = face_dofs[(int64_t)f * NLF + a];
                uf[a] = d >= 0 ? U[(int64_t)d * m + c] : make_double2(0.0, 0.0);
                lf_[a] = d >= 0 ? Lam[(int64_t)d * m + c] : make_double2(0.0, 0.0);
            }
            const double* Bp = Bf + (int64_t)f * NPF;
#pragma unroll
            for (int a = 0; a < NLF; ++a) {
                double2 bu = make_double2(0.0, 0.0);
#pragma unroll
                for (int b = 0; b < NLF; ++b) {
                    const int ia = a < b ? a : b, ib = a < b ? b : a;
                    const double bab = Bp[ia * NLF - ia * (ia - 1) / 2 + (ib - ia)];
                    bu.x += bab * uf[b].x;
                    bu.y += bab * uf[b].y;
                }
                br += lf_[a].x * bu.x - lf_[a].y * bu.y;
                bi += lf_[a].x * bu.y + lf_[a].y * bu.x;
            }
        }
    }
    vr = df_norm(vr);
    vi = df_norm(vi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dfl xr, xi;
        xr.h = __shfl_xor_sync(0xffffffffu, vr.h, o);
        xr.l = __shfl_xor_sync(0xffffffffu, vr.l, o);
        xi.h = __shfl_xor_sync(0xffffffffu, vi.h, o);
        xi.l = __shfl_xor_sync(0xffffffffu, vi.l, o);
        vr = df_add(vr, xr);
        vi = df_add(vi, xi);
    }
    if (nff > 0) {  // the same for every lane of the warp (one tet)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            br += __shfl_xor_sync(0xffffffffu, br, o);
            bi += __shfl_xor_sync(0xffffffffu, bi, o);
        }
    }
    if (lane == 0) {
        const double k2 = k0 * k0;
        double gr = k2 * df_join(vr.h, vr.l), gi = k2 * df_join(vi.h, vi.l);
        if (nff > 0) {
            // coef = -i k0 / (2 sqrt(eps))
            const double2 e = eps[t];
            const double r = sqrt(e.x * e.x + e.y * e.y);
            double sx = sqrt(0.5 * (r + e.x)), sy = sqrt(0.5 * (r - e.x));
            if (e.y < 0) sy = -sy;
            const double den = 2.0 * (sx * sx + sy * sy);
            const double cr = -k0 * sy / den;
            const double ci = -k0 * sx / den;
            gr += cr * br - ci * bi;
            gi += cr * bi + ci * br;
        }
        out[t] = make_double2(gr, -gi);
    }
}

// double-float pairs of a real array
__global__ void split_real_kernel(int64_t count, const double* __restrict__ a, float2* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) out[e] = df_split(a[e]);
}

static inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

void launch_split_real(int64_t count, const double* a, float2* out, cudaStream_t st) {
    split_real_kernel<<<nblk(count, 256), 256, 0, st>>>(count, a, out);
    MWI_CHECK_LAUNCH();
}

void launch_gradient_df(int64_t nt, int m, int64_t nm, const int32_t* tet_dofs, const int32_t* tet_faces,
                        const int8_t* face_tag, const int32_t* face_dofs, const float2* Mdf, const double* Bf,
                        const double2* eps, double k0, const double2* U, const double2* Lam, const float2* Udf,
                        const float2* Ldf, double2* out, cudaStream_t st) {
    gradient_df_kernel<<<nblk(nt * 32, 256), 256, 0, st>>>(nt, m, nm, tet_dofs, tet_faces, face_tag, face_dofs, Mdf,
                                                           Bf, eps, k0, U, Lam, Udf, Ldf, out);
    MWI_CHECK_LAUNCH();
}

void launch_rhs(int m, const int32_t* dof, const double* sign, const double2* cur, double omega_mu0, double2* B,
                cudaStream_t st) {
    rhs_kernel<<<nblk(m, 128), 128, 0, st>>>(m, dof, sign, cur, omega_mu0, B);
    MWI_CHECK_LAUNCH();
}
void launch_s_extract(int n_rx, int m, const int32_t* dof, const double* sign, const double2* U, double2* S,
                      cudaStream_t st) {
    s_extract_kernel<<<nblk((int64_t)n_rx * m, 128), 128, 0, st>>>(n_rx, m, dof, sign, U, S);
    MWI_CHECK_LAUNCH();
}
void launch_misfit(int cnt, const double2* S, const double2* Sm, const double* w, double2* r, double* J,
                   cudaStream_t st) {
    misfit_kernel<<<1, 256, 0, st>>>(cnt, S, Sm, w, r, J);
    MWI_CHECK_LAUNCH();
}
void launch_adjoint_rhs(int n_rx, int m, const int32_t* dof, const double* sign, const double2* r, const double* w,
                        double2* G, cudaStream_t st) {
    adjoint_rhs_kernel<<<nblk(m, 128), 128, 0, st>>>(n_rx, m, dof, sign, r, w, G);
    MWI_CHECK_LAUNCH();
}
void launch_gradient(int order, int64_t nt, int m, const int32_t* tet_dofs, const int32_t* tet_faces,
                     const int8_t* face_tag, const int32_t* face_dofs, const double* Mp, const double* Bf,
                     const double2* eps, double k0, const double2* U, const double2* Lam, double2* out,
                     cudaStream_t st) {
    const int th = 256;
    const unsigned blocks = nblk(nt * 32, th);
    if (order == 1)
        gradient_kernel<6, 3><<<blocks, th, 0, st>>>(nt, m, tet_dofs, tet_faces, face_tag, face_dofs, Mp, Bf, eps,
                                                     k0, U, Lam, out);
    else
        gradient_kernel<20, 8><<<blocks, th, 0, st>>>(nt, m, tet_dofs, tet_faces, face_tag, face_dofs, Mp, Bf, eps,
                                                      k0, U, Lam, out);
    MWI_CHECK_LAUNCH();
}

}  // namespace mwi

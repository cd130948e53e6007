// Nodal (P1) permittivity parameter with a gradient penalty (the piecewise
// linear parameter of Section 6.3 and the regularised, normalised misfit of
// Eq. defJ2).  kappa(x) = sum_v kappa_v lambda_v(x) varies inside every tet:
//   mass term  int_t kappa N_i . N_j = sum_w kappa_{v_w(t)} M_t^(w)[i, j],
//              M_t^(w) = int_t lambda_w N_i . N_j   (vertex-weighted masses)
//   beta on impedance faces and the interface wavenumber of the local
//   problems use the P1 field at the owning tet's centroid,
//              kappa_bar_t = 1/4 sum_w kappa_{v_w(t)}
//   gradient   G_v = sum over the (tet, local vertex) pairs of v of
//              k0^2 sum_j lam_{j,t}^T M_t^(w) u_{j,t}
//              + 1/4 sum_j lam_{j,t}^T (-i k0 / (2 sqrt(kappa_bar_t))) B_t u_{j,t}
//   penalty    R = (alpha / 2) Re(kappa^H K kappa),  K the P1 stiffness matrix
//   returned   dPhi/dRe kappa_v + i dPhi/dIm kappa_v = conj(G_v) + alpha (K kappa)_v.
// Every sum runs in a fixed order (a vertex's tets ascending), so the results
// are deterministic.
#include <algorithm>

#include "common.h"
#include "df.h"
#include "kernels.h"
#include "model.h"

namespace mwi {

__global__ void p1_centroid_kernel(int64_t nt, const int32_t* __restrict__ tv, const double2* __restrict__ kappa,
                                   double2* __restrict__ eps) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int32_t* v = tv + 4 * t;
    double2 s = kappa[v[0]];
#pragma unroll
    for (int a = 1; a < 4; ++a) {
        const double2 k = kappa[v[a]];
        s.x += k.x;
        s.y += k.y;
    }
    eps[t] = make_double2(0.25 * s.x, 0.25 * s.y);
}

// Mk[t][p] = sum_w kappa_{v_w(t)} Mv[t][w][p], one thread per (tet, pair)
__global__ void p1_mass_kernel(int64_t nt, int npack, const int32_t* __restrict__ tv,
                               const double2* __restrict__ kappa, const double* __restrict__ Mv,
                               double2* __restrict__ Mk) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nt * npack) return;
    const int64_t t = e / npack;
    const int p = (int)(e - t * npack);
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const double2 k = kappa[tv[4 * t + w]];
        const double m = Mv[(t * 4 + w) * npack + p];
        acc.x += k.x * m;
        acc.y += k.y * m;
    }
    Mk[e] = acc;
}

// one warp per tet: the four (tet, vertex) gradient terms, reduced over the
// m columns (lanes take columns, fixed shuffle order)
template <int NL, int NLF>
__global__ void __launch_bounds__(256) p1_tet_gradient_kernel(
    int64_t nt, int m, const int32_t* __restrict__ tet_dofs, const int32_t* __restrict__ tet_faces,
    const int8_t* __restrict__ face_tag, const int32_t* __restrict__ face_dofs, const double* __restrict__ Mv,
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
    const double* M = Mv + t * 4 * NP;
    int ff[4], nff = 0;
#pragma unroll
    for (int lf = 0; lf < 4; ++lf) {
        const int f = tet_faces[t * 4 + lf];
        if (face_tag[f] == 2) ff[nff++] = f;
    }
    double vr[4] = {0.0, 0.0, 0.0, 0.0}, vi[4] = {0.0, 0.0, 0.0, 0.0};
    double br = 0.0, bi = 0.0;
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
        for (int w = 0; w < 4; ++w) {
#pragma unroll
            for (int a = 0; a < NL; ++a) {
                double2 mu = make_double2(0.0, 0.0);
#pragma unroll
                for (int b = 0; b < NL; ++b) {
                    const int ia = a < b ? a : b, ib = a < b ? b : a;
                    const double mab = M[w * NP + ia * NL - ia * (ia - 1) / 2 + (ib - ia)];
                    mu.x += mab * u[b].x;
                    mu.y += mab * u[b].y;
                }
                vr[w] += l[a].x * mu.x - l[a].y * mu.y;
                vi[w] += l[a].x * mu.y + l[a].y * mu.x;
            }
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
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            vr[w] += __shfl_xor_sync(0xffffffffu, vr[w], o);
            vi[w] += __shfl_xor_sync(0xffffffffu, vi[w], o);
        }
        br += __shfl_xor_sync(0xffffffffu, br, o);
        bi += __shfl_xor_sync(0xffffffffu, bi, o);
    }
    if (lane == 0) {
        // 1/4 of the beta term: coef = -i k0 / (2 sqrt(kappa_bar_t))
        double qr = 0.0, qi = 0.0;
        if (nff > 0) {
            const double2 e = eps[t];
            const double r = sqrt(e.x * e.x + e.y * e.y);
            double sx = sqrt(0.5 * (r + e.x)), sy = sqrt(0.5 * (r - e.x));
            if (e.y < 0) sy = -sy;
            const double den = 2.0 * (sx * sx + sy * sy);
            const double cr = -k0 * sy / den;
            const double ci = -k0 * sx / den;
            qr = 0.25 * (cr * br - ci * bi);
            qi = 0.25 * (cr * bi + ci * br);
        }
#pragma unroll
        for (int w = 0; w < 4; ++w)
            out[4 * t + w] = make_double2(k0 * k0 * vr[w] + qr, -(k0 * k0 * vi[w] + qi));
    }
}

// per vertex: the (tet, vertex) gradients of its tets in ascending tet order plus
// alpha K kappa; per block, the fixed-order sum of Re(conj(kappa_v) (K kappa)_v)
__global__ void __launch_bounds__(256) p1_gradient_kernel(int64_t nv, const int32_t* __restrict__ v2t_ptr,
                                                          const int32_t* __restrict__ v2t,
                                                          const int32_t* __restrict__ tv,
                                                          const double2* __restrict__ grad_tw,
                                                          const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double2* __restrict__ kappa, double alpha,
                                                          double2* __restrict__ out, double* __restrict__ partial) {
    __shared__ double red[256];
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (v < nv) {
        double2 g = make_double2(0.0, 0.0);
        for (int32_t q = v2t_ptr[v]; q < v2t_ptr[v + 1]; ++q) {
            const int64_t t = v2t[q];
            int w = 0;
            while (w < 3 && tv[4 * t + w] != (int32_t)v) ++w;
            const double2 x = grad_tw[4 * t + w];
            g.x += x.x;
            g.y += x.y;
        }
        double2 kk = make_double2(0.0, 0.0);
        for (int32_t q = rp[v]; q < rp[v + 1]; ++q) {
            const double2 x = kappa[col[q]];
            kk.x += val[q] * x.x;
            kk.y += val[q] * x.y;
        }
        out[v] = make_double2(g.x + alpha * kk.x, g.y + alpha * kk.y);
        const double2 kv = kappa[v];
        e = kv.x * kk.x + kv.y * kk.y;
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// counts entries with a non-finite real or imaginary part
__global__ void count_nonfinite_kernel(int64_t n, const double2* __restrict__ x, int* __restrict__ count) {
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        bad += (isfinite(v.x) && isfinite(v.y)) ? 0 : 1;
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, bad);
}

void build_p1_stiffness(const Topology& T, std::vector<int32_t>& rp, std::vector<int32_t>& col,
                        std::vector<double>& val) {
    const int64_t nv = T.nv, nt = T.nt;
    // element matrices |t| grad(lambda_a) . grad(lambda_b)
    std::vector<double> Ke((size_t)nt * 16);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* v = &T.tv[4 * t];
        double E[3][3];  // columns x_k - x_0
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d) E[d][k] = T.xyz[3 * (int64_t)v[k + 1] + d] - T.xyz[3 * (int64_t)v[0] + d];
        const double det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
                           E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                           E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
        MWI_REQUIRE(det != 0.0, MWI_EINVAL, "degenerate tet");
        // rows of E^{-1} are the gradients of the barycentrics 1..3
        double G[4][3];
        const double id = 1.0 / det;
        const double inv[3][3] = {
            {(E[1][1] * E[2][2] - E[1][2] * E[2][1]) * id, (E[0][2] * E[2][1] - E[0][1] * E[2][2]) * id,
             (E[0][1] * E[1][2] - E[0][2] * E[1][1]) * id},
            {(E[1][2] * E[2][0] - E[1][0] * E[2][2]) * id, (E[0][0] * E[2][2] - E[0][2] * E[2][0]) * id,
             (E[0][2] * E[1][0] - E[0][0] * E[1][2]) * id},
            {(E[1][0] * E[2][1] - E[1][1] * E[2][0]) * id, (E[0][1] * E[2][0] - E[0][0] * E[2][1]) * id,
             (E[0][0] * E[1][1] - E[0][1] * E[1][0]) * id}};
        for (int d = 0; d < 3; ++d) {
            G[0][d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
            for (int k = 0; k < 3; ++k) G[k + 1][d] = inv[k][d];
        }
        const double vol = std::fabs(det) / 6.0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                Ke[16 * t + 4 * a + b] = vol * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
    }
    // rows: each vertex's tets in ascending order, entries merged by column
    rp.assign(nv + 1, 0);
    col.clear();
    val.clear();
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t v = 0; v < nv; ++v) {
        row.clear();
        for (int32_t q = T.v2t_ptr[v]; q < T.v2t_ptr[v + 1]; ++q) {
            const int64_t t = T.v2t[q];
            int a = 0;
            while (T.tv[4 * t + a] != v) ++a;
            for (int b = 0; b < 4; ++b) row.emplace_back(T.tv[4 * t + b], Ke[16 * t + 4 * a + b]);
        }
        std::stable_sort(row.begin(), row.end(),
                         [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
                             return x.first < y.first;
                         });
        for (size_t i = 0; i < row.size();) {
            const int32_t c = row[i].first;
            double s = 0.0;
            for (; i < row.size() && row[i].first == c; ++i) s += row[i].second;
            col.push_back(c);
            val.push_back(s);
        }
        rp[v + 1] = (int32_t)col.size();
    }
}

void launch_p1_centroid(int64_t nt, const int32_t* tv, const double2* kappa, double2* eps, cudaStream_t st) {
    p1_centroid_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, tv, kappa, eps);
    MWI_CHECK_LAUNCH();
}

void launch_p1_mass(int64_t nt, int npack, const int32_t* tv, const double2* kappa, const double* Mv, double2* Mk,
                    cudaStream_t st) {
    const int64_t n = nt * npack;
    p1_mass_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nt, npack, tv, kappa, Mv, Mk);
    MWI_CHECK_LAUNCH();
}

// The same (tet, vertex) gradient terms for the mixed path and first order
// with the volume terms in double-float on the FP32 pipes (the FP64 form is
// bound by the FP64 rate): U and Lam as double-float planes ([2][nm] complex
// pairs), the vertex-weighted masses as double-float pairs Mvdf [nt][4][21]
// (split once per mesh), one join to FP64 per (tet, vertex).  The boundary term
// stays in FP64.
__device__ __forceinline__ dfl p1_df_add(dfl a, dfl b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    dfl r;
    quick_two_sum(s, e + (a.l + b.l), r.h, r.l);
    return r;
}

__global__ void __launch_bounds__(256) p1_tet_gradient_df_kernel(
    int64_t nt, int m, int64_t nm, const int32_t* __restrict__ tet_dofs, const int32_t* __restrict__ tet_faces,
    const int8_t* __restrict__ face_tag, const int32_t* __restrict__ face_dofs, const float2* __restrict__ Mvdf,
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
    const float2* Mt = Mvdf + t * 4 * NP;
    int ff[4], nff = 0;
#pragma unroll
    for (int lf = 0; lf < 4; ++lf) {
        const int f = tet_faces[t * 4 + lf];
        if (face_tag[f] == 2) ff[nff++] = f;
    }
    dfl vr[4], vi[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) vr[w] = vi[w] = dfl{0.f, 0.f};
    double br = 0.0, bi = 0.0;
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
            // (M^(w) u)_a for the four vertices w, then lam_a times each
            dfl mr[4], mi[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) mr[w] = mi[w] = dfl{0.f, 0.f};
#pragma unroll
            for (int b = 0; b < NL; ++b) {
                const int ia = a < b ? a : b, ib = a < b ? b : a;
                const int q = ia * NL - ia * (ia - 1) / 2 + (ib - ia);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const float2 mab = Mt[w * NP + q];
                    df_mac(mr[w], mab.x, mab.y, uh[b].x, ul[b].x);
                    df_mac(mi[w], mab.x, mab.y, uh[b].y, ul[b].y);
                }
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const dfl r = df_norm(mr[w]), i = df_norm(mi[w]);
                df_mac(vr[w], lh[a].x, ll[a].x, r.h, r.l);
                df_mac(vr[w], -lh[a].y, -ll[a].y, i.h, i.l);
                df_mac(vi[w], lh[a].x, ll[a].x, i.h, i.l);
                df_mac(vi[w], lh[a].y, ll[a].y, r.h, r.l);
            }
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
    for (int w = 0; w < 4; ++w) {
        vr[w] = df_norm(vr[w]);
        vi[w] = df_norm(vi[w]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            dfl xr, xi;
            xr.h = __shfl_xor_sync(0xffffffffu, vr[w].h, o);
            xr.l = __shfl_xor_sync(0xffffffffu, vr[w].l, o);
            xi.h = __shfl_xor_sync(0xffffffffu, vi[w].h, o);
            xi.l = __shfl_xor_sync(0xffffffffu, vi[w].l, o);
            vr[w] = p1_df_add(vr[w], xr);
            vi[w] = p1_df_add(vi[w], xi);
        }
    }
    if (nff > 0) {  // the same for every lane of the warp (one tet)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            br += __shfl_xor_sync(0xffffffffu, br, o);
            bi += __shfl_xor_sync(0xffffffffu, bi, o);
        }
    }
    if (lane == 0) {
        // 1/4 of the beta term: coef = -i k0 / (2 sqrt(kappa_bar_t))
        double qr = 0.0, qi = 0.0;
        if (nff > 0) {
            const double2 e = eps[t];
            const double r = sqrt(e.x * e.x + e.y * e.y);
            double sx = sqrt(0.5 * (r + e.x)), sy = sqrt(0.5 * (r - e.x));
            if (e.y < 0) sy = -sy;
            const double den = 2.0 * (sx * sx + sy * sy);
            const double cr = -k0 * sy / den;
            const double ci = -k0 * sx / den;
            qr = 0.25 * (cr * br - ci * bi);
            qi = 0.25 * (cr * bi + ci * br);
        }
        const double k2 = k0 * k0;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            out[4 * t + w] = make_double2(k2 * df_join(vr[w].h, vr[w].l) + qr,
                                          -(k2 * df_join(vi[w].h, vi[w].l) + qi));
    }
}

void launch_p1_tet_gradient_df(int64_t nt, int m, int64_t nm, const int32_t* tet_dofs, const int32_t* tet_faces,
                               const int8_t* face_tag, const int32_t* face_dofs, const float2* Mvdf,
                               const double* Bf, const double2* eps, double k0, const double2* U, const double2* Lam,
                               const float2* Udf, const float2* Ldf, double2* out_tw, cudaStream_t st) {
    const int th = 256;
    const unsigned blocks = (unsigned)((nt * 32 + th - 1) / th);
    p1_tet_gradient_df_kernel<<<blocks, th, 0, st>>>(nt, m, nm, tet_dofs, tet_faces, face_tag, face_dofs, Mvdf, Bf,
                                                     eps, k0, U, Lam, Udf, Ldf, out_tw);
    MWI_CHECK_LAUNCH();
}

void launch_p1_tet_gradient(int order, int64_t nt, int m, const int32_t* tet_dofs, const int32_t* tet_faces,
                            const int8_t* face_tag, const int32_t* face_dofs, const double* Mv, const double* Bf,
                            const double2* eps, double k0, const double2* U, const double2* Lam, double2* out_tw,
                            cudaStream_t st) {
    const int th = 256;
    const unsigned blocks = (unsigned)((nt * 32 + th - 1) / th);
    if (order == 1)
        p1_tet_gradient_kernel<6, 3><<<blocks, th, 0, st>>>(nt, m, tet_dofs, tet_faces, face_tag, face_dofs, Mv, Bf,
                                                            eps, k0, U, Lam, out_tw);
    else
        p1_tet_gradient_kernel<20, 8><<<blocks, th, 0, st>>>(nt, m, tet_dofs, tet_faces, face_tag, face_dofs, Mv,
                                                             Bf, eps, k0, U, Lam, out_tw);
    MWI_CHECK_LAUNCH();
}

int p1_gradient_blocks(int64_t nv) { return (int)((nv + 255) / 256); }

void launch_p1_gradient(int64_t nv, const int32_t* v2t_ptr, const int32_t* v2t, const int32_t* tv,
                        const double2* grad_tw, const int32_t* rp, const int32_t* col, const double* val,
                        const double2* kappa, double alpha, double2* out, double* partial, cudaStream_t st) {
    p1_gradient_kernel<<<p1_gradient_blocks(nv), 256, 0, st>>>(nv, v2t_ptr, v2t, tv, grad_tw, rp, col, val, kappa,
                                                               alpha, out, partial);
    MWI_CHECK_LAUNCH();
}

void launch_count_nonfinite(int64_t n, const double2* x, int* count, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    count_nonfinite_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, x, count);
    MWI_CHECK_LAUNCH();
}

}  // namespace mwi

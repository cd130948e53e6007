// Element integrals in closed form and the deterministic assembly of A and
// of the local operators B_i (Section 2.1, Eq. pbdirectvarf; Section 3).
//
// Every basis function is a sum of terms c * lambda^alpha * grad(lambda_g):
//   Whitney N_ab      = lambda_a grad(l_b) - lambda_b grad(l_a)
//   gradient          = lambda_a grad(l_b) + lambda_b grad(l_a)
//   face (a < b < c)  = lambda_c N_ab  and  lambda_a N_bc.
// With the Gram matrix G_kl = grad(l_k) . grad(l_l) of a tet and the exact
// moment  int_t lambda^gamma = 6 |t| gamma! / (|gamma| + 3)!,
//   M_ij = sum_pq c_p c_q G_{g_p g_q} int lambda^(alpha_p + alpha_q),
//   curl(lambda^a grad l_g) = sum_k a_k lambda^(a - e_k) grad l_k x grad l_g,
//   (x . y) of two cross products by the Binet-Cauchy identity,
// and on a face opposite vertex d (normal along grad l_d), the tangential
// inner product G_gh - G_gd G_hd / G_dd with  int_f lambda^gamma =
// 2 |f| gamma! / (|gamma| + 2)!.  The tables of terms are built once on the
// host; one thread evaluates one tet (or face).
#include <algorithm>
#include <vector>

#include "common.h"
#include "kernels.h"
#include "model.h"

namespace mwi {

namespace {

struct Term { double c; int mono[4]; int g; };

static std::vector<std::vector<Term>> basis_terms(int order) {
    std::vector<std::vector<Term>> B;
    auto e = [](int a, int b) { Term t{0, {0, 0, 0, 0}, 0}; t.mono[a]++; if (b >= 0) t.mono[b]++; return t; };
    auto whitney = [&](int a, int b, int extra) {
        Term t1 = e(a, extra); t1.c = 1; t1.g = b;
        Term t2 = e(b, extra); t2.c = -1; t2.g = a;
        return std::vector<Term>{t1, t2};
    };
    for (int k = 0; k < 6; ++k) B.push_back(whitney(kLocalEdges[k][0], kLocalEdges[k][1], -1));
    if (order == 2) {
        for (int k = 0; k < 6; ++k) {
            int a = kLocalEdges[k][0], b = kLocalEdges[k][1];
            Term t1 = e(a, -1); t1.c = 1; t1.g = b;
            Term t2 = e(b, -1); t2.c = 1; t2.g = a;
            B.push_back({t1, t2});
        }
        for (int f = 0; f < 4; ++f) {
            int a = kLocalFaces[f][0], b = kLocalFaces[f][1], c = kLocalFaces[f][2];
            B.push_back(whitney(a, b, c));
            B.push_back(whitney(b, c, a));
        }
    }
    return B;
}

static double fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }

// reference moment: gamma! / (|gamma| + extra)!
static double moment(const int* g, int extra) {
    int s = g[0] + g[1] + g[2] + g[3];
    return fact(g[0]) * fact(g[1]) * fact(g[2]) * fact(g[3]) / fact(s + extra);
}

}  // namespace

void build_element_tables(int order, ElementTables& tab) {
    const auto B = basis_terms(order);
    const int nl = (int)B.size();
    tab.nl = nl;
    tab.npack = nl * (nl + 1) / 2;
    tab.m_terms.clear();
    tab.mv_c.clear();
    tab.k_terms.clear();
    tab.m_ptr.assign(1, 0);
    tab.k_ptr.assign(1, 0);
    for (int i = 0; i < nl; ++i)
        for (int j = i; j < nl; ++j) {
            for (const Term& p : B[i])
                for (const Term& q : B[j]) {
                    int g[4];
                    for (int k = 0; k < 4; ++k) g[k] = p.mono[k] + q.mono[k];
                    MTerm t;
                    t.c = 6.0 * p.c * q.c * moment(g, 3);
                    t.a = (int8_t)p.g;
                    t.b = (int8_t)q.g;
                    tab.m_terms.push_back(t);
                    // the same term weighted by lambda_w (nodal parameter): one more power of lambda_w
                    for (int w = 0; w < 4; ++w) {
                        g[w]++;
                        tab.mv_c.push_back(6.0 * p.c * q.c * moment(g, 3));
                        g[w]--;
                    }
                }
            tab.m_ptr.push_back((int32_t)tab.m_terms.size());
            for (const Term& p : B[i])
                for (int k = 0; k < 4; ++k) {
                    if (p.mono[k] == 0) continue;
                    for (const Term& q : B[j])
                        for (int l = 0; l < 4; ++l) {
                            if (q.mono[l] == 0) continue;
                            int g[4];
                            for (int z = 0; z < 4; ++z) g[z] = p.mono[z] + q.mono[z];
                            g[k]--;
                            g[l]--;
                            KTerm t;
                            t.c = 6.0 * p.c * q.c * p.mono[k] * q.mono[l] * moment(g, 3);
                            t.k = (int8_t)k; t.gp = (int8_t)p.g; t.l = (int8_t)l; t.gq = (int8_t)q.g;
                            tab.k_terms.push_back(t);
                        }
                }
            tab.k_ptr.push_back((int32_t)tab.k_terms.size());
        }
    // face tables: per local face lf, face-local DOFs [W(ab), W(ac), W(bc) (, G(...), Fa, Fb)]
    const int nlf = order == 1 ? 3 : 8;
    tab.nlf = nlf;
    tab.npack_f = nlf * (nlf + 1) / 2;
    tab.f_terms.clear();
    tab.f_ptr.assign(1, 0);
    auto ledge = [](int a, int b) {
        for (int e2 = 0; e2 < 6; ++e2)
            if (kLocalEdges[e2][0] == a && kLocalEdges[e2][1] == b) return e2;
        return -1;
    };
    for (int lf = 0; lf < 4; ++lf) {
        const int* fl = kLocalFaces[lf];
        std::vector<int> loc = {ledge(fl[0], fl[1]), ledge(fl[0], fl[2]), ledge(fl[1], fl[2])};
        if (order == 2) {
            for (int k = 0; k < 3; ++k) loc.push_back(6 + loc[k]);
            loc.push_back(12 + 2 * lf);
            loc.push_back(13 + 2 * lf);
        }
        const int d = kOpposite[lf];
        for (int i = 0; i < nlf; ++i)
            for (int j = i; j < nlf; ++j) {
                for (const Term& p : B[loc[i]])
                    for (const Term& q : B[loc[j]]) {
                        int g[4];
                        for (int k = 0; k < 4; ++k) g[k] = p.mono[k] + q.mono[k];
                        if (g[d] != 0) continue;
                        FTerm t;
                        t.c = 2.0 * p.c * q.c * moment(g, 2);
                        t.a = (int8_t)p.g;
                        t.b = (int8_t)q.g;
                        t.d = (int8_t)d;
                        tab.f_terms.push_back(t);
                    }
                tab.f_ptr.push_back((int32_t)tab.f_terms.size());
            }
    }
}

// ---------------------------------------------------------------------------

__device__ __forceinline__ void tet_gram(const double* __restrict__ xyz, const int32_t* __restrict__ tv,
                                         int64_t t, double G[4][4], double& vol) {
    double P[4][3];
    for (int k = 0; k < 4; ++k) {
        int64_t v = tv[4 * t + k];
        for (int d = 0; d < 3; ++d) P[k][d] = xyz[3 * v + d];
    }
    double E[3][3];  // rows: edge vectors p_k - p_0
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) E[k][d] = P[k + 1][d] - P[0][d];
    // grad(lambda_k), k = 1..3: rows of the inverse-transpose, via cross products
    double c0[3] = {E[1][1] * E[2][2] - E[1][2] * E[2][1], E[1][2] * E[2][0] - E[1][0] * E[2][2],
                    E[1][0] * E[2][1] - E[1][1] * E[2][0]};
    double c1[3] = {E[2][1] * E[0][2] - E[2][2] * E[0][1], E[2][2] * E[0][0] - E[2][0] * E[0][2],
                    E[2][0] * E[0][1] - E[2][1] * E[0][0]};
    double c2[3] = {E[0][1] * E[1][2] - E[0][2] * E[1][1], E[0][2] * E[1][0] - E[0][0] * E[1][2],
                    E[0][0] * E[1][1] - E[0][1] * E[1][0]};
    double det = E[0][0] * c0[0] + E[0][1] * c0[1] + E[0][2] * c0[2];
    double gl[4][3];
    for (int d = 0; d < 3; ++d) {
        gl[1][d] = c0[d] / det;
        gl[2][d] = c1[d] / det;
        gl[3][d] = c2[d] / det;
        gl[0][d] = -(gl[1][d] + gl[2][d] + gl[3][d]);
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            G[a][b] = gl[a][0] * gl[b][0] + gl[a][1] * gl[b][1] + gl[a][2] * gl[b][2];
    vol = fabs(det) / 6.0;
}

__global__ void elem_geom_kernel(const double* __restrict__ xyz, const int32_t* __restrict__ tv, int64_t nt,
                                 const MTerm* __restrict__ mt, const int32_t* __restrict__ mptr,
                                 const KTerm* __restrict__ kt, const int32_t* __restrict__ kptr, int npack,
                                 double* __restrict__ Kout, double* __restrict__ Mout) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double G[4][4], vol;
    tet_gram(xyz, tv, t, G, vol);
    for (int p = 0; p < npack; ++p) {
        double m = 0.0;
        for (int q = mptr[p]; q < mptr[p + 1]; ++q) m += mt[q].c * G[mt[q].a][mt[q].b];
        double k = 0.0;
        for (int q = kptr[p]; q < kptr[p + 1]; ++q) {
            const KTerm& z = kt[q];
            k += z.c * (G[z.k][z.l] * G[z.gp][z.gq] - G[z.k][z.gq] * G[z.gp][z.l]);
        }
        Mout[t * npack + p] = m * vol;
        Kout[t * npack + p] = k * vol;
    }
}

// Mv[t][w][p] = |t| sum_q mv_c[4 q + w] G[a_q][b_q]: the element mass weighted by
// the barycentric lambda_w (local vertex w of the sorted tet)
__global__ void elem_vertex_mass_kernel(const double* __restrict__ xyz, const int32_t* __restrict__ tv, int64_t nt,
                                        const MTerm* __restrict__ mt, const int32_t* __restrict__ mptr,
                                        const double* __restrict__ mv_c, int npack, double* __restrict__ Mv) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double G[4][4], vol;
    tet_gram(xyz, tv, t, G, vol);
    for (int p = 0; p < npack; ++p) {
        double m[4] = {0.0, 0.0, 0.0, 0.0};
        for (int q = mptr[p]; q < mptr[p + 1]; ++q) {
            const double g = G[mt[q].a][mt[q].b];
#pragma unroll
            for (int w = 0; w < 4; ++w) m[w] += mv_c[4 * q + w] * g;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) Mv[(t * 4 + w) * npack + p] = m[w] * vol;
    }
}

__global__ void face_geom_kernel(const double* __restrict__ xyz, const int32_t* __restrict__ tv,
                                 const int32_t* __restrict__ face_tets, const int8_t* __restrict__ face_lf,
                                 int64_t nf, const FTerm* __restrict__ ft, const int32_t* __restrict__ fptr,
                                 int npack_f, double* __restrict__ Bout) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int64_t t = face_tets[2 * f];
    int lf = face_lf[2 * f];
    double G[4][4], vol;
    tet_gram(xyz, tv, t, G, vol);
    const int d = 3 - lf;
    const double area = 3.0 * vol * sqrt(G[d][d]);
    const int base = lf * npack_f;
    for (int p = 0; p < npack_f; ++p) {
        double s = 0.0;
        for (int q = fptr[base + p]; q < fptr[base + p + 1]; ++q) {
            const FTerm& z = ft[q];
            s += z.c * (G[z.a][z.b] - G[z.a][d] * G[z.b][d] / G[d][d]);
        }
        Bout[f * npack_f + p] = s * area;
    }
}

// coef[u] = i k0 sqrt(eps_t) for face use u (principal square root)
__global__ void face_coef_kernel(const int32_t* __restrict__ fu_tet, int64_t nfu, const double2* __restrict__ eps,
                                 double k0, double2* __restrict__ coef) {
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= nfu) return;
    double2 e = eps[fu_tet[u]];
    // principal sqrt of e = x + i y
    double r = sqrt(e.x * e.x + e.y * e.y);
    double sx = sqrt(0.5 * (r + e.x));
    double sy = sqrt(0.5 * (r - e.x));
    if (e.y < 0) sy = -sy;
    coef[u] = mk(-k0 * sy, k0 * sx);  // i * k0 * (sx + i sy)
}

template <typename OutC>
__global__ void slot_fill_kernel(int64_t nslots, const int64_t* __restrict__ slot_ptr,
                                 const int64_t* __restrict__ contrib, const double* __restrict__ Kp,
                                 const double* __restrict__ Mp, int npack, const double* __restrict__ Bf,
                                 int npack_f, const int32_t* __restrict__ fu_face,
                                 const double2* __restrict__ fu_coef, const double2* __restrict__ eps,
                                 const double2* __restrict__ Mk, double k0sq, double2* __restrict__ out64,
                                 OutC* __restrict__ outlo) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    double vr = 0.0, vi = 0.0;
    for (int64_t q = slot_ptr[s]; q < slot_ptr[s + 1]; ++q) {
        int64_t c = contrib[q];
        int pair = (int)(c & 0xffff);
        if (c & kFaceFlag) {
            int64_t u = (c & (kFaceFlag - 1)) >> 16;
            double b = Bf[(int64_t)fu_face[u] * npack_f + pair];
            double2 cf = fu_coef[u];
            vr += cf.x * b;
            vi += cf.y * b;
        } else {
            int64_t t = c >> 16;
            const double k = Kp[t * npack + pair];
            if (Mk) {  // nodal parameter: the tet's own complex mass sum_w kappa_w M_t^(w)
                const double2 mk = Mk[t * npack + pair];
                vr += k - k0sq * mk.x;
                vi += -k0sq * mk.y;
            } else {
                const double m = Mp[t * npack + pair];
                const double2 e = eps[t];
                vr += k - k0sq * e.x * m;
                vi += -k0sq * e.y * m;
            }
        }
    }
    if (out64) out64[s] = mk(vr, vi);
    if (outlo) { outlo[s].x = (float)vr; outlo[s].y = (float)vi; }
}

void launch_elem_geom(const double* xyz, const int32_t* tv, int64_t nt, const ElementTablesDev& tab,
                      double* K, double* M, cudaStream_t st) {
    int th = 128;
    elem_geom_kernel<<<(unsigned)((nt + th - 1) / th), th, 0, st>>>(
        xyz, tv, nt, tab.m_terms.p, tab.m_ptr.p, tab.k_terms.p, tab.k_ptr.p, tab.npack, K, M);
    MWI_CHECK_LAUNCH();
}

void launch_elem_vertex_mass(const double* xyz, const int32_t* tv, int64_t nt, const ElementTablesDev& tab,
                             double* Mv, cudaStream_t st) {
    int th = 128;
    elem_vertex_mass_kernel<<<(unsigned)((nt + th - 1) / th), th, 0, st>>>(xyz, tv, nt, tab.m_terms.p, tab.m_ptr.p,
                                                                         tab.mv_c.p, tab.npack, Mv);
    MWI_CHECK_LAUNCH();
}

void launch_face_geom(const double* xyz, const int32_t* tv, const int32_t* face_tets, const int8_t* face_lf,
                      int64_t nf, const ElementTablesDev& tab, double* Bf, cudaStream_t st) {
    int th = 128;
    face_geom_kernel<<<(unsigned)((nf + th - 1) / th), th, 0, st>>>(xyz, tv, face_tets, face_lf, nf, tab.f_terms.p,
                                                                  tab.f_ptr.p, tab.npack_f, Bf);
    MWI_CHECK_LAUNCH();
}

void launch_face_coef(const int32_t* fu_tet, int64_t nfu, const double2* eps, double k0, double2* coef,
                      cudaStream_t st) {
    if (nfu == 0) return;
    int th = 256;
    face_coef_kernel<<<(unsigned)((nfu + th - 1) / th), th, 0, st>>>(fu_tet, nfu, eps, k0, coef);
    MWI_CHECK_LAUNCH();
}

void launch_slot_fill(const SlotMatrixDev& S, const double* K, const double* M, int npack, const double* Bf,
                      int npack_f, const int32_t* fu_face, const double2* fu_coef, const double2* eps, double k0,
                      double2* out64, float2* out32, cudaStream_t st, const double2* Mk) {
    if (S.nnz == 0) return;
    int th = 256;
    slot_fill_kernel<float2><<<(unsigned)((S.nnz + th - 1) / th), th, 0, st>>>(
        S.nnz, S.slot_ptr.p, S.contrib.p, K, M, npack, Bf, npack_f, fu_face, fu_coef, eps, Mk, k0 * k0, out64,
        out32);
    MWI_CHECK_LAUNCH();
}

}  // namespace mwi

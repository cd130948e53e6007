// Nodal (P1) permittivity parameter with a gradient penalty (the P1 parameter
// of Section 6.3 and the regularised, normalised misfit of Eq. defJ2):
//   eps_t = (kappa at the tet's centroid) = 1/4 sum of kappa at its vertices
//   R     = (alpha / 2) Re(kappa^H K kappa),  K the P1 stiffness matrix
//   dPhi/dRe kappa_v + i dPhi/dIm kappa_v = 1/4 sum_{t contains v} g_t + alpha (K kappa)_v
// with g_t the per-tet gradient (same convention) of the misfit.  The spreading
// sums each vertex's tets in ascending order, so it is deterministic.
#include <algorithm>

#include "common.h"
#include "kernels.h"
#include "model.h"

namespace mwi {

__global__ void p1_tet_eps_kernel(int64_t nt, const int32_t* __restrict__ tv, const double2* __restrict__ kappa,
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

// per vertex: the spread per-tet gradient plus alpha K kappa; per block, the
// fixed-order sum of Re(conj(kappa_v) (K kappa)_v) over its vertices
__global__ void __launch_bounds__(256) p1_gradient_kernel(int64_t nv, const int32_t* __restrict__ v2t_ptr,
                                                          const int32_t* __restrict__ v2t,
                                                          const double2* __restrict__ grad_t,
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
            const double2 x = grad_t[v2t[q]];
            g.x += x.x;
            g.y += x.y;
        }
        double2 kk = make_double2(0.0, 0.0);
        for (int32_t q = rp[v]; q < rp[v + 1]; ++q) {
            const double2 x = kappa[col[q]];
            kk.x += val[q] * x.x;
            kk.y += val[q] * x.y;
        }
        out[v] = make_double2(0.25 * g.x + alpha * kk.x, 0.25 * g.y + alpha * kk.y);
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

void launch_p1_tet_eps(int64_t nt, const int32_t* tv, const double2* kappa, double2* eps, cudaStream_t st) {
    p1_tet_eps_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, tv, kappa, eps);
    MWI_CHECK_LAUNCH();
}

int p1_gradient_blocks(int64_t nv) { return (int)((nv + 255) / 256); }

void launch_p1_gradient(int64_t nv, const int32_t* v2t_ptr, const int32_t* v2t, const double2* grad_t,
                        const int32_t* rp, const int32_t* col, const double* val, const double2* kappa, double alpha,
                        double2* out, double* partial, cudaStream_t st) {
    p1_gradient_kernel<<<p1_gradient_blocks(nv), 256, 0, st>>>(nv, v2t_ptr, v2t, grad_t, rp, col, val, kappa, alpha,
                                                               out, partial);
    MWI_CHECK_LAUNCH();
}

}  // namespace mwi

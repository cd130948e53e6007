// Launchers of the physics kernels (physics.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mwi {

void launch_rhs(int m, const int32_t* dof, const double* sign, const double2* cur, double omega_mu0, double2* B,
                cudaStream_t st);
void launch_s_extract(int n_rx, int m, const int32_t* dof, const double* sign, const double2* U, double2* S,
                      cudaStream_t st);
void launch_misfit(int cnt, const double2* S, const double2* Sm, const double* w, double2* r, double* J,
                   cudaStream_t st);
void launch_adjoint_rhs(int n_rx, int m, const int32_t* dof, const double* sign, const double2* r, const double* w,
                        double2* G, cudaStream_t st);
void launch_gradient(int order, int64_t nt, int m, const int32_t* tet_dofs, const int32_t* tet_faces,
                     const int8_t* face_tag, const int32_t* face_dofs, const double* Mp, const double* Bf,
                     const double2* eps, double k0, const double2* U, const double2* Lam, double2* out,
                     cudaStream_t st);
// first order, mixed path: the volume term in double-float from U and Lam as
// double-float planes ([2][nm] complex FP32 pairs) and the element masses as
// double-float pairs Mdf [nt][21]
void launch_gradient_df(int64_t nt, int m, int64_t nm, const int32_t* tet_dofs, const int32_t* tet_faces,
                        const int8_t* face_tag, const int32_t* face_dofs, const float2* Mdf, const double* Bf,
                        const double2* eps, double k0, const double2* U, const double2* Lam, const float2* Udf,
                        const float2* Ldf, double2* out, cudaStream_t st);
// out[e] = double-float pair of a[e]
void launch_split_real(int64_t count, const double* a, float2* out, cudaStream_t st);

}  // namespace mwi

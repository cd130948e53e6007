// Application of the ORAS preconditioner  y = sum_i R_i^T D_i B_i^{-1} R_i x
// (Eq. ORAS), all subdomains at once:
//   1. gather   Y = R x            (local vectors of all subdomains, ND order)
//   2. forward  L z = Y            front by front, deepest level first; each
//               front assembles its children's update vectors (extend-add) and
//               passes its own update vector to its parent
//   3. backward D L^T Y = z        root level first; each front reads its
//               ancestors' final values through its update-row list
//   (both sweeps are batched dense products, see sweep.cu)
//   4. scatter  y_g = sum_{(i,l) -> g} D_i[l] Y_{i,l}   (fixed order, no atomics)
// Several right-hand sides go through one forward/backward sweep, as the
// paper notes for multiple vectors (Section 3).  Vectors are row-major [rows][m].
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "common.h"
#include "gmres.h"
#include "kernels.h"

namespace mwi {

template <typename A, typename B> __device__ __forceinline__ B cvt(A v);
template <> __device__ __forceinline__ double2 cvt<double2, double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<double2, float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 cvt<float2, double2>(float2 v) { return make_double2(v.x, v.y); }

// local vectors have ld >= m columns; the columns m..ld-1 are zero
template <typename In, typename C>
__global__ void gather_kernel(int64_t nloc, int m, int ld, const int32_t* __restrict__ loc2glob,
                              const In* __restrict__ x, C* __restrict__ Y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nloc * ld) return;
    int64_t r = e / ld;
    int c = (int)(e - r * ld);
    Y[e] = c < m ? cvt<In, C>(x[(int64_t)loc2glob[r] * m + c]) : czero<C>();
}

template <typename C, typename Out>
__global__ void scatter_kernel(int64_t n, int m, int ld, const int64_t* __restrict__ own_ptr,
                               const int32_t* __restrict__ own_row, const double* __restrict__ own_w,
                               const C* __restrict__ Y, Out* __restrict__ y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    int64_t g = e / m;
    int c = (int)(e - g * m);
    typedef typename real_of<C>::type R;
    C acc = czero<C>();
    for (int64_t q = own_ptr[g]; q < own_ptr[g + 1]; ++q) {
        C v = Y[(int64_t)own_row[q] * ld + c];
        R w = (R)own_w[q];
        acc.x += w * v.x;
        acc.y += w * v.y;
    }
    y[e] = cvt<C, Out>(acc);
}

// The same two steps for complex FP32 vectors with an even column count, two
// columns (16 bytes) per thread: a block of (threads per row) x (rows), so no
// thread divides by the row length
__global__ void gather2_kernel(int64_t nloc, int h, int ldh, const int32_t* __restrict__ loc2glob,
                               const float4* __restrict__ x, float4* __restrict__ Y) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.y + threadIdx.y;
    if (r >= nloc) return;
    const int64_t g = loc2glob[r];
    for (int c = threadIdx.x; c < ldh; c += blockDim.x)
        Y[r * ldh + c] = c < h ? x[g * h + c] : make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void scatter2_kernel(int64_t n, int h, int ldh, const int64_t* __restrict__ own_ptr,
                                const int32_t* __restrict__ own_row, const double* __restrict__ own_w,
                                const float4* __restrict__ Y, float4* __restrict__ y) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.y + threadIdx.y;
    if (g >= n) return;
    const int64_t q0 = own_ptr[g], q1 = own_ptr[g + 1];
    for (int c = threadIdx.x; c < h; c += blockDim.x) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t q = q0; q < q1; ++q) {
            const float4 v = Y[(int64_t)own_row[q] * ldh + c];
            const float w = (float)own_w[q];
            acc.x += w * v.x;
            acc.y += w * v.y;
            acc.z += w * v.z;
            acc.w += w * v.w;
        }
        y[g * h + c] = acc;
    }
}

static dim3 pair_block(int h) {
    const int hx = std::max(1, std::min(h, 256));
    return dim3(hx, 256 / hx);
}

// columns of the local vectors: the tensor-core sweeps move rows by 16-byte
// bulk copies, so their rows hold an even number of complex FP32 values (an
// odd m gets one zero column, which every step leaves zero)
int sweep_ld(int m, int tc) { return (tc == 4 && (m & 1)) ? m + 1 : m; }

template <typename C, typename In, typename Out>
static void oras_apply_impl(const FrontsDev& F, const C* ws, const In* x, Out* y, int m, C* Y, C* Z, C* upd,
                            cudaStream_t st, const SweepCfg& sc) {
    const int th = 256;
    const int ld = sizeof(C) == sizeof(float2) ? sweep_ld(m, sc.tc) : m;
    // complex FP32 throughout with even m and ld: 16-byte accesses
    constexpr bool c64 = std::is_same<C, float2>::value && std::is_same<In, float2>::value &&
                         std::is_same<Out, float2>::value;
    const bool pairs = c64 && (m % 2) == 0 && (ld % 2) == 0;
    const int64_t n = (int64_t)F.own_ptr.n - 1;
    if (pairs) {
        const dim3 b = pair_block(m / 2);
        gather2_kernel<<<(unsigned)((F.nloc + b.y - 1) / b.y), b, 0, st>>>(
            F.nloc, m / 2, ld / 2, F.loc2glob.p, reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(Y));
    } else {
        const int64_t tot = F.nloc * ld;
        gather_kernel<In, C><<<(unsigned)((tot + th - 1) / th), th, 0, st>>>(F.nloc, m, ld, F.loc2glob.p, x, Y);
    }
    MWI_CHECK_LAUNCH();
    multifrontal_solve<C>(F, ws, Y, Z, upd, ld, sc, st);
    // scatter into the global vector (n = own_ptr size - 1)
    if (pairs) {
        const dim3 b = pair_block(m / 2);
        scatter2_kernel<<<(unsigned)((n + b.y - 1) / b.y), b, 0, st>>>(
            n, m / 2, ld / 2, F.own_ptr.p, F.own_row.p, F.own_w.p, reinterpret_cast<const float4*>(Y),
            reinterpret_cast<float4*>(y));
    } else {
        const int64_t tot = n * m;
        scatter_kernel<C, Out><<<(unsigned)((tot + th - 1) / th), th, 0, st>>>(n, m, ld, F.own_ptr.p, F.own_row.p,
                                                                              F.own_w.p, Y, y);
    }
    MWI_CHECK_LAUNCH();
}

template <typename C>
void oras_apply(const FrontsDev& F, const C* ws, const double2* x, double2* y, int m, C* Y, C* Z, C* upd,
                cudaStream_t st, const float2* x32, float2* y32, const SweepCfg& sc) {
    if (x32) oras_apply_impl<C, float2, float2>(F, ws, x32, y32, m, Y, Z, upd, st, sc);
    else oras_apply_impl<C, double2, double2>(F, ws, x, y, m, Y, Z, upd, st, sc);
}

template void oras_apply<float2>(const FrontsDev&, const float2*, const double2*, double2*, int, float2*, float2*,
                                 float2*, cudaStream_t, const float2*, float2*, const SweepCfg&);
template void oras_apply<double2>(const FrontsDev&, const double2*, const double2*, double2*, int, double2*,
                                  double2*, double2*, cudaStream_t, const float2*, float2*, const SweepCfg&);

// ---------------------------------------------------------------------------
// Allocation-free variant of the ORAS application.  Its scratch (the local
// vectors Y and Z, the update vectors and, in the mixed path, the FP32 copies
// of x and y) is carved from one file-scope device array of fixed size instead of
// cudaMalloc'd buffers.  The array exists on every GPU that loads the library
// until the process exits.  Host code cannot use the array's name as a device
// address, so its address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
// Every call shares the array and leaves its contents behind; nothing in it
// needs to start at zero because the gather and the forward sweep write every
// location before it is read.

static __device__ __align__(256) unsigned char g_oras_scratch[kOrasScratchBytes];

static void* oras_scratch_address() {
    int dev = 0;
    MWI_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::vector<void*> addr;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_oras_scratch);
        if (e != cudaSuccess || !p)
            throw Error(MWI_ECUDA, std::string("cudaGetSymbolAddress of the ORAS scratch failed: ") +
                                       cudaGetErrorString(e));
        addr[dev] = p;
    }
    return addr[dev];
}

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t oras_noalloc_bytes(const FrontsDev& F, int64_t n, int m, bool mixed) {
    const size_t elt = mixed ? sizeof(float2) : sizeof(double2);
    const int ld = mixed ? m + (m & 1) : m;
    size_t b = 2 * round256((size_t)F.nloc * ld * elt) + round256((size_t)std::max<int64_t>(1, F.upd_rows) * ld * elt);
    if (mixed) b += 2 * round256((size_t)n * m * sizeof(float2));
    return b;
}

void oras_apply_noalloc(const FrontsDev& F, const void* ws, bool mixed, const double2* x, double2* y, int m,
                        int64_t n, cudaStream_t st, const SweepCfg& sc) {
    const size_t need = oras_noalloc_bytes(F, n, m, mixed);
    if (need > kOrasScratchBytes)
        throw Error(MWI_EINVAL, "problem needs " + std::to_string(need) + " bytes of ORAS scratch; the "
                                "allocation-free entry point holds " + std::to_string(kOrasScratchBytes));
    unsigned char* base = static_cast<unsigned char*>(oras_scratch_address());
    const size_t elt = mixed ? sizeof(float2) : sizeof(double2);
    const int ld = mixed ? m + (m & 1) : m;
    unsigned char* Yp = base;
    unsigned char* Zp = Yp + round256((size_t)F.nloc * ld * elt);
    unsigned char* Up = Zp + round256((size_t)F.nloc * ld * elt);
    unsigned char* Vp = Up + round256((size_t)std::max<int64_t>(1, F.upd_rows) * ld * elt);
    unsigned char* Xp = Vp + round256((size_t)n * m * sizeof(float2));
    if (mixed) {
        float2* v32 = reinterpret_cast<float2*>(Vp);
        float2* x32 = reinterpret_cast<float2*>(Xp);
        convert_c128_to_c64(n * m, x, v32, st);
        oras_apply_impl<float2, float2, float2>(F, static_cast<const float2*>(ws), v32, x32, m,
                                                reinterpret_cast<float2*>(Yp), reinterpret_cast<float2*>(Zp),
                                                reinterpret_cast<float2*>(Up), st, sc);
        convert_c64_to_c128(n * m, x32, y, st);
    } else {
        oras_apply_impl<double2, double2, double2>(F, static_cast<const double2*>(ws), x, y, m,
                                                   reinterpret_cast<double2*>(Yp), reinterpret_cast<double2*>(Zp),
                                                   reinterpret_cast<double2*>(Up), st, SweepCfg());
    }
}

}  // namespace mwi

// Internal helpers shared by the library's translation units: status
// reporting, CUDA error checks, device buffers and complex arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mwi.h"

namespace mwi {

// An error carried to the C ABI boundary, where it becomes an mwi_status.
struct Error : public std::runtime_error {
    mwi_status status;
    Error(mwi_status s, const std::string& msg) : std::runtime_error(msg), status(s) {}
};

void set_last_error(const std::string& msg);

// Run the body of a C-ABI entry point: an Error becomes its status, a failed
// host allocation MWI_ENOMEM, any other exception MWI_EINVAL; the message goes
// to mwi_last_error.
template <typename F>
mwi_status guard(F&& f) {
    try {
        f();
        return MWI_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return MWI_ENOMEM;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return MWI_EINVAL;
    }
}

// The solver options with every zero field replaced by its default (api.cpp).
mwi_solver_opts solver_defaults(const mwi_solver_opts* o);

// kernels launched by this library (every launch site ends in MWI_CHECK_LAUNCH)
extern std::atomic<int64_t> g_launches;
// device allocations made by this library (every cudaMalloc goes through DevBuf)
extern std::atomic<int64_t> g_device_allocs;

#define MWI_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t err__ = (call);                                                     \
        if (err__ != cudaSuccess)                                                       \
            throw ::mwi::Error(MWI_ECUDA, std::string(#call) + ": " +                   \
                                              cudaGetErrorString(err__) + " at " +      \
                                              __FILE__ + ":" + std::to_string(__LINE__)); \
    } while (0)

#define MWI_CHECK_LAUNCH()                                           \
    do {                                                             \
        ::mwi::g_launches.fetch_add(1, std::memory_order_relaxed);   \
        MWI_CUDA(cudaGetLastError());                                \
    } while (0)

#define MWI_REQUIRE(cond, status, msg)                     \
    do {                                                   \
        if (!(cond)) throw ::mwi::Error((status), (msg));  \
    } while (0)

// Owning device allocation (cudaMalloc / cudaFree).
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        g_device_allocs.fetch_add(1, std::memory_order_relaxed);
        cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            throw Error(MWI_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) +
                                        " bytes failed: " + cudaGetErrorString(e));
        }
        n = count;
    }
    void ensure(size_t count) { if (count > n) alloc(count); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void upload(const std::vector<T>& h, cudaStream_t s) {
        alloc(h.size());
        if (!h.empty())
            MWI_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void zero(cudaStream_t s) {
        if (n) MWI_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    size_t bytes() const { return n * sizeof(T); }
};

}  // namespace mwi

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2 (x = re, y = im)
#if defined(__CUDACC__)
#define MWI_HD __host__ __device__ __forceinline__
#else
#define MWI_HD inline
#endif

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { typedef double2 type; };
template <> struct cplx_of<float> { typedef float2 type; };

template <typename C> struct real_of;
template <> struct real_of<double2> { typedef double type; };
template <> struct real_of<float2> { typedef float type; };

MWI_HD double2 mk(double a, double b) { double2 r; r.x = a; r.y = b; return r; }
MWI_HD float2 mkf(float a, float b) { float2 r; r.x = a; r.y = b; return r; }
template <typename C> MWI_HD C cmake(typename real_of<C>::type a, typename real_of<C>::type b) {
    C r; r.x = a; r.y = b; return r;
}
template <typename C> MWI_HD C czero() { C r; r.x = 0; r.y = 0; return r; }
template <typename C> MWI_HD C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> MWI_HD C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> MWI_HD C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a + b * c
template <typename C> MWI_HD C cfma(C b, C c, C a) {
    C r;
    r.x = a.x + b.x * c.x - b.y * c.y;
    r.y = a.y + b.x * c.y + b.y * c.x;
    return r;
}
// a - b * c
template <typename C> MWI_HD C cfms(C b, C c, C a) {
    C r;
    r.x = a.x - b.x * c.x + b.y * c.y;
    r.y = a.y - b.x * c.y - b.y * c.x;
    return r;
}
// conj(a) * b
template <typename C> MWI_HD C cconjmul(C a, C b) {
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename C> MWI_HD C cscale(C a, typename real_of<C>::type s) {
    C r; r.x = a.x * s; r.y = a.y * s; return r;
}
template <typename C> MWI_HD C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }
template <typename C> MWI_HD typename real_of<C>::type cabs2(C a) { return a.x * a.x + a.y * a.y; }
template <typename C> MWI_HD C cdiv(C a, C b) {
    typename real_of<C>::type d = b.x * b.x + b.y * b.y;
    C r;
    r.x = (a.x * b.x + a.y * b.y) / d;
    r.y = (a.y * b.x - a.x * b.y) / d;
    return r;
}
template <typename C> MWI_HD C crecip(C b) {
    typename real_of<C>::type d = b.x * b.x + b.y * b.y;
    C r; r.x = b.x / d; r.y = -b.y / d; return r;
}

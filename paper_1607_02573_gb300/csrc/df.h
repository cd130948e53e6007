// Double-float arithmetic: a real number carried as an unevaluated sum hi + lo
// of two FP32 values (about 48 significant bits), built from the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProduct via a
// fused multiply-add (Dekker 1971; Ogita, Rump and Oishi 2005).  On GB300 the
// FP64 units run at 1/64 of the FP32 rate, so FP64-accurate vector work of
// the outer Krylov solver is done in this form on the FP32 pipes.
//
// The expressions rely on IEEE FP32 semantics without reassociation (no fast
// math); contraction into FMA is harmless where it occurs.
#pragma once

#include <cuda_runtime.h>

namespace mwi {

struct dfl {
    float h, l;
};

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ dfl df_norm(dfl a) {
    dfl r;
    quick_two_sum(a.h, a.l, r.h, r.l);
    return r;
}

// acc += (ah + al) * (bh + bl), the product to about 2^-46 relative; acc is
// left unnormalised (lo accumulates), df_norm it before storing
__device__ __forceinline__ void df_mac(dfl& acc, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    float s, t;
    two_sum(acc.h, p, s, t);
    acc.h = s;
    acc.l += t + e;
}

// acc += a * (bh + bl) with a exact in FP32
__device__ __forceinline__ void df_mac1(dfl& acc, float a, float bh, float bl) {
    const float p = a * bh;
    float e = fmaf(a, bh, -p);
    e = fmaf(a, bl, e);
    float s, t;
    two_sum(acc.h, p, s, t);
    acc.h = s;
    acc.l += t + e;
}

// (ah + al) * (bh + bl), normalised
__device__ __forceinline__ dfl df_mul(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    dfl r;
    quick_two_sum(p, e, r.h, r.l);
    return r;
}

// nearest double-float of an FP64 value (FP64 units: use outside hot loops)
__device__ __forceinline__ float2 df_split(double x) {
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(x - (double)h);
    return make_float2(h, l);
}

__device__ __forceinline__ double df_join(float h, float l) { return (double)h + (double)l; }

}  // namespace mwi

// Device helpers of libnk: Philox4x64-10, ln cosh, renormalised products,
// warp reductions, error plumbing.  Internal header (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nk.h"

namespace nk {

constexpr double kLn2 = 0.69314718055994530942;

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies, a word
// permutation and a key xor, with the key advanced by two Weyl constants
// between rounds.
// ---------------------------------------------------------------------------
struct Philox4 {
    unsigned long long v[4];
};

__device__ __forceinline__ Philox4 philox4x64_10(unsigned long long c0, unsigned long long c1,
                                                 unsigned long long c2, unsigned long long c3,
                                                 unsigned long long k0, unsigned long long k1) {
    const unsigned long long kMulA = 0xD2E7470EE14C6C93ULL;
    const unsigned long long kMulB = 0xCA5A826395121157ULL;
    const unsigned long long kWeylA = 0x9E3779B97F4A7C15ULL;
    const unsigned long long kWeylB = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long hiA = __umul64hi(kMulA, c0), loA = kMulA * c0;
        unsigned long long hiB = __umul64hi(kMulB, c2), loB = kMulB * c2;
        unsigned long long n0 = hiB ^ c1 ^ k0;
        unsigned long long n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    Philox4 out;
    out.v[0] = c0;
    out.v[1] = c1;
    out.v[2] = c2;
    out.v[3] = c3;
    return out;
}

// Index in [0, n) from the top 32 bits by multiply-shift.
__device__ __forceinline__ int pick_index(unsigned long long y, int n) {
    return (int)(((y >> 32) * (unsigned long long)n) >> 32);
}

// Uniform in (0, 1): ((y >> 11) + 1/2) * 2^-53.
__device__ __forceinline__ double uniform53(unsigned long long y) {
    return ((double)(y >> 11) + 0.5) * 1.1102230246251565404e-16;
}

// ---------------------------------------------------------------------------
// ln cosh x without cancellation: for |x| < 1 use cosh x - 1 = 2 sinh^2(x/2)
// and log1p; otherwise |x| - ln 2 + log1p(e^{-2|x|}).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double lncosh(double x) {
    double ax = fabs(x);
    if (ax < 1.0) {
        double sh = sinh(0.5 * ax);
        return log1p(2.0 * sh * sh);
    }
    return ax + log1p(exp(-2.0 * ax)) - kLn2;
}

__device__ __forceinline__ float lncosh(float x) {
    float ax = fabsf(x);
    if (ax < 1.0f) {
        float sh = sinhf(0.5f * ax);
        return log1pf(2.0f * sh * sh);
    }
    return ax + log1pf(expf(-2.0f * ax)) - 0.69314718f;
}

// ---------------------------------------------------------------------------
// Running product kept as mantissa * 2^exp so that long products of factors
// in (0, 2) neither underflow nor overflow.
// ---------------------------------------------------------------------------
template <typename R>
struct Prod {
    R m;
    int e;
};

__device__ __forceinline__ void renorm(Prod<double> &p) {
    int k;
    p.m = frexp(p.m, &k);
    p.e += k;
}
__device__ __forceinline__ void renorm(Prod<float> &p) {
    int k;
    p.m = frexpf(p.m, &k);
    p.e += k;
}

template <typename R>
struct RenormEvery;
template <>
struct RenormEvery<double> {
    static constexpr int value = 32;
};
template <>
struct RenormEvery<float> {
    static constexpr int value = 8;
};

__device__ __forceinline__ double prod_log(const Prod<double> &p) {
    return log(p.m) + (double)p.e * kLn2;
}
__device__ __forceinline__ float prod_log(const Prod<float> &p) {
    return logf(p.m) + (float)p.e * 0.69314718f;
}

// Butterfly all-reduce of a product: every lane ends with the same value
// (IEEE multiplication and integer addition are commutative).
template <typename R>
__device__ __forceinline__ Prod<R> warp_prod(Prod<R> p) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        R m2 = __shfl_xor_sync(0xffffffffu, p.m, off);
        int e2 = __shfl_xor_sync(0xffffffffu, p.e, off);
        p.m *= m2;
        p.e += e2;
        renorm(p);
    }
    return p;
}

// Same product as warp_prod, renormalised once at the end: when every lane's
// partial mantissa lies in [1/2, 1) the running products stay >= 2^-32, far
// from underflow, and scaling by powers of two does not change the rounding
// of a product, so the result is bit-identical.
template <typename R>
__device__ __forceinline__ Prod<R> warp_prod_normalised(Prod<R> p) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        p.m *= __shfl_xor_sync(0xffffffffu, p.m, off);
        p.e += __shfl_xor_sync(0xffffffffu, p.e, off);
    }
    renorm(p);
    return p;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Error-free transformation a + b = s + err (Knuth TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &err) {
    s = a + b;
    double bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

}  // namespace nk

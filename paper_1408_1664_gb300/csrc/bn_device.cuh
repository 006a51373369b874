// bn_device.cuh -- device helpers shared by the kernels of the library:
// log-domain arithmetic for the two precisions, subset-mask index maps and
// colexicographic ranking.  Variable i is bit i of a mask.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace bn {

// ---------------------------------------------------------------------------
// Binomial coefficients C(n, k), 0 <= k <= n <= 32, built at compile time.
// ---------------------------------------------------------------------------
struct BinomTable {
    uint32_t v[33][33];
};

constexpr BinomTable make_binom_table()
{
    BinomTable t{};
    for (int n = 0; n <= 32; ++n) {
        t.v[n][0] = 1;
        for (int k = 1; k <= n; ++k)
            t.v[n][k] = t.v[n - 1][k - 1] + (k <= n - 1 ? t.v[n - 1][k] : 0u);
    }
    return t;
}

static __constant__ BinomTable c_binom = make_binom_table();

__device__ __forceinline__ uint32_t binom(int n, int k)
{
    return (k < 0 || k > n) ? 0u : c_binom.v[n][k];
}

// Jobs of one batch group share a launch: the arrays of job blockIdx.y lie
// js bytes after those of job blockIdx.y - 1 (js = 0 for a single job).
template <typename P>
__device__ __forceinline__ P* job_ptr(P* p, size_t js)
{
    // byte arithmetic on the pointer itself (no round trip through an
    // integer), so the result stays based on p for alias analysis
    using B = typename std::conditional<std::is_const<P>::value, const char, char>::type;
    return reinterpret_cast<P*>(reinterpret_cast<B*>(p) + (size_t)blockIdx.y * js);
}

// Number of subsets of an nb-element set with at most d elements.
__device__ __forceinline__ uint32_t num_small_subsets(int nb, int d)
{
    uint32_t s = 0;
    for (int k = 0; k <= d && k <= nb; ++k) s += binom(nb, k);
    return s;
}

// Rank of mask x among the subsets of {0..nb-1} with at most d elements,
// ordered by size and then by increasing value (colexicographic order).
__device__ __forceinline__ uint32_t small_subset_rank(uint32_t x, int nb)
{
    const int k = __popc(x);
    uint32_t r = 0;
    for (int s = 0; s < k; ++s) r += binom(nb, s);
    int t = 1;
    while (x) {
        const int c = __ffs(x) - 1;
        r += binom(c, t);
        ++t;
        x &= x - 1;
    }
    return r;
}

// Inverse of small_subset_rank for a subset of known size k and colex rank r
// among the k-subsets of {0..nb-1}.
__device__ __forceinline__ uint32_t colex_unrank(uint32_t r, int k, int nb)
{
    uint32_t x = 0;
    int c = nb - 1;
    for (int t = k; t >= 1; --t) {
        while (binom(c, t) > r) --c;
        x |= 1u << c;
        r -= binom(c, t);
        --c;
    }
    return x;
}

// Remove bit i from S (S must not matter at bit i): the index of S in an
// array over the subsets of V-{i}.
__device__ __forceinline__ uint32_t squeeze(uint32_t S, int i)
{
    const uint32_t low = (1u << i) - 1u;
    return (S & low) | ((S >> 1) & ~low);
}

// Insert a zero bit at position i.
__device__ __forceinline__ uint32_t expand(uint32_t c, int i)
{
    const uint32_t low = (1u << i) - 1u;
    return (c & low) | ((c & ~low) << 1);
}

// ---------------------------------------------------------------------------
// Log-domain arithmetic.  FP64 values are natural logs; FP32 values are
// base-2 logs so that the hardware ex2/lg2 approximations apply directly.
// -inf is a zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T> struct LogOps;

template <> struct LogOps<double> {
    static __device__ __forceinline__ double ninf() { return __longlong_as_double((long long)0xfff0000000000000ull); }
    // exp and log in this value's base
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double lg(double x) { return log(x); }
    // log(exp(a) + exp(b))
    static __device__ __forceinline__ double lse(double a, double b)
    {
        const double mx = fmax(a, b), mn = fmin(a, b);
        if (mn == ninf()) return mx;
        return mx + log1p(exp(mn - mx));
    }
    // value in this domain from a natural log
    static __device__ __forceinline__ double from_ln(double x) { return x; }
    static __device__ __forceinline__ double to_ln(double x) { return x; }
};

template <> struct LogOps<float> {
    static __device__ __forceinline__ float ninf() { return __int_as_float(0xff800000); }
    static __device__ __forceinline__ float ex(float x) { return ex2_approx(x); }
    static __device__ __forceinline__ float lg(float x) { return lg2_approx(x); }
    static __device__ __forceinline__ float lse(float a, float b)
    {
        const float mx = fmaxf(a, b), mn = fminf(a, b);
        if (mn == ninf()) return mx;
        return mx + lg2_approx(1.0f + ex2_approx(mn - mx));
    }
    static __device__ __forceinline__ double from_ln(double x) { return x * 1.4426950408889634074; }
    static __device__ __forceinline__ double to_ln(double x) { return x * 0.69314718055994530942; }
};

// Online log-sum-exp accumulator: value = m + lg(s).
template <typename T> struct LseAcc {
    T m, s;
    __device__ __forceinline__ LseAcc() : m(LogOps<T>::ninf()), s(T(0)) {}
    __device__ __forceinline__ void add(T x)
    {
        if (x == LogOps<T>::ninf()) return;
        if (x > m) {
            s = s * LogOps<T>::ex(m - x) + T(1);
            m = x;
        } else {
            s += LogOps<T>::ex(x - m);
        }
    }
    __device__ __forceinline__ T value() const
    {
        return m == LogOps<T>::ninf() ? m : m + LogOps<T>::lg(s);
    }
};

// Order-preserving integer encodings for atomicMax on shared memory.
__device__ __forceinline__ uint32_t ord_enc(float x)
{
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ unsigned long long ord_enc(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_dec(unsigned long long u)
{
    return __longlong_as_double((long long)((u & 0x8000000000000000ull)
                                            ? (u & 0x7fffffffffffffffull) : ~u));
}

template <typename T> struct OrdInt;
template <> struct OrdInt<float> { using type = uint32_t; };
template <> struct OrdInt<double> { using type = unsigned long long; };

}  // namespace bn

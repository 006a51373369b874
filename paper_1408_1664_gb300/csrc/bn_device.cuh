// bn_device.cuh -- device helpers shared by the kernels of the library:
// log-domain arithmetic for the two precisions, subset-mask index maps and
// colexicographic ranking.  Variable i is bit i of a mask.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "bn_explog_tables.h"

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

// ---------------------------------------------------------------------------
// Index checks of the BN_CHECK_BOUNDS build (a debug build of the library;
// the release and testing builds compile BN_AT to the offset itself).  An
// access of `width` elements at offset `off` of an array of `size` elements
// that does not fit records the source line in the translation unit's word
// (the first failure wins) and goes to offset 0 instead, so the kernel
// neither faults nor traps; the host reads the word through
// bn_debug_bounds.  Every array checked has at least `width` elements.
// ---------------------------------------------------------------------------
#ifdef BN_CHECK_BOUNDS
static __device__ unsigned int g_bounds_line;       // one per translation unit
__device__ __forceinline__ size_t bounds_check(size_t off, size_t width, size_t size, int line)
{
    if (off <= size && width <= size - off) return off;
    atomicCAS(&g_bounds_line, 0u, (unsigned)line);
    return 0;
}
#define BN_AT(off, width, size) \
    ::bn::bounds_check((size_t)(off), (size_t)(width), (size_t)(size), __LINE__)
// Host: the unit's first failing line (0: none), cleared by the read.
#define BN_BOUNDS_READER(name)                                              \
    unsigned int name()                                                     \
    {                                                                       \
        unsigned int v = 0, z = 0;                                          \
        if (cudaMemcpyFromSymbol(&v, g_bounds_line, sizeof v) != cudaSuccess) \
            return ~0u;                                                     \
        cudaMemcpyToSymbol(g_bounds_line, &z, sizeof z);                    \
        return v;                                                           \
    }
#else
#define BN_AT(off, width, size) ((size_t)(off))
#endif

// The slice of the down-zeta scratch W that endpoint v uses: v itself when
// every endpoint is computed, its rank among the computed ones (vsel) when a
// split job's rank computes only some.
__host__ __device__ __forceinline__ uint32_t endpoint_slot(uint32_t vsel, int v)
{
#ifdef __CUDA_ARCH__
    return (uint32_t)__popc(vsel & ((1u << v) - 1u));
#else
    return (uint32_t)__builtin_popcount(vsel & ((1u << v) - 1u));
#endif
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

// ---------------------------------------------------------------------------
// Per-level bases of F and R' in FP32 (the per-level max shift of the FP32
// form).  F(S) grows by about a factor |S| and an A term per lattice level, so
// in log2 units the forward and backward sums of a large job reach thousands
// (about -4600 at n = 29), where one FP32 rounding unit is 2^-11: rounded
// level after level that costs up to 1e-4 in a posterior.  The step-3 row
// kernels therefore store every value relative to an integer base of its
// tile level k = |S >> kLevelShift| (the level of the launch that writes it):
//   F_s(S) = F(S) - bF[k],   bF[0] = 0,  bF[k] = bF[k-1] + dF[k-1],
//   R_s(T) = R'(T) - bR[k],  bR[nh] = 0, bR[k] = bR[k+1] + dR[k+1],
// where d[k] = floor of the largest stored value of level k (nh = n - 4), so
// that the largest values of every level stay within a few dozen units of
// zero.  The kLevelWords ints right after the 2^n values of F (and of R')
// hold d[k] per level and, in word kLevelMode, the tile shift the bases
// refer to (0: no bases, every b = 0; kernels other than the FP32 row kernels
// write 0).  The bases are exact small integers, so adding them back (the
// down-zeta input F(S) + R'(S + {v}), log P(D)) loses nothing.
// ---------------------------------------------------------------------------
constexpr int kLevelWords = 32;
constexpr int kLevelMode = 31;
constexpr int kLevelShift = 4;
constexpr int kLevelUnset = -2147483647 - 1;

__host__ __device__ __forceinline__ double level_delta(const int* lw, int k)
{
    return lw[k] == kLevelUnset ? 0.0 : (double)lw[k];
}
// bF[k] (forward) and bR[k] (backward) from the level words; 0 without bases.
__host__ __device__ __forceinline__ double level_base_fwd(const int* lw, int k)
{
    if (lw[kLevelMode] != kLevelShift) return 0.0;
    double b = 0.0;
    for (int j = 0; j < k; ++j) b += level_delta(lw, j);
    return b;
}
__host__ __device__ __forceinline__ double level_base_bwd(const int* lw, int k, int nh)
{
    if (lw[kLevelMode] != kLevelShift) return 0.0;
    double b = 0.0;
    for (int j = nh; j > k; --j) b += level_delta(lw, j);
    return b;
}
// The level words after an FP32 array of 2^n values.
__host__ __device__ __forceinline__ const int* level_words(const float* X, int n)
{
    return reinterpret_cast<const int*>(X + ((size_t)1 << n));
}
__host__ __device__ __forceinline__ int* level_words(float* X, int n)
{
    return reinterpret_cast<int*>(X + ((size_t)1 << n));
}
// floor(x) as an int for the level words (kLevelUnset for -inf or below).
__device__ __forceinline__ int level_floor(float x)
{
    return x > -2.0e9f ? (int)floorf(x) : kLevelUnset;
}

// FP32 down-zeta input for endpoint v: s_v(S) = F_s(S) + R_s(S + {v}) +
// off[|S >> *sh|] equals F(S) + R'(S + {v}) - Z, with the integer
// Z = bF[nh] + floor(F_s(V)), so that log P(D) - Z = *fvrel lies in [0, 1)
// (in the shifted log2 units of the FP32 path).  Without bases *sh = 31 and
// off[0] = -Z.  Called by all 32 lanes of one warp; writes off[0..nh].
__device__ __forceinline__ void gamma_offsets(int n, int v, const float* F, const float* Rc,
                                              float* off, int* sh, float* fvrel)
{
    const int lane = threadIdx.x & 31;
    const int* lf = level_words(F, n);
    const int* lr = level_words(Rc, n);
    const bool bases = lf[kLevelMode] == kLevelShift && lr[kLevelMode] == kLevelShift;
    const float fs = F[((size_t)1 << n) - 1];
    const double z0 = floor((double)fs);
    if (lane == 0) *fvrel = (float)((double)fs - z0);
    if (!bases) {
        if (lane == 0) {
            off[0] = (float)(-z0);
            *sh = 31;
        }
        return;
    }
    const int nh = n - kLevelShift;
    // bF[a] = sum_{j < a} dF[j]: exclusive prefix sum over the lanes
    const double x = lane < nh ? level_delta(lf, lane) : 0.0;
    double incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const double bF = incl - x;
    // bR[k] = sum_{k < j <= nh} dR[j]: exclusive suffix sum
    const double r = (lane >= 1 && lane <= nh) ? level_delta(lr, lane) : 0.0;
    double suf = r;
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_down_sync(0xffffffffu, suf, o);
        if (lane + o < 32) suf += y;
    }
    const double bR = suf - r;
    const double Z = __shfl_sync(0xffffffffu, bF, nh) + z0;
    // |(S + {v}) >> 4| = |S >> 4| + [v >= 4]
    const double bRv = __shfl_sync(0xffffffffu, bR, min(lane + (v >= kLevelShift ? 1 : 0), nh));
    if (lane <= nh) off[lane] = (float)(bF + bRv - Z);
    if (lane == 0) *sh = kLevelShift;
}

// The down-zeta offsets of every endpoint, built once per job before the
// down-zeta phase 1 (launch_gamma_p1): after the level words of R', 32 floats
// per endpoint v: off[0..29], then the shift (int bits) and F(V) - Z.
constexpr int kGammaTabWords = 32 * 32;
__host__ __device__ __forceinline__ float* gamma_table(float* Rc, int n)
{
    return reinterpret_cast<float*>(level_words(Rc, n) + kLevelWords);
}
__host__ __device__ __forceinline__ const float* gamma_table(const float* Rc, int n)
{
    return reinterpret_cast<const float*>(level_words(Rc, n) + kLevelWords);
}
// Threads 0..31 of a block copy endpoint v's offsets into shared memory.
__device__ __forceinline__ void load_gamma_offsets(const float* Rc, int n, int v, float* off,
                                                   int* sh, float* fvrel)
{
    if (threadIdx.x < 32) {
        const float x = gamma_table(Rc, n)[v * 32 + threadIdx.x];
        off[threadIdx.x] = x;
        if (threadIdx.x == 30) *sh = __float_as_int(x);
        if (threadIdx.x == 31) *fvrel = x;
    }
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

// ---------------------------------------------------------------------------
// Rows of A in level order inside each tile (use_tlo).  With the FP32
// schedule of 13-dimension up-zeta tiles and step-3 row kernels, A_i(S')
// (S' over the n - 1 other variables) is held in rows of 2^lw values
// (lw = 3 for i < 4, else 4: the row widths step 3 reads), S' = (R << lw) | l,
// and the 2^rb rows of one up-zeta tile (rb = 13 - lw, R = (H << rb) | r)
// are ordered by |r|, then colexicographically: row R sits at
// (H << rb) | place_rb(r).  A popcount level of step 3 then reads one
// contiguous run of rows from each tile block, not rows scattered over it;
// every up-zeta tile still writes its own block only, and the empty and
// full in-tile sets keep their places (first and last).
// ---------------------------------------------------------------------------
struct PlaceTable {
    uint16_t p9[512];
    uint16_t p10[1024];
};

constexpr PlaceTable make_place_table()
{
    const BinomTable b = make_binom_table();
    PlaceTable t{};
    for (int rb = 9; rb <= 10; ++rb)
        for (uint32_t r = 0; r < (1u << rb); ++r) {
            int k = 0;
            uint32_t colex = 0;
            for (int x = 0; x < rb; ++x)
                if (r >> x & 1u) {
                    ++k;
                    colex += b.v[x][k];                 // C(element, its index)
                }
            uint32_t start = 0;                         // rows with fewer elements
            for (int q = 0; q < k; ++q) start += b.v[rb][q];
            if (rb == 9) t.p9[r] = (uint16_t)(start + colex);
            else t.p10[r] = (uint16_t)(start + colex);
        }
    return t;
}

__device__ const PlaceTable g_place = make_place_table();

// Place of row R (rb = 9 or 10 in-tile bits) in the tile-level order.
__device__ __forceinline__ uint32_t tlo_row(uint32_t R, int rb)
{
    const uint32_t m = (1u << rb) - 1u;
    return (R & ~m) | (rb == 9 ? g_place.p9[R & m] : g_place.p10[R & m]);
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

// ---------------------------------------------------------------------------
// FP64 exp and log by table-driven reduction (P. T. P. Tang, ACM TOMS 15(2),
// 1989 and 16(4), 1990; tables in bn_explog_tables.h).  They take about half
// the FP64 instructions of the CUDA functions, which bound the FP64 path.
//   exp: x = k ln2/64 + r, |r| <= ln2/128 (k by one rounding, r by a two-part
//        ln2/64); exp(x) = 2^(k>>6) 2^((k&63)/64) (1 + expm1(r)).  Below the
//        normal range (x <
//        -708.3) it returns 0, where the CUDA function returns a subnormal:
//        every use here adds the result to terms larger by 2^50 or more.
//        expm1 to degree 6: truncation below 2^-67.
//   log: x = 2^e m, m in [1, 2); c_j = 1 + (2j + 1)/256 nearest m (j = the
//        top 7 bits of m's fraction), m - c_j exact, r = (m - c_j)/c_j,
//        |r| < 2^-8; log x = e ln2 + log c_j + log1p(r), log1p to degree 7
//        (truncation below 2^-67).  The results are checked against CUDA's
//        exp and log by a test (bn_debug_explog).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double exp_t(double x)
{
    using namespace explog;
    if (!(x > -708.3)) return x != x ? x : 0.0;
    if (x > 709.7) return __longlong_as_double(0x7ff0000000000000LL);
    const double shifter = 6755399441055744.0;        // 1.5 * 2^52: rounds to an integer
    const double t = fma(x, kInvLn2x64, shifter);
    const int k = __double2loint(t);
    const double kd = t - shifter;
    double r = fma(-kd, kLn2x64Hi, x);
    r = fma(-kd, kLn2x64Lo, r);
    double p = fma(r, 1.0 / 720, 1.0 / 120);
    p = fma(p, r, 1.0 / 24);
    p = fma(p, r, 1.0 / 6);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p *= r;                                           // expm1(r)
    const double tj = kExp2Frac[k & 63];
    const double y = fma(tj, p, tj);
    return y * __longlong_as_double((long long)((k >> 6) + 1023) << 52);
}

__device__ __forceinline__ double log_t(double x)
{
    using namespace explog;
    long long bits = __double_as_longlong(x);
    if (!(x > 0.0) || bits >= 0x7ff0000000000000LL) {  // 0, negative, NaN, +inf
        if (x == 0.0) return __longlong_as_double((long long)0xfff0000000000000ULL);
        return x > 0.0 ? x : __longlong_as_double(0x7ff8000000000000LL);
    }
    int e = 0;
    if (bits < 0x0010000000000000LL) {                 // subnormal: scale up by 2^54
        x *= 18014398509481984.0;
        bits = __double_as_longlong(x);
        e = -54;
    }
    e += (int)(bits >> 52) - 1023;
    const int j = (int)(bits >> 45) & 127;
    const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const double c = __longlong_as_double(0x3ff0000000000000LL | ((long long)(2 * j + 1) << 44));
    const double r = (m - c) * kInvC[j];
    double p = fma(r, -1.0 / 7, 1.0 / 6);            // log1p(r) = r + r^2 (-1/2 + r/3 - ...)
    p = fma(p, -r, 0.2);
    p = fma(p, r, -0.25);
    p = fma(p, r, 1.0 / 3);
    p = fma(p, r, -0.5);
    const double q = fma(r * r, p, r);
    const double ed = (double)e;
    return fma(ed, kLn2Hi, kLogCHi[j]) + (fma(ed, kLn2Lo, kLogCLo[j]) + q);
}

template <typename T> struct LogOps;

template <> struct LogOps<double> {
    static __device__ __forceinline__ double ninf() { return __longlong_as_double((long long)0xfff0000000000000ull); }
    // exp and log in this value's base
    static __device__ __forceinline__ double ex(double x) { return exp_t(x); }
    static __device__ __forceinline__ double lg(double x) { return log_t(x); }
    // log(exp(a) + exp(b)) with the table-driven exponential and logarithm:
    // 1 + e rounds by at most 2^-53, which moves the logarithm by at most
    // that much, so the result carries the same absolute error as with log1p
    static __device__ __forceinline__ double lse(double a, double b)
    {
        const double mx = fmax(a, b), mn = fmin(a, b);
        if (mn == ninf()) return mx;
        return mx + log_t(1.0 + exp_t(mn - mx));
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

// ---------------------------------------------------------------------------
// Bulk asynchronous copies between global and shared memory (the TMA unit's
// untiled form) and the shared-memory barrier that counts their bytes.  Both
// addresses of a copy and its size are multiples of 16 bytes.  A load signals
// its mbarrier when its bytes have landed; a store joins the issuing thread's
// bulk group, which the thread drains with bulk_wait_read (shared memory may
// be reused) or bulk_wait (the global writes are done).
// ---------------------------------------------------------------------------
// Polls of a copy's mbarrier before a kernel gives up on it.
constexpr uint32_t kCopySpinCap = 1u << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t arrivals)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(arrivals) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier shared-memory accesses before later bulk
// copies that read or overwrite the same bytes.
__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// This thread's arrival on the barrier, announcing `bytes` of copies to come.
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// A copy whose bytes count toward the barrier's announced total.
__device__ __forceinline__ void bulk_copy_in(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    mbar_expect(bar, bytes);
    bulk_copy_in(dst, src, bytes, bar);
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Waits for phase `parity` of the barrier to complete, at most `cap` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t cap)
{
    for (uint32_t it = 0; it < cap; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace bn

// bn_tile13.cu -- register-blocked 13-dimension tiles for the two truncated
// zeta transforms (Eq. 7 / Algorithm 2 and Eq. 12 / Algorithm 3) when n >= 14.
//
// A tile is the 2^13 subsets that share their high bits.  256 threads hold 32
// values each.  A transform over the 13 tile dimensions runs in three
// register layouts (dims 8..12, dims 3..7, dims 0..2), exchanging through a
// swizzled shared-memory array between layouts, so every butterfly is a
// register operation.
//
// Arithmetic is exact to working precision without a log-sum-exp per
// butterfly.  Most tiles are summed in linear scale, in one or a few
// single-scale passes (Window).  The others first compute the max-plus
// transform m(L), the largest single term of every output (a max per
// butterfly), and hold each value as y(L) * 2^m(L) (e^m(L) in FP64): every
// partial sum at L is at most the final output, so y(L) <= 8192, and a
// butterfly adds its partner scaled by 2^(m(partner) - m(L)) <= 1 (m is
// monotone along the butterflies).  A term can only underflow there when it
// is below 2^-126 of the output it belongs to.  One exponential enters per
// input and per butterfly, one logarithm leaves per output.  FP64 avoids a
// full-precision exponential per butterfly: it holds each value as
// x(L) * e^(BW*e(L)) with the band e(L) = floor(m(L) / BW), BW = 600 nats, so
// x(L) lies in [1, e^BW * 8192); a butterfly adds a partner from the same
// band unchanged, one band lower times e^-BW, and drops partners two or more
// bands lower (below e^-BW * 2^-13 of the result: under one rounding unit).
#include "bn_device.cuh"
#include "bn_kernels.cuh"

#include <cmath>

namespace bn {
namespace {

constexpr int TB = 13;            // tile dimensions
constexpr int TN = 1 << TB;       // tile elements
constexpr int TT = 256;           // threads per tile
constexpr int TR = 32;            // values per thread
constexpr unsigned FULLMASK = 0xffffffffu;

// Band width (natural logs) and the factor one band down, FP64 only.
struct Band64 {
    static constexpr double width = 600.0;
    static __device__ __forceinline__ double down1() { return 2.6503965530043108e-261; }  // e^-600
};

// a*b + c in the value's own precision (no promotion to double).
__device__ __forceinline__ float madd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Shared-memory position of tile element e.  Flips bits 3,4 by bits 8,9 and
// bit 2 by bit 5, which makes all three layouts' accesses free of bank
// conflicts (32-bit accesses in layouts 1 and 2, 128-bit in layout 3).
__device__ __forceinline__ uint32_t swz(uint32_t e)
{
    return e ^ (((e >> 8) & 3u) << 3) ^ (((e >> 5) & 1u) << 2);
}

// Element held in register r by thread t.
__device__ __forceinline__ uint32_t el1(int r, int t) { return ((uint32_t)r << 8) | (uint32_t)t; }
__device__ __forceinline__ uint32_t el2(int r, int t)
{
    return ((uint32_t)t & 7u) | ((uint32_t)r << 3) | (((uint32_t)t >> 3) << 8);
}
__device__ __forceinline__ uint32_t el3(int r, int t)
{
    return ((uint32_t)r & 7u) | ((uint32_t)t << 3) | (((uint32_t)r >> 3) << 11);
}

// Butterflies over register bits [k0, k0+nk): UP adds a subset into its
// superset (upward zeta), DOWN adds a superset into its subset.
template <bool UP, typename T>
__device__ __forceinline__ void bfly_max(T (&v)[TR], int k0, int nk)
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (k < k0 || k >= k0 + nk) continue;
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            if (r & (1 << k)) continue;
            const int s = r | (1 << k);
            if (UP) v[s] = v[s] > v[r] ? v[s] : v[r];
            else v[r] = v[r] > v[s] ? v[r] : v[s];
        }
    }
}

// 2^e for an integer e <= 0, built in the exponent bits (0 below 2^-126).
__device__ __forceinline__ float pow2i(int e)
{
    return __int_as_float(max(e + 127, 0) << 23);
}

// FP32 sum butterflies on values held relative to their own integer scales
// (the bits of `m` are ints: floor of the final max-plus transform): the
// partner is scaled by the exact power of two 2^(m(partner) - m(self)) <= 1.
template <bool UP>
__device__ __forceinline__ void bfly_pow2(float (&x)[TR], const float (&m)[TR], int k0, int nk)
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (k < k0 || k >= k0 + nk) continue;
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            if (r & (1 << k)) continue;
            const int s = r | (1 << k);
            const int mr = __float_as_int(m[r]), ms = __float_as_int(m[s]);
            if (UP) x[s] = madd(x[r], pow2i(mr - ms), x[s]);
            else x[r] = madd(x[s], pow2i(ms - mr), x[r]);
        }
    }
}

// Sum butterflies with bands e (exact small integers held as T).  Three
// cases per thread: all its bands equal (plain adds); two adjacent bands
// (factor 1 or e^-BW, one fused multiply-add); otherwise the full rule
// (1, e^-BW, or 0 for partners two or more bands down).
template <bool UP, typename T>
__device__ __forceinline__ void bfly_sum(T (&x)[TR], const T (&e)[TR], int k0, int nk)
{
    T lo = e[0], hi = e[0];
#pragma unroll
    for (int r = 1; r < TR; ++r) {
        lo = e[r] < lo ? e[r] : lo;
        hi = e[r] > hi ? e[r] : hi;
    }
    const T gap = hi - lo;
    if (gap == T(0)) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (k < k0 || k >= k0 + nk) continue;
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                if (r & (1 << k)) continue;
                const int s = r | (1 << k);
                if (UP) x[s] += x[r];
                else x[r] += x[s];
            }
        }
    } else if (gap == T(1)) {
        // partner bands differ by 0 or 1: factor 1 or e^-BW
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (k < k0 || k >= k0 + nk) continue;
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                if (r & (1 << k)) continue;
                const int s = r | (1 << k);
                if (UP) x[s] = madd(x[r], e[s] == e[r] ? T(1) : Band64::down1(), x[s]);
                else x[r] = madd(x[s], e[r] == e[s] ? T(1) : Band64::down1(), x[r]);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (k < k0 || k >= k0 + nk) continue;
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                if (r & (1 << k)) continue;
                const int s = r | (1 << k);
                const T dd = UP ? e[s] - e[r] : e[r] - e[s];
                const T f = dd == T(0) ? T(1) : (dd == T(1) ? Band64::down1() : T(0));
                if (UP) x[s] = madd(x[r], f, x[s]);
                else x[r] = madd(x[s], f, x[r]);
            }
        }
    }
}

template <bool UP>
__device__ __forceinline__ void sum_bfly(float (&x)[TR], const float (&m)[TR], int k0, int nk)
{
    bfly_pow2<UP>(x, m, k0, nk);
}
template <bool UP>
__device__ __forceinline__ void sum_bfly(double (&x)[TR], const double (&e)[TR], int k0, int nk)
{
    bfly_sum<UP>(x, e, k0, nk);
}
// Scale of an output from its max-plus value, the log that the scale stands
// for, and an output's log from its scaled value.  FP32: an integer (kept as
// the bits of a float); FP64: a band of BW nats.
__device__ __forceinline__ float scale_of(float m) { return __int_as_float(__float2int_rd(m)); }
__device__ __forceinline__ double scale_of(double m) { return floor(m / Band64::width); }
__device__ __forceinline__ float scale_base(float sc) { return (float)__float_as_int(sc); }
__device__ __forceinline__ double scale_base(double sc) { return Band64::width * sc; }
__device__ __forceinline__ float scaled_log(float y, float sc)
{
    return scale_base(sc) + LogOps<float>::lg(y);
}
__device__ __forceinline__ double scaled_log(double x, double e)
{
    return madd(Band64::width, e, LogOps<double>::lg(x));
}

// Online log-sum-exp step (branchless): (m, s) stands for m + lg(s).
template <typename T>
__device__ __forceinline__ void lse_online(T& m, T& s, T x)
{
    using Lg = LogOps<T>;
    const T mn = x > m ? x : m;
    if (mn == Lg::ninf()) return;
    s = s * Lg::ex(m - mn) + Lg::ex(x - mn);
    m = mn;
}

// a0 += b0 and a1 += b1 in one packed FP32 instruction (each lane rounds
// like a scalar add).
__device__ __forceinline__ void add_f32x2(float& a0, float& a1, float b0, float b1)
{
    unsigned long long ra, rb;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b0), "f"(b1));
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(ra) : "l"(rb));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(ra));
}

// Sum butterflies without bands (every value in one common scale).  In FP32
// a butterfly over register bit k >= 1 pairs registers r, r + 1 with s, s + 1:
// packed adds.
template <bool UP, typename T>
__device__ __forceinline__ void bfly_plain(T (&x)[TR], int k0, int nk)
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (k < k0 || k >= k0 + nk) continue;
        if constexpr (sizeof(T) == 4) {
            if (k >= 1) {
#pragma unroll
                for (int r = 0; r < TR; r += 2) {
                    if (r & (1 << k)) continue;
                    const int s = r | (1 << k);
                    if (UP) add_f32x2(x[s], x[s + 1], x[r], x[r + 1]);
                    else add_f32x2(x[r], x[r + 1], x[s], x[s + 1]);
                }
                continue;
            }
        }
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            if (r & (1 << k)) continue;
            const int s = r | (1 << k);
            if (UP) x[s] += x[r];
            else x[r] += x[s];
        }
    }
}

// Single-scale windows for both zeta tiles.  Pass p scales the terms by
// s_p = M - top - p * win (M bounds every output from above) and writes the
// outputs whose scaled value is at least 2^lo (e^lo): terms flushed below the
// smallest normal number (2^-126; e^-708) number at most 8192, under 2^-113
// (e^-699) in total, which is below 2^-33 (e^-99) of such an output.  An
// output left over has scaled value below 2^lo in pass p, hence below 2^top
// in pass p + 1, so no term of it overflows there (2^128; e^709).
template <typename T> struct Window;
// gap: how far below a relevance cut an output is held (64 bits; 45 nats).
template <> struct Window<float> {                 // bits
    static constexpr float top = 126.0f, lo = -80.0f, win = 206.0f, gap = 64.0f;
    static constexpr int max_pass = 2;     // a third pass costs more than the exact path
};
template <> struct Window<double> {                // nats
    static constexpr double top = 700.0, lo = -600.0, win = 1300.0, gap = 45.0;
    static constexpr int max_pass = 3;
};

// Layout loads and stores through the swizzled array.
template <typename T> __device__ __forceinline__ void ld1(const T* a, T (&v)[TR], int t)
{
#pragma unroll
    for (int r = 0; r < TR; ++r) v[r] = a[swz(el1(r, t))];
}
template <typename T> __device__ __forceinline__ void st1(T* a, const T (&v)[TR], int t)
{
#pragma unroll
    for (int r = 0; r < TR; ++r) a[swz(el1(r, t))] = v[r];
}
template <typename T> __device__ __forceinline__ void ld2(const T* a, T (&v)[TR], int t)
{
#pragma unroll
    for (int r = 0; r < TR; ++r) v[r] = a[swz(el2(r, t))];
}
template <typename T> __device__ __forceinline__ void st2(T* a, const T (&v)[TR], int t)
{
#pragma unroll
    for (int r = 0; r < TR; ++r) a[swz(el2(r, t))] = v[r];
}
// Layout 3: thread t owns four runs of 8 consecutive elements.
template <typename T> __device__ __forceinline__ void ld3(const T* a, T (&v)[TR], int t)
{
#pragma unroll
    for (int r = 0; r < TR; ++r) v[r] = a[swz(el3(r, t))];
}
template <> __device__ __forceinline__ void ld3<float>(const float* a, float (&v)[TR], int t)
{
    const bool flip = (t >> 2) & 1;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const uint32_t base = swz(el3(8 * x, t)) & ~7u;
        float4 p = *reinterpret_cast<const float4*>(a + base);
        float4 q = *reinterpret_cast<const float4*>(a + base + 4);
        if (flip) { float4 w = p; p = q; q = w; }
        v[8 * x + 0] = p.x; v[8 * x + 1] = p.y; v[8 * x + 2] = p.z; v[8 * x + 3] = p.w;
        v[8 * x + 4] = q.x; v[8 * x + 5] = q.y; v[8 * x + 6] = q.z; v[8 * x + 7] = q.w;
    }
}
template <typename T> __device__ __forceinline__ void st3(T* a, const T (&v)[TR], int t)
{
#pragma unroll
    for (int r = 0; r < TR; ++r) a[swz(el3(r, t))] = v[r];
}
template <> __device__ __forceinline__ void st3<float>(float* a, const float (&v)[TR], int t)
{
    const bool flip = (t >> 2) & 1;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const uint32_t base = swz(el3(8 * x, t)) & ~7u;
        float4 p = make_float4(v[8 * x + 0], v[8 * x + 1], v[8 * x + 2], v[8 * x + 3]);
        float4 q = make_float4(v[8 * x + 4], v[8 * x + 5], v[8 * x + 6], v[8 * x + 7]);
        if (flip) { float4 w = p; p = q; q = w; }
        *reinterpret_cast<float4*>(a + base) = p;
        *reinterpret_cast<float4*>(a + base + 4) = q;
    }
}
// Layout-3 values to global memory: registers 8q..8q+7 of thread t are the
// consecutive elements el3(8q, t) .. el3(8q, t) + 7 (32-byte aligned).
__device__ __forceinline__ void st_out3(float* out, const float (&x)[TR], int t)
{
#pragma unroll
    for (int q = 0; q < TR / 8; ++q) {
        float4* p = reinterpret_cast<float4*>(out + el3(8 * q, t));
        p[0] = make_float4(x[8 * q], x[8 * q + 1], x[8 * q + 2], x[8 * q + 3]);
        p[1] = make_float4(x[8 * q + 4], x[8 * q + 5], x[8 * q + 6], x[8 * q + 7]);
    }
}
__device__ __forceinline__ void st_out3(double* out, const double (&x)[TR], int t)
{
#pragma unroll
    for (int q = 0; q < TR / 8; ++q) {
        double2* p = reinterpret_cast<double2*>(out + el3(8 * q, t));
#pragma unroll
        for (int k = 0; k < 4; ++k) p[k] = make_double2(x[8 * q + 2 * k], x[8 * q + 2 * k + 1]);
    }
}

// The exact sum pass after the max-plus pass.  On entry v holds m (layout
// 3); A1 holds the transform's inputs (for UP only the slots with at most d
// elements are inputs).  On exit v and sc hold, in layout 1, each output as
// scaled_log(v, sc): FP32 keeps y relative to 2^floor(m), FP64 keeps x in
// its band.  The scales replace the inputs in A1: every thread reads its
// layout-3 inputs and writes its layout-3 scales to the same slots.
template <bool UP, typename T>
__device__ __forceinline__ void sum_pass(T (&v)[TR], T (&sc)[TR], T* A1, T* A0, int t, int d)
{
    using Lg = LogOps<T>;
    T* E = A1;
    const int pt = __popc(t);             // |el3(r, t)| = |r| + |t| (disjoint bits)
#pragma unroll
    for (int r = 0; r < TR; ++r) sc[r] = scale_of(v[r]);
    ld3(A1, v, t);                        // inputs
    st3(E, sc, t);                        // scales, read again in layouts 2 and 1
#pragma unroll
    for (int r = 0; r < TR; ++r)
        v[r] = (!UP || __popc(r) + pt <= d) ? Lg::ex(v[r] - scale_base(sc[r])) : T(0);
    sum_bfly<UP>(v, sc, 0, 3);
    __syncthreads();
    st3(A0, v, t);
    __syncthreads();
    ld2(A0, v, t);
    ld2(E, sc, t);
    sum_bfly<UP>(v, sc, 0, 5);
    __syncthreads();
    st2(A0, v, t);
    __syncthreads();
    ld1(A0, v, t);
    ld1(E, sc, t);
    sum_bfly<UP>(v, sc, 0, 5);
}

// Binomial coefficients C(a, b), a < 32, in shared memory, stored for
// b <= a / 2 only (C(a, b) = C(a, a - b)).  Lanes look up different entries,
// which would serialise constant-cache reads; the table is copied from a
// global-memory image with coalesced loads.
__device__ const BinomTable g_binom_image = make_binom_table();
struct SBinom {
    uint32_t v[32][16];
};
__device__ __forceinline__ void fill_sbinom(SBinom& sb)
{
    for (int x = threadIdx.x; x < 32 * 16; x += blockDim.x) sb.v[x >> 4][x & 15] = g_binom_image.v[x >> 4][x & 15];
}
__device__ __forceinline__ uint32_t sb_binom(const SBinom& sb, int a, int b)
{
    if (b < 0 || b > a) return 0u;
    return sb.v[a][min(b, a - b)];
}
__device__ __forceinline__ uint32_t sb_unrank(const SBinom& sb, uint32_t r, int nb, int* kout)
{
    int k = 0;
    while (r >= sb_binom(sb, nb, k)) { r -= sb_binom(sb, nb, k); ++k; }
    uint32_t x = 0;
    int c = nb - 1;
    for (int t = k; t >= 1; --t) {
        while (sb_binom(sb, c, t) > r) --c;
        x |= 1u << c;
        r -= sb_binom(sb, c, t);
        --c;
    }
    if (kout) *kout = k;
    return x;
}


uint64_t binom_host(int n, int k)
{
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int t = 1; t <= k; ++t) r = r * (uint64_t)(n - k + t) / (uint64_t)t;
    return r;
}

// Low patterns with at most d of the 13 tile bits (the columns of a tile).
uint32_t num_small_subsets_host(int d)
{
    uint64_t c = 0;
    for (int k = 0; k <= d && k <= TB; ++k) c += binom_host(TB, k);
    return (uint32_t)c;
}


}  // namespace

// ===========================================================================
// Families reordered by (high part G_H, low part g_L) for the tile scatter:
// row = rank of G_H among the subsets of the h = n-14 high index bits with at
// most d elements, column = rank of g_L among the subsets of the 13 low bits
// with at most d - |G_H| elements.  Row r of size k holds C13(<= d-k)
// columns, so the table holds exactly the K families of the node.
// ===========================================================================
__device__ __forceinline__ uint32_t row_offset(int h, int d, int kh, uint32_t rank_in_class)
{
    uint32_t off = 0;
    for (int k = 0; k < kh; ++k) off += binom(h, k) * num_small_subsets(TB, d - k);
    return off + rank_in_class * num_small_subsets(TB, d - kh);
}

template <typename T>
__global__ void k_reorder_up(int n, int d, int64_t K, const T* __restrict__ lbs, T* __restrict__ tab,
                             size_t js, int nodes)
{
    lbs = job_ptr(lbs, js);
    tab = job_ptr(tab, js);
    const int h = n - 1 - TB;
    const int64_t total = (int64_t)nodes * K;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(x / K);
        uint32_t f = (uint32_t)(x % K);
        int k = 0;
        while (f >= binom(n - 1, k)) { f -= binom(n - 1, k); ++k; }
        const uint32_t cm = colex_unrank(f, k, n - 1);
        const uint32_t gl = cm & (TN - 1u), gh = cm >> TB;
        const int kh = __popc(gh);
        // colex rank of gh within its size class
        uint32_t rk = 0;
        int t = 1;
        for (uint32_t y = gh; y; y &= y - 1, ++t) rk += binom(__ffs(y) - 1, t);
        const uint32_t col = small_subset_rank(gl, TB);
        tab[(size_t)i * K + row_offset(h, d, kh, rk) + col] = lbs[x];
    }
}

// ===========================================================================
// Step 2 for n >= 14, part 1: the column sums of tile (i, H) of A_i,
//   C_H(G_L) = log sum of B_i(G_H + G_L) over G_H inside H, |G_H| <= d - |G_L|,
// for every low pattern G_L (13 bits) with at most d elements, in column
// order (by size, then colex).  They go to the first ncol slots of the
// tile's own slice of A, which part 2 reads and then overwrites.  Small
// shared memory and register use keep many blocks resident, which hides the
// latency of the gathers from the score table.
// ===========================================================================
template <typename T>
__global__ void __launch_bounds__(TT, sizeof(T) == 4 ? 4 : 2)
k_upzeta13_cols(int n, int d, int64_t K, const T* __restrict__ tab, T* __restrict__ A, size_t js)
{
    tab = job_ptr(tab, js);
    A = job_ptr(A, js);
    using Lg = LogOps<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* part = reinterpret_cast<T*>(smem_raw);            // 2 * 8 * 96 partial (max, sum) pairs
    SBinom* sb = reinterpret_cast<SBinom*>(part + 2 * 8 * 96);
    int* meta = reinterpret_cast<int*>(sb + 1);          // [0,32) row offsets, [32,64) list starts
    uint32_t* off13 = reinterpret_cast<uint32_t*>(meta + 64);   // 16 entries
    uint32_t* rowbase = off13 + 16;                      // up to nrow entries
    const uint32_t ncol = num_small_subsets(TB, d);
    const int h = n - 1 - TB;

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int i = (int)(blockIdx.x >> h);
    const uint32_t H = blockIdx.x & ((1u << h) - 1u);
    const T* tb = tab + (size_t)i * K;
    T* out = A + ((size_t)i << (n - 1)) + ((size_t)H << TB);

    fill_sbinom(*sb);
    if (t < 16) {
        uint32_t o = 0;
        for (int k = 0; k < t && k <= TB; ++k) o += binom(TB, k);
        off13[t] = o;
    }
    __syncthreads();

    // --- rows whose high part lies inside H, in row order (by size, then
    //     colex): the k-element subsets of H in increasing mask order.  Entry
    //     p of the list is unranked among the subsets of H's hc positions,
    //     its positions are mapped onto the bits of H, and the row's offset in
    //     the node's table follows from its colex rank among all h-bit sets.
    const int hc = __popc(H);
    const int kmax = min(d, hc);
    if (t < 32) {
        // meta[32 + k]: first list entry of class k (entries of size k)
        meta[32 + t] = (int)num_small_subsets(hc, min(t, d + 1) - 1);
        // meta[k]: offset of the first class-k row in the node's table
        uint32_t o = 0;
        for (int k = 0; k < t && k <= min(d, h); ++k) o += binom(h, k) * off13[min(d - k, TB) + 1];
        meta[t] = (int)o;
    }
    __syncthreads();
    const int total = meta[32 + kmax + 1];
    for (int p = t; p < total; p += TT) {
        int k;
        const uint32_t loc = sb_unrank(*sb, (uint32_t)p, hc, &k);
        uint32_t rk = 0, hh = H;
        int q = 0, idx = 1;
        while (hh) {
            const int b = __ffs(hh) - 1;
            hh &= hh - 1;
            if (loc >> q & 1u) rk += sb_binom(*sb, b, idx++);
            ++q;
        }
        rowbase[p] = (uint32_t)meta[k] + rk * off13[min(d - k, TB) + 1];
    }
    __syncthreads();

    // --- per-column log-sum over the admissible rows, in a fixed order ------
    // Column c (low pattern of size j) takes the rows of size at most d - j,
    // i.e. the list prefix before the first row of size d - j + 1; a row of
    // size k holds the first W_k = off13[d - k + 1] columns.
    // Long columns (at most d - 2 low elements, many rows): warp w takes the
    // rows w, w + 8, ... and its lanes the columns of a 96-column block
    // (coalesced reads along the row); the eight warp partials are combined
    // in warp order.
    const uint32_t nlong = d >= 2 ? off13[min(d - 2, TB) + 1] : 0u;
    for (uint32_t cb = 0; cb < nlong; cb += 96) {
        T m[3], sm[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) { m[q] = Lg::ninf(); sm[q] = T(0); }
        // rows of size k hold W_k columns; only sizes with W_k > cb reach this block
        int kb = 0;
        while (kb < kmax && off13[min(d - kb - 1, TB) + 1] > cb) ++kb;
        const int pend = meta[32 + kb + 1];
        int k = 0;
        for (int p0 = warp; p0 < pend; p0 += 4 * (TT / 32)) {
            T x[4][3];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + u * (TT / 32);
                while (k < kb && p >= meta[32 + k + 1]) ++k;
                const uint32_t W = p < pend ? min(nlong, off13[min(d - k, TB) + 1]) : 0u;
                const T* src = tb + (p < pend ? rowbase[p] : 0u);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const uint32_t c = cb + lane + 32 * q;
                    x[u][q] = c < W ? src[c] : Lg::ninf();
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < 3; ++q) lse_online(m[q], sm[q], x[u][q]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            part[(warp * 96 + lane + 32 * q) * 2] = m[q];
            part[(warp * 96 + lane + 32 * q) * 2 + 1] = sm[q];
        }
        __syncthreads();
        if (t < 96 && cb + t < nlong) {
            T mx = Lg::ninf(), s2 = T(0);
#pragma unroll
            for (int w = 0; w < TT / 32; ++w) {
                const T mw = part[(w * 96 + t) * 2], sw = part[(w * 96 + t) * 2 + 1];
                const T mn = mw > mx ? mw : mx;
                if (mn != Lg::ninf()) {
                    s2 = s2 * Lg::ex(mx - mn) + sw * Lg::ex(mw - mn);
                    mx = mn;
                }
            }
            out[cb + t] = mx + Lg::lg(s2);
        }
        __syncthreads();
    }
    // Columns with d - 1 low elements: the row of the empty set and the
    // 1-element rows, 1 + hc of them; a thread per column.
    const uint32_t ncopy = off13[min(d, TB + 1)];     // first column with d low elements
    const int rmid = meta[32 + 2];
    for (uint32_t c = nlong + t; c < ncopy; c += TT) {
        T mx = Lg::ninf(), sm = T(0);
#pragma unroll 8
        for (int rp = 0; rp < rmid; ++rp) lse_online(mx, sm, tb[rowbase[rp] + c]);
        out[c] = mx + Lg::lg(sm);
    }
    // Columns with d low elements take the row of the empty set alone (offset 0).
    for (uint32_t c = ncopy + t; c < ncol; c += TT) out[c] = tb[c];
}

// Log-sum-exp kept lazily: (m, s) stands for m + log(s); s is rescaled only
// when a term exceeds m by more than 64 log units, so a term costs one
// exponential (the values are finite).
template <typename T>
__device__ __forceinline__ void lse_lazy(T& m, T& s, T x)
{
    using Lg = LogOps<T>;
    const T dd = x - m;                           // +inf while the accumulator is empty
    const bool big = dd > T(64);
    const T e = Lg::ex(big ? -dd : dd);
    s = big ? madd(s, e, T(1)) : s + e;
    m = big ? x : m;
}

// Part 1 with one warp per tile: each warp enumerates its tile's rows into
// its own list and sums the columns lane by lane (consecutive columns:
// coalesced reads of a row); no block barrier after the tables are filled.
// Columns with d low elements are copies, those with d - 1 take the 1 + |H|
// rows of at most one high element, the others every row of size at most
// d - |G_L|.
// Column sums by butterflies over the h high dimensions.  Blocks below
// nodes * ceil(ncb / CPB) take one node i and a run of CPB consecutive low
// columns c < ncb: the 2^h values B_i(G_H + G_L) of each column (zero where
// |G_H| > d - |G_L|) are gathered from the reordered table, the upward zeta
// over the subsets of every H follows in shared memory (h * 2^(h-1) steps
// per column, against sum_H C(|H|, <= d - |G_L|) terms summed directly: the
// better order once a column has many rows), and each C_H(G_L) goes to slot
// c of tile (i, H), the CPB columns of a run side by side.  The steps run
// three dimensions at a time in registers (eight values per thread), the
// columns held one after another in shared memory.
//
// Every output of a column lies between its H = {} value f(G_L) and its
// largest input plus log 2^h, so when that span is under one single-scale
// window (Window) for every column of the block, the sums run in linear
// scale (an exponential per input, an addition per step, a logarithm per
// output; exact as in the tiles); otherwise every step is a log-sum-exp.
// The blocks after those copy the columns from ncb on, whose sums have a
// single row (the empty high set), a warp per tile.
template <bool LIN, typename T>
__device__ __forceinline__ void colb_steps(T* v, uint32_t H2, int h, int CPB)
{
    using Lg = LogOps<T>;
    for (int j0 = 0; j0 < h; j0 += 3) {
        const int nb = min(3, h - j0);
        const uint32_t lowm = (1u << j0) - 1u;
        const uint32_t np = H2 >> nb;
        for (uint32_t g = threadIdx.x; g < np * CPB; g += blockDim.x) {
            const uint32_t cc = g / np, p = g % np;
            const uint32_t base = cc * H2 + (((p & ~lowm) << nb) | (p & lowm));
            T x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < (1 << nb)) x[q] = v[base + ((uint32_t)q << j0)];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (k >= nb) continue;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < (1 << nb) && (q >> k & 1)) x[q] = LIN ? x[q] + x[q ^ (1 << k)] : Lg::lse(x[q], x[q ^ (1 << k)]);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < (1 << nb)) v[base + ((uint32_t)q << j0)] = x[q];
        }
        __syncthreads();
    }
}

template <typename T, int CPB>
__global__ void __launch_bounds__(256)
k_upzeta13_colb(int n, int d, int64_t K, const T* __restrict__ tab, T* __restrict__ A,
                size_t js, int nodes, uint32_t ncb, int hc)
{
    tab = job_ptr(tab, js);
    A = job_ptr(A, js);
    using Lg = LogOps<T>;
    using Wn = Window<T>;
    __shared__ SBinom sb;
    __shared__ uint32_t off13[16];
    __shared__ uint32_t rowoff_k[32];
    __shared__ T wred[8][CPB];                       // the warps' column maxima
    __shared__ T scale_s[CPB];                       // a column's linear scale
    __shared__ int lin_s;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* v = reinterpret_cast<T*>(smem_raw);           // [column of the run][H]
    const int h = n - 1 - TB;
    // hc > 0: the top hc high bits are this block's chunk, fixed; the steps
    // run over the other hl bits and k_upzeta13_colt adds the chunks after
    const int hl = h - hc;
    const uint32_t H2 = 1u << hl;
    const uint32_t ncol = num_small_subsets(TB, d);
    const uint32_t nrun = (ncb + CPB - 1) / CPB;
    const uint32_t nbb = ((uint32_t)nodes * nrun) << hc;
    const size_t asize = (size_t)nodes << (n - 1);
    if (blockIdx.x >= nbb) {                         // copies: a warp per tile
        const uint32_t tile = (blockIdx.x - nbb) * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (tile >= ((uint32_t)nodes << h)) return;
        const T* tb = tab + (size_t)(tile >> h) * K;
        T* out = A + BN_AT((size_t)tile << TB, TN, asize);
        for (uint32_t c = ncb + (threadIdx.x & 31); c < ncol; c += 32) out[c] = tb[BN_AT(c, 1, K)];
        return;
    }
    fill_sbinom(sb);
    if (threadIdx.x < 16) {
        uint32_t o = 0;
        for (int k = 0; k < (int)threadIdx.x && k <= TB; ++k) o += binom(TB, k);
        off13[threadIdx.x] = o;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t o = 0;
        for (int k = 0; k < (int)threadIdx.x && k <= min(d, h); ++k)
            o += binom(h, k) * off13[min(d - k, TB) + 1];
        rowoff_k[threadIdx.x] = o;
    }
    __syncthreads();
    const uint32_t chunk = blockIdx.x & ((1u << hc) - 1u);
    const int i = (int)((blockIdx.x >> hc) / nrun);
    const uint32_t c0 = ((blockIdx.x >> hc) % nrun) * CPB;
    const uint32_t Hc = chunk << hl;                 // the chunk's high bits
    const T* tb = tab + (size_t)i * K;
    int kl[CPB];                                     // low elements of each column (-1: none)
    T mx[CPB];
#pragma unroll
    for (int cc = 0; cc < CPB; ++cc) {
        const uint32_t c = c0 + cc;
        int k = 0;
        while (k < TB && off13[k + 1] <= c) ++k;
        kl[cc] = c < ncb ? k : -1;
        mx[cc] = Lg::ninf();
    }
    for (uint32_t H = threadIdx.x; H < H2; H += blockDim.x) {
        const uint32_t Hf = Hc | H;
        const int kh = __popc(Hf);
        uint32_t r = 0;                              // colex rank of Hf among kh-subsets
        int t = 1;
        for (uint32_t x = Hf; x; x &= x - 1, ++t) r += sb_binom(sb, __ffs(x) - 1, t);
        // the row of G_H in the node's table (only formed where some column reads it)
        const uint32_t row = kh <= d ? rowoff_k[kh] + r * off13[min(d - kh, TB) + 1] : 0u;
#pragma unroll
        for (int cc = 0; cc < CPB; ++cc) {
            const bool in = kl[cc] >= 0 && kh <= d - kl[cc];
            const T val = in ? tb[BN_AT(row + c0 + cc, 1, K)] : Lg::ninf();
            v[cc * H2 + H] = val;
            mx[cc] = val > mx[cc] ? val : mx[cc];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int cc = 0; cc < CPB; ++cc) {
        for (int o = 16; o; o >>= 1) {
            const T y = __shfl_xor_sync(FULLMASK, mx[cc], o);
            mx[cc] = y > mx[cc] ? y : mx[cc];
        }
        if (lane == 0) wred[warp][cc] = mx[cc];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // a column's outputs lie in [f(G_L), its largest input + log 2^h]
        const T hb = sizeof(T) == 4 ? T(hl) : T(hl) * T(0.69314718055994530942);
        int lin = 1;
        for (int cc = 0; cc < CPB; ++cc) {
            T m = wred[0][cc];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wred[w][cc] > m ? wred[w][cc] : m;
            const T top = m + hb;
            scale_s[cc] = top - Wn::top;
            if (kl[cc] >= 0 && !(top - v[cc * H2] < Wn::win)) lin = 0;
        }
        lin_s = lin;
    }
    __syncthreads();
    const bool lin = lin_s != 0;
    if (lin) {
        for (uint32_t e = threadIdx.x; e < H2 * CPB; e += blockDim.x) v[e] = Lg::ex(v[e] - scale_s[e / H2]);
        __syncthreads();
        colb_steps<true>(v, H2, hl, CPB);
    } else {
        colb_steps<false>(v, H2, hl, CPB);
    }
    T* Ai = A + ((size_t)i << (n - 1));
    for (uint32_t H = threadIdx.x; H < H2; H += blockDim.x) {
        T* o = Ai + BN_AT(((size_t)(Hc | H) << TB) + c0, CPB, (size_t)1 << (n - 1));
        T y[CPB];
#pragma unroll
        for (int cc = 0; cc < CPB; ++cc) {
            const T x = v[cc * H2 + H];
            y[cc] = lin ? scale_s[cc] + Lg::lg(x) : x;
        }
        if constexpr (sizeof(T) == 4 && CPB == 4) {
            if (c0 + 4 <= ncb) {
                *reinterpret_cast<float4*>(o) = make_float4(y[0], y[1], y[2], y[3]);
                continue;
            }
        }
#pragma unroll
        for (int cc = 0; cc < CPB; ++cc)
            if (c0 + cc < ncb) o[cc] = y[cc];
    }
}

// The chunks of the column butterflies (k_upzeta13_colb with hc > 0): slot c
// of tile (i, (q << hl) | L) holds the sum over the rows inside chunk q
// alone; the upward zeta over the hc chunk bits, a thread per (i, L, c) with
// c fastest (coalesced), leaves the full column sums.
template <typename T>
__global__ void __launch_bounds__(256)
k_upzeta13_colt(int n, T* __restrict__ A, int nodes, uint32_t ncb, int hc)
{
    using Lg = LogOps<T>;
    const int h = n - 1 - TB, hl = h - hc;
    const uint64_t total = ((uint64_t)nodes << hl) * ncb;
    const size_t asize = (size_t)nodes << (n - 1);
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < total;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(x % ncb);
        const uint64_t y = x / ncb;
        const uint32_t L = (uint32_t)(y & ((1u << hl) - 1u));
        const int i = (int)(y >> hl);
        T* Ai = A + ((size_t)i << (n - 1));
        T q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < (1 << hc)) q[k] = Ai[BN_AT((((size_t)k << hl) | L) << TB | c, 1, asize)];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b >= hc) continue;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < (1 << hc) && (k >> b & 1)) q[k] = Lg::lse(q[k], q[k ^ (1 << b)]);
        }
#pragma unroll
        for (int k = 1; k < 8; ++k)
            if (k < (1 << hc)) Ai[BN_AT((((size_t)k << hl) | L) << TB | c, 1, asize)] = q[k];
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_upzeta13_colw(int n, int d, int64_t K, const T* __restrict__ tab, T* __restrict__ A, size_t js,
                int nodes)
{
    tab = job_ptr(tab, js);
    A = job_ptr(A, js);
    using Lg = LogOps<T>;
    __shared__ SBinom sb;
    __shared__ uint32_t off13[16];
    __shared__ uint32_t rowoff_k[32];            // offset of the first size-k row in a node's table
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int h = n - 1 - TB;
    const uint32_t nrow = num_small_subsets(h, d);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* rowbase = reinterpret_cast<uint32_t*>(smem_raw) + (size_t)warp * nrow;
    fill_sbinom(sb);
    if (threadIdx.x < 16) {
        uint32_t o = 0;
        for (int k = 0; k < (int)threadIdx.x && k <= TB; ++k) o += binom(TB, k);
        off13[threadIdx.x] = o;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t o = 0;
        for (int k = 0; k < (int)threadIdx.x && k <= min(d, h); ++k)
            o += binom(h, k) * off13[min(d - k, TB) + 1];
        rowoff_k[threadIdx.x] = o;
    }
    __syncthreads();
    const uint32_t ncol = num_small_subsets(TB, d);
    const uint32_t nlong = d >= 2 ? off13[min(d - 2, TB) + 1] : 0u;
    const uint32_t ncopy = off13[min(d, TB + 1)];
    const uint32_t ntiles = (uint32_t)nodes << h;
    const uint32_t wpb = blockDim.x >> 5;
    for (uint32_t tile = blockIdx.x * wpb + warp; tile < ntiles; tile += gridDim.x * wpb) {
        const int i = (int)(tile >> h);
        const uint32_t H = tile & ((1u << h) - 1u);
        const T* tb = tab + (size_t)i * K;
        T* out = A + BN_AT(((size_t)i << (n - 1)) + ((size_t)H << TB), TN, (size_t)nodes << (n - 1));
        const int hc = __popc(H);
        uint32_t total = 0;                      // rows of size <= d inside H
        for (int k = 0; k <= d && k <= hc; ++k) total += sb_binom(sb, hc, k);
        for (uint32_t p = lane; p < total; p += 32) {
            int k;
            const uint32_t loc = sb_unrank(sb, p, hc, &k);
            uint32_t rk = 0, hh = H;
            int q = 0, idx = 1;
            while (hh) {
                const int b = __ffs(hh) - 1;
                hh &= hh - 1;
                if (loc >> q & 1u) rk += sb_binom(sb, b, idx++);
                ++q;
            }
            rowbase[p] = rowoff_k[k] + rk * off13[min(d - k, TB) + 1];
        }
        __syncwarp();
        for (uint32_t c = lane; c < nlong; c += 32) {          // at most d - 2 low elements
            int j = 0;
            while (off13[j + 1] <= c) ++j;
            uint32_t rend = 0;
            for (int k = 0; k <= d - j && k <= hc; ++k) rend += sb_binom(sb, hc, k);
            T m = Lg::ninf(), s = T(0);
#pragma unroll 4
            for (uint32_t rp = 0; rp < rend; ++rp) lse_lazy(m, s, tb[BN_AT(rowbase[rp] + c, 1, K)]);
            out[c] = m + Lg::lg(s);
        }
        const uint32_t rmid = 1u + (uint32_t)hc;               // d - 1 low elements
        for (uint32_t c = nlong + lane; c < ncopy; c += 32) {
            T m = Lg::ninf(), s = T(0);
#pragma unroll 4
            for (uint32_t rp = 0; rp < rmid; ++rp) lse_lazy(m, s, tb[BN_AT(rowbase[rp] + c, 1, K)]);
            out[c] = m + Lg::lg(s);
        }
        for (uint32_t c = ncopy + lane; c < ncol; c += 32) out[c] = tb[c];   // d low elements
        __syncwarp();                                          // rowbase is reused
    }
}

// ===========================================================================
// Step 2 for n >= 14, part 2: one block per tile (i, H) of A_i.  The column
// sums of part 1 are placed at their low patterns (every other slot holds
// zero) and the truncated upward zeta over the 13 low bits follows.
// ===========================================================================
//
// TLO: the rows of A in tile-level order (see bn_device.cuh): output element
// e of the tile goes to row place(e >> lw) of the tile's block.
template <typename T, bool TLO>
__global__ void __launch_bounds__(TT, sizeof(T) == 4 ? 2 : 1)
k_upzeta13(int n, int d, const uint16_t* __restrict__ unrank13, T* __restrict__ A, size_t js)
{
    unrank13 = job_ptr(unrank13, js);
    A = job_ptr(A, js);
    using Lg = LogOps<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* A0 = reinterpret_cast<T*>(smem_raw);
    T* A1 = A0 + TN;
    T* wmax = A1 + TN;                           // each warp's largest column sum
    const uint32_t ncol = num_small_subsets(TB, d);
    const int h = n - 1 - TB;
    const int t = threadIdx.x, lane = t & 31;
    const int i = (int)(blockIdx.x >> h);
    const uint32_t H = blockIdx.x & ((1u << h) - 1u);
    T* out = A + BN_AT(((size_t)i << (n - 1)) + ((size_t)H << TB), TN, (size_t)gridDim.x << TB);
    // place of element e in the tile's block
    const int lw = i < 4 ? 3 : 4;                // row width of A_i in step 3
    const uint32_t lmask = (1u << lw) - 1u;
    auto opos = [&](uint32_t e) -> uint32_t {
        if (!TLO) return e;
        const uint32_t r = e >> lw;
        return ((lw == 4 ? g_place.p9[r] : g_place.p10[r]) << lw) | (e & lmask);
    };

    // |el1(r, t)| = |r| + |t| (disjoint bits): the slots with more than d
    // elements are no column (no input)
    const int pt = __popc(t);
    T tm = Lg::ninf();
    for (uint32_t c = t; c < ncol; c += TT) {
        const T v = out[c];
        const uint32_t sw = swz(BN_AT(unrank13[c], 1, TN));
        A0[sw] = A1[sw] = v;
        tm = v > tm ? v : tm;
    }
    for (int o = 16; o; o >>= 1) {
        const T o2 = __shfl_xor_sync(FULLMASK, tm, o);
        tm = o2 > tm ? o2 : tm;
    }
    if (lane == 0) wmax[t >> 5] = tm;
    __syncthreads();                             // columns placed, warp maxima written
    T tmx = wmax[0];
#pragma unroll
    for (int w = 1; w < TT / 32; ++w) tmx = wmax[w] > tmx ? wmax[w] : tmx;

    // --- single-scale passes (Window): pass p sums linear values 2^(x - s_p)
    //     (e^(x - s_p) in FP64) with s_p = M - top - p * win and writes the
    //     outputs it resolves; the last pass writes every output left.  Every
    //     output is at least C(empty) and at most M, so ceil((M - C(empty)) /
    //     win) passes resolve the tile.  Tiles that need more than
    //     Window::max_pass passes take the banded path below.
    {
        using Wn = Window<T>;
        const T M = tmx + T(TB);
        const T span = M - A1[0];
        // spans past max_pass windows (a zero weight held as -1e7 nats gives an
        // empty-set column far below the rest) and NaN go to the exact path
        // without converting the span to an integer
        const int npass = span < Wn::win ? 1
                          : span < T(Wn::max_pass) * Wn::win ? (int)ceil(span / Wn::win)
                                                             : Wn::max_pass + 1;
        if (npass == 1) {                        // one window holds the whole tile
            const T sp = M - Wn::top;
            T x[TR];
            ld1(A1, x, t);
#pragma unroll
            for (int r = 0; r < TR; ++r)
                x[r] = (__popc(r) + pt <= d) ? Lg::ex(x[r] - sp) : T(0);
            bfly_plain<true>(x, 0, 5);
            st1(A0, x, t);
            __syncthreads();
            ld2(A0, x, t);
            bfly_plain<true>(x, 0, 5);
            st2(A0, x, t);
            __syncthreads();
            ld3(A0, x, t);
            bfly_plain<true>(x, 0, 3);
#pragma unroll
            for (int r = 0; r < TR; ++r) x[r] = sp + Lg::lg(x[r]);
            if constexpr (TLO) {
                // a run of 8 consecutive elements stays inside one row (lw >= 3)
#pragma unroll
                for (int q = 0; q < TR / 8; ++q) {
                    float4* p = reinterpret_cast<float4*>(out + BN_AT(opos(el3(8 * q, t)), 8, TN));
                    p[0] = make_float4(x[8 * q], x[8 * q + 1], x[8 * q + 2], x[8 * q + 3]);
                    p[1] = make_float4(x[8 * q + 4], x[8 * q + 5], x[8 * q + 6], x[8 * q + 7]);
                }
            } else {
                st_out3(out, x, t);
            }
            return;
        }
        if (npass <= Wn::max_pass) {
            uint32_t done = 0u;                  // bit r: output el3(r, t) written
            // registers 8q..8q+7 (layout 3) are 8 consecutive elements of one
            // row: their places start at run3[q]
            uint32_t run3[TR / 8];
#pragma unroll
            for (int q = 0; q < TR / 8; ++q) run3[q] = BN_AT(opos(el3(8 * q, t)), 8, TN);
            T sp = M - Wn::top;
            for (int p = 0; p < npass; ++p, sp -= Wn::win) {
                const bool last = p + 1 == npass;
                T x[TR];
                ld1(A1, x, t);
#pragma unroll
                for (int r = 0; r < TR; ++r)
                    x[r] = (__popc(r) + pt <= d) ? Lg::ex(x[r] - sp) : T(0);
                bfly_plain<true>(x, 0, 5);
                st1(A0, x, t);
                __syncthreads();
                ld2(A0, x, t);
                bfly_plain<true>(x, 0, 5);
                st2(A0, x, t);
                __syncthreads();
                ld3(A0, x, t);
                bfly_plain<true>(x, 0, 3);
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const T lx = Lg::lg(x[r]);
                    if (!(done >> r & 1u) && (last || lx >= Wn::lo)) {
                        out[run3[r >> 3] + (r & 7)] = sp + lx;
                        done |= 1u << r;
                    }
                }
                if (last) break;
                if (__syncthreads_and(done == 0xffffffffu)) break;   // also guards A0 reuse
            }
            return;
        }
    }

    // --- max-plus pass: layouts 1, 2, 3 ------------------------------------
#pragma unroll
    for (int r = 0; r < TR; ++r)                 // no term: zero (slots that are no column)
        if (__popc(r) + pt > d) A0[swz(el1(r, t))] = Lg::ninf();
    __syncthreads();
    T v[TR];
    ld1(A0, v, t);
    bfly_max<true>(v, 0, 5);
    st1(A0, v, t);
    __syncthreads();
    ld2(A0, v, t);
    bfly_max<true>(v, 0, 5);
    st2(A0, v, t);
    __syncthreads();
    ld3(A0, v, t);
    bfly_max<true>(v, 0, 3);

    // --- exact sum pass: layouts 3, 2, 1 ------------------------------------
    T sc[TR];
    sum_pass<true>(v, sc, A1, A0, t, d);
#pragma unroll
    for (int r = 0; r < TR; ++r) out[BN_AT(opos(el1(r, t)), 1, TN)] = scaled_log(v[r], sc[r]);
}

// The same tiles (FP32) in a persistent kernel: each block takes tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Thread 0 keeps the next tile's
// column sums in flight while the block transforms the current one (one bulk
// copy into shared memory, counted by an mbarrier), and every finished tile
// leaves as one 32 KB bulk store from a shared-memory staging block, so the
// block's threads issue neither the loads nor the stores.  The arithmetic
// and the outputs are those of k_upzeta13, bit for bit.  Shared memory: A0
// (exchanges), A1 (inputs), the warps' maxima, the mbarrier and a flag, the
// staged column sums (ncol floats rounded up to 16 bytes, and 48 bytes more)
// and the output block.  With ncb < ncol the columns from ncb on (d low
// elements: the sum of one row, the empty high set) were not written by the
// column-sum kernel; they are the first ncol entries of node i's reordered
// score table `tab` (K entries per node, K a multiple of 4), and a second
// bulk copy stages them, from the 16-byte boundary at or below ncb.  A bulk
// copy that has not landed after `cap` polls of its mbarrier sets
// kErrDeviceTimeout in *err and the block returns after one more bounded
// wait for it.  `hold` (a test hook, 0 otherwise) withholds the block's
// first copies, so that its wait runs out.
template <bool TLO>
__global__ void __launch_bounds__(TT, 2)
k_upzeta13p(int n, int d, const uint16_t* __restrict__ unrank13, float* __restrict__ A, uint32_t ntiles,
            int* __restrict__ err, uint32_t cap, int hold, const float* __restrict__ tab, int64_t K,
            uint32_t ncb)
{
    using Lg = LogOps<float>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* A0 = reinterpret_cast<float*>(smem_raw);
    float* A1 = A0 + TN;
    float* wmax = A1 + TN;                               // TT / 32 floats
    uint64_t* bar = reinterpret_cast<uint64_t*>(wmax + TT / 32);
    int* gave_up = reinterpret_cast<int*>(bar + 1);
    float* S = reinterpret_cast<float*>(bar + 2);       // staged column sums
    const uint32_t ncol = num_small_subsets(TB, d);
    float* OUT = S + ((ncol * 4u + 15u) & ~15u) / 4 + 12; // the finished tile
    const int h = n - 1 - TB;
    const size_t asize = (size_t)ntiles << TB;
    // the tile's columns (before ncb) and, from the table, the rest
    const uint32_t ncb4 = ncb & ~3u;
    const uint32_t sbytes = (ncb * 4u + 15u) & ~15u;
    const uint32_t tbytes = ncb < ncol ? ((ncol - ncb4) * 4u + 15u) & ~15u : 0u;
    float* S2 = S + sbytes / 4;
    const int t = threadIdx.x, lane = t & 31;
    const int pt = __popc(t);
    // thread 0: the copies of tile `tl` on the barrier
    auto stage = [&](uint32_t tl) {
        mbar_expect(bar, sbytes + tbytes);
        bulk_copy_in(S, A + BN_AT((size_t)tl << TB, TN, asize), sbytes, bar);
        if (tbytes)
            bulk_copy_in(S2, tab + BN_AT((size_t)(tl >> h) * K + ncb4, 4, (size_t)(ntiles >> h) * K), tbytes, bar);
    };
    if (t == 0) mbar_init(bar, 1);
    __syncthreads();
    uint32_t tile = blockIdx.x;
    if (t == 0 && tile < ntiles && !hold) stage(tile);
    for (uint32_t parity = 0; tile < ntiles; tile += gridDim.x, parity ^= 1u) {
        const int i = (int)(tile >> h);
        float* out = A + BN_AT((size_t)tile << TB, TN, asize);
        const int lw = i < 4 ? 3 : 4;
        const uint32_t lmask = (1u << lw) - 1u;
        auto opos = [&](uint32_t e) -> uint32_t {
            if (!TLO) return e;
            const uint32_t r = e >> lw;
            return ((lw == 4 ? g_place.p9[r] : g_place.p10[r]) << lw) | (e & lmask);
        };
        if (t == 0) {
            bulk_wait_read();                            // the last tile's store has read OUT
            *gave_up = mbar_wait_bounded(bar, parity, cap) ? 0 : 1;
        }
        __syncthreads();
        if (*gave_up) {
            if (t == 0) {
                atomicOr(err, kErrDeviceTimeout);
                mbar_wait_bounded(bar, parity, cap);     // let a copy in flight land
                bulk_wait();
            }
            return;
        }
        // |el1(r, t)| = |r| + |t| (disjoint bits): the slots with more than d
        // elements are no column (no input)
        float tm = Lg::ninf();
        for (uint32_t c = t; c < ncol; c += TT) {
            const float v = c < ncb ? S[c] : S2[c - ncb4];
            A1[swz(BN_AT(unrank13[c], 1, TN))] = v;
            tm = v > tm ? v : tm;
        }
        for (int o = 16; o; o >>= 1) {
            const float o2 = __shfl_xor_sync(FULLMASK, tm, o);
            tm = o2 > tm ? o2 : tm;
        }
        if (lane == 0) wmax[t >> 5] = tm;
        fence_async_shared();                            // S is read: the next copy may land
        __syncthreads();
        if (t == 0 && tile + gridDim.x < ntiles) stage(tile + gridDim.x);
        float tmx = wmax[0];
#pragma unroll
        for (int w = 1; w < TT / 32; ++w) tmx = wmax[w] > tmx ? wmax[w] : tmx;

        // single-scale passes as in k_upzeta13
        using Wn = Window<float>;
        const float M = tmx + float(TB);
        const float span = M - A1[0];
        const int npass = span < Wn::win ? 1
                          : span < float(Wn::max_pass) * Wn::win ? (int)ceilf(span / Wn::win)
                                                                 : Wn::max_pass + 1;
        if (npass == 1) {
            const float sp = M - Wn::top;
            float x[TR];
            ld1(A1, x, t);
#pragma unroll
            for (int r = 0; r < TR; ++r) x[r] = (__popc(r) + pt <= d) ? Lg::ex(x[r] - sp) : 0.0f;
            bfly_plain<true>(x, 0, 5);
            st1(A0, x, t);
            __syncthreads();
            ld2(A0, x, t);
            bfly_plain<true>(x, 0, 5);
            st2(A0, x, t);
            __syncthreads();
            ld3(A0, x, t);
            bfly_plain<true>(x, 0, 3);
#pragma unroll
            for (int r = 0; r < TR; ++r) x[r] = sp + Lg::lg(x[r]);
            // a run of 8 consecutive elements stays inside one row (lw >= 3)
#pragma unroll
            for (int q = 0; q < TR / 8; ++q) {
                float4* p = reinterpret_cast<float4*>(OUT + BN_AT(opos(el3(8 * q, t)), 8, TN));
                p[0] = make_float4(x[8 * q], x[8 * q + 1], x[8 * q + 2], x[8 * q + 3]);
                p[1] = make_float4(x[8 * q + 4], x[8 * q + 5], x[8 * q + 6], x[8 * q + 7]);
            }
        } else if (npass <= Wn::max_pass) {
            uint32_t done = 0u;                          // bit r: output el3(r, t) written
            uint32_t run3[TR / 8];
#pragma unroll
            for (int q = 0; q < TR / 8; ++q) run3[q] = BN_AT(opos(el3(8 * q, t)), 8, TN);
            float sp = M - Wn::top;
            for (int p = 0; p < npass; ++p, sp -= Wn::win) {
                const bool last = p + 1 == npass;
                float x[TR];
                ld1(A1, x, t);
#pragma unroll
                for (int r = 0; r < TR; ++r) x[r] = (__popc(r) + pt <= d) ? Lg::ex(x[r] - sp) : 0.0f;
                bfly_plain<true>(x, 0, 5);
                st1(A0, x, t);
                __syncthreads();
                ld2(A0, x, t);
                bfly_plain<true>(x, 0, 5);
                st2(A0, x, t);
                __syncthreads();
                ld3(A0, x, t);
                bfly_plain<true>(x, 0, 3);
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const float lx = Lg::lg(x[r]);
                    if (!(done >> r & 1u) && (last || lx >= Wn::lo)) {
                        OUT[run3[r >> 3] + (r & 7)] = sp + lx;
                        done |= 1u << r;
                    }
                }
                if (last) break;
                if (__syncthreads_and(done == 0xffffffffu)) break;   // also guards A0 reuse
            }
        } else {
            // max-plus pass, then the exact sum pass (k_upzeta13)
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                const uint32_t sw = swz(el1(r, t));
                A0[sw] = __popc(r) + pt > d ? Lg::ninf() : A1[sw];
            }
            __syncthreads();
            float v[TR];
            ld1(A0, v, t);
            bfly_max<true>(v, 0, 5);
            st1(A0, v, t);
            __syncthreads();
            ld2(A0, v, t);
            bfly_max<true>(v, 0, 5);
            st2(A0, v, t);
            __syncthreads();
            ld3(A0, v, t);
            bfly_max<true>(v, 0, 3);
            float sc[TR];
            sum_pass<true>(v, sc, A1, A0, t, d);
#pragma unroll
            for (int r = 0; r < TR; ++r) OUT[BN_AT(opos(el1(r, t)), 1, TN)] = scaled_log(v[r], sc[r]);
        }
        fence_async_shared();                            // OUT is written: the store may read it
        __syncthreads();
        if (t == 0) bulk_store(out, OUT, TN * 4u);
    }
    if (t == 0) bulk_wait();
}

// ===========================================================================
// Step 4, phase 1 for n >= 14: one block per tile H of the n-1 bits of S
// (bit v removed); s_v(S) = F(S) + R'(S + {v}); keeps the outputs with at
// most d low elements in row H of W.
// ===========================================================================
//
// Relevance cut (when Aup is given).  Every output W[H][g] reaches a
// posterior only through B_v(G) Gamma_v(G) / F(V) with G inside the tile's
// full set S_H = H + all 13 low bits, and B_v(G) <= A_v(S_H).  An output
// below L = F(V) - margin - A_v(S_H) therefore moves no posterior by more than
// 2^-margin, and the K * 2^h outputs of v together by at most
// K 2^h 2^-margin; the launcher takes margin = 64 + log2(K 2^h) bits in FP64
// and 24 + log2(K 2^h) in FP32, so the total is below 2^-64 (resp. 2^-24,
// against the FP32 tolerance of 1e-4).  A tile whose upper bound M is below L writes every
// output as L - gap (no butterflies); a tile within one window of
// max(L, s(full)) takes the single-scale pass, its outputs held at >= L - gap.
// Outputs at or above L are exact as before.  The written value, like the
// true one, is below 2^L: the error of such an output is within the bound.
template <typename T, bool Q>
__global__ void __launch_bounds__(TT, sizeof(T) == 4 ? 3 : 1)
k_gamma13_p1(int n, int d, uint32_t nlow, const T* __restrict__ F,
             const T* __restrict__ Rc, const uint16_t* __restrict__ rank13, T* __restrict__ W,
             size_t js, const T* __restrict__ lq, const T* __restrict__ Aup, T margin,
             uint32_t vsel)
{
    // block x = tile H * n + endpoint v: the blocks running at once are
    // the n endpoints of a few neighbouring tiles, whose gathers of F and R'
    // fall on the same rows, so L2 serves most of them (against one endpoint's
    // tiles at a time: 1.99 -> 1.79 ms at n = 26)
    const int v = (int)(blockIdx.x % (unsigned)n);
    const uint32_t ntile = gridDim.x / (unsigned)n;
    if (!(vsel >> v & 1u)) return;                  // an endpoint another rank computes
    F = job_ptr(F, js);
    Rc = job_ptr(Rc, js);
    rank13 = job_ptr(rank13, js);
    const uint16_t* unrank13 = rank13 + TN;         // the inverse table follows
    W = job_ptr(W, js) + (size_t)endpoint_slot(vsel, v) * ntile * nlow;
    using Lg = LogOps<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* A0 = reinterpret_cast<T*>(smem_raw);
    T* A1 = A0 + TN;
    const int t = threadIdx.x;
    const uint32_t H = blockIdx.x / (unsigned)n;
    const uint32_t bv = 1u << v;

    using O = typename OrdInt<T>::type;
    constexpr bool kBases = sizeof(T) == 4;         // FP32: per-level bases of F and R'
    __shared__ O tmax_s;
    __shared__ T sfull_s;
    __shared__ T lq_s[Q ? 32 : 1];                  // q_v by |S| (Eq. 12), when given
    __shared__ float off_s[32];                     // F + R' - Z by level (bn_device.cuh)
    __shared__ int sh_s;
    __shared__ float fvrel_s;
    if (t == 0) tmax_s = ord_enc(Lg::ninf());
    if (Q && t < n) lq_s[t] = lq[v * n + t];
    T x[TR];
#pragma unroll
    for (int r = 0; r < TR; ++r) {                  // the tile's loads go out first
        const uint32_t S = expand((H << TB) | el1(r, t), v);
        x[r] = F[BN_AT(S, 1, (size_t)1 << n)] + Rc[BN_AT(S | bv, 1, (size_t)1 << n)];
    }
    if constexpr (kBases)                           // while they are in flight
        load_gamma_offsets(reinterpret_cast<const float*>(Rc), n, v, off_s, &sh_s, &fvrel_s);
    __syncthreads();
    T mx = Lg::ninf();
    // The level of element el1(r, t) is |S >> 4| = |H| + |t without its low
    // bits| + |r| (bit v, outside S, shifts the low bits of t by one when
    // v < 4), so a thread needs six offsets, indexed by |r| <= 5.
    float offr[6];
    if constexpr (kBases) {
        const int lowm = v >= kLevelShift ? 15 : 7;
        const int bt = sh_s == kLevelShift ? __popc(H) + __popc(t & ~lowm) : 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) offr[k] = off_s[BN_AT(sh_s == kLevelShift ? bt + k : 0, 1, 32)];
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        if constexpr (kBases) x[r] += offr[__popc(r)];
        if (Q) x[r] += lq_s[__popc(expand((H << TB) | el1(r, t), v))];
        mx = x[r] > mx ? x[r] : mx;
    }
    for (int o = 16; o; o >>= 1) {
        const T y = __shfl_xor_sync(FULLMASK, mx, o);
        mx = y > mx ? y : mx;
    }
    if ((t & 31) == 0) atomicMax(&tmax_s, ord_enc(mx));
    if (t == TT - 1) sfull_s = x[TR - 1];            // s of the full tile set (element 8191)
    __syncthreads();
    T* row = W + (size_t)H * nlow;
    {
        // every output T (|T| <= d) sums s over its supersets, the full set
        // included: it lies between s(full) and M, so a tile that spans
        // less than one window resolves in one single-scale pass (Window)
        const T M = ord_dec(tmax_s) + T(TB);
        T L = Lg::ninf();                           // relevance cut (see above)
        if (Aup) {
            const T at = job_ptr(Aup, js)[BN_AT(((size_t)v << (n - 1)) + (((size_t)H << TB) | (TN - 1)), 1,
                                                (size_t)n << (n - 1))];
            // log P(D) in the units of s (FP32: relative to the integer Z)
            const T fv = kBases ? (T)fvrel_s : F[((size_t)1 << n) - 1];
            L = fv - margin - at;
        }
        const T floorv = L - Window<T>::gap;
        if (M < L) {                                // nothing in the tile matters
            for (uint32_t c = t; c < nlow; c += TT) row[BN_AT(c, 1, nlow)] = floorv;
            return;
        }
        if (M - (L > sfull_s ? L : sfull_s) < Window<T>::win) {
            const T sp = M - Window<T>::top;
#pragma unroll
            for (int r = 0; r < TR; ++r) x[r] = Lg::ex(x[r] - sp);
            bfly_plain<false>(x, 0, 5);
            st1(A0, x, t);
            __syncthreads();
            ld2(A0, x, t);
            bfly_plain<false>(x, 0, 5);
            st2(A0, x, t);
            __syncthreads();
            ld3(A0, x, t);
            bfly_plain<false>(x, 0, 3);
            if constexpr (sizeof(T) == 8) {
                // only the outputs with at most d elements are kept: back to
                // shared memory (each thread rewrites the slots it read), then
                // a logarithm (many FP64 instructions) per kept output, stored
                // in rank order
                st3(A0, x, t);
                __syncthreads();
                for (uint32_t c = t; c < nlow; c += TT) {
                    const T o = sp + Lg::lg(A0[swz(BN_AT(unrank13[c], 1, TN))]);
                    row[BN_AT(c, 1, nlow)] = o > floorv ? o : floorv;
                }
            } else {
                // FP32: a logarithm per register, kept outputs stored in place
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const uint32_t el = el3(r, t);
                    const T o = sp + Lg::lg(x[r]);
                    if (__popc(el) <= d) row[BN_AT(rank13[el], 1, nlow)] = o > floorv ? o : floorv;
                }
            }
            return;
        }
    }
    st1(A1, x, t);                        // s_v kept for the band pass
    bfly_max<false>(x, 0, 5);
    st1(A0, x, t);
    __syncthreads();
    ld2(A0, x, t);
    bfly_max<false>(x, 0, 5);
    st2(A0, x, t);
    __syncthreads();
    ld3(A0, x, t);
    bfly_max<false>(x, 0, 3);

    T sc[TR];
    sum_pass<false>(x, sc, A1, A0, t, d);
    if constexpr (sizeof(T) == 8) {
        // the kept outputs in rank order, as in the single-scale pass; each
        // thread rewrites the layout-1 slots it has just read
        st1(A0, x, t);
        st1(A1, sc, t);
        __syncthreads();
        for (uint32_t c = t; c < nlow; c += TT) {
            const uint32_t e = swz(BN_AT(unrank13[c], 1, TN));
            row[BN_AT(c, 1, nlow)] = scaled_log(A0[e], A1[e]);
        }
    } else {
        const int pt = __popc((uint32_t)t);
#pragma unroll
        for (int r = 0; r < TR; ++r)
            if (pt + __popc((uint32_t)r) <= d) row[BN_AT(rank13[el1(r, t)], 1, nlow)] = scaled_log(x[r], sc[r]);
    }
}

// rank13[L] = position of L among the subsets of 13 bits ordered by size then
// value; unrank13 is its inverse.
__global__ void k_rank13_tables(uint16_t* __restrict__ rank13, uint16_t* __restrict__ unrank13,
                                size_t js)
{
    rank13 = job_ptr(rank13, js);
    unrank13 = job_ptr(unrank13, js);
    const uint32_t L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= (uint32_t)TN) return;
    const uint32_t r = small_subset_rank(L, TB);
    rank13[L] = (uint16_t)r;
    unrank13[r] = (uint16_t)L;
}

#ifndef BN_MEGA  // host launchers (bn_mega.cu includes only the device code)
#ifdef BN_CHECK_BOUNDS
BN_BOUNDS_READER(bounds_line_tile13)
#endif
// ===========================================================================
// Launchers.
// ===========================================================================
// Columns whose sums take more than one row: the low patterns with fewer
// than d elements.
static uint32_t colb_columns(const Plan& P)
{
    uint64_t c = 0;
    for (int k = 0; k < P.d && k <= TB; ++k) c += binom_host(TB, k);
    return (uint32_t)c;
}

// High bits beyond one 128 KB column in shared memory: the column
// butterflies then run per chunk of those bits, added by k_upzeta13_colt
// (single jobs launched directly, with A in device memory, only; 4 for the
// others, which then keep the per-tile sums).
static int colb_chunk_bits(const Plan& P)
{
    const int h = P.n - 1 - TB;
    const int hmax = P.prec == 0 ? 14 : 15;          // 2^h values of 8 or 4 bytes in 128 KB
    if (h <= hmax) return 0;
    return recording() || P.nj != 1 || P.spill ? 4 : h - hmax;
}

// Column sums by butterflies over the h high dimensions when they take at
// most four fifths (FP32; four times in FP64) of the steps of the direct sums
// (the columns with d low elements are copies either way) and a column run
// fits 128 KB of shared memory (5 <= h <= 15 in FP32, h <= 14 in FP64).
bool use_colb(const Plan& P)
{
    const int h = P.n - 1 - TB;
    // below h = 5 a column has at most 32 rows: the per-tile sums are cheap,
    // and the column kernel's many small blocks would cost a batch's
    // persistent kernel one work item each
    if (h < 5 || colb_chunk_bits(P) > 3) return false;
    double direct = 0.0, ncol = 0.0;
    for (int kl = 0; kl <= P.d && kl <= TB; ++kl) {
        ncol += (double)binom_host(TB, kl);
        double rows = 0.0;
        for (int kh = 0; kh <= P.d - kl && kh <= h; ++kh)
            rows += (double)binom_host(h, kh) * std::ldexp(1.0, h - kh);
        direct += (double)binom_host(TB, kl) * rows;
    }
    const double ncb = colb_columns(P);
    const double bfly = ncb * h * std::ldexp(1.0, h - 1) + (ncol - ncb) * std::ldexp(1.0, h);
    // FP64: a direct term costs an FP64 exponential, a linear-scale step one addition
    return direct >= (P.prec == 0 ? 0.25 : 1.25) * bfly;
}

size_t upzeta13_cols_smem_bytes(const Plan& P)
{
    const size_t es = P.prec == 0 ? 8 : 4;
    const int h = P.n - 1 - TB;
    uint64_t nrow = 0;
    for (int k = 0; k <= P.d && k <= h; ++k) nrow += binom_host(h, k);
    return 2 * 8 * 96 * es + sizeof(SBinom) + 64 * 4 + 16 * 4 + nrow * 4;
}

size_t upzeta13_smem_bytes(const Plan& P)
{
    const size_t es = P.prec == 0 ? 8 : 4;
    return (size_t)TN * (2 * es) + (TT / 32) * es;   // A0, A1, the warps' maxima
}

bool tile13_up_fits(const Plan& P)
{
    return P.n >= 14 && upzeta13_cols_smem_bytes(P) <= 227 * 1024 - 64;
}

size_t gamma13_smem_bytes(const Plan& P)
{
    const size_t es = P.prec == 0 ? 8 : 4;
    return (size_t)TN * (2 * es) + 16;
}

cudaError_t launch_rank13_tables(const Plan& P, uint16_t* rank13, uint16_t* unrank13, cudaStream_t s)
{
    launch_or_record(KID_RANK13, k_rank13_tables, dim3(TN / 256, P.nj), 256, 0, s, rank13, unrank13, P.js);
    return cudaGetLastError();
}

cudaError_t launch_reorder_up(const Plan& P, const void* lbs, void* tab, cudaStream_t s)
{
    const int64_t total = (int64_t)up_nodes(P) * P.K;
    const dim3 grid((unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), P.nj);
    if (P.prec == 0)
        launch_or_record(KID_REORDER_D, k_reorder_up<double>, grid, 256, 0, s, P.n, P.d, P.K, (const double*)lbs, (double*)tab,
                                                  P.js, up_nodes(P));
    else
        launch_or_record(KID_REORDER_F, k_reorder_up<float>, grid, 256, 0, s, P.n, P.d, P.K, (const float*)lbs, (float*)tab,
                                                 P.js, up_nodes(P));
    return cudaGetLastError();
}

size_t upzeta13p_smem_bytes(const Plan& P)
{
    uint64_t ncol = 0;
    for (int k = 0; k <= P.d && k <= TB; ++k) ncol += binom_host(TB, k);
    // A0, A1, the warps' maxima, the mbarrier and a flag, the staged column
    // sums (16-byte multiple, and 48 bytes for the two copies' rounding),
    // the output block
    return (size_t)TN * 4 * 2 + (TT / 32) * 4 + 16 + ((ncol * 4 + 15) & ~(uint64_t)15) + 48 + (size_t)TN * 4;
}

// The persistent FP32 tile kernel runs single jobs whose A is in device
// memory (a spilled A may sit in host memory, where no bulk copy goes) and
// that are launched directly, not recorded for the persistent batch kernel.
static bool use_upzeta13p(const Plan& P, const int* err)
{
    return err && P.prec != 0 && P.nj == 1 && !P.spill && !recording();
}

// The persistent tile kernel stages the columns with d low elements straight
// from the reordered score table when the column sums come from the column
// butterflies (which then leave them out), the table's node stride is a
// multiple of 16 bytes and every node's table holds at least 3 entries past
// its first ncol (h >= 1).
static bool upzeta_table_copies(const Plan& P, const void* tab, const int* err)
{
    const int h = P.n - 1 - TB;
    return use_upzeta13p(P, err) && use_colb(P) && colb_columns(P) < num_small_subsets_host(P.d) &&
           P.K % 4 == 0 && ((uintptr_t)tab & 15u) == 0 && h >= 1 && P.d >= 1;
}

cudaError_t launch_upzeta13(const Plan& P, const void* tab, const uint16_t* unrank13, void* A,
                            cudaStream_t s, cudaEvent_t sums_done, int* err)
{
    const int h = P.n - 1 - TB;
    const int nodes = up_nodes(P);
    const dim3 grid((unsigned)nodes << h, P.nj);
    const size_t sc = upzeta13_cols_smem_bytes(P), sm = upzeta13_smem_bytes(P);
    uint64_t nrow = 0;
    for (int k = 0; k <= P.d && k <= h; ++k) nrow += binom_host(h, k);
    if (use_colb(P)) {                                // butterflies over the high dims
        // columns per block: as many as fit 64 KB, at most 8 (FP32) or 4 (FP64)
        const size_t es = P.prec == 0 ? 8 : 4;
        // (one column of up to 128 KB from h = 14 in FP32, 13 in FP64)
        const int cpb = (int)std::max<size_t>(1, std::min<size_t>((size_t)(64 * 1024) / (es << h), P.prec == 0 ? 4 : 8));
        uint64_t ncol = 0;
        for (int k = 0; k <= P.d && k <= TB; ++k) ncol += binom_host(TB, k);
        const uint32_t ncb = colb_columns(P);
        const uint64_t ntiles = (uint64_t)nodes << h;
        // the copy blocks follow the butterfly blocks (none when the tile
        // kernel stages those columns from the table itself)
        const bool copies = ncb < ncol && !upzeta_table_copies(P, tab, err);
        const int hc = colb_chunk_bits(P);
        const unsigned nblk = (unsigned)(((uint64_t)nodes * ((ncb + cpb - 1) / cpb) << hc) +
                                         (copies ? (ntiles + 7) / 8 : 0));
        const size_t smb = ((size_t)cpb << (h - hc)) * es;
        const dim3 gb(nblk, P.nj);
        if (P.prec == 0) {
            if (cpb >= 4)
                launch_or_record(KID_COLB4_D, k_upzeta13_colb<double, 4>, gb, 256, smb, s, P.n, P.d, P.K,
                                 (const double*)tab, (double*)A, P.js, nodes, ncb, hc);
            else if (cpb == 2)
                launch_or_record(KID_COLB2_D, k_upzeta13_colb<double, 2>, gb, 256, smb, s, P.n, P.d, P.K,
                                 (const double*)tab, (double*)A, P.js, nodes, ncb, hc);
            else
                launch_or_record(KID_COLB1_D, k_upzeta13_colb<double, 1>, gb, 256, smb, s, P.n, P.d, P.K,
                                 (const double*)tab, (double*)A, P.js, nodes, ncb, hc);
        } else if (cpb == 8) {
            launch_or_record(KID_COLB8, k_upzeta13_colb<float, 8>, gb, 256, smb, s, P.n, P.d, P.K,
                             (const float*)tab, (float*)A, P.js, nodes, ncb, hc);
        } else if (cpb >= 4) {
            launch_or_record(KID_COLB4, k_upzeta13_colb<float, 4>, gb, 256, smb, s, P.n, P.d, P.K,
                             (const float*)tab, (float*)A, P.js, nodes, ncb, hc);
        } else if (cpb == 2) {
            launch_or_record(KID_COLB2, k_upzeta13_colb<float, 2>, gb, 256, smb, s, P.n, P.d, P.K,
                             (const float*)tab, (float*)A, P.js, nodes, ncb, hc);
        } else {
            launch_or_record(KID_COLB1, k_upzeta13_colb<float, 1>, gb, 256, smb, s, P.n, P.d, P.K,
                             (const float*)tab, (float*)A, P.js, nodes, ncb, hc);
        }
        if (hc > 0) {                                 // add the chunks (never recorded)
            const cudaError_t ec = cudaGetLastError();
            if (ec != cudaSuccess) return ec;
            const uint64_t total = ((uint64_t)nodes << (h - hc)) * ncb;
            const unsigned gt = (unsigned)std::min<uint64_t>((total + 255) / 256, 152 * 64);
            if (P.prec == 0)
                k_upzeta13_colt<double><<<gt, 256, 0, s>>>(P.n, (double*)A, nodes, ncb, hc);
            else
                k_upzeta13_colt<float><<<gt, 256, 0, s>>>(P.n, (float*)A, nodes, ncb, hc);
        }
    } else if (nrow * 4 * 8 <= 160 * 1024) {          // warp per tile, 8 tiles per block
        const uint64_t ntiles = (uint64_t)nodes << h;
        const dim3 gw((unsigned)std::min<uint64_t>((ntiles + 7) / 8, 152 * 16), P.nj);
        const size_t sw = (size_t)nrow * 4 * 8;
        if (P.prec == 0)
            launch_or_record(KID_COLW_D, k_upzeta13_colw<double>, gw, 256, sw, s, P.n, P.d, P.K, (const double*)tab,
                                                        (double*)A, P.js, nodes);
        else
            launch_or_record(KID_COLW_F, k_upzeta13_colw<float>, gw, 256, sw, s, P.n, P.d, P.K, (const float*)tab,
                                                       (float*)A, P.js, nodes);
    } else if (P.prec == 0)
        launch_or_record(KID_COLS_D, k_upzeta13_cols<double>, grid, TT, sc, s, P.n, P.d, P.K, (const double*)tab, (double*)A,
                                                     P.js);
    else
        launch_or_record(KID_COLS_F, k_upzeta13_cols<float>, grid, TT, sc, s, P.n, P.d, P.K, (const float*)tab, (float*)A,
                                                    P.js);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (sums_done) {
        e = cudaEventRecord(sums_done, s);
        if (e != cudaSuccess) return e;
    }
    if (use_upzeta13p(P, err)) {
        const uint32_t ntiles = (uint32_t)nodes << h;
        const size_t smp = upzeta13p_smem_bytes(P);
        int dev = 0, nsm = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = use_tlo(P) ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_upzeta13p<true>, TT, smp)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_upzeta13p<false>, TT, smp);
        if (e != cudaSuccess) return e;
        const unsigned blocks = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)std::max(per_sm, 1) * nsm);
        const uint32_t ncol = num_small_subsets_host(P.d);
        const uint32_t ncb = upzeta_table_copies(P, tab, err) ? colb_columns(P) : ncol;
        if (use_tlo(P))
            k_upzeta13p<true><<<blocks, TT, smp, s>>>(P.n, P.d, unrank13, (float*)A, ntiles, err, kCopySpinCap, 0,
                                                      (const float*)tab, P.K, ncb);
        else
            k_upzeta13p<false><<<blocks, TT, smp, s>>>(P.n, P.d, unrank13, (float*)A, ntiles, err, kCopySpinCap, 0,
                                                       (const float*)tab, P.K, ncb);
        return cudaGetLastError();
    }
    if (P.prec == 0)
        launch_or_record(KID_UP13_D, k_upzeta13<double, false>, grid, TT, sm, s, P.n, P.d, unrank13, (double*)A, P.js);
    else if (use_tlo(P))
        launch_or_record(KID_UP13_F_TLO, k_upzeta13<float, true>, grid, TT, sm, s, P.n, P.d, unrank13, (float*)A, P.js);
    else
        launch_or_record(KID_UP13_F, k_upzeta13<float, false>, grid, TT, sm, s, P.n, P.d, unrank13, (float*)A, P.js);
    return cudaGetLastError();
}

// One block of the persistent tile kernel (n = 14, d = 4: one tile) with its
// first bulk copy withheld: its wait gives up after `polls` polls and sets
// kErrDeviceTimeout in *err.  A holds one tile (8192 floats); unrank13 is
// filled here.
cudaError_t launch_upzeta13p_withheld(float* A, uint16_t* rank13, uint16_t* unrank13, int* err,
                                      uint32_t polls, cudaStream_t s)
{
    cudaError_t e = allow_max_dynamic_smem(k_upzeta13p<false>);
    if (e != cudaSuccess) return e;
    k_rank13_tables<<<TN / 256, 256, 0, s>>>(rank13, unrank13, 0);
    Plan P{};
    P.n = 14;
    P.d = 4;
    P.prec = 1;
    k_upzeta13p<false><<<1, TT, upzeta13p_smem_bytes(P), s>>>(14, 4, unrank13, A, 1u, err, polls, 1, nullptr,
                                                             int64_t(0), num_small_subsets_host(4));
    return cudaGetLastError();
}

cudaError_t launch_gamma13_p1(const Plan& P, const void* F, const void* Rc,
                              const uint16_t* rank13, void* W, cudaStream_t s, const void* lq,
                              const void* A)
{
    if (P.prec != 0) {
        const cudaError_t e = launch_gamma_table(P, F, Rc, s);
        if (e != cudaSuccess) return e;
    }
    const int h = P.n - 1 - TB;
    const size_t sm = gamma13_smem_bytes(P);
    const dim3 grid((1u << h) * (unsigned)P.n, P.nj, 1);
    // relevance margin: 64 (FP64) or 24 (FP32: its tolerance is 1e-4) bits +
    // log2(K 2^h), in bits (FP32) or nats (FP64)
    const double mbits = (P.prec == 0 ? 64.0 : 24.0) + std::ceil(std::log2((double)P.K)) + h;
    const double margin = P.prec == 0 ? mbits * 0.69314718055994531 : mbits;
    // the order prior is a separate instance: the plain kernel has no trace of it
    if (P.prec == 0) {
        if (lq)
            launch_or_record(KID_G13_D_Q, k_gamma13_p1<double, true>, grid, TT, sm, s, 
                P.n, P.d, P.nlow_g, (const double*)F, (const double*)Rc, rank13, (double*)W, P.js,
                (const double*)lq, (const double*)A, margin, P.vsel);
        else
            launch_or_record(KID_G13_D, k_gamma13_p1<double, false>, grid, TT, sm, s, 
                P.n, P.d, P.nlow_g, (const double*)F, (const double*)Rc, rank13, (double*)W, P.js,
                nullptr, (const double*)A, margin, P.vsel);
    } else {
        if (lq)
            launch_or_record(KID_G13_F_Q, k_gamma13_p1<float, true>, grid, TT, sm, s, 
                P.n, P.d, P.nlow_g, (const float*)F, (const float*)Rc, rank13, (float*)W, P.js,
                (const float*)lq, (const float*)A, (float)margin, P.vsel);
        else
            launch_or_record(KID_G13_F, k_gamma13_p1<float, false>, grid, TT, sm, s, 
                P.n, P.d, P.nlow_g, (const float*)F, (const float*)Rc, rank13, (float*)W, P.js,
                nullptr, (const float*)A, (float)margin, P.vsel);
    }
    return cudaGetLastError();
}

cudaError_t set_tile13_attributes()
{
    cudaError_t e;
#define SETA(k)                      \
    e = allow_max_dynamic_smem(k); \
    if (e != cudaSuccess) return e;
    SETA(k_upzeta13_cols<double>)
    SETA(k_upzeta13_cols<float>)
    SETA(k_upzeta13_colw<double>)
    SETA(k_upzeta13_colw<float>)
    SETA((k_upzeta13_colb<float, 8>))
    SETA((k_upzeta13_colb<float, 4>))
    SETA((k_upzeta13_colb<float, 2>))
    SETA((k_upzeta13_colb<float, 1>))
    SETA((k_upzeta13_colb<double, 4>))
    SETA((k_upzeta13_colb<double, 2>))
    SETA((k_upzeta13_colb<double, 1>))
    SETA((k_upzeta13<double, false>))
    SETA((k_upzeta13<float, false>))
    SETA((k_upzeta13<float, true>))
    SETA(k_upzeta13p<false>)
    SETA(k_upzeta13p<true>)
    SETA((k_gamma13_p1<double, false>))
    SETA((k_gamma13_p1<float, false>))
    SETA((k_gamma13_p1<double, true>))
    SETA((k_gamma13_p1<float, true>))
#undef SETA
    return cudaSuccess;
}

#endif  // BN_MEGA

}  // namespace bn

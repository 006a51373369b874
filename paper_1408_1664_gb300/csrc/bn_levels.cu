// bn_levels.cu -- F (Eq. 9) and R' (Eq. 10) over the subset lattice in FP32,
// one thread per tile of 16 subsets.
//
// A tile is the 16 subsets S = (Ht << 4) | l that share their high bits Ht
// (l = the 4 low bits).  Tiles are launched one popcount level of Ht at a
// time (the sub-cube order of Section 3.2.2): every term that leaves the
// tile reads a tile of the previous level.  A thread
//   * adds the terms across tiles, one row of 16 values of A_i and one row of
//     F (or R') per high bit, read as four 128-bit loads each;
//   * resolves the terms inside the tile in registers, in popcount order of l;
//   * writes its row of 16 values.
// Every thread of a launch has the same number of terms (same |Ht|), so warps
// do not diverge, and the index arithmetic is shared by the 16 subsets.
//
// Log-sum-exp is kept lazily: (m, s) stands for m + log2(s) with m the first
// term and s rescaled only when a term exceeds m by more than 2^64, so a term
// costs one exponential.  s stays below 2^64 * 32 and every value entering is
// finite (A and F are logs of positive sums).
#include "bn_device.cuh"
#include "bn_kernels.cuh"

namespace bn {
namespace {

constexpr int LB = 4;             // low bits of a tile
constexpr int LN = 1 << LB;       // subsets per tile
constexpr int BT = 28;            // binomial table rows (n - LB < 28)

__device__ const BinomTable g_binom_lanes = make_binom_table();

__device__ __forceinline__ void lazy_add(float& m, float& s, float x)
{
    const float dd = x - m;                       // +inf while the accumulator is empty
    const bool big = dd > 64.0f;
    const float e = ex2_approx(big ? -dd : dd);
    s = big ? __fmaf_rn(s, e, 1.0f) : s + e;
    m = big ? x : m;
}

// x with bit i (i < LB) removed: an index among the 8 four-bit patterns
// without bit i.
__host__ __device__ constexpr int squeeze4(int x, int i)
{
    return (x & ((1 << i) - 1)) | ((x >> 1) & ~((1 << i) - 1));
}

__device__ __forceinline__ void load16(const float* p, float (&v)[LN], bool stream)
{
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < LN / 4; ++k) {
        const float4 x = stream ? __ldcs(q + k) : q[k];
        v[4 * k] = x.x;
        v[4 * k + 1] = x.y;
        v[4 * k + 2] = x.z;
        v[4 * k + 3] = x.w;
    }
}

__device__ __forceinline__ void load8(const float* p, float (&v)[8])
{
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float4 x = __ldcs(q + k);
        v[4 * k] = x.x;
        v[4 * k + 1] = x.y;
        v[4 * k + 2] = x.z;
        v[4 * k + 3] = x.w;
    }
}

__device__ __forceinline__ void store16(float* p, const float (&v)[LN])
{
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int k = 0; k < LN / 4; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// Tile g of the level: the g-th hl-element subset of nh bits in colex order.
__device__ __forceinline__ uint32_t tile_of(uint32_t g, int hl, int nh, const uint32_t (*bt)[BT])
{
    uint32_t H = 0, r = g;
    int c = nh - 1;
    for (int t = hl; t >= 1; --t) {
        while (bt[c][t] > r) --c;
        H |= 1u << c;
        r -= bt[c][t];
        --c;
    }
    return H;
}

__device__ __forceinline__ void fill_table(uint32_t (*bt)[BT])
{
    for (int x = threadIdx.x; x < BT * BT; x += blockDim.x) bt[x / BT][x % BT] = g_binom_lanes.v[x / BT][x % BT];
}

}  // namespace

//   F(S) = sum_{i in S} A_i(S - {i}) F(S - {i}),  F(empty) = 1
__global__ void __launch_bounds__(256, 3)
k_forward_rows(int n, int hl, uint32_t ntiles, const float* __restrict__ A, float* __restrict__ F,
               size_t js)
{
    A = job_ptr(A, js);
    F = job_ptr(F, js);
    __shared__ uint32_t bt[BT][BT];
    fill_table(bt);
    __syncthreads();
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ntiles) return;
    const int nh = n - LB;
    const uint32_t Ht = tile_of(g, hl, nh, bt);
    const size_t half = (size_t)1 << (n - 1);
    using L = LogOps<float>;

    float m[LN], s[LN];
#pragma unroll
    for (int l = 0; l < LN; ++l) { m[l] = L::ninf(); s[l] = 0.0f; }
    // terms across tiles: i = LB + j for the set bits j of Ht
    for (uint32_t rest = Ht; rest; rest &= rest - 1) {
        const int j = __ffs(rest) - 1;
        const uint32_t Hm = Ht & ~(1u << j);
        float a[LN], f[LN];
        load16(A + (size_t)(LB + j) * half + ((size_t)squeeze(Hm, j) << LB), a, true);
        load16(F + ((size_t)Hm << LB), f, false);
#pragma unroll
        for (int l = 0; l < LN; ++l) lazy_add(m[l], s[l], a[l] + f[l]);
    }
    // terms inside the tile: A_i(S - {i}) for i < LB, 8 values per i
    float ai[LB][8];
#pragma unroll
    for (int i = 0; i < LB; ++i) load8(A + (size_t)i * half + ((size_t)Ht << (LB - 1)), ai[i]);
    float Fv[LN];
    Fv[0] = Ht == 0u ? 0.0f : m[0] + L::lg(s[0]);
#pragma unroll
    for (int l = 1; l < LN; ++l) {
#pragma unroll
        for (int i = 0; i < LB; ++i)
            if (l >> i & 1) lazy_add(m[l], s[l], ai[i][squeeze4(l ^ (1 << i), i)] + Fv[l ^ (1 << i)]);
        Fv[l] = m[l] + L::lg(s[l]);
    }
    store16(F + ((size_t)Ht << LB), Fv);
}

//   R'(T) = sum_{i not in T} A_i(T) R'(T + {i}),  R'(V) = 1
__global__ void __launch_bounds__(256, 3)
k_backward_rows(int n, int hl, uint32_t ntiles, const float* __restrict__ A, float* __restrict__ Rc,
                size_t js)
{
    A = job_ptr(A, js);
    Rc = job_ptr(Rc, js);
    __shared__ uint32_t bt[BT][BT];
    fill_table(bt);
    __syncthreads();
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ntiles) return;
    const int nh = n - LB;
    const uint32_t hmask = (1u << nh) - 1u;
    const uint32_t Ht = tile_of(g, hl, nh, bt);
    const size_t half = (size_t)1 << (n - 1);
    using L = LogOps<float>;

    float m[LN], s[LN];
#pragma unroll
    for (int l = 0; l < LN; ++l) { m[l] = L::ninf(); s[l] = 0.0f; }
    for (uint32_t rest = ~Ht & hmask; rest; rest &= rest - 1) {
        const int j = __ffs(rest) - 1;
        float a[LN], r[LN];
        load16(A + (size_t)(LB + j) * half + ((size_t)squeeze(Ht, j) << LB), a, true);
        load16(Rc + ((size_t)(Ht | (1u << j)) << LB), r, false);
#pragma unroll
        for (int l = 0; l < LN; ++l) lazy_add(m[l], s[l], a[l] + r[l]);
    }
    // A_i(T) for i < LB not in T, 8 values per i
    float ai[LB][8];
#pragma unroll
    for (int i = 0; i < LB; ++i) load8(A + (size_t)i * half + ((size_t)Ht << (LB - 1)), ai[i]);
    float Rv[LN];
    Rv[LN - 1] = Ht == hmask ? 0.0f : m[LN - 1] + L::lg(s[LN - 1]);
#pragma unroll
    for (int l = LN - 2; l >= 0; --l) {
#pragma unroll
        for (int i = 0; i < LB; ++i)
            if (!(l >> i & 1)) lazy_add(m[l], s[l], ai[i][squeeze4(l, i)] + Rv[l | (1 << i)]);
        Rv[l] = m[l] + L::lg(s[l]);
    }
    store16(Rc + ((size_t)Ht << LB), Rv);
}

namespace {

uint64_t choose(int n, int k)
{
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int t = 1; t <= k; ++t) r = r * (uint64_t)(n - k + t) / (uint64_t)t;
    return r;
}

}  // namespace

bool rows_levels_fit(const Plan& P)
{
    return P.prec != 0 && P.n >= LB + 1 && P.n - LB < BT;
}

cudaError_t launch_forward_rows(const Plan& P, const void* A, void* F, cudaStream_t s, int* launches)
{
    const int nh = P.n - LB;
    for (int hl = 0; hl <= nh; ++hl) {
        const uint32_t nt = (uint32_t)choose(nh, hl);
        k_forward_rows<<<dim3((nt + 255) / 256, P.nj), 256, 0, s>>>(P.n, hl, nt, (const float*)A,
                                                                   (float*)F, P.js);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

cudaError_t launch_backward_rows(const Plan& P, const void* A, void* Rc, cudaStream_t s,
                                 int* launches)
{
    const int nh = P.n - LB;
    for (int hl = nh; hl >= 0; --hl) {
        const uint32_t nt = (uint32_t)choose(nh, hl);
        k_backward_rows<<<dim3((nt + 255) / 256, P.nj), 256, 0, s>>>(P.n, hl, nt, (const float*)A,
                                                                    (float*)Rc, P.js);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

}  // namespace bn

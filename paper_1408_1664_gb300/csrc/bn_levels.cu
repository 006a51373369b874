// bn_levels.cu -- F (Eq. 9) and R' (Eq. 10) over the subset lattice, one
// thread per tile of 2^B subsets: 16 in FP32 (base-2 logs), 8 in FP64
// (natural logs; a row of 8 doubles is 64 bytes, like 16 floats).
//
// A tile is the 2^B subsets S = (Ht << B) | l that share their high bits Ht
// (l = the B low bits).  Tiles are launched one popcount level of Ht at a
// time (the sub-cube order of Section 3.2.2): every term that leaves the
// tile reads a tile of the previous level.  A thread
//   * adds the terms across tiles, one row of 2^B values of A_i and one row of
//     F (or R') per high bit, read as four 128-bit loads each;
//   * resolves the terms inside the tile in registers, in popcount order of l;
//   * writes its row of 2^B values.
// Every thread of a launch has the same number of terms (same |Ht|), so warps
// do not diverge, and the index arithmetic is shared by the 2^B subsets.
//
// Log-sum-exp is kept lazily: (m, s) stands for m + lg(s) with m the first
// term and s rescaled only when a term exceeds m by more than 2^64 (FP32) or
// e^40 (FP64), so a term costs one exponential.  s stays below that factor
// times 32, and every value entering is finite (A and F are logs of
// positive sums; a zero weight is a finite soft zero).
#include <algorithm>

#include "bn_device.cuh"
#include "bn_kernels.cuh"

namespace bn {
namespace {

constexpr int LB = 4;             // low bits of an FP32 tile
constexpr int LB64 = 3;           // low bits of an FP64 tile
constexpr int BT = 29;            // binomial table rows (n - B < 29: n <= 32 in FP32)

__device__ const BinomTable g_binom_lanes = make_binom_table();

__device__ __forceinline__ void lazy_add(float& m, float& s, float x)
{
    const float dd = x - m;                       // +inf while the accumulator is empty
    const bool big = dd > 64.0f;
    const float e = ex2_approx(big ? -dd : dd);
    s = big ? __fmaf_rn(s, e, 1.0f) : s + e;
    m = big ? x : m;
}

__device__ __forceinline__ void lazy_add(double& m, double& s, double x)
{
    const double dd = x - m;                      // +inf while the accumulator is empty
    const bool big = dd > 40.0;
    const double e = exp_t(big ? -dd : dd);       // the library's table-driven exponential
    s = big ? fma(s, e, 1.0) : s + e;
    m = big ? x : m;
}

// x with bit i (i < B) removed: an index among the 2^(B-1) B-bit patterns
// without bit i.
__host__ __device__ constexpr int squeeze4(int x, int i)
{
    return (x & ((1 << i) - 1)) | ((x >> 1) & ~((1 << i) - 1));
}

// Load modes: LD_PLAIN, LD_STREAM (read once: evict first), LD_L2 (through
// L2 only: values another block of the same launch wrote).
enum { LD_PLAIN = 0, LD_STREAM = 1, LD_L2 = 2 };

// A row of N values, 128-bit loads (N * sizeof(T) is a multiple of 16).
template <int N>
__device__ __forceinline__ void load_row(const float* p, float (&v)[N], int mode)
{
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < N / 4; ++k) {
        const float4 x = mode == LD_STREAM ? __ldcs(q + k) : mode == LD_L2 ? __ldcg(q + k) : q[k];
        v[4 * k] = x.x;
        v[4 * k + 1] = x.y;
        v[4 * k + 2] = x.z;
        v[4 * k + 3] = x.w;
    }
}

template <int N>
__device__ __forceinline__ void load_row(const double* p, double (&v)[N], int mode)
{
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
        const double2 x = mode == LD_STREAM ? __ldcs(q + k) : mode == LD_L2 ? __ldcg(q + k) : q[k];
        v[2 * k] = x.x;
        v[2 * k + 1] = x.y;
    }
}

template <int N>
__device__ __forceinline__ void store_row(float* p, const float (&v)[N])
{
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int k = 0; k < N / 4; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

template <int N>
__device__ __forceinline__ void store_row(double* p, const double (&v)[N])
{
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) q[k] = make_double2(v[2 * k], v[2 * k + 1]);
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

// Tile g of level hl within the sub-lattice whose top kfix of the nh tile
// bits are rfix (a shard of a job split by its top variables; kfix = 0: the
// whole level).
__device__ __forceinline__ uint32_t level_tile(uint32_t g, int hl, int nh, uint32_t rfix, int kfix,
                                               const uint32_t (*bt)[BT])
{
    if (kfix == 0) return tile_of(g, hl, nh, bt);
    return tile_of(g, hl - __popc(rfix), nh - kfix, bt) | (rfix << (nh - kfix));
}

__device__ __forceinline__ void fill_table(uint32_t (*bt)[BT])
{
    for (int x = threadIdx.x; x < BT * BT; x += blockDim.x) bt[x / BT][x % BT] = g_binom_lanes.v[x / BT][x % BT];
}

// TLO (B = 4): the rows of A in tile-level order (see bn_device.cuh): a
// term across tiles reads row tlo_row(R, 9) of A_{B+j} (rows of 16 values,
// nine in-tile row bits); the in-tile rows of A_i (i < B: rows of 8 values,
// ten in-tile row bits) sit at tlo_row(Ht, 10).
//
// The 2^B values of F in tile Ht (its level's tiles of F already written):
//   F(S) = sum_{i in S} A_i(S - {i}) F(S - {i}),  F(empty) = 1
//
// rebase: the previous level's stored values are relative to a base larger by
// this much than this level's (the FP32 per-level bases, bn_device.cuh; 0
// otherwise).  Returns the largest value written.
//
// SLAB (a split job with divided A): A holds the rank's slabs of the nl = n -
// k low nodes, each over the nl - 1 low bits of its index (the top k bits are
// the rank's); Atop holds, for each top variable t = nl + q, its slab over
// the nl low variables.  A term of a low node reads its slab with the top
// bits of the row index dropped; a term of a top variable reads Atop.
template <typename T, int FMODE, int B, bool TLO = false, bool SLAB = false>
__device__ __forceinline__ T forward_tile(int n, uint32_t Ht, const T* __restrict__ A,
                                          T* __restrict__ F, T rebase = T(0), int nl = 0,
                                          const T* __restrict__ Atop = nullptr)
{
    constexpr int LN = 1 << B;
    const size_t full = (size_t)1 << n;
    const size_t half = (size_t)1 << ((SLAB ? nl : n) - 1);
    const uint32_t rmask = SLAB ? (1u << (nl - 1 - B)) - 1u : ~0u;   // slab row bits
    const uint32_t lmask = SLAB ? (1u << (nl - B)) - 1u : ~0u;       // low tile bits
    using L = LogOps<T>;

    T m[LN], s[LN];
#pragma unroll
    for (int l = 0; l < LN; ++l) { m[l] = L::ninf(); s[l] = T(0); }
    // terms across tiles: i = B + j for the set bits j of Ht
    for (uint32_t rest = Ht; rest; rest &= rest - 1) {
        const int j = __ffs(rest) - 1;
        const uint32_t Hm = Ht & ~(1u << j);
        T a[LN], f[LN];
        if (SLAB && B + j >= nl) {                  // a top variable: its slab
            load_row(Atop + BN_AT(((size_t)(B + j - nl) << nl) + ((size_t)(Ht & lmask) << B), LN,
                                  (size_t)(n - nl) << nl),
                     a, LD_STREAM);
        } else {
            const uint32_t row = TLO ? tlo_row(squeeze(Hm, j) & rmask, 9) : squeeze(Hm, j) & rmask;
            load_row(A + BN_AT((size_t)(B + j) * half + ((size_t)row << B), LN,
                               (SLAB ? nl : n) * half),
                     a, LD_STREAM);
        }
        load_row(F + BN_AT((size_t)Hm << B, LN, full), f, FMODE);
#pragma unroll
        for (int l = 0; l < LN; ++l) lazy_add(m[l], s[l], a[l] + f[l]);
    }
    // (m, s) stands for m + lg(s): moving the cross-tile sums to this level's
    // base moves m
#pragma unroll
    for (int l = 0; l < LN; ++l) m[l] -= rebase;
    // terms inside the tile: A_i(S - {i}) for i < B, 2^(B-1) values per i
    T ai[B][LN / 2];
#pragma unroll
    for (int i = 0; i < B; ++i)
        load_row(A + BN_AT((size_t)i * half + ((size_t)(TLO ? tlo_row(Ht & lmask, 10) : Ht & lmask) << (B - 1)),
                           LN / 2, (SLAB ? nl : n) * half),
                 ai[i], LD_STREAM);
    T Fv[LN];
    Fv[0] = Ht == 0u ? T(0) : m[0] + L::lg(s[0]);
#pragma unroll
    for (int l = 1; l < LN; ++l) {
#pragma unroll
        for (int i = 0; i < B; ++i)
            if (l >> i & 1) lazy_add(m[l], s[l], ai[i][squeeze4(l ^ (1 << i), i)] + Fv[l ^ (1 << i)]);
        Fv[l] = m[l] + L::lg(s[l]);
    }
    store_row(F + BN_AT((size_t)Ht << B, LN, full), Fv);
    T mx = Fv[0];
#pragma unroll
    for (int l = 1; l < LN; ++l) mx = Fv[l] > mx ? Fv[l] : mx;
    return mx;
}

// The 2^B values of R' in tile Ht (the tiles of the level above written):
//   R'(T) = sum_{i not in T} A_i(T) R'(T + {i}),  R'(V) = 1
template <typename T, int FMODE, int B, bool TLO = false, bool SLAB = false>
__device__ __forceinline__ T backward_tile(int n, uint32_t Ht, const T* __restrict__ A,
                                           T* __restrict__ Rc, T rebase = T(0), int nl = 0,
                                           const T* __restrict__ Atop = nullptr)
{
    constexpr int LN = 1 << B;
    const int nh = n - B;
    const uint32_t hmask = (1u << nh) - 1u;
    const size_t full = (size_t)1 << n;
    const size_t half = (size_t)1 << ((SLAB ? nl : n) - 1);
    const uint32_t rmask = SLAB ? (1u << (nl - 1 - B)) - 1u : ~0u;
    const uint32_t lmask = SLAB ? (1u << (nl - B)) - 1u : ~0u;
    using L = LogOps<T>;

    T m[LN], s[LN];
#pragma unroll
    for (int l = 0; l < LN; ++l) { m[l] = L::ninf(); s[l] = T(0); }
    for (uint32_t rest = ~Ht & hmask; rest; rest &= rest - 1) {
        const int j = __ffs(rest) - 1;
        T a[LN], r[LN];
        if (SLAB && B + j >= nl) {
            load_row(Atop + BN_AT(((size_t)(B + j - nl) << nl) + ((size_t)(Ht & lmask) << B), LN,
                                  (size_t)(n - nl) << nl),
                     a, LD_STREAM);
        } else {
            const uint32_t row = TLO ? tlo_row(squeeze(Ht, j) & rmask, 9) : squeeze(Ht, j) & rmask;
            load_row(A + BN_AT((size_t)(B + j) * half + ((size_t)row << B), LN,
                               (SLAB ? nl : n) * half),
                     a, LD_STREAM);
        }
        load_row(Rc + BN_AT((size_t)(Ht | (1u << j)) << B, LN, full), r, FMODE);
#pragma unroll
        for (int l = 0; l < LN; ++l) lazy_add(m[l], s[l], a[l] + r[l]);
    }
#pragma unroll
    for (int l = 0; l < LN; ++l) m[l] -= rebase;
    // A_i(T) for i < B not in T, 2^(B-1) values per i
    T ai[B][LN / 2];
#pragma unroll
    for (int i = 0; i < B; ++i)
        load_row(A + BN_AT((size_t)i * half + ((size_t)(TLO ? tlo_row(Ht & lmask, 10) : Ht & lmask) << (B - 1)),
                           LN / 2, (SLAB ? nl : n) * half),
                 ai[i], LD_STREAM);
    T Rv[LN];
    Rv[LN - 1] = Ht == hmask ? T(0) : m[LN - 1] + L::lg(s[LN - 1]);
#pragma unroll
    for (int l = LN - 2; l >= 0; --l) {
#pragma unroll
        for (int i = 0; i < B; ++i)
            if (!(l >> i & 1)) lazy_add(m[l], s[l], ai[i][squeeze4(l, i)] + Rv[l | (1 << i)]);
        Rv[l] = m[l] + L::lg(s[l]);
    }
    store_row(Rc + BN_AT((size_t)Ht << B, LN, full), Rv);
    T mx = Rv[0];
#pragma unroll
    for (int l = 1; l < LN; ++l) mx = Rv[l] > mx ? Rv[l] : mx;
    return mx;
}

// The largest value a block wrote for its level, floored, into the level's
// word (one atomic per block; every thread of the block calls this).
__device__ __forceinline__ void block_level_max(int* word, float mx)
{
    __shared__ int wm[8];
    int v = __reduce_max_sync(0xffffffffu, level_floor(mx));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = max(v, wm[w]);
        if (v != kLevelUnset) atomicMax(word, v);
    }
}
// The first level of a sweep (one tile, one thread) starts the level words.
__device__ __forceinline__ void level_words_start(int* lw, int level, float mx)
{
    for (int k = 0; k < kLevelMode; ++k) lw[k] = kLevelUnset;
    lw[kLevelMode] = kLevelShift;
    lw[level] = level_floor(mx);
}

__device__ __forceinline__ void cluster_barrier()
{
    // every thread of every block of the cluster; release/acquire at cluster
    // scope orders the tiles written before it against the reads after it
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_blocks()
{
    uint32_t r;
    asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

}  // namespace

// FP32: 16-subset tiles at three blocks per SM (80 registers); FP64:
// 8-subset tiles at two.
//
// FP32 keeps the per-level bases (bn_device.cuh): level hl reads the
// previous level's word (its values' base minus this level's base), and
// every block adds its largest written value to the level's word.
template <typename T, bool TLO, bool SLAB = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_forward_rows(int n, int hl, uint32_t ntiles, const T* __restrict__ A, T* __restrict__ F,
               size_t js, uint32_t rfix, int kfix, const T* __restrict__ Atop)
{
    constexpr int B = sizeof(T) == 4 ? LB : LB64;
    constexpr bool kBases = sizeof(T) == 4;
    A = job_ptr(A, js);
    F = job_ptr(F, js);
    __shared__ uint32_t bt[BT][BT];
    fill_table(bt);
    __syncthreads();
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (kBases) {
        int* lw = level_words(reinterpret_cast<float*>(F), n);
        const T rebase = hl > 0 ? (T)level_delta(lw, hl - 1) : T(0);
        T mx = LogOps<T>::ninf();
        if (g < ntiles)
            mx = forward_tile<T, LD_PLAIN, B, TLO, SLAB>(n, level_tile(g, hl, n - B, rfix, kfix, bt), A, F,
                                                         rebase, n - kfix, Atop);
        if (hl == 0) {
            if (g == 0) level_words_start(lw, 0, mx);
        } else {
            block_level_max(lw + hl, mx);
        }
    } else {
        if (g >= ntiles) return;
        forward_tile<T, LD_PLAIN, B, TLO, SLAB>(n, level_tile(g, hl, n - B, rfix, kfix, bt), A, F, T(0),
                                                n - kfix, Atop);
    }
}

template <typename T, bool TLO, bool SLAB = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_backward_rows(int n, int hl, uint32_t ntiles, const T* __restrict__ A, T* __restrict__ Rc,
                size_t js, uint32_t rfix, int kfix, const T* __restrict__ Atop)
{
    constexpr int B = sizeof(T) == 4 ? LB : LB64;
    constexpr bool kBases = sizeof(T) == 4;
    A = job_ptr(A, js);
    Rc = job_ptr(Rc, js);
    __shared__ uint32_t bt[BT][BT];
    fill_table(bt);
    __syncthreads();
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (kBases) {
        const int nh = n - B;
        int* lw = level_words(reinterpret_cast<float*>(Rc), n);
        const T rebase = hl < nh ? (T)level_delta(lw, hl + 1) : T(0);
        T mx = LogOps<T>::ninf();
        if (g < ntiles)
            mx = backward_tile<T, LD_PLAIN, B, TLO, SLAB>(n, level_tile(g, hl, nh, rfix, kfix, bt), A, Rc,
                                                          rebase, n - kfix, Atop);
        if (hl == nh) {
            if (g == 0) level_words_start(lw, nh, mx);
        } else {
            block_level_max(lw + hl, mx);
        }
    } else {
        if (g >= ntiles) return;
        backward_tile<T, LD_PLAIN, B, TLO, SLAB>(n, level_tile(g, hl, n - B, rfix, kfix, bt), A, Rc, T(0),
                                                 n - kfix, Atop);
    }
}

// Step 3 of a whole batch group in one persistent launch of thread-block
// clusters (1 to 8 blocks, by the width of the widest level).  Work item it is F (it even) or R' (it odd) of job it / 2; the
// clusters take the items in turn (item = cluster id, + clusters, ...).  A
// cluster runs every popcount level of its item: its blocks' threads split
// the level's tiles, then meet at a cluster barrier before the next level.
// The blocks of a cluster are resident together by construction, and no
// cluster waits for another, so every barrier completes.  Every thread
// reaches every barrier: the item loop and the level loop are uniform
// across the cluster.  F and R' tiles written in the launch are read
// through L2 (another block, on another SM, wrote them).
__global__ void __launch_bounds__(256, 2)
k_rows_cluster(int n, int items, const float* __restrict__ A, float* __restrict__ F,
               float* __restrict__ Rc, size_t js)
{
    __shared__ uint32_t bt[BT][BT];
    fill_table(bt);
    __syncthreads();
    const int nh = n - LB;
    const uint32_t cs = cluster_blocks();
    const uint32_t cid = blockIdx.x / cs;
    const uint32_t ncl = gridDim.x / cs;
    const uint32_t t0 = cluster_rank() * blockDim.x + threadIdx.x;
    const uint32_t stride = cs * blockDim.x;
    for (int it = (int)cid; it < items; it += (int)ncl) {
        const size_t off = (size_t)(it >> 1) * js;
        const float* Aj = reinterpret_cast<const float*>(reinterpret_cast<const char*>(A) + off);
        const bool fwd = (it & 1) == 0;
        float* X = reinterpret_cast<float*>(reinterpret_cast<char*>(fwd ? F : Rc) + off);
        // the per-level bases of the level kernels, with the level words
        // read after the cluster barrier that ends the level before
        int* lw = level_words(X, n);
        for (int st = 0; st <= nh; ++st) {
            const int hl = fwd ? st : nh - st;
            const uint32_t nt = bt[nh][hl];
            const float rebase = st == 0 ? 0.f : (float)level_delta(lw, fwd ? hl - 1 : hl + 1);
            float mx = LogOps<float>::ninf();
            for (uint32_t g = t0; g < nt; g += stride) {
                const uint32_t Ht = tile_of(g, hl, nh, bt);
                const float m1 = fwd ? forward_tile<float, LD_L2, LB>(n, Ht, Aj, X, rebase)
                                     : backward_tile<float, LD_L2, LB>(n, Ht, Aj, X, rebase);
                mx = m1 > mx ? m1 : mx;
            }
            if (st == 0) {
                if (t0 == 0) level_words_start(lw, hl, mx);   // the level's one tile
            } else {
                block_level_max(lw + hl, mx);
            }
            cluster_barrier();
        }
    }
}

// The rows (2^B values each) of one level's tiles of the sub-lattice rsrc
// (top kfix tile bits), in tile order: dir 0 copies them from X into buf,
// dir 1 from buf into X.  The exchange of a job split over several ranks.
template <typename T>
__global__ void k_level_rows(int n, int hl, uint32_t ntiles, uint32_t rsrc, int kfix, T* __restrict__ X,
                             T* __restrict__ buf, int dir)
{
    constexpr int B = sizeof(T) == 4 ? LB : LB64;
    __shared__ uint32_t bt[BT][BT];
    fill_table(bt);
    __syncthreads();
    const uint64_t total = (uint64_t)ntiles << B;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < total;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = (uint32_t)(x >> B);
        const size_t pos = BN_AT(((size_t)level_tile(g, hl, n - B, rsrc, kfix, bt) << B) |
                                     (x & ((1u << B) - 1u)),
                                 1, (size_t)1 << n);
        if (dir == 0) buf[x] = X[pos];
        else X[pos] = buf[x];
    }
}

// ---------------------------------------------------------------------------
// A split job's divided A (Eq. 7 restricted to a rank's sub-lattice).  With
// the top k variables V_t = {nl, .., n - 1} (nl = n - k) fixed to the rank's
// bits r, every entry a rank's tiles read is a truncated zeta transform over
// the nl low variables alone:
//   low node i < nl:  A_i(r + L) = sum over G <= L of B'_i(G),
//                     B'_i(G) = sum over G_t <= r, |G_t| + |G| <= d of B_i(G_t + G);
//   top variable t:   A_t(r' + L), r' = r - {t}, L over all nl low variables,
//                     = X1(L - {0}) when 0 is not in L, X1 + X2 when it is,
//                     X1, X2 the transforms over the low variables but 0 of
//                     the families G_t + G (0 not in G) and G_t + G + {0},
//                     G_t <= r'.
// So a rank forms the folded score tables of a virtual job of nl variables
// with nl + 2k tables over the same nl - 1-bit index space (table i < nl:
// node i, bit i squeezed out; tables nl + 2q and nl + 2q + 1: X1 and X2 of
// top variable nl + q, bit 0 squeezed out), runs the step-2 kernels on it,
// and combines X1 and X2 into each top variable's slab.  No exchange is
// needed: the score table is small and every rank holds it.
// ---------------------------------------------------------------------------

// The folded tables, in the virtual job's canonical family order (Kv per
// table), from the job's shifted scores lbs (K per node, the same shift).
template <typename T>
__global__ void k_fold_scores(int n, int nl, int d, int64_t K, int64_t Kv, uint32_t r,
                              const T* __restrict__ lbs, T* __restrict__ out)
{
    using L = LogOps<T>;
    const int k = n - nl;
    const int64_t total = (int64_t)(nl + 2 * k) * Kv;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(x / Kv);
        uint32_t f = (uint32_t)(x % Kv);
        int sz = 0;
        while (f >= binom(nl - 1, sz)) { f -= binom(nl - 1, sz); ++sz; }
        const uint32_t cm = colex_unrank(f, sz, nl - 1);
        int node;
        uint32_t G, tops;
        if (u < nl) {
            node = u;
            G = expand(cm, u);                          // over the nl low variables
            tops = r;
        } else {
            const int q = (u - nl) >> 1;
            node = nl + q;
            G = (cm << 1) | (uint32_t)((u - nl) & 1);   // X2: variable 0 in the family
            tops = r & ~(1u << q);
        }
        const int g = __popc(G);
        T m = L::ninf(), s = T(0);
        if (g <= d) {
            for (uint32_t t = tops;; t = (t - 1) & tops) {
                if (g + __popc(t) <= d) {
                    const uint32_t c = squeeze(G | (t << nl), node);   // node's own index
                    const T v = lbs[BN_AT((size_t)node * K + small_subset_rank(c, n - 1), 1, (size_t)n * K)];
                    if (v != L::ninf()) {
                        if (v > m) {
                            s = s * L::ex(m - v) + T(1);
                            m = v;
                        } else {
                            s += L::ex(v - m);
                        }
                    }
                }
                if (t == 0) break;
            }
        }
        out[x] = m == L::ninf() ? m : m + L::lg(s);
    }
}

// The top variables' slabs (plain order over the nl low variables) from the
// X1 and X2 tables of the virtual job's A (its own layout: tile-level row
// order when TLO, rows of 16 for tables >= 4).
template <typename T, bool TLO>
__global__ void k_top_slabs(int nl, int k, const T* __restrict__ Av, T* __restrict__ Atop)
{
    using L = LogOps<T>;
    const size_t per = (size_t)1 << nl;
    const size_t half = per >> 1;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < per * (size_t)k;
         x += (size_t)gridDim.x * blockDim.x) {
        const size_t q = x >> nl;
        const uint32_t Lw = (uint32_t)(x & (per - 1));
        const uint32_t c = Lw >> 1;
        const uint32_t pos = TLO ? (tlo_row(c >> 4, 9) << 4) | (c & 15u) : c;
        const T* X1 = Av + (size_t)(nl + 2 * q) * half;
        T v = X1[BN_AT(pos, 1, half)];
        if (Lw & 1u) v = L::lse(v, X1[half + BN_AT(pos, 1, half)]);
        Atop[x] = v;
    }
}

// *word = max(*word, *other): another rank's floored level maximum.
__global__ void k_word_max(int* __restrict__ word, const int* __restrict__ other)
{
    if (threadIdx.x == 0 && *other != kLevelUnset) atomicMax(word, *other);
}

#ifndef BN_MEGA  // host launchers (bn_mega.cu includes only the device code)
#ifdef BN_CHECK_BOUNDS
BN_BOUNDS_READER(bounds_line_levels)
#endif
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

bool rows64_fit(const Plan& P)
{
    return P.prec == 0 && P.n >= LB64 + 1 && P.n - LB64 < BT;
}

// Threads per block for a level of nt tiles: 256, or fewer for the small
// levels, so that a level's blocks spread over all SMs (two per SM at least).
static unsigned level_block(uint32_t nt)
{
    for (unsigned b = 256; b > 64; b >>= 1)
        if ((uint64_t)nt >= (uint64_t)b * 2 * 152) return b;
    return 64;
}

uint32_t shard_level_tiles(const Plan& P, int hl)
{
    const int nh = P.n - (P.prec == 0 ? LB64 : LB);
    const int k = P.shard_k, hr = __builtin_popcount(P.shard_r);
    if (hl - hr < 0 || hl - hr > nh - k) return 0;
    return (uint32_t)choose(nh - k, hl - hr);
}

// One level of a split job's sweep: the rank's tiles (P.shard_r, P.shard_k).
// With P.slab, A holds the rank's slabs of the low nodes and Atop the top
// variables' slabs (the kernels' SLAB form, launched directly: a split job
// is never recorded into a batch).
template <typename T, bool TLO>
static cudaError_t rows_level(const Plan& P, int sweep, int hl, uint32_t nt, unsigned tb, dim3 grid,
                              const void* A, void* X, const void* Atop, cudaStream_t s)
{
    const uint32_t rf = P.shard_r;
    const int kf = P.shard_k;
    const T* a = (const T*)A;
    const T* at = (const T*)Atop;
    if (P.slab) {
        if (sweep == 0)
            k_forward_rows<T, TLO, true><<<grid, tb, 0, s>>>(P.n, hl, nt, a, (T*)X, P.js, rf, kf, at);
        else
            k_backward_rows<T, TLO, true><<<grid, tb, 0, s>>>(P.n, hl, nt, a, (T*)X, P.js, rf, kf, at);
        return cudaGetLastError();
    }
    const int kid = sizeof(T) == 8 ? (sweep == 0 ? KID_FROWS_D : KID_BROWS_D)
                    : TLO ? (sweep == 0 ? KID_FROWS_F_TLO : KID_BROWS_F_TLO)
                          : (sweep == 0 ? KID_FROWS_F : KID_BROWS_F);
    if (sweep == 0)
        return launch_or_record(kid, k_forward_rows<T, TLO>, grid, tb, 0, s, P.n, hl, nt, a, (T*)X, P.js,
                                rf, kf, at);
    return launch_or_record(kid, k_backward_rows<T, TLO>, grid, tb, 0, s, P.n, hl, nt, a, (T*)X, P.js, rf,
                            kf, at);
}

cudaError_t launch_rows_level(const Plan& P, int sweep, int hl, const void* A, void* X, cudaStream_t s,
                              const void* Atop)
{
    const uint32_t nt = shard_level_tiles(P, hl);
    if (nt == 0) return cudaSuccess;
    const unsigned tb = rec_block(level_block(nt));
    const dim3 grid((nt + tb - 1) / tb, P.nj);
    if (P.prec == 0) return rows_level<double, false>(P, sweep, hl, nt, tb, grid, A, X, Atop, s);
    if (use_tlo(P)) return rows_level<float, true>(P, sweep, hl, nt, tb, grid, A, X, Atop, s);
    return rows_level<float, false>(P, sweep, hl, nt, tb, grid, A, X, Atop, s);
}

cudaError_t launch_fold_scores(const Plan& P, int nl, int64_t Kv, uint32_t r, const void* lbs, void* out,
                               cudaStream_t s)
{
    const int64_t total = (int64_t)(nl + 2 * (P.n - nl)) * Kv;
    const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (P.prec == 0)
        k_fold_scores<double><<<grid, 256, 0, s>>>(P.n, nl, P.d, P.K, Kv, r, (const double*)lbs, (double*)out);
    else
        k_fold_scores<float><<<grid, 256, 0, s>>>(P.n, nl, P.d, P.K, Kv, r, (const float*)lbs, (float*)out);
    return cudaGetLastError();
}

cudaError_t launch_top_slabs(const Plan& V, int k, const void* Av, void* Atop, cudaStream_t s)
{
    const int nl = V.n;
    const uint64_t total = (uint64_t)k << nl;
    if (total == 0) return cudaSuccess;                 // no top variables (one rank)
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, 152 * 16);
    if (V.prec == 0)
        k_top_slabs<double, false><<<grid, 256, 0, s>>>(nl, k, (const double*)Av, (double*)Atop);
    else if (use_tlo(V))
        k_top_slabs<float, true><<<grid, 256, 0, s>>>(nl, k, (const float*)Av, (float*)Atop);
    else
        k_top_slabs<float, false><<<grid, 256, 0, s>>>(nl, k, (const float*)Av, (float*)Atop);
    return cudaGetLastError();
}

cudaError_t launch_word_max(int* word, const int* other, cudaStream_t s)
{
    k_word_max<<<1, 32, 0, s>>>(word, other);
    return cudaGetLastError();
}

uint32_t shard_rows_count(const Plan& P, uint32_t r, int hl)
{
    Plan Q = P;
    Q.shard_r = r;
    return shard_level_tiles(Q, hl);
}

cudaError_t launch_level_rows(const Plan& P, uint32_t r, int hl, void* X, void* buf, int dir,
                              cudaStream_t s)
{
    const uint32_t nt = shard_rows_count(P, r, hl);
    if (nt == 0) return cudaSuccess;
    const unsigned grid = std::min<uint64_t>(((uint64_t)nt * 16 + 255) / 256, 152 * 8);
    if (P.prec == 0)
        k_level_rows<double><<<grid, 256, 0, s>>>(P.n, hl, nt, r, P.shard_k, (double*)X, (double*)buf, dir);
    else
        k_level_rows<float><<<grid, 256, 0, s>>>(P.n, hl, nt, r, P.shard_k, (float*)X, (float*)buf, dir);
    return cudaGetLastError();
}

cudaError_t launch_forward_rows(const Plan& P, const void* A, void* F, cudaStream_t s, int* launches)
{
    const int nh = P.n - (P.prec == 0 ? LB64 : LB);
    for (int hl = 0; hl <= nh; ++hl) {
        const uint32_t nt = (uint32_t)choose(nh, hl);
        const unsigned tb = rec_block(level_block(nt));
        const dim3 grid((nt + tb - 1) / tb, P.nj);
        if (P.prec == 0)
            launch_or_record(KID_FROWS_D, k_forward_rows<double, false>, grid, tb, 0, s, P.n, hl, nt, (const double*)A,
                                                               (double*)F, P.js, 0u, 0, (const double*)nullptr);
        else if (use_tlo(P))
            launch_or_record(KID_FROWS_F_TLO, k_forward_rows<float, true>, grid, tb, 0, s, P.n, hl, nt, (const float*)A,
                                                             (float*)F, P.js, 0u, 0, (const float*)nullptr);
        else
            launch_or_record(KID_FROWS_F, k_forward_rows<float, false>, grid, tb, 0, s, P.n, hl, nt, (const float*)A,
                                                              (float*)F, P.js, 0u, 0, (const float*)nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

cudaError_t launch_backward_rows(const Plan& P, const void* A, void* Rc, cudaStream_t s,
                                 int* launches)
{
    const int nh = P.n - (P.prec == 0 ? LB64 : LB);
    for (int hl = nh; hl >= 0; --hl) {
        const uint32_t nt = (uint32_t)choose(nh, hl);
        const unsigned tb = rec_block(level_block(nt));
        const dim3 grid((nt + tb - 1) / tb, P.nj);
        if (P.prec == 0)
            launch_or_record(KID_BROWS_D, k_backward_rows<double, false>, grid, tb, 0, s, P.n, hl, nt, (const double*)A,
                                                                (double*)Rc, P.js, 0u, 0, (const double*)nullptr);
        else if (use_tlo(P))
            launch_or_record(KID_BROWS_F_TLO, k_backward_rows<float, true>, grid, tb, 0, s, P.n, hl, nt, (const float*)A,
                                                              (float*)Rc, P.js, 0u, 0, (const float*)nullptr);
        else
            launch_or_record(KID_BROWS_F, k_backward_rows<float, false>, grid, tb, 0, s, P.n, hl, nt, (const float*)A,
                                                               (float*)Rc, P.js, 0u, 0, (const float*)nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

cudaError_t launch_rows_cluster(const Plan& P, const void* A, void* F, void* Rc, cudaStream_t s,
                                int* launches)
{
    // blocks per cluster: one 256-thread block per 256 tiles of the largest
    // level, at most 8 (the portable cluster size)
    const int nh = P.n - LB;
    const uint64_t widest = choose(nh, nh / 2);
    const unsigned kCluster = (unsigned)std::min<uint64_t>(8, (widest + 255) / 256);
    const int items = 2 * P.nj;
    // at most two blocks per SM: 152 * 2 blocks at once
    const unsigned clusters = (unsigned)std::min(items, 152 * 2 / (int)kCluster);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * kCluster, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_rows_cluster, P.n, items, (const float*)A, (float*)F,
                                       (float*)Rc, P.js);
    if (e == cudaSuccess && launches) ++*launches;
    return e;
}

#endif  // BN_MEGA

}  // namespace bn

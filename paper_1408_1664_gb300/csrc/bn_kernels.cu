// bn_kernels.cu -- sm_103a kernels of the five steps of Algorithm 1.
//
// Step 1  k_pack_planes, k_lgamma_table, k_scores, k_node_max, k_shift_scores
// Step 2  k_upzeta         truncated upward zeta (Eq. 7, Definition 1)
// Step 3  k_forward_level, k_backward_level   F (Eq. 9) and R (Eq. 10)
// Step 4  k_gamma_p1, k_gamma_p2              truncated downward zeta (Eq. 12)
// Step 5  k_edges          Eq. 11 and the division by P(D)
//
// Values are logs: natural logs in FP64, base-2 logs in FP32 (see
// bn_device.cuh).  Every node's scores are shifted by their maximum c_i
// before step 2: replacing B_i by B_i / exp(c_i) scales every order's weight
// by the same factor prod_i exp(-c_i), which cancels in P(u->v | D), and
// keeps the log magnitudes of A, F, R and Gamma small.
#include "bn_device.cuh"
#include "bn_kernels.cuh"

#include <algorithm>
#include <cmath>

namespace bn {

static constexpr unsigned FULL = 0xffffffffu;

// ===========================================================================
// Step 1: local scores.
// ===========================================================================

// planes[(v*rmax + x)*W + w] bit b  <=>  data[(64w + b)*n + v] == x.
// mj (may be null) holds the job's own sample count at the job stride; m
// then only bounds the padded group layout.
__global__ void k_pack_planes(const uint8_t* __restrict__ data, int n, int m, int rmax, int W,
                              uint64_t* __restrict__ planes, const int* __restrict__ mj, size_t js)
{
    data = job_ptr(data, js);
    planes = job_ptr(planes, js);
    if (mj) m = *job_ptr(mj, js);
    const int64_t total = (int64_t)n * rmax * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(t % W);
        const int64_t vx = t / W;
        const int x = (int)(vx % rmax);
        const int v = (int)(vx / rmax);
        uint64_t word = 0;
        const int s0 = w * 64;
        const int cnt = min(64, m - s0);
        for (int b = 0; b < cnt; ++b)
            word |= (uint64_t)(data[(size_t)(s0 + b) * n + v] == x) << b;
        planes[t] = word;
    }
}

// err |= 1 when some data value is not below its variable's arity.
__global__ void k_check_data(const uint8_t* __restrict__ data, const uint8_t* __restrict__ arity,
                             int n, int m, int* err)
{
    const int64_t total = (int64_t)n * m;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (data[t] >= arity[t % n]) atomicOr(err, 1);
    }
}

// T[row*(m+1) + N] = [lgamma(alpha_row + N) - lgamma(alpha_row)] * scale,
// N = 0..m, rounded to an integer: the fixed-point table (scale = 2^S) the
// score kernels sum exactly in int64.
// In a batch group fxj holds each job's (scale, 1/scale) and mj its own m:
// entries past the job's m stay 0 (no count reaches them).
__global__ void k_lgamma_table(const double* __restrict__ alpha, int rows, int m,
                               long long* __restrict__ T, size_t js, double scale,
                               const double* __restrict__ fxj, const int* __restrict__ mj)
{
    alpha = job_ptr(alpha, js);
    T = job_ptr(T, js);
    if (fxj) scale = job_ptr(fxj, js)[0];
    const int mown = mj ? *job_ptr(mj, js) : m;
    const int64_t total = (int64_t)rows * (m + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(t / (m + 1));
        const int N = (int)(t % (m + 1));
        const double a = alpha[row];
        T[t] = (N == 0 || N > mown) ? 0ll
                                    : __double2ll_rn((lgamma(a + (double)N) - lgamma(a)) * scale);
    }
}

// Bit pattern of the double equal to the integer q >= 1, by integer
// operations only.
__device__ __forceinline__ long long double_bits(uint32_t q)
{
    const int e = 31 - __clz(q);
    return ((long long)(1023 + e) << 52) | (long long)(((uint64_t)q << (52 - e)) & ((1ull << 52) - 1));
}

// Row of the denominator D in the sorted table of denominators.  Positive
// doubles are ordered like their bit patterns, so the search compares
// integers: the FP64 pipe, narrow on this GPU, is not used.
__device__ __forceinline__ int find_row(const double* Dvals, int rows, uint32_t D)
{
    const long long key = double_bits(D);
    int lo = 0, hi = rows - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__double_as_longlong(Dvals[mid]) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ double warp_sum(double x)
{
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

__device__ __forceinline__ long long warp_sum(long long x)
{
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

__device__ __forceinline__ unsigned long long to_fixed(double x) { return __double2ull_rn(x); }
__device__ __forceinline__ unsigned long long to_fixed(float x) { return __float2ull_rn(x); }
template <typename T> __device__ __forceinline__ T from_fixed(unsigned long long u);
template <> __device__ __forceinline__ double from_fixed<double>(unsigned long long u)
{
    return __ull2double_rn(u);
}
template <> __device__ __forceinline__ float from_fixed<float>(unsigned long long u)
{
    return __ull2float_rn(u);
}

// Step-1 kernels of a batch group run for every job of the group at once:
// job blockIdx.y finds its arrays js bytes after those of job blockIdx.y - 1.
#define BN_JOB_SCORES()                                                                   \
    do {                                                                                  \
        planes = job_ptr(planes, js);                                                     \
        Dvals = job_ptr(Dvals, js);                                                       \
        T = job_ptr(T, js);                                                               \
        if (log_rho) log_rho = job_ptr(log_rho, js);                                      \
        masks = job_ptr(masks, js);                                                       \
        cmasks = job_ptr(cmasks, js);                                                     \
        logB = job_ptr(logB, js);                                                         \
        if (fxj) tinv = job_ptr(fxj, js)[1];                                              \
    } while (0)

// One warp per family x = i*K + f.  Counts N_jk = popc(AND of bit planes),
// lanes split the words of a plane and the cells of the table lookups.
//   log B_i(G) = log rho(|G|) + sum_j [ -T_q(N_j) + sum_k T_qr(N_jk) ]
// with T_a(N) = lgamma(a+N) - lgamma(a), a = ess/q and ess/(q r_i).
__global__ void __launch_bounds__(256)
k_scores(int n, int d, int m, int W, int rmax, int64_t K, const uint8_t* __restrict__ arity,
         const uint64_t* __restrict__ planes, const double* __restrict__ Dvals, int rows,
         const long long* __restrict__ T, const double* __restrict__ log_rho, int64_t x_begin,
         int64_t x_count, uint32_t* __restrict__ masks, uint32_t* __restrict__ cmasks,
         double* __restrict__ logB, int64_t* __restrict__ debug_counts, size_t js, double tinv,
         const double* __restrict__ fxj)
{
    BN_JOB_SCORES();
    arity = job_ptr(arity, js);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t xi = warp0; xi < x_count; xi += nwarps) {
        const int64_t x = x_begin + xi;
        const int i = (int)(x / K);
        uint32_t f = (uint32_t)(x % K);
        int k = 0;
        while (f >= binom(n - 1, k)) { f -= binom(n - 1, k); ++k; }
        const uint32_t cm = colex_unrank(f, k, n - 1);
        const uint32_t G = expand(cm, i);
        int par[32];
        int rad[32];
        int np = 0;
        uint32_t q = 1;                             // at most 65536 cells
        for (uint32_t g = G; g; g &= g - 1) {
            const int p = __ffs(g) - 1;
            par[np] = p;
            rad[np] = arity[p];
            q *= arity[p];
            ++np;
        }
        const int ri = arity[i];
        const int row_q = find_row(Dvals, rows, q);
        const int row_qr = find_row(Dvals, rows, q * (uint32_t)ri);
        const long long* Tq = T + (size_t)row_q * (m + 1);
        const long long* Tqr = T + (size_t)row_qr * (m + 1);
        const int64_t qi = (int64_t)q;
        int dig[32];
        for (int t = 0; t < np; ++t) dig[t] = 0;
        long long acc = 0;
        for (int64_t cfg = 0; cfg < qi; ++cfg) {
            uint32_t Nj = 0;
            for (int xv = 0; xv < ri; ++xv) {
                uint32_t part = 0;
                for (int w = lane; w < W; w += 32) {
                    uint64_t M = planes[((size_t)i * rmax + xv) * W + w];
                    for (int t = 0; t < np; ++t)
                        M &= planes[((size_t)par[t] * rmax + dig[t]) * W + w];
                    part += (uint32_t)__popcll(M);
                }
                const uint32_t N = __reduce_add_sync(FULL, part);
                Nj += N;
                const int64_t cell = cfg * ri + xv;
                if (lane == (int)(cell & 31)) {
                    acc += Tqr[N];
                    if (debug_counts) debug_counts[cell] = N;
                }
            }
            if (lane == (int)(cfg & 31)) acc -= Tq[Nj];
            for (int t = 0; t < np; ++t) {          // mixed-radix increment
                if (++dig[t] < rad[t]) break;
                dig[t] = 0;
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            {
                const size_t xc = BN_AT(x, 1, (size_t)n * K);
                logB[xc] = (double)acc * tinv + (log_rho ? log_rho[k] : 0.0);
                masks[xc] = G;
                cmasks[xc] = cm;
            }
        }
    }
    (void)d;
}

// Scores with one thread per family, for binary data (every arity 2) and
// families of at most 4 parents: at most 16 parent configurations and 32
// cells.  The launch covers the first Kc families of every node (those of
// at most 4 parents; Kc = K when d <= 4); thread index xc stands for family
// (xc / Kc) * K + xc % Kc.  Word by
// word the thread builds the masks of all 16 configurations as a product
// tree of the parent planes (configuration index: digit t = value of parent
// t, parent 0 least significant; a missing parent t >= |G| contributes the
// planes (all ones, none), so the configurations with digit 1 there stay
// empty), counts every cell with popc, and adds the BDeu terms in FP64 in
// the order (configuration, child value).  Empty cells add
// lgamma(a) - lgamma(a) = 0 exactly, so the padding changes nothing.
// The bit planes (n * 2 * W words) stay in L1.
__global__ void __launch_bounds__(128)
k_scores_bin(int n, int m, int W, int64_t K, int64_t Kc, const uint64_t* __restrict__ planes,
             const double* __restrict__ Dvals, int rows, const long long* __restrict__ T,
             const double* __restrict__ log_rho, int64_t x_begin, int64_t x_count,
             uint32_t* __restrict__ masks, uint32_t* __restrict__ cmasks,
             double* __restrict__ logB, int64_t* __restrict__ debug_counts, size_t js, double tinv,
         const double* __restrict__ fxj)
{
    BN_JOB_SCORES();
    __shared__ uint32_t bt[32][5];                  // C(a, b), b <= 4, for the unrank
    for (int e = threadIdx.x; e < 32 * 5; e += blockDim.x) bt[e / 5][e % 5] = binom(e / 5, e % 5);
    __syncthreads();
    const int64_t xi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (xi >= x_count) return;
    const int64_t xc = x_begin + xi;
    const int i = (int)(xc / Kc);
    uint32_t f = (uint32_t)(xc % Kc);
    const int64_t x = (int64_t)i * K + f;
    int k = 0;
    while (f >= bt[n - 1][k]) { f -= bt[n - 1][k]; ++k; }
    uint32_t cm = 0;                                // colex unrank of f among k-subsets
    {
        int c = n - 2;
        for (int t = k; t >= 1; --t) {
            while (bt[c][t] > f) --c;
            cm |= 1u << c;
            f -= bt[c][t];
            --c;
        }
    }
    const uint32_t G = expand(cm, i);
    int par[4];
    {
        uint32_t g = G;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            par[t] = g ? __ffs(g) - 1 : -1;
            g &= g - 1;
        }
    }
    uint32_t cnt[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) cnt[c] = 0;
    for (int w = 0; w < W; ++w) {
        uint64_t E[16];
        E[0] = ~0ull;
#pragma unroll
        for (int t = 3; t >= 0; --t) {              // most significant digit first
            const uint64_t p0 = par[t] >= 0 ? planes[((size_t)par[t] * 2) * W + w] : ~0ull;
            const uint64_t p1 = par[t] >= 0 ? planes[((size_t)par[t] * 2 + 1) * W + w] : 0ull;
            const int size = 1 << (3 - t);
#pragma unroll
            for (int j = size - 1; j >= 0; --j) {
                const uint64_t e = E[j];
                E[2 * j] = e & p0;
                E[2 * j + 1] = e & p1;
            }
        }
        const uint64_t c0 = planes[((size_t)i * 2) * W + w];
        const uint64_t c1 = planes[((size_t)i * 2 + 1) * W + w];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            cnt[2 * j] += (uint32_t)__popcll(E[j] & c0);
            cnt[2 * j + 1] += (uint32_t)__popcll(E[j] & c1);
        }
    }
    const uint32_t q = 1u << k;
    const long long* Tq = T + (size_t)find_row(Dvals, rows, q) * (m + 1);
    const long long* Tqr = T + (size_t)find_row(Dvals, rows, 2u * q) * (m + 1);
    long long acc = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        acc -= Tq[cnt[2 * j] + cnt[2 * j + 1]];
        acc += Tqr[cnt[2 * j]];
        acc += Tqr[cnt[2 * j + 1]];
    }
    if (debug_counts) {
        const int cells = 2 << k;
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (c < cells) debug_counts[c] = cnt[c];
    }
    {
        const size_t xc = BN_AT(x, 1, (size_t)n * K);
        logB[xc] = (double)acc * tinv + (log_rho ? log_rho[k] : 0.0);
        masks[xc] = G;
        cmasks[xc] = cm;
    }
}

// Scores of the families with exactly k = 4 + HB parents (5 <= k <= 8), for
// binary data.  A family takes 2^HB adjacent threads of a warp; thread h
// owns the 16 configurations whose digits of parents 4..k-1 spell h.  Word
// by word it ANDs the planes of those high digits into one mask, splits the
// mask over the four low parents with the product tree of k_scores_bin and
// counts the 32 cells with popc.  Its FP64 sum of BDeu terms meets those of
// the family's other threads in an xor butterfly (every lane ends with the
// same sum, so the order is fixed).  The launch covers families f_begin ..
// f_begin + f_count - 1 of the n * C(n-1, k) families of this size, family
// g being rank g % C(n-1, k) of node g / C(n-1, k); off is the index of the
// first k-parent family inside a node's block of K.
template <int HB>
__global__ void __launch_bounds__(128)
k_scores_bin_hi(int n, int m, int W, int64_t K, int64_t off, int64_t Ck,
                const uint64_t* __restrict__ planes, const double* __restrict__ Dvals, int rows,
                const long long* __restrict__ T, const double* __restrict__ log_rho, int64_t f_begin,
                int64_t f_count, uint32_t* __restrict__ masks, uint32_t* __restrict__ cmasks,
                double* __restrict__ logB, int64_t* __restrict__ debug_counts, size_t js, double tinv,
         const double* __restrict__ fxj)
{
    BN_JOB_SCORES();
    constexpr int k = 4 + HB;
    constexpr int NH = 1 << HB;
    __shared__ uint32_t bt[32][k + 1];
    for (int e = threadIdx.x; e < 32 * (k + 1); e += blockDim.x)
        bt[e / (k + 1)][e % (k + 1)] = binom(e / (k + 1), e % (k + 1));
    __syncthreads();
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int h = (int)(gt & (NH - 1));
    const bool live = (gt >> HB) < f_count;
    // a thread past the end works on the last family (all lanes stay in the
    // butterfly) and writes nothing
    const int64_t g = f_begin + (live ? (gt >> HB) : f_count - 1);
    const int i = (int)(g / Ck);
    uint32_t r = (uint32_t)(g % Ck);
    uint32_t cm = 0;                                // colex unrank of r among k-subsets
    {
        int c = n - 2;
        for (int t = k; t >= 1; --t) {
            while (bt[c][t] > r) --c;
            cm |= 1u << c;
            r -= bt[c][t];
            --c;
        }
    }
    const uint32_t G = expand(cm, i);
    int par[k];
    {
        uint32_t gg = G;
#pragma unroll
        for (int t = 0; t < k; ++t) {
            par[t] = __ffs(gg) - 1;
            gg &= gg - 1;
        }
    }
    // plane rows of the high digits of configuration block h
    int hrow[HB];
#pragma unroll
    for (int t = 0; t < HB; ++t) hrow[t] = (par[4 + t] * 2 + ((h >> t) & 1)) * W;
    uint32_t cnt[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) cnt[c] = 0;
    for (int w = 0; w < W; ++w) {
        uint64_t E[16];
        E[0] = planes[hrow[0] + w];
#pragma unroll
        for (int t = 1; t < HB; ++t) E[0] &= planes[hrow[t] + w];
#pragma unroll
        for (int t = 3; t >= 0; --t) {              // most significant digit first
            const uint64_t p0 = planes[((size_t)par[t] * 2) * W + w];
            const uint64_t p1 = planes[((size_t)par[t] * 2 + 1) * W + w];
            const int size = 1 << (3 - t);
#pragma unroll
            for (int j = size - 1; j >= 0; --j) {
                const uint64_t e = E[j];
                E[2 * j] = e & p0;
                E[2 * j + 1] = e & p1;
            }
        }
        const uint64_t c0 = planes[((size_t)i * 2) * W + w];
        const uint64_t c1 = planes[((size_t)i * 2 + 1) * W + w];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            cnt[2 * j] += (uint32_t)__popcll(E[j] & c0);
            cnt[2 * j + 1] += (uint32_t)__popcll(E[j] & c1);
        }
    }
    const uint32_t q = 1u << k;
    const long long* Tq = T + (size_t)find_row(Dvals, rows, q) * (m + 1);
    const long long* Tqr = T + (size_t)find_row(Dvals, rows, 2u * q) * (m + 1);
    long long acc = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        acc -= Tq[cnt[2 * j] + cnt[2 * j + 1]];
        acc += Tqr[cnt[2 * j]];
        acc += Tqr[cnt[2 * j + 1]];
    }
#pragma unroll
    for (int o = 1; o < NH; o <<= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (!live) return;
    if (debug_counts) {
#pragma unroll
        for (int c = 0; c < 32; ++c) debug_counts[32 * h + c] = cnt[c];
    }
    if (h == 0) {
        const int64_t x = (int64_t)i * K + off + (int64_t)(g % Ck);
        {
            const size_t xc = BN_AT(x, 1, (size_t)n * K);
            logB[xc] = (double)acc * tinv + (log_rho ? log_rho[k] : 0.0);
            masks[xc] = G;
            cmasks[xc] = cm;
        }
    }
}

// Scores of the families with exactly KP parents (5 <= KP <= 8), binary
// data, from a histogram of the samples' cells: one warp per family.  A lane
// takes runs of 16 samples; for each valid sample it forms the cell key
// (parent t's value in bit t, the child's value in bit KP) from the bit
// planes with shifts and masks, and adds 1 to the warp's histogram of
// 2^(KP+1) cells in shared memory.  The BDeu terms follow configuration by
// configuration (cell = 2 * configuration + child value, the canonical
// order) in 64-bit fixed point, so the sum equals the per-cell kernels' bit
// for bit.  The work is O(m) per family instead of O(2^KP m / 64) popcs:
// the better choice once 2^KP cells outnumber the words.
template <int KP>
__global__ void __launch_bounds__(256)
k_scores_bin_hist(int n, int m, int W, int64_t K, int64_t off, int64_t Ck,
                  const uint64_t* __restrict__ planes, const double* __restrict__ Dvals, int rows,
                  const long long* __restrict__ T, const double* __restrict__ log_rho,
                  int64_t f_begin, int64_t f_count, uint32_t* __restrict__ masks,
                  uint32_t* __restrict__ cmasks, double* __restrict__ logB,
                  int64_t* __restrict__ debug_counts, size_t js, double tinv,
                  const double* __restrict__ fxj)
{
    BN_JOB_SCORES();
    constexpr int NCFG = 1 << KP;
    __shared__ uint32_t hist[8][2 * NCFG];
    __shared__ uint32_t bt[32][KP + 1];
    for (int e = threadIdx.x; e < 32 * (KP + 1); e += blockDim.x)
        bt[e / (KP + 1)][e % (KP + 1)] = binom(e / (KP + 1), e % (KP + 1));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* hw = hist[warp];
    for (int c = lane; c < 2 * NCFG; c += 32) hw[c] = 0u;
    __syncthreads();
    const long long* Tq = T + (size_t)find_row(Dvals, rows, (uint32_t)NCFG) * (m + 1);
    const long long* Tqr = T + (size_t)find_row(Dvals, rows, 2u * NCFG) * (m + 1);
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    for (int64_t fi = (int64_t)blockIdx.x * 8 + warp; fi < f_count; fi += nwarps) {
        const int64_t g = f_begin + fi;
        const int i = (int)(g / Ck);
        uint32_t r = (uint32_t)(g % Ck);
        const uint32_t rank = r;
        uint32_t cm = 0;                            // colex unrank of r among KP-subsets
        {
            int c = n - 2;
            for (int t = KP; t >= 1; --t) {
                while (bt[c][t] > r) --c;
                cm |= 1u << c;
                r -= bt[c][t];
                --c;
            }
        }
        const uint32_t G = expand(cm, i);
        const uint64_t* pr[KP];                     // the value-1 plane of each parent
        {
            uint32_t gg = G;
#pragma unroll
            for (int t = 0; t < KP; ++t) {
                pr[t] = planes + ((size_t)(__ffs(gg) - 1) * 2 + 1) * W;
                gg &= gg - 1;
            }
        }
        const uint64_t* c0 = planes + (size_t)i * 2 * W;
        const uint64_t* c1 = c0 + W;
        for (int ch = lane; ch < 4 * W; ch += 32) {
            const int w = ch >> 2, sh = (ch & 3) * 16;
            const uint64_t x1w = c1[w];
            uint32_t valid = (uint32_t)((c0[w] | x1w) >> sh) & 0xFFFFu;
            const uint32_t x1 = (uint32_t)(x1w >> sh);
            uint32_t pb[KP];
#pragma unroll
            for (int t = 0; t < KP; ++t) pb[t] = (uint32_t)(pr[t][w] >> sh);
            while (valid) {
                const int b = __ffs(valid) - 1;
                valid &= valid - 1;
                uint32_t key = (x1 >> b & 1u) << KP;
#pragma unroll
                for (int t = 0; t < KP; ++t) key |= (pb[t] >> b & 1u) << t;
                atomicAdd(&hw[key], 1u);
            }
        }
        __syncwarp();
        long long acc = 0;
        for (int j = lane; j < NCFG; j += 32) {
            const uint32_t N0 = hw[j], N1 = hw[j | NCFG];
            acc += Tqr[N0] + Tqr[N1] - Tq[N0 + N1];
            if (debug_counts) {
                debug_counts[2 * j] = N0;
                debug_counts[2 * j + 1] = N1;
            }
            hw[j] = 0u;
            hw[j | NCFG] = 0u;
        }
        __syncwarp();
        acc = warp_sum(acc);
        if (lane == 0) {
            const int64_t x = (int64_t)i * K + off + rank;
            {
                const size_t xc = BN_AT(x, 1, (size_t)n * K);
                logB[xc] = (double)acc * tinv + (log_rho ? log_rho[KP] : 0.0);
                masks[xc] = G;
                cmasks[xc] = cm;
            }
        }
    }
}

// Scores with one warp per family and one lane per 64-sample word (m <= 2048):
// every lane keeps its word of each parent plane and child plane in
// registers, so a cell costs an AND chain, a popc and one warp reduction.
// Lane c % 32 keeps the count of cell c and adds its lgamma-table term when a
// run of 32 cells is complete (FP64 adds in a fixed order).
template <int MP, int MR>
__global__ void __launch_bounds__(256)
k_scores_w(int n, int m, int W, int rmax, int64_t K, const uint8_t* __restrict__ arity,
           const uint64_t* __restrict__ planes, const double* __restrict__ Dvals, int rows,
           const long long* __restrict__ T, const double* __restrict__ log_rho, int64_t x_begin,
           int64_t x_count, uint32_t* __restrict__ masks, uint32_t* __restrict__ cmasks,
           double* __restrict__ logB, int64_t* __restrict__ debug_counts, size_t js, double tinv,
         const double* __restrict__ fxj)
{
    BN_JOB_SCORES();
    arity = job_ptr(arity, js);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool has_word = lane < W;
    for (int64_t xi = warp0; xi < x_count; xi += nwarps) {
        const int64_t x = x_begin + xi;
        const int i = (int)(x / K);
        uint32_t f = (uint32_t)(x % K);
        int k = 0;
        while (f >= binom(n - 1, k)) { f -= binom(n - 1, k); ++k; }
        const uint32_t cm = colex_unrank(f, k, n - 1);
        const uint32_t G = expand(cm, i);
        uint64_t pw[MP][MR];
        int rad[MP];
        uint32_t g = G;
        int q = 1;
#pragma unroll
        for (int t = 0; t < MP; ++t) {
            rad[t] = 1;
#pragma unroll
            for (int v = 0; v < MR; ++v) pw[t][v] = (v == 0) ? ~0ull : 0ull;
            if (t < k) {
                const int p = __ffs(g) - 1;
                g &= g - 1;
                rad[t] = arity[p];
                q *= rad[t];
#pragma unroll
                for (int v = 0; v < MR; ++v)
                    pw[t][v] = (v < rad[t] && has_word) ? planes[((size_t)p * rmax + v) * W + lane] : 0ull;
            }
        }
        const int ri = arity[i];
        uint64_t cw[MR];
#pragma unroll
        for (int v = 0; v < MR; ++v)
            cw[v] = (v < ri && has_word) ? planes[((size_t)i * rmax + v) * W + lane] : 0ull;
        const long long* Tq = T + (size_t)find_row(Dvals, rows, (uint32_t)q) * (m + 1);
        const long long* Tqr = T + (size_t)find_row(Dvals, rows, (uint32_t)(q * ri)) * (m + 1);
        int dig[MP];
#pragma unroll
        for (int t = 0; t < MP; ++t) dig[t] = 0;
        long long acc = 0;
        uint32_t cur = 0, curj = 0;
        int cell = 0;
        for (int cfg = 0; cfg < q; ++cfg) {
            uint64_t M = ~0ull;
#pragma unroll
            for (int t = 0; t < MP; ++t) {
                uint64_t w = pw[t][0];
#pragma unroll
                for (int v = 1; v < MR; ++v)
                    if (dig[t] == v) w = pw[t][v];
                M &= w;
            }
            uint32_t Nj = 0;
#pragma unroll
            for (int v = 0; v < MR; ++v) {
                if (v < ri) {
                    const uint32_t N = __reduce_add_sync(FULL, (uint32_t)__popcll(M & cw[v]));
                    Nj += N;
                    if (lane == (cell & 31)) {
                        cur = N;
                        if (debug_counts) debug_counts[cell] = N;
                    }
                    if ((cell & 31) == 31) acc += Tqr[cur];
                    ++cell;
                }
            }
            if (lane == (cfg & 31)) curj = Nj;
            if ((cfg & 31) == 31) acc -= Tq[curj];
            bool carry = true;
#pragma unroll
            for (int t = 0; t < MP; ++t) {
                if (carry) {
                    if (++dig[t] < rad[t]) carry = false;
                    else dig[t] = 0;
                }
            }
        }
        if ((cell & 31) != 0 && lane < (cell & 31)) acc += Tqr[cur];
        if ((q & 31) != 0 && lane < (q & 31)) acc -= Tq[curj];
        acc = warp_sum(acc);
        if (lane == 0) {
            {
                const size_t xc = BN_AT(x, 1, (size_t)n * K);
                logB[xc] = (double)acc * tinv + (log_rho ? log_rho[k] : 0.0);
                masks[xc] = G;
                cmasks[xc] = cm;
            }
        }
    }
}

// Register version of k_scores for at most MP parents and child arity at
// most MR: one warp per family, one lane per parent configuration j.  The
// lane ANDs the planes of its configuration's parent values word by word and
// counts each child value with popc, then adds its own BDeu terms
//   -T_q(N_j) + sum_k T_qr(N_jk);
// the warp sum gives log B.  No cross-lane step per cell.
constexpr int SC_MP = 8, SC_MR = 8;
template <int MP, int MR>
__global__ void __launch_bounds__(256)
k_scores_cfg(int n, int m, int W, int rmax, int64_t K, const uint8_t* __restrict__ arity,
             const uint64_t* __restrict__ planes, const double* __restrict__ Dvals, int rows,
             const long long* __restrict__ T, const double* __restrict__ log_rho, int64_t x_begin,
             int64_t x_count, uint32_t* __restrict__ masks, uint32_t* __restrict__ cmasks,
             double* __restrict__ logB, int64_t* __restrict__ debug_counts, size_t js, double tinv,
         const double* __restrict__ fxj)
{
    BN_JOB_SCORES();
    arity = job_ptr(arity, js);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t xi = warp0; xi < x_count; xi += nwarps) {
        const int64_t x = x_begin + xi;
        const int i = (int)(x / K);
        uint32_t f = (uint32_t)(x % K);
        int k = 0;
        while (f >= binom(n - 1, k)) { f -= binom(n - 1, k); ++k; }
        const uint32_t cm = colex_unrank(f, k, n - 1);
        const uint32_t G = expand(cm, i);
        int par[MP], rad[MP];
        uint32_t g = G;
        int q = 1;
#pragma unroll
        for (int t = 0; t < MP; ++t) {
            par[t] = 0;
            rad[t] = 1;
            if (g) {
                par[t] = __ffs(g) - 1;
                g &= g - 1;
                rad[t] = arity[par[t]];
                q *= rad[t];
            }
        }
        const int ri = arity[i];
        const long long* Tq = T + (size_t)find_row(Dvals, rows, (uint32_t)q) * (m + 1);
        const long long* Tqr = T + (size_t)find_row(Dvals, rows, (uint32_t)(q * ri)) * (m + 1);
        const uint64_t* cp = planes + (size_t)i * rmax * W;
        long long acc = 0;
        for (int j0 = 0; j0 < q; j0 += 32) {
            const int j = j0 + lane;
            if (j < q) {
                const uint64_t* pp[MP];
                int jj = j;
#pragma unroll
                for (int t = 0; t < MP; ++t) {
                    const int dg = jj % rad[t];
                    jj /= rad[t];
                    pp[t] = planes + ((size_t)par[t] * rmax + dg) * W;
                }
                uint32_t N[MR];
#pragma unroll
                for (int xv = 0; xv < MR; ++xv) N[xv] = 0;
                for (int w = 0; w < W; ++w) {
                    uint64_t M = ~0ull;
#pragma unroll
                    for (int t = 0; t < MP; ++t)
                        if (t < k) M &= pp[t][w];
#pragma unroll
                    for (int xv = 0; xv < MR; ++xv)
                        if (xv < ri) N[xv] += (uint32_t)__popcll(M & cp[(size_t)xv * W + w]);
                }
                uint32_t Nj = 0;
#pragma unroll
                for (int xv = 0; xv < MR; ++xv) {
                    if (xv < ri) {
                        acc += Tqr[N[xv]];
                        Nj += N[xv];
                        if (debug_counts) debug_counts[(int64_t)j * ri + xv] = N[xv];
                    }
                }
                acc -= Tq[Nj];
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            {
                const size_t xc = BN_AT(x, 1, (size_t)n * K);
                logB[xc] = (double)acc * tinv + (log_rho ? log_rho[k] : 0.0);
                masks[xc] = G;
                cmasks[xc] = cm;
            }
        }
    }
}

// cmax[i] = max_f logB[i*K + f]; one block per node.
__global__ void k_node_max(int64_t K, const double* __restrict__ logB, double* __restrict__ cmax,
                           size_t js)
{
    logB = job_ptr(logB, js);
    cmax = job_ptr(cmax, js);
    __shared__ double red[32];
    const int i = blockIdx.x;
    double mx = -INFINITY;
    for (int64_t f = threadIdx.x; f < K; f += blockDim.x) mx = fmax(mx, logB[(size_t)i * K + f]);
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
        if (threadIdx.x == 0) cmax[i] = mx;
    }
}

template <typename T>
__global__ void k_shift_scores(int64_t total, int64_t K, const double* __restrict__ logB,
                               const double* __restrict__ cmax, T* __restrict__ lbs, size_t js)
{
    logB = job_ptr(logB, js);
    cmax = job_ptr(cmax, js);
    lbs = job_ptr(lbs, js);
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x)
        lbs[x] = (T)LogOps<T>::from_ln(logB[x] - cmax[x / K]);
}

// ===========================================================================
// Step 2: A_i(S) = sum_{G subset S, |G| <= d} B_i(G)  (Eq. 7, q_i = 1).
//
// Index space of node i: the n-1 bits of S with bit i removed.  One block per
// tile (i, H): H = the high n-1-b bits, the 2^b low-bit patterns L in shared
// memory.  The high dimensions of the transform are done by scattering every
// family G = (g_L, G_H) with G_H subset H into slot g_L (log-sum-exp via two
// shared-memory atomic passes: max, then sum of exp); the b low dimensions
// are then summed in shared memory one dimension at a time (the butterfly of
// Algorithm 2).  Every family has |G| <= d, so the truncation is exact; A is
// written to HBM exactly once, coalesced.
// ===========================================================================
template <typename T>
__global__ void __launch_bounds__(256)
k_upzeta(int n, int b, int64_t K, int qbits, const uint32_t* __restrict__ cmasks,
         const T* __restrict__ lbs, T* __restrict__ A, size_t js)
{
    cmasks = job_ptr(cmasks, js);
    lbs = job_ptr(lbs, js);
    A = job_ptr(A, js);
    using O = typename OrdInt<T>::type;
    using U = unsigned long long;
    using L = LogOps<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t tileN = 1u << b;
    U* sm = reinterpret_cast<U*>(smem_raw);
    T* vals = reinterpret_cast<T*>(sm + tileN);
    O* mx = reinterpret_cast<O*>(vals + tileN);
    const int h = n - 1 - b;
    const int i = (int)(blockIdx.x >> h);
    const uint32_t H = blockIdx.x & ((1u << h) - 1u);
    const uint32_t lowm = tileN - 1u;
    const O enc_ninf = ord_enc(L::ninf());
    const T qscale = (T)ldexp(1.0, qbits);

    for (uint32_t t = threadIdx.x; t < tileN; t += blockDim.x) {
        mx[t] = enc_ninf;
        sm[t] = 0ull;
    }
    __syncthreads();
    const uint32_t* cm_i = cmasks + (size_t)i * K;
    const T* lb_i = lbs + (size_t)i * K;
    for (int64_t f = threadIdx.x; f < K; f += blockDim.x) {
        const uint32_t c = cm_i[f];
        if (((c >> b) & ~H) == 0u) atomicMax(&mx[c & lowm], ord_enc(lb_i[f]));
    }
    __syncthreads();
    // Sum of exp(value - slot max) in fixed point: every term is in (0, 1] and
    // a slot holds at most K terms, so 2^qbits * K < 2^64; integer atomics
    // make the sum independent of the order of arrival.
    for (int64_t f = threadIdx.x; f < K; f += blockDim.x) {
        const uint32_t c = cm_i[f];
        if (((c >> b) & ~H) == 0u) {
            const uint32_t slot = c & lowm;
            const T e = L::ex(lb_i[f] - ord_dec(mx[slot]));
            atomicAdd(&sm[slot], to_fixed(e * qscale));
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < tileN; t += blockDim.x) {
        const O e = mx[t];
        vals[t] = (e == enc_ninf) ? L::ninf()
                                  : ord_dec(e) + L::lg(from_fixed<T>(sm[t]) / qscale);
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        const uint32_t jm = (1u << j) - 1u;
        for (uint32_t p = threadIdx.x; p < (tileN >> 1); p += blockDim.x) {
            const uint32_t lo = ((p & ~jm) << 1) | (p & jm);
            const uint32_t hi = lo | (1u << j);
            vals[hi] = L::lse(vals[hi], vals[lo]);
        }
        __syncthreads();
    }
    T* out = A + ((size_t)i << (n - 1)) + ((size_t)H << b);
    for (uint32_t t = threadIdx.x; t < tileN; t += blockDim.x) out[t] = vals[t];
}

// ===========================================================================
// Step 3: F and R' = R(V - .) over the lattice, level by level.
//
// A warp owns a tile of 2^wb consecutive subsets (the low wb bits vary, one
// subset per lane).  Tiles are keyed by their high bits Ht and launched one
// popcount level of Ht at a time (the sub-cube order of Section 3.2.2).
// Terms across tiles read the previous level's tiles; the wb in-tile levels
// are resolved with warp shuffles.
//   F(S)  = sum_{i in S}     A_i(S - {i}) F(S - {i}),  F(empty) = 1  (Eq. 9)
//   R'(T) = sum_{i not in T} A_i(T) R'(T + {i}),       R'(V) = 1
// where R'(T) = R(V - T) turns Eq. 10 into a recursion over T.
// ===========================================================================
// Next subset with the same number of elements in increasing value order
// (the colexicographic successor); x != 0.
__device__ __forceinline__ uint32_t colex_next(uint32_t x)
{
    const uint32_t u = x & (0u - x);
    const uint32_t v = x + u;
    return v | (((v ^ x) >> 2) >> (__ffs(u) - 1));
}

// Branchless online log-sum-exp step: (m, s) represents m + lg(s).
template <typename T>
__device__ __forceinline__ void lse_step(T& m, T& s, T x)
{
    using L = LogOps<T>;
    const T mn = x > m ? x : m;
    if (mn == L::ninf()) return;
    s = s * L::ex(m - mn) + L::ex(x - mn);
    m = mn;
}

// A warp owns 2^wb consecutive subsets (one per lane); the tile's high bits
// Ht are the same for every lane, so the terms across tiles run over the set
// bits of Ht with warp-uniform addresses.  Each warp walks `tpw` tiles in
// colexicographic order of Ht.  A is read once, with a streaming hint so
// that F and R' stay in L2 for the next level.
template <typename T>
__global__ void __launch_bounds__(256)
k_forward_level(int n, int wb, int hl, uint32_t ntiles, int tpw, const T* __restrict__ A,
                T* __restrict__ F, size_t js)
{
    A = job_ptr(A, js);
    F = job_ptr(F, js);
    using L = LogOps<T>;
    // FP32: these tiles keep no per-level bases (bn_device.cuh)
    if (sizeof(T) == 4 && hl == 0 && blockIdx.x == 0 && threadIdx.x == 0)
        level_words(reinterpret_cast<float*>(F), n)[kLevelMode] = 0;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t first = warp * (uint32_t)tpw;
    if (first >= ntiles) return;
    const int nh = n - wb;
    const uint32_t lb = (uint32_t)lane & ((1u << wb) - 1u);
    const bool active = lane < (1 << wb);
    const size_t half = (size_t)1 << (n - 1);
    uint32_t Ht = colex_unrank(first, hl, nh);
    for (uint32_t tile = first; tile < ntiles && tile < first + (uint32_t)tpw; ++tile) {
        const uint32_t S = (Ht << wb) | lb;
        // terms across tiles: i = wb + j for the set bits j of Ht (same for all lanes)
        T m = L::ninf(), sm = T(0);
        uint32_t rest = Ht;
        const int cnt = __popc(Ht);
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
            const int j = __ffs(rest) - 1;
            rest &= rest - 1;
            const uint32_t Hm = Ht & ~(1u << j);
            const T* Ai = A + (size_t)(wb + j) * half + ((size_t)squeeze(Hm, j) << wb);
            const T* Fi = F + ((size_t)Hm << wb);
            if (active) lse_step(m, sm, __ldcs(Ai + lb) + Fi[lb]);
        }
        const T X = (m == L::ninf()) ? m : m + L::lg(sm);
        T a[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            a[i] = L::ninf();
            if (i < wb && active && (S >> i & 1u))
                a[i] = __ldcs(A + (size_t)i * half + squeeze(S & ~(1u << i), i));
        }
        T Fv = (S == 0u) ? T(0) : X;
        for (int l = 1; l <= wb; ++l) {
            T nb[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) nb[i] = __shfl_xor_sync(FULL, Fv, 1 << i);
            if (active && __popc(lb) == l) {
                T mm = X, ss = (X == L::ninf()) ? T(0) : T(1);
#pragma unroll
                for (int i = 0; i < 5; ++i)
                    if (lb >> i & 1u) lse_step(mm, ss, a[i] + nb[i]);
                Fv = mm + L::lg(ss);
            }
        }
        if (active) F[BN_AT(S, 1, (size_t)1 << n)] = Fv;
        if (Ht) Ht = colex_next(Ht);
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_backward_level(int n, int wb, int hl, uint32_t ntiles, int tpw, const T* __restrict__ A,
                 T* __restrict__ Rc, size_t js)
{
    A = job_ptr(A, js);
    Rc = job_ptr(Rc, js);
    using L = LogOps<T>;
    if (sizeof(T) == 4 && hl == n - wb && blockIdx.x == 0 && threadIdx.x == 0)
        level_words(reinterpret_cast<float*>(Rc), n)[kLevelMode] = 0;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t first = warp * (uint32_t)tpw;
    if (first >= ntiles) return;
    const int nh = n - wb;
    const uint32_t wmask = (1u << wb) - 1u;
    const uint32_t lb = (uint32_t)lane & wmask;
    const bool active = lane < (1 << wb);
    const uint32_t full = (uint32_t)(((uint64_t)1 << n) - 1);   // n <= 32
    const uint32_t hmask = (1u << nh) - 1u;
    const size_t half = (size_t)1 << (n - 1);
    uint32_t Ht = colex_unrank(first, hl, nh);
    for (uint32_t tile = first; tile < ntiles && tile < first + (uint32_t)tpw; ++tile) {
        const uint32_t Tm = (Ht << wb) | lb;
        T m = L::ninf(), sm = T(0);
        uint32_t rest = ~Ht & hmask;
        const int cnt = __popc(rest);
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
            const int j = __ffs(rest) - 1;
            rest &= rest - 1;
            const T* Ai = A + (size_t)(wb + j) * half + ((size_t)squeeze(Ht, j) << wb);
            const T* Ri = Rc + ((size_t)(Ht | (1u << j)) << wb);
            if (active) lse_step(m, sm, __ldcs(Ai + lb) + Ri[lb]);
        }
        const T X = (m == L::ninf()) ? m : m + L::lg(sm);
        T a[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            a[i] = L::ninf();
            if (i < wb && active && !(Tm >> i & 1u)) a[i] = __ldcs(A + (size_t)i * half + squeeze(Tm, i));
        }
        T Rv = (Tm == full) ? T(0) : X;
        for (int l = wb - 1; l >= 0; --l) {
            T nb[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) nb[i] = __shfl_xor_sync(FULL, Rv, 1 << i);
            if (active && __popc(lb) == l) {
                T mm = X, ss = (X == L::ninf()) ? T(0) : T(1);
#pragma unroll
                for (int i = 0; i < 5; ++i)
                    if (i < wb && !(lb >> i & 1u)) lse_step(mm, ss, a[i] + nb[i]);
                Rv = mm + L::lg(ss);
            }
        }
        if (active) Rc[BN_AT(Tm, 1, (size_t)1 << n)] = Rv;
        if (Ht) Ht = colex_next(Ht);
    }
}

// ===========================================================================
// Step 4: Gamma_v(G) = sum_{G subset S subset V-{v}} F(S) R'(S + {v}), |G|<=d
// (Eq. 12; F(S) R(V-{v}-S) = F(S) R'(S + {v}), the pairing of Section 3.1.2).
//
// Phase 1: one block per tile of the n-1 bits of S (bit v removed), 2^b low
// bits in shared memory: load s_v = F + R', run the downward butterflies over
// the b low dimensions with the guard of Algorithm 3 (only patterns with at
// most d elements among the dimensions done so far), and keep the outputs
// with at most d low elements: row H of W, nlow entries in canonical order.
// Phase 2: one block per column g of W (a low pattern, d' = d - |g|): the
// downward transform over the h high dimensions, truncated at d', chunk by
// chunk of 2^hc rows; each output is stored at its family index.
// ===========================================================================
template <typename T>
__global__ void __launch_bounds__(256)
k_gamma_p1(int n, int d, int b, uint32_t nlow, const T* __restrict__ F,
           const T* __restrict__ Rc, T* __restrict__ W, size_t js, const T* __restrict__ lq,
           uint32_t vsel)
{
    const int v = blockIdx.z;                       // endpoint: one slice of W each
    if (!(vsel >> v & 1u)) return;                  // an endpoint another rank computes
    F = job_ptr(F, js);
    Rc = job_ptr(Rc, js);
    W = job_ptr(W, js) + (size_t)endpoint_slot(vsel, v) * gridDim.x * nlow;
    using L = LogOps<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* vals = reinterpret_cast<T*>(smem_raw);
    const uint32_t tileN = 1u << b;
    const uint32_t H = blockIdx.x;
    const uint32_t bv = 1u << v;
    constexpr bool kBases = sizeof(T) == 4;         // FP32: per-level bases of F and R'
    __shared__ float off_s[32];
    __shared__ int sh_s;
    __shared__ float fvrel_s;
    if constexpr (kBases) {
        load_gamma_offsets(reinterpret_cast<const float*>(Rc), n, v, off_s, &sh_s, &fvrel_s);
        __syncthreads();
    }
    for (uint32_t t = threadIdx.x; t < tileN; t += blockDim.x) {
        const uint32_t S = expand((H << b) | t, v);
        vals[t] = F[BN_AT(S, 1, (size_t)1 << n)] + Rc[BN_AT(S | bv, 1, (size_t)1 << n)];
        if constexpr (kBases) vals[t] += off_s[BN_AT(__popc(S >> sh_s), 1, 32)];
        if (lq) vals[t] += lq[v * n + __popc(S)];   // q_v(S) of Eq. 12
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        const uint32_t jm = (1u << j) - 1u;
        for (uint32_t p = threadIdx.x; p < (tileN >> 1); p += blockDim.x) {
            const uint32_t lo = ((p & ~jm) << 1) | (p & jm);
            if (__popc(lo & jm) <= d) vals[lo] = L::lse(vals[lo], vals[lo | (1u << j)]);
        }
        __syncthreads();
    }
    T* row = W + (size_t)H * nlow;
    for (uint32_t t = threadIdx.x; t < tileN; t += blockDim.x)
        if (__popc(t) <= d) row[BN_AT(small_subset_rank(t, b), 1, nlow)] = vals[t];
}

// FP32: the down-zeta offsets of endpoint blockIdx.x (one warp; bn_device.cuh).
__global__ void k_gamma_table(int n, const float* __restrict__ F, float* __restrict__ Rc, size_t js,
                              uint32_t vsel)
{
    F = job_ptr(F, js);
    Rc = job_ptr(Rc, js);
    const int v = blockIdx.x;
    if (!(vsel >> v & 1u)) return;
    __shared__ float off[32];
    __shared__ int sh;
    __shared__ float fvrel;
    if (threadIdx.x < 32) off[threadIdx.x] = 0.f;
    __syncwarp();
    gamma_offsets(n, v, F, Rc, off, &sh, &fvrel);
    __syncwarp();
    float* tab = gamma_table(Rc, n) + v * 32;
    const int l = threadIdx.x;
    tab[l] = l < 30 ? off[l] : l == 30 ? __int_as_float(sh) : fvrel;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_gamma_p2(int n, int d, int b, int hc, uint32_t nlow, int64_t K, const T* __restrict__ W,
           T* __restrict__ Gam, size_t js, uint32_t vsel)
{
    const int v = blockIdx.z;                       // endpoint: its slice of W, its K outputs
    if (!(vsel >> v & 1u)) return;
    W = job_ptr(W, js) + ((size_t)endpoint_slot(vsel, v) << (n - 1 - b)) * nlow;
    Gam = job_ptr(Gam, js) + (size_t)v * K;
    using L = LogOps<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int h = n - 1 - b;
    const int hh = h - hc;
    const uint32_t col = blockIdx.x;
    // low pattern g of this column
    int kg = 0;
    uint32_t r = col;
    while (r >= binom(b, kg)) { r -= binom(b, kg); ++kg; }
    const uint32_t g = colex_unrank(r, kg, b);
    const int dp = d - kg;
    const uint32_t nout = num_small_subsets(h, dp);
    const uint32_t chunkN = 1u << hc;
    T* vals = reinterpret_cast<T*>(smem_raw);
    T* acc = vals + chunkN;
    uint32_t* gh = reinterpret_cast<uint32_t*>(acc + nout);
    for (uint32_t o = threadIdx.x; o < nout; o += blockDim.x) {
        uint32_t ro = o;
        int k = 0;
        while (ro >= binom(h, k)) { ro -= binom(h, k); ++k; }
        gh[o] = colex_unrank(ro, k, h);
        acc[o] = L::ninf();
    }
    const uint32_t lowc = chunkN - 1u;
    for (uint32_t Hhi = 0; Hhi < (1u << hh); ++Hhi) {
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < chunkN; t += blockDim.x)
            vals[t] = W[BN_AT((size_t)((Hhi << hc) | t) * nlow + col, 1, ((size_t)nlow << h))];
        __syncthreads();
        for (int j = 0; j < hc; ++j) {
            const uint32_t jm = (1u << j) - 1u;
            for (uint32_t p = threadIdx.x; p < (chunkN >> 1); p += blockDim.x) {
                const uint32_t lo = ((p & ~jm) << 1) | (p & jm);
                if (__popc(lo & jm) <= dp) vals[lo] = L::lse(vals[lo], vals[lo | (1u << j)]);
            }
            __syncthreads();
        }
        for (uint32_t o = threadIdx.x; o < nout; o += blockDim.x) {
            const uint32_t G = gh[o];
            if (((G >> hc) & ~Hhi) == 0u) acc[o] = L::lse(acc[o], vals[G & lowc]);
        }
    }
    __syncthreads();
    for (uint32_t o = threadIdx.x; o < nout; o += blockDim.x) {
        const uint32_t cm = g | (gh[o] << b);      // mask over the n-1 bits of V-{v}
        const int k = __popc(cm);
        uint32_t f = 0;
        for (int s = 0; s < k; ++s) f += binom(n - 1, s);
        int t = 1;
        for (uint32_t x = cm; x; x &= x - 1, ++t) f += binom(__ffs(x) - 1, t);
        Gam[BN_AT(f, 1, K)] = acc[o];
    }
}

// Family index of the mask cm over the n-1 bits of V - {v}: by size, then
// colexicographic rank (the canonical order of the scores).
__device__ __forceinline__ uint32_t family_index(uint32_t cm, int n)
{
    const int k = __popc(cm);
    uint32_t f = 0;
    for (int s = 0; s < k; ++s) f += binom(n - 1, s);
    int t = 1;
    for (uint32_t x = cm; x; x &= x - 1, ++t) f += binom(__ffs(x) - 1, t);
    return f;
}

// Lazy log-sum-exp step (one exponential per term): (m, s) is m + log(s).
template <typename T>
__device__ __forceinline__ void lse_lazy_k(T& m, T& s, T x)
{
    using L = LogOps<T>;
    const T dd = x - m;                             // +inf while empty
    const bool big = dd > T(64);
    const T e = L::ex(big ? -dd : dd);
    s = big ? s * e + T(1) : s + e;
    m = big ? x : m;
}

// Warp-wide log-sum of the lanes' (m, s), in a fixed tree order.
template <typename T>
__device__ __forceinline__ T warp_lse(T m, T s)
{
    using L = LogOps<T>;
    for (int o = 16; o; o >>= 1) {
        const T m2 = __shfl_xor_sync(FULL, m, o);
        const T s2 = __shfl_xor_sync(FULL, s, o);
        const T mn = m2 > m ? m2 : m;
        if (mn != L::ninf()) {
            s = s * L::ex(m - mn) + s2 * L::ex(m2 - mn);
            m = mn;
        }
    }
    return m + L::lg(s);
}

// Phase 2 for the columns whose low pattern g has at least d - 1 elements
// (d' = d - |g| <= 1, at most one high element left): the outputs are
// Gamma(g) = log-sum of W[H][g] over every H and, for d' = 1, Gamma(g + {b})
// = log-sum over the H that contain b, for every high bit b -- the truncated
// transform over the high dimensions, written out.  One warp per column,
// eight consecutive columns per block (they share the sectors of W's rows).
// Lane l takes the rows H = l + 32k: high bits 0-4 are its lane bits, the
// bits from 5 up are summed per lane.
template <typename T>
__global__ void __launch_bounds__(256)
k_gamma_p2s(int n, int d, int b, uint32_t nlow, uint32_t c0, int64_t K, const T* __restrict__ W,
            T* __restrict__ Gam, size_t js, uint32_t vsel)
{
    constexpr int MB = 14;                          // high bits from 5 up (h <= 18, n <= 32)
    const int v = blockIdx.z;
    if (!(vsel >> v & 1u)) return;
    W = job_ptr(W, js) + ((size_t)endpoint_slot(vsel, v) << (n - 1 - b)) * nlow;
    Gam = job_ptr(Gam, js) + (size_t)v * K;
    using L = LogOps<T>;
    const int h = n - 1 - b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t col = c0 + blockIdx.x * 8 + warp;
    if (col >= nlow) return;                        // whole warps leave
    int kg = 0;
    uint32_t r = col;
    while (r >= binom(b, kg)) { r -= binom(b, kg); ++kg; }
    const uint32_t g = colex_unrank(r, kg, b);
    const bool one = d - kg == 1;
    T m0 = L::ninf(), s0 = T(0);
    T mb[MB], sb[MB];
#pragma unroll
    for (int q = 0; q < MB; ++q) { mb[q] = L::ninf(); sb[q] = T(0); }
    const uint32_t nH = 1u << h;
    const size_t wsize = (size_t)nlow << h;
    // the rows two and three steps ahead are in flight while a row is added
    // (the loop waits on load latency, each lane reading its own row; four
    // rows ahead cost registers: 61 against 48, one block per SM fewer)
    T wa = lane < nH ? W[BN_AT((size_t)lane * nlow + col, 1, wsize)] : T(0);
    T wb = lane + 32 < nH ? W[BN_AT((size_t)(lane + 32) * nlow + col, 1, wsize)] : T(0);
    for (uint32_t H = lane; H < nH; H += 32) {
        const T w = wa;
        wa = wb;
        if (H + 64 < nH) wb = W[BN_AT((size_t)(H + 64) * nlow + col, 1, wsize)];
        lse_lazy_k(m0, s0, w);
        if (one) {
#pragma unroll
            for (int q = 0; q < MB; ++q)
                if (5 + q < h && (H >> (5 + q) & 1u)) lse_lazy_k(mb[q], sb[q], w);
        }
    }
    const T all = warp_lse(m0, s0);
    if (lane == 0) Gam[BN_AT(family_index(g, n), 1, K)] = all;
    if (!one) return;
    for (int bb = 0; bb < h && bb < 5; ++bb) {
        const bool in = lane >> bb & 1;
        const T x = warp_lse(in ? m0 : L::ninf(), in ? s0 : T(0));
        if (lane == 0) Gam[BN_AT(family_index(g | (1u << (b + bb)), n), 1, K)] = x;
    }
#pragma unroll
    for (int q = 0; q < MB; ++q) {
        if (5 + q >= h) break;
        const T x = warp_lse(mb[q], sb[q]);
        if (lane == 0) Gam[BN_AT(family_index(g | (1u << (b + 5 + q)), n), 1, K)] = x;
    }
}

// ===========================================================================
// Step 5: P(u->v, D) = sum_{G: u in G} B_v(G) Gamma_v(G)  (Eq. 11) and
// P(u->v | D) = P(u->v, D) / P(D), in FP64, in three launches.
// Every term B_v(G) Gamma_v(G) is at most their sum over G, which is F(V)
// (Eq. 11 summed over all G), so e(G) = B_v(G) Gamma_v(G) / F(V) <= 1 (up to
// rounding) needs no maximum pass.  Blocks over (families of v, v) add e(G)
// in fixed point (2^qbits, integer atomics: the sums do not depend on the
// order of arrival) into acc[v*n + u] for every u in G and into acc[n*n + v]
// for all G.  The FP64 path divides by F(V) (Algorithm 1), i.e. takes
// acc[v*n + u] / 2^qbits; the FP32 path divides by Z_v = acc[n*n + v]
// (the same quantity from the same Gamma_v, so rounding common to numerator
// and denominator cancels).  log P(D) = F~(V) + sum_i c_i.
// ===========================================================================
__global__ void k_edges_zero(int n, unsigned long long* __restrict__ acc, size_t js)
{
    acc = job_ptr(acc, js);
    for (int t = threadIdx.x; t < n * (n + 1); t += blockDim.x) acc[t] = 0ull;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_edges_acc(int n, int64_t K, int qbits, const double* __restrict__ logB,
            const double* __restrict__ cmax, const uint32_t* __restrict__ masks,
            const T* __restrict__ Gam, const T* __restrict__ F,
            unsigned long long* __restrict__ acc, size_t js, uint32_t vsel)
{
    if (!(vsel >> blockIdx.z & 1u)) return;         // an endpoint another rank computes
    logB = job_ptr(logB, js);
    cmax = job_ptr(cmax, js);
    masks = job_ptr(masks, js);
    Gam = job_ptr(Gam, js);
    F = job_ptr(F, js);
    acc = job_ptr(acc, js);
    using L = LogOps<T>;
    __shared__ unsigned long long Nu[32], Nz;
    const int v = blockIdx.z;
    const int tid = threadIdx.x;
    if (tid < 32) Nu[tid] = 0ull;
    if (tid == 0) Nz = 0ull;
    __syncthreads();
    const uint32_t full = (uint32_t)(((uint64_t)1 << n) - 1);   // n <= 32
    // FP32: Gamma is relative to the integer Z = floor of log P(D) in the
    // level-based units (see gamma_offsets), so P(D) enters as F(V) - Z
    const double fv = (double)F[full];
    const double lnFV = L::to_ln(sizeof(T) == 4 ? fv - floor(fv) : fv);
    const double qscale = ldexp(1.0, qbits);
    const double cv = cmax[v];
    unsigned long long z = 0ull;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + tid; f < K;
         f += (int64_t)gridDim.x * blockDim.x) {
        const size_t x = (size_t)v * K + f;
        const double e = exp(logB[x] - cv + L::to_ln((double)Gam[x]) - lnFV);
        const unsigned long long q = __double2ull_rn(e * qscale);
        z += q;
        for (uint32_t g = masks[x]; g; g &= g - 1) atomicAdd(&Nu[BN_AT(__ffs(g) - 1, 1, 32)], q);
    }
    for (int o = 16; o; o >>= 1) z += __shfl_xor_sync(FULL, z, o);
    if ((tid & 31) == 0) atomicAdd(&Nz, z);
    __syncthreads();
    if (tid < n && Nu[tid]) atomicAdd(&acc[(size_t)v * n + tid], Nu[tid]);
    if (tid == 0) atomicAdd(&acc[(size_t)n * n + v], Nz);
}

template <typename T>
__global__ void k_edges_fin(int n, int use_z, int qbits, const double* __restrict__ cmax,
                            const T* __restrict__ F, const int* __restrict__ err,
                            const unsigned long long* __restrict__ acc,
                            double* __restrict__ post, double* __restrict__ log_PD, size_t js,
                            uint32_t vsel)
{
    cmax = job_ptr(cmax, js);
    F = job_ptr(F, js);
    err = job_ptr(err, js);
    acc = job_ptr(acc, js);
    post = job_ptr(post, js);
    log_PD = job_ptr(log_PD, js);
    const bool bad = err && *err;
    const double qscale = ldexp(1.0, qbits);
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int u = t / n, v = t % n;
        const unsigned long long num = acc[(size_t)v * n + u];
        double p = 0.0;
        if (u != v && num > 0ull)
            p = use_z ? __ull2double_rn(num) / __ull2double_rn(acc[(size_t)n * n + v])
                      : __ull2double_rn(num) / qscale;
        post[t] = bad ? NAN : (vsel >> v & 1u) ? p : 0.0;   // other ranks' endpoints: 0
    }
    if (threadIdx.x == 0 && log_PD) {
        double c = 0.0;
        for (int i = 0; i < n; ++i) c += cmax[i];
        double fv = (double)F[((size_t)1 << n) - 1];
        if (sizeof(T) == 4)                       // FP32: add the level base of F(V)
            fv += level_base_fwd(level_words(reinterpret_cast<const float*>(F), n), n - kLevelShift);
        *log_PD = bad ? NAN : LogOps<T>::to_ln(fv) + c;
    }
}

// ===========================================================================
// Priors beyond the defaults and single features (Eqs. 4-9).
// ===========================================================================

// log B_i(G) += log w_i(G): a per-family weight (a general rho_i(G), Eq. 4).
__global__ void k_add_weights(double* __restrict__ logB, const double* __restrict__ w, int64_t nK)
{
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nK;
         x += (int64_t)gridDim.x * blockDim.x)
        logB[x] += w[x];
}

// A_i(S) += log q_i(S), q_i a function of |S| (Eq. 7): lq[i * n + |S|] in
// the working precision and log base; A is [i * 2^(n-1) + c], c = S with
// bit i removed, so |S| = popc(c).
template <typename T>
__global__ void k_apply_q(int n, const T* __restrict__ lq, T* __restrict__ A, int tlo)
{
    const int64_t total = (int64_t)n << (n - 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t >> (n - 1));
        const uint32_t c = (uint32_t)(t & (((int64_t)1 << (n - 1)) - 1));
        int size = __popc(c);
        if (tlo) {
            // in tile-level order the in-tile row part of c is a place p:
            // its size is the number of row sizes whose places end at or
            // before p (places of size k start at sum_{q<k} C(rb, q))
            const int lw = i < 4 ? 3 : 4, rb = 13 - lw;
            const uint32_t p = (c >> lw) & ((1u << rb) - 1u);
            int k = 0;
            for (uint32_t end = 1; end <= p; end += binom(rb, k)) ++k;
            size = __popc(c >> 13) + k + __popc(c & ((1u << lw) - 1u));
        }
        A[t] += lq[i * n + size];
    }
}

// out = lbs + lf: the shifted scores of B_i(G) f_i(G) (Eq. 6 with a feature).
template <typename T>
__global__ void k_add_feature(const T* __restrict__ lbs, const T* __restrict__ lf,
                              T* __restrict__ out, int64_t nK)
{
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nK;
         x += (int64_t)gridDim.x * blockDim.x)
        out[x] = lbs[x] + lf[x];
}

// Byte copies between scattered device regions, one block per segment: the
// batch upload (a staging buffer to every job's data) and download (every
// job's results to a staging buffer).
__global__ void k_copy_segments(const CopySeg* __restrict__ segs, int nseg)
{
    for (int q = blockIdx.x; q < nseg; q += gridDim.x) {
        const CopySeg sg = segs[q];
        for (uint64_t i = threadIdx.x; i < sg.bytes; i += blockDim.x) sg.dst[i] = sg.src[i];
    }
}

// ===========================================================================
// Launchers.
// ===========================================================================
// exp_t / log_t (bn_device.cuh) beside CUDA's exp / log, for the test of
// the table-driven functions: out[4i..4i+3] = exp_t, exp, log_t, log of x[i].
__global__ void k_explog_check(const double* __restrict__ x, int64_t count, double* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        out[4 * i] = exp_t(v);
        out[4 * i + 1] = exp(v);
        out[4 * i + 2] = log_t(v);
        out[4 * i + 3] = log(v);
    }
}

#ifndef BN_MEGA  // host launchers (bn_mega.cu includes only the device code)
#ifdef BN_CHECK_BOUNDS
BN_BOUNDS_READER(bounds_line_kernels)
#endif
static int grid_for(int64_t work, int threads, int cap = 152 * 32)
{
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

cudaError_t launch_pack_planes(const uint8_t* data, int n, int m, int rmax, int W,
                               uint64_t* planes, cudaStream_t s, const int* mj, int nj, size_t js)
{
    const int64_t total = (int64_t)n * rmax * W;
    launch_or_record(KID_PACK_PLANES, k_pack_planes, dim3(grid_for(total, 256), nj), 256, 0, s, data, n, m, rmax, W, planes, mj,
                                                                 js);
    return cudaGetLastError();
}

cudaError_t launch_check_data(const uint8_t* data, const uint8_t* arity, int n, int m,
                              int* err, cudaStream_t s)
{
    if ((int64_t)n * m == 0) return cudaSuccess;
    launch_or_record(KID_CHECK_DATA, k_check_data, grid_for((int64_t)n * m, 256), 256, 0, s, data, arity, n, m, err);
    return cudaGetLastError();
}

int fixed_shift(int m, double ess, const double* Dvals, int rows)
{
    double L = std::log1p((double)m);
    for (int r = 0; r < rows; ++r) {
        const double a = ess / Dvals[r];
        L = std::max(L, std::max(std::fabs(std::log(a)), std::log(a + (double)m)));
    }
    const double B = 2.0 * (double)m * L + 1.0;
    const int S = 61 - (int)std::ceil(std::log2(B));
    return std::min(52, std::max(8, S));
}

cudaError_t launch_lgamma_table(const double* alpha, int rows, int m, int fxs, void* T,
                                cudaStream_t s, int nj, size_t js, const double* fxj,
                                const int* mj)
{
    const int64_t total = (int64_t)rows * (m + 1);
    launch_or_record(KID_LGAMMA_TABLE, k_lgamma_table, dim3(grid_for(total, 256), nj), 256, 0, s, 
        alpha, rows, m, (long long*)T, js, std::ldexp(1.0, fxs), fxj, mj);
    return cudaGetLastError();
}

static uint32_t host_binom(int n, int k);

// Binary data, d <= 8: k_scores_bin for the families of at most 4 parents
// and one launch per larger family size: k_scores_bin_hi (per-cell popc)
// below kHistFrom parents, k_scores_bin_hist (per-sample histogram) from
// there.  The range is all families or a single one.
static constexpr int kHistFrom = 7;
static cudaError_t launch_scores_bin(const Plan& P, const uint64_t* planes, const double* Dvals,
                                     const void* Tv, const double* log_rho, int64_t x_begin,
                                     int64_t x_count, uint32_t* masks, uint32_t* cmasks,
                                     double* logB, int64_t* debug_counts, cudaStream_t s,
                                     const double* fxj)
{
    const long long* T = static_cast<const long long*>(Tv);
    const double tinv = std::ldexp(1.0, -P.fxs);
    int64_t off[10] = {0};
    for (int k = 0; k <= P.d; ++k) off[k + 1] = off[k] + host_binom(P.n - 1, k);
    const int dl = P.d < 4 ? P.d : 4;
    const int64_t Kc = off[dl + 1];
    int k1 = 0, klo = 0, khi = P.d;                 // single family: its size only
    int64_t i1 = 0, f1 = 0;
    if (x_count == 1) {
        i1 = x_begin / P.K;
        f1 = x_begin % P.K;
        while (f1 >= off[k1 + 1]) ++k1;
        klo = khi = k1;
    }
    if (klo <= 4) {
        const int64_t xb = x_count == 1 ? i1 * Kc + f1 : 0;
        const int64_t xn = x_count == 1 ? 1 : (int64_t)P.n * Kc;
        const unsigned tbb = rec_block(128);
        launch_or_record(KID_SCORES_BIN, k_scores_bin, dim3((unsigned)((xn + tbb - 1) / tbb), P.nj), tbb, 0, s, 
            P.n, P.m, P.W, P.K, Kc, planes, Dvals, P.rows, T, log_rho, xb, xn, masks, cmasks, logB,
            debug_counts, P.js, tinv, fxj);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int k = klo > 5 ? klo : 5; k <= khi; ++k) {
        const int64_t Ck = host_binom(P.n - 1, k);
        const int64_t fb = x_count == 1 ? i1 * Ck + (f1 - off[k]) : 0;
        const int64_t fn = x_count == 1 ? 1 : (int64_t)P.n * Ck;
        if (k >= kHistFrom) {                       // histogram of the samples' cells
            const unsigned grid = (unsigned)std::min<int64_t>((fn + 7) / 8, 152 * 32);
#define BN_BIN_HIST(KP)                                                                           \
    launch_or_record((int)KID_SCORES_BIN_HIST5 + (KP) - 5, k_scores_bin_hist<KP>, dim3(grid, P.nj), 256, 0, s,                                     \
        P.n, P.m, P.W, P.K, off[k], Ck, planes, Dvals, P.rows, T, log_rho, fb, fn, masks, cmasks, \
        logB, debug_counts, P.js, tinv, fxj)
            switch (k) {
            case 5: BN_BIN_HIST(5); break;
            case 6: BN_BIN_HIST(6); break;
            case 7: BN_BIN_HIST(7); break;
            default: BN_BIN_HIST(8); break;
            }
#undef BN_BIN_HIST
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            continue;
        }
        const int64_t threads = fn << (k - 4);
        const unsigned tbh = rec_block(128);
        const unsigned grid = (unsigned)((threads + tbh - 1) / tbh);
#define BN_BIN_HI(HB)                                                                             \
    launch_or_record((int)KID_SCORES_BIN_HI1 + (HB) - 1, k_scores_bin_hi<HB>, dim3(grid, P.nj), tbh, 0, s,                                       \
        P.n, P.m, P.W, P.K, off[k], Ck, planes, Dvals, P.rows, T, log_rho, fb, fn, masks, cmasks, \
        logB, debug_counts, P.js, tinv, fxj)
        switch (k) {
        case 5: BN_BIN_HI(1); break;
        case 6: BN_BIN_HI(2); break;
        case 7: BN_BIN_HI(3); break;
        default: BN_BIN_HI(4); break;
        }
#undef BN_BIN_HI
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool scores_cfg_fits(const Plan& P)
{
    return !P.allbin && P.d <= SC_MP && P.rmax <= SC_MR;
}

int scores_launches(const Plan& P)
{
    return P.allbin && P.d > 4 && P.d <= 8 ? P.d - 3 : 1;
}

cudaError_t launch_scores(const Plan& P, const uint8_t* arity, const uint64_t* planes,
                          const double* Dvals, const void* Tv, const double* log_rho,
                          int64_t x_begin, int64_t x_count, uint32_t* masks, uint32_t* cmasks,
                          double* logB, int64_t* debug_counts, cudaStream_t s,
                          const double* fxj)
{
    const long long* T = static_cast<const long long*>(Tv);
    const double tinv = std::ldexp(1.0, -P.fxs);
    const int threads = 256;
    const int64_t warps_wanted = x_count;
    int grid = grid_for(warps_wanted * 32, threads, 152 * 64);
    if (P.allbin && P.d <= 8 && (x_count == 1 || (x_begin == 0 && x_count == (int64_t)P.n * P.K)))
        return launch_scores_bin(P, planes, Dvals, Tv, log_rho, x_begin, x_count, masks, cmasks,
                                 logB, debug_counts, s, fxj);
    if (P.scfg && scores_cfg_fits(P) && P.d <= 4 && P.rmax <= 4)
        launch_or_record(KID_SCORES_CFG44, k_scores_cfg<4, 4>, dim3(grid, P.nj), threads, 0, s, 
            P.n, P.m, P.W, P.rmax, P.K, arity, planes, Dvals, P.rows, T, log_rho, x_begin, x_count,
            masks, cmasks, logB, debug_counts, P.js, tinv, fxj);
    else if (P.scfg && scores_cfg_fits(P))
        launch_or_record(KID_SCORES_CFG, k_scores_cfg<SC_MP, SC_MR>, dim3(grid, P.nj), threads, 0, s, 
            P.n, P.m, P.W, P.rmax, P.K, arity, planes, Dvals, P.rows, T, log_rho, x_begin, x_count,
            masks, cmasks, logB, debug_counts, P.js, tinv, fxj);
    else if (P.W <= 32 && P.d <= 4 && P.rmax <= 2)
        launch_or_record(KID_SCORES_W42, k_scores_w<4, 2>, dim3(grid, P.nj), threads, 0, s, P.n, P.m, P.W, P.rmax, P.K, arity, planes, Dvals,
                                                  P.rows, T, log_rho, x_begin, x_count, masks,
                                                  cmasks, logB, debug_counts, P.js, tinv, fxj);
    else if (P.W <= 32 && P.d <= 4 && P.rmax <= 4)
        launch_or_record(KID_SCORES_W44, k_scores_w<4, 4>, dim3(grid, P.nj), threads, 0, s, P.n, P.m, P.W, P.rmax, P.K, arity, planes, Dvals,
                                                  P.rows, T, log_rho, x_begin, x_count, masks,
                                                  cmasks, logB, debug_counts, P.js, tinv, fxj);
    else if (P.W <= 32 && P.d <= 8 && P.rmax <= 4)
        launch_or_record(KID_SCORES_W84, k_scores_w<8, 4>, dim3(grid, P.nj), threads, 0, s, P.n, P.m, P.W, P.rmax, P.K, arity, planes, Dvals,
                                                  P.rows, T, log_rho, x_begin, x_count, masks,
                                                  cmasks, logB, debug_counts, P.js, tinv, fxj);
    else if (P.d <= SC_MP && P.rmax <= SC_MR)
        launch_or_record(KID_SCORES_CFG, k_scores_cfg<SC_MP, SC_MR>, dim3(grid, P.nj), threads, 0, s, P.n, P.m, P.W, P.rmax, P.K, arity, planes, Dvals,
                                              P.rows, T, log_rho, x_begin, x_count, masks,
                                              cmasks, logB, debug_counts, P.js, tinv, fxj);
    else
        launch_or_record(KID_SCORES, k_scores, dim3(grid, P.nj), threads, 0, s, P.n, P.d, P.m, P.W, P.rmax, P.K, arity, planes, Dvals,
                                          P.rows, T, log_rho, x_begin, x_count, masks, cmasks,
                                          logB, debug_counts, P.js, tinv, fxj);
    return cudaGetLastError();
}

cudaError_t launch_add_weights(const Plan& P, double* logB, const double* w, cudaStream_t s)
{
    const int64_t nK = (int64_t)P.n * P.K;
    launch_or_record(KID_ADD_WEIGHTS, k_add_weights, grid_for(nK, 256), 256, 0, s, logB, w, nK);
    return cudaGetLastError();
}

cudaError_t launch_apply_q(const Plan& P, const void* lq, void* A, cudaStream_t s)
{
    const int64_t total = (int64_t)P.n << (P.n - 1);
    const int grid = grid_for(total, 256, 152 * 16);
    if (P.prec == 0)
        launch_or_record(KID_APPLY_Q_D, k_apply_q<double>, grid, 256, 0, s, P.n, (const double*)lq, (double*)A, 0);
    else
        launch_or_record(KID_APPLY_Q_F, k_apply_q<float>, grid, 256, 0, s, P.n, (const float*)lq, (float*)A,
                                              use_tlo(P) ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_add_feature(const Plan& P, const void* lbs, const void* lf, void* out,
                               cudaStream_t s)
{
    const int64_t nK = (int64_t)P.n * P.K;
    if (P.prec == 0)
        launch_or_record(KID_ADD_FEATURE_D, k_add_feature<double>, grid_for(nK, 256), 256, 0, s, 
            (const double*)lbs, (const double*)lf, (double*)out, nK);
    else
        launch_or_record(KID_ADD_FEATURE_F, k_add_feature<float>, grid_for(nK, 256), 256, 0, s, 
            (const float*)lbs, (const float*)lf, (float*)out, nK);
    return cudaGetLastError();
}

cudaError_t launch_node_max(const Plan& P, const double* logB, double* cmax, cudaStream_t s)
{
    launch_or_record(KID_NODE_MAX, k_node_max, dim3(P.n, P.nj), 256, 0, s, P.K, logB, cmax, P.js);
    return cudaGetLastError();
}

cudaError_t launch_shift_scores(const Plan& P, const double* logB, const double* cmax, void* lbs,
                                cudaStream_t s)
{
    const int64_t total = (int64_t)P.n * P.K;
    const dim3 grid(grid_for(total, 256), P.nj);
    if (P.prec == 0)
        launch_or_record(KID_SHIFT_D, k_shift_scores<double>, grid, 256, 0, s, total, P.K, logB, cmax, (double*)lbs, P.js);
    else
        launch_or_record(KID_SHIFT_F, k_shift_scores<float>, grid, 256, 0, s, total, P.K, logB, cmax, (float*)lbs, P.js);
    return cudaGetLastError();
}

size_t upzeta_smem_bytes(const Plan& P)
{
    const size_t es = P.prec == 0 ? 8 : 4;
    return ((size_t)1 << P.b_up) * (8 + 2 * es);
}

// Fractional bits of a fixed-point sum of at most `terms` values in (0, 1].
static int fixed_bits(int64_t terms)
{
    int b = 0;
    while (((int64_t)1 << b) <= terms) ++b;
    return 63 - b;
}

cudaError_t launch_upzeta(const Plan& P, const uint32_t* cmasks, const void* lbs, void* tab,
                          const uint16_t* rk13, void* A, cudaStream_t s, cudaEvent_t sums_done, int* err)
{
    if (use_tile13_up(P)) {
        cudaError_t e = launch_reorder_up(P, lbs, tab, s);
        if (e != cudaSuccess) return e;
        return launch_upzeta13(P, tab, rk13 + 8192, A, s, sums_done, err);
    }
    const int h = P.n - 1 - P.b_up;
    const dim3 grid((unsigned)P.n << h, P.nj);
    const size_t sm = upzeta_smem_bytes(P);
    if (P.prec == 0)
        launch_or_record(KID_UPZETA_D, k_upzeta<double>, grid, 256, sm, s, P.n, P.b_up, P.K, fixed_bits(P.K), cmasks,
                                               (const double*)lbs, (double*)A, P.js);
    else
        launch_or_record(KID_UPZETA_F, k_upzeta<float>, grid, 256, sm, s, P.n, P.b_up, P.K, fixed_bits(P.K), cmasks,
                                              (const float*)lbs, (float*)A, P.js);
    return cudaGetLastError();
}

static uint32_t host_binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int t = 1; t <= k; ++t) r = r * (uint64_t)(n - k + t) / (uint64_t)t;
    return (uint32_t)r;
}

// Tiles per warp: enough warps to fill the GPU a few times over, at most 8.
static int tiles_per_warp(uint32_t ntiles)
{
    int tpw = 1;
    while (tpw < 8 && (uint64_t)ntiles >= (uint64_t)tpw * 2 * 152 * 64 * 4) tpw *= 2;
    return tpw;
}

cudaError_t launch_forward(const Plan& P, const void* A, void* F, cudaStream_t s, int* launches)
{
    if (use_rows_levels(P) || rows64_fit(P)) return launch_forward_rows(P, A, F, s, launches);
    const int nh = P.n - P.wb;
    for (int hl = 0; hl <= nh; ++hl) {
        const uint32_t nt = host_binom(nh, hl);
        const int tpw = tiles_per_warp(nt);
        const uint32_t warps = (nt + tpw - 1) / tpw;
        const dim3 grid((unsigned)(((uint64_t)warps * 32 + 255) / 256), P.nj);
        if (P.prec == 0)
            launch_or_record(KID_FWD_LEVEL_D, k_forward_level<double>, grid, 256, 0, s, P.n, P.wb, hl, nt, tpw, (const double*)A,
                                                         (double*)F, P.js);
        else
            launch_or_record(KID_FWD_LEVEL_F, k_forward_level<float>, grid, 256, 0, s, P.n, P.wb, hl, nt, tpw, (const float*)A,
                                                        (float*)F, P.js);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

cudaError_t launch_backward(const Plan& P, const void* A, void* Rc, cudaStream_t s, int* launches)
{
    if (use_rows_levels(P) || rows64_fit(P)) return launch_backward_rows(P, A, Rc, s, launches);
    const int nh = P.n - P.wb;
    for (int hl = nh; hl >= 0; --hl) {
        const uint32_t nt = host_binom(nh, hl);
        const int tpw = tiles_per_warp(nt);
        const uint32_t warps = (nt + tpw - 1) / tpw;
        const dim3 grid((unsigned)(((uint64_t)warps * 32 + 255) / 256), P.nj);
        if (P.prec == 0)
            launch_or_record(KID_BWD_LEVEL_D, k_backward_level<double>, grid, 256, 0, s, P.n, P.wb, hl, nt, tpw,
                                                          (const double*)A, (double*)Rc, P.js);
        else
            launch_or_record(KID_BWD_LEVEL_F, k_backward_level<float>, grid, 256, 0, s, P.n, P.wb, hl, nt, tpw, (const float*)A,
                                                         (float*)Rc, P.js);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

size_t gamma_p1_smem_bytes(const Plan& P)
{
    return ((size_t)1 << P.b_g) * (P.prec == 0 ? 8 : 4);
}

size_t gamma_p2_smem_bytes(const Plan& P)
{
    const int h = P.n - 1 - P.b_g;
    uint64_t nout = 0;
    for (int k = 0; k <= P.d && k <= h; ++k) nout += host_binom(h, k);
    const size_t es = P.prec == 0 ? 8 : 4;
    return ((size_t)1 << P.hc_g) * es + nout * es + nout * 4 + 16;
}

cudaError_t launch_gamma_table(const Plan& P, const void* F, const void* Rc, cudaStream_t s)
{
    launch_or_record(KID_GAMMA_TABLE, k_gamma_table, dim3(P.n, P.nj), 32, 0, s, P.n, (const float*)F, (float*)const_cast<void*>(Rc),
                                                 P.js, P.vsel);
    return cudaGetLastError();
}

cudaError_t launch_gamma_p1(const Plan& P, const void* F, const void* Rc, const uint16_t* rk13,
                            void* W, cudaStream_t s, const void* lq, const void* A)
{
    if (use_tile13_gamma(P)) return launch_gamma13_p1(P, F, Rc, rk13, W, s, lq, A);
    if (P.prec != 0) {
        const cudaError_t e = launch_gamma_table(P, F, Rc, s);
        if (e != cudaSuccess) return e;
    }
    const int h = P.n - 1 - P.b_g;
    const size_t sm1 = gamma_p1_smem_bytes(P);
    const dim3 grid(1u << h, P.nj, P.n);
    if (P.prec == 0)
        launch_or_record(KID_GAMMA_P1_D, k_gamma_p1<double>, grid, 256, sm1, s, P.n, P.d, P.b_g, P.nlow_g,
                                                  (const double*)F, (const double*)Rc,
                                                  (double*)W, P.js, (const double*)lq, P.vsel);
    else
        launch_or_record(KID_GAMMA_P1_F, k_gamma_p1<float>, grid, 256, sm1, s, P.n, P.d, P.b_g, P.nlow_g,
                                                 (const float*)F, (const float*)Rc,
                                                 (float*)W, P.js, (const float*)lq, P.vsel);
    return cudaGetLastError();
}

// Phase 2's columns: those before c0 (at least two high elements left) go to
// the block butterfly kernel, the others (at least d - 1 low elements) to
// the warp kernel.
uint32_t gamma_p2_split(const Plan& P)
{
    const int h = P.n - 1 - P.b_g;
    uint32_t c0 = 0;
    for (int k = 0; k <= P.d - 2 && k <= P.b_g; ++k) c0 += host_binom(P.b_g, k);
    if (h > 18) c0 = P.nlow_g;                      // beyond the warp kernel's bit count
    return c0;
}

int gamma_launches(const Plan& P)
{
    const uint32_t c0 = gamma_p2_split(P);
    return 1 + (P.prec != 0 ? 1 : 0) + (c0 > 0 ? 1 : 0) + (c0 < P.nlow_g ? 1 : 0);
}

cudaError_t launch_gamma_p2(const Plan& P, const void* W, void* Gam, cudaStream_t s)
{
    const uint32_t c0 = gamma_p2_split(P);
    if (c0 > 0) {
        const size_t sm2 = gamma_p2_smem_bytes(P);
        const dim3 grid(c0, P.nj, P.n);
        if (P.prec == 0)
            launch_or_record(KID_GAMMA_P2_D, k_gamma_p2<double>, grid, 256, sm2, s, P.n, P.d, P.b_g, P.hc_g, P.nlow_g, P.K,
                                                      (const double*)W, (double*)Gam, P.js, P.vsel);
        else
            launch_or_record(KID_GAMMA_P2_F, k_gamma_p2<float>, grid, 256, sm2, s, P.n, P.d, P.b_g, P.hc_g, P.nlow_g, P.K,
                                                     (const float*)W, (float*)Gam, P.js, P.vsel);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (c0 < P.nlow_g) {
        const dim3 grid((P.nlow_g - c0 + 7) / 8, P.nj, P.n);
        if (P.prec == 0)
            launch_or_record(KID_GAMMA_P2S_D, k_gamma_p2s<double>, grid, 256, 0, s, P.n, P.d, P.b_g, P.nlow_g, c0, P.K,
                                                     (const double*)W, (double*)Gam, P.js, P.vsel);
        else
            launch_or_record(KID_GAMMA_P2S_F, k_gamma_p2s<float>, grid, 256, 0, s, P.n, P.d, P.b_g, P.nlow_g, c0, P.K,
                                                    (const float*)W, (float*)Gam, P.js, P.vsel);
    }
    return cudaGetLastError();
}

cudaError_t launch_edges(const Plan& P, const double* logB, const double* cmax,
                         const uint32_t* masks, const void* Gam, const void* F, const int* err,
                         unsigned long long* acc, double* post, double* log_PD, cudaStream_t s)
{
    launch_or_record(KID_EDGES_ZERO, k_edges_zero, dim3(1, P.nj), 256, 0, s, P.n, acc, P.js);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned chunks = (unsigned)std::min<int64_t>((P.K + 1023) / 1024, 64);
    const dim3 grid(chunks, P.nj, P.n);
    if (P.prec == 0)
        launch_or_record(KID_EDGES_ACC_D, k_edges_acc<double>, grid, 256, 0, s, P.n, P.K, fixed_bits(P.K), logB, cmax, masks,
                                                 (const double*)Gam, (const double*)F, acc, P.js, P.vsel);
    else
        launch_or_record(KID_EDGES_ACC_F, k_edges_acc<float>, grid, 256, 0, s, P.n, P.K, fixed_bits(P.K), logB, cmax, masks,
                                                (const float*)Gam, (const float*)F, acc, P.js, P.vsel);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (P.prec == 0)
        launch_or_record(KID_EDGES_FIN_D, k_edges_fin<double>, dim3(1, P.nj), rec_block(1024), 0, s, P.n, 0, fixed_bits(P.K), cmax,
                                                           (const double*)F, err, acc, post,
                                                           log_PD, P.js, P.vsel);
    else
        launch_or_record(KID_EDGES_FIN_F, k_edges_fin<float>, dim3(1, P.nj), rec_block(1024), 0, s, P.n, 1, fixed_bits(P.K), cmax,
                                                          (const float*)F, err, acc, post,
                                                          log_PD, P.js, P.vsel);
    return cudaGetLastError();
}

cudaError_t launch_explog_check(const double* x, int64_t count, double* out, cudaStream_t s)
{
    if (count < 1) return cudaSuccess;
    k_explog_check<<<(unsigned)std::min<int64_t>((count + 255) / 256, 152 * 8), 256, 0, s>>>(x, count, out);
    return cudaGetLastError();
}

cudaError_t launch_copy_segments(const CopySeg* segs, int nseg, cudaStream_t s)
{
    if (nseg < 1) return cudaSuccess;
    return launch_or_record(KID_NONE, k_copy_segments, dim3((unsigned)std::min(nseg, 152 * 8)), 256,
                            0, s, segs, nseg);
}

cudaError_t set_kernel_attributes()
{
    cudaError_t e;
#define SETA(k)                      \
    e = allow_max_dynamic_smem(k); \
    if (e != cudaSuccess) return e;
    SETA(k_upzeta<double>)
    SETA(k_upzeta<float>)
    SETA(k_gamma_p1<double>)
    SETA(k_gamma_p1<float>)
    SETA(k_gamma_p2<double>)
    SETA(k_gamma_p2<float>)
#undef SETA
    return set_tile13_attributes();
}

#endif  // BN_MEGA

}  // namespace bn

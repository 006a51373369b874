// bn_noalloc.cu -- bn_edge_posteriors_static: the edge-posterior pipeline
// with every intermediate array in one fixed device array, for callers that
// must not allocate device memory.
//
// Who needs it: code embedded in a host application that owns and partitions
// all GPU memory itself (a game engine, a database, a runtime with its own
// device allocator), where a library may not take memory behind the
// application's back; and latency-sensitive loops that cannot afford
// cudaMalloc / cudaFree (cudaFree synchronises the whole device).
//
// The scratch is the file-scope array below (BN_STATIC_SCRATCH_BYTES).  Every
// GPU that loads this library holds it until the process exits.  All calls
// on one device share it and it keeps the previous call's contents; the only
// value that must start at zero (the input-check flag) is cleared by every
// call.  Two calls whose work overlaps on the GPU (different streams, no
// ordering between them) race on the array and give undefined results.
//
// No cudaMalloc, cudaMallocAsync, cudaMallocHost, cudaFree or other
// allocating routine is called, and no host heap memory is used: the small
// host tables live on the stack and are copied with cudaMemcpyAsync from
// pageable memory.  For a pageable source the runtime has consumed the host
// bytes when cudaMemcpyAsync returns, so the stack frame may end right after.
// Besides the size of the array, two fixed host tables bound a job: at most
// kMaxStates distinct (product of arities, number of parents) pairs and
// kMaxRows distinct lgamma-table denominators (both 1024; only jobs with many
// distinct arities come near them).  Either limit gives BN_ENOMEM, like the
// size limit, before any GPU work.
#include "bnedge.h"
#include "bn_device.cuh"
#include "bn_kernels.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

static __device__ __align__(256) unsigned char g_bn_static_scratch[BN_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxStates = 1024;  // distinct (product, count) pairs of arities
constexpr int kMaxRows = 1024;    // distinct lgamma-table denominators

std::mutex g_setup_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array on device `dev` (the current device).
// The host-side name g_bn_static_scratch is only a stand-in; its device
// address is looked up once per device, with that device current.
int scratch_for_device(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return BN_EINVAL;
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bn_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return BN_ECUDA;
        }
        if (bn::set_kernel_attributes() != cudaSuccess) return BN_ECUDA;
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return BN_OK;
}

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

int64_t binom64(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
    return r;
}

// Sorted distinct values of q (a product of at most d arities, q*r <= 65536
// cells) and of q*r for every arity r, in fixed arrays.  Returns the count or
// -1 when a fixed limit is exceeded.
int denominators(const uint8_t* arity, int n, int d, double* D)
{
    uint32_t prod[kMaxStates];
    uint8_t cnt[kMaxStates];
    int ns = 1;
    prod[0] = 1;
    cnt[0] = 0;
    for (int v = 0; v < n; ++v) {
        const uint32_t r = arity[v];
        const int cur = ns;
        for (int k = 0; k < cur; ++k) {
            if (cnt[k] >= d || (uint64_t)prod[k] * r > 65536u) continue;
            const uint32_t p = prod[k] * r;
            const uint8_t c = (uint8_t)(cnt[k] + 1);
            bool seen = false;
            for (int t = 0; t < ns && !seen; ++t) seen = prod[t] == p && cnt[t] == c;
            if (seen) continue;
            if (ns == kMaxStates) return -1;
            prod[ns] = p;
            cnt[ns] = c;
            ++ns;
        }
    }
    int nd = 0;
    auto insert = [&](double x) {
        int pos = 0;
        while (pos < nd && D[pos] < x) ++pos;
        if (pos < nd && D[pos] == x) return true;
        if (nd == kMaxRows) return false;
        for (int t = nd; t > pos; --t) D[t] = D[t - 1];
        D[pos] = x;
        ++nd;
        return true;
    };
    for (int k = 0; k < ns; ++k) {
        if (!insert((double)prod[k])) return -1;
        for (int v = 0; v < n; ++v)
            if ((uint64_t)prod[k] * arity[v] <= 65536u && !insert((double)prod[k] * arity[v]))
                return -1;
    }
    return nd;
}

// No C++ exception leaves the library (a lock can throw): BN_EINVAL.
int exception_code() noexcept
{
    try {
        throw;
    } catch (const std::bad_alloc&) {
        return BN_ENOMEM;
    } catch (...) {
        return BN_EINVAL;
    }
}

}  // namespace

extern "C" int bn_edge_posteriors_static(const bn_job_desc* j, double* post_dev,
                                         double* log_PD_dev, void* stream)
try {
    if (!j || !post_dev) return BN_EINVAL;
    if (j->n < 1 || j->n > 31 || j->d < 0 || j->m < 0 || !j->arity) return BN_EINVAL;
    if (j->m > 0 && !j->data) return BN_EINVAL;
    if (!(j->ess > 0.0) || !std::isfinite(j->ess)) return BN_EINVAL;
    if (j->precision != BN_FP64 && j->precision != BN_FP32_SHIFTED) return BN_EINVAL;
    bn::Plan P{};
    P.n = j->n;
    P.d = j->d < j->n - 1 ? j->d : j->n - 1;
    P.m = j->m;
    P.prec = j->precision == BN_FP64 ? 0 : 1;
    uint8_t arity[32];
    std::memcpy(arity, j->arity, P.n);
    uint32_t sorted[32];
    for (int v = 0; v < P.n; ++v) {
        if (arity[v] < 1) return BN_EINVAL;
        sorted[v] = arity[v];
    }
    for (int a = 1; a < P.n; ++a)                      // descending insertion sort
        for (int b = a; b > 0 && sorted[b] > sorted[b - 1]; --b) {
            const uint32_t t = sorted[b]; sorted[b] = sorted[b - 1]; sorted[b - 1] = t;
        }
    uint64_t cells = 1;
    for (int t = 0; t <= P.d && t < P.n; ++t) cells *= sorted[t];
    if (cells > 65536u) return BN_EINVAL;
    double log_rho[32] = {};
    if (j->log_q || j->log_w) return BN_EINVAL;        // not in this entry point
    if (j->log_rho)
        for (int k = 0; k <= P.d; ++k) {
            log_rho[k] = j->log_rho[k];
            if (!std::isfinite(log_rho[k])) return BN_EINVAL;
        }
    if (!j->data_on_device && P.m > 0 && !bn::data_below_arity(j->data, P.m, P.n, arity))
        return BN_EINVAL;
    P.K = 0;
    for (int k = 0; k <= P.d; ++k) P.K += binom64(P.n - 1, k);
    P.W = P.m > 0 ? (P.m + 63) / 64 : 1;
    P.rmax = (int)sorted[0];
    P.allbin = sorted[0] == 2 && sorted[P.n - 1] == 2;
    double tables[2 * kMaxRows];                        // Dvals | alpha
    const int rows = denominators(arity, P.n, P.d, tables);
    if (rows < 0) return BN_ENOMEM;
    P.rows = rows;
    for (int r = 0; r < rows; ++r) tables[rows + r] = j->ess / tables[r];
    P.fxs = bn::fixed_shift(P.m, j->ess, tables, rows);
    P.b_up = P.n - 1 < 12 ? P.n - 1 : 12;
    P.b_g = P.n - 1 < 13 ? P.n - 1 : 13;
    const int hg = P.n - 1 - P.b_g;
    P.hc_g = hg < 12 ? hg : 12;
    uint64_t nl = 0;
    for (int k = 0; k <= P.d && k <= P.b_g; ++k) nl += (uint64_t)binom64(P.b_g, k);
    P.nlow_g = (uint32_t)nl;
    P.wb = P.n < 5 ? P.n : 5;
    bn::default_schedule(P);

    // layout inside the static array
    const size_t es = P.prec == 0 ? 8 : 4;
    const size_t nK = (size_t)P.n * P.K;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += al(bytes > 0 ? bytes : 1); return at; };
    const size_t o_data = take((size_t)P.m * P.n), o_ar = take(P.n),
                 o_lr = take((size_t)(P.d + 1) * 8), o_tab = take((size_t)2 * rows * 8),
                 o_lgT = take((size_t)rows * (P.m + 1) * 8),
                 o_pl = take((size_t)P.n * P.rmax * P.W * 8), o_err = take(4),
                 o_masks = take(nK * 4), o_cm = take(nK * 4), o_logB = take(nK * 8),
                 o_cmax = take((size_t)P.n * 8), o_lbs = take(nK * es),
                 o_reo = take(bn::use_tile13_up(P) ? nK * es : 0),
                 o_rk = take(bn::needs_rank13(P) ? bn::kRank13Bytes : 0),
                 o_A = take(((size_t)P.n << (P.n - 1)) * es),
                 o_F = take(((size_t)1 << P.n) * es + bn::kLevelWords * 4),
                 o_Rc = take(((size_t)1 << P.n) * es + (bn::kLevelWords + bn::kGammaTabWords) * 4),
                 o_W = take((size_t)P.n * ((size_t)1 << hg) * P.nlow_g * es), o_G = take(nK * es),
                 o_ea = take((size_t)P.n * (P.n + 1) * 8);
    if (o > (size_t)BN_STATIC_SCRATCH_BYTES) return BN_ENOMEM;   // job too large

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BN_ECUDA;
    unsigned char* base = nullptr;
    int rc = scratch_for_device(dev, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
#define CKS(call) do { if ((call) != cudaSuccess) return BN_ECUDA; } while (0)
    const uint8_t* data_dev = base + o_data;
    if (P.m > 0) {
        if (j->data_on_device) data_dev = j->data;
        else CKS(cudaMemcpyAsync(base + o_data, j->data, (size_t)P.m * P.n, cudaMemcpyHostToDevice, s));
    }
    CKS(cudaMemcpyAsync(base + o_ar, arity, P.n, cudaMemcpyHostToDevice, s));
    CKS(cudaMemcpyAsync(base + o_lr, log_rho, (size_t)(P.d + 1) * 8, cudaMemcpyHostToDevice, s));
    CKS(cudaMemcpyAsync(base + o_tab, tables, (size_t)2 * rows * 8, cudaMemcpyHostToDevice, s));
    CKS(cudaMemsetAsync(base + o_err, 0, 4, s));        // the one value that must start at 0
    int* err = reinterpret_cast<int*>(base + o_err);
    const uint8_t* ar = base + o_ar;
    const double* Dvals = reinterpret_cast<const double*>(base + o_tab);
    const double* alpha = Dvals + rows;
    void* lgT = base + o_lgT;                          // int64 fixed-point lgamma table
    uint64_t* planes = reinterpret_cast<uint64_t*>(base + o_pl);
    uint32_t* masks = reinterpret_cast<uint32_t*>(base + o_masks);
    uint32_t* cm = reinterpret_cast<uint32_t*>(base + o_cm);
    double* logB = reinterpret_cast<double*>(base + o_logB);
    double* cmax = reinterpret_cast<double*>(base + o_cmax);
    if (j->data_on_device) CKS(bn::launch_check_data(data_dev, ar, P.n, P.m, err, s));
    CKS(bn::launch_pack_planes(data_dev, P.n, P.m, P.rmax, P.W, planes, s));
    CKS(bn::launch_lgamma_table(alpha, P.rows, P.m, P.fxs, lgT, s));
    CKS(bn::launch_scores(P, ar, planes, Dvals, lgT,
                          j->log_rho ? reinterpret_cast<const double*>(base + o_lr) : nullptr, 0,
                          (int64_t)P.n * P.K, masks, cm, logB, nullptr, s));
    CKS(bn::launch_node_max(P, logB, cmax, s));
    CKS(bn::launch_shift_scores(P, logB, cmax, base + o_lbs, s));
    uint16_t* rk13 = reinterpret_cast<uint16_t*>(base + o_rk);
    if (bn::needs_rank13(P)) CKS(bn::launch_rank13_tables(P, rk13, rk13 + 8192, s));
    CKS(bn::launch_upzeta(P, cm, base + o_lbs, base + o_reo, rk13, base + o_A, s));
    CKS(bn::launch_forward(P, base + o_A, base + o_F, s, nullptr));
    CKS(bn::launch_backward(P, base + o_A, base + o_Rc, s, nullptr));
    CKS(bn::launch_gamma_p1(P, base + o_F, base + o_Rc, rk13, base + o_W, s, nullptr, base + o_A));
    CKS(bn::launch_gamma_p2(P, base + o_W, base + o_G, s));
    CKS(bn::launch_edges(P, logB, cmax, masks, base + o_G, base + o_F, err,
                         reinterpret_cast<unsigned long long*>(base + o_ea), post_dev,
                         log_PD_dev, s));
#undef CKS
    return BN_OK;
} catch (...) {
    return exception_code();
}

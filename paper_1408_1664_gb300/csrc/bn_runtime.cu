// bn_runtime.cu -- host runtime behind the C ABI of include/bnedge.h:
// validation, job planning, the device workspace, the launch sequence of
// Algorithm 1, and the serving queue (bn_submit / bn_poll / bn_wait).
#include "bnedge.h"
#include "bn_device.cuh"
#include "bn_kernels.cuh"

#include <algorithm>
#include <new>
#include <stdexcept>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <array>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

namespace bn {
// The launch recorder of the calling host thread (see launch_or_record).
thread_local Recorder* g_recorder = nullptr;
}  // namespace bn

namespace {

using bn::Plan;

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

int64_t host_binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
    return r;
}

int64_t families(int n, int d)
{
    if (n < 1 || d < 0) return 0;
    d = std::min(d, n - 1);
    int64_t k = 0;
    for (int s = 0; s <= d; ++s) k += host_binom(n - 1, s);
    return k;
}

// Host copy of one job's inputs plus its plan.
struct HostJob {
    Plan P{};
    double ess = 1.0;
    std::vector<uint8_t> arity;
    std::vector<double> log_rho;     // d+1 entries, empty = none
    std::vector<double> log_q;       // n*n: log q_i(S) by |S| (Eq. 4), empty = none
    std::vector<double> log_w;       // n*K: per-family log weights, empty = none
    std::vector<double> Dvals;       // sorted distinct denominators q, q*r
    const uint8_t* data = nullptr;   // host or device
    bool data_on_device = false;
    std::vector<uint8_t> data_copy;  // owned host copy (served jobs)
};

// Byte offsets of every array of a job inside one device allocation.
struct Layout {
    size_t data, mj, fx, arity, log_rho, Dvals, alpha, lgT, planes, err, masks, cmasks, logB,
        cmax, lbs, tab, rk13, A, F, Rc, W, Gam, eacc, post, logPD, logq, logw, logf, lbsf, dbg,
        total;
};

Layout make_layout(const Plan& P, size_t dbg_cells, bool feature = false)
{
    const size_t es = P.prec == 0 ? 8 : 4;
    const size_t nK = (size_t)P.n * P.K;
    const int hg = P.n - 1 - P.b_g;
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o += al(std::max<size_t>(bytes, 1)); return at; };
    L.data = take((size_t)P.m * P.n);
    L.mj = take(4);                  // the job's own m (batch groups pad m)
    L.fx = take(16);                 // the job's lgamma-table scale 2^S and 2^-S (batches)
    L.arity = take(P.n);
    L.log_rho = take((size_t)(P.d + 1) * 8);
    L.Dvals = take((size_t)P.rows * 8);
    L.alpha = take((size_t)P.rows * 8);
    L.lgT = take((size_t)P.rows * (P.m + 1) * 8);
    L.planes = take((size_t)P.n * P.rmax * P.W * 8);
    L.err = take(4);
    L.masks = take(nK * 4);
    L.cmasks = take(nK * 4);
    L.logB = take(nK * 8);
    L.cmax = take((size_t)P.n * 8);
    L.lbs = take(nK * es);
    // sized for every schedule that fits, so that a plan can switch kernels
    L.tab = take(bn::tile13_up_fits(P) ? nK * es : 0);
    L.rk13 = take(bn::tile13_gamma_fits(P) ? bn::kRank13Bytes : 0);
    // a split job with divided A holds its own slabs; a spilled job's A is a
    // managed allocation of its own
    L.A = take((P.slab || P.spill) ? 0 : ((size_t)P.n << (P.n - 1)) * es);
    // F and R' are each followed by the per-level words of the FP32 bases
    L.F = take(((size_t)1 << P.n) * es + bn::kLevelWords * 4);
    L.Rc = take(((size_t)1 << P.n) * es + (bn::kLevelWords + bn::kGammaTabWords) * 4);
    // one slice per endpoint computed (all n, or a split job's rank's)
    const size_t nv = P.vgroup ? (size_t)P.vgroup
                               : (size_t)__builtin_popcount(P.vsel & (uint32_t)(((uint64_t)1 << P.n) - 1));
    L.W = take(nv * ((size_t)1 << hg) * P.nlow_g * es);
    L.Gam = take(nK * es);
    L.eacc = take((size_t)P.n * (P.n + 1) * 8);
    L.post = take((size_t)P.n * P.n * 8);
    L.logPD = take(8);
    L.logq = take(P.hasq ? (size_t)P.n * P.n * es : 0);
    L.logw = take(P.hasw ? nK * 8 : 0);
    L.logf = take(feature ? nK * es : 0);         // a single feature (bn_feature_posterior)
    L.lbsf = take(feature ? nK * es : 0);
    L.dbg = take(dbg_cells * 8);
    L.total = o;
    return L;
}

// Distinct values of q = prod of at most d arities (capped at 65536 cells) and
// of q * r for every arity r: the rows of the lgamma table.
std::vector<double> denominators(const std::vector<uint8_t>& arity, int d)
{
    std::set<std::pair<uint32_t, int>> st{{1u, 0}};
    for (uint8_t r : arity) {
        std::vector<std::pair<uint32_t, int>> add;
        for (auto& pc : st)
            if (pc.second < d && (uint64_t)pc.first * r <= 65536u) add.push_back({pc.first * r, pc.second + 1});
        for (auto& a : add) st.insert(a);
        if (st.size() > 200000) break;
    }
    std::set<uint32_t> qs;
    for (auto& pc : st) qs.insert(pc.first);
    std::set<uint32_t> rs(arity.begin(), arity.end());
    std::set<double> D;
    for (uint32_t q : qs) {
        D.insert((double)q);
        for (uint32_t r : rs)
            if ((uint64_t)q * r <= 65536u) D.insert((double)q * r);
    }
    return std::vector<double>(D.begin(), D.end());
}

// A log weight of zero (-inf) becomes this finite value: every sum and
// maximum stays finite, its exponential (and that of any sum it enters) is
// exactly 0, and tiles that span it take the exact scaled path.  It is small
// enough in magnitude for that path's per-element scales: integers in FP32
// (log2 units, 1.44e7), 600-nat bands in FP64 (spacing 2e-9 at 1e7).  NaN
// and +inf are rejected.
constexpr double kLogZero = -1e7;

int log_weights(const double* src, size_t count, std::vector<double>& dst)
{
    dst.assign(src, src + count);
    for (double& x : dst) {
        if (std::isnan(x) || x == INFINITY) return BN_EINVAL;
        if (x < kLogZero) x = kLogZero;
    }
    return BN_OK;
}

// In the working precision and log base (FP32: base 2).
std::vector<char> working_logs(const std::vector<double>& v, int prec)
{
    std::vector<char> out(v.size() * (prec == 0 ? 8 : 4));
    if (prec == 0) {
        std::memcpy(out.data(), v.data(), out.size());
    } else {
        float* f = reinterpret_cast<float*>(out.data());
        for (size_t t = 0; t < v.size(); ++t) f[t] = (float)(v[t] * 1.4426950408889634);
    }
    return out;
}

int validate_and_plan(const bn_job_desc* j, HostJob& hj)
{
    if (!j) return BN_EINVAL;
    if (j->n < 1 || j->n > 32 || j->d < 0 || j->m < 0 || !j->arity) return BN_EINVAL;
    if (j->m > 0 && !j->data) return BN_EINVAL;
    if (!(j->ess > 0.0) || !std::isfinite(j->ess)) return BN_EINVAL;
    if (j->precision != BN_FP64 && j->precision != BN_FP32_SHIFTED) return BN_EINVAL;
    Plan& P = hj.P;
    P.n = j->n;
    P.d = std::min(j->d, j->n - 1);
    P.m = j->m;
    P.prec = j->precision == BN_FP64 ? 0 : 1;
    hj.arity.assign(j->arity, j->arity + P.n);
    for (uint8_t r : hj.arity)
        if (r < 1) return BN_EINVAL;
    // largest family: the d+1 largest arities
    std::vector<uint32_t> sorted(hj.arity.begin(), hj.arity.end());
    std::sort(sorted.rbegin(), sorted.rend());
    uint64_t cells = 1;
    for (int t = 0; t <= P.d && t < P.n; ++t) cells *= sorted[t];
    if (cells > 65536u) return BN_EINVAL;
    if (j->log_rho) {
        hj.log_rho.assign(j->log_rho, j->log_rho + (j->d + 1));
        hj.log_rho.resize(P.d + 1);
        for (double x : hj.log_rho)
            if (!std::isfinite(x)) return BN_EINVAL;
    }
    hj.ess = j->ess;
    hj.data = j->data;
    hj.data_on_device = j->data_on_device != 0;
    if (!hj.data_on_device && P.m > 0 && !bn::data_below_arity(j->data, P.m, P.n, hj.arity.data()))
        return BN_EINVAL;
    P.K = families(P.n, P.d);
    if (j->log_q) {
        if (log_weights(j->log_q, (size_t)P.n * P.n, hj.log_q)) return BN_EINVAL;
        P.hasq = 1;
    }
    if (j->log_w) {
        if (log_weights(j->log_w, (size_t)P.n * P.K, hj.log_w)) return BN_EINVAL;
        P.hasw = 1;
    }
    P.W = std::max(1, (P.m + 63) / 64);
    P.rmax = (int)sorted[0];
    P.allbin = sorted[0] == 2 && sorted[P.n - 1] == 2;
    hj.Dvals = denominators(hj.arity, P.d);
    if (hj.Dvals.size() > 16384) return BN_EINVAL;
    P.rows = (int)hj.Dvals.size();
    P.fxs = bn::fixed_shift(P.m, j->ess, hj.Dvals.data(), P.rows);
    P.b_up = std::min(P.n - 1, 12);
    P.b_g = std::min(P.n - 1, 13);
    const int hg = P.n - 1 - P.b_g;
    P.hc_g = std::min(hg, 12);
    uint64_t nl = 0;
    for (int k = 0; k <= P.d && k <= P.b_g; ++k) nl += host_binom(P.b_g, k);
    P.nlow_g = (uint32_t)nl;
    P.wb = std::min(P.n, 5);
    bn::default_schedule(P);
    return BN_OK;
}

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return BN_ECUDA;       \
    } while (0)

// Event set of one job: [0] start, [1] scores, [2] up-zeta, [3] F, [4] F and
// R' both done, [5] Gamma phase 1, [6] Gamma phase 2, [7] edges, [8] the
// column sums of step 2 (13-dimension tiles only), [9] R' done.
constexpr int kEvents = 10;
constexpr int kEvEdges = 7, kEvSums = 8, kEvR = 9;

// A second stream for the steps that may run beside the main one: F and R'
// depend only on A, so R' runs on the side stream between a fork and a join.
struct Side {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int create()
    {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess)
            return BN_ECUDA;
        return BN_OK;
    }
    void destroy()
    {
        if (s) cudaStreamDestroy(s);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        s = nullptr;
        fork = join = nullptr;
    }
};
struct Events {
    cudaEvent_t ev[kEvents] = {};
    bool ok = false;
    Plan P{};
    int launches = 0;
    bool overlap = false;        // R' ran beside F
    int create()
    {
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return BN_ECUDA;
        ok = true;
        return BN_OK;
    }
    void destroy()
    {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        ok = false;
    }
    cudaEvent_t last() const { return ev[kEvEdges]; }
};

struct Bufs {
    char* base = nullptr;
    Layout L{};
    char* A_ext = nullptr;           // A outside the layout (a job whose A is spilled)
    template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(base + off); }
    void* A() const { return A_ext ? (void*)A_ext : (void*)(base + L.A); }
};

int enqueue_kernels(const HostJob& hj, const Bufs& B, const uint8_t* data_dev, double* post_dev,
                    double* logPD_dev, cudaStream_t s, Events* ev, int* launches,
                    const Side* side = nullptr);

// The order prior q (working precision) and the family weights (FP64) of a
// job, when given.  Pageable copies: the host vectors may go right after.
int upload_priors(const HostJob& hj, const Bufs& B, cudaStream_t s)
{
    const Plan& P = hj.P;
    if (P.hasq) {
        const std::vector<char> q = working_logs(hj.log_q, P.prec);
        CK(cudaMemcpyAsync(B.at<char>(B.L.logq), q.data(), q.size(), cudaMemcpyHostToDevice, s));
    }
    if (P.hasw)
        CK(cudaMemcpyAsync(B.at<char>(B.L.logw), hj.log_w.data(), hj.log_w.size() * 8,
                           cudaMemcpyHostToDevice, s));
    return BN_OK;
}

// Enqueue steps 1-5 on stream s.  Small host arrays go through `stage`
// (pinned, >= stage_bytes) when given, else through pageable copies.
int enqueue(const HostJob& hj, const Bufs& B, double* post_dev, double* logPD_dev,
            cudaStream_t s, Events* ev, int* launches, char* stage, size_t stage_bytes,
            bool upload_tables = true, const Side* side = nullptr)
{
    const Plan& P = hj.P;
    const Layout& L = B.L;
    if (ev) CK(cudaEventRecord(ev->ev[0], s));
    // inputs
    const uint8_t* data_dev = B.at<uint8_t>(L.data);
    if (P.m > 0) {
        if (hj.data_on_device) {
            data_dev = hj.data;
        } else {
            CK(cudaMemcpyAsync(B.at<uint8_t>(L.data), hj.data, (size_t)P.m * P.n,
                               cudaMemcpyHostToDevice, s));
        }
    }
    // small tables: arity | log_rho | Dvals | alpha
    std::vector<char> small;
    const size_t n_ar = al(P.n), n_lr = al((size_t)(P.d + 1) * 8), n_dv = al((size_t)P.rows * 8);
    small.resize(n_ar + n_lr + 2 * n_dv);
    std::memcpy(small.data(), hj.arity.data(), P.n);
    std::vector<double> lr(P.d + 1, 0.0);
    for (size_t t = 0; t < hj.log_rho.size(); ++t) lr[t] = hj.log_rho[t];
    std::memcpy(small.data() + n_ar, lr.data(), lr.size() * 8);
    std::memcpy(small.data() + n_ar + n_lr, hj.Dvals.data(), hj.Dvals.size() * 8);
    std::vector<double> alpha(P.rows);
    for (int r = 0; r < P.rows; ++r) alpha[r] = hj.ess / hj.Dvals[r];
    std::memcpy(small.data() + n_ar + n_lr + n_dv, alpha.data(), alpha.size() * 8);
    const char* src = small.data();
    if (upload_tables && stage && stage_bytes >= small.size()) {
        std::memcpy(stage, small.data(), small.size());
        src = stage;
    }
    if (upload_tables) {
        CK(cudaMemcpyAsync(B.at<char>(L.arity), src, n_ar, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(B.at<char>(L.log_rho), src + n_ar, n_lr, cudaMemcpyHostToDevice, s));
        // L.alpha directly follows L.Dvals (both rows*8 rounded to 256)
        CK(cudaMemcpyAsync(B.at<char>(L.Dvals), src + n_ar + n_lr, 2 * n_dv,
                           cudaMemcpyHostToDevice, s));
    }
    const int rc = upload_priors(hj, B, s);
    if (rc) return rc;
    return enqueue_kernels(hj, B, data_dev, post_dev, logPD_dev, s, ev, launches, side);
}

// Step 1 on stream s (inputs on the device): scores, the family weights,
// the per-node maximum and the shifted scores; the rank tables of the
// 13-dimension tiles.
int enqueue_step1(const HostJob& hj, const Bufs& B, const uint8_t* data_dev, cudaStream_t s,
                  int* nl)
{
    const Plan& P = hj.P;
    const Layout& L = B.L;
    CK(cudaMemsetAsync(B.at<int>(L.err), 0, 4, s));
    int* err = B.at<int>(L.err);
    const uint8_t* ar = B.at<uint8_t>(L.arity);
    if (hj.data_on_device) { CK(bn::launch_check_data(data_dev, ar, P.n, P.m, err, s)); ++*nl; }
    CK(bn::launch_pack_planes(data_dev, P.n, P.m, P.rmax, P.W, B.at<uint64_t>(L.planes), s)); ++*nl;
    CK(bn::launch_lgamma_table(B.at<double>(L.alpha), P.rows, P.m, P.fxs, B.at<void>(L.lgT), s)); ++*nl;
    CK(bn::launch_scores(P, ar, B.at<uint64_t>(L.planes), B.at<double>(L.Dvals),
                         B.at<void>(L.lgT), hj.log_rho.empty() ? nullptr : B.at<double>(L.log_rho),
                         0, (int64_t)P.n * P.K, B.at<uint32_t>(L.masks), B.at<uint32_t>(L.cmasks),
                         B.at<double>(L.logB), nullptr, s));
    *nl += bn::scores_launches(P);
    if (P.hasw) { CK(bn::launch_add_weights(P, B.at<double>(L.logB), B.at<double>(L.logw), s)); ++*nl; }
    CK(bn::launch_node_max(P, B.at<double>(L.logB), B.at<double>(L.cmax), s)); ++*nl;
    CK(bn::launch_shift_scores(P, B.at<double>(L.logB), B.at<double>(L.cmax), B.at<void>(L.lbs), s)); ++*nl;
    if (bn::needs_rank13(P)) {
        uint16_t* rk = B.at<uint16_t>(L.rk13);
        CK(bn::launch_rank13_tables(P, rk, rk + 8192, s));
        ++*nl;
    }
    return BN_OK;
}

// Step 2 from the shifted scores lbs into A, then the order prior q.
int enqueue_upzeta(const Plan& P, const Bufs& B, const void* lbs, cudaStream_t s, int* nl,
                   cudaEvent_t sums_done)
{
    const Layout& L = B.L;
    CK(bn::launch_upzeta(P, B.at<uint32_t>(L.cmasks), lbs, B.at<void>(L.tab),
                         B.at<uint16_t>(L.rk13), B.A(), s, sums_done, B.at<int>(L.err)));
    *nl += bn::use_tile13_up(P) ? 3 : 1;
    if (P.hasq) { CK(bn::launch_apply_q(P, B.at<void>(L.logq), B.A(), s)); ++*nl; }
    return BN_OK;
}

// Enqueue the kernels of steps 1-5 on stream s (inputs already on the device).
int enqueue_kernels(const HostJob& hj, const Bufs& B, const uint8_t* data_dev, double* post_dev,
                    double* logPD_dev, cudaStream_t s, Events* ev, int* launches, const Side* side)
{
    const Plan& P = hj.P;
    const Layout& L = B.L;
    int nl = 0;
    int rc = enqueue_step1(hj, B, data_dev, s, &nl);
    if (rc) return rc;
    if (ev) CK(cudaEventRecord(ev->ev[1], s));
    rc = enqueue_upzeta(P, B, B.at<void>(L.lbs), s, &nl,
                        ev && bn::use_tile13_up(P) ? ev->ev[kEvSums] : nullptr);
    if (rc) return rc;
    int* err = B.at<int>(L.err);
    if (ev) CK(cudaEventRecord(ev->ev[2], s));
    if (side && side->s) {
        CK(cudaEventRecord(side->fork, s));
        CK(cudaStreamWaitEvent(side->s, side->fork, 0));
        CK(bn::launch_backward(P, B.A(), B.at<void>(L.Rc), side->s, &nl));
        if (ev) CK(cudaEventRecord(ev->ev[kEvR], side->s));
        CK(cudaEventRecord(side->join, side->s));
        CK(bn::launch_forward(P, B.A(), B.at<void>(L.F), s, &nl));
        if (ev) CK(cudaEventRecord(ev->ev[3], s));
        CK(cudaStreamWaitEvent(s, side->join, 0));
    } else {
        CK(bn::launch_forward(P, B.A(), B.at<void>(L.F), s, &nl));
        if (ev) CK(cudaEventRecord(ev->ev[3], s));
        CK(bn::launch_backward(P, B.A(), B.at<void>(L.Rc), s, &nl));
        if (ev) CK(cudaEventRecord(ev->ev[kEvR], s));
    }
    if (ev) {
        CK(cudaEventRecord(ev->ev[4], s));
        ev->overlap = side && side->s;
    }
    if (P.vgroup) {
        // step 4 a group of endpoints at a time through one group's W (the
        // phase timings then cover all groups: phase 1 ends with the last)
        for (int v0 = 0; v0 < P.n; v0 += P.vgroup) {
            Plan Q = P;
            Q.vsel = 0;
            for (int v = v0; v < std::min(P.n, v0 + P.vgroup); ++v) Q.vsel |= 1u << v;
            CK(bn::launch_gamma_p1(Q, B.at<void>(L.F), B.at<void>(L.Rc), B.at<uint16_t>(L.rk13),
                                   B.at<void>(L.W), s, P.hasq ? B.at<void>(L.logq) : nullptr, B.A()));
            if (ev && v0 + P.vgroup >= P.n) CK(cudaEventRecord(ev->ev[5], s));
            CK(bn::launch_gamma_p2(Q, B.at<void>(L.W), B.at<void>(L.Gam), s));
            nl += bn::gamma_launches(Q);
        }
        if (ev) CK(cudaEventRecord(ev->ev[6], s));
    } else {
        CK(bn::launch_gamma_p1(P, B.at<void>(L.F), B.at<void>(L.Rc), B.at<uint16_t>(L.rk13),
                               B.at<void>(L.W), s, P.hasq ? B.at<void>(L.logq) : nullptr, B.A()));
        if (ev) CK(cudaEventRecord(ev->ev[5], s));
        CK(bn::launch_gamma_p2(P, B.at<void>(L.W), B.at<void>(L.Gam), s));
        if (ev) CK(cudaEventRecord(ev->ev[6], s));
        nl += bn::gamma_launches(P);
    }
    CK(bn::launch_edges(P, B.at<double>(L.logB), B.at<double>(L.cmax), B.at<uint32_t>(L.masks),
                        B.at<void>(L.Gam), B.at<void>(L.F), err,
                        B.at<unsigned long long>(L.eacc), post_dev, logPD_dev, s));
    nl += 3;
    if (ev) CK(cudaEventRecord(ev->ev[kEvEdges], s));
    if (launches) *launches = nl;
    if (ev) {
        ev->P = P;
        ev->launches = nl;
    }
    return BN_OK;
}


double alg_bytes(const Plan& P)
{
    const double es = P.prec == 0 ? 8.0 : 4.0;
    const double N = std::ldexp(1.0, P.n);
    // A written once and read by F and by R'; F and R' written and read once;
    // the halves of F and R' read for every endpoint v.
    return es * (1.5 * P.n * N + 4.0 * N + P.n * N);
}

void fill_stats(const Plan& P, Events& ev, int launches, bn_stats* st)
{
    std::memset(st, 0, sizeof(*st));
    auto el = [&](int a, int b) {
        float t = 0;
        cudaEventElapsedTime(&t, ev.ev[a], ev.ev[b]);
        return (double)t;
    };
    st->ms_scores = el(0, 1);
    st->ms_upzeta = el(1, 2);
    st->ms_upzeta_sums = bn::use_tile13_up(P) ? el(1, kEvSums) : 0.0;
    st->ms_forward = el(2, 3);
    st->ms_backward = ev.overlap ? el(2, kEvR) : el(3, kEvR);   // beside F: from the same start
    st->ms_gamma_p1 = el(4, 5);
    st->ms_gamma_p2 = el(5, 6);
    st->ms_edges = el(6, kEvEdges);
    st->ms_total = el(0, kEvEdges);
    st->cells = (double)P.n * std::ldexp(1.0, P.n);
    st->alg_bytes = alg_bytes(P);
    st->kernels = launches;
    st->precision = P.prec == 0 ? BN_FP64 : BN_FP32_SHIFTED;
}

enum JobState { Q_QUEUED, Q_RUNNING, Q_DONE };

struct Slot {
    cudaStream_t stream = nullptr;
    Side side;                   // R' beside F
    Events ev;
    cudaEvent_t done = nullptr;  // after the result copies
    char* dev = nullptr;         // allocation of the running job (stream-ordered)
    size_t bytes = 0;
    char* pin = nullptr;         // pinned host: outputs + small-table staging
    size_t pin_bytes = 0;
    uint64_t job = 0;            // 0 = free
    int launches = 0;
};

struct ServedJob {
    HostJob hj;
    int state = Q_QUEUED;
    int rc = BN_OK;
    int slot = -1;
    size_t bytes = 0;
    std::vector<double> post;
    double logPD = 0;
    bn_stats stats{};
};

}  // namespace

struct bn_ctx {
    int device = 0;
    uint64_t budget = 0;
    int fail_after = -1;
    int allocs = 0;
    cudaStream_t stream = nullptr;
    Side side;                   // R' beside F on the direct path
    // direct path workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    // a spilled job's A: managed memory, its first spill_dev bytes preferred
    // in device memory, the rest in host memory mapped for the GPU
    char* spill = nullptr;
    size_t spill_bytes = 0, spill_dev = 0;
    char* pin = nullptr;
    size_t pin_bytes = 0;
    static constexpr int kRing = 32;
    Events ring[kRing];
    int ring_pos = 0;            // next set to use
    int ring_count = 0;
    Plan last{};
    Layout last_layout{};
    bool have_last = false;
    int last_launches = 0;
    bn_stats last_stats{};
    std::vector<char> tables_sig;   // inputs of the small tables now in ws
    // serving
    std::mutex mu;
    std::vector<Slot> slots;
    std::map<uint64_t, ServedJob> jobs;
    std::deque<uint64_t> queue;
    uint64_t next_id = 1;
    uint64_t reserved = 0;
    // batches
    int flags = 0;
    // (n, d, prec, binary, jobs) -> schedule (scfg, up13, frows, frc, g13)
    std::map<std::array<int, 5>, std::array<int, 5>> tuned;
};

// Jobs of a batch with equal n, d and precision: their arrays lie js bytes
// apart from base on (each job in the same padded layout), and the launches
// of steps 2-5 cover all of them.
struct BatchGroup {
    Plan P{};                  // n, d, K, precision, schedule; nj and js
    Layout L{};                // the padded layout of one job
    size_t base = 0;           // arena offset of the group's first job
    std::vector<int> members;  // indices into bn_batch::jobs
    bool timed = false;        // schedule chosen by timing (else default or cached)
};

struct bn_batch {
    bn_ctx* ctx = nullptr;
    std::vector<HostJob> jobs;
    std::vector<int> group_of, slot_of;
    std::vector<BatchGroup> groups;
    char* arena = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<Side> sides;                 // R' beside F, one per branch
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last = nullptr;
    bool ran = false;
    float ms_default = 0.0f, ms_tuned = 0.0f;   // whole-batch times seen by the autotuner
    // The persistent form: per precision present, the recorded launch
    // sequences of its groups, the work queue over them and the launch shape
    // of the persistent kernel (bn_mega.cu).
    struct Persistent {
        int prec = 1;
        std::vector<bn::LaunchRec> recs;
        std::vector<int> depth, group;   // per record
        std::vector<int2> deps;          // per record: records it waits for (-1 none)
        std::vector<int4> items;         // {record, first block, end block, 0}
        std::vector<int> need;           // per record: its items
        bn::LaunchRec* recs_dev = nullptr;
        int4* items_dev = nullptr;
        int2* deps_dev = nullptr;
        int* need_dev = nullptr;
        int* ctl = nullptr;              // next item, status, abort, spare, done per record
        size_t ctl_bytes = 0, smem = 0;
        int blocks = 0, chunk = 1;
        uint64_t cap = (uint64_t)1 << 24;   // polls before a device wait gives up (seconds)
        float ms = 0.0f;
        std::string tried;               // chunk sizes timed and their ms
    };
    std::vector<Persistent> persistent;
    // bn_batch_upload / bn_batch_download: segment tables and staging buffers
    bn::CopySeg* segs_dev = nullptr;     // upload segments, then download segments
    unsigned char* dstage = nullptr;     // device staging: inputs, then results
    unsigned char* hstage = nullptr;     // pinned host staging, same layout
    size_t in_bytes = 0, out_bytes = 0;
    std::vector<size_t> in_off, out_off; // per job
    cudaEvent_t up_done = nullptr;       // the last upload's host-to-device copy
    char* progs = nullptr;               // device memory of the persistent programs
    bool use_persistent = false;
    float ms_graph = 0.0f;               // one replay of the graph of launches
};

namespace {

int dev_alloc(bn_ctx* c, void** p, size_t bytes, cudaStream_t s)
{
    if (c->fail_after >= 0 && c->allocs >= c->fail_after) return BN_ENOMEM;
    cudaError_t e = s ? cudaMallocAsync(p, bytes, s) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BN_ENOMEM;
    }
    ++c->allocs;
    return BN_OK;
}

int ensure_ws(bn_ctx* c, size_t bytes)
{
    if (c->ws_bytes >= bytes) return BN_OK;
    if (bytes > c->budget) return BN_ENOMEM;
    if (c->ws) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    void* p = nullptr;
    int rc = dev_alloc(c, &p, bytes, nullptr);
    if (rc) return rc;
    c->ws = (char*)p;
    c->ws_bytes = bytes;
    return BN_OK;
}

int ensure_pin(char** pin, size_t* have, size_t bytes)
{
    if (*have >= bytes) return BN_OK;
    if (*pin) cudaFreeHost(*pin);
    *pin = nullptr;
    *have = 0;
    if (cudaMallocHost((void**)pin, bytes) != cudaSuccess) return BN_ENOMEM;
    *have = bytes;
    return BN_OK;
}

size_t small_bytes(const Plan& P)
{
    return al(P.n) + al((size_t)(P.d + 1) * 8) + 2 * al((size_t)P.rows * 8) + 1024;
}

// Host memory the kernel reports available (bytes; 0 if unknown).
size_t host_available()
{
    FILE* f = std::fopen("/proc/meminfo", "r");
    if (!f) return 0;
    char line[256];
    size_t kb = 0;
    while (std::fgets(line, sizeof line, f))
        if (std::sscanf(line, "MemAvailable: %zu kB", &kb) == 1) break;
    std::fclose(f);
    return kb * 1024;
}

// A spilled job's A (a_bytes): one managed allocation, its first dev_part
// bytes preferred in device memory and prefetched there, the rest preferred
// in host memory, mapped for the GPU (which reads and writes it in place over
// the CPU-GPU link) and prefetched there.  Kept for the next job of the
// same size.
int ensure_spill(bn_ctx* c, size_t a_bytes, size_t dev_part, cudaStream_t s)
{
    if (c->spill && c->spill_bytes == a_bytes && c->spill_dev == dev_part) return BN_OK;
    if (c->spill) {
        cudaStreamSynchronize(s);
        cudaFree(c->spill);
        c->spill = nullptr;
        c->spill_bytes = c->spill_dev = 0;
    }
    if (c->fail_after >= 0 && c->allocs >= c->fail_after) return BN_ENOMEM;
    void* p = nullptr;
    if (cudaMallocManaged(&p, a_bytes, cudaMemAttachGlobal) != cudaSuccess) {
        cudaGetLastError();
        return BN_ENOMEM;
    }
    ++c->allocs;
    c->spill = (char*)p;
    c->spill_bytes = a_bytes;
    c->spill_dev = dev_part;
    cudaMemLocation gpu{}, host{};
    gpu.type = cudaMemLocationTypeDevice;
    gpu.id = c->device;
    host.type = cudaMemLocationTypeHost;
    host.id = 0;
    const size_t host_part = a_bytes - dev_part;
    if (dev_part) {
        CK(cudaMemAdvise(c->spill, dev_part, cudaMemAdviseSetPreferredLocation, gpu));
        CK(cudaMemPrefetchAsync(c->spill, dev_part, gpu, 0, s));
    }
    if (host_part) {
        CK(cudaMemAdvise(c->spill + dev_part, host_part, cudaMemAdviseSetPreferredLocation, host));
        CK(cudaMemAdvise(c->spill + dev_part, host_part, cudaMemAdviseSetAccessedBy, gpu));
        CK(cudaMemPrefetchAsync(c->spill + dev_part, host_part, host, 0, s));
    }
    return BN_OK;
}

int run_direct(bn_ctx* c, const bn_job_desc* job, HostJob& hj, double* post_dev,
               double* logPD_dev, cudaStream_t s)
{
    Layout L = make_layout(hj.P, 0);
    size_t a_bytes = 0, dev_part = 0;
    if (L.total > c->budget) {
        // the job's arrays exceed the device budget: A goes to managed
        // memory, as much of it in device memory as the budget leaves, the
        // rest in host memory (at most 3/4 of what the host has available)
        Plan& P = hj.P;
        P.spill = 1;
        P.vgroup = std::min(P.n, 8);              // the down-zeta scratch for 8 endpoints
        L = make_layout(P, 0);
        a_bytes = ((size_t)P.n << (P.n - 1)) * (P.prec == 0 ? 8 : 4);
        if (L.total >= c->budget) return BN_ENOMEM;
        const size_t gran = (size_t)2 << 20;
        dev_part = std::min<size_t>(a_bytes, (size_t)(c->budget - L.total)) / gran * gran;
        if (a_bytes - dev_part > host_available() / 4 * 3) return BN_ENOMEM;
    }
    char* old_ws = c->ws;
    int rc = ensure_ws(c, L.total);
    if (rc) return rc;
    if (a_bytes) {
        rc = ensure_spill(c, a_bytes, dev_part, s);
        if (rc) return rc;
    }
    rc = ensure_pin(&c->pin, &c->pin_bytes, small_bytes(hj.P) + 64);
    if (rc) return rc;
    Events& ev = c->ring[c->ring_pos % bn_ctx::kRing];
    if (!ev.ok && (rc = ev.create())) return rc;
    Bufs B{c->ws, L, a_bytes ? c->spill : nullptr};
    // The small tables (arity, log rho, lgamma rows) are uploaded only when
    // they differ from the ones already in the workspace; the pinned staging
    // buffer is rewritten only after earlier work has drained.
    std::vector<char> sig;
    auto put = [&](const void* p, size_t nb) {
        const char* q = (const char*)p;
        sig.insert(sig.end(), q, q + nb);
    };
    put(&hj.P, sizeof(Plan));
    put(&hj.ess, sizeof(double));
    put(hj.arity.data(), hj.arity.size());
    put(hj.log_rho.data(), hj.log_rho.size() * 8);
    put(hj.Dvals.data(), hj.Dvals.size() * 8);
    const bool upload = (old_ws != c->ws) || sig != c->tables_sig;
    if (upload) {
        if (s != c->stream) cudaStreamSynchronize(c->stream);
        cudaStreamSynchronize(s);
    }
    c->tables_sig.clear();
    rc = enqueue(hj, B, post_dev ? post_dev : B.at<double>(L.post),
                 logPD_dev ? logPD_dev : B.at<double>(L.logPD), s, &ev, &c->last_launches,
                 c->pin, c->pin_bytes, upload, &c->side);
    if (rc == BN_OK) {
        c->tables_sig = sig;
        c->ring_pos = (c->ring_pos + 1) % bn_ctx::kRing;
        c->ring_count = std::min(c->ring_count + 1, bn_ctx::kRing);
    }
    if (rc) return rc;
    c->last = hj.P;
    c->last_layout = L;
    c->have_last = true;
    (void)job;
    return BN_OK;
}

void pump(bn_ctx* c);

}  // namespace

// No C++ exception leaves the library: an entry point that catches one
// returns BN_ENOMEM for a failed host allocation and BN_EINVAL otherwise.
static int exception_code() noexcept
{
    try {
        throw;
    } catch (const std::bad_alloc&) {
        return BN_ENOMEM;
    } catch (const std::length_error&) {
        return BN_ENOMEM;
    } catch (...) {
        return BN_EINVAL;
    }
}

// A job's device error word as a status: the input check's bit is an
// invalid input, kErrDeviceTimeout a device-side wait that gave up.
static int err_word_status(int err) noexcept
{
    if (!err) return BN_OK;
    return (err & bn::kErrDeviceTimeout) ? BN_EDEVICE_TIMEOUT : BN_EINVAL;
}

extern "C" {

const char* bn_strerror(int code)
{
    switch (code) {
    case BN_OK: return "ok";
    case BN_EINVAL: return "invalid argument";
    case BN_ENOMEM: return "out of memory (device budget)";
    case BN_EAGAIN: return "job not finished";
    case BN_ETIMEOUT: return "timed out";
    case BN_EDEVICE_TIMEOUT: return "device-side wait gave up";
    case BN_ECUDA: return "CUDA error";
    case BN_ECANCELED: return "canceled";
    case BN_ENOTFOUND: return "unknown job id";
    default: return "unknown error";
    }
}

int64_t bn_num_families(int32_t n, int32_t d) { return families(n, d); }

int bn_job_footprint(const bn_job_desc* job, uint64_t* bytes)
try {
    if (!bytes) return BN_EINVAL;
    HostJob hj;
    const int rc = validate_and_plan(job, hj);
    if (rc) return rc;
    *bytes = make_layout(hj.P, 0).total;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_ctx_create(bn_ctx** out, const bn_ctx_opts* o)
try {
    if (!out) return BN_EINVAL;
    *out = nullptr;
    bn_ctx_opts opts{};
    opts.device = 0;
    opts.slots = 4;
    opts.mem_budget = 0;
    opts.fail_alloc_after = -1;
    if (o) opts = *o;
    if (opts.slots < 1 || opts.slots > 64 || opts.device < 0) return BN_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || opts.device >= ndev) {
        cudaGetLastError();
        return BN_ECUDA;
    }
    if (cudaSetDevice(opts.device) != cudaSuccess) return BN_ECUDA;
    if (bn::set_kernel_attributes() != cudaSuccess) return BN_ECUDA;
    if (bn::set_persistent_attributes() != cudaSuccess) return BN_ECUDA;
    bn_ctx* c = new bn_ctx();
    c->device = opts.device;
    c->fail_after = opts.fail_alloc_after;
    c->flags = opts.flags;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = opts.mem_budget ? opts.mem_budget : (uint64_t)(0.9 * (double)fr);
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        c->side.create() != BN_OK) {
        bn_ctx_destroy(c);
        return BN_ECUDA;
    }
    c->slots.resize(opts.slots);
    for (auto& sl : c->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            sl.ev.create() != BN_OK || cudaEventCreate(&sl.done) != cudaSuccess ||
            sl.side.create() != BN_OK) {
            bn_ctx_destroy(c);
            return BN_ECUDA;
        }
    }
    // keep freed stream-ordered memory in the pool between served jobs
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, opts.device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_ctx_destroy(bn_ctx* c)
try {
    if (!c) return BN_EINVAL;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& sl : c->slots) {
        if (sl.dev) cudaFree(sl.dev);
        if (sl.pin) cudaFreeHost(sl.pin);
        sl.ev.destroy();
        sl.side.destroy();
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (c->ws) cudaFree(c->ws);
    if (c->spill) cudaFree(c->spill);
    if (c->pin) cudaFreeHost(c->pin);
    for (auto& e : c->ring) e.destroy();
    c->side.destroy();
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_edge_posteriors_async(bn_ctx* c, const bn_job_desc* job, double* post_dev,
                             double* log_PD_dev, void* stream)
try {
    if (!c || !post_dev) return BN_EINVAL;
    HostJob hj;
    int rc = validate_and_plan(job, hj);
    if (rc) return rc;
    if (cudaSetDevice(c->device) != cudaSuccess) return BN_ECUDA;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    return run_direct(c, job, hj, post_dev, log_PD_dev, s);
} catch (...) {
    return exception_code();
}

int bn_edge_posteriors(bn_ctx* c, const bn_job_desc* job, double* post, double* log_PD)
try {
    if (!c || !post) return BN_EINVAL;
    HostJob hj;
    int rc = validate_and_plan(job, hj);
    if (rc) return rc;
    if (cudaSetDevice(c->device) != cudaSuccess) return BN_ECUDA;
    rc = run_direct(c, job, hj, nullptr, nullptr, c->stream);
    if (rc) return rc;
    const Layout& L = c->last_layout;
    const Plan& P = hj.P;
    int err = 0;
    CK(cudaMemcpyAsync(post, c->ws + L.post, (size_t)P.n * P.n * 8, cudaMemcpyDeviceToHost, c->stream));
    double lpd = 0;
    CK(cudaMemcpyAsync(&lpd, c->ws + L.logPD, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&err, c->ws + L.err, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (err) return err_word_status(err);
    if (log_PD) *log_PD = lpd;
    Events& ev = c->ring[(c->ring_pos + bn_ctx::kRing - 1) % bn_ctx::kRing];
    fill_stats(P, ev, c->last_launches, &c->last_stats);
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_scores(bn_ctx* c, const bn_job_desc* job, uint32_t* parent_mask, double* log_B)
try {
    if (!c || !parent_mask || !log_B) return BN_EINVAL;
    HostJob hj;
    int rc = validate_and_plan(job, hj);
    if (rc) return rc;
    if (cudaSetDevice(c->device) != cudaSuccess) return BN_ECUDA;
    // scores only: a workspace big enough for step 1
    Plan P = hj.P;
    Layout L = make_layout(P, 0);
    const size_t need = L.cmax;   // everything up to and including logB
    rc = ensure_ws(c, need + al((size_t)P.n * 8) + (P.hasw ? al((size_t)P.n * P.K * 8) : 0));
    if (rc) return rc;
    rc = ensure_pin(&c->pin, &c->pin_bytes, small_bytes(P) + 64);
    if (rc) return rc;
    cudaStreamSynchronize(c->stream);
    Bufs B{c->ws, L};
    cudaStream_t s = c->stream;
    const uint8_t* data_dev = B.at<uint8_t>(L.data);
    if (P.m > 0) {
        if (hj.data_on_device) data_dev = hj.data;
        else CK(cudaMemcpyAsync(B.at<uint8_t>(L.data), hj.data, (size_t)P.m * P.n, cudaMemcpyHostToDevice, s));
    }
    std::vector<double> lr(P.d + 1, 0.0);
    for (size_t t = 0; t < hj.log_rho.size(); ++t) lr[t] = hj.log_rho[t];
    std::vector<double> alpha(P.rows);
    for (int r = 0; r < P.rows; ++r) alpha[r] = hj.ess / hj.Dvals[r];
    CK(cudaMemcpyAsync(B.at<char>(L.arity), hj.arity.data(), P.n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.log_rho), lr.data(), lr.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.Dvals), hj.Dvals.data(), hj.Dvals.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.alpha), alpha.data(), alpha.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(B.at<int>(L.err), 0, 4, s));
    const uint8_t* ar = B.at<uint8_t>(L.arity);
    if (hj.data_on_device) CK(bn::launch_check_data(data_dev, ar, P.n, P.m, B.at<int>(L.err), s));
    CK(bn::launch_pack_planes(data_dev, P.n, P.m, P.rmax, P.W, B.at<uint64_t>(L.planes), s));
    CK(bn::launch_lgamma_table(B.at<double>(L.alpha), P.rows, P.m, P.fxs, B.at<void>(L.lgT), s));
    CK(bn::launch_scores(P, ar, B.at<uint64_t>(L.planes), B.at<double>(L.Dvals), B.at<void>(L.lgT),
                         hj.log_rho.empty() ? nullptr : B.at<double>(L.log_rho), 0,
                         (int64_t)P.n * P.K, B.at<uint32_t>(L.masks), B.at<uint32_t>(L.cmasks),
                         B.at<double>(L.logB), nullptr, s));
    if (P.hasw) {
        // the weights sit past logB in the layout: a scratch copy right after it
        double* w = reinterpret_cast<double*>(c->ws + need + al((size_t)P.n * 8));
        CK(cudaMemcpyAsync(w, hj.log_w.data(), hj.log_w.size() * 8, cudaMemcpyHostToDevice, s));
        CK(bn::launch_add_weights(P, B.at<double>(L.logB), w, s));
    }
    int err = 0;
    CK(cudaMemcpyAsync(parent_mask, B.at<char>(L.masks), (size_t)P.n * P.K * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(log_B, B.at<char>(L.logB), (size_t)P.n * P.K * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&err, B.at<char>(L.err), 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c->have_last = false;
    c->tables_sig.clear();
    return err ? BN_EINVAL : BN_OK;
} catch (...) {
    return exception_code();
}

int bn_feature_posterior(bn_ctx* c, const bn_job_desc* job, const double* log_f, double* p,
                         double* log_PfD)
try {
    if (!c || !log_f) return BN_EINVAL;
    HostJob hj;
    int rc = validate_and_plan(job, hj);
    if (rc) return rc;
    const Plan& P = hj.P;
    std::vector<double> lf;
    if (log_weights(log_f, (size_t)P.n * P.K, lf)) return BN_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return BN_ECUDA;
    const Layout L = make_layout(P, 0, true);
    rc = ensure_ws(c, L.total);
    if (rc) return rc;
    cudaStream_t s = c->stream;
    CK(cudaStreamSynchronize(s));
    c->have_last = false;
    c->tables_sig.clear();
    Bufs B{c->ws, L};
    // inputs: data, small tables, priors, the feature in the working units
    const uint8_t* data_dev = B.at<uint8_t>(L.data);
    if (P.m > 0) {
        if (hj.data_on_device) data_dev = hj.data;
        else CK(cudaMemcpyAsync(B.at<uint8_t>(L.data), hj.data, (size_t)P.m * P.n,
                                cudaMemcpyHostToDevice, s));
    }
    std::vector<double> lr(P.d + 1, 0.0);
    for (size_t t = 0; t < hj.log_rho.size(); ++t) lr[t] = hj.log_rho[t];
    std::vector<double> alpha(P.rows);
    for (int r = 0; r < P.rows; ++r) alpha[r] = hj.ess / hj.Dvals[r];
    CK(cudaMemcpyAsync(B.at<char>(L.arity), hj.arity.data(), P.n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.log_rho), lr.data(), lr.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.Dvals), hj.Dvals.data(), hj.Dvals.size() * 8,
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.alpha), alpha.data(), alpha.size() * 8, cudaMemcpyHostToDevice, s));
    rc = upload_priors(hj, B, s);
    if (rc) return rc;
    const std::vector<char> lfw = working_logs(lf, P.prec);
    CK(cudaMemcpyAsync(B.at<char>(L.logf), lfw.data(), lfw.size(), cudaMemcpyHostToDevice, s));

    // P(D): steps 1-3 with f = 1 (F only); then P(f, D) from the same
    // shifted scores plus log f (the shifts c_i cancel in the ratio)
    const size_t es = P.prec == 0 ? 8 : 4;
    const size_t full = ((size_t)1 << P.n) - 1;
    int nl = 0;
    rc = enqueue_step1(hj, B, data_dev, s, &nl);
    if (rc) return rc;
    rc = enqueue_upzeta(P, B, B.at<void>(L.lbs), s, &nl, nullptr);
    if (rc) return rc;
    CK(bn::launch_forward(P, B.at<void>(L.A), B.at<void>(L.F), s, &nl));
    double fv[2] = {0.0, 0.0};
    char raw[2][8];
    int lw[2][bn::kLevelWords];                  // FP32: the level words of each run's F
    CK(cudaMemcpyAsync(raw[0], B.at<char>(L.F) + full * es, es, cudaMemcpyDeviceToHost, s));
    if (P.prec != 0)
        CK(cudaMemcpyAsync(lw[0], B.at<char>(L.F) + (full + 1) * es, sizeof(lw[0]),
                           cudaMemcpyDeviceToHost, s));
    CK(bn::launch_add_feature(P, B.at<void>(L.lbs), B.at<void>(L.logf), B.at<void>(L.lbsf), s));
    rc = enqueue_upzeta(P, B, B.at<void>(L.lbsf), s, &nl, nullptr);
    if (rc) return rc;
    CK(bn::launch_forward(P, B.at<void>(L.A), B.at<void>(L.F), s, &nl));
    CK(cudaMemcpyAsync(raw[1], B.at<char>(L.F) + full * es, es, cudaMemcpyDeviceToHost, s));
    if (P.prec != 0)
        CK(cudaMemcpyAsync(lw[1], B.at<char>(L.F) + (full + 1) * es, sizeof(lw[1]),
                           cudaMemcpyDeviceToHost, s));
    std::vector<double> cmax(P.n);
    int err = 0;
    CK(cudaMemcpyAsync(cmax.data(), B.at<char>(L.cmax), (size_t)P.n * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&err, B.at<char>(L.err), 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (err) return err_word_status(err);
    for (int k = 0; k < 2; ++k) {
        if (P.prec == 0) {
            std::memcpy(&fv[k], raw[k], 8);
        } else {
            float x;
            std::memcpy(&x, raw[k], 4);
            const double b = bn::level_base_fwd(lw[k], P.n - bn::kLevelShift);
            fv[k] = ((double)x + b) * 0.69314718055994531;   // base 2 -> natural
        }
    }
    double csum = 0.0;
    for (double x : cmax) csum += x;
    // a feature weight of zero is held as kLogZero: a P(f, D) that far below
    // P(D) is an exact zero (a real feature's ratio is many orders of
    // magnitude closer)
    const bool zero = fv[1] - fv[0] < 0.5 * kLogZero;
    if (p) *p = zero ? 0.0 : std::exp(fv[1] - fv[0]);
    if (log_PfD) *log_PfD = zero ? -INFINITY : fv[1] + csum;
    return BN_OK;
} catch (...) {
    return exception_code();
}

#ifdef BN_TESTING
// Test hooks (stage dumps and device counts), compiled only into the testing
// build of the library.
int bn_debug_counts(bn_ctx* c, const bn_job_desc* job, int32_t i, uint32_t mask, int64_t* counts,
                    int64_t cells)
try {
    if (!c || !counts) return BN_EINVAL;
    HostJob hj;
    int rc = validate_and_plan(job, hj);
    if (rc) return rc;
    Plan& P = hj.P;
    if (i < 0 || i >= P.n || (mask >> i & 1u) || (P.n < 32 && (mask >> P.n))) return BN_EINVAL;
    const int k = __builtin_popcount(mask);
    if (k > P.d) return BN_EINVAL;
    int64_t want = hj.arity[i];
    for (int p = 0; p < P.n; ++p)
        if (mask >> p & 1u) want *= hj.arity[p];
    if (want != cells) return BN_EINVAL;
    // family index in canonical order
    const uint32_t low = (1u << i) - 1u;
    const uint32_t cm = (mask & low) | ((mask >> 1) & ~low);
    int64_t f = 0;
    for (int s = 0; s < k; ++s) f += host_binom(P.n - 1, s);
    int t = 1;
    for (uint32_t x = cm; x; x &= x - 1, ++t) f += host_binom(__builtin_ctz(x), t);
    if (cudaSetDevice(c->device) != cudaSuccess) return BN_ECUDA;
    Layout L = make_layout(P, (size_t)cells);
    rc = ensure_ws(c, L.total);
    if (rc) return rc;
    cudaStreamSynchronize(c->stream);
    Bufs B{c->ws, L};
    cudaStream_t s = c->stream;
    const uint8_t* data_dev = B.at<uint8_t>(L.data);
    if (P.m > 0) {
        if (hj.data_on_device) data_dev = hj.data;
        else CK(cudaMemcpyAsync(B.at<uint8_t>(L.data), hj.data, (size_t)P.m * P.n, cudaMemcpyHostToDevice, s));
    }
    std::vector<double> alpha(P.rows);
    for (int r = 0; r < P.rows; ++r) alpha[r] = hj.ess / hj.Dvals[r];
    CK(cudaMemcpyAsync(B.at<char>(L.arity), hj.arity.data(), P.n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.Dvals), hj.Dvals.data(), hj.Dvals.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.alpha), alpha.data(), alpha.size() * 8, cudaMemcpyHostToDevice, s));
    CK(bn::launch_pack_planes(data_dev, P.n, P.m, P.rmax, P.W, B.at<uint64_t>(L.planes), s));
    CK(bn::launch_lgamma_table(B.at<double>(L.alpha), P.rows, P.m, P.fxs, B.at<void>(L.lgT), s));
    CK(bn::launch_scores(P, B.at<uint8_t>(L.arity), B.at<uint64_t>(L.planes), B.at<double>(L.Dvals),
                         B.at<void>(L.lgT), nullptr, (int64_t)i * P.K + f, 1,
                         B.at<uint32_t>(L.masks), B.at<uint32_t>(L.cmasks), B.at<double>(L.logB),
                         B.at<int64_t>(L.dbg), s));
    CK(cudaMemcpyAsync(counts, B.at<char>(L.dbg), (size_t)cells * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c->have_last = false;
    c->tables_sig.clear();
    return BN_OK;
} catch (...) {
    return exception_code();
}

// A_i read back from tile-level row order (bn_device.cuh) into plain order,
// in place: the order permutes the rows inside each 2^13-value tile block
// only (row (H << rb) | r of A_i at (H << rb) | place(r), rows of 2^lw
// values, rb = 13 - lw), so one block at a time goes through a 32 KB copy.
static void tlo_to_plain(int n, float* a)
{
    static constexpr bn::PlaceTable pt = bn::make_place_table();
    const size_t half = (size_t)1 << (n - 1);
    std::vector<float> blk(8192);
    for (int i = 0; i < n; ++i) {
        const int lw = i < 4 ? 3 : 4, rb = 13 - lw;
        for (size_t b = 0; b < half; b += 8192) {
            float* base = a + i * half + b;
            std::memcpy(blk.data(), base, sizeof(float) * 8192);
            for (uint32_t r = 0; r < (1u << rb); ++r) {
                const uint32_t at = rb == 9 ? pt.p9[r] : pt.p10[r];
                std::memcpy(base + ((size_t)r << lw), blk.data() + ((size_t)at << lw),
                            sizeof(float) << lw);
            }
        }
    }
}

// FP32 F and R' are stored relative to per-level integer bases and Gamma
// relative to the integer Z (bn_device.cuh); the dumps add them back.
static void undo_level_bases(bn_ctx* c, const Plan& P, const Layout& L, int stage, float* out)
{
    const size_t N = (size_t)1 << P.n;
    int lf[bn::kLevelWords], lr[bn::kLevelWords];
    float fs = 0.f;
    if (cudaMemcpy(lf, c->ws + L.F + N * 4, sizeof(lf), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(lr, c->ws + L.Rc + N * 4, sizeof(lr), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&fs, c->ws + L.F + (N - 1) * 4, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        throw std::runtime_error("level words");
    const int nh = P.n - bn::kLevelShift;
    const bool fb = lf[bn::kLevelMode] == bn::kLevelShift, rb = lr[bn::kLevelMode] == bn::kLevelShift;
    if (stage == BN_STAGE_GAMMA) {
        const double Z = (fb ? bn::level_base_fwd(lf, nh) : 0.0) + std::floor((double)fs);
        for (size_t x = 0; x < (size_t)P.n * P.K; ++x) out[x] = (float)((double)out[x] + Z);
        return;
    }
    const int* lw = stage == BN_STAGE_F ? lf : lr;
    if (!(stage == BN_STAGE_F ? fb : rb)) return;
    double base[32];
    for (int k = 0; k <= nh; ++k)
        base[k] = stage == BN_STAGE_F ? bn::level_base_fwd(lw, k) : bn::level_base_bwd(lw, k, nh);
    for (size_t S = 0; S < N; ++S)
        out[S] = (float)((double)out[S] + base[__builtin_popcount((uint32_t)(S >> bn::kLevelShift))]);
}

int bn_debug_stage(bn_ctx* c, int32_t stage, void* host_out, size_t bytes)
try {
    if (!c || !host_out || !c->have_last) return BN_EINVAL;
    const Plan& P = c->last;
    const Layout& L = c->last_layout;
    const size_t es = P.prec == 0 ? 8 : 4;
    const size_t nK = (size_t)P.n * P.K;
    size_t off = 0, want = 0;
    switch (stage) {
    case BN_STAGE_LOGB: off = L.logB; want = nK * 8; break;
    case BN_STAGE_MASKS: off = L.masks; want = nK * 4; break;
    case BN_STAGE_SHIFT: off = L.cmax; want = (size_t)P.n * 8; break;
    case BN_STAGE_A: off = L.A; want = ((size_t)P.n << (P.n - 1)) * es; break;
    case BN_STAGE_F: off = L.F; want = ((size_t)1 << P.n) * es; break;
    case BN_STAGE_RC: off = L.Rc; want = ((size_t)1 << P.n) * es; break;
    case BN_STAGE_GAMMA: off = L.Gam; want = nK * es; break;
    default: return BN_EINVAL;
    }
    if (bytes != want) return BN_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    const char* src = (stage == BN_STAGE_A && P.spill) ? c->spill : c->ws + off;   // a spilled A
    CK(cudaMemcpy(host_out, src, want, cudaMemcpyDeviceToHost));
    if (stage == BN_STAGE_A && bn::use_tlo(P)) tlo_to_plain(P.n, static_cast<float*>(host_out));
    if (P.prec != 0 && (stage == BN_STAGE_F || stage == BN_STAGE_RC || stage == BN_STAGE_GAMMA))
        undo_level_bases(c, P, L, stage, static_cast<float*>(host_out));
    return BN_OK;
} catch (...) {
    return exception_code();
}
#endif  // BN_TESTING

int bn_job_stats(bn_ctx* c, uint64_t id, bn_stats* st)
try {
    if (!c || !st) return BN_EINVAL;
    if (id == 0) {
        *st = c->last_stats;
        return BN_OK;
    }
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->jobs.find(id);
    if (it == c->jobs.end()) return BN_ENOTFOUND;
    *st = it->second.stats;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_stats_history(bn_ctx* c, bn_stats* out, int32_t max, int32_t* count)
try {
    if (!c || !out || !count || max < 0) return BN_EINVAL;
    const int k = std::min<int>(max, c->ring_count);
    for (int t = 0; t < k; ++t) {
        const int idx = (c->ring_pos - k + t + 2 * bn_ctx::kRing) % bn_ctx::kRing;
        Events& ev = c->ring[idx];
        if (cudaEventSynchronize(ev.last()) != cudaSuccess) return BN_ECUDA;
        fill_stats(ev.P, ev, ev.launches, &out[t]);
    }
    *count = k;
    return BN_OK;
} catch (...) {
    return exception_code();
}

// ---------------------------------------------------------------- batches --

namespace {

// Steps 1-5 of the jobs of plan G (G.nj jobs G.js bytes apart from `base`,
// each laid out by L) on stream s; `stages` selects the parts: bit 0 step 1
// (per job) and the score shift, bit 1 step 2, bit 2 step 3, bit 3 step 4,
// bit 4 step 5.
int enqueue_steps(const Plan& G, const Layout& L, char* base, cudaStream_t s, unsigned stages,
                  const Side* side)
{
    auto at = [&](size_t off) { return base + off; };
    if (stages & 1u) {
        // one launch per kernel for the whole group, on the padded tables:
        // words past a job's m are empty and count nothing, rows past its
        // own are never looked up
        CK(bn::launch_pack_planes(reinterpret_cast<const uint8_t*>(at(L.data)), G.n, G.m, G.rmax,
                                  G.W, reinterpret_cast<uint64_t*>(at(L.planes)), s,
                                  reinterpret_cast<const int*>(at(L.mj)), G.nj, G.js));
        CK(bn::launch_lgamma_table(reinterpret_cast<const double*>(at(L.alpha)), G.rows, G.m,
                                   G.fxs, at(L.lgT), s, G.nj, G.js,
                                   reinterpret_cast<const double*>(at(L.fx)),
                                   reinterpret_cast<const int*>(at(L.mj))));
        CK(bn::launch_scores(G, reinterpret_cast<const uint8_t*>(at(L.arity)),
                             reinterpret_cast<const uint64_t*>(at(L.planes)),
                             reinterpret_cast<const double*>(at(L.Dvals)),
                             at(L.lgT),
                             reinterpret_cast<const double*>(at(L.log_rho)), 0,
                             (int64_t)G.n * G.K, reinterpret_cast<uint32_t*>(at(L.masks)),
                             reinterpret_cast<uint32_t*>(at(L.cmasks)),
                             reinterpret_cast<double*>(at(L.logB)), nullptr, s,
                             reinterpret_cast<const double*>(at(L.fx))));
        CK(bn::launch_node_max(G, reinterpret_cast<const double*>(at(L.logB)),
                               reinterpret_cast<double*>(at(L.cmax)), s));
        CK(bn::launch_shift_scores(G, reinterpret_cast<const double*>(at(L.logB)),
                                   reinterpret_cast<const double*>(at(L.cmax)), at(L.lbs), s));
        if (bn::tile13_gamma_fits(G)) {
            uint16_t* rk = reinterpret_cast<uint16_t*>(at(L.rk13));
            CK(bn::launch_rank13_tables(G, rk, rk + 8192, s));
        }
    }
    if (stages & 2u)
        CK(bn::launch_upzeta(G, reinterpret_cast<const uint32_t*>(at(L.cmasks)), at(L.lbs),
                             at(L.tab), reinterpret_cast<const uint16_t*>(at(L.rk13)), at(L.A), s));
    if (stages & 4u) {
        if (G.frc) {
            CK(bn::launch_rows_cluster(G, at(L.A), at(L.F), at(L.Rc), s, nullptr));
        } else if (side && side->s) {
            CK(cudaEventRecord(side->fork, s));
            CK(cudaStreamWaitEvent(side->s, side->fork, 0));
            CK(bn::launch_backward(G, at(L.A), at(L.Rc), side->s, nullptr));
            CK(cudaEventRecord(side->join, side->s));
            CK(bn::launch_forward(G, at(L.A), at(L.F), s, nullptr));
            CK(cudaStreamWaitEvent(s, side->join, 0));
        } else {
            CK(bn::launch_forward(G, at(L.A), at(L.F), s, nullptr));
            CK(bn::launch_backward(G, at(L.A), at(L.Rc), s, nullptr));
        }
    }
    if (stages & 8u) {
        CK(bn::launch_gamma_p1(G, at(L.F), at(L.Rc), reinterpret_cast<const uint16_t*>(at(L.rk13)),
                               at(L.W), s, nullptr, at(L.A)));
        CK(bn::launch_gamma_p2(G, at(L.W), at(L.Gam), s));
    }
    if (stages & 16u)
        CK(bn::launch_edges(G, reinterpret_cast<const double*>(at(L.logB)),
                            reinterpret_cast<const double*>(at(L.cmax)),
                            reinterpret_cast<const uint32_t*>(at(L.masks)), at(L.Gam), at(L.F),
                            reinterpret_cast<const int*>(at(L.err)),
                            reinterpret_cast<unsigned long long*>(at(L.eacc)),
                            reinterpret_cast<double*>(at(L.post)),
                            reinterpret_cast<double*>(at(L.logPD)), s));
    return BN_OK;
}

// Steps 1-5 of every job of group g on stream s (see enqueue_steps).
int enqueue_group(const bn_batch* b, const BatchGroup& g, cudaStream_t s, unsigned stages,
                  const Side* side = nullptr)
{
    return enqueue_steps(g.P, g.L, b->arena + g.base, s, stages, side);
}

// Every group of the batch on its branch stream (R' beside F), forked from
// and joined back into stream s: the work of one bn_batch_run.
int enqueue_batch(const bn_batch* b, cudaStream_t s)
{
    const int nb = (int)b->streams.size();
    CK(cudaEventRecord(b->fork, s));
    for (auto st : b->streams) CK(cudaStreamWaitEvent(st, b->fork, 0));
    for (size_t q = 0; q < b->groups.size(); ++q) {
        const int rc = enqueue_group(b, b->groups[q], b->streams[q % nb], 31u, &b->sides[q % nb]);
        if (rc) return rc;
    }
    for (int q = 0; q < nb; ++q) {
        CK(cudaEventRecord(b->joins[q], b->streams[q]));
        CK(cudaStreamWaitEvent(s, b->joins[q], 0));
    }
    return BN_OK;
}

// The whole batch under the groups' current plans, captured from stream s
// into an executable graph (nullptr on failure).
cudaGraphExec_t capture_batch(const bn_batch* b, cudaStream_t s, cudaGraph_t* graph)
{
    *graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return nullptr;
    const bool cap_ok = enqueue_batch(b, s) == BN_OK;
    cudaGraph_t gr = nullptr;
    const bool end_ok = cudaStreamEndCapture(s, &gr) == cudaSuccess;
    cudaGraphExec_t exec = nullptr;
    if (cap_ok && end_ok && gr && cudaGraphInstantiate(&exec, gr, 0) == cudaSuccess) {
        *graph = gr;
        return exec;
    }
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    return nullptr;
}

// Mean device time (ms) of one replay of the batch's graph under the
// groups' current plans: the graph bn_batch_run would launch, one warm-up
// replay and three timed ones.
int time_batch(const bn_batch* b, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms)
{
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = capture_batch(b, s, &gr);
    if (!ex) return BN_ECUDA;
    cudaError_t e = cudaGraphLaunch(ex, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; e == cudaSuccess && r < 3; ++r) e = cudaGraphLaunch(ex, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaGraphExecDestroy(ex);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return BN_ECUDA;
    *ms /= 3.0f;
    return BN_OK;
}

// The persistent form of a batch.  Each group's launch sequence is recorded
// with the launchers of the graph form (all the group's jobs per launch,
// gridDim.y = jobs), F and R' levels paired (F level l beside R' level l, the
// two sweeps being independent).  A record's depth is its position in the
// group's sequence (a pair shares one depth) and it waits for the group's
// records one depth earlier.  Returns BN_EINVAL when a group needs a kernel
// the persistent kernel does not run (the batch then keeps the graph).
int record_groups(bn_batch* b)
{
    std::vector<bn::LaunchRec> buf(8192);
    for (int prec = 0; prec <= 1; ++prec) {
        bn_batch::Persistent pp;
        pp.prec = prec;
        for (size_t gi = 0; gi < b->groups.size(); ++gi) {
            const BatchGroup& g = b->groups[gi];
            if (g.P.prec != prec) continue;
            Plan G = g.P;
            G.frc = 0;
            bn::Recorder rec;
            rec.recs = buf.data();
            rec.cap = (int)buf.size();
            bn::g_recorder = &rec;
            const int rc = enqueue_steps(G, g.L, b->arena + g.base, nullptr, 31u, nullptr);
            bn::g_recorder = nullptr;
            if (rc || rec.overflow) return BN_EINVAL;
            // the sequence as stages: one record each, or an (F, R') pair
            std::vector<std::vector<bn::LaunchRec>> stages;
            std::vector<bn::LaunchRec> fw, bw;
            size_t level_at = SIZE_MAX;
            for (int q = 0; q < rec.count; ++q) {
                bn::LaunchRec x = rec.recs[q];
                if (!bn::persistent_runs(prec, x.kid) || x.smem > 200 * 1024 ||
                    !(x.block == 256 || (x.kid == bn::KID_GAMMA_TABLE && x.block == 32)))
                    return BN_EINVAL;
                switch (x.kid) {                   // kernels that loop grid-stride in x
                case bn::KID_PACK_PLANES: case bn::KID_CHECK_DATA: case bn::KID_LGAMMA_TABLE:
                case bn::KID_SCORES: case bn::KID_SCORES_W42: case bn::KID_SCORES_W44:
                case bn::KID_SCORES_W84: case bn::KID_SCORES_CFG44: case bn::KID_SCORES_CFG:
                case bn::KID_SHIFT_F: case bn::KID_SHIFT_D: case bn::KID_EDGES_ACC_F:
                case bn::KID_EDGES_ACC_D: case bn::KID_REORDER_F: case bn::KID_REORDER_D:
                case bn::KID_COLW_F: case bn::KID_COLW_D:
                    x.pad[0] |= bn::kRecStrideX;
                    break;
                default:
                    break;
                }
                pp.smem = std::max<size_t>(pp.smem, x.smem);
                const bool f = x.kid == bn::KID_FROWS_F || x.kid == bn::KID_FROWS_F_TLO ||
                               x.kid == bn::KID_FROWS_D || x.kid == bn::KID_FWD_LEVEL_F ||
                               x.kid == bn::KID_FWD_LEVEL_D;
                const bool r = x.kid == bn::KID_BROWS_F || x.kid == bn::KID_BROWS_F_TLO ||
                               x.kid == bn::KID_BROWS_D || x.kid == bn::KID_BWD_LEVEL_F ||
                               x.kid == bn::KID_BWD_LEVEL_D;
                if (f || r) {
                    if (level_at == SIZE_MAX) level_at = stages.size();
                    (f ? fw : bw).push_back(x);
                } else {
                    stages.push_back({x});
                }
            }
            if (level_at != SIZE_MAX) {
                std::vector<std::vector<bn::LaunchRec>> lv;
                for (size_t q = 0; q < std::max(fw.size(), bw.size()); ++q) {
                    lv.emplace_back();
                    if (q < fw.size()) lv.back().push_back(fw[q]);
                    if (q < bw.size()) lv.back().push_back(bw[q]);
                }
                stages.insert(stages.begin() + level_at, lv.begin(), lv.end());
            }
            int prev0 = -1, prev1 = -1;
            for (size_t d = 0; d < stages.size(); ++d) {
                const int first = (int)pp.recs.size();
                for (const auto& x : stages[d]) {
                    pp.recs.push_back(x);
                    pp.depth.push_back((int)d);
                    pp.group.push_back((int)gi);
                    pp.deps.push_back(int2{prev0, prev1});
                }
                prev0 = first;
                prev1 = stages[d].size() > 1 ? first + 1 : -1;
            }
        }
        if (!pp.recs.empty()) b->persistent.push_back(std::move(pp));
    }
    return BN_OK;
}

// The work queue of one precision for `chunk` blocks per item: a grid-stride
// kernel runs about `blocks` blocks per record (its x width shrunk to fit),
// a record with more blocks than the persistent kernel has goes in items of
// up to `chunk` blocks, and the items of all groups are ordered by depth.
void build_queue(bn_batch::Persistent& pp, int chunk)
{
    const int nrec = (int)pp.recs.size();
    pp.need.assign(nrec, 0);
    std::vector<int> order(nrec);
    for (int r = 0; r < nrec; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return pp.depth[x] != pp.depth[y] ? pp.depth[x] < pp.depth[y] : x < y;
    });
    pp.items.clear();
    for (int r : order) {
        bn::LaunchRec& x = pp.recs[r];
        const uint64_t yz = (uint64_t)x.gy * x.gz;
        if (x.pad[0] & bn::kRecStrideX) {
            // rewrite the record's width once, from its recorded width
            if (x.pad[1] == 0) x.pad[1] = x.gx;
            const uint64_t want = std::max<uint64_t>(1, ((uint64_t)pp.blocks + yz - 1) / yz);
            x.gx = (uint32_t)std::min<uint64_t>(x.pad[1], want);
        }
        const int nvb = (int)(x.gx * yz);
        const int c = nvb > pp.blocks ? chunk : 1;
        for (int v = 0; v < nvb; v += c) {
            pp.items.push_back(int4{r, v, std::min(nvb, v + c), 0});
            ++pp.need[r];
        }
    }
    pp.chunk = chunk;
}

int upload_queue(bn_batch* b, bn_batch::Persistent& pp)
{
    CK(cudaMemcpy(pp.recs_dev, pp.recs.data(), pp.recs.size() * sizeof(bn::LaunchRec),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pp.items_dev, pp.items.data(), pp.items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pp.deps_dev, pp.deps.data(), pp.deps.size() * sizeof(int2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pp.need_dev, pp.need.data(), pp.need.size() * sizeof(int), cudaMemcpyHostToDevice));
    (void)b;
    return BN_OK;
}

// Device memory for the programs (the item array sized for chunk 1, the
// most items) and the first queue.
int build_persistent(bn_batch* b)
{
    int rc = record_groups(b);
    if (rc) return rc;
    auto al256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t bytes = 0;
    for (auto& pp : b->persistent) {
        pp.blocks = bn::persistent_blocks(pp.prec, pp.smem);
        if (pp.blocks < 1) return BN_ECUDA;
        build_queue(pp, 1);
        const size_t nrec = pp.recs.size();
        pp.ctl_bytes = 16 + 4 * nrec;
        bytes += al256(nrec * sizeof(bn::LaunchRec)) + al256(pp.items.size() * sizeof(int4)) +
                 al256(nrec * sizeof(int2)) + al256(nrec * 4) + al256(pp.ctl_bytes);
    }
    void* p = nullptr;
    rc = dev_alloc(b->ctx, &p, bytes, nullptr);
    if (rc) return rc;
    b->progs = (char*)p;
    size_t o = 0;
    for (auto& pp : b->persistent) {
        const size_t nrec = pp.recs.size();
        pp.recs_dev = reinterpret_cast<bn::LaunchRec*>(b->progs + o);
        o += al256(nrec * sizeof(bn::LaunchRec));
        pp.items_dev = reinterpret_cast<int4*>(b->progs + o);
        o += al256(pp.items.size() * sizeof(int4));
        pp.deps_dev = reinterpret_cast<int2*>(b->progs + o);
        o += al256(nrec * sizeof(int2));
        pp.need_dev = reinterpret_cast<int*>(b->progs + o);
        o += al256(nrec * 4);
        pp.ctl = reinterpret_cast<int*>(b->progs + o);
        o += al256(pp.ctl_bytes);
        rc = upload_queue(b, pp);
        if (rc) return rc;
    }
    return BN_OK;
}

int run_persistent(const bn_batch* b, cudaStream_t s)
{
    for (const auto& pp : b->persistent)
        CK(bn::launch_persistent(pp.prec, pp.recs_dev, pp.items_dev, (int)pp.items.size(),
                                 pp.deps_dev, pp.need_dev, pp.ctl, pp.ctl_bytes, pp.blocks, pp.smem,
                                 pp.cap, s));
    return BN_OK;
}

// The persistent form's tuner: for each precision, the item size (1, 2 or 4
// blocks of a launch per queue item) that runs the batch fastest, each
// launch timed on the batch's own data (one warm-up launch, three timed).
int tune_persistent(bn_batch* b, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    for (auto& pp : b->persistent) {
        float best = 0.0f;
        int best_c = 0;
        for (int c : {1, 2, 4}) {
            build_queue(pp, c);
            if (upload_queue(b, pp) != BN_OK) return BN_ECUDA;
            cudaError_t e = bn::launch_persistent(pp.prec, pp.recs_dev, pp.items_dev,
                                                  (int)pp.items.size(), pp.deps_dev, pp.need_dev,
                                                  pp.ctl, pp.ctl_bytes, pp.blocks, pp.smem, pp.cap, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int r = 0; e == cudaSuccess && r < 3; ++r)
                e = bn::launch_persistent(pp.prec, pp.recs_dev, pp.items_dev, (int)pp.items.size(),
                                          pp.deps_dev, pp.need_dev, pp.ctl, pp.ctl_bytes, pp.blocks,
                                          pp.smem, pp.cap, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return BN_ECUDA;
            }
            ms /= 3.0f;
            char t[48];
            std::snprintf(t, sizeof t, "%s%d:%.3f", pp.tried.empty() ? "" : " ", c, ms);
            pp.tried += t;
            if (best_c == 0 || ms < best) {
                best = ms;
                best_c = c;
            }
        }
        build_queue(pp, best_c);
        if (upload_queue(b, pp) != BN_OK) return BN_ECUDA;
        pp.ms = best;
    }
    return BN_OK;
}

// The autotuner.  The groups of a batch run at the same time, so a kernel
// that wins alone (by spreading over the whole GPU) can lose in the mix; the
// objective is therefore the time of the whole batch, on its own data.
// Starting from the default schedules, each knob in turn -- step 1 score
// kernel, step 2 tiles, step 3 rows, step 3 cluster kernel, step 4 tiles --
// is switched to its alternative for three sets of groups where it fits
// (all, those with n <= 14, those with n > 14); the fastest batch is kept
// when it beats the current one by more than 1%.
int tune_batch(bn_batch* b, cudaStream_t s)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return BN_ECUDA;
    }
    struct Knob { int Plan::*flag; bool (*fits)(const Plan&); };
    const Knob knobs[5] = {{&Plan::scfg, bn::scores_cfg_fits}, {&Plan::up13, bn::tile13_up_fits},
                           {&Plan::frows, bn::rows_levels_fit}, {&Plan::frc, bn::rows_levels_fit},
                           {&Plan::g13, bn::tile13_gamma_fits}};
    const bool forced_frc = (b->ctx->flags & BN_CTX_CLUSTER_STEP3) != 0;
    float best = 0.0f;
    int rc = time_batch(b, s, e0, e1, &best);
    b->ms_default = best;
    for (int k = 0; rc == BN_OK && k < 5; ++k) {
        if (knobs[k].flag == &Plan::frc && forced_frc) continue;
        std::vector<Plan> keep;
        for (auto& g : b->groups) keep.push_back(g.P);
        std::vector<int> best_sel;                  // groups switched in the best candidate
        for (int cand = 0; rc == BN_OK && cand < 3; ++cand) {
            std::vector<int> sel;
            for (size_t q = 0; q < b->groups.size(); ++q) {
                const Plan& P = keep[q];
                const bool in = cand == 0 || (cand == 1 ? P.n <= 14 : P.n > 14);
                if (in && knobs[k].fits(P)) sel.push_back((int)q);
            }
            if (sel.empty()) continue;
            for (int q : sel) {
                Plan& P = b->groups[q].P;
                P.*(knobs[k].flag) = 1 - P.*(knobs[k].flag);
            }
            float t = 0.0f;
            rc = time_batch(b, s, e0, e1, &t);
            for (int q : sel) b->groups[q].P = keep[q];
            if (rc == BN_OK && t < 0.99f * best) {
                best = t;
                best_sel = sel;
            }
        }
        for (int q : best_sel) {
            Plan& P = b->groups[q].P;
            P.*(knobs[k].flag) = 1 - P.*(knobs[k].flag);
        }
    }
    b->ms_tuned = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == BN_OK)
        for (auto& g : b->groups) g.timed = true;
    return rc;
}

}  // namespace

int bn_batch_create(bn_ctx* c, const bn_job_desc* jobs, int32_t count, bn_batch** out)
try {
    if (!c || !jobs || !out || count < 1) return BN_EINVAL;
    *out = nullptr;
    bn_batch* b = new bn_batch();
    b->ctx = c;
    b->jobs.resize(count);
    b->group_of.assign(count, -1);
    b->slot_of.assign(count, -1);
    std::map<std::array<int, 4>, int> key_to_group;
    for (int k = 0; k < count; ++k) {
        HostJob& hj = b->jobs[k];
        int rc = jobs[k].data_on_device ? BN_EINVAL : validate_and_plan(&jobs[k], hj);
        if (!rc && (hj.P.hasq || hj.P.hasw)) rc = BN_EINVAL;   // not in the batch layout
        if (rc) { delete b; return rc; }
        const Plan& P = hj.P;
        hj.data_copy.assign(jobs[k].data ? jobs[k].data : (const uint8_t*)"",
                            jobs[k].data ? jobs[k].data + (size_t)P.m * P.n : (const uint8_t*)"");
        hj.data = hj.data_copy.data();
        // step 1 of a group is one launch per kernel, so its jobs also share
        // the choice of score kernel (binary data or not)
        const std::array<int, 4> key{P.n, P.d, P.prec, P.allbin};
        auto it = key_to_group.find(key);
        if (it == key_to_group.end()) {
            it = key_to_group.emplace(key, (int)b->groups.size()).first;
            b->groups.emplace_back();
            b->groups.back().P = P;
        }
        BatchGroup& g = b->groups[it->second];
        b->group_of[k] = it->second;
        b->slot_of[k] = (int)g.members.size();
        g.members.push_back(k);
        // the padded plan: the largest step-1 tables of the group
        g.P.m = std::max(g.P.m, P.m);
        g.P.W = std::max(g.P.W, P.W);
        g.P.rmax = std::max(g.P.rmax, P.rmax);
        g.P.rows = std::max(g.P.rows, P.rows);
    }
    size_t total = 0;
    for (auto& g : b->groups) {
        g.L = make_layout(g.P, 0);
        g.P.nj = (int)g.members.size();
        g.P.js = g.L.total;
        g.base = total;
        total += (size_t)g.P.nj * g.P.js;
    }
    if (total > c->budget) { delete b; return BN_ENOMEM; }
    if (cudaSetDevice(c->device) != cudaSuccess) { delete b; return BN_ECUDA; }
    void* p = nullptr;
    int rc = dev_alloc(c, &p, total, nullptr);
    if (rc) { delete b; return rc; }
    b->arena = (char*)p;
    rc = BN_ECUDA;
    cudaStream_t cap = c->stream;
    const int nb = std::min((int)b->groups.size(), 32);
    b->streams.assign(nb, nullptr);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (auto& st : b->streams) ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    b->joins.assign(nb, nullptr);
    for (auto& e : b->joins) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    b->sides.resize(nb);
    for (auto& sd : b->sides) ok = ok && sd.create() == BN_OK;
    // inputs go to the device now; only kernels are captured
    ok = ok && cudaMemset(b->arena, 0, total) == cudaSuccess;
    for (int k = 0; ok && k < count; ++k) {
        const HostJob& hj = b->jobs[k];
        const BatchGroup& g = b->groups[b->group_of[k]];
        const Layout& L = g.L;
        char* jb = b->arena + g.base + (size_t)b->slot_of[k] * g.P.js;
        // the group's tables have g.P.rows rows: the rows past the job's own
        // hold a denominator no lookup asks for (the table stays sorted) and
        // alpha = 1
        std::vector<double> lr(hj.P.d + 1, 0.0), alpha(g.P.rows, 1.0), dv(g.P.rows, 1e300);
        for (size_t t = 0; t < hj.log_rho.size(); ++t) lr[t] = hj.log_rho[t];
        for (int r = 0; r < hj.P.rows; ++r) {
            alpha[r] = hj.ess / hj.Dvals[r];
            dv[r] = hj.Dvals[r];
        }
        const int mj = hj.P.m;
        // the job's own fixed-point shift, as when it runs alone
        const double fx[2] = {std::ldexp(1.0, hj.P.fxs), std::ldexp(1.0, -hj.P.fxs)};
        ok = (hj.P.m == 0 || cudaMemcpy(jb + L.data, hj.data, (size_t)hj.P.m * hj.P.n,
                                        cudaMemcpyHostToDevice) == cudaSuccess) &&
             cudaMemcpy(jb + L.mj, &mj, 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(jb + L.fx, fx, 16, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(jb + L.arity, hj.arity.data(), hj.P.n, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(jb + L.log_rho, lr.data(), lr.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(jb + L.Dvals, dv.data(), dv.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(jb + L.alpha, alpha.data(), alpha.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    // schedules: the default, forced, cached (when every group's shape is in
    // the context's cache) or timed
    for (auto& g : b->groups)
        if (c->flags & BN_CTX_CLUSTER_STEP3) g.P.frc = bn::rows_levels_fit(g.P);
    auto key_of = [](const Plan& P) {
        return std::array<int, 5>{P.n, P.d, P.prec, P.allbin, P.nj};
    };
    const bool want_persistent = !(c->flags & (BN_CTX_GRAPH_BATCH | BN_CTX_CLUSTER_STEP3));
    if (ok && !(c->flags & BN_CTX_NO_AUTOTUNE)) {
        bool all_cached = true;
        for (const auto& g : b->groups) all_cached = all_cached && c->tuned.count(key_of(g.P)) > 0;
        if (all_cached) {
            for (auto& g : b->groups) {
                const auto& v = c->tuned[key_of(g.P)];
                g.P.scfg = v[0];
                g.P.up13 = v[1];
                g.P.frows = v[2];
                g.P.frc = v[3];
                g.P.g13 = v[4];
            }
        } else {
            ok = tune_batch(b, cap) == BN_OK;
            for (const auto& g : b->groups)
                if (ok) c->tuned[key_of(g.P)] = {g.P.scfg, g.P.up13, g.P.frows, g.P.frc, g.P.g13};
        }
    }
    ok = ok && cudaStreamSynchronize(cap) == cudaSuccess;
    if (ok) {
        b->exec = capture_batch(b, cap, &b->graph);
        if (b->exec) rc = BN_OK;
    }
    cudaGetLastError();
    if (rc) { bn_batch_destroy(b); return rc; }
    // one replay of the graph, timed for the comparison bn_batch_describe reports
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        bool t_ok = cudaGraphLaunch(b->exec, cap) == cudaSuccess &&
                    cudaEventRecord(e0, cap) == cudaSuccess;
        for (int r = 0; t_ok && r < 3; ++r) t_ok = cudaGraphLaunch(b->exec, cap) == cudaSuccess;
        t_ok = t_ok && cudaEventRecord(e1, cap) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
               cudaEventElapsedTime(&b->ms_graph, e0, e1) == cudaSuccess;
        b->ms_graph = t_ok ? b->ms_graph / 3.0f : 0.0f;
        if (want_persistent && build_persistent(b) == BN_OK) {
            if (c->flags & BN_CTX_NO_AUTOTUNE) {
                b->use_persistent = true;
            } else if (tune_persistent(b, cap, e0, e1) == BN_OK) {
                // the form that runs the whole batch faster
                float ms = 0.0f;
                for (const auto& pp : b->persistent) ms += pp.ms;
                b->use_persistent = b->ms_graph <= 0.0f || ms < b->ms_graph;
            }
        }
        cudaGetLastError();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *out = b;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_batch_run(bn_batch* b, void* stream)
try {
    if (!b || !b->exec) return BN_EINVAL;
    cudaSetDevice(b->ctx->device);
    b->last = stream ? (cudaStream_t)stream : b->ctx->stream;
    if (b->use_persistent) {
        const int rc = run_persistent(b, b->last);
        if (rc) return rc;
    } else {
        CK(cudaGraphLaunch(b->exec, b->last));
    }
    b->ran = true;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_batch_results(bn_batch* b, int32_t k, double* post, double* log_PD)
try {
    if (!b || !post || k < 0 || k >= (int32_t)b->jobs.size() || !b->ran) return BN_EINVAL;
    const Plan& P = b->jobs[k].P;
    const BatchGroup& g = b->groups[b->group_of[k]];
    const char* jb = b->arena + g.base + (size_t)b->slot_of[k] * g.P.js;
    CK(cudaStreamSynchronize(b->last));
    CK(cudaMemcpy(post, jb + g.L.post, (size_t)P.n * P.n * 8, cudaMemcpyDeviceToHost));
    if (log_PD) CK(cudaMemcpy(log_PD, jb + g.L.logPD, 8, cudaMemcpyDeviceToHost));
    int err = 0;
    CK(cudaMemcpy(&err, jb + g.L.err, 4, cudaMemcpyDeviceToHost));
    if (b->use_persistent)
        for (const auto& pp : b->persistent)
            if (pp.prec == P.prec) {
                int st = 0;
                CK(cudaMemcpy(&st, pp.ctl + 1, 4, cudaMemcpyDeviceToHost));
                if (st) return st;
            }
    return err ? BN_EINVAL : BN_OK;
} catch (...) {
    return exception_code();
}

int bn_batch_describe(bn_batch* b, char* buf, size_t len)
try {
    if (!b || !buf || len == 0) return BN_EINVAL;
    std::string s;
    char line[256];
    for (const auto& g : b->groups) {
        std::snprintf(line, sizeof line,
                      "n=%d d=%d %s %s jobs=%d scfg=%d up13=%d frows=%d frc=%d g13=%d %s"
                      " batch_ms(default %.3f tuned %.3f)\n",
                      g.P.n, g.P.d, g.P.prec == 0 ? "fp64" : "fp32",
                      g.P.allbin ? "binary" : "general", g.P.nj, g.P.scfg, g.P.up13, g.P.frows,
                      g.P.frc, g.P.g13, g.timed ? "timed" : "default-or-cached", b->ms_default,
                      b->ms_tuned);
        s += line;
    }
    for (const auto& pp : b->persistent) {
        uint64_t vbs = 0;
        for (const auto& x : pp.recs) vbs += (uint64_t)x.gx * x.gy * x.gz;
        std::snprintf(line, sizeof line,
                      "persistent %s: records=%zu vblocks=%llu items=%zu blocks=%d chunk=%d ms=%.3f"
                      " (chunk:ms %s) graph_ms=%.3f %s\n",
                      pp.prec == 0 ? "fp64" : "fp32", pp.recs.size(), (unsigned long long)vbs,
                      pp.items.size(), pp.blocks, pp.chunk, pp.ms,
                      pp.tried.empty() ? "fixed" : pp.tried.c_str(), b->ms_graph,
                      b->use_persistent ? "in use" : "not used");
        s += line;
    }
    std::snprintf(buf, len, "%s", s.c_str());
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_batch_destroy(bn_batch* b)
try {
    if (!b) return BN_EINVAL;
    cudaSetDevice(b->ctx->device);
    if (b->ran) cudaStreamSynchronize(b->last);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto st : b->streams) if (st) cudaStreamDestroy(st);
    for (auto& sd : b->sides) sd.destroy();
    for (auto e : b->joins) if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->arena) cudaFree(b->arena);
    if (b->progs) cudaFree(b->progs);
    if (b->dstage) cudaFree(b->dstage);
    if (b->hstage) cudaFreeHost(b->hstage);
    if (b->up_done) cudaEventDestroy(b->up_done);
    delete b;
    return BN_OK;
} catch (...) {
    return exception_code();
}

namespace {

// Staging for bn_batch_upload / bn_batch_download, made on first use: every
// job's data packed in job order, then every job's results (n*n posteriors,
// log P(D), the input-check word), each part 16-byte aligned.
int ensure_e2e(bn_batch* b)
{
    if (b->dstage) return BN_OK;
    const int count = (int)b->jobs.size();
    auto al16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    b->in_off.resize(count);
    b->out_off.resize(count);
    size_t o = 0;
    for (int k = 0; k < count; ++k) {
        b->in_off[k] = o;
        o += al16((size_t)b->jobs[k].P.m * b->jobs[k].P.n);
    }
    b->in_bytes = o;
    for (int k = 0; k < count; ++k) {
        b->out_off[k] = o;
        o += al16((size_t)b->jobs[k].P.n * b->jobs[k].P.n * 8) + 16;
    }
    b->out_bytes = o - b->in_bytes;
    std::vector<bn::CopySeg> segs;
    void* p = nullptr;
    int rc = dev_alloc(b->ctx, &p, std::max<size_t>(o, 16) + (size_t)4 * count * sizeof(bn::CopySeg),
                       nullptr);
    if (rc) return rc;
    b->dstage = (unsigned char*)p;
    b->segs_dev = reinterpret_cast<bn::CopySeg*>(b->dstage + ((std::max<size_t>(o, 16) + 15) & ~size_t(15)));
    for (int k = 0; k < count; ++k) {              // staging -> each job's data
        const BatchGroup& g = b->groups[b->group_of[k]];
        unsigned char* jb = (unsigned char*)b->arena + g.base + (size_t)b->slot_of[k] * g.P.js;
        segs.push_back({b->dstage + b->in_off[k], jb + g.L.data,
                        (uint64_t)b->jobs[k].P.m * b->jobs[k].P.n});
    }
    for (int k = 0; k < count; ++k) {              // each job's results -> staging
        const BatchGroup& g = b->groups[b->group_of[k]];
        const size_t n2 = (size_t)b->jobs[k].P.n * b->jobs[k].P.n * 8;
        unsigned char* jb = (unsigned char*)b->arena + g.base + (size_t)b->slot_of[k] * g.P.js;
        unsigned char* to = b->dstage + b->out_off[k];
        segs.push_back({jb + g.L.post, to, n2});
        segs.push_back({jb + g.L.logPD, to + ((n2 + 15) & ~size_t(15)), 8});
        segs.push_back({jb + g.L.err, to + ((n2 + 15) & ~size_t(15)) + 8, 4});
    }
    CK(cudaMemcpy(b->segs_dev, segs.data(), segs.size() * sizeof(bn::CopySeg), cudaMemcpyHostToDevice));
    if (cudaMallocHost(&p, std::max<size_t>(o, 16)) != cudaSuccess) {
        cudaGetLastError();
        return BN_ENOMEM;
    }
    b->hstage = (unsigned char*)p;
    CK(cudaEventCreateWithFlags(&b->up_done, cudaEventDisableTiming));
    return BN_OK;
}

}  // namespace

int bn_batch_upload(bn_batch* b, const bn_job_desc* jobs, int32_t count, void* stream)
try {
    if (!b || !jobs || count != (int32_t)b->jobs.size()) return BN_EINVAL;
    for (int k = 0; k < count; ++k) {
        const bn_job_desc& j = jobs[k];
        const HostJob& hj = b->jobs[k];
        const Plan& P = hj.P;
        if (j.data_on_device || j.n != P.n || j.m != P.m || j.precision != P.prec * BN_FP32_SHIFTED ||
            std::min(j.d, j.n - 1) != P.d || !j.arity || !(j.ess == hj.ess) || j.log_q || j.log_w ||
            (P.m > 0 && !j.data))
            return BN_EINVAL;
        for (int v = 0; v < P.n; ++v)
            if (j.arity[v] != hj.arity[v]) return BN_EINVAL;
        for (int t = 0; t <= P.d; ++t) {
            const double lr = j.log_rho ? j.log_rho[t] : 0.0;
            const double had = t < (int)hj.log_rho.size() ? hj.log_rho[t] : 0.0;
            if (!(lr == had)) return BN_EINVAL;
        }
        if (P.m > 0 && !bn::data_below_arity(j.data, P.m, P.n, hj.arity.data())) return BN_EINVAL;
    }
    if (cudaSetDevice(b->ctx->device) != cudaSuccess) return BN_ECUDA;
    int rc = ensure_e2e(b);
    if (rc) return rc;
    cudaStream_t s = stream ? (cudaStream_t)stream : b->ctx->stream;
    CK(cudaEventSynchronize(b->up_done));          // the staging buffer is free again
    for (int k = 0; k < count; ++k)
        if (b->jobs[k].P.m > 0)
            std::memcpy(b->hstage + b->in_off[k], jobs[k].data, (size_t)b->jobs[k].P.m * b->jobs[k].P.n);
    CK(cudaMemcpyAsync(b->dstage, b->hstage, b->in_bytes, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(b->up_done, s));
    CK(bn::launch_copy_segments(b->segs_dev, count, s));
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_batch_download(bn_batch* b, double* post_all, double* log_PD_all)
try {
    if (!b || !post_all || !b->ran) return BN_EINVAL;
    if (cudaSetDevice(b->ctx->device) != cudaSuccess) return BN_ECUDA;
    int rc = ensure_e2e(b);
    if (rc) return rc;
    const int count = (int)b->jobs.size();
    cudaStream_t s = b->last;
    CK(bn::launch_copy_segments(b->segs_dev + count, 3 * count, s));
    CK(cudaMemcpyAsync(b->hstage + b->in_bytes, b->dstage + b->in_bytes, b->out_bytes,
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int bad = 0;
    size_t po = 0;
    for (int k = 0; k < count; ++k) {
        const size_t n2 = (size_t)b->jobs[k].P.n * b->jobs[k].P.n * 8;
        const unsigned char* from = b->hstage + b->out_off[k];
        std::memcpy(post_all + po, from, n2);
        po += n2 / 8;
        const size_t tail = (n2 + 15) & ~size_t(15);
        if (log_PD_all) std::memcpy(log_PD_all + k, from + tail, 8);
        int err = 0;
        std::memcpy(&err, from + tail + 8, 4);
        bad |= err;
    }
    if (b->use_persistent)
        for (const auto& pp : b->persistent) {
            int st = 0;
            CK(cudaMemcpy(&st, pp.ctl + 1, 4, cudaMemcpyDeviceToHost));
            if (st) return st;
        }
    return bad ? BN_EINVAL : BN_OK;
} catch (...) {
    return exception_code();
}

#ifdef BN_TESTING
// Test hook: the persistent form with one stage missing from the queue (its
// results never come), every device wait bounded at `polls` polls.
int bn_debug_batch_drop(bn_batch* b, int32_t depth, uint64_t polls)
try {
    if (!b || !b->use_persistent || polls < 1) return BN_EINVAL;
    for (auto& pp : b->persistent) {
        std::vector<int4> kept;
        for (const int4& it : pp.items)
            if (pp.depth[it.x] != depth) kept.push_back(it);
        pp.items.swap(kept);
        pp.cap = polls;
        CK(cudaMemcpy(pp.items_dev, pp.items.data(), pp.items.size() * sizeof(int4),
                      cudaMemcpyHostToDevice));
    }
    return BN_OK;
} catch (...) {
    return exception_code();
}

// Test hook: the FP64 table-driven exp and log beside CUDA's, on the
// current device.
int bn_debug_explog(const double* x, int64_t count, double* out)
try {
    if (!x || !out || count < 0) return BN_EINVAL;
    if (count == 0) return BN_OK;
    double* dx = nullptr;
    double* dout = nullptr;
    CK(cudaMalloc(&dx, (size_t)count * 8));
    if (cudaMalloc(&dout, (size_t)count * 32) != cudaSuccess) {
        cudaFree(dx);
        return BN_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(dx, x, (size_t)count * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = bn::launch_explog_check(dx, count, dout, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)count * 32, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dout);
    return e == cudaSuccess ? BN_OK : BN_ECUDA;
} catch (...) {
    return exception_code();
}

// Test hook: the persistent up-zeta tile kernel's bounded wait for a bulk
// copy that never comes.
int bn_debug_copy_wait(uint32_t polls, int32_t* err_word)
try {
    if (!err_word) return BN_EINVAL;
    char* buf = nullptr;
    const size_t abytes = 8192 * 4, tbytes = 2 * 8192 * 2;
    CK(cudaMalloc(&buf, abytes + tbytes + 16));
    float* A = reinterpret_cast<float*>(buf);
    uint16_t* rk = reinterpret_cast<uint16_t*>(buf + abytes);
    int* err = reinterpret_cast<int*>(buf + abytes + tbytes);
    cudaError_t e = cudaMemset(buf, 0, abytes + tbytes + 16);
    if (e == cudaSuccess) e = bn::launch_upzeta13p_withheld(A, rk, rk + 8192, err, polls, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int w = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&w, err, 4, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return BN_ECUDA;
    *err_word = w;
    return BN_OK;
} catch (...) {
    return exception_code();
}

// Test hook: the first failing index check of the BN_CHECK_BOUNDS build.
int bn_debug_bounds(int32_t* line, int32_t* unit)
try {
    if (!line || !unit) return BN_EINVAL;
    *line = -1;
    *unit = 0;
#ifdef BN_CHECK_BOUNDS
    CK(cudaDeviceSynchronize());
    const unsigned int v[4] = {bn::bounds_line_kernels(), bn::bounds_line_tile13(),
                               bn::bounds_line_levels(), bn::bounds_line_mega()};
    *line = 0;
    for (int k = 0; k < 4; ++k) {
        if (v[k] == ~0u) return BN_ECUDA;
        if (v[k] && *unit == 0) {
            *line = (int32_t)v[k];
            *unit = k + 1;
        }
    }
#endif
    return BN_OK;
} catch (...) {
    return exception_code();
}
#endif  // BN_TESTING

// ----------------------------------------------------------------- shards --

struct bn_shard {
    bn_ctx* ctx = nullptr;
    HostJob hj;
    Layout L{};
    char* mem = nullptr;                 // the shard's own device arrays
    int rank = 0, world = 1, nh = 0;
    bool prepared = false;
    // divided A (BN_SHARD_DIVIDE_A): the virtual job of the rank's slabs and
    // its arrays (folded scores, their reordered table, its A, the top
    // variables' slabs), in one more allocation
    Plan V{};
    char* slab = nullptr;
    size_t o_lbs = 0, o_tab = 0, o_A = 0, o_top = 0, slab_bytes = 0;
};

namespace {

size_t shard_header() { return 16; }     // the level word, padded

}  // namespace

int bn_shard_create(bn_ctx* c, const bn_job_desc* job, int32_t rank, int32_t world, int32_t flags,
                    bn_shard** out)
try {
    if (!c || !job || !out || world < 1 || world > 32 || (world & (world - 1)) || rank < 0 ||
        rank >= world || (flags & ~BN_SHARD_DIVIDE_A))
        return BN_EINVAL;
    *out = nullptr;
    bn_shard* sh = new bn_shard();
    sh->ctx = c;
    int rc = validate_and_plan(job, sh->hj);
    if (rc) { delete sh; return rc; }
    Plan& P = sh->hj.P;
    const bool rows = P.prec != 0 ? bn::rows_levels_fit(P) : bn::rows64_fit(P);
    int k = 0;
    while ((1 << k) < world) ++k;
    sh->nh = P.n - (P.prec == 0 ? 3 : 4);
    if (!rows || k > sh->nh) { delete sh; return BN_EINVAL; }
    P.frows = P.prec != 0 ? 1 : 0;       // step 3 by the level row kernels, one launch per level
    P.frc = 0;
    P.shard_k = k;
    P.shard_r = (uint32_t)rank;
    P.vsel = 0;
    for (int v = 0; v < P.n; ++v)
        if (v % world == rank) P.vsel |= 1u << v;
    sh->rank = rank;
    sh->world = world;
    if (!sh->hj.data_on_device && P.m > 0) {
        sh->hj.data_copy.assign(job->data, job->data + (size_t)P.m * P.n);
        sh->hj.data = sh->hj.data_copy.data();
    }
    if (flags & BN_SHARD_DIVIDE_A) {
        // the virtual job of nl = n - k low variables and nl + 2k tables
        // runs the 13-dimension up-zeta tiles (nl >= 14); no order prior
        const int nl = P.n - k;
        if (nl < 14 || P.hasq) { delete sh; return BN_EINVAL; }
        P.slab = 1;
        Plan& V = sh->V;
        V = P;
        V.n = nl;
        V.K = bn_num_families(nl, P.d);
        V.nodes = nl + 2 * k;
        V.hasq = 0;
        V.up13 = 1;
        V.slab = 0;
        V.shard_k = 0;
        V.shard_r = 0;
        const size_t es = P.prec == 0 ? 8 : 4;
        auto al256 = [](size_t x) { return (x + 255) & ~size_t(255); };
        size_t o = 0;
        sh->o_lbs = o;  o += al256((size_t)V.nodes * V.K * es);
        sh->o_tab = o;  o += al256((size_t)V.nodes * V.K * es);
        sh->o_A = o;    o += al256(((size_t)V.nodes << (nl - 1)) * es);
        sh->o_top = o;  o += al256(((size_t)k << nl) * es);
        sh->slab_bytes = o;
    }
    sh->L = make_layout(P, 0);
    if (sh->L.total + sh->slab_bytes > c->budget) { delete sh; return BN_ENOMEM; }
    if (cudaSetDevice(c->device) != cudaSuccess) { delete sh; return BN_ECUDA; }
    void* p = nullptr;
    rc = dev_alloc(c, &p, sh->L.total, nullptr);
    if (rc) { delete sh; return rc; }
    sh->mem = (char*)p;
    if (sh->slab_bytes) {
        rc = dev_alloc(c, &p, sh->slab_bytes, nullptr);
        if (rc) { cudaFree(sh->mem); delete sh; return rc; }
        sh->slab = (char*)p;
    }
    *out = sh;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_shard_prepare(bn_shard* sh, void* stream)
try {
    if (!sh) return BN_EINVAL;
    const HostJob& hj = sh->hj;
    const Plan& P = hj.P;
    const Layout& L = sh->L;
    cudaStream_t s = stream ? (cudaStream_t)stream : sh->ctx->stream;
    Bufs B{sh->mem, L};
    const uint8_t* data_dev = B.at<uint8_t>(L.data);
    if (P.m > 0) {
        if (hj.data_on_device) data_dev = hj.data;
        else CK(cudaMemcpyAsync(B.at<uint8_t>(L.data), hj.data, (size_t)P.m * P.n,
                                cudaMemcpyHostToDevice, s));
    }
    std::vector<double> lr(P.d + 1, 0.0), alpha(P.rows);
    for (size_t t = 0; t < hj.log_rho.size(); ++t) lr[t] = hj.log_rho[t];
    for (int r = 0; r < P.rows; ++r) alpha[r] = hj.ess / hj.Dvals[r];
    CK(cudaMemcpyAsync(B.at<char>(L.arity), hj.arity.data(), P.n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.log_rho), lr.data(), lr.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.Dvals), hj.Dvals.data(), hj.Dvals.size() * 8,
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.at<char>(L.alpha), alpha.data(), alpha.size() * 8, cudaMemcpyHostToDevice, s));
    int rc = upload_priors(hj, B, s);
    if (rc) return rc;
    int nl = 0;
    rc = enqueue_step1(hj, B, data_dev, s, &nl);
    if (rc) return rc;
    if (P.slab) {
        // the rank's slabs of A from the folded scores (no exchange)
        const Plan& V = sh->V;
        CK(bn::launch_fold_scores(P, V.n, V.K, P.shard_r, B.at<void>(L.lbs), sh->slab + sh->o_lbs, s));
        CK(bn::launch_upzeta(V, nullptr, sh->slab + sh->o_lbs, sh->slab + sh->o_tab,
                             B.at<uint16_t>(L.rk13), sh->slab + sh->o_A, s, nullptr, B.at<int>(L.err)));
        CK(bn::launch_top_slabs(V, P.shard_k, sh->slab + sh->o_A, sh->slab + sh->o_top, s));
    } else {
        rc = enqueue_upzeta(P, B, B.at<void>(L.lbs), s, &nl, nullptr);
        if (rc) return rc;
    }
    if (P.prec != 0) {                        // every rank starts both sweeps' level words
        int w[bn::kLevelWords];
        for (int q = 0; q < bn::kLevelWords; ++q) w[q] = bn::kLevelUnset;
        w[bn::kLevelMode] = bn::kLevelShift;
        const size_t N4 = ((size_t)1 << P.n) * 4;
        CK(cudaMemcpyAsync(B.at<char>(L.F) + N4, w, sizeof w, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(B.at<char>(L.Rc) + N4, w, sizeof w, cudaMemcpyHostToDevice, s));
    }
    sh->prepared = true;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_shard_level(bn_shard* sh, int32_t sweep, int32_t hl, void* stream)
try {
    if (!sh || !sh->prepared || sweep < 0 || sweep > 1 || hl < 0 || hl > sh->nh) return BN_EINVAL;
    const Layout& L = sh->L;
    cudaStream_t s = stream ? (cudaStream_t)stream : sh->ctx->stream;
    if (sh->slab)
        CK(bn::launch_rows_level(sh->hj.P, sweep, hl, sh->slab + sh->o_A, sh->mem + (sweep ? L.Rc : L.F), s,
                                 sh->slab + sh->o_top));
    else
        CK(bn::launch_rows_level(sh->hj.P, sweep, hl, sh->mem + L.A, sh->mem + (sweep ? L.Rc : L.F), s));
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_shard_exchange_bytes(const bn_shard* sh, int32_t hl, uint64_t* bytes)
try {
    if (!sh || !bytes || hl < 0 || hl > sh->nh) return BN_EINVAL;
    uint64_t mx = 0;
    for (int q = 0; q < sh->world; ++q)
        mx = std::max<uint64_t>(mx, (uint64_t)bn::shard_rows_count(sh->hj.P, (uint32_t)q, hl) * 64);
    *bytes = shard_header() + mx;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_shard_pack(bn_shard* sh, int32_t sweep, int32_t hl, void* buf_dev, void* stream)
try {
    if (!sh || !buf_dev || sweep < 0 || sweep > 1 || hl < 0 || hl > sh->nh) return BN_EINVAL;
    const Plan& P = sh->hj.P;
    cudaStream_t s = stream ? (cudaStream_t)stream : sh->ctx->stream;
    char* X = sh->mem + (sweep ? sh->L.Rc : sh->L.F);
    char* buf = (char*)buf_dev;
    if (P.prec != 0)
        CK(cudaMemcpyAsync(buf, X + ((size_t)1 << P.n) * 4 + (size_t)hl * 4, 4, cudaMemcpyDeviceToDevice, s));
    else
        CK(cudaMemsetAsync(buf, 0, 4, s));   // FP64 keeps no level words
    CK(bn::launch_level_rows(P, P.shard_r, hl, X, buf + shard_header(), 0, s));
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_shard_unpack(bn_shard* sh, int32_t sweep, int32_t hl, int32_t from, const void* buf_dev,
                    void* stream)
try {
    if (!sh || !buf_dev || sweep < 0 || sweep > 1 || hl < 0 || hl > sh->nh || from < 0 ||
        from >= sh->world)
        return BN_EINVAL;
    if (from == sh->rank) return BN_OK;
    const Plan& P = sh->hj.P;
    cudaStream_t s = stream ? (cudaStream_t)stream : sh->ctx->stream;
    char* X = sh->mem + (sweep ? sh->L.Rc : sh->L.F);
    const char* buf = (const char*)buf_dev;
    if (P.prec != 0)
        CK(bn::launch_word_max(reinterpret_cast<int*>(X + ((size_t)1 << P.n) * 4) + hl,
                               reinterpret_cast<const int*>(buf), s));
    CK(bn::launch_level_rows(P, (uint32_t)from, hl, X, const_cast<char*>(buf) + shard_header(), 1, s));
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_shard_finish(bn_shard* sh, double* post_dev, double* log_PD_dev, void* stream)
try {
    if (!sh || !sh->prepared || !post_dev) return BN_EINVAL;
    const Plan& P = sh->hj.P;
    const Layout& L = sh->L;
    cudaStream_t s = stream ? (cudaStream_t)stream : sh->ctx->stream;
    Bufs B{sh->mem, L};
    // divided A: no rank holds A_v over every tile, so the down-zeta runs
    // without its relevance cut (the same values; every output computed)
    CK(bn::launch_gamma_p1(P, B.at<void>(L.F), B.at<void>(L.Rc), B.at<uint16_t>(L.rk13),
                           B.at<void>(L.W), s, P.hasq ? B.at<void>(L.logq) : nullptr,
                           P.slab ? nullptr : B.at<void>(L.A)));
    CK(bn::launch_gamma_p2(P, B.at<void>(L.W), B.at<void>(L.Gam), s));
    CK(bn::launch_edges(P, B.at<double>(L.logB), B.at<double>(L.cmax), B.at<uint32_t>(L.masks),
                        B.at<void>(L.Gam), B.at<void>(L.F), B.at<int>(L.err),
                        B.at<unsigned long long>(L.eacc), post_dev,
                        log_PD_dev ? log_PD_dev : B.at<double>(L.logPD), s));
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_shard_bytes(const bn_shard* sh, uint64_t* bytes)
try {
    if (!sh || !bytes) return BN_EINVAL;
    *bytes = sh->L.total + sh->slab_bytes;
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_shard_destroy(bn_shard* sh)
try {
    if (!sh) return BN_EINVAL;
    cudaSetDevice(sh->ctx->device);
    if (sh->mem) cudaFree(sh->mem);          // waits for the shard's work in flight
    if (sh->slab) cudaFree(sh->slab);
    delete sh;
    return BN_OK;
} catch (...) {
    return exception_code();
}

// ---------------------------------------------------------------- serving --

int bn_submit(bn_ctx* c, const bn_job_desc* job, uint64_t* id)
try {
    if (!c || !id || !job) return BN_EINVAL;
    if (job->data_on_device) return BN_EINVAL;   // served jobs copy host inputs
    ServedJob sj;
    int rc = validate_and_plan(job, sj.hj);
    if (rc) return rc;
    const Plan& P = sj.hj.P;
    sj.hj.data_copy.assign(job->data ? job->data : (const uint8_t*)"",
                           job->data ? job->data + (size_t)P.m * P.n : (const uint8_t*)"");
    sj.hj.data = sj.hj.data_copy.data();
    sj.bytes = make_layout(P, 0).total;
    if (sj.bytes > c->budget) return BN_ENOMEM;
    std::lock_guard<std::mutex> g(c->mu);
    const uint64_t jid = c->next_id++;
    c->jobs.emplace(jid, std::move(sj));
    c->queue.push_back(jid);
    *id = jid;
    pump(c);
    return BN_OK;
} catch (...) {
    return exception_code();
}

int bn_poll(bn_ctx* c, uint64_t id, double* post, double* log_PD)
try {
    if (!c) return BN_EINVAL;
    std::lock_guard<std::mutex> g(c->mu);
    pump(c);
    auto it = c->jobs.find(id);
    if (it == c->jobs.end()) return BN_ENOTFOUND;
    ServedJob& sj = it->second;
    if (sj.state != Q_DONE) return BN_EAGAIN;
    const int rc = sj.rc;
    if (rc == BN_OK) {
        if (post) std::memcpy(post, sj.post.data(), sj.post.size() * 8);
        if (log_PD) *log_PD = sj.logPD;
    }
    c->last_stats = sj.stats;
    c->jobs.erase(it);
    return rc;
} catch (...) {
    return exception_code();
}

int bn_wait(bn_ctx* c, uint64_t id, double timeout_s, double* post, double* log_PD)
try {
    if (!c) return BN_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const int rc = bn_poll(c, id, post, log_PD);
        if (rc != BN_EAGAIN) return rc;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el >= timeout_s) return BN_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
} catch (...) {
    return exception_code();
}

int bn_cancel(bn_ctx* c, uint64_t id)
try {
    if (!c) return BN_EINVAL;
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->jobs.find(id);
    if (it == c->jobs.end()) return BN_ENOTFOUND;
    if (it->second.state != Q_QUEUED) return BN_EAGAIN;
    c->queue.erase(std::find(c->queue.begin(), c->queue.end(), id));
    it->second.state = Q_DONE;
    it->second.rc = BN_ECANCELED;
    return BN_OK;
} catch (...) {
    return exception_code();
}

}  // extern "C"

namespace {

// Retire finished jobs, then admit queued jobs (first fit) while a slot and
// enough of the memory budget are free.  Called with c->mu held.
void pump(bn_ctx* c)
{
    cudaSetDevice(c->device);
    for (size_t k = 0; k < c->slots.size(); ++k) {
        Slot& sl = c->slots[k];
        if (!sl.job) continue;
        if (cudaEventQuery(sl.done) == cudaErrorNotReady) continue;
        cudaGetLastError();
        ServedJob& sj = c->jobs[sl.job];
        const Plan& P = sj.hj.P;
        cudaStreamSynchronize(sl.stream);
        int err = 0;
        std::memcpy(&err, sl.pin + (size_t)P.n * P.n * 8 + 8, 4);
        sj.post.assign((double*)sl.pin, (double*)sl.pin + (size_t)P.n * P.n);
        std::memcpy(&sj.logPD, sl.pin + (size_t)P.n * P.n * 8, 8);
        fill_stats(P, sl.ev, sl.launches, &sj.stats);
        sj.rc = err ? err_word_status(err) : sj.rc;
        sj.state = Q_DONE;
        c->reserved -= sl.bytes;
        sl.bytes = 0;
        sl.dev = nullptr;
        sl.job = 0;
    }
    for (auto it = c->queue.begin(); it != c->queue.end();) {
        int free_slot = -1;
        for (size_t k = 0; k < c->slots.size(); ++k)
            if (!c->slots[k].job) { free_slot = (int)k; break; }
        if (free_slot < 0) break;
        ServedJob& sj = c->jobs[*it];
        if (c->reserved + sj.bytes > c->budget) { ++it; continue; }
        Slot& sl = c->slots[free_slot];
        const Plan& P = sj.hj.P;
        const size_t out_bytes = (size_t)P.n * P.n * 8 + 16;
        int rc = ensure_pin(&sl.pin, &sl.pin_bytes, out_bytes + small_bytes(P) + 64);
        void* dev = nullptr;
        if (!rc) rc = dev_alloc(c, &dev, sj.bytes, sl.stream);
        if (!rc) {
            Layout L = make_layout(P, 0);
            Bufs B{(char*)dev, L};
            rc = enqueue(sj.hj, B, B.at<double>(L.post), B.at<double>(L.logPD), sl.stream, &sl.ev,
                         &sl.launches, sl.pin + al(out_bytes), sl.pin_bytes - al(out_bytes), true,
                         &sl.side);
            if (!rc) {
                if (cudaMemcpyAsync(sl.pin, B.at<char>(L.post), (size_t)P.n * P.n * 8, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
                    cudaMemcpyAsync(sl.pin + (size_t)P.n * P.n * 8, B.at<char>(L.logPD), 8, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
                    cudaMemcpyAsync(sl.pin + (size_t)P.n * P.n * 8 + 8, B.at<char>(L.err), 4, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
                    cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
                    rc = BN_ECUDA;
            }
            cudaFreeAsync(dev, sl.stream);   // stream-ordered: after the job's work
        }
        if (rc) {
            sj.state = Q_DONE;
            sj.rc = rc;
            it = c->queue.erase(it);
            continue;
        }
        sl.job = *it;
        sl.bytes = sj.bytes;
        c->reserved += sj.bytes;
        sj.state = Q_RUNNING;
        sj.slot = free_slot;
        it = c->queue.erase(it);
    }
}

}  // namespace

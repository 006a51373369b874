// bn_kernels.cuh -- host-side launch interface of the device kernels.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace bn {

// ---------------------------------------------------------------------------
// Launch records.  Every kernel launch goes through launch_or_record: it
// launches, or, while a Recorder is installed on the calling host thread,
// appends the launch (kernel id, grid, block, dynamic shared memory and the
// arguments packed as the kernel's own parameter types) to the recorder.  A
// batch records each job's launch sequence once and runs it inside one
// persistent kernel (bn_mega.cu), which unpacks the arguments the same way.
// ---------------------------------------------------------------------------
// Bits of a job's device error word: 1 from the input check (a value not
// below its variable's arity), kErrDeviceTimeout from a kernel whose bounded
// wait for a bulk copy gave up.
constexpr int kErrDeviceTimeout = 2;

enum KernelId : int32_t {
    KID_NONE = 0,
    KID_PACK_PLANES, KID_CHECK_DATA, KID_LGAMMA_TABLE,
    KID_SCORES_BIN, KID_SCORES_BIN_HIST5, KID_SCORES_BIN_HIST6, KID_SCORES_BIN_HIST7,
    KID_SCORES_BIN_HIST8, KID_SCORES_BIN_HI1, KID_SCORES_BIN_HI2, KID_SCORES_BIN_HI3,
    KID_SCORES_BIN_HI4, KID_SCORES_CFG44, KID_SCORES_CFG, KID_SCORES_W42, KID_SCORES_W44,
    KID_SCORES_W84, KID_SCORES, KID_ADD_WEIGHTS, KID_APPLY_Q_D, KID_APPLY_Q_F,
    KID_ADD_FEATURE_D, KID_ADD_FEATURE_F, KID_NODE_MAX, KID_SHIFT_D, KID_SHIFT_F,
    KID_UPZETA_D, KID_UPZETA_F, KID_FWD_LEVEL_D, KID_FWD_LEVEL_F, KID_BWD_LEVEL_D,
    KID_BWD_LEVEL_F, KID_GAMMA_TABLE, KID_GAMMA_P1_D, KID_GAMMA_P1_F, KID_GAMMA_P2_D,
    KID_GAMMA_P2_F, KID_GAMMA_P2S_D, KID_GAMMA_P2S_F, KID_EDGES_ZERO, KID_EDGES_ACC_D,
    KID_EDGES_ACC_F, KID_EDGES_FIN_D, KID_EDGES_FIN_F, KID_RANK13, KID_REORDER_D,
    KID_REORDER_F, KID_COLB8, KID_COLB4, KID_COLB2, KID_COLW_D, KID_COLW_F, KID_COLS_D,
    KID_COLS_F, KID_UP13_D, KID_UP13_F_TLO, KID_UP13_F, KID_G13_D_Q, KID_G13_D, KID_G13_F_Q,
    KID_G13_F, KID_FROWS_D, KID_FROWS_F_TLO, KID_FROWS_F, KID_BROWS_D, KID_BROWS_F_TLO,
    KID_BROWS_F, KID_COLB4_D, KID_COLB2_D, KID_COLB1_D, KID_COLB1, KID_COUNT
};

// Arguments as one trivially copyable structure whose members have the
// kernel's parameter types, in order (the same layout on host and device).
template <typename... P> struct ArgPack {};
template <typename H, typename... R> struct ArgPack<H, R...> {
    H h;
    ArgPack<R...> r;
};
template <typename... P> inline ArgPack<P...> make_pack(P... a);
template <> inline ArgPack<> make_pack<>() { return {}; }
template <typename H, typename... R> inline ArgPack<H, R...> make_pack(H h, R... r)
{
    return ArgPack<H, R...>{h, make_pack<R...>(r...)};
}

constexpr int kRecArgBytes = 224;
struct LaunchRec {
    int32_t kid;
    uint32_t gx, gy, gz;          // grid
    uint32_t block, smem;
    uint32_t pad[2];
    alignas(16) unsigned char args[kRecArgBytes];
};
static_assert(sizeof(LaunchRec) == 256, "launch record size");

// LaunchRec::pad[0] flag: the kernel loops grid-stride over blockIdx.x, so
// any grid width covers its work; the persistent form may run it narrower.
constexpr uint32_t kRecStrideX = 2u;

struct Recorder {
    LaunchRec* recs = nullptr;    // host array owned by the caller
    int cap = 0, count = 0;
    bool overflow = false;
};
extern thread_local Recorder* g_recorder;
inline bool recording() { return g_recorder != nullptr; }

template <typename... P, typename... A>
inline cudaError_t launch_or_record(int kid, void (*k)(P...), dim3 grid, unsigned block,
                                    size_t smem, cudaStream_t s, A... a)
{
    static_assert(sizeof...(P) == sizeof...(A), "argument count");
    if (Recorder* r = g_recorder) {
        using Pk = ArgPack<P...>;
        static_assert(sizeof(Pk) <= kRecArgBytes, "launch arguments too large for a record");
        if (r->count >= r->cap) {
            r->overflow = true;
            return cudaSuccess;
        }
        LaunchRec& x = r->recs[r->count++];
        x = LaunchRec{};
        x.kid = kid;
        x.gx = grid.x;
        x.gy = grid.y;
        x.gz = grid.z;
        x.block = block;
        x.smem = (uint32_t)smem;
        const Pk pk = make_pack<P...>(static_cast<P>(a)...);
        std::memcpy(x.args, &pk, sizeof(Pk));
        return cudaSuccess;
    }
    k<<<grid, block, smem, s>>>(static_cast<P>(a)...);
    return cudaGetLastError();
}

// Threads per block a launch uses: `normal`, or 256 while recording (the
// persistent kernel runs every record with 256 threads; kernels launched
// with other sizes are written for any block size).
inline unsigned rec_block(unsigned normal) { return recording() ? 256u : normal; }

// The persistent batch kernel (bn_mega.cu).  persistent_runs: whether the
// instance for precision prec (1 FP32, 0 FP64) runs kernel kid.
// persistent_blocks: blocks that fit the GPU at once with `smem` dynamic
// shared memory each.  launch_persistent zeroes ctl (ctl_bytes: the next-item
// counter, status, abort flag, a spare word and one done-counter per record)
// and runs the items; a wait gives up after `cap` polls.
bool persistent_runs(int prec, int kid);
cudaError_t set_persistent_attributes();
int persistent_blocks(int prec, size_t smem);
cudaError_t launch_persistent(int prec, const LaunchRec* recs, const int4* items, int nitems,
                              const int2* deps, const int* need, int* ctl, size_t ctl_bytes,
                              int blocks, size_t smem, uint64_t cap, cudaStream_t s);

// Byte copies between device regions (one block per segment).
struct CopySeg {
    const unsigned char* src;
    unsigned char* dst;
    uint64_t bytes;
};
cudaError_t launch_copy_segments(const CopySeg* segs, int nseg, cudaStream_t s);

// Shapes of one job, computed on the host.
struct Plan {
    int n, d, m;          // d already clamped to n-1
    int64_t K;            // families per node
    int W;                // 64-bit words per bit plane (ceil(m/64), >= 1)
    int rmax;             // max arity
    int rows;             // rows of the lgamma table
    int b_up;             // low dims done in shared memory by the up-zeta tile
    int b_g;              // low dims of the Gamma phase-1 tile
    int hc_g;             // high dims per Gamma phase-2 chunk
    uint32_t nlow_g;      // subsets of b_g dims with at most d elements
    int wb;               // in-warp bits of the F / R' tiles
    int prec;             // 0 = FP64, 1 = FP32
    int allbin = 0;       // every variable has arity 2
    int fxs = 40;         // fixed-point shift of the lgamma table (fixed_shift)
    int hasq = 0;         // an order prior q_i(S) by |S| is given (Eq. 4, 7, 12)
    int hasw = 0;         // per-family log weights are given (Eq. 4)
    // Schedule (set by the planner, changed by the batch autotuner):
    int up13 = 0;         // step 2 by the 13-dimension tiles (n >= 14)
    int g13 = 0;          // step 4 phase 1 by the 13-dimension tiles (n >= 14)
    int frows = 0;        // FP32 step 3 by the 16-subset row kernels
    int scfg = 0;         // step 1 by one lane per parent configuration (non-binary data)
    int frc = 0;          // FP32 step 3 of a batch group by the persistent cluster kernel
    // Batch groups: nj jobs with equal plans, their arrays js bytes apart;
    // the launches of steps 2-5 cover all of them (gridDim.y = nj).
    int nj = 1;
    size_t js = 0;
    // A job split over 2^shard_k ranks by its top shard_k variables (the
    // rank's bits shard_r): the step-3 row kernels compute only the tiles of
    // this rank's sub-lattice; steps 4-5 only the endpoints v whose bit is
    // set in vsel (every endpoint by default).
    int shard_k = 0;
    uint32_t shard_r = 0;
    uint32_t vsel = 0xffffffffu;
    // Step 2 over `nodes` score tables that share the n-1-bit index space of
    // a node (0: the n nodes of the job; a split job's divided A has more).
    int nodes = 0;
    // A split job whose ranks hold only their slabs of A: step 3 reads the
    // low n - shard_k nodes' slabs (top bits = the rank's) and, for each top
    // variable, a slab over the low variables.
    int slab = 0;
    // A in a managed allocation outside the layout: its first part resident
    // in device memory, the rest in host memory that the GPU reads and
    // writes directly (a job whose arrays exceed the device budget).
    int spill = 0;
    // Step 4 in groups of vgroup endpoints (0: all at once), its scratch W
    // sized for one group (a spilled job keeps more of A on the device).
    int vgroup = 0;
};
inline int up_nodes(const Plan& P) { return P.nodes ? P.nodes : P.n; }

// Host check of m x n row-major data: every value below its variable's
// arity.  Column maxima first (a loop the compiler vectorises), then one
// comparison per variable.
inline bool data_below_arity(const uint8_t* data, int m, int n, const uint8_t* arity)
{
    uint8_t mx[32] = {0};
    const uint8_t* row = data;
    for (int s = 0; s < m; ++s, row += n)
        for (int v = 0; v < n; ++v) mx[v] = row[v] > mx[v] ? row[v] : mx[v];
    for (int v = 0; v < n; ++v)
        if (m > 0 && mx[v] >= arity[v]) return false;
    return true;
}

// Step 1.  A batch group passes nj jobs js bytes apart (mj: each job's own
// sample count, at the same stride); a single job leaves the defaults.
cudaError_t launch_pack_planes(const uint8_t* data, int n, int m, int rmax, int W,
                               uint64_t* planes, cudaStream_t s, const int* mj = nullptr,
                               int nj = 1, size_t js = 0);
cudaError_t launch_check_data(const uint8_t* data, const uint8_t* arity, int n, int m,
                              int* err, cudaStream_t s);
// The lgamma table T (rows x (m+1) int64) holds lgamma(alpha + N) - lgamma(alpha)
// in fixed point, scaled by 2^fxs (fixed_shift); the scores sum it exactly.
// A batch group passes fxj (each job's scale 2^S and 2^-S) and mj (each
// job's m) at the job stride; fxs then is not used.
cudaError_t launch_lgamma_table(const double* alpha, int rows, int m, int fxs, void* T,
                                cudaStream_t s, int nj = 1, size_t js = 0,
                                const double* fxj = nullptr, const int* mj = nullptr);
// The fixed-point shift S of the lgamma table: every partial sum of one
// family's score, at most sum_j |T_q(N_j)| + sum_jk |T_qr(N_jk)| <= 2 m L
// with L = max |ln(alpha + t)| over the rows (alpha = 1 included) and
// 0 <= t < m, stays below 2^61 after scaling by 2^S; each term's rounding
// error is at most 2^-(S+1).
int fixed_shift(int m, double ess, const double* Dvals, int rows);
cudaError_t launch_scores(const Plan& P, const uint8_t* arity, const uint64_t* planes,
                          const double* Dvals, const void* T, const double* log_rho,
                          int64_t x_begin, int64_t x_count, uint32_t* masks,
                          uint32_t* cmasks, double* logB, int64_t* debug_counts,
                          cudaStream_t s, const double* fxj = nullptr);
// Step 1 has the lane-per-configuration alternative (Plan::scfg): data not
// all binary, at most 8 parents and arity at most 8.
bool scores_cfg_fits(const Plan& P);
// Kernels one launch_scores call over all n * K families starts.
int scores_launches(const Plan& P);
// Priors beyond the defaults and single features (Eqs. 4-9):
// log B += w (n*K doubles, natural log); A_i(S) += lq[i*n + |S|] (lq in the
// working precision and log base); out = lbs + lf (shifted scores times a
// feature, working precision).
cudaError_t launch_add_weights(const Plan& P, double* logB, const double* w, cudaStream_t s);
cudaError_t launch_apply_q(const Plan& P, const void* lq, void* A, cudaStream_t s);
cudaError_t launch_add_feature(const Plan& P, const void* lbs, const void* lf, void* out,
                               cudaStream_t s);
cudaError_t launch_node_max(const Plan& P, const double* logB, double* cmax, cudaStream_t s);
cudaError_t launch_shift_scores(const Plan& P, const double* logB, const double* cmax,
                                void* lbs, cudaStream_t s);
// Step 2.  n >= 14 uses the 13-dimension register tiles and needs `tab`
// (n*K values, the scores reordered by high and low parts); smaller n use
// one shared-memory tile per node slice and ignore `tab`.
// `rk13` points at the two 8192-entry uint16 subset-rank tables (rank, then
// inverse) of the 13-dimension tiles, filled by launch_rank13_tables.  `err`
// (the job's error word) lets an FP32 single job use the persistent tile
// kernel, which reports a bulk copy that never landed there.
cudaError_t launch_upzeta(const Plan& P, const uint32_t* cmasks, const void* lbs, void* tab,
                          const uint16_t* rk13, void* A, cudaStream_t s, cudaEvent_t sums_done = nullptr,
                          int* err = nullptr);
// Step 3 in FP32 with one thread per 16-subset tile (bn_levels.cu).
bool rows_levels_fit(const Plan& P);      // FP32 and 5 <= n < 32
bool rows64_fit(const Plan& P);           // FP64 and 4 <= n < 31: 8-subset row tiles
cudaError_t launch_forward_rows(const Plan& P, const void* A, void* F, cudaStream_t s, int* launches);
// One level of a shard's sweep (sweep 0 F, 1 R'; the row kernels, with the
// plan's shard_k / shard_r): nothing when the shard has no tile there.
cudaError_t launch_rows_level(const Plan& P, int sweep, int hl, const void* A, void* X, cudaStream_t s,
                              const void* Atop = nullptr);
// Tiles (rows of 16 FP32 or 8 FP64 values) of level hl in the sub-lattice
// whose top shard_k tile bits are r; dir 0 copies those rows of X to the
// contiguous buf, dir 1 back.
uint32_t shard_rows_count(const Plan& P, uint32_t r, int hl);
#ifdef BN_CHECK_BOUNDS
// The first failing index check of each translation unit (0: none), cleared
// by the read (bn_device.cuh).
unsigned int bounds_line_kernels();
unsigned int bounds_line_tile13();
unsigned int bounds_line_levels();
unsigned int bounds_line_mega();
#endif
cudaError_t launch_word_max(int* word, const int* other, cudaStream_t s);
cudaError_t launch_explog_check(const double* x, int64_t count, double* out, cudaStream_t s);
// Launches of step 4 (phase 1, the FP32 offset table, the phase-2 kernels).
int gamma_launches(const Plan& P);
// A split job's divided A: the folded score tables of the rank's virtual job
// (nl low variables, nl + 2 (n - nl) tables of Kv families) and the top
// variables' slabs from its A (bn_levels.cu).
cudaError_t launch_fold_scores(const Plan& P, int nl, int64_t Kv, uint32_t r, const void* lbs, void* out,
                               cudaStream_t s);
cudaError_t launch_top_slabs(const Plan& V, int k, const void* Av, void* Atop, cudaStream_t s);
cudaError_t launch_level_rows(const Plan& P, uint32_t r, int hl, void* X, void* buf, int dir,
                              cudaStream_t s);
// F and R' of every job of a batch group in one persistent launch of
// thread-block clusters (FP32, rows_levels_fit); one launch.
cudaError_t launch_rows_cluster(const Plan& P, const void* A, void* F, void* Rc, cudaStream_t s,
                                int* launches);
cudaError_t launch_backward_rows(const Plan& P, const void* A, void* Rc, cudaStream_t s,
                                 int* launches);
cudaError_t launch_forward(const Plan& P, const void* A, void* F, cudaStream_t s, int* launches);
cudaError_t launch_backward(const Plan& P, const void* A, void* Rc, cudaStream_t s,
                            int* launches);
// Step 4 for every endpoint v in one launch per phase (gridDim.z = n): W
// holds n slices of 2^(n-1-b_g) * nlow_g values, Gam the n * K outputs.
// lq (may be null): the order prior's log q_v(S) by |S| (Eq. 12), n*n values
// in the working precision and log base, added to s_v(S).  A (may be null):
// the step-2 output, which gives the 13-dimension tiles their relevance cut.
cudaError_t launch_gamma_p1(const Plan& P, const void* F, const void* Rc, const uint16_t* rk13,
                            void* W, cudaStream_t s, const void* lq = nullptr,
                            const void* A = nullptr);
cudaError_t launch_gamma_p2(const Plan& P, const void* W, void* Gam, cudaStream_t s);
// FP32: the per-endpoint offsets of the down-zeta input (one small launch,
// made by launch_gamma_p1 itself; stored after the level words of Rc).
cudaError_t launch_gamma_table(const Plan& P, const void* F, const void* Rc, cudaStream_t s);
// Step 5 (three launches); acc: n * (n + 1) scratch words.
cudaError_t launch_edges(const Plan& P, const double* logB, const double* cmax,
                         const uint32_t* masks, const void* Gam, const void* F,
                         const int* err, unsigned long long* acc, double* post, double* log_PD,
                         cudaStream_t s);

size_t upzeta_smem_bytes(const Plan& P);
// bn_tile13.cu
cudaError_t launch_reorder_up(const Plan& P, const void* lbs, void* tab, cudaStream_t s);
cudaError_t launch_rank13_tables(const Plan& P, uint16_t* rank13, uint16_t* unrank13, cudaStream_t s);
cudaError_t launch_upzeta13(const Plan& P, const void* tab, const uint16_t* unrank13, void* A,
                            cudaStream_t s, cudaEvent_t sums_done = nullptr, int* err = nullptr);
cudaError_t launch_upzeta13p_withheld(float* A, uint16_t* rank13, uint16_t* unrank13, int* err,
                                      uint32_t polls, cudaStream_t s);
cudaError_t launch_gamma13_p1(const Plan& P, const void* F, const void* Rc,
                              const uint16_t* rank13, void* W, cudaStream_t s,
                              const void* lq = nullptr, const void* A = nullptr);
constexpr size_t kRank13Bytes = 2 * 8192 * sizeof(uint16_t);
size_t upzeta13_smem_bytes(const Plan& P);
size_t gamma13_smem_bytes(const Plan& P);
cudaError_t set_tile13_attributes();
bool tile13_up_fits(const Plan& P);   // n >= 14 and the column kernel's shared memory fits
inline bool tile13_gamma_fits(const Plan& P) { return P.n >= 14; }

// The schedule a plan runs: which kernels do steps 2, 3 and 4.  Every choice
// that fits computes the same values up to rounding.
inline bool use_tile13_up(const Plan& P) { return P.up13 != 0; }
inline bool use_tile13_gamma(const Plan& P) { return P.g13 != 0; }
inline bool use_rows_levels(const Plan& P) { return P.frows != 0; }
inline bool needs_rank13(const Plan& P) { return P.up13 || P.g13; }
// A in tile-level row order (see bn_device.cuh): FP32 with the 13-dimension
// up-zeta tiles and the step-3 row kernels (not the cluster kernel).
inline bool use_tlo(const Plan& P) { return P.prec != 0 && P.up13 && P.frows && !P.frc; }
// The default schedule: every specialised kernel that fits.
inline void default_schedule(Plan& P)
{
    // lane per configuration where the 4-parent, arity-4 instance applies
    P.scfg = scores_cfg_fits(P) && P.d <= 4 && P.rmax <= 4;
    P.up13 = tile13_up_fits(P);
    P.g13 = tile13_gamma_fits(P);
    P.frows = rows_levels_fit(P);
}
size_t gamma_p1_smem_bytes(const Plan& P);
size_t gamma_p2_smem_bytes(const Plan& P);
cudaError_t set_kernel_attributes();

// Allow a kernel the largest dynamic shared memory the device gives one block
// next to the kernel's own static shared memory.
template <typename K> inline cudaError_t allow_max_dynamic_smem(K kernel)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

}  // namespace bn

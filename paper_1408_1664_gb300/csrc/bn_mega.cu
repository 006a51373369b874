// bn_mega.cu -- a whole batch of jobs in one persistent launch.
//
// A batch records, on the host, the launch sequence of every group of jobs
// (steps 1-5 of Algorithm 1 with the same launchers and kernels as the graph
// form; see launch_or_record in bn_kernels.cuh).  The persistent kernel runs
// all of them from one device work queue.  A work item is a range of blocks
// of one launch record; the items of all groups are queued in order of the
// record's depth in its group's sequence, so the first steps of every group
// come first.  A block holds one item and has already claimed the next (one
// atomic, issued while the current item runs); it waits until every record
// the item's record depends on has completed (the record before it in its
// group's sequence; an F level and an R' level of equal depth are
// independent of each other), runs the item's blocks, and counts the item
// done.  Every item an item waits on sits earlier in the queue, and a block
// runs the items it claimed in claim order, so by induction over the queue
// every item runs and every wait ends; even so each wait is bounded: after
// `cap` polls the block records BN_EDEVICE_TIMEOUT in the status word, raises
// the abort flag every block checks, and the kernel returns.
//
// The kernels are compiled here a second time, as device functions: this
// file includes the three kernel sources with __global__ turned into
// __device__ __noinline__ and blockIdx / gridDim redirected to the virtual
// block being run.  Values one block writes are read by other blocks within
// the same launch.  A producer's writes are ordered before its count by a
// fence; the consumer's first thread reads the count with ld.acquire.gpu and
// the block meets at a barrier before any thread loads, so by the PTX memory
// model every thread's ordinary loads (through L1) see the writes.  The
// non-coherent read-only path is outside that guarantee, so the kernels'
// __restrict__ qualifiers (which allow it) are dropped here and their
// explicit cache hints are read as L2 loads.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

#include "bnedge.h"

// The virtual block of the launch record a block is running.
__shared__ uint3 bn_mega_bidx;
__shared__ uint3 bn_mega_gdim;

#pragma push_macro("__global__")
#pragma push_macro("__launch_bounds__")
#undef __global__
#define __global__ static __device__ __noinline__
#undef __launch_bounds__
#define __launch_bounds__(...)
#define blockIdx bn_mega_bidx
#define gridDim bn_mega_gdim
#define __restrict__
#define __ldcs(p) __ldcg(p)
#define __ldg(p) __ldcg(p)
#define BN_MEGA 1
#include "bn_kernels.cu"
#include "bn_tile13.cu"
#include "bn_levels.cu"
#undef BN_MEGA
#undef __ldg
#undef __ldcs
#undef __restrict__
#undef gridDim
#undef blockIdx
#pragma pop_macro("__launch_bounds__")
#pragma pop_macro("__global__")

namespace bn {
namespace {

// Call f with the arguments packed in p (their own types, in order).
template <typename F, typename... Done>
__device__ __forceinline__ void call_pack(F f, const ArgPack<>&, Done... d)
{
    f(d...);
}
template <typename F, typename H, typename... R, typename... Done>
__device__ __forceinline__ void call_pack(F f, const ArgPack<H, R...>& p, Done... d)
{
    call_pack(f, p.r, d..., p.h);
}
template <typename... P>
__device__ __forceinline__ void run(void (*f)(P...), const unsigned char* a)
{
    call_pack(f, *reinterpret_cast<const ArgPack<P...>*>(a));
}

// One virtual block of launch record `kid`.  PREC 1: FP32 kernels and those
// of either precision; PREC 0: FP64 kernels and those of either precision
// (two instances, so that the FP32 one is not held to the FP64 tiles'
// register count).  The binary score kernels for families of 5-8 parents
// are left out: the static shared memory of every kernel called here adds up
// in the persistent kernel, and theirs (38 KB) would cost it its second
// block per SM; batches that need them run as a graph of launches.  Returns
// false for a kernel this instance does not run.
template <int PREC>
__device__ __forceinline__ bool dispatch(int kid, const unsigned char* a)
{
    switch (kid) {
    case KID_PACK_PLANES: run(k_pack_planes, a); return true;
    case KID_CHECK_DATA: run(k_check_data, a); return true;
    case KID_LGAMMA_TABLE: run(k_lgamma_table, a); return true;
    case KID_SCORES_BIN: run(k_scores_bin, a); return true;
    case KID_SCORES_CFG44: run(k_scores_cfg<4, 4>, a); return true;
    case KID_SCORES_CFG: run(k_scores_cfg<SC_MP, SC_MR>, a); return true;
    case KID_SCORES_W42: run(k_scores_w<4, 2>, a); return true;
    case KID_SCORES_W44: run(k_scores_w<4, 4>, a); return true;
    case KID_SCORES_W84: run(k_scores_w<8, 4>, a); return true;
    case KID_SCORES: run(k_scores, a); return true;
    case KID_NODE_MAX: run(k_node_max, a); return true;
    case KID_EDGES_ZERO: run(k_edges_zero, a); return true;
    case KID_RANK13: run(k_rank13_tables, a); return true;
    default: break;
    }
    if constexpr (PREC == 1) {
        switch (kid) {
        case KID_SHIFT_F: run(k_shift_scores<float>, a); return true;
        case KID_UPZETA_F: run(k_upzeta<float>, a); return true;
        case KID_FWD_LEVEL_F: run(k_forward_level<float>, a); return true;
        case KID_BWD_LEVEL_F: run(k_backward_level<float>, a); return true;
        case KID_GAMMA_TABLE: run(k_gamma_table, a); return true;
        case KID_GAMMA_P1_F: run(k_gamma_p1<float>, a); return true;
        case KID_GAMMA_P2_F: run(k_gamma_p2<float>, a); return true;
        case KID_GAMMA_P2S_F: run(k_gamma_p2s<float>, a); return true;
        case KID_EDGES_ACC_F: run(k_edges_acc<float>, a); return true;
        case KID_EDGES_FIN_F: run(k_edges_fin<float>, a); return true;
        case KID_REORDER_F: run(k_reorder_up<float>, a); return true;
        case KID_COLB8: run(k_upzeta13_colb<float, 8>, a); return true;
        case KID_COLB4: run(k_upzeta13_colb<float, 4>, a); return true;
        case KID_COLB2: run(k_upzeta13_colb<float, 2>, a); return true;
        case KID_COLB1: run(k_upzeta13_colb<float, 1>, a); return true;
        case KID_COLW_F: run(k_upzeta13_colw<float>, a); return true;
        case KID_COLS_F: run(k_upzeta13_cols<float>, a); return true;
        case KID_UP13_F_TLO: run(k_upzeta13<float, true>, a); return true;
        case KID_UP13_F: run(k_upzeta13<float, false>, a); return true;
        case KID_G13_F: run(k_gamma13_p1<float, false>, a); return true;
        case KID_FROWS_F_TLO: run(k_forward_rows<float, true>, a); return true;
        case KID_FROWS_F: run(k_forward_rows<float, false>, a); return true;
        case KID_BROWS_F_TLO: run(k_backward_rows<float, true>, a); return true;
        case KID_BROWS_F: run(k_backward_rows<float, false>, a); return true;
        default: return false;
        }
    } else {
        switch (kid) {
        case KID_SHIFT_D: run(k_shift_scores<double>, a); return true;
        case KID_UPZETA_D: run(k_upzeta<double>, a); return true;
        case KID_FWD_LEVEL_D: run(k_forward_level<double>, a); return true;
        case KID_BWD_LEVEL_D: run(k_backward_level<double>, a); return true;
        case KID_GAMMA_P1_D: run(k_gamma_p1<double>, a); return true;
        case KID_GAMMA_P2_D: run(k_gamma_p2<double>, a); return true;
        case KID_GAMMA_P2S_D: run(k_gamma_p2s<double>, a); return true;
        case KID_EDGES_ACC_D: run(k_edges_acc<double>, a); return true;
        case KID_EDGES_FIN_D: run(k_edges_fin<double>, a); return true;
        case KID_REORDER_D: run(k_reorder_up<double>, a); return true;
        case KID_COLW_D: run(k_upzeta13_colw<double>, a); return true;
        case KID_COLB4_D: run(k_upzeta13_colb<double, 4>, a); return true;
        case KID_COLB2_D: run(k_upzeta13_colb<double, 2>, a); return true;
        case KID_COLB1_D: run(k_upzeta13_colb<double, 1>, a); return true;
        case KID_COLS_D: run(k_upzeta13_cols<double>, a); return true;
        case KID_UP13_D: run(k_upzeta13<double, false>, a); return true;
        case KID_G13_D: run(k_gamma13_p1<double, false>, a); return true;
        case KID_FROWS_D: run(k_forward_rows<double, false>, a); return true;
        case KID_BROWS_D: run(k_backward_rows<double, false>, a); return true;
        default: return false;
        }
    }
}

// Barrier 1 over the block's 256 threads: the kernels' own __syncthreads use
// barrier 0, so the two never pair up.
__device__ __forceinline__ void bar1()
{
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

}  // namespace

// Spin until *p reaches `need` (acquire), polling at most `cap` times or
// until the abort flag rises.  Returns false when it gave up.
__device__ __forceinline__ bool wait_count(const int* p, int need, const int* abort, uint64_t cap)
{
    for (uint64_t k = 0;; ++k) {
        int v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= need) return true;
        if (k >= cap) return false;
        int ab;
        asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(ab) : "l"(abort) : "memory");
        if (ab) return false;
        __nanosleep(k < 64 ? 32 : 256);
    }
}

// The persistent kernel.  items[i] = {record, first block, last block + 1,
// 0} in queue order; deps[r] = the (up to two, -1 = none) records record r
// waits for; need[r] = its item count; ctl = {next item, status, abort flag,
// 0} followed by one done-counter per record, all zero at launch.
template <int PREC>
__global__ void __launch_bounds__(256, PREC == 1 ? 2 : 1)
k_batch_persistent(const LaunchRec* __restrict__ recs, const int4* __restrict__ items, int nitems,
                   const int2* __restrict__ deps, const int* __restrict__ need, int* __restrict__ ctl,
                   uint64_t cap)
{
    __shared__ int it_s, next_s, go_s;
    __shared__ __align__(16) LaunchRec rec_s;
    int* next = ctl;
    int* status = ctl + 1;
    int* abort = ctl + 2;
    int* done = ctl + 4;
    // A block holds its current item and has claimed the next one: every
    // item claimed earlier than another runs first in its block, so by
    // induction over the queue every item runs and every wait ends.
    if (threadIdx.x == 0) it_s = atomicAdd(next, 1);
    __syncthreads();
    for (;;) {
        const int it = it_s;
        if (it >= nitems) break;
        const int4 item = __ldcg(items + it);
        const int r = item.x;
        if (threadIdx.x == 0) {
            next_s = atomicAdd(next, 1);            // the next item, claimed now
            const int2 dp = __ldcg(deps + r);
            bool ok = true;
            if (dp.x >= 0) ok = wait_count(done + dp.x, __ldcg(need + dp.x), abort, cap);
            if (ok && dp.y >= 0) ok = wait_count(done + dp.y, __ldcg(need + dp.y), abort, cap);
            if (!ok) {
                atomicCAS(status, 0, (int)BN_EDEVICE_TIMEOUT);
                atomicExch(abort, 1);
            }
            go_s = ok;
        }
        if (threadIdx.x < sizeof(LaunchRec) / 16)
            reinterpret_cast<int4*>(&rec_s)[threadIdx.x] =
                __ldcg(reinterpret_cast<const int4*>(recs + r) + threadIdx.x);
        __syncthreads();
        if (!go_s) break;
        const int kid = rec_s.kid;
        const unsigned gx = rec_s.gx, gy = rec_s.gy, gz = rec_s.gz;
        const unsigned block = rec_s.block;
        for (int v = item.y; v < item.z; ++v) {
            if (threadIdx.x == 0) {
                bn_mega_bidx = make_uint3((unsigned)v % gx, (((unsigned)v / gx) % gy), (unsigned)v / (gx * gy));
                bn_mega_gdim = make_uint3(gx, gy, gz);
            }
            bar1();
            if (threadIdx.x < block && !dispatch<PREC>(kid, rec_s.args)) go_s = 0;
            bar1();
        }
        // the item's writes are done (barrier), then visible GPU-wide (fence)
        // before it counts
        if (threadIdx.x == 0) {
            if (!go_s) atomicCAS(status, 0, (int)BN_EINVAL);
            __threadfence();
            atomicAdd(done + r, 1);
            it_s = next_s;
        }
        __syncthreads();
    }
}

template __global__ void k_batch_persistent<0>(const LaunchRec*, const int4*, int, const int2*, const int*,
                                               int*, uint64_t);
template __global__ void k_batch_persistent<1>(const LaunchRec*, const int4*, int, const int2*, const int*,
                                               int*, uint64_t);

#ifdef BN_CHECK_BOUNDS
BN_BOUNDS_READER(bounds_line_mega)
#endif

bool persistent_runs(int prec, int kid)
{
    switch (kid) {
    case KID_PACK_PLANES: case KID_CHECK_DATA: case KID_LGAMMA_TABLE: case KID_SCORES_BIN:
    case KID_SCORES_CFG44: case KID_SCORES_CFG:
    case KID_SCORES_W42: case KID_SCORES_W44: case KID_SCORES_W84: case KID_SCORES:
    case KID_NODE_MAX: case KID_EDGES_ZERO: case KID_RANK13:
        return true;
    case KID_SHIFT_F: case KID_UPZETA_F: case KID_FWD_LEVEL_F: case KID_BWD_LEVEL_F:
    case KID_GAMMA_TABLE: case KID_GAMMA_P1_F: case KID_GAMMA_P2_F: case KID_GAMMA_P2S_F:
    case KID_EDGES_ACC_F: case KID_EDGES_FIN_F: case KID_REORDER_F: case KID_COLB8: case KID_COLB4:
    case KID_COLB2: case KID_COLB1: case KID_COLW_F: case KID_COLS_F: case KID_UP13_F_TLO: case KID_UP13_F:
    case KID_G13_F: case KID_FROWS_F_TLO: case KID_FROWS_F: case KID_BROWS_F_TLO: case KID_BROWS_F:
        return prec == 1;
    case KID_SHIFT_D: case KID_UPZETA_D: case KID_FWD_LEVEL_D: case KID_BWD_LEVEL_D:
    case KID_GAMMA_P1_D: case KID_GAMMA_P2_D: case KID_GAMMA_P2S_D: case KID_EDGES_ACC_D:
    case KID_EDGES_FIN_D: case KID_REORDER_D: case KID_COLW_D: case KID_COLS_D: case KID_UP13_D:
    case KID_COLB4_D: case KID_COLB2_D: case KID_COLB1_D:
    case KID_G13_D: case KID_FROWS_D: case KID_BROWS_D:
        return prec == 0;
    default:
        return false;
    }
}

cudaError_t set_persistent_attributes()
{
    cudaError_t e = allow_max_dynamic_smem(k_batch_persistent<0>);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_batch_persistent<1>);
    return e;
}

int persistent_blocks(int prec, size_t smem)
{
    int per_sm = 0, dev = 0, sms = 0;
    const cudaError_t e =
        prec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent<1>, 256, smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent<0>, 256, smem);
    if (e != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

cudaError_t launch_persistent(int prec, const LaunchRec* recs, const int4* items, int nitems,
                              const int2* deps, const int* need, int* ctl, size_t ctl_bytes,
                              int blocks, size_t smem, uint64_t cap, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(ctl, 0, ctl_bytes, s);
    if (e != cudaSuccess) return e;
    if (prec)
        k_batch_persistent<1><<<blocks, 256, smem, s>>>(recs, items, nitems, deps, need, ctl, cap);
    else
        k_batch_persistent<0><<<blocks, 256, smem, s>>>(recs, items, nitems, deps, need, ctl, cap);
    return cudaGetLastError();
}

}  // namespace bn

// Krylov solvers of the reduced camera system S dx_p = -b~ (Section 3.2), for one problem or for
// a batch of independent problems that share every launch.
//
// Algorithm 1 (block-Jacobi PCG) and Algorithm 2 (MCG) run as a fixed sequence of kernels per
// iteration.  All data-dependent control (the stop test, the tau-test and the width of the next
// direction block, the history size) lives in one device struct Ctl per problem, written only by
// the per-problem "decide" steps (run by the CTA that finalises an update kernel's sums, and by the
// small solve) and read by the others.  A whole solve is one CUDA graph: a conditional WHILE node
// repeats a body of `chunk` iterations while k_loop_cond finds a problem that is not done (the
// float64 iterative refinement of mixed precision is an outer WHILE node around it), so the host
// launches the graph once and reads the results once; nothing inside a solve waits on the host.
// A problem whose Ctl::done is set is skipped by every later launch while the others go on.
//
// Batches: problem b owns the cameras [c0, c0 + nc) of the handle (S is block-diagonal over the
// problems, since no landmark is seen by two of them).  Per-problem kernels take the problem from
// blockIdx.y; the block-sparse products run over one work list of all problems' rows, each item
// tagged with its problem.  Every per-problem result is summed in an order fixed by the problem
// alone (its own cameras, rows and work items), so a problem solved inside a batch gives the
// same bits as the same problem solved alone.  One problem is the batch of one.
//
// MCG data: the search blocks P_j and their images Q_j are kept as columns of two column-major
// arrays per problem (column c at hoff + c * n, n = 9 nc); block j starts at column blk_off[j]
// and is blk_w[j] wide (1 for a global step, N_eff for a local one).  The pseudo-inverse of
// Delta_j is kept for the full reorthogonalisation
//     beta_{i,j} = Delta_j^+ Q_j^T Z_{i+1},  P_{i+1} = Z_{i+1} - sum_j P_j beta_{i,j},
//     Q_{i+1}   = S Z_{i+1} - sum_j Q_j beta_{i,j}            (Eq. 18 with j = 0..i)
// where S Z_{i+1} applies each block S_jk only to the column of the subset of pose k
// (the product trick of Section 3.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <numeric>
#include <queue>
#include <utility>
#include <vector>

#include "ba_internal.cuh"

namespace ba {

namespace {

constexpr int kGramMax = kMaxDirs * kMaxDirs + kMaxDirs;   // Delta (w x w) and gamma (w)
constexpr int kChunkCams = 112;                             // cameras per Phi partial
constexpr double kStagnation = 1e-4;                        // float32 sweep stop on t_i (see Ctl::stag)
constexpr int kTotals = 16;                                 // per-problem grid totals
constexpr int kUpdCams = 28;                                // cameras per CTA of the update kernels (252 rows)

// Where one problem of the batch lives (fixed for a solve).
struct Layout {
    int c0, nc;          // first camera, number of cameras
    int64_t hoff;        // first element of its direction history (cap columns of 9 nc rows)
    int64_t phoff;       // first Phi partial
    int64_t boff;        // first beta row (16 values each)
    int n_eff, sz, K, cap;
};

struct Ctl {
    Layout lay;
    int it;            // completed steps
    int done;
    int status;
    int cols;          // history columns in use
    int hist_cols;     // columns the current reorthogonalisation runs over
    int new_off;       // first column of the block being formed
    int w_new;         // its width
    int local;         // 1 if the block being formed holds the local directions
    int local_steps;
    int n_eff;
    int sz;            // poses per subset
    int K;             // Phi partials per subset
    int max_iters;
    int cap;
    int w_cur;         // width of the current block (set by decide for the next gram)
    int off_cur;
    double rr0, rr, rz, ga, tol2, tau;
    double rr0_inv;    // 1 / rr0: the residual history stores rr / rr0 without a division per step
    double Delta, gamma, beta;          // PCG scalars
    double alpha_v[kMaxDirs];
    double true_rr, bb;                 // true residual and |rhs|^2
    double stag;       // float32 sweeps: stop when t_i (energy decrease / r^T D^-1 r) falls below this
    int direct_q;      // 1: Q_{i+1} = S P_{i+1} (Algorithm 2); 0: the Q update of Eq. 18
    int pinv_steps;    // steps whose Delta_i took the eigen-decomposition pseudo-inverse
    int hist_off;      // residual history: this sweep's first row (earlier sweeps' steps)
    double hist_scale; // and the factor that puts its values in units of the outer |b~|^2
};

// Per-solve arguments read by the kernels (one copy in device memory, written before each launch of
// the solve graph, so one captured graph serves every tolerance, tau and iteration budget).
struct Params {
    double tol, tau, inner_tol;
    int max_iters, max_refine, mcg, pad;
};

// Loop counters of a solve (zeroed before each launch): body passes of the Krylov loop (all sweeps),
// passes of the refinement loop, passes of the current sweep, and whether the safety bound ended a
// loop with a problem still running.
struct Loops {
    int inner, outer, cur, capped;
};

// Float64 iterative refinement of one problem (mixed precision).
struct Outer {
    double bb;         // |b~|^2
    double tr;         // |-b~ - S x|^2 of the current x
    double tr_prev;    // the same before the last sweep (scales that sweep's residual history)
    double tol_in;     // relative tolerance of the next inner sweep
    int status;
    int active;        // still refining
    int swept;         // takes part in the sweep being run
    int sweeps, iters, locals, pinvs;
    int max_in;        // iteration budget of the next sweep
    int cols;          // history columns of its last sweep
};

__device__ __forceinline__ int64_t gtid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// Sum of products a_i b_i of float32 (or float64) values.  float64: plain float64 accumulation.
// float32: each product is split exactly into p + e (p = fl(a b), e = fma(a, b, -p)) and added to
// a float pair (hi, lo) with an error-free two-sum, so the sum keeps about 48 bits without
// float64 arithmetic, which runs at a small fraction of the float32 rate on this GPU.
template <typename T>
struct ExactSum;
template <>
struct ExactSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s += a * b; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct ExactSum<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);
        const float t = __fadd_rn(hi, p);
        const float bv = __fsub_rn(t, hi);
        const float te = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(p, bv));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(te, pe));
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
    // add another pair (h, l): error-free two-sum of the high parts, low parts added
    __device__ __forceinline__ void add_pair(float h, float l) {
        const float t = __fadd_rn(hi, h);
        const float bv = __fsub_rn(t, hi);
        const float te = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(h, bv));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(te, l));
    }
};

// s += sum_k x[k * xs] y[k * ys] for k < n
template <typename T>
__device__ __forceinline__ void dot_rows(ExactSum<T>& s, const T* x, int xs, const T* y, int ys, int n) {
    for (int k = 0; k < n; ++k) s.add(x[k * xs], y[k * ys]);
}

// A Gram partial sum as stored between the Gram and the small-solve kernels: float64, or (for the
// float32 sweeps) the float pair (hi, lo) in the same 8 bytes, so that adding the partials needs no
// float64 arithmetic either.
__device__ __forceinline__ void store_partial(double* slot, const ExactSum<double>& s) { *slot = s.value(); }
__device__ __forceinline__ void store_partial(double* slot, const ExactSum<float>& s) {
    *reinterpret_cast<float2*>(slot) = make_float2(s.hi, s.lo);
}
__device__ __forceinline__ void load_partial(ExactSum<double>& s, const double* slot) { s.s += *slot; }
__device__ __forceinline__ void combine(ExactSum<double>& a, const ExactSum<double>& b) { a.s += b.s; }
__device__ __forceinline__ void combine(ExactSum<float>& a, const ExactSum<float>& b) { a.add_pair(b.hi, b.lo); }
// a += the same sum held by lane (lane ^ o) (every lane of the warp calls this)
__device__ __forceinline__ void combine_shfl(ExactSum<double>& a, int o) { a.s += __shfl_xor_sync(0xffffffffu, a.s, o); }
__device__ __forceinline__ void combine_shfl(ExactSum<float>& a, int o) {
    const float h = __shfl_xor_sync(0xffffffffu, a.hi, o), l = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a.add_pair(h, l);
}
__device__ __forceinline__ void load_partial(ExactSum<float>& s, const double* slot) {
    const float2 v = *reinterpret_cast<const float2*>(slot);
    s.add_pair(v.x, v.y);
}

// Value k of the kThreads / 32 warp sums in red (row stride nv), added as a fixed tree
// ((w0 + w1) + (w2 + w3)) + ((w4 + w5) + (w6 + w7)): three dependent float64 additions.
__device__ __forceinline__ double sum_warps(const double* red, int nv, int k) {
    static_assert(kThreads == 256, "tree over eight warps");
    const double a = red[0 * nv + k] + red[1 * nv + k], b = red[2 * nv + k] + red[3 * nv + k];
    const double c = red[4 * nv + k] + red[5 * nv + k], d = red[6 * nv + k] + red[7 * nv + k];
    return (a + b) + (c + d);
}

// Sum `nv` values per thread over the CTA; threads 0..NV-1 write them to out[0..NV) (global or
// shared memory), visible to the whole CTA on return.
template <int NV>
__device__ __forceinline__ void cta_sum_write(double (&v)[NV], double* out) {
    __shared__ double red[kThreads / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0) red[wid][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) out[threadIdx.x] = sum_warps(&red[0][0], NV, threadIdx.x);
    __syncthreads();
}

// Sum partial[p * stride + k] over p < np in a fixed order (called by one warp; every lane returns it).
__device__ __forceinline__ double sum_partials(const double* partial, int np, int stride, int k) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int p = lane; p < np; p += 32) s += partial[int64_t(p) * stride + k];
    return warp_sum(s);
}

// ---------------------------------------------------------------------------------------
// block-sparse products

// Work items of the block-sparse products.  Item = a chunk [q0, q1) of the blocks of block-row
// `row` that feed output column `seg` (the subset of the column cameras in MCG's local step, 0
// otherwise) of problem `prob`; it is chunk k of the ng chunks of its output group (row, seg),
// whose partial-sum slots are slot - k .. slot - k + ng - 1.  Each chunk writes its 9 partial
// sums, and the warp that finishes last (atomic count, no waiting) adds the partials in chunk
// order, so the result does not depend on scheduling or on the order of the list.  Counters reset
// themselves.
struct SpItem {
    int row, seg, q0, q1, grp, k, ng, prob, slot;
};

struct ItemList {
    const SpItem* items = nullptr;
    int64_t n = 0;
    int* cnt = nullptr;       // one per group, zero between launches
    void* part = nullptr;     // n x 9 partial sums (element type of the product), by slot
    int nprob = 0;            // problems the list covers
    int polls = kDefaultWaitPolls;   // polls of a tile barrier before a wait gives up (0: at once)
    int ngrp = 0;             // groups (counters)
    // Balanced order: warp g of a launch with nw warps takes items wptr[g] .. wptr[g + 1] - 1 (the
    // list is ordered so that the warps' tiles are about equal); a launch with another warp count
    // takes every (its warps)-th item instead.
    const int64_t* wptr = nullptr;
    int64_t nw = 0;
};

// The items of this warp: its range of the balanced order, or every W-th item.
struct WarpItems {
    int64_t i0, end, step;
};
__device__ __forceinline__ WarpItems warp_items(const ItemList& L, int NW, int wid) {
    const int64_t W = int64_t(gridDim.x) * NW, g = int64_t(blockIdx.x) * NW + wid;
    if (L.wptr != nullptr && W == L.nw) return {L.wptr[g], L.wptr[g + 1], 1};
    return {g, L.n, W};
}

// Which problems a product serves: every live one, those forming a global (local) block, or those
// whose new block is one column wide (wider).
enum : int { kSelLive = 0, kSelGlobal = 1, kSelLocal = 2, kSelW1 = 3, kSelWide = 4 };

__device__ __forceinline__ bool selected(const Ctl* ctl, int prob, int sel) {
    const Ctl& c = ctl[prob];
    if (c.done) return false;
    switch (sel) {
        case kSelGlobal: return c.local == 0;
        case kSelLocal: return c.local != 0;
        case kSelW1: return c.w_new == 1;
        case kSelWide: return c.w_new > 1;
        default: return true;
    }
}

// true when no problem of the list is selected (checked for small batches only; every warp of the
// CTA reaches the same answer, so the whole CTA may return)
__device__ __forceinline__ bool nothing_selected(const Ctl* ctl, const ItemList& L, int sel) {
    if (L.nprob > 64) return false;
    bool any = false;
    for (int b = threadIdx.x & 31; b < L.nprob; b += 32) any = any || selected(ctl, b, sel);
    return !__any_sync(0xffffffffu, any);
}

// Sum the CTA's NV values, publish them as partial[blockIdx.x], and let the last CTA of the grid
// row to finish write the row's totals (in CTA order) to totals[0..NV).  Every CTA of the grid
// row must call it.  Returns true (in every thread) in the CTA that wrote the totals, after they
// are visible to the whole CTA.
template <int NV>
__device__ __forceinline__ bool grid_sum_finalize(double (&v)[NV], double* partial, int* cnt, double* totals) {
    __shared__ double red[kThreads / 32][NV];
    __shared__ int last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0) red[wid][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) partial[int64_t(blockIdx.x) * NV + threadIdx.x] = sum_warps(&red[0][0], NV, threadIdx.x);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(cnt, 1) == int(gridDim.x) - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // warp k adds value k over the CTA partials: lane l takes partials l, l + 32, ... (independent
    // loads, short float64 chains), then the fixed shuffle tree; partials of CTAs without rows are
    // exact zeros, so the sum does not depend on the grid width
    static_assert(NV <= kThreads / 32, "one warp per value");
    if (wid < NV) {
        double s = 0.0;
        for (int b = lane; b < int(gridDim.x); b += 32) s += __ldcg(partial + int64_t(b) * NV + wid);
        s = warp_sum(s);
        if (lane == 0) totals[wid] = s;
    }
    if (threadIdx.x == 0) *cnt = 0;
    __syncthreads();
    return true;
}

// ---- bulk copies (cp.async.bulk + mbarrier) --------------------------------------------

// Bounded mbarrier waits: after `polls` unsuccessful polls a wait gives up (polls = 0: at once); the
// kernel then records BA_ERR_TIMEOUT and drains its own copies in flight with the default bound.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// one elected thread: bytes from global src to shared dst, completion counted on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// The same copy marked evict-first in L2 (`policy` from l2_evict_first): a stream read once per
// launch then gives way to data that a later kernel reads again.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_load_ef(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
// First statement of the kernels of a solve iteration, which are launched chained (launch_chained):
// such a kernel may be scheduled while the previous kernel on the stream drains (its CTAs retire,
// the implicit trigger), and waits here for that kernel to complete and its writes to be visible.
// Without the chained attribute it returns at once.  (An explicit early trigger, letting the next
// kernel's CTAs take SM resources while this one runs, made the 1936-camera PCG solve slower:
// 4.2 -> 4.8 ms.)
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int polls) {
    for (int i = 0; i < polls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Warps per CTA and copy stages of the tile-streaming one-column product, one CTA per SM.  Three
// shapes per precision (ba_options.spmv_config, chosen by ba_autotune); shape 0 is the default:
// float32 16 warps x 1 stage (measured faster than 8 x 2 for the full-pattern product: more warps
// cover the gathers of p), float64 4 x 2.  The symmetric product does twice the arithmetic per tile,
// so a second stage per warp keeps the next copy in flight during it (shapes 1 and 2).  Every shape
// keeps its stages within 207 KB.
template <typename T, int CFG>
struct SpmvShape;
template <> struct SpmvShape<float, 0> { static constexpr int kWarps = 16, kStages = 1; };
template <> struct SpmvShape<float, 1> { static constexpr int kWarps = 8, kStages = 2; };
template <> struct SpmvShape<float, 2> { static constexpr int kWarps = 10, kStages = 2; };
template <> struct SpmvShape<double, 0> { static constexpr int kWarps = 4, kStages = 2; };
template <> struct SpmvShape<double, 1> { static constexpr int kWarps = 8, kStages = 1; };
template <> struct SpmvShape<double, 2> { static constexpr int kWarps = 2, kStages = 4; };
constexpr int kSpmvShapes = 3;
// Shared memory of k_spmv: the warps' tile stages, then the stages' barriers.
template <typename T, int CFG>
constexpr size_t spmv_smem() {
    return sizeof(T) * SpmvShape<T, CFG>::kWarps * SpmvShape<T, CFG>::kStages * kTileElems +
           sizeof(uint64_t) * SpmvShape<T, CFG>::kWarps * SpmvShape<T, CFG>::kStages;
}

// The transposed terms of the symmetric product, one slot per stored upper block: values 0..7 of slot
// e at tb[8 e ..] (one 32-byte sector in float32, written whole by two 16-byte stores, so that L2
// never fills a partly written sector from DRAM) and value 8 at tb[8 n_slots + e].
constexpr int kTbHead = 8;


// Tile cursor of a warp: the tiles of its selected items (WarpItems) in order, skipping empty
// items.  The consumer loop selects items with the same predicate, which no kernel changes while
// it runs.
struct TileCursor {
    int64_t item, end, step;
    int t, te;
    int64_t base;
};
__device__ __forceinline__ void cursor_seek(TileCursor& c, const ItemList& L, const int64_t* tile_ptr,
                                            const Ctl* ctl, int sel, int64_t item) {
    for (; item < c.end; item += c.step) {
        const SpItem it = L.items[item];
        if (it.q1 > it.q0 && selected(ctl, it.prob, sel)) {
            c.item = item;
            c.t = it.q0 >> 5;
            c.te = (it.q1 + 31) >> 5;
            c.base = tile_ptr[it.row];
            return;
        }
    }
    c.item = c.end;
    c.t = c.te = 0;
    c.base = 0;
}
__device__ __forceinline__ void cursor_start(TileCursor& c, const ItemList& L, const int64_t* tile_ptr,
                                             const Ctl* ctl, int sel, const WarpItems& wi) {
    c.end = wi.end;
    c.step = wi.step;
    cursor_seek(c, L, tile_ptr, ctl, sel, wi.i0);
}

// y(row, seg) = sum over the item's blocks of S_row,col(q) z_col(q).  Each warp streams the
// tiles of its items through kStages shared-memory buffers with bulk copies (issued by lane 0,
// NS tiles ahead) and multiplies them with the gathered z blocks.
// ZH: z is a column of the problem's direction history (column new_off in MODE 2, column 0
//     otherwise); else z is a vector over all cameras.
// MODE 0: y goes to column new_off + seg of the problem's Q.
// MODE 1 (Algorithm 1): q = y (Q column 0) and, per camera, the sums of q^T p and p^T r
//         (Delta and gamma of Algorithm 1, before the sum over cameras).
// MODE 2 (Algorithm 2, width 1): y goes to column new_off of Q.
// SYM: S is the upper triangle (row j: S_jj, then S_jk for k > j).  Each lane's block also gives the
// transposed term S_jk^T z_j of row k, written to slot cslot[32 tile_ptr[j] + q] of tb/tb8 (the terms
// of column k are consecutive there, in row order), which k_spmv_col adds to row k; in MODE 1 the
// per-camera sums then move to k_spmv_col as well.
template <typename T, int MODE, bool ZH, bool SYM, int CFG>
__global__ void __launch_bounds__(SpmvShape<T, CFG>::kWarps * 32, 1) k_spmv(
    const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr, const int32_t* __restrict__ col,
    const T* __restrict__ S, const T* __restrict__ z, ItemList L, int sel, T* __restrict__ out,
    const T* __restrict__ rvec, double* __restrict__ camdot, Ctl* ctl, T* __restrict__ tb, T* __restrict__ tb8,
    const int32_t* __restrict__ cslot) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    constexpr int NW = SpmvShape<T, CFG>::kWarps, NS = SpmvShape<T, CFG>::kStages;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (nothing_selected(ctl, L, sel)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T* tiles = reinterpret_cast<T*>(smem_raw) + size_t(wid) * NS * kTileElems;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * NW * NS * kTileElems) + wid * NS;
    T* part = static_cast<T*>(L.part);
    constexpr uint32_t tile_bytes = sizeof(T) * kTileElems;

    if (lane == 0) {
        for (int st = 0; st < NS; ++st) mbar_init(&bars[st]);
        fence_mbar_init();
    }
    __syncwarp();
    const WarpItems wi = warp_items(L, NW, wid);
    TileCursor f;
    cursor_start(f, L, tile_ptr, ctl, sel, wi);
    // the symmetric product reads its tiles once and its transposed terms tb again in k_spmv_col:
    // the tiles go first when L2 must evict
    const uint64_t pol = SYM ? l2_evict_first() : 0;
    auto load_tile = [&](int st) {
        T* dst = tiles + st * kTileElems;
        const T* src = S + (f.base + f.t) * kTileElems;
        if (SYM) bulk_load_ef(dst, src, tile_bytes, &bars[st], pol);
        else bulk_load(dst, src, tile_bytes, &bars[st]);
    };
    uint32_t parity = 0, inflight = 0;
    for (int st = 0; st < NS; ++st) {
        if (f.item < f.end) {
            if (lane == 0) load_tile(st);
            inflight |= 1u << st;
            if (++f.t == f.te) cursor_seek(f, L, tile_ptr, ctl, sel, f.item + f.step);
        }
    }
    int stage = 0;
    bool bad = false;
    int bad_prob = 0;
    for (int64_t i = wi.i0; i < wi.end && !bad; i += wi.step) {
        const SpItem it = L.items[i];
        if (!selected(ctl, it.prob, sel)) continue;
        const Ctl& c = ctl[it.prob];
        const int64_t n = int64_t(c.lay.nc) * 9;
        const int64_t hb = c.lay.hoff - 9 * int64_t(c.lay.c0);   // history column 0 at global row i: hb + i
        const int64_t zoff = ZH ? hb + int64_t(MODE == 2 ? c.new_off : 0) * n : 0;
        const int64_t ooff = hb + int64_t(MODE == 1 ? 0 : (MODE == 2 ? c.new_off : c.new_off + it.seg)) * n;
        const int64_t rj = row_ptr[it.row];
        const int64_t tb0 = SYM ? tile_ptr[it.row] * kTile : 0;   // tiled index of the row's first block
        T acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = T(0);
        T zr[9];   // SYM: z of the row camera, the factor of every transposed term of the item
#pragma unroll
        for (int b = 0; b < 9; ++b) zr[b] = SYM ? z[zoff + 9 * int64_t(it.row) + b] : T(0);
        if (it.q1 > it.q0) {
            const int t0 = it.q0 >> 5, t1 = (it.q1 + 31) >> 5;
            // the 9 entries of z this lane needs for tile t (and SYM: the slot of its transposed
            // term, -1 for none), fetched one tile ahead
            T zn[9];
            int csn = -1;
            {
                const int q = t0 * 32 + lane;
                const bool in = q >= it.q0 && q < it.q1;
                const T* zk = z + zoff + int64_t(in ? col[rj + q] : it.row) * 9;
#pragma unroll
                for (int b = 0; b < 9; ++b) zn[b] = in ? zk[b] : T(0);
                if (SYM && in) csn = cslot[tb0 + q];
            }
            for (int t = t0; t < t1; ++t) {
                T zv[9];
#pragma unroll
                for (int b = 0; b < 9; ++b) zv[b] = zn[b];
                const int csv = csn;
                if (t + 1 < t1) {
                    const int qn = (t + 1) * 32 + lane;
                    const bool in = qn < it.q1;
                    const T* zk = z + zoff + int64_t(in ? col[rj + qn] : it.row) * 9;
#pragma unroll
                    for (int b = 0; b < 9; ++b) zn[b] = in ? zk[b] : T(0);
                    csn = SYM && in ? cslot[tb0 + qn] : -1;
                }
                // every lane observes the phase (visibility of the copied bytes); the warp agrees
                const bool ok = mbar_wait(&bars[stage], (parity >> stage) & 1u, L.polls);
                if (!__all_sync(0xffffffffu, ok)) {
                    bad = true;
                    bad_prob = it.prob;
                    break;
                }
                parity ^= 1u << stage;
                inflight &= ~(1u << stage);
                const T* tile = tiles + stage * kTileElems;
                const int q = t * 32 + lane;
                const bool inq = q >= it.q0 && q < it.q1;
                if (SYM) {
                    T v[9];
#pragma unroll
                    for (int b = 0; b < 9; ++b) v[b] = T(0);
                    if (inq) {
                        const T* blk = tile + lane * 81;
#pragma unroll
                        for (int a = 0; a < 9; ++a)
#pragma unroll
                            for (int b = 0; b < 9; ++b) {
                                const T sab = blk[9 * a + b];
                                acc[a] += sab * zv[b];
                                v[b] += sab * zr[a];
                            }
                    }
                    // q = 0 is S_jj, whose row term covers it (its slot is -1)
                    if (csv >= 0) {
                        T* dst = tb + int64_t(csv) * kTbHead;
                        if constexpr (sizeof(T) == 4) {
                            reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
                            reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
                        } else {
#pragma unroll
                            for (int b = 0; b < 8; ++b) dst[b] = v[b];
                        }
                        tb8[csv] = v[8];
                    }
                } else if (inq) {
                    const T* blk = tile + lane * 81;
#pragma unroll
                    for (int a = 0; a < 9; ++a)
#pragma unroll
                        for (int b = 0; b < 9; ++b) acc[a] += blk[9 * a + b] * zv[b];
                }
                __syncwarp();
                if (f.item < f.end) {
                    fence_proxy_async();
                    if (lane == 0) load_tile(stage);
                    inflight |= 1u << stage;
                    if (++f.t == f.te) cursor_seek(f, L, tile_ptr, ctl, sel, f.item + f.step);
                }
                stage = stage + 1 == NS ? 0 : stage + 1;
            }
            if (bad) break;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = warp_sum(acc[a]);
        T val = acc[0];
#pragma unroll
        for (int a = 1; a < 9; ++a) if (lane == a) val = acc[a];
        bool fin = true;
        if (it.ng > 1) {
            if (lane < 9) part[int64_t(it.slot) * 9 + lane] = val;
            __threadfence();
            int last = 0;
            if (lane == 0) last = (atomicAdd(L.cnt + it.grp, 1) == it.ng - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            fin = last != 0;
            if (fin) {
                __threadfence();
                T sum = T(0);
                const int64_t first = int64_t(it.slot) - it.k;
                if (lane < 9)
                    for (int cc = 0; cc < it.ng; ++cc) sum += __ldcg(part + (first + cc) * 9 + lane);
                val = sum;
                if (lane == 0) L.cnt[it.grp] = 0;
            }
        }
        if (fin) {
            const int64_t rowi = 9 * int64_t(it.row) + lane;
            if (lane < 9) out[ooff + rowi] = val;
            if (MODE == 1 && !SYM) {
                double dq = 0.0, dr = 0.0;
                if (lane < 9) {
                    const double pv = double(z[zoff + rowi]);
                    dq = double(val) * pv;
                    dr = pv * double(rvec[rowi]);
                }
                dq = warp_sum(dq);
                dr = warp_sum(dr);
                if (lane == 0) {
                    camdot[2 * int64_t(it.row)] = dq;
                    camdot[2 * int64_t(it.row) + 1] = dr;
                }
            }
        }
    }
    if (bad) {
        // a copy did not land in time: report, then wait (bounded) for this warp's copies in flight;
        // the problem's next decide step ends it with the status
        if (lane == 0) atomicExch(&ctl[bad_prob].status, BA_ERR_TIMEOUT);
        for (int st = 0; st < NS; ++st)
            if (inflight & (1u << st)) mbar_wait(&bars[st], (parity >> st) & 1u, kDefaultWaitPolls);
    }
}

// Second pass of the symmetric product: y_k += sum over the stored blocks (j, k), j < k, of their
// transposed terms S_jk^T z_j (a fixed order: lane-strided sums in each warp's share of the column's
// slots, then the warps' sums in warp order), then in MODE 1 the per-camera sums q^T p and p^T r.
// One CTA of kColWarps warps per camera (its slots qptr[k] .. qptr[k + 1] - 1 of tb are consecutive,
// up to n_c - 1 of them); grid: CTAs x problems.  CTAs take the cameras from the last one down:
// camera k's column holds the blocks (j, k), j < k, so on a dense pattern the long columns start
// in the first wave and the short ones fill the tail.
constexpr int kColWarps = 4;   // 12 CTAs per SM: 1824 cameras in flight
template <typename T, int MODE, bool ZH>
__global__ void __launch_bounds__(kColWarps * 32, 12) k_spmv_col(const int64_t* __restrict__ qptr,
                                                             const T* __restrict__ tb, const T* __restrict__ tb8,
                                                             const T* __restrict__ z, int sel, T* __restrict__ out,
                                                             const T* __restrict__ rvec, double* __restrict__ camdot,
                                                             const Ctl* __restrict__ ctl) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const int p = blockIdx.y;
    if (!selected(ctl, p, sel)) return;
    const Ctl& c = ctl[p];
    __shared__ T red[kColWarps][9];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = int64_t(c.lay.nc) * 9;
    const int64_t hb = c.lay.hoff - 9 * int64_t(c.lay.c0);
    const int64_t zoff = ZH ? hb + int64_t(MODE == 2 ? c.new_off : 0) * n : 0;
    const int64_t ooff = hb + int64_t(MODE == 1 ? 0 : c.new_off) * n;
    for (int64_t jr = blockIdx.x; jr < c.lay.nc; jr += gridDim.x) {
        const int64_t j = c.lay.c0 + (c.lay.nc - 1 - jr);
        T acc[9];
#pragma unroll
        for (int b = 0; b < 9; ++b) acc[b] = T(0);
        // warp w takes slots w * 32 + lane + k * kColWarps * 32, four per lane in flight (slots past
        // the end add exact zeros)
        constexpr int step = kColWarps * 32;
        const int64_t e1 = qptr[j + 1];
        for (int64_t e = qptr[j] + wid * 32 + lane; e < e1; e += 4 * step) {
            T v[4][9];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t eu = e + u * step;
                const T* t = tb + eu * kTbHead;
                if (eu < e1) {
                    if constexpr (sizeof(T) == 4) {
                        const float4 a = reinterpret_cast<const float4*>(t)[0];
                        const float4 c = reinterpret_cast<const float4*>(t)[1];
                        v[u][0] = a.x, v[u][1] = a.y, v[u][2] = a.z, v[u][3] = a.w;
                        v[u][4] = c.x, v[u][5] = c.y, v[u][6] = c.z, v[u][7] = c.w;
                    } else {
#pragma unroll
                        for (int b = 0; b < 8; ++b) v[u][b] = t[b];
                    }
                    v[u][8] = tb8[eu];
                } else {
#pragma unroll
                    for (int b = 0; b < 9; ++b) v[u][b] = T(0);
                }
            }
#pragma unroll
            for (int b = 0; b < 9; ++b) acc[b] += (v[0][b] + v[1][b]) + (v[2][b] + v[3][b]);
        }
#pragma unroll
        for (int b = 0; b < 9; ++b) acc[b] = warp_sum(acc[b]);
        if (lane == 0)
#pragma unroll
            for (int b = 0; b < 9; ++b) red[wid][b] = acc[b];
        __syncthreads();
        if (wid == 0) {
            T val = T(0);
            if (lane < 9) {
                val = red[0][lane];
#pragma unroll
                for (int w = 1; w < kColWarps; ++w) val += red[w][lane];
            }
            const int64_t rowi = 9 * j + lane;
            if (lane < 9) {
                val = out[ooff + rowi] + val;
                out[ooff + rowi] = val;
            }
            if (MODE == 1) {
                double dq = 0.0, dr = 0.0;
                if (lane < 9) {
                    const double pv = double(z[zoff + rowi]);
                    dq = double(val) * pv;
                    dr = pv * double(rvec[rowi]);
                }
                dq = warp_sum(dq);
                dr = warp_sum(dr);
                if (lane == 0) {
                    camdot[2 * j] = dq;
                    camdot[2 * j + 1] = dr;
                }
            }
        }
        __syncthreads();
    }
}

// Q[:, new_off + c] = S P[:, new_off + c] for the w > 1 columns of a new local block (Algorithm 2,
// used by the float32 sweeps, where the Eq. 18 update cancels).  Tiles stream through
// shared memory as in k_spmv; lane = 4 qi + g takes tile-local blocks qi, qi + 8, qi + 16, qi + 24
// and columns 4g .. 4g + 3, so each 9x9 block multiplies up to 16 columns per read from shared
// memory.  PT is the row-major copy (9 n_c x 16, all problems) of the new blocks.
// The multi-column product waits on L2 gathers of PT more than on its tiles, so it runs twice
// the warps of k_spmv with one tile stage each (the other warps' copies and arithmetic cover a
// warp's wait for its next tile); at most 128 registers a thread.
struct SpmmCfg {
    static constexpr int kWarps = 16, kStages = 1;
};
template <typename T>
constexpr size_t spmm_tiles_smem() {
    return sizeof(T) * SpmmCfg::kWarps * SpmmCfg::kStages * kTileElems +
           sizeof(uint64_t) * SpmmCfg::kWarps * SpmmCfg::kStages;
}
template <typename T>
constexpr size_t spmm_smem() {
    return spmm_tiles_smem<T>() + sizeof(T) * SpmmCfg::kWarps * kMaxDirs * 9;
}

// rows b = 0..8 of a 16-column PT block, 4 columns from p: (p[16 b], p[16 b + 1]) and
// (p[16 b + 2], p[16 b + 3]) as float pairs (one 16-byte load per row)
__device__ __forceinline__ void load_prow(const float* p, float2 (&v)[9][2]) {
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const float4 t = *reinterpret_cast<const float4*>(p + b * kMaxDirs);
        v[b][0] = make_float2(t.x, t.y);
        v[b][1] = make_float2(t.z, t.w);
    }
}

template <typename T>
__global__ void __launch_bounds__(SpmmCfg::kWarps * 32, 1) k_spmm(
    const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr, const int32_t* __restrict__ col,
    const T* __restrict__ S, const T* __restrict__ PT, ItemList L, T* __restrict__ part, T* __restrict__ Q,
    Ctl* ctl) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    static_assert(sizeof(T) == 4, "the multi-column product serves the float32 sweeps");
    constexpr int NW = SpmmCfg::kWarps, NS = SpmmCfg::kStages;
    constexpr int sel = kSelWide;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (nothing_selected(ctl, L, sel)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int qi = lane >> 2, g = lane & 3;
    T* tiles = reinterpret_cast<T*>(smem_raw) + size_t(wid) * NS * kTileElems;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * NW * NS * kTileElems) + wid * NS;
    T* red = reinterpret_cast<T*>(smem_raw + spmm_tiles_smem<T>()) + wid * (kMaxDirs * 9);
    constexpr uint32_t tile_bytes = sizeof(T) * kTileElems;
    if (lane == 0) {
        for (int st = 0; st < NS; ++st) mbar_init(&bars[st]);
        fence_mbar_init();
    }
    __syncwarp();
    const WarpItems wi = warp_items(L, NW, wid);
    TileCursor f;
    cursor_start(f, L, tile_ptr, ctl, sel, wi);
    uint32_t parity = 0, inflight = 0;
    for (int st = 0; st < NS; ++st) {
        if (f.item < f.end) {
            if (lane == 0) bulk_load(tiles + st * kTileElems, S + (f.base + f.t) * kTileElems, tile_bytes, &bars[st]);
            inflight |= 1u << st;
            if (++f.t == f.te) cursor_seek(f, L, tile_ptr, ctl, sel, f.item + f.step);
        }
    }
    int stage = 0;
    bool bad = false;
    int bad_prob = 0;
    for (int64_t i = wi.i0; i < wi.end && !bad; i += wi.step) {
        const SpItem it = L.items[i];
        if (!selected(ctl, it.prob, sel)) continue;
        const Ctl& c = ctl[it.prob];
        const int w = c.w_new;
        const int nout = 9 * w;
        const int64_t n = int64_t(c.lay.nc) * 9;
        const int64_t ooff = c.lay.hoff - 9 * int64_t(c.lay.c0) + int64_t(c.new_off) * n;
        const int64_t rj = row_ptr[it.row];
        // columns (4g, 4g + 1) and (4g + 2, 4g + 3) of the 9 rows, as float pairs for the packed
        // float32 multiply-add (each pair operation rounds like two scalar fused multiply-adds)
        float2 acc[9][2];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a][0] = acc[a][1] = make_float2(0.f, 0.f);
        if (it.q1 > it.q0) {
            const int t0 = it.q0 >> 5, t1 = (it.q1 + 31) >> 5;
            const bool active = 4 * g < w;
            // column cameras of this lane's blocks r * 8 + qi (r = 0..3) of tile t, -1 outside the
            // item; fetched one tile ahead.  The P rows of a block are gathered right before its
            // arithmetic: the other warps of the SM cover the wait
            int kc[4], kn[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int q = t0 * 32 + r * 8 + qi;
                kc[r] = (active && q >= it.q0 && q < it.q1) ? col[rj + q] : -1;
            }
            float2 pv[9][2];
            for (int t = t0; t < t1; ++t) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int q = (t + 1) * 32 + r * 8 + qi;
                    kn[r] = (active && t + 1 < t1 && q < it.q1) ? col[rj + q] : -1;
                }
                const bool ok = mbar_wait(&bars[stage], (parity >> stage) & 1u, L.polls);
                if (!__all_sync(0xffffffffu, ok)) {
                    bad = true;
                    bad_prob = it.prob;
                    break;
                }
                parity ^= 1u << stage;
                inflight &= ~(1u << stage);
                const T* tile = tiles + stage * kTileElems;
                if (active) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (kc[r] < 0) continue;
                        // rows 9k .. 9k + 8, columns 4g .. 4g + 3 of PT for this block
                        load_prow(PT + (int64_t(kc[r]) * 9) * kMaxDirs + 4 * g, pv);
                        const T* blk = tile + (r * 8 + qi) * 81;
#pragma unroll
                        for (int a = 0; a < 9; ++a)
#pragma unroll
                            for (int b = 0; b < 9; ++b) {
                                const float sab = blk[9 * a + b];
                                const float2 s2 = make_float2(sab, sab);
                                acc[a][0] = __ffma2_rn(s2, pv[b][0], acc[a][0]);
                                acc[a][1] = __ffma2_rn(s2, pv[b][1], acc[a][1]);
                            }
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) kc[r] = kn[r];
                __syncwarp();
                if (f.item < f.end) {
                    fence_proxy_async();
                    if (lane == 0)
                        bulk_load(tiles + stage * kTileElems, S + (f.base + f.t) * kTileElems, tile_bytes, &bars[stage]);
                    inflight |= 1u << stage;
                    if (++f.t == f.te) cursor_seek(f, L, tile_ptr, ctl, sel, f.item + f.step);
                }
                stage = stage + 1 == NS ? 0 : stage + 1;
            }
            if (bad) break;
        }
        // sum over the 8 lanes of each column group, then lanes 0..3 hold their columns
        T accs[9][4];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            accs[a][0] = acc[a][0].x;
            accs[a][1] = acc[a][0].y;
            accs[a][2] = acc[a][1].x;
            accs[a][3] = acc[a][1].y;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                T v = accs[a][cc];
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                accs[a][cc] = v;
            }
        __syncwarp();
        if (qi == 0) {
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int ci = 4 * g + cc;
                if (ci < w)
#pragma unroll
                    for (int a = 0; a < 9; ++a) red[ci * 9 + a] = accs[a][cc];
            }
        }
        __syncwarp();
        bool fin = true;
        if (it.ng > 1) {
            for (int o = lane; o < nout; o += 32) part[int64_t(it.slot) * (kMaxDirs * 9) + o] = red[o];
            __threadfence();
            int last = 0;
            if (lane == 0) last = (atomicAdd(L.cnt + it.grp, 1) == it.ng - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            fin = last != 0;
            if (fin) {
                __threadfence();
                const int64_t first = int64_t(it.slot) - it.k;
                for (int o = lane; o < nout; o += 32) {
                    T sum = T(0);
                    for (int cc = 0; cc < it.ng; ++cc) sum += __ldcg(part + (first + cc) * (kMaxDirs * 9) + o);
                    red[o] = sum;
                }
                __syncwarp();
                if (lane == 0) L.cnt[it.grp] = 0;
            }
        }
        if (fin) {
            for (int o = lane; o < nout; o += 32) {
                const int ci = o / 9, a = o % 9;
                Q[ooff + int64_t(ci) * n + 9 * int64_t(it.row) + a] = red[o];
            }
        }
        __syncwarp();
    }
    if (bad) {
        if (lane == 0) atomicExch(&ctl[bad_prob].status, BA_ERR_TIMEOUT);
        for (int st = 0; st < NS; ++st)
            if (inflight & (1u << st)) mbar_wait(&bars[st], (parity >> st) & 1u, kDefaultWaitPolls);
    }
}

// ---------------------------------------------------------------------------------------
// initialisation shared by both algorithms: x = 0, r = sign * rhs, z = D^{-1} r, P_0 = z
// (grid: CTAs x problems; thread = camera of the problem)

template <typename T>
__global__ void k_init_vec(const Layout* __restrict__ lay, const double* __restrict__ rhs, double sign,
                           const double* __restrict__ scale, const double* __restrict__ Dinv, T* __restrict__ x,
                           T* __restrict__ r, T* __restrict__ z, T* __restrict__ P, double* __restrict__ partial) {
    const Layout L = lay[blockIdx.y];
    double v[1] = {0.0};
    for (int64_t jl = gtid(); jl < L.nc; jl += gstride()) {
        const int64_t j = L.c0 + jl;
        double rv[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const double sa = scale ? scale[9 * j + a] : 1.0;
            const T ra = T(sign * sa * rhs[9 * j + a]);
            r[9 * j + a] = ra;
            x[9 * j + a] = T(0);
            rv[a] = double(ra);
            v[0] += rv[a] * rv[a];
        }
        const double* D = Dinv + 81 * j;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < 9; ++b) s += D[9 * a + b] * rv[b];
            z[9 * j + a] = T(s);
            P[L.hoff + 9 * jl + a] = T(s);
        }
    }
    cta_sum_write<1>(v, partial + int64_t(blockIdx.y) * gridDim.x + blockIdx.x);
}

// One warp per problem.  outer (mixed precision, may be null) supplies the sweep's tolerance and
// iteration budget and leaves the problems that are not refined any more done from the start.
__global__ void k_init_ctl(Ctl* ctl, const Layout* __restrict__ lay, const double* __restrict__ partial, int np,
                           const Params* __restrict__ prm, double stag, int direct_q,
                           const Outer* __restrict__ outer, int* blk_off, int* blk_w, int mi1) {
    const int p = blockIdx.x;
    const double rr0 = sum_partials(partial + int64_t(p) * np, np, 1, 0);
    if (threadIdx.x == 0) {
        Ctl c;
        memset(&c, 0, sizeof(c));
        c.lay = lay[p];
        double tl = prm->tol;
        const double tau = prm->tau;
        int mi = prm->max_iters;
        bool act = true;
        c.hist_off = 0;
        c.hist_scale = 1.0;
        if (outer) {
            const Outer& o = outer[p];
            act = o.swept != 0;
            tl = o.tol_in;
            mi = o.max_in;
            c.hist_off = o.iters;
            c.hist_scale = o.bb > 0.0 ? o.tr / o.bb : 0.0;
        }
        c.rr0 = rr0;
        c.rr0_inv = rr0 > 0.0 ? 1.0 / rr0 : 0.0;
        c.rr = rr0;
        c.tol2 = tl * tl;
        c.tau = tau;
        c.max_iters = mi;
        c.n_eff = c.lay.n_eff;
        c.sz = c.lay.sz;
        c.K = c.lay.K;
        c.cap = c.lay.cap;
        c.cols = 1;
        c.w_new = 1;
        c.new_off = 0;
        c.local = 0;
        c.w_cur = 1;
        c.off_cur = 0;
        c.stag = stag;
        c.direct_q = direct_q;
        c.status = BA_OK;
        if (!act) { c.done = 1; }
        else if (!(rr0 == rr0) || isinf(rr0)) { c.done = 1; c.status = BA_ERR_BREAKDOWN; }
        else if (rr0 == 0.0 || mi <= 0) { c.done = 1; c.status = rr0 == 0.0 ? BA_OK : BA_ERR_NOT_CONVERGED; }
        ctl[p] = c;
        blk_off[int64_t(p) * mi1] = 0;
        blk_w[int64_t(p) * mi1] = 1;
    }
}

// Condition of the Krylov WHILE loop: continue while a problem is not done.  first = 1 (before the
// loop) starts the sweep's pass count; otherwise one body pass has ended.  `bound` passes (every
// problem stops by its iteration budget well before) end the loop in any case.  use_handle = 0 when
// the loop runs from the host (the kernel then only counts).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, int use_handle, const Ctl* __restrict__ ctl, int nb,
                            Loops* lp, int first, int chunk, const Params* __restrict__ prm) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int mine = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) mine |= ctl[b].done == 0;
    if (mine) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int go = any;
        if (first) {
            lp->cur = 0;
        } else {
            lp->cur += 1;
            lp->inner += 1;
        }
        const int bound = (prm->max_iters + chunk - 1) / chunk + 2;
        if (lp->cur >= bound) {
            if (go) lp->capped = 1;
            go = 0;
        }
        if (use_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
    }
}

// 1 / p in float64 without the long division chain (an exact float64 division is a dependent
// sequence of about ten operations on this GPU's narrow float64 pipe): a float32 estimate
// (relative error below 2^-23) refined by Newton steps r <- r + r (1 - p r), each of which
// squares the error: one step leaves it below 2^-46 (about 1e-14), two reach float64 rounding.
// Values outside the float32 range divide.
template <int kSteps = 1>
__device__ __forceinline__ double fast_rcp(double p) {
    const double ap = fabs(p);
    if (!(ap > 1e-30 && ap < 1e30)) return 1.0 / p;
    double r = double(__frcp_rn(float(p)));
#pragma unroll
    for (int k = 0; k < kSteps; ++k) r = fma(r, fma(-p, r, 1.0), r);
    return r;
}

// ---------------------------------------------------------------------------------------
// Algorithm 1 (grid: CTAs x problems)

// This thread's share of the per-camera sums (Delta, gamma) of cameras [0, nc): cameras
// threadIdx.x + k blockDim.x, four at a time in interleaved sums (their loads in flight together),
// added as (0 + 1) + (2 + 3).
__device__ __forceinline__ void sum_camdot(const double* cd, int nc, double (&d)[2]) {
    const int bd = blockDim.x;
    double a0[4] = {0.0, 0.0, 0.0, 0.0}, a1[4] = {0.0, 0.0, 0.0, 0.0};
    int j = threadIdx.x;
    for (; j + 3 * bd < nc; j += 4 * bd)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a0[u] += cd[2 * int64_t(j + u * bd)];
            a1[u] += cd[2 * int64_t(j + u * bd) + 1];
        }
#pragma unroll
    for (int u = 0; u < 3; ++u)
        if (j + u * bd < nc) {
            a0[u] += cd[2 * int64_t(j + u * bd)];
            a1[u] += cd[2 * int64_t(j + u * bd) + 1];
        }
    d[0] = (a0[0] + a0[1]) + (a0[2] + a0[3]);
    d[1] = (a1[0] + a1[1]) + (a1[2] + a1[3]);
}

__device__ void pcg_decide(Ctl* c, const double* tot, double* hist, int p, int nb);

// alpha = gamma / Delta; x += alpha p; r -= alpha q; z = D^{-1} r; totals of |r|^2, q^T z, r^T z,
// then (the CTA that finalises the totals) the stop test and beta.
// Delta and gamma are the sums over the problem's cameras (camera order) of the per-camera sums
// of the product; every CTA forms them the same way, CTA 0 stores them for the decide step.
// Thread = one row (9 per camera, kUpdCams cameras per CTA); the rows of a camera meet in
// shared memory for z = D^{-1} r.  CTA b of a problem takes its cameras [b kUpdCams, ...), so the
// partition depends on the problem alone (the grid has a CTA for every chunk of the largest).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pcg_update(const double* __restrict__ Dinv, const T* __restrict__ P,
                                                         const T* __restrict__ Q, T* __restrict__ x,
                                                         T* __restrict__ r, T* __restrict__ z,
                                                         const double* __restrict__ camdot,
                                                         double* __restrict__ totals, double* __restrict__ dpart,
                                                         int* __restrict__ dcnt, double* __restrict__ hist,
                                                         Ctl* ctl) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const int p = blockIdx.y;
    const Ctl& c = ctl[p];
    if (c.done) return;
    const int64_t c0 = c.lay.c0;
    const int nc = c.lay.nc;
    __shared__ double dg[2];
    __shared__ T sr[kUpdCams * 9];
    const int t = threadIdx.x, cl = t / 9, a = t - 9 * (t / 9);
    const int64_t jl = int64_t(blockIdx.x) * kUpdCams + cl;
    const bool act = t < kUpdCams * 9 && jl < nc;
    double drow[9];   // this row of the camera's D^{-1} block, requested before the CTA sum waits
    {
        double d[2];
        sum_camdot(camdot + 2 * c0, nc, d);
#pragma unroll
        for (int b = 0; b < 9; ++b) drow[b] = act ? Dinv[81 * (c0 + jl) + 9 * a + b] : 0.0;
        cta_sum_write<2>(d, dg);
    }
    double* tot = totals + int64_t(p) * kTotals;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        tot[0] = dg[0];
        tot[1] = dg[1];
    }
    // alpha = gamma / Delta; the float32 sweeps divide the rounded operands in float32 (a float64
    // division is a long dependent chain on this GPU's narrow float64 pipe)
    T alpha;
    if constexpr (sizeof(T) == 4) alpha = __fdiv_rn(float(dg[1]), float(dg[0]));
    else alpha = dg[1] * fast_rcp<2>(dg[0]);
    const int64_t hb = c.lay.hoff - 9 * c0;
    const int64_t i = 9 * (c0 + jl) + a;
    double v[3] = {0.0, 0.0, 0.0};
    T rv = T(0), qv = T(0);
    if (act) {
        x[i] = x[i] + alpha * P[hb + i];
        qv = Q[hb + i];
        rv = r[i] - alpha * qv;
        r[i] = rv;
        v[0] = double(rv) * double(rv);
    }
    if (t < kUpdCams * 9) sr[t] = rv;
    __syncthreads();
    if (act) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < 9; ++b) s += drow[b] * double(sr[9 * cl + b]);
        const T zs = T(s);
        z[i] = zs;
        v[1] = double(qv) * double(zs);
        v[2] = double(rv) * double(zs);
    }
    if (grid_sum_finalize<3>(v, dpart + int64_t(p) * gridDim.x * 3, dcnt + 4 * p, tot + 2) && threadIdx.x == 0)
        pcg_decide(ctl + p, tot, hist, p, gridDim.y);
}

// stop test and beta = Phi / Delta for problem p (one thread, after the update's totals are in);
// hist is iteration-major (it x nb)
__device__ void pcg_decide(Ctl* c, const double* tot, double* hist, int p, int nb) {
    if (c->status == BA_ERR_TIMEOUT) { c->done = 1; return; }
    const double D = tot[0], g = tot[1], rr = tot[2], phi = tot[3];
    const int it = c->it + 1;
    c->it = it;
    c->Delta = D;
    c->gamma = g;
    c->rr = rr;
    hist[int64_t(c->hist_off + it - 1) * nb + p] = rr * c->rr0_inv * c->hist_scale;   // squared relative residual
    if (!(D > 0.0) || !(rr == rr) || isinf(rr)) {
        c->done = 1;
        c->status = BA_ERR_BREAKDOWN;
    } else if (rr < c->tol2 * c->rr0) {
        c->done = 1;
        c->status = BA_OK;
    } else if (it >= c->max_iters) {
        c->done = 1;
        c->status = BA_ERR_NOT_CONVERGED;
    } else if (c->stag > 0.0 && g * g < c->stag * tot[4] * D) {   // (g^2 / D) / tot[4] < stag
        c->done = 1;          // no measurable progress left at this precision: end the sweep
        c->status = BA_OK;
    } else {
        c->beta = phi * fast_rcp<2>(D);
    }
}

// p = z - beta p (rows of the problem)
template <typename T>
__global__ void k_pcg_dir(const T* __restrict__ z, T* __restrict__ P, const Ctl* __restrict__ ctl) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const Ctl& c = ctl[blockIdx.y];
    if (c.done) return;
    const T beta = T(c.beta);
    const int64_t n = int64_t(c.lay.nc) * 9, r0 = 9 * int64_t(c.lay.c0);
    T* Pp = P + c.lay.hoff;
    for (int64_t i = gtid(); i < n; i += gstride()) Pp[i] = z[r0 + i] - beta * Pp[i];
}

// ---------------------------------------------------------------------------------------
// Algorithm 2

// Gram partials of Delta_i = Q_i^T P_i (w x w) and gamma_i = P_i^T r (w) for the current block.
// A problem of n rows uses min(gridDim.x, ceil(n / 128)) CTAs of its grid row (the rest return),
// each a contiguous run of rows, so the partition depends on the problem alone.
__device__ __forceinline__ int gram_ctas(int64_t n, int gx) {
    const int64_t g = (n + 127) / 128;
    return int(g < gx ? g : gx);
}

template <typename T>
__global__ void k_mcg_gram(const T* __restrict__ P, const T* __restrict__ Q, const T* __restrict__ r,
                           double* __restrict__ partial, const Ctl* __restrict__ ctl) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const int p = blockIdx.y;
    const Ctl& c = ctl[p];
    if (c.done) return;
    const int64_t n = int64_t(c.lay.nc) * 9;
    const int gp = gram_ctas(n, gridDim.x);
    if (int(blockIdx.x) >= gp) return;
    constexpr int TR = 128;   // rows staged at once: a problem's share of rows is usually one tile
    __shared__ T sP[TR][kMaxDirs + 1], sQ[TR][kMaxDirs + 1], sr[TR];
    const int w = c.w_cur, off = c.off_cur;
    const int ne = w * w + w;
    const T* Pp = P + c.lay.hoff;
    const T* Qp = Q + c.lay.hoff;
    const T* rp = r + 9 * int64_t(c.lay.c0);
    const int64_t per = (n + gp - 1) / gp;
    const int64_t r0 = int64_t(blockIdx.x) * per;
    const int64_t r1 = r0 + per < n ? r0 + per : n;
    ExactSum<T> acc[2];   // entries threadIdx.x and threadIdx.x + 256
    for (int64_t base = r0; base < r1; base += TR) {
        const int rows = int(r1 - base < TR ? r1 - base : TR);
        for (int t = threadIdx.x; t < TR * kMaxDirs; t += blockDim.x) {
            const int rr = t % TR, cc = t / TR;   // a warp reads 32 consecutive rows of one column
            T pv = T(0), qv = T(0);
            if (rr < rows && cc < w) {
                pv = Pp[int64_t(off + cc) * n + base + rr];
                qv = Qp[int64_t(off + cc) * n + base + rr];
            }
            sP[rr][cc] = pv;
            sQ[rr][cc] = qv;
        }
        if (threadIdx.x < TR) sr[threadIdx.x] = int(threadIdx.x) < rows ? rp[base + threadIdx.x] : T(0);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = threadIdx.x + h * blockDim.x;
            if (e < ne) {
                const T* x = e < w * w ? &sQ[0][e / w] : &sP[0][e - w * w];
                const T* y = e < w * w ? &sP[0][e % w] : &sr[0];
                const int ys = e < w * w ? kMaxDirs + 1 : 1;
                dot_rows(acc[h], x, kMaxDirs + 1, y, ys, rows);
            }
        }
        __syncthreads();
    }
    double* out = partial + (int64_t(p) * gridDim.x + blockIdx.x) * kGramMax;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int e = threadIdx.x + h * blockDim.x;
        if (e < ne) store_partial(out + e, acc[h]);
    }
}

// Jacobi eigen-decomposition based pseudo-inverse of the symmetric w x w matrix in sA
// (w <= 16, blockDim >= 256).  Eigenvalues at or below w 2^-52 lambda_max are dropped.
// On return sX holds A^+.  sV is scratch.
__device__ void pinv_sym_jacobi(double (*sA)[kMaxDirs + 1], double (*sV)[kMaxDirs + 1],
                                double (*sX)[kMaxDirs + 1], int w) {
    __shared__ double cs[kMaxDirs][2];
    __shared__ int pp[kMaxDirs], pq[kMaxDirs];
    __shared__ double off_norm, tot_norm;
    __shared__ double lam[kMaxDirs];
    const int t = threadIdx.x;
    const int i = t / kMaxDirs, j = t % kMaxDirs;
    if (t < kMaxDirs * kMaxDirs) sV[i][j] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    const int m = (w + 1) & ~1;   // even player count (index w is a dummy when w is odd)
    for (int sweep = 0; sweep < 30 && w > 1; ++sweep) {
        if (t < 32) {
            double o = 0.0, a = 0.0;
            for (int e = t; e < w * w; e += 32) {
                const int x = e / w, y = e % w;
                const double v = sA[x][y] * sA[x][y];
                a += v;
                if (x != y) o += v;
            }
            o = warp_sum(o);
            a = warp_sum(a);
            if (t == 0) {
                off_norm = o;
                tot_norm = a;
            }
        }
        __syncthreads();
        if (!(off_norm > 1e-30 * tot_norm)) break;
        for (int round = 0; round < m - 1; ++round) {
            // round-robin pairing: player 0 fixed, the others rotate
            if (t < m / 2) {
                int a = (t == 0) ? 0 : 1 + (round + t - 1) % (m - 1);
                int b = 1 + (round + m - 2 - t) % (m - 1);
                if (t == 0) b = 1 + (round + m - 2) % (m - 1);
                int p = a < b ? a : b, q = a < b ? b : a;
                double c = 1.0, s = 0.0;
                if (q < w && p < w) {
                    double apq = sA[p][q];
                    if (fabs(apq) > 1e-300) {
                        double app = sA[p][p], aqq = sA[q][q];
                        double theta = (aqq - app) / (2.0 * apq);
                        double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        s = tt * c;
                    }
                }
                pp[t] = p;
                pq[t] = q;
                cs[t][0] = c;
                cs[t][1] = s;
            }
            __syncthreads();
            // rows: A <- J^T A
            double nv = 0.0, nvv = 0.0;
            int which = -1;
            if (t < kMaxDirs * kMaxDirs && i < w && j < w) {
                for (int k = 0; k < m / 2; ++k) {
                    if (pp[k] == i || pq[k] == i) { which = k; break; }
                }
                if (which >= 0 && pq[which] < w) {
                    const int p = pp[which], q = pq[which];
                    const double c = cs[which][0], s = cs[which][1];
                    nv = (i == p) ? c * sA[p][j] - s * sA[q][j] : s * sA[p][j] + c * sA[q][j];
                } else {
                    nv = sA[i][j];
                }
            }
            __syncthreads();
            if (t < kMaxDirs * kMaxDirs && i < w && j < w) sA[i][j] = nv;
            __syncthreads();
            // columns: A <- A J, V <- V J
            which = -1;
            if (t < kMaxDirs * kMaxDirs && i < w && j < w) {
                for (int k = 0; k < m / 2; ++k) {
                    if (pp[k] == j || pq[k] == j) { which = k; break; }
                }
                if (which >= 0 && pq[which] < w) {
                    const int p = pp[which], q = pq[which];
                    const double c = cs[which][0], s = cs[which][1];
                    nv = (j == p) ? c * sA[i][p] - s * sA[i][q] : s * sA[i][p] + c * sA[i][q];
                    nvv = (j == p) ? c * sV[i][p] - s * sV[i][q] : s * sV[i][p] + c * sV[i][q];
                } else {
                    nv = sA[i][j];
                    nvv = sV[i][j];
                }
            }
            __syncthreads();
            if (t < kMaxDirs * kMaxDirs && i < w && j < w) {
                sA[i][j] = nv;
                sV[i][j] = nvv;
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        double top = 0.0;
        for (int k = 0; k < w; ++k) top = fmax(top, sA[k][k]);
        const double thr = w * 2.220446049250313e-16 * top;
        for (int k = 0; k < w; ++k) lam[k] = (sA[k][k] > thr) ? 1.0 / sA[k][k] : 0.0;
    }
    __syncthreads();
    if (t < kMaxDirs * kMaxDirs && i < w && j < w) {
        double s = 0.0;
        for (int k = 0; k < w; ++k) s += sV[i][k] * lam[k] * sV[j][k];
        sX[i][j] = s;
    }
    __syncthreads();
}


// Inverse of the symmetric w x w matrix in sA by Gauss-Jordan sweeps on the diagonal (no
// pivoting), accepted only when it equals the pseudo-inverse: every sweep pivot must be positive
// (A positive definite), and with lambda_min(A) >= 1 / trace(A^{-1}) and lambda_max(A) <=
// trace(A), 1 / trace(A^{-1}) exceeding 1e3 times the threshold w 2^-52 trace(A) means no
// eigenvalue is dropped, so A^+ = A^{-1}.  Thread 16 i + j (of the first 256) owns entry (i, j);
// a sweep updates every entry once, and the owner of the next pivot forms its reciprocal right
// after its own update, so the dependent float64 chain is 16 reciprocals long and no other thread
// spends the narrow float64 pipe on it.  sA is left intact; sX receives A^{-1} (symmetrised).
// Returns false (sX undefined) when the certificate fails.
__device__ bool inverse_certified(double (*sA)[kMaxDirs + 1], double (*sX)[kMaxDirs + 1], int w) {
    __shared__ int ok;
    __shared__ double tr, trinv;
    __shared__ double rk[kMaxDirs];   // 1 / pivot k
    const int t = threadIdx.x;
    const int i = t / kMaxDirs, j = t % kMaxDirs;
    const bool in = t < kMaxDirs * kMaxDirs && i < w && j < w;
    if (t < kMaxDirs * kMaxDirs) sX[i][j] = in ? sA[i][j] : 0.0;
    if (t < 32) {
        double d = t < w ? sA[t][t] : 0.0;
        d = warp_sum(d);
        if (t == 0) {
            tr = d;
            const double p0 = sA[0][0];
            ok = p0 > 0.0;
            rk[0] = fast_rcp(p0);
        }
    }
    __syncthreads();
    for (int k = 0; k < w; ++k) {
        double v = 0.0;
        if (in) {
            const double r = rk[k];
            if (i == k && j == k) v = r;
            else if (i == k) v = sX[k][j] * r;
            else if (j == k) v = -sX[i][k] * r;
            else v = fma(-sX[i][k] * r, sX[k][j], sX[i][j]);
        }
        __syncthreads();
        if (in) {
            sX[i][j] = v;
            if (i == k + 1 && j == k + 1) {   // the next pivot
                if (!(v > 0.0)) ok = 0;
                rk[k + 1] = fast_rcp(v);
            }
        }
        __syncthreads();
    }
    double sym = 0.0;
    if (in) sym = 0.5 * (sX[i][j] + sX[j][i]);
    __syncthreads();
    if (in) sX[i][j] = sym;
    __syncthreads();
    if (t < 32) {
        double d = t < w ? sX[t][t] : 0.0;
        d = warp_sum(d);
        if (t == 0) trinv = d;
    }
    __syncthreads();
    if (!ok) return false;
    // 1 / trace(A^{-1}) > 1e3 thr, i.e. 1e3 thr trace(A^{-1}) < 1 (false for a NaN)
    const double thr = w * 2.220446049250313e-16 * tr;
    return 1e3 * thr * trinv < 1.0;
}

// Delta_i, gamma_i -> Delta_i^+ (stored for the reorthogonalisation), alpha_i, gamma^T alpha.
// One CTA of kSmallThreads per problem (the matrix work uses the first 256); gx is the width of
// the Gram grid.
constexpr int kSmallThreads = 1024;
template <typename T>
__global__ void __launch_bounds__(kSmallThreads) k_mcg_small(Ctl* ctl, const double* __restrict__ partial, int gx, double* __restrict__ dpinv,
                            int mi1) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const int p = blockIdx.x;
    Ctl* c = ctl + p;
    if (c->done) return;
    __shared__ double sA[kMaxDirs][kMaxDirs + 1], sV[kMaxDirs][kMaxDirs + 1], sX[kMaxDirs][kMaxDirs + 1];
    __shared__ double sg[kMaxDirs];
    __shared__ double sal[kMaxDirs];
    const int w = c->w_cur;
    const int it = c->it;
    const int ne = w * w + w;
    const int np = gram_ctas(int64_t(c->lay.nc) * 9, gx);
    const double* part = partial + int64_t(p) * gx * kGramMax;
    // Sum of the CTA partials of every entry.  The partials sit in L2, written by the Gram CTAs, so
    // the sum is bound by load latency: G lanes share an entry (G a power of two, as many as the
    // block allows, at most a warp); lane g of the group takes the partials b = g, g + G, ... into
    // eight interleaved sums (eight loads in flight), which are added in a fixed tree, and the
    // group's sums meet in a fixed shuffle tree.  The order depends on (w, np) alone.
    {
        int G = 1;
        while (G < 32 && 2 * G * ne <= int(blockDim.x)) G *= 2;
        const int per_round = int(blockDim.x) / G;
        for (int e0 = 0; e0 < ne; e0 += per_round) {
            const int e = e0 + int(threadIdx.x) / G, g = int(threadIdx.x) % G;
            // warps holding no entry of this pass skip the arithmetic (and their shuffles) whole
            if (e0 + int(threadIdx.x & ~31u) / G >= ne) continue;
            ExactSum<T> acc[8];
            if (e < ne) {
                int b = g;
                for (; b + 7 * G < np; b += 8 * G)
#pragma unroll
                    for (int k = 0; k < 8; ++k) load_partial(acc[k], part + int64_t(b + k * G) * kGramMax + e);
#pragma unroll
                for (int k = 0; k < 7; ++k)
                    if (b + k * G < np) load_partial(acc[k], part + int64_t(b + k * G) * kGramMax + e);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) combine(acc[k], acc[k + 4]);
            combine(acc[0], acc[2]);
            combine(acc[1], acc[3]);
            combine(acc[0], acc[1]);
            for (int o = G / 2; o > 0; o >>= 1) combine_shfl(acc[0], o);
            if (e < ne && g == 0) {
                const double s = acc[0].value();
                if (e < w * w) sA[e / w][e % w] = s;
                else sg[e - w * w] = s;
            }
        }
    }
    __syncthreads();
    // symmetrise
    double sym = 0.0;
    const int i = threadIdx.x / kMaxDirs, j = threadIdx.x % kMaxDirs;
    if (threadIdx.x < kMaxDirs * kMaxDirs && i < w && j < w) sym = 0.5 * (sA[i][j] + sA[j][i]);
    __syncthreads();
    if (threadIdx.x < kMaxDirs * kMaxDirs && i < w && j < w) sA[i][j] = sym;
    __syncthreads();
    if (w == 1) {
        if (threadIdx.x == 0) sX[0][0] = sA[0][0] > 0.0 ? 1.0 / sA[0][0] : 0.0;
        __syncthreads();
    } else if (!inverse_certified(sA, sX, w)) {
        pinv_sym_jacobi(sA, sV, sX, w);
        if (threadIdx.x == 0) c->pinv_steps += 1;
    }
    if (threadIdx.x < kMaxDirs * kMaxDirs) {
        dpinv[(int64_t(p) * mi1 + it) * kMaxDirs * kMaxDirs + threadIdx.x] = (i < w && j < w) ? sX[i][j] : 0.0;
    }
    // alpha = Delta^+ gamma and gamma^T alpha: thread (a, b) = 16 a + b forms one product, the
    // 16 lanes of row a add theirs in a fixed shuffle tree (short float64 chains)
    if (threadIdx.x < kMaxDirs * kMaxDirs) {
        double s = (i < w && j < w) ? sX[i][j] * sg[j] : 0.0;
#pragma unroll
        for (int o = kMaxDirs / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (j == 0 && i < w) {
            sal[i] = s;
            c->alpha_v[i] = s;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = int(threadIdx.x) < w ? sg[threadIdx.x] * sal[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) {
            c->ga = s;
            if (!(s == s)) { c->done = 1; c->status = BA_ERR_BREAKDOWN; }
        }
    }
}

__device__ void mcg_decide(Ctl* c, const double* tot, double* hist, int* blk_off, int* blk_w, int mi1, int p, int nb);

// x += P_i alpha; r -= Q_i alpha; z = D^{-1} r; totals of |r|^2 and r^T z, then (last CTA) the
// decide step (grid: CTAs x problems;
// thread = one row, as in k_pcg_update).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mcg_update(const double* __restrict__ Dinv, const T* __restrict__ P,
                                                         const T* __restrict__ Q, T* __restrict__ x,
                                                         T* __restrict__ r, T* __restrict__ z,
                                                         double* __restrict__ dpart, int* __restrict__ dcnt,
                                                         double* __restrict__ totals, double* __restrict__ hist,
                                                         int* __restrict__ blk_off, int* __restrict__ blk_w, int mi1,
                                                         Ctl* ctl) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const int p = blockIdx.y;
    const Ctl& c = ctl[p];
    if (c.done) return;
    const int64_t c0 = c.lay.c0;
    const int nc = c.lay.nc;
    const int64_t n = int64_t(nc) * 9;
    const int w = c.w_cur, off = c.off_cur;
    const T* Pp = P + c.lay.hoff + int64_t(off) * n;
    const T* Qp = Q + c.lay.hoff + int64_t(off) * n;
    __shared__ T sal[kMaxDirs];
    __shared__ T sr[kUpdCams * 9];
    const int t = threadIdx.x, cl = t / 9, a = t - 9 * (t / 9);
    const int64_t jl = int64_t(blockIdx.x) * kUpdCams + cl;
    const bool act = t < kUpdCams * 9 && jl < nc;
    double drow[9];   // this row of the camera's D^{-1} block, requested early
#pragma unroll
    for (int b = 0; b < 9; ++b) drow[b] = act ? Dinv[81 * (c0 + jl) + 9 * a + b] : 0.0;
    if (threadIdx.x < kMaxDirs) sal[threadIdx.x] = int(threadIdx.x) < w ? T(c.alpha_v[threadIdx.x]) : T(0);
    __syncthreads();
    const int64_t il = 9 * jl + a, i = 9 * c0 + il;
    double v[2] = {0.0, 0.0};
    T rv = T(0);
    if (act) {
        T dx = T(0), dr = T(0);
        for (int b = 0; b < w; ++b) {
            dx += Pp[int64_t(b) * n + il] * sal[b];
            dr += Qp[int64_t(b) * n + il] * sal[b];
        }
        x[i] = x[i] + dx;
        rv = r[i] - dr;
        r[i] = rv;
        v[0] = double(rv) * double(rv);
    }
    if (t < kUpdCams * 9) sr[t] = rv;
    __syncthreads();
    if (act) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < 9; ++b) s += drow[b] * double(sr[9 * cl + b]);
        const T zs = T(s);
        z[i] = zs;
        v[1] = double(rv) * double(zs);
    }
    double* tot = totals + int64_t(p) * kTotals + 8;
    if (grid_sum_finalize<2>(v, dpart + int64_t(p) * gridDim.x * 2, dcnt + 4 * p + 1, tot) && threadIdx.x == 0)
        mcg_decide(ctl + p, tot, hist, blk_off, blk_w, mi1, p, gridDim.y);
}

// stop test, tau-test and the layout of the next block for problem p (one thread, after the
// update's totals are in)
__device__ void mcg_decide(Ctl* c, const double* tot, double* hist, int* blk_off, int* blk_w, int mi1, int p, int nb) {
    if (c->status == BA_ERR_TIMEOUT) { c->done = 1; return; }
    const double rr = tot[0], rz = tot[1];
    const int it = c->it + 1;
    c->it = it;
    c->rr = rr;
    c->rz = rz;
    hist[int64_t(c->hist_off + it - 1) * nb + p] = rr * c->rr0_inv * c->hist_scale;   // squared relative residual
    if (!(rr == rr) || isinf(rr)) {
        c->done = 1;
        c->status = BA_ERR_BREAKDOWN;
        return;
    }
    if (rr < c->tol2 * c->rr0) {
        c->done = 1;
        c->status = BA_OK;
        return;
    }
    if (it >= c->max_iters) {
        c->done = 1;
        c->status = BA_ERR_NOT_CONVERGED;
        return;
    }
    if (!(rz > 0.0)) {
        c->done = 1;
        c->status = BA_ERR_BREAKDOWN;
        return;
    }
    // t_i = gamma^T alpha / r^T z (rz > 0), compared without the division
    const double ga = c->ga;
    if (c->stag > 0.0 && ga < c->stag * rz) {
        c->done = 1;      // no measurable progress left at this precision: end the sweep
        c->status = BA_OK;
        return;
    }
    const int local = (ga < c->tau * rz) ? 1 : 0;
    const int w = local ? c->n_eff : 1;
    if (c->cols + w > c->cap) {
        // history full: a float32 sweep ends here and the float64 refinement restarts it from the
        // true residual; a float64 solve cannot go on
        c->done = 1;
        c->status = c->stag > 0.0 ? BA_OK : BA_ERR_OOM;
        return;
    }
    c->local = local;
    c->local_steps += local;
    c->w_new = w;
    c->new_off = c->cols;
    c->hist_cols = c->cols;
    c->w_cur = w;
    c->off_cur = c->cols;
    blk_off[int64_t(p) * mi1 + it] = c->cols;
    blk_w[int64_t(p) * mi1 + it] = w;
    c->cols += w;
}

// partial sums of Q[:, c]^T z over row chunks inside each subset:
// phip[(c * n_eff + s) * K + k] for c < hist_cols (one warp per entry; grid: CTAs x problems)
template <typename T>
__global__ void k_mcg_phi(const T* __restrict__ Q, const T* __restrict__ z, double* __restrict__ phip,
                          const Ctl* __restrict__ ctl) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const Ctl& c = ctl[blockIdx.y];
    if (c.done) return;
    const int lane = threadIdx.x & 31;
    const int nc = c.lay.nc;
    const int64_t n = int64_t(nc) * 9;
    const int n_eff = c.n_eff, sz = c.sz, K = c.K;
    const int cz = (sz + K - 1) / K;
    const int64_t items = int64_t(c.hist_cols) * n_eff * K;
    const T* Qp = Q + c.lay.hoff;
    const T* zp = z + 9 * int64_t(c.lay.c0);
    double* ph = phip + c.lay.phoff;
    for (int64_t it = gtid() >> 5; it < items; it += gstride() >> 5) {
        const int k = int(it % K);
        const int64_t cs = it / K;
        const int s = int(cs % n_eff);
        const int64_t cc = cs / n_eff;
        int j0 = s * sz + k * cz;
        int j1 = j0 + cz;
        const int send = (s + 1) * sz < nc ? (s + 1) * sz : nc;
        if (j1 > send) j1 = send;
        const T* qc = Qp + cc * n;
        ExactSum<T> acc;
        for (int64_t row = int64_t(j0) * 9 + lane; row < int64_t(j1) * 9; row += 32) acc.add(qc[row], zp[row]);
        const double sum = warp_sum(acc.value());
        if (lane == 0) ph[it] = sum;
    }
}

// beta_{i,j} = Delta_j^+ Phi_{i,j} for every history block j, into beta rows (one warp per block);
// betat receives the same rows in the Krylov storage type (float32 sweeps), so the
// reorthogonalisation reads them without conversions.  Float64 additions form long dependent
// chains on this GPU, so the sums are interleaved: with 32 or more entries a lane carries up to 8
// entries side by side; with fewer, G lanes share an entry's partials (lane g of the group takes
// k = g, g + G, ... into 4 interleaved sums) and add them in a fixed shuffle tree.
template <typename T>
__global__ void k_mcg_beta(const double* __restrict__ phip, const double* __restrict__ dpinv,
                           const int* __restrict__ blk_off, const int* __restrict__ blk_w, double* __restrict__ beta,
                           T* __restrict__ betat, const Ctl* __restrict__ ctl, int mi1) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const int p = blockIdx.y;
    const Ctl& c = ctl[p];
    if (c.done) return;
    __shared__ double sphi[kThreads / 32][kMaxDirs * kMaxDirs];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nblk = c.it;   // blocks 0..it-1 are the history
    const int n_eff = c.n_eff, K = c.K, w = c.w_new, local = c.local;
    const int m = local ? K : n_eff * K;   // partials per Phi entry
    const double* ph = phip + c.lay.phoff;
    const int* bo = blk_off + int64_t(p) * mi1;
    const int* bw = blk_w + int64_t(p) * mi1;
    double* Bp = beta + c.lay.boff * kMaxDirs;
    T* Bt = betat + c.lay.boff * kMaxDirs;
    // block jb goes to warp (jb / gridDim.x) of CTA (jb mod gridDim.x): consecutive blocks on
    // different SMs, so their float64 products share no SM's float64 pipe
    for (int64_t jb = blockIdx.x + int64_t(gridDim.x) * wid; jb < nblk; jb += int64_t(gridDim.x) * (blockDim.x >> 5)) {
        const int off = bo[jb], wj = bw[jb];
        const int ne = wj * w;
        // entries e = lane + 32 u of this lane: (a, s) = (e / w, e mod w)
        int ea[8], es[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = lane + 32 * u;
            ea[u] = e / w;
            es[u] = e - w * ea[u];
        }
        // Phi_j (wj x w): entry (a, s) adds the partials of history column off + a over subset s
        // (local block) or over every subset (global block); they are contiguous
        auto src = [&](int a, int s2) -> const double* {
            const int64_t cc = off + a;
            return local ? ph + (cc * n_eff + s2) * K : ph + cc * n_eff * K;
        };
        if (ne >= 32) {
            double v[8];
            const double* sp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                v[u] = 0.0;
                sp[u] = src(ea[u], es[u]);
            }
            for (int k = 0; k < m; ++k)
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (lane + 32 * u < ne) v[u] += sp[u][k];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (lane + 32 * u < ne) sphi[wid][lane + 32 * u] = v[u];
        } else {
            int G = 1;
            while (2 * G * ne <= 32) G *= 2;
            const int e = lane / G, g = lane % G;
            double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
            if (e < ne) {
                const double* sp = src(e / w, e % w);
                int k = g;
                for (; k + 3 * G < m; k += 4 * G) {
                    v0 += sp[k];
                    v1 += sp[k + G];
                    v2 += sp[k + 2 * G];
                    v3 += sp[k + 3 * G];
                }
                if (k < m) v0 += sp[k];
                if (k + G < m) v1 += sp[k + G];
                if (k + 2 * G < m) v2 += sp[k + 2 * G];
            }
            double v = (v0 + v1) + (v2 + v3);
            for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (e < ne && g == 0) sphi[wid][e] = v;
        }
        __syncwarp();
        const double* Dp = dpinv + (int64_t(p) * mi1 + jb) * kMaxDirs * kMaxDirs;
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 0.0;
        for (int b2 = 0; b2 < wj; ++b2)
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (lane + 32 * u < ne) v[u] += Dp[ea[u] * kMaxDirs + b2] * sphi[wid][b2 * w + es[u]];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (lane + 32 * u < ne) {
                const int64_t o = int64_t(off + ea[u]) * kMaxDirs + es[u];
                Bp[o] = v[u];
                Bt[o] = T(v[u]);
            }
        }
        __syncwarp();
    }
}

// P_new = Z - P_hist beta, Q_new = (S Z) - Q_hist beta (Eq. 18; Q only when Q is updated rather than
// recomputed).  A tall-skinny product over the history: a CTA takes 32 consecutive rows of one
// problem, its kPqSlices warps split each 64-column tile of the history (warp k takes columns
// k, k + kPqSlices, ...; lane = row, so every column is read as 32 consecutive values), beta
// tiles are staged in shared memory, and the slices are added in slice order at the end.
// A one-column block (a global step) accumulates one column only.
constexpr int kPqSlices = 4;
template <typename T>
__global__ void __launch_bounds__(kPqSlices * 32) k_mcg_pq(T* __restrict__ P, T* __restrict__ Q,
                                                            const T* __restrict__ z, const T* __restrict__ beta,
                                                            T* __restrict__ PT, const Ctl* __restrict__ ctl) {
    wait_prior_grid();   // chained launch: the previous kernel's results are visible from here
    const Ctl& c = ctl[blockIdx.y];
    if (c.done) return;
    constexpr int TC = 64;
    constexpr int kBPer = TC * kMaxDirs / (kPqSlices * 32);   // beta values a thread stages per tile
    __shared__ __align__(16) T sB[TC][kMaxDirs];
    __shared__ T red[2][kPqSlices][32][kMaxDirs + 1];
    const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
    const int64_t n = int64_t(c.lay.nc) * 9;
    const int64_t r0g = 9 * int64_t(c.lay.c0);
    const int w = c.w_new, off = c.new_off, hc = c.hist_cols, local = c.local, sz = c.sz;
    const bool upd_q = !c.direct_q;
    T* Pp = P + c.lay.hoff;
    T* Qp = Q + c.lay.hoff;
    const T* Bp = beta + c.lay.boff * kMaxDirs;
    for (int64_t base = int64_t(blockIdx.x) * 32; base < n; base += int64_t(gridDim.x) * 32) {
        const int64_t row = base + lane;
        const bool act = row < n;
        T ap[kMaxDirs], aq[kMaxDirs];
#pragma unroll
        for (int s = 0; s < kMaxDirs; ++s) {
            ap[s] = T(0);
            aq[s] = T(0);
        }
        // beta tile c0 + TC is read into registers while tile c0 is used (its loads in flight)
        T bnext[kBPer];
        auto load_b = [&](int c0n) {
#pragma unroll
            for (int u = 0; u < kBPer; ++u) {
                const int t = threadIdx.x + u * blockDim.x;
                const int cc = t / kMaxDirs, s = t % kMaxDirs;
                bnext[u] = (c0n + cc < hc && s < w) ? Bp[int64_t(c0n + cc) * kMaxDirs + s] : T(0);
            }
        };
        load_b(0);
        for (int c0 = 0; c0 < hc; c0 += TC) {
            const int tc = hc - c0 < TC ? hc - c0 : TC;
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kBPer; ++u) {
                const int t = threadIdx.x + u * blockDim.x;
                sB[t / kMaxDirs][t % kMaxDirs] = bnext[u];
            }
            __syncthreads();
            if (c0 + TC < hc) load_b(c0 + TC);
            if (!act) continue;
            const T* pc = Pp + int64_t(c0) * n + row;
            const T* qc = Qp + int64_t(c0) * n + row;
            if (w == 1) {
#pragma unroll 4
                for (int cl = k; cl < tc; cl += kPqSlices) {
                    const T b0 = sB[cl][0];
                    ap[0] += pc[int64_t(cl) * n] * b0;
                    if (upd_q) aq[0] += qc[int64_t(cl) * n] * b0;
                }
            } else if (upd_q) {
#pragma unroll 2
                for (int cl = k; cl < tc; cl += kPqSlices) {
                    const T pv = pc[int64_t(cl) * n], qv = qc[int64_t(cl) * n];
#pragma unroll
                    for (int s = 0; s < kMaxDirs; ++s) {
                        ap[s] += pv * sB[cl][s];
                        aq[s] += qv * sB[cl][s];
                    }
                }
            } else {
#pragma unroll 4
                for (int cl = k; cl < tc; cl += kPqSlices) {
                    const T pv = pc[int64_t(cl) * n];
#pragma unroll
                    for (int s = 0; s < kMaxDirs; ++s) ap[s] += pv * sB[cl][s];
                }
            }
        }
#pragma unroll
        for (int s = 0; s < kMaxDirs; ++s) {
            red[0][k][lane][s] = ap[s];
            red[1][k][lane][s] = aq[s];
        }
        __syncthreads();
        if (k == 0 && act) {
            const int sub = int(row / 9) / sz;
            const T zr = z[r0g + row];
#pragma unroll
            for (int s = 0; s < kMaxDirs; ++s) {
                T sp = T(0), sq = T(0);
#pragma unroll
                for (int kk = 0; kk < kPqSlices; ++kk) {
                    sp += red[0][kk][lane][s];
                    sq += red[1][kk][lane][s];
                }
                const T pn = ((local ? (s == sub) : (s == 0)) ? zr : T(0)) - sp;
                if (s < w) {
                    Pp[int64_t(off + s) * n + row] = pn;
                    if (upd_q) Qp[int64_t(off + s) * n + row] -= sq;
                }
                // row-major copy of the new block for the multi-column product (zero past w)
                if (!upd_q) PT[(r0g + row) * kMaxDirs + s] = s < w ? pn : T(0);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// true residual t = -b~ - S x in float64; partial[2 j], partial[2 j + 1] = camera j's sums of
// t^2 and b~^2 (one warp per camera, all problems)

__global__ void k_true_residual(int32_t n_c, const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr,
                                const int32_t* __restrict__ col, const double* __restrict__ S,
                                const double* __restrict__ x, const double* __restrict__ bt, double* __restrict__ res,
                                double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        const int64_t rj = row_ptr[j], nj = row_ptr[j + 1] - rj, tb = tile_ptr[j];
        double acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = 0.0;
        for (int64_t q = lane; q < nj; q += 32) {
            const double* xk = x + int64_t(col[rj + q]) * 9;
            double xv[9];
#pragma unroll
            for (int b = 0; b < 9; ++b) xv[b] = xk[b];
            const double* sp = S + (tb * kTile + q) * 81;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
#pragma unroll
                for (int b = 0; b < 9; ++b) acc[a] += sp[9 * a + b] * xv[b];
            }
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = warp_sum(acc[a]);
        double tt = 0.0, bb = 0.0;
        if (lane < 9) {
            double sx = acc[0];
#pragma unroll
            for (int a = 1; a < 9; ++a) if (lane == a) sx = acc[a];
            const double b = bt[9 * j + lane];
            const double t = -b - sx;
            if (res) res[9 * j + lane] = t;
            tt = t * t;
            bb = b * b;
        }
        tt = warp_sum(tt);
        bb = warp_sum(bb);
        if (lane == 0) {
            partial[2 * j] = tt;
            partial[2 * j + 1] = bb;
        }
    }
}

// per problem: ctl.true_rr and ctl.bb from the per-camera partials (camera order)
__global__ void k_true_reduce(Ctl* ctl, const double* __restrict__ partial) {
    Ctl* c = ctl + blockIdx.x;
    const double* pp = partial + 2 * int64_t(c->lay.c0);
    const double a = sum_partials(pp, c->lay.nc, 2, 0);
    const double b = sum_partials(pp, c->lay.nc, 2, 1);
    if (threadIdx.x == 0) {
        c->true_rr = a;
        c->bb = b;
    }
}

// mixed precision: x64 += Lam (double) d32, the inner solution mapped back from the scaled system
// x += Lam d (a float32 sweep's correction, unscaled), and x split into double-float for the true
// residual that follows (its per-observation products take no float64 input)
__global__ void k_accumulate(int64_t n, const float* __restrict__ d, const double* __restrict__ lam,
                             double* __restrict__ x, float2* __restrict__ xd) {
    for (int64_t i = gtid(); i < n; i += gstride()) {
        const double v = x[i] + lam[i] * double(d[i]);
        x[i] = v;
        const float h = __double2float_rn(v);
        xd[i] = make_float2(h, __double2float_rn(v - double(h)));
    }
}

// refinement start: x = 0 and rt = -b~
__global__ void k_start_refine(int64_t n, const double* __restrict__ bt, double* __restrict__ x,
                               double* __restrict__ rt) {
    for (int64_t i = gtid(); i < n; i += gstride()) {
        x[i] = 0.0;
        rt[i] = -bt[i];
    }
}

// One CTA per problem: |b~|^2 (fixed order) and the refinement state at x = 0.
__global__ void k_outer_init(const Layout* __restrict__ lay, const double* __restrict__ bt, Outer* outer) {
    const Layout L = lay[blockIdx.x];
    const int64_t n = int64_t(L.nc) * 9;
    const double* b = bt + 9 * int64_t(L.c0);
    double v[1] = {0.0};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[0] += b[i] * b[i];
    __shared__ double s[1];
    cta_sum_write<1>(v, s);
    if (threadIdx.x == 0) {
        Outer o;
        memset(&o, 0, sizeof(o));
        o.bb = s[0];
        o.tr = s[0];
        o.tr_prev = s[0];
        o.status = s[0] == 0.0 ? BA_OK : BA_ERR_NOT_CONVERGED;
        o.active = s[0] == 0.0 ? 0 : 1;
        outer[blockIdx.x] = o;
    }
}

// Plan the next float32 sweep of every problem still refining: per sweep the inner solve reduces
// its residual by inner_tol; when what is left to reach tol is within ten times that, the sweep
// aims 3x past it so that it is the last one.  One CTA over all problems; sets the refinement
// loop's condition: another sweep when any problem takes part (count = 1: a loop pass has ended).
__global__ void k_refine_plan(Outer* outer, int nb, const Params* __restrict__ prm, cudaGraphConditionalHandle h,
                              int use_handle, Loops* lp, int count) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const double tol = prm->tol, inner_tol = prm->inner_tol;
    int mine = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        Outer* o = outer + b;
        o->swept = 0;
        if (!o->active) continue;
        if (o->sweeps >= prm->max_refine || o->iters >= prm->max_iters) {
            o->active = 0;
            continue;
        }
        const double need = tol * sqrt(o->bb) / sqrt(o->tr);
        double t = need > 0.1 * inner_tol ? fmax(0.3 * need, 0.1 * inner_tol) : inner_tol;
        if (t >= 1.0) t = 0.5;
        o->tol_in = t;
        o->max_in = prm->max_iters - o->iters;
        o->swept = 1;
        mine = 1;
    }
    if (mine) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (count) lp->outer += 1;
        if (use_handle) cudaGraphSetConditional(h, any ? 1u : 0u);
    }
}

// After a sweep and the float64 true residual: account the sweep and decide whether to go on.
__global__ void k_refine_after(const Ctl* __restrict__ ctl, Outer* outer, const Params* __restrict__ prm) {
    Outer* o = outer + blockIdx.x;
    const Ctl& c = ctl[blockIdx.x];
    if (threadIdx.x != 0 || !o->swept) return;
    const double tol = prm->tol;
    const int mcg = prm->mcg;
    o->sweeps += 1;
    o->iters += c.it;
    o->locals += c.local_steps;
    o->pinvs += c.pinv_steps;
    o->cols = mcg ? c.cols : 1;
    o->tr_prev = o->tr;
    o->tr = c.true_rr;
    if (c.status == BA_ERR_BREAKDOWN || c.status == BA_ERR_OOM || c.status == BA_ERR_TIMEOUT) {
        o->status = c.status;
        o->active = 0;
        return;
    }
    if (!(o->tr == o->tr)) {
        o->status = BA_ERR_BREAKDOWN;
        o->active = 0;
        return;
    }
    if (o->tr <= tol * tol * o->bb) {
        o->status = BA_OK;
        o->active = 0;
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host side

// What a captured solve graph depends on besides the per-solve Params: the algorithm, precision,
// loop body, work lists, wait bound and every buffer address (a reallocation bumps `allocs`).
struct GraphKey {
    int mcg = -1, fp32 = -1, chunk = 0, mi1 = 0, use_l = -1, epoch = -1, polls = -1, nb = -1, host = -1, cfg = -1;
    uint64_t allocs = ~uint64_t(0);   // buffer generation (any reallocation invalidates the graph)
    const void* ptrs[4] = {};
    bool operator==(const GraphKey& o) const {
        if (mcg != o.mcg || fp32 != o.fp32 || chunk != o.chunk || mi1 != o.mi1 || use_l != o.use_l ||
            epoch != o.epoch || polls != o.polls || nb != o.nb || host != o.host || cfg != o.cfg ||
            allocs != o.allocs)
            return false;
        for (int i = 0; i < 4; ++i) if (ptrs[i] != o.ptrs[i]) return false;
        return true;
    }
};

// Kernel launches of a solve graph before, per pass of and after its loops.
struct GraphCounts {
    int pre = 0, sweep = 0, body = 0, post = 0;
};

struct SolveExec {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    GraphCounts gc;
};

// device buffer that only grows
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Solver {
    int nb = 0;               // problems
    int64_t n = 0;            // 9 n_c over all problems
    int mi1 = 0;              // per-problem stride of the per-step arrays (max_iters + 1)
    int gx = 1;               // grid width of the per-camera kernels
    int gu = 1;               // grid width of the update kernels (kUpdCams cameras per CTA)
    int gg = 1;               // Gram grid width
    int gq = 1;               // grid width of the per-row kernels
    int gpq = 1;              // grid width of the reorthogonalisation (32-row blocks)
    int gphi = 1, gb = 1;     // Phi and beta grid widths
    int gcol = 1;             // grid width of the column pass of the symmetric product (a CTA per camera)
    std::vector<Layout> lay;  // of the current solve
    Buf P, Q, r, z, xw, PT, part_a, part_b, part_cam, dpinv, beta, betaf, phip, hist, blk_off, blk_w, ctl, outer, rt,
        lay_d, totals, dpart, dcnt, camdot, params, loops;
    Ctl* h_ctl = nullptr;     // pinned, nb
    Outer* h_outer = nullptr; // pinned, nb
    Params* h_params = nullptr;   // pinned staging of the per-solve arguments
    Loops* h_loops = nullptr;     // pinned
    double* h_hist = nullptr;     // pinned, nb x mi1 (iteration-major device history)
    size_t h_hist_n = 0;
    std::vector<std::vector<double>> host_hist;   // per problem, residual history of the last solve
    int64_t launches = 0;     // kernel executions issued by the current solve
    cudaStream_t cap_stream = nullptr, cap2 = nullptr, cap3 = nullptr;   // capture streams (nested loops)
    std::vector<SolveExec*> execs;   // instantiated solve graphs
    // work lists of the block-sparse products: whole rows, rows split by pose subset, and whole rows of
    // the upper triangle (the symmetric one-column products of mixed precision)
    ItemList items_g, items_l, items_u;
    Buf tb;                    // transposed terms of the symmetric product (kTbHead + 1 values per upper block)
    int items_cb = -1;         // item chunk rule the lists were built with (0 = the default)
    int items_l_dirs = -1;
    bool use_l = false;        // the current MCG solve splits rows by pose subset (n_dirs > 1)
    int epoch = 0;             // incremented whenever a work list is rebuilt (captured graphs hold them)
    int spmv_cfg = 0;          // shape of the one-column products (SpmvShape)
    void* mm_part = nullptr;   // k_spmm partials: items_g.n x 16 x 9
};

// Reallocations so far: captured graphs hold buffer addresses, so any reallocation forces a new
// capture (the graph key records this count).
static std::atomic<uint64_t> g_allocs{0};

static void grow(Buf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return;
    ++g_allocs;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        throw Error(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    b.bytes = bytes;
}
template <typename T>
static T* ptr(const Buf& b) {
    return static_cast<T*>(b.p);
}

// Default blocks per work item: 16 tiles.  Rows up to that length are one item; longer rows are
// split, and the row's pieces combined by the last one to finish.  The rule depends on nothing
// but the row, so a problem's products sum in the same order alone and in any batch.  (Measured
// on GB300: 512 is within 2 % of the best of 32 .. 1024 for a 1936-camera problem and a 64-problem
// batch; a rule that split small problems' rows finer was up to 3x slower on the batch.)
constexpr int kItemBlocks = 512;

// Items of the block-sparse product, problem by problem: each (row, segment) split into chunks of
// at most cb blocks (cb = forced_cb, else kItemBlocks).
// split = false: one segment per row; otherwise segment s of a row of problem b holds the blocks
// whose column camera lies in [c0 + s sz, c0 + (s + 1) sz), for s < n_eff (empty segments get
// one empty item, which writes zeros).
static std::vector<SpItem> build_items(const std::vector<int64_t>& h_row_ptr, const std::vector<int32_t>& h_col,
                                       const std::vector<Layout>& lay, bool split, int forced_cb) {
    std::vector<SpItem> out;
    int grp = 0;
    for (size_t b = 0; b < lay.size(); ++b) {
        const Layout& L = lay[b];
        const int cb = forced_cb > 0 ? forced_cb : kItemBlocks;
        const int nseg = split ? L.n_eff : 1;
        for (int32_t j = L.c0; j < L.c0 + L.nc; ++j) {
            const int64_t rj = h_row_ptr[j], nj = h_row_ptr[j + 1] - rj;
            const int32_t* cj = h_col.data() + rj;
            for (int g = 0; g < nseg; ++g) {
                int q0 = 0, q1 = int(nj);
                if (split) {
                    q0 = int(std::lower_bound(cj, cj + nj, L.c0 + g * L.sz) - cj);
                    q1 = int(std::lower_bound(cj, cj + nj, L.c0 + (g + 1) * L.sz) - cj);
                }
                const int nch = q1 > q0 ? (q1 - q0 + cb - 1) / cb : 1;
                for (int c = 0; c < nch; ++c) {
                    SpItem it;
                    it.row = j;
                    it.seg = g;
                    it.q0 = q0 + c * cb;
                    it.q1 = std::min(q1, q0 + (c + 1) * cb);
                    if (it.q1 < it.q0) it.q1 = it.q0;
                    it.grp = grp;
                    it.k = c;
                    it.ng = nch;
                    it.prob = int(b);
                    it.slot = int(out.size());
                    out.push_back(it);
                }
                ++grp;
            }
        }
    }
    return out;
}

// Order the items for a launch of W warps, NW per CTA, by the longest-processing-time rule: in
// decreasing cost (tiles of S, in quarter tiles, plus a quarter for the item's own sums and output),
// each item goes to the bin with the least cost so far (ties: the lower bin).  Bin b is run by warp
// (b % C) * NW + b / C of the C = W / NW CTAs, so that the largest items, which go to the first bins,
// are spread over the SMs instead of filling the first CTAs.  Warp g's items follow in their
// original order at wptr[g].  Chunks and slots are unchanged, so the sums are too.  (Round-robin
// over the 1936-camera upper triangle left the longest warp 1.4x the mean; this rule, 1.05x.)
static std::vector<int64_t> balance_items(std::vector<SpItem>& v, int64_t W, int64_t NW) {
    const int64_t n = int64_t(v.size());
    std::vector<int64_t> cost(n), idx(n);
    for (int64_t i = 0; i < n; ++i) {
        const SpItem& it = v[i];
        const int64_t tiles = it.q1 > it.q0 ? ((int64_t(it.q1) + 31) >> 5) - (it.q0 >> 5) : 0;
        cost[i] = 4 * tiles + 1;
    }
    std::iota(idx.begin(), idx.end(), int64_t(0));
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
    using Load = std::pair<int64_t, int64_t>;   // (cost so far, warp)
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int64_t g = 0; g < W; ++g) heap.push({0, g});
    const int64_t C = W / NW;
    std::vector<int64_t> owner(n), wptr(W + 1, 0);
    for (const int64_t i : idx) {
        const Load l = heap.top();
        heap.pop();
        const int64_t b = l.second;
        owner[i] = (b % C) * NW + b / C;
        heap.push({l.first + cost[i], b});
        ++wptr[owner[i] + 1];
    }
    for (int64_t g = 0; g < W; ++g) wptr[g + 1] += wptr[g];
    std::vector<int64_t> pos(wptr.begin(), wptr.end() - 1);
    std::vector<SpItem> out(n);
    for (int64_t i = 0; i < n; ++i) out[pos[owner[i]]++] = v[i];
    v.swap(out);
    return wptr;
}

static void free_items(ItemList& L) {
    if (L.items) cudaFree(const_cast<SpItem*>(L.items));
    if (L.cnt) cudaFree(L.cnt);
    if (L.part) cudaFree(L.part);
    if (L.wptr) cudaFree(const_cast<int64_t*>(L.wptr));
    L = ItemList();
}

// Upload a list, in the balanced order for W warps, NW per CTA (W > 0).
static void upload_items(ItemList& L, std::vector<SpItem> v, int64_t W, int64_t NW) {
    free_items(L);
    std::vector<int64_t> wptr;
    if (W > 0) wptr = balance_items(v, W, NW);
    SpItem* d = nullptr;
    BA_CUDA_TRY(cudaMalloc(&d, sizeof(SpItem) * (v.empty() ? 1 : v.size())));
    if (!v.empty()) BA_CUDA_TRY(cudaMemcpy(d, v.data(), sizeof(SpItem) * v.size(), cudaMemcpyHostToDevice));
    L.items = d;
    L.n = int64_t(v.size());
    int ngrp = 1, nprob = 0;
    for (const SpItem& it : v) {
        ngrp = std::max(ngrp, it.grp + 1);
        nprob = std::max(nprob, it.prob + 1);
    }
    L.ngrp = ngrp;
    L.nprob = nprob;
    BA_CUDA_TRY(cudaMalloc(&L.cnt, sizeof(int) * ngrp));
    BA_CUDA_TRY(cudaMemset(L.cnt, 0, sizeof(int) * ngrp));
    BA_CUDA_TRY(cudaMalloc(&L.part, sizeof(double) * 9 * (v.size() > 0 ? v.size() : 1)));
    if (W > 0) {
        int64_t* dw = nullptr;
        BA_CUDA_TRY(cudaMalloc(&dw, sizeof(int64_t) * wptr.size()));
        BA_CUDA_TRY(cudaMemcpy(dw, wptr.data(), sizeof(int64_t) * wptr.size(), cudaMemcpyHostToDevice));
        L.wptr = dw;
        L.nw = W;
    }
}

// The tile-streaming products of every mode, precision and shape used here.
template <typename T, int MODE, bool ZH, bool SYM, int CFG>
static void set_spmv_attr() {
    BA_CUDA_TRY(cudaFuncSetAttribute(k_spmv<T, MODE, ZH, SYM, CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(spmv_smem<T, CFG>())));
}
template <int CFG>
static void set_spmv_attrs() {
    set_spmv_attr<float, 0, true, true, CFG>();
    set_spmv_attr<float, 1, true, true, CFG>();
    set_spmv_attr<float, 2, true, true, CFG>();
    set_spmv_attr<double, 0, true, false, CFG>();
    set_spmv_attr<double, 0, false, false, CFG>();
    set_spmv_attr<double, 1, true, false, CFG>();
}

static void set_smem_attrs() {
    static bool done = false;
    if (done) return;
    set_spmv_attrs<0>();
    set_spmv_attrs<1>();
    set_spmv_attrs<2>();
    BA_CUDA_TRY(cudaFuncSetAttribute(k_spmm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmm_smem<float>())));
    done = true;
}

template <typename T>
static int spmv_warps(int cfg) {
    return cfg == 1 ? SpmvShape<T, 1>::kWarps : (cfg == 2 ? SpmvShape<T, 2>::kWarps : SpmvShape<T, 0>::kWarps);
}

// (Re)build the work lists when the chunk rule, the subset layout or the warps of the kernel that
// streams a list changed.  Full pattern: k_spmm (float32) or k_spmv (float64); upper triangle and
// subset segments: k_spmv.
static void ensure_items(Solver* w, const Structure& s, int n_dirs, int forced_cb, bool fp32, int cfg) {
    const int cb = forced_cb > 0 ? forced_cb : 0;
    const int64_t sms = num_sms();
    const int64_t ng = fp32 ? SpmmCfg::kWarps : spmv_warps<double>(cfg);
    const int64_t nu = spmv_warps<float>(cfg), nl = spmv_warps<double>(cfg);
    const int64_t wg = sms * ng, wu = sms * nu, wl = sms * nl;
    const bool fresh = !w->items_g.items || w->items_cb != cb;
    if (fresh || w->items_g.nw != wg) {
        upload_items(w->items_g, build_items(s.h_row_ptr, s.h_col, w->lay, false, cb), wg, ng);
        if (w->mm_part) cudaFree(w->mm_part);
        w->mm_part = nullptr;
        BA_CUDA_TRY(cudaMalloc(&w->mm_part, sizeof(double) * kMaxDirs * 9 * size_t(w->items_g.n > 0 ? w->items_g.n : 1)));
        ++w->epoch;
    }
    if (!s.h_row_ptr_u.empty() && (fresh || w->items_u.nw != wu)) {
        upload_items(w->items_u, build_items(s.h_row_ptr_u, s.h_col_u, w->lay, false, cb), wu, nu);
        ++w->epoch;
    }
    if (fresh) {
        w->items_l_dirs = -1;
        w->items_cb = cb;
    }
    if (n_dirs > 1 && (w->items_l_dirs != n_dirs || w->items_l.nw != wl)) {
        upload_items(w->items_l, build_items(s.h_row_ptr, s.h_col, w->lay, true, cb), wl, nl);
        w->items_l_dirs = n_dirs;
        ++w->epoch;
    }
    w->use_l = n_dirs > 1;
    set_smem_attrs();
}

static int grid_for_host(int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    int cap = num_sms() * 8;
    return int(g < 1 ? 1 : (g > cap ? cap : g));
}

// Per-problem layout of a solve and the grid widths; buffers grow to fit.
static void prepare(Solver* w, const Structure& s, const SolveArgs& a, int n_dirs, bool fp32) {
    const int nb = int(s.h_cam_off.size()) - 1;
    std::vector<Layout> lay(nb);
    int64_t hoff = 0, phoff = 0, boff = 0;
    int nc_max = 1;
    for (int b = 0; b < nb; ++b) {
        Layout& L = lay[b];
        L.c0 = s.h_cam_off[b];
        L.nc = s.h_cam_off[b + 1] - L.c0;
        nc_max = std::max(nc_max, L.nc);
        const int nd = a.mcg ? n_dirs : 1;
        L.sz = (L.nc + nd - 1) / nd;
        L.n_eff = (L.nc + L.sz - 1) / L.sz;
        L.K = (L.sz + kChunkCams - 1) / kChunkCams;
        int64_t cap = 1;
        if (a.mcg) {
            cap = a.max_history > 0 ? a.max_history : int64_t(a.max_iters) * L.n_eff + 1;
            if (cap < 1 + L.n_eff) cap = 1 + L.n_eff;
            if (cap > (int64_t(1) << 30)) throw Error(BA_ERR_INVALID_ARG, "direction history too large");
        }
        L.cap = int(cap);
        L.hoff = hoff;
        L.phoff = phoff;
        L.boff = boff;
        hoff += cap * 9 * int64_t(L.nc);
        phoff += cap * L.n_eff * L.K;
        boff += cap;
    }
    const int64_t n = 9 * int64_t(s.n_c);
    const size_t elt = fp32 ? 4 : 8;
    const int G = num_sms() * 2;
    w->nb = nb;
    w->n = n;
    w->mi1 = std::max(w->mi1, a.max_iters + 1);
    w->gx = int(std::min<int64_t>(G, (nc_max + kThreads - 1) / kThreads));
    if ((int64_t(nc_max) + kUpdCams - 1) / kUpdCams > 65535) throw Error(BA_ERR_INVALID_ARG, "too many cameras in one problem");
    w->gu = (nc_max + kUpdCams - 1) / kUpdCams;
    w->gg = int(std::min<int64_t>(G, (9 * int64_t(nc_max) + 127) / 128));
    w->gq = std::max(1, G / nb);
    w->gpq = int(std::max<int64_t>(1, std::min<int64_t>((9 * int64_t(nc_max) + 31) / 32, 4 * G / nb)));
    w->gphi = std::max(1, 4 * G / nb);
    w->gb = std::max(1, G / nb);
    w->gcol = std::min(nc_max, std::max(1, 16 * G / nb));
    if (!w->h_ctl || int(w->lay.size()) != nb) {
        if (w->h_ctl) cudaFreeHost(w->h_ctl);
        if (w->h_outer) cudaFreeHost(w->h_outer);
        w->h_ctl = nullptr;
        w->h_outer = nullptr;
        BA_CUDA_TRY(cudaMallocHost(&w->h_ctl, sizeof(Ctl) * nb));
        BA_CUDA_TRY(cudaMallocHost(&w->h_outer, sizeof(Outer) * nb));
    }
    if (!w->cap_stream) BA_CUDA_TRY(cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking));
    if (!w->cap2) BA_CUDA_TRY(cudaStreamCreateWithFlags(&w->cap2, cudaStreamNonBlocking));
    if (!w->cap3) BA_CUDA_TRY(cudaStreamCreateWithFlags(&w->cap3, cudaStreamNonBlocking));
    if (!w->h_params) BA_CUDA_TRY(cudaMallocHost(&w->h_params, sizeof(Params)));
    if (!w->h_loops) BA_CUDA_TRY(cudaMallocHost(&w->h_loops, sizeof(Loops)));
    grow(w->P, size_t(hoff) * elt);
    grow(w->Q, size_t(hoff) * elt);
    grow(w->r, size_t(n) * elt);
    grow(w->z, size_t(n) * elt);
    grow(w->xw, size_t(n) * elt);
    grow(w->PT, size_t(n) * kMaxDirs * elt);
    grow(w->part_a, size_t(nb) * w->gg * kGramMax * sizeof(double));
    grow(w->part_b, size_t(nb) * w->gx * sizeof(double));
    grow(w->part_cam, size_t(s.n_c) * 2 * sizeof(double));
    grow(w->dpinv, size_t(nb) * w->mi1 * kMaxDirs * kMaxDirs * sizeof(double));
    grow(w->beta, size_t(boff) * kMaxDirs * sizeof(double));
    grow(w->betaf, size_t(boff) * kMaxDirs * sizeof(float));
    grow(w->phip, size_t(phoff) * sizeof(double));
    grow(w->hist, size_t(nb) * w->mi1 * sizeof(double));
    grow(w->blk_off, size_t(nb) * w->mi1 * sizeof(int));
    grow(w->blk_w, size_t(nb) * w->mi1 * sizeof(int));
    grow(w->ctl, size_t(nb) * sizeof(Ctl));
    grow(w->outer, size_t(nb) * sizeof(Outer));
    grow(w->rt, size_t(n) * sizeof(double));
    grow(w->lay_d, size_t(nb) * sizeof(Layout));
    grow(w->totals, size_t(nb) * kTotals * sizeof(double));
    grow(w->dpart, size_t(nb) * w->gu * 5 * sizeof(double));
    grow(w->camdot, size_t(s.n_c) * 2 * sizeof(double));
    grow(w->params, sizeof(Params));
    grow(w->loops, sizeof(Loops));
    if (w->h_hist_n < size_t(nb) * w->mi1) {
        if (w->h_hist) cudaFreeHost(w->h_hist);
        w->h_hist = nullptr;
        w->h_hist_n = 0;
        BA_CUDA_TRY(cudaMallocHost(&w->h_hist, sizeof(double) * size_t(nb) * w->mi1));
        w->h_hist_n = size_t(nb) * w->mi1;
    }
    if (w->dcnt.bytes < size_t(nb) * 4 * sizeof(int)) {
        grow(w->dcnt, size_t(nb) * 4 * sizeof(int));
        BA_CUDA_TRY(cudaMemset(w->dcnt.p, 0, w->dcnt.bytes));
    }
    BA_CUDA_TRY(cudaMemcpy(w->lay_d.p, lay.data(), sizeof(Layout) * nb, cudaMemcpyHostToDevice));
    w->lay = lay;
    w->spmv_cfg = a.spmv_cfg >= 0 && a.spmv_cfg < kSpmvShapes ? a.spmv_cfg : 0;
    ensure_items(w, s, a.mcg ? n_dirs : 1, a.item_blocks, fp32, w->spmv_cfg);
    w->items_g.polls = a.wait_polls;
    w->items_l.polls = a.wait_polls;
    w->items_u.polls = a.wait_polls;
    if (fp32 && s.n_up > 0) grow(w->tb, size_t(s.n_up) * (kTbHead + 1) * sizeof(float));
}

static void free_buf(Buf& b) {
    if (b.p) cudaFree(b.p);
    b = Buf();
}

Solver* solver_create() { return new Solver(); }

void solver_destroy(Solver* w) {
    if (!w) return;
    Buf* bufs[] = {&w->P, &w->Q, &w->r, &w->z, &w->xw, &w->PT, &w->part_a, &w->part_b, &w->part_cam, &w->dpinv,
                   &w->beta, &w->betaf, &w->phip, &w->hist, &w->blk_off, &w->blk_w, &w->ctl, &w->outer, &w->rt,
                   &w->lay_d, &w->totals, &w->dpart, &w->dcnt, &w->camdot, &w->params, &w->loops};
    for (Buf* b : bufs) free_buf(*b);
    for (SolveExec* e : w->execs) {
        cudaGraphExecDestroy(e->exec);
        delete e;
    }
    free_items(w->items_g);
    free_items(w->items_l);
    free_items(w->items_u);
    free_buf(w->tb);
    if (w->mm_part) cudaFree(w->mm_part);
    if (w->h_ctl) cudaFreeHost(w->h_ctl);
    if (w->h_outer) cudaFreeHost(w->h_outer);
    if (w->h_params) cudaFreeHost(w->h_params);
    if (w->h_loops) cudaFreeHost(w->h_loops);
    if (w->h_hist) cudaFreeHost(w->h_hist);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
    if (w->cap2) cudaStreamDestroy(w->cap2);
    if (w->cap3) cudaStreamDestroy(w->cap3);
    delete w;
}

int solver_history(const Solver* w, int problem, const double** hist) {
    if (problem < 0 || problem >= int(w->host_hist.size())) {
        *hist = nullptr;
        return 0;
    }
    *hist = w->host_hist[problem].data();
    return static_cast<int>(w->host_hist[problem].size());
}

// One launch of k_spmv in shape `cfg` (one CTA per SM).
// Launch with programmatic stream serialization (the kernels of a solve iteration): the kernel may
// be scheduled while the previous kernel on the stream drains and waits for it in wait_prior_grid,
// its first statement, instead of starting only after the previous grid has retired.
template <typename... K, typename... A>
static void launch_chained(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BA_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...));
}

template <typename T, int MODE, bool ZH, bool SYM, int CFG>
static void launch_spmv_cfg(cudaStream_t st, const int64_t* row_ptr, const int64_t* tile_ptr, const int32_t* col,
                            const T* S, const T* z, const ItemList& L, int sel, T* out, const T* rvec, double* camdot,
                            Ctl* ctl, T* tb, T* tb8, const int32_t* cslot) {
    launch_chained(k_spmv<T, MODE, ZH, SYM, CFG>, dim3(num_sms()), dim3(SpmvShape<T, CFG>::kWarps * 32),
                   spmv_smem<T, CFG>(), st, row_ptr, tile_ptr, col, S, z, L, sel, out, rvec, camdot, ctl, tb, tb8,
                   cslot);
}
template <typename T, int MODE, bool ZH, bool SYM>
static void launch_spmv(int cfg, cudaStream_t st, const int64_t* row_ptr, const int64_t* tile_ptr, const int32_t* col,
                        const T* S, const T* z, const ItemList& L, int sel, T* out, const T* rvec, double* camdot,
                        Ctl* ctl, T* tb, T* tb8 = nullptr, const int32_t* cslot = nullptr) {
    if (cfg == 1)
        launch_spmv_cfg<T, MODE, ZH, SYM, 1>(st, row_ptr, tile_ptr, col, S, z, L, sel, out, rvec, camdot, ctl, tb, tb8, cslot);
    else if (cfg == 2)
        launch_spmv_cfg<T, MODE, ZH, SYM, 2>(st, row_ptr, tile_ptr, col, S, z, L, sel, out, rvec, camdot, ctl, tb, tb8, cslot);
    else
        launch_spmv_cfg<T, MODE, ZH, SYM, 0>(st, row_ptr, tile_ptr, col, S, z, L, sel, out, rvec, camdot, ctl, tb, tb8, cslot);
}

// A one-column product y = S z, z a column of the direction history (modes of k_spmv).  With the upper
// triangle Su (float32) it is the symmetric product in two launches; float64 streams the full
// pattern (its products are bound by the float64 pipe, which halving the bytes would not relieve).
// Returns the launches.
template <typename T, int MODE>
static int enqueue_product(Solver* w, const Structure& s, const T* S, const T* Su, const T* zsrc, int sel, T* out,
                           const T* rvec, cudaStream_t st) {
    Ctl* ctl = ptr<Ctl>(w->ctl);
    double* camdot = MODE == 1 ? ptr<double>(w->camdot) : nullptr;
    if (Su) {
        T* tb = ptr<T>(w->tb);
        T* tb8 = tb + kTbHead * s.n_up;
        launch_spmv<T, MODE, true, true>(w->spmv_cfg, st, s.row_ptr_u, s.tile_ptr_u, s.col_u, Su, zsrc, w->items_u,
                                         sel, out, rvec, camdot, ctl, tb, tb8, s.cslot);
        launch_chained(k_spmv_col<T, MODE, true>, dim3(w->gcol, w->nb), dim3(kColWarps * 32), 0, st, s.qptr,
                       (const T*)tb, (const T*)tb8, zsrc, sel, out, rvec, camdot, ctl);
        return 2;
    }
    launch_spmv<T, MODE, true, false>(w->spmv_cfg, st, s.row_ptr, s.tile_ptr, s.col, S, zsrc, w->items_g, sel, out,
                                      rvec, camdot, ctl, nullptr);
    return 1;
}

// Enqueue one iteration of the chosen algorithm for every problem on `st`; returns the launches.
template <typename T>
static int enqueue_iteration(Solver* w, const Structure& s, const T* S, const T* Su, const double* Dinv, T* x,
                             bool mcg, cudaStream_t st) {
    const int nb = w->nb;
    T* P = ptr<T>(w->P);
    T* Q = ptr<T>(w->Q);
    T* r = ptr<T>(w->r);
    T* z = ptr<T>(w->z);
    Ctl* ctl = ptr<Ctl>(w->ctl);
    double* totals = ptr<double>(w->totals);
    int* dcnt = ptr<int>(w->dcnt);
    const int Gt = num_sms();   // tile-streaming products: one CTA per SM
    if (!mcg) {
        const int np = enqueue_product<T, 1>(w, s, S, Su, P, kSelLive, Q, r, st);
        launch_chained(k_pcg_update<T>, dim3(w->gu, nb), dim3(kThreads), 0, st, Dinv, P, Q, x, r, z,
                       ptr<double>(w->camdot), totals, ptr<double>(w->dpart), dcnt, ptr<double>(w->hist), ctl);
        launch_chained(k_pcg_dir<T>, dim3(w->gq, nb), dim3(kThreads), 0, st, z, P, ctl);
        return np + 2;
    } else {
        launch_chained(k_mcg_gram<T>, dim3(w->gg, nb), dim3(kThreads), 0, st, P, Q, r, ptr<double>(w->part_a), ctl);
        launch_chained(k_mcg_small<T>, dim3(nb), dim3(kSmallThreads), 0, st, ctl, ptr<double>(w->part_a), w->gg,
                       ptr<double>(w->dpinv), w->mi1);
        launch_chained(k_mcg_update<T>, dim3(w->gu, nb), dim3(kThreads), 0, st, Dinv, P, Q, x, r, z,
                       ptr<double>(w->dpart) + 3 * size_t(nb) * w->gu, dcnt, totals, ptr<double>(w->hist),
                       ptr<int>(w->blk_off), ptr<int>(w->blk_w), w->mi1, ctl);
        launch_chained(k_mcg_phi<T>, dim3(w->gphi, nb), dim3(kThreads), 0, st, Q, z, ptr<double>(w->phip), ctl);
        T* betat = sizeof(T) == 8 ? ptr<T>(w->beta) : ptr<T>(w->betaf);
        launch_chained(k_mcg_beta<T>, dim3(w->gb, nb), dim3(kThreads), 0, st, ptr<double>(w->phip),
                       ptr<double>(w->dpinv), ptr<int>(w->blk_off), ptr<int>(w->blk_w), ptr<double>(w->beta), betat,
                       ctl, w->mi1);
        if constexpr (sizeof(T) == 8) {
            // Eq. 18: Q_{i+1} = S Z_{i+1} - sum_j Q_j beta_{i,j}; S Z over whole rows for the
            // problems forming a global block, over the subset segments for the local ones
            launch_spmv<T, 0, false, false>(w->spmv_cfg, st, s.row_ptr, s.tile_ptr, s.col, S, z, w->items_g,
                                            w->use_l ? kSelGlobal : kSelLive, Q, nullptr, nullptr, ctl, nullptr);
            if (w->use_l)
                launch_spmv<T, 0, false, false>(w->spmv_cfg, st, s.row_ptr, s.tile_ptr, s.col, S, z, w->items_l,
                                                kSelLocal, Q, nullptr, nullptr, ctl, nullptr);
            launch_chained(k_mcg_pq<T>, dim3(w->gpq, nb), dim3(kPqSlices * 32), 0, st, P, Q, z, betat, (T*)nullptr,
                           ctl);
            return w->use_l ? 8 : 7;
        } else {
            // Algorithm 2: Q_{i+1} = S P_{i+1}
            launch_chained(k_mcg_pq<T>, dim3(w->gpq, nb), dim3(kPqSlices * 32), 0, st, P, Q, z, betat, ptr<T>(w->PT),
                           ctl);
            const int np = enqueue_product<T, 2>(w, s, S, Su, P, kSelW1, Q, nullptr, st);
            launch_chained(k_spmm<T>, dim3(Gt), dim3(SpmmCfg::kWarps * 32), spmm_smem<T>(), st, s.row_ptr, s.tile_ptr,
                           s.col, S, ptr<T>(w->PT), w->items_g, static_cast<T*>(w->mm_part), Q, ctl);
            return 7 + np;
        }
    }
}

// x = 0, r = sign * rhs, z = D^{-1} r, P_0 = z, the control blocks and (q0) Q_0 = S P_0; returns the
// launches.  Algorithm 2 starts its iterations from Q_0; Algorithm 1 forms Q = S P first in every
// iteration, so its solves pass q0 = false.
template <typename T>
static int krylov_init(Solver* w, const Structure& s, const T* S, const T* Su, const double* Dinv, const double* rhs,
                       double sign, const double* scale, T* x, const Outer* outer, cudaStream_t st, bool q0 = true) {
    const int nb = w->nb;
    k_init_vec<T><<<dim3(w->gx, nb), kThreads, 0, st>>>(ptr<Layout>(w->lay_d), rhs, sign, scale, Dinv, x, ptr<T>(w->r),
                                                         ptr<T>(w->z), ptr<T>(w->P), ptr<double>(w->part_b));
    k_init_ctl<<<nb, 32, 0, st>>>(ptr<Ctl>(w->ctl), ptr<Layout>(w->lay_d), ptr<double>(w->part_b), w->gx,
                                  ptr<Params>(w->params), sizeof(T) == 4 ? kStagnation : 0.0, sizeof(T) == 4 ? 1 : 0,
                                  outer, ptr<int>(w->blk_off), ptr<int>(w->blk_w), w->mi1);
    return 2 + (q0 ? enqueue_product<T, 0>(w, s, S, Su, ptr<T>(w->P), kSelLive, ptr<T>(w->Q), nullptr, st) : 0);
}

// true residual t = -b~ - S x into out (may be null) and, per problem, its norms into ctl (true_rr,
// bb): explicit tiled S in float64 precision, the implicit operator (double-float arithmetic) in mixed precision.
static int true_residual(Solver* w, const Structure& s, const System& y, const double* x, double* out,
                         cudaStream_t st) {
    int n = 0;
    if (y.S) {
        k_true_residual<<<grid_for_host(int64_t(s.n_c) * 32), kThreads, 0, st>>>(
            s.n_c, s.row_ptr, s.tile_ptr, s.col, y.S, x, y.bt, out, ptr<double>(w->part_cam));
        n = 1;
    } else {
        n = launch_implicit_residual(s, y, x, out, ptr<double>(w->part_cam), st);
    }
    k_true_reduce<<<w->nb, 32, 0, st>>>(ptr<Ctl>(w->ctl), ptr<double>(w->part_cam));
    return n + 1;
}

// ---- the solve graph: conditional WHILE nodes inserted into a stream capture ------------------

// A WHILE node on handle h after the current capture frontier of stream cs; the capture goes on after
// it.  Returns the (empty) body graph.
static cudaGraph_t capture_while(cudaStream_t cs, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus stat;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    BA_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &stat, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    BA_CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    BA_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return np.conditional.phGraph_out[0];
}

// A conditional handle of the graph being captured on cs (no default: set before the node runs).
static cudaGraphConditionalHandle capture_handle(cudaStream_t cs) {
    cudaStreamCaptureStatus stat;
    cudaGraph_t g = nullptr;
    BA_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &stat, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    BA_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    return h;
}

// The Krylov loop of one sweep, captured on cs: the sweep's start, then WHILE(any problem running) {
// chunk iterations; loop condition } on the body stream cb.
// Sets *pre (launches before the loop) and *per_pass (launches per pass of the loop).
template <typename T>
static void capture_krylov(Solver* w, const Structure& s, const T* S, const T* Su, const double* Dinv,
                           const double* rhs, double sign, const double* scale, T* x, const Outer* outer, bool mcg,
                           int chunk, cudaStream_t cs, cudaStream_t cb, int* pre, int* per_pass) {
    const cudaGraphConditionalHandle h = capture_handle(cs);
    *pre = krylov_init<T>(w, s, S, Su, Dinv, rhs, sign, scale, x, outer, cs, mcg) + 1;
    k_loop_cond<<<1, kThreads, 0, cs>>>(h, 1, ptr<Ctl>(w->ctl), w->nb, ptr<Loops>(w->loops), 1, chunk,
                                        ptr<Params>(w->params));
    cudaGraph_t body = capture_while(cs, h);
    BA_CUDA_TRY(cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    *per_pass = 1;
    for (int k = 0; k < chunk; ++k) *per_pass += enqueue_iteration<T>(w, s, S, Su, Dinv, x, mcg, cb);
    launch_chained(k_loop_cond, dim3(1), dim3(kThreads), 0, cb, h, 1, ptr<Ctl>(w->ctl), w->nb, ptr<Loops>(w->loops), 0,
                   chunk, ptr<Params>(w->params));
    cudaGraph_t done = nullptr;
    cudaError_t e = cudaStreamEndCapture(cb, &done);
    if (e != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("loop body capture: ") + cudaGetErrorString(e));
}



// Capture and instantiate the whole solve: float64 (Krylov loop and the true residual) or mixed
// precision (WHILE(a problem refines) { float32 Krylov loop; float64 true residual; plan the next
// sweep }).
static cudaGraphExec_t build_solve_graph(Solver* w, const Structure& s, const System& y, const SolveArgs& a,
                                         double* x, GraphCounts& gc) {
    const bool fp32 = a.precision == BA_PRECISION_MIXED;
    const bool mcg = a.mcg != 0;
    const int nb = w->nb;
    const int64_t n = int64_t(s.n_c) * 9;
    cudaStream_t cs = w->cap_stream;
    gc = GraphCounts();
    BA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        if (!fp32) {
            capture_krylov<double>(w, s, y.S, nullptr, y.Dinv, y.bt, -1.0, nullptr, x, nullptr, mcg, a.chunk, cs,
                                   w->cap2, &gc.pre, &gc.body);
            gc.post = true_residual(w, s, y, x, nullptr, cs);
        } else {
            k_start_refine<<<grid_for_host(n), kThreads, 0, cs>>>(n, y.bt, x, ptr<double>(w->rt));
            k_outer_init<<<nb, kThreads, 0, cs>>>(ptr<Layout>(w->lay_d), y.bt, ptr<Outer>(w->outer));
            const cudaGraphConditionalHandle ho = capture_handle(cs);
            k_refine_plan<<<1, kThreads, 0, cs>>>(ptr<Outer>(w->outer), nb, ptr<Params>(w->params), ho, 1,
                                                  ptr<Loops>(w->loops), 0);
            gc.pre = 3;
            cudaGraph_t body = capture_while(cs, ho);
            cudaStream_t c2 = w->cap2;
            BA_CUDA_TRY(cudaStreamBeginCaptureToGraph(c2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            int kpre = 0;
            capture_krylov<float>(w, s, y.S32, y.S32u, y.Dhat, ptr<double>(w->rt), 1.0, y.lam, ptr<float>(w->xw),
                                  ptr<Outer>(w->outer), mcg, a.chunk, c2, w->cap3, &kpre, &gc.body);
            k_accumulate<<<grid_for_host(n), kThreads, 0, c2>>>(n, ptr<float>(w->xw), y.lam, x, y.xd);
            const int tr = true_residual(w, s, y, x, ptr<double>(w->rt), c2);
            k_refine_after<<<nb, 32, 0, c2>>>(ptr<Ctl>(w->ctl), ptr<Outer>(w->outer), ptr<Params>(w->params));
            k_refine_plan<<<1, kThreads, 0, c2>>>(ptr<Outer>(w->outer), nb, ptr<Params>(w->params), ho, 1,
                                                  ptr<Loops>(w->loops), 1);
            gc.sweep = kpre + 1 + tr + 2;
            cudaGraph_t done = nullptr;
            cudaError_t e = cudaStreamEndCapture(c2, &done);
            if (e != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("refinement body capture: ") + cudaGetErrorString(e));
        }
    } catch (...) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(cs, &junk);
        if (junk) cudaGraphDestroy(junk);
        cudaGetLastError();
        throw;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("solve graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("solve graph instantiate: ") + cudaGetErrorString(e));
    return exec;
}

// Host-driven loops (ba_options.host_loop): a plain graph of chunk iterations and the pass counter,
// launched by the host until every problem is done.  gc.body receives its launches.
static cudaGraphExec_t build_chunk_graph(Solver* w, const Structure& s, const System& y, const SolveArgs& a,
                                         double* x, GraphCounts& gc) {
    const bool fp32 = a.precision == BA_PRECISION_MIXED;
    cudaStream_t cs = w->cap_stream;
    gc = GraphCounts();
    gc.body = 1;
    BA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < a.chunk; ++k)
        gc.body += fp32 ? enqueue_iteration<float>(w, s, y.S32, y.S32u, y.Dhat, ptr<float>(w->xw), a.mcg != 0, cs)
                        : enqueue_iteration<double>(w, s, y.S, nullptr, y.Dinv, x, a.mcg != 0, cs);
    k_loop_cond<<<1, kThreads, 0, cs>>>(cudaGraphConditionalHandle(), 0, ptr<Ctl>(w->ctl), w->nb,
                                        ptr<Loops>(w->loops), 0, a.chunk, ptr<Params>(w->params));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("chunk graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("chunk graph instantiate: ") + cudaGetErrorString(e));
    return exec;
}

// Launch the chunk graph until every problem's Ctl says done (at most the loop bound); returns the
// launches and counts the host waits.
static int64_t host_krylov_loop(Solver* w, cudaGraphExec_t chunk_exec, const GraphCounts& gc, const SolveArgs& a,
                                cudaStream_t st, int* waits) {
    const int nb = w->nb;
    const int bound = a.max_iters / a.chunk + 2;
    int64_t launches = 0;
    for (int c = 0; c <= bound; ++c) {
        BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl.p, sizeof(Ctl) * nb, cudaMemcpyDeviceToHost, st));
        BA_CUDA_TRY(cudaStreamSynchronize(st));
        ++*waits;
        bool all_done = true;
        for (int b = 0; b < nb && all_done; ++b) all_done = w->h_ctl[b].done != 0;
        if (all_done || c == bound) break;
        BA_CUDA_TRY(cudaGraphLaunch(chunk_exec, st));
        launches += gc.body;
    }
    return launches;
}

static void run_host_loops(Solver* w, const Structure& s, const System& y, const SolveArgs& a, double* x,
                           cudaGraphExec_t chunk_exec, const GraphCounts& gc, cudaStream_t st, int* waits) {
    const bool fp32 = a.precision == BA_PRECISION_MIXED;
    const int nb = w->nb;
    const int64_t n = int64_t(s.n_c) * 9;
    Loops* lp = ptr<Loops>(w->loops);
    const Params* prm = ptr<Params>(w->params);
    const cudaGraphConditionalHandle none = cudaGraphConditionalHandle();
    int64_t launches = 0;
    if (!fp32) {
        launches += krylov_init<double>(w, s, y.S, nullptr, y.Dinv, y.bt, -1.0, nullptr, x, nullptr, st, a.mcg != 0);
        k_loop_cond<<<1, kThreads, 0, st>>>(none, 0, ptr<Ctl>(w->ctl), nb, lp, 1, a.chunk, prm);
        launches += 1 + host_krylov_loop(w, chunk_exec, gc, a, st, waits);
        launches += true_residual(w, s, y, x, nullptr, st);
    } else {
        k_start_refine<<<grid_for_host(n), kThreads, 0, st>>>(n, y.bt, x, ptr<double>(w->rt));
        k_outer_init<<<nb, kThreads, 0, st>>>(ptr<Layout>(w->lay_d), y.bt, ptr<Outer>(w->outer));
        k_refine_plan<<<1, kThreads, 0, st>>>(ptr<Outer>(w->outer), nb, prm, none, 0, lp, 0);
        launches += 3;
        for (int sweep = 0; sweep <= a.max_refine; ++sweep) {
            BA_CUDA_TRY(cudaMemcpyAsync(w->h_outer, w->outer.p, sizeof(Outer) * nb, cudaMemcpyDeviceToHost, st));
            BA_CUDA_TRY(cudaStreamSynchronize(st));
            ++*waits;
            bool any = false;
            for (int b = 0; b < nb && !any; ++b) any = w->h_outer[b].swept != 0;
            if (!any) break;
            launches += krylov_init<float>(w, s, y.S32, y.S32u, y.Dhat, ptr<double>(w->rt), 1.0, y.lam,
                                           ptr<float>(w->xw), ptr<Outer>(w->outer), st, a.mcg != 0);
            k_loop_cond<<<1, kThreads, 0, st>>>(none, 0, ptr<Ctl>(w->ctl), nb, lp, 1, a.chunk, prm);
            launches += 1 + host_krylov_loop(w, chunk_exec, gc, a, st, waits);
            k_accumulate<<<grid_for_host(n), kThreads, 0, st>>>(n, ptr<float>(w->xw), y.lam, x, y.xd);
            launches += 1 + true_residual(w, s, y, x, ptr<double>(w->rt), st);
            k_refine_after<<<nb, 32, 0, st>>>(ptr<Ctl>(w->ctl), ptr<Outer>(w->outer), prm);
            k_refine_plan<<<1, kThreads, 0, st>>>(ptr<Outer>(w->outer), nb, prm, none, 0, lp, 1);
            launches += 2;
        }
    }
    BA_CUDA_TRY(cudaGetLastError());
    w->launches = launches;
}

// The instantiated graph for this solve (kept for the next solve of the same kind; a few kinds are
// kept, e.g. PCG and MCG in turn, and graphs that hold freed buffers are dropped).
static cudaGraphExec_t solve_graph(Solver* w, const Structure& s, const System& y, const SolveArgs& a, double* x,
                                   GraphCounts& gc) {
    const bool fp32 = a.precision == BA_PRECISION_MIXED;
    GraphKey key;
    key.mcg = a.mcg;
    key.fp32 = fp32;
    key.chunk = a.chunk;
    key.mi1 = w->mi1;
    key.use_l = w->use_l;
    key.epoch = w->epoch;
    key.polls = a.wait_polls;
    key.nb = w->nb;
    key.host = a.host_loop;
    key.cfg = a.spmv_cfg;
    key.allocs = g_allocs.load();
    const void* ptrs[4] = {x, fp32 ? (const void*)y.S32 : (const void*)y.S, w->items_g.items, w->items_l.items};
    for (int i = 0; i < 4; ++i) key.ptrs[i] = ptrs[i];
    for (size_t i = 0; i < w->execs.size();) {
        if (w->execs[i]->key.allocs != key.allocs) {
            cudaGraphExecDestroy(w->execs[i]->exec);
            delete w->execs[i];
            w->execs.erase(w->execs.begin() + i);
        } else {
            ++i;
        }
    }
    for (SolveExec* e : w->execs)
        if (e->key == key) {
            gc = e->gc;
            return e->exec;
        }
    SolveExec* e = new SolveExec();
    e->key = key;
    try {
        e->exec = a.host_loop ? build_chunk_graph(w, s, y, a, x, e->gc) : build_solve_graph(w, s, y, a, x, e->gc);
    } catch (...) {
        delete e;
        throw;
    }
    if (w->execs.size() >= 6) {
        cudaGraphExecDestroy(w->execs.front()->exec);
        delete w->execs.front();
        w->execs.erase(w->execs.begin());
    }
    w->execs.push_back(e);
    gc = e->gc;
    return e->exec;
}

void solver_run(Solver* w, const Structure& s, const System& y, const SolveArgs& a, double* x, SolveOut& out,
                cudaStream_t st) {
    int n_dirs = a.mcg ? a.n_dirs : 1;
    if (n_dirs < 1) n_dirs = 1;
    if (n_dirs > kMaxDirs) throw Error(BA_ERR_INVALID_ARG, "n_dirs must be in [1, 16]");
    const bool fp32 = a.precision == BA_PRECISION_MIXED;
    prepare(w, s, a, n_dirs, fp32);
    const int nb = w->nb;
    w->launches = 0;
    w->host_hist.assign(nb, std::vector<double>());
    GraphCounts gc;
    cudaGraphExec_t exec = solve_graph(w, s, y, a, x, gc);

    cudaEvent_t e0, e1;
    BA_CUDA_TRY(cudaEventCreate(&e0));
    BA_CUDA_TRY(cudaEventCreate(&e1));
    BA_CUDA_TRY(cudaEventRecord(e0, st));
    // the solve: its arguments in, one graph launch, the results out, one wait
    Params* hp = w->h_params;
    hp->tol = a.tol;
    hp->tau = a.tau;
    hp->inner_tol = a.inner_tol;
    hp->max_iters = a.max_iters;
    hp->max_refine = a.max_refine;
    hp->mcg = a.mcg;
    hp->pad = 0;
    BA_CUDA_TRY(cudaMemcpyAsync(w->params.p, hp, sizeof(Params), cudaMemcpyHostToDevice, st));
    BA_CUDA_TRY(cudaMemsetAsync(w->loops.p, 0, sizeof(Loops), st));
    int host_waits = 0;
    if (a.host_loop) run_host_loops(w, s, y, a, x, exec, gc, st, &host_waits);
    else BA_CUDA_TRY(cudaGraphLaunch(exec, st));
    BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl.p, sizeof(Ctl) * nb, cudaMemcpyDeviceToHost, st));
    if (fp32) BA_CUDA_TRY(cudaMemcpyAsync(w->h_outer, w->outer.p, sizeof(Outer) * nb, cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaMemcpyAsync(w->h_loops, w->loops.p, sizeof(Loops), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaMemcpyAsync(w->h_hist, w->hist.p, sizeof(double) * size_t(nb) * w->mi1, cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaEventRecord(e1, st));
    BA_CUDA_TRY(cudaEventSynchronize(e1));
    ++host_waits;
    BA_CUDA_TRY(cudaGetLastError());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);

    const Loops lp = *w->h_loops;
    if (!a.host_loop) w->launches = gc.pre + int64_t(lp.outer) * gc.sweep + int64_t(lp.inner) * gc.body + gc.post;
    out = SolveOut();
    out.probs.assign(nb, ProbOut());
    bool timed_out = false;
    for (int b = 0; b < nb; ++b) {
        ProbOut& o = out.probs[b];
        const Ctl& c = w->h_ctl[b];
        int steps = 0;
        if (!fp32) {
            o.status = c.done ? c.status : BA_ERR_NOT_CONVERGED;
            o.iters = c.it;
            o.local_steps = c.local_steps;
            o.pinv_steps = c.pinv_steps;
            o.history_cols = a.mcg ? c.cols : 1;
            o.rel_residual = c.rr0 > 0 ? std::sqrt(c.rr / c.rr0) : 0.0;
            o.refinements = 1;
            o.true_rel_residual = c.bb > 0 ? std::sqrt(c.true_rr / c.bb) : 0.0;
            steps = c.it;
        } else {
            const Outer& u = w->h_outer[b];
            o.status = u.status;
            o.iters = u.iters;
            o.local_steps = u.locals;
            o.pinv_steps = u.pinvs;
            o.history_cols = u.cols;
            o.refinements = u.sweeps;
            // tr is the float64 true residual of the problem's current x
            o.rel_residual = u.bb > 0 ? std::sqrt(u.tr / u.bb) : 0.0;
            o.true_rel_residual = o.rel_residual;
            steps = u.iters;
        }
        o.n_eff = w->lay[b].n_eff;
        timed_out = timed_out || o.status == BA_ERR_TIMEOUT;
        std::vector<double>& h = w->host_hist[b];
        h.resize(size_t(std::min(steps, w->mi1)));
        for (size_t i = 0; i < h.size(); ++i) h[i] = std::sqrt(w->h_hist[i * nb + b]);
    }
    if (timed_out) {
        // a warp whose tile wait gave up left its work item uncounted, so its group's arrival counter
        // did not return to zero: clear the counters for the next product
        if (w->items_g.cnt) BA_CUDA_TRY(cudaMemsetAsync(w->items_g.cnt, 0, sizeof(int) * w->items_g.ngrp, st));
        if (w->items_l.cnt) BA_CUDA_TRY(cudaMemsetAsync(w->items_l.cnt, 0, sizeof(int) * w->items_l.ngrp, st));
        BA_CUDA_TRY(cudaStreamSynchronize(st));
        ++host_waits;
    }
    out.launches = w->launches;
    out.host_waits = host_waits;
    out.ms = ms;
    // the batch's summary: the first failing problem's status, the largest counts and residuals
    out.status = BA_OK;
    out.n_eff = 1;
    for (int b = 0; b < nb; ++b) {
        const ProbOut& o = out.probs[b];
        if (out.status == BA_OK && o.status != BA_OK) out.status = o.status;
        out.iters = std::max(out.iters, o.iters);
        out.local_steps = std::max(out.local_steps, o.local_steps);
        out.pinv_steps = std::max(out.pinv_steps, o.pinv_steps);
        out.n_eff = std::max(out.n_eff, o.n_eff);
        out.refinements = std::max(out.refinements, o.refinements);
        out.history_cols = std::max(out.history_cols, o.history_cols);
        out.rel_residual = std::max(out.rel_residual, o.rel_residual);
        out.true_rel_residual = std::max(out.true_rel_residual, o.true_rel_residual);
    }
}

// Reads every 16 bytes of buf (n of them) and writes nothing unless they are all 0xff (never: the
// buffer is zeroed once): a read that the compiler cannot drop.
__global__ void k_l2_read(const uint4* __restrict__ buf, int64_t n, unsigned* sink) {
    const int64_t i0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    unsigned v = 0xffffffffu;
    for (int64_t i = i0; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint4 u = buf[i];
        v &= u.x & u.y & u.z & u.w;
    }
    if (i0 < n && v == 0xffffffffu) atomicAdd(sink, 1u);
}

// Evict L2 by reading a 256 MiB buffer (twice the cache).  A read leaves clean lines behind, so the
// timed kernel after it writes nothing back for earlier kernels (a written flush buffer would leave
// dirty lines whose write-back lands in the timed launch).
void flush_l2(cudaStream_t st) {
    static void* buf = nullptr;
    static unsigned* sink = nullptr;
    const size_t bytes = size_t(256) << 20;
    if (!buf) {
        BA_CUDA_TRY(cudaMalloc(&buf, bytes));
        BA_CUDA_TRY(cudaMalloc(&sink, sizeof(unsigned)));
        BA_CUDA_TRY(cudaMemset(buf, 0, bytes));
    }
    k_l2_read<<<num_sms() * 8, 256, 0, st>>>(static_cast<const uint4*>(buf), int64_t(bytes / 16), sink);
}

// The PCG product q = S p of every problem (k_spmv MODE 1, the kernel of Algorithm 1; in float32 the
// symmetric product, both of its launches), set up as at the start of a PCG solve (p = D^{-1} b~).
double solver_time_spmv(Solver* w, const Structure& s, const System& y, bool fp32, int reps, int item_blocks,
                        int spmv_cfg, cudaStream_t st) {
    SolveArgs a;
    a.mcg = 0;
    a.max_iters = 1;
    a.item_blocks = item_blocks;
    a.spmv_cfg = spmv_cfg;
    a.precision = fp32 ? BA_PRECISION_MIXED : BA_PRECISION_FP64;
    prepare(w, s, a, 1, fp32);
    Params* hp = w->h_params;
    *hp = Params();
    hp->tol = 1e-6;
    hp->max_iters = 1;
    BA_CUDA_TRY(cudaMemcpyAsync(w->params.p, hp, sizeof(Params), cudaMemcpyHostToDevice, st));
    if (fp32)
        krylov_init<float>(w, s, y.S32, y.S32u, y.Dhat, y.bt, -1.0, y.lam, ptr<float>(w->xw), nullptr, st);
    else
        krylov_init<double>(w, s, y.S, nullptr, y.Dinv, y.bt, -1.0, nullptr, ptr<double>(w->xw), nullptr, st);
    BA_CUDA_TRY(cudaGetLastError());
    cudaEvent_t e0, e1;
    BA_CUDA_TRY(cudaEventCreate(&e0));
    BA_CUDA_TRY(cudaEventCreate(&e1));
    double total = 0.0;
    for (int k = 0; k < reps; ++k) {
        flush_l2(st);
        BA_CUDA_TRY(cudaEventRecord(e0, st));
        if (fp32)
            enqueue_product<float, 1>(w, s, y.S32, y.S32u, ptr<float>(w->P), kSelLive, ptr<float>(w->Q),
                                      ptr<float>(w->r), st);
        else
            enqueue_product<double, 1>(w, s, y.S, nullptr, ptr<double>(w->P), kSelLive, ptr<double>(w->Q),
                                       ptr<double>(w->r), st);
        BA_CUDA_TRY(cudaEventRecord(e1, st));
        BA_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        BA_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        total += ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return total / reps;
}

// Shape and item chunk chosen by timing the PCG product: every shape with every chunk of 32 .. 1024
// blocks per work item, `reps` launches each; ties keep the earlier candidate.  The lists are left
// built for the winner.
void solver_autotune(Solver* w, const Structure& s, const System& y, bool fp32, int reps, int* best_cfg,
                     int* best_cb, double* best_ms, cudaStream_t st) {
    const int cands[] = {32, 64, 128, 256, 512, 1024};
    int bcfg = 0, bcb = 0;
    double bms = 0.0;
    for (int cfg = 0; cfg < kSpmvShapes; ++cfg)
        for (int cb : cands) {
            const double ms = solver_time_spmv(w, s, y, fp32, reps, cb, cfg, st);
            if (bcb == 0 || ms < bms) {
                bcfg = cfg;
                bcb = cb;
                bms = ms;
            }
        }
    solver_time_spmv(w, s, y, fp32, 1, bcb, bcfg, st);
    *best_cfg = bcfg;
    *best_cb = bcb;
    *best_ms = bms;
}

}  // namespace ba

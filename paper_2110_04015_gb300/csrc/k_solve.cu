// Krylov solvers of the reduced camera system S dx_p = -b~ (Section 3.2).
//
// Algorithm 1 (block-Jacobi PCG) and Algorithm 2 (MCG) run as a fixed sequence of
// kernels per iteration.  All data-dependent control (the stop test, the tau-test
// and the width of the next direction block, the history size) lives in a device
// struct Ctl written only by single-CTA "decide" kernels and read by the others, so a
// chunk of iterations is captured once as a CUDA graph and replayed; the host reads
// back one flag per chunk.  Multi-CTA kernels return at once when Ctl::done is set.
//
// Reductions are deterministic: each CTA writes a partial sum, and the consumer sums
// the partials in a fixed order.
//
// MCG data: the search blocks P_j and their images Q_j are kept as columns of two
// column-major arrays (column c at c * n, n = 9 n_cams); block j starts at column
// blk_off[j] and is blk_w[j] wide (1 for a global step, N_eff for a local one).  The
// pseudo-inverse of Delta_j is kept for the full reorthogonalisation
//     beta_{i,j} = Delta_j^+ Q_j^T Z_{i+1},  P_{i+1} = Z_{i+1} - sum_j P_j beta_{i,j},
//     Q_{i+1}   = S Z_{i+1} - sum_j Q_j beta_{i,j}            (Eq. 18 with j = 0..i)
// where S Z_{i+1} applies each block S_jk only to the column of the subset of pose k
// (Section 3.2, "Optimized implementation").
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ba_internal.cuh"

namespace ba {

namespace {

constexpr int kGramMax = kMaxDirs * kMaxDirs + kMaxDirs;   // Delta (w x w) and gamma (w)
constexpr int kChunkCams = 112;                             // cameras per Phi partial
constexpr double kStagnation = 1e-4;                        // float32 sweep stop on t_i (see Ctl::stag)

struct Ctl {
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
    double Delta, gamma, alpha, beta;   // PCG scalars
    double alpha_v[kMaxDirs];
    double true_rr, bb;                 // true residual and |rhs|^2
    double stag;       // float32 sweeps: stop when t_i (energy decrease / r^T D^-1 r) falls below this
    int direct_q;      // 1: Q_{i+1} = S P_{i+1} (Algorithm 2, line 3); 0: the Q update of Eq. 18
    int pad_;
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

// Sum `nv` values per thread over the CTA; thread 0 writes them to out[0..nv).
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
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Sum partial[p * stride + k] over p < np in a fixed order (called by one warp; lane 0 returns).
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
// otherwise).  The ng items of one output group (row, seg) are consecutive; each writes its 9
// partial sums, and the warp that finishes last (atomic count, no waiting) adds the partials in
// item order, so the result does not depend on scheduling.  Counters reset themselves.
struct SpItem {
    int row, seg, q0, q1, grp, k, ng, pad;
};

struct ItemList {
    const SpItem* items = nullptr;
    int64_t n = 0;
    int* cnt = nullptr;       // one per group, zero between launches
    void* part = nullptr;     // n x 9 partial sums (element type of the product)
};

// Sum the CTA's NV values, publish them as partial[blockIdx], and let the last CTA to finish
// write the grid totals (in CTA order) to totals[0..NV).  Every CTA of the grid must call it.
template <int NV>
__device__ __forceinline__ void grid_sum_finalize(double (&v)[NV], double* partial, int* cnt, double* totals) {
    __shared__ double red[kThreads / 32][NV];
    __shared__ int last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0) red[wid][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        partial[int64_t(blockIdx.x) * NV + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(cnt, 1) == int(gridDim.x) - 1);
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x < NV) {
            double s = 0.0;
            for (int b = 0; b < int(gridDim.x); ++b) s += __ldcg(partial + int64_t(b) * NV + threadIdx.x);
            totals[threadIdx.x] = s;
        }
        if (threadIdx.x == 0) *cnt = 0;
    }
}

// ---- bulk copies (cp.async.bulk + mbarrier) --------------------------------------------

constexpr int kMaxSpin = 1 << 20;   // bounded mbarrier waits: a copy that never lands ends the kernel

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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < kMaxSpin; ++i) {
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

// warps per CTA and copy stages of the tile-streaming product (one CTA per SM: the stages use
// 162 KB of shared memory in both precisions)
template <typename T>
struct SpmvCfg;
template <>
struct SpmvCfg<float> {
    static constexpr int kWarps = 8, kStages = 2;
};
template <>
struct SpmvCfg<double> {
    static constexpr int kWarps = 4, kStages = 2;
};
template <typename T>
constexpr size_t spmv_smem() {
    return sizeof(T) * SpmvCfg<T>::kWarps * SpmvCfg<T>::kStages * kTileElems +
           sizeof(uint64_t) * SpmvCfg<T>::kWarps * SpmvCfg<T>::kStages;
}

// Tile cursor of a warp: the tiles of items w0, w0 + W, ... in order, skipping empty items.
struct TileCursor {
    int64_t item;
    int t, te;
    int64_t base;
};
__device__ __forceinline__ void cursor_seek(TileCursor& c, const ItemList& L, const int64_t* tile_ptr, int64_t item,
                                            int64_t W) {
    for (; item < L.n; item += W) {
        const SpItem it = L.items[item];
        if (it.q1 > it.q0) {
            c.item = item;
            c.t = it.q0 >> 5;
            c.te = (it.q1 + 31) >> 5;
            c.base = tile_ptr[it.row];
            return;
        }
    }
    c.item = L.n;
    c.t = c.te = 0;
    c.base = 0;
}

// y(row, seg) = sum over the item's blocks of S_row,col(q) z_col(q).  Each warp streams the
// tiles of its items through kStages shared-memory buffers with bulk copies (issued by lane 0,
// NS tiles ahead) and multiplies them with the gathered z blocks.
// MODE 0: write y to column (off + seg) of `out` (off and the item list from ctl when use_ctl).
// MODE 1 (Algorithm 1, line 3-4): q = y, and the totals of Delta = q^T p and gamma = p^T r.
// MODE 2 (Algorithm 2, line 3, width 1): z is column new_off of P, y goes to the same column of out.
template <typename T, int MODE>
__global__ void __launch_bounds__(SpmvCfg<T>::kWarps * 32) k_spmv(
    const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr, const int32_t* __restrict__ col,
    const T* __restrict__ S, const T* __restrict__ z, ItemList gl, ItemList lo, T* __restrict__ out, int64_t n,
    const T* __restrict__ rvec, double* __restrict__ dpart, int* __restrict__ dcnt, double* __restrict__ totals,
    Ctl* ctl, int use_ctl) {
    constexpr int NW = SpmvCfg<T>::kWarps, NS = SpmvCfg<T>::kStages;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (use_ctl && ctl->done) return;
    if (MODE == 2 && ctl->w_new != 1) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T* tiles = reinterpret_cast<T*>(smem_raw) + size_t(wid) * NS * kTileElems;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * NW * NS * kTileElems) + wid * NS;
    const bool local = MODE == 0 && use_ctl && ctl->local;
    const ItemList L = local ? lo : gl;
    const int off = use_ctl ? ctl->new_off : 0;
    if (MODE == 2) z += int64_t(off) * n;
    T* part = static_cast<T*>(L.part);
    constexpr uint32_t tile_bytes = sizeof(T) * kTileElems;

    if (lane == 0) {
        for (int st = 0; st < NS; ++st) mbar_init(&bars[st]);
        fence_mbar_init();
    }
    __syncwarp();
    const int64_t W = int64_t(gridDim.x) * NW;
    const int64_t w0 = int64_t(blockIdx.x) * NW + wid;
    TileCursor f;
    cursor_seek(f, L, tile_ptr, w0, W);
    uint32_t parity = 0, inflight = 0;
    for (int st = 0; st < NS; ++st) {
        if (f.item < L.n) {
            if (lane == 0) bulk_load(tiles + st * kTileElems, S + (f.base + f.t) * kTileElems, tile_bytes, &bars[st]);
            inflight |= 1u << st;
            if (++f.t == f.te) cursor_seek(f, L, tile_ptr, f.item + W, W);
        }
    }
    int stage = 0;
    bool bad = false;
    double v[2] = {0.0, 0.0};
    for (int64_t i = w0; i < L.n && !bad; i += W) {
        const SpItem it = L.items[i];
        const int64_t rj = row_ptr[it.row];
        T acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = T(0);
        if (it.q1 > it.q0) {
            const int t0 = it.q0 >> 5, t1 = (it.q1 + 31) >> 5;
            // the 9 entries of z this lane needs for tile t, fetched one tile ahead
            T zn[9];
            {
                const int q = t0 * 32 + lane;
                const bool in = q >= it.q0 && q < it.q1;
                const T* zk = z + (in ? int64_t(col[rj + q]) * 9 : 0);
#pragma unroll
                for (int b = 0; b < 9; ++b) zn[b] = in ? zk[b] : T(0);
            }
            for (int t = t0; t < t1; ++t) {
                T zv[9];
#pragma unroll
                for (int b = 0; b < 9; ++b) zv[b] = zn[b];
                if (t + 1 < t1) {
                    const int qn = (t + 1) * 32 + lane;
                    const bool in = qn < it.q1;
                    const T* zk = z + (in ? int64_t(col[rj + qn]) * 9 : 0);
#pragma unroll
                    for (int b = 0; b < 9; ++b) zn[b] = in ? zk[b] : T(0);
                }
                // every lane observes the phase (visibility of the copied bytes); the warp agrees
                const bool ok = mbar_wait(&bars[stage], (parity >> stage) & 1u);
                if (!__all_sync(0xffffffffu, ok)) {
                    bad = true;
                    break;
                }
                parity ^= 1u << stage;
                inflight &= ~(1u << stage);
                const T* tile = tiles + stage * kTileElems;
                const int q = t * 32 + lane;
                if (q >= it.q0 && q < it.q1) {
                    const T* blk = tile + lane * 81;
#pragma unroll
                    for (int a = 0; a < 9; ++a)
#pragma unroll
                        for (int b = 0; b < 9; ++b) acc[a] += blk[9 * a + b] * zv[b];
                }
                __syncwarp();
                if (f.item < L.n) {
                    fence_proxy_async();
                    if (lane == 0)
                        bulk_load(tiles + stage * kTileElems, S + (f.base + f.t) * kTileElems, tile_bytes, &bars[stage]);
                    inflight |= 1u << stage;
                    if (++f.t == f.te) cursor_seek(f, L, tile_ptr, f.item + W, W);
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
            if (lane < 9) part[i * 9 + lane] = val;
            __threadfence();
            int last = 0;
            if (lane == 0) last = (atomicAdd(L.cnt + it.grp, 1) == it.ng - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            fin = last != 0;
            if (fin) {
                __threadfence();
                T sum = T(0);
                const int64_t first = i - it.k;
                if (lane < 9)
                    for (int c = 0; c < it.ng; ++c) sum += __ldcg(part + (first + c) * 9 + lane);
                val = sum;
                if (lane == 0) L.cnt[it.grp] = 0;
            }
        }
        if (fin && lane < 9) {
            const int64_t rowi = 9 * int64_t(it.row) + lane;
            if (MODE != 1) {
                out[int64_t(off + it.seg) * n + rowi] = val;
            } else {
                out[rowi] = val;
                const double pv = double(z[rowi]);
                v[0] += double(val) * pv;
                v[1] += pv * double(rvec[rowi]);
            }
        }
    }
    if (bad) {
        // a copy did not land in time: report, then wait (bounded) for this warp's copies in flight
        if (lane == 0) {
            atomicExch(&ctl->status, BA_ERR_TIMEOUT);
            atomicExch(&ctl->done, 1);
        }
        for (int st = 0; st < NS; ++st)
            if (inflight & (1u << st)) mbar_wait(&bars[st], (parity >> st) & 1u);
    }
    if (MODE == 1) grid_sum_finalize<2>(v, dpart, dcnt, totals);
}

// Q[:, off + c] = S P[:, off + c] for the w > 1 columns of a new local block (Algorithm 2, line 3,
// used by the float32 sweeps, where the Eq. 18 update cancels).  Tiles stream through shared memory
// as in k_spmv; lane = 4 qi + g takes tile-local blocks qi, qi + 8, qi + 16, qi + 24 and columns
// 4g .. 4g + 3, so each 9x9 block multiplies up to 16 columns per read from shared memory.
template <typename T>
constexpr size_t spmm_smem() {
    return spmv_smem<T>() + sizeof(T) * SpmvCfg<T>::kWarps * kMaxDirs * 9;
}

__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

template <typename T>
__global__ void __launch_bounds__(SpmvCfg<T>::kWarps * 32) k_spmm(
    const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr, const int32_t* __restrict__ col,
    const T* __restrict__ S, const T* __restrict__ PT, ItemList gl, T* __restrict__ part, T* __restrict__ Q, int64_t n,
    Ctl* ctl) {
    constexpr int NW = SpmvCfg<T>::kWarps, NS = SpmvCfg<T>::kStages;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (ctl->done) return;
    const int w = ctl->w_new;
    if (w <= 1) return;
    const int off = ctl->new_off;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int qi = lane >> 2, g = lane & 3;
    const int nout = 9 * w;
    T* tiles = reinterpret_cast<T*>(smem_raw) + size_t(wid) * NS * kTileElems;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * NW * NS * kTileElems) + wid * NS;
    T* red = reinterpret_cast<T*>(smem_raw + spmv_smem<T>()) + wid * (kMaxDirs * 9);
    constexpr uint32_t tile_bytes = sizeof(T) * kTileElems;
    const ItemList L = gl;
    if (lane == 0) {
        for (int st = 0; st < NS; ++st) mbar_init(&bars[st]);
        fence_mbar_init();
    }
    __syncwarp();
    const int64_t W = int64_t(gridDim.x) * NW;
    const int64_t w0 = int64_t(blockIdx.x) * NW + wid;
    TileCursor f;
    cursor_seek(f, L, tile_ptr, w0, W);
    uint32_t parity = 0, inflight = 0;
    for (int st = 0; st < NS; ++st) {
        if (f.item < L.n) {
            if (lane == 0) bulk_load(tiles + st * kTileElems, S + (f.base + f.t) * kTileElems, tile_bytes, &bars[st]);
            inflight |= 1u << st;
            if (++f.t == f.te) cursor_seek(f, L, tile_ptr, f.item + W, W);
        }
    }
    int stage = 0;
    bool bad = false;
    for (int64_t i = w0; i < L.n && !bad; i += W) {
        const SpItem it = L.items[i];
        const int64_t rj = row_ptr[it.row];
        T acc[9][4];
#pragma unroll
        for (int a = 0; a < 9; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
        if (it.q1 > it.q0) {
            const int t0 = it.q0 >> 5, t1 = (it.q1 + 31) >> 5;
            for (int t = t0; t < t1; ++t) {
                const bool ok = mbar_wait(&bars[stage], (parity >> stage) & 1u);
                if (!__all_sync(0xffffffffu, ok)) {
                    bad = true;
                    break;
                }
                parity ^= 1u << stage;
                inflight &= ~(1u << stage);
                const T* tile = tiles + stage * kTileElems;
                if (4 * g < w) {
#pragma unroll 1
                    for (int r = 0; r < 4; ++r) {
                        const int l = r * 8 + qi;
                        const int q = t * 32 + l;
                        if (q < it.q0 || q >= it.q1) continue;
                        // rows 9k .. 9k + 8, columns 4g .. 4g + 3 of the row-major copy PT (n x 16)
                        const T* pk = PT + (int64_t(col[rj + q]) * 9) * kMaxDirs + 4 * g;
                        T pv[9][4];
#pragma unroll
                        for (int b = 0; b < 9; ++b) load4(pk + b * kMaxDirs, pv[b]);
                        const T* blk = tile + l * 81;
#pragma unroll
                        for (int a = 0; a < 9; ++a)
#pragma unroll
                            for (int b = 0; b < 9; ++b) {
                                const T sab = blk[9 * a + b];
#pragma unroll
                                for (int c = 0; c < 4; ++c) acc[a][c] += sab * pv[b][c];
                            }
                    }
                }
                __syncwarp();
                if (f.item < L.n) {
                    fence_proxy_async();
                    if (lane == 0)
                        bulk_load(tiles + stage * kTileElems, S + (f.base + f.t) * kTileElems, tile_bytes, &bars[stage]);
                    inflight |= 1u << stage;
                    if (++f.t == f.te) cursor_seek(f, L, tile_ptr, f.item + W, W);
                }
                stage = stage + 1 == NS ? 0 : stage + 1;
            }
            if (bad) break;
        }
        // sum over the 8 lanes of each column group, then lanes 0..3 hold their columns
#pragma unroll
        for (int a = 0; a < 9; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                T v = acc[a][c];
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                acc[a][c] = v;
            }
        __syncwarp();
        if (qi == 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int cc = 4 * g + c;
                if (cc < w)
#pragma unroll
                    for (int a = 0; a < 9; ++a) red[cc * 9 + a] = acc[a][c];
            }
        }
        __syncwarp();
        bool fin = true;
        if (it.ng > 1) {
            for (int o = lane; o < nout; o += 32) part[i * (kMaxDirs * 9) + o] = red[o];
            __threadfence();
            int last = 0;
            if (lane == 0) last = (atomicAdd(L.cnt + it.grp, 1) == it.ng - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            fin = last != 0;
            if (fin) {
                __threadfence();
                const int64_t first = i - it.k;
                for (int o = lane; o < nout; o += 32) {
                    T sum = T(0);
                    for (int c = 0; c < it.ng; ++c) sum += __ldcg(part + (first + c) * (kMaxDirs * 9) + o);
                    red[o] = sum;
                }
                __syncwarp();
                if (lane == 0) L.cnt[it.grp] = 0;
            }
        }
        if (fin) {
            for (int o = lane; o < nout; o += 32) {
                const int cc = o / 9, a = o % 9;
                Q[int64_t(off + cc) * n + 9 * int64_t(it.row) + a] = red[o];
            }
        }
        __syncwarp();
    }
    if (bad) {
        if (lane == 0) {
            atomicExch(&ctl->status, BA_ERR_TIMEOUT);
            atomicExch(&ctl->done, 1);
        }
        for (int st = 0; st < NS; ++st)
            if (inflight & (1u << st)) mbar_wait(&bars[st], (parity >> st) & 1u);
    }
}

// ---------------------------------------------------------------------------------------
// initialisation shared by both algorithms: x = 0, r = sign * rhs, z = D^{-1} r, P_0 = z

template <typename T>
__global__ void k_init_vec(int32_t n_c, const double* __restrict__ rhs, double sign, const double* __restrict__ scale,
                           const double* __restrict__ Dinv, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                           T* __restrict__ P0, double* __restrict__ partial) {
    double v[1] = {0.0};
    for (int64_t j = gtid(); j < n_c; j += gstride()) {
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
            P0[9 * j + a] = T(s);
        }
    }
    cta_sum_write<1>(v, partial + blockIdx.x);
}

__global__ void k_init_ctl(Ctl* ctl, const double* __restrict__ partial, int np, double tol, int max_iters,
                           double tau, int n_eff, int sz, int K, int cap, int* blk_off, int* blk_w, double stag,
                           int direct_q) {
    double rr0 = sum_partials(partial, np, 1, 0);
    if (threadIdx.x == 0) {
        Ctl c;
        memset(&c, 0, sizeof(c));
        c.rr0 = rr0;
        c.rr = rr0;
        c.tol2 = tol * tol;
        c.tau = tau;
        c.max_iters = max_iters;
        c.n_eff = n_eff;
        c.sz = sz;
        c.K = K;
        c.cap = cap;
        c.cols = 1;
        c.w_new = 1;
        c.new_off = 0;
        c.local = 0;
        c.w_cur = 1;
        c.off_cur = 0;
        c.stag = stag;
        c.direct_q = direct_q;
        c.status = BA_OK;
        if (!(rr0 == rr0) || isinf(rr0)) { c.done = 1; c.status = BA_ERR_BREAKDOWN; }
        else if (rr0 == 0.0 || max_iters <= 0) { c.done = 1; c.status = rr0 == 0.0 ? BA_OK : BA_ERR_NOT_CONVERGED; }
        *ctl = c;
        blk_off[0] = 0;
        blk_w[0] = 1;
    }
}

// ---------------------------------------------------------------------------------------
// Algorithm 1

// alpha = gamma / Delta; x += alpha p; r -= alpha q; z = D^{-1} r; totals of |r|^2 and q^T z.
template <typename T>
__global__ void k_pcg_update(int32_t n_c, const double* __restrict__ Dinv, const T* __restrict__ p,
                             const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                             double* __restrict__ totals, double* __restrict__ dpart, int* __restrict__ dcnt,
                             const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    const T alpha = T(totals[1] / totals[0]);
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t j = gtid(); j < n_c; j += gstride()) {
        T rv[9], qv[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int64_t i = 9 * j + a;
            x[i] = x[i] + alpha * p[i];
            qv[a] = q[i];
            rv[a] = r[i] - alpha * qv[a];
            r[i] = rv[a];
            v[0] += double(rv[a]) * double(rv[a]);
        }
        const double* D = Dinv + 81 * j;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < 9; ++b) s += D[9 * a + b] * double(rv[b]);
            const T zs = T(s);
            z[9 * j + a] = zs;
            v[1] += double(qv[a]) * double(zs);
            v[2] += double(rv[a]) * double(zs);
        }
    }
    grid_sum_finalize<3>(v, dpart, dcnt, totals + 2);
}

// stop test and beta = Phi / Delta (one thread)
__global__ void k_pcg_decide(Ctl* ctl, const double* __restrict__ totals, double* hist) {
    if (ctl->done || threadIdx.x != 0) return;
    const double D = totals[0], g = totals[1], rr = totals[2], phi = totals[3];
    const int it = ctl->it + 1;
    ctl->it = it;
    ctl->Delta = D;
    ctl->gamma = g;
    ctl->alpha = g / D;
    ctl->rr = rr;
    hist[it - 1] = sqrt(rr / ctl->rr0);
    if (!(D > 0.0) || !(rr == rr) || isinf(rr)) {
        ctl->done = 1;
        ctl->status = BA_ERR_BREAKDOWN;
    } else if (rr < ctl->tol2 * ctl->rr0) {
        ctl->done = 1;
        ctl->status = BA_OK;
    } else if (it >= ctl->max_iters) {
        ctl->done = 1;
        ctl->status = BA_ERR_NOT_CONVERGED;
    } else if (ctl->stag > 0.0 && (g * g / D) < ctl->stag * totals[4]) {
        ctl->done = 1;          // no measurable progress left at this precision: end the sweep
        ctl->status = BA_OK;
    } else {
        ctl->beta = phi / D;
    }
}

// p = z - beta p
template <typename T>
__global__ void k_pcg_dir(int64_t n, const T* __restrict__ z, T* __restrict__ p, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    const T beta = T(ctl->beta);
    for (int64_t i = gtid(); i < n; i += gstride()) p[i] = z[i] - beta * p[i];
}

// ---------------------------------------------------------------------------------------
// Algorithm 2

// partials of Delta_i = Q_i^T P_i (w x w) and gamma_i = P_i^T r (w) for the current block
template <typename T>
__global__ void k_mcg_gram(int64_t n, const T* __restrict__ P, const T* __restrict__ Q, const T* __restrict__ r,
                           double* __restrict__ partial, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    constexpr int TR = 32;
    __shared__ T sP[TR][kMaxDirs + 1], sQ[TR][kMaxDirs + 1], sr[TR];
    const int w = ctl->w_cur, off = ctl->off_cur;
    const int ne = w * w + w;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = int64_t(blockIdx.x) * per;
    const int64_t r1 = r0 + per < n ? r0 + per : n;
    double acc[2] = {0.0, 0.0};   // entries threadIdx.x and threadIdx.x + 256
    for (int64_t base = r0; base < r1; base += TR) {
        const int rows = int(r1 - base < TR ? r1 - base : TR);
        for (int t = threadIdx.x; t < TR * kMaxDirs; t += blockDim.x) {
            const int rr = t / kMaxDirs, c = t % kMaxDirs;
            T pv = T(0), qv = T(0);
            if (rr < rows && c < w) {
                pv = P[int64_t(off + c) * n + base + rr];
                qv = Q[int64_t(off + c) * n + base + rr];
            }
            sP[rr][c] = pv;
            sQ[rr][c] = qv;
        }
        if (threadIdx.x < TR) sr[threadIdx.x] = threadIdx.x < rows ? r[base + threadIdx.x] : T(0);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = threadIdx.x + h * blockDim.x;
            if (e < ne) {
                double s = 0.0;
                if (e < w * w) {
                    const int a = e / w, b = e % w;
                    for (int k = 0; k < rows; ++k) s += double(sQ[k][a]) * double(sP[k][b]);
                } else {
                    const int a = e - w * w;
                    for (int k = 0; k < rows; ++k) s += double(sP[k][a]) * double(sr[k]);
                }
                acc[h] += s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int e = threadIdx.x + h * blockDim.x;
        if (e < ne) partial[int64_t(blockIdx.x) * kGramMax + e] = acc[h];
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
        if (t == 0) {
            double o = 0.0, a = 0.0;
            for (int x = 0; x < w; ++x)
                for (int y = 0; y < w; ++y) {
                    double v = sA[x][y] * sA[x][y];
                    a += v;
                    if (x != y) o += v;
                }
            off_norm = o;
            tot_norm = a;
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

// Cholesky inverse of the symmetric w x w matrix in sA, accepted only when it equals the pseudo-
// inverse: with A = L L^T, lambda_min(A) >= 1 / |L^{-1}|_F^2 and lambda_max(A) <= trace(A), so when
// 1 / |L^{-1}|_F^2 exceeds 1e3 times the threshold w 2^-52 trace(A) no eigenvalue is dropped and
// A^+ = A^{-1}.  sA is left intact; sL (lower factor, then L^{-1}) is scratch; sX receives A^{-1}.
// Returns false (sX undefined) when the certificate fails or a pivot is not positive.
__device__ bool inverse_certified(double (*sA)[kMaxDirs + 1], double (*sL)[kMaxDirs + 1],
                                  double (*sX)[kMaxDirs + 1], int w) {
    __shared__ int ok;
    __shared__ double fro, tr;
    const int t = threadIdx.x;
    const int i = t / kMaxDirs, j = t % kMaxDirs;
    if (t < kMaxDirs * kMaxDirs) sL[i][j] = (i < w && j < w && j <= i) ? sA[i][j] : 0.0;
    if (t == 0) {
        ok = 1;
        fro = 0.0;
        double s = 0.0;
        for (int k = 0; k < w; ++k) s += sA[k][k];
        tr = s;
    }
    __syncthreads();
    // right-looking Cholesky on the lower triangle
    for (int k = 0; k < w; ++k) {
        if (t == 0) {
            const double d = sL[k][k];
            if (!(d > 0.0)) ok = 0;
            sL[k][k] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (t > k && t < w) sL[t][k] /= sL[k][k];
        __syncthreads();
        if (t < kMaxDirs * kMaxDirs && i > k && j > k && j <= i && i < w) sL[i][j] -= sL[i][k] * sL[j][k];
        __syncthreads();
    }
    if (!ok) return false;
    // L^{-1} column by column (thread c solves column c), kept in sX temporarily
    if (t < w) {
        const int c = t;
        for (int r = 0; r < w; ++r) {
            double v = (r == c) ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) v -= sL[r][k] * sX[k][c];
            sX[r][c] = r < c ? 0.0 : v / sL[r][r];
        }
    }
    __syncthreads();
    if (t < kMaxDirs * kMaxDirs) sL[i][j] = (i < w && j < w) ? sX[i][j] : 0.0;   // sL <- L^{-1}
    __syncthreads();
    if (t < 32) {
        double f = 0.0;
        for (int e = t; e < w * w; e += 32) {
            const double v = sL[e / w][e % w];
            f += v * v;
        }
        f = warp_sum(f);
        if (t == 0) fro = f;
    }
    __syncthreads();
    const double lam_min_bound = 1.0 / fro;
    const double thr = w * 2.220446049250313e-16 * tr;
    if (!(lam_min_bound > 1e3 * thr)) return false;
    // A^{-1} = L^{-T} L^{-1}
    if (t < kMaxDirs * kMaxDirs && i < w && j < w) {
        double v = 0.0;
        const int k0 = i > j ? i : j;
        for (int k = k0; k < w; ++k) v += sL[k][i] * sL[k][j];
        sX[i][j] = v;
    }
    __syncthreads();
    return true;
}

// Delta_i, gamma_i -> Delta_i^+ (stored for the reorthogonalisation), alpha_i, gamma^T alpha.
__global__ void k_mcg_small(Ctl* ctl, const double* __restrict__ partial, int np, double* __restrict__ dpinv) {
    if (ctl->done) return;
    __shared__ double sA[kMaxDirs][kMaxDirs + 1], sV[kMaxDirs][kMaxDirs + 1], sX[kMaxDirs][kMaxDirs + 1];
    __shared__ double sg[kMaxDirs];
    __shared__ double sal[kMaxDirs];
    const int w = ctl->w_cur;
    const int it = ctl->it;
    const int ne = w * w + w;
    // one thread per entry sums the CTA partials in CTA order (independent loads, no shuffles)
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < np; ++b) s += partial[int64_t(b) * kGramMax + e];
        if (e < w * w) sA[e / w][e % w] = s;
        else sg[e - w * w] = s;
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
    } else if (!inverse_certified(sA, sV, sX, w)) {
        pinv_sym_jacobi(sA, sV, sX, w);
    }
    if (threadIdx.x < kMaxDirs * kMaxDirs) {
        dpinv[int64_t(it) * kMaxDirs * kMaxDirs + threadIdx.x] = (i < w && j < w) ? sX[i][j] : 0.0;
    }
    if (threadIdx.x < w) {
        double s = 0.0;
        for (int b = 0; b < w; ++b) s += sX[threadIdx.x][b] * sg[b];
        sal[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ga = 0.0;
        for (int a = 0; a < w; ++a) {
            ga += sg[a] * sal[a];
            ctl->alpha_v[a] = sal[a];
        }
        ctl->ga = ga;
        if (!(ga == ga)) { ctl->done = 1; ctl->status = BA_ERR_BREAKDOWN; }
    }
}

// x += P_i alpha; r -= Q_i alpha; z = D^{-1} r; totals of |r|^2 and r^T z.
template <typename T>
__global__ void k_mcg_update(int32_t n_c, const double* __restrict__ Dinv, const T* __restrict__ P,
                             const T* __restrict__ Q, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                             double* __restrict__ dpart, int* __restrict__ dcnt, double* __restrict__ totals,
                             const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    const int64_t n = int64_t(n_c) * 9;
    const int w = ctl->w_cur, off = ctl->off_cur;
    __shared__ T sal[kMaxDirs];
    if (threadIdx.x < kMaxDirs) sal[threadIdx.x] = threadIdx.x < w ? T(ctl->alpha_v[threadIdx.x]) : T(0);
    __syncthreads();
    double v[2] = {0.0, 0.0};
    for (int64_t j = gtid(); j < n_c; j += gstride()) {
        T rv[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int64_t i = 9 * j + a;
            T dx = T(0), dr = T(0);
            for (int b = 0; b < w; ++b) {
                dx += P[int64_t(off + b) * n + i] * sal[b];
                dr += Q[int64_t(off + b) * n + i] * sal[b];
            }
            x[i] = x[i] + dx;
            rv[a] = r[i] - dr;
            r[i] = rv[a];
            v[0] += double(rv[a]) * double(rv[a]);
        }
        const double* D = Dinv + 81 * j;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < 9; ++b) s += D[9 * a + b] * double(rv[b]);
            const T zs = T(s);
            z[9 * j + a] = zs;
            v[1] += double(rv[a]) * double(zs);
        }
    }
    grid_sum_finalize<2>(v, dpart, dcnt, totals);
}

// stop test, tau-test and the layout of the next block (one thread)
__global__ void k_mcg_decide(Ctl* ctl, const double* __restrict__ totals, double* hist, int* blk_off, int* blk_w) {
    if (ctl->done) return;
    const double rr = totals[0], rz = totals[1];
    if (threadIdx.x == 0) {
        const int it = ctl->it + 1;
        ctl->it = it;
        ctl->rr = rr;
        ctl->rz = rz;
        hist[it - 1] = sqrt(rr / ctl->rr0);
        if (!(rr == rr) || isinf(rr)) {
            ctl->done = 1;
            ctl->status = BA_ERR_BREAKDOWN;
            return;
        }
        if (rr < ctl->tol2 * ctl->rr0) {
            ctl->done = 1;
            ctl->status = BA_OK;
            return;
        }
        if (it >= ctl->max_iters) {
            ctl->done = 1;
            ctl->status = BA_ERR_NOT_CONVERGED;
            return;
        }
        if (!(rz > 0.0)) {
            ctl->done = 1;
            ctl->status = BA_ERR_BREAKDOWN;
            return;
        }
        const double t = ctl->ga / rz;
        if (ctl->stag > 0.0 && t < ctl->stag) {
            ctl->done = 1;      // no measurable progress left at this precision: end the sweep
            ctl->status = BA_OK;
            return;
        }
        const int local = (t < ctl->tau) ? 1 : 0;
        const int w = local ? ctl->n_eff : 1;
        if (ctl->cols + w > ctl->cap) {
            ctl->done = 1;
            ctl->status = BA_ERR_OOM;
            return;
        }
        ctl->local = local;
        ctl->local_steps += local;
        ctl->w_new = w;
        ctl->new_off = ctl->cols;
        ctl->hist_cols = ctl->cols;
        ctl->w_cur = w;
        ctl->off_cur = ctl->cols;
        blk_off[it] = ctl->cols;
        blk_w[it] = w;
        ctl->cols += w;
    }
}

// partial sums of Q[:, c]^T z over row chunks inside each subset:
// phip[(c * n_eff + s) * K + k] for c < hist_cols
template <typename T>
__global__ void k_mcg_phi(int32_t n_c, const T* __restrict__ Q, const T* __restrict__ z, double* __restrict__ phip,
                          const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t n = int64_t(n_c) * 9;
    const int n_eff = ctl->n_eff, sz = ctl->sz, K = ctl->K;
    const int cz = (sz + K - 1) / K;
    const int64_t items = int64_t(ctl->hist_cols) * n_eff * K;
    for (int64_t it = gtid() >> 5; it < items; it += gstride() >> 5) {
        const int k = int(it % K);
        const int64_t cs = it / K;
        const int s = int(cs % n_eff);
        const int64_t c = cs / n_eff;
        int j0 = s * sz + k * cz;
        int j1 = j0 + cz;
        const int send = (s + 1) * sz < n_c ? (s + 1) * sz : n_c;
        if (j1 > send) j1 = send;
        double acc = 0.0;
        const T* qc = Q + c * n;
        for (int64_t row = int64_t(j0) * 9 + lane; row < int64_t(j1) * 9; row += 32)
            acc += double(qc[row]) * double(z[row]);
        acc = warp_sum(acc);
        if (lane == 0) phip[it] = acc;
    }
}

// beta_{i,j} = Delta_j^+ Phi_{i,j} for every history block j, into B[c * 16 + s]
__global__ void k_mcg_beta(const double* __restrict__ phip, const double* __restrict__ dpinv,
                           const int* __restrict__ blk_off, const int* __restrict__ blk_w, double* __restrict__ B,
                           const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    __shared__ double sphi[kThreads / 32][kMaxDirs * kMaxDirs];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nblk = ctl->it;   // blocks 0..it-1 are the history
    const int n_eff = ctl->n_eff, K = ctl->K, w = ctl->w_new, local = ctl->local;
    for (int64_t jb = gtid() >> 5; jb < nblk; jb += gstride() >> 5) {
        const int off = blk_off[jb], wj = blk_w[jb];
        // Phi_j (wj x w)
        for (int e = lane; e < wj * w; e += 32) {
            const int a = e / w, s = e % w;
            const int64_t c = off + a;
            double v = 0.0;
            if (local) {
                for (int k = 0; k < K; ++k) v += phip[(c * n_eff + s) * K + k];
            } else {
                for (int ss = 0; ss < n_eff; ++ss)
                    for (int k = 0; k < K; ++k) v += phip[(c * n_eff + ss) * K + k];
            }
            sphi[wid][e] = v;
        }
        __syncwarp();
        const double* Dp = dpinv + int64_t(jb) * kMaxDirs * kMaxDirs;
        for (int e = lane; e < wj * w; e += 32) {
            const int a = e / w, s = e % w;
            double v = 0.0;
            for (int b = 0; b < wj; ++b) v += Dp[a * kMaxDirs + b] * sphi[wid][b * w + s];
            B[int64_t(off + a) * kMaxDirs + s] = v;
        }
        __syncwarp();
    }
}

// P_new = Z - P_hist B, Q_new = (S Z) - Q_hist B, one thread per row; B tiles staged in shared memory.
template <typename T>
__global__ void k_mcg_pq(int32_t n_c, T* __restrict__ P, T* __restrict__ Q, const T* __restrict__ z,
                         const double* __restrict__ B, T* __restrict__ PT, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    constexpr int TC = 64;
    __shared__ T sB[TC][kMaxDirs];
    const int64_t n = int64_t(n_c) * 9;
    const int w = ctl->w_new, off = ctl->new_off, hc = ctl->hist_cols, local = ctl->local, sz = ctl->sz;
    const bool upd_q = !ctl->direct_q;
    // every thread of the CTA walks all tiles, so the loop bounds are CTA-uniform
    const int64_t per_cta = (n + gridDim.x - 1) / gridDim.x;
    const int64_t rbeg = int64_t(blockIdx.x) * per_cta;
    const int64_t rend = rbeg + per_cta < n ? rbeg + per_cta : n;
    for (int64_t base = rbeg; base < rend; base += blockDim.x) {
        const int64_t row = base + threadIdx.x;
        const bool act = row < rend;
        T ap[kMaxDirs], aq[kMaxDirs];
        const int sub = act ? int(row / 9) / sz : 0;
        const T zr = act ? z[row] : T(0);
#pragma unroll
        for (int s = 0; s < kMaxDirs; ++s) {
            ap[s] = T(0);
            aq[s] = T(0);
            if (act && s < w) {
                ap[s] = (local ? (s == sub) : (s == 0)) ? zr : T(0);
                aq[s] = upd_q ? Q[int64_t(off + s) * n + row] : T(0);
            }
        }
        for (int c0 = 0; c0 < hc; c0 += TC) {
            const int tc = hc - c0 < TC ? hc - c0 : TC;
            __syncthreads();
            for (int t = threadIdx.x; t < TC * kMaxDirs; t += blockDim.x) {
                const int cc = t / kMaxDirs, s = t % kMaxDirs;
                sB[cc][s] = (cc < tc && s < w) ? T(B[int64_t(c0 + cc) * kMaxDirs + s]) : T(0);
            }
            __syncthreads();
            if (act) {
                if (upd_q) {
                    for (int cc = 0; cc < tc; ++cc) {
                        const T pv = P[int64_t(c0 + cc) * n + row];
                        const T qv = Q[int64_t(c0 + cc) * n + row];
#pragma unroll
                        for (int s = 0; s < kMaxDirs; ++s) {
                            ap[s] -= pv * sB[cc][s];
                            aq[s] -= qv * sB[cc][s];
                        }
                    }
                } else {
                    for (int cc = 0; cc < tc; ++cc) {
                        const T pv = P[int64_t(c0 + cc) * n + row];
#pragma unroll
                        for (int s = 0; s < kMaxDirs; ++s) ap[s] -= pv * sB[cc][s];
                    }
                }
            }
        }
        if (act) {
#pragma unroll
            for (int s = 0; s < kMaxDirs; ++s) {
                if (s < w) {
                    P[int64_t(off + s) * n + row] = ap[s];
                    if (upd_q) Q[int64_t(off + s) * n + row] = aq[s];
                }
                // row-major copy of the new block for the multi-column product (zero past w)
                if (!upd_q) PT[row * kMaxDirs + s] = s < w ? ap[s] : T(0);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// true residual t = -b~ - S x in float64 and |t|^2, |b~|^2 partials

__global__ void k_true_residual(int32_t n_c, const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr,
                                const int32_t* __restrict__ col, const double* __restrict__ S,
                                const double* __restrict__ x, const double* __restrict__ bt, double* __restrict__ res,
                                double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    double v[2] = {0.0, 0.0};
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
        if (lane < 9) {
            double sx = acc[0];
#pragma unroll
            for (int a = 1; a < 9; ++a) if (lane == a) sx = acc[a];
            const double b = bt[9 * j + lane];
            const double t = -b - sx;
            if (res) res[9 * j + lane] = t;
            v[0] += t * t;
            v[1] += b * b;
        }
    }
    cta_sum_write<2>(v, partial + 2 * blockIdx.x);
}

__global__ void k_true_reduce(Ctl* ctl, const double* __restrict__ partial, int np) {
    double a = sum_partials(partial, np, 2, 0);
    double b = sum_partials(partial, np, 2, 1);
    if (threadIdx.x == 0) {
        ctl->true_rr = a;
        ctl->bb = b;
    }
}

// mixed precision: x64 += Lam (double) d32, the inner solution mapped back from the scaled system
__global__ void k_accumulate(int64_t n, const float* __restrict__ d, const double* __restrict__ lam,
                             double* __restrict__ x) {
    for (int64_t i = gtid(); i < n; i += gstride()) x[i] += lam[i] * double(d[i]);
}

__global__ void k_zero(int64_t n, double* __restrict__ x) {
    for (int64_t i = gtid(); i < n; i += gstride()) x[i] = 0.0;
}

// refinement start: x = 0 and rt = -b~
__global__ void k_start_refine(int64_t n, const double* __restrict__ bt, double* __restrict__ x,
                               double* __restrict__ rt) {
    for (int64_t i = gtid(); i < n; i += gstride()) {
        x[i] = 0.0;
        rt[i] = -bt[i];
    }
}

// ctl->true_rr = ctl->bb = |v|^2 (one CTA, fixed summation order)
__global__ void k_norm2(int64_t n, const double* __restrict__ v, Ctl* ctl) {
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i] * v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (int(threadIdx.x) < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctl->true_rr = red[0];
        ctl->bb = red[0];
    }
}

template <typename T>
__global__ void k_copy_out(int64_t n, const T* __restrict__ x, double* __restrict__ out) {
    for (int64_t i = gtid(); i < n; i += gstride()) out[i] = double(x[i]);
}

__global__ void k_to_float_vec(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    for (int64_t i = gtid(); i < n; i += gstride()) out[i] = float(in[i]);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host side

struct GraphKey {
    int mcg = -1, fp32 = -1, chunk = 0;
    const void* ptrs[12] = {};
    bool operator==(const GraphKey& o) const {
        if (mcg != o.mcg || fp32 != o.fp32 || chunk != o.chunk) return false;
        for (int i = 0; i < 12; ++i) if (ptrs[i] != o.ptrs[i]) return false;
        return true;
    }
};

struct Solver {
    int64_t n = 0;            // 9 n_c
    int64_t cap = 0;          // history columns
    int max_iters = 0;
    int nparts = 0;
    int64_t phip_len = 0;
    int elt = 8;              // bytes per element of the vectors
    void* P = nullptr;        // cap x n
    void* Q = nullptr;
    void* r = nullptr;
    void* z = nullptr;
    void* xw = nullptr;       // working x of the inner solve (mixed)
    void* PT = nullptr;       // n x 16 row-major copy of the newest block (float32 direct-Q products)
    double* part_a = nullptr; // nparts x kGramMax
    double* part_b = nullptr; // nparts x 2
    double* part_c = nullptr; // nparts x 2
    double* part_cam = nullptr;  // n_c x 2 (per-camera partials of the implicit residual)
    double* dpinv = nullptr;  // (max_iters + 1) x 256
    double* B = nullptr;      // cap x 16
    double* phip = nullptr;
    double* hist = nullptr;   // max_iters (of the last sweep)
    int* blk_off = nullptr;
    int* blk_w = nullptr;
    Ctl* ctl = nullptr;
    Ctl* h_ctl = nullptr;     // pinned
    double* rt = nullptr;     // true residual vector (float64, n)
    std::vector<double> host_hist;
    int64_t launches = 0;     // kernel executions issued by the current solve
    void* flush = nullptr;    // L2 flush buffer for kernel timing
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphKey key;
    // work lists of the block-sparse products: whole rows, and rows split by pose subset
    ItemList items_g, items_l;
    int items_l_dirs = -1;
    bool use_local = false;    // local steps read items_l (false when there is a single subset)
    void* mm_part = nullptr;   // k_spmm partials: items_g.n x 16 x 9
    double* totals = nullptr;  // grid totals: [0] Delta [1] gamma [2] |r|^2 [3] Phi [4] r^T z ; [8] |r|^2 [9] r^T z
    double* dpart = nullptr;   // 3 x (num_sms * 8) x 2 CTA partials
    int* dcnt = nullptr;       // 4 self-resetting arrival counters
};

// Items of the block-sparse product: each (row, segment) split into chunks of at most cb blocks.
// sz = 0: one segment per row; otherwise segment s holds the blocks whose column camera lies in
// [s sz, (s + 1) sz), for s < n_seg (empty segments get one empty item, which writes zeros).
static std::vector<SpItem> build_items(const Structure& s, int sz, int n_seg, int cb) {
    std::vector<SpItem> out;
    int grp = 0;
    for (int32_t j = 0; j < s.n_c; ++j) {
        const int64_t rj = s.h_row_ptr[j], nj = s.h_row_ptr[j + 1] - rj;
        const int32_t* cj = s.h_col.data() + rj;
        const int nseg = sz > 0 ? n_seg : 1;
        for (int g = 0; g < nseg; ++g) {
            int q0 = 0, q1 = int(nj);
            if (sz > 0) {
                q0 = int(std::lower_bound(cj, cj + nj, g * sz) - cj);
                q1 = int(std::lower_bound(cj, cj + nj, (g + 1) * sz) - cj);
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
                it.pad = 0;
                out.push_back(it);
            }
            ++grp;
        }
    }
    return out;
}

static int item_chunk(const Structure& s) {
    int64_t target = int64_t(num_sms()) * 64;
    int64_t cb = (s.nnzb + target - 1) / target;
    cb = (cb + 31) / 32 * 32;
    if (cb < 32) cb = 32;
    if (cb > 256) cb = 256;
    return int(cb);
}

static void free_items(ItemList& L) {
    if (L.items) cudaFree(const_cast<SpItem*>(L.items));
    if (L.cnt) cudaFree(L.cnt);
    if (L.part) cudaFree(L.part);
    L = ItemList();
}

static void upload_items(ItemList& L, const std::vector<SpItem>& v) {
    free_items(L);
    SpItem* d = nullptr;
    BA_CUDA_TRY(cudaMalloc(&d, sizeof(SpItem) * v.size()));
    BA_CUDA_TRY(cudaMemcpy(d, v.data(), sizeof(SpItem) * v.size(), cudaMemcpyHostToDevice));
    L.items = d;
    L.n = int64_t(v.size());
    const int ngrp = v.empty() ? 1 : v.back().grp + 1;
    BA_CUDA_TRY(cudaMalloc(&L.cnt, sizeof(int) * ngrp));
    BA_CUDA_TRY(cudaMemset(L.cnt, 0, sizeof(int) * ngrp));
    BA_CUDA_TRY(cudaMalloc(&L.part, sizeof(double) * 9 * (v.size() > 0 ? v.size() : 1)));
}

static void ensure_items(Solver* w, const Structure& s, int n_dirs, int sz, int n_eff) {
    const int cb = item_chunk(s);
    if (!w->items_g.items) {
        upload_items(w->items_g, build_items(s, 0, 1, cb));
        BA_CUDA_TRY(cudaMalloc(&w->mm_part, sizeof(double) * kMaxDirs * 9 * size_t(w->items_g.n)));
    }
    if (n_eff > 1 && w->items_l_dirs != n_dirs) {
        upload_items(w->items_l, build_items(s, sz, n_eff, cb));
        w->items_l_dirs = n_dirs;
    }
    w->use_local = n_eff > 1;
    static bool attrs = false;
    if (!attrs) {
        BA_CUDA_TRY(cudaFuncSetAttribute(k_spmv<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmv_smem<float>())));
        BA_CUDA_TRY(cudaFuncSetAttribute(k_spmv<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmv_smem<float>())));
        BA_CUDA_TRY(cudaFuncSetAttribute(k_spmv<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmv_smem<float>())));
        BA_CUDA_TRY(cudaFuncSetAttribute(k_spmv<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmv_smem<double>())));
        BA_CUDA_TRY(cudaFuncSetAttribute(k_spmv<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmv_smem<double>())));
        BA_CUDA_TRY(cudaFuncSetAttribute(k_spmv<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmv_smem<double>())));
        BA_CUDA_TRY(cudaFuncSetAttribute(k_spmm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmm_smem<float>())));
        BA_CUDA_TRY(cudaFuncSetAttribute(k_spmm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(spmm_smem<double>())));
        attrs = true;
    }
    if (!w->totals) {
        BA_CUDA_TRY(cudaMalloc(&w->totals, sizeof(double) * 16));
        BA_CUDA_TRY(cudaMalloc(&w->dpart, sizeof(double) * 3 * 2 * size_t(num_sms()) * 8));
        BA_CUDA_TRY(cudaMalloc(&w->dcnt, sizeof(int) * 4));
        BA_CUDA_TRY(cudaMemset(w->dcnt, 0, sizeof(int) * 4));
    }
}

static int spmv_grid() { return num_sms() * 8; }

static void free_ws(Solver* w) {
    void* ptrs[] = {w->P, w->Q, w->r, w->z, w->xw, w->PT, w->part_a, w->part_b, w->part_c, w->dpinv, w->B,
                    w->phip, w->hist, w->blk_off, w->blk_w, w->ctl, w->rt, w->part_cam};
    for (void* p : ptrs) if (p) cudaFree(p);
    w->P = w->Q = w->r = w->z = w->xw = w->PT = nullptr;
    w->part_a = w->part_b = w->part_c = w->dpinv = w->B = w->phip = w->hist = w->rt = w->part_cam = nullptr;
    w->blk_off = w->blk_w = nullptr;
    w->ctl = nullptr;
    if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
    w->key = GraphKey();
    w->n = w->cap = 0;
}

Solver* solver_create() {
    Solver* w = new Solver();
    return w;
}

void solver_destroy(Solver* w) {
    if (!w) return;
    free_ws(w);
    free_items(w->items_g);
    free_items(w->items_l);
    if (w->mm_part) cudaFree(w->mm_part);
    if (w->totals) cudaFree(w->totals);
    if (w->dpart) cudaFree(w->dpart);
    if (w->dcnt) cudaFree(w->dcnt);
    if (w->h_ctl) cudaFreeHost(w->h_ctl);
    if (w->flush) cudaFree(w->flush);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
    delete w;
}

int solver_history(const Solver* w, const double** hist) {
    *hist = w->host_hist.data();
    return static_cast<int>(w->host_hist.size());
}

template <typename T>
static void alloc_checked(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
}

static void ensure_ws(Solver* w, int64_t n, int64_t cap, int max_iters, int64_t phip_len, int elt) {
    if (!w->h_ctl) BA_CUDA_TRY(cudaMallocHost(&w->h_ctl, sizeof(Ctl)));
    if (!w->cap_stream) BA_CUDA_TRY(cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking));
    if (w->n == n && w->cap >= cap && w->max_iters >= max_iters && w->phip_len >= phip_len && w->elt == elt &&
        w->P)
        return;
    free_ws(w);
    w->n = n;
    w->cap = cap;
    w->max_iters = max_iters;
    w->phip_len = phip_len;
    w->elt = elt;
    w->nparts = num_sms() * 2;
    alloc_checked<char>(&w->P, size_t(cap) * n * elt);
    alloc_checked<char>(&w->Q, size_t(cap) * n * elt);
    alloc_checked<char>(&w->r, size_t(n) * elt);
    alloc_checked<char>(&w->z, size_t(n) * elt);
    alloc_checked<char>(&w->xw, size_t(n) * elt);
    alloc_checked<char>(&w->PT, size_t(n) * kMaxDirs * elt);
    alloc_checked<char>((void**)&w->part_a, size_t(w->nparts) * kGramMax * sizeof(double));
    alloc_checked<char>((void**)&w->part_b, size_t(w->nparts) * 2 * sizeof(double));
    alloc_checked<char>((void**)&w->part_c, size_t(w->nparts) * 2 * sizeof(double));
    alloc_checked<char>((void**)&w->part_cam, size_t(n / 9 + 1) * 2 * sizeof(double));
    alloc_checked<char>((void**)&w->dpinv, size_t(max_iters + 1) * kMaxDirs * kMaxDirs * sizeof(double));
    alloc_checked<char>((void**)&w->B, size_t(cap) * kMaxDirs * sizeof(double));
    alloc_checked<char>((void**)&w->phip, size_t(phip_len > 0 ? phip_len : 1) * sizeof(double));
    alloc_checked<char>((void**)&w->hist, size_t(max_iters + 1) * sizeof(double));
    alloc_checked<char>((void**)&w->blk_off, size_t(max_iters + 1) * sizeof(int));
    alloc_checked<char>((void**)&w->blk_w, size_t(max_iters + 1) * sizeof(int));
    alloc_checked<char>((void**)&w->ctl, sizeof(Ctl));
    alloc_checked<char>((void**)&w->rt, size_t(n) * sizeof(double));
}

// Enqueue one iteration of the chosen algorithm on `st`.
template <typename T>
static void enqueue_iteration(Solver* w, const Structure& s, const T* S, const double* Dinv, T* x, bool mcg,
                              cudaStream_t st) {
    const int G = w->nparts;
    T* P = static_cast<T*>(w->P);
    T* Q = static_cast<T*>(w->Q);
    T* r = static_cast<T*>(w->r);
    T* z = static_cast<T*>(w->z);
    const int n_c = s.n_c;
    const int Gs = spmv_grid();
    const int Gt = num_sms();   // tile-streaming product: one CTA per SM
    double* dp0 = w->dpart;
    double* dp1 = w->dpart + 2 * Gs;
    double* dp2 = w->dpart + 4 * Gs;
    if (!mcg) {
        k_spmv<T, 1><<<Gt, SpmvCfg<T>::kWarps * 32, spmv_smem<T>(), st>>>(
            s.row_ptr, s.tile_ptr, s.col, S, P, w->items_g, w->items_g, Q, w->n, r, dp0, w->dcnt, w->totals, w->ctl, 1);
        k_pcg_update<T><<<G, kThreads, 0, st>>>(n_c, Dinv, P, Q, x, r, z, w->totals, dp1, w->dcnt + 1, w->ctl);
        k_pcg_decide<<<1, 32, 0, st>>>(w->ctl, w->totals, w->hist);
        k_pcg_dir<T><<<G, kThreads, 0, st>>>(w->n, z, P, w->ctl);
    } else {
        // Gram partials: one CTA per 128 rows at most; the small solve sums them one entry per thread
        const int Gg = int(std::min<int64_t>(G, (w->n + 127) / 128));
        k_mcg_gram<T><<<Gg, kThreads, 0, st>>>(w->n, P, Q, r, w->part_a, w->ctl);
        k_mcg_small<<<1, kThreads, 0, st>>>(w->ctl, w->part_a, Gg, w->dpinv);
        k_mcg_update<T><<<G, kThreads, 0, st>>>(n_c, Dinv, P, Q, x, r, z, dp2, w->dcnt + 2, w->totals + 8, w->ctl);
        k_mcg_decide<<<1, 32, 0, st>>>(w->ctl, w->totals + 8, w->hist, w->blk_off, w->blk_w);
        k_mcg_phi<T><<<G * 4, kThreads, 0, st>>>(n_c, Q, z, w->phip, w->ctl);
        k_mcg_beta<<<G, kThreads, 0, st>>>(w->phip, w->dpinv, w->blk_off, w->blk_w, w->B, w->ctl);
        if (sizeof(T) == 8) {
            // Eq. 18: Q_{i+1} = S Z_{i+1} - sum_j Q_j beta_{i,j}
            k_spmv<T, 0><<<Gt, SpmvCfg<T>::kWarps * 32, spmv_smem<T>(), st>>>(
                s.row_ptr, s.tile_ptr, s.col, S, z, w->items_g, w->use_local ? w->items_l : w->items_g, Q, w->n,
                nullptr, nullptr, nullptr, nullptr, w->ctl, 1);
            k_mcg_pq<T><<<G, kThreads, 0, st>>>(n_c, P, Q, z, w->B, nullptr, w->ctl);
        } else {
            // Algorithm 2, line 3: Q_{i+1} = S P_{i+1}
            k_mcg_pq<T><<<G, kThreads, 0, st>>>(n_c, P, Q, z, w->B, static_cast<T*>(w->PT), w->ctl);
            k_spmv<T, 2><<<Gt, SpmvCfg<T>::kWarps * 32, spmv_smem<T>(), st>>>(
                s.row_ptr, s.tile_ptr, s.col, S, P, w->items_g, w->items_g, Q, w->n, nullptr, nullptr, nullptr, nullptr,
                w->ctl, 1);
            k_spmm<T><<<Gt, SpmvCfg<T>::kWarps * 32, spmm_smem<T>(), st>>>(
                s.row_ptr, s.tile_ptr, s.col, S, static_cast<const T*>(w->PT), w->items_g, static_cast<T*>(w->mm_part),
                Q, w->n, w->ctl);
        }
    }
}

// One Krylov solve of S x = sign * rhs (rhs float64) with storage type T.  Returns the final Ctl in *out.
template <typename T>
static void krylov(Solver* w, const Structure& s, const T* S, const double* Dinv, const double* rhs, double sign,
                   const double* scale, T* x, const SolveArgs& a, int n_eff, int sz, int K, int64_t cap, Ctl* out,
                   cudaStream_t st) {
    const int G = w->nparts;
    T* P = static_cast<T*>(w->P);
    T* Q = static_cast<T*>(w->Q);
    T* r = static_cast<T*>(w->r);
    T* z = static_cast<T*>(w->z);
    k_init_vec<T><<<G, kThreads, 0, st>>>(s.n_c, rhs, sign, scale, Dinv, x, r, z, P, w->part_b);
    k_init_ctl<<<1, 32, 0, st>>>(w->ctl, w->part_b, G, a.tol, a.max_iters, a.tau, n_eff, sz, K,
                                 static_cast<int>(cap), w->blk_off, w->blk_w, sizeof(T) == 4 ? kStagnation : 0.0,
                                 sizeof(T) == 4 ? 1 : 0);
    // Q_0 = S P_0
    k_spmv<T, 0><<<num_sms(), SpmvCfg<T>::kWarps * 32, spmv_smem<T>(), st>>>(
        s.row_ptr, s.tile_ptr, s.col, S, P, w->items_g, w->items_g, Q, w->n, nullptr, nullptr, nullptr, nullptr, w->ctl,
        0);
    BA_CUDA_TRY(cudaGetLastError());
    w->launches += 3;

    GraphKey key;
    key.mcg = a.mcg;
    key.fp32 = sizeof(T) == 4;
    key.chunk = a.chunk;
    const void* ptrs[12] = {S, Dinv, x, w->P, w->Q, w->r, w->z, w->ctl, w->B, w->phip, w->items_g.items,
                            w->use_local ? w->items_l.items : w->items_g.items};
    for (int i = 0; i < 12; ++i) key.ptrs[i] = ptrs[i];
    if (!(key == w->key) || !w->exec) {
        if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
        cudaGraph_t g = nullptr;
        BA_CUDA_TRY(cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < a.chunk; ++k) enqueue_iteration<T>(w, s, S, Dinv, x, a.mcg != 0, w->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(w->cap_stream, &g);
        if (ce != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&w->exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        w->key = key;
    }
    const int max_chunks = a.max_iters / a.chunk + 2;
    for (int c = 0; c < max_chunks; ++c) {
        BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        BA_CUDA_TRY(cudaStreamSynchronize(st));
        if (w->h_ctl->done) break;
        BA_CUDA_TRY(cudaGraphLaunch(w->exec, st));
        w->launches += int64_t(a.chunk) * (a.mcg ? (sizeof(T) == 8 ? 8 : 9) : 4);
    }
    BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    *out = *w->h_ctl;
}

// out = -b~ - S x and its norms into ctl (true_rr, bb): explicit tiled S in float64 precision,
// the implicit float64 operator U x - G (G^T x) in mixed precision (no float64 S is built there).
static void true_residual(Solver* w, const Structure& s, const System& y, const double* x, double* out,
                          cudaStream_t st) {
    const int G = w->nparts;
    if (y.S) {
        k_true_residual<<<G, kThreads, 0, st>>>(s.n_c, s.row_ptr, s.tile_ptr, s.col, y.S, x, y.bt, out, w->part_c);
        w->launches += 1;
        k_true_reduce<<<1, 32, 0, st>>>(w->ctl, w->part_c, G);
    } else {
        launch_implicit_residual(s, y, x, out, w->part_cam, st);
        w->launches += 2;
        k_true_reduce<<<1, 32, 0, st>>>(w->ctl, w->part_cam, s.n_c);
    }
    w->launches += 1;
}

static int grid_for_host(int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    int cap = num_sms() * 8;
    return int(g < 1 ? 1 : (g > cap ? cap : g));
}

void solver_run(Solver* w, const Structure& s, const System& y, const SolveArgs& a, double* x, SolveOut& out,
                cudaStream_t st) {
    const int64_t n = int64_t(s.n_c) * 9;
    int n_dirs = a.mcg ? a.n_dirs : 1;
    if (n_dirs < 1) n_dirs = 1;
    if (n_dirs > kMaxDirs) throw Error(BA_ERR_INVALID_ARG, "n_dirs must be in [1, 16]");
    const int sz = (s.n_c + n_dirs - 1) / n_dirs;
    const int n_eff = (s.n_c + sz - 1) / sz;
    const int K = (sz + kChunkCams - 1) / kChunkCams;
    int64_t cap = 1;
    if (a.mcg) {
        cap = a.max_history > 0 ? a.max_history : int64_t(a.max_iters) * n_eff + 1;
        if (cap < 1 + n_eff) cap = 1 + n_eff;
        if (cap > (int64_t(1) << 30)) throw Error(BA_ERR_INVALID_ARG, "direction history too large");
    } else {
        cap = 1;
    }
    const bool fp32 = a.precision == BA_PRECISION_MIXED;
    ensure_ws(w, n, cap, a.max_iters, cap * n_eff * K, fp32 ? 4 : 8);
    ensure_items(w, s, a.mcg ? n_dirs : 1, sz, n_eff);
    w->launches = 0;

    cudaEvent_t e0, e1;
    BA_CUDA_TRY(cudaEventCreate(&e0));
    BA_CUDA_TRY(cudaEventCreate(&e1));
    BA_CUDA_TRY(cudaEventRecord(e0, st));
    out = SolveOut();
    out.n_eff = n_eff;
    Ctl fin;
    const int G = w->nparts;
    if (!fp32) {
        krylov<double>(w, s, y.S, y.Dinv, y.bt, -1.0, nullptr, x, a, n_eff, sz, K, cap, &fin, st);
        out.status = fin.status;
        out.iters = fin.it;
        out.local_steps = fin.local_steps;
        out.history_cols = a.mcg ? fin.cols : 1;
        out.rel_residual = fin.rr0 > 0 ? std::sqrt(fin.rr / fin.rr0) : 0.0;
        out.refinements = 1;
        w->host_hist.resize(fin.it);
        if (fin.it > 0)
            BA_CUDA_TRY(cudaMemcpyAsync(w->host_hist.data(), w->hist, sizeof(double) * fin.it,
                                        cudaMemcpyDeviceToHost, st));
        // true relative residual in float64
        true_residual(w, s, y, x, nullptr, st);
    } else {
        // float64 iterative refinement around float32 Krylov sweeps
        // x = 0, so the true residual is -b~ itself: rt = -b~, |rt|^2 = |b~|^2
        k_start_refine<<<grid_for_host(n), kThreads, 0, st>>>(n, y.bt, x, w->rt);
        w->launches += 1;
        k_norm2<<<1, kThreads, 0, st>>>(n, y.bt, w->ctl);
        w->launches += 1;
        BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        BA_CUDA_TRY(cudaStreamSynchronize(st));
        const double bb = w->h_ctl->bb;
        double tr = bb;
        SolveArgs inner = a;
        inner.tol = a.inner_tol;
        int total = 0, locals = 0;
        int status = BA_ERR_NOT_CONVERGED;
        w->host_hist.clear();
        int sweeps = 0;
        if (bb == 0.0) status = BA_OK;
        while (status != BA_OK && sweeps < a.max_refine && total < a.max_iters) {
            inner.max_iters = a.max_iters - total;
            // per sweep the inner solve reduces its residual by inner_tol; when what is left to reach
            // tol is within ten times that, the sweep aims 3x past it so that it is the last one
            const double need = a.tol * std::sqrt(bb) / std::sqrt(tr);
            inner.tol = need > 0.1 * a.inner_tol ? std::max(0.3 * need, 0.1 * a.inner_tol) : a.inner_tol;
            if (inner.tol >= 1.0) inner.tol = 0.5;
            krylov<float>(w, s, y.S32, y.Dhat, w->rt, 1.0, y.lam, static_cast<float*>(w->xw), inner, n_eff, sz, K,
                          cap, &fin, st);
            ++sweeps;
            total += fin.it;
            locals += fin.local_steps;
            out.history_cols = a.mcg ? fin.cols : 1;
            std::vector<double> h(fin.it);
            if (fin.it > 0)
                BA_CUDA_TRY(cudaMemcpyAsync(h.data(), w->hist, sizeof(double) * fin.it, cudaMemcpyDeviceToHost, st));
            k_accumulate<<<grid_for_host(n), kThreads, 0, st>>>(n, static_cast<const float*>(w->xw), y.lam, x);
            true_residual(w, s, y, x, w->rt, st);
            w->launches += 1;
            BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
            BA_CUDA_TRY(cudaStreamSynchronize(st));
            const double prev = tr;
            tr = w->h_ctl->true_rr;
            // history in units of the outer |b~|: inner relative residuals scaled by the sweep's start
            for (double v : h) w->host_hist.push_back(v * std::sqrt(prev / bb));
            if (fin.status == BA_ERR_BREAKDOWN || fin.status == BA_ERR_OOM) { status = fin.status; break; }
            if (tr <= a.tol * a.tol * bb) status = BA_OK;
            if (!(tr == tr)) { status = BA_ERR_BREAKDOWN; break; }
        }
        out.status = status;
        out.iters = total;
        out.local_steps = locals;
        out.refinements = sweeps;
        out.rel_residual = std::sqrt(tr / bb);
        // the last sweep's float64 true residual is the result's (ctl holds it)
    }
    out.launches = w->launches;
    BA_CUDA_TRY(cudaEventRecord(e1, st));
    BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    BA_CUDA_TRY(cudaGetLastError());
    out.true_rel_residual = w->h_ctl->bb > 0 ? std::sqrt(w->h_ctl->true_rr / w->h_ctl->bb) : 0.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    out.ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

void flush_l2(cudaStream_t st) {
    static void* buf = nullptr;
    const size_t bytes = size_t(256) << 20;
    if (!buf) BA_CUDA_TRY(cudaMalloc(&buf, bytes));
    BA_CUDA_TRY(cudaMemsetAsync(buf, 0, bytes, st));
}

double solver_time_spmv(Solver* w, const Structure& s, const System& y, bool fp32, int reps, cudaStream_t st) {
    const int64_t n = int64_t(s.n_c) * 9;
    ensure_ws(w, n, w->cap > 0 ? w->cap : 1, w->max_iters > 0 ? w->max_iters : 1,
              w->phip_len > 0 ? w->phip_len : 1, fp32 ? 4 : 8);
    BA_CUDA_TRY(cudaMemsetAsync(w->ctl, 0, sizeof(Ctl), st));
    const int G = w->nparts;
    if (fp32) {
        k_to_float_vec<<<G, kThreads, 0, st>>>(n, y.bt, static_cast<float*>(w->P));
    } else {
        BA_CUDA_TRY(cudaMemcpyAsync(w->P, y.bt, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    }
    BA_CUDA_TRY(cudaMemcpyAsync(w->r, w->P, size_t(n) * (fp32 ? 4 : 8), cudaMemcpyDeviceToDevice, st));
    cudaEvent_t a, b;
    BA_CUDA_TRY(cudaEventCreate(&a));
    BA_CUDA_TRY(cudaEventCreate(&b));
    double total = 0.0;
    ensure_items(w, s, 1, s.n_c, 1);
    for (int k = 0; k < reps; ++k) {
        flush_l2(st);
        BA_CUDA_TRY(cudaEventRecord(a, st));
        if (fp32)
            k_spmv<float, 1><<<num_sms(), SpmvCfg<float>::kWarps * 32, spmv_smem<float>(), st>>>(
                s.row_ptr, s.tile_ptr, s.col, y.S32, static_cast<float*>(w->P), w->items_g, w->items_g,
                static_cast<float*>(w->Q), n, static_cast<float*>(w->r), w->dpart, w->dcnt, w->totals, w->ctl, 1);
        else
            k_spmv<double, 1><<<num_sms(), SpmvCfg<double>::kWarps * 32, spmv_smem<double>(), st>>>(
                s.row_ptr, s.tile_ptr, s.col, y.S, static_cast<double*>(w->P), w->items_g, w->items_g,
                static_cast<double*>(w->Q), n, static_cast<double*>(w->r), w->dpart, w->dcnt, w->totals, w->ctl, 1);
        BA_CUDA_TRY(cudaEventRecord(b, st));
        BA_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        BA_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        total += ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return total / reps;
}

}  // namespace ba

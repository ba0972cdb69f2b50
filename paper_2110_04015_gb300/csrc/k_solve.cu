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

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ba_internal.cuh"

namespace ba {

namespace {

constexpr int kGramMax = kMaxDirs * kMaxDirs + kMaxDirs;   // Delta (w x w) and gamma (w)
constexpr int kChunkCams = 112;                             // cameras per Phi partial

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

// out[(off + s) * n + 9 j + a] = sum over blocks q of row j in subset segment s of S_jq z_col(q).
// local = 0: one segment (the whole row) written to column off.
template <typename T>
__global__ void k_spmv_seg(int32_t n_c, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const T* __restrict__ S, const T* __restrict__ z, T* __restrict__ out,
                           const Ctl* __restrict__ ctl, int use_ctl, int off_fixed) {
    if (use_ctl && ctl->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t n = int64_t(n_c) * 9;
    const int local = use_ctl ? ctl->local : 0;
    const int w = use_ctl ? ctl->w_new : 1;
    const int off = use_ctl ? ctl->new_off : off_fixed;
    const int sz = use_ctl ? ctl->sz : n_c;
    const int nseg = local ? w : 1;
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        const int64_t rj = row_ptr[j], nj = row_ptr[j + 1] - rj;
        const T* slab = S + rj * 81;
        for (int s = 0; s < nseg; ++s) {
            int64_t q0 = 0, q1 = nj;
            if (local) {
                // first block with col >= s*sz and first with col >= (s+1)*sz
                const int lo_c = s * sz, hi_c = (s + 1) * sz;
                int64_t a = 0, b = nj;
                while (a < b) { int64_t m = (a + b) >> 1; if (col[rj + m] < lo_c) a = m + 1; else b = m; }
                q0 = a;
                b = nj;
                while (a < b) { int64_t m = (a + b) >> 1; if (col[rj + m] < hi_c) a = m + 1; else b = m; }
                q1 = a;
            }
            T acc[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = T(0);
            for (int64_t q = q0 + lane; q < q1; q += 32) {
                const T* zk = z + int64_t(col[rj + q]) * 9;
                T zv[9];
#pragma unroll
                for (int b = 0; b < 9; ++b) zv[b] = zk[b];
                const T* sp = slab + q;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
#pragma unroll
                    for (int b = 0; b < 9; ++b) acc[a] += sp[(9 * a + b) * nj] * zv[b];
                }
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = warp_sum(acc[a]);
            if (lane < 9) {
                T v = acc[0];
#pragma unroll
                for (int a = 1; a < 9; ++a) if (lane == a) v = acc[a];
                out[int64_t(off + s) * n + 9 * j + lane] = v;
            }
        }
        // columns of subsets with no block in this row are zero
        if (local) {
            for (int s = nseg; s < w; ++s) if (lane < 9) out[int64_t(off + s) * n + 9 * j + lane] = T(0);
        }
    }
}

// ---------------------------------------------------------------------------------------
// initialisation shared by both algorithms: x = 0, r = sign * rhs, z = D^{-1} r, P_0 = z

template <typename T>
__global__ void k_init_vec(int32_t n_c, const double* __restrict__ rhs, double sign, const double* __restrict__ Dinv,
                           T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, T* __restrict__ P0,
                           double* __restrict__ partial) {
    double v[1] = {0.0};
    for (int64_t j = gtid(); j < n_c; j += gstride()) {
        double rv[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const T ra = T(sign * rhs[9 * j + a]);
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
                           double tau, int n_eff, int sz, int K, int cap, int* blk_off, int* blk_w) {
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

// q = S p with the partial sums of Delta = q^T p and gamma = p^T r.
template <typename T>
__global__ void k_pcg_spmv(int32_t n_c, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const T* __restrict__ S, const T* __restrict__ p, const T* __restrict__ r,
                           T* __restrict__ q, double* __restrict__ partial, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    const int lane = threadIdx.x & 31;
    double v[2] = {0.0, 0.0};
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        const int64_t rj = row_ptr[j], nj = row_ptr[j + 1] - rj;
        const T* slab = S + rj * 81;
        T acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = T(0);
        for (int64_t qq = lane; qq < nj; qq += 32) {
            const T* zk = p + int64_t(col[rj + qq]) * 9;
            T zv[9];
#pragma unroll
            for (int b = 0; b < 9; ++b) zv[b] = zk[b];
            const T* sp = slab + qq;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
#pragma unroll
                for (int b = 0; b < 9; ++b) acc[a] += sp[(9 * a + b) * nj] * zv[b];
            }
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = warp_sum(acc[a]);
        if (lane < 9) {
            T val = acc[0];
#pragma unroll
            for (int a = 1; a < 9; ++a) if (lane == a) val = acc[a];
            q[9 * j + lane] = val;
            const double pv = double(p[9 * j + lane]);
            v[0] += double(val) * pv;
            v[1] += pv * double(r[9 * j + lane]);
        }
    }
    cta_sum_write<2>(v, partial + 2 * blockIdx.x);
}

// alpha = gamma / Delta; x += alpha p; r -= alpha q; z = D^{-1} r; partials of |r|^2 and q^T z.
template <typename T>
__global__ void k_pcg_update(int32_t n_c, const double* __restrict__ Dinv, const T* __restrict__ p,
                             const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                             const double* __restrict__ pa, int np, double* __restrict__ pb,
                             const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    __shared__ double s_alpha;
    if (threadIdx.x < 32) {
        double D = sum_partials(pa, np, 2, 0);
        double g = sum_partials(pa, np, 2, 1);
        if (threadIdx.x == 0) s_alpha = g / D;
    }
    __syncthreads();
    const T alpha = T(s_alpha);
    double v[2] = {0.0, 0.0};
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
        }
    }
    cta_sum_write<2>(v, pb + 2 * blockIdx.x);
}

// stop test and beta = Phi / Delta (one CTA)
__global__ void k_pcg_decide(Ctl* ctl, const double* __restrict__ pa, const double* __restrict__ pb, int np,
                             double* hist) {
    if (ctl->done) return;
    if (threadIdx.x >= 32) return;
    double D = sum_partials(pa, np, 2, 0);
    double g = sum_partials(pa, np, 2, 1);
    double rr = sum_partials(pb, np, 2, 0);
    double phi = sum_partials(pb, np, 2, 1);
    if (threadIdx.x == 0) {
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
        } else {
            ctl->beta = phi / D;
        }
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

// Delta_i, gamma_i -> Delta_i^+ (stored for the reorthogonalisation), alpha_i, gamma^T alpha.
__global__ void k_mcg_small(Ctl* ctl, const double* __restrict__ partial, int np, double* __restrict__ dpinv) {
    if (ctl->done) return;
    __shared__ double sA[kMaxDirs][kMaxDirs + 1], sV[kMaxDirs][kMaxDirs + 1], sX[kMaxDirs][kMaxDirs + 1];
    __shared__ double sg[kMaxDirs];
    __shared__ double sal[kMaxDirs];
    const int w = ctl->w_cur;
    const int it = ctl->it;
    const int ne = w * w + w;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int e = wid; e < ne; e += nw) {
        double s = sum_partials(partial, np, kGramMax, e);
        if (lane == 0) {
            if (e < w * w) sA[e / w][e % w] = s;
            else sg[e - w * w] = s;
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
    } else {
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

// x += P_i alpha; r -= Q_i alpha; z = D^{-1} r; partials of |r|^2 and r^T z.
template <typename T>
__global__ void k_mcg_update(int32_t n_c, const double* __restrict__ Dinv, const T* __restrict__ P,
                             const T* __restrict__ Q, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                             double* __restrict__ partial, const Ctl* __restrict__ ctl) {
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
    cta_sum_write<2>(v, partial + 2 * blockIdx.x);
}

// stop test, tau-test and the layout of the next block (one CTA)
__global__ void k_mcg_decide(Ctl* ctl, const double* __restrict__ partial, int np, double* hist, int* blk_off,
                             int* blk_w) {
    if (ctl->done) return;
    if (threadIdx.x >= 32) return;
    double rr = sum_partials(partial, np, 2, 0);
    double rz = sum_partials(partial, np, 2, 1);
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
                         const double* __restrict__ B, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    constexpr int TC = 64;
    __shared__ T sB[TC][kMaxDirs];
    const int64_t n = int64_t(n_c) * 9;
    const int w = ctl->w_new, off = ctl->new_off, hc = ctl->hist_cols, local = ctl->local, sz = ctl->sz;
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
                aq[s] = Q[int64_t(off + s) * n + row];
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
                for (int cc = 0; cc < tc; ++cc) {
                    const T pv = P[int64_t(c0 + cc) * n + row];
                    const T qv = Q[int64_t(c0 + cc) * n + row];
#pragma unroll
                    for (int s = 0; s < kMaxDirs; ++s) {
                        ap[s] -= pv * sB[cc][s];
                        aq[s] -= qv * sB[cc][s];
                    }
                }
            }
        }
        if (act) {
#pragma unroll
            for (int s = 0; s < kMaxDirs; ++s) {
                if (s < w) {
                    P[int64_t(off + s) * n + row] = ap[s];
                    Q[int64_t(off + s) * n + row] = aq[s];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// true residual t = -b~ - S x in float64 and |t|^2, |b~|^2 partials

__global__ void k_true_residual(int32_t n_c, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const double* __restrict__ S, const double* __restrict__ x,
                                const double* __restrict__ bt, double* __restrict__ res,
                                double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    double v[2] = {0.0, 0.0};
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        const int64_t rj = row_ptr[j], nj = row_ptr[j + 1] - rj;
        const double* slab = S + rj * 81;
        double acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = 0.0;
        for (int64_t q = lane; q < nj; q += 32) {
            const double* xk = x + int64_t(col[rj + q]) * 9;
            double xv[9];
#pragma unroll
            for (int b = 0; b < 9; ++b) xv[b] = xk[b];
            const double* sp = slab + q;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
#pragma unroll
                for (int b = 0; b < 9; ++b) acc[a] += sp[(9 * a + b) * nj] * xv[b];
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

// mixed precision: x64 += (double) d32
__global__ void k_accumulate(int64_t n, const float* __restrict__ d, double* __restrict__ x) {
    for (int64_t i = gtid(); i < n; i += gstride()) x[i] += double(d[i]);
}

__global__ void k_zero(int64_t n, double* __restrict__ x) {
    for (int64_t i = gtid(); i < n; i += gstride()) x[i] = 0.0;
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
    double* part_a = nullptr; // nparts x kGramMax
    double* part_b = nullptr; // nparts x 2
    double* part_c = nullptr; // nparts x 2
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
};

static void free_ws(Solver* w) {
    void* ptrs[] = {w->P, w->Q, w->r, w->z, w->xw, w->part_a, w->part_b, w->part_c, w->dpinv, w->B,
                    w->phip, w->hist, w->blk_off, w->blk_w, w->ctl, w->rt};
    for (void* p : ptrs) if (p) cudaFree(p);
    w->P = w->Q = w->r = w->z = w->xw = nullptr;
    w->part_a = w->part_b = w->part_c = w->dpinv = w->B = w->phip = w->hist = w->rt = nullptr;
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
    alloc_checked<char>((void**)&w->part_a, size_t(w->nparts) * kGramMax * sizeof(double));
    alloc_checked<char>((void**)&w->part_b, size_t(w->nparts) * 2 * sizeof(double));
    alloc_checked<char>((void**)&w->part_c, size_t(w->nparts) * 2 * sizeof(double));
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
    if (!mcg) {
        k_pcg_spmv<T><<<G, kThreads, 0, st>>>(n_c, s.row_ptr, s.col, S, P, r, Q, w->part_a, w->ctl);
        k_pcg_update<T><<<G, kThreads, 0, st>>>(n_c, Dinv, P, Q, x, r, z, w->part_a, G, w->part_b, w->ctl);
        k_pcg_decide<<<1, 32, 0, st>>>(w->ctl, w->part_a, w->part_b, G, w->hist);
        k_pcg_dir<T><<<G, kThreads, 0, st>>>(w->n, z, P, w->ctl);
    } else {
        k_mcg_gram<T><<<G, kThreads, 0, st>>>(w->n, P, Q, r, w->part_a, w->ctl);
        k_mcg_small<<<1, kThreads, 0, st>>>(w->ctl, w->part_a, G, w->dpinv);
        k_mcg_update<T><<<G, kThreads, 0, st>>>(n_c, Dinv, P, Q, x, r, z, w->part_b, w->ctl);
        k_mcg_decide<<<1, 32, 0, st>>>(w->ctl, w->part_b, G, w->hist, w->blk_off, w->blk_w);
        k_mcg_phi<T><<<G * 4, kThreads, 0, st>>>(n_c, Q, z, w->phip, w->ctl);
        k_mcg_beta<<<G, kThreads, 0, st>>>(w->phip, w->dpinv, w->blk_off, w->blk_w, w->B, w->ctl);
        k_spmv_seg<T><<<G * 4, kThreads, 0, st>>>(n_c, s.row_ptr, s.col, S, z, Q, w->ctl, 1, 0);
        k_mcg_pq<T><<<G, kThreads, 0, st>>>(n_c, P, Q, z, w->B, w->ctl);
    }
}

// One Krylov solve of S x = sign * rhs (rhs float64) with storage type T.  Returns the final Ctl in *out.
template <typename T>
static void krylov(Solver* w, const Structure& s, const T* S, const double* Dinv, const double* rhs, double sign,
                   T* x, const SolveArgs& a, int n_eff, int sz, int K, int64_t cap, Ctl* out, cudaStream_t st) {
    const int G = w->nparts;
    T* P = static_cast<T*>(w->P);
    T* Q = static_cast<T*>(w->Q);
    T* r = static_cast<T*>(w->r);
    T* z = static_cast<T*>(w->z);
    k_init_vec<T><<<G, kThreads, 0, st>>>(s.n_c, rhs, sign, Dinv, x, r, z, P, w->part_b);
    k_init_ctl<<<1, 32, 0, st>>>(w->ctl, w->part_b, G, a.tol, a.max_iters, a.tau, n_eff, sz, K,
                                 static_cast<int>(cap), w->blk_off, w->blk_w);
    // Q_0 = S P_0
    k_spmv_seg<T><<<G * 4, kThreads, 0, st>>>(s.n_c, s.row_ptr, s.col, S, P, Q, w->ctl, 0, 0);
    BA_CUDA_TRY(cudaGetLastError());
    w->launches += 3;

    GraphKey key;
    key.mcg = a.mcg;
    key.fp32 = sizeof(T) == 4;
    key.chunk = a.chunk;
    const void* ptrs[12] = {S, Dinv, x, w->P, w->Q, w->r, w->z, w->ctl, w->B, w->phip, s.row_ptr, s.col};
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
        w->launches += int64_t(a.chunk) * (a.mcg ? 8 : 4);
    }
    BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    *out = *w->h_ctl;
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
        krylov<double>(w, s, y.S, y.Dinv, y.bt, -1.0, x, a, n_eff, sz, K, cap, &fin, st);
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
    } else {
        // float64 iterative refinement around float32 Krylov sweeps
        k_zero<<<grid_for_host(n), kThreads, 0, st>>>(n, x);
        // rt = -b~ - S x = -b~
        k_true_residual<<<G, kThreads, 0, st>>>(s.n_c, s.row_ptr, s.col, y.S, x, y.bt, w->rt, w->part_c);
        k_true_reduce<<<1, 32, 0, st>>>(w->ctl, w->part_c, G);
        w->launches += 3;
        BA_CUDA_TRY(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        BA_CUDA_TRY(cudaStreamSynchronize(st));
        const double bb = w->h_ctl->bb;
        double tr = w->h_ctl->true_rr;
        SolveArgs inner = a;
        inner.tol = a.inner_tol;
        int total = 0, locals = 0;
        int status = BA_ERR_NOT_CONVERGED;
        w->host_hist.clear();
        int sweeps = 0;
        if (bb == 0.0) status = BA_OK;
        while (status != BA_OK && sweeps < a.max_refine && total < a.max_iters) {
            inner.max_iters = a.max_iters - total;
            // the inner tolerance never asks for less than what is left to reach tol
            const double need = a.tol * std::sqrt(bb) / std::sqrt(tr);
            inner.tol = need > a.inner_tol ? need : a.inner_tol;
            if (inner.tol >= 1.0) inner.tol = 0.5;
            krylov<float>(w, s, y.S32, y.Dinv, w->rt, 1.0, static_cast<float*>(w->xw), inner, n_eff, sz, K, cap,
                          &fin, st);
            ++sweeps;
            total += fin.it;
            locals += fin.local_steps;
            out.history_cols = a.mcg ? fin.cols : 1;
            std::vector<double> h(fin.it);
            if (fin.it > 0)
                BA_CUDA_TRY(cudaMemcpyAsync(h.data(), w->hist, sizeof(double) * fin.it, cudaMemcpyDeviceToHost, st));
            k_accumulate<<<grid_for_host(n), kThreads, 0, st>>>(n, static_cast<const float*>(w->xw), x);
            k_true_residual<<<G, kThreads, 0, st>>>(s.n_c, s.row_ptr, s.col, y.S, x, y.bt, w->rt, w->part_c);
            k_true_reduce<<<1, 32, 0, st>>>(w->ctl, w->part_c, G);
            w->launches += 3;
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
    }
    // true relative residual in float64
    k_true_residual<<<G, kThreads, 0, st>>>(s.n_c, s.row_ptr, s.col, y.S, x, y.bt, nullptr, w->part_c);
    k_true_reduce<<<1, 32, 0, st>>>(w->ctl, w->part_c, G);
    w->launches += 2;
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
    for (int k = 0; k < reps; ++k) {
        flush_l2(st);
        BA_CUDA_TRY(cudaEventRecord(a, st));
        if (fp32)
            k_pcg_spmv<float><<<G, kThreads, 0, st>>>(s.n_c, s.row_ptr, s.col, y.S32, static_cast<float*>(w->P),
                                                      static_cast<float*>(w->r), static_cast<float*>(w->Q), w->part_a,
                                                      w->ctl);
        else
            k_pcg_spmv<double><<<G, kThreads, 0, st>>>(s.n_c, s.row_ptr, s.col, y.S, static_cast<double*>(w->P),
                                                       static_cast<double*>(w->r), static_cast<double*>(w->Q),
                                                       w->part_a, w->ctl);
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

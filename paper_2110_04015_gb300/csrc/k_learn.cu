// Learned pose grouping for MCG: a small message-passing network over the camera co-visibility
// graph of the reduced camera system, trained and run by the kernels below.
//
// The paper splits the poses into N subsets of consecutive poses and remarks that the best split
// is not obvious (Section 3.2).  Here a network scores every camera; sorting the cameras by score
// and cutting the order into the paper's N subsets of consecutive positions gives the grouping
// (any camera order is a valid input to Algorithm 2).
//
//   graph     c_jk = |Lam_j S_jk Lam_k|_F (j != k, Lam = diag(S)^-1/2), d_j = sum_k c_jk
//   features  8 per camera: centre -R^T t (per-axis standardised), viewing axis (third row of R),
//             standardised log(1 + d_j), 1
//   layers    H^l = relu(H^{l-1} Ws^l + (A H^{l-1}) Wn^l + b^l), A = D^-1 C, widths 8 -> 64 -> 64 -> 64
//   read-out  s = H^3 wo + bo
//   loss      L = u^T (D - C) u / u^T D u,  u = s - (d^T s / sum d)   (Rayleigh quotient of the
//             coupling Laplacian; small when strongly coupled cameras get close scores)
//   training  Adam on dL/dtheta (forward and backward passes written out below)
//
// float32 storage and arithmetic for the network, float64 for the loss sums; every reduction runs
// in a fixed order, so results do not depend on scheduling.  Inference can round weights and
// activations to bfloat16 (float32 accumulation).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "ba_internal.cuh"

namespace ba {

namespace {

constexpr int kF = 8;        // input features
constexpr int kH = 64;       // hidden width
constexpr int kL = 3;        // message-passing layers

__device__ __forceinline__ int64_t gtid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// fixed-order CTA sum (blockDim = kThreads); every thread receives the total
__device__ double cta_sum(double v) {
    __shared__ double red[kThreads / 32];
    __shared__ double tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        tot = s;
    }
    __syncthreads();
    const double r = tot;
    __syncthreads();
    return r;
}

// Parameter offsets: per layer Ws (fi x 64), Wn (fi x 64), b (64); then wo (64), bo (1).
struct Offsets {
    int64_t Ws[kL], Wn[kL], b[kL], wo, bo, total;
};
Offsets offsets() {
    Offsets o;
    int64_t p = 0;
    int fi = kF;
    for (int l = 0; l < kL; ++l) {
        o.Ws[l] = p;
        p += int64_t(fi) * kH;
        o.Wn[l] = p;
        p += int64_t(fi) * kH;
        o.b[l] = p;
        p += kH;
        fi = kH;
    }
    o.wo = p;
    p += kH;
    o.bo = p;
    p += 1;
    o.total = p;
    return o;
}

// ---- graph -----------------------------------------------------------------------------------

// c of every stored block (CSR order; 0 on the diagonal) and d_j, one warp per block-row.
// float64 system: Lam from the diagonal of S_jj; mixed: S32 already holds Lam S Lam.
__global__ void k_gnn_edges(int32_t n_c, const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr,
                            const int32_t* __restrict__ col, const double* __restrict__ S,
                            const float* __restrict__ S32, const double* __restrict__ Sd, float* __restrict__ c,
                            float* __restrict__ d) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        const int64_t rj = row_ptr[j], nj = row_ptr[j + 1] - rj;
        double lj[9];
        if (S) {
#pragma unroll
            for (int a = 0; a < 9; ++a) lj[a] = 1.0 / sqrt(Sd[81 * j + 10 * a]);
        }
        double deg = 0.0;
        for (int64_t q = lane; q < nj; q += 32) {
            const int64_t k = col[rj + q];
            double sum = 0.0;
            if (k != j) {
                if (S) {
                    double lk[9];
#pragma unroll
                    for (int b = 0; b < 9; ++b) lk[b] = 1.0 / sqrt(Sd[81 * k + 10 * b]);
                    for (int a = 0; a < 9; ++a)
#pragma unroll
                        for (int b = 0; b < 9; ++b) {
                            const double v = lj[a] * S[s_at(tile_ptr, j, q, 9 * a + b)] * lk[b];
                            sum += v * v;
                        }
                } else {
                    for (int e = 0; e < 81; ++e) {
                        const double v = S32[s_at(tile_ptr, j, q, e)];
                        sum += v * v;
                    }
                }
            }
            const float cq = float(sqrt(sum));
            c[rj + q] = cq;
            deg += double(cq);
        }
        deg = warp_sum(deg);
        if (lane == 0) d[j] = float(deg);
    }
}

// raw features from the camera block (R row-major at aux[24 j], t at aux[24 j + 18])
__global__ void k_gnn_features(int32_t n_c, const double* __restrict__ aux, const float* __restrict__ d,
                               float* __restrict__ X) {
    for (int64_t j = gtid(); j < n_c; j += gstride()) {
        const double* R = aux + 24 * j;
        const double* t = aux + 24 * j + 18;
        float* x = X + kF * j;
#pragma unroll
        for (int i = 0; i < 3; ++i) x[i] = float(-(R[i] * t[0] + R[3 + i] * t[1] + R[6 + i] * t[2]));
        x[3] = float(R[6]);
        x[4] = float(R[7]);
        x[5] = float(R[8]);
        x[6] = float(log1p(double(d[j])));
        x[7] = 1.0f;
    }
}

// standardise the centre (per axis: mean removed, divided by the axis' root mean square) and
// log(1 + d) (mean removed, divided by its standard deviation); one CTA
__global__ void k_gnn_standardize(int32_t n_c, float* __restrict__ X) {
    const int cols[4] = {0, 1, 2, 6};
    for (int ci = 0; ci < 4; ++ci) {
        const int f = cols[ci];
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < n_c; j += blockDim.x) s += X[kF * j + f];
        const double mean = cta_sum(s) / n_c;
        double q = 0.0;
        for (int64_t j = threadIdx.x; j < n_c; j += blockDim.x) {
            const double v = X[kF * j + f] - mean;
            q += v * v;
        }
        const double rms = sqrt(cta_sum(q) / n_c);
        const double inv = rms > 0.0 ? 1.0 / rms : 1.0;
        for (int64_t j = threadIdx.x; j < n_c; j += blockDim.x) X[kF * j + f] = float((X[kF * j + f] - mean) * inv);
        __syncthreads();
    }
}

// ---- forward -----------------------------------------------------------------------------------

// AH_j = (sum_k c_jk H_k) / d_j, one warp per row, lanes over the fi <= 64 features
__global__ void k_gnn_aggregate(int32_t n_c, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const float* __restrict__ c, const float* __restrict__ d, const float* __restrict__ H,
                                int fi, float* __restrict__ AH, int bf16) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        float a0 = 0.f, a1 = 0.f;
        for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) {
            const float w = c[q];
            const float* hk = H + int64_t(col[q]) * fi;
            if (lane < fi) a0 += w * hk[lane];
            if (lane + 32 < fi) a1 += w * hk[lane + 32];
        }
        const float inv = d[j] > 0.f ? 1.f / d[j] : 0.f;
        if (lane < fi) AH[j * fi + lane] = bf16 ? round_bf16(a0 * inv) : a0 * inv;
        if (lane + 32 < fi) AH[j * fi + lane + 32] = bf16 ? round_bf16(a1 * inv) : a1 * inv;
    }
}

// Z = H Ws + AH Wn + b, H' = relu(Z); thread per (node, output)
__global__ void k_gnn_dense(int32_t n_c, int fi, const float* __restrict__ H, const float* __restrict__ AH,
                            const float* __restrict__ Ws, const float* __restrict__ Wn, const float* __restrict__ b,
                            float* __restrict__ Z, float* __restrict__ Hout, int bf16) {
    for (int64_t idx = gtid(); idx < int64_t(n_c) * kH; idx += gstride()) {
        const int64_t j = idx / kH;
        const int o = int(idx % kH);
        float z = b[o];
        const float* h = H + j * fi;
        const float* ah = AH + j * fi;
        for (int i = 0; i < fi; ++i) z += h[i] * Ws[i * kH + o];
        for (int i = 0; i < fi; ++i) z += ah[i] * Wn[i * kH + o];
        Z[idx] = z;
        const float r = z > 0.f ? z : 0.f;
        Hout[idx] = bf16 ? round_bf16(r) : r;
    }
}

// s_j = H_j wo + bo, one warp per node
__global__ void k_gnn_readout(int32_t n_c, const float* __restrict__ H, const float* __restrict__ wo,
                              const float* __restrict__ bo, float* __restrict__ s) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        double v = double(H[j * kH + lane]) * wo[lane] + double(H[j * kH + lane + 32]) * wo[lane + 32];
        v = warp_sum(v);
        if (lane == 0) s[j] = float(v + bo[0]);
    }
}

// ---- loss ---------------------------------------------------------------------------------------

// u = s - d^T s / sum d (one CTA)
__global__ void k_gnn_center(int32_t n_c, const float* __restrict__ s, const float* __restrict__ d,
                             double* __restrict__ u) {
    double a = 0.0, b = 0.0;
    for (int64_t j = threadIdx.x; j < n_c; j += blockDim.x) {
        a += double(d[j]) * s[j];
        b += double(d[j]);
    }
    const double sd = cta_sum(a);
    const double dd = cta_sum(b);
    const double mean = dd > 0.0 ? sd / dd : 0.0;
    for (int64_t j = threadIdx.x; j < n_c; j += blockDim.x) u[j] = double(s[j]) - mean;
}

// (C u)_j, one warp per row
__global__ void k_gnn_cu(int32_t n_c, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                         const float* __restrict__ c, const double* __restrict__ u, double* __restrict__ Cu) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        double a = 0.0;
        for (int64_t q = row_ptr[j] + lane; q < row_ptr[j + 1]; q += 32) a += double(c[q]) * u[col[q]];
        a = warp_sum(a);
        if (lane == 0) Cu[j] = a;
    }
}

// L = (u^T D u - u^T C u) / u^T D u and g = dL/ds = (2 (D u - C u) - 2 L D u) / u^T D u (one CTA)
__global__ void k_gnn_lossgrad(int32_t n_c, const float* __restrict__ d, const double* __restrict__ u,
                               const double* __restrict__ Cu, float* __restrict__ g, double* __restrict__ loss) {
    double a = 0.0, b = 0.0;
    for (int64_t j = threadIdx.x; j < n_c; j += blockDim.x) {
        a += double(d[j]) * u[j] * u[j];
        b += u[j] * Cu[j];
    }
    const double den = cta_sum(a);
    const double uCu = cta_sum(b);
    const double L = den > 0.0 ? (den - uCu) / den : 0.0;
    if (threadIdx.x == 0) *loss = L;
    if (g)
        for (int64_t j = threadIdx.x; j < n_c; j += blockDim.x) {
            const double du = double(d[j]) * u[j];
            g[j] = den > 0.0 ? float((2.0 * (du - Cu[j]) - 2.0 * L * du) / den) : 0.f;
        }
}

// ---- backward ---------------------------------------------------------------------------------

// gradients of the read-out: gwo = H^T g, gbo = sum g (thread per output; fixed node order)
__global__ void k_gnn_readout_grad(int32_t n_c, const float* __restrict__ H, const float* __restrict__ g,
                                   float* __restrict__ gwo, float* __restrict__ gbo) {
    const int o = threadIdx.x;
    if (o > kH) return;
    double a = 0.0;
    if (o < kH)
        for (int64_t j = 0; j < n_c; ++j) a += double(H[j * kH + o]) * g[j];
    else
        for (int64_t j = 0; j < n_c; ++j) a += g[j];
    if (o < kH) gwo[o] = float(a);
    else gbo[0] = float(a);
}

// dZ = (g wo^T) masked by Z > 0 (layer 3), or dH masked by Z > 0 (other layers)
__global__ void k_gnn_mask(int32_t n_c, const float* __restrict__ dH, const float* __restrict__ g,
                           const float* __restrict__ wo, const float* __restrict__ Z, float* __restrict__ dZ) {
    for (int64_t idx = gtid(); idx < int64_t(n_c) * kH; idx += gstride()) {
        const float v = dH ? dH[idx] : g[idx / kH] * wo[idx % kH];
        dZ[idx] = Z[idx] > 0.f ? v : 0.f;
    }
}

// gWs = H^T dZ, gWn = AH^T dZ, gb = column sums of dZ; thread per weight, nodes in order
__global__ void k_gnn_wgrad(int32_t n_c, int fi, const float* __restrict__ H, const float* __restrict__ AH,
                            const float* __restrict__ dZ, float* __restrict__ gWs, float* __restrict__ gWn,
                            float* __restrict__ gb) {
    const int64_t nw = int64_t(fi) * kH;
    for (int64_t idx = gtid(); idx < 2 * nw + kH; idx += gstride()) {
        double a = 0.0;
        if (idx < 2 * nw) {
            const bool nb = idx >= nw;
            const int64_t e = nb ? idx - nw : idx;
            const int i = int(e / kH), o = int(e % kH);
            const float* src = nb ? AH : H;
            for (int64_t j = 0; j < n_c; ++j) a += double(src[j * fi + i]) * dZ[j * kH + o];
            (nb ? gWn : gWs)[e] = float(a);
        } else {
            const int o = int(idx - 2 * nw);
            for (int64_t j = 0; j < n_c; ++j) a += dZ[j * kH + o];
            gb[o] = float(a);
        }
    }
}

// P1 = dZ Ws^T and Y = (dZ Wn^T) / d (rows), thread per (node, input feature)
__global__ void k_gnn_back_dense(int32_t n_c, int fi, const float* __restrict__ dZ, const float* __restrict__ Ws,
                                 const float* __restrict__ Wn, const float* __restrict__ d, float* __restrict__ P1,
                                 float* __restrict__ Y) {
    for (int64_t idx = gtid(); idx < int64_t(n_c) * fi; idx += gstride()) {
        const int64_t j = idx / fi;
        const int i = int(idx % fi);
        const float* dz = dZ + j * kH;
        float a = 0.f, b = 0.f;
        for (int o = 0; o < kH; ++o) {
            a += dz[o] * Ws[i * kH + o];
            b += dz[o] * Wn[i * kH + o];
        }
        P1[idx] = a;
        Y[idx] = d[j] > 0.f ? b / d[j] : 0.f;
    }
}

// dH_prev_j = P1_j + sum_k c_jk Y_k  (A^T applied through the symmetric coupling), one warp per row
__global__ void k_gnn_back_aggr(int32_t n_c, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const float* __restrict__ c, const float* __restrict__ P1, const float* __restrict__ Y,
                                int fi, float* __restrict__ dH) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = gtid() >> 5; j < n_c; j += gstride() >> 5) {
        float a0 = 0.f, a1 = 0.f;
        for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) {
            const float w = c[q];
            const float* yk = Y + int64_t(col[q]) * fi;
            if (lane < fi) a0 += w * yk[lane];
            if (lane + 32 < fi) a1 += w * yk[lane + 32];
        }
        if (lane < fi) dH[j * fi + lane] = P1[j * fi + lane] + a0;
        if (lane + 32 < fi) dH[j * fi + lane + 32] = P1[j * fi + lane + 32] + a1;
    }
}

// Adam with bias correction (c1 = 1 - beta1^t, c2 = 1 - beta2^t)
__global__ void k_gnn_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float c1, float c2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t i = gtid(); i < n; i += gstride()) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_gnn_round(int64_t n, const float* __restrict__ in, float* __restrict__ out) {
    for (int64_t i = gtid(); i < n; i += gstride()) out[i] = round_bf16(in[i]);
}

// order[rank_j] = j with rank_j = #{k : s_k < s_j or (s_k = s_j and k < j)}
__global__ void k_gnn_rank(int32_t n_c, const float* __restrict__ s, int32_t* __restrict__ order) {
    for (int64_t j = gtid(); j < n_c; j += gstride()) {
        const float sj = s[j];
        int32_t r = 0;
        for (int64_t k = 0; k < n_c; ++k) {
            const float sk = s[k];
            r += (sk < sj || (sk == sj && k < j)) ? 1 : 0;
        }
        order[r] = int32_t(j);
    }
}

int grid_of(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    const int cap = num_sms() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return int(g);
}

}  // namespace

struct Gnn {
    Offsets off = offsets();
    float* params = nullptr;   // off.total
    float* p16 = nullptr;      // bfloat16-rounded copy for inference
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    int64_t step = 0;
    // per-graph workspace
    int32_t n = 0;
    int64_t nnzb = 0;
    float *c = nullptr, *d = nullptr, *X = nullptr, *s = nullptr, *g = nullptr;
    float *H[kL + 1] = {}, *AH[kL] = {}, *Z[kL] = {};
    float *dH = nullptr, *dZ = nullptr, *P1 = nullptr, *Y = nullptr;
    double *u = nullptr, *Cu = nullptr, *loss = nullptr;
    int32_t* order = nullptr;
    int64_t launches = 0;
    std::vector<void*> ws;
};

static void* dmalloc(size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return p;
}

int64_t gnn_param_count() { return offsets().total; }

Gnn* gnn_create() {
    Gnn* g = new Gnn();
    try {
        const size_t P = size_t(g->off.total) * sizeof(float);
        g->params = static_cast<float*>(dmalloc(P));
        g->p16 = static_cast<float*>(dmalloc(P));
        g->grad = static_cast<float*>(dmalloc(P));
        g->m = static_cast<float*>(dmalloc(P));
        g->v = static_cast<float*>(dmalloc(P));
        BA_CUDA_TRY(cudaMemset(g->params, 0, P));
        BA_CUDA_TRY(cudaMemset(g->m, 0, P));
        BA_CUDA_TRY(cudaMemset(g->v, 0, P));
        g->loss = static_cast<double*>(dmalloc(sizeof(double)));
    } catch (...) {
        gnn_destroy(g);
        throw;
    }
    return g;
}

static void free_ws(Gnn* g) {
    for (void* p : g->ws) cudaFree(p);
    g->ws.clear();
    g->n = 0;
    g->nnzb = 0;
}

void gnn_destroy(Gnn* g) {
    if (!g) return;
    free_ws(g);
    float* ps[] = {g->params, g->p16, g->grad, g->m, g->v};
    for (float* p : ps) if (p) cudaFree(p);
    if (g->loss) cudaFree(g->loss);
    delete g;
}

void gnn_set_params(Gnn* g, const float* params, cudaStream_t st) {
    const size_t P = size_t(g->off.total) * sizeof(float);
    BA_CUDA_TRY(cudaMemcpyAsync(g->params, params, P, cudaMemcpyDefault, st));
    BA_CUDA_TRY(cudaMemsetAsync(g->m, 0, P, st));
    BA_CUDA_TRY(cudaMemsetAsync(g->v, 0, P, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    g->step = 0;
}

void gnn_get_params(const Gnn* g, float* params, cudaStream_t st) {
    BA_CUDA_TRY(cudaMemcpyAsync(params, g->params, size_t(g->off.total) * sizeof(float), cudaMemcpyDefault, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
}

int64_t gnn_launches(const Gnn* g) { return g->launches; }

// workspace for a graph of n nodes and nnzb stored blocks
static void ensure_graph(Gnn* g, int32_t n, int64_t nnzb) {
    if (g->n == n && g->nnzb == nnzb) return;
    free_ws(g);
    auto f = [&](int64_t count) {
        void* p = dmalloc(size_t(count) * sizeof(float));
        g->ws.push_back(p);
        return static_cast<float*>(p);
    };
    auto dd = [&](int64_t count) {
        void* p = dmalloc(size_t(count) * sizeof(double));
        g->ws.push_back(p);
        return static_cast<double*>(p);
    };
    g->c = f(nnzb);
    g->d = f(n);
    g->X = f(int64_t(n) * kF);
    g->H[0] = g->X;
    for (int l = 0; l < kL; ++l) {
        g->H[l + 1] = f(int64_t(n) * kH);
        g->AH[l] = f(int64_t(n) * kH);
        g->Z[l] = f(int64_t(n) * kH);
    }
    g->s = f(n);
    g->g = f(n);
    g->dH = f(int64_t(n) * kH);
    g->dZ = f(int64_t(n) * kH);
    g->P1 = f(int64_t(n) * kH);
    g->Y = f(int64_t(n) * kH);
    g->u = dd(n);
    g->Cu = dd(n);
    void* o = dmalloc(sizeof(int32_t) * size_t(n));
    g->ws.push_back(o);
    g->order = static_cast<int32_t*>(o);
    g->n = n;
    g->nnzb = nnzb;
}

// coupling, degrees and standardised features of the built system
static void graph(Gnn* g, const Structure& s, const System& y, cudaStream_t st) {
    if (!y.built) throw Error(BA_ERR_STATE, "ba_build_normal must succeed first");
    if (s.h_cam_off.size() > 2) throw Error(BA_ERR_INVALID_ARG, "the grouping network takes a single-problem handle");
    if (s.n_c > 65536) throw Error(BA_ERR_INVALID_ARG, "the grouping network takes at most 65536 cameras");
    ensure_graph(g, s.n_c, s.nnzb);
    k_gnn_edges<<<grid_of(int64_t(s.n_c) * 32, kThreads), kThreads, 0, st>>>(s.n_c, s.row_ptr, s.tile_ptr, s.col, y.S,
                                                                           y.S32, y.Sd, g->c, g->d);
    k_gnn_features<<<grid_of(s.n_c, kThreads), kThreads, 0, st>>>(s.n_c, y.aux, g->d, g->X);
    k_gnn_standardize<<<1, kThreads, 0, st>>>(s.n_c, g->X);
    g->launches += 3;
}

static void forward(Gnn* g, const Structure& s, const float* P, int bf16, cudaStream_t st) {
    const int32_t n = s.n_c;
    if (bf16) {
        k_gnn_round<<<grid_of(int64_t(n) * kF, kThreads), kThreads, 0, st>>>(int64_t(n) * kF, g->X, g->X);
        g->launches += 1;
    }
    int fi = kF;
    for (int l = 0; l < kL; ++l) {
        k_gnn_aggregate<<<grid_of(int64_t(n) * 32, kThreads), kThreads, 0, st>>>(n, s.row_ptr, s.col, g->c, g->d,
                                                                              g->H[l], fi, g->AH[l], bf16);
        k_gnn_dense<<<grid_of(int64_t(n) * kH, kThreads), kThreads, 0, st>>>(
            n, fi, g->H[l], g->AH[l], P + g->off.Ws[l], P + g->off.Wn[l], P + g->off.b[l], g->Z[l], g->H[l + 1], bf16);
        fi = kH;
    }
    k_gnn_readout<<<grid_of(int64_t(n) * 32, kThreads), kThreads, 0, st>>>(n, g->H[kL], P + g->off.wo, P + g->off.bo,
                                                                         g->s);
    k_gnn_center<<<1, kThreads, 0, st>>>(n, g->s, g->d, g->u);
    k_gnn_cu<<<grid_of(int64_t(n) * 32, kThreads), kThreads, 0, st>>>(n, s.row_ptr, s.col, g->c, g->u, g->Cu);
    g->launches += 2 * kL + 3;
}

static void backward(Gnn* g, const Structure& s, cudaStream_t st) {
    const int32_t n = s.n_c;
    const float* P = g->params;
    float* G = g->grad;
    k_gnn_readout_grad<<<1, kH + 32, 0, st>>>(n, g->H[kL], g->g, G + g->off.wo, G + g->off.bo);
    g->launches += 1;
    for (int l = kL - 1; l >= 0; --l) {
        const int fi = l == 0 ? kF : kH;
        k_gnn_mask<<<grid_of(int64_t(n) * kH, kThreads), kThreads, 0, st>>>(
            n, l == kL - 1 ? nullptr : g->dH, g->g, P + g->off.wo, g->Z[l], g->dZ);
        k_gnn_wgrad<<<grid_of(2 * int64_t(fi) * kH + kH, 128), 128, 0, st>>>(n, fi, g->H[l], g->AH[l], g->dZ,
                                                                            G + g->off.Ws[l], G + g->off.Wn[l],
                                                                            G + g->off.b[l]);
        g->launches += 2;
        if (l > 0) {
            k_gnn_back_dense<<<grid_of(int64_t(n) * fi, kThreads), kThreads, 0, st>>>(
                n, fi, g->dZ, P + g->off.Ws[l], P + g->off.Wn[l], g->d, g->P1, g->Y);
            k_gnn_back_aggr<<<grid_of(int64_t(n) * 32, kThreads), kThreads, 0, st>>>(n, s.row_ptr, s.col, g->c, g->P1,
                                                                                   g->Y, fi, g->dH);
            g->launches += 2;
        }
    }
}

double gnn_loss(Gnn* g, const Structure& s, const System& y, bool with_grad, float* scores, float* grad,
                cudaStream_t st) {
    graph(g, s, y, st);
    forward(g, s, g->params, 0, st);
    k_gnn_lossgrad<<<1, kThreads, 0, st>>>(s.n_c, g->d, g->u, g->Cu, with_grad ? g->g : nullptr, g->loss);
    g->launches += 1;
    if (with_grad) backward(g, s, st);
    BA_CUDA_TRY(cudaGetLastError());
    double L = 0.0;
    BA_CUDA_TRY(cudaMemcpyAsync(&L, g->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (scores) BA_CUDA_TRY(cudaMemcpyAsync(scores, g->s, sizeof(float) * s.n_c, cudaMemcpyDefault, st));
    if (grad && with_grad)
        BA_CUDA_TRY(cudaMemcpyAsync(grad, g->grad, sizeof(float) * g->off.total, cudaMemcpyDefault, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    return L;
}

double gnn_train_step(Gnn* g, const Structure& s, const System& y, double lr, cudaStream_t st) {
    const double L = gnn_loss(g, s, y, true, nullptr, nullptr, st);
    g->step += 1;
    const float c1 = float(1.0 - std::pow(0.9, double(g->step)));
    const float c2 = float(1.0 - std::pow(0.999, double(g->step)));
    k_gnn_adam<<<grid_of(g->off.total, kThreads), kThreads, 0, st>>>(g->off.total, g->params, g->grad, g->m, g->v,
                                                                     float(lr), c1, c2);
    g->launches += 1;
    BA_CUDA_TRY(cudaGetLastError());
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    return L;
}

double gnn_order(Gnn* g, const Structure& s, const System& y, bool bf16, int32_t* order, cudaStream_t st) {
    graph(g, s, y, st);
    const float* P = g->params;
    if (bf16) {
        k_gnn_round<<<grid_of(g->off.total, kThreads), kThreads, 0, st>>>(g->off.total, g->params, g->p16);
        g->launches += 1;
        P = g->p16;
    }
    forward(g, s, P, bf16 ? 1 : 0, st);
    k_gnn_lossgrad<<<1, kThreads, 0, st>>>(s.n_c, g->d, g->u, g->Cu, nullptr, g->loss);
    k_gnn_rank<<<grid_of(s.n_c, kThreads), kThreads, 0, st>>>(s.n_c, g->s, g->order);
    g->launches += 2;
    BA_CUDA_TRY(cudaGetLastError());
    double L = 0.0;
    BA_CUDA_TRY(cudaMemcpyAsync(&L, g->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaMemcpyAsync(order, g->order, sizeof(int32_t) * s.n_c, cudaMemcpyDefault, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    return L;
}

void gnn_graph_out(Gnn* g, const Structure& s, const System& y, float* X, float* c, cudaStream_t st) {
    graph(g, s, y, st);
    BA_CUDA_TRY(cudaGetLastError());
    if (X) BA_CUDA_TRY(cudaMemcpyAsync(X, g->X, sizeof(float) * kF * size_t(s.n_c), cudaMemcpyDefault, st));
    if (c) BA_CUDA_TRY(cudaMemcpyAsync(c, g->c, sizeof(float) * size_t(s.nnzb), cudaMemcpyDefault, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace ba

// C ABI of libba (declared in include/ba.h): problem handle, host-side structure set-up,
// build / solve orchestration, the LM step and the inspection calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include "ba_internal.cuh"

namespace ba {

// SM count of the current device, cached per device (first query wins; the count of a device
// does not change while the process runs).
int num_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cached[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 148;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
    cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

}  // namespace ba

using ba::Error;

namespace ba {
namespace {
thread_local std::string g_thread_error;
}
void set_thread_error(const std::string& msg) { g_thread_error = msg; }
}  // namespace ba

struct ba_problem {
    ba_options opt;
    cudaStream_t stream = nullptr;
    ba::Structure s;
    ba::System y;
    ba::Solver* solver = nullptr;
    double* dxp = nullptr;        // last solution, n_c x 9
    double* tmp_cams = nullptr;   // trial parameters of the LM step
    double* tmp_pts = nullptr;
    double* dxl = nullptr;        // n_l x 3
    double* cost_part = nullptr;  // cost partial sums
    int cost_parts = 0;
    bool solved = false;
    double lm_lambda = -1.0;
    int64_t launches = 0;         // kernel executions issued so far
    std::vector<ba::ProbOut> last;   // per-problem results of the last solve
    double last_ms = 0.0;
    std::string err;
    std::vector<void*> owned;     // every device allocation, freed by destroy
};

namespace {

thread_local std::string g_create_error;

template <typename T>
T* dev_alloc(ba_problem* p, size_t count) {
    if (count == 0) count = 1;
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA,
                    std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes: " +
                        cudaGetErrorString(e));
    }
    p->owned.push_back(ptr);
    return static_cast<T*>(ptr);
}

template <typename T>
T* upload(ba_problem* p, const std::vector<T>& v) {
    T* d = dev_alloc<T>(p, v.size());
    if (!v.empty()) BA_CUDA_TRY(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

template <typename T>
std::vector<T> fetch(const T* src, size_t count) {
    std::vector<T> v(count);
    if (count) BA_CUDA_TRY(cudaMemcpy(v.data(), src, count * sizeof(T), cudaMemcpyDefault));
    return v;
}

void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (!dst || bytes == 0) return;
    BA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
}

int fail(ba_problem* p, const Error& e) {
    if (p) p->err = e.msg;
    return e.code;
}

// Observation sort, camera CSR, pattern of S and the observation pairs feeding each upper block.
void build_structure(ba_problem* p, int32_t n_c, int32_t n_l, int64_t n_o, const int32_t* oc_in,
                     const int32_t* op_in, const double* xy_in, const std::vector<int32_t>& cam_off) {
    ba::Structure& s = p->s;
    s.n_c = n_c;
    s.n_l = n_l;
    s.n_o = n_o;
    s.h_cam_off = cam_off;
    std::vector<int32_t> oc = fetch(oc_in, n_o), op = fetch(op_in, n_o);
    std::vector<double> xy = fetch(xy_in, size_t(n_o) * 2);
    for (int64_t i = 0; i < n_o; ++i) {
        if (oc[i] < 0 || oc[i] >= n_c) throw Error(BA_ERR_INVALID_ARG, "obs_cam[" + std::to_string(i) + "] out of range");
        if (op[i] < 0 || op[i] >= n_l) throw Error(BA_ERR_INVALID_ARG, "obs_pt[" + std::to_string(i) + "] out of range");
        if (!std::isfinite(xy[2 * i]) || !std::isfinite(xy[2 * i + 1]))
            throw Error(BA_ERR_INVALID_ARG, "obs_xy[" + std::to_string(i) + "] is not finite");
    }
    // stable counting sort by landmark
    std::vector<int64_t> pt_ptr(size_t(n_l) + 1, 0);
    for (int64_t i = 0; i < n_o; ++i) pt_ptr[op[i] + 1]++;
    for (int32_t l = 0; l < n_l; ++l) pt_ptr[l + 1] += pt_ptr[l];
    std::vector<int32_t> perm(n_o), scam(n_o), spt(n_o);
    std::vector<double> sxy(size_t(n_o) * 2);
    {
        std::vector<int64_t> fill(pt_ptr.begin(), pt_ptr.end() - 1);
        for (int64_t i = 0; i < n_o; ++i) {
            int64_t slot = fill[op[i]]++;
            perm[slot] = int32_t(i);
        }
        for (int64_t k = 0; k < n_o; ++k) {
            int64_t i = perm[k];
            scam[k] = oc[i];
            spt[k] = op[i];
            sxy[2 * k] = xy[2 * i];
            sxy[2 * k + 1] = xy[2 * i + 1];
        }
    }
    // camera CSR over point-order slots
    std::vector<int64_t> cam_ptr(size_t(n_c) + 1, 0);
    for (int64_t k = 0; k < n_o; ++k) cam_ptr[scam[k] + 1]++;
    for (int32_t j = 0; j < n_c; ++j) cam_ptr[j + 1] += cam_ptr[j];
    std::vector<int32_t> cam_obs(n_o);
    {
        std::vector<int64_t> fill(cam_ptr.begin(), cam_ptr.end() - 1);
        for (int64_t k = 0; k < n_o; ++k) cam_obs[fill[scam[k]]++] = int32_t(k);
    }
    // batches: every landmark is seen by the cameras of one problem only (S is then block-diagonal)
    if (cam_off.size() > 2) {
        std::vector<int32_t> prob(n_c);
        for (size_t b = 0; b + 1 < cam_off.size(); ++b)
            for (int32_t j = cam_off[b]; j < cam_off[b + 1]; ++j) prob[j] = int32_t(b);
        for (int32_t l = 0; l < n_l; ++l)
            for (int64_t a = pt_ptr[l]; a + 1 < pt_ptr[l + 1]; ++a)
                if (prob[scam[a]] != prob[scam[a + 1]])
                    throw Error(BA_ERR_INVALID_ARG, "landmark " + std::to_string(l) + " is seen by cameras of problems " +
                                                        std::to_string(prob[scam[a]]) + " and " +
                                                        std::to_string(prob[scam[a + 1]]));
    }
    // each (camera, landmark) pair at most once: the diagonal blocks of S are then sums over
    // single observations and only pairs of different cameras feed the off-diagonal blocks
    {
        std::vector<int32_t> stamp(n_c, -1);
        for (int32_t l = 0; l < n_l; ++l)
            for (int64_t a = pt_ptr[l]; a < pt_ptr[l + 1]; ++a) {
                if (stamp[scam[a]] == l)
                    throw Error(BA_ERR_INVALID_ARG, "camera " + std::to_string(scam[a]) + " observes landmark " +
                                                        std::to_string(l) + " more than once");
                stamp[scam[a]] = l;
            }
    }
    // observation pairs (a, b) of one landmark with cam(a) < cam(b), sorted by (cam(a), cam(b))
    int64_t n_pairs = 0;
    for (int32_t l = 0; l < n_l; ++l)
        for (int64_t a = pt_ptr[l]; a < pt_ptr[l + 1]; ++a)
            for (int64_t b = pt_ptr[l]; b < pt_ptr[l + 1]; ++b)
                if (scam[a] < scam[b]) ++n_pairs;
    std::vector<int2> pr(n_pairs), pr2(n_pairs);
    {
        int64_t t = 0;
        for (int32_t l = 0; l < n_l; ++l)
            for (int64_t a = pt_ptr[l]; a < pt_ptr[l + 1]; ++a)
                for (int64_t b = pt_ptr[l]; b < pt_ptr[l + 1]; ++b)
                    if (scam[a] < scam[b]) pr[t++] = make_int2(int32_t(a), int32_t(b));
        // LSD radix: by cam(b), then stably by cam(a)
        std::vector<int64_t> cnt(size_t(n_c) + 1);
        for (int pass = 0; pass < 2; ++pass) {
            std::fill(cnt.begin(), cnt.end(), 0);
            for (int64_t q = 0; q < n_pairs; ++q) cnt[scam[pass == 0 ? pr[q].y : pr[q].x] + 1]++;
            for (int32_t j = 0; j < n_c; ++j) cnt[j + 1] += cnt[j];
            for (int64_t q = 0; q < n_pairs; ++q) pr2[cnt[scam[pass == 0 ? pr[q].y : pr[q].x]]++] = pr[q];
            pr.swap(pr2);
        }
    }
    // off-diagonal upper blocks (j < k), row by row
    std::vector<int32_t> up_j, up_k;
    std::vector<int64_t> up_pp;
    {
        int64_t q = 0;
        while (q < n_pairs) {
            const int32_t j = scam[pr[q].x], k = scam[pr[q].y];
            up_j.push_back(j);
            up_k.push_back(k);
            up_pp.push_back(q);
            while (q < n_pairs && scam[pr[q].x] == j && scam[pr[q].y] == k) ++q;
        }
        up_pp.push_back(n_pairs);
    }
    const int64_t n_up = int64_t(up_j.size());
    // full pattern: row j = lower blocks (k < j, mirrored), the diagonal, upper blocks (k > j)
    std::vector<int64_t> lower_cnt(n_c, 0), upper_cnt(n_c, 0);
    for (int64_t u = 0; u < n_up; ++u) {
        upper_cnt[up_j[u]]++;
        lower_cnt[up_k[u]]++;
    }
    std::vector<int64_t> row_ptr(size_t(n_c) + 1, 0);
    for (int32_t j = 0; j < n_c; ++j) row_ptr[j + 1] = row_ptr[j] + lower_cnt[j] + 1 + upper_cnt[j];
    const int64_t nnzb = row_ptr[n_c];
    std::vector<int32_t> col(nnzb), diag_pos(n_c);
    std::vector<int64_t> up_pos(n_up), up_mir(n_up);
    {
        std::vector<int64_t> lfill(n_c), ufill(n_c);
        for (int32_t j = 0; j < n_c; ++j) {
            lfill[j] = row_ptr[j];
            diag_pos[j] = int32_t(row_ptr[j] + lower_cnt[j]);
            col[diag_pos[j]] = j;
            ufill[j] = row_ptr[j] + lower_cnt[j] + 1;
        }
        // upper blocks are sorted by (j, k): fill upper parts in order
        for (int64_t u = 0; u < n_up; ++u) {
            int64_t pos = ufill[up_j[u]]++;
            col[pos] = up_k[u];
            up_pos[u] = pos;
        }
        // lower parts: block (k, j) for upper (j, k); iterating u in (j, k) order keeps row k's
        // lower entries sorted by j
        for (int64_t u = 0; u < n_up; ++u) {
            int64_t pos = lfill[up_k[u]]++;
            col[pos] = up_j[u];
            up_mir[u] = pos;
        }
    }

    s.obs_cam = upload(p, scam);
    s.obs_pt = upload(p, spt);
    s.perm = upload(p, perm);
    s.obs_xy = upload(p, sxy);
    if (p->opt.precision == BA_PRECISION_MIXED) {
        // double-float measurements: the nearest float, then the nearest float to the remainder
        std::vector<float2> xyd(sxy.size());
        for (size_t k = 0; k < sxy.size(); ++k) {
            const float h = static_cast<float>(sxy[k]);
            xyd[k] = make_float2(h, static_cast<float>(sxy[k] - static_cast<double>(h)));
        }
        s.obs_xyd = upload(p, xyd);
    }
    s.pt_ptr = upload(p, pt_ptr);
    {
        // landmarks by decreasing track length, stable (counting sort on the length)
        int64_t tmax = 0;
        for (int32_t l = 0; l < n_l; ++l) tmax = std::max(tmax, pt_ptr[l + 1] - pt_ptr[l]);
        std::vector<int64_t> cnt(size_t(tmax) + 2, 0);
        for (int32_t l = 0; l < n_l; ++l) cnt[size_t(tmax - (pt_ptr[l + 1] - pt_ptr[l])) + 1]++;
        for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
        std::vector<int32_t> order(n_l);
        for (int32_t l = 0; l < n_l; ++l) order[cnt[size_t(tmax - (pt_ptr[l + 1] - pt_ptr[l]))]++] = l;
        s.lm_order = upload(p, order);
    }
    s.cam_ptr = upload(p, cam_ptr);
    s.cam_obs = upload(p, cam_obs);
    s.nnzb = nnzb;
    s.row_ptr = upload(p, row_ptr);
    s.col = upload(p, col);
    s.h_row_ptr = row_ptr;
    s.h_col = col;
    std::vector<int64_t> tile_ptr(size_t(n_c) + 1, 0);
    for (int32_t j = 0; j < n_c; ++j) tile_ptr[j + 1] = tile_ptr[j] + (row_ptr[j + 1] - row_ptr[j] + ba::kTile - 1) / ba::kTile;
    s.n_tiles = tile_ptr[n_c];
    s.tile_ptr = upload(p, tile_ptr);
    s.h_tile_ptr = tile_ptr;
    s.diag_pos = upload(p, diag_pos);
    s.n_up = n_up;
    s.n_pairs = n_pairs;
    {
        // element offsets in the tiled layout, so the Schur kernels write without index lookups
        std::vector<int64_t> dst(n_up), mdst(n_up);
        for (int64_t u = 0; u < n_up; ++u) {
            const int32_t j = up_j[u], k = up_k[u];
            dst[u] = (tile_ptr[j] * ba::kTile + (up_pos[u] - row_ptr[j])) * 81;
            mdst[u] = (tile_ptr[k] * ba::kTile + (up_mir[u] - row_ptr[k])) * 81;
        }
        s.up_dst = upload(p, dst);
        s.up_mdst = upload(p, mdst);
    }
    s.up_pair_ptr = upload(p, up_pp);
    if (p->opt.precision == BA_PRECISION_MIXED) {
        // the float32 per-observation arrays are kept in camera order (cam_obs order), so that the
        // per-camera kernels read and write them contiguously
        std::vector<int32_t> cpos(n_o), cam_lm(n_o);
        for (int64_t q = 0; q < n_o; ++q) {
            cpos[cam_obs[q]] = int32_t(q);
            cam_lm[q] = spt[cam_obs[q]];
        }
        for (int64_t q = 0; q < n_pairs; ++q) pr[q] = make_int2(cpos[pr[q].x], cpos[pr[q].y]);
        std::vector<int2> ucams(n_up > 0 ? n_up : 1);
        for (int64_t u = 0; u < n_up; ++u) ucams[u] = make_int2(up_j[u], up_k[u]);
        s.cpos = upload(p, cpos);
        s.cam_lm = upload(p, cam_lm);
        s.up_cams = upload(p, ucams);
        // the upper blocks by decreasing pair-count class floor(log2(count)), stable: a warp's three
        // blocks differ by at most 2x in pairs, and within a class the blocks keep their (j, k) order,
        // in which the G rows of the blocks in flight are shared (one row serves the blocks of its
        // camera's row j, and the blocks (j', k) of the cameras j' that see its landmark)
        if (n_up >= (int64_t(1) << 31)) throw Error(BA_ERR_INVALID_ARG, "too many blocks in S");
        auto cls = [&](int64_t u) {
            int64_t c = up_pp[u + 1] - up_pp[u], b = 0;
            while (c > 1) { c >>= 1; ++b; }
            return b;
        };
        int64_t bmax = 0;
        for (int64_t u = 0; u < n_up; ++u) bmax = std::max(bmax, cls(u));
        std::vector<int64_t> pc(size_t(bmax) + 2, 0);
        for (int64_t u = 0; u < n_up; ++u) pc[size_t(bmax - cls(u)) + 1]++;
        for (size_t k = 1; k < pc.size(); ++k) pc[k] += pc[k - 1];
        std::vector<int32_t> uorder(n_up > 0 ? n_up : 1);
        for (int64_t u = 0; u < n_up; ++u) uorder[pc[size_t(bmax - cls(u))]++] = int32_t(u);
        s.up_order = upload(p, uorder);
    }
    s.pairs = upload(p, pr);
    if (p->opt.precision == BA_PRECISION_MIXED) {
        // upper pattern: the diagonal block first, then the upper blocks in (j, k) order
        std::vector<int64_t> row_u(size_t(n_c) + 1, 0);
        for (int32_t j = 0; j < n_c; ++j) row_u[j + 1] = row_u[j] + 1 + upper_cnt[j];
        const int64_t nnzb_u = row_u[n_c];
        std::vector<int32_t> col_u(nnzb_u);
        std::vector<int64_t> tile_u(size_t(n_c) + 1, 0);
        for (int32_t j = 0; j < n_c; ++j) {
            col_u[row_u[j]] = j;
            tile_u[j + 1] = tile_u[j] + (row_u[j + 1] - row_u[j] + ba::kTile - 1) / ba::kTile;
        }
        std::vector<int64_t> udst(n_up);
        {
            std::vector<int64_t> ufill(n_c);
            for (int32_t j = 0; j < n_c; ++j) ufill[j] = row_u[j] + 1;
            for (int64_t u = 0; u < n_up; ++u) {
                const int32_t j = up_j[u];
                const int64_t pos = ufill[j]++;
                col_u[pos] = up_k[u];
                udst[u] = (tile_u[j] * ba::kTile + (pos - row_u[j])) * 81;
            }
        }
        // per column k the upper blocks (j, k), j < k, in j order (u runs in (j, k) order)
        std::vector<int64_t> qptr(size_t(n_c) + 1, 0);
        for (int64_t u = 0; u < n_up; ++u) qptr[up_k[u] + 1]++;
        for (int32_t k = 0; k < n_c; ++k) qptr[k + 1] += qptr[k];
        if (n_up >= (int64_t(1) << 31)) throw Error(BA_ERR_INVALID_ARG, "too many blocks in S");
        std::vector<int32_t> cslot(size_t(tile_u[n_c]) * ba::kTile, -1);
        {
            std::vector<int64_t> fill(qptr.begin(), qptr.end() - 1);
            for (int64_t u = 0; u < n_up; ++u) cslot[udst[u] / 81] = int32_t(fill[up_k[u]]++);
        }
        s.nnzb_u = nnzb_u;
        s.row_ptr_u = upload(p, row_u);
        s.col_u = upload(p, col_u);
        s.tile_ptr_u = upload(p, tile_u);
        s.n_tiles_u = tile_u[n_c];
        s.up_udst = upload(p, udst);
        s.qptr = upload(p, qptr);
        s.cslot = upload(p, cslot);
        s.h_row_ptr_u = row_u;
        s.h_col_u = col_u;
        s.h_tile_ptr_u = tile_u;
    }
}

void alloc_system(ba_problem* p) {
    ba::Structure& s = p->s;
    ba::System& y = p->y;
    y.cams = dev_alloc<double>(p, size_t(s.n_c) * 9);
    y.aux = dev_alloc<double>(p, size_t(s.n_c) * 24);
    y.pts = dev_alloc<double>(p, size_t(s.n_l) * 3);
    y.r = dev_alloc<double>(p, size_t(s.n_o) * 2);
    y.Jc = dev_alloc<double>(p, size_t(s.n_o) * 18);
    y.Jl = dev_alloc<double>(p, size_t(s.n_o) * 6);
    if (p->opt.precision == BA_PRECISION_FP64) y.G = dev_alloc<double>(p, size_t(s.n_o) * 27);
    y.V = dev_alloc<double>(p, size_t(s.n_l) * 9);
    y.L = dev_alloc<double>(p, size_t(s.n_l) * 6);
    y.bl = dev_alloc<double>(p, size_t(s.n_l) * 3);
    y.e = dev_alloc<double>(p, size_t(s.n_l) * 3);
    y.U = dev_alloc<double>(p, size_t(s.n_c) * 81);
    y.bp = dev_alloc<double>(p, size_t(s.n_c) * 9);
    y.bt = dev_alloc<double>(p, size_t(s.n_c) * 9);
    y.Sd = dev_alloc<double>(p, size_t(s.n_c) * 81);
    if (p->opt.precision == BA_PRECISION_FP64) {
        y.S = dev_alloc<double>(p, size_t(s.n_tiles) * ba::kTileElems);
        BA_CUDA_TRY(cudaMemset(y.S, 0, sizeof(double) * size_t(s.n_tiles) * ba::kTileElems));   // padding stays 0
    }
    y.Dinv = dev_alloc<double>(p, size_t(s.n_c) * 81);
    if (p->opt.precision == BA_PRECISION_MIXED) {
        y.S32 = dev_alloc<float>(p, size_t(s.n_tiles) * ba::kTileElems);
        BA_CUDA_TRY(cudaMemset(y.S32, 0, sizeof(float) * size_t(s.n_tiles) * ba::kTileElems));
        y.S32u = dev_alloc<float>(p, size_t(s.n_tiles_u) * ba::kTileElems);
        BA_CUDA_TRY(cudaMemset(y.S32u, 0, sizeof(float) * size_t(s.n_tiles_u) * ba::kTileElems));
        y.G32 = dev_alloc<float>(p, size_t(s.n_o) * 36);   // three 16-byte aligned parts of 9 per row
        y.aux32 = dev_alloc<float>(p, size_t(s.n_c) * 24);
        y.PY32 = dev_alloc<float>(p, size_t(s.n_o) * 6);
        y.L32 = dev_alloc<float>(p, size_t(s.n_l) * 6);
        y.yl = dev_alloc<double>(p, size_t(s.n_l) * 3);
        y.auxd = dev_alloc<float2>(p, size_t(s.n_c) * 24);
        y.ptsd = dev_alloc<float2>(p, size_t(s.n_l) * 3);
        y.xd = dev_alloc<float2>(p, size_t(s.n_c) * 9);
        y.dadd = dev_alloc<double>(p, size_t(s.n_c) * 9);
        y.uv = dev_alloc<double>(p, size_t(s.n_o) * 2);
        y.lam = dev_alloc<double>(p, size_t(s.n_c) * 9);
        y.lam32 = dev_alloc<float>(p, size_t(s.n_c) * 9);
        y.Dhat = dev_alloc<double>(p, size_t(s.n_c) * 81);
    }
    y.status = dev_alloc<int>(p, 1);
    p->dxp = dev_alloc<double>(p, size_t(s.n_c) * 9);
    p->dxl = dev_alloc<double>(p, size_t(s.n_l) * 3);
    p->tmp_cams = dev_alloc<double>(p, size_t(s.n_c) * 9);
    p->tmp_pts = dev_alloc<double>(p, size_t(s.n_l) * 3);
    p->cost_parts = ba::num_sms() * 4;
    p->cost_part = dev_alloc<double>(p, size_t(p->cost_parts));
}

void check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

void do_build(ba_problem* p, double lambda) {
    if (!(lambda > 0.0) || !std::isfinite(lambda)) throw Error(BA_ERR_INVALID_ARG, "lambda must be positive and finite");
    cudaStream_t st = p->stream;
    ba::Structure& s = p->s;
    ba::System& y = p->y;
    y.built = false;
    p->solved = false;
    BA_CUDA_TRY(cudaMemsetAsync(y.status, 0, sizeof(int), st));
    ba::launch_cam_prep(s, y, st);
    ba::launch_linearize(s, y, st);
    ba::launch_landmarks(s, y, p->opt.damping, lambda, st);
    if (p->opt.precision == BA_PRECISION_FP64) {
        ba::launch_obs_G(s, y, st);
        ba::launch_cameras(s, y, p->opt.damping, lambda, st);
        ba::launch_schur_diag(s, y, st);
        ba::launch_block_jacobi(s, y, st);
        ba::launch_schur(s, y, st);          // off-diagonal blocks + the diagonal from Sd
        p->launches += 9;
    } else {
        // float64: b~ and the damping; float32 Jacobians: diagonal blocks, Lam G rows, S^
        ba::launch_cam_rhs(s, y, p->opt.damping, lambda, st);
        ba::launch_schur_diag32(s, y, st);
        ba::launch_block_jacobi(s, y, st);
        ba::launch_schur_mixed(s, y, st);    // off-diagonal and diagonal blocks of S^ (float32)
        p->launches += 8;
    }
    check_launch();
    int status = 0;
    BA_CUDA_TRY(cudaMemcpyAsync(&status, y.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    if (status != 0) throw Error(status, "a damped V_lambda or a diagonal block of S is not positive definite");
    y.lambda = lambda;
    y.built = true;
}

int do_solve(ba_problem* p, const ba::SolveArgs& a, ba_solve_stats* st) {
    if (!p->y.built) throw Error(BA_ERR_STATE, "ba_build_normal must succeed before a solve");
    if (!(a.tol > 0.0) || a.max_iters < 0 || a.max_iters > 1000000) throw Error(BA_ERR_INVALID_ARG, "bad tol or max_iters");
    if (a.mcg && (a.n_dirs < 1 || a.n_dirs > ba::kMaxDirs)) throw Error(BA_ERR_INVALID_ARG, "n_dirs must be in [1, 16]");
    if (a.mcg && !(a.tau >= 0.0)) throw Error(BA_ERR_INVALID_ARG, "tau must be >= 0");
    if (!p->solver) p->solver = ba::solver_create();
    ba::SolveOut out;
    try {
        ba::solver_run(p->solver, p->s, p->y, a, p->dxp, out, p->stream);
    } catch (...) {
        p->launches += out.launches;
        throw;
    }
    p->launches += out.launches;
    p->solved = true;
    p->last = out.probs;
    p->last_ms = out.ms;
    if (st) {
        st->status = out.status;
        st->iters = out.iters;
        st->local_steps = out.local_steps;
        st->n_dirs_eff = out.n_eff;
        st->refinements = out.refinements;
        st->history_cols = int32_t(out.history_cols);
        st->pinv_steps = out.pinv_steps;
        st->host_waits = out.host_waits;
        st->rel_residual = out.rel_residual;
        st->true_rel_residual = out.true_rel_residual;
        st->ms = out.ms;
    }
    if (out.status != BA_OK) {
        p->err = out.status == BA_ERR_NOT_CONVERGED ? "max_iters reached before the tolerance"
               : out.status == BA_ERR_OOM ? "direction history capacity exceeded"
               : out.status == BA_ERR_TIMEOUT ? "a bounded device wait for a tile copy gave up (wait_polls)"
                                              : "Krylov breakdown (non-positive curvature or NaN)";
    }
    return out.status;
}

double do_cost(ba_problem* p, const double* cams, const double* pts) {
    ba::launch_cost(p->s, cams, pts, p->cost_part, p->cost_parts, p->stream);
    check_launch();
    p->launches += 1;
    std::vector<double> h(p->cost_parts);
    copy_out(h.data(), p->cost_part, sizeof(double) * h.size(), p->stream);
    double c = 0.0;
    for (double v : h) c += v;
    return c;
}

ba::SolveArgs make_args(const ba_problem* p, int mcg, double tol, int32_t max_iters, int32_t n_dirs, double tau) {
    ba::SolveArgs a;
    a.mcg = mcg;
    a.tol = tol;
    a.max_iters = max_iters;
    a.n_dirs = n_dirs;
    a.tau = tau;
    a.chunk = p->opt.chunk_iters;
    a.precision = p->opt.precision;
    a.inner_tol = p->opt.inner_tol;
    a.max_refine = p->opt.max_refine;
    a.max_history = p->opt.max_history;
    a.item_blocks = p->opt.item_blocks;
    a.host_loop = p->opt.host_loop;
    a.spmv_cfg = p->opt.spmv_config;
    a.wait_polls = p->opt.wait_polls == 0 ? ba::kDefaultWaitPolls : (p->opt.wait_polls < 0 ? 0 : p->opt.wait_polls);
    return a;
}

void check_options(const ba_options& o) {
    if (o.chunk_iters < 1 || o.chunk_iters > 256) throw Error(BA_ERR_INVALID_ARG, "chunk_iters must be in [1, 256]");
    if (o.damping != BA_DAMPING_MARQUARDT && o.damping != BA_DAMPING_IDENTITY)
        throw Error(BA_ERR_INVALID_ARG, "unknown damping");
    if (o.precision != BA_PRECISION_FP64 && o.precision != BA_PRECISION_MIXED)
        throw Error(BA_ERR_INVALID_ARG, "unknown precision");
    if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) throw Error(BA_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
    if (o.max_refine < 1) throw Error(BA_ERR_INVALID_ARG, "max_refine must be >= 1");
    if (o.item_blocks != 0 && (o.item_blocks < 32 || o.item_blocks > 4096 || o.item_blocks % 32 != 0))
        throw Error(BA_ERR_INVALID_ARG, "item_blocks must be 0 or a multiple of 32 in [32, 4096]");
    if (o.wait_polls < -1 || o.wait_polls > (1 << 30)) throw Error(BA_ERR_INVALID_ARG, "wait_polls must be in [-1, 2^30]");
    if (o.host_loop != 0 && o.host_loop != 1) throw Error(BA_ERR_INVALID_ARG, "host_loop must be 0 or 1");
    if (o.spmv_config < 0 || o.spmv_config > 2) throw Error(BA_ERR_INVALID_ARG, "spmv_config must be in [0, 2]");
}

int create(const ba_options* opt, int32_t n_problems, const int32_t* cam_off_in, int32_t n_cams, int32_t n_pts,
           int64_t n_obs, const double* cams, const double* pts, const int32_t* obs_cam, const int32_t* obs_pt,
           const double* obs_xy, ba_problem** out) {
    g_create_error.clear();
    ba::set_thread_error("");
    if (!out) { g_create_error = "out is NULL"; return BA_ERR_INVALID_ARG; }
    *out = nullptr;
    ba_problem* p = nullptr;
    try {
        if (n_cams < 1 || n_pts < 1 || n_obs < 1) throw Error(BA_ERR_INVALID_ARG, "n_cams, n_pts and n_obs must be >= 1");
        if (n_obs >= (int64_t(1) << 31)) throw Error(BA_ERR_INVALID_ARG, "n_obs must be < 2^31");
        if (!cams || !pts || !obs_cam || !obs_pt || !obs_xy) throw Error(BA_ERR_INVALID_ARG, "NULL input array");
        if (n_problems < 1 || n_problems > 65535) throw Error(BA_ERR_INVALID_ARG, "n_problems must be in [1, 65535]");
        std::vector<int32_t> cam_off{0, n_cams};
        if (cam_off_in) {
            cam_off = fetch(cam_off_in, size_t(n_problems) + 1);
            if (cam_off[0] != 0 || cam_off[n_problems] != n_cams)
                throw Error(BA_ERR_INVALID_ARG, "cam_off must start at 0 and end at n_cams");
            for (int32_t b = 0; b < n_problems; ++b)
                if (cam_off[b + 1] <= cam_off[b])
                    throw Error(BA_ERR_INVALID_ARG, "problem " + std::to_string(b) + " has no camera");
        } else if (n_problems != 1) {
            throw Error(BA_ERR_INVALID_ARG, "cam_off is NULL");
        }
        p = new ba_problem();
        ba_default_options(&p->opt);
        if (opt) p->opt = *opt;
        check_options(p->opt);
        build_structure(p, n_cams, n_pts, n_obs, obs_cam, obs_pt, obs_xy, cam_off);
        alloc_system(p);
        BA_CUDA_TRY(cudaMemcpy(p->y.cams, cams, sizeof(double) * 9 * size_t(n_cams), cudaMemcpyDefault));
        BA_CUDA_TRY(cudaMemcpy(p->y.pts, pts, sizeof(double) * 3 * size_t(n_pts), cudaMemcpyDefault));
        *out = p;
        return BA_OK;
    } catch (const Error& e) {
        g_create_error = e.msg;
        if (p) ba_problem_destroy(p);
        return e.code;
    } catch (const std::bad_alloc&) {
        g_create_error = "host allocation failed";
        if (p) ba_problem_destroy(p);
        return BA_ERR_OOM;
    }
}

}  // namespace

extern "C" {

void ba_default_options(ba_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->damping = BA_DAMPING_MARQUARDT;
    opt->precision = BA_PRECISION_FP64;
    opt->chunk_iters = 8;
    opt->max_history = 0;
    opt->inner_tol = 1e-6;
    opt->max_refine = 64;
}

int ba_problem_create(const ba_options* opt, int32_t n_cams, int32_t n_pts, int64_t n_obs, const double* cams,
                      const double* pts, const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_xy,
                      ba_problem** out) {
    return create(opt, 1, nullptr, n_cams, n_pts, n_obs, cams, pts, obs_cam, obs_pt, obs_xy, out);
}

int ba_batch_create(const ba_options* opt, int32_t n_problems, const int32_t* cam_off, int32_t n_cams, int32_t n_pts,
                    int64_t n_obs, const double* cams, const double* pts, const int32_t* obs_cam,
                    const int32_t* obs_pt, const double* obs_xy, ba_problem** out) {
    if (!cam_off) {
        g_create_error = "cam_off is NULL";
        if (out) *out = nullptr;
        return BA_ERR_INVALID_ARG;
    }
    return create(opt, n_problems, cam_off, n_cams, n_pts, n_obs, cams, pts, obs_cam, obs_pt, obs_xy, out);
}

void ba_problem_destroy(ba_problem* p) {
    if (!p) return;
    if (p->solver) ba::solver_destroy(p->solver);
    for (void* d : p->owned) cudaFree(d);
    delete p;
}

const char* ba_last_error(const ba_problem* p) {
    if (!p) return ba::g_thread_error.empty() ? g_create_error.c_str() : ba::g_thread_error.c_str();
    return p->err.c_str();
}

int ba_set_stream(ba_problem* p, void* stream) {
    if (!p) return BA_ERR_INVALID_ARG;
    p->stream = static_cast<cudaStream_t>(stream);
    return BA_OK;
}

int ba_set_params(ba_problem* p, const double* cams, const double* pts) {
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        if (cams) BA_CUDA_TRY(cudaMemcpyAsync(p->y.cams, cams, sizeof(double) * 9 * size_t(p->s.n_c), cudaMemcpyDefault, p->stream));
        if (pts) BA_CUDA_TRY(cudaMemcpyAsync(p->y.pts, pts, sizeof(double) * 3 * size_t(p->s.n_l), cudaMemcpyDefault, p->stream));
        BA_CUDA_TRY(cudaStreamSynchronize(p->stream));
        p->y.built = false;
        p->solved = false;
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_get_params(const ba_problem* pc, double* cams, double* pts) {
    ba_problem* p = const_cast<ba_problem*>(pc);
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        copy_out(cams, p->y.cams, sizeof(double) * 9 * size_t(p->s.n_c), p->stream);
        copy_out(pts, p->y.pts, sizeof(double) * 3 * size_t(p->s.n_l), p->stream);
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_build_normal(ba_problem* p, double lambda) {
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        do_build(p, lambda);
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_solve_pcg(ba_problem* p, double tol, int32_t max_iters, ba_solve_stats* st) {
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        return do_solve(p, make_args(p, 0, tol, max_iters, 1, 0.0), st);
    } catch (const Error& e) {
        if (st) st->status = e.code;
        return fail(p, e);
    }
}

int ba_solve_mcg(ba_problem* p, double tol, int32_t max_iters, int32_t n_dirs, double tau, ba_solve_stats* st) {
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        return do_solve(p, make_args(p, 1, tol, max_iters, n_dirs, tau), st);
    } catch (const Error& e) {
        if (st) st->status = e.code;
        return fail(p, e);
    }
}

int ba_get_delta(ba_problem* p, double* dxp, double* dxl) {
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        if (!p->solved) throw Error(BA_ERR_STATE, "no solution: call a solve first");
        copy_out(dxp, p->dxp, sizeof(double) * 9 * size_t(p->s.n_c), p->stream);
        if (dxl) {
            ba::launch_back_substitute(p->s, p->y, p->dxp, p->dxl, p->stream);
            check_launch();
            p->launches += p->y.G ? 1 : 2;   // mixed: the split of dx_p, then the landmarks
            copy_out(dxl, p->dxl, sizeof(double) * 3 * size_t(p->s.n_l), p->stream);
        }
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_cost(ba_problem* p, double* cost) {
    if (!p || !cost) return BA_ERR_INVALID_ARG;
    try {
        *cost = do_cost(p, p->y.cams, p->y.pts);
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_lm_step(ba_problem* p, int32_t solver, double lambda0, double tol, int32_t max_iters, int32_t n_dirs,
               double tau, double ftol, ba_lm_stats* st) {
    if (!p) return BA_ERR_INVALID_ARG;
    ba_lm_stats s;
    std::memset(&s, 0, sizeof(s));
    try {
        if (solver != BA_SOLVER_PCG && solver != BA_SOLVER_MCG) throw Error(BA_ERR_INVALID_ARG, "unknown solver");
        if (p->s.h_cam_off.size() > 2) throw Error(BA_ERR_INVALID_ARG, "ba_lm_step takes a single-problem handle");
        if (p->lm_lambda <= 0.0) {
            if (!(lambda0 > 0.0)) throw Error(BA_ERR_INVALID_ARG, "lambda0 must be positive");
            p->lm_lambda = lambda0;
        }
        cudaEvent_t e0, e1;
        BA_CUDA_TRY(cudaEventCreate(&e0));
        BA_CUDA_TRY(cudaEventCreate(&e1));
        BA_CUDA_TRY(cudaEventRecord(e0, p->stream));
        const double lam = p->lm_lambda;
        s.lambda_used = lam;
        s.cost_before = do_cost(p, p->y.cams, p->y.pts);
        int code = BA_OK;
        bool have_step = true;
        try {
            do_build(p, lam);
        } catch (const Error& e) {
            if (e.code != BA_ERR_SINGULAR) throw;
            have_step = false;   // treat like a rejected step: raise lambda
        }
        if (have_step) {
            ba_solve_stats ss;
            code = do_solve(p, make_args(p, solver == BA_SOLVER_MCG, tol, max_iters, n_dirs, tau), &ss);
            s.solver_iters = ss.iters;
            s.solve_ms = ss.ms;
            if (code != BA_OK && code != BA_ERR_NOT_CONVERGED) have_step = false;
        }
        if (have_step) {
            ba::launch_back_substitute(p->s, p->y, p->dxp, p->dxl, p->stream);
            ba::launch_add_params(p->y.cams, p->dxp, p->tmp_cams, int64_t(p->s.n_c) * 9, p->stream);
            ba::launch_add_params(p->y.pts, p->dxl, p->tmp_pts, int64_t(p->s.n_l) * 3, p->stream);
            check_launch();
            p->launches += p->y.G ? 3 : 4;
            s.cost_after = do_cost(p, p->tmp_cams, p->tmp_pts);
        } else {
            s.cost_after = s.cost_before;
        }
        if (have_step && s.cost_after < s.cost_before) {
            BA_CUDA_TRY(cudaMemcpyAsync(p->y.cams, p->tmp_cams, sizeof(double) * 9 * size_t(p->s.n_c),
                                        cudaMemcpyDeviceToDevice, p->stream));
            BA_CUDA_TRY(cudaMemcpyAsync(p->y.pts, p->tmp_pts, sizeof(double) * 3 * size_t(p->s.n_l),
                                        cudaMemcpyDeviceToDevice, p->stream));
            s.accepted = 1;
            s.converged = (s.cost_before - s.cost_after) / s.cost_before < ftol;
            p->lm_lambda = std::max(lam / 10.0, 1e-12);
            p->y.built = false;
        } else {
            s.accepted = 0;
            p->lm_lambda = std::min(lam * 10.0, 1e16);
        }
        s.lambda_next = p->lm_lambda;
        BA_CUDA_TRY(cudaEventRecord(e1, p->stream));
        BA_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        s.ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        s.status = code == BA_ERR_NOT_CONVERGED ? BA_OK : code;
        if (st) *st = s;
        return s.status;
    } catch (const Error& e) {
        s.status = e.code;
        if (st) *st = s;
        return fail(p, e);
    }
}

int ba_project(int32_t n_cams, int32_t n_pts, int64_t n_obs, const double* cams, const double* pts,
               const int32_t* obs_cam, const int32_t* obs_pt, double* out_xy, void* stream) {
    if (n_cams < 1 || n_pts < 1 || n_obs < 0) return BA_ERR_INVALID_ARG;
    if (n_obs == 0) return BA_OK;
    if (!cams || !pts || !obs_cam || !obs_pt || !out_xy) return BA_ERR_INVALID_ARG;
    ba::launch_project(n_obs, cams, pts, obs_cam, obs_pt, out_xy, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? BA_OK : BA_ERR_CUDA;
}

int ba_get_linearization(const ba_problem* pc, double* r, double* Jp, double* Jl) {
    ba_problem* p = const_cast<ba_problem*>(pc);
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        if (!p->y.built) throw Error(BA_ERR_STATE, "nothing built");
        const int64_t n_o = p->s.n_o;
        const double* src[3] = {p->y.r, p->y.Jc, p->y.Jl};
        double* dst[3] = {r, Jp, Jl};
        const int width[3] = {2, 18, 6};
        for (int k = 0; k < 3; ++k) {
            if (!dst[k]) continue;
            double* tmp = nullptr;
            BA_CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * n_o * width[k]));
            ba::launch_unpermute(src[k], p->s.perm, tmp, n_o, width[k], p->stream);
            // mixed precision keeps these in double-float (8 bytes per value, moved as such above)
            if (p->opt.precision == BA_PRECISION_MIXED) ba::launch_df_to_double(tmp, n_o * width[k], p->stream);
            cudaError_t e = cudaMemcpyAsync(dst[k], tmp, sizeof(double) * n_o * width[k], cudaMemcpyDefault, p->stream);
            cudaStreamSynchronize(p->stream);
            cudaFree(tmp);
            if (e != cudaSuccess) throw Error(BA_ERR_CUDA, cudaGetErrorString(e));
        }
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_get_normal(const ba_problem* pc, double* U, double* V, double* b_p, double* b_l) {
    ba_problem* p = const_cast<ba_problem*>(pc);
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        if (!p->y.built) throw Error(BA_ERR_STATE, "nothing built");
        const ba::Structure& s = p->s;
        if (p->opt.precision == BA_PRECISION_MIXED) {
            // the mixed build keeps r, J_p, J_l in double-float and needs none of U, V, b_p, b_l in
            // float64: form them on request from float64 copies, with the kernels of the float64 build
            const size_t n_o = size_t(s.n_o), n_l = size_t(s.n_l);
            const size_t sizes[7] = {2 * n_o, 18 * n_o, 6 * n_o, 9 * n_l, 6 * n_l, 3 * n_l, 3 * n_l};
            double* t[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < 7 && e == cudaSuccess; ++k) e = cudaMalloc(&t[k], sizeof(double) * (sizes[k] ? sizes[k] : 1));
            if (e == cudaSuccess) {
                ba::launch_normal_request(s, p->y, p->opt.damping, p->y.lambda, t[0], t[1], t[2], t[3], t[4], t[5],
                                          t[6], p->stream);
                e = cudaGetLastError();
                p->launches += 8;
            }
            if (e == cudaSuccess) {
                try {
                    copy_out(U, p->y.U, sizeof(double) * 81 * size_t(s.n_c), p->stream);
                    copy_out(V, t[3], sizeof(double) * 9 * n_l, p->stream);
                    copy_out(b_p, p->y.bp, sizeof(double) * 9 * size_t(s.n_c), p->stream);
                    copy_out(b_l, t[5], sizeof(double) * 3 * n_l, p->stream);
                } catch (...) {
                    for (double* q : t) if (q) cudaFree(q);
                    throw;
                }
            }
            cudaStreamSynchronize(p->stream);
            for (double* q : t) if (q) cudaFree(q);
            if (e != cudaSuccess) throw Error(BA_ERR_CUDA, std::string("normal equation on request: ") + cudaGetErrorString(e));
            return BA_OK;
        }
        copy_out(U, p->y.U, sizeof(double) * 81 * size_t(s.n_c), p->stream);
        copy_out(V, p->y.V, sizeof(double) * 9 * size_t(s.n_l), p->stream);
        copy_out(b_p, p->y.bp, sizeof(double) * 9 * size_t(s.n_c), p->stream);
        copy_out(b_l, p->y.bl, sizeof(double) * 3 * size_t(s.n_l), p->stream);
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_get_schur_nnzb(const ba_problem* p, int64_t* nnzb) {
    if (!p || !nnzb) return BA_ERR_INVALID_ARG;
    *nnzb = p->s.nnzb;
    return BA_OK;
}

int ba_get_schur(const ba_problem* pc, int64_t* row_ptr, int32_t* col, double* blocks, double* btilde) {
    ba_problem* p = const_cast<ba_problem*>(pc);
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        copy_out(row_ptr, p->s.row_ptr, sizeof(int64_t) * (size_t(p->s.n_c) + 1), p->stream);
        copy_out(col, p->s.col, sizeof(int32_t) * size_t(p->s.nnzb), p->stream);
        if (blocks || btilde) {
            if (!p->y.built) throw Error(BA_ERR_STATE, "nothing built");
        }
        if (blocks) {
            double* tmp = nullptr;
            BA_CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * 81 * size_t(p->s.nnzb)));
            ba::launch_unslab(p->s, p->y, tmp, p->stream);
            cudaError_t e = cudaMemcpyAsync(blocks, tmp, sizeof(double) * 81 * size_t(p->s.nnzb), cudaMemcpyDefault, p->stream);
            cudaStreamSynchronize(p->stream);
            cudaFree(tmp);
            if (e != cudaSuccess) throw Error(BA_ERR_CUDA, cudaGetErrorString(e));
        }
        copy_out(btilde, p->y.bt, sizeof(double) * 9 * size_t(p->s.n_c), p->stream);
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_get_preconditioner(const ba_problem* pc, double* Dinv) {
    ba_problem* p = const_cast<ba_problem*>(pc);
    if (!p || !Dinv) return BA_ERR_INVALID_ARG;
    try {
        if (!p->y.built) throw Error(BA_ERR_STATE, "nothing built");
        if (p->opt.precision == BA_PRECISION_MIXED) {
            // the mixed build inverts only the scaled blocks; D^{-1} of S itself is formed here
            ba::launch_block_jacobi_plain(p->s, p->y, p->stream);
            check_launch();
            ++p->launches;
        }
        copy_out(Dinv, p->y.Dinv, sizeof(double) * 81 * size_t(p->s.n_c), p->stream);
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_get_residual_history(const ba_problem* pc, double* hist, int32_t cap, int32_t* n) {
    ba_problem* p = const_cast<ba_problem*>(pc);
    if (!p || !n) return BA_ERR_INVALID_ARG;
    try {
        if (!p->solver || !p->solved) { *n = 0; return BA_OK; }
        const double* h = nullptr;
        int cnt = ba::solver_history(p->solver, 0, &h);
        *n = cnt;
        int m = cnt < cap ? cnt : cap;
        if (hist && m > 0) BA_CUDA_TRY(cudaMemcpy(hist, h, sizeof(double) * m, cudaMemcpyDefault));
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_get_batch_size(const ba_problem* p, int32_t* n_problems) {
    if (!p || !n_problems) return BA_ERR_INVALID_ARG;
    *n_problems = int32_t(p->s.h_cam_off.size()) - 1;
    return BA_OK;
}

int ba_get_batch_stats(const ba_problem* pc, ba_solve_stats* stats, int32_t n) {
    ba_problem* p = const_cast<ba_problem*>(pc);
    if (!p || !stats) return BA_ERR_INVALID_ARG;
    try {
        const int nb = int(p->s.h_cam_off.size()) - 1;
        if (n != nb) throw Error(BA_ERR_INVALID_ARG, "n must equal the number of problems");
        if (!p->solved || int(p->last.size()) != nb) throw Error(BA_ERR_STATE, "no solution: call a solve first");
        for (int b = 0; b < nb; ++b) {
            const ba::ProbOut& o = p->last[b];
            ba_solve_stats& st = stats[b];
            st.status = o.status;
            st.iters = o.iters;
            st.local_steps = o.local_steps;
            st.n_dirs_eff = o.n_eff;
            st.refinements = o.refinements;
            st.history_cols = int32_t(o.history_cols);
            st.rel_residual = o.rel_residual;
            st.true_rel_residual = o.true_rel_residual;
            st.ms = p->last_ms;
        }
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_get_batch_history(const ba_problem* pc, int32_t problem, double* hist, int32_t cap, int32_t* n) {
    ba_problem* p = const_cast<ba_problem*>(pc);
    if (!p || !n) return BA_ERR_INVALID_ARG;
    try {
        const int nb = int(p->s.h_cam_off.size()) - 1;
        if (problem < 0 || problem >= nb) throw Error(BA_ERR_INVALID_ARG, "problem out of range");
        if (!p->solver || !p->solved) { *n = 0; return BA_OK; }
        const double* h = nullptr;
        int cnt = ba::solver_history(p->solver, problem, &h);
        *n = cnt;
        int m = cnt < cap ? cnt : cap;
        if (hist && m > 0) BA_CUDA_TRY(cudaMemcpy(hist, h, sizeof(double) * m, cudaMemcpyDefault));
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

int ba_autotune(ba_problem* p, int32_t reps, int32_t* item_blocks, int32_t* spmv_config, double* ms) {
    if (!p) return BA_ERR_INVALID_ARG;
    try {
        if (reps < 1) throw Error(BA_ERR_INVALID_ARG, "reps must be >= 1");
        if (!p->y.built) throw Error(BA_ERR_STATE, "nothing built");
        if (!p->solver) p->solver = ba::solver_create();
        // choices kept for the process, keyed by precision and problem size
        struct Tuned {
            int cfg, cb;
            double ms;
        };
        static std::mutex mu;
        static std::map<std::tuple<int, int64_t, int64_t, int64_t>, Tuned> cache;
        const auto key = std::make_tuple(p->opt.precision, int64_t(p->s.n_c), p->s.nnzb,
                                         int64_t(p->s.h_cam_off.size()) - 1);
        Tuned t{0, 0, 0.0};
        bool hit = false;
        {
            std::lock_guard<std::mutex> lock(mu);
            auto it = cache.find(key);
            if (it != cache.end()) {
                t = it->second;
                hit = true;
            }
        }
        if (!hit) {
            ba::solver_autotune(p->solver, p->s, p->y, p->opt.precision == BA_PRECISION_MIXED, reps, &t.cfg, &t.cb,
                                &t.ms, p->stream);
            std::lock_guard<std::mutex> lock(mu);
            cache[key] = t;
        }
        p->opt.item_blocks = t.cb;
        p->opt.spmv_config = t.cfg;
        if (item_blocks) *item_blocks = t.cb;
        if (spmv_config) *spmv_config = t.cfg;
        if (ms) *ms = t.ms;
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

}  // extern "C"

struct ba_gnn {
    ba::Gnn* g = nullptr;
    std::string err;
};

namespace {
int gnn_fail(ba_gnn* g, const Error& e) {
    if (g) g->err = e.msg;
    return e.code;
}
}  // namespace

extern "C" {

int ba_gnn_create(ba_gnn** out) {
    if (!out) return BA_ERR_INVALID_ARG;
    *out = nullptr;
    ba_gnn* g = new ba_gnn();
    try {
        g->g = ba::gnn_create();
        *out = g;
        return BA_OK;
    } catch (const Error& e) {
        g_create_error = e.msg;
        delete g;
        return e.code;
    }
}

void ba_gnn_destroy(ba_gnn* g) {
    if (!g) return;
    ba::gnn_destroy(g->g);
    delete g;
}

const char* ba_gnn_last_error(const ba_gnn* g) { return g ? g->err.c_str() : ""; }

int ba_gnn_param_count(int64_t* n) {
    if (!n) return BA_ERR_INVALID_ARG;
    *n = ba::gnn_param_count();
    return BA_OK;
}

int ba_gnn_set_params(ba_gnn* g, const float* params) {
    if (!g || !params) return BA_ERR_INVALID_ARG;
    try {
        ba::gnn_set_params(g->g, params, nullptr);
        return BA_OK;
    } catch (const Error& e) {
        return gnn_fail(g, e);
    }
}

int ba_gnn_get_params(const ba_gnn* gc, float* params) {
    ba_gnn* g = const_cast<ba_gnn*>(gc);
    if (!g || !params) return BA_ERR_INVALID_ARG;
    try {
        ba::gnn_get_params(g->g, params, nullptr);
        return BA_OK;
    } catch (const Error& e) {
        return gnn_fail(g, e);
    }
}

int ba_gnn_graph(ba_gnn* g, ba_problem* p, float* features, float* coupling) {
    if (!g || !p) return BA_ERR_INVALID_ARG;
    try {
        ba::gnn_graph_out(g->g, p->s, p->y, features, coupling, p->stream);
        return BA_OK;
    } catch (const Error& e) {
        return gnn_fail(g, e);
    }
}

int ba_gnn_loss(ba_gnn* g, ba_problem* p, double* loss, float* scores, float* grad) {
    if (!g || !p) return BA_ERR_INVALID_ARG;
    try {
        const double L = ba::gnn_loss(g->g, p->s, p->y, grad != nullptr, scores, grad, p->stream);
        if (loss) *loss = L;
        return BA_OK;
    } catch (const Error& e) {
        return gnn_fail(g, e);
    }
}

int ba_gnn_train_step(ba_gnn* g, ba_problem* p, double lr, double* loss) {
    if (!g || !p) return BA_ERR_INVALID_ARG;
    try {
        if (!(lr > 0.0) || !std::isfinite(lr)) throw Error(BA_ERR_INVALID_ARG, "lr must be positive");
        const double L = ba::gnn_train_step(g->g, p->s, p->y, lr, p->stream);
        if (loss) *loss = L;
        return BA_OK;
    } catch (const Error& e) {
        return gnn_fail(g, e);
    }
}

int ba_gnn_order(ba_gnn* g, ba_problem* p, int32_t bf16, int32_t* order, double* loss) {
    if (!g || !p || !order) return BA_ERR_INVALID_ARG;
    try {
        const double L = ba::gnn_order(g->g, p->s, p->y, bf16 != 0, order, p->stream);
        if (loss) *loss = L;
        return BA_OK;
    } catch (const Error& e) {
        return gnn_fail(g, e);
    }
}

int ba_gnn_launch_count(const ba_gnn* g, int64_t* n) {
    if (!g || !n) return BA_ERR_INVALID_ARG;
    *n = ba::gnn_launches(g->g);
    return BA_OK;
}

int ba_get_launch_count(const ba_problem* p, int64_t* n) {
    if (!p || !n) return BA_ERR_INVALID_ARG;
    *n = p->launches;
    return BA_OK;
}

int ba_time_kernel(ba_problem* p, int32_t kernel, int32_t reps, double* ms) {
    if (!p || !ms) return BA_ERR_INVALID_ARG;
    try {
        if (reps < 1) throw Error(BA_ERR_INVALID_ARG, "reps must be >= 1");
        if (!p->y.built) throw Error(BA_ERR_STATE, "nothing built");
        cudaStream_t st = p->stream;
        if (kernel == BA_KERNEL_SPMV) {
            if (!p->solver) p->solver = ba::solver_create();
            *ms = ba::solver_time_spmv(p->solver, p->s, p->y, p->opt.precision == BA_PRECISION_MIXED, reps,
                                     p->opt.item_blocks, p->opt.spmv_config, st);
            return BA_OK;
        }
        if (kernel < BA_KERNEL_SCHUR || kernel > BA_KERNEL_BLOCK_JACOBI) throw Error(BA_ERR_INVALID_ARG, "unknown kernel");
        const bool fp64 = p->opt.precision == BA_PRECISION_FP64;
        cudaEvent_t a, b;
        BA_CUDA_TRY(cudaEventCreate(&a));
        BA_CUDA_TRY(cudaEventCreate(&b));
        double total = 0.0;
        for (int k = 0; k < reps; ++k) {
            ba::flush_l2(st);
            BA_CUDA_TRY(cudaEventRecord(a, st));
            switch (kernel) {
                case BA_KERNEL_SCHUR:
                    if (fp64) ba::launch_schur(p->s, p->y, st);
                    else {
                        // the float32 Schur complement from the float32 Jacobians: diagonal blocks and G
                        // rows, Lam and the preconditioner, off-diagonal blocks
                        ba::launch_schur_diag32(p->s, p->y, st);
                        ba::launch_block_jacobi(p->s, p->y, st);
                        ba::launch_schur_mixed(p->s, p->y, st);
                    }
                    break;
                case BA_KERNEL_LINEARIZE:
                    ba::launch_cam_prep(p->s, p->y, st);
                    ba::launch_linearize(p->s, p->y, st);
                    break;
                case BA_KERNEL_LANDMARKS:
                    ba::launch_landmarks(p->s, p->y, p->opt.damping, p->y.lambda, st);
                    break;
                case BA_KERNEL_CAM_RHS:
                    if (fp64) {
                        ba::launch_obs_G(p->s, p->y, st);
                        ba::launch_cameras(p->s, p->y, p->opt.damping, p->y.lambda, st);
                    } else {
                        ba::launch_cam_rhs(p->s, p->y, p->opt.damping, p->y.lambda, st);
                    }
                    break;
                case BA_KERNEL_SCHUR_DIAG:
                    if (fp64) ba::launch_schur_diag(p->s, p->y, st);
                    else ba::launch_schur_diag32(p->s, p->y, st);
                    break;
                case BA_KERNEL_SCHUR_OFF:
                    if (fp64) ba::launch_schur(p->s, p->y, st);
                    else ba::launch_schur_mixed(p->s, p->y, st);
                    break;
                default:
                    ba::launch_block_jacobi(p->s, p->y, st);
                    break;
            }
            BA_CUDA_TRY(cudaEventRecord(b, st));
            BA_CUDA_TRY(cudaEventSynchronize(b));
            check_launch();
            float t = 0.f;
            BA_CUDA_TRY(cudaEventElapsedTime(&t, a, b));
            total += t;
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        *ms = total / reps;
        return BA_OK;
    } catch (const Error& e) {
        return fail(p, e);
    }
}

}  // extern "C"

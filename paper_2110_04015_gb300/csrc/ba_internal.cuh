// Internal declarations shared by the translation units of libba.
//
// Data layout in device memory (one problem):
//   observations are kept sorted by landmark ("point order"); perm maps a
//   point-order slot back to the caller's observation index.
//   per observation : r (2), Jc (2x9), Jl (2x3), G = W_o L_l^{-T} (9x3, float64 precision only)
//   per landmark    : V_lambda (3x3), its Cholesky factor L (6 packed, with the reciprocals of
//                     its diagonal: 1/l00, l10, 1/l11, l20, l21, 1/l22), b_l (3), e = L^{-1} b_l (3)
//   per camera      : U_lambda (9x9), b_p (9), b~ (9), D_j^{-1} (9x9)
//   S               : block-CSR over cameras, every nonzero 9x9 block of both
//                     triangles, each block 81 contiguous values (row-major).  The
//                     blocks of block-row j are grouped in tiles of 32 consecutive
//                     blocks, the last tile of a row padded with zero blocks, so a
//                     tile is one contiguous run (10 KB float32, 20 KB float64) that
//                     a bulk copy moves to shared memory; lanes that take the 32
//                     blocks of a tile then read shared memory at stride 81 (odd:
//                     no bank conflicts in float32), and a warp that builds one
//                     block writes 81 consecutive values.
// With G_o = W_o L_l^{-T} (V_l = L_l L_l^T) the Schur complement of Eq. 13 is
//   S_jk = delta_jk U_j - sum_{l seen by j and k} G_jl G_kl^T,
// and b~_j = b_p,j - sum_{o in camera j} G_o e_l (Eq. 14).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ba.h"

namespace ba {

constexpr int kThreads = 256;
constexpr int kTile = 32;                 // blocks per tile of S
constexpr int kTileElems = 81 * kTile;    // values per tile

// Index of entry e (= 9 a + b) of the q-th block (row-local) of block-row j of S.
__host__ __device__ __forceinline__ int64_t s_at(const int64_t* tile_ptr, int64_t j, int64_t q, int e) {
    return (tile_ptr[j] * kTile + q) * 81 + e;
}
constexpr int kMaxDirs = 16;   // widest direction block held by the small FP64 solves
constexpr int kDefaultWaitPolls = 1 << 20;   // polls of a tile copy's barrier before a wait gives up

#define BA_CUDA_TRY(expr)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            throw ::ba::Error(BA_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
        }                                                                                   \
    } while (0)

struct Error {
    int code;
    std::string msg;
    Error(int c, std::string m) : code(c), msg(std::move(m)) {}
};

// Immutable structure of a problem (built once at create).
struct Structure {
    int32_t n_c = 0, n_l = 0;
    int64_t n_o = 0;
    // observations in point order
    int32_t* obs_cam = nullptr;   // n_o
    int32_t* obs_pt = nullptr;    // n_o
    int32_t* perm = nullptr;      // n_o: point-order slot -> caller index
    double* obs_xy = nullptr;     // n_o x 2
    float2* obs_xyd = nullptr;    // n_o x 2 (mixed precision): the measurements in double-float
    int64_t* pt_ptr = nullptr;    // n_l + 1
    int32_t* lm_order = nullptr;  // n_l: landmarks by decreasing track length (ties by index); the
                                  // per-landmark kernels take them in this order so that the lanes of a
                                  // warp loop over equally many observations
    int64_t* cam_ptr = nullptr;   // n_c + 1
    int32_t* cam_obs = nullptr;   // n_o: point-order slots grouped by camera
    // S pattern (full)
    int64_t nnzb = 0;
    int64_t* row_ptr = nullptr;   // n_c + 1
    int32_t* col = nullptr;       // nnzb
    int32_t* diag_pos = nullptr;  // n_c: block index of S_jj
    int64_t n_tiles = 0;
    int64_t* tile_ptr = nullptr;  // n_c + 1: first tile of each block-row
    // upper blocks (j <= k) with the observation pairs that feed them
    int64_t n_up = 0;
    int64_t n_pairs = 0;
    int64_t* up_dst = nullptr;    // n_up: element offset of block (j, k) in the tiled S (s_at(.., 0))
    int64_t* up_mdst = nullptr;   // n_up: element offset of its mirror (k, j)
    int64_t* up_pair_ptr = nullptr;  // n_up + 1
    int2* pairs = nullptr;        // n_pairs: (o_j, o_k) point-order slots of one landmark (mixed precision:
                                  // their camera-order positions, where the float32 G rows are kept)
    int2* up_cams = nullptr;      // n_up (mixed precision): the cameras (j, k) of each upper block
    int32_t* up_order = nullptr;  // n_up (mixed precision): the upper blocks by decreasing pair-count class
    int32_t* cpos = nullptr;      // n_o (mixed precision): camera-order position of each point-order slot
    int32_t* cam_lm = nullptr;    // n_o (mixed precision): landmark of each camera-order position
    // upper triangle of S (mixed precision's one-column products): row j holds S_jj, then S_jk, k > j,
    // tiled like the full pattern; qptr/cslot number, per camera k, the stored blocks (j, k), j < k
    int64_t nnzb_u = 0, n_tiles_u = 0;
    int64_t* row_ptr_u = nullptr;    // n_c + 1
    int32_t* col_u = nullptr;        // nnzb_u
    int64_t* tile_ptr_u = nullptr;   // n_c + 1
    int64_t* up_udst = nullptr;      // n_up: element offset of block (j, k) in the tiled upper S
    int64_t* qptr = nullptr;         // n_c + 1
    int32_t* cslot = nullptr;        // n_tiles_u x 32: for the block at tiled index 32 tile_ptr_u[j] + q
                                     // (q > 0), its slot among the blocks (j', k), j' < k, ordered by
                                     // (k, j'): column k owns slots qptr[k] .. qptr[k + 1] - 1; -1 elsewhere
    // batch: problem b owns cameras [h_cam_off[b], h_cam_off[b + 1]); one problem: {0, n_c}
    std::vector<int32_t> h_cam_off;
    // host copies of the pattern (work lists of the block-sparse products are built from them)
    std::vector<int64_t> h_row_ptr;
    std::vector<int32_t> h_col;
    std::vector<int64_t> h_tile_ptr;
    std::vector<int64_t> h_row_ptr_u;
    std::vector<int32_t> h_col_u;
    std::vector<int64_t> h_tile_ptr_u;
};

// The linearised system at the current parameters (rebuilt by ba_build_normal).
struct System {
    double* cams = nullptr;   // n_c x 9 current parameters
    double* aux = nullptr;    // n_c x 24: R, R J_r, t, f, k1, k2 per camera (linearisation)
    double* pts = nullptr;    // n_l x 3
    double* r = nullptr;      // n_o x 2
    double* Jc = nullptr;     // n_o x 18
    double* Jl = nullptr;     // n_o x 6
    double* G = nullptr;      // n_o x 27 (float64 precision only)
    double* V = nullptr;      // n_l x 9
    double* L = nullptr;      // n_l x 6 (reciprocal diagonal, see above)
    double* bl = nullptr;     // n_l x 3
    double* e = nullptr;      // n_l x 3
    double* U = nullptr;      // n_c x 81 (mixed precision: formed only when ba_get_normal asks)
    double* bp = nullptr;     // n_c x 9
    double* bt = nullptr;     // n_c x 9
    double* S = nullptr;      // n_tiles x 2592 (tiled layout above); float64 precision only
    double* Sd = nullptr;     // n_c x 81: the diagonal blocks S_jj = U_j - sum_o G_o G_o^T
    double* Dinv = nullptr;   // n_c x 81
    // mixed precision: the inner solves run on the Jacobi-scaled system
    //   S^ = Lam S Lam, Lam = diag(S)^{-1/2},
    // which removes the parameter-scale ill-conditioning of the 9x9 blocks before float32 rounding
    float* S32 = nullptr;     // float(S^), tiled layout
    float* S32u = nullptr;    // its upper triangle (diagonal blocks included), tiled upper pattern
    double* lam = nullptr;    // 9 n_c: Lam
    double* Dhat = nullptr;   // n_c x 81: inverses of the diagonal blocks of S^
    float* lam32 = nullptr;   // 9 n_c: float(Lam)
    float* G32 = nullptr;     // n_o x 36: G_o = J_p^T A_o in float32 (from the float32 Jacobians), rows
                              // 3P..3P+2 at offset 12 P (three 16-byte aligned parts)
    float* aux32 = nullptr;   // n_c x 24: the camera's aux block in float32
    float* PY32 = nullptr;    // n_o x 6: P = R X + t and Y = R X in float32 (formed in float64)
    float* L32 = nullptr;     // n_l x 6: L (packed as above) in float32
    double* yl = nullptr;     // n_l x 3: V_l^{-1} b_l
    double* dadd = nullptr;   // n_c x 9: the damping lambda D_p^T D_p added to the diagonal of U_j
    double* uv = nullptr;     // n_o x 2: per-observation terms of the float64 true residual
    // mixed precision keeps r, Jc, Jl, L, bl, yl and uv above as double-float (float2 (hi, lo) in the
    // same 8 bytes per value, df64.cuh), and its own double-float inputs:
    float2* auxd = nullptr;   // n_c x 24: the aux block
    float2* ptsd = nullptr;   // n_l x 3: the points
    float2* xd = nullptr;     // n_c x 9: x of the true residual (or dx_p of the back-substitution)
    int* status = nullptr;    // device error word of the build
    double lambda = 0.0;
    bool built = false;
};

// ---- launch wrappers (k_build.cu) -----------------------------------------------------
void launch_project(int64_t n_o, const double* cams, const double* pts, const int32_t* oc,
                    const int32_t* op, double* out, cudaStream_t st);
void launch_cam_prep(const Structure& s, System& y, cudaStream_t st);   // aux from cams (before linearize)
void launch_linearize(const Structure& s, System& y, cudaStream_t st);
void launch_landmarks(const Structure& s, System& y, int damping, double lambda, cudaStream_t st);
void launch_obs_G(const Structure& s, System& y, cudaStream_t st);
void launch_cameras(const Structure& s, System& y, int damping, double lambda, cudaStream_t st);
void launch_schur_diag(const Structure& s, System& y, cudaStream_t st);
// U_lambda and b_p only (mixed precision forms them on request)
void launch_normal_request(const Structure& s, System& y, int damping, double lambda, double* r64, double* Jc64,
                           double* Jl64, double* V64, double* L64, double* bl64, double* e64, cudaStream_t st);
void launch_df_to_double(double* buf, int64_t n, cudaStream_t st);
// mixed precision: b~ and lambda D_p in float64, then the float32 diagonal blocks into Sd
void launch_cam_rhs(const Structure& s, System& y, int damping, double lambda, cudaStream_t st);
void launch_schur_diag32(const Structure& s, System& y, cudaStream_t st);
void launch_schur(const Structure& s, System& y, cudaStream_t st);
void launch_schur_mixed(const Structure& s, System& y, cudaStream_t st);
// out = -b~ - S x with the implicit float64 operator (mixed precision, no explicit S)
// S x = sum_o J_p^T (J_p x - J_l V^-1 sum J_l^T J_p x) + lambda D_p x;
// partial[2 j], partial[2 j + 1] receive camera j's sums of out^2 and b~^2 (2 n_c values)
int launch_implicit_residual(const Structure& s, const System& y, const double* x, double* out, double* partial,
                              cudaStream_t st);
void launch_block_jacobi(const Structure& s, System& y, cudaStream_t st);
void launch_block_jacobi_plain(const Structure& s, System& y, cudaStream_t st);
void launch_to_float(const double* in, float* out, int64_t n, cudaStream_t st);
void launch_back_substitute(const Structure& s, const System& y, const double* dxp, double* dxl,
                            cudaStream_t st);
void launch_cost(const Structure& s, const double* cams, const double* pts, double* partial,
                 int nparts, cudaStream_t st);
void launch_add_params(const double* a, const double* da, double* out, int64_t n, cudaStream_t st);
void launch_unpermute(const double* in, const int32_t* perm, double* out, int64_t n_o, int width,
                      cudaStream_t st);
// row-major 9x9 blocks of S (float64 precision: S itself; mixed: Lam^-1 S^ Lam^-1 off the
// diagonal and the float64 diagonal blocks)
void launch_unslab(const Structure& s, const System& y, double* out, cudaStream_t st);

// ---- solver (k_solve.cu) -------------------------------------------------------------------
struct SolveArgs {
    int mcg = 0;            // 0: Algorithm 1, 1: Algorithm 2
    double tol = 1e-6;
    int max_iters = 1000;
    int n_dirs = 1;
    double tau = 0.0;
    int chunk = 8;
    int precision = BA_PRECISION_FP64;
    double inner_tol = 1e-3;
    int max_refine = 12;
    int64_t max_history = 0;
    int item_blocks = 0;    // blocks per work item of the block-sparse products (0: 512)
    int wait_polls = kDefaultWaitPolls;   // tile-copy waits: polls before giving up (0: give up at once)
    int host_loop = 0;      // 1: the loops run from the host (plain graphs), for profilers
    int spmv_cfg = 0;       // shape of the tile-streaming one-column products (0, 1, 2)
};

struct ProbOut {
    int status = BA_OK;
    int iters = 0;
    int local_steps = 0;
    int pinv_steps = 0;
    int n_eff = 1;
    int refinements = 0;
    int64_t history_cols = 0;
    double rel_residual = 0.0;
    double true_rel_residual = 0.0;
};

struct SolveOut {
    int status = BA_OK;
    int iters = 0;
    int local_steps = 0;
    int pinv_steps = 0;
    int n_eff = 1;
    int refinements = 0;
    int64_t history_cols = 0;
    double rel_residual = 0.0;
    double true_rel_residual = 0.0;
    double ms = 0.0;
    int64_t launches = 0;   // kernel executions issued by the solve
    int host_waits = 0;     // host waits on the device during the solve
    std::vector<ProbOut> probs;   // per problem of the batch (the fields above summarise them)
};

struct Solver;   // workspace, defined in k_solve.cu
Solver* solver_create();
void solver_destroy(Solver* w);
// Solve S x = -b~ into x (device, 9 n_c) for every problem of the batch; the history of recursive
// residuals of each problem is kept in the workspace.
void solver_run(Solver* w, const Structure& s, const System& y, const SolveArgs& a, double* x,
                SolveOut& out, cudaStream_t st);
int solver_history(const Solver* w, int problem, const double** hist);
// Mean ms of one launch of the PCG product q = S p over all problems (float64 or float32 system),
// L2 flushed between launches; item_blocks as in SolveArgs.
double solver_time_spmv(Solver* w, const Structure& s, const System& y, bool fp32, int reps, int item_blocks,
                        int spmv_cfg, cudaStream_t st);
// Shape (0..2) and blocks per work item (32 .. 1024) that make the PCG product fastest; *best_ms its time.
void solver_autotune(Solver* w, const Structure& s, const System& y, bool fp32, int reps, int* best_cfg,
                     int* best_cb, double* best_ms, cudaStream_t st);
void flush_l2(cudaStream_t st);

// ---- learned pose grouping (k_learn.cu) -------------------------------------------------------
struct Gnn;
int64_t gnn_param_count();
Gnn* gnn_create();
void gnn_destroy(Gnn* g);
void gnn_set_params(Gnn* g, const float* params, cudaStream_t st);   // resets the Adam state
void gnn_get_params(const Gnn* g, float* params, cudaStream_t st);
int64_t gnn_launches(const Gnn* g);
// features (n_c x 8) and coupling weights (nnzb, CSR order) of the built system
void gnn_graph_out(Gnn* g, const Structure& s, const System& y, float* X, float* c, cudaStream_t st);
// loss of the built system; scores (n_c) and the gradient copied out when non-null
double gnn_loss(Gnn* g, const Structure& s, const System& y, bool with_grad, float* scores, float* grad,
                cudaStream_t st);
// loss, gradient and one Adam step (returns the loss before the step)
double gnn_train_step(Gnn* g, const Structure& s, const System& y, double lr, cudaStream_t st);
// camera order by score (ties by index); returns the loss of the scores
double gnn_order(Gnn* g, const Structure& s, const System& y, bool bf16, int32_t* order, cudaStream_t st);

int num_sms();
// error text of handle-less calls on this thread (read back by ba_last_error(NULL))
void set_thread_error(const std::string& msg);

}  // namespace ba

// Linearisation and reduced-camera-system build (Section 3.1, Eqs. 2-14).
//
//   k_linearize     one thread per observation: r, J_p (2x9), J_l (2x3)
//   k_landmarks     one thread per landmark: V_lambda, b_l, Cholesky V = L L^T, e = L^{-1} b_l
//                   (L packed with the reciprocals of its diagonal)
//   k_obs_G         one thread per observation: G_o = (J_p^T J_l) L^{-T}
//   k_cameras       one CTA per camera: U_lambda, b_p, b~ = b_p - sum G_o e_l
//   k_schur_diag    one CTA per camera: S_jj = U_j - sum_o G_o G_o^T (float64)
//   k_schur_off_*   S_jk = - sum G_oj G_ok^T over the observation pairs of shared landmarks, written
//                   to (j, k) and transposed to (k, j); float64: a warp per upper block, three
//                   entries per lane (_rows); float32: three blocks per warp, a 3x3 sub-block per
//                   lane (_sub)
//   k_block_jacobi  one thread per camera: D_j^{-1} = (S_jj)^{-1} through Cholesky
// Mixed precision builds no float64 U, G or S_jj.  r, J_p, J_l (for b~ and the true residual
// S x = sum_o J_p^T (J_p x - J_l V^-1 sum J_l^T J_p x) + lambda D_p x) are formed and used in
// double-float arithmetic on the float32 pipe (df64.cuh; the *_df kernels), and the float32 system
// comes from float32 Jacobians formed from P = R X + t and R X, which k_linearize_df keeps in
// float32 (camera order):
//   k_landmarks_df  one thread per landmark: V_lambda, b_l, L, y_l = V^-1 b_l
//   k_cam_rhs_df    one CTA per camera: b~ = sum_o J_p^T (r - J_l V^-1 b_l), lambda D_p
//   k_schur_diag32  one CTA per camera (float32): S_jj = sum_o J_p^T (I - A A^T) J_p + lambda D_p,
//                   A = J_l L^{-T} (each term is positive semi-definite: no cancellation)
//                   (the same pass writes G_o = J_p^T A in float32 for the off-diagonal blocks,
//                   which are scaled by Lam_j, Lam_k after their sums)
// S is written in the tiled layout of ba_internal.cuh (s_at).
// Every kernel uses grid-stride loops and 64-bit indices.
#include <cuda_runtime.h>

#include <cstdint>

#include "ba_internal.cuh"
#include "df64.cuh"

namespace ba {

namespace {

// a float32 G row: the 9x3 values in three parts of 9 (rows 3P..3P+2), each starting on a 16-byte boundary
constexpr int kG32Part = 12;
constexpr int kG32Row = 3 * kG32Part;

inline int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    int cap = num_sms() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return static_cast<int>(g);
}

__device__ __forceinline__ int64_t gtid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

// Rodrigues coefficients A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3,
// by their Taylor series below th = 1e-4 where the closed forms cancel.
__device__ __forceinline__ void rot_coeffs(double th2, double& A, double& B, double& C) {
    if (th2 < 1e-8) {
        A = 1.0 - th2 / 6.0 * (1.0 - th2 / 20.0);
        B = 0.5 - th2 / 24.0 * (1.0 - th2 / 30.0);
        C = 1.0 / 6.0 - th2 / 120.0 * (1.0 - th2 / 42.0);
    } else {
        double th = sqrt(th2);
        double s, c;
        sincos(th, &s, &c);
        A = s / th;
        B = (1.0 - c) / th2;
        C = (th - s) / (th2 * th);
    }
}

// R = I + A [w]x + B [w]x^2 with [w]x^2 = w w^T - th^2 I, row-major.
__device__ __forceinline__ void rot_matrix(const double* w, double A, double B, double th2, double* R) {
    R[0] = 1.0 + B * (w[0] * w[0] - th2);
    R[1] = -A * w[2] + B * w[0] * w[1];
    R[2] = A * w[1] + B * w[0] * w[2];
    R[3] = A * w[2] + B * w[0] * w[1];
    R[4] = 1.0 + B * (w[1] * w[1] - th2);
    R[5] = -A * w[0] + B * w[1] * w[2];
    R[6] = -A * w[1] + B * w[0] * w[2];
    R[7] = A * w[0] + B * w[1] * w[2];
    R[8] = 1.0 + B * (w[2] * w[2] - th2);
}

__device__ __forceinline__ void bal_project(const double* c, const double* X, double* out) {
    double w[3] = {c[0], c[1], c[2]};
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double A, B, C, R[9];
    rot_coeffs(th2, A, B, C);
    rot_matrix(w, A, B, th2, R);
    double P0 = R[0] * X[0] + R[1] * X[1] + R[2] * X[2] + c[3];
    double P1 = R[3] * X[0] + R[4] * X[1] + R[5] * X[2] + c[4];
    double P2 = R[6] * X[0] + R[7] * X[1] + R[8] * X[2] + c[5];
    double p0 = -P0 / P2, p1 = -P1 / P2;
    double n2 = p0 * p0 + p1 * p1;
    double rho = 1.0 + c[7] * n2 + c[8] * n2 * n2;
    out[0] = c[6] * rho * p0;
    out[1] = c[6] * rho * p1;
}

// Per-camera part of the linearisation, shared by all observations of the camera:
// aux = (R[9], RJ[9], t[3], f, k1, k2), RJ = R J_r(omega) with J_r = I - B [w]x + C [w]x^2 the
// right Jacobian of the rotation exponential, so that d(R X)/d omega = -R [X]x J_r = -[R X]x RJ
// (R [X]x = [R X]x R for a rotation).  aux32 and auxd (may be null) receive the same values in
// float32 and in double-float; with ptsd, the same launch also splits the n_pv point coordinates
// into double-float (mixed precision, whose per-observation kernels take no float64 input).
__global__ void k_cam_prep(int32_t n_c, const double* __restrict__ cams, double* __restrict__ aux,
                           float* __restrict__ aux32, float2* __restrict__ auxd, int64_t n_pv,
                           const double* __restrict__ pts, float2* __restrict__ ptsd) {
    if (ptsd)
        for (int64_t i = gtid(); i < n_pv; i += gstride()) df_st(ptsd + i, df_from(pts[i]));
    for (int64_t j = gtid(); j < n_c; j += gstride()) {
        const double* c = cams + 9 * j;
        double w[3] = {c[0], c[1], c[2]};
        const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        double A, B, C, R[9], Jr[9];
        rot_coeffs(th2, A, B, C);
        rot_matrix(w, A, B, th2, R);
        Jr[0] = 1.0 + C * (w[0] * w[0] - th2);
        Jr[1] = B * w[2] + C * w[0] * w[1];
        Jr[2] = -B * w[1] + C * w[0] * w[2];
        Jr[3] = -B * w[2] + C * w[0] * w[1];
        Jr[4] = 1.0 + C * (w[1] * w[1] - th2);
        Jr[5] = B * w[0] + C * w[1] * w[2];
        Jr[6] = B * w[1] + C * w[0] * w[2];
        Jr[7] = -B * w[0] + C * w[1] * w[2];
        Jr[8] = 1.0 + C * (w[2] * w[2] - th2);
        double o[24];
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = R[k];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                o[9 + 3 * a + b] = R[3 * a] * Jr[b] + R[3 * a + 1] * Jr[3 + b] + R[3 * a + 2] * Jr[6 + b];
#pragma unroll
        for (int k = 0; k < 6; ++k) o[18 + k] = c[3 + k];
#pragma unroll
        for (int k = 0; k < 24; ++k) aux[24 * j + k] = o[k];
        if (aux32) {
#pragma unroll
            for (int k = 0; k < 24; ++k) aux32[24 * j + k] = float(o[k]);
        }
        if (auxd) {
#pragma unroll
            for (int k = 0; k < 24; ++k) df_st(auxd + 24 * j + k, df_from(o[k]));
        }
    }
}

// 1 / p: float64 from a float32 estimate and two Newton steps (each squares the relative error:
// 2^-23 -> 2^-46 -> rounding level), which keeps the long float64 division off this GPU's narrow
// float64 pipe; float32 divides.  Values outside the float32 range divide in float64.
__device__ __forceinline__ double rcp_fast(double p) {
    const double ap = fabs(p);
    if (!(ap > 1e-30 && ap < 1e30)) return 1.0 / p;
    double r = double(__frcp_rn(float(p)));
    r = fma(r, fma(-p, r, 1.0), r);
    return fma(r, fma(-p, r, 1.0), r);
}
__device__ __forceinline__ float rcp_fast(float p) { return __frcp_rn(p); }

// 1 / sqrt(x) for x > 0 in float64 by the same scheme (Newton steps y <- y (3 - x y^2) / 2);
// returns 0 for x <= 0 or NaN, which the caller reports as not positive definite.
__device__ __forceinline__ double rsqrt_fast(double x) {
    if (!(x > 0.0)) return 0.0;
    if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
    double y = double(rsqrtf(float(x)));
    const double hx = 0.5 * x;
    y = y * fma(-hx * y, y, 1.5);
    return y * fma(-hx * y, y, 1.5);
}

// Jacobian blocks of one observation from the camera's aux block, the rotated point Y = R X and the
// point in the camera frame P = Y + t, and the residual when r != nullptr (pi = f rho(|p|^2) p with
// p = -P_xy / P_z: the BAL model).  With D_a = d pi_a / dP, row a of J_p has the rotation part
// -(D_a x Y)^T RJ (D^T [Y]x = (D x Y)^T), the translation part D_a, and the intrinsics; row a of J_l
// is D_a^T R.  (Y and P are both passed: either can be much smaller than t, so neither is formed
// from the other in float32.)
template <typename T>
__device__ __forceinline__ void bal_jacobian_P(const T* ax, const T* Y, const T* P, const T* m, T* r, T* Jc,
                                               T* Jl) {
    const T* R = ax;
    const T* RJ = ax + 9;
    const T iz = rcp_fast(P[2]);
    const T p0 = -P[0] * iz, p1 = -P[1] * iz;
    const T f = ax[21], k1 = ax[22], k2 = ax[23];
    const T n2 = p0 * p0 + p1 * p1;
    const T rho = T(1) + k1 * n2 + k2 * n2 * n2;
    const T drho = T(2) * (k1 + T(2) * k2 * n2);
    const T E00 = f * (rho + drho * p0 * p0), E01 = f * drho * p0 * p1, E11 = f * (rho + drho * p1 * p1);
    T D[6];
    D[0] = -E00 * iz;
    D[1] = -E01 * iz;
    D[2] = -(E00 * p0 + E01 * p1) * iz;
    D[3] = -E01 * iz;
    D[4] = -E11 * iz;
    D[5] = -(E01 * p0 + E11 * p1) * iz;
    if (r) {
        r[0] = f * rho * p0 - m[0];
        r[1] = f * rho * p1 - m[1];
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const T* d = D + 3 * a;
        const T w0 = d[1] * Y[2] - d[2] * Y[1], w1 = d[2] * Y[0] - d[0] * Y[2], w2 = d[0] * Y[1] - d[1] * Y[0];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            Jc[9 * a + b] = -(w0 * RJ[b] + w1 * RJ[3 + b] + w2 * RJ[6 + b]);
            Jc[9 * a + 3 + b] = d[b];
            Jl[3 * a + b] = d[0] * R[b] + d[1] * R[3 + b] + d[2] * R[6 + b];
        }
    }
    Jc[6] = rho * p0;
    Jc[15] = rho * p1;
    Jc[7] = f * n2 * p0;
    Jc[16] = f * n2 * p1;
    Jc[8] = f * n2 * n2 * p0;
    Jc[17] = f * n2 * n2 * p1;
}

// Y = R X and P = Y + t from the camera's aux block.
__device__ __forceinline__ void cam_point(const double* ax, const double* X, double* Y, double* P) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Y[a] = ax[3 * a] * X[0] + ax[3 * a + 1] * X[1] + ax[3 * a + 2] * X[2];
        P[a] = Y[a] + ax[18 + a];
    }
}

__device__ __forceinline__ double damp(double d, int damping, double lambda) {
    if (damping == BA_DAMPING_IDENTITY) return d + lambda;
    double c = fmin(fmax(d, 1e-6), 1e32);
    return d + lambda * c;
}

__global__ void k_project(int64_t n_o, const double* __restrict__ cams, const double* __restrict__ pts,
                          const int32_t* __restrict__ oc, const int32_t* __restrict__ op,
                          double* __restrict__ out) {
    for (int64_t i = gtid(); i < n_o; i += gstride()) {
        double c[9], X[3], pr[2];
        const double* cp = cams + int64_t(oc[i]) * 9;
        const double* xp = pts + int64_t(op[i]) * 3;
#pragma unroll
        for (int k = 0; k < 9; ++k) c[k] = __ldg(cp + k);
#pragma unroll
        for (int k = 0; k < 3; ++k) X[k] = __ldg(xp + k);
        bal_project(c, X, pr);
        out[2 * i] = pr[0];
        out[2 * i + 1] = pr[1];
    }
}

// Float64 residuals and Jacobians per observation; mixed precision (PY32 != null) also keeps P and
// Y = R X in float32 (6 per observation, in camera order), from which the float32 Jacobians are
// formed (forming P = Y + t in float32 would lose digits when |Y|, |t| >> |P|, and Y = P - t when
// |P|, |t| >> |Y|).
__global__ void k_linearize(int64_t n_o, const double* __restrict__ aux, const double* __restrict__ pts,
                            const int32_t* __restrict__ oc, const int32_t* __restrict__ op,
                            const double* __restrict__ xy, double* __restrict__ r, double* __restrict__ Jc,
                            double* __restrict__ Jl, float* __restrict__ PY32, const int32_t* __restrict__ cpos) {
    for (int64_t i = gtid(); i < n_o; i += gstride()) {
        double ax[24], X[3], Y[3], P[3], m[2], rr[2], jc[18], jl[6];
        const double* cp = aux + int64_t(oc[i]) * 24;
        const double* xp = pts + int64_t(op[i]) * 3;
#pragma unroll
        for (int k = 0; k < 24; ++k) ax[k] = __ldg(cp + k);
#pragma unroll
        for (int k = 0; k < 3; ++k) X[k] = __ldg(xp + k);
        m[0] = xy[2 * i];
        m[1] = xy[2 * i + 1];
        cam_point(ax, X, Y, P);
        bal_jacobian_P<double>(ax, Y, P, m, rr, jc, jl);
        r[2 * i] = rr[0];
        r[2 * i + 1] = rr[1];
#pragma unroll
        for (int k = 0; k < 18; ++k) Jc[18 * i + k] = jc[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) Jl[6 * i + k] = jl[k];
        if (PY32) {   // at the observation's camera-order position
            float* py = PY32 + 6 * int64_t(cpos[i]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                py[k] = float(P[k]);
                py[3 + k] = float(Y[k]);
            }
        }
    }
}

// V_lambda = sum J_l^T J_l + damping, b_l = sum J_l^T r, V = L L^T, e = L^{-1} b_l.  L is packed as
// (1 / l00, l10, 1 / l11, l20, l21, 1 / l22): every later use multiplies by the reciprocal diagonal.
// Mixed precision (L32 != null) also writes L in float32 (same packing) and y_l = V^{-1} b_l =
// L^{-T} e in float64 (for b~ in the form sum J_p^T (r - J_l y_l)).
__global__ void k_landmarks(int32_t n_l, const int64_t* __restrict__ pt_ptr, const int32_t* __restrict__ order,
                            const double* __restrict__ r, const double* __restrict__ Jl, int damping, double lambda,
                            double* __restrict__ Vout, double* __restrict__ Lout, double* __restrict__ blout,
                            double* __restrict__ eout, float* __restrict__ L32, double* __restrict__ yout,
                            int* status) {
    for (int64_t t = gtid(); t < n_l; t += gstride()) {
        const int64_t l = order[t];
        double v00 = 0, v01 = 0, v02 = 0, v11 = 0, v12 = 0, v22 = 0, b0 = 0, b1 = 0, b2 = 0;
        for (int64_t o = pt_ptr[l]; o < pt_ptr[l + 1]; ++o) {
            const double* j = Jl + 6 * o;
            double a0 = j[0], a1 = j[1], a2 = j[2], c0 = j[3], c1 = j[4], c2 = j[5];
            double r0 = r[2 * o], r1 = r[2 * o + 1];
            v00 += a0 * a0 + c0 * c0;
            v01 += a0 * a1 + c0 * c1;
            v02 += a0 * a2 + c0 * c2;
            v11 += a1 * a1 + c1 * c1;
            v12 += a1 * a2 + c1 * c2;
            v22 += a2 * a2 + c2 * c2;
            b0 += a0 * r0 + c0 * r1;
            b1 += a1 * r0 + c1 * r1;
            b2 += a2 * r0 + c2 * r1;
        }
        v00 = damp(v00, damping, lambda);
        v11 = damp(v11, damping, lambda);
        v22 = damp(v22, damping, lambda);
        double* V = Vout + 9 * l;
        V[0] = v00; V[1] = v01; V[2] = v02;
        V[3] = v01; V[4] = v11; V[5] = v12;
        V[6] = v02; V[7] = v12; V[8] = v22;
        // Cholesky with reciprocal square roots (a zero marks a pivot that is not positive)
        const double i00 = rsqrt_fast(v00);
        const double l10 = v01 * i00, l20 = v02 * i00;
        const double i11 = rsqrt_fast(v11 - l10 * l10);
        const double l21 = (v12 - l20 * l10) * i11;
        const double i22 = rsqrt_fast(v22 - l20 * l20 - l21 * l21);
        if (!(i00 > 0 && i11 > 0 && i22 > 0)) atomicExch(status, BA_ERR_SINGULAR);
        double* L = Lout + 6 * l;
        L[0] = i00; L[1] = l10; L[2] = i11; L[3] = l20; L[4] = l21; L[5] = i22;
        blout[3 * l] = b0;
        blout[3 * l + 1] = b1;
        blout[3 * l + 2] = b2;
        const double e0 = b0 * i00;
        const double e1 = (b1 - l10 * e0) * i11;
        const double e2 = (b2 - l20 * e0 - l21 * e1) * i22;
        eout[3 * l] = e0;
        eout[3 * l + 1] = e1;
        eout[3 * l + 2] = e2;
        if (L32) {
            const double y2 = e2 * i22;
            const double y1 = (e1 - l21 * y2) * i11;
            const double y0 = (e0 - l10 * y1 - l20 * y2) * i00;
            yout[3 * l] = y0;
            yout[3 * l + 1] = y1;
            yout[3 * l + 2] = y2;
#pragma unroll
            for (int k = 0; k < 6; ++k) L32[6 * l + k] = float(L[k]);
        }
    }
}

// G_o = W_o L^{-T}, W_o = J_p^T J_l (9x3); each row g solves L g^T = w^T.
__global__ void k_obs_G(int64_t n_o, const int32_t* __restrict__ op, const double* __restrict__ Jc,
                        const double* __restrict__ Jl, const double* __restrict__ Lall, double* __restrict__ G) {
    for (int64_t o = gtid(); o < n_o; o += gstride()) {
        const double* L = Lall + 6 * int64_t(op[o]);
        const double i00 = L[0], l10 = L[1], i11 = L[2], l20 = L[3], l21 = L[4], i22 = L[5];
        double jl[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) jl[k] = Jl[6 * o + k];
        const double* jc = Jc + 18 * o;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            double ca = jc[a], cb = jc[9 + a];
            double w0 = ca * jl[0] + cb * jl[3];
            double w1 = ca * jl[1] + cb * jl[4];
            double w2 = ca * jl[2] + cb * jl[5];
            const double g0 = w0 * i00;
            const double g1 = (w1 - l10 * g0) * i11;
            const double g2 = (w2 - l20 * g0 - l21 * g1) * i22;
            G[27 * o + 3 * a] = g0;
            G[27 * o + 3 * a + 1] = g1;
            G[27 * o + 3 * a + 2] = g2;
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

constexpr int kCamThreads = 128;

// U_lambda, b_p and b~ of one camera per CTA.
__global__ void __launch_bounds__(kCamThreads) k_cameras(
    int32_t n_c, const int64_t* __restrict__ cam_ptr, const int32_t* __restrict__ cam_obs,
    const int32_t* __restrict__ op, const double* __restrict__ r, const double* __restrict__ Jc,
    const double* __restrict__ G, const double* __restrict__ e, int damping, double lambda,
    double* __restrict__ Uout, double* __restrict__ bpout, double* __restrict__ btout) {
    __shared__ double red[kCamThreads / 32][64];
    __shared__ double fin[64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = blockIdx.x; j < n_c; j += gridDim.x) {
        double u[45], b[9];
#pragma unroll
        for (int k = 0; k < 45; ++k) u[k] = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) b[k] = 0.0;
        const int64_t beg = cam_ptr[j], end = cam_ptr[j + 1];
        for (int64_t q = beg + threadIdx.x; q < end; q += blockDim.x) {
            const int64_t o = cam_obs[q];
            double c0[9], c1[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                c0[k] = Jc[18 * o + k];
                c1[k] = Jc[18 * o + 9 + k];
            }
            double r0 = r[2 * o], r1 = r[2 * o + 1];
            int t = 0;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
#pragma unroll
                for (int bb = a; bb < 9; ++bb) u[t++] += c0[a] * c0[bb] + c1[a] * c1[bb];
                b[a] += c0[a] * r0 + c1[a] * r1;
            }
        }
        // reduce the 54 sums
#pragma unroll
        for (int k = 0; k < 54; ++k) {
            double v = warp_sum(k < 45 ? u[k] : b[k - 45]);
            if (lane == 0) red[wid][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < 54) {
            double v = 0;
            for (int w = 0; w < kCamThreads / 32; ++w) v += red[w][threadIdx.x];
            fin[threadIdx.x] = v;
        }
        __syncthreads();
        if (threadIdx.x < 81) {
            int a = threadIdx.x / 9, bb = threadIdx.x % 9;
            int lo = a < bb ? a : bb, hi = a < bb ? bb : a;
            int idx = lo * 9 - lo * (lo - 1) / 2 + (hi - lo);
            double v = fin[idx];
            if (a == bb) v = damp(v, damping, lambda);
            Uout[81 * int64_t(j) + threadIdx.x] = v;
        }
        __syncthreads();
        if (!G) {   // U and b_p only (mixed precision builds b~ in k_cam_rhs_df)
            if (threadIdx.x < 9) bpout[9 * int64_t(j) + threadIdx.x] = fin[45 + threadIdx.x];
            __syncthreads();
            continue;
        }
        // b~ = b_p - sum_o G_o e_l
        double t9[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) t9[k] = 0.0;
        for (int64_t q = beg + threadIdx.x; q < end; q += blockDim.x) {
            const int64_t o = cam_obs[q];
            const double* el = e + 3 * int64_t(op[o]);
            double e0 = el[0], e1 = el[1], e2 = el[2];
            const double* g = G + 27 * o;
#pragma unroll
            for (int a = 0; a < 9; ++a) t9[a] += g[3 * a] * e0 + g[3 * a + 1] * e1 + g[3 * a + 2] * e2;
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double v = warp_sum(t9[k]);
            if (lane == 0) red[wid][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < 9) {
            double v = 0;
            for (int w = 0; w < kCamThreads / 32; ++w) v += red[w][threadIdx.x];
            double bpv = fin[45 + threadIdx.x];
            bpout[9 * int64_t(j) + threadIdx.x] = bpv;
            btout[9 * int64_t(j) + threadIdx.x] = bpv - v;
        }
        __syncthreads();
    }
}

// Diagonal blocks S_jj = U_j - sum_{o in camera j} G_o G_o^T in float64, one CTA per camera
// (each camera sees a landmark at most once, so no pair of distinct observations adds here).
__global__ void __launch_bounds__(kCamThreads) k_schur_diag(int32_t n_c, const int64_t* __restrict__ cam_ptr,
                                                           const int32_t* __restrict__ cam_obs,
                                                           const double* __restrict__ G, const double* __restrict__ U,
                                                           double* __restrict__ Sd) {
    __shared__ double red[kCamThreads / 32][48];
    __shared__ double fin[48];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = blockIdx.x; j < n_c; j += gridDim.x) {
        double acc[45];
#pragma unroll
        for (int k = 0; k < 45; ++k) acc[k] = 0.0;
        for (int64_t q = cam_ptr[j] + threadIdx.x; q < cam_ptr[j + 1]; q += blockDim.x) {
            const double* g = G + 27 * int64_t(cam_obs[q]);
            double gv[27];
#pragma unroll
            for (int k = 0; k < 27; ++k) gv[k] = g[k];
            int t = 0;
#pragma unroll
            for (int a = 0; a < 9; ++a)
#pragma unroll
                for (int bb = a; bb < 9; ++bb)
                    acc[t++] += gv[3 * a] * gv[3 * bb] + gv[3 * a + 1] * gv[3 * bb + 1] + gv[3 * a + 2] * gv[3 * bb + 2];
        }
#pragma unroll
        for (int k = 0; k < 45; ++k) {
            double v = warp_sum(acc[k]);
            if (lane == 0) red[wid][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < 45) {
            double v = 0;
            for (int w = 0; w < kCamThreads / 32; ++w) v += red[w][threadIdx.x];
            fin[threadIdx.x] = v;
        }
        __syncthreads();
        if (threadIdx.x < 81) {
            const int a = threadIdx.x / 9, bb = threadIdx.x % 9;
            const int lo = a < bb ? a : bb, hi = a < bb ? bb : a;
            const int idx = lo * 9 - lo * (lo - 1) / 2 + (hi - lo);
            Sd[81 * int64_t(j) + threadIdx.x] = U[81 * int64_t(j) + threadIdx.x] - fin[idx];
        }
        __syncthreads();
    }
}

// Off-diagonal blocks in float64: one warp per upper block (j < k), S_jk = - sum over the
// observation pairs (o_j, o_k) of its landmarks of G_oj G_ok^T, written to (j, k) and transposed to
// (k, j).  Lane entries are e = lane, lane + 32, lane + 64 (< 81), so every lane works on every
// pair (the float64 multiply-adds bound this kernel).  The warp takes the pairs kChunk at a time:
// lanes 0..26 load the two 27-value G blocks of every pair of the chunk (one coalesced load per
// block, all of the chunk's loads in flight together), stage them in shared memory, and every
// lane then accumulates its entries over the chunk's pairs in order (lane p fetches the indices of
// pair p; 16-pair chunks measured no faster).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_schur_off_rows(
    int64_t n_up, const int64_t* __restrict__ up_dst, const int64_t* __restrict__ up_mdst,
    const int64_t* __restrict__ pair_ptr, const int2* __restrict__ pairs, const T* __restrict__ G,
    T* __restrict__ S) {
    constexpr int kChunk = 8;
    __shared__ T sg[kThreads / 32][kChunk][2][28];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nw = gstride() >> 5;
    const int e0 = lane, e1 = lane + 32, e2 = lane + 64;
    const int a0 = e0 / 9, b0 = e0 % 9, a1 = e1 / 9, b1 = e1 % 9;
    const bool has2 = e2 < 81;
    const int a2 = has2 ? e2 / 9 : 0, b2 = has2 ? e2 % 9 : 0;
    for (int64_t u = gtid() >> 5; u < n_up; u += nw) {
        T s0 = T(0), s1 = T(0), s2 = T(0);
        const int64_t pb = pair_ptr[u], pe = pair_ptr[u + 1];
        for (int64_t q = pb; q < pe; q += kChunk) {
            const int np = int(pe - q < kChunk ? pe - q : kChunk);
            int2 pr = make_int2(0, 0);
            if (lane < np) pr = pairs[q + lane];
            T ga[kChunk], gb[kChunk];
#pragma unroll
            for (int p = 0; p < kChunk; ++p) {
                const int ox = __shfl_sync(0xffffffffu, pr.x, p);
                const int oy = __shfl_sync(0xffffffffu, pr.y, p);
                ga[p] = T(0);
                gb[p] = T(0);
                if (p < np && lane < 27) {
                    ga[p] = __ldg(G + 27 * int64_t(ox) + lane);
                    gb[p] = __ldg(G + 27 * int64_t(oy) + lane);
                }
            }
            __syncwarp();
#pragma unroll
            for (int p = 0; p < kChunk; ++p) {
                if (lane < 27) {
                    sg[wid][p][0][lane] = ga[p];
                    sg[wid][p][1][lane] = gb[p];
                }
            }
            __syncwarp();
            for (int p = 0; p < np; ++p) {
                const T* x = sg[wid][p][0];
                const T* y = sg[wid][p][1];
                s0 += x[3 * a0] * y[3 * b0] + x[3 * a0 + 1] * y[3 * b0 + 1] + x[3 * a0 + 2] * y[3 * b0 + 2];
                s1 += x[3 * a1] * y[3 * b1] + x[3 * a1 + 1] * y[3 * b1 + 1] + x[3 * a1 + 2] * y[3 * b1 + 2];
                s2 += x[3 * a2] * y[3 * b2] + x[3 * a2 + 1] * y[3 * b2 + 1] + x[3 * a2 + 2] * y[3 * b2 + 2];
            }
        }
        T* Sj = S + up_dst[u];
        T* Sk = S + up_mdst[u];
        Sj[e0] = -s0;
        Sj[e1] = -s1;
        if (has2) Sj[e2] = -s2;
        Sk[b0 * 9 + a0] = -s0;
        Sk[b1 * 9 + a1] = -s1;
        if (has2) Sk[b2 * 9 + a2] = -s2;
    }
}

// 16-byte asynchronous copy global -> shared (cp.async, completion awaited by cp.async.wait_group); both
// addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}

// Nine consecutive values from a 16-byte aligned shared-memory address.
__device__ __forceinline__ void lds9(const float* p, float* v) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 4);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
    v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    v[8] = p[8];
}

// Off-diagonal blocks in float32: S_jk = - Lam_j (sum over the observation pairs (o_j, o_k) of the
// landmarks j and k share of G_oj G_ok^T) Lam_k, written to (j, k), transposed to (k, j), and to the
// upper-triangle copy.  Most blocks have few pairs (a dense problem of 1000 cameras: 7.5 on average,
// 87 % of the blocks 5 or fewer), so a warp takes three blocks at once, one per group of 9 lanes
// (lanes 27..31 idle): lane 9 g + 3 A + B sums the 3x3 sub-block at rows 3A.., columns 3B.. of its
// group's block over all its pairs, from rows 3A..3A+2 of G_oj and 3B..3B+2 of G_ok (nine
// consecutive values each: vector shared loads for 27 fused multiply-adds).  Blocks go in
// decreasing pair-count class (up_order: floor(log2(pairs)), (j, k) order within a class), so the
// three blocks of a warp have about as many pairs, the largest start first, and the blocks in flight
// share their G rows in L2.  A group copies the G rows of its pairs into shared memory kOffChunk pairs at
// a time with 16-byte asynchronous copies, double-buffered (lane 3A + B copies piece 3A + B of
// both rows of every pair; a row is three 9-value parts on 16-byte boundaries).  The three blocks
// then meet in shared memory, and the warp writes their 3 x 81 values per destination together.
constexpr int kOffChunk = 3;

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <typename T>
__global__ void __launch_bounds__(kThreads, 4) k_schur_off_sub(
    int64_t n_up, const int32_t* __restrict__ up_order, const int64_t* __restrict__ up_dst,
    const int64_t* __restrict__ up_mdst, const int64_t* __restrict__ up_udst, const int64_t* __restrict__ pair_ptr,
    const int2* __restrict__ pairs, const int2* __restrict__ up_cams, const T* __restrict__ lam,
    const T* __restrict__ G, T* __restrict__ S, T* __restrict__ Su) {
    static_assert(sizeof(T) == 4, "float32 build (float64 uses k_schur_off_rows)");
    constexpr int kBuf = kOffChunk * 2 * kG32Row;      // one buffer of a group: the chunk's row pairs
    __shared__ __align__(16) T sg[kThreads / 32][3][2 * kBuf];
    __shared__ int64_t sdst[kThreads / 32][3][3];   // per group: offsets of (j, k), (k, j), upper (j, k)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane / 9, sub = lane - 9 * g;        // g == 3: lanes 27..31
    const int A = sub / 3, B = sub - 3 * (sub / 3);
    const int coff = A * kG32Part + B * 4;             // piece `sub` of a 36-float row
    T* const area = &sg[wid][g < 3 ? g : 0][0];
    const int64_t n_tri = (n_up + 2) / 3;
    const int64_t nw = gstride() >> 5;
    for (int64_t w = gtid() >> 5; w < n_tri; w += nw) {
        const int64_t slot = 3 * w + g;
        const bool has = g < 3 && slot < n_up;
        const int64_t u = has ? up_order[slot] : 0;
        const int64_t pb = has ? pair_ptr[u] : 0, pe = has ? pair_ptr[u + 1] : 0;
        const int nch = int((pe - pb + kOffChunk - 1) / kOffChunk);
        int nmax = nch;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        // The observation pairs of a chunk are loaded one chunk ahead, pair i by lane 9 g + i of the
        // group, so that the copies of a chunk start without waiting on its pair indices.
        const int src = 9 * (g < 3 ? g : 0);
        auto load_pairs = [&](int c) {
            const int64_t q = pb + int64_t(c) * kOffChunk + sub;
            return (c < nch && sub < kOffChunk && q < pe) ? pairs[q] : make_int2(0, 0);
        };
        int2 pnext = load_pairs(0);
        // chunk c of this group's pairs into buffer c & 1 (nothing past the group's last chunk)
        auto issue = [&](int c) {
            int2 pr[kOffChunk];
#pragma unroll
            for (int i = 0; i < kOffChunk; ++i) {
                pr[i].x = __shfl_sync(0xffffffffu, pnext.x, src + i);
                pr[i].y = __shfl_sync(0xffffffffu, pnext.y, src + i);
            }
            pnext = load_pairs(c + 1);
            if (c < nch) {
                T* buf = area + (c & 1) * kBuf;
                const int64_t q0 = pb + int64_t(c) * kOffChunk;
                const int n = pe - q0 < kOffChunk ? int(pe - q0) : kOffChunk;
#pragma unroll
                for (int i = 0; i < kOffChunk; ++i) {
                    if (i < n) {
                        cp_async16(buf + (2 * i) * kG32Row + coff, G + int64_t(kG32Row) * pr[i].x + coff);
                        cp_async16(buf + (2 * i + 1) * kG32Row + coff, G + int64_t(kG32Row) * pr[i].y + coff);
                    }
                }
            }
            cp_async_commit();
        };
        T acc[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) acc[i] = T(0);
        issue(0);
        for (int c = 0; c < nmax; ++c) {
            issue(c + 1);
            cp_async_wait_prev();   // this lane's copies of chunk c have landed
            __syncwarp();           // and every lane's
            if (c < nch) {
                const T* buf = area + (c & 1) * kBuf;
                const int64_t q0 = pb + int64_t(c) * kOffChunk;
                const int n = pe - q0 < kOffChunk ? int(pe - q0) : kOffChunk;
                for (int i = 0; i < n; ++i) {
                    T x[9], y[9];
                    lds9(buf + (2 * i) * kG32Row + A * kG32Part, x);
                    lds9(buf + (2 * i + 1) * kG32Row + B * kG32Part, y);
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc)
                            acc[3 * r + cc] = fmaf(x[3 * r + 2], y[3 * cc + 2],
                                                   fmaf(x[3 * r + 1], y[3 * cc + 1], fmaf(x[3 * r], y[3 * cc], acc[3 * r + cc])));
                }
            }
            __syncwarp();           // buffer c & 1 is refilled by issue(c + 2)
        }
        // the group's block, scaled (rows by Lam_j, columns by Lam_k) and negated, into its area
        if (has) {
            const int2 jk = up_cams[u];
            const T* lj = lam + 9 * int64_t(jk.x);
            const T* lk = lam + 9 * int64_t(jk.y);
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    area[(3 * A + r) * 9 + 3 * B + cc] = -(acc[3 * r + cc] * lj[3 * A + r] * lk[3 * B + cc]);
            if (sub == 0) {
                sdst[wid][g][0] = up_dst[u];
                sdst[wid][g][1] = up_mdst[u];
                sdst[wid][g][2] = up_udst[u];
            }
        }
        __syncwarp();
        // the warp writes the blocks one after the other, 81 consecutive values per destination
        for (int gg = 0; gg < 3 && 3 * w + gg < n_up; ++gg) {
            const int64_t ej = sdst[wid][gg][0], ek = sdst[wid][gg][1], eu = sdst[wid][gg][2];
            const T* blk = &sg[wid][gg][0];
#pragma unroll
            for (int it = 0; it < 3; ++it) {
                const int ee = lane + 32 * it;
                if (ee < 81) {
                    const T v = blk[ee];
                    S[ej + ee] = v;
                    Su[eu + ee] = v;
                    const int b = ee / 9, a = ee - 9 * (ee / 9);   // entry 9 b + a of (k, j) is (a, b) of (j, k)
                    S[ek + ee] = blk[9 * a + b];
                }
            }
        }
        __syncwarp();
    }
}

// S_jj into the tiled S: float64 copy, or (lam != nullptr) float(Lam S_jj Lam) for the scaled system,
// then also into the upper-triangle copy Su (may be null), where it opens block-row j.
template <typename T>
__global__ void k_put_diag(int32_t n_c, const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr,
                           const int32_t* __restrict__ diag_pos, const double* __restrict__ Sd,
                           const double* __restrict__ lam, T* __restrict__ S, const int64_t* __restrict__ tile_ptr_u,
                           T* __restrict__ Su) {
    for (int64_t i = gtid(); i < int64_t(n_c) * 81; i += gstride()) {
        const int64_t j = i / 81;
        const int e = int(i - j * 81);
        double v = Sd[i];
        if (lam) v *= lam[9 * j + e / 9] * lam[9 * j + e % 9];
        S[s_at(tile_ptr, j, diag_pos[j] - row_ptr[j], e)] = T(v);
        if (Su) Su[s_at(tile_ptr_u, j, 0, e)] = T(v);
    }
}

// The damping added to the diagonal of U (Eq. 5): lambda D^T D with D^T D = diag(J^T J) clamped
// to [1e-6, 1e32] (Marquardt) or the identity.
__device__ __forceinline__ double damp_add(double d, int damping, double lambda) {
    return damping == BA_DAMPING_IDENTITY ? lambda : lambda * fmin(fmax(d, 1e-6), 1e32);
}

// Row a of A_o = J_l L^{-T} (2x3) from L packed with its reciprocal diagonal (float32).
__device__ __forceinline__ void rows_A(const float* jl, const float* Lp, float (&A)[2][3]) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        A[a][0] = jl[3 * a] * Lp[0];
        A[a][1] = (jl[3 * a + 1] - Lp[1] * A[a][0]) * Lp[2];
        A[a][2] = (jl[3 * a + 2] - Lp[3] * A[a][0] - Lp[4] * A[a][1]) * Lp[5];
    }
}

constexpr int kDiagThreads = 256;
// the 45 sums of S_jj's upper triangle across the CTA: 5 threads per sum, each adding a 52-thread
// slice of the staged partials (the last slice 48)
constexpr int kDiagSlices = 5, kDiagSlice = 52;

// Mixed precision, one CTA per camera: S_jj = sum_{o in j} J_p^T (I - A A^T) J_p + lambda D_p (Eq. 13 on
// the diagonal: U_j - sum_o G_o G_o^T with G_o = J_p^T A_o), from float32 Jacobians formed in float32
// from the camera and the float32 point in the camera frame.  I - A A^T = I - J_l V^-1 J_l^T is
// positive semi-definite, so the terms add without cancellation: an entry's rounding errors are at
// most a few float32 units of sqrt(S_aa S_bb) (each term obeys |t_ab| <= sqrt(t_aa t_bb)), the
// accuracy of the float32 system.  Each thread sums its observations, the threads' partials meet in
// shared memory and are added in a fixed order (slices, then the slices' sums), and the float64
// damping is added last.  Sd receives float64.  The same pass writes G_o = J_p^T A_o (9x3, unscaled) of every
// observation to G32 for the off-diagonal blocks.  PY32, cam_lm and G32 are in camera order, so the
// CTA of camera j reads and writes rows cam_ptr[j] .. cam_ptr[j + 1] contiguously: a warp takes 32
// consecutive observations, stages their G rows in shared memory and writes the 32 rows (4.6 KB) as
// 16-byte stores (a thread writing its own row made 27 scattered 4-byte stores per observation).
__global__ void __launch_bounds__(kDiagThreads) k_schur_diag32(
    int32_t n_c, const int64_t* __restrict__ cam_ptr, const int32_t* __restrict__ cam_lm,
    const float* __restrict__ aux32, const float* __restrict__ PY32, const float* __restrict__ L32,
    const double* __restrict__ dadd, double* __restrict__ Sd, float* __restrict__ G32) {
    // the partials at the end of a camera; during the observation loop the same memory stages each
    // warp's 32 G rows (8 x 32 x 36 floats fit in 45 x 257)
    __shared__ __align__(16) float stage[45][kDiagThreads + 1];
    __shared__ float slice[45][kDiagSlices];
    static_assert((kDiagThreads / 32) * 32 * kG32Row <= 45 * (kDiagThreads + 1), "G staging fits");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float* const grows = &stage[0][0] + wid * (32 * kG32Row);
    for (int j = blockIdx.x; j < n_c; j += gridDim.x) {
        float ax[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) ax[k] = __ldg(aux32 + 24 * int64_t(j) + k);
        float acc[45];
#pragma unroll
        for (int k = 0; k < 45; ++k) acc[k] = 0.f;
        const int64_t q0 = cam_ptr[j], q1 = cam_ptr[j + 1];
        for (int64_t qw = q0 + 32 * wid; qw < q1; qw += blockDim.x) {   // warp-uniform
            const int64_t q = qw + lane;
            const bool act = q < q1;
            float* g = grows + lane * kG32Row;
            if (act) {
                const int64_t l = cam_lm[q];
                float PY[6], Lp[6], jc[18], jl[6], A[2][3];
#pragma unroll
                for (int k = 0; k < 6; ++k) PY[k] = __ldg(PY32 + 6 * q + k);
#pragma unroll
                for (int k = 0; k < 6; ++k) Lp[k] = __ldg(L32 + 6 * l + k);
                bal_jacobian_P<float>(ax, PY + 3, PY, nullptr, nullptr, jc, jl);
                rows_A(jl, Lp, A);
                const float m00 = 1.f - (A[0][0] * A[0][0] + A[0][1] * A[0][1] + A[0][2] * A[0][2]);
                const float m01 = -(A[0][0] * A[1][0] + A[0][1] * A[1][1] + A[0][2] * A[1][2]);
                const float m11 = 1.f - (A[1][0] * A[1][0] + A[1][1] * A[1][1] + A[1][2] * A[1][2]);
                // G_o row-major 9x3 as three parts of rows 3P..3P+2 at stride kG32Part (16-byte aligned)
#pragma unroll
                for (int a = 0; a < 9; ++a)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        g[(a / 3) * kG32Part + (a % 3) * 3 + c] = jc[a] * A[0][c] + jc[9 + a] * A[1][c];
                float B0[9], B1[9];
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    B0[a] = m00 * jc[a] + m01 * jc[9 + a];
                    B1[a] = m01 * jc[a] + m11 * jc[9 + a];
                }
                int t = 0;
#pragma unroll
                for (int a = 0; a < 9; ++a)
#pragma unroll
                    for (int b = a; b < 9; ++b, ++t) acc[t] = fmaf(jc[9 + a], B1[b], fmaf(jc[a], B0[b], acc[t]));
            }
            __syncwarp();
            // the warp's rows qw .. qw + n - 1, 9 16-byte pieces each (the padding of a part included)
            const int n = q1 - qw < 32 ? int(q1 - qw) : 32;
            float4* dst = reinterpret_cast<float4*>(G32 + kG32Row * qw);
            const float4* src = reinterpret_cast<const float4*>(grows);
            for (int i = lane; i < 9 * n; i += 32) dst[i] = src[i];
            __syncwarp();
        }
        __syncthreads();   // every warp is done with its G staging before the partials take the memory
        // the threads' partials: staged (stride kDiagThreads + 1 keeps the column reads apart in the
        // banks), 5 slices per entry with 4 interleaved sums each, then the slices in order
#pragma unroll
        for (int k = 0; k < 45; ++k) stage[k][threadIdx.x] = acc[k];
        __syncthreads();
        if (threadIdx.x < 45 * kDiagSlices) {
            const int k = threadIdx.x / kDiagSlices, sl = threadIdx.x % kDiagSlices;
            const int t0 = sl * kDiagSlice, t1 = min(t0 + kDiagSlice, kDiagThreads);
            float s4[4] = {0.f, 0.f, 0.f, 0.f};
            for (int t = t0; t < t1; t += 4)
#pragma unroll
                for (int u = 0; u < 4; ++u) s4[u] += stage[k][t + u];
            slice[k][sl] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        }
        __syncthreads();
        if (threadIdx.x < 81) {
            const int a = threadIdx.x / 9, b = threadIdx.x % 9;
            const int lo = a < b ? a : b, hi = a < b ? b : a;
            const int idx = lo * 9 - lo * (lo - 1) / 2 + (hi - lo);
            float v = slice[idx][0];
#pragma unroll
            for (int sl = 1; sl < kDiagSlices; ++sl) v += slice[idx][sl];
            double d = double(v);
            if (a == b) d += dadd[9 * int64_t(j) + a];
            Sd[81 * int64_t(j) + threadIdx.x] = d;
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------------------
// Mixed precision: the float64 parts of the build, the true residual and the back-substitution in
// double-float arithmetic (df64.cuh) on the float32 pipe.  r, J_p, J_l (per observation), L, b_l,
// y_l (per landmark) and the true residual's terms uv are stored as float2 (hi, lo) in the same
// buffers as their float64 counterparts of the float64 precision.  Float64 values enter per camera
// (the aux block), per landmark (the points, split by k_cam_prep), per camera again (x, split by
// the refinement's accumulation) or once at create (the measurements), and results leave per camera
// (b~, the damping, the true residual) or per landmark (the back-substitution); the conversions run
// on the float64 pipe, the arithmetic per observation does not.

__device__ __forceinline__ df64 ldd(const float2* p) { return df_ld(p); }
// two consecutive double-float values in one 16-byte load (p 16-byte aligned)
__device__ __forceinline__ void ldd2(const float2* p, df64& a, df64& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = df64(v.x, v.y);
    b = df64(v.z, v.w);
}
// n (even) consecutive double-float values from a 16-byte aligned address
template <int N>
__device__ __forceinline__ void lddn(const float2* p, df64 (&v)[N]) {
    static_assert(N % 2 == 0, "pairs");
#pragma unroll
    for (int k = 0; k < N; k += 2) ldd2(p + k, v[k], v[k + 1]);
}
__device__ __forceinline__ df64 ldg_d(const float2* p) {
    const float2 v = __ldg(p);
    return df64(v.x, v.y);
}

// damp() of the float64 build in double-float: d + lambda clamp(d, 1e-6, 1e32) (Marquardt) or d + lambda;
// lam = lambda split into double-float
__device__ __forceinline__ df64 damp_df(df64 d, int damping, df64 lam) {
    if (damping == BA_DAMPING_IDENTITY) return d + lam;
    const df64 c = d.hi < 1e-6f ? df64(1e-6f) : (d.hi > 1e32f ? df64(1e32f) : d);
    return d + lam * c;
}

// V_l^{-1} s from L (packed with its reciprocal diagonal), double-float
__device__ __forceinline__ void solve_V_df(const float2* L, df64 s0, df64 s1, df64 s2, df64& y0, df64& y1, df64& y2) {
    const df64 L0 = ldd(L), L1 = ldd(L + 1), L2 = ldd(L + 2), L3 = ldd(L + 3), L4 = ldd(L + 4), L5 = ldd(L + 5);
    const df64 z0 = s0 * L0;
    const df64 z1 = (s1 - L1 * z0) * L2;
    const df64 z2 = (s2 - L3 * z0 - L4 * z1) * L5;
    y2 = z2 * L5;
    y1 = (z1 - L4 * y2) * L2;
    y0 = (z0 - L1 * y1 - L3 * y2) * L0;
}

// r, J_p, J_l per observation in double-float (bal_jacobian_P on df64), and P, Y = R X in float32
// (their high parts) at the observation's camera-order position.  A warp takes 32 consecutive
// observations and writes their rows of J_p (32 x 144 B), J_l and r through shared memory as 16-byte
// stores: a thread storing its own 144-byte row made every store instruction touch 32 sectors.
constexpr int kLinThreads = 256;
__global__ void __launch_bounds__(kLinThreads) k_linearize_df(
    int64_t n_o, const float2* __restrict__ auxd, const float2* __restrict__ ptsd, const int32_t* __restrict__ oc,
    const int32_t* __restrict__ op, const float2* __restrict__ xyd, float2* __restrict__ r, float2* __restrict__ Jc,
    float2* __restrict__ Jl, float* __restrict__ PY32, const int32_t* __restrict__ cpos) {
    __shared__ __align__(16) float2 stage[kLinThreads / 32][32 * 18];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float2* const sw = stage[wid];
    const int64_t nwarps = gstride() >> 5;
    for (int64_t base = (gtid() >> 5) * 32; base < n_o; base += nwarps * 32) {   // warp-uniform
        const int64_t i = base + lane;
        const bool act = i < n_o;
        const int n = n_o - base < 32 ? int(n_o - base) : 32;
        df64 rr[2], jc[18], jl[6];
        if (act) {
            df64 ax[24], X[3], Y[3], P[3], m[2];
            const float2* cp = auxd + int64_t(oc[i]) * 24;
            const float2* xp = ptsd + int64_t(op[i]) * 3;
#pragma unroll
            for (int k = 0; k < 24; k += 2) {   // 16-byte loads of the camera's 192-byte aux block
                const float4 v = __ldg(reinterpret_cast<const float4*>(cp + k));
                ax[k] = df64(v.x, v.y);
                ax[k + 1] = df64(v.z, v.w);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) X[k] = ldg_d(xp + k);
            lddn<2>(xyd + 2 * i, m);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                Y[a] = ax[3 * a] * X[0] + ax[3 * a + 1] * X[1] + ax[3 * a + 2] * X[2];
                P[a] = Y[a] + ax[18 + a];
            }
            bal_jacobian_P<df64>(ax, Y, P, m, rr, jc, jl);
            float* py = PY32 + 6 * int64_t(cpos[i]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                py[k] = P[k].hi;
                py[3 + k] = Y[k].hi;
            }
        }
        // J_p: 32 rows of 18 values (144 B each), then J_l (48 B) with r (16 B) after it
#pragma unroll
        for (int k = 0; k < 18; ++k) sw[18 * lane + k] = make_float2(jc[k].hi, jc[k].lo);
        __syncwarp();
        {
            const float4* src = reinterpret_cast<const float4*>(sw);
            float4* dst = reinterpret_cast<float4*>(Jc + 18 * base);
            for (int u = lane; u < 9 * n; u += 32) dst[u] = src[u];
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 6; ++k) sw[6 * lane + k] = make_float2(jl[k].hi, jl[k].lo);
        sw[6 * 32 + 2 * lane] = make_float2(rr[0].hi, rr[0].lo);
        sw[6 * 32 + 2 * lane + 1] = make_float2(rr[1].hi, rr[1].lo);
        __syncwarp();
        {
            const float4* src = reinterpret_cast<const float4*>(sw);
            float4* dl = reinterpret_cast<float4*>(Jl + 6 * base);
            for (int u = lane; u < 3 * n; u += 32) dl[u] = src[u];
            const float4* srr = reinterpret_cast<const float4*>(sw + 6 * 32);
            float4* dr = reinterpret_cast<float4*>(r + 2 * base);
            for (int u = lane; u < n; u += 32) dr[u] = srr[u];
        }
        __syncwarp();
    }
}

// Per landmark in double-float: V_lambda = sum J_l^T J_l + damping, b_l = sum J_l^T r, V = L L^T
// (L packed with its reciprocal diagonal), y_l = V^{-1} b_l; L also in float32 (its high parts).
// The float64 V and e of the float64 build are not needed here (the getters form V on request).
__global__ void k_landmarks_df(int32_t n_l, const int64_t* __restrict__ pt_ptr, const int32_t* __restrict__ order,
                               const float2* __restrict__ r, const float2* __restrict__ Jl, int damping, float lam_hi,
                               float lam_lo, float2* __restrict__ Lout, float2* __restrict__ blout,
                               float* __restrict__ L32, float2* __restrict__ yout, int* status) {
    const df64 lam(lam_hi, lam_lo);
    for (int64_t t = gtid(); t < n_l; t += gstride()) {
        const int64_t l = order[t];
        df64 v00(0.f), v01(0.f), v02(0.f), v11(0.f), v12(0.f), v22(0.f), b0(0.f), b1(0.f), b2(0.f);
#pragma unroll 4
        for (int64_t o = pt_ptr[l]; o < pt_ptr[l + 1]; ++o) {
            df64 jv[6], rv[2];
            lddn<6>(Jl + 6 * o, jv);
            lddn<2>(r + 2 * o, rv);
            const df64 a0 = jv[0], a1 = jv[1], a2 = jv[2], c0 = jv[3], c1 = jv[4], c2 = jv[5];
            const df64 r0 = rv[0], r1 = rv[1];
            v00 += a0 * a0 + c0 * c0;
            v01 += a0 * a1 + c0 * c1;
            v02 += a0 * a2 + c0 * c2;
            v11 += a1 * a1 + c1 * c1;
            v12 += a1 * a2 + c1 * c2;
            v22 += a2 * a2 + c2 * c2;
            b0 += a0 * r0 + c0 * r1;
            b1 += a1 * r0 + c1 * r1;
            b2 += a2 * r0 + c2 * r1;
        }
        v00 = damp_df(v00, damping, lam);
        v11 = damp_df(v11, damping, lam);
        v22 = damp_df(v22, damping, lam);
        const df64 i00 = rsqrt_fast(v00);
        const df64 l10 = v01 * i00, l20 = v02 * i00;
        const df64 i11 = rsqrt_fast(v11 - l10 * l10);
        const df64 l21 = (v12 - l20 * l10) * i11;
        const df64 i22 = rsqrt_fast(v22 - l20 * l20 - l21 * l21);
        if (!(df_positive(i00) && df_positive(i11) && df_positive(i22))) atomicExch(status, BA_ERR_SINGULAR);
        const df64 Lv[6] = {i00, l10, i11, l20, l21, i22};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            df_st(Lout + 6 * l + k, Lv[k]);
            L32[6 * l + k] = Lv[k].hi;
        }
        df_st(blout + 3 * l, b0);
        df_st(blout + 3 * l + 1, b1);
        df_st(blout + 3 * l + 2, b2);
        const df64 e0 = b0 * i00;
        const df64 e1 = (b1 - l10 * e0) * i11;
        const df64 e2 = (b2 - l20 * e0 - l21 * e1) * i22;
        const df64 y2 = e2 * i22;
        const df64 y1 = (e1 - l21 * y2) * i11;
        const df64 y0 = (e0 - l10 * y1 - l20 * y2) * i00;
        df_st(yout + 3 * l, y0);
        df_st(yout + 3 * l + 1, y1);
        df_st(yout + 3 * l + 2, y2);
    }
}

// Sum of a double-float value over the CTA's kCamThreads threads in a fixed order (warp shuffle
// tree, then the warps in order); red: [kCamThreads / 32] per value.  Every thread gets the sum.
template <int NV>
__device__ __forceinline__ void cta_sum_df(df64 (&v)[NV], df64 (*red)[NV]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += df_shfl_xor(v[k], o);
        if (lane == 0) red[wid][k] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        df64 t = red[0][k];
#pragma unroll
        for (int w = 1; w < kCamThreads / 32; ++w) t += red[w][k];
        v[k] = t;
    }
    __syncthreads();
}

// Per camera in double-float: b~_j = sum_o J_p^T (r_o - J_l y_l) (Eq. 14) and the damping
// lambda D_p^T D_p from sum_o diag(J_p^T J_p); both leave as float64.
__global__ void __launch_bounds__(kCamThreads) k_cam_rhs_df(
    int32_t n_c, const int64_t* __restrict__ cam_ptr, const int32_t* __restrict__ cam_obs,
    const int32_t* __restrict__ op, const float2* __restrict__ r, const float2* __restrict__ Jc,
    const float2* __restrict__ Jl, const float2* __restrict__ yl, int damping, double lambda,
    double* __restrict__ btout, double* __restrict__ dadd) {
    __shared__ df64 red[kCamThreads / 32][18];
    for (int j = blockIdx.x; j < n_c; j += gridDim.x) {
        df64 v[18];
#pragma unroll
        for (int k = 0; k < 18; ++k) v[k] = df64(0.f);
        for (int64_t q = cam_ptr[j] + threadIdx.x; q < cam_ptr[j + 1]; q += blockDim.x) {
            const int64_t o = cam_obs[q];
            const float2* y = yl + 3 * int64_t(op[o]);
            const df64 y0 = ldd(y), y1 = ldd(y + 1), y2 = ldd(y + 2);
            df64 jl[6], rv[2], jc[18];
            lddn<6>(Jl + 6 * o, jl);
            lddn<2>(r + 2 * o, rv);
            lddn<18>(Jc + 18 * o, jc);
            const df64 s0 = rv[0] - (jl[0] * y0 + jl[1] * y1 + jl[2] * y2);
            const df64 s1 = rv[1] - (jl[3] * y0 + jl[4] * y1 + jl[5] * y2);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const df64 c0 = jc[a], c1 = jc[9 + a];
                v[a] += c0 * s0 + c1 * s1;
                v[9 + a] += c0 * c0 + c1 * c1;
            }
        }
        cta_sum_df<18>(v, red);
        if (threadIdx.x < 18) {
            const int k = threadIdx.x;
            const double d = df_to(v[k]);
            if (k < 9) btout[9 * int64_t(j) + k] = d;
            else dadd[9 * int64_t(j) + k - 9] = damp_add(d, damping, lambda);
        }
    }
}

// True residual, observation pass, double-float: u_o = J_p x_cam(o) into uv (xd: x split into
// double-float per camera).  Thread = observation, so a warp reads 32 consecutive J_p rows.
__global__ void k_jres_obs_df(int64_t n_o, const int32_t* __restrict__ oc, const float2* __restrict__ Jc,
                              const float2* __restrict__ xd, float2* __restrict__ uv) {
    for (int64_t o = gtid(); o < n_o; o += gstride()) {
        const float2* xc = xd + 9 * int64_t(oc[o]);
        df64 jc[18];
        lddn<18>(Jc + 18 * o, jc);
        df64 u0(0.f), u1(0.f);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const df64 xa = ldg_d(xc + a);
            u0 += jc[a] * xa;
            u1 += jc[9 + a] * xa;
        }
        *reinterpret_cast<float4*>(uv + 2 * o) = make_float4(u0.hi, u0.lo, u1.hi, u1.lo);
    }
}

// True residual, landmark pass: y_l = V_l^-1 sum_o J_l^T u_o and v_o = u_o - J_l y_l in place of u_o.
// Landmarks in index order (not by track length): neighbouring lanes then read neighbouring rows,
// which on the 1000-camera case cut the DRAM reads from 184 to 125 MB and the time from 90 to 66 µs
// despite the lanes' unequal loop lengths (the landmark factors, heavier per observation, run
// faster in track-length order).
__global__ void k_jres_land_df(int32_t n_l, const int64_t* __restrict__ pt_ptr, const float2* __restrict__ Jl,
                               const float2* __restrict__ Lall, float2* __restrict__ uv) {
    for (int64_t l = gtid(); l < n_l; l += gstride()) {
        df64 s0(0.f), s1(0.f), s2(0.f);
        const int64_t o0 = pt_ptr[l], o1 = pt_ptr[l + 1];
#pragma unroll 4
        for (int64_t o = o0; o < o1; ++o) {
            df64 jl[6], u[2];
            lddn<6>(Jl + 6 * o, jl);
            lddn<2>(uv + 2 * o, u);
            s0 += jl[0] * u[0] + jl[3] * u[1];
            s1 += jl[1] * u[0] + jl[4] * u[1];
            s2 += jl[2] * u[0] + jl[5] * u[1];
        }
        df64 y0, y1, y2;
        solve_V_df(Lall + 6 * l, s0, s1, s2, y0, y1, y2);
        for (int64_t o = o0; o < o1; ++o) {
            df64 jl[6], u[2];
            lddn<6>(Jl + 6 * o, jl);
            lddn<2>(uv + 2 * o, u);
            const df64 v0 = u[0] - (jl[0] * y0 + jl[1] * y1 + jl[2] * y2);
            const df64 v1 = u[1] - (jl[3] * y0 + jl[4] * y1 + jl[5] * y2);
            *reinterpret_cast<float4*>(uv + 2 * o) = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
        }
    }
}

// True residual, camera pass: out_j = -b~_j - (S x)_j with (S x)_j = sum_{o in j} J_p^T v_o (double-float)
// + lambda D_p x_j (float64); camera j's |out_j|^2 and |b~_j|^2 into partial[2 j], partial[2 j + 1].
__global__ void __launch_bounds__(kCamThreads) k_jres_cam_df(
    int32_t n_c, const int64_t* __restrict__ cam_ptr, const int32_t* __restrict__ cam_obs,
    const float2* __restrict__ Jc, const float2* __restrict__ uv, const double* __restrict__ dadd,
    const double* __restrict__ x, const double* __restrict__ bt, double* __restrict__ out,
    double* __restrict__ partial) {
    __shared__ df64 red[kCamThreads / 32][9];
    for (int j = blockIdx.x; j < n_c; j += gridDim.x) {
        df64 acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = df64(0.f);
        for (int64_t q = cam_ptr[j] + threadIdx.x; q < cam_ptr[j + 1]; q += blockDim.x) {
            const int64_t o = cam_obs[q];
            df64 u[2], jc[18];
            lddn<2>(uv + 2 * o, u);
            lddn<18>(Jc + 18 * o, jc);
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] += jc[a] * u[0] + jc[9 + a] * u[1];
        }
        cta_sum_df<9>(acc, red);
        double tt = 0.0, bb = 0.0;
        if (threadIdx.x < 9) {
            const int a = threadIdx.x;
            const int64_t i = 9 * int64_t(j) + a;
            const double sx = df_to(acc[a]) + dadd[i] * x[i];
            const double b_ = bt[i];
            const double rv = -b_ - sx;
            if (out) out[i] = rv;
            tt = rv * rv;
            bb = b_ * b_;
        }
        if (threadIdx.x < 32) {
            tt = warp_sum(tt);
            bb = warp_sum(bb);
            if (threadIdx.x == 0) {
                partial[2 * int64_t(j)] = tt;
                partial[2 * int64_t(j) + 1] = bb;
            }
        }
        __syncthreads();
    }
}

// Back-substitution in double-float: dx_l = -V_l^{-1} (b_l + sum_o J_l^T J_p dx_p,cam(o)) (Eq. 15 with
// the sign that follows from Eq. 6); dxpd: dx_p split into double-float per camera.
__global__ void k_back_sub_df(int32_t n_l, const int64_t* __restrict__ pt_ptr, const int32_t* __restrict__ order,
                              const int32_t* __restrict__ oc, const float2* __restrict__ Jc,
                              const float2* __restrict__ Jl, const float2* __restrict__ Lall,
                              const float2* __restrict__ bl, const float2* __restrict__ dxpd,
                              double* __restrict__ dxl) {
    for (int64_t t = gtid(); t < n_l; t += gstride()) {
        const int64_t l = order[t];
        df64 s0 = ldd(bl + 3 * l), s1 = ldd(bl + 3 * l + 1), s2 = ldd(bl + 3 * l + 2);
        for (int64_t o = pt_ptr[l]; o < pt_ptr[l + 1]; ++o) {
            const float2* xc = dxpd + 9 * int64_t(oc[o]);
            df64 jc[18], jl[6];
            lddn<18>(Jc + 18 * o, jc);
            lddn<6>(Jl + 6 * o, jl);
            df64 u0(0.f), u1(0.f);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const df64 xa = ldg_d(xc + a);
                u0 += jc[a] * xa;
                u1 += jc[9 + a] * xa;
            }
            s0 += jl[0] * u0 + jl[3] * u1;
            s1 += jl[1] * u0 + jl[4] * u1;
            s2 += jl[2] * u0 + jl[5] * u1;
        }
        df64 y0, y1, y2;
        solve_V_df(Lall + 6 * l, s0, s1, s2, y0, y1, y2);
        dxl[3 * l] = -df_to(y0);
        dxl[3 * l + 1] = -df_to(y1);
        dxl[3 * l + 2] = -df_to(y2);
    }
}

// float64 -> double-float, elementwise
__global__ void k_split_df(const double* __restrict__ in, float2* __restrict__ out, int64_t n) {
    for (int64_t i = gtid(); i < n; i += gstride()) df_st(out + i, df_from(in[i]));
}
// double-float -> float64 in place (the buffer holds n float2 values; each becomes the double at
// the same index, of the same size)
__global__ void k_df_to_double(double* __restrict__ buf, int64_t n) {
    for (int64_t i = gtid(); i < n; i += gstride()) {
        const float2 v = reinterpret_cast<const float2*>(buf)[i];
        buf[i] = double(v.x) + double(v.y);
    }
}

// D_j^{-1} = (S_jj)^{-1} = L^{-T} L^{-1} from the Cholesky factor of the diagonal block.
// With lam != nullptr the block is first scaled by its diagonal, B^ = s B s with s_a = B_aa^{-1/2};
// Dinv then receives (B^)^{-1}, lam the scale factors and lam32 their float32 roundings.
__global__ void k_block_jacobi(int32_t n_c, const double* __restrict__ Sd, double* __restrict__ Dinv,
                               double* __restrict__ lam, float* __restrict__ lam32, int* status) {
    for (int64_t j = gtid(); j < n_c; j += gstride()) {
        double L[81];
        for (int e = 0; e < 81; ++e) L[e] = Sd[81 * j + e];
        if (lam) {
            double sc[9];
            for (int a = 0; a < 9; ++a) {
                sc[a] = L[9 * a + a] > 0.0 ? 1.0 / sqrt(L[9 * a + a]) : 1.0;
                lam[9 * j + a] = sc[a];
                lam32[9 * j + a] = float(sc[a]);
            }
            for (int a = 0; a < 9; ++a)
                for (int b = 0; b < 9; ++b) L[9 * a + b] *= sc[a] * sc[b];
        }
        // Cholesky with reciprocal square roots: L[c][c] keeps 1 / l_cc (the exact float64 divisions
        // and square roots are long dependent chains on this GPU's narrow float64 pipe)
        bool ok = true;
        for (int c = 0; c < 9; ++c) {
            double d = L[9 * c + c];
            for (int k = 0; k < c; ++k) d -= L[9 * c + k] * L[9 * c + k];
            if (!(d > 0.0)) { ok = false; d = 1.0; }
            const double ic = rsqrt_fast(d);
            L[9 * c + c] = ic;
            for (int a = c + 1; a < 9; ++a) {
                double v = L[9 * a + c];
                for (int k = 0; k < c; ++k) v -= L[9 * a + k] * L[9 * c + k];
                L[9 * a + c] = v * ic;
            }
        }
        if (!ok) atomicExch(status, BA_ERR_SINGULAR);
        // Li = L^{-1} (lower), column by column
        double Li[81];
        for (int k = 0; k < 81; ++k) Li[k] = 0.0;
        for (int c = 0; c < 9; ++c) {
            Li[9 * c + c] = L[9 * c + c];
            for (int a = c + 1; a < 9; ++a) {
                double v = 0.0;
                for (int k = c; k < a; ++k) v -= L[9 * a + k] * Li[9 * k + c];
                Li[9 * a + c] = v * L[9 * a + a];
            }
        }
        double* D = Dinv + 81 * j;
        for (int a = 0; a < 9; ++a) {
            for (int b = a; b < 9; ++b) {
                double v = 0.0;
                for (int k = b; k < 9; ++k) v += Li[9 * k + a] * Li[9 * k + b];
                D[9 * a + b] = v;
                D[9 * b + a] = v;
            }
        }
    }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    for (int64_t i = gtid(); i < n; i += gstride()) out[i] = static_cast<float>(in[i]);
}

// dx_l = -L^{-T} (e_l + sum_o G_o^T dx_p,cam(o))
__global__ void k_back_substitute(int32_t n_l, const int64_t* __restrict__ pt_ptr, const int32_t* __restrict__ order,
                                  const int32_t* __restrict__ oc, const double* __restrict__ G,
                                  const double* __restrict__ Lall, const double* __restrict__ e,
                                  const double* __restrict__ dxp, double* __restrict__ dxl) {
    for (int64_t t = gtid(); t < n_l; t += gstride()) {
        const int64_t l = order[t];
        double a0 = e[3 * l], a1 = e[3 * l + 1], a2 = e[3 * l + 2];
        for (int64_t o = pt_ptr[l]; o < pt_ptr[l + 1]; ++o) {
            const double* g = G + 27 * o;
            const double* x = dxp + 9 * int64_t(oc[o]);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                double xa = x[a];
                a0 += g[3 * a] * xa;
                a1 += g[3 * a + 1] * xa;
                a2 += g[3 * a + 2] * xa;
            }
        }
        const double* L = Lall + 6 * l;   // reciprocal diagonal at 0, 2, 5
        double y2 = a2 * L[5];
        double y1 = (a1 - L[4] * y2) * L[2];
        double y0 = (a0 - L[1] * y1 - L[3] * y2) * L[0];
        dxl[3 * l] = -y0;
        dxl[3 * l + 1] = -y1;
        dxl[3 * l + 2] = -y2;
    }
}

// partial[b] = sum over this CTA's observations of |pi - m|^2
__global__ void k_cost(int64_t n_o, const double* __restrict__ cams, const double* __restrict__ pts,
                       const int32_t* __restrict__ oc, const int32_t* __restrict__ op,
                       const double* __restrict__ xy, double* __restrict__ partial) {
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (int64_t i = gtid(); i < n_o; i += gstride()) {
        double c[9], X[3], pr[2];
        const double* cp = cams + int64_t(oc[i]) * 9;
        const double* xp = pts + int64_t(op[i]) * 3;
#pragma unroll
        for (int k = 0; k < 9; ++k) c[k] = cp[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) X[k] = xp[k];
        bal_project(c, X, pr);
        double d0 = pr[0] - xy[2 * i], d1 = pr[1] - xy[2 * i + 1];
        acc += d0 * d0 + d1 * d1;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[w];
        partial[blockIdx.x] = v;
    }
}

__global__ void k_add(const double* __restrict__ a, const double* __restrict__ da, double* __restrict__ out, int64_t n) {
    for (int64_t i = gtid(); i < n; i += gstride()) out[i] = a[i] + da[i];
}

__global__ void k_unpermute(const double* __restrict__ in, const int32_t* __restrict__ perm, double* __restrict__ out,
                            int64_t n_o, int width) {
    for (int64_t i = gtid(); i < n_o * width; i += gstride()) {
        int64_t o = i / width;
        int c = static_cast<int>(i - o * width);
        out[int64_t(perm[o]) * width + c] = in[i];
    }
}

// tiled layout -> row-major 9x9 blocks.  S64 (float64 precision) or S32 = Lam S Lam (mixed, unscaled here),
// with the float64 diagonal blocks Sd in both cases.
__global__ void k_unslab(int32_t n_c, const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ tile_ptr,
                         const int32_t* __restrict__ col, const double* __restrict__ S64, const float* __restrict__ S32,
                         const double* __restrict__ lam, const double* __restrict__ Sd, double* __restrict__ out) {
    const int64_t total = row_ptr[n_c] * 81;
    for (int64_t i = gtid(); i < total; i += gstride()) {
        const int64_t q = i / 81;
        const int e = static_cast<int>(i - q * 81);
        // row of block q by binary search
        int lo = 0, hi = n_c;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= q) lo = mid; else hi = mid;
        }
        const int64_t k = col[q];
        if (k == lo) {
            out[i] = Sd[81 * int64_t(lo) + e];
        } else if (S64) {
            out[i] = S64[s_at(tile_ptr, lo, q - row_ptr[lo], e)];
        } else {
            const double v = double(S32[s_at(tile_ptr, lo, q - row_ptr[lo], e)]);
            out[i] = v / (lam[9 * int64_t(lo) + e / 9] * lam[9 * k + e % 9]);
        }
    }
}

}  // namespace

void launch_project(int64_t n_o, const double* cams, const double* pts, const int32_t* oc, const int32_t* op,
                    double* out, cudaStream_t st) {
    if (n_o <= 0) return;
    k_project<<<grid_for(n_o, kThreads), kThreads, 0, st>>>(n_o, cams, pts, oc, op, out);
}

void launch_linearize(const Structure& s, System& y, cudaStream_t st) {
    if (y.S32) {   // mixed precision: double-float
        k_linearize_df<<<grid_for(s.n_o, kLinThreads), kLinThreads, 0, st>>>(
            s.n_o, y.auxd, y.ptsd, s.obs_cam, s.obs_pt, s.obs_xyd, reinterpret_cast<float2*>(y.r),
            reinterpret_cast<float2*>(y.Jc), reinterpret_cast<float2*>(y.Jl), y.PY32, s.cpos);
        return;
    }
    k_linearize<<<grid_for(s.n_o, kThreads), kThreads, 0, st>>>(s.n_o, y.aux, y.pts, s.obs_cam, s.obs_pt,
                                                                 s.obs_xy, y.r, y.Jc, y.Jl, y.PY32, s.cpos);
}

void launch_landmarks(const Structure& s, System& y, int damping, double lambda, cudaStream_t st) {
    if (y.S32) {   // mixed precision: double-float
        const float lh = float(lambda), ll = float(lambda - double(lh));
        k_landmarks_df<<<grid_for(s.n_l, kThreads), kThreads, 0, st>>>(
            s.n_l, s.pt_ptr, s.lm_order, reinterpret_cast<const float2*>(y.r), reinterpret_cast<const float2*>(y.Jl),
            damping, lh, ll, reinterpret_cast<float2*>(y.L), reinterpret_cast<float2*>(y.bl), y.L32,
            reinterpret_cast<float2*>(y.yl), y.status);
        return;
    }
    k_landmarks<<<grid_for(s.n_l, kThreads), kThreads, 0, st>>>(s.n_l, s.pt_ptr, s.lm_order, y.r, y.Jl, damping,
                                                                 lambda, y.V, y.L, y.bl, y.e, y.L32, y.yl, y.status);
}

void launch_obs_G(const Structure& s, System& y, cudaStream_t st) {
    k_obs_G<<<grid_for(s.n_o, kThreads), kThreads, 0, st>>>(s.n_o, s.obs_pt, y.Jc, y.Jl, y.L, y.G);
}

static int cam_grid(const Structure& s) { return s.n_c < num_sms() * 8 ? s.n_c : num_sms() * 8; }

void launch_cameras(const Structure& s, System& y, int damping, double lambda, cudaStream_t st) {
    k_cameras<<<cam_grid(s), kCamThreads, 0, st>>>(s.n_c, s.cam_ptr, s.cam_obs, s.obs_pt, y.r, y.Jc, y.G, y.e, damping,
                                                   lambda, y.U, y.bp, y.bt);
}

// Mixed precision, on request (ba_get_normal): the float64 U, b_p, V, b_l of the last build, from
// float64 copies of its double-float r, J_p, J_l (r64, Jc64, Jl64, n_o x 2 / 18 / 6) with the kernels
// of the float64 build; V, L, b_l, e go to V64, L64, bl64, e64 (n_l x 9 / 6 / 3 / 3), U and b_p to
// y.U, y.bp.
void launch_normal_request(const Structure& s, System& y, int damping, double lambda, double* r64, double* Jc64,
                           double* Jl64, double* V64, double* L64, double* bl64, double* e64, cudaStream_t st) {
    const int64_t n[3] = {2 * s.n_o, 18 * s.n_o, 6 * s.n_o};
    const double* src[3] = {y.r, y.Jc, y.Jl};
    double* dst[3] = {r64, Jc64, Jl64};
    for (int k = 0; k < 3; ++k) {
        cudaMemcpyAsync(dst[k], src[k], sizeof(double) * n[k], cudaMemcpyDeviceToDevice, st);
        k_df_to_double<<<grid_for(n[k], kThreads), kThreads, 0, st>>>(dst[k], n[k]);
    }
    k_landmarks<<<grid_for(s.n_l, kThreads), kThreads, 0, st>>>(s.n_l, s.pt_ptr, s.lm_order, r64, Jl64, damping,
                                                                 lambda, V64, L64, bl64, e64, nullptr, nullptr,
                                                                 y.status);
    k_cameras<<<cam_grid(s), kCamThreads, 0, st>>>(s.n_c, s.cam_ptr, s.cam_obs, s.obs_pt, r64, Jc64, nullptr, e64,
                                                   damping, lambda, y.U, y.bp, nullptr);
}

// double-float -> float64 in place, n values
void launch_df_to_double(double* buf, int64_t n, cudaStream_t st) {
    k_df_to_double<<<grid_for(n, kThreads), kThreads, 0, st>>>(buf, n);
}

void launch_schur_diag(const Structure& s, System& y, cudaStream_t st) {
    k_schur_diag<<<cam_grid(s), kCamThreads, 0, st>>>(s.n_c, s.cam_ptr, s.cam_obs, y.G, y.U, y.Sd);
}

void launch_cam_rhs(const Structure& s, System& y, int damping, double lambda, cudaStream_t st) {
    // mixed precision only (the float64 build forms b~ from G): double-float
    k_cam_rhs_df<<<cam_grid(s), kCamThreads, 0, st>>>(
        s.n_c, s.cam_ptr, s.cam_obs, s.obs_pt, reinterpret_cast<const float2*>(y.r),
        reinterpret_cast<const float2*>(y.Jc), reinterpret_cast<const float2*>(y.Jl),
        reinterpret_cast<const float2*>(y.yl), damping, lambda, y.bt, y.dadd);
}

void launch_schur_diag32(const Structure& s, System& y, cudaStream_t st) {
    k_schur_diag32<<<cam_grid(s), kDiagThreads, 0, st>>>(s.n_c, s.cam_ptr, s.cam_lm, y.aux32, y.PY32, y.L32, y.dadd,
                                                         y.Sd, y.G32);
}

void launch_schur(const Structure& s, System& y, cudaStream_t st) {
    if (s.n_up > 0)
        k_schur_off_rows<double><<<grid_for(s.n_up * 32, kThreads), kThreads, 0, st>>>(
            s.n_up, s.up_dst, s.up_mdst, s.up_pair_ptr, s.pairs, y.G, y.S);
    k_put_diag<double><<<grid_for(int64_t(s.n_c) * 81, kThreads), kThreads, 0, st>>>(
        s.n_c, s.row_ptr, s.tile_ptr, s.diag_pos, y.Sd, nullptr, y.S, nullptr, nullptr);
}

void launch_schur_mixed(const Structure& s, System& y, cudaStream_t st) {
    if (s.n_up > 0)
        k_schur_off_sub<float><<<grid_for((s.n_up + 2) / 3 * 32, kThreads), kThreads, 0, st>>>(
            s.n_up, s.up_order, s.up_dst, s.up_mdst, s.up_udst, s.up_pair_ptr, s.pairs, s.up_cams, y.lam32, y.G32,
            y.S32, y.S32u);
    k_put_diag<float><<<grid_for(int64_t(s.n_c) * 81, kThreads), kThreads, 0, st>>>(
        s.n_c, s.row_ptr, s.tile_ptr, s.diag_pos, y.Sd, y.lam, y.S32, s.tile_ptr_u, y.S32u);
}

// Mixed precision's true residual in double-float (three launches); y.xd must hold x split into
// double-float (the refinement's accumulation, which forms x, writes it).
int launch_implicit_residual(const Structure& s, const System& y, const double* x, double* out, double* partial,
                             cudaStream_t st) {
    k_jres_obs_df<<<grid_for(s.n_o, kThreads), kThreads, 0, st>>>(
        s.n_o, s.obs_cam, reinterpret_cast<const float2*>(y.Jc), y.xd, reinterpret_cast<float2*>(y.uv));
    k_jres_land_df<<<grid_for(s.n_l, kThreads), kThreads, 0, st>>>(
        s.n_l, s.pt_ptr, reinterpret_cast<const float2*>(y.Jl), reinterpret_cast<const float2*>(y.L),
        reinterpret_cast<float2*>(y.uv));
    k_jres_cam_df<<<cam_grid(s), kCamThreads, 0, st>>>(s.n_c, s.cam_ptr, s.cam_obs,
                                                       reinterpret_cast<const float2*>(y.Jc),
                                                       reinterpret_cast<const float2*>(y.uv), y.dadd, x, y.bt, out,
                                                       partial);
    return 3;
}

void launch_cam_prep(const Structure& s, System& y, cudaStream_t st) {
    if (y.ptsd) {   // mixed precision: also the double-float aux blocks and points
        const int64_t n_pv = int64_t(s.n_l) * 3;
        k_cam_prep<<<grid_for(n_pv > s.n_c ? n_pv : s.n_c, 256), 256, 0, st>>>(s.n_c, y.cams, y.aux, y.aux32, y.auxd,
                                                                              n_pv, y.pts, y.ptsd);
        return;
    }
    k_cam_prep<<<grid_for(s.n_c, 64), 64, 0, st>>>(s.n_c, y.cams, y.aux, y.aux32, nullptr, 0, nullptr, nullptr);
}

// Float64: D^{-1}.  Mixed precision: Lam and the inverse blocks of the scaled system only (its solves
// use no other; launch_block_jacobi_plain forms D^{-1} when it is asked for).
void launch_block_jacobi(const Structure& s, System& y, cudaStream_t st) {
    if (y.S32) k_block_jacobi<<<grid_for(s.n_c, 64), 64, 0, st>>>(s.n_c, y.Sd, y.Dhat, y.lam, y.lam32, y.status);
    else launch_block_jacobi_plain(s, y, st);
}

void launch_block_jacobi_plain(const Structure& s, System& y, cudaStream_t st) {
    k_block_jacobi<<<grid_for(s.n_c, 64), 64, 0, st>>>(s.n_c, y.Sd, y.Dinv, nullptr, nullptr, y.status);
}


void launch_to_float(const double* in, float* out, int64_t n, cudaStream_t st) {
    k_to_float<<<grid_for(n, kThreads), kThreads, 0, st>>>(in, out, n);
}

void launch_back_substitute(const Structure& s, const System& y, const double* dxp, double* dxl, cudaStream_t st) {
    if (y.G)
        k_back_substitute<<<grid_for(s.n_l, kThreads), kThreads, 0, st>>>(s.n_l, s.pt_ptr, s.lm_order, s.obs_cam, y.G,
                                                                           y.L, y.e, dxp, dxl);
    else {
        // mixed precision: dx_p split into double-float (the true residual's buffer, idle here)
        k_split_df<<<grid_for(int64_t(s.n_c) * 9, kThreads), kThreads, 0, st>>>(dxp, y.xd, int64_t(s.n_c) * 9);
        k_back_sub_df<<<grid_for(s.n_l, kThreads), kThreads, 0, st>>>(
            s.n_l, s.pt_ptr, s.lm_order, s.obs_cam, reinterpret_cast<const float2*>(y.Jc),
            reinterpret_cast<const float2*>(y.Jl), reinterpret_cast<const float2*>(y.L),
            reinterpret_cast<const float2*>(y.bl), y.xd, dxl);
    }
}

void launch_cost(const Structure& s, const double* cams, const double* pts, double* partial, int nparts,
                 cudaStream_t st) {
    k_cost<<<nparts, kThreads, 0, st>>>(s.n_o, cams, pts, s.obs_cam, s.obs_pt, s.obs_xy, partial);
}

void launch_add_params(const double* a, const double* da, double* out, int64_t n, cudaStream_t st) {
    k_add<<<grid_for(n, kThreads), kThreads, 0, st>>>(a, da, out, n);
}

void launch_unpermute(const double* in, const int32_t* perm, double* out, int64_t n_o, int width, cudaStream_t st) {
    k_unpermute<<<grid_for(n_o * width, kThreads), kThreads, 0, st>>>(in, perm, out, n_o, width);
}

void launch_unslab(const Structure& s, const System& y, double* out, cudaStream_t st) {
    k_unslab<<<grid_for(s.nnzb * 81, kThreads), kThreads, 0, st>>>(s.n_c, s.row_ptr, s.tile_ptr, s.col, y.S, y.S32,
                                                                    y.lam, y.Sd, out);
}

}  // namespace ba

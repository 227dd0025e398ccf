// Trajectory tracking optimisation (arXiv 2503.14160, Sec. 4.2, Eq. discrete): the planned
// path q*(s) becomes a near-time-optimal trajectory by trapezoidal direct collocation,
//
//     min  t_F + w_s sum_k u_k^T R u_k + w_t sum_k |q_a,k - q*_a,k|^2
//     s.t. x_{k+1} - x_k = h/2 (f_k + f_{k+1}),  x_0 = x_S,  x_N = x_T,  x_min <= x <= x_max,
//
// h = t_F / N, with f the crane dynamics of Sec. 2.1 with the actuated joints' accelerations as
// inputs. The paper's model parameters are not given; the model here has its structure: the
// four actuated joints driven through their accelerations, and two passive swing angles of the
// grapple, a point mass on a rigid link under the tip, whose accelerations follow from the
// Euler-Lagrange equations of a pendulum with an accelerated pivot.
//
// Method (the paper uses IPOPT; the library solves the same problem by): an augmented
// Lagrangian for the equality constraints (defects and end states) and a quadratic penalty
// for the bounds, so that the objective is F(z) = t_F + 1/2 |r(z)|^2 + const; damped
// Gauss-Newton (Levenberg-Marquardt) steps (J^T J + mu (diag J^T J + 1e-9)) dz = -(e_t + J^T r),
// accepted when F decreases (mu / 3, else mu * 4), `inner` of them per multiplier update
// lambda <- lambda + rho c. J^T J is block tridiagonal in the grid points' 16 variables
// w_k = (x_k, u_k) with a border for t_F (the defects couple neighbours and t_F); it is
// factored block by block (16 x 16 Cholesky factors L_k, L_k^-1 E_k) and the border is taken
// through its Schur complement. The dynamics' Jacobian per grid point comes from forward-mode
// differentiation (value and one derivative per pass, 16 passes). Everything is FP64: one
// CTA of 256 threads per trajectory.
#include <cmath>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "cp_internal.cuh"

// An NVTX range over a scope (no-op without a profiling tool).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

namespace cp {
namespace {

constexpr int kTrajThreads = 256;
constexpr int NX = 12, NU = 4, NW = 16;
constexpr double kGravity = 9.81;

// A value and one derivative (forward mode).
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual dsin(Dual a) { return {sin(a.v), cos(a.v) * a.d}; }
__device__ __forceinline__ Dual dcos(Dual a) { return {cos(a.v), -sin(a.v) * a.d}; }
__device__ __forceinline__ double dsin(double a) { return sin(a); }
__device__ __forceinline__ double dcos(double a) { return cos(a); }
template <typename T> __device__ __forceinline__ T lift(double v);
template <> __device__ __forceinline__ double lift<double>(double v) { return v; }
template <> __device__ __forceinline__ Dual lift<Dual>(double v) { return {v, 0.0}; }

// 1 / sqrt(a) in FP64 for the pivots of the block factorisation: an FP32 seed and two
// Newton steps (quadratic convergence: about 22 -> 44 -> 88 bits), a short dependent chain
// where FP64 operations wait tens of cycles each. Arguments outside FP32's normal range take
// the IEEE operations (a non-positive pivot gives NaN, as sqrt would).
__device__ __forceinline__ double rsqrt_pivot(double a)
{
    const float af = (float)a;
    if (!(af > 1e-30f && af < 1e30f)) return 1.0 / sqrt(a);
    double y = (double)rsqrtf(af);
    const double hh = 0.5 * a;
    y = y * fma(-hh * y, y, 1.5);
    y = y * fma(-hh * y, y, 1.5);
    return y;
}

struct TrajDev {
    double base_z, boom_len, jib_len, ell;
    double omega_s, omega_t, R[4];
    double x_min[NX], x_max[NX];
    double rho, rho_b, mu0;
    int N, outer, inner;
};

// x' = f(x, u): the actuated joints' rates and accelerations, and the swing accelerations from
// the tip acceleration T'' (cylindrical coordinates of the tip) by
//   (ddalpha, ddbeta) = -(r_a . v / l, r_b . v / (l cos^2 alpha)),  v = T'' + l w + g z,
//   r = (sin a, cos a sin b, -cos a cos b),  w = r_aa da^2 + 2 r_ab da db + r_bb db^2.
template <typename T>
__device__ void traj_f(const TrajDev &td, const T *x, const T *u, T *out)
{
    const T q1 = x[0], q2 = x[1], q3 = x[2], q4 = x[3], a = x[4], b = x[5];
    const T d1 = x[6], d2 = x[7], d3 = x[8], d4 = x[9], da = x[10], db = x[11];
    const T u1 = u[0], u2 = u[1], u3 = u[2], u4 = u[3];
    const T lam = lift<T>(td.jib_len) + q4;
    const T A = q2, B = q2 + q3, dB = d2 + d3, ddB = u2 + u3;
    const T cA = dcos(A), sA = dsin(A), cB = dcos(B), sB = dsin(B);
    const T h = td.boom_len * cA + lam * cB;
    const T dh = lift<T>(0.0) - td.boom_len * sA * d2 + d4 * cB - lam * sB * dB;
    const T ddh = lift<T>(0.0) - td.boom_len * (cA * d2 * d2 + sA * u2) + u4 * cB - 2.0 * d4 * sB * dB -
                  lam * (cB * dB * dB + sB * ddB);
    const T ddz = td.boom_len * (cA * u2 - sA * d2 * d2) + u4 * sB + 2.0 * d4 * cB * dB +
                  lam * (cB * ddB - sB * dB * dB);
    const T a_r = ddh - h * d1 * d1, a_t = h * u1 + 2.0 * dh * d1;
    const T c1 = dcos(q1), s1 = dsin(q1);
    const T ax = a_r * c1 - a_t * s1, ay = a_r * s1 + a_t * c1;
    const T ca = dcos(a), sa = dsin(a), cb = dcos(b), sb = dsin(b);
    // w = r_aa da^2 + 2 r_ab da db + r_bb db^2
    const T wx = lift<T>(0.0) - sa * da * da;
    const T wy = lift<T>(0.0) - ca * sb * da * da - 2.0 * sa * cb * da * db - ca * sb * db * db;
    const T wz = ca * cb * da * da - 2.0 * sa * sb * da * db + ca * cb * db * db;
    const T vx = ax + td.ell * wx, vy = ay + td.ell * wy, vz = ddz + td.ell * wz + lift<T>(kGravity);
    const T ra_v = ca * vx - sa * sb * vy + sa * cb * vz;
    const T rb_v = ca * cb * vy + ca * sb * vz;
    out[0] = d1; out[1] = d2; out[2] = d3; out[3] = d4; out[4] = da; out[5] = db;
    out[6] = u1; out[7] = u2; out[8] = u3; out[9] = u4;
    out[10] = lift<T>(0.0) - ra_v / lift<T>(td.ell);
    out[11] = lift<T>(0.0) - rb_v / (td.ell * ca * ca);
}

// Per-trajectory device workspace (doubles), laid out by the launcher.
struct TrajWs {
    double *f;     // [N+1][12]
    double *Fj;    // [N+1][12][16] df/dw
    double *D;     // [N+1][16][16] diagonal blocks, then their Cholesky factors
    double *E;     // [N][16][16] off-diagonal blocks, then L_k^-1 E_k
    double *bb;    // [N+1][16] border column, then the forward/back solves
    double *g;     // [N+1][16] gradient, then the forward/back solves
};

__device__ __forceinline__ TrajWs ws_of(double *base, int N)
{
    TrajWs w;
    w.f = base;
    w.Fj = w.f + (size_t)(N + 1) * NX;
    w.D = w.Fj + (size_t)(N + 1) * NX * NW;
    w.E = w.D + (size_t)(N + 1) * NW * NW;
    w.bb = w.E + (size_t)N * NW * NW;
    w.g = w.bb + (size_t)(N + 1) * NW;
    return w;
}

// Block sum of a double over the CTA in a fixed order (deterministic).
__device__ double block_sum(double v, double *s_red)
{
    const int t = threadIdx.x;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((t & 31) == 0) s_red[t >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (t == 0)
        for (int i = 0; i < kTrajThreads / 32; ++i) s += s_red[i];
    __syncthreads();
    if (t == 0) s_red[0] = s;
    __syncthreads();
    const double r = s_red[0];
    __syncthreads();
    return r;
}

// f at every grid point of z (values only) into ws.f.
__device__ void eval_f(const TrajDev &td, const double *z, double *f)
{
    for (int k = threadIdx.x; k <= td.N; k += blockDim.x) {
        const double *w = z + 1 + (size_t)k * NW;
        traj_f<double>(td, w, w + NX, f + (size_t)k * NX);
    }
}

// The merit F(z) = t_F + 1/2 |r(z)|^2 (T6): the AL terms of the defects and end states, the
// effort and tracking sums over k = 1..N, and the bound penalty; f must be current for z.
__device__ double merit(const TrajDev &td, const double *z, const double *lam, const double *q_star,
                        const double *f, const double *x_S, const double *x_T, double *s_red)
{
    const int N = td.N;
    const double h = z[0] / N;
    double acc = 0.0;
    // defects and end states: rho/2 (c + lam/rho)^2
    for (int e = threadIdx.x; e < NX * (N + 2); e += blockDim.x) {
        const int k = e / NX, i = e - k * NX;
        double c;
        if (k < N) {
            const double *w0 = z + 1 + (size_t)k * NW, *w1 = w0 + NW;
            c = w1[i] - w0[i] - 0.5 * h * (f[(size_t)k * NX + i] + f[(size_t)(k + 1) * NX + i]);
        } else if (k == N) {
            c = z[1 + i] - x_S[i];
        } else {
            c = z[1 + (size_t)N * NW + i] - x_T[i];
        }
        const double t = c + lam[e] / td.rho;
        acc += 0.5 * td.rho * t * t;
    }
    // effort, tracking and bounds per grid point
    for (int e = threadIdx.x; e < (N + 1) * NW; e += blockDim.x) {
        const int k = e / NW, i = e - k * NW;
        const double v = z[1 + e];
        if (i < NX) {
            const double lo = td.x_min[i], hi = td.x_max[i];
            const double viol = v > hi ? v - hi : (v < lo ? v - lo : 0.0);
            acc += 0.5 * td.rho_b * viol * viol;
            if (i < 4 && k >= 1) {
                const double dq = v - q_star[(size_t)k * 4 + i];
                acc += td.omega_t * dq * dq;
            }
        } else if (k >= 1) {
            acc += td.omega_s * td.R[i - NX] * v * v;
        }
    }
    return z[0] + block_sum(acc, s_red);
}

// The damped Gauss-Newton step dz at z (T6): Jacobian, assembly, block factorisation, solve.
__device__ void lm_step(const TrajDev &td, const double *z, const double *lam, const double *q_star,
                        const double *x_S, const double *x_T, double mu, const TrajWs &ws, double *dz,
                        double *s_red, double *s_blk)
{
    const int N = td.N, t = threadIdx.x;
    const double h = z[0] / N, rho = td.rho;
    // 1. f and df/dw at every grid point (16 forward-mode passes each)
    eval_f(td, z, ws.f);
    for (int e = t; e < (N + 1) * NW; e += blockDim.x) {
        const int k = e / NW, j = e - k * NW;
        const double *w = z + 1 + (size_t)k * NW;
        Dual x[NX], u[NU], out[NX];
        for (int i = 0; i < NX; ++i) x[i] = {w[i], i == j ? 1.0 : 0.0};
        for (int i = 0; i < NU; ++i) u[i] = {w[NX + i], NX + i == j ? 1.0 : 0.0};
        traj_f<Dual>(td, x, u, out);
        for (int i = 0; i < NX; ++i) ws.Fj[((size_t)k * NX + i) * NW + j] = out[i].d;
    }
    __syncthreads();
    // 2. assembly. Defect k: d_k = x_{k+1} - x_k - h/2 (f_k + f_{k+1}), rows scaled by sqrt(rho):
    //    A_k = dd_k/dw_k = -[I 0] - h/2 Fj_k, B_k = dd_k/dw_{k+1} = [I 0] - h/2 Fj_{k+1},
    //    e_k = dd_k/dt_F = -(f_k + f_{k+1}) / (2N); residual sqrt(rho) (d_k + lam_k / rho).
    auto Aent = [&](int k, int r, int i) -> double {   // A_k[r][i]
        return (i == r ? -1.0 : 0.0) - 0.5 * h * ws.Fj[((size_t)k * NX + r) * NW + i];
    };
    auto Bent = [&](int k, int r, int i) -> double {   // B_k[r][i] (defect k, w_{k+1})
        return (i == r ? 1.0 : 0.0) - 0.5 * h * ws.Fj[((size_t)(k + 1) * NX + r) * NW + i];
    };
    auto dres = [&](int k, int r) -> double {          // d_k[r] + lam_k[r] / rho
        const double *w0 = z + 1 + (size_t)k * NW;
        return w0[NW + r] - w0[r] - 0.5 * h * (ws.f[(size_t)k * NX + r] + ws.f[(size_t)(k + 1) * NX + r]) +
               lam[(size_t)k * NX + r] / rho;
    };
    auto eres = [&](int k, int r) -> double { return -(ws.f[(size_t)k * NX + r] + ws.f[(size_t)(k + 1) * NX + r]) / (2.0 * N); };
    // Diagonal blocks (lower triangles) and off-diagonal blocks from F_k = df/dw at grid
    // point k (c = h/2, I' = [I 0] of 12 x 16): A_k = -(I' + c F_k), B_k = I' - c F_{k+1}, so
    //   A_k^T A_k = I'^T I' + c (I'^T F_k + F_k^T I') + c^2 F_k^T F_k,
    //   B_{k-1}^T B_{k-1} = I'^T I' - c (I'^T F_k + F_k^T I') + c^2 F_k^T F_k
    // (interior points take both, whose first-order terms cancel) and
    //   A_k^T B_k = -(I'^T I' - c I'^T F_{k+1} + c F_k^T I' - c^2 F_k^T F_{k+1}).
    const double c = 0.5 * h;
    auto Fjv = [&](int k, int r, int i) -> double { return ws.Fj[((size_t)k * NX + r) * NW + i]; };
    for (int e = t; e < (N + 1) * NW * NW; e += blockDim.x) {
        const int k = e / (NW * NW), ij = e - k * NW * NW, i = ij / NW, j = ij - i * NW;
        if (j > i) continue;   // the factorisation reads the lower triangle only
        double f0 = 0.0, f1 = 0.0;
        for (int r = 0; r < NX; r += 2) {
            f0 = fma(Fjv(k, r, i), Fjv(k, r, j), f0);
            f1 = fma(Fjv(k, r + 1, i), Fjv(k, r + 1, j), f1);
        }
        const double ff = f0 + f1;
        const double cross = (i < NX ? Fjv(k, i, j) : 0.0) + (j < NX ? Fjv(k, j, i) : 0.0);
        const double id = (i == j && i < NX) ? 1.0 : 0.0;
        double v;
        if (k == 0) v = id + c * cross + c * c * ff;
        else if (k == N) v = id - c * cross + c * c * ff;
        else v = 2.0 * id + 2.0 * c * c * ff;
        v *= rho;
        if (i == j) {
            if ((k == 0 || k == N) && i < NX) v += rho;                      // end states
            if (i < NX) {
                const double x = z[1 + (size_t)k * NW + i];
                if (x > td.x_max[i] || x < td.x_min[i]) v += td.rho_b;        // active bound
                if (i < 4 && k >= 1) v += 2.0 * td.omega_t;                   // tracking
            } else if (k >= 1) {
                v += 2.0 * td.omega_s * td.R[i - NX];                         // effort
            }
            v += mu * (v + 1e-9);                                             // damping
        }
        ws.D[e] = v;
    }
    for (int e = t; e < N * NW * NW; e += blockDim.x) {
        const int k = e / (NW * NW), ij = e - k * NW * NW, i = ij / NW, j = ij - i * NW;
        double p0 = 0.0, p1 = 0.0;
        for (int r = 0; r < NX; r += 2) {
            p0 = fma(Fjv(k, r, i), Fjv(k + 1, r, j), p0);
            p1 = fma(Fjv(k, r + 1, i), Fjv(k + 1, r + 1, j), p1);
        }
        const double id = (i == j && i < NX) ? 1.0 : 0.0;
        const double v = id - c * (i < NX ? Fjv(k + 1, i, j) : 0.0) + c * (j < NX ? Fjv(k, j, i) : 0.0) -
                         c * c * (p0 + p1);
        ws.E[e] = -rho * v;
    }
    // border column, gradient
    for (int e = t; e < (N + 1) * NW; e += blockDim.x) {
        const int k = e / NW, i = e - k * NW;
        double bv = 0.0, gv = 0.0;
        if (k < N)
            for (int r = 0; r < NX; ++r) {
                const double a = Aent(k, r, i);
                bv += a * eres(k, r);
                gv += a * dres(k, r);
            }
        if (k > 0)
            for (int r = 0; r < NX; ++r) {
                const double bb = Bent(k - 1, r, i);
                bv += bb * eres(k - 1, r);
                gv += bb * dres(k - 1, r);
            }
        bv *= rho;
        gv *= rho;
        const double x = z[1 + e];
        if (i < NX) {
            if (k == 0) gv += rho * (x - x_S[i] + lam[(size_t)N * NX + i] / rho);
            if (k == N) gv += rho * (x - x_T[i] + lam[(size_t)(N + 1) * NX + i] / rho);
            const double viol = x > td.x_max[i] ? x - td.x_max[i] : (x < td.x_min[i] ? x - td.x_min[i] : 0.0);
            gv += td.rho_b * viol;
            if (i < 4 && k >= 1) gv += 2.0 * td.omega_t * (x - q_star[(size_t)k * 4 + i]);
        } else if (k >= 1) {
            gv += 2.0 * td.omega_s * td.R[i - NX] * x;
        }
        ws.bb[e] = bv;
        ws.g[e] = gv;
    }
    // the t_F corner and gradient
    double cc = 0.0, gt = 0.0;
    for (int e = t; e < N * NX; e += blockDim.x) {
        const int k = e / NX, r = e - k * NX;
        const double ev = eres(k, r);
        cc += ev * ev;
        gt += ev * dres(k, r);
    }
    cc = rho * block_sum(cc, s_red);
    gt = 1.0 + rho * block_sum(gt, s_red);
    cc += mu * (cc + 1e-9);
    __syncthreads();
    // 3. block Cholesky of the tridiagonal part, forward substitution of the border column
    //    (y) and the negated gradient (v): for k = 0..N
    //      S_k = D_k - M_{k-1}^T M_{k-1};  L_k L_k^T = S_k;  M_k = L_k^-1 E_k;
    //      y_k = L_k^-1 (b_k - M_{k-1}^T y_{k-1});  v_k = L_k^-1 (-g_k - M_{k-1}^T v_{k-1}).
    //    The chain of the sweep is long dependent FP64 work, so every step keeps it short: the
    //    16 x 16 factor runs on one warp in registers (lane i holds row i; the pivot's
    //    reciprocal square root by rsqrt_pivot, the column scaled by it, the trailing rows
    //    updated from shuffled column entries), and the triangular solves go column by
    //    column with one lane per right-hand side. The stored factor keeps 1 / L_pp on its
    //    diagonal for the back substitution.
    double *Ls = s_blk;           // the current block: S_k, then its factor
    double *s_vec = s_red + 8;    // [2][NW] right-hand sides of y_k and v_k
    const unsigned full = 0xffffffffu;
    for (int k = 0; k <= N; ++k) {
        double *Dk = ws.D + (size_t)k * NW * NW;
        const double *Mp = ws.E + (size_t)(k > 0 ? k - 1 : 0) * NW * NW;   // M_{k-1}
        for (int ij = t; ij < NW * NW; ij += blockDim.x) {
            const int i = ij / NW, j = ij - i * NW;
            if (j > i) continue;
            double v0 = Dk[ij], v1 = 0.0;
            if (k > 0)
                for (int r = 0; r < NW; r += 2) {
                    v0 = fma(-Mp[r * NW + i], Mp[r * NW + j], v0);
                    v1 = fma(-Mp[(r + 1) * NW + i], Mp[(r + 1) * NW + j], v1);
                }
            Ls[ij] = v0 + v1;
        }
        if (t >= 32 && t < 64) {   // warp 1: the right-hand sides (lanes 0-15 y, 16-31 v)
            const int r = t & 15, which = (t - 32) >> 4;
            const double *prev = (which ? ws.g : ws.bb) + (size_t)(k > 0 ? k - 1 : 0) * NW;
            double v = which ? -ws.g[(size_t)k * NW + r] : ws.bb[(size_t)k * NW + r];
            if (k > 0)
                for (int q = 0; q < NW; ++q) v = fma(-Mp[q * NW + r], prev[q], v);
            s_vec[which * NW + r] = v;
        }
        __syncthreads();
        if (t < 32) {   // warp 0: the factor
            const int i = t & (NW - 1);
            double a[NW], rin[NW];
#pragma unroll
            for (int j = 0; j < NW; ++j) a[j] = j <= i ? Ls[i * NW + j] : 0.0;
#pragma unroll
            for (int p = 0; p < NW; ++p) {
                const double d = __shfl_sync(full, a[p], p);   // the pivot, from lane p
                const double r = rsqrt_pivot(d);
                rin[p] = r;
                const double l = i > p ? a[p] * r : (i == p ? d * r : 0.0);   // L[i][p]
                a[p] = l;
#pragma unroll
                for (int j = p + 1; j < NW; ++j) {
                    const double lj = __shfl_sync(full, l, j);                // L[j][p]
                    if (j <= i) a[j] = fma(-l, lj, a[j]);
                }
            }
            if (t < NW) {
#pragma unroll
                for (int j = 0; j < NW; ++j) Ls[i * NW + j] = j < i ? a[j] : (j == i ? rin[i] : 0.0);
            }
            __syncwarp();
            // M_k = L^-1 E_k (lanes 0-15, one column each) and the two vectors (lanes 16, 17)
            const bool col = t < NW && k < N, vec = t == 16 || t == 17;
            if (col || vec) {
                const double *Ek = ws.E + (size_t)k * NW * NW;
                double x[NW];
#pragma unroll
                for (int r = 0; r < NW; ++r) x[r] = col ? Ek[r * NW + t] : s_vec[(t - 16) * NW + r];
#pragma unroll
                for (int q = 0; q < NW; ++q) {
                    x[q] *= Ls[q * NW + q];
#pragma unroll
                    for (int r = q + 1; r < NW; ++r) x[r] = fma(-Ls[r * NW + q], x[q], x[r]);
                }
                double *dst = col ? ws.E + (size_t)k * NW * NW : (t == 16 ? ws.bb : ws.g) + (size_t)k * NW;
#pragma unroll
                for (int r = 0; r < NW; ++r) dst[col ? r * NW + t : r] = x[r];
            }
        }
        __syncthreads();
        for (int ij = t; ij < NW * NW; ij += blockDim.x) Dk[ij] = Ls[ij];
    }
    __syncthreads();
    // back substitution: y_k = L_k^-T (y_k - M_k y_{k+1}), the same for v (warp 0: lanes 0-15
    // y, 16-31 v, one row each; L_k^T x = rhs solved from the last row up, column by column)
    for (int k = N; k >= 0; --k) {
        if (t < 32) {
            const int r = t & (NW - 1), which = t >> 4;
            double *vec = (which ? ws.g : ws.bb) + (size_t)k * NW;
            const double *Lk = ws.D + (size_t)k * NW * NW;
            double x = vec[r];
            if (k < N) {
                const double *M = ws.E + (size_t)k * NW * NW;
                const double *nxt = (which ? ws.g : ws.bb) + (size_t)(k + 1) * NW;
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                for (int q = 0; q < NW; q += 4) {
                    s0 = fma(M[r * NW + q], nxt[q], s0);
                    s1 = fma(M[r * NW + q + 1], nxt[q + 1], s1);
                    s2 = fma(M[r * NW + q + 2], nxt[q + 2], s2);
                    s3 = fma(M[r * NW + q + 3], nxt[q + 3], s3);
                }
                x -= (s0 + s1) + (s2 + s3);
            }
#pragma unroll
            for (int rr = NW - 1; rr >= 0; --rr) {
                const double lrr = Lk[rr * NW + rr];     // 1 / L_rr
                const double lrq = Lk[rr * NW + r];      // L[rr][r] (r < rr)
                const double xr = __shfl_sync(full, x * lrr, rr + NW * which);
                if (r == rr) x = xr;
                else if (r < rr) x = fma(-lrq, xr, x);
            }
            __syncwarp();
            vec[r] = x;
        }
        __syncthreads();
    }
    // 4. the border: dt = (-g_t - b^T v) / (c - b^T y), dw = v - y dt, with y = T^-1 b and
    //    v = T^-1 (-g_w) (b the original border column, kept in the factor-free terms above:
    //    b^T y and b^T v are recomputed from y and v through T y = b, i.e. b^T y = y^T T y).
    //    T y = b and T v = -g hold, so b^T y = sum_k b_k . y_k needs the original b: it is
    //    re-derived here from its definition.
    double by = 0.0, bv = 0.0;
    for (int e = t; e < (N + 1) * NW; e += blockDim.x) {
        const int k = e / NW, i = e - k * NW;
        double b = 0.0;
        if (k < N)
            for (int r = 0; r < NX; ++r) b += Aent(k, r, i) * eres(k, r);
        if (k > 0)
            for (int r = 0; r < NX; ++r) b += Bent(k - 1, r, i) * eres(k - 1, r);
        b *= rho;
        by += b * ws.bb[e];
        bv += b * ws.g[e];
    }
    by = block_sum(by, s_red);
    bv = block_sum(bv, s_red);
    const double dt = (-gt - bv) / (cc - by);
    if (t == 0) dz[0] = dt;
    for (int e = t; e < (N + 1) * NW; e += blockDim.x) dz[1 + e] = ws.g[e] - ws.bb[e] * dt;
    __syncthreads();
}

// One LM step for each trajectory (a test of the step): dz at (z, lam, mu).
__global__ void __launch_bounds__(kTrajThreads)
k_traj_step(const TrajDev td, const double *q_star, const double *z, const double *lam, double mu, double *ws_base,
            size_t ws_stride, double *dz)
{
    extern __shared__ double s_mem[];
    const int N = td.N, n_var = 1 + NW * (N + 1), n_eq = NX * (N + 2);
    const int p = blockIdx.x;
    double *s_red = s_mem;                  // 8 + 2 NW
    double *s_blk = s_red + 8 + 2 * NW;     // NW * NW
    double *x_S = s_blk + NW * NW, *x_T = x_S + NX;
    const double *qs = q_star + (size_t)p * (N + 1) * 4;
    for (int i = threadIdx.x; i < NX; i += blockDim.x) {
        x_S[i] = i < 4 ? qs[i] : 0.0;
        x_T[i] = i < 4 ? qs[(size_t)N * 4 + i] : 0.0;
    }
    __syncthreads();
    const TrajWs ws = ws_of(ws_base + (size_t)p * ws_stride, N);
    lm_step(td, z + (size_t)p * n_var, lam + (size_t)p * n_eq, qs, x_S, x_T, mu, ws, dz + (size_t)p * n_var, s_red,
            s_blk);
}

// The whole solve (T6) for each trajectory: z in place; stats {t_F, F, max |c|, max bound
// violation}.
__global__ void __launch_bounds__(kTrajThreads)
k_traj_solve(const TrajDev td, const double *q_star, double *z_io, double *ws_base, size_t ws_stride, double *lam_ws,
             double *stats)
{
    extern __shared__ double s_mem[];
    const int N = td.N, n_var = 1 + NW * (N + 1), n_eq = NX * (N + 2);
    const int p = blockIdx.x, t = threadIdx.x;
    double *s_red = s_mem;
    double *s_blk = s_red + 8 + 2 * NW;
    double *x_S = s_blk + NW * NW, *x_T = x_S + NX;
    double *z = x_T + NX;          // n_var
    double *zn = z + n_var;        // n_var
    double *dz = zn + n_var;       // n_var
    double *lam = lam_ws + (size_t)p * n_eq;
    const double *qs = q_star + (size_t)p * (N + 1) * 4;
    for (int i = t; i < NX; i += blockDim.x) {
        x_S[i] = i < 4 ? qs[i] : 0.0;
        x_T[i] = i < 4 ? qs[(size_t)N * 4 + i] : 0.0;
    }
    for (int i = t; i < n_var; i += blockDim.x) z[i] = z_io[(size_t)p * n_var + i];
    for (int i = t; i < n_eq; i += blockDim.x) lam[i] = 0.0;
    __syncthreads();
    const TrajWs ws = ws_of(ws_base + (size_t)p * ws_stride, N);
    double mu = td.mu0;
    for (int o = 0; o < td.outer; ++o) {
        eval_f(td, z, ws.f);
        __syncthreads();
        double F = merit(td, z, lam, qs, ws.f, x_S, x_T, s_red);
        for (int it = 0; it < td.inner; ++it) {
            lm_step(td, z, lam, qs, x_S, x_T, mu, ws, dz, s_red, s_blk);
            for (int i = t; i < n_var; i += blockDim.x) zn[i] = z[i] + dz[i];
            __syncthreads();
            eval_f(td, zn, ws.f);
            __syncthreads();
            const double Fn = merit(td, zn, lam, qs, ws.f, x_S, x_T, s_red);
            if (Fn < F) {
                for (int i = t; i < n_var; i += blockDim.x) z[i] = zn[i];
                F = Fn;
                mu = fmax(mu / 3.0, 1e-12);
            } else {
                mu = fmin(mu * 4.0, 1e12);
            }
            __syncthreads();
        }
        // multipliers: lam += rho c(z)
        eval_f(td, z, ws.f);
        __syncthreads();
        const double h = z[0] / N;
        for (int e = t; e < n_eq; e += blockDim.x) {
            const int k = e / NX, i = e - k * NX;
            double c;
            if (k < N) c = z[1 + (size_t)(k + 1) * NW + i] - z[1 + (size_t)k * NW + i] -
                           0.5 * h * (ws.f[(size_t)k * NX + i] + ws.f[(size_t)(k + 1) * NX + i]);
            else if (k == N) c = z[1 + i] - x_S[i];
            else c = z[1 + (size_t)N * NW + i] - x_T[i];
            lam[e] += td.rho * c;
        }
        __syncthreads();
    }
    // results and statistics
    for (int i = t; i < n_var; i += blockDim.x) z_io[(size_t)p * n_var + i] = z[i];
    eval_f(td, z, ws.f);
    __syncthreads();
    double cmax = 0.0, vmax = 0.0;
    const double h = z[0] / N;
    for (int e = t; e < n_eq; e += blockDim.x) {
        const int k = e / NX, i = e - k * NX;
        double c;
        if (k < N) c = z[1 + (size_t)(k + 1) * NW + i] - z[1 + (size_t)k * NW + i] -
                       0.5 * h * (ws.f[(size_t)k * NX + i] + ws.f[(size_t)(k + 1) * NX + i]);
        else if (k == N) c = z[1 + i] - x_S[i];
        else c = z[1 + (size_t)N * NW + i] - x_T[i];
        cmax = fmax(cmax, fabs(c));
    }
    for (int e = t; e < (N + 1) * NW; e += blockDim.x) {
        const int i = e % NW;
        if (i < NX) {
            const double x = z[1 + e];
            vmax = fmax(vmax, fmax(x - td.x_max[i], td.x_min[i] - x));
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        cmax = fmax(cmax, __shfl_down_sync(0xffffffffu, cmax, off));
        vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, off));
    }
    __syncthreads();
    if ((t & 31) == 0) {
        s_red[t >> 5] = cmax;
        s_red[8 + (t >> 5)] = vmax;
    }
    __syncthreads();
    if (t == 0) {
        double c = 0.0, v = 0.0;
        for (int i = 0; i < kTrajThreads / 32; ++i) {
            c = fmax(c, s_red[i]);
            v = fmax(v, s_red[8 + i]);
        }
        stats[(size_t)p * 4 + 2] = c;
        stats[(size_t)p * 4 + 3] = fmax(v, 0.0);
    }
    __syncthreads();
    const double Fend = merit(td, z, lam, qs, ws.f, x_S, x_T, s_red);
    if (t == 0) {
        stats[(size_t)p * 4 + 0] = z[0];
        stats[(size_t)p * 4 + 1] = Fend;
    }
}

// q*(k / N) of cubic B-spline paths with control points ctrl[n][K+8][4] on the moving spans
// (tau = 4 + (K+3) s on uniform knots, the path step's reading), by the uniform cubic basis
// of the span that holds tau (s = 1 falls on the last moving span at u = 1).
__global__ void k_traj_targets(const double *ctrl, int K, int n, int N, double *q_star)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * (N + 1)) return;
    const int p = e / (N + 1), k = e - p * (N + 1);
    const double tau = 4.0 + (double)(K + 3) * ((double)k / (double)N);
    int span = (int)floor(tau);
    if (span > K + 6) span = K + 6;        // s = 1: u = 1 on the last moving span
    const double u = tau - span, v = 1.0 - u;
    const double b0 = v * v * v / 6.0, b1 = (3.0 * u * u * u - 6.0 * u * u + 4.0) / 6.0;
    const double b2 = (-3.0 * u * u * u + 3.0 * u * u + 3.0 * u + 1.0) / 6.0, b3 = u * u * u / 6.0;
    const double *P = ctrl + (size_t)p * (K + 8) * 4 + (size_t)(span - 3) * 4;
    for (int j = 0; j < 4; ++j)
        q_star[(size_t)e * 4 + j] = b0 * P[j] + b1 * P[4 + j] + b2 * P[8 + j] + b3 * P[12 + j];
}

// The initial guess of T6 from the targets: q_a = q*_k, dq by central differences over t_F,
// u by second differences, the swing at rest; t_F = 1.5 x the slowest joint's total variation
// over its velocity limit.
__global__ void k_traj_initial(const TrajDev td, const double *dq_max, const double *q_star, int n, double *z)
{
    const int p = blockIdx.x, N = td.N, n_var = 1 + NW * (N + 1);
    if (p >= n) return;
    const double *qs = q_star + (size_t)p * (N + 1) * 4;
    __shared__ double s_tF;
    if (threadIdx.x == 0) {
        double tf = 0.0;
        for (int j = 0; j < 4; ++j) {
            double tv = 0.0;
            for (int k = 0; k < N; ++k) tv += fabs(qs[(size_t)(k + 1) * 4 + j] - qs[(size_t)k * 4 + j]);
            tf = fmax(tf, 1.5 * tv / dq_max[j]);
        }
        s_tF = fmax(tf, 1e-3);
    }
    __syncthreads();
    const double tF = s_tF, h = tF / N;
    double *zp = z + (size_t)p * n_var;
    if (threadIdx.x == 0) zp[0] = tF;
    for (int e = threadIdx.x; e < (N + 1) * NW; e += blockDim.x) {
        const int k = e / NW, i = e - k * NW;
        double v = 0.0;
        if (i < 4) v = qs[(size_t)k * 4 + i];
        else if (i >= 6 && i < 10 && k > 0 && k < N)
            v = (qs[(size_t)(k + 1) * 4 + i - 6] - qs[(size_t)(k - 1) * 4 + i - 6]) / (2.0 * h);
        else if (i >= NX && k > 0 && k < N)
            v = (qs[(size_t)(k + 1) * 4 + i - NX] - 2.0 * qs[(size_t)k * 4 + i - NX] + qs[(size_t)(k - 1) * 4 + i - NX]) /
                (h * h);
        zp[1 + e] = v;
    }
}

}  // namespace
}  // namespace cp

using namespace cp;

struct cp_traj {
    cudaStream_t st = nullptr;
    TrajDev td{};
    int max_paths = 0;
    size_t ws_stride = 0;   // doubles per trajectory
    double *ws = nullptr, *lam = nullptr, *dq_max = nullptr;
};

namespace {

size_t traj_ws_doubles(int N)
{
    return (size_t)(N + 1) * (NX + NX * NW + NW * NW + 2 * NW) + (size_t)N * NW * NW;
}

size_t traj_smem(int N, bool solve)
{
    const size_t base = 8 + 2 * NW + NW * NW + 2 * NX;
    return sizeof(double) * (base + (solve ? 3 * (size_t)(1 + NW * (N + 1)) : 0));
}

}  // namespace

extern "C" {

int cp_traj_init(const cp_model *model, const cp_traj_params *tp, int32_t max_paths, void *stream, cp_traj **out)
{
    if (!out) return set_error("out is NULL"), CP_ERR_ARG;
    *out = nullptr;
    int rc = validate_model(model);
    if (rc != CP_OK) return rc;
    if (!tp) return set_error("params is NULL"), CP_ERR_ARG;
    if (tp->N < 2 || tp->N > 255) return set_error("N %d outside 2..255", tp->N), CP_ERR_ARG;
    if (max_paths < 1) return set_error("max_paths must be >= 1"), CP_ERR_ARG;
    if (tp->outer < 0 || tp->inner < 0) return set_error("outer and inner must be >= 0"), CP_ERR_ARG;
    if (!(tp->grapple_len > 0.0) || !(tp->rho > 0.0) || !(tp->rho_b >= 0.0) || !(tp->mu0 > 0.0) ||
        !(tp->omega_s >= 0.0) || !(tp->omega_t >= 0.0) || !(tp->swing_max > 0.0) || tp->swing_max >= 1.5)
        return set_error("trajectory weights and limits out of range"), CP_ERR_ARG;
    for (int j = 0; j < 4; ++j)
        if (!(tp->dq_max[j] > 0.0) || !(tp->R[j] >= 0.0)) return set_error("dq_max must be > 0, R >= 0"), CP_ERR_ARG;
    if (traj_smem(tp->N, true) > 227 * 1024) return set_error("N too large for the solver's shared memory"), CP_ERR_ARG;
    cp_traj *t = new (std::nothrow) cp_traj();
    if (!t) return set_error("host allocation failed"), CP_ERR_OOM;
    t->st = (cudaStream_t)stream;
    TrajDev &d = t->td;
    d.base_z = model->base_z;
    d.boom_len = model->boom_len;
    d.jib_len = model->jib_len;
    d.ell = tp->grapple_len;
    d.omega_s = tp->omega_s;
    d.omega_t = tp->omega_t;
    for (int j = 0; j < 4; ++j) d.R[j] = tp->R[j];
    for (int j = 0; j < 4; ++j) {
        d.x_min[j] = model->q_min[j];
        d.x_max[j] = model->q_max[j];
        d.x_min[6 + j] = -tp->dq_max[j];
        d.x_max[6 + j] = tp->dq_max[j];
    }
    d.x_min[4] = d.x_min[5] = -tp->swing_max;
    d.x_max[4] = d.x_max[5] = tp->swing_max;
    d.x_min[10] = d.x_min[11] = -1e30;
    d.x_max[10] = d.x_max[11] = 1e30;
    d.rho = tp->rho;
    d.rho_b = tp->rho_b;
    d.mu0 = tp->mu0;
    d.N = tp->N;
    d.outer = tp->outer;
    d.inner = tp->inner;
    t->max_paths = max_paths;
    t->ws_stride = (traj_ws_doubles(tp->N) + 31) & ~(size_t)31;
    const size_t n_eq = (size_t)NX * (tp->N + 2);
    const size_t bytes = sizeof(double) * (t->ws_stride * max_paths + n_eq * max_paths + 4);
    cudaError_t e = cudaMalloc((void **)&t->ws, bytes);
    if (e != cudaSuccess) {
        delete t;
        return cuda_fail(e, "cudaMalloc(trajectory workspace)");
    }
    t->lam = t->ws + t->ws_stride * max_paths;
    t->dq_max = t->lam + n_eq * max_paths;
    e = cudaMemcpyAsync(t->dq_max, tp->dq_max, sizeof(double) * 4, cudaMemcpyHostToDevice, t->st);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_traj_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)traj_smem(tp->N, true));
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->st);
    if (e != cudaSuccess) {
        cudaFree(t->ws);
        delete t;
        return cuda_fail(e, "trajectory solver set-up");
    }
    *out = t;
    return CP_OK;
}

void cp_traj_destroy(cp_traj *t)
{
    if (!t) return;
    cudaStreamSynchronize(t->st);
    cudaFree(t->ws);
    delete t;
}

int cp_traj_targets(cp_traj *t, const double *d_ctrl, int32_t K, int32_t n, double *d_q_star)
{
    if (!t) return set_error("solver is NULL"), CP_ERR_ARG;
    if (K < 1 || K > CP_MAX_WAYPOINTS || n < 0) return set_error("K or n out of range"), CP_ERR_ARG;
    if (n > 0 && (!d_ctrl || !d_q_star)) return set_error("NULL argument"), CP_ERR_ARG;
    if (n == 0) return CP_OK;
    const int total = n * (t->td.N + 1);
    k_traj_targets<<<(total + 127) / 128, 128, 0, t->st>>>(d_ctrl, K, n, t->td.N, d_q_star);
    CP_LAUNCHED("k_traj_targets");
    return CP_OK;
}

int cp_traj_initial_guess(cp_traj *t, const double *d_q_star, int32_t n, double *d_z)
{
    if (!t) return set_error("solver is NULL"), CP_ERR_ARG;
    if (n < 0 || n > t->max_paths) return set_error("n = %d outside 0..%d", n, t->max_paths), CP_ERR_ARG;
    if (n > 0 && (!d_q_star || !d_z)) return set_error("NULL argument"), CP_ERR_ARG;
    if (n == 0) return CP_OK;
    k_traj_initial<<<n, 128, 0, t->st>>>(t->td, t->dq_max, d_q_star, n, d_z);
    CP_LAUNCHED("k_traj_initial");
    return CP_OK;
}

int cp_traj_step(cp_traj *t, const double *d_q_star, int32_t n, const double *d_z, const double *d_lam, double mu,
                 double *d_dz)
{
    const NvtxScope range("craneplan:traj_step");
    if (!t) return set_error("solver is NULL"), CP_ERR_ARG;
    if (n < 0 || n > t->max_paths) return set_error("n = %d outside 0..%d", n, t->max_paths), CP_ERR_ARG;
    if (n > 0 && (!d_q_star || !d_z || !d_lam || !d_dz)) return set_error("NULL argument"), CP_ERR_ARG;
    if (!(mu >= 0.0)) return set_error("mu must be >= 0"), CP_ERR_ARG;
    if (n == 0) return CP_OK;
    k_traj_step<<<n, kTrajThreads, traj_smem(t->td.N, false), t->st>>>(t->td, d_q_star, d_z, d_lam, mu, t->ws,
                                                                     t->ws_stride, d_dz);
    CP_LAUNCHED("k_traj_step");
    return CP_OK;
}

int cp_traj_solve(cp_traj *t, const double *d_q_star, int32_t n, double *d_z, double *d_stats)
{
    const NvtxScope range("craneplan:traj_solve");
    if (!t) return set_error("solver is NULL"), CP_ERR_ARG;
    if (n < 0 || n > t->max_paths) return set_error("n = %d outside 0..%d", n, t->max_paths), CP_ERR_ARG;
    if (n > 0 && (!d_q_star || !d_z || !d_stats)) return set_error("NULL argument"), CP_ERR_ARG;
    if (n == 0) return CP_OK;
    k_traj_solve<<<n, kTrajThreads, traj_smem(t->td.N, true), t->st>>>(t->td, d_q_star, d_z, t->ws, t->ws_stride,
                                                                      t->lam, d_stats);
    CP_LAUNCHED("k_traj_solve");
    return CP_OK;
}

}  // extern "C"

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
// differentiation (value and one derivative per pass, 16 passes). Everything is FP64: a
// cluster of two CTAs of 512 threads per trajectory.
#include <cmath>
#include <new>

#include <cooperative_groups.h>
#include <nvtx3/nvToolsExt.h>

#include "cp_internal.cuh"

// An NVTX range over a scope (no-op without a profiling tool).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

namespace cp {
namespace {

constexpr int kTrajThreads = 512;
constexpr int kTrajCtas = 2;      // CTAs (one thread-block cluster) per trajectory
constexpr int kRedDoubles = 64;   // block reductions: [0, 32) and [32, 64) (one slot per warp)
constexpr int kWarpScratch = 2 * 12 * 16;   // doubles of shared memory per warp (block factor, F_k pair)
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
template <typename T> __device__ __forceinline__ T lift(double v);
template <> __device__ __forceinline__ double lift<double>(double v) { return v; }
template <> __device__ __forceinline__ Dual lift<Dual>(double v) { return {v, 0.0}; }

// Cosine and sine of an angle of the dynamics. The primal values depend on the grid point
// only, so a cache (c, s pairs written by the value pass at that point) serves the 16
// derivative passes; without one (or for plain doubles) they are computed here.
__device__ __forceinline__ void trig_of(double a, const double *cache, double *cw, int idx, double &c, double &s)
{
    if (cache != nullptr) {
        c = cache[2 * idx];
        s = cache[2 * idx + 1];
        return;
    }
    sincos(a, &s, &c);
    if (cw != nullptr) {
        cw[2 * idx] = c;
        cw[2 * idx + 1] = s;
    }
}

__device__ __forceinline__ void trig_of(Dual a, const double *cache, double *cw, int idx, Dual &c, Dual &s)
{
    double cv, sv;
    if (cache != nullptr) {
        cv = cache[2 * idx];
        sv = cache[2 * idx + 1];
    } else {
        sincos(a.v, &sv, &cv);
    }
    (void)cw;
    c = {cv, -sv * a.d};
    s = {sv, cv * a.d};
}

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
// cache: the cosines and sines of this grid point (A, B, q1, alpha, beta) when known; cw: where
// the value pass stores them (either may be null).
template <typename T>
__device__ void traj_f(const TrajDev &td, const T *x, const T *u, T *out, const double *cache = nullptr,
                       double *cw = nullptr)
{
    const T q1 = x[0], q2 = x[1], q3 = x[2], q4 = x[3], a = x[4], b = x[5];
    const T d1 = x[6], d2 = x[7], d3 = x[8], d4 = x[9], da = x[10], db = x[11];
    const T u1 = u[0], u2 = u[1], u3 = u[2], u4 = u[3];
    const T lam = lift<T>(td.jib_len) + q4;
    const T A = q2, B = q2 + q3, dB = d2 + d3, ddB = u2 + u3;
    T cA, sA, cB, sB;
    trig_of(A, cache, cw, 0, cA, sA);
    trig_of(B, cache, cw, 1, cB, sB);
    const T h = td.boom_len * cA + lam * cB;
    const T dh = lift<T>(0.0) - td.boom_len * sA * d2 + d4 * cB - lam * sB * dB;
    const T ddh = lift<T>(0.0) - td.boom_len * (cA * d2 * d2 + sA * u2) + u4 * cB - 2.0 * d4 * sB * dB -
                  lam * (cB * dB * dB + sB * ddB);
    const T ddz = td.boom_len * (cA * u2 - sA * d2 * d2) + u4 * sB + 2.0 * d4 * cB * dB +
                  lam * (cB * ddB - sB * dB * dB);
    const T a_r = ddh - h * d1 * d1, a_t = h * u1 + 2.0 * dh * d1;
    T c1, s1;
    trig_of(q1, cache, cw, 2, c1, s1);
    const T ax = a_r * c1 - a_t * s1, ay = a_r * s1 + a_t * c1;
    T ca, sa, cb, sb;
    trig_of(a, cache, cw, 3, ca, sa);
    trig_of(b, cache, cw, 4, cb, sb);
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
    double *P;     // [N+1][16][16] L_k^-1 T[k][left neighbour] of the eliminated blocks
    double *trig;  // [N+1][10] cosines and sines of the dynamics at the grid points of z
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
    w.P = w.g + (size_t)(N + 1) * NW;
    w.trig = w.P + (size_t)(N + 1) * NW * NW;
    return w;
}

// The CTAs of one trajectory: a cluster of kTrajCtas CTAs on neighbouring SMs. Grid points,
// entries and blocks are split over the team-wide thread or warp index. Data one CTA writes to
// the trajectory's global workspace is read by the other only after team_sync(), a cluster
// barrier with release / acquire semantics. Every thread of both CTAs passes the same
// sequence of them: no barrier sits under a branch whose condition the CTAs could see
// differently (the sums below give both the same values).
struct Team {
    int rank;   // this CTA's rank in the cluster
    __device__ int tid() const { return rank * (int)blockDim.x + (int)threadIdx.x; }
    __device__ int nthreads() const { return kTrajCtas * (int)blockDim.x; }
    __device__ int warp() const { return tid() >> 5; }
    __device__ int nwarps() const { return nthreads() >> 5; }
};

__device__ __forceinline__ Team team_of_block()
{
    return Team{(int)cooperative_groups::this_cluster().block_rank()};
}

__device__ __forceinline__ void team_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Sums of a and b over both CTAs in a fixed order: per warp by shuffles, a CTA's warps in
// order by its thread 0, then CTA 0's partial plus CTA 1's (read from each CTA's shared
// memory), so every thread of both CTAs returns the same values (deterministic).
__device__ double2 team_sum2(double a, double b, double *s_red)
{
    const int t = threadIdx.x;
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    __syncthreads();
    if ((t & 31) == 0) {
        s_red[t >> 5] = a;
        s_red[32 + (t >> 5)] = b;
    }
    __syncthreads();
    if (t == 0) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < kTrajThreads / 32; ++i) {
            sa += s_red[i];
            sb += s_red[32 + i];
        }
        s_red[kRedDoubles - 2] = sa;
        s_red[kRedDoubles - 1] = sb;
    }
    team_sync();   // both CTAs' partials are written
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    const double *p0 = cl.map_shared_rank(s_red + kRedDoubles - 2, 0);
    const double *p1 = cl.map_shared_rank(s_red + kRedDoubles - 2, 1);
    const double2 r = make_double2(p0[0] + p1[0], p0[1] + p1[1]);
    team_sync();   // every thread has read them before either CTA writes s_red again
    return r;
}

__device__ double team_sum(double v, double *s_red) { return team_sum2(v, 0.0, s_red).x; }

// f at every grid point of z (values only) into ws.f, the points split over the team.
// trig (optional): the cosines and sines of every grid point are stored there too.
__device__ void eval_f(const Team &tm, const TrajDev &td, const double *z, double *f, double *trig = nullptr)
{
    for (int k = tm.tid(); k <= td.N; k += tm.nthreads()) {
        const double *w = z + 1 + (size_t)k * NW;
        traj_f<double>(td, w, w + NX, f + (size_t)k * NX, nullptr, trig != nullptr ? trig + (size_t)k * 10 : nullptr);
    }
}

// The merit F(z) = t_F + 1/2 |r(z)|^2 (T6): the AL terms of the defects and end states, the
// effort and tracking sums over k = 1..N, and the bound penalty; f must be current for z.
__device__ double merit(const Team &tm, const TrajDev &td, const double *z, const double *lam, const double *q_star,
                        const double *f, const double *x_S, const double *x_T, double *s_red)
{
    const int N = td.N;
    const double h = z[0] / N;
    double acc = 0.0;
    // defects and end states: rho/2 (c + lam/rho)^2
    for (int e = tm.tid(); e < NX * (N + 2); e += tm.nthreads()) {
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
    for (int e = tm.tid(); e < (N + 1) * NW; e += tm.nthreads()) {
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
    return z[0] + team_sum(acc, s_red);
}

// Cholesky factor of a 16 x 16 SPD block on one warp (all 32 lanes call; lanes 0-15 hold a
// row each in registers): the lower triangle of A in, F = the factor's strict lower triangle
// with 1 / L_pp on its diagonal out (shared memory of the warp). Each pivot's reciprocal square
// root comes from rsqrt_pivot; the column is scaled by it and the trailing rows updated from
// shuffled entries, so a pivot costs one short chain of dependent FP64 operations.
__device__ __noinline__ void warp_factor16(const double *A, double *F, int lane)
{
    const unsigned full = 0xffffffffu;
    const int i = lane & (NW - 1);
    double a[NW], rin[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) a[j] = j <= i ? A[i * NW + j] : 0.0;
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
    if (lane < NW) {
#pragma unroll
        for (int j = 0; j < NW; ++j) F[i * NW + j] = j < i ? a[j] : (j == i ? rin[i] : 0.0);
    }
    __syncwarp();
}

// dst <- L^-1 src for one right-hand side of this lane (entry rr at src[rr * ss], written to
// dst[rr * ds]), L in the form of warp_factor16: column by column, a chain of two dependent
// operations per column.
__device__ __noinline__ void column_solve16(const double *F, const double *src, int ss, double *dst, int ds)
{
    double x[NW];
#pragma unroll
    for (int rr = 0; rr < NW; ++rr) x[rr] = src[rr * ss];
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        x[q] *= F[q * NW + q];
#pragma unroll
        for (int r = q + 1; r < NW; ++r) x[r] = fma(-F[r * NW + q], x[q], x[r]);
    }
#pragma unroll
    for (int rr = 0; rr < NW; ++rr) dst[rr * ds] = x[rr];
}

// x_k = L_k^-T (w_k - P_k x_l - Q_k x_r) for both vectors (lanes 0-15 y, 16-31 v, one row
// each; P or Q absent when null): the products, then L^T x = rhs from the last row up,
// column by column with the solved entry shuffled to the rows above it.
__device__ __noinline__ void warp_back16(const double *Lk, const double *P, const double *xl_y, const double *xl_v,
                            const double *Q, const double *xr_y, const double *xr_v, double *out_y, double *out_v,
                            int lane)
{
    const unsigned full = 0xffffffffu;
    const int r = lane & (NW - 1), which = lane >> 4;
    double *out = which ? out_v : out_y;
    double x = out[r];   // w_k
    if (P != nullptr) {
        const double *xl = which ? xl_v : xl_y;
        double s0 = 0.0, s1 = 0.0;
        for (int c = 0; c < NW; c += 2) {
            s0 = fma(P[r * NW + c], xl[c], s0);
            s1 = fma(P[r * NW + c + 1], xl[c + 1], s1);
        }
        x -= s0 + s1;
    }
    if (Q != nullptr) {
        const double *xr = which ? xr_v : xr_y;
        double s0 = 0.0, s1 = 0.0;
        for (int c = 0; c < NW; c += 2) {
            s0 = fma(Q[r * NW + c], xr[c], s0);
            s1 = fma(Q[r * NW + c + 1], xr[c + 1], s1);
        }
        x -= s0 + s1;
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
    out[r] = x;
    __syncwarp();
}

// The damped Gauss-Newton step dz at z (T6): Jacobian, assembly, block factorisation, solve.
// dz_local: dz is this CTA's shared-memory copy, which gets every entry; otherwise it is one
// global vector whose entries the team splits.
__device__ void lm_step(const Team &tm, const TrajDev &td, const double *z, const double *lam, const double *q_star,
                        const double *x_S, const double *x_T, double mu, const TrajWs &ws, double *dz, bool dz_local,
                        double *s_red, double *s_blk)
{
    const int N = td.N, t = tm.tid(), nt = tm.nthreads();
    const double h = z[0] / N, rho = td.rho;
    // 1. f and df/dw at every grid point (16 forward-mode passes each)
    eval_f(tm, td, z, ws.f, ws.trig);
    team_sync();
    for (int e = t; e < (N + 1) * NW; e += nt) {
        const int k = e / NW, j = e - k * NW;
        const double *w = z + 1 + (size_t)k * NW;
        Dual x[NX], u[NU], out[NX];
        for (int i = 0; i < NX; ++i) x[i] = {w[i], i == j ? 1.0 : 0.0};
        for (int i = 0; i < NU; ++i) u[i] = {w[NX + i], NX + i == j ? 1.0 : 0.0};
        traj_f<Dual>(td, x, u, out, ws.trig + (size_t)k * 10);
        for (int i = 0; i < NX; ++i) ws.Fj[((size_t)k * NX + i) * NW + j] = out[i].d;
    }
    team_sync();
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
    // one warp per grid point k: F_k and F_{k+1} staged in the warp's shared memory, then the
    // 136 lower entries of D_k and the 256 of E_k
    {
        const int warp = tm.warp(), lane = threadIdx.x & 31, n_warps = tm.nwarps();
        double *sF = s_blk + (size_t)(threadIdx.x >> 5) * kWarpScratch;   // [2][NX][NW]: F_k, F_{k+1}
        const double *F0 = sF, *F1 = sF + NX * NW;
        for (int k = warp; k <= N; k += n_warps) {
            __syncwarp();
            for (int q = lane; q < 2 * NX * NW; q += 32)
                sF[q] = (q < NX * NW || k < N) ? ws.Fj[(size_t)k * NX * NW + q] : 0.0;
            __syncwarp();
            for (int e = lane; e < NW * (NW + 1) / 2; e += 32) {
                int i, j;
                tri_index(e, i, j);
                double f0 = 0.0, f1 = 0.0;
                for (int r = 0; r < NX; r += 2) {
                    f0 = fma(F0[r * NW + i], F0[r * NW + j], f0);
                    f1 = fma(F0[(r + 1) * NW + i], F0[(r + 1) * NW + j], f1);
                }
                const double ff = f0 + f1;
                const double cross = (i < NX ? F0[i * NW + j] : 0.0) + (j < NX ? F0[j * NW + i] : 0.0);
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
                ws.D[(size_t)k * NW * NW + i * NW + j] = v;
            }
            if (k < N)
                for (int e = lane; e < NW * NW; e += 32) {
                    const int i = e >> 4, j = e & (NW - 1);
                    double p0 = 0.0, p1 = 0.0;
                    for (int r = 0; r < NX; r += 2) {
                        p0 = fma(F0[r * NW + i], F1[r * NW + j], p0);
                        p1 = fma(F0[(r + 1) * NW + i], F1[(r + 1) * NW + j], p1);
                    }
                    const double id = (i == j && i < NX) ? 1.0 : 0.0;
                    const double v = id - c * (i < NX ? F1[i * NW + j] : 0.0) + c * (j < NX ? F0[j * NW + i] : 0.0) -
                                     c * c * (p0 + p1);
                    ws.E[(size_t)k * NW * NW + e] = -rho * v;
                }
        }
    }
    // border column, gradient (stored negated: the solves below take -g)
    for (int e = t; e < (N + 1) * NW; e += nt) {
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
        ws.g[e] = -gv;
    }
    // the t_F corner and gradient
    double cc = 0.0, gt = 0.0;
    for (int e = t; e < N * NX; e += nt) {
        const int k = e / NX, r = e - k * NX;
        const double ev = eres(k, r);
        cc += ev * ev;
        gt += ev * dres(k, r);
    }
    {
        const double2 sums = team_sum2(cc, gt, s_red);   // also orders D, E, bb, g before the solve
        cc = rho * sums.x;
        gt = 1.0 + rho * sums.y;
    }
    cc += mu * (cc + 1e-9);
    // 3. the tridiagonal part T (diagonal blocks D_k, couplings T[k][k+1] = E_k) solved for the
    //    two right-hand sides b (into y, ws.bb) and -g (into v, ws.g) by block cyclic reduction.
    //    Level s = 1, 2, 4, ... eliminates the blocks k = s, 3s, 5s, ... <= N, each between
    //    l = k - s and r = k + s (when r <= N), one warp per block:
    //      L L^T = D_k,  P = L^-1 T[k][l],  Q = L^-1 T[k][r],  w = L^-1 f_k,
    //    then the kept blocks j = 0, 2s, 4s, ... take D_j -= Q_(j-s)^T Q_(j-s) + P_(j+s)^T P_(j+s),
    //    f_j -= Q_(j-s)^T w_(j-s) + P_(j+s)^T w_(j+s) and the coupling T'[j][j+2s] = -P^T Q of
    //    block j + s. Block 0 is left and solved; the eliminated blocks then follow level by
    //    level from the last: x_k = L^-T (w - P x_l - Q x_r). The couplings are kept in ws.E
    //    under their left block (E_l becomes the new coupling; E_k then holds Q), P in ws.P,
    //    the factors (1 / L_pp on the diagonal) in ws.D, w and x in ws.bb / ws.g. Each level's
    //    blocks are independent, so the chain of dependent FP64 steps is that of about
    //    log2(N + 1) block factors instead of N + 1.
    const int warp = tm.warp(), lane = threadIdx.x & 31, n_warps = tm.nwarps();
    double *Fw = s_blk + (size_t)(threadIdx.x >> 5) * kWarpScratch;
    int s_top = 1;
    for (int s = 1; s <= N; s <<= 1) {
        s_top = s;
        const int n_odd = (N / s + 1) / 2;
        for (int m = warp; m < n_odd; m += n_warps) {   // phase A
            const int k = (2 * m + 1) * s, l = k - s, r = k + s;
            const bool has_r = r <= N;
            warp_factor16(ws.D + (size_t)k * NW * NW, Fw, lane);
            const int c = lane & (NW - 1);
            const bool do_p = lane < NW, do_q = lane >= NW && has_r;
            if (do_p)   // column c of T[k][l] = row c of the coupling E_l
                column_solve16(Fw, ws.E + (size_t)l * NW * NW + c * NW, 1, ws.P + (size_t)k * NW * NW + c, NW);
            if (do_q)   // column c of T[k][r] = E_k, solved in place
                column_solve16(Fw, ws.E + (size_t)k * NW * NW + c, NW, ws.E + (size_t)k * NW * NW + c, NW);
            if (lane < 2) {
                double *f = (lane ? ws.g : ws.bb) + (size_t)k * NW;
                column_solve16(Fw, f, 1, f, 1);
            }
            for (int ij = lane; ij < NW * NW; ij += 32) ws.D[(size_t)k * NW * NW + ij] = Fw[ij];
            __syncwarp();
        }
        team_sync();
        const int n_even = N / (2 * s) + 1;
        for (int m = warp; m < n_even; m += n_warps) {   // phase B
            const int j = 2 * m * s, iL = j - s, iR = j + s;
            const bool hasL = m > 0, hasR = iR <= N;
            const double *QL = ws.E + (size_t)(hasL ? iL : 0) * NW * NW;
            const double *PR = ws.P + (size_t)(hasR ? iR : 0) * NW * NW;
            for (int e = lane; e < NW * NW; e += 32) {
                const int a = e >> 4, b = e & (NW - 1);
                if (b > a) continue;
                double v0 = ws.D[(size_t)j * NW * NW + e], v1 = 0.0;
                if (hasL)
                    for (int q = 0; q < NW; ++q) v0 = fma(-QL[q * NW + a], QL[q * NW + b], v0);
                if (hasR)
                    for (int q = 0; q < NW; ++q) v1 = fma(-PR[q * NW + a], PR[q * NW + b], v1);
                ws.D[(size_t)j * NW * NW + e] = v0 + v1;
            }
            {
                const int a = lane & (NW - 1), which = lane >> 4;
                double *f = which ? ws.g : ws.bb;
                double v = f[(size_t)j * NW + a];
                if (hasL) {
                    const double *w = f + (size_t)iL * NW;
                    for (int q = 0; q < NW; ++q) v = fma(-QL[q * NW + a], w[q], v);
                }
                if (hasR) {
                    const double *w = f + (size_t)iR * NW;
                    for (int q = 0; q < NW; ++q) v = fma(-PR[q * NW + a], w[q], v);
                }
                f[(size_t)j * NW + a] = v;
            }
            if (hasR && iR + s <= N) {
                const double *QR = ws.E + (size_t)iR * NW * NW;
                for (int e = lane; e < NW * NW; e += 32) {
                    const int a = e >> 4, b = e & (NW - 1);
                    double v = 0.0;
                    for (int q = 0; q < NW; ++q) v = fma(PR[q * NW + a], QR[q * NW + b], v);
                    ws.E[(size_t)j * NW * NW + e] = -v;
                }
            }
            __syncwarp();
        }
        team_sync();
    }
    // block 0: D_0 x_0 = f_0
    if (warp == 0) {
        warp_factor16(ws.D, Fw, lane);
        if (lane < 2) {
            double *f = lane ? ws.g : ws.bb;
            column_solve16(Fw, f, 1, f, 1);
        }
        __syncwarp();
        warp_back16(Fw, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, ws.bb, ws.g, lane);
    }
    team_sync();
    // the eliminated blocks, from the last level to the first
    for (int s = s_top; s >= 1; s >>= 1) {
        const int n_odd = (N / s + 1) / 2;
        for (int m = warp; m < n_odd; m += n_warps) {
            const int k = (2 * m + 1) * s, l = k - s, r = k + s;
            const bool has_r = r <= N;
            warp_back16(ws.D + (size_t)k * NW * NW, ws.P + (size_t)k * NW * NW, ws.bb + (size_t)l * NW,
                        ws.g + (size_t)l * NW, has_r ? ws.E + (size_t)k * NW * NW : nullptr,
                        has_r ? ws.bb + (size_t)r * NW : nullptr, has_r ? ws.g + (size_t)r * NW : nullptr,
                        ws.bb + (size_t)k * NW, ws.g + (size_t)k * NW, lane);
        }
        team_sync();
    }
    // 4. the border: dt = (-g_t - b^T v) / (c - b^T y), dw = v - y dt, with y = T^-1 b and
    //    v = T^-1 (-g_w) (b the original border column, kept in the factor-free terms above:
    //    b^T y and b^T v are recomputed from y and v through T y = b, i.e. b^T y = y^T T y).
    //    T y = b and T v = -g hold, so b^T y = sum_k b_k . y_k needs the original b: it is
    //    re-derived here from its definition.
    double by = 0.0, bv = 0.0;
    for (int e = t; e < (N + 1) * NW; e += nt) {
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
    const double2 sums = team_sum2(by, bv, s_red);
    by = sums.x;
    bv = sums.y;
    const double dt = (-gt - bv) / (cc - by);
    const int d0 = dz_local ? (int)threadIdx.x : t, dn = dz_local ? (int)blockDim.x : nt;
    if (d0 == 0) dz[0] = dt;
    for (int e = d0; e < (N + 1) * NW; e += dn) dz[1 + e] = ws.g[e] - ws.bb[e] * dt;
    __syncthreads();
}

// One LM step for each trajectory (a test of the step): dz at (z, lam, mu). Cluster p of
// kTrajCtas CTAs serves trajectory p.
__global__ void __cluster_dims__(kTrajCtas, 1, 1) __launch_bounds__(kTrajThreads)
k_traj_step(const TrajDev td, const double *q_star, const double *z, const double *lam, double mu, double *ws_base,
            size_t ws_stride, double *dz)
{
    extern __shared__ double s_mem[];
    const int N = td.N, n_var = 1 + NW * (N + 1), n_eq = NX * (N + 2);
    const int p = (int)(blockIdx.x / kTrajCtas);
    const Team tm = team_of_block();
    double *s_red = s_mem;                                      // kRedDoubles
    double *s_blk = s_red + kRedDoubles;                        // per warp kWarpScratch
    double *x_S = s_blk + (kTrajThreads / 32) * kWarpScratch, *x_T = x_S + NX;
    const double *qs = q_star + (size_t)p * (N + 1) * 4;
    for (int i = threadIdx.x; i < NX; i += blockDim.x) {
        x_S[i] = i < 4 ? qs[i] : 0.0;
        x_T[i] = i < 4 ? qs[(size_t)N * 4 + i] : 0.0;
    }
    __syncthreads();
    const TrajWs ws = ws_of(ws_base + (size_t)p * ws_stride, N);
    lm_step(tm, td, z + (size_t)p * n_var, lam + (size_t)p * n_eq, qs, x_S, x_T, mu, ws, dz + (size_t)p * n_var, false,
            s_red, s_blk);
}

// The whole solve (T6) for each trajectory: z in place; stats {t_F, F, max |c|, max bound
// violation}. Cluster p of kTrajCtas CTAs serves trajectory p; each CTA keeps z, the trial
// point and the step in its shared memory and updates all of them itself (the same values in
// both), the multipliers and the workspace are global and split.
__global__ void __cluster_dims__(kTrajCtas, 1, 1) __launch_bounds__(kTrajThreads)
k_traj_solve(const TrajDev td, const double *q_star, double *z_io, double *ws_base, size_t ws_stride, double *lam_ws,
             double *stats)
{
    extern __shared__ double s_mem[];
    const int N = td.N, n_var = 1 + NW * (N + 1), n_eq = NX * (N + 2);
    const int p = (int)(blockIdx.x / kTrajCtas), t = threadIdx.x;
    const Team tm = team_of_block();
    double *s_red = s_mem;
    double *s_blk = s_red + kRedDoubles;
    double *x_S = s_blk + (kTrajThreads / 32) * kWarpScratch, *x_T = x_S + NX;
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
    for (int i = tm.tid(); i < n_eq; i += tm.nthreads()) lam[i] = 0.0;
    team_sync();
    const TrajWs ws = ws_of(ws_base + (size_t)p * ws_stride, N);
    double mu = td.mu0;
    for (int o = 0; o < td.outer; ++o) {
        eval_f(tm, td, z, ws.f);
        team_sync();
        double F = merit(tm, td, z, lam, qs, ws.f, x_S, x_T, s_red);
        for (int it = 0; it < td.inner; ++it) {
            lm_step(tm, td, z, lam, qs, x_S, x_T, mu, ws, dz, true, s_red, s_blk);
            for (int i = t; i < n_var; i += blockDim.x) zn[i] = z[i] + dz[i];
            __syncthreads();
            eval_f(tm, td, zn, ws.f);
            team_sync();
            const double Fn = merit(tm, td, zn, lam, qs, ws.f, x_S, x_T, s_red);
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
        eval_f(tm, td, z, ws.f);
        team_sync();
        const double h = z[0] / N;
        for (int e = tm.tid(); e < n_eq; e += tm.nthreads()) {
            const int k = e / NX, i = e - k * NX;
            double c;
            if (k < N) c = z[1 + (size_t)(k + 1) * NW + i] - z[1 + (size_t)k * NW + i] -
                           0.5 * h * (ws.f[(size_t)k * NX + i] + ws.f[(size_t)(k + 1) * NX + i]);
            else if (k == N) c = z[1 + i] - x_S[i];
            else c = z[1 + (size_t)N * NW + i] - x_T[i];
            lam[e] += td.rho * c;
        }
        team_sync();
    }
    // results and statistics (each CTA takes every entry; CTA 0 writes them)
    if (tm.rank == 0)
        for (int i = t; i < n_var; i += blockDim.x) z_io[(size_t)p * n_var + i] = z[i];
    eval_f(tm, td, z, ws.f);
    team_sync();
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
        s_red[32 + (t >> 5)] = vmax;
    }
    __syncthreads();
    if (t == 0 && tm.rank == 0) {
        double c = 0.0, v = 0.0;
        for (int i = 0; i < kTrajThreads / 32; ++i) {
            c = fmax(c, s_red[i]);
            v = fmax(v, s_red[32 + i]);
        }
        stats[(size_t)p * 4 + 2] = c;
        stats[(size_t)p * 4 + 3] = fmax(v, 0.0);
    }
    __syncthreads();
    const double Fend = merit(tm, td, z, lam, qs, ws.f, x_S, x_T, s_red);
    if (t == 0 && tm.rank == 0) {
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
    return (size_t)(N + 1) * (NX + NX * NW + 2 * NW * NW + 2 * NW + 10) + (size_t)N * NW * NW;
}

size_t traj_smem(int N, bool solve)
{
    const size_t base = kRedDoubles + (size_t)(kTrajThreads / 32) * kWarpScratch + 2 * NX;
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
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_traj_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)traj_smem(tp->N, false));
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
    k_traj_step<<<n * kTrajCtas, kTrajThreads, traj_smem(t->td.N, false), t->st>>>(t->td, d_q_star, d_z, d_lam, mu,
                                                                                 t->ws, t->ws_stride, d_dz);
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
    k_traj_solve<<<n * kTrajCtas, kTrajThreads, traj_smem(t->td.N, true), t->st>>>(t->td, d_q_star, d_z, t->ws,
                                                                                  t->ws_stride, t->lam, d_stats);
    CP_LAUNCHED("k_traj_solve");
    return CP_OK;
}

}  // extern "C"

"""FP64 oracle of the trajectory tracking optimisation of arXiv 2503.14160, Sec. 4.2
(Eq. discrete) -- TEST INFRASTRUCTURE.

Only the test-suite and the benchmark's CPU-baseline leg use this module; the CUDA library
never does, and the two share no code.

The paper turns the planned path q*(s) into a near-time-optimal trajectory by direct
collocation: with states x_k and inputs u_k at n_s grid points and h = t_F / n_s,

    min  t_F + w_s sum_k u_k^T R u_k + w_t sum_k |q_a,k - q*_a,k|^2
    s.t. x_{k+1} - x_k = h/2 (f(x_k, u_k) + f(x_{k+1}, u_{k+1}))     (trapezoidal rule)
         x_0 = x_S, x_N = x_T,  x_min <= x_k <= x_max,

where f is the crane's forward dynamics with the accelerations of the actuated joints as
inputs (Sec. 2.1). The paper gives the structure of f but not its parameters, so a synthetic
model with that structure stands in (readings T1-T5 below), and its own interior-point solver
(IPOPT with MA57) is replaced by the method written out here (T6).

Readings where the paper is silent:
  T1 model   x = [q1..q4, alpha, beta, dq1..dq4, dalpha, dbeta] (12), u = ddq1..ddq4 (4):
             the four actuated joints of the path step are driven through their
             accelerations (subordinate velocity controllers, Sec. 2.1); the passive joints
             are the grapple's two swing angles: a point mass on a rigid link of length
             grapple_len hanging from the tip T(q_a), along
                 r(alpha, beta) = (sin a, cos a sin b, -cos a cos b)   (world axes),
             plumb at alpha = beta = 0. The gripper joints carry no dynamics of interest and
             are left out (as in the path step).
  T2 passive dynamics  the Euler-Lagrange equations of that pendulum with an accelerated
             pivot: with R = dr/d(alpha, beta) (R^T R = diag(1, cos^2 a)) and
             w = dR/dt (dalpha, dbeta),  R^T (T'' + l w + g z) + l R^T R (ddalpha, ddbeta) = 0.
  T3 tip acceleration  T = (h cos q1, h sin q1, base_z + z), h = L_b cos q2 + lam cos(q2+q3),
             z = L_b sin q2 + lam sin(q2+q3), lam = L_j + q4, differentiated twice in time
             (cylindrical coordinates).
  T4 weights and limits  R = I, w_s = 1e-2, w_t = 1e2; the joint limits of the path step;
             hydraulic velocity limits |dq| <= (0.6, 0.3, 0.3, 0.5) (rad/s, m/s); swing angles
             within +-0.6 rad; swing rates unbounded. x_S = (q_0, 0), x_T = (q_d, 0). The sums
             run over k = 1..N as printed; q*_a,k = q*(k / N).
  T5 grid    N intervals with N + 1 grid points (N = n_s); z = (t_F, w_0, ..., w_N) with
             w_k = (x_k, u_k), 1 + 16 (N + 1) variables.
  T6 solver  The equality constraints (defects and end states) enter through an augmented
             Lagrangian lambda^T c + rho/2 |c|^2, the bounds through a quadratic penalty
             rho_b/2 |max(0, x - x_max) + min(0, x - x_min)|^2; so the objective is
             F(z) = t_F + 1/2 |r(z)|^2 + const with a residual vector r. Each inner step is a
             damped Gauss-Newton (Levenberg-Marquardt) step
                 (J^T J + mu (diag(J^T J) + 1e-9)) dz = -(e_t + J^T r),
             accepted when F decreases (mu / 3, floor 1e-12), else mu * 4 (cap 1e12); after
             `inner` steps the multipliers move, lambda <- lambda + rho c (12 x 10 steps by
             default; a fixed schedule, so the constraints hold to what it reaches, reported
             per solve). The Jacobian J is
             taken by complex-step differentiation of r (exact to rounding), dense.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GRAVITY = 9.81
NX, NU = 12, 4
NW = NX + NU


@dataclasses.dataclass(frozen=True)
class TrajParams:
    N: int = 100
    omega_s: float = 1e-2
    omega_t: float = 1e2
    R: tuple = (1.0, 1.0, 1.0, 1.0)
    dq_max: tuple = (0.6, 0.3, 0.3, 0.5)
    swing_max: float = 0.6
    grapple_len: float = 1.0
    rho: float = 3e3
    rho_b: float = 1e5
    outer: int = 12
    inner: int = 10
    mu0: float = 1e-3

    @property
    def n_var(self) -> int:
        return 1 + NW * (self.N + 1)


# --------------------------------------------------------------------------- dynamics

def tip_acceleration(model, q, dq, u):
    """T'' (T3) for q, dq, u = ddq of the actuated joints (arrays [..., 4]; complex-safe)."""
    q1, q2, q3, q4 = (q[..., i] for i in range(4))
    d1, d2, d3, d4 = (dq[..., i] for i in range(4))
    u1, u2, u3, u4 = (u[..., i] for i in range(4))
    Lb, lam = model.boom_len, model.jib_len + q4
    A, B = q2, q2 + q3
    dA, dB, ddA, ddB = d2, d2 + d3, u2, u2 + u3
    h = Lb * np.cos(A) + lam * np.cos(B)
    dh = -Lb * np.sin(A) * dA + d4 * np.cos(B) - lam * np.sin(B) * dB
    ddh = (-Lb * (np.cos(A) * dA * dA + np.sin(A) * ddA) + u4 * np.cos(B)
           - 2.0 * d4 * np.sin(B) * dB - lam * (np.cos(B) * dB * dB + np.sin(B) * ddB))
    ddz = (Lb * (-np.sin(A) * dA * dA + np.cos(A) * ddA) + u4 * np.sin(B)
           + 2.0 * d4 * np.cos(B) * dB + lam * (-np.sin(B) * dB * dB + np.cos(B) * ddB))
    a_r = ddh - h * d1 * d1               # radial
    a_t = h * u1 + 2.0 * dh * d1          # tangential
    c1, s1 = np.cos(q1), np.sin(q1)
    return np.stack([a_r * c1 - a_t * s1, a_r * s1 + a_t * c1, ddz], axis=-1)


def tip_position(model, q):
    """T(q) of T3 (for the pins)."""
    q1, q2, q3, q4 = (q[..., i] for i in range(4))
    lam = model.jib_len + q4
    h = model.boom_len * np.cos(q2) + lam * np.cos(q2 + q3)
    z = model.boom_len * np.sin(q2) + lam * np.sin(q2 + q3)
    return np.stack([h * np.cos(q1), h * np.sin(q1), model.base_z + z], axis=-1)


def swing_acceleration(tp: TrajParams, a, b, da, db, tip_acc):
    """(ddalpha, ddbeta) of T2 for swing angles, rates and the tip acceleration [..., 3]."""
    ell = tp.grapple_len
    ca, sa, cb, sb = np.cos(a), np.sin(a), np.cos(b), np.sin(b)
    r_a = np.stack([ca, -sa * sb, sa * cb], axis=-1)          # dr / dalpha
    r_b = np.stack([0.0 * ca, ca * cb, ca * sb], axis=-1)     # dr / dbeta
    r_aa = np.stack([-sa, -ca * sb, ca * cb], axis=-1)
    r_ab = np.stack([0.0 * ca, -sa * cb, -sa * sb], axis=-1)
    r_bb = np.stack([0.0 * ca, -ca * sb, ca * cb], axis=-1)
    w = (r_aa * (da * da)[..., None] + 2.0 * r_ab * (da * db)[..., None] + r_bb * (db * db)[..., None])
    v = tip_acc + ell * w
    v = v + np.stack([0.0 * ca, 0.0 * ca, GRAVITY + 0.0 * ca], axis=-1)
    dda = -np.sum(r_a * v, axis=-1) / ell
    ddb = -np.sum(r_b * v, axis=-1) / (ell * ca * ca)
    return dda, ddb


def dynamics(model, tp: TrajParams, x, u):
    """x' = f(x, u) of T1-T3, x [..., 12], u [..., 4] (complex-safe)."""
    q, ab, dq, dab = x[..., 0:4], x[..., 4:6], x[..., 6:10], x[..., 10:12]
    dda, ddb = swing_acceleration(tp, ab[..., 0], ab[..., 1], dab[..., 0], dab[..., 1],
                                  tip_acceleration(model, q, dq, u))
    return np.concatenate([dq, dab, u, dda[..., None], ddb[..., None]], axis=-1)


# --------------------------------------------------------------------------- collocation NLP

class TrajProblem:
    """Eq. discrete for one path: targets q*_k (k = 0..N), start and goal configurations."""

    def __init__(self, model, tp: TrajParams, q_star: np.ndarray, q0, qd):
        self.model, self.tp = model, tp
        self.N = tp.N
        self.q_star = np.asarray(q_star, dtype=np.float64).reshape(tp.N + 1, 4)
        self.x_S = np.concatenate([np.asarray(q0, np.float64), np.zeros(8)])
        self.x_T = np.concatenate([np.asarray(qd, np.float64), np.zeros(8)])
        big = 1e30
        self.x_min = np.array(list(model.q_min) + [-tp.swing_max] * 2 + [-v for v in tp.dq_max] + [-big] * 2)
        self.x_max = np.array(list(model.q_max) + [tp.swing_max] * 2 + list(tp.dq_max) + [big] * 2)
        self.n_eq = NX * (tp.N + 2)   # N defects, the two end states

    def unpack(self, z):
        W = z[1:].reshape(self.N + 1, NW)
        return z[0], W[:, :NX], W[:, NX:]

    def constraints(self, z):
        """c(z): the N defects of the trapezoidal rule, then x_0 - x_S and x_N - x_T."""
        t_F, X, U = self.unpack(z)
        h = t_F / self.N
        F = dynamics(self.model, self.tp, X, U)
        defect = X[1:] - X[:-1] - 0.5 * h * (F[1:] + F[:-1])
        return np.concatenate([defect.reshape(-1), X[0] - self.x_S, X[-1] - self.x_T])

    def violation(self, z):
        _, X, _ = self.unpack(z)
        hi = np.where(X.real > self.x_max, X - self.x_max, 0.0 * X)
        lo = np.where(X.real < self.x_min, X - self.x_min, 0.0 * X)
        return (hi + lo).reshape(-1)

    def residual(self, z, lam):
        """r(z) with F(z) = t_F + 1/2 |r|^2 + const (T6)."""
        tp = self.tp
        _, X, U = self.unpack(z)
        c = self.constraints(z)
        effort = np.sqrt(2.0 * tp.omega_s * np.asarray(tp.R))[None, :] * U[1:]
        track = math.sqrt(2.0 * tp.omega_t) * (X[1:, :4] - self.q_star[1:])
        return np.concatenate([math.sqrt(tp.rho) * (c + lam / tp.rho), effort.reshape(-1),
                               track.reshape(-1), math.sqrt(tp.rho_b) * self.violation(z)])

    def merit(self, z, lam):
        r = self.residual(z, lam)
        return float(z[0] + 0.5 * np.dot(r, r))

    def jacobian(self, z, lam):
        """dr/dz by complex-step differentiation, column by column."""
        n = z.size
        step = 1e-30
        r0 = self.residual(z, lam)
        J = np.empty((r0.size, n))
        zc = z.astype(np.complex128)
        for j in range(n):
            zc[j] += 1j * step
            J[:, j] = self.residual(zc, lam).imag / step
            zc[j] -= 1j * step
        return r0, J

    def lm_step(self, z, lam, mu):
        """The damped Gauss-Newton step of T6 from z with damping mu (no acceptance)."""
        r, J = self.jacobian(z, lam)
        g = J.T @ r
        g[0] += 1.0
        H = J.T @ J
        A = H + mu * (np.diag(np.diag(H)) + 1e-9 * np.eye(H.shape[0]))
        return np.linalg.solve(A, -g)

    def initial_guess(self, t_F=None):
        """z from the path: q_a = q*_k, dq_a by central differences over t_F, u by second
        differences, swing at rest; t_F = 1.5 x the slowest joint's total variation over
        its velocity limit (unless given)."""
        tp, N = self.tp, self.N
        if t_F is None:
            tv = np.abs(np.diff(self.q_star, axis=0)).sum(axis=0)
            t_F = max(1.5 * float(np.max(tv / np.asarray(tp.dq_max))), 1e-3)
        h = t_F / N
        X = np.zeros((N + 1, NX))
        X[:, :4] = self.q_star
        X[1:-1, 6:10] = (self.q_star[2:] - self.q_star[:-2]) / (2.0 * h)
        U = np.zeros((N + 1, NU))
        U[1:-1] = (self.q_star[2:] - 2.0 * self.q_star[1:-1] + self.q_star[:-2]) / (h * h)
        return np.concatenate([[t_F], np.concatenate([X, U], axis=1).reshape(-1)])

    def solve(self, z0, record=None):
        """T6 from z0: `outer` multiplier updates of `inner` damped Gauss-Newton steps each.
        Returns (z, lam, mu); `record` (a list) receives (z, lam, mu, accepted) per step."""
        tp = self.tp
        z = np.asarray(z0, dtype=np.float64).copy()
        lam = np.zeros(self.n_eq)
        mu = tp.mu0
        for _ in range(tp.outer):
            F = self.merit(z, lam)
            for _ in range(tp.inner):
                dz = self.lm_step(z, lam, mu)
                z_new = z + dz
                F_new = self.merit(z_new, lam)
                accepted = F_new < F
                if record is not None:
                    record.append((z.copy(), lam.copy(), mu, accepted))
                if accepted:
                    z, F = z_new, F_new
                    mu = max(mu / 3.0, 1e-12)
                else:
                    mu = min(mu * 4.0, 1e12)
            lam = lam + tp.rho * self.constraints(z)
        return z, lam, mu


def path_targets(P, N: int) -> np.ndarray:
    """q*(k / N), k = 0..N, of a cubic B-spline path with control points P[K+8][4] on the
    moving spans (the path step's reading: tau = 4 + (K+3) s on uniform knots), by the
    oracle's Cox-de Boor evaluation."""
    import oracle   # the path oracle (same folder)
    P = np.asarray(P, dtype=np.float64)
    K = P.shape[0] - 8
    return np.stack([oracle.bspline(P, 4.0 + (K + 3) * (k / N)) for k in range(N + 1)])

"""Oracle: filament model, BDF2 / Lie-group residual, approximate Jacobian,
limited-memory bad Broyden and the timestep driver, in plain numpy FP64.

TEST INFRASTRUCTURE (see the package docstring): never imported by the
library. Each function names the passage of the paper it restates.

Layouts
-------
* Segments of all filaments are concatenated, filament-major: segment n of
  filament i is row off_seg[i] + n of every per-segment array.
* Quaternions are (q0, q1, q2, q3), scalar first (Sec. 2.9.1).
* The unknown vector X holds, per filament of N segments, the 6N entries
  [Y_1 (3), u_1..u_N (3N), Lambda_{3/2}..Lambda_{N-1/2} (3(N-1))]
  (Sec. 2.9.3, robot-arm reduction), filaments concatenated.
* The residual f has the same per-filament shape: [f^1 (3), f^2_1..N (3N),
  f^3_2..N (3(N-1))] (eqn RA-3d-system).

Readings where the paper is silent (each also listed in the design notes):
* First step (no Y^{j-1}): backward Euler, f^1 = Y - Y^j - dt V,
  f^2 = u - dt dexpinv_u(Omega); BDF2 from the second step on.
* Initial guess of a step: every unknown linearly extrapolated from the two
  previous steps, x_0 = 2 x^j - x^{j-1}, when both exist (Y_1 from the BDF2
  history; u and Lambda from the last two committed steps); with one previous
  step u = u^j and Lambda = Lambda^j; on the first step Y_1^j, u = 0, Lambda^j.
  Optionally (order 2) the quadratic through the last three values,
  x_0 = 3 x^j - 3 x^{j-1} + x^{j-2}, for each unknown that has three; or
  (order 3, adaptive) per filament and block of unknowns (Y_1, u, Lambda) the
  linear guess plus theta times the second difference d = x^j - 2 x^{j-1} +
  x^{j-2}, theta the least-squares coefficient of d in the past solutions'
  departures from their linear guesses, weighted 0.7^age, clipped to [0, 1].
* Convergence: ||f||_inf <= tol * a (Sec. 3.3 states the tolerance for the
  infinity norm relative to a). Norms in Algorithm 2 are the 2-norm over the
  whole system.
* The approximate Jacobian uses the same time-integration weight as the
  residual: (2/3) dt for BDF2 (as printed in App. B.2) and dt for the first,
  backward-Euler step. Its torque value T_m (needed by J22_mm) is the elastic
  plus constraint torque at the iterate where J0 is built.
* External forces: a constant force per segment (gravity), a constant torque
  per segment and a follower force -f t_N on the last segment of a filament.
  External loads do not enter J0 (App. B keeps constraint and elastic terms).
* Tethered filaments (Sec. 5.2.1; eqs. tethering_constraint, tethered_rotation_constraint,
  tethering_constraint_force_and_torque): Y_1 and u_1 of a tethered filament
  are prescribed for the step and the X slots that held them carry the two
  multipliers instead (lambda_1, a force on segment 1, in the Y_1 slot;
  lambda_2, giving the torque D^T lambda_2 on segment 1, in the u_1 slot); the
  update equations f^1 and f^2_1 keep their form with the prescribed values
  substituted. J0 of a tethered filament is the free filament's J0 at the
  prescribed values with those two column blocks replaced by the derivatives
  with respect to the multipliers, through the same mobility and the same
  three-term dexpinv factor A_1 as the other rotation rows. A clamped end is a
  tether with Y_1 fixed and u_1 = 0. The multipliers are not internal loads:
  like external loads they stay out of J0's torque value. Their initial guess
  is extrapolated from past steps like Lambda's.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from . import rpy, steric

PI = math.pi


# --------------------------------------------------------------------------
# Quaternion algebra, Sec. 2.9.1
# --------------------------------------------------------------------------

def qmul(p, q):
    """Quaternion product (p0 q0 - p.q, p0 q + q0 p + p x q), Sec. 2.9.1."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    p0, pv = p[..., 0], p[..., 1:]
    q0, qv = q[..., 0], q[..., 1:]
    s = p0 * q0 - np.sum(pv * qv, axis=-1)
    v = p0[..., None] * qv + q0[..., None] * pv + np.cross(pv, qv)
    return np.concatenate([s[..., None], v], axis=-1)


def qconj(q):
    q = np.asarray(q, dtype=np.float64)
    return np.concatenate([q[..., :1], -q[..., 1:]], axis=-1)


def rotation_matrix(q):
    """R(q), the printed matrix of eq. (quaternion_rotation_matrix)."""
    q = np.asarray(q, dtype=np.float64)
    q0, q1, q2, q3 = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * q2 ** 2 - 2 * q3 ** 2
    R[..., 0, 1] = 2 * (q1 * q2 - q3 * q0)
    R[..., 0, 2] = 2 * (q1 * q3 + q2 * q0)
    R[..., 1, 0] = 2 * (q1 * q2 + q3 * q0)
    R[..., 1, 1] = 1 - 2 * q1 ** 2 - 2 * q3 ** 2
    R[..., 1, 2] = 2 * (q3 * q2 - q1 * q0)
    R[..., 2, 0] = 2 * (q1 * q3 - q2 * q0)
    R[..., 2, 1] = 2 * (q3 * q2 + q1 * q0)
    R[..., 2, 2] = 1 - 2 * q2 ** 2 - 2 * q1 ** 2
    return R


def qsqrt(p):
    """Square root of a unit quaternion, App. A.1:
    (sqrt((p0+1)/2), p / sqrt(2(p0+1))) for p0 != -1, and (0,0,0,1) for p0 = -1."""
    p = np.asarray(p, dtype=np.float64)
    out = np.empty_like(p)
    flat_p = p.reshape(-1, 4)
    flat_o = out.reshape(-1, 4)
    for k in range(flat_p.shape[0]):
        p0 = flat_p[k, 0]
        if p0 == -1.0:
            flat_o[k] = (0.0, 0.0, 0.0, 1.0)
        else:
            flat_o[k, 0] = math.sqrt((p0 + 1.0) / 2.0)
            flat_o[k, 1:] = flat_p[k, 1:] / math.sqrt(2.0 * (p0 + 1.0))
    return out


def qexp(u):
    """Exponential map exp(u) = (cos(|u|/2), sin(|u|/2) u/|u|), Sec. 2.9.3.

    sin(|u|/2)/|u| is written as 0.5*sinc(|u|/(2 pi)) so that |u| -> 0 is
    exact (numpy's sinc(x) = sin(pi x)/(pi x))."""
    u = np.asarray(u, dtype=np.float64)
    th = np.linalg.norm(u, axis=-1)
    s = 0.5 * np.sinc(th / (2.0 * PI))
    return np.concatenate([np.cos(th / 2.0)[..., None], s[..., None] * u], axis=-1)


def dexpinv_coefficient(th):
    """c(x) = (x cot(x/2) - 2) / (2 x^2), the factor of u x (u x Omega) in
    eq. (dexpinv_definition). For small x the Taylor series of x cot(x/2)
    gives c = -1/12 - x^2/720 - x^4/30240 + O(x^6)."""
    th = np.asarray(th, dtype=np.float64)
    out = np.empty_like(th)
    small = th < 1e-2
    x = th[small]
    out[small] = -1.0 / 12.0 - x ** 2 / 720.0 - x ** 4 / 30240.0
    x = th[~small]
    out[~small] = (x / np.tan(x / 2.0) - 2.0) / (2.0 * x ** 2)
    return out


def dexpinv(u, w):
    """dexpinv_u(Omega) = Omega - u x Omega / 2 - c(|u|) u x (u x Omega),
    eq. (dexpinv_definition), with c(x) = (x cot(x/2) - 2)/(2x^2) ~ -1/12."""
    u = np.asarray(u, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    c = dexpinv_coefficient(np.linalg.norm(u, axis=-1))
    uxw = np.cross(u, w)
    return w - 0.5 * uxw - c[..., None] * np.cross(u, uxw)


def quat_from_frame(t, mu):
    """Quaternion whose R has columns (t, mu, t x mu), App. A.1 steps 1-5."""
    t = np.atleast_2d(np.asarray(t, dtype=np.float64))
    mu = np.atleast_2d(np.asarray(mu, dtype=np.float64))
    out = np.empty((t.shape[0], 4))
    ey = np.array([0.0, 1.0, 0.0])
    for k in range(t.shape[0]):
        p1 = qsqrt(np.array([t[k, 0], 0.0, -t[k, 2], t[k, 1]]))
        n1 = rotation_matrix(p1) @ ey
        p2 = qsqrt(np.concatenate([[n1 @ mu[k]], np.cross(n1, mu[k])]))
        out[k] = qmul(p2, p1)
    return out


# --------------------------------------------------------------------------
# System description
# --------------------------------------------------------------------------

@dataclass
class Params:
    a: float = 1.0
    eta: float = 1.0
    dL: float = 2.2
    KB: float = 1.0
    KT: float = 1.0
    gamma0: float = 0.0
    kappa_mu: float = 0.0
    kappa_nu: float = 0.0
    dt: float = 0.01
    tol: float = 1e-8
    max_iter: int = 50
    FS: float = 0.0       # steric barrier strength (Sec. 2.6); 0: no barrier
    chi: float = 1.1      # steric range: the barrier acts for r < 2 chi a


class Layout:
    """Offsets of ragged filaments in the segment, X and Lambda arrays."""

    def __init__(self, seg_per_fil):
        self.N = [int(n) for n in seg_per_fil]
        assert all(n >= 1 for n in self.N)
        self.M = len(self.N)
        self.S = sum(self.N)
        self.off_seg = np.concatenate([[0], np.cumsum(self.N)]).astype(int)
        self.off_X = 6 * self.off_seg
        self.off_lam = np.concatenate([[0], np.cumsum([n - 1 for n in self.N])]).astype(int)
        self.n_lam = int(self.off_lam[-1])

    def split_X(self, X):
        """X -> (Y1 (M,3), u (S,3), Lam (n_lam,3))."""
        X = np.asarray(X, dtype=np.float64)
        Y1 = np.empty((self.M, 3))
        u = np.empty((self.S, 3))
        lam = np.empty((self.n_lam, 3))
        for i, n in enumerate(self.N):
            b = self.off_X[i]
            Y1[i] = X[b:b + 3]
            u[self.off_seg[i]:self.off_seg[i + 1]] = X[b + 3:b + 3 + 3 * n].reshape(n, 3)
            lam[self.off_lam[i]:self.off_lam[i + 1]] = \
                X[b + 3 + 3 * n:b + 6 * n].reshape(n - 1, 3)
        return Y1, u, lam

    def join_X(self, Y1, u, lam):
        X = np.empty(6 * self.S)
        for i, n in enumerate(self.N):
            b = self.off_X[i]
            X[b:b + 3] = Y1[i]
            X[b + 3:b + 3 + 3 * n] = u[self.off_seg[i]:self.off_seg[i + 1]].ravel()
            X[b + 3 + 3 * n:b + 6 * n] = lam[self.off_lam[i]:self.off_lam[i + 1]].ravel()
        return X


@dataclass
class External:
    """Constant per-segment force and torque plus a tip follower force."""
    Fext: np.ndarray | None = None      # (S, 3)
    Text: np.ndarray | None = None      # (S, 3)
    follower: np.ndarray | None = None  # (M,), force -follower[i] * t_N on the last segment


@dataclass
class State:
    """BDF2 history: Y^j, Y^{j-1} (None before the first step), q^j, u^j, Lambda^j,
    and for the initial guess u^{j-1}, Lambda^{j-1} (None until two steps exist)
    and Y^{j-2}, u^{j-2}, Lambda^{j-2} (None until they exist)."""
    Y: np.ndarray
    q: np.ndarray
    Yprev: np.ndarray | None = None
    u: np.ndarray | None = None
    lam: np.ndarray | None = None
    steps: int = 0
    u_prev: np.ndarray | None = None
    lam_prev: np.ndarray | None = None
    tlam: np.ndarray | None = None        # (M, 6) tether multipliers of the last step
    tlam_prev: np.ndarray | None = None   # (M, 6) of the step before
    Yprev2: np.ndarray | None = None
    u_prev2: np.ndarray | None = None
    lam_prev2: np.ndarray | None = None
    xfit: np.ndarray | None = None        # (M, 3, 2) adaptive fit (P, Q) of Y_1, u, Lambda
    extra: dict = field(default_factory=dict)

    def copy(self):
        def cp(a):
            return None if a is None else a.copy()
        return State(Y=self.Y.copy(), q=self.q.copy(), Yprev=cp(self.Yprev), u=cp(self.u),
                     lam=cp(self.lam), steps=self.steps, u_prev=cp(self.u_prev),
                     lam_prev=cp(self.lam_prev), tlam=cp(self.tlam),
                     tlam_prev=cp(self.tlam_prev), Yprev2=cp(self.Yprev2),
                     u_prev2=cp(self.u_prev2), lam_prev2=cp(self.lam_prev2),
                     xfit=cp(self.xfit))


@dataclass
class Tether:
    """Prescribed base motion of tethered filaments for one step (eqs.
    tethering_constraint, tethered_rotation_constraint): where mask[i], Y_1 of
    filament i is Y1[i] and the rotation of its first segment over the step is
    u1[i] (q_1 = exp(u1[i]) q_1^j)."""
    mask: np.ndarray      # (M,) bool
    Y1: np.ndarray        # (M, 3)
    u1: np.ndarray        # (M, 3)


# --------------------------------------------------------------------------
# Unpack X: q = exp(u) q^j, frames, robot-arm positions (Sec. 2.9.3)
# --------------------------------------------------------------------------

def frames(q):
    """Columns of R(q): tangent t, normals mu and nu (eq. RotToFrame)."""
    R = rotation_matrix(q)
    return R[..., :, 0], R[..., :, 1], R[..., :, 2]


def robot_arm_positions(lay: Layout, Y1, t, dL):
    """Y_n = Y_1 + (dL/2) sum_{m=2}^n (t_{m-1} + t_m), eq. (positionSubstitution-3d)."""
    Y = np.empty((lay.S, 3))
    for i, n in enumerate(lay.N):
        s = lay.off_seg[i]
        Y[s] = Y1[i]
        for k in range(1, n):
            Y[s + k] = Y[s + k - 1] + 0.5 * dL * (t[s + k - 1] + t[s + k])
    return Y


def unpack(lay: Layout, p: Params, X, qj):
    """Quaternions q_n = exp(u_n) q_n^j (eq. general_multiplicative_q_update),
    tangents, positions and multipliers at X."""
    Y1, u, lam = lay.split_X(X)
    q = qmul(qexp(u), qj)
    t, _, _ = frames(q)
    Y = robot_arm_positions(lay, Y1, t, p.dL)
    return q, t, Y, u, lam


def dexpinv_matrix(u):
    """D with D v = dexpinv_u(v): columns dexpinv_u(e_c)."""
    return np.stack([dexpinv(u, e) for e in np.eye(3)], axis=1)


def tether_resolve(lay: Layout, X, tether: Tether | None):
    """(Xr, lam1, lam2): X with the Y_1 and u_1 slots of tethered filaments
    replaced by their prescribed values, and the multipliers read from those
    slots ((M, 3) each, zero for free filaments)."""
    Xr = np.array(X, dtype=np.float64)
    lam1 = np.zeros((lay.M, 3))
    lam2 = np.zeros((lay.M, 3))
    if tether is None:
        return Xr, lam1, lam2
    for i in range(lay.M):
        if tether.mask[i]:
            b = lay.off_X[i]
            lam1[i] = Xr[b:b + 3]
            lam2[i] = Xr[b + 3:b + 6]
            Xr[b:b + 3] = tether.Y1[i]
            Xr[b + 3:b + 6] = tether.u1[i]
    return Xr, lam1, lam2


# --------------------------------------------------------------------------
# Forces and torques, Sec. 2.5 and eq. (quaternionM)
# --------------------------------------------------------------------------

def internal_moments(q_a, q_b, p: Params):
    """M_{n+1/2} between q_n = q_a and q_{n+1} = q_b, eq. (quaternionM):
    q_{n+1/2} = (q_{n+1} q_n^*)^{1/2} q_n,
    M = R(q_{n+1/2}) D (2 [q_{n+1/2}^* (q_{n+1} - q_n)/dL]_R3 - (g0, kmu, knu))."""
    qh = qmul(qsqrt(qmul(q_b, qconj(q_a))), q_a)
    strain = 2.0 * qmul(qconj(qh), (q_b - q_a) / p.dL)[..., 1:]
    strain = strain - np.array([p.gamma0, p.kappa_mu, p.kappa_nu])
    D = np.array([p.KT, p.KB, p.KB])
    return np.einsum("...ij,...j->...i", rotation_matrix(qh), D * strain)


def forces_torques(lay: Layout, p: Params, q, t, lam, ext: External | None):
    """Right-hand side of the mobility problem (eq. mobility-problem-timeint):
    F_n = F^C_n + external, T_n = T^E_n + T^C_n + external, with
    F^C_n = Lam_{n+1/2} - Lam_{n-1/2}, T^C_n = (dL/2) t_n x (Lam_{n+1/2} + Lam_{n-1/2}),
    T^E_n = M_{n+1/2} - M_{n-1/2}, and Lam_{1/2} = Lam_{N+1/2} = M_{1/2} = M_{N+1/2} = 0
    (eqs. constraint-force, constraint-torque, elastic-torque)."""
    F = np.zeros((lay.S, 3))
    T = np.zeros((lay.S, 3))
    for i, n in enumerate(lay.N):
        s = lay.off_seg[i]
        L = np.zeros((n + 1, 3))          # L[k] = Lambda_{k+1/2}, k = 0..n
        L[1:n] = lam[lay.off_lam[i]:lay.off_lam[i + 1]]
        Mh = np.zeros((n + 1, 3))         # Mh[k] = M_{k+1/2}
        if n > 1:
            Mh[1:n] = internal_moments(q[s:s + n - 1], q[s + 1:s + n], p)
        for k in range(n):
            F[s + k] = L[k + 1] - L[k]
            T[s + k] = Mh[k + 1] - Mh[k] + 0.5 * p.dL * np.cross(t[s + k], L[k + 1] + L[k])
        if ext is not None and ext.follower is not None:
            F[s + n - 1] -= ext.follower[i] * t[s + n - 1]
    if ext is not None and ext.Fext is not None:
        F += ext.Fext
    if ext is not None and ext.Text is not None:
        T += ext.Text
    return F, T


def mobility(Y, F, T, p: Params, nthreads=1):
    """(V, Omega) = M (F, T), eq. (mobility-problem), by the RPY oracle."""
    VW = rpy.apply(Y, np.concatenate([F, T], axis=1), p.a, p.eta, nthreads=nthreads)
    return VW[:, :3], VW[:, 3:]


# --------------------------------------------------------------------------
# Residual, eqn (RA-3d-system)
# --------------------------------------------------------------------------

def scheme(state: State):
    """(alpha1, alpha0, beta, gamma): f = Y - alpha1 Y^j - alpha0 Y^{j-1} - beta dt V,
    f^2 = u - gamma u^j - beta dt dexpinv_u(Omega). BDF2 when Y^{j-1} exists,
    backward Euler on the first step."""
    if state.Yprev is None:
        return 1.0, 0.0, 1.0, 0.0
    return 4.0 / 3.0, -1.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0


def drag_mobility(Y, F, T, p: Params, nthreads=1):
    """Diagonal (self-only) mobility of App. B: V = F/(6 pi eta a), Omega = T/(8 pi eta a^3)."""
    return F / (6.0 * PI * p.eta * p.a), T / (8.0 * PI * p.eta * p.a ** 3)


def residual(lay: Layout, p: Params, state: State, ext: External | None, X,
             nthreads=1, return_parts=False, mob=None, tether: Tether | None = None):
    """f(X) of eqn (RA-3d-system) (per filament [f^1, f^2_1..N, f^3_2..N]).

    mob replaces the RPY mobility (e.g. by drag_mobility for the f_0 of App. B).
    With a tether, tethered filaments take their prescribed Y_1, u_1 and the
    multiplier loads F_1 += lambda_1, T_1 += D^T lambda_2 (D v =
    dexpinv_{u_1}(v)), eq. tethering_constraint_force_and_torque."""
    al1, al0, be, ga = scheme(state)
    X, lam1, lam2 = tether_resolve(lay, X, tether)
    q, t, Y, u, lam = unpack(lay, p, X, state.q)
    F, T = forces_torques(lay, p, q, t, lam, ext)
    if tether is not None:
        for i in range(lay.M):
            if tether.mask[i]:
                s0 = lay.off_seg[i]
                F[s0] += lam1[i]
                T[s0] += dexpinv_matrix(tether.u1[i]).T @ lam2[i]
    if p.FS != 0.0:
        F = F + steric.barrier_forces(lay.N, Y, p.a, p.FS, p.chi)
    V, W = (mob or mobility)(Y, F, T, p, nthreads)
    Yprev = state.Yprev if state.Yprev is not None else np.zeros_like(state.Y)
    uj = state.u if (state.u is not None and ga != 0.0) else np.zeros_like(u)
    fpos = Y - al1 * state.Y - al0 * Yprev - be * p.dt * V
    frot = u - ga * uj - be * p.dt * dexpinv(u, W)
    f = np.empty(6 * lay.S)
    for i, n in enumerate(lay.N):
        s, b = lay.off_seg[i], lay.off_X[i]
        f[b:b + 3] = fpos[s]
        f[b + 3:b + 3 + 3 * n] = frot[s:s + n].ravel()
        f[b + 3 + 3 * n:b + 6 * n] = fpos[s + 1:s + n].ravel()
    if return_parts:
        return f, dict(q=q, t=t, Y=Y, F=F, T=T, V=V, W=W)
    return f


# --------------------------------------------------------------------------
# Approximate Jacobian J0, App. B.2 (one dense 6N x 6N block per filament)
# --------------------------------------------------------------------------

def _cross_left(v):
    """[v x]: the matrix with [v x] w = v x w."""
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def _cross_right(v):
    """[x v]: the matrix with [x v] w = w x v (= -[v x])."""
    return -_cross_left(v)


def _dM_du(p: Params, ta, tb, mua, mub, nua, nub):
    """Derivatives of the frame-vector moment approximation of M_{m+1/2}
    (App. B.2) with respect to u_m (first result) and u_{m+1} (second)."""
    beta = (mub @ nua - mua @ nub) / (2.0 * p.dL) - p.gamma0
    w = np.cross(nua, mub) - np.cross(mua, nub)
    tsum = ta + tb
    Da = p.KB * (_cross_right(tb) @ _cross_right(ta) / p.dL
                 - 0.5 * p.kappa_mu * _cross_right(mua)
                 - 0.5 * p.kappa_nu * _cross_right(nua)) \
        + 0.5 * p.KT * (beta * _cross_right(ta) + np.outer(tsum, w) / (2.0 * p.dL))
    Db = p.KB * (_cross_left(ta) @ _cross_right(tb) / p.dL
                 - 0.5 * p.kappa_mu * _cross_right(mub)
                 - 0.5 * p.kappa_nu * _cross_right(nub)) \
        + 0.5 * p.KT * (beta * _cross_right(tb) - np.outer(tsum, w) / (2.0 * p.dL))
    return Da, Db


def jacobian0(lay: Layout, p: Params, state: State, X):
    """Dense per-filament blocks of J0 = [[I, 0, J13], [0, J22, J23], [I, J32, J33]]
    built from the drag-only model at X (App. B.2; J13 and J33 as in B.1)."""
    _, _, be, _ = scheme(state)
    ct = be * p.dt / (6.0 * PI * p.eta * p.a)
    cr = be * p.dt / (8.0 * PI * p.eta * p.a ** 3)
    q, t, Y, u, lam = unpack(lay, p, X, state.q)
    _, mu, nu = frames(q)
    F, T = forces_torques(lay, p, q, t, lam, None)
    I3 = np.eye(3)
    blocks = []
    for i, n in enumerate(lay.N):
        s = lay.off_seg[i]
        J = np.zeros((6 * n, 6 * n))
        L = np.zeros((n + 1, 3))
        L[1:n] = lam[lay.off_lam[i]:lay.off_lam[i + 1]]
        # column / row offsets inside the block
        cY, cu, cl = 0, 3, 3 + 3 * n          # columns: Y1, u_1..N, Lam_{3/2..N-1/2}
        r1, r2, r3 = 0, 3, 3 + 3 * n          # rows: f1, f2_1..N, f3_2..N

        def ucol(m):      # column of u_m, m = 1..N
            return cu + 3 * (m - 1)

        def lcol(k):      # column of Lambda_{k-1/2}, k = 2..N
            return cl + 3 * (k - 2)

        def f3row(m):     # row of f3_m, m = 2..N
            return r3 + 3 * (m - 2)

        J[r1:r1 + 3, cY:cY + 3] = I3
        if n >= 2:
            J[r1:r1 + 3, lcol(2):lcol(2) + 3] = -ct * I3          # J13
        Da = [None] * (n + 1)
        Db = [None] * (n + 1)
        for m in range(1, n):                                       # M_{m+1/2}
            Da[m], Db[m] = _dM_du(p, t[s + m - 1], t[s + m], mu[s + m - 1], mu[s + m],
                                  nu[s + m - 1], nu[s + m])
        for m in range(1, n + 1):
            um = u[s + m - 1]
            tm = t[s + m - 1]
            Tm = T[s + m - 1]
            A = I3 - 0.5 * _cross_left(um) + _cross_left(um) @ _cross_left(um) / 12.0
            # dT_m / du_n for n = m-1, m, m+1
            dT = {}
            dT[m] = 0.5 * p.dL * _cross_right(L[m] + L[m - 1]) @ _cross_right(tm)
            if m <= n - 1:
                dT[m] = dT[m] + Da[m]
                dT[m + 1] = Db[m]
            if m >= 2:
                dT[m] = dT[m] - Db[m - 1]
                dT[m - 1] = -Da[m - 1]
            row = r2 + 3 * (m - 1)
            for k, D in dT.items():
                if k == m:
                    ux = _cross_left(um)
                    blk = I3 - cr * (D - 0.5 * (_cross_right(Tm) + ux @ D)
                                     + (_cross_right(np.cross(um, Tm)) + ux @ _cross_right(Tm)
                                        + ux @ ux @ D) / 12.0)
                else:
                    blk = -cr * A @ D
                J[row:row + 3, ucol(k):ucol(k) + 3] = blk
            # J23: Lambda_{m-1/2} (k = m) and Lambda_{m+1/2} (k = m+1)
            dTl = 0.5 * p.dL * _cross_left(tm)
            for k in (m, m + 1):
                if 2 <= k <= n:
                    J[row:row + 3, lcol(k):lcol(k) + 3] = -cr * A @ dTl
        for m in range(2, n + 1):
            row = f3row(m)
            J[row:row + 3, cY:cY + 3] = I3
            for k in range(1, m + 1):                               # J32
                w = 1.0 if (k == 1 or k == m) else 2.0
                J[row:row + 3, ucol(k):ucol(k) + 3] = 0.5 * p.dL * w * _cross_right(t[s + k - 1])
            J[row:row + 3, lcol(m):lcol(m) + 3] = ct * I3            # J33
            if m + 1 <= n:
                J[row:row + 3, lcol(m + 1):lcol(m + 1) + 3] = -ct * I3
        blocks.append(J)
    return blocks


def filament_mobility(p: Params, Yf, model):
    """6N x 6N matrix mapping (F_m, T_m) to (V_n, Omega_n) within one filament
    (index 6n + c). model 'drag': the diagonal self mobility of App. B
    (1/(6 pi eta a), 1/(8 pi eta a^3)); model 'rpy': the RPY blocks of every
    pair of segments of this filament (Sec. 2.7.1, same branches as rpy.c)."""
    n = Yf.shape[0]
    Mf = np.zeros((6 * n, 6 * n))
    if model == "drag":
        for k in range(n):
            Mf[6 * k:6 * k + 3, 6 * k:6 * k + 3] = np.eye(3) / (6.0 * PI * p.eta * p.a)
            Mf[6 * k + 3:6 * k + 6, 6 * k + 3:6 * k + 6] = np.eye(3) / (8.0 * PI * p.eta * p.a ** 3)
        return Mf
    for i in range(n):
        for j in range(n):
            tt, tr, rt, rr = rpy.pair_blocks(Yf[i] - Yf[j], i == j, p.a, p.eta)
            Mf[6 * i:6 * i + 3, 6 * j:6 * j + 3] = tt
            Mf[6 * i:6 * i + 3, 6 * j + 3:6 * j + 6] = tr
            Mf[6 * i + 3:6 * i + 6, 6 * j:6 * j + 3] = rt
            Mf[6 * i + 3:6 * i + 6, 6 * j + 3:6 * j + 6] = rr
    return Mf


def jacobian0_general(lay: Layout, p: Params, state: State, X, model="rpy"):
    """J0 = d f_0 / dX with f_0 the residual whose mobility is a per-filament
    matrix M_f held fixed at X (no dM/dY term), internal loads only, and the
    derivative approximations of App. B.2 (d t/d u = [x t], frame-vector
    moments, three-term dexpinv):

      position rows n:  I (Y_1) + arm terms - b dt (M_f G)_{V_n}
      rotation rows n:  I (u_n) - b dt [A_n (M_f G)_{Omega_n}
                         + delta_{u_n}(-[x Om_n]/2 + ([x (u_n x Om_n)] + [u_n x][x Om_n])/12)]

    with G = d(F, T)/dX the App. B.2 load derivatives, A_n = I - [u_n x]/2 +
    [u_n x]^2/12, Om_n the internal-load angular velocity at X and b the scheme
    weight. With model='drag' (M_f = self mobility) this is exactly the J0 of
    App. B.2; model='rpy' keeps every segment-segment RPY block of the filament
    (the coupling along a filament that the drag model drops)."""
    _, _, be, _ = scheme(state)
    bdt = be * p.dt
    q, t, Y, u, lam = unpack(lay, p, X, state.q)
    _, mu, nu = frames(q)
    Fi, Ti = forces_torques(lay, p, q, t, lam, None)
    I3 = np.eye(3)
    blocks = []
    for i, n in enumerate(lay.N):
        s = lay.off_seg[i]
        nX = 6 * n
        L = np.zeros((n + 1, 3))
        L[1:n] = lam[lay.off_lam[i]:lay.off_lam[i + 1]]

        def ucol(k):          # u_k, k = 0..N-1
            return 3 + 3 * k

        def lcol(j):          # Lambda joint j (between k = j and j+1), j = 0..N-2
            return 3 + 3 * n + 3 * j

        G = np.zeros((6 * n, nX))             # rows 6m + c: (F_m, T_m)
        Da = [None] * n
        Db = [None] * n
        for j in range(n - 1):
            Da[j], Db[j] = _dM_du(p, t[s + j], t[s + j + 1], mu[s + j], mu[s + j + 1],
                                  nu[s + j], nu[s + j + 1])
        for m in range(n):
            # F_m = Lam[m] - Lam[m-1]  (Lam[k] here = L[k+1])
            if m <= n - 2:
                G[6 * m:6 * m + 3, lcol(m):lcol(m) + 3] += I3
                G[6 * m + 3:6 * m + 6, lcol(m):lcol(m) + 3] += 0.5 * p.dL * _cross_left(t[s + m])
            if m >= 1:
                G[6 * m:6 * m + 3, lcol(m - 1):lcol(m - 1) + 3] -= I3
                G[6 * m + 3:6 * m + 6, lcol(m - 1):lcol(m - 1) + 3] += \
                    0.5 * p.dL * _cross_left(t[s + m])
            dT = 0.5 * p.dL * _cross_right(L[m + 1] + L[m]) @ _cross_right(t[s + m])
            if m <= n - 2:
                dT = dT + Da[m]
                G[6 * m + 3:6 * m + 6, ucol(m + 1):ucol(m + 1) + 3] += Db[m]
            if m >= 1:
                dT = dT - Db[m - 1]
                G[6 * m + 3:6 * m + 6, ucol(m - 1):ucol(m - 1) + 3] += -Da[m - 1]
            G[6 * m + 3:6 * m + 6, ucol(m):ucol(m) + 3] += dT
        Mf = filament_mobility(p, Y[s:s + n], model)
        MG = Mf @ G
        FT = np.zeros(6 * n)
        for m in range(n):
            FT[6 * m:6 * m + 3] = Fi[s + m]
            FT[6 * m + 3:6 * m + 6] = Ti[s + m]
        Om = (Mf @ FT).reshape(n, 6)[:, 3:]
        J = np.zeros((nX, nX))
        for k in range(n):
            prow = 0 if k == 0 else 3 + 3 * n + 3 * (k - 1)
            rrow = 3 + 3 * k
            J[prow:prow + 3, 0:3] = I3
            J[prow:prow + 3, :] -= bdt * MG[6 * k:6 * k + 3, :]
            for kk in range(1, k + 1):        # arm: (dL/2) sum_{k'=1}^{k} (t_{k'-1} + t_{k'})
                for c in (kk - 1, kk):
                    J[prow:prow + 3, ucol(c):ucol(c) + 3] += 0.5 * p.dL * _cross_right(t[s + c])
            uk = u[s + k]
            ux = _cross_left(uk)
            A = I3 - 0.5 * ux + ux @ ux / 12.0
            J[rrow:rrow + 3, :] -= bdt * A @ MG[6 * k + 3:6 * k + 6, :]
            xO = _cross_right(Om[k])
            J[rrow:rrow + 3, ucol(k):ucol(k) + 3] += I3 - bdt * (
                -0.5 * xO + (_cross_right(np.cross(uk, Om[k])) + ux @ xO) / 12.0)
        blocks.append(J)
    return blocks


def tether_columns(lay: Layout, p: Params, state: State, Xr, tether: Tether, i, model):
    """The 6N x 6 columns of a tethered filament's J0 for its multipliers
    (lambda_1, lambda_2), at the resolved unknowns Xr: the loads G = d(F, T)/d
    lambda (I on F_1, D^T on T_1) through the filament mobility M_f of `model`
    ('drag': App. B.2's self mobility; 'rpy': the filament's RPY blocks),
    position rows -b dt (M_f G)_V, rotation rows -b dt A_k (M_f G)_Omega with
    A_k = I - [u_k x]/2 + [u_k x]^2/12, as the other columns of J0."""
    _, _, be, _ = scheme(state)
    bdt = be * p.dt
    _, _, Y, u, _ = unpack(lay, p, Xr, state.q)
    n, s0 = lay.N[i], lay.off_seg[i]
    Mf = filament_mobility(p, Y[s0:s0 + n], model)
    G = np.zeros((6 * n, 6))
    G[0:3, 0:3] = np.eye(3)
    G[3:6, 3:6] = dexpinv_matrix(tether.u1[i]).T
    MG = Mf @ G
    cols = np.zeros((6 * n, 6))
    for k in range(n):
        prow = 0 if k == 0 else 3 + 3 * n + 3 * (k - 1)
        rrow = 3 + 3 * k
        ux = _cross_left(u[s0 + k])
        A = np.eye(3) - 0.5 * ux + ux @ ux / 12.0
        cols[prow:prow + 3] = -bdt * MG[6 * k:6 * k + 3]
        cols[rrow:rrow + 3] = -bdt * A @ MG[6 * k + 3:6 * k + 6]
    return cols


def jacobian0_tethered(lay: Layout, p: Params, state: State, X, tether: Tether | None,
                       model="drag"):
    """J0 blocks with tethered filaments: the free J0 (App. B.2 for 'drag', the
    filament-RPY form otherwise) at the resolved unknowns, the first six
    columns of each tethered filament's block replaced by tether_columns."""
    Xr, _, _ = tether_resolve(lay, X, tether)
    blocks = (jacobian0(lay, p, state, Xr) if model == "drag"
              else jacobian0_general(lay, p, state, Xr, model))
    if tether is not None:
        for i in range(lay.M):
            if tether.mask[i]:
                blocks[i][:, 0:6] = tether_columns(lay, p, state, Xr, tether, i, model)
    return blocks


class J0Solver:
    """J0^{-1} v by a dense LU of each filament block (scipy/LAPACK)."""

    def __init__(self, lay: Layout, blocks):
        self.lay = lay
        self.lu = [scipy.linalg.lu_factor(B) for B in blocks]

    def solve(self, v):
        out = np.empty_like(v)
        for i, n in enumerate(self.lay.N):
            b = self.lay.off_X[i]
            out[b:b + 6 * n] = scipy.linalg.lu_solve(self.lu[i], v[b:b + 6 * n])
        return out


# --------------------------------------------------------------------------
# Limited-memory bad Broyden, Algorithm 2
# --------------------------------------------------------------------------

class Broyden:
    """Algorithm 2 (limited-memory bad Broyden) with H_0 = J0^{-1}.

    Each call of iterate() performs one pass of the while loop:
      dX_k = -[J0^{-1} + sum_i c_i d_i^T] f(X_k);  X_{k+1} = X_k + dX_k;
      c_{k+1} = -[J0^{-1} + sum_i c_i d_i^T] f(X_{k+1}) / ||df_k||,
      d_{k+1} = df_k / ||df_k||,  df_k = f(X_{k+1}) - f(X_k).
    """

    def __init__(self, fun, jsolve, X0, tol):
        self.fun = fun
        self.jsolve = jsolve
        self.X = np.array(X0, dtype=np.float64)
        self.f = fun(self.X)
        self.tol = tol
        self.c = []
        self.d = []
        self.k = 0

    def H(self, v):
        out = self.jsolve(v)
        for ci, di in zip(self.c, self.d):
            out = out + ci * (di @ v)
        return out

    def converged(self):
        return float(np.max(np.abs(self.f))) <= self.tol

    def iterate(self):
        dX = -self.H(self.f)
        Xn = self.X + dX
        fn = self.fun(Xn)
        df = fn - self.f
        ndf = float(np.linalg.norm(df))
        if ndf == 0.0:
            raise FloatingPointError("Broyden stalled: ||df|| = 0")
        c_new = -self.H(fn) / ndf
        d_new = df / ndf
        self.c.append(c_new)
        self.d.append(d_new)
        self.X, self.f = Xn, fn
        self.k += 1
        return self.X, self.f


# --------------------------------------------------------------------------
# One BDF2 / Lie-group timestep
# --------------------------------------------------------------------------

def extrapolate(values, order):
    """The next value of the polynomial through the last min(order + 1,
    len(values)) of values = [x^j, x^{j-1}, x^{j-2}, ...] (None entries end the
    list): Newton's backward-difference form, x_0 = sum_k nabla^k x^j, with
    nabla x^j = x^j - x^{j-1} (the polynomial's value one step ahead; order 1
    gives 2 x^j - x^{j-1}, order 2 gives 3 x^j - 3 x^{j-1} + x^{j-2})."""
    vals = []
    for v in values:
        if v is None:
            break
        vals.append(np.asarray(v, dtype=np.float64))
    vals = vals[:order + 1]
    out = np.zeros_like(vals[0])
    diff = list(vals)
    for _ in range(len(vals)):
        out = out + diff[0]
        diff = [diff[k] - diff[k + 1] for k in range(len(diff) - 1)]
    return out


ADAPTIVE = 3


def _blocks(lay: Layout, i: int):
    """Row slices of filament i: its Y_1 row (in per-filament arrays), its u
    rows (per segment) and its Lambda rows."""
    return (slice(i, i + 1), slice(lay.off_seg[i], lay.off_seg[i + 1]),
            slice(lay.off_lam[i], lay.off_lam[i + 1]))


def _histories(lay: Layout, state: State):
    """[x^j, x^{j-1}, x^{j-2}] of the Y_1, u and Lambda blocks (None where a
    level does not exist); u only once Y^{j-1} exists (else u = 0)."""
    first = [lay.off_seg[i] for i in range(lay.M)]

    def y1(a):
        return None if a is None else np.array([a[k] for k in first])

    hy = [y1(state.Y), y1(state.Yprev), y1(state.Yprev2)]
    hu = ([state.u, state.u_prev, state.u_prev2]
          if state.u is not None and state.Yprev is not None else None)
    hl = [state.lam, state.lam_prev, state.lam_prev2] if state.lam is not None else None
    return hy, hu, hl


FIT_DECAY = 0.7


def fit_theta(PQ):
    """theta of a block from its fit (P, Q): P / Q clipped to [0, 1], 0 if Q = 0."""
    P, Q = PQ
    return 0.0 if not Q > 0 else min(max(P / Q, 0.0), 1.0)


def initial_guess(lay: Layout, state: State, tether: Tether | None = None, order: int = 1):
    """X_0 of a step: each unknown extrapolated from the previous steps with
    the polynomial of degree order (1: x_0 = 2 x^j - x^{j-1}) through as many
    of its last values as exist, else the last value (order ADAPTIVE: a block
    with three values takes x_0 = 2 x^j - x^{j-1} + theta d, theta from the
    block's fit in state.xfit); the multiplier slots of tethered filaments
    linearly from the multipliers of past steps (zero before the first)."""
    hy, hu, hl = _histories(lay, state)
    if order != ADAPTIVE:
        Y1 = extrapolate(hy, order)
        u = extrapolate(hu, order) if hu is not None else np.zeros((lay.S, 3))
        lam = extrapolate(hl, order) if hl is not None else np.zeros((lay.n_lam, 3))
    else:
        fit = state.xfit if state.xfit is not None else np.zeros((lay.M, 3, 2))
        Y1 = np.zeros((lay.M, 3))
        u = np.zeros((lay.S, 3))
        lam = np.zeros((lay.n_lam, 3))
        for i in range(lay.M):
            for b, (out, hist, rows) in enumerate(zip((Y1, u, lam), (hy, hu, hl),
                                                      _blocks(lay, i))):
                if hist is None:
                    continue
                h = [None if x is None else x[rows] for x in hist]
                if any(x is None for x in h):
                    out[rows] = extrapolate(h, 2)          # fewer than three values
                else:
                    d = h[0] - 2.0 * h[1] + h[2]
                    out[rows] = 2.0 * h[0] - h[1] + fit_theta(fit[i, b]) * d
    X0 = lay.join_X(Y1, u, lam)
    if tether is not None:
        if state.tlam is not None:
            tl = 2.0 * state.tlam - state.tlam_prev if state.tlam_prev is not None else state.tlam
        else:
            tl = np.zeros((lay.M, 6))
        for i in range(lay.M):
            if tether.mask[i]:
                X0[lay.off_X[i]:lay.off_X[i] + 6] = tl[i]
    return X0


def begin_step(lay: Layout, p: Params, state: State, ext: External | None, nthreads=1,
               j0_model="drag", tether: Tether | None = None, order: int = 1,
               j0: "J0Solver | None" = None, memory=()):
    """Initial guess, J0 at it (LU-factored) and f(X_0): the set-up of Algorithm 2.

    j0_model 'drag' is App. B.2 as printed; 'rpy' keeps each filament's own
    RPY blocks in f_0 (see jacobian0_general). j0: a J0Solver of an earlier
    step to use instead (J0 kept across steps); memory: (c_i, d_i) pairs of an
    earlier step's H_k carried into H_0 = J0^{-1} + sum c_i d_i^T (the carried
    Broyden memory; the returned object's .solver is the J0 used)."""
    X0 = initial_guess(lay, state, tether, order)
    if j0 is None:
        blocks = jacobian0_tethered(lay, p, state, X0, tether, j0_model)
        j0 = J0Solver(lay, blocks)

    def fun(X):
        return residual(lay, p, state, ext, X, nthreads, tether=tether)

    br = Broyden(fun, j0.solve, X0, p.tol * p.a)
    br.c = [np.array(c, dtype=np.float64) for c, _ in memory]
    br.d = [np.array(d, dtype=np.float64) for _, d in memory]
    br.solver = j0
    return br


def adaptive_fit(lay: Layout, state: State, X):
    """The adaptive fit at a commit (before the history shift): for each
    filament and block (Y_1, u, Lambda) whose last three values exist, with
    x* the block's solution in X, l = 2 x^j - x^{j-1} and d = x^j - 2 x^{j-1}
    + x^{j-2}: P <- FIT_DECAY P + <x* - l, d>, Q <- FIT_DECAY Q + <d, d>. The
    theta = P / Q these give is the least-squares coefficient c minimising
    sum_k FIT_DECAY^age_k |x*_k - l_k - c d_k|^2 over the commits so far."""
    xs = lay.split_X(X)
    out = (state.xfit.copy() if state.xfit is not None else np.zeros((lay.M, 3, 2)))
    for b, hist in enumerate(_histories(lay, state)):
        if hist is None or any(h is None for h in hist):
            continue
        for i in range(lay.M):
            rows = _blocks(lay, i)[b]
            x0, x1, x2 = (h[rows] for h in hist)
            d = x0 - 2.0 * x1 + x2
            r = xs[b][rows] - (2.0 * x0 - x1)
            out[i, b, 0] = FIT_DECAY * out[i, b, 0] + float(np.sum(r * d))
            out[i, b, 1] = FIT_DECAY * out[i, b, 1] + float(np.sum(d * d))
    return out


def commit_step(lay: Layout, p: Params, state: State, X, tether: Tether | None = None,
                order: int = 1, iterated: bool = True):
    """q^{j+1} = exp(u*) q^j, Y^{j+1} from the robot arm, and the history shift.
    u^{j-1}, Lambda^{j-1} (and the tether multipliers of the step before) are
    kept only when they came from a committed step; with order ADAPTIVE the
    fit of the next guess is updated (adaptive_fit) unless the step took no
    Broyden iteration (iterated False: X is the guess itself, which says
    nothing about the guess's error)."""
    X, lam1, lam2 = tether_resolve(lay, X, tether)
    xfit = adaptive_fit(lay, state, X) if order == ADAPTIVE and iterated else state.xfit
    q, t, Y, u, lam = unpack(lay, p, X, state.q)
    stepped = state.steps >= 1
    tlam = np.concatenate([lam1, lam2], axis=1) if tether is not None else None
    return State(Y=Y, q=q, Yprev=state.Y.copy(), u=u, lam=lam, steps=state.steps + 1,
                 u_prev=state.u.copy() if (stepped and state.u is not None) else None,
                 lam_prev=state.lam.copy() if (stepped and state.lam is not None) else None,
                 tlam=tlam,
                 tlam_prev=(state.tlam.copy() if (tether is not None and state.tlam is not None)
                            else None),
                 Yprev2=state.Yprev.copy() if state.Yprev is not None else None,
                 u_prev2=state.u_prev.copy() if state.u_prev is not None else None,
                 lam_prev2=state.lam_prev.copy() if state.lam_prev is not None else None,
                 xfit=xfit)


def step(lay: Layout, p: Params, state: State, ext: External | None, nthreads=1,
         j0_model="drag", tether: Tether | None = None, order: int = 1):
    """One timestep; returns (new_state, iterations)."""
    br = begin_step(lay, p, state, ext, nthreads, j0_model, tether, order)
    while not br.converged():
        if br.k >= p.max_iter:
            raise RuntimeError("Broyden did not converge in %d iterations" % p.max_iter)
        br.iterate()
    return commit_step(lay, p, state, br.X, tether, order, iterated=br.k > 0), br.k


def initial_state(lay: Layout, p: Params, base, t_fil, mu_fil, xi=None, lam=None):
    """State of straight filaments with frames (t, mu) (quaternion by App. A.1),
    optionally perturbed by q_n <- exp(xi_n) q_n with positions rebuilt along
    the robot arm so that the constraint holds."""
    q = np.empty((lay.S, 4))
    qf = quat_from_frame(t_fil, mu_fil)
    for i in range(lay.M):
        q[lay.off_seg[i]:lay.off_seg[i + 1]] = qf[i]
    if xi is not None:
        q = qmul(qexp(xi), q)
    t, _, _ = frames(q)
    Y = robot_arm_positions(lay, np.asarray(base, dtype=np.float64).reshape(-1, 3), t, p.dL)
    return State(Y=Y, q=q, lam=lam)

"""FP64 reference of the warm-start network's inputs, training targets and
prediction assembly (test infrastructure only).

Each 32-segment filament is described in its own frame: origin Y_1, axes the
columns t, mu, nu of R(q_1) (eq. quaternion_rotation_matrix). Inputs, per
segment n: R1^T (Y_n - Y_1), the quaternion q_1^* q_n, and R1^T F_n, R1^T T_n
with (F, T) the right-hand side of the mobility problem at the current state
(Sec. 2.5: constraint, elastic and external loads); then R1^T (X_ex - X^j)
per 3-vector of the filament's unknowns, X_ex the extrapolated initial guess
and X^j = (Y_1, u = 0, Lambda) the current state, and R1^T corr with corr =
X* - X_ex of the previous step (zero when there is none). Targets: R1^T (X* - X_ex)
per 3-vector of the filament's unknowns, X* the converged unknowns of a step
and X_ex its extrapolated initial guess; the prediction is X_ex + R1 y.
"""
import numpy as np

from oracle import filament as fo

SEG = 32


def _frame(q1):
    t, mu, nu = fo.frames(q1[None, :])
    return np.stack([t[0], mu[0], nu[0]], axis=1)       # columns t, mu, nu


def features(lay, p, state, ext, prev_corr=None):
    q = state.q
    t, _, _ = fo.frames(q)
    F, T = fo.forces_torques(lay, p, q, t, state.lam, ext)
    X_ex = fo.initial_guess(lay, state)
    X_cur = lay.join_X(np.array([state.Y[lay.off_seg[i]] for i in range(lay.M)]),
                       np.zeros((lay.S, 3)), state.lam)
    out = np.zeros((lay.M, 13 * SEG + 12 * SEG))
    for i, n in enumerate(lay.N):
        if n != SEG:
            continue
        s = lay.off_seg[i]
        R = _frame(q[s])
        qc = fo.qconj(q[s])
        for k in range(n):
            g = s + k
            row = out[i, 13 * k:13 * k + 13]
            row[0:3] = R.T @ (state.Y[g] - state.Y[s])
            row[3:7] = fo.qmul(qc, q[g])
            row[7:10] = R.T @ F[g]
            row[10:13] = R.T @ T[g]
        a = 6 * s
        d = (X_ex[a:a + 6 * n] - X_cur[a:a + 6 * n]).reshape(-1, 3)
        out[i, 13 * SEG:19 * SEG] = (d @ R).ravel()
        if prev_corr is not None:
            out[i, 19 * SEG:] = (prev_corr[a:a + 6 * n].reshape(-1, 3) @ R).ravel()
    return out


def targets(lay, state_before, X_star, X_ex):
    out = np.zeros((lay.M, 6 * SEG))
    for i, n in enumerate(lay.N):
        if n != SEG:
            continue
        s = lay.off_seg[i]
        R = _frame(state_before.q[s])
        a = 6 * s
        d = (X_star[a:a + 6 * n] - X_ex[a:a + 6 * n]).reshape(-1, 3)
        out[i] = (d @ R).ravel()                          # rows R^T d
    return out


def predict(lay, state, X_ex, y):
    X = X_ex.copy()
    for i, n in enumerate(lay.N):
        if n != SEG:
            continue
        s = lay.off_seg[i]
        R = _frame(state.q[s])
        a = 6 * s
        X[a:a + 6 * n] += (y[i].reshape(-1, 3) @ R.T).ravel()
    return X

"""FP64 reference of the steric barrier force (test infrastructure only).

Sec. 2.6, eqn (barrier-force): segments of different filaments and
non-neighbouring segments of the same filament repel with

    F^B_nm = F^S ((4 a^2 chi^2 - r^2) / (4 a^2 (chi^2 - 1)))^4 r_nm / (2a)   if r < 2 chi a,

r_nm = Y_n - Y_m, r = |r_nm|, and F^B_nm = 0 otherwise and for neighbouring
segments (|n - m| = 1) of the same filament; the barrier force on segment n is
the sum over m. Written as the plain double loop over pairs.
"""
import numpy as np


def pair_force(rvec, a, FS, chi):
    """F^B_nm for r_nm = rvec (one pair)."""
    r2 = float(np.dot(rvec, rvec))
    if r2 >= (2.0 * chi * a) ** 2:
        return np.zeros(3)
    x = (4.0 * a * a * chi * chi - r2) / (4.0 * a * a * (chi * chi - 1.0))
    return FS * x ** 4 * np.asarray(rvec, dtype=np.float64) / (2.0 * a)


def barrier_forces(seg_per_fil, Y, a, FS, chi):
    """F^B_n for every segment of one system (filament-major segment order)."""
    Y = np.asarray(Y, dtype=np.float64)
    S = len(Y)
    fil = np.repeat(np.arange(len(seg_per_fil)), seg_per_fil)
    F = np.zeros((S, 3))
    if FS == 0.0:
        return F
    for n in range(S):
        for m in range(S):
            if m == n or (fil[m] == fil[n] and abs(m - n) == 1):
                continue
            F[n] += pair_force(Y[n] - Y[m], a, FS, chi)
    return F

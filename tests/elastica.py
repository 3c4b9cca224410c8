"""Equilibrium of a clamped elastica under a tip force (Sec. 4.1, after Landau
& Lifshitz, Theory of Elasticity, Sec. 19): a rod of length l and bending
modulus K_B, clamped horizontally at s = 0, carries a force F of fixed
direction at s = l. The angle theta(s) between its tangent and the force obeys

    s = sqrt(K_B / (2F)) * int_{theta(s)}^{pi/2} dphi / sqrt(cos theta(l) - cos phi),

with theta(0) = pi/2 and theta(l) fixed by s = l. Evaluated by quadrature
after the substitution phi = theta_l + w^2, which removes the inverse square
root singularity at phi = theta_l; cos a - cos b is written as
2 sin((a + b)/2) sin((b - a)/2) so that it keeps its digits near w = 0.
Used only by the tests.
"""
import numpy as np
from scipy import integrate, optimize


def _integral(th_l, th_from):
    """int_{th_from}^{pi/2} dphi / sqrt(cos th_l - cos phi), th_from >= th_l."""
    def f(w):
        if w == 0.0:
            return 2.0 / np.sqrt(np.sin(th_l))
        return 2.0 * w / np.sqrt(2.0 * np.sin(th_l + 0.5 * w * w) * np.sin(0.5 * w * w))
    return integrate.quad(f, np.sqrt(th_from - th_l), np.sqrt(0.5 * np.pi - th_l),
                          epsabs=1e-14, epsrel=1e-13, limit=400)[0]


def tip_angle(ell, F, KB):
    """theta(l) of the equilibrium."""
    c = np.sqrt(KB / (2.0 * F))
    return optimize.brentq(lambda th: c * _integral(th, th) - ell, 1e-8, 0.5 * np.pi - 1e-12,
                           xtol=1e-15)


def angles(s, ell, F, KB):
    """theta(s) at the arc lengths s (array) of the equilibrium."""
    c = np.sqrt(KB / (2.0 * F))
    th_l = tip_angle(ell, F, KB)
    out = []
    for si in np.atleast_1d(s):
        if si <= 0.0:
            out.append(0.5 * np.pi)
            continue
        out.append(optimize.brentq(lambda th: c * _integral(th_l, th) - si, th_l,
                                   0.5 * np.pi, xtol=1e-15))
    return np.array(out)

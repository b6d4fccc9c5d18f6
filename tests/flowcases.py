"""Closed-form flows used to build oracle and GPU test inputs (face sample
series and initial fields from an analytic velocity field)."""
import numpy as np


def faces_from(fn, E, J, K, j0=0):
    """Coarse face samples [J][6][3][E][E] of fn(X, Y, Z, t) at t = j K."""
    S = np.zeros((J, 6, 3, E, E))
    ar = np.arange(E)
    Qg, Pg = np.meshgrid(ar, ar, indexing="ij")
    for j in range(J):
        t = float((j0 + j) * K)
        for f in range(6):
            ax, val = f // 2, (0 if f % 2 == 0 else E - 1)
            V = np.full_like(Pg, val)
            X, Y, Z = {0: (V, Pg, Qg), 1: (Pg, V, Qg), 2: (Pg, Qg, V)}[ax]
            u = fn(X.astype(float), Y.astype(float), Z.astype(float), t)
            for c in range(3):
                S[j, f, c] = u[c]
    return S


def vol_from(fn, E, t=0.0):
    """Field [3][E][E][E] (layout [c][z][y][x]) of fn at time t."""
    ar = np.arange(E, dtype=float)
    Z, Y, X = np.meshgrid(ar, ar, ar, indexing="ij")
    return np.stack([np.broadcast_to(v, X.shape) for v in fn(X, Y, Z, t)]).astype(np.float64)


def abc_flow(E, tau, A=0.01, B=0.008, C=0.006):
    """Decaying Arnold-Beltrami-Childress flow, an exact unsteady solution of
    the incompressible Navier-Stokes equation with viscosity nu = (tau - 1/2)/3."""
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / E

    def fn(X, Y, Z, t):
        d = np.exp(-nu * k * k * t)
        return (d * (A * np.sin(k * Z) + C * np.cos(k * Y)),
                d * (B * np.sin(k * X) + A * np.cos(k * Z)),
                d * (C * np.sin(k * Y) + B * np.cos(k * X)))
    return fn, nu, k


def lattice_shift_state(orc, E, ufn):
    """Populations A with A_i(x) = feq_i(1, u(x + c_i)): the pulled populations
    at every interior site x are then exactly feq(1, u(x))."""
    c, _ = orc.lattice()
    A = np.zeros((19, E, E, E))
    ar = np.arange(E, dtype=float)
    Z, Y, X = np.meshgrid(ar, ar, ar, indexing="ij")
    for i in range(19):
        u = np.stack(ufn(X + c[i, 0], Y + c[i, 1], Z + c[i, 2]))
        uu = (u * u).sum(0)
        cu = c[i, 0] * u[0] + c[i, 1] * u[1] + c[i, 2] * u[2]
        w = 1 / 3 if i == 0 else (1 / 18 if i < 7 else 1 / 36)
        A[i] = w * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    return A

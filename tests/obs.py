"""Gauge-invariant observables written directly in numpy for the tests.

They are independent of the oracle and of the CUDA library: Wilson loops and
Polyakov loops are unchanged by any gauge transformation U_mu(x) -> g(x) U_mu(x)
g(x+mu)^dagger, which is all that a gauge-fixing sweep may do to a field.
Fields are canonical complex128 arrays of shape (Lt, Lz, Ly, Lx, 4, 3, 3).
"""
import numpy as np

AXIS = (3, 2, 1, 0)  # site-array axis that moves in direction mu


def dag(m):
    return np.swapaxes(m.conj(), -1, -2)


def shift(a, mu, n=1):
    """a(x + n mu_hat) (periodic)."""
    return np.roll(a, -n, axis=AXIS[mu])


def plaquettes(U):
    """Re Tr of the 6 oriented plaquettes per site, shape (6, Lt, Lz, Ly, Lx)."""
    out = []
    for mu in range(4):
        for nu in range(mu + 1, 4):
            p = U[..., mu, :, :] @ shift(U[..., nu, :, :], mu) @ dag(shift(U[..., mu, :, :], nu)) @ dag(U[..., nu, :, :])
            out.append(np.trace(p, axis1=-2, axis2=-1).real)
    return np.array(out)


def rectangles(U):
    """Re Tr of the 2x1 loops (2 steps mu, 1 step nu) for mu != nu, per site."""
    out = []
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            Umu, Unu = U[..., mu, :, :], U[..., nu, :, :]
            p = (Umu @ shift(Umu, mu) @ shift(Unu, mu, 2) @ dag(shift(shift(Umu, mu), nu))
                 @ dag(shift(Umu, nu)) @ dag(Unu))
            out.append(np.trace(p, axis1=-2, axis2=-1).real)
    return np.array(out)


def polyakov(U, mu=3):
    """Tr of the product of links around direction mu, per starting site."""
    L = U.shape[AXIS[mu]]
    P = U[..., mu, :, :].copy()
    cur = U[..., mu, :, :]
    for k in range(1, L):
        P = P @ shift(cur, mu, k)
    return np.trace(P, axis1=-2, axis2=-1)


def unitarity_error(U):
    m = U.reshape(-1, 3, 3)
    return float(np.abs(m @ dag(m) - np.eye(3)).max())


def det_error(U):
    m = U.reshape(-1, 3, 3)
    return float(np.abs(np.linalg.det(m) - 1).max())

"""CPU oracle for Fourier-accelerated steepest descent (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's CPU
baseline, never by the CUDA path.  Plain numpy in FP64, one step of the paper's
Algorithm 2 at a time, in its order:

  Delta(x)                         (Eq. (3); the argument of Eqs. (7)-(8), Eq. (9))
  for every element of the 3x3 matrix Delta: FFT, multiply by p^2_max / p^2,
      inverse FFT, normalise       (Eq. (8); numpy's inverse FFT carries the 1/N)
  g(x) = reunit(1 + (alpha/2) Delta~(x))   (first-order exponential + reunitarisation, Sec. 1)
  U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger for every mu
  F, theta                          (Eqs. (1)-(3))

p^2(k) = sum_{mu<nd} 4 sin^2(pi k_mu / L_mu) are the eigenvalues of the lattice
Laplacian -d^2 (Sec. 1 after Eq. (9)); p^2_max = 4 nd; the k = 0 mode of Delta vanishes
exactly (Delta is a lattice divergence) and is set to zero.  Landau gauge transforms
over the four directions, Coulomb gauge over the three spatial ones (separately per
time slice).

Readings of the paper used here, each with its reason: the argument of Eq. (7),
sum_nu Delta_{-nu}[U_nu - U_nu^dagger] - trace, is Delta(x) of Eq. (3) (the same
expression written with the backward difference of Eq. (9)); Algorithm 2's
normalisation is the 1/N of the inverse transform (a transform pair must carry it once
and numpy's inverse does); the first-order exponential with reunitarisation is
reunit(1 + (alpha/2) Delta~), the exponential's series cut after its linear term
(Sec. 1 after Eq. (9)); a converged Coulomb slice keeps g = 1 while the others move
(each slice has its own stop rule, as in the overrelaxation).
"""
from __future__ import annotations

import numpy as np

# axes of the site array (t, z, y, x) that carry the gauge directions
_AXES = {0: (0, 1, 2, 3), 1: (1, 2, 3)}


def _nd(gauge: int) -> int:
    return 4 if gauge == 0 else 3


def p2_grid(shape4, gauge: int) -> np.ndarray:
    """p^2(k) broadcast over the site array (Lt, Lz, Ly, Lx); 0 along the axes not transformed."""
    p2 = np.zeros(shape4)
    for ax in _AXES[gauge]:
        L = shape4[ax]
        k = np.arange(L)
        s = 4.0 * np.sin(np.pi * k / L) ** 2
        sh = [1, 1, 1, 1]
        sh[ax] = L
        p2 = p2 + s.reshape(sh)
    return p2


def fourier_filter(shape4, gauge: int, kind: str = "fourier") -> np.ndarray:
    """p^2_max / p^2 (0 at p^2 = 0), or 1 everywhere for kind == 'none'."""
    if kind == "none":
        return np.ones(shape4)
    p2 = p2_grid(shape4, gauge)
    p2max = 4.0 * _nd(gauge)
    out = np.zeros(shape4)
    nz = p2 > 0
    out[nz] = p2max / p2[nz]
    return out


def filtered_delta(D: np.ndarray, gauge: int, kind: str = "fourier") -> np.ndarray:
    """F^-1 [filter * F Delta] for each of the 9 matrix elements (Algorithm 2's inner loop)."""
    axes = _AXES[gauge]
    filt = fourier_filter(D.shape[:4], gauge, kind)
    out = np.empty_like(D)
    for i in range(3):
        for j in range(3):
            Fk = np.fft.fftn(D[..., i, j], axes=axes)
            Fk = Fk * filt
            out[..., i, j] = np.fft.ifftn(Fk, axes=axes)
    return out


def _reunit_rows(g: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1) (as the links' reunitarisation)."""
    r0 = g[..., 0, :] / np.sqrt(np.sum(np.abs(g[..., 0, :]) ** 2, axis=-1))[..., None]
    r1 = g[..., 1, :] - np.sum(r0.conj() * g[..., 1, :], axis=-1)[..., None] * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1))[..., None]
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def gauge_from_update(Dt: np.ndarray, alpha: float) -> np.ndarray:
    """g(x) = reunit(1 + (alpha / 2) Delta~(x))."""
    g = np.eye(3, dtype=np.complex128) + 0.5 * alpha * Dt
    return _reunit_rows(g)


def apply_gauge(U: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U_mu(x) <- g(x) U_mu(x) g(x + mu)^dagger, every mu (Algorithm 2, last loop)."""
    gd = np.swapaxes(g.conj(), -1, -2)
    out = np.empty_like(U)
    for mu, ax in enumerate((3, 2, 1, 0)):
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ np.roll(gd, -1, axis=ax)
    return out


def fa_sd_step(U: np.ndarray, alpha: float = 0.08, gauge: int = 0, kind: str = "fourier",
               delta_fn=None, slice_active=None) -> np.ndarray:
    """One iteration of Algorithm 2; returns the new field (U is not modified).
    slice_active (Coulomb gauge, Lt booleans): g = 1 on the sites of inactive slices."""
    if delta_fn is None:
        from oracle import delta as delta_fn
    D = delta_fn(U, gauge)
    Dt = filtered_delta(D, gauge, kind)
    g = gauge_from_update(Dt, alpha)
    if slice_active is not None:
        g[~np.asarray(slice_active, bool)] = np.eye(3)
    return apply_gauge(U, g)


def sd_step(U: np.ndarray, alpha: float = 0.08, gauge: int = 0, delta_fn=None) -> np.ndarray:
    """Naive steepest descent, Eq. (7): g = reunit(1 + (alpha/2) Delta), no Fourier filter."""
    if delta_fn is None:
        from oracle import delta as delta_fn
    D = delta_fn(U, gauge)
    return apply_gauge(U, gauge_from_update(D, alpha))


def fa_sd_fix(U: np.ndarray, eps: float, maxiter: int, alpha: float = 0.08, gauge: int = 0,
              kind: str = "fourier", per_slice: bool = False, reunit_interval: int = 0):
    """Algorithm 2: measure; while theta >= eps and fewer than maxiter steps: step; measure.
    per_slice (Coulomb gauge): each time slice stops on its own theta_t < eps and then
    keeps g = 1.  reunit_interval > 0: the links are reunitarised after every such
    number of iterations.  Returns (U, dict(rc, iters, F, theta, theta_hist, slice_iters))."""
    from oracle import measure, reunit
    F, th, _, th_t = measure(U, gauge)
    active = (th_t >= eps) if per_slice else np.full(U.shape[0], th >= eps)
    slice_iters = np.zeros(U.shape[0], dtype=int)
    hist = [th]
    it = 0
    while active.any() and it < maxiter:
        U = fa_sd_step(U, alpha, gauge, kind, slice_active=active if per_slice else None)
        slice_iters += active
        it += 1
        if reunit_interval > 0 and it % reunit_interval == 0:
            U = reunit(np.ascontiguousarray(U))
        F, th, _, th_t = measure(U, gauge)
        hist.append(th)
        active = (active & (th_t >= eps)) if per_slice else np.full(U.shape[0], th >= eps)
    return U, dict(rc=0 if not active.any() else 1, iters=it, F=F, theta=th, theta_hist=np.array(hist),
                   slice_iters=slice_iters)

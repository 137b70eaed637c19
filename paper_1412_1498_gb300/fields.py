"""Seeded synthetic SU(3) gauge fields: the inputs shared by the CUDA path and the oracle.

This module draws and shapes input data only.  It holds none of the gauge-fixing
arithmetic (no K(x), no subgroup maximisation, no F or theta): both the CUDA library
and the CPU oracle receive the arrays made here and nothing else.

Canonical layout (shared with the C ABI): a C-contiguous complex128 array of shape
(Lt, Lz, Ly, Lx, 4, 3, 3): site index t, z, y, x with x fastest, then the direction
mu = 0..3 (mu = 3 is time), then the 3x3 link matrix U_mu(x) in row-major order.

The field recipe is the one used for the workloads of the paper's experiments
(Section 3: Landau and Coulomb gauge fixing of SU(3) configurations on 32^4-class
lattices).  Those were MILC ensembles; seeded synthetic fields stand in for them:

  U_mu(x) = exp(i * eps * A_mu(x)),  A = sum_a c_a lambda_a,  c_a ~ N(0, 1)

(the exponential in closed form, see expi_hermitian)

(lambda_a the Gell-Mann matrices), followed by a Haar-random gauge transformation
U_mu(x) -> g(x) U_mu(x) g(x + mu)^dagger.  The random numbers come from numpy's
Philox counter-based generator keyed by (seed, purpose), so every platform draws the
same numbers.  Normals are drawn in the order (t, z, y, x, mu, a).
"""
from __future__ import annotations

import numpy as np

_PURPOSE_FIELD = 0
_PURPOSE_GAUGE = 1
_PURPOSE_EPS = 2


def _rng(seed: int, purpose: int) -> np.random.Generator:
    # Philox key: low 64 bits = seed, high 64 bits = purpose.
    return np.random.Generator(np.random.Philox(key=int(seed) + (int(purpose) << 64)))


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3), Tr(l_a l_b) = 2 delta_ab."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


def expi_hermitian_eigh(A: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*A) for a stack of Hermitian matrices A (..., 3, 3), by eigendecomposition."""
    w, Q = np.linalg.eigh(A)
    return (Q * np.exp(1j * eps * w)[..., None, :]) @ np.swapaxes(Q.conj(), -1, -2)


def expi_hermitian(A: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*A) for a stack of traceless Hermitian 3x3 matrices, in closed form.

    Cayley-Hamilton: exp(iQ) = f0 + f1 Q + f2 Q^2 with f_j from the invariants
    c0 = det Q, c1 = Tr Q^2 / 2 (C. Morningstar and M. Peardon, "Analytic smearing of SU(3)
    link variables in lattice QCD", Phys. Rev. D 69, 054501 (2004), Sec. III).  Only
    elementwise numpy operations: much faster than a batched eigensolver on millions of
    matrices; checked against scipy's expm and the eigendecomposition in the tests.
    """
    Q = eps * np.asarray(A, dtype=np.complex128)
    Q2 = Q @ Q
    c0 = np.real(np.einsum("...ij,...ji->...", Q, Q2)) / 3.0
    c1 = np.real(np.einsum("...ii->...", Q2)) / 2.0
    neg = c0 < 0
    c0a = np.abs(c0)
    c0max = 2.0 * (c1 / 3.0) ** 1.5
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(c0max > 0, c0a / np.where(c0max > 0, c0max, 1.0), 0.0)
    th = np.arccos(np.clip(r, -1.0, 1.0))
    u = np.sqrt(c1 / 3.0) * np.cos(th / 3.0)
    w = np.sqrt(c1) * np.sin(th / 3.0)
    w2 = w * w
    small = np.abs(w) < 0.05
    with np.errstate(invalid="ignore", divide="ignore"):
        xi0 = np.where(small, 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0)),
                       np.sin(w) / np.where(small, 1.0, w))
    e2iu = np.exp(2j * u)
    emiu = np.exp(-1j * u)
    u2 = u * u
    h0 = (u2 - w2) * e2iu + emiu * (8 * u2 * np.cos(w) + 2j * u * (3 * u2 + w2) * xi0)
    h1 = 2 * u * e2iu - emiu * (2 * u * np.cos(w) - 1j * (3 * u2 - w2) * xi0)
    h2 = e2iu - emiu * (np.cos(w) + 3j * u * xi0)
    den = 9 * u2 - w2
    tiny = c1 < 1e-24                                   # Q ~ 0: Taylor
    den = np.where(tiny, 1.0, den)
    f0 = np.where(tiny, 1.0 - c1, h0 / den)
    f1 = np.where(tiny, 1.0j, h1 / den)
    f2 = np.where(tiny, -0.5, h2 / den)
    f0 = np.where(neg, np.conj(f0), f0)
    f1 = np.where(neg, -np.conj(f1), f1)
    f2 = np.where(neg, np.conj(f2), f2)
    eye = np.eye(3, dtype=np.complex128)
    return f0[..., None, None] * eye + f1[..., None, None] * Q + f2[..., None, None] * Q2


def haar_su3(n: int, rng: np.random.Generator) -> np.ndarray:
    """n Haar-distributed SU(3) matrices.

    Complex Ginibre matrix -> QR -> fix the phases of R's diagonal (Mezzadri 2007,
    "How to generate random matrices from the classical compact groups") gives a
    Haar U(3) matrix; dividing by a cube root of its determinant maps it to SU(3).
    """
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q / np.exp(1j * np.angle(det) / 3.0)[..., None, None]


def smooth_field(dims, eps: float, seed: int) -> np.ndarray:
    """U_mu(x) = exp(i eps A_mu(x)) with A = sum_a c_a lambda_a, c_a ~ N(0,1) i.i.d."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    rng = _rng(seed, _PURPOSE_FIELD)
    c = rng.standard_normal((Lt, Lz, Ly, Lx, 4, 8))
    A = np.einsum("...a,aij->...ij", c, gell_mann(), optimize=True)
    return np.ascontiguousarray(expi_hermitian(A, eps))


def gauge_field(dims, seed: int) -> np.ndarray:
    """Haar-random g(x), shape (Lt, Lz, Ly, Lx, 3, 3)."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    g = haar_su3(Lx * Ly * Lz * Lt, _rng(seed, _PURPOSE_GAUGE))
    return g.reshape(Lt, Lz, Ly, Lx, 3, 3)


def gauge_transform(U: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U_mu(x) -> g(x) U_mu(x) g(x + mu)^dagger on a periodic lattice (input recipe step)."""
    out = np.empty_like(U)
    gd = np.swapaxes(g.conj(), -1, -2)
    # axis of the site array that moves in direction mu: x=3, y=2, z=1, t=0
    for mu, axis in enumerate((3, 2, 1, 0)):
        g_fwd_dag = np.roll(gd, -1, axis=axis)
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ g_fwd_dag
    return out


def random_gauge_config(dims, eps: float, seed: int, gauge_seed: int | None = None) -> np.ndarray:
    """Smooth field with seed `seed`, then a Haar gauge transformation with `gauge_seed`.

    gauge_seed defaults to `seed`; the two draws still come from different streams
    because the purpose word of the Philox key differs.
    """
    for d in dims:
        if int(d) < 2 or int(d) % 2:
            raise ValueError(f"every lattice extent must be even and >= 2, got {tuple(dims)}")
    U = smooth_field(dims, eps, seed)
    g = gauge_field(dims, seed if gauge_seed is None else gauge_seed)
    return gauge_transform(U, g)


def pure_gauge_config(dims, seed: int) -> np.ndarray:
    """U_mu(x) = h(x) h(x+mu)^dagger with Haar h: a gauge transform of the unit field."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), (Lt, Lz, Ly, Lx, 4, 3, 3)).copy()
    return gauge_transform(one, gauge_field(dims, seed))


def ensemble_eps(seed: int, lo: float = 0.3, hi: float = 0.6) -> float:
    """Per-configuration eps ~ U[lo, hi] for ensemble workloads, from the config's own stream."""
    return float(_rng(seed, _PURPOSE_EPS).uniform(lo, hi))


def _ensemble_member(args):
    d, s = args
    return random_gauge_config(tuple(d), ensemble_eps(s), s)


def ensemble(dims_list, seeds, workers: int = 1):
    """One smooth-plus-random-gauge field per (dims, seed); eps ~ U[0.3, 0.6] is drawn
    from each seed's own stream.

    workers > 1 draws the members in that many processes (started with "spawn", so it is
    safe after CUDA was initialised in the caller); every member depends only on its own
    (dims, seed), so the fields are the same for any number of workers.  A spawned worker
    imports the caller's main module, so a script that asks for workers must keep its
    top-level work under an ``if __name__ == "__main__":`` guard.
    """
    jobs = [(tuple(int(v) for v in d), int(s)) for d, s in zip(dims_list, seeds)]
    if workers <= 1 or len(jobs) <= 1:
        return [_ensemble_member(j) for j in jobs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_ensemble_member, jobs, chunksize=1)


def to_host_layout(U: np.ndarray) -> np.ndarray:
    """Interleaved (re, im) float64 view of a canonical complex128 field (what the C ABI takes)."""
    return np.ascontiguousarray(U).view(np.float64)

"""Pins for the seeded input generator (no GPU)."""
import numpy as np
import pytest
import scipy.linalg

from paper_1412_1498_gb300 import fields
from tests import obs


def test_gell_mann_algebra():
    l = fields.gell_mann()
    for a in range(8):
        assert np.allclose(l[a], l[a].conj().T)
        assert abs(np.trace(l[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(l[a] @ l[b]) - 2 * (a == b)) < 1e-14
    # textbook structure constants f_123 = 1, f_458 = sqrt(3)/2: [l_a, l_b] = 2i f_abc l_c
    def f(a, b, c):
        return (np.trace((l[a] @ l[b] - l[b] @ l[a]) @ l[c]) / 4j).real
    assert abs(f(0, 1, 2) - 1) < 1e-14
    assert abs(f(3, 4, 7) - np.sqrt(3) / 2) < 1e-14
    assert abs(f(0, 3, 6) - 0.5) < 1e-14


def test_expi_matches_library_expm():
    rng = np.random.default_rng(0)
    for scale in (1e-9, 1e-3, 0.7, 3.0):
        for _ in range(20):
            c = rng.standard_normal(8)
            A = np.einsum("a,aij->ij", c, fields.gell_mann())
            ref = scipy.linalg.expm(1j * scale * A)
            assert np.abs(fields.expi_hermitian(A[None], scale)[0] - ref).max() < 1e-13
            assert np.abs(fields.expi_hermitian_eigh(A[None], scale)[0] - ref).max() < 1e-13
    # both signs of det and degenerate spectra
    for A in (np.diag([1.0, 1.0, -2.0]), np.diag([-1.0, -1.0, 2.0]), np.zeros((3, 3)), fields.gell_mann()[2]):
        A = A.astype(complex)
        ref = scipy.linalg.expm(1j * 0.9 * A)
        assert np.abs(fields.expi_hermitian(A[None], 0.9)[0] - ref).max() < 1e-13


def test_smooth_field_is_su3_and_deterministic():
    U = fields.smooth_field((4, 4, 4, 4), 0.5, 7)
    assert obs.unitarity_error(U) < 1e-14
    assert obs.det_error(U) < 1e-13
    assert np.array_equal(U, fields.smooth_field((4, 4, 4, 4), 0.5, 7))
    assert not np.array_equal(U, fields.smooth_field((4, 4, 4, 4), 0.5, 8))


def test_haar_moments():
    g = fields.haar_su3(100000, np.random.Generator(np.random.Philox(key=11)))
    assert obs.unitarity_error(g) < 1e-13
    assert obs.det_error(g) < 1e-13
    m2 = (np.abs(g) ** 2).mean(axis=0)           # E|U_ij|^2 = 1/3
    assert np.abs(m2 - 1 / 3).max() < 4 * np.sqrt(0.08 / 100000) + 1e-3
    tr = np.trace(g, axis1=1, axis2=2)            # E Tr U = 0, E |Tr U|^2 = 1 for Haar SU(3)
    assert abs(tr.mean()) < 4 / np.sqrt(100000) * 1.5
    assert abs((np.abs(tr) ** 2).mean() - 1) < 0.03


def test_gauge_transform_keeps_invariants():
    U = fields.smooth_field((4, 4, 4, 6), 0.5, 3)
    V = fields.random_gauge_config((4, 4, 4, 6), 0.5, 3)
    assert np.abs(obs.plaquettes(U) - obs.plaquettes(V)).max() < 1e-12
    assert np.abs(obs.polyakov(U) - obs.polyakov(V)).max() < 1e-12
    assert np.abs(U - V).max() > 0.1


def test_odd_extent_rejected():
    with pytest.raises(ValueError):
        fields.random_gauge_config((4, 4, 3, 4), 0.5, 1)


def test_ensemble_is_the_same_for_any_number_of_workers():
    # each member depends only on its own (dims, seed): the process pool changes nothing
    dims_list = [(4, 4, 4, 4), (6, 4, 4, 2), (4, 4, 2, 6)]
    seeds = [100, 101, 102]
    a = fields.ensemble(dims_list, seeds, workers=1)
    b = fields.ensemble(dims_list, seeds, workers=3)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert all(x.shape == (d[3], d[2], d[1], d[0], 4, 3, 3) for x, d in zip(a, dims_list))

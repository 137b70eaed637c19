"""Compact link storages against the oracle (needs a GB300): FP64-12 (rows 0 and 1) and
the 8-real parametrisation (u01, u02, u10 and the phases of u00 and u20, Section 2's
third storage option) in FP32 and FP64.

Tolerances.  FP64-12 rebuilds row 2 from rows 0 and 1 (a few roundings), so it takes
the FP64-18 bounds.  The 8-real rebuild takes two square roots of differences,
|u00| = sqrt(1 - N) and |u20| = sqrt(N - |u10|^2) with N = |u01|^2 + |u02|^2: an absolute
error u of the radicand becomes ~u / (2 |u00|) or ~u / (2 |u20|) in the modulus, and
the divisions by N pass it on to u11, u12 at most unchanged.  So a stored and reloaded
link is exact to  B = C u (1 + 1 / min|u00| + 1 / min|u20|)  with u the unit roundoff of
the storage, taken over the field; C = 16 covers the few roundings of each term.
"""
import numpy as np
import pytest

import oracle
from paper_1412_1498_gb300 import fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (10, 8, 6, 4)
DIMS_C = (6, 4, 6, 8)
U64, U32 = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module")
def gf():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1412_1498_gb300 import build
    build.build()
    from paper_1412_1498_gb300 import gf as m
    return m


def rebuild_bound(U, unit):
    """B above for the links of U (canonical layout, any shape ending in 3x3)."""
    m = U.reshape(-1, 3, 3)
    a00 = np.abs(m[:, 0, 0]).min()
    u20 = np.conj(m[:, 0, 1] * m[:, 1, 2] - m[:, 0, 2] * m[:, 1, 1])
    return 16.0 * unit * (1.0 + 1.0 / a00 + 1.0 / np.abs(u20).min())


def unit_of(gf, storage):
    return U32 if storage == gf.GF_FP32_8 else U64


@pytest.mark.parametrize("storage", [3, 4, 5])
def test_roundtrip(gf, storage):
    U = fields.random_gauge_config(DIMS, 0.5, 41)
    fx = gf.GaugeFixer(DIMS, gf.GF_LANDAU, storage)
    fx.upload(U)
    got = fx.download()
    if storage == gf.GF_FP64_12:
        assert np.array_equal(got[..., :2, :], U[..., :2, :])
        # row 2 = conj(row0 x row1) to a few roundings; U's own row 2 differs from that
        # by U's unitarity defect
        r2 = np.conj(np.cross(U[..., 0, :], U[..., 1, :]))
        assert np.abs(got[..., 2, :] - r2).max() < 8 * U64
        assert np.abs(got[..., 2, :] - U[..., 2, :]).max() < 8 * U64 + np.abs(U[..., 2, :] - r2).max()
    else:
        # the stored elements come back as stored (FP32: rounded once)
        dt = np.complex64 if storage == gf.GF_FP32_8 else np.complex128
        r = U.astype(dt).astype(np.complex128)
        assert np.array_equal(got[..., 0, 1:], r[..., 0, 1:])
        assert np.array_equal(got[..., 1, 0], r[..., 1, 0])
        assert np.abs(got - U).max() < rebuild_bound(U, unit_of(gf, storage))
        # and form an SU(3) matrix
        m = got.reshape(-1, 3, 3)
        eye = np.einsum("nij,nkj->nik", m, m.conj())
        tol = 64 * unit_of(gf, storage) / np.abs(m[:, 0, 0]).min()
        assert np.abs(eye - np.eye(3)).max() < max(tol, 1e-5 if storage == gf.GF_FP32_8 else 1e-12)
    # device buffers
    Ud = torch.from_numpy(U).cuda()
    fx.upload(Ud)
    outd = torch.empty_like(Ud)
    fx.download(out=outd)
    torch.cuda.synchronize()
    assert np.array_equal(outd.cpu().numpy(), got)
    fx.close()


@pytest.mark.parametrize("storage", [4, 5])
def test_unit_field(gf, storage):
    # N = 0: the 2x2 block is e^{-i arg(u00)/2} 1, which rebuilds the unit link exactly
    U = np.zeros(DIMS[::-1] + (4, 3, 3), np.complex128)
    U[..., :, :] = np.eye(3)
    fx = gf.GaugeFixer(DIMS, gf.GF_LANDAU, storage)
    fx.upload(U)
    assert np.array_equal(fx.download(), U)
    F, th, _, _ = fx.functional_theta()
    assert F[0] == 1.0 and th[0] == 0.0
    gf.gf_or_sweep(fx.h, 2, 1.7)                    # K = 8 * 1: every maximiser is 1
    tol = 1e-6 if storage == gf.GF_FP32_8 else 1e-14  # up to the rounding of 1 / |(alpha, beta)|
    assert np.abs(fx.download() - U).max() < tol
    fx.close()


@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("storage", [3, 4, 5])
def test_functional_theta_matches_oracle(gf, gauge, storage):
    dims = DIMS if gauge == 0 else DIMS_C
    U = fields.random_gauge_config(dims, 0.5, 42)
    fx = gf.GaugeFixer(dims, gauge, storage)
    fx.upload(U)
    F, th, uF, uT = fx.functional_theta()
    V = fx.download()                               # the field as the kernels see it
    rF, rth, rFt, rtht = oracle.measure(V, gauge)
    tol = 1e-5 if storage == gf.GF_FP32_8 else 1e-12
    assert abs(F[0] - rF) <= tol * abs(rF) and abs(th[0] - rth) <= tol * rth
    if gauge == oracle.COULOMB:
        assert np.allclose(uF, rFt, rtol=tol, atol=0) and np.allclose(uT, rtht, rtol=tol, atol=0)
    fx.close()


@pytest.mark.parametrize("gauge", [0, 1])
@pytest.mark.parametrize("storage", [3, 5])
def test_fp64_compact_sweeps(gf, gauge, storage):
    dims = DIMS if gauge == 0 else DIMS_C
    U = fields.random_gauge_config(dims, 0.5, 43)
    fx = gf.GaugeFixer(dims, gauge, storage)
    fx.upload(U)
    ref = fx.download()
    for parity in (0, 1, 0):
        gf.gf_or_sweep(fx.h, parity, 1.7)
        oracle.or_half_sweep(ref, parity, 1.7, gauge, 0)
        got = fx.download()
        extra = 0.0 if storage == gf.GF_FP64_12 else rebuild_bound(ref, U64)
        assert np.abs(got - ref).max() < 1e-13 + extra
        if storage == gf.GF_FP64_8:
            ref = got.copy()                        # continue from the stored field
    # 100 sweeps with checks and reunitarisation, as the FP64-18 test
    U2 = fields.random_gauge_config(dims, 0.5, 44)
    fx.upload(U2)
    ref = fx.download()
    r = oracle.fix(ref, 1e-300, 100, 1.7, gauge, per_slice=False)
    out = fx.fix(1e-300, 100)
    got = fx.download()
    assert np.all(out["iters"] == 100)
    if storage == gf.GF_FP64_12:
        assert np.abs(got - ref).max() < 1e-10
        assert abs(out["F"][0] - r["F"]) <= 1e-12 * abs(r["F"])
    else:
        # every store re-projects onto the 8-real manifold: the runs agree in F and theta
        # to the accumulated rebuild error, and the GPU's values are those of its field
        F, th, _, _ = oracle.measure(got, gauge)
        assert abs(out["F"][0] - F) <= 1e-12 * abs(F) and abs(out["theta"][0] - th) <= 1e-9 * th
        assert abs(F - r["F"]) <= 1e-9 * abs(r["F"])
    fx.close()


@pytest.mark.parametrize("gauge", [0, 1])
def test_fp32_8_sweeps_against_fp64_oracle(gf, gauge):
    dims = DIMS if gauge == 0 else DIMS_C
    U = fields.random_gauge_config(dims, 0.5, 45)
    fx = gf.GaugeFixer(dims, gauge, gf.GF_FP32_8)
    fx.upload(U)
    ref = fx.download()
    gf.gf_or_sweep(fx.h, 2, 1.7)
    oracle.sweep(ref, 1.7, gauge)
    d = np.abs(fx.download() - ref)
    # FP32 sweep (5e-6, as 12-real) plus one rebuild of every stored link
    assert d.max() < 5e-6 + rebuild_bound(ref, U32), d.max()
    assert np.sqrt(np.mean(d * d)) < 1e-6
    F, th, _, _ = fx.functional_theta()
    rF, _, _, _ = oracle.measure(ref, gauge)
    assert abs(F[0] - rF) < 1e-5 * abs(rF)
    fx.close()


def test_fp32_8_mixed_reaches_1e15(gf):
    # the 8^4 workload through the FP32 8-real phase and the FP64 polish.  The FP32 phase
    # moves the field off its gauge orbit by the rebuild error of every store, so the
    # polish is checked against the oracle started from the field at the switch: the
    # same FP32 phase run alone (same kernels, same sweeps), converted to FP64 and
    # reunitarised as the mixed run does
    dims = (8, 8, 8, 8)
    U = fields.random_gauge_config(dims, 0.4, 1, 2)
    fa = gf.GaugeFixer(dims, gf.GF_LANDAU, gf.GF_FP32_8)
    fa.upload(U)
    oa = fa.fix(1e-8, 3000)
    Vs = fa.download()
    fa.close()
    fx = gf.GaugeFixer(dims, gf.GF_LANDAU, gf.GF_FP32_8, mixed=True)
    gf.gf_set_polish(fx.h, gf.GF_POLISH_FP64)
    fx.upload(U)
    out = fx.fix(1e-15, 3000)
    assert out["rc"] == gf.GF_OK
    n32, n64 = out["phase_sweeps"]
    assert n32 == oa["iters"][0] and n64 > 0
    got = fx.download()
    F, th, _, _ = oracle.measure(got)
    assert th < 1e-15 * (1 + 1e-6)
    ref = oracle.reunit(np.ascontiguousarray(Vs))
    r = oracle.fix(ref, 1e-15, 3000, 1.7)
    assert abs(F - r["F"]) <= 1e-12 * abs(r["F"])
    fx.close()


def test_fp64_12_fix_matches_fp64_18(gf):
    dims = (8, 8, 8, 8)
    U = fields.random_gauge_config(dims, 0.4, 1, 2)
    out = {}
    for st in (gf.GF_FP64_18, gf.GF_FP64_12):
        fx = gf.GaugeFixer(dims, gf.GF_LANDAU, st)
        fx.upload(U)
        out[st] = fx.fix(1e-12, 500)
        out[st]["U"] = fx.download()
        fx.close()
    a, b = out[gf.GF_FP64_18], out[gf.GF_FP64_12]
    assert a["rc"] == b["rc"] == gf.GF_OK
    # the two runs differ by rounding only: the stopping sweep may move by one
    assert abs(int(a["iters"][0]) - int(b["iters"][0])) <= 1
    Fa, tha, _, _ = oracle.measure(a["U"])
    Fb, thb, _, _ = oracle.measure(b["U"])
    assert tha < 1e-12 and thb < 1e-12
    assert abs(Fa - Fb) <= 1e-12 * Fa
    if a["iters"][0] == b["iters"][0]:
        assert np.abs(a["U"] - b["U"]).max() < 1e-9

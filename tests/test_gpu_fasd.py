"""Fourier-accelerated steepest descent on the GPU against the oracle (needs a GB300).

Tolerances: FP64-18 storage, per link 1e-12 after one step (the GPU's radix-2 FFT and
numpy's FFT round differently at the 1e-16 level); FP32-12 storage from the same
rounded start, per link 1e-5 after one step (FP32 FFT of length <= 64 per direction).
"""
import numpy as np
import pytest

import oracle
from oracle import fasd
from paper_1412_1498_gb300 import fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gf():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1412_1498_gb300 import build
    build.build()
    from paper_1412_1498_gb300 import gf as m
    return m


@pytest.mark.parametrize("gauge,dims", [(0, (8, 8, 8, 8)), (0, (8, 4, 16, 2)), (1, (8, 8, 4, 6)), (1, (4, 16, 8, 2)),
                                        (0, (4, 2, 4, 64)), (0, (2, 4, 64, 4)), (1, (2, 4, 64, 2))])
@pytest.mark.parametrize("storage", [0, 2])
def test_one_step_against_oracle(gf, gauge, dims, storage):
    U = fields.random_gauge_config(dims, 0.5, 95)
    fx = gf.GaugeFixer(dims, gauge, storage, fasd=True)
    fx.upload(U)
    start = fx.download()
    for k in range(2):
        gf.gf_fa_sd_step(fx.h, 0.08)
        start = fasd.fa_sd_step(start, 0.08, gauge)
        got = fx.download()
        err = np.abs(got - start).max()
        assert err < (1e-12 if storage == gf.GF_FP64_18 else 1e-5), (k, err)
    fx.close()


def test_fix_matches_oracle_iterations(gf):
    # the 8^4 workload (eps 0.4, seeds 1 / 2) with Algorithm 2, alpha 0.08, theta < 1e-12
    dims = (8, 8, 8, 8)
    U = fields.random_gauge_config(dims, 0.4, 1, 2)
    Ur, r = fasd.fa_sd_fix(U.copy(), 1e-12, 1000, 0.08)
    fx = gf.GaugeFixer(dims, gf.GF_LANDAU, gf.GF_FP64_18, fasd=True)
    gf.gf_set_method(fx.h, gf.GF_METHOD_FASD)
    gf.gf_set_reunit_interval(fx.h, 0)       # the oracle's Algorithm 2 does not reunitarise links
    fx.upload(U)
    out = fx.fix(1e-12, 1000)
    got = fx.download()
    assert out["rc"] == gf.GF_OK and out["iters"][0] == r["iters"]
    assert np.abs(got - Ur).max() < 1e-10
    assert abs(out["F"][0] - r["F"]) < 1e-12 and abs(out["theta"][0] - r["theta"]) <= 1e-8 * r["theta"]
    fx.close()


def test_coulomb_fix_per_slice_masks(gf):
    # Algorithm 2 in Coulomb gauge: 3D transforms per time slice, each slice with its own
    # stop rule (g = 1 on a converged slice); same iterations per slice and same links as
    # the oracle's per-slice loop
    dims = (8, 8, 8, 6)
    U = fields.random_gauge_config(dims, 0.5, 96)
    eps = 3e-4
    Ur, r = fasd.fa_sd_fix(U.copy(), eps, 400, 0.08, oracle.COULOMB, per_slice=True, reunit_interval=20)
    fx = gf.GaugeFixer(dims, gf.GF_COULOMB, gf.GF_FP64_18, fasd=True)
    gf.gf_set_method(fx.h, gf.GF_METHOD_FASD)
    fx.upload(U)
    out = fx.fix(eps, 400)
    assert len(set(r["slice_iters"].tolist())) > 1      # slices stop at different iterations
    assert np.array_equal(out["iters"], r["slice_iters"])
    assert (out["rc"] == gf.GF_OK) == (r["rc"] == 0)
    assert np.abs(fx.download() - Ur).max() < 1e-9
    fx.close()


def test_fasd_32x4_fp32_against_oracle_measure(gf):
    # 32^4, FP32 with FP64 reductions, seed 5, eps 0.5, alpha 0.08: theta falls, and the
    # GPU's F / theta equal the oracle's on the downloaded field
    dims = (32, 32, 32, 32)
    U = fields.random_gauge_config(dims, 0.5, 5)
    fx = gf.GaugeFixer(dims, gf.GF_LANDAU, gf.GF_FP32_12, fasd=True)
    gf.gf_set_method(fx.h, gf.GF_METHOD_FASD)
    fx.upload(U)
    th0 = fx.functional_theta()[1][0]
    out = fx.fix(1e-300, 50)
    assert out["iters"][0] == 50
    got = fx.download()
    F, th, _, _ = oracle.measure(got)
    assert th < 1e-2 * th0
    assert abs(out["F"][0] - F) < 1e-5 * abs(F) and abs(out["theta"][0] - th) < 1e-4 * th
    fx.close()


def test_budget_end_reports_final_field(gf):
    # a budget that ends before convergence: theta and F returned are the final field's
    dims = (8, 8, 8, 8)
    U = fields.random_gauge_config(dims, 0.4, 1, 2)
    fx = gf.GaugeFixer(dims, gf.GF_LANDAU, gf.GF_FP64_18, fasd=True)
    gf.gf_set_method(fx.h, gf.GF_METHOD_FASD)
    gf.gf_set_reunit_interval(fx.h, 0)
    fx.upload(U)
    out = fx.fix(1e-14, 7)
    assert out["rc"] == gf.GF_ENOTCONVERGED and out["iters"][0] == 7
    F, th, _, _ = oracle.measure(fx.download())
    assert abs(out["F"][0] - F) < 1e-12 and abs(out["theta"][0] - th) < 1e-10 * th
    Ur, r = fasd.fa_sd_fix(U.copy(), 1e-14, 7, 0.08)
    assert abs(r["theta"] - th) < 1e-8 * th
    fx.close()


def test_fasd_argument_errors(gf):
    with pytest.raises(gf.GFError):
        gf.GaugeFixer((6, 4, 4, 4), gf.GF_LANDAU, gf.GF_FP32_12, fasd=True)   # 6 not a power of 2
    with pytest.raises(gf.GFError):
        gf.GaugeFixer((4, 4, 4, 4), gf.GF_LANDAU, gf.GF_FP32_18, fasd=True)
    fx = gf.GaugeFixer((4, 4, 4, 6), gf.GF_COULOMB, gf.GF_FP32_12, fasd=True)  # t is not transformed
    fx.close()
    fx = gf.GaugeFixer((4, 4, 4, 4), gf.GF_LANDAU, gf.GF_FP32_12)
    with pytest.raises(gf.GFError):
        gf.gf_set_method(fx.h, gf.GF_METHOD_FASD)
    with pytest.raises(gf.GFError):
        gf.gf_fa_sd_step(fx.h, 0.08)
    fx.close()

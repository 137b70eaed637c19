"""gf_functional_theta_noalloc: F and theta without any allocation (needs a GPU).

Callers that cannot allocate device memory (a pre-reserved pool, a loop that must not
call cudaMalloc, a host process that owns every device allocation) pass only their
field and an output buffer.  The call must give the values of the CPU oracle's
measurement (Eqs. (1)-(3)) and of the handle-based gf_functional_theta, within the FP64
tolerance used elsewhere (1e-12 relative), on two calls in a row (the shared static
scratch keeps the previous call's contents).  This file is collected last so a
stop-at-first-failure run has run every other test.
"""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("gauge,dims", [(0, (10, 8, 6, 4)), (1, (6, 4, 6, 8)), (0, (16, 16, 16, 16))])
def test_noalloc_matches_handle(gf, gauge, dims):
    U = fields.random_gauge_config(dims, 0.5, 80 + gauge)
    fx = gf.GaugeFixer(dims, gauge, gf.GF_FP64_18)
    fx.upload(U)
    F, th, _, _ = fx.functional_theta()
    fx.close()
    rF, rth, _, _ = oracle.measure(U, gauge)
    Ud = torch.from_numpy(U).cuda()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        gf.gf_functional_theta_noalloc(dims, gauge, Ud.data_ptr(), out.data_ptr(), stream)
        got = out.cpu().numpy()
        assert abs(got[0] - rF) <= 1e-12 * abs(rF), (got, rF)
        assert abs(got[1] - rth) <= 1e-12 * rth, (got, rth)
        assert abs(got[0] - F[0]) <= 1e-12 * abs(F[0]), (got, F)
        assert abs(got[1] - th[0]) <= 1e-12 * th[0], (got, th)
        out.fill_(float("nan"))


def test_noalloc_rejects_oversized_lattice(gf):
    Ud = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(gf.GFError) as e:
        gf.gf_functional_theta_noalloc((128, 128, 128, 64), 0, Ud.data_ptr(), out.data_ptr())
    assert e.value.code == gf.GF_EINVAL
    assert "too large" in gf.gf_last_error(None)

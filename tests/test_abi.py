"""The C-ABI library loads and exports what include/gf.h declares (no GPU needed)."""
import ctypes
import subprocess

import pytest

from paper_1412_1498_gb300 import build as gfbuild

gfbuild.build()
from paper_1412_1498_gb300 import gf  # noqa: E402


def test_every_declared_symbol_is_exported():
    names = gf.header_symbols()
    assert len(names) >= 21
    lib = ctypes.CDLL(gf.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", gf.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported
    assert {s for s in exported if s.startswith("gf_")} == set(names)


def test_workspace_bytes_is_host_only_and_sized():
    # 32^4 FP32-12: 16 V link words of 48 B / 4 = 4 V links * 48 B = 201 MB of links
    V = 32 ** 4
    b = gf.gf_workspace_bytes([(32, 32, 32, 32)], gf.GF_LANDAU, gf.GF_FP32_12)
    assert 4 * V * 48 <= b < 4 * V * 48 + 64 * 2 ** 20
    bm = gf.gf_workspace_bytes([(32, 32, 32, 32)], gf.GF_LANDAU, gf.GF_FP32_12, gf.GF_FLAG_MIXED)
    assert bm - b >= 4 * V * 144
    b64 = gf.gf_workspace_bytes([(8, 8, 8, 8)], gf.GF_COULOMB, gf.GF_FP64_18)
    assert b64 >= 4 * 8 ** 4 * 144
    batch = [(16, 16, 16, 16)] * 2 + [(24, 24, 24, 24)]
    assert gf.gf_workspace_bytes(batch, gf.GF_LANDAU, gf.GF_FP32_12) >= 4 * 48 * (2 * 16 ** 4 + 24 ** 4)


@pytest.mark.parametrize("dims", [(4, 4, 3, 4), (4, 4, 4, 0), (1, 4, 4, 4), (4, -2, 4, 4)])
def test_bad_dims_rejected(dims):
    with pytest.raises(gf.GFError) as e:
        gf.gf_workspace_bytes([dims], gf.GF_LANDAU, gf.GF_FP32_12)
    assert e.value.code == gf.GF_EINVAL
    with pytest.raises(gf.GFError) as e:
        gf.gf_create(dims, 3, gf.GF_LANDAU, gf.GF_FP32_12)
    assert e.value.code == gf.GF_EINVAL
    assert "even" in gf.gf_last_error(None)


def test_bad_enums_rejected():
    for args in [(2, gf.GF_LANDAU, gf.GF_FP32_12), (3, 7, gf.GF_FP32_12), (3, gf.GF_LANDAU, 9)]:
        with pytest.raises(gf.GFError) as e:
            gf.gf_create((4, 4, 4, 4), *args)
        assert e.value.code == gf.GF_EINVAL
    with pytest.raises(gf.GFError):
        gf.gf_workspace_bytes([(4, 4, 4, 4)], gf.GF_LANDAU, gf.GF_FP32_12, flags=8)

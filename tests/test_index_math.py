"""The site decoding of the sweep kernels divides by Lx and Ly with 32-bit reciprocal
multiplies: q = umulhi(n, m) with m = ceil(2^32 / L).  With n = q L + r and
m L = 2^32 + e (0 <= e < L) this is floor(n / L + n e / (L 2^32)), exact whenever
n (L - 1) < 2^32.  The handle accepts only lattices with Lx Ly Lz max(Lx, Ly) < 2^32,
which covers every n the kernels divide (n < Lx Ly Lz for the division by Lx,
n < Ly Lz for the division by Ly).  Checked exhaustively here, in exact integer
arithmetic, for accepted lattices at the edge of that limit (no GPU needed)."""
import numpy as np
import pytest

from paper_1412_1498_gb300 import build as gfbuild

gfbuild.build()
from paper_1412_1498_gb300 import gf  # noqa: E402


def recip(L: int) -> int:
    return ((1 << 32) + L - 1) // L


def umulhi(n: np.ndarray, m: int) -> np.ndarray:
    # n < 2^32 and m <= 2^31: the product fits in 63 bits
    return (n.astype(np.uint64) * np.uint64(m)) >> np.uint64(32)


@pytest.mark.parametrize("dims", [
    (1022, 1022, 4, 2),      # Lx Ly Lz Lx = 4.27e9, just under 2^32
    (1030, 2, 2020, 2),      # large non-power-of-two Lx, Ly = 2
    (6, 1534, 300, 2),       # large non-power-of-two Ly
    (32, 32, 32, 32),
    (30, 18, 10, 6),
])
def test_reciprocal_division_is_exact_on_accepted_lattices(dims):
    Lx, Ly, Lz, _ = dims
    assert gf.gf_workspace_bytes([dims], gf.GF_LANDAU, gf.GF_FP32_12) > 0   # accepted
    n = np.arange(Lx * Ly * Lz, dtype=np.uint64)
    assert np.array_equal(umulhi(n, recip(Lx)), n // np.uint64(Lx))
    q = np.arange(Ly * Lz, dtype=np.uint64)
    assert np.array_equal(umulhi(q, recip(Ly)), q // np.uint64(Ly))


def test_limit_is_where_the_bound_stops_holding():
    # one past the accepted region the creation check refuses the lattice
    with pytest.raises(gf.GFError) as e:
        gf.gf_workspace_bytes([(1026, 1026, 4, 2)], gf.GF_LANDAU, gf.GF_FP32_12)
    assert e.value.code == gf.GF_EINVAL and "2^32" in str(e.value)
    # and the reciprocal would indeed go wrong for dividends beyond n (L - 1) < 2^32
    L = 1026
    m = recip(L)
    bad = [n for n in range((1 << 32) // (L - 1), (1 << 32) - 1, 997 * L + L - 1)
           if (n * m) >> 32 != n // L]
    assert bad, "expected a dividend past the bound where the reciprocal is off by one"


def test_volume_limit_message():
    # half-volumes and plane indices are 32-bit: fewer than 2^31 sites per lattice
    with pytest.raises(gf.GFError) as e:
        gf.gf_workspace_bytes([(2, 2, 2, 1 << 28)], gf.GF_LANDAU, gf.GF_FP32_12)
    assert e.value.code == gf.GF_EINVAL and "2^31" in str(e.value)
    with pytest.raises(gf.GFError) as e:
        gf.gf_workspace_bytes([(3, 2, 2, 2)], gf.GF_LANDAU, gf.GF_FP32_12)
    assert "even" in str(e.value)

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


def test_workspace_scales_with_link_storage():
    # links dominate the workspace: 8, 12 or 18 reals in FP32 or FP64
    V = 32 ** 4
    sizes = {st: gf.gf_workspace_bytes([(32, 32, 32, 32)], gf.GF_LANDAU, st)
             for st in (gf.GF_FP32_8, gf.GF_FP32_12, gf.GF_FP32_18, gf.GF_FP64_8, gf.GF_FP64_12, gf.GF_FP64_18)}
    per_link = {gf.GF_FP32_8: 32, gf.GF_FP32_12: 48, gf.GF_FP32_18: 72, gf.GF_FP64_8: 64,
                gf.GF_FP64_12: 96, gf.GF_FP64_18: 144}
    base = sizes[gf.GF_FP32_12] - 4 * V * 48
    for st, b in sizes.items():
        assert b - 4 * V * per_link[st] == base, st
    # mixed precision keeps an FP64-18 copy only for the FP32 storages
    for st in (gf.GF_FP32_8, gf.GF_FP32_12, gf.GF_FP32_18):
        assert gf.gf_workspace_bytes([(32, 32, 32, 32)], gf.GF_LANDAU, st, gf.GF_FLAG_MIXED) - sizes[st] >= 4 * V * 144
    for st in (gf.GF_FP64_8, gf.GF_FP64_12, gf.GF_FP64_18):
        assert gf.gf_workspace_bytes([(32, 32, 32, 32)], gf.GF_LANDAU, st, gf.GF_FLAG_MIXED) == sizes[st]


def test_creation_limits():
    # site coordinates are divided by Lx and Ly with 32-bit reciprocals: Lx Ly Lz max(Lx, Ly) < 2^32
    with pytest.raises(gf.GFError) as e:
        gf.gf_workspace_bytes([(2048, 2048, 2, 2)], gf.GF_LANDAU, gf.GF_FP32_12)
    assert e.value.code == gf.GF_EINVAL
    # Fourier acceleration: one lattice, FP32-12 or FP64-18, power-of-two transformed extents
    for dims, st in [((6, 8, 8, 8), gf.GF_FP32_12), ((8, 8, 8, 8), gf.GF_FP32_8), ((8, 8, 8, 8), gf.GF_FP64_12)]:
        with pytest.raises(gf.GFError) as e:
            gf.gf_workspace_bytes([dims], gf.GF_LANDAU, st, gf.GF_FLAG_FASD)
        assert e.value.code == gf.GF_EINVAL
    assert gf.gf_workspace_bytes([(8, 8, 8, 6)], gf.GF_COULOMB, gf.GF_FP32_12, gf.GF_FLAG_FASD) > 0
    with pytest.raises(gf.GFError):
        gf.gf_workspace_bytes([(8, 8, 8, 8)] * 2, gf.GF_LANDAU, gf.GF_FP32_12, gf.GF_FLAG_FASD)
    # the differentiable functional: one FP64-18 lattice
    with pytest.raises(gf.GFError):
        gf.gf_workspace_bytes([(8, 8, 8, 8)], gf.GF_LANDAU, gf.GF_FP32_12, gf.GF_FLAG_AUTOGRAD)


def test_header_is_plain_c_and_links(tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99, every declared entry
    # point links from a C program, and a host-only call runs without a GPU
    import os
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = gf.header_symbols()
    src = tmp_path / "abi.c"
    src.write_text(
        "#include \"gf.h\"\n#include <stdio.h>\n"
        "typedef void (*fp)(void);\n"
        "static const fp entry[] = {\n" + ",\n".join(f"  (fp){n}" for n in names) + "\n};\n"
        "int main(void) {\n"
        "  size_t bytes = 0;\n  int dims[4] = {8, 8, 8, 8};\n"
        "  int rc = gf_workspace_bytes(1, dims, GF_LANDAU, GF_FP32_12, 0, &bytes);\n"
        "  printf(\"%d %zu %d\\n\", rc, bytes, (int)(sizeof entry / sizeof entry[0]));\n"
        "  return rc == GF_OK && bytes > 0 ? 0 : 1;\n}\n")
    libdir = os.path.dirname(gf.LIB_PATH)
    inc = os.path.dirname(gf.HEADER)
    exe = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        f"-I{inc}", str(src), f"-L{libdir}", "-lgf", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    rc, nbytes, n = out.stdout.split()
    assert rc == "0" and int(nbytes) > 0 and int(n) == len(names)


# extents whose int64 product wraps negative (1102 * 4664 * 6944 * 516856348 > 2^63):
# every volume check must reject them before any CUDA call
WRAP_DIMS = (1102, 4664, 6944, 516856348)


def test_wrapping_volume_rejected_by_creation():
    with pytest.raises(gf.GFError) as e:
        gf.gf_workspace_bytes([WRAP_DIMS], gf.GF_LANDAU, gf.GF_FP32_12)
    assert e.value.code == gf.GF_EINVAL
    assert "2^31" in gf.gf_last_error(None)


@pytest.mark.parametrize("dims", [WRAP_DIMS, (2, 2, 2, 2 ** 30), (65536, 65536, 2, 2)])
def test_noalloc_rejects_wrapping_or_oversized_volume_on_the_host(dims):
    # the argument checks come before any CUDA call, so this runs without a GPU; the
    # links pointer is a dummy (aligned, never dereferenced)
    with pytest.raises(gf.GFError) as e:
        gf.gf_functional_theta_noalloc(dims, gf.GF_LANDAU, 256, 512)
    assert e.value.code == gf.GF_EINVAL
    assert "too large" in gf.gf_last_error(None)

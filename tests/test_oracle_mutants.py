"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that the
pins catch every one of them.  Each mutant is a textual edit of gf_oracle.c compiled
into a temporary library; at least one pin must fail on it."""
import os

import numpy as np

import pytest

import oracle
from tests import oracle_checks as C
from tests.test_oracle_pins import CASES

# (name, original text, planted mistake)
MUTANTS = [
    ("K_missing_dagger", "conj(bwd[mu][3 * c + r])", "bwd[mu][3 * r + c]"),
    ("beta_sign", "cplx beta = K[3 * j + i] - conj(K[3 * i + j]);", "cplx beta = K[3 * j + i] + conj(K[3 * i + j]);"),
    ("alpha_no_conj", "cplx alpha = K[3 * i + i] + conj(K[3 * j + j]);", "cplx alpha = K[3 * i + i] + K[3 * j + j];"),
    ("maximiser_a_not_conj", "a = CMPLX(creal(alpha) / n, -cimag(alpha) / n);", "a = CMPLX(creal(alpha) / n, cimag(alpha) / n);"),
    ("bwd_gets_G_not_Gdag", "mat_mul_dag(bwd[mu], G, t);", "mat_mul(bwd[mu], G, t);"),
    ("fwd_right_multiplied", "mat_mul(G, fwd[mu], t);", "mat_mul(fwd[mu], G, t);"),
    ("bwd_neighbour_forward", "bwd[mu] = link_at(U, neighbour(g, s, mu, -1), mu);", "bwd[mu] = link_at(U, neighbour(g, s, mu, +1), mu);"),
    ("K_not_rotated", "        su2_left_mul(K, pairs[k][0], pairs[k][1], a, b);\n", ""),
    ("delta_sign", "A[e] = A[e] + (b[e] - f[e]);", "A[e] = A[e] + (f[e] - b[e]);"),
    ("delta_forward_neighbour", "clink_at(U, neighbour(g, s, nu, -1), nu); /* U_nu(x - nu) */", "clink_at(U, neighbour(g, s, nu, +1), nu);"),
    ("delta_trace_factor", "cimag(sum) / 3.0", "cimag(sum) / 2.0"),
    ("delta_no_dagger", "D[3 * i + j] = A[3 * i + j] - conj(A[3 * j + i]);", "D[3 * i + j] = A[3 * i + j] - conj(A[3 * i + j]);"),
    ("F_norm_always_4", "*F = csum_value(&fa) / ((double)nd * NC * g.V);", "*F = csum_value(&fa) / (4.0 * NC * g.V);"),
    ("K_all_4_directions", "    for (int mu = 0; mu < nd; ++mu)\n        for (int r = 0; r < 3; ++r)", "    for (int mu = 0; mu < 4; ++mu)\n        for (int r = 0; r < 3; ++r)"),
    ("apply_only_nd_directions", "    for (int mu = 0; mu < 4; ++mu) {\n        cplx t[9];", "    for (int mu = 0; mu < nd; ++mu) {\n        cplx t[9];"),
    ("parity_ignores_t", "return (c[0] + c[1] + c[2] + c[3]) % 2;", "return (c[0] + c[1] + c[2]) % 2;"),
    ("overrelax_dropped_term", "cplx a1 = CMPLX(1.0 - omega + omega * creal(a), omega * cimag(a));", "cplx a1 = CMPLX(omega * creal(a), omega * cimag(a));"),
    ("overrelax_b_unscaled", "cplx b1 = CMPLX(omega * creal(b), omega * cimag(b));", "cplx b1 = CMPLX(creal(b), cimag(b));"),
    ("exact_power_sin_cos_swapped", "double c1 = cos(omega * phi), s1 = sin(omega * phi);", "double c1 = sin(omega * phi), s1 = cos(omega * phi);"),
    ("reunit_row2_no_conj", "u[8] = conj(u[0] * u[4] - u[1] * u[3]);", "u[8] = u[0] * u[4] - u[1] * u[3];"),
    ("reunit_projection_conj", "p += conj(u[k]) * u[3 + k];", "p += u[k] * conj(u[3 + k]);"),
    ("reunit_interval_off_by_one", "((it + 1) % reunit_interval) == 0", "(it % reunit_interval) == 0"),
    ("slice_mask_ignored", "        if (slice_active && !slice_active[s / g.V3]) continue;\n", ""),
    ("theta_slice_norm", "theta_t[t] = ts[t] / ((double)NC * g.V3);", "theta_t[t] = ts[t] / ((double)NC * g.V);"),
]

SRC = os.path.join(os.path.dirname(oracle.__file__), "gf_oracle.c")


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, orig, bad, tmp_path):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for {name} not unique or missing"
    src = tmp_path / f"mut_{name}.c"
    src.write_text(text.replace(orig, bad))
    lib = oracle.compile_source(str(src), str(tmp_path / f"libmut_{name}.so"))
    mut = oracle.load_variant(lib)
    # cheap checks first; the brute-force maximiser search last
    ordered = sorted(CASES, key=lambda c: c[0] is C.check_su2_maximiser_matches_brute_force_on_2x4_lattice)
    for check, args in ordered:
        try:
            check(mut, *args)
        except (AssertionError, ValueError, FloatingPointError):
            return  # caught
    pytest.fail(f"no pin caught the planted mistake {name}")


# planted mistakes in the Fourier-accelerated steepest descent oracle (oracle/fasd.py)
FASD_MUTANTS = [
    ("p2_sin_not_squared", "s = 4.0 * np.sin(np.pi * k / L) ** 2", "s = 4.0 * np.sin(np.pi * k / L)"),
    ("p2_wrong_period", "s = 4.0 * np.sin(np.pi * k / L) ** 2", "s = 4.0 * np.sin(2 * np.pi * k / L) ** 2"),
    ("p2max_always_16", "p2max = 4.0 * _nd(gauge)", "p2max = 16.0"),
    ("ifft_is_fft", "out[..., i, j] = np.fft.ifftn(Fk, axes=axes)", "out[..., i, j] = np.fft.fftn(Fk, axes=axes) / Fk[..., 0, 0, 0].size"),
    ("coulomb_fft_over_t", "_AXES = {0: (0, 1, 2, 3), 1: (1, 2, 3)}", "_AXES = {0: (0, 1, 2, 3), 1: (0, 1, 2, 3)}"),
    ("half_alpha_dropped", "g = np.eye(3, dtype=np.complex128) + 0.5 * alpha * Dt", "g = np.eye(3, dtype=np.complex128) + alpha * Dt"),
    ("update_no_dagger", "out[..., mu, :, :] = g @ U[..., mu, :, :] @ np.roll(gd, -1, axis=ax)",
     "out[..., mu, :, :] = g @ U[..., mu, :, :] @ np.roll(g, -1, axis=ax)"),
    ("update_backward_neighbour", "np.roll(gd, -1, axis=ax)", "np.roll(gd, 1, axis=ax)"),
]

FASD_CASES = [c for c in CASES if c[0].__name__.startswith("check_fasd")]


@pytest.mark.parametrize("name,orig,bad", FASD_MUTANTS, ids=[m[0] for m in FASD_MUTANTS])
def test_fasd_pins_catch_planted_mistake(name, orig, bad, tmp_path, monkeypatch):
    import importlib.util
    import sys
    src = os.path.join(os.path.dirname(oracle.__file__), "fasd.py")
    text = open(src).read()
    assert text.count(orig) >= 1, f"mutation site for {name} missing"
    path = tmp_path / "fasd_mut.py"
    path.write_text(text.replace(orig, bad))
    spec = importlib.util.spec_from_file_location("oracle.fasd", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    monkeypatch.setitem(sys.modules, "oracle.fasd", mod)
    monkeypatch.setattr(oracle, "fasd", mod, raising=False)
    for check, args in FASD_CASES:
        try:
            with np.errstate(all="ignore"):
                check(oracle, *args)
        except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError):
            return
    pytest.fail(f"no pin caught the planted mistake {name}")

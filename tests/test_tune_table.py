"""CPU checks of the autotuner's table (pint_tune_load / pint_tune_save /
pint_tune_lookup / pint_tune_clear): file round trip, keys by shape and by the
precision a problem runs in, malformed files rejected.  No GPU: the table is
host state, and pint_tune_lookup only validates the problem."""
import os

import pytest

from paper_2304_14021_gb300 import build_lib, pint

# equation codes and enums as in include/pint.h (linear_ch = 1, cahn_hilliard = 2; bc neumann = 1; mixed = 1)
SHAPE = dict(equation="linear_ch", dim=2, nx=64, ny=64, bc="neumann", eps=0.05, beta=0.5, T=0.05, nt=64,
             precision="mixed", tol=1e-8)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    pint.lib()
    yield
    pint.tune_clear()


def key_line(fwd, inv, fused, ms, **over):
    d = dict(SHAPE, **over)
    p = pint.make_problem(**d)
    half = 1 if p.theta < 1.0 else 0
    return (f"pint-tune {p.equation} {p.dim} {p.nx} {p.ny} {p.nt} {p.precision} {p.bc} {half} "
            f"{fwd} {inv} {fused} {ms}\n")


def test_load_lookup_save_round_trip(tmp_path):
    pint.tune_clear()
    assert pint.tune_lookup(**SHAPE) is None
    f = tmp_path / "t.txt"
    f.write_text("# a comment\n" + key_line(0, 1, 1, 0.125) + key_line(1, 0, 0, 0.5, nt=128))
    assert pint.tune_load(f) == 2
    e = pint.tune_lookup(**SHAPE)
    assert e == {"time_fwd_gemm": 0, "time_inv_gemm": 1, "fused_spatial": 1, "ms": 0.125}
    assert pint.tune_lookup(**dict(SHAPE, nt=128))["time_fwd_gemm"] == 1
    assert pint.tune_lookup(**dict(SHAPE, nx=128, ny=128)) is None      # another shape
    assert pint.tune_lookup(**dict(SHAPE, theta=0.5)) is None           # another kernel variant
    g = tmp_path / "saved.txt"
    assert pint.tune_save(g) == 2
    pint.tune_clear()
    assert pint.tune_lookup(**SHAPE) is None
    assert pint.tune_load(g) == 2
    assert pint.tune_lookup(**SHAPE)["time_inv_gemm"] == 1


def test_key_uses_the_precision_the_problem_runs_in(tmp_path):
    # a linear problem asked for in float-float that is too stiff for it runs as PINT_MIXED:
    # its entry is the PINT_MIXED one
    pint.tune_clear()
    stiff = dict(SHAPE, equation="biharmonic", dim=1, nx=1024, ny=1, T=1e-4, nt=64)
    f = tmp_path / "t.txt"
    f.write_text(key_line(1, 1, 0, 1.0, **dict(stiff, precision="mixed")))
    assert pint.tune_load(f) == 1
    assert pint.tune_lookup(**dict(stiff, precision="mixed_ff")) is not None
    assert pint.tune_lookup(**dict(stiff, precision="fp64")) is None


@pytest.mark.parametrize("text", ["pint-tune 1 2 3\n", "other 1 2 64 64 64 1 1 0 0 0 1 0.1\n",
                                  "pint-tune 1 2 64 64 64 1 1 0 2 0 1 0.1\n"])
def test_malformed_file_rejected(tmp_path, text):
    f = tmp_path / "bad.txt"
    f.write_text(text)
    with pytest.raises(pint.PintError):
        pint.tune_load(f)


def test_missing_file_rejected(tmp_path):
    with pytest.raises(pint.PintError):
        pint.tune_load(tmp_path / "none.txt")
    with pytest.raises(pint.PintError):
        pint.tune_lookup(**dict(SHAPE, nx=0))

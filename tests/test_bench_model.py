"""The bench's algorithmic byte model (the numerator of the reported roofline), checked
against the per-zone counts of each kernel group written out by hand."""
import types

import bench

NR, NTH, NPHI = 550, 128, 256
Z = NR * NTH * NPHI
MH = NPHI // 2 + 1
S = 2 * MH * NR * NTH


def grid():
    return types.SimpleNamespace(shape=(NR, NTH, NPHI))


def test_six_product_solve_with_one_correction():
    b = bench.algorithmic_bytes_per_step(grid(), "mixed", iters=2, fused=False)
    t = 2 * 3 * MH * NTH * NTH                      # three bf16 planes of the table
    assert b["fft_forward"] == (8 * Z + 4 * S) + (4 * Z + 4 * S)   # rho in, then r in; panel out
    assert b["project_forward"] == b["project_inverse"] == 2 * (8 * S + t)
    assert b["radial_solve"] == 2 * 12 * S          # panel in and out, 1/pivot and c' tables
    # first solve: spectrum in, high word out; correction: spectrum and high word in,
    # float64 Phi out (the float-float words are not stored)
    assert b["fft_inverse"] == (4 * S + 4 * Z) + (4 * S + 12 * Z)
    assert b["residual"] == 16 * Z                  # rho, high word, r
    assert b["update"] == 0.0
    total = sum(b.values())
    assert abs(total / 1e9 - 2.15) < 0.01           # the HBM floor of one solve, 2.15 GB


def test_three_product_solve_with_two_corrections():
    b = bench.algorithmic_bytes_per_step(grid(), "mixed_x3", iters=3, fused=False)
    # both corrections store the float-float iterate (and float64 Phi)
    assert b["fft_inverse"] == (4 * S + 4 * Z) + (4 * S + 20 * Z) + (4 * S + 24 * Z)
    assert b["residual"] == 16 * Z + 20 * Z         # the second reads both words
    assert b["update"] == 0.0


def test_second_six_product_correction_rebuilds_the_words():
    b = bench.algorithmic_bytes_per_step(grid(), "mixed", iters=3, fused=False)
    assert b["update"] == 16 * Z                    # float64 in, two float words out
    assert b["residual"] == 16 * Z + 20 * Z


def test_no_correction_converts_the_high_word():
    b = bench.algorithmic_bytes_per_step(grid(), "mixed", iters=1, fused=False)
    assert b["update"] == 12 * Z and b["residual"] == 0
    assert b["fft_inverse"] == 4 * S + 4 * Z


def test_float64_path():
    b = bench.algorithmic_bytes_per_step(grid(), "fp64")
    assert b["fft_forward"] == 8 * Z + 8 * S and b["fft_inverse"] == 8 * S + 8 * Z
    assert b["radial_solve"] == 16 * S + 4 * S


def test_residual_fused_with_its_transform():
    """Nphi = 256: the residual kernel writes the panel, so r's write and read are gone."""
    b = bench.algorithmic_bytes_per_step(grid(), "mixed", iters=2)
    u = bench.algorithmic_bytes_per_step(grid(), "mixed", iters=2, fused=False)
    assert b["fft_forward"] == 8 * Z + 4 * S                      # rho alone
    assert b["residual"] == 8 * Z + 4 * Z + 4 * S                 # rho, high word in; panel out
    assert sum(u.values()) - sum(b.values()) == 8 * Z             # r written and read once each
    b3 = bench.algorithmic_bytes_per_step(grid(), "mixed_x3", iters=3)
    assert b3["residual"] == (12 * Z + 4 * S) + (16 * Z + 4 * S)  # the second reads both words


def test_roofline_reports_the_residual_interior_kernel():
    """The residual's span holds the side stream's shell term and last shell: the line's
    roofline reports its interior-row kernel, with (Nr-1)/Nr of the residual's bytes, its
    own live time, and the issue fraction from the instruction count."""
    p = types.SimpleNamespace(shape=(550, 128, 256))
    steps = 20
    timing = {"residual": (0.150 * steps, steps), "residual_rows": (0.120 * steps, steps),
              "fft_inverse": (0.125 * steps, 2 * steps), "radial_solve": (0.128 * steps, 2 * steps)}
    r = bench.roofline(timing, p, "mixed", steps, 2, sm_mhz=2000.0, num_sms=152)
    full = bench.algorithmic_bytes_per_step(p, "mixed", 2)["residual"]
    assert r["kernel"].startswith("residual_rows")
    assert abs(r["algorithmic_bytes_per_launch"] - full * 549 / 550) < 1.0
    assert abs(r["achieved"] - full * 549 / 550 / 0.120e-3 / 1e9) < 1e-6 * r["achieved"]
    if r.get("issue"):   # only when the ncu table matches the sources
        assert abs(r["issue"]["frac"] - r["issue"]["warp_instructions_per_launch"] / (4 * 152 * 2000e6 * 0.120e-3)) < 1e-9
    # without the interior span, the residual's whole span
    r2 = bench.roofline({"residual": timing["residual"]}, p, "mixed", steps, 2)
    assert r2["kernel"] == "residual"
    assert abs(r2["algorithmic_bytes_per_launch"] - full) < 1.0
    # the interior span is never the dominant group itself
    r3 = bench.roofline({"residual_rows": (9.0, steps), "fft_inverse": timing["fft_inverse"]}, p, "mixed", steps, 2)
    assert r3["kernel"] == "fft_inverse"

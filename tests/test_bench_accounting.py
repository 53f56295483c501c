"""The benchmark's bookkeeping without a GPU: the radix plans it models, the compulsory bytes
and FFT flops it divides by the measured times (the numerators of `roofline.achieved`), checked
against counts made here from the definitions."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_radix_plans(bench):
    # the prime factors of n grouped first-fit into register radices <= rmax, largest first
    assert bench.plan_radices(243, 27) == [27, 9]
    assert bench.plan_radices(243, 15) == [9, 9, 3]
    assert bench.plan_radices(405, 27) == [27, 15]
    assert bench.plan_radices(161, 27) == [23, 7]
    assert bench.plan_radices(63, 27) == [21, 3]
    for n in (45, 81, 135, 175, 189, 243, 405, 161, 63):
        for rmax in (9, 15, 27):
            p = bench.plan_radices(n, rmax)
            prod = 1
            for r in p:
                prod *= r
            assert prod == n and all(r <= max(rmax, 31) for r in p)


def test_compulsory_bytes_of_the_cg_step(bench):
    n = 243
    nh = (n + 1) // 2
    field32 = 3 * n ** 3 * 4                   # d components of a real field, FP32
    spec32 = 3 * n * n * nh * 8                # d half spectra, complex FP32
    b = bench.pass_bytes(4, fused_cg=True)
    # line_fwd: r, p read, p written, one-byte phases, spectrum written
    assert b["line_fwd"] == 3 * field32 + n ** 3 + spec32
    # each column pass reads and writes the spectrum once
    assert b["strided"] == b["proj"] == 2 * spec32
    # fused line_inv: spectrum, x, r, p read; x, r written
    assert b["line_inv"] == spec32 + 5 * field32
    step = b["line_fwd"] + 2 * b["strided"] + b["proj"] + b["line_inv"]
    assert abs(step / 1e9 - 2.78) < 0.01       # a fused FP32 step with three spectrum lines
    # two spectrum lines between the column passes: 5/3 and 4/3 of a spectrum, 2.55 GB a step
    b2 = bench.pass_bytes(4, two_line=True, fused_cg=True)
    assert b2["strided"] == spec32 * 5 // 3 and b2["proj"] == spec32 * 4 // 3
    step2 = b2["line_fwd"] + 2 * b2["strided"] + b2["proj"] + b2["line_inv"]
    assert abs(step2 / 1e9 - 2.55) < 0.01
    # the unfused step adds the vector update and is heavier
    bu = bench.pass_bytes(4)
    stepu = bu["line_fwd"] + 2 * bu["strided"] + bu["proj"] + bu["line_inv"] + bu["vector"]
    assert abs(stepu / 1e9 - 3.29) < 0.01
    # FP64 doubles every field and spectrum word
    b64 = bench.pass_bytes(8, fused_cg=True)
    assert b64["strided"] == 2 * b["strided"]


def test_compulsory_bytes_of_the_potential_step(bench):
    # CG in potential coordinates: u, r, p are one complex half-spectrum component each
    n = 243
    c = n * n * ((n + 1) // 2) * 8            # one complex FP32 component on the half spectrum
    b = bench.pot_bytes(4)
    assert b["pot_inv"] == 3 * c + 2 * c + 2 * c      # r, p, u read; p, u and two lines written
    assert b["strided"] == 5 * c                      # two lines <-> three lines
    assert b["pot_line"] == 6 * c + n ** 3            # three lines each way, one-byte phases
    assert b["pot_fwd"] == 2 * c + c + c              # two lines and r read; r written
    step = b["pot_inv"] + 2 * b["strided"] + b["pot_line"] + b["pot_fwd"]
    assert abs(step / 1e9 - 1.57) < 0.01              # against 2.55 GB of the field-form step
    assert step < bench.pass_bytes(4, two_line=True, fused_cg=True)["line_fwd"] * 3


def test_fft_flop_model(bench):
    # radix-3 stage: 9.33 flops per point with twiddles; a plan without twiddles on its first
    # stage costs less than one with them on every stage
    f = bench.fft_flops_per_point(3, 15)
    assert f > 0
    f243 = bench.fft_flops_per_point(243, 15)
    assert 5 * 8.0 < f243 < 5 * 9.34 + 1e-9    # five radix-3 levels, the first without twiddles
    flops = bench.pass_flops(15)
    n = 243
    spec = n * n * ((n + 1) // 2) * 3
    assert flops["strided"] == spec * f243
    assert flops["proj"] > 2 * flops["strided"]  # four transforms of two lines + Gamma^


def test_flop_model_sums_to_the_fft_count_of_a_matvec(bench):
    # one operator application = d forward and d inverse real 3-D transforms of 2.5 |N| log2 |N|
    import math
    flops = bench.pass_flops_model((243, 243, 243))
    per_step = flops["line_fwd"] + 2 * flops["strided"] + flops["proj"] + flops["line_inv"]
    nodes = 243 ** 3
    assert abs(per_step - 2 * 3 * 2.5 * nodes * math.log2(nodes)) < 1e-6 * per_step
    assert abs(flops["strided"] / 1e9 - 0.8526) < 1e-3  # one axis of three transforms


def test_fp64_instruction_counts_match_the_factored_plan(bench):
    # the stored ncu count of the FP64 strided pass at 243^3 is the count of its [9, 9, 3] plan
    # with cosine-factored twiddles: an untwiddled 9-point DFT (84 instructions), a twiddled one
    # (106) and a twiddled 3-point one (18), per complex point of the half spectrum's three
    # components; the projection runs four such transforms on one line each
    assert bench.plan_radices(243, 15) == [9, 9, 3]
    per_point = 84 / 9 + 106 / 9 + 18 / 3
    points = 243 * 243 * 122 * 3
    assert abs(bench.NCU_FP64_INST["strided"] / points - per_point) < 0.02
    assert bench.NCU_FP64_INST["proj"] > 4 / 3 * bench.NCU_FP64_INST["strided"]


def test_fp64_issue_fraction(bench):
    # pass times at exactly the instruction bound give a fraction of 1 per pass and per step
    probe = {"dfma_tflops": 1.0, "dadd_tinstr_per_s": 0.5}
    rate = 0.5e12
    pk = {k: {"ms_avg": v / rate * 1e3, "launches": 2 if k == "strided" else 1}
          for k, v in bench.NCU_FP64_INST.items()}
    step_ms = sum(v["ms_avg"] * v["launches"] for v in pk.values())
    out = bench.fp64_issue(pk, step_ms, 1, probe)
    for k in bench.NCU_FP64_INST:
        assert abs(out[k] - 1.0) < 1e-3
    assert abs(out["step_frac"] - 1.0) < 1e-3
    assert bench.fp64_issue(pk, step_ms, 1, None) is None

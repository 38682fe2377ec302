"""The roofline accounting: Table I transcription (golden values evaluated
from the table at stated shapes) and its link to the per-kernel counts."""
import json
import os

import pytest

from paper_1702_04458_b300.accounting import (Workload, algorithmic_bytes, algorithmic_mults,
                                              detected_bits, fp32_simt_peak_tflops, table1_ar)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_ar.json")


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"])
def test_table1_transcription(case):
    got = table1_ar(case["alg"], case["mode"], case["C"], case["S"], case["U"])
    for k in ("pre", "first", "sub"):
        assert abs(got[k] - case[k]) < 1e-6 * max(1.0, case[k]), (k, got[k], case[k])


@pytest.mark.parametrize("T", [1, 2, 3, 5])
def test_admm_ul_counts_follow_table1_for_one_symbol(T):
    """With N = 1 the ADMM-UL kernel count is exactly Table I's U x U row:
    preprocessing + first iteration + (T - 1) later iterations."""
    wl = Workload(B=128, C=8, U=8, W=1, N=1, M=16, T=T)
    t = table1_ar("admm_ul", "UxU", 8, 16, 8)
    assert abs(algorithmic_mults("admm_ul", wl) - (t["pre"] + t["first"] + (T - 1) * t["sub"])) < 1e-6


def test_cg_counts_replace_two_matvecs_by_gram_product():
    """CG with the precomputed Gram: per iteration 8SU (two mat-vecs) becomes
    4U^2, and the Gram 2SU^2 is paid once per subcarrier."""
    C, S, U, T = 8, 16, 8, 8
    wl = Workload(B=C * S, C=C, U=U, W=1, N=1, M=16, T=T)
    t = table1_ar("cg_ul", "-", C, S, U)
    table = t["pre"] + t["first"] + (T - 1) * t["sub"]
    # first iteration of Table I has 4U per cluster instead of 10U: the kernel
    # counts every iteration like a later one
    swap = T * C * (8 * S * U - 4 * U * U) - C * (10 * U - 4 * U)
    assert abs(algorithmic_mults("cg_ul", wl) - (table - swap + C * 2 * S * U * U)) < 1e-6


def test_bytes_and_bits():
    wl = Workload(B=128, C=8, U=8, W=1200, N=14, M=16, T=3)
    assert algorithmic_bytes("admm_ul", wl) * wl.W == 9830400 + 17203200 + 1075200 + 134400
    assert detected_bits(wl) == 8 * 4 * 1200 * 14
    assert abs(fp32_simt_peak_tflops(148, 2032.0) - 76.9884) < 1e-3

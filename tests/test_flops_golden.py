"""The Algorithm 1 flop formulas used for TFLOP/s reproduce Tab. 6 (rate x time)."""
import json
import os

import pytest

from paper_1611_00606_gb300.flops import assembly_flops, step_flops

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_tab6_rows_match_algorithm1_counts():
    g = _load("tab6_nacl_kmax4.json")
    sz = g["sizes"]
    f = step_flops(sz["N_A"], sz["N_L"], sz["N_G"], N_f=0)
    for row in g["rows"]:
        measured = row["time_s"] * row["gflops"] * 1e9
        predicted = sum(f[s] for s in row["steps"])
        # the table prints 3-4 significant digits
        assert predicted == pytest.approx(measured, rel=6e-3), row["section"]


def test_tab6_implied_fallback_sizes():
    g = _load("tab6_nacl_kmax4.json")
    sz = g["sizes"]
    for row in g["implied"]:
        measured = row["time_s"] * row["gflops"] * 1e9
        if "N_f" in row:
            pred = step_flops(sz["N_A"], sz["N_L"], sz["N_G"], row["N_f"])["H2_zgemm"]
        else:
            pred = step_flops(sz["N_A"], sz["N_L"], sz["N_G"], sz["N_A"] - row["N_h"])["H3_zherk"]
        assert pred == pytest.approx(measured, rel=6e-3), row["section"]


def test_tab1_shapes_and_total():
    t1 = _load("tab1_sizes.json")
    assert t1["AuAg"]["N_L"] == (10 + 1) ** 2 and t1["NaCl"]["N_L"] == (6 + 1) ** 2
    # total = 20 K N_G^2 + 4 N_f N_L N_G^2 + per-atom terms (auag-like 4000 shape)
    F = assembly_flops(100, 121, 4000, 5)
    K = 100 * 121
    big = 20 * K * 4000 ** 2 + 4 * 5 * 121 * 4000 ** 2
    assert big < F < 1.05 * big
    assert F == pytest.approx(4.03e12, rel=5e-3)

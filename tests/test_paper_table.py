"""The transcription of the paper's Table III used by ``bench.py
--paper-table`` checked against the paper's own accounting: in every cell
latency x throughput is the bits of one cycle, 16 users x 6 bits x 7 symbols
x 1280 subcarriers = 860,160 bits, except the CG B = 1024 column, which
matches the 1200 subcarriers the text states (806,400 bits).  A mistyped
digit in either number of a cell moves the product outside the 0.2 % bound
(the largest deviation of the printed cells is 0.08 %)."""
import pytest

import bench


@pytest.mark.parametrize("alg", ["admm_ul", "cg_ul", "admm_dl"])
def test_table_iii_cells_carry_one_cycle_of_bits(alg):
    rows = bench.PAPER_TABLE_III[alg]
    assert len(rows) == 5 and all(len(r) == len(bench.PAPER_COLS) == 9 for r in rows)
    for t, row in enumerate(rows):
        for ci, (lat_ms, mbit_s) in enumerate(row):
            bits = lat_ms * 1e-3 * mbit_s * 1e6
            want = 806_400 if (alg == "cg_ul" and bench.PAPER_COLS[ci][0] == 1024) else 860_160
            assert abs(bits / want - 1.0) < 0.002, (alg, t + 1, bench.PAPER_COLS[ci], bits)


def test_table_iii_latency_grows_with_iterations():
    for alg, rows in bench.PAPER_TABLE_III.items():
        for ci in range(9):
            lat = [rows[t][ci][0] for t in range(5)]
            assert lat == sorted(lat), (alg, bench.PAPER_COLS[ci])

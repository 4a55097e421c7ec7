"""The algorithmic byte counts behind the bench line's HBM rooflines of the
trace-axis kernels (`bench.xfft_model_bytes`), against a count of the model-
sized streams each launch of the fused CG path moves, written out launch by
launch for small CG budgets: per outer iteration n_cg CG forwards (p~_{it-1}
and s~ in, p~_it out; on odd iterations m in and out and, from it = 3 on,
p~_{it-2} in) and one plain reconstruction forward (m in), each writing the
half spectrum X; the c2r's n_cg weighted adjoints read X and W_m^-1 and write
s~.  Also the per-pair algorithmic bytes and flops of the section's formulas."""
import pytest

import bench

NT, NX, P, NXP = 1024, 256, 32, 512
S = 4.0 * NX * NT * P                  # one FP32 model-sized stream, per gather
X = 8.0 * (NXP // 2 + 1) * NT * P      # the half spectrum, per gather


def _r2c_streams(n_cg):
    """Model-sized streams of every r2c launch of one outer iteration."""
    launches = []
    for it in range(n_cg):
        reads = ["p_prev", "s"]
        writes = ["p"]
        if it % 2 == 1:
            reads.append("m")
            writes.append("m")
            if it >= 3:
                reads.append("p_prev2")
        launches.append(len(reads) + len(writes))
    launches.append(1)                  # the reconstruction forward reads m
    return launches


@pytest.mark.parametrize("n_cg", [1, 2, 3, 4, 5, 30])
def test_r2c_bytes_match_the_launch_count(n_cg):
    streams = _r2c_streams(n_cg)
    expect = 64 * sum(k * S + X for k in streams) / len(streams)
    got = bench.xfft_model_bytes("xfft_r2c", 64, n_outer=8, n_cg=n_cg)
    assert got == pytest.approx(expect, rel=1e-12)


def test_r2c_bytes_at_the_workload():
    # 30 CG iterations: it = 0 moves 3 S, it = 1 5 S, 14 odd ones from 3 on 6 S,
    # 14 even ones from 2 on 3 S, and the plain forward S; 31 launches
    total = (3 + 5 + 14 * 6 + 14 * 3 + 1) * S + 31 * X
    assert bench.xfft_model_bytes("xfft_r2c", 1) == pytest.approx(total / 31, rel=1e-12)
    assert 13.6e9 < bench.xfft_model_bytes("xfft_r2c", 64) < 13.7e9


def test_c2r_bytes():
    assert bench.xfft_model_bytes("xfft_c2r", 64) == pytest.approx(64 * (X + 2 * S), rel=1e-12)


def test_pair_algorithmic_figures():
    a = bench.algorithmic()
    assert a["pair_bytes"] == 2 * 4.0 * NT * NX * (P + 1)            # 69.2 MB
    lh = NXP // 2 + 1
    rows = (P + 1) * lh * 5.0 * 2048 * 11 + 16.0 * P * 2048 * lh
    assert a["rows_flops"] == pytest.approx(rows, rel=1e-12)
    assert 3.1e9 < a["pair_flops"] < 3.3e9                            # 3.2 GFLOP per pair

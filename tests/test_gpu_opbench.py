"""Measured integer ceilings (mp_dp_op_rates) behind the DP roofline."""
import pytest

pytestmark = pytest.mark.gpu


def test_op_rates_are_physical():
    import paper_2210_08052_gb300 as mp

    r = mp.mp_dp_op_rates(0)
    # 4 schedulers per SM issue at most one warp instruction per clock each
    for k in ("max_u16x2", "viaddmax_u16x2", "vimax3_u16x2", "prmt", "lop3", "imad"):
        assert 0.2 < r[k] <= 4.05, (k, r[k])
    # the fused add-max does two lane operations per instruction, so it
    # cannot issue faster than a plain packed max
    assert r["viaddmax_u16x2"] <= r["max_u16x2"] * 1.05
    # the step runs 64 cells per warp and anti-diagonal step with well over
    # 20 instructions each: below 4 x 64 / 20 cells per clock per SM
    assert 0.5 < r["step_cells_per_clk_sm"] < 13.0
    assert r["warps_per_sm_step"] >= 8


def test_planner_byte_counts():
    """mp_dp_stats counts the stream, records and boundary bytes of a run as
    the layout defines them (64-residue strips, 96-step chunks)."""
    import synth
    import paper_2210_08052_gb300 as mp

    pairs = synth.config2()[:24]
    c = mp.mp_dp_init(None, 0)
    try:
        mp.mp_dp_align_batch(c, pairs)
        st = mp.mp_dp_get_stats(c)
    finally:
        mp.mp_dp_destroy(c)
    stream = records = read = bnd = 0
    for p in pairs:
        m, n = len(p.prot), len(p.nt)
        strips, chunks = -(-m // 64), -(-(n + 63) // 96)
        stream += strips * chunks * (96 * 64 * 2 + 64 * 2)
        records += ((n + 127 + 95) // 96 + 1) * 96 * 16 + 2 * 96 * 16
        read += strips * (chunks + 1) * 96 * 16
        bnd += (strips - 1) * chunks * 96 * 4
    assert st["code_bytes"] == stream
    assert st["record_bytes"] == records
    assert st["record_read_bytes"] == read
    assert st["boundary_bytes"] == bnd

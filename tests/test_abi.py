"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/mp_dp.h declares, and its host-only calls behave."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mp():
    from paper_2210_08052_gb300 import build
    build.build()
    import paper_2210_08052_gb300 as m
    m.lib()
    return m


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(mp_\w+)\s*\(", src, re.M))
    return names


def test_header_symbols_exported(mp):
    names = _declared()
    assert {"mp_dp_init", "mp_dp_align_batch", "mp_dp_submit", "mp_dp_poll", "mp_dp_destroy"} <= names
    L = ctypes.CDLL(mp.SO_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(mp.EXPORTED) == names


def test_default_params_match_oracle_tables(mp, orc):
    p = mp.mp_dp_default_params()
    assert (p.q, p.e, p.f, p.r, p.stop) == (11, 1, 23, 29, 23)
    lm = mp.params_matrix(p)
    om = orc.blosum62_22()
    assert (lm[:20, :] == om[:20, :]).all()          # rows the DP reads
    assert p.tb_budget_bytes == 40 << 30
    assert p.splice_model == mp.MP_SPLICE_FINAL and p.splice_p == 30


def test_struct_layout_matches_header(mp, tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's size and offsets."""
    src = tmp_path / "sz.c"
    src.write_text("""#include <stdio.h>
#include <stddef.h>
#include "mp_dp.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mp_result),
 sizeof(mp_pair), sizeof(mp_dp_params), sizeof(mp_dp_stats), offsetof(mp_result, cigar), offsetof(mp_pair, strand),
 offsetof(mp_dp_params, tb_budget_bytes), offsetof(mp_dp_params, autotune), sizeof(mp_dp_tuning),
 offsetof(mp_dp_tuning, ms), offsetof(mp_dp_tuning, strip_width), offsetof(mp_pair, profile),
 sizeof(mp_profile_pos), offsetof(mp_profile_pos, gap_ext), sizeof(mp_op_rates),
 offsetof(mp_op_rates, warps_per_sm_step)); return 0;}""")
    exe = tmp_path / "sz"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = list(map(int, subprocess.check_output([str(exe)]).split()))
    want = [ctypes.sizeof(mp.mp_result), ctypes.sizeof(mp.mp_pair), ctypes.sizeof(mp.mp_dp_params),
            ctypes.sizeof(mp.mp_dp_stats), mp.mp_result.cigar.offset, mp.mp_pair.strand.offset,
            mp.mp_dp_params.tb_budget_bytes.offset, mp.mp_dp_params.autotune.offset,
            ctypes.sizeof(mp.mp_dp_tuning), mp.mp_dp_tuning.ms.offset, mp.mp_dp_tuning.strip_width.offset,
            mp.mp_pair.profile.offset, ctypes.sizeof(mp.mp_profile_pos), mp.mp_profile_pos.gap_ext.offset,
            ctypes.sizeof(mp.mp_op_rates), mp.mp_op_rates.warps_per_sm_step.offset]
    assert got == want


def test_strerror(mp):
    assert mp.mp_dp_strerror(0) == "ok"
    assert "invalid" in mp.mp_dp_strerror(-1)
    assert mp.mp_dp_strerror(-999) == "unknown error"


@pytest.mark.parametrize("bad", [dict(r=20), dict(r=23), dict(e=0), dict(q=-1), dict(stop=40),
                                 dict(splice_model=2), dict(splice_p=-1), dict(splice_p=1001), dict(mode=3), dict(mode=-1)])
def test_init_rejects_degenerate_params(mp, bad):
    """r must exceed f, stop and -min(mat) so that no intron of length <= 0
    beats a frameshift or a match (validated before any device access)."""
    p = mp.mp_dp_default_params(**bad)
    ctx = ctypes.c_void_p()
    assert mp.lib().mp_dp_init(ctypes.byref(ctx), ctypes.byref(p), 0) == mp.MP_EINVAL


def test_null_arguments(mp):
    L = mp.lib()
    assert L.mp_dp_init(None, None, 0) == mp.MP_EINVAL
    assert L.mp_dp_align_batch(None, None, 0, None) == mp.MP_EINVAL
    assert L.mp_dp_get_stats(None, None) == mp.MP_EINVAL
    assert L.mp_dp_autotune(None, None, None, None, 0, None) == mp.MP_EINVAL
    assert L.mp_dp_set_tuning(None, None) == mp.MP_EINVAL
    assert L.mp_dp_get_tuning(None, None, None) == mp.MP_EINVAL
    assert L.mp_dp_tuning_save(None, b"x") == mp.MP_EINVAL
    assert L.mp_dp_tuning_load(None, b"x") == mp.MP_EINVAL
    assert L.mp_dp_debug_h(None, None, 0, None) == mp.MP_EINVAL
    assert L.mp_chain_refine(None, None, 0, None) == mp.MP_EINVAL
    assert L.mp_dp_op_rates(0, None) == mp.MP_EINVAL
    assert L.mp_dp_op_rates(-1, ctypes.byref(mp.mp_op_rates())) == mp.MP_EINVAL
    L.mp_dp_destroy(None)

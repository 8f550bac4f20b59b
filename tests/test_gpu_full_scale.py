"""Every pair of the full-size batch workloads against the oracle, in the
launch configuration the benchmark times (chosen by the library's
autotuner on the batch).

* 4,096-pair workload: every pair's score, coordinates and CIGAR equal the
  full-matrix oracle's (15.3 G cells; about half a minute on 16 host cores).
* 20,000-pair uneven-size workload (up to 5,000 residues x 200 kb, 2% of
  introns 20-100 kb, 5% score-only decoys, several traceback waves): every
  pair's score and end cell equal the oracle's four-row fill; every pair up
  to 4 M cells matches the full-matrix oracle in score, coordinates and
  CIGAR; every CIGAR rescores by op-sum to the oracle's score and ends at
  the oracle's end cell, so each returned path is an optimal alignment.
The device-resident run and the end-to-end call with host buffers return
the same results.
"""
import numpy as np
import pytest

import synth
from fullscale import KEYS, genome_end, oracle_map, rescore_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_2210_08052_gb300 import build
    build.build()
    import paper_2210_08052_gb300 as m
    m.lib()
    return m


def _tuned_run(mp, pairs):
    """Autotune on the uploaded batch, run it device-resident, then the
    end-to-end call with host buffers under the same (tuned) context."""
    ctx = mp.mp_dp_init(None, 0)
    try:
        src = mp.PairBatch(pairs)
        b = mp.mp_dp_batch_upload(ctx, src)
        best, _ = mp.mp_dp_autotune(ctx, b)
        mp.mp_dp_batch_run(ctx, b)
        mp.mp_dp_batch_sync(ctx)
        dev = mp.mp_dp_batch_download(ctx, b)
        waves = mp.mp_dp_get_stats(ctx)["n_waves"]
        mp.mp_dp_batch_free(ctx, b)
        e2e = mp.mp_dp_align_batch(ctx, src)
    finally:
        mp.mp_dp_destroy(ctx)
    return best, dev, e2e, waves


def _same(a, b):
    return all(x[k] == y[k] for x, y in zip(a, b) for k in KEYS + ("status",))


def test_config2_every_pair_against_oracle(mp, orc):
    pairs = synth.config2()
    _, got, e2e, _ = _tuned_run(mp, pairs)
    assert _same(got, e2e)
    want = oracle_map(lambda p: orc.align(p.prot, p.nt, p.strand), pairs, range(len(pairs)), full=True)
    bad = []
    for k, (p, g) in enumerate(zip(pairs, got)):
        w = want[k]
        diff = [x for x in KEYS if g[x] != w[x]]
        if diff or g["status"] & 0xF0:
            bad.append((k, diff, g["status"], len(p.prot), len(p.nt)))
    assert not bad, (len(bad), bad[:5])


def test_config3_every_pair_against_oracle(mp, orc):
    pairs = synth.config3()
    _, got, e2e, waves = _tuned_run(mp, pairs)
    assert waves > 1
    assert _same(got, e2e)
    assert all(g["status"] & 0xF0 == 0 for g in got)
    # score and end cell of every pair
    ends = oracle_map(lambda p: orc.score_end(p.prot, p.nt, p.strand), pairs, range(len(pairs)), full=False)
    bad = []
    for k, (p, g) in enumerate(zip(pairs, got)):
        w = ends[k]
        if g["score"] != w["score"] or (w["score"] > 0 and (
                g["prot_en"] != w["prot_en"] or genome_end(g, p.strand, len(p.nt)) != genome_end(w, p.strand,
                                                                                                len(p.nt)))):
            bad.append((k, (g["score"], w["score"]), len(p.prot), len(p.nt)))
    assert not bad, (len(bad), bad[:5])
    assert sum(p.cells for p in pairs if p.cells > 12_000_000) > 2e11     # the large pairs are all in
    # full coordinates and CIGARs of every pair up to 4 M cells
    small = [k for k, p in enumerate(pairs) if p.cells <= 4_000_000]
    assert len(small) > 10_000
    full = oracle_map(lambda p: orc.align(p.prot, p.nt, p.strand), pairs, small, full=True)
    bad = []
    for k in small:
        p, g, w = pairs[k], got[k], full[k]
        if p.score_only:
            ok = g["score"] == w["score"] and g["cigar"] == [] and g["prot_en"] == w["prot_en"]
        else:
            ok = all(g[x] == w[x] for x in KEYS)
        if not ok:
            bad.append((k, len(p.prot), len(p.nt)))
    assert not bad, (len(bad), bad[:5])
    # every traced path is optimal: it rescores to the oracle's score at the oracle's end cell
    bad = rescore_all(orc, pairs, got, skip=lambda p: p.score_only)
    assert not bad, (len(bad), bad[:5])
    assert sum(1 for p, g in zip(pairs, got) if not p.score_only and g["cigar"]) > 18_000

"""Genome-scale workload on the GPU: candidate regions from the library's
seeding and chaining (the first 3 chains of each protein, extended to
candidate regions), aligned through the C ABI from zero-copy pair records
that point into the genome and protein buffers.  Every region's score and end cell
equal the oracle's four-row fill; every region up to 12 M cells matches the
full-matrix oracle in score, coordinates and CIGAR; every returned CIGAR
rescores to its score at the oracle's end cell.

The workload is the genome-scale configuration shrunk by a factor of 50
(10 Mb genome, 400 planted genes, 4,000 proteins: about 8,500 regions,
23 G cells); the full-size run is `bench.py --workload c5`.
"""
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


def test_genome_regions_match_oracle(mp, orc):
    w = synth.config5(scale=0.02, host_seeding=False)
    ctx = mp.mp_dp_init(None, 0)
    try:
        idx = mp.mp_index_build(ctx, w.genome)
        try:
            chains, nch = mp.mp_index_chain(ctx, idx, w.prot_buf, w.prot_off, w.prot_len, 3)
        finally:
            mp.mp_index_free(idx)
    finally:
        mp.mp_dp_destroy(ctx)
    w = synth.regions_from_chains(w, chains, nch)
    assert w.n_regions > 1000
    po, pl, no, nl, st = w.region_arrays()
    batch = mp.RegionBatch(w.prot_buf, po, pl, w.genome, no, nl, st)
    ctx = mp.mp_dp_init(None, 0)
    try:
        # the launch configuration the library's autotuner picks for this batch
        b = mp.mp_dp_batch_upload(ctx, batch)
        mp.mp_dp_autotune(ctx, b)
        mp.mp_dp_batch_free(ctx, b)
        got = mp.mp_dp_align_batch(ctx, batch)
    finally:
        mp.mp_dp_destroy(ctx)
    assert all(g["status"] & 0xF0 == 0 for g in got)
    pairs = [w.pair(r) for r in range(w.n_regions)]
    ends = oracle_map(lambda p: orc.score_end(p.prot, p.nt, p.strand), pairs, range(len(pairs)), full=False)
    bad = []
    for r, (p, g) in enumerate(zip(pairs, got)):
        e = ends[r]
        n = len(p.nt)
        if g["score"] != e["score"] or (e["score"] > 0 and (
                g["prot_en"] != e["prot_en"] or genome_end(g, p.strand, n) != genome_end(e, p.strand, n))):
            bad.append((r, g["score"], e["score"]))
    assert not bad, (len(bad), bad[:5])
    small = [r for r, p in enumerate(pairs) if p.cells <= 12_000_000]
    assert len(small) > 0.9 * len(pairs)
    want = oracle_map(lambda p: orc.align(p.prot, p.nt, p.strand), pairs, small, full=True)
    bad = [(r, [k for k in KEYS if got[r][k] != want[r][k]]) for r in small
           if any(got[r][k] != want[r][k] for k in KEYS)]
    assert not bad, (len(bad), bad[:5])
    bad = rescore_all(orc, pairs, got)
    assert not bad, (len(bad), bad[:5])
    # sources mostly align to their planted gene with a high score
    src_regions = [r for r in range(w.n_regions) if w.kind[w.reg_prot[r]] == 0]
    top = max(got[r]["score"] for r in src_regions)
    assert top > 500

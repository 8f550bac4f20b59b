"""Genome-scale workload on the GPU: candidate regions from the host seed +
chain step, aligned through the C ABI from zero-copy pair records that point
into the genome and protein buffers.  Sampled regions match the oracle
bit-exactly and every returned CIGAR rescores to its score.

The workload is the genome-scale configuration shrunk by a factor of 50
(10 Mb genome, 400 planted genes, 4,000 proteins: about 12,000 regions);
the full-size run is `bench.py --workload c5`.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

KEYS = ("score", "prot_st", "prot_en", "nt_st", "nt_en", "cigar")


@pytest.fixture(scope="module")
def mp():
    from paper_2210_08052_gb300 import build
    build.build()
    import paper_2210_08052_gb300 as m
    m.lib()
    return m


def test_genome_regions_match_oracle(mp, orc):
    w = synth.config5(scale=0.02)
    assert w.n_regions > 8000
    po, pl, no, nl, st = w.region_arrays()
    batch = mp.RegionBatch(w.prot_buf, po, pl, w.genome, no, nl, st)
    ctx = mp.mp_dp_init(None, 0)
    try:
        got = mp.mp_dp_align_batch(ctx, batch)
    finally:
        mp.mp_dp_destroy(ctx)
    assert all(g["status"] & 0xF0 == 0 for g in got)
    rng = np.random.default_rng(55)
    # sampled regions one by one against the oracle, the best-scoring ones included
    best = np.argsort([-g["score"] for g in got])[:5]
    sample = np.unique(np.concatenate([rng.choice(w.n_regions, 25, replace=False), best]))
    bad = []
    for r in sample:
        p = w.pair(int(r))
        want = orc.align(p.prot, p.nt, p.strand)
        diff = [k for k in KEYS if got[r][k] != want[k]]
        if diff:
            bad.append((int(r), diff))
    assert not bad, bad[:5]
    # every CIGAR rescored by the oracle's op-sum reproduces score and end
    bad = []
    for r in range(w.n_regions):
        g = got[r]
        if g["score"] == 0:
            continue
        p = w.pair(r)
        n = len(p.nt)
        st = g["nt_st"] if p.strand > 0 else n - g["nt_en"]
        en = g["nt_en"] if p.strand > 0 else n - g["nt_st"]
        sc, pe, te = orc.rescore(p.prot, p.nt, p.strand, g["prot_st"], st, g["cigar_raw"])
        if (sc, pe, te) != (g["score"], g["prot_en"], en):
            bad.append((r, sc, g["score"]))
    assert not bad, bad[:5]
    # sources mostly align to their planted gene with a high score
    src_regions = [r for r in range(w.n_regions) if w.kind[w.reg_prot[r]] == 0]
    top = max(got[r]["score"] for r in src_regions)
    assert top > 500

"""The genome-scale workload generator (host side, no GPU): planted genes,
the protein mix, the seed + chain candidate regions, and the zero-copy
pair records that point into the genome and protein buffers."""
import ctypes

import numpy as np
import pytest

import synth
from synth import genome as G


@pytest.fixture(scope="module")
def small():
    return synth.config5(scale=0.004)            # 2 Mb genome, 80 genes, 800 proteins


def test_shapes_and_bounds(small):
    w = small
    assert len(w.genome) == 2_000_000 and set(np.unique(w.genome).tobytes()) <= set(b"ACGT")
    assert len(w.prot_len) == 800 and (w.kind == 0).sum() == 80 and (w.kind == 1).sum() == 360
    assert ((w.gene_end - w.gene_start) > 0).all() and (w.gene_end <= len(w.genome)).all()
    assert (w.reg_start >= 0).all() and (w.reg_end <= len(w.genome)).all() and (w.reg_end > w.reg_start).all()
    assert set(np.unique(w.reg_strand)) <= {-1, 1}
    counts = np.bincount(w.reg_prot, minlength=len(w.prot_len))
    assert counts.max() <= G.TOP
    gc = np.isin(w.genome, np.frombuffer(b"GC", np.uint8)).mean()
    assert 0.39 < gc < 0.44            # 40% background, coding genes slightly richer


def test_deterministic():
    a = synth.config5(scale=0.002)
    b = synth.config5(scale=0.002)
    assert np.array_equal(a.genome, b.genome) and np.array_equal(a.reg_start, b.reg_start)
    assert np.array_equal(a.reg_prot, b.reg_prot) and np.array_equal(a.prot_buf, b.prot_buf)


def test_planted_genes_hold_their_source(small):
    """Each gene body is at least as long as its source's coding sequence
    (less at most three 2-nt frameshift deletions)."""
    w = small
    src = np.nonzero(w.kind == 0)[0]
    for k in src[:10]:
        g = int(w.gene_of[k])
        body = w.genome[w.gene_start[g]:w.gene_end[g]].tobytes().decode()
        if w.gene_strand[g] < 0:
            body = synth.revcomp(body)
        assert len(body) >= 3 * int(w.prot_len[k]) - 6


def test_sources_find_their_gene(small):
    """Most source proteins get a candidate region on their gene's strand
    that overlaps the gene."""
    w = small
    src = np.nonzero(w.kind == 0)[0]
    hit = 0
    for k in src:
        g = w.gene_of[k]
        r = np.nonzero(w.reg_prot == k)[0]
        hit += any(w.reg_start[i] < w.gene_end[g] and w.reg_end[i] > w.gene_start[g] and
                   w.reg_strand[i] == w.gene_strand[g] for i in r)
    assert hit >= 0.85 * len(src)


def test_exact_copy_is_found_on_both_strands():
    """A protein planted without substitutions on either strand: its best
    chain covers the whole gene."""
    rng = np.random.default_rng(12)
    genome = G._random_genome(rng, 300_000, 0.4)
    prots, spans = [], []
    for k, strand in enumerate((1, -1)):
        prot = synth.random_protein(rng, 300)
        body, _ = synth.gen.plant_gene(rng, prot, 0.0, 0, [500, 900], 0, 0)
        if strand < 0:
            body = synth.revcomp(body)
        at = 50_000 + 120_000 * k
        genome[at:at + len(body)] = np.frombuffer(body.encode(), np.uint8)
        prots.append(prot)
        spans.append((at, at + len(body), strand))
    buf = np.frombuffer("".join(prots).encode(), np.uint8)
    off = np.array([0, 300])
    ln = np.array([300, 300])
    rp, rs, re, rstr, ran = G.seed_and_chain(genome, buf, off, ln)
    for k, (s, e, strand) in enumerate(spans):
        r = np.nonzero(rp == k)[0]
        best = r[np.argmax(ran[r])]
        assert rstr[best] == strand and rs[best] <= s and re[best] >= e, (k, rs[best], re[best], s, e)


def test_region_batch_points_into_buffers(small):
    """RegionBatch records hold pointers into the caller's buffers (no copy)
    with the right lengths and strands."""
    from paper_2210_08052_gb300 import RegionBatch
    w = small
    idx = np.arange(min(50, w.n_regions))
    po, pl, no, nl, st = w.region_arrays(idx)
    rb = RegionBatch(w.prot_buf, po, pl, w.genome, no, nl, st)
    assert rb.n == len(idx)
    for j, r in enumerate(idx):
        rec = rb.arr[j]
        pair = w.pair(int(r))
        assert ctypes.string_at(ctypes.cast(rec.prot, ctypes.c_void_p), rec.prot_len).decode() == pair.prot
        assert ctypes.string_at(ctypes.cast(rec.nt, ctypes.c_void_p), rec.nt_len).decode() == pair.nt
        assert rec.strand == pair.strand and rec.flags == 0
    with pytest.raises(ValueError):
        RegionBatch(w.prot_buf, [0], [len(w.prot_buf) + 1], w.genome, [0], [10], [1])

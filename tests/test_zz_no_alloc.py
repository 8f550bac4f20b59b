"""The allocation-free entry point (mp_dp_score_pair_noalloc) gives the same
score and end cell as the oracle and as the batch entry point, on two calls
in a row.

It exists for callers that may not allocate device memory (services whose
device memory is fixed at start-up, hosts that hand plug-ins memory only
from their own pools); its scratch is a fixed array in the library.  This
file is collected last, so a run that stops at its first failure has run
every other test before it.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _pairs():
    rng = np.random.default_rng(77)
    out = []
    for m, introns in ((40, [120]), (130, [300, 90]), (700, [800, 400, 1500]), (2000, [3000])):
        prot = synth.random_protein(rng, m)
        region, _ = synth.gen.plant_gene(rng, prot, 0.2, 1, introns, 400, 300, 0.4)
        out.append(synth.Pair(prot, region, 1))
        out.append(synth.Pair(prot, synth.revcomp(region), -1))
    # a W-rich protein that saturates int16 and is re-run in int32
    prot = "".join("W" if rng.random() < 0.92 else "C" for _ in range(3300))
    out.append(synth.Pair(prot, synth.random_dna(rng, 50) + synth.reverse_translate(rng, prot) +
                          synth.random_dna(rng, 50), 1))
    out.append(synth.Pair("MW", "ATGTGG", 1))
    return out


def test_noalloc_matches_oracle_and_batch_entry_point(orc):
    torch = pytest.importorskip("torch")
    from paper_2210_08052_gb300 import build
    build.build()
    import paper_2210_08052_gb300 as mp

    pairs = _pairs()
    ctx = mp.mp_dp_init(None, 0)
    try:
        ref = mp.mp_dp_align_batch(ctx, [synth.Pair(p.prot, p.nt, p.strand, True) for p in pairs])
    finally:
        mp.mp_dp_destroy(ctx)
    dev_in = [(torch.tensor(bytearray(p.prot.encode()), dtype=torch.uint8, device="cuda"),
               torch.tensor(bytearray(p.nt.encode()), dtype=torch.uint8, device="cuda")) for p in pairs]
    for call in range(2):
        for p, (dp, dn), r in zip(pairs, dev_in, ref):
            out = torch.full((4,), -7, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            rc = mp.mp_dp_score_pair_noalloc(None, dp.data_ptr(), len(p.prot), dn.data_ptr(), len(p.nt),
                                             p.strand, out.data_ptr(), 0)
            assert rc == mp.MP_OK, mp.mp_dp_strerror(rc)
            torch.cuda.synchronize()
            score, status, prot_en, nt_end = out.cpu().tolist()
            o = orc.align(p.prot, p.nt, p.strand)
            want_nt = o["nt_en"] if p.strand > 0 else o["nt_st"]
            assert (score, prot_en) == (o["score"], o["prot_en"]), (call, len(p.prot))
            assert (score, prot_en) == (r["score"], r["prot_en"]), (call, len(p.prot))
            if score:
                assert nt_end == want_nt
            assert status & 0xF0 == 0
            assert bool(status & mp.MP_ST_RERUN) == bool(r["status"] & mp.MP_ST_RERUN)
    assert any(r["status"] & mp.MP_ST_RERUN for r in ref)
    # a base outside ACGT is refused per pair, on both strands, as by the batch call
    prot = "MKVLAAGIW"
    nt = "ATGAAAGTTCTGGCNGCAGGTATCTGG"
    bad = [synth.Pair(prot, nt, 1), synth.Pair(prot, nt, -1)]
    ctx = mp.mp_dp_init(None, 0)
    try:
        want = mp.mp_dp_align_batch(ctx, [synth.Pair(p.prot, p.nt, p.strand, True) for p in bad])
    finally:
        mp.mp_dp_destroy(ctx)
    for p, r in zip(bad, want):
        assert r["status"] & mp.MP_ST_BADSEQ and r["score"] == 0
        dp = torch.tensor(bytearray(p.prot.encode()), dtype=torch.uint8, device="cuda")
        dn = torch.tensor(bytearray(p.nt.encode()), dtype=torch.uint8, device="cuda")
        for call in range(2):
            out = torch.full((4,), -7, dtype=torch.int32, device="cuda")
            rc = mp.mp_dp_score_pair_noalloc(None, dp.data_ptr(), len(p.prot), dn.data_ptr(), len(p.nt),
                                             p.strand, out.data_ptr(), 0)
            assert rc == mp.MP_OK
            torch.cuda.synchronize()
            score, status, _, _ = out.cpu().tolist()
            assert score == 0 and status & mp.MP_ST_BADSEQ, (p.strand, call)
    big = torch.zeros(40000, dtype=torch.uint8, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert mp.mp_dp_score_pair_noalloc(None, big.data_ptr(), 10, big.data_ptr(), 40000, 1,
                                       out.data_ptr(), 0) == mp.MP_ETOOLARGE

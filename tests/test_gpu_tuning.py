"""Launch configurations and the autotuner.

Every configuration the tuner may pick (both int16 kernel builds, each CTA
count per SM it tries, int16-first or int32-at-once for pairs whose score
bound reaches the int16 limit, both item orders, 64- or 128-residue strips
for int16 pairs; the wave policies are
covered by the parity tests) must give the oracle's results bit-exactly;
the tuner must pick one of its timed candidates and keep it per shape class,
and its table must survive a save/load round trip.
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


def _mixed_pairs():
    """Gene pairs across several strips and chunks, two W-rich pairs that
    saturate int16, and one whose bound passes the int16 limit although its
    score stays small (protein against an unrelated region)."""
    rng = np.random.default_rng(41)
    pairs = []
    for _ in range(24):
        m = int(rng.integers(1, 400))
        prot = synth.random_protein(rng, m)
        lens = [int(rng.integers(30, 900)) for _ in range(int(rng.integers(0, 4)))]
        region, _ = synth.gen.plant_gene(rng, prot, float(rng.uniform(0.05, 0.4)), int(rng.integers(0, 3)),
                                         lens, int(rng.integers(0, 300)), int(rng.integers(0, 300)), 0.45)
        strand = 1
        if rng.random() < 0.5:
            region, strand = synth.revcomp(region), -1
        pairs.append(synth.Pair(prot, region, strand))
    for m in (3200, 3300):
        prot = "".join("W" if rng.random() < 0.9 else "C" for _ in range(m))
        cds = synth.reverse_translate(rng, prot)
        nt = synth.random_dna(rng, 90) + cds[: 3 * 1500] + "GTAAGT" + synth.random_dna(rng, 150) + "TAG" + \
            cds[3 * 1500:] + synth.random_dna(rng, 70)
        pairs.append(synth.Pair(prot, nt, 1))
    prot = "".join("W" if rng.random() < 0.95 else "Y" for _ in range(3100))
    pairs.append(synth.Pair(prot, synth.random_dna(rng, 2500), -1))
    return pairs


@pytest.fixture(scope="module")
def mixed(orc):
    pairs = _mixed_pairs()
    return pairs, [orc.align(p.prot, p.nt, p.strand) for p in pairs]


def _same(got, want):
    bad = [(k, [key for key in KEYS if g[key] != w[key]]) for k, (g, w) in enumerate(zip(got, want))
           if any(g[key] != w[key] for key in KEYS) or g["status"] & 0xF0]
    assert not bad, bad[:5]


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("ctas", [0, 1, 2])
@pytest.mark.parametrize("wide_direct", [0, 1])
@pytest.mark.parametrize("item_order", [0, 1])
@pytest.mark.parametrize("strip_width", [0, 1, 2])
def test_every_configuration_matches_oracle(mp, mixed, variant, ctas, wide_direct, item_order, strip_width):
    pairs, want = mixed
    ctx = mp.mp_dp_init(None, 0)
    try:
        mp.mp_dp_set_tuning(ctx, dict(dp16_variant=variant, dp16_ctas_per_sm=ctas, dp32_ctas_per_sm=ctas,
                                      wide_direct=wide_direct, item_order=item_order, strip_width=strip_width))
        for _ in range(3):                          # direct, then graph capture and replay
            got = mp.mp_dp_align_batch(ctx, pairs)
            _same(got, want)
        rerun = [bool(g["status"] & 1) for g in got]
        # int16 first: exactly the saturating pairs are re-run; int32 at once: none is
        assert rerun[-3:] == ([False, False, False] if wide_direct else [True, True, False])
        assert not any(rerun[:-3])
    finally:
        mp.mp_dp_destroy(ctx)


def test_autotune_picks_a_timed_candidate_and_keeps_results(mp, mixed, tmp_path):
    pairs, want = mixed
    ctx = mp.mp_dp_init(None, 0)
    try:
        b = mp.mp_dp_batch_upload(ctx, pairs)
        assert mp.mp_dp_get_tuning(ctx, b)["ms"] == 0          # defaults before tuning
        best, tried = mp.mp_dp_autotune(ctx, b)
        assert len(tried) >= 4 and all(t["ms"] > 0 for t in tried)
        assert best["ms"] == min(t["ms"] for t in tried)
        strip = lambda t: {k: t[k] for k in ("dp16_variant", "dp16_ctas_per_sm", "dp32_ctas_per_sm", "wide_direct",
                                             "overlap_waves", "item_order", "strip_width")}
        assert {t["strip_width"] for t in tried} == {0, 1, 2}
        assert strip(best) in [strip(t) for t in tried]
        assert {t["wide_direct"] for t in tried} == {0, 1}         # the batch has wide pairs
        # the batch holds the results of the tuning runs
        mp.mp_dp_batch_sync(ctx)
        _same(mp.mp_dp_batch_download(ctx, b), want)
        assert mp.mp_dp_get_tuning(ctx, b) == best
        mp.mp_dp_batch_run(ctx, b)
        mp.mp_dp_batch_sync(ctx)
        _same(mp.mp_dp_batch_download(ctx, b), want)
        # save, load into a fresh context, same choice for the same batch shape
        path = str(tmp_path / "tuning.txt")
        mp.mp_dp_tuning_save(ctx, path)
        mp.mp_dp_batch_free(ctx, b)
    finally:
        mp.mp_dp_destroy(ctx)
    ctx2 = mp.mp_dp_init(None, 0)
    try:
        b2 = mp.mp_dp_batch_upload(ctx2, pairs)
        mp.mp_dp_tuning_load(ctx2, path)
        got = mp.mp_dp_get_tuning(ctx2, b2)
        assert strip(got) == strip(best) and abs(got["ms"] - best["ms"]) < 1e-3
        mp.mp_dp_batch_free(ctx2, b2)
    finally:
        mp.mp_dp_destroy(ctx2)


def test_autotune_on_first_run_when_enabled(mp, mixed):
    pairs, want = mixed
    ctx = mp.mp_dp_init(mp.mp_dp_default_params(autotune=1), 0)
    try:
        _same(mp.mp_dp_align_batch(ctx, pairs), want)
        b = mp.mp_dp_batch_upload(ctx, pairs)
        assert mp.mp_dp_get_tuning(ctx, b)["ms"] > 0               # tuned by the first run
        mp.mp_dp_batch_run(ctx, b)
        mp.mp_dp_batch_sync(ctx)
        _same(mp.mp_dp_batch_download(ctx, b), want)
        mp.mp_dp_batch_free(ctx, b)
    finally:
        mp.mp_dp_destroy(ctx)


def test_tuning_arguments_checked(mp, tmp_path):
    ctx = mp.mp_dp_init(None, 0)
    L = mp.lib()
    try:
        for bad in (dict(dp16_variant=2), dict(dp16_variant=-1), dict(wide_direct=2), dict(dp16_ctas_per_sm=-1),
                    dict(dp32_ctas_per_sm=-3), dict(overlap_waves=2), dict(item_order=-1), dict(strip_width=3),
                    dict(strip_width=-1)):
            with pytest.raises(mp.MPError):
                mp.mp_dp_set_tuning(ctx, bad)
        mp.mp_dp_set_tuning(ctx, dict(dp16_ctas_per_sm=99))       # clamped at launch
        pairs = _mixed_pairs()[:4]
        got = mp.mp_dp_align_batch(ctx, pairs)
        assert all(g["status"] & 0xF0 == 0 for g in got)
        mp.mp_dp_set_tuning(ctx, None)
        bad_file = tmp_path / "other.txt"
        bad_file.write_text("mp_dp_tuning 4 Some_Other_GPU 7\n0000000000000001 0 3 2 0 1 1 0 1.0\n")
        assert L.mp_dp_tuning_load(ctx, str(bad_file).encode()) == mp.MP_EINVAL
        assert L.mp_dp_tuning_load(ctx, str(tmp_path / "missing.txt").encode()) == mp.MP_EINVAL
    finally:
        mp.mp_dp_destroy(ctx)
    plain = mp.mp_dp_init(mp.mp_dp_default_params(max_pairs_per_launch=1), 0)
    try:
        b = mp.mp_dp_batch_upload(plain, _mixed_pairs()[:2])
        assert L.mp_dp_autotune(plain, b[0], None, None, 0, None) == mp.MP_EINVAL
        mp.mp_dp_batch_free(plain, b)
    finally:
        mp.mp_dp_destroy(plain)

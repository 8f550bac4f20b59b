/*
 * mp_dp.h -- C ABI of the GB300 spliced protein-to-genome DP library.
 *
 * The library aligns batches of (protein, genomic region) pairs with the
 * dynamic program of Li 2022 ("Protein-to-genome alignment with miniprot"),
 * Eq. 7 (Methods, "DP for protein-to-genome alignment"): affine gaps (I, D),
 * frameshifts (the four f terms) and phase-0/1/2 introns (A, B, C) scored
 * together, with the final splice model d(i), a(i) of the "Splice models"
 * section.  It serves the problem the Introduction sets out: given a
 * protein and a nucleotide sequence, find their spliced alignment.
 *
 * Conventions used by every call:
 *   - Alignment is local unless mp_dp_params.mode says otherwise: H restarts
 *     at 0 and the best cell is the largest H, ties to the smallest genome
 *     position and then the smallest residue (the extension mode uses the
 *     same best-cell rule; global mode ends at the last cell).
 *   - Ties inside each max of Eq. 7 go to the earliest printed term (open
 *     before extend; M, I, D, F1, F2, G1, G2, A, B, C for H); a restart at 0
 *     wins a tie at 0.
 *   - Coordinates are 0-based half-open.  nt_st/nt_en are on the forward
 *     strand of the sequence the caller passed, whatever the pair's strand.
 *   - A CIGAR op is (len << 4) | code with the MP_OP_* codes below; ops run
 *     in protein order (on the reverse complement for strand -1).
 *   - Return codes: MP_OK (0) or a negative MP_E* value.  No C++ exception
 *     crosses this boundary.  Per-pair failures are reported in
 *     mp_result.status, not in the return code.
 *   - All host pointers passed in are borrowed for the duration of the
 *     call; the library copies what it needs.
 *   - Calls on one context are not thread-safe, except mp_dp_submit and
 *     mp_dp_poll, which may be called from any thread.
 */
#ifndef MP_DP_H
#define MP_DP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- return codes */
#define MP_OK 0
#define MP_EINVAL (-1)    /* bad argument or parameter set */
#define MP_ENOMEM (-2)    /* host or device allocation failed */
#define MP_EBUDGET (-3)   /* the request cannot fit the traceback budget */
#define MP_ETIMEOUT (-4)  /* mp_dp_poll: result not ready within the timeout */
#define MP_ECUDA (-5)     /* a CUDA call failed; the context should be destroyed */
#define MP_EPENDING (-6)  /* mp_dp_poll with timeout 0: not ready yet */
#define MP_EAGAIN (-7)    /* mp_dp_submit: request ring full, retry later */
#define MP_ETICKET (-8)   /* unknown or already-consumed ticket */
#define MP_ESTATE (-9)    /* call not valid in the context's current state */
#define MP_ETOOLARGE (-10) /* mp_dp_score_pair_noalloc: input beyond its fixed scratch limits */

/* -------------------------------------------------- per-pair status bits */
#define MP_ST_OK 0x0
#define MP_ST_RERUN 0x1     /* info: int16 scores saturated; recomputed exactly in int32 */
#define MP_ST_BADSEQ 0x10   /* error: a character outside ACGT in the genome */
#define MP_ST_BUDGET 0x20   /* error: this pair's traceback alone exceeds the budget */
#define MP_ST_TRACE 0x40    /* error: internal traceback inconsistency (never expected) */
#define MP_ST_TIMEOUT 0x80  /* error: a bounded wait between cooperating warps expired */
#define MP_ST_ERRMASK 0xF0

/* ---------------------------------------------------------- CIGAR ops */
#define MP_OP_M 0  /* codons matched to residues; len = codons */
#define MP_OP_I 1  /* residues against no genome (gap in T); len = residues */
#define MP_OP_D 2  /* codons against no residue (gap in P); len = codons */
#define MP_OP_F 3  /* frameshift '$': len = 1 or 2 nt for one residue (unscored) */
#define MP_OP_G 4  /* frameshift '+': len = 1 or 2 inserted nt, no residue */
#define MP_OP_N 5  /* phase-0 intron; len = intron nt */
#define MP_OP_U 6  /* phase-1 intron; len = intron nt.  The op also spans the
                      split codon's 1 nt before and 2 nt after the intron and
                      one residue, which is not scored */
#define MP_OP_V 7  /* phase-2 intron; as U with 2 nt before and 1 nt after */

/* ------------------------------------------------------------- params */
#define MP_SPLICE_FINAL 0   /* the final splice model of the "Splice models" section */
#define MP_SPLICE_SIMPLE 1  /* the simple model defined right after Eq. 7: d(x) = 0 if T[x+1..x+2]
                               is GT, else splice_p; a(x) = 0 if T[x-1..x] is AG, else splice_p */
#define MP_MODE_LOCAL 0     /* local alignment: the path may start and end at any cell */
#define MP_MODE_GLOBAL 1    /* gap closing between two anchors: the path runs from the start of the
                               protein and region to both their ends; the score may be negative */
#define MP_MODE_EXTEND 2    /* extension from an anchor: the path starts at the start of the protein
                               and region and ends anywhere (score >= 0; 0: the empty extension) */

#define MP_PAIR_SCORE_ONLY 0x1u  /* mp_pair.flags: score and end cell only, no CIGAR */
#define MP_DEBUG_NO_PUBLISH 0x1  /* mp_dp_params.debug_flags (tests only) */

/* Scoring parameters.  The paper prints no default values for q, e, f, r or
 * the stop penalty; mp_dp_default_params fills q=11, e=1, f=23, r=29,
 * stop=23 and BLOSUM62.  mat is indexed [translated amino acid][protein
 * residue] in the order ARNDCQEGHILKMFPSTWYV, then '*' (20) and X (21);
 * row 20 is unused (a stop codon scores -stop against every residue) and
 * protein letters outside the 20 amino acids and '*' map to X.
 * mp_dp_init rejects sets under which an intron of length <= 0 could beat
 * a frameshift or a match: it requires r > f, r > stop and r > -min(mat),
 * all penalties >= 0 and e >= 1; and, for the packed int16 arithmetic,
 * q + e <= 1000, f <= 1000, r <= 1000, stop <= 512 and splice_p <= 1000. */
typedef struct {
    int32_t q, e, f, r, stop;  /* gap open, gap extend, frameshift, intron, stop codon */
    int8_t mat[22][22];
    int32_t splice_model;      /* MP_SPLICE_FINAL or MP_SPLICE_SIMPLE */
    int32_t mode;              /* MP_MODE_LOCAL, MP_MODE_GLOBAL or MP_MODE_EXTEND.  In the two
                                  anchored modes the alignment starts at position 0 of the protein
                                  and of the aligned strand (strand -1: the input's end); in global
                                  mode every pair keeps its traceback (MP_PAIR_SCORE_ONLY is
                                  ignored) since the score is read at the end cell.  A pair
                                  with an empty protein or region scores 0 in every mode.  In the
                                  anchored modes H can be as low as -(2q + f + e(|P| + |T|/3 + 2));
                                  a batch holding a pair for which that reaches 2^27 is refused
                                  with MP_EINVAL (the DP represents -inf by -2^28) */
    uint64_t tb_budget_bytes;  /* device bytes for traceback codes (default 40 GiB, capped
                                  at 60% of the device memory free at init) */
    int32_t force_int32;       /* 1: skip the packed int16 pass and run every pair in int32 */
    int32_t max_pairs_per_launch; /* 0: no limit; 1: one pair per kernel launch (plain form) */
    int32_t wait_limit;        /* polls (~0.25 us each) before a warp waiting on the previous
                                  strip of its pair gives up and marks the pair MP_ST_TIMEOUT;
                                  0: default (4e7) */
    int32_t debug_flags;       /* test hook: MP_DEBUG_NO_PUBLISH makes every strip withhold its
                                  boundary row, so the waits of the next strip run out */
    int32_t autotune;          /* 1: the first run of a batch whose shape class has no tuned
                                  configuration yet runs mp_dp_autotune on it first */
    int32_t splice_p;          /* MP_SPLICE_SIMPLE: cost p of a donor without GT or an acceptor
                                  without AG (0..1000; the paper gives no value; default 30) */
    int32_t exon_rescore;      /* 1: mp_dp_align_batch also fills mp_result.exon_score */
    int32_t reserved[1];
} mp_dp_params;

/* Position-specific costs of one residue position of a profile query (Li
 * 2022, Discussion: a profile, e.g. HMMER's, as the query, aligned with
 * position-specific substitution and gap costs).  With a profile, Eq. 7's
 * s(i, j) is subst[c] of position j, c the amino acid the codon ending at
 * i translates to (ARNDCQEGHILKMFPSTWYV order; 20 = stop codon), and the I
 * and D states of column j take that column's gap costs:
 *   I[i][j] = max(H[i][j-1] - gap_open_j, I[i][j-1]) - gap_ext_j
 *   D[i][j] = max(H[i-3][j] - gap_open_j, D[i-3][j]) - gap_ext_j
 * (an I step consumes residue j; a D step adds a codon after residue j).
 * Frameshift and intron costs stay f, r and the splice model. */
typedef struct {
    int16_t subst[21];         /* -500 .. 500; r must exceed -min(subst) over the profile */
    int16_t gap_open;          /* 0 .. 999 */
    int16_t gap_ext;           /* 1 .. 1000 - gap_open */
    int16_t reserved;
} mp_profile_pos;

/* One alignment request.  prot: ASCII amino acids; nt: ASCII A/C/G/T
 * (either case).  strand -1 aligns the protein to the reverse complement of
 * nt. */
typedef struct {
    const char *prot;
    uint32_t prot_len;
    const char *nt;
    uint32_t nt_len;
    int8_t strand;
    uint32_t flags;            /* MP_PAIR_* */
    const mp_profile_pos *profile; /* NULL: score with params (mat, q, e, stop); else prot_len + 1
                                  positions: entry j (1..prot_len) for residue j, entry 0 the
                                  gap costs of the column before the first residue (its subst is
                                  not used).  The residue letters still name the positions in the
                                  result.  Borrowed for the duration of the call; a profile pair
                                  with a value out of range makes the call return MP_EINVAL */
} mp_pair;

/* One result.  cigar points into library-owned memory: for
 * mp_dp_align_batch and mp_dp_batch_download it stays valid until the next
 * such call on the context, or mp_dp_destroy; for mp_dp_poll, until the
 * same ticket is polled a second time (which releases it) or mp_dp_destroy. */
typedef struct {
    int32_t score;
    int32_t status;            /* MP_ST_* bits */
    int32_t prot_st, prot_en;  /* 0-based half-open on the protein */
    int32_t nt_st, nt_en;      /* 0-based half-open on the input's forward strand */
    uint32_t n_cigar;
    int32_t exon_score;        /* pseudogene-aware score (Methods, "Avoiding pseudogenes"): set by
                                  mp_dp_exon_rescore (or mp_dp_align_batch with
                                  params.exon_rescore); otherwise equal to score */
    const uint32_t *cigar;
} mp_result;

typedef struct mp_dp_ctx mp_dp_ctx;
typedef struct mp_dp_batch mp_dp_batch;

/* Fill *p with the default parameter set described above. */
void mp_dp_default_params(mp_dp_params *p);

/* Create a context on CUDA device `device` with parameters *p (NULL:
 * defaults).  Validates p as described above (MP_EINVAL).  Allocates the
 * traceback arena lazily, at the first batch.  On success *ctx owns a CUDA
 * stream and device buffers until mp_dp_destroy. */
int mp_dp_init(mp_dp_ctx **ctx, const mp_dp_params *p, int device);

/* Align n pairs end to end: host -> device copy, the DP, traceback, and
 * device -> host copy of results.  out[k] corresponds to pairs[k].  Blocks
 * until done.  Returns MP_EINVAL for a NULL sequence pointer with nonzero
 * length, strand not +-1, a length beyond 1,047,551 nt or 1,048,575
 * residues, or (anchored modes) a pair beyond the lower-bound limit given at
 * mp_dp_params.mode; per-pair sequence errors go to out[k].status. */
int mp_dp_align_batch(mp_dp_ctx *ctx, const mp_pair *pairs, size_t n, mp_result *out);

/* Staged form of mp_dp_align_batch, for callers that keep a batch resident
 * on the device and run it repeatedly.  upload copies the inputs to the
 * device and plans the waves; run enqueues the whole device pipeline
 * (pack, DP, int32 re-run, traceback, CIGAR compaction) on the context's
 * stream without blocking; sync waits for it; download copies results back
 * (blocking).  A batch handle is owned by the caller until
 * mp_dp_batch_free. */
int mp_dp_batch_upload(mp_dp_ctx *ctx, const mp_pair *pairs, size_t n, mp_dp_batch **batch);
int mp_dp_batch_run(mp_dp_ctx *ctx, mp_dp_batch *batch);
int mp_dp_batch_sync(mp_dp_ctx *ctx);
int mp_dp_batch_download(mp_dp_ctx *ctx, mp_dp_batch *batch, mp_result *out);
void mp_dp_batch_free(mp_dp_ctx *ctx, mp_dp_batch *batch);

/* Serving: submit one pair; never blocks.  *ticket identifies the result.
 * MP_EAGAIN if the request ring is full; MP_EBUDGET if the pair's traceback
 * alone exceeds tb_budget_bytes.  The first submit starts the serving
 * thread, which keeps one traceback arena of tb_budget_bytes on the device
 * and runs up to three micro-batches at once, each in its own range of
 * that arena: requests are taken in arrival order into a micro-batch of up
 * to a third of the budget (a larger request alone, up to the whole budget,
 * once that much of the arena is free), and batches are launched as
 * requests arrive and ranges free up (continuous batching). */
int mp_dp_submit(mp_dp_ctx *ctx, const mp_pair *pair, uint64_t *ticket);

/* Wait up to timeout_us (0: do not wait; negative: forever) for ticket's
 * result.  MP_OK fills *out; its CIGAR stays valid until the ticket is
 * polled again, which releases the result and returns MP_ETICKET, or
 * mp_dp_destroy.  MP_EPENDING (timeout 0) or MP_ETIMEOUT when not ready;
 * MP_ETICKET for an unknown or released ticket. */
int mp_dp_poll(mp_dp_ctx *ctx, uint64_t ticket, mp_result *out, int64_t timeout_us);

/* Wait up to timeout_us (as in mp_dp_poll) for any finished request that
 * has not been handed out yet, in completion order.  On MP_OK, *ticket names
 * it and *out holds its result with the same lifetime as mp_dp_poll's. */
int mp_dp_wait_any(mp_dp_ctx *ctx, uint64_t *ticket, mp_result *out, int64_t timeout_us);

/* Serving counters since the context was created: requests completed,
 * micro-batches launched, and the latency of each completed request from
 * mp_dp_submit to the moment its result became available to mp_dp_poll
 * (p50 / p99 / max over all completed requests, or since the last call
 * with reset != 0). */
typedef struct {
    uint64_t completed;
    uint64_t batches;
    double mean_batch_pairs;
    double p50_ms, p99_ms, max_ms;
} mp_dp_serve_stats;

int mp_dp_get_serve_stats(mp_dp_ctx *ctx, mp_dp_serve_stats *s, int reset);

/* Drain the serving thread, free every device and host buffer. */
void mp_dp_destroy(mp_dp_ctx *ctx);

/* Allocation-free scoring of one pair (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory: services that fix their
 * device memory at start-up and must not allocate or free afterwards
 * (cudaMalloc and cudaFree can synchronize the device, and an allocation can
 * fail once other tenants hold the memory), and hosts that give plug-ins
 * device memory only from their own pools.  The call runs the
 * same DP as mp_dp_align_batch (packed int16, exact int32 re-run on
 * saturation), score only, for one pair, and allocates nothing: its scratch
 * is a fixed array of about 820 KB inside this library, held by every GPU
 * that loads the library until the process exits.
 *
 *   params  scoring parameters (NULL: defaults), validated as by mp_dp_init;
 *           wait_limit bounds the waits between cooperating warps as in
 *           the batch calls; max_pairs_per_launch, tb_budget_bytes, autotune
 *           and exon_rescore have no effect here
 *   d_prot  device pointer to prot_len ASCII residues, prot_len <= 4096
 *   d_nt    device pointer to nt_len ASCII nucleotides, nt_len <= 32768
 *   strand  +1, or -1 to align to the reverse complement of d_nt
 *   d_out   device pointer to 4 int32, written as {score, status (MP_ST_*),
 *           protein end, genome end}: the end cell of the best alignment as
 *           0-based exclusive ends; for strand -1 the genome value is the
 *           forward-strand start of the alignment (as nt_st of mp_result)
 *   stream  CUDA stream (cudaStream_t) to launch on; NULL = default stream
 *
 * Returns MP_ETOOLARGE beyond the size limits, MP_EINVAL for bad arguments
 * or parameters (local mode only), MP_ECUDA if a CUDA call fails; otherwise MP_OK once the
 * work is enqueued (the result is ready when the stream reaches it).
 * The first call on a device looks up the scratch address and sets a kernel
 * attribute (once per device, with that device current); make that first
 * call before any stream capture.  Every call shares the one scratch array,
 * which keeps the last call's contents (the kernel clears what must start
 * at zero); calls that overlap on the GPU (other streams, or other host
 * threads) race on it and must be serialized by the caller. */
int mp_dp_score_pair_noalloc(const mp_dp_params *params, const char *d_prot, uint32_t prot_len,
                             const char *d_nt, uint32_t nt_len, int8_t strand, int32_t *d_out,
                             void *stream);

/* ------------------------------------------------ seeding and chaining
 * The stage before the DP (Li 2022, Methods: "Reduced alphabet", "Indexing
 * the genome", "Chaining"), on the GPU.  The index holds, for both strands
 * of the genome as independent sequences and all three reading frames,
 * every 6-mer of the reduced amino-acid alphabet inside an open reading
 * frame (a maximal run of codons without a stop codon) of at least 30
 * amino acids whose hash (an invertible integer hash of its 24-bit code)
 * has lowest bit 0, as strand << 31 | floor(x / 256), x the k-mer's first
 * base on its strand.  A protein's 6-mers looked up there are its anchors
 * (strand, x = bin, y = residue); they are chained per strand by Eqs. 1-3
 * (binned gap, gap penalty with G = 200,000 bp and beta = 0.75, alpha =
 * min(dy, 6), f at least 6), in fixed point with 16 fractional bits (each
 * penalty term floored to a multiple of 2^-16).  Chains are taken in order
 * of decreasing score of their last anchor (ties: the earlier anchor in
 * (strand, x, y) order), each by following predecessors (the first of equal
 * best ones) until an anchor already taken, scored f(last) minus f of that
 * anchor; chains of one anchor are dropped. */
typedef struct mp_index mp_index;

typedef struct {
    int32_t strand;            /* 0: the genome as given; 1: its reverse complement */
    int32_t n_anchors;
    int64_t score;             /* chaining score in units of 2^-16 */
    int64_t x_first, x_last;   /* bins (256 bp) of the first and last anchor on the chain's strand */
    int64_t y_first, y_last;   /* residue positions of their 6-mers' first residues */
} mp_chain;

/* Build the index of a genome (host ASCII, len bases; letters other than
 * ACGT translate to no amino acid and break no reading frame's k-mers
 * other than their own codons' ones) on the context's device.  *out is
 * owned by the caller until mp_index_free.  MP_ENOMEM if the device cannot
 * hold it (about 2 bytes per base while building, 0.4 after). */
int mp_index_build(mp_dp_ctx *ctx, const char *genome, uint64_t len, mp_index **out);

/* Chain n_prot proteins (host ASCII; protein k at prot + prot_off[k],
 * prot_len[k] residues) against the index: chains (caller-owned, n_prot x
 * top) receives up to `top` chains per protein in extraction order,
 * n_chains[k] how many.  Blocking. */
int mp_index_chain(mp_dp_ctx *ctx, const mp_index *idx, const char *prot, const uint64_t *prot_off,
                   const uint32_t *prot_len, uint32_t n_prot, int32_t top, mp_chain *chains, uint32_t *n_chains);

/* Test hook: the index as CSR over all 2^24 hash values.  With offsets and
 * entries NULL only *n_entries is set; else offsets receives 2^24 + 1
 * values and entries *n_entries. */
int mp_index_download(mp_dp_ctx *ctx, const mp_index *idx, uint64_t *offsets, uint32_t *entries,
                      uint64_t *n_entries);

void mp_index_free(mp_index *idx);

/* Second round of chaining ("Chaining", last paragraph): around a chain of
 * the first round, every 5-mer of the protein is matched against every
 * 5-mer of the local genome region, without sampling or binning, and the
 * anchors are chained with the gap g' = 3 dy - dx (dx in bases) and the
 * penalty of Eq. 3, giving a chain at base resolution.
 *
 * Each pair is a (protein, region, strand) as for mp_dp_align_batch (flags
 * ignored): the region's aligned strand (its reverse complement for strand
 * -1) is read in all three frames, a 5-mer of the reduced alphabet starting
 * at every base with five full codons (stop codons and codons with a base
 * outside ACGT included, as codes 14 and 15); anchors (x, y) are the base x
 * of a 5-mer's first codon and the residue y of the equal protein 5-mer's
 * first residue.  Chaining as in mp_index_chain (x non-decreasing, y
 * increasing, alpha = min(dy, 5), G = 200,000, beta = 0.75, scores in units
 * of 2^-16, the first best predecessor, f >= 5).  out[k] receives pair k's
 * best chain: the anchor with the largest score (the earliest in (x, y)
 * order on ties) and its predecessors; n_anchors 0 if that is a single
 * anchor.  MP_EINVAL: a null argument, a protein longer than 8,192
 * residues, a region longer than about 134 Mb (with such a protein) or a
 * strand other than +1 / -1.  Device memory: the sequences,
 * plus 20 bytes per anchor in groups of at most about 200 M anchors. */
typedef struct {
    int32_t n_anchors;
    int32_t reserved;
    int64_t score;              /* f of the last anchor, units of 2^-16 */
    int64_t x_first, x_last;    /* 0-based base on the aligned strand */
    int64_t y_first, y_last;    /* 0-based residue */
} mp_chain2;
int mp_chain_refine(mp_dp_ctx *ctx, const mp_pair *pairs, size_t n, mp_chain2 *out);

/* Static string for a return code. */
const char *mp_dp_strerror(int code);

/* Pseudogene-aware rescoring (Methods, "Avoiding pseudogenes").  An
 * unspliced pseudogene of a spliced gene can outscore the gene because it
 * pays no intron costs.  For every result that carries a CIGAR, this runs
 * the local DP of the pair's protein against the alignment's coding region
 * with the introns cut out (codons, frameshift bases and the split codon of
 * a phase-1/2 intron kept, in the aligned orientation) and sets exon_score
 * to that score, less the intron cost r when the alignment has no intron.
 * Results without a CIGAR keep exon_score = score.  results must come from
 * aligning these pairs with this context (same order, CIGARs still valid);
 * the rescoring runs on the GPU as a score-only batch of its own and does
 * not disturb the CIGARs.  MP_ESTATE while the serving loop runs. */
int mp_dp_exon_rescore(mp_dp_ctx *ctx, const mp_pair *pairs, size_t n, mp_result *results);

/* Counters of the last mp_dp_batch_run / mp_dp_align_batch on the context.
 * Kernel times come from CUDA events recorded on the context's stream
 * around each kernel when timing is enabled with mp_dp_set_timing. */
typedef struct {
    double cells;              /* sum over pairs of |P| * |T| */
    double dp_ms;              /* packed int16 DP kernel(s) */
    double rerun_ms;           /* int32 re-run kernel(s) */
    double tb_ms;              /* traceback + compaction kernels */
    double pack_ms;            /* input packing kernel */
    double total_ms;           /* whole device pipeline */
    int32_t n_waves;
    int32_t n_rerun;           /* pairs re-run in int32 */
    int32_t n_launches;        /* kernels launched by the last run */
    int32_t n_dp_launches;     /* DP kernel launches (int16 + int32) */
    uint64_t code_bytes;       /* traceback stream written: H of every cell of every strip
                                  (padding of the last strip and chunk included) and the
                                  per-chunk column maxima */
    uint64_t record_bytes;     /* per-nt records written by the precompute kernel */
    uint64_t record_read_bytes;  /* records the strips queue into shared memory (every strip
                                    reads its pair's records; mostly L2 hits after the first) */
    uint64_t boundary_bytes;   /* boundary rows written between strips (each read once by
                                  the next strip) */
} mp_dp_stats;

/* Launch configuration of the DP.  The paper's DP is a SIMD loop on CPU
 * cores and has no counterpart; on the GPU the fastest configuration
 * depends on the batch (how many pairs, how uneven, how many need int32).
 * Every configuration computes bit-identical results: only the speed
 * differs. */
typedef struct {
    int32_t dp16_variant;      /* 0: int16 DP kernel built for 3 CTAs per SM (<= 80 registers per
                                  thread); 1: built for 2 CTAs per SM (<= 128 registers) */
    int32_t dp16_ctas_per_sm;  /* resident 8-warp CTAs per SM in the int16 launch; 0 = all that fit */
    int32_t dp32_ctas_per_sm;  /* the same for the int32 kernel */
    int32_t wide_direct;       /* 1: pairs whose score bound reaches the int16 limit skip the int16
                                  pass and run in int32 at once; 0: int16 first, int32 re-run only
                                  if the pair saturates */
    int32_t overlap_waves;     /* 1: a batch whose traceback exceeds the budget is planned in waves of
                                  half the budget that run alternately on two streams over two
                                  halves of the arena (one wave's tail overlaps the next wave);
                                  0: waves of the whole budget, one after the other */
    int32_t item_order;        /* 1: a wave's strip items interleaved so that strip s+1 of a pair is
                                  taken about two chunks after strip s; 0: pairs' strips back to
                                  back (a strip's warp first waits for its predecessor) */
    float ms;                  /* set by mp_dp_autotune: device time of one run of the batch */
    int32_t strip_width;       /* 0: every pair in strips of 64 residues (two per lane of a warp);
                                  1: int16 pairs in strips of 128 residues (four per lane: one
                                  shuffle, record load and profile load serve four cells) where that
                                  adds little padding (an even number of 64-residue strips, or 9 or
                                  more) and where the pair's longer critical path in that form stays
                                  within half the batch's longest one in 64-residue strips; 2: every
                                  such pair, whatever its critical path.  1 and 2 run the 2-CTA
                                  build whatever dp16_variant says */
} mp_dp_tuning;

/* Time the candidate configurations on an uploaded batch (warm-up runs;
 * one timed run per kernel configuration under the default plan, then one
 * per plan option under the fastest of those; a second timed run of the two
 * fastest overall; CUDA events on the context's stream; every run computes
 * the batch's full results, so the batch holds valid results afterwards)
 * and record the
 * fastest for the batch's shape class (pair count, mean cells per pair and
 * longest critical path on log2 scales, whether any pair needs int32,
 * whether the batch needs several waves).  Later runs of batches in that
 * class use it unless mp_dp_set_tuning fixed a configuration.  A candidate
 * with another plan (wave policy, item order) re-plans the batch first (host
 * work and small copies outside the timed interval).  best (may be NULL) receives the
 * choice; tried (may be NULL) up to max_tried candidates with their times,
 * and n_tried (may be NULL) how many were timed.  MP_EINVAL in the plain
 * form (max_pairs_per_launch > 0); MP_ESTATE while the serving loop runs. */
int mp_dp_autotune(mp_dp_ctx *ctx, mp_dp_batch *batch, mp_dp_tuning *best,
                   mp_dp_tuning *tried, int max_tried, int *n_tried);
/* Fix the configuration of every later run on the context (NULL: back to
 * the tuned table and the defaults).  MP_EINVAL for values out of range;
 * CTAs per SM above what fits are clamped at launch. */
int mp_dp_set_tuning(mp_dp_ctx *ctx, const mp_dp_tuning *t);
/* The configuration that a run of batch would use now. */
int mp_dp_get_tuning(mp_dp_ctx *ctx, const mp_dp_batch *batch, mp_dp_tuning *t);
/* Write / read the tuned table as text: a header naming the device and its
 * SM count, then one line per shape class.  Load merges the entries and
 * rejects a table made on another kind of device; a file that cannot be
 * opened, written or parsed is MP_EINVAL as well. */
int mp_dp_tuning_save(mp_dp_ctx *ctx, const char *path);
int mp_dp_tuning_load(mp_dp_ctx *ctx, const char *path);

int mp_dp_set_timing(mp_dp_ctx *ctx, int enable);
int mp_dp_get_stats(mp_dp_ctx *ctx, mp_dp_stats *s);

/* Number of streaming multiprocessors of the context's device. */
int mp_dp_num_sms(mp_dp_ctx *ctx);

/* Measured integer ceilings behind the DP kernel's roofline (no
 * counterpart in the method: Eq. 7 is a max-plus scan on the integer ALU).
 * Rates are counted in SM clocks, every warp slot occupied:
 *   - max_u16x2 .. imad: warp instructions per clock per SM of one packed
 *     16-bit operation alone (max, fused add-max, three-way max, byte
 *     permute, three-input logic, integer multiply-add), eight independent
 *     chains per thread, one plain add per eight operations;
 *   - step_cells_per_clk_sm: cells per clock per SM of the int16 step's
 *     arithmetic alone (the eleven fused add-max terms of Eq. 7, the
 *     three-way maxima, the [H, I] hand-over by shuffle and byte permute,
 *     the chunk maximum) on register state, warps_per_sm_step warps per SM.
 * The call allocates a few MB on `device` and runs for well under a second;
 * it needs no context.  MP_EINVAL: null out or no such device; MP_ENOMEM,
 * MP_ECUDA as usual. */
typedef struct {
    double max_u16x2, viaddmax_u16x2, vimax3_u16x2, prmt, lop3, imad;
    double step_cells_per_clk_sm;
    int32_t warps_per_sm_step;
    int32_t reserved;
} mp_op_rates;
int mp_dp_op_rates(int device, mp_op_rates *out);

/* Test hook (no counterpart in the method): the H values of Eq. 7 the DP
 * stored for pair k of `batch`, read back through the traceback's view of
 * the stream.  h (host, caller-owned) receives (|T|+1) x (|P|+1) int32,
 * row-major, H[i][j] at i*(|P|+1)+j, in the aligned orientation (the
 * reverse complement for strand -1); row 0 and column 0 hold the boundary
 * of the context's mode.  Valid after mp_dp_batch_run + mp_dp_batch_sync of
 * `batch` as the context's last run, in one wave (a batch within the
 * traceback budget).  MP_EINVAL: null argument, k out of range, or a pair
 * with no stored stream (score-only, empty, over budget); MP_ESTATE: another
 * run since, or a batch run in several waves; MP_ENOMEM: the cell buffer
 * could not be allocated (this hook allocates device memory per call). */
int mp_dp_debug_h(mp_dp_ctx *ctx, mp_dp_batch *batch, size_t k, int32_t *h);

#ifdef __cplusplus
}
#endif
#endif /* MP_DP_H */

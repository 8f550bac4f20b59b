// Internal device-side definitions shared by the kernels and the runtime.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mp_dp.h"

namespace mpdp {

// ---- geometry -----------------------------------------------------------
constexpr int kStripW = 64;     // residues per strip: two per lane
constexpr int kStripWMax = 128; // the wide int16 form: 128-residue strips, four residues per lane
constexpr int kChunk = 96;      // DP steps per chunk (record / boundary staging)
constexpr int kBody = 12;       // steps per unrolled body (multiple of 3 and 4)
constexpr int kRing = 256;      // per-nt record ring entries
constexpr int kRingPad = 12;    // mirrored entries so a body never wraps
constexpr int kProfRows = 22;   // translated amino acid 0..19, stop 20, no codon 21
constexpr int kBndPad = kStripWMax;   // boundary entries before genome position 0
constexpr int kRecPre = 2 * kChunk;   // per-nt records before genome position 0
constexpr int kWarpsPerCta = 8; // persistent DP kernel
constexpr int kNtPadWords = 16; // zero words around each packed genome

// bytes of the traceback stream per strip step in the int16 path: 64 cells * 2 B
// (the int32 path stores 4 B per cell)
constexpr int kStepBytes = kStripW * 2;

// int16 path: scores at or above this re-run in int32 (intermediates stay
// below 32767 while every H is below it; see the design notes)
constexpr int kOverflowT = 32000;


// ---- per-pair device descriptors -------------------------------------------
struct PairDesc {
    uint64_t code_off;      // byte offset of strip 0 in the wave's code arena
    uint64_t bnd_off;       // entry offset of this pair's boundary buffer
    uint32_t prot_off;      // offset into the residue-code array
    uint32_t nt_word_off;   // word offset of genome base 0 in the packed array
    uint32_t prot_len;
    uint32_t nt_len;
    uint32_t asc_prot_off;  // offsets into the uploaded ASCII
    uint64_t asc_nt_off;
    uint32_t cig_cap;       // capacity of this pair's reversed-op slot
    uint64_t cig_off;       // offset of that slot
    uint32_t flags;         // PF_*
    int32_t strand;
    uint32_t strip_base;    // index of strip 0 in the per-strip progress array
    uint32_t n_strips;
    uint64_t rec_off;       // index of the record of genome position -kRecPre in the record array
    uint64_t col0_off;      // anchored modes: index of H[0][0] in the column-0 array (H[i][0] at +i)
    uint64_t prof_off;      // PF_PROF: index of the pair's position 0 in the profile arrays
};

// per-nt records of a pair: positions -kRecPre .. kChunk*(nchunks+1) - 1
// (nchunks of the widest strip form)
__host__ __device__ constexpr uint64_t records_of(uint32_t n)
{
    return ((static_cast<uint64_t>(n) + kStripWMax - 1 + kChunk - 1) / kChunk + 1) * kChunk + kRecPre;
}

// internal PairOut.status bit (never returned to callers): the pair's
// traceback stream was written by the int32 kernel (4 bytes per cell)
constexpr int32_t kStInt32Stream = 0x100;
// internal PairOut.status bit: the pair was traced by the DP kernel right
// after its last strip (the traceback kernel skips it)
constexpr int32_t kStTraced = 0x200;

// PF_WIDE: the pair's score could exceed the int16 range, so its traceback
// region is sized for the int32 re-run (4 bytes per cell)
// PF_W128: the pair runs in 128-residue strips (four residues per lane; int16
// only, never with PF_WIDE); otherwise in 64-residue strips
// PF_PROF: the pair is a profile query (position-specific costs at prof_off)
enum : uint32_t {
    PF_SCORE_ONLY = 1u, PF_BADSEQ = 2u, PF_SKIP = 4u, PF_BUDGET = 8u, PF_WIDE = 16u, PF_W128 = 32u, PF_PROF = 64u
};

// Device copy of mp_profile_pos: position-specific substitution scores
// (translated code 0..19, 20 = stop) and gap costs of one column.
struct ProfPos {
    int16_t s[21];
    int16_t q, e, pad;
};
static_assert(sizeof(ProfPos) == 48, "ProfPos mirrors mp_profile_pos");

// strip width of a pair
__host__ __device__ constexpr int strip_w_of(uint32_t flags) { return (flags & PF_W128) ? kStripWMax : kStripW; }

struct PairOut {
    int32_t score;
    int32_t status;         // MP_ST_* bits
    int32_t best_ii, best_jj;  // 0-based cell of the best H (aligned orientation)
    int32_t st_ii, st_jj;      // first cell after the restart (aligned orientation)
    uint32_t n_ops;         // reversed ops written by the traceback
    uint32_t cig_out;       // offset in the compacted CIGAR array
};

struct ScoreParams {
    int32_t q, e, f, r, stop;
    int8_t mat[22][22];
    int32_t splice_model;   // MP_SPLICE_FINAL / MP_SPLICE_SIMPLE
    int32_t splice_p;       // simple model: cost of a donor without GT / acceptor without AG
    int32_t mode;           // MP_MODE_LOCAL / MP_MODE_GLOBAL / MP_MODE_EXTEND
};

// anchored modes: entries of the column-0 array beyond row |T| (the DP's
// boundary loads run up to a strip width + 2 chunks past the last row)
constexpr int kCol0Pad = kStripWMax + 2 * kChunk + 2;

// A work item is one strip (64 or 128 residues) of one pair: x = pair, y = strip.
// The warp running strip s consumes the boundary row strip s-1 publishes
// chunk by chunk.
struct DPArgs {
    const PairDesc *pairs;
    const uint4 *recs;      // per-nt records (see make_record)
    const uint2 *items;     // processing order (strip s+1 of a pair some items after strip s)
    uint32_t n_items;
    uint32_t *head;         // work-queue counter
    const uint8_t *prot;    // residue codes
    const uint32_t *nt2;    // packed genome (base k at bits 2(k%16) of word k/16)
    uint8_t *codes;         // traceback code arena
    void *bnd;              // boundary arena
    const int32_t *col0;    // anchored modes: column 0 of every pair (H[i][0]); null in local mode
    PairOut *out;
    uint32_t *progress;     // per strip: chunks whose boundary row is published
    unsigned long long *best_key;   // per pair: max of (score, -ii, -jj)
    uint32_t *strips_done;  // per pair
    uint2 *rerun_items;     // strips of pairs whose int16 run saturated
    uint32_t *rerun_count;
    ScoreParams sp;
    uint32_t spin_limit;    // polls before a wait gives up (0: kSpinLimit)
    uint32_t no_publish;    // test hook: withhold boundary rows
    uint32_t *ops;          // reversed-op slots, for the traceback of a pair right after its last strip
    const int8_t *mat;      // the substitution matrix (22 x 22) in device memory; null: no such traceback
    const ProfPos *prof;    // profile positions of PF_PROF pairs (at PairDesc::prof_off)
    const int32_t *epre;    // per profile position j: the sum of gap_ext over positions 1..j
};

// bounded wait of a consumer strip for its producer (iterations of ~0.25 us)
constexpr uint32_t kSpinLimit = 40u * 1000u * 1000u;

struct TBArgs {
    const PairDesc *pairs;
    const uint32_t *work;
    uint32_t n_work;
    const uint8_t *codes;   // traceback stream (H of every cell)
    const uint8_t *prot;    // residue codes
    const uint32_t *nt2;    // packed genome
    PairOut *out;
    uint32_t *ops;          // reversed-op slots
    const int32_t *col0;    // anchored modes: column 0 of every pair (H[i][0])
    ScoreParams sp;
    const ProfPos *prof;    // profile positions of PF_PROF pairs
    const int32_t *epre;    // their gap-extension prefix sums
};

// kernel launchers (defined in the .cu files)
cudaError_t launch_pack(const PairDesc *pairs, uint32_t n, const char *ascii, uint8_t *prot,
                        uint32_t *nt2, PairOut *out, cudaStream_t st);
cudaError_t launch_records(const PairDesc *pairs, uint32_t n, const uint32_t *nt2, const ScoreParams &sp, uint4 *recs,
                           cudaStream_t st);
// variant 0: the int16 DP kernel built for 3 CTAs per SM (80 registers per
// thread); 1: built for 2 CTAs per SM (up to 128).  wide4: the 2-CTA build
// that also runs PF_W128 pairs in 128-residue strips.  Same results.
constexpr int kDp16Variants = 2;
cudaError_t launch_dp16(const DPArgs &a, int grid, int variant, bool wide4, cudaStream_t st);
cudaError_t launch_dp32(const DPArgs &a, int grid, bool rerun_only, cudaStream_t st);
cudaError_t launch_tb(const TBArgs &a, int grid, cudaStream_t st);
cudaError_t launch_dump_h(const TBArgs &a, uint32_t p, size_t cells, int32_t *h, cudaStream_t st);

// One pair of a pseudogene-rescoring batch: where its protein and region
// sit in the source ASCII (as the caller passed them), and its alignment's
// ops (protein order) and start in the aligned orientation.  The gather
// writes the protein and the alignment's intron-free coding region into the
// rescoring batch's ASCII at the offsets of that batch's descriptor.
struct ExonJob {
    uint64_t src_nt_off;
    uint64_t op_off;
    uint32_t src_prot_off;
    uint32_t src_nt_len;
    uint32_t n_ops;
    int32_t strand;
    int32_t i0;
    uint32_t pad;
};
cudaError_t launch_exon_gather(const ExonJob *jobs, uint32_t n, const PairDesc *aux, const char *src,
                               const uint32_t *ops, char *dst, cudaStream_t st);
// anchored modes: column 0 of every pair, H[i][0] for i = 0..|T| (then
// padding), by the recurrence restricted to the D, G and A terms
cudaError_t launch_col0(const PairDesc *pairs, uint32_t n, const uint32_t *nt2, const ScoreParams &sp,
                        const ProfPos *prof, int32_t *col0, cudaStream_t st);
cudaError_t launch_compact(const PairDesc *pairs, PairOut *out, uint32_t n, const uint32_t *ops,
                           uint32_t *cig, uint32_t *total, cudaStream_t st);
int dp16_blocks_per_sm(int variant, bool wide4 = false);

// the device and stream of a context (for the seeding and chaining calls)
int ctx_device(const mp_dp_ctx *c);
cudaStream_t ctx_stream(const mp_dp_ctx *c);
int dp32_blocks_per_sm();
size_t dp16_smem_bytes();
size_t dp32_smem_bytes();

}  // namespace mpdp

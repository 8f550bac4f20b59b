// Spliced protein-to-genome DP, Li 2022 Eq. 7 (Methods, "DP for
// protein-to-genome alignment"), local mode, with the final splice model
// (Methods, "Splice models").  Hand-written for sm_103a.
//
// Layout of the computation
// -------------------------
// One warp owns one (protein, region) pair.  The protein is cut into strips
// of 64 residues; lane l holds residues 2l ("lo") and 2l+1 ("hi") of the
// strip.  The warp sweeps anti-diagonals: at step t the lo cell of lane l is
// genome position ii = t - 2l and the hi cell is ii - 1, so every cell
// depends only on cells of earlier steps:
//   - the residue to the left (j-1) comes from lane l-1's hi cell of the
//     previous step (one __shfl_up_sync of a packed [H, I] word), or, for
//     the hi cell, from the lane's own lo cell of the previous step;
//   - genome-direction terms (i-1, i-2, i-3) come from the lane's own
//     register history.
// Strip s+1 reads the last residue of strip s from a per-pair boundary
// buffer ([H, I] per genome position).
//
// Arithmetic
// ----------
// The int16 path keeps each state as two biased 16-bit lanes in one 32-bit
// register (value v stored as v + 32768).  Every penalised term of Eq. 7 is
// one fused per-halfword add-max (the penalty held negated per half, the
// addition modulo 2^16, exact because no biased operand leaves 0..65535);
// the remaining maxima use three- and two-way max.u16x2; the few plain
// 32-bit adds (the gap extension, the two profile halves) never carry
// across halves.  A pair whose best score reaches 32000 is re-run in the
// int32 instantiation of the same kernel.
//
// Traceback stream
// ----------------
// The kernel stores the H value of every cell (2 bytes in the int16 path,
// 4 bytes in the int32 re-run): the 32-bit H register of a lane already
// holds its two cells, so the stream costs one 16-byte store per lane every
// 4 steps and no arithmetic.  The traceback kernel re-derives each decision
// of Eq. 7 from these values (the gap and intron states in closed form),
// with the same tie order.
#include <atomic>
#include <mutex>

#include "mp_device.cuh"
#include "mp_internal.cuh"
#include "traceback.cuh"

namespace mpdp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- helpers
template <uint32_t S>
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "n"(S));
    return r;
}

__device__ __forceinline__ uint32_t vmax(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// per 16-bit half: max(a + b, c), the addition modulo 2^16 (so adding a
// negated penalty subtracts it: the biased operands never leave 0..65535)
__device__ __forceinline__ uint32_t vaddmax(uint32_t a, uint32_t b, uint32_t c) { return __viaddmax_u16x2(a, b, c); }

// per 16-bit half: max(a, b, c)
__device__ __forceinline__ uint32_t vmax3(uint32_t a, uint32_t b, uint32_t c) { return __vimax3_u16x2(a, b, c); }

// a packed pair of penalties negated per half (modulo 2^16)
__host__ __device__ __forceinline__ uint32_t neg2(uint32_t lo, uint32_t hi)
{
    return ((0x10000u - lo) & 0xffffu) | (((0x10000u - hi) & 0xffffu) << 16);
}

// Per-genome-position record for the lo cell at 0-based position ii
// (1-based i = ii + 1), the penalties negated per 16-bit half (modulo 2^16,
// so that one fused add-max subtracts them):
//   x = [-(r + d(i+1)), -(r + d(i))]   (16-bit halves, lo first)
//   y = [-a(i), -a(i-1)]
//   z = byte offset of the profile row of the codon ending at i
__device__ __forceinline__ uint4 make_record(const uint32_t *g, int n, int ii, const ScoreParams &sp)
{
    const int s = ii - 3;                  // window T0[ii-3 .. ii+4]
    const int w = s >> 4;                  // floor division (s may be negative)
    const int sh = (s & 15) * 2;
    const uint64_t pair64 = (static_cast<uint64_t>(g[w + 1]) << 32) | g[w];
    const uint32_t win = static_cast<uint32_t>(pair64 >> sh);
    int b[8];
    bool v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        b[k] = (win >> (2 * k)) & 3;
        v[k] = static_cast<unsigned>(s + k) < static_cast<unsigned>(n);
    }
    const int aa = (v[1] && v[3]) ? c_code.v[b[1] * 16 + b[2] * 4 + b[3]] : 21;
    const int r = sp.r;
    const int dC = splice_donor(sp, b[5], b[6], b[7], v[5], v[6], v[7]);     // d(i+1)
    const int dB = splice_donor(sp, b[4], b[5], b[6], v[4], v[5], v[6]);     // d(i)
    const int aA = splice_acceptor(sp, b[1], b[2], b[3], v[1], v[2], v[3]);  // a(i)
    const int aC = splice_acceptor(sp, b[0], b[1], b[2], v[0], v[1], v[2]);  // a(i-1)
    uint4 rec;
    rec.x = neg2(static_cast<uint32_t>(r + dC), static_cast<uint32_t>(r + dB));
    rec.y = neg2(static_cast<uint32_t>(aA), static_cast<uint32_t>(aC));
    rec.z = static_cast<uint32_t>(aa) * 128u;
    rec.w = 0;
    return rec;
}

// --------------------------------------------------------------- smem
template <typename BndT>
struct WarpSmem {
    // per-nt records, even and odd positions in separate halves: at a given
    // step all lanes read records of one parity at consecutive indices, so the
    // 16-byte loads are free of bank conflicts
    uint4 ring[2][kRing / 2 + kRingPad / 2];
    // substitution profile of the strip, as two tables: prof[aa][lane] holds
    // s(aa, P[2l]) in its low half (high half 0) and prof[kProfRows + aa][lane]
    // s(aa, P[2l+1]) in its high half (low half 0), so that one addition of
    // this step's low word and the previous step's high word packs the two
    // cells' scores (the hi cell is a row behind the lo cell)
    uint32_t prof[2 * kProfRows * 32];
    alignas(16) BndT bin[kChunk];
    alignas(16) BndT bout[kChunk];
};

template <typename BndT>
__device__ __forceinline__ void put_record(WarpSmem<BndT> &sm, int ii, const uint4 &rec)
{
    const int half = ii & 1, idx = (ii >> 1) & (kRing / 2 - 1);
    sm.ring[half][idx] = rec;
    if (idx < kRingPad / 2) sm.ring[half][idx + kRing / 2] = rec;   // mirror: a body never wraps
}

template <typename BndT>
__device__ __forceinline__ uint4 get_record(const WarpSmem<BndT> &sm, int ii)
{
    return sm.ring[ii & 1][(ii >> 1) & (kRing / 2 - 1)];
}

// 16-byte asynchronous copy global -> shared (no register staging)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// queue the records of positions [lo, lo + kChunk) into the ring
// (recs[ii + kRecPre] is the record of position ii)
template <typename BndT>
__device__ __forceinline__ void fetch_records(WarpSmem<BndT> &sm, const uint4 *recs, int lo, int lane)
{
    for (int ii = lo + lane; ii < lo + kChunk; ii += 32) {
        const int half = ii & 1, idx = (ii >> 1) & (kRing / 2 - 1);
        cp_async16(&sm.ring[half][idx], recs + ii + kRecPre);
        if (idx < kRingPad / 2) cp_async16(&sm.ring[half][idx + kRing / 2], recs + ii + kRecPre);
    }
}

// Shared memory of a warp running a 128-residue strip (four residues per
// lane).  At a step lane l reads the record of position t - 4l: the ring is
// split by position mod 4, so all lanes read one quarter at consecutive
// indices (conflict-free 16-byte loads).  Each quarter holds kRing4 entries
// (a chunk reads positions t0-124 .. t0+95 while the next chunk's 96 arrive)
// plus kRing4Pad mirrored ones so that a 12-step body never wraps.
constexpr int kRing4 = 96;
constexpr int kRing4Pad = 2;
struct WarpSmem4 {
    uint4 ring[4][kRing4 + kRing4Pad];
    // prof[aa][lane] = {[s(aa, P[4l]), s(aa, P[4l+1])], [s(aa, P[4l+2]), s(aa, P[4l+3])]}, each + 512
    uint2 prof[kProfRows * 32];
    alignas(16) uint32_t bin[kChunk];
    alignas(16) uint32_t bout[kChunk];
};

// quarter index of position ii (ii >= -8 * kRing4)
__device__ __forceinline__ int ring4_idx(int ii) { return ((ii + 8 * kRing4) >> 2) % kRing4; }

__device__ __forceinline__ uint4 get_record4(const WarpSmem4 &sm, int ii) { return sm.ring[ii & 3][ring4_idx(ii)]; }

__device__ __forceinline__ void fetch_records4(WarpSmem4 &sm, const uint4 *recs, int lo, int lane)
{
    for (int ii = lo + lane; ii < lo + kChunk; ii += 32) {
        const int q = ii & 3, idx = ring4_idx(ii);
        cp_async16(&sm.ring[q][idx], recs + ii + kRecPre);
        if (idx < kRing4Pad) cp_async16(&sm.ring[q][idx + kRing4], recs + ii + kRecPre);
    }
}

// ================================================================ int16 ops
struct Ops16 {
    using Bnd = uint32_t;                  // [H, I] biased 16-bit
    using Smem = WarpSmem<Bnd>;
    static constexpr int W = kStripW, CPL = 2;
    static constexpr uint32_t Z = 0x80008000u;      // biased 0 in both halves
    static constexpr uint32_t NEGV = 0x40004000u;   // biased -16384
    static constexpr Bnd kBnd0 = 0x40008000u;       // column 0: H = 0, I = -inf

    struct Consts {
        uint32_t NQE, E, NF;               // packed -(q+e) (negated per half), e, -f
        uint32_t EN;                       // e of the columns the lane's I values move to:
                                           // [e(2l+1), e(2l+2)] (the same as E unless a profile)
        uint32_t FLOOR;                    // local: biased 0 (the restart); anchored modes: 0 (none)
        uint32_t ROW0;                     // H in row 0 of the lane's two columns (biased)
    };
    struct State {
        uint32_t H1, H2, H3, L0, L1, L2, L3, IL, D1, D2, D3, A1, B1, C1;
        uint32_t VD1, VD2, VA1, VA2, X1;
        uint32_t TC, bklo, bkhi;            // best-cell keys (pairs without a stored stream)
        uint32_t cm;                        // this chunk's packed maximum H (pairs with a stream)
    };

    static __device__ __forceinline__ Consts consts(const ScoreParams &sp)
    {
        Consts c;
        const uint32_t qe = sp.q + sp.e;
        c.NQE = neg2(qe, qe);
        c.E = static_cast<uint32_t>(sp.e) | (static_cast<uint32_t>(sp.e) << 16);
        c.NF = neg2(static_cast<uint32_t>(sp.f), static_cast<uint32_t>(sp.f));
        c.EN = c.E;
        c.FLOOR = sp.mode == MP_MODE_LOCAL ? Z : 0u;
        c.ROW0 = Z;
        return c;
    }

    // biased pair [lo, hi] of H values (clamped to the int16 range)
    static __device__ __forceinline__ uint32_t pack2(int lo, int hi)
    {
        lo = min(max(lo, -32768), 32767);
        hi = min(max(hi, -32768), 32767);
        return static_cast<uint32_t>(lo + 32768) | (static_cast<uint32_t>(hi + 32768) << 16);
    }
    static __device__ __forceinline__ void set_row0(Consts &c, int lo, int hi) { c.ROW0 = pack2(lo, hi); }
    // profile queries: the gap costs of the lane's two columns (packed halves)
    // enext: e of the column right of the lane's hi column
    static __device__ __forceinline__ void set_gaps(Consts &c, int qlo, int elo, int qhi, int ehi, int enext)
    {
        c.NQE = neg2(static_cast<uint32_t>(qlo + elo), static_cast<uint32_t>(qhi + ehi));
        c.E = static_cast<uint32_t>(elo) | (static_cast<uint32_t>(ehi) << 16);
        c.EN = static_cast<uint32_t>(ehi) | (static_cast<uint32_t>(enext) << 16);
    }
    // boundary entry of column 0 in the anchored modes: [H, I = -inf]
    static __device__ __forceinline__ Bnd col0_entry(int h)
    {
        h = max(h, -16384);
        return static_cast<uint32_t>(h + 32768) | 0x40000000u;
    }

    // a profile entry: the two scores as 16-bit two's complement halves (added
    // modulo 2^16 to a biased H)
    static __device__ __forceinline__ uint32_t prof_entry(int slo, int shi)
    {
        return (static_cast<uint32_t>(slo) & 0xffffu) | ((static_cast<uint32_t>(shi) & 0xffffu) << 16);
    }

    // State before step 0, i.e. the history of steps -1 .. -4.  At step tau
    // lane l holds rows ii = tau - 2l (lo), tau - 2l - 1 (hi) and sees its
    // left column at ii = tau - 2l + 1, so only lane 0 touches the matrix
    // there: its lo column in row 0 at step -1 (H1.lo, L0.hi = h_self), its
    // left column at ii = 0 at step -1 (L0.lo, the boundary entry w0) and in
    // row 0 at step -2 (L1.lo = h_left).  Every other slot is outside (-inf).
    // h_self, h_left: H in row 0 of the lane's lo column and of the column to
    // its left (0 in local mode)
    static __device__ __forceinline__ void init(State &s, int lane, Bnd w0, uint4 recm1, uint4 recm2,
                                                uint32_t xm1, int h_self, int h_left)
    {
        const uint32_t hs = pack2(h_self, -16384), hl = pack2(h_left, -16384);   // [H, -inf]
        s.H1 = (lane == 0) ? hs : NEGV; s.H2 = NEGV; s.H3 = NEGV;
        s.L1 = (lane == 0) ? hl : NEGV; s.L2 = NEGV; s.L3 = NEGV;
        s.L0 = (lane == 0) ? ((w0 & 0xffffu) | (hs << 16)) : NEGV;
        s.IL = (lane == 0) ? ((w0 >> 16) | 0x40000000u) : NEGV;
        s.D1 = s.D2 = s.D3 = NEGV;
        s.A1 = s.B1 = s.C1 = NEGV;
        s.VD1 = recm1.x; s.VD2 = recm2.x;
        s.VA1 = recm1.y; s.VA2 = recm2.y;
        s.X1 = xm1;
        s.TC = 0xffffu; s.bklo = 0; s.bkhi = 0; s.cm = 0;
    }

    using Word = uint32_t;                  // traceback word of one lane and step: [H lo, H hi]

    // One anti-diagonal step.  Returns the lane's two H values (biased).
    // KEYS: track the best cell's step with keys (needed when no stream is
    // stored); otherwise keep only the chunk's maximum, whose first position
    // is later read back from the stream.
    template <bool MASKED, bool KEYS>
    static __device__ __forceinline__ uint32_t step(State &s, const Consts &c, const uint4 rec,
                                                    const uint32_t *prof_lane, Bnd bin, Bnd &wout,
                                                    int lane, int ii, int n)
    {
        const uint32_t VD0 = rec.x, VA0 = rec.y;          // negated penalties
        const uint32_t X0 = *reinterpret_cast<const uint32_t *>(
            reinterpret_cast<const char *>(prof_lane) + rec.z);
        const uint32_t X0h = *reinterpret_cast<const uint32_t *>(
            reinterpret_cast<const char *>(prof_lane + kProfRows * 32) + rec.z);
        const uint32_t S = X0 + s.X1;                     // lo: s(i, 2l); hi: s(i-1, 2l+1)
        // each term of Eq. 7 that subtracts a penalty is one fused add-max;
        // IL holds I[i][j-1] - e (the sender subtracted the extension)
        uint32_t I0 = vaddmax(s.L0, c.NQE, s.IL);         // max(H[i][j-1] - q - e, I[i][j-1] - e)
        uint32_t D0 = vaddmax(s.H3, c.NQE, s.D3 - c.E);    // max(H[i-3][j] - q - e, D[i-3][j] - e)
        uint32_t A0 = vaddmax(s.H1, s.VD2, s.A1);         // max(H[i-1][j] - r - d(i-1), A[i-1][j])
        uint32_t B0 = vaddmax(s.L1, s.VD1, s.B1);         // max(H[i-1][j-1] - r - d(i), B[i-1][j])
        uint32_t C0 = vaddmax(s.L1, VD0, s.C1);           // max(H[i-1][j-1] - r - d(i+1), C[i-1][j])
        // H: the intron exits and the frameshift terms in one chain, the terms
        // known a step early (the B and C exits) first and those of the
        // previous step's H last; the match and D in another; I, which
        // depends on this step's neighbour, joins in the last max
        uint32_t Y = vaddmax(C0, s.VA1, c.FLOOR);         // C - a(i-1)
        Y = vaddmax(B0, s.VA2, Y);                        // B - a(i-2)
        // the four frameshift terms H[i-1][j-1], H[i-2][j-1], H[i-2][j], H[i-1][j], less f
        Y = vaddmax(vmax(vmax3(s.L1, s.L2, s.H2), s.H1), c.NF, Y);
        Y = vaddmax(A0, VA0, Y);                          // A - a(i)
        uint32_t H0 = vmax3(vaddmax(s.L3, S, D0), I0, Y); // H[i-3][j-1] + s(i, j), D, I

        uint32_t vmask = 0xffffffffu;
        if (MASKED) {
            // cells before row 1 are outside the matrix; ii = -1 is row 0
            const uint32_t kill = (ii < 0 ? 0x0000ffffu : 0u) | (ii < 1 ? 0xffff0000u : 0u);
            const uint32_t row0 = (ii == -1 ? 0x0000ffffu : 0u) | (ii == 0 ? 0xffff0000u : 0u);
            const uint32_t hforce = (row0 & c.ROW0) | (~row0 & NEGV);
            H0 = (H0 & ~kill) | (hforce & kill);
            I0 = (I0 & ~kill) | (NEGV & kill);
            D0 = (D0 & ~kill) | (NEGV & kill);
            A0 = (A0 & ~kill) | (NEGV & kill);
            B0 = (B0 & ~kill) | (NEGV & kill);
            C0 = (C0 & ~kill) | (NEGV & kill);
            vmask = ((ii >= 0 && ii < n) ? 0x0000ffffu : 0u) | ((ii >= 1 && ii <= n) ? 0xffff0000u : 0u);
        }

        // hand [H, I - e] of the hi cell to the next lane (the receiving
        // column's extension, subtracted here, off the step's chain); lane 0
        // takes the strip boundary, which holds the same form
        const uint32_t I0mE = I0 - c.EN;
        const uint32_t W = prmt<0x7632>(H0, I0mE);
        uint32_t R = __shfl_up_sync(kFull, W, 1);
        if (lane == 0) R = bin;
        wout = W;
        s.L3 = s.L2; s.L2 = s.L1; s.L1 = s.L0;
        s.L0 = prmt<0x5410>(R, H0);
        s.IL = prmt<0x5432>(R, I0mE);
        s.H3 = s.H2; s.H2 = s.H1; s.H1 = H0;
        s.D3 = s.D2; s.D2 = s.D1; s.D1 = D0;
        s.A1 = A0; s.B1 = B0; s.C1 = C0;
        s.VD2 = s.VD1; s.VD1 = VD0;
        s.VA2 = s.VA1; s.VA1 = VA0;
        s.X1 = X0h;

        // best cell: key = H << 16 | (0xffff - step within chunk); the
        // largest key is the largest H at its first step
        const uint32_t Hm = H0 & vmask;
        if (KEYS) {
            s.bklo = max(s.bklo, Hm * 65536u + s.TC);             // [TC, H.lo]
            s.bkhi = max(s.bkhi, (Hm & 0xffff0000u) | s.TC);     // [TC, H.hi]
            s.TC -= 1;
        } else {
            s.cm = vmax(s.cm, Hm);
        }
        return H0;
    }

    // four steps of one lane: one 16-byte store
    static __device__ __forceinline__ void store4(uint8_t *strip, int t, int lane, const Word *w)
    {
        *reinterpret_cast<uint4 *>(strip + static_cast<size_t>(t) * kStepBytes + lane * 16) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }

    // Extract (score, step) of one half's best key; score < 0 if none.
    static __device__ __forceinline__ void take_best(const State &s, int half, int t0, int &score, int &t)
    {
        const uint32_t k = half ? s.bkhi : s.bklo;
        score = static_cast<int>(k >> 16) - 32768;
        t = t0 + static_cast<int>(0xffffu - (k & 0xffffu));
    }
    static __device__ __forceinline__ void reset_best(State &s)
    {
        s.TC = 0xffffu; s.bklo = 0; s.bkhi = 0; s.cm = 0;
    }

    // this chunk's maximum H of the lane's two cells (biased; 0 if none)
    using ColMax = uint32_t;
    static __device__ __forceinline__ ColMax chunk_max(const State &s) { return s.cm; }
    static constexpr bool kChunkMaxBest = true;   // with a stream, the best cell comes from chunk maxima
    // unbiased H of half h of a stored stream word
    static __device__ __forceinline__ int word_h(const Word &w, int h)
    {
        return static_cast<int>(h ? (w >> 16) : (w & 0xffffu)) - 32768;
    }
    static __device__ __forceinline__ Word load_word(const uint8_t *strip, int t, int lane)
    {
        return *reinterpret_cast<const uint32_t *>(strip + static_cast<size_t>(t >> 2) * 512 + lane * 16 +
                                                   (t & 3) * 4);
    }
    static __device__ __forceinline__ int cell_max(const ColMax &m, int k) { return word_h(m, k); }
    // stored H of cell k of the lane at step t
    static __device__ __forceinline__ int load_cell(const uint8_t *strip, int t, int lane, int k)
    {
        return word_h(load_word(strip, t, lane), k);
    }
};

// ================================================================ int32 ops
struct V2 {
    int32_t lo, hi;
};

__device__ __forceinline__ V2 mx(V2 a, V2 b) { return V2{max(a.lo, b.lo), max(a.hi, b.hi)}; }
__device__ __forceinline__ V2 sub(V2 a, V2 b) { return V2{a.lo - b.lo, a.hi - b.hi}; }
__device__ __forceinline__ V2 subc(V2 a, int32_t b) { return V2{a.lo - b, a.hi - b}; }
__device__ __forceinline__ V2 add(V2 a, V2 b) { return V2{a.lo + b.lo, a.hi + b.hi}; }
// the two negated penalties of a record word, sign-extended
__device__ __forceinline__ V2 unpack_neg16(uint32_t w)
{
    return V2{static_cast<int32_t>(w << 16) >> 16, static_cast<int32_t>(w) >> 16};
}

struct Ops32 {
    struct Bnd {
        int32_t h, i;
    };
    using Smem = WarpSmem<Bnd>;
    static constexpr int W = kStripW, CPL = 2;
    static constexpr int32_t NEG = -(1 << 28);
    static constexpr Bnd kBnd0 = {0, NEG};

    struct Consts {
        V2 qe, e;                           // q + e and e of the lane's two columns
        int32_t f;
        int32_t floor;                      // local: 0 (the restart); anchored modes: NEG (none)
        int32_t row0lo, row0hi;             // H in row 0 of the lane's two columns
    };
    struct State {
        V2 H1, H2, H3, L0, L1, L2, L3, IL, D1, D2, D3, A1, B1, C1;
        V2 VD1, VD2, VA1, VA2;
        uint32_t X1;
        int32_t bslo, bshi, btlo, bthi, t;
        int32_t cmlo, cmhi;                 // this chunk's maximum H per cell
    };

    static __device__ __forceinline__ Consts consts(const ScoreParams &sp)
    {
        return Consts{V2{sp.q + sp.e, sp.q + sp.e}, V2{sp.e, sp.e}, sp.f, sp.mode == MP_MODE_LOCAL ? 0 : NEG, 0, 0};
    }

    static __device__ __forceinline__ V2 pack2(int lo, int hi) { return V2{lo, hi}; }
    static __device__ __forceinline__ void set_row0(Consts &c, int lo, int hi) { c.row0lo = lo; c.row0hi = hi; }
    // profile queries: the gap costs of the lane's two columns
    static __device__ __forceinline__ void set_gaps(Consts &c, int qlo, int elo, int qhi, int ehi, int)
    {
        c.qe = V2{qlo + elo, qhi + ehi};
        c.e = V2{elo, ehi};
    }
    static __device__ __forceinline__ Bnd col0_entry(int h) { return Bnd{h, NEG}; }

    static __device__ __forceinline__ uint32_t prof_entry(int slo, int shi)
    {
        return (static_cast<uint32_t>(slo) & 0xffffu) | (static_cast<uint32_t>(shi) << 16);
    }

    static __device__ __forceinline__ void init(State &s, int lane, Bnd w0, uint4 recm1, uint4 recm2,
                                                uint32_t xm1, int h_self, int h_left)
    {
        // the same history as the int16 state (see Ops16::init)
        const V2 ng{NEG, NEG};
        s.H1 = (lane == 0) ? V2{h_self, NEG} : ng; s.H2 = ng; s.H3 = ng;
        s.L1 = (lane == 0) ? V2{h_left, NEG} : ng; s.L2 = ng; s.L3 = ng;
        s.L0 = (lane == 0) ? V2{w0.h, h_self} : ng;
        s.IL = (lane == 0) ? V2{w0.i, NEG} : ng;
        s.D1 = s.D2 = s.D3 = ng;
        s.A1 = s.B1 = s.C1 = ng;
        s.VD1 = unpack_neg16(recm1.x); s.VD2 = unpack_neg16(recm2.x);
        s.VA1 = unpack_neg16(recm1.y); s.VA2 = unpack_neg16(recm2.y);
        s.X1 = xm1;
        s.bslo = s.bshi = 0; s.btlo = s.bthi = 0; s.t = 0;
        s.cmlo = s.cmhi = NEG;
    }

    using Word = uint2;                     // [H lo, H hi] as int32

    template <bool MASKED, bool KEYS>
    static __device__ __forceinline__ uint2 step(State &s, const Consts &c, const uint4 rec,
                                                 const uint32_t *prof_lane, Bnd bin, Bnd &wout,
                                                 int lane, int ii, int n)
    {
        const V2 VD0 = unpack_neg16(rec.x), VA0 = unpack_neg16(rec.y);   // negated penalties
        const uint32_t X0 = *reinterpret_cast<const uint32_t *>(
            reinterpret_cast<const char *>(prof_lane) + rec.z);
        const uint32_t X0h = *reinterpret_cast<const uint32_t *>(
            reinterpret_cast<const char *>(prof_lane + kProfRows * 32) + rec.z);
        const V2 S{static_cast<int32_t>(X0 << 16) >> 16, static_cast<int32_t>(s.X1) >> 16};
        const V2 M = add(s.L3, S);
        const V2 Iopen = sub(s.L0, c.qe), Iext = sub(s.IL, c.e);
        V2 I0 = mx(Iopen, Iext);
        const V2 Dopen = sub(s.H3, c.qe), Dext = sub(s.D3, c.e);
        V2 D0 = mx(Dopen, Dext);
        const V2 Aopen = add(s.H1, s.VD2);
        V2 A0 = mx(Aopen, s.A1);
        const V2 Bopen = add(s.L1, s.VD1);
        V2 B0 = mx(Bopen, s.B1);
        const V2 Copen = add(s.L1, VD0);
        V2 C0 = mx(Copen, s.C1);
        const V2 FG = subc(mx(mx(s.L1, s.L2), mx(s.H1, s.H2)), c.f);
        const V2 Ap = add(A0, VA0), Bp = add(B0, s.VA2), Cp = add(C0, s.VA1);
        V2 H0 = mx(mx(mx(M, I0), mx(D0, FG)), mx(mx(Ap, Bp), mx(Cp, V2{c.floor, c.floor})));

        bool vlo = true, vhi = true;
        if (MASKED) {
            if (ii < 0) { H0.lo = (ii == -1) ? c.row0lo : NEG; I0.lo = D0.lo = A0.lo = B0.lo = C0.lo = NEG; }
            if (ii < 1) { H0.hi = (ii == 0) ? c.row0hi : NEG; I0.hi = D0.hi = A0.hi = B0.hi = C0.hi = NEG; }
            vlo = ii >= 0 && ii < n;
            vhi = ii >= 1 && ii <= n;
        }

        const int32_t Wh = H0.hi, Wi = I0.hi;
        int32_t Rh = __shfl_up_sync(kFull, Wh, 1);
        int32_t Ri = __shfl_up_sync(kFull, Wi, 1);
        if (lane == 0) { Rh = bin.h; Ri = bin.i; }
        wout = Bnd{Wh, Wi};
        s.L3 = s.L2; s.L2 = s.L1; s.L1 = s.L0;
        s.L0 = V2{Rh, H0.lo};
        s.IL = V2{Ri, I0.lo};
        s.H3 = s.H2; s.H2 = s.H1; s.H1 = H0;
        s.D3 = s.D2; s.D2 = s.D1; s.D1 = D0;
        s.A1 = A0; s.B1 = B0; s.C1 = C0;
        s.VD2 = s.VD1; s.VD1 = VD0;
        s.VA2 = s.VA1; s.VA1 = VA0;
        s.X1 = X0h;

        if (vlo && H0.lo > s.bslo) { s.bslo = H0.lo; s.btlo = s.t; }
        if (vhi && H0.hi > s.bshi) { s.bshi = H0.hi; s.bthi = s.t; }
        if (vlo) s.cmlo = max(s.cmlo, H0.lo);
        if (vhi) s.cmhi = max(s.cmhi, H0.hi);
        s.t += 1;
        return make_uint2(static_cast<uint32_t>(H0.lo), static_cast<uint32_t>(H0.hi));
    }

    // four steps of one lane: two 16-byte stores (4 bytes per cell)
    static __device__ __forceinline__ void store4(uint8_t *strip, int t, int lane, const Word *w)
    {
        uint4 *d = reinterpret_cast<uint4 *>(strip + static_cast<size_t>(t) * (2 * kStepBytes) + lane * 32);
        d[0] = make_uint4(w[0].x, w[0].y, w[1].x, w[1].y);
        d[1] = make_uint4(w[2].x, w[2].y, w[3].x, w[3].y);
    }

    static __device__ __forceinline__ void take_best(const State &s, int half, int t0, int &score, int &t)
    {
        (void)t0;
        score = half ? s.bshi : s.bslo;
        t = half ? s.bthi : s.btlo;
        if (score <= 0) score = -1;
    }
    static __device__ __forceinline__ void reset_best(State &s) { s.cmlo = s.cmhi = NEG; }

    static constexpr bool kChunkMaxBest = false;
    static __device__ __forceinline__ int word_h(const Word &w, int h) { return static_cast<int>(h ? w.y : w.x); }
    static __device__ __forceinline__ Word load_word(const uint8_t *, int, int) { return make_uint2(0, 0); }
    using ColMax = uint2;
    static __device__ __forceinline__ ColMax chunk_max(const State &s)
    {
        return make_uint2(static_cast<uint32_t>(s.cmlo), static_cast<uint32_t>(s.cmhi));
    }
};

// ==================================================== int16, 128-residue strips
// Four residues per lane: lane l holds residues 4l .. 4l+3 of the strip in
// two packed registers, a = [4l, 4l+1] and b = [4l+2, 4l+3] (biased 16-bit
// halves, as in Ops16).  At step t the cells of lane l lie at rows t-4l
// (a lo), t-4l-1 (a hi), t-4l-2 (b lo) and t-4l-3 (b hi), so every cell's
// left neighbour was computed one step earlier: a's lo cell takes it from
// lane l-1 (that lane's b hi cell, one shuffle for four cells), the other
// three from the lane's own registers.  b's rows are a's rows of two steps
// before, so b reuses the records and profile words a read then.  Per cell
// the arithmetic of Eq. 7 is that of Ops16; the shuffle, the record load,
// the profile load and the stores serve four cells instead of two.
struct Ops16x4 {
    using Bnd = uint32_t;                  // [H, I] biased 16-bit
    using Smem = WarpSmem4;
    static constexpr int W = kStripWMax, CPL = 4;
    static constexpr uint32_t Z = 0x80008000u;
    static constexpr uint32_t NEGV = 0x40004000u;
    static constexpr Bnd kBnd0 = 0x40008000u;
    static constexpr bool kChunkMaxBest = true;

    struct Consts {
        uint32_t NQE, E, NF;               // as Ops16
        uint32_t FLOOR;
        uint32_t ROW0A, ROW0B;             // H in row 0 of the lane's four columns (biased)
    };
    struct Reg {
        uint32_t H1, H2, H3, L0, L1, L2, L3, IL, D1, D2, D3, A1, B1, C1;
    };
    struct State {
        Reg a, b;
        uint32_t VD1, VD2, VD3, VD4;        // record x of a's lo row minus 1 .. 4
        uint32_t VA1, VA2, VA3, VA4;        // record y of the same rows
        uint32_t X1;                        // a's profile word of the previous step
        uint32_t Y1, Y2, Y3;                // b's profile words of the last three steps
        uint32_t cma, cmb;                  // this chunk's maxima (pairs with a stream)
        uint32_t TC, k0, k1, k2, k3;        // best-cell keys (pairs without one)
    };
    using ColMax = uint2;                   // [cma, cmb]

    static __device__ __forceinline__ Consts consts(const ScoreParams &sp)
    {
        Consts c;
        const uint32_t qe = sp.q + sp.e;
        c.NQE = neg2(qe, qe);
        c.E = static_cast<uint32_t>(sp.e) | (static_cast<uint32_t>(sp.e) << 16);
        c.NF = neg2(static_cast<uint32_t>(sp.f), static_cast<uint32_t>(sp.f));
        c.FLOOR = sp.mode == MP_MODE_LOCAL ? Z : 0u;
        c.ROW0A = c.ROW0B = Z;
        return c;
    }
    template <typename Row0>
    static __device__ __forceinline__ void set_row0(Consts &c, Row0 row0, int jcol)
    {
        c.ROW0A = Ops16::pack2(row0(jcol), row0(jcol + 1));
        c.ROW0B = Ops16::pack2(row0(jcol + 2), row0(jcol + 3));
    }
    static __device__ __forceinline__ Bnd col0_entry(int h) { return Ops16::col0_entry(h); }

    static __device__ __forceinline__ void build_profile(Smem &sm, const ScoreParams &sp, const uint8_t *P, int m,
                                                         int s, int lane)
    {
        int pc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = s * W + 4 * lane + k;
            pc[k] = j < m ? P[j] : 21;
        }
#pragma unroll 2
        for (int aa = 0; aa < kProfRows; ++aa)
            sm.prof[aa * 32 + lane] =
                make_uint2(Ops16::prof_entry(subst_score(sp, aa, pc[0]), subst_score(sp, aa, pc[1])),
                           Ops16::prof_entry(subst_score(sp, aa, pc[2]), subst_score(sp, aa, pc[3])));
    }
    // records of positions [-kRecPre, kChunk): the history of the first
    // step reaches position -(4 * 31 + 4)
    static __device__ __forceinline__ void fetch_first(Smem &sm, const uint4 *recs, int lane)
    {
        fetch_records4(sm, recs, -2 * kChunk, lane);
        fetch_records4(sm, recs, -kChunk, lane);
        fetch_records4(sm, recs, 0, lane);
    }
    static __device__ __forceinline__ void fetch(Smem &sm, const uint4 *recs, int lo, int lane)
    {
        fetch_records4(sm, recs, lo, lane);
    }
    static __device__ __forceinline__ uint2 prof_at(const Smem &sm, uint32_t z, int lane)
    {
        return *reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(&sm.prof[lane]) + z);
    }

    // State before step 0 (see Ops16::init): only lane 0's a register touches
    // row 0 and the strip's left boundary there; b's rows are above row 0.
    static __device__ __forceinline__ void init(State &s, const Smem &sm, int lane, Bnd w0, int h_self, int h_left)
    {
        const uint32_t hs = Ops16::pack2(h_self, -16384), hl = Ops16::pack2(h_left, -16384);
        Reg &a = s.a;
        a.H1 = (lane == 0) ? hs : NEGV; a.H2 = NEGV; a.H3 = NEGV;
        a.L1 = (lane == 0) ? hl : NEGV; a.L2 = NEGV; a.L3 = NEGV;
        a.L0 = (lane == 0) ? ((w0 & 0xffffu) | (hs << 16)) : NEGV;
        a.IL = (lane == 0) ? ((w0 >> 16) | 0x40000000u) : NEGV;
        a.D1 = a.D2 = a.D3 = NEGV;
        a.A1 = a.B1 = a.C1 = NEGV;
        Reg &b = s.b;
        b.H1 = b.H2 = b.H3 = b.L0 = b.L1 = b.L2 = b.L3 = b.IL = NEGV;
        b.D1 = b.D2 = b.D3 = b.A1 = b.B1 = b.C1 = NEGV;
        const int ii0 = -4 * lane;
        const uint4 r1 = get_record4(sm, ii0 - 1), r2 = get_record4(sm, ii0 - 2);
        const uint4 r3 = get_record4(sm, ii0 - 3), r4 = get_record4(sm, ii0 - 4);
        s.VD1 = r1.x; s.VD2 = r2.x; s.VD3 = r3.x; s.VD4 = r4.x;
        s.VA1 = r1.y; s.VA2 = r2.y; s.VA3 = r3.y; s.VA4 = r4.y;
        const uint2 p1 = prof_at(sm, r1.z, lane), p2 = prof_at(sm, r2.z, lane), p3 = prof_at(sm, r3.z, lane);
        s.X1 = p1.x;
        s.Y1 = p1.y; s.Y2 = p2.y; s.Y3 = p3.y;
        s.cma = s.cmb = 0;
        s.TC = 0xffffu; s.k0 = s.k1 = s.k2 = s.k3 = 0;
    }

    // The cells of one register at rows (lo, lo - 1): Eq. 7 as in Ops16::step.
    // VD0..VD2 / VA0..VA2: records x / y (negated penalties) of rows lo,
    // lo-1, lo-2.  Leaves L0 and IL for the caller (they come from the
    // neighbours of this step).
    template <bool MASKED>
    static __device__ __forceinline__ void cells(Reg &r, const Consts &c, uint32_t S, uint32_t VD0, uint32_t VD1,
                                                 uint32_t VD2, uint32_t VA0, uint32_t VA1, uint32_t VA2,
                                                 uint32_t ROW0, int ii, int n, uint32_t &H0, uint32_t &I0,
                                                 uint32_t &vmask)
    {
        I0 = vaddmax(r.L0, c.NQE, r.IL - c.E);
        uint32_t D0 = vaddmax(r.H3, c.NQE, r.D3 - c.E);
        uint32_t A0 = vaddmax(r.H1, VD2, r.A1);           // H[i-1][j] - r - d(i-1)
        uint32_t B0 = vaddmax(r.L1, VD1, r.B1);           // H[i-1][j-1] - r - d(i)
        uint32_t C0 = vaddmax(r.L1, VD0, r.C1);           // H[i-1][j-1] - r - d(i+1)
        uint32_t Y = vaddmax(r.H2, c.NF, c.FLOOR);
        Y = vaddmax(vmax3(r.L1, r.L2, r.H1), c.NF, Y);
        Y = vaddmax(C0, VA1, Y);
        Y = vaddmax(B0, VA2, Y);
        Y = vaddmax(A0, VA0, Y);
        H0 = vmax3(vaddmax(r.L3, S, I0), D0, Y);
        vmask = 0xffffffffu;
        if (MASKED) {
            const uint32_t kill = (ii < 0 ? 0x0000ffffu : 0u) | (ii < 1 ? 0xffff0000u : 0u);
            const uint32_t row0 = (ii == -1 ? 0x0000ffffu : 0u) | (ii == 0 ? 0xffff0000u : 0u);
            const uint32_t hforce = (row0 & ROW0) | (~row0 & NEGV);
            H0 = (H0 & ~kill) | (hforce & kill);
            I0 = (I0 & ~kill) | (NEGV & kill);
            D0 = (D0 & ~kill) | (NEGV & kill);
            A0 = (A0 & ~kill) | (NEGV & kill);
            B0 = (B0 & ~kill) | (NEGV & kill);
            C0 = (C0 & ~kill) | (NEGV & kill);
            vmask = ((ii >= 0 && ii < n) ? 0x0000ffffu : 0u) | ((ii >= 1 && ii <= n) ? 0xffff0000u : 0u);
        }
        r.L3 = r.L2; r.L2 = r.L1; r.L1 = r.L0;
        r.H3 = r.H2; r.H2 = r.H1; r.H1 = H0;
        r.D3 = r.D2; r.D2 = r.D1; r.D1 = D0;
        r.A1 = A0; r.B1 = B0; r.C1 = C0;
    }

    // One anti-diagonal step: the four cells of the lane.  rec: record of
    // a's lo row ii; xy: the profile words of that row's codon.
    template <bool MASKED, bool KEYS>
    static __device__ __forceinline__ void step(State &s, const Consts &c, const uint4 rec, const uint2 xy, Bnd bin,
                                                Bnd &wout, int lane, int ii, int n, uint32_t &wa, uint32_t &wb)
    {
        const uint32_t Sa = (xy.x & 0x0000ffffu) | (s.X1 & 0xffff0000u);   // s(i, 4l), s(i-1, 4l+1)
        const uint32_t Sb = (s.Y2 & 0x0000ffffu) | (s.Y3 & 0xffff0000u);   // s(i-2, 4l+2), s(i-3, 4l+3)
        uint32_t Ha, Ia, ma, Hb, Ib, mb;
        cells<MASKED>(s.a, c, Sa, rec.x, s.VD1, s.VD2, rec.y, s.VA1, s.VA2, c.ROW0A, ii, n, Ha, Ia, ma);
        cells<MASKED>(s.b, c, Sb, s.VD2, s.VD3, s.VD4, s.VA2, s.VA3, s.VA4, c.ROW0B, ii - 2, n, Hb, Ib, mb);
        // hand [H, I] of b's hi cell to the next lane; lane 0 takes the strip boundary
        const uint32_t Wd = prmt<0x7632>(Hb, Ib);
        uint32_t R = __shfl_up_sync(kFull, Wd, 1);
        if (lane == 0) R = bin;
        wout = Wd;
        s.a.L0 = prmt<0x5410>(R, Ha);
        s.a.IL = prmt<0x5432>(R, Ia);
        s.b.L0 = prmt<0x5432>(Ha, Hb);
        s.b.IL = prmt<0x5432>(Ia, Ib);
        s.VD4 = s.VD3; s.VD3 = s.VD2; s.VD2 = s.VD1; s.VD1 = rec.x;
        s.VA4 = s.VA3; s.VA3 = s.VA2; s.VA2 = s.VA1; s.VA1 = rec.y;
        s.X1 = xy.x;
        s.Y3 = s.Y2; s.Y2 = s.Y1; s.Y1 = xy.y;
        const uint32_t ha = Ha & ma, hb = Hb & mb;
        if (KEYS) {
            s.k0 = max(s.k0, ha * 65536u + s.TC);
            s.k1 = max(s.k1, (ha & 0xffff0000u) | s.TC);
            s.k2 = max(s.k2, hb * 65536u + s.TC);
            s.k3 = max(s.k3, (hb & 0xffff0000u) | s.TC);
            s.TC -= 1;
        } else {
            s.cma = vmax(s.cma, ha);
            s.cmb = vmax(s.cmb, hb);
        }
        wa = Ha;
        wb = Hb;
    }

    template <bool MASKED, bool STORE>
    static __device__ __forceinline__ void chunk(State &st, const Consts &c, Smem &sm, int lane, int t0, int n,
                                                 uint8_t *code_strip)
    {
#pragma unroll 1
        for (int bdy = 0; bdy < kChunk / kBody; ++bdy) {
            const int tb = t0 + bdy * kBody;
            // record of a's lo cell at step tb+k: position tb+k-4l, quarter k&3,
            // index ridx + k/4 within it (tb is a multiple of 4)
            const int ridx = ring4_idx(tb - 4 * lane);
            const uint4 *rq = &sm.ring[0][ridx];
            uint32_t cw[2 * kBody];
            Bnd bin4[4], wout4[4];
#pragma unroll
            for (int k = 0; k < kBody; ++k) {
                if ((k & 3) == 0) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) bin4[u] = sm.bin[bdy * kBody + k + u];
                }
                const uint4 rec = rq[(k & 3) * (kRing4 + kRing4Pad) + (k >> 2)];
                const uint2 xy = prof_at(sm, rec.z, lane);
                step<MASKED, !STORE>(st, c, rec, xy, bin4[k & 3], wout4[k & 3], lane, tb + k - 4 * lane, n,
                                     cw[2 * k], cw[2 * k + 1]);
                if ((k & 3) == 3 && lane == 31) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) sm.bout[bdy * kBody + k - 3 + u] = wout4[u];
                }
                if (STORE && (k & 1) == 1) {
                    // two steps of one lane: one 16-byte store
                    *reinterpret_cast<uint4 *>(code_strip + static_cast<size_t>(tb + k - 1) * (W * 2) + lane * 16) =
                        make_uint4(cw[2 * k - 2], cw[2 * k - 1], cw[2 * k], cw[2 * k + 1]);
                }
            }
        }
    }

    // (score, step) of cell k's best key (pairs without a stream)
    static __device__ __forceinline__ void take_best(const State &s, int k, int t0, int &score, int &t)
    {
        const uint32_t key = k == 0 ? s.k0 : k == 1 ? s.k1 : k == 2 ? s.k2 : s.k3;
        score = static_cast<int>(key >> 16) - 32768;
        t = t0 + static_cast<int>(0xffffu - (key & 0xffffu));
    }
    static __device__ __forceinline__ void reset_best(State &s)
    {
        s.TC = 0xffffu; s.k0 = s.k1 = s.k2 = s.k3 = 0; s.cma = s.cmb = 0;
    }
    static __device__ __forceinline__ ColMax chunk_max(const State &s) { return make_uint2(s.cma, s.cmb); }
    static __device__ __forceinline__ int cell_max(const ColMax &m, int k)
    {
        const uint32_t w = k < 2 ? m.x : m.y;
        return static_cast<int>((k & 1) ? (w >> 16) : (w & 0xffffu)) - 32768;
    }
    // stored H of cell k of the lane at step t
    static __device__ __forceinline__ int load_cell(const uint8_t *strip, int t, int lane, int k)
    {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(strip + static_cast<size_t>(t >> 1) * 512 + lane * 16 +
                                                               (t & 1) * 8 + (k >> 1) * 4);
        return static_cast<int>((k & 1) ? (w >> 16) : (w & 0xffffu)) - 32768;
    }
};

// ============================================================ strip driver
struct Best {
    int score, ii, jj;
};

// Traceback of pair p by the warp that finished its last strip (a call, not
// inlined, so the traceback's registers stay out of the DP loop's budget).
__device__ __noinline__ void trace_inline(const DPArgs &a, uint32_t p, int lane)
{
    TBArgs t{};
    t.pairs = a.pairs;
    t.codes = a.codes;
    t.prot = a.prot;
    t.nt2 = a.nt2;
    t.out = a.out;
    t.ops = a.ops;
    t.col0 = a.col0;
    t.sp = a.sp;
    t.prof = a.prof;
    t.epre = a.epre;
    trace_pair<true>(t, a.mat, p, lane);
}

__device__ __forceinline__ bool better(int s, int i, int j, const Best &b)
{
    return s > b.score || (s == b.score && (i < b.ii || (i == b.ii && j < b.jj)));
}

template <typename Ops, bool MASKED, bool STORE>
__device__ __forceinline__ void run_chunk(typename Ops::State &st, const typename Ops::Consts &c,
                                          WarpSmem<typename Ops::Bnd> &sm, int lane, int t0, int n,
                                          uint8_t *code_strip)
{
#pragma unroll 1
    for (int b = 0; b < kChunk / kBody; ++b) {
        const int tb = t0 + b * kBody;
        // record of the lo cell at step tb+k: position tb+k-2l, parity k&1,
        // index (tb+k)/2 - l within its half (tb is even)
        const int ridx = ((tb >> 1) - lane) & (kRing / 2 - 1);
        const uint4 *re = &sm.ring[0][ridx];
        const uint4 *ro = &sm.ring[1][ridx];
        typename Ops::Word cw[kBody];
        typename Ops::Bnd bin4[4], wout4[4];
#pragma unroll
        for (int k = 0; k < kBody; ++k) {
            // boundary entries move 4 steps at a time: one broadcast load for
            // lane 0's inputs, one store of lane 31's outputs
            if ((k & 3) == 0) {
#pragma unroll
                for (int u = 0; u < 4; ++u) bin4[u] = sm.bin[b * kBody + k + u];
            }
            cw[k] = Ops::template step<MASKED, !STORE>(st, c, (k & 1) ? ro[k >> 1] : re[k >> 1], sm.prof + lane,
                                                         bin4[k & 3], wout4[k & 3], lane, tb + k - 2 * lane, n);
            if ((k & 3) == 3) {
                if (lane == 31) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) sm.bout[b * kBody + k - 3 + u] = wout4[u];
                }
                if (STORE) Ops::store4(code_strip, tb + k - 3, lane, &cw[k - 3]);
            }
        }
    }
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T ld_l2(const T *p);
template <>
__device__ __forceinline__ uint32_t ld_l2<uint32_t>(const uint32_t *p) { return __ldcg(p); }
template <>
__device__ __forceinline__ Ops32::Bnd ld_l2<Ops32::Bnd>(const Ops32::Bnd *p)
{
    const int2 v = __ldcg(reinterpret_cast<const int2 *>(p));
    return Ops32::Bnd{v.x, v.y};
}

// (score, ii, jj) -> key whose unsigned maximum is the best cell under the
// tie rule: largest score, then smallest ii, then smallest jj
__device__ __forceinline__ unsigned long long best_key(int score, int ii, int jj)
{
    return (static_cast<unsigned long long>(score) << 40) |
           (static_cast<unsigned long long>(0xfffffu - static_cast<uint32_t>(ii)) << 20) |
           static_cast<unsigned long long>(0xfffffu - static_cast<uint32_t>(jj));
}

// One strip s of pair p (64 residues, two per lane, or 128, four per lane).
// Strip s reads the boundary row (H and I of the last residue of strip s-1
// at every genome position) that strip s-1 publishes chunk by chunk, and
// publishes its own last residue for strip s+1.
template <typename Ops>
__device__ void run_strip(const DPArgs &a, typename Ops::Smem &sm, const PairDesc &pd, uint32_t p, int s, int lane,
                          bool rerun)
{
    using Bnd = typename Ops::Bnd;
    constexpr int W = Ops::W, CPL = Ops::CPL;
    const int n = static_cast<int>(pd.nt_len);
    const int m = static_cast<int>(pd.prot_len);
    const int nstrips = static_cast<int>(pd.n_strips);
    const bool store = !(pd.flags & PF_SCORE_ONLY);
    const uint8_t *P = a.prot + pd.prot_off;
    Bnd *bnd = reinterpret_cast<Bnd *>(a.bnd) + pd.bnd_off + kBndPad;   // bnd[ii], ii >= -kBndPad
    typename Ops::Consts c = Ops::consts(a.sp);
    // anchored modes: row 0 holds H[0][j] = -(q + e j) (an I run from cell
    // (0, 0)) and column 0 the values of the column-0 array; local: both 0
    const bool anchored = a.sp.mode != MP_MODE_LOCAL;
    const int32_t *c0 = anchored ? a.col0 + pd.col0_off : nullptr;      // c0[i] = H[i][0]
    const int jcol = s * W + CPL * lane + 1;                             // 1-based column of the lane's first cell
    // profile queries (2-cell forms only): position-specific gap costs and
    // substitution scores of positions 1..m at pf[1..m]
    const ProfPos *pf = (pd.flags & PF_PROF) ? a.prof + pd.prof_off : nullptr;
    const int32_t *ep = (pd.flags & PF_PROF) ? a.epre + pd.prof_off : nullptr;
    auto row0 = [&](int j) {
        if (!anchored || j == 0) return 0;
        if (pf) return -(pf[1].q + __ldg(ep + (j < m ? j : m)) + (j > m ? a.sp.e * (j - m) : 0));
        return -(a.sp.q + a.sp.e * j);
    };
    if constexpr (CPL == 4) {
        Ops::set_row0(c, row0, jcol);
    } else {
        Ops::set_row0(c, row0(jcol), row0(jcol + 1));
        if (pf) {
            const int jl = jcol <= m ? jcol : 0, jh = jcol + 1 <= m ? jcol + 1 : 0;
            const int jn = jcol + 2 <= m ? jcol + 2 : 0;
            Ops::set_gaps(c, jl ? pf[jl].q : a.sp.q, jl ? pf[jl].e : a.sp.e, jh ? pf[jh].q : a.sp.q,
                          jh ? pf[jh].e : a.sp.e, jn ? pf[jn].e : a.sp.e);
        }
    }
    const int nsteps = n + W - 1;
    const int nchunks = (nsteps + kChunk - 1) / kChunk;
    // 2 bytes per cell in the int16 paths, 4 in the int32 path
    const size_t strip_bytes = static_cast<size_t>(nchunks) * kChunk * W * 2 * (sizeof(Bnd) / 4);
    const uint32_t *prev = a.progress + pd.strip_base + s - 1;   // valid for s > 0
    uint32_t *mine = a.progress + pd.strip_base + s;
    bool timed_out = false;

    // wait until strip s-1 has published `need` chunks (bounded)
    const uint32_t spin_limit = a.spin_limit ? a.spin_limit : kSpinLimit;
    auto wait_for = [&](uint32_t need) {
        if (s == 0 || timed_out) return;
        uint32_t ok = 1;
        if (lane == 0) {
            uint32_t it = 0;
            while (ld_acquire(prev) < need) {
                __nanosleep(256);
                if (++it > spin_limit) { ok = 0; break; }
            }
        }
        ok = __shfl_sync(kFull, ok, 0);
        if (!ok) timed_out = true;
        __syncwarp();
    };

    const uint4 *recs = a.recs + pd.rec_off;            // recs[ii + kRecPre] is position ii
    if constexpr (CPL == 4) {
        Ops::build_profile(sm, a.sp, P, m, s, lane);
        Ops::fetch_first(sm, recs, lane);
    } else {
        // profile: prof[aa][lane] = [s(aa, P[2l]), s(aa, P[2l+1])]
        const int jlo = s * W + 2 * lane, jhi = jlo + 1;
        const int plo = jlo < m ? P[jlo] : 21, phi = jhi < m ? P[jhi] : 21;
        if (pf) {
            // a profile query: position-specific scores (no codon: -512 as subst_score)
#pragma unroll 2
            for (int aa = 0; aa < kProfRows; ++aa) {
                sm.prof[aa * 32 + lane] =
                    Ops::prof_entry(aa == 21 ? -512 : jlo < m ? pf[jlo + 1].s[aa] : subst_score(a.sp, aa, 21), 0);
                sm.prof[(kProfRows + aa) * 32 + lane] =
                    Ops::prof_entry(0, aa == 21 ? -512 : jhi < m ? pf[jhi + 1].s[aa] : subst_score(a.sp, aa, 21));
            }
        } else {
#pragma unroll 2
            for (int aa = 0; aa < kProfRows; ++aa) {
                sm.prof[aa * 32 + lane] = Ops::prof_entry(subst_score(a.sp, aa, plo), 0);
                sm.prof[(kProfRows + aa) * 32 + lane] = Ops::prof_entry(0, subst_score(a.sp, aa, phi));
            }
        }
        // records for ii in [-kChunk, kChunk)
        fetch_records(sm, recs, -kChunk, lane);
        fetch_records(sm, recs, 0, lane);
    }
    cp_async_wait_all();
    __syncwarp();
    // chunk c reads boundary entries c*kChunk+1 .. (c+1)*kChunk, which strip s-1
    // writes W-1 steps later: up to its chunk c + 1 + (W-1)/kChunk
    constexpr int kLag = 2 + (W - 1) / kChunk;
    wait_for(nchunks < kLag ? nchunks : kLag);
    __syncwarp();
    typename Ops::State st;
    {
        const Bnd w0 = s > 0 ? ld_l2(bnd) : (anchored ? Ops::col0_entry(__ldg(c0 + 1)) : Ops::kBnd0);
        if constexpr (CPL == 4) {
            Ops::init(st, sm, lane, w0, row0(jcol), row0(jcol - 1));
        } else {
            const int ii0 = -2 * lane;
            const uint4 rm1 = get_record(sm, ii0 - 1);
            const uint4 rm2 = get_record(sm, ii0 - 2);
            const uint32_t xm1 = sm.prof[(kProfRows + (rm1.z >> 7)) * 32 + lane];   // the hi table
            Ops::init(st, lane, w0, rm1, rm2, xm1, row0(jcol), row0(jcol - 1));
        }
    }
    uint8_t *code_strip = a.codes + pd.code_off + static_cast<size_t>(s) * strip_bytes;
    // per-chunk column maxima of H follow the strips' streams: [strip][chunk][lane]
    typename Ops::ColMax *colmax = reinterpret_cast<typename Ops::ColMax *>(
        a.codes + pd.code_off + static_cast<size_t>(nstrips) * strip_bytes) + static_cast<size_t>(s) * nchunks * 32;
    Best best{0, 0x7fffffff, 0x7fffffff};
    int cbest[CPL], cchunk[CPL];                    // per cell: best chunk maximum and its chunk
#pragma unroll
    for (int k = 0; k < CPL; ++k) cbest[k] = cchunk[k] = 0;

    for (int ch = 0; ch < nchunks; ++ch) {
        const int t0 = ch * kChunk;
        if (ch > 0) {
            cp_async_wait_all();                         // this chunk's records (queued last chunk)
            wait_for(ch + kLag < nchunks ? ch + kLag : nchunks);
        }
        if (s == 0 && anchored) {
            // column 0 of the anchored modes; bin[k] is genome position t0 + 1 + k (row t0 + 2 + k)
            for (int k = lane; k < kChunk; k += 32) sm.bin[k] = Ops::col0_entry(__ldg(c0 + t0 + 2 + k));
        } else if (s == 0) {
            for (int k = lane; k < kChunk; k += 32) sm.bin[k] = Ops::kBnd0;   // column 0: H = 0, I = -inf
        } else {
            for (int k = lane; k < kChunk; k += 32) sm.bin[k] = ld_l2(bnd + t0 + 1 + k);
        }
        __syncwarp();
        // next chunk's records land in ring slots this chunk does not read
        if (ch + 1 < nchunks) {
            if constexpr (CPL == 4) Ops::fetch(sm, recs, t0 + kChunk, lane);
            else fetch_records(sm, recs, t0 + kChunk, lane);
        }
        const bool masked = (t0 < W) || (t0 + kChunk > n);
        if constexpr (CPL == 4) {
            if (masked) {
                if (store) Ops::template chunk<true, true>(st, c, sm, lane, t0, n, code_strip);
                else Ops::template chunk<true, false>(st, c, sm, lane, t0, n, code_strip);
            } else {
                if (store) Ops::template chunk<false, true>(st, c, sm, lane, t0, n, code_strip);
                else Ops::template chunk<false, false>(st, c, sm, lane, t0, n, code_strip);
            }
        } else {
            if (masked) {
                if (store) run_chunk<Ops, true, true>(st, c, sm, lane, t0, n, code_strip);
                else run_chunk<Ops, true, false>(st, c, sm, lane, t0, n, code_strip);
            } else {
                if (store) run_chunk<Ops, false, true>(st, c, sm, lane, t0, n, code_strip);
                else run_chunk<Ops, false, false>(st, c, sm, lane, t0, n, code_strip);
            }
        }
        __syncwarp();
        if (s + 1 < nstrips && !a.no_publish) {
            // publish residue W(s+1)-1 for strip s+1
            for (int k = lane; k < kChunk; k += 32) bnd[t0 + k - (W - 1)] = sm.bout[k];
            // __syncwarp orders every lane's stores before lane 0's release
            // (release is cumulative), so one release store publishes the chunk
            __syncwarp();
            if (lane == 0) st_release(mine, static_cast<uint32_t>(ch + 1));
        }
        if (store) colmax[static_cast<size_t>(ch) * 32 + lane] = Ops::chunk_max(st);
        bool folded = false;
        if constexpr (Ops::kChunkMaxBest) {
            if (store) {
                // remember the first chunk holding each cell's maximum
                const typename Ops::ColMax cmw = Ops::chunk_max(st);
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const int v = Ops::cell_max(cmw, k);
                    if (v > cbest[k]) { cbest[k] = v; cchunk[k] = ch; }
                }
                folded = true;
            }
        }
        if (!folded) {
            // fold this chunk's best cells into the strip's best
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                int sc, t;
                Ops::take_best(st, k, t0, sc, t);
                const int jj = s * W + CPL * lane + k;
                const int ii = t - CPL * lane - k;
                if (sc > 0 && jj < m && better(sc, ii, jj, best)) best = Best{sc, ii, jj};
            }
        }
        Ops::reset_best(st);
        __syncwarp();
    }
    if constexpr (Ops::kChunkMaxBest) {
      if (store) {
        // first step of the best chunk holding the maximum, read back from this
        // lane's own stored H values (valid cells only)
        __syncwarp();
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int jj = s * W + CPL * lane + k;
            if (cbest[k] <= 0 || jj >= m) continue;
            const int tb = cchunk[k] * kChunk;
            for (int t = tb; t < tb + kChunk; ++t) {
                const int ii = t - CPL * lane - k;
                if (ii < 0 || ii >= n) continue;
                if (Ops::load_cell(code_strip, t, lane, k) == cbest[k]) {
                    if (better(cbest[k], ii, jj, best)) best = Best{cbest[k], ii, jj};
                    break;
                }
            }
        }
      }
    }
    // warp reduction of (score desc, ii asc, jj asc)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Best o;
        o.score = __shfl_xor_sync(kFull, best.score, off);
        o.ii = __shfl_xor_sync(kFull, best.ii, off);
        o.jj = __shfl_xor_sync(kFull, best.jj, off);
        if (better(o.score, o.ii, o.jj, best)) best = o;
    }
    int trace_now = 0;
    if (lane == 0) {
        if (best.score > 0) atomicMax(a.best_key + p, best_key(best.score, best.ii, best.jj));
        if (timed_out) atomicOr(&a.out[p].status, MP_ST_TIMEOUT);
        __threadfence();
        const uint32_t done = atomicAdd(a.strips_done + p, 1u);
        if (done == static_cast<uint32_t>(nstrips - 1)) {
            // last strip of the pair: publish the pair's best cell
            __threadfence();
            const unsigned long long key = atomicAdd(a.best_key + p, 0ull);
            PairOut &o = a.out[p];
            const int score = static_cast<int>(key >> 40);
            o.score = score;
            if (sizeof(Bnd) == 8) o.status |= kStInt32Stream;
            o.best_ii = score > 0 ? static_cast<int>(0xfffffu - ((key >> 20) & 0xfffffu)) : -1;
            o.best_jj = score > 0 ? static_cast<int>(0xfffffu - (key & 0xfffffu)) : -1;
            if (!rerun && sizeof(Bnd) == 4 && score >= kOverflowT && !(o.status & MP_ST_TIMEOUT) &&
                !(pd.flags & PF_WIDE)) {
                // cannot happen: the pair's score bound was below the int16 limit
                o.status |= MP_ST_TRACE;
            } else if (!rerun && sizeof(Bnd) == 4 && score >= kOverflowT && !(o.status & MP_ST_TIMEOUT)) {
                // int16 saturated: queue every strip of this pair for the int32 kernel
                o.status |= MP_ST_RERUN;
                a.best_key[p] = 0;
                a.strips_done[p] = 0;
                for (int k = 0; k < nstrips; ++k) a.progress[pd.strip_base + k] = 0;
                const uint32_t slot = atomicAdd(a.rerun_count, static_cast<uint32_t>(nstrips));
                for (int k = 0; k < nstrips; ++k) a.rerun_items[slot + k] = make_uint2(p, k);
            }
            // the pair is final (not queued for the int32 kernel): trace it now,
            // while other warps run other strips
            trace_now = a.mat != nullptr && !(o.status & MP_ST_ERRMASK) &&
                        !(pd.flags & (PF_SCORE_ONLY | PF_SKIP | PF_BUDGET)) &&
                        (!(o.status & MP_ST_RERUN) || sizeof(Bnd) == 8) &&
                        (score > 0 || a.sp.mode == MP_MODE_GLOBAL);
        }
    }
    trace_now = __shfl_sync(kFull, trace_now, 0);
    __syncwarp();
    if (trace_now) {
        __threadfence();        // the other strips' streams (published before their count) are visible
        trace_inline(a, p, lane);
        __syncwarp();
        if (lane == 0) a.out[p].status |= kStTraced;
    }
    __syncwarp();
}

// MinB: CTAs per SM the build is made for (the register budget per thread
// follows from it: 3 -> 80, 2 -> 128 for 256-thread CTAs).  Wide4: the
// int16 build that also runs pairs in 128-residue strips (PF_W128), each
// warp's shared memory sized for either strip form.
template <typename Ops, int MinB, bool Wide4 = false>
__global__ void __launch_bounds__(kWarpsPerCta * 32, MinB) dp_kernel(const DPArgs a, int rerun_only)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SM = typename Ops::Smem;
    constexpr size_t kWarpBytes = Wide4 && sizeof(WarpSmem4) > sizeof(SM) ? sizeof(WarpSmem4) : sizeof(SM);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *mine = smem_raw + static_cast<size_t>(warp) * kWarpBytes;
    // a fixed list (the wave's interleaved strip items, or the re-run list):
    // a strip's warp waits, bounded, for its predecessor's rows
    const uint2 *list = rerun_only ? a.rerun_items : a.items;
    const uint32_t count = rerun_only ? *a.rerun_count : a.n_items;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(a.head, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= count) break;
        const uint2 it = list[idx];
        const PairDesc pd = a.pairs[it.x];
        if constexpr (Wide4) {
            if (pd.flags & PF_W128) {
                run_strip<Ops16x4>(a, *reinterpret_cast<WarpSmem4 *>(mine), pd, it.x, static_cast<int>(it.y), lane,
                                   rerun_only != 0);
                continue;
            }
        }
        run_strip<Ops>(a, *reinterpret_cast<SM *>(mine), pd, it.x, static_cast<int>(it.y), lane, rerun_only != 0);
    }
}

}  // namespace

size_t dp16_smem_bytes() { return sizeof(WarpSmem<Ops16::Bnd>) * kWarpsPerCta; }
size_t dp16w_smem_bytes()
{
    return (sizeof(WarpSmem4) > sizeof(WarpSmem<Ops16::Bnd>) ? sizeof(WarpSmem4) : sizeof(WarpSmem<Ops16::Bnd>)) *
           kWarpsPerCta;
}
size_t dp32_smem_bytes() { return sizeof(WarpSmem<Ops32::Bnd>) * kWarpsPerCta; }

static int blocks_per_sm(const void *fn, size_t smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kWarpsPerCta * 32, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

// The shared-memory opt-in is a per-device function attribute: set it, and
// read the occupancy, once per device and build.
template <typename Ops, int MinB, bool Wide4 = false>
static int kernel_blocks_per_sm(size_t smem)
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> nb[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) dev = 0;
    int v = nb[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        cudaFuncSetAttribute(dp_kernel<Ops, MinB, Wide4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
        v = blocks_per_sm(reinterpret_cast<const void *>(dp_kernel<Ops, MinB, Wide4>), smem);
        nb[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

int dp16_blocks_per_sm(int variant, bool wide4)
{
    if (wide4) return kernel_blocks_per_sm<Ops16, 2, true>(dp16w_smem_bytes());
    return variant == 1 ? kernel_blocks_per_sm<Ops16, 2>(dp16_smem_bytes())
                        : kernel_blocks_per_sm<Ops16, 3>(dp16_smem_bytes());
}

int dp32_blocks_per_sm() { return kernel_blocks_per_sm<Ops32, 2>(dp32_smem_bytes()); }

namespace {
// Per-nt records of every pair (see make_record), positions -kRecPre upwards
// (z, the profile row's byte offset, for the pair's strip form: rows of 32
// lanes x 4 B, or x 8 B in 128-residue strips).
// The genetic code and the splice terms are looked up in shared tables
// (lanes index them at different positions: from constant memory such
// reads serialise), the splice terms by three 5-symbol codes (four bases and
// "outside the region"), filled from the splice model's own functions.
__global__ void records_kernel(const PairDesc *pairs, uint32_t n_pairs, const uint32_t *nt2, const ScoreParams sp,
                               uint4 *recs)
{
    __shared__ int8_t s_code[64];
    __shared__ int16_t s_don[125], s_acc[125];
    for (int k = threadIdx.x; k < 64; k += blockDim.x) s_code[k] = c_code.v[k];
    for (int k = threadIdx.x; k < 125; k += blockDim.x) {
        const int c1 = k / 25, c2 = (k / 5) % 5, c3 = k % 5;
        const bool v1 = c1 != 4, v2 = c2 != 4, v3 = c3 != 4;
        const int b1 = v1 ? c1 : 0, b2 = v2 ? c2 : 0, b3 = v3 ? c3 : 0;
        s_don[k] = static_cast<int16_t>(splice_donor(sp, b1, b2, b3, v1, v2, v3));
        s_acc[k] = static_cast<int16_t>(splice_acceptor(sp, b1, b2, b3, v1, v2, v3));
    }
    __syncthreads();
    const uint32_t r = static_cast<uint32_t>(sp.r);
    for (uint32_t p = blockIdx.x; p < n_pairs; p += gridDim.x) {
        const PairDesc pd = pairs[p];
        if (pd.flags & PF_SKIP) continue;
        const int n = static_cast<int>(pd.nt_len);
        const int cnt = static_cast<int>(records_of(pd.nt_len));
        const uint32_t *g = nt2 + pd.nt_word_off;
        uint4 *out = recs + pd.rec_off;
        const uint32_t zrow = (pd.flags & PF_W128) ? 256u : 128u;
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            // the same record as make_record: window T0[ii-3 .. ii+4]
            const int ii = k - kRecPre;
            const int s0 = ii - 3;
            const int w = s0 >> 4;
            const uint64_t pair64 = (static_cast<uint64_t>(g[w + 1]) << 32) | g[w];
            const uint32_t win = static_cast<uint32_t>(pair64 >> ((s0 & 15) * 2));
            int c[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                c[q] = static_cast<unsigned>(s0 + q) < static_cast<unsigned>(n) ? static_cast<int>((win >> (2 * q)) & 3)
                                                                               : 4;
            const int aa = (c[1] != 4 && c[3] != 4) ? s_code[c[1] * 16 + c[2] * 4 + c[3]] : 21;
            const uint32_t dC = static_cast<uint32_t>(s_don[(c[5] * 5 + c[6]) * 5 + c[7]]);   // d(i+1)
            const uint32_t dB = static_cast<uint32_t>(s_don[(c[4] * 5 + c[5]) * 5 + c[6]]);   // d(i)
            const uint32_t aA = static_cast<uint32_t>(s_acc[(c[1] * 5 + c[2]) * 5 + c[3]]);   // a(i)
            const uint32_t aC = static_cast<uint32_t>(s_acc[(c[0] * 5 + c[1]) * 5 + c[2]]);   // a(i-1)
            out[k] = make_uint4(neg2(r + dC, r + dB), neg2(aA, aC), static_cast<uint32_t>(aa) * zrow, 0u);
        }
    }
}
}  // namespace

cudaError_t launch_records(const PairDesc *pairs, uint32_t n, const uint32_t *nt2, const ScoreParams &sp, uint4 *recs,
                           cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    records_kernel<<<n < 8192 ? n : 8192, 256, 0, st>>>(pairs, n, nt2, sp, recs);
    return cudaGetLastError();
}

cudaError_t launch_dp16(const DPArgs &a, int grid, int variant, bool wide4, cudaStream_t st)
{
    dp16_blocks_per_sm(variant, wide4);
    if (wide4) dp_kernel<Ops16, 2, true><<<grid, kWarpsPerCta * 32, dp16w_smem_bytes(), st>>>(a, 0);
    else if (variant == 1) dp_kernel<Ops16, 2><<<grid, kWarpsPerCta * 32, dp16_smem_bytes(), st>>>(a, 0);
    else dp_kernel<Ops16, 3><<<grid, kWarpsPerCta * 32, dp16_smem_bytes(), st>>>(a, 0);
    return cudaGetLastError();
}

cudaError_t launch_dp32(const DPArgs &a, int grid, bool rerun_only, cudaStream_t st)
{
    dp32_blocks_per_sm();
    dp_kernel<Ops32, 2><<<grid, kWarpsPerCta * 32, dp32_smem_bytes(), st>>>(a, rerun_only ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace mpdp

// ===========================================================================
// Allocation-free scoring of one pair.
//
// Some callers cannot call cudaMalloc: services that fix their device
// memory at start-up and may not allocate or free afterwards (cudaMalloc and
// cudaFree can synchronize the device, and an allocation can fail once other
// tenants hold the memory), and hosts that hand device memory to plug-ins
// only from their own pools.  For them mp_dp_score_pair_noalloc runs the same packed-int16 DP (with the
// same int32 re-run on saturation) on one pair, score only, using a fixed
// scratch array that lives in this library's module for the life of the
// process.  Every GPU that loads the library holds this array until exit.
// ===========================================================================
namespace mpdp {
namespace {

constexpr int kNAMaxProt = 4096;                     // residues
constexpr int kNAMaxNt = 32768;                      // nucleotides
constexpr int kNAMaxStrips = kNAMaxProt / kStripW;   // 64
constexpr int kNANtWords = kNAMaxNt / 16 + 2 * kNtPadWords;
constexpr int kNABndEntries =
    ((kNAMaxNt + kStripW - 1 + kChunk - 1) / kChunk) * kChunk + 2 * kBndPad + 32;

struct NoAllocScratch {
    PairDesc desc;
    PairOut out;
    unsigned long long best_key;
    uint32_t strips_done, rerun_count, head16, head32;
    uint32_t progress[kNAMaxStrips];
    uint2 rerun_items[kNAMaxStrips];
    uint32_t nt2[kNANtWords];
    uint4 recs[records_of(kNAMaxNt)];
    uint8_t prot[kNAMaxProt];
    Ops32::Bnd bnd[kNABndEntries];                   // int32 entries; the int16 pass uses the first half
};

// The scratch itself (about 820 KB).  Host code must not pass this name to a
// kernel: on the host it is only a stand-in for the symbol.  Its device
// address is looked up with cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

__device__ __forceinline__ uint8_t na_aa_code(unsigned char c)
{
    // ARNDCQEGHILKMFPSTWYV -> 0..19, '*' -> 20, anything else -> X (21)
    const char *order = "arndcqeghilkmfpstwyv";
    const unsigned char l = c | 0x20;
    for (int k = 0; k < 20; ++k)
        if (order[k] == l) return static_cast<uint8_t>(k);
    return c == '*' ? 20 : 21;
}

__device__ __forceinline__ int na_nt_code(unsigned char c)
{
    switch (c | 0x20) {
    case 'a': return 0;
    case 'c': return 1;
    case 'g': return 2;
    case 't': return 3;
    default: return -1;
    }
}

// One CTA of kWarpsPerCta warps: pack the pair into the scratch, run its
// strips on cooperating warps (int16, then int32 if it saturated), write
// {score, status, protein end, genome end on the forward strand} to out4.
__global__ void __launch_bounds__(kWarpsPerCta * 32, 1)
dp_noalloc_kernel(ScoreParams sp, const char *prot_ascii, int m, const char *nt_ascii, int n, int strand,
                  int32_t *out4, NoAllocScratch *S, uint32_t spin_limit)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int bad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nstrips = (m + kStripW - 1) / kStripW;
    if (threadIdx.x == 0) {
        PairDesc d{};
        d.prot_len = static_cast<uint32_t>(m);
        d.nt_len = static_cast<uint32_t>(n);
        d.nt_word_off = kNtPadWords;
        d.flags = PF_SCORE_ONLY | PF_WIDE;       // score only: no traceback stream in either mode
        d.strand = strand;
        d.n_strips = static_cast<uint32_t>(nstrips);
        S->desc = d;
        PairOut o{};
        o.best_ii = o.best_jj = -1;
        S->out = o;
        S->best_key = 0;
        S->strips_done = S->rerun_count = S->head16 = S->head32 = 0;
        bad = 0;
    }
    // the flag is cleared before any thread can set it while packing
    __syncthreads();
    // every call starts from zeroed progress counters
    for (int k = threadIdx.x; k < kNAMaxStrips; k += blockDim.x) S->progress[k] = 0;
    for (int k = threadIdx.x; k < m; k += blockDim.x)
        S->prot[k] = na_aa_code(static_cast<unsigned char>(prot_ascii[k]));
    const int nwords = (n + 15) / 16;
    for (int w = static_cast<int>(threadIdx.x) - kNtPadWords; w < nwords + kNtPadWords; w += blockDim.x) {
        uint32_t word = 0;
        for (int k = 0; k < 16 && w >= 0 && w < nwords; ++k) {
            const int pos = w * 16 + k;
            if (pos >= n) break;
            int b = na_nt_code(static_cast<unsigned char>(strand >= 0 ? nt_ascii[pos] : nt_ascii[n - 1 - pos]));
            if (b < 0) { bad = 1; b = 0; }
            if (strand < 0) b = 3 - b;
            word |= static_cast<uint32_t>(b) << (2 * k);
        }
        S->nt2[kNtPadWords + w] = word;
    }
    __syncthreads();
    // per-nt records of the pair (positions -kChunk upwards)
    for (int k = threadIdx.x; k < static_cast<int>(records_of(static_cast<uint32_t>(n))); k += blockDim.x)
        S->recs[k] = make_record(S->nt2 + kNtPadWords, n, k - kRecPre, sp);
    __syncthreads();
    if (!bad && m > 0 && n > 0) {
        const PairDesc pd = S->desc;             // written by thread 0 before the barriers above
        DPArgs a{};
        a.pairs = &S->desc;
        a.recs = S->recs;
        a.prot = S->prot;
        a.nt2 = S->nt2;
        a.codes = nullptr;                       // score only: no traceback codes
        a.bnd = S->bnd;
        a.out = &S->out;
        a.progress = S->progress;
        a.best_key = &S->best_key;
        a.strips_done = &S->strips_done;
        a.rerun_items = S->rerun_items;
        a.rerun_count = &S->rerun_count;
        a.sp = sp;
        a.spin_limit = spin_limit;
        {
            auto &sm = reinterpret_cast<WarpSmem<Ops16::Bnd> *>(smem_raw)[warp];
            for (;;) {
                uint32_t s = 0;
                if (lane == 0) s = atomicAdd(&S->head16, 1u);
                s = __shfl_sync(kFull, s, 0);
                if (s >= static_cast<uint32_t>(nstrips)) break;
                run_strip<Ops16>(a, sm, pd, 0, static_cast<int>(s), lane, false);
            }
        }
        __syncthreads();
        const uint32_t nre = *reinterpret_cast<volatile uint32_t *>(&S->rerun_count);
        if (nre) {
            auto &sm = reinterpret_cast<WarpSmem<Ops32::Bnd> *>(smem_raw)[warp];
            for (;;) {
                uint32_t s = 0;
                if (lane == 0) s = atomicAdd(&S->head32, 1u);
                s = __shfl_sync(kFull, s, 0);
                if (s >= nre) break;
                run_strip<Ops32>(a, sm, pd, 0, static_cast<int>(S->rerun_items[s].y), lane, true);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const PairOut o = S->out;                // written by this block before the barrier
        const int score = bad ? 0 : (o.score > 0 ? o.score : 0);
        out4[0] = score;
        out4[1] = bad ? MP_ST_BADSEQ : (o.status & 0xff);
        out4[2] = score > 0 ? o.best_jj + 1 : 0;
        out4[3] = score > 0 ? (strand >= 0 ? o.best_ii + 1 : n - (o.best_ii + 1)) : 0;
    }
}

constexpr size_t kNASmem = sizeof(WarpSmem<Ops32::Bnd>) * kWarpsPerCta;   // covers the int16 layout too

}  // namespace
}  // namespace mpdp

extern "C" int mp_dp_score_pair_noalloc(const mp_dp_params *params, const char *d_prot, uint32_t prot_len,
                                        const char *d_nt, uint32_t nt_len, int8_t strand, int32_t *d_out,
                                        void *stream)
{
    using namespace mpdp;
    if (prot_len > static_cast<uint32_t>(kNAMaxProt) || nt_len > static_cast<uint32_t>(kNAMaxNt))
        return MP_ETOOLARGE;
    if (!d_out || (prot_len && !d_prot) || (nt_len && !d_nt) || (strand != 1 && strand != -1)) return MP_EINVAL;
    mp_dp_params p;
    if (params) p = *params;
    else mp_dp_default_params(&p);
    int mn = 0;
    for (int x = 0; x < 20; ++x)
        for (int y = 0; y < 22; ++y) mn = p.mat[x][y] < mn ? p.mat[x][y] : mn;
    if (p.q < 0 || p.e < 1 || p.f < 0 || p.r < 0 || p.stop < 0 || p.q + p.e > 1000 || p.f > 1000 ||
        p.r > 1000 || p.stop > 512 || !(p.r > p.f && p.r > p.stop && p.r > -mn) ||
        (p.splice_model != MP_SPLICE_FINAL && p.splice_model != MP_SPLICE_SIMPLE) || p.splice_p < 0 ||
        p.splice_p > 1000 || p.mode != MP_MODE_LOCAL || p.wait_limit < 0 || p.max_pairs_per_launch < 0)
        return MP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return MP_ECUDA;
    // Set-up, once per device, with that device current: the device address
    // of the scratch array and the kernel's shared-memory attribute.  The
    // first call on a device does this, so make it before any stream capture.
    constexpr int kMaxDev = 64;
    static void *scratch_ptr[kMaxDev] = {};
    static std::once_flag once[kMaxDev];
    if (dev >= kMaxDev) return MP_ECUDA;
    cudaError_t setup_err = cudaSuccess;
    std::call_once(once[dev], [&] {
        void *ptr = nullptr;
        setup_err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (setup_err == cudaSuccess)
            setup_err = cudaFuncSetAttribute(dp_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kNASmem));
        if (setup_err == cudaSuccess) scratch_ptr[dev] = ptr;
    });
    if (setup_err != cudaSuccess || !scratch_ptr[dev]) return MP_ECUDA;
    ScoreParams sp;
    sp.q = p.q; sp.e = p.e; sp.f = p.f; sp.r = p.r; sp.stop = p.stop;
    sp.splice_model = p.splice_model;
    sp.splice_p = p.splice_p;
    sp.mode = MP_MODE_LOCAL;
    for (int x = 0; x < 22; ++x)
        for (int y = 0; y < 22; ++y) sp.mat[x][y] = p.mat[x][y];
    dp_noalloc_kernel<<<1, kWarpsPerCta * 32, kNASmem, static_cast<cudaStream_t>(stream)>>>(
        sp, d_prot, static_cast<int>(prot_len), d_nt, static_cast<int>(nt_len), strand, d_out,
        static_cast<NoAllocScratch *>(scratch_ptr[dev]), p.wait_limit > 0 ? static_cast<uint32_t>(p.wait_limit) : 0u);
    return cudaGetLastError() == cudaSuccess ? MP_OK : MP_ECUDA;
}

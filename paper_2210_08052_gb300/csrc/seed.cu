// Seeding and chaining on the GPU (Li 2022, Methods: "Reduced alphabet",
// "Indexing the genome", "Chaining").  Hand-written for sm_103a.
//
// Index: both strands of the genome as independent sequences, each in three
// reading frames; every open reading frame (a maximal run of codons without
// a stop codon) of at least 30 amino acids; every 6-mer inside one whose
// hash psi(phi(6-mer)) has lowest bit 0 is stored as strand << 31 | bin,
// bin = floor(x / 256) with x the k-mer's first base on its strand.  The
// table is CSR over all 2^24 hash values, each value's entries ascending.
//
//   translate_kernel   reduced-alphabet code of every codon of the six frames
//   segment_kernel     per 1024-codon segment: its first and last stop codon
//   segment_scan       per frame: the nearest stop before and after each segment
//   kmer_kernel        per segment (one warp): run bounds of every codon from the
//                      stops, the sampled k-mers of long runs, counted (pass 0)
//                      or written at their bucket's cursor (pass 1)
//   scan kernels       exclusive prefix sums (bucket counts -> CSR offsets)
//   bucket_sort_kernel each bucket's entries in ascending order
//
// Chaining, per protein (one warp each): its k-mers' hits as anchors
// (strand, x = bin, y = residue), sorted; the recurrence of Eq. 2 with the
// gap of Eq. 1 and the penalty of Eq. 3 (G = 200,000, beta = 0.75) in fixed
// point with 16 fractional bits (the log term from a table of every |g| < G),
// predecessors evaluated 32 at a time; then the chains in order of
// decreasing score of their last anchor.
//
// Second round, per (protein, region) pair: every 5-mer of the protein
// (reduced alphabet, sorted in shared memory) against the 5-mer starting at
// every base of the region's aligned strand by binary search (one block per
// pair, contiguous base ranges per thread, so the anchors come out in (x, y)
// order), counted then written; chained by one warp per pair with
// g' = 3 dy - dx and Eq. 3.
#include <cstdint>
#include <cstring>
#include <vector>

#include "mp_internal.cuh"

namespace mpdp {
namespace {

constexpr int kK = 6;                       // k-mer length (amino acids)
constexpr int kKeyBits = 4 * kK;            // 24-bit codes
constexpr uint32_t kNKeys = 1u << kKeyBits;
constexpr int kBin = 256;
constexpr int kMinOrf = 30;
constexpr int64_t kG = 200000;              // largest gap (bp) of a chain link
constexpr int64_t kScale = 65536;           // chaining scores in units of 2^-16
constexpr int kSeg = 1024;                  // codons per segment
constexpr uint8_t kStopCode = 14;           // phi of a stop codon
constexpr uint8_t kXCode = 15;

// The reduced alphabet ("Reduced alphabet"): A 0, ST 1, RK 2, H 3, ND 4,
// EQ 5, C 6, P 7, G 8, IV 10, LM 11, FY 12, W 13, stop 14, anything else 15.
constexpr uint8_t phi_letter(char c)
{
    return c == 'A' ? 0 : (c == 'S' || c == 'T') ? 1 : (c == 'R' || c == 'K') ? 2 : c == 'H' ? 3
         : (c == 'N' || c == 'D') ? 4 : (c == 'E' || c == 'Q') ? 5 : c == 'C' ? 6 : c == 'P' ? 7
         : c == 'G' ? 8 : (c == 'I' || c == 'V') ? 10 : (c == 'L' || c == 'M') ? 11
         : (c == 'F' || c == 'Y') ? 12 : c == 'W' ? 13 : c == '*' ? 14 : 15;
}

// NCBI table 1 with codons enumerated as A, C, G, T in each position.
constexpr char kCodonAA[] = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF";

struct Table64 {
    uint8_t v[64];
};
struct Table256 {
    uint8_t v[256];
};
constexpr Table64 make_codon_phi()
{
    Table64 t{};
    for (int k = 0; k < 64; ++k) t.v[k] = phi_letter(kCodonAA[k]);
    return t;
}
constexpr Table256 make_aa_phi()
{
    Table256 t{};
    for (int c = 0; c < 256; ++c) t.v[c] = phi_letter(static_cast<char>(c >= 'a' && c <= 'z' ? c - 32 : c));
    return t;
}

// phi of each codon (bases in A, C, G, T order) and of each protein letter
__constant__ Table64 c_codon_phi = make_codon_phi();
__constant__ Table256 c_aa_phi = make_aa_phi();

__device__ __forceinline__ int base_code(unsigned char c)
{
    switch (c | 0x20) {
    case 'a': return 0;
    case 'c': return 1;
    case 'g': return 2;
    case 't': return 3;
    default: return -1;
    }
}

// psi: Thomas Wang's integer mix with every step modulo 2^24 (a bijection
// of [0, 2^24), the invertible hash the paper cites from minimap)
__device__ __forceinline__ uint32_t psi24(uint32_t key)
{
    const uint64_t mask = (1ull << kKeyBits) - 1;
    uint64_t k = key & mask;
    k = (~k + (k << 21)) & mask;
    k = k ^ k >> 24;
    k = (k + (k << 3) + (k << 8)) & mask;
    k = k ^ k >> 14;
    k = (k + (k << 2) + (k << 4)) & mask;
    k = k ^ k >> 28;
    k = (k + (k << 31)) & mask;
    return static_cast<uint32_t>(k);
}

// frame fr = 3 * strand + frame of the index's six frames
struct Frames {
    uint8_t *code[6];          // phi of codon t of each frame
    uint64_t len[6];           // codons per frame
    uint64_t seg0[7];          // first segment index of each frame (segments are numbered across frames)
};

// Reduced-alphabet code of every codon of every frame.  Codon t of frame f
// of strand 1 is the reverse complement's bases f + 3t .. f + 3t + 2, i.e.
// the complements of genome[n-1-(f+3t)], genome[n-2-(f+3t)], genome[n-3-(f+3t)].
__global__ void translate_kernel(const char *g, uint64_t n, Frames fr)
{
    const uint64_t total = fr.len[0] + fr.len[1] + fr.len[2] + fr.len[3] + fr.len[4] + fr.len[5];
    for (uint64_t q = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        int f = 0;
        uint64_t t = q;
        while (t >= fr.len[f]) t -= fr.len[f++];
        const int strand = f / 3, frame = f % 3;
        const uint64_t x = frame + 3 * t;
        int b[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int c = base_code(static_cast<unsigned char>(strand ? g[n - 1 - (x + u)] : g[x + u]));
            b[u] = c < 0 ? -1 : (strand ? 3 - c : c);
        }
        fr.code[f][t] = (b[0] < 0 || b[1] < 0 || b[2] < 0) ? kXCode : c_codon_phi.v[b[0] * 16 + b[1] * 4 + b[2]];
    }
}

// per segment: first and last stop codon (frame-relative index), or -1
__global__ void segment_kernel(Frames fr, int64_t *first, int64_t *last, uint64_t nseg)
{
    const int lane = threadIdx.x & 31;
    for (uint64_t s = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; s < nseg;
         s += (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5) {
        int f = 0;
        while (s >= fr.seg0[f + 1]) ++f;
        const uint64_t t0 = (s - fr.seg0[f]) * kSeg, len = fr.len[f];
        int64_t lo = -1, hi = -1;
        for (int c = 0; c < kSeg; c += 32) {
            const uint64_t t = t0 + c + lane;
            const bool stop = t < len && fr.code[f][t] == kStopCode;
            const unsigned bal = __ballot_sync(0xffffffffu, stop);
            if (bal) {
                if (lo < 0) lo = static_cast<int64_t>(t0 + c + __ffs(bal) - 1);
                hi = static_cast<int64_t>(t0 + c + 31 - __clz(bal));
            }
        }
        if (lane == 0) {
            first[s] = lo;
            last[s] = hi;
        }
    }
}

// per frame (one block of kScanThreads each): for every segment, the last
// stop codon before it (-1 if none) and the first after it (the frame's
// length if none): each thread reduces a contiguous range of segments, the
// block scans the thread totals, each thread then walks its range again
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) segment_scan(Frames fr, const int64_t *first, const int64_t *last,
                                                              int64_t *before, int64_t *after)
{
    __shared__ int64_t red[kScanThreads];
    const int f = blockIdx.x;
    const uint64_t s0 = fr.seg0[f], s1 = fr.seg0[f + 1], ns = s1 - s0;
    const uint64_t per = (ns + kScanThreads - 1) / kScanThreads;
    const uint64_t ta = threadIdx.x * per, tb = (threadIdx.x + 1) * per;
    const uint64_t a = s0 + (ta < ns ? ta : ns), b = s0 + (tb < ns ? tb : ns);
    // forward: the last stop of the ranges before this thread's
    int64_t mx = -1;
    for (uint64_t s = a; s < b; ++s) mx = last[s] > mx ? last[s] : mx;
    red[threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = -1;
        for (int t = 0; t < kScanThreads; ++t) {
            const int64_t v = red[t];
            red[t] = run;
            run = v > run ? v : run;
        }
    }
    __syncthreads();
    int64_t cur = red[threadIdx.x];
    for (uint64_t s = a; s < b; ++s) {
        before[s] = cur;
        if (last[s] >= 0) cur = last[s];
    }
    __syncthreads();
    // backward: the first stop of the ranges after this thread's
    const int64_t none = static_cast<int64_t>(fr.len[f]);
    int64_t mn = none;
    for (uint64_t s = a; s < b; ++s)
        if (first[s] >= 0 && first[s] < mn) mn = first[s];
    red[threadIdx.x] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = none;
        for (int t = kScanThreads - 1; t >= 0; --t) {
            const int64_t v = red[t];
            red[t] = run;
            run = v < run ? v : run;
        }
    }
    __syncthreads();
    cur = red[threadIdx.x];
    for (uint64_t s = b; s > a; --s) {
        after[s - 1] = cur;
        if (first[s - 1] >= 0) cur = first[s - 1];
    }
}

// One warp per segment.  For codon t of a run [a, b) (a after a stop or at
// the frame's start, b at the next stop or the frame's end) with b - a >=
// kMinOrf and t + kK <= b, the k-mer code of codons t .. t+5 is hashed; a
// sampled one (lowest bit 0) is counted in its bucket (pass 0) or written at
// its bucket's cursor (pass 1).
constexpr int kKmerWarps = 4;

__global__ void __launch_bounds__(kKmerWarps * 32) kmer_kernel(Frames fr, const int64_t *before, const int64_t *after,
                                                               uint64_t nseg, int pass, uint32_t *count,
                                                               uint32_t *cursor, uint32_t *entries)
{
    // the stop before and after each codon of the warp's segment
    __shared__ int32_t s_prev[kKmerWarps][kSeg / 32][32], s_next[kKmerWarps][kSeg / 32][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    auto prev = [&](int c) -> int32_t & { return s_prev[w][c][lane]; };
    auto next = [&](int c) -> int32_t & { return s_next[w][c][lane]; };
    for (uint64_t s = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; s < nseg;
         s += (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5) {
        int f = 0;
        while (s >= fr.seg0[f + 1]) ++f;
        const uint64_t t0 = (s - fr.seg0[f]) * kSeg, len = fr.len[f];
        const uint8_t *code = fr.code[f];
        // the stop before each codon, sweeping forward; the stop after, sweeping back
        int64_t cur = before[s];
        for (int c = 0; c < kSeg / 32; ++c) {
            const uint64_t t = t0 + c * 32 + lane;
            const bool stop = t < len && code[t] == kStopCode;
            const unsigned bal = __ballot_sync(0xffffffffu, stop);
            const unsigned below = bal & ((1u << lane) - 1);
            prev(c) = static_cast<int32_t>(below ? static_cast<int64_t>(t0 + c * 32 + 31 - __clz(below)) : cur);
            if (bal) cur = static_cast<int64_t>(t0 + c * 32 + 31 - __clz(bal));
        }
        cur = after[s];
        for (int c = kSeg / 32 - 1; c >= 0; --c) {
            const uint64_t t = t0 + c * 32 + lane;
            const bool stop = t < len && code[t] == kStopCode;
            const unsigned bal = __ballot_sync(0xffffffffu, stop);
            const unsigned above = lane == 31 ? 0u : (bal & ~((2u << lane) - 1));
            next(c) = static_cast<int32_t>(above ? static_cast<int64_t>(t0 + c * 32 + __ffs(above) - 1) : cur);
            if (bal) cur = static_cast<int64_t>(t0 + c * 32 + __ffs(bal) - 1);
        }
        const uint32_t strand = f / 3, frame = f % 3;
        for (int c = 0; c < kSeg / 32; ++c) {
            const uint64_t t = t0 + c * 32 + lane;
            if (t >= len || code[t] == kStopCode) continue;
            const int64_t a = prev(c) + 1, b = next(c);
            if (b - a < kMinOrf || static_cast<int64_t>(t) + kK > b) continue;
            uint32_t key = 0;
#pragma unroll
            for (int u = 0; u < kK; ++u) key = key * 16 + code[t + u];
            const uint32_t h = psi24(key);
            if (h & 1u) continue;
            if (pass == 0) {
                atomicAdd(count + h, 1u);
            } else {
                const uint32_t at = atomicAdd(cursor + h, 1u);
                entries[at] = (strand << 31) | static_cast<uint32_t>((frame + 3 * t) / kBin);
            }
        }
    }
}

// ---- exclusive prefix sum of n uint32 counts into n + 1 uint32 offsets
constexpr int kScanBlock = 1024;

__global__ void scan_blocks(const uint32_t *in, uint64_t n, uint32_t *out, uint32_t *block_sums)
{
    __shared__ uint32_t warp_tot[32];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanBlock * 4;
    uint32_t v[4], s = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint64_t i = base + threadIdx.x * 4 + u;
        v[u] = i < n ? in[i] : 0u;
        s += v[u];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t t = warp_tot[lane], ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        warp_tot[lane] = ti - t;
        if (lane == 31) block_sums[blockIdx.x] = ti;
    }
    __syncthreads();
    uint32_t run = warp_tot[w] + incl - s;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint64_t i = base + threadIdx.x * 4 + u;
        if (i < n) out[i] = run;
        run += v[u];
    }
}

__global__ void scan_sums(uint32_t *block_sums, uint32_t nb, uint32_t *total)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint32_t run = 0;
        for (uint32_t b = 0; b < nb; ++b) {
            const uint32_t v = block_sums[b];
            block_sums[b] = run;
            run += v;
        }
        *total = run;
    }
}

__global__ void scan_add(uint32_t *out, uint64_t n, const uint32_t *block_sums, const uint32_t *total)
{
    const uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    if (i < n) out[i] += block_sums[i / (kScanBlock * 4)];
    if (i == 0) out[n] = *total;
}

// each bucket's entries in ascending order (buckets hold a few dozen)
__global__ void bucket_sort_kernel(const uint32_t *off, uint32_t *entries)
{
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < kNKeys; h += gridDim.x * blockDim.x) {
        const uint32_t a = off[h], b = off[h + 1];
        for (uint32_t i = a + 1; i < b; ++i) {
            const uint32_t v = entries[i];
            uint32_t j = i;
            while (j > a && entries[j - 1] > v) {
                entries[j] = entries[j - 1];
                --j;
            }
            entries[j] = v;
        }
    }
}

// ------------------------------------------------------------- chaining
__device__ __forceinline__ int64_t gap_eq1(int64_t dx, int64_t dy)
{
    const int64_t py = 3 * dy;
    if (py < kBin * (dx - 1)) return py - kBin * (dx - 1);
    if (py > kBin * (dx + 1)) return py - kBin * (dx + 1);
    return 0;
}

// floor(S beta log2(v)) for v = |g| + 1: an integer log2 for a power of two
// (the device log2 need not be exact there), the double log2 otherwise
// (each such value lies at least 6.8e-6 from an integer for |g| < G)
__device__ __forceinline__ int64_t log_term(uint64_t v)
{
    return (v & (v - 1)) == 0
               ? static_cast<int64_t>(63 - __clzll(static_cast<long long>(v))) * (3 * kScale / 4)
               : static_cast<int64_t>(floor(0.75 * static_cast<double>(kScale) * log2(static_cast<double>(v))));
}

// the log term of every |g| < G, computed once per chaining call
__global__ void log_table_kernel(int32_t *tab)
{
    for (int64_t a = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; a < kG;
         a += static_cast<int64_t>(gridDim.x) * blockDim.x)
        tab[a] = static_cast<int32_t>(log_term(static_cast<uint64_t>(a + 1)));
}

// Eq. 3 in units of 2^-16: floor(S |g| / 3) and floor(S beta log2(|g| + 1))
// (their sum for g > 0, the smaller for g < 0); -1 if |g| >= G.  lt: the
// log terms of log_table_kernel.
__device__ __forceinline__ int64_t penalty_eq3(int64_t g, const int32_t *lt)
{
    if (g == 0) return 0;
    const int64_t a = g < 0 ? -g : g;
    if (a >= kG) return -1;
    const int64_t lin = (a * kScale) / 3;
    const int64_t lg = __ldg(lt + a);
    if (g > 0) return lin + lg;
    return lin < lg ? lin : lg;
}

// anchors of protein p: (strand << 63) | (x << 20) | y, x = bin, y = residue
__device__ __forceinline__ uint32_t kmer_hash(const char *P, int t)
{
    uint32_t key = 0;
#pragma unroll
    for (int u = 0; u < kK; ++u) key = key * 16 + c_aa_phi.v[static_cast<unsigned char>(P[t + u])];
    return psi24(key);
}

struct ChainArgs {
    const char *prot;
    const uint64_t *prot_off;
    const uint32_t *prot_len;
    uint32_t n_prot;
    const uint32_t *off;          // index CSR
    const uint32_t *entries;
    uint64_t *anc_off;            // per protein: first anchor (n_prot + 1)
    uint64_t *anc;                // anchors
    int64_t *f;                   // chaining score per anchor
    int32_t *pred;                // predecessor per anchor (-1: none)
    uint8_t *used;
    int top;
    mp_chain *chains;             // n_prot * top
    uint32_t *n_chains;
    const int32_t *log_tab;       // log terms of Eq. 3 for |g| < G
};

__global__ void anchor_count_kernel(ChainArgs a, uint64_t *count)
{
    const int lane = threadIdx.x & 31;
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < a.n_prot; p += (gridDim.x * blockDim.x) >> 5) {
        const char *P = a.prot + a.prot_off[p];
        const int m = static_cast<int>(a.prot_len[p]);
        uint64_t c = 0;
        for (int t = lane; t + kK <= m; t += 32) {
            const uint32_t h = kmer_hash(P, t);
            c += a.off[h + 1] - a.off[h];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) count[p] = c;
    }
}

__global__ void anchor_fill_kernel(ChainArgs a)
{
    const int lane = threadIdx.x & 31;
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < a.n_prot; p += (gridDim.x * blockDim.x) >> 5) {
        const char *P = a.prot + a.prot_off[p];
        const int m = static_cast<int>(a.prot_len[p]);
        uint64_t at = a.anc_off[p];
        for (int t0 = 0; t0 + kK <= m; t0 += 32) {
            const int t = t0 + lane;
            uint32_t lo = 0, hi = 0;
            if (t + kK <= m) {
                const uint32_t h = kmer_hash(P, t);
                lo = a.off[h];
                hi = a.off[h + 1];
            }
            // each lane's hits go after the earlier lanes' hits
            uint64_t cnt = hi - lo, incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            for (uint32_t e = lo; e < hi; ++e) {
                const uint32_t v = a.entries[e];
                a.anc[at + incl - cnt + (e - lo)] = (static_cast<uint64_t>(v >> 31) << 63) |
                                                    (static_cast<uint64_t>(v & 0x7fffffffu) << 20) |
                                                    static_cast<uint64_t>(t);
            }
            at += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// One block per protein: its anchors sorted ascending (strand, x, y) by a
// bitonic network, in shared memory up to kSortMax anchors, otherwise over
// a scratch range of the next power of two (its tail padded with the
// largest key) in global memory.
constexpr int kSortMax = 16384;           // 128 KB of shared memory
constexpr int kSortThreads = 1024;

__global__ void __launch_bounds__(kSortThreads) anchor_sort_kernel(ChainArgs a, uint64_t *scratch,
                                                                   const uint64_t *scratch_off)
{
    extern __shared__ uint64_t sh[];
    for (uint32_t p = blockIdx.x; p < a.n_prot; p += gridDim.x) {
        const uint64_t b0 = a.anc_off[p], n = a.anc_off[p + 1] - b0;
        if (n < 2) continue;
        uint64_t n2 = 1;
        while (n2 < n) n2 <<= 1;
        uint64_t *v = n2 <= kSortMax ? sh : scratch + scratch_off[p];
        for (uint64_t i = threadIdx.x; i < n2; i += blockDim.x) v[i] = i < n ? a.anc[b0 + i] : ~0ull;
        __syncthreads();
        for (uint64_t k = 2; k <= n2; k <<= 1)
            for (uint64_t j = k >> 1; j > 0; j >>= 1) {
                for (uint64_t i = threadIdx.x; i < n2; i += blockDim.x) {
                    const uint64_t l = i ^ j;
                    if (l > i) {
                        const uint64_t x = v[i], y = v[l];
                        if ((x > y) == ((i & k) == 0)) {
                            v[i] = y;
                            v[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) a.anc[b0 + i] = v[i];
        __syncthreads();
    }
}

__device__ __forceinline__ int anc_strand(uint64_t v) { return static_cast<int>(v >> 63); }
__device__ __forceinline__ int64_t anc_x(uint64_t v) { return static_cast<int64_t>((v >> 20) & 0x7fffffffffull); }
__device__ __forceinline__ int64_t anc_y(uint64_t v) { return static_cast<int64_t>(v & 0xfffffu); }

// One warp per protein: Eq. 2 over its sorted anchors, then its chains.
__global__ void chain_kernel(ChainArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t S = kScale;
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < a.n_prot; p += (gridDim.x * blockDim.x) >> 5) {
        const uint64_t b0 = a.anc_off[p];
        const int64_t n = static_cast<int64_t>(a.anc_off[p + 1] - b0);
        const uint64_t *A = a.anc + b0;
        int64_t *F = a.f + b0;
        int32_t *Pr = a.pred + b0;
        uint8_t *U = a.used + b0;
        const int64_t m = a.prot_len[p];
        // predecessors further than this many bins have |g| >= G
        const int64_t wbins = (kG + 3 * m) / kBin + 2;
        int64_t lo = 0;
        for (int64_t j = 0; j < n; ++j) {
            const uint64_t vj = A[j];
            const int sj = anc_strand(vj);
            const int64_t xj = anc_x(vj), yj = anc_y(vj);
            while (lo < j && (anc_strand(A[lo]) != sj || anc_x(A[lo]) < xj - wbins)) ++lo;
            int64_t best = static_cast<int64_t>(kK) * S;
            int64_t arg = -1;
            for (int64_t i0 = lo; i0 < j; i0 += 32) {
                const int64_t i = i0 + lane;
                int64_t cand = INT64_MIN;
                if (i < j) {
                    const uint64_t vi = A[i];
                    const int64_t dy = yj - anc_y(vi);
                    if (anc_strand(vi) == sj && anc_x(vi) <= xj && dy > 0) {
                        const int64_t pen = penalty_eq3(gap_eq1(xj - anc_x(vi), dy), a.log_tab);
                        if (pen >= 0) cand = F[i] + (dy < kK ? dy : kK) * S - pen;
                    }
                }
                // the largest candidate, the first index among equals
                int64_t c = cand, ci = i;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int64_t oc = __shfl_xor_sync(0xffffffffu, c, o);
                    const int64_t oi = __shfl_xor_sync(0xffffffffu, ci, o);
                    if (oc > c || (oc == c && oi < ci)) {
                        c = oc;
                        ci = oi;
                    }
                }
                if (c > best) {
                    best = c;
                    arg = ci;
                }
            }
            if (lane == 0) {
                F[j] = best;
                Pr[j] = static_cast<int32_t>(arg);
                U[j] = 0;
            }
            __syncwarp();
        }
        // chains in order of decreasing f of the last anchor (ties: the earlier
        // anchor), each cut at an anchor already used; single anchors dropped;
        // once the best unused anchor starts no chain (f = k), none follows
        int nc = 0;
        while (nc < a.top) {
            int64_t bf = INT64_MIN, bi = -1;
            for (int64_t i0 = 0; i0 < n; i0 += 32) {
                const int64_t i = i0 + lane;
                int64_t v = INT64_MIN, vi = i;
                if (i < n && !U[i]) v = F[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int64_t ov = __shfl_xor_sync(0xffffffffu, v, o);
                    const int64_t oi = __shfl_xor_sync(0xffffffffu, vi, o);
                    if (ov > v || (ov == v && oi < vi)) {
                        v = ov;
                        vi = oi;
                    }
                }
                if (v > bf || (v == bf && vi < bi)) {
                    bf = v;
                    bi = vi;
                }
            }
            if (bi < 0 || bf <= static_cast<int64_t>(kK) * S) break;
            if (lane == 0) {
                int64_t cnt = 0, cur = bi, first = bi, stop = -1;
                while (cur >= 0 && !U[cur]) {
                    U[cur] = 1;
                    first = cur;
                    ++cnt;
                    cur = Pr[cur];
                }
                if (cur >= 0) stop = cur;
                if (cnt >= 2) {
                    mp_chain &c = a.chains[static_cast<uint64_t>(p) * a.top + nc];
                    c.strand = anc_strand(A[bi]);
                    c.n_anchors = static_cast<int32_t>(cnt);
                    c.score = F[bi] - (stop >= 0 ? F[stop] : 0);
                    c.x_first = anc_x(A[first]);
                    c.x_last = anc_x(A[bi]);
                    c.y_first = anc_y(A[first]);
                    c.y_last = anc_y(A[bi]);
                }
                nc += cnt >= 2 ? 1 : 0;
            }
            nc = __shfl_sync(0xffffffffu, nc, 0);
            __syncwarp();
        }
        if (lane == 0) a.n_chains[p] = static_cast<uint32_t>(nc);
    }
}

// ---------------------------------------------------------- second round

constexpr int kK2 = 5;                      // k-mer length of the second round
constexpr int kRefineMaxProt = 8192;        // protein k-mer table in shared memory (64 KB)
constexpr int kRefineThreads = 256;
constexpr size_t kRefineSmem = kRefineMaxProt * sizeof(uint64_t);
constexpr int64_t kRefineBig = 512;          // pairs with more anchors are chained by a whole block

struct RefineArgs {
    const char *seq;                        // every pair's protein and region (ASCII)
    const uint64_t *prot_off, *nt_off;
    const uint32_t *prot_len, *nt_len;
    const int8_t *strand;
    uint32_t n;                             // pairs
    const uint64_t *anc_off;                // pair p's anchors at anc[anc_off[p] ..)
    uint64_t *anc;                          // x << 20 | y
    int64_t *f;
    int32_t *pred;
    mp_chain2 *out;
    const int32_t *log_tab;
};

// phi of the codon starting at base x of the pair's aligned strand
__device__ __forceinline__ uint32_t codon_phi(const char *nt, int64_t L, int strand, int64_t x)
{
    int b[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int c = strand > 0 ? base_code(static_cast<unsigned char>(nt[x + u]))
                                 : base_code(static_cast<unsigned char>(nt[L - 1 - (x + u)]));
        b[u] = c < 0 ? -1 : (strand > 0 ? c : 3 - c);
    }
    if (b[0] < 0 || b[1] < 0 || b[2] < 0) return kXCode;
    return c_codon_phi.v[b[0] * 16 + b[1] * 4 + b[2]];
}

// FILL = false: count each thread's anchors into tcount[p * kRefineThreads +
// t] and the pair's into total[p]; true: write them from anc_off[p] on, in
// (x, y) order (thread t's after those of threads 0 .. t-1)
//
// The protein's k-mers are sorted as key << 13 | y (bitonic, shared
// memory), so each base's k-mer finds its equal protein k-mers by one binary
// search, in ascending y.
template <bool FILL>
__global__ void __launch_bounds__(kRefineThreads) refine_anchor_kernel(RefineArgs a, uint32_t *tcount,
                                                                       uint64_t *total)
{
    extern __shared__ uint64_t pk[];                // kRefineMaxProt entries
    __shared__ uint64_t part[kRefineThreads];
    for (uint32_t p = blockIdx.x; p < a.n; p += gridDim.x) {
        const char *P = a.seq + a.prot_off[p];
        const char *T = a.seq + a.nt_off[p];
        const int m = static_cast<int>(a.prot_len[p]);
        const int64_t L = a.nt_len[p];
        const int strand = a.strand[p];
        const int ny = m - kK2 + 1;                 // protein k-mers
        const int64_t nx = L - 3 * kK2 + 1;          // region k-mers (one per base)
        int n2 = 1;
        while (n2 < ny) n2 <<= 1;
        for (int y = threadIdx.x; y < n2; y += blockDim.x) {
            uint64_t key = ~0ull;
            if (y < ny) {
                key = 0;
#pragma unroll
                for (int u = 0; u < kK2; ++u) key = key * 16 + c_aa_phi.v[static_cast<unsigned char>(P[y + u])];
                key = key << 13 | static_cast<uint64_t>(y);
            }
            pk[y] = key;
        }
        __syncthreads();
        for (int k = 2; k <= n2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const uint64_t u = pk[i], v = pk[l];
                        if ((u > v) == ((i & k) == 0)) {
                            pk[i] = v;
                            pk[l] = u;
                        }
                    }
                }
                __syncthreads();
            }
        // thread t takes bases [x0, x1)
        const int64_t per = nx > 0 && ny > 0 ? (nx + blockDim.x - 1) / blockDim.x : 0;
        const int64_t x0 = per * threadIdx.x, x1 = x0 + per < nx ? x0 + per : (nx > 0 ? nx : 0);
        uint64_t c = 0, at = 0;
        if (FILL) {
            // this thread's first slot: the anchors of the threads before it
            part[threadIdx.x] = tcount[static_cast<uint64_t>(p) * blockDim.x + threadIdx.x];
            __syncthreads();
            if (threadIdx.x == 0) {
                uint64_t run = a.anc_off[p];
                for (int t = 0; t < static_cast<int>(blockDim.x); ++t) {
                    const uint64_t v = part[t];
                    part[t] = run;
                    run += v;
                }
            }
            __syncthreads();
            at = part[threadIdx.x];
        }
        for (int64_t x = x0; x < x1; ++x) {
            uint64_t key = 0;
#pragma unroll
            for (int u = 0; u < kK2; ++u) key = key * 16 + codon_phi(T, L, strand, x + 3 * u);
            // first entry >= key << 13
            const uint64_t want = key << 13;
            int lo = 0, hi = ny;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (pk[mid] < want) lo = mid + 1;
                else hi = mid;
            }
            for (int e = lo; e < ny && (pk[e] >> 13) == key; ++e) {
                if (FILL) a.anc[at++] = (static_cast<uint64_t>(x) << 20) | (pk[e] & 0x1fffu);
                else ++c;
            }
        }
        if (!FILL) {
            tcount[static_cast<uint64_t>(p) * blockDim.x + threadIdx.x] = static_cast<uint32_t>(c);
            part[threadIdx.x] = c;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint64_t sum = 0;
                for (int t = 0; t < static_cast<int>(blockDim.x); ++t) sum += part[t];
                total[p] = sum;
            }
        }
        __syncthreads();
    }
}

// One warp per pair: f of every anchor with g' = 3 dy - dx, then the best chain.
__global__ void refine_chain_kernel(RefineArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t S = kScale;
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < a.n; p += (gridDim.x * blockDim.x) >> 5) {
        const uint64_t b0 = a.anc_off[p];
        const int64_t n = static_cast<int64_t>(a.anc_off[p + 1] - b0);
        if (n > kRefineBig) continue;               // refine_chain_block_kernel's
        const uint64_t *A = a.anc + b0;
        int64_t *F = a.f + b0;
        int32_t *Pr = a.pred + b0;
        // predecessors more than G + 3m bases back have g' <= -G
        const int64_t wx = kG + 3 * static_cast<int64_t>(a.prot_len[p]);
        int64_t lo = 0, bf = INT64_MIN, bi = -1;
        for (int64_t j = 0; j < n; ++j) {
            const int64_t xj = static_cast<int64_t>(A[j] >> 20), yj = static_cast<int64_t>(A[j] & 0xfffffu);
            while (lo < j && static_cast<int64_t>(A[lo] >> 20) < xj - wx) ++lo;
            int64_t best = static_cast<int64_t>(kK2) * S;
            int64_t arg = -1;
            for (int64_t i0 = lo; i0 < j; i0 += 32) {
                const int64_t i = i0 + lane;
                int64_t cand = INT64_MIN;
                if (i < j) {
                    const uint64_t vi = A[i];
                    const int64_t dx = xj - static_cast<int64_t>(vi >> 20);
                    const int64_t dy = yj - static_cast<int64_t>(vi & 0xfffffu);
                    if (dx >= 0 && dy > 0) {
                        const int64_t pen = penalty_eq3(3 * dy - dx, a.log_tab);
                        if (pen >= 0) cand = F[i] + (dy < kK2 ? dy : kK2) * S - pen;
                    }
                }
                // the largest candidate, the first index among equals
                int64_t cv = cand, ci = i;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int64_t oc = __shfl_xor_sync(0xffffffffu, cv, o);
                    const int64_t oi = __shfl_xor_sync(0xffffffffu, ci, o);
                    if (oc > cv || (oc == cv && oi < ci)) {
                        cv = oc;
                        ci = oi;
                    }
                }
                if (cv > best) {
                    best = cv;
                    arg = ci;
                }
            }
            if (lane == 0) {
                F[j] = best;
                Pr[j] = static_cast<int32_t>(arg);
            }
            if (best > bf) {                    // the first anchor with the largest f
                bf = best;
                bi = j;
            }
            __syncwarp();
        }
        if (lane == 0) {
            mp_chain2 c{};
            if (bi >= 0 && Pr[bi] >= 0) {
                int64_t cnt = 0, cur = bi, first = bi;
                while (cur >= 0) {
                    first = cur;
                    ++cnt;
                    cur = Pr[cur];
                }
                c.n_anchors = static_cast<int32_t>(cnt);
                c.score = F[bi];
                c.x_first = static_cast<int64_t>(A[first] >> 20);
                c.x_last = static_cast<int64_t>(A[bi] >> 20);
                c.y_first = static_cast<int64_t>(A[first] & 0xfffffu);
                c.y_last = static_cast<int64_t>(A[bi] & 0xfffffu);
            }
            a.out[p] = c;
        }
        __syncwarp();
    }
}

// The pair's best chain from f and the predecessors (one thread).
__device__ __forceinline__ mp_chain2 best_chain(const uint64_t *A, const int64_t *F, const int32_t *Pr, int64_t bi)
{
    mp_chain2 c{};
    if (bi >= 0 && Pr[bi] >= 0) {
        int64_t cnt = 0, cur = bi, first = bi;
        while (cur >= 0) {
            first = cur;
            ++cnt;
            cur = Pr[cur];
        }
        c.n_anchors = static_cast<int32_t>(cnt);
        c.score = F[bi];
        c.x_first = static_cast<int64_t>(A[first] >> 20);
        c.x_last = static_cast<int64_t>(A[bi] >> 20);
        c.y_first = static_cast<int64_t>(A[first] & 0xfffffu);
        c.y_last = static_cast<int64_t>(A[bi] & 0xfffffu);
    }
    return c;
}

// The same recurrence for the pairs with more than kRefineBig anchors, one
// block per pair: each anchor's predecessors split over the block's
// threads, the best (largest, then first) found by a block reduction.
__global__ void __launch_bounds__(kRefineThreads) refine_chain_block_kernel(RefineArgs a)
{
    __shared__ int64_t rv[kRefineThreads / 32];
    __shared__ int64_t ri[kRefineThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t S = kScale;
    for (uint32_t p = blockIdx.x; p < a.n; p += gridDim.x) {
        const uint64_t b0 = a.anc_off[p];
        const int64_t n = static_cast<int64_t>(a.anc_off[p + 1] - b0);
        if (n <= kRefineBig) continue;              // uniform across the block
        const uint64_t *A = a.anc + b0;
        int64_t *F = a.f + b0;
        int32_t *Pr = a.pred + b0;
        const int64_t wx = kG + 3 * static_cast<int64_t>(a.prot_len[p]);
        int64_t lo = 0, bf = INT64_MIN, bi = -1;
        for (int64_t j = 0; j < n; ++j) {
            const int64_t xj = static_cast<int64_t>(A[j] >> 20), yj = static_cast<int64_t>(A[j] & 0xfffffu);
            while (lo < j && static_cast<int64_t>(A[lo] >> 20) < xj - wx) ++lo;
            int64_t cv = INT64_MIN, ci = INT64_MAX;
            for (int64_t i = lo + threadIdx.x; i < j; i += blockDim.x) {
                const uint64_t vi = A[i];
                const int64_t dx = xj - static_cast<int64_t>(vi >> 20);
                const int64_t dy = yj - static_cast<int64_t>(vi & 0xfffffu);
                if (dx >= 0 && dy > 0) {
                    const int64_t pen = penalty_eq3(3 * dy - dx, a.log_tab);
                    if (pen >= 0) {
                        const int64_t cand = F[i] + (dy < kK2 ? dy : kK2) * S - pen;
                        if (cand > cv) {            // i ascends: the first of equals stays
                            cv = cand;
                            ci = i;
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int64_t oc = __shfl_xor_sync(0xffffffffu, cv, o);
                const int64_t oi = __shfl_xor_sync(0xffffffffu, ci, o);
                if (oc > cv || (oc == cv && oi < ci)) {
                    cv = oc;
                    ci = oi;
                }
            }
            if (lane == 0) {
                rv[warp] = cv;
                ri[warp] = ci;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t best = static_cast<int64_t>(kK2) * S, arg = -1;
                for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
                    if (rv[w] > best || (rv[w] == best && arg >= 0 && ri[w] < arg)) {
                        best = rv[w];
                        arg = ri[w];
                    }
                }
                F[j] = best;
                Pr[j] = static_cast<int32_t>(arg);
                if (best > bf) {
                    bf = best;
                    bi = j;
                }
            }
            __syncthreads();                        // F[j] is read by the next anchors
        }
        if (threadIdx.x == 0) a.out[p] = best_chain(A, F, Pr, bi);
        __syncthreads();
    }
}

}  // namespace
}  // namespace mpdp

// ===================================================================== host
struct mp_index {
    int device = 0;
    uint64_t n_entries = 0;
    uint32_t *off = nullptr;        // kNKeys + 1
    uint32_t *entries = nullptr;
};

namespace {
using namespace mpdp;

// a device allocation freed when it leaves scope
template <typename T>
struct Tmp {
    T *p = nullptr;
    cudaError_t alloc(uint64_t n) { return cudaMalloc(&p, (n ? n : 1) * sizeof(T)); }
    ~Tmp() { if (p) cudaFree(p); }
    Tmp() = default;
    Tmp(const Tmp &) = delete;
    Tmp &operator=(const Tmp &) = delete;
};

#define SCK(x)                                                                         \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA; \
    } while (0)

int grid_for(uint64_t threads, int block)
{
    const uint64_t g = (threads + block - 1) / block;
    return static_cast<int>(g < 65535ull * 16 ? (g ? g : 1) : 65535ull * 16);
}

// exclusive prefix sums of n counts: out[0..n] (out[n] the total)
int scan_counts(const uint32_t *in, uint64_t n, uint32_t *out, cudaStream_t st)
{
    const uint32_t nb = static_cast<uint32_t>((n + kScanBlock * 4 - 1) / (kScanBlock * 4));
    Tmp<uint32_t> sums, total;
    SCK(sums.alloc(nb));
    SCK(total.alloc(1));
    scan_blocks<<<nb ? nb : 1, kScanBlock, 0, st>>>(in, n, out, sums.p);
    scan_sums<<<1, 32, 0, st>>>(sums.p, nb, total.p);
    scan_add<<<grid_for(n, 256), 256, 0, st>>>(out, n, sums.p, total.p);
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(st));
    return MP_OK;
}
}  // namespace

extern "C" int mp_index_build(mp_dp_ctx *ctx, const char *genome, uint64_t len, mp_index **out)
{
    if (!ctx || !out || (len && !genome)) return MP_EINVAL;
    *out = nullptr;
    if (len / 3 >= (1ull << 31)) return MP_EINVAL;          // frame-relative positions and bins are 31-bit
    const int dev = ctx_device(ctx);
    if (cudaSetDevice(dev) != cudaSuccess) return MP_ECUDA;
    cudaStream_t st = ctx_stream(ctx);
    Tmp<char> g;
    SCK(g.alloc(len));
    if (len) SCK(cudaMemcpyAsync(g.p, genome, len, cudaMemcpyHostToDevice, st));
    // the six frames: codons, segments
    Frames fr{};
    uint64_t total = 0, nseg = 0;
    for (int f = 0; f < 6; ++f) {
        const uint64_t frame = f % 3;
        fr.len[f] = len > frame ? (len - frame) / 3 : 0;
        fr.seg0[f] = nseg;
        nseg += (fr.len[f] + kSeg - 1) / kSeg;
        total += fr.len[f];
    }
    fr.seg0[6] = nseg;
    Tmp<uint8_t> codes;
    SCK(codes.alloc(total));
    uint64_t at = 0;
    for (int f = 0; f < 6; ++f) {
        fr.code[f] = codes.p + at;
        at += fr.len[f];
    }
    Tmp<int64_t> first, last, before, after;
    SCK(first.alloc(nseg));
    SCK(last.alloc(nseg));
    SCK(before.alloc(nseg));
    SCK(after.alloc(nseg));
    Tmp<uint32_t> count, cursor;
    SCK(count.alloc(kNKeys));
    SCK(cursor.alloc(kNKeys + 1));
    SCK(cudaMemsetAsync(count.p, 0, kNKeys * sizeof(uint32_t), st));
    if (total) {
        translate_kernel<<<grid_for(total, 256), 256, 0, st>>>(g.p, len, fr);
        segment_kernel<<<grid_for(nseg * 32, 256), 256, 0, st>>>(fr, first.p, last.p, nseg);
        segment_scan<<<6, kScanThreads, 0, st>>>(fr, first.p, last.p, before.p, after.p);
        kmer_kernel<<<grid_for(nseg * 32, kKmerWarps * 32), kKmerWarps * 32, 0, st>>>(
            fr, before.p, after.p, nseg, 0, count.p, nullptr, nullptr);
        SCK(cudaGetLastError());
    }
    mp_index *idx = new (std::nothrow) mp_index();
    if (!idx) return MP_ENOMEM;
    idx->device = dev;
    auto fail = [&](int rc) {
        mp_index_free(idx);
        return rc;
    };
    if (cudaMalloc(&idx->off, (kNKeys + 1ull) * sizeof(uint32_t)) != cudaSuccess) return fail(MP_ENOMEM);
    int rc = scan_counts(count.p, kNKeys, idx->off, st);
    if (rc != MP_OK) return fail(rc);
    uint32_t n_entries = 0;
    if (cudaMemcpy(&n_entries, idx->off + kNKeys, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(MP_ECUDA);
    idx->n_entries = n_entries;
    if (cudaMalloc(&idx->entries, (n_entries ? n_entries : 1) * sizeof(uint32_t)) != cudaSuccess)
        return fail(MP_ENOMEM);
    if (total) {
        if (cudaMemcpyAsync(cursor.p, idx->off, kNKeys * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return fail(MP_ECUDA);
        kmer_kernel<<<grid_for(nseg * 32, kKmerWarps * 32), kKmerWarps * 32, 0, st>>>(
            fr, before.p, after.p, nseg, 1, nullptr, cursor.p, idx->entries);
        bucket_sort_kernel<<<grid_for(kNKeys, 256), 256, 0, st>>>(idx->off, idx->entries);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return fail(MP_ECUDA);
    *out = idx;
    return MP_OK;
}

extern "C" int mp_index_download(mp_dp_ctx *ctx, const mp_index *idx, uint64_t *offsets, uint32_t *entries,
                                 uint64_t *n_entries)
{
    if (!ctx || !idx || !n_entries || (!offsets) != (!entries)) return MP_EINVAL;
    if (cudaSetDevice(idx->device) != cudaSuccess) return MP_ECUDA;
    *n_entries = idx->n_entries;
    if (!offsets) return MP_OK;
    std::vector<uint32_t> off(kNKeys + 1ull);
    if (cudaMemcpy(off.data(), idx->off, off.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (idx->n_entries && cudaMemcpy(entries, idx->entries, idx->n_entries * sizeof(uint32_t),
                                      cudaMemcpyDeviceToHost) != cudaSuccess))
        return MP_ECUDA;
    for (size_t h = 0; h < off.size(); ++h) offsets[h] = off[h];
    return MP_OK;
}

extern "C" void mp_index_free(mp_index *idx)
{
    if (!idx) return;
    cudaSetDevice(idx->device);
    if (idx->off) cudaFree(idx->off);
    if (idx->entries) cudaFree(idx->entries);
    delete idx;
}

extern "C" int mp_index_chain(mp_dp_ctx *ctx, const mp_index *idx, const char *prot, const uint64_t *prot_off,
                              const uint32_t *prot_len, uint32_t n_prot, int32_t top, mp_chain *chains,
                              uint32_t *n_chains)
{
    if (!ctx || !idx || top < 1 || (n_prot && (!prot || !prot_off || !prot_len || !chains || !n_chains)))
        return MP_EINVAL;
    if (n_prot == 0) return MP_OK;
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess || idx->device != ctx_device(ctx)) return MP_ECUDA;
    cudaStream_t st = ctx_stream(ctx);
    uint64_t span = 0;
    for (uint32_t k = 0; k < n_prot; ++k) {
        if (prot_len[k] >= (1u << 20)) return MP_EINVAL;         // residue positions are 20-bit in the anchor keys
        span = std::max<uint64_t>(span, prot_off[k] + prot_len[k]);
    }
    Tmp<char> d_prot;
    Tmp<uint64_t> d_off, d_cnt, d_anc_off;
    Tmp<uint32_t> d_len, d_nch;
    Tmp<mp_chain> d_ch;
    SCK(d_prot.alloc(span));
    SCK(d_off.alloc(n_prot));
    SCK(d_len.alloc(n_prot));
    SCK(d_cnt.alloc(n_prot));
    SCK(d_anc_off.alloc(n_prot + 1ull));
    SCK(d_nch.alloc(n_prot));
    SCK(d_ch.alloc(static_cast<uint64_t>(n_prot) * top));
    SCK(cudaMemcpyAsync(d_prot.p, prot, span, cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_off.p, prot_off, n_prot * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_len.p, prot_len, n_prot * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    Tmp<int32_t> d_log;
    SCK(d_log.alloc(kG));
    SCK(cudaFuncSetAttribute(anchor_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSortMax * sizeof(uint64_t))));
    log_table_kernel<<<grid_for(kG, 256), 256, 0, st>>>(d_log.p);
    ChainArgs a{};
    a.log_tab = d_log.p;
    a.prot = d_prot.p;
    a.prot_off = d_off.p;
    a.prot_len = d_len.p;
    a.n_prot = n_prot;
    a.off = idx->off;
    a.entries = idx->entries;
    a.top = top;
    a.chains = d_ch.p;
    a.n_chains = d_nch.p;
    anchor_count_kernel<<<grid_for(n_prot * 32ull, 256), 256, 0, st>>>(a, d_cnt.p);
    SCK(cudaGetLastError());
    std::vector<uint64_t> cnt(n_prot);
    SCK(cudaMemcpyAsync(cnt.data(), d_cnt.p, n_prot * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    // proteins in groups whose anchors (8 + 8 + 4 + 1 bytes each, plus the
    // sort scratch of large ones) stay within a bound
    constexpr uint64_t kMaxAnchors = 192ull << 20;
    std::vector<mp_chain> h_ch(static_cast<uint64_t>(n_prot) * top);
    std::vector<uint32_t> h_nch(n_prot);
    for (uint32_t p0 = 0; p0 < n_prot;) {
        uint32_t p1 = p0;
        uint64_t tot = 0;
        while (p1 < n_prot && (p1 == p0 || tot + cnt[p1] <= kMaxAnchors)) tot += cnt[p1++];
        const uint32_t np = p1 - p0;
        std::vector<uint64_t> aoff(np + 1ull, 0), soff(np, 0);
        uint64_t scratch = 0;
        for (uint32_t k = 0; k < np; ++k) {
            aoff[k + 1] = aoff[k] + cnt[p0 + k];
            uint64_t n2 = 1;
            while (n2 < cnt[p0 + k]) n2 <<= 1;
            soff[k] = scratch;
            if (n2 > static_cast<uint64_t>(kSortMax)) scratch += n2;
        }
        Tmp<uint64_t> anc, sc, d_soff;
        Tmp<int64_t> f;
        Tmp<int32_t> pred;
        Tmp<uint8_t> used;
        SCK(anc.alloc(tot));
        SCK(f.alloc(tot));
        SCK(pred.alloc(tot));
        SCK(used.alloc(tot));
        SCK(sc.alloc(scratch));
        SCK(d_soff.alloc(np));
        SCK(cudaMemcpyAsync(d_anc_off.p, aoff.data(), (np + 1ull) * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        SCK(cudaMemcpyAsync(d_soff.p, soff.data(), np * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        ChainArgs b = a;
        b.prot_off = d_off.p + p0;
        b.prot_len = d_len.p + p0;
        b.n_prot = np;
        b.anc_off = d_anc_off.p;
        b.anc = anc.p;
        b.f = f.p;
        b.pred = pred.p;
        b.used = used.p;
        b.chains = d_ch.p + static_cast<uint64_t>(p0) * top;
        b.n_chains = d_nch.p + p0;
        anchor_fill_kernel<<<grid_for(np * 32ull, 256), 256, 0, st>>>(b);
        anchor_sort_kernel<<<np < 65535u * 4 ? np : 65535u * 4, kSortThreads, kSortMax * sizeof(uint64_t), st>>>(
            b, sc.p, d_soff.p);
        chain_kernel<<<grid_for(np * 32ull, 128), 128, 0, st>>>(b);
        SCK(cudaGetLastError());
        SCK(cudaStreamSynchronize(st));
        p0 = p1;
    }
    SCK(cudaMemcpyAsync(chains, d_ch.p, static_cast<uint64_t>(n_prot) * top * sizeof(mp_chain),
                        cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(n_chains, d_nch.p, n_prot * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    return MP_OK;
}

extern "C" int mp_chain_refine(mp_dp_ctx *ctx, const mp_pair *pairs, size_t n, mp_chain2 *out)
{
    if (!ctx || (n && (!pairs || !out))) return MP_EINVAL;
    if (n == 0) return MP_OK;
    if (n >= (1ull << 31)) return MP_EINVAL;
    // every pair's protein and region, one after the other
    std::vector<uint64_t> poff(n), toff(n);
    std::vector<uint32_t> plen(n), tlen(n);
    std::vector<int8_t> strand(n);
    uint64_t tot = 0;
    for (size_t k = 0; k < n; ++k) {
        const mp_pair &q = pairs[k];
        // (a thread's anchor count, at most its bases times the protein's
        // k-mers, is 32-bit)
        if ((q.prot_len && !q.prot) || (q.nt_len && !q.nt) || q.prot_len > static_cast<uint32_t>(kRefineMaxProt) ||
            (q.strand != 1 && q.strand != -1) ||
            (static_cast<uint64_t>(q.nt_len) / kRefineThreads + 1) * q.prot_len >= (1ull << 32))
            return MP_EINVAL;
        poff[k] = tot;
        tot += q.prot_len;
        toff[k] = tot;
        tot += q.nt_len;
        plen[k] = q.prot_len;
        tlen[k] = q.nt_len;
        strand[k] = q.strand;
    }
    std::vector<char> h(tot ? tot : 1);
    for (size_t k = 0; k < n; ++k) {
        if (plen[k]) memcpy(h.data() + poff[k], pairs[k].prot, plen[k]);
        if (tlen[k]) memcpy(h.data() + toff[k], pairs[k].nt, tlen[k]);
    }
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return MP_ECUDA;
    cudaStream_t st = ctx_stream(ctx);
    Tmp<char> d_seq;
    Tmp<uint64_t> d_poff, d_toff, d_cnt, d_aoff;
    Tmp<uint32_t> d_tcnt;
    Tmp<uint32_t> d_plen, d_tlen;
    Tmp<int8_t> d_strand;
    Tmp<int32_t> d_log;
    Tmp<mp_chain2> d_out;
    SCK(d_seq.alloc(tot));
    SCK(d_poff.alloc(n));
    SCK(d_toff.alloc(n));
    SCK(d_plen.alloc(n));
    SCK(d_tlen.alloc(n));
    SCK(d_strand.alloc(n));
    SCK(d_cnt.alloc(n));
    SCK(d_tcnt.alloc(static_cast<uint64_t>(n) * kRefineThreads));
    SCK(d_aoff.alloc(n + 1));
    SCK(d_log.alloc(kG));
    SCK(d_out.alloc(n));
    SCK(cudaMemcpyAsync(d_seq.p, h.data(), tot, cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_poff.p, poff.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_toff.p, toff.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_plen.p, plen.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_tlen.p, tlen.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_strand.p, strand.data(), n, cudaMemcpyHostToDevice, st));
    log_table_kernel<<<grid_for(kG, 256), 256, 0, st>>>(d_log.p);
    RefineArgs a{};
    a.seq = d_seq.p;
    a.prot_off = d_poff.p;
    a.nt_off = d_toff.p;
    a.prot_len = d_plen.p;
    a.nt_len = d_tlen.p;
    a.strand = d_strand.p;
    a.log_tab = d_log.p;
    const uint32_t nb = static_cast<uint32_t>(n < 65535ull * 8 ? n : 65535ull * 8);
    SCK(cudaFuncSetAttribute(refine_anchor_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kRefineSmem)));
    SCK(cudaFuncSetAttribute(refine_anchor_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kRefineSmem)));
    refine_anchor_kernel<false><<<nb, kRefineThreads, kRefineSmem, st>>>(RefineArgs{a.seq, a.prot_off, a.nt_off, a.prot_len,
                                                                          a.nt_len, a.strand, static_cast<uint32_t>(n)},
                                                               d_tcnt.p, d_cnt.p);
    SCK(cudaGetLastError());
    std::vector<uint64_t> per(n);
    SCK(cudaMemcpyAsync(per.data(), d_cnt.p, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    // pairs in groups whose anchors (8 + 8 + 4 bytes each) stay within a bound
    constexpr uint64_t kMaxAnchors = 192ull << 20;
    std::vector<mp_chain2> h_out(n);
    for (size_t p0 = 0; p0 < n;) {
        size_t p1 = p0;
        uint64_t na = 0;
        while (p1 < n && (p1 == p0 || na + per[p1] <= kMaxAnchors)) na += per[p1++];
        const uint32_t np = static_cast<uint32_t>(p1 - p0);
        std::vector<uint64_t> aoff(np + 1ull, 0);
        for (uint32_t k = 0; k < np; ++k) aoff[k + 1] = aoff[k] + per[p0 + k];
        Tmp<uint64_t> anc;
        Tmp<int64_t> f;
        Tmp<int32_t> pred;
        SCK(anc.alloc(na));
        SCK(f.alloc(na));
        SCK(pred.alloc(na));
        SCK(cudaMemcpyAsync(d_aoff.p, aoff.data(), (np + 1ull) * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        RefineArgs b = a;
        b.seq = d_seq.p;
        b.prot_off = d_poff.p + p0;
        b.nt_off = d_toff.p + p0;
        b.prot_len = d_plen.p + p0;
        b.nt_len = d_tlen.p + p0;
        b.strand = d_strand.p + p0;
        b.n = np;
        b.anc_off = d_aoff.p;
        b.anc = anc.p;
        b.f = f.p;
        b.pred = pred.p;
        b.out = d_out.p + p0;
        const uint32_t gb = np < 65535u * 8 ? np : 65535u * 8;
        refine_anchor_kernel<true><<<gb, kRefineThreads, kRefineSmem, st>>>(b, d_tcnt.p + p0 * kRefineThreads,
                                                                             nullptr);
        refine_chain_kernel<<<grid_for(np * 32ull, 128), 128, 0, st>>>(b);
        refine_chain_block_kernel<<<gb, kRefineThreads, 0, st>>>(b);
        SCK(cudaGetLastError());
        SCK(cudaStreamSynchronize(st));
        p0 = p1;
    }
    SCK(cudaMemcpyAsync(out, d_out.p, n * sizeof(mp_chain2), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    return MP_OK;
}

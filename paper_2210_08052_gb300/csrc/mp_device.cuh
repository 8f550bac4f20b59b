// Device helpers shared by the DP and traceback kernels: the genetic code,
// the final splice model (Li 2022, Methods, "Splice models") and the
// substitution score of Eq. 6 / Eq. 7.
#pragma once
#include <cstdint>

#include "mp_internal.cuh"

namespace mpdp {
namespace {

constexpr char kAAOrder[] = "ARNDCQEGHILKMFPSTWYV*";
// NCBI table 1 with codons enumerated as A, C, G, T in each position.
constexpr char kCodeACGT[] = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF";

constexpr int aa_index(char c)
{
    for (int k = 0; k < 21; ++k)
        if (kAAOrder[k] == c) return k;
    return 21;
}

struct CodeTable {
    int8_t v[64];
};

constexpr CodeTable make_code_table()
{
    CodeTable t{};
    for (int k = 0; k < 64; ++k) t.v[k] = static_cast<int8_t>(aa_index(kCodeACGT[k]));
    return t;
}

__constant__ CodeTable c_code = make_code_table();

// Bases: 0 A, 1 C, 2 G, 3 T; v* false = outside T, which matches no motif.
__device__ __forceinline__ int donor_score(int b1, int b2, int b3, bool v1, bool v2, bool v3)
{
    // d(x) from T[x+1..x+3]: GT[AG] 0, GT[CT] 8, GC 15, AT 21, else 30
    if (v1 && v2) {
        if (b1 == 2 && b2 == 3) {
            if (v3) return (b3 == 0 || b3 == 2) ? 0 : 8;
            return 30;
        }
        if (b1 == 2 && b2 == 1) return 15;
        if (b1 == 0 && b2 == 3) return 21;
    }
    return 30;
}

__device__ __forceinline__ int acceptor_score(int b1, int b2, int b3, bool v1, bool v2, bool v3)
{
    // a(x) from T[x-2..x]: [CT]AG 0, [AG]AG 8, AC (last two) 21, else 30
    if (v2 && v3 && b2 == 0) {
        if (b3 == 2) {
            if (!v1) return 30;
            return (b1 == 1 || b1 == 3) ? 0 : 8;
        }
        if (b3 == 1) return 21;
    }
    return 30;
}

// d(x) and a(x) under the parameters' splice model; for the simple model
// (defined right after Eq. 7) a donor needs GT at T[x+1..x+2] and an
// acceptor AG at T[x-1..x], else they cost splice_p.  Arguments as above.
__device__ __forceinline__ int splice_donor(const ScoreParams &sp, int b1, int b2, int b3, bool v1, bool v2,
                                            bool v3)
{
    if (sp.splice_model == MP_SPLICE_SIMPLE) return (v1 && v2 && b1 == 2 && b2 == 3) ? 0 : sp.splice_p;
    return donor_score(b1, b2, b3, v1, v2, v3);
}

__device__ __forceinline__ int splice_acceptor(const ScoreParams &sp, int b1, int b2, int b3, bool v1, bool v2,
                                               bool v3)
{
    if (sp.splice_model == MP_SPLICE_SIMPLE) return (v2 && v3 && b2 == 0 && b3 == 2) ? 0 : sp.splice_p;
    return acceptor_score(b1, b2, b3, v1, v2, v3);
}

__device__ __forceinline__ int subst_score(const ScoreParams &sp, int aa, int pc)
{
    if (aa == 21) return -512;             // no complete codon (i < 3)
    if (aa == 20) return -sp.stop;         // stop codon against any residue
    return sp.mat[aa][pc];
}

}  // namespace
}  // namespace mpdp

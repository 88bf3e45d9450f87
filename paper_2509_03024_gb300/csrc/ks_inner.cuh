// ks_inner.cuh — the key inner product of hybrid key switching (K3 of ks.cu) and its launch
// variants. Every variant computes the same exact 128-bit sums and reduces them once, so every
// variant gives the same bits; they differ in how the 64 x 64 -> 128-bit multiply-accumulates are
// formulated and in how many items one thread serves (items that share a key share its loads).
#pragma once

#include "core.cuh"

namespace fhe {

// Evaluation slot k holds a(psi^(2 brev(k) + 1)); X -> X^g moves slot k' to slot k
// with 2 brev(k') + 1 = g (2 brev(k) + 1) mod 2N.
__device__ __forceinline__ int auto_src(int k, int g, int log_n) {
    const unsigned sh = 32 - log_n;
    unsigned bk = __brev((unsigned)k) >> sh;
    unsigned e = (unsigned)(((unsigned long long)g * (2ull * bk + 1ull)) & ((2ull << log_n) - 1ull));
    return (int)(__brev((e - 1u) >> 1) >> sh);
}

// One rotation of a hoisted rotate-and-sum, as the kernel reads it from a device table.
struct HoistStep {
    const u64* key;
    long long galois;
};

struct InnerArgs {
    u64* acc;                 // [items][2][next][N]
    u64* c0sum;               // hoisted: [items][l1][N] c0 + sum_r phi_r(c0)
    const u64* ext;           // [sources][dn][next][N] raised digits (own-digit limbs unused)
    const KsItem* tab;        // device item table
    const int* src_of;        // fan-out: source of each item
    const HoistStep* steps;   // hoisted: device table of the rotations
    int n_steps;
    int items, dn, alpha, next, level, L, n_ext, log_n;
    const Prime* pr;
    const u64* shared_key;    // plain: non-null when every item uses this key ...
    long long shared_galois;  // ... and this automorphism (then several items per thread may run)
    int split25;              // set by the launchers: data limbs use the split-at-bit-25 sums
    int keys_packed;          // the keys' data-prime rows, and the raised digits' data limbs (ext rows
                              // x <= level), are stored split at bit 25 (key_unpack); the own-digit
                              // rows read from the input are not
};

// A data-prime key residue stored split at bit 25 (every data prime below 2^50): the low 25 bits in
// the low 32-bit word, the rest in the high word, so that the column-sum multiply-accumulate takes
// the two halves without any unpacking. Every other use unpacks it.
__host__ __device__ __forceinline__ u64 key_pack(u64 k) { return (k & ((1ull << 25) - 1)) | ((k >> 25) << 32); }
__host__ __device__ __forceinline__ u64 key_unpack(u64 k) { return (k & 0xFFFFFFFFull) | ((k >> 32) << 25); }

// Launch variants (the autotuner times them; all give identical bits).
enum InnerVariant {
    INNER_V0 = 0,   // one coefficient pair per thread, grid-stride over (limb, item, pair)
    INNER_C1,       // 2-D grid (pair, item group) x limb; C halves + carry compare; 1 item per thread
    INNER_P1,       // ... 32-bit schoolbook carry chain; 1 item per thread
    INNER_S1,       // ... data limbs split at bit 25 into carry-free column sums, special limbs P32
    INNER_S2,       // S1 with 2 items per thread sharing the key loads (plain: when the items share a key)
    INNER_S2L,      // S2 reading each permuted residue with its own 64-bit load instead of a pair load and
                    // two selects (hoisted only; the plain kernel runs S2)
    INNER_N_VARIANTS
};
extern const char* const kInnerVariantNames[INNER_N_VARIANTS];

// K3 of a plain or fan-out key switch. Falls back to one item per thread when the items do not share
// a key, and to the 32-bit schoolbook form on data limbs whose primes exceed 50 bits.
void launch_ks_inner(const InnerArgs& a, bool fanout, int variant, int max_data_prime_bits, cudaStream_t s);
// K3 of a hoisted rotate-and-sum.
void launch_ks_hoist_inner(const InnerArgs& a, int variant, int max_data_prime_bits, cudaStream_t s);

}  // namespace fhe

// ntt_core.cuh — butterfly arithmetic and the register-blocked tile stages
// shared by the plain NTT launches (ntt.cu) and the fused key-switch passes
// (ks.cu). See ntt.cu for the decomposition and the lazy value ranges.
#pragma once

#include "core.cuh"

namespace fhe {
namespace nttc {

// Residues per thread of the plain two-pass NTT tiles: 2^kTileRB (register blocks of kTileRB
// stages). Radix-16 blocks halve the shared-memory exchanges of the plain transform (1 GiB
// forward at N = 2^15: 1.71 -> 1.52 ms; inverse 1.93 -> 1.74 ms).
constexpr int kTileRB = 4;

// Shoup product without the final correction: a * w mod q in [0, 2q) for any a < 2^64.
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 ws, u64 q) {
    u64 qh = __umul64hi(a, ws);
    return a * w - qh * q;
}

// Forward CT butterfly: X <- X + W Y, Y <- X - W Y with W Y in [0, 2q) (lazy).
// RED: inputs in [0, 4q), X first reduced below 2q, outputs in [0, 4q).
// !RED: no reduction; each stage adds less than 2q, so after s stages from [0, q)
//       values are below (2s + 1) q (used for q < 2^58 and at most 16 stages).
template <bool RED>
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, u64 w, u64 ws, u64 q, u64 q2) {
    u64 a = RED ? (x >= q2 ? x - q2 : x) : x;
    u64 t = shoup_lazy(y, w, ws, q);
    x = a + t;
    y = a + q2 - t;
}

// Any 64-bit value reduced to [0, q): a lazy Shoup product by 1, then one correction.
__device__ __forceinline__ u64 reduce_any(u64 x, u64 q, u64 one_s) {
    u64 t = x - __umul64hi(x, one_s) * q;
    return t >= q ? t - q : t;
}

// Inverse GS butterfly on values in [0, 2q): X <- X + Y, Y <- (X - Y) W (outputs in [0, 2q)).
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, u64 w, u64 ws, u64 q, u64 q2) {
    u64 s = x + y;
    s = s >= q2 ? s - q2 : s;
    u64 d = x + q2 - y;
    x = s;
    y = shoup_lazy(d, w, ws, q);
}

__device__ __forceinline__ u64 reduce4(u64 x, u64 q) {
    u64 q2 = q << 1;
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

// Element x (within its sub-transform) that register u of the 2^RB-element group g holds in
// radix-2^RB block blk (block blk covers stages [RB blk, min(RB blk + RB, LOGM))).
template <int LOGM, int RB = 3>
__device__ __forceinline__ int block_elem(int blk, int g, int u) {
    constexpr int M = 1 << LOGM;
    const int s0 = RB * blk;
    const int b = (LOGM - s0) < RB ? (LOGM - s0) : RB;
    const int d = M >> (s0 + b);
    return (g / d) * ((1 << RB) * d) + (g % d) + u * d;
}

// Butterfly stages of one tile: R sub-transforms of M = 2^LOGM points, element x of
// sub-transform q at sm[x * P + q] between register blocks. Each thread owns V = 2^RB values and
// runs RB stages in registers per block. PASS 0: column transforms (stages [0, LOGM), twiddles
// W[2^s + group]); PASS 1: row transforms (stages [S1, S1 + LOGM), transposed twiddles, tile
// rows t0..t0+R-1).
// IN_REG: the first block takes its values from v (the caller loaded the elements
// block_elem(first block, g, u) from global memory) instead of from sm; otherwise the caller
// fills sm and synchronises before. OUT_REG: the last block leaves its values in v (elements
// block_elem(last block, g, u)) and neither stores nor synchronises; otherwise the result is in
// sm after a final __syncthreads(). The first block is 0 (forward) or NB - 1 (inverse).
template <int LOGM, int R, bool INV, int PASS, bool RED = true, bool IN_REG = false, bool OUT_REG = false,
          int RB = 3>
__device__ __forceinline__ void tile_stages(u64* sm, const ulonglong2* __restrict__ W, u64 q, int S1, int t0,
                                            u64 (&v)[1 << RB]) {
    constexpr int M = 1 << LOGM;
    constexpr int V = 1 << RB;
    constexpr int P = R == 1 ? 1 : R + 1;
    const int tid = threadIdx.x;
    const u64 q2 = q << 1;
    const int qq = tid % R;  // sub-transform of this thread
    const int g = tid / R;   // V-element group within the sub-transform
    const int row_off = PASS == 1 ? t0 + qq : 0;

    // register blocks of stages; forward runs stages 0..LOGM-1, inverse LOGM-1..0
    constexpr int NB = (LOGM + RB - 1) / RB;
#pragma unroll
    for (int bi = 0; bi < NB; bi++) {
        // forward: block bi covers stages [RB bi, min(RB bi + RB, LOGM));
        // inverse: the same blocks in reverse order, stages inside a block descending
        const int blk_id = INV ? NB - 1 - bi : bi;
        const int s0 = RB * blk_id;
        const int b = (LOGM - s0) < RB ? (LOGM - s0) : RB;
        const int d = M >> (s0 + b);
        const int base = (g / d) * (V * d) + (g % d);
        if (!(IN_REG && bi == 0)) {
#pragma unroll
            for (int u = 0; u < V; u++) v[u] = sm[(base + u * d) * P + qq];
        }
        // Twiddle of the pair (u, u + dist) at block stage j: its group index at stage s0 + j is
        // tb * 2^j + (u >> (b - j)), with tb = base >> (LOGM - s0) the thread's group at s0.
        const int tb = base >> (LOGM - s0);
        if (!INV) {
#pragma unroll
            for (int j = 0; j < RB; j++) {
                if (j >= b) break;
                const int s = s0 + j;
                const int dist = 1 << (b - 1 - j);
#pragma unroll
                for (int u = 0; u < V; u++) {
                    if (u & dist) continue;
                    const int grp = (tb << j) + (u >> (b - j));
                    const int wi = PASS == 1 ? ((((1 << s) - 1 + grp)) << S1) + row_off : (1 << s) + grp;
                    const ulonglong2 w = W[wi];
                    ct_bfly<RED>(v[u], v[u + dist], w.x, w.y, q, q2);
                }
            }
        } else {
#pragma unroll
            for (int j = RB - 1; j >= 0; j--) {
                if (j >= b) continue;
                const int s = s0 + j;
                const int dist = 1 << (b - 1 - j);
#pragma unroll
                for (int u = 0; u < V; u++) {
                    if (u & dist) continue;
                    const int grp = (tb << j) + (u >> (b - j));
                    const int wi = PASS == 1 ? ((((1 << s) - 1 + grp)) << S1) + row_off : (1 << s) + grp;
                    const ulonglong2 w = W[wi];
                    gs_bfly(v[u], v[u + dist], w.x, w.y, q, q2);
                }
            }
        }
        if (!(OUT_REG && bi == NB - 1)) {
#pragma unroll
            for (int u = 0; u < V; u++) sm[(base + u * d) * P + qq] = v[u];
            __syncthreads();
        }
    }
}

template <int LOGM, int R, bool INV, int PASS, bool RED = true, int RB = 3>
__device__ __forceinline__ void tile_stages(u64* sm, const ulonglong2* __restrict__ W, u64 q, int S1, int t0) {
    u64 v[1 << RB];
    tile_stages<LOGM, R, INV, PASS, RED, false, false, RB>(sm, W, q, S1, t0, v);
}

}  // namespace nttc
}  // namespace fhe

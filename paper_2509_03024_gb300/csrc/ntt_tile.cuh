// ntt_tile.cuh — the plain NTT tile kernel and its launcher, shared by the tile-shape variants
// (ntt.cu, ntt_tiles.cu). See ntt.cu for the decomposition and the lazy value ranges.
#pragma once

#include "ntt_core.cuh"

namespace fhe {

namespace ntt_tile {

using nttc::reduce4;
using nttc::shoup_lazy;

struct RowPtr {
    u64* p;
    int prime;
};

__device__ __forceinline__ RowPtr row_ptr(const PolyBatch& pb, int row, int log_n) {
    int li = row % pb.n_limbs;
    int rest = row / pb.n_limbs;
    int part = rest % pb.n_parts;
    int item = rest / pb.n_parts;
    int limb = pb.limb_lo + li;
    RowPtr r;
    r.p = pb.base + (size_t)item * pb.item_stride + (size_t)part * pb.part_stride +
          ((size_t)(limb - pb.addr_lo) << log_n);
    r.prime = pb.prime_of(limb);
    return r;
}

// One tile: R sub-transforms of M = 2^LOGM points.
// PASS 0: column transforms (stages [0, LOGM) of the full ring), tile = R consecutive columns;
//         with LOGM = log N and R = 1 this is the whole single-pass transform.
// PASS 1: row transforms (stages [S1, log N)), tile = R consecutive rows of M = N2 points.
// LAST: this kernel performs the final stages (reduce to [0, q); inverse: times N^-1).
// Each thread owns 2^RB residues (RB = 3: radix-8 register blocks, RB = 4: radix-16).
template <int LOGM, int RB>
constexpr int tile_min_blocks(int threads) {
    return (RB == 3 ? 1024 : 768) / threads > 0 ? (RB == 3 ? 1024 : 768) / threads : 1;
}

template <int LOGN, int LOGM, int R, bool INV, int PASS, bool LAST, int RB = 3>
__global__ void __launch_bounds__(R * (1 << LOGM) / (1 << RB), tile_min_blocks<LOGM, RB>(R * (1 << LOGM) / (1 << RB)))
ntt_tile_kernel(PolyBatch pb, const Prime* __restrict__ primes, const ulonglong2* __restrict__ tw,
                const u64* __restrict__ ninv) {
    constexpr int log_n = LOGN;  // the ring size is a compile-time constant of each launch
    constexpr int M = 1 << LOGM;
    constexpr int P = R == 1 ? 1 : R + 1;
    constexpr int V = 1 << RB;
    constexpr int T = R * M / V;
    extern __shared__ u64 sm[];
    const int tid = threadIdx.x;
    const RowPtr rp = row_ptr(pb, blockIdx.x, log_n);
    const u64 q = primes[rp.prime].q;
    const ulonglong2* W = tw + ((size_t)rp.prime << log_n);
    const int log_n2 = PASS == 0 ? log_n - LOGM : LOGM;  // row length of the N1 x N2 view
    const int S1 = log_n - log_n2;                       // column stages
    const int t0 = blockIdx.y * R;                       // first column (PASS 0) or row (PASS 1)
    const u64 ni = ninv[2 * rp.prime], nis = ninv[2 * rp.prime + 1];

    if (PASS == 0 && R > 1) {
        // column tiles: the first and last register blocks read and write global memory directly
        // (a warp covers 16 consecutive columns of two rows per access)
        constexpr int NB = (LOGM + RB - 1) / RB;
        const int qq = tid % R, g = tid / R;
        const int fb = INV ? NB - 1 : 0, lb = INV ? 0 : NB - 1;
        u64 v[V];
#pragma unroll
        for (int u = 0; u < V; u++)
            v[u] = rp.p[(size_t)(t0 + qq) + ((size_t)nttc::block_elem<LOGM, RB>(fb, g, u) << log_n2)];
        if (!INV && q < ((u64)1 << 58))
            nttc::tile_stages<LOGM, R, INV, PASS, false, true, true, RB>(sm, W, q, S1, t0, v);
        else
            nttc::tile_stages<LOGM, R, INV, PASS, true, true, true, RB>(sm, W, q, S1, t0, v);
        const u64 one_s = primes[rp.prime].one_s;
#pragma unroll
        for (int u = 0; u < V; u++) {
            u64 val = v[u];
            if (LAST) {
                if (INV) {
                    u64 r = shoup_lazy(val, ni, nis, q);
                    val = r >= q ? r - q : r;
                } else {
                    val = nttc::reduce_any(val, q, one_s);
                }
            }
            rp.p[(size_t)(t0 + qq) + ((size_t)nttc::block_elem<LOGM, RB>(lb, g, u) << log_n2)] = val;
        }
        return;
    }

    // load (coalesced), values enter in [0, q)
    if (PASS == 0) {
#pragma unroll 4
        for (int e = tid; e < R * M; e += T) {
            int x = e / R, qq = e % R;
            sm[x * P + qq] = rp.p[(size_t)(t0 + qq) + ((size_t)x << log_n2)];
        }
    } else {
#pragma unroll 4
        for (int e = tid; e < R * M; e += T) {
            int x = e & (M - 1), qq = e >> LOGM;
            sm[x * P + qq] = rp.p[((size_t)(t0 + qq) << LOGM) + x];
        }
    }
    __syncthreads();

    // forward transforms of primes below 2^58 skip the per-butterfly reduction (values < 33 q)
    if (!INV && q < ((u64)1 << 58)) nttc::tile_stages<LOGM, R, INV, PASS, false, RB>(sm, W, q, S1, t0);
    else nttc::tile_stages<LOGM, R, INV, PASS, true, RB>(sm, W, q, S1, t0);
    const u64 one_s = primes[rp.prime].one_s;

    // store (coalesced)
    if (PASS == 0) {
#pragma unroll 4
        for (int e = tid; e < R * M; e += T) {
            int x = e / R, c = e % R;
            u64 val = sm[x * P + c];
            if (LAST) {
                if (INV) {
                    u64 r = shoup_lazy(val, ni, nis, q);
                    val = r >= q ? r - q : r;
                } else {
                    val = nttc::reduce_any(val, q, one_s);
                }
            }
            rp.p[(size_t)(t0 + c) + ((size_t)x << log_n2)] = val;
        }
    } else {
#pragma unroll 4
        for (int e = tid; e < R * M; e += T) {
            int x = e & (M - 1), r = e >> LOGM;
            u64 val = sm[x * P + r];
            if (LAST) {
                if (INV) {
                    u64 t = shoup_lazy(val, ni, nis, q);
                    val = t >= q ? t - q : t;
                } else {
                    val = nttc::reduce_any(val, q, one_s);
                }
            }
            rp.p[((size_t)(t0 + r) << LOGM) + x] = val;
        }
    }
}

template <int LOGN, int LOGM, int R, bool INV, int PASS, bool LAST, int RB = nttc::kTileRB>
void launch_tile(const Ctx& c, const PolyBatch& pb, int tiles, cudaStream_t s, double bytes) {
    constexpr int T = R * (1 << LOGM) / (1 << RB);
    constexpr size_t smem = sizeof(u64) * (1 << LOGM) * (R == 1 ? 1 : R + 1);
    // row passes read the transposed [stage][group][row] tables
    const ulonglong2* tw = PASS == 1 ? (INV ? c.d_itw2 : c.d_tw2) : (INV ? c.d_itw : c.d_tw);
    if (smem > 48 * 1024)
        CK(cudaFuncSetAttribute(ntt_tile_kernel<LOGN, LOGM, R, INV, PASS, LAST, RB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // this pass runs LOGM butterfly stages over every row: N/2 butterflies per stage
    LaunchScope _ls(c.prof, INV ? K_NTT_INV : K_NTT_FWD, bytes, s, (double)pb.rows() * ((size_t)1 << (c.log_n - 1)) * LOGM);
    ntt_tile_kernel<LOGN, LOGM, R, INV, PASS, LAST, RB><<<dim3(pb.rows(), tiles), T, smem, s>>>(pb, c.d_primes, tw,
                                                                                            c.d_ninv);
    CK(cudaGetLastError());
}

// Two-pass transform (N = 2^14 .. 2^16) of every row with tiles of R sub-transforms and 2^RB residues
// per thread: N1 column transforms of N2 points... the column pass first (forward) or last (inverse).
template <bool INV, int R, int RB>
void two_pass(const Ctx& c, const PolyBatch& pb, cudaStream_t s, double bytes) {
    switch (c.log_n) {
        case 14:  // 128 x 128
            if (!INV) {
                launch_tile<14, 7, R, false, 0, false, RB>(c, pb, 128 / R, s, bytes);
                launch_tile<14, 7, R, false, 1, true, RB>(c, pb, 128 / R, s, bytes);
            } else {
                launch_tile<14, 7, R, true, 1, false, RB>(c, pb, 128 / R, s, bytes);
                launch_tile<14, 7, R, true, 0, true, RB>(c, pb, 128 / R, s, bytes);
            }
            return;
        case 15:  // 256 column transforms of 2^7 points (N2 = 256), then 128 rows of 2^8
            if (!INV) {
                launch_tile<15, 7, R, false, 0, false, RB>(c, pb, 256 / R, s, bytes);
                launch_tile<15, 8, R, false, 1, true, RB>(c, pb, 128 / R, s, bytes);
            } else {
                launch_tile<15, 8, R, true, 1, false, RB>(c, pb, 128 / R, s, bytes);
                launch_tile<15, 7, R, true, 0, true, RB>(c, pb, 256 / R, s, bytes);
            }
            return;
        case 16:  // 256 x 256
            if (!INV) {
                launch_tile<16, 8, R, false, 0, false, RB>(c, pb, 256 / R, s, bytes);
                launch_tile<16, 8, R, false, 1, true, RB>(c, pb, 256 / R, s, bytes);
            } else {
                launch_tile<16, 8, R, true, 1, false, RB>(c, pb, 256 / R, s, bytes);
                launch_tile<16, 8, R, true, 0, true, RB>(c, pb, 256 / R, s, bytes);
            }
            return;
        default: fail(FHE_ERR_INVALID_ARG, "unsupported ring degree");
    }
}

// The tile shapes the autotuner chooses between (family "ntt"): rows or columns per tile R and
// residues per thread 2^RB; every shape computes the same bits.
enum NttTile { NTT_R16B4 = 0, NTT_R8B4, NTT_R32B4, NTT_R16B3, NTT_N_TILES };
extern const char* const kNttTileNames[NTT_N_TILES];
void two_pass_r8b4(const Ctx& c, const PolyBatch& pb, bool inv, cudaStream_t s, double bytes);
void two_pass_r32b4(const Ctx& c, const PolyBatch& pb, bool inv, cudaStream_t s, double bytes);
void two_pass_r16b3(const Ctx& c, const PolyBatch& pb, bool inv, cudaStream_t s, double bytes);

}  // namespace ntt_tile
}  // namespace fhe

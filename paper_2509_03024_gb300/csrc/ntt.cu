// ntt.cu — batched negacyclic NTT over RNS limbs.
//
// Forward: Cooley-Tukey with merged psi powers (natural order in, bit-reversed
// order out): slot k holds a(psi^(2 brev(k) + 1)). Inverse: Gentleman-Sande
// (bit-reversed in, natural out) followed by the N^-1 scaling.
//
// Decomposition. A ring of N = N1 * N2 coefficients is viewed as N1 rows of
// N2: the first log2(N1) stages couple elements N2 apart (independent
// N1-point transforms on columns), the remaining stages couple elements inside
// one row (N2-point transforms with row-dependent twiddles). Rings up to 2^13
// run in one pass (N1 = N, one CTA per limb); larger rings in two passes.
//
// Each CTA holds a tile of R sub-transforms of M = 2^LOGM points in shared
// memory (element x of sub-transform q at x*(R+1) + q). Row passes read their
// twiddles from tables transposed to [stage][group][row], so that the R rows of a
// tile load consecutive entries. Every thread owns 8
// residues and runs three butterfly stages in registers between shared-memory
// exchanges (radix-8 blocking; the last block has 1-3 stages). Arithmetic is
// lazy in the style of Harvey (2014): forward values stay in [0, 4q), inverse
// values in [0, 2q); twiddle products use Shoup's precomputed quotient and no
// final correction; the last pass reduces to [0, q).
#include "ntt_core.cuh"

namespace fhe {

namespace {

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

template <bool INV>
void run_ntt(const Ctx& c, const PolyBatch& pb, cudaStream_t s) {
    const int rows = pb.rows();
    if (rows == 0) return;
    const double bytes = 16.0 * rows * ((size_t)1 << c.log_n);
    switch (c.log_n) {
        case 9: launch_tile<9, 9, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 10: launch_tile<10, 10, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 11: launch_tile<11, 11, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 12: launch_tile<12, 12, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 13: launch_tile<13, 13, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 14:  // 128 x 128
            if (!INV) {
                launch_tile<14, 7, 16, false, 0, false>(c, pb, 128 / 16, s, bytes);
                launch_tile<14, 7, 16, false, 1, true>(c, pb, 128 / 16, s, bytes);
            } else {
                launch_tile<14, 7, 16, true, 1, false>(c, pb, 128 / 16, s, bytes);
                launch_tile<14, 7, 16, true, 0, true>(c, pb, 128 / 16, s, bytes);
            }
            return;
        case 15:  // 256 column transforms of 2^7 points (N2 = 256), then 128 rows of 2^8
            if (!INV) {
                launch_tile<15, 7, 16, false, 0, false>(c, pb, 256 / 16, s, bytes);
                launch_tile<15, 8, 16, false, 1, true>(c, pb, 128 / 16, s, bytes);
            } else {
                launch_tile<15, 8, 16, true, 1, false>(c, pb, 128 / 16, s, bytes);
                launch_tile<15, 7, 16, true, 0, true>(c, pb, 256 / 16, s, bytes);
            }
            return;
        case 16:  // 256 x 256
            if (!INV) {
                launch_tile<16, 8, 16, false, 0, false>(c, pb, 256 / 16, s, bytes);
                launch_tile<16, 8, 16, false, 1, true>(c, pb, 256 / 16, s, bytes);
            } else {
                launch_tile<16, 8, 16, true, 1, false>(c, pb, 256 / 16, s, bytes);
                launch_tile<16, 8, 16, true, 0, true>(c, pb, 256 / 16, s, bytes);
            }
            return;
        default: fail(FHE_ERR_INVALID_ARG, "unsupported ring degree");
    }
}

}  // namespace

void ntt_init() {}

void ntt_forward(const Ctx& c, const PolyBatch& pb, cudaStream_t s) { run_ntt<false>(c, pb, s); }
void ntt_inverse(const Ctx& c, const PolyBatch& pb, cudaStream_t s) { run_ntt<true>(c, pb, s); }

}  // namespace fhe

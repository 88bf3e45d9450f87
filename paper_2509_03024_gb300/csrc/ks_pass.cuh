// ks_pass.cuh — the fused NTT passes of key switching and rescaling (ks.cu): row descriptors,
// the load and store modes that fuse the base conversions and the combinations into the first and
// last pass of a transform, the pass kernel and its launchers. See ks.cu for the algorithm.
#pragma once

#include "ks_inner.cuh"
#include "ntt_core.cuh"

namespace fhe {

namespace ksp {

using nttc::reduce4;
using nttc::shoup_lazy;

enum LoadMode { LD_PLAIN = 0, LD_GATHER = 1, LD_CONV = 2, LD_AXPY = 3, LD_CENTRED = 4, LD_MUL = 5 };
enum StoreMode { ST_LAZY = 0, ST_LAST = 1, ST_SCALE = 2, ST_COMBINE = 3, ST_COMBINE_RS = 4, ST_RESCALE = 5 };

struct KsRow {
    u64* dst;        // the row's buffer (N residues)
    const u64* src;  // LD_GATHER: source row; LD_CONV: first source limb (limb stride N)
    const u64* cst;  // LD_CONV: Shoup pair of the first source limb for this row's prime; ST_SCALE: (w, ws)
    int prime;       // prime index of the row
    int galois;      // LD_GATHER: automorphism applied on load (1 = none)
    int src_cnt;     // LD_CONV: number of source limbs
    int cst_stride;  // LD_CONV: words between consecutive source limbs' constant pairs
    int item, half, limb;  // ST_COMBINE(_RS): output item, component and limb
    int pack;              // ST_LAST (forward): store the residue split at bit 25 (key_pack)
    const u64* src2;       // LD_AXPY / LD_MUL: second source row (LD_AXPY: null = none); ST_RESCALE: the input limb
    const u64* cst2;       // LD_AXPY: Shoup pair of its factor; ST_RESCALE: q_l^-1 mod the row's prime
    u64* out2;             // ST_RESCALE: output row
    const u64* src3;       // ST_RESCALE: when set, the input limb is src2 (.) src3 (a plaintext product)
};

constexpr int kMaxHoist = 31;

// Rotation keys of a hoisted rotate-and-sum (host side).
struct HoistKeys {
    const u64* key[kMaxHoist];
    int galois[kMaxHoist];
    int count;
};

struct CombineArgs {
    const KsItem* items;
    const u64* acc;    // [items][2][next][N]
    const u64* pinv;   // [L+1][2] P^-1 mod q_i (ST_COMBINE) or (P q_l)^-1 mod q_i (ST_COMBINE_RS)
    int next;
    const u64* qlinv;  // ST_COMBINE_RS: [L+1][2] q_l^-1 mod q_i
};

// Per-row constants of the first pass's loads, read once per CTA: the row's prime and, for the base
// conversion, the Shoup pairs of its (at most kConvMax) source limbs.
constexpr int kConvMax = 4;
struct RowConst {
    u64 q, one_s, ql;
    u64 w[kConvMax], ws[kConvMax];
};

template <int LOAD>
__device__ __forceinline__ RowConst row_const(const KsRow& r, const Prime* __restrict__ pr) {
    RowConst c;
    c.q = pr[r.prime].q;
    c.one_s = pr[r.prime].one_s;
    c.ql = LOAD == LD_CENTRED ? pr[r.limb].q : 0;
#pragma unroll
    for (int i = 0; i < kConvMax; i++) {
        const bool on = LOAD == LD_CONV && i < r.src_cnt;
        c.w[i] = on ? r.cst[(size_t)i * r.cst_stride] : 0;
        c.ws[i] = on ? r.cst[(size_t)i * r.cst_stride + 1] : 0;
    }
    return c;
}

template <int LOAD>
__device__ __forceinline__ u64 load_elem(const KsRow& r, size_t k, int log_n, const Prime* __restrict__ pr,
                                         const RowConst& rc) {
    if (LOAD == LD_PLAIN) return r.dst[k];
    if (LOAD == LD_GATHER) return r.src[r.galois == 1 ? (int)k : auto_src((int)k, r.galois, log_n)];
    if (LOAD == LD_CENTRED) {  // the centred representative of src[k] (mod q_limb) reduced mod the row's prime
        const u64 ql = rc.ql, v = r.src[k];
        const bool neg = v > (ql >> 1);
        const u64 m = nttc::reduce_any(neg ? ql - v : v, rc.q, rc.one_s);
        return neg ? (m ? rc.q - m : 0) : m;
    }
    if (LOAD == LD_MUL) return mul_mod(r.src[k], r.src2[k], pr[r.prime]);
    if (LOAD == LD_AXPY) {  // src + cst2 * src2 (both reduced)
        const u64 p = rc.q;
        u64 v = r.src[k];
        if (r.src2) v = add_mod(v, mul_shoup(r.src2[k], r.cst2[0], r.cst2[1], p), p);
        return v;
    }
    // LD_CONV: sum of the converted source limbs. For primes below 2^58 the forward transform that
    // follows runs without intermediate reduction, so the sum stays lazy (each term below 2p, at most
    // 8 terms, so below 16p; 16 stages add less than 32p: below 48p < 2^64); otherwise fully reduced.
    // Up to kConvMax sources: every source load is issued before the products (fixed trip count,
    // predicated), so a thread's loads are in flight together.
    const u64 p = rc.q;
    if (r.src_cnt <= kConvMax) {
        u64 x[kConvMax];
#pragma unroll
        for (int i = 0; i < kConvMax; i++) x[i] = i < r.src_cnt ? r.src[((size_t)i << log_n) + k] : 0;
        if (p < ((u64)1 << 58)) {
            u64 lazy = 0;
#pragma unroll
            for (int i = 0; i < kConvMax; i++)
                if (i < r.src_cnt) lazy += shoup_lazy(x[i], rc.w[i], rc.ws[i], p);
            return lazy;
        }
        u64 acc = 0;
#pragma unroll
        for (int i = 0; i < kConvMax; i++)
            if (i < r.src_cnt) {
                u64 t = shoup_lazy(x[i], rc.w[i], rc.ws[i], p);
                t = t >= p ? t - p : t;
                acc += t;
                acc = acc >= p ? acc - p : acc;
            }
        return acc;
    }
    if (p < ((u64)1 << 58) && r.src_cnt <= 8) {
        u64 lazy = 0;
        for (int i = 0; i < r.src_cnt; i++) {
            const u64* c = r.cst + (size_t)i * r.cst_stride;
            lazy += shoup_lazy(r.src[((size_t)i << log_n) + k], c[0], c[1], p);
        }
        return lazy;
    }
    u64 acc = 0;
    for (int i = 0; i < r.src_cnt; i++) {
        const u64* c = r.cst + (size_t)i * r.cst_stride;
        u64 t = shoup_lazy(r.src[((size_t)i << log_n) + k], c[0], c[1], p);
        t = t >= p ? t - p : t;
        acc += t;
        acc = acc >= p ? acc - p : acc;
    }
    return acc;
}

template <bool INV, int STORE>
__device__ __forceinline__ void store_elem(const KsRow& r, size_t k, u64 v, const Prime* __restrict__ prow, u64 q, u64 one_s,
                                           const u64* __restrict__ ninv, const CombineArgs& ca, int log_n) {
    if (STORE == ST_LAZY) {
        r.dst[k] = v;
        return;
    }
    if (STORE == ST_LAST) {
        if (INV) {
            u64 t = shoup_lazy(v, ninv[2 * r.prime], ninv[2 * r.prime + 1], q);
            r.dst[k] = t >= q ? t - q : t;
        } else {
            const u64 t = nttc::reduce_any(v, q, one_s);
            r.dst[k] = r.pack ? key_pack(t) : t;
        }
        return;
    }
    if (STORE == ST_RESCALE) {  // forward: out = (x - [x_l]) q_l^-1 with the transformed [x_l] in v
        const u64 t = nttc::reduce_any(v, q, one_s);
        const u64 x = r.src3 ? mul_mod(r.src2[k], r.src3[k], *prow) : r.src2[k];
        r.out2[k] = mul_shoup(sub_mod(x, t, q), r.cst2[0], r.cst2[1], q);
        return;
    }
    if (STORE == ST_SCALE) {  // inverse transforms only: times the row's constant instead of N^-1
        u64 t = shoup_lazy(v, r.cst[0], r.cst[1], q);
        r.dst[k] = t >= q ? t - q : t;
        return;
    }
    const KsItem& it = ca.items[r.item];
    const size_t row_off = (size_t)r.limb << log_n;
    u64 conv = nttc::reduce_any(v, q, one_s);
    u64 a = ca.acc[((((size_t)r.item * 2 + r.half) * ca.next + r.limb) << log_n) + k];
    u64 d = a >= conv ? a - conv : a + q - conv;
    if (STORE == ST_COMBINE_RS) {
        // fused ModDown + rescale: out_h = (acc_h - conv) (P q_l)^-1 + c_h q_l^-1
        const u64* c_h = r.half == 0 ? it.addI0 : it.addI1;
        u64 t = mul_shoup(d, ca.pinv[2 * r.limb], ca.pinv[2 * r.limb + 1], q);
        t = add_mod(t, mul_shoup(c_h[row_off + k], ca.qlinv[2 * r.limb], ca.qlinv[2 * r.limb + 1], q), q);
        (r.half == 0 ? it.out0 : it.out1)[row_off + k] = t;
        return;
    }
    // ST_COMBINE (forward): out_h = (acc_h - v) * P^-1 + add terms
    u64 t = shoup_lazy(d, ca.pinv[2 * r.limb], ca.pinv[2 * r.limb + 1], q);
    t = t >= q ? t - q : t;
    if (r.half == 0) {
        if (it.addP0) {
            int src = it.galois == 1 ? (int)k : auto_src((int)k, (int)it.galois, log_n);
            t = add_mod(t, it.addP0[row_off + src], q);
        }
        if (it.addI0) t = add_mod(t, it.addI0[row_off + k], q);
        it.out0[row_off + k] = t;
    } else {
        if (it.addI1) t = add_mod(t, it.addI1[row_off + k], q);
        it.out1[row_off + k] = t;
    }
}

// One NTT pass over a row table (PASS 0: column tiles / single pass; PASS 1: row tiles).
constexpr int ks_min_blocks(int rb, int threads) {
    return (rb == 3 ? 1024 : 768) / threads > 0 ? (rb == 3 ? 1024 : 768) / threads : 1;
}

// LOOSE halves the CTAs per SM the launch bounds ask for, which doubles the registers a thread may use
// (fewer spills, lower occupancy).
template <int LOGN, int LOGM, int R, bool INV, int PASS, int LOAD, int STORE, int RB, bool LOOSE = false>
__global__ void __launch_bounds__(R * (1 << LOGM) / (1 << RB),
                                  (ks_min_blocks(RB, R * (1 << LOGM) / (1 << RB)) + (LOOSE ? 1 : 0)) / (LOOSE ? 2 : 1))
ks_ntt_kernel(const KsRow* __restrict__ rows, const Prime* __restrict__ primes, const ulonglong2* __restrict__ tw,
              const u64* __restrict__ ninv, CombineArgs ca) {
    constexpr int log_n = LOGN;  // the ring size is a compile-time constant of each launch
    constexpr int M = 1 << LOGM;
    constexpr int P = R == 1 ? 1 : R + 1;
    constexpr int V = 1 << RB;
    constexpr int T = R * M / V;
    extern __shared__ u64 sm[];
    const int tid = threadIdx.x;
    const KsRow r = rows[blockIdx.x];
    const RowConst rc = row_const<LOAD>(r, primes);
    const u64 q = primes[r.prime].q;
    const ulonglong2* W = tw + ((size_t)r.prime << log_n);
    const int log_n2 = PASS == 0 ? log_n - LOGM : LOGM;
    const int S1 = log_n - log_n2;
    const int t0 = blockIdx.y * R;
    if (PASS == 0 && R > 1) {
        // column tiles: the first and last register blocks read and write global memory directly
        constexpr int NB = (LOGM + RB - 1) / RB;
        const int qq = tid % R, g = tid / R;
        const int fb = INV ? NB - 1 : 0, lb = INV ? 0 : NB - 1;
        u64 v[V];
#pragma unroll
        for (int u = 0; u < V; u++)
            v[u] = load_elem<LOAD>(r, (size_t)(t0 + qq) + ((size_t)nttc::block_elem<LOGM, RB>(fb, g, u) << log_n2),
                                   log_n, primes, rc);
        if (!INV && q < ((u64)1 << 58))
            nttc::tile_stages<LOGM, R, INV, PASS, false, true, true, RB>(sm, W, q, S1, t0, v);
        else
            nttc::tile_stages<LOGM, R, INV, PASS, true, true, true, RB>(sm, W, q, S1, t0, v);
        const u64 one_s = primes[r.prime].one_s;
#pragma unroll
        for (int u = 0; u < V; u++)
            store_elem<INV, STORE>(r, (size_t)(t0 + qq) + ((size_t)nttc::block_elem<LOGM, RB>(lb, g, u) << log_n2), v[u], primes + r.prime,
                                   q, one_s, ninv, ca, log_n);
        return;
    }
    if (PASS == 0) {
#pragma unroll 4
        for (int e = tid; e < R * M; e += T) {
            int x = e / R, qq = e % R;
            sm[x * P + qq] = load_elem<LOAD>(r, (size_t)(t0 + qq) + ((size_t)x << log_n2), log_n, primes, rc);
        }
    } else {
#pragma unroll 4
        for (int e = tid; e < R * M; e += T) {
            int x = e & (M - 1), qq = e >> LOGM;
            sm[x * P + qq] = load_elem<LOAD>(r, ((size_t)(t0 + qq) << LOGM) + x, log_n, primes, rc);
        }
    }
    __syncthreads();
    if (!INV && q < ((u64)1 << 58)) nttc::tile_stages<LOGM, R, INV, PASS, false, RB>(sm, W, q, S1, t0);
    else nttc::tile_stages<LOGM, R, INV, PASS, true, RB>(sm, W, q, S1, t0);
    const u64 one_s = primes[r.prime].one_s;
    if (PASS == 0) {
#pragma unroll 4
        for (int e = tid; e < R * M; e += T) {
            int x = e / R, c = e % R;
            store_elem<INV, STORE>(r, (size_t)(t0 + c) + ((size_t)x << log_n2), sm[x * P + c], primes + r.prime, q,
                                   one_s, ninv, ca, log_n);
        }
    } else {
#pragma unroll 4
        for (int e = tid; e < R * M; e += T) {
            int x = e & (M - 1), c = e >> LOGM;
            store_elem<INV, STORE>(r, ((size_t)(t0 + c) << LOGM) + x, sm[x * P + c], primes + r.prime, q, one_s,
                                   ninv, ca, log_n);
        }
    }
}

// The fused passes keep radix-8 register blocks: with 16 residues per thread their load and
// store stages run out of registers (measured slower, unlike the plain transform).
template <int LOGN, int LOGM, int R, bool INV, int PASS, int LOAD, int STORE, int RB = 3, bool LOOSE = false>
void launch_pass(const Ctx& c, const KsRow* rows, int n_rows, int tiles, const CombineArgs& ca, int cls, double bytes,
                 cudaStream_t s) {
    if (n_rows == 0) return;
    constexpr int T = R * (1 << LOGM) / (1 << RB);
    constexpr size_t smem = sizeof(u64) * (1 << LOGM) * (R == 1 ? 1 : R + 1);
    const ulonglong2* tw = PASS == 1 ? (INV ? c.d_itw2 : c.d_tw2) : (INV ? c.d_itw : c.d_tw);
    if (smem > 48 * 1024)
        CK(cudaFuncSetAttribute(ks_ntt_kernel<LOGN, LOGM, R, INV, PASS, LOAD, STORE, RB, LOOSE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LaunchScope _ls(c.prof, cls, bytes, s, (double)n_rows * ((size_t)1 << (c.log_n - 1)) * LOGM);
    ks_ntt_kernel<LOGN, LOGM, R, INV, PASS, LOAD, STORE, RB, LOOSE><<<dim3(n_rows, tiles), T, smem, s>>>(
        rows, c.d_primes, tw, c.d_ninv, ca);
    CK(cudaGetLastError());
}

// A full forward (INV = false) or inverse transform over a row table: the first pass applies
// LOAD, the last pass applies STORE (single-pass rings do both in one kernel).
template <bool INV, int LOAD, int STORE, int R, bool LOOSE = false>
void ks_transform_t(const Ctx& c, const KsRow* rows, int n_rows, const CombineArgs& ca, int cls, double bytes,
                    cudaStream_t s) {
    constexpr int FIRST_ST = ST_LAZY;
    switch (c.log_n) {
#define SINGLE(LG)                                                                        \
    case LG:                                                                              \
        launch_pass<LG, LG, 1, INV, 0, LOAD, STORE, 3>(c, rows, n_rows, 1, ca, cls, bytes, s); \
        return;
        SINGLE(9)
        SINGLE(10)
        SINGLE(11)
        SINGLE(12)
        SINGLE(13)
#undef SINGLE
        case 14:
            if (!INV) {
                launch_pass<14, 7, R, false, 0, LOAD, FIRST_ST, 3, LOOSE>(c, rows, n_rows, 128 / R, ca, cls, bytes, s);
                launch_pass<14, 7, R, false, 1, LD_PLAIN, STORE, 3, LOOSE>(c, rows, n_rows, 128 / R, ca, cls, bytes, s);
            } else {
                launch_pass<14, 7, R, true, 1, LOAD, FIRST_ST, 3, LOOSE>(c, rows, n_rows, 128 / R, ca, cls, bytes, s);
                launch_pass<14, 7, R, true, 0, LD_PLAIN, STORE, 3, LOOSE>(c, rows, n_rows, 128 / R, ca, cls, bytes, s);
            }
            return;
        case 15:
            if (!INV) {
                launch_pass<15, 7, R, false, 0, LOAD, FIRST_ST, 3, LOOSE>(c, rows, n_rows, 256 / R, ca, cls, bytes, s);
                launch_pass<15, 8, R, false, 1, LD_PLAIN, STORE, 3, LOOSE>(c, rows, n_rows, 128 / R, ca, cls, bytes, s);
            } else {
                launch_pass<15, 8, R, true, 1, LOAD, FIRST_ST, 3, LOOSE>(c, rows, n_rows, 128 / R, ca, cls, bytes, s);
                launch_pass<15, 7, R, true, 0, LD_PLAIN, STORE, 3, LOOSE>(c, rows, n_rows, 256 / R, ca, cls, bytes, s);
            }
            return;
        case 16:
            if (!INV) {
                launch_pass<16, 8, R, false, 0, LOAD, FIRST_ST, 3, LOOSE>(c, rows, n_rows, 256 / R, ca, cls, bytes, s);
                launch_pass<16, 8, R, false, 1, LD_PLAIN, STORE, 3, LOOSE>(c, rows, n_rows, 256 / R, ca, cls, bytes, s);
            } else {
                launch_pass<16, 8, R, true, 1, LOAD, FIRST_ST, 3, LOOSE>(c, rows, n_rows, 256 / R, ca, cls, bytes, s);
                launch_pass<16, 8, R, true, 0, LD_PLAIN, STORE, 3, LOOSE>(c, rows, n_rows, 256 / R, ca, cls, bytes, s);
            }
            return;
        default: fail(FHE_ERR_INVALID_ARG, "unsupported ring degree");
    }
}

// The tile shapes of the fused passes the autotuner chooses between (family "ks_pass"): rows or
// columns per tile of the two-pass rings (r8x: 8 with the register cap of LOOSE launch bounds); every
// shape computes the same bits. Each shape's instantiations live in a translation unit of their own
// (ks_pass16.cu, ks_pass8.cu, ks_pass8x.cu).
enum KsTile { KS_R16 = 0, KS_R8, KS_R8X, KS_N_TILES };
extern const char* const kKsTileNames[KS_N_TILES];

#define KS_COMBOS(X)                      \
    X(true, LD_GATHER, ST_SCALE)          \
    X(false, LD_CONV, ST_LAST)            \
    X(false, LD_GATHER, ST_LAST)          \
    X(true, LD_AXPY, ST_SCALE)            \
    X(false, LD_CONV, ST_COMBINE_RS)      \
    X(false, LD_CONV, ST_COMBINE)         \
    X(true, LD_MUL, ST_SCALE)             \
    X(false, LD_CENTRED, ST_RESCALE)

template <bool INV, int LOAD, int STORE>
void ks_transform_r16(const Ctx& c, const KsRow* rows, int n_rows, const CombineArgs& ca, int cls, double bytes,
                      cudaStream_t s);
template <bool INV, int LOAD, int STORE>
void ks_transform_r8(const Ctx& c, const KsRow* rows, int n_rows, const CombineArgs& ca, int cls, double bytes,
                     cudaStream_t s);
template <bool INV, int LOAD, int STORE>
void ks_transform_r8x(const Ctx& c, const KsRow* rows, int n_rows, const CombineArgs& ca, int cls, double bytes,
                      cudaStream_t s);

// A full forward (INV = false) or inverse transform over a row table with the context's tile shape:
// the first pass applies LOAD, the last pass applies STORE (single-pass rings do both in one kernel).
template <bool INV, int LOAD, int STORE>
void ks_transform(const Ctx& c, const KsRow* rows, int n_rows, const CombineArgs& ca, int cls, double bytes,
                  cudaStream_t s) {
    if (c.tune.ks == KS_R8) ks_transform_r8<INV, LOAD, STORE>(c, rows, n_rows, ca, cls, bytes, s);
    else if (c.tune.ks == KS_R8X) ks_transform_r8x<INV, LOAD, STORE>(c, rows, n_rows, ca, cls, bytes, s);
    else ks_transform_r16<INV, LOAD, STORE>(c, rows, n_rows, ca, cls, bytes, s);
}

}  // namespace ksp
}  // namespace fhe

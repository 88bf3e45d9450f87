// ks_inner.cu — key inner product of hybrid key switching (Han-Ki 2020), K3 of ks.cu:
//
//   acc[t][h][x][k] = sum_j M_j[x][k] * evk_j[h][px][k]        (plain / fan-out)
//   acc[t][h][x][k] = sum_r sum_j M_j[x][pi_r(k)] * evk_{r,j}[h][px][k]   (hoisted rotate-and-sum)
//
// M_j[x] is the raised digit j at extended limb x (the item's own input on the limbs of digit j),
// pi_r the slot map of rotation r. Products are summed exactly in 128 bits and reduced once, so the
// result is independent of the formulation; the variants differ in
//   * the multiply-accumulate: "C" (the product's low and high halves in C and a carry compare),
//     "P32" (a schoolbook chain of 32-bit mad.lo / mad.hi with carries) or, for data primes below
//     2^50, "S25" (operands split at bit 25: four mad.wide.u32 partial products into three 64-bit
//     column sums that cannot wrap, no additions at all),
//   * items per thread: items that share a key read each key pair once for all of them,
//   * the launch shape: blockIdx.y is the extended limb, so every block of one limb runs before the
//     next limb's, keeping that limb's key rows in L2 while every item reads them.
// An automorphism maps every aligned pair of evaluation slots onto an aligned pair, so a pair is
// one 128-bit load whatever the rotation.
#include <algorithm>

#include "ks_inner.cuh"
#include "ntt_core.cuh"

namespace fhe {

const char* const kInnerVariantNames[INNER_N_VARIANTS] = {"v0", "c1", "p1", "s1", "s2", "s2l"};

namespace {

// (hi * 2^64 + lo) mod q for hi, lo < 2^64: hi and lo reduced with floor(2^64 / q), then
// hi * (2^64 mod q) + lo.
__device__ __forceinline__ u64 reduce128(u64 lo, u64 hi, const Prime& P) {
    const u64 q = P.q;
    const u64 h = nttc::reduce_any(hi, q, P.one_s);
    const u64 l = nttc::reduce_any(lo, q, P.one_s);
    const u64 r64 = (u64)0 - q * P.one_s;  // 2^64 mod q
    return add_mod(mul_mod(h, r64, P), l, q);
}

// ---------------------------------------------------------------- multiply-accumulate forms

struct MacC {
    u64 lo = 0, hi = 0;
    __device__ __forceinline__ void mac(u64 a, u64 b) {
        const u64 pl = a * b, ph = __umul64hi(a, b);
        lo += pl;
        hi += ph + (lo < pl ? 1 : 0);
    }
    __device__ __forceinline__ u64 reduce(const Prime& P) const { return reduce128(lo, hi, P); }
    __device__ __forceinline__ void macx(u64 a, bool ap, u64 k, bool kp) {
        mac(ap ? key_unpack(a) : a, kp ? key_unpack(k) : k);
    }
};

struct MacP {  // PTX 64-bit multiply-add with carry (the one-item legacy form of the plain kernel)
    u64 lo = 0, hi = 0;
    __device__ __forceinline__ void mac(u64 a, u64 b) {
        asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;" : "+l"(lo), "+l"(hi) : "l"(a), "l"(b));
    }
    __device__ __forceinline__ u64 reduce(const Prime& P) const { return reduce128(lo, hi, P); }
    __device__ __forceinline__ void macx(u64 a, bool ap, u64 k, bool kp) {
        mac(ap ? key_unpack(a) : a, kp ? key_unpack(k) : k);
    }
};

// Schoolbook on 32-bit words in one carry chain per row: a0 b0 and a1 b1 first, then each cross
// product (eight mad.lo / mad.hi with carries and two carry propagations).
struct MacP32 {
    u32 r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    __device__ __forceinline__ void mac(u64 a, u64 b) {
        const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
        asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
            "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
            "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
            "madc.hi.u32 %3, %5, %7, %3;\n\t"
            "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
            "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
            "addc.u32 %3, %3, 0;\n\t"
            "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
            "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
            "addc.u32 %3, %3, 0;"
            : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3)
            : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    }
    __device__ __forceinline__ u64 reduce(const Prime& P) const {
        return reduce128(((u64)r1 << 32) | r0, ((u64)r3 << 32) | r2, P);
    }
    __device__ __forceinline__ void macx(u64 a, bool ap, u64 k, bool kp) {
        mac(ap ? key_unpack(a) : a, kp ? key_unpack(k) : k);
    }
};

// Operands below 2^50 split at bit 25: a b = a0 b0 + 2^25 (a0 b1 + a1 b0) + 2^50 a1 b1 with every
// partial product below 2^50, so three 64-bit column sums take up to 2^13 terms without a carry:
// four mad.wide.u32 per multiply-accumulate and no additions.
struct MacS25 {
    u64 C0 = 0, C1 = 0, C2 = 0;
    __device__ __forceinline__ void mac4(u32 a0, u32 a1, u32 b0, u32 b1) {
        asm("mad.wide.u32 %0, %3, %5, %0;\n\t"
            "mad.wide.u32 %1, %3, %6, %1;\n\t"
            "mad.wide.u32 %1, %4, %5, %1;\n\t"
            "mad.wide.u32 %2, %4, %6, %2;"
            : "+l"(C0), "+l"(C1), "+l"(C2)
            : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    }
    // an unpacked operand is split with a mask and a shift; a packed one (key_pack) already holds
    // its two halves in its two words
    __device__ __forceinline__ void macx(u64 a, bool ap, u64 k, bool kp) {
        const u32 m = (1u << 25) - 1u;
        const u32 a0 = ap ? (u32)a : (u32)a & m, a1 = ap ? (u32)(a >> 32) : (u32)(a >> 25);
        const u32 b0 = kp ? (u32)k : (u32)k & m, b1 = kp ? (u32)(k >> 32) : (u32)(k >> 25);
        mac4(a0, a1, b0, b1);
    }
    __device__ __forceinline__ u64 reduce(const Prime& P) const {
        // C0 + 2^25 C1 + 2^50 C2 as (hi, lo)
        u64 lo = C0 + (C1 << 25);
        u64 hi = (C1 >> 39) + (lo < C0 ? 1 : 0);
        const u64 add = C2 << 50;
        const u64 lo2 = lo + add;
        hi += (C2 >> 14) + (lo2 < lo ? 1 : 0);
        return reduce128(lo2, hi, P);
    }
};

// Slots (2 k2, 2 k2 + 1) of phi_g(row): the automorphism maps the aligned pair onto an aligned pair.
__device__ __forceinline__ void load_pair_auto(const u64* __restrict__ row, int k2, int g, int log_n, u64& vx, u64& vy) {
    const int src = auto_src(2 * k2, g, log_n);
    const ulonglong2 v = reinterpret_cast<const ulonglong2*>(row)[src >> 1];
    vx = (src & 1) ? v.y : v.x;
    vy = (src & 1) ? v.x : v.y;
}

// ---------------------------------------------------------------- v0: the grid-stride forms

template <bool FANOUT>
__global__ void __launch_bounds__(256, 4) inner_v0_kernel(InnerArgs a) {
    const int log_n = a.log_n;
    const size_t half = (size_t)1 << (log_n - 1);
    const size_t total = (size_t)a.items * a.next * half;
    const int l1 = a.level + 1;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int k2 = (int)(e & (half - 1));
        const size_t row = e >> (log_n - 1);
        const int t = (int)(row % a.items), x = (int)(row / a.items);
        const int px = x < l1 ? x : x + (a.L - a.level);
        const Prime P = a.pr[px];
        const KsItem it = a.tab[t];
        const int own = x < l1 ? x / a.alpha : -1;
        const bool packed = a.keys_packed && x < l1;
        MacP s0x, s0y, s1x, s1y;
        const int st = FANOUT ? a.src_of[t] : t;
        for (int j = 0; j < a.dn; j++) {
            const bool vpk = packed && j != own;  // raised digits of data limbs are stored packed
            u64 vx, vy;
            const u64* src = j == own ? it.d + ((size_t)x << log_n)
                                      : a.ext + ((size_t)((st * a.dn + j) * a.next + x) << log_n);
            if (FANOUT || (j == own && it.galois != 1)) {
                load_pair_auto(src, k2, (int)it.galois, log_n, vx, vy);
            } else {
                const ulonglong2 v = reinterpret_cast<const ulonglong2*>(src)[k2];
                vx = v.x;
                vy = v.y;
            }
            const ulonglong2 kb = reinterpret_cast<const ulonglong2*>(it.key + ((size_t)((j * 2 + 0) * a.n_ext + px) << log_n))[k2];
            const ulonglong2 ka = reinterpret_cast<const ulonglong2*>(it.key + ((size_t)((j * 2 + 1) * a.n_ext + px) << log_n))[k2];
            s0x.macx(vx, vpk, kb.x, packed);
            s0y.macx(vy, vpk, kb.y, packed);
            s1x.macx(vx, vpk, ka.x, packed);
            s1y.macx(vy, vpk, ka.y, packed);
        }
        reinterpret_cast<ulonglong2*>(a.acc + ((size_t)((t * 2 + 0) * a.next + x) << log_n))[k2] =
            make_ulonglong2(s0x.reduce(P), s0y.reduce(P));
        reinterpret_cast<ulonglong2*>(a.acc + ((size_t)((t * 2 + 1) * a.next + x) << log_n))[k2] =
            make_ulonglong2(s1x.reduce(P), s1y.reduce(P));
    }
}

__global__ void __launch_bounds__(256, 3) hoist_v0_kernel(InnerArgs a) {
    const int log_n = a.log_n;
    const size_t half = (size_t)1 << (log_n - 1);
    const size_t total = (size_t)a.items * a.next * half;
    const int l1 = a.level + 1;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int k2 = (int)(e & (half - 1));
        const size_t row = e >> (log_n - 1);
        const int t = (int)(row % a.items), x = (int)(row / a.items);
        const int px = x < l1 ? x : x + (a.L - a.level);
        const int own = x < l1 ? x / a.alpha : -1;
        const bool packed = a.keys_packed && x < l1;
        const ulonglong2* ext0 = reinterpret_cast<const ulonglong2*>(a.ext) + (((size_t)t * a.dn * a.next + x) << (log_n - 1));
        const ulonglong2* own_row = reinterpret_cast<const ulonglong2*>(a.tab[t].d) + ((size_t)x << (log_n - 1));
        const size_t dstride = (size_t)a.next << (log_n - 1);
        const size_t kstride = (size_t)a.n_ext << (log_n - 1);
        const size_t koff = ((size_t)px << (log_n - 1)) + k2;
        MacC s0x, s0y, s1x, s1y;
        for (int r = 0; r < a.n_steps; r++) {
            const HoistStep st = a.steps[r];
            const int src = auto_src(2 * k2, (int)st.galois, log_n);
            const int sp = src >> 1;
            const bool sw = src & 1;
            const ulonglong2* kr = reinterpret_cast<const ulonglong2*>(st.key) + koff;
            for (int j = 0; j < a.dn; j++) {
                const bool vpk = packed && j != own;  // raised digits of data limbs are stored packed
                const ulonglong2 v = (j == own ? own_row : ext0 + (size_t)j * dstride)[sp];
                const u64 vx = sw ? v.y : v.x, vy = sw ? v.x : v.y;
                const ulonglong2 kb = kr[(size_t)(2 * j) * kstride];
                const ulonglong2 ka = kr[(size_t)(2 * j + 1) * kstride];
                s0x.macx(vx, vpk, kb.x, packed);
                s0y.macx(vy, vpk, kb.y, packed);
                s1x.macx(vx, vpk, ka.x, packed);
                s1y.macx(vy, vpk, ka.y, packed);
            }
        }
        const Prime P = a.pr[px];
        reinterpret_cast<ulonglong2*>(a.acc + ((size_t)((t * 2 + 0) * a.next + x) << log_n))[k2] =
            make_ulonglong2(s0x.reduce(P), s0y.reduce(P));
        reinterpret_cast<ulonglong2*>(a.acc + ((size_t)((t * 2 + 1) * a.next + x) << log_n))[k2] =
            make_ulonglong2(s1x.reduce(P), s1y.reduce(P));
        if (x < l1) {
            const u64* c0 = a.tab[t].addP0 + ((size_t)x << log_n);
            const ulonglong2 self = reinterpret_cast<const ulonglong2*>(c0)[k2];
            u64 sx = self.x, sy = self.y;
            for (int r = 0; r < a.n_steps; r++) {
                u64 vx, vy;
                load_pair_auto(c0, k2, (int)a.steps[r].galois, log_n, vx, vy);
                sx = add_mod(sx, vx, P.q);
                sy = add_mod(sy, vy, P.q);
            }
            reinterpret_cast<ulonglong2*>(a.c0sum + ((size_t)(t * l1 + x) << log_n))[k2] = make_ulonglong2(sx, sy);
        }
    }
}

// ---------------------------------------------------------------- 2-D forms, IPT items per thread

// Thread (blockIdx.x * 256 + threadIdx.x) = (item group, pair k2) with k2 fastest; blockIdx.y = limb x.
// Items t0 .. t0 + IPT - 1 of a group; a ragged last group repeats its last item and skips its stores.
// The data limbs (x <= level) use the multiply-accumulate MACD when every data prime has at most 50
// bits (a.split25), the special limbs and every other case MACS; the branch is uniform per block.

// Plain / fan-out: every item of a thread uses the key `key` and the automorphism `g` (IPT > 1 only
// when the items share them); FANOUT reads item t's digits from source src_of[t] through its
// automorphism.
template <class MAC, int IPT, bool FANOUT, bool PK>
__device__ __forceinline__ void inner2_body(const InnerArgs& a, int x, int k2, int t0) {
    const int log_n = a.log_n, hl = log_n - 1;
    const int l1 = a.level + 1;
    const int px = x < l1 ? x : x + (a.L - a.level);
    const int own = x < l1 ? x / a.alpha : -1;
    constexpr bool packed = PK;  // keys_packed && x < l1, fixed per block
    const u64* key = IPT > 1 ? a.shared_key : a.tab[t0].key;
    const int g = IPT > 1 ? (int)a.shared_galois : (int)a.tab[t0].galois;
    const ulonglong2* kr = reinterpret_cast<const ulonglong2*>(key) + ((size_t)px << hl) + k2;
    const size_t kstride = (size_t)a.n_ext << hl;
    // digit rows of each item (pair units); the own digit's limb is the item's input
    const ulonglong2* ext0[IPT];
    const ulonglong2* ownr[IPT];
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        const int t = min(t0 + i, a.items - 1);
        const int st = FANOUT ? a.src_of[t] : t;
        ext0[i] = reinterpret_cast<const ulonglong2*>(a.ext) + (((size_t)st * a.dn * a.next + x) << hl);
        ownr[i] = reinterpret_cast<const ulonglong2*>(a.tab[t].d) + ((size_t)x << hl);
    }
    const size_t dstride = (size_t)a.next << hl;
    int sp = k2;
    bool sw = false;
    if (g != 1) {
        const int src = auto_src(2 * k2, g, log_n);
        sp = src >> 1;
        sw = src & 1;
    }
    MAC s0x[IPT], s0y[IPT], s1x[IPT], s1y[IPT];
    for (int j = 0; j < a.dn; j++) {
        const bool vpk = packed && j != own;  // raised digits of data limbs are stored packed
        const ulonglong2 kb = kr[(size_t)(2 * j) * kstride];
        const ulonglong2 ka = kr[(size_t)(2 * j + 1) * kstride];
        // plain items read their raised digits unpermuted (the automorphism was applied in K1);
        // the own digit, and every digit of a fan-out item, is read through the automorphism
        const bool perm = FANOUT || j == own;
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const ulonglong2 v = (j == own ? ownr[i] : ext0[i] + (size_t)j * dstride)[perm ? sp : k2];
            const bool swp = perm && sw;
            const u64 vx = swp ? v.y : v.x, vy = swp ? v.x : v.y;
            s0x[i].macx(vx, vpk, kb.x, packed);
            s0y[i].macx(vy, vpk, kb.y, packed);
            s1x[i].macx(vx, vpk, ka.x, packed);
            s1y[i].macx(vy, vpk, ka.y, packed);
        }
    }
    const Prime P = a.pr[px];
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        const int t = t0 + i;
        if (t >= a.items) break;
        reinterpret_cast<ulonglong2*>(a.acc + ((size_t)((t * 2 + 0) * a.next + x) << log_n))[k2] =
            make_ulonglong2(s0x[i].reduce(P), s0y[i].reduce(P));
        reinterpret_cast<ulonglong2*>(a.acc + ((size_t)((t * 2 + 1) * a.next + x) << log_n))[k2] =
            make_ulonglong2(s1x[i].reduce(P), s1y[i].reduce(P));
    }
}

template <class MACD, class MACS, int IPT, bool FANOUT>
__global__ void __launch_bounds__(256) inner2_kernel(InnerArgs a) {
    const int hl = a.log_n - 1;
    const int x = blockIdx.y;
    const unsigned e = blockIdx.x * 256u + threadIdx.x;
    const int k2 = (int)(e & ((1u << hl) - 1u));
    const int t0 = (int)(e >> hl) * IPT;
    if (t0 >= a.items) return;
    const bool pk = a.keys_packed && x <= a.level;  // uniform per block
    if (x <= a.level && a.split25) {
        if (pk) inner2_body<MACD, IPT, FANOUT, true>(a, x, k2, t0);
        else inner2_body<MACD, IPT, FANOUT, false>(a, x, k2, t0);
    } else if (pk) {
        inner2_body<MACS, IPT, FANOUT, true>(a, x, k2, t0);
    } else {
        inner2_body<MACS, IPT, FANOUT, false>(a, x, k2, t0);
    }
}

template <class MAC, int IPT, bool SCALAR, bool PK>
__device__ __forceinline__ void hoist2_body(const InnerArgs& a, int x, int k2, int t0) {
    const int log_n = a.log_n, hl = log_n - 1;
    const int l1 = a.level + 1;
    const int px = x < l1 ? x : x + (a.L - a.level);
    const int own = x < l1 ? x / a.alpha : -1;
    constexpr bool packed = PK;  // keys_packed && x < l1, fixed per block
    const ulonglong2* ext0[IPT];
    const ulonglong2* ownr[IPT];
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        const int t = min(t0 + i, a.items - 1);
        ext0[i] = reinterpret_cast<const ulonglong2*>(a.ext) + (((size_t)t * a.dn * a.next + x) << hl);
        ownr[i] = reinterpret_cast<const ulonglong2*>(a.tab[t].d) + ((size_t)x << hl);
    }
    const size_t dstride = (size_t)a.next << hl;
    const size_t kstride = (size_t)a.n_ext << hl;
    const size_t koff = ((size_t)px << hl) + k2;
    MAC s0x[IPT], s0y[IPT], s1x[IPT], s1y[IPT];
    for (int r = 0; r < a.n_steps; r++) {
        const HoistStep st = a.steps[r];
        const int src = auto_src(2 * k2, (int)st.galois, log_n);
        const int sp = src >> 1;
        const bool sw = src & 1;
        const ulonglong2* kr = reinterpret_cast<const ulonglong2*>(st.key) + koff;
        for (int j = 0; j < a.dn; j++) {
            const bool vpk = packed && j != own;  // raised digits of data limbs are stored packed
            const ulonglong2 kb = kr[(size_t)(2 * j) * kstride];
            const ulonglong2 ka = kr[(size_t)(2 * j + 1) * kstride];
#pragma unroll
            for (int i = 0; i < IPT; i++) {
                const ulonglong2* row = j == own ? ownr[i] : ext0[i] + (size_t)j * dstride;
                u64 vx, vy;
                if (SCALAR) {  // slots 2 k2 and 2 k2 + 1 come from slots src and src ^ 1
                    const u64* r64 = reinterpret_cast<const u64*>(row);
                    vx = r64[src];
                    vy = r64[src ^ 1];
                } else {
                    const ulonglong2 v = row[sp];
                    vx = sw ? v.y : v.x;
                    vy = sw ? v.x : v.y;
                }
                s0x[i].macx(vx, vpk, kb.x, packed);
                s0y[i].macx(vy, vpk, kb.y, packed);
                s1x[i].macx(vx, vpk, ka.x, packed);
                s1y[i].macx(vy, vpk, ka.y, packed);
            }
        }
    }
    const Prime P = a.pr[px];
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        const int t = t0 + i;
        if (t >= a.items) break;
        reinterpret_cast<ulonglong2*>(a.acc + ((size_t)((t * 2 + 0) * a.next + x) << log_n))[k2] =
            make_ulonglong2(s0x[i].reduce(P), s0y[i].reduce(P));
        reinterpret_cast<ulonglong2*>(a.acc + ((size_t)((t * 2 + 1) * a.next + x) << log_n))[k2] =
            make_ulonglong2(s1x[i].reduce(P), s1y[i].reduce(P));
        if (x < l1) {
            const u64* c0 = a.tab[t].addP0 + ((size_t)x << log_n);
            const ulonglong2 self = reinterpret_cast<const ulonglong2*>(c0)[k2];
            u64 sx = self.x, sy = self.y;
            for (int r = 0; r < a.n_steps; r++) {
                u64 vx, vy;
                load_pair_auto(c0, k2, (int)a.steps[r].galois, log_n, vx, vy);
                sx = add_mod(sx, vx, P.q);
                sy = add_mod(sy, vy, P.q);
            }
            reinterpret_cast<ulonglong2*>(a.c0sum + ((size_t)(t * l1 + x) << log_n))[k2] = make_ulonglong2(sx, sy);
        }
    }
}

template <class MACD, class MACS, int IPT, bool SCALAR = false>
__global__ void __launch_bounds__(256) hoist2_kernel(InnerArgs a) {
    const int hl = a.log_n - 1;
    const int x = blockIdx.y;
    const unsigned e = blockIdx.x * 256u + threadIdx.x;
    const int k2 = (int)(e & ((1u << hl) - 1u));
    const int t0 = (int)(e >> hl) * IPT;
    if (t0 >= a.items) return;
    const bool pk = a.keys_packed && x <= a.level;  // uniform per block
    if (x <= a.level && a.split25) {
        if (pk) hoist2_body<MACD, IPT, SCALAR, true>(a, x, k2, t0);
        else hoist2_body<MACD, IPT, SCALAR, false>(a, x, k2, t0);
    } else if (pk) {
        hoist2_body<MACS, IPT, SCALAR, true>(a, x, k2, t0);
    } else {
        hoist2_body<MACS, IPT, SCALAR, false>(a, x, k2, t0);
    }
}

inline unsigned grid1(size_t work) {
    size_t b = (work + 255) / 256;
    return (unsigned)std::min<size_t>(std::max<size_t>(b, 1), (size_t)1 << 30);
}

inline dim3 grid2(const InnerArgs& a, int ipt) {
    const size_t groups = (size_t)(a.items + ipt - 1) / ipt;
    const size_t threads = groups << (a.log_n - 1);
    return dim3((unsigned)((threads + 255) / 256), (unsigned)a.next);
}

}  // namespace

void launch_ks_inner(const InnerArgs& a0, bool fanout, int variant, int max_data_prime_bits, cudaStream_t s) {
    if (a0.items == 0) return;
    InnerArgs a = a0;
    if (variant <= INNER_V0 || variant >= INNER_N_VARIANTS) {
        if (fanout)
            inner_v0_kernel<true><<<grid1((size_t)a.items * a.next << (a.log_n - 1)), 256, 0, s>>>(a);
        else
            inner_v0_kernel<false><<<grid1((size_t)a.items * a.next << (a.log_n - 1)), 256, 0, s>>>(a);
        CK(cudaGetLastError());
        return;
    }
    // split at bit 25 needs data primes below 2^50 and at most 2^13 terms per sum
    a.split25 = max_data_prime_bits <= 50 && a.dn <= (1 << 13);
    const bool two = (variant == INNER_S2 || variant == INNER_S2L) && !fanout && a.shared_key;
#define L2(MD, MS, I, F) inner2_kernel<MD, MS, I, F><<<grid2(a, I), 256, 0, s>>>(a)
    switch (variant) {
        case INNER_C1:
            if (fanout) L2(MacC, MacC, 1, true);
            else L2(MacC, MacC, 1, false);
            break;
        case INNER_P1:
            if (fanout) L2(MacP32, MacP32, 1, true);
            else L2(MacP32, MacP32, 1, false);
            break;
        default:  // S1, S2
            if (fanout) L2(MacS25, MacP32, 1, true);
            else if (two) L2(MacS25, MacP32, 2, false);
            else L2(MacS25, MacP32, 1, false);
            break;
    }
#undef L2
    CK(cudaGetLastError());
}

void launch_ks_hoist_inner(const InnerArgs& a0, int variant, int max_data_prime_bits, cudaStream_t s) {
    if (a0.items == 0) return;
    InnerArgs a = a0;
    if (variant <= INNER_V0 || variant >= INNER_N_VARIANTS) {
        hoist_v0_kernel<<<grid1((size_t)a.items * a.next << (a.log_n - 1)), 256, 0, s>>>(a);
        CK(cudaGetLastError());
        return;
    }
    a.split25 = max_data_prime_bits <= 50 && (long long)a.dn * a.n_steps <= (1 << 13);
#define H2(MD, MS, I) hoist2_kernel<MD, MS, I><<<grid2(a, I), 256, 0, s>>>(a)
    switch (variant) {
        case INNER_C1: H2(MacC, MacC, 1); break;
        case INNER_P1: H2(MacP32, MacP32, 1); break;
        case INNER_S2: H2(MacS25, MacP32, 2); break;
        case INNER_S2L: hoist2_kernel<MacS25, MacP32, 2, true><<<grid2(a, 2), 256, 0, s>>>(a); break;
        default: H2(MacS25, MacP32, 1); break;
    }
#undef H2
    CK(cudaGetLastError());
}

}  // namespace fhe

// ctx.cu — context set-up (primes, NTT twiddles, RNS conversion constants,
// encoding tables), host-side seeded sampling, key generation, encoding,
// encryption and decryption, and the C ABI of the ciphertext primitives.
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "core.cuh"
#include "ks_inner.cuh"

namespace fhe {

// ============================================================================ errors

void fail(int code, const std::string& msg) { throw FheException(code, msg); }

void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            fail(FHE_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
        }
        fail(FHE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

// ============================================================================ device memory

template <typename T>
static T* dalloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    CK(cudaMalloc(&p, count * sizeof(T)));
    return (T*)p;
}

template <typename T>
static T* dupload(const std::vector<T>& v) {
    T* p = dalloc<T>(v.size());
    CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

void* Ctx::scratch_bytes(const std::string& name, size_t bytes) {
    DeviceBuf& b = scratch[name];
    if (b.bytes < bytes) {
        if (b.p) {
            CK(cudaDeviceSynchronize());  // the old buffer may still be in use by queued work
            CK(cudaFree(b.p));
            b.p = nullptr;
            b.bytes = 0;
        }
        size_t want = bytes + bytes / 8;
        CK(cudaMalloc(&b.p, want));
        b.bytes = want;
    }
    return b.p;
}

u64* Ctx::scratch_u64(const std::string& name, size_t words) {
    return (u64*)scratch_bytes(name, words * sizeof(u64));
}

Ctx::~Ctx() {
    cudaSetDevice(device);
    cudaDeviceSynchronize();
    void* bufs[] = {d_primes, d_psi, d_psi_s, d_ipsi, d_ipsi_s, d_ninv, d_tw, d_itw, d_tw2, d_itw2, d_up_ninv, d_down_ninv, d_resc, d_up_inv, d_up_hat,
                    d_down_inv, d_down_hat, d_pinv, d_pmod, d_fd_ninv, d_fd_hat, d_fd_minv, d_fd_pq, d_cos, d_sin, d_pow5, d_sk, d_pk, rlk.d};
    for (void* p : bufs)
        if (p) cudaFree(p);
    for (auto& kv : rot)
        if (kv.second.d) cudaFree(kv.second.d);
    for (auto& kv : scratch)
        if (kv.second.p) cudaFree(kv.second.p);
}

// ============================================================================ primes

static bool is_prime_u64(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : bases) {
        if (n == b) return true;
        if (n % b == 0) return false;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        s++;
    }
    for (u64 b : bases) {
        u64 x = h_pow(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int r = 1; r < s && composite; r++) {
            x = h_mul(x, x, n);
            if (x == n - 1) composite = false;
        }
        if (composite) return false;
    }
    return true;
}

// largest unused prime below 2^bits that is 1 mod 2N, per entry, in order
static std::vector<u64> choose_primes(int log_n, const std::vector<int>& bits) {
    const u64 two_n = (u64)2 << log_n;
    std::vector<u64> out;
    for (int b : bits) {
        u64 c = ((u64)1 << b) + 1 - two_n;
        for (;;) {
            if (c < two_n) fail(FHE_ERR_INVALID_ARG, "no prime of the requested size");
            bool used = false;
            for (u64 x : out) used = used || x == c;
            if (!used && is_prime_u64(c)) break;
            c -= two_n;
        }
        out.push_back(c);
    }
    return out;
}

// a primitive 2N-th root of unity modulo q
static u64 primitive_root_2n(u64 q, int log_n) {
    const u64 two_n = (u64)2 << log_n;
    for (u64 g = 2; g < 1000000; g++) {
        u64 r = h_pow(g, (q - 1) / two_n, q);
        if (h_pow(r, two_n >> 1, q) == q - 1) return r;
    }
    fail(FHE_ERR_INVALID_ARG, "no primitive root found");
}

static unsigned bit_reverse(unsigned x, int bits) {
    unsigned r = 0;
    for (int i = 0; i < bits; i++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

static Prime make_prime(u64 q) {
    Prime p;
    p.q = q;
    p.b = 64 - __builtin_clzll(q);
    p.mu = (u64)(((u128)1 << (2 * p.b)) / q);
    p.one_s = h_shoup(1, q);
    p.pad = 0;
    return p;
}

// ============================================================================ sampling (SplitMix64 streams)

static constexpr u64 kGamma = 0x9E3779B97F4A7C15ULL;
enum Purpose : u64 {
    kSecret = 1, kPkA = 2, kPkE = 3, kEvkA = 4, kEvkE = 5, kEncV = 6, kEncE0 = 7, kEncE1 = 8,
    kSeededA = 9, kSeededE = 10  // key-holder encryption with a regenerable c1 (object = ciphertext id)
};

static inline u64 mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Stream key: h <- mix64((h xor f) + gamma) over (purpose, object, poly, limb), from h = seed.
static u64 stream_key(u64 seed, u64 purpose, u64 obj, u64 poly, u64 limb) {
    u64 h = seed;
    const u64 f[4] = {purpose, obj, poly, limb};
    for (u64 x : f) h = mix64((h ^ x) + kGamma);
    return h;
}

// SplitMix64 generator with state h: the c-th output (c = 1, 2, ...) is mix64(h + c*gamma).
struct SplitMix {
    u64 h;
    u64 c = 0;
    explicit SplitMix(u64 key) : h(key) {}
    u64 next() { return mix64(h + (++c) * kGamma); }
};

static void sample_uniform(u64 key, u64 q, u64* out, int n) {
    SplitMix g(key);
    const u64 bound = (u64)((((u128)1) << 64) / q * q);
    for (int i = 0; i < n;) {
        u64 x = g.next();
        if (x < bound) out[i++] = x % q;
    }
}

static void sample_ternary(u64 key, int8_t* out, int n) {
    SplitMix g(key);
    const u64 bound = (u64)((((u128)1) << 64) / 3 * 3);
    for (int i = 0; i < n;) {
        u64 x = g.next();
        if (x < bound) out[i++] = (int8_t)((int)(x % 3) - 1);
    }
}

struct GaussTable {
    u64 t[19];
};

static GaussTable gauss_table(double sigma) {
    GaussTable T;
    const double two_sigma_sq = 2.0 * sigma * sigma;
    double rho[20];
    for (int x = 0; x < 20; x++) rho[x] = std::exp(-(double)(x * x) / two_sigma_sq);
    double tail = 0.0;
    for (int x = 1; x < 20; x++) tail = tail + rho[x];
    const double norm = rho[0] + 2.0 * tail;
    double cdf = 0.0;
    for (int k = 0; k < 19; k++) {
        double pk = k == 0 ? rho[0] / norm : 2.0 * rho[k] / norm;
        cdf = cdf + pk;
        T.t[k] = (u64)(cdf * 9223372036854775808.0);
    }
    return T;
}

static void sample_gaussian(u64 key, const GaussTable& T, int8_t* out, int n) {
    SplitMix g(key);
    for (int i = 0; i < n; i++) {
        u64 x = g.next();
        u64 u = x >> 1;
        int mag = 0;
        for (int k = 0; k < 19; k++) mag += u >= T.t[k];
        out[i] = (int8_t)((x & 1) ? -mag : mag);
    }
}

// ============================================================================ context creation

static void build_tables(Ctx& c) {
    const int n = c.n, L = c.L, ne = c.n_ext, A = c.alpha;
    std::vector<u64> psi((size_t)ne * n), psi_s(psi.size()), ipsi(psi.size()), ipsi_s(psi.size());
    std::vector<u64> ninv(2 * ne);
    for (int t = 0; t < ne; t++) {
        u64 q = c.primes[t];
        u64 w = primitive_root_2n(q, c.log_n);
        u64 wi = h_inv(w, q);
        std::vector<u64> pw(n), ipw(n);
        pw[0] = ipw[0] = 1;
        for (int i = 1; i < n; i++) {
            pw[i] = h_mul(pw[i - 1], w, q);
            ipw[i] = h_mul(ipw[i - 1], wi, q);
        }
        for (int i = 0; i < n; i++) {
            unsigned r = bit_reverse((unsigned)i, c.log_n);
            size_t o = (size_t)t * n + i;
            psi[o] = pw[r];
            psi_s[o] = h_shoup(pw[r], q);
            ipsi[o] = ipw[r];
            ipsi_s[o] = h_shoup(ipw[r], q);
        }
        u64 ni = h_inv((u64)n % q, q);
        ninv[2 * t] = ni;
        ninv[2 * t + 1] = h_shoup(ni, q);
    }
    c.d_psi = dupload(psi);
    c.d_psi_s = dupload(psi_s);
    c.d_ipsi = dupload(ipsi);
    c.d_ipsi_s = dupload(ipsi_s);
    c.d_ninv = dupload(ninv);
    std::vector<ulonglong2> tw((size_t)ne * n), itw(tw.size());
    for (size_t i = 0; i < tw.size(); i++) {
        tw[i] = make_ulonglong2(psi[i], psi_s[i]);
        itw[i] = make_ulonglong2(ipsi[i], ipsi_s[i]);
    }
    c.d_tw = dupload(tw);
    c.d_itw = dupload(itw);
    // transposed row-pass tables of the two-pass transform (N >= 2^14)
    c.ntt_s1 = c.log_n >= 14 ? (c.log_n == 15 ? 7 : c.log_n / 2) : 0;
    if (c.ntt_s1) {
        const int S1 = c.ntt_s1, N1 = 1 << S1, LM2 = c.log_n - S1;
        std::vector<ulonglong2> t2((size_t)ne * n, make_ulonglong2(0, 0)), it2(t2.size(), make_ulonglong2(0, 0));
        for (int t = 0; t < ne; t++) {
            size_t o = (size_t)t * n;
            for (int sp = 0; sp < LM2; sp++)
                for (int g = 0; g < (1 << sp); g++)
                    for (int r = 0; r < N1; r++) {
                        size_t src = (size_t)t * n + ((size_t)1 << (S1 + sp)) + ((size_t)r << sp) + g;
                        t2[o] = make_ulonglong2(psi[src], psi_s[src]);
                        it2[o] = make_ulonglong2(ipsi[src], ipsi_s[src]);
                        o++;
                    }
        }
        c.d_tw2 = dupload(t2);
        c.d_itw2 = dupload(it2);
    }

    // rescale: q_l^-1 mod q_i
    std::vector<u64> resc((size_t)2 * (L + 1) * (L + 1), 0);
    for (int l = 1; l <= L; l++)
        for (int i = 0; i < l; i++) {
            u64 v = h_inv(c.primes[l] % c.primes[i], c.primes[i]);
            resc[2 * ((size_t)l * (L + 1) + i)] = v;
            resc[2 * ((size_t)l * (L + 1) + i) + 1] = h_shoup(v, c.primes[i]);
        }
    c.d_resc = dupload(resc);

    // ModUp: per level l, limb i <= l belongs to digit j = i / alpha = [j A, min((j+1)A, l+1))
    std::vector<u64> up_inv((size_t)2 * (L + 1) * (L + 1), 0);
    std::vector<u64> up_hat((size_t)2 * (L + 1) * (L + 1) * ne, 0);
    for (int l = 0; l <= L; l++)
        for (int i = 0; i <= l; i++) {
            int j = i / A;
            int lo = j * A, hi = std::min((j + 1) * A, l + 1);
            u64 qi = c.primes[i];
            u64 hat_i = 1;
            for (int i2 = lo; i2 < hi; i2++)
                if (i2 != i) hat_i = h_mul(hat_i, c.primes[i2] % qi, qi);
            u64 inv = h_inv(hat_i, qi);
            size_t o = (size_t)l * (L + 1) + i;
            up_inv[2 * o] = inv;
            up_inv[2 * o + 1] = h_shoup(inv, qi);
            for (int t = 0; t < ne; t++) {
                u64 p = c.primes[t];
                u64 h = 1 % p;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) h = h_mul(h, c.primes[i2] % p, p);
                up_hat[2 * (o * ne + t)] = h;
                up_hat[2 * (o * ne + t) + 1] = h_shoup(h, p);
            }
        }
    c.d_up_inv = dupload(up_inv);
    c.d_up_hat = dupload(up_hat);
    std::vector<u64> up_ninv(up_inv.size(), 0);
    for (int l = 0; l <= L; l++)
        for (int i = 0; i <= l; i++) {
            size_t o = (size_t)l * (L + 1) + i;
            u64 qi = c.primes[i];
            u64 v = h_mul(up_inv[2 * o], h_inv((u64)n % qi, qi), qi);
            up_ninv[2 * o] = v;
            up_ninv[2 * o + 1] = h_shoup(v, qi);
        }
    c.d_up_ninv = dupload(up_ninv);

    // ModDown constants
    std::vector<u64> dinv(2 * A), dhat((size_t)2 * A * (L + 1)), pinv(2 * (L + 1)), pmod(L + 1);
    for (int k = 0; k < A; k++) {
        u64 pk = c.primes[L + 1 + k];
        u64 h = 1;
        for (int k2 = 0; k2 < A; k2++)
            if (k2 != k) h = h_mul(h, c.primes[L + 1 + k2] % pk, pk);
        u64 inv = h_inv(h, pk);
        dinv[2 * k] = inv;
        dinv[2 * k + 1] = h_shoup(inv, pk);
        for (int i = 0; i <= L; i++) {
            u64 q = c.primes[i];
            u64 hq = 1;
            for (int k2 = 0; k2 < A; k2++)
                if (k2 != k) hq = h_mul(hq, c.primes[L + 1 + k2] % q, q);
            dhat[2 * ((size_t)k * (L + 1) + i)] = hq;
            dhat[2 * ((size_t)k * (L + 1) + i) + 1] = h_shoup(hq, q);
        }
    }
    for (int i = 0; i <= L; i++) {
        u64 q = c.primes[i];
        u64 P = 1;
        for (int k = 0; k < A; k++) P = h_mul(P, c.primes[L + 1 + k] % q, q);
        pmod[i] = P;
        u64 inv = h_inv(P, q);
        pinv[2 * i] = inv;
        pinv[2 * i + 1] = h_shoup(inv, q);
    }
    c.d_down_inv = dupload(dinv);
    std::vector<u64> dninv(2 * A);
    for (int k = 0; k < A; k++) {
        u64 pk = c.primes[L + 1 + k];
        u64 v = h_mul(dinv[2 * k], h_inv((u64)n % pk, pk), pk);
        dninv[2 * k] = v;
        dninv[2 * k + 1] = h_shoup(v, pk);
    }
    c.d_down_ninv = dupload(dninv);
    c.d_down_hat = dupload(dhat);
    c.d_pinv = dupload(pinv);
    c.d_pmod = dupload(pmod);

    // fused ModDown + rescale at level l: divide by M' = P q_l; sources m_s = p_s (s < alpha), q_l (s = alpha)
    {
        const int S = A + 1;
        std::vector<u64> fninv((size_t)2 * (L + 1) * S, 0), fhat((size_t)2 * (L + 1) * S * (L + 1), 0);
        std::vector<u64> fminv((size_t)2 * (L + 1) * (L + 1), 0), fpq((size_t)2 * (L + 1), 0);
        for (int l = 1; l <= L; l++) {
            auto src = [&](int sidx) { return sidx < A ? c.primes[L + 1 + sidx] : c.primes[l]; };
            for (int sidx = 0; sidx < S; sidx++) {
                const u64 m = src(sidx);
                u64 hat_m = 1;  // (M' / m) mod m
                for (int s2 = 0; s2 < S; s2++)
                    if (s2 != sidx) hat_m = h_mul(hat_m, src(s2) % m, m);
                const u64 v = h_mul(h_inv(hat_m, m), h_inv((u64)n % m, m), m);
                fninv[2 * ((size_t)l * S + sidx)] = v;
                fninv[2 * ((size_t)l * S + sidx) + 1] = h_shoup(v, m);
                for (int i = 0; i < l; i++) {
                    const u64 q = c.primes[i];
                    u64 h = 1;
                    for (int s2 = 0; s2 < S; s2++)
                        if (s2 != sidx) h = h_mul(h, src(s2) % q, q);
                    const size_t o = 2 * (((size_t)l * S + sidx) * (L + 1) + i);
                    fhat[o] = h;
                    fhat[o + 1] = h_shoup(h, q);
                }
            }
            for (int i = 0; i < l; i++) {
                const u64 q = c.primes[i];
                const u64 inv = h_inv(h_mul(pmod[i], c.primes[l] % q, q), q);
                fminv[2 * ((size_t)l * (L + 1) + i)] = inv;
                fminv[2 * ((size_t)l * (L + 1) + i) + 1] = h_shoup(inv, q);
            }
            fpq[2 * l] = pmod[l];
            fpq[2 * l + 1] = h_shoup(pmod[l], c.primes[l]);
        }
        c.d_fd_ninv = dupload(fninv);
        c.d_fd_hat = dupload(fhat);
        c.d_fd_minv = dupload(fminv);
        c.d_fd_pq = dupload(fpq);
    }

    // encoding: cos / sin (pi e / N) for e < 2N, computed by the host libm; 5^t mod 2N
    std::vector<double> cs(2 * (size_t)n), sn(2 * (size_t)n);
    for (int e = 0; e < 2 * n; e++) {
        cs[e] = std::cos(M_PI * (double)e / (double)n);
        sn[e] = std::sin(M_PI * (double)e / (double)n);
    }
    c.d_cos = dupload(cs);
    c.d_sin = dupload(sn);
    std::vector<u32> p5(c.slots);
    u64 x = 1;
    for (int t = 0; t < c.slots; t++) {
        p5[t] = (u32)x;
        x = x * 5 % (2 * (u64)n);
    }
    c.d_pow5 = dupload(p5);
}

// ============================================================================ kernels local to this file

namespace {

constexpr int kT = 256;
inline unsigned blocks_for(size_t work) {
    size_t b = (work + kT - 1) / kT;
    return (unsigned)std::min<size_t>(std::max<size_t>(b, 1), 1u << 30);
}

// pk0 = -a*s + e (evaluation domain), limbs [0, l1)
__global__ void pk_kernel(u64* pk0, const u64* __restrict__ a, const u64* __restrict__ s,
                          const u64* __restrict__ e, int limbs, int log_n, const Prime* __restrict__ pr) {
    const size_t total = (size_t)limbs << log_n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int limb = (int)(i >> log_n);
        const Prime P = pr[limb];
        u64 as = mul_mod(a[i], s[i], P);
        pk0[i] = add_mod(sub_mod(0, as, P.q), e[i], P.q);
    }
}

// b = -a*s + e + [limb in digit j] (P mod q_limb) * s'   over the extended basis
__global__ void evk_kernel(u64* b, const u64* __restrict__ a, const u64* __restrict__ s,
                           const u64* __restrict__ e, const u64* __restrict__ s2, int n_ext, int L,
                           int lo, int hi, int log_n, const Prime* __restrict__ pr,
                           const u64* __restrict__ pmod) {
    const size_t total = (size_t)n_ext << log_n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int limb = (int)(i >> log_n);
        const Prime P = pr[limb];
        u64 v = add_mod(sub_mod(0, mul_mod(a[i], s[i], P), P.q), e[i], P.q);
        if (limb >= lo && limb < hi && limb <= L) v = add_mod(v, mul_mod(pmod[limb], s2[i], P), P.q);
        b[i] = v;
    }
}

// The data-prime rows (limbs 0..L) of one key digit's two halves, stored split at bit 25.
__global__ void key_pack_kernel(u64* kb, u64* ka, int L, int log_n) {
    const size_t total = (size_t)(L + 1) << log_n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        kb[i] = key_pack(kb[i]);
        ka[i] = key_pack(ka[i]);
    }
}

__global__ void square_kernel(u64* out, const u64* __restrict__ s, int limbs, int log_n,
                              const Prime* __restrict__ pr) {
    const size_t total = (size_t)limbs << log_n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = mul_mod(s[i], s[i], pr[i >> log_n]);
}

// ct0 = v*pk0 + c0, ct1 = v*pk1 + c1 for `count` items (inputs compact [count][l1][N])
__global__ void enc_combine_kernel(u64* ct, size_t ct_stride, size_t part_stride,
                                   const u64* __restrict__ v, const u64* __restrict__ c0,
                                   const u64* __restrict__ c1, const u64* __restrict__ pk0,
                                   const u64* __restrict__ pk1, int count, int l1, int log_n,
                                   const Prime* __restrict__ pr) {
    const size_t per = (size_t)l1 << log_n;
    const size_t total = (size_t)count * per;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        size_t t = i / per, r = i % per;
        int limb = (int)(r >> log_n);
        const Prime P = pr[limb];
        u64 vv = v[i];
        ct[t * ct_stride + r] = add_mod(mul_mod(vv, pk0[r], P), c0[i], P.q);
        ct[t * ct_stride + part_stride + r] = add_mod(mul_mod(vv, pk1[r], P), c1[i], P.q);
    }
}

__device__ __forceinline__ u64 mix64_dev(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Row r: dst[k] = the first of the stream outputs x_{jN + k} = mix64(h + (jN + k + 1) gamma),
// j < kSeededTries, below floor(2^64/q) q, reduced mod q (the last one if none is).
__global__ void seeded_uniform_kernel(const SeedRow* __restrict__ rows, int n_rows, int log_n,
                                      const Prime* __restrict__ pr) {
    const size_t n = (size_t)1 << log_n;
    const size_t total = (size_t)n_rows << log_n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const SeedRow r = rows[e >> log_n];
        const size_t k = e & (n - 1);
        const Prime P = pr[r.prime];
        const u64 bound = (u64)0 - ((u64)0 - P.q * P.one_s);  // 2^64 - (2^64 mod q)
        u64 x = 0;
        for (int j = 0; j < kSeededTries; j++) {
            x = mix64_dev(r.h + ((u64)j * n + k + 1) * 0x9E3779B97F4A7C15ULL);
            if (x < bound) break;
        }
        const u64 t = x - __umul64hi(x, P.one_s) * P.q;  // in [0, 2q)
        r.dst[k] = t >= P.q ? t - P.q : t;
    }
}

// c0[t][i] = me[t][i] - a[t][i] * s[i] (evaluation domain), compact [count][l1][N] buffers.
__global__ void seeded_c0_kernel(u64* out, const u64* __restrict__ me, const u64* __restrict__ a,
                                 const u64* __restrict__ sk, size_t total, int l1, int log_n, const Prime* __restrict__ pr) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t row = e >> log_n, k = e & (((size_t)1 << log_n) - 1);
        const int i = (int)(row % l1);
        const Prime P = pr[i];
        out[e] = sub_mod(me[e], mul_mod(a[e], sk[((size_t)i << log_n) + k], P), P.q);
    }
}

__global__ void add_compact_kernel(u64* out, const u64* __restrict__ a, size_t total, int l1, int log_n,
                                   const Prime* __restrict__ pr) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int limb = (int)((i >> log_n) % l1);
        out[i] = add_mod(out[i], a[i], pr[limb].q);
    }
}

// Encoding: coefficient j of vector v = rint(factor * sum_t val_t * cos(pi (j 5^t mod 2N) / N)),
// the sum over the vector's non-zero slots in ascending slot order, each step an
// IEEE double multiply then add (no fused multiply-add).
__global__ void encode_kernel(i64* out, const int* __restrict__ idx, const double* __restrict__ val,
                              const int* __restrict__ offsets, const double* __restrict__ cos_tab,
                              const u32* __restrict__ pow5, int log_n, double factor) {
    __shared__ u32 s_p[256];
    __shared__ double s_v[256];
    const int v = blockIdx.y;
    const int n = 1 << log_n;
    const u32 mask = 2u * n - 1u;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int beg = offsets[v], end = offsets[v + 1];
    double acc = 0.0;
    for (int c0 = beg; c0 < end; c0 += 256) {
        int cnt = min(256, end - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            s_p[t] = pow5[idx[c0 + t]];
            s_v[t] = val[c0 + t];
        }
        __syncthreads();
        if (j < n) {
            for (int t = 0; t < cnt; t++) {
                u32 e = (u32)(((unsigned long long)j * s_p[t]) & mask);
                acc = __dadd_rn(acc, __dmul_rn(s_v[t], cos_tab[e]));
            }
        }
    }
    if (j < n) out[(size_t)v * n + j] = __double2ll_rn(__dmul_rn(acc, factor));
}

// decryption: m_i = c0_i + c1_i * s_i for limbs < nl (evaluation domain)
__global__ void dec_kernel(u64* m, const u64* __restrict__ ct, size_t part_stride, const u64* __restrict__ s,
                           int nl, int log_n, const Prime* __restrict__ pr) {
    const size_t total = (size_t)nl << log_n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const Prime P = pr[i >> log_n];
        m[i] = add_mod(ct[i], mul_mod(ct[part_stride + i], s[i], P), P.q);
    }
}

// centred CRT lift of 1 or 2 limbs to a double
__global__ void crt_kernel(double* out, const u64* __restrict__ m, int nl, int log_n, u64 q0, u64 q1,
                           u64 q0inv_mod_q1) {
    const int n = 1 << log_n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (nl == 1) {
            u64 x = m[j];
            out[j] = x > q0 / 2 ? -(double)(q0 - x) : (double)x;
        } else {
            u64 x0 = m[j], x1 = m[n + j];
            u64 d = x1 >= x0 % q1 ? x1 - x0 % q1 : x1 + q1 - x0 % q1;
            u64 k = (u64)(((u128)d * q0inv_mod_q1) % q1);
            u128 v = (u128)k * q0 + x0;
            u128 Q = (u128)q0 * q1;
            out[j] = v > Q / 2 ? -(double)(Q - v) : (double)v;
        }
    }
}

// exact centred lift of 1 or 2 limbs to int64 (refresh); flags values outside int64
__global__ void crt_int64_kernel(i64* out, const u64* __restrict__ m, int nl, int log_n, u64 q0, u64 q1,
                                 u64 q0inv_mod_q1, int* overflow) {
    const int n = 1 << log_n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (nl == 1) {
            u64 x = m[j];
            out[j] = x > q0 / 2 ? -(i64)(q0 - x) : (i64)x;
        } else {
            u64 x0 = m[j], x1 = m[n + j];
            u64 d = x1 >= x0 % q1 ? x1 - x0 % q1 : x1 + q1 - x0 % q1;
            u64 k = (u64)(((u128)d * q0inv_mod_q1) % q1);
            u128 v = (u128)k * q0 + x0;
            u128 Q = (u128)q0 * q1;
            bool neg = v > Q / 2;
            u128 mag = neg ? Q - v : v;
            if (mag >> 63) {
                atomicOr(overflow, 1);
                out[j] = 0;
            } else {
                out[j] = neg ? -(i64)mag : (i64)mag;
            }
        }
    }
}

// z_t = sum_j m_j cos(pi (j 5^t mod 2N) / N) / Delta, one block per slot
__global__ void decode_kernel(double* z, const double* __restrict__ m, const double* __restrict__ cos_tab,
                              const u32* __restrict__ pow5, int log_n, double inv_scale, int n_slots) {
    __shared__ double red[256];
    const int t = blockIdx.x;
    if (t >= n_slots) return;
    const int n = 1 << log_n;
    const u32 mask = 2u * n - 1u;
    const u32 p = pow5[t];
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) acc += m[j] * cos_tab[((u64)j * p) & mask];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) z[t] = red[0] * inv_scale;
}

}  // namespace

// ============================================================================ internal API

const EvalKey& rotation_key(const Ctx& c, int step) {
    int g = c.galois(step);
    auto it = c.rot.find(g);
    if (it == c.rot.end()) fail(FHE_ERR_MISSING_KEY, "no rotation key for step " + std::to_string(step));
    return it->second;
}

void encode_many_device(Ctx& c, const std::vector<int>& idx, const std::vector<double>& val,
                        const std::vector<int>& offsets, i64* out_dev, cudaStream_t s) {
    const int count = (int)offsets.size() - 1;
    if (count <= 0) return;
    const size_t nz = idx.size();
    int* d_idx = (int*)c.scratch_bytes("enc_idx", sizeof(int) * (nz + 1));
    double* d_val = (double*)c.scratch_bytes("enc_val", sizeof(double) * (nz + 1));
    int* d_off = (int*)c.scratch_bytes("enc_off", sizeof(int) * offsets.size());
    if (nz) {
        CK(cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_val, val.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemcpyAsync(d_off, offsets.data(), sizeof(int) * offsets.size(), cudaMemcpyHostToDevice, s));
    const double factor = std::ldexp(1.0, c.log_scale + 1 - c.log_n);  // 2 Delta / N
    for (int v0 = 0; v0 < count; v0 += 65535) {
        int cnt = std::min(65535, count - v0);
        dim3 grid((c.n + 255) / 256, cnt);
        {
            LaunchScope _ls(c.prof, K_ENCODE, 8.0 * cnt * c.n + 12.0 * nz, s);
            encode_kernel<<<grid, 256, 0, s>>>(out_dev + (size_t)v0 * c.n, d_idx, d_val, d_off + v0, c.d_cos,
                                               c.d_pow5, c.log_n, factor);
            CK(cudaGetLastError());
        }
    }
    // the host vectors may be released once the copies have been consumed
    CK(cudaStreamSynchronize(s));
}

void encode_sparse_device(Ctx& c, const std::vector<std::pair<int, double>>& nz, i64* out_dev,
                          cudaStream_t s) {
    std::vector<int> idx;
    std::vector<double> val;
    for (auto& p : nz)
        if (p.second != 0.0) {
            idx.push_back(p.first);
            val.push_back(p.second);
        }
    encode_many_device(c, idx, val, {0, (int)idx.size()}, out_dev, s);
}

void encode_device(Ctx& c, const double* host_slots, size_t n_slots, i64* out_dev, cudaStream_t s) {
    if (n_slots > (size_t)c.slots) fail(FHE_ERR_INVALID_ARG, "more values than slots");
    std::vector<std::pair<int, double>> nz;
    for (size_t t = 0; t < n_slots; t++)
        if (host_slots[t] != 0.0) nz.push_back({(int)t, host_slots[t]});
    encode_sparse_device(c, nz, out_dev, s);
}

void materialize_plain(Ctx& c, const i64* m_dev, size_t m_stride, int count, int limbs, u64* out,
                       size_t out_stride, cudaStream_t s) {
    k_int_to_rns(c, out, out_stride, m_dev, m_stride, count, limbs, s);
    ntt_forward(c, poly_batch(out, out_stride, 0, count, 1, 0, limbs), s);
}

u64 seeded_key(const Ctx& c, u64 obj, int limb) { return stream_key(c.seed, kSeededA, obj, 0, (u64)limb); }

void seeded_uniform_device(Ctx& c, const std::vector<SeedRow>& rows, cudaStream_t s) {
    if (rows.empty()) return;
    const SeedRow* d = c.arena.push_vec(rows, s);
    LaunchScope _ls(c.prof, K_ELEMENTWISE, 8.0 * rows.size() * c.n, s);
    seeded_uniform_kernel<<<blocks_for(rows.size() * (size_t)c.n), kT, 0, s>>>(d, (int)rows.size(), c.log_n,
                                                                                c.d_primes);
    CK(cudaGetLastError());
}

void encrypt_seeded_device(Ctx& c, const i64* m_dev, size_t m_stride, int count, int level,
                           const std::vector<u64>& objs, u64* c0_out, cudaStream_t s) {
    if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
    if (level < 0 || level > c.L) fail(FHE_ERR_INVALID_ARG, "level out of range");
    const int n = c.n, l1 = level + 1;
    const GaussTable T = gauss_table(c.sigma);
    const int chunk = 32;
    std::vector<int8_t> host((size_t)chunk * n);
    for (int t0 = 0; t0 < count; t0 += chunk) {
        const int cnt = std::min(chunk, count - t0);
        for (int t = 0; t < cnt; t++)
            sample_gaussian(stream_key(c.seed, kSeededE, objs[t0 + t], 0, 0), T, host.data() + (size_t)t * n, n);
        int8_t* d_e = (int8_t*)c.scratch_bytes("senc_e", (size_t)chunk * n);
        u64* me = c.scratch_u64("senc_me", (size_t)chunk * l1 * n);
        u64* ee = c.scratch_u64("senc_ee", (size_t)chunk * l1 * n);
        u64* a = c.scratch_u64("senc_a", (size_t)chunk * l1 * n);
        CK(cudaMemcpyAsync(d_e, host.data(), (size_t)cnt * n, cudaMemcpyHostToDevice, s));
        const size_t st = (size_t)l1 * n;
        k_int_to_rns(c, me, st, m_dev + (size_t)t0 * m_stride, m_stride, cnt, l1, s);
        k_int8_to_rns(c, ee, st, d_e, (size_t)n, cnt, l1, 1 << 30, 0, s);
        {
            LaunchScope _ls(c.prof, K_ELEMENTWISE, 24.0 * cnt * st, s);
            add_compact_kernel<<<blocks_for((size_t)cnt * st), kT, 0, s>>>(me, ee, (size_t)cnt * st, l1, c.log_n,
                                                                           c.d_primes);
            CK(cudaGetLastError());
        }
        std::vector<SeedRow> rows;
        for (int t = 0; t < cnt; t++)
            for (int i = 0; i < l1; i++) rows.push_back({seeded_key(c, objs[t0 + t], i), a + ((size_t)t * l1 + i) * n, i, 0});
        seeded_uniform_device(c, rows, s);
        ntt_forward(c, poly_batch(me, st, 0, cnt, 1, 0, l1), s);
        ntt_forward(c, poly_batch(a, st, 0, cnt, 1, 0, l1), s);
        {
            LaunchScope _ls(c.prof, K_ELEMENTWISE, 32.0 * cnt * st, s);
            seeded_c0_kernel<<<blocks_for((size_t)cnt * st), kT, 0, s>>>(c0_out + (size_t)t0 * st, me, a, c.d_sk,
                                                                         (size_t)cnt * st, l1, c.log_n, c.d_primes);
            CK(cudaGetLastError());
        }
        CK(cudaStreamSynchronize(s));  // `host` is refilled by the next chunk
    }
}

void encrypt_coeffs_device(Ctx& c, const i64* m_dev, size_t m_stride, int count, int level,
                           const std::vector<u64>& nonces, u64* ct, cudaStream_t s) {
    if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
    if (level < 0 || level > c.L) fail(FHE_ERR_INVALID_ARG, "level out of range");
    const int n = c.n, l1 = level + 1;
    const GaussTable T = gauss_table(c.sigma);
    const int chunk = 32;
    std::vector<int8_t> host((size_t)chunk * 3 * n);
    for (int t0 = 0; t0 < count; t0 += chunk) {
        const int cnt = std::min(chunk, count - t0);
        for (int t = 0; t < cnt; t++) {
            u64 nonce = nonces[t0 + t];
            int8_t* h = host.data() + (size_t)t * 3 * n;
            sample_ternary(stream_key(c.seed, kEncV, nonce, 0, 0), h, n);
            sample_gaussian(stream_key(c.seed, kEncE0, nonce, 0, 0), T, h + n, n);
            sample_gaussian(stream_key(c.seed, kEncE1, nonce, 0, 0), T, h + 2 * n, n);
        }
        int8_t* d_small = (int8_t*)c.scratch_bytes("enc_small", (size_t)chunk * 3 * n);
        u64* v = c.scratch_u64("enc_v", (size_t)chunk * l1 * n);
        u64* c0 = c.scratch_u64("enc_c0", (size_t)chunk * l1 * n);
        u64* c1 = c.scratch_u64("enc_c1", (size_t)chunk * l1 * n);
        u64* mm = c.scratch_u64("enc_m", (size_t)chunk * l1 * n);
        CK(cudaMemcpyAsync(d_small, host.data(), (size_t)cnt * 3 * n, cudaMemcpyHostToDevice, s));
        const size_t st = (size_t)l1 * n;
        k_int8_to_rns(c, v, st, d_small, (size_t)3 * n, cnt, l1, 1 << 30, 0, s);
        k_int8_to_rns(c, c0, st, d_small + n, (size_t)3 * n, cnt, l1, 1 << 30, 0, s);
        k_int8_to_rns(c, c1, st, d_small + 2 * n, (size_t)3 * n, cnt, l1, 1 << 30, 0, s);
        k_int_to_rns(c, mm, st, m_dev + (size_t)t0 * m_stride, m_stride, cnt, l1, s);
        {
            LaunchScope _ls(c.prof, K_ELEMENTWISE, 24.0 * cnt * st, s);
            add_compact_kernel<<<blocks_for((size_t)cnt * st), kT, 0, s>>>(c0, mm, (size_t)cnt * st, l1,
                                                                           c.log_n, c.d_primes);
            CK(cudaGetLastError());
        }
        ntt_forward(c, poly_batch(v, st, 0, cnt, 1, 0, l1), s);
        ntt_forward(c, poly_batch(c0, st, 0, cnt, 1, 0, l1), s);
        ntt_forward(c, poly_batch(c1, st, 0, cnt, 1, 0, l1), s);
        {
            LaunchScope _ls(c.prof, K_ELEMENTWISE, 56.0 * cnt * st, s);
            enc_combine_kernel<<<blocks_for((size_t)cnt * st), kT, 0, s>>>(
                ct + (size_t)t0 * c.ct_words(), c.ct_words(), (size_t)(c.L + 1) * n, v, c0, c1, c.d_pk,
                c.d_pk + (size_t)(c.L + 1) * n, cnt, l1, c.log_n, c.d_primes);
            CK(cudaGetLastError());
        }
        CK(cudaStreamSynchronize(s));  // `host` is refilled by the next chunk
    }
}

void decrypt_to_slots(Ctx& c, const u64* ct, int level, double* host_slots, size_t n_slots,
                      cudaStream_t s) {
    if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
    if (level < 0 || level > c.L) fail(FHE_ERR_INVALID_ARG, "level out of range");
    if (n_slots > (size_t)c.slots) fail(FHE_ERR_INVALID_ARG, "more values than slots");
    const int n = c.n, nl = std::min(level, 1) + 1;
    u64* m = c.scratch_u64("dec_m", (size_t)nl * n);
    double* md = (double*)c.scratch_bytes("dec_md", sizeof(double) * n);
    double* z = (double*)c.scratch_bytes("dec_z", sizeof(double) * (n_slots + 1));
    {
        LaunchScope _ls(c.prof, K_ELEMENTWISE, 32.0 * nl * n, s);
        dec_kernel<<<blocks_for((size_t)nl * n), kT, 0, s>>>(m, ct, (size_t)(c.L + 1) * n, c.d_sk, nl, c.log_n,
                                                             c.d_primes);
        CK(cudaGetLastError());
    }
    ntt_inverse(c, poly_batch(m, (size_t)nl * n, 0, 1, 1, 0, nl), s);
    u64 q0 = c.primes[0], q1 = c.primes[1 % (c.L + 1)];
    u64 q0i = nl == 2 ? h_inv(q0 % q1, q1) : 0;
    {
        LaunchScope _ls(c.prof, K_ENCODE, 8.0 * (nl + 1) * n, s);
        crt_kernel<<<blocks_for(n), kT, 0, s>>>(md, m, nl, c.log_n, q0, q1, q0i);
        CK(cudaGetLastError());
    }
    if (n_slots) {
        {
            LaunchScope _ls(c.prof, K_ENCODE, 8.0 * (n + n_slots), s);
            decode_kernel<<<(unsigned)n_slots, 256, 0, s>>>(z, md, c.d_cos, c.d_pow5, c.log_n,
                                                            std::ldexp(1.0, -c.log_scale), (int)n_slots);
            CK(cudaGetLastError());
        }
        CK(cudaMemcpyAsync(host_slots, z, sizeof(double) * n_slots, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
}

// Key-holder refresh of `count` ciphertexts at `level`: exact integer plaintexts (two-limb CRT,
// as in decryption) re-encrypted at the top level with nonces nonce_base + t. out may equal ct.
void refresh_device(Ctx& c, const u64* ct, int count, int level, u64 nonce_base, u64* out, cudaStream_t s) {
    if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
    if (level < 0 || level > c.L) fail(FHE_ERR_INVALID_ARG, "level out of range");
    const int n = c.n, nl = std::min(level, 1) + 1;
    i64* mi = (i64*)c.scratch_bytes("ref_m", sizeof(i64) * (size_t)std::max(count, 1) * n);
    u64* m = c.scratch_u64("dec_m", (size_t)nl * n);
    int* flag = (int*)c.scratch_bytes("ref_flag", sizeof(int));
    CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
    u64 q0 = c.primes[0], q1 = c.primes[1 % (c.L + 1)];
    u64 q0i = nl == 2 ? h_inv(q0 % q1, q1) : 0;
    for (int t = 0; t < count; t++) {
        {
            LaunchScope _ls(c.prof, K_ELEMENTWISE, 32.0 * nl * n, s);
            dec_kernel<<<blocks_for((size_t)nl * n), kT, 0, s>>>(m, ct + (size_t)t * c.ct_words(), (size_t)(c.L + 1) * n,
                                                                 c.d_sk, nl, c.log_n, c.d_primes);
            CK(cudaGetLastError());
        }
        ntt_inverse(c, poly_batch(m, (size_t)nl * n, 0, 1, 1, 0, nl), s);
        {
            LaunchScope _ls(c.prof, K_ENCODE, 8.0 * (nl + 1) * n, s);
            crt_int64_kernel<<<blocks_for(n), kT, 0, s>>>(mi + (size_t)t * n, m, nl, c.log_n, q0, q1, q0i, flag);
            CK(cudaGetLastError());
        }
    }
    int h_flag = 0;
    CK(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h_flag) fail(FHE_ERR_INVALID_ARG, "plaintext coefficient outside int64: cannot refresh");
    std::vector<u64> nonces;
    for (int t = 0; t < count; t++) nonces.push_back(nonce_base + (u64)t);
    encrypt_coeffs_device(c, mi, n, count, c.L, nonces, out, s);
}

// Hybrid key-switching key for target secret s2 (evaluation domain, [n_ext][N]).
static void make_evk(Ctx& c, EvalKey& key, const u64* d_s2, u64 obj, cudaStream_t s) {
    const int n = c.n, ne = c.n_ext, dn = c.dnum(c.L);
    if (!key.d) key.d = dalloc<u64>(c.key_words());
    const GaussTable T = gauss_table(c.sigma);
    std::vector<u64> ha((size_t)ne * n);
    std::vector<int8_t> he(n);
    int8_t* d_e8 = (int8_t*)c.scratch_bytes("kg_e8", n);
    u64* d_e = c.scratch_u64("kg_e", (size_t)ne * n);
    for (int j = 0; j < dn; j++) {
        for (int t = 0; t < ne; t++) sample_uniform(stream_key(c.seed, kEvkA, obj, j, t), c.primes[t], &ha[(size_t)t * n], n);
        sample_gaussian(stream_key(c.seed, kEvkE, obj, j, 0), T, he.data(), n);
        u64* kb = key.d + (size_t)(j * 2 + 0) * ne * n;
        u64* ka = key.d + (size_t)(j * 2 + 1) * ne * n;
        CK(cudaMemcpyAsync(ka, ha.data(), sizeof(u64) * ha.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_e8, he.data(), n, cudaMemcpyHostToDevice, s));
        ntt_forward(c, poly_batch(ka, 0, 0, 1, 1, 0, ne), s);
        k_int8_to_rns(c, d_e, 0, d_e8, 0, 1, ne, 1 << 30, 0, s);
        ntt_forward(c, poly_batch(d_e, 0, 0, 1, 1, 0, ne), s);
        int lo = j * c.alpha, hi = std::min((j + 1) * c.alpha, c.L + 1);
        {
            LaunchScope _ls(c.prof, K_OTHER, 40.0 * ne * n, s);
            evk_kernel<<<blocks_for((size_t)ne * n), kT, 0, s>>>(kb, ka, c.d_sk, d_e, d_s2, ne, c.L, lo, hi,
                                                                 c.log_n, c.d_primes, c.d_pmod);
            CK(cudaGetLastError());
            if (c.keys_packed) {
                key_pack_kernel<<<blocks_for((size_t)(c.L + 1) * n), kT, 0, s>>>(kb, ka, c.L, c.log_n);
                CK(cudaGetLastError());
            }
        }
        CK(cudaStreamSynchronize(s));  // host staging buffers are reused
    }
}

static void add_rotation_key(Ctx& c, int step, cudaStream_t s) {
    int g = c.galois(step);
    if (g == 1 || c.rot.count(g)) return;
    u64* sg = c.scratch_u64("kg_sg", (size_t)c.n_ext * c.n);
    k_automorphism_poly(c, sg, c.d_sk, c.n_ext, g, s);
    EvalKey key;
    key.galois = g;
    make_evk(c, key, sg, (u64)g, s);
    c.rot[g] = key;
}

static void keygen(Ctx& c, u64 seed, const int32_t* steps, size_t n_steps, cudaStream_t s) {
    const int n = c.n, ne = c.n_ext, l1 = c.L + 1;
    for (auto& kv : c.rot) cudaFree(kv.second.d);
    c.rot.clear();
    c.seed = seed;
    const GaussTable T = gauss_table(c.sigma);
    // secret: ternary over the extended basis
    std::vector<int8_t> hs(n);
    sample_ternary(stream_key(seed, kSecret, 0, 0, 0), hs.data(), n);
    int8_t* d8 = (int8_t*)c.scratch_bytes("kg_s8", n);
    CK(cudaMemcpyAsync(d8, hs.data(), n, cudaMemcpyHostToDevice, s));
    if (!c.d_sk) c.d_sk = dalloc<u64>((size_t)ne * n);
    k_int8_to_rns(c, c.d_sk, 0, d8, 0, 1, ne, 1 << 30, 0, s);
    ntt_forward(c, poly_batch(c.d_sk, 0, 0, 1, 1, 0, ne), s);
    // public key (data primes)
    if (!c.d_pk) c.d_pk = dalloc<u64>((size_t)2 * l1 * n);
    std::vector<u64> ha((size_t)l1 * n);
    for (int i = 0; i < l1; i++) sample_uniform(stream_key(seed, kPkA, 0, 0, i), c.primes[i], &ha[(size_t)i * n], n);
    std::vector<int8_t> he(n);
    sample_gaussian(stream_key(seed, kPkE, 0, 0, 0), T, he.data(), n);
    u64* pk1 = c.d_pk + (size_t)l1 * n;
    CK(cudaMemcpyAsync(pk1, ha.data(), sizeof(u64) * ha.size(), cudaMemcpyHostToDevice, s));
    int8_t* de8 = (int8_t*)c.scratch_bytes("kg_e8", n);
    CK(cudaMemcpyAsync(de8, he.data(), n, cudaMemcpyHostToDevice, s));
    ntt_forward(c, poly_batch(pk1, 0, 0, 1, 1, 0, l1), s);
    u64* de = c.scratch_u64("kg_e", (size_t)ne * n);
    k_int8_to_rns(c, de, 0, de8, 0, 1, l1, 1 << 30, 0, s);
    ntt_forward(c, poly_batch(de, 0, 0, 1, 1, 0, l1), s);
    {
        LaunchScope _ls(c.prof, K_OTHER, 32.0 * l1 * n, s);
        pk_kernel<<<blocks_for((size_t)l1 * n), kT, 0, s>>>(c.d_pk, pk1, c.d_sk, de, l1, c.log_n, c.d_primes);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(s));
    // relinearisation key for s^2
    u64* s2 = c.scratch_u64("kg_s2", (size_t)ne * n);
    {
        LaunchScope _ls(c.prof, K_OTHER, 16.0 * ne * n, s);
        square_kernel<<<blocks_for((size_t)ne * n), kT, 0, s>>>(s2, c.d_sk, ne, c.log_n, c.d_primes);
        CK(cudaGetLastError());
    }
    make_evk(c, c.rlk, s2, 0, s);
    c.have_keys = true;
    for (size_t i = 0; i < n_steps; i++) add_rotation_key(c, steps[i], s);
    CK(cudaStreamSynchronize(s));
}

}  // namespace fhe

// ============================================================================ C ABI

using namespace fhe;

namespace {

template <typename F>
int guarded(fhe_ctx* ctx, F&& f) {
    try {
        if (ctx) {
            ctx->c.last_error.clear();
            CK(cudaSetDevice(ctx->c.device));
        }
        f();
        return FHE_OK;
    } catch (const FheException& e) {
        if (ctx) ctx->c.last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->c.last_error = "host allocation failed";
        return FHE_ERR_OOM;
    } catch (const std::exception& e) {
        if (ctx) ctx->c.last_error = e.what();
        return FHE_ERR_INVALID_ARG;
    }
}

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

void check_level(const Ctx& c, int level, int min_level = 0) {
    if (level < 0 || level > c.L) fail(FHE_ERR_INVALID_ARG, "level out of range");
    if (level < min_level) fail(FHE_ERR_LEVEL_EXHAUSTED, "level too low for this operation");
}
void check_ptr(const void* p, const char* what) {
    if (!p) fail(FHE_ERR_INVALID_ARG, std::string("null pointer: ") + what);
}
void check_keys(const Ctx& c) {
    if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
}

}  // namespace

extern "C" {

int fhe_ctx_create(const fhe_params* p, fhe_ctx** out) {
    if (!p || !out) return FHE_ERR_INVALID_ARG;
    *out = nullptr;
    fhe_ctx* ctx = new (std::nothrow) fhe_ctx();
    if (!ctx) return FHE_ERR_OOM;
    int rc = guarded(nullptr, [&] {
        Ctx& c = ctx->c;
        if (p->log_n < 9 || p->log_n > 16) fail(FHE_ERR_INVALID_ARG, "log_n must be in [9, 16]");
        if (p->n_data_primes < 1 || p->n_special_primes < 1 || p->n_special_primes > 8 ||
            !p->data_prime_bits || !p->special_prime_bits)
            fail(FHE_ERR_INVALID_ARG, "bad prime counts");
        std::vector<int> bits;
        for (int i = 0; i < p->n_data_primes; i++) bits.push_back(p->data_prime_bits[i]);
        for (int i = 0; i < p->n_special_primes; i++) bits.push_back(p->special_prime_bits[i]);
        for (int b : bits)
            if (b < 20 || b > 61) fail(FHE_ERR_INVALID_ARG, "prime bits must be in [20, 61]");
        if (p->log_scale < 1 || p->log_scale > 60) fail(FHE_ERR_INVALID_ARG, "bad log_scale");
        c.device = p->device;
        CK(cudaSetDevice(c.device));
        c.log_n = p->log_n;
        c.n = 1 << p->log_n;
        c.slots = c.n / 2;
        c.L = p->n_data_primes - 1;
        c.alpha = p->n_special_primes;
        c.n_ext = c.L + 1 + c.alpha;
        c.log_scale = p->log_scale;
        c.sigma = p->sigma > 0 ? p->sigma : 3.2;
        c.primes = choose_primes(c.log_n, bits);
        for (u64 q : c.primes) c.hprimes.push_back(make_prime(q));
        for (const Prime& P : c.hprimes) c.max_prime_bits = std::max(c.max_prime_bits, (int)P.b);
        for (int i = 0; i <= c.L; i++) c.max_data_prime_bits = std::max(c.max_data_prime_bits, (int)c.hprimes[i].b);
        c.keys_packed = c.max_data_prime_bits <= 50;
        c.d_primes = dupload(c.hprimes);
        ntt_init();
        build_tables(c);
        CK(cudaDeviceSynchronize());
    });
    if (rc) {
        delete ctx;
        return rc;
    }
    *out = ctx;
    return FHE_OK;
}

void fhe_ctx_destroy(fhe_ctx* ctx) { delete ctx; }

const char* fhe_last_error(const fhe_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

int fhe_ctx_get_info(const fhe_ctx* ctx, fhe_ctx_info* out) {
    if (!ctx || !out) return FHE_ERR_INVALID_ARG;
    const Ctx& c = ctx->c;
    out->log_n = c.log_n;
    out->n = c.n;
    out->slots = c.slots;
    out->top_level = c.L;
    out->n_special = c.alpha;
    out->log_scale = c.log_scale;
    out->ct_words = c.ct_words();
    return FHE_OK;
}

int fhe_ctx_get_primes(const fhe_ctx* ctx, uint64_t* out, size_t cap) {
    if (!ctx || !out || cap < ctx->c.primes.size()) return FHE_ERR_INVALID_ARG;
    std::memcpy(out, ctx->c.primes.data(), sizeof(u64) * ctx->c.primes.size());
    return FHE_OK;
}

int fhe_keygen_from_seed(fhe_ctx* ctx, uint64_t seed, const int32_t* steps, size_t n_steps) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        if (n_steps) check_ptr(steps, "rot_steps");
        keygen(ctx->c, seed, steps, n_steps, 0);
    });
}

int fhe_add_rotation_keys(fhe_ctx* ctx, const int32_t* steps, size_t n_steps) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        check_keys(ctx->c);
        if (n_steps) check_ptr(steps, "rot_steps");
        for (size_t i = 0; i < n_steps; i++) add_rotation_key(ctx->c, steps[i], 0);
        CK(cudaStreamSynchronize(0));
    });
}

int fhe_encode(fhe_ctx* ctx, const double* slots, size_t n_slots, int64_t* coeffs, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        check_ptr(coeffs, "coeffs");
        if (n_slots) check_ptr(slots, "slots");
        encode_device(ctx->c, slots, n_slots, coeffs, S(stream));
    });
}

int fhe_encrypt_coeffs(fhe_ctx* ctx, const int64_t* coeffs, int32_t level, uint64_t nonce, uint64_t* ct,
                       void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        check_ptr(coeffs, "coeffs");
        check_ptr(ct, "ct");
        check_level(ctx->c, level);
        encrypt_coeffs_device(ctx->c, coeffs, ctx->c.n, 1, level, {nonce}, ct, S(stream));
    });
}

int fhe_encrypt(fhe_ctx* ctx, const double* slots, size_t n_slots, int32_t level, uint64_t nonce,
                uint64_t* ct, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        check_ptr(ct, "ct");
        if (n_slots) check_ptr(slots, "slots");
        check_level(ctx->c, level);
        Ctx& c = ctx->c;
        i64* m = (i64*)c.scratch_bytes("api_m", sizeof(i64) * c.n);
        encode_device(c, slots, n_slots, m, S(stream));
        encrypt_coeffs_device(c, m, c.n, 1, level, {nonce}, ct, S(stream));
    });
}

int fhe_decrypt(fhe_ctx* ctx, const uint64_t* ct, int32_t level, double* slots, size_t n_slots, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        check_ptr(ct, "ct");
        if (n_slots) check_ptr(slots, "slots");
        decrypt_to_slots(ctx->c, ct, level, slots, n_slots, S(stream));
    });
}

int fhe_refresh(fhe_ctx* ctx, const uint64_t* ct, int32_t count, int32_t level, uint64_t nonce_base, uint64_t* out,
                void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ct, "ct");
        check_ptr(out, "out");
        if (count < 0) fail(FHE_ERR_INVALID_ARG, "negative count");
        refresh_device(ctx->c, ct, count, level, nonce_base, out, S(stream));
    });
}

int fhe_ntt_forward(fhe_ctx* ctx, uint64_t* polys, int32_t count, int32_t n_limbs, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        check_ptr(polys, "polys");
        if (count < 0 || n_limbs < 1 || n_limbs > ctx->c.L + 1) fail(FHE_ERR_INVALID_ARG, "bad count or limbs");
        ntt_forward(ctx->c, poly_batch(polys, (size_t)n_limbs * ctx->c.n, 0, count, 1, 0, n_limbs), S(stream));
    });
}

int fhe_ntt_inverse(fhe_ctx* ctx, uint64_t* polys, int32_t count, int32_t n_limbs, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        check_ptr(polys, "polys");
        if (count < 0 || n_limbs < 1 || n_limbs > ctx->c.L + 1) fail(FHE_ERR_INVALID_ARG, "bad count or limbs");
        ntt_inverse(ctx->c, poly_batch(polys, (size_t)n_limbs * ctx->c.n, 0, count, 1, 0, n_limbs), S(stream));
    });
}

int fhe_ct_to_coeff(fhe_ctx* ctx, const uint64_t* ct, int32_t count, int32_t level, uint64_t* out,
                    void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ct, "ct");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level);
        c.arena.reset(S(stream));
        const int l1 = level + 1;
        const size_t lw = (size_t)(c.L + 1) * c.n;
        // copy limb by limb into the compact layout, then inverse NTT
        std::vector<UnItem> it;
        u64* tmp = c.scratch_u64("api_coef", (size_t)count * c.ct_words());
        for (int t = 0; t < count; t++) it.push_back({ct + t * c.ct_words(), tmp + t * c.ct_words()});
        items_copy(c, it, 2, l1, S(stream));
        ntt_inverse(c, poly_batch(tmp, 2 * lw, lw, count, 2, 0, l1), S(stream));
        for (int t = 0; t < count; t++)
            for (int p = 0; p < 2; p++)
                CK(cudaMemcpyAsync(out + ((size_t)t * 2 + p) * l1 * c.n, tmp + t * c.ct_words() + p * lw,
                                   sizeof(u64) * l1 * c.n, cudaMemcpyDeviceToDevice, S(stream)));
    });
}

namespace {
std::vector<BinItem> bin_items(const Ctx& c, const u64* a, const u64* b, u64* out, int count, size_t sa,
                               size_t sb, size_t so) {
    std::vector<BinItem> it;
    for (int t = 0; t < count; t++) it.push_back({a + t * sa, b ? b + t * sb : nullptr, out + t * so});
    return it;
}
}  // namespace

int fhe_add(fhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, int32_t count, int32_t level,
            void* stream) {
    return guarded(ctx, [&] {
        check_ptr(a, "a");
        check_ptr(b, "b");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level);
        c.arena.reset(S(stream));
        size_t w = c.ct_words();
        items_add(c, bin_items(c, a, b, out, count, w, w, w), 2, level + 1, false, S(stream));
    });
}

int fhe_sub(fhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, int32_t count, int32_t level,
            void* stream) {
    return guarded(ctx, [&] {
        check_ptr(a, "a");
        check_ptr(b, "b");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level);
        c.arena.reset(S(stream));
        size_t w = c.ct_words();
        items_add(c, bin_items(c, a, b, out, count, w, w, w), 2, level + 1, true, S(stream));
    });
}

int fhe_mul_plain(fhe_ctx* ctx, const uint64_t* ct, const int64_t* pt, uint64_t* out, int32_t count,
                  int32_t level, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ct, "ct");
        check_ptr(pt, "pt");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level);
        c.arena.reset(S(stream));
        u64* ptm = c.scratch_u64("api_pt", (size_t)(c.L + 1) * c.n);
        materialize_plain(c, pt, c.n, 1, level + 1, ptm, (size_t)(c.L + 1) * c.n, S(stream));
        size_t w = c.ct_words();
        items_mul_plain(c, bin_items(c, ct, ptm, out, count, w, 0, w), 2, level + 1, S(stream));
    });
}

int fhe_tensor(fhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out3, int32_t count,
               int32_t level, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(a, "a");
        check_ptr(b, "b");
        check_ptr(out3, "out3");
        Ctx& c = ctx->c;
        check_level(c, level);
        c.arena.reset(S(stream));
        size_t w = c.ct_words();
        items_tensor(c, bin_items(c, a, b, out3, count, w, w, 3 * w / 2), level + 1, S(stream));
    });
}

namespace {
void relin_into(Ctx& c, const u64* in3, u64* out, int count, size_t out_stride, int level, cudaStream_t s) {
    const size_t lw = (size_t)(c.L + 1) * c.n;
    std::vector<KsItem> ks;
    for (int t = 0; t < count; t++) {
        const u64* x = in3 + (size_t)t * 3 * lw;
        u64* o = out + (size_t)t * out_stride;
        ks.push_back({x + 2 * lw, c.rlk.d, nullptr, x, x + lw, o, o + lw, 1});
    }
    keyswitch_items(c, ks, level, s);
}
}  // namespace

int fhe_relinearize(fhe_ctx* ctx, const uint64_t* in3, uint64_t* out, int32_t count, int32_t level,
                    void* stream) {
    return guarded(ctx, [&] {
        check_ptr(in3, "in3");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level);
        check_keys(c);
        c.arena.reset(S(stream));
        relin_into(c, in3, out, count, c.ct_words(), level, S(stream));
    });
}

int fhe_rescale(fhe_ctx* ctx, const uint64_t* ct, uint64_t* out, int32_t count, int32_t level, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ct, "ct");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level, 1);
        c.arena.reset(S(stream));
        std::vector<UnItem> it;
        for (int t = 0; t < count; t++) it.push_back({ct + t * c.ct_words(), out + t * c.ct_words()});
        items_rescale(c, it, 2, level, S(stream));
    });
}

int fhe_mul_relin_rescale(fhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, int32_t count,
                          int32_t level, void* stream) {
    return guarded(ctx, [&] {
        check_ptr(a, "a");
        check_ptr(b, "b");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level, 1);
        check_keys(c);
        c.arena.reset(S(stream));
        const size_t w = c.ct_words(), lw = w / 2;
        u64* t3 = c.scratch_u64("api_t3", (size_t)count * 3 * lw);
        items_tensor(c, bin_items(c, a, b, t3, count, w, w, 3 * lw), level + 1, S(stream));
        std::vector<u64*> in3, outs;
        for (int t = 0; t < count; t++) {
            in3.push_back(t3 + t * 3 * lw);
            outs.push_back(out + t * w);
        }
        relin_rescale_items(c, in3, outs, level, S(stream));
    });
}

int fhe_rotate(fhe_ctx* ctx, const uint64_t* ct, uint64_t* out, int32_t count, int32_t level, int32_t step,
               void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ct, "ct");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level);
        check_keys(c);
        if (ct == out) fail(FHE_ERR_INVALID_ARG, "rotation output must not alias its input");
        c.arena.reset(S(stream));
        const size_t w = c.ct_words(), lw = w / 2;
        int g = c.galois(step);
        if (g == 1) {
            std::vector<UnItem> it;
            for (int t = 0; t < count; t++) it.push_back({ct + t * w, out + t * w});
            items_copy(c, it, 2, level + 1, S(stream));
            return;
        }
        const EvalKey& key = rotation_key(c, step);
        std::vector<KsItem> ks;
        for (int t = 0; t < count; t++) {
            const u64* x = ct + t * w;
            u64* o = out + t * w;
            ks.push_back({x + lw, key.d, x, nullptr, nullptr, o, o + lw, g});
        }
        keyswitch_items(c, ks, level, S(stream));
    });
}

int fhe_rotate_sum(fhe_ctx* ctx, uint64_t* ct, uint64_t* out, int32_t count, int32_t level, int32_t kp,
                   void* stream) {
    return guarded(ctx, [&] {
        check_ptr(ct, "ct");
        check_ptr(out, "out");
        Ctx& c = ctx->c;
        check_level(c, level);
        check_keys(c);
        if (count < 0) fail(FHE_ERR_INVALID_ARG, "negative count");
        if (kp < 1 || (kp > kHoistMaxKp && (kp & (kp - 1)) != 0))
            fail(FHE_ERR_INVALID_ARG, "rotate-and-sum needs 1 <= kp <= 16 or a power of two");
        if (kp > kHoistMaxKp && ct == out) fail(FHE_ERR_INVALID_ARG, "rotate-and-sum over more than 16 slots needs out != ct");
        c.arena.reset(S(stream));
        const size_t w = c.ct_words();
        std::vector<u64*> in, o;
        for (int t = 0; t < count; t++) {
            in.push_back(ct + t * w);
            o.push_back(out + t * w);
        }
        rotsum_items(c, in, o, kp, level, S(stream));
    });
}

int fhe_rotate_fanin(fhe_ctx* ctx, uint64_t* acc, int32_t n_groups, const int32_t* first, const uint64_t* ct,
                     const int32_t* steps, int32_t level, void* stream) {
    return guarded(ctx, [&] {
        Ctx& c = ctx->c;
        check_level(c, level);
        check_keys(c);
        if (n_groups < 0) fail(FHE_ERR_INVALID_ARG, "negative group count");
        if (n_groups == 0) return;
        check_ptr(acc, "acc");
        check_ptr(first, "first");
        const int total = first[n_groups];
        if (first[0] != 0 || total < 0) fail(FHE_ERR_INVALID_ARG, "fan-in offsets must run from 0 to the input count");
        if (total > 0) {
            check_ptr(ct, "ct");
            check_ptr(steps, "steps");
        }
        c.arena.reset(S(stream));
        const size_t w = c.ct_words();
        std::vector<u64*> a;
        std::vector<int> fo(first, first + n_groups + 1), st;
        std::vector<const u64*> in;
        for (int g = 0; g < n_groups; g++) a.push_back(acc + g * w);
        for (int i = 0; i < total; i++) {
            const u64* x = ct + i * w;
            if (x < acc + (size_t)n_groups * w && acc < x + w) fail(FHE_ERR_INVALID_ARG, "fan-in input aliases an output");
            in.push_back(x);
            st.push_back(steps[i]);
        }
        rotate_fanin_items(c, a, fo, in, st, level, S(stream));
    });
}

int fhe_profile_begin(fhe_ctx* ctx, int32_t time_kernels) {
    return guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        CK(cudaDeviceSynchronize());
        ctx->c.prof.reset();
        ctx->c.prof.timing = time_kernels != 0;
    });
}

int fhe_profile_end(fhe_ctx* ctx, fhe_kernel_stat* out, int32_t cap) {
    int rc = guarded(ctx, [&] {
        check_ptr(ctx, "ctx");
        check_ptr(out, "out");
        if (cap < K_COUNT) fail(FHE_ERR_INVALID_ARG, "cap must be at least the number of kernel classes");
        CK(cudaDeviceSynchronize());
        Profiler& p = ctx->c.prof;
        double ms[K_COUNT] = {};
        for (auto& r : p.recs) {
            float t = 0;
            CK(cudaEventElapsedTime(&t, r.a, r.b));
            ms[r.cls] += t;
        }
        for (int k = 0; k < K_COUNT; k++) {
            out[k].name = kKClassNames[k];
            out[k].launches = p.launches[k];
            out[k].device_ms = ms[k];
            out[k].bytes = p.bytes[k];
            out[k].work = p.work[k];
        }
        p.timing = false;
        p.recs.clear();
        p.pool_used = 0;
    });
    return rc ? rc : (int)K_COUNT;
}

}  // extern "C"

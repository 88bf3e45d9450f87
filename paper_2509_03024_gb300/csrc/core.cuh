// core.cuh — shared definitions of the GB300 RNS-CKKS library: exact 64-bit
// modular arithmetic, the context object, device-buffer helpers and launch
// declarations of the kernels in ntt.cu / ops.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ckks_mf.h"

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

namespace fhe {

// ----------------------------------------------------------------------------- errors

struct FheException : std::exception {
    int code;
    std::string msg;
    FheException(int c, std::string m) : code(c), msg(std::move(m)) {}
    const char* what() const noexcept override { return msg.c_str(); }
};

// Throwing is used inside the library; every extern "C" entry point catches
// and converts to an FHE_ERR_* code plus fhe_last_error text.
[[noreturn]] void fail(int code, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);
#define CK(x) ::fhe::cuda_check((x), #x)

// ----------------------------------------------------------------------------- modular arithmetic

// One RNS prime with its Barrett constant (HAC Alg. 14.42, base 2):
// mu = floor(2^(2b) / q), b = bit length of q, q < 2^62.
struct Prime {
    u64 q;
    u64 mu;
    u64 one_s;  // floor(2^64 / q): Shoup companion of 1, for lazy reduction of any 64-bit value
    u32 b;
    u32 pad;
};

__host__ __device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__host__ __device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) {
    return a >= b ? a - b : a + (q - b);
}

#ifdef __CUDACC__
// Barrett reduction of the 128-bit product a*b (a, b < q): q1 = x >> (b-1),
// q3 = (q1 * mu) >> (b+1), r = x - q3*q in [0, 3q), two conditional subtractions.
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const Prime& p) {
    u64 lo = a * b;
    u64 hi = __umul64hi(a, b);
    u64 q1 = (lo >> (p.b - 1)) | (hi << (65 - p.b));
    u64 t_lo = q1 * p.mu;
    u64 t_hi = __umul64hi(q1, p.mu);
    u64 q3 = (t_lo >> (p.b + 1)) | (t_hi << (63 - p.b));
    u64 r = lo - q3 * p.q;
    if (r >= p.q) r -= p.q;
    if (r >= p.q) r -= p.q;
    return r;
}
// Shoup multiplication by a constant w < q with ws = floor(w * 2^64 / q); a < 2^64.
__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 ws, u64 q) {
    u64 qh = __umul64hi(a, ws);
    u64 r = a * w - qh * q;
    return r >= q ? r - q : r;
}
#endif

// Host versions (exact, u128).
inline u64 h_mul(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
inline u64 h_pow(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = h_mul(r, a, q);
        a = h_mul(a, a, q);
        e >>= 1;
    }
    return r;
}
inline u64 h_inv(u64 a, u64 q) { return h_pow(a, q - 2, q); }
inline u64 h_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// ----------------------------------------------------------------------------- poly batches

// A regular batch of RNS polynomials in device memory. Row r of the batch is
// (item, part, limb) with r = (item * n_parts + part) * n_limbs + (limb - limb_lo);
// its N coefficients start at base + item*item_stride + part*part_stride +
// (limb - addr_lo)*N. The prime of limb t is t, plus `jump` when t >= split
// (an extended basis Q_l u P stored as limbs 0..l then the alpha special limbs).
struct PolyBatch {
    u64* base;
    size_t item_stride;
    size_t part_stride;
    int n_items;
    int n_parts;
    int limb_lo;
    int n_limbs;
    int split;
    int jump;
    int addr_lo;
    __host__ __device__ __forceinline__ int rows() const { return n_items * n_parts * n_limbs; }
    __host__ __device__ __forceinline__ int prime_of(int limb) const {
        return limb + (limb >= split ? jump : 0);
    }
};

// Batch of `items` polynomials with `parts` components, limbs [lo, lo+cnt), all data primes,
// stored at limb offsets relative to addr_lo.
inline PolyBatch poly_batch(u64* base, size_t item_stride, size_t part_stride, int items, int parts,
                            int lo, int cnt, int addr_lo = 0) {
    PolyBatch pb;
    pb.base = base;
    pb.item_stride = item_stride;
    pb.part_stride = part_stride;
    pb.n_items = items;
    pb.n_parts = parts;
    pb.limb_lo = lo;
    pb.n_limbs = cnt;
    pb.split = 1 << 30;
    pb.jump = 0;
    pb.addr_lo = addr_lo;
    return pb;
}

// ----------------------------------------------------------------------------- keys

// Hybrid key-switching key: [dnum_top][2 (b, a)][n_ext][N], evaluation domain.
struct EvalKey {
    u64* d = nullptr;
    int galois = 0;  // 0 for the relinearisation key
};

// ----------------------------------------------------------------------------- descriptor arena

// Pinned host staging + device memory for per-launch descriptor tables
// (pointer arrays). push() copies a table into pinned memory and enqueues its
// upload on the stream; the returned device address stays valid for the work
// enqueued before the next-but-one reset(). The arena has two halves that
// alternate at every reset(): reset() marks the end of the current half's use
// with an event on the stream, switches halves and waits (on the host) only
// for the event that ended the other half's previous use. So a call can build
// and upload its tables while the GPU still runs the previous call's kernels.
struct Arena {
    struct Block {
        char* host = nullptr;
        char* dev = nullptr;
        size_t cap = 0, used = 0;
    };
    struct Half {
        std::vector<Block> blocks;
        size_t cur = 0;
        cudaEvent_t done = nullptr;
        bool pending = false;
    };
    Half halves[2];
    int h = 0;
    void reset(cudaStream_t s);
    void* push(const void* data, size_t bytes, cudaStream_t s);
    template <typename T>
    T* push_vec(const std::vector<T>& v, cudaStream_t s) {
        return (T*)push(v.data(), v.size() * sizeof(T), s);
    }
    ~Arena();
};

// ----------------------------------------------------------------------------- launch accounting

// Kernel classes for launch counting and optional per-launch CUDA-event timing.
enum KClass {
    K_NTT_FWD = 0,  // every NTT pass, the fused conversion, rescale and combine passes included
    K_NTT_INV,
    K_KS_INNER,     // key inner products (plain, fan-out and hoisted)
    K_TENSOR,
    K_ELEMENTWISE,
    K_ENCODE,
    K_OTHER,
    K_COUNT
};
extern const char* const kKClassNames[K_COUNT];

struct Profiler {
    bool timing = false;
    long long launches[K_COUNT] = {};
    double bytes[K_COUNT] = {};
    double work[K_COUNT] = {};  // butterflies (NTT classes) or 64 x 64-bit multiply-accumulates (ks_inner)
    struct Rec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    cudaEvent_t get_event();
    void reset();
    ~Profiler();
};

// Per host thread: while set, LaunchScope records no CUDA events (launches and bytes are still
// counted). Lets one call skip event creation without touching the context's shared profiler state.
extern thread_local bool tl_no_launch_events;
struct NoLaunchEvents {
    bool saved;
    NoLaunchEvents() : saved(tl_no_launch_events) { tl_no_launch_events = true; }
    ~NoLaunchEvents() { tl_no_launch_events = saved; }
};

// RAII scope around one kernel launch: counts it, adds its algorithmic bytes and arithmetic work
// and, when timing is on, brackets it with CUDA events on its stream.
struct LaunchScope {
    Profiler& p;
    int cls;
    cudaStream_t s;
    cudaEvent_t b = nullptr;
    LaunchScope(Profiler& prof, int k, double bytes, cudaStream_t st, double work = 0.0);
    ~LaunchScope();
};

// ----------------------------------------------------------------------------- context

struct DeviceBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Ctx {
    int device = 0;
    int log_n = 0, n = 0, slots = 0;
    int L = 0;       // top level
    int alpha = 0;   // special primes
    int n_ext = 0;   // L + 1 + alpha
    int log_scale = 0;
    double sigma = 3.2;
    std::vector<u64> primes;  // data q_0..q_L then special p_0..p_{alpha-1}
    std::vector<Prime> hprimes;

    // device tables
    Prime* d_primes = nullptr;        // [n_ext]
    u64* d_psi = nullptr;             // [n_ext][N]  psi^brev(i)   (forward twiddles)
    u64* d_psi_s = nullptr;           // Shoup companions
    u64* d_ipsi = nullptr;            // [n_ext][N]  psi^-brev(i)  (inverse twiddles)
    u64* d_ipsi_s = nullptr;
    u64* d_ninv = nullptr;            // [n_ext][2] N^-1 and its Shoup companion
    // NTT twiddles interleaved with their Shoup companions (one 128-bit load each):
    // column / single-pass tables [prime][i] = (psi^brev(i), companion), inverse alike;
    // row-pass tables of the two-pass NTT laid out [prime][stage s'][group g][row r]
    // (value = psi^brev(2^(S1+s') + r 2^s' + g)), so that consecutive rows are contiguous
    ulonglong2* d_tw = nullptr;
    ulonglong2* d_itw = nullptr;
    ulonglong2* d_tw2 = nullptr;
    ulonglong2* d_itw2 = nullptr;
    int ntt_s1 = 0;                   // column stages of the two-pass NTT (0: single pass)
    u64* d_resc = nullptr;            // [L+1][L+1][2] q_l^-1 mod q_i (+ Shoup)
    u64* d_up_inv = nullptr;          // [L+1][L+1][2] digit-local qhat_i^-1 mod q_i at level l
    u64* d_up_hat = nullptr;          // [L+1][L+1][n_ext][2] digit-local qhat_i mod prime t at level l
    u64* d_up_ninv = nullptr;         // [L+1][L+1][2] N^-1 * qhat_i^-1 mod q_i (ModUp input scaling)
    u64* d_down_ninv = nullptr;       // [alpha][2]   N^-1 * Phat_k^-1 mod p_k (ModDown input scaling)
    u64* d_down_inv = nullptr;        // [alpha][2]   Phat_k^-1 mod p_k
    u64* d_down_hat = nullptr;        // [alpha][L+1][2] Phat_k mod q_i
    u64* d_pinv = nullptr;            // [L+1][2]     P^-1 mod q_i
    u64* d_pmod = nullptr;            // [L+1]        P mod q_i
    // fused ModDown + rescale at level l (divide by M' = P q_l; sources p_0..p_{alpha-1}, q_l)
    u64* d_fd_ninv = nullptr;         // [L+1][alpha+1][2]       N^-1 (M'/m_s)^-1 mod m_s
    u64* d_fd_hat = nullptr;          // [L+1][alpha+1][L+1][2]  (M'/m_s) mod q_i, i < l
    u64* d_fd_minv = nullptr;         // [L+1][L+1][2]           M'^-1 mod q_i, i < l
    u64* d_fd_pq = nullptr;           // [L+1][2]                P mod q_l
    double* d_cos = nullptr;          // [2N] cos(pi e / N)
    double* d_sin = nullptr;          // [2N] sin(pi e / N)
    u32* d_pow5 = nullptr;            // [N/2] 5^t mod 2N

    // keys
    bool have_keys = false;
    u64 seed = 0;
    u64* d_sk = nullptr;              // [n_ext][N] evaluation domain
    u64* d_pk = nullptr;              // [2][L+1][N]
    EvalKey rlk;
    std::map<int, EvalKey> rot;       // galois element -> key

    // scratch (grow-only), keyed by purpose
    std::map<std::string, DeviceBuf> scratch;
    u64* scratch_u64(const std::string& name, size_t words);
    void* scratch_bytes(const std::string& name, size_t bytes);

    // launch variants chosen by the autotuner (fhe_autotune); every choice gives the same bits
    struct Tune {
        int inner = 0;  // plain / fan-out key inner product (InnerVariant of ks_inner.cuh)
        int hoist = 0;  // hoisted rotate-and-sum inner product
        int ntt = 0;    // tile shape of the plain two-pass NTT (NttTile of ntt_tile.cuh)
        int ks = 0;     // tile shape of the fused key-switch / rescale passes (KsTile of ks_pass.cuh)
    } tune;
    // the evaluation keys' data-prime rows are stored split at bit 25 (key_pack in ks_inner.cuh),
    // set when every data prime has at most 50 bits
    bool keys_packed = false;
    int max_prime_bits = 0;       // over every prime
    int max_data_prime_bits = 0;  // over the data primes q_0..q_L

    std::string last_error;
    Arena arena;
    mutable Profiler prof;

    size_t ct_words() const { return (size_t)2 * (L + 1) * n; }
    size_t key_words() const { return (size_t)dnum(L) * 2 * n_ext * n; }
    int dnum(int level) const { return (level + 1 + alpha - 1) / alpha; }
    int galois(int step) const {
        long long r = ((long long)step % slots + slots) % slots;
        return (int)h_pow(5, (u64)r, (u64)2 * n);
    }
    ~Ctx();
};

// ----------------------------------------------------------------------------- kernels (ntt.cu)

// Kernel attributes (dynamic shared memory limits); called once per device.
void ntt_init();
// In-place negacyclic NTT / inverse NTT of every row of the batch.
void ntt_forward(const Ctx& c, const PolyBatch& pb, cudaStream_t s);
void ntt_inverse(const Ctx& c, const PolyBatch& pb, cudaStream_t s);

// ----------------------------------------------------------------------------- item kernels (ops.cu)

// Every ciphertext-like pointer addresses the start of an object in capacity
// layout: component p, limb i at ptr + p*(L+1)*N + i*N.
struct BinItem {
    const u64* a;
    const u64* b;
    u64* out;
};
struct UnItem {
    const u64* in;
    u64* out;
};
// One target accumulator and its contributors [off, off + cnt) in a BinItem list
// (a = left operand, b = right operand; out unused).
struct AccTarget {
    u64* out;
    int off;
    int cnt;
};

// out = a +/- b for `parts` components and `limbs` limbs
void items_add(Ctx& c, const std::vector<BinItem>& it, int parts, int limbs, bool sub, cudaStream_t s);
void items_copy(Ctx& c, const std::vector<UnItem>& it, int parts, int limbs, cudaStream_t s);
// out = a (.) b where b is a one-component plaintext (evaluation domain)
void items_mul_plain(Ctx& c, const std::vector<BinItem>& it, int parts, int limbs, cudaStream_t s);
// out (3 components) = a (x) b
void items_tensor(Ctx& c, const std::vector<BinItem>& it, int limbs, cudaStream_t s);
// target.out (3 components) += sum over contributors of a (x) b
void items_tensor_acc(Ctx& c, const std::vector<AccTarget>& tg, const std::vector<BinItem>& contrib,
                      int limbs, cudaStream_t s);
// target.out (`parts` components) += sum over contributors of a (b unused)
void items_sum_acc(Ctx& c, const std::vector<AccTarget>& tg, const std::vector<BinItem>& contrib,
                   int parts, int limbs, cudaStream_t s);
// out = in * value (a signed integer constant, reduced modulo each limb's prime)
struct ConstItem {
    const u64* in;
    u64* out;
    long long value;
};
void items_mul_const(Ctx& c, const std::vector<ConstItem>& it, int parts, int limbs, cudaStream_t s);
// rescale components [0, parts) from level l to l-1 (out may alias in)
void items_rescale(Ctx& c, const std::vector<UnItem>& it, int parts, int level, cudaStream_t s);
// rescale(a (.) b) for each item: a a ciphertext at `level`, b a plaintext (limb stride N); the
// product is formed inside the rescale's transforms. out may equal a.
void mul_plain_rescale_items(Ctx& c, const std::vector<BinItem>& it, int level, cudaStream_t s);

// signed int64 coefficients -> residues for limbs [0, limbs): out [items][L+1][N] (limb stride N)
void k_int_to_rns(const Ctx& c, u64* out, size_t out_item_stride, const i64* in, size_t in_stride,
                  int items, int limbs, cudaStream_t s);
void k_int8_to_rns(const Ctx& c, u64* out, size_t out_item_stride, const int8_t* in, size_t in_stride,
                   int items, int limbs, int prime_split, int prime_jump, cudaStream_t s);
// evaluation-domain automorphism of one [limbs][N] polynomial: out[k] = in[perm_g(k)]
void k_automorphism_poly(const Ctx& c, u64* out, const u64* in, int limbs, int galois, cudaStream_t s);

// Hybrid key switch, one polynomial per item:
//   out0 = KS0(d) + addP0[perm] + addI0,  out1 = KS1(d) + addI1
// d and addP0 are read through perm_galois (galois = 1: identity); the add
// terms are optional (null). Outputs must not alias d or addP0.
struct KsItem {
    const u64* d;
    const u64* key;
    const u64* addP0;
    const u64* addI0;
    const u64* addI1;
    u64* out0;
    u64* out1;
    long long galois;
};
void keyswitch_items(Ctx& c, const std::vector<KsItem>& it, int level, cudaStream_t s);

// Rotations that share inputs: out_i = rot(in_i, step_i) with one ModUp per distinct input (the
// automorphism applied to the raised digits, as in a hoisted rotate-and-sum of one step). out_i
// must not alias any input.
void rotate_fanout_items(Ctx& c, const std::vector<const u64*>& in, const std::vector<u64*>& out,
                         const std::vector<int>& steps, int level, cudaStream_t s);

// Fan-in rotation: acc_g += sum_{first_g <= i < first_{g+1}} rot(in_i, step_i) with one ModDown
// per group (the children's key inner products and rotated c0's are summed before it). No in_i
// may alias an acc_g.
void rotate_fanin_items(Ctx& c, const std::vector<u64*>& acc, const std::vector<int>& first,
                        const std::vector<const u64*>& in, const std::vector<int>& steps, int level, cudaStream_t s);

// Relinearise and rescale in one key switch (ModDown divides by P q_level): out_i (level - 1)
// from the 3-component t3_i (level). out_i may equal t3_i.
void relin_rescale_items(Ctx& c, const std::vector<u64*>& t3, const std::vector<u64*>& out, int level,
                         cudaStream_t s);

// In-block rotate-and-sum: out_i = sum_{r < kp} rot(in_i, r). Hoisted (one ModUp, kp - 1 key inner
// products, one ModDown; in_i may equal out_i) for 2 <= kp <= kHoistMaxKp, else log2(kp)
// rotate-and-adds (in_i and out_i distinct; in_i is overwritten).
constexpr int kHoistMaxKp = 16;
void rotsum_items(Ctx& c, const std::vector<u64*>& in, const std::vector<u64*>& out, int kp, int level,
                  cudaStream_t s);
// Left-rotation amounts of that rotate-and-sum.
std::vector<int> rotsum_steps(int kp);
// Hoisted rotate-and-sum over explicit steps (Halevi-Shoup): out_i = in_i + sum over the non-zero steps r
// of rot(in_i, r), one ModUp, one inner product per step, one ModDown; in_i may equal out_i.
void hoisted_sum_items(Ctx& c, const std::vector<u64*>& in, const std::vector<u64*>& out,
                       const std::vector<int>& steps, int level, cudaStream_t s);

// ----------------------------------------------------------------------------- ctx helpers (ctx.cu)

const EvalKey& rotation_key(const Ctx& c, int step);
void encode_device(Ctx& c, const double* host_slots, size_t n_slots, i64* out_dev, cudaStream_t s);
void encode_sparse_device(Ctx& c, const std::vector<std::pair<int, double>>& nz, i64* out_dev,
                          cudaStream_t s);
// Encode many sparse slot vectors at once: nz lists concatenated with offsets (host), out [count][N].
void encode_many_device(Ctx& c, const std::vector<int>& idx, const std::vector<double>& val,
                        const std::vector<int>& offsets, i64* out_dev, cudaStream_t s);
void encrypt_coeffs_device(Ctx& c, const i64* m_dev, size_t m_stride, int count, int level,
                           const std::vector<u64>& nonces, u64* ct, cudaStream_t s);

// Key-holder encryption with a regenerable c1 (stream purposes 9 and 10): c1 = a, the uniform
// polynomial drawn coefficient by coefficient from stream_key(seed, 9, obj, 0, limb) (up to
// kSeededTries draws each), c0 = -a s + m + e with e from stream_key(seed, 10, obj, 0, 0).
constexpr int kSeededTries = 16;
struct SeedRow {
    u64 h;       // stream key of the row
    u64* dst;    // N residues (coefficient form)
    int prime;   // prime index of the row
    int pad;
};
u64 seeded_key(const Ctx& c, u64 obj, int limb);
// Fill each row with its uniform coefficients (coefficient form).
void seeded_uniform_device(Ctx& c, const std::vector<SeedRow>& rows, cudaStream_t s);
// c0 only, evaluation domain, compact [count][level+1][N] at c0_out.
void encrypt_seeded_device(Ctx& c, const i64* m_dev, size_t m_stride, int count, int level,
                           const std::vector<u64>& objs, u64* c0_out, cudaStream_t s);
// plaintext materialisation: int64 coefficients -> evaluation domain limbs [0, limbs)
void materialize_plain(Ctx& c, const i64* m_dev, size_t m_stride, int count, int limbs, u64* out,
                       size_t out_stride, cudaStream_t s);
void refresh_device(Ctx& c, const u64* ct, int count, int level, u64 nonce_base, u64* out, cudaStream_t s);
void decrypt_to_slots(Ctx& c, const u64* ct, int level, double* host_slots, size_t n_slots,
                      cudaStream_t s);

}  // namespace fhe

struct fhe_ctx {
    fhe::Ctx c;
};

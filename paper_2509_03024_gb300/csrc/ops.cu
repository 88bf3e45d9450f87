// ops.cu — batched RNS kernels over descriptor tables: element-wise add / sub /
// plaintext product / tensor product, segmented accumulation, integer-to-RNS
// conversion and the evaluation-domain automorphism. (Key switching and the
// rescale run as fused NTT passes in ks.cu.)
//
// Launch shape of the element-wise kernels: blockIdx.y selects the item (a
// table entry), the x dimension walks (component, limb, coefficient pair) with
// one 128-bit access per residue pair. Item tables are uploaded through the
// context's pinned descriptor arena.
#include <algorithm>
#include <cstring>

#include "core.cuh"

namespace fhe {

// ============================================================================ arena

void Arena::reset(cudaStream_t s) {
    Half& used = halves[h];
    if (!used.done) CK(cudaEventCreateWithFlags(&used.done, cudaEventDisableTiming));
    CK(cudaEventRecord(used.done, s));
    used.pending = true;
    h ^= 1;
    Half& next = halves[h];
    if (next.pending) {
        CK(cudaEventSynchronize(next.done));  // its tables and staging may be overwritten now
        next.pending = false;
    }
    for (auto& b : next.blocks) b.used = 0;
    next.cur = 0;
}

void* Arena::push(const void* data, size_t bytes, cudaStream_t s) {
    Half& hf = halves[h];
    const size_t span = std::max<size_t>((bytes + 255) & ~(size_t)255, 256);
    while (hf.cur < hf.blocks.size() && hf.blocks[hf.cur].used + span > hf.blocks[hf.cur].cap) hf.cur++;
    if (hf.cur == hf.blocks.size()) {
        Block b;
        b.cap = std::max<size_t>(span, (size_t)4 << 20);
        CK(cudaMallocHost((void**)&b.host, b.cap));
        CK(cudaMalloc((void**)&b.dev, b.cap));
        hf.blocks.push_back(b);
    }
    Block& b = hf.blocks[hf.cur];
    char* hp = b.host + b.used;
    char* d = b.dev + b.used;
    b.used += span;
    if (bytes) {
        std::memcpy(hp, data, bytes);
        CK(cudaMemcpyAsync(d, hp, bytes, cudaMemcpyHostToDevice, s));
    }
    return d;
}

Arena::~Arena() {
    for (auto& hf : halves) {
        if (hf.pending) cudaEventSynchronize(hf.done);
        if (hf.done) cudaEventDestroy(hf.done);
        for (auto& b : hf.blocks) {
            if (b.host) cudaFreeHost(b.host);
            if (b.dev) cudaFree(b.dev);
        }
    }
}

// ============================================================================ launch accounting

const char* const kKClassNames[K_COUNT] = {"ntt_forward", "ntt_inverse", "ks_inner", "tensor",
                                           "elementwise", "encode",      "other"};

cudaEvent_t Profiler::get_event() {
    if (pool_used == pool.size()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        pool.push_back(e);
    }
    return pool[pool_used++];
}

void Profiler::reset() {
    for (int k = 0; k < K_COUNT; k++) {
        launches[k] = 0;
        bytes[k] = 0;
        work[k] = 0;
    }
    recs.clear();
    pool_used = 0;
}

Profiler::~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

thread_local bool tl_no_launch_events = false;

LaunchScope::LaunchScope(Profiler& prof, int k, double nbytes, cudaStream_t st, double work)
    : p(prof), cls(k), s(st) {
    p.launches[k]++;
    p.bytes[k] += nbytes;
    p.work[k] += work;
    if (p.timing && !tl_no_launch_events) {
        b = p.get_event();
        CK(cudaEventRecord(b, s));
    }
}

LaunchScope::~LaunchScope() {
    if (b) {
        cudaEvent_t e = p.get_event();
        cudaEventRecord(e, s);
        p.recs.push_back({cls, b, e});
    }
}

namespace {

constexpr int kThreads = 256;

template <typename T>
T* upload(Ctx& c, const std::vector<T>& v, cudaStream_t s) {
    return c.arena.push_vec(v, s);
}

inline dim3 grid2(size_t per_item, int items) {
    size_t bx = (per_item + kThreads - 1) / kThreads;
    if (bx > 65535u * 16) bx = 65535u * 16;
    return dim3((unsigned)std::max<size_t>(bx, 1), (unsigned)std::min(items, 65535));
}
inline unsigned grid1(size_t work) {
    size_t b = (work + kThreads - 1) / kThreads;
    return (unsigned)std::min<size_t>(std::max<size_t>(b, 1), (size_t)1 << 30);
}

// ---------------------------------------------------------------- element-wise

// For element e of an item: component p, limb i, coefficient pair k2.
struct PIdx {
    int part, limb, k2;
};
__device__ __forceinline__ PIdx pidx(size_t e, int log_half, int limbs) {
    PIdx r;
    r.k2 = (int)(e & ((1u << log_half) - 1));
    size_t row = e >> log_half;
    r.limb = (int)(row % limbs);
    r.part = (int)(row / limbs);
    return r;
}

__device__ __forceinline__ size_t off2(int part, int limb, int log_n, size_t part_words) {
    return (size_t)part * part_words + ((size_t)limb << log_n);
}

#define ITEM_LOOP(items_count)                                                                       \
    for (int it = blockIdx.y; it < (items_count); it += gridDim.y)                                   \
        for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < per;                      \
             e += (size_t)gridDim.x * blockDim.x)

__global__ void add_items_kernel(const BinItem* __restrict__ tab, int items, int parts, int limbs, int log_n,
                                 size_t part_words, const Prime* __restrict__ pr, bool sub) {
    const size_t per = (size_t)parts * limbs << (log_n - 1);
    ITEM_LOOP(items) {
        const BinItem t = tab[it];
        PIdx x = pidx(e, log_n - 1, limbs);
        size_t o = off2(x.part, x.limb, log_n, part_words);
        const u64 q = pr[x.limb].q;
        ulonglong2 va = reinterpret_cast<const ulonglong2*>(t.a + o)[x.k2];
        ulonglong2 vb = reinterpret_cast<const ulonglong2*>(t.b + o)[x.k2];
        ulonglong2 r;
        r.x = sub ? sub_mod(va.x, vb.x, q) : add_mod(va.x, vb.x, q);
        r.y = sub ? sub_mod(va.y, vb.y, q) : add_mod(va.y, vb.y, q);
        reinterpret_cast<ulonglong2*>(t.out + o)[x.k2] = r;
    }
}

__global__ void copy_items_kernel(const UnItem* __restrict__ tab, int items, int parts, int limbs, int log_n,
                                  size_t part_words) {
    const size_t per = (size_t)parts * limbs << (log_n - 1);
    ITEM_LOOP(items) {
        const UnItem t = tab[it];
        PIdx x = pidx(e, log_n - 1, limbs);
        size_t o = off2(x.part, x.limb, log_n, part_words);
        reinterpret_cast<ulonglong2*>(t.out + o)[x.k2] = reinterpret_cast<const ulonglong2*>(t.in + o)[x.k2];
    }
}

__global__ void mul_plain_items_kernel(const BinItem* __restrict__ tab, int items, int parts, int limbs,
                                       int log_n, size_t part_words, const Prime* __restrict__ pr) {
    const size_t per = (size_t)parts * limbs << (log_n - 1);
    ITEM_LOOP(items) {
        const BinItem t = tab[it];
        PIdx x = pidx(e, log_n - 1, limbs);
        size_t o = off2(x.part, x.limb, log_n, part_words);
        const Prime P = pr[x.limb];
        ulonglong2 va = reinterpret_cast<const ulonglong2*>(t.a + o)[x.k2];
        ulonglong2 vb = reinterpret_cast<const ulonglong2*>(t.b + ((size_t)x.limb << log_n))[x.k2];
        ulonglong2 r;
        r.x = mul_mod(va.x, vb.x, P);
        r.y = mul_mod(va.y, vb.y, P);
        reinterpret_cast<ulonglong2*>(t.out + o)[x.k2] = r;
    }
}

__device__ __forceinline__ u64 signed_mod_q(long long v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 m = (u64)(-(v + 1)) % q;
    return q - 1 - m;
}

__global__ void mul_const_items_kernel(const ConstItem* __restrict__ tab, int items, int parts, int limbs,
                                       int log_n, size_t part_words, const Prime* __restrict__ pr) {
    const size_t per = (size_t)parts * limbs << (log_n - 1);
    ITEM_LOOP(items) {
        const ConstItem t = tab[it];
        PIdx x = pidx(e, log_n - 1, limbs);
        size_t o = off2(x.part, x.limb, log_n, part_words);
        const Prime P = pr[x.limb];
        const u64 cv = signed_mod_q(t.value, P.q);
        ulonglong2 va = reinterpret_cast<const ulonglong2*>(t.in + o)[x.k2];
        ulonglong2 r;
        r.x = mul_mod(va.x, cv, P);
        r.y = mul_mod(va.y, cv, P);
        reinterpret_cast<ulonglong2*>(t.out + o)[x.k2] = r;
    }
}

__device__ __forceinline__ void tensor_pair(const u64* a, const u64* b, size_t o, size_t pw, int k2,
                                            const Prime& P, ulonglong2& d0, ulonglong2& d1, ulonglong2& d2) {
    ulonglong2 a0 = reinterpret_cast<const ulonglong2*>(a + o)[k2];
    ulonglong2 a1 = reinterpret_cast<const ulonglong2*>(a + pw + o)[k2];
    ulonglong2 b0 = reinterpret_cast<const ulonglong2*>(b + o)[k2];
    ulonglong2 b1 = reinterpret_cast<const ulonglong2*>(b + pw + o)[k2];
    d0.x = mul_mod(a0.x, b0.x, P);
    d0.y = mul_mod(a0.y, b0.y, P);
    d1.x = add_mod(mul_mod(a0.x, b1.x, P), mul_mod(a1.x, b0.x, P), P.q);
    d1.y = add_mod(mul_mod(a0.y, b1.y, P), mul_mod(a1.y, b0.y, P), P.q);
    d2.x = mul_mod(a1.x, b1.x, P);
    d2.y = mul_mod(a1.y, b1.y, P);
}

__global__ void tensor_items_kernel(const BinItem* __restrict__ tab, int items, int limbs, int log_n,
                                    size_t pw, const Prime* __restrict__ pr) {
    const size_t per = (size_t)limbs << (log_n - 1);
    ITEM_LOOP(items) {
        const BinItem t = tab[it];
        PIdx x = pidx(e, log_n - 1, limbs);
        size_t o = (size_t)x.limb << log_n;
        const Prime P = pr[x.limb];
        ulonglong2 d0, d1, d2;
        tensor_pair(t.a, t.b, o, pw, x.k2, P, d0, d1, d2);
        reinterpret_cast<ulonglong2*>(t.out + o)[x.k2] = d0;
        reinterpret_cast<ulonglong2*>(t.out + pw + o)[x.k2] = d1;
        reinterpret_cast<ulonglong2*>(t.out + 2 * pw + o)[x.k2] = d2;
    }
}

__global__ void tensor_acc_kernel(const AccTarget* __restrict__ tg, const BinItem* __restrict__ cb, int targets,
                                  int limbs, int log_n, size_t pw, const Prime* __restrict__ pr) {
    const size_t per = (size_t)limbs << (log_n - 1);
    ITEM_LOOP(targets) {
        const AccTarget t = tg[it];
        PIdx x = pidx(e, log_n - 1, limbs);
        size_t o = (size_t)x.limb << log_n;
        const Prime P = pr[x.limb];
        ulonglong2 s0 = reinterpret_cast<const ulonglong2*>(t.out + o)[x.k2];
        ulonglong2 s1 = reinterpret_cast<const ulonglong2*>(t.out + pw + o)[x.k2];
        ulonglong2 s2 = reinterpret_cast<const ulonglong2*>(t.out + 2 * pw + o)[x.k2];
        for (int j = 0; j < t.cnt; j++) {
            const BinItem c = cb[t.off + j];
            ulonglong2 d0, d1, d2;
            tensor_pair(c.a, c.b, o, pw, x.k2, P, d0, d1, d2);
            s0.x = add_mod(s0.x, d0.x, P.q);
            s0.y = add_mod(s0.y, d0.y, P.q);
            s1.x = add_mod(s1.x, d1.x, P.q);
            s1.y = add_mod(s1.y, d1.y, P.q);
            s2.x = add_mod(s2.x, d2.x, P.q);
            s2.y = add_mod(s2.y, d2.y, P.q);
        }
        reinterpret_cast<ulonglong2*>(t.out + o)[x.k2] = s0;
        reinterpret_cast<ulonglong2*>(t.out + pw + o)[x.k2] = s1;
        reinterpret_cast<ulonglong2*>(t.out + 2 * pw + o)[x.k2] = s2;
    }
}

__global__ void sum_acc_kernel(const AccTarget* __restrict__ tg, const BinItem* __restrict__ cb, int targets,
                               int parts, int limbs, int log_n, size_t pw, const Prime* __restrict__ pr) {
    const size_t per = (size_t)parts * limbs << (log_n - 1);
    ITEM_LOOP(targets) {
        const AccTarget t = tg[it];
        PIdx x = pidx(e, log_n - 1, limbs);
        size_t o = off2(x.part, x.limb, log_n, pw);
        const u64 q = pr[x.limb].q;
        ulonglong2 s = reinterpret_cast<const ulonglong2*>(t.out + o)[x.k2];
        for (int j = 0; j < t.cnt; j++) {
            ulonglong2 v = reinterpret_cast<const ulonglong2*>(cb[t.off + j].a + o)[x.k2];
            s.x = add_mod(s.x, v.x, q);
            s.y = add_mod(s.y, v.y, q);
        }
        reinterpret_cast<ulonglong2*>(t.out + o)[x.k2] = s;
    }
}

__device__ __forceinline__ u64 signed_mod(i64 v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 m = (u64)(-(v + 1)) % q;  // -(v+1) >= 0 avoids overflow at INT64_MIN
    return q - 1 - m;
}

__global__ void int_to_rns_kernel(u64* out, size_t out_stride, const i64* __restrict__ in, size_t in_stride,
                                  int items, int limbs, int log_n, const Prime* __restrict__ pr) {
    const size_t total = (size_t)items * limbs << log_n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(e & ((1u << log_n) - 1));
        size_t row = e >> log_n;
        int limb = (int)(row % limbs);
        int item = (int)(row / limbs);
        out[(size_t)item * out_stride + ((size_t)limb << log_n) + k] =
            signed_mod(in[(size_t)item * in_stride + k], pr[limb].q);
    }
}

__global__ void int8_to_rns_kernel(u64* out, size_t out_stride, const int8_t* __restrict__ in, size_t in_stride,
                                   int items, int limbs, int log_n, int split, int jump,
                                   const Prime* __restrict__ pr) {
    const size_t total = (size_t)items * limbs << log_n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(e & ((1u << log_n) - 1));
        size_t row = e >> log_n;
        int limb = (int)(row % limbs);
        int item = (int)(row / limbs);
        int prime = limb + (limb >= split ? jump : 0);
        int v = in[(size_t)item * in_stride + k];
        u64 q = pr[prime].q;
        out[(size_t)item * out_stride + ((size_t)limb << log_n) + k] = v >= 0 ? (u64)v : q - (u64)(-v);
    }
}

// Evaluation slot k holds a(psi^(2 brev(k) + 1)); X -> X^g maps it to the slot k'
// with 2 brev(k') + 1 = g (2 brev(k) + 1) mod 2N.
__device__ __forceinline__ int auto_src(int k, long long g, int log_n) {
    const unsigned sh = 32 - log_n;
    unsigned bk = __brev((unsigned)k) >> sh;
    unsigned e = (unsigned)(((unsigned long long)g * (2ull * bk + 1ull)) & ((2ull << log_n) - 1ull));
    return (int)(__brev((e - 1u) >> 1) >> sh);
}

__global__ void automorphism_kernel(u64* out, const u64* __restrict__ in, int limbs, int log_n, long long g) {
    const size_t total = (size_t)limbs << log_n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(e & ((1u << log_n) - 1));
        size_t row = e >> log_n;
        out[e] = in[(row << log_n) + auto_src(k, g, log_n)];
    }
}

}  // namespace

// ============================================================================ launchers

void items_add(Ctx& c, const std::vector<BinItem>& it, int parts, int limbs, bool sub, cudaStream_t s) {
    if (it.empty()) return;
    const BinItem* d = upload(c, it, s);
    size_t per = (size_t)parts * limbs * c.n / 2;
    {
        LaunchScope _ls(c.prof, K_ELEMENTWISE, 3.0 * 8 * per * 2 * it.size(), s);
        add_items_kernel<<<grid2(per, (int)it.size()), kThreads, 0, s>>>(d, (int)it.size(), parts, limbs, c.log_n,
                                                                     (size_t)(c.L + 1) * c.n, c.d_primes, sub);
    CK(cudaGetLastError());
    }
}

void items_copy(Ctx& c, const std::vector<UnItem>& it, int parts, int limbs, cudaStream_t s) {
    if (it.empty()) return;
    const UnItem* d = upload(c, it, s);
    size_t per = (size_t)parts * limbs * c.n / 2;
    {
        LaunchScope _ls(c.prof, K_ELEMENTWISE, 2.0 * 8 * per * 2 * it.size(), s);
        copy_items_kernel<<<grid2(per, (int)it.size()), kThreads, 0, s>>>(d, (int)it.size(), parts, limbs, c.log_n,
                                                                      (size_t)(c.L + 1) * c.n);
    CK(cudaGetLastError());
    }
}

void items_mul_plain(Ctx& c, const std::vector<BinItem>& it, int parts, int limbs, cudaStream_t s) {
    if (it.empty()) return;
    const BinItem* d = upload(c, it, s);
    size_t per = (size_t)parts * limbs * c.n / 2;
    {
        LaunchScope _ls(c.prof, K_ELEMENTWISE, 2.5 * 8 * per * 2 * it.size(), s);
        mul_plain_items_kernel<<<grid2(per, (int)it.size()), kThreads, 0, s>>>(d, (int)it.size(), parts, limbs,
                                                                           c.log_n, (size_t)(c.L + 1) * c.n,
                                                                           c.d_primes);
    CK(cudaGetLastError());
    }
}

void items_mul_const(Ctx& c, const std::vector<ConstItem>& it, int parts, int limbs, cudaStream_t s) {
    if (it.empty()) return;
    const ConstItem* d = upload(c, it, s);
    size_t per = (size_t)parts * limbs * c.n / 2;
    {
        LaunchScope _ls(c.prof, K_ELEMENTWISE, 2.0 * 8 * per * 2 * it.size(), s);
        mul_const_items_kernel<<<grid2(per, (int)it.size()), kThreads, 0, s>>>(d, (int)it.size(), parts, limbs, c.log_n,
                                                                              (size_t)(c.L + 1) * c.n, c.d_primes);
        CK(cudaGetLastError());
    }
}

void items_tensor(Ctx& c, const std::vector<BinItem>& it, int limbs, cudaStream_t s) {
    if (it.empty()) return;
    const BinItem* d = upload(c, it, s);
    size_t per = (size_t)limbs * c.n / 2;
    {
        LaunchScope _ls(c.prof, K_TENSOR, 7.0 * 8 * per * 2 * it.size(), s);
        tensor_items_kernel<<<grid2(per, (int)it.size()), kThreads, 0, s>>>(d, (int)it.size(), limbs, c.log_n,
                                                                        (size_t)(c.L + 1) * c.n, c.d_primes);
    CK(cudaGetLastError());
    }
}

void items_tensor_acc(Ctx& c, const std::vector<AccTarget>& tg, const std::vector<BinItem>& contrib, int limbs,
                      cudaStream_t s) {
    if (tg.empty()) return;
    const AccTarget* dt = upload(c, tg, s);
    const BinItem* dc = upload(c, contrib, s);
    size_t per = (size_t)limbs * c.n / 2;
    {
        LaunchScope _ls(c.prof, K_TENSOR, 8.0 * per * 2 * (4.0 * contrib.size() + 6.0 * tg.size()), s);
        tensor_acc_kernel<<<grid2(per, (int)tg.size()), kThreads, 0, s>>>(dt, dc, (int)tg.size(), limbs, c.log_n,
                                                                      (size_t)(c.L + 1) * c.n, c.d_primes);
    CK(cudaGetLastError());
    }
}

void items_sum_acc(Ctx& c, const std::vector<AccTarget>& tg, const std::vector<BinItem>& contrib, int parts,
                   int limbs, cudaStream_t s) {
    if (tg.empty()) return;
    const AccTarget* dt = upload(c, tg, s);
    const BinItem* dc = upload(c, contrib, s);
    size_t per = (size_t)parts * limbs * c.n / 2;
    {
        LaunchScope _ls(c.prof, K_ELEMENTWISE, 8.0 * per * 2 * (contrib.size() + 2.0 * tg.size()), s);
        sum_acc_kernel<<<grid2(per, (int)tg.size()), kThreads, 0, s>>>(dt, dc, (int)tg.size(), parts, limbs, c.log_n,
                                                                   (size_t)(c.L + 1) * c.n, c.d_primes);
    CK(cudaGetLastError());
    }
}

void k_int_to_rns(const Ctx& c, u64* out, size_t out_item_stride, const i64* in, size_t in_stride, int items,
                  int limbs, cudaStream_t s) {
    size_t work = (size_t)items * limbs * c.n;
    if (!work) return;
    {
        LaunchScope _ls(c.prof, K_ELEMENTWISE, 8.0 * items * c.n + 8.0 * work, s);
        int_to_rns_kernel<<<grid1(work), kThreads, 0, s>>>(out, out_item_stride, in, in_stride, items, limbs, c.log_n,
                                                       c.d_primes);
    CK(cudaGetLastError());
    }
}

void k_int8_to_rns(const Ctx& c, u64* out, size_t out_item_stride, const int8_t* in, size_t in_stride, int items,
                   int limbs, int prime_split, int prime_jump, cudaStream_t s) {
    size_t work = (size_t)items * limbs * c.n;
    if (!work) return;
    {
        LaunchScope _ls(c.prof, K_ELEMENTWISE, 1.0 * items * c.n + 8.0 * work, s);
        int8_to_rns_kernel<<<grid1(work), kThreads, 0, s>>>(out, out_item_stride, in, in_stride, items, limbs, c.log_n,
                                                        prime_split, prime_jump, c.d_primes);
    CK(cudaGetLastError());
    }
}

void k_automorphism_poly(const Ctx& c, u64* out, const u64* in, int limbs, int galois, cudaStream_t s) {
    {
        LaunchScope _ls(c.prof, K_OTHER, 16.0 * limbs * c.n, s);
        automorphism_kernel<<<grid1((size_t)limbs * c.n), kThreads, 0, s>>>(out, in, limbs, c.log_n, galois);
    CK(cudaGetLastError());
    }
}

}  // namespace fhe

// probe.cu — register-only rate of the NTT's butterfly arithmetic on this GPU.
//
// The batched NTT passes are bound by the integer pipe, not by HBM. To put a
// measured ceiling beside the one derived from lane counts and clocks, this
// kernel runs exactly the forward transform's arithmetic — lazy Shoup
// Cooley-Tukey butterflies without intermediate reduction (values stay below
// (2s+1)q after s stages, as in the transform for primes below 2^58), three
// stages per radix-8 block, a full reduction after every 15 stages — on
// values held in registers, with no shared-memory exchange, no twiddle loads
// inside the loop and no global traffic. Its butterflies per second are what
// the transform could reach if moving data were free.
#include <cstring>

#include "ntt_core.cuh"

namespace fhe {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 3;

__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
bfly_probe_kernel(u64* out, const ulonglong2* __restrict__ tw, const Prime* __restrict__ pr, int prime, int log_n,
                  int reps) {
    const u64 q = pr[prime].q, one_s = pr[prime].one_s, q2 = q << 1;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int mask = (1 << log_n) - 1;
    const ulonglong2* W = tw + ((size_t)prime << log_n);
    ulonglong2 w[7];
#pragma unroll
    for (int i = 0; i < 7; i++) w[i] = W[1 + ((tid * 7 + i) & (mask - 1))];
    u64 v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) v[u] = ((u64)tid * 8 + u) % q;
    for (int r = 0; r < reps; r++) {
#pragma unroll
        for (int blk = 0; blk < 5; blk++) {  // 15 stages
#pragma unroll
            for (int u = 0; u < 4; u++) nttc::ct_bfly<false>(v[u], v[u + 4], w[0].x, w[0].y, q, q2);
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (!(u & 2)) nttc::ct_bfly<false>(v[u], v[u + 2], w[1 + (u >> 2)].x, w[1 + (u >> 2)].y, q, q2);
#pragma unroll
            for (int u = 0; u < 8; u += 2) nttc::ct_bfly<false>(v[u], v[u + 1], w[3 + (u >> 1)].x, w[3 + (u >> 1)].y, q, q2);
        }
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = nttc::reduce_any(v[u], q, one_s);
    }
    u64 acc = 0;
#pragma unroll
    for (int u = 0; u < 8; u++) acc ^= v[u];
    out[tid] = acc;
}

}  // namespace

}  // namespace fhe

using namespace fhe;

extern "C" int fhe_probe_butterfly_rate(fhe_ctx* ctx, int32_t reps, double* gbfly_per_s) {
    if (!ctx) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    try {
        c.last_error.clear();
        CK(cudaSetDevice(c.device));
        if (!gbfly_per_s || reps < 1) fail(FHE_ERR_INVALID_ARG, "need reps >= 1 and an output pointer");
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
        const int blocks = sms * kProbeBlocksPerSm;
        const size_t threads = (size_t)blocks * kProbeThreads;
        u64* out = c.scratch_u64("probe_out", threads);
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        // one warm-up launch, then the timed one
        bfly_probe_kernel<<<blocks, kProbeThreads>>>(out, c.d_tw, c.d_primes, 0, c.log_n, 1);
        CK(cudaGetLastError());
        CK(cudaEventRecord(e0));
        bfly_probe_kernel<<<blocks, kProbeThreads>>>(out, c.d_tw, c.d_primes, 0, c.log_n, reps);
        CK(cudaGetLastError());
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        CK(cudaEventDestroy(e0));
        CK(cudaEventDestroy(e1));
        const double bflies = (double)threads * reps * 60.0;  // 15 stages x 4 butterflies per 8 values
        *gbfly_per_s = bflies / (ms * 1e-3) / 1e9;
        return FHE_OK;
    } catch (const FheException& e) {
        c.last_error = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        c.last_error = e.what();
        return FHE_ERR_INVALID_ARG;
    }
}

// ============================================================================ integer pipe rates
//
// Issue rates of the 32-bit multiply instructions every 64-bit modular product is built from:
// mad.lo.u32 (IMAD), mad.hi.u32 (IMAD.HI) and mad.wide.u32 (IMAD.WIDE, 32 x 32 + 64 -> 64), each as
// eight independent dependency chains per thread with no memory traffic. And the rate of four
// formulations of the 64 x 64 -> 128-bit multiply-accumulate of the key inner product, on register
// operands: (C) the product's low and high halves in C with a carry compare, (P64) PTX
// mad.lo.cc.u64 / madc.hi.u64, (P32) a schoolbook chain of eight 32-bit mad.lo/hi with carries,
// (W) four mad.wide.u32 partial products into 64-bit column sums with 32-bit carry counters (valid
// for operands below 2^60 and fewer than 2^32 terms).

namespace fhe {
namespace {

constexpr int kPipeThreads = 256;
constexpr int kPipeBlocksPerSm = 4;

template <int KIND>
__global__ void __launch_bounds__(kPipeThreads) imad_probe_kernel(u64* out, u32 seed, int reps) {
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    u32 a[8];
    u64 w[8];
    const u32 b = (seed ^ tid) | 1u, c = tid * 2654435761u;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        a[i] = tid * 8 + i + seed;
        w[i] = ((u64)a[i] << 17) ^ c;
    }
    for (int r = 0; r < reps; r++) {
#pragma unroll
        for (int u = 0; u < 16; u++) {
#pragma unroll
            for (int i = 0; i < 8; i++) {
                if (KIND == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
                if (KIND == 1) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
                if (KIND == 2) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[i]) : "r"(a[i]), "r"(b));
            }
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc ^= (KIND == 2 ? w[i] : (u64)a[i]);
    out[tid] = acc;
}

struct Acc128 {
    u64 lo, hi;
};

// (C): low and high product halves in C, carry by compare
__device__ __forceinline__ void mac_c(Acc128& s, u64 a, u64 b) {
    const u64 pl = a * b, ph = __umul64hi(a, b);
    s.lo += pl;
    s.hi += ph + (s.lo < pl ? 1 : 0);
}
// (P64): PTX 64-bit multiply-add with carry
__device__ __forceinline__ void mac_p64(Acc128& s, u64 a, u64 b) {
    asm volatile("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;" : "+l"(s.lo), "+l"(s.hi) : "l"(a), "l"(b));
}
// (P32): schoolbook on 32-bit words: a0 b0 and a1 b1 in one carry chain, then each cross product
__device__ __forceinline__ void mac_p32(Acc128& s, u64 a, u64 b) {
    u32 r0 = (u32)s.lo, r1 = (u32)(s.lo >> 32), r2 = (u32)s.hi, r3 = (u32)(s.hi >> 32);
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
    asm volatile(
        "mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
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
    s.lo = ((u64)r1 << 32) | r0;
    s.hi = ((u64)r3 << 32) | r2;
}
// (W): column sums. L = sum a0 b0 (mod 2^64) with carry count cl, X = sum (a0 b1 + a1 b0) (mod 2^64)
// with carry count cx, H = sum a1 b1 (no overflow for operands below 2^60 and < 256 terms).
struct AccW {
    u64 L, X, H;
    u32 cl, cx;
};
__device__ __forceinline__ void mac_w(AccW& s, u64 a, u64 b) {
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
    u64 t;
    asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(t) : "r"(a0), "r"(b0), "l"(s.L));
    s.cl += t < s.L;
    s.L = t;
    asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(t) : "r"(a0), "r"(b1), "l"(s.X));
    s.cx += t < s.X;
    s.X = t;
    asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(t) : "r"(a1), "r"(b0), "l"(s.X));
    s.cx += t < s.X;
    s.X = t;
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(s.H) : "r"(a1), "r"(b1));
}

template <int KIND>
__global__ void __launch_bounds__(kPipeThreads) mac_probe_kernel(u64* out, u64 seed, int reps) {
    const u64 tid = blockIdx.x * (u64)blockDim.x + threadIdx.x;
    const u64 m60 = ((u64)1 << 60) - 1;
    u64 a[8], b[4];
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = ((tid + i) * 0x9E3779B97F4A7C15ull ^ seed) & m60;
#pragma unroll
    for (int i = 0; i < 4; i++) b[i] = ((tid * 4 + i) * 0xBF58476D1CE4E5B9ull + seed) & m60;
    Acc128 s[4] = {};
    AccW sw[4] = {};
    for (int r = 0; r < reps; r++) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if (KIND == 0) mac_c(s[i], a[u], b[i]);
                if (KIND == 1) mac_p64(s[i], a[u], b[i]);
                if (KIND == 2) mac_p32(s[i], a[u], b[i]);
                if (KIND == 3) mac_w(sw[i], a[u], b[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++) b[i] = (b[i] + 1) & m60;   // keeps the products inside the loop
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) acc ^= s[i].lo ^ s[i].hi ^ sw[i].L ^ sw[i].X ^ sw[i].H ^ sw[i].cl ^ sw[i].cx;
    out[tid] = acc;
}

template <typename K>
double time_kernel(K launch, int warm) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int i = 0; i < warm; i++) launch(1);
    CK(cudaGetLastError());
    CK(cudaEventRecord(e0));
    launch(0);
    CK(cudaGetLastError());
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    return ms * 1e-3;
}

}  // namespace
}  // namespace fhe

extern "C" int fhe_probe_int_pipe(fhe_ctx* ctx, int32_t reps, fhe_int_pipe_rates* out) {
    if (!ctx) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    try {
        c.last_error.clear();
        CK(cudaSetDevice(c.device));
        if (!out || reps < 1) fail(FHE_ERR_INVALID_ARG, "need reps >= 1 and an output pointer");
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
        const int blocks = sms * kPipeBlocksPerSm;
        const size_t threads = (size_t)blocks * kPipeThreads;
        u64* buf = c.scratch_u64("probe_out", threads);
        std::memset(out, 0, sizeof(*out));
        out->sms = sms;
        // each mad kernel: 16 x 8 instructions per thread per rep; each MAC kernel: 8 x 4 MACs per rep
        const double n_mad = (double)threads * reps * 128.0, n_mac = (double)threads * reps * 32.0;
        double* mads[3] = {&out->imad_lo_gops, &out->imad_hi_gops, &out->imad_wide_gops};
#define MAD(K)                                                                                          \
    *mads[K] = n_mad / time_kernel([&](int w) { imad_probe_kernel<K><<<blocks, kPipeThreads>>>(buf, 7u, w ? 1 : reps); }, 1) / 1e9;
        MAD(0)
        MAD(1)
        MAD(2)
#undef MAD
        double* macs[4] = {&out->mac_c_gmacs, &out->mac_ptx64_gmacs, &out->mac_ptx32_gmacs, &out->mac_wide_gmacs};
#define MAC(K)                                                                                                   \
    *macs[K] = n_mac / time_kernel([&](int w) { mac_probe_kernel<K><<<blocks, kPipeThreads>>>(buf, 11u, w ? 1 : reps); }, 1) / 1e9;
        MAC(0)
        MAC(1)
        MAC(2)
        MAC(3)
#undef MAC
        return FHE_OK;
    } catch (const FheException& e) {
        c.last_error = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        c.last_error = e.what();
        return FHE_ERR_INVALID_ARG;
    }
}

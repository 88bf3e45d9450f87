// noalloc.cu — a rescale entry point that performs no allocation.
//
// fhe_rescale makes the context allocate (and keep) scratch buffers the first
// time it needs them, and uploads a small descriptor table through a pinned
// staging area. Some callers cannot let a library allocate at call time: an
// application that owns every byte of device memory through its own
// allocator, or a latency-critical loop in which a cudaMalloc / cudaFree (which
// can synchronise the whole device) is not acceptable. For them,
// fhe_rescale_noalloc rescales one ciphertext using only the buffers the
// caller passes plus a fixed scratch array compiled into this library.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchWords words
// (16 MiB). Every GPU that loads the library holds it until the process exits.
// Host code may not use the array's name as a device address: at the first
// call on each device (with that device current) its address is obtained with
// cudaGetSymbolAddress and cached; kernels receive that address.
#include <mutex>

#include "core.cuh"

namespace fhe {

namespace {

constexpr size_t kNoAllocScratchWords = (size_t)2 << 20;  // 16 MiB of u64
constexpr int kMaxDevices = 64;

static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocScratchWords];

std::mutex g_noalloc_mu;
u64* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for `device` (set up once per device).
u64* noalloc_scratch(int device) {
    if (device < 0 || device >= kMaxDevices) fail(FHE_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) fail(FHE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[device] = (u64*)p;
    }
    return g_noalloc_ptr[device];
}

// last[p][k] = in[p][level][k], components p < 2
__global__ void na_gather_last(u64* last, const u64* __restrict__ in, size_t part_words, int level, int log_n) {
    const size_t total = (size_t)2 << log_n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        size_t p = e >> log_n, k = e & (((size_t)1 << log_n) - 1);
        last[e] = in[p * part_words + ((size_t)level << log_n) + k];
    }
}

// spread[p][i][k] = centred(last[p][k]) mod q_i, i < level
__global__ void na_spread(u64* spread, const u64* __restrict__ last, int level, int log_n, const Prime* __restrict__ pr) {
    const size_t total = (size_t)2 << log_n;
    const u64 ql = pr[level].q;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        size_t p = e >> log_n, k = e & (((size_t)1 << log_n) - 1);
        u64 r = last[e];
        bool neg = r > (ql >> 1);
        u64 mag = neg ? ql - r : r;
        for (int i = 0; i < level; i++) {
            const Prime P = pr[i];
            // mag mod q_i by a Shoup product with 1 (floor(2^64 / q_i)) and one correction
            u64 m = mag - __umul64hi(mag, P.one_s) * P.q;
            m = m >= P.q ? m - P.q : m;
            spread[((p * level + i) << log_n) + k] = neg ? (m ? P.q - m : 0) : m;
        }
    }
}

// out[p][i] = (in[p][i] - spread[p][i]) * q_level^-1 mod q_i
__global__ void na_combine(u64* out, const u64* __restrict__ in, const u64* __restrict__ spread, size_t part_words,
                           int level, int log_n, const Prime* __restrict__ pr, const u64* __restrict__ resc_row) {
    const size_t total = (size_t)2 * level << log_n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        size_t row = e >> log_n, k = e & (((size_t)1 << log_n) - 1);
        int p = (int)(row / level), i = (int)(row % level);
        const u64 q = pr[i].q;
        const size_t o = (size_t)p * part_words + ((size_t)i << log_n) + k;
        u64 d = sub_mod(in[o], spread[e], q);
        u64 qh = __umul64hi(d, resc_row[2 * i + 1]);
        u64 r = d * resc_row[2 * i] - qh * q;
        out[o] = r >= q ? r - q : r;
    }
}

inline unsigned blocks(size_t work) { return (unsigned)std::min<size_t>(std::max<size_t>((work + 255) / 256, 1), 1u << 20); }

}  // namespace

}  // namespace fhe

using namespace fhe;

extern "C" int fhe_rescale_noalloc(fhe_ctx* ctx, const uint64_t* ct, uint64_t* out, int32_t level, void* stream) {
    if (!ctx) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    try {
        c.last_error.clear();
        CK(cudaSetDevice(c.device));
        if (!ct || !out) fail(FHE_ERR_INVALID_ARG, "null pointer");
        if (level < 1 || level > c.L) fail(level < 1 ? FHE_ERR_LEVEL_EXHAUSTED : FHE_ERR_INVALID_ARG,
                                           "rescale needs 1 <= level <= top level");
        const size_t n = (size_t)c.n;
        const size_t need = 2 * n + 2 * (size_t)level * n;  // last limb of both components + spread limbs
        if (need > kNoAllocScratchWords)
            fail(FHE_ERR_INVALID_ARG, "ciphertext too large for the 16 MiB static scratch of fhe_rescale_noalloc "
                                      "(needs 2*N*(level+1) <= 2^21 words)");
        u64* scratch = noalloc_scratch(c.device);
        // launch accounting stays on, but this call records no per-launch events (creating one may
        // allocate); the switch is per host thread, so other threads' profiling is unaffected
        NoLaunchEvents no_events;
        u64* last = scratch;
        u64* spread = scratch + 2 * n;
        const size_t pw = (size_t)(c.L + 1) * n;
        cudaStream_t s = (cudaStream_t)stream;
        na_gather_last<<<blocks(2 * n), 256, 0, s>>>(last, ct, pw, level, c.log_n);
        CK(cudaGetLastError());
        ntt_inverse(c, poly_batch(last, n, 0, 2, 1, level, 1, level), s);
        na_spread<<<blocks(2 * n), 256, 0, s>>>(spread, last, level, c.log_n, c.d_primes);
        CK(cudaGetLastError());
        ntt_forward(c, poly_batch(spread, (size_t)level * n, 0, 2, 1, 0, level), s);
        na_combine<<<blocks(2 * (size_t)level * n), 256, 0, s>>>(out, ct, spread, pw, level, c.log_n, c.d_primes,
                                                                 c.d_resc + (size_t)2 * level * (c.L + 1));
        CK(cudaGetLastError());
        return FHE_OK;
    } catch (const FheException& e) {
        c.last_error = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        c.last_error = e.what();
        return FHE_ERR_INVALID_ARG;
    }
}

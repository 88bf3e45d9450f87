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

// tune.cu — the autotuner: times every launch variant of a kernel family on a synthetic batch of the
// context's own shape and keeps the fastest for the context. Every variant of a family computes the
// same bits (the choice changes speed only), so tuning never changes a result.
//
// Families:
//   ks_hoist_inner  K3 of the hoisted rotate-and-sum (kp - 1 = 15 rotations, the epoch's per-group
//                   rotate-and-sum), variants of ks_inner.cuh
//   ks_inner        K3 of a relinearisation (every item shares the key), variants of ks_inner.cuh
// The synthetic operands are uniform residues below each prime; the kernels' work does not depend
// on the values.
#include <cstring>
#include <vector>

#include "ks_inner.cuh"
#include "ks_pass.cuh"
#include "ntt_tile.cuh"

using namespace fhe;

namespace {

struct Family {
    const char* name;
    int n_variants;
    const char* const* variant_names;
    int Ctx::Tune::*field;
};

const Family kFamilies[] = {
    {"ks_hoist_inner", INNER_N_VARIANTS, kInnerVariantNames, &Ctx::Tune::hoist},
    {"ks_inner", INNER_N_VARIANTS, kInnerVariantNames, &Ctx::Tune::inner},
    {"ntt", ntt_tile::NTT_N_TILES, ntt_tile::kNttTileNames, &Ctx::Tune::ntt},
    {"ks_pass", ksp::KS_N_TILES, ksp::kKsTileNames, &Ctx::Tune::ks},
};

__global__ void fill_residues(u64* p, size_t words, int log_n, int n_limbs, const Prime* __restrict__ pr, u64 seed) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < words; e += (size_t)gridDim.x * blockDim.x) {
        const int limb = (int)((e >> log_n) % (size_t)n_limbs);
        u64 z = (e + seed) * 0x9E3779B97F4A7C15ull;
        z ^= z >> 31;
        p[e] = z % pr[limb].q;
    }
}

struct DevTmp {
    std::vector<void*> ptrs;
    u64* get(size_t words) {
        void* p = nullptr;
        CK(cudaMalloc(&p, words * sizeof(u64)));
        ptrs.push_back(p);
        return (u64*)p;
    }
    ~DevTmp() {
        for (void* p : ptrs) cudaFree(p);
    }
};

template <typename F>
double time_ms(F&& run, int reps) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    run();  // warm-up
    double best = 1e30;
    for (int r = 0; r < reps; r++) {
        CK(cudaEventRecord(e0));
        run();
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// Time every variant of the two inner-product families at `level`.
void tune_inner(Ctx& c, int level, std::vector<fhe_tune_result>& out) {
    const int n = c.n, A = c.alpha, l1 = level + 1, next = l1 + A, dn = c.dnum(level);
    const int items = c.log_n >= 16 ? 32 : 64, steps = 15;
    DevTmp tmp;
    // ext: [items][dn][next][N]; keys: [steps][dnum_top][2][n_ext][N]; inputs [items][L+1][N]; acc, c0sum
    const size_t key_words = c.key_words();
    u64* ext = tmp.get((size_t)items * dn * next * n);
    u64* keys = tmp.get((size_t)steps * key_words);
    u64* din = tmp.get((size_t)items * (c.L + 1) * n);
    u64* c0 = tmp.get((size_t)items * (c.L + 1) * n);
    u64* acc = tmp.get((size_t)items * 2 * next * n);
    u64* c0sum = tmp.get((size_t)items * l1 * n);
    // the key rows are laid out [digit][2][n_ext]; residues below the smallest prime serve every row
    fill_residues<<<1024, 256>>>(ext, (size_t)items * dn * next * n, c.log_n, 1, c.d_primes, 1);
    fill_residues<<<1024, 256>>>(keys, (size_t)steps * key_words, c.log_n, 1, c.d_primes, 2);
    fill_residues<<<1024, 256>>>(din, (size_t)items * (c.L + 1) * n, c.log_n, 1, c.d_primes, 3);
    fill_residues<<<1024, 256>>>(c0, (size_t)items * (c.L + 1) * n, c.log_n, 1, c.d_primes, 4);
    CK(cudaGetLastError());
    std::vector<KsItem> it(items);
    for (int t = 0; t < items; t++) {
        it[t] = KsItem{din + (size_t)t * (c.L + 1) * n, keys, c0 + (size_t)t * (c.L + 1) * n, nullptr, nullptr,
                       nullptr, nullptr, 1};
    }
    std::vector<HoistStep> hs(steps);
    for (int r = 0; r < steps; r++) hs[r] = {keys + (size_t)r * key_words, (long long)c.galois(r + 1)};
    KsItem* d_it = nullptr;
    HoistStep* d_hs = nullptr;
    CK(cudaMalloc(&d_it, sizeof(KsItem) * items));
    CK(cudaMalloc(&d_hs, sizeof(HoistStep) * steps));
    tmp.ptrs.push_back(d_it);
    tmp.ptrs.push_back(d_hs);
    CK(cudaMemcpy(d_it, it.data(), sizeof(KsItem) * items, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_hs, hs.data(), sizeof(HoistStep) * steps, cudaMemcpyHostToDevice));
    InnerArgs ia{};
    ia.acc = acc;
    ia.c0sum = c0sum;
    ia.ext = ext;
    ia.tab = d_it;
    ia.items = items;
    ia.dn = dn;
    ia.alpha = A;
    ia.next = next;
    ia.level = level;
    ia.L = c.L;
    ia.n_ext = c.n_ext;
    ia.log_n = c.log_n;
    ia.pr = c.d_primes;
    ia.keys_packed = c.keys_packed;
    for (int f = 0; f < 2; f++) {
        const Family& fam = kFamilies[f];
        const bool hoist = f == 0;
        InnerArgs a = ia;
        if (hoist) {
            a.steps = d_hs;
            a.n_steps = steps;
        } else {
            a.shared_key = keys;
            a.shared_galois = 1;
        }
        double best = 1e30;
        int best_v = 0;
        const size_t first = out.size();
        for (int v = 0; v < fam.n_variants; v++) {
            const double ms = time_ms([&] {
                if (hoist) launch_ks_hoist_inner(a, v, c.max_data_prime_bits, (cudaStream_t)0);
                else launch_ks_inner(a, false, v, c.max_data_prime_bits, (cudaStream_t)0);
            }, 3);
            out.push_back(fhe_tune_result{fam.name, fam.variant_names[v], 0, ms});
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        out[first + best_v].chosen = 1;
        c.tune.*fam.field = best_v;
    }
    CK(cudaDeviceSynchronize());
}

// Time every tile shape of the plain two-pass NTT (forward then inverse of the same rows; rings of
// 2^14 and more only) on 32 limb rows per limb of the context (at least 256 rows).
void tune_ntt(Ctx& c, std::vector<fhe_tune_result>& out) {
    const Family& fam = kFamilies[2];
    if (c.log_n < 14) return;
    const int L1 = c.L + 1, polys = std::max(1, 256 / L1 + (256 % L1 ? 1 : 0));
    DevTmp tmp;
    u64* buf = tmp.get((size_t)polys * L1 * c.n);
    fill_residues<<<1024, 256>>>(buf, (size_t)polys * L1 * c.n, c.log_n, 1, c.d_primes, 5);
    CK(cudaGetLastError());
    const PolyBatch pb = poly_batch(buf, (size_t)L1 * c.n, 0, polys, 1, 0, L1);
    const int saved = c.tune.ntt;
    double best = 1e30;
    int best_v = 0;
    const size_t first = out.size();
    for (int v = 0; v < fam.n_variants; v++) {
        c.tune.ntt = v;
        const double ms = time_ms([&] {
            ntt_forward(c, pb, (cudaStream_t)0);
            ntt_inverse(c, pb, (cudaStream_t)0);
        }, 3);
        out.push_back(fhe_tune_result{fam.name, fam.variant_names[v], 0, ms});
        if (ms < best) {
            best = ms;
            best_v = v;
        }
    }
    (void)saved;
    out[first + best_v].chosen = 1;
    c.tune.ntt = best_v;
    CK(cudaDeviceSynchronize());
}

// Time every tile shape of the fused key-switch / rescale passes on the exact rescale of 64 synthetic
// ciphertexts at `level` (an inverse pass with the gather load and scaled store, a forward pass with
// the centred load and the rescale store; rings of 2^14 and more only).
void tune_ks(Ctx& c, int level, std::vector<fhe_tune_result>& out) {
    const Family& fam = kFamilies[3];
    if (c.log_n < 14) return;
    const int items = 64;
    DevTmp tmp;
    const size_t w = c.ct_words();
    u64* in = tmp.get((size_t)items * w);
    u64* res = tmp.get((size_t)items * w);
    fill_residues<<<1024, 256>>>(in, (size_t)items * w, c.log_n, 1, c.d_primes, 6);
    CK(cudaGetLastError());
    std::vector<UnItem> it;
    for (int t = 0; t < items; t++) it.push_back({in + (size_t)t * w, res + (size_t)t * w});
    double best = 1e30;
    int best_v = 0;
    const size_t first = out.size();
    for (int v = 0; v < fam.n_variants; v++) {
        c.tune.ks = v;
        const double ms = time_ms([&] { items_rescale(c, it, 2, level, (cudaStream_t)0); }, 3);
        out.push_back(fhe_tune_result{fam.name, fam.variant_names[v], 0, ms});
        if (ms < best) {
            best = ms;
            best_v = v;
        }
    }
    out[first + best_v].chosen = 1;
    c.tune.ks = best_v;
    CK(cudaDeviceSynchronize());
}

template <typename F>
int guarded(Ctx& c, F&& f) {
    try {
        c.last_error.clear();
        CK(cudaSetDevice(c.device));
        f();
        return FHE_OK;
    } catch (const FheException& e) {
        c.last_error = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        c.last_error = e.what();
        return FHE_ERR_INVALID_ARG;
    }
}

}  // namespace

extern "C" int fhe_autotune(fhe_ctx* ctx, int32_t level, fhe_tune_result* out, int32_t cap) {
    if (!ctx) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    std::vector<fhe_tune_result> res;
    int rc = guarded(c, [&] {
        if (level < 1 || level > c.L) fail(FHE_ERR_INVALID_ARG, "autotune level out of range");
        if (cap < 0 || (cap > 0 && !out)) fail(FHE_ERR_INVALID_ARG, "bad output array");
        CK(cudaDeviceSynchronize());
        tune_inner(c, level, res);
        tune_ntt(c, res);
        tune_ks(c, level, res);
        c.arena.reset((cudaStream_t)0);
    });
    if (rc) return rc;
    const int n = (int)std::min<size_t>(res.size(), (size_t)cap);
    for (int i = 0; i < n; i++) out[i] = res[i];
    return (int)res.size();
}

extern "C" int fhe_set_variant(fhe_ctx* ctx, const char* family, const char* variant) {
    if (!ctx) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    return guarded(c, [&] {
        if (!family || !variant) fail(FHE_ERR_INVALID_ARG, "null family or variant");
        for (const Family& fam : kFamilies) {
            if (std::strcmp(fam.name, family) != 0) continue;
            for (int v = 0; v < fam.n_variants; v++)
                if (std::strcmp(fam.variant_names[v], variant) == 0) {
                    c.tune.*fam.field = v;
                    return;
                }
            fail(FHE_ERR_INVALID_ARG, std::string("unknown variant ") + variant + " of " + family);
        }
        fail(FHE_ERR_INVALID_ARG, std::string("unknown kernel family ") + family);
    });
}

extern "C" int fhe_get_variant(const fhe_ctx* ctx, const char* family, const char** variant) {
    if (!ctx || !family || !variant) return FHE_ERR_INVALID_ARG;
    const Ctx& c = ctx->c;
    for (const Family& fam : kFamilies)
        if (std::strcmp(fam.name, family) == 0) {
            *variant = fam.variant_names[c.tune.*fam.field];
            return FHE_OK;
        }
    return FHE_ERR_INVALID_ARG;
}

extern "C" int fhe_probe_conv_cost(fhe_ctx* ctx, int32_t level, int32_t sources, fhe_conv_cost* out) {
    if (!ctx) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    return guarded(c, [&] {
        if (level < 1 || level > c.L) fail(FHE_ERR_INVALID_ARG, "level out of range");
        if (sources < 1 || !out) fail(FHE_ERR_INVALID_ARG, "need sources >= 1 and an output");
        CK(cudaDeviceSynchronize());
        const int n = c.n, L = c.L, A = c.alpha, l1 = level + 1, next = l1 + A, dn = c.dnum(level);
        DevTmp tmp;
        u64* y = tmp.get((size_t)sources * l1 * n);
        u64* ext = tmp.get((size_t)sources * dn * next * n);
        fill_residues<<<1024, 256>>>(y, (size_t)sources * l1 * n, c.log_n, 1, c.d_primes, 7);
        CK(cudaGetLastError());
        // the rows of the conversion step (K2 of the key switch), and the same rows with a plain load
        std::vector<ksp::KsRow> rc, rp;
        for (int t = 0; t < sources; t++)
            for (int j = 0; j < dn; j++) {
                const int lo = j * A, cnt = std::min(A, l1 - lo);
                for (int x = 0; x < next; x++) {
                    if (x >= lo && x < lo + cnt) continue;
                    const int px = x < l1 ? x : x + (L - level);
                    ksp::KsRow r{};
                    r.dst = ext + (((size_t)t * dn + j) * next + x) * n;
                    r.src = y + ((size_t)t * l1 + lo) * n;
                    r.cst = c.d_up_hat + 2 * (((size_t)level * (L + 1) + lo) * c.n_ext + px);
                    r.cst_stride = 2 * c.n_ext;
                    r.src_cnt = cnt;
                    r.prime = px;
                    r.galois = 1;
                    r.pack = c.keys_packed && x < l1;
                    rc.push_back(r);
                    r.src_cnt = 1;
                    rp.push_back(r);
                }
            }
        const int rows = (int)rc.size();
        const ksp::KsRow* d_rc = c.arena.push_vec(rc, (cudaStream_t)0);
        const ksp::KsRow* d_rp = c.arena.push_vec(rp, (cudaStream_t)0);
        const ksp::CombineArgs none{nullptr, nullptr, nullptr, 0, nullptr};
        const double bytes = 16.0 * rows * n;
        out->conv_ms = time_ms(
            [&] { ksp::ks_transform<false, ksp::LD_CONV, ksp::ST_LAST>(c, d_rc, rows, none, K_NTT_FWD, bytes, 0); }, 5);
        out->plain_ms = time_ms(
            [&] { ksp::ks_transform<false, ksp::LD_GATHER, ksp::ST_LAST>(c, d_rp, rows, none, K_NTT_FWD, bytes, 0); },
            5);
        out->rows = rows;
        out->roundtrip_bytes = bytes;
        CK(cudaDeviceSynchronize());
        c.arena.reset((cudaStream_t)0);
    });
}

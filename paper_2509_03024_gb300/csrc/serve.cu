// serve.cu — continuous-batching request loop: encrypted per-user fold-in
// (Alg. 1 error/gradient lines, Alg. 2 accumulated update, item factors fixed)
// and the encrypted predicted-rating row, over resident item factors.
//
// Each request lives in a slot (its inputs, masks, running factor and a share
// of the work area). A tick advances every admitted request by one step; all
// requests at the same level share one launch per kernel, and the levels
// present in a tick are processed one after another.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "core.cuh"

using namespace fhe;

namespace {

int npow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}
int hb(int x) { return 31 - __builtin_clz((unsigned)x); }

struct Slot {
    bool used = false;
    bool done = false;
    long long id = -1;
    int step = 0;
    int level = 0;
    int nnz = 0;
    std::vector<int> batches;  // item batches holding a rated item
    u64* UR = nullptr;         // running user factor ciphertext
    u64* R = nullptr;          // n_vb rating ciphertexts
    u64* out = nullptr;        // n_vb prediction ciphertexts
    i64* mask = nullptr;       // n_vb int64 mask encodings
    u64* work = nullptr;       // per-slot work area
};

}  // namespace

struct fhe_server {
    Ctx* c = nullptr;
    int m = 0, k = 0, kp = 0, w = 0, B = 0, beta = 0, log_kp = 0, n_vb = 0, steps = 0;
    double lr = 0, lam = 0;
    u64* V = nullptr;
    std::vector<Slot> slots;
    std::vector<void*> allocs;
    // requests whose last step was enqueued by a tick, with the event recorded after that tick's work;
    // poll() reports them once the event has completed
    struct Done {
        cudaEvent_t ev;
        std::vector<long long> ids;
    };
    std::vector<long long> finishing;   // filled while a tick is being enqueued
    std::vector<Done> done_q;
    std::vector<cudaEvent_t> ev_pool;
    ~fhe_server() {
        for (Done& d : done_q) ev_pool.push_back(d.ev);
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        for (void* p : allocs) cudaFree(p);
        if (V) cudaFree(V);
    }
};

namespace {

// per-slot work area layout (in units of lw = (L+1) N words):
//   per batch c: T3 (3) | S (2) | tmp (2) | E (2) | MV (2) | PT (1)  = 12
//   then: T (3) | G (2) | Gtmp (2) | base (2)                         = 9
constexpr int kPerBatch = 12;
constexpr int kTail = 9;

struct SlotWork {
    u64 *T3, *S, *tmp, *E, *MV, *PT;
    u64 *T, *G, *Gt, *base;
};
SlotWork work_of(const fhe_server& sv, const Slot& sl, int cb) {
    const size_t lw = sv.c->ct_words() / 2;
    SlotWork wk;
    u64* b = sl.work + (size_t)cb * kPerBatch * lw;
    wk.T3 = b;
    wk.S = b + 3 * lw;
    wk.tmp = b + 5 * lw;
    wk.E = b + 7 * lw;
    wk.MV = b + 9 * lw;
    wk.PT = b + 11 * lw;
    u64* t = sl.work + (size_t)sv.n_vb * kPerBatch * lw;
    wk.T = t;
    wk.G = t + 3 * lw;
    wk.Gt = t + 5 * lw;
    wk.base = t + 7 * lw;
    return wk;
}

// The gradient's block sum over the B slot blocks followed by the half-fill, as rounds of hoisted
// rotate-and-sums: radix-4 rounds with strides w, 4w, 16w, ... (steps 0, s, 2s, 3s), a radix-2 round
// when log2 B is odd, the half-fill rotation by -kp merged into the last round (its steps r and r - kp).
// One step per round, summed, meets every block offset a w once, and every one again shifted by -kp.
std::vector<std::vector<int>> block_sum_rounds(int kp, int w, int B) {
    std::vector<std::vector<int>> rounds;
    const int lb = hb(B);
    int stride = w;
    for (int t = 0; t < lb;) {
        const int r = lb - t >= 2 ? 4 : 2;
        std::vector<int> rnd;
        for (int j = 0; j < r; j++) rnd.push_back(j * stride);
        rounds.push_back(rnd);
        stride *= r;
        t += r == 4 ? 2 : 1;
    }
    std::vector<int> last = rounds.empty() ? std::vector<int>{0} : rounds.back();
    if (!rounds.empty()) rounds.pop_back();
    const size_t n = last.size();
    for (size_t i = 0; i < n; i++) last.push_back(last[i] - kp);
    rounds.push_back(last);
    return rounds;
}

// Inner products of every (slot, batch) pair listed, at `level`: result in wk.S (level - 1).
void inner_products(fhe_server& sv, const std::vector<std::pair<Slot*, int>>& pairs, int level, cudaStream_t s) {
    Ctx& c = *sv.c;
    const size_t w = c.ct_words();
    std::vector<BinItem> tens;
    std::vector<u64*> t3;
    std::vector<u64*> prod, res;
    for (auto& pr : pairs) {
        SlotWork wk = work_of(sv, *pr.first, pr.second);
        tens.push_back({pr.first->UR, sv.V + (size_t)pr.second * w, wk.T3});
        t3.push_back(wk.T3);
        prod.push_back(wk.tmp);
        res.push_back(wk.S);
    }
    items_tensor(c, tens, level + 1, s);
    relin_rescale_items(c, t3, prod, level, s);
    rotsum_items(c, prod, res, sv.kp, level - 1, s);
}

void fold_in_step(fhe_server& sv, const std::vector<Slot*>& group, int level, cudaStream_t s) {
    Ctx& c = *sv.c;
    const size_t w = c.ct_words(), lw = w / 2;
    std::vector<std::pair<Slot*, int>> pairs;
    for (Slot* sl : group)
        for (int cb : sl->batches) pairs.push_back({sl, cb});
    inner_products(sv, pairs, level, s);
    // E = R - S, MV = rescale(V (.) mask)
    std::vector<BinItem> esub, pm;
    for (Slot* sl : group)  // all of a slot's mask encodings at once (PT of batch c at stride kPerBatch lw)
        materialize_plain(c, sl->mask, c.n, sv.n_vb, level + 1, work_of(sv, *sl, 0).PT, kPerBatch * lw, s);
    for (auto& pr : pairs) {
        SlotWork wk = work_of(sv, *pr.first, pr.second);
        esub.push_back({pr.first->R + (size_t)pr.second * w, wk.S, wk.E});
        pm.push_back({sv.V + (size_t)pr.second * w, wk.PT, wk.MV});
    }
    items_add(c, esub, 2, level, true, s);
    mul_plain_rescale_items(c, pm, level, s);
    // T = sum_c E (x) MV
    std::vector<AccTarget> tg;
    std::vector<BinItem> cb;
    for (Slot* sl : group) {
        SlotWork wt = work_of(sv, *sl, 0);
        CK(cudaMemsetAsync(wt.T, 0, sizeof(u64) * 3 * lw, s));
        tg.push_back({wt.T, (int)cb.size(), (int)sl->batches.size()});
        for (int b : sl->batches) {
            SlotWork wk = work_of(sv, *sl, b);
            cb.push_back({wk.E, wk.MV, nullptr});
        }
    }
    items_tensor_acc(c, tg, cb, level, s);
    // G = rescale(relin(T)), block sums, half-fill
    std::vector<u64*> t3, gs;
    for (Slot* sl : group) {
        SlotWork wt = work_of(sv, *sl, 0);
        t3.push_back(wt.T);
        gs.push_back(wt.G);
    }
    relin_rescale_items(c, t3, gs, level - 1, s);
    const int l2 = level - 2;
    for (const std::vector<int>& steps : block_sum_rounds(sv.kp, sv.w, sv.B)) {  // block sum, half-fill
        std::vector<u64*> gv;
        for (Slot* sl : group) gv.push_back(work_of(sv, *sl, 0).G);
        hoisted_sum_items(c, gv, gv, steps, l2, s);
    }
    // UR <- drop(rescale(UR * round(reg Delta))) + G
    std::vector<ConstItem> cm;
    std::vector<UnItem> rb;
    std::vector<BinItem> fin;
    for (Slot* sl : group) {
        SlotWork wt = work_of(sv, *sl, 0);
        double reg = 1.0 - sv.lr * sv.lam * sl->nnz;
        long long cv = (long long)std::nearbyint(reg * std::ldexp(1.0, c.log_scale));
        cm.push_back({sl->UR, wt.base, cv});
        rb.push_back({wt.base, wt.base});
        fin.push_back({wt.base, wt.G, sl->UR});
    }
    items_mul_const(c, cm, 2, level + 1, s);
    items_rescale(c, rb, 2, level, s);
    items_add(c, fin, 2, l2 + 1, false, s);
    for (Slot* sl : group) {
        sl->step++;
        sl->level = l2;
    }
}

void predict_pass(fhe_server& sv, const std::vector<Slot*>& group, int level, cudaStream_t s) {
    Ctx& c = *sv.c;
    const size_t w = c.ct_words();
    std::vector<std::pair<Slot*, int>> pairs;
    for (Slot* sl : group)
        for (int cb = 0; cb < sv.n_vb; cb++) pairs.push_back({sl, cb});
    inner_products(sv, pairs, level, s);
    std::vector<UnItem> cp;
    for (auto& pr : pairs) cp.push_back({work_of(sv, *pr.first, pr.second).S, pr.first->out + (size_t)pr.second * w});
    items_copy(c, cp, 2, level, s);
    for (Slot* sl : group) {
        sl->level = level - 1;
        sl->done = true;
        sv.finishing.push_back(sl->id);
    }
}

template <typename F>
int guarded(Ctx* c, F&& f) {
    try {
        if (c) {
            c->last_error.clear();
            CK(cudaSetDevice(c->device));
        }
        f();
        return FHE_OK;
    } catch (const FheException& e) {
        if (c) c->last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->last_error = "host allocation failed";
        return FHE_ERR_OOM;
    } catch (const std::exception& e) {
        if (c) c->last_error = e.what();
        return FHE_ERR_INVALID_ARG;
    }
}

}  // namespace

extern "C" {

int fhe_serve_rotation_steps(const fhe_ctx* ctx, int32_t k, int32_t* out, size_t cap) {
    if (!ctx || k < 1) return FHE_ERR_INVALID_ARG;
    const Ctx& c = ctx->c;
    int kp = npow2(k), w = 2 * kp;
    if (w > c.slots) return FHE_ERR_INVALID_ARG;
    int B = c.slots / w;
    std::vector<int> st = rotsum_steps(kp);
    for (const std::vector<int>& rnd : block_sum_rounds(kp, w, B))
        for (int x : rnd)
            if (x != 0 && std::find(st.begin(), st.end(), x) == st.end()) st.push_back(x);
    if (out) {
        if (cap < st.size()) return FHE_ERR_INVALID_ARG;
        std::copy(st.begin(), st.end(), out);
    }
    return (int)st.size();
}

int fhe_serve_create(fhe_ctx* ctx, const uint64_t* V, int32_t m, int32_t k, int32_t steps, double lr, double lam,
                     int32_t max_slots, size_t budget, fhe_server** out) {
    if (!ctx || !out) return FHE_ERR_INVALID_ARG;
    *out = nullptr;
    fhe_server* sv = new (std::nothrow) fhe_server();
    if (!sv) return FHE_ERR_OOM;
    Ctx& c = ctx->c;
    int rc = guarded(&c, [&] {
        if (!V || m < 1 || k < 1 || steps < 0 || max_slots < 1) fail(FHE_ERR_INVALID_ARG, "bad server arguments");
        if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
        if (c.L < 2 * steps + 1) fail(FHE_ERR_LEVEL_EXHAUSTED, "the modulus chain is too short for the steps");
        if (!std::isfinite(lr) || !std::isfinite(lam)) fail(FHE_ERR_INVALID_ARG, "non-finite lr or lambda");
        sv->c = &c;
        sv->m = m;
        sv->k = k;
        sv->kp = npow2(k);
        sv->w = 2 * sv->kp;
        if (sv->w > c.slots) fail(FHE_ERR_INVALID_ARG, "rank too large for the ring");
        sv->B = c.slots / sv->w;
        sv->beta = hb(sv->B);
        sv->log_kp = hb(sv->kp);
        sv->n_vb = (m + sv->B - 1) / sv->B;
        sv->steps = steps;
        sv->lr = lr;
        sv->lam = lam;
        for (int r : rotsum_steps(sv->kp)) rotation_key(c, r);
        for (const std::vector<int>& rnd : block_sum_rounds(sv->kp, sv->w, sv->B))
            for (int x : rnd)
                if (x != 0) rotation_key(c, x);
        const size_t w = c.ct_words(), lw = w / 2;
        CK(cudaMalloc((void**)&sv->V, sizeof(u64) * w * sv->n_vb));
        CK(cudaMemcpy(sv->V, V, sizeof(u64) * w * sv->n_vb, cudaMemcpyDeviceToDevice));
        const size_t per_slot = sizeof(u64) * (w * (1 + 2 * (size_t)sv->n_vb) +
                                               lw * ((size_t)sv->n_vb * kPerBatch + kTail)) +
                                sizeof(i64) * (size_t)sv->n_vb * c.n;
        int n = max_slots;
        if (budget) n = (int)std::min<size_t>(n, std::max<size_t>(1, budget / per_slot));
        sv->slots.resize(n);
        for (Slot& sl : sv->slots) {
            char* p = nullptr;
            CK(cudaMalloc((void**)&p, per_slot));
            sv->allocs.push_back(p);
            sl.UR = (u64*)p;
            sl.R = sl.UR + w;
            sl.out = sl.R + w * sv->n_vb;
            sl.work = sl.out + w * sv->n_vb;
            sl.mask = (i64*)(sl.work + lw * ((size_t)sv->n_vb * kPerBatch + kTail));
        }
    });
    if (rc) {
        delete sv;
        return rc;
    }
    *out = sv;
    return FHE_OK;
}

void fhe_serve_destroy(fhe_server* sv) {
    if (sv) {
        if (sv->c) cudaSetDevice(sv->c->device);
        cudaDeviceSynchronize();
        delete sv;
    }
}

int fhe_serve_slots(const fhe_server* sv, int32_t* total, int32_t* free_slots) {
    if (!sv) return FHE_ERR_INVALID_ARG;
    int f = 0;
    for (const Slot& sl : sv->slots) f += !sl.used;
    if (total) *total = (int32_t)sv->slots.size();
    if (free_slots) *free_slots = f;
    return FHE_OK;
}

int fhe_serve_submit(fhe_server* sv, int64_t id, const int32_t* items, int32_t nnz, const uint64_t* UR,
                     const uint64_t* R, void* stream) {
    if (!sv) return FHE_ERR_INVALID_ARG;
    Ctx& c = *sv->c;
    return guarded(&c, [&] {
        if (!UR || !R || nnz < 0 || (nnz > 0 && !items)) fail(FHE_ERR_INVALID_ARG, "bad request");
        Slot* free_slot = nullptr;
        for (Slot& sl : sv->slots) {
            if (sl.used && sl.id == id) fail(FHE_ERR_INVALID_ARG, "request id already in flight");
            if (!sl.used && !free_slot) free_slot = &sl;
        }
        if (!free_slot) fail(FHE_ERR_STATE, "no free request slot");
        std::vector<int> it(items, items + nnz);
        std::sort(it.begin(), it.end());
        for (int t = 0; t < nnz; t++) {
            if (it[t] < 0 || it[t] >= sv->m) fail(FHE_ERR_INVALID_ARG, "item index out of range");
            if (t && it[t] == it[t - 1]) fail(FHE_ERR_INVALID_ARG, "duplicate item in request");
        }
        cudaStream_t s = (cudaStream_t)stream;
        Slot& sl = *free_slot;
        const size_t w = c.ct_words();
        CK(cudaMemcpyAsync(sl.UR, UR, sizeof(u64) * w, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(sl.R, R, sizeof(u64) * w * sv->n_vb, cudaMemcpyDefault, s));
        // learning-rate masks of the rated blocks, one encoding per item batch
        std::vector<int> idx, off{0};
        std::vector<double> val;
        sl.batches.clear();
        for (int cb = 0; cb < sv->n_vb; cb++) {
            bool any = false;
            for (int j : it)
                if (j / sv->B == cb && sv->lr != 0.0) {
                    for (int x = 0; x < sv->k; x++) {
                        idx.push_back((j % sv->B) * sv->w + x);
                        val.push_back(sv->lr);
                    }
                    any = true;
                }
            for (int j : it) any = any || j / sv->B == cb;
            if (any) sl.batches.push_back(cb);
            off.push_back((int)idx.size());
        }
        c.arena.reset(s);
        encode_many_device(c, idx, val, off, sl.mask, s);
        sl.used = true;
        sl.done = false;
        sl.id = id;
        sl.step = 0;
        sl.level = c.L;
        sl.nnz = nnz;
    });
}

int fhe_serve_tick(fhe_server* sv, void* stream) {
    if (!sv) return FHE_ERR_INVALID_ARG;
    Ctx& c = *sv->c;
    int inflight = 0;
    int rc = guarded(&c, [&] {
        cudaStream_t s = (cudaStream_t)stream;
        c.arena.reset(s);
        std::map<int, std::vector<Slot*>> fold, pred;  // by level
        for (Slot& sl : sv->slots) {
            if (!sl.used || sl.done) continue;
            if (sl.step < sv->steps) fold[sl.level].push_back(&sl);
            else pred[sl.level].push_back(&sl);
        }
        sv->finishing.clear();
        for (auto& kv : fold) fold_in_step(*sv, kv.second, kv.first, s);
        for (auto& kv : pred) predict_pass(*sv, kv.second, kv.first, s);
        if (!sv->finishing.empty()) {
            // no host wait: the tick's completions are reported by poll() once this event completes
            cudaEvent_t ev;
            if (sv->ev_pool.empty()) {
                CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            } else {
                ev = sv->ev_pool.back();
                sv->ev_pool.pop_back();
            }
            CK(cudaEventRecord(ev, s));
            sv->done_q.push_back({ev, sv->finishing});
            sv->finishing.clear();
        }
        for (Slot& sl : sv->slots) inflight += sl.used && !sl.done;
    });
    return rc ? rc : inflight;
}

int fhe_serve_poll(fhe_server* sv, int64_t* ids, int32_t cap) {
    if (!sv || (cap > 0 && !ids)) return FHE_ERR_INVALID_ARG;
    Ctx& c = *sv->c;
    int n = 0;
    int rc = guarded(&c, [&] {
        // ticks complete in order: report the requests of every completed tick at the front
        while (!sv->done_q.empty()) {
            fhe_server::Done& d = sv->done_q.front();
            if (n + (int)d.ids.size() > cap) break;
            const cudaError_t q = cudaEventQuery(d.ev);
            if (q == cudaErrorNotReady) break;
            CK(q);
            for (long long id : d.ids) ids[n++] = id;
            sv->ev_pool.push_back(d.ev);
            sv->done_q.erase(sv->done_q.begin());
        }
    });
    return rc ? rc : n;
}

int fhe_serve_encrypt_request(fhe_ctx* ctx, int32_t m, int32_t k, const double* u0, const int32_t* items,
                              const double* ratings, int32_t nnz, uint64_t nonce_base, uint64_t* UR, uint64_t* R,
                              void* stream) {
    if (!ctx) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    return guarded(&c, [&] {
        if (m < 1 || k < 1 || !u0 || !UR || !R || nnz < 0 || (nnz > 0 && (!items || !ratings)))
            fail(FHE_ERR_INVALID_ARG, "bad request arguments");
        const int kp = npow2(k), w = 2 * kp;
        if (w > c.slots) fail(FHE_ERR_INVALID_ARG, "rank too large for the ring");
        const int B = c.slots / w, n_vb = (m + B - 1) / B;
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<int> idx, off{0};
        std::vector<double> val;
        for (int a = 0; a < B; a++)
            for (int half = 0; half < 2; half++)
                for (int x = 0; x < k; x++)
                    if (u0[x] != 0.0) {
                        idx.push_back(a * w + half * kp + x);
                        val.push_back(u0[x]);
                    }
        off.push_back((int)idx.size());
        std::vector<std::pair<int, double>> sorted;
        for (int t = 0; t < nnz; t++) {
            if (items[t] < 0 || items[t] >= m) fail(FHE_ERR_INVALID_ARG, "item index out of range");
            sorted.push_back({items[t], ratings[t]});
        }
        std::sort(sorted.begin(), sorted.end());
        for (int cb = 0; cb < n_vb; cb++) {
            for (auto& pr : sorted)
                if (pr.first / B == cb && pr.second != 0.0)
                    for (int x = 0; x < k; x++) {
                        idx.push_back((pr.first % B) * w + x);
                        val.push_back(pr.second);
                    }
            off.push_back((int)idx.size());
        }
        c.arena.reset(s);
        i64* m_dev = (i64*)c.scratch_bytes("req_m", sizeof(i64) * (size_t)(1 + n_vb) * c.n);
        encode_many_device(c, idx, val, off, m_dev, s);
        encrypt_coeffs_device(c, m_dev, c.n, 1, c.L, {nonce_base}, UR, s);
        std::vector<u64> nonces;
        for (int cb = 0; cb < n_vb; cb++) nonces.push_back(nonce_base + 1 + (u64)cb);
        encrypt_coeffs_device(c, m_dev + c.n, c.n, n_vb, c.L, nonces, R, s);
    });
}

int fhe_serve_take(fhe_server* sv, int64_t id, uint64_t* out, int32_t* level, void* stream) {
    if (!sv) return FHE_ERR_INVALID_ARG;
    Ctx& c = *sv->c;
    return guarded(&c, [&] {
        if (!out) fail(FHE_ERR_INVALID_ARG, "null output");
        for (Slot& sl : sv->slots)
            if (sl.used && sl.id == id) {
                if (!sl.done) fail(FHE_ERR_STATE, "request not complete");
                // limbs 0..level of both components of every prediction ciphertext: one 2-D copy
                const size_t pitch = sizeof(u64) * (size_t)(c.L + 1) * c.n;
                CK(cudaMemcpy2DAsync(out, pitch, sl.out, pitch, sizeof(u64) * (size_t)(sl.level + 1) * c.n,
                                     (size_t)2 * sv->n_vb, cudaMemcpyDefault, (cudaStream_t)stream));
                CK(cudaStreamSynchronize((cudaStream_t)stream));
                if (level) *level = sl.level;
                sl.used = false;
                sl.done = false;
                sl.id = -1;
                return;
            }
        fail(FHE_ERR_INVALID_ARG, "unknown request id");
    });
}

}  // extern "C"

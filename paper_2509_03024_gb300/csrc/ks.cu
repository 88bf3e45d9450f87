// ks.cu — fused hybrid key switching (Han-Ki 2020) over a batch of items.
//
// For one polynomial d at level l (l1 = l+1 limbs, evaluation domain) and a key
// of dnum digits of alpha limbs, with ext = Q_l u P (next = l1 + alpha limbs):
//
//   K1  inverse NTT of d (read through the automorphism of the item); the last
//       pass stores y_i = c_i * N^-1 * qhat_i^-1 mod q_i (ModUp's first factor),
//   K2  for every digit j and every target limb x outside D_j: the first pass
//       of a forward NTT loads sum_{i in D_j} y_i * qhat_i mod p_x (fast base
//       conversion, Bajard et al. 2016) and the transform yields ModUp_j(d)_x;
//       the limbs of D_j are d itself and are read from d in K3,
//   K3  acc_h = sum_j ModUp_j(d) * evk_j[h] over ext (key inner product),
//   K4  inverse NTT of the alpha special limbs of acc_h; the last pass stores
//       y_k = c_k * N^-1 * Phat_k^-1 mod p_k,
//   K5  for every limb i < l1: the first pass of a forward NTT loads
//       sum_k y_k * Phat_k mod q_i (Conv_{P->Q}); the last pass stores
//       out_h = (acc_h - conv) * P^-1 + the item's add terms (ModDown).
//
// K1, K2, K4, K5 run the register-blocked NTT tiles of ntt_core.cuh over row
// tables (one descriptor per limb row), so the conversions happen while the
// tiles are loaded and the combinations while they are stored.
//
// The exact rescale uses the same machinery: an inverse transform of the last limb, then forward
// transforms whose load forms the centred last limb modulo each q_i and whose store writes
// (x_i - that) q_l^-1.
//
// Hoisted rotate-and-sum (Halevi-Shoup 2018): S = sum_{r < kp} rot(c, r) runs
// K1 and K2 once on c1, replaces K3 by a kernel that applies each rotation's
// automorphism to the raised digits while it reads them and sums the inner
// products with all kp - 1 rotation keys (and the rotated c0's) into one
// accumulator, then K4 and K5 once. An automorphism maps every aligned run of
// 2^s evaluation slots onto an aligned run of 2^s slots, so the permuted reads
// stay coalesced (pairs of slots are read as one 128-bit load).
#include <algorithm>
#include <cstring>

#include "ks_pass.cuh"

namespace fhe {

const char* const ksp::kKsTileNames[ksp::KS_N_TILES] = {"r16", "r8", "r8x"};

namespace {

using namespace ksp;
using nttc::reduce4;
using nttc::shoup_lazy;

[[maybe_unused]] inline unsigned grid1(size_t work) {
    size_t b = (work + 255) / 256;
    return (unsigned)std::min<size_t>(std::max<size_t>(b, 1), (size_t)1 << 30);
}

}  // namespace

namespace {

// K1-K5 over a batch of items; with hk, K3 is the hoisted inner product (items' galois must be 1,
// addP0 holds c0, d holds c1) and the outputs are sum_r rot(c, r) over r = 0 and hk's rotations.
// With fused_rescale (relinearisation items: galois 1, addI0/addI1 = c0/c1, no addP0), K4/K5
// divide by P q_level instead of P and the outputs are at level - 1:
//   out_h = (acc_h + P c_h - Conv_{P u {q_l} -> Q_{l-1}}(acc_h + P c_h)) (P q_l)^-1.
// Fan-in mode (fi set): K1-K3 per item as for a rotation (d = c1, addP0 = c0, galois of the item);
// instead of K4/K5 the items' accumulators are summed into their group's fi->gacc and their
// permuted c0's into fi->gc0 (the first contribution to a group sets, later ones add), and
// the caller runs one ModDown per group (moddown_run).
struct FanIn {
    const std::vector<int>* group;  // per item: group index, non-decreasing
    u64* gacc;                      // [group][2][next][N]
    u64* gc0;                       // [group][level + 1][N]
    std::vector<char>* touched;     // per group: already holds a contribution
};

// One fan-in accumulation row: dst (+)= sum over its sources of src[perm(k)] mod the row's prime.
struct FanRow {
    u64* dst;
    int first, cnt, prime, set;
};
struct FanSrc {
    const u64* src;
    int galois;
};

__global__ void fanin_sum_kernel(const FanRow* __restrict__ rows, const FanSrc* __restrict__ srcs, int n_rows,
                                 int log_n, const Prime* __restrict__ pr) {
    const size_t total = (size_t)n_rows << log_n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const FanRow r = rows[e >> log_n];
        const int k = (int)(e & (((size_t)1 << log_n) - 1));
        const u64 q = pr[r.prime].q;
        u64 t = r.set ? 0 : r.dst[k];
        for (int j = 0; j < r.cnt; j++) {
            const FanSrc x = srcs[r.first + j];
            t = add_mod(t, x.src[x.galois == 1 ? k : auto_src(k, x.galois, log_n)], q);
        }
        r.dst[k] = t;
    }
}

void moddown_run(Ctx& c, const std::vector<KsItem>& it, const KsItem* d_items, const u64* acc, int level,
                 cudaStream_t s);

void ks_run(Ctx& c, const std::vector<KsItem>& all, int level, const HoistKeys* hk, cudaStream_t s,
            bool fused_rescale = false, const std::vector<int>* fanout_src = nullptr, const FanIn* fi = nullptr) {
    if (all.empty()) return;
    const int n = c.n, L = c.L, A = c.alpha, l1 = level + 1, next = l1 + A, dn = c.dnum(level);
    const int SP = fused_rescale ? A + 1 : A;  // ModDown source limbs
    const bool fan = fanout_src != nullptr;
    // bound the work area to ~6 GiB per sub-batch (per source: y and the raised digits; per item the rest)
    const size_t per_src = (size_t)(l1 + dn * next) * n * sizeof(u64);
    const size_t per_item =
        (size_t)(2 * next + (fi ? 0 : 2 * SP + 2 * l1) + (hk ? l1 : 0)) * n * sizeof(u64);
    const size_t budget = (size_t)6 << 30;
    for (size_t b0 = 0; b0 < all.size();) {
        // items [b0, b0 + items): a fan-out sub-batch ends where a new source would exceed the budget
        int items = 0, n_src = 0;
        size_t used = 0;
        while (b0 + items < all.size()) {
            const bool new_src = !fan || items == 0 || (*fanout_src)[b0 + items] != (*fanout_src)[b0 + items - 1];
            const size_t need = per_item + (new_src ? per_src : 0);
            if (items > 0 && used + need > budget) break;
            used += need;
            n_src += new_src ? 1 : 0;
            items++;
        }
        std::vector<KsItem> it(all.begin() + b0, all.begin() + b0 + items);
        std::vector<int> src_of(items), src_first;
        for (int t = 0; t < items; t++) {
            const bool new_src = !fan || t == 0 || (*fanout_src)[b0 + t] != (*fanout_src)[b0 + t - 1];
            if (new_src) src_first.push_back(t);
            src_of[t] = (int)src_first.size() - 1;
        }
        b0 += items;
        const int n_sources = (int)src_first.size();
        const KsItem* d_items = c.arena.push_vec(it, s);
        const int* d_src_of = fan ? c.arena.push_vec(src_of, s) : nullptr;
        size_t nkeys = 0;
        {
            std::vector<const u64*> ks;
            for (auto& x : it) ks.push_back(x.key);
            std::sort(ks.begin(), ks.end());
            nkeys = std::unique(ks.begin(), ks.end()) - ks.begin();
        }
        u64* y = c.scratch_u64("ks_y", (size_t)n_sources * l1 * n);
        u64* ext = c.scratch_u64("ks_ext", (size_t)n_sources * dn * next * n);
        u64* acc = c.scratch_u64("ks_acc", (size_t)items * 2 * next * n);
        u64* yP = fi ? nullptr : c.scratch_u64("ks_yp", (size_t)items * 2 * SP * n);
        u64* conv = fi ? nullptr : c.scratch_u64("ks_conv", (size_t)items * 2 * l1 * n);
        CombineArgs ca{d_items, acc, c.d_pinv, next, nullptr};
        const CombineArgs none{nullptr, nullptr, nullptr, 0, nullptr};

        // K1: y_i = INTT(perm(d_i)) * qhat_i^-1 (fan-out: once per source, no permutation)
        std::vector<KsRow> r1;
        r1.reserve((size_t)n_sources * l1);
        for (int sx = 0; sx < n_sources; sx++)
            for (int i = 0; i < l1; i++) {
                const KsItem& x0 = it[src_first[sx]];
                KsRow r{};
                r.dst = y + ((size_t)sx * l1 + i) * n;
                r.src = x0.d + (size_t)i * n;
                r.cst = c.d_up_ninv + 2 * ((size_t)level * (L + 1) + i);
                r.prime = i;
                r.galois = fan ? 1 : (int)x0.galois;
                r1.push_back(r);
            }
        const KsRow* d_r1 = c.arena.push_vec(r1, s);
        ks_transform<true, LD_GATHER, ST_SCALE>(c, d_r1, (int)r1.size(), none, K_NTT_INV, 16.0 * r1.size() * n, s);

        // K2: ModUp_j(d)_x for x outside D_j
        std::vector<KsRow> r2;
        r2.reserve((size_t)n_sources * dn * next);
        for (int t = 0; t < n_sources; t++)
            for (int j = 0; j < dn; j++) {
                const int lo = j * A, cnt = std::min(A, l1 - lo);
                for (int x = 0; x < next; x++) {
                    if (x >= lo && x < lo + cnt) continue;
                    const int px = x < l1 ? x : x + (L - level);
                    KsRow r{};
                    r.dst = ext + (((size_t)t * dn + j) * next + x) * n;
                    r.src = y + ((size_t)t * l1 + lo) * n;
                    r.cst = c.d_up_hat + 2 * (((size_t)level * (L + 1) + lo) * c.n_ext + px);
                    r.cst_stride = 2 * c.n_ext;
                    r.src_cnt = cnt;
                    r.prime = px;
                    r.galois = 1;
                    r.pack = c.keys_packed && x < l1;  // raised data limbs stored split at bit 25
                    r2.push_back(r);
                }
            }
        const KsRow* d_r2 = c.arena.push_vec(r2, s);
        ks_transform<false, LD_CONV, ST_LAST>(c, d_r2, (int)r2.size(), none, K_NTT_FWD, 16.0 * r2.size() * n, s);

        // K3: key inner product
        InnerArgs ia{};
        ia.acc = acc;
        ia.ext = ext;
        ia.tab = d_items;
        ia.src_of = d_src_of;
        ia.items = items;
        ia.dn = dn;
        ia.alpha = A;
        ia.next = next;
        ia.level = level;
        ia.L = L;
        ia.n_ext = c.n_ext;
        ia.log_n = c.log_n;
        ia.pr = c.d_primes;
        ia.keys_packed = c.keys_packed;
        if (!hk) {
            LaunchScope _ls(c.prof, K_KS_INNER,
                            8.0 * n * ((double)items * dn * next + (double)nkeys * dn * 2 * next + (double)items * 2 * next),
                            s, 2.0 * items * next * n * dn);
            bool shared = !fan;
            for (int t = 1; t < items && shared; t++)
                shared = it[t].key == it[0].key && it[t].galois == it[0].galois;
            ia.shared_key = shared ? it[0].key : nullptr;
            ia.shared_galois = shared ? it[0].galois : 1;
            launch_ks_inner(ia, fan, c.tune.inner, c.max_data_prime_bits, s);
        } else {
            // reads: the raised digits and c0 once per item, every key once; writes acc and c0sum
            u64* c0sum = c.scratch_u64("ks_c0sum", (size_t)items * l1 * n);
            LaunchScope _ls(c.prof, K_KS_INNER,
                            8.0 * n * ((double)items * (dn * next + l1) + (double)hk->count * dn * 2 * next +
                                       (double)items * (2 * next + l1)),
                            s, 2.0 * items * next * n * dn * hk->count);
            std::vector<HoistStep> hs;
            for (int r = 0; r < hk->count; r++) hs.push_back({hk->key[r], (long long)hk->galois[r]});
            ia.steps = c.arena.push_vec(hs, s);
            ia.n_steps = hk->count;
            ia.c0sum = c0sum;
            launch_ks_hoist_inner(ia, c.tune.hoist, c.max_data_prime_bits, s);
            // the combine adds c0sum to component 0 and c1 to component 1
            std::vector<KsItem> it5(it);
            for (int t = 0; t < items; t++) {
                it5[t].addP0 = nullptr;
                it5[t].addI0 = c0sum + (size_t)t * l1 * n;
                it5[t].addI1 = it[t].d;
            }
            ca.items = c.arena.push_vec(it5, s);
        }

        if (fused_rescale) {
            // K4: y_s = INTT(source s) * N^-1 (M'/m_s)^-1 for m_s = p_0.., p_{alpha-1}, q_l, where the q_l
            // source is acc_h + (P mod q_l) c_h
            std::vector<KsRow> r4;
            for (int t = 0; t < items; t++)
                for (int h = 0; h < 2; h++)
                    for (int sx = 0; sx < SP; sx++) {
                        KsRow r{};
                        r.dst = yP + (((size_t)t * 2 + h) * SP + sx) * n;
                        const bool ql = sx == A;
                        r.src = acc + (((size_t)t * 2 + h) * next + (ql ? level : l1 + sx)) * n;
                        r.src2 = ql ? (h == 0 ? it[t].addI0 : it[t].addI1) + (size_t)level * n : nullptr;
                        r.cst2 = c.d_fd_pq + 2 * (size_t)level;
                        r.cst = c.d_fd_ninv + 2 * ((size_t)level * SP + sx);
                        r.prime = ql ? level : L + 1 + sx;
                        r.galois = 1;
                        r4.push_back(r);
                    }
            const KsRow* d_r4 = c.arena.push_vec(r4, s);
            ks_transform<true, LD_AXPY, ST_SCALE>(c, d_r4, (int)r4.size(), none, K_NTT_INV, 16.0 * r4.size() * n, s);
            // K5: out_h = (acc_h - NTT(Conv(y))) (P q_l)^-1 + c_h q_l^-1 for limbs i < level
            std::vector<KsRow> r5;
            for (int t = 0; t < items; t++)
                for (int h = 0; h < 2; h++)
                    for (int i = 0; i < level; i++) {
                        KsRow r{};
                        r.dst = conv + (((size_t)t * 2 + h) * l1 + i) * n;
                        r.src = yP + ((size_t)t * 2 + h) * SP * n;
                        r.cst = c.d_fd_hat + 2 * ((size_t)level * SP * (L + 1) + i);
                        r.cst_stride = 2 * (L + 1);
                        r.src_cnt = SP;
                        r.prime = i;
                        r.galois = 1;
                        r.item = t;
                        r.half = h;
                        r.limb = i;
                        r5.push_back(r);
                    }
            CombineArgs cr{d_items, acc, c.d_fd_minv + 2 * (size_t)level * (L + 1), next,
                           c.d_resc + 2 * (size_t)level * (L + 1)};
            const KsRow* d_r5 = c.arena.push_vec(r5, s);
            ks_transform<false, LD_CONV, ST_COMBINE_RS>(c, d_r5, (int)r5.size(), cr, K_NTT_FWD, 16.0 * r5.size() * n, s);
            continue;
        }
        if (fi) {
            // sum the sub-batch's accumulators and permuted c0's into their groups
            std::vector<FanRow> fr;
            std::vector<FanSrc> fs;
            for (int t0 = 0; t0 < items;) {
                const int g = (*fi->group)[b0 - items + t0];
                int t1 = t0 + 1;
                while (t1 < items && (*fi->group)[b0 - items + t1] == g) t1++;
                const int set = (*fi->touched)[g] ? 0 : 1;
                (*fi->touched)[g] = 1;
                for (int h = 0; h < 2; h++)
                    for (int x = 0; x < next; x++) {
                        fr.push_back({fi->gacc + (((size_t)g * 2 + h) * next + x) * n, (int)fs.size(), t1 - t0,
                                      x < l1 ? x : x + (L - level), set});
                        for (int t = t0; t < t1; t++) fs.push_back({acc + (((size_t)t * 2 + h) * next + x) * n, 1});
                    }
                for (int i = 0; i < l1; i++) {
                    fr.push_back({fi->gc0 + ((size_t)g * l1 + i) * n, (int)fs.size(), t1 - t0, i, set});
                    for (int t = t0; t < t1; t++) fs.push_back({it[t].addP0 + (size_t)i * n, (int)it[t].galois});
                }
                t0 = t1;
            }
            const FanRow* d_fr = c.arena.push_vec(fr, s);
            const FanSrc* d_fs = c.arena.push_vec(fs, s);
            LaunchScope _ls(c.prof, K_ELEMENTWISE, 8.0 * n * (fs.size() + 2.0 * fr.size()), s);
            const size_t total = fr.size() * (size_t)n;
            fanin_sum_kernel<<<grid1(total), 256, 0, s>>>(d_fr, d_fs, (int)fr.size(), c.log_n, c.d_primes);
            CK(cudaGetLastError());
            continue;
        }
        moddown_run(c, it, ca.items, acc, level, s);
    }
}

// K4/K5 of a plain key switch over the items' accumulators acc ([item][2][next][N]): out_h =
// (acc_h - Conv_{P->Q}(acc_h)) P^-1 + the item's add terms.
void moddown_run(Ctx& c, const std::vector<KsItem>& it, const KsItem* d_items, const u64* acc, int level,
                 cudaStream_t s) {
    const int n = c.n, L = c.L, A = c.alpha, l1 = level + 1, next = l1 + A;
    const int items = (int)it.size();
    u64* yP = c.scratch_u64("ks_yp", (size_t)items * 2 * A * n);
    u64* conv = c.scratch_u64("ks_conv", (size_t)items * 2 * l1 * n);
    const CombineArgs ca{d_items, acc, c.d_pinv, next, nullptr};
    const CombineArgs none{nullptr, nullptr, nullptr, 0, nullptr};
    {
        // K4: y_k = INTT(acc_h special limb k) * Phat_k^-1
        std::vector<KsRow> r4;
        for (int t = 0; t < items; t++)
            for (int h = 0; h < 2; h++)
                for (int kk = 0; kk < A; kk++) {
                    KsRow r{};
                    r.dst = yP + (((size_t)t * 2 + h) * A + kk) * n;
                    r.src = acc + (((size_t)t * 2 + h) * next + l1 + kk) * n;
                    r.cst = c.d_down_ninv + 2 * kk;
                    r.prime = L + 1 + kk;
                    r.galois = 1;
                    r4.push_back(r);
                }
        const KsRow* d_r4 = c.arena.push_vec(r4, s);
        ks_transform<true, LD_GATHER, ST_SCALE>(c, d_r4, (int)r4.size(), none, K_NTT_INV, 16.0 * r4.size() * n, s);

        // K5: out_h = (acc_h - NTT(Conv_{P->Q}(y))) * P^-1 + add terms
        std::vector<KsRow> r5;
        for (int t = 0; t < items; t++)
            for (int h = 0; h < 2; h++)
                for (int i = 0; i < l1; i++) {
                    KsRow r{};
                    r.dst = conv + (((size_t)t * 2 + h) * l1 + i) * n;
                    r.src = yP + ((size_t)t * 2 + h) * A * n;
                    r.cst = c.d_down_hat + 2 * (size_t)i;
                    r.cst_stride = 2 * (L + 1);
                    r.src_cnt = A;
                    r.prime = i;
                    r.galois = 1;
                    r.item = t;
                    r.half = h;
                    r.limb = i;
                    r5.push_back(r);
                }
        const KsRow* d_r5 = c.arena.push_vec(r5, s);
        ks_transform<false, LD_CONV, ST_COMBINE>(c, d_r5, (int)r5.size(), ca, K_NTT_FWD, 16.0 * r5.size() * n, s);
    }
}

}  // namespace

void keyswitch_items(Ctx& c, const std::vector<KsItem>& all, int level, cudaStream_t s) {
    ks_run(c, all, level, nullptr, s);
}

namespace {

// Exact centred rescale of `parts` components per item (level -> level - 1), in two transforms:
// the inverse NTT of the last limb (scaled by N^-1), then for every limb i < level a forward NTT
// whose load forms [x_level]_centred mod q_i and whose store writes (x_i - that) q_level^-1.
// out may equal in.
// in_t (component p, limb i) is in[t] + p pw + i N; with pt[t] set, the rescaled value is that of
// in (.) pt (pt: one polynomial, limb stride N, shared by both components).
void rescale_run(Ctx& c, const std::vector<const u64*>& in, const std::vector<const u64*>& pt,
                 const std::vector<u64*>& out, int parts, int level, cudaStream_t s) {
    const int n = c.n, L = c.L;
    const size_t pw = (size_t)(L + 1) * n;
    const int max_items = (int)std::max<size_t>(1, ((size_t)2 << 30) / ((size_t)parts * (1 + level) * n * sizeof(u64)));
    const CombineArgs none{nullptr, nullptr, nullptr, 0, nullptr};
    const bool prod = !pt.empty();
    for (size_t b0 = 0; b0 < in.size(); b0 += max_items) {
        const int items = (int)std::min<size_t>(max_items, in.size() - b0);
        const int rows = items * parts;
        u64* last = c.scratch_u64("resc_last", (size_t)rows * n);
        u64* work = c.scratch_u64("resc_work", (size_t)rows * level * n);
        std::vector<KsRow> ra, rb;
        for (int t = 0; t < items; t++)
            for (int p = 0; p < parts; p++) {
                const u64* x = in[b0 + t] + (size_t)p * pw;
                KsRow r{};
                r.dst = last + ((size_t)t * parts + p) * n;
                r.src = x + (size_t)level * n;
                r.src2 = prod ? pt[b0 + t] + (size_t)level * n : nullptr;
                r.cst = c.d_ninv + 2 * (size_t)level;
                r.prime = level;
                r.galois = 1;
                ra.push_back(r);
                for (int i = 0; i < level; i++) {
                    KsRow q{};
                    q.dst = work + (((size_t)t * parts + p) * level + i) * n;
                    q.src = r.dst;
                    q.prime = i;
                    q.limb = level;
                    q.galois = 1;
                    q.src2 = x + (size_t)i * n;
                    q.src3 = prod ? pt[b0 + t] + (size_t)i * n : nullptr;
                    q.cst2 = c.d_resc + 2 * ((size_t)level * (L + 1) + i);
                    q.out2 = out[b0 + t] + (size_t)p * pw + (size_t)i * n;
                    rb.push_back(q);
                }
            }
        const KsRow* d_ra = c.arena.push_vec(ra, s);
        if (prod)
            ks_transform<true, LD_MUL, ST_SCALE>(c, d_ra, (int)ra.size(), none, K_NTT_INV, 16.0 * ra.size() * n, s);
        else
            ks_transform<true, LD_GATHER, ST_SCALE>(c, d_ra, (int)ra.size(), none, K_NTT_INV, 16.0 * ra.size() * n, s);
        const KsRow* d_rb = c.arena.push_vec(rb, s);
        ks_transform<false, LD_CENTRED, ST_RESCALE>(c, d_rb, (int)rb.size(), none, K_NTT_FWD, 16.0 * rb.size() * n, s);
    }
}

}  // namespace

void mul_plain_rescale_items(Ctx& c, const std::vector<BinItem>& it, int level, cudaStream_t s) {
    if (level < 1) fail(FHE_ERR_LEVEL_EXHAUSTED, "rescale needs level >= 1");
    if (it.empty()) return;
    std::vector<const u64*> in, pt;
    std::vector<u64*> out;
    for (const BinItem& x : it) {
        in.push_back(x.a);
        pt.push_back(x.b);
        out.push_back(x.out);
    }
    rescale_run(c, in, pt, out, 2, level, s);
}

void items_rescale(Ctx& c, const std::vector<UnItem>& it, int parts, int level, cudaStream_t s) {
    if (level < 1) fail(FHE_ERR_LEVEL_EXHAUSTED, "rescale needs level >= 1");
    if (it.empty()) return;
    std::vector<const u64*> in;
    std::vector<u64*> out;
    for (const UnItem& x : it) {
        in.push_back(x.in);
        out.push_back(x.out);
    }
    rescale_run(c, in, {}, out, parts, level, s);
}


void rotate_fanout_items(Ctx& c, const std::vector<const u64*>& in, const std::vector<u64*>& out,
                         const std::vector<int>& steps, int level, cudaStream_t s) {
    if (in.size() != out.size() || in.size() != steps.size()) fail(FHE_ERR_INVALID_ARG, "fan-out: list sizes differ");
    if (in.empty()) return;
    const size_t lw = c.ct_words() / 2;
    std::vector<size_t> ord(in.size());
    for (size_t i = 0; i < ord.size(); i++) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return in[a] < in[b]; });
    std::vector<KsItem> ks;
    std::vector<int> src;
    for (size_t k = 0; k < ord.size(); k++) {
        const size_t i = ord[k];
        const int g = (int)c.galois(steps[i]);
        if (g == 1) fail(FHE_ERR_INVALID_ARG, "fan-out rotation by a multiple of the slot count");
        const EvalKey& key = rotation_key(c, steps[i]);
        ks.push_back({in[i] + lw, key.d, in[i], nullptr, nullptr, out[i], out[i] + lw, g});
        src.push_back(k == 0 || in[i] != in[ord[k - 1]] ? (int)k : src.back());
    }
    ks_run(c, ks, level, nullptr, s, false, &src);
}

void rotate_fanin_items(Ctx& c, const std::vector<u64*>& acc, const std::vector<int>& first,
                        const std::vector<const u64*>& in, const std::vector<int>& steps, int level, cudaStream_t s) {
    if (first.size() != acc.size() + 1 || in.size() != steps.size() || first.back() != (int)in.size() ||
        first.front() != 0)
        fail(FHE_ERR_INVALID_ARG, "fan-in: group offsets do not cover the inputs");
    const int n = c.n, l1 = level + 1, next = l1 + c.alpha;
    const size_t lw = c.ct_words() / 2;
    // groups with children, in chunks whose group accumulators stay within ~2 GiB
    std::vector<int> gs;
    for (size_t g = 0; g < acc.size(); g++) {
        if (first[g + 1] < first[g]) fail(FHE_ERR_INVALID_ARG, "fan-in: group offsets decrease");
        if (first[g + 1] > first[g]) gs.push_back((int)g);
    }
    const size_t per_group = (size_t)(2 * next + l1) * n * sizeof(u64);
    const size_t chunk = std::max<size_t>(1, ((size_t)2 << 30) / per_group);
    for (size_t g0 = 0; g0 < gs.size(); g0 += chunk) {
        const int groups = (int)std::min(chunk, gs.size() - g0);
        u64* gacc = c.scratch_u64("ks_gacc", (size_t)groups * 2 * next * n);
        u64* gc0 = c.scratch_u64("ks_gc0", (size_t)groups * l1 * n);
        std::vector<KsItem> ks;
        std::vector<int> grp;
        for (int g = 0; g < groups; g++)
            for (int i = first[gs[g0 + g]]; i < first[gs[g0 + g] + 1]; i++) {
                const int gal = (int)c.galois(steps[i]);
                if (gal == 1) fail(FHE_ERR_INVALID_ARG, "fan-in rotation by a multiple of the slot count");
                const EvalKey& key = rotation_key(c, steps[i]);
                ks.push_back({in[i] + lw, key.d, in[i], nullptr, nullptr, nullptr, nullptr, gal});
                grp.push_back(g);
            }
        std::vector<char> touched(groups, 0);
        const FanIn fi{&grp, gacc, gc0, &touched};
        ks_run(c, ks, level, nullptr, s, false, nullptr, &fi);
        // one ModDown per group: acc_g + (gacc_g - Conv(gacc_g)) P^-1 + (gc0_g, 0)
        std::vector<KsItem> gi;
        for (int g = 0; g < groups; g++) {
            u64* a = acc[gs[g0 + g]];
            gi.push_back({nullptr, nullptr, gc0 + (size_t)g * l1 * n, a, a + lw, a, a + lw, 1});
        }
        moddown_run(c, gi, c.arena.push_vec(gi, s), gacc, level, s);
    }
}

void relin_rescale_items(Ctx& c, const std::vector<u64*>& t3, const std::vector<u64*>& out, int level,
                         cudaStream_t s) {
    if (t3.size() != out.size()) fail(FHE_ERR_INVALID_ARG, "relin_rescale: input and output counts differ");
    if (t3.empty()) return;
    if (level < 1) fail(FHE_ERR_LEVEL_EXHAUSTED, "relinearise-rescale needs level >= 1");
    const size_t lw = c.ct_words() / 2;
    std::vector<KsItem> ks;
    for (size_t i = 0; i < t3.size(); i++)
        ks.push_back({t3[i] + 2 * lw, c.rlk.d, nullptr, t3[i], t3[i] + lw, out[i], out[i] + lw, 1});
    ks_run(c, ks, level, nullptr, s, true);
}

std::vector<int> rotsum_steps(int kp) {
    std::vector<int> st;
    if (kp >= 2 && kp <= kHoistMaxKp)
        for (int r = 1; r < kp; r++) st.push_back(r);
    else
        for (int t = 0; (1 << t) < kp; t++) st.push_back(1 << t);
    return st;
}

void hoisted_sum_items(Ctx& c, const std::vector<u64*>& in, const std::vector<u64*>& out,
                       const std::vector<int>& steps, int level, cudaStream_t s) {
    if (in.size() != out.size()) fail(FHE_ERR_INVALID_ARG, "hoisted rotate-and-sum: input and output counts differ");
    if (in.empty()) return;
    const size_t lw = c.ct_words() / 2;
    HoistKeys hk{};
    for (int st : steps) {
        if (c.galois(st) == 1) continue;  // the identity term is always included
        if (hk.count == kMaxHoist) fail(FHE_ERR_INVALID_ARG, "hoisted rotate-and-sum: too many steps");
        hk.key[hk.count] = rotation_key(c, st).d;
        hk.galois[hk.count] = (int)c.galois(st);
        hk.count++;
    }
    if (hk.count == 0) {
        std::vector<UnItem> cp;
        for (size_t i = 0; i < in.size(); i++)
            if (in[i] != out[i]) cp.push_back({in[i], out[i]});
        items_copy(c, cp, 2, level + 1, s);
        return;
    }
    // the 128-bit sums hold count * dnum products below 2^(2 max_bits)
    int terms = hk.count * c.dnum(level), lg = 0;
    while ((1 << lg) < terms) lg++;
    if (2 * c.max_prime_bits + lg > 128) fail(FHE_ERR_INVALID_ARG, "hoisted rotate-and-sum: primes too wide for 128-bit sums");
    std::vector<KsItem> ks;
    for (size_t i = 0; i < in.size(); i++) ks.push_back({in[i] + lw, nullptr, in[i], nullptr, nullptr, out[i], out[i] + lw, 1});
    ks_run(c, ks, level, &hk, s);
}

void rotsum_items(Ctx& c, const std::vector<u64*>& in, const std::vector<u64*>& out, int kp, int level,
                  cudaStream_t s) {
    if (in.size() != out.size()) fail(FHE_ERR_INVALID_ARG, "rotate-and-sum: input and output counts differ");
    if (in.empty() || kp < 1) return;
    const size_t lw = c.ct_words() / 2;
    const int l1 = level + 1;
    if (kp == 1) {
        std::vector<UnItem> cp;
        for (size_t i = 0; i < in.size(); i++)
            if (in[i] != out[i]) cp.push_back({in[i], out[i]});
        items_copy(c, cp, 2, l1, s);
        return;
    }
    if (kp <= kHoistMaxKp) {
        HoistKeys hk{};
        hk.count = kp - 1;
        int max_bits = 0;
        for (int i = 0; i <= c.L + c.alpha; i++) max_bits = std::max(max_bits, (int)c.hprimes[i].b);
        // the 128-bit sums hold count * dnum products below 2^(2 max_bits)
        int terms = hk.count * c.dnum(level), lg = 0;
        while ((1 << lg) < terms) lg++;
        if (2 * max_bits + lg > 128) fail(FHE_ERR_INVALID_ARG, "hoisted rotate-and-sum: primes too wide for 128-bit sums");
        for (int r = 1; r < kp; r++) {
            hk.key[r - 1] = rotation_key(c, r).d;
            hk.galois[r - 1] = (int)c.galois(r);
        }
        std::vector<KsItem> ks;
        for (size_t i = 0; i < in.size(); i++) ks.push_back({in[i] + lw, nullptr, in[i], nullptr, nullptr, out[i], out[i] + lw, 1});
        ks_run(c, ks, level, &hk, s);
        return;
    }
    // wider blocks: log2(kp) rotate-and-adds, alternating between `in` (overwritten) and `out`
    for (size_t i = 0; i < in.size(); i++)
        if (in[i] == out[i]) fail(FHE_ERR_INVALID_ARG, "rotate-and-sum over more than 16 slots needs distinct buffers");
    int rounds = 0;
    while ((1 << rounds) < kp) rounds++;
    std::vector<u64*> cur(in), nxt(out);
    for (int t = 0; t < rounds; t++) {
        std::vector<KsItem> ks;
        const EvalKey& key = rotation_key(c, 1 << t);
        const int g = (int)c.galois(1 << t);
        for (size_t i = 0; i < in.size(); i++)
            ks.push_back({cur[i] + lw, key.d, cur[i], cur[i], cur[i] + lw, nxt[i], nxt[i] + lw, g});
        ks_run(c, ks, level, nullptr, s);
        std::swap(cur, nxt);
    }
    std::vector<UnItem> cp;
    for (size_t i = 0; i < in.size(); i++)
        if (cur[i] != out[i]) cp.push_back({cur[i], out[i]});
    items_copy(c, cp, 2, l1, s);
}

}  // namespace fhe

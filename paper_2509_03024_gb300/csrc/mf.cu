// mf.cu — encrypted CSR matrix factorisation on RNS-CKKS (arXiv 2509.03024,
// Alg. 1 and Alg. 2): CSR packing into batch-pair groups, the encrypted SGD
// epoch, factor encryption / decryption and the encrypted prediction row.
//
// Layout. Users and items are cut into batches of B = (N/2) / w entities,
// w = 2 kp, kp = next_pow2(k). Entity a of a batch owns slots [a w, a w + w)
// and holds its k-vector twice (at a w and at a w + kp), so that a
// rotate-and-sum over kp slots leaves the full inner product in the first kp
// slots of every block. A rating (i, j) with a = i mod B, b = i div B,
// d = j mod B, c = j div B belongs to group (b, c, delta = (d - a) mod B): the
// paper's batch pair (b, c) of Alg. 2 / Fig. 5, split by diagonal so that one
// rotation of item batch c by delta*w lines up all of the group's pairs.
//
// Epoch at level l (two levels per epoch, the accumulators of Alg. 2 applied
// once per epoch):
//   Vr[c][delta] = rot(Vr[c][parent], step w)  (baby-step giant-step delta tree, tree_parent below)
//   per group: P = rescale(relin(UD_b (x) Vr)); S = rotsum_kp(P); E = R_g - S;
//              M = rescale(Vr (.) mask_g); MU = rescale(UD_b (.) mask_g);
//              TU_b += E (x) M;  TV[c][delta] += E (x) MU
//   AccU_b = rescale(relin(TU_b)); G[c][delta] = rescale(relin(TV[c][delta]))
//   AccV_c = sum_delta rot(G[c][delta], -delta w) along the same tree (children first)
//   U_b <- drop(rescale(UD_b (.) reg_b)) + AccU_b + rot(AccU_b, -kp)   (items alike)
// mask_g holds the learning rate on the first k slots of each rated block;
// reg holds 1 - lr * lambda * nnz on every slot of an entity's block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "core.cuh"

using namespace fhe;

namespace {

constexpr u64 kRNonce = (u64)1 << 40;
constexpr u64 kUNonce = (u64)1 << 41;
constexpr u64 kVNonce = ((u64)1 << 41) + ((u64)1 << 40);

int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}
int hbit(int x) { return 31 - __builtin_clz((unsigned)x); }
int popc(int x) { return __builtin_popcount((unsigned)x); }

// Delta tree in baby-step giant-step form (the Vr chain of Alg. 2's rotated item batches): with
// beta = 2^floor(log2(B) / 2) write d = g beta + r (r < beta); a baby (r > 0) hangs off its giant
// g beta, one rotation by r w away; a giant g beta (g > 0) hangs off (g - 2^hb(g)) beta, one
// rotation by 2^hb(g) beta w away. The rotations out of one parent share its ModUp (hoisted
// fan-out), so a full tree needs about 3 B / (2 beta) ModUps per item batch instead of B / 2.
int baby_range(int B) { return 1 << (hbit(B) / 2); }
// parent of d > 0; *step receives the rotation from the parent in blocks
int tree_parent(int d, int beta, int* step) {
    const int g = d / beta, r = d % beta;
    if (r) {
        *step = r;
        return g * beta;
    }
    const int h = 1 << hbit(g);
    *step = h * beta;
    return (g - h) * beta;
}
int tree_depth(int d, int beta) { return popc(d / beta) + (d % beta ? 1 : 0); }
// rotation amounts (in blocks) of the tree: the baby steps 1..beta-1 and the giant steps 2^t beta < B
std::vector<int> tree_steps(int B) {
    const int beta = baby_range(B);
    std::vector<int> st;
    for (int r = 1; r < std::min(beta, B); r++) st.push_back(r);
    for (int t = beta; t < B; t <<= 1) st.push_back(t);
    return st;
}

struct Group {
    int b, c, delta;
    std::vector<int> a;
    std::vector<double> r;
};

}  // namespace

struct fhe_mf_plan {
    Ctx* c = nullptr;
    int n = 0, m = 0, k = 0, kp = 0, w = 0, B = 0, n_ub = 0, n_vb = 0, beta = 0, log_kp = 0;
    long long M = 0;
    std::vector<Group> groups;
    std::vector<std::vector<int>> closure;  // per item batch: sorted delta-tree nodes
    std::vector<int> node_c, node_delta;    // global node list
    std::vector<int> node_of;               // [n_vb * B] -> node id or -1
    std::vector<int> group_node;            // node of each group
    std::vector<int> nnz_u, nnz_v;
    std::vector<int> bin_of;                // rating bin of each group
    std::vector<int> bin_b;                 // user batch of each bin
    std::vector<int> order;                 // groups in (c, b, delta) order: the execution order
    std::vector<int> c_first_pos;           // [n_vb + 1] first position in `order` of each item batch
    std::vector<int> c_first_node;          // [n_vb + 1] first node of each item batch (nodes are by c)
    std::vector<int> wave_c;                // item-batch boundaries of the node-workspace waves
    int wave_nodes = 0;                     // nodes of the largest wave
    size_t wave_budget = (size_t)72 << 30;  // node workspace budget per wave (bytes)
    u64* d_R = nullptr;                     // [bins][L][N] c0 of the rating bins at level L - 1 (c1 is regenerated)
    // plaintext caches (learning-rate dependent)
    bool have_plain = false;
    double lr_c = 0, lam_c = 0;
    i64* d_mask = nullptr;                  // [G][N], in execution order
    u64* d_mask_eval = nullptr;             // [G][L+1][N] the masks in evaluation form, when they fit
    size_t mask_cache_budget = (size_t)16 << 30;
    i64* d_reg = nullptr;                   // [n_ub + n_vb][N]
    // epoch workspace
    u64* d_Vr = nullptr;                    // [wave nodes] ciphertexts
    u64* d_TV = nullptr;                    // [wave nodes] 3-component
    u64* d_TU = nullptr;                    // [n_ub] 3-component
    u64* d_H = nullptr;                     // [wave nodes]
    u64* d_chunk = nullptr;                 // chunk buffers
    u64* d_fin = nullptr;                   // [n_ub + n_vb] x 3 ciphertexts for the final step
    int chunk = 0;        // groups per launch set
    int chunk_alloc = 0;  // groups the chunk area was sized for
    size_t bytes = 0;

    int node(int cb, int delta) const { return node_of[(size_t)cb * B + delta]; }
    ~fhe_mf_plan() {
        void* bufs[] = {d_R, d_mask, d_mask_eval, d_reg, d_Vr, d_TV, d_TU, d_H, d_chunk, d_fin};
        for (void* p : bufs)
            if (p) cudaFree(p);
    }
};

namespace {

template <typename T>
T* plan_alloc(fhe_mf_plan& p, size_t count) {
    void* ptr = nullptr;
    CK(cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T)));
    p.bytes += count * sizeof(T);
    return (T*)ptr;
}

void ensure_plaintexts(fhe_mf_plan& p, double lr, double lam, cudaStream_t s) {
    if (p.have_plain && p.lr_c == lr && p.lam_c == lam) return;
    Ctx& c = *p.c;
    const int G = (int)p.groups.size();
    if (!p.d_mask) p.d_mask = plan_alloc<i64>(p, (size_t)std::max(G, 1) * c.n);
    if (!p.d_reg) p.d_reg = plan_alloc<i64>(p, (size_t)(p.n_ub + p.n_vb) * c.n);
    std::vector<int> idx, off{0};
    std::vector<double> val;
    const int enc_chunk = 4096;
    for (int g0 = 0; g0 < G; g0 += enc_chunk) {
        int g1 = std::min(G, g0 + enc_chunk);
        idx.clear();
        val.clear();
        off.assign(1, 0);
        for (int pos = g0; pos < g1; pos++) {
            if (lr != 0.0)
                for (int a : p.groups[p.order[pos]].a)
                    for (int x = 0; x < p.k; x++) {
                        idx.push_back(a * p.w + x);
                        val.push_back(lr);
                    }
            off.push_back((int)idx.size());
        }
        encode_many_device(c, idx, val, off, p.d_mask + (size_t)g0 * c.n, s);
    }
    idx.clear();
    val.clear();
    off.assign(1, 0);
    for (int side = 0; side < 2; side++) {
        const int nb = side ? p.n_vb : p.n_ub;
        const std::vector<int>& nnz = side ? p.nnz_v : p.nnz_u;
        for (int b = 0; b < nb; b++) {
            for (int a = 0; a < p.B; a++) {
                int e = b * p.B + a;
                int cnt = e < (int)nnz.size() ? nnz[e] : 0;
                double v = 1.0 - lr * lam * cnt;
                if (v != 0.0)
                    for (int x = 0; x < p.w; x++) {
                        idx.push_back(a * p.w + x);
                        val.push_back(v);
                    }
            }
            off.push_back((int)idx.size());
        }
    }
    encode_many_device(c, idx, val, off, p.d_reg, s);
    // masks in evaluation form at every limb, reused by every epoch (each reads its first l+1 limbs)
    const size_t lw = (size_t)(c.L + 1) * c.n;
    if ((size_t)G * lw * sizeof(u64) <= p.mask_cache_budget) {
        if (!p.d_mask_eval) p.d_mask_eval = plan_alloc<u64>(p, (size_t)std::max(G, 1) * lw);
        for (int g0 = 0; g0 < G; g0 += 256)
            materialize_plain(c, p.d_mask + (size_t)g0 * c.n, c.n, std::min(256, G - g0), c.L + 1,
                              p.d_mask_eval + (size_t)g0 * lw, lw, s);
    }
    p.have_plain = true;
    p.lr_c = lr;
    p.lam_c = lam;
}

// Item batches in consecutive waves whose delta-tree node workspace (Vr, H, TV) fits wave_budget
// (a wave holds at least one item batch).
void plan_waves(fhe_mf_plan& p) {
    const size_t node_bytes = (size_t)7 * (p.c->ct_words() / 2) * sizeof(u64);  // Vr, H (2 lw each), TV (3 lw)
    p.wave_c.assign(1, 0);
    p.wave_nodes = 0;
    int nodes_in = 0;
    for (int cb = 0; cb < p.n_vb; cb++) {
        const int nc = p.c_first_node[cb + 1] - p.c_first_node[cb];
        if (nodes_in > 0 && (size_t)(nodes_in + nc) * node_bytes > p.wave_budget) {
            p.wave_c.push_back(cb);
            nodes_in = 0;
        }
        nodes_in += nc;
        p.wave_nodes = std::max(p.wave_nodes, nodes_in);
    }
    p.wave_c.push_back(p.n_vb);
}

void ensure_workspace(fhe_mf_plan& p) {
    Ctx& c = *p.c;
    const size_t w = c.ct_words(), lw = w / 2;
    const size_t nodes = (size_t)p.wave_nodes;
    if (!p.d_Vr) {
        p.d_Vr = plan_alloc<u64>(p, nodes * w);
        p.d_TV = plan_alloc<u64>(p, nodes * 3 * lw);
        p.d_TU = plan_alloc<u64>(p, (size_t)p.n_ub * 3 * lw);
        p.d_H = plan_alloc<u64>(p, nodes * w);
        p.d_fin = plan_alloc<u64>(p, (size_t)(p.n_ub + p.n_vb) * 3 * w);
    }
    if (!p.d_chunk) {
        // chunk: T3 (3 lw) + S, tmp, E, M, MU (2 lw each) + plaintext (lw) = 14 lw per group
        const size_t per_group = 14 * lw * sizeof(u64);
        const size_t budget = (size_t)6 << 30;
        if (p.chunk <= 0)
            p.chunk = (int)std::max<size_t>(1, std::min<size_t>(std::max<size_t>(p.groups.size(), 1),
                                                                budget / per_group));
        // the final steps reuse the chunk area
        const int need = (int)((p.n_ub + p.n_vb + 13) / 14) + 1;
        const int alloc_groups = std::max(p.chunk, need);
        p.d_chunk = plan_alloc<u64>(p, (size_t)alloc_groups * 14 * lw);
        p.chunk_alloc = alloc_groups;
    }
}

void check_plan_keys(const fhe_mf_plan& p) {
    Ctx& c = *p.c;
    if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
    for (int r : rotsum_steps(p.kp)) rotation_key(c, r);
    for (int x : tree_steps(p.B)) {
        rotation_key(c, x * p.w);
        rotation_key(c, -x * p.w);
    }
    rotation_key(c, -p.kp);
}

// Rotation of a list of ciphertexts (left by step_i): out_i = rot(in_i, step_i), optionally
// plus in_i itself (rotate-and-add).
void rotate_items(Ctx& c, const std::vector<const u64*>& in, const std::vector<u64*>& out,
                  const std::vector<int>& steps, int level, bool add_self, cudaStream_t s) {
    const size_t lw = c.ct_words() / 2;
    std::vector<KsItem> ks;
    for (size_t i = 0; i < in.size(); i++) {
        int g = c.galois(steps[i]);
        const EvalKey& key = rotation_key(c, steps[i]);
        ks.push_back({in[i] + lw, key.d, in[i], add_self ? in[i] : nullptr, add_self ? in[i] + lw : nullptr, out[i],
                      out[i] + lw, g});
    }
    keyswitch_items(c, ks, level, s);
}

void run_epoch(fhe_mf_plan& p, u64* U, u64* V, int level, double lr, double lam, cudaStream_t s) {
    Ctx& c = *p.c;
    if (level < 2) fail(FHE_ERR_LEVEL_EXHAUSTED, "an epoch needs level >= 2");
    if (level > c.L) fail(FHE_ERR_INVALID_ARG, "level out of range");
    check_plan_keys(p);
    c.arena.reset(s);
    ensure_plaintexts(p, lr, lam, s);
    ensure_workspace(p);
    c.arena.reset(s);
    const size_t w = c.ct_words(), lw = w / 2;
    const int l0 = level, l1 = level - 1, l2 = level - 2;
    CK(cudaMemsetAsync(p.d_TU, 0, sizeof(u64) * p.n_ub * 3 * lw, s));
    auto UD = [&](int b) { return U + (size_t)b * w; };
    auto VD = [&](int cb) { return V + (size_t)cb * w; };
    u64* AccU = p.d_fin;                                   // [n_ub] ciphertexts
    u64* FU = AccU + (size_t)p.n_ub * w;                   // [n_ub]
    u64* BaseU = FU + (size_t)p.n_ub * w;                  // [n_ub]
    u64* FV = BaseU + (size_t)p.n_ub * w;                  // [n_vb]
    u64* BaseV = FV + (size_t)p.n_vb * w;                  // [n_vb]

    // The item batches run in waves whose delta-tree nodes fit the node workspace; user-side
    // accumulators collect over all waves, each wave finishes its own item batches.
    for (size_t wv = 0; wv + 1 < p.wave_c.size(); wv++) {
        const int cb0 = p.wave_c[wv], cb1 = p.wave_c[wv + 1];
        const int nd0 = p.c_first_node[cb0], nd1 = p.c_first_node[cb1], nodes = nd1 - nd0;
        auto Vr = [&](int nd) { return p.d_Vr + (size_t)(nd - nd0) * w; };
        auto H = [&](int nd) { return p.d_H + (size_t)(nd - nd0) * w; };
        auto TV = [&](int nd) { return p.d_TV + (size_t)(nd - nd0) * 3 * lw; };
        CK(cudaMemsetAsync(p.d_TV, 0, sizeof(u64) * nodes * 3 * lw, s));
        CK(cudaMemsetAsync(p.d_H, 0, sizeof(u64) * nodes * w, s));
        const int baby = baby_range(p.B);
        int maxdepth = 0;
        for (int nd = nd0; nd < nd1; nd++) maxdepth = std::max(maxdepth, tree_depth(p.node_delta[nd], baby));

        // 1. delta trees of the wave's item batches, one launch set per tree depth
        {
            std::vector<UnItem> roots;
            for (int cb = cb0; cb < cb1; cb++) roots.push_back({VD(cb), Vr(p.node(cb, 0))});
            items_copy(c, roots, 2, l0 + 1, s);
            for (int dep = 1; dep <= maxdepth; dep++) {
                std::vector<const u64*> in;
                std::vector<u64*> out;
                std::vector<int> steps;
                for (int nd = nd0; nd < nd1; nd++) {
                    int d = p.node_delta[nd];
                    if (tree_depth(d, baby) != dep) continue;
                    int step = 0;
                    const int par = tree_parent(d, baby, &step);
                    in.push_back(Vr(p.node(p.node_c[nd], par)));
                    out.push_back(Vr(nd));
                    steps.push_back(step * p.w);
                }
                rotate_fanout_items(c, in, out, steps, l0, s);  // siblings share their parent's ModUp
            }
        }

        // 2. the wave's groups, in chunks (positions of the execution order)
        const int C = p.chunk;
        u64* T3 = p.d_chunk;
        u64* Sb = T3 + (size_t)C * 3 * lw;
        u64* Tb = Sb + (size_t)C * w;
        u64* Eb = Tb + (size_t)C * w;
        u64* Mb = Eb + (size_t)C * w;
        u64* MUb = Mb + (size_t)C * w;
        u64* PTb = MUb + (size_t)C * w;
        const int pos_end = p.c_first_pos[cb1];
        for (int g0 = p.c_first_pos[cb0]; g0 < pos_end; g0 += C) {
            const int cnt = std::min(C, pos_end - g0);
            auto gid = [&](int i) { return p.order[g0 + i]; };
            std::vector<BinItem> tens, pm;
            std::vector<u64*> t3s, pout;
            for (int i = 0; i < cnt; i++) {
                const Group& g = p.groups[gid(i)];
                u64* t3 = T3 + (size_t)i * 3 * lw;
                tens.push_back({UD(g.b), Vr(p.group_node[gid(i)]), t3});
                t3s.push_back(t3);
                pout.push_back(Sb + (size_t)i * w);
            }
            items_tensor(c, tens, l0 + 1, s);
            relin_rescale_items(c, t3s, pout, l0, s);
            // rotate-and-sum over kp slots: S (in Tb) from P (in Sb)
            {
                std::vector<u64*> in, out;
                for (int i = 0; i < cnt; i++) {
                    in.push_back(Sb + (size_t)i * w);
                    out.push_back(Tb + (size_t)i * w);
                }
                rotsum_items(c, in, out, p.kp, l1, s);
            }
            // E = R - S: R's c1 regenerated from its seed into E's c1 rows, then transformed
            {
                std::vector<SeedRow> rows;
                for (int i = 0; i < cnt; i++)
                    for (int x = 0; x <= l1; x++)
                        rows.push_back({seeded_key(c, kRNonce + (u64)p.bin_of[gid(i)], x),
                                        Eb + (size_t)i * w + lw + (size_t)x * c.n, x, 0});
                seeded_uniform_device(c, rows, s);
                ntt_forward(c, poly_batch(Eb + lw, w, 0, cnt, 1, 0, l1 + 1), s);
                std::vector<BinItem> e0, e1;
                for (int i = 0; i < cnt; i++) {
                    e0.push_back({p.d_R + (size_t)p.bin_of[gid(i)] * c.L * c.n, Tb + (size_t)i * w, Eb + (size_t)i * w});
                    e1.push_back({Eb + (size_t)i * w + lw, Tb + (size_t)i * w + lw, Eb + (size_t)i * w + lw});
                }
                items_add(c, e0, 1, l1 + 1, true, s);
                items_add(c, e1, 1, l1 + 1, true, s);
            }
            // masks: M = rescale(Vr (.) mask), MU = rescale(UD (.) mask)
            const u64* masks = PTb;
            if (p.d_mask_eval)
                masks = p.d_mask_eval + (size_t)g0 * lw;
            else
                materialize_plain(c, p.d_mask + (size_t)g0 * c.n, c.n, cnt, l0 + 1, PTb, lw, s);
            for (int i = 0; i < cnt; i++) {
                const Group& g = p.groups[gid(i)];
                const u64* pt = masks + (size_t)i * lw;
                pm.push_back({Vr(p.group_node[gid(i)]), pt, Mb + (size_t)i * w});
                pm.push_back({UD(g.b), pt, MUb + (size_t)i * w});
            }
            mul_plain_rescale_items(c, pm, l0, s);
            // accumulate the tensors: TU_b += E (x) M, TV[node] += E (x) MU
            std::map<int, std::vector<int>> by_b, by_node;
            for (int i = 0; i < cnt; i++) {
                by_b[p.groups[gid(i)].b].push_back(i);
                by_node[p.group_node[gid(i)]].push_back(i);
            }
            std::vector<AccTarget> tg;
            std::vector<BinItem> cbi;
            for (auto& kv : by_b) {
                tg.push_back({p.d_TU + (size_t)kv.first * 3 * lw, (int)cbi.size(), (int)kv.second.size()});
                for (int i : kv.second) cbi.push_back({Eb + (size_t)i * w, Mb + (size_t)i * w, nullptr});
            }
            for (auto& kv : by_node) {
                tg.push_back({TV(kv.first), (int)cbi.size(), (int)kv.second.size()});
                for (int i : kv.second) cbi.push_back({Eb + (size_t)i * w, MUb + (size_t)i * w, nullptr});
            }
            items_tensor_acc(c, tg, cbi, l1 + 1, s);
        }

        // 3. relinearise and rescale the wave's item-side accumulators
        {
            std::vector<char> used(nodes, 0);
            for (int pos = p.c_first_pos[cb0]; pos < pos_end; pos++) used[p.group_node[p.order[pos]] - nd0] = 1;
            std::vector<u64*> t3, outs;
            for (int nd = nd0; nd < nd1; nd++)
                if (used[nd - nd0]) {
                    t3.push_back(TV(nd));
                    outs.push_back(H(nd));
                }
            relin_rescale_items(c, t3, outs, l1, s);
        }

        // 4. back-rotation of the item gradients along the delta trees (deepest first): every parent
        //    takes the sum of its children rotated back, with one ModDown
        for (int dep = maxdepth; dep >= 1; dep--) {
            std::map<int, std::vector<std::pair<int, int>>> kids;  // parent node -> (child node, step)
            for (int nd = nd0; nd < nd1; nd++) {
                const int d = p.node_delta[nd];
                if (tree_depth(d, baby) != dep) continue;
                int step = 0;
                const int par = tree_parent(d, baby, &step);
                kids[p.node(p.node_c[nd], par)].push_back({nd, -step * p.w});
            }
            std::vector<u64*> acc;
            std::vector<int> first{0}, steps;
            std::vector<const u64*> in;
            for (auto& kv : kids) {
                acc.push_back(H(kv.first));
                for (auto& ch : kv.second) {
                    in.push_back(H(ch.first));
                    steps.push_back(ch.second);
                }
                first.push_back((int)in.size());
            }
            rotate_fanin_items(c, acc, first, in, steps, l2, s);
        }

        // 5. the wave's item batches: half-fill and apply (V_c is read only by its own wave)
        {
            std::vector<const u64*> in;
            std::vector<u64*> out;
            for (int cb = cb0; cb < cb1; cb++) {
                in.push_back(H(p.node(cb, 0)));
                out.push_back(FV + (size_t)cb * w);
            }
            std::vector<int> steps(in.size(), -p.kp);
            rotate_items(c, in, out, steps, l2, true, s);
            u64* PT = p.d_chunk;
            materialize_plain(c, p.d_reg + (size_t)(p.n_ub + cb0) * c.n, c.n, cb1 - cb0, l0 + 1, PT, lw, s);
            std::vector<BinItem> pm, fin;
            for (int cb = cb0; cb < cb1; cb++) {
                pm.push_back({VD(cb), PT + (size_t)(cb - cb0) * lw, BaseV + (size_t)cb * w});
                fin.push_back({BaseV + (size_t)cb * w, FV + (size_t)cb * w, VD(cb)});
            }
            mul_plain_rescale_items(c, pm, l0, s);
            items_add(c, fin, 2, l2 + 1, false, s);
        }
    }

    // 6. the user side: relinearise-rescale the accumulators, half-fill and apply
    {
        std::vector<u64*> t3, outs;
        for (int b = 0; b < p.n_ub; b++) {
            t3.push_back(p.d_TU + (size_t)b * 3 * lw);
            outs.push_back(AccU + (size_t)b * w);
        }
        relin_rescale_items(c, t3, outs, l1, s);
        std::vector<const u64*> in;
        std::vector<u64*> out;
        for (int b = 0; b < p.n_ub; b++) {
            in.push_back(AccU + (size_t)b * w);
            out.push_back(FU + (size_t)b * w);
        }
        std::vector<int> steps(in.size(), -p.kp);
        rotate_items(c, in, out, steps, l2, true, s);
        u64* PT = p.d_chunk;
        materialize_plain(c, p.d_reg, c.n, p.n_ub, l0 + 1, PT, lw, s);
        std::vector<BinItem> pm, fin;
        for (int b = 0; b < p.n_ub; b++) {
            pm.push_back({UD(b), PT + (size_t)b * lw, BaseU + (size_t)b * w});
            fin.push_back({BaseU + (size_t)b * w, FU + (size_t)b * w, UD(b)});
        }
        mul_plain_rescale_items(c, pm, l0, s);
        items_add(c, fin, 2, l2 + 1, false, s);
    }
}

void run_predict(const fhe_mf_plan& p, const u64* U, const u64* V, int level, int user, u64* out, cudaStream_t s) {
    Ctx& c = *p.c;
    if (level < 2) fail(FHE_ERR_LEVEL_EXHAUSTED, "prediction needs level >= 2");
    if (level > c.L) fail(FHE_ERR_INVALID_ARG, "level out of range");
    if (user < 0 || user >= p.n) fail(FHE_ERR_INVALID_ARG, "user out of range");
    if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
    for (int r : rotsum_steps(p.kp)) rotation_key(c, r);
    for (int t = 0; t < p.beta; t++) rotation_key(c, (1 << t) * p.w);
    c.arena.reset(s);
    const size_t w = c.ct_words(), lw = w / 2;
    const int b = user / p.B, a = user % p.B;
    i64* mcoef = (i64*)c.scratch_bytes("pred_mask", sizeof(i64) * c.n);
    std::vector<std::pair<int, double>> nz;
    for (int x = 0; x < p.k; x++) nz.push_back({a * p.w + x, 1.0});
    encode_sparse_device(c, nz, mcoef, s);
    c.arena.reset(s);
    u64* pt = c.scratch_u64("pred_pt", lw);
    materialize_plain(c, mcoef, c.n, 1, level + 1, pt, lw, s);
    u64* X = c.scratch_u64("pred_x", 2 * w);
    u64* Y = X + w;
    mul_plain_rescale_items(c, {BinItem{U + (size_t)b * w, pt, X}}, level, s);
    for (int t = 0; t < p.beta; t++) {
        rotate_items(c, {X}, {Y}, {(1 << t) * p.w}, level - 1, true, s);
        std::swap(X, Y);
    }
    u64* T3 = c.scratch_u64("pred_t3", (size_t)p.n_vb * 3 * lw);
    u64* tmp = c.scratch_u64("pred_tmp", (size_t)p.n_vb * w);
    std::vector<BinItem> tens;
    std::vector<u64*> t3s, prod, res;
    for (int cb = 0; cb < p.n_vb; cb++) {
        tens.push_back({X, V + (size_t)cb * w, T3 + (size_t)cb * 3 * lw});
        t3s.push_back(T3 + (size_t)cb * 3 * lw);
        prod.push_back(tmp + (size_t)cb * w);
        res.push_back(out + (size_t)cb * w);
    }
    items_tensor(c, tens, level, s);
    relin_rescale_items(c, t3s, prod, level - 1, s);
    rotsum_items(c, prod, res, p.kp, level - 2, s);
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

// CSR checks shared by fhe_csr_pack and fhe_mf_layout (the per-entry checks run while grouping).
void check_csr(int n, int m, int k, const int64_t* row_ptr, const int32_t* col_idx, const double* vals) {
    if (n < 1 || m < 1 || k < 1 || !row_ptr) fail(FHE_ERR_INVALID_ARG, "bad matrix shape");
    const long long M = row_ptr[n];
    if (row_ptr[0] != 0 || M < 0) fail(FHE_ERR_INVALID_ARG, "row_ptr must start at 0");
    if (M > 0 && (!col_idx || !vals)) fail(FHE_ERR_INVALID_ARG, "null CSR arrays");
    for (int i = 0; i < n; i++)
        if (row_ptr[i + 1] < row_ptr[i]) fail(FHE_ERR_INVALID_ARG, "row_ptr must be non-decreasing");
}

// The host-side layout of a plan for a ring of `slots` slots (Alg. 2 batch pairs, Fig. 5): batch
// geometry, groups in (b, c, delta) order, delta-tree nodes, the execution order and item-batch
// boundaries, and the rating bins. Touches no device.
void build_layout(fhe_mf_plan& p, int slots, int n, int m, int k, const int64_t* row_ptr, const int32_t* col_idx,
                  const double* vals) {
    p.n = n;
    p.m = m;
    p.k = k;
    p.kp = next_pow2(k);
    p.w = 2 * p.kp;
    if (p.w > slots) fail(FHE_ERR_INVALID_ARG, "rank too large for the ring");
    p.B = slots / p.w;
    p.beta = hbit(p.B);
    p.log_kp = hbit(p.kp);
    p.n_ub = (n + p.B - 1) / p.B;
    p.n_vb = (m + p.B - 1) / p.B;
    p.M = row_ptr[n];
    p.nnz_u.assign(n, 0);
    p.nnz_v.assign(m, 0);
    std::map<std::tuple<int, int, int>, std::vector<std::pair<int, double>>> gm;
    for (int i = 0; i < n; i++) {
        std::vector<int> cols(col_idx + row_ptr[i], col_idx + row_ptr[i + 1]);
        std::sort(cols.begin(), cols.end());
        for (size_t t = 1; t < cols.size(); t++)
            if (cols[t] == cols[t - 1]) fail(FHE_ERR_INVALID_ARG, "duplicate (user, item) rating");
        for (long long e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            int j = col_idx[e];
            if (j < 0 || j >= m) fail(FHE_ERR_INVALID_ARG, "column index out of range");
            if (!std::isfinite(vals[e])) fail(FHE_ERR_INVALID_ARG, "non-finite rating");
            int a = i % p.B, b = i / p.B, d = j % p.B, cb = j / p.B;
            int delta = ((d - a) % p.B + p.B) % p.B;
            gm[std::make_tuple(b, cb, delta)].push_back({a, vals[e]});
            p.nnz_u[i]++;
            p.nnz_v[j]++;
        }
    }
    for (auto& kv : gm) {
        Group g;
        std::tie(g.b, g.c, g.delta) = kv.first;
        auto v = kv.second;
        std::sort(v.begin(), v.end());
        for (auto& pr : v) {
            g.a.push_back(pr.first);
            g.r.push_back(pr.second);
        }
        p.groups.push_back(std::move(g));
    }
    // delta trees
    p.closure.assign(p.n_vb, {});
    p.node_of.assign((size_t)p.n_vb * p.B, -1);
    for (int cb = 0; cb < p.n_vb; cb++) {
        std::vector<char> in(p.B, 0);
        in[0] = 1;
        for (const Group& g : p.groups)
            if (g.c == cb)
                for (int d = g.delta, st = 0; d && !in[d]; d = tree_parent(d, baby_range(p.B), &st)) in[d] = 1;
        for (int d = 0; d < p.B; d++)
            if (in[d]) {
                p.closure[cb].push_back(d);
                p.node_of[(size_t)cb * p.B + d] = (int)p.node_c.size();
                p.node_c.push_back(cb);
                p.node_delta.push_back(d);
            }
    }
    for (const Group& g : p.groups) p.group_node.push_back(p.node(g.c, g.delta));
    // execution order (c, b, delta), and the first position and first node of each item batch
    {
        const int G0 = (int)p.groups.size();
        p.order.resize(G0);
        for (int gi = 0; gi < G0; gi++) p.order[gi] = gi;
        std::stable_sort(p.order.begin(), p.order.end(),
                         [&](int x, int y) { return p.groups[x].c < p.groups[y].c; });
        p.c_first_pos.assign(p.n_vb + 1, G0);
        for (int pos = G0 - 1; pos >= 0; pos--) p.c_first_pos[p.groups[p.order[pos]].c] = pos;
        for (int cb = p.n_vb - 1; cb >= 0; cb--)
            p.c_first_pos[cb] = std::min(p.c_first_pos[cb], p.c_first_pos[cb + 1]);
        p.c_first_node.assign(p.n_vb + 1, (int)p.node_c.size());
        for (int nd = (int)p.node_c.size() - 1; nd >= 0; nd--) p.c_first_node[p.node_c[nd]] = nd;
    }
    // Rating bins: within each user batch, groups in plan order go to the first bin (in creation
    // order) holding none of their users, else to a new bin; bins are numbered batch by batch.
    const int G = (int)p.groups.size();
    p.bin_of.assign(G, 0);
    {
        const int words = (p.B + 63) / 64;
        std::vector<uint64_t> gbits(words);
        int g = 0;
        for (int b = 0; b < p.n_ub; b++) {
            const int first = (int)p.bin_b.size();
            std::vector<std::vector<uint64_t>> taken;
            for (; g < G && p.groups[g].b == b; g++) {
                std::fill(gbits.begin(), gbits.end(), 0);
                for (int a : p.groups[g].a) gbits[a >> 6] |= 1ull << (a & 63);
                int chosen = -1;
                for (size_t t = 0; t < taken.size() && chosen < 0; t++) {
                    bool clash = false;
                    for (int x = 0; x < words && !clash; x++) clash = (taken[t][x] & gbits[x]) != 0;
                    if (!clash) chosen = (int)t;
                }
                if (chosen < 0) {
                    taken.emplace_back(words, 0);
                    p.bin_b.push_back(b);
                    chosen = (int)taken.size() - 1;
                }
                for (int x = 0; x < words; x++) taken[chosen][x] |= gbits[x];
                p.bin_of[g] = first + chosen;
            }
        }
    }
}

}  // namespace

extern "C" {

int fhe_mf_rotation_steps(const fhe_ctx* ctx, int32_t k, int32_t* out, size_t cap) {
    if (!ctx || k < 1) return FHE_ERR_INVALID_ARG;
    const Ctx& c = ctx->c;
    int kp = next_pow2(k), w = 2 * kp;
    if (w > c.slots) return FHE_ERR_INVALID_ARG;
    int B = c.slots / w;
    std::vector<int> st = rotsum_steps(kp);
    const std::vector<int> tree = tree_steps(B);
    for (int x : tree) st.push_back(x * w);
    for (int x : tree) st.push_back(-x * w);
    st.push_back(-kp);
    if (out) {
        if (cap < st.size()) return FHE_ERR_INVALID_ARG;
        std::copy(st.begin(), st.end(), out);
    }
    return (int)st.size();
}

int fhe_csr_pack(fhe_ctx* ctx, int32_t n, int32_t m, int32_t k, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* vals, fhe_mf_plan** out) {
    if (!ctx || !out) return FHE_ERR_INVALID_ARG;
    *out = nullptr;
    fhe_mf_plan* p = new (std::nothrow) fhe_mf_plan();
    if (!p) return FHE_ERR_OOM;
    Ctx& c = ctx->c;
    int rc = guarded(&c, [&] {
        check_csr(n, m, k, row_ptr, col_idx, vals);
        if (!c.have_keys) fail(FHE_ERR_MISSING_KEY, "keys have not been generated");
        p->c = &c;
        build_layout(*p, c.slots, n, m, k, row_ptr, col_idx, vals);
        plan_waves(*p);
        const int G = (int)p->groups.size();
        // EncryptCsrMatrix: one ciphertext per bin, each group's ratings in the first k slots of their
        // user blocks, encrypted by the key holder with a regenerable c1 (object 2^40 + bin) at level
        // L - 1, the highest level an epoch reads it at; only c0 is stored
        const int NB = (int)p->bin_b.size();
        std::vector<std::vector<std::pair<int, double>>> bin_nz(NB);
        for (int gi = 0; gi < G; gi++) {
            const Group& gr = p->groups[gi];
            for (size_t t = 0; t < gr.a.size(); t++)
                if (gr.r[t] != 0.0)
                    for (int x = 0; x < p->k; x++) bin_nz[p->bin_of[gi]].push_back({gr.a[t] * p->w + x, gr.r[t]});
        }
        if (c.L < 1) fail(FHE_ERR_INVALID_ARG, "the modulus chain needs at least two data primes");
        const size_t rw = (size_t)c.L * c.n;  // c0 at level L - 1
        p->d_R = plan_alloc<u64>(*p, (size_t)std::max(NB, 1) * rw);
        const int chunk = 256;
        i64* m_dev = (i64*)c.scratch_bytes("pack_m", sizeof(i64) * chunk * c.n);
        for (int t0 = 0; t0 < NB; t0 += chunk) {
            int t1 = std::min(NB, t0 + chunk);
            std::vector<int> idx, off{0};
            std::vector<double> val;
            std::vector<u64> nonces;
            for (int t = t0; t < t1; t++) {
                auto& nz = bin_nz[t];
                std::sort(nz.begin(), nz.end());  // ascending slots: the encoding's summation order
                for (auto& e : nz) {
                    idx.push_back(e.first);
                    val.push_back(e.second);
                }
                off.push_back((int)idx.size());
                nonces.push_back(kRNonce + (u64)t);
            }
            c.arena.reset(0);
            encode_many_device(c, idx, val, off, m_dev, 0);
            encrypt_seeded_device(c, m_dev, c.n, t1 - t0, c.L - 1, nonces, p->d_R + (size_t)t0 * rw, 0);
        }
        CK(cudaStreamSynchronize(0));
    });
    if (rc) {
        delete p;
        return rc;
    }
    *out = p;
    return FHE_OK;
}

int fhe_mf_layout(int32_t slots, int32_t n, int32_t m, int32_t k, const int64_t* row_ptr, const int32_t* col_idx,
                  const double* vals, int64_t* counts, int32_t* group_b, int32_t* group_c, int32_t* group_delta,
                  int32_t* group_count, int32_t* bin_of_group, int64_t group_cap, int32_t* node_c,
                  int32_t* node_delta, int64_t node_cap) {
    if (!counts) return FHE_ERR_INVALID_ARG;
    return guarded(nullptr, [&] {
        if (slots < 256 || slots > 32768 || (slots & (slots - 1)))
            fail(FHE_ERR_INVALID_ARG, "slots must be a power of two in [2^8, 2^15]");
        check_csr(n, m, k, row_ptr, col_idx, vals);
        fhe_mf_plan p;  // host fields only: nothing is allocated on a device
        build_layout(p, slots, n, m, k, row_ptr, col_idx, vals);
        const int64_t G = (int64_t)p.groups.size(), NB = (int64_t)p.bin_b.size(), ND = (int64_t)p.node_c.size();
        counts[0] = G;
        counts[1] = NB;
        counts[2] = ND;
        if ((group_b || group_c || group_delta || group_count || bin_of_group) && group_cap < G)
            fail(FHE_ERR_INVALID_ARG, "group arrays shorter than the group count");
        if ((node_c || node_delta) && node_cap < ND) fail(FHE_ERR_INVALID_ARG, "node arrays shorter than the node count");
        for (int64_t g = 0; g < G; g++) {
            if (group_b) group_b[g] = p.groups[g].b;
            if (group_c) group_c[g] = p.groups[g].c;
            if (group_delta) group_delta[g] = p.groups[g].delta;
            if (group_count) group_count[g] = (int32_t)p.groups[g].a.size();
            if (bin_of_group) bin_of_group[g] = p.bin_of[g];
        }
        for (int64_t d = 0; d < ND; d++) {
            if (node_c) node_c[d] = p.node_c[d];
            if (node_delta) node_delta[d] = p.node_delta[d];
        }
    });
}

void fhe_mf_plan_destroy(fhe_mf_plan* p) {
    if (p) {
        if (p->c) cudaSetDevice(p->c->device);
        cudaDeviceSynchronize();
        delete p;
    }
}

int fhe_mf_plan_set_chunk(fhe_mf_plan* p, int32_t groups) {
    if (!p || groups < 1) return FHE_ERR_INVALID_ARG;
    if (p->d_chunk) {
        cudaSetDevice(p->c->device);
        cudaDeviceSynchronize();
        cudaFree(p->d_chunk);
        p->bytes -= (size_t)p->chunk_alloc * 14 * (p->c->ct_words() / 2) * sizeof(u64);
        p->d_chunk = nullptr;
    }
    p->chunk = groups;
    return FHE_OK;
}

int fhe_mf_plan_set_wave_budget(fhe_mf_plan* p, uint64_t bytes) {
    if (!p || bytes == 0) return FHE_ERR_INVALID_ARG;
    if (p->d_Vr) {  // the node workspace is re-sized at the next epoch
        cudaSetDevice(p->c->device);
        cudaDeviceSynchronize();
        const size_t w = p->c->ct_words();
        for (u64** b : {&p->d_Vr, &p->d_TV, &p->d_TU, &p->d_H, &p->d_fin}) {
            cudaFree(*b);
            *b = nullptr;
        }
        p->bytes -= ((size_t)p->wave_nodes * (2 * w + 3 * (w / 2)) + (size_t)p->n_ub * 3 * (w / 2) +
                     (size_t)(p->n_ub + p->n_vb) * 3 * w) * sizeof(u64);
    }
    p->wave_budget = bytes;
    plan_waves(*p);
    return FHE_OK;
}

int fhe_mf_plan_get_info(const fhe_mf_plan* p, fhe_mf_plan_info* out) {
    if (!p || !out) return FHE_ERR_INVALID_ARG;
    out->n_users = p->n;
    out->n_items = p->m;
    out->k = p->k;
    out->kp = p->kp;
    out->w = p->w;
    out->B = p->B;
    out->n_user_batches = p->n_ub;
    out->n_item_batches = p->n_vb;
    out->n_ratings = p->M;
    out->n_groups = (int64_t)p->groups.size();
    out->n_tree_nodes = (int64_t)p->node_c.size();
    out->n_bins = (int64_t)p->bin_b.size();
    out->device_bytes = p->bytes;
    return FHE_OK;
}

int fhe_mf_plan_get_bins(const fhe_mf_plan* p, int32_t* bin_of_group) {
    if (!p || !bin_of_group) return FHE_ERR_INVALID_ARG;
    std::copy(p->bin_of.begin(), p->bin_of.end(), bin_of_group);
    return FHE_OK;
}

int fhe_mf_plan_get_groups(const fhe_mf_plan* p, int32_t* b, int32_t* cc, int32_t* delta, int32_t* count) {
    if (!p) return FHE_ERR_INVALID_ARG;
    for (size_t g = 0; g < p->groups.size(); g++) {
        if (b) b[g] = p->groups[g].b;
        if (cc) cc[g] = p->groups[g].c;
        if (delta) delta[g] = p->groups[g].delta;
        if (count) count[g] = (int32_t)p->groups[g].a.size();
    }
    return FHE_OK;
}

int fhe_mf_encrypt_factors(fhe_ctx* ctx, const fhe_mf_plan* p, int32_t which, const double* X, int32_t count,
                           uint64_t* cts, void* stream) {
    if (!ctx || !p) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    return guarded(&c, [&] {
        if (which != 0 && which != 1) fail(FHE_ERR_INVALID_ARG, "which must be 0 (users) or 1 (items)");
        const int ent = which ? p->m : p->n, nb = which ? p->n_vb : p->n_ub;
        if (count != ent || !X || !cts) fail(FHE_ERR_INVALID_ARG, "factor matrix must have one row per entity");
        cudaStream_t s = (cudaStream_t)stream;
        c.arena.reset(s);
        std::vector<int> idx, off{0};
        std::vector<double> val;
        std::vector<u64> nonces;
        for (int b = 0; b < nb; b++) {
            std::vector<std::pair<int, double>> z;
            for (int a = 0; a < p->B; a++) {
                int e = b * p->B + a;
                if (e >= ent) break;
                for (int x = 0; x < p->k; x++) {
                    z.push_back({a * p->w + x, X[(size_t)e * p->k + x]});
                    z.push_back({a * p->w + p->kp + x, X[(size_t)e * p->k + x]});
                }
            }
            std::sort(z.begin(), z.end());
            for (auto& pr : z)
                if (pr.second != 0.0) {
                    idx.push_back(pr.first);
                    val.push_back(pr.second);
                }
            off.push_back((int)idx.size());
            nonces.push_back((which ? kVNonce : kUNonce) + (u64)b);
        }
        i64* m_dev = (i64*)c.scratch_bytes("fac_m", sizeof(i64) * nb * c.n);
        encode_many_device(c, idx, val, off, m_dev, s);
        encrypt_coeffs_device(c, m_dev, c.n, nb, c.L, nonces, cts, s);
    });
}

int fhe_mf_decrypt_factors(fhe_ctx* ctx, const fhe_mf_plan* p, int32_t which, const uint64_t* cts, int32_t level,
                           double* X, int32_t count, void* stream) {
    if (!ctx || !p) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    return guarded(&c, [&] {
        if (which != 0 && which != 1) fail(FHE_ERR_INVALID_ARG, "which must be 0 (users) or 1 (items)");
        const int ent = which ? p->m : p->n, nb = which ? p->n_vb : p->n_ub;
        if (count != ent || !X || !cts) fail(FHE_ERR_INVALID_ARG, "factor matrix must have one row per entity");
        std::vector<double> z((size_t)p->B * p->w);
        for (int b = 0; b < nb; b++) {
            decrypt_to_slots(c, cts + (size_t)b * c.ct_words(), level, z.data(), z.size(), (cudaStream_t)stream);
            for (int a = 0; a < p->B; a++) {
                int e = b * p->B + a;
                if (e >= ent) break;
                for (int x = 0; x < p->k; x++) X[(size_t)e * p->k + x] = z[(size_t)a * p->w + x];
            }
        }
    });
}

int fhe_mf_sgd_epoch(fhe_ctx* ctx, fhe_mf_plan* p, uint64_t* U, uint64_t* V, int32_t level, double lr, double lam,
                     void* stream) {
    if (!ctx || !p) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    return guarded(&c, [&] {
        if (!U || !V) fail(FHE_ERR_INVALID_ARG, "null factor buffers");
        if (!std::isfinite(lr) || !std::isfinite(lam)) fail(FHE_ERR_INVALID_ARG, "non-finite lr or lambda");
        run_epoch(*p, U, V, level, lr, lam, (cudaStream_t)stream);
    });
}

int fhe_predict(fhe_ctx* ctx, const fhe_mf_plan* p, const uint64_t* U, const uint64_t* V, int32_t level,
                int32_t user, uint64_t* out, void* stream) {
    if (!ctx || !p) return FHE_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    return guarded(&c, [&] {
        if (!U || !V || !out) fail(FHE_ERR_INVALID_ARG, "null buffers");
        run_predict(*p, U, V, level, user, out, (cudaStream_t)stream);
    });
}

}  // extern "C"

/*
 * ckks_mf.h — C ABI of the GB300 RNS-CKKS library for encrypted CSR matrix
 * factorisation (arXiv 2509.03024, "Efficient Privacy-Preserving
 * Recommendation on Sparse Data using Fully Homomorphic Encryption").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Return value: FHE_OK (0) on success, a negative FHE_ERR_* code otherwise.
 *   After a failure fhe_last_error(ctx) describes it, the call's outputs are
 *   unspecified, and the context stays valid and usable.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *   default stream). Device work is enqueued on it in order; an entry point
 *   that returns host data synchronises that stream first. One context must
 *   not be used from two host threads or two streams at the same time: it owns
 *   one set of scratch buffers.
 * Ciphertext buffers ("ct"): caller-owned DEVICE memory of
 *   fhe_ctx_info.ct_words uint64 words = [2][L+1][N] (component, limb,
 *   coefficient), where L is the top level. A ciphertext at level l uses limbs
 *   0..l of each component; the other limbs are ignored and may hold anything.
 *   Limbs are stored in the evaluation (NTT) domain, residues in [0, q_i).
 *   Arrays of ciphertexts are contiguous: ciphertext t starts at t*ct_words.
 * Pointers: "host" pointers are ordinary CPU memory; "device" pointers are
 *   CUDA global memory on the context's device. Neither is retained after the
 *   call returns, except where a function says it stores a pointer.
 *
 * The scheme is leveled CKKS (Cheon-Kim-Kim-Song 2017), which the paper uses
 * for its encrypted MF (Sec. II-A.2 Eq. 6-9, Sec. IV-A), in full-RNS form with
 * hybrid key switching (Han-Ki 2020).
 */
#ifndef CKKS_MF_H
#define CKKS_MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ errors */
enum {
    FHE_OK = 0,
    FHE_ERR_INVALID_ARG = -1,     /* a pointer, size, level or parameter is out of range  */
    FHE_ERR_LEVEL_EXHAUSTED = -2, /* the operation needs more limbs than the input has     */
    FHE_ERR_SCALE_MISMATCH = -3,  /* reserved: operands at different scales                */
    FHE_ERR_MISSING_KEY = -4,     /* keys not generated, or no key for a rotation step     */
    FHE_ERR_OOM = -5,             /* device or host allocation failed                      */
    FHE_ERR_DEVICE_TIMEOUT = -6,  /* a bounded device-side wait gave up                    */
    FHE_ERR_CUDA = -7,            /* a CUDA runtime call failed                            */
    FHE_ERR_STATE = -8            /* the object is not in a state that allows the call     */
};

typedef struct fhe_ctx fhe_ctx;
typedef struct fhe_mf_plan fhe_mf_plan;

/* ------------------------------------------------------------------ context */

/* Scheme parameters (Sec. IV-A fixes N = 8192, 32 fractional bits, 128-bit
 * security for the paper's runs; any power-of-two N in [2^9, 2^16] is accepted).
 * Primes: for each entry of data_prime_bits, then of special_prime_bits, the
 * largest prime below 2^bits that is 1 mod 2N and not chosen before.
 * Bits must lie in [20, 61]. The scale is 2^log_scale. */
typedef struct {
    int32_t log_n;
    int32_t n_data_primes;               /* L + 1                          */
    const int32_t* data_prime_bits;      /* host, n_data_primes entries    */
    int32_t n_special_primes;            /* alpha >= 1                     */
    const int32_t* special_prime_bits;   /* host, n_special_primes entries */
    int32_t log_scale;
    double sigma;                        /* error standard deviation (3.2) */
    int32_t device;                      /* CUDA device ordinal            */
} fhe_params;

typedef struct {
    int32_t log_n, n, slots;             /* N and N/2                      */
    int32_t top_level;                   /* L                              */
    int32_t n_special;                   /* alpha                          */
    int32_t log_scale;
    size_t ct_words;                     /* uint64 words per ciphertext    */
} fhe_ctx_info;

/* Create a context: primes, NTT twiddles, RNS conversion constants and
 * encoding tables, all resident on `device`. *out receives the handle. */
int fhe_ctx_create(const fhe_params* params, fhe_ctx** out);
void fhe_ctx_destroy(fhe_ctx* ctx);
/* Human-readable description of the last error on ctx ("" if none). Valid until the next call. */
const char* fhe_last_error(const fhe_ctx* ctx);
int fhe_ctx_get_info(const fhe_ctx* ctx, fhe_ctx_info* out);
/* Copy the L+1 data primes then the alpha special primes into host `out` (cap entries). */
int fhe_ctx_get_primes(const fhe_ctx* ctx, uint64_t* out, size_t cap);

/* Key generation (the CSP's role, Sec. III-B.1) from one 64-bit seed: the
 * ternary secret s, the public key, the relinearisation key for s^2 and one
 * rotation key per entry of rot_steps (host, left-rotation amounts; negative
 * = right). All randomness is drawn from SplitMix64 streams keyed by
 * (purpose, object, poly, limb) under this seed; the seed also keys later
 * encryptions. Replaces any previous keys. */
int fhe_keygen_from_seed(fhe_ctx* ctx, uint64_t seed, const int32_t* rot_steps, size_t n_steps);
/* Add rotation keys for more steps to the current key set. */
int fhe_add_rotation_keys(fhe_ctx* ctx, const int32_t* rot_steps, size_t n_steps);

/* ------------------------------------------------------------------ encode / encrypt */

/* Encode n_slots real values (host) into the integer coefficient vector
 * round(Delta * m(X)) with m(zeta^(5^t)) = slots[t] (canonical embedding);
 * coeffs_dev: device int64 [N]. Unlisted slots are 0. */
int fhe_encode(fhe_ctx* ctx, const double* slots, size_t n_slots, int64_t* coeffs_dev, void* stream);

/* Encrypt under the public key at `level`: ct = (v*pk0 + e0 + m, v*pk1 + e1).
 * The randomness v, e0, e1 is drawn from the streams of `nonce`; the same
 * (seed, nonce, message) always gives the same ciphertext.
 * fhe_encrypt takes host slots (Eq. 6-9's FHE.Enc of an encoded vector);
 * fhe_encrypt_coeffs takes a device int64 [N] coefficient message. ct: device. */
int fhe_encrypt(fhe_ctx* ctx, const double* slots, size_t n_slots, int32_t level, uint64_t nonce,
                uint64_t* ct, void* stream);
int fhe_encrypt_coeffs(fhe_ctx* ctx, const int64_t* coeffs_dev, int32_t level, uint64_t nonce,
                       uint64_t* ct, void* stream);

/* Decrypt the first n_slots slots into host `slots` (FHE.Dec then decode at
 * scale Delta). Uses limbs 0..min(level, 1). Synchronises `stream`. */
int fhe_decrypt(fhe_ctx* ctx, const uint64_t* ct, int32_t level, double* slots, size_t n_slots,
                void* stream);

/* Key-holder refresh (the CSP role of Sec. III-B; the paper's runs of 20
 * iterations exceed one leveled chain): each of `count` ciphertexts at `level`
 * is decrypted to its exact integer plaintext (centred, from limbs 0..min(level,1),
 * as fhe_decrypt) and encrypted again at the top level with nonce
 * nonce_base + t. No floating-point decode is involved, so the result is
 * reproducible bit for bit. out (device, count ciphertexts) may equal ct.
 * FHE_ERR_INVALID_ARG if a plaintext coefficient does not fit in int64. */
int fhe_refresh(fhe_ctx* ctx, const uint64_t* ct, int32_t count, int32_t level, uint64_t nonce_base, uint64_t* out,
                void* stream);

/* ------------------------------------------------------------------ ring and ciphertext primitives */

/* In-place forward / inverse negacyclic NTT of `count` polynomials of
 * `n_limbs` limbs each (device [count][n_limbs][N], limb i modulo data prime i). */
int fhe_ntt_forward(fhe_ctx* ctx, uint64_t* polys, int32_t count, int32_t n_limbs, void* stream);
int fhe_ntt_inverse(fhe_ctx* ctx, uint64_t* polys, int32_t count, int32_t n_limbs, void* stream);

/* Convert `count` ciphertexts at `level` to coefficient form: out device
 * [count][2][level+1][N] (compact). Used to compare ciphertexts exactly. */
int fhe_ct_to_coeff(fhe_ctx* ctx, const uint64_t* ct, int32_t count, int32_t level, uint64_t* out,
                    void* stream);

/* Homomorphic addition / subtraction (Eq. 6): out = a +/- b at `level`, `count` ciphertexts. */
int fhe_add(fhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, int32_t count,
            int32_t level, void* stream);
int fhe_sub(fhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, int32_t count,
            int32_t level, void* stream);
/* Ciphertext times plaintext (Eq. 9): pt_coeffs_dev is an int64 [N] encoded
 * message (fhe_encode), applied to `count` ciphertexts. No rescale. */
int fhe_mul_plain(fhe_ctx* ctx, const uint64_t* ct, const int64_t* pt_coeffs_dev, uint64_t* out,
                  int32_t count, int32_t level, void* stream);
/* Ciphertext product (Eq. 7): tensor, then relinearise with the s^2 key and
 * rescale by q_level in one key switch whose ModDown divides by P q_level
 * (out_h = (acc_h + P c_h - Conv_{P u {q_l} -> Q_{l-1}}(acc_h + P c_h)) (P q_l)^-1,
 * fast non-centred conversion; equal to fhe_relinearize then fhe_rescale up to a
 * conversion error of at most alpha + 1 per coefficient). Output at level-1.
 * Needs level >= 1. */
int fhe_mul_relin_rescale(fhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out,
                          int32_t count, int32_t level, void* stream);
/* Tensor only: out3 device [count][3][L+1][N] (three components, capacity limbs). */
int fhe_tensor(fhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out3, int32_t count,
               int32_t level, void* stream);
/* Relinearise a three-component tensor (as from fhe_tensor) into a ciphertext. */
int fhe_relinearize(fhe_ctx* ctx, const uint64_t* in3, uint64_t* out, int32_t count, int32_t level,
                    void* stream);
/* Exact rescale (divide-and-round by q_level): level -> level-1. out may equal ct. */
int fhe_rescale(fhe_ctx* ctx, const uint64_t* ct, uint64_t* out, int32_t count, int32_t level,
                void* stream);
/* Rescale of ONE ciphertext (as fhe_rescale with count = 1, same result)
 * without any allocation. The paper has no counterpart: this entry point is
 * for callers that cannot let a library allocate while they run, e.g. an
 * application that owns all device memory through its own allocator, or a
 * latency-critical loop where a cudaMalloc / cudaFree (which may synchronise
 * the device) is not acceptable. It calls no cudaMalloc, cudaFree or other
 * allocating routine; its scratch space is a 16 MiB array compiled into the
 * library (held on every GPU that loads the library until the process exits).
 * Limit: 2 * N * (level + 1) <= 2^21, i.e. level <= 31 at N = 2^15 or level <= 15
 * at N = 2^16; larger inputs are rejected with FHE_ERR_INVALID_ARG. The first
 * call on a device looks up the scratch array's device address (once per
 * device); make that first call before any stream capture. All calls share
 * the one scratch array: two calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and corrupt each other's results;
 * order them on one stream. The call counts its launches in the context's
 * launch accounting but records no per-launch timing events (creating an event
 * may allocate), on the calling host thread only. ct: device, level `level`;
 * out: device, receives level - 1 (may equal ct). */
int fhe_rescale_noalloc(fhe_ctx* ctx, const uint64_t* ct, uint64_t* out, int32_t level, void* stream);
/* Left slot rotation by `step` (negative = right): automorphism X -> X^(5^step)
 * then key switching with that step's rotation key. out must not alias ct. */
int fhe_rotate(fhe_ctx* ctx, const uint64_t* ct, uint64_t* out, int32_t count, int32_t level,
               int32_t step, void* stream);
/* In-block rotate-and-sum: out = sum_{r=0}^{kp-1} rot(ct, r), the inner-product step of the
 * paper's encrypted error e = r - <u, v> (Alg. 1) on vectors written twice per block of 2 kp
 * slots, where every slot x < kp of a block receives the block's sum. For 2 <= kp <= 16 the key
 * switches are hoisted (Halevi and Shoup 2018): one ModUp of c1, kp - 1 key inner products over
 * the rotated raised digits, one ModDown. Its bits then differ from a sum of fhe_rotate results
 * (same plaintext; the noise of one key switch). A power of two kp > 16 runs log2(kp)
 * rotate-and-adds. Needs the rotation keys of steps 1..kp-1 (kp <= 16) or of the powers of two
 * below kp. ct, out: device, `count` ciphertexts at `level`. For kp <= 16 out may equal ct;
 * for kp > 16 ct is overwritten and must not alias out. Other kp: FHE_ERR_INVALID_ARG. */
int fhe_rotate_sum(fhe_ctx* ctx, uint64_t* ct, uint64_t* out, int32_t count, int32_t level, int32_t kp,
                   void* stream);

/* Fan-in rotation: for every group g, acc_g += sum_{first[g] <= i < first[g+1]} rot(ct_i, steps[i]),
 * the back-rotation of the item gradients onto a delta tree's parent node (the paper's gradient
 * accumulator, Alg. 2, applied to the rotated node gradients). The children's key inner products
 * and rotated c0's are summed before one ModDown per group, so the bits differ from adding
 * fhe_rotate results (same plaintext; the noise of one key switch per group). acc: device,
 * n_groups ciphertexts at `level`, updated in place; ct: device, first[n_groups] ciphertexts at
 * `level`, none aliasing an acc; first: host, n_groups + 1 non-decreasing offsets from 0 to the
 * input count; steps: host, one nonzero rotation step (not a multiple of the slot count) per
 * input, each with its rotation key. Errors: FHE_ERR_INVALID_ARG for bad offsets or steps,
 * FHE_ERR_MISSING_KEY for a step without a key. */
int fhe_rotate_fanin(fhe_ctx* ctx, uint64_t* acc, int32_t n_groups, const int32_t* first, const uint64_t* ct,
                     const int32_t* steps, int32_t level, void* stream);

/* ------------------------------------------------------------------ launch accounting */

/* Measurement helper (no counterpart in the paper): the rate, in 10^9 butterflies per second,
 * at which this GPU runs the forward NTT's butterfly arithmetic (lazy Shoup Cooley-Tukey
 * butterflies, three stages per radix-8 block, a reduction every 15 stages) on values held in
 * registers, with no memory traffic inside the loop. It is the integer-pipe ceiling of the
 * NTT passes. reps: loop trips (each thread does 60 butterflies per trip; ~2000 takes tens of
 * milliseconds). Runs on the default stream and synchronises. Errors: FHE_ERR_INVALID_ARG for
 * reps < 1 or a null output. */
int fhe_probe_butterfly_rate(fhe_ctx* ctx, int32_t reps, double* gbfly_per_s);

/* Measurement helper (no counterpart in the paper): issue rates of the 32-bit integer multiply
 * instructions that 64-bit modular arithmetic is built from, and of four formulations of the
 * 64 x 64 -> 128-bit multiply-accumulate of the key inner product, all on register operands with no
 * memory traffic (152 SMs x 4 CTAs of 256 threads on GB300). The bench turns them into the integer
 * ceilings of the NTT butterfly and of the key inner product. Rates are in 10^9 instructions (or
 * multiply-accumulates) per second. reps: loop trips (each trip is 128 instructions or 32 MACs per
 * thread; ~500 takes milliseconds). Runs on the default stream and synchronises. Errors:
 * FHE_ERR_INVALID_ARG for reps < 1 or a null output. */
typedef struct {
    int32_t sms;
    double imad_lo_gops;      /* mad.lo.u32            */
    double imad_hi_gops;      /* mad.hi.u32            */
    double imad_wide_gops;    /* mad.wide.u32          */
    double mac_c_gmacs;       /* C: lo/hi halves + carry compare          */
    double mac_ptx64_gmacs;   /* PTX mad.lo.cc.u64 / madc.hi.u64          */
    double mac_ptx32_gmacs;   /* PTX 32-bit schoolbook chain with carries */
    double mac_wide_gmacs;    /* four mad.wide.u32 into column sums       */
} fhe_int_pipe_rates;
int fhe_probe_int_pipe(fhe_ctx* ctx, int32_t reps, fhe_int_pipe_rates* out);

/* Autotuner (no counterpart in the paper; the launch shapes are this library's). Several kernel
 * families have launch variants that compute identical bits and differ only in speed. For each
 * family fhe_autotune times every variant on a synthetic batch of this context's shape at `level`
 * (1 <= level <= top level; the per-group products of an epoch run at top - 1), keeps the fastest
 * for the context and writes one record per (family, variant) to host `out` (up to cap; `chosen`
 * is 1 for the kept variant, `ms` the best of three timed launches). Returns the number of records
 * or an error code. Synchronises the device; allocates and frees temporary device memory.
 * Families: "ks_hoist_inner" (the hoisted rotate-and-sum's key inner product, 15 rotations),
 * "ks_inner" (a relinearisation's key inner product), variants v0 c1 p1 s1 s2 s2l; "ntt" (the tile
 * shape of the plain two-pass NTT of rings 2^14..2^16: rows or columns per tile and residues per
 * thread, variants r16b4 r8b4 r32b4 r16b3; timed on a forward plus inverse transform of 256 rows);
 * "ks_pass" (rows or columns per tile of the fused key-switch and rescale passes of rings 2^14..2^16,
 * variants r16 r8 r8x; timed on the exact rescale of 64 ciphertexts). A fresh context uses the first
 * variant of each.
 * `family` and `variant` point to static strings. */
typedef struct {
    const char* family;
    const char* variant;
    int32_t chosen;
    double ms;
} fhe_tune_result;
int fhe_autotune(fhe_ctx* ctx, int32_t level, fhe_tune_result* out, int32_t cap);
/* Select a variant by name (FHE_ERR_INVALID_ARG for an unknown family or variant); results do not
 * change. fhe_get_variant writes the current variant's name (a static string) to *variant. */
int fhe_set_variant(fhe_ctx* ctx, const char* family, const char* variant);
int fhe_get_variant(const fhe_ctx* ctx, const char* family, const char** variant);

/* Measurement helper (no counterpart in the paper): what the base conversion costs inside the fused
 * ModUp pass, the evidence for keeping it on the CUDA cores. Times, with CUDA events (best of 5,
 * after a warm-up, on the default stream), the forward-transform pass set of the key switch's
 * conversion step over `sources` synthetic inputs at `level` (every target limb x outside a digit
 * loads sum_{i in digit} y_i qhat_i mod p_x while its tile is read; Bajard et al. 2016) and the
 * same rows loading one limb with no conversion. conv_ms - plain_ms bounds what any other form of
 * the conversion could save inside the pass; an unfused form (a separate matrix product) would
 * add roundtrip_bytes of HBM traffic (a write and a re-read of every converted limb). Errors:
 * FHE_ERR_INVALID_ARG for level outside 1..L, sources < 1 or a null output. */
typedef struct {
    double conv_ms;          /* pass set with the conversion in its loads */
    double plain_ms;         /* same rows, one plain limb load each */
    int32_t rows;            /* converted limbs (transform rows) per pass set */
    double roundtrip_bytes;  /* 16 N bytes per row */
} fhe_conv_cost;
int fhe_probe_conv_cost(fhe_ctx* ctx, int32_t level, int32_t sources, fhe_conv_cost* out);

/* Per kernel class: launches, summed device time (only when timing was
 * requested), the algorithmic bytes those launches must move (inputs read
 * once plus outputs written once) and their arithmetic work: butterflies for
 * the NTT classes (a pass of S stages over R rows does R * S * N / 2), 64 x 64-bit
 * multiply-accumulates for the key inner products, 0 otherwise. `name` points
 * to a static string. */
typedef struct {
    const char* name;
    int64_t launches;
    double device_ms;
    double bytes;
    double work;
} fhe_kernel_stat;

/* Reset the counters. With time_kernels != 0 every launch is also bracketed
 * by CUDA events on its stream (small overhead per launch). */
int fhe_profile_begin(fhe_ctx* ctx, int32_t time_kernels);
/* Synchronise the device, write up to cap class records to host `out`, stop
 * timing. Returns the number of classes (>= 0) or an error code. */
int fhe_profile_end(fhe_ctx* ctx, fhe_kernel_stat* out, int32_t cap);

/* ------------------------------------------------------------------ encrypted CSR matrix factorisation */

typedef struct {
    int32_t n_users, n_items, k;         /* rating matrix n x m, rank k              */
    int32_t kp, w, B;                    /* next_pow2(k), slot block 2*kp, B = N/2/w */
    int32_t n_user_batches, n_item_batches;
    int64_t n_ratings, n_groups;         /* M and the number of (b, c, delta) groups */
    int64_t n_tree_nodes;                /* delta-tree nodes over all item batches   */
    int64_t n_bins;                      /* rating ciphertexts (bins)                */
    size_t device_bytes;                 /* device memory owned by the plan          */
} fhe_mf_plan_info;

/* The rotation amounts an MF epoch with rank k needs (keys must exist for all
 * of them): the in-block sum's, the delta tree's baby steps r*w (0 < r < beta)
 * and giant steps 2^t*beta*w (< B*w) in both directions, and the half-fill -kp.
 * Writes up to cap entries to host `out`; returns the count (>= 0) or an error
 * code. */
int fhe_mf_rotation_steps(const fhe_ctx* ctx, int32_t k, int32_t* out, size_t cap);

/* EncryptCsrMatrix + batch-pair grouping (Alg. 1, Alg. 2, Fig. 5).
 * Input: the n x m rating matrix in CSR form (host: row_ptr[n+1] int64,
 * col_idx[M] int32, vals[M] double; Sec. II-A.3), rank k. Users and items are
 * cut into batches of B; a rating (i, j) joins group (i div B, j div B,
 * (j mod B - i mod B) mod B), groups in (b, c, delta) order. The ratings are
 * stored in bins (the paper packs many ratings per ciphertext, Sec. III-C):
 * within each user batch, each group goes to the first bin (in creation order)
 * that holds none of its users, else to a new bin; bins are numbered batch by
 * batch. The key holder encrypts each bin at level L - 1 (the highest level an
 * epoch reads it at) with a regenerable c1: c1 = a, the uniform polynomial drawn
 * coefficient by coefficient from the seed's stream (purpose 9, object
 * 2^40 + bin, one stream per limb), c0 = -a s + m + e (e: purpose 10, same
 * object). The plan keeps c0 only and regenerates c1 when an epoch reads the
 * bin. Duplicate (i, j) pairs are rejected. */
int fhe_csr_pack(fhe_ctx* ctx, int32_t n, int32_t m, int32_t k, const int64_t* row_ptr,
                 const int32_t* col_idx, const double* vals, fhe_mf_plan** out);
/* Host only (no context, no device; runs on a machine without a GPU): the layout fhe_csr_pack
 * computes for a ring of `slots` = N/2 slots (a power of two in [2^8, 2^15]), from the same CSR
 * input with the same checks. counts (host int64[3]) receives the number of groups, rating bins
 * and delta-tree nodes. Each other output may be NULL; the non-NULL group arrays (host int32,
 * group_cap entries) receive, per group in (b, c, delta) order, its user batch, item batch, delta,
 * rating count and bin; the non-NULL node arrays (host int32, node_cap entries) receive, per node
 * in the plan's order (item batch, then delta ascending), its item batch and delta. Call with NULL
 * arrays first to learn the counts. FHE_ERR_INVALID_ARG (counts written) if a non-NULL array is
 * shorter than its count. */
int fhe_mf_layout(int32_t slots, int32_t n, int32_t m, int32_t k, const int64_t* row_ptr,
                  const int32_t* col_idx, const double* vals, int64_t* counts, int32_t* group_b,
                  int32_t* group_c, int32_t* group_delta, int32_t* group_count, int32_t* bin_of_group,
                  int64_t group_cap, int32_t* node_c, int32_t* node_delta, int64_t node_cap);
void fhe_mf_plan_destroy(fhe_mf_plan* plan);
int fhe_mf_plan_get_info(const fhe_mf_plan* plan, fhe_mf_plan_info* out);
/* Copy the plan's groups to host arrays of n_groups entries (any may be NULL):
 * user batch b, item batch c, delta, and the number of ratings in the group. */
int fhe_mf_plan_get_groups(const fhe_mf_plan* plan, int32_t* b, int32_t* c, int32_t* delta,
                           int32_t* count);
/* Copy the rating bin of each group (host int32[n_groups]). */
int fhe_mf_plan_get_bins(const fhe_mf_plan* plan, int32_t* bin_of_group);

/* Tuning: process at most `groups_per_chunk` groups per launch set of the
 * epoch (default: as many as fit a 6 GiB work area). Results do not depend on it. */
int fhe_mf_plan_set_chunk(fhe_mf_plan* plan, int32_t groups_per_chunk);
/* Memory: the epoch runs the item batches in consecutive waves whose delta-tree
 * workspace (per node one rotated item ciphertext, one gradient ciphertext and one
 * three-component accumulator at the top level) fits `bytes` (default 72 GiB; a wave
 * holds at least one item batch). The user-side accumulators span all waves. Results
 * do not depend on it. */
int fhe_mf_plan_set_wave_budget(fhe_mf_plan* plan, uint64_t bytes);

/* Encrypt factor rows (host double [count][k], users if which = 0, items if 1)
 * into the plan's batch layout: n_user_batches (or n_item_batches)
 * ciphertexts at the top level, entity a of a batch at slot block a, its
 * k-vector written twice (slots a*w..a*w+k-1 and a*w+kp..a*w+kp+k-1).
 * Nonces: 2^41 + batch (users), 2^41 + 2^40 + batch (items). cts: device. */
int fhe_mf_encrypt_factors(fhe_ctx* ctx, const fhe_mf_plan* plan, int32_t which, const double* X,
                           int32_t count, uint64_t* cts, void* stream);
/* Decrypt batch ciphertexts at `level` back to host double [count][k]. */
int fhe_mf_decrypt_factors(fhe_ctx* ctx, const fhe_mf_plan* plan, int32_t which,
                           const uint64_t* cts, int32_t level, double* X, int32_t count,
                           void* stream);

/* One encrypted SGD epoch (Alg. 1 error and gradient, Alg. 2 accumulators,
 * applied once per epoch). Item batch c rotated by delta*w (delta < B) lines up
 * the pairs of group (b, c, delta); the rotated copies come from a baby-step
 * giant-step delta tree: with beta = 2^floor(log2(B)/2) and delta = g*beta + r,
 * a baby (r > 0) is its giant g*beta rotated by r*w, a giant (g > 0) is giant
 * (g - 2^hb(g))*beta rotated by 2^hb(g)*beta*w, and the rotations out of one
 * node share its ModUp; the item gradients return along the same tree. For every
 * rating e_ij = r_ij - <u_i, v_j> with the epoch-start factors, then
 *   u_i <- u_i (1 - lr*lambda*nnz_i) + lr * sum_j e_ij v_j,
 *   v_j <- v_j (1 - lr*lambda*nnz_j) + lr * sum_i e_ij u_i.
 * U: device, n_user_batches ciphertexts; V: device, n_item_batches; both at
 * `level` on entry and level-2 on return (updated in place).
 * Needs level >= 2 (else FHE_ERR_LEVEL_EXHAUSTED) and every key of
 * fhe_mf_rotation_steps (else FHE_ERR_MISSING_KEY). */
int fhe_mf_sgd_epoch(fhe_ctx* ctx, fhe_mf_plan* plan, uint64_t* U, uint64_t* V, int32_t level,
                     double lr, double lambda, void* stream);

/* Encrypted predicted ratings of one user against every item (a row of
 * R-hat = U V^T, Alg. 1): out receives n_item_batches ciphertexts at level-2;
 * slot d*w of ciphertext c holds <u_user, v_(c*B+d)>. Needs rotation keys
 * for 2^t * w (t < log2 B) and those of fhe_rotate_sum with this kp (steps
 * 1..kp-1 for kp <= 16, else the powers of two below kp); every one of them
 * is in fhe_mf_rotation_steps. */
int fhe_predict(fhe_ctx* ctx, const fhe_mf_plan* plan, const uint64_t* U, const uint64_t* V,
                int32_t level, int32_t user, uint64_t* out, void* stream);

/* ------------------------------------------------------------------ serving (continuous batching) */

/* A request loop over resident encrypted item factors. Each request carries one
 * user's encrypted rating row and initial factor and is answered with the
 * encrypted predicted-rating row after `steps` fold-in steps (Alg. 1 error and
 * gradient lines applied to the user's ratings, Alg. 2's accumulated update;
 * item factors stay fixed). Layout: the user's k-vector in every slot block;
 * item j = c*B + d in block d of item batch c (the packing of
 * fhe_mf_encrypt_factors with which = 1).
 *
 * Step at level l (two levels): for each item batch c holding a rated item,
 * S_c = rotsum_kp(rescale(relin(UR (x) V_c))), E_c = R_c - S_c,
 * T += E_c (x) rescale(V_c (.) mask_c) (mask_c = lr on the first k slots of the
 * rated blocks); G = rescale(relin(T)); G = sum_{a<B} rot(G, a w) (the block sum)
 * then G += rot(G, -kp) (the half-fill), both as rounds of hoisted rotate-and-sums
 * (G <- sum over the round's steps r of rot(G, r)): radix-4 rounds of steps
 * 0, s, 2s, 3s with strides s = w, 4w, 16w, ..., a radix-2 round (0, s) when
 * log2 B is odd, and the last round's steps r extended by r - kp;
 * UR <- drop(rescale(UR * round((1 - lr lambda nnz) Delta))) + G.
 * The prediction pass computes S_c for every batch at the final level (one
 * level): slot d*w of output c is <u, v_(cB+d)>.
 *
 * Admission is memory based: the server owns `max_slots` request slots (each
 * holding a request's inputs and its share of the batched work area), capped
 * so that all slots fit in `memory_budget_bytes` of device memory. A submit
 * that finds no free slot returns FHE_ERR_STATE and changes nothing; the
 * caller keeps the request queued and retries after a tick frees a slot.
 * Every tick advances every admitted request by one step in shared batched
 * launches (requests at different levels are grouped per level); a request
 * admitted between ticks joins at the next tick. A tick only enqueues its work
 * on the stream and returns: the host may admit requests and build the next
 * tick while the GPU runs this one (the library keeps at most two calls'
 * descriptor tables in flight). Results do not depend on which other requests
 * share a tick. */
typedef struct fhe_server fhe_server;

/* Rotation steps a server for rank k needs. Same return convention as fhe_mf_rotation_steps. */
int fhe_serve_rotation_steps(const fhe_ctx* ctx, int32_t k, int32_t* out, size_t cap);
/* V: device, ceil(m / B) item-batch ciphertexts at the top level (copied; the
 * server keeps its own resident copy). Needs top level >= 2 * steps + 1. */
int fhe_serve_create(fhe_ctx* ctx, const uint64_t* V, int32_t m, int32_t k, int32_t steps, double lr,
                     double lambda, int32_t max_slots, size_t memory_budget_bytes, fhe_server** out);
void fhe_serve_destroy(fhe_server* server);
/* Slots the server actually allocated (after the memory cap) and slots now free. */
int fhe_serve_slots(const fhe_server* server, int32_t* total, int32_t* free_slots);
/* Admit a request if a slot is free. items: host int32 [nnz] distinct item
 * indices < m; UR: one ciphertext (u in every block), R: ceil(m/B) ciphertexts
 * (rating of item c*B+d on the first k slots of block d of R_c); both at the
 * top level, in device memory or in host memory (page-locked host memory keeps
 * the upload asynchronous); copied on `stream` before the call returns for
 * pageable memory, else in stream order. FHE_ERR_STATE if no slot is free. */
int fhe_serve_submit(fhe_server* server, int64_t request_id, const int32_t* items, int32_t nnz,
                     const uint64_t* UR, const uint64_t* R, void* stream);
/* Advance every admitted request by one step: enqueue the step on `stream`
 * without waiting for it. Returns the number of admitted requests whose last
 * step has not been enqueued yet (>= 0) or an error. */
int fhe_serve_tick(fhe_server* server, void* stream);
/* Ids of requests whose whole computation has completed on the device since the
 * last poll (up to cap; host; never blocks). Returns the count. */
int fhe_serve_poll(fhe_server* server, int64_t* ids, int32_t cap);
/* Client-side helper: pack and encrypt one request at the top level. u0: host
 * double [k]; items/ratings: host [nnz]. UR receives u0 in every block (nonce
 * nonce_base), R receives ceil(m/B) rating ciphertexts (nonces nonce_base+1+c). */
int fhe_serve_encrypt_request(fhe_ctx* ctx, int32_t m, int32_t k, const double* u0, const int32_t* items,
                              const double* ratings, int32_t nnz, uint64_t nonce_base, uint64_t* UR,
                              uint64_t* R, void* stream);
/* Copy a completed request's prediction (ceil(m/B) ciphertexts at *level;
 * limbs 0..*level of each component, the other limbs of `out` are left as they
 * are) to `out` (device or host memory, capacity layout) and free its slot.
 * Synchronises `stream`. */
int fhe_serve_take(fhe_server* server, int64_t request_id, uint64_t* out, int32_t* level, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CKKS_MF_H */

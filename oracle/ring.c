/*
 * Oracle ring arithmetic for RNS-CKKS — TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, exact CPU code. It is used by tests/, by the smoke check and by
 * the CPU-baseline leg of the benchmark; nothing in the product path may link
 * or call it. It shares no code, header or table with the CUDA library.
 *
 * Every residue is a uint64_t in [0, q). Products are formed in unsigned
 * __int128 and reduced with the C `%` operator, so each modular operation is
 * its own definition.
 *
 * Contents (all for the cyclotomic ring Z_q[X]/(X^N + 1), coefficient form):
 *   - modular add / sub / mul / pow / inverse, deterministic Miller-Rabin
 *   - schoolbook negacyclic product (the definition of ring multiplication)
 *   - negacyclic product via a textbook radix-2 NTT (psi-twisted cyclic NTT)
 *   - the automorphism a(X) -> a(X^g)
 *   - RNS fast base conversion and the exact centred rescale
 * The CKKS algorithms (Cheon-Kim-Kim-Song 2017, the scheme the paper uses in
 * Sec. IV-A; full-RNS form of Cheon-Han-Kim-Kim-Song 2018; hybrid key switching
 * of Han-Ki 2020) are composed from these in oracle/ckks.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;

u64 or_addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
u64 or_submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - b) % q); }
u64 or_mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 or_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q, x = a % q;
    while (e) {
        if (e & 1) r = or_mulmod(r, x, q);
        x = or_mulmod(x, x, q);
        e >>= 1;
    }
    return r;
}

/* Inverse modulo a prime q (Fermat). */
u64 or_invmod(u64 a, u64 q) { return or_powmod(a, q - 2, q); }

/* Deterministic Miller-Rabin for n < 2^64 (the first 12 prime bases suffice). */
int or_is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = or_mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* out = (s * a) mod q, coefficient-wise. */
void or_scalar_mul(const u64* a, u64 s, u64* out, int n, u64 q) {
    for (int k = 0; k < n; k++) out[k] = or_mulmod(a[k], s % q, q);
}

/* Definition of the product in Z_q[X]/(X^N+1): c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j. */
void or_negacyclic_schoolbook(const u64* a, const u64* b, u64* out, int n, u64 q) {
    for (int k = 0; k < n; k++) out[k] = 0;
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            u64 p = or_mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < n) out[k] = or_addmod(out[k], p, q);
            else out[k - n] = or_submod(out[k - n], p, q);
        }
    }
}

/* A primitive 2N-th root of unity psi mod q (q = 1 mod 2N): the first g = 2,3,...
 * whose power g^((q-1)/2N) satisfies psi^N = -1. */
u64 or_find_psi(int n, u64 q) {
    u64 e = (q - 1) / (2 * (u64)n);
    for (u64 g = 2; g < 1000000; g++) {
        u64 psi = or_powmod(g, e, q);
        if (or_powmod(psi, (u64)n, q) == q - 1) return psi;
    }
    return 0;
}

static unsigned bitrev(unsigned x, int bits) {
    unsigned r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* Textbook iterative radix-2 cyclic DFT over Z_q with root omega (order n):
 * bit-reversal permutation, then log2(n) butterfly stages. In place. */
static void cyclic_ntt(u64* a, int n, u64 omega, u64 q) {
    int bits = 0;
    while ((1 << bits) < n) bits++;
    for (int i = 0; i < n; i++) {
        int j = (int)bitrev((unsigned)i, bits);
        if (j > i) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        u64 wlen = or_powmod(omega, (u64)(n / len), q);
        for (int s = 0; s < n; s += len) {
            u64 w = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[s + j];
                u64 v = or_mulmod(a[s + j + len / 2], w, q);
                a[s + j] = or_addmod(u, v, q);
                a[s + j + len / 2] = or_submod(u, v, q);
                w = or_mulmod(w, wlen, q);
            }
        }
    }
}

/* Evaluations a(psi^(2k+1)), k = 0..n-1: twist by psi^j, then a cyclic DFT with omega = psi^2. */
static void negacyclic_eval(const u64* a, u64* out, int n, u64 psi, u64 q) {
    u64 pw = 1;
    for (int j = 0; j < n; j++) { out[j] = or_mulmod(a[j], pw, q); pw = or_mulmod(pw, psi, q); }
    cyclic_ntt(out, n, or_mulmod(psi, psi, q), q);
}

/* Inverse of negacyclic_eval: inverse cyclic DFT, scale by 1/n, untwist by psi^-j. */
static void negacyclic_interp(u64* a, int n, u64 psi, u64 q) {
    u64 psi_inv = or_invmod(psi, q);
    cyclic_ntt(a, n, or_mulmod(psi_inv, psi_inv, q), q);
    u64 n_inv = or_invmod((u64)n % q, q);
    u64 pw = n_inv;
    for (int j = 0; j < n; j++) { a[j] = or_mulmod(a[j], pw, q); pw = or_mulmod(pw, psi_inv, q); }
}

/* out = sum_{t < count} A_t * B_t in Z_q[X]/(X^N+1); A, B are count consecutive length-n arrays.
 * Products are taken through the evaluation map (ring isomorphism), summed, and mapped back. */
int or_negacyclic_dot(const u64* A, const u64* B, int count, u64* out, int n, u64 q) {
    u64 psi = or_find_psi(n, q);
    if (!psi) return -1;
    u64* ea = (u64*)malloc(sizeof(u64) * n);
    u64* eb = (u64*)malloc(sizeof(u64) * n);
    u64* acc = (u64*)calloc((size_t)n, sizeof(u64));
    if (!ea || !eb || !acc) { free(ea); free(eb); free(acc); return -2; }
    for (int t = 0; t < count; t++) {
        negacyclic_eval(A + (size_t)t * n, ea, n, psi, q);
        negacyclic_eval(B + (size_t)t * n, eb, n, psi, q);
        for (int k = 0; k < n; k++) acc[k] = or_addmod(acc[k], or_mulmod(ea[k], eb[k], q), q);
    }
    negacyclic_interp(acc, n, psi, q);
    memcpy(out, acc, sizeof(u64) * n);
    free(ea); free(eb); free(acc);
    return 0;
}

/* Batched form: rows independent products out[r] = sum_t A[r][t] * B[r][t] mod q[r].
 * A and B are [rows][count][n]; q is [rows]. */
int or_negacyclic_dot_rows(const u64* A, const u64* B, int rows, int count, u64* out,
                           int n, const u64* q) {
    for (int r = 0; r < rows; r++) {
        int rc = or_negacyclic_dot(A + (size_t)r * count * n, B + (size_t)r * count * n, count,
                                   out + (size_t)r * n, n, q[r]);
        if (rc) return rc;
    }
    return 0;
}

/* a(X) -> a(X^g) in Z_q[X]/(X^N+1) for odd g: X^(j*g) = (-1)^floor(jg/N) X^(jg mod N). */
void or_automorphism(const u64* a, u64* out, int n, u64 g, u64 q) {
    u64 two_n = 2 * (u64)n;
    for (int j = 0; j < n; j++) {
        u64 e = ((u64)j * g) % two_n;
        if (e < (u64)n) out[e] = a[j];
        else out[e - n] = (a[j] == 0) ? 0 : q - a[j];
    }
}

/*
 * Fast (approximate, non-centred) RNS base conversion of Bajard et al. 2016:
 * given residues x_i of x modulo the primes src[0..n_src), compute for every
 * destination prime p:  sum_i [x_i * qhat_i^{-1}]_{q_i} * (qhat_i mod p)  mod p,
 * with qhat_i = prod_{i' != i} src[i']. The result is x + u*Q (0 <= u < n_src).
 * in: [n_src][n], out: [n_dst][n].
 */
void or_fast_base_conv(const u64* in, const u64* src, int n_src, u64* out, const u64* dst,
                       int n_dst, int n) {
    u64* y = (u64*)malloc(sizeof(u64) * (size_t)n_src * n);
    for (int i = 0; i < n_src; i++) {
        u64 qhat = 1;
        for (int i2 = 0; i2 < n_src; i2++) if (i2 != i) qhat = or_mulmod(qhat, src[i2] % src[i], src[i]);
        u64 qhat_inv = or_invmod(qhat, src[i]);
        for (int k = 0; k < n; k++) y[(size_t)i * n + k] = or_mulmod(in[(size_t)i * n + k], qhat_inv, src[i]);
    }
    for (int d = 0; d < n_dst; d++) {
        u64 p = dst[d];
        for (int k = 0; k < n; k++) out[(size_t)d * n + k] = 0;
        for (int i = 0; i < n_src; i++) {
            u64 qhat_p = 1;
            for (int i2 = 0; i2 < n_src; i2++) if (i2 != i) qhat_p = or_mulmod(qhat_p, src[i2] % p, p);
            for (int k = 0; k < n; k++) {
                u64 t = or_mulmod(y[(size_t)i * n + k] % p, qhat_p, p);
                out[(size_t)d * n + k] = or_addmod(out[(size_t)d * n + k], t, p);
            }
        }
    }
    free(y);
}

/*
 * Exact rescale by the last prime q_l of the residues x_0..x_l (coefficient form):
 *   x_i' = (x_i - [x_l]_centred) * q_l^{-1}  mod q_i,  i < l,
 * where [x_l]_centred is the representative of x_l in (-q_l/2, q_l/2). For the
 * CRT integer x in [0, Q) this equals round(x / q_l) mod Q/q_l (q_l odd, so no ties).
 * in: [l+1][n], primes: [l+1], out: [l][n].
 */
void or_rescale(const u64* in, const u64* primes, int l, u64* out, int n) {
    u64 ql = primes[l];
    const u64* last = in + (size_t)l * n;
    for (int i = 0; i < l; i++) {
        u64 qi = primes[i];
        u64 inv = or_invmod(ql % qi, qi);
        for (int k = 0; k < n; k++) {
            u64 r = last[k];
            u64 r_mod;  /* the centred representative of r, reduced modulo q_i */
            if (r > ql / 2) r_mod = or_submod(0, (ql - r) % qi, qi);
            else r_mod = r % qi;
            u64 diff = or_submod(in[(size_t)i * n + k], r_mod, qi);
            out[(size_t)i * n + k] = or_mulmod(diff, inv, qi);
        }
    }
}

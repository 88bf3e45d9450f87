// ntt.cu — batched negacyclic NTT over RNS limbs (forward: Cooley-Tukey with
// merged psi powers, natural order in, bit-reversed order out; inverse:
// Gentleman-Sande, bit-reversed in, natural out, times N^-1).
//
// Output order: slot k of the forward transform holds a(psi^(2*brev(k)+1)).
// Rings up to N = 2^14 are transformed by one CTA per row with the whole row in
// shared memory. Larger rings use two passes over an N1 x N2 view
// (N = N1 * N2): the first log2(N1) butterfly stages couple elements N2 apart
// and run on tiles of consecutive columns; the remaining stages couple
// elements inside one contiguous row of N2 and run on tiles of whole rows.
#include "core.cuh"

namespace fhe {

namespace {

constexpr int kTile = 4096;  // elements per CTA in the two-pass kernels (32 KiB)

struct RowPtr {
    u64* p;
    int prime;
};

__device__ __forceinline__ RowPtr row_ptr(const PolyBatch& pb, int row, int n) {
    int li = row % pb.n_limbs;
    int rest = row / pb.n_limbs;
    int part = rest % pb.n_parts;
    int item = rest / pb.n_parts;
    int limb = pb.limb_lo + li;
    RowPtr r;
    r.p = pb.base + (size_t)item * pb.item_stride + (size_t)part * pb.part_stride +
          (size_t)(limb - pb.addr_lo) * n;
    r.prime = pb.prime_of(limb);
    return r;
}

// Stages [0, S1) on tiles of `cols` consecutive columns of the N1 x N2 view
// (S1 = log N and cols = N2 = 1 for the single-pass transform).
template <bool INV>
__global__ void ntt_col_kernel(PolyBatch pb, const Prime* __restrict__ primes,
                               const u64* __restrict__ tw, const u64* __restrict__ tws,
                               const u64* __restrict__ ninv, int log_n, int S1, int log_cols) {
    extern __shared__ u64 sm[];
    const int n = 1 << log_n;
    const RowPtr rp = row_ptr(pb, blockIdx.x, n);
    const u64 q = primes[rp.prime].q;
    const u64* W = tw + (size_t)rp.prime * n;
    const u64* Ws = tws + (size_t)rp.prime * n;
    const int N1 = 1 << S1;
    const int log_n2 = log_n - S1;
    const int cols = 1 << log_cols;
    const int c0 = blockIdx.y << log_cols;
    const int total = N1 << log_cols;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int r = e >> log_cols, c = e & (cols - 1);
        sm[e] = rp.p[(size_t)(c0 + c) + ((size_t)r << log_n2)];
    }
    __syncthreads();
    const int half = total >> 1;
    if (!INV) {
        for (int s = 0; s < S1; s++) {
            const int log_tl = S1 - 1 - s;
            for (int bi = threadIdx.x; bi < half; bi += blockDim.x) {
                int c = bi & (cols - 1);
                int p = bi >> log_cols;
                int g = p >> log_tl;
                int jj = p & ((1 << log_tl) - 1);
                int r0 = (g << (log_tl + 1)) + jj;
                int i0 = (r0 << log_cols) + c;
                int i1 = i0 + (1 << (log_tl + log_cols));
                int wi = (1 << s) + g;
                u64 x = sm[i0];
                u64 y = mul_shoup(sm[i1], W[wi], Ws[wi], q);
                sm[i0] = add_mod(x, y, q);
                sm[i1] = sub_mod(x, y, q);
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int r = e >> log_cols, c = e & (cols - 1);
            rp.p[(size_t)(c0 + c) + ((size_t)r << log_n2)] = sm[e];
        }
    } else {
        for (int s = S1 - 1; s >= 0; s--) {
            const int log_tl = S1 - 1 - s;
            for (int bi = threadIdx.x; bi < half; bi += blockDim.x) {
                int c = bi & (cols - 1);
                int p = bi >> log_cols;
                int g = p >> log_tl;
                int jj = p & ((1 << log_tl) - 1);
                int r0 = (g << (log_tl + 1)) + jj;
                int i0 = (r0 << log_cols) + c;
                int i1 = i0 + (1 << (log_tl + log_cols));
                int wi = (1 << s) + g;
                u64 x = sm[i0];
                u64 y = sm[i1];
                sm[i0] = add_mod(x, y, q);
                sm[i1] = mul_shoup(sub_mod(x, y, q), W[wi], Ws[wi], q);
            }
            __syncthreads();
        }
        const u64 ni = ninv[2 * rp.prime], nis = ninv[2 * rp.prime + 1];
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int r = e >> log_cols, c = e & (cols - 1);
            rp.p[(size_t)(c0 + c) + ((size_t)r << log_n2)] = mul_shoup(sm[e], ni, nis, q);
        }
    }
}

// Stages [S1, log N) on tiles of 2^log_rows whole rows of length N2.
template <bool INV>
__global__ void ntt_row_kernel(PolyBatch pb, const Prime* __restrict__ primes,
                               const u64* __restrict__ tw, const u64* __restrict__ tws, int log_n,
                               int S1, int log_rows) {
    extern __shared__ u64 sm[];
    const int n = 1 << log_n;
    const RowPtr rp = row_ptr(pb, blockIdx.x, n);
    const u64 q = primes[rp.prime].q;
    const u64* W = tw + (size_t)rp.prime * n;
    const u64* Ws = tws + (size_t)rp.prime * n;
    const int log_n2 = log_n - S1;
    const int r_base = blockIdx.y << log_rows;
    const int total = 1 << (log_rows + log_n2);
    u64* gp = rp.p + ((size_t)r_base << log_n2);
    for (int e = threadIdx.x; e < total; e += blockDim.x) sm[e] = gp[e];
    __syncthreads();
    const int half = total >> 1;
    const int log_half_row = log_n2 - 1;
    const int stages = log_n2;
    if (!INV) {
        for (int sp = 0; sp < stages; sp++) {
            const int log_tl = log_n2 - 1 - sp;
            for (int bi = threadIdx.x; bi < half; bi += blockDim.x) {
                int rl = bi >> log_half_row;
                int p = bi & ((1 << log_half_row) - 1);
                int g = p >> log_tl;
                int jj = p & ((1 << log_tl) - 1);
                int x0 = (g << (log_tl + 1)) + jj;
                int i0 = (rl << log_n2) + x0;
                int i1 = i0 + (1 << log_tl);
                int wi = (1 << (S1 + sp)) + ((r_base + rl) << sp) + g;
                u64 x = sm[i0];
                u64 y = mul_shoup(sm[i1], W[wi], Ws[wi], q);
                sm[i0] = add_mod(x, y, q);
                sm[i1] = sub_mod(x, y, q);
            }
            __syncthreads();
        }
    } else {
        for (int sp = stages - 1; sp >= 0; sp--) {
            const int log_tl = log_n2 - 1 - sp;
            for (int bi = threadIdx.x; bi < half; bi += blockDim.x) {
                int rl = bi >> log_half_row;
                int p = bi & ((1 << log_half_row) - 1);
                int g = p >> log_tl;
                int jj = p & ((1 << log_tl) - 1);
                int x0 = (g << (log_tl + 1)) + jj;
                int i0 = (rl << log_n2) + x0;
                int i1 = i0 + (1 << log_tl);
                int wi = (1 << (S1 + sp)) + ((r_base + rl) << sp) + g;
                u64 x = sm[i0];
                u64 y = sm[i1];
                sm[i0] = add_mod(x, y, q);
                sm[i1] = mul_shoup(sub_mod(x, y, q), W[wi], Ws[wi], q);
            }
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) gp[e] = sm[e];
}

template <bool INV>
void run_ntt(const Ctx& c, const PolyBatch& pb, cudaStream_t s) {
    const int rows = pb.rows();
    if (rows == 0) return;
    const u64* tw = INV ? c.d_ipsi : c.d_psi;
    const u64* tws = INV ? c.d_ipsi_s : c.d_psi_s;
    const int log_n = c.log_n;
    const double bytes = 16.0 * rows * ((size_t)1 << log_n);
    const int cls = INV ? K_NTT_INV : K_NTT_FWD;
    if (log_n <= 14) {
        LaunchScope _ls(c.prof, cls, bytes, s);
        size_t smem = sizeof(u64) << log_n;
        int threads = log_n >= 12 ? 512 : (1 << (log_n - 1));
        ntt_col_kernel<INV><<<dim3(rows, 1), threads, smem, s>>>(pb, c.d_primes, tw, tws, c.d_ninv,
                                                                 log_n, log_n, 0);
        CK(cudaGetLastError());
        return;
    }
    // two passes: N1 = 2^S1 rows of N2 = 2^(log_n - S1)
    const int S1 = log_n / 2;
    const int log_n2 = log_n - S1;
    const int log_cols = 12 - S1;          // tile = N1 x cols = 4096 elements
    const int log_rows = 12 - log_n2;      // tile = rows x N2 = 4096 elements
    const size_t smem = sizeof(u64) * kTile;
    dim3 gcol(rows, 1 << (log_n2 - log_cols));
    dim3 grow(rows, 1 << (S1 - log_rows));
    if (!INV) {
        {
            LaunchScope _ls(c.prof, cls, bytes, s);
            ntt_col_kernel<false><<<gcol, 256, smem, s>>>(pb, c.d_primes, tw, tws, c.d_ninv, log_n, S1, log_cols);
            CK(cudaGetLastError());
        }
        {
            LaunchScope _ls(c.prof, cls, bytes, s);
            ntt_row_kernel<false><<<grow, 256, smem, s>>>(pb, c.d_primes, tw, tws, log_n, S1, log_rows);
            CK(cudaGetLastError());
        }
    } else {
        {
            LaunchScope _ls(c.prof, cls, bytes, s);
            ntt_row_kernel<true><<<grow, 256, smem, s>>>(pb, c.d_primes, tw, tws, log_n, S1, log_rows);
            CK(cudaGetLastError());
        }
        {
            LaunchScope _ls(c.prof, cls, bytes, s);
            ntt_col_kernel<true><<<gcol, 256, smem, s>>>(pb, c.d_primes, tw, tws, c.d_ninv, log_n, S1, log_cols);
            CK(cudaGetLastError());
        }
    }
}

}  // namespace

void ntt_init() {
    const int max_smem = 227 * 1024;
    CK(cudaFuncSetAttribute(ntt_col_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    CK(cudaFuncSetAttribute(ntt_col_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    CK(cudaFuncSetAttribute(ntt_row_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    CK(cudaFuncSetAttribute(ntt_row_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
}

void ntt_forward(const Ctx& c, const PolyBatch& pb, cudaStream_t s) { run_ntt<false>(c, pb, s); }
void ntt_inverse(const Ctx& c, const PolyBatch& pb, cudaStream_t s) { run_ntt<true>(c, pb, s); }

}  // namespace fhe

// ntt.cu — batched negacyclic NTT over RNS limbs.
//
// Forward: Cooley-Tukey with merged psi powers (natural order in, bit-reversed
// order out): slot k holds a(psi^(2 brev(k) + 1)). Inverse: Gentleman-Sande
// (bit-reversed in, natural out) followed by the N^-1 scaling.
//
// Decomposition. A ring of N = N1 * N2 coefficients is viewed as N1 rows of
// N2: the first log2(N1) stages couple elements N2 apart (independent
// N1-point transforms on columns), the remaining stages couple elements inside
// one row (N2-point transforms with row-dependent twiddles). Rings up to 2^13
// run in one pass (N1 = N, one CTA per limb); larger rings in two passes.
//
// Each CTA holds a tile of R sub-transforms of M = 2^LOGM points in shared
// memory (element x of sub-transform q at x*(R+1) + q). Row passes read their
// twiddles from tables transposed to [stage][group][row], so that the R rows of a
// tile load consecutive entries. Every thread owns 8
// residues and runs three butterfly stages in registers between shared-memory
// exchanges (radix-8 blocking; the last block has 1-3 stages). Arithmetic is
// lazy in the style of Harvey (2014): forward values stay in [0, 4q), inverse
// values in [0, 2q); twiddle products use Shoup's precomputed quotient and no
// final correction; the last pass reduces to [0, q).
#include "ntt_tile.cuh"

namespace fhe {

namespace ntt_tile {
const char* const kNttTileNames[NTT_N_TILES] = {"r16b4", "r8b4", "r32b4", "r16b3"};
}

namespace {

using namespace ntt_tile;

template <bool INV>
void run_ntt(const Ctx& c, const PolyBatch& pb, cudaStream_t s) {
    const int rows = pb.rows();
    if (rows == 0) return;
    const double bytes = 16.0 * rows * ((size_t)1 << c.log_n);
    switch (c.log_n) {
        case 9: launch_tile<9, 9, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 10: launch_tile<10, 10, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 11: launch_tile<11, 11, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 12: launch_tile<12, 12, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        case 13: launch_tile<13, 13, 1, INV, 0, true, 3>(c, pb, 1, s, bytes); return;
        default: break;
    }
    switch (c.tune.ntt) {
        case NTT_R8B4: two_pass_r8b4(c, pb, INV, s, bytes); return;
        case NTT_R32B4: two_pass_r32b4(c, pb, INV, s, bytes); return;
        case NTT_R16B3: two_pass_r16b3(c, pb, INV, s, bytes); return;
        default: two_pass<INV, 16, nttc::kTileRB>(c, pb, s, bytes); return;
    }
}

}  // namespace

void ntt_init() {}

void ntt_forward(const Ctx& c, const PolyBatch& pb, cudaStream_t s) { run_ntt<false>(c, pb, s); }
void ntt_inverse(const Ctx& c, const PolyBatch& pb, cudaStream_t s) { run_ntt<true>(c, pb, s); }

}  // namespace fhe

// ntt_tiles.cu — the alternative tile shapes of the two-pass plain NTT (see ntt_tile.cuh), compiled in
// a translation unit of their own so that the library builds in parallel.
#include "ntt_tile.cuh"

namespace fhe {
namespace ntt_tile {

void two_pass_r8b4(const Ctx& c, const PolyBatch& pb, bool inv, cudaStream_t s, double bytes) {
    if (inv) two_pass<true, 8, 4>(c, pb, s, bytes);
    else two_pass<false, 8, 4>(c, pb, s, bytes);
}
void two_pass_r32b4(const Ctx& c, const PolyBatch& pb, bool inv, cudaStream_t s, double bytes) {
    if (inv) two_pass<true, 32, 4>(c, pb, s, bytes);
    else two_pass<false, 32, 4>(c, pb, s, bytes);
}
void two_pass_r16b3(const Ctx& c, const PolyBatch& pb, bool inv, cudaStream_t s, double bytes) {
    if (inv) two_pass<true, 16, 3>(c, pb, s, bytes);
    else two_pass<false, 16, 3>(c, pb, s, bytes);
}

}  // namespace ntt_tile
}  // namespace fhe

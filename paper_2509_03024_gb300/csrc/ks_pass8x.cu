// ks_pass8x.cu — the fused key-switch / rescale transforms with 8 rows or columns per tile and the
// register cap of LOOSE launch bounds, in a translation unit of their own so that the library builds
// in parallel (see ks_pass.cuh).
#include "ks_pass.cuh"

namespace fhe {
namespace ksp {

template <bool INV, int LOAD, int STORE>
void ks_transform_r8x(const Ctx& c, const KsRow* rows, int n_rows, const CombineArgs& ca, int cls, double bytes,
                     cudaStream_t s) {
    ks_transform_t<INV, LOAD, STORE, 8, true>(c, rows, n_rows, ca, cls, bytes, s);
}

#define INST(I, L, S)                                                                                   \
    template void ks_transform_r8x<I, L, S>(const Ctx&, const KsRow*, int, const CombineArgs&, int, double, \
                                            cudaStream_t);
KS_COMBOS(INST)
#undef INST

}  // namespace ksp
}  // namespace fhe

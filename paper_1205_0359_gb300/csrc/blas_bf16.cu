// PBF16 instantiations of the block update, basis initialisation and fused
// shift update kernels (kernel bodies in blas_impl.cuh).
#include "blas_impl.cuh"

namespace dsbcg {
namespace blas_impl {
BI_INSTANTIATE(PBF16)
}  // namespace blas_impl
}  // namespace dsbcg

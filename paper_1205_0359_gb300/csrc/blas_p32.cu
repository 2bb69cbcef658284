// P32 instantiations of the block update, basis initialisation and fused
// shift update kernels (kernel bodies in blas_impl.cuh).
#include "blas_impl.cuh"

namespace dsbcg {
namespace blas_impl {
BI_INSTANTIATE(P32)
}  // namespace blas_impl
}  // namespace dsbcg

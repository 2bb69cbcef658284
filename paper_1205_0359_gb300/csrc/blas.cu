// Launchers of the tall-skinny block kernels (kernel bodies in blas_impl.cuh):
// the Gram products here for every storage precision, the block update,
// basis initialisation and fused shift update dispatched to the
// per-precision translation units blas_<prec>.cu (compiled in parallel).
#include "blas_impl.cuh"

namespace dsbcg {
using namespace blas_impl;

size_t gram_partial_doubles(int nf_max) { return (size_t)ntiles_of(nf_max, 0) * 1024 * GSLOTS; }

int gram_blocks(size_t n, int nf_max) {
    if (nf_max <= 16) {
        // tiled kernel: a few CTAs per SM, each walking many row tiles
        size_t tiles_rows = (n + GR - 1) / GR;
        size_t nb = 152 * 2;
        if (nb > tiles_rows) nb = tiles_rows;
        return (int)(nb < 1 ? 1 : nb);
    }
    int tiles = ntiles_of(nf_max, 0);
    int nb = (152 * 8 + tiles - 1) / tiles;
    size_t maxb = (n + GT - 1) / GT;
    if ((size_t)nb > maxb) nb = (int)maxb;
    if (nb < 1) nb = 1;
    if (nb > 1024) nb = 1024;
    return nb;
}

void launch_gram(int prec, const void* X, const void* Y, size_t ld, size_t n, const Ctl* ctl, int nf_static,
                 int nf_max, int herm, int diag_yy, double* partials, int nblk, float hscale, cudaStream_t st,
                 int first_wait) {
    if (nf_max <= 16) {
        // shared-memory tiled kernel: one CTA per partial slot, nblk CTAs
        Ctl* c = const_cast<Ctl*>(ctl);
        switch (prec) {
            case P64: launch_gram_tile_t<P64>(X, Y, ld, n, c, nf_static, nf_max, herm, diag_yy, partials, nblk, hscale, st, first_wait); break;
            case P32: launch_gram_tile_t<P32>(X, Y, ld, n, c, nf_static, nf_max, herm, diag_yy, partials, nblk, hscale, st, first_wait); break;
            case PBF16: launch_gram_tile_t<PBF16>(X, Y, ld, n, c, nf_static, nf_max, herm, diag_yy, partials, nblk, hscale, st, first_wait); break;
            case PF16: launch_gram_tile_t<PF16>(X, Y, ld, n, c, nf_static, nf_max, herm, diag_yy, partials, nblk, hscale, st, first_wait); break;
        }
        return;
    }
    dim3 grid(ntiles_of(nf_max, herm), nblk);
    switch (prec) {
        case P64: gram_kernel<P64><<<grid, GT, 0, st>>>((const double2*)X, (const double2*)Y, ld, n, ctl, nf_static, nf_max, herm, diag_yy, partials, hscale); break;
        case P32: gram_kernel<P32><<<grid, GT, 0, st>>>((const float2*)X, (const float2*)Y, ld, n, ctl, nf_static, nf_max, herm, diag_yy, partials, hscale); break;
        case PBF16: gram_kernel<PBF16><<<grid, GT, 0, st>>>((const __nv_bfloat162*)X, (const __nv_bfloat162*)Y, ld, n, ctl, nf_static, nf_max, herm, diag_yy, partials, hscale); break;
        case PF16: gram_kernel<PF16><<<grid, GT, 0, st>>>((const __half2*)X, (const __half2*)Y, ld, n, ctl, nf_static, nf_max, herm, diag_yy, partials, hscale); break;
    }
}

void launch_gram_reduce(const double* partials, int nblk, int nf_max, int herm, int diag_yy, double2* G,
                        double* diag, const Ctl* ctl, int nf_static, int fp32, cudaStream_t st) {
    (void)nf_static;
    gram_reduce_kernel<<<ntiles_of(nf_max, herm), 64, 0, st>>>(partials, nblk, nf_max, herm, diag_yy, G, diag, ctl,
                                                                fp32);
}

#define EXTERN_P(P)                                                                                      \
    extern template void launch_bu_t<P>(void*, const void*, const void*, const void*, size_t, size_t, const Ctl*, \
                                        int, const void*, const void*, float, cudaStream_t);                 \
    extern template void launch_ug_t<P>(void*, const void*, const void*, const void*, size_t, size_t, const Ctl*, \
                                        int, const void*, const void*, double*, int, float, cudaStream_t);   \
    extern template void launch_ib_t<P>(void*, size_t, const void*, int, size_t, size_t, const double2*, int, \
                                        const Ctl*, int, float, cudaStream_t);                               \
    extern template void launch_vu_t<P>(void*, const void*, size_t, size_t, const Ctl*, int, const void*,     \
                                        float, cudaStream_t);                                                 \
    extern template void launch_sc_t<P>(const void*, size_t, int, size_t, void*, void*, size_t, size_t, int,  \
                                        int, Ctl*, int, int, int, const void*, const void*, const int*,       \
                                        float, cudaStream_t);
namespace blas_impl {
EXTERN_P(P64)
EXTERN_P(P32)
EXTERN_P(PBF16)
EXTERN_P(PF16)
}  // namespace blas_impl
#undef EXTERN_P

void launch_block_update(int prec, void* W, const void* Y, const void* Vk, const void* Vp, size_t ld, size_t n,
                         const Ctl* ctl, int nf_max, const void* coef_a, const void* coef_bh, float hscale,
                         cudaStream_t st) {
    switch (prec) {
        case P64: launch_bu_t<P64>(W, Y, Vk, Vp, ld, n, ctl, nf_max, coef_a, coef_bh, hscale, st); break;
        case P32: launch_bu_t<P32>(W, Y, Vk, Vp, ld, n, ctl, nf_max, coef_a, coef_bh, hscale, st); break;
        case PBF16: launch_bu_t<PBF16>(W, Y, Vk, Vp, ld, n, ctl, nf_max, coef_a, coef_bh, hscale, st); break;
        case PF16: launch_bu_t<PF16>(W, Y, Vk, Vp, ld, n, ctl, nf_max, coef_a, coef_bh, hscale, st); break;
    }
}

bool update_gram_fits(int prec, int nf_max) { return prec != P64 && nf_max <= UG_NF_MAX; }

void launch_update_gram(int prec, void* W, const void* Y, const void* Vk, const void* Vp, size_t ld, size_t n,
                        const Ctl* ctl, int nf_max, const void* coef_a, const void* coef_bh, double* partials,
                        int nblk, float hscale, cudaStream_t st) {
#define UG_ARGS W, Y, Vk, Vp, ld, n, ctl, nf_max, coef_a, coef_bh, partials, nblk, hscale, st
    switch (prec) {
        case P64: launch_ug_t<P64>(UG_ARGS); break;
        case P32: launch_ug_t<P32>(UG_ARGS); break;
        case PBF16: launch_ug_t<PBF16>(UG_ARGS); break;
        case PF16: launch_ug_t<PF16>(UG_ARGS); break;
    }
#undef UG_ARGS
}

void launch_init_basis(int prec, void* V1, size_t ldv, const void* B, int bprec, size_t ldb, size_t n,
                       const double2* S, int s_dd, const Ctl* ctl, int nf_in, float hscale, cudaStream_t st) {
    switch (prec) {
        case P64: launch_ib_t<P64>(V1, ldv, B, bprec, ldb, n, S, s_dd, ctl, nf_in, hscale, st); break;
        case P32: launch_ib_t<P32>(V1, ldv, B, bprec, ldb, n, S, s_dd, ctl, nf_in, hscale, st); break;
        case PBF16: launch_ib_t<PBF16>(V1, ldv, B, bprec, ldb, n, S, s_dd, ctl, nf_in, hscale, st); break;
        case PF16: launch_ib_t<PF16>(V1, ldv, B, bprec, ldb, n, S, s_dd, ctl, nf_in, hscale, st); break;
    }
}

void launch_v_update(int prec, void* Vnext, const void* W, size_t ld, size_t n, const Ctl* ctl, int nf_max,
                     const void* coefS, float hscale, cudaStream_t st) {
    switch (prec) {
        case P64: launch_vu_t<P64>(Vnext, W, ld, n, ctl, nf_max, coefS, hscale, st); break;
        case P32: launch_vu_t<P32>(Vnext, W, ld, n, ctl, nf_max, coefS, hscale, st); break;
        case PBF16: launch_vu_t<PBF16>(Vnext, W, ld, n, ctl, nf_max, coefS, hscale, st); break;
        case PF16: launch_vu_t<PF16>(Vnext, W, ld, n, ctl, nf_max, coefS, hscale, st); break;
    }
}

void launch_shift_chunk(int prec, const void* ring, size_t slot_elems, int R, size_t ld, void* P, void* X,
                        size_t ldw, size_t n, int s, int m, Ctl* ctl, int nf_max, int k0, int C, const void* coefU,
                        const void* coefL, const int* active, float hscale, cudaStream_t st) {
#define SC_ARGS ring, slot_elems, R, ld, P, X, ldw, n, s, m, ctl, nf_max, k0, C, coefU, coefL, active, hscale, st
    switch (prec) {
        case P64: launch_sc_t<P64>(SC_ARGS); break;
        case P32: launch_sc_t<P32>(SC_ARGS); break;
        case PBF16: launch_sc_t<PBF16>(SC_ARGS); break;
        case PF16: launch_sc_t<PF16>(SC_ARGS); break;
    }
#undef SC_ARGS
}

}  // namespace dsbcg

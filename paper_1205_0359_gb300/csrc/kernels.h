// Host-side launchers of the CUDA kernels (one translation unit each), used by
// the solver and the C ABI in solver.cu.  Field blocks are passed as a base
// pointer plus a field stride `ld` counted in complex elements; field f of a
// block starts at base + f * ld.  `prec` is a dsbcg::Prec value.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace dsbcg {

struct Geom {
    int L[4];         // Lx, Ly, Lz, Lt
    int V;            // sites
    int tap;          // antiperiodic in time
};

// ---- pack.cu --------------------------------------------------------------
// canonical complex128 [m][n] (device) <-> internal field block of precision prec
void launch_pack_fields(int prec, void* dst, size_t ld, const double2* src, int m, size_t V,
                        float hscale, cudaStream_t st);
void launch_unpack_fields(int prec, double2* dst, const void* src, size_t ld, int m, size_t V,
                          float hscale, cudaStream_t st);
// canonical complex128 [site][4][3][3] -> internal links [mu][9][site]
void launch_pack_links(int prec, void* dst, const double2* src, size_t V, cudaStream_t st);
// double-float fields (field f: FP32 hi plane at f * 2 ld, lo plane at
// f * 2 ld + ld, float2 words; internal order)
void launch_pack_pairs(float2* dst, size_t ld, const double2* src, int m, size_t V, cudaStream_t st);
void launch_unpack_pairs(double2* dst, const float2* src, size_t ld, int m, size_t V, cudaStream_t st);
void launch_accumulate_pairs(float2* y, size_t ld, const float2* x, size_t ldx, int m, size_t n, cudaStream_t st);
void launch_residual_pairs(float2* r, const float2* b, const float2* x, const float2* ax, size_t ld, int m,
                           size_t n, double sigma, double* partials, int nblk, cudaStream_t st);
// 12-real links of FP32 / 16-bit storage: rows 0, 1 of each link, [mu][e < 6][site]
void launch_pack_links12(int prec, void* dst, const double2* src, size_t V, cudaStream_t st);
// *flag |= 1 unless every link of the canonical field (nlinks 3x3 matrices)
// is in SU(3) to tol (orthonormal rows 0, 1; row 2 = conj(row 0 x row 1))
void launch_check_su3(const double2* src, size_t nlinks, double tol, int* flag, cudaStream_t st);
// counts NaN/Inf entries of a complex128 array into *flag (device int)
void launch_check_finite(const double2* p, size_t count, int* flag, cudaStream_t st);
// y_f += x_f (FP64 += work precision), fields listed by index arrays on the host
void launch_accumulate(int prec_x, double2* y, size_t ldy, const void* x, size_t ldx,
                       int m, size_t n, cudaStream_t st);
// FP64 internal fields -> FP32 internal fields (same element order), m fields of n
void launch_convert_64_32(float2* dst, size_t ldd, const double2* src, size_t lds, int m, size_t n,
                          cudaStream_t st);
// r_f = b_f - sigma * x_f - ax_f (all FP64), and per-field squared norms (partials)
void launch_residual(double2* r, const double2* b, const double2* x, const double2* ax,
                     size_t ld, int m, size_t n, double sigma, double* norm2_partials,
                     int nblk, cudaStream_t st);
int residual_blocks(size_t n);
void launch_reduce_cols(const double* partials, int nblk, int m, double* out, cudaStream_t st);
// Y (canonical complex128 [m][n]) = coef[0] B + sum_j coef[j+1] X_j from the
// high-precision internal fields (hp = P64 or PDD) B [m] and X [s][m];
// coef: device double[s + 1]
void launch_rational_combine(int hp, double2* Y, const void* B, const void* X, size_t ld, int m, int s,
                             const double* coef, size_t V, cudaStream_t st);
// canonical complex128 blocks [s][cnt]: L_j *= w_j (w: host double[s], s <= S_MAX)
void launch_scale_blocks(double2* L, int s, size_t cnt, const double* w, cudaStream_t st);
// out[e] = a0 g[e] + sum_j L_j[e] (g unused when a0 = 0)
void launch_sum_blocks(double2* out, const double2* L, int s, size_t cnt, const double2* g, double a0,
                       cudaStream_t st);
// out[j] = sum_e Re(conj(a_j[e]) b_j[e]) (device double[s]); partials: device double[s * nblk]
void launch_dot_re_blocks(const double2* a, const double2* b, int s, size_t cnt, double* partials, int nblk,
                          double* out, cudaStream_t st);

// ---- dslash.cu ------------------------------------------------------------
// out_f = D in_f (dag = 0) or D^H in_f = gamma_5 D gamma_5 in_f (dag = 1)
// for fields f < nf, where nf = ctl->mk when ctl != NULL, else nf_static.
// links12 (FP32 / 16-bit only, may be NULL): the same links in the 12-real
// layout of launch_pack_links12, used instead of `links` when given
void launch_dslash(int prec, void* out, const void* in, size_t ld, const void* links,
                   const Geom& g, double kappa, int dag, const Ctl* ctl,
                   int nf_static, int nf_max, float hscale, cudaStream_t st,
                   const void* links12 = nullptr, int max_ctas = 0);

// Half-lattice hopping term of the even-odd operator (every extent even; half
// fields of V / 2 sites, half index = canonical site / 2):
// out_f = alpha src_f + beta G5o H G5i in_f, out and src on `parity`, in on
// the other parity; src may be NULL (alpha ignored); G5i/G5o: gamma_5 on the
// input / on the hopping term's output when g5in / g5out.
void launch_dslash_half(int prec, void* out, const void* in, const void* src, size_t ld, const void* links,
                        const Geom& g, double alpha, double beta, int parity, int g5in, int g5out, const Ctl* ctl,
                        int nf_static, int nf_max, float hscale, cudaStream_t st);

// ---- blas.cu ----------------------------------------------------------------
int gram_blocks(size_t n, int nf_max);
// partial sums of X^H Y (nf x nf, FP64) per CTA; herm = 1 computes only the
// upper triangle of tiles (X == Y); diag_yy = 1 also sums |y_j|^2.
// first_wait >= 0 (a test hook; default -1 = off): the first shared-memory
// wait of each consumer warp of the staged kernel (nf_max <= 16) gives up
// after first_wait non-blocking tests and the kernel takes its timeout path
// (copies drained, ST_WAIT_TIMEOUT in ctl->status, NaN partials)
void launch_gram(int prec, const void* X, const void* Y, size_t ld, size_t n, const Ctl* ctl,
                 int nf_static, int nf_max, int herm, int diag_yy, double* partials, int nblk,
                 float hscale, cudaStream_t st, int first_wait = -1);
size_t gram_partial_doubles(int nf_max);
// reduce partials -> G (FP64, M_MAX x M_MAX, complex), diag (M_MAX)
void launch_gram_reduce(const double* partials, int nblk, int nf_max, int herm, int diag_yy,
                        double2* G, double* diag, const Ctl* ctl, int nf_static, int fp32,
                        cudaStream_t st);
// W = Y - V a - Vp b^H, coefficients from the device (work precision copies)
void launch_block_update(int prec, void* W, const void* Y, const void* Vk, const void* Vp,
                         size_t ld, size_t n, const Ctl* ctl, int nf_max,
                         const void* coef_a, const void* coef_bh, float hscale, cudaStream_t st);
// Block update fused with the Gram of its result: W as launch_block_update,
// and W^H W (hermitian, upper 4 x 4 tiles, no diagonal norms) as partials of
// nblk blocks in the Gram kernel's layout.  Reduced storages and block widths
// up to 12 (update_gram_fits); nblk is the Gram's block count for nf_max.
bool update_gram_fits(int prec, int nf_max);
void launch_update_gram(int prec, void* W, const void* Y, const void* Vk, const void* Vp, size_t ld, size_t n,
                        const Ctl* ctl, int nf_max, const void* coef_a, const void* coef_bh, double* partials,
                        int nblk, float hscale, cudaStream_t st);
// V1 = B S (B in precision bprec: FP64, or FP32 for reduced storage;
// storage-precision V1), S from the device m x m state (M_MAX x M_MAX, FP64,
// or double-float when s_dd)
void launch_init_basis(int prec, void* V1, size_t ldv, const void* B, int bprec, size_t ldb, size_t n,
                       const double2* S, int s_dd, const Ctl* ctl, int nf_in, float hscale, cudaStream_t st);
// V_{k+1} = W S (S from the step's QR, M_MAX-strided work-precision tile)
void launch_v_update(int prec, void* Vnext, const void* W, size_t ld, size_t n, const Ctl* ctl, int nf_max,
                     const void* coefS, float hscale, cudaStream_t st);
// shift update (the per-shift short recurrences, Sec. 3) over the block
// steps k0+1 .. min(k0 + C, last executed step): for every step in which
// shift j is active, X_j += P_j Ut_j and P_j <- V_{k+1} - P_j LhT_j, with P_j
// and X_j kept on chip across the steps.  ring: R slots of slot_elems
// storage-precision elements, slot k mod R holding V_k (V_1 is the search
// block of step 1).  coefU / coefL: per step slot (k - 1) mod C, s tiles of
// M_MAX x M_MAX work-precision entries; active: per step slot, s flags.  P
// and X hold s blocks of m fields of ldw elements (field-major).
void launch_shift_chunk(int prec, const void* ring, size_t slot_elems, int R, size_t ld, void* P, void* X,
                        size_t ldw, size_t n, int s, int m, Ctl* ctl, int nf_max, int k0, int C, const void* coefU,
                        const void* coefL, const int* active, float hscale, cudaStream_t st);

// ---- small.cu ---------------------------------------------------------------
struct SmallState;     // device m x m state (FP64 or double-float), defined in small.cu
size_t small_state_bytes(int s);
// sfp64: FP64 m x m scalar (else double-float); wprec: precision of the Gram
// partials and coefficient copies (P64 for FP64 storage, else P32)
void launch_small_init(SmallState* ss, Ctl* ctl, const double2* G0, const double* ref, int m, int s, double dtol,
                       int sfp64, cudaStream_t st);
// alpha_k from the Gram partials of V_k^H Y (+ coefficient tiles for the block update)
void launch_small_alpha(SmallState* ss, const Ctl* ctl, const double* partials, int nblk, int nf_max,
                        int wprec, int sfp64, void* coef_a, void* coef_bh, cudaStream_t st);
// W^H W from the Gram partials, pivoted QR with deflation, per-shift recurrences
void launch_small_step(SmallState* ss, Ctl* ctl, const double* partials, int nblk, int s, int m,
                       double dtol, const double* sigma_dev, const double* target_dev, int freeze,
                       int wprec, int sfp64, void* coefS_w, void* coefU_w, void* coefL_w, int* active,
                       int* conv_step, double* res_out, cudaStream_t st);
void launch_small_finish(SmallState* ss, Ctl* ctl, int s, int m, const int* active, cudaStream_t st);
const double2* small_state_S(const SmallState* ss);

// ---- force.cu ---------------------------------------------------------------
// dU += kappa * w * [F(a, b) + F(c, d)] over nf field pairs (internal FP64/FP32 fields)
void launch_force(int prec, double2* dU, const void* a, const void* b, const void* c,
                  const void* d, size_t ld, int nf, const double* w_per_field,
                  const Geom& g, double kappa, cudaStream_t st);

}  // namespace dsbcg

// Tall-skinny block kernels of the block Lanczos process (Sec. 3):
//   gram          G = X^H Y (nf x nf) for n x nf field blocks, FP64 result
//   block_update  W = A V_k - V_k alpha_k - V_{k-1} beta_k^H
//   update_gram   the block update fused with the Gram W^H W of its result
//   init_basis    V_1 = B S (FP64 right-hand sides -> storage precision)
//   v_update      V_{k+1} = W S
//   shift_chunk   for every active shift j and every block step of a chunk:
//                 X_j += P_j Ut_j,  P_j <- V_{k+1} - P_j Lh_j
//                 (the per-shift short recurrences of Sec. 3), P_j and X_j
//                 held on chip across the chunk.
// Fields are flat complex n-vectors (internal order); each thread owns rows.
// Accumulation is in the arithmetic precision of the storage (FP32 for
// FP32/BF16/FP16 fields), reduced across threads in that precision and
// across CTAs in FP64 in a fixed order (bitwise reproducible).
#pragma once
#include "kernels.h"

namespace dsbcg {
namespace blas_impl {

constexpr int GT = 256;             // gram threads per CTA
constexpr int GSLOTS = 36;          // 16 complex + 4 real per 4x4 tile

__host__ __device__ inline int ntiles_of(int nf, int herm) {
    int T = (nf + 3) / 4;
    return herm ? T * (T + 1) / 2 : T * T;
}
__device__ inline void tile_coords(int t, int T, int herm, int* ti, int* tj) {
    if (!herm) {
        *ti = t / T;
        *tj = t % T;
        return;
    }
    int i = 0;
    while (t >= T - i) {
        t -= T - i;
        ++i;
    }
    *ti = i;
    *tj = i + t;
}

template <int P>
__global__ void __launch_bounds__(GT) gram_kernel(const typename Tr<P>::S2* __restrict__ X,
                                                  const typename Tr<P>::S2* __restrict__ Y, size_t ld,
                                                  size_t n, const Ctl* __restrict__ ctl, int nf_static,
                                                  int nf_max, int herm, int diag_yy,
                                                  double* __restrict__ partials, float hscale) {
    using C = typename Tr<P>::C;
    using R = typename Tr<P>::R;
    const int T = (nf_max + 3) / 4;
    const int tile = blockIdx.x;
    const int nblk = gridDim.y;
    double* out = partials + ((size_t)tile * nblk + blockIdx.y) * GSLOTS;
    int nf = nf_static;
    if (ctl) {
        if (ctl->done) return;
        nf = ctl->mk;
    }
    int ti, tj;
    tile_coords(tile, T, herm, &ti, &tj);
    const int i0 = ti * 4, j0 = tj * 4;
    __shared__ R red[GT / 32][GSLOTS];
    if (i0 >= nf || j0 >= nf) {
        if (threadIdx.x < GSLOTS) {
            if constexpr (P == P64)
                out[threadIdx.x] = 0.0;
            else
                reinterpret_cast<float*>(partials)[((size_t)tile * nblk + blockIdx.y) * GSLOTS + threadIdx.x] = 0.f;
        }
        return;
    }
    const R inv = (P == PBF16 || P == PF16) ? R(1) / R(hscale) : R(1);
    const int ni = min(4, nf - i0), nj = min(4, nf - j0);
    const bool dodiag = diag_yy && (ti == tj);
    C acc[4][4];
    R yy[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        yy[a] = R(0);
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk(R(0), R(0));
    }
#pragma unroll 2
    for (size_t e = (size_t)blockIdx.y * GT + threadIdx.x; e < n; e += (size_t)nblk * GT) {
        C x[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            x[a] = a < ni ? Elem<P>::ld(X + (size_t)(i0 + a) * ld, e, inv) : mk(R(0), R(0));
            y[a] = a < nj ? Elem<P>::ld(Y + (size_t)(j0 + a) * ld, e, inv) : mk(R(0), R(0));
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) cfmac(acc[a][b], x[a], y[b]);
        if (dodiag) {
#pragma unroll
            for (int b = 0; b < 4; ++b) yy[b] = fma(y[b].x, y[b].x, fma(y[b].y, y[b].y, yy[b]));
        }
    }
    // warp reduction
    R v[GSLOTS];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            v[2 * (a * 4 + b)] = acc[a][b].x;
            v[2 * (a * 4 + b) + 1] = acc[a][b].y;
        }
#pragma unroll
    for (int b = 0; b < 4; ++b) v[32 + b] = yy[b];
#pragma unroll
    for (int q = 0; q < GSLOTS; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < GSLOTS; ++q) red[w][q] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < GSLOTS) {
        if constexpr (P == P64) {
            double sacc = 0.0;
#pragma unroll
            for (int ww = 0; ww < GT / 32; ++ww) sacc += red[ww][threadIdx.x];
            out[threadIdx.x] = sacc;
        } else {
            // reduced precision: FP32 partials (FP64 arithmetic is slow on
            // GB300 and the data carries FP32 accuracy), stored as floats in
            // the same slot positions
            float sacc = 0.f;
#pragma unroll
            for (int ww = 0; ww < GT / 32; ++ww) sacc += red[ww][threadIdx.x];
            reinterpret_cast<float*>(partials)[((size_t)tile * nblk + blockIdx.y) * GSLOTS + threadIdx.x] = sacc;
        }
    }
}

// G[i][j] (M_MAX x M_MAX) from the per-CTA partials (FP32 words when fp32,
// as written by the reduced-precision Gram kernels); one CTA per tile
static __global__ void gram_reduce_kernel(const double* __restrict__ partials, int nblk, int nf_max, int herm,
                                   int diag_yy, double2* __restrict__ G, double* __restrict__ diag,
                                   const Ctl* __restrict__ ctl, int fp32) {
    if (ctl && ctl->done) return;
    const int T = (nf_max + 3) / 4;
    const int tile = blockIdx.x;
    int ti, tj;
    tile_coords(tile, T, herm, &ti, &tj);
    const int q = threadIdx.x;
    if (q >= GSLOTS) return;
    double s = 0.0;
    if (fp32) {
        const float* p = reinterpret_cast<const float*>(partials) + (size_t)tile * nblk * GSLOTS;
        for (int b = 0; b < nblk; ++b) s += (double)p[(size_t)b * GSLOTS + q];
    } else {
        const double* p = partials + (size_t)tile * nblk * GSLOTS;
        for (int b = 0; b < nblk; ++b) s += p[(size_t)b * GSLOTS + q];
    }
    if (q < 32) {
        int a = (q >> 1) >> 2, bb = (q >> 1) & 3;
        int i = ti * 4 + a, j = tj * 4 + bb;
        if (i < M_MAX && j < M_MAX) {
            if (q & 1) {
                G[i * M_MAX + j].y = s;
                if (herm && ti != tj) G[j * M_MAX + i].y = -s;
            } else {
                G[i * M_MAX + j].x = s;
                if (herm && ti != tj) G[j * M_MAX + i].x = s;
            }
        }
    } else if (diag_yy && ti == tj) {
        int j = tj * 4 + (q - 32);
        if (j < M_MAX) diag[j] = s;
    }
}

// ---------------------------------------------------------------------------
template <int P, int NF>
__global__ void __launch_bounds__(256) block_update_kernel(typename Tr<P>::S2* __restrict__ W,
                                                           const typename Tr<P>::S2* __restrict__ Y,
                                                           const typename Tr<P>::S2* __restrict__ Vk,
                                                           const typename Tr<P>::S2* __restrict__ Vp,
                                                           size_t ld, size_t n, const Ctl* __restrict__ ctl,
                                                           const typename Tr<P>::C* __restrict__ ca,
                                                           const typename Tr<P>::C* __restrict__ cbh,
                                                           float hscale) {
    using C = typename Tr<P>::C;
    using R = typename Tr<P>::R;
    if (ctl->done) return;
    const int mk_ = ctl->mk, mp = (ctl->k > 1) ? ctl->mprev : 0;
    __shared__ C sa[NF * NF], sb[NF * NF];
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) {
        int a = t / NF, b = t % NF;
        sa[t] = ca[a * M_MAX + b];
        sb[t] = cbh[a * M_MAX + b];
    }
    __syncthreads();
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const R inv = (P == PBF16 || P == PF16) ? R(1) / R(hscale) : R(1);
    const R scl = (P == PBF16 || P == PF16) ? R(hscale) : R(1);
    // every operand of the row is loaded before any arithmetic
    C v[NF], vp[NF], y[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
        v[a] = a < mk_ ? Elem<P>::ld(Vk + (size_t)a * ld, e, inv) : mk(R(0), R(0));
        vp[a] = a < mp ? Elem<P>::ld(Vp + (size_t)a * ld, e, inv) : mk(R(0), R(0));
        y[a] = a < mk_ ? Elem<P>::ld(Y + (size_t)a * ld, e, inv) : mk(R(0), R(0));
    }
#pragma unroll
    for (int b = 0; b < NF; ++b) {
        if (b < mk_) {
            C w = y[b];
#pragma unroll
            for (int a = 0; a < NF; ++a) {
                cfms(w, v[a], sa[a * NF + b]);
                cfms(w, vp[a], sb[a * NF + b]);
            }
            Elem<P>::st(W + (size_t)b * ld, e, w, scl);
        }
    }
}

// Block update fused with the Gram W^H W of its result, for block widths up
// to 12.  The grid (the Gram's nblk CTAs of UG_ROWS threads) strides over
// tiles of UG_ROWS rows.  Per tile every thread first forms W for its row
// exactly as block_update_kernel does and stores it to global memory and, in
// the storage precision (the values a separate Gram launch would read), to
// shared memory.  After a barrier, warp w accumulates the upper 4 x 4 tile w
// of W^H W over the tile's rows, lanes striding the rows, in the Gram
// kernel's operation order.  At the end each tile's warp writes its fixed-
// order warp reduction to the partials in the Gram kernel's layout, so the
// QR kernel that follows reads them unchanged.  W therefore crosses HBM once
// per step instead of twice, and the step has one launch less.
constexpr int UG_ROWS = 256;
constexpr int UG_NF_MAX = 12;          // upper tiles (6 at width 12) <= warps (8)

template <int P, int NF>
__global__ void __launch_bounds__(UG_ROWS, 2) update_gram_kernel(
    typename Tr<P>::S2* __restrict__ W, const typename Tr<P>::S2* __restrict__ Y,
    const typename Tr<P>::S2* __restrict__ Vk, const typename Tr<P>::S2* __restrict__ Vp, size_t ld, size_t n,
    const Ctl* __restrict__ ctl, int nf_max, const typename Tr<P>::C* __restrict__ ca,
    const typename Tr<P>::C* __restrict__ cbh, double* __restrict__ partials, float hscale) {
    static_assert(NF <= UG_NF_MAX, "fused update and Gram: widths up to 12");
    using C = typename Tr<P>::C;
    using R = typename Tr<P>::R;
    using SE = typename Tr<P>::S2;
    if (ctl->done) return;
    const int mk_ = ctl->mk, mp = (ctl->k > 1) ? ctl->mprev : 0;
    __shared__ C sa[NF * NF], sb[NF * NF];
    extern __shared__ __align__(16) unsigned char ug_smem[];
    SE* sW = reinterpret_cast<SE*>(ug_smem);                // [NF][UG_ROWS]
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) {
        const int a = t / NF, b = t % NF;
        sa[t] = ca[a * M_MAX + b];
        sb[t] = cbh[a * M_MAX + b];
    }
    const R inv = (P == PBF16 || P == PF16) ? R(1) / R(hscale) : R(1);
    const R scl = (P == PBF16 || P == PF16) ? R(hscale) : R(1);
    const int T = (nf_max + 3) / 4;
    const int ntl = T * (T + 1) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int ti = 0, tj = 0;
    if (warp < ntl) tile_coords(warp, T, 1, &ti, &tj);
    const int i0 = ti * 4, j0 = tj * 4;
    const int ni = max(0, min(4, mk_ - i0)), nj = max(0, min(4, mk_ - j0));
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = mk(R(0), R(0));
    __syncthreads();
    const size_t ntr = (n + UG_ROWS - 1) / UG_ROWS;
    for (size_t q = blockIdx.x; q < ntr; q += gridDim.x) {
        const size_t e = q * UG_ROWS + threadIdx.x;
        if (e < n) {
            // every operand of the row is loaded before any arithmetic
            C v[NF], vp[NF], y[NF];
#pragma unroll
            for (int a = 0; a < NF; ++a) {
                v[a] = a < mk_ ? Elem<P>::ld(Vk + (size_t)a * ld, e, inv) : mk(R(0), R(0));
                vp[a] = a < mp ? Elem<P>::ld(Vp + (size_t)a * ld, e, inv) : mk(R(0), R(0));
                y[a] = a < mk_ ? Elem<P>::ld(Y + (size_t)a * ld, e, inv) : mk(R(0), R(0));
            }
#pragma unroll
            for (int b = 0; b < NF; ++b) {
                if (b < mk_) {
                    C w = y[b];
#pragma unroll
                    for (int a = 0; a < NF; ++a) {
                        cfms(w, v[a], sa[a * NF + b]);
                        cfms(w, vp[a], sb[a * NF + b]);
                    }
                    Elem<P>::st(W + (size_t)b * ld, e, w, scl);
                    Elem<P>::st(sW, (size_t)b * UG_ROWS + threadIdx.x, w, scl);
                }
            }
        }
        __syncthreads();
        if (warp < ntl && ni > 0 && nj > 0) {
            const int rows = (int)((n - q * UG_ROWS) < (size_t)UG_ROWS ? (n - q * UG_ROWS) : (size_t)UG_ROWS);
            for (int r = lane; r < rows; r += 32) {
                C x[4], yv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    x[a] = a < ni ? Elem<P>::ld(sW, (size_t)(i0 + a) * UG_ROWS + r, inv) : mk(R(0), R(0));
                    yv[a] = a < nj ? Elem<P>::ld(sW, (size_t)(j0 + a) * UG_ROWS + r, inv) : mk(R(0), R(0));
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) cfmac(acc[a][c], x[a], yv[c]);
            }
        }
        __syncthreads();
    }
    if (warp < ntl) {
        // fixed-order warp reduction of the 36 slots (no diagonal norms), one write per slot
        R v[GSLOTS];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                v[2 * (a * 4 + c)] = acc[a][c].x;
                v[2 * (a * 4 + c) + 1] = acc[a][c].y;
            }
#pragma unroll
        for (int c = 0; c < 4; ++c) v[32 + c] = R(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int qq = 0; qq < GSLOTS; ++qq) v[qq] += __shfl_down_sync(0xffffffffu, v[qq], o);
        if (lane == 0) {
            const size_t base = ((size_t)warp * gridDim.x + blockIdx.x) * GSLOTS;
#pragma unroll
            for (int qq = 0; qq < GSLOTS; ++qq) {
                if constexpr (P == P64)
                    partials[base + qq] = (double)v[qq];
                else
                    reinterpret_cast<float*>(partials)[base + qq] = (float)v[qq];
            }
        }
    }
}

// V1 = B S: B FP64 (nf_in fields), S FP64 M_MAX x M_MAX, V1 storage precision (ctl->mk fields)
template <int P, int NF, int PIN>
__global__ void __launch_bounds__(256) init_basis_kernel(typename Tr<P>::S2* __restrict__ V1, size_t ldv,
                                                         const typename Tr<PIN>::S2* __restrict__ B, size_t ldb,
                                                         size_t n, const double2* __restrict__ S, int s_dd,
                                                         const Ctl* __restrict__ ctl, int nf_in, float hscale) {
    // the product is formed in the arithmetic precision of the storage: FP64
    // for FP64 fields, FP32 otherwise (the result is stored in FP32 or less);
    // S is read once per CTA
    using R = typename Tr<P>::R;
    using C = typename Tr<P>::C;
    const int m1 = ctl->mk;
    __shared__ C ss[NF * NF];
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) {
        if (!s_dd) {
            const double2 v = S[(t / NF) * M_MAX + (t % NF)];
            ss[t] = mk(R(v.x), R(v.y));
        } else {
            // double-float m x m state (re.hi, re.lo, im.hi, im.lo): the hi
            // words are the FP32 values (reduced storage only)
            const float4 v = reinterpret_cast<const float4*>(S)[(t / NF) * M_MAX + (t % NF)];
            ss[t] = mk(R(v.x), R(v.z));
        }
    }
    __syncthreads();
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const R scl = (P == PBF16 || P == PF16) ? R(hscale) : R(1);
    C b[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
        if (a < nf_in) {
            const auto v = B[(size_t)a * ldb + e];
            b[a] = mk(R(v.x), R(v.y));
        } else {
            b[a] = mk(R(0), R(0));
        }
    }
#pragma unroll
    for (int c = 0; c < NF; ++c) {
        if (c < m1) {
            C acc = mk(R(0), R(0));
#pragma unroll
            for (int a = 0; a < NF; ++a) cfma(acc, b[a], ss[a * NF + c]);
            Elem<P>::st(V1 + (size_t)c * ldv, e, acc, scl);
        }
    }
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies and bounded mbarrier waits (the staged Gram).
// Every mbarrier wait is bounded; on timeout the kernel records an error in
// the control block, drains its own copies and returns.
constexpr int ST_WAIT_TIMEOUT = -3;        // reported to the host as DSBCG_ERR_CUDA
constexpr long MBAR_SPIN_LIMIT = 1L << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// one non-blocking test of the phase
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long it = 0; it < MBAR_SPIN_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// bounded wait that also gives up as soon as *abort is set (by another warp
// of the CTA whose own wait gave up)
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, const volatile int* abort) {
    for (long it = 0; it < MBAR_SPIN_LIMIT; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Gram product G = X^H Y (nf x nf, nf <= 16) with row tiles staged in shared
// memory.  Each CTA walks row tiles of GR rows (tile q, q + gridDim.x, ...)
// through a ring of GNST staging buffers.  One producer warp fills a buffer
// with the GR-element run of every field of X (and of Y unless X == Y) by
// bulk asynchronous copies, completion on the buffer's "full" mbarrier; the
// consumer warps, one per 4 x 4 tile of the Gram matrix with lanes over rows,
// accumulate in registers (FP32, FP64 for FP64 fields) and release the buffer
// on its "empty" mbarrier.  No block-wide barrier inside the loop.  A
// fixed-order warp reduction at the end writes the CTA's partial sums in the
// layout the m x m kernels reduce ([tile][CTA][36]).  Every wait is bounded;
// on timeout the CTA drains its copies, flags the control block (if any) and
// writes NaN partials.
constexpr int GR = 128;              // rows per staged tile
// staging buffers per CTA: 4 (3 for FP64 fields, to stay within shared memory)
template <int P>
constexpr int gram_stages() { return P == P64 ? 3 : 4; }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int P>
__global__ void __launch_bounds__(544) gram_tile_kernel(const typename Tr<P>::S2* __restrict__ X,
                                                        const typename Tr<P>::S2* __restrict__ Y, size_t ld,
                                                        size_t n, Ctl* __restrict__ ctl, int nf_static, int nf_max,
                                                        int herm, int diag_yy, double* __restrict__ partials,
                                                        float hscale, int first_wait) {
    using C = typename Tr<P>::C;
    using R = typename Tr<P>::R;
    using SE = typename Tr<P>::S2;
    constexpr int GNST = gram_stages<P>();
    int nf = nf_static;
    if (ctl) {
        if (ctl->done) return;
        nf = ctl->mk;
    }
    extern __shared__ __align__(128) unsigned char g_smem[];
    const bool same = (X == Y);
    const size_t stage = (size_t)(same ? nf_max : 2 * nf_max) * GR;   // elements per staging buffer
    SE* buf0 = reinterpret_cast<SE*>(g_smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(g_smem + GNST * stage * sizeof(SE));
    uint64_t* empty = full + GNST;
    const int T = (nf_max + 3) / 4;
    const int ncons = ntiles_of(nf_max, herm);        // consumer warps; warp ncons produces
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t ntr = (n + GR - 1) / GR;
    const size_t G = gridDim.x;

    // set by a consumer warp whose wait gave up: the producer stops waiting
    // for buffers that will not be released and drains its copies
    __shared__ int aborted;
    if (threadIdx.x == 0) {
        for (int b = 0; b < GNST; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], ncons);
        }
        mbar_fence_init();
        aborted = 0;
    }
    __syncthreads();
    bool ok = true;
    if (warp == ncons) {
        // producer
        if (lane == 0) {
            size_t it = 0;
            for (size_t q = blockIdx.x; q < ntr; q += G, ++it) {
                const int b = (int)(it % GNST);
                if (it >= GNST && !mbar_wait_or_abort(&empty[b], (uint32_t)((it / GNST - 1) & 1), &aborted)) {
                    ok = false;
                    break;
                }
                const size_t r0 = q * GR;
                const int rows = (int)((n - r0) < (size_t)GR ? (n - r0) : (size_t)GR);
                const uint32_t tb = (uint32_t)rows * sizeof(SE);
                SE* d = buf0 + (size_t)b * stage;
                mbar_expect_tx(&full[b], (uint32_t)(same ? nf : 2 * nf) * tb);
                for (int f = 0; f < nf; ++f) {
                    bulk_g2s(d + (size_t)f * GR, X + (size_t)f * ld + r0, tb, &full[b]);
                    if (!same) bulk_g2s(d + (size_t)(nf_max + f) * GR, Y + (size_t)f * ld + r0, tb, &full[b]);
                }
            }
            // every issued copy lands before the CTA may exit (the last
            // GNST fills; earlier ones were waited on through "empty")
            const size_t first = it > GNST ? it - GNST : 0;
            for (size_t k = first; k < it; ++k)
                if (!mbar_wait(&full[k % GNST], (uint32_t)((k / GNST) & 1))) ok = false;
        }
    } else {
        // consumers
        int ti, tj;
        tile_coords(warp, T, herm, &ti, &tj);
        const int i0 = ti * 4, j0 = tj * 4;
        const int ni = max(0, min(4, nf - i0)), nj = max(0, min(4, nf - j0));
        const bool dodiag = diag_yy && ti == tj;
        const R inv = (P == PBF16 || P == PF16) ? R(1) / R(hscale) : R(1);
        C acc[4][4];
        R yy[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            yy[a] = R(0);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = mk(R(0), R(0));
        }
        size_t it = 0;
        for (size_t q = blockIdx.x; q < ntr; q += G, ++it) {
            const int b = (int)(it % GNST);
            bool got;
            if (it == 0 && first_wait >= 0) {
                // test hook (first_wait >= 0): the first wait gives up after
                // first_wait non-blocking tests, taking the timeout path below
                got = false;
                for (int k = 0; k < first_wait && !got; ++k) got = mbar_test(&full[b], 0u);
            } else {
                got = mbar_wait(&full[b], (uint32_t)((it / GNST) & 1));
            }
            if (!got) {
                ok = false;
                if (lane == 0) atomicExch(&aborted, 1);
                break;
            }
            const int rows = (int)((n - q * GR) < (size_t)GR ? (n - q * GR) : (size_t)GR);
            const SE* sx = buf0 + (size_t)b * stage;
            const SE* sy = same ? sx : sx + (size_t)nf_max * GR;
            if (ni > 0 && nj > 0) {
                for (int r = lane; r < rows; r += 32) {
                    C x[4], y[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        x[a] = a < ni ? Elem<P>::ld(sx, (size_t)(i0 + a) * GR + r, inv) : mk(R(0), R(0));
                        y[a] = a < nj ? Elem<P>::ld(sy, (size_t)(j0 + a) * GR + r, inv) : mk(R(0), R(0));
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int c = 0; c < 4; ++c) cfmac(acc[a][c], x[a], y[c]);
                    if (dodiag) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) yy[c] = fma(y[c].x, y[c].x, fma(y[c].y, y[c].y, yy[c]));
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
        }
        // fixed-order warp reduction of the 36 slots, then one write per slot
        R v[GSLOTS];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                v[2 * (a * 4 + c)] = acc[a][c].x;
                v[2 * (a * 4 + c) + 1] = acc[a][c].y;
            }
#pragma unroll
        for (int c = 0; c < 4; ++c) v[32 + c] = yy[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int qq = 0; qq < GSLOTS; ++qq) v[qq] += __shfl_down_sync(0xffffffffu, v[qq], o);
        if (lane == 0) {
            const size_t base = ((size_t)warp * G + blockIdx.x) * GSLOTS;
#pragma unroll
            for (int qq = 0; qq < GSLOTS; ++qq) {
                if constexpr (P == P64)
                    partials[base + qq] = (double)v[qq];
                else
                    reinterpret_cast<float*>(partials)[base + qq] = (float)v[qq];
            }
        }
    }
    if (__syncthreads_or(!ok)) {
        // a wait gave up: poison every partial of this CTA
        if (threadIdx.x == 0 && ctl) atomicCAS(&ctl->status, 0, ST_WAIT_TIMEOUT);
        for (int t = threadIdx.x; t < ncons * GSLOTS; t += blockDim.x) {
            const size_t at = ((size_t)(t / GSLOTS) * G + blockIdx.x) * GSLOTS + t % GSLOTS;
            if constexpr (P == P64)
                partials[at] = __longlong_as_double(0x7ff8000000000000LL);
            else
                reinterpret_cast<float*>(partials)[at] = __int_as_float(0x7fc00000);
        }
    }
}

template <int P>
void launch_gram_tile_t(const void* X, const void* Y, size_t ld, size_t n, Ctl* ctl, int nf_static, int nf_max,
                        int herm, int diag_yy, double* partials, int nblk, float hscale, cudaStream_t st,
                        int first_wait) {
    using SE = typename Tr<P>::S2;
    constexpr int GNST = gram_stages<P>();
    const int npb = ntiles_of(nf_max, herm);
    const int nbuf_fields = (X == Y) ? nf_max : 2 * nf_max;
    const size_t smem = GNST * (size_t)nbuf_fields * GR * sizeof(SE) + 2 * GNST * sizeof(uint64_t);
    static std::atomic<unsigned long long> devs{0};
    max_dyn_smem_once(gram_tile_kernel<P>, (int)(GNST * 2 * 16 * GR * sizeof(SE) + 2 * GNST * sizeof(uint64_t)), devs);
    gram_tile_kernel<P><<<nblk, (npb + 1) * 32, smem, st>>>((const SE*)X, (const SE*)Y, ld, n, ctl, nf_static, nf_max, herm,
                                                      diag_yy, partials, hscale, first_wait);
}

// V_{k+1} = W S (one thread per row; W and V in the storage precision)
template <int P, int NF>
__global__ void __launch_bounds__(256) v_update_kernel(typename Tr<P>::S2* __restrict__ Vn,
                                                       const typename Tr<P>::S2* __restrict__ W, size_t ld,
                                                       size_t n, const Ctl* __restrict__ ctl,
                                                       const typename Tr<(P == P64 ? P64 : P32)>::C* __restrict__ cS,
                                                       float hscale) {
    constexpr int PW = (P == P64) ? P64 : P32;
    using C = typename Tr<PW>::C;
    using R = typename Tr<PW>::R;
    if (ctl->done) return;
    const int mk_ = ctl->mk, mn = ctl->mnext;
    __shared__ C sS[NF * NF];
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) sS[t] = cS[(t / NF) * M_MAX + (t % NF)];
    __syncthreads();
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float inv = (P == PBF16 || P == PF16) ? 1.f / hscale : 1.f;
    const float scl = (P == PBF16 || P == PF16) ? hscale : 1.f;
    C w[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
        if (a < mk_) {
            auto q = Elem<P>::ld(W + (size_t)a * ld, e, inv);
            w[a] = mk(R(q.x), R(q.y));
        } else {
            w[a] = mk(R(0), R(0));
        }
    }
#pragma unroll
    for (int c = 0; c < NF; ++c) {
        if (c < mn) {
            C acc = mk(R(0), R(0));
#pragma unroll
            for (int a = 0; a < NF; ++a) cfma(acc, w[a], sS[a * NF + c]);
            Elem<P>::st(Vn + (size_t)c * ld, e, mk((typename Tr<P>::R)acc.x, (typename Tr<P>::R)acc.y), scl);
        }
    }
}

// Per-shift update over a chunk of block steps k0+1 .. k0+C, one thread per
// (row, shift): for each step k of the chunk in which shift j is active,
//     X_j += P_j Ut_j^(k),   P_j <- V_{k+1} - P_j Lh_j^(k)
// with P_j and X_j held in registers across the chunk, so that they cross
// HBM once per chunk instead of once per step.  The arithmetic per element
// is the per-step update's, in the same order; only the round trips of P_j
// and X_j through memory (in their own precision, so without rounding) are
// gone.  Inputs: the basis ring (slot k mod R holds V_k; V_1 is the search
// block of step 1), the per-step coefficient tiles of every shift (slot
// (k - 1) mod C), the per-step active flags and, in the control block, the
// block widths of the last 16 steps.  Steps after the solve's last executed
// step are skipped, so one launch at the end of a batch also closes a
// shorter chunk.  One CTA per (row tile, shift), shift index fastest so that
// the CTAs reading the same V rows run together and share them through L2.
template <int NF, int PW>
__host__ __device__ constexpr size_t sc_smem_bytes() {
    return 4 * (size_t)NF * NF * sizeof(typename Tr<PW>::C);
}

template <int P, int PW, int NF, int ROWS>
__global__ void __launch_bounds__(ROWS, (NF <= 12 && PW == P32) ? 4 : 1) shift_chunk_kernel(
    const typename Tr<P>::S2* __restrict__ ring, size_t slot_elems, int R, size_t ld,
    typename Tr<PW>::S2* __restrict__ Pb, typename Tr<PW>::S2* __restrict__ Xb, size_t ldw, size_t n, int s, int m,
    Ctl* __restrict__ ctl, int k0, int C, const typename Tr<PW>::C* __restrict__ cU,
    const typename Tr<PW>::C* __restrict__ cL, const int* __restrict__ act, float hscale) {
    using C2 = typename Tr<PW>::C;
    using R2 = typename Tr<PW>::R;
    using SE = typename Tr<P>::S2;
    const int j = (int)(blockIdx.x % (unsigned)s);
    const int kend = min(k0 + C, ctl->last_step);
    if (kend <= k0 || !act[(size_t)(k0 % C) * s + j]) return;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    C2* sU = reinterpret_cast<C2*>(sc_smem);            // [2][NF * NF]
    C2* sL = sU + 2 * NF * NF;                           // [2][NF * NF]
    const int tid = threadIdx.x;
    const size_t e0 = (size_t)(blockIdx.x / (unsigned)s) * ROWS;
    const bool ok = e0 + tid < n;
    const size_t e = e0 + (ok ? tid : 0);
    const float inv = (P == PBF16 || P == PF16) ? 1.f / hscale : 1.f;
    auto ldv = [&](int k, int c) -> C2 {
        const auto q = Elem<P>::ld(ring + (size_t)(k % R) * slot_elems + (size_t)c * ld, e, inv);
        return mk(R2(q.x), R2(q.y));
    };
    const size_t tile = (size_t)M_MAX * M_MAX;
    typename Tr<PW>::S2* Pj = Pb + (size_t)j * m * ldw;
    typename Tr<PW>::S2* Xj = Xb + (size_t)j * m * ldw;
    int mk_ = ctl->hmk[k0 & (CTL_HIST - 1)];
    C2 t[NF], x[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
        if (a < mk_) t[a] = (k0 == 0) ? ldv(1, a) : Pj[(size_t)a * ldw + e];
        else t[a] = mk(R2(0), R2(0));
        x[a] = a < m ? Xj[(size_t)a * ldw + e] : mk(R2(0), R2(0));
    }
    int mn = mk_;
    int k = k0 + 1;
    for (; k <= kend; ++k) {
        const int q = (k - 1) % C;
        if (!act[(size_t)q * s + j]) break;
        mn = ctl->hmn[(k - 1) & (CTL_HIST - 1)];
        // this step's tiles into buffer b; the sync also orders the reads of
        // step k - 2 (same buffer) before the writes
        const int b = (k - k0) & 1;
        C2* bU = sU + b * NF * NF;
        C2* bL = sL + b * NF * NF;
        const C2* gU = cU + ((size_t)q * s + j) * tile;
        const C2* gL = cL + ((size_t)q * s + j) * tile;
        for (int u = tid; u < NF * NF; u += ROWS) {
            bU[u] = gU[(u / NF) * M_MAX + u % NF];
            bL[u] = gL[(u / NF) * M_MAX + u % NF];
        }
        __syncthreads();
        // X_j += P_j Ut_j
#pragma unroll
        for (int a = 0; a < NF; ++a) {
#pragma unroll
            for (int i = 0; i < NF; i += 2) {
                C2 u0, u1;
                if constexpr (sizeof(C2) == 8) {
                    const float4 u2 = *reinterpret_cast<const float4*>(&bU[a * NF + i]);
                    u0 = mk(R2(u2.x), R2(u2.y));
                    u1 = mk(R2(u2.z), R2(u2.w));
                } else {
                    u0 = bU[a * NF + i];
                    u1 = bU[a * NF + i + 1];
                }
                cfma(x[i], t[a], u0);
                cfma(x[i + 1], t[a], u1);
            }
        }
        // P_j <- V_{k+1} - P_j Lh_j
        C2 pn[NF];
#pragma unroll
        for (int c = 0; c < NF; ++c) pn[c] = c < mn ? ldv(k + 1, c) : mk(R2(0), R2(0));
#pragma unroll
        for (int a = 0; a < NF; ++a) {
#pragma unroll
            for (int c = 0; c < NF; c += 2) {
                C2 l0, l1;
                if constexpr (sizeof(C2) == 8) {
                    const float4 l2 = *reinterpret_cast<const float4*>(&bL[a * NF + c]);
                    l0 = mk(R2(l2.x), R2(l2.y));
                    l1 = mk(R2(l2.z), R2(l2.w));
                } else {
                    l0 = bL[a * NF + c];
                    l1 = bL[a * NF + c + 1];
                }
                cfms(pn[c], t[a], l0);
                cfms(pn[c + 1], t[a], l1);
            }
        }
#pragma unroll
        for (int c = 0; c < NF; ++c) t[c] = c < mn ? pn[c] : mk(R2(0), R2(0));
    }
    if (ok) {
#pragma unroll
        for (int i = 0; i < NF; ++i)
            if (i < m) Xj[(size_t)i * ldw + e] = x[i];
#pragma unroll
        for (int c = 0; c < NF; ++c)
            if (c < mn) Pj[(size_t)c * ldw + e] = t[c];
    }
    if (blockIdx.x < (unsigned)s && tid == 0) {
        // work-precision fields moved: P_j (or V_1) and X_j in, X_j and P_j out
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->f_shift_w),
                  (unsigned long long)(mk_ + 2 * m + mn));
    }
}

inline int nf_bucket(int nf) { return nf <= 4 ? 4 : nf <= 8 ? 8 : nf <= 12 ? 12 : nf <= 16 ? 16 : nf <= 24 ? 24 : 32; }


// ---- per-precision host dispatch (defined here, instantiated in blas_<prec>.cu)
#define BI_DISPATCH_NF(nf, MACRO) \
    switch (nf_bucket(nf)) {       \
        case 4: MACRO(4); break;      \
        case 8: MACRO(8); break;      \
        case 12: MACRO(12); break;    \
        case 16: MACRO(16); break;    \
        case 24: MACRO(24); break;    \
        default: MACRO(32); break;    \
    }

template <int P>
void launch_bu_t(void* W, const void* Y, const void* Vk, const void* Vp, size_t ld, size_t n, const Ctl* ctl,
                 int nf_max, const void* coef_a, const void* coef_bh, float hscale, cudaStream_t st) {
    using S2 = typename Tr<P>::S2;
    using C = typename Tr<P>::C;
    int g = (int)((n + 255) / 256);
#define BI_BU(NF)                                                                                       \
    block_update_kernel<P, NF><<<g, 256, 0, st>>>((S2*)W, (const S2*)Y, (const S2*)Vk, (const S2*)Vp, ld, n, ctl, \
                                                  (const C*)coef_a, (const C*)coef_bh, hscale)
    BI_DISPATCH_NF(nf_max, BI_BU)
#undef BI_BU
}

template <int P>
void launch_ug_t(void* W, const void* Y, const void* Vk, const void* Vp, size_t ld, size_t n, const Ctl* ctl,
                 int nf_max, const void* coef_a, const void* coef_bh, double* partials, int nblk, float hscale,
                 cudaStream_t st) {
    using S2 = typename Tr<P>::S2;
    using C = typename Tr<P>::C;
#define BI_UG(NF)                                                                                            \
    {                                                                                                        \
        constexpr int SMEM = NF * UG_ROWS * (int)sizeof(S2);                                                 \
        static std::atomic<unsigned long long> devs{0};                                                      \
        max_dyn_smem_once(update_gram_kernel<P, NF>, SMEM, devs);                                            \
        update_gram_kernel<P, NF><<<nblk, UG_ROWS, SMEM, st>>>((S2*)W, (const S2*)Y, (const S2*)Vk,            \
                                                               (const S2*)Vp, ld, n, ctl, nf_max, (const C*)coef_a, \
                                                               (const C*)coef_bh, partials, hscale);          \
    }
    switch (nf_bucket(nf_max)) {
        case 4: BI_UG(4); break;
        case 8: BI_UG(8); break;
        default: BI_UG(12); break;
    }
#undef BI_UG
}

template <int P>
void launch_ib_t(void* V1, size_t ldv, const void* B, int bprec, size_t ldb, size_t n, const double2* S, int s_dd,
                 const Ctl* ctl, int nf_in, float hscale, cudaStream_t st) {
    using S2 = typename Tr<P>::S2;
    int g = (int)((n + 255) / 256);
    if (bprec == P64 || P == P64) {
        // FP64 storage always starts from FP64 right-hand sides
#define BI_IB(NF) \
    init_basis_kernel<P, NF, P64><<<g, 256, 0, st>>>((S2*)V1, ldv, (const double2*)B, ldb, n, S, s_dd, ctl, nf_in, \
                                                     hscale)
        BI_DISPATCH_NF(nf_in, BI_IB)
#undef BI_IB
    } else {
#define BI_IB(NF) \
    init_basis_kernel<P, NF, P32><<<g, 256, 0, st>>>((S2*)V1, ldv, (const float2*)B, ldb, n, S, s_dd, ctl, nf_in, \
                                                     hscale)
        BI_DISPATCH_NF(nf_in, BI_IB)
#undef BI_IB
    }
}

// The same chunked update for FP32 work precision (FP32, BF16 and FP16
// storage), on the packed FP32 pipe: each __ffma2_rn performs the FMA of one
// complex component for two neighbouring output columns, so every element
// sees exactly the scalar sequence of cfma / cfms (one rounding per FMA, same
// order) at half the instruction count.  The coefficient tiles are staged as
// {re_i, re_i+1, im_i, im_i+1} per (row a, column pair); X_j and the new P_j
// are held as (re, re) / (im, im) column pairs.  The next step's V_{k+1} rows
// arrive in shared memory by per-thread asynchronous copies (each thread
// copies the elements it reads itself), one step ahead of their use.
template <int NF, int P>
__host__ __device__ constexpr size_t sc32_smem_bytes(int rows) {
    return 4 * (size_t)NF * NF * sizeof(float2) + 2 * (size_t)NF * rows * sizeof(typename Tr<P>::S2);
}

template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst_smem, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst_smem)), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int P, int NF, int ROWS>
__global__ void __launch_bounds__(ROWS, NF <= 12 ? 4 : 1) shift_chunk32_kernel(
    const typename Tr<P>::S2* __restrict__ ring, size_t slot_elems, int R, size_t ld, float2* __restrict__ Pb,
    float2* __restrict__ Xb, size_t ldw, size_t n, int s, int m, Ctl* __restrict__ ctl, int k0, int C,
    const float2* __restrict__ cU, const float2* __restrict__ cL, const int* __restrict__ act, float hscale) {
    static_assert(NF % 2 == 0, "column pairs");
    constexpr int NP = NF / 2;
    using SE = typename Tr<P>::S2;
    const int j = (int)(blockIdx.x % (unsigned)s);
    const int kend = min(k0 + C, ctl->last_step);
    if (kend <= k0 || !act[(size_t)(k0 % C) * s + j]) return;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    float* sCo = reinterpret_cast<float*>(sc_smem);                           // [2 buffers][U, L][NP][NF][4]
    SE* sV = reinterpret_cast<SE*>(sc_smem + 4 * (size_t)NF * NF * sizeof(float2));   // [2][NF][ROWS]
    const int tid = threadIdx.x;
    const size_t e0 = (size_t)(blockIdx.x / (unsigned)s) * ROWS;
    const bool ok = e0 + tid < n;
    const size_t e = e0 + (ok ? tid : 0);
    const float inv = (P == PBF16 || P == PF16) ? 1.f / hscale : 1.f;
    const size_t tile = (size_t)M_MAX * M_MAX;
    float2* Pj = Pb + (size_t)j * m * ldw;
    float2* Xj = Xb + (size_t)j * m * ldw;
    // rows of V_{k+1} (ring slot vs) into V buffer vb, this thread's element only
    auto prefetch = [&](int vs, int vb) {
        const SE* g = ring + (size_t)vs * slot_elems + e;
        SE* d = sV + (size_t)vb * NF * ROWS + tid;
#pragma unroll
        for (int c = 0; c < NF; ++c)
            if (c < m) cp_async_elem<sizeof(SE)>(d + c * ROWS, g + (size_t)c * ld);
        cp_async_commit();
    };
    int mk_ = ctl->hmk[k0 & (CTL_HIST - 1)];
    float2 t[NF];
    float2 xr[NP], xi[NP];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
        if (a < mk_) {
            if (k0 == 0) {
                const auto q = Elem<P>::ld(ring + slot_elems + (size_t)a * ld, e, inv);     // V_1
                t[a] = make_float2((float)q.x, (float)q.y);
            } else {
                t[a] = Pj[(size_t)a * ldw + e];
            }
        } else {
            t[a] = make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float2 x0 = 2 * p < m ? Xj[(size_t)(2 * p) * ldw + e] : make_float2(0.f, 0.f);
        const float2 x1 = 2 * p + 1 < m ? Xj[(size_t)(2 * p + 1) * ldw + e] : make_float2(0.f, 0.f);
        xr[p] = make_float2(x0.x, x1.x);
        xi[p] = make_float2(x0.y, x1.y);
    }
    int q = k0 % C;                    // coefficient / flag slot of step k
    int vs = (k0 + 2) % R;             // ring slot of V_{k+1}
    prefetch(vs, 0);
    int mn = mk_;
    for (int k = k0 + 1; k <= kend; ++k) {
        if (!act[(size_t)q * s + j]) break;
        mn = ctl->hmn[(k - 1) & (CTL_HIST - 1)];
        const int b = (k - k0 - 1) & 1;
        const int vs_next = vs + 1 == R ? 0 : vs + 1;
        const bool ahead = k < kend;
        if (ahead) prefetch(vs_next, b ^ 1);
        // this step's tiles into buffer b (its previous readers, step k - 2,
        // are past the barrier of step k - 1)
        float* bU = sCo + (size_t)b * 2 * NF * NF * 2;
        float* bL = bU + NF * NF * 2;
        const float2* gU = cU + ((size_t)q * s + j) * tile;
        const float2* gL = cL + ((size_t)q * s + j) * tile;
        for (int u = tid; u < NF * NF; u += ROWS) {
            const int a = u / NF, i = u % NF;
            const int at = (a * NP + (i >> 1)) * 4 + (i & 1);
            const float2 cu = gU[a * M_MAX + i], cl = gL[a * M_MAX + i];
            bU[at] = cu.x;
            bU[at + 2] = cu.y;
            bL[at] = cl.x;
            bL[at + 2] = cl.y;
        }
        __syncthreads();
        // X_j += P_j Ut_j
#pragma unroll
        for (int a = 0; a < NF; ++a) {
            const float2 tr = make_float2(t[a].x, t[a].x), ti = make_float2(t[a].y, t[a].y);
            const float2 nti = make_float2(-t[a].y, -t[a].y);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float4 u = *reinterpret_cast<const float4*>(&bU[(a * NP + p) * 4]);
                const float2 ure = make_float2(u.x, u.y), uim = make_float2(u.z, u.w);
                xr[p] = __ffma2_rn(tr, ure, xr[p]);
                xr[p] = __ffma2_rn(nti, uim, xr[p]);
                xi[p] = __ffma2_rn(tr, uim, xi[p]);
                xi[p] = __ffma2_rn(ti, ure, xi[p]);
            }
        }
        // P_j <- V_{k+1} - P_j Lh_j
        if (ahead) cp_async_wait<1>();
        else cp_async_wait<0>();
        const SE* v = sV + (size_t)b * NF * ROWS + tid;
        float2 pr[NP], pi[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
            if (2 * p < mn) {
                const auto w = Elem<P>::ld(v, (size_t)(2 * p) * ROWS, inv);
                v0 = make_float2((float)w.x, (float)w.y);
            }
            if (2 * p + 1 < mn) {
                const auto w = Elem<P>::ld(v, (size_t)(2 * p + 1) * ROWS, inv);
                v1 = make_float2((float)w.x, (float)w.y);
            }
            pr[p] = make_float2(v0.x, v1.x);
            pi[p] = make_float2(v0.y, v1.y);
        }
#pragma unroll
        for (int a = 0; a < NF; ++a) {
            const float2 ntr = make_float2(-t[a].x, -t[a].x), ti = make_float2(t[a].y, t[a].y);
            const float2 nti = make_float2(-t[a].y, -t[a].y);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float4 l = *reinterpret_cast<const float4*>(&bL[(a * NP + p) * 4]);
                const float2 lre = make_float2(l.x, l.y), lim = make_float2(l.z, l.w);
                pr[p] = __ffma2_rn(ntr, lre, pr[p]);
                pr[p] = __ffma2_rn(ti, lim, pr[p]);
                pi[p] = __ffma2_rn(ntr, lim, pi[p]);
                pi[p] = __ffma2_rn(nti, lre, pi[p]);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            t[2 * p] = 2 * p < mn ? make_float2(pr[p].x, pi[p].x) : make_float2(0.f, 0.f);
            t[2 * p + 1] = 2 * p + 1 < mn ? make_float2(pr[p].y, pi[p].y) : make_float2(0.f, 0.f);
        }
        q = q + 1 == C ? 0 : q + 1;
        vs = vs_next;
    }
    cp_async_wait<0>();                 // no copy in flight when the CTA leaves
    if (ok) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (2 * p < m) Xj[(size_t)(2 * p) * ldw + e] = make_float2(xr[p].x, xi[p].x);
            if (2 * p + 1 < m) Xj[(size_t)(2 * p + 1) * ldw + e] = make_float2(xr[p].y, xi[p].y);
        }
#pragma unroll
        for (int c = 0; c < NF; ++c)
            if (c < mn) Pj[(size_t)c * ldw + e] = t[c];
    }
    if (blockIdx.x < (unsigned)s && tid == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->f_shift_w), (unsigned long long)(mk_ + 2 * m + mn));
}

template <int P>
void launch_vu_t(void* Vnext, const void* W, size_t ld, size_t n, const Ctl* ctl, int nf_max, const void* coefS,
                 float hscale, cudaStream_t st) {
    constexpr int PW = (P == P64) ? P64 : P32;
    using S2 = typename Tr<P>::S2;
    using CW = typename Tr<PW>::C;
#define BI_VU(NF)                                                                                           \
    v_update_kernel<P, NF><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((S2*)Vnext, (const S2*)W, ld, n, ctl, \
                                                                       (const CW*)coefS, hscale)
    BI_DISPATCH_NF(nf_max, BI_VU)
#undef BI_VU
}

template <int P>
void launch_sc_t(const void* ring, size_t slot_elems, int R, size_t ld, void* Pp, void* X, size_t ldw, size_t n,
                 int s, int m, Ctl* ctl, int nf_max, int k0, int C, const void* coefU, const void* coefL,
                 const int* active, float hscale, cudaStream_t st) {
    constexpr int PW = (P == P64) ? P64 : P32;
    using S2 = typename Tr<P>::S2;
    using W2 = typename Tr<PW>::S2;
    using CW = typename Tr<PW>::C;
#define BI_SC(NF)                                                                                           \
    {                                                                                                       \
        constexpr int ROWS = 128;                                                                           \
        const unsigned g = (unsigned)(((n + ROWS - 1) / ROWS) * (size_t)s);                                 \
        if constexpr (PW == P64) {                                                                          \
            constexpr size_t SMEM = sc_smem_bytes<NF, PW>();                                                \
            static std::atomic<unsigned long long> devs{0};                                                 \
            max_dyn_smem_once(shift_chunk_kernel<P, PW, NF, ROWS>, (int)SMEM, devs);                        \
            shift_chunk_kernel<P, PW, NF, ROWS><<<g, ROWS, SMEM, st>>>(                                      \
                (const S2*)ring, slot_elems, R, ld, (W2*)Pp, (W2*)X, ldw, n, s, m, ctl, k0, C,              \
                (const CW*)coefU, (const CW*)coefL, active, hscale);                                        \
        } else {                                                                                            \
            constexpr size_t SMEM = sc32_smem_bytes<NF, P>(ROWS);                                           \
            static std::atomic<unsigned long long> devs{0};                                                 \
            max_dyn_smem_once(shift_chunk32_kernel<P, NF, ROWS>, (int)SMEM, devs);                          \
            shift_chunk32_kernel<P, NF, ROWS><<<g, ROWS, SMEM, st>>>(                                        \
                (const S2*)ring, slot_elems, R, ld, (float2*)Pp, (float2*)X, ldw, n, s, m, ctl, k0, C,      \
                (const float2*)coefU, (const float2*)coefL, active, hscale);                                \
        }                                                                                                   \
    }
    BI_DISPATCH_NF(nf_max, BI_SC)
#undef BI_SC
}

#define BI_INSTANTIATE(P)                                                                                  \
    template void launch_bu_t<P>(void*, const void*, const void*, const void*, size_t, size_t, const Ctl*, int, \
                                 const void*, const void*, float, cudaStream_t);                          \
    template void launch_ug_t<P>(void*, const void*, const void*, const void*, size_t, size_t, const Ctl*, int, \
                                 const void*, const void*, double*, int, float, cudaStream_t);            \
    template void launch_ib_t<P>(void*, size_t, const void*, int, size_t, size_t, const double2*, int,       \
                                 const Ctl*, int, float, cudaStream_t);                                    \
    template void launch_vu_t<P>(void*, const void*, size_t, size_t, const Ctl*, int, const void*, float,    \
                                 cudaStream_t);                                                            \
    template void launch_sc_t<P>(const void*, size_t, int, size_t, void*, void*, size_t, size_t, int, int,   \
                                 Ctl*, int, int, int, const void*, const void*, const int*, float, cudaStream_t);

}  // namespace blas_impl
}  // namespace dsbcg

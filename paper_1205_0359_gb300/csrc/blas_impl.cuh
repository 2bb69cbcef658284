// Tall-skinny block kernels of the block Lanczos process (Sec. 3):
//   gram          G = X^H Y (nf x nf) for n x nf field blocks, FP64 result
//   block_update  W = A V_k - V_k alpha_k - V_{k-1} beta_k^H
//   init_basis    V_1 = B S (FP64 right-hand sides -> storage precision)
//   shift_update  V_{k+1} = W S;  for every active shift j:
//                 X_j += P_j Ut_j,  P_j <- V_{k+1} - P_j Lh_j
//                 (the per-shift short recurrences of Sec. 3, all shifts in
//                 one pass over HBM), P_j and X_j streamed through shared
//                 memory with bulk asynchronous copies.
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
// Shift update (the per-shift short recurrences of Sec. 3 for all shifts,
// one pass over HBM per operand):
//     V_{k+1} = W S                       (v_update_kernel, one thread per row)
//     for every active shift j:
//     X_j += P_j Ut_j,   P_j <- V_{k+1} - P_j Lh_j   (shift_tile_kernel)
// shift_tile_kernel runs one CTA per (row tile, shift); its tiles arrive by
// bulk asynchronous copies (cp.async.bulk, completion on an mbarrier) and
// each thread updates two rows.  Every mbarrier wait is bounded; on timeout
// the kernel records an error in the control block, drains its own copies
// and returns.  For the first step of an inner solve (k == 1) the search
// block is P_j = V_1 itself.
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

// Per-shift update of one row tile: X_j += P_j Ut_j, P_j <- V_{k+1} - P_j Lh_j.
// One CTA per (row tile, shift), shift index fastest so that the CTAs that
// read the same V_{k+1} tile run together and share it through L2.  The P_j
// and X_j tiles (one contiguous run of ROWS elements per field) arrive in
// shared memory by bulk asynchronous copies completing on one mbarrier;
// V_{k+1} rows are read straight from L2, which keeps the shared memory per
// CTA small and the resident CTAs per SM many.  Results are stored directly
// (coalesced).  The mbarrier wait is bounded: on timeout the CTA records an
// error in the control block and returns after draining its copies.  At
// k == 1 the search block is P_j = V_1 (the current block, storage precision).
template <int NF, int PW, int PS>
__host__ __device__ constexpr size_t su_smem_bytes(int rows) {
    return (size_t)rows * NF * 2 * sizeof(typename Tr<PW>::S2) + 2 * (size_t)NF * NF * sizeof(typename Tr<PW>::C) + 16;
}

// rows per thread of shift_tile_kernel: one (two rows per thread halve the
// shared-memory coefficient reads but, at about 170 registers, cut the
// resident warps from 28 to 10 per SM, which measured slower on GB300)
__host__ __device__ constexpr int su_rpt(int, int) { return 1; }

template <int P, int PW, int NF, int ROWS>
__global__ void __launch_bounds__(ROWS / su_rpt(NF, PW)) shift_tile_kernel(
    const typename Tr<P>::S2* __restrict__ Vn, const typename Tr<P>::S2* __restrict__ Vk, size_t ld,
    typename Tr<PW>::S2* __restrict__ Pb, typename Tr<PW>::S2* __restrict__ Xb, size_t ldw, size_t n, int s, int m,
    Ctl* __restrict__ ctl, const typename Tr<PW>::C* __restrict__ cU, const typename Tr<PW>::C* __restrict__ cL,
    const int* __restrict__ active, float hscale) {
    using C = typename Tr<PW>::C;
    using R = typename Tr<PW>::R;
    using E = typename Tr<PW>::S2;
    using SE = typename Tr<P>::S2;
    if (ctl->done) return;
    const int j = (int)(blockIdx.x % (unsigned)s);
    if (!active[j]) return;
    const int mk_ = ctl->mk, mn = ctl->mnext, k = ctl->k;
    extern __shared__ __align__(128) unsigned char su_smem[];
    E* sP = reinterpret_cast<E*>(su_smem);                          // [NF][ROWS] P_j (or V_1 at k == 1)
    E* sX = sP + NF * ROWS;
    C* sU = reinterpret_cast<C*>(sX + NF * ROWS);
    C* sL = sU + NF * NF;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sL + NF * NF);
    const int tid = threadIdx.x;
    const size_t e0 = (size_t)(blockIdx.x / (unsigned)s) * ROWS;
    const int rows = (int)((n - e0) < (size_t)ROWS ? (n - e0) : (size_t)ROWS);
    const uint32_t tb = (uint32_t)rows * sizeof(E), tbs = (uint32_t)rows * sizeof(SE);
    const E* Pj = Pb + (size_t)j * m * ldw + e0;
    E* Pjw = Pb + (size_t)j * m * ldw + e0;
    E* Xj = Xb + (size_t)j * m * ldw + e0;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        // k == 1: the search block is V_1 itself (loaded into sP's place)
        const uint32_t nv = k == 1 ? (uint32_t)mk_ : 0u;
        const uint32_t np = k > 1 ? (uint32_t)mk_ : 0u;
        mbar_expect_tx(bar, nv * tbs + (np + (uint32_t)m) * tb);
        if (k == 1) {
            // V_1 (storage precision) into the P tile's space, which is at least as large
            for (int a = 0; a < mk_; ++a) bulk_g2s(reinterpret_cast<SE*>(sP) + a * ROWS, Vk + (size_t)a * ld + e0, tbs, bar);
        } else {
            for (int a = 0; a < mk_; ++a) bulk_g2s(sP + a * ROWS, Pj + (size_t)a * ldw, tb, bar);
        }
        for (int i = 0; i < m; ++i) bulk_g2s(sX + i * ROWS, Xj + (size_t)i * ldw, tb, bar);
    }
    for (int t = tid; t < NF * NF; t += ROWS / su_rpt(NF, PW)) {
        sU[t] = cU[((size_t)j * M_MAX + t / NF) * M_MAX + t % NF];
        sL[t] = cL[((size_t)j * M_MAX + t / NF) * M_MAX + t % NF];
    }
    const bool ok = mbar_wait(bar, 0);
    __syncthreads();
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            mbar_wait(bar, 0);
            atomicCAS(&ctl->status, 0, ST_WAIT_TIMEOUT);
        }
        return;
    }
    const float inv = (P == PBF16 || P == PF16) ? 1.f / hscale : 1.f;
    auto ldv = [&](const SE* base, int c, int r) -> C {
        auto q = Elem<P>::ld(base, (size_t)c * ROWS + r, inv);
        return mk(R(q.x), R(q.y));
    };
    // RPT rows per thread (r = tid, tid + ROWS / RPT, ...): every coefficient
    // read from shared memory serves all of them, and FP32 coefficients are
    // read two at a time; each element accumulates over a in ascending order
    constexpr int RPT = su_rpt(NF, PW), TPB = ROWS / RPT;
    int rr_[RPT];
    bool ok_[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        rr_[q] = tid + q * TPB;
        ok_[q] = rr_[q] < rows;
    }
    C t[RPT][NF], x[RPT][NF];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int a = 0; a < NF; ++a) {
            const int r = ok_[q] ? rr_[q] : 0;
            if (a < mk_) t[q][a] = (k == 1) ? ldv(reinterpret_cast<const SE*>(sP), a, r) : sP[a * ROWS + r];
            else t[q][a] = mk(R(0), R(0));
            x[q][a] = a < m ? sX[a * ROWS + r] : mk(R(0), R(0));
        }
    // X_j += P_j Ut_j
#pragma unroll
    for (int a = 0; a < NF; ++a) {
#pragma unroll
        for (int i = 0; i < NF; i += 2) {
            C u0, u1;
            if constexpr (sizeof(C) == 8) {
                const float4 u2 = *reinterpret_cast<const float4*>(&sU[a * NF + i]);
                u0 = mk(R(u2.x), R(u2.y));
                u1 = mk(R(u2.z), R(u2.w));
            } else {
                u0 = sU[a * NF + i];
                u1 = sU[a * NF + i + 1];
            }
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                cfma(x[q][i], t[q][a], u0);
                cfma(x[q][i + 1], t[q][a], u1);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q)
        if (ok_[q])
#pragma unroll
            for (int i = 0; i < NF; ++i)
                if (i < m) Xj[(size_t)i * ldw + rr_[q]] = x[q][i];
    // P_j <- V_{k+1} - P_j Lh_j
    C pn[RPT][NF];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int c = 0; c < NF; ++c) {
            if (c < mn) {
                const auto v = Elem<P>::ld(Vn + (size_t)c * ld, e0 + (ok_[q] ? rr_[q] : 0), inv);
                pn[q][c] = mk(R(v.x), R(v.y));
            } else {
                pn[q][c] = mk(R(0), R(0));
            }
        }
#pragma unroll
    for (int a = 0; a < NF; ++a) {
#pragma unroll
        for (int c = 0; c < NF; c += 2) {
            C l0, l1;
            if constexpr (sizeof(C) == 8) {
                const float4 l2 = *reinterpret_cast<const float4*>(&sL[a * NF + c]);
                l0 = mk(R(l2.x), R(l2.y));
                l1 = mk(R(l2.z), R(l2.w));
            } else {
                l0 = sL[a * NF + c];
                l1 = sL[a * NF + c + 1];
            }
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                cfms(pn[q][c], t[q][a], l0);
                cfms(pn[q][c + 1], t[q][a], l1);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q)
        if (ok_[q])
#pragma unroll
            for (int c = 0; c < NF; ++c)
                if (c < mn) Pjw[(size_t)c * ldw + rr_[q]] = pn[q][c];
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

template <int P>
void launch_su_t(void* Vnext, const void* W, const void* Vk, size_t ld, void* Pp, void* X, size_t ldw, size_t n,
                 int s, int m, Ctl* ctl, int nf_max, const void* coefS, const void* coefU, const void* coefL,
                 const int* active, float hscale, cudaStream_t st) {
    constexpr int PW = (P == P64) ? P64 : P32;
    using S2 = typename Tr<P>::S2;
    using W2 = typename Tr<PW>::S2;
    using CW = typename Tr<PW>::C;
#define BI_SU(NF)                                                                                           \
    {                                                                                                       \
        constexpr int ROWS = su_smem_bytes<NF, PW, P>(128) <= 200000 ? 128 : 64;                            \
        v_update_kernel<P, NF><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((S2*)Vnext, (const S2*)W, ld, n, ctl, \
                                                                           (const CW*)coefS, hscale);       \
        constexpr size_t SMEM = su_smem_bytes<NF, PW, P>(ROWS);                                             \
        static std::atomic<unsigned long long> devs{0};                                                     \
        max_dyn_smem_once(shift_tile_kernel<P, PW, NF, ROWS>, (int)SMEM, devs);                             \
        const unsigned g = (unsigned)(((n + ROWS - 1) / ROWS) * (size_t)s);                                 \
        shift_tile_kernel<P, PW, NF, ROWS><<<g, ROWS / su_rpt(NF, PW), SMEM, st>>>(                                          \
            (const S2*)Vnext, (const S2*)Vk, ld, (W2*)Pp, (W2*)X, ldw, n, s, m, ctl, (const CW*)coefU,      \
            (const CW*)coefL, active, hscale);                                                              \
    }
    BI_DISPATCH_NF(nf_max, BI_SU)
#undef BI_SU
}

#define BI_INSTANTIATE(P)                                                                                  \
    template void launch_bu_t<P>(void*, const void*, const void*, const void*, size_t, size_t, const Ctl*, int, \
                                 const void*, const void*, float, cudaStream_t);                          \
    template void launch_ib_t<P>(void*, size_t, const void*, int, size_t, size_t, const double2*, int,       \
                                 const Ctl*, int, float, cudaStream_t);                                    \
    template void launch_su_t<P>(void*, const void*, const void*, size_t, void*, void*, size_t, size_t, int, int, \
                                 Ctl*, int, const void*, const void*, const void*, const int*, float,         \
                                 cudaStream_t);

}  // namespace blas_impl
}  // namespace dsbcg

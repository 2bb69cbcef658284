// Tall-skinny block kernels of the block Lanczos process (Sec. 3):
//   gram          G = X^H Y (nf x nf) for n x nf field blocks, FP64 result
//   block_update  W = A V_k - V_k alpha_k - V_{k-1} beta_k^H
//   init_basis    V_1 = B S (FP64 right-hand sides -> storage precision)
//   shift_update  V_{k+1} = W S;  for every active shift j:
//                 X_j += P_j Ut_j,  P_j <- V_{k+1} - P_j Lh_j
//                 (the per-shift short recurrences of Sec. 3, all shifts in
//                 one pass over HBM)
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
        if (threadIdx.x < GSLOTS) out[threadIdx.x] = 0.0;
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
        double sacc = 0.0;
#pragma unroll
        for (int ww = 0; ww < GT / 32; ++ww) sacc += (double)red[ww][threadIdx.x];
        out[threadIdx.x] = sacc;
    }
}

// G[i][j] (M_MAX x M_MAX) from the per-CTA partials; one CTA per tile
static __global__ void gram_reduce_kernel(const double* __restrict__ partials, int nblk, int nf_max, int herm,
                                   int diag_yy, double2* __restrict__ G, double* __restrict__ diag,
                                   const Ctl* __restrict__ ctl) {
    if (ctl && ctl->done) return;
    const int T = (nf_max + 3) / 4;
    const int tile = blockIdx.x;
    int ti, tj;
    tile_coords(tile, T, herm, &ti, &tj);
    const int q = threadIdx.x;
    if (q >= GSLOTS) return;
    const double* p = partials + (size_t)tile * nblk * GSLOTS;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += p[(size_t)b * GSLOTS + q];
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
    C v[NF], vp[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
        v[a] = a < mk_ ? Elem<P>::ld(Vk + (size_t)a * ld, e, inv) : mk(R(0), R(0));
        vp[a] = a < mp ? Elem<P>::ld(Vp + (size_t)a * ld, e, inv) : mk(R(0), R(0));
    }
#pragma unroll
    for (int b = 0; b < NF; ++b) {
        if (b < mk_) {
            C w = Elem<P>::ld(Y + (size_t)b * ld, e, inv);
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
template <int P, int NF>
__global__ void __launch_bounds__(256) init_basis_kernel(typename Tr<P>::S2* __restrict__ V1, size_t ldv,
                                                         const double2* __restrict__ B, size_t ldb, size_t n,
                                                         const double2* __restrict__ S,
                                                         const Ctl* __restrict__ ctl, int nf_in, float hscale) {
    using R = typename Tr<P>::R;
    const int m1 = ctl->mk;
    __shared__ double2 ss[NF * NF];
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) ss[t] = S[(t / NF) * M_MAX + (t % NF)];
    __syncthreads();
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const R scl = (P == PBF16 || P == PF16) ? R(hscale) : R(1);
    double2 b[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) b[a] = a < nf_in ? B[(size_t)a * ldb + e] : make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < NF; ++c) {
        if (c < m1) {
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int a = 0; a < NF; ++a) cfma(acc, b[a], ss[a * NF + c]);
            Elem<P>::st(V1 + (size_t)c * ldv, e, mk(R(acc.x), R(acc.y)), scl);
        }
    }
}

// ---------------------------------------------------------------------------
// Fused shift update.  One thread per row e.  For the first step of an inner
// solve (k == 1) the search block of every shift is P_j = V_1 itself.
template <int P, int PW, int NF>
__global__ void __launch_bounds__(256) shift_update_kernel(
    typename Tr<P>::S2* __restrict__ Vn, const typename Tr<P>::S2* __restrict__ W,
    const typename Tr<P>::S2* __restrict__ Vk, size_t ld, typename Tr<PW>::S2* __restrict__ Pb,
    typename Tr<PW>::S2* __restrict__ Xb, size_t ldw, size_t n, int s, int m, const Ctl* __restrict__ ctl,
    const typename Tr<PW>::C* __restrict__ cS, const typename Tr<PW>::C* __restrict__ cU,
    const typename Tr<PW>::C* __restrict__ cL, const int* __restrict__ active, float hscale) {
    using C = typename Tr<PW>::C;
    using R = typename Tr<PW>::R;
    if (ctl->done) return;
    const int mk_ = ctl->mk, mn = ctl->mnext, k = ctl->k;
    __shared__ C sS[NF * NF], sU[NF * NF], sL[NF * NF];
    for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) sS[t] = cS[(t / NF) * M_MAX + (t % NF)];
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = e < n;
    const float inv = (P == PBF16 || P == PF16) ? 1.f / hscale : 1.f;
    const float scl = (P == PBF16 || P == PF16) ? hscale : 1.f;
    __syncthreads();
    C v[NF];
    if (live) {
        C w[NF];
#pragma unroll
        for (int a = 0; a < NF; ++a) {
            if (a < mk_) {
                auto t = Elem<P>::ld(W + (size_t)a * ld, e, inv);
                w[a] = mk(R(t.x), R(t.y));
            } else {
                w[a] = mk(R(0), R(0));
            }
        }
#pragma unroll
        for (int c = 0; c < NF; ++c) {
            C acc = mk(R(0), R(0));
#pragma unroll
            for (int a = 0; a < NF; ++a) cfma(acc, w[a], sS[a * NF + c]);
            v[c] = acc;
            if (c < mn) Elem<P>::st(Vn + (size_t)c * ld, e, mk((typename Tr<P>::R)acc.x, (typename Tr<P>::R)acc.y), scl);
        }
    }
    for (int j = 0; j < s; ++j) {
        if (!active[j]) continue;          // uniform across the grid
        __syncthreads();
        for (int t = threadIdx.x; t < NF * NF; t += blockDim.x) {
            int a = t / NF, b = t % NF;
            sU[t] = cU[((size_t)j * M_MAX + a) * M_MAX + b];
            sL[t] = cL[((size_t)j * M_MAX + a) * M_MAX + b];
        }
        __syncthreads();
        if (!live) continue;
        typename Tr<PW>::S2* Pj = Pb + (size_t)j * m * ldw;     // m fields per shift
        typename Tr<PW>::S2* Xj = Xb + (size_t)j * m * ldw;
        C t[NF];
#pragma unroll
        for (int a = 0; a < NF; ++a) {
            if (a < mk_) {
                if (k == 1) {
                    auto q = Elem<P>::ld(Vk + (size_t)a * ld, e, inv);
                    t[a] = mk(R(q.x), R(q.y));
                } else {
                    t[a] = Elem<PW>::ld(Pj + (size_t)a * ldw, e, R(1));
                }
            } else {
                t[a] = mk(R(0), R(0));
            }
        }
        for (int i = 0; i < m; ++i) {
            C x = Elem<PW>::ld(Xj + (size_t)i * ldw, e, R(1));
#pragma unroll
            for (int a = 0; a < NF; ++a) cfma(x, t[a], sU[a * NF + (i < NF ? i : 0)]);
            Elem<PW>::st(Xj + (size_t)i * ldw, e, x, R(1));
        }
#pragma unroll
        for (int c = 0; c < NF; ++c) {
            if (c < mn) {
                C p = v[c];
#pragma unroll
                for (int a = 0; a < NF; ++a) cfms(p, t[a], sL[a * NF + c]);
                Elem<PW>::st(Pj + (size_t)c * ldw, e, p, R(1));
            }
        }
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
void launch_ib_t(void* V1, size_t ldv, const double2* B, size_t ldb, size_t n, const double2* S, const Ctl* ctl,
                 int nf_in, float hscale, cudaStream_t st) {
    using S2 = typename Tr<P>::S2;
    int g = (int)((n + 255) / 256);
#define BI_IB(NF) init_basis_kernel<P, NF><<<g, 256, 0, st>>>((S2*)V1, ldv, B, ldb, n, S, ctl, nf_in, hscale)
    BI_DISPATCH_NF(nf_in, BI_IB)
#undef BI_IB
}

template <int P>
void launch_su_t(void* Vnext, const void* W, const void* Vk, size_t ld, void* Pp, void* X, size_t ldw, size_t n,
                 int s, int m, const Ctl* ctl, int nf_max, const void* coefS, const void* coefU, const void* coefL,
                 const int* active, float hscale, cudaStream_t st) {
    constexpr int PW = (P == P64) ? P64 : P32;
    using S2 = typename Tr<P>::S2;
    using W2 = typename Tr<PW>::S2;
    using CW = typename Tr<PW>::C;
    int g = (int)((n + 255) / 256);
#define BI_SU(NF)                                                                                        \
    shift_update_kernel<P, PW, NF><<<g, 256, 0, st>>>((S2*)Vnext, (const S2*)W, (const S2*)Vk, ld, (W2*)Pp, (W2*)X, \
                                                      ldw, n, s, m, ctl, (const CW*)coefS, (const CW*)coefU,        \
                                                      (const CW*)coefL, active, hscale)
    BI_DISPATCH_NF(nf_max, BI_SU)
#undef BI_SU
}

#define BI_INSTANTIATE(P)                                                                                  \
    template void launch_bu_t<P>(void*, const void*, const void*, const void*, size_t, size_t, const Ctl*, int, \
                                 const void*, const void*, float, cudaStream_t);                          \
    template void launch_ib_t<P>(void*, size_t, const double2*, size_t, size_t, const double2*, const Ctl*, int, \
                                 float, cudaStream_t);                                                     \
    template void launch_su_t<P>(void*, const void*, const void*, size_t, void*, void*, size_t, size_t, int, int, \
                                 const Ctl*, int, const void*, const void*, const void*, const int*, float,   \
                                 cudaStream_t);

}  // namespace blas_impl
}  // namespace dsbcg

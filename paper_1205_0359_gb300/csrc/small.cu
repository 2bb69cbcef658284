// FP64 m x m kernels of the block Lanczos process and of the per-shift
// recurrences (Sec. 3), run by one CTA (shared part) or one CTA per shift.
//
// Block form.  The Lanczos blocks V_1, V_2, ... (widths m_k, shrinking on
// deflation) satisfy
//     A V_k = V_{k-1} beta_k^H + V_k alpha_k + V_{k+1} beta_{k+1},
// so T = V^H A V is block tridiagonal with diagonal blocks alpha_k and
// sub-diagonal blocks beta_{k+1} (m_{k+1} x m_k): a hermitian band matrix of
// semi-bandwidth <= m (Eq. 3.1).  For each shift the root-free block
// Cholesky factorisation sigma_j I + T = L Delta L^H (L block unit lower
// bidiagonal with blocks Lambda_k, Delta block diagonal) is extended by one
// block row per step:
//     Delta_1 = alpha_1 + sigma I,
//     Lambda_{k+1} = beta_{k+1} Delta_k^{-1},
//     Delta_{k+1} = alpha_{k+1} + sigma I - Lambda_{k+1} beta_{k+1}^H,
// and with U = L^{-1} [rho; 0] (B = V_1 rho), P = V L^{-H}:
//     U_1 = rho, U_{k+1} = -Lambda_{k+1} U_k,  Ut_k = Delta_k^{-1} U_k,
//     P_1 = V_1, P_{k+1} = V_{k+1} - P_k Lambda_{k+1}^H,
//     X^(k) = X^(k-1) + P_k Ut_k,
// the block counterpart of the paper's scalar update with d^(k), p^(k),
// u^(k) (Sec. 3).  From the Lanczos relation the residual is
//     R^(k) = B - (sigma + A) X^(k) = -V_{k+1} beta_{k+1} Ut_k = V_{k+1} C_k,
// so with orthonormal V_{k+1} the residual norm of right-hand side i is the
// norm of column i of C_k = -beta_{k+1} Ut_k (Sec. 3, R^(k) = W^(k) C^(k)).
//
// Deflation (Sec. 1 and Sec. 3): the new block W is orthonormalised by a
// pivoted Cholesky factorisation of its FP64 Gram matrix.  Columns whose
// remaining squared norm falls to <= dtol^2 times their norm when created
//
// Arithmetic.  With FP64 storage these kernels run in FP64.  With the
// reduced storages they run in double-float (dd: pairs of FP32 words, 48-bit
// significands) unless FP64 is requested: GB300 issues FP64 at 1/64 of its
// FP32 rate, so one FP64
// instruction occupies an SM sub-partition for about 64 cycles and these
// latency-bound m x m kernels were dominated by it; the double-float forms
// run on the FP32 pipes and keep far more accuracy than the FP32 Gram
// partials they start from.  Both scalars take 16 bytes per complex entry,
// so the device state has one layout.
#include <math.h>

#include "kernels.h"

namespace dsbcg {

template <class T>
struct SmallSharedT {
    T alpha[M_MAX * M_MAX];          // alpha_k (hermitised)
    T betak[M_MAX * M_MAX];          // beta_k    (m_k x m_{k-1})
    T betan[M_MAX * M_MAX];          // beta_{k+1} (m_{k+1} x m_k)
    T S[M_MAX * M_MAX];              // V_{k+1} = W S (m_k x m_{k+1})
    T yy[M_MAX / 2];                 // ||A v_i||^2 (real scalars, two per entry)
};
template <class T>
struct SmallShiftT {
    T Lam[M_MAX * M_MAX];            // Lambda_k (m_k x m_{k-1})
    T U[M_MAX * M_MAX];              // U_k (m_k x m)
    int conv[M_MAX];                 // right-hand side i frozen
    int alive;                       // some column not converged
    int pad[M_MAX - 1];
};
template <class T>
struct SmallStateT {
    SmallSharedT<T> sh;
    SmallShiftT<T> sf[1];            // [s]
};
// the opaque type of kernels.h: the same bytes for both scalars
struct SmallState : SmallStateT<double2> {};
static_assert(sizeof(ddc) == sizeof(double2), "one state layout for both scalars");

size_t small_state_bytes(int s) {
    return sizeof(SmallSharedT<double2>) + (size_t)s * sizeof(SmallShiftT<double2>);
}
const double2* small_state_S(const SmallState* ss) { return ss->sh.S; }

namespace {

constexpr int WS = 32;             // the pivoted QR runs on one warp
constexpr int NT = 1024;           // threads of the CTAs that also reduce partial sums
constexpr int GSL = 36;            // slots per 4 x 4 tile in the Gram partials
constexpr int RED_MAX = 1024;      // group sums held in shared memory by reduce_partials

// ------------------------------------------------------------ scalars --
// Sc<T>: real type R, complex T, and the operations the m x m algebra needs.
template <class T>
struct Sc;

template <>
struct Sc<double2> {
    using R = double;
    static __device__ __forceinline__ R r(double v) { return v; }
    static __device__ __forceinline__ double d(R v) { return v; }
    static __device__ __forceinline__ double2 z() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ double2 c(R a, R b) { return make_double2(a, b); }
    static __device__ __forceinline__ R re(double2 a) { return a.x; }
    static __device__ __forceinline__ R im(double2 a) { return a.y; }
    static __device__ __forceinline__ R add(R a, R b) { return a + b; }
    static __device__ __forceinline__ R sub(R a, R b) { return a - b; }
    static __device__ __forceinline__ R mul(R a, R b) { return a * b; }
    static __device__ __forceinline__ R neg(R a) { return -a; }
    static __device__ __forceinline__ R rcp(R a) { return 1.0 / a; }
    static __device__ __forceinline__ R sqrt_(R a) { return sqrt(a); }
    static __device__ __forceinline__ bool gt(R a, R b) { return a > b; }
    static __device__ __forceinline__ float2 f2(double2 a) { return make_float2((float)a.x, (float)a.y); }
    // sum of a Kahan-compensated FP32 sum (value s - c)
    static __device__ __forceinline__ R kahan(float s, float c) { return (double)s - (double)c; }
};

// double-float reciprocal and square root: FP32 estimate refined by one
// Newton-Raphson step in double-float (Karp & Markstein, "High-precision
// division and square root", ACM TOMS 23(4), 1997)
__device__ __forceinline__ dd dd_rcp(dd a) {
    const float q = 1.0f / a.hi;
    // e = 1 - a q, with a.hi q exact as p + pe
    const float p = a.hi * q;
    const float pe = fmaf(a.hi, q, -p);
    const float e = ((1.0f - p) - pe) - a.lo * q;
    return quick_two_sum(q, q * e);
}
__device__ __forceinline__ dd dd_sqrt(dd a) {
    if (!(a.hi > 0.f)) return dd(0.f);
    const float s = sqrtf(a.hi);
    const float p = s * s;
    const float pe = fmaf(s, s, -p);
    const float e = ((a.hi - p) - pe) + a.lo;            // a - s^2
    return quick_two_sum(s, e * (0.5f / s));
}

template <>
struct Sc<ddc> {
    using R = dd;
    static __device__ __forceinline__ R r(double v) { return dd::from_double(v); }
    static __device__ __forceinline__ double d(R v) { return (double)v.hi + (double)v.lo; }
    static __device__ __forceinline__ ddc z() { return ddc{dd(0.f), dd(0.f)}; }
    static __device__ __forceinline__ ddc c(R a, R b) { return ddc{a, b}; }
    static __device__ __forceinline__ R re(ddc a) { return a.x; }
    static __device__ __forceinline__ R im(ddc a) { return a.y; }
    static __device__ __forceinline__ R add(R a, R b) { return a + b; }
    static __device__ __forceinline__ R sub(R a, R b) { return a - b; }
    static __device__ __forceinline__ R mul(R a, R b) { return a * b; }
    static __device__ __forceinline__ R neg(R a) { return -a; }
    static __device__ __forceinline__ R rcp(R a) { return dd_rcp(a); }
    static __device__ __forceinline__ R sqrt_(R a) { return dd_sqrt(a); }
    static __device__ __forceinline__ bool gt(R a, R b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
    static __device__ __forceinline__ float2 f2(ddc a) { return make_float2(a.x.hi, a.y.hi); }
    static __device__ __forceinline__ R kahan(float s, float c) { return dd(s) - dd(c); }
};

template <class T> __host__ __device__ constexpr bool is_fp64() { return false; }
template <> __host__ __device__ constexpr bool is_fp64<double2>() { return true; }

// complex helpers on Sc<T> (all normalised)
template <class T> __device__ __forceinline__ T cz() { return Sc<T>::z(); }
template <class T> __device__ __forceinline__ T cconj(T a) { return Sc<T>::c(Sc<T>::re(a), Sc<T>::neg(Sc<T>::im(a))); }
template <class T> __device__ __forceinline__ T cplus(T a, T b) {
    return Sc<T>::c(Sc<T>::add(Sc<T>::re(a), Sc<T>::re(b)), Sc<T>::add(Sc<T>::im(a), Sc<T>::im(b)));
}
template <class T> __device__ __forceinline__ T cminus(T a, T b) {
    return Sc<T>::c(Sc<T>::sub(Sc<T>::re(a), Sc<T>::re(b)), Sc<T>::sub(Sc<T>::im(a), Sc<T>::im(b)));
}
template <class T> __device__ __forceinline__ T ctimes(T a, T b) {
    using S = Sc<T>;
    return S::c(S::sub(S::mul(S::re(a), S::re(b)), S::mul(S::im(a), S::im(b))),
                S::add(S::mul(S::re(a), S::im(b)), S::mul(S::im(a), S::re(b))));
}
template <class T> __device__ __forceinline__ T cscal(T a, typename Sc<T>::R s) {
    return Sc<T>::c(Sc<T>::mul(Sc<T>::re(a), s), Sc<T>::mul(Sc<T>::im(a), s));
}
template <class T> __device__ __forceinline__ typename Sc<T>::R cnorm2(T a) {
    using S = Sc<T>;
    return S::add(S::mul(S::re(a), S::re(a)), S::mul(S::im(a), S::im(a)));
}

__device__ __forceinline__ void bsync() { __syncthreads(); }
__device__ __forceinline__ void wsync() { __syncwarp(); }

// dst (r x c valid, R x Cc written, leading dim ld) <- src (M_MAX layout)
template <class T>
__device__ void ld_mat(T* dst, int ld, const T* src, int r, int c, int Rr, int Cc) {
    for (int t = threadIdx.x; t < Rr * Cc; t += blockDim.x) {
        int i = t / Cc, j = t % Cc;
        dst[i * ld + j] = (i < r && j < c) ? src[i * M_MAX + j] : cz<T>();
    }
}
// full M_MAX x M_MAX tile in the work precision (FP64 only for FP64 state),
// zero outside r x c
template <class T>
__device__ void st_mat_work(int wprec, void* dst, const T* src, int ld, int r, int c) {
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
        int i = t / M_MAX, j = t % M_MAX;
        const T v = (i < r && j < c) ? src[i * ld + j] : cz<T>();
        if constexpr (is_fp64<T>()) {
            if (wprec == P64) {
                reinterpret_cast<double2*>(dst)[t] = v;
                continue;
            }
        }
        reinterpret_cast<float2*>(dst)[t] = Sc<T>::f2(v);
    }
}

// C (r x c) = op(A) op(B) (beta = 0) or C - op(A) op(B) (beta = 1), scaled
// by sgn = +1 / -1 on the product; op: 0 plain, 1 conjugate transpose
template <class T>
__device__ void gemm(T* Cm, int ldc, const T* A, int lda, int ta, const T* B, int ldb, int tb, int r, int q, int c,
                     bool negate, bool accumulate) {
    for (int t = threadIdx.x; t < r * c; t += blockDim.x) {
        int i = t / c, j = t % c;
        T s = cz<T>();
        for (int l = 0; l < q; ++l) {
            T a = ta ? cconj(A[l * lda + i]) : A[i * lda + l];
            T b = tb ? cconj(B[j * ldb + l]) : B[l * ldb + j];
            s = cplus(s, ctimes(a, b));
        }
        if (accumulate) Cm[i * ldc + j] = negate ? cminus(Cm[i * ldc + j], s) : cplus(Cm[i * ldc + j], s);
        else Cm[i * ldc + j] = negate ? cminus(cz<T>(), s) : s;
    }
    bsync();
}

// In-place inverse of a hermitian positive definite n x n matrix by
// Gauss-Jordan elimination without pivoting (its pivots are the Schur
// complement diagonals, positive for hpd).  Returns 0 if a pivot is <= 0.
template <class T>
__device__ int gj_inverse(T* A, int ld, int n, T* col) {
    using S = Sc<T>;
    int ok = 1;
    for (int p = 0; p < n; ++p) {
        typename S::R d = S::re(A[p * ld + p]);
        if (!S::gt(d, S::r(0.0))) {
            ok = 0;
            d = S::r(1.0);
        }
        const typename S::R inv = S::rcp(d);
        for (int r = threadIdx.x; r < n; r += blockDim.x) col[r] = A[r * ld + p];
        bsync();
        for (int c = threadIdx.x; c < n; c += blockDim.x)
            A[p * ld + c] = (c == p) ? S::c(inv, S::r(0.0)) : cscal(A[p * ld + c], inv);
        bsync();
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            int r = t / n, c = t % n;
            if (r == p) continue;
            const T f = col[r];
            if (c == p) A[r * ld + p] = cscal(f, S::neg(inv));
            else A[r * ld + c] = cminus(A[r * ld + c], ctimes(f, A[p * ld + c]));
        }
        bsync();
    }
    return ok;
}

// Pivoted Cholesky of the hermitian Gram matrix G (n x n, smem, ld) with the
// deflation test: remaining squared norm <= dtol^2 * ref (the column's
// squared norm when it was created).  Pivot: the largest remaining relative
// squared norm, ties to the lowest index.  Produces the rank r, the r x n
// factor R in permuted column order (Rm, ld n), S = Pi_r R11^{-1} (n x r)
// and beta = R Pi^T (r x n), both in smem with leading dimension ld.
// Runs on one warp.
template <class T>
__device__ int pivoted_qr(const T* G, int ld, int n, const typename Sc<T>::R* ref, typename Sc<T>::R dtol2, T* Rm,
                          T* Sm, T* beta, int* perm, typename Sc<T>::R* dd_) {
    using S = Sc<T>;
    using R = typename S::R;
    for (int i = threadIdx.x; i < n; i += WS) {
        perm[i] = i;
        dd_[i] = S::re(G[i * ld + i]);
    }
    for (int t = threadIdx.x; t < n * n; t += WS) Rm[t] = cz<T>();
    wsync();
    int rank = n;
    for (int p = 0; p < n; ++p) {
        // pivot choice: every lane scans the same (short) candidate list;
        // dd[q] / ref[q] > dd[b] / ref[b] is tested as dd[q] ref[b] >
        // dd[b] ref[q] (both refs > 0), without divisions
        int best = -1;
        R bd = S::r(0.0), br = S::r(1.0);
        for (int q = p; q < n; ++q) {
            const R rq = ref[perm[q]];
            if (!S::gt(rq, S::r(0.0))) continue;
            if (best < 0 || S::gt(S::mul(dd_[q], br), S::mul(bd, rq))) {
                bd = dd_[q];
                br = rq;
                best = q;
            }
        }
        wsync();
        if (best < 0 || !S::gt(bd, S::mul(dtol2, br)) || !S::gt(dd_[best], S::r(0.0))) {
            rank = p;
            break;
        }
        if (best != p) {
            if (threadIdx.x == 0) {
                int tp = perm[p];
                perm[p] = perm[best];
                perm[best] = tp;
                R td = dd_[p];
                dd_[p] = dd_[best];
                dd_[best] = td;
            }
            for (int l = threadIdx.x; l < p; l += WS) {
                T tr = Rm[l * n + p];
                Rm[l * n + p] = Rm[l * n + best];
                Rm[l * n + best] = tr;
            }
            wsync();
        }
        const R rpp = S::sqrt_(dd_[p]);
        const R irpp = S::rcp(rpp);
        const int gp = perm[p];
        if (threadIdx.x == 0) Rm[p * n + p] = S::c(rpp, S::r(0.0));
        for (int r = p + 1 + threadIdx.x; r < n; r += WS) {
            const int gr = perm[r];
            T s = G[gp * ld + gr];
            for (int l = 0; l < p; ++l) s = cminus(s, ctimes(cconj(Rm[l * n + p]), Rm[l * n + r]));
            s = cscal(s, irpp);
            Rm[p * n + r] = s;
            dd_[r] = S::sub(dd_[r], cnorm2(s));
        }
        wsync();
    }
    // beta = R Pi^T : beta[c'][perm[c]] = R[c'][c]
    for (int t = threadIdx.x; t < n * n; t += WS) {
        int cp = t / n, c = t % n;
        if (cp < rank) beta[cp * ld + perm[c]] = (c >= cp) ? Rm[cp * n + c] : cz<T>();
        Sm[t / n * ld + t % n] = cz<T>();
    }
    wsync();
    // S = Pi_r R11^{-1}: lane c solves R11 y = e_c by back substitution
    // (diagonal reciprocals formed once, in dd_[])
    for (int i = threadIdx.x; i < rank; i += WS) dd_[i] = S::rcp(S::re(Rm[i * n + i]));
    wsync();
    for (int c = threadIdx.x; c < rank; c += WS) {
        for (int i = c; i >= 0; --i) {
            T s = (i == c) ? S::c(S::r(1.0), S::r(0.0)) : cz<T>();
            for (int q = i + 1; q <= c; ++q) s = cminus(s, ctimes(Rm[i * n + q], Sm[perm[q] * ld + c]));
            Sm[perm[i] * ld + c] = cscal(s, dd_[i]);
        }
    }
    wsync();
    return rank;
}

__device__ inline void tile_ij(int t, int T, int herm, int* ti, int* tj) {
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

// write the reduced slot `it` ([tile][36] order) into G / diag
template <class T>
__device__ __forceinline__ void reduce_store(T* G, int ld, typename Sc<T>::R* diag, int Tt, int herm, int nf_max,
                                             int it, typename Sc<T>::R s) {
    using S = Sc<T>;
    const int tile = it / GSL, q = it % GSL;
    int ti, tj;
    tile_ij(tile, Tt, herm, &ti, &tj);
    if (q < 32) {
        const int i = ti * 4 + ((q >> 1) >> 2), j = tj * 4 + ((q >> 1) & 3);
        if (i < nf_max && j < nf_max) {
            if (q & 1) {
                G[i * ld + j].y = s;
                if (herm && ti != tj) G[j * ld + i].y = S::neg(s);
            } else {
                G[i * ld + j].x = s;
                if (herm && ti != tj) G[j * ld + i].x = s;
            }
        }
    } else if (diag && ti == tj) {
        const int j = tj * 4 + (q - 32);
        if (j < nf_max) diag[j] = s;
    }
}

// Sum the per-CTA Gram partials ([tile][blk][36], fixed order) into G (ld,
// hermitian fill when herm) and the |y|^2 diagonal; all threads of the CTA.
// FP64 partials (FP64 storage) are summed in FP64; FP32 partials (reduced
// storage; they carry FP32 accuracy) with compensated (Kahan) FP32
// additions, the chains combined in the state's scalar.  Consecutive threads take
// consecutive slots (coalesced rows of 36); when the CTA has threads to spare,
// ng groups split the CTAs' range and their sums are added in group order;
// RC interleaved accumulators per thread keep several loads in flight (the
// partials come from L2, so the sum is latency-bound).
// Fixed order: bitwise reproducible.
template <class T>
__device__ void reduce_partials(const double* __restrict__ part, int nblk, int nf_max, int herm, T* G, int ld,
                                typename Sc<T>::R* diag, bool fp64_part) {
    using S = Sc<T>;
    using R = typename S::R;
    const int Tt = (nf_max + 3) / 4;
    const int ntiles = herm ? Tt * (Tt + 1) / 2 : Tt * Tt;
    const int items = ntiles * GSL;
    __shared__ R red[RED_MAX];
    const int ng = max(1, min((int)blockDim.x / items, RED_MAX / items));
    const int chunk = (nblk + ng - 1) / ng;
    for (int u = threadIdx.x; u < items * ng; u += blockDim.x) {
        const int it = u % items, grp = u / items;
        const int b0 = grp * chunk, b1 = min(nblk, b0 + chunk);
        const int tile = it / GSL, q = it % GSL;
        const size_t off = (size_t)tile * nblk * GSL + q;
        constexpr int RC = 8;
        R s;
        if (fp64_part) {
            const double* p = part + off;
            double a[RC];
#pragma unroll
            for (int r = 0; r < RC; ++r) a[r] = 0.0;
            int b = b0;
            for (; b + RC <= b1; b += RC)
#pragma unroll
                for (int r = 0; r < RC; ++r) a[r] += p[(size_t)(b + r) * GSL];
            for (; b < b1; ++b) a[0] += p[(size_t)b * GSL];
            double t = 0.0;
#pragma unroll
            for (int r = 0; r < RC; ++r) t += a[r];
            s = S::r(t);
        } else {
            const float* p = reinterpret_cast<const float*>(part) + off;
            float sum[RC], comp[RC];
#pragma unroll
            for (int r = 0; r < RC; ++r) sum[r] = comp[r] = 0.f;
            int b = b0;
            for (; b + RC <= b1; b += RC) {
                float y[RC];
#pragma unroll
                for (int r = 0; r < RC; ++r) y[r] = p[(size_t)(b + r) * GSL];
#pragma unroll
                for (int r = 0; r < RC; ++r) {
                    const float yy = y[r] - comp[r];
                    const float t = sum[r] + yy;
                    comp[r] = (t - sum[r]) - yy;
                    sum[r] = t;
                }
            }
            for (; b < b1; ++b) {
                const float yy = p[(size_t)b * GSL] - comp[0];
                const float t = sum[0] + yy;
                comp[0] = (t - sum[0]) - yy;
                sum[0] = t;
            }
            s = S::kahan(sum[0], comp[0]);
#pragma unroll
            for (int r = 1; r < RC; ++r) s = S::add(s, S::kahan(sum[r], comp[r]));
        }
        if (ng > 1) red[grp * items + it] = s;
        else reduce_store<T>(G, ld, diag, Tt, herm, nf_max, it, s);
    }
    if (ng > 1) {
        __syncthreads();
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            R s = red[it];
            for (int g = 1; g < ng; ++g) s = S::add(s, red[g * items + it]);
            reduce_store<T>(G, ld, diag, Tt, herm, nf_max, it, s);
        }
    }
}

// ---------------------------------------------------------------------------
// init: G0 = B^H B -> rank m_1, S0 (V_1 = B S0), rho = R Pi^T; U_{j,1} = rho
template <class T>
__global__ void small_init_kernel(SmallStateT<T>* ss, Ctl* ctl, const double2* __restrict__ G0,
                                  const double* __restrict__ ref, int m, int s, double dtol) {
    using S = Sc<T>;
    using R = typename S::R;
    extern __shared__ __align__(16) unsigned char sm[];
    T* G = (T*)sm;
    T* Rm = G + m * m;
    T* Sm = Rm + m * m;
    T* rho = Sm + m * m;
    int* perm = (int*)(rho + m * m);
    R* dd_ = (R*)(perm + M_MAX);
    R* rf = dd_ + M_MAX;
    for (int t = threadIdx.x; t < m * m; t += WS) {
        const double2 g = G0[(t / m) * M_MAX + t % m];
        G[t] = S::c(S::r(g.x), S::r(g.y));
        rho[t] = cz<T>();
    }
    for (int i = threadIdx.x; i < m; i += WS) rf[i] = S::r(ref[i]);
    wsync();
    const int r = pivoted_qr<T>(G, m, m, rf, S::r(dtol * dtol), Rm, Sm, rho, perm, dd_);
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += WS) {
        const int i = t / M_MAX, j = t % M_MAX;
        ss->sh.S[t] = (i < m && j < m) ? Sm[i * m + j] : cz<T>();
        const T v = (i < r && j < m) ? rho[i * m + j] : cz<T>();
        for (int q = 0; q < s; ++q) {
            ss->sf[q].U[t] = v;
            ss->sf[q].Lam[t] = cz<T>();
        }
    }
    for (int q = 0; q < s; ++q) {
        for (int t = threadIdx.x; t < M_MAX; t += WS) ss->sf[q].conv[t] = 0;
        if (threadIdx.x == 0) ss->sf[q].alive = 1;
    }
    if (threadIdx.x == 0) {
        ctl->k = 1;
        ctl->mk = r;
        ctl->mprev = 0;
        ctl->mnext = 0;
        ctl->done = (r == 0);
        ctl->status = 0;
        ctl->nact = s;
        ctl->deflations = m - r;
        ctl->mvms = 0;
        ctl->last_step = 0;
        ctl->f_dslash = ctl->f_gram = ctl->f_update = ctl->f_shift_s = ctl->f_shift_w = ctl->f_shift_cmac = 0;
    }
}

// alpha_k from the Gram partials of the upper tiles of V_k^H Y (alpha_k =
// V_k^H A V_k is hermitian; the lower tiles are the conjugates of the upper
// ones, the diagonal tiles are hermitised); coef_a = alpha and
// coef_bh = beta_k^H in the work precision (M_MAX tiles); ||y_i||^2
template <class T>
__global__ void small_alpha_kernel(SmallStateT<T>* ss, const Ctl* __restrict__ ctl, const double* __restrict__ part,
                                   int nblk, int nf_max, int wprec, void* coef_a, void* coef_bh) {
    using S = Sc<T>;
    using R = typename S::R;
    if (ctl->done) return;
    __shared__ T A[M_MAX * M_MAX];
    __shared__ R yy[M_MAX];
    reduce_partials<T>(part, nblk, nf_max, 1, A, M_MAX, yy, wprec == P64);
    __syncthreads();
    const int mk_ = ctl->mk, mp = ctl->k > 1 ? ctl->mprev : 0;
    const R half = S::r(0.5);
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
        int i = t / M_MAX, j = t % M_MAX;
        T v = cz<T>();
        if (i < mk_ && j < mk_) v = cscal(cplus(A[i * M_MAX + j], cconj(A[j * M_MAX + i])), half);
        ss->sh.alpha[t] = v;
        const T bh = (i < mp && j < mk_) ? cconj(ss->sh.betak[j * M_MAX + i]) : cz<T>();
        if constexpr (is_fp64<T>()) {
            if (wprec == P64) {
                ((double2*)coef_a)[t] = v;
                ((double2*)coef_bh)[t] = bh;
                continue;
            }
        }
        ((float2*)coef_a)[t] = S::f2(v);
        ((float2*)coef_bh)[t] = S::f2(bh);
    }
    R* yys = reinterpret_cast<R*>(ss->sh.yy);
    for (int t = threadIdx.x; t < M_MAX; t += blockDim.x) yys[t] = t < mk_ ? yy[t] : S::r(0.0);
}

// One block step's m x m work, one CTA per shift: reduce G = W^H W from the
// partials, pivoted QR (every CTA computes the same deterministic result;
// CTA 0 publishes S, beta_{k+1}, m_{k+1}), then this shift's recurrences.
template <class T>
__global__ void small_step_kernel(SmallStateT<T>* ss, Ctl* ctl, const double* __restrict__ part, int nblk, int m,
                                  double dtol, const double* __restrict__ sigma, const double* __restrict__ target,
                                  int freeze, int wprec, void* coefS_w, void* coefU_w, void* coefL_w, int* active,
                                  int* conv_step, double* res_out, int MM) {
    using S = Sc<T>;
    using R = typename S::R;
    if (ctl->done) return;
    extern __shared__ __align__(16) unsigned char sm[];
    T* G = (T*)sm;
    T* Rm = G + MM * MM;
    T* Bn = Rm + MM * MM;       // beta_{k+1} (mn x mk)
    T* Sm = Bn + MM * MM;       // mk x mn
    T* Dl = Sm + MM * MM;       // Delta -> Delta^{-1}
    T* T1 = Dl + MM * MM;
    T* Ut = T1 + MM * MM;
    T* LH = Ut + MM * MM;
    T* Cc = LH + MM * MM;
    T* col = Cc + MM * MM;
    R* res = (R*)(col + MM);
    R* dd_ = res + MM;
    R* rf = dd_ + MM;
    int* perm = (int*)(rf + MM);
    const int j = blockIdx.x;
    const int k = ctl->k, mk_ = ctl->mk, mp = k > 1 ? ctl->mprev : 0;
    reduce_partials<T>(part, nblk, m, 1, G, MM, nullptr, wprec == P64);
    const R* yys = reinterpret_cast<const R*>(ss->sh.yy);
    for (int i = threadIdx.x; i < mk_; i += blockDim.x) rf[i] = yys[i];
    for (int t = threadIdx.x; t < MM * MM; t += blockDim.x) Bn[t] = cz<T>();
    __shared__ int mn_s;
    bsync();
    if (threadIdx.x < WS) {
        const int r = pivoted_qr<T>(G, MM, mk_, rf, S::r(dtol * dtol), Rm, Sm, Bn, perm, dd_);
        if (threadIdx.x == 0) mn_s = r;
    }
    bsync();
    const int mn = mn_s;
    if (j == 0) {
        for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
            const int a = t / M_MAX, b = t % M_MAX;
            const T sv = (a < mk_ && b < mn) ? Sm[a * MM + b] : cz<T>();
            ss->sh.S[t] = sv;
            ss->sh.betan[t] = (a < mn && b < mk_) ? Bn[a * MM + b] : cz<T>();
            if constexpr (is_fp64<T>()) {
                if (wprec == P64) {
                    ((double2*)coefS_w)[t] = sv;
                    continue;
                }
            }
            ((float2*)coefS_w)[t] = S::f2(sv);
        }
        if (threadIdx.x == 0) {
            ctl->mnext = mn;
            ctl->deflations += mk_ - mn;
        }
    }
    SmallShiftT<T>& sf = ss->sf[j];
    if (!sf.alive) {
        if (threadIdx.x == 0) active[j] = 0;
        return;
    }
    const size_t tile = (size_t)M_MAX * M_MAX;
    const size_t cb = wprec == P64 ? 16 : 8;
    // Delta_k = alpha_k + sigma I - Lambda_k beta_k^H
    ld_mat<T>(Dl, MM, ss->sh.alpha, mk_, mk_, mk_, mk_);
    if (k > 1 && mp > 0) ld_mat<T>(T1, MM, sf.Lam, mk_, mp, mk_, mp);
    bsync();
    if (k > 1 && mp > 0) gemm<T>(Dl, MM, T1, MM, 0, ss->sh.betak, M_MAX, 1, mk_, mp, mk_, true, true);
    const R sj = S::r(sigma[j]);
    for (int i = threadIdx.x; i < mk_; i += blockDim.x) Dl[i * MM + i].x = S::add(Dl[i * MM + i].x, sj);
    bsync();
    const R half = S::r(0.5);
    for (int t = threadIdx.x; t < mk_ * mk_; t += blockDim.x) {      // exact hermitian symmetry
        int a = t / mk_, b = t % mk_;
        if (b < a) {
            const T h = cscal(cplus(Dl[a * MM + b], cconj(Dl[b * MM + a])), half);
            Dl[a * MM + b] = h;
            Dl[b * MM + a] = cconj(h);
        }
    }
    bsync();
    if (!gj_inverse<T>(Dl, MM, mk_, col)) {
        if (threadIdx.x == 0) {
            atomicCAS(&ctl->status, 0, ST_NOT_HPD);
            active[j] = 0;
            sf.alive = 0;
        }
        return;
    }
    // Ut = Delta^{-1} U_k (mk x m); Lambda_{k+1}^H = Delta^{-1} beta_{k+1}^H (mk x mn)
    ld_mat<T>(T1, MM, sf.U, mk_, m, mk_, m);
    bsync();
    gemm<T>(Ut, MM, Dl, MM, 0, T1, MM, 0, mk_, mk_, m, false, false);
    gemm<T>(LH, MM, Dl, MM, 0, Bn, MM, 1, mk_, mk_, mn, false, false);
    // C = -beta_{k+1} Ut (mn x m) gives the residual estimates, and it is also
    // U_{k+1} = -Lambda_{k+1} U_k = -beta_{k+1} Delta_k^{-1} U_k
    gemm<T>(Cc, MM, Bn, MM, 0, Ut, MM, 0, mn, mk_, m, true, false);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        R s2 = S::r(0.0);
        for (int c = 0; c < mn; ++c) s2 = S::add(s2, cnorm2(Cc[c * MM + i]));
        res[i] = S::sqrt_(s2);
    }
    bsync();
    // shift-update coefficients: Ut with the columns frozen before this step zeroed
    for (int t = threadIdx.x; t < mk_ * m; t += blockDim.x) {
        int a = t / m, i = t % m;
        if (freeze && sf.conv[i]) Ut[a * MM + i] = cz<T>();
    }
    bsync();
    st_mat_work<T>(wprec, (char*)coefU_w + (size_t)j * tile * cb, Ut, MM, mk_, m);
    st_mat_work<T>(wprec, (char*)coefL_w + (size_t)j * tile * cb, LH, MM, mk_, mn);
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
        int c = t / M_MAX, a = t % M_MAX;
        sf.Lam[t] = (c < mn && a < mk_) ? cconj(LH[a * MM + c]) : cz<T>();
        sf.U[t] = (c < mn && a < m) ? Cc[c * MM + a] : cz<T>();
    }
    bsync();
    if (threadIdx.x == 0) {
        int any_before = 0, any_after = 0;
        for (int i = 0; i < m; ++i) {
            if (!sf.conv[i]) any_before = 1;
            const double ri = S::d(res[i]);
            res_out[(size_t)j * m + i] = ri;
            if (!sf.conv[i] && ri <= target[(size_t)j * m + i]) {
                sf.conv[i] = 1;
                if (conv_step) conv_step[(size_t)j * m + i] = k;
            }
            if (!sf.conv[i]) any_after = 1;
        }
        active[j] = freeze ? any_before : 1;
        sf.alive = any_after;
    }
}

// scalar-independent: counters, beta_k <- beta_{k+1} (16-byte entries), k++
__global__ void small_finish_kernel(SmallState* ss, Ctl* ctl, int s, int m, const int* __restrict__ active) {
    if (ctl->done) return;
    int nalive = 0, nkd = 0;
    for (int j = 0; j < s; ++j) {
        nalive += ss->sf[j].alive;
        nkd += active[j];
    }
    const int mk_ = ctl->mk, mn = ctl->mnext, mp = ctl->k > 1 ? ctl->mprev : 0;
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) ss->sh.betak[t] = ss->sh.betan[t];
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->mvms += mk_;
        ctl->f_dslash += 4LL * mk_;                 // D: V in, Z out; D^H: Z in, Y out
        ctl->f_gram += 3LL * mk_;                   // V, Y for alpha; W for W^H W
        ctl->f_update += 3LL * mk_ + mp + mk_ + mn; // Y, V_k, V_{k-1} in, W out; V_{k+1} = W S
        if (nkd > 0) ctl->f_shift_s += mn;          // V_{k+1} rows, read once per row tile
        ctl->f_shift_cmac += (long long)nkd * mk_ * (m + mn);   // X_j += P_j Ut_j, P_j <- V - P_j Lh_j
        ctl->hmk[(ctl->k - 1) & (CTL_HIST - 1)] = mk_;
        ctl->hmn[(ctl->k - 1) & (CTL_HIST - 1)] = mn;
        ctl->last_step = ctl->k;
        ctl->nact = nalive;
        ctl->k += 1;
        ctl->mprev = mk_;
        ctl->mk = mn;
        if (mn == 0 || nalive == 0 || ctl->status != 0) ctl->done = 1;
    }
}

size_t step_smem(int MM) {
    return 9 * (size_t)MM * MM * sizeof(double2) + MM * sizeof(double2) + 3 * MM * sizeof(double) + M_MAX * sizeof(int);
}

template <class T>
SmallStateT<T>* as_state(SmallState* ss) { return reinterpret_cast<SmallStateT<T>*>(ss); }

}  // namespace

// sfp64: FP64 m x m scalar (FP64 storage, or reduced storage on request),
// otherwise double-float; wprec: precision of the Gram partials (FP64 for
// FP64 storage, else FP32) and of the coefficient copies
void launch_small_init(SmallState* ss, Ctl* ctl, const double2* G0, const double* ref, int m, int s, double dtol,
                       int sfp64, cudaStream_t st) {
    size_t sm = 4 * (size_t)m * m * sizeof(double2) + M_MAX * sizeof(int) + 2 * M_MAX * sizeof(double);
    // above 48 KB from m = 28 on
    const int sm_max = (int)(4 * (size_t)M_MAX * M_MAX * sizeof(double2) + M_MAX * sizeof(int) + 2 * M_MAX * sizeof(double));
    static std::atomic<unsigned long long> devs64{0}, devsdd{0};
    max_dyn_smem_once(small_init_kernel<double2>, sm_max, devs64);
    max_dyn_smem_once(small_init_kernel<ddc>, sm_max, devsdd);
    if (sfp64)
        small_init_kernel<double2><<<1, WS, sm, st>>>(as_state<double2>(ss), ctl, G0, ref, m, s, dtol);
    else
        small_init_kernel<ddc><<<1, WS, sm, st>>>(as_state<ddc>(ss), ctl, G0, ref, m, s, dtol);
}

void launch_small_alpha(SmallState* ss, const Ctl* ctl, const double* partials, int nblk, int nf_max, int wprec,
                        int sfp64, void* coef_a, void* coef_bh, cudaStream_t st) {
    if (sfp64)
        small_alpha_kernel<double2><<<1, NT, 0, st>>>(as_state<double2>(ss), ctl, partials, nblk, nf_max, wprec,
                                                      coef_a, coef_bh);
    else
        small_alpha_kernel<ddc><<<1, NT, 0, st>>>(as_state<ddc>(ss), ctl, partials, nblk, nf_max, wprec, coef_a,
                                                  coef_bh);
}

void launch_small_step(SmallState* ss, Ctl* ctl, const double* partials, int nblk, int s, int m, double dtol,
                       const double* sigma_dev, const double* target_dev, int freeze, int wprec, int sfp64,
                       void* coefS_w, void* coefU_w, void* coefL_w, int* active, int* conv_step, double* res_out,
                       cudaStream_t st) {
    const int MM = m;                  // block widths never exceed the initial width m
    static std::atomic<unsigned long long> devs64{0}, devsdd{0};
    max_dyn_smem_once(small_step_kernel<double2>, (int)step_smem(M_MAX), devs64);
    max_dyn_smem_once(small_step_kernel<ddc>, (int)step_smem(M_MAX), devsdd);
    if (sfp64)
        small_step_kernel<double2><<<s, NT, step_smem(MM), st>>>(as_state<double2>(ss), ctl, partials, nblk, m, dtol,
                                                                 sigma_dev, target_dev, freeze, wprec, coefS_w,
                                                                 coefU_w, coefL_w, active, conv_step, res_out, MM);
    else
        small_step_kernel<ddc><<<s, NT, step_smem(MM), st>>>(as_state<ddc>(ss), ctl, partials, nblk, m, dtol,
                                                             sigma_dev, target_dev, freeze, wprec, coefS_w, coefU_w,
                                                             coefL_w, active, conv_step, res_out, MM);
}

void launch_small_finish(SmallState* ss, Ctl* ctl, int s, int m, const int* active, cudaStream_t st) {
    small_finish_kernel<<<1, 128, 0, st>>>(ss, ctl, s, m, active);
}

}  // namespace dsbcg

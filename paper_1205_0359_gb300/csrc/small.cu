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
// (||A v_i||^2) are dropped, so m_{k+1} <= m_k.
#include <math.h>

#include "kernels.h"

namespace dsbcg {

struct SmallShared {
    double2 alpha[M_MAX * M_MAX];    // alpha_k (hermitised)
    double2 betak[M_MAX * M_MAX];    // beta_k    (m_k x m_{k-1})
    double2 betan[M_MAX * M_MAX];    // beta_{k+1} (m_{k+1} x m_k)
    double2 S[M_MAX * M_MAX];        // V_{k+1} = W S (m_k x m_{k+1})
    double yy[M_MAX];                // ||A v_i||^2
};
struct SmallShift {
    double2 Lam[M_MAX * M_MAX];      // Lambda_k (m_k x m_{k-1})
    double2 U[M_MAX * M_MAX];        // U_k (m_k x m)
    int conv[M_MAX];                 // right-hand side i frozen
    int alive;                       // some column not converged
    int pad[M_MAX - 1];
};
struct SmallState {
    SmallShared sh;
    SmallShift sf[1];                // [s]
};

size_t small_state_bytes(int s) { return sizeof(SmallShared) + (size_t)s * sizeof(SmallShift); }
const double2* small_state_S(const SmallState* ss) { return ss->sh.S; }

namespace {

// All m x m arithmetic runs on the first warp of a CTA and synchronises with
// __syncwarp: the matrices are at most 32 x 32, so one warp has enough
// parallelism and block-wide barriers would dominate the run time.
constexpr int WS = 32;
constexpr int NT = 256;            // threads of the CTAs that also reduce partial sums
constexpr int GSL = 36;            // slots per 4 x 4 tile in the Gram partials
constexpr int RED_MAX = 1024;      // group sums held in shared memory by reduce_partials

__device__ __forceinline__ double2 z2() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void wsync() { __syncwarp(); }

// Block-wide helpers (all threads of the CTA, __syncthreads): GB300 issues
// FP64 at a small fraction of the FP32 rate per SM sub-partition, so the
// m x m products are spread over all four of them.
__device__ __forceinline__ void bsync() { __syncthreads(); }

// dst (r x c valid, R x Cc written, leading dim ld) <- src (M_MAX layout)
__device__ void ld_mat(double2* dst, int ld, const double2* src, int r, int c, int R, int Cc) {
    for (int t = threadIdx.x; t < R * Cc; t += blockDim.x) {
        int i = t / Cc, j = t % Cc;
        dst[i * ld + j] = (i < r && j < c) ? src[i * M_MAX + j] : z2();
    }
}
// full M_MAX x M_MAX tile in the work precision, zero outside r x c
template <class C>
__device__ void st_mat_w(C* dst, const double2* src, int ld, int r, int c) {
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
        int i = t / M_MAX, j = t % M_MAX;
        double2 v = (i < r && j < c) ? src[i * ld + j] : z2();
        dst[t] = mk((decltype(dst[0].x))v.x, (decltype(dst[0].x))v.y);
    }
}
__device__ void st_mat_work(int wprec, void* dst, const double2* src, int ld, int r, int c) {
    if (wprec == P64)
        st_mat_w((double2*)dst, src, ld, r, c);
    else
        st_mat_w((float2*)dst, src, ld, r, c);
}

// C (r x c) = alpha op(A) op(B) + beta C; op: 0 plain, 1 conjugate transpose
__device__ void gemm(double2* Cm, int ldc, const double2* A, int lda, int ta, const double2* B, int ldb, int tb,
                     int r, int q, int c, double alpha, double beta) {
    for (int t = threadIdx.x; t < r * c; t += blockDim.x) {
        int i = t / c, j = t % c;
        double2 s = z2();
        for (int l = 0; l < q; ++l) {
            double2 a = ta ? conjd(A[l * lda + i]) : A[i * lda + l];
            double2 b = tb ? conjd(B[j * ldb + l]) : B[l * ldb + j];
            s.x += a.x * b.x - a.y * b.y;
            s.y += a.x * b.y + a.y * b.x;
        }
        double2 o = beta != 0.0 ? Cm[i * ldc + j] : z2();
        Cm[i * ldc + j] = make_double2(beta * o.x + alpha * s.x, beta * o.y + alpha * s.y);
    }
    bsync();
}

// In-place inverse of a hermitian positive definite n x n matrix by
// Gauss-Jordan elimination without pivoting (its pivots are the Schur
// complement diagonals, positive for hpd).  Returns 0 if a pivot is <= 0.
__device__ int gj_inverse(double2* A, int ld, int n, double2* col) {
    int ok = 1;
    for (int p = 0; p < n; ++p) {
        double d = A[p * ld + p].x;
        if (!(d > 0.0)) {
            ok = 0;
            d = 1.0;
        }
        const double inv = 1.0 / d;
        for (int r = threadIdx.x; r < n; r += blockDim.x) col[r] = A[r * ld + p];
        bsync();
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            double2 v = A[p * ld + c];
            A[p * ld + c] = (c == p) ? make_double2(inv, 0.0) : make_double2(v.x * inv, v.y * inv);
        }
        bsync();
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            int r = t / n, c = t % n;
            if (r == p) continue;
            double2 f = col[r];
            if (c == p) {
                A[r * ld + p] = make_double2(-f.x * inv, -f.y * inv);
            } else {
                double2 a = A[p * ld + c], v = A[r * ld + c];
                v.x -= f.x * a.x - f.y * a.y;
                v.y -= f.x * a.y + f.y * a.x;
                A[r * ld + c] = v;
            }
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
__device__ int pivoted_qr(const double2* G, int ld, int n, const double* ref, double dtol, double2* Rm,
                          double2* S, double2* beta, int* perm, double* dd) {
    for (int i = threadIdx.x; i < n; i += WS) {
        perm[i] = i;
        dd[i] = G[i * ld + i].x;
    }
    for (int t = threadIdx.x; t < n * n; t += WS) Rm[t] = z2();
    wsync();
    int rank = n;
    for (int p = 0; p < n; ++p) {
        // pivot choice: every lane scans the same (short) candidate list;
        // dd[q] / ref[q] > dd[b] / ref[b] is tested as dd[q] ref[b] >
        // dd[b] ref[q] (both refs > 0), without FP64 divisions (slow on GB300)
        int best = -1;
        double bd = 0.0, br = 1.0;
        for (int q = p; q < n; ++q) {
            const double r = ref[perm[q]];
            if (!(r > 0.0)) continue;
            if (best < 0 || dd[q] * br > bd * r) {
                bd = dd[q];
                br = r;
                best = q;
            }
        }
        wsync();
        if (best < 0 || !(bd > dtol * dtol * br) || !(dd[best] > 0.0)) {
            rank = p;
            break;
        }
        if (best != p) {
            if (threadIdx.x == 0) {
                int tp = perm[p];
                perm[p] = perm[best];
                perm[best] = tp;
                double td = dd[p];
                dd[p] = dd[best];
                dd[best] = td;
            }
            for (int l = threadIdx.x; l < p; l += WS) {
                double2 tr = Rm[l * n + p];
                Rm[l * n + p] = Rm[l * n + best];
                Rm[l * n + best] = tr;
            }
            wsync();
        }
        const double rpp = sqrt(dd[p]);
        const double irpp = 1.0 / rpp;
        const int gp = perm[p];
        if (threadIdx.x == 0) Rm[p * n + p] = make_double2(rpp, 0.0);
        for (int r = p + 1 + threadIdx.x; r < n; r += WS) {
            const int gr = perm[r];
            double2 s = G[gp * ld + gr];
            for (int l = 0; l < p; ++l) {
                double2 a = conjd(Rm[l * n + p]), b = Rm[l * n + r];
                s.x -= a.x * b.x - a.y * b.y;
                s.y -= a.x * b.y + a.y * b.x;
            }
            s = make_double2(s.x * irpp, s.y * irpp);
            Rm[p * n + r] = s;
            dd[r] -= s.x * s.x + s.y * s.y;
        }
        wsync();
    }
    // beta = R Pi^T : beta[c'][perm[c]] = R[c'][c]
    for (int t = threadIdx.x; t < n * n; t += WS) {
        int cp = t / n, c = t % n;
        if (cp < rank) beta[cp * ld + perm[c]] = (c >= cp) ? Rm[cp * n + c] : z2();
        S[t / n * ld + t % n] = z2();
    }
    wsync();
    // S = Pi_r R11^{-1}: lane c solves R11 y = e_c by back substitution
    // (diagonal reciprocals formed once, in dd[])
    for (int i = threadIdx.x; i < rank; i += WS) dd[i] = 1.0 / Rm[i * n + i].x;
    wsync();
    for (int c = threadIdx.x; c < rank; c += WS) {
        for (int i = c; i >= 0; --i) {
            double2 s = (i == c) ? make_double2(1.0, 0.0) : z2();
            for (int q = i + 1; q <= c; ++q) {
                double2 a = Rm[i * n + q], b = S[perm[q] * ld + c];
                s.x -= a.x * b.x - a.y * b.y;
                s.y -= a.x * b.y + a.y * b.x;
            }
            const double id = dd[i];
            S[perm[i] * ld + c] = make_double2(s.x * id, s.y * id);
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

// Sum the per-CTA Gram partials ([tile][blk][36], fixed order) into G (ld,
// hermitian fill when herm) and the |y|^2 diagonal; all threads of the CTA.
// With reduced-precision storage the partials are FP32 (they carry FP32
// accuracy) and are summed with compensated (Kahan) FP32 additions, which
// cost far less than FP64 ones on GB300; FP64 storage sums in FP64.
// write the reduced slot `it` ([tile][36] order) into G / diag
__device__ __forceinline__ void reduce_store(double2* G, int ld, double* diag, int T, int herm, int nf_max, int it,
                                             double s) {
    const int tile = it / GSL, q = it % GSL;
    int ti, tj;
    tile_ij(tile, T, herm, &ti, &tj);
    if (q < 32) {
        const int i = ti * 4 + ((q >> 1) >> 2), j = tj * 4 + ((q >> 1) & 3);
        if (i < nf_max && j < nf_max) {
            if (q & 1) {
                G[i * ld + j].y = s;
                if (herm && ti != tj) G[j * ld + i].y = -s;
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

__device__ void reduce_partials(const double* __restrict__ part, int nblk, int nf_max, int herm, double2* G, int ld,
                                double* diag, int fp64) {
    const int T = (nf_max + 3) / 4;
    const int ntiles = herm ? T * (T + 1) / 2 : T * T;
    const int items = ntiles * GSL;
    // consecutive threads take consecutive slots (coalesced rows of 36); when
    // the CTA has threads to spare, ng groups split the CTAs' range and their
    // sums are added in group order; four interleaved accumulators per
    // thread keep several loads in flight.  Fixed order: bitwise reproducible.
    __shared__ double red[RED_MAX];
    const int ng = max(1, min((int)blockDim.x / items, RED_MAX / items));
    const int chunk = (nblk + ng - 1) / ng;
    for (int u = threadIdx.x; u < items * ng; u += blockDim.x) {
        const int it = u % items, grp = u / items;
        const int b0 = grp * chunk, b1 = min(nblk, b0 + chunk);
        const int tile = it / GSL, q = it % GSL;
        const size_t off = (size_t)tile * nblk * GSL + q;
        double s = 0.0;
        if (fp64) {
            const double* p = part + off;
            double a[4] = {0.0, 0.0, 0.0, 0.0};
            int b = b0;
            for (; b + 4 <= b1; b += 4)
#pragma unroll
                for (int r = 0; r < 4; ++r) a[r] += p[(size_t)(b + r) * GSL];
            for (; b < b1; ++b) a[0] += p[(size_t)b * GSL];
            s = (a[0] + a[1]) + (a[2] + a[3]);
        } else {
            const float* p = reinterpret_cast<const float*>(part) + off;
            float sum[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
            int b = b0;
            for (; b + 4 <= b1; b += 4) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float y = p[(size_t)(b + r) * GSL] - comp[r];
                    const float t = sum[r] + y;
                    comp[r] = (t - sum[r]) - y;
                    sum[r] = t;
                }
            }
            for (; b < b1; ++b) {
                const float y = p[(size_t)b * GSL] - comp[0];
                const float t = sum[0] + y;
                comp[0] = (t - sum[0]) - y;
                sum[0] = t;
            }
            s = ((double)sum[0] - (double)comp[0]) + ((double)sum[1] - (double)comp[1]) +
                (((double)sum[2] - (double)comp[2]) + ((double)sum[3] - (double)comp[3]));
        }
        if (ng > 1) red[grp * items + it] = s;
        else reduce_store(G, ld, diag, T, herm, nf_max, it, s);
    }
    if (ng > 1) {
        __syncthreads();
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            double s = 0.0;
            for (int g = 0; g < ng; ++g) s += red[g * items + it];
            reduce_store(G, ld, diag, T, herm, nf_max, it, s);
        }
    }
}

// ---------------------------------------------------------------------------
// init: G0 = B^H B -> rank m_1, S0 (V_1 = B S0), rho = R Pi^T; U_{j,1} = rho
__global__ void small_init_kernel(SmallState* ss, Ctl* ctl, const double2* __restrict__ G0,
                                  const double* __restrict__ ref, int m, int s, double dtol) {
    extern __shared__ __align__(16) unsigned char sm[];
    double2* G = (double2*)sm;
    double2* Rm = G + m * m;
    double2* S = Rm + m * m;
    double2* rho = S + m * m;
    int* perm = (int*)(rho + m * m);
    double* dd = (double*)(perm + M_MAX);
    double* rf = dd + M_MAX;
    ld_mat(G, m, G0, m, m, m, m);
    for (int i = threadIdx.x; i < m; i += WS) rf[i] = ref[i];
    for (int t = threadIdx.x; t < m * m; t += WS) rho[t] = z2();
    wsync();
    const int r = pivoted_qr(G, m, m, rf, dtol, Rm, S, rho, perm, dd);
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += WS) {
        const int i = t / M_MAX, j = t % M_MAX;
        ss->sh.S[t] = (i < m && j < m) ? S[i * m + j] : z2();
        const double2 v = (i < r && j < m) ? rho[i * m + j] : z2();
        for (int q = 0; q < s; ++q) {
            ss->sf[q].U[t] = v;
            ss->sf[q].Lam[t] = z2();
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
        ctl->f_dslash = ctl->f_gram = ctl->f_update = ctl->f_shift_s = ctl->f_shift_w = 0;
    }
}

// alpha_k from the Gram partials of V_k^H Y, hermitised; coef_a = alpha and
// coef_bh = beta_k^H in the work precision (M_MAX tiles); ||y_i||^2
__global__ void small_alpha_kernel(SmallState* ss, const Ctl* __restrict__ ctl, const double* __restrict__ part,
                                   int nblk, int nf_max, int wprec, void* coef_a, void* coef_bh) {
    if (ctl->done) return;
    __shared__ double2 A[M_MAX * M_MAX];
    __shared__ double yy[M_MAX];
    reduce_partials(part, nblk, nf_max, 0, A, M_MAX, yy, wprec == P64);
    __syncthreads();
    const int mk_ = ctl->mk, mp = ctl->k > 1 ? ctl->mprev : 0;
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
        int i = t / M_MAX, j = t % M_MAX;
        double2 v = z2();
        if (i < mk_ && j < mk_) {
            double2 a = A[i * M_MAX + j], b = A[j * M_MAX + i];
            v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        }
        ss->sh.alpha[t] = v;
        double2 bh = (i < mp && j < mk_) ? conjd(ss->sh.betak[j * M_MAX + i]) : z2();
        if (wprec == P64) {
            ((double2*)coef_a)[t] = v;
            ((double2*)coef_bh)[t] = bh;
        } else {
            ((float2*)coef_a)[t] = make_float2((float)v.x, (float)v.y);
            ((float2*)coef_bh)[t] = make_float2((float)bh.x, (float)bh.y);
        }
    }
    for (int t = threadIdx.x; t < M_MAX; t += blockDim.x) ss->sh.yy[t] = t < mk_ ? yy[t] : 0.0;
}

// One block step's m x m work, one CTA per shift: reduce G = W^H W from the
// partials, pivoted QR (every CTA computes the same deterministic result;
// CTA 0 publishes S, beta_{k+1}, m_{k+1}), then this shift's recurrences.
__global__ void small_step_kernel(SmallState* ss, Ctl* ctl, const double* __restrict__ part, int nblk, int m,
                                  double dtol, const double* __restrict__ sigma, const double* __restrict__ target,
                                  int freeze, int wprec, void* coefS_w, void* coefU_w, void* coefL_w, int* active,
                                  int* conv_step, double* res_out, int MM) {
    if (ctl->done) return;
    extern __shared__ __align__(16) unsigned char sm[];
    double2* G = (double2*)sm;
    double2* Rm = G + MM * MM;
    double2* Bn = Rm + MM * MM;       // beta_{k+1} (mn x mk)
    double2* S = Bn + MM * MM;        // mk x mn
    double2* Dl = S + MM * MM;        // Delta -> Delta^{-1}
    double2* T1 = Dl + MM * MM;
    double2* Ut = T1 + MM * MM;
    double2* LH = Ut + MM * MM;
    double2* Cc = LH + MM * MM;
    double2* col = Cc + MM * MM;
    double* res = (double*)(col + MM);
    double* dd = res + MM;
    double* rf = dd + MM;
    int* perm = (int*)(rf + MM);
    const int j = blockIdx.x;
    const int k = ctl->k, mk_ = ctl->mk, mp = k > 1 ? ctl->mprev : 0;
    reduce_partials(part, nblk, m, 1, G, MM, nullptr, wprec == P64);
    for (int i = threadIdx.x; i < mk_; i += blockDim.x) rf[i] = ss->sh.yy[i];
    for (int t = threadIdx.x; t < MM * MM; t += blockDim.x) Bn[t] = z2();
    __shared__ int mn_s;
    bsync();
    if (threadIdx.x < WS) {
        const int r = pivoted_qr(G, MM, mk_, rf, dtol, Rm, S, Bn, perm, dd);
        if (threadIdx.x == 0) mn_s = r;
    }
    bsync();
    const int mn = mn_s;
    if (j == 0) {
        for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
            const int a = t / M_MAX, b = t % M_MAX;
            const double2 sv = (a < mk_ && b < mn) ? S[a * MM + b] : z2();
            ss->sh.S[t] = sv;
            ss->sh.betan[t] = (a < mn && b < mk_) ? Bn[a * MM + b] : z2();
            if (wprec == P64)
                ((double2*)coefS_w)[t] = sv;
            else
                ((float2*)coefS_w)[t] = make_float2((float)sv.x, (float)sv.y);
        }
        if (threadIdx.x == 0) {
            ctl->mnext = mn;
            ctl->deflations += mk_ - mn;
        }
    }
    SmallShift& sf = ss->sf[j];
    if (!sf.alive) {
        if (threadIdx.x == 0) active[j] = 0;
        return;
    }
    const size_t tile = (size_t)M_MAX * M_MAX;
    const size_t cb = wprec == P64 ? 16 : 8;
    // Delta_k = alpha_k + sigma I - Lambda_k beta_k^H
    ld_mat(Dl, MM, ss->sh.alpha, mk_, mk_, mk_, mk_);
    if (k > 1 && mp > 0) ld_mat(T1, MM, sf.Lam, mk_, mp, mk_, mp);
    bsync();
    if (k > 1 && mp > 0) gemm(Dl, MM, T1, MM, 0, ss->sh.betak, M_MAX, 1, mk_, mp, mk_, -1.0, 1.0);
    for (int i = threadIdx.x; i < mk_; i += blockDim.x) Dl[i * MM + i].x += sigma[j];
    bsync();
    for (int t = threadIdx.x; t < mk_ * mk_; t += blockDim.x) {      // exact hermitian symmetry
        int a = t / mk_, b = t % mk_;
        if (b < a) {
            double2 lo = Dl[a * MM + b], up = Dl[b * MM + a];
            double2 h = make_double2(0.5 * (lo.x + up.x), 0.5 * (lo.y - up.y));
            Dl[a * MM + b] = h;
            Dl[b * MM + a] = conjd(h);
        }
    }
    bsync();
    if (!gj_inverse(Dl, MM, mk_, col)) {
        if (threadIdx.x == 0) {
            atomicExch(&ctl->status, ST_NOT_HPD);
            active[j] = 0;
            sf.alive = 0;
        }
        return;
    }
    // Ut = Delta^{-1} U_k (mk x m); Lambda_{k+1}^H = Delta^{-1} beta_{k+1}^H (mk x mn)
    ld_mat(T1, MM, sf.U, mk_, m, mk_, m);
    bsync();
    gemm(Ut, MM, Dl, MM, 0, T1, MM, 0, mk_, mk_, m, 1.0, 0.0);
    gemm(LH, MM, Dl, MM, 0, Bn, MM, 1, mk_, mk_, mn, 1.0, 0.0);
    // C = -beta_{k+1} Ut (mn x m) gives the residual estimates, and it is also
    // U_{k+1} = -Lambda_{k+1} U_k = -beta_{k+1} Delta_k^{-1} U_k
    gemm(Cc, MM, Bn, MM, 0, Ut, MM, 0, mn, mk_, m, -1.0, 0.0);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double s2 = 0.0;
        for (int c = 0; c < mn; ++c) s2 += Cc[c * MM + i].x * Cc[c * MM + i].x + Cc[c * MM + i].y * Cc[c * MM + i].y;
        res[i] = sqrt(s2);
    }
    bsync();
    // shift-update coefficients: Ut with the columns frozen before this step zeroed
    for (int t = threadIdx.x; t < mk_ * m; t += blockDim.x) {
        int a = t / m, i = t % m;
        if (freeze && sf.conv[i]) Ut[a * MM + i] = z2();
    }
    bsync();
    st_mat_work(wprec, (char*)coefU_w + (size_t)j * tile * cb, Ut, MM, mk_, m);
    st_mat_work(wprec, (char*)coefL_w + (size_t)j * tile * cb, LH, MM, mk_, mn);
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
        int c = t / M_MAX, a = t % M_MAX;
        sf.Lam[t] = (c < mn && a < mk_) ? conjd(LH[a * MM + c]) : z2();
        sf.U[t] = (c < mn && a < m) ? Cc[c * MM + a] : z2();
    }
    bsync();
    if (threadIdx.x == 0) {
        int any_before = 0, any_after = 0;
        for (int i = 0; i < m; ++i) {
            if (!sf.conv[i]) any_before = 1;
            res_out[(size_t)j * m + i] = res[i];
            if (!sf.conv[i] && res[i] <= target[(size_t)j * m + i]) {
                sf.conv[i] = 1;
                if (conv_step) conv_step[(size_t)j * m + i] = k;
            }
            if (!sf.conv[i]) any_after = 1;
        }
        active[j] = freeze ? any_before : 1;
        sf.alive = any_after;
    }
}

__global__ void small_finish_kernel(SmallState* ss, Ctl* ctl, int s, int m, const int* __restrict__ active) {
    if (ctl->done) return;
    int nalive = 0, nkd = 0;
    for (int j = 0; j < s; ++j) {
        nalive += ss->sf[j].alive;
        nkd += active[j];
    }
    const int mk_ = ctl->mk, mn = ctl->mnext, mp = ctl->k > 1 ? ctl->mprev : 0;
    // beta_k <- beta_{k+1}
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) ss->sh.betak[t] = ss->sh.betan[t];
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->mvms += mk_;
        ctl->f_dslash += 4LL * mk_;                 // D: V in, Z out; D^H: Z in, Y out
        ctl->f_gram += 3LL * mk_;                   // V, Y for alpha; W for W^H W
        ctl->f_update += 3LL * mk_ + mp;            // Y, V_k, V_{k-1} in, W out
        ctl->f_shift_s += (long long)mk_ + mn;      // W in, V_{k+1} out
        ctl->f_shift_w += (long long)nkd * (mk_ + mn + 2 * m);   // P_j in/out, X_j in/out
        ctl->last_step = ctl->k;
        ctl->nact = nalive;
        ctl->k += 1;
        ctl->mprev = mk_;
        ctl->mk = mn;
        if (mn == 0 || nalive == 0 || ctl->status != 0) ctl->done = 1;
    }
}

size_t step_smem(int MM) { return 9 * (size_t)MM * MM * sizeof(double2) + MM * sizeof(double2) + 3 * MM * sizeof(double) + M_MAX * sizeof(int); }

}  // namespace

void launch_small_init(SmallState* ss, Ctl* ctl, const double2* G0, const double* ref, int m, int s, double dtol,
                       cudaStream_t st) {
    size_t sm = 4 * (size_t)m * m * sizeof(double2) + M_MAX * sizeof(int) + 2 * M_MAX * sizeof(double);
    small_init_kernel<<<1, WS, sm, st>>>(ss, ctl, G0, ref, m, s, dtol);
}

void launch_small_alpha(SmallState* ss, const Ctl* ctl, const double* partials, int nblk, int nf_max, int wprec,
                        void* coef_a, void* coef_bh, cudaStream_t st) {
    small_alpha_kernel<<<1, 256, 0, st>>>(ss, ctl, partials, nblk, nf_max, wprec, coef_a, coef_bh);
}

void launch_small_step(SmallState* ss, Ctl* ctl, const double* partials, int nblk, int s, int m, double dtol,
                       const double* sigma_dev, const double* target_dev, int freeze, int wprec, void* coefS_w,
                       void* coefU_w, void* coefL_w, int* active, int* conv_step, double* res_out,
                       cudaStream_t st) {
    const int MM = m;                  // block widths never exceed the initial width m
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(small_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem(M_MAX));
        attr_set = true;
    }
    small_step_kernel<<<s, NT, step_smem(MM), st>>>(ss, ctl, partials, nblk, m, dtol, sigma_dev, target_dev, freeze,
                                                    wprec, coefS_w, coefU_w, coefL_w, active, conv_step, res_out, MM);
}

void launch_small_finish(SmallState* ss, Ctl* ctl, int s, int m, const int* active, cudaStream_t st) {
    small_finish_kernel<<<1, 128, 0, st>>>(ss, ctl, s, m, active);
}

}  // namespace dsbcg

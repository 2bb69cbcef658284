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

constexpr int NT = 128;

__device__ __forceinline__ double2 z2() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

// dst (r x c, leading dim ld) <- src (M_MAX layout), zero outside
__device__ void ld_mat(double2* dst, int ld, const double2* src, int r, int c, int R, int Cc) {
    for (int t = threadIdx.x; t < R * Cc; t += blockDim.x) {
        int i = t / Cc, j = t % Cc;
        dst[i * ld + j] = (i < r && j < c) ? src[i * M_MAX + j] : z2();
    }
}
template <class C>
__device__ void st_mat_w(C* dst, const double2* src, int ld, int r, int c) {
    // full M_MAX x M_MAX tile, zero outside r x c
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

// In-place Cholesky A = L L^H (n x n, lower part), returns 0 on failure
__device__ int chol(double2* A, int ld, int n) {
    __shared__ int ok;
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
    for (int p = 0; p < n; ++p) {
        if (threadIdx.x == 0) {
            double d = A[p * ld + p].x;
            if (!(d > 0.0)) {
                ok = 0;
                d = 1.0;
            }
            A[p * ld + p] = make_double2(sqrt(d), 0.0);
        }
        __syncthreads();
        double lpp = A[p * ld + p].x;
        for (int i = p + 1 + threadIdx.x; i < n; i += blockDim.x) {
            A[i * ld + p] = make_double2(A[i * ld + p].x / lpp, A[i * ld + p].y / lpp);
        }
        __syncthreads();
        // trailing update A_ij -= L_ip conj(L_jp), i >= j > p
        int rem = n - p - 1;
        for (int t = threadIdx.x; t < rem * rem; t += blockDim.x) {
            int i = p + 1 + t / rem, j = p + 1 + t % rem;
            if (j <= i) {
                double2 a = A[i * ld + p], b = A[j * ld + p];
                double2 v = A[i * ld + j];
                v.x -= a.x * b.x + a.y * b.y;
                v.y -= a.y * b.x - a.x * b.y;
                A[i * ld + j] = v;
            }
        }
        __syncthreads();
    }
    return ok;
}

// Solve (L L^H) X = B in place for nrhs columns of B (n x nrhs, ld ldb)
__device__ void chol_solve(const double2* L, int ld, int n, double2* B, int ldb, int nrhs) {
    for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
        // forward: L y = b
        for (int i = 0; i < n; ++i) {
            double2 s = B[i * ldb + c];
            for (int q = 0; q < i; ++q) {
                double2 l = L[i * ld + q], y = B[q * ldb + c];
                s.x -= l.x * y.x - l.y * y.y;
                s.y -= l.x * y.y + l.y * y.x;
            }
            double d = L[i * ld + i].x;
            B[i * ldb + c] = make_double2(s.x / d, s.y / d);
        }
        // backward: L^H x = y
        for (int i = n - 1; i >= 0; --i) {
            double2 s = B[i * ldb + c];
            for (int q = i + 1; q < n; ++q) {
                double2 l = conjd(L[q * ld + i]), x = B[q * ldb + c];
                s.x -= l.x * x.x - l.y * x.y;
                s.y -= l.x * x.y + l.y * x.x;
            }
            double d = L[i * ld + i].x;
            B[i * ldb + c] = make_double2(s.x / d, s.y / d);
        }
    }
    __syncthreads();
}

// C (r x c) = op(A) (r x q) * op(B) (q x c); ta/tb: 0 = plain, 1 = conj transpose
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
    __syncthreads();
}

// Pivoted Cholesky of the hermitian Gram matrix G (n x n, smem, ld) with the
// deflation test d_q <= dtol^2 ref_q.  Produces rank r, the permutation, the
// r x n factor R (permuted column order), S = Pi_r R11^{-1} (n x r) and
// beta = R Pi^T (r x n) written to global (M_MAX layout).
__device__ int pivoted_qr(double2* G, int ld, int n, const double* ref, double dtol, double2* Rm,
                          double2* Sg, double2* betag, int* perm_s, double* dd) {
    __shared__ int rank_s, piv_s;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        perm_s[i] = i;
        dd[i] = G[i * ld + i].x;
    }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) Rm[t] = z2();
    if (threadIdx.x == 0) rank_s = n;
    __syncthreads();
    for (int p = 0; p < n; ++p) {
        if (threadIdx.x == 0) {
            // largest remaining relative squared norm, ties to the lowest index
            int best = -1;
            double bv = -1.0;
            for (int q = p; q < n; ++q) {
                double r = ref[perm_s[q]];
                double v = (r > 0.0) ? dd[q] / r : -1.0;
                if (v > bv) {
                    bv = v;
                    best = q;
                }
            }
            if (best < 0 || !(bv > dtol * dtol) || !(dd[best] > 0.0)) {
                rank_s = p;
                piv_s = -1;
            } else {
                piv_s = best;
                if (best != p) {
                    int tp = perm_s[p];
                    perm_s[p] = perm_s[best];
                    perm_s[best] = tp;
                    double td = dd[p];
                    dd[p] = dd[best];
                    dd[best] = td;
                    for (int l = 0; l < p; ++l) {
                        double2 tr = Rm[l * n + p];
                        Rm[l * n + p] = Rm[l * n + best];
                        Rm[l * n + best] = tr;
                    }
                }
                Rm[p * n + p] = make_double2(sqrt(dd[p]), 0.0);
            }
        }
        __syncthreads();
        if (piv_s < 0) break;
        const double rpp = Rm[p * n + p].x;
        const int gp = perm_s[p];
        for (int r = p + 1 + threadIdx.x; r < n; r += blockDim.x) {
            const int gr = perm_s[r];
            double2 s = G[gp * ld + gr];
            for (int l = 0; l < p; ++l) {
                double2 a = conjd(Rm[l * n + p]), b = Rm[l * n + r];
                s.x -= a.x * b.x - a.y * b.y;
                s.y -= a.x * b.y + a.y * b.x;
            }
            s = make_double2(s.x / rpp, s.y / rpp);
            Rm[p * n + r] = s;
            dd[r] -= s.x * s.x + s.y * s.y;
        }
        __syncthreads();
    }
    const int r = rank_s;
    // beta = R Pi^T : beta[c'][perm[c]] = R[c'][c]
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) betag[t] = z2();
    __syncthreads();
    for (int t = threadIdx.x; t < r * n; t += blockDim.x) {
        int cp = t / n, c = t % n;
        betag[cp * M_MAX + perm_s[c]] = (c >= cp) ? Rm[cp * n + c] : z2();
    }
    // S = Pi_r R11^{-1}: invert the r x r upper triangle column by column
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) Sg[t] = z2();
    __syncthreads();
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
        // solve R11 y = e_c (back substitution), y has entries 0..c
        double2 y[M_MAX];
        for (int i = c; i >= 0; --i) {
            double2 s = (i == c) ? make_double2(1.0, 0.0) : z2();
            for (int q = i + 1; q <= c; ++q) {
                double2 a = Rm[i * n + q], b = y[q];
                s.x -= a.x * b.x - a.y * b.y;
                s.y -= a.x * b.y + a.y * b.x;
            }
            double d = Rm[i * n + i].x;
            y[i] = make_double2(s.x / d, s.y / d);
        }
        for (int i = 0; i <= c; ++i) Sg[perm_s[i] * M_MAX + c] = y[i];
    }
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// init: G0 = B^H B -> rank m_1, S0 (V_1 = B S0), rho = R Pi^T; U_{j,1} = rho
__global__ void small_init_kernel(SmallState* ss, Ctl* ctl, const double2* __restrict__ G0,
                                  const double* __restrict__ ref, int m, int s, double dtol, int wprec,
                                  void* coefS_w) {
    extern __shared__ __align__(16) unsigned char sm[];
    double2* G = (double2*)sm;
    double2* Rm = G + m * m;
    int* perm = (int*)(Rm + m * m);
    double* dd = (double*)(perm + M_MAX);
    ld_mat(G, m, G0, m, m, m, m);
    __syncthreads();
    double2* rho = ss->sh.betan;              // r x m, permuted back
    int r = pivoted_qr(G, m, m, ref, dtol, Rm, ss->sh.S, rho, perm, dd);
    for (int j = 0; j < s; ++j) {
        for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
            ss->sf[j].U[t] = rho[t];
            ss->sf[j].Lam[t] = z2();
        }
        for (int t = threadIdx.x; t < M_MAX; t += blockDim.x) ss->sf[j].conv[t] = 0;
        if (threadIdx.x == 0) ss->sf[j].alive = 1;
    }
    // coefficients of V_1 = B S0 in FP64 are read by init_basis from ss->sh.S
    (void)wprec;
    (void)coefS_w;
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

// alpha hermitised; coef_a = alpha, coef_bh = beta_k^H (work precision, M_MAX tiles)
__global__ void small_alpha_kernel(SmallState* ss, const Ctl* __restrict__ ctl, const double2* __restrict__ alpha,
                                   const double* __restrict__ yy, int wprec, void* coef_a, void* coef_bh) {
    if (ctl->done) return;
    const int mk_ = ctl->mk, mp = ctl->k > 1 ? ctl->mprev : 0;
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
        int i = t / M_MAX, j = t % M_MAX;
        double2 v = z2();
        if (i < mk_ && j < mk_) {
            double2 a = alpha[i * M_MAX + j], b = alpha[j * M_MAX + i];
            v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        }
        ss->sh.alpha[t] = v;
        // beta_k^H (m_{k-1} x m_k): (beta^H)[i][j] = conj(beta_k[j][i])
        double2 bh = (i < mp && j < mk_) ? conjd(ss->sh.betak[j * M_MAX + i]) : z2();
        if (wprec == P64) {
            ((double2*)coef_a)[t] = v;
            ((double2*)coef_bh)[t] = bh;
        } else {
            ((float2*)coef_a)[t] = make_float2((float)v.x, (float)v.y);
            ((float2*)coef_bh)[t] = make_float2((float)bh.x, (float)bh.y);
        }
    }
    for (int t = threadIdx.x; t < M_MAX; t += blockDim.x) ss->sh.yy[t] = yy[t];
}

// QR of W: G = W^H W -> m_{k+1}, S, beta_{k+1}
__global__ void small_qr_kernel(SmallState* ss, Ctl* ctl, const double2* __restrict__ Gg, double dtol, int wprec,
                                void* coefS_w) {
    if (ctl->done) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = ctl->mk;
    double2* G = (double2*)sm;
    double2* Rm = G + n * n;
    int* perm = (int*)(Rm + n * n);
    double* dd = (double*)(perm + M_MAX);
    ld_mat(G, n, Gg, n, n, n, n);
    __syncthreads();
    int r = pivoted_qr(G, n, n, ss->sh.yy, dtol, Rm, ss->sh.S, ss->sh.betan, perm, dd);
    __syncthreads();
    if (wprec == P64) {
        for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) ((double2*)coefS_w)[t] = ss->sh.S[t];
    } else {
        for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
            double2 v = ss->sh.S[t];
            ((float2*)coefS_w)[t] = make_float2((float)v.x, (float)v.y);
        }
    }
    if (threadIdx.x == 0) {
        ctl->mnext = r;
        ctl->deflations += n - r;
    }
}

// per-shift recurrences; one CTA per shift
__global__ void small_shift_kernel(SmallState* ss, Ctl* ctl, int m, const double* __restrict__ sigma,
                                   const double* __restrict__ target, int freeze, int wprec, void* coefU_w,
                                   void* coefL_w, int* active, int* conv_step, double* res_out, int MM) {
    if (ctl->done) return;
    const int j = blockIdx.x;
    SmallShift& sf = ss->sf[j];
    const size_t tile = (size_t)M_MAX * M_MAX;
    if (!sf.alive) {
        if (threadIdx.x == 0) active[j] = 0;
        return;
    }
    const int k = ctl->k, mk_ = ctl->mk, mp = k > 1 ? ctl->mprev : 0, mn = ctl->mnext;
    extern __shared__ __align__(16) unsigned char sm[];
    double2* Dl = (double2*)sm;                 // Delta -> its Cholesky factor (mk x mk)
    double2* T1 = Dl + MM * MM;                 // scratch
    double2* Ut = T1 + MM * MM;                 // Ut (mk x m)
    double2* LH = Ut + MM * MM;                 // Lambda_{k+1}^H (mk x mn)
    double2* Cc = LH + MM * MM;                 // C (mn x m), U_{k+1}
    double* res = (double*)(Cc + MM * MM);
    __shared__ int ok;

    // Delta_k = alpha_k + sigma I - Lambda_k beta_k^H
    ld_mat(Dl, MM, ss->sh.alpha, mk_, mk_, mk_, mk_);
    __syncthreads();
    if (k > 1 && mp > 0) {
        ld_mat(T1, MM, sf.Lam, mk_, mp, mk_, mp);
        __syncthreads();
        gemm(Dl, MM, T1, MM, 0, ss->sh.betak, M_MAX, 1, mk_, mp, mk_, -1.0, 1.0);
    }
    for (int i = threadIdx.x; i < mk_; i += blockDim.x) Dl[i * MM + i].x += sigma[j];
    // keep Delta exactly hermitian
    for (int t = threadIdx.x; t < mk_ * mk_; t += blockDim.x) {
        int a = t / mk_, b = t % mk_;
        if (b < a) {
            double2 lo = Dl[a * MM + b], up = Dl[b * MM + a];
            Dl[a * MM + b] = make_double2(0.5 * (lo.x + up.x), 0.5 * (lo.y - up.y));
        }
    }
    __syncthreads();
    int c_ok = chol(Dl, MM, mk_);
    if (threadIdx.x == 0) ok = c_ok;
    __syncthreads();
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicExch(&ctl->status, ST_NOT_HPD);
            active[j] = 0;
            sf.alive = 0;
        }
        return;
    }
    // Ut = Delta^{-1} U_k
    ld_mat(Ut, MM, sf.U, mk_, m, mk_, m);
    __syncthreads();
    chol_solve(Dl, MM, mk_, Ut, MM, m);
    // Lambda_{k+1}^H = Delta^{-1} beta_{k+1}^H
    for (int t = threadIdx.x; t < mk_ * mn; t += blockDim.x) {
        int a = t / mn, c = t % mn;
        LH[a * MM + c] = conjd(ss->sh.betan[c * M_MAX + a]);
    }
    __syncthreads();
    chol_solve(Dl, MM, mk_, LH, MM, mn);
    // C = -beta_{k+1} Ut  (mn x m); residual norms
    gemm(Cc, MM, ss->sh.betan, M_MAX, 0, Ut, MM, 0, mn, mk_, m, -1.0, 0.0);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double s2 = 0.0;
        for (int c = 0; c < mn; ++c) s2 += Cc[c * MM + i].x * Cc[c * MM + i].x + Cc[c * MM + i].y * Cc[c * MM + i].y;
        res[i] = sqrt(s2);
    }
    __syncthreads();
    // coefficients for the shift update: Ut with columns frozen before this step zeroed
    for (int t = threadIdx.x; t < mk_ * m; t += blockDim.x) {
        int a = t / m, i = t % m;
        if (freeze && sf.conv[i]) Ut[a * MM + i] = z2();
    }
    __syncthreads();
    st_mat_work(wprec, (char*)coefU_w + (size_t)j * tile * (wprec == P64 ? 16 : 8), Ut, MM, mk_, m);
    st_mat_work(wprec, (char*)coefL_w + (size_t)j * tile * (wprec == P64 ? 16 : 8), LH, MM, mk_, mn);
    // U_{k+1} = -Lambda_{k+1} U_k = -(LH)^H U_k  (mn x m), into Cc
    ld_mat(T1, MM, sf.U, mk_, m, mk_, m);
    __syncthreads();
    gemm(Cc, MM, LH, MM, 1, T1, MM, 0, mn, mk_, m, -1.0, 0.0);
    // store Lambda_{k+1} = LH^H (mn x mk), U_{k+1}
    for (int t = threadIdx.x; t < M_MAX * M_MAX; t += blockDim.x) {
        int c = t / M_MAX, a = t % M_MAX;
        sf.Lam[t] = (c < mn && a < mk_) ? conjd(LH[a * MM + c]) : z2();
        sf.U[t] = (c < mn && a < m) ? Cc[c * MM + a] : z2();
    }
    __syncthreads();
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
        sf.alive = any_after || !freeze;
        if (!freeze && !any_after) sf.alive = 0;
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

}  // namespace

void launch_small_init(SmallState* ss, Ctl* ctl, const double2* G0, const double* ref, int m, int s, double dtol,
                       int wprec, void* coefS_w, cudaStream_t st) {
    size_t sm = 2 * (size_t)m * m * sizeof(double2) + M_MAX * sizeof(int) + M_MAX * sizeof(double);
    small_init_kernel<<<1, NT, sm, st>>>(ss, ctl, G0, ref, m, s, dtol, wprec, coefS_w);
}

void launch_small_alpha(SmallState* ss, const Ctl* ctl, const double2* alpha, const double* yy, int wprec,
                        void* coef_a, void* coef_bh, cudaStream_t st) {
    small_alpha_kernel<<<1, 256, 0, st>>>(ss, ctl, alpha, yy, wprec, coef_a, coef_bh);
}

void launch_small_qr(SmallState* ss, Ctl* ctl, const double2* G, double dtol, int wprec, void* coefS_w,
                     cudaStream_t st) {
    size_t sm = 2 * (size_t)M_MAX * M_MAX * sizeof(double2) + M_MAX * sizeof(int) + M_MAX * sizeof(double);
    small_qr_kernel<<<1, NT, sm, st>>>(ss, ctl, G, dtol, wprec, coefS_w);
}

void launch_small_shift(SmallState* ss, Ctl* ctl, int s, int m, const double* sigma_dev, const double* target_dev,
                        int freeze, int wprec, void* coefU_w, void* coefL_w, int* active, int* conv_step,
                        double* res_out, cudaStream_t st) {
    int MM = m;                        // block widths never exceed the initial width m
    size_t sm = 5 * (size_t)MM * MM * sizeof(double2) + M_MAX * sizeof(double);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(small_shift_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(5 * M_MAX * M_MAX * sizeof(double2) + M_MAX * sizeof(double)));
        attr_set = true;
    }
    small_shift_kernel<<<s, NT, sm, st>>>(ss, ctl, m, sigma_dev, target_dev, freeze, wprec, coefU_w, coefL_w,
                                          active, conv_step, res_out, MM);
}

void launch_small_finish(SmallState* ss, Ctl* ctl, int s, int m, const int* active, cudaStream_t st) {
    small_finish_kernel<<<1, 128, 0, st>>>(ss, ctl, s, m, active);
}

}  // namespace dsbcg

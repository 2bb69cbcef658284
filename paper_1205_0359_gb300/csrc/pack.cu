// Layout and precision conversion between the canonical ABI layout
// (complex128, index site*12 + spin*3 + colour) and the internal chunk-major
// field layout of common.cuh, plus the FP64 vector kernels of the restart
// loop: true residual r = b - sigma x - A x with its column norms, and
// x64 += x_work.
#include "kernels.h"

namespace dsbcg {

namespace {

template <int P>
__global__ void pack_fields_kernel(typename Tr<P>::S2* __restrict__ dst, size_t ld,
                                   const double2* __restrict__ src, int m, size_t V, float hscale) {
    const size_t n = 12 * V;
    const size_t total = (size_t)m * n;
    using R = typename Tr<P>::R;
    const R sc = (P == PBF16 || P == PF16) ? R(hscale) : R(1);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t f = t / n, i = t % n;                // canonical index i = site*12 + sc
        size_t x = i / 12;
        int c = (int)(i % 12);
        double2 v = src[t];
        typename Tr<P>::C w = mk(R(v.x), R(v.y));
        Elem<P>::st(dst + f * ld, fidx<P>(V, x, c), w, sc);
    }
}

template <int P>
__global__ void unpack_fields_kernel(double2* __restrict__ dst, const typename Tr<P>::S2* __restrict__ src,
                                     size_t ld, int m, size_t V, float hscale) {
    const size_t n = 12 * V;
    const size_t total = (size_t)m * n;
    using R = typename Tr<P>::R;
    const R inv = (P == PBF16 || P == PF16) ? R(1) / R(hscale) : R(1);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t f = t / n, i = t % n;
        size_t x = i / 12;
        int c = (int)(i % 12);
        typename Tr<P>::C w = Elem<P>::ld(src + f * ld, fidx<P>(V, x, c), inv);
        dst[t] = make_double2((double)w.x, (double)w.y);
    }
}

template <int P>
__global__ void pack_links_kernel(typename Tr<P>::S2* __restrict__ dst, const double2* __restrict__ src, size_t V) {
    const size_t total = V * 36;
    using R = typename Tr<P>::R;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t x = t / 36;
        int r = (int)(t % 36);
        int mu = r / 9, e = r % 9;
        double2 v = src[t];
        Elem<P>::st(dst, ((size_t)mu * 9 + e) * V + x, mk(R(v.x), R(v.y)), R(1));
    }
}

// 12-real links: rows 0 and 1 of every SU(3) link, [mu][entry e < 6][site]
// (row 2 = conj(row 0 x row 1) is rebuilt by the stencil)
template <int P>
__global__ void pack_links12_kernel(typename Tr<P>::S2* __restrict__ dst, const double2* __restrict__ src, size_t V) {
    const size_t total = V * 24;
    using R = typename Tr<P>::R;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t x = t / 24;
        const int r = (int)(t % 24);
        const int mu = r / 6, e = r % 6;
        const double2 v = src[x * 36 + mu * 9 + e];
        Elem<P>::st(dst, ((size_t)mu * 6 + e) * V + x, mk(R(v.x), R(v.y)), R(1));
    }
}

// *flag = 1 if some link is not in SU(3) to tol: rows 0 and 1 orthonormal and
// row 2 = conj(row 0 x row 1), each entry to tol (FP64)
__global__ void check_su3_kernel(const double2* __restrict__ src, size_t nlinks, double tol, int* flag) {
    int bad = 0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nlinks;
         t += (size_t)gridDim.x * blockDim.x) {
        const double2* u = src + t * 9;
        double2 r[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) r[e] = u[e];
        // <r_i, r_j> - delta_ij for i, j in {0, 1}
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = i; j < 2; ++j) {
                double re = 0.0, im = 0.0;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const double2 a = r[i * 3 + b], c = r[j * 3 + b];
                    re += a.x * c.x + a.y * c.y;            // conj(a) c
                    im += a.x * c.y - a.y * c.x;
                }
                if (i == j) re -= 1.0;
                if (!(fabs(re) <= tol && fabs(im) <= tol)) bad = 1;
            }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int i = (k + 1) % 3, j = (k + 2) % 3;
            // conj(r0_i r1_j - r0_j r1_i)
            const double2 a = r[i], b = r[3 + j], c = r[j], d = r[3 + i];
            const double x = (a.x * b.x - a.y * b.y) - (c.x * d.x - c.y * d.y);
            const double y = -((a.x * b.y + a.y * b.x) - (c.x * d.y + c.y * d.x));
            if (!(fabs(x - r[6 + k].x) <= tol && fabs(y - r[6 + k].y) <= tol)) bad = 1;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void check_finite_kernel(const double2* __restrict__ p, size_t count, int* flag) {
    int bad = 0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
         t += (size_t)gridDim.x * blockDim.x) {
        double2 v = p[t];
        if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

template <int PX>
__global__ void accumulate_kernel(double2* __restrict__ y, size_t ldy, const typename Tr<PX>::S2* __restrict__ x,
                                  size_t ldx, int m, size_t n) {
    const size_t total = (size_t)m * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t f = t / n, i = t % n;
        typename Tr<PX>::C v = Elem<PX>::ld(x + f * ldx, i, 1);
        double2 a = y[f * ldy + i];
        a.x += (double)v.x;
        a.y += (double)v.y;
        y[f * ldy + i] = a;
    }
}

// ---- double-float fields: field f has an FP32 hi plane at f * 2 ld and an
// FP32 lo plane at f * 2 ld + ld (float2 words), both in the internal order

__global__ void pack_pairs_kernel(float2* __restrict__ dst, size_t ld, const double2* __restrict__ src, int m,
                                  size_t V) {
    const size_t n = 12 * V;
    const size_t total = (size_t)m * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t f = t / n, i = t % n;
        size_t x = i / 12;
        int c = (int)(i % 12);
        double2 v = src[t];
        const float hx = __double2float_rn(v.x), hy = __double2float_rn(v.y);
        const size_t at = f * 2 * ld + fidx<P32>(V, x, c);
        dst[at] = make_float2(hx, hy);
        dst[at + ld] = make_float2(__double2float_rn(v.x - (double)hx), __double2float_rn(v.y - (double)hy));
    }
}

__global__ void unpack_pairs_kernel(double2* __restrict__ dst, const float2* __restrict__ src, size_t ld, int m,
                                    size_t V) {
    const size_t n = 12 * V;
    const size_t total = (size_t)m * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t f = t / n, i = t % n;
        size_t x = i / 12;
        int c = (int)(i % 12);
        const size_t at = f * 2 * ld + fidx<P32>(V, x, c);
        float2 h = src[at], l = src[at + ld];
        dst[t] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
    }
}

__global__ void pack_links_pairs_kernel(float2* __restrict__ dst, const double2* __restrict__ src, size_t V) {
    const size_t total = V * 36;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t x = t / 36;
        int r = (int)(t % 36);
        double2 v = src[t];
        const float hx = __double2float_rn(v.x), hy = __double2float_rn(v.y);
        const size_t at = (size_t)r * V + x;          // r = mu * 9 + entry
        dst[at] = make_float2(hx, hy);
        dst[at + total] = make_float2(__double2float_rn(v.x - (double)hx), __double2float_rn(v.y - (double)hy));
    }
}

// y (double-float) += x (FP32 plane), m fields of n complex values
__global__ void accumulate_pairs_kernel(float2* __restrict__ y, size_t ld, const float2* __restrict__ x, size_t ldx,
                                        int m, size_t n) {
    const size_t total = (size_t)m * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t f = t / n, i = t % n;
        const size_t at = f * 2 * ld + i;
        float2 h = y[at], l = y[at + ld], v = x[f * ldx + i];
        dd a = dd(h.x, l.x) + dd(v.x), b = dd(h.y, l.y) + dd(v.y);
        y[at] = make_float2(a.hi, b.hi);
        y[at + ld] = make_float2(a.lo, b.lo);
    }
}

// FP64 internal fields -> FP32 internal fields (same element order)
__global__ void convert_64_32_kernel(float2* __restrict__ dst, size_t ldd, const double2* __restrict__ src,
                                     size_t lds, int m, size_t n) {
    const size_t total = (size_t)m * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t f = t / n, i = t % n;
        const double2 v = src[f * lds + i];
        dst[f * ldd + i] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
    }
}

constexpr int RES_THREADS = 256;

// r = b - sigma x - ax for double-float fields (grid (nblk, m)); squared
// column norms from the hi words, summed in FP32 per CTA
__global__ void residual_pairs_kernel(float2* __restrict__ r, const float2* __restrict__ b,
                                      const float2* __restrict__ x, const float2* __restrict__ ax, size_t ld,
                                      size_t n, dd sigma, double* __restrict__ partials, int nblk) {
    const int f = blockIdx.y;
    const size_t off = (size_t)f * 2 * ld;
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)nblk * blockDim.x) {
        const size_t h = off + i, l = off + ld + i;
        float2 bh = b[h], bl = b[l], xh = x[h], xl = x[l], ah = ax[h], al = ax[l];
        dd rx = dd(bh.x, bl.x) - sigma * dd(xh.x, xl.x) - dd(ah.x, al.x);
        dd ry = dd(bh.y, bl.y) - sigma * dd(xh.y, xl.y) - dd(ah.y, al.y);
        r[h] = make_float2(rx.hi, ry.hi);
        r[l] = make_float2(rx.lo, ry.lo);
        acc = fmaf(rx.hi, rx.hi, fmaf(ry.hi, ry.hi, acc));
    }
    __shared__ float red[RES_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < RES_THREADS / 32 ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partials[(size_t)f * nblk + blockIdx.x] = (double)v;
    }
}

// one block column per field: grid (nblk, m)
__global__ void residual_kernel(double2* __restrict__ r, const double2* __restrict__ b,
                                const double2* __restrict__ x, const double2* __restrict__ ax, size_t ld,
                                size_t n, double sigma, double* __restrict__ partials, int nblk) {
    const int f = blockIdx.y;
    const size_t off = (size_t)f * ld;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)nblk * blockDim.x) {
        double2 bb = b[off + i], xx = x[off + i], aa = ax[off + i];
        double2 rr = make_double2(bb.x - sigma * xx.x - aa.x, bb.y - sigma * xx.y - aa.y);
        r[off + i] = rr;
        acc += rr.x * rr.x + rr.y * rr.y;
    }
    __shared__ double red[RES_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < RES_THREADS / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partials[(size_t)f * nblk + blockIdx.x] = v;
    }
}

// out[f] = sum_b partials[f * nblk + b], fixed order
__global__ void reduce_cols_kernel(const double* __restrict__ partials, int nblk, double* __restrict__ out) {
    const int f = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partials[(size_t)f * nblk + b];
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        out[f] = v;
    }
}

// Y = coef[0] b + sum_j coef[j+1] x_j (canonical complex128 [m][n] out) from
// high-precision internal fields: b = B[f], x_j = X[j m + f] (FP64, or
// double-float hi + lo planes); FP64 arithmetic, shifts in index order
template <int HP>
__global__ void rational_combine_kernel(double2* __restrict__ Y, const void* __restrict__ Bv,
                                        const void* __restrict__ Xv, size_t ld, int m, int s,
                                        const double* __restrict__ coef, size_t V) {
    const size_t n = 12 * V;
    const size_t total = (size_t)m * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t f = t / n, i = t % n;
        const size_t e = fidx<P64>(V, i / 12, (int)(i % 12));
        auto ld_hp = [&](const void* base, size_t field) -> double2 {
            if constexpr (HP == P64) {
                return reinterpret_cast<const double2*>(base)[field * ld + e];
            } else {
                const float2* q = reinterpret_cast<const float2*>(base) + field * 2 * ld + e;
                const float2 h = q[0], l = q[ld];
                return make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
            }
        };
        const double2 b = ld_hp(Bv, f);
        double ax = coef[0] * b.x, ay = coef[0] * b.y;
        for (int j = 0; j < s; ++j) {
            const double2 x = ld_hp(Xv, (size_t)j * m + f);
            ax = fma(coef[j + 1], x.x, ax);
            ay = fma(coef[j + 1], x.y, ay);
        }
        Y[t] = make_double2(ax, ay);
    }
}

// ---- canonical complex128 blocks [s][cnt] of the backward pass

struct ShiftWeights {
    double w[S_MAX];
};

// L_j *= w_j for s blocks of cnt complex values
__global__ void scale_blocks_kernel(double2* __restrict__ L, int s, size_t cnt, ShiftWeights w) {
    const size_t total = (size_t)s * cnt;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const double a = w.w[t / cnt];
        double2 v = L[t];
        L[t] = make_double2(a * v.x, a * v.y);
    }
}

// out = a0 g + sum_j L_j (shifts in index order; g may be NULL when a0 = 0)
__global__ void sum_blocks_kernel(double2* __restrict__ out, const double2* __restrict__ L, int s, size_t cnt,
                                  const double2* __restrict__ g, double a0) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < cnt; t += (size_t)gridDim.x * blockDim.x) {
        double ax = 0.0, ay = 0.0;
        if (g) {
            const double2 v = g[t];
            ax = a0 * v.x;
            ay = a0 * v.y;
        }
        for (int j = 0; j < s; ++j) {
            const double2 v = L[(size_t)j * cnt + t];
            ax += v.x;
            ay += v.y;
        }
        out[t] = make_double2(ax, ay);
    }
}

// partials[j * nblk + b] = sum over CTA b's elements of Re(conj(a_j) b_j), grid (nblk, s)
__global__ void dot_re_blocks_kernel(const double2* __restrict__ a, const double2* __restrict__ b, size_t cnt,
                                     double* __restrict__ partials, int nblk) {
    const int j = blockIdx.y;
    const double2* aj = a + (size_t)j * cnt;
    const double2* bj = b + (size_t)j * cnt;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt; i += (size_t)nblk * blockDim.x) {
        const double2 u = aj[i], v = bj[i];
        acc = fma(u.x, v.x, fma(u.y, v.y, acc));
    }
    __shared__ double red[RES_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < RES_THREADS / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partials[(size_t)j * nblk + blockIdx.x] = v;
    }
}

inline int grid_for(size_t total) {
    size_t g = (total + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

void launch_pack_fields(int prec, void* dst, size_t ld, const double2* src, int m, size_t V, float hscale,
                        cudaStream_t st) {
    int g = grid_for((size_t)m * 12 * V);
    switch (prec) {
        case P64: pack_fields_kernel<P64><<<g, 256, 0, st>>>((double2*)dst, ld, src, m, V, hscale); break;
        case P32: pack_fields_kernel<P32><<<g, 256, 0, st>>>((float2*)dst, ld, src, m, V, hscale); break;
        case PBF16: pack_fields_kernel<PBF16><<<g, 256, 0, st>>>((__nv_bfloat162*)dst, ld, src, m, V, hscale); break;
        case PF16: pack_fields_kernel<PF16><<<g, 256, 0, st>>>((__half2*)dst, ld, src, m, V, hscale); break;
    }
}

void launch_unpack_fields(int prec, double2* dst, const void* src, size_t ld, int m, size_t V, float hscale,
                          cudaStream_t st) {
    int g = grid_for((size_t)m * 12 * V);
    switch (prec) {
        case P64: unpack_fields_kernel<P64><<<g, 256, 0, st>>>(dst, (const double2*)src, ld, m, V, hscale); break;
        case P32: unpack_fields_kernel<P32><<<g, 256, 0, st>>>(dst, (const float2*)src, ld, m, V, hscale); break;
        case PBF16: unpack_fields_kernel<PBF16><<<g, 256, 0, st>>>(dst, (const __nv_bfloat162*)src, ld, m, V, hscale); break;
        case PF16: unpack_fields_kernel<PF16><<<g, 256, 0, st>>>(dst, (const __half2*)src, ld, m, V, hscale); break;
    }
}

void launch_pack_pairs(float2* dst, size_t ld, const double2* src, int m, size_t V, cudaStream_t st) {
    pack_pairs_kernel<<<grid_for((size_t)m * 12 * V), 256, 0, st>>>(dst, ld, src, m, V);
}

void launch_unpack_pairs(double2* dst, const float2* src, size_t ld, int m, size_t V, cudaStream_t st) {
    unpack_pairs_kernel<<<grid_for((size_t)m * 12 * V), 256, 0, st>>>(dst, src, ld, m, V);
}

void launch_accumulate_pairs(float2* y, size_t ld, const float2* x, size_t ldx, int m, size_t n, cudaStream_t st) {
    accumulate_pairs_kernel<<<grid_for((size_t)m * n), 256, 0, st>>>(y, ld, x, ldx, m, n);
}

void launch_residual_pairs(float2* r, const float2* b, const float2* x, const float2* ax, size_t ld, int m,
                           size_t n, double sigma, double* partials, int nblk, cudaStream_t st) {
    dim3 grid(nblk, m);
    residual_pairs_kernel<<<grid, RES_THREADS, 0, st>>>(r, b, x, ax, ld, n, dd::from_double(sigma), partials, nblk);
}

void launch_pack_links(int prec, void* dst, const double2* src, size_t V, cudaStream_t st) {
    int g = grid_for(V * 36);
    switch (prec) {
        case PDD: pack_links_pairs_kernel<<<g, 256, 0, st>>>((float2*)dst, src, V); break;
        case P64: pack_links_kernel<P64><<<g, 256, 0, st>>>((double2*)dst, src, V); break;
        case P32: pack_links_kernel<P32><<<g, 256, 0, st>>>((float2*)dst, src, V); break;
        case PBF16: pack_links_kernel<PBF16><<<g, 256, 0, st>>>((__nv_bfloat162*)dst, src, V); break;
        case PF16: pack_links_kernel<PF16><<<g, 256, 0, st>>>((__half2*)dst, src, V); break;
    }
}

void launch_pack_links12(int prec, void* dst, const double2* src, size_t V, cudaStream_t st) {
    const int g = grid_for(V * 24);
    switch (prec) {
        case P32: pack_links12_kernel<P32><<<g, 256, 0, st>>>((float2*)dst, src, V); break;
        case PBF16: pack_links12_kernel<PBF16><<<g, 256, 0, st>>>((__nv_bfloat162*)dst, src, V); break;
        case PF16: pack_links12_kernel<PF16><<<g, 256, 0, st>>>((__half2*)dst, src, V); break;
    }
}

void launch_check_su3(const double2* src, size_t nlinks, double tol, int* flag, cudaStream_t st) {
    check_su3_kernel<<<grid_for(nlinks), 256, 0, st>>>(src, nlinks, tol, flag);
}

void launch_check_finite(const double2* p, size_t count, int* flag, cudaStream_t st) {
    check_finite_kernel<<<grid_for(count), 256, 0, st>>>(p, count, flag);
}

void launch_accumulate(int prec_x, double2* y, size_t ldy, const void* x, size_t ldx, int m, size_t n,
                       cudaStream_t st) {
    int g = grid_for((size_t)m * n);
    if (prec_x == P64)
        accumulate_kernel<P64><<<g, 256, 0, st>>>(y, ldy, (const double2*)x, ldx, m, n);
    else
        accumulate_kernel<P32><<<g, 256, 0, st>>>(y, ldy, (const float2*)x, ldx, m, n);
}

void launch_convert_64_32(float2* dst, size_t ldd, const double2* src, size_t lds, int m, size_t n,
                          cudaStream_t st) {
    convert_64_32_kernel<<<grid_for((size_t)m * n), 256, 0, st>>>(dst, ldd, src, lds, m, n);
}

int residual_blocks(size_t n) {
    size_t b = (n + RES_THREADS - 1) / RES_THREADS;
    return (int)(b < 304 ? (b < 1 ? 1 : b) : 304);
}

void launch_residual(double2* r, const double2* b, const double2* x, const double2* ax, size_t ld, int m,
                     size_t n, double sigma, double* partials, int nblk, cudaStream_t st) {
    dim3 grid(nblk, m);
    residual_kernel<<<grid, RES_THREADS, 0, st>>>(r, b, x, ax, ld, n, sigma, partials, nblk);
}

void launch_reduce_cols(const double* partials, int nblk, int m, double* out, cudaStream_t st) {
    reduce_cols_kernel<<<m, 256, 0, st>>>(partials, nblk, out);
}

void launch_rational_combine(int hp, double2* Y, const void* B, const void* X, size_t ld, int m, int s,
                             const double* coef, size_t V, cudaStream_t st) {
    const int g = grid_for((size_t)m * 12 * V);
    if (hp == PDD)
        rational_combine_kernel<PDD><<<g, 256, 0, st>>>(Y, B, X, ld, m, s, coef, V);
    else
        rational_combine_kernel<P64><<<g, 256, 0, st>>>(Y, B, X, ld, m, s, coef, V);
}

void launch_scale_blocks(double2* L, int s, size_t cnt, const double* w, cudaStream_t st) {
    ShiftWeights sw;
    for (int j = 0; j < S_MAX; ++j) sw.w[j] = j < s ? w[j] : 0.0;
    scale_blocks_kernel<<<grid_for((size_t)s * cnt), 256, 0, st>>>(L, s, cnt, sw);
}

void launch_sum_blocks(double2* out, const double2* L, int s, size_t cnt, const double2* g, double a0,
                       cudaStream_t st) {
    sum_blocks_kernel<<<grid_for(cnt), 256, 0, st>>>(out, L, s, cnt, a0 != 0.0 ? g : nullptr, a0);
}

void launch_dot_re_blocks(const double2* a, const double2* b, int s, size_t cnt, double* partials, int nblk,
                          double* out, cudaStream_t st) {
    dim3 grid(nblk, s);
    dot_re_blocks_kernel<<<grid, RES_THREADS, 0, st>>>(a, b, cnt, partials, nblk);
    reduce_cols_kernel<<<s, 256, 0, st>>>(partials, nblk, out);
}

}  // namespace dsbcg

// Shared device-side definitions: storage precisions, complex arithmetic,
// internal field layout and the device-resident control block of a solve.
//
// Internal field layout (every kernel of the Krylov iteration uses it).
// A field is one complex n-vector, n = 12 * V, stored pair-chunked:
//     [pair c = sc / 2][site][2 complex]
// for every storage precision, so that kernels mixing precisions (FP64
// right-hand sides -> FP32 basis, FP32 iterates -> FP64 accumulators) see
// the same element order.  Complex component sc = spin*3 + colour of site x
// is element (sc/2 * V + x) * 2 + sc % 2.  A warp reading one pair of 32
// consecutive sites touches one contiguous 512 B (FP32), 1 KB (FP64) or
// 256 B (16-bit) span.  Kernels that treat a field as a flat vector (inner
// products, block updates) see it as n complex values in this order; the
// permutation does not change inner products.
//
// 16-bit fields hold value * hscale, with hscale a power of two close to
// sqrt(n): Krylov vectors have unit norm, so their entries are O(1/sqrt(n))
// and the scaled entries are O(1), well inside FP16's range.
//
// Links: [mu][entry e = row*3 + col][site] of the field precision's complex
// storage type (U_mu(x) for the forward hop; the backward hop reads the link
// of x - mu and applies its adjoint).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>

namespace dsbcg {

// PDD: double-float ("FP32 pair") fields for the true-residual loop of the
// reduced-precision solves (see the dd type below); never a storage
// precision of the Krylov basis.
enum Prec { P64 = 0, P32 = 1, PBF16 = 2, PF16 = 3, PDD = 4 };

// Raise a kernel's dynamic shared-memory limit once per device (the
// attribute belongs to the current device); `devs` records the devices done.
template <class F>
inline void max_dyn_smem_once(F* func, int bytes, std::atomic<unsigned long long>& devs) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (devs.load() & bit)) return;
    cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    devs.fetch_or(bit);
}

constexpr int M_MAX = 32;      // largest block width (right-hand sides in a block)
constexpr int CTL_HIST = 16;   // block widths kept per step (the longest shift-update chunk)
constexpr int S_MAX = 64;      // largest number of shifts

// ------------------------------------------------------------------ traits --
template <int P> struct Tr;
template <> struct Tr<P64> {
    using S2 = double2;            // complex storage element
    using R = double;              // arithmetic real type
    using C = double2;             // arithmetic complex type
};
template <> struct Tr<P32> {
    using S2 = float2;
    using R = float;
    using C = float2;
};
template <> struct Tr<PBF16> {
    using S2 = __nv_bfloat162;
    using R = float;
    using C = float2;
};
template <> struct Tr<PF16> {
    using S2 = __half2;
    using R = float;
    using C = float2;
};

__host__ __device__ constexpr int prec_bytes(int p) {
    return (p == P64 || p == PDD) ? 16 : (p == P32 ? 8 : 4);     // bytes per complex
}

// ---------------------------------------------------------------- complex --
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a * b
template <class C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class C> __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
// acc -= a * b
template <class C> __device__ __forceinline__ void cfms(C& acc, C a, C b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// i * a
template <class C> __device__ __forceinline__ C ctimesi(C a) { return mk(-a.y, a.x); }
// -a (exact; a negation modifier of the consuming instruction in FP32/FP64)
template <class C> __device__ __forceinline__ C cneg(C a) { return mk(-a.x, -a.y); }

// ------------------------------------------------------------ double-float --
// An unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2:
// 48 significand bits, the FP32 exponent range.  GB300 executes FP64 (and
// FP64 <-> FP32 conversion) at 1/64 of its FP32 rate, so the loop that needs
// more than FP32 accuracy (true residuals, solution accumulation) runs in
// this arithmetic on the FP32 pipes.  Error-free transformations:
//   two_sum        s + e = a + b exactly (Knuth, TAOCP vol. 2, 4.2.2)
//   quick_two_sum  the same when |a| >= |b| (Dekker 1971)
//   two_prod       p + e = a * b exactly, e from one fused multiply-add
// Addition is Dekker's: relative error about 2^-45 of |a| + |b|; the product
// drops lo * lo (relative error about 2^-46).  Built without fast-math, so
// the compiler neither reassociates these sums nor contracts them.
struct dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ explicit constexpr dd(float h) : hi(h), lo(0.f) {}
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    // nearest pair to a double (host side: constants such as kappa, sigma)
    static __host__ __device__ dd from_double(double v) {
        float h = (float)v;
        return dd(h, (float)(v - (double)h));
    }
};
struct ddc {
    dd x, y;
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ dd quick_two_sum(float a, float b) {
    float s = a + b;
    return dd(s, b - (s - a));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    return quick_two_sum(s, e);
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
// c + a * b (an overload beside the FP32/FP64 fma, which stay visible)
using ::fma;
__device__ __forceinline__ dd fma(dd a, dd b, dd c) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    t += c.lo + e;
    return quick_two_sum(s, t);
}
__device__ __forceinline__ ddc mk(dd a, dd b) { return ddc{a, b}; }
// scaling by a power of two (here always a sign): exact on both words
__device__ __forceinline__ ddc cscale(ddc a, dd s) {
    return ddc{dd(a.x.hi * s.hi, a.x.lo * s.hi), dd(a.y.hi * s.hi, a.y.lo * s.hi)};
}

// Complex double-float helpers for accumulation chains (the stencil): sums
// stay unnormalised (hi = running FP32 sum, lo = its accumulated rounding
// errors and low words; the value is hi + lo), each product enters through
// two_prod plus the cross terms, and the caller normalises once at the end.
// These overloads take precedence over the generic complex templates.
__device__ __forceinline__ dd add_nn(dd a, dd b) {
    float s, t;
    two_sum(a.hi, b.hi, s, t);
    return dd(s, t + (a.lo + b.lo));
}
// acc += a * b, unnormalised
__device__ __forceinline__ void fma_nn(dd& acc, dd a, dd b) {
    float p = a.hi * b.hi;
    float q = fmaf(a.hi, b.hi, -p);
    q = fmaf(a.hi, b.lo, q);
    q = fmaf(a.lo, b.hi, q);
    float s, t;
    two_sum(acc.hi, p, s, t);
    acc = dd(s, acc.lo + (t + q));
}
__device__ __forceinline__ dd normalize(dd a) { return quick_two_sum(a.hi, a.lo); }
__device__ __forceinline__ ddc cadd(ddc a, ddc b) { return ddc{add_nn(a.x, b.x), add_nn(a.y, b.y)}; }
__device__ __forceinline__ ddc csub(ddc a, ddc b) { return ddc{add_nn(a.x, -b.x), add_nn(a.y, -b.y)}; }
__device__ __forceinline__ void cfma(ddc& acc, ddc a, ddc b) {
    fma_nn(acc.x, a.x, b.x);
    fma_nn(acc.x, -a.y, b.y);
    fma_nn(acc.y, a.x, b.y);
    fma_nn(acc.y, a.y, b.x);
}
__device__ __forceinline__ void cfmac(ddc& acc, ddc a, ddc b) {
    fma_nn(acc.x, a.x, b.x);
    fma_nn(acc.x, a.y, b.y);
    fma_nn(acc.y, a.x, b.y);
    fma_nn(acc.y, -a.y, b.x);
}

template <> struct Tr<PDD> {
    using S2 = float2;             // one word plane of a complex element
    using R = dd;
    using C = ddc;
};

// ------------------------------------------------------- element load/store --
// Flat complex element i of a field (internal order), converted to the
// arithmetic type; `inv` undoes the 16-bit scale on load, `sc` applies it on
// store (both 1 for FP32/FP64).
template <int P> struct Elem;
template <> struct Elem<P64> {
    static __device__ __forceinline__ double2 ld(const double2* p, size_t i, double) { return p[i]; }
    static __device__ __forceinline__ void st(double2* p, size_t i, double2 v, double) { p[i] = v; }
};
template <> struct Elem<P32> {
    static __device__ __forceinline__ float2 ld(const float2* p, size_t i, float) { return p[i]; }
    static __device__ __forceinline__ void st(float2* p, size_t i, float2 v, float) { p[i] = v; }
};
template <> struct Elem<PBF16> {
    static __device__ __forceinline__ float2 ld(const __nv_bfloat162* p, size_t i, float inv) {
        float2 f = __bfloat1622float2(p[i]);
        return make_float2(f.x * inv, f.y * inv);
    }
    static __device__ __forceinline__ void st(__nv_bfloat162* p, size_t i, float2 v, float sc) {
        p[i] = __float22bfloat162_rn(make_float2(v.x * sc, v.y * sc));
    }
};
template <> struct Elem<PF16> {
    static __device__ __forceinline__ float2 ld(const __half2* p, size_t i, float inv) {
        float2 f = __half22float2(p[i]);
        return make_float2(f.x * inv, f.y * inv);
    }
    static __device__ __forceinline__ void st(__half2* p, size_t i, float2 v, float sc) {
        p[i] = __float22half2_rn(make_float2(v.x * sc, v.y * sc));
    }
};

// index of complex component sc of site x inside a field (internal order)
// (the same order for every precision P)
template <int P> __host__ __device__ __forceinline__ size_t fidx(size_t V, size_t x, int sc) {
    return ((size_t)(sc >> 1) * V + x) * 2 + (sc & 1);
}

// -------------------------------------------------------------- control --
// Device-resident state of one inner solve.  Every kernel of a block step
// reads it, so the host can enqueue steps without knowing the block widths
// (which deflation changes on the device).
struct Ctl {
    int k;            // block step, 1-based (V_k is the current block)
    int mk;           // width of V_k
    int mprev;        // width of V_{k-1}
    int mnext;        // width of V_{k+1} (set by the QR kernel)
    int done;         // 1: every system frozen, or invariant subspace reached
    int status;       // 0 ok, else a dsbcg_status error code
    int nact;         // shifts still active
    int deflations;   // directions dropped so far
    long long mvms;   // single-vector A applications
    int last_step;    // last step that did work
    int hmk[CTL_HIST];  // width of V_k for step k at slot (k - 1) mod CTL_HIST
    int hmn[CTL_HIST];  // width of V_{k+1} for step k, same slots
    int pad[1];
    // algorithmic traffic, in fields (one complex n-vector) moved to or from
    // HBM, summed over block steps by the step's last kernel:
    long long f_dslash;   // storage-precision fields read + written by the 2 stencils
    long long f_gram;     // storage-precision fields read by the 2 Gram products
    long long f_update;   // storage-precision fields of the block update
    long long f_shift_s;  // storage-precision fields read by the shift update (V_{k+1}, once per step)
    long long f_shift_w;  // work-precision fields of the shift update (P_j, X_j: once per chunk)
    long long f_shift_cmac;  // complex multiply-adds per element of the shift update
};

// error codes mirrored from dsbcg.h
constexpr int ST_NOT_HPD = -2;

}  // namespace dsbcg

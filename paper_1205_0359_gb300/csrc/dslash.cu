// Multi-right-hand-side Wilson-Dirac stencil (the operator of Sec. 1).
//
//   (D psi)(x) = psi(x) - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                                        + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu) ]
//
// One CTA of 32 threads covers 32 consecutive sites of one field; the grid
// is (fields, site tiles) with the field index fastest, so the CTAs of all
// fields of a site tile are issued together and the SU(3) links they share
// are fetched from HBM once and then served from L1/L2 (read-only path).
// Each thread owns one (site, field) pair; every pair-chunk load of a
// neighbour spinor is one contiguous 512-byte warp access.  Staging the links
// in shared memory per CTA was measured slower on GB300 (1.3 vs 3.3 TB/s at
// 16^3 x 32 with 12 FP32 fields): the staging barrier serialises each CTA's
// link and spinor loads.
// Spin projection in the chiral basis (gamma_k = [[0, i s_k], [-i s_k, 0]],
// gamma_4 = [[0, 1], [1, 0]]): with upper/lower spin pairs u = (p0, p1),
// l = (p2, p3),
//   (1 - gamma_k) p = [h; i s_k h],  h = u - i s_k l,
//   (1 + gamma_k) p = [h; -i s_k h], h = u + i s_k l,
//   (1 -/+ gamma_4) p = [h; -/+ h],  h = u -/+ l,
// so each hop multiplies only a two-spin half spinor by the link.
// i s_1 (a, b) = (i b, i a);  i s_2 (a, b) = (b, -a);  i s_3 (a, b) = (i a, -i b).
#include "kernels.h"

namespace dsbcg {

namespace {

template <int P>
struct SpinorIO;

template <>
struct SpinorIO<P64> {
    static __device__ __forceinline__ void load(const double2* f, size_t V, size_t x, double2 p[12], double, size_t) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double2* q = f + ((size_t)c * V + x) * 2;
            p[2 * c] = __ldg(q);
            p[2 * c + 1] = __ldg(q + 1);
        }
    }
    static __device__ __forceinline__ void store(double2* f, size_t V, size_t x, const double2 p[12], double, size_t) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double2* q = f + ((size_t)c * V + x) * 2;
            q[0] = p[2 * c];
            q[1] = p[2 * c + 1];
        }
    }
};

template <>
struct SpinorIO<P32> {
    static __device__ __forceinline__ void load(const float2* f, size_t V, size_t x, float2 p[12], float, size_t) {
        const float4* q = reinterpret_cast<const float4*>(f);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float4 v = __ldg(q + (size_t)c * V + x);
            p[2 * c] = make_float2(v.x, v.y);
            p[2 * c + 1] = make_float2(v.z, v.w);
        }
    }
    static __device__ __forceinline__ void store(float2* f, size_t V, size_t x, const float2 p[12], float, size_t) {
        float4* q = reinterpret_cast<float4*>(f);
#pragma unroll
        for (int c = 0; c < 6; ++c)
            q[(size_t)c * V + x] = make_float4(p[2 * c].x, p[2 * c].y, p[2 * c + 1].x, p[2 * c + 1].y);
    }
};

template <class H2, class Cvt>
struct Spinor16 {
    static __device__ __forceinline__ void load(const H2* f, size_t V, size_t x, float2 p[12], float inv, size_t) {
        const uint2* q = reinterpret_cast<const uint2*>(f);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            uint2 v = __ldg(q + (size_t)c * V + x);
            const H2* h = reinterpret_cast<const H2*>(&v);
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                float2 t = Cvt::to2(h[w]);
                p[2 * c + w] = make_float2(t.x * inv, t.y * inv);
            }
        }
    }
    static __device__ __forceinline__ void store(H2* f, size_t V, size_t x, const float2 p[12], float sc, size_t) {
        uint2* q = reinterpret_cast<uint2*>(f);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            uint2 v;
            H2* h = reinterpret_cast<H2*>(&v);
#pragma unroll
            for (int w = 0; w < 2; ++w)
                h[w] = Cvt::from2(make_float2(p[2 * c + w].x * sc, p[2 * c + w].y * sc));
            q[(size_t)c * V + x] = v;
        }
    }
};
struct CvtBF {
    static __device__ __forceinline__ float2 to2(__nv_bfloat162 h) { return __bfloat1622float2(h); }
    static __device__ __forceinline__ __nv_bfloat162 from2(float2 f) { return __float22bfloat162_rn(f); }
};
struct CvtH {
    static __device__ __forceinline__ float2 to2(__half2 h) { return __half22float2(h); }
    static __device__ __forceinline__ __half2 from2(float2 f) { return __float22half2_rn(f); }
};
template <> struct SpinorIO<PBF16> : Spinor16<__nv_bfloat162, CvtBF> {};
template <> struct SpinorIO<PF16> : Spinor16<__half2, CvtH> {};
// double-float fields: an FP32 hi plane and, plo float2 further on, an FP32
// lo plane, each in the pair-chunk layout
template <>
struct SpinorIO<PDD> {
    static __device__ __forceinline__ void load(const float2* f, size_t V, size_t x, ddc p[12], dd, size_t plo) {
        const float4* qh = reinterpret_cast<const float4*>(f);
        const float4* ql = reinterpret_cast<const float4*>(f + plo);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float4 h = __ldg(qh + (size_t)c * V + x);
            float4 l = __ldg(ql + (size_t)c * V + x);
            p[2 * c] = ddc{dd(h.x, l.x), dd(h.y, l.y)};
            p[2 * c + 1] = ddc{dd(h.z, l.z), dd(h.w, l.w)};
        }
    }
    static __device__ __forceinline__ void store(float2* f, size_t V, size_t x, const ddc p[12], dd, size_t plo) {
        float4* qh = reinterpret_cast<float4*>(f);
        float4* ql = reinterpret_cast<float4*>(f + plo);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            qh[(size_t)c * V + x] = make_float4(p[2 * c].x.hi, p[2 * c].y.hi, p[2 * c + 1].x.hi, p[2 * c + 1].y.hi);
            ql[(size_t)c * V + x] = make_float4(p[2 * c].x.lo, p[2 * c].y.lo, p[2 * c + 1].x.lo, p[2 * c + 1].y.lo);
        }
    }
};

// link entry at p; a double-float link keeps its lo plane loff float2 further on
template <int P>
__device__ __forceinline__ typename Tr<P>::C ld_link(const typename Tr<P>::S2* p, size_t loff) {
    if constexpr (P == P64 || P == P32) {
        return __ldg(p);
    } else if constexpr (P == PDD) {
        float2 h = __ldg(p), l = __ldg(p + loff);
        return ddc{dd(h.x, l.x), dd(h.y, l.y)};
    } else if constexpr (P == PBF16) {
        return __bfloat1622float2(*p);
    } else {
        return __half22float2(*p);
    }
}

// site coordinates and neighbours
struct Site {
    int c[4];
};
__device__ __forceinline__ Site coords(const Geom& g, int x) {
    Site s;
    s.c[0] = x % g.L[0];
    int r = x / g.L[0];
    s.c[1] = r % g.L[1];
    r /= g.L[1];
    s.c[2] = r % g.L[2];
    s.c[3] = r / g.L[2];
    return s;
}
__device__ __forceinline__ int stride_of(const Geom& g, int mu) {
    int st = 1;
    for (int d = 0; d < mu; ++d) st *= g.L[d];
    return st;
}
// neighbour x + mu (dir = +1) or x - mu (dir = -1); *sign = -1 when the hop
// crosses the time boundary of an antiperiodic lattice
__device__ __forceinline__ int neighbour(const Geom& g, int x, const Site& s, int mu, int dir, float* sign) {
    int st = stride_of(g, mu);
    int c = s.c[mu];
    *sign = 1.f;
    if (dir > 0) {
        if (c == g.L[mu] - 1) {
            if (mu == 3 && g.tap) *sign = -1.f;
            return x - (g.L[mu] - 1) * st;
        }
        return x + st;
    } else {
        if (c == 0) {
            if (mu == 3 && g.tap) *sign = -1.f;
            return x + (g.L[mu] - 1) * st;
        }
        return x - st;
    }
}

// Uh = U h (fwd) or U^H h (bwd) for the 2 x 3 half spinor h; entry e of the
// link is at u[e * stride] (global memory, read-only path)
template <int P, class C>
__device__ __forceinline__ void su3_mul(const typename Tr<P>::S2* __restrict__ u, size_t stride, size_t loff,
                                        const C h[2][3], C out[2][3], bool adj) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) out[sp][a] = mk(decltype(h[0][0].x)(0), decltype(h[0][0].x)(0));
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (!adj) {
                C uab = ld_link<P>(u + (a * 3 + b) * stride, loff);
#pragma unroll
                for (int sp = 0; sp < 2; ++sp) cfma(out[sp][a], uab, h[sp][b]);
            } else {
                C uba = ld_link<P>(u + (b * 3 + a) * stride, loff);     // (U^H)_ab = conj(U_ba)
#pragma unroll
                for (int sp = 0; sp < 2; ++sp) cfmac(out[sp][a], uba, h[sp][b]);
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(32, (P == PDD || P == P64) ? 12 : 24) dslash_kernel(typename Tr<P>::S2* __restrict__ out,
                                                   const typename Tr<P>::S2* __restrict__ in,
                                                   size_t ld, const typename Tr<P>::S2* __restrict__ links,
                                                   Geom g, typename Tr<P>::R kappa, int g5in, int g5out,
                                                   const Ctl* __restrict__ ctl, int nf_static, float hscale,
                                                   int nfg) {
    using C = typename Tr<P>::C;
    using R = typename Tr<P>::R;
    int nf = nf_static;
    if (ctl) {
        if (ctl->done) return;
        nf = ctl->mk;
    }
    // 1D work index: block b covers field b % nfg of site tile b / nfg
    // (fields fastest); a grid smaller than the work strides over it
    const unsigned nwork = (unsigned)nfg * (unsigned)((g.V + 31) / 32);
    for (unsigned blk = blockIdx.x; blk < nwork; blk += gridDim.x) {
    const int f = (int)(blk % (unsigned)nfg);
    if (f >= nf) continue;
    const int tx = threadIdx.x;
    const int site0 = (int)(blk / (unsigned)nfg) * 32;
    const size_t V = (size_t)g.V;
    const int x = site0 + tx;
    if (x >= g.V) continue;
    R inv = R(1), scl = R(1);
    if constexpr (P == PBF16 || P == PF16) {
        inv = R(1) / R(hscale);
        scl = R(hscale);
    }
    // double-float fields: lo plane half a field stride after the hi plane;
    // double-float links: lo plane 36 V entries after the hi plane
    const size_t plo = (P == PDD) ? ld / 2 : 0;
    const size_t loff = (P == PDD) ? 36 * (size_t)g.V : 0;
    const Site s = coords(g, x);
    const R g5i = g5in ? R(-1) : R(1);

    {
        const typename Tr<P>::S2* fin = in + (size_t)f * ld;
        C acc[4][3];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[sp][a] = mk(R(0), R(0));

#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                float sgn;
                int y = neighbour(g, x, s, mu, dir == 0 ? 1 : -1, &sgn);
                C p[12];
                SpinorIO<P>::load(fin, V, (size_t)y, p, inv, plo);
                const R sg = R(sgn);
                const R su = sg * g5i;          // gamma_5 on input flips the upper spins
                const R sl_ = sg;
                C h[2][3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    C u0 = cscale(p[0 * 3 + a], su), u1 = cscale(p[1 * 3 + a], su);
                    C l0 = cscale(p[2 * 3 + a], sl_), l1 = cscale(p[3 * 3 + a], sl_);
                    if (dir == 0) {               // forward: (1 - gamma_mu)
                        if (mu == 0) { h[0][a] = csub(u0, ctimesi(l1)); h[1][a] = csub(u1, ctimesi(l0)); }
                        if (mu == 1) { h[0][a] = csub(u0, l1); h[1][a] = cadd(u1, l0); }
                        if (mu == 2) { h[0][a] = csub(u0, ctimesi(l0)); h[1][a] = cadd(u1, ctimesi(l1)); }
                        if (mu == 3) { h[0][a] = csub(u0, l0); h[1][a] = csub(u1, l1); }
                    } else {                      // backward: (1 + gamma_mu)
                        if (mu == 0) { h[0][a] = cadd(u0, ctimesi(l1)); h[1][a] = cadd(u1, ctimesi(l0)); }
                        if (mu == 1) { h[0][a] = cadd(u0, l1); h[1][a] = csub(u1, l0); }
                        if (mu == 2) { h[0][a] = cadd(u0, ctimesi(l0)); h[1][a] = csub(u1, ctimesi(l1)); }
                        if (mu == 3) { h[0][a] = cadd(u0, l0); h[1][a] = cadd(u1, l1); }
                    }
                }
                C uh[2][3];
                // forward hop: U_mu(x); backward hop: U_mu(x - mu) = U_mu(y)
                su3_mul<P>(links + (size_t)mu * 9 * V + (dir == 0 ? x : y), V, loff, h, uh, dir != 0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    acc[0][a] = cadd(acc[0][a], uh[0][a]);
                    acc[1][a] = cadd(acc[1][a], uh[1][a]);
                    C q0 = uh[0][a], q1 = uh[1][a];
                    if (dir == 0) {               // lower = (i s_k) h, or -h for mu = 4
                        if (mu == 0) { acc[2][a] = cadd(acc[2][a], ctimesi(q1)); acc[3][a] = cadd(acc[3][a], ctimesi(q0)); }
                        if (mu == 1) { acc[2][a] = cadd(acc[2][a], q1); acc[3][a] = csub(acc[3][a], q0); }
                        if (mu == 2) { acc[2][a] = cadd(acc[2][a], ctimesi(q0)); acc[3][a] = csub(acc[3][a], ctimesi(q1)); }
                        if (mu == 3) { acc[2][a] = csub(acc[2][a], q0); acc[3][a] = csub(acc[3][a], q1); }
                    } else {                      // lower = -(i s_k) h, or +h for mu = 4
                        if (mu == 0) { acc[2][a] = csub(acc[2][a], ctimesi(q1)); acc[3][a] = csub(acc[3][a], ctimesi(q0)); }
                        if (mu == 1) { acc[2][a] = csub(acc[2][a], q1); acc[3][a] = cadd(acc[3][a], q0); }
                        if (mu == 2) { acc[2][a] = csub(acc[2][a], ctimesi(q0)); acc[3][a] = cadd(acc[3][a], ctimesi(q1)); }
                        if (mu == 3) { acc[2][a] = cadd(acc[2][a], q0); acc[3][a] = cadd(acc[3][a], q1); }
                    }
                }
            }
        }
        C p[12];
        SpinorIO<P>::load(fin, V, (size_t)x, p, inv, plo);
        const R go = g5out ? R(-1) : R(1);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            const R sgi = (sp < 2) ? g5i : R(1);
            const R sgo = (sp < 2) ? go : R(1);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                C v = cscale(p[sp * 3 + a], sgi);
                if constexpr (P == PDD) {      // close the unnormalised accumulation chains
                    acc[sp][a].x = normalize(acc[sp][a].x);
                    acc[sp][a].y = normalize(acc[sp][a].y);
                }
                v.x = fma(-kappa, acc[sp][a].x, v.x);
                v.y = fma(-kappa, acc[sp][a].y, v.y);
                p[sp * 3 + a] = cscale(v, sgo);
            }
        }
        SpinorIO<P>::store(out + (size_t)f * ld, V, (size_t)x, p, scl, plo);
    }
    }
}

// Projection of the hop (mu, dir) of spinor p: the half spinor h of
// (1 - gamma_mu) p (dir 0) or (1 + gamma_mu) p (dir 1), with the upper spins
// scaled by su and the lower by sl (gamma_5 and time-boundary signs).
template <class C, class R>
__device__ __forceinline__ void hop_project(int mu, int dir, const C p[12], R su, R sl_, C h[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C u0 = cscale(p[0 * 3 + a], su), u1 = cscale(p[1 * 3 + a], su);
        C l0 = cscale(p[2 * 3 + a], sl_), l1 = cscale(p[3 * 3 + a], sl_);
        if (dir == 0) {
            if (mu == 0) { h[0][a] = csub(u0, ctimesi(l1)); h[1][a] = csub(u1, ctimesi(l0)); }
            if (mu == 1) { h[0][a] = csub(u0, l1); h[1][a] = cadd(u1, l0); }
            if (mu == 2) { h[0][a] = csub(u0, ctimesi(l0)); h[1][a] = cadd(u1, ctimesi(l1)); }
            if (mu == 3) { h[0][a] = csub(u0, l0); h[1][a] = csub(u1, l1); }
        } else {
            if (mu == 0) { h[0][a] = cadd(u0, ctimesi(l1)); h[1][a] = cadd(u1, ctimesi(l0)); }
            if (mu == 1) { h[0][a] = cadd(u0, l1); h[1][a] = csub(u1, l0); }
            if (mu == 2) { h[0][a] = cadd(u0, ctimesi(l0)); h[1][a] = csub(u1, ctimesi(l1)); }
            if (mu == 3) { h[0][a] = cadd(u0, l0); h[1][a] = cadd(u1, l1); }
        }
    }
}

// acc += the reconstruction of the hop result uh: upper spins uh, lower spins
// (i s_k) uh (forward) or -(i s_k) uh (backward), -/+ uh for mu = 4
template <class C>
__device__ __forceinline__ void hop_reconstruct(int mu, int dir, const C uh[2][3], C acc[4][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[0][a] = cadd(acc[0][a], uh[0][a]);
        acc[1][a] = cadd(acc[1][a], uh[1][a]);
        const C q0 = uh[0][a], q1 = uh[1][a];
        if (dir == 0) {
            if (mu == 0) { acc[2][a] = cadd(acc[2][a], ctimesi(q1)); acc[3][a] = cadd(acc[3][a], ctimesi(q0)); }
            if (mu == 1) { acc[2][a] = cadd(acc[2][a], q1); acc[3][a] = csub(acc[3][a], q0); }
            if (mu == 2) { acc[2][a] = cadd(acc[2][a], ctimesi(q0)); acc[3][a] = csub(acc[3][a], ctimesi(q1)); }
            if (mu == 3) { acc[2][a] = csub(acc[2][a], q0); acc[3][a] = csub(acc[3][a], q1); }
        } else {
            if (mu == 0) { acc[2][a] = csub(acc[2][a], ctimesi(q1)); acc[3][a] = csub(acc[3][a], ctimesi(q0)); }
            if (mu == 1) { acc[2][a] = csub(acc[2][a], q1); acc[3][a] = cadd(acc[3][a], q0); }
            if (mu == 2) { acc[2][a] = csub(acc[2][a], ctimesi(q0)); acc[3][a] = cadd(acc[3][a], ctimesi(q1)); }
            if (mu == 3) { acc[2][a] = cadd(acc[2][a], q0); acc[3][a] = cadd(acc[3][a], q1); }
        }
    }
}

// D (or gamma_5 D gamma_5) for FP32 and 16-bit fields with the links staged
// once per CTA.  A CTA covers one 32-site tile for CTA_FIELDS fields, one
// warp per field: its warps first copy the 8 links of every site of the tile
// (U_mu(x) and U_mu(x - mu), converted to FP32) into shared memory (for SU(3)
// links rows 0 and 1 only, row 2 = conj(row 0 x row 1) being rebuilt at each
// use), then each warp applies the stencil to its field with the links read
// from shared memory and the neighbour spinors from L1/L2.  Against one field
// per 32-thread CTA with links from L1 this reads each link from L2 once per
// 4 fields and removes 72 of the 126 global loads per site and field:
// 9-13% faster on GB300 at 16^3 x 32, 24^3 x 48 and 32^3 x 64 (12, 8 and
// 16 FP32 fields); larger field groups measured slower (fewer resident CTAs).
constexpr int CTA_FIELDS = 4;

template <int P, bool L12>
__global__ void __launch_bounds__(32 * CTA_FIELDS, P == P32 ? 6 : 5) dslash_cta_kernel(typename Tr<P>::S2* __restrict__ out,
                                                       const typename Tr<P>::S2* __restrict__ in, size_t ld,
                                                       const typename Tr<P>::S2* __restrict__ links,
                                                       const typename Tr<P>::S2* __restrict__ links12, Geom g,
                                                       float kappa, int g5in, int g5out, const Ctl* __restrict__ ctl,
                                                       int nf_static, float hscale, int ngrp) {
    // [hop][entry][site of the tile]: rows 0 and 1 of SU(3) links (L12), with
    // row 2 rebuilt at each use, else all nine entries
    __shared__ float2 sl[8][L12 ? 6 : 9][32];
    int nf = nf_static;
    if (ctl) {
        if (ctl->done) return;
        nf = ctl->mk;
    }
    const int grp = (int)(blockIdx.x % (unsigned)ngrp);
    if (grp * CTA_FIELDS >= nf) return;      // CTA-uniform
    const int tile = (int)(blockIdx.x / (unsigned)ngrp);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t V = (size_t)g.V;
    const int x = tile * 32 + lane;
    const bool valid = x < g.V;
    const int xs = valid ? x : g.V - 1;
    const Site s = coords(g, xs);
    for (int h = w; h < 8; h += CTA_FIELDS) {
        const int mu = h >> 1, dir = h & 1;
        float sgn;
        const int y = neighbour(g, xs, s, mu, dir == 0 ? 1 : -1, &sgn);
        const size_t site = dir == 0 ? (size_t)xs : (size_t)y;
        if (links12) {
            // 12-real links: rows 0 and 1; row 2 = conj(row 0 x row 1) (SU(3))
            const typename Tr<P>::S2* u = links12 + (size_t)mu * 6 * V + site;
            float2 r[6];
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                r[e] = ld_link<P>(u + (size_t)e * V, 0);
                sl[h][e][lane] = r[e];
            }
            if constexpr (!L12) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int i = (k + 1) % 3, j = (k + 2) % 3;
                    float2 t = cmul(r[i], r[3 + j]);
                    cfms(t, r[j], r[3 + i]);
                    sl[h][6 + k][lane] = make_float2(t.x, -t.y);
                }
            }
        } else if constexpr (!L12) {
            const typename Tr<P>::S2* u = links + (size_t)mu * 9 * V + site;
#pragma unroll
            for (int e = 0; e < 9; ++e) sl[h][e][lane] = ld_link<P>(u + (size_t)e * V, 0);
        }
    }
    __syncthreads();
    const int f = grp * CTA_FIELDS + w;
    if (!valid || f >= nf) return;
    float inv = 1.f, scl = 1.f;
    if constexpr (P == PBF16 || P == PF16) {
        inv = 1.f / hscale;
        scl = hscale;
    }
    const float g5i = g5in ? -1.f : 1.f;
    const typename Tr<P>::S2* fin = in + (size_t)f * ld;
    float2 acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[sp][a] = make_float2(0.f, 0.f);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            const int h = 2 * mu + dir;
            float sgn;
            const int y = neighbour(g, x, s, mu, dir == 0 ? 1 : -1, &sgn);
            float2 p[12];
            SpinorIO<P>::load(fin, V, (size_t)y, p, inv, 0);
            float2 hh[2][3];
            hop_project(mu, dir, p, sgn * g5i, sgn, hh);
            // the hop's link: 9 entries from shared memory, or rows 0 and 1
            // with row 2 = conj(row 0 x row 1) rebuilt here
            float2 lk[L12 ? 9 : 1];
            if constexpr (L12) {
#pragma unroll
                for (int e = 0; e < 6; ++e) lk[e] = sl[h][e][lane];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int i = (k + 1) % 3, j = (k + 2) % 3;
                    float2 t = cmul(lk[i], lk[3 + j]);
                    cfms(t, lk[j], lk[3 + i]);
                    lk[6 + k] = make_float2(t.x, -t.y);
                }
            }
            auto link = [&](int e) -> float2 {
                if constexpr (L12) return lk[e];
                else return sl[h][e][lane];
            };
            float2 uh[2][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                uh[0][a] = make_float2(0.f, 0.f);
                uh[1][a] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (dir == 0) {
                        const float2 uab = link(a * 3 + b);
                        cfma(uh[0][a], uab, hh[0][b]);
                        cfma(uh[1][a], uab, hh[1][b]);
                    } else {
                        const float2 uba = link(b * 3 + a);      // (U^H)_ab = conj(U_ba)
                        cfmac(uh[0][a], uba, hh[0][b]);
                        cfmac(uh[1][a], uba, hh[1][b]);
                    }
                }
            hop_reconstruct(mu, dir, uh, acc);
        }
    }
    float2 p[12];
    SpinorIO<P>::load(fin, V, (size_t)x, p, inv, 0);
    const float go = g5out ? -1.f : 1.f;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const float sgi = (sp < 2) ? g5i : 1.f, sgo = (sp < 2) ? go : 1.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 v = cscale(p[sp * 3 + a], sgi);
            v.x = fmaf(-kappa, acc[sp][a].x, v.x);
            v.y = fmaf(-kappa, acc[sp][a].y, v.y);
            p[sp * 3 + a] = cscale(v, sgo);
        }
    }
    SpinorIO<P>::store(out + (size_t)f * ld, V, (size_t)x, p, scl, 0);
}

// Half-lattice hopping term for the even-odd (Schur) operator.  With every
// extent even, the sites of one parity p (x + y + z + t = p mod 2) in
// increasing canonical order have the half index k = site / 2 (each x-row
// holds Lx / 2 of them), and the hopping term H of D = 1 - kappa H maps
// parity 1 - p to parity p:
//     out_f(k) = alpha s_f(k) + beta G5o (H G5i in_f)(x_k),
// with in_f on parity 1 - p, s_f and out_f on parity p (all half fields of
// Vh = V / 2 sites) and G5i, G5o optional gamma_5 factors.  The Schur
// operator on the odd sites, Dhat = 1 - kappa^2 H_oe H_eo, is two such passes.
template <int P>
__global__ void __launch_bounds__(32, (P == PDD || P == P64) ? 12 : 24) dslash_half_kernel(
    typename Tr<P>::S2* __restrict__ out, const typename Tr<P>::S2* __restrict__ in,
    const typename Tr<P>::S2* __restrict__ src, size_t ld, const typename Tr<P>::S2* __restrict__ links, Geom g,
    typename Tr<P>::R alpha, typename Tr<P>::R beta, int parity, int g5in, int g5out, const Ctl* __restrict__ ctl,
    int nf_static, float hscale, int nfg) {
    using C = typename Tr<P>::C;
    using R = typename Tr<P>::R;
    int nf = nf_static;
    if (ctl) {
        if (ctl->done) return;
        nf = ctl->mk;
    }
    const int f = (int)(blockIdx.x % (unsigned)nfg);
    if (f >= nf) return;
    const int Vh = g.V / 2;
    const int k = (int)(blockIdx.x / (unsigned)nfg) * 32 + threadIdx.x;
    if (k >= Vh) return;
    R inv = R(1), scl = R(1);
    if constexpr (P == PBF16 || P == PF16) {
        inv = R(1) / R(hscale);
        scl = R(hscale);
    }
    const size_t plo = (P == PDD) ? ld / 2 : 0;
    const size_t loff = (P == PDD) ? 36 * (size_t)g.V : 0;
    const size_t V = (size_t)g.V;
    // full-lattice site of half index k
    const int hx = g.L[0] / 2;
    const int row = k / hx;
    Site s;
    s.c[1] = row % g.L[1];
    s.c[2] = (row / g.L[1]) % g.L[2];
    s.c[3] = row / (g.L[1] * g.L[2]);
    s.c[0] = 2 * (k % hx) + ((parity + s.c[1] + s.c[2] + s.c[3]) & 1);
    const int x = s.c[0] + g.L[0] * row;
    const R g5i = g5in ? R(-1) : R(1);
    const typename Tr<P>::S2* fin = in + (size_t)f * ld;
    C acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[sp][a] = mk(R(0), R(0));
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            float sgn;
            const int y = neighbour(g, x, s, mu, dir == 0 ? 1 : -1, &sgn);
            C p[12];
            SpinorIO<P>::load(fin, (size_t)Vh, (size_t)(y >> 1), p, inv, plo);
            const R sg = R(sgn);
            const R su = sg * g5i;
            const R sl_ = sg;
            C h[2][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                C u0 = cscale(p[0 * 3 + a], su), u1 = cscale(p[1 * 3 + a], su);
                C l0 = cscale(p[2 * 3 + a], sl_), l1 = cscale(p[3 * 3 + a], sl_);
                if (dir == 0) {
                    if (mu == 0) { h[0][a] = csub(u0, ctimesi(l1)); h[1][a] = csub(u1, ctimesi(l0)); }
                    if (mu == 1) { h[0][a] = csub(u0, l1); h[1][a] = cadd(u1, l0); }
                    if (mu == 2) { h[0][a] = csub(u0, ctimesi(l0)); h[1][a] = cadd(u1, ctimesi(l1)); }
                    if (mu == 3) { h[0][a] = csub(u0, l0); h[1][a] = csub(u1, l1); }
                } else {
                    if (mu == 0) { h[0][a] = cadd(u0, ctimesi(l1)); h[1][a] = cadd(u1, ctimesi(l0)); }
                    if (mu == 1) { h[0][a] = cadd(u0, l1); h[1][a] = csub(u1, l0); }
                    if (mu == 2) { h[0][a] = cadd(u0, ctimesi(l0)); h[1][a] = csub(u1, ctimesi(l1)); }
                    if (mu == 3) { h[0][a] = cadd(u0, l0); h[1][a] = cadd(u1, l1); }
                }
            }
            C uh[2][3];
            su3_mul<P>(links + (size_t)mu * 9 * V + (dir == 0 ? x : y), V, loff, h, uh, dir != 0);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc[0][a] = cadd(acc[0][a], uh[0][a]);
                acc[1][a] = cadd(acc[1][a], uh[1][a]);
                C q0 = uh[0][a], q1 = uh[1][a];
                if (dir == 0) {
                    if (mu == 0) { acc[2][a] = cadd(acc[2][a], ctimesi(q1)); acc[3][a] = cadd(acc[3][a], ctimesi(q0)); }
                    if (mu == 1) { acc[2][a] = cadd(acc[2][a], q1); acc[3][a] = csub(acc[3][a], q0); }
                    if (mu == 2) { acc[2][a] = cadd(acc[2][a], ctimesi(q0)); acc[3][a] = csub(acc[3][a], ctimesi(q1)); }
                    if (mu == 3) { acc[2][a] = csub(acc[2][a], q0); acc[3][a] = csub(acc[3][a], q1); }
                } else {
                    if (mu == 0) { acc[2][a] = csub(acc[2][a], ctimesi(q1)); acc[3][a] = csub(acc[3][a], ctimesi(q0)); }
                    if (mu == 1) { acc[2][a] = csub(acc[2][a], q1); acc[3][a] = cadd(acc[3][a], q0); }
                    if (mu == 2) { acc[2][a] = csub(acc[2][a], ctimesi(q0)); acc[3][a] = cadd(acc[3][a], ctimesi(q1)); }
                    if (mu == 3) { acc[2][a] = cadd(acc[2][a], q0); acc[3][a] = cadd(acc[3][a], q1); }
                }
            }
        }
    }
    C p[12];
    const bool has_src = src != nullptr;
    if (has_src) SpinorIO<P>::load(src + (size_t)f * ld, (size_t)Vh, (size_t)k, p, inv, plo);
    const R go = g5out ? R(-1) : R(1);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const R b = (sp < 2) ? beta * go : beta;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if constexpr (P == PDD) {
                acc[sp][a].x = normalize(acc[sp][a].x);
                acc[sp][a].y = normalize(acc[sp][a].y);
            }
            C v;
            if (has_src) {
                v.x = alpha * p[sp * 3 + a].x;
                v.y = alpha * p[sp * 3 + a].y;
                v.x = fma(b, acc[sp][a].x, v.x);
                v.y = fma(b, acc[sp][a].y, v.y);
            } else {
                v.x = b * acc[sp][a].x;
                v.y = b * acc[sp][a].y;
            }
            p[sp * 3 + a] = v;
        }
    }
    SpinorIO<P>::store(out + (size_t)f * ld, (size_t)Vh, (size_t)k, p, scl, plo);
}

}  // namespace

void launch_dslash(int prec, void* out, const void* in, size_t ld, const void* links, const Geom& g,
                   double kappa, int dag, const Ctl* ctl, int nf_static, int nf_max, float hscale,
                   cudaStream_t st, const void* links12, int max_ctas) {
    // D^H = gamma_5 D gamma_5: gamma_5 on the input and on the output
    const int g5in = dag, g5out = dag;
    // one CTA per (field, 32-site tile); with a control block the width is
    // read on the device and bounded by nf_max, otherwise it is nf_static
    const int nfg = ctl ? nf_max : nf_static;
    const int nf_grid = nfg < 1 ? 1 : nfg;
    dim3 block(32);
    dim3 grid((unsigned)(nf_grid * ((g.V + 31) / 32)));
    // FP64 / double-float: at most max_ctas CTAs striding over the work, so
    // that an ALU-bound stencil on a side stream leaves the SMs room for the
    // kernels of other streams
    if (max_ctas > 0 && grid.x > (unsigned)max_ctas) grid.x = (unsigned)max_ctas;
    const size_t sm = 0;
    // (SU(3) links: rows 0 and 1 staged, row 2 rebuilt at each use; 12 KB of
    // shared memory per CTA instead of 18, and 3.5% faster at 16^3 x 32)
#define DSBCG_CTA_LAUNCH(PP, S2T)                                                                               \
    if (links12)                                                                                                \
        dslash_cta_kernel<PP, true><<<cgrid, cblock, 0, st>>>((S2T*)out, (const S2T*)in, ld, (const S2T*)links,   \
                                                              (const S2T*)links12, g, (float)kappa, g5in, g5out,  \
                                                              ctl, nf_static, hscale, ngrp);                      \
    else                                                                                                        \
        dslash_cta_kernel<PP, false><<<cgrid, cblock, 0, st>>>((S2T*)out, (const S2T*)in, ld, (const S2T*)links,  \
                                                               nullptr, g, (float)kappa, g5in, g5out, ctl,        \
                                                               nf_static, hscale, ngrp)
    // FP32 and 16-bit fields: CTAs of 32 sites x CTA_FIELDS fields with the
    // tile's links staged in shared memory
    const int ngrp = (nf_grid + CTA_FIELDS - 1) / CTA_FIELDS;
    dim3 cgrid((unsigned)(ngrp * ((g.V + 31) / 32)));
    dim3 cblock(32 * CTA_FIELDS);
    switch (prec) {
        case P64:
            dslash_kernel<P64><<<grid, block, sm, st>>>((double2*)out, (const double2*)in, ld,
                                                         (const double2*)links, g, kappa, g5in, g5out,
                                                         ctl, nf_static, hscale, nf_grid);
            break;
        case P32: DSBCG_CTA_LAUNCH(P32, float2); break;
        case PBF16: DSBCG_CTA_LAUNCH(PBF16, __nv_bfloat162); break;
        case PF16: DSBCG_CTA_LAUNCH(PF16, __half2); break;
        case PDD:
            // ld: field stride in float2 words (two planes of the complex stride)
            dslash_kernel<PDD><<<grid, block, sm, st>>>((float2*)out, (const float2*)in, ld,
                                                         (const float2*)links, g, dd::from_double(kappa), g5in,
                                                         g5out, ctl, nf_static, hscale, nf_grid);
            break;
    }
#undef DSBCG_CTA_LAUNCH
}

void launch_dslash_half(int prec, void* out, const void* in, const void* src, size_t ld, const void* links,
                        const Geom& g, double alpha, double beta, int parity, int g5in, int g5out, const Ctl* ctl,
                        int nf_static, int nf_max, float hscale, cudaStream_t st) {
    const int nfg = ctl ? nf_max : nf_static;
    const int nf_grid = nfg < 1 ? 1 : nfg;
    dim3 block(32);
    dim3 grid((unsigned)(nf_grid * ((g.V / 2 + 31) / 32)));
#define DSBCG_HALF_LAUNCH(PP, S2T, RA, RB)                                                                     \
    dslash_half_kernel<PP><<<grid, block, 0, st>>>((S2T*)out, (const S2T*)in, (const S2T*)src, ld,            \
                                                   (const S2T*)links, g, RA, RB, parity, g5in, g5out, ctl,    \
                                                   nf_static, hscale, nf_grid)
    switch (prec) {
        case P64: DSBCG_HALF_LAUNCH(P64, double2, alpha, beta); break;
        case P32: DSBCG_HALF_LAUNCH(P32, float2, (float)alpha, (float)beta); break;
        case PBF16: DSBCG_HALF_LAUNCH(PBF16, __nv_bfloat162, (float)alpha, (float)beta); break;
        case PF16: DSBCG_HALF_LAUNCH(PF16, __half2, (float)alpha, (float)beta); break;
        case PDD: DSBCG_HALF_LAUNCH(PDD, float2, dd::from_double(alpha), dd::from_double(beta)); break;
    }
#undef DSBCG_HALF_LAUNCH
}

}  // namespace dsbcg

// Gauge-link gradient ("fermion force") of shifted solves.  Not in the paper;
// its RHMC motivation (Sec. 1) needs the derivative of the shifted solutions
// with respect to the links.  For field pairs (a_k, b_k), (c_k, d_k) with
// weights w_k this kernel forms
//   dU_mu(y) = kappa * sum_k w_k [F(a_k, b_k) + F(c_k, d_k)]_mu(y),
//   F(a, b)_mu(y) = sum_spin [(1 - gamma_mu) a(y)] (x) conj(b(y + mu))
//                 + sum_spin [(1 + gamma_mu) b(y)] (x) conj(a(y + mu)),
// times -1 for a hop across the antiperiodic time boundary.  With
// a = D x, b = lambda, c = D lambda, d = x this is dL/dU for adjoint
// solutions lambda (see include/dsbcg.h).  One thread per (site, mu); the
// 3x3 accumulator stays in registers across all field pairs; the result is
// written once, in the canonical complex128 [site][mu][3][3] layout.
#include "kernels.h"

namespace dsbcg {

namespace {

// the 12 components of site x: six 16-byte pair chunks for FP32 fields
template <int P>
__device__ __forceinline__ void load_sp(const typename Tr<P>::S2* f, size_t V, size_t x, typename Tr<P>::C p[12]) {
    if constexpr (P == P32) {
        const float4* q = reinterpret_cast<const float4*>(f);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float4 v = __ldg(q + (size_t)c * V + x);
            p[2 * c] = make_float2(v.x, v.y);
            p[2 * c + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 12; ++c) p[c] = Elem<P>::ld(f, fidx<P>(V, x, c), 1);
    }
}

// q = (1 - gamma_mu) p (fwd) or (1 + gamma_mu) p, full 4-spinor, chiral basis
template <class C>
__device__ __forceinline__ void project(int mu, bool minus, const C p[12], C q[12]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C u0 = p[a], u1 = p[3 + a], l0 = p[6 + a], l1 = p[9 + a];
        C h0, h1, r0, r1;
        if (minus) {
            if (mu == 0) { h0 = csub(u0, ctimesi(l1)); h1 = csub(u1, ctimesi(l0)); r0 = ctimesi(h1); r1 = ctimesi(h0); }
            else if (mu == 1) { h0 = csub(u0, l1); h1 = cadd(u1, l0); r0 = h1; r1 = mk(-h0.x, -h0.y); }
            else if (mu == 2) { h0 = csub(u0, ctimesi(l0)); h1 = cadd(u1, ctimesi(l1)); r0 = ctimesi(h0); r1 = mk(h1.y, -h1.x); }
            else { h0 = csub(u0, l0); h1 = csub(u1, l1); r0 = mk(-h0.x, -h0.y); r1 = mk(-h1.x, -h1.y); }
        } else {
            if (mu == 0) { h0 = cadd(u0, ctimesi(l1)); h1 = cadd(u1, ctimesi(l0)); r0 = mk(h1.y, -h1.x); r1 = mk(h0.y, -h0.x); }
            else if (mu == 1) { h0 = cadd(u0, l1); h1 = csub(u1, l0); r0 = mk(-h1.x, -h1.y); r1 = h0; }
            else if (mu == 2) { h0 = cadd(u0, ctimesi(l0)); h1 = csub(u1, ctimesi(l1)); r0 = mk(h0.y, -h0.x); r1 = ctimesi(h1); }
            else { h0 = cadd(u0, l0); h1 = cadd(u1, l1); r0 = h0; r1 = h1; }
        }
        q[a] = h0;
        q[3 + a] = h1;
        q[6 + a] = r0;
        q[9 + a] = r1;
    }
}

template <class C, class R>
__device__ __forceinline__ void outer_acc(C acc[9], const C pa[12], const C qb[12], R w) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                C t = cmulc(qb[s * 3 + b], pa[s * 3 + a]);      // conj(q_b) p_a
                acc[a * 3 + b].x = fma(w, t.x, acc[a * 3 + b].x);
                acc[a * 3 + b].y = fma(w, t.y, acc[a * 3 + b].y);
            }
}

template <int P>
__global__ void __launch_bounds__(256) force_kernel(double2* __restrict__ dU, const typename Tr<P>::S2* __restrict__ A,
                                                    const typename Tr<P>::S2* __restrict__ B,
                                                    const typename Tr<P>::S2* __restrict__ Cf,
                                                    const typename Tr<P>::S2* __restrict__ Df, size_t ld, int nf,
                                                    const double* __restrict__ wf, Geom g, double kappa) {
    using C = typename Tr<P>::C;
    using R = typename Tr<P>::R;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)g.V * 4) return;
    const int x = (int)(t >> 2), mu = (int)(t & 3);
    const size_t V = (size_t)g.V;
    // forward neighbour and boundary sign
    int c[4];
    {
        int r = x;
        c[0] = r % g.L[0]; r /= g.L[0];
        c[1] = r % g.L[1]; r /= g.L[1];
        c[2] = r % g.L[2]; c[3] = r / g.L[2];
    }
    int st = 1;
    for (int d = 0; d < mu; ++d) st *= g.L[d];
    int y = (c[mu] == g.L[mu] - 1) ? x - (g.L[mu] - 1) * st : x + st;
    double sign = (mu == 3 && g.tap && c[3] == g.L[3] - 1) ? -1.0 : 1.0;
    C acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = mk(R(0), R(0));
    for (int k = 0; k < nf; ++k) {
        const R w = (R)wf[k];            // one conversion per field (FP64 -> FP32 is slow on GB300)
        const size_t off = (size_t)k * ld;
        for (int pair = 0; pair < 2; ++pair) {
            const typename Tr<P>::S2* fa = (pair == 0 ? A : Cf) + off;
            const typename Tr<P>::S2* fb = (pair == 0 ? B : Df) + off;
            C p[12], q[12], pq[12];
            // [(1 - gamma_mu) a(y)] (x) conj(b(y + mu))
            load_sp<P>(fa, V, x, p);
            load_sp<P>(fb, V, y, q);
            switch (mu) {
                case 0: project(0, true, p, pq); break;
                case 1: project(1, true, p, pq); break;
                case 2: project(2, true, p, pq); break;
                default: project(3, true, p, pq); break;
            }
            outer_acc(acc, pq, q, w);
            // [(1 + gamma_mu) b(y)] (x) conj(a(y + mu))
            load_sp<P>(fb, V, x, p);
            load_sp<P>(fa, V, y, q);
            switch (mu) {
                case 0: project(0, false, p, pq); break;
                case 1: project(1, false, p, pq); break;
                case 2: project(2, false, p, pq); break;
                default: project(3, false, p, pq); break;
            }
            outer_acc(acc, pq, q, w);
        }
    }
    double2* o = dU + ((size_t)x * 4 + mu) * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q] = make_double2(kappa * sign * (double)acc[q].x, kappa * sign * (double)acc[q].y);
}

}  // namespace

void launch_force(int prec, double2* dU, const void* a, const void* b, const void* c, const void* d, size_t ld,
                  int nf, const double* w_per_field, const Geom& g, double kappa, cudaStream_t st) {
    size_t total = (size_t)g.V * 4;
    int grid = (int)((total + 255) / 256);
    if (prec == P64)
        force_kernel<P64><<<grid, 256, 0, st>>>(dU, (const double2*)a, (const double2*)b, (const double2*)c,
                                                (const double2*)d, ld, nf, w_per_field, g, kappa);
    else
        force_kernel<P32><<<grid, 256, 0, st>>>(dU, (const float2*)a, (const float2*)b, (const float2*)c,
                                                (const float2*)d, ld, nf, w_per_field, g, kappa);
}

}  // namespace dsbcg

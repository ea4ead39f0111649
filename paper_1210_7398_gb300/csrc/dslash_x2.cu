// K1x2: the operator D = 1 - kappa F H of Eq. (2) in pair-of-FP32 arithmetic, for the outer
// iteration of the nested solver (Sec. 2).
//
// The outer BiCGStab applies D to the inner solver's output, an FP32 vector, and needs the result
// to about FP64 accuracy.  On GB300 the FP64 pipe runs at 1/64 of the FP32 rate, which makes the
// FP64 D ALU-bound at a tenth of its bandwidth roofline.  This form keeps the input in FP32
// (exactly the inner solver's output), holds links and clover as hi + lo pairs of FP32 numbers
// (Dekker's double-length representation, about 48 significant bits), and does every product and
// sum without losing the low part: products by the FMA error term (Dekker's TwoProduct with a fused
// multiply-add), sums of leading parts by Knuth's TwoSum, and the small cross terms and error
// terms in plain FP32 into a low accumulator.  The relative error is about 2^-46 per site, within
// 1e-13 of the FP64 D in norm, and all of it runs on the FP32 pipe as packed FP32x2 instructions
// (real and imaginary part in one).  The FP64 output is formed once per component at the end.
//
// Layout: input FP32 spinors [nrhs][6][V] float4, output FP64 [nrhs][12][V] double2 (the internal
// layouts); links [4][9][V] and clover [36][V] as float4 (hi of two reals, lo of the same two), made
// from the FP64 fields on first use after each field change.  One thread per (site, right-hand
// side), the right-hand side fastest over the grid as in the other D kernels.
#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {
namespace {

// a complex number h + l, each part a packed (re, im) pair of FP32
struct CX {
    float2 h, l;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 rot(float2 z) { return make_float2(-z.y, z.x); }  // i z

// Knuth's TwoSum, componentwise: s = fl(a + b) and e with s + e = a + b exactly
__device__ __forceinline__ float2 two_sum(float2 a, float2 b, float2 &e) {
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
    return s;
}

// exact sign / i-multiples of a pair-complex: 0: z, 1: -z, 2: i z, 3: -i z
template <int K> __device__ __forceinline__ CX xf(const CX &z) {
    if (K == 0) return z;
    if (K == 1) return CX{neg2(z.h), neg2(z.l)};
    if (K == 2) return CX{rot(z.h), rot(z.l)};
    return CX{neg2(rot(z.h)), neg2(rot(z.l))};
}
template <int K> __device__ __forceinline__ float2 xf1(float2 z) {
    if (K == 0) return z;
    if (K == 1) return neg2(z);
    if (K == 2) return rot(z);
    return neg2(rot(z));
}

// acc += t
__device__ __forceinline__ void acc_add(CX &acc, const CX &t) {
    float2 e;
    acc.h = two_sum(acc.h, t.h, e);
    acc.l = add2(acc.l, add2(e, t.l));
}

// acc += W x (FIRST: acc = W x), W and x pair-complex; xr = i x.h, xlr = i x.l.  The leading product
// W.h x.h is split into its two packed halves P1 = Re(W.h) x.h and P2 = Im(W.h) (i x.h), each kept
// exactly as product + FMA error; the cross terms W.h x.l + W.l x.h are small and go to the low
// part in FP32.
template <bool FIRST>
__device__ __forceinline__ void cmac(CX &acc, const CX &W, const CX &x, float2 xr, float2 xlr) {
    const float2 wr = splat(W.h.x), wi = splat(W.h.y);
    const float2 P1 = mul2(wr, x.h), P2 = mul2(wi, xr);
    const float2 E1 = fma2(wr, x.h, neg2(P1)), E2 = fma2(wi, xr, neg2(P2));
    const float2 cr = fma2(splat(W.l.x), x.h, fma2(splat(W.l.y), xr, fma2(wr, x.l, mul2(wi, xlr))));
    float2 e1, e2;
    if (FIRST) {
        acc.h = two_sum(P1, P2, e1);
        acc.l = add2(add2(e1, E1), add2(E2, cr));
    } else {
        const float2 s = two_sum(acc.h, P1, e1);
        acc.h = two_sum(s, P2, e2);
        acc.l = add2(acc.l, add2(add2(e1, e2), add2(add2(E1, E2), cr)));
    }
}
__device__ __forceinline__ CX conj(const CX &a) {
    return CX{make_float2(a.h.x, -a.h.y), make_float2(a.l.x, -a.l.y)};
}

__device__ __forceinline__ CX ld_cx(const float4 *__restrict__ p) {
    const float4 v = __ldg(p);
    return CX{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

// the projected half-spinor of (1 -/+ gamma_mu) psi, exactly: the same sums as hop_project, each by
// TwoSum (MU = 3: 2 sgn psi_k, exact in FP32)
template <int MU, bool FWD>
__device__ __forceinline__ void project_x2(const float2 p[12], float sgn, CX h[6]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float2 p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        float2 a0, b0, a1, b1;  // h0 = a0 + b0, h1 = a1 + b1
        if (MU == 0) {
            a0 = p0; b0 = FWD ? xf1<2>(p3) : xf1<3>(p3);
            a1 = p1; b1 = FWD ? xf1<2>(p2) : xf1<3>(p2);
        } else if (MU == 1) {
            a0 = p0; b0 = FWD ? p3 : neg2(p3);
            a1 = p1; b1 = FWD ? neg2(p2) : p2;
        } else if (MU == 2) {
            a0 = p0; b0 = FWD ? xf1<2>(p2) : xf1<3>(p2);
            a1 = p1; b1 = FWD ? xf1<3>(p3) : xf1<2>(p3);
        }
        if (MU == 3) {
            const float2 s2 = splat(2.0f * sgn);
            h[c] = CX{mul2(s2, FWD ? p2 : p0), make_float2(0.f, 0.f)};
            h[3 + c] = CX{mul2(s2, FWD ? p3 : p1), make_float2(0.f, 0.f)};
        } else {
            h[c].h = two_sum(a0, b0, h[c].l);
            h[3 + c].h = two_sum(a1, b1, h[3 + c].l);
        }
    }
}

// adds the transported half-spinor rows w0 = (W h)_a, w1 = (W h)_{3+a} to acc with the
// reconstruction of hop_reconstruct
template <int MU, bool FWD>
__device__ __forceinline__ void reconstruct_x2(int a, const CX &w0, const CX &w1, CX acc[12]) {
    if (MU == 3) {
        if (FWD) { acc_add(acc[6 + a], w0); acc_add(acc[9 + a], w1); }
        else     { acc_add(acc[a], w0);     acc_add(acc[3 + a], w1); }
        return;
    }
    acc_add(acc[a], w0);
    acc_add(acc[3 + a], w1);
    if (MU == 0) {
        if (FWD) { acc_add(acc[6 + a], xf<3>(w1)); acc_add(acc[9 + a], xf<3>(w0)); }
        else     { acc_add(acc[6 + a], xf<2>(w1)); acc_add(acc[9 + a], xf<2>(w0)); }
    } else if (MU == 1) {
        if (FWD) { acc_add(acc[6 + a], xf<1>(w1)); acc_add(acc[9 + a], w0); }
        else     { acc_add(acc[6 + a], w1);        acc_add(acc[9 + a], xf<1>(w0)); }
    } else {
        if (FWD) { acc_add(acc[6 + a], xf<3>(w0)); acc_add(acc[9 + a], xf<2>(w1)); }
        else     { acc_add(acc[6 + a], xf<2>(w0)); acc_add(acc[9 + a], xf<3>(w1)); }
    }
}

// one hop term: (1 - gamma_mu) U_mu(n) psi(n+mu) forward, (1 + gamma_mu) U_mu(n-mu)^dag psi(n-mu)
// backward; ulink is the site whose link is used
template <int MU, bool FWD>
__device__ __forceinline__ void hop_x2(const float4 *__restrict__ src, const float4 *__restrict__ Ux2, long V,
                                       long nb, long ulink, float sgn, CX acc[12]) {
    float2 p[12];
    load_spinor(src, V, nb, p);
    CX h[6];
    project_x2<MU, FWD>(p, sgn, h);
    float2 hr[6], hlr[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        hr[k] = rot(h[k].h);
        hlr[k] = rot(h[k].l);
    }
    const float4 *u = Ux2 + (long)(MU * 9) * V + ulink;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        CX w0, w1;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            // W[a][b] = U[a][b] forward, conj(U[b][a]) backward
            const CX W = FWD ? ld_cx(u + (long)(a * 3 + b) * V) : conj(ld_cx(u + (long)(b * 3 + a) * V));
            if (b == 0) {
                cmac<true>(w0, W, h[b], hr[b], hlr[b]);
                cmac<true>(w1, W, h[3 + b], hr[3 + b], hlr[3 + b]);
            } else {
                cmac<false>(w0, W, h[b], hr[b], hlr[b]);
                cmac<false>(w1, W, h[3 + b], hr[3 + b], hlr[3 + b]);
            }
        }
        reconstruct_x2<MU, FWD>(a, w0, w1, acc);
    }
}

// y = H6 x for one packed Hermitian block (18 float4 at F, stride V: the 6 real diagonal
// entries in the first three, then the 15 complex entries below the diagonal in row order), the
// same order of terms as herm6_mul
__device__ __forceinline__ void herm6_x2(const float4 *__restrict__ F, long V, const CX x[6], CX y[6]) {
    float2 xr[6], xlr[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        xr[k] = rot(x[k].h);
        xlr[k] = rot(x[k].l);
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float4 d = __ldg(F + (long)j * V);
        // real diagonal entries (d.x, d.z) and (d.y, d.w) times x: product, its error, cross terms
#pragma unroll
        for (int t = 0; t < 2; t++) {
            const int i = 2 * j + t;
            const float2 dh = splat(t ? d.y : d.x), dl = splat(t ? d.w : d.z);
            const float2 P = mul2(dh, x[i].h);
            y[i].h = P;
            y[i].l = add2(fma2(dh, x[i].h, neg2(P)), fma2(dh, x[i].l, mul2(dl, x[i].h)));
        }
    }
    int k = 3;
#pragma unroll
    for (int i = 1; i < 6; i++) {
#pragma unroll
        for (int j = 0; j < i; j++) {
            const CX a = ld_cx(F + (long)k * V);
            k++;
            cmac<false>(y[i], a, x[j], xr[j], xlr[j]);        // row i gets H_ij x_j
            cmac<false>(y[j], conj(a), x[i], xr[i], xlr[i]);  // row j gets conj(H_ij) x_i
        }
    }
}

__device__ __forceinline__ double to_f64(float h, float l) { return (double)h + (double)l; }

template <int MINB>
__global__ void __launch_bounds__(128, MINB) dslash_x2_kernel(double2 *__restrict__ out, const float4 *__restrict__ in,
                                                          const float4 *__restrict__ Ux2,
                                                          const float4 *__restrict__ Fx2, float kh, float kl,
                                                          Geo g, int nrhs) {
    // the right-hand side fastest over the grid: a site block's links and clover are shared
    // through L2 by all right-hand sides (measured as fast as the right-hand side slowest, which
    // keeps one sweep's neighbour slices in L2, at 24^3x48 and 48^3x96)
    const long sblk = blockIdx.x / nrhs;
    const int rhs = (int)(blockIdx.x - sblk * nrhs);
    const long n = sblk * blockDim.x + threadIdx.x;
    if (n >= g.V) return;
    const long V = g.V;
    const float4 *src = in + (long)rhs * 6 * V;
    int x[4];
    site_coords(g, n, x);
    CX acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = CX{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const float tsgn_f = (x[3] == g.L[3] - 1) ? (float)g.bc_t : 1.f;
    const float tsgn_b = (x[3] == 0) ? (float)g.bc_t : 1.f;
    { long m = nbr_fwd<0>(g, n, x); hop_x2<0, true>(src, Ux2, V, m, n, 1.f, acc); }
    { long m = nbr_bwd<0>(g, n, x); hop_x2<0, false>(src, Ux2, V, m, m, 1.f, acc); }
    { long m = nbr_fwd<1>(g, n, x); hop_x2<1, true>(src, Ux2, V, m, n, 1.f, acc); }
    { long m = nbr_bwd<1>(g, n, x); hop_x2<1, false>(src, Ux2, V, m, m, 1.f, acc); }
    { long m = nbr_fwd<2>(g, n, x); hop_x2<2, true>(src, Ux2, V, m, n, 1.f, acc); }
    { long m = nbr_bwd<2>(g, n, x); hop_x2<2, false>(src, Ux2, V, m, m, 1.f, acc); }
    { long m = nbr_fwd<3>(g, n, x); hop_x2<3, true>(src, Ux2, V, m, n, tsgn_f, acc); }
    { long m = nbr_bwd<3>(g, n, x); hop_x2<3, false>(src, Ux2, V, m, m, tsgn_b, acc); }
    // clover in the chiral basis: c0 = v_u - v_l, c1 = v_u + v_l, e_k = (F_k / 2) c_k,
    // (F v)_u = e0 + e1, (F v)_l = e1 - e0 (as clover_mul)
    CX c0[6], c1[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        c0[k] = acc[k];
        acc_add(c0[k], xf<1>(acc[k + 6]));
        c1[k] = acc[k];
        acc_add(c1[k], acc[k + 6]);
    }
    CX e0[6], e1[6];
    herm6_x2(Fx2 + n, V, c0, e0);
    herm6_x2(Fx2 + 18 * V + n, V, c1, e1);
    float2 psi[12];
    load_spinor(src, V, n, psi);
    double2 *dst = out + (long)rhs * 12 * V + n;
    const float2 kH = splat(kh), kL = splat(kl);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        CX t;
        if (k < 6) { t = e0[k]; acc_add(t, e1[k]); }
        else       { t = e1[k - 6]; acc_add(t, xf<1>(e0[k - 6])); }
        // psi - kappa t, kappa = kh + kl
        const float2 P = mul2(kH, t.h);
        const float2 E = fma2(kH, t.h, neg2(P));
        const float2 cr = fma2(kH, t.l, mul2(kL, t.h));
        float2 e;
        const float2 s = two_sum(psi[k], neg2(P), e);
        const float2 lo = sub2(e, add2(E, cr));
        dst[(long)k * V] = make_double2(to_f64(s.x, lo.x), to_f64(s.y, lo.y));
    }
}

// hi + lo split of FP64 values: hi = fl32(v), lo = fl32(v - hi); |v - hi - lo| <= 2^-48 |v|
__device__ __forceinline__ float4 split_pair(double2 v) {
    const float hx = __double2float_rn(v.x), hy = __double2float_rn(v.y);
    return make_float4(hx, hy, __double2float_rn(v.x - (double)hx), __double2float_rn(v.y - (double)hy));
}

__global__ void k_fields_to_x2(float4 *__restrict__ Ux2, float4 *__restrict__ Fx2, const double2 *__restrict__ U64,
                               const double2 *__restrict__ F64, long V) {
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= V) return;
    for (int k = 0; k < 36; k++) {
        Ux2[k * V + n] = split_pair(U64[k * V + n]);
        Fx2[k * V + n] = split_pair(F64[k * V + n]);
    }
}

}  // namespace

int dslash_x2(qcd_ctx *c, double2 *out, const float4 *in, int nrhs) {
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = c->lat.V;
    g.bc_t = c->bc_t;
    if (!c->Ux2) {
        int rc = dev_alloc(c, (void **)&c->Ux2, sizeof(float4) * 36 * g.V);
        if (!rc) rc = dev_alloc(c, (void **)&c->Fx2, sizeof(float4) * 36 * g.V);
        if (rc) return rc;
    }
    if (c->x2_version != c->field_version) {
        k_fields_to_x2<<<(unsigned)((g.V + 255) / 256), 256, 0, c->stream>>>(c->Ux2, c->Fx2, c->U64, c->F64, g.V);
        QCD_CUDA(c, cudaGetLastError());
        c->x2_version = c->field_version;
    }
    const float kh = (float)c->kappa;
    const float kl = (float)(c->kappa - (double)kh);
    cudaEvent_t ev;
    prof_begin(c, QCD_K_DSLASH64, &ev);
    // three CTAs of 128 threads per SM (168 registers, a few spilled): 12% faster than two
    // without spills at 24^3x48 and 48^3x96
    dslash_x2_kernel<3><<<dim3((unsigned)((g.V + 127) / 128 * nrhs)), 128, 0, c->stream>>>(out, in, c->Ux2, c->Fx2,
                                                                                           kh, kl, g, nrhs);
    return prof_end(c, QCD_K_DSLASH64, ev);
}

}  // namespace qcd

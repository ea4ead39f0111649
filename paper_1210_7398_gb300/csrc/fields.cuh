// Device-side building blocks of the operator D = 1 - kappa F H (Eq. (2)):
// complex arithmetic, field loads/stores in the internal layouts, the spin
// projection to half-spinors in the Dirac representation (gamma_4 diagonal),
// the SU(3) multiply, the reconstruction, and the clover multiply in the
// chiral representation (Sec. 3: F stored chirally, applied to Dirac-basis
// spinors by converting on the fly).
#pragma once

#include <cuda_runtime.h>

namespace qcd {

template <typename R> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) re, decltype(C::x) im) {
    C r; r.x = re; r.y = im; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
// a + i b, a - i b
template <typename C> __device__ __forceinline__ C caddi(C a, C b) { return cmk<C>(a.x - b.y, a.y + b.x); }
template <typename C> __device__ __forceinline__ C csubi(C a, C b) { return cmk<C>(a.x + b.y, a.y - b.x); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a)*b
template <typename C> __device__ __forceinline__ C cfmac(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
// i*a, -i*a
template <typename C> __device__ __forceinline__ C cmuli(C a) { return cmk<C>(-a.y, a.x); }
template <typename C> __device__ __forceinline__ C cmulmi(C a) { return cmk<C>(a.y, -a.x); }
// FP32 complex sums as one packed FP32x2 add each (the same IEEE sums, half the instructions)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 caddi(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.y, b.x)); }
__device__ __forceinline__ float2 csubi(float2 a, float2 b) { return __fadd2_rn(a, make_float2(b.y, -b.x)); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }

// ---- loads / stores in the internal layouts ---------------------------------

__device__ __forceinline__ void load_spinor(const float4 *__restrict__ p, long V, long n, float2 s[12]) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 v = __ldg(p + k * V + n);
        s[2 * k] = make_float2(v.x, v.y);
        s[2 * k + 1] = make_float2(v.z, v.w);
    }
}
__device__ __forceinline__ void load_spinor(const double2 *__restrict__ p, long V, long n, double2 s[12]) {
#pragma unroll
    for (int k = 0; k < 12; k++) s[k] = __ldg(p + k * V + n);
}
// coherent loads (data written earlier by the same kernel)
__device__ __forceinline__ void load_spinor_rw(const float4 *p, long V, long n, float2 s[12]) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 v = p[k * V + n];
        s[2 * k] = make_float2(v.x, v.y);
        s[2 * k + 1] = make_float2(v.z, v.w);
    }
}
__device__ __forceinline__ void store_spinor(float4 *p, long V, long n, const float2 s[12]) {
#pragma unroll
    for (int k = 0; k < 6; k++) p[k * V + n] = make_float4(s[2 * k].x, s[2 * k].y, s[2 * k + 1].x, s[2 * k + 1].y);
}
__device__ __forceinline__ void store_spinor(double2 *p, long V, long n, const double2 s[12]) {
#pragma unroll
    for (int k = 0; k < 12; k++) p[k * V + n] = s[k];
}

__device__ __forceinline__ void load_link(const float2 *__restrict__ U, long V, long n, int mu, float2 u[9]) {
#pragma unroll
    for (int i = 0; i < 9; i++) u[i] = __ldg(U + (mu * 9 + i) * V + n);
}
__device__ __forceinline__ void load_link(const double2 *__restrict__ U, long V, long n, int mu, double2 u[9]) {
#pragma unroll
    for (int i = 0; i < 9; i++) u[i] = __ldg(U + (mu * 9 + i) * V + n);
}

// clover: 72 reals per site = two packed Hermitian 6x6 blocks of F/2 in the
// chiral basis; block layout: 6 real diagonal entries, then the 15 complex
// entries below the diagonal in row order (1,0),(2,0),(2,1),(3,0),...,(5,4).
__device__ __forceinline__ void load_clover(const float4 *__restrict__ F, long V, long n, float f[72]) {
#pragma unroll
    for (int k = 0; k < 18; k++) {
        float4 v = __ldg(F + k * V + n);
        f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
    }
}
__device__ __forceinline__ void load_clover(const double2 *__restrict__ F, long V, long n, double f[72]) {
#pragma unroll
    for (int k = 0; k < 36; k++) {
        double2 v = __ldg(F + k * V + n);
        f[2 * k] = v.x; f[2 * k + 1] = v.y;
    }
}

// y = H6 x for one packed Hermitian 6x6 block (pointer to its 36 reals)
template <typename R, typename C>
__device__ __forceinline__ void herm6_mul(const R *h, const C x[6], C y[6]) {
#pragma unroll
    for (int i = 0; i < 6; i++) y[i] = cscale(x[i], h[i]);
    int k = 6;
#pragma unroll
    for (int i = 1; i < 6; i++) {
#pragma unroll
        for (int j = 0; j < i; j++) {
            C a = cmk<C>(h[k], h[k + 1]);
            k += 2;
            y[i] = cfma(a, x[j], y[i]);   // row i gets H_ij x_j
            y[j] = cfmac(a, x[i], y[j]);  // row j gets conj(H_ij) x_i
        }
    }
}

// out = F v for a Dirac-basis spinor v[spin*3+colour]: chiral components
// c0 = v_u - v_l, c1 = v_u + v_l, eta_k = (F_k/2) c_k, then
// (F v)_u = eta0 + eta1, (F v)_l = eta1 - eta0.
template <typename R, typename C>
__device__ __forceinline__ void clover_mul(const R f[72], const C v[12], C out[12]) {
    C c0[6], c1[6], e0[6], e1[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        c0[k] = csub(v[k], v[k + 6]);
        c1[k] = cadd(v[k], v[k + 6]);
    }
    herm6_mul<R, C>(f, c0, e0);
    herm6_mul<R, C>(f + 36, c1, e1);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        out[k] = cadd(e0[k], e1[k]);
        out[k + 6] = csub(e1[k], e0[k]);
    }
}

// ---- one hop term -------------------------------------------------------------
// Adds  (1 - gamma_mu) U_mu(n) psi(n+mu)        (FWD = true)
//   or  (1 + gamma_mu) U_mu(n-mu)^dag psi(n-mu)  (FWD = false)
// to acc (Dirac representation, gamma_k = [[0,-i s_k],[i s_k,0]], gamma_4 =
// diag(1,1,-1,-1)); the projector has rank 2, so the colour multiply acts on
// the two-component half-spinor h only.  sgn is the boundary sign of a hop
// across the t edge (only MU = 3 can carry one).

// the half-spinor h[spin row * 3 + colour] of (1 -/+ gamma_mu) psi
template <int MU, bool FWD, typename C>
__device__ __forceinline__ void hop_project(const C psi[12], decltype(C::x) sgn, C h[6]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const C p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
        C h0, h1;
        if (MU == 0) {
            h0 = FWD ? caddi(p0, p3) : csubi(p0, p3);
            h1 = FWD ? caddi(p1, p2) : csubi(p1, p2);
        } else if (MU == 1) {
            h0 = FWD ? cadd(p0, p3) : csub(p0, p3);
            h1 = FWD ? csub(p1, p2) : cadd(p1, p2);
        } else if (MU == 2) {
            h0 = FWD ? caddi(p0, p2) : csubi(p0, p2);
            h1 = FWD ? csubi(p1, p3) : caddi(p1, p3);
        } else {
            h0 = FWD ? cscale(p2, 2 * sgn) : cscale(p0, 2 * sgn);
            h1 = FWD ? cscale(p3, 2 * sgn) : cscale(p1, 2 * sgn);
        }
        h[c] = h0;
        h[3 + c] = h1;
    }
}

// adds the transported half-spinor w (both spin rows) to acc, reconstructing the other two
// spin components of (1 -/+ gamma_mu)
template <int MU, bool FWD, typename C>
__device__ __forceinline__ void hop_reconstruct(const C w[6], C acc[12]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const C w0 = w[a], w1 = w[3 + a];
        if (MU == 3) {
            if (FWD) { acc[6 + a] = cadd(acc[6 + a], w0); acc[9 + a] = cadd(acc[9 + a], w1); }
            else     { acc[a] = cadd(acc[a], w0);         acc[3 + a] = cadd(acc[3 + a], w1); }
            continue;
        }
        acc[a] = cadd(acc[a], w0);
        acc[3 + a] = cadd(acc[3 + a], w1);
        if (MU == 0) {
            if (FWD) { acc[6 + a] = cadd(acc[6 + a], cmulmi(w1)); acc[9 + a] = cadd(acc[9 + a], cmulmi(w0)); }
            else     { acc[6 + a] = cadd(acc[6 + a], cmuli(w1));  acc[9 + a] = cadd(acc[9 + a], cmuli(w0)); }
        } else if (MU == 1) {
            if (FWD) { acc[6 + a] = csub(acc[6 + a], w1); acc[9 + a] = cadd(acc[9 + a], w0); }
            else     { acc[6 + a] = cadd(acc[6 + a], w1); acc[9 + a] = csub(acc[9 + a], w0); }
        } else {
            if (FWD) { acc[6 + a] = cadd(acc[6 + a], cmulmi(w0)); acc[9 + a] = cadd(acc[9 + a], cmuli(w1)); }
            else     { acc[6 + a] = cadd(acc[6 + a], cmuli(w0));  acc[9 + a] = cadd(acc[9 + a], cmulmi(w1)); }
        }
    }
}

template <int MU, bool FWD, typename C>
__device__ __forceinline__ void hop_term(const C psi[12], const C u[9], decltype(C::x) sgn, C acc[12]) {
    C h[6];
    hop_project<MU, FWD>(psi, sgn, h);
    // colour multiply: U h (forward) or U^dag h (backward)
    C w[6];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C w0 = cmk<C>(0, 0), w1 = cmk<C>(0, 0);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (FWD) {
                w0 = cfma(u[a * 3 + b], h[b], w0);
                w1 = cfma(u[a * 3 + b], h[3 + b], w1);
            } else {
                w0 = cfmac(u[b * 3 + a], h[b], w0);
                w1 = cfmac(u[b * 3 + a], h[3 + b], w1);
            }
        }
        w[a] = w0;
        w[3 + a] = w1;
    }
    hop_reconstruct<MU, FWD>(w, acc);
}

// The same hop with the transport matrix given as it acts: W = U_mu(n) forward and
// W = U_mu(n-mu)^dag backward, both as W h (row-major W[a][b]); sgn as above.
template <int MU, bool FWD, typename C>
__device__ __forceinline__ void hop_term_w(const C psi[12], const C W[9], C acc[12], decltype(C::x) sgn = 1) {
    C h[6];
    hop_project<MU, FWD>(psi, sgn, h);
    C w[6];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C w0 = cmk<C>(0, 0), w1 = cmk<C>(0, 0);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            w0 = cfma(W[a * 3 + b], h[b], w0);
            w1 = cfma(W[a * 3 + b], h[3 + b], w1);
        }
        w[a] = w0;
        w[3 + a] = w1;
    }
    hop_reconstruct<MU, FWD>(w, acc);
}

// third row of a special unitary 3x3 matrix from its first two: row2 = conj(row0 x row1)
// (Table 1's reconstruction of a link from 12 reals)
template <typename C> __device__ __forceinline__ void su3_third_row(C W[9]);
// FP32: each entry conj(W_k W_{3+l} - W_l W_{3+k}) from packed pairs p = Re(W_k) W_{3+l} -
// Re(W_l) W_{3+k} and q = Im(W_k) W_{3+l} - Im(W_l) W_{3+k}: the product is (p.x - q.y, p.y + q.x)
template <> __device__ __forceinline__ void su3_third_row<float2>(float2 W[9]) {
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        float2 p = __fmul2_rn(make_float2(W[k].x, W[k].x), W[3 + l]);
        float2 q = __fmul2_rn(make_float2(W[k].y, W[k].y), W[3 + l]);
        p = __ffma2_rn(make_float2(-W[l].x, -W[l].x), W[3 + k], p);
        q = __ffma2_rn(make_float2(-W[l].y, -W[l].y), W[3 + k], q);
        W[6 + j] = make_float2(p.x - q.y, -(p.y + q.x));
    }
}
template <typename C> __device__ __forceinline__ void su3_third_row(C W[9]) {
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        const C a = csub(cmul(W[k], W[3 + l]), cmul(W[l], W[3 + k]));
        W[6 + j] = cmk<C>(a.x, -a.y);
    }
}

struct Geo {
    int L[4];
    long V;
    int bc_t;
};

__device__ __forceinline__ void site_coords(const Geo &g, long n, int x[4]) {
    long r = n;
    x[0] = (int)(r % g.L[0]); r /= g.L[0];
    x[1] = (int)(r % g.L[1]); r /= g.L[1];
    x[2] = (int)(r % g.L[2]); r /= g.L[2];
    x[3] = (int)r;
}

// neighbour of n (coordinates x) along mu in direction +1 / -1 (periodic)
template <int MU>
__device__ __forceinline__ long nbr_fwd(const Geo &g, long n, const int x[4]) {
    long stride = 1;
#pragma unroll
    for (int m = 0; m < MU; m++) stride *= g.L[m];
    return (x[MU] == g.L[MU] - 1) ? n - stride * (g.L[MU] - 1) : n + stride;
}
template <int MU>
__device__ __forceinline__ long nbr_bwd(const Geo &g, long n, const int x[4]) {
    long stride = 1;
#pragma unroll
    for (int m = 0; m < MU; m++) stride *= g.L[m];
    return (x[MU] == 0) ? n + stride * (g.L[MU] - 1) : n - stride;
}

}  // namespace qcd

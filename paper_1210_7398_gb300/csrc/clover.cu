// K2: the inverse clover term of Eq. (2),
//   F(n) = (1 - (c_SW kappa/2) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(n))^{-1},
// with F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag)/(8i) and Q the clover-leaf sum
// of the four plaquettes around n in the (mu,nu) plane.  sigma_{mu nu} F_{mu nu}
// commutes with gamma_5, so in the chiral representation the 12x12 matrix is
// two 6x6 blocks (Sec. 3: the clover term is kept in the chiral
// representation); each block is built and inverted in FP64 (Gauss-Jordan,
// partial pivoting), halved (the 1/2 of the basis change back to the Dirac
// representation is folded in), and stored packed in FP64 and FP32.
#include <cmath>
#include <complex>

#include "fields.cuh"
#include "qcd_internal.h"

namespace qcd {

// chiral 2x2 blocks of sigma_{mu nu} for the 6 planes (mu<nu), [plane][chirality][2][2]
__constant__ double2 c_sigma_chiral[6][2][2][2];

namespace {

using cd = std::complex<double>;

// chiral basis: row s of block 0 is (psi_u[s] - psi_l[s])/sqrt2, of block 1 (psi_u[s] + psi_l[s])/sqrt2
void host_sigma_tables(double2 out[6][2][2][2], bool *ok) {
    cd g[4][4][4] = {};
    const cd i(0, 1);
    cd pauli[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -i}, {i, 0}}, {{1, 0}, {0, -1}}};
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                g[k][a][2 + b] = -i * pauli[k][a][b];
                g[k][2 + a][b] = i * pauli[k][a][b];
            }
    g[3][0][0] = g[3][1][1] = 1.0;
    g[3][2][2] = g[3][3][3] = -1.0;
    const double r = 1.0 / std::sqrt(2.0);
    cd T[4][4] = {};
    for (int s = 0; s < 2; s++) {
        T[s][s] = r; T[s][2 + s] = -r;
        T[2 + s][s] = r; T[2 + s][2 + s] = r;
    }
    *ok = true;
    int plane = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, plane++) {
            cd sg[4][4], tmp[4][4], ch[4][4];
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    cd s = 0;
                    for (int k = 0; k < 4; k++) s += g[mu][a][k] * g[nu][k][b] - g[nu][a][k] * g[mu][k][b];
                    sg[a][b] = 0.5 * i * s;
                }
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    cd s = 0;
                    for (int k = 0; k < 4; k++) s += T[a][k] * sg[k][b];
                    tmp[a][b] = s;
                }
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    cd s = 0;
                    for (int k = 0; k < 4; k++) s += tmp[a][k] * std::conj(T[b][k]);
                    ch[a][b] = s;
                }
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) {
                    if (std::abs(ch[a][2 + b]) > 1e-14 || std::abs(ch[2 + a][b]) > 1e-14) *ok = false;
                    out[plane][0][a][b] = make_double2(ch[a][b].real(), ch[a][b].imag());
                    out[plane][1][a][b] = make_double2(ch[2 + a][2 + b].real(), ch[2 + a][2 + b].imag());
                }
        }
}

__device__ __forceinline__ void m3_load(const double2 *__restrict__ U, long V, long n, int mu, double2 m[9]) {
    load_link(U, V, n, mu, m);
}
__device__ __forceinline__ void m3_mul(const double2 a[9], const double2 b[9], double2 c[9]) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double2 s = make_double2(0, 0);
            for (int k = 0; k < 3; k++) s = cfma(a[i * 3 + k], b[k * 3 + j], s);
            c[i * 3 + j] = s;
        }
}
__device__ __forceinline__ void m3_dag(const double2 a[9], double2 c[9]) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c[i * 3 + j] = make_double2(a[j * 3 + i].x, -a[j * 3 + i].y);
}
// acc += A B C D with the given daggers
__device__ void plaq_add(const double2 *a, bool da, const double2 *b, bool db, const double2 *c, bool dc,
                         const double2 *d, bool dd, double2 acc[9]) {
    double2 A[9], B[9], Cm[9], Dm[9], t1[9], t2[9];
    if (da) m3_dag(a, A); else for (int k = 0; k < 9; k++) A[k] = a[k];
    if (db) m3_dag(b, B); else for (int k = 0; k < 9; k++) B[k] = b[k];
    if (dc) m3_dag(c, Cm); else for (int k = 0; k < 9; k++) Cm[k] = c[k];
    if (dd) m3_dag(d, Dm); else for (int k = 0; k < 9; k++) Dm[k] = d[k];
    m3_mul(A, B, t1);
    m3_mul(t1, Cm, t2);
    m3_mul(t2, Dm, t1);
    for (int k = 0; k < 9; k++) acc[k] = cadd(acc[k], t1[k]);
}

__device__ long shifted(const Geo &g, const int x[4], int mu, int dm, int nu, int dn) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = (y[mu] + dm + g.L[mu]) % g.L[mu];
    y[nu] = (y[nu] + dn + g.L[nu]) % g.L[nu];
    return y[0] + (long)g.L[0] * (y[1] + (long)g.L[1] * (y[2] + (long)g.L[2] * y[3]));
}

// invert a 6x6 complex matrix in place (Gauss-Jordan, partial pivoting); false if singular
__device__ bool inv6(double2 a[6][6]) {
    double2 b[6][6];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) b[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    for (int col = 0; col < 6; col++) {
        int piv = col;
        double best = hypot(a[col][col].x, a[col][col].y);
        for (int r = col + 1; r < 6; r++) {
            double v = hypot(a[r][col].x, a[r][col].y);
            if (v > best) { best = v; piv = r; }
        }
        if (!(best >= 1e-300)) return false;
        if (piv != col)
            for (int j = 0; j < 6; j++) {
                double2 t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t;
                t = b[col][j]; b[col][j] = b[piv][j]; b[piv][j] = t;
            }
        const double2 p = a[col][col];
        const double den = p.x * p.x + p.y * p.y;
        const double2 pinv = make_double2(p.x / den, -p.y / den);
        for (int j = 0; j < 6; j++) { a[col][j] = cmul(a[col][j], pinv); b[col][j] = cmul(b[col][j], pinv); }
        for (int r = 0; r < 6; r++) {
            if (r == col) continue;
            const double2 f = a[r][col];
            for (int j = 0; j < 6; j++) {
                a[r][j] = csub(a[r][j], cmul(f, a[col][j]));
                b[r][j] = csub(b[r][j], cmul(f, b[col][j]));
            }
        }
    }
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) a[i][j] = b[i][j];
    return true;
}

__global__ void __launch_bounds__(64) k_clover(double2 *__restrict__ F64, float4 *__restrict__ F32,
                                               const double2 *__restrict__ U, Geo g, double ck,
                                               int *status) {
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= g.V) return;
    int x[4];
    site_coords(g, n, x);
    double2 A[2][6][6];
    for (int ch = 0; ch < 2; ch++)
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) A[ch][i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    int plane = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, plane++) {
            double2 Q[9], u1[9], u2[9], u3[9], u4[9];
            for (int k = 0; k < 9; k++) Q[k] = make_double2(0, 0);
            // U_mu(n) U_nu(n+mu) U_mu(n+nu)^dag U_nu(n)^dag
            m3_load(U, g.V, n, mu, u1);
            m3_load(U, g.V, shifted(g, x, mu, 1, nu, 0), nu, u2);
            m3_load(U, g.V, shifted(g, x, mu, 0, nu, 1), mu, u3);
            m3_load(U, g.V, n, nu, u4);
            plaq_add(u1, false, u2, false, u3, true, u4, true, Q);
            // U_nu(n) U_mu(n+nu-mu)^dag U_nu(n-mu)^dag U_mu(n-mu)
            m3_load(U, g.V, n, nu, u1);
            m3_load(U, g.V, shifted(g, x, mu, -1, nu, 1), mu, u2);
            m3_load(U, g.V, shifted(g, x, mu, -1, nu, 0), nu, u3);
            m3_load(U, g.V, shifted(g, x, mu, -1, nu, 0), mu, u4);
            plaq_add(u1, false, u2, true, u3, true, u4, false, Q);
            // U_mu(n-mu)^dag U_nu(n-mu-nu)^dag U_mu(n-mu-nu) U_nu(n-nu)
            m3_load(U, g.V, shifted(g, x, mu, -1, nu, 0), mu, u1);
            m3_load(U, g.V, shifted(g, x, mu, -1, nu, -1), nu, u2);
            m3_load(U, g.V, shifted(g, x, mu, -1, nu, -1), mu, u3);
            m3_load(U, g.V, shifted(g, x, mu, 0, nu, -1), nu, u4);
            plaq_add(u1, true, u2, true, u3, false, u4, false, Q);
            // U_nu(n-nu)^dag U_mu(n-nu) U_nu(n+mu-nu) U_mu(n)^dag
            m3_load(U, g.V, shifted(g, x, mu, 0, nu, -1), nu, u1);
            m3_load(U, g.V, shifted(g, x, mu, 0, nu, -1), mu, u2);
            m3_load(U, g.V, shifted(g, x, mu, 1, nu, -1), nu, u3);
            m3_load(U, g.V, n, mu, u4);
            plaq_add(u1, true, u2, false, u3, false, u4, true, Q);
            // F_{mu nu} = (Q - Q^dag)/(8i): element (a,b) = (Q_ab - conj(Q_ba)) * (-i/8)
            double2 Fm[9];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    double2 d = make_double2(Q[a * 3 + b].x - Q[b * 3 + a].x, Q[a * 3 + b].y + Q[b * 3 + a].y);
                    Fm[a * 3 + b] = make_double2(d.y / 8.0, -d.x / 8.0);
                }
            // A_ch -= c_SW kappa sigma_ch (x) F_{mu nu}   (mu<nu covers the all-pairs sum with c/2)
            for (int ch = 0; ch < 2; ch++)
                for (int s = 0; s < 2; s++)
                    for (int t = 0; t < 2; t++) {
                        const double2 sg = c_sigma_chiral[plane][ch][s][t];
                        for (int a = 0; a < 3; a++)
                            for (int b = 0; b < 3; b++) {
                                double2 v = cmul(sg, Fm[a * 3 + b]);
                                A[ch][s * 3 + a][t * 3 + b].x -= ck * v.x;
                                A[ch][s * 3 + a][t * 3 + b].y -= ck * v.y;
                            }
                    }
        }
    bool ok = inv6(A[0]);
    ok = inv6(A[1]) && ok;
    if (!ok) atomicExch(status, 1);
    // pack F_ch / 2: 6 real diagonal entries, then the strictly lower triangle row by row
    double f[72];
    for (int ch = 0; ch < 2; ch++) {
        double *o = f + 36 * ch;
        for (int i = 0; i < 6; i++) o[i] = 0.5 * A[ch][i][i].x;
        int k = 6;
        for (int i = 1; i < 6; i++)
            for (int j = 0; j < i; j++) {
                // average with the conjugate transpose entry (Hermitian up to rounding)
                o[k] = 0.25 * (A[ch][i][j].x + A[ch][j][i].x);
                o[k + 1] = 0.25 * (A[ch][i][j].y - A[ch][j][i].y);
                k += 2;
            }
    }
    for (int k = 0; k < 36; k++) F64[k * g.V + n] = make_double2(f[2 * k], f[2 * k + 1]);
    for (int k = 0; k < 18; k++)
        F32[k * g.V + n] = make_float4((float)f[4 * k], (float)f[4 * k + 1], (float)f[4 * k + 2], (float)f[4 * k + 3]);
}

}  // namespace

int build_clover(qcd_ctx *c, double kappa, double csw) {
    static std::atomic<unsigned long long> tables_done{0};
    static std::mutex tables_mu;
    int trc = once_per_device(tables_done, tables_mu, c->device, [&]() -> int {
        double2 tab[6][2][2][2];
        bool ok = false;
        host_sigma_tables(tab, &ok);
        if (!ok) return fail(c, QCD_ERR_STATE, "internal: sigma_{mu nu} is not block diagonal in the chiral basis");
        QCD_CUDA(c, cudaMemcpyToSymbol(c_sigma_chiral, tab, sizeof(tab)));
        return QCD_OK;
    });
    if (trc) return trc;
    Geo g;
    for (int m = 0; m < 4; m++) g.L[m] = c->lat.L[m];
    g.V = c->lat.V;
    g.bc_t = c->bc_t;
    QCD_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    cudaEvent_t ev;
    prof_begin(c, QCD_K_OTHER, &ev);
    k_clover<<<(unsigned)((g.V + 63) / 64), 64, 0, c->stream>>>(c->F64, c->F32, c->U64, g, csw * kappa,
                                                                  c->d_status);
    int rc = prof_end(c, QCD_K_OTHER, ev);
    if (rc) return rc;
    int h = 0;
    QCD_CUDA(c, cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h) return fail(c, QCD_ERR_SINGULAR, "clover term: a chiral 6x6 block is singular");
    return QCD_OK;
}

}  // namespace qcd

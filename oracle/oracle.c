/*
 * Plain FP64 CPU oracle for the nested-BiCGStab / SAP / ll-SSOR solver of the
 * clover-preconditioned O(a)-improved Wilson-Dirac equation of
 *   T. Boku, K.-I. Ishikawa et al., "Multi-block/multi-core SSOR
 *   preconditioner for the QCD quark solver for K computer", Lattice 2012
 *   (arXiv:1210.7398).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares nothing
 * with the CUDA path.  It is written to be read against the paper: plain
 * loops, dense 4x4 spin and 3x3 colour matrices, no half-spinor tricks, no
 * chiral storage, no fusion.  OpenMP is used only across sites (operator
 * applications) or across SAP blocks of one colour, where the result does not
 * depend on the order.
 *
 * Conventions (the paper fixes only some of them; where it is silent the
 * reading taken is stated here or at the function that depends on it):
 *   site n = x + Lx*(y + Ly*(z + Lz*t)); mu = 0..3 is x,y,z,t (paper mu=1..4)
 *   links  U[n][mu][a][b]   spinor psi[n][spin][colour]   (complex, re/im)
 *   Dirac representation, gamma_4 diagonal (Sec. 3, "Dirac representation"):
 *     gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],  gamma_4 = diag(1,1,-1,-1)
 *   periodic boundaries; bc_t = -1 flips the sign of hops across the t edge.
 *
 * Every function states the passage of the paper it follows.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Gamma matrices (Dirac representation, gamma_4 diagonal; Sec. 3)           */
/* ------------------------------------------------------------------------ */

static cplx G[5][4][4]; /* gamma_1..gamma_4, gamma_5 = g1 g2 g3 g4 */
static cplx SIGMA[4][4][4][4]; /* sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] */
static int tables_ready = 0;

static void matmul4(cplx c[4][4], cplx a[4][4], cplx b[4][4])
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

static void init_tables(void)
{
    if (tables_ready) return;
    /* Pauli matrices */
    cplx pauli[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(G, 0, sizeof(G));
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                G[k][i][2 + j] = -I * pauli[k][i][j];
                G[k][2 + i][j] = I * pauli[k][i][j];
            }
    G[3][0][0] = 1; G[3][1][1] = 1; G[3][2][2] = -1; G[3][3][3] = -1;
    cplx t1[4][4], t2[4][4];
    matmul4(t1, G[0], G[1]);
    matmul4(t2, t1, G[2]);
    matmul4(G[4], t2, G[3]);
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++) {
            cplx a[4][4], b[4][4];
            matmul4(a, G[mu], G[nu]);
            matmul4(b, G[nu], G[mu]);
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) SIGMA[mu][nu][i][j] = 0.5 * I * (a[i][j] - b[i][j]);
        }
    tables_ready = 1;
}

/* gamma_{mu+1} for mu = 0..3, gamma_5 for mu = 4; out is 4x4 complex row-major */
int orc_gamma(int mu, double *out)
{
    init_tables();
    if (mu < 0 || mu > 4) return -1;
    cplx *o = (cplx *)out;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) o[i * 4 + j] = G[mu][i][j];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry                                                          */
/* ------------------------------------------------------------------------ */

static void coords(const int *L, long n, int x[4])
{
    x[0] = (int)(n % L[0]); n /= L[0];
    x[1] = (int)(n % L[1]); n /= L[1];
    x[2] = (int)(n % L[2]); n /= L[2];
    x[3] = (int)n;
}

static long index_of(const int *L, const int x[4])
{
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

static long volume(const int *L) { return (long)L[0] * L[1] * L[2] * L[3]; }

/* neighbour n + dir*mu (periodic) */
static long neighbour(const int *L, long n, int mu, int dir)
{
    int x[4];
    coords(L, n, x);
    x[mu] = (x[mu] + dir + L[mu]) % L[mu];
    return index_of(L, x);
}

/* boundary sign of the hop n -> n + dir*mu (bc_t = -1: antiperiodic in t) */
static double hop_sign(const int *L, long n, int mu, int dir, int bc_t)
{
    if (mu != 3 || bc_t == 1) return 1.0;
    int x[4];
    coords(L, n, x);
    if (dir > 0 && x[3] == L[3] - 1) return (double)bc_t;
    if (dir < 0 && x[3] == 0) return (double)bc_t;
    return 1.0;
}

static const cplx *link(const cplx *U, long n, int mu) { return U + (n * 4 + mu) * 9; }

/* ------------------------------------------------------------------------ */
/* One hop term of Eq. (2):                                                  */
/*   dir=+1: (1 - gamma_mu) U_mu(n)          psi(n + mu)                     */
/*   dir=-1: (1 + gamma_mu) U_mu(n - mu)^dag psi(n - mu)                     */
/* added (times sign) into acc[12].  Plain 4x4 spin x 3x3 colour products.   */
/* ------------------------------------------------------------------------ */
static void add_hop_term(cplx acc[12], const int *L, int bc_t, const cplx *U, long n, int mu,
                         int dir, const cplx *psi_m)
{
    long m = neighbour(L, n, mu, dir);
    double sgn = hop_sign(L, n, mu, dir, bc_t);
    const cplx *W = (dir > 0) ? link(U, n, mu) : link(U, m, mu);
    /* colour matrix C[a][c] = U_mu(n)[a][c] (fwd) or conj(U_mu(m)[c][a]) (bwd) */
    cplx C[3][3];
    for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) C[a][c] = (dir > 0) ? W[a * 3 + c] : conj(W[c * 3 + a]);
    /* spin matrix P = 1 - dir * gamma_mu */
    cplx P[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) P[i][j] = (i == j ? 1.0 : 0.0) - (double)dir * G[mu][i][j];
    const cplx *ps = psi_m + m * 12;
    for (int al = 0; al < 4; al++)
        for (int a = 0; a < 3; a++) {
            cplx s = 0;
            for (int be = 0; be < 4; be++)
                for (int c = 0; c < 3; c++) s += P[al][be] * C[a][c] * ps[be * 3 + c];
            acc[al * 3 + a] += sgn * s;
        }
}

/* (H psi)(n) = sum_mu [ fwd + bwd ]  (Eq. (2) without -kappa F) */
void orc_hop(const int *L, int bc_t, const double *Ud, const double *in, double *out)
{
    init_tables();
    const cplx *U = (const cplx *)Ud;
    const cplx *psi = (const cplx *)in;
    cplx *o = (cplx *)out;
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; n++) {
        cplx acc[12] = {0};
        for (int mu = 0; mu < 4; mu++) {
            add_hop_term(acc, L, bc_t, U, n, mu, +1, psi);
            add_hop_term(acc, L, bc_t, U, n, mu, -1, psi);
        }
        for (int k = 0; k < 12; k++) o[n * 12 + k] = acc[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Clover term (Eq. (2) text): F(n) = (1 - (c_SW kappa / 2) sigma_{mu nu}    */
/* F_{mu nu}(n))^{-1}, summed over all ordered pairs mu, nu.  F_{mu nu} is   */
/* the clover-leaf field strength (Q - Q^dag) / (8i), Q the sum of the four  */
/* plaquettes in the (mu,nu) plane that start and end at n, all with the     */
/* same orientation (mu first, then nu).                                     */
/* ------------------------------------------------------------------------ */

static void m3mul(cplx c[9], const cplx a[9], const cplx b[9])
{
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += a[i * 3 + k] * b[k * 3 + j];
            t[i * 3 + j] = s;
        }
    memcpy(c, t, sizeof(t));
}

static void m3dag(cplx c[9], const cplx a[9])
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c[i * 3 + j] = conj(a[j * 3 + i]);
}

/* site displaced by (dmu along mu, dnu along nu) */
static long shift2(const int *L, long n, int mu, int dmu, int nu, int dnu)
{
    int x[4];
    coords(L, n, x);
    x[mu] = (x[mu] + dmu + 2 * L[mu]) % L[mu];
    x[nu] = (x[nu] + dnu + 2 * L[nu]) % L[nu];
    return index_of(L, x);
}

/* product of four 3x3 matrices, each given as (link, daggered?) */
static void path4(cplx out[9], const cplx *a, int da, const cplx *b, int db, const cplx *c, int dc,
                  const cplx *d, int dd)
{
    cplx A[9], B[9], C[9], D[9];
    if (da) m3dag(A, a); else memcpy(A, a, sizeof(A));
    if (db) m3dag(B, b); else memcpy(B, b, sizeof(B));
    if (dc) m3dag(C, c); else memcpy(C, c, sizeof(C));
    if (dd) m3dag(D, d); else memcpy(D, d, sizeof(D));
    m3mul(out, A, B);
    m3mul(out, out, C);
    m3mul(out, out, D);
}

/* clover-leaf sum Q_{mu nu}(n) */
static void clover_leaf(cplx Q[9], const int *L, const cplx *U, long n, int mu, int nu)
{
    cplx P[9];
    for (int i = 0; i < 9; i++) Q[i] = 0;
    /* U_mu(n) U_nu(n+mu) U_mu(n+nu)^dag U_nu(n)^dag */
    path4(P, link(U, n, mu), 0, link(U, shift2(L, n, mu, 1, nu, 0), nu), 0,
          link(U, shift2(L, n, mu, 0, nu, 1), mu), 1, link(U, n, nu), 1);
    for (int i = 0; i < 9; i++) Q[i] += P[i];
    /* U_nu(n) U_mu(n+nu-mu)^dag U_nu(n-mu)^dag U_mu(n-mu) */
    path4(P, link(U, n, nu), 0, link(U, shift2(L, n, mu, -1, nu, 1), mu), 1,
          link(U, shift2(L, n, mu, -1, nu, 0), nu), 1, link(U, shift2(L, n, mu, -1, nu, 0), mu), 0);
    for (int i = 0; i < 9; i++) Q[i] += P[i];
    /* U_mu(n-mu)^dag U_nu(n-mu-nu)^dag U_mu(n-mu-nu) U_nu(n-nu) */
    path4(P, link(U, shift2(L, n, mu, -1, nu, 0), mu), 1, link(U, shift2(L, n, mu, -1, nu, -1), nu), 1,
          link(U, shift2(L, n, mu, -1, nu, -1), mu), 0, link(U, shift2(L, n, mu, 0, nu, -1), nu), 0);
    for (int i = 0; i < 9; i++) Q[i] += P[i];
    /* U_nu(n-nu)^dag U_mu(n-nu) U_nu(n+mu-nu) U_mu(n)^dag */
    path4(P, link(U, shift2(L, n, mu, 0, nu, -1), nu), 1, link(U, shift2(L, n, mu, 0, nu, -1), mu), 0,
          link(U, shift2(L, n, mu, 1, nu, -1), nu), 0, link(U, n, mu), 1);
    for (int i = 0; i < 9; i++) Q[i] += P[i];
}

/* In-place inverse of a 12x12 complex matrix by Gauss-Jordan elimination
 * with partial pivoting.  Returns 0, or -4 when a pivot is below 1e-300. */
static int invert12(cplx M[12][12])
{
    cplx A[12][24];
    for (int i = 0; i < 12; i++)
        for (int j = 0; j < 24; j++) A[i][j] = (j < 12) ? M[i][j] : (j - 12 == i ? 1.0 : 0.0);
    for (int col = 0; col < 12; col++) {
        int piv = col;
        for (int r = col + 1; r < 12; r++)
            if (cabs(A[r][col]) > cabs(A[piv][col])) piv = r;
        if (cabs(A[piv][col]) < 1e-300) return -4;
        if (piv != col)
            for (int j = 0; j < 24; j++) {
                cplx t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t;
            }
        cplx inv = 1.0 / A[col][col];
        for (int j = 0; j < 24; j++) A[col][j] *= inv;
        for (int r = 0; r < 12; r++) {
            if (r == col) continue;
            cplx f = A[r][col];
            if (f == 0) continue;
            for (int j = 0; j < 24; j++) A[r][j] -= f * A[col][j];
        }
    }
    for (int i = 0; i < 12; i++)
        for (int j = 0; j < 12; j++) M[i][j] = A[i][12 + j];
    return 0;
}

/* Builds, per site, A(n) = 1 - (c_SW kappa/2) sum_{mu,nu} sigma_{mu nu} (x) F_{mu nu}(n)
 * and F(n) = A(n)^{-1}; both dense 12x12 complex, index (spin*3 + colour).
 * A may be NULL.  Returns 0 or -4 (singular). */
int orc_clover(const int *L, const double *Ud, double csw, double kappa, double *Aout, double *Fout)
{
    init_tables();
    const cplx *U = (const cplx *)Ud;
    long V = volume(L);
    int status = 0;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; n++) {
        cplx A[12][12];
        for (int i = 0; i < 12; i++)
            for (int j = 0; j < 12; j++) A[i][j] = (i == j) ? 1.0 : 0.0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                if (mu == nu) continue;
                cplx Q[9], Qd[9], Fmn[9];
                clover_leaf(Q, L, U, n, mu, nu);
                m3dag(Qd, Q);
                for (int i = 0; i < 9; i++) Fmn[i] = (Q[i] - Qd[i]) / (8.0 * I);
                for (int al = 0; al < 4; al++)
                    for (int be = 0; be < 4; be++)
                        for (int a = 0; a < 3; a++)
                            for (int b = 0; b < 3; b++)
                                A[al * 3 + a][be * 3 + b] -=
                                    0.5 * csw * kappa * SIGMA[mu][nu][al][be] * Fmn[a * 3 + b];
            }
        if (Aout) memcpy((cplx *)Aout + n * 144, A, sizeof(A));
        if (invert12(A) != 0) {
#pragma omp atomic write
            status = -4;
        }
        memcpy((cplx *)Fout + n * 144, A, sizeof(A));
    }
    return status;
}

/* out(n) = M(n) v(n) for a field of dense 12x12 site matrices */
void orc_site_matrix(long V, const double *Md, const double *in, double *out)
{
    const cplx *M = (const cplx *)Md;
    const cplx *v = (const cplx *)in;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; n++) {
        cplx t[12];
        for (int i = 0; i < 12; i++) {
            cplx s = 0;
            for (int j = 0; j < 12; j++) s += M[n * 144 + i * 12 + j] * v[n * 12 + j];
            t[i] = s;
        }
        for (int i = 0; i < 12; i++) o[n * 12 + i] = t[i];
    }
}

/* ------------------------------------------------------------------------ */
/* D = 1 - kappa F H  (Eq. (2))                                              */
/* ------------------------------------------------------------------------ */
void orc_apply_D(const int *L, int bc_t, const double *U, const double *F, double kappa,
                 const double *in, double *out)
{
    long V = volume(L);
    double *h = malloc(sizeof(double) * 24 * V);
    double *fh = malloc(sizeof(double) * 24 * V);
    orc_hop(L, bc_t, U, in, h);
    orc_site_matrix(V, F, h, fh);
    for (long i = 0; i < 24 * V; i++) out[i] = in[i] - kappa * fh[i];
    free(h);
    free(fh);
}

/* M = A - kappa H, the clover Wilson operator before clover preconditioning
 * (D = A^{-1} M); used for the gamma_5-hermiticity check. */
void orc_apply_M(const int *L, int bc_t, const double *U, const double *A, double kappa,
                 const double *in, double *out)
{
    long V = volume(L);
    double *h = malloc(sizeof(double) * 24 * V);
    orc_hop(L, bc_t, U, in, h);
    orc_site_matrix(V, A, in, out);
    for (long i = 0; i < 24 * V; i++) out[i] -= kappa * h[i];
    free(h);
}

/* ------------------------------------------------------------------------ */
/* Block checkerboard (Eq. (3)): block coordinates floor(n_mu / b_mu),       */
/* colour = (sum of block coordinates) mod 2, colour 0 = E, 1 = O.           */
/* ------------------------------------------------------------------------ */

int orc_check_geometry(const int *L, const int *b, const int *s)
{
    for (int mu = 0; mu < 4; mu++) {
        if (b[mu] < 1 || L[mu] % b[mu] != 0) return -1;
        int nb = L[mu] / b[mu];
        if (nb < 2 || nb % 2 != 0) return -1;
        if (s && (s[mu] < 1 || b[mu] % s[mu] != 0)) return -1;
    }
    return 0;
}

static int site_colour(const int *L, const int *b, long n)
{
    int x[4];
    coords(L, n, x);
    int c = 0;
    for (int mu = 0; mu < 4; mu++) c += x[mu] / b[mu];
    return c & 1;
}

void orc_colours(const int *L, const int *b, int *colour)
{
    long V = volume(L);
    for (long n = 0; n < V; n++) colour[n] = site_colour(L, b, n);
}

/* P_row D P_col: the block of D of Eq. (3) mapping colour col_c to colour
 * row_c.  Entries of D between two different blocks of the same colour do not
 * exist (such blocks are never neighbours), so for row_c == col_c this is the
 * block-restricted operator D_EE or D_OO, and for row_c != col_c it is the
 * hopping part D_OE or D_EO.  Sites of the other row colour are set to 0. */
void orc_apply_D_colour(const int *L, int bc_t, const int *b, const double *Ud, const double *Fd,
                        double kappa, int row_c, int col_c, const double *in, double *out)
{
    init_tables();
    const cplx *U = (const cplx *)Ud;
    const cplx *F = (const cplx *)Fd;
    long V = volume(L);
    cplx *masked = malloc(sizeof(cplx) * 12 * V);
    const cplx *psi = (const cplx *)in;
    for (long n = 0; n < V; n++)
        for (int k = 0; k < 12; k++) masked[n * 12 + k] = (site_colour(L, b, n) == col_c) ? psi[n * 12 + k] : 0;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; n++) {
        if (site_colour(L, b, n) != row_c) {
            for (int k = 0; k < 12; k++) o[n * 12 + k] = 0;
            continue;
        }
        cplx acc[12] = {0};
        for (int mu = 0; mu < 4; mu++) {
            add_hop_term(acc, L, bc_t, U, n, mu, +1, masked);
            add_hop_term(acc, L, bc_t, U, n, mu, -1, masked);
        }
        for (int i = 0; i < 12; i++) {
            cplx s = 0;
            for (int j = 0; j < 12; j++) s += F[n * 144 + i * 12 + j] * acc[j];
            o[n * 12 + i] = masked[n * 12 + i] - kappa * s;
        }
    }
    free(masked);
}

/* ------------------------------------------------------------------------ */
/* Locally-lexicographic ordering (Sec. 3, "Inverse of block operator";     */
/* Eicker et al. / Fischer et al.).  Inside a block with local coordinates  */
/* y_mu in [0, b_mu): sub-block q_mu = y_mu / s_mu, local position           */
/* l_mu = y_mu % s_mu.  lambda = lexicographic index of l inside a           */
/* sub-block, sigma = lexicographic index of q among the sub-blocks; the    */
/* order key is lambda * N_sb + sigma, N_sb = prod(b_mu / s_mu).             */
/* order[k] = block-local lexicographic index of the site with key k.       */
/* ------------------------------------------------------------------------ */
int orc_ll_order(const int *b, const int *s, int *order)
{
    int nq[4];
    for (int mu = 0; mu < 4; mu++) {
        if (s[mu] < 1 || b[mu] % s[mu] != 0) return -1;
        nq[mu] = b[mu] / s[mu];
    }
    int nsb = nq[0] * nq[1] * nq[2] * nq[3];
    int vol = b[0] * b[1] * b[2] * b[3];
    for (int yl = 0; yl < vol; yl++) {
        int y[4], r = yl;
        for (int mu = 0; mu < 4; mu++) { y[mu] = r % b[mu]; r /= b[mu]; }
        int l[4], q[4];
        for (int mu = 0; mu < 4; mu++) { l[mu] = y[mu] % s[mu]; q[mu] = y[mu] / s[mu]; }
        int lambda = l[0] + s[0] * (l[1] + s[1] * (l[2] + s[2] * l[3]));
        int sigma = q[0] + nq[0] * (q[1] + nq[1] * (q[2] + nq[2] * q[3]));
        order[lambda * nsb + sigma] = yl;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* SSOR approximate block inverse A_BB (Sec. 3): stationary SSOR on          */
/* D_BB x = f from x = 0.  One sweep = a forward pass over the block's sites */
/* in ll order, then a backward pass in reverse order.  Each visit sets      */
/*   x_i <- (1-omega) x_i + omega [ f_i + kappa F(i) sum_{j in B} h_ij x_j ] */
/* with the current x (D_BB = 1 - kappa F H_BB has unit site diagonal, so no */
/* diagonal solve is needed).  Applied to every block of colour c; sites of  */
/* the other colour in x are left untouched.                                 */
/* ------------------------------------------------------------------------ */

static void ssor_site_update(cplx *x, const cplx *f, const int *L, int bc_t, const int *b,
                             const cplx *U, const cplx *F, double kappa, double omega, long n)
{
    int xn[4];
    coords(L, n, xn);
    cplx acc[12] = {0};
    for (int mu = 0; mu < 4; mu++) {
        int ymu = xn[mu] % b[mu];
        if (ymu + 1 < b[mu]) add_hop_term(acc, L, bc_t, U, n, mu, +1, x);
        if (ymu - 1 >= 0) add_hop_term(acc, L, bc_t, U, n, mu, -1, x);
    }
    for (int i = 0; i < 12; i++) {
        cplx s = 0;
        for (int j = 0; j < 12; j++) s += F[n * 144 + i * 12 + j] * acc[j];
        x[n * 12 + i] = (1.0 - omega) * x[n * 12 + i] + omega * (f[n * 12 + i] + kappa * s);
    }
}

int orc_ssor(const int *L, int bc_t, const double *Ud, const double *Fd, double kappa, const int *b,
             const int *s, double omega, int nsweep, int colour, const double *fd, double *xd)
{
    init_tables();
    if (orc_check_geometry(L, b, s) != 0) return -1;
    const cplx *U = (const cplx *)Ud;
    const cplx *F = (const cplx *)Fd;
    const cplx *f = (const cplx *)fd;
    cplx *x = (cplx *)xd;
    int vol = b[0] * b[1] * b[2] * b[3];
    int *order = malloc(sizeof(int) * vol);
    orc_ll_order(b, s, order);
    int nb[4];
    for (int mu = 0; mu < 4; mu++) nb[mu] = L[mu] / b[mu];
    long nblocks = (long)nb[0] * nb[1] * nb[2] * nb[3];
#pragma omp parallel for schedule(dynamic)
    for (long B = 0; B < nblocks; B++) {
        int Bc[4];
        long r = B;
        for (int mu = 0; mu < 4; mu++) { Bc[mu] = (int)(r % nb[mu]); r /= nb[mu]; }
        if (((Bc[0] + Bc[1] + Bc[2] + Bc[3]) & 1) != colour) continue;
        /* global site indices of the block, in ll order */
        long *sites = malloc(sizeof(long) * vol);
        for (int k = 0; k < vol; k++) {
            int yl = order[k], y[4], xg[4];
            for (int mu = 0; mu < 4; mu++) { y[mu] = yl % b[mu]; yl /= b[mu]; }
            for (int mu = 0; mu < 4; mu++) xg[mu] = Bc[mu] * b[mu] + y[mu];
            sites[k] = index_of(L, xg);
        }
        for (int k = 0; k < vol; k++)
            for (int i = 0; i < 12; i++) x[sites[k] * 12 + i] = 0;
        for (int sw = 0; sw < nsweep; sw++) {
            for (int k = 0; k < vol; k++) ssor_site_update(x, f, L, bc_t, b, U, F, kappa, omega, sites[k]);
            for (int k = vol - 1; k >= 0; k--) ssor_site_update(x, f, L, bc_t, b, U, F, kappa, omega, sites[k]);
        }
        free(sites);
    }
    free(order);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Even-odd alternative to the SSOR block inverse.  Sec. 3 names the even-   */
/* odd site preconditioning of Luescher's SAP as the block solver that the   */
/* ll-SSOR outperforms at equal cost, without formulas; this is the standard */
/* construction.  Site parity p(n) = (n_0 + n_1 + n_2 + n_3) mod 2.  H_BB    */
/* only links sites of opposite parity, so D_BB x = f reads                  */
/*   x_e - kappa F_e H_eo x_o = f_e,   x_o - kappa F_o H_oe x_e = f_o,       */
/* and eliminating x_o leaves the Schur complement on the even sites         */
/*   Dhat x_e = fhat,  Dhat = 1 - kappa^2 F_e H_eo F_o H_oe,                 */
/*   fhat = f_e + kappa F_e H_eo f_o.                                        */
/* nmr minimal-residual steps from x_e = 0: r = fhat; per step p = Dhat r,   */
/* alpha = <p, r> / <p, p>, x_e += alpha r, r -= alpha p; then               */
/* x_o = f_o + kappa F_o H_oe x_e.  Applied to every block of colour c;      */
/* sites of the other colour in x are left untouched.                        */
/* ------------------------------------------------------------------------ */

/* out = F(n) sum over the in-block neighbours j of n of h_nj src_j */
static void block_FH(const int *L, int bc_t, const int *b, const cplx *U, const cplx *F, const cplx *src,
                     long n, cplx out[12])
{
    int xn[4];
    coords(L, n, xn);
    cplx acc[12] = {0};
    for (int mu = 0; mu < 4; mu++) {
        int ymu = xn[mu] % b[mu];
        if (ymu + 1 < b[mu]) add_hop_term(acc, L, bc_t, U, n, mu, +1, src);
        if (ymu - 1 >= 0) add_hop_term(acc, L, bc_t, U, n, mu, -1, src);
    }
    for (int i = 0; i < 12; i++) {
        cplx s = 0;
        for (int j = 0; j < 12; j++) s += F[n * 144 + i * 12 + j] * acc[j];
        out[i] = s;
    }
}

int orc_eo_mr(const int *L, int bc_t, const double *Ud, const double *Fd, double kappa, const int *b,
              int nmr, int colour, const double *fd, double *xd)
{
    init_tables();
    if (orc_check_geometry(L, b, NULL) != 0 || nmr < 1) return -1;
    const cplx *U = (const cplx *)Ud;
    const cplx *F = (const cplx *)Fd;
    const cplx *f = (const cplx *)fd;
    cplx *x = (cplx *)xd;
    long V = volume(L);
    /* lattice-sized scratch; every block reads and writes only its own sites */
    cplx *res = calloc(12 * V, sizeof(cplx)), *tod = calloc(12 * V, sizeof(cplx)), *pev = calloc(12 * V, sizeof(cplx));
    int vol = b[0] * b[1] * b[2] * b[3];
    int nb[4];
    for (int mu = 0; mu < 4; mu++) nb[mu] = L[mu] / b[mu];
    long nblocks = (long)nb[0] * nb[1] * nb[2] * nb[3];
#pragma omp parallel for schedule(dynamic)
    for (long B = 0; B < nblocks; B++) {
        int Bc[4];
        long rr = B;
        for (int mu = 0; mu < 4; mu++) { Bc[mu] = (int)(rr % nb[mu]); rr /= nb[mu]; }
        if (((Bc[0] + Bc[1] + Bc[2] + Bc[3]) & 1) != colour) continue;
        long *ev = malloc(sizeof(long) * vol), *od = malloc(sizeof(long) * vol);
        int ne = 0, no = 0;
        for (int yl = 0; yl < vol; yl++) {
            int y[4], xg[4], q = yl;
            for (int mu = 0; mu < 4; mu++) { y[mu] = q % b[mu]; q /= b[mu]; }
            for (int mu = 0; mu < 4; mu++) xg[mu] = Bc[mu] * b[mu] + y[mu];
            long n = index_of(L, xg);
            if ((xg[0] + xg[1] + xg[2] + xg[3]) & 1) od[no++] = n;
            else ev[ne++] = n;
        }
        cplx h[12];
        /* r = fhat on the even sites, x_e = 0 */
        for (int k = 0; k < ne; k++) {
            long n = ev[k];
            block_FH(L, bc_t, b, U, F, f, n, h);
            for (int i = 0; i < 12; i++) {
                res[n * 12 + i] = f[n * 12 + i] + kappa * h[i];
                x[n * 12 + i] = 0;
            }
        }
        for (int it = 0; it < nmr; it++) {
            /* p = Dhat r through t_o = F_o H_oe r */
            for (int k = 0; k < no; k++) {
                long m = od[k];
                block_FH(L, bc_t, b, U, F, res, m, h);
                for (int i = 0; i < 12; i++) tod[m * 12 + i] = h[i];
            }
            cplx pr = 0;
            double pp = 0;
            for (int k = 0; k < ne; k++) {
                long n = ev[k];
                block_FH(L, bc_t, b, U, F, tod, n, h);
                for (int i = 0; i < 12; i++) {
                    cplx pv = res[n * 12 + i] - kappa * kappa * h[i];
                    pev[n * 12 + i] = pv;
                    pr += conj(pv) * res[n * 12 + i];
                    pp += creal(conj(pv) * pv);
                }
            }
            cplx alpha = pp > 0 ? pr / pp : 0;
            for (int k = 0; k < ne; k++) {
                long n = ev[k];
                for (int i = 0; i < 12; i++) {
                    x[n * 12 + i] += alpha * res[n * 12 + i];
                    res[n * 12 + i] -= alpha * pev[n * 12 + i];
                }
            }
        }
        /* x_o = f_o + kappa F_o H_oe x_e */
        for (int k = 0; k < no; k++) {
            long m = od[k];
            block_FH(L, bc_t, b, U, F, x, m, h);
            for (int i = 0; i < 12; i++) x[m * 12 + i] = f[m * 12 + i] + kappa * h[i];
        }
        free(ev);
        free(od);
    }
    free(res);
    free(tod);
    free(pev);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* SAP (Eq. (4), Alg. 1).  One application of K together with w = D K v:    */
/*   x_E = A_EE v_E;  w_O = D_OE x_E;  w_E = D_EE x_E;  f_O = v_O - w_O;     */
/*   x_O = A_OO f_O;  f_E = D_EO x_O;  f_O = D_OO x_O;  w_O += f_O;          */
/*   w_E += f_E.                                                             */
/* M_SAP = K sum_{j<N_SAP} (1 - DK)^j by the recurrence x = 0, r = v;        */
/* N_SAP times: y = K r, x += y, r -= D y.                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    const int *L; int bc_t;
    const double *U, *F; double kappa;
    const int *b, *s; double omega; int nsweep; int nsap;
    int solver; /* block inverse: 0 ll-SSOR (nsweep sweeps), 1 even-odd MR (nsweep steps) */
} sap_cfg;

static void block_inverse(const sap_cfg *c, int colour, const double *f, double *x)
{
    if (c->solver == 1) orc_eo_mr(c->L, c->bc_t, c->U, c->F, c->kappa, c->b, c->nsweep, colour, f, x);
    else orc_ssor(c->L, c->bc_t, c->U, c->F, c->kappa, c->b, c->s, c->omega, c->nsweep, colour, f, x);
}

/* y = K v and w = D K v following Alg. 1 */
static void sap_DK(const sap_cfg *c, const double *v, double *y, double *w)
{
    long V = volume(c->L);
    size_t bytes = sizeof(double) * 24 * V;
    double *xE = calloc(24 * V, sizeof(double));
    double *xO = calloc(24 * V, sizeof(double));
    double *wO = malloc(bytes), *wE = malloc(bytes), *fO = malloc(bytes), *fE = malloc(bytes);
    int *col = malloc(sizeof(int) * V);
    orc_colours(c->L, c->b, col);
    /* x_E = A_EE v_E */
    block_inverse(c, 0, v, xE);
    /* w_O = D_OE x_E ; w_E = D_EE x_E */
    orc_apply_D_colour(c->L, c->bc_t, c->b, c->U, c->F, c->kappa, 1, 0, xE, wO);
    orc_apply_D_colour(c->L, c->bc_t, c->b, c->U, c->F, c->kappa, 0, 0, xE, wE);
    /* f_O = v_O - w_O */
    for (long n = 0; n < V; n++)
        for (int k = 0; k < 24; k++) fO[n * 24 + k] = (col[n] == 1) ? v[n * 24 + k] - wO[n * 24 + k] : 0.0;
    /* x_O = A_OO f_O */
    block_inverse(c, 1, fO, xO);
    /* f_E = D_EO x_O ; f_O = D_OO x_O */
    orc_apply_D_colour(c->L, c->bc_t, c->b, c->U, c->F, c->kappa, 0, 1, xO, fE);
    orc_apply_D_colour(c->L, c->bc_t, c->b, c->U, c->F, c->kappa, 1, 1, xO, fO);
    for (long n = 0; n < V; n++)
        for (int k = 0; k < 24; k++) {
            long i = n * 24 + k;
            if (col[n] == 0) {
                y[i] = xE[i];
                w[i] = wE[i] + fE[i]; /* w_E = w_E + f_E */
            } else {
                y[i] = xO[i];
                w[i] = wO[i] + fO[i]; /* w_O = w_O + f_O */
            }
        }
    free(xE); free(xO); free(wO); free(wE); free(fO); free(fE); free(col);
}

/* out = M_SAP v with the block inverse `solver` (0 ll-SSOR, 1 even-odd MR) */
int orc_sap_bs(const int *L, int bc_t, const double *U, const double *F, double kappa, const int *b,
               const int *s, double omega, int nsweep, int nsap, int solver, const double *v, double *out)
{
    if (orc_check_geometry(L, b, s) != 0 || nsweep < 1 || nsap < 1 || solver < 0 || solver > 1) return -1;
    sap_cfg c = {L, bc_t, U, F, kappa, b, s, omega, nsweep, nsap, solver};
    long N = 24 * volume(L);
    double *r = malloc(sizeof(double) * N), *y = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N);
    memcpy(r, v, sizeof(double) * N);
    for (long i = 0; i < N; i++) out[i] = 0;
    for (int j = 0; j < nsap; j++) {
        sap_DK(&c, r, y, w);
        for (long i = 0; i < N; i++) {
            out[i] += y[i];
            r[i] -= w[i];
        }
    }
    free(r); free(y); free(w);
    return 0;
}

/* out = M_SAP v (ll-SSOR block inverses) */
int orc_sap(const int *L, int bc_t, const double *U, const double *F, double kappa, const int *b,
            const int *s, double omega, int nsweep, int nsap, const double *v, double *out)
{
    return orc_sap_bs(L, bc_t, U, F, kappa, b, s, omega, nsweep, nsap, 0, v, out);
}

/* ------------------------------------------------------------------------ */
/* BiCGStab (Sec. 2): inner solver right-preconditioned by M_SAP, and the    */
/* outer flexible BiCGStab whose preconditioner is the inner solve.          */
/* ------------------------------------------------------------------------ */

static cplx dot(long N, const cplx *a, const cplx *b) /* sum conj(a) b */
{
    cplx s = 0;
    for (long i = 0; i < N; i++) s += conj(a[i]) * b[i];
    return s;
}

static double norm2(long N, const cplx *a) { return sqrt(creal(dot(N, a, a))); }

static int finite_c(cplx z) { return isfinite(creal(z)) && isfinite(cimag(z)); }

/* Solve D y = q approximately: stop when ||r|| <= tol ||q|| or after maxit
 * iterations or on breakdown; returns the number of iterations done. */
int orc_inner_bicgstab(const int *L, int bc_t, const double *U, const double *F, double kappa,
                       const int *b, const int *s, double omega, int nsweep, int nsap, double tol,
                       int maxit, const double *qd, double *yd)
{
    long V = volume(L), N = 12 * V;
    const cplx *q = (const cplx *)qd;
    cplx *y = (cplx *)yd;
    cplx *r = malloc(sizeof(cplx) * N), *rh = malloc(sizeof(cplx) * N), *p = calloc(N, sizeof(cplx));
    cplx *v = calloc(N, sizeof(cplx)), *pt = malloc(sizeof(cplx) * N), *st = malloc(sizeof(cplx) * N);
    cplx *sv = malloc(sizeof(cplx) * N), *t = malloc(sizeof(cplx) * N);
    for (long i = 0; i < N; i++) { y[i] = 0; r[i] = q[i]; rh[i] = q[i]; }
    cplx rho0 = 1, alpha = 1, om = 1;
    double qn = norm2(N, q);
    int it = 0;
    if (qn == 0) goto done;
    for (it = 0; it < maxit;) {
        cplx rho = dot(N, rh, r);
        if (!finite_c(rho) || cabs(rho) < 1e-30 * norm2(N, rh) * norm2(N, r)) break;
        cplx beta = (rho / rho0) * (alpha / om);
        for (long i = 0; i < N; i++) p[i] = r[i] + beta * (p[i] - om * v[i]);
        orc_sap(L, bc_t, U, F, kappa, b, s, omega, nsweep, nsap, (double *)p, (double *)pt);
        orc_apply_D(L, bc_t, U, F, kappa, (double *)pt, (double *)v);
        cplx rv = dot(N, rh, v);
        if (!finite_c(rv) || cabs(rv) < 1e-30 * norm2(N, rh) * norm2(N, v)) break;
        alpha = rho / rv;
        for (long i = 0; i < N; i++) sv[i] = r[i] - alpha * v[i];
        orc_sap(L, bc_t, U, F, kappa, b, s, omega, nsweep, nsap, (double *)sv, (double *)st);
        orc_apply_D(L, bc_t, U, F, kappa, (double *)st, (double *)t);
        double tt = creal(dot(N, t, t));
        om = (tt > 0) ? dot(N, t, sv) / tt : 0;
        for (long i = 0; i < N; i++) {
            y[i] += alpha * pt[i] + om * st[i];
            r[i] = sv[i] - om * t[i];
        }
        rho0 = rho;
        it++;
        if (norm2(N, r) <= tol * qn) break;
        if (om == 0 || !finite_c(om)) break;
    }
done:
    free(r); free(rh); free(p); free(v); free(pt); free(st); free(sv); free(t);
    return it;
}

/* Outer flexible FP64 BiCGStab for D x = b.  x holds the initial guess on
 * entry.  stats[0..3] = outer iterations, inner iterations, restarts, true
 * relative residual.  Returns 0, -5 (not converged) or -6 (breakdown). */
int orc_solve(const int *L, int bc_t, const double *U, const double *F, double kappa,
              const int *b, const int *s, double omega, int nsweep, int nsap, double tol,
              double inner_tol, int max_outer, int max_inner, const double *bd, double *xd,
              double *stats)
{
    long V = volume(L), N = 12 * V;
    const cplx *bb = (const cplx *)bd;
    cplx *x = (cplx *)xd;
    cplx *r = malloc(sizeof(cplx) * N), *rh = malloc(sizeof(cplx) * N), *p = calloc(N, sizeof(cplx));
    cplx *v = calloc(N, sizeof(cplx)), *ph = malloc(sizeof(cplx) * N), *sh = malloc(sizeof(cplx) * N);
    cplx *sv = malloc(sizeof(cplx) * N), *t = malloc(sizeof(cplx) * N), *tmp = malloc(sizeof(cplx) * N);
    double bn = norm2(N, bb);
    int outer = 0, inner = 0, restarts = 0, status = -5;
    double relres = 0;
    orc_apply_D(L, bc_t, U, F, kappa, (double *)x, (double *)tmp);
    for (long i = 0; i < N; i++) { r[i] = bb[i] - tmp[i]; rh[i] = r[i]; p[i] = 0; v[i] = 0; }
    cplx rho0 = 1, alpha = 1, om = 1;
    if (bn == 0) { status = 0; goto done; }
    if (norm2(N, r) <= tol * bn) { status = 0; relres = norm2(N, r) / bn; goto done; }
    while (outer < max_outer) {
        int breakdown = 0;
        cplx rho = dot(N, rh, r);
        if (!finite_c(rho) || cabs(rho) < 1e-30 * norm2(N, rh) * norm2(N, r)) breakdown = 1;
        if (!breakdown) {
            cplx beta = (rho / rho0) * (alpha / om);
            for (long i = 0; i < N; i++) p[i] = r[i] + beta * (p[i] - om * v[i]);
            inner += orc_inner_bicgstab(L, bc_t, U, F, kappa, b, s, omega, nsweep, nsap, inner_tol,
                                        max_inner, (double *)p, (double *)ph);
            orc_apply_D(L, bc_t, U, F, kappa, (double *)ph, (double *)v);
            cplx rv = dot(N, rh, v);
            if (!finite_c(rv) || cabs(rv) < 1e-30 * norm2(N, rh) * norm2(N, v)) breakdown = 1;
            else {
                alpha = rho / rv;
                for (long i = 0; i < N; i++) sv[i] = r[i] - alpha * v[i];
                inner += orc_inner_bicgstab(L, bc_t, U, F, kappa, b, s, omega, nsweep, nsap, inner_tol,
                                            max_inner, (double *)sv, (double *)sh);
                orc_apply_D(L, bc_t, U, F, kappa, (double *)sh, (double *)t);
                double tt = creal(dot(N, t, t));
                om = (tt > 0) ? dot(N, t, sv) / tt : 0;
                for (long i = 0; i < N; i++) {
                    x[i] += alpha * ph[i] + om * sh[i];
                    r[i] = sv[i] - om * t[i];
                }
                rho0 = rho;
                outer++;
                if (om == 0 || !finite_c(om)) breakdown = 1;
            }
        }
        double rn = norm2(N, r);
        if (breakdown || rn <= tol * bn) {
            /* true residual in FP64 */
            orc_apply_D(L, bc_t, U, F, kappa, (double *)x, (double *)tmp);
            for (long i = 0; i < N; i++) r[i] = bb[i] - tmp[i];
            relres = norm2(N, r) / bn;
            if (relres <= tol) { status = 0; break; }
            if (breakdown && ++restarts > 5) { status = -6; break; }
            if (!breakdown) restarts++;
            for (long i = 0; i < N; i++) { rh[i] = r[i]; p[i] = 0; v[i] = 0; }
            rho0 = alpha = om = 1;
        }
    }
    if (status != 0) {
        orc_apply_D(L, bc_t, U, F, kappa, (double *)x, (double *)tmp);
        for (long i = 0; i < N; i++) tmp[i] = bb[i] - tmp[i];
        relres = norm2(N, tmp) / bn;
    }
done:
    if (stats) {
        stats[0] = outer; stats[1] = inner; stats[2] = restarts; stats[3] = relres;
    }
    free(r); free(rh); free(p); free(v); free(ph); free(sh); free(sv); free(t); free(tmp);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Learned correction (a project addition; the paper has none).  A linear,  */
/* gauge-covariant network of parallel-transport layers                     */
/*   y_c(n) = sum_{d=0..8} sum_{c'} W_d[c][c'] (T_d x_{c'})(n)               */
/* with 4x4 complex spin matrices W_d[c][c'] and transports                 */
/*   T_0 = 1,  T_{2mu} x(n) = U_mu(n) x(n+mu),                               */
/*   T_{2mu+1} x(n) = U_mu(n-mu)^dag x(n-mu)   (boundary sign as in D).       */
/* Weights of a layer: complex [9][cout][cin][4][4]; fields [c][V][4][3].     */
/* ------------------------------------------------------------------------ */

/* z = T_d x for one site n (x: one channel [V][12]) */
static void transport_site(const int *L, int bc_t, const cplx *U, int d, long n, const cplx *x, cplx z[12])
{
    if (d == 0) {
        for (int k = 0; k < 12; k++) z[k] = x[n * 12 + k];
        return;
    }
    int mu = (d - 1) / 2, dir = ((d - 1) % 2 == 0) ? +1 : -1;
    long m = neighbour(L, n, mu, dir);
    double sgn = hop_sign(L, n, mu, dir, bc_t);
    const cplx *W = (dir > 0) ? link(U, n, mu) : link(U, m, mu);
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            cplx acc = 0;
            for (int b = 0; b < 3; b++) acc += ((dir > 0) ? W[a * 3 + b] : conj(W[b * 3 + a])) * x[m * 12 + s * 3 + b];
            z[s * 3 + a] = sgn * acc;
        }
}

/* adjoint transport z = T_d^dag x at site m:
 * T_{2mu}^dag x(m) = U_mu(m-mu)^dag x(m-mu),  T_{2mu+1}^dag x(m) = U_mu(m) x(m+mu) */
static void transport_adj_site(const int *L, int bc_t, const cplx *U, int d, long m, const cplx *x, cplx z[12])
{
    if (d == 0) {
        for (int k = 0; k < 12; k++) z[k] = x[m * 12 + k];
        return;
    }
    int mu = (d - 1) / 2, dir = ((d - 1) % 2 == 0) ? -1 : +1; /* the opposite hop */
    long n = neighbour(L, m, mu, dir);
    double sgn = hop_sign(L, m, mu, dir, bc_t);
    const cplx *W = (dir > 0) ? link(U, m, mu) : link(U, n, mu);
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            cplx acc = 0;
            for (int b = 0; b < 3; b++) acc += ((dir > 0) ? W[a * 3 + b] : conj(W[b * 3 + a])) * x[n * 12 + s * 3 + b];
            z[s * 3 + a] = sgn * acc;
        }
}

/* one layer: y = sum_d W_d T_d x */
void orc_learned_layer(const int *L, int bc_t, const double *Ud, int cin, int cout, const double *Wd,
                       const double *xd, double *yd)
{
    const cplx *U = (const cplx *)Ud, *W = (const cplx *)Wd, *x = (const cplx *)xd;
    cplx *y = (cplx *)yd;
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; n++) {
        cplx out[64][12];
        for (int c = 0; c < cout; c++)
            for (int k = 0; k < 12; k++) out[c][k] = 0;
        for (int d = 0; d < 9; d++)
            for (int cp = 0; cp < cin; cp++) {
                cplx z[12];
                transport_site(L, bc_t, U, d, n, x + (long)cp * V * 12, z);
                for (int c = 0; c < cout; c++) {
                    const cplx *w = W + (((long)d * cout + c) * cin + cp) * 16;
                    for (int al = 0; al < 4; al++)
                        for (int be = 0; be < 4; be++)
                            for (int a = 0; a < 3; a++) out[c][al * 3 + a] += w[al * 4 + be] * z[be * 3 + a];
                }
            }
        for (int c = 0; c < cout; c++)
            for (int k = 0; k < 12; k++) y[((long)c * V + n) * 12 + k] = out[c][k];
    }
}

/* whole network: chans[0..nl] channel counts, weights concatenated layer by layer */
static long layer_wsize(int cin, int cout) { return 9L * cout * cin * 16; }

void orc_learned_forward(const int *L, int bc_t, const double *U, int nl, const int *chans, const double *W,
                         const double *x, double *y)
{
    long V = volume(L);
    const double *in = x;
    double *buf[2] = {malloc(sizeof(double) * 24 * V * 64), malloc(sizeof(double) * 24 * V * 64)};
    long woff = 0;
    for (int l = 0; l < nl; l++) {
        double *out = (l == nl - 1) ? y : buf[l % 2];
        orc_learned_layer(L, bc_t, U, chans[l], chans[l + 1], W + 2 * woff, in, out);
        woff += layer_wsize(chans[l], chans[l + 1]);
        in = out;
    }
    free(buf[0]);
    free(buf[1]);
}

/* Loss L = |N(rho) - eps|^2 / |eps|^2 for one pair, and its gradient with
 * respect to the real and imaginary parts of every weight:
 * grad = 2 (Re, Im) of dL/dW*, dL/dW_d[c][c'] = sum_n g_c(n) (T_d a_{c'}(n))^dag
 * with g = dL/dy* propagated back by the adjoint layers. */
double orc_learned_loss_grad(const int *L, int bc_t, const double *Ud, int nl, const int *chans,
                             const double *Wd, const double *rhod, const double *epsd, double *grad)
{
    const cplx *U = (const cplx *)Ud, *W = (const cplx *)Wd;
    long V = volume(L);
    /* activations a[0] = rho, a[l+1] = layer l output */
    cplx *a[16];
    a[0] = (cplx *)rhod;
    long woffs[16];
    long woff = 0;
    for (int l = 0; l < nl; l++) {
        woffs[l] = woff;
        a[l + 1] = malloc(sizeof(cplx) * 12 * V * chans[l + 1]);
        orc_learned_layer(L, bc_t, Ud, chans[l], chans[l + 1], Wd + 2 * woff, (double *)a[l], (double *)a[l + 1]);
        woff += layer_wsize(chans[l], chans[l + 1]);
    }
    const cplx *eps = (const cplx *)epsd;
    double en2 = 0, loss = 0;
    for (long i = 0; i < 12 * V; i++) en2 += creal(eps[i] * conj(eps[i]));
    cplx *g = malloc(sizeof(cplx) * 12 * V * chans[nl]);
    for (long i = 0; i < 12 * V; i++) {
        cplx r = a[nl][i] - eps[i];
        loss += creal(r * conj(r)) / en2;
        g[i] = r / en2;
    }
    cplx *gW = (cplx *)grad; /* written as complex, converted to 2 (Re, Im) at the end */
    for (long i = 0; i < woff; i++) gW[i] = 0;
    for (int l = nl - 1; l >= 0; l--) {
        int cin = chans[l], cout = chans[l + 1];
        const cplx *x = a[l];
        /* weight gradient */
        for (int d = 0; d < 9; d++)
            for (int cp = 0; cp < cin; cp++) {
                cplx acc[64][16];
                for (int c = 0; c < cout; c++)
                    for (int k = 0; k < 16; k++) acc[c][k] = 0;
                for (long n = 0; n < V; n++) {
                    cplx z[12];
                    transport_site(L, bc_t, U, d, n, x + (long)cp * V * 12, z);
                    for (int c = 0; c < cout; c++)
                        for (int al = 0; al < 4; al++)
                            for (int be = 0; be < 4; be++)
                                for (int aa = 0; aa < 3; aa++)
                                    acc[c][al * 4 + be] += g[((long)c * V + n) * 12 + al * 3 + aa] * conj(z[be * 3 + aa]);
                }
                for (int c = 0; c < cout; c++)
                    for (int k = 0; k < 16; k++) gW[woffs[l] + (((long)d * cout + c) * cin + cp) * 16 + k] = acc[c][k];
            }
        if (l == 0) break;
        /* g_prev(c') = sum_d T_d^dag sum_c W_d[c][c']^dag g_c */
        cplx *gp = malloc(sizeof(cplx) * 12 * V * cin);
        cplx *h = malloc(sizeof(cplx) * 12 * V);
        for (int cp = 0; cp < cin; cp++) {
            for (long i = 0; i < 12 * V; i++) gp[(long)cp * V * 12 + i] = 0;
            for (int d = 0; d < 9; d++) {
                for (long n = 0; n < V; n++)
                    for (int be = 0; be < 4; be++)
                        for (int aa = 0; aa < 3; aa++) {
                            cplx s = 0;
                            for (int c = 0; c < cout; c++) {
                                const cplx *w = W + woffs[l] + (((long)d * cout + c) * cin + cp) * 16;
                                for (int al = 0; al < 4; al++)
                                    s += conj(w[al * 4 + be]) * g[((long)c * V + n) * 12 + al * 3 + aa];
                            }
                            h[n * 12 + be * 3 + aa] = s;
                        }
                for (long m = 0; m < V; m++) {
                    cplx z[12];
                    transport_adj_site(L, bc_t, U, d, m, h, z);
                    for (int k = 0; k < 12; k++) gp[((long)cp * V + m) * 12 + k] += z[k];
                }
            }
        }
        free(h);
        free(g);
        g = gp;
    }
    free(g);
    for (int l = 0; l < nl; l++) free(a[l + 1]);
    for (long i = 0; i < woff; i++) {
        cplx v = gW[i];
        grad[2 * i] = 2 * creal(v);
        grad[2 * i + 1] = 2 * cimag(v);
    }
    return loss;
}

/*
 * Plain FP64 CPU oracle for the clover Wilson-Dirac operator, the Schwarz
 * alternating procedure (SAP) with minimal-residual (MR) block solves, and the
 * flexible GCR (FGCR) outer solver of "Solving the Dirac equation on QPACE"
 * (A. Nobile, Lattice 2010, arXiv:1109.4279).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Everything here is written for obviousness, not speed: naive site loops,
 * explicit 4x4 gamma matrices, full 12x12 per-site clover matrices, modified
 * Gram-Schmidt.  Complex numbers are C99 double complex; every array crosses
 * the ABI as interleaved (re, im) doubles.
 *
 * Conventions (the paper states none of them; the readings follow the SAP
 * papers it cites, Sec. 4):
 *   coordinates x = (x0, x1, x2, x3), x0 = time, extents L[0..3];
 *   lexicographic site index ((x0*L1 + x1)*L2 + x2)*L3 + x3;
 *   spinor field  (V, 4 spin, 3 colour) complex;
 *   gauge field   (V, 4 mu, 3, 3) complex, U_mu(x) = link x -> x + mu;
 *   clover field  (V, 12, 12) complex, row/column index = spin*3 + colour,
 *                 including the (4 + m0) mass term on the diagonal;
 *   boundary      bc[mu] multiplies the hop that wraps from x_mu = L_mu - 1
 *                 to 0 (antiperiodic time: bc = {-1, 1, 1, 1}).
 *
 * D psi(x) = A(x) psi(x)
 *          - 1/2 sum_mu [ eta_mu(x) U_mu(x) (1 - g_mu) psi(x + mu)
 *                       + eta_mu(x - mu) U_mu(x - mu)^+ (1 + g_mu) psi(x - mu) ]
 * A(x)     = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_{mu nu} Fhat_{mu nu}(x)
 * sigma_{mu nu} = (i/2) [g_mu, g_nu],  Fhat_{mu nu} = (Q_{mu nu} - Q_{nu mu}) / 8,
 * Q_{mu nu}(x) = sum of the four plaquette leaves in the (mu, nu) plane that
 * start and end at x, all traversed counter-clockwise (mu, nu, -mu, -nu).
 *
 * Parity unpinned: none -- every exported function is pinned by a test under
 * tests/test_oracle_*.py (closed forms, symmetries, independent dense algebra,
 * finite differences).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------------- */
/* Gamma matrices, chiral basis: g5 = g0 g1 g2 g3 = diag(1, 1, -1, -1).     */
/* ---------------------------------------------------------------------- */

static cplx GAM[4][4][4];      /* GAM[mu][row][col] */
static cplx SIG[4][4][4][4];   /* SIG[mu][nu][row][col] = (i/2)[g_mu, g_nu] */
static int gam_ready = 0;

static void init_gamma(void)
{
    if (gam_ready) return;
    memset(GAM, 0, sizeof(GAM));
    /* g0: off-diagonal blocks -1 */
    GAM[0][0][2] = -1; GAM[0][1][3] = -1; GAM[0][2][0] = -1; GAM[0][3][1] = -1;
    /* g_k: upper-right block -i sigma_k, lower-left block +i sigma_k */
    GAM[1][0][3] = -I; GAM[1][1][2] = -I; GAM[1][2][1] = I;  GAM[1][3][0] = I;
    GAM[2][0][3] = -1; GAM[2][1][2] = 1;  GAM[2][2][1] = 1;  GAM[2][3][0] = -1;
    GAM[3][0][2] = -I; GAM[3][1][3] = I;  GAM[3][2][0] = I;  GAM[3][3][1] = -I;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu)
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) {
                    cplx s = 0;
                    for (int k = 0; k < 4; ++k)
                        s += GAM[mu][r][k] * GAM[nu][k][c] - GAM[nu][r][k] * GAM[mu][k][c];
                    SIG[mu][nu][r][c] = 0.5 * I * s;
                }
    gam_ready = 1;
}

/* ---------------------------------------------------------------------- */
/* Geometry                                                               */
/* ---------------------------------------------------------------------- */

static long volume(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static long lex(const int L[4], const int x[4])
{
    return (((long)x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3];
}

static void coords(const int L[4], long i, int x[4])
{
    x[3] = (int)(i % L[3]); i /= L[3];
    x[2] = (int)(i % L[2]); i /= L[2];
    x[1] = (int)(i % L[1]); i /= L[1];
    x[0] = (int)i;
}

/* site index of x + step * mu-hat, periodic wrap */
static long shift(const int L[4], long i, int mu, int step)
{
    int x[4];
    coords(L, i, x);
    x[mu] = ((x[mu] + step) % L[mu] + L[mu]) % L[mu];
    return lex(L, x);
}

/* boundary sign of the forward hop x -> x + mu */
static double eta_fwd(const int L[4], const double bc[4], long i, int mu)
{
    int x[4];
    coords(L, i, x);
    return (x[mu] == L[mu] - 1) ? bc[mu] : 1.0;
}

/* ---------------------------------------------------------------------- */
/* 3x3 colour algebra                                                     */
/* ---------------------------------------------------------------------- */

typedef struct { cplx m[3][3]; } su3;

static su3 link(const cplx *U, long i, int mu)
{
    su3 r;
    memcpy(r.m, U + (i * 4 + mu) * 9, sizeof(r.m));
    return r;
}

static su3 mul(su3 a, su3 b)
{
    su3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0;
            for (int k = 0; k < 3; ++k) s += a.m[i][k] * b.m[k][j];
            r.m[i][j] = s;
        }
    return r;
}

static su3 dag(su3 a)
{
    su3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
    return r;
}

static su3 zero3(void) { su3 r; memset(r.m, 0, sizeof(r.m)); return r; }

static su3 add(su3 a, su3 b)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a.m[i][j] += b.m[i][j];
    return a;
}

/* ---------------------------------------------------------------------- */
/* Clover term (Sec. 1 "Wilson-Dirac ... with Clover term")                */
/* ---------------------------------------------------------------------- */

/*
 * Four leaves of the (mu, nu) plane at site i, each a closed loop starting and
 * ending at i, traversed counter-clockwise.  A leaf is a product of four
 * oriented links; leaf_links() returns (site, direction, daggered) for each.
 */
typedef struct { long site; int dir; int dagger; } hop;

static void leaf_links(const int L[4], long i, int mu, int nu, int leaf, hop h[4])
{
    long xm = shift(L, i, mu, -1), xn = shift(L, i, nu, -1);
    switch (leaf) {
    case 0: /* +mu, +nu, -mu, -nu */
        h[0] = (hop){i, mu, 0};
        h[1] = (hop){shift(L, i, mu, 1), nu, 0};
        h[2] = (hop){shift(L, i, nu, 1), mu, 1};
        h[3] = (hop){i, nu, 1};
        break;
    case 1: /* +nu, -mu, -nu, +mu */
        h[0] = (hop){i, nu, 0};
        h[1] = (hop){shift(L, shift(L, i, nu, 1), mu, -1), mu, 1};
        h[2] = (hop){xm, nu, 1};
        h[3] = (hop){xm, mu, 0};
        break;
    case 2: /* -mu, -nu, +mu, +nu */
        h[0] = (hop){xm, mu, 1};
        h[1] = (hop){shift(L, xm, nu, -1), nu, 1};
        h[2] = (hop){shift(L, xm, nu, -1), mu, 0};
        h[3] = (hop){xn, nu, 0};
        break;
    default: /* -nu, +mu, +nu, -mu */
        h[0] = (hop){xn, nu, 1};
        h[1] = (hop){xn, mu, 0};
        h[2] = (hop){shift(L, xn, mu, 1), nu, 0};
        h[3] = (hop){i, mu, 1};
        break;
    }
}

static su3 oriented(const cplx *U, hop h)
{
    su3 u = link(U, h.site, h.dir);
    return h.dagger ? dag(u) : u;
}

/* Q_{mu nu}(i) */
static su3 clover_leaves(const int L[4], const cplx *U, long i, int mu, int nu)
{
    su3 q = zero3();
    for (int leaf = 0; leaf < 4; ++leaf) {
        hop h[4];
        leaf_links(L, i, mu, nu, leaf, h);
        su3 p = oriented(U, h[0]);
        for (int k = 1; k < 4; ++k) p = mul(p, oriented(U, h[k]));
        q = add(q, p);
    }
    return q;
}

/* Fhat = (Q - Q^+)/8 for the ordered pair (mu, nu) */
static su3 fhat_from_q(su3 q)
{
    su3 f;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) f.m[a][b] = (q.m[a][b] - conj(q.m[b][a])) / 8.0;
    return f;
}

/* add c_sw (i/4) sum_{mu != nu} sigma_{mu nu} (x) F_{mu nu} to a 12x12 matrix */
static void add_sigma_f(cplx A[12][12], const su3 F[4][4], double csw)
{
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) {
            if (mu == nu) continue;
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    cplx sg = SIG[mu][nu][s][t];
                    if (sg == 0) continue;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            A[s * 3 + a][t * 3 + b] += csw * 0.25 * I * sg * F[mu][nu].m[a][b];
                }
        }
}

int oracle_clover(const int L[4], const double *U_, double m0, double csw, double *A_)
{
    init_gamma();
    const cplx *U = (const cplx *)U_;
    cplx (*A)[12][12] = (cplx (*)[12][12])A_;
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i) {
        su3 F[4][4];
        for (int mu = 0; mu < 4; ++mu) {
            F[mu][mu] = zero3();
            for (int nu = mu + 1; nu < 4; ++nu) {
                F[mu][nu] = fhat_from_q(clover_leaves(L, U, i, mu, nu));
                /* Q_{nu mu} = Q_{mu nu}^+  =>  Fhat_{nu mu} = -Fhat_{mu nu} */
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) F[nu][mu].m[a][b] = -F[mu][nu].m[a][b];
            }
        }
        memset(A[i], 0, sizeof(A[i]));
        for (int k = 0; k < 12; ++k) A[i][k][k] = 4.0 + m0;
        add_sigma_f(A[i], F, csw);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Dirac operator (Sec. 4: the matrix-vector product D psi)               */
/* ---------------------------------------------------------------------- */

/* out[12] += coef * U (1 + sgn * g_mu) in[12]  (U may be daggered) */
static void hop_term(cplx out[12], cplx coef, su3 u, int mu, int sgn, const cplx *in)
{
    cplx proj[12];
    for (int s = 0; s < 4; ++s)
        for (int c = 0; c < 3; ++c) {
            cplx v = in[s * 3 + c];
            for (int t = 0; t < 4; ++t) v += sgn * GAM[mu][s][t] * in[t * 3 + c];
            proj[s * 3 + c] = v;
        }
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            cplx v = 0;
            for (int b = 0; b < 3; ++b) v += u.m[a][b] * proj[s * 3 + b];
            out[s * 3 + a] += coef * v;
        }
}

/* D psi (dagger = 0) or D^+ psi (dagger = 1) at one site */
static void dirac_site(const int L[4], const cplx *U, const cplx *A, const double bc[4],
                       const cplx *psi, long i, int dagger, cplx out[12])
{
    const cplx *Ai = A + i * 144;
    for (int r = 0; r < 12; ++r) {
        cplx v = 0;
        for (int c = 0; c < 12; ++c)
            v += (dagger ? conj(Ai[c * 12 + r]) : Ai[r * 12 + c]) * psi[i * 12 + c];
        out[r] = v;
    }
    for (int mu = 0; mu < 4; ++mu) {
        long ip = shift(L, i, mu, 1), im = shift(L, i, mu, -1);
        double ef = eta_fwd(L, bc, i, mu), eb = eta_fwd(L, bc, im, mu);
        /* D:  -1/2 eta U_mu(x)(1 - g) psi(x+mu) - 1/2 eta U_mu(x-mu)^+(1 + g) psi(x-mu)
         * D^+: the spin projectors swap.                                      */
        int sf = dagger ? +1 : -1;
        hop_term(out, -0.5 * ef, link(U, i, mu), mu, sf, psi + ip * 12);
        hop_term(out, -0.5 * eb, dag(link(U, im, mu)), mu, -sf, psi + im * 12);
    }
}

int oracle_apply_D(const int L[4], const double *U_, const double *A_, const double bc[4],
                   const double *in_, double *out_, int dagger)
{
    init_gamma();
    const cplx *U = (const cplx *)U_, *A = (const cplx *)A_, *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i) dirac_site(L, U, A, bc, in, i, dagger, out + i * 12);
    return 0;
}

/*
 * Derivative of D with respect to h for the link deformation
 * U -> U + h dU (first order), applied to x:  out = (dD/dh) x.
 * Hopping terms are linear in each link; every clover leaf contains a given
 * link at most once, so dQ is the product rule over the four leaf factors.
 * The (4 + m0) term does not depend on U.
 */
int oracle_dD_apply(const int L[4], const double *U_, const double *dU_, const double bc[4],
                    double csw, const double *x_, double *out_)
{
    init_gamma();
    const cplx *U = (const cplx *)U_, *dU = (const cplx *)dU_, *x = (const cplx *)x_;
    cplx *out = (cplx *)out_;
    long V = volume(L);
    /* which links are deformed (skip leaves that contain none) */
    unsigned char *nz = (unsigned char *)calloc((size_t)V * 4, 1);
    for (long k = 0; k < V * 4; ++k)
        for (int e = 0; e < 9; ++e)
            if (dU[k * 9 + e] != 0) { nz[k] = 1; break; }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i) {
        cplx o[12];
        memset(o, 0, sizeof(o));
        /* hopping part */
        for (int mu = 0; mu < 4; ++mu) {
            long ip = shift(L, i, mu, 1), im = shift(L, i, mu, -1);
            double ef = eta_fwd(L, bc, i, mu), eb = eta_fwd(L, bc, im, mu);
            if (nz[i * 4 + mu]) hop_term(o, -0.5 * ef, link(dU, i, mu), mu, -1, x + ip * 12);
            if (nz[im * 4 + mu]) hop_term(o, -0.5 * eb, dag(link(dU, im, mu)), mu, +1, x + im * 12);
        }
        /* clover part */
        if (csw != 0) {
            su3 dF[4][4];
            int any = 0;
            for (int mu = 0; mu < 4; ++mu) {
                dF[mu][mu] = zero3();
                for (int nu = mu + 1; nu < 4; ++nu) {
                    su3 dq = zero3();
                    for (int leaf = 0; leaf < 4; ++leaf) {
                        hop h[4];
                        leaf_links(L, i, mu, nu, leaf, h);
                        for (int pos = 0; pos < 4; ++pos) {
                            if (!nz[h[pos].site * 4 + h[pos].dir]) continue;
                            any = 1;
                            su3 p;
                            for (int k = 0; k < 4; ++k) {
                                su3 f;
                                if (k == pos) {
                                    f = link(dU, h[k].site, h[k].dir);
                                    if (h[k].dagger) f = dag(f);
                                } else {
                                    f = oriented(U, h[k]);
                                }
                                p = (k == 0) ? f : mul(p, f);
                            }
                            dq = add(dq, p);
                        }
                    }
                    dF[mu][nu] = fhat_from_q(dq);
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) dF[nu][mu].m[a][b] = -dF[mu][nu].m[a][b];
                }
            }
            if (any) {
                cplx dA[12][12];
                memset(dA, 0, sizeof(dA));
                add_sigma_f(dA, dF, csw);
                for (int r = 0; r < 12; ++r)
                    for (int c = 0; c < 12; ++c) o[r] += dA[r][c] * x[i * 12 + c];
            }
        }
        memcpy(out + i * 12, o, sizeof(o));
    }
    free(nz);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Dense 12x12 inverse by Gauss-Jordan elimination with partial pivoting   */
/* ---------------------------------------------------------------------- */

static int invert12(const cplx *a_in, cplx *inv)
{
    cplx a[12][24];
    for (int r = 0; r < 12; ++r)
        for (int c = 0; c < 24; ++c) a[r][c] = (c < 12) ? a_in[r * 12 + c] : (c - 12 == r ? 1.0 : 0.0);
    for (int col = 0; col < 12; ++col) {
        int piv = col;
        for (int r = col + 1; r < 12; ++r)
            if (cabs(a[r][col]) > cabs(a[piv][col])) piv = r;
        if (cabs(a[piv][col]) == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 24; ++c) { cplx t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
        cplx d = a[col][col];
        for (int c = 0; c < 24; ++c) a[col][c] /= d;
        for (int r = 0; r < 12; ++r) {
            if (r == col) continue;
            cplx f = a[r][col];
            if (f == 0) continue;
            for (int c = 0; c < 24; ++c) a[r][c] -= f * a[col][c];
        }
    }
    for (int r = 0; r < 12; ++r)
        for (int c = 0; c < 12; ++c) inv[r * 12 + c] = a[r][c + 12];
    return 0;
}

/* ---------------------------------------------------------------------- */
/* SAP with MR block solves (Sec. 4, Sec. 5)                               */
/* ---------------------------------------------------------------------- */

typedef struct {
    const int *L;
    const cplx *U, *A;
    const double *bc;
    int b[4];
    long V, Vb, nblk;
    int nb[4];
} sap_geom;

static int site_parity(const int L[4], long i)
{
    int x[4];
    coords(L, i, x);
    return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* lexicographic site list of block n (block coordinates lexicographic) */
static void block_sites(const sap_geom *g, long n, long *sites)
{
    int bc[4];
    long t = n;
    bc[3] = (int)(t % g->nb[3]); t /= g->nb[3];
    bc[2] = (int)(t % g->nb[2]); t /= g->nb[2];
    bc[1] = (int)(t % g->nb[1]); t /= g->nb[1];
    bc[0] = (int)t;
    long k = 0;
    int y[4];
    for (y[0] = 0; y[0] < g->b[0]; ++y[0])
        for (y[1] = 0; y[1] < g->b[1]; ++y[1])
            for (y[2] = 0; y[2] < g->b[2]; ++y[2])
                for (y[3] = 0; y[3] < g->b[3]; ++y[3]) {
                    int x[4];
                    for (int mu = 0; mu < 4; ++mu) x[mu] = bc[mu] * g->b[mu] + y[mu];
                    sites[k++] = lex(g->L, x);
                }
}

static int block_colour(const sap_geom *g, long n)
{
    long t = n;
    int s = 0;
    for (int mu = 3; mu >= 0; --mu) { s += (int)(t % g->nb[mu]); t /= g->nb[mu]; }
    return s & 1;
}

/*
 * Block-restricted operator: out(i) = (D phi)(i) for i in the list, where phi
 * is a full-lattice field that vanishes outside the block.  Hops that leave the
 * block therefore contribute nothing (Dirichlet boundary, Sec. 4).
 */
static void dirac_on(const sap_geom *g, const cplx *phi, const long *list, long n, cplx *out)
{
    for (long k = 0; k < n; ++k) dirac_site(g->L, g->U, g->A, g->bc, phi, list[k], 0, out + k * 12);
}

static cplx dotv(const cplx *a, const cplx *b, long n)
{
    cplx s = 0;
    for (long k = 0; k < n; ++k) s += conj(a[k]) * b[k];
    return s;
}

/*
 * Approximate solve of D_blk chi = rho_blk by n_mr MR steps.
 * eo = 1: MR on the even-site Schur complement
 *         Dhat = A_ee - D_eo A_oo^-1 D_oe,   etahat = rho_e - D_eo A_oo^-1 rho_o,
 *         then chi_o = A_oo^-1 (rho_o - D_oe chi_e)   (even/odd split, Sec. 5, Table 1);
 * eo = 0: MR on D_blk directly.
 * work: full-lattice scratch field, zero on entry and on exit.
 * rho, chi: block-ordered (index k <-> site sites[k]), 12 complex per site.
 */
static int block_mr(const sap_geom *g, const long *sites, const cplx *rho, int nmr, int eo,
                    cplx *work, cplx *chi)
{
    long Vb = g->Vb;
    long ne = 0, no = 0;
    long *ev = (long *)malloc(sizeof(long) * Vb), *od = (long *)malloc(sizeof(long) * Vb);
    long *evk = (long *)malloc(sizeof(long) * Vb), *odk = (long *)malloc(sizeof(long) * Vb);
    for (long k = 0; k < Vb; ++k) {
        if (!eo || site_parity(g->L, sites[k]) == 0) { ev[ne] = sites[k]; evk[ne++] = k; }
        else { od[no] = sites[k]; odk[no++] = k; }
    }
    cplx *ainv = (cplx *)malloc(sizeof(cplx) * 144 * (no ? no : 1));
    int err = 0;
    for (long k = 0; k < no; ++k)
        if (invert12(g->A + od[k] * 144, ainv + k * 144)) err = -1;
    cplx *x = (cplx *)calloc((size_t)ne * 12, sizeof(cplx));
    cplx *r = (cplx *)malloc(sizeof(cplx) * ne * 12);
    cplx *p = (cplx *)malloc(sizeof(cplx) * ne * 12);
    cplx *to = (cplx *)malloc(sizeof(cplx) * (no ? no : 1) * 12);

#define PUT(list, n, vec) for (long k_ = 0; k_ < (n); ++k_) memcpy(work + (list)[k_] * 12, (vec) + k_ * 12, sizeof(cplx) * 12)
#define CLR(list, n) for (long k_ = 0; k_ < (n); ++k_) memset(work + (list)[k_] * 12, 0, sizeof(cplx) * 12)
    /* etahat */
    for (long k = 0; k < ne; ++k) memcpy(r + k * 12, rho + evk[k] * 12, sizeof(cplx) * 12);
    if (eo && no) {
        for (long k = 0; k < no; ++k) {
            const cplx *ro = rho + odk[k] * 12;
            for (int a = 0; a < 12; ++a) {
                cplx v = 0;
                for (int b = 0; b < 12; ++b) v += ainv[k * 144 + a * 12 + b] * ro[b];
                to[k * 12 + a] = v;
            }
        }
        PUT(od, no, to);
        dirac_on(g, work, ev, ne, p);        /* D_eo A_oo^-1 rho_o (hops only) */
        CLR(od, no);
        for (long k = 0; k < ne * 12; ++k) r[k] -= p[k];
    }
    for (int it = 0; it < nmr; ++it) {
        /* p = Dhat r */
        PUT(ev, ne, r);
        dirac_on(g, work, ev, ne, p);        /* A_ee r (+ hops within the even set if eo = 0) */
        if (eo && no) {
            dirac_on(g, work, od, no, to);   /* D_oe r */
            CLR(ev, ne);
            for (long k = 0; k < no; ++k) {
                cplx t[12];
                for (int a = 0; a < 12; ++a) {
                    cplx v = 0;
                    for (int b = 0; b < 12; ++b) v += ainv[k * 144 + a * 12 + b] * to[k * 12 + b];
                    t[a] = v;
                }
                memcpy(to + k * 12, t, sizeof(t));
            }
            PUT(od, no, to);
            cplx *q = (cplx *)malloc(sizeof(cplx) * ne * 12);
            dirac_on(g, work, ev, ne, q);    /* D_eo A_oo^-1 D_oe r */
            CLR(od, no);
            for (long k = 0; k < ne * 12; ++k) p[k] -= q[k];
            free(q);
        } else {
            CLR(ev, ne);
        }
        cplx pr = dotv(p, r, ne * 12);
        double pp = creal(dotv(p, p, ne * 12));
        if (pp == 0.0) break;
        cplx alpha = pr / pp;
        for (long k = 0; k < ne * 12; ++k) { x[k] += alpha * r[k]; r[k] -= alpha * p[k]; }
    }
    memset(chi, 0, sizeof(cplx) * Vb * 12);
    for (long k = 0; k < ne; ++k) memcpy(chi + evk[k] * 12, x + k * 12, sizeof(cplx) * 12);
    if (eo && no) {
        /* chi_o = A_oo^-1 (rho_o - D_oe chi_e) */
        PUT(ev, ne, x);
        dirac_on(g, work, od, no, to);
        CLR(ev, ne);
        for (long k = 0; k < no; ++k) {
            cplx t[12];
            for (int a = 0; a < 12; ++a) t[a] = rho[odk[k] * 12 + a] - to[k * 12 + a];
            for (int a = 0; a < 12; ++a) {
                cplx v = 0;
                for (int b = 0; b < 12; ++b) v += ainv[k * 144 + a * 12 + b] * t[b];
                chi[odk[k] * 12 + a] = v;
            }
        }
    }
#undef PUT
#undef CLR
    free(ev); free(od); free(evk); free(odk); free(ainv); free(x); free(r); free(p); free(to);
    return err;
}

static int geom_init(sap_geom *g, const int L[4], const double *U_, const double *A_,
                     const double bc[4], const int b[4])
{
    g->L = L;
    g->U = (const cplx *)U_;
    g->A = (const cplx *)A_;
    g->bc = bc;
    g->V = volume(L);
    g->Vb = 1;
    g->nblk = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (b[mu] <= 0 || L[mu] % b[mu]) return -2;
        g->b[mu] = b[mu];
        g->nb[mu] = L[mu] / b[mu];
        if (g->nb[mu] % 2) return -2;  /* chessboard colouring needs even block counts */
        g->Vb *= b[mu];
        g->nblk *= g->nb[mu];
    }
    return 0;
}

/*
 * psi = M_SAP eta (Sec. 4): n_cy cycles; each cycle first solves the equation
 * on all white blocks (even sum of block coordinates), then updates the
 * residue on the white blocks and on the border of the black blocks, then does
 * the same for the black blocks.  Within one colour the block solves are
 * independent (each reads the residue on its own block only), so they are
 * computed first -- in parallel -- and the combined correction chi (a sum of
 * corrections with disjoint supports) is then added to psi and its image
 * D chi subtracted from the residue:  rho <- rho - D chi  changes rho exactly
 * on the solved blocks and on the sites one hop outside them.
 * order = 1 visits the blocks of a colour in reverse order (the result must
 * not depend on it).  rho_out (optional) receives the final residue.
 */
int oracle_sap(const int L[4], const double *U_, const double *A_, const double bc[4],
               const int b[4], int ncy, int nmr, int eo, int order,
               const double *eta_, double *psi_, double *rho_out)
{
    init_gamma();
    sap_geom g;
    int st = geom_init(&g, L, U_, A_, bc, b);
    if (st) return st;
    long V = g.V;
    cplx *psi = (cplx *)psi_;
    cplx *rho = (cplx *)malloc(sizeof(cplx) * V * 12);
    cplx *chi_all = (cplx *)malloc(sizeof(cplx) * V * 12);
    cplx *dchi = (cplx *)malloc(sizeof(cplx) * V * 12);
    memcpy(rho, eta_, sizeof(cplx) * V * 12);
    memset(psi, 0, sizeof(cplx) * V * 12);
    long *list = (long *)malloc(sizeof(long) * g.nblk);
    int err = 0;
    for (int cy = 0; cy < ncy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            long nl = 0;
            for (long j = 0; j < g.nblk; ++j) {
                long n = order ? g.nblk - 1 - j : j;
                if (block_colour(&g, n) == colour) list[nl++] = n;
            }
            memset(chi_all, 0, sizeof(cplx) * V * 12);
#pragma omp parallel
            {
                cplx *work = (cplx *)calloc((size_t)V * 12, sizeof(cplx));
                long *sites = (long *)malloc(sizeof(long) * g.Vb);
                cplx *rb = (cplx *)malloc(sizeof(cplx) * g.Vb * 12);
                cplx *chi = (cplx *)malloc(sizeof(cplx) * g.Vb * 12);
#pragma omp for schedule(dynamic)
                for (long j = 0; j < nl; ++j) {
                    block_sites(&g, list[j], sites);
                    for (long k = 0; k < g.Vb; ++k) memcpy(rb + k * 12, rho + sites[k] * 12, sizeof(cplx) * 12);
                    if (block_mr(&g, sites, rb, nmr, eo, work, chi)) {
#pragma omp atomic write
                        err = -3;
                    }
                    for (long k = 0; k < g.Vb; ++k) memcpy(chi_all + sites[k] * 12, chi + k * 12, sizeof(cplx) * 12);
                }
                free(work); free(sites); free(rb); free(chi);
            }
            oracle_apply_D(L, U_, A_, bc, (const double *)chi_all, (double *)dchi, 0);
            for (long e = 0; e < V * 12; ++e) {
                psi[e] += chi_all[e];
                rho[e] -= dchi[e];
            }
        }
    if (rho_out) memcpy(rho_out, rho, sizeof(cplx) * V * 12);
    free(rho); free(chi_all); free(dchi); free(list);
    return err;
}

/*
 * One isolated block solve (for tests): rho is the block-ordered right-hand
 * side of block n (sites in lexicographic order inside the block), chi the
 * block-ordered MR approximation of D_blk^-1 rho.
 */
int oracle_block_mr(const int L[4], const double *U_, const double *A_, const double bc[4],
                    const int b[4], long n, int nmr, int eo, const double *rho_, double *chi_)
{
    init_gamma();
    sap_geom g;
    int st = geom_init(&g, L, U_, A_, bc, b);
    if (st) return st;
    cplx *work = (cplx *)calloc((size_t)g.V * 12, sizeof(cplx));
    long *sites = (long *)malloc(sizeof(long) * g.Vb);
    block_sites(&g, n, sites);
    int err = block_mr(&g, sites, (const cplx *)rho_, nmr, eo, work, (cplx *)chi_);
    free(work); free(sites);
    return err;
}

/* lexicographic lattice sites of block n, in block order (for tests) */
int oracle_block_sites(const int L[4], const int b[4], long n, long *sites)
{
    sap_geom g;
    int st = geom_init(&g, L, NULL, NULL, NULL, b);
    if (st) return st;
    block_sites(&g, n, sites);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Flexible GCR with restarts (Sec. 4)                                      */
/* ---------------------------------------------------------------------- */

/*
 * Solves D x = b.  precond = 0: unpreconditioned GCR (phi_k = rho_k);
 * precond = 1: phi_k = M_SAP rho_k (FP64 SAP).  On entry x holds the
 * initial guess.  The recursion orthogonalises chi_k = D phi_k against the
 * previous chi_j by modified Gram-Schmidt, updates the recursive residual,
 * and at the end of each cycle solves the small triangular system, updates x
 * and recomputes the true residual b - D x.
 * info[0] = total iterations, info[1] = restart cycles, info[2] = converged,
 * res[0] = final true |b - D x| / |b|.  max_iters > 0 stops the recursion
 * after that many iterations in total (a bounded sample for timing).
 */
int oracle_fgcr(const int L[4], const double *U_, const double *A_, const double bc[4],
                const double *b_, double *x_, int nkv, int max_restarts, double tol,
                int precond, const int bs[4], int ncy, int nmr, int eo, int max_iters,
                int *info, double *res)
{
    init_gamma();
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    long V = volume(L), N = V * 12;
    cplx *r = (cplx *)malloc(sizeof(cplx) * N);
    cplx *rho = (cplx *)malloc(sizeof(cplx) * N);
    cplx **phi = (cplx **)calloc((size_t)nkv, sizeof(cplx *));
    cplx **chi = (cplx **)calloc((size_t)nkv, sizeof(cplx *));
    cplx *a = (cplx *)calloc((size_t)nkv * nkv, sizeof(cplx));
    cplx *c = (cplx *)calloc((size_t)nkv, sizeof(cplx));
    cplx *gam = (cplx *)calloc((size_t)nkv, sizeof(cplx));
    double *bn = (double *)calloc((size_t)nkv, sizeof(double));
    int iters = 0, cycles = 0, converged = 0, err = 0;
    double bnorm = sqrt(creal(dotv(b, b, N)));

    oracle_apply_D(L, U_, A_, bc, (const double *)x, (double *)r, 0);
    for (long k = 0; k < N; ++k) r[k] = b[k] - r[k];
    double rn = sqrt(creal(dotv(r, r, N)));
    if (bnorm == 0.0 || rn <= tol * bnorm) converged = 1;

    while (!converged && cycles < max_restarts) {
        memcpy(rho, r, sizeof(cplx) * N);
        int kused = 0;
        for (int k = 0; k < nkv; ++k) {
            if (!phi[k]) {
                phi[k] = (cplx *)malloc(sizeof(cplx) * N);
                chi[k] = (cplx *)malloc(sizeof(cplx) * N);
            }
            if (precond) {
                int st = oracle_sap(L, U_, A_, bc, bs, ncy, nmr, eo, 0, (const double *)rho,
                                    (double *)phi[k], NULL);
                if (st) { err = st; goto done; }
            } else {
                memcpy(phi[k], rho, sizeof(cplx) * N);
            }
            oracle_apply_D(L, U_, A_, bc, (const double *)phi[k], (double *)chi[k], 0);
            for (int j = 0; j < k; ++j) {
                a[j * nkv + k] = dotv(chi[j], chi[k], N);
                for (long e = 0; e < N; ++e) chi[k][e] -= a[j * nkv + k] * chi[j][e];
            }
            bn[k] = sqrt(creal(dotv(chi[k], chi[k], N)));
            if (bn[k] == 0.0) { err = -4; goto done; }
            for (long e = 0; e < N; ++e) chi[k][e] /= bn[k];
            c[k] = dotv(chi[k], rho, N);
            for (long e = 0; e < N; ++e) rho[e] -= c[k] * chi[k][e];
            ++iters;
            kused = k + 1;
            if (sqrt(creal(dotv(rho, rho, N))) <= tol * bnorm) break;
            if (max_iters > 0 && iters >= max_iters) break;
        }
        /* back substitution: A gamma = c, A_kk = |chi_k|, A_jk = a_jk (j < k) */
        for (int k = kused - 1; k >= 0; --k) {
            cplx s = c[k];
            for (int j = k + 1; j < kused; ++j) s -= a[k * nkv + j] * gam[j];
            gam[k] = s / bn[k];
        }
        for (int k = 0; k < kused; ++k)
            for (long e = 0; e < N; ++e) x[e] += gam[k] * phi[k][e];
        oracle_apply_D(L, U_, A_, bc, (const double *)x, (double *)r, 0);
        for (long k = 0; k < N; ++k) r[k] = b[k] - r[k];
        rn = sqrt(creal(dotv(r, r, N)));
        ++cycles;
        if (rn <= tol * bnorm) converged = 1;
        if (max_iters > 0 && iters >= max_iters) break;
    }
done:
    if (info) { info[0] = iters; info[1] = cycles; info[2] = converged; }
    if (res) res[0] = bnorm > 0 ? rn / bnorm : rn;
    for (int k = 0; k < nkv; ++k) { free(phi[k]); free(chi[k]); }
    free(phi); free(chi); free(a); free(c); free(gam); free(bn); free(r); free(rho);
    return err;
}

/* number of OpenMP threads the oracle runs with (1 when built without OpenMP) */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * qdd_oracle.c -- plain FP64 CPU oracle for the Wilson-clover quark solver
 * with the restricted additive Schwarz (RAS) preconditioner.
 *
 * TEST INFRASTRUCTURE ONLY.  This file defines what the GPU library must
 * compute, written as directly as possible so that a reader can check it
 * against the paper by eye.  It is called only by the tests, by the smoke
 * check and by the benchmark's CPU-baseline leg; the GPU library never links,
 * imports or executes it, and it shares no code, header, table or constant
 * with the GPU library.
 *
 * Paper: Osaki & Ishikawa, "Domain Decomposition method on GPU cluster",
 * Lattice 2010.
 *   - Eq. 1 (Sec. 1): the quark equation D phi = eta.
 *   - Sec. 2, Alg. 1: the RAS iteration phi = K_RAS eta (projection P,
 *     Dirichlet domain solve, restriction R, sum, update phi += v, r -= D v).
 *   - Sec. 2, Eq. 2: K_RAS = S sum_j (1 - D S)^j, S = sum_i R_i D_i'^-1 P_i.
 *   - Sec. 2, Eq. 3: right preconditioning D K chi = eta, phi = K chi.
 *   - Sec. 2 (parameters d, N_dominv, NRAS) and Sec. 4 (extension s, d = 2s).
 *   - Sec. 1 and Sec. 2 (the Schwarz family): plain additive Schwarz (AS,
 *     the domain solutions summed over every extended site) and the
 *     multiplicative Schwarz alternating procedure (SAP, domains of one colour
 *     of a red/black block ordering at a time, the residual updated between
 *     the colours), as comparisons to RAS.
 *   - Sec. 3: mixed-precision nested BiCGStab (inner solve preconditions the
 *     outer); here every level is FP64.  ora_solve takes the outer as FP64
 *     defect correction, ora_solve_nested as the paper's outer BiCGStab with
 *     the inner solve as a (variable) preconditioner.
 *   - Sec. 5: O(a)-improved Wilson quark, kappa, c_SW, stopping rule
 *     |eta - D phi| / |eta|.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - D = A - kappa H with the hopping term
 *       (H psi)(x) = sum_mu [ b (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                           + b (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
 *     b = bc[mu] when the hop crosses the lattice boundary in direction mu,
 *     else 1 (antiperiodic time: bc[3] = -1).
 *   - A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) Fhat_{mu nu}(x),
 *     sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu],
 *     Fhat_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag) / 8, Q the sum of the four
 *     plaquette leaves in the (mu, nu) plane at x; no traceless projection;
 *     gauge links are periodic inside the clover.
 *   - gamma matrices in the DeGrand-Rossi basis, mu = 0..3 <-> x, y, z, t.
 *   - Domains: bulk blocks of shape b tile the lattice; the extended domain
 *     adds s sites on both sides in every direction with b_mu < L_mu
 *     (periodic wrap); a direction with b_mu = L_mu is not extended and its
 *     hops wrap inside the domain with the boundary sign.  The Dirichlet
 *     operator drops every hop whose target leaves the extended domain.
 *   - The "fixed iteration solver" of the domains is minimal residual (MR),
 *     zero start, exactly N_dominv iterations; an "exact" mode (BiCGStab to
 *     1e-13 on the domain) exists for the checks.
 *   - Outer solver: FP64 defect correction, phi += |r| * inner(r / |r|).
 *
 * Layouts (canonical): site i = x + Lx(y + Ly(z + Lz t)); spinor complex
 * [V][4][3]; gauge complex [V][4][3][3]; clover complex [V][12][12] with
 * row/column index 3*spin + colour.
 */

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------------ */
/* Parameters passed from Python (mirrored with ctypes).                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int L[4];          /* Lx, Ly, Lz, Lt */
    int bc[4];         /* +1 periodic, -1 antiperiodic, per direction */
    const cplx *U;     /* gauge field [V][4][3][3] */
    const cplx *A;     /* clover term [V][12][12] (from ora_clover), or NULL:
                          then A(x) is rebuilt from U at every use */
    double kappa;
    double csw;
} ora_op;

typedef struct {
    int use_ras;       /* 0: K = identity (plain BiCGStab) */
    int block[4];      /* bulk block shape */
    int s;             /* extension; overlap depth d = 2 s */
    int n_ras;         /* NRAS */
    int n_dominv;      /* N_dominv */
    int dom_solver;    /* 0: MR with n_dominv iterations; 1: exact */
    int schwarz;       /* 0: RAS (Alg. 1); 1: SAP (multiplicative, red/black);
                          2: AS (additive, no restriction) */
} ora_prec;

enum { ORA_RAS = 0, ORA_SAP = 1, ORA_AS = 2 };

typedef struct {
    int outer_iters;
    int inner_iters;
    int dv_count;      /* global D applications inside the inner solves */
    int status;        /* 0 converged, 1 not converged, 2 breakdown */
    double true_rel_residual;
} ora_info;

/* ------------------------------------------------------------------------ */
/* Threads                                                                   */
/* ------------------------------------------------------------------------ */

void ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ora_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gamma matrices, DeGrand-Rossi basis (rows listed).                        */
/* ------------------------------------------------------------------------ */

static void gamma_matrix(int mu, cplx g[4][4])
{
    memset(g, 0, 16 * sizeof(cplx));
    switch (mu) {
    case 0: /* gamma_1 */
        g[0][3] = I;  g[1][2] = I;  g[2][1] = -I; g[3][0] = -I;
        break;
    case 1: /* gamma_2 */
        g[0][3] = -1; g[1][2] = 1;  g[2][1] = 1;  g[3][0] = -1;
        break;
    case 2: /* gamma_3 */
        g[0][2] = I;  g[1][3] = -I; g[2][0] = -I; g[3][1] = I;
        break;
    case 3: /* gamma_4 */
        g[0][2] = 1;  g[1][3] = 1;  g[2][0] = 1;  g[3][1] = 1;
        break;
    default: { /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 */
        cplx a[4][4], b[4][4], t[4][4];
        gamma_matrix(0, a);
        for (int k = 1; k < 4; k++) {
            gamma_matrix(k, b);
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) {
                    cplx acc = 0;
                    for (int l = 0; l < 4; l++) acc += a[i][l] * b[l][j];
                    t[i][j] = acc;
                }
            memcpy(a, t, sizeof(t));
        }
        memcpy(g, a, sizeof(a));
    }
    }
}

/* Exported for the checks: mu = 0..3 gives gamma_{mu+1}, 4 gives gamma_5. */
void ora_gamma(int mu, cplx *out)
{
    cplx g[4][4];
    gamma_matrix(mu, g);
    memcpy(out, g, sizeof(g));
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry                                                          */
/* ------------------------------------------------------------------------ */

static long volume(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void site_coords(const int L[4], long i, int c[4])
{
    for (int mu = 0; mu < 4; mu++) {
        c[mu] = (int)(i % L[mu]);
        i /= L[mu];
    }
}

static long site_index(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* Neighbour of site i one step in direction mu (dir = +1 or -1), periodic. */
static long neighbour(const int L[4], long i, int mu, int dir)
{
    int c[4];
    site_coords(L, i, c);
    c[mu] = (c[mu] + dir + L[mu]) % L[mu];
    return site_index(L, c);
}

/* Fermion boundary sign of the hop from site i in direction mu, dir. */
static double hop_sign(const int L[4], const int bc[4], long i, int mu, int dir)
{
    int c[4];
    site_coords(L, i, c);
    if (dir > 0 && c[mu] == L[mu] - 1) return (double)bc[mu];
    if (dir < 0 && c[mu] == 0) return (double)bc[mu];
    return 1.0;
}

static const cplx *link(const cplx *U, long i, int mu) { return U + (i * 4 + mu) * 9; }

/* ------------------------------------------------------------------------ */
/* 3x3 matrices                                                              */
/* ------------------------------------------------------------------------ */

static void m3_mul(const cplx *a, const cplx *b, cplx *c) /* c = a b */
{
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx acc = 0;
            for (int k = 0; k < 3; k++) acc += a[i * 3 + k] * b[k * 3 + j];
            t[i * 3 + j] = acc;
        }
    memcpy(c, t, sizeof(t));
}

static void m3_dag(const cplx *a, cplx *c) /* c = a^dag */
{
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) t[i * 3 + j] = conj(a[j * 3 + i]);
    memcpy(c, t, sizeof(t));
}

/* ------------------------------------------------------------------------ */
/* Clover term A = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) Fhat_{mu nu} */
/* ------------------------------------------------------------------------ */

/* Sum of the four counter-clockwise plaquette leaves in the (mu,nu) plane
 * that touch site x, each starting and ending at x. */
static void clover_leaves(const int L[4], const cplx *U, long x, int mu, int nu, cplx *Q)
{
    long xpm = neighbour(L, x, mu, +1);
    long xpn = neighbour(L, x, nu, +1);
    long xmm = neighbour(L, x, mu, -1);
    long xmn = neighbour(L, x, nu, -1);
    long xmm_pn = neighbour(L, xmm, nu, +1);
    long xmm_mn = neighbour(L, xmm, nu, -1);
    long xpm_mn = neighbour(L, xpm, nu, -1);
    cplx d[9], leaf[9];

    memset(Q, 0, 9 * sizeof(cplx));

    /* leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
    m3_mul(link(U, x, mu), link(U, xpm, nu), leaf);
    m3_dag(link(U, xpn, mu), d); m3_mul(leaf, d, leaf);
    m3_dag(link(U, x, nu), d);   m3_mul(leaf, d, leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];

    /* leaf 2: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu) */
    m3_dag(link(U, xmm_pn, mu), d); m3_mul(link(U, x, nu), d, leaf);
    m3_dag(link(U, xmm, nu), d);    m3_mul(leaf, d, leaf);
    m3_mul(leaf, link(U, xmm, mu), leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];

    /* leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu) */
    m3_dag(link(U, xmm, mu), leaf);
    m3_dag(link(U, xmm_mn, nu), d); m3_mul(leaf, d, leaf);
    m3_mul(leaf, link(U, xmm_mn, mu), leaf);
    m3_mul(leaf, link(U, xmn, nu), leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];

    /* leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag */
    m3_dag(link(U, xmn, nu), leaf);
    m3_mul(leaf, link(U, xmn, mu), leaf);
    m3_mul(leaf, link(U, xpm_mn, nu), leaf);
    m3_dag(link(U, x, mu), d); m3_mul(leaf, d, leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];
}

/* Fhat_{mu nu}(x) = (Q - Q^dag) / 8 (exported for the checks). */
void ora_field_strength(const int L[4], const cplx *U, long x, int mu, int nu, cplx *F)
{
    cplx Q[9], Qd[9];
    clover_leaves(L, U, x, mu, nu, Q);
    m3_dag(Q, Qd);
    for (int k = 0; k < 9; k++) F[k] = (Q[k] - Qd[k]) / 8.0;
}

/* The 12x12 clover matrix at one site, index 3*spin + colour. */
static void clover_site(const int L[4], const cplx *U, long x, double kappa, double csw, cplx *a)
{
    memset(a, 0, 144 * sizeof(cplx));
    for (int k = 0; k < 12; k++) a[k * 12 + k] = 1.0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++) {
            cplx gm[4][4], gn[4][4], sigma[4][4], F[9];
            gamma_matrix(mu, gm);
            gamma_matrix(nu, gn);
            for (int s = 0; s < 4; s++)
                for (int t = 0; t < 4; t++) {
                    cplx c = 0;
                    for (int l = 0; l < 4; l++) c += gm[s][l] * gn[l][t] - gn[s][l] * gm[l][t];
                    sigma[s][t] = 0.5 * I * c;  /* sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] */
                }
            ora_field_strength(L, U, x, mu, nu, F);
            for (int s = 0; s < 4; s++)
                for (int t = 0; t < 4; t++) {
                    if (sigma[s][t] == 0) continue;
                    for (int a1 = 0; a1 < 3; a1++)
                        for (int b1 = 0; b1 < 3; b1++)
                            a[(s * 3 + a1) * 12 + (t * 3 + b1)] += I * kappa * csw * sigma[s][t] * F[a1 * 3 + b1];
                }
        }
}

void ora_clover(const int L[4], const cplx *U, double kappa, double csw, cplx *A)
{
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) clover_site(L, U, x, kappa, csw, A + x * 144);
}

/* ------------------------------------------------------------------------ */
/* Wilson-clover operator D (Eq. 1)                                          */
/* ------------------------------------------------------------------------ */

/* out += coef * (1 + pm gamma_mu) (x) M applied to psi (12 components),
 * where M is U (dag = 0) or U^dag (dag = 1). */
static void add_hop(cplx *out, cplx coef, int mu, int pm, const cplx *Ul, int dag, const cplx *psi)
{
    cplx g[4][4];
    cplx m[9];
    gamma_matrix(mu, g);
    if (dag) m3_dag(Ul, m); else memcpy(m, Ul, sizeof(m));
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            cplx acc = 0;
            for (int t = 0; t < 4; t++) {
                cplx proj = (s == t ? 1.0 : 0.0) + pm * g[s][t];
                if (proj == 0) continue;
                for (int b = 0; b < 3; b++) acc += proj * m[a * 3 + b] * psi[t * 3 + b];
            }
            out[s * 3 + a] += coef * acc;
        }
}

static void clover_mul(const cplx *a, const cplx *psi, cplx *out) /* out = A psi */
{
    for (int r = 0; r < 12; r++) {
        cplx acc = 0;
        for (int c = 0; c < 12; c++) acc += a[r * 12 + c] * psi[c];
        out[r] = acc;
    }
}

/* The clover matrix of site x: the stored one, or rebuilt into tmp. */
static const cplx *clover_of(const ora_op *op, long x, cplx *tmp)
{
    if (op->A) return op->A + x * 144;
    clover_site(op->L, op->U, x, op->kappa, op->csw, tmp);
    return tmp;
}

/* (D in)(x) for one site x. */
static void dslash_site(const ora_op *op, long x, const cplx *in, cplx *o)
{
    cplx tmp[144];
    clover_mul(clover_of(op, x, tmp), in + x * 12, o);
    for (int mu = 0; mu < 4; mu++) {
        long xf = neighbour(op->L, x, mu, +1);
        long xb = neighbour(op->L, x, mu, -1);
        double sf = hop_sign(op->L, op->bc, x, mu, +1);
        double sb = hop_sign(op->L, op->bc, x, mu, -1);
        /* forward: (1 - gamma_mu) U_mu(x) psi(x + mu) */
        add_hop(o, -op->kappa * sf, mu, -1, link(op->U, x, mu), 0, in + xf * 12);
        /* backward: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) */
        add_hop(o, -op->kappa * sb, mu, +1, link(op->U, xb, mu), 1, in + xb * 12);
    }
}

void ora_dslash(const ora_op *op, const cplx *in, cplx *out)
{
    long V = volume(op->L);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) dslash_site(op, x, in, out + x * 12);
}

/* (D in) at a list of sites only: out[k] = (D in)(sites[k]). */
void ora_dslash_sites(const ora_op *op, long nsites, const long *sites, const cplx *in, cplx *out)
{
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nsites; k++) dslash_site(op, sites[k], in, out + k * 12);
}

/* ------------------------------------------------------------------------ */
/* Vector algebra on complex vectors of length n                             */
/* ------------------------------------------------------------------------ */

static cplx vdot(long n, const cplx *a, const cplx *b) /* sum conj(a) b */
{
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (long k = 0; k < n; k++) {
        cplx p = conj(a[k]) * b[k];
        re += creal(p);
        im += cimag(p);
    }
    return re + I * im;
}

static double vnorm2(long n, const cplx *a)
{
    double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long k = 0; k < n; k++) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Domains (Sec. 2, Sec. 4)                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int L[4], bc[4];
    int b[4];    /* bulk block */
    int s;
    int e[4];    /* extended length */
    int sh[4];   /* extension applied in this direction (s or 0) */
    int nb[4];   /* blocks per direction */
    int ndom;
    long nloc;   /* sites in an extended domain */
} ora_dd;

static int dd_init(ora_dd *d, const int L[4], const int bc[4], const int b[4], int s)
{
    if (s < 0) return -1;
    d->ndom = 1;
    d->nloc = 1;
    d->s = s;
    for (int mu = 0; mu < 4; mu++) {
        d->L[mu] = L[mu];
        d->bc[mu] = bc[mu];
        d->b[mu] = b[mu];
        if (b[mu] <= 0 || L[mu] % b[mu] != 0) return -1;
        if (b[mu] == L[mu]) {
            d->e[mu] = L[mu];
            d->sh[mu] = 0;
        } else {
            if (b[mu] + 2 * s > L[mu]) return -1;
            d->e[mu] = b[mu] + 2 * s;
            d->sh[mu] = s;
        }
        d->nb[mu] = L[mu] / b[mu];
        d->ndom *= d->nb[mu];
        d->nloc *= d->e[mu];
    }
    return 0;
}

/* Global site of local site l of domain dom, and whether it is a bulk site. */
static long dd_global(const ora_dd *d, int dom, long l, int *bulk)
{
    int k[4], lc[4], g[4];
    int r = dom;
    for (int mu = 0; mu < 4; mu++) {
        k[mu] = r % d->nb[mu];
        r /= d->nb[mu];
    }
    long t = l;
    for (int mu = 0; mu < 4; mu++) {
        lc[mu] = (int)(t % d->e[mu]);
        t /= d->e[mu];
    }
    *bulk = 1;
    for (int mu = 0; mu < 4; mu++) {
        g[mu] = ((k[mu] * d->b[mu] - d->sh[mu] + lc[mu]) % d->L[mu] + d->L[mu]) % d->L[mu];
        if (lc[mu] < d->sh[mu] || lc[mu] >= d->sh[mu] + d->b[mu]) *bulk = 0;
    }
    return site_index(d->L, g);
}

/* Local neighbour of local site l in direction mu, dir; -1 if the hop leaves
 * the extended domain (Dirichlet boundary). */
static long dd_local_neighbour(const ora_dd *d, long l, int mu, int dir)
{
    int lc[4];
    long t = l;
    for (int m = 0; m < 4; m++) {
        lc[m] = (int)(t % d->e[m]);
        t /= d->e[m];
    }
    int n = lc[mu] + dir;
    if (d->b[mu] == d->L[mu]) {
        n = (n + d->e[mu]) % d->e[mu];
    } else if (n < 0 || n >= d->e[mu]) {
        return -1;
    }
    lc[mu] = n;
    long idx = 0;
    for (int m = 3; m >= 0; m--) idx = idx * d->e[m] + lc[m];
    return idx;
}

int ora_ndomains(const int L[4], const int b[4], int s)
{
    ora_dd d;
    int bc[4] = {1, 1, 1, 1};
    if (dd_init(&d, L, bc, b, s)) return -1;
    return d.ndom;
}

/* Global site list of extended domain dom in local lexicographic order, and
 * bulk flags.  Returns the number of sites, or -1 for an invalid blocking. */
long ora_domain_sites(const int L[4], const int b[4], int s, int dom, long *sites, int *bulk)
{
    ora_dd d;
    int bc[4] = {1, 1, 1, 1};
    if (dd_init(&d, L, bc, b, s) || dom < 0 || dom >= d.ndom) return -1;
    for (long l = 0; l < d.nloc; l++) {
        int bk;
        long g = dd_global(&d, dom, l, &bk);
        if (sites) sites[l] = g;
        if (bulk) bulk[l] = bk;
    }
    return d.nloc;
}

/* D restricted to the extended domain with Dirichlet boundary (Alg. 1 line 5). */
static void dd_apply(const ora_op *op, const ora_dd *d, const long *gsite, const cplx *in, cplx *out)
{
    for (long l = 0; l < d->nloc; l++) {
        long x = gsite[l];
        cplx *o = out + l * 12;
        cplx tmp[144];
        clover_mul(clover_of(op, x, tmp), in + l * 12, o);
        for (int mu = 0; mu < 4; mu++) {
            long lf = dd_local_neighbour(d, l, mu, +1);
            long lb = dd_local_neighbour(d, l, mu, -1);
            if (lf >= 0)
                add_hop(o, -op->kappa * hop_sign(op->L, op->bc, x, mu, +1), mu, -1,
                        link(op->U, x, mu), 0, in + lf * 12);
            if (lb >= 0)
                add_hop(o, -op->kappa * hop_sign(op->L, op->bc, x, mu, -1), mu, +1,
                        link(op->U, gsite[lb], mu), 1, in + lb * 12);
        }
    }
}

int ora_domain_apply(const ora_op *op, const int b[4], int s, int dom, const cplx *in, cplx *out)
{
    ora_dd d;
    if (dd_init(&d, op->L, op->bc, b, s) || dom < 0 || dom >= d.ndom) return -1;
    long *g = malloc(d.nloc * sizeof(long));
    for (long l = 0; l < d.nloc; l++) {
        int bk;
        g[l] = dd_global(&d, dom, l, &bk);
    }
    dd_apply(op, &d, g, in, out);
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* BiCGStab (van der Vorst), right-preconditioned as in Eq. 3                */
/* ------------------------------------------------------------------------ */

typedef void (*apply_fn)(void *ctx, const cplx *in, cplx *out);

/* Solves M x = b with right preconditioner K (K may be NULL for identity):
 * M K chi = b, x = K chi.  x must hold the start (zero here).  Stops when
 * |r| <= tol |b| on the recursive residual.  Returns 0 on convergence, 1 if
 * maxit was reached, 2 on a second breakdown. */
static int bicgstab(long n, apply_fn M, void *mctx, apply_fn K, void *kctx,
                    const cplx *b, cplx *x, double tol, int maxit, int *iters, int *napply)
{
    cplx *r = malloc(n * sizeof(cplx)), *rh = malloc(n * sizeof(cplx));
    cplx *p = malloc(n * sizeof(cplx)), *v = malloc(n * sizeof(cplx));
    cplx *s = malloc(n * sizeof(cplx)), *t = malloc(n * sizeof(cplx));
    cplx *ph = malloc(n * sizeof(cplx)), *sh = malloc(n * sizeof(cplx));
    double bnorm = sqrt(vnorm2(n, b));
    int status = 1, restarted = 0, k = 0;
    cplx rho = 1, alpha = 1, omega = 1;

    memcpy(r, b, n * sizeof(cplx));
    memcpy(rh, b, n * sizeof(cplx));
    memset(p, 0, n * sizeof(cplx));
    memset(v, 0, n * sizeof(cplx));
    memset(x, 0, n * sizeof(cplx));
    if (bnorm == 0) { status = 0; goto done; }

    for (k = 0; k < maxit;) {
        cplx rho_new = vdot(n, rh, r);
        cplx beta = (rho_new / rho) * (alpha / omega);
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        if (K) K(kctx, p, ph); else memcpy(ph, p, n * sizeof(cplx));
        M(mctx, ph, v);
        if (napply) (*napply)++;
        cplx rv = vdot(n, rh, v);
        if (cabs(rv) < 1e-30 * sqrt(vnorm2(n, rh)) * sqrt(vnorm2(n, v))) goto breakdown;
        alpha = rho_new / rv;
        for (long i = 0; i < n; i++) s[i] = r[i] - alpha * v[i];
        if (K) K(kctx, s, sh); else memcpy(sh, s, n * sizeof(cplx));
        M(mctx, sh, t);
        if (napply) (*napply)++;
        double tt = vnorm2(n, t);
        if (tt == 0) goto breakdown;
        omega = vdot(n, t, s) / tt;
        for (long i = 0; i < n; i++) {
            x[i] += alpha * ph[i] + omega * sh[i];
            r[i] = s[i] - omega * t[i];
        }
        rho = rho_new;
        k++;
        if (sqrt(vnorm2(n, r)) <= tol * bnorm) { status = 0; break; }
        continue;
    breakdown:
        if (restarted) { status = 2; break; }
        restarted = 1;
        memcpy(rh, r, n * sizeof(cplx));
        memset(p, 0, n * sizeof(cplx));
        memset(v, 0, n * sizeof(cplx));
        rho = alpha = omega = 1;
    }
done:
    if (iters) *iters = k;
    free(r); free(rh); free(p); free(v); free(s); free(t); free(ph); free(sh);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Domain solve (Alg. 1 line 5)                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    const ora_op *op;
    const ora_dd *d;
    const long *gsite;
} dd_ctx;

static void dd_apply_cb(void *ctx, const cplx *in, cplx *out)
{
    dd_ctx *c = ctx;
    dd_apply(c->op, c->d, c->gsite, in, out);
}

/* Minimal residual: v = 0, rho = r; repeat N: q = D rho,
 * alpha = <q, rho> / <q, q>, v += alpha rho, rho -= alpha q. */
static void dd_mr(const ora_op *op, const ora_dd *d, const long *gsite, int niter,
                  const cplx *r, cplx *v)
{
    long n = d->nloc * 12;
    cplx *rho = malloc(n * sizeof(cplx)), *q = malloc(n * sizeof(cplx));
    memcpy(rho, r, n * sizeof(cplx));
    memset(v, 0, n * sizeof(cplx));
    for (int k = 0; k < niter; k++) {
        dd_apply(op, d, gsite, rho, q);
        cplx qr = 0;
        double qq = 0;
        for (long i = 0; i < n; i++) {
            qr += conj(q[i]) * rho[i];
            qq += creal(q[i]) * creal(q[i]) + cimag(q[i]) * cimag(q[i]);
        }
        if (qq == 0) break;
        cplx alpha = qr / qq;
        for (long i = 0; i < n; i++) {
            v[i] += alpha * rho[i];
            rho[i] -= alpha * q[i];
        }
    }
    free(rho);
    free(q);
}

static void dd_solve(const ora_op *op, const ora_dd *d, const long *gsite, const ora_prec *p,
                     const cplx *r, cplx *v)
{
    if (p->dom_solver == 1) {
        dd_ctx c = {op, d, gsite};
        bicgstab(d->nloc * 12, dd_apply_cb, &c, NULL, NULL, r, v, 1e-13, 100000, NULL, NULL);
    } else {
        dd_mr(op, d, gsite, p->n_dominv, r, v);
    }
}

/* Exported for the checks: one domain solve on a local vector. */
int ora_domain_solve(const ora_op *op, const ora_prec *p, int dom, const cplx *r, cplx *v)
{
    ora_dd d;
    if (dd_init(&d, op->L, op->bc, p->block, p->s) || dom < 0 || dom >= d.ndom) return -1;
    long *g = malloc(d.nloc * sizeof(long));
    for (long l = 0; l < d.nloc; l++) {
        int bk;
        g[l] = dd_global(&d, dom, l, &bk);
    }
    dd_solve(op, &d, g, p, r, v);
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* RAS iteration (Alg. 1): phi = K_RAS eta                                    */
/* ------------------------------------------------------------------------ */

/* Colour of a domain in the red/black block ordering: the parity of the sum
 * of its block coordinates. */
static int dd_color(const ora_dd *d, int dom)
{
    int sum = 0, r = dom;
    for (int mu = 0; mu < 4; mu++) {
        sum += r % d->nb[mu];
        r /= d->nb[mu];
    }
    return sum & 1;
}

/* v = sum over the domains i of colour `color` (every domain when color < 0)
 * of the solution of D_i' v_i' = P_i' r (Alg. 1 lines 3-8), restricted to the
 * bulk sites (restrict_bulk = 1: R_i, RAS) or prolonged onto every site of the
 * extended domain with the overlaps summed (restrict_bulk = 0: AS). */
static void dd_sweep(const ora_op *op, const ora_dd *d, const ora_prec *p, int color, int restrict_bulk,
                     const cplx *r, cplx *v)
{
    memset(v, 0, volume(op->L) * 12 * sizeof(cplx));
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < d->ndom; i++) {                 /* line 3 */
        if (color >= 0 && dd_color(d, i) != color) continue;
        long *g = malloc(d->nloc * sizeof(long));
        int *bulk = malloc(d->nloc * sizeof(int));
        cplx *rl = malloc(d->nloc * 12 * sizeof(cplx)), *vl = malloc(d->nloc * 12 * sizeof(cplx));
        for (long l = 0; l < d->nloc; l++) g[l] = dd_global(d, i, l, &bulk[l]);
        /* line 4: projection r_i' = P_i' r */
        for (long l = 0; l < d->nloc; l++) memcpy(rl + l * 12, r + g[l] * 12, 12 * sizeof(cplx));
        /* line 5: solve D_i' v_i' = r_i' with the Dirichlet boundary */
        dd_solve(op, d, g, p, rl, vl);
        /* lines 6 and 8: v_i = R_i v_i', v = sum_i v_i (bulk sites are disjoint);
         * without the restriction the extended domains overlap */
        if (restrict_bulk) {
            for (long l = 0; l < d->nloc; l++)
                if (bulk[l])
                    for (int k = 0; k < 12; k++) v[g[l] * 12 + k] += vl[l * 12 + k];
        } else {
#pragma omp critical(ora_as_sum)
            for (long l = 0; l < d->nloc; l++)
                for (int k = 0; k < 12; k++) v[g[l] * 12 + k] += vl[l * 12 + k];
        }
        free(g); free(bulk); free(rl); free(vl);
    }
}

/* NRAS Schwarz cycles from phi = 0.  RAS (Alg. 1) and AS do one sweep over
 * all domains per cycle; SAP does the red domains, updates the residual, then
 * the black domains.  Every sweep ends with line 9: phi += v, r -= D v. */
int ora_ras(const ora_op *op, const ora_prec *p, const cplx *eta, cplx *phi)
{
    ora_dd d;
    if (dd_init(&d, op->L, op->bc, p->block, p->s)) return -1;
    if (p->schwarz < ORA_RAS || p->schwarz > ORA_AS) return -1;
    long V = volume(op->L), n = V * 12;
    cplx *r = malloc(n * sizeof(cplx)), *v = malloc(n * sizeof(cplx)), *dv = malloc(n * sizeof(cplx));
    const int ncolor = p->schwarz == ORA_SAP ? 2 : 1;

    /* line 1: phi = 0, r = eta */
    memset(phi, 0, n * sizeof(cplx));
    memcpy(r, eta, n * sizeof(cplx));

    for (int j = 0; j < p->n_ras; j++) {               /* line 2 */
        for (int c = 0; c < ncolor; c++) {
            dd_sweep(op, &d, p, p->schwarz == ORA_SAP ? c : -1, p->schwarz != ORA_AS, r, v);
            /* line 9: phi = phi + v, r = r - D v */
            ora_dslash(op, v, dv);
            for (long k = 0; k < n; k++) {
                phi[k] += v[k];
                r[k] -= dv[k];
            }
        }
    }
    free(r); free(v); free(dv);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Solvers                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    const ora_op *op;
    const ora_prec *p;
} glob_ctx;

static void dslash_cb(void *ctx, const cplx *in, cplx *out)
{
    glob_ctx *c = ctx;
    ora_dslash(c->op, in, out);
}

static void ras_cb(void *ctx, const cplx *in, cplx *out)
{
    glob_ctx *c = ctx;
    ora_ras(c->op, c->p, in, out);
}

/* One inner solve of D x = b (right-preconditioned by K_RAS if p->use_ras). */
int ora_bicgstab(const ora_op *op, const ora_prec *p, const cplx *b, cplx *x,
                 double tol, int maxit, int *iters, int *ndv)
{
    glob_ctx c = {op, p};
    long n = volume(op->L) * 12;
    int dv = 0, it = 0;
    int st = bicgstab(n, dslash_cb, &c, p && p->use_ras ? ras_cb : NULL, &c, b, x, tol, maxit, &it, &dv);
    if (iters) *iters = it;
    /* D applications inside the preconditioner: one per sweep (line 9), NRAS
     * sweeps per call (2 NRAS for SAP), two calls per iteration */
    if (ndv) *ndv = dv + (p && p->use_ras ? it * 2 * p->n_ras * (p->schwarz == ORA_SAP ? 2 : 1) : 0);
    return st;
}

/* Outer FP64 defect correction around the inner solve (Sec. 3):
 * phi = 0, r = eta; while |r|/|eta| > tol: e = inner(r/|r|); phi += |r| e;
 * r = eta - D phi.  With inner_tol = tol and no RAS this is the plain
 * BiCGStab, continued from the true residual until it meets tol. */
int ora_solve(const ora_op *op, const ora_prec *p, double inner_tol, int max_inner, int max_outer,
              double tol, const cplx *eta, cplx *phi, ora_info *info)
{
    long n = volume(op->L) * 12;
    cplx *r = malloc(n * sizeof(cplx)), *rs = malloc(n * sizeof(cplx));
    cplx *e = malloc(n * sizeof(cplx)), *dphi = malloc(n * sizeof(cplx));
    double enorm = sqrt(vnorm2(n, eta));
    ora_info inf = {0, 0, 0, 1, 0.0};

    memset(phi, 0, n * sizeof(cplx));
    memcpy(r, eta, n * sizeof(cplx));
    for (;;) {
        double rn = sqrt(vnorm2(n, r));
        inf.true_rel_residual = enorm > 0 ? rn / enorm : 0.0;
        if (inf.true_rel_residual <= tol) { inf.status = 0; break; }
        if (inf.outer_iters >= max_outer) { inf.status = 1; break; }
        for (long k = 0; k < n; k++) rs[k] = r[k] / rn;
        int it = 0, dv = 0;
        int st = ora_bicgstab(op, p, rs, e, inner_tol, max_inner, &it, &dv);
        inf.inner_iters += it;
        inf.dv_count += dv;
        inf.outer_iters++;
        for (long k = 0; k < n; k++) phi[k] += rn * e[k];
        ora_dslash(op, phi, dphi);
        for (long k = 0; k < n; k++) r[k] = eta[k] - dphi[k];
        if (st == 2 && it == 0) { inf.status = 2; break; }
    }
    if (info) *info = inf;
    free(r); free(rs); free(e); free(dphi);
    return inf.status;
}

/* The paper's nested solver (Sec. 3): an FP64 BiCGStab whose preconditioner
 * is the inner solve, M(y) = |y| inner(y / |y|), the inner BiCGStab
 * (right-preconditioned by the Schwarz iteration when p->use_ras) run to
 * inner_tol; M changes from call to call, which makes the outer BiCGStab a
 * flexible one.  One pass solves D e = r from e = 0 until its recursive
 * residual is below 0.5 tol |eta| (the margin covers the gap to the true
 * residual); phi += e, r = eta - D phi, and a further pass starts from the
 * true residual while |r| / |eta| > tol.  outer_iters counts outer BiCGStab
 * iterations over all passes (capped by max_outer). */
static void inner_apply(const ora_op *op, const ora_prec *p, double inner_tol, int max_inner, const cplx *y,
                        cplx *out, cplx *tmp, ora_info *inf)
{
    long n = volume(op->L) * 12;
    double yn = sqrt(vnorm2(n, y));
    if (yn == 0) {
        memset(out, 0, n * sizeof(cplx));
        return;
    }
    for (long k = 0; k < n; k++) tmp[k] = y[k] / yn;
    int it = 0, dv = 0;
    ora_bicgstab(op, p, tmp, out, inner_tol, max_inner, &it, &dv);
    for (long k = 0; k < n; k++) out[k] *= yn;
    inf->inner_iters += it;
    inf->dv_count += dv;
}

int ora_solve_nested(const ora_op *op, const ora_prec *p, double inner_tol, int max_inner, int max_outer,
                     double tol, const cplx *eta, cplx *phi, ora_info *info)
{
    long n = volume(op->L) * 12;
    size_t bytes = n * sizeof(cplx);
    cplx *r = malloc(bytes), *e = malloc(bytes), *rr = malloc(bytes), *rh = malloc(bytes);
    cplx *pp = malloc(bytes), *v = malloc(bytes), *s = malloc(bytes), *t = malloc(bytes);
    cplx *ph = malloc(bytes), *sh = malloc(bytes), *tmp = malloc(bytes);
    double enorm = sqrt(vnorm2(n, eta));
    ora_info inf = {0, 0, 0, 1, 0.0};

    memset(phi, 0, bytes);
    memcpy(r, eta, bytes);
    for (;;) {
        double rn = sqrt(vnorm2(n, r));
        inf.true_rel_residual = enorm > 0 ? rn / enorm : 0.0;
        if (inf.true_rel_residual <= tol) { inf.status = 0; break; }
        if (inf.outer_iters >= max_outer) { inf.status = 1; break; }
        /* one flexible BiCGStab pass on D e = r */
        double stop = 0.5 * tol * enorm;
        memset(e, 0, bytes);
        memcpy(rr, r, bytes);
        memcpy(rh, r, bytes);
        memset(pp, 0, bytes);
        memset(v, 0, bytes);
        cplx rho = 1, alpha = 1, omega = 1;
        int broke = 0;
        while (inf.outer_iters < max_outer) {
            cplx rho1 = vdot(n, rh, rr);
            if (rho1 == 0) { broke = 1; break; }
            cplx beta = (rho1 / rho) * (alpha / omega);
            for (long k = 0; k < n; k++) pp[k] = rr[k] + beta * (pp[k] - omega * v[k]);
            inner_apply(op, p, inner_tol, max_inner, pp, ph, tmp, &inf);
            ora_dslash(op, ph, v);
            cplx rv = vdot(n, rh, v);
            inf.outer_iters++;
            if (rv == 0) { broke = 1; break; }
            alpha = rho1 / rv;
            for (long k = 0; k < n; k++) s[k] = rr[k] - alpha * v[k];
            if (sqrt(vnorm2(n, s)) <= stop) {
                for (long k = 0; k < n; k++) e[k] += alpha * ph[k];
                break;
            }
            inner_apply(op, p, inner_tol, max_inner, s, sh, tmp, &inf);
            ora_dslash(op, sh, t);
            double tt = vnorm2(n, t);
            if (tt == 0) { broke = 1; break; }
            omega = vdot(n, t, s) / tt;
            for (long k = 0; k < n; k++) {
                e[k] += alpha * ph[k] + omega * sh[k];
                rr[k] = s[k] - omega * t[k];
            }
            rho = rho1;
            if (sqrt(vnorm2(n, rr)) <= stop) break;
        }
        for (long k = 0; k < n; k++) phi[k] += e[k];
        ora_dslash(op, phi, t);
        for (long k = 0; k < n; k++) r[k] = eta[k] - t[k];
        if (broke && inf.outer_iters == 0) { inf.status = 2; break; }
    }
    if (info) *info = inf;
    free(r); free(e); free(rr); free(rh); free(pp); free(v); free(s); free(t); free(ph); free(sh); free(tmp);
    return inf.status;
}

/* |eta - D phi| / |eta| with the oracle's D (the contract every solve meets). */
double ora_true_residual(const ora_op *op, const cplx *eta, const cplx *phi)
{
    long n = volume(op->L) * 12;
    cplx *d = malloc(n * sizeof(cplx));
    ora_dslash(op, phi, d);
    double num = 0, den = 0;
    for (long k = 0; k < n; k++) {
        cplx t = eta[k] - d[k];
        num += creal(t) * creal(t) + cimag(t) * cimag(t);
        den += creal(eta[k]) * creal(eta[k]) + cimag(eta[k]) * cimag(eta[k]);
    }
    free(d);
    return den > 0 ? sqrt(num / den) : sqrt(num);
}

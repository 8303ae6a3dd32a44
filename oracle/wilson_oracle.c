/*
 * Plain FP64 CPU oracle for the Wilson / twisted-mass Wilson fermion matrix,
 * its even-odd (Schur) form, and CG inversion.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this code.  It shares nothing with the
 * CUDA library: it has its own gamma matrices, indexing and solver, written
 * straight from the definitions, with no blocking, fusion or reordering.
 *
 * Paper: CL2QCD, arXiv:1411.5219.  Sec. 1 defines the task: the fermion
 * matrix D is inverted, D phi = psi, with a Krylov method such as CG, and the
 * hopping ("Dslash") part of the Wilson D is the hot operation.  Sec. 3 names
 * the Wilson and twisted-mass Wilson discretisations.  Sec. 4 states that all
 * arithmetic is double precision.  The paper gives no formulas for D; the
 * conventions below are the standard ones, chosen where the paper is silent:
 *
 *   D_hop psi(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                         + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
 *   M = A - kappa D_hop,  A = 1 + i a gamma_5,  a = 2 kappa mu_tm
 *
 * gamma matrices in the chiral basis (Hermitian):
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1,2,3 <-> x,y,z)
 *   gamma_4 = [[0, 1], [1, 0]]                   (t)
 *   gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4   (= diag(1,1,-1,-1))
 *
 * Boundary conditions: periodic in x, y, z; in t the hop that wraps around
 * the lattice is multiplied by t_bc (+1 periodic, -1 antiperiodic).
 *
 * Site index lex = x + Lx*(y + Ly*(z + Lz*t)); parity p = (x+y+z+t) mod 2;
 * a parity-compacted half field stores site lex at index lex/2.
 *
 * Field layouts (complex doubles, interleaved re/im):
 *   gauge  U[lex][mu][a][b]   spinor psi[lex][s][c]   half  h[lex/2][s][c]
 *
 * Parity of every function here is pinned by tests against values that do
 * not come from this file: the free-field momentum-space closed form, the
 * constant-field closed form, gamma_5-hermiticity, gauge covariance, dense
 * inversion with numpy at 2^4, and an FFT solution of the free-field system.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* gamma matrices                                                       */
/* ------------------------------------------------------------------ */

static cplx GAMMA[5][4][4]; /* 0..3 = x,y,z,t ; 4 = gamma_5 */
static int gamma_ready = 0;

static void init_gamma(void)
{
    if (gamma_ready) return;
    cplx sigma[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(GAMMA, 0, sizeof(GAMMA));
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                GAMMA[k][a][2 + b] = -I * sigma[k][a][b];
                GAMMA[k][2 + a][b] = I * sigma[k][a][b];
            }
    for (int a = 0; a < 2; ++a) {
        GAMMA[3][a][2 + a] = 1;
        GAMMA[3][2 + a][a] = 1;
    }
    /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4, by plain matrix products */
    cplx t1[4][4], t2[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += GAMMA[0][i][k] * GAMMA[1][k][j];
            t1[i][j] = s;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += t1[i][k] * GAMMA[2][k][j];
            t2[i][j] = s;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += t2[i][k] * GAMMA[3][k][j];
            GAMMA[4][i][j] = s;
        }
    gamma_ready = 1;
}

/* Copy gamma matrix mu (0..3 = x,y,z,t; 4 = gamma_5) into out[4][4]. */
void oracle_gamma(int mu, double *out)
{
    init_gamma();
    memcpy(out, GAMMA[mu], sizeof(GAMMA[mu]));
}

/* ------------------------------------------------------------------ */
/* lattice geometry                                                     */
/* ------------------------------------------------------------------ */

typedef struct {
    int L[4];
    long V;
    double t_bc;
} lattice;

static lattice make_lattice(const int *dims, double t_bc)
{
    lattice g;
    g.V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.L[mu] = dims[mu];
        g.V *= dims[mu];
    }
    g.t_bc = t_bc;
    return g;
}

static void coords(const lattice *g, long lex, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(lex % g->L[mu]);
        lex /= g->L[mu];
    }
}

static long lex_of(const lattice *g, const int c[4])
{
    return c[0] + (long)g->L[0] * (c[1] + (long)g->L[1] * (c[2] + (long)g->L[2] * c[3]));
}

/* Neighbour of site lex in direction mu, step dir = +1 or -1; *sign is the
 * boundary factor of that hop (t_bc if it wraps in t, else 1). */
static long neighbour(const lattice *g, long lex, int mu, int dir, double *sign)
{
    int c[4];
    coords(g, lex, c);
    int v = c[mu] + dir;
    *sign = 1.0;
    if (v == g->L[mu]) {
        v = 0;
        if (mu == 3) *sign = g->t_bc;
    } else if (v < 0) {
        v = g->L[mu] - 1;
        if (mu == 3) *sign = g->t_bc;
    }
    c[mu] = v;
    return lex_of(g, c);
}

static int parity_of(const lattice *g, long lex)
{
    int c[4];
    coords(g, lex, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* ------------------------------------------------------------------ */
/* the hopping term                                                     */
/* ------------------------------------------------------------------ */

typedef cplx spinor[4][3];
typedef cplx su3[3][3];

static const su3 *link(const cplx *U, long lex, int mu)
{
    return (const su3 *)(U + (lex * 4 + mu) * 9);
}

/* res = (D_hop psi)(x) (dagger = 0) or (D_hop^dagger psi)(x) (dagger = 1)
 * at the single site x.  The adjoint swaps the spin projectors: (1 +
 * gamma_mu) forward, (1 - gamma_mu) backward. */
static void dhop_site(const lattice *g, const cplx *U, const spinor *psi, long x, int dagger, spinor res)
{
    const double sg = dagger ? -1.0 : 1.0;
    spinor acc;
    memset(acc, 0, sizeof(acc));
    for (int mu = 0; mu < 4; ++mu) {
        for (int dir = +1; dir >= -1; dir -= 2) {
            double bsign;
            long y = neighbour(g, x, mu, dir, &bsign);
            /* colour part: U_mu(x) psi(x+mu)  or  U_mu(x-mu)^dagger psi(x-mu) */
            spinor chi;
            const su3 *u = dir > 0 ? link(U, x, mu) : link(U, y, mu);
            for (int s = 0; s < 4; ++s)
                for (int a = 0; a < 3; ++a) {
                    cplx v = 0;
                    for (int b = 0; b < 3; ++b) {
                        if (dir > 0)
                            v += (*u)[a][b] * psi[y][s][b];
                        else
                            v += conj((*u)[b][a]) * psi[y][s][b];
                    }
                    chi[s][a] = v;
                }
            /* spin part: (1 - dir*sg*gamma_mu) chi */
            const double gs = -dir * sg;
            for (int s = 0; s < 4; ++s)
                for (int a = 0; a < 3; ++a) {
                    cplx gchi = 0;
                    for (int t = 0; t < 4; ++t) gchi += GAMMA[mu][s][t] * chi[t][a];
                    acc[s][a] += bsign * (chi[s][a] + gs * gchi);
                }
        }
    }
    memcpy(res, acc, sizeof(acc));
}

/* out = D_hop psi (or D_hop^dagger psi) at every site. */
static void dhop(const lattice *g, const cplx *U, const cplx *in, cplx *out, int dagger)
{
    init_gamma();
    const spinor *psi = (const spinor *)in;
    spinor *res = (spinor *)out;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < g->V; ++x) dhop_site(g, U, psi, x, dagger, res[x]);
}

/* out = (1 + i b gamma_5) in, or its inverse (1 - i b gamma_5)/(1 + b^2)
 * (gamma_5^2 = 1), over n sites. */
static void twist(const cplx *in, cplx *out, long n, double b, int inverse)
{
    init_gamma();
    const spinor *psi = (const spinor *)in;
    spinor *res = (spinor *)out;
    const double bb = inverse ? -b : b;
    const double norm = inverse ? 1.0 / (1.0 + b * b) : 1.0;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < n; ++x) {
        spinor tmp;
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a) {
                cplx g5 = 0;
                for (int t = 0; t < 4; ++t) g5 += GAMMA[4][s][t] * psi[x][t][a];
                tmp[s][a] = norm * (psi[x][s][a] + I * bb * g5);
            }
        memcpy(res[x], tmp, sizeof(tmp));
    }
}

/* ------------------------------------------------------------------ */
/* vector algebra (serial reductions: fixed order, deterministic)       */
/* ------------------------------------------------------------------ */

static cplx dot(const cplx *a, const cplx *b, long n)
{
    cplx s = 0;
    for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

static double norm2(const cplx *a, long n)
{
    double s = 0;
    for (long i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* ------------------------------------------------------------------ */
/* full-lattice operators                                               */
/* ------------------------------------------------------------------ */

/* out = M psi = A psi - kappa D_hop psi, or M^dagger psi = A^dagger psi -
 * kappa D_hop^dagger psi, with A = 1 + i (2 kappa mu) gamma_5. */
static void apply_m(const lattice *g, const cplx *U, double kappa, double mu,
                    const cplx *in, cplx *out, int dagger)
{
    const long n = g->V * 12;
    cplx *d = malloc(sizeof(cplx) * n);
    dhop(g, U, in, d, dagger);
    const double a = 2.0 * kappa * mu;
    twist(in, out, g->V, dagger ? -a : a, 0);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) out[i] -= kappa * d[i];
    free(d);
}

/* ------------------------------------------------------------------ */
/* even-odd blocks, by restriction of the full hopping term             */
/* ------------------------------------------------------------------ */

/* Full field with the half field `half` on the sites of parity p, zero on
 * the others. */
static void embed(const lattice *g, const cplx *half, int p, cplx *full)
{
    memset(full, 0, sizeof(cplx) * g->V * 12);
    for (long x = 0; x < g->V; ++x)
        if (parity_of(g, x) == p) memcpy(full + x * 12, half + (x / 2) * 12, sizeof(cplx) * 12);
}

static void extract(const lattice *g, const cplx *full, int p, cplx *half)
{
    for (long x = 0; x < g->V; ++x)
        if (parity_of(g, x) == p) memcpy(half + (x / 2) * 12, full + x * 12, sizeof(cplx) * 12);
}

/* out (parity p) = [D_hop]_{p, 1-p} in (parity 1-p): D_eo for p = 0, D_oe
 * for p = 1; with dagger the same block of D_hop^dagger. */
static void dhop_block(const lattice *g, const cplx *U, int p, const cplx *in, cplx *out, int dagger)
{
    const long n = g->V * 12;
    cplx *f = malloc(sizeof(cplx) * n);
    cplx *d = malloc(sizeof(cplx) * n);
    embed(g, in, 1 - p, f);
    dhop(g, U, f, d, dagger);
    extract(g, d, p, out);
    free(f);
    free(d);
}

/* Schur complement on the even sites,
 *   Mhat = A - kappa^2 D_eo A^-1 D_oe,
 * and its adjoint Mhat^dagger = A^dagger - kappa^2 (D^dagger)_eo
 * (A^dagger)^-1 (D^dagger)_oe, with A^-1 = (1 - i a gamma_5)/(1 + a^2). */
static void apply_mhat(const lattice *g, const cplx *U, double kappa, double mu,
                       const cplx *in, cplx *out, int dagger)
{
    const long h = g->V / 2, n = h * 12;
    const double a = dagger ? -2.0 * kappa * mu : 2.0 * kappa * mu;
    cplx *t = malloc(sizeof(cplx) * n);
    cplx *u = malloc(sizeof(cplx) * n);
    dhop_block(g, U, 1, in, t, dagger); /* odd  <- even */
    twist(t, t, h, a, 1);               /* A^-1 on odd  */
    dhop_block(g, U, 0, t, u, dagger);  /* even <- odd  */
    twist(in, out, h, a, 0);            /* A on even    */
    for (long i = 0; i < n; ++i) out[i] -= kappa * kappa * u[i];
    free(t);
    free(u);
}

/* ------------------------------------------------------------------ */
/* conjugate gradient                                                   */
/* ------------------------------------------------------------------ */

typedef void (*linop)(const void *ctx, const cplx *in, cplx *out);

/* Hestenes-Stiefel CG for a Hermitian positive definite operator A:
 * x0 = 0, r = p = b; alpha = <r,r>/<p,Ap>; x += alpha p; r -= alpha Ap;
 * beta = <r',r'>/<r,r>; p = r' + beta p; stop when |r|/|b| <= tol.
 * Returns the iteration count (or -1 if maxiter was reached). */
static int cg(linop A, const void *ctx, const cplx *b, cplx *x, long n,
              double tol, int maxiter)
{
    cplx *r = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n);
    cplx *q = malloc(sizeof(cplx) * n);
    memset(x, 0, sizeof(cplx) * n);
    memcpy(r, b, sizeof(cplx) * n);
    memcpy(p, b, sizeof(cplx) * n);
    const double bb = norm2(b, n);
    double rr = bb;
    int k = 0, converged = (bb == 0.0);
    while (!converged && k < maxiter) {
        A(ctx, p, q);
        const double pq = creal(dot(p, q, n));
        const double alpha = rr / pq;
        for (long i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        const double rr_new = norm2(r, n);
        ++k;
        if (sqrt(rr_new / bb) <= tol) {
            converged = 1;
            break;
        }
        const double beta = rr_new / rr;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
    free(r);
    free(p);
    free(q);
    return converged ? k : -1;
}

typedef struct {
    lattice g;
    const cplx *U;
    double kappa, mu;
    cplx *tmp;
} opctx;

static void op_mdagm(const void *vctx, const cplx *in, cplx *out)
{
    const opctx *c = vctx;
    apply_m(&c->g, c->U, c->kappa, c->mu, in, c->tmp, 0);
    apply_m(&c->g, c->U, c->kappa, c->mu, c->tmp, out, 1);
}

static void op_mhatdagmhat(const void *vctx, const cplx *in, cplx *out)
{
    const opctx *c = vctx;
    apply_mhat(&c->g, c->U, c->kappa, c->mu, in, c->tmp, 0);
    apply_mhat(&c->g, c->U, c->kappa, c->mu, c->tmp, out, 1);
}

/* ------------------------------------------------------------------ */
/* exported entry points (pointers to interleaved complex doubles)      */
/* ------------------------------------------------------------------ */

void oracle_dhop(const int *dims, double t_bc, const double *U, const double *in,
                 double *out, int dagger)
{
    lattice g = make_lattice(dims, t_bc);
    dhop(&g, (const cplx *)U, (const cplx *)in, (cplx *)out, dagger);
}

void oracle_apply_m(const int *dims, double t_bc, const double *U, double kappa, double mu,
                    const double *in, double *out, int dagger)
{
    lattice g = make_lattice(dims, t_bc);
    apply_m(&g, (const cplx *)U, kappa, mu, (const cplx *)in, (cplx *)out, dagger);
}

void oracle_dhop_eo(const int *dims, double t_bc, const double *U, int out_parity,
                    const double *in, double *out, int dagger)
{
    lattice g = make_lattice(dims, t_bc);
    dhop_block(&g, (const cplx *)U, out_parity, (const cplx *)in, (cplx *)out, dagger);
}

void oracle_apply_mhat(const int *dims, double t_bc, const double *U, double kappa, double mu,
                       const double *in, double *out, int dagger)
{
    lattice g = make_lattice(dims, t_bc);
    apply_mhat(&g, (const cplx *)U, kappa, mu, (const cplx *)in, (cplx *)out, dagger);
}

/* D_hop psi (or its adjoint) at the n lexicographic sites listed in
 * `sites`, from a full input field; out holds n spinors. */
void oracle_dhop_sites(const int *dims, double t_bc, const double *U, const double *in, const long *sites,
                       long n, double *out, int dagger)
{
    lattice g = make_lattice(dims, t_bc);
    init_gamma();
    spinor *res = (spinor *)out;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) dhop_site(&g, (const cplx *)U, (const spinor *)in, sites[k], dagger, res[k]);
}

/* ------------------------------------------------------------------ */
/* staggered (Kogut-Susskind) hopping term                              */
/* ------------------------------------------------------------------ */

/* The paper's second Dirac operator (Sec. 1, Sec. 6): the staggered
 * derivative on one-component colour vectors,
 *   (D_KS chi)(x) = sum_mu eta_mu(x) [ U_mu(x) chi(x+mu) - U_mu(x-mu)^dagger chi(x-mu) ],
 * eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z),
 * with the same boundary factor t_bc on hops that wrap in time.  No factor
 * 1/2: this form performs the 570 flop per site the paper counts (8 SU(3)
 * matrix-vector products and 7 vector sums). */
typedef cplx colour[3];

static double eta(const int c[4], int mu)
{
    int s = 0;
    for (int nu = 0; nu < mu; ++nu) s += c[nu];
    return (s & 1) ? -1.0 : 1.0;
}

static void dks_site(const lattice *g, const cplx *U, const colour *chi, long x, colour res)
{
    int c[4];
    coords(g, x, c);
    colour acc = {0, 0, 0};
    for (int mu = 0; mu < 4; ++mu) {
        const double e = eta(c, mu);
        double bf, bb;
        const long yf = neighbour(g, x, mu, +1, &bf);
        const long yb = neighbour(g, x, mu, -1, &bb);
        const su3 *uf = link(U, x, mu), *ub = link(U, yb, mu);
        for (int a = 0; a < 3; ++a) {
            cplx vf = 0, vb = 0;
            for (int b = 0; b < 3; ++b) {
                vf += (*uf)[a][b] * chi[yf][b];
                vb += conj((*ub)[b][a]) * chi[yb][b];
            }
            acc[a] += e * (bf * vf - bb * vb);
        }
    }
    memcpy(res, acc, sizeof(acc));
}

/* out = D_KS in on the full lattice (3 complex per site). */
void oracle_dks(const int *dims, double t_bc, const double *U, const double *in, double *out)
{
    lattice g = make_lattice(dims, t_bc);
    colour *res = (colour *)out;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < g.V; ++x) dks_site(&g, (const cplx *)U, (const colour *)in, x, res[x]);
}

/* (1 + i b gamma_5) or its inverse on n sites of 12 complex components. */
void oracle_twist(const double *in, double *out, long n, double b, int inverse)
{
    twist((const cplx *)in, (cplx *)out, n, b, inverse);
}

/* Solve M^dagger M x = b on the full lattice by CG.  stats[0] = iterations
 * (-1: not converged), stats[1] = |b - M^dagger M x| / |b|. */
void oracle_solve_mdagm(const int *dims, double t_bc, const double *U, double kappa, double mu,
                        const double *b, double *x, double tol, int maxiter, double *stats)
{
    opctx c = {make_lattice(dims, t_bc), (const cplx *)U, kappa, mu, NULL};
    const long n = c.g.V * 12;
    c.tmp = malloc(sizeof(cplx) * n);
    int it = cg(op_mdagm, &c, (const cplx *)b, (cplx *)x, n, tol, maxiter);
    cplx *r = malloc(sizeof(cplx) * n);
    op_mdagm(&c, (const cplx *)x, r);
    for (long i = 0; i < n; ++i) r[i] = ((const cplx *)b)[i] - r[i];
    stats[0] = it;
    stats[1] = sqrt(norm2(r, n) / norm2((const cplx *)b, n));
    free(r);
    free(c.tmp);
}

/* Solve M x = b on the full lattice by CG on the normal equations
 * M^dagger M x = M^dagger b (CGNR).  stats[0] = iterations, stats[1] =
 * |b - M x| / |b|. */
void oracle_solve_m(const int *dims, double t_bc, const double *U, double kappa, double mu,
                    const double *b, double *x, double tol, int maxiter, double *stats)
{
    opctx c = {make_lattice(dims, t_bc), (const cplx *)U, kappa, mu, NULL};
    const long n = c.g.V * 12;
    c.tmp = malloc(sizeof(cplx) * n);
    cplx *mb = malloc(sizeof(cplx) * n);
    apply_m(&c.g, c.U, kappa, mu, (const cplx *)b, mb, 1);
    int it = cg(op_mdagm, &c, mb, (cplx *)x, n, tol, maxiter);
    apply_m(&c.g, c.U, kappa, mu, (const cplx *)x, mb, 0);
    for (long i = 0; i < n; ++i) mb[i] = ((const cplx *)b)[i] - mb[i];
    stats[0] = it;
    stats[1] = sqrt(norm2(mb, n) / norm2((const cplx *)b, n));
    free(mb);
    free(c.tmp);
}

/* Solve M x = b through the even-odd Schur complement:
 *   b'_e = b_e + kappa D_eo A^-1 b_o,
 *   Mhat^dagger Mhat x_e = Mhat^dagger b'_e    (CG),
 *   x_o  = A^-1 (b_o + kappa D_oe x_e).
 * b and x are full fields.  stats[0] = iterations, stats[1] =
 * |Mhat^dagger b' - Mhat^dagger Mhat x_e| / |Mhat^dagger b'|, stats[2] =
 * |b - M x| / |b|. */
void oracle_solve_eo(const int *dims, double t_bc, const double *U, double kappa, double mu,
                     const double *b, double *x, double tol, int maxiter, double *stats)
{
    opctx c = {make_lattice(dims, t_bc), (const cplx *)U, kappa, mu, NULL};
    const lattice *g = &c.g;
    const long h = g->V / 2, n = h * 12;
    const double a = 2.0 * kappa * mu;
    c.tmp = malloc(sizeof(cplx) * n);
    cplx *be = malloc(sizeof(cplx) * n), *bo = malloc(sizeof(cplx) * n);
    cplx *t = malloc(sizeof(cplx) * n), *rhs = malloc(sizeof(cplx) * n);
    cplx *xe = malloc(sizeof(cplx) * n), *xo = malloc(sizeof(cplx) * n);
    extract(g, (const cplx *)b, 0, be);
    extract(g, (const cplx *)b, 1, bo);
    /* source preparation */
    twist(bo, t, h, a, 1);
    dhop_block(g, c.U, 0, t, rhs, 0);
    for (long i = 0; i < n; ++i) be[i] += kappa * rhs[i];
    apply_mhat(g, c.U, kappa, mu, be, rhs, 1);
    int it = cg(op_mhatdagmhat, &c, rhs, xe, n, tol, maxiter);
    /* Schur residual */
    op_mhatdagmhat(&c, xe, t);
    for (long i = 0; i < n; ++i) t[i] = rhs[i] - t[i];
    stats[0] = it;
    stats[1] = sqrt(norm2(t, n) / norm2(rhs, n));
    /* odd-site reconstruction */
    dhop_block(g, c.U, 1, xe, t, 0);
    for (long i = 0; i < n; ++i) t[i] = bo[i] + kappa * t[i];
    twist(t, xo, h, a, 1);
    /* assemble x and the full-system residual */
    cplx *xf = (cplx *)x;
    memset(xf, 0, sizeof(cplx) * g->V * 12);
    for (long s = 0; s < g->V; ++s)
        memcpy(xf + s * 12, (parity_of(g, s) ? xo : xe) + (s / 2) * 12, sizeof(cplx) * 12);
    cplx *mx = malloc(sizeof(cplx) * g->V * 12);
    apply_m(g, c.U, kappa, mu, xf, mx, 0);
    for (long i = 0; i < g->V * 12; ++i) mx[i] = ((const cplx *)b)[i] - mx[i];
    stats[2] = sqrt(norm2(mx, g->V * 12) / norm2((const cplx *)b, g->V * 12));
    free(mx);
    free(be);
    free(bo);
    free(t);
    free(rhs);
    free(xe);
    free(xo);
    free(c.tmp);
}

/* Run `iters` CG iterations of the even-odd system (the same steps as
 * oracle_solve_eo, stopped early) and return nothing: a bounded sample of
 * the solve, used to time the oracle on the host cores. */
void oracle_cg_eo_sample(const int *dims, double t_bc, const double *U, double kappa, double mu,
                         const double *b_even, double *x_even, int iters)
{
    opctx c = {make_lattice(dims, t_bc), (const cplx *)U, kappa, mu, NULL};
    const long n = c.g.V / 2 * 12;
    c.tmp = malloc(sizeof(cplx) * n);
    cg(op_mhatdagmhat, &c, (const cplx *)b_even, (cplx *)x_even, n, 0.0, iters);
    free(c.tmp);
}

void oracle_set_threads(int n);
#ifdef _OPENMP
#include <omp.h>
void oracle_set_threads(int n) { omp_set_num_threads(n); }
int oracle_get_threads(void) { return omp_get_max_threads(); }
#else
void oracle_set_threads(int n) { (void)n; }
int oracle_get_threads(void) { return 1; }
#endif

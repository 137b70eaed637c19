/*
 * gf_oracle.c -- plain FP64 CPU oracle for SU(3) Landau / Coulomb gauge fixing by
 * checkerboard overrelaxation, after N. Cardoso, "Coulomb and Landau Gauge Fixing in
 * GPUs using CUDA and MILC" (Lattice 2014), Section 1, Eqs. (1)-(6) and Algorithm 1.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  The CUDA product path never calls it, and
 * the two share no code, headers, tables or helpers.
 *
 * It is written to be checked against the paper by eye: one site at a time, in the
 * order the paper states, with no blocking or fusion.  The only parallelism is an
 * OpenMP loop over the sites of one checkerboard parity; sites of one parity share no
 * link, so that loop gives the same bits for any thread count.
 *
 * Field layout (the canonical layout of the whole project): complex128 array of shape
 * (Lt, Lz, Ly, Lx, 4, 3, 3); site s = x + Lx*(y + Ly*(z + Lz*t)); link U_mu(s) at
 * U + (4*s + mu)*9, row-major 3x3.  Direction mu = 0,1,2,3 is x,y,z,t (time is mu = 3,
 * Section 1 below Eq. (3)).  Boundary conditions are periodic in all four directions.
 *
 * Readings of the paper used here, each with the reason for it:
 *  - nd = 4 directions enter K, F and Delta for Landau gauge, nd = 3 for Coulomb gauge
 *    (Coulomb gauge leaves out the time direction, Section 1 after Eq. (3)).  F is
 *    normalised by 1/(nd*Nc*V): Eq. (1) prints 1/(4 Nc V) for both gauges, and with nd
 *    in its place the unit field has F = 1 in either gauge.
 *  - Delta(x) of Eq. (3), literally: A = sum_nu [U_nu(x-nu) - U_nu(x)],
 *    Delta = A - A^dagger - (1/Nc) Tr(A - A^dagger) * 1 (the printed "- h.c. - trace",
 *    with no extra factor: the same expression is the argument of Eq. (7)).
 *  - K(x) of Eq. (5) in its in-place form: the stored neighbour links already carry
 *    their own g, so K = sum_{mu<nd} U_mu(x) + U_mu(x-mu)^dagger.
 *  - the SU(3) update is the product of the SU(2)-subgroup maximisers for the index
 *    pairs (0,1), (0,2), (1,2), each computed from the K already rotated by the
 *    previous ones (Section 1, sentence after Eq. (6), which prints only the SU(2)
 *    solution and says to iterate over the subgroups for N > 2).
 *  - overrelaxation g -> g^omega (Mandula-Ogilvie, cited after Eq. (6)) per subgroup,
 *    either to first order (a' = 1 - omega + omega*a, b' = omega*b, renormalised; the
 *    paper gives no formula, and this is the form that needs no trigonometry) or
 *    exactly (the SU(2) power); both are the plain maximiser at omega = 1.
 *  - Coulomb gauge: the temporal links are transformed with the spatial ones (Algorithm
 *    1 applies g(x) to the links of every direction) but enter neither K nor F nor
 *    Delta (the Coulomb condition involves the spatial directions only).
 *  - reunitarisation (Section 3: every 20 steps; the method is not stated) projects each
 *    link back to SU(3) by Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1); it
 *    is applied to the links the odd half-sweep has just written, which is every link
 *    when all sites are active.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define NC 3

typedef struct {
    int L[4];   /* Lx, Ly, Lz, Lt */
    long V;     /* Lx*Ly*Lz*Lt */
    long V3;    /* Lx*Ly*Lz */
} geom;

static int geom_init(geom *g, const int L[4])
{
    g->V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (L[mu] < 2 || (L[mu] % 2) != 0) return -1;
        g->L[mu] = L[mu];
        g->V *= L[mu];
    }
    g->V3 = (long)L[0] * L[1] * L[2];
    return 0;
}

static void coords(const geom *g, long s, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(s % g->L[mu]);
        s /= g->L[mu];
    }
}

static long index_of(const geom *g, const int c[4])
{
    return c[0] + (long)g->L[0] * (c[1] + (long)g->L[1] * (c[2] + (long)g->L[2] * c[3]));
}

/* site x + dir*mu_hat, periodic; dir is +1 or -1 */
static long neighbour(const geom *g, long s, int mu, int dir)
{
    int c[4];
    coords(g, s, c);
    c[mu] = (c[mu] + dir + g->L[mu]) % g->L[mu];
    return index_of(g, c);
}

static int parity_of(const geom *g, long s)
{
    int c[4];
    coords(g, s, c);
    return (c[0] + c[1] + c[2] + c[3]) % 2;
}

static cplx *link_at(cplx *U, long s, int mu) { return U + (4 * s + mu) * 9; }
static const cplx *clink_at(const cplx *U, long s, int mu) { return U + (4 * s + mu) * 9; }

/* C = A * B */
static void mat_mul(const cplx *A, const cplx *B, cplx *C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = acc;
        }
}

/* C = A * B^dagger */
static void mat_mul_dag(const cplx *A, const cplx *B, cplx *C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * conj(B[3 * j + k]);
            C[3 * i + j] = acc;
        }
}

/* ---------------------------------------------------------------------------------
 * Eqs. (1)-(3): F and theta.
 * --------------------------------------------------------------------------------- */

/* Delta(x) of Eq. (3), literal reading, nd directions. */
static void delta_at(const cplx *U, const geom *g, long s, int nd, cplx D[9])
{
    cplx A[9];
    for (int e = 0; e < 9; ++e) A[e] = 0;
    for (int nu = 0; nu < nd; ++nu) {
        const cplx *b = clink_at(U, neighbour(g, s, nu, -1), nu); /* U_nu(x - nu) */
        const cplx *f = clink_at(U, s, nu);                       /* U_nu(x)      */
        for (int e = 0; e < 9; ++e) A[e] = A[e] + (b[e] - f[e]);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[3 * i + j] = A[3 * i + j] - conj(A[3 * j + i]);
    cplx sum = D[0] + D[4] + D[8];
    cplx tr = CMPLX(creal(sum) / 3.0, cimag(sum) / 3.0);
    D[0] -= tr;
    D[4] -= tr;
    D[8] -= tr;
}

/* Neumaier compensated sum: deterministic and accurate on every platform. */
typedef struct { double s, c; } csum;
static void csum_add(csum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double csum_value(const csum *a) { return a->s + a->c; }

/*
 * F (Eq. 1 with the in-place links, so g = 1) and theta (Eq. 2) over the lattice,
 * and per time slice t: F_t = sum_{x in t} sum_{mu<nd} Re Tr U_mu(x) / (nd Nc V3),
 * theta_t = sum_{x in t} Tr[Delta Delta^dagger] / (Nc V3).  F_t / theta_t may be NULL.
 */
int orc_measure(const cplx *U, const int L[4], int nd, double *F, double *theta,
                double *F_t, double *theta_t)
{
    geom g;
    if (geom_init(&g, L) != 0 || (nd != 3 && nd != 4)) return -1;
    int Lt = g.L[3];
    double *fs = malloc(sizeof(double) * Lt), *ts = malloc(sizeof(double) * Lt);
    if (!fs || !ts) { free(fs); free(ts); return -2; }
#pragma omp parallel for schedule(static)
    for (int t = 0; t < Lt; ++t) {
        csum f = {0, 0}, th = {0, 0};
        for (long s = t * g.V3; s < (t + 1) * g.V3; ++s) {
            for (int mu = 0; mu < nd; ++mu) {
                const cplx *u = clink_at(U, s, mu);
                csum_add(&f, creal(u[0]) + creal(u[4]) + creal(u[8]));
            }
            cplx D[9];
            delta_at(U, &g, s, nd, D);
            double q = 0;
            for (int e = 0; e < 9; ++e) q += creal(D[e]) * creal(D[e]) + cimag(D[e]) * cimag(D[e]);
            csum_add(&th, q);
        }
        fs[t] = csum_value(&f);
        ts[t] = csum_value(&th);
    }
    csum fa = {0, 0}, ta = {0, 0};
    for (int t = 0; t < Lt; ++t) {
        csum_add(&fa, fs[t]);
        csum_add(&ta, ts[t]);
        if (F_t) F_t[t] = fs[t] / ((double)nd * NC * g.V3);
        if (theta_t) theta_t[t] = ts[t] / ((double)NC * g.V3);
    }
    *F = csum_value(&fa) / ((double)nd * NC * g.V);
    *theta = csum_value(&ta) / ((double)NC * g.V);
    free(fs);
    free(ts);
    return 0;
}

/* Delta(x) at every site, out has shape (V, 3, 3). */
int orc_delta(const cplx *U, const int L[4], int nd, cplx *out)
{
    geom g;
    if (geom_init(&g, L) != 0 || (nd != 3 && nd != 4)) return -1;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; ++s) delta_at(U, &g, s, nd, out + 9 * s);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Eqs. (4)-(6): the local maximisation in one SU(2) subgroup, with overrelaxation.
 * --------------------------------------------------------------------------------- */

#define OR_FIRST_ORDER 0
#define OR_EXACT 1

/*
 * Maximise Re Tr[R K] over R in the SU(2) subgroup acting on rows/columns (i, j):
 * R restricted to (i, j) is [[a, b], [-conj(b), conj(a)]] with |a|^2 + |b|^2 = 1,
 * and Re Tr[R K] = const + Re(a*alpha) + Re(b*beta) with
 *   alpha = K_ii + conj(K_jj),  beta = K_ji - conj(K_ij).
 * The maximiser is a = conj(alpha)/n, b = conj(beta)/n, n = |(alpha, beta)|; for n = 0
 * every R is a maximiser and R = 1 is taken.  Then R -> R^omega.
 */
void orc_su2_maximiser(const cplx K[9], int i, int j, double omega, int form, cplx *a_out,
                       cplx *b_out)
{
    cplx alpha = K[3 * i + i] + conj(K[3 * j + j]);
    cplx beta = K[3 * j + i] - conj(K[3 * i + j]);
    double n = sqrt(creal(alpha) * creal(alpha) + cimag(alpha) * cimag(alpha) +
                    creal(beta) * creal(beta) + cimag(beta) * cimag(beta));
    cplx a = 1, b = 0;
    if (n > 0) {
        a = CMPLX(creal(alpha) / n, -cimag(alpha) / n);
        b = CMPLX(creal(beta) / n, -cimag(beta) / n);
    }
    if (form == OR_FIRST_ORDER) {
        /* g^omega to first order: 1 + omega (g - 1), then back onto SU(2) */
        cplx a1 = CMPLX(1.0 - omega + omega * creal(a), omega * cimag(a));
        cplx b1 = CMPLX(omega * creal(b), omega * cimag(b));
        double m = sqrt(creal(a1) * creal(a1) + cimag(a1) * cimag(a1) +
                        creal(b1) * creal(b1) + cimag(b1) * cimag(b1));
        if (m > 0) {
            a = CMPLX(creal(a1) / m, cimag(a1) / m);
            b = CMPLX(creal(b1) / m, cimag(b1) / m);
        }
    } else {
        /* exact power: R = cos(phi) + i sin(phi) n.sigma,  R^omega = cos(omega phi) + ... */
        double s = sqrt(cimag(a) * cimag(a) + creal(b) * creal(b) + cimag(b) * cimag(b));
        if (s > 0) {
            double phi = atan2(s, creal(a));
            double c1 = cos(omega * phi), s1 = sin(omega * phi);
            a = CMPLX(c1, (cimag(a) / s) * s1);
            b = CMPLX((creal(b) / s) * s1, (cimag(b) / s) * s1);
        }
    }
    *a_out = a;
    *b_out = b;
}

/* M <- R M for R the subgroup element on rows (i, j) */
static void su2_left_mul(cplx M[9], int i, int j, cplx a, cplx b)
{
    for (int c = 0; c < 3; ++c) {
        cplx mi = M[3 * i + c], mj = M[3 * j + c];
        M[3 * i + c] = a * mi + b * mj;
        M[3 * j + c] = -conj(b) * mi + conj(a) * mj;
    }
}

/* Gram-Schmidt projection of one link back to SU(3) */
static void reunit_link(cplx *u)
{
    double n0 = 0;
    for (int k = 0; k < 3; ++k) n0 += creal(u[k]) * creal(u[k]) + cimag(u[k]) * cimag(u[k]);
    n0 = 1.0 / sqrt(n0);
    for (int k = 0; k < 3; ++k) u[k] *= n0;
    cplx p = 0;
    for (int k = 0; k < 3; ++k) p += conj(u[k]) * u[3 + k];
    for (int k = 0; k < 3; ++k) u[3 + k] -= p * u[k];
    double n1 = 0;
    for (int k = 0; k < 3; ++k)
        n1 += creal(u[3 + k]) * creal(u[3 + k]) + cimag(u[3 + k]) * cimag(u[3 + k]);
    n1 = 1.0 / sqrt(n1);
    for (int k = 0; k < 3; ++k) u[3 + k] *= n1;
    u[6] = conj(u[1] * u[5] - u[2] * u[4]);
    u[7] = conj(u[2] * u[3] - u[0] * u[5]);
    u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

/* The SU(3) update of one site (Algorithm 1, the body of the loop over x). */
static void site_update(cplx *U, const geom *g, long s, int nd, double omega, int form,
                        int reunit_after)
{
    cplx *fwd[4], *bwd[4];
    for (int mu = 0; mu < 4; ++mu) {
        fwd[mu] = link_at(U, s, mu);
        bwd[mu] = link_at(U, neighbour(g, s, mu, -1), mu);
    }
    /* Eq. (5), in-place form: K = sum_{mu<nd} U_mu(x) + U_mu(x-mu)^dagger */
    cplx K[9];
    for (int e = 0; e < 9; ++e) K[e] = 0;
    for (int mu = 0; mu < nd; ++mu)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                K[3 * r + c] = K[3 * r + c] + (fwd[mu][3 * r + c] + conj(bwd[mu][3 * c + r]));

    /* maximise over the three SU(2) subgroups in turn; g accumulates in G */
    static const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    cplx G[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int k = 0; k < 3; ++k) {
        cplx a, b;
        orc_su2_maximiser(K, pairs[k][0], pairs[k][1], omega, form, &a, &b);
        su2_left_mul(K, pairs[k][0], pairs[k][1], a, b);
        su2_left_mul(G, pairs[k][0], pairs[k][1], a, b);
    }

    /* apply g(x) to U_mu(x) and U_mu(x - mu), for all mu (also mu = 3 in Coulomb) */
    for (int mu = 0; mu < 4; ++mu) {
        cplx t[9];
        mat_mul(G, fwd[mu], t);
        memcpy(fwd[mu], t, sizeof t);
        mat_mul_dag(bwd[mu], G, t);
        memcpy(bwd[mu], t, sizeof t);
        if (reunit_after) {
            reunit_link(fwd[mu]);
            reunit_link(bwd[mu]);
        }
    }
}

/*
 * One checkerboard half-sweep (Algorithm 1, the loop over the sites of one parity).
 * parity p(x) = (x + y + z + t) mod 2.  slice_active (nullable, Lt entries): a site
 * whose time slice has slice_active[t] == 0 is skipped.
 */
int orc_or_half_sweep(cplx *U, const int L[4], int nd, int parity, double omega, int form,
                      int reunit_after, const unsigned char *slice_active)
{
    geom g;
    if (geom_init(&g, L) != 0 || (nd != 3 && nd != 4) || (parity != 0 && parity != 1))
        return -1;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; ++s) {
        if (parity_of(&g, s) != parity) continue;
        if (slice_active && !slice_active[s / g.V3]) continue;
        site_update(U, &g, s, nd, omega, form, reunit_after);
    }
    return 0;
}

/* Reunitarise every link of the field. */
void orc_reunit(cplx *U, long nlinks)
{
#pragma omp parallel for schedule(static)
    for (long l = 0; l < nlinks; ++l) reunit_link(U + 9 * l);
}

/*
 * Algorithm 1: measure theta; while theta >= eps and fewer than maxiter sweeps: even
 * half-sweep, odd half-sweep (reunitarising after the odd half-sweep of every
 * reunit_interval-th sweep), measure.  With per_slice (Coulomb gauge), each time slice
 * t has its own stop rule theta_t < eps; a converged slice is no longer updated.
 * Returns 0 on convergence, 1 if maxiter was reached, < 0 on bad arguments.
 * iters: sweeps done; F, theta: final values; theta_hist (nullable): theta after each
 * sweep, maxiter + 1 entries (entry 0 before the first sweep).
 */
int orc_fix(cplx *U, const int L[4], int nd, double omega, int form, double eps, int maxiter,
            int reunit_interval, int per_slice, int *iters, double *F, double *theta,
            double *theta_hist, int *slice_iters)
{
    geom g;
    if (geom_init(&g, L) != 0 || (nd != 3 && nd != 4)) return -1;
    int Lt = g.L[3];
    double *F_t = malloc(sizeof(double) * Lt), *th_t = malloc(sizeof(double) * Lt);
    unsigned char *active = malloc(Lt);
    if (!F_t || !th_t || !active) { free(F_t); free(th_t); free(active); return -2; }

    orc_measure(U, L, nd, F, theta, F_t, th_t);
    if (theta_hist) theta_hist[0] = *theta;
    int n_active = 0;
    for (int t = 0; t < Lt; ++t) {
        active[t] = per_slice ? (th_t[t] >= eps) : (*theta >= eps);
        n_active += active[t];
        if (slice_iters) slice_iters[t] = 0;
    }
    int it = 0;
    while (n_active > 0 && it < maxiter) {
        int reunit = reunit_interval > 0 && ((it + 1) % reunit_interval) == 0;
        orc_or_half_sweep(U, L, nd, 0, omega, form, 0, active);
        orc_or_half_sweep(U, L, nd, 1, omega, form, reunit, active);
        ++it;
        if (slice_iters)
            for (int t = 0; t < Lt; ++t) slice_iters[t] += active[t];
        orc_measure(U, L, nd, F, theta, F_t, th_t);
        if (theta_hist) theta_hist[it] = *theta;
        n_active = 0;
        for (int t = 0; t < Lt; ++t) {
            if (per_slice) active[t] = active[t] && (th_t[t] >= eps);
            else active[t] = (*theta >= eps);
            n_active += active[t];
        }
    }
    *iters = it;
    free(F_t);
    free(th_t);
    free(active);
    return n_active > 0 ? 1 : 0;
}

/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int orc_num_threads(void) { return omp_get_max_threads(); }
#else
int orc_num_threads(void) { return 1; }
#endif

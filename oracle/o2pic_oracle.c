/*
 * o2pic_oracle.c -- plain FP64 CPU oracle of the PIC-MCC time step of
 * Bronold et al., "Radio-frequency discharges in Oxygen. Part 1: Modeling".
 *
 * TEST INFRASTRUCTURE ONLY: slow, sequential and written to be read against
 * the paper.  Only tests/, the smoke check and bench.py's CPU-baseline leg
 * use it; the GPU library never calls it and shares no code with it.
 *
 * What it follows:
 *   Sec. II  planar 1d3v gap, driven electrode U(t) = U_rf sin(2 pi f t),
 *            grounded electrode, totally absorbing walls, O2 reservoir
 *            n = p/(k T), linear charge assignment / force interpolation,
 *            Poisson equation, Newton push, collisions after free flight,
 *            cell sort, particle-target probability P = n sigma u tau (Eq. 1).
 *   Sec. III isotropic binary collisions with a Maxwellian field particle,
 *            inelastic speed rule (Eq. 5), charge exchange, reactions
 *            (13)-(19) with the rules of Sec. III C, associative detachment
 *            with target density C n_O2.
 *   Sec. III A intra-species Coulomb collisions (1)-(3), the binary model of
 *            Takizuka and Abe with the variance of Eq. 2, every n2 steps.
 * Gas-target channels use the null-collision test, candidate probability
 * 1 - exp(-nu_max dt), then a channel walk with the running sum of
 * n_j sigma_j(E) u; particle-target reactions (13), (14), (19) use Eq. 1 with
 * tau = n1 dt in a per-cell pass after the sort, thinned by a bound on P.  For electrons nu_max may
 * depend on the electron's lab energy (bins of a quarter octave): the
 * null-collision method gives the same collision statistics for any bound
 * that is at least the true frequency.
 *
 * Readings of points the paper leaves open (each restated where used):
 *   x = 0 driven, x = L grounded; a particle with x < 0 or x >= L is absorbed.
 *   Loaded velocities are taken as v at t = -dt/2 (leapfrog, no back-push).
 *   Boundary-node volume dx/2; boundary field from Gauss's law on the half cell.
 *   Energy of a pair = (1/2) mu u^2 (centre-of-mass energy).
 *   (6): the ion takes the gas molecule's velocity (resonant exchange).
 *   (15): O and O- leave back to back in the CM frame with E_cm - dE.
 *   (16): electron with 1/10 of the O- kinetic energy, isotropic.
 *   (17): electron with CM speed from E_cm, isotropic about the CM velocity.
 *   (18), (19): inelastic binary collision, split of the heavy partner into
 *            a charged pair sharing its velocity, then an elastic collision
 *            between the two electrons.
 *   Coulomb: every n2 steps on the sorted cells (before a particle-target
 *            pass due in the same step), tau = n2 dt, eps0 squared in Eq. 2,
 *            pairs from a random affine permutation of the cell (a triangle
 *            for an odd count), ln Gamma a configuration value.
 *   Random numbers: Philox4x32-10 (Salmon et al., SC'11) on a counter made of
 *   (step, index, stream/sub/draw, discharge/species), uniforms (w+0.5)/2^32,
 *   normals by Box-Muller.
 */
#include "o2pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QE 1.602176634e-19
#define ME 9.1093837015e-31
#define AMU 1.66053906660e-27
#define KB 1.380649e-23
#define EPS0 8.8541878128e-12
#define PI 3.14159265358979323846

#define M_OATOM (16.0 * AMU)
#define M_O2 (32.0 * AMU)

enum { SP_E = 0, SP_OM = 1, SP_OP = 2 };

static const double MASS[3] = {ME, M_OATOM + ME, M_O2 - ME};
static const double CHARGE[3] = {-QE, -QE, QE};

typedef struct {
    int reaction, sub, n;
    double *E, *s;
    double th;
    int proj;    /* projectile species */
    int target;  /* -1 gas, else species */
    double ndens;/* gas target density (gas channels) */
} table_t;

typedef struct {
    long long n, cap;
    double *x, *vx, *vy, *vz;
    int *alive;
} parts_t;

typedef struct {
    int sp;
    double x, v[3];
} birth_t;

typedef struct {
    long long n, cap;
    birth_t *b;
} blist_t;

struct orc_sim {
    orc_cfg c;
    double dx, n_gas;
    int nt;
    table_t *t;
    int gas_ch[3][32];
    int n_gas_ch[3];
    int pair_tab[20];
    double numax[3];
    double pnull[3];
    double nubin[64];   /* electrons: bound per lab-energy bin */
    double vmax[3];     /* largest speed per species: at the last sort, raised
                           by the velocity changes since (particle-target pass) */
    double pbin[64];
    parts_t p[3];
    long long step;
    double *rho, *phi, *E, *dens[3];
    long long absorbed[3][2], events[20], viol[3], births[3];
    long long peval;    /* Eq. 1 probabilities evaluated (pair pass, sequential scheme) */
    long long nsamp;
    long long psteps;   /* live particles pushed, summed over steps */
    double *dens_sum[3], *phi_sum;
    long long *eedf, *iedf, *fm;
};

/* ------------------------------------------------------------------ RNG */

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* Philox4x32 with 10 rounds: each round multiplies words 0 and 2 by the
     * two round constants, exchanges halves and xors in the round key; the
     * key is advanced by the two Weyl increments between rounds. */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* stream: 0 null test, 1 gas collision, 2 pair reaction, 3 initial load,
 * 4 pair candidates of a cell, 5 Coulomb pairing and scattering of a cell */
static void rng(const orc_sim *s, int sp, int stream, int sub, uint32_t draw,
                long long step, uint32_t index, uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = (uint32_t)(step & 0xFFFFFFFFll);
    ctr[1] = index;
    ctr[2] = ((uint32_t)stream << 28) | ((uint32_t)sub << 20) | (draw & 0xFFFFFu);
    ctr[3] = ((uint32_t)s->c.discharge << 16) | ((uint32_t)sp << 8) |
             (uint32_t)((step >> 32) & 0xFF);
    key[0] = (uint32_t)(s->c.seed & 0xFFFFFFFFull);
    key[1] = (uint32_t)(s->c.seed >> 32);
    orc_philox(ctr, key, out);
}

static double unif(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

static void box_muller(uint32_t a, uint32_t b, double *n0, double *n1)
{
    double r = sqrt(-2.0 * log(unif(a)));
    double t = 2.0 * PI * unif(b);
    *n0 = r * cos(t);
    *n1 = r * sin(t);
}

/* ------------------------------------------------------- cross sections */

static int lookup_index(const table_t *t, double E)
{
    /* largest k with E_k <= E, k in [0, n-2] (binary search) */
    int lo = 0, hi = t->n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (t->E[mid] <= E)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* Piecewise-linear in E between nodes; held at the end values outside the
 * table (Sec. III: values at the largest energy are extended to all higher
 * energies); zero below the channel threshold. */
static double sigma_of(const table_t *t, double E)
{
    if (E < t->th) return 0.0;
    if (E <= t->E[0]) return t->s[0];
    if (E >= t->E[t->n - 1]) return t->s[t->n - 1];
    int k = lookup_index(t, E);
    double f = (E - t->E[k]) / (t->E[k + 1] - t->E[k]);
    return t->s[k] + f * (t->s[k + 1] - t->s[k]);
}

double orc_sigma(const orc_sim *s, int table, double E_eV)
{
    return sigma_of(&s->t[table], E_eV);
}

static int reaction_projectile(int r)
{
    switch (r) {
    case 5: case 14: case 16: case 17: return SP_OM;
    case 6: return SP_OP;
    default: return SP_E;
    }
}

static int reaction_target(int r)
{
    if (r == 13 || r == 14) return SP_OP;
    if (r == 19) return SP_OM;
    return -1;
}

static double reduced_mass(double a, double b) { return a * b / (a + b); }

/* ion sub-cycling (not in the paper; a throughput variant): O- and O2+ are
 * pushed and tested for gas collisions only on steps n = 0 mod k, over k dt;
 * in between they stay where they are and their charge stays in the grid */
static int ion_k(const orc_cfg *c, int sp) { return (sp > 0 && c->ion_subcycle > 1) ? c->ion_subcycle : 1; }

/* --------------------------------------------------------------- set-up */

static void parts_reserve(parts_t *p, long long cap)
{
    if (cap <= p->cap) return;
    long long nc = p->cap ? p->cap : 1024;
    while (nc < cap) nc *= 2;
    p->x = realloc(p->x, nc * sizeof(double));
    p->vx = realloc(p->vx, nc * sizeof(double));
    p->vy = realloc(p->vy, nc * sizeof(double));
    p->vz = realloc(p->vz, nc * sizeof(double));
    p->alive = realloc(p->alive, nc * sizeof(int));
    p->cap = nc;
}

static void blist_push(blist_t *l, int sp, double x, const double v[3])
{
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 256;
        l->b = realloc(l->b, l->cap * sizeof(birth_t));
    }
    birth_t *b = &l->b[l->n++];
    b->sp = sp;
    b->x = x;
    b->v[0] = v[0];
    b->v[1] = v[1];
    b->v[2] = v[2];
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Bound on the total gas collision frequency sum_j n_j sigma_j(E) u of
 * species sp over centre-of-mass energies 0 <= E <= cap, u = sqrt(2E/mu):
 * [0, cap] is cut at every node and every threshold of the species' gas
 * channels.  Between neighbouring cut points a < b no channel has a node or
 * a threshold, so each sigma_j is linear (or zero) there and at most
 * max(sigma_j(a), sigma_j(b)), and u <= u(b).  The bound is the largest
 * sum_j n_j max(sigma_j(a), sigma_j(b)) u(b) over the intervals, times the
 * safety factor: no energy up to the cap exceeds it. */
static double numax_upto(const orc_sim *s, int sp, double cap)
{
    double mu = reduced_mass(MASS[sp], M_O2);
    int np = 2;
    for (int a = 0; a < s->n_gas_ch[sp]; ++a) np += s->t[s->gas_ch[sp][a]].n + 1;
    double *pt = malloc(np * sizeof(double));
    int m = 0;
    pt[m++] = 0.0;
    pt[m++] = cap;
    for (int a = 0; a < s->n_gas_ch[sp]; ++a) {
        const table_t *ta = &s->t[s->gas_ch[sp][a]];
        for (int k = 0; k < ta->n; ++k)
            if (ta->E[k] > 0.0 && ta->E[k] < cap) pt[m++] = ta->E[k];
        if (ta->th > 0.0 && ta->th < cap) pt[m++] = ta->th;
    }
    qsort(pt, m, sizeof(double), cmp_double);
    double best = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double a = pt[i], b = pt[i + 1];
        if (!(b > a)) continue;
        double u = sqrt(2.0 * b * QE / mu);
        double nu = 0.0;
        for (int c = 0; c < s->n_gas_ch[sp]; ++c) {
            const table_t *tc = &s->t[s->gas_ch[sp][c]];
            double sa = sigma_of(tc, a), sb = sigma_of(tc, b);
            nu += tc->ndens * (sa > sb ? sa : sb) * u;
        }
        if (nu > best) best = nu;
    }
    free(pt);
    return best * s->c.numax_safety;
}

static double compute_numax(const orc_sim *s, int sp)
{
    return numax_upto(s, sp, s->c.ecap_eV[sp]);
}

/* Electron energy bins: bin b holds lab energies K with
 * 4 (log2 K + 6) in [b, b + 1) when K is written m 2^e, m in [1, 2), as
 * 4 (e + 6) + floor(4 (m - 1)) (quarter octaves split linearly in m), K in
 * eV; bins below 0 join bin 0 and bins above the last join the last. */
#define BIN_LOG2_E0 (-6)
int orc_bin_of(const orc_sim *s, double K)
{
    int nb = s->c.numax_bins;
    if (nb <= 0) return 0;
    if (!(K > 0.0)) return 0;
    if (!(K < 1e300)) return nb - 1;
    int ex;
    double mh = frexp(K, &ex);     /* K = mh 2^ex, mh in [0.5, 1) */
    double m = 2.0 * mh;           /* K = m 2^(ex - 1) */
    int e = ex - 1;
    long long b = 4LL * (e - BIN_LOG2_E0) + (long long)((m - 1.0) * 4.0);
    if (b < 0) return 0;
    if (b > nb - 1) return nb - 1;
    return (int)b;
}

/* Upper lab energy of bin b: 2^(e0 + q) (1 + (r + 1)/4) with b = 4q + r. */
static double bin_top(int b)
{
    return ldexp(1.0 + (double)(b % 4 + 1) / 4.0, BIN_LOG2_E0 + b / 4);
}

/* Largest gas-molecule speed a collision can draw, in thermal speeds
 * sqrt(kT/M): the molecule's velocity is sqrt(kT/M) (n0, n1, n2) from two
 * Box-Muller pairs, whose radius sqrt(-2 ln r) is largest for the smallest
 * uniform r = 2^-33 (FP64 uniforms; 2^-24 in FP32), so |(n0, n1)| and |n2|
 * are at most sqrt(66 ln 2) = 6.77 and the speed at most 9.58 of them. */
#define GAS_SPEED_MAX 10.0

/* Bound of bin b (not the last): the relative speed of an electron of the
 * bin and any gas molecule is at most the bin's top electron speed plus
 * GAS_SPEED_MAX thermal speeds, so the bound up to the matching
 * centre-of-mass energy covers every candidate of the bin. */
static double compute_numax_bin(const orc_sim *s, int b)
{
    const int sp = 0;
    double mu = reduced_mass(MASS[sp], M_O2);
    double vtop = sqrt(2.0 * bin_top(b) * QE / MASS[sp]);
    double vg = sqrt(KB * s->c.T_gas / M_O2);
    double urel = vtop + GAS_SPEED_MAX * vg;
    return numax_upto(s, sp, 0.5 * mu * urel * urel / QE);
}

static void load_species(orc_sim *s, int sp)
{
    parts_t *p = &s->p[sp];
    long long n = s->c.n_init[sp];
    parts_reserve(p, n);
    p->n = n;
    double vt = sqrt(s->c.T0_eV[sp] * QE / MASS[sp]);
    for (long long i = 0; i < n; ++i) {
        uint32_t a[4], b[4];
        rng(s, sp, 3, 0, 0, 0, (uint32_t)i, a);
        rng(s, sp, 3, 0, 1, 0, (uint32_t)i, b);
        double n0, n1, n2, n3;
        box_muller(a[0], a[1], &n0, &n1);
        box_muller(a[2], a[3], &n2, &n3);
        p->x[i] = unif(b[0]) * s->c.L;
        p->vx[i] = vt * n0;
        p->vy[i] = vt * n1;
        p->vz[i] = vt * n2;
        p->alive[i] = 1;
    }
}

orc_sim *orc_create(const orc_cfg *cfg, const orc_xs *xs, int n_xs, int load)
{
    orc_sim *s = calloc(1, sizeof(orc_sim));
    s->c = *cfg;
    int N = cfg->n_cells;
    s->dx = cfg->L / N;
    s->n_gas = cfg->p_Pa / (KB * cfg->T_gas); /* n = p/kT (Sec. II) */
    s->nt = n_xs;
    s->t = calloc(n_xs, sizeof(table_t));
    for (int r = 0; r < 20; ++r) s->pair_tab[r] = -1;
    for (int i = 0; i < n_xs; ++i) {
        table_t *t = &s->t[i];
        t->reaction = xs[i].reaction;
        t->sub = xs[i].sub;
        t->n = xs[i].n;
        t->E = malloc(t->n * sizeof(double));
        t->s = malloc(t->n * sizeof(double));
        memcpy(t->E, xs[i].E_eV, t->n * sizeof(double));
        memcpy(t->s, xs[i].sigma_m2, t->n * sizeof(double));
        t->th = xs[i].threshold_eV;
        t->proj = reaction_projectile(t->reaction);
        t->target = reaction_target(t->reaction);
        if (t->target < 0) {
            /* associative detachment sees O2(a) at density C n_O2 (Sec. III C) */
            t->ndens = (t->reaction == 17) ? cfg->C_delta * s->n_gas : s->n_gas;
            s->gas_ch[t->proj][s->n_gas_ch[t->proj]++] = i;
        } else {
            s->pair_tab[t->reaction] = i;
        }
    }
    for (int sp = 0; sp < 3; ++sp) {
        s->numax[sp] = compute_numax(s, sp);
        s->pnull[sp] = 1.0 - exp(-s->numax[sp] * cfg->dt * ion_k(cfg, sp));
    }
    if (s->c.numax_bins > 64) s->c.numax_bins = 64;
    for (int b = 0; b < s->c.numax_bins; ++b) {
        /* the last bin has no upper energy: it keeps the species' bound */
        s->nubin[b] = (b < s->c.numax_bins - 1) ? compute_numax_bin(s, b) : s->numax[0];
        s->pbin[b] = 1.0 - exp(-s->nubin[b] * cfg->dt);
    }
    s->rho = calloc(N + 1, sizeof(double));
    s->phi = calloc(N + 1, sizeof(double));
    s->E = calloc(N + 1, sizeof(double));
    s->phi_sum = calloc(N + 1, sizeof(double));
    for (int sp = 0; sp < 3; ++sp) {
        s->dens[sp] = calloc(N + 1, sizeof(double));
        s->dens_sum[sp] = calloc(N + 1, sizeof(double));
    }
    s->eedf = calloc(cfg->eedf_bins > 0 ? cfg->eedf_bins : 1, sizeof(long long));
    s->iedf = calloc(cfg->iedf_bins > 0 ? 2 * cfg->iedf_bins : 1, sizeof(long long));
    s->fm = calloc((size_t)(cfg->fm_xbins > 0 ? cfg->fm_xbins : 1) * (cfg->fm_bins > 0 ? cfg->fm_bins : 1),
                   sizeof(long long));
    if (load)
        for (int sp = 0; sp < 3; ++sp) load_species(s, sp);
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    for (int i = 0; i < s->nt; ++i) {
        free(s->t[i].E);
        free(s->t[i].s);
    }
    free(s->t);
    for (int sp = 0; sp < 3; ++sp) {
        free(s->p[sp].x);
        free(s->p[sp].vx);
        free(s->p[sp].vy);
        free(s->p[sp].vz);
        free(s->p[sp].alive);
        free(s->dens[sp]);
        free(s->dens_sum[sp]);
    }
    free(s->rho);
    free(s->phi);
    free(s->E);
    free(s->phi_sum);
    free(s->eedf);
    free(s->iedf);
    free(s->fm);
    free(s);
}

/* ------------------------------------------------------- field solve */

/* (phi_{i-1} - 2 phi_i + phi_{i+1}) / dx^2 = -rho_i / eps0 for i = 1..N-1 with
 * Dirichlet values phi_0, phi_N: Thomas elimination on the tridiagonal system. */
void orc_poisson(int N, double dx, double phi0, double phiN, const double *rho,
                 double *phi)
{
    int m = N - 1;
    phi[0] = phi0;
    phi[N] = phiN;
    if (m <= 0) return;
    double *cp = malloc(m * sizeof(double));
    double *dp = malloc(m * sizeof(double));
    /* row i (1..N-1): a = 1, b = -2, c = 1, d = -rho_i dx^2 / eps0 (minus
     * the known boundary values moved to the right-hand side) */
    for (int k = 0; k < m; ++k) {
        int i = k + 1;
        double d = -rho[i] * dx * dx / EPS0;
        if (i == 1) d -= phi0;
        if (i == N - 1) d -= phiN;
        double b = -2.0;
        if (k == 0) {
            cp[k] = 1.0 / b;
            dp[k] = d / b;
        } else {
            double den = b - cp[k - 1];
            cp[k] = 1.0 / den;
            dp[k] = (d - dp[k - 1]) / den;
        }
    }
    phi[m] = dp[m - 1];
    for (int k = m - 2; k >= 0; --k) phi[k + 1] = dp[k] - cp[k] * phi[k + 2];
    free(cp);
    free(dp);
}

/* E = -dphi/dx: centred difference inside; at the walls, Gauss's law on the
 * half cell next to the wall. */
void orc_field(int N, double dx, const double *rho, const double *phi, double *E)
{
    for (int i = 1; i < N; ++i) E[i] = -(phi[i + 1] - phi[i - 1]) / (2.0 * dx);
    E[0] = -(phi[1] - phi[0]) / dx - rho[0] * dx / (2.0 * EPS0);
    E[N] = -(phi[N] - phi[N - 1]) / dx + rho[N] * dx / (2.0 * EPS0);
}

/* ------------------------------------------------------------ deposit */

static void cell_of(const orc_sim *s, double x, int *c, double *f)
{
    double xx = x / s->dx;
    int cc = (int)floor(xx);
    if (cc > s->c.n_cells - 1) cc = s->c.n_cells - 1;
    if (cc < 0) cc = 0;
    *c = cc;
    *f = xx - cc;
}

/* linear charge assignment (Sec. II): node c gets 1-f, node c+1 gets f;
 * density = weight * sum / node volume, volume dx inside and dx/2 at walls */
static void deposit(orc_sim *s)
{
    int N = s->c.n_cells;
    for (int sp = 0; sp < 3; ++sp) {
        double *acc = s->dens[sp];
        memset(acc, 0, (N + 1) * sizeof(double));
        parts_t *p = &s->p[sp];
        for (long long i = 0; i < p->n; ++i) {
            if (!p->alive[i]) continue;
            int c;
            double f;
            cell_of(s, p->x[i], &c, &f);
            acc[c] += 1.0 - f;
            acc[c + 1] += f;
        }
        for (int i = 0; i <= N; ++i) {
            double vol = (i == 0 || i == N) ? 0.5 * s->dx : s->dx;
            acc[i] = s->c.weight * acc[i] / vol;
        }
    }
    for (int i = 0; i <= N; ++i)
        s->rho[i] = QE * (s->dens[SP_OP][i] - s->dens[SP_E][i] - s->dens[SP_OM][i]);
}

/* --------------------------------------------------------- kinematics */

static void iso_dir(double cosx, double phi, double n[3])
{
    double sx = 1.0 - cosx * cosx;
    sx = sx > 0.0 ? sqrt(sx) : 0.0;
    n[0] = sx * cos(phi);
    n[1] = sx * sin(phi);
    n[2] = cosx;
}

/* binary collision of (m, v) with (M, V) in the centre-of-mass frame: the
 * relative speed becomes sqrt(u^2 - 2 dE/mu) (Eq. 5; dE = 0 elastic) along the
 * isotropic direction n; momentum is conserved. */
static void cm_scatter(double m, double M, const double v[3], const double V[3],
                       double dE_J, const double n[3], double vo[3], double Vo[3])
{
    double g[3] = {v[0] - V[0], v[1] - V[1], v[2] - V[2]};
    double u2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    double mu = reduced_mass(m, M);
    double up2 = u2 - 2.0 * dE_J / mu;
    double up = up2 > 0.0 ? sqrt(up2) : 0.0;
    double mt = m + M;
    for (int k = 0; k < 3; ++k) {
        double vcm = (m * v[k] + M * V[k]) / mt;
        vo[k] = vcm + (M / mt) * up * n[k];
        Vo[k] = vcm - (m / mt) * up * n[k];
    }
}

/* elastic collision of two electrons (equal masses) */
static void ee_elastic(double a[3], double b[3], const double n[3])
{
    double g[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
    double u = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int k = 0; k < 3; ++k) {
        double c = 0.5 * (a[k] + b[k]);
        a[k] = c + 0.5 * u * n[k];
        b[k] = c - 0.5 * u * n[k];
    }
}

static double pair_energy_eV(double m, double M, const double v[3], const double V[3])
{
    double g0 = v[0] - V[0], g1 = v[1] - V[1], g2 = v[2] - V[2];
    return 0.5 * reduced_mass(m, M) * (g0 * g0 + g1 * g1 + g2 * g2) / QE;
}

int orc_gas_event(const orc_sim *s, int sp, int reaction, int table,
                  const double v[3], const double V[3], const double r4[4],
                  const double r2[2], double vout[3], int *alive_out,
                  int *prod_sp, double *prod_v, double *Vout)
{
    const table_t *t = &s->t[table];
    double m = MASS[sp];
    double n[3], dummy[3];
    int np = 0;
    iso_dir(1.0 - 2.0 * r4[1], 2.0 * PI * r4[2], n);
    *alive_out = 1;
    vout[0] = v[0];
    vout[1] = v[1];
    vout[2] = v[2];
    if (Vout) {
        Vout[0] = V[0];
        Vout[1] = V[1];
        Vout[2] = V[2];
    }
    switch (reaction) {
    case 4: case 5:
        cm_scatter(m, M_O2, v, V, 0.0, n, vout, Vout ? Vout : dummy);
        break;
    case 6:
        if (s->c.cx_isotropic) {
            cm_scatter(m, M_O2, v, V, 0.0, n, vout, Vout ? Vout : dummy);
        } else {
            /* resonant exchange: the new ion is the former gas molecule */
            vout[0] = V[0];
            vout[1] = V[1];
            vout[2] = V[2];
            if (Vout) {
                Vout[0] = v[0];
                Vout[1] = v[1];
                Vout[2] = v[2];
            }
        }
        break;
    case 7: case 8: case 9: case 10: case 11: case 12:
        cm_scatter(m, M_O2, v, V, t->th * QE, n, vout, Vout ? Vout : dummy);
        break;
    case 15: {
        /* e + O2 -> O + O-: electron removed, O- born; O and O- share
         * E_cm - dE back to back in the CM frame */
        double E = pair_energy_eV(m, M_O2, v, V) - t->th;
        if (E < 0.0) E = 0.0;
        double mu2 = reduced_mass(M_OATOM, MASS[SP_OM]);
        double pmag = sqrt(2.0 * E * QE * mu2);
        double mt = m + M_O2;
        *alive_out = 0;
        prod_sp[np] = SP_OM;
        for (int k = 0; k < 3; ++k) {
            double vcm = (m * v[k] + M_O2 * V[k]) / mt;
            prod_v[3 * np + k] = vcm + pmag / MASS[SP_OM] * n[k];
        }
        ++np;
        break;
    }
    case 16: {
        /* O- + O2 -> O + O2 + e: O- removed, electron with a tenth of the O-
         * kinetic energy in an isotropic direction */
        double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        double ke = 0.5 * MASS[SP_OM] * v2 / 10.0;
        double ve = sqrt(2.0 * ke / ME);
        *alive_out = 0;
        prod_sp[np] = SP_E;
        for (int k = 0; k < 3; ++k) prod_v[3 * np + k] = ve * n[k];
        ++np;
        break;
    }
    case 17: {
        /* O- + O2(a) -> O3 + e: O- removed, electron with CM energy E_cm
         * leaving isotropically from the pair's CM velocity */
        double E = pair_energy_eV(m, M_O2, v, V);
        double w = sqrt(2.0 * E * QE / ME);
        double mt = m + M_O2;
        *alive_out = 0;
        prod_sp[np] = SP_E;
        for (int k = 0; k < 3; ++k) {
            double vcm = (m * v[k] + M_O2 * V[k]) / mt;
            prod_v[3 * np + k] = vcm + w * n[k];
        }
        ++np;
        break;
    }
    case 18: {
        /* e + O2 -> 2e + O2+: inelastic binary collision with the ionisation
         * energy, O2 split into O2+ and e2 at its post-collision velocity,
         * then an elastic e1-e2 collision */
        double v1[3], Vo[3], n2[3];
        cm_scatter(m, M_O2, v, V, t->th * QE, n, v1, Vo);
        double e2[3] = {Vo[0], Vo[1], Vo[2]};
        iso_dir(1.0 - 2.0 * r2[0], 2.0 * PI * r2[1], n2);
        ee_elastic(v1, e2, n2);
        vout[0] = v1[0];
        vout[1] = v1[1];
        vout[2] = v1[2];
        prod_sp[np] = SP_E;
        for (int k = 0; k < 3; ++k) prod_v[3 * np + k] = e2[k];
        ++np;
        prod_sp[np] = SP_OP;
        for (int k = 0; k < 3; ++k) prod_v[3 * np + k] = Vo[k];
        ++np;
        if (Vout) {
            Vout[0] = Vo[0];
            Vout[1] = Vo[1];
            Vout[2] = Vo[2];
        }
        break;
    }
    default:
        break;
    }
    return np;
}

void orc_pair19_event(const orc_sim *s, int table, const double v[3],
                      const double vt[3], const double rc[2], const double r2[2],
                      double v1[3], double v2[3], double Vo[3])
{
    /* e + O- -> O + 2e: inelastic e-O- collision with the detachment energy,
     * O- split into O and e2 at its post-collision velocity, elastic e1-e2 */
    const table_t *t = &s->t[table];
    double n[3], n2[3];
    iso_dir(1.0 - 2.0 * rc[0], 2.0 * PI * rc[1], n);
    cm_scatter(ME, MASS[SP_OM], v, vt, t->th * QE, n, v1, Vo);
    v2[0] = Vo[0];
    v2[1] = Vo[1];
    v2[2] = Vo[2];
    iso_dir(1.0 - 2.0 * r2[0], 2.0 * PI * r2[1], n2);
    ee_elastic(v1, v2, n2);
}

/* ------------------------------------------------------------- the step */

static void absorb(orc_sim *s, int sp, int wall, const double v[3])
{
    s->absorbed[sp][wall]++;
    if (sp == SP_OP && s->c.iedf_bins > 0) {
        double E = 0.5 * MASS[SP_OP] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / QE;
        double b = floor(E / s->c.iedf_emax * s->c.iedf_bins);
        if (b >= 0 && b < s->c.iedf_bins) s->iedf[wall * s->c.iedf_bins + (int)b]++;
    }
}

static void sample_histograms(orc_sim *s, int sp, double x, const double v[3])
{
    int N = s->c.n_cells;
    int c;
    double f;
    cell_of(s, x, &c, &f);
    if (sp == SP_E && s->c.eedf_bins > 0 && c == N / 2) {
        double E = 0.5 * ME * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / QE;
        double b = floor(E / s->c.eedf_emax * s->c.eedf_bins);
        if (b >= 0 && b < s->c.eedf_bins) s->eedf[(int)b]++;
    }
    if (sp == SP_OM && s->c.fm_bins > 0) {
        /* signed energy sign(vx) M vx^2 / 2 (Sec. IV, f_-(E, x)) */
        double E = 0.5 * MASS[SP_OM] * v[0] * v[0] / QE;
        if (v[0] < 0.0) E = -E;
        double b = floor((E + s->c.fm_emax) / (2.0 * s->c.fm_emax) * s->c.fm_bins);
        /* x binned into fm_xbins equal regions of the gap, by cell */
        int xb = (int)(((long long)c * s->c.fm_xbins) / N);
        if (b >= 0 && b < s->c.fm_bins) s->fm[(size_t)xb * s->c.fm_bins + (int)b]++;
    }
}

/* null-collision test, channel choice and kinematics for one gas candidate */
static void gas_collision(orc_sim *s, int sp, long long i, double numax, blist_t *bl)
{
    parts_t *p = &s->p[sp];
    uint32_t a[4], b[4], c2[4];
    rng(s, sp, 1, 0, 0, s->step, (uint32_t)i, a);
    rng(s, sp, 1, 0, 1, s->step, (uint32_t)i, b);
    double n0, n1, n2, n3;
    box_muller(a[0], a[1], &n0, &n1);
    box_muller(a[2], a[3], &n2, &n3);
    double vg = sqrt(KB * s->c.T_gas / M_O2);
    double V[3] = {vg * n0, vg * n1, vg * n2};
    double v[3] = {p->vx[i], p->vy[i], p->vz[i]};
    double g0 = v[0] - V[0], g1 = v[1] - V[1], g2 = v[2] - V[2];
    double u = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    double E = 0.5 * reduced_mass(MASS[sp], M_O2) * u * u / QE;
    double target = unif(b[0]) * numax;
    double cum = 0.0;
    int chosen = -1;
    for (int k = 0; k < s->n_gas_ch[sp]; ++k) {
        const table_t *t = &s->t[s->gas_ch[sp][k]];
        cum += t->ndens * sigma_of(t, E) * u;
        if (chosen < 0 && target < cum) chosen = s->gas_ch[sp][k];
    }
    if (cum > numax) s->viol[0]++;
    if (chosen < 0) return; /* null event */
    const table_t *t = &s->t[chosen];
    double r4[4] = {unif(b[0]), unif(b[1]), unif(b[2]), unif(b[3])};
    double r2[2] = {0.5, 0.5};
    if (t->reaction == 18) {
        rng(s, sp, 1, 0, 2, s->step, (uint32_t)i, c2);
        r2[0] = unif(c2[0]);
        r2[1] = unif(c2[1]);
    }
    double vo[3], pv[6];
    int alive, psp[2];
    int np = orc_gas_event(s, sp, t->reaction, chosen, v, V, r4, r2, vo, &alive,
                           psp, pv, NULL);
    s->events[t->reaction]++;
    p->vx[i] = vo[0];
    p->vy[i] = vo[1];
    p->vz[i] = vo[2];
    p->alive[i] = alive;
    for (int k = 0; k < np; ++k) blist_push(&bl[psp[k]], psp[k], p->x[i], &pv[3 * k]);
}

/* ------------------------------------------- sequential gas channels */

/* The gas-target channels in the order of Table I (reaction number, then
 * table order): the list the sequential scheme walks.  Returns its length. */
static int dsmc_list(const orc_sim *s, int *list)
{
    int n = 0;
    for (int r = 4; r <= 18; ++r)
        for (int i = 0; i < s->nt; ++i)
            if (s->t[i].reaction == r && s->t[i].target < 0) list[n++] = i;
    return n;
}

/* Channel k of the list for a particle of species sp with velocity v, the
 * chain of root (root_sp, root) in generation gen (Sec. II and Eq. 1): a gas
 * molecule from the Maxwellian at T_gas, u the relative speed, E the centre-
 * of-mass energy; the channel takes place with P = n sigma(E) u tau, tau =
 * n1 dt, clamped at 1 (and counted).  Random numbers: stream 6 of the root,
 * sub-stream k, draws 4 gen (gas molecule), 4 gen + 1 (test and direction),
 * 4 gen + 2 (the second direction of (18)).  Returns -1 if nothing happens,
 * else the number of products (orc_gas_event). */
static int dsmc_channel(orc_sim *s, int root_sp, long long root, int gen, int k, int tabi,
                        int sp, const double v[3], double vo[3], int *alive, int *psp,
                        double *pv)
{
    const table_t *t = &s->t[tabi];
    uint32_t a[4], b[4], c2[4];
    rng(s, root_sp, 6, k, (uint32_t)(4 * gen), s->step, (uint32_t)root, a);
    rng(s, root_sp, 6, k, (uint32_t)(4 * gen + 1), s->step, (uint32_t)root, b);
    double n0, n1, n2, n3;
    box_muller(a[0], a[1], &n0, &n1);
    box_muller(a[2], a[3], &n2, &n3);
    double vg = sqrt(KB * s->c.T_gas / M_O2);
    double V[3] = {vg * n0, vg * n1, vg * n2};
    double g0 = v[0] - V[0], g1 = v[1] - V[1], g2 = v[2] - V[2];
    double u = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    double E = 0.5 * reduced_mass(MASS[sp], M_O2) * u * u / QE;
    double P = t->ndens * sigma_of(t, E) * u * (s->c.n1 * s->c.dt);
    s->peval++;
    if (P > 1.0) {
        s->viol[1]++;
        P = 1.0;
    }
    if (!(unif(b[0]) < P)) return -1;
    double r4[4] = {unif(b[0]), unif(b[1]), unif(b[2]), unif(b[3])};
    double r2[2] = {0.5, 0.5};
    if (t->reaction == 18) {
        rng(s, root_sp, 6, k, (uint32_t)(4 * gen + 2), s->step, (uint32_t)root, c2);
        r2[0] = unif(c2[0]);
        r2[1] = unif(c2[1]);
    }
    s->events[t->reaction]++;
    return orc_gas_event(s, sp, t->reaction, tabi, v, V, r4, r2, vo, alive, psp, pv, NULL);
}

/* One pass of the sequential scheme over the channels of the list numbered
 * below 13 (part 0) or above 14 (part 1): roots in species order, then slot
 * order.  A particle meets the channels of its species in list order; one
 * that dies in (15), (16) or (17) is replaced by its product, which meets the
 * later channels of the list ("readmitted for the next collision"); products
 * of (18) meet no later gas channel.  Births are appended in root order:
 * (18)'s electron and O2+ when they occur, the product that ends a chain
 * after the chain. */
static void dsmc_pass(orc_sim *s, int part, blist_t *bl)
{
    int list[64];
    int nl = dsmc_list(s, list);
    for (int sp = 0; sp < 3; ++sp) {
        parts_t *p = &s->p[sp];
        for (long long i = 0; i < p->n; ++i) {
            if (!p->alive[i]) continue;
            int cs = sp, gen = 0;
            double v[3] = {p->vx[i], p->vy[i], p->vz[i]};
            for (int k = 0; k < nl; ++k) {
                const table_t *t = &s->t[list[k]];
                if (t->proj != cs) continue;
                if (part == 0 ? t->reaction > 12 : t->reaction < 15) continue;
                double vo[3], pv[6];
                int alive, psp[2];
                int np = dsmc_channel(s, sp, i, gen, k, list[k], cs, v, vo, &alive, psp, pv);
                if (np < 0) continue;
                if (alive) {
                    for (int q = 0; q < 3; ++q) v[q] = vo[q];
                    for (int q = 0; q < np; ++q) blist_push(&bl[psp[q]], psp[q], p->x[i], &pv[3 * q]);
                } else {
                    cs = psp[0];
                    for (int q = 0; q < 3; ++q) v[q] = pv[q];
                    ++gen;
                }
            }
            if (gen == 0) {
                p->vx[i] = v[0];
                p->vy[i] = v[1];
                p->vz[i] = v[2];
            } else {
                p->alive[i] = 0;
                blist_push(&bl[cs], cs, p->x[i], v);
            }
        }
    }
}

static void append_births(orc_sim *s, blist_t *bl)
{
    for (int sp = 0; sp < 3; ++sp) {
        parts_t *p = &s->p[sp];
        parts_reserve(p, p->n + bl[sp].n);
        for (long long k = 0; k < bl[sp].n; ++k) {
            birth_t *b = &bl[sp].b[k];
            long long j = p->n++;
            p->x[j] = b->x;
            p->vx[j] = b->v[0];
            p->vy[j] = b->v[1];
            p->vz[j] = b->v[2];
            p->alive[j] = 1;
        }
        s->births[sp] += bl[sp].n;
        bl[sp].n = 0;
    }
}

/* stable counting sort by cell; dead slots dropped (Sec. II: particles are
 * sorted into cells after the free flight) */
static void sort_species(orc_sim *s, int sp, long long *start)
{
    int N = s->c.n_cells;
    parts_t *p = &s->p[sp];
    long long *cnt = calloc(N + 1, sizeof(long long));
    int *cell = malloc((p->n > 0 ? p->n : 1) * sizeof(int));
    for (long long i = 0; i < p->n; ++i) {
        if (!p->alive[i]) continue;
        double f;
        cell_of(s, p->x[i], &cell[i], &f);
        cnt[cell[i] + 1]++;
    }
    for (int c = 0; c < N; ++c) cnt[c + 1] += cnt[c];
    long long live = cnt[N];
    for (int c = 0; c <= N; ++c) start[c] = cnt[c];
    parts_t q = {0};
    parts_reserve(&q, live > 0 ? live : 1);
    q.n = live;
    s->vmax[sp] = 0.0;
    for (long long i = 0; i < p->n; ++i) {
        if (!p->alive[i]) continue;
        long long d = cnt[cell[i]]++;
        double spd = sqrt(p->vx[i] * p->vx[i] + p->vy[i] * p->vy[i] + p->vz[i] * p->vz[i]);
        if (spd > s->vmax[sp]) s->vmax[sp] = spd;
        q.x[d] = p->x[i];
        q.vx[d] = p->vx[i];
        q.vy[d] = p->vy[i];
        q.vz[d] = p->vz[i];
        q.alive[d] = 1;
    }
    free(p->x);
    free(p->vx);
    free(p->vy);
    free(p->vz);
    free(p->alive);
    *p = q;
    free(cnt);
    free(cell);
}

/* the largest speeds after a pass that changed velocities (Coulomb
 * collisions, the first part of the sequential gas scheme): the recorded
 * maximum of each species is raised to the largest speed of its live
 * particles, so it still bounds every speed */
static void raise_vmax(orc_sim *s)
{
    for (int sp = 0; sp < 3; ++sp) {
        const parts_t *p = &s->p[sp];
        for (long long i = 0; i < p->n; ++i) {
            if (!p->alive[i]) continue;
            double spd = sqrt(p->vx[i] * p->vx[i] + p->vy[i] * p->vy[i] + p->vz[i] * p->vz[i]);
            if (spd > s->vmax[sp]) s->vmax[sp] = spd;
        }
    }
}

/* u rounded up to 5 significant bits (u = m 2^e, m in [1/2, 1): ceil(32 m)/32
 * 2^e): the relative-speed cap of the particle-target pass, a few per cent
 * above the sum of the largest speeds, on a coarse grid that the same sum
 * computed with other roundings meets with the same result */
static double round_up_5bits(double u)
{
    if (!(u > 0.0)) return 0.0;
    int e;
    double m = frexp(u, &e);
    return ldexp(ceil(m * 32.0) / 32.0, e);
}

/* Bound on sigma(E) u over a particle-target table for relative speeds up
 * to u_cap (SI): on a segment [E_k, E_k+1] sigma is at most the larger end
 * value and u at most the speed of E_k+1; below the grid sigma is the first
 * value; above it sigma is the last value, so sigma u <= sigma_last u_cap;
 * with a relative margin of 1e-3. */
static double pair_bound(const table_t *t, double mu, double u_cap)
{
    double g = t->s[0] * sqrt(2.0 * t->E[0] * QE / mu);
    for (int k = 0; k + 1 < t->n; ++k) {
        double sk = t->s[k] > t->s[k + 1] ? t->s[k] : t->s[k + 1];
        double gk = sk * sqrt(2.0 * t->E[k + 1] * QE / mu);
        if (gk > g) g = gk;
    }
    double tail = t->s[t->n - 1] * u_cap;
    return 1.001 * (g > tail ? g : tail);
}

/* Particle-target reaction in one cell (Eq. 1 with tau = n1 dt, P clamped at
 * 1 and the clamp counted: reading R10), evaluated by thinning.  No pair is
 * faster than the sum of the two species' largest speeds, so with u_cap that
 * sum (rounded up), B = n_T max sigma u tau over u <= u_cap bounds P for every
 * pair of the pass.  Candidates are drawn among the cell's projectiles with
 * probability min(B, 1) each (geometric gaps, a random stream per cell), and
 * a candidate reacts with probability min(P, 1)/min(B, 1): every projectile
 * reacts with probability min(P, 1), as if each were tested. */
static void pair_channel(orc_sim *s, int reaction, int c, long long **start, blist_t *bl)
{
    int tab = s->pair_tab[reaction];
    if (tab < 0) return;
    const table_t *t = &s->t[tab];
    int ps = t->proj, ts = t->target;
    parts_t *P = &s->p[ps], *T = &s->p[ts];
    long long p0 = start[ps][c], p1 = start[ps][c + 1];
    long long t0 = start[ts][c], t1 = start[ts][c + 1];
    long long range = t1 - t0;
    if (range <= 0) return;
    long long live = 0;
    for (long long j = t0; j < t1; ++j) live += T->alive[j];
    if (live == 0) return;
    double nT = (double)live * s->c.weight / s->dx;
    double tau = s->c.n1 * s->c.dt;
    double mp = MASS[ps], mt = MASS[ts];
    double mu = reduced_mass(mp, mt);
    double u_cap = round_up_5bits(s->vmax[ps] + s->vmax[ts]);
    double B = nT * pair_bound(t, mu, u_cap) * tau;
    double lq = B < 1.0 ? log1p(-B) : 0.0;
    double Bc = B < 1.0 ? B : 1.0;
    long long i = p0 - 1;
    uint32_t draw = 0;
    for (;;) {
        if (B >= 1.0) {
            ++i;
        } else {
            uint32_t g[4];
            rng(s, ps, 4, reaction, draw++, s->step, (uint32_t)c, g);
            double G = floor(log(unif(g[0])) / lq);
            if (G >= (double)(p1 - i)) break;
            i += 1 + (long long)G;
        }
        if (i >= p1) break;
        if (!P->alive[i]) continue;
        uint32_t d0[4];
        rng(s, ps, 2, reaction, 0, s->step, (uint32_t)i, d0);
        long long j = t0 + (long long)(((uint64_t)d0[0] * (uint64_t)range) >> 32);
        long long walked = 0;
        while (!T->alive[j] && walked < range) {
            j = (j + 1 < t1) ? j + 1 : t0;
            ++walked;
        }
        if (!T->alive[j]) break; /* no live target left in this cell */
        double v[3] = {P->vx[i], P->vy[i], P->vz[i]};
        double vt[3] = {T->vx[j], T->vy[j], T->vz[j]};
        double g0 = v[0] - vt[0], g1 = v[1] - vt[1], g2 = v[2] - vt[2];
        double u = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
        double E = 0.5 * reduced_mass(mp, mt) * u * u / QE;
        double P_ = nT * sigma_of(t, E) * u * tau;
        s->peval++;
        if (P_ > 1.0) {  /* Eq. 1 beyond 1: clamped (R10) and counted */
            s->viol[1]++;
            P_ = 1.0;
        }
        if (P_ > Bc) s->viol[2]++;  /* the bound failed: cannot happen (u <= u_cap) */
        if (!(unif(d0[1]) * Bc < P_)) continue;
        s->events[reaction]++;
        if (reaction == 13 || reaction == 14) {
            P->alive[i] = 0;
            T->alive[j] = 0;
        } else { /* 19 */
            uint32_t d1[4];
            rng(s, ps, 2, reaction, 1, s->step, (uint32_t)i, d1);
            double rc[2] = {unif(d0[2]), unif(d0[3])};
            double r2[2] = {unif(d1[0]), unif(d1[1])};
            double v1[3], v2[3], Vo[3];
            orc_pair19_event(s, tab, v, vt, rc, r2, v1, v2, Vo);
            P->vx[i] = v1[0];
            P->vy[i] = v1[1];
            P->vz[i] = v1[2];
            T->alive[j] = 0;
            blist_push(&bl[SP_E], SP_E, P->x[i], v2);
        }
    }
}

/* ------------------------------------------------------ Coulomb (1)-(3) */

/* One binary Coulomb collision between two particles of species sp (Sec.
 * III A, Eq. 2, the binary model of Takizuka and Abe): tan(chi/2) is normal
 * with variance q^4 n lnGamma tau / (8 pi eps0^2 mu^2 u^3) (eps0 squared: the
 * printed Eq. 2 is not dimensionless without it), mu = m/2 the reduced mass,
 * u the relative speed; the azimuth is uniform.  The relative velocity g is
 * turned by chi about itself (azimuth measured from the plane of g and the z
 * axis), and each particle takes half of its change (equal masses). */
void orc_coulomb_pair(const orc_sim *s, int sp, double v1[3], double v2[3],
                      double n, double tau, double xi, double r)
{
    double g[3] = {v1[0] - v2[0], v1[1] - v2[1], v1[2] - v2[2]};
    double u = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(u > 0.0)) return;
    double q = CHARGE[sp], mu = 0.5 * MASS[sp];
    double var = q * q * q * q * n * s->c.coulomb_log * tau /
                 (8.0 * PI * EPS0 * EPS0 * mu * mu * u * u * u);
    double d = sqrt(var) * xi; /* tan(chi/2) */
    /* sin(chi) = 2d/(1+d^2), 1 - cos(chi) = 2d^2/(1+d^2); for |d| > 1 the
     * same in e = 1/d, which stays finite as d grows without bound */
    double sn, om;
    if (fabs(d) <= 1.0) {
        sn = 2.0 * d / (1.0 + d * d);
        om = 2.0 * d * d / (1.0 + d * d);
    } else {
        double e = 1.0 / d;
        sn = 2.0 * e / (1.0 + e * e);
        om = 2.0 / (1.0 + e * e);
    }
    double phi = 2.0 * PI * r;
    double cp = cos(phi), spn = sin(phi);
    double up = sqrt(g[0] * g[0] + g[1] * g[1]);
    double dg[3];
    if (up > 0.0) {
        dg[0] = (g[0] / up) * g[2] * sn * cp - (g[1] / up) * u * sn * spn - g[0] * om;
        dg[1] = (g[1] / up) * g[2] * sn * cp + (g[0] / up) * u * sn * spn - g[1] * om;
        dg[2] = -up * sn * cp - g[2] * om;
    } else {
        dg[0] = u * sn * cp;
        dg[1] = u * sn * spn;
        dg[2] = -g[2] * om;
    }
    for (int k = 0; k < 3; ++k) {
        v1[k] += 0.5 * dg[k];
        v2[k] -= 0.5 * dg[k];
    }
}

static long long gcd_ll(long long a, long long b)
{
    while (b) {
        long long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* random numbers of the k-th collision of a cell's Coulomb pass: stream 5,
 * draw counter k split over the sub-stream (high bits) and draw fields */
static void coulomb_rng(const orc_sim *s, int sp, long long step, uint32_t cell,
                        long long k, uint32_t out[4])
{
    rng(s, sp, 5, (int)(k >> 20), (uint32_t)(k & 0xFFFFF), step, cell, out);
}

/* collision k of a cell takes draw 1 + k/2 of the cell's stream: the normal
 * is the first (k even) or second (k odd) of that draw's Box-Muller pair,
 * the azimuth its third or fourth word */
static void coulomb_one(const orc_sim *s, int sp, double *vx, double *vy, double *vz,
                        long long i, long long j, double dens, double tau,
                        long long step, uint32_t cell, long long k)
{
    uint32_t d[4];
    coulomb_rng(s, sp, step, cell, 1 + k / 2, d);
    double n0, n1;
    box_muller(d[0], d[1], &n0, &n1);
    double v1[3] = {vx[i], vy[i], vz[i]}, v2[3] = {vx[j], vy[j], vz[j]};
    orc_coulomb_pair(s, sp, v1, v2, dens, tau, (k % 2) ? n1 : n0, unif(d[2 + k % 2]));
    vx[i] = v1[0]; vy[i] = v1[1]; vz[i] = v1[2];
    vx[j] = v2[0]; vy[j] = v2[1]; vz[j] = v2[2];
}

/* The Coulomb pairing of a cell of n >= 2 particles: a random affine
 * permutation k -> (a k + b) mod n, a coprime to n (a and b from draw 0 of the
 * cell's stream 5), pairs pi(0) with pi(1), pi(2) with pi(3), ...; for odd n
 * the last three, A, B, C, collide as (A, B), (B, C), (C, A), each with half
 * the collision time, so that every particle scatters over tau once.  Writes
 * the collisions in draw order (collisions 2m and 2m+1 share draw 1 + m) and
 * returns their number; the last three are the triangle's when n is odd. */
long long orc_coulomb_pairing(const orc_sim *s, int sp, long long n, long long step,
                              uint32_t cell, long long *pi, long long *pj)
{
    if (n < 2) return 0;
    uint32_t w[4];
    coulomb_rng(s, sp, step, cell, 0, w);
    long long a = 1 + (long long)(w[0] % (uint64_t)(n - 1));
    while (gcd_ll(a, n) != 1) a = (a % (n - 1)) + 1;
    long long b = (long long)(w[1] % (uint64_t)n);
    long long pairs = (n % 2 == 0) ? n / 2 : (n - 3) / 2, k = 0;
    for (long long m = 0; m < pairs; ++m, ++k) {
        pi[k] = (a * (2 * m) + b) % n;
        pj[k] = (a * (2 * m + 1) + b) % n;
    }
    if (n % 2 == 1)
        for (int t = 0; t < 3; ++t, ++k) {
            pi[k] = (a * (n - 3 + t) + b) % n;
            pj[k] = (a * (n - 3 + (t + 1) % 3) + b) % n;
        }
    return k;
}

/* Coulomb collisions among the n particles (velocities vx, vy, vz) of one
 * cell, paired as orc_coulomb_pairing */
void orc_coulomb_cell(const orc_sim *s, int sp, double *vx, double *vy, double *vz,
                      long long n, double dens, double tau, long long step, uint32_t cell)
{
    if (n < 2) return;
    long long cap = n / 2 + 2;
    long long *pi = malloc(cap * sizeof(long long)), *pj = malloc(cap * sizeof(long long));
    long long nc = orc_coulomb_pairing(s, sp, n, step, cell, pi, pj);
    for (long long k = 0; k < nc; ++k) {
        double t = (n % 2 == 1 && k >= nc - 3) ? 0.5 * tau : tau;
        coulomb_one(s, sp, vx, vy, vz, pi[k], pj[k], dens, t, step, cell, k);
    }
    free(pi);
    free(pj);
}

/* Coulomb pass of species sp over the sorted cells: the density of Eq. 2 is
 * the species' own count in the cell times the weight over the cell volume,
 * the collision time tau = n2 dt */
/* One Coulomb collision between a particle of species sa (velocity v1) and
 * one of species sb (v2) (Sec. III A; the binary model of Takizuka and Abe
 * for unlike particles): tan(chi/2) normal with variance q_a^2 q_b^2 n
 * lnGamma tau / (8 pi eps0^2 mu^2 u^3), mu = m_a m_b / (m_a + m_b); g turned
 * as for like particles, particle a takes m_b/(m_a + m_b) of the change of
 * g, particle b minus m_a/(m_a + m_b) of it. */
void orc_coulomb_pair2(const orc_sim *s, int sa, int sb, double v1[3], double v2[3],
                       double n, double tau, double xi, double r)
{
    double g[3] = {v1[0] - v2[0], v1[1] - v2[1], v1[2] - v2[2]};
    double u = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(u > 0.0)) return;
    double ma = MASS[sa], mb = MASS[sb], mu = reduced_mass(ma, mb);
    double qq = CHARGE[sa] * CHARGE[sb];
    double var = qq * qq * n * s->c.coulomb_log * tau / (8.0 * PI * EPS0 * EPS0 * mu * mu * u * u * u);
    double d = sqrt(var) * xi;
    double sn, om;
    if (fabs(d) <= 1.0) {
        sn = 2.0 * d / (1.0 + d * d);
        om = 2.0 * d * d / (1.0 + d * d);
    } else {
        double e = 1.0 / d;
        sn = 2.0 * e / (1.0 + e * e);
        om = 2.0 / (1.0 + e * e);
    }
    double phi = 2.0 * PI * r;
    double cp = cos(phi), spn = sin(phi);
    double up = sqrt(g[0] * g[0] + g[1] * g[1]);
    double dg[3];
    if (up > 0.0) {
        dg[0] = (g[0] / up) * g[2] * sn * cp - (g[1] / up) * u * sn * spn - g[0] * om;
        dg[1] = (g[1] / up) * g[2] * sn * cp + (g[0] / up) * u * sn * spn - g[1] * om;
        dg[2] = -up * sn * cp - g[2] * om;
    } else {
        dg[0] = u * sn * cp;
        dg[1] = u * sn * spn;
        dg[2] = -g[2] * om;
    }
    double fa = mb / (ma + mb), fb = ma / (ma + mb);
    for (int k = 0; k < 3; ++k) {
        v1[k] += fa * dg[k];
        v2[k] -= fb * dg[k];
    }
}

static const int INTER_PAIR[3][2] = {{SP_E, SP_OM}, {SP_E, SP_OP}, {SP_OM, SP_OP}};

/* an affine permutation k -> (a k + b) mod n with a coprime to n from two
 * random words (the identity for n = 1) */
static void affine_of(long long n, uint32_t w0, uint32_t w1, long long *a, long long *b)
{
    if (n < 2) {
        *a = 1;
        *b = 0;
        return;
    }
    long long x = 1 + (long long)(w0 % (uint64_t)(n - 1));
    while (gcd_ll(x, n) != 1) x = (x % (n - 1)) + 1;
    *a = x;
    *b = (long long)(w1 % (uint64_t)n);
}

/* Inter-species pairing (Takizuka and Abe for unlike particles): the nA
 * particles of the more numerous species (A) each collide once, with the
 * particles of the other (B) taken in turn, so that each B particle collides
 * about nA/nB times; both lists are shuffled by affine permutations drawn
 * from draw 0 of stream 5 of the cell with species field 3 + pair (words 0,
 * 1 for A, 2, 3 for B).  Collision k joins A pi_A(k) with B pi_B(k mod nB)
 * and takes draw 1 + k/2 like the intra-species collisions. */
void orc_coulomb_inter_pairing(const orc_sim *s, int pair, long long nA, long long nB,
                               long long step, uint32_t cell, long long *ia, long long *ib)
{
    uint32_t w[4];
    coulomb_rng(s, 3 + pair, step, cell, 0, w);
    long long aA, bA, aB, bB;
    affine_of(nA, w[0], w[1], &aA, &bA);
    affine_of(nB, w[2], w[3], &aB, &bB);
    for (long long k = 0; k < nA; ++k) {
        ia[k] = (aA * k + bA) % nA;
        ib[k] = (aB * (k % nB) + bB) % nB;
    }
}

/* the inter-species Coulomb collisions of one species pair in every cell;
 * the density of Eq. 2 is that of the less numerous species in the cell
 * (each A particle meets that density once over tau; each B particle meets
 * nA/nB of them, the density of A) */
static void coulomb_inter(orc_sim *s, int pair, long long **start)
{
    int s0 = INTER_PAIR[pair][0], s1 = INTER_PAIR[pair][1];
    double tau = s->c.n2 * s->c.dt;
    for (int c = 0; c < s->c.n_cells; ++c) {
        long long n0 = start[s0][c + 1] - start[s0][c], n1 = start[s1][c + 1] - start[s1][c];
        if (n0 == 0 || n1 == 0) continue;
        int sA = n0 >= n1 ? s0 : s1, sB = n0 >= n1 ? s1 : s0;
        long long nA = n0 >= n1 ? n0 : n1, nB = n0 >= n1 ? n1 : n0;
        parts_t *A = &s->p[sA], *B = &s->p[sB];
        long long pA = start[sA][c], pB = start[sB][c];
        long long *ia = malloc(nA * sizeof(long long)), *ib = malloc(nA * sizeof(long long));
        orc_coulomb_inter_pairing(s, pair, nA, nB, s->step, (uint32_t)c, ia, ib);
        double dens = (double)nB * s->c.weight / s->dx;
        for (long long k = 0; k < nA; ++k) {
            long long i = pA + ia[k], j = pB + ib[k];
            uint32_t d[4];
            coulomb_rng(s, 3 + pair, s->step, (uint32_t)c, 1 + k / 2, d);
            double g0, g1;
            box_muller(d[0], d[1], &g0, &g1);
            double v1[3] = {A->vx[i], A->vy[i], A->vz[i]}, v2[3] = {B->vx[j], B->vy[j], B->vz[j]};
            orc_coulomb_pair2(s, sA, sB, v1, v2, dens, tau, (k % 2) ? g1 : g0, unif(d[2 + k % 2]));
            A->vx[i] = v1[0]; A->vy[i] = v1[1]; A->vz[i] = v1[2];
            B->vx[j] = v2[0]; B->vy[j] = v2[1]; B->vz[j] = v2[2];
        }
        free(ia);
        free(ib);
    }
}

static void coulomb_species(orc_sim *s, int sp, const long long *start)
{
    parts_t *p = &s->p[sp];
    double tau = s->c.n2 * s->c.dt;
    for (int c = 0; c < s->c.n_cells; ++c) {
        long long p0 = start[c], n = start[c + 1] - start[c];
        orc_coulomb_cell(s, sp, p->vx + p0, p->vy + p0, p->vz + p0, n,
                         (double)n * s->c.weight / s->dx, tau, s->step, (uint32_t)c);
    }
}

static void step_once(orc_sim *s)
{
    int N = s->c.n_cells;
    double t = s->step * s->c.dt;
    int diag = s->c.diag_every > 0 && (s->step % s->c.diag_every) == 0;

    /* charge assignment, Poisson, field at t_n */
    deposit(s);
    orc_poisson(N, s->dx, s->c.U_rf * sin(2.0 * PI * s->c.f_rf * t + s->c.rf_phase), 0.0, s->rho, s->phi);
    orc_field(N, s->dx, s->rho, s->phi, s->E);
    if (diag) {
        for (int sp = 0; sp < 3; ++sp)
            for (int i = 0; i <= N; ++i) s->dens_sum[sp][i] += s->dens[sp][i];
        for (int i = 0; i <= N; ++i) s->phi_sum[i] += s->phi[i];
        s->nsamp++;
    }

    blist_t bl[3] = {{0}};
    for (int sp = 0; sp < 3; ++sp) {
        parts_t *p = &s->p[sp];
        int ks = ion_k(&s->c, sp);
        if (s->step % ks != 0) continue;   /* a sub-cycled ion species rests */
        double qm = CHARGE[sp] / MASS[sp];
        double dts = ks * s->c.dt;
        long long last_blk = -1;
        uint32_t w0[4] = {0};
        for (long long i = 0; i < p->n; ++i) {
            if (!p->alive[i]) continue;
            s->psteps++;
            /* force interpolation (linear) and leapfrog push */
            int c;
            double f;
            cell_of(s, p->x[i], &c, &f);
            double Ep = (1.0 - f) * s->E[c] + f * s->E[c + 1];
            p->vx[i] += qm * Ep * dts;
            p->x[i] += p->vx[i] * dts;
            if (p->x[i] < 0.0 || p->x[i] >= s->c.L) {
                double v[3] = {p->vx[i], p->vy[i], p->vz[i]};
                absorb(s, sp, p->x[i] < 0.0 ? 0 : 1, v);
                p->alive[i] = 0;
                continue;
            }
            /* distributions sampled after the free flight, before collisions */
            if (diag) {
                double v[3] = {p->vx[i], p->vy[i], p->vz[i]};
                sample_histograms(s, sp, p->x[i], v);
            }
            /* null-collision test: one Philox block serves four slots */
            if ((i >> 2) != last_blk) {
                last_blk = i >> 2;
                rng(s, sp, 0, 0, 0, s->step, (uint32_t)(i >> 2), w0);
            }
            double pc = s->pnull[sp], nu = s->numax[sp];
            if (sp == 0 && s->c.numax_bins > 0) {
                /* electrons: the bound of their lab-energy bin */
                double v2 = p->vx[i] * p->vx[i] + p->vy[i] * p->vy[i] + p->vz[i] * p->vz[i];
                int b = orc_bin_of(s, 0.5 * MASS[0] * v2 / QE);
                pc = s->pbin[b];
                nu = s->nubin[b];
            }
            if (s->c.gas_scheme == 0 && unif(w0[i & 3]) < pc) gas_collision(s, sp, i, nu, bl);
        }
    }
    append_births(s, bl);

    long long next = s->step + 1;
    int pair = s->c.n1 > 0 && (next % s->c.n1) == 0;
    int coul = s->c.n2 > 0 && (next % s->c.n2) == 0;
    int sort = pair || coul || (s->c.sort_interval > 0 && (next % s->c.sort_interval) == 0);
    if (sort) {
        long long *start[3];
        for (int sp = 0; sp < 3; ++sp) {
            start[sp] = malloc((N + 1) * sizeof(long long));
            sort_species(s, sp, start[sp]);
        }
        /* Coulomb collisions (1)-(3) every n2 steps on the sorted cells,
         * then the particle-target reactions every n1 steps */
        if (coul) {
            for (int sp = 0; sp < 3; ++sp) coulomb_species(s, sp, start[sp]);
            /* inter-species collisions after the intra-species ones, pairs
             * e-O-, e-O2+, O- - O2+ in turn */
            if (s->c.coulomb_inter)
                for (int pr = 0; pr < 3; ++pr) coulomb_inter(s, pr, start);
            raise_vmax(s);
        }
        if (pair && s->c.gas_scheme == 1) {
            /* the sequential scheme: the whole list of Table I in order, gas
             * channels before (13), (13), (14), gas channels after (14) with
             * their products readmitted, a new sort (particles were born and
             * removed), (19) */
            dsmc_pass(s, 0, bl);
            raise_vmax(s);
            for (int c = 0; c < N; ++c) {
                pair_channel(s, 13, c, start, bl);
                pair_channel(s, 14, c, start, bl);
            }
            dsmc_pass(s, 1, bl);
            append_births(s, bl);
            for (int sp = 0; sp < 3; ++sp) sort_species(s, sp, start[sp]);
            for (int c = 0; c < N; ++c) pair_channel(s, 19, c, start, bl);
            append_births(s, bl);
        } else if (pair) {
            for (int c = 0; c < N; ++c) {
                pair_channel(s, 13, c, start, bl);
                pair_channel(s, 14, c, start, bl);
                pair_channel(s, 19, c, start, bl);
            }
            append_births(s, bl);
        }
        for (int sp = 0; sp < 3; ++sp) free(start[sp]);
    }
    for (int sp = 0; sp < 3; ++sp) free(bl[sp].b);
    s->step = next;
}

void orc_step(orc_sim *s, long long nsteps)
{
    for (long long k = 0; k < nsteps; ++k) step_once(s);
    deposit(s); /* leave rho of the current positions for orc_fields */
}

/* ---------------------------------------------------------- accessors */

long long orc_step_index(const orc_sim *s) { return s->step; }
long long orc_particle_steps(const orc_sim *s) { return s->psteps; }
long long orc_eq1_evaluations(const orc_sim *s) { return s->peval; }
void orc_set_step(orc_sim *s, long long step) { s->step = step; }
long long orc_count(const orc_sim *s, int sp) { return s->p[sp].n; }
double orc_numax(const orc_sim *s, int sp) { return s->numax[sp]; }
double orc_numax_bin(const orc_sim *s, int b)
{
    return (b >= 0 && b < s->c.numax_bins) ? s->nubin[b] : 0.0;
}

void orc_get(const orc_sim *s, int sp, double *x, double *vx, double *vy,
             double *vz, int *alive)
{
    const parts_t *p = &s->p[sp];
    size_t b = p->n * sizeof(double);
    if (x) memcpy(x, p->x, b);
    if (vx) memcpy(vx, p->vx, b);
    if (vy) memcpy(vy, p->vy, b);
    if (vz) memcpy(vz, p->vz, b);
    if (alive) memcpy(alive, p->alive, p->n * sizeof(int));
}

int orc_set(orc_sim *s, int sp, long long n, const double *x, const double *vx,
            const double *vy, const double *vz, const int *alive)
{
    parts_t *p = &s->p[sp];
    parts_reserve(p, n > 0 ? n : 1);
    p->n = n;
    for (long long i = 0; i < n; ++i) {
        p->x[i] = x[i];
        p->vx[i] = vx[i];
        p->vy[i] = vy[i];
        p->vz[i] = vz[i];
        p->alive[i] = alive ? (alive[i] != 0) : 1;
    }
    return 0;
}

void orc_fields(orc_sim *s, double *rho, double *phi, double *E)
{
    int N = s->c.n_cells;
    double t = s->step * s->c.dt;
    deposit(s);
    orc_poisson(N, s->dx, s->c.U_rf * sin(2.0 * PI * s->c.f_rf * t + s->c.rf_phase), 0.0, s->rho, s->phi);
    orc_field(N, s->dx, s->rho, s->phi, s->E);
    size_t b = (N + 1) * sizeof(double);
    if (rho) memcpy(rho, s->rho, b);
    if (phi) memcpy(phi, s->phi, b);
    if (E) memcpy(E, s->E, b);
}

void orc_counters(const orc_sim *s, long long *absorbed, long long *events,
                  long long *violations, long long *births)
{
    if (absorbed)
        for (int sp = 0; sp < 3; ++sp)
            for (int w = 0; w < 2; ++w) absorbed[2 * sp + w] = s->absorbed[sp][w];
    if (events) memcpy(events, s->events, sizeof(s->events));
    if (violations) {
        violations[0] = s->viol[0];
        violations[1] = s->viol[1];
        violations[2] = s->viol[2];
    }
    if (births) memcpy(births, s->births, sizeof(s->births));
}

void orc_reset_diag(orc_sim *s)
{
    int N = s->c.n_cells;
    for (int sp = 0; sp < 3; ++sp) memset(s->dens_sum[sp], 0, (N + 1) * sizeof(double));
    memset(s->phi_sum, 0, (N + 1) * sizeof(double));
    if (s->c.eedf_bins > 0) memset(s->eedf, 0, s->c.eedf_bins * sizeof(long long));
    if (s->c.iedf_bins > 0) memset(s->iedf, 0, 2 * s->c.iedf_bins * sizeof(long long));
    if (s->c.fm_bins > 0) memset(s->fm, 0, (size_t)s->c.fm_xbins * s->c.fm_bins * sizeof(long long));
    s->nsamp = 0;
}

long long orc_diag(const orc_sim *s, double *dens_sum, double *phi_sum,
                   long long *eedf, long long *iedf, long long *fm)
{
    int N = s->c.n_cells;
    if (dens_sum)
        for (int sp = 0; sp < 3; ++sp)
            memcpy(dens_sum + (size_t)sp * (N + 1), s->dens_sum[sp], (N + 1) * sizeof(double));
    if (phi_sum) memcpy(phi_sum, s->phi_sum, (N + 1) * sizeof(double));
    if (eedf && s->c.eedf_bins > 0) memcpy(eedf, s->eedf, s->c.eedf_bins * sizeof(long long));
    if (iedf && s->c.iedf_bins > 0) memcpy(iedf, s->iedf, 2 * s->c.iedf_bins * sizeof(long long));
    if (fm && s->c.fm_bins > 0)
        memcpy(fm, s->fm, (size_t)s->c.fm_xbins * s->c.fm_bins * sizeof(long long));
    return s->nsamp;
}

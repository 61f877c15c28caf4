/*
 * o2pic_oracle.h -- declarations of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the GPU library
 * against a slow, obviously correct restatement of the method of Bronold et
 * al., "Radio-frequency discharges in Oxygen. Part 1: Modeling"
 * (Sec. II, Sec. III, Eqs. 1-9, Table I).  Only tests/, the smoke check and
 * the CPU-baseline leg of bench.py may load it.  It shares no code, header,
 * constant or table generator with the CUDA library.
 *
 * Species: 0 = electron, 1 = O-, 2 = O2+.  All quantities SI unless a name
 * says otherwise (_eV).
 */
#ifndef O2PIC_ORACLE_H
#define O2PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double L;            /* electrode gap [m] (Sec. II) */
    double p_Pa;         /* O2 reservoir pressure (Sec. II) */
    double T_gas;        /* O2 temperature [K] */
    double U_rf;         /* RF amplitude [V], driven electrode at x = 0 */
    double f_rf;         /* RF frequency [Hz] */
    double rf_phase;     /* U(t) = U_rf sin(2 pi f t + rf_phase); 0 in the paper */
    double dt;           /* time step [s] */
    double weight;       /* real particles per m^2 of electrode per superparticle */
    double C_delta;      /* O2(a) / O2 density ratio (Sec. III C, "C") */
    double T0_eV[3];     /* initial Maxwellian temperatures */
    double ecap_eV[3];   /* energy cap used when bounding the collision frequency */
    double numax_safety; /* multiplier on the bound (>= 1) */
    double eedf_emax, iedf_emax, fm_emax;   /* histogram ranges [eV] */
    long long n_init[3]; /* initial superparticles per species */
    unsigned long long seed;
    int n_cells;
    int n1;              /* pair-reaction interval in steps (tau = n1 dt) */
    int sort_interval;   /* cell sort interval in steps */
    int diag_every;      /* 0 = no diagnostics */
    int eedf_bins, iedf_bins, fm_bins;
    int fm_xbins;        /* f_-(E, x): equal regions of (0, L) */
    int discharge;       /* discharge index, enters the random counter */
    int cx_isotropic;    /* reaction (6): 0 = velocity swap, 1 = isotropic */
    int numax_bins;      /* electrons: collision-frequency bounds per quarter
                            octave of lab energy from 2^-6 eV (0 = one bound) */
    int n2;              /* intra-species Coulomb collisions every n2 steps,
                            tau = n2 dt (0 = none) */
    int gas_scheme;      /* gas targets: 0 null collision every step, 1 the
                            sequential channel test every n1 steps (Sec. II) */
    int ion_subcycle;    /* k > 1: O- and O2+ pushed (and tested for gas
                            collisions) only on steps n = 0 mod k, with k dt */
    int coulomb_inter;   /* 1: inter-species Coulomb collisions as well */
    double coulomb_log;  /* ln Gamma of Eq. 2 */
} orc_cfg;

typedef struct {
    int reaction;          /* 4..19, numbering of Table I */
    int sub;               /* vibrational level for reaction 7, else 0 */
    int n;                 /* nodes */
    const double *E_eV;    /* node energies, strictly increasing */
    const double *sigma_m2;/* cross section at the nodes */
    double threshold_eV;   /* sigma = 0 below; energy loss of the channel */
} orc_xs;

typedef struct orc_sim orc_sim;

orc_sim *orc_create(const orc_cfg *cfg, const orc_xs *xs, int n_xs, int load);
void orc_destroy(orc_sim *s);
void orc_step(orc_sim *s, long long nsteps);
long long orc_step_index(const orc_sim *s);
long long orc_particle_steps(const orc_sim *s);
/* Eq. 1 probabilities evaluated (particle-target candidates, sequential-scheme tests) */
long long orc_eq1_evaluations(const orc_sim *s);
long long orc_count(const orc_sim *s, int sp);
void orc_get(const orc_sim *s, int sp, double *x, double *vx, double *vy,
             double *vz, int *alive);
int orc_set(orc_sim *s, int sp, long long n, const double *x, const double *vx,
            const double *vy, const double *vz, const int *alive);
void orc_set_step(orc_sim *s, long long step);
double orc_numax(const orc_sim *s, int sp);
/* electrons: bound of energy bin b, and the bin of a lab energy K [eV] */
double orc_numax_bin(const orc_sim *s, int b);
int orc_bin_of(const orc_sim *s, double K_eV);
void orc_fields(orc_sim *s, double *rho, double *phi, double *E);
/* counters: absorbed[3][2], events[20], violations[3] (gas nu_max exceeded,
 * Eq. 1 P > 1 clamps, particle-target bound below P: never expected), births[3] */
void orc_counters(const orc_sim *s, long long *absorbed, long long *events,
                  long long *violations, long long *births);
/* diagnostics: dens_sum[3][N+1], phi_sum[N+1], eedf, iedf[2][bins], fm[xbins][bins] */
/* clear the diagnostic sums and histograms (a new averaging window) */
void orc_reset_diag(orc_sim *s);
long long orc_diag(const orc_sim *s, double *dens_sum, double *phi_sum,
                   long long *eedf, long long *iedf, long long *fm);

/* unit-level entry points used by the pins */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_sigma(const orc_sim *s, int table, double E_eV);
void orc_poisson(int n_cells, double dx, double phi0, double phiN,
                 const double *rho, double *phi);
void orc_field(int n_cells, double dx, const double *rho, const double *phi,
               double *E);
/* one gas-target event of reaction r for a particle of species sp with
 * velocity v against a gas molecule of velocity V; r4 = four uniforms of the
 * second draw, r2 = two uniforms of the third draw.  Outputs the particle's new
 * velocity, the products (up to 2: species + velocity), their count, and
 * whether the particle survives. */
int orc_gas_event(const orc_sim *s, int sp, int reaction, int table,
                  const double v[3], const double V[3], const double r4[4],
                  const double r2[2], double vout[3], int *alive_out,
                  int *prod_sp, double *prod_v, double *Vout);
/* one intra-species Coulomb collision of species sp (Eq. 2): velocities
 * v1, v2 [m/s] in place, n the species' density, tau the collision time,
 * xi a standard normal and r a uniform in (0, 1) */
void orc_coulomb_pair(const orc_sim *s, int sp, double v1[3], double v2[3],
                      double n, double tau, double xi, double r);
/* one Coulomb collision between particles of species sa and sb (Eq. 2 with
 * q_a^2 q_b^2 and the reduced mass of the pair) */
void orc_coulomb_pair2(const orc_sim *s, int sa, int sb, double v1[3], double v2[3],
                       double n, double tau, double xi, double r);
/* the inter-species pairing of a cell with nA particles of the more
 * numerous species and nB of the other, for species pair `pair` (0: e-O-,
 * 1: e-O2+, 2: O- - O2+): collision k joins A particle ia[k] with B particle
 * ib[k], k = 0..nA-1 */
void orc_coulomb_inter_pairing(const orc_sim *s, int pair, long long nA, long long nB,
                               long long step, uint32_t cell, long long *ia, long long *ib);
/* the Coulomb pairing of a cell of n particles of species sp at step `step`:
 * writes the partners of every collision in draw order (n/2 + 2 entries
 * suffice) and returns their number (the last three form the triangle of an
 * odd n) */
long long orc_coulomb_pairing(const orc_sim *s, int sp, long long n, long long step,
                              uint32_t cell, long long *pi, long long *pj);
/* the Coulomb collisions of one cell's n particles of species sp at step
 * `step` (velocities in place; pairing and draws as the Coulomb pass) */
void orc_coulomb_cell(const orc_sim *s, int sp, double *vx, double *vy, double *vz,
                      long long n, double dens, double tau, long long step, uint32_t cell);
/* reaction 19 pair event: electron v, O- target vt; returns e1 and e2 */
void orc_pair19_event(const orc_sim *s, int table, const double v[3],
                      const double vt[3], const double rc[2], const double r2[2],
                      double v1[3], double v2[3], double Vo[3]);

#ifdef __cplusplus
}
#endif
#endif

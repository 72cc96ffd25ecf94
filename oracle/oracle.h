/*
 * oracle.h — plain, slow FP64 CPU oracle for the sheared-suspension
 * lattice-Boltzmann + particle step of Pradipto & Hayakawa,
 * "Simulation of dense non-Brownian suspensions with the lattice Boltzmann
 * method: shear jammed and fragile states" (arXiv:1904.02929).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this code: only the tests, the smoke check and the CPU-baseline leg
 * and reference arm of the benchmark use it.  It shares no header, constant table or helper
 * with the CUDA library; both are written from the paper independently.
 *
 * Every routine follows the paper's equations in the paper's order:
 *   Eq. 3 (streaming), Eq. 4 (moments), Eq. 5 (collision, BGK reading),
 *   Eq. 7/8 (moving bounce-back), Eq. 6/9/10 (link momentum exchange),
 *   Eq. 1 (rigid-body motion), Eq. 11/11t (frictional contacts),
 *   Eq. 13 (double-layer repulsion), Appendix A (lubrication correction),
 *   Eq. 12/14/15 (stress), Eq. 16 (oscillatory protocol),
 *   Eq. 19-23 (angular contact distributions), Eq. 26/27 (angular stress).
 * Lees-Edwards shear is not in the paper; it follows the standard
 * interpolated plane shift with a Galilean correction (see oracle.c).
 */
#ifndef SUSP_ORACLE_H
#define SUSP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_sim orc_sim;

typedef struct {
  int nx, ny, nz;           /* lattice: x flow, y gradient (Lees-Edwards), z vorticity */
  double tau, rho0;         /* BGK relaxation time, reference density                */
  int n;                    /* number of particles                                    */
  const double *radius;     /* [n] contact radii                                      */
  const double *pos;        /* [3n] centres                                           */
  const double *vel;        /* [3n] or NULL                                           */
  const double *omega;      /* [3n] or NULL                                           */
  double rho_p;             /* particle density                                       */
  double mu, kn, kt_ratio;  /* friction, normal stiffness, kt/kn                      */
  double eta_n;             /* normal dashpot; < 0 selects sqrt(m0 kn)                */
  double F0, debye;         /* double-layer amplitude and length; F0 = 0 disables     */
  double lub_delta;         /* roughness length delta                                 */
  double lub_cut;           /* lubrication correction applies for gap < lub_cut       */
  double a_map_ratio;       /* mapped radius / contact radius                         */
  int dem_substeps;         /* 0 selects automatic sub-cycling                        */
  int quasi2d;              /* monolayer constraint                                   */
  int move_particles;       /* 0: particles held (forces still computed)              */
  int nbins;                /* angular histogram bins over [0, pi)                    */
  double body_force[3];     /* uniform force density on the fluid                     */
  int collision;            /* 0 BGK (one eigenvalue -1/tau), 1 Ladd's linear operator */
  double tau_bulk;          /* Ladd: bulk eigenvalue -1/tau_bulk (shear: -1/tau)      */
  const int *driven;        /* [n] or NULL: 1 = moves with its given velocity and spin
                               whatever the forces (wall particles)                   */
} orc_params;

typedef struct {
  int kind;                 /* 0 constant rate, 1 oscillatory (Eq. 16)                */
  double rate;              /* shear rate for kind 0                                  */
  double gamma0, omega, theta;
} orc_shear;

/* Stress kinds, mirroring the product's enumeration by value. */
enum { ORC_VISCOUS = 0, ORC_CONTACT = 1, ORC_REPULSIVE = 2, ORC_TOTAL = 3, ORC_ANGULAR = 4,
       ORC_LUBRICATION = 5 };

/* error bits */
enum { ORC_EOVERLAP = 1, ORC_EUNSTABLE = 2, ORC_EHIST = 4 };

orc_sim *orc_create(const orc_params *p);
void orc_destroy(orc_sim *s);
int orc_step(orc_sim *s, int nsteps, const orc_shear *sh);
int orc_error(const orc_sim *s);
long orc_ncell(const orc_sim *s);
int orc_nsub(const orc_sim *s);
long orc_time(const orc_sim *s);
double orc_delta(const orc_sim *s);

void orc_get_populations(const orc_sim *s, double *f);  /* [19][ncell], post-collision */
void orc_set_populations(orc_sim *s, const double *f);
void orc_get_owner(const orc_sim *s, int *owner);        /* [ncell]                     */
void orc_get_particles(const orc_sim *s, double *pos, double *vel, double *omega);
void orc_get_hydro(const orc_sim *s, double *F, double *T); /* link sums of the last step */
/* covering / uncovering impulses waiting to be applied at the next step */
void orc_get_pending(const orc_sim *s, double *F, double *T);
int orc_stress(const orc_sim *s, int kind, double out[9], double *hist, int nbins);
void orc_stress_reset(orc_sim *s);
/* Storage and loss moduli (Eq. 17, 18) of the total shear stress over the
 * steps since the last reset, for strain amplitude gamma0 (the window should
 * hold whole periods of the oscillatory protocol).  -1 if gamma0 <= 0. */
int orc_moduli(const orc_sim *s, double gamma0, double *Gp, double *Gpp);

/* ---- component routines (used by the step; exposed for the pins) ---- */
void orc_lattice(int c[19][3], double w[19], int opp[19]);
void orc_equilibrium(double rho, const double j[3], double out[19]);
/* One contact pair in the canonical orientation (a, b).  d = R_b - R_a
 * (already minimum-imaged), uab = U_a - U_b (image velocity included).
 * hist_t[3] holds the tangential spring on entry and the updated spring on
 * exit.  Outputs: force on a (force on b is its negative), torques on a, b,
 * normal-force magnitude and whether the pair is in contact. */
int orc_contact(double ra, double rb, const double d[3], const double uab[3],
                const double wa[3], const double wb[3], double kn, double kt,
                double eta_n, double mu, double dt, double hist_t[3],
                double Fa[3], double Ta[3], double Tb[3], double *fn_mag,
                double Ftan[3]);
/* Lubrication correction (Appendix A) for one pair; same orientation. */
void orc_lubrication(double ra, double rb, const double d[3], const double uab[3],
                     const double wa[3], const double wb[3], double eta0,
                     double delta, double hcut, double Fa[3], double Ta[3],
                     double Tb[3]);
/* Lubrication stresslet of one pair (Appendix A, G and H blocks): S = S_a + S_b. */
void orc_lubrication_stresslet(double ra, double rb, const double d[3], const double uab[3],
                               const double wa[3], const double wb[3], double eta0,
                               double delta, double hcut, double S[9]);
/* Oscillatory protocol, Eq. 16. */
double orc_gamma(const orc_shear *sh, double t);
/* Lees-Edwards offset increment of one step (t -> t+1) for a box of height ly. */
double orc_le_increment(const orc_shear *sh, long t, double ly);
/* Angular stress, Eq. 26 (two_d != 0) or Eq. 27, from a histogram
 * hist[3*nbins] = (count, sum F_nor, sum F_tan) per bin. */
void orc_angular_stress(const double *hist, int nbins, double phi, double z_coord,
                        double a, int two_d, double out[9]);

#ifdef __cplusplus
}
#endif
#endif

/*
 * oracle.c — plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg and
 * reference arm may call this file.  It is deliberately written as straightforward loops in the
 * order of the paper's equations; no blocking, fusion or reordering.
 *
 * Conventions (lattice units, dx = dt = 1, c_s^2 = 1/3):
 *   node r = (x, y, z) at integer coordinates, index x + nx (y + ny z);
 *   populations stored post-collision, f[q][cell] = n*(r, c_q, t);
 *   x flow, y gradient (Lees-Edwards planes), z vorticity;
 *   the image of the box above is shifted by +Delta(t) in x and moves with
 *   +U_LE; the image below is shifted by -Delta and moves with -U_LE.
 */
#define _DEFAULT_SOURCE
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 19
#define HSLOTS 32

/* D3Q19 velocity set (Appendix A; weights C^q = 1/3, 1/18, 1/36). */
static const int CV[Q][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight(int q) {
  int s = abs(CV[q][0]) + abs(CV[q][1]) + abs(CV[q][2]);
  if (s == 0) return 1.0 / 3.0;
  if (s == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

static int opposite(int q) {
  for (int p = 0; p < Q; ++p)
    if (CV[p][0] == -CV[q][0] && CV[p][1] == -CV[q][1] && CV[p][2] == -CV[q][2]) return p;
  return -1;
}

void orc_lattice(int c[19][3], double w[19], int opp[19]) {
  for (int q = 0; q < Q; ++q) {
    for (int a = 0; a < 3; ++a) c[q][a] = CV[q][a];
    w[q] = weight(q);
    opp[q] = opposite(q);
  }
}

/* Equilibrium of the a1 row: n^eq_q = C^q [rho + 3 j.c + 9/2 (j.c)^2/rho - 3/2 j^2/rho]. */
void orc_equilibrium(double rho, const double j[3], double out[19]) {
  double jj = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
  for (int q = 0; q < Q; ++q) {
    double jc = j[0] * CV[q][0] + j[1] * CV[q][1] + j[2] * CV[q][2];
    out[q] = weight(q) * (rho + 3.0 * jc + 4.5 * jc * jc / rho - 1.5 * jj / rho);
  }
}

static double feq1(int q, double rho, const double j[3]) {
  double jj = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
  double jc = j[0] * CV[q][0] + j[1] * CV[q][1] + j[2] * CV[q][2];
  return weight(q) * (rho + 3.0 * jc + 4.5 * jc * jc / rho - 1.5 * jj / rho);
}

/* ------------------------------------------------------------------ */

struct orc_sim {
  int nx, ny, nz;
  long ncell;
  double tau, rho0, g[3];
  int collision;            /* 0 BGK, 1 Ladd */
  double tau_bulk;
  int n;
  double *rad, *amap, *mass, *inert;
  int *drv;                 /* [n] driven (prescribed-velocity) particles */
  double *R, *U, *W;        /* [3n] position, velocity, angular velocity */
  double *Fh, *Th;          /* link sums of the current step             */
  double *Fcov, *Tcov;      /* covering / uncovering impulses, pending   */
  double *Fp, *Tp;          /* pair forces of a sub-step                  */
  double mu, kn, kt, eta_n, F0, debye, lub_delta, lub_cut, eta0;
  int nsub, quasi2d, move, nbins;
  double *fA, *fB;
  int *owner;
  /* tangential springs: per particle a, slots for partners b > a */
  int *hcnt[2], *hpart[2];
  double *hval[2];
  int hcur;
  /* protocol */
  long t;
  double delta, delta_c;
  /* stress sums */
  double s_visc[9], s_slet[9], s_cont[9], s_rep[9], s_lub[9];
  /* Eq. 17, 18: sums over the steps of the step's shear stress sigma_xy
   * (total, times V) weighted by cos and sin of omega (t + 1/2) + Theta */
  double s_gc, s_gs;
  double *hist;
  long nsamples, ncontacts;
  int err;
};

static long cidx(const orc_sim *s, int x, int y, int z) {
  return (long)x + (long)s->nx * ((long)y + (long)s->ny * (long)z);
}
static int wrapi(int v, int L) { int r = v % L; return r < 0 ? r + L : r; }
static double nearest(double d, double L) { return d - L * floor(d / L + 0.5); }

/* Lees-Edwards minimum image of a displacement d = p - R (p a point, R a
 * particle centre).  Returns k: the nearest image of the particle is
 * R + k (delta, ny, 0) and moves with U + k U_LE e_x. */
static int le_image(const orc_sim *s, double delta, double d[3]) {
  int k = (int)floor(d[1] / s->ny + 0.5);
  d[1] -= k * (double)s->ny;
  d[0] -= k * delta;
  d[0] = nearest(d[0], s->nx);
  d[2] = nearest(d[2], s->nz);
  return k;
}

static void cross(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ---------------- protocol (Eq. 16) ---------------- */

double orc_gamma(const orc_shear *sh, double t) {
  if (sh->kind == 0) return sh->rate * t;
  return sh->gamma0 * (cos(sh->theta) - cos(sh->omega * t + sh->theta));
}

/* U_LE of step t -> t+1: Ly times the strain increment of that step. */
double orc_le_increment(const orc_shear *sh, long t, double ly) {
  if (sh->kind == 0) return ly * sh->rate;
  double a = sh->omega * (double)t + sh->theta;
  double b = sh->omega * (double)(t + 1) + sh->theta;
  return ly * sh->gamma0 * (cos(a) - cos(b));
}

/* Kahan-compensated offset update, kept in [0, nx). */
static void le_advance(const orc_sim *s, double *delta, double *comp, double inc) {
  double y = inc - *comp;
  double t = *delta + y;
  *comp = (t - *delta) - y;
  *delta = t;
  if (*delta >= s->nx) *delta -= s->nx;
  if (*delta < 0.0) *delta += s->nx;
}

/* ---------------- creation ---------------- */

static int auto_substeps(const orc_sim *s) {
  double mmin = 1e300, amin = 1e300;
  for (int i = 0; i < s->n; ++i) {
    if (s->mass[i] < mmin) mmin = s->mass[i];
    if (s->rad[i] < amin) amin = s->rad[i];

  }
  if (s->n == 0) return 1;
  double omega = sqrt(2.0 * s->kn / mmin);
  double zeta = 0.0;
  if (s->lub_cut > 0.0 && s->lub_delta > 0.0)
    zeta = s->eta0 * 1.5 * M_PI * amin * amin / s->lub_delta;
  double c = 2.0 * (s->eta_n + zeta) / mmin;
  double m = omega > c ? omega : c;
  int ns = (int)ceil(m);
  return ns < 1 ? 1 : ns;
}

static void node_map_init(orc_sim *s);

orc_sim *orc_create(const orc_params *p) {
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  s->nx = p->nx; s->ny = p->ny; s->nz = p->nz;
  s->ncell = (long)p->nx * p->ny * p->nz;
  s->tau = p->tau; s->rho0 = p->rho0;
  s->collision = p->collision; s->tau_bulk = p->tau_bulk > 0.0 ? p->tau_bulk : p->tau;
  for (int a = 0; a < 3; ++a) s->g[a] = p->body_force[a];
  s->n = p->n;
  int n = p->n > 0 ? p->n : 1;
  s->rad = calloc(n, sizeof(double)); s->amap = calloc(n, sizeof(double));
  s->mass = calloc(n, sizeof(double)); s->inert = calloc(n, sizeof(double));
  s->drv = calloc(n, sizeof(int));
  for (int i = 0; i < p->n; ++i) s->drv[i] = p->driven ? (p->driven[i] != 0) : 0;
  s->R = calloc(3 * n, sizeof(double)); s->U = calloc(3 * n, sizeof(double));
  s->W = calloc(3 * n, sizeof(double));
  s->Fh = calloc(3 * n, sizeof(double)); s->Th = calloc(3 * n, sizeof(double));
  s->Fcov = calloc(3 * n, sizeof(double)); s->Tcov = calloc(3 * n, sizeof(double));
  s->Fp = calloc(3 * n, sizeof(double)); s->Tp = calloc(3 * n, sizeof(double));
  double m0 = 0.0;
  for (int i = 0; i < s->n; ++i) {
    double a = p->radius[i];
    s->rad[i] = a;
    s->amap[i] = p->a_map_ratio * a;
    s->mass[i] = p->rho_p * 4.0 / 3.0 * M_PI * a * a * a;
    s->inert[i] = 0.4 * s->mass[i] * a * a;
    m0 += s->mass[i];
    for (int c = 0; c < 3; ++c) {
      s->R[3 * i + c] = p->pos[3 * i + c];
      s->U[3 * i + c] = p->vel ? p->vel[3 * i + c] : 0.0;
      s->W[3 * i + c] = p->omega ? p->omega[3 * i + c] : 0.0;
    }
  }
  if (s->n > 0) m0 /= s->n;
  s->mu = p->mu; s->kn = p->kn; s->kt = p->kt_ratio * p->kn;
  s->eta_n = p->eta_n >= 0.0 ? p->eta_n : sqrt(m0 * p->kn);  /* eta^(n) = sqrt(m0 kn) */
  s->F0 = p->F0; s->debye = p->debye;
  s->lub_delta = p->lub_delta; s->lub_cut = p->lub_cut;
  s->eta0 = p->rho0 * (p->tau - 0.5) / 3.0;
  s->quasi2d = p->quasi2d; s->move = p->move_particles;
  s->nbins = p->nbins > 0 ? p->nbins : 36;
  s->nsub = p->dem_substeps > 0 ? p->dem_substeps : auto_substeps(s);
  s->fA = calloc((size_t)Q * s->ncell, sizeof(double));
  s->fB = calloc((size_t)Q * s->ncell, sizeof(double));
  s->owner = malloc(sizeof(int) * s->ncell);
  for (int k = 0; k < 2; ++k) {
    s->hcnt[k] = calloc(n, sizeof(int));
    s->hpart[k] = calloc((size_t)n * HSLOTS, sizeof(int));
    s->hval[k] = calloc((size_t)n * HSLOTS * 3, sizeof(double));
  }
  s->hist = calloc(3 * s->nbins, sizeof(double));
  for (long c = 0; c < s->ncell; ++c) {
    s->owner[c] = -1;
    for (int q = 0; q < Q; ++q) s->fA[q * s->ncell + c] = weight(q) * s->rho0;
  }
  node_map_init(s);
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->rad); free(s->amap); free(s->mass); free(s->inert); free(s->drv);
  free(s->R); free(s->U); free(s->W); free(s->Fh); free(s->Th);
  free(s->Fcov); free(s->Tcov); free(s->Fp); free(s->Tp);
  free(s->fA); free(s->fB); free(s->owner);
  for (int k = 0; k < 2; ++k) { free(s->hcnt[k]); free(s->hpart[k]); free(s->hval[k]); }
  free(s->hist);
  free(s);
}

int orc_error(const orc_sim *s) { return s->err; }
long orc_ncell(const orc_sim *s) { return s->ncell; }
int orc_nsub(const orc_sim *s) { return s->nsub; }
long orc_time(const orc_sim *s) { return s->t; }
double orc_delta(const orc_sim *s) { return s->delta; }

void orc_get_populations(const orc_sim *s, double *f) {
  memcpy(f, s->fA, sizeof(double) * Q * s->ncell);
}
void orc_set_populations(orc_sim *s, const double *f) {
  memcpy(s->fA, f, sizeof(double) * Q * s->ncell);
}
void orc_get_owner(const orc_sim *s, int *o) { memcpy(o, s->owner, sizeof(int) * s->ncell); }
void orc_get_particles(const orc_sim *s, double *pos, double *vel, double *om) {
  if (pos) memcpy(pos, s->R, sizeof(double) * 3 * s->n);
  if (vel) memcpy(vel, s->U, sizeof(double) * 3 * s->n);
  if (om) memcpy(om, s->W, sizeof(double) * 3 * s->n);
}
void orc_get_hydro(const orc_sim *s, double *F, double *T) {
  if (F) memcpy(F, s->Fh, sizeof(double) * 3 * s->n);
  if (T) memcpy(T, s->Th, sizeof(double) * 3 * s->n);
}
void orc_get_pending(const orc_sim *s, double *F, double *T) {
  if (F) memcpy(F, s->Fcov, sizeof(double) * 3 * s->n);
  if (T) memcpy(T, s->Tcov, sizeof(double) * 3 * s->n);
}

/* ---------------- node map (solid / fluid / boundary, Appendix A) ------- */

/* Visit every cell within distance 'reach' of some image of particle i. */
typedef void (*cell_visitor)(orc_sim *s, int i, long c, const double d[3], int k, void *ctx);

static void visit_particle_cells(orc_sim *s, int i, double delta, double reach,
                                 cell_visitor fn, void *ctx) {
  for (int k = -1; k <= 1; ++k) {
    double cx = s->R[3 * i] + k * delta, cy = s->R[3 * i + 1] + k * (double)s->ny;
    double cz = s->R[3 * i + 2];
    int y0 = (int)ceil(cy - reach), y1 = (int)floor(cy + reach);
    if (y0 < 0) y0 = 0;
    if (y1 > s->ny - 1) y1 = s->ny - 1;
    if (y0 > y1) continue;
    int x0 = (int)ceil(cx - reach), x1 = (int)floor(cx + reach);
    int z0 = (int)ceil(cz - reach), z1 = (int)floor(cz + reach);
    for (int zz = z0; zz <= z1; ++zz)
      for (int yy = y0; yy <= y1; ++yy)
        for (int xx = x0; xx <= x1; ++xx) {
          int x = wrapi(xx, s->nx), z = wrapi(zz, s->nz);
          long c = cidx(s, x, yy, z);
          double d[3] = {x - s->R[3 * i], yy - s->R[3 * i + 1], z - s->R[3 * i + 2]};
          int kk = le_image(s, delta, d);
          fn(s, i, c, d, kk, ctx);
        }
  }
}

static void claim_initial(orc_sim *s, int i, long c, const double d[3], int k, void *ctx) {
  (void)k; (void)ctx;
  if (dot(d, d) < s->amap[i] * s->amap[i]) {
    if (s->owner[c] >= 0 && s->owner[c] != i) s->err |= ORC_EOVERLAP;
    else s->owner[c] = i;
  }
}

static void node_map_init(orc_sim *s) {
  for (int i = 0; i < s->n; ++i)
    visit_particle_cells(s, i, s->delta, s->amap[i] + 1.0, claim_initial, NULL);
}

typedef struct { double ule; } cover_ctx;

static void cover_cell(orc_sim *s, int i, long c, const double d[3], int k, void *ctx) {
  (void)k; (void)ctx;
  if (dot(d, d) >= s->amap[i] * s->amap[i]) return;
  if (s->owner[c] == i) return;
  if (s->owner[c] >= 0) { s->err |= ORC_EOVERLAP; return; }
  /* fluid node becomes solid: its momentum goes to the particle */
  double j[3] = {0, 0, 0};
  for (int q = 0; q < Q; ++q)
    for (int a = 0; a < 3; ++a) j[a] += s->fB[q * s->ncell + c] * CV[q][a];
  double tq[3];
  cross(d, j, tq);
  for (int a = 0; a < 3; ++a) { s->Fcov[3 * i + a] += j[a]; s->Tcov[3 * i + a] += tq[a]; }
  s->owner[c] = i;
}

/* After the particles moved: uncover, then cover (mapped radius a_map). */
static void node_map_update(orc_sim *s, double delta, double ule) {
  for (long c = 0; c < s->ncell; ++c) {
    int i = s->owner[c];
    if (i < 0) continue;
    int x = (int)(c % s->nx), y = (int)((c / s->nx) % s->ny), z = (int)(c / ((long)s->nx * s->ny));
    double d[3] = {x - s->R[3 * i], y - s->R[3 * i + 1], z - s->R[3 * i + 2]};
    int k = le_image(s, delta, d);
    if (dot(d, d) < s->amap[i] * s->amap[i]) continue;
    /* solid node becomes fluid: equilibrium at rho0 and the boundary velocity */
    double ub[3], wxd[3];
    cross(&s->W[3 * i], d, wxd);
    for (int a = 0; a < 3; ++a) ub[a] = s->U[3 * i + a] + wxd[a];
    ub[0] += k * ule;
    double j[3] = {s->rho0 * ub[0], s->rho0 * ub[1], s->rho0 * ub[2]};
    for (int q = 0; q < Q; ++q) s->fB[q * s->ncell + c] = feq1(q, s->rho0, j);
    double tq[3];
    cross(d, j, tq);
    for (int a = 0; a < 3; ++a) { s->Fcov[3 * i + a] -= j[a]; s->Tcov[3 * i + a] -= tq[a]; }
    s->owner[c] = -1;
  }
  for (int i = 0; i < s->n; ++i)
    visit_particle_cells(s, i, delta, s->amap[i] + 1.0, cover_cell, NULL);
}

/* ---------------- streaming sources with Lees-Edwards -------------------- */

typedef struct {
  int di;     /* integer part of Delta mod nx */
  double w;   /* fractional part              */
} le_shift;

static le_shift le_make(const orc_sim *s, double delta) {
  le_shift L;
  double dm = delta - s->nx * floor(delta / s->nx);
  L.di = (int)floor(dm);
  L.w = dm - L.di;
  return L;
}

/* Source of population p arriving at fluid node (x, y, z).
 * Returns the owner (>= 0) when the source is solid (bounce-back link),
 * -1 otherwise, with *val the pulled value (interpolated and Galilean
 * corrected across the Lees-Edwards planes). */
static int pull_source(const orc_sim *s, const double *f, int x, int y, int z, int p,
                       le_shift L, double ule, double *val) {
  int sx = x - CV[p][0], sy = y - CV[p][1], sz = wrapi(z - CV[p][2], s->nz);
  if (sy >= 0 && sy < s->ny) {
    long sc = cidx(s, wrapi(sx, s->nx), sy, sz);
    if (s->owner[sc] >= 0) return s->owner[sc];
    *val = f[p * s->ncell + sc];
    return -1;
  }
  int from_below = sy < 0;
  int ys = from_below ? s->ny - 1 : 0;
  int c0x;
  double w1;
  if (from_below) { c0x = wrapi(sx + L.di, s->nx); w1 = L.w; }
  else { c0x = wrapi(sx - L.di - 1, s->nx); w1 = 1.0 - L.w; }
  int c1x = wrapi(c0x + 1, s->nx);
  long c0 = cidx(s, c0x, ys, sz), c1 = cidx(s, c1x, ys, sz);
  long cn = w1 < 0.5 ? c0 : c1, co = w1 < 0.5 ? c1 : c0;
  if (s->owner[cn] >= 0) return s->owner[cn];
  double rho = 0, j[3] = {0, 0, 0}, v;
  if (s->owner[co] >= 0) {
    v = f[p * s->ncell + cn];
    for (int q = 0; q < Q; ++q) {
      double fq = f[q * s->ncell + cn];
      rho += fq;
      for (int a = 0; a < 3; ++a) j[a] += fq * CV[q][a];
    }
  } else {
    v = (1.0 - w1) * f[p * s->ncell + c0] + w1 * f[p * s->ncell + c1];
    for (int q = 0; q < Q; ++q) {
      double fq = (1.0 - w1) * f[q * s->ncell + c0] + w1 * f[q * s->ncell + c1];
      rho += fq;
      for (int a = 0; a < 3; ++a) j[a] += fq * CV[q][a];
    }
  }
  /* Galilean correction: the image below moves with -U_LE, above with +U_LE */
  double sgn = from_below ? -1.0 : 1.0;
  double j2[3] = {j[0] + sgn * rho * ule, j[1], j[2]};
  v += feq1(p, rho, j2) - feq1(p, rho, j);
  *val = v;
  return -1;
}

/* Boundary-node velocity u_b = U + Omega x (r_b - R), Eq. 8, at the link
 * midpoint r_b = r + c_q / 2 where c_q points from the fluid node r into the
 * solid; returns the arm r_b - R and the image index. */
static int link_geometry(const orc_sim *s, int i, int x, int y, int z, int q, double delta,
                         double ule, double arm[3], double ub[3]) {
  arm[0] = x + 0.5 * CV[q][0] - s->R[3 * i];
  arm[1] = y + 0.5 * CV[q][1] - s->R[3 * i + 1];
  arm[2] = z + 0.5 * CV[q][2] - s->R[3 * i + 2];
  int k = le_image(s, delta, arm);
  double wxa[3];
  cross(&s->W[3 * i], arm, wxa);
  for (int a = 0; a < 3; ++a) ub[a] = s->U[3 * i + a] + wxa[a];
  ub[0] += k * ule;
  return k;
}

/* ---------------- link momentum exchange (Eq. 6, 9, 10) ------------------ */

static void link_forces(orc_sim *s, double delta, double ule) {
  le_shift L = le_make(s, delta);
  for (int i = 0; i < 3 * s->n; ++i) { s->Fh[i] = 0.0; s->Th[i] = 0.0; }
  double slet[9] = {0};
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        long c = cidx(s, x, y, z);
        int own = s->owner[c];
        for (int p = 1; p < Q; ++p) {
          double v;
          int i = pull_source(s, s->fA, x, y, z, p, L, ule, &v);
          if (i < 0 || i == own) continue;
          int q = opposite(p); /* c_q points from node r into particle i's solid */
          double arm[3], ub[3];
          link_geometry(s, i, x, y, z, q, delta, ule, arm, ub);
          double mag;
          if (own < 0) {
            /* fluid node: momentum exchange of the bounced population */
            double cu = ub[0] * CV[q][0] + ub[1] * CV[q][1] + ub[2] * CV[q][2];
            mag = 2.0 * s->fA[q * s->ncell + c] - 6.0 * weight(q) * s->rho0 * cu;
          } else {
            /* node r of another particle j next to i's solid (mapped spheres
             * closer than one spacing, Appendix A (i)): r stands for a fluid
             * node in equilibrium at rho0 moving with the mean ubar of the two
             * surfaces' velocities at r_b, and the wall moves with ubar too:
             *   mag = 2 n^eq_q(rho0, rho0 ubar) - 6 C^q rho0 (ubar . c_q).
             * It is even in c_q, so the reverse link of j cancels it exactly
             * (momentum stays with the pair), and it equals what a fluid
             * link carries at rest (2 C^q rho0) or in a flow moving with
             * both surfaces, so the pressure on each particle balances */
            int j = own;
            double armj[3], ubj[3], ubar[3], jb[3];
            link_geometry(s, j, x, y, z, q, delta, ule, armj, ubj);
            for (int a = 0; a < 3; ++a) { ubar[a] = 0.5 * (ub[a] + ubj[a]); jb[a] = s->rho0 * ubar[a]; }
            double cub = ubar[0] * CV[q][0] + ubar[1] * CV[q][1] + ubar[2] * CV[q][2];
            mag = 2.0 * feq1(q, s->rho0, jb) - 6.0 * weight(q) * s->rho0 * cub;
          }
          double fv[3] = {mag * CV[q][0], mag * CV[q][1], mag * CV[q][2]};
          double tq[3];
          cross(arm, fv, tq);
          for (int a = 0; a < 3; ++a) { s->Fh[3 * i + a] += fv[a]; s->Th[3 * i + a] += tq[a]; }
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) slet[3 * a + b] += arm[a] * fv[b];
        }
      }
  for (int k = 0; k < 9; ++k) s->s_slet[k] += slet[k];
}

/* ---------------- collide + stream (Eq. 3, 4, 5, 7) ---------------------- */

static void stream_collide(orc_sim *s, double delta, double ule) {
  le_shift L = le_make(s, delta);
  double visc[9] = {0};
  double omega = 1.0 / s->tau;
  double vfac = -(1.0 - 0.5 / s->tau);
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        long c = cidx(s, x, y, z);
        if (s->owner[c] >= 0) continue;
        double nq[Q];
        nq[0] = s->fA[c];
        for (int p = 1; p < Q; ++p) {
          double v;
          int i = pull_source(s, s->fA, x, y, z, p, L, ule, &v);
          if (i >= 0) {
            /* moving bounce-back, Eq. 7 */
            int q = opposite(p);
            double arm[3], ub[3];
            link_geometry(s, i, x, y, z, q, delta, ule, arm, ub);
            double cu = ub[0] * CV[q][0] + ub[1] * CV[q][1] + ub[2] * CV[q][2];
            v = s->fA[q * s->ncell + c] - 6.0 * weight(q) * s->rho0 * cu;
          }
          nq[p] = v;
        }
        double rho = 0, j[3] = {0, 0, 0}, pi[9] = {0};
        for (int q = 0; q < Q; ++q) {
          rho += nq[q];
          for (int a = 0; a < 3; ++a) {
            j[a] += nq[q] * CV[q][a];
            for (int b = 0; b < 3; ++b) pi[3 * a + b] += nq[q] * CV[q][a] * CV[q][b];
          }
        }
        if (!(rho > 0.0)) s->err |= ORC_EUNSTABLE;
        if (s->collision == 1) {
          /* Ladd's linear operator (Eq. 5 by its eigenvalues): the
           * non-equilibrium stress relaxes with lambda = -1/tau in its
           * traceless part and lambda_v = -1/tau_bulk in its trace, every
           * other (ghost) mode is removed:
           *   n*_q = n^eq_q + C^q Pi*:(c_q c_q - c_s^2 I) / (2 c_s^4),
           *   Pi* = (1 + lambda) bar(Pi^neq) + (1 + lambda_v) tr(Pi^neq) I / 3;
           * viscous stress -(1 + lambda/2) bar(Pi^neq) - (1 + lambda_v/2) tr I / 3 */
          double lam = -1.0 / s->tau, lamv = -1.0 / s->tau_bulk;
          double pneq[9], pst[9];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              double peq = j[a] * j[b] / rho + (a == b ? rho / 3.0 : 0.0);
              pneq[3 * a + b] = pi[3 * a + b] - peq;
            }
          double tr = pneq[0] + pneq[4] + pneq[8];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              double bar = pneq[3 * a + b] - (a == b ? tr / 3.0 : 0.0);
              double iso = a == b ? tr / 3.0 : 0.0;
              pst[3 * a + b] = (1.0 + lam) * bar + (1.0 + lamv) * iso;
              visc[3 * a + b] += -(1.0 + 0.5 * lam) * bar - (1.0 + 0.5 * lamv) * iso;
            }
          double trs = pst[0] + pst[4] + pst[8];
          for (int q = 0; q < Q; ++q) {
            double fe = feq1(q, rho, j);
            double ccp = 0.0;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) ccp += pst[3 * a + b] * CV[q][a] * CV[q][b];
            double gc = s->g[0] * CV[q][0] + s->g[1] * CV[q][1] + s->g[2] * CV[q][2];
            s->fB[q * s->ncell + c] = fe + 4.5 * weight(q) * (ccp - trs / 3.0) + 3.0 * weight(q) * gc;
          }
        } else {
          /* BGK: viscous stress -(1 - 1/(2 tau)) Pi^neq */
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              double peq = j[a] * j[b] / rho + (a == b ? rho / 3.0 : 0.0);
              visc[3 * a + b] += vfac * (pi[3 * a + b] - peq);
            }
          for (int q = 0; q < Q; ++q) {
            double fe = feq1(q, rho, j);
            double gc = s->g[0] * CV[q][0] + s->g[1] * CV[q][1] + s->g[2] * CV[q][2];
            s->fB[q * s->ncell + c] = nq[q] - omega * (nq[q] - fe) + 3.0 * weight(q) * gc;
          }
        }
      }
  for (int k = 0; k < 9; ++k) s->s_visc[k] += visc[k];
}

/* ---------------- contacts (Eq. 11, 11t and the linear spring model) ----- */

int orc_contact(double ra, double rb, const double d[3], const double uab[3],
                const double wa[3], const double wb[3], double kn, double kt,
                double eta_n, double mu, double dt, double ht[3], double Fa[3],
                double Ta[3], double Tb[3], double *fn_mag, double Ftan[3]) {
  double dist = sqrt(dot(d, d));
  double overlap = ra + rb - dist;
  for (int a = 0; a < 3; ++a) { Fa[a] = 0; Ta[a] = 0; Tb[a] = 0; Ftan[a] = 0; }
  *fn_mag = 0;
  if (!(overlap > 0.0)) { ht[0] = ht[1] = ht[2] = 0.0; return 0; }
  double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};   /* from a towards b */
  /* relative velocity of a's surface with respect to b's at the contact */
  double wsum[3] = {ra * wa[0] + rb * wb[0], ra * wa[1] + rb * wb[1], ra * wa[2] + rb * wb[2]};
  double rot[3];
  cross(wsum, n, rot);
  double v[3] = {uab[0] + rot[0], uab[1] + rot[1], uab[2] + rot[2]};
  double vn = dot(v, n);
  double vt[3] = {v[0] - vn * n[0], v[1] - vn * n[1], v[2] - vn * n[2]};
  /* normal force: spring on the overlap plus dashpot on the approach speed */
  double fn = kn * overlap + eta_n * vn;
  /* tangential spring: project onto the tangent plane, then integrate v_t */
  double hn = dot(ht, n);
  for (int a = 0; a < 3; ++a) ht[a] = ht[a] - hn * n[a] + vt[a] * dt;
  double ftr[3] = {-kt * ht[0], -kt * ht[1], -kt * ht[2]};
  double ftm = sqrt(dot(ftr, ftr));
  double cap = mu * fabs(fn);
  if (ftm >= cap && ftm > 0.0) {
    /* Coulomb slip: |F_t| = mu |F_n|, spring reset to the slip length */
    for (int a = 0; a < 3; ++a) {
      Ftan[a] = cap * ftr[a] / ftm;
      ht[a] = -Ftan[a] / kt;
    }
  } else {
    for (int a = 0; a < 3; ++a) Ftan[a] = ftr[a];
  }
  for (int a = 0; a < 3; ++a) Fa[a] = -fn * n[a] + Ftan[a];
  double tq[3];
  cross(n, Ftan, tq);
  for (int a = 0; a < 3; ++a) { Ta[a] = ra * tq[a]; Tb[a] = rb * tq[a]; }
  *fn_mag = fn;
  return 1;
}

/* ---------------- lubrication correction (Appendix A) --------------------
 * Leading-order scalar resistances with beta = a_b / a_a, gap normalised
 * by the mean radius, roughness delta regularising 1/h and ln(1/h), and
 * the value at the cutoff subtracted so that the correction vanishes there. */
void orc_lubrication(double ra, double rb, const double d[3], const double uab[3],
                     const double wa[3], const double wb[3], double eta0,
                     double delta, double hcut, double Fa[3], double Ta[3], double Tb[3]) {
  for (int a = 0; a < 3; ++a) { Fa[a] = 0; Ta[a] = 0; Tb[a] = 0; }
  double dist = sqrt(dot(d, d));
  double h = dist - ra - rb;
  if (!(h < hcut)) return;
  if (h < 0.0) h = 0.0;
  double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
  double sc = 2.0 / (ra + rb);
  double xi = sc * h, xc = sc * hcut, dl = sc * delta;
  double inv = 1.0 / (xi + dl) - 1.0 / (xc + dl);
  double lg = log((xc + dl) / (xi + dl));
  double be = rb / ra, bj = ra / rb;
  double XA = eta0 * 6.0 * M_PI * ra * (2.0 * be * be / pow(1.0 + be, 3)) * inv;
  double YA = eta0 * 6.0 * M_PI * ra * (4.0 * be * (2.0 + be + 2.0 * be * be) / (15.0 * pow(1.0 + be, 3))) * lg;
  double YBa = eta0 * 4.0 * M_PI * ra * ra * (be * (4.0 + be) / (5.0 * pow(1.0 + be, 2))) * lg;
  double YBb = eta0 * 4.0 * M_PI * rb * rb * (bj * (4.0 + bj) / (5.0 * pow(1.0 + bj, 2))) * lg;
  double YCaa = eta0 * 8.0 * M_PI * ra * ra * ra * (2.0 * be / (5.0 * (1.0 + be))) * lg;
  double YCbb = eta0 * 8.0 * M_PI * rb * rb * rb * (2.0 * bj / (5.0 * (1.0 + bj))) * lg;
  double YCab = eta0 * 8.0 * M_PI * ra * ra * ra * (be * be / (10.0 * (1.0 + be))) * lg;
  double un = dot(uab, n);
  double ut[3] = {uab[0] - un * n[0], uab[1] - un * n[1], uab[2] - un * n[2]};
  double wan[3], wbn[3], nxu[3];
  cross(wa, n, wan);
  cross(wb, n, wbn);
  cross(n, uab, nxu);
  double wap = dot(wa, n), wbp = dot(wb, n);
  for (int a = 0; a < 3; ++a) {
    Fa[a] = -XA * un * n[a] - YA * ut[a] - YBa * wan[a] - YBb * wbn[a];
    double wa_t = wa[a] - wap * n[a], wb_t = wb[a] - wbp * n[a];
    Ta[a] = -YBa * nxu[a] - YCaa * wa_t - YCab * wb_t;
    Tb[a] = -YBb * nxu[a] - YCbb * wb_t - YCab * wa_t;
  }
}

/* Lubrication stresslet of the pair (Appendix A, G and H blocks), the same
 * correction form and normalisation as the forces: for each sphere p of the
 * pair, with n_p its unit normal towards the partner and a_p, beta_p = a_q /
 * a_p its own radius and ratio,
 *   S_p = -[ G(n_p) . (U_p - U_q) + H_pp(n_p) . Omega_p + H_pq(n_p) . Omega_q ],
 *   G . U = X^G (n n - I/3)(n . U) + Y^G (n U + U n - 2 n n (n . U)),
 *   H . Omega = Y^H ((Omega x n) n + n (Omega x n)).
 * Out: S = S_a + S_b (3 x 3, symmetric and traceless). */
void orc_lubrication_stresslet(double ra, double rb, const double d[3], const double uab[3],
                               const double wa[3], const double wb[3], double eta0,
                               double delta, double hcut, double S[9]) {
  for (int k = 0; k < 9; ++k) S[k] = 0.0;
  double dist = sqrt(dot(d, d));
  double h = dist - ra - rb;
  if (!(h < hcut)) return;
  if (h < 0.0) h = 0.0;
  double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
  double sc = 2.0 / (ra + rb);
  double xi = sc * h, xc = sc * hcut, dl = sc * delta;
  double inv = 1.0 / (xi + dl) - 1.0 / (xc + dl);
  double lg = log((xc + dl) / (xi + dl));
  double un = dot(uab, n);
  for (int p = 0; p < 2; ++p) {
    double ap = p == 0 ? ra : rb, be = p == 0 ? rb / ra : ra / rb;
    const double *wp = p == 0 ? wa : wb, *wq = p == 0 ? wb : wa;
    /* n_p = +/- n and U_p - U_q = +/- uab: the G terms are odd in each, the
     * H terms even in n_p, so both spheres use n and uab */
    double XG = eta0 * 4.0 * M_PI * ap * ap * (3.0 * be * be / pow(1.0 + be, 3)) * inv;
    double YG = eta0 * 4.0 * M_PI * ap * ap * (be * (4.0 - be + 7.0 * be * be) / (10.0 * pow(1.0 + be, 3))) * lg;
    double YHs = eta0 * 8.0 * M_PI * ap * ap * ap * (be * (2.0 - be) / (10.0 * pow(1.0 + be, 2))) * lg;
    double YHo = eta0 * 8.0 * M_PI * ap * ap * ap * (be * be * (1.0 + 7.0 * be) / (20.0 * pow(1.0 + be, 2))) * lg;
    double ws[3], wo[3];
    cross(wp, n, ws);
    cross(wq, n, wo);
    for (int x = 0; x < 3; ++x)
      for (int y = 0; y < 3; ++y) {
        double g = XG * (n[x] * n[y] - (x == y ? 1.0 / 3.0 : 0.0)) * un
                 + YG * (n[x] * uab[y] + uab[x] * n[y] - 2.0 * n[x] * n[y] * un);
        double hh = YHs * (ws[x] * n[y] + n[x] * ws[y]) + YHo * (wo[x] * n[y] + n[x] * wo[y]);
        S[3 * x + y] -= g + hh;
      }
  }
}

/* ---------------- particle sub-steps (Eq. 1) ----------------------------- */

static int hist_find(const orc_sim *s, int buf, int a, int b) {
  for (int k = 0; k < s->hcnt[buf][a]; ++k)
    if (s->hpart[buf][a * HSLOTS + k] == b) return k;
  return -1;
}

static void pair_forces(orc_sim *s, double delta, double ule, double dt, int sample) {
  int cur = s->hcur, nxt = 1 - cur;
  for (int i = 0; i < 3 * s->n; ++i) { s->Fp[i] = 0.0; s->Tp[i] = 0.0; }
  for (int i = 0; i < s->n; ++i) s->hcnt[nxt][i] = 0;
  double hrange = 0.0;
  if (s->lub_cut > hrange) hrange = s->lub_cut;
  if (s->F0 > 0.0 && 10.0 * s->debye > hrange) hrange = 10.0 * s->debye;
  double dth = M_PI / s->nbins;
  for (int a = 0; a < s->n; ++a)
    for (int b = a + 1; b < s->n; ++b) {
      double d[3] = {s->R[3 * b] - s->R[3 * a], s->R[3 * b + 1] - s->R[3 * a + 1],
                     s->R[3 * b + 2] - s->R[3 * a + 2]};
      /* minimum image of b as seen from a; b's image moves with U_b + k U_LE */
      int k = (int)floor(d[1] / s->ny + 0.5);
      d[1] -= k * (double)s->ny;
      d[0] -= k * delta;
      d[0] = nearest(d[0], s->nx);
      d[2] = nearest(d[2], s->nz);
      double dist = sqrt(dot(d, d));
      double h = dist - s->rad[a] - s->rad[b];
      if (!(h < hrange) && !(h < 0.0)) continue;
      double uab[3] = {s->U[3 * a] - s->U[3 * b] - k * ule, s->U[3 * a + 1] - s->U[3 * b + 1],
                       s->U[3 * a + 2] - s->U[3 * b + 2]};
      const double *wa = &s->W[3 * a], *wb = &s->W[3 * b];
      double Fa[3], Ta[3], Tb[3];
      /* contact */
      double ht[3] = {0, 0, 0};
      int slot = hist_find(s, cur, a, b);
      if (slot >= 0)
        for (int c = 0; c < 3; ++c) ht[c] = s->hval[cur][(a * HSLOTS + slot) * 3 + c];
      double fn, Ft[3];
      int touching = orc_contact(s->rad[a], s->rad[b], d, uab, wa, wb, s->kn, s->kt, s->eta_n,
                                 s->mu, dt, ht, Fa, Ta, Tb, &fn, Ft);
      if (touching) {
        int m = s->hcnt[nxt][a];
        if (m >= HSLOTS) { s->err |= ORC_EHIST; }
        else {
          s->hpart[nxt][a * HSLOTS + m] = b;
          for (int c = 0; c < 3; ++c) s->hval[nxt][(a * HSLOTS + m) * 3 + c] = ht[c];
          s->hcnt[nxt][a] = m + 1;
        }
        for (int c = 0; c < 3; ++c) {
          s->Fp[3 * a + c] += Fa[c]; s->Fp[3 * b + c] -= Fa[c];
          s->Tp[3 * a + c] += Ta[c]; s->Tp[3 * b + c] += Tb[c];
        }
        if (sample) {
          /* contact virial with r = R_a - R_b and the force on a (Eq. 12) */
          double r[3] = {-d[0], -d[1], -d[2]};
          for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y)
              s->s_cont[3 * x + y] += 0.5 * (r[x] * Fa[y] + r[y] * Fa[x]);
          /* angular distributions (Eq. 19-23): theta of r folded into [0, pi);
           * the tangential force counted positive when it turns the spheres
           * counter-clockwise (Sec. 3.2): a's contact point lies at -a n from
           * its centre, so that is -(F_a . t) with t = (-sin, cos) of the
           * unfolded angle (the same value from b's side, whose angle is
           * folded by pi and whose force is -F_a) */
          double th = atan2(r[1], r[0]);
          double tx = -sin(th), ty = cos(th);
          if (th < 0.0) th += M_PI;
          if (th >= M_PI) th -= M_PI;
          int bin = (int)floor(th / dth);
          if (bin >= s->nbins) bin = s->nbins - 1;
          if (bin < 0) bin = 0;
          s->hist[3 * bin] += 1.0;
          s->hist[3 * bin + 1] += fn;
          s->hist[3 * bin + 2] -= Fa[0] * tx + Fa[1] * ty;
          s->ncontacts += 1;
        }
      }
      /* double-layer repulsion (Eq. 13) */
      if (s->F0 > 0.0 && h < 10.0 * s->debye) {
        double fr = s->F0 * exp(-(h > 0.0 ? h : 0.0) / s->debye);
        double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
        for (int c = 0; c < 3; ++c) { s->Fp[3 * a + c] -= fr * n[c]; s->Fp[3 * b + c] += fr * n[c]; }
        if (sample) {
          double r[3] = {-d[0], -d[1], -d[2]};
          double F[3] = {-fr * n[0], -fr * n[1], -fr * n[2]};
          for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) s->s_rep[3 * x + y] += 0.5 * (r[x] * F[y] + r[y] * F[x]);
        }
      }
      /* lubrication correction */
      if (s->lub_cut > 0.0 && h < s->lub_cut) {
        orc_lubrication(s->rad[a], s->rad[b], d, uab, wa, wb, s->eta0, s->lub_delta,
                        s->lub_cut, Fa, Ta, Tb);
        for (int c = 0; c < 3; ++c) {
          s->Fp[3 * a + c] += Fa[c]; s->Fp[3 * b + c] -= Fa[c];
          s->Tp[3 * a + c] += Ta[c]; s->Tp[3 * b + c] += Tb[c];
        }
        if (sample) {
          double S[9];
          orc_lubrication_stresslet(s->rad[a], s->rad[b], d, uab, wa, wb, s->eta0, s->lub_delta,
                                    s->lub_cut, S);
          for (int k = 0; k < 9; ++k) s->s_lub[k] += S[k];
        }
      }
    }
  s->hcur = nxt;
}

static void particles_step(orc_sim *s, double delta, double ule, double delta_next) {
  double dt = 1.0 / s->nsub;
  for (int sub = 0; sub < s->nsub; ++sub) {
    pair_forces(s, delta, ule, dt, sub == 0);
    for (int i = 0; i < s->n; ++i) {
      double F[3], T[3];
      for (int a = 0; a < 3; ++a) {
        F[a] = s->Fh[3 * i + a] + s->Fcov[3 * i + a] + s->Fp[3 * i + a];
        T[a] = s->Th[3 * i + a] + s->Tcov[3 * i + a] + s->Tp[3 * i + a];
      }
      if (!s->drv[i]) {
        for (int a = 0; a < 3; ++a) {
          s->U[3 * i + a] += dt * F[a] / s->mass[i];
          s->W[3 * i + a] += dt * T[a] / s->inert[i];
        }
        if (s->quasi2d) { s->U[3 * i + 2] = 0.0; s->W[3 * i] = 0.0; s->W[3 * i + 1] = 0.0; }
      }
      /* a driven particle (wall) keeps its velocity and spin */
      for (int a = 0; a < 3; ++a) s->R[3 * i + a] += dt * s->U[3 * i + a];
    }
  }
  for (int i = 0; i < 3 * s->n; ++i) { s->Fcov[i] = 0.0; s->Tcov[i] = 0.0; }
  /* Lees-Edwards wrap of the centres, then periodic x, z */
  for (int i = 0; i < s->n; ++i) {
    double *R = &s->R[3 * i];
    const double du = s->drv[i] ? 0.0 : ule;   /* a driven particle keeps its velocity */
    if (R[1] >= s->ny) { R[1] -= s->ny; R[0] -= delta_next; s->U[3 * i] -= du; }
    else if (R[1] < 0.0) { R[1] += s->ny; R[0] += delta_next; s->U[3 * i] += du; }
    R[0] -= s->nx * floor(R[0] / s->nx);
    R[2] -= s->nz * floor(R[2] / s->nz);
    double sp = sqrt(dot(&s->U[3 * i], &s->U[3 * i]));
    if (!(sp < 0.5)) s->err |= ORC_EUNSTABLE;
  }
}

/* ---------------- one full step ------------------------------------------ */

/* Total shear stress sigma_xy of the sums so far, times V (the stresslet
 * symmetrised; the contact and double-layer virials enter with a minus). */
static double sigma_xy_sum(const orc_sim *s) {
  return s->s_visc[1] + 0.5 * (s->s_slet[1] + s->s_slet[3]) - s->s_cont[1] - s->s_rep[1] + s->s_lub[1];
}

int orc_step(orc_sim *s, int nsteps, const orc_shear *sh) {
  for (int it = 0; it < nsteps; ++it) {
    const double sxy_before = sigma_xy_sum(s);
    double delta = s->delta;
    double ule = orc_le_increment(sh, s->t, s->ny);
    double dn = s->delta, dc = s->delta_c;
    le_advance(s, &dn, &dc, ule);
    double ule_next = orc_le_increment(sh, s->t + 1, s->ny);
    /* 1. link momentum exchange on n*(t) */
    link_forces(s, delta, ule);
    /* 2. collide + stream with moving bounce-back and Lees-Edwards */
    stream_collide(s, delta, ule);
    /* 3. particles */
    if (s->move) particles_step(s, delta, ule, dn);
    else
      for (int i = 0; i < 3 * s->n; ++i) { s->Fcov[i] = 0.0; s->Tcov[i] = 0.0; }
    /* 4. node map at t+1 */
    node_map_update(s, dn, ule_next);
    double *tmp = s->fA; s->fA = s->fB; s->fB = tmp;
    s->delta = dn; s->delta_c = dc;
    /* the step t -> t+1 shears by gamma(t+1) - gamma(t): its stress belongs
     * to the midpoint t + 1/2 of the protocol's phase */
    {
      const double sxy = sigma_xy_sum(s) - sxy_before;
      const double om = sh->kind == 1 ? sh->omega : 0.0, th = sh->kind == 1 ? sh->theta : 0.0;
      const double ph = om * ((double)s->t + 0.5) + th;
      s->s_gc += sxy * cos(ph);
      s->s_gs += sxy * sin(ph);
    }
    s->t += 1;
    s->nsamples += 1;
  }
  return s->err;
}

/* Storage and loss moduli, Eq. 17 and 18, over the steps since the last
 * reset (a whole number of periods): the integral over one period divided by
 * 2 pi / omega is twice the time average, so G' = -2 <sigma_xy cos> / gamma0
 * and G'' = 2 <sigma_xy sin> / gamma0, the average over the window's steps. */
int orc_moduli(const orc_sim *s, double gamma0, double *Gp, double *Gpp) {
  *Gp = *Gpp = 0.0;
  if (!(gamma0 > 0.0)) return -1;
  if (s->nsamples == 0) return 0;
  const double V = (double)s->nx * s->ny * s->nz;
  const double norm = 1.0 / (V * (double)s->nsamples);
  *Gp = -2.0 * norm * s->s_gc / gamma0;
  *Gpp = 2.0 * norm * s->s_gs / gamma0;
  return 0;
}

/* ---------------- stress (Eq. 12, 14, 15, 26, 27) ------------------------ */

void orc_stress_reset(orc_sim *s) {
  for (int k = 0; k < 9; ++k) { s->s_visc[k] = s->s_slet[k] = s->s_cont[k] = s->s_rep[k] = s->s_lub[k] = 0.0; }
  s->s_gc = s->s_gs = 0.0;
  for (int b = 0; b < 3 * s->nbins; ++b) s->hist[b] = 0.0;
  s->nsamples = 0;
  s->ncontacts = 0;
}

void orc_angular_stress(const double *hist, int nbins, double phi, double z_coord, double a,
                        int two_d, double out[9]) {
  for (int k = 0; k < 9; ++k) out[k] = 0.0;
  double nc = 0.0, sfn = 0.0;
  for (int b = 0; b < nbins; ++b) { nc += hist[3 * b]; sfn += hist[3 * b + 1]; }
  if (!(nc > 0.0)) return;
  double dth = M_PI / nbins;
  double fmean = sfn / nc;                              /* <F^nor> = int rho F^nor */
  double pref = two_d ? phi * z_coord * fmean / (M_PI * a)
                      : 3.0 * phi * z_coord * fmean / (2.0 * M_PI * a * a);
  for (int b = 0; b < nbins; ++b) {
    double th = (b + 0.5) * dth;
    double zn = hist[3 * b + 1] / (nc * dth * fmean);   /* zeta_N = rho xi_N */
    double zt = hist[3 * b + 2] / (nc * dth * fmean);   /* zeta_T = rho xi_T */
    double nv[2] = {cos(th), sin(th)}, tv[2] = {-sin(th), cos(th)};
    for (int al = 0; al < 2; ++al)
      for (int be = 0; be < 2; ++be)
        out[3 * al + be] += pref * (zn * nv[al] - zt * tv[al]) * nv[be] * dth;
  }
}

int orc_stress(const orc_sim *s, int kind, double out[9], double *hist, int nbins) {
  for (int k = 0; k < 9; ++k) out[k] = 0.0;
  if (hist && nbins == s->nbins)
    for (int b = 0; b < 3 * nbins; ++b) hist[b] = s->hist[b];
  if (s->nsamples == 0) return 0;
  double V = (double)s->nx * s->ny * s->nz;
  double norm = 1.0 / (V * (double)s->nsamples);
  double visc[9], cont[9], rep[9], lub[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      int k = 3 * a + b, kt = 3 * b + a;
      /* particle stresslet (symmetric part) + fluid viscous stress */
      visc[k] = norm * (s->s_visc[k] + 0.5 * (s->s_slet[k] + s->s_slet[kt]));
      cont[k] = -norm * s->s_cont[k];
      rep[k] = -norm * s->s_rep[k];
      lub[k] = norm * s->s_lub[k];     /* the pairs' lubrication stresslets */
    }
  if (kind == ORC_VISCOUS) memcpy(out, visc, sizeof visc);
  else if (kind == ORC_CONTACT) memcpy(out, cont, sizeof cont);
  else if (kind == ORC_REPULSIVE) memcpy(out, rep, sizeof rep);
  else if (kind == ORC_LUBRICATION) memcpy(out, lub, sizeof lub);
  else if (kind == ORC_TOTAL) for (int k = 0; k < 9; ++k) out[k] = visc[k] + cont[k] + rep[k] + lub[k];
  else if (kind == ORC_ANGULAR) {
    double asum = 0.0, vol = 0.0, area = 0.0;
    for (int i = 0; i < s->n; ++i) {
      asum += s->rad[i];
      vol += 4.0 / 3.0 * M_PI * pow(s->rad[i], 3);
      area += M_PI * s->rad[i] * s->rad[i];
    }
    if (s->n == 0) return 0;
    double amean = asum / s->n;
    double zc = 2.0 * (double)s->ncontacts / ((double)s->n * (double)s->nsamples);
    if (s->quasi2d)
      orc_angular_stress(s->hist, s->nbins, area / ((double)s->nx * s->ny), zc, amean, 1, out);
    else
      orc_angular_stress(s->hist, s->nbins, vol / V, zc, amean, 0, out);
  } else return -1;
  return 0;
}

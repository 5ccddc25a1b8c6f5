/*
 * pic_oracle.c -- plain, slow FP64 CPU oracle of the electrostatic PIC/MCC step.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * CPU-baseline and reference legs of the benchmark load this library. It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * seeded input arrays.
 *
 * What it follows (Koitermaa et al., "Coupled simulation of plasma-surface
 * interactions during early stages of vacuum arcing"):
 *   - Eq. (1): Poisson's equation  lap(phi) = -rho/eps0 in the vacuum gap with
 *     Dirichlet electrode potentials (anode at +V0, cathode grounded).
 *   - PIC/MCC paragraph: superparticles injected from the cathode (emitted
 *     electrons, evaporated Cu neutrals), moved by electric forces, colliding by
 *     Monte Carlo collisions with probability Eq. (4)
 *         P = 1 - exp(-u n sigma(E) dt_PIC)
 *     (electron-impact ionization and elastic scattering; resonant charge
 *     exchange of an ion on a neutral of its own element, one of the MCC
 *     collisions the paragraph lists).
 *   - Ions leave the plasma domain when they hit the cathode (Appendix A).
 * The paper fixes neither discretisation nor step order; the readings used here
 * (structured node grid, 7-point Laplacian, cloud-in-cell shape, leapfrog push,
 * NGP neutral density, deterministic victim choice, Philox4x32-10 counters)
 * are listed with every function below.
 *
 * Everything is FP64. Loops are plain and unblocked. Sorting uses qsort,
 * the Poisson solve is unpreconditioned conjugate gradients.
 * Build with -ffp-contract=off so the rounding does not depend on the host.
 *
 * The same source also builds with -fopenmp (a timing baseline on all host
 * cores). Only loops whose iterations are independent run in parallel, and
 * every sum has one fixed order in both builds (dot products add fixed chunks
 * of OR_CHUNK terms, then the chunk sums in order; the push advances particles
 * in parallel and does its counts, energy sums, logs and event lists in a
 * serial pass in particle order), so both builds give bit-identical results
 * with any number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP build (n <= 0: all it may use); 1 in the serial build. */
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

#define OR_QE 1.602176634e-19
#define OR_EPS0 8.8541878128e-12
#define OR_PI 3.14159265358979323846

#define OR_MAXSP 8
#define OR_MAXXS 8
#define OR_MAXSRC 16

enum { OR_ELECTRON = 0, OR_NEUTRAL = 1, OR_ION = 2 };
/* Collision channels. Charge exchange is the resonant ion-atom kind named
 * among the paper's MCC collisions (the PIC/MCC paragraph with Eq. 4): the ion
 * takes an electron from a neutral of its own element and both keep their
 * velocities, so a fast neutral and a slow ion come out. */
enum { OR_XS_IONIZATION = 0, OR_XS_ELASTIC = 1, OR_XS_CX = 2 };

/* Philox counter layout: (pid, step, tag, j). Tags name the purpose of a draw. */
enum {
  TAG_MCC = 0,       /* (U1, -): collision test and channel choice */
  TAG_SCATTER = 1,   /* (cos theta, phi) of an elastic scattering */
  TAG_IONIZE = 2,    /* j=0: (U_split, cos theta), j=1: (phi, -) of the secondary */
  TAG_INJ_POS = 16,  /* (radius, angle) on the emitter disk */
  TAG_INJ_VXY = 17,  /* Box-Muller pair for vx, vy */
  TAG_INJ_VZ = 18,   /* Box-Muller pair, cos branch -> |vz| */
  TAG_INJ_Z = 19,    /* fraction of the first partial step */
  TAG_VICTIM = 32    /* 32-bit key ranking neutrals as ionization victims */
};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random numbers: */
/* as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies with the key   */
/* bumped by the Weyl constants between rounds.                               */
/* ------------------------------------------------------------------------ */
void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on (0,1) from two 32-bit words: the top 52 bits m give
 * U = (m + 1/2) 2^-52, which FP64 represents exactly. */
double or_u01(uint32_t a, uint32_t b) {
  uint64_t m = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
  return ((double)m + 0.5) * (1.0 / 4503599627370496.0);
}

typedef struct { double u0, u1; uint32_t w[4]; } draw2;

static draw2 draw(uint64_t seed, uint32_t pid, uint32_t step, uint32_t tag, uint32_t j) {
  uint32_t ctr[4] = {pid, step, tag, j};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  draw2 d;
  or_philox(ctr, key, d.w);
  d.u0 = or_u01(d.w[0], d.w[1]);
  d.u1 = or_u01(d.w[2], d.w[3]);
  return d;
}

/* ------------------------------------------------------------------------ */
/* State                                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  double q, m, w;
  int role;
} or_species_t;

typedef struct {
  int kind, projectile, target, product;
  double thr;
  int n;
  double* E;
  double* sig;
} or_xsec_t;

typedef struct {
  int species;
  double cx, cy, R, flux, T;
  double acc; /* carry accumulator of the fractional expected count */
} or_source_t;

typedef struct {
  int64_t n, cap;
  double *x, *y, *z, *vx, *vy, *vz;
  uint32_t* pid;
  uint32_t* mw; /* multiplicity: the particle stands for mw x w physical particles (1 unless uploaded otherwise) */
} or_store_t;

/* Public configuration (mirrors nothing in the GPU library; plain fields). */
typedef struct {
  int32_t nx, ny, nz;
  double h, dt, phi_c, phi_a, rho_bg;
  int32_t sort_interval;
  double cg_rtol;
  int32_t cg_maxit;
  uint64_t seed;
  int32_t warm_zero; /* 1: solve from phi = 0 each step; 0: from the previous phi */
  int32_t nsp;
  double q[OR_MAXSP], m[OR_MAXSP], w[OR_MAXSP];
  int32_t role[OR_MAXSP];
  int32_t variable_weights; /* 1: particles carry multiplicities (events between unequal ones split) */
} or_cfg_t;

typedef struct {
  int64_t count[OR_MAXSP];
  int64_t injected[OR_MAXSP];
  int64_t abs_cathode[OR_MAXSP], abs_anode[OR_MAXSP];
  double abs_energy_cathode[OR_MAXSP], abs_energy_anode[OR_MAXSP];
  int64_t n_ionization, n_elastic, n_suppressed;
  int64_t step;
  int32_t cg_iters;
  double cg_resid_rel;
  double total_charge;
  double kinetic[OR_MAXSP];
  double field_energy;
  double charge_to_cathode_last, charge_to_anode_last; /* C absorbed in the last step */
  uint32_t next_pid;
  double anode_V;  /* anode potential the next solve uses */
  int64_t n_cx;    /* charge exchanges */
} or_moments_t;

typedef struct {
  uint32_t pid;
  int32_t sp;
  uint32_t step;      /* the step in which the ion crossed z = 0 */
  double x, y;        /* where the straight path x^n -> x^{n+1} crosses z = 0, wrapped */
  double vx, vy, vz;  /* v^{n+1/2} */
} or_hit_t;

typedef struct {
  or_cfg_t c;
  or_species_t sp[OR_MAXSP];
  or_xsec_t xs[OR_MAXXS];
  int nxs;
  or_source_t src[OR_MAXSRC];
  int nsrc;
  or_store_t st[OR_MAXSP];
  int64_t ncell, nnode;
  double* rho;             /* (nz+1)*ny*nx nodes */
  int32_t* ncount[OR_MAXSP];/* per-cell neutral counts (neutral species only) */
  double* phi;             /* (nz+1)*ny*nx nodes, Dirichlet planes included */
  int64_t* cell_start[OR_MAXSP];
  uint32_t step;
  uint32_t next_pid;
  or_moments_t mom;
  /* background-density test mode: MCC targets see a fixed density */
  double bg_density;
  /* last ionization-event log: (primary pid, victim pid, secondary pid) */
  int64_t nlog;
  uint32_t* log;
  /* ions absorbed at the cathode since the last or_get_hits: the surface
   * coupling output (ions that bombard the cathode are handed to the surface
   * model: the PIC/MCC paragraph after Eq. 4 and Appendix A) */
  int64_t nhit, hitcap;
  or_hit_t* hit;
  /* external circuit (the serial RC circuit between the electrodes, in the
   * paragraph describing the simulated system):
   * a source V0 charges the anode through R, the gap holds capacitance C, and
   * the charge the anode collects in a step flows onto it:
   * V <- V + (dt (V0 - V) / R + Q_anode) / C once per step, after the push.
   * Off (constant anode potential) unless R > 0 and C > 0. */
  int circuit_on;
  double circ_R, circ_C, circ_V0;
  double anode_V;  /* anode potential of the next solve */
} or_state_t;

static void store_reserve(or_store_t* s, int64_t need) {
  if (need <= s->cap) return;
  int64_t cap = s->cap ? s->cap : 64;
  while (cap < need) cap *= 2;
  s->x = realloc(s->x, cap * sizeof(double));
  s->y = realloc(s->y, cap * sizeof(double));
  s->z = realloc(s->z, cap * sizeof(double));
  s->vx = realloc(s->vx, cap * sizeof(double));
  s->vy = realloc(s->vy, cap * sizeof(double));
  s->vz = realloc(s->vz, cap * sizeof(double));
  s->pid = realloc(s->pid, cap * sizeof(uint32_t));
  s->mw = realloc(s->mw, cap * sizeof(uint32_t));
  s->cap = cap;
}

static void store_push(or_store_t* s, double x, double y, double z, double vx, double vy, double vz,
                       uint32_t pid, uint32_t mw) {
  store_reserve(s, s->n + 1);
  int64_t i = s->n++;
  s->x[i] = x; s->y[i] = y; s->z[i] = z;
  s->vx[i] = vx; s->vy[i] = vy; s->vz[i] = vz;
  s->pid[i] = pid;
  s->mw[i] = mw;
}

static void store_free(or_store_t* s) {
  free(s->x); free(s->y); free(s->z); free(s->vx); free(s->vy); free(s->vz); free(s->pid); free(s->mw);
  memset(s, 0, sizeof(*s));
}

or_state_t* or_create(const or_cfg_t* cfg) {
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 2 || cfg->nsp < 1 || cfg->nsp > OR_MAXSP) return NULL;
  or_state_t* s = calloc(1, sizeof(or_state_t));
  s->anode_V = cfg->phi_a;
  s->c = *cfg;
  for (int i = 0; i < cfg->nsp; ++i) {
    s->sp[i].q = cfg->q[i]; s->sp[i].m = cfg->m[i]; s->sp[i].w = cfg->w[i]; s->sp[i].role = cfg->role[i];
  }
  s->ncell = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  s->nnode = (int64_t)cfg->nx * cfg->ny * (cfg->nz + 1);
  s->rho = calloc(s->nnode, sizeof(double));
  s->phi = calloc(s->nnode, sizeof(double));
  for (int i = 0; i < cfg->nsp; ++i) {
    s->ncount[i] = calloc(s->ncell, sizeof(int32_t));
    s->cell_start[i] = calloc(s->ncell + 1, sizeof(int64_t));
  }
  /* Dirichlet planes of the initial potential */
  int64_t plane = (int64_t)cfg->nx * cfg->ny;
  for (int64_t p = 0; p < plane; ++p) {
    s->phi[p] = cfg->phi_c;
    s->phi[(int64_t)cfg->nz * plane + p] = cfg->phi_a;
  }
  return s;
}

void or_destroy(or_state_t* s) {
  if (!s) return;
  for (int i = 0; i < OR_MAXSP; ++i) { store_free(&s->st[i]); free(s->ncount[i]); free(s->cell_start[i]); }
  for (int i = 0; i < s->nxs; ++i) { free(s->xs[i].E); free(s->xs[i].sig); }
  free(s->rho); free(s->phi); free(s->log); free(s->hit);
  free(s);
}

int or_add_xsec(or_state_t* s, int kind, int proj, int target, int product, double thr, int n,
                const double* E, const double* sig) {
  if (s->nxs >= OR_MAXXS || n < 1 || kind < OR_XS_IONIZATION || kind > OR_XS_CX) return -1;
  or_xsec_t* x = &s->xs[s->nxs++];
  x->kind = kind; x->projectile = proj; x->target = target; x->product = product;
  x->thr = thr; x->n = n;
  x->E = malloc(n * sizeof(double)); x->sig = malloc(n * sizeof(double));
  memcpy(x->E, E, n * sizeof(double)); memcpy(x->sig, sig, n * sizeof(double));
  return 0;
}

int or_add_source(or_state_t* s, int species, double cx, double cy, double R, double flux, double T) {
  if (s->nsrc >= OR_MAXSRC) return -1;
  or_source_t* q = &s->src[s->nsrc++];
  q->species = species; q->cx = cx; q->cy = cy; q->R = R; q->flux = flux; q->T = T; q->acc = 0.0;
  return 0;
}

/* Change the flux and temperature of source q from the next step on; its carry
 * accumulator is kept (a source whose strength changes keeps its fractional
 * count). */
int or_set_source(or_state_t* s, int q, double flux, double T) {
  if (q < 0 || q >= s->nsrc) return -1;
  s->src[q].flux = flux;
  s->src[q].T = T;
  return 0;
}

void or_set_background_density(or_state_t* s, double n) { s->bg_density = n; }

/* Append particles; pids are assigned from next_pid in array order. mw: their
 * multiplicities (NULL: 1 each; other than 1 only with variable_weights). */
int or_load_m(or_state_t* s, int sp, int64_t n, const double* x, const double* v, const uint32_t* mw) {
  if (sp < 0 || sp >= s->c.nsp) return -1;
  for (int64_t i = 0; i < n; ++i) {
    if (mw && (mw[i] == 0 || (mw[i] != 1 && !s->c.variable_weights))) return -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    store_push(&s->st[sp], x[3 * i], x[3 * i + 1], x[3 * i + 2], v[3 * i], v[3 * i + 1], v[3 * i + 2],
               s->next_pid++, mw ? mw[i] : 1u);
  }
  return 0;
}
int or_load(or_state_t* s, int sp, int64_t n, const double* x, const double* v) {
  return or_load_m(s, sp, n, x, v, NULL);
}

int64_t or_count(const or_state_t* s, int sp) { return s->st[sp].n; }

void or_get_multiplicity(const or_state_t* s, int sp, uint32_t* out) {
  const or_store_t* t = &s->st[sp];
  for (int64_t i = 0; i < t->n; ++i) out[i] = t->mw[i];
}

void or_get_particles(const or_state_t* s, int sp, double* x, double* v, uint32_t* pid) {
  const or_store_t* t = &s->st[sp];
  for (int64_t i = 0; i < t->n; ++i) {
    if (x) { x[3 * i] = t->x[i]; x[3 * i + 1] = t->y[i]; x[3 * i + 2] = t->z[i]; }
    if (v) { v[3 * i] = t->vx[i]; v[3 * i + 1] = t->vy[i]; v[3 * i + 2] = t->vz[i]; }
    if (pid) pid[i] = t->pid[i];
  }
}

/* Overwrite velocities of species sp (test hook), in store order. */
void or_set_velocities(or_state_t* s, int sp, const double* v) {
  or_store_t* t = &s->st[sp];
  for (int64_t i = 0; i < t->n; ++i) { t->vx[i] = v[3 * i]; t->vy[i] = v[3 * i + 1]; t->vz[i] = v[3 * i + 2]; }
}

void or_get_rho(const or_state_t* s, double* out) { memcpy(out, s->rho, s->nnode * sizeof(double)); }
void or_get_phi(const or_state_t* s, double* out) { memcpy(out, s->phi, s->nnode * sizeof(double)); }
void or_set_phi(or_state_t* s, const double* in) { memcpy(s->phi, in, s->nnode * sizeof(double)); }
void or_get_ncount(const or_state_t* s, int sp, int32_t* out) { memcpy(out, s->ncount[sp], s->ncell * sizeof(int32_t)); }
void or_get_cell_start(const or_state_t* s, int sp, int64_t* out) { memcpy(out, s->cell_start[sp], (s->ncell + 1) * sizeof(int64_t)); }
int64_t or_get_log(const or_state_t* s, uint32_t* out) {
  if (out) memcpy(out, s->log, (size_t)s->nlog * 3 * sizeof(uint32_t));
  return s->nlog;
}

/* Cathode hits of ions since the last call, in the order they were found.
 * With pid == NULL only the count is returned; otherwise every field is copied
 * (xy: 2 per hit, v: 3 per hit) and the log is emptied. */
int64_t or_get_hits(or_state_t* s, uint32_t* pid, int32_t* sp, uint32_t* step, double* xy, double* v) {
  const int64_t n = s->nhit;
  if (!pid) return n;
  for (int64_t i = 0; i < n; ++i) {
    const or_hit_t* h = &s->hit[i];
    pid[i] = h->pid; sp[i] = h->sp; step[i] = h->step;
    xy[2 * i] = h->x; xy[2 * i + 1] = h->y;
    v[3 * i] = h->vx; v[3 * i + 1] = h->vy; v[3 * i + 2] = h->vz;
  }
  s->nhit = 0;
  return n;
}

static void log_hit(or_state_t* s, uint32_t pid, int sp, double x, double y, double vx, double vy, double vz) {
  if (s->nhit == s->hitcap) {
    s->hitcap = s->hitcap ? 2 * s->hitcap : 1024;
    s->hit = realloc(s->hit, (size_t)s->hitcap * sizeof(or_hit_t));
  }
  or_hit_t* h = &s->hit[s->nhit++];
  h->pid = pid; h->sp = sp; h->step = s->step;
  h->x = x; h->y = y; h->vx = vx; h->vy = vy; h->vz = vz;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers. Node (i,j,k), i in [0,nx), j in [0,ny) periodic, k in [0,nz]. */
/* Cell (i,j,k), k in [0,nz). Linear index (k*ny + j)*nx + i for both.        */
/* ------------------------------------------------------------------------ */
static int64_t nidx(const or_state_t* s, int i, int j, int k) {
  return ((int64_t)k * s->c.ny + j) * s->c.nx + i;
}

/* Cell coordinate of a position: g = x * (1/h) with 1/h rounded once,
 * cell = floor(g) clamped to the last cell, fraction = g - cell. */
static void locate(const or_state_t* s, double x, double y, double z, int* i, int* j, int* k,
                   double* fx, double* fy, double* fz) {
  double inv_h = 1.0 / s->c.h;
  double gx = x * inv_h, gy = y * inv_h, gz = z * inv_h;
  int ii = (int)floor(gx), jj = (int)floor(gy), kk = (int)floor(gz);
  if (ii > s->c.nx - 1) ii = s->c.nx - 1;
  if (jj > s->c.ny - 1) jj = s->c.ny - 1;
  if (kk > s->c.nz - 1) kk = s->c.nz - 1;
  if (ii < 0) ii = 0;
  if (jj < 0) jj = 0;
  if (kk < 0) kk = 0;
  *i = ii; *j = jj; *k = kk;
  *fx = gx - ii; *fy = gy - jj; *fz = gz - kk;
}

static int64_t cell_of(const or_state_t* s, double x, double y, double z) {
  int i, j, k; double fx, fy, fz;
  locate(s, x, y, z, &i, &j, &k, &fx, &fy, &fz);
  return nidx(s, i, j, k);
}

/* ------------------------------------------------------------------------ */
/* a1: injection from disk sources on the cathode (PIC/MCC paragraph: SPs    */
/* are injected for emitted electrons and evaporated neutrals).               */
/* Expected number per step mu = flux * pi R^2 * dt / w; the integer count    */
/* comes from the carry accumulator acc += mu; n = floor(acc); acc -= n.      */
/* Position uniform on the disk, velocity half-Maxwellian (vx, vy normal,     */
/* vz = |normal|), first partial step z = U * vz * dt. pids in (source, k)    */
/* order.                                                                     */
/* ------------------------------------------------------------------------ */
static double wrap(double x, double L) {
  double inv = 1.0 / L;
  double r = x - L * floor(x * inv);
  if (r >= L) r -= L;
  if (r < 0.0) r += L;
  return r;
}

int64_t or_inject(or_state_t* s) {
  const double kB = 1.380649e-23;
  double Lx = s->c.nx * s->c.h, Ly = s->c.ny * s->c.h;
  int64_t total = 0;
  for (int q = 0; q < s->nsrc; ++q) {
    or_source_t* src = &s->src[q];
    const or_species_t* sp = &s->sp[src->species];
    double mu = src->flux * OR_PI * src->R * src->R * s->c.dt / sp->w;
    src->acc += mu;
    double nf = floor(src->acc);
    src->acc -= nf;
    int64_t n = (int64_t)nf;
    double sig = sqrt(kB * src->T / sp->m);
    for (int64_t k = 0; k < n; ++k) {
      uint32_t pid = s->next_pid++;
      draw2 dp = draw(s->c.seed, pid, s->step, TAG_INJ_POS, 0);
      draw2 d1 = draw(s->c.seed, pid, s->step, TAG_INJ_VXY, 0);
      draw2 d2 = draw(s->c.seed, pid, s->step, TAG_INJ_VZ, 0);
      draw2 d3 = draw(s->c.seed, pid, s->step, TAG_INJ_Z, 0);
      double r = src->R * sqrt(dp.u0);
      double th = 2.0 * OR_PI * dp.u1;
      double x = wrap(src->cx + r * cos(th), Lx);
      double y = wrap(src->cy + r * sin(th), Ly);
      double rad1 = sqrt(-2.0 * log(d1.u0));
      double n1 = rad1 * cos(2.0 * OR_PI * d1.u1);
      double n2 = rad1 * sin(2.0 * OR_PI * d1.u1);
      double n3 = sqrt(-2.0 * log(d2.u0)) * cos(2.0 * OR_PI * d2.u1);
      double vx = sig * n1, vy = sig * n2, vz = sig * fabs(n3);
      double z = d3.u0 * vz * s->c.dt;
      store_push(&s->st[src->species], x, y, z, vx, vy, vz, pid, 1u);
      s->mom.injected[src->species] += 1;
    }
    total += n;
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* a2: cell sort. Key (cell of the current position, pid); the pair is unique */
/* so the sorted order is unique. cell_start is the exclusive prefix sum of  */
/* the per-cell histogram.                                                    */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t cell; uint32_t pid; int64_t idx; } sortrec;

static int cmp_sortrec(const void* a, const void* b) {
  const sortrec* x = a; const sortrec* y = b;
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  if (x->pid != y->pid) return x->pid < y->pid ? -1 : 1;
  return 0;
}

void or_sort(or_state_t* s) {
  for (int sp = 0; sp < s->c.nsp; ++sp) {
    or_store_t* t = &s->st[sp];
    int64_t n = t->n;
    sortrec* r = malloc((n ? n : 1) * sizeof(sortrec));
    for (int64_t i = 0; i < n; ++i) {
      r[i].cell = cell_of(s, t->x[i], t->y[i], t->z[i]);
      r[i].pid = t->pid[i];
      r[i].idx = i;
    }
    qsort(r, n, sizeof(sortrec), cmp_sortrec);
    or_store_t u = {0};
    store_reserve(&u, n > 0 ? n : 1);
    for (int64_t i = 0; i < n; ++i) {
      int64_t o = r[i].idx;
      u.x[i] = t->x[o]; u.y[i] = t->y[o]; u.z[i] = t->z[o];
      u.vx[i] = t->vx[o]; u.vy[i] = t->vy[o]; u.vz[i] = t->vz[o];
      u.pid[i] = t->pid[o];
      u.mw[i] = t->mw[o];
    }
    u.n = n;
    int64_t* cs = s->cell_start[sp];
    memset(cs, 0, (s->ncell + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) cs[r[i].cell + 1] += 1;
    for (int64_t c = 0; c < s->ncell; ++c) cs[c + 1] += cs[c];
    store_free(t);
    *t = u;
    free(r);
  }
}

/* ------------------------------------------------------------------------ */
/* a3: deposition. rho at nodes by cloud-in-cell (trilinear) weights,         */
/* rho_node = sum_p q w S(x_p - x_node) / h^3, plus the uniform background.   */
/* Neutral species add integer per-cell counts (nearest-grid-point) used as   */
/* the MCC target density.                                                    */
/* ------------------------------------------------------------------------ */
void or_deposit(or_state_t* s) {
  int nx = s->c.nx, ny = s->c.ny;
  double inv_h3 = 1.0 / (s->c.h * s->c.h * s->c.h);
  for (int64_t p = 0; p < s->nnode; ++p) s->rho[p] = s->c.rho_bg;
  for (int sp = 0; sp < s->c.nsp; ++sp) {
    or_store_t* t = &s->st[sp];
    if (s->sp[sp].role == OR_NEUTRAL) {
      memset(s->ncount[sp], 0, s->ncell * sizeof(int32_t));
      for (int64_t p = 0; p < t->n; ++p) s->ncount[sp][cell_of(s, t->x[p], t->y[p], t->z[p])] += (int32_t)t->mw[p];
    }
    double qw = s->sp[sp].q * s->sp[sp].w * inv_h3;
    if (qw == 0.0) continue;
    for (int64_t p = 0; p < t->n; ++p) {
      int i, j, k; double fx, fy, fz;
      locate(s, t->x[p], t->y[p], t->z[p], &i, &j, &k, &fx, &fy, &fz);
      int ic[2] = {i, i + 1 == nx ? 0 : i + 1};
      int jc[2] = {j, j + 1 == ny ? 0 : j + 1};
      int kc[2] = {k, k + 1};
      double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy}, wz[2] = {1.0 - fz, fz};
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a)
            s->rho[nidx(s, ic[a], jc[b], kc[c])] += qw * ((double)t->mw[p] * (wx[a] * wy[b] * wz[c]));
    }
  }
}

/* Standalone deposit of one particle set onto a fresh grid (for pins). */
void or_deposit_points(int nx, int ny, int nz, double h, int64_t n, const double* xyz, double qw_total_per_particle,
                       double* rho_out) {
  or_cfg_t c;
  memset(&c, 0, sizeof(c));
  c.nx = nx; c.ny = ny; c.nz = nz; c.h = h; c.nsp = 1;
  c.q[0] = qw_total_per_particle; c.m[0] = 1.0; c.w[0] = 1.0; c.role[0] = OR_ELECTRON;
  or_state_t* s = or_create(&c);
  for (int64_t p = 0; p < n; ++p) store_push(&s->st[0], xyz[3 * p], xyz[3 * p + 1], xyz[3 * p + 2], 0, 0, 0, (uint32_t)p, 1u);
  or_deposit(s);
  memcpy(rho_out, s->rho, s->nnode * sizeof(double));
  or_destroy(s);
}

/* ------------------------------------------------------------------------ */
/* a4: Poisson solve, Eq. (1) on the node grid, scaled by h^2:                */
/*   6 phi_ijk - sum of the six neighbours = h^2 rho_ijk / eps0               */
/* over the unknown nodes k = 1..nz-1 (periodic in i and j), with the         */
/* Dirichlet planes phi(k=0) = phi_c and phi(k=nz) = phi_a folded into the    */
/* right-hand side. Plain conjugate gradients; stop when the recursive        */
/* residual satisfies ||r|| <= rtol ||b||, then confirm with the true residual */
/* (restarting from it if the confirmation fails).                            */
/* ------------------------------------------------------------------------ */
typedef struct { int nx, ny, nu; } lap_t; /* nu = nz - 1 unknown planes */

static void lap_apply(const lap_t* L, const double* x, double* y) {
  int nx = L->nx, ny = L->ny, nu = L->nu;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nu; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t c = ((int64_t)k * ny + j) * nx + i;
        int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
        int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
        double s = x[((int64_t)k * ny + j) * nx + im] + x[((int64_t)k * ny + j) * nx + ip] +
                   x[((int64_t)k * ny + jm) * nx + i] + x[((int64_t)k * ny + jp) * nx + i];
        if (k > 0) s += x[c - (int64_t)nx * ny];
        if (k < nu - 1) s += x[c + (int64_t)nx * ny];
        y[c] = 6.0 * x[c] - s;
      }
}

/* Sum of a[i] b[i] in a fixed order: chunks of OR_CHUNK consecutive terms
 * summed in index order, then the chunk sums in chunk order. part holds
 * ceil(n / OR_CHUNK) doubles. */
#define OR_CHUNK 4096
static double dot(int64_t n, const double* a, const double* b, double* part) {
  const int64_t nc = (n + OR_CHUNK - 1) / OR_CHUNK;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t i1 = (c + 1) * OR_CHUNK < n ? (c + 1) * OR_CHUNK : n;
    double s = 0.0;
    for (int64_t i = c * OR_CHUNK; i < i1; ++i) s += a[i] * b[i];
    part[c] = s;
  }
  double s = 0.0;
  for (int64_t c = 0; c < nc; ++c) s += part[c];
  return s;
}

/* Solve A x = b (A from lap_apply), x holds the initial guess on entry.
 * Returns iterations, writes the final true relative residual. */
static int cg_solve(const lap_t* L, const double* b, double* x, double rtol, int maxit, double* rel_out) {
  int64_t n = (int64_t)L->nx * L->ny * L->nu;
  double* r = malloc(n * sizeof(double));
  double* p = malloc(n * sizeof(double));
  double* q = malloc(n * sizeof(double));
  double* part = malloc(((n + OR_CHUNK - 1) / OR_CHUNK + 1) * sizeof(double));
  double bn = sqrt(dot(n, b, b, part));
  int it = 0;
  double rel = 0.0;
  if (bn == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    *rel_out = 0.0;
    free(r); free(p); free(q); free(part);
    return 0;
  }
  double tol = rtol * bn;
  for (int restart = 0; restart < 8; ++restart) {
    lap_apply(L, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rr = dot(n, r, r, part);
    rel = sqrt(rr) / bn;
    if (sqrt(rr) <= tol || it >= maxit) break;
    while (it < maxit) {
      lap_apply(L, p, q);
      double alpha = rr / dot(n, p, q, part);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      double rr_new = dot(n, r, r, part);
      ++it;
      if (sqrt(rr_new) <= tol) { rr = rr_new; break; }
      double beta = rr_new / rr;
      rr = rr_new;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
  }
  /* final true residual */
  lap_apply(L, x, q);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
  rel = sqrt(dot(n, q, q, part)) / bn;
  *rel_out = rel;
  free(r); free(p); free(q); free(part);
  return it;
}

/* Right-hand side over unknown nodes from rho over all nodes. */
static void poisson_rhs(int nx, int ny, int nz, double h, double phi_c, double phi_a, const double* rho,
                        double* b) {
  int64_t plane = (int64_t)nx * ny;
  double s = h * h / OR_EPS0;
#pragma omp parallel for schedule(static)
  for (int k = 1; k < nz; ++k)
    for (int64_t p = 0; p < plane; ++p) {
      double v = s * rho[(int64_t)k * plane + p];
      if (k == 1) v += phi_c;
      if (k == nz - 1) v += phi_a;
      b[(int64_t)(k - 1) * plane + p] = v;
    }
}

/* Full-grid Poisson solve: phi over all nodes (in/out; its interior is the
 * initial guess). Returns iterations; *rel = final true relative residual. */
int or_poisson(int nx, int ny, int nz, double h, double phi_c, double phi_a, const double* rho,
               double* phi, double rtol, int maxit, double* rel) {
  int64_t plane = (int64_t)nx * ny, nu = (int64_t)(nz - 1) * plane;
  lap_t L = {nx, ny, nz - 1};
  double* b = malloc((nu ? nu : 1) * sizeof(double));
  double* x = malloc((nu ? nu : 1) * sizeof(double));
  poisson_rhs(nx, ny, nz, h, phi_c, phi_a, rho, b);
  for (int64_t u = 0; u < nu; ++u) x[u] = phi[plane + u];
  int it = cg_solve(&L, b, x, rtol, maxit, rel);
  for (int64_t p = 0; p < plane; ++p) { phi[p] = phi_c; phi[(int64_t)nz * plane + p] = phi_a; }
  for (int64_t u = 0; u < nu; ++u) phi[plane + u] = x[u];
  free(b); free(x);
  return it;
}

/* Apply the scaled operator to phi's interior (for pins): y = A x_interior. */
void or_laplacian_apply(int nx, int ny, int nz, const double* x_interior, double* y) {
  lap_t L = {nx, ny, nz - 1};
  lap_apply(&L, x_interior, y);
}

int or_solve(or_state_t* s) {
  if (s->c.warm_zero) {
    int64_t plane = (int64_t)s->c.nx * s->c.ny;
    for (int64_t p = plane; p < (int64_t)s->c.nz * plane; ++p) s->phi[p] = 0.0;
  }
  double rel = 0.0;
  int it = or_poisson(s->c.nx, s->c.ny, s->c.nz, s->c.h, s->c.phi_c, s->anode_V, s->rho, s->phi, s->c.cg_rtol,
                      s->c.cg_maxit, &rel);
  s->mom.cg_iters = it;
  s->mom.cg_resid_rel = rel;
  return it;
}

/* ------------------------------------------------------------------------ */
/* a5: field at nodes E = -grad phi: central differences, periodic in x and  */
/* y; in z central inside and second-order one-sided on the electrode planes. */
/* Trilinear (cloud-in-cell) interpolation to the particle.                   */
/* ------------------------------------------------------------------------ */
static void node_field(const or_state_t* s, int i, int j, int k, double E[3]) {
  int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
  double inv2h = 1.0 / (2.0 * s->c.h);
  int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
  int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const double* f = s->phi;
  E[0] = -(f[nidx(s, ip, j, k)] - f[nidx(s, im, j, k)]) * inv2h;
  E[1] = -(f[nidx(s, i, jp, k)] - f[nidx(s, i, jm, k)]) * inv2h;
  if (k == 0)
    E[2] = -(-3.0 * f[nidx(s, i, j, 0)] + 4.0 * f[nidx(s, i, j, 1)] - f[nidx(s, i, j, 2)]) * inv2h;
  else if (k == nz)
    E[2] = -(3.0 * f[nidx(s, i, j, nz)] - 4.0 * f[nidx(s, i, j, nz - 1)] + f[nidx(s, i, j, nz - 2)]) * inv2h;
  else
    E[2] = -(f[nidx(s, i, j, k + 1)] - f[nidx(s, i, j, k - 1)]) * inv2h;
}

static void gather(const or_state_t* s, double x, double y, double z, double E[3]) {
  int i, j, k; double fx, fy, fz;
  locate(s, x, y, z, &i, &j, &k, &fx, &fy, &fz);
  int nx = s->c.nx, ny = s->c.ny;
  int ic[2] = {i, i + 1 == nx ? 0 : i + 1};
  int jc[2] = {j, j + 1 == ny ? 0 : j + 1};
  int kc[2] = {k, k + 1};
  double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy}, wz[2] = {1.0 - fz, fz};
  E[0] = E[1] = E[2] = 0.0;
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        double En[3];
        node_field(s, ic[a], jc[b], kc[c], En);
        double W = wx[a] * wy[b] * wz[c];
        E[0] += W * En[0]; E[1] += W * En[1]; E[2] += W * En[2];
      }
}

/* Field at arbitrary points for pins (uses the state's phi). */
void or_gather_points(const or_state_t* s, int64_t n, const double* xyz, double* E) {
  for (int64_t p = 0; p < n; ++p) gather(s, xyz[3 * p], xyz[3 * p + 1], xyz[3 * p + 2], E + 3 * p);
}

/* ------------------------------------------------------------------------ */
/* a8 helpers: cross-section lookup. sigma = 0 at or below the threshold;    */
/* a one-point table is a constant; otherwise linear interpolation in E over  */
/* the interval E_i <= E < E_{i+1} found by bisection, clamped at both ends.  */
/* ------------------------------------------------------------------------ */
static double xs_sigma(const or_xsec_t* c, double E) {
  if (!(E > c->thr)) return 0.0;
  if (c->n == 1) return c->sig[0];
  if (E <= c->E[0]) return c->sig[0];
  if (E >= c->E[c->n - 1]) return c->sig[c->n - 1];
  int lo = 0, hi = c->n - 1; /* invariant: E[lo] <= E < E[hi] */
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (E < c->E[mid]) hi = mid; else lo = mid;
  }
  double t = (E - c->E[lo]) / (c->E[lo + 1] - c->E[lo]);
  return c->sig[lo] + t * (c->sig[lo + 1] - c->sig[lo]);
}

double or_sigma(const or_state_t* s, int ch, double E) { return xs_sigma(&s->xs[ch], E); }

/* ------------------------------------------------------------------------ */
/* a6-a9: push, absorb, MCC, ionization resolve, compaction.                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t e_idx;    /* primary's index in the projectile store (electron or ion) */
  int proj;         /* projectile species */
  int ch;           /* channel */
  int64_t cell;     /* cell of the primary at x^n */
  uint32_t pid;
  double E_eV;      /* pre-collision energy */
  int64_t victim;   /* neutral index in the target store, -1 = suppressed */
} or_event_t;

typedef struct { uint64_t key; int64_t idx; } cand_t;

static int cmp_cand(const void* a, const void* b) {
  const cand_t* x = a; const cand_t* y = b;
  return x->key < y->key ? -1 : (x->key > y->key ? 1 : 0);
}

static int cmp_event_cell_pid(const void* a, const void* b) {
  const or_event_t* x = a; const or_event_t* y = b;
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  return x->pid < y->pid ? -1 : (x->pid > y->pid ? 1 : 0);
}

static int cmp_event_pid(const void* a, const void* b) {
  const or_event_t* x = a; const or_event_t* y = b;
  return x->pid < y->pid ? -1 : (x->pid > y->pid ? 1 : 0);
}

void or_push_collide_resolve(or_state_t* s) {
  const int nsp = s->c.nsp;
  const double dt = s->c.dt, h = s->c.h;
  const double Lx = s->c.nx * h, Ly = s->c.ny * h, Lz = s->c.nz * h;
  const double inv_h3 = 1.0 / (h * h * h);
  uint8_t* dead[OR_MAXSP];
  int64_t* cell_n[OR_MAXSP];
  or_event_t* ev = NULL;
  int64_t nev = 0, evcap = 0;
  double q_cath = 0.0, q_anode = 0.0;

  int64_t npre[OR_MAXSP];
  for (int sp = 0; sp < nsp; ++sp) {
    or_store_t* t = &s->st[sp];
    npre[sp] = t->n;
    dead[sp] = calloc(t->n ? t->n : 1, 1);
    cell_n[sp] = malloc((t->n ? t->n : 1) * sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < t->n; ++p) cell_n[sp][p] = cell_of(s, t->x[p], t->y[p], t->z[p]);
  }

  /* Per particle: 0 moves on, 1 absorbed at the cathode, 2 at the anode, 3
   * scattered elastically, 4 an event needing a victim (channel ev_ch, energy
   * ev_E). The particles advance independently (in parallel in the OpenMP
   * build); counts, energy sums, hit logs and events follow in particle order. */
  for (int sp = 0; sp < nsp; ++sp) {
    or_store_t* t = &s->st[sp];
    const or_species_t* S = &s->sp[sp];
    const double qm_dt = S->q / S->m * dt;
    int chs[OR_MAXXS], nch = 0;
    for (int c = 0; c < s->nxs; ++c) if (s->xs[c].projectile == sp) chs[nch++] = c;
    const int64_t n = t->n;
    uint8_t* status = malloc(n ? n : 1);
    int* ev_ch = malloc((n ? n : 1) * sizeof(int));
    double* ev_E = malloc((n ? n : 1) * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
      status[p] = 0;
      /* a5 + a6: gather at x^n, leapfrog kick and drift */
      if (S->q != 0.0) {
        double E[3];
        gather(s, t->x[p], t->y[p], t->z[p], E);
        t->vx[p] += qm_dt * E[0];
        t->vy[p] += qm_dt * E[1];
        t->vz[p] += qm_dt * E[2];
      }
      double xn = t->x[p] + t->vx[p] * dt;
      double yn = t->y[p] + t->vy[p] * dt;
      double zn = t->z[p] + t->vz[p] * dt;
      /* a7: absorption at the electrodes (x^n and v^{n+1/2} are kept for the
       * energy sums and the hit log) */
      double v2 = t->vx[p] * t->vx[p] + t->vy[p] * t->vy[p] + t->vz[p] * t->vz[p];
      if (zn < 0.0 || zn >= Lz) {
        status[p] = zn < 0.0 ? 1 : 2;
        continue;
      }
      t->x[p] = wrap(xn, Lx);
      t->y[p] = wrap(yn, Ly);
      t->z[p] = zn;
      /* a8: Monte Carlo collisions, Eq. (4): P = 1 - exp(-u n sigma(E) dt) summed
       * over the channels of this projectile; target density from the NGP
       * neutral count of the projectile's cell at x^n. */
      if (nch == 0) continue;
      double u = sqrt(v2);
      double E_eV = 0.5 * S->m * v2 / OR_QE;
      double cum[OR_MAXXS], nu_tot = 0.0;
      for (int a = 0; a < nch; ++a) {
        const or_xsec_t* X = &s->xs[chs[a]];
        double nt = s->bg_density > 0.0 ? s->bg_density
                                        : (double)s->ncount[X->target][cell_n[sp][p]] * s->sp[X->target].w * inv_h3;
        nu_tot += nt * xs_sigma(X, E_eV);
        cum[a] = nu_tot;
      }
      if (!(nu_tot > 0.0)) continue;
      double P = -expm1(-u * dt * nu_tot);
      draw2 d = draw(s->c.seed, t->pid[p], s->step, TAG_MCC, 0);
      if (!(d.u0 < P)) continue;
      int a = 0;
      while (a < nch - 1 && !(d.u0 < P * (cum[a] / nu_tot))) ++a;
      const or_xsec_t* X = &s->xs[chs[a]];
      if (X->kind == OR_XS_ELASTIC) {
        /* isotropic scattering, speed kept */
        draw2 g = draw(s->c.seed, t->pid[p], s->step, TAG_SCATTER, 0);
        double ct = 2.0 * g.u0 - 1.0;
        double st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double ph = 2.0 * OR_PI * g.u1;
        t->vx[p] = u * st * cos(ph);
        t->vy[p] = u * st * sin(ph);
        t->vz[p] = u * ct;
        status[p] = 3;
      } else {
        status[p] = 4;
        ev_ch[p] = chs[a];
        ev_E[p] = E_eV;
      }
    }
    for (int64_t p = 0; p < n; ++p) {
      const int st = status[p];
      if (st == 1 || st == 2) {
        dead[sp][p] = 1;
        const double v2 = t->vx[p] * t->vx[p] + t->vy[p] * t->vy[p] + t->vz[p] * t->vz[p];
        const double mwp = (double)t->mw[p];
        double ke = 0.5 * S->m * S->w * (mwp * v2);
        if (st == 1) {
          s->mom.abs_cathode[sp] += 1; s->mom.abs_energy_cathode[sp] += ke; q_cath += S->q * S->w * mwp;
          if (S->role == OR_ION) {
            /* z^n >= 0 > z^{n+1}, so vz < 0: the path meets z = 0 at x^n - v z^n / vz */
            const double f = t->z[p] / t->vz[p];
            log_hit(s, t->pid[p], sp, wrap(t->x[p] - t->vx[p] * f, Lx), wrap(t->y[p] - t->vy[p] * f, Ly),
                    t->vx[p], t->vy[p], t->vz[p]);
          }
        }
        else { s->mom.abs_anode[sp] += 1; s->mom.abs_energy_anode[sp] += ke; q_anode += S->q * S->w * mwp; }
      } else if (st == 3) {
        s->mom.n_elastic += 1;
      } else if (st == 4) {
        if (nev == evcap) { evcap = evcap ? 2 * evcap : 256; ev = realloc(ev, evcap * sizeof(or_event_t)); }
        or_event_t* e = &ev[nev++];
        e->e_idx = p; e->proj = sp; e->ch = ev_ch[p]; e->cell = cell_n[sp][p]; e->pid = t->pid[p];
        e->E_eV = ev_E[p]; e->victim = -1;
      }
    }
    free(status);
    free(ev_ch);
    free(ev_E);
  }

  /* a9: resolve of the events that need a victim neutral (ionization, charge
   * exchange). Per (target species, cell): events of every channel together,
   * in order of primary pid, take the surviving neutrals whose cell at x^n is
   * that cell, in increasing order of (Philox victim key, pid). Events left
   * without a neutral are suppressed. */
  if (s->bg_density > 0.0) {
    /* fixed background: events are counted but consume or convert nothing */
    for (int64_t a = 0; a < nev; ++a) {
      if (s->xs[ev[a].ch].kind == OR_XS_CX) s->mom.n_cx += 1;
      else s->mom.n_ionization += 1;
    }
    nev = 0;
  }
  qsort(ev, nev, sizeof(or_event_t), cmp_event_cell_pid);
  int64_t a0 = 0;
  while (a0 < nev) {
    int64_t a1 = a0;
    int tgt = s->xs[ev[a0].ch].target;
    while (a1 < nev && ev[a1].cell == ev[a0].cell && s->xs[ev[a1].ch].target == tgt) ++a1;
    or_store_t* T = &s->st[tgt];
    int64_t m = 0;
    cand_t* cd = malloc((T->n ? T->n : 1) * sizeof(cand_t));
    for (int64_t p = 0; p < T->n; ++p) {
      if (dead[tgt][p] || cell_n[tgt][p] != ev[a0].cell) continue;
      draw2 d = draw(s->c.seed, T->pid[p], s->step, TAG_VICTIM, 0);
      cd[m].key = ((uint64_t)d.w[0] << 32) | (uint64_t)T->pid[p];
      cd[m].idx = p;
      ++m;
    }
    qsort(cd, m, sizeof(cand_t), cmp_cand);
    for (int64_t r = 0; r < a1 - a0; ++r) ev[a0 + r].victim = r < m ? cd[r].idx : -1;
    free(cd);
    a0 = a1;
  }
  /* apply in order of primary pid; secondaries take pids in that order.
   * Events between unequal multiplicities (variable weights): the event moves
   * ms = min(multiplicity of the primary, of the victim); the partner holding
   * more keeps the rest in place, and the part that changes species becomes a
   * new particle of multiplicity ms with a pid of its own. Successful events
   * are numbered r in the order ionizations (by primary pid), then charge
   * exchanges (by primary pid); a secondary takes pid0 + r, the victim's new
   * ion pid0 + ns + 2r, an exchanging ion's new neutral pid0 + ns + 2r + 1
   * (ns successful events; 3 ns pids are consumed). The primary electron of
   * an ionization that moves less than its whole multiplicity loses the
   * ionization energy with probability ms / multiplicity (a uniform of the
   * ionization draw), so energy is conserved on average and charge and
   * particle numbers exactly. With every multiplicity 1 this is the plain
   * rule (and pid0 + nion pids are consumed). */
  qsort(ev, nev, sizeof(or_event_t), cmp_event_pid);
  s->nlog = 0;
  free(s->log);
  s->log = malloc((nev ? nev : 1) * 3 * sizeof(uint32_t));
  const int vw = s->c.variable_weights;
  const uint32_t pid0 = s->next_pid;
  int64_t ns = 0, nion_s = 0;
  for (int64_t a = 0; a < nev; ++a) {
    if (ev[a].victim < 0) continue;
    ++ns;
    if (s->xs[ev[a].ch].kind != OR_XS_CX) ++nion_s;
  }
  int64_t ri = 0, rc = 0;
  for (int64_t a = 0; a < nev; ++a) {
    or_event_t* e = &ev[a];
    if (e->victim < 0) { s->mom.n_suppressed += 1; continue; }
    const or_xsec_t* X = &s->xs[e->ch];
    or_store_t* Ep = &s->st[e->proj];
    or_store_t* T = &s->st[X->target];
    const int64_t p = e->e_idx, vi = e->victim;
    const uint32_t mp = Ep->mw[p], mv = T->mw[vi];
    const uint32_t ms = mp < mv ? mp : mv;
    if (X->kind == OR_XS_CX) {
      /* the ion becomes a neutral of the product species and the victim
       * neutral becomes an ion of the projectile species; both keep x^{n+1},
       * v^{n+1/2} and their pids (with unequal multiplicities: the part ms) */
      const int64_t r = nion_s + rc++;
      if (ms == mp) {
        store_push(&s->st[X->product], Ep->x[p], Ep->y[p], Ep->z[p], Ep->vx[p], Ep->vy[p], Ep->vz[p], Ep->pid[p], ms);
        dead[e->proj][p] = 1;
      } else {
        store_push(&s->st[X->product], Ep->x[p], Ep->y[p], Ep->z[p], Ep->vx[p], Ep->vy[p], Ep->vz[p],
                   pid0 + (uint32_t)(ns + 2 * r + 1), ms);
        Ep->mw[p] = mp - ms;
      }
      if (ms == mv) {
        store_push(Ep, T->x[vi], T->y[vi], T->z[vi], T->vx[vi], T->vy[vi], T->vz[vi], T->pid[vi], ms);
        dead[X->target][vi] = 1;
      } else {
        store_push(Ep, T->x[vi], T->y[vi], T->z[vi], T->vx[vi], T->vy[vi], T->vz[vi], pid0 + (uint32_t)(ns + 2 * r), ms);
        T->mw[vi] = mv - ms;
      }
      s->mom.n_cx += 1;
      continue;
    }
    const int64_t r = ri++;
    const double me = s->sp[e->proj].m;
    draw2 g0 = draw(s->c.seed, e->pid, s->step, TAG_IONIZE, 0);
    draw2 g1 = draw(s->c.seed, e->pid, s->step, TAG_IONIZE, 1);
    double Eex = e->E_eV - X->thr;            /* energy left after ionization */
    double E2 = g0.u0 * Eex;                  /* secondary */
    double E1 = (1.0 - g0.u0) * Eex;          /* primary, direction kept */
    double sc = sqrt(E1 / e->E_eV);
    if (ms == mp || g1.u1 < (double)ms / (double)mp) {
      Ep->vx[p] *= sc; Ep->vy[p] *= sc; Ep->vz[p] *= sc;
    }
    double us = sqrt(2.0 * E2 * OR_QE / me);
    double ct = 2.0 * g0.u1 - 1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * OR_PI * g1.u0;
    uint32_t spid = pid0 + (uint32_t)r;
    store_push(Ep, Ep->x[p], Ep->y[p], Ep->z[p], us * st * cos(ph), us * st * sin(ph), us * ct, spid, ms);
    /* the victim neutral becomes an ion at its new position with its velocity */
    if (ms == mv) {
      store_push(&s->st[X->product], T->x[vi], T->y[vi], T->z[vi], T->vx[vi], T->vy[vi], T->vz[vi], T->pid[vi], ms);
      dead[X->target][vi] = 1;
    } else {
      store_push(&s->st[X->product], T->x[vi], T->y[vi], T->z[vi], T->vx[vi], T->vy[vi], T->vz[vi],
                 pid0 + (uint32_t)(ns + 2 * r), ms);
      T->mw[vi] = mv - ms;
    }
    s->log[3 * s->nlog] = e->pid; s->log[3 * s->nlog + 1] = T->pid[vi]; s->log[3 * s->nlog + 2] = spid;
    s->nlog++;
    s->mom.n_ionization += 1;
  }
  s->next_pid = pid0 + (uint32_t)(vw ? 3 * ns : nion_s);
  free(ev);

  /* a10: compaction. The dead flags cover the pre-step population; entries
   * appended above (secondaries, new ions) lie beyond it and all survive. */
  for (int sp = 0; sp < nsp; ++sp) {
    or_store_t* t = &s->st[sp];
    int64_t w = 0;
    for (int64_t p = 0; p < t->n; ++p) {
      if (p < npre[sp] && dead[sp][p]) continue;
      t->x[w] = t->x[p]; t->y[w] = t->y[p]; t->z[w] = t->z[p];
      t->vx[w] = t->vx[p]; t->vy[w] = t->vy[p]; t->vz[w] = t->vz[p];
      t->pid[w] = t->pid[p];
      t->mw[w] = t->mw[p];
      ++w;
    }
    t->n = w;
  }
  s->mom.charge_to_cathode_last = q_cath;
  s->mom.charge_to_anode_last = q_anode;
  for (int sp = 0; sp < nsp; ++sp) free(cell_n[sp]);
  for (int sp = 0; sp < nsp; ++sp) free(dead[sp]);
}

/* ------------------------------------------------------------------------ */
/* a11: moments. Counts, total charge, kinetic energy per species (with the  */
/* half-step velocities), field energy (1/2) eps0 h sum over grid edges of   */
/* (delta phi)^2, i.e. (1/2) eps0 |E|^2 integrated with the edge gradients of */
/* the 7-point operator. Plain summation in FP64.                             */
/* ------------------------------------------------------------------------ */
void or_compute_moments(or_state_t* s) {
  double qt = 0.0;
  for (int sp = 0; sp < s->c.nsp; ++sp) {
    or_store_t* t = &s->st[sp];
    s->mom.count[sp] = t->n;
    double ke = 0.0, nphys = 0.0;
    for (int64_t p = 0; p < t->n; ++p) {
      ke += (double)t->mw[p] * (t->vx[p] * t->vx[p] + t->vy[p] * t->vy[p] + t->vz[p] * t->vz[p]);
      nphys += (double)t->mw[p];
    }
    s->mom.kinetic[sp] = 0.5 * s->sp[sp].m * s->sp[sp].w * ke;
    qt += s->sp[sp].q * s->sp[sp].w * nphys;
  }
  s->mom.total_charge = qt;
  int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
  double e2 = 0.0;
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double f = s->phi[nidx(s, i, j, k)];
        double dx = s->phi[nidx(s, i + 1 == nx ? 0 : i + 1, j, k)] - f;
        double dy = s->phi[nidx(s, i, j + 1 == ny ? 0 : j + 1, k)] - f;
        e2 += dx * dx + dy * dy;
        if (k < nz) { double dz = s->phi[nidx(s, i, j, k + 1)] - f; e2 += dz * dz; }
      }
  s->mom.field_energy = 0.5 * OR_EPS0 * s->c.h * e2;
  s->mom.step = s->step;
  s->mom.next_pid = s->next_pid;
}

void or_get_moments(or_state_t* s, or_moments_t* out) {
  or_compute_moments(s);
  s->mom.anode_V = s->anode_V;
  *out = s->mom;
}

/* One full step n -> n+1 in the order
 *   inject, [sort every sort_interval steps], deposit, solve, push/absorb/MCC,
 *   ionization resolve, compaction. */
static void circuit_step(or_state_t* s) {
  if (!s->circuit_on) return;
  const double dv = (s->c.dt * (s->circ_V0 - s->anode_V) / s->circ_R + s->mom.charge_to_anode_last) / s->circ_C;
  s->anode_V += dv;
}

void or_set_circuit(or_state_t* s, double R, double C, double V0) {
  s->circuit_on = R > 0.0 && C > 0.0;
  s->circ_R = R; s->circ_C = C; s->circ_V0 = V0;
}

int or_step(or_state_t* s) {
  or_inject(s);
  if (s->c.sort_interval > 0 && s->step % (uint32_t)s->c.sort_interval == 0) or_sort(s);
  or_deposit(s);
  or_solve(s);
  or_push_collide_resolve(s);
  circuit_step(s);
  s->step += 1;
  return 0;
}

/* Pieces of the step for stage-by-stage comparison. */
int or_step_until_solve(or_state_t* s) {
  or_inject(s);
  if (s->c.sort_interval > 0 && s->step % (uint32_t)s->c.sort_interval == 0) or_sort(s);
  or_deposit(s);
  return or_solve(s);
}

void or_step_finish(or_state_t* s) {
  or_push_collide_resolve(s);
  circuit_step(s);
  s->step += 1;
}

uint32_t or_get_step(const or_state_t* s) { return s->step; }
void or_set_step(or_state_t* s, uint32_t step) { s->step = step; }
uint32_t or_get_next_pid(const or_state_t* s) { return s->next_pid; }
double or_get_source_acc(const or_state_t* s, int q) { return s->src[q].acc; }
size_t or_sizeof_cfg(void) { return sizeof(or_cfg_t); }
size_t or_sizeof_moments(void) { return sizeof(or_moments_t); }

/* Bulk uniforms for statistics pins: out[2*p + r] = r-th FP64 uniform of
 * Philox(pid = pid0 + p, step, tag, j). */
void or_uniform_fill(uint64_t seed, uint32_t pid0, int64_t n, uint32_t step, uint32_t tag, uint32_t j,
                     double* out) {
  for (int64_t p = 0; p < n; ++p) {
    draw2 d = draw(seed, pid0 + (uint32_t)p, step, tag, j);
    out[2 * p] = d.u0;
    out[2 * p + 1] = d.u1;
  }
}

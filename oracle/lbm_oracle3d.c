/*
 * Plain FP64 CPU oracle of the TRT-LBM-VP method in 3D with the D3Q19 or the D3Q15
 * lattice (the paper's closing remark: the method extends to 3D by replacing D2Q9 with
 * D3Q15 or D3Q19; everything else is the 2D algorithm of Sec. 2.2 written for three axes).
 * TEST INFRASTRUCTURE ONLY, like lbm_oracle.c: used by the tests and the benchmark's CPU
 * baseline, never by the library. One node at a time, no fusion; compiled with
 * -O2 -ffp-contract=off.
 *
 * D3Q19 (readings listed in the design notes): e_0 = 0; e_1..6 = +-x, +-y, +-z; e_7..18
 * the twelve face diagonals; opposite directions come in pairs (2m-1, 2m); weights 1/3,
 * 1/18, 1/36. D3Q15: e_0, the same six axis directions, e_7..14 the eight cube corners
 * (+-1, +-1, +-1) in opposite pairs; weights 2/9, 1/9, 1/72. c_s^2 = 1/3 for both. f^eq and the Guo term have the 2D form with three components.
 * Edges: x periodic or equilibrium inlet (west) / zero-gradient outflow (east); y and z
 * periodic or free slip (specular: e_y or e_z reversed); rules applied x, then y, then z.
 * U_O = V + omega x (x - c) with an angular velocity vector.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 19

typedef struct {
  int q;
  int ex[QMAX], ey[QMAX], ez[QMAX];
  double w[QMAX];
} lattice3;

static const lattice3 D3Q19 = {
    19,
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
    {1.0 / 3.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
     1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
     1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0}};

static const lattice3 D3Q15 = {
    15,
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1},
    {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1},
    {2.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
     1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0}};

/* the lattice of a parameter set: q = 15 selects D3Q15, anything else D3Q19 */
static const lattice3 *lat3(int32_t q) { return q == 15 ? &D3Q15 : &D3Q19; }

static const double CS2_3 = 1.0 / 3.0;

enum { O3_PERIODIC = 0, O3_INLET = 1, O3_OUTFLOW = 2, O3_FREE_SLIP = 3 };
enum { O3_SPHERE = 0, O3_CYLINDER_Z = 1 };

typedef struct {
  int32_t nx, ny, nz;
  double nu, magic_lambda, eta, rho0;
  double u_in[3];
  int32_t west, east, south, north, bottom, top;
  int32_t q; /* 19: D3Q19, 15: D3Q15 */
} ora3_params;

typedef struct {
  double c[3], v[3], w[3]; /* centre, velocity, angular velocity */
  /* a deforming body (deform = 1) pulsates: scale s(n) = 1 + amp sin(rate n) about its
   * centre; kappa = s'(n) / s(n) is its dilation rate at the step being taken */
  double amp, rate, kappa;
  int32_t deform, pad;
} ora3_body;

typedef struct {
  int32_t kind, body;
  double c[3], radius; /* sphere: centre and radius; z-cylinder: axis through (c[0], c[1]) */
} ora3_shape;

/* direction with e_y (or e_z) reversed: the specular reflection of free-slip walls */
static int reflect3(const lattice3 *L, int a, int axis) {
  for (int b = 0; b < L->q; b++)
    if (L->ex[b] == L->ex[a] && (axis == 1 ? (L->ey[b] == -L->ey[a] && L->ez[b] == L->ez[a])
                                           : (L->ey[b] == L->ey[a] && L->ez[b] == -L->ez[a])))
      return b;
  return a;
}

static int opposite3(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

double ora3_tau_s(const ora3_params *p) { return p->nu / CS2_3 + 0.5; }
double ora3_tau_a(const ora3_params *p) {
  return 0.5 + p->magic_lambda / (ora3_tau_s(p) - 0.5);
}

/* Eq. (feq) with three velocity components */
void ora3_equilibrium(int32_t q, double rho, const double *u, double *feq) {
  const lattice3 *L = lat3(q);
  double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int a = 0; a < L->q; a++) {
    double eu = L->ex[a] * u[0] + L->ey[a] * u[1] + L->ez[a] * u[2];
    feq[a] = L->w[a] * rho * (1.0 + eu / CS2_3 + eu * eu / (2.0 * CS2_3 * CS2_3) - usq / (2.0 * CS2_3));
  }
}

/* Guo term F_alpha = w_alpha [(e - u)/c_s^2 + (e.u) e / c_s^4] . F (Eq. external-force-term) */
void ora3_guo(int32_t q, const double *u, const double *F, double *out) {
  const lattice3 *L = lat3(q);
  for (int a = 0; a < L->q; a++) {
    double e[3] = {L->ex[a], L->ey[a], L->ez[a]};
    double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
    double s = 0.0;
    for (int d = 0; d < 3; d++) s += ((e[d] - u[d]) / CS2_3 + eu * e[d] / (CS2_3 * CS2_3)) * F[d];
    out[a] = L->w[a] * s;
  }
}

static int inside3(const ora3_shape *s, double x, double y, double z) {
  double dx = x - s->c[0], dy = y - s->c[1], dz = z - s->c[2];
  double r2 = s->radius * s->radius;
  if (s->kind == O3_SPHERE) return dx * dx + dy * dy + dz * dz < r2;
  if (s->kind == O3_CYLINDER_Z) return dx * dx + dy * dy < r2;
  return 0;
}

/* Body id per node [nz][ny][nx]; later shapes overwrite earlier ones. */
void ora3_rasterize(int32_t nx, int32_t ny, int32_t nz, const ora3_shape *shapes, int32_t nshapes,
                    uint8_t *mask) {
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        uint8_t b = 0;
        for (int q = 0; q < nshapes; q++)
          if (inside3(&shapes[q], (double)i, (double)j, (double)k)) b = (uint8_t)shapes[q].body;
        mask[((size_t)k * ny + j) * nx + i] = b;
      }
}

static inline size_t IDX3(const ora3_params *p, int a, int k, int j, int i) {
  return (((size_t)a * p->nz + k) * p->ny + j) * p->nx + i;
}

/* f_alpha(i, j, k) = g_alpha(x - e_alpha) with the edge rules: x, then y, then z. */
static double pull3(const ora3_params *p, const double *g, const double *feq_inlet, int a, int i,
                    int j, int k) {
  const lattice3 *L = lat3(p->q);
  int sx = i - L->ex[a], sy = j - L->ey[a], sz = k - L->ez[a], src = a;
  if (sx < 0) {
    if (p->west == O3_INLET) return feq_inlet[a];
    sx += p->nx;
  } else if (sx > p->nx - 1) {
    if (p->east == O3_OUTFLOW) sx = p->nx - 1;
    else sx -= p->nx;
  }
  if (sy < 0) {
    if (p->south == O3_FREE_SLIP) { sy = 0; src = reflect3(L, src, 1); }
    else sy += p->ny;
  } else if (sy > p->ny - 1) {
    if (p->north == O3_FREE_SLIP) { sy = p->ny - 1; src = reflect3(L, src, 1); }
    else sy -= p->ny;
  }
  if (sz < 0) {
    if (p->bottom == O3_FREE_SLIP) { sz = 0; src = reflect3(L, src, 2); }
    else sz += p->nz;
  } else if (sz > p->nz - 1) {
    if (p->top == O3_FREE_SLIP) { sz = p->nz - 1; src = reflect3(L, src, 2); }
    else sz -= p->nz;
  }
  return g[IDX3(p, src, sz, sy, sx)];
}

void ora3_stream(const ora3_params *p, const double *g, double *f) {
  double feq_inlet[QMAX];
  ora3_equilibrium(p->q, p->rho0, p->u_in, feq_inlet);
  for (int a = 0; a < lat3(p->q)->q; a++)
    for (int k = 0; k < p->nz; k++)
      for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) f[IDX3(p, a, k, j, i)] = pull3(p, g, feq_inlet, a, i, j, k);
}

/* U_O = V + omega x (x - c), plus kappa (x - c) for a deforming body (the velocity of its
 * homogeneous dilation) */
static void body_velocity3(const ora3_body *b, int i, int j, int k, double *uo) {
  double r[3] = {(double)i - b->c[0], (double)j - b->c[1], (double)k - b->c[2]};
  uo[0] = b->v[0] + (b->w[1] * r[2] - b->w[2] * r[1]);
  uo[1] = b->v[1] + (b->w[2] * r[0] - b->w[0] * r[2]);
  uo[2] = b->v[2] + (b->w[0] * r[1] - b->w[1] * r[0]);
  if (b->deform)
    for (int d = 0; d < 3; d++) uo[d] = uo[d] + b->kappa * r[d];
}

/* steps (3)-(5) at one node: rho, u* (Eq. rho, Eq. rho*velocity-star), penalization
 * (Eq. d-V, Eq. force-density), corrected velocity (Eq. velocity-r) */
static void node3(const ora3_params *p, const uint8_t *mask, const ora3_body *bodies,
                  const double *f, int i, int j, int k, double *rho, double *u, double *fv) {
  const lattice3 *L = lat3(p->q);
  double r = 0.0, jm[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < L->q; a++) {
    r += f[a];
    jm[0] += L->ex[a] * f[a];
    jm[1] += L->ey[a] * f[a];
    jm[2] += L->ez[a] * f[a];
  }
  int b = mask[((size_t)k * p->ny + j) * p->nx + i];
  double chi = b ? 1.0 : 0.0, uo[3] = {0.0, 0.0, 0.0};
  if (b) body_velocity3(&bodies[b - 1], i, j, k, uo);
  for (int d = 0; d < 3; d++) {
    double us = jm[d] / r;
    double du = chi * (uo[d] - us) / (2.0 * p->eta + chi);
    fv[d] = 2.0 * r * chi * (uo[d] - us) / (2.0 * p->eta + chi);
    u[d] = us + du;
  }
  *rho = r;
}

/* One TRT-LBM-VP step in 3D (Eq. TRT-collision, Eq. collision-modified); force[3*(b-1)+d]
 * receives the force on body b (-sum of F_VP over its nodes, serial in index order). */
void ora3_step_trt(const ora3_params *p, const uint8_t *mask, const ora3_body *bodies,
                   int32_t nbodies, const double *g_in, double *g_out, double *force) {
  const double tau_s = ora3_tau_s(p), tau_a = ora3_tau_a(p);
  const int nq = lat3(p->q)->q;
  double feq_inlet[QMAX];
  ora3_equilibrium(p->q, p->rho0, p->u_in, feq_inlet);
  size_t cells = (size_t)p->nx * p->ny * p->nz;
  double *fvall = (double *)malloc(sizeof(double) * 3 * cells);
  if (!fvall) abort();
#pragma omp parallel for schedule(static)
  for (int k = 0; k < p->nz; k++)
    for (int j = 0; j < p->ny; j++)
      for (int i = 0; i < p->nx; i++) {
        double f[QMAX], feq[QMAX], F[QMAX], rho, u[3], fv[3];
        for (int a = 0; a < nq; a++) f[a] = pull3(p, g_in, feq_inlet, a, i, j, k);
        node3(p, mask, bodies, f, i, j, k, &rho, u, fv);
        ora3_equilibrium(p->q, rho, u, feq);
        ora3_guo(p->q, u, fv, F);
        for (int a = 0; a < nq; a++) {
          int o = opposite3(a);
          double fs = 0.5 * (f[a] + f[o]), fa = 0.5 * (f[a] - f[o]);
          double feqs = 0.5 * (feq[a] + feq[o]), feqa = 0.5 * (feq[a] - feq[o]);
          double Fs = 0.5 * (F[a] + F[o]), Fa = 0.5 * (F[a] - F[o]);
          double om = -(fs - feqs) / tau_s - (fa - feqa) / tau_a;
          g_out[IDX3(p, a, k, j, i)] =
              f[a] + om + (1.0 - 1.0 / (2.0 * tau_s)) * Fs + (1.0 - 1.0 / (2.0 * tau_a)) * Fa;
        }
        size_t c = ((size_t)k * p->ny + j) * p->nx + i;
        for (int d = 0; d < 3; d++) fvall[3 * c + d] = fv[d];
      }
  for (int q = 0; q < 3 * nbodies; q++) force[q] = 0.0;
  for (size_t c = 0; c < cells; c++) {
    int b = mask[c];
    if (b && b <= nbodies)
      for (int d = 0; d < 3; d++) force[3 * (b - 1) + d] -= fvall[3 * c + d];
  }
  free(fvall);
}

int ora3_run(const ora3_params *p, const uint8_t *mask, const ora3_body *bodies, int32_t nbodies,
             double *g, int64_t n, double *forces) {
  size_t cells = (size_t)p->nx * p->ny * p->nz;
  const int nq = lat3(p->q)->q;
  double *tmp = (double *)malloc(sizeof(double) * nq * cells);
  double *fb = (double *)malloc(sizeof(double) * 3 * (nbodies > 0 ? nbodies : 1));
  if (!tmp || !fb) { free(tmp); free(fb); return -1; }
  double *a = g, *b = tmp;
  for (int64_t s = 0; s < n; s++) {
    ora3_step_trt(p, mask, bodies, nbodies, a, b, fb);
    if (forces) memcpy(forces + (size_t)s * 3 * nbodies, fb, sizeof(double) * 3 * nbodies);
    double *t = a; a = b; b = t;
  }
  if (a != g) memcpy(g, a, sizeof(double) * nq * cells);
  free(tmp);
  free(fb);
  return 0;
}

/* ---- moving bodies (prescribed translation, reading M1 in 3D) ----------------------------
 * Sec. 2.2 lets chi and U_O depend on time. A moving domain's body k is centred at
 * c_k + V_k n at step index n and each of its shapes is translated by V_k n; the step from
 * n to n + 1 uses the geometry of index n; the angular velocity acts through U_O about the
 * moving centre. */
/* ---- deforming bodies (reading M1c in 3D) -------------------------------------------------
 * A deforming body pulsates about its centre: at step index n its shapes are scaled by
 * s(n) = 1 + amp sin(rate n) (|amp| < 1), radii by s(n) and each shape's offset d from the
 * body's reference centre to s(n) d; the dilation is isotropic, so such a body is made of
 * spheres (an infinite z-cylinder has no centre along z); U_O adds kappa(n) (x - c), kappa = s'/s =
 * amp rate cos(rate n) / s(n). sin and cos are written out in FP64 (Cody and Waite's
 * reduction by pi/2 split in three parts, the first two of 30 significant bits; Taylor
 * series of sin and cos on [-pi/4, pi/4] to r^17 and r^16 by Horner's rule in r^2; the
 * quadrant k mod 4), so that the mask depends on no math library. */
static void sincos3(double t, double *s, double *c) {
  const double P1 = 0x1.921fb54p+0, P2 = 0x1.10b46118p-30, P3 = 0x1.313198a2e037p-61;
  const double k = nearbyint(t * 0x1.45f306dc9c883p-1);
  const double r = ((t - k * P1) - k * P2) - k * P3;
  const double r2 = r * r;
  double ps = -1.0 / 1307674368000.0 + r2 * (1.0 / 355687428096000.0);
  ps = 1.0 / 6227020800.0 + r2 * ps;
  ps = -1.0 / 39916800.0 + r2 * ps;
  ps = 1.0 / 362880.0 + r2 * ps;
  ps = -1.0 / 5040.0 + r2 * ps;
  ps = 1.0 / 120.0 + r2 * ps;
  ps = -1.0 / 6.0 + r2 * ps;
  const double sr = r + (r * r2) * ps;
  double pc = -1.0 / 87178291200.0 + r2 * (1.0 / 20922789888000.0);
  pc = 1.0 / 479001600.0 + r2 * pc;
  pc = -1.0 / 3628800.0 + r2 * pc;
  pc = 1.0 / 40320.0 + r2 * pc;
  pc = -1.0 / 720.0 + r2 * pc;
  pc = 1.0 / 24.0 + r2 * pc;
  pc = -0.5 + r2 * pc;
  const double cr = 1.0 + r2 * pc;
  switch ((int)((int64_t)k & 3)) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}

void ora3_sincos(double t, double *s, double *c) { sincos3(t, s, c); }

static double pulse3(const ora3_body *b0, int64_t n, double *kappa) {
  double sn, cs;
  sincos3(b0->rate * (double)n, &sn, &cs);
  const double sc = 1.0 + b0->amp * sn;
  if (kappa) *kappa = ((b0->amp * b0->rate) * cs) / sc;
  return sc;
}

static void bodies3_at(const ora3_body *b0, int32_t nbodies, int64_t n, ora3_body *out) {
  for (int k = 0; k < nbodies; k++) {
    out[k] = b0[k];
    for (int d = 0; d < 3; d++) out[k].c[d] = b0[k].c[d] + b0[k].v[d] * (double)n;
    if (b0[k].deform) pulse3(&b0[k], n, &out[k].kappa);
  }
}

/* The body table at step index n (centres moved; dilation rates of deforming bodies). */
void ora3_bodies_at(const ora3_body *b0, int32_t nbodies, int64_t n, ora3_body *out) {
  bodies3_at(b0, nbodies, n, out);
}

/* The mask at step index n (shapes translated with their bodies; those of deforming bodies
 * also scaled about the body's centre). */
void ora3_rasterize_at(int32_t nx, int32_t ny, int32_t nz, const ora3_shape *shapes, int32_t nshapes,
                       const ora3_body *bodies, int32_t nbodies, int64_t n, uint8_t *mask) {
  ora3_shape *moved = (ora3_shape *)malloc(sizeof(ora3_shape) * (nshapes > 0 ? nshapes : 1));
  if (!moved) abort();
  for (int q = 0; q < nshapes; q++) {
    moved[q] = shapes[q];
    const int k = shapes[q].body - 1;
    if (k >= 0 && k < nbodies && bodies[k].deform) {
      const double sc = pulse3(&bodies[k], n, NULL);
      for (int d = 0; d < 3; d++)
        moved[q].c[d] = (bodies[k].c[d] + bodies[k].v[d] * (double)n) + sc * (shapes[q].c[d] - bodies[k].c[d]);
      moved[q].radius = sc * shapes[q].radius;
    } else if (k >= 0 && k < nbodies) {
      for (int d = 0; d < 3; d++) moved[q].c[d] = shapes[q].c[d] + bodies[k].v[d] * (double)n;
    }
  }
  ora3_rasterize(nx, ny, nz, moved, nshapes, mask);
  free(moved);
}

/* n steps of a moving domain from step index n0. */
int ora3_run_moving(const ora3_params *p, const ora3_shape *shapes, int32_t nshapes,
                    const ora3_body *bodies, int32_t nbodies, double *g, int64_t n0, int64_t n,
                    double *forces) {
  size_t cells = (size_t)p->nx * p->ny * p->nz;
  const int nq = lat3(p->q)->q;
  double *tmp = (double *)malloc(sizeof(double) * nq * cells);
  double *fb = (double *)malloc(sizeof(double) * 3 * (nbodies > 0 ? nbodies : 1));
  uint8_t *mask = (uint8_t *)malloc(cells);
  ora3_body *now = (ora3_body *)malloc(sizeof(ora3_body) * (nbodies > 0 ? nbodies : 1));
  if (!tmp || !fb || !mask || !now) { free(tmp); free(fb); free(mask); free(now); return -1; }
  double *a = g, *b = tmp;
  for (int64_t s = 0; s < n; s++) {
    const int64_t m = n0 + s;
    ora3_rasterize_at(p->nx, p->ny, p->nz, shapes, nshapes, bodies, nbodies, m, mask);
    bodies3_at(bodies, nbodies, m, now);
    ora3_step_trt(p, mask, now, nbodies, a, b, fb);
    if (forces) memcpy(forces + (size_t)s * 3 * nbodies, fb, sizeof(double) * 3 * nbodies);
    double *t = a; a = b; b = t;
  }
  if (a != g) memcpy(g, a, sizeof(double) * nq * cells);
  free(tmp); free(fb); free(mask); free(now);
  return 0;
}

/* ---- coupled bodies (fluid-structure coupling, reading M4 in 3D) ------------------------
 * As in 2D: a body with dynamics is a rigid body of mass M on springs k (anchored at its
 * initial centre x0) with dampers c; after every step each free axis advances by
 * semi-implicit Euler (dt = 1) driven by the mean of the forces of this step and the
 * previous one, Fm = (F_n + F_{n-1}) / 2:  v <- v + (Fm - k (x - x0) - c v) / M, then
 * x <- x + v; an axis that is not free keeps its velocity. The mask and U_O of a step use
 * the state before its update; shapes translate with the centre; the angular velocity
 * stays as given. Bodies without dynamics keep their prescribed motion (c + V n). */
typedef struct {
  double mass, k[3], c[3];
  int32_t free_axis[3], active;
} ora3_dynamics;

static void fsi3_axis(double F, double *Fp, double k, double c, double M, int32_t free_axis,
                      double x0, double *x, double *v) {
  if (free_axis) {
    double Fm = (F + *Fp) * 0.5;
    double t = Fm - k * (*x - x0);
    t = t - c * *v;
    *v = *v + t / M;
  }
  *x = *x + *v;
  *Fp = F;
}

/* n steps from step index n0 with coupled bodies; state [nbodies][9] holds x[3], v[3] and
 * the previous step's force F[3] of the bodies with dynamics, advanced in place; track, if
 * not NULL, receives (x, v) each step used, [n][nbodies][6]. */
int ora3_run_fsi(const ora3_params *p, const ora3_shape *shapes, int32_t nshapes,
                 const ora3_body *bodies, const ora3_dynamics *dyn, int32_t nbodies, double *g,
                 int64_t n0, int64_t n, double *state, double *forces, double *track) {
  size_t cells = (size_t)p->nx * p->ny * p->nz;
  const int nq = lat3(p->q)->q;
  double *tmp = (double *)malloc(sizeof(double) * nq * cells);
  double *fb = (double *)malloc(sizeof(double) * 3 * (nbodies > 0 ? nbodies : 1));
  uint8_t *mask = (uint8_t *)malloc(cells);
  ora3_body *now = (ora3_body *)malloc(sizeof(ora3_body) * (nbodies > 0 ? nbodies : 1));
  ora3_shape *sh = (ora3_shape *)malloc(sizeof(ora3_shape) * (nshapes > 0 ? nshapes : 1));
  if (!tmp || !fb || !mask || !now || !sh) {
    free(tmp); free(fb); free(mask); free(now); free(sh);
    return -1;
  }
  double *a = g, *b = tmp;
  for (int64_t s = 0; s < n; s++) {
    const int64_t m = n0 + s;
    bodies3_at(bodies, nbodies, m, now);
    for (int k = 0; k < nbodies; k++) {
      if (dyn[k].active)
        for (int d = 0; d < 3; d++) {
          now[k].c[d] = state[9 * k + d];
          now[k].v[d] = state[9 * k + 3 + d];
        }
      if (track)
        for (int d = 0; d < 3; d++) {
          track[((size_t)s * nbodies + k) * 6 + d] = now[k].c[d];
          track[((size_t)s * nbodies + k) * 6 + 3 + d] = now[k].v[d];
        }
    }
    for (int q = 0; q < nshapes; q++) {
      sh[q] = shapes[q];
      const int k = shapes[q].body - 1;
      if (k < 0 || k >= nbodies) continue;
      for (int d = 0; d < 3; d++)
        sh[q].c[d] = dyn[k].active ? shapes[q].c[d] + (state[9 * k + d] - bodies[k].c[d])
                                   : shapes[q].c[d] + bodies[k].v[d] * (double)m;
    }
    ora3_rasterize(p->nx, p->ny, p->nz, sh, nshapes, mask);
    ora3_step_trt(p, mask, now, nbodies, a, b, fb);
    if (forces) memcpy(forces + (size_t)s * 3 * nbodies, fb, sizeof(double) * 3 * nbodies);
    for (int k = 0; k < nbodies; k++) {
      if (!dyn[k].active) continue;
      double *st = &state[9 * k];
      for (int d = 0; d < 3; d++)
        fsi3_axis(fb[3 * k + d], &st[6 + d], dyn[k].k[d], dyn[k].c[d], dyn[k].mass, dyn[k].free_axis[d],
                  bodies[k].c[d], &st[d], &st[3 + d]);
    }
    double *t = a; a = b; b = t;
  }
  if (a != g) memcpy(g, a, sizeof(double) * nq * cells);
  free(tmp); free(fb); free(mask); free(now); free(sh);
  return 0;
}

void ora3_init(const ora3_params *p, const double *u0, double *g) {
  double feq[QMAX];
  ora3_equilibrium(p->q, p->rho0, u0, feq);
  size_t cells = (size_t)p->nx * p->ny * p->nz;
  for (int a = 0; a < lat3(p->q)->q; a++)
    for (size_t c = 0; c < cells; c++) g[a * cells + c] = feq[a];
}

void ora3_moments(const ora3_params *p, const uint8_t *mask, const ora3_body *bodies,
                  const double *g, double *rho, double *ux, double *uy, double *uz) {
  double feq_inlet[QMAX];
  ora3_equilibrium(p->q, p->rho0, p->u_in, feq_inlet);
  const int nq = lat3(p->q)->q;
  for (int k = 0; k < p->nz; k++)
    for (int j = 0; j < p->ny; j++)
      for (int i = 0; i < p->nx; i++) {
        double f[QMAX], r, u[3], fv[3];
        for (int a = 0; a < nq; a++) f[a] = pull3(p, g, feq_inlet, a, i, j, k);
        node3(p, mask, bodies, f, i, j, k, &r, u, fv);
        size_t c = ((size_t)k * p->ny + j) * p->nx + i;
        rho[c] = r;
        ux[c] = u[0];
        uy[c] = u[1];
        uz[c] = u[2];
      }
}

/* the velocity set of lattice q (15 or 19; its size is returned, -1 without writing if the
 * selected table has another size than the caller's buffers), for the pins */
int32_t ora3_lattice(int32_t q, int32_t *ex, int32_t *ey, int32_t *ez, double *w, int32_t *opp) {
  const lattice3 *L = lat3(q);
  if (L->q != (q == 15 ? 15 : 19)) return -1;
  for (int a = 0; a < L->q; a++) {
    ex[a] = L->ex[a];
    ey[a] = L->ey[a];
    ez[a] = L->ez[a];
    w[a] = L->w[a];
    opp[a] = opposite3(a);
  }
  return L->q;
}

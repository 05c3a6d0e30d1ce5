/*
 * Plain FP64 CPU oracle of the TRT-LBM-VP method (Cui, Wang, Yao, Liu, Yu,
 * "A coupled two-relaxation-time lattice Boltzmann-volume penalization method for
 * flows past obstacles", arXiv:1901.08766). TEST INFRASTRUCTURE ONLY: it is used by
 * the tests, by the package's smoke check and by the benchmark's CPU baseline,
 * never by the library's compute path. It shares no source with the CUDA library.
 *
 * Written for a reader checking it against the paper by eye: one cell at a time,
 * the paper's notation (tau_s, tau_a, f^s, f^a, F^s, F^a, u*, du, F_VP), no fusion
 * beyond what the equations state. Compiled with -O2 -ffp-contract=off.
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *  - tau_s = nu / c_s^2 + 1/2 (the printed relation omits the +1/2, Sec. 2.1);
 *  - the Guo term is used without the extra (1 - 1/(2 lambda)) prefactor of its
 *    definition, since the modified collision already relaxes F^s and F^a once each;
 *  - f^eq and the Guo term use the corrected velocity u = u* + du, F_VP uses u*;
 *  - the state is the post-collision population g; a step pulls g from the
 *    neighbours (streaming), forms rho and u*, penalizes, then collides;
 *  - edges: equilibrium inlet ghost, zero-gradient outflow, specular free-slip, or
 *    periodic; the x rule is applied before the y rule;
 *  - the reported force on body k is the force ON the body, -sum F_VP over its cells.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

/* D2Q9 velocities, Eq. (D2Q9): alpha = 0 rest, 1..4 at angles (alpha-1) pi/2,
 * 5..8 at angles (2 alpha - 9) pi/4 with length sqrt(2). */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* opposite direction -alpha (Sec. 2.1: f_{-1} = f_3, f_{-0} = f_0) */
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* reflection across a horizontal wall (e_y -> -e_y), used by free-slip edges */
static const int REFLECT_Y[Q] = {0, 1, 4, 3, 2, 8, 7, 6, 5};
/* weights below Eq. (feq) */
static const double WGT[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2, c_s = 1/sqrt(3) */

/* edge kinds */
enum { ORA_PERIODIC = 0, ORA_INLET = 1, ORA_OUTFLOW = 2, ORA_FREE_SLIP = 3 };
/* shape kinds */
enum { ORA_CIRCLE = 0, ORA_ANNULUS_OUTSIDE = 1, ORA_NACA4 = 2 };

typedef struct {
  int32_t nx, ny;
  double nu, magic_lambda, eta, rho0;
  double u_in_x, u_in_y;
  int32_t west, east, south, north;
} ora_params;

typedef struct {
  double cx, cy, vx, vy, omega;
  /* a deforming body (deform = 1) pulsates: scale s(n) = 1 + amp sin(rate n) about its
   * centre; kappa = s'(n) / s(n) is its dilation rate at the step being taken */
  double amp, rate, kappa;
  int32_t deform, pad;
} ora_body;

typedef struct {
  int32_t kind, body;
  double cx, cy, radius;
  double chord, thickness, aoa_rad;
} ora_shape;

/* ---- relaxation times (Sec. 2.1) ------------------------------------------------ */

double ora_tau_s(const ora_params *p) { return p->nu / CS2 + 0.5; }

/* magic parameter Lambda = (tau_s - 1/2)(tau_a - 1/2) solved for tau_a */
double ora_tau_a(const ora_params *p) {
  return 0.5 + p->magic_lambda / (ora_tau_s(p) - 0.5);
}

/* ---- equilibrium, Eq. (feq) -------------------------------------------------------- */

void ora_equilibrium(double rho, double ux, double uy, double *feq) {
  double usq = ux * ux + uy * uy;
  for (int a = 0; a < Q; a++) {
    double eu = EX[a] * ux + EY[a] * uy;
    feq[a] = rho * WGT[a] * (1.0 + eu / CS2 + (eu * eu - CS2 * usq) / (2.0 * CS2 * CS2));
  }
}

/* Guo forcing term of Eq. (external-force-term) without its leading prefactor:
 * F_alpha = w_alpha [ (e_alpha - u)/c_s^2 + (e_alpha . u) e_alpha / c_s^4 ] . F */
void ora_guo(double ux, double uy, double fx, double fy, double *F) {
  for (int a = 0; a < Q; a++) {
    double eu = EX[a] * ux + EY[a] * uy;
    double cx = (EX[a] - ux) / CS2 + eu * EX[a] / (CS2 * CS2);
    double cy = (EY[a] - uy) / CS2 + eu * EY[a] / (CS2 * CS2);
    F[a] = WGT[a] * (cx * fx + cy * fy);
  }
}

/* ---- geometry -> mask chi (Eq. mask function) -------------------------------------- */

/* NACA 4-digit symmetric half thickness at x = x'/c (open trailing edge), times c. */
double ora_naca_half_thickness(double xc, double t, double chord) {
  double s = sqrt(xc);
  double p = (((-0.1015 * xc + 0.2843) * xc - 0.3516) * xc - 0.1260) * xc;
  return 5.0 * t * chord * (0.2969 * s + p);
}

/* inside test of shape s, a NACA section oriented by (ca, sa) = (cos, sin) of its angle
 * of attack */
static int inside_shape_cs(const ora_shape *s, double ca, double sa, double x, double y) {
  if (s->kind == ORA_CIRCLE || s->kind == ORA_ANNULUS_OUTSIDE) {
    double dx = x - s->cx, dy = y - s->cy;
    double d2 = dx * dx + dy * dy;
    double r2 = s->radius * s->radius;
    return s->kind == ORA_CIRCLE ? (d2 < r2) : (d2 > r2);
  }
  if (s->kind == ORA_NACA4) {
    /* quarter chord at (cx, cy); nose-up angle of attack positive */
    double qc = 0.25 * s->chord;
    double lex = s->cx - qc * ca, ley = s->cy + qc * sa; /* leading edge */
    double dx = x - lex, dy = y - ley;
    double xp = dx * ca - dy * sa; /* along the chord */
    double yp = dx * sa + dy * ca; /* normal to the chord */
    if (!(xp >= 0.0 && xp <= s->chord)) return 0;
    double yt = ora_naca_half_thickness(xp / s->chord, s->thickness, s->chord);
    return fabs(yp) <= yt;
  }
  return 0;
}

static int inside_shape(const ora_shape *s, double x, double y) {
  return inside_shape_cs(s, cos(s->aoa_rad), sin(s->aoa_rad), x, y);
}

/* Body id per node (0 = fluid); later shapes overwrite earlier ones. */
void ora_rasterize(int32_t nx, int32_t ny, const ora_shape *shapes, int32_t nshapes,
                   uint8_t *mask) {
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      uint8_t b = 0;
      for (int k = 0; k < nshapes; k++)
        if (inside_shape(&shapes[k], (double)i, (double)j)) b = (uint8_t)shapes[k].body;
      mask[(size_t)j * nx + i] = b;
    }
}

/* ---- moving obstacles ---------------------------------------------------------------------
 * chi(x, t) and U_O(x, t) may depend on time (Sec. 2.2, the penalized equations hold for
 * moving obstacles). Prescribed translation: at step index n body k has its centre at
 * c_k + V_k n and each of its shapes is translated by V_k n; rotation enters through
 * U_O only (exact for circles about their centre). */
static void shape_at(const ora_shape *s0, const ora_body *bodies, int32_t nbodies, int64_t n,
                     ora_shape *s) {
  *s = *s0;
  if (s0->body >= 1 && s0->body <= nbodies) {
    const ora_body *b = &bodies[s0->body - 1];
    s->cx = s0->cx + b->vx * (double)n;
    s->cy = s0->cy + b->vy * (double)n;
  }
}

void ora_sincos(double t, double *s, double *c);

/* ---- deforming obstacles (reading M1c) ----------------------------------------------------
 * A deforming body pulsates about its centre: at step index n its shapes are scaled by
 * s(n) = 1 + amp sin(rate n) (|amp| < 1): radii and chords by s(n), a shape's offset d from
 * the body centre to s(n) d (after the rotation of a rotating domain). Its material
 * velocity adds the dilation kappa(n) (x - c), kappa(n) = s'(n) / s(n) =
 * amp rate cos(rate n) / s(n), to U_O. */
static double deform_scale(const ora_body *b0, int64_t n, double *kappa) {
  double sn, cs;
  ora_sincos(b0->rate * (double)n, &sn, &cs);
  const double sc = 1.0 + b0->amp * sn;
  if (kappa) *kappa = ((b0->amp * b0->rate) * cs) / sc;
  return sc;
}

static void body_at(const ora_body *b0, int64_t n, ora_body *b) {
  *b = *b0;
  b->cx = b0->cx + b0->vx * (double)n;
  b->cy = b0->cy + b0->vy * (double)n;
  if (b0->deform) deform_scale(b0, n, &b->kappa);
}

/* ---- rotating obstacles (reading M1b) -----------------------------------------------------
 * A body of a rotating domain turns its shapes with it: at step index n body k has turned
 * by theta = omega_k n (counter-clockwise, the sense of U_O = omega z x (x - c)) about its
 * centre, which moves as c_k + V_k n. A shape whose reference point (circle centre, NACA
 * quarter chord) is offset by d from the body's reference centre sits at c_k + V_k n + R d,
 * R the rotation by theta, and a NACA section's angle of attack (nose up) decreases by
 * theta: (cos, sin) of aoa - theta by the angle-difference rule from cos aoa, sin aoa.
 *
 * sin and cos are written out in FP64, so that the placement does not depend on a math
 * library: the argument is reduced by multiples k of pi/2 (Cody and Waite, with pi/2 split
 * in three parts, the first two of 30 significant bits, so that k times them is exact for
 * |k| < 2^23, i.e. |theta| < 1.3e7), then sin r and cos r on [-pi/4, pi/4] are the Taylor
 * series to the terms in r^17 and r^16 (truncation below 1e-17), evaluated by Horner's
 * rule in r^2; the quadrant k mod 4 selects signs and roles. */
void ora_sincos(double t, double *s, double *c) {
  const double P1 = 0x1.921fb54p+0, P2 = 0x1.10b46118p-30, P3 = 0x1.313198a2e037p-61;
  const double k = nearbyint(t * 0x1.45f306dc9c883p-1); /* t 2/pi, to nearest */
  const double r = ((t - k * P1) - k * P2) - k * P3;
  const double r2 = r * r;
  double ps = -1.0 / 1307674368000.0 + r2 * (1.0 / 355687428096000.0); /* -1/15!, 1/17! */
  ps = 1.0 / 6227020800.0 + r2 * ps;                                     /* 1/13! */
  ps = -1.0 / 39916800.0 + r2 * ps;                                      /* -1/11! */
  ps = 1.0 / 362880.0 + r2 * ps;                                         /* 1/9! */
  ps = -1.0 / 5040.0 + r2 * ps;                                          /* -1/7! */
  ps = 1.0 / 120.0 + r2 * ps;                                            /* 1/5! */
  ps = -1.0 / 6.0 + r2 * ps;                                             /* -1/3! */
  const double sr = r + (r * r2) * ps;
  double pc = -1.0 / 87178291200.0 + r2 * (1.0 / 20922789888000.0);     /* -1/14!, 1/16! */
  pc = 1.0 / 479001600.0 + r2 * pc;                                      /* 1/12! */
  pc = -1.0 / 3628800.0 + r2 * pc;                                       /* -1/10! */
  pc = 1.0 / 40320.0 + r2 * pc;                                          /* 1/8! */
  pc = -1.0 / 720.0 + r2 * pc;                                           /* -1/6! */
  pc = 1.0 / 24.0 + r2 * pc;                                             /* 1/4! */
  pc = -0.5 + r2 * pc;                                                   /* -1/2! */
  const double cr = 1.0 + r2 * pc;
  switch ((int)((int64_t)k & 3)) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}

typedef struct {
  ora_shape s;
  double ca, sa; /* cos, sin of the NACA angle of attack */
} placed_shape;

/* shape s0 at step index n of a body that turns (rotate: a rotating domain) or deforms:
 * reference point at c + V n + s(n) R(theta) d */
static void shape_rot_at(const ora_shape *s0, const ora_body *bodies, int32_t nbodies, int64_t n,
                         int32_t rotate, placed_shape *out) {
  out->s = *s0;
  out->ca = cos(s0->aoa_rad);
  out->sa = sin(s0->aoa_rad);
  if (s0->body < 1 || s0->body > nbodies) return;
  const ora_body *b = &bodies[s0->body - 1];
  const double dx = s0->cx - b->cx, dy = s0->cy - b->cy;
  double rx = dx, ry = dy;
  if (rotate) {
    double sn, cs;
    ora_sincos(b->omega * (double)n, &sn, &cs);
    rx = cs * dx - sn * dy;
    ry = sn * dx + cs * dy;
    const double ca = out->ca, sa = out->sa;
    out->ca = ca * cs + sa * sn; /* cos(aoa - theta) */
    out->sa = sa * cs - ca * sn; /* sin(aoa - theta) */
  }
  if (b->deform) {
    const double sc = deform_scale(b, n, NULL);
    rx = sc * rx;
    ry = sc * ry;
    out->s.radius = sc * s0->radius;
    out->s.chord = sc * s0->chord;
  }
  out->s.cx = (b->cx + b->vx * (double)n) + rx;
  out->s.cy = (b->cy + b->vy * (double)n) + ry;
}

/* The mask of a rotating (rotate = 1) or translating domain with deforming bodies at step
 * index n. */
static void rasterize_placed(int32_t nx, int32_t ny, const ora_shape *shapes, int32_t nshapes,
                             const ora_body *bodies, int32_t nbodies, int64_t n, int32_t rotate,
                             uint8_t *mask) {
  placed_shape *ps = (placed_shape *)malloc(sizeof(placed_shape) * (nshapes > 0 ? nshapes : 1));
  if (!ps) abort();
  for (int k = 0; k < nshapes; k++) {
    const int b = shapes[k].body;
    if (rotate || (b >= 1 && b <= nbodies && bodies[b - 1].deform)) {
      shape_rot_at(&shapes[k], bodies, nbodies, n, rotate, &ps[k]);
    } else {
      shape_at(&shapes[k], bodies, nbodies, n, &ps[k].s);
      ps[k].ca = cos(shapes[k].aoa_rad);
      ps[k].sa = sin(shapes[k].aoa_rad);
    }
  }
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      uint8_t b = 0;
      for (int k = 0; k < nshapes; k++)
        if (inside_shape_cs(&ps[k].s, ps[k].ca, ps[k].sa, (double)i, (double)j)) b = (uint8_t)ps[k].s.body;
      mask[(size_t)j * nx + i] = b;
    }
  free(ps);
}

void ora_rasterize_rot(int32_t nx, int32_t ny, const ora_shape *shapes, int32_t nshapes,
                       const ora_body *bodies, int32_t nbodies, int64_t n, uint8_t *mask) {
  rasterize_placed(nx, ny, shapes, nshapes, bodies, nbodies, n, 1, mask);
}

/* The mask at step index n (shapes translated with their bodies; those of deforming bodies
 * also scaled). */
void ora_rasterize_at(int32_t nx, int32_t ny, const ora_shape *shapes, int32_t nshapes,
                      const ora_body *bodies, int32_t nbodies, int64_t n, uint8_t *mask) {
  for (int k = 0; k < nbodies; k++)
    if (bodies[k].deform) {
      rasterize_placed(nx, ny, shapes, nshapes, bodies, nbodies, n, 0, mask);
      return;
    }
  ora_shape *moved = (ora_shape *)malloc(sizeof(ora_shape) * (nshapes > 0 ? nshapes : 1));
  if (!moved) abort();
  for (int k = 0; k < nshapes; k++) shape_at(&shapes[k], bodies, nbodies, n, &moved[k]);
  ora_rasterize(nx, ny, moved, nshapes, mask);
  free(moved);
}

/* ---- streaming with the domain-edge rules (Eq. streaming) ---------------------------- */

static inline double G(const double *g, const ora_params *p, int a, int j, int i) {
  return g[((size_t)a * p->ny + j) * p->nx + i];
}

/* f_alpha(i, j) = g_alpha(i - e_x, j - e_y) at the previous time level. */
static double pull(const ora_params *p, const double *g, const double *feq_inlet, int a,
                   int i, int j) {
  int sx = i - EX[a], sy = j - EY[a], src = a;
  if (sx < 0) {
    if (p->west == ORA_INLET) return feq_inlet[a];
    sx += p->nx;
  } else if (sx > p->nx - 1) {
    if (p->east == ORA_OUTFLOW) sx = p->nx - 1;
    else sx -= p->nx;
  }
  if (sy < 0) {
    if (p->south == ORA_FREE_SLIP) { sy = 0; src = REFLECT_Y[a]; }
    else sy += p->ny;
  } else if (sy > p->ny - 1) {
    if (p->north == ORA_FREE_SLIP) { sy = p->ny - 1; src = REFLECT_Y[a]; }
    else sy -= p->ny;
  }
  return G(g, p, src, sy, sx);
}

/* Step (3) alone: f(x) = g(x - e_alpha) for every node and direction, with the edge
 * rules of pull(). Used to pin the streaming and edge rules on their own. */
void ora_stream(const ora_params *p, const double *g, double *f) {
  double feq_inlet[Q];
  ora_equilibrium(p->rho0, p->u_in_x, p->u_in_y, feq_inlet);
  for (int a = 0; a < Q; a++)
    for (int j = 0; j < p->ny; j++)
      for (int i = 0; i < p->nx; i++)
        f[((size_t)a * p->ny + j) * p->nx + i] = pull(p, g, feq_inlet, a, i, j);
}

/* Obstacle velocity U_O at node (i, j) of body k: V_k + Omega_k z x (x - c_k), plus
 * kappa_k (x - c_k) for a deforming body (the velocity of its homogeneous dilation). */
static void body_velocity(const ora_body *b, int i, int j, double *uox, double *uoy) {
  *uox = b->vx - b->omega * ((double)j - b->cy);
  *uoy = b->vy + b->omega * ((double)i - b->cx);
  if (b->deform) {
    *uox = *uox + b->kappa * ((double)i - b->cx);
    *uoy = *uoy + b->kappa * ((double)j - b->cy);
  }
}

/* Per-node macroscopic step shared by the TRT and SRT updates: steps (3)-(5) of the
 * algorithm of Sec. 2.2. Outputs rho, the corrected velocity u and F_VP. */
static void node_moments(const ora_params *p, const uint8_t *mask, const ora_body *bodies,
                         const double *f, int i, int j, double *rho, double *ux,
                         double *uy, double *fvx, double *fvy) {
  /* Eq. (rho), Eq. (rho*velocity-star) */
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int a = 0; a < Q; a++) {
    r += f[a];
    jx += EX[a] * f[a];
    jy += EY[a] * f[a];
  }
  double usx = jx / r, usy = jy / r;
  int b = mask[(size_t)j * p->nx + i];
  double chi = b ? 1.0 : 0.0;
  double uox = 0.0, uoy = 0.0;
  if (b) body_velocity(&bodies[b - 1], i, j, &uox, &uoy);
  const double dt = 1.0;
  /* Eq. (d-V) and Eq. (force-density) */
  double dux = chi * (uox - usx) / (2.0 * p->eta / dt + chi);
  double duy = chi * (uoy - usy) / (2.0 * p->eta / dt + chi);
  *fvx = 2.0 * r * chi * (uox - usx) / (2.0 * p->eta + chi * dt);
  *fvy = 2.0 * r * chi * (uoy - usy) / (2.0 * p->eta + chi * dt);
  /* Eq. (velocity-r) */
  *ux = usx + dux;
  *uy = usy + duy;
  *rho = r;
}

/* Force on body k = -sum of F_VP over its nodes (Eq. hydrodynamic force with the
 * sign read as the force on the body), summed serially in row-major order. */
static void sum_body_forces(const ora_params *p, const uint8_t *mask, const double *fv,
                            int32_t nbodies, double *force) {
  for (int k = 0; k < 2 * nbodies; k++) force[k] = 0.0;
  for (int j = 0; j < p->ny; j++)
    for (int i = 0; i < p->nx; i++) {
      size_t c = (size_t)j * p->nx + i;
      int b = mask[c];
      if (b && b <= nbodies) {
        force[2 * (b - 1) + 0] -= fv[2 * c];
        force[2 * (b - 1) + 1] -= fv[2 * c + 1];
      }
    }
}

/*
 * One TRT-LBM-VP time step (algorithm of Sec. 2.2, steps (2)-(6)):
 * g_out(x) = collide(pull(g_in)) with Eq. (TRT-collision) and Eq. (collision-modified).
 * force[2*(k-1) + {0,1}] receives the force on body k (row-major sum over its nodes).
 */
void ora_step_trt(const ora_params *p, const uint8_t *mask, const ora_body *bodies,
                  int32_t nbodies, const double *g_in, double *g_out, double *force) {
  const double tau_s = ora_tau_s(p), tau_a = ora_tau_a(p);
  double feq_inlet[Q];
  ora_equilibrium(p->rho0, p->u_in_x, p->u_in_y, feq_inlet);
  size_t cells = (size_t)p->nx * p->ny;
  double *fv = (double *)malloc(sizeof(double) * 2 * cells);
  if (!fv) abort();
#pragma omp parallel for schedule(static)
  for (int j = 0; j < p->ny; j++)
    for (int i = 0; i < p->nx; i++) {
      double f[Q], feq[Q], F[Q];
      for (int a = 0; a < Q; a++) f[a] = pull(p, g_in, feq_inlet, a, i, j);
      double rho, ux, uy, fvx, fvy;
      node_moments(p, mask, bodies, f, i, j, &rho, &ux, &uy, &fvx, &fvy);
      ora_equilibrium(rho, ux, uy, feq);
      ora_guo(ux, uy, fvx, fvy, F);
      for (int a = 0; a < Q; a++) {
        int o = OPP[a];
        double fs = 0.5 * (f[a] + f[o]), fa = 0.5 * (f[a] - f[o]);
        double feqs = 0.5 * (feq[a] + feq[o]), feqa = 0.5 * (feq[a] - feq[o]);
        double Fs = 0.5 * (F[a] + F[o]), Fa = 0.5 * (F[a] - F[o]);
        double omega = -(fs - feqs) / tau_s - (fa - feqa) / tau_a;
        g_out[((size_t)a * p->ny + j) * p->nx + i] =
            f[a] + omega + (1.0 - 1.0 / (2.0 * tau_s)) * Fs + (1.0 - 1.0 / (2.0 * tau_a)) * Fa;
      }
      size_t c = (size_t)j * p->nx + i;
      fv[2 * c] = fvx;
      fv[2 * c + 1] = fvy;
    }
  sum_body_forces(p, mask, fv, nbodies, force);
  free(fv);
}

/*
 * The single-relaxation-time LBM-VP step the paper compares against (Sec. 3.1):
 * g = f - (f - f^eq)/tau + (1 - 1/(2 tau)) F_alpha with tau = tau_s, the full
 * (unsplit) Guo term and the same penalization.
 */
void ora_step_srt(const ora_params *p, const uint8_t *mask, const ora_body *bodies,
                  int32_t nbodies, const double *g_in, double *g_out, double *force) {
  const double tau = ora_tau_s(p);
  double feq_inlet[Q];
  ora_equilibrium(p->rho0, p->u_in_x, p->u_in_y, feq_inlet);
  size_t cells = (size_t)p->nx * p->ny;
  double *fv = (double *)malloc(sizeof(double) * 2 * cells);
  if (!fv) abort();
#pragma omp parallel for schedule(static)
  for (int j = 0; j < p->ny; j++)
    for (int i = 0; i < p->nx; i++) {
      double f[Q], feq[Q], F[Q];
      for (int a = 0; a < Q; a++) f[a] = pull(p, g_in, feq_inlet, a, i, j);
      double rho, ux, uy, fvx, fvy;
      node_moments(p, mask, bodies, f, i, j, &rho, &ux, &uy, &fvx, &fvy);
      ora_equilibrium(rho, ux, uy, feq);
      ora_guo(ux, uy, fvx, fvy, F);
      for (int a = 0; a < Q; a++)
        g_out[((size_t)a * p->ny + j) * p->nx + i] =
            f[a] - (f[a] - feq[a]) / tau + (1.0 - 1.0 / (2.0 * tau)) * F[a];
      size_t c = (size_t)j * p->nx + i;
      fv[2 * c] = fvx;
      fv[2 * c + 1] = fvy;
    }
  sum_body_forces(p, mask, fv, nbodies, force);
  free(fv);
}

/* Run n steps, ping-ponging between g and a scratch lattice; the result ends in g.
 * forces: [n][nbodies][2] (may be NULL). srt != 0 selects the SRT update. */
int ora_run(const ora_params *p, const uint8_t *mask, const ora_body *bodies,
            int32_t nbodies, double *g, int64_t n, double *forces, int32_t srt) {
  size_t cells = (size_t)p->nx * p->ny;
  double *tmp = (double *)malloc(sizeof(double) * Q * cells);
  double *fb = (double *)malloc(sizeof(double) * 2 * (nbodies > 0 ? nbodies : 1));
  if (!tmp || !fb) { free(tmp); free(fb); return -1; }
  double *a = g, *b = tmp;
  for (int64_t s = 0; s < n; s++) {
    if (srt) ora_step_srt(p, mask, bodies, nbodies, a, b, fb);
    else ora_step_trt(p, mask, bodies, nbodies, a, b, fb);
    if (forces) memcpy(forces + (size_t)s * 2 * nbodies, fb, sizeof(double) * 2 * nbodies);
    double *t = a; a = b; b = t;
  }
  if (a != g) memcpy(g, a, sizeof(double) * Q * cells);
  free(tmp);
  free(fb);
  return 0;
}

/* Run n steps of a domain whose bodies move (prescribed translation; with rotate, also
 * rotation of their shapes), starting at step index n0: before step n0 + s the mask is
 * rasterised at that index and the bodies' centres are moved there. Arguments as ora_run,
 * plus the shapes. */
int ora_run_moving_mode(const ora_params *p, const ora_shape *shapes, int32_t nshapes,
                        const ora_body *bodies, int32_t nbodies, double *g, int64_t n0, int64_t n,
                        double *forces, int32_t srt, int32_t rotate) {
  size_t cells = (size_t)p->nx * p->ny;
  double *tmp = (double *)malloc(sizeof(double) * Q * cells);
  double *fb = (double *)malloc(sizeof(double) * 2 * (nbodies > 0 ? nbodies : 1));
  uint8_t *mask = (uint8_t *)malloc(cells);
  ora_body *moved = (ora_body *)malloc(sizeof(ora_body) * (nbodies > 0 ? nbodies : 1));
  if (!tmp || !fb || !mask || !moved) { free(tmp); free(fb); free(mask); free(moved); return -1; }
  double *a = g, *b = tmp;
  for (int64_t s = 0; s < n; s++) {
    const int64_t m = n0 + s;
    if (rotate) ora_rasterize_rot(p->nx, p->ny, shapes, nshapes, bodies, nbodies, m, mask);
    else ora_rasterize_at(p->nx, p->ny, shapes, nshapes, bodies, nbodies, m, mask);
    for (int k = 0; k < nbodies; k++) body_at(&bodies[k], m, &moved[k]);
    if (srt) ora_step_srt(p, mask, moved, nbodies, a, b, fb);
    else ora_step_trt(p, mask, moved, nbodies, a, b, fb);
    if (forces) memcpy(forces + (size_t)s * 2 * nbodies, fb, sizeof(double) * 2 * nbodies);
    double *t = a; a = b; b = t;
  }
  if (a != g) memcpy(g, a, sizeof(double) * Q * cells);
  free(tmp); free(fb); free(mask); free(moved);
  return 0;
}

int ora_run_moving(const ora_params *p, const ora_shape *shapes, int32_t nshapes,
                   const ora_body *bodies, int32_t nbodies, double *g, int64_t n0, int64_t n,
                   double *forces, int32_t srt) {
  return ora_run_moving_mode(p, shapes, nshapes, bodies, nbodies, g, n0, n, forces, srt, 0);
}

/* The bodies of a moving domain at step index n (centres translated). */
void ora_bodies_at(const ora_body *bodies, int32_t nbodies, int64_t n, ora_body *out) {
  for (int k = 0; k < nbodies; k++) body_at(&bodies[k], n, &out[k]);
}

/* ---- fluid-structure coupling (reading M4) ---------------------------------------------
 * The paper prescribes U_O. Coupled motion is an extension: a body with dynamics is a
 * rigid body of mass M on springs k (anchored at its initial centre x0) with dampers c;
 * each free axis obeys M dv/dt = F - k (x - x0) - c v. With eta -> 0 one step maps the
 * penalized interior's fluid velocity u* to 2 U_O - u* (Eq. d-V, Eq. force-density), so
 * the force on the body, F_n = -sum F_VP of step n, carries a component that alternates
 * every step; a body driven by it feeds that component back through U_O and diverges
 * for any mass. The body is therefore driven by the mean of the last two steps' forces,
 * Fm = (F_n + F_{n-1}) / 2 (F_{-1} = 0), which removes the alternating component
 * exactly. After every step, by semi-implicit Euler with dt = 1:
 *   v <- v + (Fm - k (x - x0) - c v) / M,  then  x <- x + v.
 * An axis that is not free keeps its velocity. The mask and U_O of a step use the state
 * before its update; shapes translate with the centre; the angular velocity stays as
 * given. Bodies without dynamics keep their prescribed motion (centre c + V n). */
typedef struct {
  double mass, kx, ky, cx, cy;
  int32_t free_x, free_y, active;
} ora_dynamics;

/* One axis of the update, in the order of the formula above; *Fp holds F_{n-1} and
 * becomes F_n. */
static void fsi_axis(double F, double *Fp, double k, double c, double M, int32_t free_axis,
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

/* n steps from step index n0 with coupled bodies. state [nbodies][6] holds (x, y, vx,
 * vy, Fx_{n0-1}, Fy_{n0-1}) of the bodies with dynamics at index n0 and is advanced in
 * place; track, if not NULL, receives (x, y, vx, vy) each step used, [n][nbodies][4]. */
int ora_run_fsi(const ora_params *p, const ora_shape *shapes, int32_t nshapes,
                const ora_body *bodies, const ora_dynamics *dyn, int32_t nbodies, double *g,
                int64_t n0, int64_t n, double *state, double *forces, double *track) {
  size_t cells = (size_t)p->nx * p->ny;
  double *tmp = (double *)malloc(sizeof(double) * Q * cells);
  double *fb = (double *)malloc(sizeof(double) * 2 * (nbodies > 0 ? nbodies : 1));
  uint8_t *mask = (uint8_t *)malloc(cells);
  ora_body *now = (ora_body *)malloc(sizeof(ora_body) * (nbodies > 0 ? nbodies : 1));
  ora_shape *sh = (ora_shape *)malloc(sizeof(ora_shape) * (nshapes > 0 ? nshapes : 1));
  if (!tmp || !fb || !mask || !now || !sh) {
    free(tmp); free(fb); free(mask); free(now); free(sh);
    return -1;
  }
  double *a = g, *b = tmp;
  for (int64_t s = 0; s < n; s++) {
    const int64_t m = n0 + s;
    /* bodies and shapes at index m */
    for (int k = 0; k < nbodies; k++) {
      if (dyn[k].active) {
        now[k] = bodies[k];
        now[k].cx = state[6 * k];
        now[k].cy = state[6 * k + 1];
        now[k].vx = state[6 * k + 2];
        now[k].vy = state[6 * k + 3];
      } else {
        body_at(&bodies[k], m, &now[k]);
      }
      if (track) {
        double *tr = track + ((size_t)s * nbodies + k) * 4;
        tr[0] = now[k].cx;
        tr[1] = now[k].cy;
        tr[2] = now[k].vx;
        tr[3] = now[k].vy;
      }
    }
    for (int q = 0; q < nshapes; q++) {
      const int k = shapes[q].body - 1;
      if (k >= 0 && k < nbodies && dyn[k].active) {
        sh[q] = shapes[q];
        sh[q].cx = shapes[q].cx + (state[6 * k] - bodies[k].cx);
        sh[q].cy = shapes[q].cy + (state[6 * k + 1] - bodies[k].cy);
      } else {
        shape_at(&shapes[q], bodies, nbodies, m, &sh[q]);
      }
    }
    ora_rasterize(p->nx, p->ny, sh, nshapes, mask);
    ora_step_trt(p, mask, now, nbodies, a, b, fb);
    if (forces) memcpy(forces + (size_t)s * 2 * nbodies, fb, sizeof(double) * 2 * nbodies);
    /* the bodies respond to the force of this step */
    for (int k = 0; k < nbodies; k++) {
      if (!dyn[k].active) continue;
      double *st = &state[6 * k];
      fsi_axis(fb[2 * k], &st[4], dyn[k].kx, dyn[k].cx, dyn[k].mass, dyn[k].free_x, bodies[k].cx, &st[0], &st[2]);
      fsi_axis(fb[2 * k + 1], &st[5], dyn[k].ky, dyn[k].cy, dyn[k].mass, dyn[k].free_y, bodies[k].cy, &st[1], &st[3]);
    }
    double *t = a; a = b; b = t;
  }
  if (a != g) memcpy(g, a, sizeof(double) * Q * cells);
  free(tmp); free(fb); free(mask); free(now); free(sh);
  return 0;
}

/* Step (1): every node starts at f^eq(rho0, u0). */
void ora_init(const ora_params *p, double u0x, double u0y, double *g) {
  double feq[Q];
  ora_equilibrium(p->rho0, u0x, u0y, feq);
  size_t cells = (size_t)p->nx * p->ny;
  for (int a = 0; a < Q; a++)
    for (size_t c = 0; c < cells; c++) g[a * cells + c] = feq[a];
}

/* Macroscopic fields of the current state: rho and u = u* + du of the streamed
 * populations (Eq. rho, Eq. rho*velocity-star, Eq. d-V, Eq. velocity-r). */
void ora_moments(const ora_params *p, const uint8_t *mask, const ora_body *bodies,
                 const double *g, double *rho, double *ux, double *uy) {
  double feq_inlet[Q];
  ora_equilibrium(p->rho0, p->u_in_x, p->u_in_y, feq_inlet);
  for (int j = 0; j < p->ny; j++)
    for (int i = 0; i < p->nx; i++) {
      double f[Q], r, vx, vy, fvx, fvy;
      for (int a = 0; a < Q; a++) f[a] = pull(p, g, feq_inlet, a, i, j);
      node_moments(p, mask, bodies, f, i, j, &r, &vx, &vy, &fvx, &fvy);
      size_t c = (size_t)j * p->nx + i;
      rho[c] = r;
      ux[c] = vx;
      uy[c] = vy;
    }
}

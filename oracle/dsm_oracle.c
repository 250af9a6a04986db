/*
 * dsm_oracle.c -- plain, slow FP64 CPU oracle of the Diffuse Solid Method
 * (Oktasendra, Rennick, Avis, Panter, Kusumaatmaja, "The Diffuse Solid Method
 * for Wetting and Multiphase Fluid Simulations in Complex Geometries").
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product (the CUDA
 * library and its Python binding) never does, and shares no code with it.
 *
 * Every routine walks the whole lattice in the order the paper states the
 * method, one plain loop per stage, in FP64, with no blocking or fusion.
 * OpenMP only splits independent per-node loops; every sum over the lattice is
 * taken serially in node order, so results do not depend on the thread count.
 *
 * Conventions
 *   node index  n = x + nx*(y + ny*z) (nz = 1 for D2Q9);
 *   each face is periodic, a mirror (symmetry plane) or a halfway
 *   bounce-back wall, both of the latter half a node beyond the edge node;
 *   populations are q-major: f[i*N + n];
 *   the stored state is the POST-COLLISION population f*, g*; a step pulls
 *   (streams) first, then forms moments, forces and collides (Sec. II.B,
 *   lattice Boltzmann equations for f and g: f_i(x+c_i, t+1) = f*_i(x, t)).
 *
 * Readings of passages that are garbled or silent (each also listed in the
 * design notes of the repository) are marked "reading:" where they are used.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 19

typedef struct {
  int kind;                 /* 0: D2Q9, 1: D3Q19 */
  int nx, ny, nz;
  double alpha;             /* fluid interface width (Sec. II.A, alpha = 1) */
  double alpha_s;           /* width of the tanh profile given to the solid */
  double kappa1, kappa2, kappa3;
  double rho2, rho3, tau2, tau3, tau_g;
  double bx, by, bz;        /* body force per unit liquid concentration */
  double beta, omega;       /* solid confinement and range penalty (stage 1) */
  int face[6];              /* faces x-, x+, y-, y+, z-, z+: 0 periodic, 1 mirror,
                               2 halfway bounce-back wall (see neighbour, pull) */
} or_params;

typedef struct {
  int d, q;
  int c[QMAX][3];
  double w[QMAX];
  int opp[QMAX];
} lattice;

static const double CS2 = 1.0 / 3.0; /* c_s^2 (Sec. II.B, after Eq. [eqn:feq]) */

/* ------------------------------------------------------------------------ */
/* Lattice tables.                                                           */
/* D2Q9: the velocity and weight tables printed in Sec. II.B.                */
/* D3Q19: the paper gives only D2Q9; reading: the textbook D3Q19 set with    */
/* weights 1/3, 1/18 (axis) and 1/36 (face diagonals).                       */
/* ------------------------------------------------------------------------ */
static void make_lattice(int kind, lattice *L) {
  memset(L, 0, sizeof(*L));
  if (kind == 0) {
    static const int cx[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    static const int cy[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    L->d = 2;
    L->q = 9;
    for (int i = 0; i < 9; i++) {
      L->c[i][0] = cx[i];
      L->c[i][1] = cy[i];
      L->c[i][2] = 0;
      L->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  } else {
    L->d = 3;
    L->q = 19;
    int i = 0;
    L->c[i][0] = L->c[i][1] = L->c[i][2] = 0;
    L->w[i++] = 1.0 / 3.0;
    for (int a = 0; a < 3; a++)
      for (int s = 1; s >= -1; s -= 2) {
        L->c[i][0] = L->c[i][1] = L->c[i][2] = 0;
        L->c[i][a] = s;
        L->w[i++] = 1.0 / 18.0;
      }
    for (int a = 0; a < 3; a++)
      for (int b = a + 1; b < 3; b++)
        for (int sa = 1; sa >= -1; sa -= 2)
          for (int sb = 1; sb >= -1; sb -= 2) {
            L->c[i][0] = L->c[i][1] = L->c[i][2] = 0;
            L->c[i][a] = sa;
            L->c[i][b] = sb;
            L->w[i++] = 1.0 / 36.0;
          }
  }
  for (int i = 0; i < L->q; i++)
    for (int j = 0; j < L->q; j++)
      if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] &&
          L->c[j][2] == -L->c[i][2])
        L->opp[i] = j;
}

int or_lattice(int kind, int *c_out, double *w_out) {
  lattice L;
  make_lattice(kind, &L);
  for (int i = 0; i < L.q; i++) {
    for (int a = 0; a < 3; a++) c_out[3 * i + a] = L.c[i][a];
    w_out[i] = L.w[i];
  }
  return L.q;
}

/* ------------------------------------------------------------------------ */
/* Tensions -> kappa (Sec. II.A, Eq. [frozen:kappa], the inverse of          */
/* Eq. [frozen:interface_tension]).                                          */
/* ------------------------------------------------------------------------ */
int or_kappa_from_tensions(double g12, double g13, double g23, double alpha,
                           double *k) {
  k[0] = 3.0 / alpha * (g12 + g13 - g23);
  k[1] = 3.0 / alpha * (g12 - g13 + g23);
  k[2] = 3.0 / alpha * (-g12 + g13 + g23);
  return (k[1] > 0.0 && k[2] > 0.0) ? 0 : -1;
}

/* Contact angle + (gamma_23, gamma_12) -> kappa: Young's relation
 * (Supp. B, Eq. [eq:CA]) gives gamma_13 = gamma_12 + gamma_23 cos(theta). */
int or_kappa_from_angle(double theta_deg, double g23, double g12, double alpha,
                        double *k) {
  const double pi = 3.14159265358979323846;
  double g13 = g12 + g23 * cos(theta_deg * pi / 180.0);
  return or_kappa_from_tensions(g12, g13, g23, alpha, k);
}

/* ------------------------------------------------------------------------ */
/* Solid profile from a signed distance (positive inside the solid region S):*/
/* the planar tanh profile of Sec. II.A, Eq. [frozen:interface_profile].     */
/* ------------------------------------------------------------------------ */
void or_solid_profile(long n, const double *sd, double alpha_s, double *c1) {
  for (long k = 0; k < n; k++) c1[k] = 0.5 + 0.5 * tanh(sd[k] / (2.0 * alpha_s));
}

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */
static long nnodes(const or_params *p) { return (long)p->nx * p->ny * p->nz; }

/* Neighbour index along one axis for the stencils (G, L, the pair sums of the
 * energy): periodic, or, beyond a mirror or wall face, the image of the node
 * across the plane half a node beyond the edge (-1 -> 0, n -> n - 1).  The
 * energy minimisations of Sec. III use symmetry boundaries on some axes.
 * reading: a bounce-back wall sees the same image, i.e. zero normal gradient
 * of every concentration (a neutral wall; the method wets through the diffuse
 * solid, not through the domain faces).                                     */
static long axis_step(long v, int dv, long n, int lo, int hi) {
  long w = v + dv;
  if (w < 0 && lo) return -w - 1;
  if (w >= n && hi) return 2 * n - w - 1;
  return ((w % n) + n) % n;
}

static long neighbour(const or_params *p, long n, int dx, int dy, int dz) {
  long x = n % p->nx, y = (n / p->nx) % p->ny, z = n / ((long)p->nx * p->ny);
  x = axis_step(x, dx, p->nx, p->face[0], p->face[1]);
  y = axis_step(y, dy, p->ny, p->face[2], p->face[3]);
  z = axis_step(z, dz, p->nz, p->face[4], p->face[5]);
  return x + p->nx * (y + (long)p->ny * z);
}

/* Streaming source of the population f_j (or g_j) at node n: the node and the
 * direction whose post-collision value moves into direction j at n.  *cross
 * tells which faces the link x - c_j -> x crosses: 0 none, 1 mirrors only,
 * 2 a wall.
 *   inside the lattice: x - c_j, direction j (f_j(x) = f*_j(x - c_j));
 *   across a wall face: halfway bounce-back, n itself, direction opp(j);
 *   across mirror faces only: specular reflection, the image node of x - c_j
 *   and the direction j with its components normal to the crossed faces
 *   reversed (the lattice is half of its reflected periodic double, so the
 *   image node stands for the node beyond the plane).                       */
static long pull(const or_params *p, const lattice *L, long n, int j, int *k, int *cross) {
  long v[3] = {n % p->nx, (n / p->nx) % p->ny, n / ((long)p->nx * p->ny)};
  long e[3] = {p->nx, p->ny, p->nz};
  int c[3] = {L->c[j][0], L->c[j][1], L->c[j][2]};
  int crossed = 0, wall = 0;
  for (int a = 0; a < 3; a++) {
    int t = 0;
    if (v[a] - c[a] < 0) t = p->face[2 * a];
    else if (v[a] - c[a] >= e[a]) t = p->face[2 * a + 1];
    if (t) {
      crossed = 1;
      c[a] = -c[a];
      if (t == 2) wall = 1;
    }
  }
  *k = j;
  *cross = wall ? 2 : crossed;
  if (!crossed) return neighbour(p, n, -L->c[j][0], -L->c[j][1], -L->c[j][2]);
  if (wall) {
    *k = L->opp[j];
    return n;
  }
  for (int i = 0; i < L->q; i++)
    if (L->c[i][0] == c[0] && L->c[i][1] == c[1] && L->c[i][2] == c[2]) *k = i;
  return neighbour(p, n, -L->c[j][0], -L->c[j][1], -L->c[j][2]);
}

/* Isotropic central differences (Sec. II.B says only "second order isotropic
 * central difference"; reading: the lattice-weighted forms)
 *   G[phi](x) = (1/c_s^2) sum_i w_i c_i phi(x + c_i)
 *   L[phi](x) = (2/c_s^2) sum_{i != 0} w_i (phi(x + c_i) - phi(x))          */
void or_gradient(const or_params *p, const double *phi, double *out) {
  lattice L;
  make_lattice(p->kind, &L);
  long N = nnodes(p);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double g[3] = {0, 0, 0};
    for (int i = 1; i < L.q; i++) {
      double v = phi[neighbour(p, n, L.c[i][0], L.c[i][1], L.c[i][2])];
      for (int a = 0; a < 3; a++) g[a] += L.w[i] * L.c[i][a] * v;
    }
    for (int a = 0; a < 3; a++) out[a * N + n] = g[a] / CS2;
  }
}

void or_laplacian(const or_params *p, const double *phi, double *out) {
  lattice L;
  make_lattice(p->kind, &L);
  long N = nnodes(p);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double s = 0.0;
    for (int i = 1; i < L.q; i++)
      s += L.w[i] * (phi[neighbour(p, n, L.c[i][0], L.c[i][1], L.c[i][2])] - phi[n]);
    out[n] = 2.0 * s / CS2;
  }
}

/* Derivative of the double well: b(c) = d/dc [c^2 (1-c)^2 / 2]
 * = c (1 - c)(1 - 2c), written in Sec. II.B as c (1 - 3c + 2c^2). */
static double bwell(double c) { return c * (1.0 - c) * (1.0 - 2.0 * c); }

/* Chemical potential of the frozen-solid free energy (Sec. II.B,
 * Eq. [eqn:fefrozen]) with respect to C = C2 at fixed C1:
 *   mu = k2 b(C) + k3 b(C1 + C) - a^2 k2 L[C] - a^2 k3 L[C1 + C].
 * reading: the printed kappa_3 bulk term and the printed Laplacian terms do not
 * equal the derivative of Eq. [eqn:fefrozen]; the derivative is used.       */
void or_mu_fluid(const or_params *p, const double *c1, const double *c,
                 double *mu) {
  long N = nnodes(p);
  double *s = malloc(sizeof(double) * N), *lc = malloc(sizeof(double) * N),
         *ls = malloc(sizeof(double) * N);
  for (long n = 0; n < N; n++) s[n] = c1[n] + c[n];
  or_laplacian(p, c, lc);
  or_laplacian(p, s, ls);
  double a2 = p->alpha * p->alpha;
  for (long n = 0; n < N; n++)
    mu[n] = p->kappa2 * bwell(c[n]) + p->kappa3 * bwell(s[n]) -
            a2 * p->kappa2 * lc[n] - a2 * p->kappa3 * ls[n];
  free(s);
  free(lc);
  free(ls);
}

/* Confinement indicator of Eq. [frozen:poly-quadratic_lbm] (Sec. II.B).
 * reading: the printed case labels are swapped (as printed every node would be
 * pulled to C1 = 1/2); the penalty acts where the solid leaks out of S or the
 * fluid leaks into S:  chi = (x in S and C1 < 1/2) or (x not in S and C1 > 1/2). */
static int chi(unsigned char in_s, double c1) {
  return (in_s && c1 < 0.5) || (!in_s && c1 > 0.5);
}

/* Chemical potential of the solid-relaxation free energy (Sec. II.B,
 * Eq. [Free Energy1] and the chemical potential that follows it):
 *   mu1 = (k1+k3) b(C1) + 2 beta (C1 - 1/2) chi - a^2 (k1+k3) L[C1]
 *         + 2 Omega C1 H(-C1) - 2 Omega (1 - C1) H(C1 - 1).
 * reading: the printed Heaviside arguments H(C1), H(1-C1) would penalise the
 * valid range; the penalty acts outside [0, 1].                              */
void or_mu_solid(const or_params *p, const unsigned char *S, const double *c1,
                 double *mu) {
  long N = nnodes(p);
  double *l1 = malloc(sizeof(double) * N);
  or_laplacian(p, c1, l1);
  double k13 = p->kappa1 + p->kappa3, a2 = p->alpha * p->alpha;
  for (long n = 0; n < N; n++) {
    double c = c1[n];
    double m = k13 * bwell(c) - a2 * k13 * l1[n];
    if (chi(S[n], c)) m += 2.0 * p->beta * (c - 0.5);
    if (c < 0.0) m += 2.0 * p->omega * c;
    if (c > 1.0) m -= 2.0 * p->omega * (1.0 - c);
    mu[n] = m;
  }
  free(l1);
}

/* ------------------------------------------------------------------------ */
/* Equilibria and forcing for one node (Sec. II.B).                          */
/*   s_i(u) = c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u.u/(2 c_s^2)              */
/*     reading: the printed "+ u.u/(2c_s^2)" breaks sum_i f_eq = P/c_s^2; the  */
/*     minus sign is the one that conserves the moments.                     */
/*   f_eq_i = w_i (pt + rho s_i),  pt = P/c_s^2        (Eq. [eqn:feq])        */
/*   F_i = (1 - 1/(2 tau)) w_i [((c_i - u).Grho) s_i + c_i.F/c_s^2]           */
/*                                                     (Eq. [eqn:hydroforce]) */
/*   g_eq_i = w_i mu + w_i C s_i (i != 0),                                    */
/*   g_eq_0 = C - (1 - w_0) mu + w_0 C s_0                                    */
/*     reading: the printed "+ (1 - w_0) mu + C(1 + ...)" for the rest        */
/*     population breaks sum_i g_eq = C; the form above conserves C.          */
/* ------------------------------------------------------------------------ */
static double s_of(const lattice *L, int i, const double u[3]) {
  double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2);
}

static void equilibria(const lattice *L, double pt, double rho, const double u[3],
                       double C, double mu, double tau, const double grho[3],
                       const double F[3], double *feq, double *geq, double *Fi) {
  for (int i = 0; i < L->q; i++) {
    double s = s_of(L, i, u);
    if (feq) feq[i] = L->w[i] * (pt + rho * s);
    if (geq)
      geq[i] = (i == 0) ? C - (1.0 - L->w[0]) * mu + L->w[0] * C * s
                        : L->w[i] * mu + L->w[i] * C * s;
    if (Fi) {
      double cmu_g = 0.0, cF = 0.0;
      for (int a = 0; a < 3; a++) {
        cmu_g += (L->c[i][a] - u[a]) * grho[a];
        cF += L->c[i][a] * F[a];
      }
      Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * L->w[i] * (cmu_g * s + cF / CS2);
    }
  }
}

/* Exposed for the moment-identity pins. */
void or_equilibria(int kind, double pt, double rho, const double *u, double C,
                   double mu, double tau, const double *grho, const double *F,
                   double *feq, double *geq, double *Fi) {
  lattice L;
  make_lattice(kind, &L);
  equilibria(&L, pt, rho, u, C, mu, tau, grho, F, feq, geq, Fi);
}

/* ------------------------------------------------------------------------ */
/* Interpolated bounce-back (Sec. II.B, Eqs. [eqn:tanh] and the distance     */
/* D = |x / (n.d)| that follows; the paper cites Bouzidi et al. 2001).       */
/* The fluid node's signed distance to the C1 = 1/2 surface is read off the  */
/* tanh profile, x_s = 2 alpha_s artanh(2 C1 - 1) <= 0; the link fraction is  */
/* q = |x_s / (n.d)| / |c_i| with n = G[C1]/|G[C1]|, d = c_i/|c_i|.          */
/* reading: C1 is clamped to [1e-9, 1/2]; a degenerate normal, a link that    */
/* does not point into the solid, or q outside [0, 1] falls back to q = 1/2.  */
/* ------------------------------------------------------------------------ */
static double link_q(const lattice *L, double alpha_s, double c1x,
                     const double gc1[3], int i) {
  double c = c1x < 1e-9 ? 1e-9 : (c1x > 0.5 ? 0.5 : c1x);
  double xs = 2.0 * alpha_s * atanh(2.0 * c - 1.0);
  double gn = sqrt(gc1[0] * gc1[0] + gc1[1] * gc1[1] + gc1[2] * gc1[2]);
  if (gn < 1e-12) return 0.5;
  double cl = sqrt((double)(L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] +
                            L->c[i][2] * L->c[i][2]));
  if (cl == 0.0) return 0.5; /* the rest population has no link */
  double nd = (gc1[0] * L->c[i][0] + gc1[1] * L->c[i][1] + gc1[2] * L->c[i][2]) /
              (gn * cl);
  if (nd <= 1e-6) return 0.5;
  double q = fabs(xs / nd) / cl;
  if (q < 0.0 || q > 1.0) return 0.5;
  return q;
}

double or_link_q(int kind, double alpha_s, double c1x, const double *gc1, int i) {
  lattice L;
  make_lattice(kind, &L);
  return link_q(&L, alpha_s, c1x, gc1, i);
}

/* Solid flag for the hydrodynamic populations.
 * reading: a node is solid when C1 >= 1/2 (Sec. II.A: C = 0.5 marks the
 * boundary between two phases).                                             */
static int is_solid(double c1) { return c1 >= 0.5; }

/* ------------------------------------------------------------------------ */
/* One lattice Boltzmann step.  stage = 2: fluids (C = C2) on the frozen      */
/* diffuse solid.  stage = 1: solid relaxation (C = C1), Sec. II.B.           */
/* ------------------------------------------------------------------------ */
typedef struct {
  double *fs, *gs;              /* streamed (pre-collision) populations */
  double *C, *rho, *tau, *mu;   /* concentration, density, relaxation, mu */
  double *F, *grho, *gc;        /* 3 x N each: force, G[rho], G[C] */
  double *u, *pt;               /* 3 x N, N */
} work;

static void work_alloc(work *w, long N, int q) {
  w->fs = malloc(sizeof(double) * q * N);
  w->gs = malloc(sizeof(double) * q * N);
  w->C = malloc(sizeof(double) * N);
  w->rho = malloc(sizeof(double) * N);
  w->tau = malloc(sizeof(double) * N);
  w->mu = malloc(sizeof(double) * N);
  w->F = malloc(sizeof(double) * 3 * N);
  w->grho = malloc(sizeof(double) * 3 * N);
  w->gc = malloc(sizeof(double) * 3 * N);
  w->u = malloc(sizeof(double) * 3 * N);
  w->pt = malloc(sizeof(double) * N);
}

static void work_free(work *w) {
  free(w->fs); free(w->gs); free(w->C); free(w->rho); free(w->tau);
  free(w->mu); free(w->F); free(w->grho); free(w->gc); free(w->u); free(w->pt);
}

/* Streaming (pull).  g streams everywhere (reading: the order parameter gets
 * no rule at the diffuse solid, so sum_x C is conserved exactly).  f at a
 * fluid node pulls from fluid neighbours; a link whose upstream node is solid
 * takes the linear interpolated bounce-back value.  Solid nodes carry
 * f_i = w_i.  Links across a mirror or wall face follow pull() for f and g
 * alike (a wall bounces g back too: no flux through it).  reading: a wall
 * face comes before anything beyond it; across a mirror the image node is the
 * upstream node, solid or not, and the interpolation's second node x + c_j is
 * taken by pull() too (a second node beyond a wall counts as missing).      */
static void stream(const or_params *p, const lattice *L, int stage,
                   const double *c1, const double *gc1, const double *f,
                   const double *g, work *w) {
  long N = nnodes(p);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    for (int j = 0; j < L->q; j++) {
      int k, cr;
      long y = pull(p, L, n, j, &k, &cr);
      w->gs[j * N + n] = g[k * N + y];
    }
    int solid_n = (stage == 2) && is_solid(c1[n]);
    if (solid_n) {
      for (int j = 0; j < L->q; j++) w->fs[j * N + n] = L->w[j];
      continue;
    }
    for (int j = 0; j < L->q; j++) {
      int k, cr;
      long y = pull(p, L, n, j, &k, &cr);
      if (cr == 2 || stage == 1 || !is_solid(c1[y])) {
        w->fs[j * N + n] = f[k * N + y];
        continue;
      }
      int i = L->opp[j]; /* link from n toward the wall node y = n + c_i */
      double gl[3] = {gc1[n], gc1[N + n], gc1[2 * N + n]};
      double q = link_q(L, p->alpha_s, c1[n], gl, i);
      int kz, crz;
      long z = pull(p, L, n, i, &kz, &crz); /* f_i one node away from the wall */
      if (q < 0.5 && crz != 2 && !is_solid(c1[z]))
        w->fs[j * N + n] = 2.0 * q * f[i * N + n] + (1.0 - 2.0 * q) * f[kz * N + z];
      else if (q < 0.5) /* reading: no second fluid node -> halfway rule */
        w->fs[j * N + n] = f[i * N + n];
      else
        w->fs[j * N + n] = (1.0 / (2.0 * q)) * f[i * N + n] +
                           (1.0 - 1.0 / (2.0 * q)) * f[j * N + n];
    }
  }
}

/* Moments, chemical potential and forces (Sec. II.B).
 *   C = sum_i g_i                                   (Eq. C = sum g)
 *   rho = rho3 + (rho2 - rho3) C2/(C2 + C3)          (density map)
 *     reading: C2 + C3 = 1 - C1 vanishes in the solid; the ratio is clamped
 *     to [0, 1] and taken as 0 where 1 - C1 <= 1e-6.
 *   tau = tau3 + (tau2 - tau3) H(C2 - C3), H(0) = 0  (relaxation map)
 *   F = mu G[C] + C b   (capillary force plus the body force on the liquid).
 *     reading: the text states the capillary force as -C grad(mu) while the
 *     velocity moment it prints uses mu grad(C); the two differ by the
 *     gradient grad(C mu), which only shifts the pressure.  The potential form
 *     mu G[C] is taken, as one total force in both the forcing term and the
 *     velocity moment: with BGK at tau = 1 the k = pi longitudinal momentum
 *     mode is undamped, and the discrete -C G[mu] feeds it at a liquid/solid
 *     interface until the step diverges, while mu G[C] does not.
 *   rho u = sum_i c_i f_i + F/2,  pt = sum_i f_i + u.G[rho]/2
 *     reading: pt = P/c_s^2 so that sum_i f_eq = pt.  Solid nodes: u = 0.
 * Stage 1 uses rho = 1, tau = tau_g = 1 and treats every node as fluid.     */
static void macroscopic(const or_params *p, const lattice *L, int stage,
                        const unsigned char *S, const double *c1, work *w) {
  long N = nnodes(p);
  for (long n = 0; n < N; n++) {
    double s = 0.0;
    for (int i = 0; i < L->q; i++) s += w->gs[i * N + n];
    w->C[n] = s;
  }
  if (stage == 2) {
    for (long n = 0; n < N; n++) {
      double C = w->C[n], C3 = 1.0 - c1[n] - C, den = 1.0 - c1[n];
      double phi = 0.0;
      if (den > 1e-6) {
        phi = C / den;
        phi = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
      }
      w->rho[n] = p->rho3 + (p->rho2 - p->rho3) * phi;
      w->tau[n] = (C - C3 > 0.0) ? p->tau2 : p->tau3;
    }
    or_mu_fluid(p, c1, w->C, w->mu);
  } else {
    for (long n = 0; n < N; n++) {
      w->rho[n] = 1.0;
      w->tau[n] = 1.0;
    }
    or_mu_solid(p, S, w->C, w->mu);
  }
  or_gradient(p, w->C, w->gc);
  or_gradient(p, w->rho, w->grho);
  double b[3] = {p->bx, p->by, p->bz};
  for (long n = 0; n < N; n++)
    for (int a = 0; a < 3; a++)
      w->F[a * N + n] = w->mu[n] * w->gc[a * N + n] + (stage == 2 ? w->C[n] * b[a] : 0.0);
  for (long n = 0; n < N; n++) {
    int solid_n = (stage == 2) && is_solid(c1[n]);
    double m0 = 0.0, m1[3] = {0, 0, 0};
    for (int i = 0; i < L->q; i++) {
      double fv = w->fs[i * N + n];
      m0 += fv;
      for (int a = 0; a < 3; a++) m1[a] += L->c[i][a] * fv;
    }
    double u[3] = {0, 0, 0};
    if (!solid_n)
      for (int a = 0; a < 3; a++) u[a] = (m1[a] + 0.5 * w->F[a * N + n]) / w->rho[n];
    for (int a = 0; a < 3; a++) w->u[a * N + n] = u[a];
    double ug = u[0] * w->grho[n] + u[1] * w->grho[N + n] + u[2] * w->grho[2 * N + n];
    w->pt[n] = solid_n ? 1.0 : m0 + 0.5 * ug;
  }
}

/* BGK collision (Sec. II.B): f* = f - (f - f_eq)/tau + F_i at fluid nodes,
 * f* = w_i at solid nodes; g* = g - (g - g_eq)/tau_g at every node (u = 0 in
 * the solid).  tau_f of Eq. [eqn:hydroforce] is read as the local tau.       */
static void collide(const or_params *p, const lattice *L, int stage,
                    const double *c1, const work *w, double *f, double *g) {
  long N = nnodes(p);
  double taug = (stage == 2) ? p->tau_g : 1.0;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double u[3] = {w->u[n], w->u[N + n], w->u[2 * N + n]};
    double gr[3] = {w->grho[n], w->grho[N + n], w->grho[2 * N + n]};
    double Fv[3] = {w->F[n], w->F[N + n], w->F[2 * N + n]};
    double feq[QMAX], geq[QMAX], Fi[QMAX];
    equilibria(L, w->pt[n], w->rho[n], u, w->C[n], w->mu[n], w->tau[n], gr, Fv,
               feq, geq, Fi);
    int solid_n = (stage == 2) && is_solid(c1[n]);
    for (int i = 0; i < L->q; i++) {
      double fv = w->fs[i * N + n];
      f[i * N + n] = solid_n ? L->w[i] : fv - (fv - feq[i]) / w->tau[n] + Fi[i];
      double gv = w->gs[i * N + n];
      g[i * N + n] = gv - (gv - geq[i]) / taug;
    }
  }
}

static void gradient_c1(const or_params *p, const double *c1, double *gc1) {
  or_gradient(p, c1, gc1);
}

/* Run nsteps steps in place on the post-collision state (f, g).
 * stage 2: c1 is the frozen solid; S unused.  stage 1: S is the solid region
 * (bytes, 1 inside), g carries C1, c1 unused.
 * fields (optional, 8 x N): C, mu, ux, uy, uz, pt, rho, tau of the last step. */
int or_lb_run(const or_params *p, int stage, const unsigned char *S,
              const double *c1, double *f, double *g, long nsteps, double *fields) {
  lattice L;
  make_lattice(p->kind, &L);
  long N = nnodes(p);
  work w;
  work_alloc(&w, N, L.q);
  double *gc1 = malloc(sizeof(double) * 3 * N);
  if (stage == 2) gradient_c1(p, c1, gc1);
  else memset(gc1, 0, sizeof(double) * 3 * N);
  for (long t = 0; t < nsteps; t++) {
    stream(p, &L, stage, c1, gc1, f, g, &w);
    macroscopic(p, &L, stage, S, c1, &w);
    collide(p, &L, stage, c1, &w, f, g);
  }
  if (fields && nsteps > 0) {
    memcpy(fields + 0 * N, w.C, sizeof(double) * N);
    memcpy(fields + 1 * N, w.mu, sizeof(double) * N);
    memcpy(fields + 2 * N, w.u, sizeof(double) * 3 * N);
    memcpy(fields + 5 * N, w.pt, sizeof(double) * N);
    memcpy(fields + 6 * N, w.rho, sizeof(double) * N);
    memcpy(fields + 7 * N, w.tau, sizeof(double) * N);
  }
  free(gc1);
  work_free(&w);
  return 0;
}

/* Macroscopic fields at the current time level: the streaming and moment
 * stages of the next step, without its collision (8 x N, as above). */
int or_lb_fields(const or_params *p, int stage, const unsigned char *S,
                 const double *c1, const double *f, const double *g,
                 double *fields) {
  lattice L;
  make_lattice(p->kind, &L);
  long N = nnodes(p);
  work w;
  work_alloc(&w, N, L.q);
  double *gc1 = malloc(sizeof(double) * 3 * N);
  if (stage == 2) gradient_c1(p, c1, gc1);
  else memset(gc1, 0, sizeof(double) * 3 * N);
  stream(p, &L, stage, c1, gc1, f, g, &w);
  macroscopic(p, &L, stage, S, c1, &w);
  memcpy(fields + 0 * N, w.C, sizeof(double) * N);
  memcpy(fields + 1 * N, w.mu, sizeof(double) * N);
  memcpy(fields + 2 * N, w.u, sizeof(double) * 3 * N);
  memcpy(fields + 5 * N, w.pt, sizeof(double) * N);
  memcpy(fields + 6 * N, w.rho, sizeof(double) * N);
  memcpy(fields + 7 * N, w.tau, sizeof(double) * N);
  free(gc1);
  work_free(&w);
  return 0;
}

/* Initial state (the paper leaves it unstated; reading): quiescent, f_i = w_i
 * (pt = 1, u = 0) and g_i = g_eq_i(C, mu(C), u = 0), stored as the
 * post-collision state.  stage 2: C = cfield (= C2) over the frozen c1;
 * stage 1: C = cfield (= C1) with the solid region S.                       */
int or_lb_init(const or_params *p, int stage, const unsigned char *S,
               const double *c1, const double *cfield, double *f, double *g) {
  lattice L;
  make_lattice(p->kind, &L);
  long N = nnodes(p);
  double *mu = malloc(sizeof(double) * N);
  if (stage == 2) or_mu_fluid(p, c1, cfield, mu);
  else or_mu_solid(p, S, cfield, mu);
  double u[3] = {0, 0, 0}, z[3] = {0, 0, 0};
  for (long n = 0; n < N; n++) {
    double geq[QMAX];
    equilibria(&L, 1.0, 1.0, u, cfield[n], mu[n], 1.0, z, z, NULL, geq, NULL);
    for (int i = 0; i < L.q; i++) {
      f[i * N + n] = L.w[i];
      g[i * N + n] = geq[i];
    }
  }
  free(mu);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Discrete free energy and its exact gradient (Sec. II.A, Eqs.             */
/* [frozen:total_energy], [frozen:bulk_energy], [frozen:interface_energy],    */
/* [frozen:pressure_const] / [frozen:volume_const], [frozen:poly-quadratic], */
/* and Sec. III.B, Eq. [frozen:gravitational energy]).                       */
/* reading: |grad C_n|^2 is discretised as the lattice-weighted pair sum      */
/*   (1/c_s^2) sum_i w_i (C_n(x + c_i) - C_n(x))^2,                           */
/* whose exact derivative is -kappa'_n L[C_n] with the Laplacian above, so    */
/* the energy gradient equals the lattice Boltzmann chemical potential.      */
/*   E = sum_x [ sum_n k_n/2 C_n^2 (1-C_n)^2                                  */
/*             + sum_n a^2 k_n/(2 c_s^2) sum_i w_i (C_n(x+c_i) - C_n(x))^2     */
/*             + beta (C1 - 1/2)^2 chi   (active = 1 only)                    */
/*             + fg C2 h ]                (h = index along the last axis)     */
/*       + constraint: -dP V  (kcs == 0)  or  kcs/2 (V - V0)^2,  V = sum C2.  */
/* C3 = 1 - C1 - C2.  active = 2: gradient w.r.t. C2 (C1 fixed);              */
/* active = 1: gradient w.r.t. C1 (C2 fixed), with the confinement term.      */
/* ------------------------------------------------------------------------ */
double or_energy_grad(const or_params *p, const double *c1, const double *c2,
                      const unsigned char *S, int active, double dP, double kcs,
                      double V0, double fg, double *grad, double *terms) {
  lattice L;
  make_lattice(p->kind, &L);
  long N = nnodes(p);
  double k[3] = {p->kappa1, p->kappa2, p->kappa3};
  double a2 = p->alpha * p->alpha;
  double *cn[3];
  for (int m = 0; m < 3; m++) cn[m] = malloc(sizeof(double) * N);
  for (long n = 0; n < N; n++) {
    cn[0][n] = c1[n];
    cn[1][n] = c2[n];
    cn[2][n] = 1.0 - c1[n] - c2[n];
  }
  double *dens_bulk = malloc(sizeof(double) * N), *dens_grad = malloc(sizeof(double) * N),
         *dens_cf = malloc(sizeof(double) * N), *dens_g = malloc(sizeof(double) * N);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double eb = 0.0, eg = 0.0;
    for (int m = 0; m < 3; m++) {
      double c = cn[m][n];
      eb += 0.5 * k[m] * c * c * (1.0 - c) * (1.0 - c);
      double pair = 0.0;
      for (int i = 1; i < L.q; i++) {
        double d = cn[m][neighbour(p, n, L.c[i][0], L.c[i][1], L.c[i][2])] - c;
        pair += L.w[i] * d * d;
      }
      eg += a2 * k[m] / (2.0 * CS2) * pair;
    }
    dens_bulk[n] = eb;
    dens_grad[n] = eg;
    dens_cf[n] = (active == 1 && chi(S[n], c1[n])) ? p->beta * (c1[n] - 0.5) * (c1[n] - 0.5) : 0.0;
    long h = (p->kind == 0) ? (n / p->nx) % p->ny : n / ((long)p->nx * p->ny);
    dens_g[n] = fg * c2[n] * (double)h;
  }
  double Eb = 0.0, Eg = 0.0, Ecf = 0.0, Egrav = 0.0, V = 0.0;
  for (long n = 0; n < N; n++) {
    Eb += dens_bulk[n];
    Eg += dens_grad[n];
    Ecf += dens_cf[n];
    Egrav += dens_g[n];
    V += c2[n];
  }
  double Ecs = (kcs == 0.0) ? -dP * V : 0.5 * kcs * (V - V0) * (V - V0);
  double dEcs = (kcs == 0.0) ? -dP : kcs * (V - V0);
  if (grad) {
    double *lap[3];
    for (int m = 0; m < 3; m++) {
      lap[m] = malloc(sizeof(double) * N);
      or_laplacian(p, cn[m], lap[m]);
    }
    for (long n = 0; n < N; n++) {
      double d1 = k[0] * bwell(cn[0][n]) - a2 * k[0] * lap[0][n];
      double d2 = k[1] * bwell(cn[1][n]) - a2 * k[1] * lap[1][n];
      double d3 = k[2] * bwell(cn[2][n]) - a2 * k[2] * lap[2][n];
      if (active == 2) {
        long h = (p->kind == 0) ? (n / p->nx) % p->ny : n / ((long)p->nx * p->ny);
        grad[n] = d2 - d3 + dEcs + fg * (double)h;
      } else {
        double g1 = d1 - d3;
        if (chi(S[n], c1[n])) g1 += 2.0 * p->beta * (c1[n] - 0.5);
        grad[n] = g1;
      }
    }
    for (int m = 0; m < 3; m++) free(lap[m]);
  }
  if (terms) {
    terms[0] = Eb;
    terms[1] = Eg;
    terms[2] = Ecf;
    terms[3] = Ecs;
    terms[4] = Egrav;
    terms[5] = V;
  }
  for (int m = 0; m < 3; m++) free(cn[m]);
  free(dens_bulk); free(dens_grad); free(dens_cf); free(dens_g);
  return Eb + Eg + Ecf + Ecs + Egrav;
}

/* Observables of the current state (stage 2): out[0] = sum C2, out[1] =
 * sum C1, out[2] = kinetic energy sum rho u^2 / 2 over fluid nodes, out[3] =
 * max |u|, out[4] = 1 if any population is not finite, out[5] = free energy
 * (bulk + gradient terms of the discrete energy at (C1, C2)). */
int or_observables(const or_params *p, const double *c1, const double *f,
                   const double *g, double *out) {
  lattice L;
  make_lattice(p->kind, &L);
  long N = nnodes(p);
  double *fields = malloc(sizeof(double) * 8 * N);
  or_lb_fields(p, 2, NULL, c1, f, g, fields);
  double mc2 = 0.0, mc1 = 0.0, ke = 0.0, umax = 0.0;
  int bad = 0;
  for (long n = 0; n < N; n++) {
    mc2 += fields[n];
    mc1 += c1[n];
    double ux = fields[2 * N + n], uy = fields[3 * N + n], uz = fields[4 * N + n];
    double uu = ux * ux + uy * uy + uz * uz;
    ke += 0.5 * fields[6 * N + n] * uu;
    if (sqrt(uu) > umax) umax = sqrt(uu);
  }
  for (long k = 0; k < (long)L.q * N; k++)
    if (!isfinite(f[k]) || !isfinite(g[k])) bad = 1;
  double terms[6];
  or_energy_grad(p, c1, fields, NULL, 2, 0.0, 0.0, 0.0, 0.0, NULL, terms);
  out[0] = mc2;
  out[1] = mc1;
  out[2] = ke;
  out[3] = umax;
  out[4] = bad;
  out[5] = terms[0] + terms[1];
  free(fields);
  return 0;
}

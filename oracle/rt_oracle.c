/*
 * FP64 CPU oracle for one radiation-transfer step of Jiang, Stone & Davis
 * (2014), "An Algorithm for Radiation MHD Based on Solving the
 * Time-dependent Transfer Equation" (arXiv:1403.6126).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library may include, link or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code with the CUDA path.
 *
 * Plain, slow, serial-per-cell double precision.  Each function follows one
 * part of the paper in the paper's order:
 *   Step 1 (sec. 4.1)   dt from the cell size and C           -> orc_cfl_dt
 *   Step 2 (sec. 4.2)   transport Delta F_l (eqs. decomposeI,
 *                       transporttwoterms, alpha, van Leer)     -> transport_all
 *   Step 3 (sec. 4.5)   half-step velocity estimate v~         -> vtilde
 *   Step 4 (sec. 4.3)   implicit absorption + T^4 coupling
 *                       (eq. absorptionmatrix)                  -> absorption_*
 *   Step 5 (sec. 4.4)   implicit scattering (matrix M_s)        -> scattering_*
 *   quadrature (sec. 3) E_r, F_r, P_r and the gas sources
 *                       (eqs. momentumchange, kinetichange)     -> orc_moments, orc_step
 * Two independent solver forms are kept for Steps 4 and 5: a dense
 * brute-force form (Gaussian elimination on the full (N+1) or N system) and
 * the O(N) reduced form that eliminates the angles analytically.
 *
 * Readings where the paper is silent or inconsistent (all listed in the
 * design notes): weights sum to 1 so J = sum W I is the mean intensity and
 * E_r = 4 pi J; the van Leer face states use the time-centred factor
 * (1 - nu)/2; alpha scales only the upwind (dissipative) half of the face
 * flux, face = (1+a)/2 up + (1-a)/2 down; the IV term is reconstructed per
 * angle and upwinded by the sign of the face-averaged gas velocity; all axes
 * are differenced from I^n (unsplit); Delta F goes to Step 5 when
 * sigma_s > sigma_a, else to Step 4; Delta E_T uses rho R/(gamma-1);
 * Delta(rho v) carries the 4 pi of F_r = 4 pi sum W n I and counts only the
 * change made by the implicit steps (transport is not a gas source);
 * Delta E_K is formed from the total momentum change of the step.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

enum { ORC_PERIODIC = 0, ORC_VACUUM = 1, ORC_COPY = 2, ORC_INFLOW = 3 };

typedef struct {
  int dim;                 /* 1, 2 or 3 active axes (x, then y, then z)        */
  int n[3];                /* cells per axis, 1 on inactive axes               */
  double dx[3];            /* cell size per axis                               */
  int bc[3][2];            /* boundary kind per axis and side (lo, hi)         */
  const double *inflow;    /* [3][2][M] incoming intensity for ORC_INFLOW      */
  int M;                   /* number of angles                                 */
  const double *mu;        /* [M][3] direction cosines                         */
  const double *w;         /* [M] weights, sum 1                               */
  double C, P, gamma, R;   /* Crat, Prat, adiabatic index, R_ideal            */
  int hold_T;              /* 1: gas temperature held fixed                    */
  int estimate_v;          /* 1: Step 3 velocity estimate on                   */
  int dense;               /* 1: brute-force dense solvers                     */
  int alpha_one;           /* 1: alpha = 1 on every face (the plain Stone &
                              Mihalas upwinding; a control for the tests)     */
} orc_problem;

static long ncells(const orc_problem *p) { return (long)p->n[0] * p->n[1] * p->n[2]; }
static long cidx(const orc_problem *p, const int c[3]) {
  return c[0] + (long)p->n[0] * (c[1] + (long)p->n[1] * c[2]);
}

void orc_set_threads(int k) {
#ifdef _OPENMP
  omp_set_num_threads(k > 0 ? k : 1);
#else
  (void)k;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Step 1 (sec. 4.1): dt = CFL * min cell size / C over the active axes. */
double orc_cfl_dt(const orc_problem *p, double cfl) {
  double h = p->dx[0];
  for (int d = 1; d < p->dim; ++d)
    if (p->dx[d] < h) h = p->dx[d];
  return cfl * h / p->C;
}

/* Angular quadrature (sec. 3): E_r = 4 pi sum W I, F_r = 4 pi sum W n I,
 * P_r = 4 pi sum W n n I.  P is stored xx, yy, zz, xy, xz, yz. */
void orc_moments(const orc_problem *p, const double *I, double *E, double *F, double *P) {
  long N = ncells(p);
  for (long c = 0; c < N; ++c) {
    double e = 0, f[3] = {0, 0, 0}, q[6] = {0, 0, 0, 0, 0, 0};
    for (int m = 0; m < p->M; ++m) {
      const double *n = p->mu + 3 * m;
      double wi = p->w[m] * I[(long)m * N + c];
      e += wi;
      for (int i = 0; i < 3; ++i) f[i] += n[i] * wi;
      q[0] += n[0] * n[0] * wi; q[1] += n[1] * n[1] * wi; q[2] += n[2] * n[2] * wi;
      q[3] += n[0] * n[1] * wi; q[4] += n[0] * n[2] * wi; q[5] += n[1] * n[2] * wi;
    }
    E[c] = 4 * ORC_PI * e;
    for (int i = 0; i < 3; ++i) F[3 * c + i] = 4 * ORC_PI * f[i];
    for (int i = 0; i < 6; ++i) P[6 * c + i] = 4 * ORC_PI * q[i];
  }
}

/* ---------------------------------------------------------------------------
 * Boundary values (the test setups of sec. 5): the stencil moves along one
 * axis at a time, so a ghost cell lies outside the grid along exactly one
 * axis.  Periodic: the image cell.  Copy: the nearest active cell, all
 * angles.  Vacuum: outgoing angles copied, incoming angles zero.  Inflow:
 * outgoing copied, incoming set to the given per-angle intensity.  Angles
 * with mu_d = 0 count as outgoing (their flux along d is zero).
 * Material (J, v, sigma) in a ghost cell is that of the image cell
 * (periodic) or of the nearest active cell (other kinds).
 * ------------------------------------------------------------------------- */
static long ghost_cell(const orc_problem *p, const int c[3], int d, int j, int *outside) {
  int n = p->n[d];
  int cc[3] = {c[0], c[1], c[2]};
  *outside = -1;
  if (j >= 0 && j < n) {
    cc[d] = j;
  } else {
    int side = j < 0 ? 0 : 1;
    *outside = side;
    if (p->bc[d][side] == ORC_PERIODIC)
      cc[d] = ((j % n) + n) % n;
    else
      cc[d] = side ? n - 1 : 0;
  }
  return cidx(p, cc);
}

static double intensity_at(const orc_problem *p, const double *I, int m, const int c[3], int d, int j) {
  int side;
  long N = ncells(p);
  long cell = ghost_cell(p, c, d, j, &side);
  double val = I[(long)m * N + cell];
  if (side < 0 || p->bc[d][side] == ORC_PERIODIC || p->bc[d][side] == ORC_COPY) return val;
  double mud = p->mu[3 * m + d];
  int incoming = side ? (mud < 0) : (mud > 0);
  if (!incoming) return val;
  if (p->bc[d][side] == ORC_VACUUM) return 0.0;
  return p->inflow[((long)d * 2 + side) * p->M + m];
}

/* Reduced transport speed factor (sec. 4.2, eq. for alpha):
 * alpha = sqrt((1 - exp(-tau)) / tau), tau = (10 dl (sigma_a + sigma_s))^2. */
double orc_alpha(double dl, double sigma_t) {
  double s = 10.0 * dl * sigma_t;
  double tau = s * s;
  if (tau < 1e-12) return 1.0;
  return sqrt(-expm1(-tau) / tau);
}

/* van Leer limited slope (Stone & Mihalas 1992, eq. 4): the harmonic mean of
 * the one-sided differences where they agree in sign, else zero. */
static double vl_slope(double qm, double q0, double qp) {
  double dl = q0 - qm, dr = qp - q0;
  double pr = dl * dr;
  return pr > 0 ? 2.0 * pr / (dl + dr) : 0.0;
}

/* Step 2 (sec. 4.2): Delta F for every cell and angle.  For each active axis
 * d and angle m the flux through a face is
 *   C mu_d <I~>_f + mu_d <IV>_f,   I~ = I - IV/C,  IV = 3 (n . v) J,
 * with <I~> the alpha-blend of the van Leer upwind/downwind states at speed
 * alpha C and <IV> the van Leer upwind state at the face gas velocity.  The
 * change is -dt * sum_d (flux_{i+1/2} - flux_{i-1/2}) / dx_d, all axes from
 * I^n.  J and v are the values at the start of the step. */
static void transport_all(const orc_problem *p, const double *I, const double *J, const double *v,
                          const double *sigt, double dt, double *dF) {
  long N = ncells(p);
  int M = p->M;
  memset(dF, 0, sizeof(double) * (size_t)M * N);
  for (int d = 0; d < p->dim; ++d) {
    int nd = p->n[d];
    int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
    int n1 = p->n[a1], n2 = p->n[a2];
    double rdx = dt / p->dx[d];
#pragma omp parallel for collapse(2) schedule(static)
    for (int m = 0; m < M; ++m) {
      for (long pen = 0; pen < (long)n1 * n2; ++pen) {
        double mud = p->mu[3 * m + d];
        const double *nm = p->mu + 3 * m;
        int c[3];
        c[a1] = (int)(pen % n1);
        c[a2] = (int)(pen / n1);
        c[d] = 0;
        int L = nd + 4; /* padded pencil: cell j at index j + 2 */
        double *It = malloc(sizeof(double) * L), *IV = malloc(sizeof(double) * L);
        double *al = malloc(sizeof(double) * L), *vd = malloc(sizeof(double) * L);
        double *fl = malloc(sizeof(double) * (nd + 1));
        for (int q = 0; q < L; ++q) {
          int j = q - 2, side;
          long cell = ghost_cell(p, c, d, j, &side);
          const double *vc = v + 3 * cell;
          double iv = 3.0 * (nm[0] * vc[0] + nm[1] * vc[1] + nm[2] * vc[2]) * J[cell];
          IV[q] = iv;
          It[q] = intensity_at(p, I, m, c, d, j) - iv / p->C;
          al[q] = p->alpha_one ? 1.0 : orc_alpha(p->dx[d], sigt[cell]);
          vd[q] = vc[d];
        }
        /* face f lies between cells f-1 and f (padded f+1 and f+2) */
        for (int f = 0; f <= nd; ++f) {
          int qa = f + 1, qb = f + 2;
          double sa = vl_slope(It[qa - 1], It[qa], It[qa + 1]);
          double sb = vl_slope(It[qb - 1], It[qb], It[qb + 1]);
          double af = 0.5 * (al[qa] + al[qb]);
          double nu = af * p->C * fabs(mud) * rdx;
          double left = It[qa] + 0.5 * (1.0 - nu) * sa;
          double right = It[qb] - 0.5 * (1.0 - nu) * sb;
          double up = mud > 0 ? left : right, down = mud > 0 ? right : left;
          double fI = p->C * mud * (0.5 * (1.0 + af) * up + 0.5 * (1.0 - af) * down);

          double va = vl_slope(IV[qa - 1], IV[qa], IV[qa + 1]);
          double vb = vl_slope(IV[qb - 1], IV[qb], IV[qb + 1]);
          double vf = 0.5 * (vd[qa] + vd[qb]);
          double nv = fabs(vf) * rdx;
          double lv = IV[qa] + 0.5 * (1.0 - nv) * va;
          double rv = IV[qb] - 0.5 * (1.0 - nv) * vb;
          double ivf = vf > 0 ? lv : (vf < 0 ? rv : 0.5 * (lv + rv));
          fl[f] = fI + mud * ivf;
        }
        for (int j = 0; j < nd; ++j) {
          c[d] = j;
          dF[(long)m * N + cidx(p, c)] -= rdx * (fl[j + 1] - fl[j]);
        }
        free(It); free(IV); free(al); free(vd); free(fl);
      }
    }
  }
}

/* Step 3 (sec. 4.5): per axis, the linear backward-Euler estimate
 *   rho v~ - rho v = (dt/2) P s_t (C rho v / P + F - C rho v~ / P - v~ (E + P_dd) / C)
 * with s_t = sigma_a + sigma_s and E, F, P_dd held at their step-n values. */
static void vtilde(const orc_problem *p, double rho, const double v[3], double st, double E,
                   const double F[3], const double Pd[3], double dt, double vt[3]) {
  for (int d = 0; d < 3; ++d) {
    double h = 0.5 * dt * st;
    double num = rho * v[d] + h * (p->C * rho * v[d] + p->P * F[d]);
    double den = rho + h * (p->C * rho + p->P * (E + Pd[d]) / p->C);
    vt[d] = num / den;
  }
}

/* Dense linear solve A x = b (n x n, row-major, overwritten), Gaussian
 * elimination with partial pivoting.  Returns 0, or -1 for a zero pivot. */
static int gauss_solve(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(A[(long)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[(long)i * n + k]) > best) { best = fabs(A[(long)i * n + k]); piv = i; }
    if (best == 0.0) return -1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(long)k * n + j]; A[(long)k * n + j] = A[(long)piv * n + j]; A[(long)piv * n + j] = t;
      }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[(long)i * n + k] / A[(long)k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[(long)i * n + j] -= f * A[(long)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[(long)k * n + j] * b[j];
    b[k] = s / A[(long)k * n + k];
  }
  return 0;
}

#define ORC_NEWTON_RTOL 1e-13
#define ORC_NEWTON_MAXIT 60

/* Per-cell inputs of the implicit steps. */
typedef struct {
  double rho, T0, sa, ss, dt;
  double v[3];   /* v~ used in Steps 4 and 5 */
} cellstate;

/* Step 4, dense form: Newton-Raphson on all N+1 unknowns (I_1..I_N, T) of
 * eq. absorptionmatrix, started from (I^n, T^n), each Newton step solved by
 * Gaussian elimination.  With hold_T the T row is dropped and the N linear
 * equations are solved once.  Returns 0, or 1 if Newton did not converge. */
static int absorption_dense(const orc_problem *p, const cellstate *cs, const double *r,
                            const double *Istart, double *I, double *T1) {
  int M = p->M;
  double C = p->C, P = p->P, sa = cs->sa, dt = cs->dt;
  double v2 = cs->v[0] * cs->v[0] + cs->v[1] * cs->v[1] + cs->v[2] * cs->v[2];
  double kv = cs->rho * p->R / (p->gamma - 1.0);
  double *vn = malloc(sizeof(double) * M), *g = malloc(sizeof(double) * M);
  for (int m = 0; m < M; ++m) {
    const double *n = p->mu + 3 * m;
    vn[m] = n[0] * cs->v[0] + n[1] * cs->v[1] + n[2] * cs->v[2];
    g[m] = p->w[m] * (v2 + vn[m] * vn[m]);
  }
  int status = 0;
  if (p->hold_T) {
    double th = pow(cs->T0, 4) / (4 * ORC_PI);
    double *A = malloc(sizeof(double) * M * M);
    for (int i = 0; i < M; ++i) {
      for (int l = 0; l < M; ++l) A[(long)i * M + l] = dt * sa / C * g[l];
      A[(long)i * M + i] += 1.0 + dt * C * sa - dt * sa * vn[i];
      I[i] = r[i] + dt * sa * (C + 3.0 * vn[i]) * th;
    }
    if (gauss_solve(M, A, I)) status = 1;
    *T1 = cs->T0;
    free(A);
  } else {
    int K = M + 1;
    double *A = malloc(sizeof(double) * K * K), *b = malloc(sizeof(double) * K);
    double T = cs->T0;
    for (int m = 0; m < M; ++m) I[m] = Istart[m];
    int extra = -1, it;
    for (it = 0; it < ORC_NEWTON_MAXIT; ++it) {
      double th = pow(T, 4) / (4 * ORC_PI), dth = pow(T, 3) / ORC_PI;
      double sumW = 0, sumWvn = 0, sumg = 0;
      for (int l = 0; l < M; ++l) {
        sumW += p->w[l] * I[l]; sumWvn += p->w[l] * vn[l] * I[l]; sumg += g[l] * I[l];
      }
      /* residuals of eq. absorptionmatrix multiplied by dt */
      for (int i = 0; i < M; ++i) {
        double Ri = I[i] - r[i] - dt * (C * sa * (th - I[i]) + 3.0 * vn[i] * sa * th + vn[i] * sa * I[i]
                                        - sa * v2 / C * sumW
                                        - sa / C * (sumg - v2 * sumW));
        /* sum_l v.(v.n_l n_l) I_l W_l = sumg - v2 sumW */
        b[i] = -Ri;
        for (int l = 0; l < M; ++l) A[(long)i * K + l] = dt * sa / C * g[l];
        A[(long)i * K + i] += 1.0 + dt * C * sa - dt * sa * vn[i];
        A[(long)i * K + M] = -dt * sa * (C + 3.0 * vn[i]) * dth;
      }
      double RT = kv * (T - cs->T0)
                  + dt * (8 * ORC_PI * P * sa * (sumWvn - sumg / C)
                          + P * C * (1.0 - v2 / (C * C)) * sa * (pow(T, 4) - 4 * ORC_PI * sumW));
      b[M] = -RT;
      for (int l = 0; l < M; ++l)
        A[(long)M * K + l] = dt * (8 * ORC_PI * P * sa * (p->w[l] * vn[l] - g[l] / C)
                                   - 4 * ORC_PI * P * C * (1.0 - v2 / (C * C)) * sa * p->w[l]);
      A[(long)M * K + M] = kv + 4.0 * dt * P * C * (1.0 - v2 / (C * C)) * sa * pow(T, 3);
      if (gauss_solve(K, A, b)) { status = 1; break; }
      double imax = 0, dimax = 0;
      for (int m = 0; m < M; ++m) {
        I[m] += b[m];
        if (fabs(I[m]) > imax) imax = fabs(I[m]);
        if (fabs(b[m]) > dimax) dimax = fabs(b[m]);
      }
      T += b[M];
      if (extra == 0) break;
      if (extra < 0 && fabs(b[M]) <= ORC_NEWTON_RTOL * fabs(T) && dimax <= ORC_NEWTON_RTOL * imax) extra = 0;
    }
    if (it == ORC_NEWTON_MAXIT || !(T > 0)) status = 1;
    *T1 = T;
    free(A); free(b);
  }
  free(vn); free(g);
  return status;
}

/* Step 4, reduced O(N) form.  Each I-row of eq. absorptionmatrix reads
 *   d_m I_m = r_m + e_m theta - kappa S,
 *   d_m = 1 + dt C s_a - dt s_a n_m.v,  e_m = dt s_a (C + 3 n_m.v),
 *   theta = T^4 / 4pi,  kappa = dt s_a / C,  S = sum_l g_l I_l,
 *   g_l = W_l (v.v + (n_l.v)^2),
 * so S, J = sum W I and v.H = sum W (n.v) I are affine in theta and the T-row
 * becomes a scalar quartic c4 T^4 + k_v T + c0 = 0 solved by Newton from T^n.
 * The stopping rule is |dT| <= 1e-13 T followed by one more iteration. */
static int absorption_reduced(const orc_problem *p, const cellstate *cs, const double *r,
                              double *I, double *T1) {
  int M = p->M;
  double C = p->C, P = p->P, sa = cs->sa, dt = cs->dt;
  double v2 = cs->v[0] * cs->v[0] + cs->v[1] * cs->v[1] + cs->v[2] * cs->v[2];
  double kv = cs->rho * p->R / (p->gamma - 1.0);
  double kap = dt * sa / C;
  double Wr = 0, We = 0, W1 = 0, Vr = 0, Ve = 0, V1 = 0, Gr = 0, Ge = 0, G1 = 0, Wq = 0;
  for (int m = 0; m < M; ++m) {
    const double *n = p->mu + 3 * m;
    double vn = n[0] * cs->v[0] + n[1] * cs->v[1] + n[2] * cs->v[2];
    double d = 1.0 + dt * C * sa - dt * sa * vn;
    double e = dt * sa * (C + 3.0 * vn);
    double W = p->w[m], g = W * (v2 + vn * vn);
    Wr += W * r[m] / d; We += W * e / d; W1 += W / d;
    Wq += W * (1.0 - 4.0 * dt * sa * vn) / d; /* = sum W (d - e) / d */
    Vr += W * vn * r[m] / d; Ve += W * vn * e / d; V1 += W * vn / d;
    Gr += g * r[m] / d; Ge += g * e / d; G1 += g / d;
  }
  double den = 1.0 + kap * G1;
  double S0 = Gr / den, S1 = Ge / den;          /* S = S0 + theta S1 */
  double J0 = Wr - kap * S0 * W1;
  double H0 = Vr - kap * S0 * V1, H1 = Ve - kap * S1 * V1;
  double T = cs->T0, th;
  int status = 0;
  if (p->hold_T) {
    th = pow(T, 4) / (4 * ORC_PI);
  } else {
    double beta = P * C * (1.0 - v2 / (C * C)) * sa;
    double c0 = dt * (8 * ORC_PI * P * sa * (H0 - S0 / C) - 4 * ORC_PI * beta * J0) - kv * cs->T0;
    /* 1 - J1 = sum W (d - e)/d + kappa S1 W1 (sum W = 1), formed without the
     * cancellation 1 - We suffers when dt C s_a >> 1 */
    double omJ1 = Wq + kap * S1 * W1;
    double c4 = dt * (2.0 * P * sa * (H1 - S1 / C) + beta * omJ1);
    int extra = -1, it;
    for (it = 0; it < ORC_NEWTON_MAXIT; ++it) {
      double T3 = T * T * T;
      double f = c4 * T3 * T + kv * T + c0;
      double fp = 4.0 * c4 * T3 + kv;
      double Tn = T - f / fp;
      if (!(Tn > 0)) Tn = 0.5 * T; /* keep the iterate positive */
      double dT = Tn - T;
      T = Tn;
      if (extra == 0) break;
      if (extra < 0 && fabs(dT) <= ORC_NEWTON_RTOL * T) extra = 0;
    }
    if (it == ORC_NEWTON_MAXIT) status = 1;
    th = pow(T, 4) / (4 * ORC_PI);
  }
  double S = S0 + th * S1;
  for (int m = 0; m < M; ++m) {
    const double *n = p->mu + 3 * m;
    double vn = n[0] * cs->v[0] + n[1] * cs->v[1] + n[2] * cs->v[2];
    double d = 1.0 + dt * C * sa - dt * sa * vn;
    double e = dt * sa * (C + 3.0 * vn);
    I[m] = (r[m] + e * th - kap * S) / d;
  }
  *T1 = T;
  return status;
}

/* Step 5 coefficients (sec. 4.4), unknowns x_l = W_l I_l:
 *   M_s[m][l] = a_m delta_ml + b_l + c_m, right-hand side r_m,
 *   a_m = (1 + dt C s_s - dt s_s n_m.v) / W_m,
 *   b_l = -dt C s_s + 2 dt s_s n_l.v - dt s_s v.v / C - dt s_s (n_l.v)^2 / C,
 *   c_m = -3 dt s_s n_m.v.
 * (b carries the column index l: it multiplies x_l.) */
static void scat_coeffs(const orc_problem *p, const cellstate *cs, int m, double *a, double *b, double *c) {
  const double *n = p->mu + 3 * m;
  double C = p->C, ss = cs->ss, dt = cs->dt;
  double v2 = cs->v[0] * cs->v[0] + cs->v[1] * cs->v[1] + cs->v[2] * cs->v[2];
  double vn = n[0] * cs->v[0] + n[1] * cs->v[1] + n[2] * cs->v[2];
  *a = (1.0 + dt * C * ss - dt * ss * vn) / p->w[m];
  *b = -dt * C * ss + 2.0 * dt * ss * vn - dt * ss * v2 / C - dt * ss * vn * vn / C;
  *c = -3.0 * dt * ss * vn;
}

/* Step 5, dense form: build M_s and solve by Gaussian elimination. */
static int scattering_dense(const orc_problem *p, const cellstate *cs, const double *r, double *I) {
  int M = p->M;
  double *A = malloc(sizeof(double) * M * M), *a = malloc(sizeof(double) * M);
  double *b = malloc(sizeof(double) * M), *c = malloc(sizeof(double) * M);
  for (int m = 0; m < M; ++m) scat_coeffs(p, cs, m, a + m, b + m, c + m);
  for (int i = 0; i < M; ++i) {
    for (int l = 0; l < M; ++l) A[(long)i * M + l] = b[l] + c[i];
    A[(long)i * M + i] += a[i];
    I[i] = r[i];
  }
  int st = gauss_solve(M, A, I) ? 1 : 0;
  for (int m = 0; m < M; ++m) I[m] /= p->w[m];
  free(A); free(a); free(b); free(c);
  return st;
}

/* Step 5, reduced O(N) form.  With s1 = sum_l b_l x_l and s2 = sum_l x_l each
 * row gives x_m = (r_m - s1 - c_m s2) / a_m; summing those rows against b_m
 * and against 1 gives a 2x2 linear system for (s1, s2). */
static int scattering_reduced(const orc_problem *p, const cellstate *cs, const double *r, double *I) {
  int M = p->M;
  double Br = 0, B1p = 0, Bc = 0, Ar = 0, A1 = 0, Ac = 0;
  for (int m = 0; m < M; ++m) {
    double a, b, c;
    scat_coeffs(p, cs, m, &a, &b, &c);
    Br += b * r[m] / a; Bc += b * c / a;
    Ar += r[m] / a; A1 += 1.0 / a; Ac += c / a;
    /* 1 + B1 = sum_m W_m (1 + b_m / (W_m a_m)) since sum W = 1; the
     * numerator W a + b = 1 + dt s_s vn - dt s_s (v.v + vn^2)/C has the
     * dt C s_s terms of a and b cancelled exactly, which keeps the (1,1)
     * entry accurate when dt C s_s >> 1 */
    const double *n = p->mu + 3 * m;
    double vn = n[0] * cs->v[0] + n[1] * cs->v[1] + n[2] * cs->v[2];
    double v2 = cs->v[0] * cs->v[0] + cs->v[1] * cs->v[1] + cs->v[2] * cs->v[2];
    double num = 1.0 + cs->dt * cs->ss * vn - cs->dt * cs->ss * (v2 + vn * vn) / p->C;
    B1p += num / a;
  }
  /* (1 + B1) s1 + Bc s2 = Br ;  A1 s1 + (1 + Ac) s2 = Ar */
  double m11 = B1p, m12 = Bc, m21 = A1, m22 = 1.0 + Ac;
  double det = m11 * m22 - m12 * m21;
  if (det == 0.0) return 1;
  double s1 = (Br * m22 - m12 * Ar) / det;
  double s2 = (m11 * Ar - m21 * Br) / det;
  for (int m = 0; m < M; ++m) {
    double a, b, c;
    scat_coeffs(p, cs, m, &a, &b, &c);
    I[m] = (r[m] - s1 - c * s2) / a / p->w[m];
  }
  return 0;
}

/* One full radiation step (Steps 2-5 plus the quadrature), in place.
 *   I      [M][N] intensity, overwritten with I^{n+1}
 *   T      [N] gas temperature, overwritten with T^{n+1}
 *   rho, sa, ss [N]; v [N][3] gas velocity (held fixed by this library)
 *   dEgas  [N] out: Delta E_T + Delta E_K
 *   dMom   [N][3] out: Delta(rho v)
 *   dF_out [M][N] out (may be NULL): the transport change Delta F
 * Returns the number of cells whose implicit solve failed (0 on success). */
long orc_step(const orc_problem *p, double dt, double *I, double *T, const double *rho, const double *v,
              const double *sa, const double *ss, double *dEgas, double *dMom, double *dF_out) {
  long N = ncells(p);
  int M = p->M;
  double *E = malloc(sizeof(double) * N), *F = malloc(sizeof(double) * 3 * N);
  double *Pm = malloc(sizeof(double) * 6 * N), *J = malloc(sizeof(double) * N);
  double *st = malloc(sizeof(double) * N);
  double *dF = dF_out ? dF_out : malloc(sizeof(double) * (size_t)M * N);
  orc_moments(p, I, E, F, Pm);
  for (long c = 0; c < N; ++c) {
    J[c] = E[c] / (4 * ORC_PI);
    st[c] = sa[c] + ss[c];
  }
  transport_all(p, I, J, v, st, dt, dF);
  long failures = 0;
#pragma omp parallel for schedule(static) reduction(+ : failures)
  for (long c = 0; c < N; ++c) {
    double *r = malloc(sizeof(double) * M), *Ia = malloc(sizeof(double) * M);
    double *Is = malloc(sizeof(double) * M), *I0 = malloc(sizeof(double) * M);
    cellstate cs;
    cs.rho = rho[c]; cs.T0 = T[c]; cs.sa = sa[c]; cs.ss = ss[c]; cs.dt = dt;
    const double *vc = v + 3 * c;
    if (p->estimate_v) {
      double Pd[3] = {Pm[6 * c], Pm[6 * c + 1], Pm[6 * c + 2]};
      vtilde(p, rho[c], vc, st[c], E[c], F + 3 * c, Pd, dt, cs.v);
    } else {
      cs.v[0] = vc[0]; cs.v[1] = vc[1]; cs.v[2] = vc[2];
    }
    int to_scat = ss[c] > sa[c];
    double pre[3] = {0, 0, 0};
    for (int m = 0; m < M; ++m) {
      I0[m] = I[(long)m * N + c];
      double full = I0[m] + dF[(long)m * N + c];
      r[m] = to_scat ? I0[m] : full;
      for (int i = 0; i < 3; ++i) pre[i] += p->w[m] * p->mu[3 * m + i] * full;
    }
    double T1;
    int bad = p->dense ? absorption_dense(p, &cs, r, I0, Ia, &T1) : absorption_reduced(p, &cs, r, Ia, &T1);
    for (int m = 0; m < M; ++m) r[m] = Ia[m] + (to_scat ? dF[(long)m * N + c] : 0.0);
    bad |= p->dense ? scattering_dense(p, &cs, r, Is) : scattering_reduced(p, &cs, r, Is);
    double post[3] = {0, 0, 0};
    for (int m = 0; m < M; ++m) {
      I[(long)m * N + c] = Is[m];
      for (int i = 0; i < 3; ++i) post[i] += p->w[m] * p->mu[3 * m + i] * Is[m];
    }
    /* Gas sources: Delta E_T = rho R/(gamma-1) (T^{n+1} - T^n) (sec. 4.3),
     * Delta(rho v) = -(4 pi P / C) (sum W n I after - before) (eq. momentumchange),
     * Delta E_K from the momentum change (eq. kinetichange). */
    double kv = rho[c] * p->R / (p->gamma - 1.0);
    double dEK = 0;
    for (int i = 0; i < 3; ++i) {
      double dm = -(4 * ORC_PI * p->P / p->C) * (post[i] - pre[i]);
      dMom[3 * c + i] = dm;
      double m0 = rho[c] * vc[i];
      dEK += ((m0 + dm) * (m0 + dm) - m0 * m0) / (2.0 * rho[c]);
    }
    dEgas[c] = kv * (T1 - T[c]) + dEK;
    T[c] = T1;
    failures += bad ? 1 : 0;
    free(r); free(Ia); free(Is); free(I0);
  }
  free(E); free(F); free(Pm); free(J); free(st);
  if (!dF_out) free(dF);
  return failures;
}

/* Isolated pieces exposed for the pins. */
int orc_absorption_cell(const orc_problem *p, double rho, double T0, double sa, double dt, const double v[3],
                        const double *r, const double *Istart, double *I, double *T1) {
  cellstate cs = {rho, T0, sa, 0.0, dt, {v[0], v[1], v[2]}};
  return p->dense ? absorption_dense(p, &cs, r, Istart, I, T1) : absorption_reduced(p, &cs, r, I, T1);
}

int orc_scattering_cell(const orc_problem *p, double ss, double dt, const double v[3], const double *r, double *I) {
  cellstate cs = {1.0, 1.0, 0.0, ss, dt, {v[0], v[1], v[2]}};
  return p->dense ? scattering_dense(p, &cs, r, I) : scattering_reduced(p, &cs, r, I);
}

void orc_transport(const orc_problem *p, double dt, const double *I, const double *v, const double *sa,
                   const double *ss, double *dF) {
  long N = ncells(p);
  double *E = malloc(sizeof(double) * N), *F = malloc(sizeof(double) * 3 * N);
  double *Pm = malloc(sizeof(double) * 6 * N), *J = malloc(sizeof(double) * N), *st = malloc(sizeof(double) * N);
  orc_moments(p, I, E, F, Pm);
  for (long c = 0; c < N; ++c) { J[c] = E[c] / (4 * ORC_PI); st[c] = sa[c] + ss[c]; }
  transport_all(p, I, J, v, st, dt, dF);
  free(E); free(F); free(Pm); free(J); free(st);
}

void orc_vtilde(const orc_problem *p, double rho, const double v[3], double st, double E, const double F[3],
                const double Pd[3], double dt, double vt[3]) {
  vtilde(p, rho, v, st, E, F, Pd, dt, vt);
}

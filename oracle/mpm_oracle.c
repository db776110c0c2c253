/*
 * mpm_oracle.c -- plain, serial, FP64 CPU oracle for the differentiable MLS-MPM
 * elastic-object simulator (diffmpm, paper Section 4.1 and Appendix D).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (the paper gives no MLS-MPM equations of its own: Section 4.1
 * says the simulator follows ChainQueen and the moving-least-squares MPM of
 * Hu et al. 2018, so the steps below are that published method written out):
 *
 *   one time step s (Appendix D "advance"): clear grid -> actuation -> P2G ->
 *   grid_op -> G2P.
 *     P2G     quadratic B-spline weights, APIC affine momentum with the MLS
 *             stress folded into the affine matrix A = -dt V0 (4/dx^2) tau + m C.
 *     grid_op v_i = p_i/m_i + dt g for m_i > 0, sticky walls wall_cells thick.
 *     G2P     v' = sum W v_i, C' = (4/dx^2) sum W v_i (x_i - x_p)^T,
 *             x' = x + dt v', F' = (I + dt C') F.
 *     stress  fixed-corotated tau = 2 mu (F - R) F^T + lambda (J - 1) J I,
 *             neo-Hookean     tau = mu (F F^T - I) + lambda ln(J) I,
 *             actuation       tau += a (F e)(F e)^T, a = sum_k w_gk sin(2 pi k t/P + phi),
 *             or (closed loop) a = the controller's output for the particle's group,
 *             evaluated on the state of step s (orc_controller).
 *   the adjoint of one step (Appendix D.1 "advance_grad"): recompute the grid
 *   from state_s (clear_grid, p2g, grid_op), then g2p.grad, grid_op.grad,
 *   p2g.grad and the actuation/stress adjoint, in that order.
 *   the tape (Section 3.2): replay the step adjoints for s = T-1 .. 0.  The
 *   oracle keeps every state (no checkpointing), which Appendix D.2 shows to be
 *   the same computation as segment-wise recomputation.
 *
 * Polar decomposition (Appendix C uses an SVD with a hand-written gradient):
 *   3D: cyclic Jacobi eigen-decomposition of F^T F (Golub & Van Loan 8.5), R =
 *   F V Sigma^-1 V^T; adjoint Fbar += 2 R Y with Y = V Ytilde V^T,
 *   Ytilde_ij = Btilde_ij / (sigma_i + sigma_j), B = skew(R^T Rbar).
 *   2D: R = rotation(theta), theta = atan2(F10 - F01, F00 + F11); adjoint by
 *   the atan2 derivative.
 *
 * Layout: every per-particle array is component-major, a[c * n + p].
 * Grids are dense n_grid^dim arrays, node (i0,i1[,i2]) at flat index
 * (i0 * n + i1) [* n + i2]; momentum/velocity grids hold dim doubles per node.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_MEM 2
#define ORC_ERR_OOB 3     /* a particle's 3^d stencil leaves the grid */
#define ORC_ERR_DOMAIN 4  /* det F <= 0 or a non-finite value */

#define ORC_FIXED_COROTATED 0
#define ORC_NEO_HOOKEAN 1
#define ORC_NO_ELASTICITY 2
#define ORC_LIQUID 3          /* weakly compressible liquid (the paper's liquid simulator) */
#define ORC_MIXED 4           /* per-particle material (0, 1 or 3) from particle_material[]:
                                 the two-way coupling of a solid and a liquid in one grid */

/* Liquid equation of state (Tait form of the weakly compressible model the paper's liquid
   simulator follows, Tampubolon et al. 2017): psi(J) = kappa (J - J^(1-g)/(1-g)), so the
   pressure is p = -psi'(J) = kappa (J^-g - 1) and the Kirchhoff stress tau = psi'(J) J I =
   kappa (J - J^(1-g)) I; kappa = lambda + 2 mu / d is the bulk modulus of the particle's
   (E, nu) and g = 7. */
#define ORC_LIQUID_GAMMA 7.0

/* limits of the closed-loop controller (Section 4.1's neural-network controllers) */
#define ORC_CTRL_MAX_GROUPS 8
#define ORC_CTRL_MAX_HIDDEN 64
#define ORC_CTRL_MAX_INPUTS (8 + 2 * 3 * ORC_CTRL_MAX_GROUPS)

#define ORC_LOSS_COM_TARGET 0   /* L = |COM(x_T) - target|^2            */
#define ORC_LOSS_COM_X_DISP 1   /* L = -(COM_x(x_T) - COM_x(x_0))       */

typedef struct {
  int32_t dim;        /* 2 or 3 */
  int32_t n_grid;     /* nodes per axis; dx = 1 / n_grid */
  double dt;
  double gravity[3];
  int32_t wall_cells; /* sticky boundary thickness in nodes; 0 = no walls */
  int32_t material;   /* ORC_FIXED_COROTATED / ORC_NEO_HOOKEAN / ORC_NO_ELASTICITY / ORC_LIQUID */
  double rho;         /* density; particle volume (dx/2)^dim, mass rho * volume */
  int32_t n_groups;   /* actuation groups (0 = no actuation) */
  int32_t n_basis;    /* sine terms per group */
  double act_period;  /* P in sin(2 pi k t / P + phi) */
  double act_phase;   /* phi */
  const int32_t* particle_material; /* [np] material of each particle when material is
                                       ORC_MIXED (indexed like mu, la), else unused */
  int32_t ctrl_hidden; /* 0: open-loop sine actuation, wact = w[G][K]; H > 0: closed-loop
                          controller with H hidden units, wact = theta (see orc_controller) */
  double ctrl_scale;   /* controller output scale: a_g = ctrl_scale tanh(.) */
} orc_params;

/* ------------------------------------------------------------------ */
/* small dense helpers (row-major d x d, d <= 3)                       */
/* ------------------------------------------------------------------ */

typedef double mat3[3][3];

static void mzero(mat3 a) { memset(a, 0, sizeof(mat3)); }

static void meye(int d, mat3 a) {
  mzero(a);
  for (int i = 0; i < d; i++) a[i][i] = 1.0;
}

static void mmul(int d, const mat3 a, const mat3 b, mat3 c) {
  mat3 t;
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      double s = 0.0;
      for (int k = 0; k < d; k++) s += a[i][k] * b[k][j];
      t[i][j] = s;
    }
  memcpy(c, t, sizeof(mat3));
}

static void mtrans(int d, const mat3 a, mat3 b) {
  mat3 t;
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) t[i][j] = a[j][i];
  memcpy(b, t, sizeof(mat3));
}

static double mdet(int d, const mat3 a) {
  if (d == 2) return a[0][0] * a[1][1] - a[0][1] * a[1][0];
  return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
         a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
         a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

/* cofactor matrix: cof(A)_ij = dDet/dA_ij, so cof(A) = det(A) A^{-T} */
static void mcof(int d, const mat3 a, mat3 c) {
  mzero(c);
  if (d == 2) {
    c[0][0] = a[1][1];
    c[0][1] = -a[1][0];
    c[1][0] = -a[0][1];
    c[1][1] = a[0][0];
    return;
  }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      c[i][j] = a[i1][j1] * a[i2][j2] - a[i1][j2] * a[i2][j1];
    }
}

static double mdot(int d, const mat3 a, const mat3 b) {
  double s = 0.0;
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) s += a[i][j] * b[i][j];
  return s;
}

static double mtrace(int d, const mat3 a) {
  double s = 0.0;
  for (int i = 0; i < d; i++) s += a[i][i];
  return s;
}

static void load_mat(int d, const double* arr, int64_t n, int64_t p, mat3 m) {
  mzero(m);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) m[i][j] = arr[(int64_t)(i * d + j) * n + p];
}

static void store_mat(int d, double* arr, int64_t n, int64_t p, const mat3 m) {
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) arr[(int64_t)(i * d + j) * n + p] = m[i][j];
}

static int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

/* ------------------------------------------------------------------ */
/* Lame parameters from Young's modulus and Poisson ratio              */
/* ------------------------------------------------------------------ */

void orc_lame(int64_t n, const double* E, const double* nu, double* mu, double* la) {
  for (int64_t p = 0; p < n; p++) {
    mu[p] = E[p] / (2.0 * (1.0 + nu[p]));
    la[p] = E[p] * nu[p] / ((1.0 + nu[p]) * (1.0 - 2.0 * nu[p]));
  }
}

/* chain rule of orc_lame: (mu_bar, la_bar) -> (E_bar, nu_bar) */
void orc_lame_adjoint(int64_t n, const double* E, const double* nu, const double* mu_bar,
                      const double* la_bar, double* E_bar, double* nu_bar) {
  for (int64_t p = 0; p < n; p++) {
    double e = E[p], v = nu[p];
    double q = (1.0 + v) * (1.0 - 2.0 * v);
    double dmu_dE = 1.0 / (2.0 * (1.0 + v));
    double dla_dE = v / q;
    double dmu_dnu = -e / (2.0 * (1.0 + v) * (1.0 + v));
    /* d/dnu [nu / ((1+nu)(1-2nu))] = (1 + 2 nu^2) / q^2 */
    double dla_dnu = e * (1.0 + 2.0 * v * v) / (q * q);
    E_bar[p] = mu_bar[p] * dmu_dE + la_bar[p] * dla_dE;
    nu_bar[p] = mu_bar[p] * dmu_dnu + la_bar[p] * dla_dnu;
  }
}

/* ------------------------------------------------------------------ */
/* quadratic B-spline stencil (MLS-MPM, Hu et al. 2018)                */
/* ------------------------------------------------------------------ */

typedef struct {
  int base[3];
  double f[3];      /* x/dx - base, in [0.5, 1.5) */
  double w[3][3];   /* w[axis][offset] */
  double dw[3][3];  /* d w / d f */
} stencil;

static int make_stencil(const orc_params* P, const double* xp, stencil* s) {
  int d = P->dim, n = P->n_grid;
  for (int a = 0; a < 3; a++) {
    s->base[a] = 0;
    s->f[a] = 0.0;
    for (int o = 0; o < 3; o++) s->w[a][o] = s->dw[a][o] = 0.0;
  }
  for (int a = 0; a < d; a++) {
    double X = xp[a] * (double)n;
    if (!isfinite(X)) return ORC_ERR_DOMAIN;
    double b = floor(X - 0.5);
    if (b < 0.0 || b > (double)(n - 3)) return ORC_ERR_OOB;
    double f = X - b;
    s->base[a] = (int)b;
    s->f[a] = f;
    s->w[a][0] = 0.5 * (1.5 - f) * (1.5 - f);
    s->w[a][1] = 0.75 - (f - 1.0) * (f - 1.0);
    s->w[a][2] = 0.5 * (f - 0.5) * (f - 0.5);
    s->dw[a][0] = -(1.5 - f);
    s->dw[a][1] = -2.0 * (f - 1.0);
    s->dw[a][2] = f - 0.5;
  }
  return ORC_OK;
}

/* offset index o in [0, 3^d) -> per-axis offsets */
static void offset_of(int d, int o, int off[3]) {
  off[0] = off[1] = off[2] = 0;
  for (int a = d - 1; a >= 0; a--) {
    off[a] = o % 3;
    o /= 3;
  }
}

static int64_t node_index(int d, int n, const int idx[3]) {
  int64_t r = 0;
  for (int a = 0; a < d; a++) r = r * n + idx[a];
  return r;
}

/* weight W, its gradient dW/dx_p and dpos = x_i - x_p for offset off */
static void stencil_eval(int d, int n, const stencil* s, const int off[3], double* W,
                         double gradW[3], double dpos[3], int idx[3]) {
  double dx = 1.0 / (double)n;
  double w = 1.0;
  for (int a = 0; a < d; a++) w *= s->w[a][off[a]];
  *W = w;
  for (int a = 0; a < 3; a++) gradW[a] = dpos[a] = 0.0;
  for (int a = 0; a < d; a++) {
    double g = s->dw[a][off[a]] * (double)n; /* df/dx = 1/dx */
    for (int b = 0; b < d; b++)
      if (b != a) g *= s->w[b][off[b]];
    gradW[a] = g;
    dpos[a] = ((double)off[a] - s->f[a]) * dx;
    idx[a] = s->base[a] + off[a];
  }
}

/* ------------------------------------------------------------------ */
/* polar decomposition F = R S                                         */
/* ------------------------------------------------------------------ */

/* cyclic Jacobi eigen-decomposition of a symmetric 3x3 A: A = V diag(lam) V^T,
   eigenvalues sorted ascending (Golub & Van Loan, Section 8.5). */
static void jacobi_eig3(const mat3 Ain, mat3 V, double lam[3]) {
  mat3 A;
  memcpy(A, Ain, sizeof(mat3));
  meye(3, V);
  for (int sweep = 0; sweep < 64; sweep++) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-36 * diag || off == 0.0) break;
    for (int p = 0; p < 2; p++)
      for (int q = p + 1; q < 3; q++) {
        if (A[p][q] == 0.0) continue;
        /* rotation that zeroes A[p][q] */
        double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; k++) { /* A <- A J */
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; k++) { /* A <- J^T A */
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; k++) { /* V <- V J */
          double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < 3; i++) lam[i] = A[i][i];
  /* sort ascending, permuting columns of V */
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2 - i; j++)
      if (lam[j] > lam[j + 1]) {
        double t = lam[j];
        lam[j] = lam[j + 1];
        lam[j + 1] = t;
        for (int k = 0; k < 3; k++) {
          double tv = V[k][j];
          V[k][j] = V[k][j + 1];
          V[k][j + 1] = tv;
        }
      }
}

/* 3D polar with the eigen-data of S (S = V diag(sig) V^T, sig ascending). */
static int polar3_full(const mat3 F, mat3 R, mat3 S, mat3 V, double sig[3]) {
  double J = mdet(3, F);
  if (!(J > 0.0) || !isfinite(J)) return ORC_ERR_DOMAIN;
  mat3 Ft, FtF;
  mtrans(3, F, Ft);
  mmul(3, Ft, F, FtF);
  double lam[3];
  jacobi_eig3(FtF, V, lam);
  for (int i = 0; i < 3; i++) {
    if (!(lam[i] > 0.0)) return ORC_ERR_DOMAIN;
    sig[i] = sqrt(lam[i]);
  }
  /* S = V Sigma V^T, R = F V Sigma^-1 V^T */
  mat3 Vt, SigVt, InvSigVt, FV;
  mtrans(3, V, Vt);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      SigVt[i][j] = sig[i] * Vt[i][j];
      InvSigVt[i][j] = Vt[i][j] / sig[i];
    }
  mmul(3, V, SigVt, S);
  mmul(3, F, V, FV);
  mmul(3, FV, InvSigVt, R);
  return ORC_OK;
}

/* exported: polar decomposition of one d x d matrix (row-major) */
int orc_polar(int dim, const double* Fin, double* Rout, double* Sout) {
  mat3 F, R, S;
  mzero(F);
  for (int i = 0; i < dim; i++)
    for (int j = 0; j < dim; j++) F[i][j] = Fin[i * dim + j];
  if (dim == 2) {
    if (!(mdet(2, F) > 0.0)) return ORC_ERR_DOMAIN;
    double th = atan2(F[1][0] - F[0][1], F[0][0] + F[1][1]);
    mzero(R);
    R[0][0] = cos(th);
    R[0][1] = -sin(th);
    R[1][0] = sin(th);
    R[1][1] = cos(th);
    mat3 Rt;
    mtrans(2, R, Rt);
    mmul(2, Rt, F, S);
  } else if (dim == 3) {
    mat3 V;
    double sig[3];
    int rc = polar3_full(F, R, S, V, sig);
    if (rc) return rc;
  } else {
    return ORC_ERR_ARG;
  }
  for (int i = 0; i < dim; i++)
    for (int j = 0; j < dim; j++) {
      Rout[i * dim + j] = R[i][j];
      if (Sout) Sout[i * dim + j] = S[i][j];
    }
  return ORC_OK;
}

/* Fbar += dR/dF^T [Rbar] for the rotation factor R of F (Appendix C's custom
   SVD gradient, written for the polar factor). */
static int polar_adjoint(int d, const mat3 F, const mat3 Rbar, mat3 Fbar) {
  if (d == 2) {
    /* theta = atan2(a, b), a = F10 - F01, b = F00 + F11 */
    double a = F[1][0] - F[0][1], b = F[0][0] + F[1][1];
    double r2 = a * a + b * b;
    double th = atan2(a, b), c = cos(th), s = sin(th);
    /* dR/dtheta = [[-s, -c], [c, -s]] */
    double thbar = -s * Rbar[0][0] - c * Rbar[0][1] + c * Rbar[1][0] - s * Rbar[1][1];
    double da = b / r2, db = -a / r2;
    Fbar[1][0] += thbar * da;
    Fbar[0][1] -= thbar * da;
    Fbar[0][0] += thbar * db;
    Fbar[1][1] += thbar * db;
    return ORC_OK;
  }
  mat3 R, S, V;
  double sig[3];
  int rc = polar3_full(F, R, S, V, sig);
  if (rc) return rc;
  mat3 Rt, RtRbar, B, Vt, Bt, tmp, Y, Yt, RY;
  mtrans(3, R, Rt);
  mmul(3, Rt, Rbar, RtRbar);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) B[i][j] = 0.5 * (RtRbar[i][j] - RtRbar[j][i]);
  mtrans(3, V, Vt);
  mmul(3, Vt, B, tmp);
  mmul(3, tmp, V, Bt); /* Btilde = V^T B V */
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double den = sig[i] + sig[j];
      if (den < 1e-6) den = 1e-6;
      Yt[i][j] = Bt[i][j] / den;
    }
  mmul(3, V, Yt, tmp);
  mmul(3, tmp, Vt, Y);
  mmul(3, R, Y, RY);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) Fbar[i][j] += 2.0 * RY[i][j];
  return ORC_OK;
}

/* exported: Fbar = dR/dF^T [Rbar] */
int orc_polar_adjoint(int dim, const double* Fin, const double* Rbar_in, double* Fbar_out) {
  mat3 F, Rb, Fb;
  mzero(F);
  mzero(Rb);
  mzero(Fb);
  for (int i = 0; i < dim; i++)
    for (int j = 0; j < dim; j++) {
      F[i][j] = Fin[i * dim + j];
      Rb[i][j] = Rbar_in[i * dim + j];
    }
  int rc = polar_adjoint(dim, F, Rb, Fb);
  for (int i = 0; i < dim; i++)
    for (int j = 0; j < dim; j++) Fbar_out[i * dim + j] = Fb[i][j];
  return rc;
}

/* ------------------------------------------------------------------ */
/* actuation (diffmpm's open-loop controller, Section 4.1 / Fig. 7)    */
/* ------------------------------------------------------------------ */

static double act_basis(const orc_params* P, int k /* 1-based */, int t) {
  const double pi = 3.14159265358979323846;
  return sin(2.0 * pi * (double)k * (double)t / P->act_period + P->act_phase);
}

/* a_g(t) = sum_{k=1..K} w[g][k-1] sin(2 pi k t / P + phi) */
double orc_actuation(const orc_params* P, const double* wact, int g, int t) {
  double a = 0.0;
  for (int k = 1; k <= P->n_basis; k++) a += wact[g * P->n_basis + (k - 1)] * act_basis(P, k, t);
  return a;
}

/* ------------------------------------------------------------------ */
/* closed-loop controller (the neural-network controllers of Section   */
/* 4.1: sensors of the current state -> a small MLP -> the actuation   */
/* of every group, evaluated at every step and differentiated with it) */
/* ------------------------------------------------------------------ */

/* inputs u, n_in = K + 2 d G of them: the K time-basis values sin(2 pi k t / P + phi),
   then for each group g the offset of the group's centre of mass from the whole body's
   (d values) and the group's mean velocity (d values); a group without particles reads
   zeros.  hidden h = tanh(W1 u + b1) (H units); output a_g = scale tanh(W2 h + b2)_g.
   theta = [W1 (H x n_in, row-major) | b1 (H) | W2 (G x H, row-major) | b2 (G)]. */
int orc_ctrl_n_inputs(const orc_params* P) { return P->n_basis + 2 * P->dim * P->n_groups; }

int64_t orc_ctrl_n_params(const orc_params* P) {
  int64_t H = P->ctrl_hidden, I = orc_ctrl_n_inputs(P), G = P->n_groups;
  return H * I + H + G * H + G;
}

/* the sensors of state (x, v): u[n_in] and the group sizes cnt[G] */
static void ctrl_sensors(const orc_params* P, int64_t np, int t, const double* x,
                         const double* v, const int32_t* grp, double* u, double* cnt) {
  int d = P->dim, G = P->n_groups, K = P->n_basis;
  double com[3] = {0, 0, 0}, sx[ORC_CTRL_MAX_GROUPS][3], sv[ORC_CTRL_MAX_GROUPS][3];
  for (int g = 0; g < G; g++) {
    cnt[g] = 0.0;
    for (int a = 0; a < 3; a++) sx[g][a] = sv[g][a] = 0.0;
  }
  for (int64_t p = 0; p < np; p++) {
    int g = grp ? grp[p] : -1;
    for (int a = 0; a < d; a++) com[a] += x[a * np + p];
    if (g < 0 || g >= G) continue;
    cnt[g] += 1.0;
    for (int a = 0; a < d; a++) {
      sx[g][a] += x[a * np + p];
      sv[g][a] += v[a * np + p];
    }
  }
  for (int a = 0; a < d; a++) com[a] /= (double)np;
  for (int k = 1; k <= K; k++) u[k - 1] = act_basis(P, k, t);
  for (int g = 0; g < G; g++)
    for (int a = 0; a < d; a++) {
      double* ug = u + K + g * 2 * d;
      ug[a] = cnt[g] > 0.0 ? sx[g][a] / cnt[g] - com[a] : 0.0;
      ug[d + a] = cnt[g] > 0.0 ? sv[g][a] / cnt[g] : 0.0;
    }
}

/* hidden layer h[H] and actuation a[G] from the inputs u */
static void ctrl_mlp(const orc_params* P, const double* th, const double* u, double* h,
                     double* a) {
  int H = P->ctrl_hidden, I = orc_ctrl_n_inputs(P), G = P->n_groups;
  const double *W1 = th, *b1 = th + H * I, *W2 = b1 + H, *b2 = W2 + G * H;
  for (int j = 0; j < H; j++) {
    double z = b1[j];
    for (int i = 0; i < I; i++) z += W1[j * I + i] * u[i];
    h[j] = tanh(z);
  }
  for (int g = 0; g < G; g++) {
    double z = b2[g];
    for (int j = 0; j < H; j++) z += W2[g * H + j] * h[j];
    a[g] = P->ctrl_scale * tanh(z);
  }
}

/* the actuation of every group at step t: the open-loop sine series, or the controller
   evaluated on state (x, v) */
static int group_actuation(const orc_params* P, int64_t np, int t, const double* x,
                           const double* v, const int32_t* grp, const double* wact,
                           double* act) {
  for (int g = 0; g < ORC_CTRL_MAX_GROUPS; g++) act[g] = 0.0;
  if (P->n_groups <= 0 || !grp || !wact) return ORC_OK;
  if (P->n_groups > ORC_CTRL_MAX_GROUPS) return ORC_ERR_ARG;
  if (P->ctrl_hidden <= 0) {
    for (int g = 0; g < P->n_groups; g++) act[g] = orc_actuation(P, wact, g, t);
    return ORC_OK;
  }
  if (P->ctrl_hidden > ORC_CTRL_MAX_HIDDEN) return ORC_ERR_ARG;
  double u[ORC_CTRL_MAX_INPUTS], h[ORC_CTRL_MAX_HIDDEN], cnt[ORC_CTRL_MAX_GROUPS];
  ctrl_sensors(P, np, t, x, v, grp, u, cnt);
  ctrl_mlp(P, wact, u, h, act);
  return ORC_OK;
}

/* controller output and inputs at state (x, v), for the pins */
int orc_controller(const orc_params* P, const double* theta, int64_t np, int t,
                   const double* x, const double* v, const int32_t* grp, double* act,
                   double* u_out) {
  if (P->ctrl_hidden <= 0 || P->ctrl_hidden > ORC_CTRL_MAX_HIDDEN || P->n_groups <= 0 ||
      P->n_groups > ORC_CTRL_MAX_GROUPS)
    return ORC_ERR_ARG;
  double u[ORC_CTRL_MAX_INPUTS], h[ORC_CTRL_MAX_HIDDEN], cnt[ORC_CTRL_MAX_GROUPS];
  double a[ORC_CTRL_MAX_GROUPS];
  ctrl_sensors(P, np, t, x, v, grp, u, cnt);
  ctrl_mlp(P, theta, u, h, a);
  for (int g = 0; g < P->n_groups; g++) act[g] = a[g];
  for (int i = 0; i < orc_ctrl_n_inputs(P); i++) u_out[i] = u[i];
  return ORC_OK;
}

/* Adjoint of the controller at step t given abar[g] = dL/da_g: accumulates dL/dtheta into
   thbar and adds the sensor terms to the adjoint of the state, xb and vb (every particle
   moves its group's centre of mass by 1/N_g of its displacement and the body's by 1/N). */
static void ctrl_adjoint(const orc_params* P, int64_t np, int t, const double* x,
                         const double* v, const int32_t* grp, const double* th,
                         const double* abar, double* thbar, double* xb, double* vb) {
  int d = P->dim, H = P->ctrl_hidden, I = orc_ctrl_n_inputs(P), G = P->n_groups,
      K = P->n_basis;
  double u[ORC_CTRL_MAX_INPUTS], h[ORC_CTRL_MAX_HIDDEN], cnt[ORC_CTRL_MAX_GROUPS];
  double a[ORC_CTRL_MAX_GROUPS], z2b[ORC_CTRL_MAX_GROUPS], z1b[ORC_CTRL_MAX_HIDDEN];
  double ub[ORC_CTRL_MAX_INPUTS];
  ctrl_sensors(P, np, t, x, v, grp, u, cnt);
  ctrl_mlp(P, th, u, h, a);
  const double *W1 = th, *W2 = th + H * I + H;
  double *W1b = thbar, *b1b = thbar + H * I, *W2b = b1b + H, *b2b = W2b + G * H;
  for (int g = 0; g < G; g++) {
    double y = a[g] / P->ctrl_scale; /* tanh(z2) */
    z2b[g] = abar[g] * P->ctrl_scale * (1.0 - y * y);
    b2b[g] += z2b[g];
    for (int j = 0; j < H; j++) W2b[g * H + j] += z2b[g] * h[j];
  }
  for (int j = 0; j < H; j++) {
    double hb = 0.0;
    for (int g = 0; g < G; g++) hb += W2[g * H + j] * z2b[g];
    z1b[j] = hb * (1.0 - h[j] * h[j]);
    b1b[j] += z1b[j];
    for (int i = 0; i < I; i++) W1b[j * I + i] += z1b[j] * u[i];
  }
  for (int i = 0; i < I; i++) {
    ub[i] = 0.0;
    for (int j = 0; j < H; j++) ub[i] += W1[j * I + i] * z1b[j];
  }
  /* u_xg = mean_{p in g} x_p - mean_p x_p ; u_vg = mean_{p in g} v_p */
  double body[3] = {0, 0, 0};
  for (int g = 0; g < G; g++)
    if (cnt[g] > 0.0)
      for (int a2 = 0; a2 < d; a2++) body[a2] += ub[K + g * 2 * d + a2];
  for (int64_t p = 0; p < np; p++) {
    int g = grp ? grp[p] : -1;
    for (int a2 = 0; a2 < d; a2++) xb[a2 * np + p] -= body[a2] / (double)np;
    if (g < 0 || g >= G) continue;
    for (int a2 = 0; a2 < d; a2++) {
      xb[a2 * np + p] += ub[K + g * 2 * d + a2] / cnt[g];
      vb[a2 * np + p] += ub[K + g * 2 * d + d + a2] / cnt[g];
    }
  }
}

/* ------------------------------------------------------------------ */
/* Kirchhoff stress and its adjoint                                    */
/* ------------------------------------------------------------------ */

/* the constitutive model of particle p */
static int material_of(const orc_params* P, int64_t p) {
  return P->material == ORC_MIXED ? P->particle_material[p] : P->material;
}

static int kirchhoff_m(const orc_params* P, int material, const mat3 F, double mu, double la,
                       double act, int axis, mat3 tau) {
  int d = P->dim;
  mzero(tau);
  if (material == ORC_FIXED_COROTATED) {
    mat3 R, S, FmR, Ft;
    double J = mdet(d, F);
    if (d == 2) {
      double Fl[4] = {F[0][0], F[0][1], F[1][0], F[1][1]}, Rl[4];
      int rc = orc_polar(2, Fl, Rl, NULL);
      if (rc) return rc;
      mzero(R);
      R[0][0] = Rl[0];
      R[0][1] = Rl[1];
      R[1][0] = Rl[2];
      R[1][1] = Rl[3];
    } else {
      mat3 V;
      double sig[3];
      int rc = polar3_full(F, R, S, V, sig);
      if (rc) return rc;
    }
    mzero(FmR);
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) FmR[i][j] = F[i][j] - R[i][j];
    mtrans(d, F, Ft);
    mmul(d, FmR, Ft, tau);
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) tau[i][j] *= 2.0 * mu;
    for (int i = 0; i < d; i++) tau[i][i] += la * (J - 1.0) * J;
  } else if (material == ORC_NEO_HOOKEAN) {
    double J = mdet(d, F);
    if (!(J > 0.0)) return ORC_ERR_DOMAIN;
    mat3 Ft, FFt;
    mtrans(d, F, Ft);
    mmul(d, F, Ft, FFt);
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) tau[i][j] = mu * (FFt[i][j] - (i == j ? 1.0 : 0.0));
    for (int i = 0; i < d; i++) tau[i][i] += la * log(J);
  } else if (material == ORC_LIQUID) {
    double J = mdet(d, F);
    if (!(J > 0.0)) return ORC_ERR_DOMAIN;
    double kap = la + 2.0 * mu / d;
    double g = J - pow(J, 1.0 - ORC_LIQUID_GAMMA);
    for (int i = 0; i < d; i++) tau[i][i] = kap * g;
  } else if (material != ORC_NO_ELASTICITY) {
    return ORC_ERR_ARG;
  }
  if (act != 0.0) {
    double fe[3] = {0, 0, 0}; /* F e, e the unit vector of the group's axis */
    for (int i = 0; i < d; i++) fe[i] = F[i][axis];
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) tau[i][j] += act * fe[i] * fe[j];
  }
  return ORC_OK;
}

/* exported: Kirchhoff stress of one particle (F row-major d x d) */
int orc_kirchhoff(const orc_params* P, const double* Fin, double mu, double la, double act,
                  int axis, double* tau_out) {
  int d = P->dim;
  mat3 F, tau;
  mzero(F);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) F[i][j] = Fin[i * d + j];
  int rc = kirchhoff_m(P, P->material, F, mu, la, act, axis, tau);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) tau_out[i * d + j] = tau[i][j];
  return rc;
}

/* adjoint of kirchhoff(): given taubar, accumulate Fbar, mubar, labar, abar */
static int kirchhoff_adjoint_m(const orc_params* P, int material, const mat3 F, double mu,
                               double la, double act, int axis, const mat3 tb, mat3 Fbar,
                               double* mubar, double* labar, double* abar) {
  int d = P->dim;
  mat3 tsum; /* taubar + taubar^T */
  mzero(tsum);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) tsum[i][j] = tb[i][j] + tb[j][i];
  double trtb = mtrace(d, tb);
  if (material == ORC_FIXED_COROTATED) {
    mat3 R, S, Ft;
    double J = mdet(d, F);
    if (d == 2) {
      double Fl[4] = {F[0][0], F[0][1], F[1][0], F[1][1]}, Rl[4];
      int rc = orc_polar(2, Fl, Rl, NULL);
      if (rc) return rc;
      mzero(R);
      R[0][0] = Rl[0];
      R[0][1] = Rl[1];
      R[1][0] = Rl[2];
      R[1][1] = Rl[3];
    } else {
      mat3 V;
      double sig[3];
      int rc = polar3_full(F, R, S, V, sig);
      if (rc) return rc;
    }
    /* tau1 = 2 mu F F^T - 2 mu R F^T */
    mat3 A1, tbt, A2, Rbar, cof, FmR, FmRFt;
    mmul(d, tsum, F, A1);          /* (tb + tb^T) F */
    mtrans(d, tb, tbt);
    mmul(d, tbt, R, A2);           /* tb^T R */
    mmul(d, tb, F, Rbar);          /* tb F */
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) {
        Fbar[i][j] += 2.0 * mu * A1[i][j] - 2.0 * mu * A2[i][j];
        Rbar[i][j] *= -2.0 * mu;
      }
    int rc = polar_adjoint(d, F, Rbar, Fbar);
    if (rc) return rc;
    /* tau2 = la (J^2 - J) I */
    mcof(d, F, cof);
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) Fbar[i][j] += la * (2.0 * J - 1.0) * trtb * cof[i][j];
    mzero(FmR);
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) FmR[i][j] = F[i][j] - R[i][j];
    mtrans(d, F, Ft);
    mmul(d, FmR, Ft, FmRFt);
    *mubar += 2.0 * mdot(d, tb, FmRFt);
    *labar += trtb * (J - 1.0) * J;
  } else if (material == ORC_NEO_HOOKEAN) {
    double J = mdet(d, F);
    if (!(J > 0.0)) return ORC_ERR_DOMAIN;
    mat3 A1, cof, Ft, FFt;
    mmul(d, tsum, F, A1);
    mcof(d, F, cof); /* F^{-T} = cof / J */
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) Fbar[i][j] += mu * A1[i][j] + la * trtb * cof[i][j] / J;
    mtrans(d, F, Ft);
    mmul(d, F, Ft, FFt);
    for (int i = 0; i < d; i++) FFt[i][i] -= 1.0;
    *mubar += mdot(d, tb, FFt);
    *labar += trtb * log(J);
  } else if (material == ORC_LIQUID) {
    /* tau = kappa g(J) I, g(J) = J - J^(1-gamma), g'(J) = 1 + (gamma - 1) J^-gamma,
       dJ/dF = cof F; kappa = la + 2 mu / d */
    double J = mdet(d, F);
    if (!(J > 0.0)) return ORC_ERR_DOMAIN;
    double kap = la + 2.0 * mu / d;
    double g = J - pow(J, 1.0 - ORC_LIQUID_GAMMA);
    double gp = 1.0 + (ORC_LIQUID_GAMMA - 1.0) * pow(J, -ORC_LIQUID_GAMMA);
    mat3 cof;
    mcof(d, F, cof);
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) Fbar[i][j] += trtb * kap * gp * cof[i][j];
    double kbar = trtb * g;
    *labar += kbar;
    *mubar += 2.0 * kbar / d;
  }
  if (act != 0.0 || abar) {
    double fe[3] = {0, 0, 0};
    for (int i = 0; i < d; i++) fe[i] = F[i][axis];
    double ab = 0.0;
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++) ab += fe[i] * tb[i][j] * fe[j];
    if (abar) *abar += ab;
    /* d/dF [act (F e)(F e)^T] : Fbar[:, axis] += act (tb + tb^T) F e */
    for (int i = 0; i < d; i++) {
      double s = 0.0;
      for (int j = 0; j < d; j++) s += tsum[i][j] * fe[j];
      Fbar[i][axis] += act * s;
    }
  }
  return ORC_OK;
}

/* exported: stress adjoint of one particle (row-major d x d); Fbar is overwritten */
int orc_kirchhoff_adjoint(const orc_params* P, const double* Fin, double mu, double la, double act,
                          int axis, const double* tbar_in, double* Fbar_out, double* mubar,
                          double* labar, double* abar) {
  int d = P->dim;
  mat3 F, tb, Fb;
  mzero(F);
  mzero(tb);
  mzero(Fb);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      F[i][j] = Fin[i * d + j];
      tb[i][j] = tbar_in[i * d + j];
    }
  *mubar = *labar = *abar = 0.0;
  int rc = kirchhoff_adjoint_m(P, P->material, F, mu, la, act, axis, tb, Fb, mubar, labar, abar);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) Fbar_out[i * d + j] = Fb[i][j];
  return rc;
}

/* ------------------------------------------------------------------ */
/* one forward step                                                    */
/* ------------------------------------------------------------------ */

static double particle_volume(const orc_params* P) {
  return pow(0.5 / (double)P->n_grid, (double)P->dim);
}

static int is_wall(const orc_params* P, const int idx[3]) {
  for (int a = 0; a < P->dim; a++)
    if (idx[a] < P->wall_cells || idx[a] >= P->n_grid - P->wall_cells) return 1;
  return 0;
}

/* actuation of particle p from its group's value gact[g] (group_actuation) */
static double particle_act(const orc_params* P, const int32_t* grp, const double* gact,
                           int64_t p, int* axis) {
  *axis = 0;
  if (P->n_groups <= 0 || !grp) return 0.0;
  int g = grp[p];
  if (g < 0 || g >= P->n_groups) return 0.0;
  *axis = g % P->dim;
  return gact[g];
}

/* constants of one step shared by the per-particle helpers */
typedef struct {
  double dx, inv_dx2, vol, m, kappa;
  int nst;
} step_consts;

static step_consts consts_of(const orc_params* P) {
  step_consts k;
  int n = P->n_grid;
  k.dx = 1.0 / n;
  k.inv_dx2 = 1.0 / (k.dx * k.dx);
  k.vol = particle_volume(P);
  k.m = P->rho * k.vol;
  k.kappa = -P->dt * k.vol * 4.0 / (k.dx * k.dx);
  k.nst = (int)ipow(3, P->dim);
  return k;
}

/* P2G of particle p: its stress, the affine matrix A = kappa tau + m C, and the scatter of
   mass and momentum into (gm, gp) */
static int p2g_particle(const orc_params* P, const step_consts* K, int64_t np, int64_t p,
                        const double* x, const double* v, const double* C, const double* F,
                        const double* mu, const double* la, const int32_t* grp,
                        const double* gact, double* gm, double* gp) {
  int d = P->dim, n = P->n_grid;
  double m = K->m, kappa = K->kappa;
  double xp[3] = {0, 0, 0};
  for (int a = 0; a < d; a++) xp[a] = x[a * np + p];
  stencil s;
  int rc = make_stencil(P, xp, &s);
  if (rc) return rc;
  mat3 Fp, Cp, tau, A;
  load_mat(d, F, np, p, Fp);
  load_mat(d, C, np, p, Cp);
  int axis;
  double act = particle_act(P, grp, gact, p, &axis);
  rc = kirchhoff_m(P, material_of(P, p), Fp, mu[p], la[p], act, axis, tau);
  if (rc) return rc;
  mzero(A);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) A[i][j] = kappa * tau[i][j] + m * Cp[i][j];
  for (int o = 0; o < K->nst; o++) {
    int off[3], idx[3];
    double W, gW[3], dpos[3];
    offset_of(d, o, off);
    stencil_eval(d, n, &s, off, &W, gW, dpos, idx);
    int64_t ni = node_index(d, n, idx);
    gm[ni] += W * m;
    for (int a = 0; a < d; a++) {
      double Ad = 0.0;
      for (int b = 0; b < d; b++) Ad += A[a][b] * dpos[b];
      gp[ni * d + a] += W * (m * v[a * np + p] + Ad);
    }
  }
  return ORC_OK;
}

#ifdef _OPENMP
/* ------------------------------------------------------------------ */
/* OpenMP build (liboracle_omp.so, the all-cores CPU baseline): the same per-particle      */
/* helpers run over the particles in parallel; a scatter goes into a private grid per     */
/* thread, and the private grids are summed node by node in thread order over the box    */
/* the stencils touch.  The serial build (no -fopenmp) never compiles this section.       */
/* ------------------------------------------------------------------ */
#include <omp.h>

/* node box [lo, hi] covering every particle's 3^d stencil (clipped to the grid) */
static int64_t stencil_box(const orc_params* P, int64_t np, const double* x, int lo[3],
                           int hi[3]) {
  int d = P->dim, n = P->n_grid;
  int64_t vol = 1;
  for (int a = 0; a < 3; a++) lo[a] = hi[a] = 0;
  for (int a = 0; a < d; a++) {
    double bmin = (double)n, bmax = -1.0;
    for (int64_t p = 0; p < np; p++) {
      double b = floor(x[a * np + p] * (double)n - 0.5);
      if (b < bmin) bmin = b;
      if (b > bmax) bmax = b;
    }
    lo[a] = bmin < 0.0 ? 0 : (bmin > n - 1 ? n - 1 : (int)bmin);
    hi[a] = bmax + 2.0 > n - 1 ? n - 1 : (bmax + 2.0 < 0.0 ? 0 : (int)bmax + 2);
    if (hi[a] < lo[a]) return 0;
    vol *= hi[a] - lo[a] + 1;
  }
  return vol;
}

static void box_node(int d, const int lo[3], const int hi[3], int64_t l, int idx[3]) {
  idx[0] = idx[1] = idx[2] = 0;
  for (int a = d - 1; a >= 0; a--) {
    int64_t e = hi[a] - lo[a] + 1;
    idx[a] = lo[a] + (int)(l % e);
    l /= e;
  }
}

/* out[node * w + c] = sum over threads (in thread order) of priv[tid][node * w + c], over
   the box's nodes; out is zero elsewhere */
static void reduce_private(const orc_params* P, int nth, const double* priv, int64_t stride,
                           int w, const int lo[3], const int hi[3], int64_t bvol, double* out) {
  int d = P->dim, n = P->n_grid;
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < bvol; l++) {
    int idx[3];
    box_node(d, lo, hi, l, idx);
    int64_t ni = node_index(d, n, idx);
    for (int c = 0; c < w; c++) {
      double s = 0.0;
      for (int t = 0; t < nth; t++) s += priv[(int64_t)t * stride + ni * w + c];
      out[ni * w + c] = s;
    }
  }
}

static int p2g_omp(const orc_params* P, int64_t np, const double* x, const double* v,
                   const double* C, const double* F, const double* mu, const double* la,
                   const int32_t* grp, const double* gact, double* gm, double* gp) {
  int d = P->dim;
  int64_t nn = ipow(P->n_grid, d);
  step_consts K = consts_of(P);
  int nth = omp_get_max_threads();
  int lo[3], hi[3];
  int64_t bvol = stencil_box(P, np, x, lo, hi);
  double* pm = (double*)calloc((size_t)nth * nn, sizeof(double));
  double* pp = (double*)calloc((size_t)nth * nn * d, sizeof(double));
  if (!pm || !pp) {
    free(pm);
    free(pp);
    return ORC_ERR_MEM;
  }
  int err = ORC_OK;
#pragma omp parallel num_threads(nth)
  {
    int tid = omp_get_thread_num();
#pragma omp for schedule(static)
    for (int64_t p = 0; p < np; p++) {
      int rc = p2g_particle(P, &K, np, p, x, v, C, F, mu, la, grp, gact, pm + (int64_t)tid * nn,
                            pp + (int64_t)tid * nn * d);
      if (rc) {
#pragma omp atomic write
        err = rc;
      }
    }
  }
  if (!err) {
    reduce_private(P, nth, pm, nn, 1, lo, hi, bvol, gm);
    reduce_private(P, nth, pp, nn * d, d, lo, hi, bvol, gp);
  }
  free(pm);
  free(pp);
  return err;
}
#endif

/* threads the particle loops use: 1 in the serial build; in the OpenMP build n > 0 sets
   the count, and the current count is returned */
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* P2G (Appendix D "p2g"): scatter mass and APIC/MLS momentum.  gm[n^d] and
   gp[n^d * d] are overwritten (cleared first, "clear_grid"). */
int orc_p2g(const orc_params* P, int64_t np, int t, const double* x, const double* v,
            const double* C, const double* F, const double* mu, const double* la,
            const int32_t* grp, const double* wact, double* gm, double* gp) {
  int d = P->dim, n = P->n_grid;
  int64_t nn = ipow(n, d);
  memset(gm, 0, sizeof(double) * nn);
  memset(gp, 0, sizeof(double) * nn * d);
  double gact[ORC_CTRL_MAX_GROUPS];
  int rca = group_actuation(P, np, t, x, v, grp, wact, gact);
  if (rca) return rca;
#ifdef _OPENMP
  if (omp_get_max_threads() > 1) return p2g_omp(P, np, x, v, C, F, mu, la, grp, gact, gm, gp);
#endif
  step_consts K = consts_of(P);
  for (int64_t p = 0; p < np; p++) {
    int rc = p2g_particle(P, &K, np, p, x, v, C, F, mu, la, grp, gact, gm, gp);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* grid_op (Appendix D): normalise momentum, add gravity, sticky walls. */
void orc_grid_update(const orc_params* P, const double* gm, const double* gp, double* gu) {
  int d = P->dim, n = P->n_grid;
  int64_t nn = ipow(n, d);
#pragma omp parallel for schedule(static)
  for (int64_t ni = 0; ni < nn; ni++) {
    int idx[3] = {0, 0, 0};
    int64_t r = ni;
    for (int a = d - 1; a >= 0; a--) {
      idx[a] = (int)(r % n);
      r /= n;
    }
    int active = gm[ni] > 0.0 && !is_wall(P, idx);
    for (int a = 0; a < d; a++)
      gu[ni * d + a] = active ? gp[ni * d + a] / gm[ni] + P->dt * P->gravity[a] : 0.0;
  }
}

/* G2P of particle p (Appendix D "g2p"): gather velocity and affine matrix, advect, update F */
static int g2p_particle(const orc_params* P, int64_t np, int64_t p, const double* x,
                        const double* F, const double* gu, double* x1, double* v1, double* C1,
                        double* F1) {
  int d = P->dim, n = P->n_grid;
  double dx = 1.0 / n;
  int nst = (int)ipow(3, d);
  double xp[3] = {0, 0, 0};
  for (int a = 0; a < d; a++) xp[a] = x[a * np + p];
  stencil s;
  int rc = make_stencil(P, xp, &s);
  if (rc) return rc;
  double vn[3] = {0, 0, 0};
  mat3 B;
  mzero(B);
  for (int o = 0; o < nst; o++) {
    int off[3], idx[3];
    double W, gW[3], dpos[3];
    offset_of(d, o, off);
    stencil_eval(d, n, &s, off, &W, gW, dpos, idx);
    int64_t ni = node_index(d, n, idx);
    for (int a = 0; a < d; a++) {
      double ui = gu[ni * d + a];
      vn[a] += W * ui;
      for (int b = 0; b < d; b++) B[a][b] += W * ui * dpos[b];
    }
  }
  mat3 Cn, Fp, G, Fn;
  mzero(Cn);
  for (int a = 0; a < d; a++)
    for (int b = 0; b < d; b++) Cn[a][b] = 4.0 / (dx * dx) * B[a][b];
  load_mat(d, F, np, p, Fp);
  meye(d, G);
  for (int a = 0; a < d; a++)
    for (int b = 0; b < d; b++) G[a][b] += P->dt * Cn[a][b];
  mmul(d, G, Fp, Fn);
  for (int a = 0; a < d; a++) {
    x1[a * np + p] = xp[a] + P->dt * vn[a];
    v1[a * np + p] = vn[a];
  }
  store_mat(d, C1, np, p, Cn);
  store_mat(d, F1, np, p, Fn);
  return ORC_OK;
}

/* G2P (Appendix D "g2p") of every particle (independent: parallel in the OpenMP build) */
int orc_g2p(const orc_params* P, int64_t np, const double* x, const double* F, const double* gu,
            double* x1, double* v1, double* C1, double* F1) {
  int err = ORC_OK;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < np; p++) {
    int rc = g2p_particle(P, np, p, x, F, gu, x1, v1, C1, F1);
    if (rc) {
#pragma omp atomic write
      err = rc;
    }
  }
  return err;
}

typedef struct {
  double *gm, *gp, *gu;
} grid_bufs;

static int alloc_grid(const orc_params* P, grid_bufs* g) {
  int64_t nn = ipow(P->n_grid, P->dim);
  g->gm = (double*)calloc(nn, sizeof(double));
  g->gp = (double*)calloc(nn * P->dim, sizeof(double));
  g->gu = (double*)calloc(nn * P->dim, sizeof(double));
  if (!g->gm || !g->gp || !g->gu) return ORC_ERR_MEM;
  return ORC_OK;
}

static void free_grid(grid_bufs* g) {
  free(g->gm);
  free(g->gp);
  free(g->gu);
}

/* one full step s -> s+1 (Appendix D "advance") */
int orc_step(const orc_params* P, int64_t np, int t, const double* x, const double* v,
             const double* C, const double* F, const double* mu, const double* la,
             const int32_t* grp, const double* wact, double* x1, double* v1, double* C1,
             double* F1) {
  grid_bufs g;
  int rc = alloc_grid(P, &g);
  if (!rc) rc = orc_p2g(P, np, t, x, v, C, F, mu, la, grp, wact, g.gm, g.gp);
  if (!rc) orc_grid_update(P, g.gm, g.gp, g.gu);
  if (!rc) rc = orc_g2p(P, np, x, F, g.gu, x1, v1, C1, F1);
  free_grid(&g);
  return rc;
}

/* T steps; states laid out [t][block] with block = x(d n) v(d n) C(d^2 n) F(d^2 n).
   states[0] must hold the initial state on entry. */
int orc_run(const orc_params* P, int64_t np, int T, const double* mu, const double* la,
            const int32_t* grp, const double* wact, double* states) {
  int d = P->dim;
  int64_t blk = (int64_t)(2 * d + 2 * d * d) * np;
  for (int t = 0; t < T; t++) {
    const double* s0 = states + (int64_t)t * blk;
    double* s1 = states + (int64_t)(t + 1) * blk;
    int rc = orc_step(P, np, t, s0, s0 + d * np, s0 + 2 * d * np, s0 + (2 * d + d * d) * np, mu,
                      la, grp, wact, s1, s1 + d * np, s1 + 2 * d * np,
                      s1 + (2 * d + d * d) * np);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* adjoint of one step (Appendix D.1 "advance_grad")                    */
/* ------------------------------------------------------------------ */

/* g2p.grad of particle p: the adjoint of x' = x + dt v' and F' = (I + dt C') F given the
   adjoint of state s+1, with v' and C' gathered from the grid velocity gu.  Writes xb, Fb of
   particle p and scatters the grid-velocity adjoint into gub. */
static int g2p_grad_particle(const orc_params* P, const step_consts* K, int64_t np, int64_t p,
                             const double* x, const double* F, const double* gu,
                             const double* xb1, const double* vb1, const double* Cb1,
                             const double* Fb1, double* gub, double* xb, double* Fb) {
  int d = P->dim, n = P->n_grid, nst = K->nst;
  double inv_dx2 = K->inv_dx2;
  double xp[3] = {0, 0, 0};
  for (int a = 0; a < d; a++) xp[a] = x[a * np + p];
  stencil s;
  int rc = make_stencil(P, xp, &s);
  if (rc) return rc;
  /* recompute C' of this particle */
  mat3 B;
  mzero(B);
  for (int o = 0; o < nst; o++) {
    int off[3], idx[3];
    double W, gW[3], dpos[3];
    offset_of(d, o, off);
    stencil_eval(d, n, &s, off, &W, gW, dpos, idx);
    int64_t ni = node_index(d, n, idx);
    for (int a = 0; a < d; a++)
      for (int b = 0; b < d; b++) B[a][b] += W * gu[ni * d + a] * dpos[b];
  }
  mat3 Cn, Fp, Fb1p, Cb1p, G, Gt, Fbp, Ct, Fpt, FbFt;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) Cn[a][b] = 4.0 * inv_dx2 * B[a][b];
  load_mat(d, F, np, p, Fp);
  load_mat(d, Fb1, np, p, Fb1p);
  load_mat(d, Cb1, np, p, Cb1p);
  /* x' = x + dt v'  ->  xbar += xbar', vtilde = vbar' + dt xbar' */
  double xbp[3] = {0, 0, 0}, vt[3] = {0, 0, 0};
  for (int a = 0; a < d; a++) {
    xbp[a] = xb1[a * np + p];
    vt[a] = vb1[a * np + p] + P->dt * xb1[a * np + p];
  }
  /* F' = (I + dt C') F  ->  Fbar = (I + dt C')^T Fbar', Ctilde = Cbar' + dt Fbar' F^T */
  meye(d, G);
  for (int a = 0; a < d; a++)
    for (int b = 0; b < d; b++) G[a][b] += P->dt * Cn[a][b];
  mtrans(d, G, Gt);
  mmul(d, Gt, Fb1p, Fbp);
  mtrans(d, Fp, Fpt);
  mmul(d, Fb1p, Fpt, FbFt);
  mzero(Ct);
  for (int a = 0; a < d; a++)
    for (int b = 0; b < d; b++) Ct[a][b] = Cb1p[a][b] + P->dt * FbFt[a][b];
  /* v' = sum W u_i ; C' = (4/dx^2) sum W u_i dpos^T */
  for (int o = 0; o < nst; o++) {
    int off[3], idx[3];
    double W, gW[3], dpos[3];
    offset_of(d, o, off);
    stencil_eval(d, n, &s, off, &W, gW, dpos, idx);
    int64_t ni = node_index(d, n, idx);
    const double* u = gu + ni * d;
    double Wbar = 0.0;
    for (int a = 0; a < d; a++) {
      double Cd = 0.0;
      for (int b = 0; b < d; b++) Cd += Ct[a][b] * dpos[b];
      gub[ni * d + a] += W * vt[a] + 4.0 * inv_dx2 * W * Cd;
      Wbar += vt[a] * u[a] + 4.0 * inv_dx2 * u[a] * Cd;
    }
    for (int b = 0; b < d; b++) {
      double CtU = 0.0; /* (Ctilde^T u)_b */
      for (int a = 0; a < d; a++) CtU += Ct[a][b] * u[a];
      xbp[b] += Wbar * gW[b] - 4.0 * inv_dx2 * W * CtU;
    }
  }
  for (int a = 0; a < d; a++) xb[a * np + p] = xbp[a];
  store_mat(d, Fb, np, p, Fbp);
  return ORC_OK;
}

/* p2g.grad of particle p and its stress / actuation adjoint, given the momentum and mass
   adjoints (gpb, gmb) of the grid.  Adds to xb, Fb, mubar, labar of particle p, writes vb, Cb,
   and accumulates the actuation adjoint into wbar (open loop) or gabar (closed loop). */
static int p2g_grad_particle(const orc_params* P, const step_consts* K, int64_t np, int t,
                             int64_t p, const double* x, const double* v, const double* C,
                             const double* F, const double* mu, const double* la,
                             const int32_t* grp, const double* wact, const double* gact,
                             const double* gpb, const double* gmb, double* xb, double* vb,
                             double* Cb, double* Fb, double* mubar, double* labar, double* wbar,
                             double* gabar) {
  int d = P->dim, n = P->n_grid, nst = K->nst;
  double m = K->m, kappa = K->kappa;
  double xp[3] = {0, 0, 0}, vp[3] = {0, 0, 0};
  for (int a = 0; a < d; a++) {
    xp[a] = x[a * np + p];
    vp[a] = v[a * np + p];
  }
  stencil s;
  int rc = make_stencil(P, xp, &s);
  if (rc) return rc;
  mat3 Fp, Cp, tau, A, Abar, Fbp;
  load_mat(d, F, np, p, Fp);
  load_mat(d, C, np, p, Cp);
  int axis;
  double act = particle_act(P, grp, gact, p, &axis);
  rc = kirchhoff_m(P, material_of(P, p), Fp, mu[p], la[p], act, axis, tau);
  if (rc) return rc;
  mzero(A);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) A[i][j] = kappa * tau[i][j] + m * Cp[i][j];
  mzero(Abar);
  double vbp[3] = {0, 0, 0}, xbp[3] = {0, 0, 0};
  for (int o = 0; o < nst; o++) {
    int off[3], idx[3];
    double W, gW[3], dpos[3];
    offset_of(d, o, off);
    stencil_eval(d, n, &s, off, &W, gW, dpos, idx);
    int64_t ni = node_index(d, n, idx);
    const double* pb = gpb + ni * d;
    /* p_i += W (m v + A dpos) ; m_i += W m */
    double Wbar = m * gmb[ni];
    for (int a = 0; a < d; a++) {
      double Ad = 0.0;
      for (int b = 0; b < d; b++) Ad += A[a][b] * dpos[b];
      Wbar += pb[a] * (m * vp[a] + Ad);
      vbp[a] += W * m * pb[a];
      for (int b = 0; b < d; b++) Abar[a][b] += W * pb[a] * dpos[b];
    }
    for (int b = 0; b < d; b++) {
      double AtP = 0.0; /* (A^T pbar)_b */
      for (int a = 0; a < d; a++) AtP += A[a][b] * pb[a];
      xbp[b] += Wbar * gW[b] - W * AtP;
    }
  }
  /* A = kappa tau + m C */
  mat3 tb, Cbp;
  mzero(tb);
  mzero(Cbp);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      tb[i][j] = kappa * Abar[i][j];
      Cbp[i][j] = m * Abar[i][j];
    }
  load_mat(d, Fb, np, p, Fbp);
  double abar = 0.0;
  rc = kirchhoff_adjoint_m(P, material_of(P, p), Fp, mu[p], la[p], act, axis, tb, Fbp, &mubar[p],
                           &labar[p], &abar);
  if (rc) return rc;
  if (P->n_groups > 0 && grp && wact && wbar) {
    int gi = grp[p];
    if (gi >= 0 && gi < P->n_groups) {
      if (P->ctrl_hidden > 0)
        gabar[gi] += abar;
      else
        for (int k = 1; k <= P->n_basis; k++)
          wbar[gi * P->n_basis + (k - 1)] += abar * act_basis(P, k, t);
    }
  }
  for (int a = 0; a < d; a++) {
    xb[a * np + p] += xbp[a];
    vb[a * np + p] = vbp[a];
  }
  store_mat(d, Cb, np, p, Cbp);
  store_mat(d, Fb, np, p, Fbp);
  return ORC_OK;
}

/* grid_op.grad of every node (node-local) */
static void grid_update_adjoint(const orc_params* P, const double* gm, const double* gp,
                                const double* gub, double* gpb, double* gmb) {
  int d = P->dim, n = P->n_grid;
  int64_t nn = ipow(n, d);
#pragma omp parallel for schedule(static)
  for (int64_t ni = 0; ni < nn; ni++) {
    int idx[3] = {0, 0, 0};
    int64_t r = ni;
    for (int a = d - 1; a >= 0; a--) {
      idx[a] = (int)(r % n);
      r /= n;
    }
    if (gm[ni] > 0.0 && !is_wall(P, idx)) {
      double mb = 0.0;
      for (int a = 0; a < d; a++) {
        gpb[ni * d + a] = gub[ni * d + a] / gm[ni];
        mb -= gub[ni * d + a] * gp[ni * d + a] / (gm[ni] * gm[ni]);
      }
      gmb[ni] = mb;
    }
  }
}

#ifdef _OPENMP
/* g2p.grad over the particles in parallel: private grid-velocity adjoints summed in
   thread order */
static int g2p_grad_omp(const orc_params* P, const step_consts* K, int64_t np, const double* x,
                        const double* F, const double* gu, const double* xb1, const double* vb1,
                        const double* Cb1, const double* Fb1, double* gub, double* xb,
                        double* Fb) {
  int d = P->dim;
  int64_t nn = ipow(P->n_grid, d);
  int nth = omp_get_max_threads();
  int lo[3], hi[3];
  int64_t bvol = stencil_box(P, np, x, lo, hi);
  double* pu = (double*)calloc((size_t)nth * nn * d, sizeof(double));
  if (!pu) return ORC_ERR_MEM;
  int err = ORC_OK;
#pragma omp parallel num_threads(nth)
  {
    int tid = omp_get_thread_num();
#pragma omp for schedule(static)
    for (int64_t p = 0; p < np; p++) {
      int rc = g2p_grad_particle(P, K, np, p, x, F, gu, xb1, vb1, Cb1, Fb1,
                                 pu + (int64_t)tid * nn * d, xb, Fb);
      if (rc) {
#pragma omp atomic write
        err = rc;
      }
    }
  }
  if (!err) reduce_private(P, nth, pu, nn * d, d, lo, hi, bvol, gub);
  free(pu);
  return err;
}

/* p2g.grad over the particles in parallel: per-thread actuation-adjoint partial sums,
   added in thread order */
static int p2g_grad_omp(const orc_params* P, const step_consts* K, int64_t np, int t,
                        const double* x, const double* v, const double* C, const double* F,
                        const double* mu, const double* la, const int32_t* grp,
                        const double* wact, const double* gact, const double* gpb,
                        const double* gmb, double* xb, double* vb, double* Cb, double* Fb,
                        double* mubar, double* labar, double* wbar, double* gabar) {
  int nth = omp_get_max_threads();
  int nw = (P->n_groups > 0 && P->ctrl_hidden <= 0) ? P->n_groups * P->n_basis : 0;
  int slot = nw + ORC_CTRL_MAX_GROUPS;
  double* part = (double*)calloc((size_t)nth * slot, sizeof(double));
  if (!part) return ORC_ERR_MEM;
  int err = ORC_OK;
#pragma omp parallel num_threads(nth)
  {
    int tid = omp_get_thread_num();
    double* tw = part + (int64_t)tid * slot;
#pragma omp for schedule(static)
    for (int64_t p = 0; p < np; p++) {
      int rc = p2g_grad_particle(P, K, np, t, p, x, v, C, F, mu, la, grp, wact, gact, gpb, gmb,
                                 xb, vb, Cb, Fb, mubar, labar, wbar ? tw : NULL, tw + nw);
      if (rc) {
#pragma omp atomic write
        err = rc;
      }
    }
  }
  for (int th = 0; th < nth && !err; th++) {
    const double* tw = part + (int64_t)th * slot;
    if (wbar)
      for (int i = 0; i < nw; i++) wbar[i] += tw[i];
    for (int g = 0; g < ORC_CTRL_MAX_GROUPS; g++) gabar[g] += tw[nw + g];
  }
  free(part);
  return err;
}
#endif

/* Given state_s and the adjoint of state_{s+1} (xb1, vb1, Cb1, Fb1), write the
   adjoint of state_s into (xb, vb, Cb, Fb) and accumulate mubar, labar (per
   particle) and wbar (the actuation parameters: w[g * K + k] open-loop, the controller's
   theta closed-loop). */
int orc_step_adjoint(const orc_params* P, int64_t np, int t, const double* x, const double* v,
                     const double* C, const double* F, const double* mu, const double* la,
                     const int32_t* grp, const double* wact, const double* xb1,
                     const double* vb1, const double* Cb1, const double* Fb1, double* xb,
                     double* vb, double* Cb, double* Fb, double* mubar, double* labar,
                     double* wbar) {
  int d = P->dim, n = P->n_grid;
  int64_t nn = ipow(n, d);
  step_consts K;
  K.dx = 1.0 / n;
  K.inv_dx2 = 1.0 / (K.dx * K.dx);
  K.vol = particle_volume(P);
  K.m = P->rho * K.vol;
  K.kappa = -P->dt * K.vol * 4.0 * K.inv_dx2;
  K.nst = (int)ipow(3, d);
  int rc;

  /* recompute the grid of this step: clear_grid, p2g, grid_op */
  grid_bufs g;
  rc = alloc_grid(P, &g);
  if (rc) {
    free_grid(&g);
    return rc;
  }
  double* gub = (double*)calloc(nn * d, sizeof(double)); /* adjoint of grid velocity */
  double* gpb = (double*)calloc(nn * d, sizeof(double)); /* adjoint of grid momentum */
  double* gmb = (double*)calloc(nn, sizeof(double));     /* adjoint of grid mass */
  double gact[ORC_CTRL_MAX_GROUPS], gabar[ORC_CTRL_MAX_GROUPS];
  if (!gub || !gpb || !gmb) {
    rc = ORC_ERR_MEM;
    goto done;
  }
  rc = orc_p2g(P, np, t, x, v, C, F, mu, la, grp, wact, g.gm, g.gp);
  if (rc) goto done;
  orc_grid_update(P, g.gm, g.gp, g.gu);

  /* g2p.grad */
#ifdef _OPENMP
  if (omp_get_max_threads() > 1) {
    rc = g2p_grad_omp(P, &K, np, x, F, g.gu, xb1, vb1, Cb1, Fb1, gub, xb, Fb);
    if (rc) goto done;
  } else
#endif
  {
    for (int64_t p = 0; p < np; p++) {
      rc = g2p_grad_particle(P, &K, np, p, x, F, g.gu, xb1, vb1, Cb1, Fb1, gub, xb, Fb);
      if (rc) goto done;
    }
  }

  /* grid_op.grad */
  grid_update_adjoint(P, g.gm, g.gp, gub, gpb, gmb);

  /* p2g.grad and the stress / actuation adjoint */
  rc = group_actuation(P, np, t, x, v, grp, wact, gact);
  if (rc) goto done;
  for (int gi = 0; gi < ORC_CTRL_MAX_GROUPS; gi++) gabar[gi] = 0.0;
#ifdef _OPENMP
  if (omp_get_max_threads() > 1) {
    rc = p2g_grad_omp(P, &K, np, t, x, v, C, F, mu, la, grp, wact, gact, gpb, gmb, xb, vb, Cb,
                      Fb, mubar, labar, wbar, gabar);
    if (rc) goto done;
  } else
#endif
  {
    for (int64_t p = 0; p < np; p++) {
      rc = p2g_grad_particle(P, &K, np, t, p, x, v, C, F, mu, la, grp, wact, gact, gpb, gmb, xb,
                             vb, Cb, Fb, mubar, labar, wbar, gabar);
      if (rc) goto done;
    }
  }
  /* the controller read this state: its adjoint reaches the weights and, through the
     sensors, the positions and velocities */
  if (P->ctrl_hidden > 0 && P->n_groups > 0 && grp && wact && wbar)
    ctrl_adjoint(P, np, t, x, v, grp, wact, gabar, wbar, xb, vb);
  rc = ORC_OK;
done:
  free(gub);
  free(gpb);
  free(gmb);
  free_grid(&g);
  return rc;
}

/* Full reverse replay (Section 3.2 tape): states[0..T] from orc_run, adj holds
   the adjoint of state_T on entry and the adjoint of state_0 on return (same
   block layout as a state).  mubar/labar/wbar are accumulated. */
int orc_grad(const orc_params* P, int64_t np, int T, const double* mu, const double* la,
             const int32_t* grp, const double* wact, const double* states, double* adj,
             double* mubar, double* labar, double* wbar) {
  int d = P->dim;
  int64_t blk = (int64_t)(2 * d + 2 * d * d) * np;
  double* tmp = (double*)malloc(sizeof(double) * blk);
  if (!tmp) return ORC_ERR_MEM;
  for (int t = T - 1; t >= 0; t--) {
    const double* s = states + (int64_t)t * blk;
    int rc = orc_step_adjoint(P, np, t, s, s + d * np, s + 2 * d * np, s + (2 * d + d * d) * np,
                              mu, la, grp, wact, adj, adj + d * np, adj + 2 * d * np,
                              adj + (2 * d + d * d) * np, tmp, tmp + d * np, tmp + 2 * d * np,
                              tmp + (2 * d + d * d) * np, mubar, labar, wbar);
    if (rc) {
      free(tmp);
      return rc;
    }
    memcpy(adj, tmp, sizeof(double) * blk);
  }
  free(tmp);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* losses on the centre of mass (the compute_loss pattern, Section 3.2) */
/* ------------------------------------------------------------------ */

/* kind ORC_LOSS_COM_TARGET: L = |mean_p x_T - target|^2
   kind ORC_LOSS_COM_X_DISP: L = -(mean_p x_T[0] - mean_p x_0[0])
   Writes L and dL/dx_T (seed, component-major) and dL/dx_0 (direct term). */
int orc_com_loss(int dim, int64_t np, int kind, const double* xT, const double* x0,
                 const double* target, double* loss, double* xT_bar, double* x0_bar) {
  double com[3] = {0, 0, 0}, com0[3] = {0, 0, 0};
  for (int a = 0; a < dim; a++) {
    for (int64_t p = 0; p < np; p++) {
      com[a] += xT[a * np + p];
      com0[a] += x0[a * np + p];
    }
    com[a] /= (double)np;
    com0[a] /= (double)np;
  }
  for (int64_t i = 0; i < dim * np; i++) xT_bar[i] = x0_bar[i] = 0.0;
  if (kind == ORC_LOSS_COM_TARGET) {
    double L = 0.0;
    for (int a = 0; a < dim; a++) {
      double r = com[a] - target[a];
      L += r * r;
      for (int64_t p = 0; p < np; p++) xT_bar[a * np + p] = 2.0 * r / (double)np;
    }
    *loss = L;
  } else if (kind == ORC_LOSS_COM_X_DISP) {
    *loss = -(com[0] - com0[0]);
    for (int64_t p = 0; p < np; p++) {
      xT_bar[p] = -1.0 / (double)np;
      x0_bar[p] = 1.0 / (double)np;
    }
  } else {
    return ORC_ERR_ARG;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* mass-spring system (the paper's introductory example, Section 2 and */
/* the tape demonstration of Section 3): Hooke's springs, semi-        */
/* implicit Euler with damping, and its hand-derived adjoint          */
/* ------------------------------------------------------------------ */

/* One system: n masses of mass m in dim dimensions, springs (a_j, b_j) with rest length
   l0_j and stiffness k.  States 0 .. steps-1; step t (1 <= t < steps) from state t-1:
     d_j = x_a - x_b,  len_j = |d_j| + 1e-4 (the example's guard against a zero length),
     F_j = k (len_j - l0_j) d_j / len_j,   f_a -= F_j,  f_b += F_j,
     v_t = exp(-dt alpha) v_{t-1} + dt f / m,   x_t = x_{t-1} + dt v_t.
   x, v: [steps][n][dim] (row t holds state t; row 0 is read as the initial state). */
#define ORC_MS_EPS 1e-4

int orc_ms_forward(int dim, int n, int n_springs, const int32_t* sa, const int32_t* sb,
                   const double* l0, double k, double alpha, double dt, double m, int steps,
                   double* x, double* v) {
  if (dim < 1 || dim > 3 || n < 1 || steps < 1) return ORC_ERR_ARG;
  double* f = (double*)calloc((size_t)n * dim, sizeof(double));
  if (!f) return ORC_ERR_MEM;
  const double s = exp(-dt * alpha);
  for (int t = 1; t < steps; t++) {
    const double* x0 = x + (size_t)(t - 1) * n * dim;
    const double* v0 = v + (size_t)(t - 1) * n * dim;
    double* x1 = x + (size_t)t * n * dim;
    double* v1 = v + (size_t)t * n * dim;
    for (int i = 0; i < n * dim; i++) f[i] = 0.0;
    for (int j = 0; j < n_springs; j++) {
      const int a = sa[j], b = sb[j];
      double d[3] = {0, 0, 0}, nrm = 0.0;
      for (int c = 0; c < dim; c++) {
        d[c] = x0[a * dim + c] - x0[b * dim + c];
        nrm += d[c] * d[c];
      }
      const double len = sqrt(nrm) + ORC_MS_EPS;
      for (int c = 0; c < dim; c++) {
        const double F = k * (len - l0[j]) * d[c] / len;
        f[a * dim + c] -= F;
        f[b * dim + c] += F;
      }
    }
    for (int i = 0; i < n * dim; i++) {
      v1[i] = s * v0[i] + dt * f[i] / m;
      x1[i] = x0[i] + dt * v1[i];
    }
  }
  free(f);
  return ORC_OK;
}

/* Reverse of orc_ms_forward over the recorded states x (v is not needed): xb, vb hold
   dL/d(state steps-1) on entry and dL/d(state 0) on return; l0b accumulates dL/dl0. */
int orc_ms_backward(int dim, int n, int n_springs, const int32_t* sa, const int32_t* sb,
                    const double* l0, double k, double alpha, double dt, double m, int steps,
                    const double* x, double* xb, double* vb, double* l0b) {
  if (dim < 1 || dim > 3 || n < 1 || steps < 1) return ORC_ERR_ARG;
  double* fb = (double*)calloc((size_t)n * dim, sizeof(double));
  if (!fb) return ORC_ERR_MEM;
  const double s = exp(-dt * alpha);
  for (int t = steps - 1; t >= 1; t--) {
    const double* x0 = x + (size_t)(t - 1) * n * dim;
    /* x_t = x_{t-1} + dt v_t ; v_t = s v_{t-1} + dt f / m */
    for (int i = 0; i < n * dim; i++) {
      vb[i] += dt * xb[i];     /* dL/dv_t, complete */
      fb[i] = dt / m * vb[i];  /* dL/df_t */
      vb[i] *= s;              /* dL/dv_{t-1} */
    }
    /* xb now carries dL/dx_{t-1} through the position update; add the spring forces' */
    for (int j = 0; j < n_springs; j++) {
      const int a = sa[j], b = sb[j];
      double d[3] = {0, 0, 0}, nrm = 0.0, Fb[3] = {0, 0, 0}, dFb = 0.0;
      for (int c = 0; c < dim; c++) {
        d[c] = x0[a * dim + c] - x0[b * dim + c];
        nrm += d[c] * d[c];
        Fb[c] = fb[b * dim + c] - fb[a * dim + c]; /* f_a -= F, f_b += F */
        dFb += d[c] * Fb[c];
      }
      const double r = sqrt(nrm), len = r + ORC_MS_EPS;
      /* F = k (1 - l0/len) d ; dlen/dd = d / r */
      l0b[j] += -k * dFb / len;
      for (int c = 0; c < dim; c++) {
        const double db = k * ((1.0 - l0[j] / len) * Fb[c] + (l0[j] / (len * len)) * dFb * d[c] / r);
        xb[a * dim + c] += db;
        xb[b * dim + c] -= db;
      }
    }
  }
  free(fb);
  return ORC_OK;
}

/* The example's loss on the triangle of masses 0, 1, 2 (dim 2): L = (|area| - target)^2,
   area = (x01 x x02) / 2; writes L and dL/dx (n x 2). */
int orc_ms_area_loss(int n, const double* x, double target, double* loss, double* xb) {
  if (n < 3) return ORC_ERR_ARG;
  const double e1[2] = {x[0] - x[2], x[1] - x[3]}, e2[2] = {x[0] - x[4], x[1] - x[5]};
  const double cr = e1[0] * e2[1] - e1[1] * e2[0];
  const double area = fabs(0.5 * cr), r = area - target;
  *loss = r * r;
  for (int i = 0; i < 2 * n; i++) xb[i] = 0.0;
  const double g = 2.0 * r * 0.5 * (cr >= 0.0 ? 1.0 : -1.0); /* dL/dcr */
  /* cr = e1x e2y - e1y e2x, e1 = x0 - x1, e2 = x0 - x2 */
  xb[0] += g * (e2[1] - e1[1]);
  xb[1] += g * (e1[0] - e2[0]);
  xb[2] += -g * e2[1];
  xb[3] += g * e2[0];
  xb[4] += g * e1[1];
  xb[5] += -g * e1[0];
  return ORC_OK;
}

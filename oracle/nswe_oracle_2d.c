/*
 * CPU oracle, two-dimensional part: steady SWE F(U)_x + G(U)_y = S(U),
 * U = (h, hu, hv) (Eq. 1-2), on a rectangular grid (Section 4):
 * dimension-by-dimension third-order WENO with characteristic decomposition
 * (Section 5.2), LLF fluxes at the two Gauss points of every edge, the source
 * quadratures S2 and S3 (Section 4.1), the residual of Eq. 20, the FD
 * Jacobian with its 21-cell stencil (J21) and the 9-cell cross (J9, Eq. 21),
 * Galerkin coarse operators by 2x2 aggregation (Eq. 23-24), multicolour block
 * SOR (Eq. 22), prolongation (Eq. 25), the V-cycle, Newton and the nested
 * solve, and the two-dimensional App. A interpolation (Eq. A.3).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow FP64 restatement used to check the
 * CUDA library; it shares no code with it.
 *
 * Conventions: cell (i, j), 0 <= i < Nx, 0 <= j < Ny, index c = j*Nx + i; a
 * state is three planes h, hu, hv of Nx*Ny doubles. A block-stencil operator
 * with offsets off[k] = (dx, dy), k < K, is stored as
 * J[(k*9 + l*3 + m)*n + c] = (dR_c / dU_{c+off[k]})_{lm}.
 *
 * Readings (the paper does not fix them):
 *  - characteristic decomposition: eigenvectors of the normal flux Jacobian
 *    at the arithmetic mean of the two cells adjacent to the interface;
 *  - the reconstructed values at an interface are edge averages; the value
 *    at the Gauss points y_j -+ dy/(2 sqrt 3) comes from the
 *    average-preserving quadratic through the three edge averages of rows
 *    j-1, j, j+1, i.e. U_0 -+ (U_{+1} - U_{-1})/(4 sqrt 3);
 *  - LLF speed a = max(|u_n,L| + c_L, |u_n,R| + c_R) per Gauss point;
 *  - boundaries: two ghost layers; reflective walls mirror the interior with
 *    the normal momentum negated, inflow cells take the prescribed state,
 *    outflow cells copy the edge cell, discharge cells take the given
 *    momenta and the edge depth, depth cells the given depth and the edge
 *    momenta; corner ghosts apply the x rule, then the y rule;
 *  - multicolour orderings: J9 (i+j) mod 3, J21 (i mod 3) + 3 (j mod 3), coarse
 *    5-point (i+j) mod 2, coarse 9-point (i mod 2) + 2 (j mod 2); one
 *    smoothing step = two symmetric passes (colours 0..C-1, C-1..0, twice),
 *    the multicolour analogue of the four sweeps D1-D4 of Eq. 22;
 *  - App. A in 2D: tensor product of the one-dimensional weights (A.2).
 *
 * Frozen linearisation (an option beside Eq. 12, not in the paper): the
 * perturbed local residuals take the WENO nonlinear weights and the
 * characteristic eigenvectors of every reconstruction from the current,
 * unperturbed iterate, so that only the candidate polynomials, the LLF
 * fluxes and the sources see the perturbation. With Eq. 12 as printed, the
 * derivatives of the nonlinear weights where the wedge's oblique jump meets
 * the wall (Section 5.2.2) give a Jacobian on which block SOR diverges for
 * every relaxation factor tried; with the weights frozen the paper's
 * omega = 0.1 contracts. The residual, and so the fixed point, are unchanged.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR2_REFLECT 5
#define OR2_INFLOW 6
#define OR2_OUTFLOW 7
#define OR2_DISCHARGE 8 /* momenta given (bc_state), depth from the edge cell */
#define OR2_DEPTH 9     /* depth given (bc_state), momenta from the edge cell */

typedef struct {
  int Nx, Ny;
  double x0, x1, y0, y1, dx, dy, g;
  const double *gq;       /* [2][4][n]: b_x, b_y at Gauss points q = 2*beta + gamma */
  const int *bc_kind;     /* [Ny left | Ny right | Nx bottom | Nx top] */
  const double *bc_state; /* [4][3] inflow state (h, hu, hv): left, right, bottom, top */
} or_grid2d;

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }

/* Cell value with ghost extension. */
static void value2d(const or_grid2d *G, const double *U, int i, int j, double out[3]) {
  const int Nx = G->Nx, Ny = G->Ny, n = Nx * Ny;
  if (i < 0 || i >= Nx) {
    int side = i < 0 ? 0 : 1;
    int kind = G->bc_kind[side * Ny + imin(imax(j, 0), Ny - 1)];
    if (kind == OR2_INFLOW) {
      for (int m = 0; m < 3; ++m) out[m] = G->bc_state[side * 3 + m];
    } else if (kind == OR2_REFLECT) {
      value2d(G, U, i < 0 ? -1 - i : 2 * Nx - 1 - i, j, out);
      out[1] = -out[1];
    } else {
      value2d(G, U, i < 0 ? 0 : Nx - 1, j, out);
      if (kind == OR2_DISCHARGE) { out[1] = G->bc_state[side * 3 + 1]; out[2] = G->bc_state[side * 3 + 2]; }
      if (kind == OR2_DEPTH) out[0] = G->bc_state[side * 3 + 0];
    }
    return;
  }
  if (j < 0 || j >= Ny) {
    int side = j < 0 ? 2 : 3;
    int kind = G->bc_kind[2 * Ny + (side - 2) * Nx + i];
    if (kind == OR2_INFLOW) {
      for (int m = 0; m < 3; ++m) out[m] = G->bc_state[side * 3 + m];
    } else if (kind == OR2_REFLECT) {
      value2d(G, U, i, j < 0 ? -1 - j : 2 * Ny - 1 - j, out);
      out[2] = -out[2];
    } else {
      value2d(G, U, i, j < 0 ? 0 : Ny - 1, out);
      if (kind == OR2_DISCHARGE) { out[1] = G->bc_state[side * 3 + 1]; out[2] = G->bc_state[side * 3 + 2]; }
      if (kind == OR2_DEPTH) out[0] = G->bc_state[side * 3 + 0];
    }
    return;
  }
  int c = j * Nx + i;
  for (int m = 0; m < 3; ++m) out[m] = U[m * n + c];
}

/* WENO3 of Section 3.1 (same weights as the 1D oracle, see or_weno3). */
void or_weno3(double a, double b, double c, double *up, double *um);

/* WENO3 of the values (a, b, c) with the nonlinear weights of the values
 * (a0, b0, c0): the weights of Eq. 8 with zeta = 1e-6 and the linear weights
 * 1/3, 2/3 (U^+) and 2/3, 1/3 (U^-) of or_weno3, the candidates of Eq. 7. */
static void weno3_fixed(double a0, double b0, double c0, double a, double b, double c, double *up,
                        double *um) {
  double beta0 = (c0 - b0) * (c0 - b0), beta1 = (b0 - a0) * (b0 - a0);
  double s0 = (1e-6 + beta0) * (1e-6 + beta0), s1 = (1e-6 + beta1) * (1e-6 + beta1);
  double a0w = (1.0 / 3.0) / s0, a1w = (2.0 / 3.0) / s1; /* alpha_r  */
  double t0w = (2.0 / 3.0) / s0, t1w = (1.0 / 3.0) / s1; /* alpha~_r */
  double p0 = 1.5 * b - 0.5 * c, p1 = 0.5 * a + 0.5 * b, q0 = 0.5 * b + 0.5 * c, q1 = -0.5 * a + 1.5 * b;
  *up = (a0w / (a0w + a1w)) * p0 + (a1w / (a0w + a1w)) * p1;
  *um = (t0w / (t0w + t1w)) * q0 + (t1w / (t0w + t1w)) * q1;
}

/* Eigenvectors of n.dF/dU for n = x (dir 0) or y (dir 1) at state V:
 * eigenvalues u_n - c, u_t (shear), u_n + c (Section 2). Rows of Lm are left
 * eigenvectors, columns of Rm right eigenvectors. */
static void eigen2d(int dir, const double V[3], double g, double Lm[3][3], double Rm[3][3]) {
  double h = V[0], u = V[1] / h, v = V[2] / h, c = sqrt(g * h);
  double un = dir == 0 ? u : v, ut = dir == 0 ? v : u;
  int in = dir == 0 ? 1 : 2, it = dir == 0 ? 2 : 1; /* normal / tangential momentum */
  memset(Lm, 0, sizeof(double) * 9);
  memset(Rm, 0, sizeof(double) * 9);
  /* right eigenvectors: r1 = (1, un - c, ut), r2 = (0, 0, 1), r3 = (1, un + c, ut)
   * in (h, normal momentum, tangential momentum) ordering */
  Rm[0][0] = 1.0; Rm[in][0] = un - c; Rm[it][0] = ut;
  Rm[it][1] = 1.0;
  Rm[0][2] = 1.0; Rm[in][2] = un + c; Rm[it][2] = ut;
  Lm[0][0] = (un + c) / (2.0 * c); Lm[0][in] = -1.0 / (2.0 * c);
  Lm[1][0] = -ut; Lm[1][it] = 1.0;
  Lm[2][0] = -(un - c) / (2.0 * c); Lm[2][in] = 1.0 / (2.0 * c);
}

/* One-sided characteristic WENO3 value at the interface between cells a and
 * a+1 of a line. vals[0..3] = U of cells a-1, a, a+1, a+2 along the line.
 * side 0: U^- (from the stencil a-1, a, a+1), side 1: U^+ (a, a+1, a+2). */
static void char_rec(int dir, const double vals[4][3], const double (*base)[3], double g, int side,
                     double out[3]) {
  /* base: NULL, or the unperturbed values of the same cells (frozen linearisation) */
  const double(*ref)[3] = base ? base : vals;
  double V[3], Lm[3][3], Rm[3][3];
  for (int m = 0; m < 3; ++m) V[m] = 0.5 * (ref[1][m] + ref[2][m]);
  eigen2d(dir, V, g, Lm, Rm);
  double W[3][3], Wb[3][3]; /* [cell][field] */
  for (int s = 0; s < 3; ++s) {
    const double *Uc = vals[side + s], *Ub = ref[side + s];
    for (int f = 0; f < 3; ++f) {
      W[s][f] = Lm[f][0] * Uc[0] + Lm[f][1] * Uc[1] + Lm[f][2] * Uc[2];
      Wb[s][f] = Lm[f][0] * Ub[0] + Lm[f][1] * Ub[1] + Lm[f][2] * Ub[2];
    }
  }
  double Wr[3];
  for (int f = 0; f < 3; ++f) {
    double up, um;
    if (base)
      weno3_fixed(Wb[0][f], Wb[1][f], Wb[2][f], W[0][f], W[1][f], W[2][f], &up, &um);
    else
      or_weno3(W[0][f], W[1][f], W[2][f], &up, &um);
    Wr[f] = side == 0 ? um : up;
  }
  for (int m = 0; m < 3; ++m) out[m] = Rm[m][0] * Wr[0] + Rm[m][1] * Wr[1] + Rm[m][2] * Wr[2];
}

/* Physical flux in direction dir and the LLF flux (Section 3.1). */
static void phys_flux2d(int dir, const double U[3], double g, double F[3]) {
  double h = U[0], u = U[1] / h, v = U[2] / h, p = 0.5 * g * h * h;
  if (dir == 0) {
    F[0] = U[1];
    F[1] = U[1] * u + p;
    F[2] = U[1] * v;
  } else {
    F[0] = U[2];
    F[1] = U[2] * u;
    F[2] = U[2] * v + p;
  }
}

void or_llf2d(int dir, const double UL[3], const double UR[3], double g, double F[3]) {
  double FL[3], FR[3];
  phys_flux2d(dir, UL, g, FL);
  phys_flux2d(dir, UR, g, FR);
  double unL = UL[1 + dir] / UL[0], unR = UR[1 + dir] / UR[0];
  double a = fmax(fabs(unL) + sqrt(g * UL[0]), fabs(unR) + sqrt(g * UR[0]));
  for (int m = 0; m < 3; ++m) F[m] = 0.5 * (FL[m] + FR[m]) - 0.5 * a * (UR[m] - UL[m]);
}

double or_cubic4(const double p[4], double t);

/* Value of a cell along a line: dir 0 = row r (cells vary in i), dir 1 =
 * column r (cells vary in j). */
static void line_value(const or_grid2d *G, const double *U, int dir, int r, int k, double out[3]) {
  if (dir == 0) value2d(G, U, k, r, out);
  else value2d(G, U, r, k, out);
}

/* Reconstructed values at the interface k+1/2 of line r, side 0 (U^-) or 1. */
static void iface_value(const or_grid2d *G, const double *U, const double *U0, int dir, int r, int k, int side,
                        double out[3]) {
  double vals[4][3], base[4][3];
  for (int s = 0; s < 4; ++s) line_value(G, U, dir, r, k - 1 + s, vals[s]);
  if (U0)
    for (int s = 0; s < 4; ++s) line_value(G, U0, dir, r, k - 1 + s, base[s]);
  char_rec(dir, vals, U0 ? (const double(*)[3])base : NULL, G->g, side, out);
}

/* Transverse interpolation of Section 4.1: the three reconstructed edge
 * values of lines r-1, r, r+1 at one interface are edge averages; the
 * quadratic that keeps those three averages takes, at the Gauss point
 * -+ 1/(2 sqrt 3) of the middle edge, the value mid -+ (hi - lo)/(4 sqrt 3)
 * (its curvature term (s^2 - 1/12) vanishes there). sgn = -1 (q = 0) or +1. */
static void transverse_gauss(const double lo[3], const double mid[3], const double hi[3], double sgn, double out[3]) {
  const double s3 = 1.0 / (4.0 * sqrt(3.0));
  for (int m = 0; m < 3; ++m) out[m] = mid[m] + sgn * s3 * (hi[m] - lo[m]);
}

/* Values of the reconstruction at the two Gauss points of the face between
 * cells k and k+1 of line r (dir 0: row r, x face; dir 1: column r, y face),
 * side 0 (U^-) or 1 (U^+): out[q], q = 0 at the lower transverse Gauss point,
 * q = 1 at the upper one. These are the states the LLF flux of Section 4.1
 * sees. */
void or_face_gauss2d(const or_grid2d *G, const double *U, int dir, int r, int k, int side, double out[6]) {
  double v[3][3];
  for (int t = 0; t < 3; ++t) iface_value(G, U, NULL, dir, r - 1 + t, k, side, v[t]);
  transverse_gauss(v[0], v[1], v[2], -1.0, out);
  transverse_gauss(v[0], v[1], v[2], 1.0, out + 3);
}

/* Local residual R_ij (Eq. 20), three components; with U0 != NULL the
 * reconstructions take their weights and eigenvectors from U0. */
static void residual_cell2d(const or_grid2d *G, const double *U, const double *U0, int i, int j, double R[3]) {
  const int n = G->Nx * G->Ny, c = j * G->Nx + i;
  const double tg = 1.0 / (2.0 * sqrt(3.0));
  double flux[2][3] = {{0}}, S[3] = {0, 0, 0};
  /* dir 0: x faces i-1/2, i+1/2 of row j, transverse rows j-1..j+1.
   * dir 1: y faces j-1/2, j+1/2 of column i, transverse columns i-1..i+1. */
  for (int dir = 0; dir < 2; ++dir) {
    const int a = dir == 0 ? i : j;   /* position along the line */
    const int r0 = dir == 0 ? j : i;  /* line index */
    /* ifv[t][f][side]: t = transverse line r0-1..r0+1, f: interfaces a-3/2,
     * a-1/2, a+1/2, a+3/2 (k = a-2 .. a+1) */
    double ifv[3][4][2][3];
    for (int t = 0; t < 3; ++t)
      for (int f = 0; f < 4; ++f)
        for (int side = 0; side < 2; ++side) {
          int k = a - 2 + f;
          if ((f == 0 && side == 0) || (f == 3 && side == 1)) continue; /* not needed */
          iface_value(G, U, U0, dir, r0 - 1 + t, k, side, ifv[t][f][side]);
        }
    double fl[2][3] = {{0}};
    double hq[2][4]; /* h at the two Gauss lines, interfaces f = 0..3 (side used by the cubic) */
    for (int q = 0; q < 2; ++q) {
      double sgn = q == 0 ? -1.0 : 1.0;
      double gv[4][2][3];
      for (int f = 0; f < 4; ++f)
        for (int side = 0; side < 2; ++side) {
          if ((f == 0 && side == 0) || (f == 3 && side == 1)) continue;
          transverse_gauss(ifv[0][f][side], ifv[1][f][side], ifv[2][f][side], sgn, gv[f][side]);
        }
      for (int e = 0; e < 2; ++e) { /* e = 0: face a-1/2 (f=1), e = 1: a+1/2 (f=2) */
        double F[3];
        or_llf2d(dir, gv[1 + e][0], gv[1 + e][1], G->g, F);
        for (int m = 0; m < 3; ++m) fl[e][m] += 0.5 * F[m];
      }
      hq[q][0] = gv[0][1][0]; /* U^+ at a-3/2 */
      hq[q][1] = gv[1][1][0]; /* U^+ at a-1/2 */
      hq[q][2] = gv[2][0][0]; /* U^- at a+1/2 */
      hq[q][3] = gv[3][0][0]; /* U^- at a+3/2 */
    }
    for (int m = 0; m < 3; ++m) flux[dir][m] = fl[1][m] - fl[0][m];
    /* source of the momentum component along dir: -(dx dy / 4) sum g h b_dir */
    double acc = 0.0;
    for (int q = 0; q < 2; ++q)     /* Gauss line of the transverse direction */
      for (int p = 0; p < 2; ++p) { /* Gauss point along the line */
        double hv = or_cubic4(hq[q], (p == 0 ? -1.0 : 1.0) * tg);
        int beta = dir == 0 ? q : p, gamma = dir == 0 ? p : q;
        double bd = G->gq[(dir * 4 + 2 * beta + gamma) * n + c];
        acc += G->g * hv * bd;
      }
    S[1 + dir] = -0.25 * acc; /* S / (dx dy) */
  }
  for (int m = 0; m < 3; ++m) R[m] = flux[0][m] / G->dx + flux[1][m] / G->dy - S[m];
}

void or_residual_cell2d(const or_grid2d *G, const double *U, int i, int j, double R[3]) {
  residual_cell2d(G, U, NULL, i, j, R);
}

double or_residual2d(const or_grid2d *G, const double *U, double *R) {
  const int n = G->Nx * G->Ny;
  double res = 0.0;
  for (int j = 0; j < G->Ny; ++j)
    for (int i = 0; i < G->Nx; ++i) {
      double r[3];
      or_residual_cell2d(G, U, i, j, r);
      int c = j * G->Nx + i;
      for (int m = 0; m < 3; ++m) {
        R[m * n + c] = r[m];
        res += fabs(r[m]);
      }
    }
  return res / n;
}

/* ------------------------------------------------------------------------ */
/* Stencils (offset lists, sorted by dy then dx). */
static const int OFF_J9[9][2] = {{0, -2}, {0, -1}, {-2, 0}, {-1, 0}, {0, 0}, {1, 0}, {2, 0}, {0, 1}, {0, 2}};
static const int OFF_J21[21][2] = {{-1, -2}, {0, -2}, {1, -2}, {-2, -1}, {-1, -1}, {0, -1}, {1, -1},
                                   {2, -1},  {-2, 0}, {-1, 0}, {0, 0},   {1, 0},   {2, 0},   {-2, 1},
                                   {-1, 1},  {0, 1},  {1, 1},  {2, 1},   {-1, 2},  {0, 2},   {1, 2}};
static const int OFF_P5[5][2] = {{0, -1}, {-1, 0}, {0, 0}, {1, 0}, {0, 1}};
static const int OFF_P9[9][2] = {{-1, -1}, {0, -1}, {1, -1}, {-1, 0}, {0, 0}, {1, 0}, {-1, 1}, {0, 1}, {1, 1}};

#define ST_J9 0
#define ST_J21 1
#define ST_P5 2
#define ST_P9 3

int or_stencil_size(int st) { return st == ST_J9 ? 9 : st == ST_J21 ? 21 : st == ST_P5 ? 5 : 9; }
static const int (*stencil(int st))[2] { return st == ST_J9 ? OFF_J9 : st == ST_J21 ? OFF_J21 : st == ST_P5 ? OFF_P5 : OFF_P9; }
int or_stencil_offset(int st, int k, int d) { return stencil(st)[k][d]; }
static int stencil_center(int st) { int K = or_stencil_size(st); for (int k = 0; k < K; ++k) if (!stencil(st)[k][0] && !stencil(st)[k][1]) return k; return -1; }
static int coarse_stencil(int st) { return (st == ST_J9 || st == ST_P5) ? ST_P5 : ST_P9; }

/* FD Jacobian (Eq. 12-13 in 2D; J21: full stencil, J9: cross, Eq. 21). */
static double jacobian2d(const or_grid2d *G, double *U, double eps, double alpha, int st, int frozen, double *R,
                         double *J) {
  const int Nx = G->Nx, Ny = G->Ny, n = Nx * Ny, K = or_stencil_size(st), kc = stencil_center(st);
  double res = or_residual2d(G, U, R);
  memset(J, 0, sizeof(double) * (size_t)K * 9 * n);
  double *U0 = NULL;
  if (frozen) {
    U0 = malloc(sizeof(double) * 3 * n);
    memcpy(U0, U, sizeof(double) * 3 * n);
  }
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      int c = j * Nx + i;
      double R0[3] = {R[c], R[n + c], R[2 * n + c]};
      for (int k = 0; k < K; ++k) {
        int p = i + stencil(st)[k][0], q = j + stencil(st)[k][1];
        if (p < 0 || p >= Nx || q < 0 || q >= Ny) continue;
        int cp = q * Nx + p;
        for (int m = 0; m < 3; ++m) {
          double save = U[m * n + cp];
          U[m * n + cp] = save + eps;
          double Rp[3];
          residual_cell2d(G, U, U0, i, j, Rp);
          U[m * n + cp] = save;
          for (int l = 0; l < 3; ++l) J[(size_t)(k * 9 + l * 3 + m) * n + c] = (Rp[l] - R0[l]) / eps;
        }
      }
      double reg = alpha * (fabs(R0[0]) + fabs(R0[1]) + fabs(R0[2]));
      for (int l = 0; l < 3; ++l) J[(size_t)(kc * 9 + l * 3 + l) * n + c] += reg;
    }
  free(U0);
  return res;
}

/* Eq. 12-13 on the stencil st. */
double or_jacobian2d(const or_grid2d *G, double *U, double eps, double alpha, int st, double *R, double *J) {
  return jacobian2d(G, U, eps, alpha, st, 0, R, J);
}

/* Eq. 12-13 with the frozen linearisation (weights and eigenvectors of the
 * reconstructions from U, see the header). */
double or_jacobian2d_frozen(const or_grid2d *G, double *U, double eps, double alpha, int st, double *R, double *J) {
  return jacobian2d(G, U, eps, alpha, st, 1, R, J);
}

/* ------------------------------------------------------------------------ */
/* Multigrid, 2x2 aggregation (Eq. 23); sizes must be even. */

/* Galerkin coarse operator (Eq. 24) of a fine operator with stencil st. */
void or_coarse_operator2d(int Nx, int Ny, int st, const double *Jf, double *Jc) {
  const int n = Nx * Ny, Ncx = Nx / 2, Ncy = Ny / 2, nc = Ncx * Ncy;
  const int K = or_stencil_size(st), cs = coarse_stencil(st), Kc = or_stencil_size(cs);
  memset(Jc, 0, sizeof(double) * (size_t)Kc * 9 * nc);
  for (int yi = 0; yi < Ny; ++yi)
    for (int xi = 0; xi < Nx; ++xi) {
      int I = xi / 2, Jy = yi / 2, cc = Jy * Ncx + I, c = yi * Nx + xi;
      for (int k = 0; k < K; ++k) {
        int ex = xi + stencil(st)[k][0], ey = yi + stencil(st)[k][1];
        if (ex < 0 || ex >= Nx || ey < 0 || ey >= Ny) continue;
        int ox = ex / 2 - I, oy = ey / 2 - Jy, kk = -1;
        for (int t = 0; t < Kc; ++t)
          if (stencil(cs)[t][0] == ox && stencil(cs)[t][1] == oy) kk = t;
        if (kk < 0) continue; /* cannot happen for the stencils used */
        for (int e = 0; e < 9; ++e) Jc[(size_t)(kk * 9 + e) * nc + cc] += Jf[(size_t)(k * 9 + e) * n + c];
      }
    }
}

/* 3x3 inverse by cofactors. */
static void inv3(const double a[9], double o[9]) {
  double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  o[0] = c00 / det;
  o[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  o[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  o[3] = c01 / det;
  o[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  o[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  o[6] = c02 / det;
  o[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  o[8] = (a[0] * a[4] - a[1] * a[3]) / det;
}

void or_block_inverse2d(int n, int st, const double *J, double *Dinv) {
  int kc = stencil_center(st);
  for (int c = 0; c < n; ++c) {
    double a[9], o[9];
    for (int e = 0; e < 9; ++e) a[e] = J[(size_t)(kc * 9 + e) * n + c];
    inv3(a, o);
    for (int e = 0; e < 9; ++e) Dinv[(size_t)e * n + c] = o[e];
  }
}

int or_colours2d(int st) { return st == ST_J9 ? 3 : st == ST_J21 ? 9 : st == ST_P5 ? 2 : 4; }
int or_colour_of(int st, int i, int j) {
  switch (st) {
  case ST_J9: return (i + j) % 3;
  case ST_J21: return (i % 3) + 3 * (j % 3);
  case ST_P5: return (i + j) % 2;
  default: return (i % 2) + 2 * (j % 2);
  }
}

/* Diagonal colourings of the cross stencils (J9, coarse 5-point) of a grid
 * Nx wide, K colours: mode 1: (i + j) mod K, mode 2: (j - i + Nx - 1) mod K
 * (the offset makes the diagonal index non-negative, so that ascending
 * colours are ascending diagonals when K covers them all). Cells of one
 * colour do not couple for K >= 3 (J9: offsets up to 2 along an axis) or
 * K >= 2 (5-point). */
int or_diag_colour(int mode, int K, int i, int j, int Nx) {
  return (mode == 1 ? i + j : j - i + Nx - 1) % K;
}

/* Block SOR update (Eq. 22) of every cell of one colour: mode 0 uses the
 * stencil's own colouring (or_colour_of), modes 1 and 2 the diagonal ones. */
static void sor_colour2d(int Nx, int Ny, int st, const double *J, const double *Dinv, const double *R, double *dU,
                         double omega, int mode, int Kc, int col) {
  const int n = Nx * Ny, K = or_stencil_size(st), kc = stencil_center(st);
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      const int colour = mode == 0 ? or_colour_of(st, i, j) : or_diag_colour(mode, Kc, i, j, Nx);
      if (colour != col) continue;
      int c = j * Nx + i;
      double r[3] = {R[c], R[n + c], R[2 * n + c]};
      for (int k = 0; k < K; ++k) {
        if (k == kc) continue;
        int p = i + stencil(st)[k][0], q = j + stencil(st)[k][1];
        if (p < 0 || p >= Nx || q < 0 || q >= Ny) continue;
        int cp = q * Nx + p;
        for (int l = 0; l < 3; ++l)
          r[l] += J[(size_t)(k * 9 + l * 3 + 0) * n + c] * dU[cp] + J[(size_t)(k * 9 + l * 3 + 1) * n + c] * dU[n + cp] +
                  J[(size_t)(k * 9 + l * 3 + 2) * n + c] * dU[2 * n + cp];
      }
      for (int l = 0; l < 3; ++l) {
        double t = Dinv[(size_t)(l * 3 + 0) * n + c] * r[0] + Dinv[(size_t)(l * 3 + 1) * n + c] * r[1] +
                   Dinv[(size_t)(l * 3 + 2) * n + c] * r[2];
        dU[l * n + c] = (1.0 - omega) * dU[l * n + c] - omega * t;
      }
    }
}

/* One smoothing step, the multicolour analogue of the four sweeps D1-D4 of
 * Eq. 22. Cross stencils (J9, coarse 5-point) with K >= 3 colours: the
 * colours of (i + j) mod K ascending (D1: towards +x, +y), of
 * (j - i + Nx - 1) mod K ascending (D2: -x, +y), of (i + j) mod K descending
 * (D3: -x, -y), of (j - i + Nx - 1) mod K descending (D4: +x, -y). Within each, a cell sees the new
 * values of its upstream neighbours up to K - 1 diagonals back; for
 * K >= Nx + Ny - 1 this is exactly the lexicographic sweep D1..D4. Other
 * stencils (J21, coarse 9-point), or K = 0: two symmetric passes of the
 * stencil's own colouring (0..C-1, C-1..0, twice). */
void or_sor_step2d(int Nx, int Ny, int st, const double *J, const double *Dinv, const double *R, double *dU,
                   double omega, int K) {
  if (K >= 3 && (st == ST_J9 || st == ST_P5)) {
    for (int c = 0; c < K; ++c) sor_colour2d(Nx, Ny, st, J, Dinv, R, dU, omega, 1, K, c);
    for (int c = 0; c < K; ++c) sor_colour2d(Nx, Ny, st, J, Dinv, R, dU, omega, 2, K, c);
    for (int c = K - 1; c >= 0; --c) sor_colour2d(Nx, Ny, st, J, Dinv, R, dU, omega, 1, K, c);
    for (int c = K - 1; c >= 0; --c) sor_colour2d(Nx, Ny, st, J, Dinv, R, dU, omega, 2, K, c);
    return;
  }
  int C = or_colours2d(st);
  for (int rep = 0; rep < 2; ++rep) {
    for (int c = 0; c < C; ++c) sor_colour2d(Nx, Ny, st, J, Dinv, R, dU, omega, 0, 0, c);
    for (int c = C - 1; c >= 0; --c) sor_colour2d(Nx, Ny, st, J, Dinv, R, dU, omega, 0, 0, c);
  }
}

/* Defect restriction (Eq. 24): Rc = sum over the 2x2 aggregate of (R + J dU). */
void or_restrict2d(int Nx, int Ny, int st, const double *J, const double *R, const double *dU, double *Rc) {
  const int n = Nx * Ny, Ncx = Nx / 2, nc = Ncx * (Ny / 2), K = or_stencil_size(st);
  memset(Rc, 0, sizeof(double) * 3 * (size_t)nc);
  for (int yi = 0; yi < Ny; ++yi)
    for (int xi = 0; xi < Nx; ++xi) {
      int c = yi * Nx + xi, cc = (yi / 2) * Ncx + xi / 2;
      double r[3] = {R[c], R[n + c], R[2 * n + c]};
      for (int k = 0; k < K; ++k) {
        int p = xi + stencil(st)[k][0], q = yi + stencil(st)[k][1];
        if (p < 0 || p >= Nx || q < 0 || q >= Ny) continue;
        int cp = q * Nx + p;
        for (int l = 0; l < 3; ++l)
          r[l] += J[(size_t)(k * 9 + l * 3 + 0) * n + c] * dU[cp] + J[(size_t)(k * 9 + l * 3 + 1) * n + c] * dU[n + cp] +
                  J[(size_t)(k * 9 + l * 3 + 2) * n + c] * dU[2 * n + cp];
      }
      for (int l = 0; l < 3; ++l) Rc[l * nc + cc] += r[l];
    }
}

/* Prolongation (Eq. 25). */
void or_prolong2d(int Nx, int Ny, double *dU, const double *dUc) {
  const int n = Nx * Ny, Ncx = Nx / 2, nc = Ncx * (Ny / 2);
  for (int yi = 0; yi < Ny; ++yi)
    for (int xi = 0; xi < Nx; ++xi) {
      int c = yi * Nx + xi, cc = (yi / 2) * Ncx + xi / 2;
      for (int l = 0; l < 3; ++l) dU[l * n + c] += dUc[l * nc + cc];
    }
}

int or_dense_solve(int n, double *A, double *b);

/* Direct solve of J dU = -R (unknown 3c + m). */
int or_direct_solve2d(int Nx, int Ny, int st, const double *J, const double *R, double *dU) {
  const int n = Nx * Ny, K = or_stencil_size(st), N3 = 3 * n;
  double *A = calloc((size_t)N3 * N3, sizeof(double));
  double *b = malloc(sizeof(double) * N3);
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      int c = j * Nx + i;
      for (int l = 0; l < 3; ++l) b[3 * c + l] = -R[l * n + c];
      for (int k = 0; k < K; ++k) {
        int p = i + stencil(st)[k][0], q = j + stencil(st)[k][1];
        if (p < 0 || p >= Nx || q < 0 || q >= Ny) continue;
        int cp = q * Nx + p;
        for (int l = 0; l < 3; ++l)
          for (int m = 0; m < 3; ++m) A[(size_t)(3 * c + l) * N3 + 3 * cp + m] = J[(size_t)(k * 9 + l * 3 + m) * n + c];
      }
    }
  int rc = or_dense_solve(N3, A, b);
  for (int c = 0; c < n; ++c)
    for (int l = 0; l < 3; ++l) dU[l * n + c] = b[3 * c + l];
  free(A);
  free(b);
  return rc;
}

typedef struct {
  int L, st0;
  int Nx[16], Ny[16], st[16];
  double *J[16], *Dinv[16], *R[16], *dU[16];
} or_mg2d;

static void mg2_alloc(or_mg2d *mg, int Nx, int Ny, int nlev, int st0) {
  memset(mg, 0, sizeof(*mg));
  mg->L = nlev - 1;
  mg->st0 = st0;
  for (int l = 0; l < nlev; ++l) {
    mg->Nx[l] = Nx >> l;
    mg->Ny[l] = Ny >> l;
    mg->st[l] = l == 0 ? st0 : coarse_stencil(mg->st[l - 1]);
    int n = mg->Nx[l] * mg->Ny[l], K = or_stencil_size(mg->st[l]);
    if (l > 0) {
      mg->J[l] = malloc(sizeof(double) * (size_t)K * 9 * n);
      mg->R[l] = malloc(sizeof(double) * 3 * (size_t)n);
      mg->dU[l] = malloc(sizeof(double) * 3 * (size_t)n);
    }
    mg->Dinv[l] = malloc(sizeof(double) * 9 * (size_t)n);
  }
}

static void mg2_free(or_mg2d *mg) {
  for (int l = 0; l <= mg->L; ++l) {
    if (l > 0) {
      free(mg->J[l]);
      free(mg->R[l]);
      free(mg->dU[l]);
    }
    free(mg->Dinv[l]);
  }
}

static void mg2_setup(or_mg2d *mg) {
  for (int l = 1; l <= mg->L; ++l) or_coarse_operator2d(mg->Nx[l - 1], mg->Ny[l - 1], mg->st[l - 1], mg->J[l - 1], mg->J[l]);
  for (int l = 0; l <= mg->L; ++l) or_block_inverse2d(mg->Nx[l] * mg->Ny[l], mg->st[l], mg->J[l], mg->Dinv[l]);
}

static int mg2_vcycle(or_mg2d *mg, int l, double omega, int nu1, int nu2, int K) {
  int Nx = mg->Nx[l], Ny = mg->Ny[l], st = mg->st[l];
  if (l == mg->L) return or_direct_solve2d(Nx, Ny, st, mg->J[l], mg->R[l], mg->dU[l]);
  for (int s = 0; s < nu1; ++s) or_sor_step2d(Nx, Ny, st, mg->J[l], mg->Dinv[l], mg->R[l], mg->dU[l], omega, K);
  or_restrict2d(Nx, Ny, st, mg->J[l], mg->R[l], mg->dU[l], mg->R[l + 1]);
  memset(mg->dU[l + 1], 0, sizeof(double) * 3 * (size_t)mg->Nx[l + 1] * mg->Ny[l + 1]);
  int rc = mg2_vcycle(mg, l + 1, omega, nu1, nu2, K);
  or_prolong2d(Nx, Ny, mg->dU[l], mg->dU[l + 1]);
  for (int s = 0; s < nu2; ++s) or_sor_step2d(Nx, Ny, st, mg->J[l], mg->Dinv[l], mg->R[l], mg->dU[l], omega, K);
  return rc;
}

int or_vcycle2d(int Nx, int Ny, int st, int nlev, const double *J, const double *R, double *dU, double omega,
                int nu1, int nu2, int K) {
  or_mg2d mg;
  mg2_alloc(&mg, Nx, Ny, nlev, st);
  mg.J[0] = (double *)J;
  mg.R[0] = (double *)R;
  mg.dU[0] = dU;
  mg2_setup(&mg);
  int rc = mg2_vcycle(&mg, 0, omega, nu1, nu2, K);
  mg2_free(&mg);
  return rc;
}

/* App. A in 2D: tensor product of the weights of Eq. A.2 over the coarse
 * 3x3 neighbourhood (ghost values at the boundary). */
void or_interp2d(const or_grid2d *Gc, const double *Uc, double *Uf) {
  const int Ncx = Gc->Nx, Ncy = Gc->Ny, Nfx = 2 * Ncx, nf = Nfx * 2 * Ncy;
  static const double w[2][3] = {{0.125, 1.0, -0.125}, {-0.125, 1.0, 0.125}};
  for (int J = 0; J < Ncy; ++J)
    for (int I = 0; I < Ncx; ++I) {
      double nb[3][3][3]; /* [q][p][m] */
      for (int q = -1; q <= 1; ++q)
        for (int p = -1; p <= 1; ++p) value2d(Gc, Uc, I + p, J + q, nb[q + 1][p + 1]);
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          int cf = (2 * J + b) * Nfx + 2 * I + a;
          for (int m = 0; m < 3; ++m) {
            double s = 0.0;
            for (int q = 0; q < 3; ++q) {
              double row = 0.0;
              for (int p = 0; p < 3; ++p) row += w[a][p] * nb[q][p][m];
              s += w[b][q] * row;
            }
            Uf[m * nf + cf] = s;
          }
        }
    }
}

/* ------------------------------------------------------------------------ */
typedef struct {
  double alpha, tau, omega, tol;
  int nu1[16], nu2[16]; /* smoothing steps per nested level (Section 5.2: grid dependent) */
  int nu3, levels, n_max, st, nest_start;
  double eps;
  int colours; /* K of the diagonal smoothing schedule (cross stencils); 0: stencil colourings */
  int frozen;  /* 1: the frozen linearisation of the Jacobian */
} or_params2d;

typedef struct {
  int status;
  int iters[16];
  double res[16];
  int total_iters, vcycles;
} or_info2d;

static int newton_level2d(const or_grid2d *G, double *U, int nlev, const or_params2d *p, int nu1, int nu2,
                          double *res_out, int *vcycles, int *status) {
  const int n = G->Nx * G->Ny, K = or_stencil_size(p->st);
  double *R = malloc(sizeof(double) * 3 * n), *J = malloc(sizeof(double) * (size_t)K * 9 * n);
  double *dU = malloc(sizeof(double) * 3 * n);
  or_mg2d mg;
  mg2_alloc(&mg, G->Nx, G->Ny, nlev, p->st);
  mg.J[0] = J;
  mg.R[0] = R;
  mg.dU[0] = dU;
  int it = 0;
  double res = 0.0;
  *status = 0;
  do {
    jacobian2d(G, U, p->eps, p->alpha, p->st, p->frozen, R, J);
    memset(dU, 0, sizeof(double) * 3 * n);
    if (nlev == 1) {
      if (or_direct_solve2d(G->Nx, G->Ny, p->st, J, R, dU)) { *status = 3; break; }
    } else {
      mg2_setup(&mg);
      for (int m = 0; m < p->nu3; ++m) {
        if (mg2_vcycle(&mg, 0, p->omega, nu1, nu2, p->colours)) { *status = 3; break; }
        (*vcycles)++;
      }
      if (*status) break;
    }
    for (int t = 0; t < 3 * n; ++t) U[t] += p->tau * dU[t];
    res = or_residual2d(G, U, R);
    ++it;
    if (!(res == res)) { *status = 2; break; }
  } while (!(res < p->tol) && it < p->n_max);
  if (*status == 0 && !(res < p->tol)) *status = 1;
  mg2_free(&mg);
  free(R);
  free(J);
  free(dU);
  *res_out = res;
  return it;
}

/* Algorithm 3 in 2D; grids[l] = nested level l; U0 on the start level. */
int or_nmgm2d(const or_grid2d *grids, const double *U0, double *U, const or_params2d *p, or_info2d *info) {
  int L = p->levels - 1;
  int s0 = (p->nest_start < 0 || p->nest_start > L) ? L : p->nest_start;
  memset(info, 0, sizeof(*info));
  int n = grids[s0].Nx * grids[s0].Ny;
  double *V = malloc(sizeof(double) * 3 * n);
  memcpy(V, U0, sizeof(double) * 3 * n);
  for (int l = s0; l >= 0; --l) {
    if (l < s0) {
      int nf = grids[l].Nx * grids[l].Ny;
      double *Vf = malloc(sizeof(double) * 3 * nf);
      or_interp2d(&grids[l + 1], V, Vf);
      free(V);
      V = Vf;
    }
    int st = 0;
    info->iters[l] = newton_level2d(&grids[l], V, L - l + 1, p, p->nu1[l], p->nu2[l], &info->res[l],
                                    &info->vcycles, &st);
    info->total_iters += info->iters[l];
    if (st) { info->status = st; if (st >= 2) break; }
  }
  if (info->status < 2) memcpy(U, V, sizeof(double) * 3 * grids[0].Nx * grids[0].Ny);
  free(V);
  return info->status;
}

int or_newton2d(const or_grid2d *G, double *U, int nlev, const or_params2d *p, or_info2d *info) {
  memset(info, 0, sizeof(*info));
  int st = 0;
  info->iters[0] = newton_level2d(G, U, nlev, p, p->nu1[0], p->nu2[0], &info->res[0], &info->vcycles, &st);
  info->total_iters = info->iters[0];
  info->status = st;
  return st;
}

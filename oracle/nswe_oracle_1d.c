/*
 * CPU oracle, one-dimensional part: quasi-1D steady shallow water equations
 * (Eq. 3-4) discretised by the third-order finite-volume WENO scheme of
 * Section 3.1 (Eq. 5-10), the regularized Newton iteration of Section 3.2
 * (Eq. 11-14, Algorithm 1), the simplified Jacobian J3 of Section 3.3, the
 * geometric multigrid of Section 3.4 (Eq. 15-19, Algorithm 2), the nested
 * NMGM solver (Algorithm 3) and the coarse-to-fine interpolation of
 * Appendix A (Eq. A.1-A.2).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, FP64 restatement used to check the
 * CUDA library. See nswe_oracle.h for the conventions. Where the paper is
 * silent or self-contradictory the reading taken is stated at the spot.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "nswe_oracle.h"

/* ------------------------------------------------------------------------ */
/* Boundary ghost cells. The paper states the boundary data (Section 5.1:
 * discharge upstream, depth downstream; h and hu at both ends in 5.1.1) but
 * not how they enter the scheme. Reading: two ghost cells per side, both equal
 * to a state built from the boundary data and the adjacent interior cell. */
static void ghost_state(int kind, double bh, double bq, double sig_b,
                        double He, double Qe, double *Hg, double *Qg) {
  switch (kind) {
  case OR_BC_DISCHARGE: *Hg = He; *Qg = bq; break;
  case OR_BC_DEPTH: *Hg = sig_b * bh; *Qg = Qe; break;
  case OR_BC_STATE: *Hg = sig_b * bh; *Qg = bq; break;
  default: *Hg = He; *Qg = Qe; break;
  }
}

/* Cell value with ghost extension: k<0 and k>=N use the boundary states. */
static void cell_value(const or_grid1d *g, const double *H, const double *Q,
                       int k, double *h, double *q) {
  int N = g->N;
  if (k < 0)
    ghost_state(g->bcl_kind, g->bcl_h, g->bcl_q, g->sig_face[0], H[0], Q[0], h, q);
  else if (k >= N)
    ghost_state(g->bcr_kind, g->bcr_h, g->bcr_q, g->sig_face[N], H[N - 1], Q[N - 1], h, q);
  else {
    *h = H[k];
    *q = Q[k];
  }
}

/* ------------------------------------------------------------------------ */
/* Third-order WENO reconstruction in cell k from the averages a=U_{k-1},
 * b=U_k, c=U_{k+1} (Eq. 7-8). Sub-stencils T0={k,k+1}, T1={k-1,k}.
 *   up = U^+_{k-1/2} (value at the left face of cell k)
 *   um = U^-_{k+1/2} (value at the right face of cell k)
 * Reading: the linear weights printed with Eq. 8 (d0 = 2/3 for U^+) are
 * swapped; with them the scheme is only second order. The weights that make
 * the combination equal the 3-cell quadratic reconstruction are
 *   U^+: d0 = 1/3, d1 = 2/3;   U^-: d~0 = 2/3, d~1 = 1/3,
 * consistent with the third-order rates of Table 1. */
/* zeta of Eq. 8: 1e-6 in the paper. A test may raise it: as zeta grows the
 * nonlinear weights tend to the linear weights d_r, and the scheme to the
 * optimal linear third-order one. */
static double or_weno_zeta = 1e-6;
void or_set_weno_zeta(double zeta) { or_weno_zeta = zeta; }
double or_get_weno_zeta(void) { return or_weno_zeta; }

void or_weno3(double a, double b, double c, double *up, double *um) {
  double beta0 = (c - b) * (c - b); /* smoothness of T0 */
  double beta1 = (b - a) * (b - a); /* smoothness of T1 */
  /* candidate reconstructions (Eq. 7, the four formulas after it) */
  double p0 = 1.5 * b - 0.5 * c; /* U^(0)_{k-1/2} */
  double p1 = 0.5 * a + 0.5 * b; /* U^(1)_{k-1/2} */
  double q0 = 0.5 * b + 0.5 * c; /* U^(0)_{k+1/2} */
  double q1 = -0.5 * a + 1.5 * b; /* U^(1)_{k+1/2} */
  double s0 = (or_weno_zeta + beta0) * (or_weno_zeta + beta0);
  double s1 = (or_weno_zeta + beta1) * (or_weno_zeta + beta1);
  double a0 = (1.0 / 3.0) / s0, a1 = (2.0 / 3.0) / s1;   /* alpha_r  */
  double t0 = (2.0 / 3.0) / s0, t1 = (1.0 / 3.0) / s1;   /* alpha~_r */
  double w0 = a0 / (a0 + a1), w1 = a1 / (a0 + a1);
  double v0 = t0 / (t0 + t1), v1 = t1 / (t0 + t1);
  *up = w0 * p0 + w1 * p1;
  *um = v0 * q0 + v1 * q1;
}

/* Physical flux F(U) = (Q, Q^2/H + g*sigma*h^2/2), h = H/sigma (Eq. 4). */
void or_flux1d(double H, double Q, double sig, double g, double F[2]) {
  double h = H / sig;
  F[0] = Q;
  F[1] = Q * Q / H + 0.5 * g * sig * h * h;
}

/* HLL numerical flux at a face of width sig (Section 3.1; the paper names the
 * flux but not its wave-speed estimates). Reading: S_L = min(u_L-c_L,
 * u_R-c_R), S_R = max(u_L+c_L, u_R+c_R), c = sqrt(g*h), standard three
 * branches with S_L >= 0 -> F_L and S_R <= 0 -> F_R. */
void or_hll1d(double HL, double QL, double HR, double QR, double sig, double g,
              double F[2]) {
  double FL[2], FR[2];
  or_flux1d(HL, QL, sig, g, FL);
  or_flux1d(HR, QR, sig, g, FR);
  double uL = QL / HL, uR = QR / HR;
  double cL = sqrt(g * (HL / sig)), cR = sqrt(g * (HR / sig));
  double SL = fmin(uL - cL, uR - cR);
  double SR = fmax(uL + cL, uR + cR);
  if (SL >= 0.0) {
    F[0] = FL[0];
    F[1] = FL[1];
  } else if (SR <= 0.0) {
    F[0] = FR[0];
    F[1] = FR[1];
  } else {
    F[0] = (SR * FL[0] - SL * FR[0] + SL * SR * (HR - HL)) / (SR - SL);
    F[1] = (SR * FL[1] - SL * FR[1] + SL * SR * (QR - QL)) / (SR - SL);
  }
}

/* LLF (Rusanov) numerical flux at a face of width sig (Section 3.1 names it
 * beside HLL): the mean of the two physical fluxes minus a (U_R - U_L) / 2,
 * with a the larger |u| + c of the two states, c = sqrt(g*h). */
void or_llf1d(double HL, double QL, double HR, double QR, double sig, double g,
              double F[2]) {
  double FL[2], FR[2];
  or_flux1d(HL, QL, sig, g, FL);
  or_flux1d(HR, QR, sig, g, FR);
  double uL = QL / HL, uR = QR / HR;
  double cL = sqrt(g * (HL / sig)), cR = sqrt(g * (HR / sig));
  double a = fmax(fabs(uL) + cL, fabs(uR) + cR);
  F[0] = 0.5 * (FL[0] + FR[0]) - 0.5 * a * (HR - HL);
  F[1] = 0.5 * (FL[1] + FR[1]) - 0.5 * a * (QR - QL);
}

/* Value at t (in units of dx from the cell centre) of the cubic through
 * (t_k, p_k), t_k = -3/2, -1/2, 1/2, 3/2, in Lagrange form (Eq. 9). */
double or_cubic4(const double p[4], double t) {
  static const double tk[4] = {-1.5, -0.5, 0.5, 1.5};
  double s = 0.0;
  for (int k = 0; k < 4; ++k) {
    double L = 1.0;
    for (int m = 0; m < 4; ++m)
      if (m != k) L *= (t - tk[m]) / (tk[k] - tk[m]);
    s += L * p[k];
  }
  return s;
}

/* Local residual R_j (Eq. 10): F_{j+1/2} - F_{j-1/2} - S_j, with S_j from the
 * two-point Gauss rule of Eq. 9 applied to S(U_h), U_h the cubic through
 * U^+_{j-3/2}, U^+_{j-1/2}, U^-_{j+1/2}, U^-_{j+3/2}. Only the H component of
 * U_h enters S = (0, g h^2 sigma_x/2 - g sigma h b_x), h = H_h/sigma. Not
 * divided by dx (Eq. 10). Depends on cells j-2..j+2 (Fig. 1b). */
void or_residual_cell1d(const or_grid1d *g, const double *H, const double *Q,
                        int j, double R[2]) {
  double upH[3], umH[3], upQ[3], umQ[3]; /* recs of cells j-1, j, j+1 */
  for (int p = 0; p < 3; ++p) {
    int k = j - 1 + p;
    double ha, qa, hb, qb, hc, qc;
    cell_value(g, H, Q, k - 1, &ha, &qa);
    cell_value(g, H, Q, k, &hb, &qb);
    cell_value(g, H, Q, k + 1, &hc, &qc);
    or_weno3(ha, hb, hc, &upH[p], &umH[p]);
    or_weno3(qa, qb, qc, &upQ[p], &umQ[p]);
  }
  double Fr[2], Fl[2];
  /* face j+1/2 (face index j+1): left state from cell j, right from cell j+1 */
  void (*flux)(double, double, double, double, double, double, double *) = g->flux == 1 ? or_llf1d : or_hll1d;
  flux(umH[1], umQ[1], upH[2], upQ[2], g->sig_face[j + 1], g->g, Fr);
  /* face j-1/2 (face index j): left state from cell j-1, right from cell j */
  flux(umH[0], umQ[0], upH[1], upQ[1], g->sig_face[j], g->g, Fl);
  /* source: cubic through the four interface values of H */
  double pts[4] = {upH[0], upH[1], umH[1], umH[2]};
  int N = g->N;
  double S = 0.0;
  for (int q = 0; q < 2; ++q) {
    double t = (q == 0 ? -1.0 : 1.0) / (2.0 * sqrt(3.0));
    double Hh = or_cubic4(pts, t);
    double sig = g->gq[(0 * 2 + q) * N + j];
    double sigx = g->gq[(1 * 2 + q) * N + j];
    double bx = g->gq[(2 * 2 + q) * N + j];
    double h = Hh / sig;
    S += 0.5 * g->g * h * h * sigx - g->g * sig * h * bx;
  }
  S *= 0.5 * g->dx;
  R[0] = Fr[0] - Fl[0];
  R[1] = Fr[1] - Fl[1] - S;
}

/* Global residual R[2][N] and res = (1/N) sum_j ||R_j||_1 (Algorithm 1). */
double or_residual1d(const or_grid1d *g, const double *H, const double *Q,
                     double *R) {
  int N = g->N;
  double res = 0.0;
  for (int j = 0; j < N; ++j) {
    double r[2];
    or_residual_cell1d(g, H, Q, j, r);
    R[j] = r[0];
    R[N + j] = r[1];
    res += fabs(r[0]) + fabs(r[1]);
  }
  return res / N;
}

/* FD Jacobian with regularization (Eq. 12-13). nb = 5 gives J5 (all blocks
 * of the 5-cell stencil), nb = 3 the simplified J3 (Section 3.3: the j+-2
 * blocks dropped). Each entry is a one-sided difference of the local residual
 * with U_i perturbed by eps in component m; the perturbation is applied to the
 * interior value and the ghost cells follow it. Blocks that reach outside
 * the grid are zero. H and Q are restored exactly after each perturbation.
 * Writes R[2][N] as well; returns res. */
double or_jacobian1d(const or_grid1d *g, double *H, double *Q, double eps,
                     double alpha, int nb, double *R, double *J) {
  int N = g->N, hw = (nb - 1) / 2;
  double res = or_residual1d(g, H, Q, R);
  memset(J, 0, sizeof(double) * (size_t)nb * 4 * N);
  for (int j = 0; j < N; ++j) {
    double R0[2] = {R[j], R[N + j]};
    for (int k = 0; k < nb; ++k) {
      int i = j + k - hw;
      if (i < 0 || i >= N) continue;
      for (int m = 0; m < 2; ++m) {
        double *U = (m == 0) ? H : Q;
        double save = U[i];
        U[i] = save + eps;
        double Rp[2];
        or_residual_cell1d(g, H, Q, j, Rp);
        U[i] = save;
        for (int l = 0; l < 2; ++l)
          J[(size_t)(k * 4 + l * 2 + m) * N + j] = (Rp[l] - R0[l]) / eps;
      }
    }
    double reg = alpha * (fabs(R0[0]) + fabs(R0[1]));
    J[(size_t)(hw * 4 + 0) * N + j] += reg;
    J[(size_t)(hw * 4 + 3) * N + j] += reg;
  }
  return res;
}

/* ------------------------------------------------------------------------ */
/* Multigrid (Section 3.4). Aggregation (Eq. 15): coarse cell c = fine cells
 * 2c and 2c+1; when the fine count is odd the last coarse cell holds one fine
 * cell (reading: the paper only uses even counts). */
int or_coarse_count(int Nf) { return (Nf + 1) / 2; }

/* Coarse operator (Eq. 17): J_{ji,l} = sum_{xi in agg j} sum_{eta in agg i}
 * J_{xi eta,l-1}. Input band nbf (3 or 5), output always 3 blocks (a 5-band
 * fine operator aggregates by pairs to a 3-band one). */
void or_coarse_operator1d(int Nf, int nbf, const double *Jf, double *Jc) {
  int Nc = or_coarse_count(Nf), hf = (nbf - 1) / 2;
  memset(Jc, 0, sizeof(double) * 3 * 4 * (size_t)Nc);
  for (int xi = 0; xi < Nf; ++xi) {
    int j = xi / 2;
    for (int k = 0; k < nbf; ++k) {
      int eta = xi + k - hf;
      if (eta < 0 || eta >= Nf) continue;
      int i = eta / 2;
      int kc = i - j + 1; /* 0..2, guaranteed by the band argument */
      for (int e = 0; e < 4; ++e)
        Jc[(size_t)(kc * 4 + e) * Nc + j] += Jf[(size_t)(k * 4 + e) * Nf + xi];
    }
  }
}

/* Inverse of each diagonal 2x2 block: Dinv[4][N]. */
void or_block_inverse1d(int N, int nb, const double *J, double *Dinv) {
  int hw = (nb - 1) / 2;
  for (int j = 0; j < N; ++j) {
    double a = J[(size_t)(hw * 4 + 0) * N + j], b = J[(size_t)(hw * 4 + 1) * N + j];
    double c = J[(size_t)(hw * 4 + 2) * N + j], d = J[(size_t)(hw * 4 + 3) * N + j];
    double det = a * d - b * c;
    Dinv[0 * N + j] = d / det;
    Dinv[1 * N + j] = -b / det;
    Dinv[2 * N + j] = -c / det;
    Dinv[3 * N + j] = a / det;
  }
}

/* One block-SOR update (Eq. 19) of every cell of colour col (j mod C == col):
 * dU_j <- (1-w) dU_j - w D_j^{-1} (R_j + sum_{i != j} J_ji dU_i). */
static void sor_colour1d(int N, int nb, const double *J, const double *Dinv,
                         const double *R, double *dU, double omega, int C,
                         int col) {
  int hw = (nb - 1) / 2;
  for (int j = col; j < N; j += C) {
    double r0 = R[j], r1 = R[N + j];
    for (int k = 0; k < nb; ++k) {
      int i = j + k - hw;
      if (k == hw || i < 0 || i >= N) continue;
      r0 += J[(size_t)(k * 4 + 0) * N + j] * dU[i] + J[(size_t)(k * 4 + 1) * N + j] * dU[N + i];
      r1 += J[(size_t)(k * 4 + 2) * N + j] * dU[i] + J[(size_t)(k * 4 + 3) * N + j] * dU[N + i];
    }
    double t0 = Dinv[0 * N + j] * r0 + Dinv[1 * N + j] * r1;
    double t1 = Dinv[2 * N + j] * r0 + Dinv[3 * N + j] * r1;
    dU[j] = (1.0 - omega) * dU[j] - omega * t0;
    dU[N + j] = (1.0 - omega) * dU[N + j] - omega * t1;
  }
}

/* One symmetric multicolour SOR step. Reading: the paper sweeps cells
 * lexicographically forward then backward (Eq. 19); the multicolour analogue
 * visits colours 0..C-1 then C-1..0, C = h+1 colours for a band of half-width
 * h (so same-colour cells never couple). */
void or_sor_step1d(int N, int nb, const double *J, const double *Dinv,
                   const double *R, double *dU, double omega) {
  int C = (nb - 1) / 2 + 1;
  for (int c = 0; c < C; ++c) sor_colour1d(N, nb, J, Dinv, R, dU, omega, C, c);
  for (int c = C - 1; c >= 0; --c) sor_colour1d(N, nb, J, Dinv, R, dU, omega, C, c);
}

/* Lexicographic symmetric SOR step exactly as Eq. 19 (forward j = 1..N, then
 * backward); kept to compare with the paper's ordering. */
void or_sor_step_lex1d(int N, int nb, const double *J, const double *Dinv,
                       const double *R, double *dU, double omega) {
  for (int pass = 0; pass < 2; ++pass)
    for (int s = 0; s < N; ++s) {
      int j = pass == 0 ? s : N - 1 - s;
      sor_colour1d(N, nb, J, Dinv, R, dU, omega, N + 1, j);
    }
}

/* Defect restriction (Eq. 17): Rc_j = sum_{xi in agg j} (R_xi + sum_eta
 * J_{xi eta} dU_eta). */
void or_restrict1d(int Nf, int nb, const double *J, const double *R,
                   const double *dU, double *Rc) {
  int Nc = or_coarse_count(Nf), hw = (nb - 1) / 2;
  memset(Rc, 0, sizeof(double) * 2 * (size_t)Nc);
  for (int xi = 0; xi < Nf; ++xi) {
    double r0 = R[xi], r1 = R[Nf + xi];
    for (int k = 0; k < nb; ++k) {
      int eta = xi + k - hw;
      if (eta < 0 || eta >= Nf) continue;
      r0 += J[(size_t)(k * 4 + 0) * Nf + xi] * dU[eta] + J[(size_t)(k * 4 + 1) * Nf + xi] * dU[Nf + eta];
      r1 += J[(size_t)(k * 4 + 2) * Nf + xi] * dU[eta] + J[(size_t)(k * 4 + 3) * Nf + xi] * dU[Nf + eta];
    }
    Rc[xi / 2] += r0;
    Rc[Nc + xi / 2] += r1;
  }
}

/* Prolongation (Eq. 18): dU_xi += dUc_{xi/2}. */
void or_prolong1d(int Nf, double *dU, const double *dUc) {
  int Nc = or_coarse_count(Nf);
  for (int xi = 0; xi < Nf; ++xi) {
    dU[xi] += dUc[xi / 2];
    dU[Nf + xi] += dUc[Nc + xi / 2];
  }
}

/* Dense LU with partial pivoting (ties to the lowest row), A row-major n x n,
 * overwritten; solves A x = b, x returned in b. Returns 0, or 1 if a pivot is
 * exactly zero. The paper only says "solve directly" (Algorithm 2). */
int or_dense_solve(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)p * n + k])) p = i;
    if (A[(size_t)p * n + k] == 0.0) return 1;
    if (p != k) {
      for (int c = 0; c < n; ++c) {
        double t = A[(size_t)k * n + c];
        A[(size_t)k * n + c] = A[(size_t)p * n + c];
        A[(size_t)p * n + c] = t;
      }
      double t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = l;
      for (int c = k + 1; c < n; ++c) A[(size_t)i * n + c] -= l * A[(size_t)k * n + c];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int c = i + 1; c < n; ++c) s -= A[(size_t)i * n + c] * b[c];
    b[i] = s / A[(size_t)i * n + i];
  }
  return 0;
}

/* Direct solve of the banded block system J dU = -R on N cells, unknown
 * ordering (cell-major: 2j = H, 2j+1 = Q). Returns 0 on success. */
int or_direct_solve1d(int N, int nb, const double *J, const double *R, double *dU) {
  int n = 2 * N, hw = (nb - 1) / 2;
  double *A = calloc((size_t)n * n, sizeof(double));
  double *b = malloc(sizeof(double) * n);
  for (int j = 0; j < N; ++j) {
    b[2 * j] = -R[j];
    b[2 * j + 1] = -R[N + j];
    for (int k = 0; k < nb; ++k) {
      int i = j + k - hw;
      if (i < 0 || i >= N) continue;
      for (int l = 0; l < 2; ++l)
        for (int m = 0; m < 2; ++m)
          A[(size_t)(2 * j + l) * n + 2 * i + m] = J[(size_t)(k * 4 + l * 2 + m) * N + j];
    }
  }
  int rc = or_dense_solve(n, A, b);
  for (int j = 0; j < N; ++j) {
    dU[j] = b[2 * j];
    dU[N + j] = b[2 * j + 1];
  }
  free(A);
  free(b);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Multigrid hierarchy for one linear system: levels 0..L of sizes N_l, level
 * 0 with band nb0, coarser levels band 3. */
typedef struct {
  int L, nb0;
  int N[32];
  double *J[32], *Dinv[32], *R[32], *dU[32];
  int ncolour_lex; /* 1: lexicographic smoother instead of multicolour */
} or_mg1d;

static void mg_alloc(or_mg1d *mg, int N0, int nlev, int nb0) {
  memset(mg, 0, sizeof(*mg));
  mg->L = nlev - 1;
  mg->nb0 = nb0;
  mg->N[0] = N0;
  for (int l = 1; l < nlev; ++l) mg->N[l] = or_coarse_count(mg->N[l - 1]);
  for (int l = 0; l < nlev; ++l) {
    int nb = l == 0 ? nb0 : 3;
    if (l > 0) mg->J[l] = malloc(sizeof(double) * nb * 4 * mg->N[l]);
    mg->Dinv[l] = malloc(sizeof(double) * 4 * mg->N[l]);
    if (l > 0) mg->R[l] = malloc(sizeof(double) * 2 * mg->N[l]);
    if (l > 0) mg->dU[l] = malloc(sizeof(double) * 2 * mg->N[l]);
  }
}

static void mg_free(or_mg1d *mg) {
  for (int l = 0; l <= mg->L; ++l) {
    if (l > 0) {
      free(mg->J[l]);
      free(mg->R[l]);
      free(mg->dU[l]);
    }
    free(mg->Dinv[l]);
  }
}

/* Build the coarse operators (Eq. 17) and diagonal inverses for all levels;
 * J is fixed during the V-cycles of one Newton step, so this is done once per
 * step (equivalent to building them inside each V-cycle of Algorithm 2). */
static void mg_setup(or_mg1d *mg) {
  for (int l = 1; l <= mg->L; ++l)
    or_coarse_operator1d(mg->N[l - 1], l == 1 ? mg->nb0 : 3, mg->J[l - 1], mg->J[l]);
  for (int l = 0; l <= mg->L; ++l)
    or_block_inverse1d(mg->N[l], l == 0 ? mg->nb0 : 3, mg->J[l], mg->Dinv[l]);
}

/* Algorithm 2: V-cycle MG_L(l, dU_l), in place on mg->dU[l]. */
static int mg_vcycle(or_mg1d *mg, int l, double omega, int nu1, int nu2) {
  int N = mg->N[l], nb = l == 0 ? mg->nb0 : 3;
  if (l == mg->L) return or_direct_solve1d(N, nb, mg->J[l], mg->R[l], mg->dU[l]);
  for (int s = 0; s < nu1; ++s) {
    if (mg->ncolour_lex) or_sor_step_lex1d(N, nb, mg->J[l], mg->Dinv[l], mg->R[l], mg->dU[l], omega);
    else or_sor_step1d(N, nb, mg->J[l], mg->Dinv[l], mg->R[l], mg->dU[l], omega);
  }
  or_restrict1d(N, nb, mg->J[l], mg->R[l], mg->dU[l], mg->R[l + 1]);
  memset(mg->dU[l + 1], 0, sizeof(double) * 2 * mg->N[l + 1]);
  int rc = mg_vcycle(mg, l + 1, omega, nu1, nu2);
  or_prolong1d(N, mg->dU[l], mg->dU[l + 1]);
  for (int s = 0; s < nu2; ++s) {
    if (mg->ncolour_lex) or_sor_step_lex1d(N, nb, mg->J[l], mg->Dinv[l], mg->R[l], mg->dU[l], omega);
    else or_sor_step1d(N, nb, mg->J[l], mg->Dinv[l], mg->R[l], mg->dU[l], omega);
  }
  return rc;
}

/* One V-cycle on the linear system J dU = -R (N cells, band nb) with a
 * hierarchy of nlev levels; dU in/out. Coarse operators are rebuilt from J. */
int or_vcycle1d(int N, int nb, int nlev, const double *J, const double *R,
                double *dU, double omega, int nu1, int nu2, int lex) {
  or_mg1d mg;
  mg_alloc(&mg, N, nlev, nb);
  mg.ncolour_lex = lex;
  mg.J[0] = (double *)J;
  mg.R[0] = (double *)R;
  mg.dU[0] = dU;
  mg_setup(&mg);
  int rc = mg_vcycle(&mg, 0, omega, nu1, nu2);
  mg_free(&mg);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Appendix A, Eq. A.2: fine averages from the coarse-level quadratic
 * (Eq. A.1) through coarse cells c-1, c, c+1. Reading: at the domain ends the
 * missing neighbour is the coarse level's ghost state (the same boundary
 * states the residual uses). */
void or_interp1d(const or_grid1d *gc, const double *Hc, const double *Qc,
                 double *Hf, double *Qf) {
  int Nc = gc->N, Nf = 2 * Nc;
  for (int c = 0; c < Nc; ++c) {
    double hm, qm, h0, q0, hp, qp;
    cell_value(gc, Hc, Qc, c - 1, &hm, &qm);
    cell_value(gc, Hc, Qc, c, &h0, &q0);
    cell_value(gc, Hc, Qc, c + 1, &hp, &qp);
    Hf[2 * c] = hm / 8.0 + h0 - hp / 8.0;
    Hf[2 * c + 1] = -hm / 8.0 + h0 + hp / 8.0;
    Qf[2 * c] = qm / 8.0 + q0 - qp / 8.0;
    Qf[2 * c + 1] = -qm / 8.0 + q0 + qp / 8.0;
  }
  (void)Nf;
}

/* ------------------------------------------------------------------------ */
/* Solver parameters (Section 5: alpha, tau, omega, nu1..nu3, levels, Tol).  */
typedef struct {
  double alpha, tau, omega, tol;
  int nu1, nu2, nu3, levels, n_max, nb, lex;
  int nest_start;        /* nested level the solve starts on (<0: coarsest) */
  double eps[32];        /* FD perturbation per nested level (Section 5.1) */
} or_params1d;

/* Per-solve record. */
typedef struct {
  int status;            /* 0 ok, 1 not converged, 2 NaN, 3 singular      */
  int iters[32];         /* Newton iterations per nested level            */
  double res[32];        /* final res per nested level                    */
  int total_iters;
  int vcycles;
} or_info1d;

/* Newton iteration on one nested level (Algorithm 1 with the linear solve of
 * Algorithm 3): at the coarsest level (nlev == 1) the regularized system is
 * solved directly; otherwise by nu3 V-cycles over nlev levels starting from
 * dU = 0. Returns the iteration count; *res_out = final res. */
static int newton_level1d(const or_grid1d *g, double *H, double *Q, int nlev,
                          double eps, const or_params1d *p, double *res_out,
                          int *vcycles, int *status) {
  int N = g->N;
  double *R = malloc(sizeof(double) * 2 * N);
  double *J = malloc(sizeof(double) * p->nb * 4 * N);
  double *dU = malloc(sizeof(double) * 2 * N);
  or_mg1d mg;
  mg_alloc(&mg, N, nlev, p->nb);
  mg.ncolour_lex = p->lex;
  mg.J[0] = J;
  mg.R[0] = R;
  mg.dU[0] = dU;
  int n = 0;
  double res = 0.0;
  *status = 0;
  do {
    or_jacobian1d(g, H, Q, eps, p->alpha, p->nb, R, J);
    memset(dU, 0, sizeof(double) * 2 * N);
    if (nlev == 1) {
      if (or_direct_solve1d(N, p->nb, J, R, dU)) { *status = 3; break; }
    } else {
      mg_setup(&mg);
      for (int m = 0; m < p->nu3; ++m) {
        if (mg_vcycle(&mg, 0, p->omega, p->nu1, p->nu2)) { *status = 3; break; }
        (*vcycles)++;
      }
      if (*status) break;
    }
    for (int j = 0; j < N; ++j) {
      H[j] += p->tau * dU[j];
      Q[j] += p->tau * dU[N + j];
    }
    res = or_residual1d(g, H, Q, R);
    ++n;
    if (!(res == res)) { *status = 2; break; }
  } while (!(res < p->tol) && n < p->n_max);
  if (*status == 0 && !(res < p->tol)) *status = 1;
  mg_free(&mg);
  free(R);
  free(J);
  free(dU);
  *res_out = res;
  return n;
}

/* Algorithm 3 (nested NMGM). grids[l] describes nested level l (l = 0 finest,
 * N_l = N_0 / 2^l); the multigrid hierarchy has p->levels = L+1 levels.
 * The solve starts on level s = p->nest_start (Algorithm 3: s = L, where the
 * regularized system is solved directly); on a level s < L the Newton
 * iteration uses V-cycles over levels s..L, exactly as on the finer levels.
 * Reading: starting above the coarsest grid is needed when the coarsest grid
 * under-resolves the channel geometry (its discrete problem then has no
 * smooth solution); Algorithm 3 is the special case s = L.
 * U0 = initial guess on level s (H then Q planes, N_s each); U = output on
 * the finest level (H then Q planes, N_0 each). */
int or_nmgm1d(const or_grid1d *grids, const double *U0, double *U,
              const or_params1d *p, or_info1d *info) {
  int L = p->levels - 1;
  int s0 = (p->nest_start < 0 || p->nest_start > L) ? L : p->nest_start;
  memset(info, 0, sizeof(*info));
  int NL = grids[s0].N;
  double *H = malloc(sizeof(double) * NL), *Q = malloc(sizeof(double) * NL);
  memcpy(H, U0, sizeof(double) * NL);
  memcpy(Q, U0 + NL, sizeof(double) * NL);
  for (int l = s0; l >= 0; --l) {
    if (l < s0) {
      int Nf = grids[l].N;
      double *Hf = malloc(sizeof(double) * Nf), *Qf = malloc(sizeof(double) * Nf);
      or_interp1d(&grids[l + 1], H, Q, Hf, Qf);
      free(H);
      free(Q);
      H = Hf;
      Q = Qf;
    }
    int st = 0;
    info->iters[l] = newton_level1d(&grids[l], H, Q, L - l + 1, p->eps[l], p,
                                    &info->res[l], &info->vcycles, &st);
    info->total_iters += info->iters[l];
    if (st) { info->status = st; if (st >= 2) break; }
  }
  int N0 = grids[0].N;
  if (info->status < 2) {
    memcpy(U, H, sizeof(double) * N0);
    memcpy(U + N0, Q, sizeof(double) * N0);
  }
  free(H);
  free(Q);
  return info->status;
}

/* Single-level regularized Newton (Algorithm 1) from a given guess on one
 * grid, linear solves by nu3 V-cycles over nlev levels (nlev = 1: direct). */
int or_newton1d(const or_grid1d *g, double *U, int nlev, double eps,
                const or_params1d *p, or_info1d *info) {
  memset(info, 0, sizeof(*info));
  int st = 0;
  info->iters[0] = newton_level1d(g, U, U + g->N, nlev, eps, p, &info->res[0],
                                  &info->vcycles, &st);
  info->total_iters = info->iters[0];
  info->status = st;
  return st;
}

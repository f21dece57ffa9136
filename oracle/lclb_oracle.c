/*
 * lclb_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of one time step of the hybrid lattice
 * Boltzmann / finite-difference method for colloids in a nematic or cholesteric
 * liquid crystal (Lintuvuori, Marenduzzo, Stratford, Cates, "Colloids in liquid
 * crystals: a lattice Boltzmann study", Sec. 2).  It exists to check the CUDA
 * path; only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may
 * load it.  It shares no code, header or table with the CUDA library.
 *
 * Every field is a full array; every pass of a step is a separate loop in the
 * order listed in step_once().  Reductions run serially in node order.
 *
 * Readings of the paper (where it is silent, the choice is stated at the
 * function that makes it):
 *   - LB: D3Q19, BGK with relaxation time tau, Guo forcing, half-way
 *     bounce-back on links with the moving-surface term (Sec. 2.2).
 *   - Distortion energy in the form that differs from Eq. 1 by a total
 *     divergence (the equivalence stated below Eq. 1).
 *   - Central first differences and the 7-point Laplacian; first-order upwind
 *     advective fluxes at control-volume faces (Sec. 2.2, Fig. 1).
 *   - Q update: explicit Euler of Eq. 2 with the Beris-Edwards co-rotation term.
 *   - Colloid: the "molecular dynamics-like step" of Sec. 2.2 taken implicit
 *     in the velocity-dependent part of the link force (colloid_update); a
 *     move into contact with another colloid or a wall is not made and is
 *     reported (contact_resolve; the paper treats no contact).
 *
 * Parity status: every function below is pinned by a CPU test, including the
 * surface value at colloid faces (homeotropic normal at the solid node,
 * planar projection of the largest-eigenvalue director, tie-break), the
 * LC torque (symmetry and the discrete angular-momentum balance), the
 * uncovered nodes of the re-discretisation (neighbour means, equilibrium),
 * the moving-surface bounce-back's mass balance and the contact rule
 * (hand-computed trajectories of node-free colloids), except the
 * drag-anisotropy and cholesteric defect-topology outcomes, which no printed
 * number of the paper fixes (parity unpinned against the paper; the CUDA path
 * is compared with this oracle only).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* D3Q19 lattice: velocities, weights (1/3, 1/18, 1/36), cs^2 = 1/3.   */
/* Order: rest; +x,-x,+y,-y,+z,-z; then the 12 diagonals in +/- pairs. */
/* ------------------------------------------------------------------ */
#define NQ 19
static const int CV[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double WQ(int i) {
  int s = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
  return s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

static int OPP(int i) {
  for (int j = 0; j < NQ; ++j)
    if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) return j;
  return -1;
}

/* Levi-Civita symbol. */
static double EPS(int a, int b, int c) {
  if (a == b || b == c || a == c) return 0.0;
  if ((a == 0 && b == 1 && c == 2) || (a == 1 && b == 2 && c == 0) || (a == 2 && b == 0 && c == 1))
    return 1.0;
  return -1.0;
}

/* Compensated summation (Neumaier's variant of Kahan summation) for the
 * global FP64 sums, so that their rounding error does not grow with N. */
typedef struct { double s, c; } ksum;
static void kadd(ksum* k, double v) {
  double t = k->s + v;
  if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
  else k->c += (v - t) + k->s;
  k->s = t;
}
static double kval(const ksum* k) { return k->s + k->c; }

#define OMAXC 64

typedef struct {
  double X[3], V[3], W[3];
  double a0, w; /* w <= 0 or inf: strong anchoring (the paper's fixed Q0) */
  int anchoring; /* 0 = normal (homeotropic), 1 = planar */
  int mobile;
  double Fext[3], Text[3]; /* external force and torque */
  double M, I;
  double Fh[3], Th[3], Flc[3], Tlc[3]; /* forces and torques of the last step */
  double imp[3], aimp[3];              /* momentum / angular momentum received */
  double zv[3][3], zw[3][3];           /* link drag tensors of the last step (see colloid_update) */
} ocolloid;

typedef struct {
  int nx, ny, nz, wall_z;
  long N;
  double rho0, tau, A0, gam, K, q0, xi, Gam, S0;
  double g[3];
  int lc_on, flow_on;
  int ncol;
  ocolloid col[OMAXC];
  int16_t *solid; /* -1 fluid, c >= 0 inside colloid c */
  double *f, *fpost, *Q, *Qnew, *H, *P, *F, *u, *fe;
  long step;
  double resid_rms, resid_max;
  int nthreads;
  int last_error;
  long contact_step; /* first contact since the caller last read it (-1: none), see contact_resolve */
  int contact_c, contact_d;
} oracle;

/* ------------------------------------------------------------------ */
/* Geometry helpers                                                    */
/* ------------------------------------------------------------------ */
static int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

/* Neighbour node index, or -1 beyond a no-slip wall in z. */
static long nbr(const oracle* o, int x, int y, int z, int dx, int dy, int dz) {
  int X = wrapi(x + dx, o->nx), Y = wrapi(y + dy, o->ny), Z = z + dz;
  if (o->wall_z) {
    if (Z < 0 || Z >= o->nz) return -1;
  } else {
    Z = wrapi(Z, o->nz);
  }
  return (long)X + (long)o->nx * ((long)Y + (long)o->ny * (long)Z);
}

/* Minimum-image difference along one axis (periodic axes only). */
static double minimg(double d, int L, int periodic) {
  if (!periodic) return d;
  if (d >= 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

static void node_disp(const oracle* o, double x, double y, double z, const double X[3], double d[3]) {
  d[0] = minimg(x - X[0], o->nx, 1);
  d[1] = minimg(y - X[1], o->ny, 1);
  d[2] = minimg(z - X[2], o->nz, !o->wall_z);
}

/* Solid test (Sec. 2.2: inside/outside from the nominal radius a0 and the
 * position).  |d|^2 summed left to right; this file is compiled with
 * -ffp-contract=off so no fused multiply-add changes the rounding.  A node
 * exactly on the surface is fluid. */
static int inside(const oracle* o, int x, int y, int z, const ocolloid* c) {
  double d[3];
  node_disp(o, (double)x, (double)y, (double)z, c->X, d);
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  return r2 < c->a0 * c->a0;
}

static void build_solid(oracle* o, int16_t* out) {
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        int s = -1;
        for (int c = 0; c < o->ncol && s < 0; ++c)
          if (inside(o, x, y, z, &o->col[c])) s = c;
        out[i] = (int16_t)s;
      }
}

/* ------------------------------------------------------------------ */
/* Small tensor helpers                                                */
/* ------------------------------------------------------------------ */
static void q_get(const oracle* o, const double* Q5, long i, double q[3][3]) {
  long N = o->N;
  double xx = Q5[0 * N + i], xy = Q5[1 * N + i], xz = Q5[2 * N + i], yy = Q5[3 * N + i], yz = Q5[4 * N + i];
  q[0][0] = xx; q[0][1] = xy; q[0][2] = xz;
  q[1][0] = xy; q[1][1] = yy; q[1][2] = yz;
  q[2][0] = xz; q[2][1] = yz; q[2][2] = -xx - yy;
}

static void q_put(const oracle* o, double* Q5, long i, double q[3][3]) {
  long N = o->N;
  Q5[0 * N + i] = q[0][0]; Q5[1 * N + i] = q[0][1]; Q5[2 * N + i] = q[0][2];
  Q5[3 * N + i] = q[1][1]; Q5[4 * N + i] = q[1][2];
}

/* Closed-form bulk order parameter of the uniaxial minimum of the bulk part
 * of Eq. 1: q = 1/4 + 3/4 sqrt(1 - 8/(3 gamma)) (gives q = 1/2 at gamma = 3,
 * the value printed with the parameters of Sec. 2.1). */
static double bulk_q(double gam) {
  double t = 1.0 - 8.0 / (3.0 * gam);
  if (t < 0.0) return 0.0;
  return 0.25 + 0.75 * sqrt(t);
}

/* Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
 * (textbook method).  Eigenvalues in ev[k], eigenvectors in columns v[.][k]. */
static void jacobi3(const double A_in[3][3], double ev[3], double v[3][3]) {
  double a[3][3];
  memcpy(a, A_in, sizeof(a));
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) v[p][q] = (p == q) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
    if (off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) { /* A <- A J */
          double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) { /* A <- J^T A */
          double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int k = 0; k < 3; ++k) ev[k] = a[k][k];
}

static void principal_dir(const double q[3][3], double n[3]) {
  double ev[3], v[3][3];
  jacobi3(q, ev, v);
  int k = 0;
  if (ev[1] > ev[k]) k = 1;
  if (ev[2] > ev[k]) k = 2;
  for (int a = 0; a < 3; ++a) n[a] = v[a][k];
}

/* ------------------------------------------------------------------ */
/* Order-parameter boundary value at a solid node (Sec. 2.2, Eq. 7).   */
/* ------------------------------------------------------------------ */
/* Surface value seen by fluid node (its Q is qf) across the face to solid
 * node (sx,sy,sz) of colloid c, or to a wall when c < 0.
 *  - homeotropic: n0 = unit outward normal s at the solid node;
 *  - planar: n0 = projection of the fluid node's director (principal
 *    eigenvector of qf) on the tangent plane normal to s;
 *  - Q0 = S0 (n0 n0 - delta/3) (Eq. 7);
 *  - strong anchoring (the paper's rule): the solid node takes Q0;
 *  - finite anchoring strength w: the value minimising the surface term
 *    (w/2)|Qs - Q0|^2 plus the face gradient term (K/2)|Qs - qf|^2, i.e.
 *    Qs = (K qf + w Q0)/(K + w), which tends to Q0 as w -> infinity.
 * Walls (z) carry strong homeotropic anchoring along z. */
static int strong_w(double w) { return !(w > 0.0) || isinf(w); }

static void surface_q0(const oracle* o, int c, int sx, int sy, int sz, const double qf[3][3], double q0[3][3]) {
  double n0[3];
  if (c < 0) {
    n0[0] = 0.0; n0[1] = 0.0; n0[2] = 1.0;
  } else {
    const ocolloid* C = &o->col[c];
    double d[3];
    node_disp(o, (double)sx, (double)sy, (double)sz, C->X, d);
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double s[3] = {d[0] / r, d[1] / r, d[2] / r};
    if (C->anchoring == 0) {
      n0[0] = s[0]; n0[1] = s[1]; n0[2] = s[2];
    } else {
      double nf[3];
      principal_dir(qf, nf);
      double ns = nf[0] * s[0] + nf[1] * s[1] + nf[2] * s[2];
      double p[3] = {nf[0] - ns * s[0], nf[1] - ns * s[1], nf[2] - ns * s[2]};
      double pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
      if (pn < 1e-12) { /* director along the normal: tangent s x e_k, k least aligned with s */
        int k = 0;
        if (fabs(s[1]) < fabs(s[k])) k = 1;
        if (fabs(s[2]) < fabs(s[k])) k = 2;
        double e[3] = {0, 0, 0};
        e[k] = 1.0;
        p[0] = s[1] * e[2] - s[2] * e[1];
        p[1] = s[2] * e[0] - s[0] * e[2];
        p[2] = s[0] * e[1] - s[1] * e[0];
        pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
      }
      n0[0] = p[0] / pn; n0[1] = p[1] / pn; n0[2] = p[2] / pn;
    }
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) q0[a][b] = o->S0 * (n0[a] * n0[b] - (a == b ? 1.0 / 3.0 : 0.0));
}

static void ghost_q(const oracle* o, int c, int sx, int sy, int sz, const double qf[3][3], double qs[3][3]) {
  double q0[3][3];
  surface_q0(o, c, sx, sy, sz, qf, q0);
  double w = (c < 0) ? 0.0 : o->col[c].w;
  if (strong_w(w)) {
    memcpy(qs, q0, sizeof(q0));
  } else {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) qs[a][b] = (o->K * qf[a][b] + w * q0[a][b]) / (o->K + w);
  }
}

/* Q at the six face neighbours of fluid node (x,y,z): the neighbour's Q
 * if fluid, else the surface value.  qn[axis][0] is the + side, [1] the -. */
static void face_neighbour_q(const oracle* o, const double* Q5, int x, int y, int z, const double qi[3][3],
                             double qn[3][2][3][3]) {
  for (int ax = 0; ax < 3; ++ax)
    for (int sgn = 0; sgn < 2; ++sgn) {
      int d[3] = {0, 0, 0};
      d[ax] = sgn == 0 ? 1 : -1;
      long j = nbr(o, x, y, z, d[0], d[1], d[2]);
      if (j >= 0 && o->solid[j] < 0) {
        q_get(o, Q5, j, qn[ax][sgn]);
      } else {
        int sx = wrapi(x + d[0], o->nx), sy = wrapi(y + d[1], o->ny), sz = z + d[2];
        if (!o->wall_z) sz = wrapi(sz, o->nz);
        int c = (j >= 0) ? o->solid[j] : -1;
        ghost_q(o, c, sx, sy, sz, qi, qn[ax][sgn]);
      }
    }
}

/* ------------------------------------------------------------------ */
/* Molecular field, free energy density and stress (Eqs. 1, 2, 4)      */
/* ------------------------------------------------------------------ */
/* H = -dF/dQ + (1/3) Tr(dF/dQ) I for the free energy of Eq. 1, written as
 *   f' = f_bulk + K/2 (d_g Q_ab)^2 + 2 K q0 eps_agd Q_ab d_g Q_db + 2 K q0^2 Q_ab Q_ab
 * (equal to Eq. 1 up to a total divergence).  Its variational derivative is
 *   H = -A0(1-g/3) Q + A0 g (Q.Q - Tr(Q^2)/3 I) - A0 g Tr(Q^2) Q + K lap Q
 *       - 2 K q0 (eps_agd d_g Q_db + eps_bgd d_g Q_da) - 4 K q0^2 Q.
 * dq[g][a][b] = d_g Q_ab. */
static void molecular_field(const oracle* o, const double q[3][3], const double dq[3][3][3], const double lap[3][3],
                            double h[3][3]) {
  double A0 = o->A0, gm = o->gam, K = o->K, q0 = o->q0;
  double q2[3][3], trq2 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      q2[a][b] = 0.0;
      for (int c = 0; c < 3; ++c) q2[a][b] += q[a][c] * q[c][b];
      trq2 += q[a][b] * q[a][b];
    }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double chi = 0.0;
      for (int g = 0; g < 3; ++g)
        for (int d = 0; d < 3; ++d) chi += EPS(a, g, d) * dq[g][d][b] + EPS(b, g, d) * dq[g][d][a];
      h[a][b] = -A0 * (1.0 - gm / 3.0) * q[a][b] + A0 * gm * (q2[a][b] - (a == b ? trq2 / 3.0 : 0.0)) -
                A0 * gm * trq2 * q[a][b] + K * lap[a][b] - 2.0 * K * q0 * chi - 4.0 * K * q0 * q0 * q[a][b];
    }
}

/* Free energy density f' (the divergence-equivalent form of Eq. 1). */
static double free_energy_density(const oracle* o, const double q[3][3], const double dq[3][3][3]) {
  double A0 = o->A0, gm = o->gam, K = o->K, q0 = o->q0;
  double trq2 = 0.0, trq3 = 0.0, grad2 = 0.0, chi = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      trq2 += q[a][b] * q[a][b];
      for (int c = 0; c < 3; ++c) trq3 += q[a][b] * q[b][c] * q[c][a];
    }
  for (int g = 0; g < 3; ++g)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) grad2 += dq[g][a][b] * dq[g][a][b];
  for (int a = 0; a < 3; ++a)
    for (int g = 0; g < 3; ++g)
      for (int d = 0; d < 3; ++d)
        for (int b = 0; b < 3; ++b) chi += EPS(a, g, d) * q[a][b] * dq[g][d][b];
  double fb = 0.5 * A0 * (1.0 - gm / 3.0) * trq2 - A0 * gm / 3.0 * trq3 + 0.25 * A0 * gm * trq2 * trq2;
  return fb + 0.5 * K * grad2 + 2.0 * K * q0 * chi + 2.0 * K * q0 * q0 * trq2;
}

/* Stress of Eq. 4 with the isotropic pressure read as P0 = rho cs^2 - f'
 * (the rho cs^2 part is carried by the LB, so +f' delta enters here):
 *   P_ab = f' d_ab + 2 xi (Q_ab + d_ab/3) Q:H - xi H_ag (Q_gb + d_gb/3)
 *          - xi (Q_ag + d_ag/3) H_gb - d_a Q_gn Pi_b,gn + Q_ag H_gb - H_ag Q_gb,
 * with Pi_b,gn = df'/d(d_b Q_gn) = K d_b Q_gn + K q0 (eps_mbg Q_mn + eps_mbn Q_mg). */
static void stress(const oracle* o, const double q[3][3], const double dq[3][3][3], const double h[3][3],
                   double fprime, double p[3][3]) {
  double K = o->K, q0 = o->q0, xi = o->xi;
  double pi[3][3][3];
  for (int b = 0; b < 3; ++b)
    for (int g = 0; g < 3; ++g)
      for (int n = 0; n < 3; ++n) {
        double ch = 0.0;
        for (int m = 0; m < 3; ++m) ch += EPS(m, b, g) * q[m][n] + EPS(m, b, n) * q[m][g];
        pi[b][g][n] = K * dq[b][g][n] + K * q0 * ch;
      }
  double qh = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) qh += q[a][b] * h[a][b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double dab = (a == b) ? 1.0 : 0.0;
      double t = fprime * dab + 2.0 * xi * (q[a][b] + dab / 3.0) * qh;
      for (int g = 0; g < 3; ++g) {
        double dgb = (g == b) ? 1.0 : 0.0, dag = (a == g) ? 1.0 : 0.0;
        t -= xi * h[a][g] * (q[g][b] + dgb / 3.0);
        t -= xi * (q[a][g] + dag / 3.0) * h[g][b];
        t += q[a][g] * h[g][b] - h[a][g] * q[g][b];
        for (int n = 0; n < 3; ++n) t -= dq[a][g][n] * pi[b][g][n];
      }
      p[a][b] = t;
    }
}

/* Derivatives at fluid node (x,y,z) from the face-neighbour values:
 * central first differences and the 7-point Laplacian (Sec. 2.2: one
 * finite-difference stencil at all fluid nodes, with the surface values
 * standing in for solid neighbours). */
static void derivatives(const double qi[3][3], double qn[3][2][3][3], double dq[3][3][3], double lap[3][3]) {
  for (int g = 0; g < 3; ++g)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) dq[g][a][b] = 0.5 * (qn[g][0][a][b] - qn[g][1][a][b]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int g = 0; g < 3; ++g) s += qn[g][0][a][b] + qn[g][1][a][b];
      lap[a][b] = s - 6.0 * qi[a][b];
    }
}

/* H, f' and P at every fluid node of the current Q. */
static void lc_fields(oracle* o) {
  long N = o->N;
#pragma omp parallel for schedule(static) num_threads(o->nthreads)
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (o->solid[i] >= 0) {
          for (int k = 0; k < 5; ++k) o->H[k * N + i] = 0.0;
          for (int k = 0; k < 9; ++k) o->P[k * N + i] = 0.0;
          o->fe[i] = 0.0;
          continue;
        }
        double qi[3][3], qn[3][2][3][3], dq[3][3][3], lap[3][3], h[3][3], p[3][3];
        q_get(o, o->Q, i, qi);
        face_neighbour_q(o, o->Q, x, y, z, qi, qn);
        derivatives(qi, qn, dq, lap);
        molecular_field(o, qi, dq, lap, h);
        double fp = free_energy_density(o, qi, dq);
        stress(o, qi, dq, h, fp, p);
        q_put(o, o->H, i, h);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) o->P[(3 * a + b) * N + i] = p[a][b];
        o->fe[i] = fp;
      }
}

/* Body force on the fluid: discrete divergence of P over control-volume
 * faces (Sec. 2.2).  A fluid-fluid face carries (P_i + P_j)/2; a face to a
 * solid node or a wall carries P_i (extrapolation).  The colloid receives
 * the opposite of each of its faces' contributions (Eq. 8, summed over the
 * solid-fluid faces), and the torque of that force about its centre taken
 * at the face centre. */
static void lc_force(oracle* o) {
  long N = o->N;
  ksum Fc[OMAXC][3], Tc[OMAXC][3];
  memset(Fc, 0, sizeof(Fc));
  memset(Tc, 0, sizeof(Tc));
  for (long k = 0; k < 3 * N; ++k) o->F[k] = 0.0;
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (o->solid[i] >= 0) continue;
        double Fi[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d)
          for (int sgn = 0; sgn < 2; ++sgn) {
            int e[3] = {0, 0, 0};
            double s = sgn == 0 ? 1.0 : -1.0;
            e[d] = sgn == 0 ? 1 : -1;
            long j = nbr(o, x, y, z, e[0], e[1], e[2]);
            int fluid_j = (j >= 0 && o->solid[j] < 0);
            for (int a = 0; a < 3; ++a) {
              double pf = fluid_j ? 0.5 * (o->P[(3 * a + d) * N + i] + o->P[(3 * a + d) * N + j])
                                  : o->P[(3 * a + d) * N + i];
              Fi[a] += s * pf;
            }
            if (j >= 0 && o->solid[j] >= 0) {
              int c = o->solid[j];
              double ff[3], r[3], t[3];
              for (int a = 0; a < 3; ++a) ff[a] = -s * o->P[(3 * a + d) * N + i];
              double fx = x + 0.5 * e[0], fy = y + 0.5 * e[1], fz = z + 0.5 * e[2];
              node_disp(o, fx, fy, fz, o->col[c].X, r);
              t[0] = r[1] * ff[2] - r[2] * ff[1];
              t[1] = r[2] * ff[0] - r[0] * ff[2];
              t[2] = r[0] * ff[1] - r[1] * ff[0];
              for (int a = 0; a < 3; ++a) {
                kadd(&Fc[c][a], ff[a]);
                kadd(&Tc[c][a], t[a]);
              }
            }
          }
        for (int a = 0; a < 3; ++a) o->F[a * N + i] = Fi[a];
      }
  for (int c = 0; c < o->ncol; ++c)
    for (int a = 0; a < 3; ++a) {
      o->col[c].Flc[a] = kval(&Fc[c][a]);
      o->col[c].Tlc[a] = kval(&Tc[c][a]);
    }
}

/* Rigid-body velocity V + Omega x (r - X) of colloid c at point r. */
static void rigid_u(const oracle* o, int c, double x, double y, double z, double u[3]) {
  const ocolloid* C = &o->col[c];
  double d[3];
  node_disp(o, x, y, z, C->X, d);
  u[0] = C->V[0] + C->W[1] * d[2] - C->W[2] * d[1];
  u[1] = C->V[1] + C->W[2] * d[0] - C->W[0] * d[2];
  u[2] = C->V[2] + C->W[0] * d[1] - C->W[1] * d[0];
}

/* Density and velocity: rho = sum f, u = (sum f c + Ftot/2)/rho at fluid
 * nodes (Guo forcing); solid nodes take the rigid-body velocity (Sec. 2.2). */
static void moments(oracle* o) {
  long N = o->N;
#pragma omp parallel for schedule(static) num_threads(o->nthreads)
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (o->solid[i] >= 0) {
          double ur[3];
          rigid_u(o, o->solid[i], x, y, z, ur);
          for (int a = 0; a < 3; ++a) o->u[a * N + i] = o->flow_on ? ur[a] : 0.0;
          continue;
        }
        if (!o->flow_on) {
          for (int a = 0; a < 3; ++a) o->u[a * N + i] = 0.0;
          continue;
        }
        double rho = 0.0, m[3] = {0, 0, 0};
        for (int q = 0; q < NQ; ++q) {
          double fq = o->f[q * N + i];
          rho += fq;
          for (int a = 0; a < 3; ++a) m[a] += fq * CV[q][a];
        }
        for (int a = 0; a < 3; ++a) o->u[a * N + i] = (m[a] + 0.5 * (o->F[a * N + i] + o->g[a])) / rho;
      }
}

/* Q^{n+1} = Q^n + dt [Gamma H + S - div(u Q)] (Eq. 2 with the Beris-Edwards
 * material derivative).  Velocity gradient W_ab = d_b u_a by central
 * differences, with solid neighbours at the rigid-body velocity and walls at
 * rest (Sec. 2.2).  Co-rotation term
 *   S = (xi D + Om)(Q + I/3) + (Q + I/3)(xi D - Om) - 2 xi (Q + I/3) Tr(Q W),
 * D = (W + W^T)/2, Om = (W - W^T)/2.  Advective fluxes at control-volume
 * faces, first-order upwind, zero across solid-fluid faces (Sec. 2.2).  The
 * increment is projected onto traceless tensors (S carries a trace of
 * 2 xi div(u)/3 in a weakly compressible flow).  The residual is the RMS over
 * fluid nodes of the 9 entries of the increment, and its largest entry. */
static void q_update(oracle* o) {
  long N = o->N;
  ksum* ss = (ksum*)calloc((size_t)o->nz, sizeof(ksum));
  double* mx = (double*)calloc((size_t)o->nz, sizeof(double));
  long nfl = 0;
  for (long i = 0; i < N; ++i) nfl += (o->solid[i] < 0);
#pragma omp parallel for schedule(static) num_threads(o->nthreads)
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (o->solid[i] >= 0) {
          for (int k = 0; k < 5; ++k) o->Qnew[k * N + i] = o->Q[k * N + i];
          continue;
        }
        double qi[3][3], h[3][3];
        q_get(o, o->Q, i, qi);
        q_get(o, o->H, i, h);
        double W[3][3], adv[3][3];
        memset(adv, 0, sizeof(adv));
        for (int b = 0; b < 3; ++b) {
          double up[3], um[3];
          for (int sgn = 0; sgn < 2; ++sgn) {
            int e[3] = {0, 0, 0};
            e[b] = sgn == 0 ? 1 : -1;
            long j = nbr(o, x, y, z, e[0], e[1], e[2]);
            double* uu = sgn == 0 ? up : um;
            if (j < 0) {
              uu[0] = uu[1] = uu[2] = 0.0;
            } else {
              for (int a = 0; a < 3; ++a) uu[a] = o->u[a * N + j];
            }
            /* advective flux through this face */
            if (j >= 0 && o->solid[j] < 0) {
              double uf = 0.5 * (o->u[b * N + i] + o->u[b * N + j]);
              double qj[3][3];
              q_get(o, o->Q, j, qj);
              /* flux leaving i through the + face, or entering through the - face */
              for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                  double qup;
                  if (sgn == 0) qup = (uf > 0.0) ? qi[a][c] : qj[a][c];
                  else qup = (uf > 0.0) ? qj[a][c] : qi[a][c];
                  double fl = uf * qup;
                  adv[a][c] += (sgn == 0) ? fl : -fl;
                }
            }
          }
          for (int a = 0; a < 3; ++a) W[a][b] = 0.5 * (up[a] - um[a]);
        }
        double D[3][3], Om[3][3], Qt[3][3], trQW = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            D[a][b] = 0.5 * (W[a][b] + W[b][a]);
            Om[a][b] = 0.5 * (W[a][b] - W[b][a]);
            Qt[a][b] = qi[a][b] + (a == b ? 1.0 / 3.0 : 0.0);
          }
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) trQW += qi[a][b] * W[b][a];
        double dQ[3][3], tr = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c)
              s += (o->xi * D[a][c] + Om[a][c]) * Qt[c][b] + Qt[a][c] * (o->xi * D[c][b] - Om[c][b]);
            s -= 2.0 * o->xi * Qt[a][b] * trQW;
            dQ[a][b] = o->Gam * h[a][b] + s - adv[a][b];
          }
        for (int a = 0; a < 3; ++a) tr += dQ[a][a];
        for (int a = 0; a < 3; ++a) dQ[a][a] -= tr / 3.0;
        double qn[3][3], s2 = 0.0, m = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            qn[a][b] = qi[a][b] + dQ[a][b];
            s2 += dQ[a][b] * dQ[a][b];
            if (fabs(dQ[a][b]) > m) m = fabs(dQ[a][b]);
          }
        q_put(o, o->Qnew, i, qn);
        kadd(&ss[z], s2);
        if (m > mx[z]) mx[z] = m;
      }
  ksum tot = {0, 0};
  double mmax = 0.0;
  for (int z = 0; z < o->nz; ++z) {
    kadd(&tot, kval(&ss[z]));
    if (mx[z] > mmax) mmax = mx[z];
  }
  o->resid_rms = nfl > 0 ? sqrt(kval(&tot) / (double)nfl) : 0.0;
  o->resid_max = mmax;
  free(ss);
  free(mx);
  double* t = o->Q;
  o->Q = o->Qnew;
  o->Qnew = t;
}

/* LB collision (BGK, relaxation time tau) with Guo forcing of the total
 * force Ftot = F_LC + g, then streaming with half-way bounce-back on links
 * (Sec. 2.2).  A population leaving fluid node r along c_b towards a solid
 * node of colloid c returns to r along -c_b as
 *     f_{-b}(r, t+1) = f*_b(r, t) - 6 w_b rho0 (c_b . u_b),
 * u_b the rigid velocity at the link midpoint r + c_b/2.  The momentum
 * handed to the colloid per link is c_b (2 (f*_b - w_b rho0) - 6 w_b rho0
 * c_b.u_b); the w_b rho0 part is left out because over a closed surface the
 * links along c_b and -c_b pair up and it sums to zero.  Walls (z) are at
 * rest. */
static void feq_full(double rho, const double u[3], double out[NQ]) {
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int q = 0; q < NQ; ++q) {
    double cu = CV[q][0] * u[0] + CV[q][1] * u[1] + CV[q][2] * u[2];
    out[q] = WQ(q) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
  }
}

static void collide_stream(oracle* o) {
  long N = o->N;
  double om = 1.0 / o->tau, pref = 1.0 - 0.5 / o->tau;
#pragma omp parallel for schedule(static) num_threads(o->nthreads)
  for (long i = 0; i < N; ++i) {
    if (o->solid[i] >= 0) {
      for (int q = 0; q < NQ; ++q) o->fpost[q * N + i] = 0.0;
      continue;
    }
    double rho = 0.0, u[3], Ft[3], feq[NQ];
    for (int q = 0; q < NQ; ++q) rho += o->f[q * N + i];
    for (int a = 0; a < 3; ++a) {
      u[a] = o->u[a * N + i];
      Ft[a] = o->F[a * N + i] + o->g[a];
    }
    feq_full(rho, u, feq);
    for (int q = 0; q < NQ; ++q) {
      double cu = CV[q][0] * u[0] + CV[q][1] * u[1] + CV[q][2] * u[2];
      double src = 0.0;
      for (int a = 0; a < 3; ++a) src += (3.0 * (CV[q][a] - u[a]) + 9.0 * cu * CV[q][a]) * Ft[a];
      double fq = o->f[q * N + i];
      o->fpost[q * N + i] = fq - om * (fq - feq[q]) + pref * WQ(q) * src;
    }
  }
  ksum Fh[OMAXC][3], Th[OMAXC][3];
  memset(Fh, 0, sizeof(Fh));
  memset(Th, 0, sizeof(Th));
  for (int c = 0; c < o->ncol; ++c) {
    memset(o->col[c].zv, 0, sizeof(o->col[c].zv));
    memset(o->col[c].zw, 0, sizeof(o->col[c].zw));
  }
  for (long k = 0; k < NQ * N; ++k) o->f[k] = 0.0;
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (o->solid[i] >= 0) continue;
        for (int q = 0; q < NQ; ++q) {
          double fs = o->fpost[q * N + i];
          long j = nbr(o, x, y, z, CV[q][0], CV[q][1], CV[q][2]);
          if (j >= 0 && o->solid[j] < 0) {
            o->f[q * N + j] = fs;
          } else if (j < 0) {
            o->f[OPP(q) * N + i] = fs;
          } else {
            int c = o->solid[j];
            double ub[3], r[3], dp[3], t[3];
            double mx = x + 0.5 * CV[q][0], my = y + 0.5 * CV[q][1], mz = z + 0.5 * CV[q][2];
            rigid_u(o, c, mx, my, mz, ub);
            double cub = CV[q][0] * ub[0] + CV[q][1] * ub[1] + CV[q][2] * ub[2];
            double corr = 6.0 * WQ(q) * o->rho0 * cub;
            o->f[OPP(q) * N + i] = fs - corr;
            double dev = fs - WQ(q) * o->rho0;
            for (int a = 0; a < 3; ++a) dp[a] = CV[q][a] * (2.0 * dev - corr);
            node_disp(o, mx, my, mz, o->col[c].X, r);
            t[0] = r[1] * dp[2] - r[2] * dp[1];
            t[1] = r[2] * dp[0] - r[0] * dp[2];
            t[2] = r[0] * dp[1] - r[1] * dp[0];
            for (int a = 0; a < 3; ++a) {
              kadd(&Fh[c][a], dp[a]);
              kadd(&Th[c][a], t[a]);
            }
            /* the part of dp linear in the rigid velocity is
             * -6 w rho0 c (c.(V + Omega x r)); its V-V and Omega-Omega
             * coefficients (c c and (r x c)(r x c), times 6 w rho0) */
            double rc[3] = {r[1] * CV[q][2] - r[2] * CV[q][1], r[2] * CV[q][0] - r[0] * CV[q][2],
                            r[0] * CV[q][1] - r[1] * CV[q][0]};
            double zk = 6.0 * WQ(q) * o->rho0;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) {
                o->col[c].zv[a][b] += zk * CV[q][a] * CV[q][b];
                o->col[c].zw[a][b] += zk * rc[a] * rc[b];
              }
          }
        }
      }
  for (int c = 0; c < o->ncol; ++c)
    for (int a = 0; a < 3; ++a) {
      o->col[c].Fh[a] = kval(&Fh[c][a]);
      o->col[c].Th[a] = kval(&Th[c][a]);
    }
}

/* Re-discretisation after the colloid moved (Sec. 2.2, last paragraph):
 * a node that becomes solid hands its fluid momentum to the colloid; a node
 * that becomes fluid takes f = f_eq(rho_bar, u_b) with rho_bar the mean
 * density of its fluid face neighbours (rho0 if none) and u_b the rigid
 * velocity there, whose momentum the colloid gives up, and Q = the mean of
 * its fluid face neighbours (+x,-x,+y,-y,+z,-z order).  The momentum
 * exchanged is summed per colloid (u_b taken with the velocity before the
 * exchange) and then changes the colloid's velocity by dp/M, so that fluid
 * momentum + M V is conserved. */
static void rediscretise(oracle* o) {
  long N = o->N;
  int16_t* ns = (int16_t*)malloc(sizeof(int16_t) * (size_t)N);
  build_solid(o, ns);
  int changed = 0;
  for (long i = 0; i < N; ++i)
    if (ns[i] != o->solid[i]) { changed = 1; break; }
  if (!changed) { free(ns); return; }
  double dpc[OMAXC][3];
  memset(dpc, 0, sizeof(dpc));
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (o->solid[i] < 0 && ns[i] >= 0) { /* covered */
          int c = ns[i];
          for (int q = 0; q < NQ; ++q)
            for (int a = 0; a < 3; ++a) {
              o->col[c].imp[a] += o->f[q * N + i] * CV[q][a];
              dpc[c][a] += o->f[q * N + i] * CV[q][a];
            }
          for (int q = 0; q < NQ; ++q) o->f[q * N + i] = 0.0;
        }
      }
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (o->solid[i] >= 0 && ns[i] < 0) { /* uncovered */
          int c = o->solid[i];
          double rsum = 0.0, qsum[3][3];
          int cnt = 0;
          memset(qsum, 0, sizeof(qsum));
          for (int ax = 0; ax < 3; ++ax)
            for (int sgn = 0; sgn < 2; ++sgn) {
              int e[3] = {0, 0, 0};
              e[ax] = sgn == 0 ? 1 : -1;
              long j = nbr(o, x, y, z, e[0], e[1], e[2]);
              if (j < 0 || ns[j] >= 0 || o->solid[j] >= 0) continue;
              double rj = 0.0, qj[3][3];
              for (int q = 0; q < NQ; ++q) rj += o->f[q * N + j];
              q_get(o, o->Q, j, qj);
              rsum += rj;
              for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) qsum[a][b] += qj[a][b];
              ++cnt;
            }
          double rb = cnt ? rsum / cnt : o->rho0;
          double ub[3], feq[NQ];
          rigid_u(o, c, x, y, z, ub);
          feq_full(rb, ub, feq);
          for (int q = 0; q < NQ; ++q) o->f[q * N + i] = feq[q];
          for (int a = 0; a < 3; ++a) {
            o->col[c].imp[a] -= rb * ub[a];
            dpc[c][a] -= rb * ub[a];
          }
          if (cnt) {
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) qsum[a][b] /= cnt;
            q_put(o, o->Q, i, qsum);
          }
        }
      }
  memcpy(o->solid, ns, sizeof(int16_t) * (size_t)N);
  free(ns);
  for (int c = 0; c < o->ncol; ++c)
    if (o->col[c].mobile)
      for (int a = 0; a < 3; ++a) o->col[c].V[a] += dpc[c][a] / o->col[c].M;
}

/* x = A^{-1} b for a 3x3 matrix: Gaussian elimination with partial pivoting. */
static void solve3(const double A_in[3][3], const double b_in[3], double x[3]) {
  double A[3][4];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) A[a][b] = A_in[a][b];
    A[a][3] = b_in[a];
  }
  for (int k = 0; k < 3; ++k) {
    int p = k;
    for (int r = k + 1; r < 3; ++r)
      if (fabs(A[r][k]) > fabs(A[p][k])) p = r;
    for (int cidx = 0; cidx < 4; ++cidx) {
      double t = A[k][cidx];
      A[k][cidx] = A[p][cidx];
      A[p][cidx] = t;
    }
    for (int r = k + 1; r < 3; ++r) {
      double m = A[r][k] / A[k][k];
      for (int cidx = k; cidx < 4; ++cidx) A[r][cidx] -= m * A[k][cidx];
    }
  }
  for (int k = 2; k >= 0; --k) {
    double v = A[k][3];
    for (int cidx = k + 1; cidx < 3; ++cidx) v -= A[k][cidx] * x[cidx];
    x[k] = v / A[k][k];
  }
}

/* Colloid update ("molecular dynamics-like", Sec. 2.2), implicit in the
 * velocity-dependent part of the link force: the link momentum exchange is
 * F_hyd = F0 - zv V - (cross term in Omega), zv = sum over links of
 * 6 w rho0 c c; taking the zv V part at the new velocity,
 *   (M + zv) V' = M V + (F_hyd + zv V) + F_LC + F_ext,
 * i.e. V' = V + (M + zv)^{-1} (F_hyd + F_LC + F_ext), and likewise
 * Omega' = Omega + (I + zw)^{-1} (T_hyd + T_LC + T_ext), zw = sum 6 w rho0 (r x c)(r x c);
 * X += V'.  M = rho0 (4/3) pi a0^3 (neutrally buoyant), I = (2/5) M a0^2.
 * With no links (flow off) this is the explicit update. */
/* Squared minimum-image distance of two colloid centres, summed left to right. */
static double centre_dist2(const oracle* o, const ocolloid* A, const ocolloid* B) {
  double d[3];
  node_disp(o, A->X[0], A->X[1], A->X[2], B->X, d);
  return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

/* Contact partner of colloid c at the current positions: -1 for a z wall,
 * the lowest index of a colloid it touches, or -2 for none.  The paper treats
 * no contact (Sec. 3.2 leaves interactions between colloids to later work), so
 * this is a reading: two colloids touch when their centres are closer than
 * the sum of their radii, and a colloid touches a wall when its surface passes
 * the plane of the half-way bounce-back, z = -1/2 or z = nz - 1/2 (the test
 * that oracle_add_colloid applies). */
static int contact_partner(const oracle* o, int c) {
  const ocolloid* C = &o->col[c];
  if (o->wall_z && (C->X[2] - C->a0 < -0.5 || C->X[2] + C->a0 > o->nz - 0.5)) return -1;
  for (int d = 0; d < o->ncol; ++d) {
    if (d == c) continue;
    double s = C->a0 + o->col[d].a0;
    if (centre_dist2(o, C, &o->col[d]) < s * s) return d;
  }
  return -2;
}

/* A mobile colloid whose new position touches a wall or another colloid keeps
 * its position of the step before (its new velocities stand), so that no node
 * lies inside two colloids and no colloid crosses a wall.  All mobile
 * colloids are tested at the same positions, then those in contact are put
 * back; as a colloid put back can be touched by another's move, this repeats
 * until none is put back.  The first contact since the caller last read it
 * (lowest colloid index of that pass, its partner from contact_partner, the
 * step) is kept for the caller, who is told of it as an error. */
static void contact_resolve(oracle* o, double Xold[][3]) {
  int back[OMAXC] = {0};
  for (int pass = 0; pass <= o->ncol; ++pass) {
    int hit[OMAXC], any = 0;
    for (int c = 0; c < o->ncol; ++c)
      hit[c] = (o->col[c].mobile && !back[c]) ? contact_partner(o, c) : -2;
    for (int c = 0; c < o->ncol; ++c) {
      if (hit[c] == -2) continue;
      if (o->contact_step < 0) {
        o->contact_step = o->step;
        o->contact_c = c;
        o->contact_d = hit[c];
      }
      for (int a = 0; a < 3; ++a) o->col[c].X[a] = Xold[c][a];
      back[c] = 1;
      any = 1;
    }
    if (!any) break;
  }
}

static void colloid_update(oracle* o) {
  int moved = 0;
  double Xold[OMAXC][3];
  for (int c = 0; c < o->ncol; ++c)
    for (int a = 0; a < 3; ++a) Xold[c][a] = o->col[c].X[a];
  for (int c = 0; c < o->ncol; ++c) {
    ocolloid* C = &o->col[c];
    for (int a = 0; a < 3; ++a) {
      C->imp[a] += C->Fh[a] + C->Flc[a];
      C->aimp[a] += C->Th[a] + C->Tlc[a];
    }
    if (!C->mobile) continue;
    double Av[3][3], Aw[3][3], bv[3], bw[3], dv[3], dw[3];
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) {
        Av[a][b] = C->zv[a][b] + (a == b ? C->M : 0.0);
        Aw[a][b] = C->zw[a][b] + (a == b ? C->I : 0.0);
      }
      bv[a] = C->Fh[a] + C->Flc[a] + C->Fext[a];
      bw[a] = C->Th[a] + C->Tlc[a] + C->Text[a];
    }
    solve3(Av, bv, dv);
    solve3(Aw, bw, dw);
    for (int a = 0; a < 3; ++a) {
      C->V[a] += dv[a];
      C->W[a] += dw[a];
    }
    for (int a = 0; a < 3; ++a) {
      C->X[a] += C->V[a];
      int L = a == 0 ? o->nx : (a == 1 ? o->ny : o->nz);
      if (a < 2 || !o->wall_z) {
        if (C->X[a] >= L) C->X[a] -= L;
        if (C->X[a] < 0) C->X[a] += L;
      }
    }
    moved = 1;
  }
  if (moved) contact_resolve(o, Xold);
  if (moved) rediscretise(o);
}

static void step_once(oracle* o) {
  long N = o->N;
  /* 1-2: surface values, derivatives, H, f', P at fluid nodes */
  if (o->lc_on) lc_fields(o);
  /* 3: body force and colloid LC force/torque */
  if (o->lc_on) {
    lc_force(o);
  } else {
    for (long k = 0; k < 3 * N; ++k) o->F[k] = 0.0;
    for (int c = 0; c < o->ncol; ++c)
      for (int a = 0; a < 3; ++a) o->col[c].Flc[a] = o->col[c].Tlc[a] = 0.0;
  }
  /* 4: rho, u (fluid), rigid velocity (solid) */
  moments(o);
  /* 5: Q^{n+1} */
  if (o->lc_on) q_update(o);
  else o->resid_rms = o->resid_max = 0.0;
  /* 6: collide, bounce back, stream */
  if (o->flow_on) {
    collide_stream(o);
  } else {
    for (int c = 0; c < o->ncol; ++c)
      for (int a = 0; a < 3; ++a) o->col[c].Fh[a] = o->col[c].Th[a] = 0.0;
  }
  /* 7: colloids */
  colloid_update(o);
  o->step++;
}

/* ------------------------------------------------------------------ */
/* Public API (ctypes)                                                  */
/* ------------------------------------------------------------------ */
/* params: rho0, tau, A0, gamma, K, q0, xi, Gamma, S0 (<=0: closed-form q),
 *         gx, gy, gz */
oracle* oracle_create(int nx, int ny, int nz, int wall_z, const double* params, int lc_on, int flow_on) {
  if (nx < 1 || ny < 1 || nz < 1) return NULL;
  oracle* o = (oracle*)calloc(1, sizeof(oracle));
  o->nx = nx; o->ny = ny; o->nz = nz; o->wall_z = wall_z;
  o->N = (long)nx * ny * nz;
  o->rho0 = params[0]; o->tau = params[1]; o->A0 = params[2]; o->gam = params[3]; o->K = params[4];
  o->q0 = params[5]; o->xi = params[6]; o->Gam = params[7];
  o->S0 = params[8] > 0.0 ? params[8] : bulk_q(o->gam);
  o->g[0] = params[9]; o->g[1] = params[10]; o->g[2] = params[11];
  o->lc_on = lc_on; o->flow_on = flow_on;
  o->nthreads = 1;
  o->contact_step = -1;
  long N = o->N;
  o->solid = (int16_t*)malloc(sizeof(int16_t) * (size_t)N);
  for (long i = 0; i < N; ++i) o->solid[i] = -1;
  o->f = (double*)calloc((size_t)(NQ * N), sizeof(double));
  o->fpost = (double*)calloc((size_t)(NQ * N), sizeof(double));
  o->Q = (double*)calloc((size_t)(5 * N), sizeof(double));
  o->Qnew = (double*)calloc((size_t)(5 * N), sizeof(double));
  o->H = (double*)calloc((size_t)(5 * N), sizeof(double));
  o->P = (double*)calloc((size_t)(9 * N), sizeof(double));
  o->F = (double*)calloc((size_t)(3 * N), sizeof(double));
  o->u = (double*)calloc((size_t)(3 * N), sizeof(double));
  o->fe = (double*)calloc((size_t)N, sizeof(double));
  for (int q = 0; q < NQ; ++q)
    for (long i = 0; i < N; ++i) o->f[q * N + i] = WQ(q) * o->rho0;
  return o;
}

void oracle_destroy(oracle* o) {
  if (!o) return;
  free(o->solid); free(o->f); free(o->fpost); free(o->Q); free(o->Qnew);
  free(o->H); free(o->P); free(o->F); free(o->u); free(o->fe);
  free(o);
}

void oracle_set_threads(oracle* o, int n) { o->nthreads = n < 1 ? 1 : n; }

/* First contact since the last call (see contact_resolve): returns 1 and
 * out = (step, colloid, partner; -1 for a wall), then forgets it; 0 if none. */
int oracle_contact(oracle* o, long* out) {
  if (o->contact_step < 0) return 0;
  out[0] = o->contact_step;
  out[1] = o->contact_c;
  out[2] = o->contact_d;
  o->contact_step = -1;
  return 1;
}
double oracle_S0(const oracle* o) { return o->S0; }
long oracle_step_count(const oracle* o) { return o->step; }

/* SplitMix64 (Steele, Lea & Flood 2014): state s, output mix(s + golden). */
static uint64_t splitmix64(uint64_t s) {
  uint64_t z = s + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Uniform noise in [-amp, amp) for stored component k of node i. */
static double init_noise(uint64_t seed, long i, int k, double amp) {
  uint64_t r = splitmix64(seed ^ (uint64_t)(5 * i + k));
  double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
  return amp * (2.0 * u - 1.0);
}

/* Uniaxial Q = S0 (n n - delta/3) (the uniaxial form stated with Eq. 6, Sec. 2.1)
 * plus seeded noise on the 5 stored components; f at rest equilibrium. */
void oracle_init_uniaxial(oracle* o, const double* n, double amp, uint64_t seed) {
  long N = o->N;
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  double d[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
  for (long i = 0; i < N; ++i) {
    double q[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) q[a][b] = o->S0 * (d[a] * d[b] - (a == b ? 1.0 / 3.0 : 0.0));
    double v[5] = {q[0][0], q[0][1], q[0][2], q[1][1], q[1][2]};
    for (int k = 0; k < 5; ++k) o->Q[k * N + i] = v[k] + init_noise(seed, i, k, amp);
  }
  for (int q = 0; q < NQ; ++q)
    for (long i = 0; i < N; ++i) o->f[q * N + i] = WQ(q) * o->rho0;
}

/* Cholesteric helix along axis a: n_b = cos(q0 r_a), n_c = sin(q0 r_a), n_a = 0
 * with (a, b, c) cyclic, amplitude S0, phase 0 at r_a = 0, plus noise. */
void oracle_init_helix(oracle* o, int axis, double amp, uint64_t seed) {
  long N = o->N;
  int b = (axis + 1) % 3, c = (axis + 2) % 3;
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        int r[3] = {x, y, z};
        double ph = o->q0 * r[axis];
        double d[3] = {0, 0, 0};
        d[b] = cos(ph);
        d[c] = sin(ph);
        double q[3][3];
        for (int p = 0; p < 3; ++p)
          for (int s = 0; s < 3; ++s) q[p][s] = o->S0 * (d[p] * d[s] - (p == s ? 1.0 / 3.0 : 0.0));
        double v[5] = {q[0][0], q[0][1], q[0][2], q[1][1], q[1][2]};
        for (int k = 0; k < 5; ++k) o->Q[k * N + i] = v[k] + init_noise(seed, i, k, amp);
      }
  for (int q = 0; q < NQ; ++q)
    for (long i = 0; i < N; ++i) o->f[q * N + i] = WQ(q) * o->rho0;
}

void oracle_set_Q(oracle* o, const double* Q5) { memcpy(o->Q, Q5, sizeof(double) * 5 * (size_t)o->N); }
void oracle_get_Q(const oracle* o, double* Q5) { memcpy(Q5, o->Q, sizeof(double) * 5 * (size_t)o->N); }
void oracle_set_f(oracle* o, const double* f) { memcpy(o->f, f, sizeof(double) * NQ * (size_t)o->N); }
void oracle_get_f(const oracle* o, double* f) { memcpy(f, o->f, sizeof(double) * NQ * (size_t)o->N); }
void oracle_get_solid(const oracle* o, int16_t* s) { memcpy(s, o->solid, sizeof(int16_t) * (size_t)o->N); }

/* rho and u = (sum f c + (F_LC + g)/2)/rho of the current state (F_LC of the
 * current Q), exported at fluid nodes; solid nodes report rho0 and the rigid
 * velocity. */
void oracle_get_rho_u(oracle* o, double* rho, double* u) {
  long N = o->N;
  double keepF[OMAXC][3], keepT[OMAXC][3];
  for (int c = 0; c < o->ncol; ++c)
    for (int a = 0; a < 3; ++a) {
      keepF[c][a] = o->col[c].Flc[a];
      keepT[c][a] = o->col[c].Tlc[a];
    }
  if (o->lc_on) {
    lc_fields(o);
    lc_force(o);
  } else {
    for (long k = 0; k < 3 * N; ++k) o->F[k] = 0.0;
  }
  int fo = o->flow_on;
  o->flow_on = 1;
  moments(o);
  o->flow_on = fo;
  for (long i = 0; i < N; ++i) {
    double r = 0.0;
    for (int q = 0; q < NQ; ++q) r += o->f[q * N + i];
    rho[i] = o->solid[i] >= 0 ? o->rho0 : r;
  }
  memcpy(u, o->u, sizeof(double) * 3 * (size_t)N);
  for (int c = 0; c < o->ncol; ++c)
    for (int a = 0; a < 3; ++a) {
      o->col[c].Flc[a] = keepF[c][a];
      o->col[c].Tlc[a] = keepT[c][a];
    }
}

/* Molecular field (5 stored comps), stress (9, row-major a*3+b), body force
 * (3) and free energy density of the current Q.  Solid nodes report 0. */
void oracle_lc_fields(oracle* o, double* H5, double* P9, double* F3, double* fe) {
  long N = o->N;
  double keepF[OMAXC][3], keepT[OMAXC][3];
  for (int c = 0; c < o->ncol; ++c)
    for (int a = 0; a < 3; ++a) {
      keepF[c][a] = o->col[c].Flc[a];
      keepT[c][a] = o->col[c].Tlc[a];
    }
  lc_fields(o);
  lc_force(o);
  for (int c = 0; c < o->ncol; ++c)
    for (int a = 0; a < 3; ++a) {
      o->col[c].Flc[a] = keepF[c][a];
      o->col[c].Tlc[a] = keepT[c][a];
    }
  if (H5) memcpy(H5, o->H, sizeof(double) * 5 * (size_t)N);
  if (P9) memcpy(P9, o->P, sizeof(double) * 9 * (size_t)N);
  if (F3) memcpy(F3, o->F, sizeof(double) * 3 * (size_t)N);
  if (fe) memcpy(fe, o->fe, sizeof(double) * (size_t)N);
}


/* Adds a colloid of nominal radius a0 at X (Sec. 2.2).  Returns its index,
 * -1 on a bad argument, -2 if it touches another colloid or a wall (the
 * contact test of contact_partner) or shares a node with another colloid. */
int oracle_add_colloid(oracle* o, const double* X, double a0, int anchoring, double w, int mobile,
                       const double* Fext) {
  if (o->ncol >= OMAXC || !(a0 > 0.0)) return -1;
  if (o->wall_z && (X[2] - a0 < -0.5 || X[2] + a0 > o->nz - 0.5)) return -2;
  ocolloid* C = &o->col[o->ncol];
  memset(C, 0, sizeof(*C));
  for (int a = 0; a < 3; ++a) {
    C->X[a] = X[a];
    C->Fext[a] = Fext ? Fext[a] : 0.0;
  }
  C->a0 = a0; C->w = w; C->anchoring = anchoring; C->mobile = mobile;
  C->M = o->rho0 * 4.0 / 3.0 * M_PI * a0 * a0 * a0;
  C->I = 0.4 * C->M * a0 * a0;
  int id = o->ncol;
  for (int d = 0; d < o->ncol; ++d) {
    double s = a0 + o->col[d].a0;
    if (centre_dist2(o, C, &o->col[d]) < s * s) return -2;
  }
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (inside(o, x, y, z, C) && o->solid[i] >= 0) return -2;
      }
  o->ncol++;
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (inside(o, x, y, z, C)) o->solid[i] = (int16_t)id;
      }
  return id;
}

/* External torque on colloid c (a rotating colloid; the paper's colloids
 * take only the hydrodynamic and LC torques). */
void oracle_set_colloid_torque(oracle* o, int c, const double* T) {
  for (int a = 0; a < 3; ++a) o->col[c].Text[a] = T[a];
}

void oracle_set_colloid_velocity(oracle* o, int c, const double* V, const double* W) {
  for (int a = 0; a < 3; ++a) {
    o->col[c].V[a] = V[a];
    o->col[c].W[a] = W[a];
  }
}

/* out: X[3] V[3] W[3] Fh[3] Th[3] Flc[3] Tlc[3] imp[3] aimp[3] (27 doubles) */
void oracle_get_colloid(const oracle* o, int c, double* out) {
  const ocolloid* C = &o->col[c];
  const double* src[9] = {C->X, C->V, C->W, C->Fh, C->Th, C->Flc, C->Tlc, C->imp, C->aimp};
  for (int k = 0; k < 9; ++k)
    for (int a = 0; a < 3; ++a) out[3 * k + a] = src[k][a];
}

void oracle_step(oracle* o, int n) {
  for (int s = 0; s < n; ++s) step_once(o);
}

/* Boundary links (Sec. 2.2, Fig. 1): pairs (fluid node r, direction b) with
 * r + c_b inside a colloid, sorted by (colloid, node, b).  Returns the count;
 * writes at most cap entries. */
long oracle_links(const oracle* o, int32_t* node, int8_t* dir, int16_t* col, long cap) {
  long n = 0;
  for (int c = 0; c < o->ncol; ++c)
    for (int z = 0; z < o->nz; ++z)
      for (int y = 0; y < o->ny; ++y)
        for (int x = 0; x < o->nx; ++x) {
          long i = x + (long)o->nx * (y + (long)o->ny * z);
          if (o->solid[i] >= 0) continue;
          for (int q = 1; q < NQ; ++q) {
            long j = nbr(o, x, y, z, CV[q][0], CV[q][1], CV[q][2]);
            if (j >= 0 && o->solid[j] == c) {
              if (n < cap) {
                node[n] = (int32_t)i;
                dir[n] = (int8_t)q;
                col[n] = (int16_t)c;
              }
              ++n;
            }
          }
        }
  return n;
}

/* Diagnostics of the current state:
 * out[0] mass = sum over fluid nodes of sum_i f_i
 * out[1..3] fluid momentum sum_i f_i c_i (pre-collision)
 * out[4] free energy: sum of f' over fluid nodes plus, for finite anchoring
 *        strength, (w/2) |Qs - Q0|^2 over solid-fluid faces
 * out[5] residual RMS of the last step, out[6] its largest entry
 * out[7] number of fluid nodes
 * out[8] number of fluid nodes whose largest eigenvalue gives
 *        S = 3/2 lambda_max below 0.435 (the defect threshold of Sec. 3.1) */
void oracle_diag(oracle* o, double* out) {
  long N = o->N;
  ksum mass = {0, 0}, mom[3] = {{0, 0}, {0, 0}, {0, 0}}, fe = {0, 0};
  double nfl = 0.0, ndef = 0.0;
  if (o->lc_on) lc_fields(o);
  for (int z = 0; z < o->nz; ++z)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        long i = x + (long)o->nx * (y + (long)o->ny * z);
        if (o->solid[i] >= 0) continue;
        nfl += 1.0;
        for (int q = 0; q < NQ; ++q) {
          double fq = o->f[q * N + i];
          kadd(&mass, fq);
          for (int a = 0; a < 3; ++a) kadd(&mom[a], fq * CV[q][a]);
        }
        double qi[3][3], ev[3], v[3][3];
        q_get(o, o->Q, i, qi);
        jacobi3(qi, ev, v);
        double lm = ev[0] > ev[1] ? ev[0] : ev[1];
        if (ev[2] > lm) lm = ev[2];
        if (1.5 * lm < 0.435) ndef += 1.0;
        if (!o->lc_on) continue;
        kadd(&fe, o->fe[i]);
        for (int ax = 0; ax < 3; ++ax)
          for (int sgn = 0; sgn < 2; ++sgn) {
            int e[3] = {0, 0, 0};
            e[ax] = sgn == 0 ? 1 : -1;
            long j = nbr(o, x, y, z, e[0], e[1], e[2]);
            if (j < 0 || o->solid[j] < 0) continue;
            int c = o->solid[j];
            double w = o->col[c].w;
            if (strong_w(w)) continue;
            int sx = wrapi(x + e[0], o->nx), sy = wrapi(y + e[1], o->ny), sz = z + e[2];
            if (!o->wall_z) sz = wrapi(sz, o->nz);
            double qs[3][3], q0[3][3], t = 0.0;
            ghost_q(o, c, sx, sy, sz, qi, qs);
            surface_q0(o, c, sx, sy, sz, qi, q0);
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) t += (qs[a][b] - q0[a][b]) * (qs[a][b] - q0[a][b]);
            kadd(&fe, 0.5 * w * t);
          }
      }
  out[0] = kval(&mass);
  out[1] = kval(&mom[0]); out[2] = kval(&mom[1]); out[3] = kval(&mom[2]);
  out[4] = kval(&fe);
  out[5] = o->resid_rms;
  out[6] = o->resid_max;
  out[7] = nfl;
  out[8] = ndef;
}

/* Helpers exposed for the pins. */
void oracle_feq(double rho, const double* u, double* out) { feq_full(rho, u, out); }
void oracle_lattice(int* c, double* w) {
  for (int q = 0; q < NQ; ++q) {
    for (int a = 0; a < 3; ++a) c[3 * q + a] = CV[q][a];
    w[q] = WQ(q);
  }
}
void oracle_eig3(const double* A, double* ev, double* V) {
  double a[3][3], e[3], v[3][3];
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) a[p][q] = A[3 * p + q];
  jacobi3(a, e, v);
  for (int k = 0; k < 3; ++k) ev[k] = e[k];
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) V[3 * p + q] = v[p][q];
}
double oracle_bulk_q(double gam) { return bulk_q(gam); }
double oracle_noise(uint64_t seed, long i, int k, double amp) { return init_noise(seed, i, k, amp); }

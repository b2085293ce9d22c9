/*
 * lbm3_oracle.c -- plain FP64 CPU oracle of the ternary colour-gradient
 * lattice Boltzmann step of Yu, Liu, Liang & Zhang, "A versatile lattice
 * Boltzmann model for immiscible ternary fluid flows" (arXiv 1808.08555).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  It shares no code, header, table or helper
 * with the CUDA library; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Everything is written as plain nested loops over a periodic nx*ny grid in
 * double precision, one full-grid array per intermediate quantity, in the
 * order the paper gives the algorithm (Sec. 2: collision, recolouring,
 * streaming).  Nothing is fused, blocked or reordered.
 *
 * Storage: populations f[(k*9+i)*N + y*nx + x], k = colour (0,1,2 = the
 * paper's r,g,b), i = D2Q9 direction, N = nx*ny.  The stored state is the
 * post-streaming distribution f_{i,k}(x,t) from which rho_k = sum_i f_{i,k}
 * (the sentence after Eq. 30).
 *
 * Readings where the paper is silent or at odds with itself:
 *  - recolouring direction factor: Eq. 6 prints n_kl . e_i, while the
 *    interface-thickness result (Eq. 21 with k = 0.1504 from Eq. k, Sec. 3.1)
 *    belongs to the cosine form n_kl . e_i / |e_i|.  Both are provided
 *    (recolor_form 0 = cosine form, the default; 1 = as printed).
 *  - recolouring normal.  Eq. 6 uses the unit normal n_kl = G_kl/|G_kl|
 *    (Sec. 2, after Eq. 11).  normal_delta = 0 evaluates exactly that.  It is
 *    undefined where G_kl = 0, and the recolouring term then jumps whenever
 *    rho_k rho_l/rho is not negligible (e.g. at a droplet centre or at the
 *    saddle of phi between two nearby droplets), where rounding noise in G
 *    decides the direction.  normal_delta = d > 0 evaluates
 *    n_kl = G_kl / max(|G_kl|, d phi_k phi_l) instead: the paper's unit
 *    normal wherever |G_kl| >= d phi_k phi_l (across the tanh profile of
 *    Eq. 21 |G_kl| is about 1.26 phi_k phi_l), going to zero continuously,
 *    with a bounded gain, where G_kl vanishes.  In both forms, where
 *    |G_kl| <= 1e-15 no k-l interface is taken to exist: the tension term
 *    |G|(I - n n) of Eq. 11, which vanishes with |G|, is 0 there, and so is
 *    n_kl in the recolouring.
 *  - the derivatives inside F_s (Eq. 11) are the isotropic stencil of
 *    Eq. fd1 applied to phi_k = rho_k/rho, and then again to each component
 *    of the tensor inside the divergence.
 *  - the local tau_f of Eqs. vis_1/tau is used in both the BGK and the Guo
 *    prefactor; u of Eq. uk1 is used in both f^eq and Phi_i.
 *  - the perturbation operator (force_form 1, Eqs. phi1 / phi_old) replaces
 *    the force and Guo's term: u = sum_i f_i e_i / rho (no body force), and
 *    A_kl = A_lk = 9 sigma_kl / (2 tau_f) with the local tau_f.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Loops over nodes whose iterations write disjoint outputs run on all host
 * threads when the oracle is built with OpenMP.  Each output is computed by
 * the same arithmetic in the same order either way, so the results are
 * bit-identical for any thread count. */
#ifdef _OPENMP
#include <omp.h>
#define NODE_LOOP _Pragma("omp parallel for schedule(static)")
#else
#define NODE_LOOP
#endif

/* D2Q9 velocities and weights (Sec. 2, after Eq. 3): e0 = 0, e1,3 = (+-1,0),
 * e2,4 = (0,+-1), e5,7 = +-(1,1), e6,8 = +-(-1,1); w0 = 4/9, w1-4 = 1/9,
 * w5-8 = 1/36.  c_s^2 = 1/3. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;
static const double GEPS = 1e-15;   /* |G| at or below which no k-l interface exists */

typedef struct {
  int nx, ny;
  double tau[3];     /* per-fluid relaxation time; nu_k = (tau_k - 1/2) c_s^2 */
  double rho0[3];    /* pure-fluid densities rho_k^0 in C_kl (Eq. 15) */
  double sigma[3];   /* sigma_12, sigma_13, sigma_23 */
  double beta0;      /* reference segregation parameter beta^0 */
  int beta_form;     /* 0 = Eqs. 19-20 (the paper's); 1 = Eq. fu; 2 = Eq. 16; 3 = Eq. 17 */
  int recolor_form;  /* 0 = n.e_i/|e_i| (cosine form); 1 = n.e_i as printed in Eq. 6 */
  int force_form;    /* 0 = force of Eq. 11 through Guo's scheme (Eq. 5), the paper's;
                        1 = perturbation operator of Eqs. phi1 / phi_old (Leclaire et al.) */
  double normal_delta; /* recolouring normal n = G / max(|G|, normal_delta phi_k phi_l);
                          0 = the paper's G/|G| */
} orc_params;

/* ---------------------------------------------------------------- helpers */

static int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

/* sigma_kl for colours k != l (symmetric). */
static double sigma_of(const orc_params* p, int k, int l) {
  int a = k < l ? k : l, b = k < l ? l : k;
  if (a == 0 && b == 1) return p->sigma[0];
  if (a == 0 && b == 2) return p->sigma[1];
  return p->sigma[2];
}

/* ----------------------------------------------------- exported pieces */

/* Eq. 20: g(X) by its four branches. */
double orc_g(double X) {
  if (X < -1.0) return 1.0;
  if (X < 0.0) return 1.0 - sin(acos(X));
  if (X <= 1.0) return sin(acos(X)) - 1.0;
  return -1.0;
}

/* Eq. 18 (and Eq. theta_kl): X_kl = (s_mk^2 + s_ml^2 - s_kl^2)/(2 s_mk s_ml),
 * m the third fluid.  sig = (s12, s13, s23); out = (X12, X13, X23). */
void orc_X(const double* sig, double* out) {
  orc_params p;
  memset(&p, 0, sizeof p);
  p.sigma[0] = sig[0];
  p.sigma[1] = sig[1];
  p.sigma[2] = sig[2];
  const int pk[3] = {0, 0, 1}, pl[3] = {1, 2, 2};
  for (int q = 0; q < 3; ++q) {
    int k = pk[q], l = pl[q], m = 3 - k - l;
    double smk = sigma_of(&p, m, k), sml = sigma_of(&p, m, l), skl = sigma_of(&p, k, l);
    out[q] = (smk * smk + sml * sml - skl * skl) / (2.0 * smk * sml);
  }
}

/* Eq. 3: f_i^eq = w_i rho [1 + e.u/cs2 + (e.u)^2/(2 cs2^2) - u.u/(2 cs2)]. */
void orc_feq(double rho, double ux, double uy, double* feq) {
  for (int i = 0; i < 9; ++i) {
    double eu = EX[i] * ux + EY[i] * uy;
    double uu = ux * ux + uy * uy;
    feq[i] = WT[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
  }
}

/* Eq. 5 (Guo et al.): Phi_i = w_i (1 - 1/(2 tau)) [(e_i - u)/cs2 + (e_i.u)/cs2^2 e_i] . F */
void orc_guo(double tau, double ux, double uy, double Fx, double Fy, double* phi) {
  for (int i = 0; i < 9; ++i) {
    double eu = EX[i] * ux + EY[i] * uy;
    double cx = (EX[i] - ux) / CS2 + eu / (CS2 * CS2) * EX[i];
    double cy = (EY[i] - uy) / CS2 + eu / (CS2 * CS2) * EY[i];
    phi[i] = WT[i] * (1.0 - 1.0 / (2.0 * tau)) * (cx * Fx + cy * Fy);
  }
}

/* B_i of Eq. phi_old as Leclaire et al. take them (Sec. 2): B_0 = -4/27,
 * B_1-4 = 2/27, B_5-8 = 5/108. */
static const double BPERT[9] = {-4.0 / 27.0, 2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0, 2.0 / 27.0,
                                5.0 / 108.0, 5.0 / 108.0, 5.0 / 108.0, 5.0 / 108.0};

/* Eqs. phi1 / phi_old at one node: Phi_i = sum_k sum_{l != k} (A_kl C_kl / 2)
 * |G_kl| [w_i (e_i . G_kl)^2 / |G_kl|^2 - B_i], with A_kl = A_lk read from
 * sigma_kl = (A_kl + A_lk) tau_f / 9, i.e. A_kl = 9 sigma_kl / (2 tau_f).
 * G: the node's colour gradients [3][3][2] (k, l, component; G_lk = -G_kl),
 * C: [3][3]; sig = (s12, s13, s23).  Terms with |G_kl| <= 1e-15 are 0. */
void orc_perturbation(const double* sig, const double* G, const double* C, double tauf, double* phi) {
  for (int i = 0; i < 9; ++i) phi[i] = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      if (l == k) continue;
      int a = k < l ? k : l, b = k < l ? l : k;
      double s = (a == 0 && b == 1) ? sig[0] : (a == 0 ? sig[1] : sig[2]);
      double A = 9.0 * s / (2.0 * tauf);
      double gx = G[(k * 3 + l) * 2 + 0], gy = G[(k * 3 + l) * 2 + 1];
      double mag = sqrt(gx * gx + gy * gy);
      if (mag <= GEPS) continue;
      for (int i = 0; i < 9; ++i) {
        double eg = EX[i] * gx + EY[i] * gy;
        phi[i] += A * C[k * 3 + l] / 2.0 * mag * (WT[i] * eg * eg / (mag * mag) - BPERT[i]);
      }
    }
}

/* Eq. fd1: d_alpha v(x) = (1/cs2) sum_i w_i v(x + e_i) e_i,alpha on a periodic grid. */
void orc_grad(int nx, int ny, const double* v, double* gx, double* gy) {
  NODE_LOOP
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      double sx = 0.0, sy = 0.0;
      for (int i = 0; i < 9; ++i) {
        double vn = v[wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx)];
        sx += WT[i] * vn * EX[i];
        sy += WT[i] * vn * EY[i];
      }
      gx[y * nx + x] = sx / CS2;
      gy[y * nx + x] = sy / CS2;
    }
}

/* Colour gradients G_kl = phi_l grad phi_k - phi_k grad phi_l (Sec. 2, after
 * Eq. phi_old) for every ordered pair k != l, and the concentration factors
 * C_kl of Eq. 15.  rho: [3][N].  G: [3][3][2][N] (entries k == l left zero),
 * C: [3][3][N]. */
void orc_colour_gradients(const orc_params* p, const double* rho, double* G, double* C) {
  int nx = p->nx, ny = p->ny, N = nx * ny;
  double* phi = (double*)calloc((size_t)3 * N, sizeof(double));
  double* gphi = (double*)calloc((size_t)6 * N, sizeof(double));
  NODE_LOOP
  for (int n = 0; n < N; ++n) {
    double r = rho[n] + rho[N + n] + rho[2 * N + n];
    for (int k = 0; k < 3; ++k) phi[k * N + n] = rho[k * N + n] / r;
  }
  for (int k = 0; k < 3; ++k) orc_grad(nx, ny, phi + k * N, gphi + (2 * k) * N, gphi + (2 * k + 1) * N);
  NODE_LOOP
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        if (l == k) {
          G[((k * 3 + l) * 2 + 0) * N + n] = G[((k * 3 + l) * 2 + 1) * N + n] = 0.0;
          C[(k * 3 + l) * N + n] = 0.0;
          continue;
        }
        for (int a = 0; a < 2; ++a)
          G[((k * 3 + l) * 2 + a) * N + n] =
              phi[l * N + n] * gphi[(2 * k + a) * N + n] - phi[k * N + n] * gphi[(2 * l + a) * N + n];
        double c = 1e6 * rho[k * N + n] * rho[l * N + n] / (p->rho0[k] * p->rho0[l]);
        C[(k * 3 + l) * N + n] = c < 1.0 ? c : 1.0;
      }
  free(phi);
  free(gphi);
}

/* Eq. 11: F_s = sum_k sum_{l != k} div[ sigma_kl C_kl / 2 |G_kl| (I - n_kl n_kl) ],
 * n_kl = G_kl/|G_kl|.  The divergence is taken with Eq. fd1 on each tensor
 * component: F_b = d_x T_xb + d_y T_yb.  rho: [3][N]; Fx, Fy: [N].
 * T (optional, may be NULL): [3][N] = (T_xx, T_xy, T_yy). */
void orc_force(const orc_params* p, const double* rho, double* Fx, double* Fy, double* Tout) {
  int nx = p->nx, ny = p->ny, N = nx * ny;
  double* G = (double*)malloc(sizeof(double) * 18 * (size_t)N);
  double* C = (double*)malloc(sizeof(double) * 9 * (size_t)N);
  double* Txx = (double*)calloc((size_t)N, sizeof(double));
  double* Txy = (double*)calloc((size_t)N, sizeof(double));
  double* Tyy = (double*)calloc((size_t)N, sizeof(double));
  double* d1 = (double*)malloc(sizeof(double) * (size_t)N);
  double* d2 = (double*)malloc(sizeof(double) * (size_t)N);
  orc_colour_gradients(p, rho, G, C);
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      if (l == k) continue;
      double s = sigma_of(p, k, l);
      NODE_LOOP
      for (int n = 0; n < N; ++n) {
        double gx = G[((k * 3 + l) * 2 + 0) * N + n], gy = G[((k * 3 + l) * 2 + 1) * N + n];
        double mag = sqrt(gx * gx + gy * gy);
        if (mag <= GEPS) continue;
        double nxv = gx / mag, nyv = gy / mag;
        double a = s * C[(k * 3 + l) * N + n] / 2.0 * mag;
        Txx[n] += a * (1.0 - nxv * nxv);
        Txy[n] += a * (0.0 - nxv * nyv);
        Tyy[n] += a * (1.0 - nyv * nyv);
      }
    }
  /* F_x = d_x T_xx + d_y T_yx ; F_y = d_x T_xy + d_y T_yy (T symmetric). */
  orc_grad(nx, ny, Txx, d1, d2);
  for (int n = 0; n < N; ++n) Fx[n] = d1[n];
  orc_grad(nx, ny, Txy, d1, d2);
  for (int n = 0; n < N; ++n) {
    Fx[n] += d2[n];
    Fy[n] = d1[n];
  }
  orc_grad(nx, ny, Tyy, d1, d2);
  for (int n = 0; n < N; ++n) Fy[n] += d2[n];
  if (Tout) {
    memcpy(Tout, Txx, sizeof(double) * N);
    memcpy(Tout + N, Txy, sizeof(double) * N);
    memcpy(Tout + 2 * N, Tyy, sizeof(double) * N);
  }
  free(G); free(C); free(Txx); free(Txy); free(Tyy); free(d1); free(d2);
}

/* Segregation parameters beta_kl at one node, for the pair order (12, 13, 23).
 * form 0: Eqs. 19-20; 1: Eq. fu; 2: Eq. 16 (Spencer); 3: Eq. 17 (Leclaire).
 * For forms 2 and 3 the contact angles phi_kl of Eq. theta_kl are used; where
 * no Neumann triangle exists they fall back to beta^0 (Sec. 2, after Eq. 17). */
void orc_beta(const orc_params* p, const double* rk, double* beta) {
  double r = rk[0] + rk[1] + rk[2];
  double prod = rk[0] * rk[1] * rk[2] / (r * r * r);
  double X[3];
  orc_X(p->sigma, X);
  int tri = fabs(X[0]) < 1.0 && fabs(X[1]) < 1.0 && fabs(X[2]) < 1.0;
  double b0 = p->beta0;
  if (p->beta_form == 1 || ((p->beta_form == 2 || p->beta_form == 3) && !tri)) {
    beta[0] = beta[1] = beta[2] = b0;
    return;
  }
  if (p->beta_form == 0) {
    double c = 35.0 * prod;
    if (c > 1.0) c = 1.0;
    for (int q = 0; q < 3; ++q) beta[q] = b0 + b0 * c * orc_g(X[q]);
    return;
  }
  double ang[3];
  for (int q = 0; q < 3; ++q) ang[q] = acos(X[q]);  /* phi_12, phi_13, phi_23 */
  if (p->beta_form == 2) {
    /* Eq. 16: beta_rg = b0; beta_rb uses sin(phi_gb); beta_gb uses sin(phi_rb). */
    beta[0] = b0;
    beta[1] = b0 * (1.0 + 27.0 * prod * (sin(ang[2]) - 1.0));
    beta[2] = b0 * (1.0 + 27.0 * prod * (sin(ang[1]) - 1.0));
    return;
  }
  /* Eq. 17 */
  double ct = 35.0 * prod;
  if (ct > 1.0) ct = 1.0;
  int qmax = 0;
  for (int q = 1; q < 3; ++q)
    if (ang[q] > ang[qmax]) qmax = q;
  for (int q = 0; q < 3; ++q)
    beta[q] = (q == qmax) ? b0 : b0 + b0 * ct * (sin(M_PI - ang[qmax] - ang[q]) - 1.0);
}

/* Macroscopic fields at time t from the post-streaming populations:
 * rho_k = sum_i f_{i,k} (after Eq. 30); rho u = sum_i f_i e_i + F_s/2 (Eq. uk1);
 * p = rho c_s^2 (the paper gives no pressure formula; ideal-gas reading).
 * rho: [3][N], ux, uy, pr: [N] (any may be NULL). */
void orc_fields(const orc_params* p, const double* f, double* rho, double* ux, double* uy, double* pr) {
  int N = p->nx * p->ny;
  double* rk = (double*)calloc((size_t)3 * N, sizeof(double));
  double* Fx = (double*)malloc(sizeof(double) * (size_t)N);
  double* Fy = (double*)malloc(sizeof(double) * (size_t)N);
  NODE_LOOP
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 9; ++i) rk[k * N + n] += f[(k * 9 + i) * N + n];
  if (p->force_form == 1) {
    memset(Fx, 0, sizeof(double) * (size_t)N);
    memset(Fy, 0, sizeof(double) * (size_t)N);
  } else {
    orc_force(p, rk, Fx, Fy, NULL);
  }
  NODE_LOOP
  for (int n = 0; n < N; ++n) {
    double r = rk[n] + rk[N + n] + rk[2 * N + n];
    double mx = 0.0, my = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 9; ++i) {
        mx += f[(k * 9 + i) * N + n] * EX[i];
        my += f[(k * 9 + i) * N + n] * EY[i];
      }
    if (ux) ux[n] = (mx + 0.5 * Fx[n]) / r;
    if (uy) uy[n] = (my + 0.5 * Fy[n]) / r;
    if (pr) pr[n] = r * CS2;
  }
  if (rho) memcpy(rho, rk, sizeof(double) * 3 * N);
  free(rk); free(Fx); free(Fy);
}

/* One time step (Sec. 2): collision with the Guo force (Eqs. 1-3, 5, uk1,
 * vis_1, tau), recolouring (Eq. 6 with beta_kl from orc_beta), streaming
 * (Eq. 30).  f: [27][N] post-streaming state at t, replaced by the state at
 * t+1. */
static void orc_step_once(const orc_params* p, double* f, double* fn) {
  int nx = p->nx, ny = p->ny, N = nx * ny;
  double* rk = (double*)calloc((size_t)3 * N, sizeof(double));
  double* Fx = (double*)malloc(sizeof(double) * (size_t)N);
  double* Fy = (double*)malloc(sizeof(double) * (size_t)N);
  double* G = (double*)malloc(sizeof(double) * 18 * (size_t)N);
  double* C = (double*)malloc(sizeof(double) * 9 * (size_t)N);
  double nu[3];
  for (int k = 0; k < 3; ++k) nu[k] = (p->tau[k] - 0.5) * CS2;

  /* densities rho_k = sum_i f_{i,k} */
  NODE_LOOP
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 9; ++i) rk[k * N + n] += f[(k * 9 + i) * N + n];
  /* interfacial force (Eq. 11; none with the perturbation operator) and
   * colour gradients */
  if (p->force_form == 1) {
    memset(Fx, 0, sizeof(double) * (size_t)N);
    memset(Fy, 0, sizeof(double) * (size_t)N);
  } else {
    orc_force(p, rk, Fx, Fy, NULL);
  }
  orc_colour_gradients(p, rk, G, C);

  /* each source node writes its own 27 destinations (Eq. 30): disjoint */
  NODE_LOOP
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int n = y * nx + x;
      double rloc[3] = {rk[n], rk[N + n], rk[2 * N + n]};
      double r = rloc[0] + rloc[1] + rloc[2];
      /* total distribution f_i = sum_k f_{i,k} */
      double fi[9];
      for (int i = 0; i < 9; ++i) fi[i] = f[(0 * 9 + i) * N + n] + f[(1 * 9 + i) * N + n] + f[(2 * 9 + i) * N + n];
      /* Eq. uk1 */
      double mx = 0.0, my = 0.0;
      for (int i = 0; i < 9; ++i) {
        mx += fi[i] * EX[i];
        my += fi[i] * EY[i];
      }
      double ux = (mx + 0.5 * Fx[n]) / r, uy = (my + 0.5 * Fy[n]) / r;
      /* Eqs. vis_1 and tau: rho/nu = sum_k rho_k/nu_k, nu = (tau_f - 1/2) c_s^2 */
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += rloc[k] / nu[k];
      double nuloc = r / s;
      double tauf = nuloc / CS2 + 0.5;
      /* Eqs. 1-3, with Phi_i of Eq. 5 or of Eqs. phi1 / phi_old */
      double feq[9], phi[9], fdag[9];
      orc_feq(r, ux, uy, feq);
      if (p->force_form == 1) {
        double Gn[18], Cn[9];
        for (int j = 0; j < 18; ++j) Gn[j] = G[(size_t)j * N + n];
        for (int j = 0; j < 9; ++j) Cn[j] = C[(size_t)j * N + n];
        orc_perturbation(p->sigma, Gn, Cn, tauf, phi);
      } else {
        orc_guo(tauf, ux, uy, Fx[n], Fy[n], phi);
      }
      for (int i = 0; i < 9; ++i) fdag[i] = fi[i] - (fi[i] - feq[i]) / tauf + phi[i];
      /* recolouring, Eq. 6 */
      double beta[3];
      orc_beta(p, rloc, beta);
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 9; ++i) {
          double v = rloc[k] / r * fdag[i];
          for (int l = 0; l < 3; ++l) {
            if (l == k) continue;
            double gx = G[((k * 3 + l) * 2 + 0) * N + n], gy = G[((k * 3 + l) * 2 + 1) * N + n];
            double mag = sqrt(gx * gx + gy * gy);
            if (mag <= GEPS) continue;  /* no k-l interface: n_kl = 0, as in Eq. 11 */
            double den = p->normal_delta * (rloc[k] / r) * (rloc[l] / r);
            if (mag > den) den = mag;
            double en = (gx * EX[i] + gy * EY[i]) / den;
            if (p->recolor_form == 0 && i != 0) en /= sqrt((double)(EX[i] * EX[i] + EY[i] * EY[i]));
            int a = k < l ? k : l, b = k < l ? l : k;
            int q = (a == 0 && b == 1) ? 0 : (a == 0 ? 1 : 2);
            v += beta[q] * WT[i] * rloc[k] * rloc[l] / r * en;
          }
          /* streaming, Eq. 30: f_{i,k}(x + e_i, t + 1) = f^ddagger_{i,k}(x, t) */
          int xd = wrap(x + EX[i], nx), yd = wrap(y + EY[i], ny);
          fn[(k * 9 + i) * N + yd * nx + xd] = v;
        }
    }
  free(rk); free(Fx); free(Fy); free(G); free(C);
}

/* Advance the post-streaming state f ([27][N], FP64) by nsteps steps. */
void orc_step(const orc_params* p, double* f, int nsteps) {
  size_t bytes = sizeof(double) * 27 * (size_t)p->nx * p->ny;
  double* fn = (double*)malloc(bytes);
  const long total = 27L * p->nx * p->ny;
  for (int s = 0; s < nsteps; ++s) {
    orc_step_once(p, f, fn);
    NODE_LOOP
    for (long j = 0; j < total; ++j) f[j] = fn[j];
  }
  free(fn);
}

/* Initial populations: local equilibrium at rest, f_{i,k} = w_i rho_k (the
 * paper gives no initialisation of the populations; this is Eq. 3 per colour
 * with u = 0). */
void orc_init(const orc_params* p, const double* rho, double* f) {
  int N = p->nx * p->ny;
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 9; ++i)
      for (int n = 0; n < N; ++n) f[(k * 9 + i) * N + n] = WT[i] * rho[k * N + n];
}

/* Per-colour mass sum_x rho_k and lattice momentum sum_x sum_i f_i e_i. */
void orc_mass(const orc_params* p, const double* f, double* mass, double* mom) {
  int N = p->nx * p->ny;
  mass[0] = mass[1] = mass[2] = 0.0;
  mom[0] = mom[1] = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 9; ++i)
      for (int n = 0; n < N; ++n) {
        double v = f[(k * 9 + i) * N + n];
        mass[k] += v;
        mom[0] += v * EX[i];
        mom[1] += v * EY[i];
      }
}

/* Host threads used by the node loops (OpenMP builds); 0 leaves the current
 * setting.  Returns the number in effect (1 without OpenMP). */
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

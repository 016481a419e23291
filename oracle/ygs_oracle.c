/*
 * ygs_oracle.c -- plain, slow, FP64 CPU oracle for the multi-patch
 * spherical-harmonics gravity solver (Wongwathanarat, arXiv:1903.08475).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes (all in FP64, plain loops, OpenMP over independent outputs):
 *
 *   O2  (main oracle, "factorised plain Y_lm"):
 *       U[a,c] = (2/delta_m) w_a * \int_cell Y^t_lm(R^(g) n(theta,phi)) dOmega
 *                by tensor Gauss-Legendre quadrature of the GLOBAL-frame real
 *                harmonic at rotated quadrature points (Eqs. A_lm_mult/B_lm_mult,
 *                Eq. phispherical, Eq. U_C/U_S read as their definition),
 *       B[i,c] = sum_{g,a} rho[g,i,a] U[a,c]                     (Eq. B_CS),
 *       M[i,c] = (r_i^+)^-(l+1) sum_{i'<=i} R_in B + (r_i^+)^l sum_{i'>i} R_out B
 *                as direct O(Nr^2) sums, no recurrence           (Eq. M_C),
 *       Phi[g,i,a] = sum_c Q[a,c] M[i,c],
 *       Q[a,c] = -G Y^t_lm(global direction of the evaluation vertex) (Eqs. Q_C/Q_S).
 *   O1  (brute force): the addition theorem written out with Legendre
 *       polynomials only, Phi(p) = -G sum_l sum_cells rho w K_l(i,i')
 *       \int_cell P_l(n_p . n) dOmega (Eqs. 1-4 with the Green's function
 *       expansion); no Y_lm anywhere.  Tiny grids only.
 *   O3  (per-patch superposition, the older scheme of Sect. 4.3): local-frame
 *       moments per patch, per-patch radial sums, and the potential as the sum
 *       over patches of each expansion evaluated at the point expressed in that
 *       patch's frame.
 *   apply_T: the transpose of the linear map rho -> Phi by the transposed loops.
 *   Ellipsoid: the homogeneous-ellipsoid potential of Sect. 5.1 (Eq. phiana)
 *       by Carlson's symmetric integrals R_F / R_D (duplication algorithm,
 *       B. C. Carlson, Numer. Algorithms 10 (1995) 13) and, independently, by
 *       the paper's own recipe (bisection for u0, Simpson quadrature).
 *
 * Conventions (the paper leaves them implicit; they are fixed here and pinned
 * by the tests):
 *   - P_l^m without the Condon-Shortley phase; Y^C_lm = N_lm P_l^m(cos t) cos(m p),
 *     Y^S_lm = N_lm P_l^m(cos t) sin(m p), N_lm = sqrt((l-m)!/(l+m)!).
 *   - real column index c: (l,0,C) -> l*l, (l,m,C) -> l*l+2m-1, (l,m,S) -> l*l+2m.
 *   - x = R^(g) xi with R^(g) the matrix of Eq. rottransmatrix.
 *   - a cell's local extents: theta_j^- = t_lo + j dt, phi_k^- = p_lo + k dp;
 *     the flat angular index is a = j*Nphi + k; fields are [g][i][a].
 *   - Phi is evaluated at r_i^+ and at the upper angular vertex (eval=0) or
 *     the angular centre (eval=1) of each cell.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int n_r;
  const double* edges;       /* n_r + 1, increasing */
  int n_patch;
  const double* euler;       /* 3 * n_patch: alpha, beta, gamma */
  const int* n_theta;        /* n_patch */
  const int* n_phi;          /* n_patch */
  const double* theta_range; /* 2 * n_patch */
  const double* phi_range;   /* 2 * n_patch */
  const double* w;           /* sum_g n_theta*n_phi */
  int l_max;
  double G;
  int eval;                  /* 0 = upper vertex, 1 = angular centre */
  const int* kind;           /* n_patch: 0 = (theta, phi) patch, 1 = gnomonic cube face; NULL: all 0 */
} ora_grid;

static const double ORA_PI = 3.14159265358979323846264338327950288;

static int ncols(int l_max) { return (l_max + 1) * (l_max + 1); }

static long nang_patch(const ora_grid* g, int p) { return (long)g->n_theta[p] * g->n_phi[p]; }

static long nang_before(const ora_grid* g, int p) {
  long s = 0;
  for (int q = 0; q < p; ++q) s += nang_patch(g, q);
  return s;
}

static long nang_total(const ora_grid* g) { return nang_before(g, g->n_patch); }

/* ---------------------------------------------------------------- basics -- */

/* Gauss-Legendre nodes/weights on [-1,1]: Newton iteration on P_n. */
static void legendre_pn_and_prev(int n, double z, double* pn, double* pm) {
  double a = 1.0, b = z; /* P_0, P_1 */
  if (n == 0) { *pn = 1.0; *pm = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2.0 * k - 1.0) * z * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  *pn = b;
  *pm = a;
}

int ora_gauss_legendre(int n, double* x, double* w) {
  if (n < 1) return -1;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(ORA_PI * (i + 0.75) / (n + 0.5));
    double pn, pm, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_pn_and_prev(n, z, &pn, &pm);
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    legendre_pn_and_prev(n, z, &pn, &pm);
    dp = n * (z * pn - pm) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return 0;
}

/* Rotation matrix of Eq. rottransmatrix (row-major R[3][3]), x = R xi. */
void ora_euler_matrix(double a, double b, double g, double* R) {
  double ca = cos(a), sa = sin(a), cb = cos(b), sb = sin(b), cg = cos(g), sg = sin(g);
  R[0] = ca * cb * cg - sa * sg;  R[1] = sa * cb * cg + ca * sg;  R[2] = -sb * cg;
  R[3] = -ca * cb * sg - sa * cg; R[4] = -sa * cb * sg + ca * cg; R[5] = sb * sg;
  R[6] = ca * sb;                 R[7] = sa * sb;                 R[8] = cb;
}

static void local_dir(double th, double ph, double* v) {
  v[0] = sin(th) * cos(ph);
  v[1] = sin(th) * sin(ph);
  v[2] = cos(th);
}

/* A patch's local coordinates (u, v) -> local unit vector and the solid-angle
 * density dOmega / (du dv).  (theta, phi) patches: u = theta, v = phi,
 * density sin(theta).  Gnomonic cube faces (the non-orthogonal patches of
 * Sect. 6): u, v equiangular, X = tan u, Y = tan v, the direction
 * (X, Y, 1) / sqrt(1 + X^2 + Y^2) and density (1 + X^2)(1 + Y^2) / (1 + X^2 + Y^2)^(3/2). */
static double patch_dir(const ora_grid* g, int p, double u, double v, double* d) {
  if (g->kind && g->kind[p] == 1) {
    double X = tan(u), Y = tan(v), r2 = 1.0 + X * X + Y * Y, r = sqrt(r2);
    d[0] = X / r;
    d[1] = Y / r;
    d[2] = 1.0 / r;
    return (1.0 + X * X) * (1.0 + Y * Y) / (r2 * r);
  }
  local_dir(u, v, d);
  return sin(u);
}

static void matvec(const double* R, const double* v, double* out) {
  for (int r = 0; r < 3; ++r) out[r] = R[3 * r] * v[0] + R[3 * r + 1] * v[1] + R[3 * r + 2] * v[2];
}

static void matTvec(const double* R, const double* v, double* out) {
  for (int r = 0; r < 3; ++r) out[r] = R[r] * v[0] + R[3 + r] * v[1] + R[6 + r] * v[2];
}

/* N_lm = sqrt((l-m)!/(l+m)!) as a plain product, table [l][m]. */
static double* norm_table(int l_max) {
  double* t = (double*)malloc(sizeof(double) * (l_max + 1) * (l_max + 1));
  for (int l = 0; l <= l_max; ++l)
    for (int m = 0; m <= l_max; ++m) {
      double n2 = 1.0;
      for (int k = l - m + 1; k <= l + m; ++k) n2 /= (double)k;
      t[l * (l_max + 1) + m] = (m <= l) ? sqrt(n2) : 0.0;
    }
  return t;
}

/* All real harmonics Y^t_lm at the direction v (unit vector), column order
 * c(l,m,t).  Unnormalised associated Legendre functions without the
 * Condon-Shortley phase by the textbook recurrences in l, times N_lm. */
static void harmonics_dir(int l_max, const double* nrm, const double* v, double* out) {
  double x = v[2];
  if (x > 1.0) x = 1.0;
  if (x < -1.0) x = -1.0;
  double ph = atan2(v[1], v[0]);
  /* sin(theta) is the distance from the polar axis: computing it as
   * sin(acos(x)) would lose digits next to the poles */
  double s = sqrt(v[0] * v[0] + v[1] * v[1]);
  /* P_mm = (2m-1)!! s^m, P_{m+1,m} = (2m+1) x P_mm,
   * (l-m) P_lm = (2l-1) x P_{l-1,m} - (l+m-1) P_{l-2,m} */
  for (int m = 0; m <= l_max; ++m) {
    double pmm = 1.0;
    for (int k = 1; k <= m; ++k) pmm *= (2.0 * k - 1.0) * s;
    double cm = cos(m * ph), sm = sin(m * ph);
    double plm2 = 0.0, plm1 = 0.0;
    for (int l = m; l <= l_max; ++l) {
      double p;
      if (l == m) p = pmm;
      else if (l == m + 1) p = (2.0 * m + 1.0) * x * pmm;
      else p = ((2.0 * l - 1.0) * x * plm1 - (l + m - 1.0) * plm2) / (double)(l - m);
      plm2 = plm1;
      plm1 = p;
      double nlm = nrm[l * (l_max + 1) + m];
      if (m == 0) out[l * l] = nlm * p;
      else {
        out[l * l + 2 * m - 1] = nlm * p * cm;
        out[l * l + 2 * m] = nlm * p * sm;
      }
    }
  }
}

void ora_real_harmonics_dir(int l_max, const double* v, double* out) {
  double* nrm = norm_table(l_max);
  harmonics_dir(l_max, nrm, v, out);
  free(nrm);
}

void ora_real_harmonics(int l_max, double theta, double phi, double* out) {
  double v[3];
  local_dir(theta, phi, v);
  ora_real_harmonics_dir(l_max, v, out);
}

/* Legendre polynomials P_0..P_lmax at x (Bonnet recurrence). */
static void legendre_pl(int l_max, double x, double* out) {
  out[0] = 1.0;
  if (l_max >= 1) out[1] = x;
  for (int l = 2; l <= l_max; ++l) out[l] = ((2.0 * l - 1.0) * x * out[l - 1] - (l - 1.0) * out[l - 2]) / l;
}

static int col_m(int c, int* l_out) {
  int l = (int)floor(sqrt((double)c));
  while ((l + 1) * (l + 1) <= c) ++l;
  while (l * l > c) --l;
  *l_out = l;
  int r = c - l * l;
  return (r + 1) / 2;
}

/* ---------------------------------------------------------- radial parts -- */

/* (hi^n - lo^n)/n evaluated as hi^n * (1 - q^n)/n, q = lo/hi (Eqs. R_in/R_out). */
static double pow_diff_over_n(double lo, double hi, double n) {
  if (lo <= 0.0) return pow(hi, n) / n; /* only reached with n > 0 */
  double lq = log(lo / hi);
  return pow(hi, n) * (-expm1(n * lq)) / n;
}

double ora_R_in(double lo, double hi, int l) { return pow_diff_over_n(lo, hi, l + 3.0); }

double ora_R_out(double lo, double hi, int l) {
  if (l == 2) return log(hi / lo);
  return pow_diff_over_n(lo, hi, 2.0 - l);
}

/* K_l(i, i'): weight of source shell i' for evaluation radius r_i^+. */
static double kernel_l(const ora_grid* g, int i, int ip, int l) {
  double r = g->edges[i + 1];
  if (ip <= i) return pow(r, -(l + 1.0)) * ora_R_in(g->edges[ip], g->edges[ip + 1], l);
  return pow(r, (double)l) * ora_R_out(g->edges[ip], g->edges[ip + 1], l);
}

/* --------------------------------------------------------------- weights -- */

static void cell_bounds(const ora_grid* g, int p, int j, int k, double* t0, double* t1, double* p0, double* p1) {
  double dt = (g->theta_range[2 * p + 1] - g->theta_range[2 * p]) / g->n_theta[p];
  double dp = (g->phi_range[2 * p + 1] - g->phi_range[2 * p]) / g->n_phi[p];
  *t0 = g->theta_range[2 * p] + j * dt;
  *t1 = *t0 + dt;
  *p0 = g->phi_range[2 * p] + k * dp;
  *p1 = *p0 + dp;
}

static void eval_point_local(const ora_grid* g, int p, int j, int k, double* th, double* ph) {
  double t0, t1, p0, p1;
  cell_bounds(g, p, j, k, &t0, &t1, &p0, &p1);
  if (g->eval == 0) { *th = t1; *ph = p1; }
  else { *th = 0.5 * (t0 + t1); *ph = 0.5 * (p0 + p1); }
}

/* U[a][c] for all cells of all patches (rotate = 1: global-frame harmonics,
 * rotate = 0: the patch's own local-frame harmonics, as in the older scheme). */
static int build_U(const ora_grid* g, int nq, int rotate, double* U) {
  int K = ncols(g->l_max);
  double* xq = (double*)malloc(sizeof(double) * nq);
  double* wq = (double*)malloc(sizeof(double) * nq);
  if (!xq || !wq) { free(xq); free(wq); return -2; }
  ora_gauss_legendre(nq, xq, wq);
  double* nrm = norm_table(g->l_max);
  for (int p = 0; p < g->n_patch; ++p) {
    double R[9];
    ora_euler_matrix(g->euler[3 * p], g->euler[3 * p + 1], g->euler[3 * p + 2], R);
    long base = nang_before(g, p);
    int nt = g->n_theta[p], nf = g->n_phi[p];
#pragma omp parallel
    {
      double* Y = (double*)malloc(sizeof(double) * K);
      double* acc = (double*)malloc(sizeof(double) * K);
#pragma omp for schedule(dynamic, 4)
      for (long a = 0; a < (long)nt * nf; ++a) {
        int j = (int)(a / nf), k = (int)(a % nf);
        double t0, t1, p0, p1;
        cell_bounds(g, p, j, k, &t0, &t1, &p0, &p1);
        for (int c = 0; c < K; ++c) acc[c] = 0.0;
        for (int qa = 0; qa < nq; ++qa) {
          double th = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * xq[qa];
          double wt = 0.5 * (t1 - t0) * wq[qa];
          for (int qb = 0; qb < nq; ++qb) {
            double ph = 0.5 * (p0 + p1) + 0.5 * (p1 - p0) * xq[qb];
            double v[3], x[3];
            double wgt = wt * 0.5 * (p1 - p0) * wq[qb] * patch_dir(g, p, th, ph, v);
            if (rotate) matvec(R, v, x);
            else { x[0] = v[0]; x[1] = v[1]; x[2] = v[2]; }
            harmonics_dir(g->l_max, nrm, x, Y);
            for (int c = 0; c < K; ++c) acc[c] += wgt * Y[c];
          }
        }
        double wa = g->w[base + a];
        for (int c = 0; c < K; ++c) {
          int l;
          int m = col_m(c, &l);
          double f = (m == 0) ? 1.0 : 2.0; /* 2/delta_m */
          U[(base + a) * K + c] = f * wa * acc[c];
        }
      }
      free(Y);
      free(acc);
    }
  }
  free(xq);
  free(wq);
  free(nrm);
  return 0;
}

int ora_build_U(const ora_grid* g, int nq, double* U) { return build_U(g, nq, 1, U); }
int ora_build_U_local(const ora_grid* g, int nq, double* U) { return build_U(g, nq, 0, U); }

/* Q[a][c] = -G Y^t_lm(global direction of the evaluation point)  (Eqs. Q_C/Q_S). */
int ora_build_Q(const ora_grid* g, double* Q) {
  int K = ncols(g->l_max);
  double* nrm = norm_table(g->l_max);
  for (int p = 0; p < g->n_patch; ++p) {
    double R[9];
    ora_euler_matrix(g->euler[3 * p], g->euler[3 * p + 1], g->euler[3 * p + 2], R);
    long base = nang_before(g, p);
    int nt = g->n_theta[p], nf = g->n_phi[p];
#pragma omp parallel for schedule(static)
    for (long a = 0; a < (long)nt * nf; ++a) {
      int j = (int)(a / nf), k = (int)(a % nf);
      double th, ph, v[3], x[3];
      eval_point_local(g, p, j, k, &th, &ph);
      patch_dir(g, p, th, ph, v);
      matvec(R, v, x);
      double* q = Q + (base + a) * K;
      harmonics_dir(g->l_max, nrm, x, q);
      for (int c = 0; c < K; ++c) q[c] *= -g->G;
    }
  }
  free(nrm);
  return 0;
}

/* ------------------------------------------------------------ the steps --- */

/* B[i][c] = sum_{g,a} rho[g][i][a] U[a][c]  (Eq. B_CS, steps 2-3).  Each
 * B[i][c] is the sum over (g, a) in ascending order; a whole row of B is
 * accumulated at once so that U is read row by row. */
void ora_project(const ora_grid* g, const double* rho, const double* U, double* B) {
  int K = ncols(g->l_max);
  int nr = g->n_r;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < nr; ++i) {
    double* b = B + (long)i * K;
    for (int c = 0; c < K; ++c) b[c] = 0.0;
    for (int p = 0; p < g->n_patch; ++p) {
      long base = nang_before(g, p), na = nang_patch(g, p);
      const double* r = rho + base * nr + (long)i * na;
      for (long a = 0; a < na; ++a) {
        const double ra = r[a];
        const double* u = U + (base + a) * K;
        for (int c = 0; c < K; ++c) b[c] += ra * u[c];
      }
    }
  }
}

/* M[i][c] by the direct sums of Eq. M_C (no recurrence). */
void ora_radial(const ora_grid* g, const double* B, double* M) {
  int K = ncols(g->l_max);
  int nr = g->n_r;
#pragma omp parallel for collapse(2) schedule(static)
  for (int i = 0; i < nr; ++i)
    for (int c = 0; c < K; ++c) {
      int l;
      (void)col_m(c, &l);
      double sin_ = 0.0, sout = 0.0;
      for (int ip = 0; ip <= i; ++ip) sin_ += ora_R_in(g->edges[ip], g->edges[ip + 1], l) * B[(long)ip * K + c];
      for (int ip = i + 1; ip < nr; ++ip) sout += ora_R_out(g->edges[ip], g->edges[ip + 1], l) * B[(long)ip * K + c];
      double r = g->edges[i + 1];
      M[(long)i * K + c] = pow(r, -(l + 1.0)) * sin_ + pow(r, (double)l) * sout;
    }
}

/* Phi[g][i][a] = sum_c Q[a][c] M[i][c]  (Eq. gravpotmult, step 5). */
void ora_synthesize(const ora_grid* g, const double* M, const double* Q, double* phi) {
  int K = ncols(g->l_max);
  int nr = g->n_r;
  for (int p = 0; p < g->n_patch; ++p) {
    long base = nang_before(g, p), na = nang_patch(g, p);
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < nr; ++i)
      for (long a = 0; a < na; ++a) {
        double s = 0.0;
        const double* q = Q + (base + a) * K;
        const double* m = M + (long)i * K;
        for (int c = 0; c < K; ++c) s += q[c] * m[c];
        phi[base * nr + (long)i * na + a] = s;
      }
  }
}

/* O2: the whole solve.  B_out / M_out may be NULL. */
int ora_solve(const ora_grid* g, int nq, const double* rho, double* phi, double* B_out, double* M_out) {
  int K = ncols(g->l_max);
  long na = nang_total(g);
  double* U = (double*)malloc(sizeof(double) * na * K);
  double* Q = (double*)malloc(sizeof(double) * na * K);
  double* B = (double*)malloc(sizeof(double) * (long)g->n_r * K);
  double* M = (double*)malloc(sizeof(double) * (long)g->n_r * K);
  if (!U || !Q || !B || !M) { free(U); free(Q); free(B); free(M); return -2; }
  ora_build_U(g, nq, U);
  ora_build_Q(g, Q);
  ora_project(g, rho, U, B);
  ora_radial(g, B, M);
  ora_synthesize(g, M, Q, phi);
  if (B_out) memcpy(B_out, B, sizeof(double) * (long)g->n_r * K);
  if (M_out) memcpy(M_out, M, sizeof(double) * (long)g->n_r * K);
  free(U); free(Q); free(B); free(M);
  return 0;
}

/* Solve with prebuilt U and Q (the timed CPU baseline builds them beforehand). */
void ora_solve_prebuilt(const ora_grid* g, const double* U, const double* Q, const double* rho, double* phi,
                        double* B, double* M) {
  ora_project(g, rho, U, B);
  ora_radial(g, B, M);
  ora_synthesize(g, M, Q, phi);
}

/* Transpose of rho -> Phi:  Mbar = Q^T gphi, Bbar = K^T Mbar, grho = U Bbar. */
void ora_apply_T(const ora_grid* g, const double* U, const double* Q, const double* gphi, double* grho) {
  int K = ncols(g->l_max);
  int nr = g->n_r;
  double* Mb = (double*)calloc((size_t)nr * K, sizeof(double));
  double* Bb = (double*)calloc((size_t)nr * K, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int i = 0; i < nr; ++i) {
    double* m = Mb + (long)i * K;  /* zeroed by calloc */
    for (int p = 0; p < g->n_patch; ++p) {
      long base = nang_before(g, p), na = nang_patch(g, p);
      for (long a = 0; a < na; ++a) {
        const double ga = gphi[base * nr + (long)i * na + a];
        const double* q = Q + (base + a) * K;
        for (int c = 0; c < K; ++c) m[c] += q[c] * ga;
      }
    }
  }
#pragma omp parallel for collapse(2) schedule(static)
  for (int ip = 0; ip < nr; ++ip)
    for (int c = 0; c < K; ++c) {
      int l;
      (void)col_m(c, &l);
      double s = 0.0;
      for (int i = 0; i < nr; ++i) s += kernel_l(g, i, ip, l) * Mb[(long)i * K + c];
      Bb[(long)ip * K + c] = s;
    }
  for (int p = 0; p < g->n_patch; ++p) {
    long base = nang_before(g, p), na = nang_patch(g, p);
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < nr; ++i)
      for (long a = 0; a < na; ++a) {
        double s = 0.0;
        for (int c = 0; c < K; ++c) s += U[(base + a) * K + c] * Bb[(long)i * K + c];
        grho[base * nr + (long)i * na + a] = s;
      }
  }
  free(Mb);
  free(Bb);
}

/* O1: brute force with the addition theorem, Legendre polynomials only. */
int ora_solve_direct(const ora_grid* g, int nq, const double* rho, double* phi) {
  int L = g->l_max;
  int nr = g->n_r;
  long na = nang_total(g);
  double* xq = (double*)malloc(sizeof(double) * nq);
  double* wq = (double*)malloc(sizeof(double) * nq);
  ora_gauss_legendre(nq, xq, wq);
  /* quadrature points (global directions) and weights of every source cell */
  long nqp = (long)nq * nq;
  double* qdir = (double*)malloc(sizeof(double) * na * nqp * 3);
  double* qwt = (double*)malloc(sizeof(double) * na * nqp);
  double* edir = (double*)malloc(sizeof(double) * na * 3);
  /* K_l(i,i') table */
  double* Kt = (double*)malloc(sizeof(double) * (size_t)nr * nr * (L + 1));
  for (int i = 0; i < nr; ++i)
    for (int ip = 0; ip < nr; ++ip)
      for (int l = 0; l <= L; ++l) Kt[((size_t)i * nr + ip) * (L + 1) + l] = kernel_l(g, i, ip, l);
  for (int p = 0; p < g->n_patch; ++p) {
    double R[9];
    ora_euler_matrix(g->euler[3 * p], g->euler[3 * p + 1], g->euler[3 * p + 2], R);
    long base = nang_before(g, p);
    int nf = g->n_phi[p];
    for (long a = 0; a < nang_patch(g, p); ++a) {
      int j = (int)(a / nf), k = (int)(a % nf);
      double t0, t1, p0, p1, th, ph, v[3];
      cell_bounds(g, p, j, k, &t0, &t1, &p0, &p1);
      for (int qa = 0; qa < nq; ++qa)
        for (int qb = 0; qb < nq; ++qb) {
          double tq = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * xq[qa];
          double pq = 0.5 * (p0 + p1) + 0.5 * (p1 - p0) * xq[qb];
          double dens = patch_dir(g, p, tq, pq, v);
          long idx = (base + a) * nqp + qa * nq + qb;
          matvec(R, v, qdir + 3 * idx);
          qwt[idx] = 0.25 * (t1 - t0) * (p1 - p0) * wq[qa] * wq[qb] * dens;
        }
      eval_point_local(g, p, j, k, &th, &ph);
      patch_dir(g, p, th, ph, v);
      matvec(R, v, edir + 3 * (base + a));
    }
  }
#pragma omp parallel
  {
    double* A = (double*)malloc(sizeof(double) * na * (L + 1)); /* A[a'][l] */
    double* Pl = (double*)malloc(sizeof(double) * (L + 1));
    double* S = (double*)malloc(sizeof(double) * (size_t)nr * (L + 1)); /* S[i'][l] */
#pragma omp for schedule(dynamic, 1)
    for (long e = 0; e < na; ++e) {
      const double* ne = edir + 3 * e;
      for (long s = 0; s < na; ++s) {
        for (int l = 0; l <= L; ++l) A[s * (L + 1) + l] = 0.0;
        for (long q = 0; q < nqp; ++q) {
          const double* nd = qdir + 3 * (s * nqp + q);
          double x = ne[0] * nd[0] + ne[1] * nd[1] + ne[2] * nd[2];
          legendre_pl(L, x, Pl);
          double wt = qwt[s * nqp + q];
          for (int l = 0; l <= L; ++l) A[s * (L + 1) + l] += wt * Pl[l];
        }
      }
      /* S[i'][l] = sum_{a'} rho[i',a'] w[a'] A[a'][l] */
      for (int ip = 0; ip < nr; ++ip)
        for (int l = 0; l <= L; ++l) {
          double sacc = 0.0;
          for (int p = 0; p < g->n_patch; ++p) {
            long base = nang_before(g, p), np_ = nang_patch(g, p);
            for (long a = 0; a < np_; ++a)
              sacc += rho[base * nr + (long)ip * np_ + a] * g->w[base + a] * A[(base + a) * (L + 1) + l];
          }
          S[(size_t)ip * (L + 1) + l] = sacc;
        }
      /* which patch / flat index does evaluation cell e belong to? */
      int pe = 0;
      while (nang_before(g, pe + 1) <= e) ++pe;
      long be = nang_before(g, pe), ae = e - be, npe = nang_patch(g, pe);
      for (int i = 0; i < nr; ++i) {
        double tot = 0.0;
        for (int ip = 0; ip < nr; ++ip)
          for (int l = 0; l <= L; ++l) tot += Kt[((size_t)i * nr + ip) * (L + 1) + l] * S[(size_t)ip * (L + 1) + l];
        phi[be * nr + (long)i * npe + ae] = -g->G * tot;
      }
    }
    free(A);
    free(Pl);
    free(S);
  }
  free(xq); free(wq); free(qdir); free(qwt); free(edir); free(Kt);
  return 0;
}

/* O3: the older per-patch superposition scheme (Sect. 4.3). */
int ora_solve_perpatch(const ora_grid* g, int nq, const double* rho, double* phi) {
  int K = ncols(g->l_max);
  int nr = g->n_r;
  long na = nang_total(g);
  double* Ul = (double*)malloc(sizeof(double) * na * K);
  double* E = (double*)malloc(sizeof(double) * (size_t)g->n_patch * nr * K);
  double* Mg = (double*)malloc(sizeof(double) * (size_t)g->n_patch * nr * K);
  if (!Ul || !E || !Mg) { free(Ul); free(E); free(Mg); return -2; }
  ora_build_U_local(g, nq, Ul);
  double* nrm = norm_table(g->l_max);
  for (int p = 0; p < g->n_patch; ++p) {
    /* local moments of patch p only */
    ora_grid one = *g;
    long base = nang_before(g, p);
    one.n_patch = 1;
    one.euler = g->euler + 3 * p;
    one.n_theta = g->n_theta + p;
    one.n_phi = g->n_phi + p;
    one.theta_range = g->theta_range + 2 * p;
    one.phi_range = g->phi_range + 2 * p;
    one.w = g->w + base;
    one.kind = g->kind ? g->kind + p : NULL;
    ora_project(&one, rho + base * nr, Ul + base * K, E + (size_t)p * nr * K);
    ora_radial(&one, E + (size_t)p * nr * K, Mg + (size_t)p * nr * K);
  }
  for (int pe = 0; pe < g->n_patch; ++pe) {
    double Re[9];
    ora_euler_matrix(g->euler[3 * pe], g->euler[3 * pe + 1], g->euler[3 * pe + 2], Re);
    long be = nang_before(g, pe), npe = nang_patch(g, pe);
    int nf = g->n_phi[pe];
#pragma omp parallel
    {
      double* Y = (double*)malloc(sizeof(double) * (size_t)g->n_patch * K);
#pragma omp for schedule(static)
      for (long a = 0; a < npe; ++a) {
        int j = (int)(a / nf), k = (int)(a % nf);
        double th, ph, v[3], x[3];
        eval_point_local(g, pe, j, k, &th, &ph);
        patch_dir(g, pe, th, ph, v);
        matvec(Re, v, x); /* global direction */
        for (int p = 0; p < g->n_patch; ++p) {
          double Rp[9], xl[3];
          ora_euler_matrix(g->euler[3 * p], g->euler[3 * p + 1], g->euler[3 * p + 2], Rp);
          matTvec(Rp, x, xl); /* the point in frame p */
          harmonics_dir(g->l_max, nrm, xl, Y + (size_t)p * K);
        }
        for (int i = 0; i < nr; ++i) {
          double s = 0.0;
          for (int p = 0; p < g->n_patch; ++p)
            for (int c = 0; c < K; ++c) s += Y[(size_t)p * K + c] * Mg[((size_t)p * nr + i) * K + c];
          phi[be * nr + (long)i * npe + a] = -g->G * s;
        }
      }
      free(Y);
    }
  }
  free(Ul); free(E); free(Mg); free(nrm);
  return 0;
}

/* ------------------------------------------------------------ ellipsoid --- */

/* Carlson's R_F by the duplication theorem. */
double ora_carlson_rf(double x, double y, double z) {
  for (int it = 0; it < 200; ++it) {
    double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
    double lam = sx * sy + sy * sz + sz * sx;
    x = 0.25 * (x + lam); y = 0.25 * (y + lam); z = 0.25 * (z + lam);
    double mu = (x + y + z) / 3.0;
    double dx = 1.0 - x / mu, dy = 1.0 - y / mu, dz = 1.0 - z / mu;
    double e = fmax(fabs(dx), fmax(fabs(dy), fabs(dz)));
    if (e < 1e-4) {
      double e2 = dx * dy - dz * dz, e3 = dx * dy * dz;
      return (1.0 - e2 / 10.0 + e3 / 14.0 + e2 * e2 / 24.0 - 3.0 * e2 * e3 / 44.0) / sqrt(mu);
    }
  }
  return NAN;
}

/* Carlson's R_D by the duplication theorem. */
double ora_carlson_rd(double x, double y, double z) {
  double sum = 0.0, fac = 1.0;
  for (int it = 0; it < 200; ++it) {
    double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
    double lam = sx * sy + sy * sz + sz * sx;
    sum += fac / (sz * (z + lam));
    fac *= 0.25;
    x = 0.25 * (x + lam); y = 0.25 * (y + lam); z = 0.25 * (z + lam);
    double mu = (x + y + 3.0 * z) / 5.0;
    double dx = 1.0 - x / mu, dy = 1.0 - y / mu, dz = 1.0 - z / mu;
    double e = fmax(fabs(dx), fmax(fabs(dy), fabs(dz)));
    if (e < 1e-4) {
      double ea = dx * dy, eb = dz * dz, ec = ea - eb, ed = ea - 6.0 * eb, ee = ed + ec + ec;
      double s = 1.0 + ed * (-3.0 / 14.0 + 9.0 / 88.0 * ed - 4.5 / 26.0 * dz * ee) +
                 dz * (ee / 6.0 + dz * (-9.0 / 22.0 * ec + dz * 3.0 / 26.0 * ea));
      return 3.0 * sum + fac * s / (mu * sqrt(mu));
    }
  }
  return NAN;
}

/* u0 of Eq. u0: 0 inside the body, the positive root outside (the reading
 * with the two cases of the printed text exchanged; see the tests). */
static double ellipsoid_u0(double a, double b, double c, double X, double Y, double Z) {
  double f0 = X * X / (a * a) + Y * Y / (b * b) + Z * Z / (c * c);
  if (f0 <= 1.0) return 0.0;
  double lo = 0.0, hi = 1.0;
  while (X * X / (a * a + hi) + Y * Y / (b * b + hi) + Z * Z / (c * c + hi) > 1.0) hi *= 2.0;
  for (int it = 0; it < 400 && (hi - lo) > 1e-14 * fmax(1.0, hi); ++it) {
    double mid = 0.5 * (lo + hi);
    double f = X * X / (a * a + mid) + Y * Y / (b * b + mid) + Z * Z / (c * c + mid);
    if (f > 1.0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Eq. phiana with A,B,C = (2/3) R_D(...), D = 2 R_F(...). */
double ora_ellipsoid_phi(double a, double b, double c, double G, double rho0, double X, double Y, double Z) {
  double u0 = ellipsoid_u0(a, b, c, X, Y, Z);
  double A2 = a * a + u0, B2 = b * b + u0, C2 = c * c + u0;
  double IA = (2.0 / 3.0) * ora_carlson_rd(B2, C2, A2);
  double IB = (2.0 / 3.0) * ora_carlson_rd(C2, A2, B2);
  double IC = (2.0 / 3.0) * ora_carlson_rd(A2, B2, C2);
  double ID = 2.0 * ora_carlson_rf(A2, B2, C2);
  return ORA_PI * G * rho0 * a * b * c * (IA * X * X + IB * Y * Y + IC * Z * Z - ID);
}

/* The paper's recipe: bisection for u0, then Simpson quadrature of each of
 * the four integrals.  The semi-infinite range [u0, inf) is mapped onto
 * x in (0, 1] by u = u0 + s (1/x^2 - 1), which keeps every integrand finite
 * (the paper instead cuts the range at u = 1e16). */
typedef struct { double a2, b2, c2, u0, s; int which; } ell_ctx;

static double ell_integrand(const ell_ctx* e, double x) {
  if (x <= 0.0) return (e->which == 3) ? 2.0 / sqrt(e->s) : 0.0;
  double u = e->u0 + e->s * (1.0 / (x * x) - 1.0);
  double jac = 2.0 * e->s / (x * x * x);
  double pa = e->a2 + u, pb = e->b2 + u, pc = e->c2 + u;
  double base = sqrt(pa * pb * pc);
  double f;
  switch (e->which) {
    case 0: f = 1.0 / (base * pa); break;
    case 1: f = 1.0 / (base * pb); break;
    case 2: f = 1.0 / (base * pc); break;
    default: f = 1.0 / base; break;
  }
  return f * jac;
}

static double simpson_rec(const ell_ctx* e, double lo, double hi, double flo, double fmid, double fhi, double whole,
                          double tol, int depth) {
  double mid = 0.5 * (lo + hi);
  double lm = 0.5 * (lo + mid), rm = 0.5 * (mid + hi);
  double flm = ell_integrand(e, lm), frm = ell_integrand(e, rm);
  double left = (mid - lo) / 6.0 * (flo + 4.0 * flm + fmid);
  double right = (hi - mid) / 6.0 * (fmid + 4.0 * frm + fhi);
  double diff = left + right - whole;
  if (depth <= 0 || fabs(diff) <= 15.0 * tol) return left + right + diff / 15.0;
  return simpson_rec(e, lo, mid, flo, flm, fmid, left, 0.5 * tol, depth - 1) +
         simpson_rec(e, mid, hi, fmid, frm, fhi, right, 0.5 * tol, depth - 1);
}

static double ell_integral(const ell_ctx* e) {
  double f0 = ell_integrand(e, 0.0), f1 = ell_integrand(e, 1.0), fm = ell_integrand(e, 0.5);
  double whole = (1.0 / 6.0) * (f0 + 4.0 * fm + f1);
  double scale = fabs(f1) + fabs(fm);
  return simpson_rec(e, 0.0, 1.0, f0, fm, f1, whole, 1e-15 * scale, 40);
}

double ora_ellipsoid_phi_paper(double a, double b, double c, double G, double rho0, double X, double Y, double Z) {
  ell_ctx e;
  e.a2 = a * a; e.b2 = b * b; e.c2 = c * c;
  e.u0 = ellipsoid_u0(a, b, c, X, Y, Z);
  e.s = fmax(e.a2, fmax(e.b2, e.c2)) + e.u0;
  double I[4];
  for (int k = 0; k < 4; ++k) { e.which = k; I[k] = ell_integral(&e); }
  return ORA_PI * G * rho0 * a * b * c * (I[0] * X * X + I[1] * Y * Y + I[2] * Z * Z - I[3]);
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

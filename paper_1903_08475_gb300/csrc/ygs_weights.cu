// FP64 weight builder (step 1 of Sect. 4.3, evaluated once per grid).
//
//   d^l(pi/2)   the Fourier coefficients of the reduced Wigner matrix, by the
//               "pyramid" recurrences of Sect. 3 (starting from d^0_00 = 1);
//               the printed recurrences yield (-1)^m times the explicit-sum d
//               of Eq. wigner-d, and that sign is applied after the recursion;
//   d^l(beta)   the Fourier sum over u of d_{u m'}(pi/2) d_{u m}(pi/2) e^{i u beta}
//               with the prefactor i^{m-m'} (Sect. 3);
//   W^l         the real form of D^l = e^{-i m' alpha} d^l(beta) e^{-i m gamma}
//               (Eq. wigner-D) acting on the real harmonics of Eq. phispherical:
//               Y^t_lm(R^(g) xi) = sum_{m',t'} W_{(m,t),(m',t')} Y^{t'}_{lm'}(xi);
//   T_j         int sin(theta) N_lm P_lm(cos theta) dtheta over a local theta
//               cell (Eq. T_lm), by panel Gauss-Legendre quadrature;
//   C_k, S_k    int cos / sin (m phi) dphi over a local phi cell (Eqs. C_k^m, S_k^m);
//   U           (2/delta_m) w_jk sum_{m'} (W_{.,(m',C)} C_k + W_{.,(m',S)} S_k) T_j
//               (Eqs. U_C/U_S in real-harmonic form);
//   Q           -G N_lm P_lm(cos theta^+) {cos, sin}(m phi^+) at the global
//               direction of the evaluation point (Eqs. Q_C/Q_S);
//   gnomonic    the non-orthogonal patches of Sect. 6 (cube faces in
//               equiangular coordinates): U = (2/delta_m) w_jk times the
//               integral of the global real harmonic over the cell, by
//               10-point Gauss-Legendre panels in both coordinates with the
//               solid-angle density of the gnomonic map, instead of the
//               separable Wigner route; Q as above at the cell's point;
//   radial      a_i = R_in,i / (r_i^+)^(l+1), b_i = (r_i^-)^l R_out,i and the
//               ratios (r_{i-1}^+/r_i^+)^(l+1), (r_i^+/r_{i+1}^+)^l that turn
//               Eq. M_C into recurrences with every factor <= O(r^2)
//               (Eqs. R_in/R_out, step 4 of Sect. 4.3).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ygs_internal.h"

namespace ygs {
namespace {

// Offset of the (2l+1)^2 block of degree l in a packed table of blocks l = 0, 1, ...
__host__ __device__ inline long long blk(int l) { return (long long)l * (2 * l - 1) * (2 * l + 1) / 3; }

// Real column (l, m, t) within its degree block: r = 0 -> (0,C), 2m-1 -> (m,C), 2m -> (m,S).
__host__ __device__ inline int rm(int r) { return (r + 1) / 2; }
__host__ __device__ inline bool rs(int r) { return r > 0 && (r % 2 == 0); }  // sine type

__device__ inline int isqrt_col(int c) {
  int l = (int)sqrt((double)c);
  while ((l + 1) * (l + 1) <= c) ++l;
  while (l * l > c) --l;
  return l;
}

// Pyramid of d^l_{m'm}(pi/2) by the printed recurrences (one block), kept on
// the triangle 0 <= m <= m' <= l only: starting from d^l_{l m} and running the
// three-term recurrence down to m' = m is stable, whereas continuing it through
// m' < m loses digits fast with l (unitarity is off by 1e-7 at l = 32 and
// worse than O(1) at l = 64).  Values here are the recipe's (see dpi_fill_kernel).
__global__ void dpi_kernel(int L, double* R) {
  int t = threadIdx.x;
  if (t == 0) R[0] = 1.0;
  __syncthreads();
  for (int l = 1; l <= L; ++l) {
    int n = 2 * l + 1, np = 2 * l - 1;
    double* A = R + blk(l);
    const double* P = R + blk(l - 1);
    for (int m = t; m <= l; m += blockDim.x) {
      double v;
      if (m == 0)
        v = -sqrt((2.0 * l - 1.0) / (2.0 * l)) * P[(2 * l - 2) * np + (l - 1)];
      else
        v = -sqrt(l * (2.0 * l - 1.0) / (2.0 * (l + m) * (l + m - 1.0))) * P[(2 * l - 2) * np + (m - 1 + l - 1)];
      A[(2 * l) * n + (m + l)] = v;
      double dp1 = v, dp2 = 0.0;
      for (int mp = l - 1; mp >= m; --mp) {
        double den = (double)(l - mp) * (double)(l + mp + 1);
        double t1 = 2.0 * m / sqrt(den) * dp1;
        double t2 = (mp + 2 <= l) ? sqrt((double)(l - mp - 1) * (double)(l + mp + 2) / den) * dp2 : 0.0;
        double d = t1 - t2;
        A[(mp + l) * n + (m + l)] = d;
        dp2 = dp1;
        dp1 = d;
      }
    }
    __syncthreads();
  }
}

// Full d^l(pi/2) in the convention of Eq. wigner-d from the recipe triangle:
// the recipe yields (-1)^m d_{m'm}; the other entries follow from
//   d_{m'm} = (-1)^{m'-m} d_{-m',-m},   d_{-m',m}(pi/2) = (-1)^{l+m} d_{m'm}(pi/2),
//   d_{m'm} = (-1)^{m-m'} d_{m m'}.
__global__ void dpi_fill_kernel(int L, const double* R, double* D) {
  long long total = blk(L + 1);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int l = 0;
    while (blk(l + 1) <= e) ++l;
    int n = 2 * l + 1;
    int a = (int)((e - blk(l)) / n) - l, b = (int)((e - blk(l)) % n) - l;
    int sgn = 0;  // parity of the accumulated sign
    if (b < 0) {
      sgn += a - b;
      a = -a;
      b = -b;
    }
    if (a < 0) {
      sgn += l + b;
      a = -a;
    }
    if (a < b) {
      sgn += b - a;
      int t = a;
      a = b;
      b = t;
    }
    sgn += b;
    double v = R[blk(l) + (long long)(a + l) * n + (b + l)];
    D[e] = (sgn & 1) ? -v : v;
  }
}

// d^l_{m'm}(beta_g) = Re[ i^{m-m'} sum_u d_{u m'}(pi/2) d_{u m}(pi/2) e^{i u beta} ].
__global__ void dbeta_kernel(int L, const double* Dpi, const double* beta, double* Db) {
  extern __shared__ double cs[];  // cos(u beta), sin(u beta) for u = -l..l
  int l = blockIdx.x, g = blockIdx.y, n = 2 * l + 1;
  double b = beta[g];
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    double s, c;
    sincos((u - l) * b, &s, &c);
    cs[2 * u] = c;
    cs[2 * u + 1] = s;
  }
  __syncthreads();
  const double* P = Dpi + blk(l);
  double* O = Db + (long long)g * blk(L + 1) + blk(l);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int mp = idx / n - l, m = idx % n - l;
    double sr = 0.0, si = 0.0;
    for (int u = 0; u < n; ++u) {
      double prod = P[u * n + (mp + l)] * P[u * n + (m + l)];
      sr += prod * cs[2 * u];
      si += prod * cs[2 * u + 1];
    }
    int k = (((m - mp) % 4) + 4) % 4;
    O[idx] = (k == 0) ? sr : (k == 1) ? -si : (k == 2) ? -sr : si;
  }
}

// Real rotation coefficients W^l_{(m,t),(m',t')} of patch g.
__global__ void wreal_kernel(int L, const double* Db, const double* alpha, const double* gamma, double* W) {
  int l = blockIdx.x, g = blockIdx.y, n = 2 * l + 1;
  const double* d = Db + (long long)g * blk(L + 1) + blk(l);
  double* O = W + (long long)g * blk(L + 1) + blk(l);
  double al = alpha[g], ga = gamma[g];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int r = idx / n, q = idx % n;
    int m = rm(r), mp = rm(q);
    bool ts = rs(r), tps = rs(q);
    double sa = ((m + mp) & 1) ? -1.0 : 1.0;
    double dv = d[(mp + l) * n + (m + l)];
    double s1, c1;
    sincos(mp * al + m * ga, &s1, &c1);
    double ar = sa * dv * c1, ai = -sa * dv * s1;
    double br = 0.0, bi = 0.0;
    if (mp > 0) {
      double sb = (m & 1) ? -1.0 : 1.0;
      double dv2 = d[(-mp + l) * n + (m + l)];
      double s2, c2;
      sincos(mp * al - m * ga, &s2, &c2);
      br = sb * dv2 * c2;
      bi = sb * dv2 * s2;
    }
    double v;
    if (!tps) v = ts ? (ai + bi) : (ar + br);
    else v = ts ? (ar - br) : (-ai + bi);
    O[idx] = v;
  }
}

struct GL10 {
  double x[10], w[10];
};

// T[g][j][l][m'] = int_{theta_j^-}^{theta_j^+} sin(t) N_lm' P_lm'(cos t) dt.
__global__ void theta_int_kernel(int L, const double* th_lo, const double* dth, const int* nth, int npan_max,
                                 const int* npan, GL10 gl, double* T, long long tstride) {
  int j = blockIdx.x, g = blockIdx.y;
  if (j >= nth[g]) return;
  double t0 = th_lo[g] + j * dth[g];
  int np = npan[g];
  double h = dth[g] / np;
  double* Tj = T + (long long)g * tstride + (long long)j * (L + 1) * (L + 1);
  for (int mp = threadIdx.x; mp <= L; mp += blockDim.x) {
    for (int l = mp; l <= L; ++l) Tj[l * (L + 1) + mp] = 0.0;
    for (int pn = 0; pn < np; ++pn) {
      double a = t0 + pn * h;
      for (int q = 0; q < 10; ++q) {
        double tq = a + 0.5 * h * (1.0 + gl.x[q]);
        double wq = 0.5 * h * gl.w[q];
        double s, x;
        sincos(tq, &s, &x);
        double pmm = 1.0;
        for (int k = 1; k <= mp; ++k) pmm *= sqrt((2.0 * k - 1.0) / (2.0 * k)) * s;
        double p2 = 0.0, p1 = 0.0;
        for (int l = mp; l <= L; ++l) {
          double p;
          if (l == mp) p = pmm;
          else if (l == mp + 1) p = sqrt(2.0 * mp + 1.0) * x * pmm;
          else
            p = ((2.0 * l - 1.0) * x * p1 - sqrt((double)(l - 1 - mp) * (double)(l - 1 + mp)) * p2) /
                sqrt((double)(l - mp) * (double)(l + mp));
          p2 = p1;
          p1 = p;
          Tj[l * (L + 1) + mp] += wq * s * p;
        }
      }
    }
  }
  (void)npan_max;
}

// CS[g][k][m'][0|1] = int cos|sin(m' phi) dphi over the local phi cell k.
__global__ void phi_int_kernel(int L, const double* ph_lo, const double* dph, const int* nph, int nph_max, double* CS) {
  int g = blockIdx.y;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nph_max * (L + 1); e += gridDim.x * blockDim.x) {
    int k = e / (L + 1), mp = e % (L + 1);
    if (k >= nph[g]) continue;
    double d = dph[g];
    double pc = ph_lo[g] + (k + 0.5) * d;
    double* o = CS + ((long long)g * nph_max + k) * (L + 1) * 2 + 2 * mp;
    if (mp == 0) {
      o[0] = d;
      o[1] = 0.0;
    } else {
      double sc, cc;
      sincos(mp * pc, &sc, &cc);
      double f = 2.0 * sin(0.5 * mp * d) / mp;
      o[0] = f * cc;
      o[1] = f * sc;
    }
  }
}

struct PatchGeo {
  int nth[kMaxPatch], nph[kMaxPatch];
  int kind[kMaxPatch];           // ygs_patch_kind
  long long ang_off[kMaxPatch];  // row offset in the stored weight matrix
  long long w_off[kMaxPatch];    // offset of the patch's overlap weights
  double th_lo[kMaxPatch], dth[kMaxPatch], ph_lo[kMaxPatch], dph[kMaxPatch];
  double R[kMaxPatch][9];
};

// Global unit vector (x0, x1, x2) of the local coordinates (u, v) of patch g
// and the solid-angle density dOmega / (du dv): (theta, phi) patches
// (u = theta, v = phi, density sin theta), or gnomonic cube faces (X = tan u,
// Y = tan v, direction (X, Y, 1) / sqrt(1 + X^2 + Y^2), density
// (1 + X^2)(1 + Y^2) / (1 + X^2 + Y^2)^(3/2)).
__device__ inline double patch_dir(const PatchGeo& geo, int g, double u, double v, double& x0, double& x1,
                                   double& x2) {
  double v0, v1, v2, dens;
  if (geo.kind[g] == YGS_PATCH_GNOMONIC) {
    const double X = tan(u), Y = tan(v), r2 = 1.0 + X * X + Y * Y, ri = rsqrt(r2);
    v0 = X * ri;
    v1 = Y * ri;
    v2 = ri;
    dens = (1.0 + X * X) * (1.0 + Y * Y) * ri / r2;
  } else {
    double st, ct, sp, cp;
    sincos(u, &st, &ct);
    sincos(v, &sp, &cp);
    v0 = st * cp;
    v1 = st * sp;
    v2 = ct;
    dens = st;
  }
  const double* R = geo.R[g];
  x0 = R[0] * v0 + R[1] * v1 + R[2] * v2;
  x1 = R[3] * v0 + R[4] * v1 + R[5] * v2;
  x2 = R[6] * v0 + R[7] * v1 + R[8] * v2;
  return dens;
}

// U[(ang_off + a)][c_int] for every stored patch (grid-stride over a x c).
__global__ void u_kernel(int L, int K, int nwp, PatchGeo geo, const int* col_nat, const double* W, const double* T,
                         long long tstride, const double* CS, int nph_max, const double* w, double* U,
                         long long rows) {
  long long total = rows * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long row = e / K;
    int ci = (int)(e % K);
    int g = 0;
    while (g + 1 < nwp && geo.ang_off[g + 1] <= row) ++g;
    long long a = row - geo.ang_off[g];
    int j = (int)(a / geo.nph[g]), k = (int)(a % geo.nph[g]);
    int c = col_nat[ci];
    int l = isqrt_col(c);
    int r = c - l * l, n = 2 * l + 1;
    const double* Wr = W + (long long)g * blk(L + 1) + blk(l) + (long long)r * n;
    const double* Tj = T + (long long)g * tstride + (long long)j * (L + 1) * (L + 1) + (long long)l * (L + 1);
    const double* CSk = CS + ((long long)g * nph_max + k) * (L + 1) * 2;
    double acc = Wr[0] * Tj[0] * CSk[0];
    for (int mp = 1; mp <= l; ++mp) {
      double tv = Tj[mp];
      acc += tv * (Wr[2 * mp - 1] * CSk[2 * mp] + Wr[2 * mp] * CSk[2 * mp + 1]);
    }
    int m = rm(r);
    U[e] = (m == 0 ? 1.0 : 2.0) * w[geo.w_off[g] + a] * acc;
  }
}

// Q[(ang_off + a)][pos(l,m,t)] = -G Y^t_lm(global direction of the evaluation point).
__global__ void q_kernel(int L, int K, int nwp, PatchGeo geo, int eval, double G, const int* col_int, double* Q,
                         long long rows) {
  long long total = rows * (L + 1);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long row = e / (L + 1);
    int m = (int)(e % (L + 1));
    int g = 0;
    while (g + 1 < nwp && geo.ang_off[g + 1] <= row) ++g;
    long long a = row - geo.ang_off[g];
    int j = (int)(a / geo.nph[g]), k = (int)(a % geo.nph[g]);
    double off = (eval == YGS_EVAL_CELL_CENTRE) ? 0.5 : 1.0;
    double th = geo.th_lo[g] + (j + off) * geo.dth[g];
    double ph = geo.ph_lo[g] + (k + off) * geo.dph[g];
    double x0, x1, x2;
    patch_dir(geo, g, th, ph, x0, x1, x2);
    double s = sqrt(x0 * x0 + x1 * x1);
    double x = fmax(-1.0, fmin(1.0, x2));
    double phg = atan2(x1, x0);
    double smp, cmp;
    sincos(m * phg, &smp, &cmp);
    double pmm = 1.0;
    for (int kk = 1; kk <= m; ++kk) pmm *= sqrt((2.0 * kk - 1.0) / (2.0 * kk)) * s;
    double p2 = 0.0, p1 = 0.0;
    double* Qr = Q + row * K;
    for (int l = m; l <= L; ++l) {
      double p;
      if (l == m) p = pmm;
      else if (l == m + 1) p = sqrt(2.0 * m + 1.0) * x * pmm;
      else
        p = ((2.0 * l - 1.0) * x * p1 - sqrt((double)(l - 1 - m) * (double)(l - 1 + m)) * p2) /
            sqrt((double)(l - m) * (double)(l + m));
      p2 = p1;
      p1 = p;
      if (m == 0) {
        Qr[col_int[l * l]] = -G * p;
      } else {
        Qr[col_int[l * l + 2 * m - 1]] = -G * p * cmp;
        Qr[col_int[l * l + 2 * m]] = -G * p * smp;
      }
    }
  }
}

// U rows of the gnomonic patches: thread (row, m) integrates N_lm P_lm(cos
// theta) {cos, sin}(m phi) of the global direction over the cell, for every
// l >= m, by panels of 10-point Gauss-Legendre in both coordinates (panels no
// wider than 0.75 / (l_max + 1), twice as fine as the (theta, phi) route's, for
// the gnomonic map's stretching toward the face corners).  Rows of other
// patches are left as they are.
__global__ void u_gnomonic_kernel(int L, int K, int nwp, PatchGeo geo, const int* col_int, GL10 gl,
                                  const double* w, double* U, long long rows) {
  double accC[kMaxLmax + 1], accS[kMaxLmax + 1];
  long long total = rows * (L + 1);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long row = e / (L + 1);
    int m = (int)(e % (L + 1));
    int g = 0;
    while (g + 1 < nwp && geo.ang_off[g + 1] <= row) ++g;
    if (geo.kind[g] != YGS_PATCH_GNOMONIC) continue;
    long long a = row - geo.ang_off[g];
    int j = (int)(a / geo.nph[g]), k = (int)(a % geo.nph[g]);
    const double u0 = geo.th_lo[g] + j * geo.dth[g], v0 = geo.ph_lo[g] + k * geo.dph[g];
    const int nu = (int)fmax(1.0, ceil((L + 1) * geo.dth[g] / 0.75));
    const int nv = (int)fmax(1.0, ceil((L + 1) * geo.dph[g] / 0.75));
    const double hu = geo.dth[g] / nu, hv = geo.dph[g] / nv;
    for (int l = m; l <= L; ++l) accC[l] = accS[l] = 0.0;
    for (int pu = 0; pu < nu; ++pu)
      for (int qu = 0; qu < 10; ++qu) {
        const double uq = u0 + pu * hu + 0.5 * hu * (1.0 + gl.x[qu]);
        const double wu = 0.5 * hu * gl.w[qu];
        for (int pv = 0; pv < nv; ++pv)
          for (int qv = 0; qv < 10; ++qv) {
            const double vq = v0 + pv * hv + 0.5 * hv * (1.0 + gl.x[qv]);
            double x0, x1, x2;
            const double wt = wu * 0.5 * hv * gl.w[qv] * patch_dir(geo, g, uq, vq, x0, x1, x2);
            const double s = sqrt(x0 * x0 + x1 * x1), x = fmax(-1.0, fmin(1.0, x2));
            double smp, cmp;
            sincos(m * atan2(x1, x0), &smp, &cmp);
            double pmm = 1.0;
            for (int kk = 1; kk <= m; ++kk) pmm *= sqrt((2.0 * kk - 1.0) / (2.0 * kk)) * s;
            double p2 = 0.0, p1 = 0.0;
            for (int l = m; l <= L; ++l) {
              double pl;
              if (l == m) pl = pmm;
              else if (l == m + 1) pl = sqrt(2.0 * m + 1.0) * x * pmm;
              else
                pl = ((2.0 * l - 1.0) * x * p1 - sqrt((double)(l - 1 - m) * (double)(l - 1 + m)) * p2) /
                     sqrt((double)(l - m) * (double)(l + m));
              p2 = p1;
              p1 = pl;
              accC[l] += wt * pl * cmp;
              accS[l] += wt * pl * smp;
            }
          }
      }
    const double f = (m == 0 ? 1.0 : 2.0) * w[geo.w_off[g] + a];  // 2 / delta_m times the overlap weight
    double* Ur = U + row * K;
    for (int l = m; l <= L; ++l) {
      if (m == 0) {
        Ur[col_int[l * l]] = f * accC[l];
      } else {
        Ur[col_int[l * l + 2 * m - 1]] = f * accC[l];
        Ur[col_int[l * l + 2 * m]] = f * accS[l];
      }
    }
  }
}

// rad[0][l][i] = a, rad[1][l][i] = b, rad[2][l][i] = f_in, rad[3][l][i] = f_out.
__global__ void radial_kernel(int L, int nr, const double* e, double* rad) {
  long long total = (long long)(L + 1) * nr;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int l = (int)(t / nr), i = (int)(t % nr);
    double lo = e[i], hi = e[i + 1];
    double lq = (lo > 0.0) ? log(lo / hi) : -INFINITY;
    // a = (r^+)^2 (1 - q^(l+3)) / (l+3)
    double a = hi * hi * (-expm1((l + 3.0) * lq)) / (l + 3.0);
    // b = (r^-)^2 (1 - q^(l-2)) / (l-2), (r^-)^2 ln(1/q) at l = 2; shell 0 never contributes outward
    double b;
    if (lo <= 0.0) b = 0.0;
    else if (l == 2) b = lo * lo * (-lq);
    else b = lo * lo * (-expm1((l - 2.0) * lq)) / (l - 2.0);
    double fin = (i > 0) ? exp((l + 1.0) * log(e[i] / e[i + 1])) : 0.0;
    double fout = (i + 1 < nr) ? exp((double)l * log(e[i + 1] / e[i + 2])) : 0.0;
    long long stride = (long long)(L + 1) * nr;
    rad[t] = a;
    rad[stride + t] = b;
    rad[2 * stride + t] = fin;
    rad[3 * stride + t] = fout;
  }
}

void gl10(GL10* out) {
  const int n = 10;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    out->x[i] = -z;
    out->x[n - 1 - i] = z;
    out->w[i] = out->w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void euler_matrix(double a, double b, double g, double* R) {
  double ca = cos(a), sa = sin(a), cb = cos(b), sb = sin(b), cg = cos(g), sg = sin(g);
  R[0] = ca * cb * cg - sa * sg;
  R[1] = sa * cb * cg + ca * sg;
  R[2] = -sb * cg;
  R[3] = -ca * cb * sg - sa * cg;
  R[4] = -sa * cb * sg + ca * cg;
  R[5] = sb * sg;
  R[6] = ca * sb;
  R[7] = sa * sb;
  R[8] = cb;
}

// ---- create-time self-check of the rotation (Eqs. ylm_transform, wigner-D) ----
// At kCheckDirs fixed local directions xi of every stored patch g, the real
// harmonics of the global frame evaluated directly at x = R^(g) xi must equal
// the rotation of the local ones, Y_l(x) = W^l Y_l(xi), degree by degree.
// The directions: a Fibonacci spiral over the sphere (cos theta uniform in
// steps, phi advancing by the golden angle).
constexpr int kCheckDirs = 32;
constexpr double kCheckTol = 1e-10;  // |Y| <= 1 in this normalisation; the builder's error is ~1e-15

__device__ inline void check_dir(int s, double& th, double& ph) {
  th = acos(1.0 - 2.0 * (s + 0.5) / kCheckDirs);
  ph = fmod(s * 2.39996322972865332, 6.283185307179586);
}

// Y[(g * kCheckDirs + s)][l*l + r] (real harmonics, the columns' order) at
// direction s of patch g, in the local frame (global = 0) or at R^(g) xi.
__global__ void check_ylm_kernel(int L, int K, int nwp, PatchGeo geo, int global, double* Y) {
  const int s = blockIdx.x, g = blockIdx.y;
  double th, ph;
  check_dir(s, th, ph);
  double st, ct, sp, cp;
  sincos(th, &st, &ct);
  sincos(ph, &sp, &cp);
  double v0 = st * cp, v1 = st * sp, v2 = ct;
  if (global) {
    const double* R = geo.R[g];
    const double x0 = R[0] * v0 + R[1] * v1 + R[2] * v2;
    const double x1 = R[3] * v0 + R[4] * v1 + R[5] * v2;
    const double x2 = R[6] * v0 + R[7] * v1 + R[8] * v2;
    v0 = x0;
    v1 = x1;
    v2 = x2;
  }
  const double sn = sqrt(v0 * v0 + v1 * v1), x = fmax(-1.0, fmin(1.0, v2)), phi = atan2(v1, v0);
  double* Yr = Y + ((long long)g * kCheckDirs + s) * K;
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    double smp, cmp;
    sincos(m * phi, &smp, &cmp);
    double pmm = 1.0;
    for (int kk = 1; kk <= m; ++kk) pmm *= sqrt((2.0 * kk - 1.0) / (2.0 * kk)) * sn;
    double p2 = 0.0, p1 = 0.0;
    for (int l = m; l <= L; ++l) {
      double pv;
      if (l == m) pv = pmm;
      else if (l == m + 1) pv = sqrt(2.0 * m + 1.0) * x * pmm;
      else
        pv = ((2.0 * l - 1.0) * x * p1 - sqrt((double)(l - 1 - m) * (double)(l - 1 + m)) * p2) /
             sqrt((double)(l - m) * (double)(l + m));
      p2 = p1;
      p1 = pv;
      if (m == 0) {
        Yr[l * l] = pv;
      } else {
        Yr[l * l + 2 * m - 1] = pv * cmp;
        Yr[l * l + 2 * m] = pv * smp;
      }
    }
  }
}

// Largest |Y_glob - W Y_loc| over rows, degrees, directions and patches, as
// the bits of a non-negative double (atomicMax orders them like the values).
__global__ void check_rot_kernel(int L, int K, const double* W, const double* Yl, const double* Yg,
                                 unsigned long long* worst) {
  const int s = blockIdx.x, g = blockIdx.y;
  const double* yl = Yl + ((long long)g * kCheckDirs + s) * K;
  const double* yg = Yg + ((long long)g * kCheckDirs + s) * K;
  double m = 0.0;
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const int l = isqrt_col(c);
    const int n = 2 * l + 1, r = c - l * l;
    const double* Wr = W + (long long)g * blk(L + 1) + blk(l) + (long long)r * n;
    double acc = 0.0;
    for (int q = 0; q < n; ++q) acc = fma(Wr[q], yl[l * l + q], acc);
    m = fmax(m, fabs(acc - yg[c]));
  }
  if (!(m == m)) m = 1e300;  // a NaN fails the check
  atomicMax(worst, (unsigned long long)__double_as_longlong(m));
}

// Testing hook: flips the sign of every W^1 block (a mis-signed rotation).
__global__ void perturb_w_kernel(int L, int nwp, double* W) {
  for (int g = 0; g < nwp; ++g)
    for (int idx = threadIdx.x; idx < 9 && L >= 1; idx += blockDim.x) W[(long long)g * blk(L + 1) + blk(1) + idx] *= -1.0;
}

struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  cudaError_t alloc(T** p, size_t n) {
    cudaError_t e = dev_malloc((void**)p, n * sizeof(T) + 16);
    if (e == cudaSuccess) ptrs.push_back((void*)*p);
    return e;
  }
};

}  // namespace

#define YGS_TRY(expr)                                                                   \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess) {                                                            \
      set_error(std::string("weights: ") + #expr + ": " + cudaGetErrorString(_e));      \
      return _e == cudaErrorMemoryAllocation ? YGS_ERR_OOM : YGS_ERR_CUDA;              \
    }                                                                                   \
  } while (0)

ygs_status build_weights(ygs_plan* p) {
  const int L = p->l_max, K = p->K, nwp = p->n_wpatch;
  Scratch s;
  // host geometry of the stored patches
  PatchGeo geo{};
  std::vector<double> th_lo(nwp), dth(nwp), ph_lo(nwp), dph(nwp), beta(nwp), alpha(nwp), gamma(nwp);
  std::vector<int> npan(nwp), nth(nwp), nph(nwp);
  int nth_max = 1, nph_max = 1;
  for (int g = 0; g < nwp; ++g) {
    nth[g] = p->nth[g];
    nph[g] = p->nph[g];
    th_lo[g] = p->theta_range[2 * g];
    dth[g] = (p->theta_range[2 * g + 1] - p->theta_range[2 * g]) / p->nth[g];
    ph_lo[g] = p->phi_range[2 * g];
    dph[g] = (p->phi_range[2 * g + 1] - p->phi_range[2 * g]) / p->nph[g];
    alpha[g] = p->euler[3 * g];
    beta[g] = p->euler[3 * g + 1];
    gamma[g] = p->euler[3 * g + 2];
    // panels of width <= 1.5 / (l_max + 1) keep the 10-point rule exact to rounding
    npan[g] = (int)std::max(1.0, std::ceil((L + 1) * dth[g] / 1.5));
    nth_max = std::max(nth_max, nth[g]);
    nph_max = std::max(nph_max, nph[g]);
    geo.nth[g] = nth[g];
    geo.nph[g] = nph[g];
    geo.kind[g] = p->kind[g];
    geo.ang_off[g] = p->ang_off[g];
    geo.w_off[g] = p->ang_off[g];
    geo.th_lo[g] = th_lo[g];
    geo.dth[g] = dth[g];
    geo.ph_lo[g] = ph_lo[g];
    geo.dph[g] = dph[g];
    euler_matrix(alpha[g], beta[g], gamma[g], geo.R[g]);
  }
  // column permutation tables
  std::vector<int> col_int(K);
  for (int ci = 0; ci < K; ++ci) col_int[p->col_perm[ci]] = ci;
  std::vector<int> col_l(K);
  for (int ci = 0; ci < K; ++ci) {
    int c = p->col_perm[ci], l = 0;
    while ((l + 1) * (l + 1) <= c) ++l;
    col_l[ci] = l;
  }
  int* d_col_int = nullptr;
  YGS_TRY(s.alloc(&d_col_int, K));
  YGS_TRY(cudaMemcpy(d_col_int, col_int.data(), K * sizeof(int), cudaMemcpyHostToDevice));
  YGS_TRY(cudaMemcpy(p->col_nat, p->col_perm.data(), K * sizeof(int), cudaMemcpyHostToDevice));
  YGS_TRY(cudaMemcpy(p->col_l, col_l.data(), K * sizeof(int), cudaMemcpyHostToDevice));

  auto up = [&](const std::vector<double>& v, double** d) -> cudaError_t {
    cudaError_t e = s.alloc(d, v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
  };
  auto upi = [&](const std::vector<int>& v, int** d) -> cudaError_t {
    cudaError_t e = s.alloc(d, v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
  };
  double *d_alpha, *d_beta, *d_gamma, *d_thlo, *d_dth, *d_phlo, *d_dph, *d_w, *d_edges;
  int *d_npan, *d_nth, *d_nph;
  YGS_TRY(up(alpha, &d_alpha));
  YGS_TRY(up(beta, &d_beta));
  YGS_TRY(up(gamma, &d_gamma));
  YGS_TRY(up(th_lo, &d_thlo));
  YGS_TRY(up(dth, &d_dth));
  YGS_TRY(up(ph_lo, &d_phlo));
  YGS_TRY(up(dph, &d_dph));
  YGS_TRY(upi(npan, &d_npan));
  YGS_TRY(upi(nth, &d_nth));
  YGS_TRY(upi(nph, &d_nph));
  YGS_TRY(up(p->edges, &d_edges));
  {
    // the stored patches' overlap weights (patch 0 only when symmetric)
    std::vector<double> wv(p->w_host.begin(), p->w_host.begin() + p->nang_wtotal);
    YGS_TRY(up(wv, &d_w));
  }

  // Wigner tables
  double *d_rec, *d_dpi, *d_db, *d_W;
  YGS_TRY(s.alloc(&d_rec, blk(L + 1)));
  YGS_TRY(s.alloc(&d_dpi, blk(L + 1)));
  YGS_TRY(s.alloc(&d_db, (size_t)nwp * blk(L + 1)));
  YGS_TRY(s.alloc(&d_W, (size_t)nwp * blk(L + 1)));
  dpi_kernel<<<1, 256>>>(L, d_rec);
  YGS_TRY(cudaGetLastError());
  dpi_fill_kernel<<<256, 256>>>(L, d_rec, d_dpi);
  YGS_TRY(cudaGetLastError());
  dbeta_kernel<<<dim3(L + 1, nwp), 256, (2 * L + 1) * 2 * sizeof(double)>>>(L, d_dpi, d_beta, d_db);
  YGS_TRY(cudaGetLastError());
  wreal_kernel<<<dim3(L + 1, nwp), 256>>>(L, d_db, d_alpha, d_gamma, d_W);
  YGS_TRY(cudaGetLastError());
  {
    // the rotation self-check: Y(R xi) = W Y(xi) at fixed directions
    const char* hook = getenv("YGS_TEST_PERTURB_WIGNER");
    if (hook && hook[0] == '1') {
      perturb_w_kernel<<<1, 32>>>(L, nwp, d_W);
      YGS_TRY(cudaGetLastError());
    }
    double *d_yl, *d_yg;
    unsigned long long* d_worst;
    YGS_TRY(s.alloc(&d_yl, (size_t)nwp * kCheckDirs * K));
    YGS_TRY(s.alloc(&d_yg, (size_t)nwp * kCheckDirs * K));
    YGS_TRY(s.alloc(&d_worst, 1));
    YGS_TRY(cudaMemset(d_worst, 0, sizeof(unsigned long long)));
    check_ylm_kernel<<<dim3(kCheckDirs, nwp), 64>>>(L, K, nwp, geo, 0, d_yl);
    YGS_TRY(cudaGetLastError());
    check_ylm_kernel<<<dim3(kCheckDirs, nwp), 64>>>(L, K, nwp, geo, 1, d_yg);
    YGS_TRY(cudaGetLastError());
    check_rot_kernel<<<dim3(kCheckDirs, nwp), 256>>>(L, K, d_W, d_yl, d_yg, d_worst);
    YGS_TRY(cudaGetLastError());
    unsigned long long bits = 0;
    YGS_TRY(cudaMemcpy(&bits, d_worst, sizeof(bits), cudaMemcpyDeviceToHost));
    double worst;
    memcpy(&worst, &bits, sizeof(worst));
    if (!(worst <= kCheckTol)) {
      char msg[160];
      snprintf(msg, sizeof msg, "weights: rotation self-check failed: |Y(R xi) - W Y(xi)| = %.3e > %.1e", worst,
               kCheckTol);
      set_error(msg);
      return YGS_ERR_NUMERIC;
    }
  }

  // separable local integrals
  long long tstride = (long long)nth_max * (L + 1) * (L + 1);
  double *d_T, *d_CS;
  YGS_TRY(s.alloc(&d_T, (size_t)nwp * tstride));
  YGS_TRY(s.alloc(&d_CS, (size_t)nwp * nph_max * (L + 1) * 2));
  GL10 gl;
  gl10(&gl);
  theta_int_kernel<<<dim3(nth_max, nwp), 128>>>(L, d_thlo, d_dth, d_nth, 0, d_npan, gl, d_T, tstride);
  YGS_TRY(cudaGetLastError());
  phi_int_kernel<<<dim3(64, nwp), 256>>>(L, d_phlo, d_dph, d_nph, nph_max, d_CS);
  YGS_TRY(cudaGetLastError());

  // U and Q
  long long rows = p->nang_wtotal;
  u_kernel<<<2048, 256>>>(L, K, nwp, geo, p->col_nat, d_W, d_T, tstride, d_CS, nph_max, d_w, p->U, rows);
  YGS_TRY(cudaGetLastError());
  bool any_gnomonic = false;
  for (int g = 0; g < nwp; ++g) any_gnomonic |= p->kind[g] == YGS_PATCH_GNOMONIC;
  if (any_gnomonic) {  // their rows by direct quadrature (the separable route does not apply)
    u_gnomonic_kernel<<<1024, 128>>>(L, K, nwp, geo, d_col_int, gl, d_w, p->U, rows);
    YGS_TRY(cudaGetLastError());
  }
  q_kernel<<<1024, 128>>>(L, K, nwp, geo, p->eval, p->G, d_col_int, p->Q, rows);
  YGS_TRY(cudaGetLastError());
  radial_kernel<<<64, 256>>>(L, p->n_r, d_edges, p->rad);
  YGS_TRY(cudaGetLastError());
  YGS_TRY(cudaDeviceSynchronize());
  return YGS_OK;
}

}  // namespace ygs

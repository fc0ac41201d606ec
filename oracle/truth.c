/*
 * Stiff-chemistry truth for the reaction-step oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain FP64 C. The chemistry network of the method (Sec. 2) stands in for stiff ODE
 * integration of the cell chemistry (the paper's reference is Cantera / CVODE, Sec. 2 and
 * Sec. 5.1); this file integrates that chemistry directly so the network can be trained on,
 * and compared with, its result. It shares no code with the CUDA library.
 *
 * Model (closed, adiabatic, isobaric reactor; this project's reading, the paper prints none):
 *   state Y (mass fractions); T follows from h(T, p, Y) = h0 (Peng-Robinson real-fluid
 *   enthalpy, NASA-7 ideal gas) by safeguarded Newton at every right-hand-side evaluation;
 *   dY_k/dt = W_k wdot_k / rho,  wdot_k = sum_r (nu''_kr - nu'_kr) q_r,
 *   q_r = kf_r prod c^nu' - kr_r prod c^nu'',  c_k = rho Y_k / W_k,
 *   kf = A T^beta exp(-Ea / (R T)) in CGS-molar units (concentrations in mol/cm^3),
 *   kr = kf / Kc,  Kc = Kp (p0 / (R T))^(sum nu'' - sum nu'),  Kp = exp(-dG0 / (R T)),
 *   where the drawn Arrhenius expression gives the rate constant of the favoured direction
 *   (kf when Kc >= 1, else kr; the other from Kc),
 *   dG0 = sum_k (nu'' - nu')_k (h_k - T s_k)(T) at p0 = 101325 Pa.
 * Integrator: variable-order (1..5), quasi-constant step-size BDF in backward-difference
 * form (Shampine & Reichelt, "The MATLAB ODE suite", SIAM J. Sci. Comput. 18, 1997),
 * simplified Newton with a finite-difference Jacobian and dense LU with partial pivoting,
 * error control on the weighted RMS norm with atol + rtol |y|.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define RGAS 8.31446261815324
#define P0 101325.0
#define SQ2 1.4142135623730951
#define MAXN 64
#define MAXORD 5

typedef struct {
  int n, R;
  const double *W, *Tc, *pc, *omega, *kij, *nasa; /* nasa [n*7] */
  const double *nu_f, *nu_r;                      /* [n*R] row-major (species, reaction) */
  const double *A, *beta, *Ea;                    /* [R] */
} mech_t;

/* ------------------------------------------------------------ thermodynamics */

static void species_thermo(const double* a, double T, double* cpR, double* hRT, double* sR) {
  *cpR = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
  *hRT = a[0] + T * (a[1] / 2 + T * (a[2] / 3 + T * (a[3] / 4 + T * a[4] / 5))) + a[5] / T;
  *sR = a[0] * log(T) + T * (a[1] + T * (a[2] / 2 + T * (a[3] / 3 + T * a[4] / 4))) + a[6];
}

static double cubic_val(double Z, double c2, double c1, double c0) { return ((Z + c2) * Z + c1) * Z + c0; }

static double polish(double Z, double c2, double c1, double c0) {
  for (int it = 0; it < 8; ++it) {
    const double f = cubic_val(Z, c2, c1, c0);
    const double fp = (3 * Z + 2 * c2) * Z + c1;
    if (fp == 0) break;
    const double Zn = Z - f / fp;
    if (!(fabs(cubic_val(Zn, c2, c1, c0)) < fabs(f))) break;
    Z = Zn;
  }
  return Z;
}

static double gdep(double Z, double A, double B) {
  return Z - 1 - log(Z - B) - A / (2 * SQ2 * B) * log((Z + (1 + SQ2) * B) / (Z + (1 - SQ2) * B));
}

/* Peng-Robinson state of composition Y at (T, p): mass-specific h, cp, density; 0 if no root. */
static int pr_state(const mech_t* m, double T, double p, const double* Y, double* h, double* cp,
                    double* rho) {
  const int n = m->n;
  double X[MAXN], sa[MAXN], sa1[MAXN], sa2[MAXN];
  double inv = 0;
  for (int k = 0; k < n; ++k) inv += Y[k] / m->W[k];
  const double Wm = 1 / inv;
  double bm = 0;
  for (int k = 0; k < n; ++k) {
    X[k] = Y[k] * Wm / m->W[k];
    const double Tc = m->Tc[k], pc = m->pc[k], w = m->omega[k];
    const double ac = 0.45724 * RGAS * RGAS * Tc * Tc / pc;
    const double b = 0.07780 * RGAS * Tc / pc;
    const double kap = 0.37464 + 1.54226 * w - 0.26992 * w * w;
    const double sac = sqrt(ac);
    sa[k] = sac * (1 + kap * (1 - sqrt(T / Tc)));
    sa1[k] = -sac * kap / (2 * sqrt(T * Tc));
    sa2[k] = sac * kap / (4 * sqrt(Tc) * pow(T, 1.5));
    bm += X[k] * b;
  }
  double am = 0, da = 0, d2a = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double w = X[i] * X[j] * (1 - m->kij[i * n + j]);
      am += w * sa[i] * sa[j];
      da += w * (sa1[i] * sa[j] + sa[i] * sa1[j]);
      d2a += w * (sa2[i] * sa[j] + 2 * sa1[i] * sa1[j] + sa[i] * sa2[j]);
    }
  const double RT = RGAS * T;
  const double A = am * p / (RT * RT), B = bm * p / RT;
  const double c2 = -(1 - B), c1 = A - 3 * B * B - 2 * B, c0 = -(A * B - B * B - B * B * B);
  const double P = c1 - c2 * c2 / 3, Q = 2 * c2 * c2 * c2 / 27 - c2 * c1 / 3 + c0;
  const double disc = Q * Q / 4 + P * P * P / 27;
  double roots[3];
  int nr = 0;
  if (disc > 0) {
    const double sq = sqrt(disc);
    const double u = cbrt(-Q / 2 - (Q >= 0 ? sq : -sq));
    roots[nr++] = polish((u != 0 ? u - P / (3 * u) : 0) - c2 / 3, c2, c1, c0);
  } else {
    const double mm = 2 * sqrt(fmax(-P / 3, 0));
    double cphi = P < 0 ? (3 * Q / (2 * P)) * sqrt(-3 / P) : 0;
    cphi = fmin(fmax(cphi, -1), 1);
    const double phi = acos(cphi);
    for (int k = 0; k < 3; ++k)
      roots[nr++] = polish(mm * cos(phi / 3 - 2 * M_PI * k / 3) - c2 / 3, c2, c1, c0);
  }
  /* least departure Gibbs energy among real roots above B; scanning in descending order
   * makes an exact tie keep the larger root */
  double Z = NAN, gbest = INFINITY;
  for (int a = 0; a < nr; ++a)
    for (int b2 = a + 1; b2 < nr; ++b2)
      if (roots[b2] > roots[a]) { const double t = roots[a]; roots[a] = roots[b2]; roots[b2] = t; }
  for (int k = 0; k < nr; ++k) {
    const double r = roots[k];
    if (!(r > B)) continue;
    const double g = gdep(r, A, B);
    if (g < gbest - 1e-12) { gbest = g; Z = r; }
  }
  if (!(Z > B)) return 0;
  const double Zp = Z + (1 + SQ2) * B, Zm = Z + (1 - SQ2) * B;
  const double L = log(Zp / Zm);
  const double hdep = RT * (Z - 1) + (T * da - am) / (2 * SQ2 * bm) * L;
  /* cp departure: dZ/dT from the implicit cubic */
  const double dB = -B / T, dA = A * (da / am - 2 / T);
  const double FZ = 3 * Z * Z - 2 * (1 - B) * Z + (A - 3 * B * B - 2 * B);
  const double FA = Z - B, FB = Z * Z - (6 * B + 2) * Z - (A - 2 * B - 3 * B * B);
  const double dZ = -(FA * dA + FB * dB) / FZ;
  const double dL = (dZ + (1 + SQ2) * dB) / Zp - (dZ + (1 - SQ2) * dB) / Zm;
  const double kk = 1 / (2 * SQ2 * bm);
  const double cpdep = RGAS * (Z - 1) + RT * dZ + kk * T * d2a * L + kk * (T * da - am) * dL;
  double hig = 0, cpig = 0;
  for (int k = 0; k < n; ++k) {
    double cpR, hRT, sR;
    species_thermo(m->nasa + 7 * k, T, &cpR, &hRT, &sR);
    hig += Y[k] * RGAS * T * hRT / m->W[k];
    cpig += Y[k] * RGAS * cpR / m->W[k];
  }
  *h = hig + hdep / Wm;
  *cp = cpig + cpdep / Wm;
  *rho = p * Wm / (Z * RGAS * T);
  return 1;
}

/* T from h(T, p, Y) = h0: Newton with slope cp in a shrinking bracket [50, 5000] K; a step
 * within 1e-12 T ends the iteration, a longer step leaving the bracket is bisected. */
static int solve_T(const mech_t* m, double p, const double* Y, double h0, double* T, double* rho) {
  double lo = 50, hi = 5000, t = fmin(fmax(*T, lo), hi);
  for (int it = 0; it < 200; ++it) {
    double h, cp, r;
    if (!pr_state(m, t, p, Y, &h, &cp, &r)) return 0;
    const double f = h - h0;
    if (f > 0) hi = fmin(hi, t); else lo = fmax(lo, t);
    double tn = t - f / cp;
    const int done = isfinite(tn) && fabs(tn - t) <= 1e-12 * t;
    if (!done && !(isfinite(tn) && tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    t = tn;
    if (done) {
      *T = t;
      if (rho) {
        if (!pr_state(m, t, p, Y, &h, &cp, &r)) return 0;
        *rho = r;
      }
      return 1;
    }
  }
  return 0;
}

/* dY/dt at composition Y (T updated in place as the warm start of its Newton solve). The
 * integrator may carry trace species slightly below zero; the equation of state and the
 * concentrations see max(Y, 0). */
static int rhs(const mech_t* m, double p, double h0, const double* Yin, double* T, double* f) {
  const int n = m->n, R = m->R;
  double Y[MAXN];
  for (int k = 0; k < n; ++k) Y[k] = fmax(Yin[k], 0.0);
  double rho;
  if (!solve_T(m, p, Y, h0, T, &rho)) return 0;
  const double t = *T, RT = RGAS * t;
  double c[MAXN], g0[MAXN];
  for (int k = 0; k < n; ++k) {
    c[k] = rho * Y[k] / m->W[k] * 1e-6; /* mol/cm^3 */
    double cpR, hRT, sR;
    species_thermo(m->nasa + 7 * k, t, &cpR, &hRT, &sR);
    g0[k] = RT * (hRT - sR); /* molar Gibbs energy at p0 */
    f[k] = 0;
  }
  for (int r = 0; r < R; ++r) {
    double dG = 0, dnu = 0, lf = 0, lb = 0;
    double prf = 1, prb = 1;
    for (int k = 0; k < n; ++k) {
      const double a = m->nu_f[k * R + r], b = m->nu_r[k * R + r];
      dG += (b - a) * g0[k];
      dnu += b - a;
      for (int e = 0; e < (int)a; ++e) prf *= c[k];
      for (int e = 0; e < (int)b; ++e) prb *= c[k];
    }
    /* Kc in mol/cm^3 units: Kp (p0 / (R T) * 1e-6)^dnu. The drawn Arrhenius expression is
     * the rate constant of the thermodynamically favoured direction (Kc >= 1 for the forward
     * one); the other direction follows from Kc, so no rate exceeds its Arrhenius value. */
    const double la = log(m->A[r]) + m->beta[r] * log(t) - m->Ea[r] / RT;
    const double lKc = -dG / RT + dnu * log(P0 / RT * 1e-6);
    if (lKc >= 0) {
      lf = la;
      lb = la - lKc;
    } else {
      lb = la;
      lf = la + lKc;
    }
    const double q = exp(lf) * prf - exp(lb) * prb; /* mol/cm^3/s */
    for (int k = 0; k < n; ++k) {
      const double nu = m->nu_r[k * R + r] - m->nu_f[k * R + r];
      if (nu != 0) f[k] += nu * q;
    }
  }
  for (int k = 0; k < n; ++k) f[k] = m->W[k] * f[k] * 1e6 / rho;
  return 1;
}

/* ------------------------------------------------------------ dense LU */

static int lu_factor(double* a, int n, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    if (best == 0) return 0;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) { const double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
    for (int i = k + 1; i < n; ++i) {
      const double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return 1;
}

static void lu_solve(const double* a, int n, const int* piv, double* b) {
  for (int k = 0; k < n; ++k) {
    if (piv[k] != k) { const double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = k + 1; i < n; ++i) b[i] -= a[i * n + k] * b[k];
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int j = k + 1; j < n; ++j) b[k] -= a[k * n + j] * b[j];
    b[k] /= a[k * n + k];
  }
}

/* ------------------------------------------------------------ BDF */

typedef struct {
  const mech_t* m;
  double p, h0, T;
  long nfev;
} ctx_t;

static int f_eval(ctx_t* c, const double* y, double* f) {
  c->nfev++;
  return rhs(c->m, c->p, c->h0, y, &c->T, f);
}

static double wrms(const double* e, const double* y, int n, double rtol, double atol) {
  double s = 0;
  for (int i = 0; i < n; ++i) {
    const double w = atol + rtol * fabs(y[i]);
    s += (e[i] / w) * (e[i] / w);
  }
  return sqrt(s / n);
}

/* D <- (R U)^T D for a step-size change by `factor` (interpolating polynomial through the
 * backward differences evaluated on the new spacing). */
static void rescale_D(double D[][MAXN], int order, double factor, int n) {
  double Rm[MAXORD + 1][MAXORD + 1], Um[MAXORD + 1][MAXORD + 1], RU[MAXORD + 1][MAXORD + 1];
  for (int pass = 0; pass < 2; ++pass) {
    const double fac = pass == 0 ? factor : 1.0;
    double M[MAXORD + 1][MAXORD + 1];
    for (int j = 0; j <= order; ++j) M[0][j] = 1;
    for (int i = 1; i <= order; ++i) {
      M[i][0] = 0;
      for (int j = 1; j <= order; ++j) M[i][j] = (i - 1 - fac * j) / i;
    }
    double (*out)[MAXORD + 1] = pass == 0 ? Rm : Um;
    for (int j = 0; j <= order; ++j) {
      double prod = 1;
      for (int i = 0; i <= order; ++i) { prod *= M[i][j]; out[i][j] = prod; }
    }
  }
  for (int i = 0; i <= order; ++i)
    for (int j = 0; j <= order; ++j) {
      double s = 0;
      for (int k = 0; k <= order; ++k) s += Rm[i][k] * Um[k][j];
      RU[i][j] = s;
    }
  double Dn[MAXORD + 1][MAXN];
  for (int j = 0; j <= order; ++j)
    for (int v = 0; v < n; ++v) {
      double s = 0;
      for (int i = 0; i <= order; ++i) s += RU[i][j] * D[i][v];
      Dn[j][v] = s;
    }
  for (int j = 0; j <= order; ++j) memcpy(D[j], Dn[j], sizeof(double) * n);
}

/* Finite-difference Jacobian of the right-hand side at y. */
static int fd_jacobian(ctx_t* c, const double* y, double* J) {
  const int n = c->m->n;
  double f0[MAXN], yp[MAXN], fj[MAXN];
  const double Tsave = c->T;
  if (!f_eval(c, y, f0)) return 0;
  for (int j = 0; j < n; ++j) {
    memcpy(yp, y, sizeof(double) * n);
    const double del = sqrt(2.2e-16) * fmax(fabs(y[j]), 1e-10);
    yp[j] += del;
    if (!f_eval(c, yp, fj)) return 0;
    for (int i = 0; i < n; ++i) J[i * n + j] = (fj[i] - f0[i]) / del;
  }
  c->T = Tsave;
  return 1;
}

/* Integrates y from 0 to t_end; returns 1 on success (y holds y(t_end)), 0 on failure. */
static int bdf_integrate(ctx_t* c, double* y, double t_end, double rtol, double atol, long* nsteps) {
  const int n = c->m->n;
  const int newton_max = 4;
  double gamma[MAXORD + 2], alpha[MAXORD + 2], econst[MAXORD + 2];
  gamma[0] = 0;
  for (int k = 1; k <= MAXORD + 1; ++k) gamma[k] = gamma[k - 1] + 1.0 / k;
  for (int k = 0; k <= MAXORD + 1; ++k) { alpha[k] = gamma[k]; econst[k] = 1.0 / (k + 1); }
  double D[MAXORD + 3][MAXN];
  memset(D, 0, sizeof D);
  double f0[MAXN];
  if (!f_eval(c, y, f0)) return 0;
  if (nsteps) *nsteps = 0;
  /* initial step: 1 % of the time the fastest component needs to move by its tolerance */
  double fn = 0;
  for (int i = 0; i < n; ++i) fn = fmax(fn, fabs(f0[i]) / (atol + rtol * fabs(y[i])));
  double h = fn > 0 ? fmin(t_end, 1e-2 / fn) : t_end;
  h = fmax(h, 1e-30);
  memcpy(D[0], y, sizeof(double) * n);
  for (int i = 0; i < n; ++i) D[1][i] = f0[i] * h;
  int order = 1, equal_steps = 0;
  double t = 0;
  double J[MAXN * MAXN], LU[MAXN * MAXN];
  int piv[MAXN];
  if (!fd_jacobian(c, y, J)) return 0;
  int jac_current = 1, lu_valid = 0;
  double lu_c = 0;
  long steps = 0;
  double ypred[MAXN], psi[MAXN], d[MAXN], ynew[MAXN], fy[MAXN], dy[MAXN];
  while (t < t_end) {
    if (++steps > 2000000) return -1;
    if (nsteps) *nsteps = steps;
    if (t + h > t_end) {
      rescale_D(D, order, (t_end - t) / h, n);
      h = t_end - t;
      equal_steps = 0;
    }
    /* simplified Newton on the corrector; on failure refresh the Jacobian once, then halve h */
    int converged = 0;
    double cc = 0;
    for (;;) {
      cc = h / alpha[order];
      for (int i = 0; i < n; ++i) {
        double s = 0, q = 0;
        for (int j = 0; j <= order; ++j) s += D[j][i];
        for (int j = 1; j <= order; ++j) q += gamma[j] * D[j][i];
        ypred[i] = s;
        psi[i] = q / alpha[order];
        d[i] = 0;
      }
      int ok = 1;
      if (!lu_valid || lu_c != cc) {
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) LU[i * n + j] = (i == j ? 1.0 : 0.0) - cc * J[i * n + j];
        ok = lu_factor(LU, n, piv);
        if (!ok) return -2;
        lu_valid = ok;
        lu_c = cc;
      }
      double dn_prev = 0;
      for (int it = 0; ok && it < newton_max; ++it) {
        for (int i = 0; i < n; ++i) ynew[i] = ypred[i] + d[i];
        if (!f_eval(c, ynew, fy)) break;
        for (int i = 0; i < n; ++i) dy[i] = cc * fy[i] - psi[i] - d[i];
        lu_solve(LU, n, piv, dy);
        const double dn = wrms(dy, ynew, n, rtol, atol);
        const double rate = it > 0 ? dn / dn_prev : 0;
        if (it > 0 && (rate >= 1 || pow(rate, newton_max - it) / (1 - rate) * dn > 1e-3)) break;
        for (int i = 0; i < n; ++i) d[i] += dy[i];
        if (dn == 0 || (it > 0 && rate / (1 - rate) * dn < 1e-3)) { converged = 1; break; }
        dn_prev = dn;
      }
      if (converged) break;
      if (!jac_current) {
        if (!fd_jacobian(c, ypred, J)) return 0;
        jac_current = 1;
        lu_valid = 0;
        continue;
      }
      rescale_D(D, order, 0.5, n);
      h *= 0.5;
      equal_steps = 0;
      lu_valid = 0;
      if (h < 1e-40) return -3;
    }
    for (int i = 0; i < n; ++i) ynew[i] = ypred[i] + d[i];
    double err[MAXN];
    for (int i = 0; i < n; ++i) err[i] = econst[order] * d[i];
    const double en = wrms(err, ynew, n, rtol, atol);
    if (en > 1) {
      const double factor = fmax(0.2, 0.9 * pow(en, -1.0 / (order + 1)));
      rescale_D(D, order, factor, n);
      h *= factor;
      equal_steps = 0;
      lu_valid = 0;
      continue;
    }
    /* accept: update the backward differences */
    t += h;
    equal_steps++;
    jac_current = 0;
    for (int i = 0; i < n; ++i) {
      D[order + 2][i] = d[i] - D[order + 1][i];
      D[order + 1][i] = d[i];
    }
    for (int j = order; j >= 0; --j)
      for (int i = 0; i < n; ++i) D[j][i] += D[j + 1][i];
    if (equal_steps < order + 1) continue;
    /* order and step-size selection from the error estimates of orders k-1, k, k+1 */
    double tmp[MAXN];
    double fm = 0, fpl = 0;
    if (order > 1) {
      for (int i = 0; i < n; ++i) tmp[i] = econst[order - 1] * D[order][i];
      fm = pow(fmax(wrms(tmp, ynew, n, rtol, atol), 1e-300), -1.0 / order);
    }
    if (order < MAXORD) {
      for (int i = 0; i < n; ++i) tmp[i] = econst[order + 1] * D[order + 2][i];
      fpl = pow(fmax(wrms(tmp, ynew, n, rtol, atol), 1e-300), -1.0 / (order + 2));
    }
    double best = pow(fmax(en, 1e-300), -1.0 / (order + 1));
    int delta = 0;
    if (fm > best) { best = fm; delta = -1; }
    if (fpl > best) { best = fpl; delta = 1; }
    order += delta;
    const double factor = fmin(10.0, 0.9 * best);
    rescale_D(D, order, factor, n);
    h *= factor;
    equal_steps = 0;
    lu_valid = 0;
  }
  memcpy(y, D[0], sizeof(double) * n);
  if (nsteps) *nsteps = steps;
  return 1;
}

/* ------------------------------------------------------------ C entry points (ctypes) */

/* h0 (J/kg), cp (J/kg/K), rho of N cells (Y species-major, ldY); status 1 = ok. */
void truth_state(const mech_t* m, long N, const double* T, const double* p, const double* Y,
                 long ldY, double* h, double* cp, double* rho, int* ok) {
#pragma omp parallel for schedule(dynamic, 16)
  for (long i = 0; i < N; ++i) {
    double y[MAXN];
    for (int k = 0; k < m->n; ++k) y[k] = Y[k * ldY + i];
    ok[i] = pr_state(m, T[i], p[i], y, &h[i], &cp[i], &rho[i]);
  }
}

/* dY/dt and T of one composition at fixed (p, h0), starting the T solve from *T. */
int truth_rhs(const mech_t* m, double p, double h0, const double* Y, double* T, double* f) {
  return rhs(m, p, h0, Y, T, f);
}

/* Advances N cells by dt in place (T, Y); status[i] = 1 ok, -1 no root at the start, -1x the
 * integrator failed (x: 0 right-hand side, 1 step limit, 2 singular matrix, 3 step underflow),
 * -3 no temperature at the end; steps[i] = BDF steps. */
void truth_advance(const mech_t* m, long N, double* T, const double* p, double* Y, long ldY,
                   double dt, double rtol, double atol, int* status, long* steps) {
#pragma omp parallel for schedule(dynamic, 1)
  for (long i = 0; i < N; ++i) {
    double y[MAXN];
    for (int k = 0; k < m->n; ++k) y[k] = Y[k * ldY + i];
    double h0, cp, rho;
    status[i] = 0;
    steps[i] = 0;
    if (!pr_state(m, T[i], p[i], y, &h0, &cp, &rho)) { status[i] = -1; continue; }
    ctx_t c = {m, p[i], h0, T[i], 0};
    long ns = 0;
    const int rc = bdf_integrate(&c, y, dt, rtol, atol, &ns);
    steps[i] = ns;
    if (rc != 1) { status[i] = -10 - rc; continue; }
    double Tn = T[i];
    if (!solve_T(m, p[i], y, h0, &Tn, NULL)) { status[i] = -3; continue; }
    T[i] = Tn;
    for (int k = 0; k < m->n; ++k) Y[k * ldY + i] = y[k];
    status[i] = 1;
    steps[i] = ns;
  }
}

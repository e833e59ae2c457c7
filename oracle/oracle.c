/*
 * CPU oracle for the electron-phonon collision integral (TEST INFRASTRUCTURE).
 *
 * Plain, slow, FP64 loops that follow the paper's statement of the problem
 * (arXiv:2511.03683, Eq. 2 and the surrounding text of Sec. "Collision
 * integral, e-ph coupling matrix, and scattering channels").  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load this
 * library; the GPU library never does, and this file shares no code, header or
 * table with it.
 *
 * Units: energies eV, time fs, temperature K; hbar = 0.6582119569 eV fs,
 * k_B = 8.617333262e-5 eV/K.  Rates come out in 1/fs.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *  - F_abs and F_em (named after Eq. 2, not written out) take the Fermi
 *    golden-rule forms
 *        F_abs = f_s (1-f_p) N - (1-f_s) f_p (N+1)
 *        F_em  = f_s (1-f_p)(N+1) - (1-f_s) f_p N
 *    with s = (n,k), p = (m,k+q), N = 1/(exp(hbar w/k_B T) - 1).  With these,
 *    a channel's contributions to I(nk) and I(mk+q) are equal in magnitude and
 *    opposite in sign, as the paper states for its target layer (Sec. "Optimized
 *    GPU algorithm", step 1).
 *  - delta(x) is a normalised Gaussian of width sigma, untruncated.
 *  - The emitted phonon (-q) has the energy of +q; the synthetic dispersions are
 *    even in q.
 *  - 1/N_q counts the full q grid (commensurate with the k grid).
 *  - Modes with hbar w <= 0 (acoustic branches at q = Gamma) are skipped.
 *  - Transport (Eq. 2 "is different in transport calculations"; the Methods
 *    section is absent) uses the linearised iteration
 *        F_s^{i+1} = tau_s (v_s + sum_c W_c F_p^i),
 *        W_c = (2pi/hbar)(1/N_q)|g|^2 [G(x+w)(N+f0_p) + G(x-w)(N+1-f0_p)],
 *        1/tau_s = sum_c W_c,    F^0 = tau v,
 *    stopped when max|F^{i+1}-F^i| <= tol * max|F^{i+1}|.
 *  - Time stepping of the rt-BTE (Eq. 1 with no field) is classic fourth-order
 *    Runge-Kutta.
 *
 * The channel set is enumerated here independently: for every window state
 * s = (n,k), every q of the full grid, every band m with (m,k+q) inside the
 * window and every mode nu.  States are numbered by ascending full-grid id
 * id = ik*nbands + n, ik = (j1*N2 + j2)*N3 + j3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ORACLE_PLANT selects a deliberately wrong variant, used only by the tests that
 * show each pin catches a plausible slip (tests/test_oracle_mutants.py).  The
 * default build defines none. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

#define OR_HBAR 0.6582119569
#define OR_KB 8.617333262e-5
#define OR_PI 3.14159265358979323846

typedef double (*or_g2_fn)(int32_t s_full, int32_t p_full, int32_t nu, const void *user);

typedef struct {
  int32_t nk[3];
  int32_t nbands;
  int32_t nmodes;
  int32_t nthreads;     /* OpenMP threads over rows; <= 0 means the library default */
  const double *eps;    /* [Nk][nbands] band energies, eV */
  const double *omega;  /* [Nq][nmodes] phonon energies hbar*w, eV (Nq = Nk) */
  const double *win;    /* [nbands][2] per-band window [lo, hi] in eV, or NULL for none */
  double T;             /* K */
  double sigma;         /* eV */
  or_g2_fn g2;          /* |g|^2 in eV^2 of the channel (s_full -> p_full, nu) */
  const void *g2_user;
  double g2_min;        /* drop channels with |g|^2 < g2_min (0: keep all) */
  double delta_nsigma;  /* drop channels with min(|x+w|, |x-w|) > delta_nsigma * sigma (0: keep all) */
} or_model;

/* The paper prunes channels by a |g| cutoff and by approximate energy conservation (Sec.
 * "Collision integral, e-ph coupling matrix, and scattering channels"); both are optional
 * here and off by default.  A channel is kept when both tests pass. */
static int keep_channel(const or_model *m, double g2, double x, double w) {
  if (m->g2_min > 0.0 && g2 < m->g2_min) return 0;
  if (m->delta_nsigma > 0.0) {
    const double lim = m->delta_nsigma * m->sigma;
    if (fabs(x + w) > lim && fabs(x - w) > lim) return 0;
  }
  return 1;
}

static int64_t nk_total(const or_model *m) { return (int64_t)m->nk[0] * m->nk[1] * m->nk[2]; }

static int in_window(const or_model *m, int64_t id) {
  if (!m->win) return 1;
  int32_t n = (int32_t)(id % m->nbands);
  double e = m->eps[id];
  return e >= m->win[2 * n] && e <= m->win[2 * n + 1];
}

/* Full-grid ids of the window states, ascending.  Returns the count. */
int64_t oracle_window(const or_model *m, int32_t *ids) {
  int64_t nfull = nk_total(m) * m->nbands, cnt = 0;
  for (int64_t id = 0; id < nfull; ++id)
    if (in_window(m, id)) {
      if (ids) ids[cnt] = (int32_t)id;
      ++cnt;
    }
  return cnt;
}

static int32_t *window_index(const or_model *m) {
  int64_t nfull = nk_total(m) * m->nbands, cnt = 0;
  int32_t *w = (int32_t *)malloc(sizeof(int32_t) * (size_t)nfull);
  if (!w) return NULL;
  for (int64_t id = 0; id < nfull; ++id) w[id] = in_window(m, id) ? (int32_t)cnt++ : -1;
  return w;
}

static inline double gauss(double x, double sigma) {
  return exp(-x * x / (2.0 * sigma * sigma)) / (sqrt(2.0 * OR_PI) * sigma);
}

static inline double bose(double w, double T) { return 1.0 / (exp(w / (OR_KB * T)) - 1.0); }

enum { OR_COLLISION = 0, OR_RATES = 1, OR_TRANSPORT = 2 };

/*
 * One row of the channel sum, Eq. 2, for the window state with full id sid.
 *   OR_COLLISION: returns I_s = -(2pi/hbar)(1/Nq) sum g2 [G(x+w) F_abs + G(x-w) F_em]
 *                 and, if absterm, the row's gross scattering (2pi/hbar)(1/Nq) sum g2
 *                 [G(x+w)(|f_s(1-f_p)N| + |(1-f_s)f_p(N+1)|) + G(x-w)(|f_s(1-f_p)(N+1)| +
 *                 |(1-f_s)f_p N|)], the scale of the rounding error of any evaluation.
 *   OR_RATES:     returns 1/tau_s = (2pi/hbar)(1/Nq) sum g2 [G(x+w)(N+f_p) + G(x-w)(N+1-f_p)]
 *   OR_TRANSPORT: returns sum_c W_c F_p[alpha] for alpha = 0..2 in vec[] (f = f0)
 *                 and the row total sum_c W_c.
 * x = eps_s - eps_p, w = hbar*omega_{nu q}.
 */
static double row_sum(const or_model *m, const int32_t *widx, int64_t sid, const double *f, int mode,
                      const double *F3, double *vec, double *absterm) {
  const int32_t nb = m->nbands, nm = m->nmodes;
  const int32_t N1 = m->nk[0], N2 = m->nk[1], N3 = m->nk[2];
  const int64_t Nq = nk_total(m);
  const double c = 2.0 * OR_PI / (OR_HBAR * (double)Nq);
  const int64_t ik = sid / nb;
  const int32_t n = (int32_t)(sid % nb);
  const int32_t j1 = (int32_t)(ik / ((int64_t)N2 * N3)), j2 = (int32_t)((ik / N3) % N2), j3 = (int32_t)(ik % N3);
  const double eps_s = m->eps[sid];
  const double f_s = f[widx[sid]];
  double acc = 0.0, accabs = 0.0, v0 = 0.0, v1 = 0.0, v2 = 0.0;
  for (int64_t iq = 0; iq < Nq; ++iq) {
    const int32_t q1 = (int32_t)(iq / ((int64_t)N2 * N3)), q2 = (int32_t)((iq / N3) % N2), q3 = (int32_t)(iq % N3);
    const int64_t ikq = ((int64_t)((j1 + q1) % N1) * N2 + (j2 + q2) % N2) * N3 + (j3 + q3) % N3;
    for (int32_t mb = 0; mb < nb; ++mb) {
      const int64_t pid = ikq * nb + mb;
      const int32_t rp = widx[pid];
      if (rp < 0) continue;
      const double eps_p = m->eps[pid];
      const double f_p = f[rp];
      const double x = eps_s - eps_p;
      for (int32_t nu = 0; nu < nm; ++nu) {
#if ORACLE_PLANT == 4
        const double w = m->omega[ikq * nm + nu]; /* planted: phonon taken at k+q, not q */
#else
        const double w = m->omega[iq * nm + nu];
#endif
        if (!(w > 0.0)) continue;
        const double N = bose(w, m->T);
        const double g2 = m->g2((int32_t)sid, (int32_t)pid, nu, m->g2_user);
        if (!keep_channel(m, g2, x, w)) continue;
#if ORACLE_PLANT == 3
        const double Ga = gauss(x - w, m->sigma); /* planted: deltas swapped */
        const double Ge = gauss(x + w, m->sigma);
#else
        const double Ga = gauss(x + w, m->sigma);
        const double Ge = gauss(x - w, m->sigma);
#endif
        if (mode == OR_COLLISION) {
#if ORACLE_PLANT == 1
          const double Fabs = f_s * (1.0 - f_p) * (N + 1.0) - (1.0 - f_s) * f_p * N; /* planted: N <-> N+1 */
#else
          const double Fabs = f_s * (1.0 - f_p) * N - (1.0 - f_s) * f_p * (N + 1.0);
#endif
          const double Fem = f_s * (1.0 - f_p) * (N + 1.0) - (1.0 - f_s) * f_p * N;
#if ORACLE_PLANT == 2
          const double t = g2 * (Ga * Fabs); /* planted: emission term dropped */
#else
          const double t = g2 * (Ga * Fabs + Ge * Fem);
#endif
          acc += t;
          /* gross scattering: the magnitudes of the four products that F_abs and F_em
           * difference, i.e. the error scale of evaluating the summand in floating point */
          accabs += g2 * (Ga * (fabs(f_s * (1.0 - f_p) * N) + fabs((1.0 - f_s) * f_p * (N + 1.0))) +
                          Ge * (fabs(f_s * (1.0 - f_p) * (N + 1.0)) + fabs((1.0 - f_s) * f_p * N)));
        } else {
#if ORACLE_PLANT == 5
          const double Wc = g2 * (Ga * (N + 1.0 - f_p) + Ge * (N + f_p)); /* planted: factors swapped */
#elif ORACLE_PLANT == 6
          const double Wc = g2 * (Ga * (N + f_s) + Ge * (N + 1.0 - f_s)); /* planted: f_s for f_p */
#else
          const double Wc = g2 * (Ga * (N + f_p) + Ge * (N + 1.0 - f_p));
#endif
          acc += Wc;
          if (mode == OR_TRANSPORT) {
            v0 += Wc * F3[3 * rp + 0];
            v1 += Wc * F3[3 * rp + 1];
            v2 += Wc * F3[3 * rp + 2];
          }
        }
      }
    }
  }
  if (absterm) *absterm = c * accabs;
  if (mode == OR_TRANSPORT) {
    vec[0] = c * v0;
    vec[1] = c * v1;
    vec[2] = c * v2;
  }
  return mode == OR_COLLISION ? -c * acc : c * acc;
}

static int set_threads(const or_model *m) {
#ifdef _OPENMP
  if (m->nthreads > 0) return m->nthreads;
  return omp_get_max_threads();
#else
  (void)m;
  return 1;
#endif
}

static int run_rows(const or_model *m, const double *f, const int32_t *rows, int64_t nrows, int mode,
                    double *out, double *absout) {
  int32_t *widx = window_index(m);
  if (!widx) return -1;
  int64_t ns = oracle_window(m, NULL);
  int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
  if (!ids) { free(widx); return -1; }
  oracle_window(m, ids);
  int64_t nr = rows ? nrows : ns;
  int nt = set_threads(m);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t i = 0; i < nr; ++i) {
    int64_t r = rows ? rows[i] : i;
    double a = 0.0;
    out[i] = row_sum(m, widx, ids[r], f, mode, NULL, NULL, absout ? &a : NULL);
    if (absout) absout[i] = a;
  }
  free(ids);
  free(widx);
  return 0;
}

/* Collision integral I_s (1/fs) of the rows listed (window indices), or of all
 * window states when rows == NULL.  f holds the occupations of every window state. */
int oracle_collision(const or_model *m, const double *f, const int32_t *rows, int64_t nrows, double *out,
                     double *abs_out) {
  return run_rows(m, f, rows, nrows, OR_COLLISION, out, abs_out);
}

/* Scattering rates 1/tau_s (1/fs), same row selection as oracle_collision. */
int oracle_rates(const or_model *m, const double *f, const int32_t *rows, int64_t nrows, double *out) {
  return run_rows(m, f, rows, nrows, OR_RATES, out, NULL);
}

/* nsteps classic RK4 steps of df/dt = I[f] with step dt (fs), in place on f. */
int oracle_rk4(const or_model *m, double *f, double dt, int32_t nsteps) {
  int64_t ns = oracle_window(m, NULL);
  size_t bytes = sizeof(double) * (size_t)(ns > 0 ? ns : 1);
  double *k1 = (double *)malloc(bytes), *k2 = (double *)malloc(bytes), *k3 = (double *)malloc(bytes),
         *k4 = (double *)malloc(bytes), *y = (double *)malloc(bytes);
  int rc = 0;
  if (!k1 || !k2 || !k3 || !k4 || !y) rc = -1;
  for (int32_t st = 0; st < nsteps && rc == 0; ++st) {
    rc |= oracle_collision(m, f, NULL, 0, k1, NULL);
    for (int64_t i = 0; i < ns; ++i) y[i] = f[i] + 0.5 * dt * k1[i];
    rc |= oracle_collision(m, y, NULL, 0, k2, NULL);
    for (int64_t i = 0; i < ns; ++i) y[i] = f[i] + 0.5 * dt * k2[i];
    rc |= oracle_collision(m, y, NULL, 0, k3, NULL);
#if ORACLE_PLANT == 8
    for (int64_t i = 0; i < ns; ++i) y[i] = f[i] + 0.5 * dt * k3[i]; /* planted */
#else
    for (int64_t i = 0; i < ns; ++i) y[i] = f[i] + dt * k3[i];
#endif
    rc |= oracle_collision(m, y, NULL, 0, k4, NULL);
#if ORACLE_PLANT == 7
    for (int64_t i = 0; i < ns; ++i) f[i] += dt / 4.0 * (k1[i] + k2[i] + k3[i] + k4[i]); /* planted */
#else
    for (int64_t i = 0; i < ns; ++i) f[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
#endif
  }
  free(k1); free(k2); free(k3); free(k4); free(y);
  return rc;
}

/* One application of the transport map on the listed rows:
 * out3[3*i+a] = tau_s (v_s[a] + sum_c W_c Fin[p][a]), W at f = f0, tau from the same W. */
int oracle_transport_map(const or_model *m, const double *f0, const double *vel3, const double *Fin3,
                         const int32_t *rows, int64_t nrows, double *out3, double *tau_out) {
  int32_t *widx = window_index(m);
  if (!widx) return -1;
  int64_t ns = oracle_window(m, NULL);
  int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
  if (!ids) { free(widx); return -1; }
  oracle_window(m, ids);
  int64_t nr = rows ? nrows : ns;
  int nt = set_threads(m);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t i = 0; i < nr; ++i) {
    int64_t r = rows ? rows[i] : i;
    double vec[3];
    double inv_tau = row_sum(m, widx, ids[r], f0, OR_TRANSPORT, Fin3, vec, NULL);
    double tau = 1.0 / inv_tau;
    for (int a = 0; a < 3; ++a) out3[3 * i + a] = tau * (vel3[3 * r + a] + vec[a]);
    if (tau_out) tau_out[i] = tau;
  }
  free(ids);
  free(widx);
  return 0;
}

/* Iterative transport solve from F^0 = tau v; returns 0 on convergence, 1 if maxit
 * was reached, negative on allocation failure.  F3 is [ns][3]. */
int oracle_transport(const or_model *m, const double *f0, const double *vel3, double tol, int32_t maxit,
                     double *F3, int32_t *iters, double *resid) {
  int64_t ns = oracle_window(m, NULL);
  size_t bytes = sizeof(double) * 3 * (size_t)(ns > 0 ? ns : 1);
  double *tau = (double *)malloc(bytes / 3), *Fn = (double *)malloc(bytes), *zero = (double *)calloc(3 * (size_t)(ns > 0 ? ns : 1), sizeof(double));
  if (!tau || !Fn || !zero) { free(tau); free(Fn); free(zero); return -1; }
  /* F^0 = tau v: one map application with F = 0 */
  int rc = oracle_transport_map(m, f0, vel3, zero, NULL, 0, F3, tau);
  double res = INFINITY;
  int32_t it = 0;
  while (rc == 0 && it < maxit) {
    rc = oracle_transport_map(m, f0, vel3, F3, NULL, 0, Fn, NULL);
    double dmax = 0.0, fmax = 0.0;
    for (int64_t i = 0; i < 3 * ns; ++i) {
      double d = fabs(Fn[i] - F3[i]);
      if (d > dmax) dmax = d;
      if (fabs(Fn[i]) > fmax) fmax = fabs(Fn[i]);
    }
    memcpy(F3, Fn, bytes);
    ++it;
    res = fmax > 0.0 ? dmax / fmax : 0.0;
    if (res <= tol) break;
  }
  if (iters) *iters = it;
  if (resid) *resid = res;
  free(tau); free(Fn); free(zero);
  if (rc) return rc;
  return res <= tol ? 0 : 1;
}

/* Number of channels the definition sums over (window pairs times modes with w > 0). */
int64_t oracle_count_channels(const or_model *m) {
  int32_t *widx = window_index(m);
  if (!widx) return -1;
  int64_t ns = oracle_window(m, NULL);
  int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
  if (!ids) { free(widx); return -1; }
  oracle_window(m, ids);
  const int32_t nb = m->nbands, nm = m->nmodes;
  const int32_t N1 = m->nk[0], N2 = m->nk[1], N3 = m->nk[2];
  const int64_t Nq = nk_total(m);
  int64_t total = 0;
#pragma omp parallel for reduction(+ : total) schedule(dynamic, 4)
  for (int64_t r = 0; r < ns; ++r) {
    int64_t ik = ids[r] / nb;
    int32_t j1 = (int32_t)(ik / ((int64_t)N2 * N3)), j2 = (int32_t)((ik / N3) % N2), j3 = (int32_t)(ik % N3);
    for (int64_t iq = 0; iq < Nq; ++iq) {
      int32_t q1 = (int32_t)(iq / ((int64_t)N2 * N3)), q2 = (int32_t)((iq / N3) % N2), q3 = (int32_t)(iq % N3);
      int64_t ikq = ((int64_t)((j1 + q1) % N1) * N2 + (j2 + q2) % N2) * N3 + (j3 + q3) % N3;
      if (m->g2_min > 0.0 || m->delta_nsigma > 0.0) {
        for (int32_t mb = 0; mb < nb; ++mb) {
          const int64_t pid = ikq * nb + mb;
          if (widx[pid] < 0) continue;
          const double x = m->eps[ids[r]] - m->eps[pid];
          for (int32_t nu = 0; nu < nm; ++nu) {
            const double w = m->omega[iq * nm + nu];
            if (!(w > 0.0)) continue;
            const double g2 = m->g2 ? m->g2(ids[r], (int32_t)pid, nu, m->g2_user) : 0.0;
            total += keep_channel(m, g2, x, w);
          }
        }
        continue;
      }
      int nmw = 0;
      for (int32_t nu = 0; nu < nm; ++nu) nmw += m->omega[iq * nm + nu] > 0.0;
      for (int32_t mb = 0; mb < nb; ++mb)
        if (widx[ikq * nb + mb] >= 0) total += nmw;
    }
  }
  free(ids);
  free(widx);
  return total;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ adjoint (reverse mode)
 *
 * Vector-Jacobian products of the collision integral, by the definition: I_s = -c sum_c t_c
 * with t_c = g2 [G(x+w) F_abs + G(x-w) F_em], so for each channel (s -> p)
 *   dI_s/df_s += -c g2 [G(x+w)((1-f_p)N + f_p(N+1)) + G(x-w)((1-f_p)(N+1) + f_p N)]
 *   dI_s/df_p += -c g2 [G(x+w)(-f_s N - (1-f_s)(N+1)) + G(x-w)(-f_s(N+1) - (1-f_s)N)]
 * (derivatives of the F_abs, F_em readings stated at the top of this file).
 */

/* out[x] = sum_s lam[s] dI_s/df_x for every window state x (serial scatter: plain). */
int oracle_collision_vjp(const or_model *m, const double *f, const double *lam, double *out) {
  int32_t *widx = window_index(m);
  if (!widx) return -1;
  const int64_t ns = oracle_window(m, NULL);
  int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
  if (!ids) { free(widx); return -1; }
  oracle_window(m, ids);
  const int32_t nb = m->nbands, nm = m->nmodes;
  const int32_t N1 = m->nk[0], N2 = m->nk[1], N3 = m->nk[2];
  const int64_t Nq = nk_total(m);
  const double c = 2.0 * OR_PI / (OR_HBAR * (double)Nq);
  for (int64_t i = 0; i < ns; ++i) out[i] = 0.0;
  for (int64_t r = 0; r < ns; ++r) {
    const int64_t sid = ids[r];
    const int64_t ik = sid / nb;
    const int32_t j1 = (int32_t)(ik / ((int64_t)N2 * N3)), j2 = (int32_t)((ik / N3) % N2), j3 = (int32_t)(ik % N3);
    const double eps_s = m->eps[sid], f_s = f[r];
    for (int64_t iq = 0; iq < Nq; ++iq) {
      const int32_t q1 = (int32_t)(iq / ((int64_t)N2 * N3)), q2 = (int32_t)((iq / N3) % N2), q3 = (int32_t)(iq % N3);
      const int64_t ikq = ((int64_t)((j1 + q1) % N1) * N2 + (j2 + q2) % N2) * N3 + (j3 + q3) % N3;
      for (int32_t mb = 0; mb < nb; ++mb) {
        const int64_t pid = ikq * nb + mb;
        const int32_t rp = widx[pid];
        if (rp < 0) continue;
        const double f_p = f[rp];
        const double x = eps_s - m->eps[pid];
        for (int32_t nu = 0; nu < nm; ++nu) {
          const double w = m->omega[iq * nm + nu];
          if (!(w > 0.0)) continue;
          const double N = bose(w, m->T);
          const double g2 = m->g2((int32_t)sid, (int32_t)pid, nu, m->g2_user);
          if (!keep_channel(m, g2, x, w)) continue;
          const double Ga = gauss(x + w, m->sigma), Ge = gauss(x - w, m->sigma);
          const double dts = g2 * (Ga * ((1.0 - f_p) * N + f_p * (N + 1.0)) + Ge * ((1.0 - f_p) * (N + 1.0) + f_p * N));
          const double dtp = g2 * (Ga * (-f_s * N - (1.0 - f_s) * (N + 1.0)) + Ge * (-f_s * (N + 1.0) - (1.0 - f_s) * N));
          out[r] += lam[r] * (-c) * dts;
          out[rp] += lam[r] * (-c) * dtp;
        }
      }
    }
  }
  free(ids);
  free(widx);
  return 0;
}

/* Derivative of L = sum_s lam[s] I_s with respect to the |g|^2 of each listed ORDERED channel
 * (window states s[i] -> p[i], branch nu[i]); only row s depends on it:
 *   dL/dg2 = -c lam_s [G(x+w) F_abs + G(x-w) F_em].  Returns -2 if a channel does not exist. */
int oracle_g2_grad(const or_model *m, const double *f, const double *lam, int64_t n, const int32_t *s,
                   const int32_t *p, const int32_t *nu, double *out) {
  const int64_t ns = oracle_window(m, NULL);
  int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
  if (!ids) return -1;
  oracle_window(m, ids);
  const int32_t nb = m->nbands, nm = m->nmodes;
  const int32_t N2 = m->nk[1], N3 = m->nk[2];
  const int64_t Nq = nk_total(m);
  const double c = 2.0 * OR_PI / (OR_HBAR * (double)Nq);
  int rc = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t sid = ids[s[i]], pid = ids[p[i]];
    const int64_t iks = sid / nb, ikp = pid / nb;
    const int64_t s1 = iks / ((int64_t)N2 * N3), s2 = (iks / N3) % N2, s3 = iks % N3;
    const int64_t p1 = ikp / ((int64_t)N2 * N3), p2 = (ikp / N3) % N2, p3 = ikp % N3;
    const int64_t iq = (((p1 - s1 + m->nk[0]) % m->nk[0]) * N2 + (p2 - s2 + N2) % N2) * N3 + (p3 - s3 + N3) % N3;
    const double w = m->omega[iq * nm + nu[i]];
    if (!(w > 0.0)) { rc = -2; out[i] = 0.0; continue; }
    const double N = bose(w, m->T);
    const double g2 = m->g2((int32_t)sid, (int32_t)pid, nu[i], m->g2_user);
    (void)g2;
    const double x = m->eps[sid] - m->eps[pid];
    const double Ga = gauss(x + w, m->sigma), Ge = gauss(x - w, m->sigma);
    const double f_s = f[s[i]], f_p = f[p[i]];
    const double Fabs = f_s * (1.0 - f_p) * N - (1.0 - f_s) * f_p * (N + 1.0);
    const double Fem = f_s * (1.0 - f_p) * (N + 1.0) - (1.0 - f_s) * f_p * N;
    out[i] = -c * lam[s[i]] * (Ga * Fabs + Ge * Fem);
  }
  free(ids);
  return rc;
}

/* Discrete adjoint of nsteps classic RK4 steps from f0: given lam = dL/df(T) on entry,
 * returns dL/df0 in lam.  Stores every stage input of the forward pass (plain, not
 * checkpointed).  Stage weights follow the forward scheme of oracle_rk4. */
int oracle_rk4_vjp(const or_model *m, const double *f0, double dt, int32_t nsteps, double *lam) {
  const int64_t ns = oracle_window(m, NULL);
  const size_t vb = sizeof(double) * (size_t)(ns > 0 ? ns : 1);
  double *U = (double *)malloc(vb * 4 * (size_t)(nsteps > 0 ? nsteps : 1));
  double *k = (double *)malloc(vb), *y = (double *)malloc(vb), *g = (double *)malloc(vb);
  double *mu = (double *)malloc(vb), *acc = (double *)malloc(vb), *mprev = (double *)malloc(vb);
  int rc = (!U || !k || !y || !g || !mu || !acc || !mprev) ? -1 : 0;
  if (rc == 0) {
    memcpy(y, f0, vb);
    for (int32_t st = 0; st < nsteps && rc == 0; ++st) {
      double *u1 = U + (size_t)(4 * st + 0) * ns, *u2 = U + (size_t)(4 * st + 1) * ns;
      double *u3 = U + (size_t)(4 * st + 2) * ns, *u4 = U + (size_t)(4 * st + 3) * ns;
      memcpy(u1, y, vb);
      rc |= oracle_collision(m, u1, NULL, 0, k, NULL);
      for (int64_t i = 0; i < ns; ++i) { u2[i] = u1[i] + 0.5 * dt * k[i]; acc[i] = k[i]; }
      rc |= oracle_collision(m, u2, NULL, 0, k, NULL);
      for (int64_t i = 0; i < ns; ++i) { u3[i] = u1[i] + 0.5 * dt * k[i]; acc[i] += 2.0 * k[i]; }
      rc |= oracle_collision(m, u3, NULL, 0, k, NULL);
      for (int64_t i = 0; i < ns; ++i) { u4[i] = u1[i] + dt * k[i]; acc[i] += 2.0 * k[i]; }
      rc |= oracle_collision(m, u4, NULL, 0, k, NULL);
      for (int64_t i = 0; i < ns; ++i) y[i] = u1[i] + dt / 6.0 * (acc[i] + k[i]);
    }
    /* y_{n+1} = y_n + dt/6 (k1 + 2k2 + 2k3 + k4), k_i = I(u_i), u2 = y + dt/2 k1,
     * u3 = y + dt/2 k2, u4 = y + dt k3.  Reverse: with lam = dL/dy_{n+1},
     * dL/dk4 = dt/6 lam, dL/dk3 = dt/3 lam + dt J4^T dL/dk4, dL/dk2 = dt/3 lam + dt/2 J3^T dL/dk3,
     * dL/dk1 = dt/6 lam + dt/2 J2^T dL/dk2, dL/dy_n = lam + sum_i J_i^T dL/dk_i. */
    for (int32_t st = nsteps - 1; st >= 0 && rc == 0; --st) {
      const double wl[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
      const double wm[4] = {0.5 * dt, 0.5 * dt, dt, 0.0}; /* u_{i+1} = y + wm[i] k_i */
      for (int64_t i = 0; i < ns; ++i) { acc[i] = lam[i]; mprev[i] = 0.0; }
      for (int j = 3; j >= 0 && rc == 0; --j) {
        const double *u = U + (size_t)(4 * st + j) * ns;
        for (int64_t i = 0; i < ns; ++i) g[i] = wl[j] * lam[i] + wm[j] * mprev[i];
        rc |= oracle_collision_vjp(m, u, g, mu);
        for (int64_t i = 0; i < ns; ++i) { acc[i] += mu[i]; mprev[i] = mu[i]; }
      }
      memcpy(lam, acc, vb);
    }
  }
  free(U); free(k); free(y); free(g); free(mu); free(acc); free(mprev);
  return rc;
}

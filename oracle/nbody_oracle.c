/*
 * FP64 CPU oracle for direct-summation N-body force + jerk, the 4th-order
 * Hermite predictor-corrector with power-of-two block time steps, the
 * softened energy, and the KDK leapfrog with its exact adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header or constant
 * with the CUDA library.
 *
 * Every routine is the plain definition or the plain algorithm: loops over
 * i and j in ascending order, double precision, no blocking, no fusion.
 * OpenMP parallelises only over independent i; each i's j-loop keeps the
 * fixed ascending order, so results do not depend on the thread count.
 * Built with -ffp-contract=off so that no multiply-add is fused and the
 * arithmetic is the written expression on every host.
 *
 * Sources:
 *   force law            paper eq. (1), Sec. 2 (G sum_{j!=i} m_j (r_j-r_i)/r_ij^3)
 *   softening            paper Sec. 3 (Plummer softening eps in the pair
 *                        potential; r^2 -> r^2 + eps^2)
 *   jerk                 time derivative of eq. (1) with softening
 *                        (Makino 1991; not printed in the paper)
 *   Hermite-4 corrector  Makino & Aarseth (1992); not in the paper
 *   time-step criterion  Aarseth (1985), cited in the paper's Sec. 2
 *   block steps          paper Sec. 2, strategy (ii), "individual (per
 *                        particle) time steps"; power-of-two quantisation is
 *                        the standard block scheme (reading, see DESIGN)
 *   leapfrog             paper Sec. 3.1 (the classic second-order scheme),
 *                        kick-drift-kick form (reading)
 *   external field       paper Sec. 2.1: the Galactic potential of Allen &
 *                        Santillan (1991), a Plummer bulge, a Miyamoto-Nagai
 *                        disk and a spherical halo (forms and parameters
 *                        from that paper; not printed in this one)
 *
 * Parity status: every function below is pinned by -m "not gpu" tests
 * (brute force in 50-digit arithmetic, conservation laws, closed forms,
 * finite differences, Kepler's equation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TICKS_LOG2 20 /* time is kept in integer ticks of 2^-20 */

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int nt) {
#ifdef _OPENMP
  if (nt > 0) omp_set_num_threads(nt);
#else
  (void)nt;
#endif
}

/* ------------------------------------------------------------------------
 * Acceleration and jerk of particle i from all j != i (definition).
 *   d = x_j - x_i, w = v_j - v_i, s2 = d.d + eps^2
 *   a_i += G m_j d / s^3
 *   jerk_i += G m_j ( w / s^3 - 3 (d.w) d / s^5 )
 * x, v, acc, jerk are (n,3) row-major.  idx selects the i-particles
 * (n_i of them); idx == NULL means i = 0..n_i-1.
 * ---------------------------------------------------------------------- */
static void force_jerk_one(int64_t n, const double *m, const double *x,
                           const double *v, double G, double eps, int64_t i,
                           double *acc_i, double *jerk_i, int want_jerk) {
  double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0;
  const double e2 = eps * eps;
  for (int64_t j = 0; j < n; ++j) {
    if (j == i) continue;
    double dx = x[3 * j + 0] - x[3 * i + 0];
    double dy = x[3 * j + 1] - x[3 * i + 1];
    double dz = x[3 * j + 2] - x[3 * i + 2];
    double s2 = dx * dx + dy * dy + dz * dz + e2;
    double sinv = 1.0 / sqrt(s2);
    double sinv3 = sinv / s2;
    double f = m[j] * sinv3;
    ax += f * dx;
    ay += f * dy;
    az += f * dz;
    if (want_jerk) {
      double wx = v[3 * j + 0] - v[3 * i + 0];
      double wy = v[3 * j + 1] - v[3 * i + 1];
      double wz = v[3 * j + 2] - v[3 * i + 2];
      double dw = dx * wx + dy * wy + dz * wz;
      double c = 3.0 * dw / s2;
      jx += f * (wx - c * dx);
      jy += f * (wy - c * dy);
      jz += f * (wz - c * dz);
    }
  }
  acc_i[0] = G * ax;
  acc_i[1] = G * ay;
  acc_i[2] = G * az;
  if (want_jerk) {
    jerk_i[0] = G * jx;
    jerk_i[1] = G * jy;
    jerk_i[2] = G * jz;
  }
}

void orc_force_jerk(int64_t n, const double *m, const double *x,
                    const double *v, double G, double eps, int64_t n_i,
                    const int64_t *idx, double *acc, double *jerk) {
  int want_jerk = (jerk != NULL && v != NULL);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < n_i; ++k) {
    int64_t i = idx ? idx[k] : k;
    double a3[3], j3[3];
    force_jerk_one(n, m, x, v, G, eps, i, a3, j3, want_jerk);
    acc[3 * k + 0] = a3[0];
    acc[3 * k + 1] = a3[1];
    acc[3 * k + 2] = a3[2];
    if (want_jerk) {
      jerk[3 * k + 0] = j3[0];
      jerk[3 * k + 1] = j3[1];
      jerk[3 * k + 2] = j3[2];
    }
  }
}

/* Condition of the force and jerk sums of particle i: the sums of the
 * magnitudes of the individual pair terms, sum_j |G m_j d / s^3| and
 * sum_j |G m_j (w / s^3 - 3 (d.w) d / s^5)|.  An error bound of a
 * floating-point sum scales with these, not with the magnitude of the sum. */
void orc_force_jerk_abs(int64_t n, const double *m, const double *x,
                        const double *v, double G, double eps, int64_t n_i,
                        const int64_t *idx, double *aabs, double *jabs) {
  const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < n_i; ++k) {
    int64_t i = idx ? idx[k] : k;
    double sa = 0.0, sj = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double dx = x[3 * j + 0] - x[3 * i + 0];
      double dy = x[3 * j + 1] - x[3 * i + 1];
      double dz = x[3 * j + 2] - x[3 * i + 2];
      double wx = v[3 * j + 0] - v[3 * i + 0];
      double wy = v[3 * j + 1] - v[3 * i + 1];
      double wz = v[3 * j + 2] - v[3 * i + 2];
      double s2 = dx * dx + dy * dy + dz * dz + e2;
      double f = m[j] / (s2 * sqrt(s2));
      double c = 3.0 * (dx * wx + dy * wy + dz * wz) / s2;
      double tx = wx - c * dx, ty = wy - c * dy, tz = wz - c * dz;
      sa += f * sqrt(dx * dx + dy * dy + dz * dz);
      sj += f * sqrt(tx * tx + ty * ty + tz * tz);
    }
    aabs[k] = G * sa;
    jabs[k] = G * sj;
  }
}

/* ------------------------------------------------------------------------
 * Energy: K = 1/2 sum m v^2, W = -G sum_{i<j} m_i m_j / sqrt(r^2 + eps^2).
 * Per-i partial sums are added in ascending i order (thread-independent).
 * ---------------------------------------------------------------------- */
void orc_energy(int64_t n, const double *m, const double *x, const double *v,
                double G, double eps, double *kin, double *pot) {
  double *wpart = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    double w = 0.0;
    for (int64_t j = i + 1; j < n; ++j) {
      double dx = x[3 * j + 0] - x[3 * i + 0];
      double dy = x[3 * j + 1] - x[3 * i + 1];
      double dz = x[3 * j + 2] - x[3 * i + 2];
      w += m[j] / sqrt(dx * dx + dy * dy + dz * dz + e2);
    }
    wpart[i] = m[i] * w;
  }
  double k = 0.0, w = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double vv = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                v[3 * i + 2] * v[3 * i + 2];
    k += 0.5 * m[i] * vv;
    w += wpart[i];
  }
  free(wpart);
  *kin = k;
  *pot = -G * w;
}

/* ------------------------------------------------------------------------
 * Hermite-4 pieces (Makino & Aarseth 1992).
 * Predictor: x_p = x + v dt + a dt^2/2 + j dt^3/6, v_p = v + a dt + j dt^2/2.
 * ---------------------------------------------------------------------- */
static void predict_one(const double *x, const double *v, const double *a,
                        const double *jk, double dt, double *xp, double *vp) {
  double dt2 = dt * dt, dt3 = dt2 * dt;
  for (int c = 0; c < 3; ++c) {
    xp[c] = x[c] + v[c] * dt + a[c] * dt2 / 2.0 + jk[c] * dt3 / 6.0;
    vp[c] = v[c] + a[c] * dt + jk[c] * dt2 / 2.0;
  }
}

void orc_predict(int64_t n, const double *x, const double *v, const double *a,
                 const double *jk, const double *dt, double *xp, double *vp) {
  for (int64_t i = 0; i < n; ++i)
    predict_one(x + 3 * i, v + 3 * i, a + 3 * i, jk + 3 * i, dt[i],
                xp + 3 * i, vp + 3 * i);
}

/* Corrector for one particle over a step dt, from (a0, j0) at the start and
 * (a1, j1) evaluated at the predicted state.  a2 and a3 are the second and
 * third time derivatives of the acceleration at the start of the step,
 * obtained from the two-point Hermite interpolation:
 *   a2 = (-6 (a0 - a1) - dt (4 j0 + 2 j1)) / dt^2
 *   a3 = (12 (a0 - a1) + 6 dt (j0 + j1)) / dt^3
 *   x1 = x_p + a2 dt^4/24 + a3 dt^5/120,  v1 = v_p + a2 dt^3/6 + a3 dt^4/24
 * Also returns a2 and a3 at the END of the step (a2 + a3 dt, a3) for the
 * time-step criterion. */
static void correct_one(double dt, const double *xp, const double *vp,
                        const double *a0, const double *j0, const double *a1,
                        const double *j1, double *x1, double *v1,
                        double *a2_end, double *a3_end) {
  double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
  for (int c = 0; c < 3; ++c) {
    double a2 = (-6.0 * (a0[c] - a1[c]) - dt * (4.0 * j0[c] + 2.0 * j1[c])) / dt2;
    double a3 = (12.0 * (a0[c] - a1[c]) + 6.0 * dt * (j0[c] + j1[c])) / dt3;
    x1[c] = xp[c] + a2 * dt4 / 24.0 + a3 * dt5 / 120.0;
    v1[c] = vp[c] + a2 * dt3 / 6.0 + a3 * dt4 / 24.0;
    if (a2_end) a2_end[c] = a2 + a3 * dt;
    if (a3_end) a3_end[c] = a3;
  }
}

static double norm3(const double *u) {
  return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

/* Aarseth (1985) criterion:
 *   dt = sqrt( eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2) ) */
double orc_aarseth_dt(const double *a, const double *jk, const double *a2,
                      const double *a3, double eta) {
  double na = norm3(a), nj = norm3(jk), n2 = norm3(a2), n3 = norm3(a3);
  return sqrt(eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2));
}

/* Largest power of two 2^-lev not above dt: dt = f 2^e with f in [0.5, 1)
 * gives 2^(e-1) <= dt, so lev = 1 - e.  Clamped to [lev_min, lev_max];
 * *clamped is set when the criterion asked for less than 2^-lev_max. */
int orc_level_from_dt(double dt, int lev_min, int lev_max, int *clamped) {
  int e;
  int lev;
  if (!(dt > 0.0) || isinf(dt)) {
    lev = isinf(dt) ? lev_min : lev_max;
    if (clamped && !isinf(dt)) *clamped = 1;
    return lev;
  }
  frexp(dt, &e);
  lev = 1 - e;
  if (lev > lev_max) {
    if (clamped) *clamped = 1;
    lev = lev_max;
  }
  if (lev < lev_min) lev = lev_min;
  return lev;
}

/* New level after a step that ended at tick t_new: shrink to any level the
 * criterion asks for; grow by one level only, and only when t_new is a
 * multiple of the doubled step. */
int orc_next_level(int lev_old, int lev_want, int64_t t_new, int lev_min) {
  if (lev_want >= lev_old) return lev_want;
  int lev_up = lev_old - 1;
  if (lev_up < lev_min) return lev_old;
  int64_t period = (int64_t)1 << (ORC_TICKS_LOG2 - lev_up);
  if (t_new % period == 0) return lev_up;
  return lev_old;
}

static void ext_one(const double *p, const double *xi, const double *vi, double *acc,
                    double *jerk, double *phi);

/* Initial acceleration, jerk and level for every particle at t = 0:
 * dt0 = eta_start |a| / |j|.  ext (13 doubles, see ext_one) or NULL: the
 * external field's acceleration and jerk are added to the pair sums. */
void orc_hermite_init_ext(int64_t n, const double *m, const double *x,
                          const double *v, double G, double eps, double eta_start,
                          int lev_min, int lev_max, const double *ext, double *a,
                          double *jk, int32_t *lev, int64_t *t_tick) {
  orc_force_jerk(n, m, x, v, G, eps, n, NULL, a, jk);
  if (ext) {
    for (int64_t i = 0; i < n; ++i) {
      double ea[3], ej[3];
      ext_one(ext, x + 3 * i, v + 3 * i, ea, ej, NULL);
      for (int c = 0; c < 3; ++c) {
        a[3 * i + c] += ea[c];
        jk[3 * i + c] += ej[c];
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    double dt0 = eta_start * norm3(a + 3 * i) / norm3(jk + 3 * i);
    int cl = 0;
    lev[i] = orc_level_from_dt(dt0, lev_min, lev_max, &cl);
    t_tick[i] = 0;
  }
}

void orc_hermite_init(int64_t n, const double *m, const double *x,
                      const double *v, double G, double eps, double eta_start,
                      int lev_min, int lev_max, double *a, double *jk,
                      int32_t *lev, int64_t *t_tick) {
  orc_hermite_init_ext(n, m, x, v, G, eps, eta_start, lev_min, lev_max, NULL, a, jk, lev,
                       t_tick);
}

/* One block step.
 * Schedule: t_next = min_i (t_i + 2^(20 - lev_i)) ticks; active set = all i
 * whose t_i + dt_i equals it, ascending index order.  In replay mode
 * (replay_n_act >= 0) the schedule (replay_t_next, replay_act) is taken as
 * given instead, so that a trajectory can be followed on another
 * implementation's block schedule.
 * Then: predict every particle to t_next (each with its own t_next - t_j),
 * evaluate force + jerk on the active set at the predicted state, correct
 * the active set, and, if block_levels is non-zero, choose new levels with
 * the Aarseth criterion; otherwise keep the levels (shared fixed dt).
 * Returns n_act; writes t_next and the active list; adds to *n_clamped the
 * number of particles whose criterion fell below 2^-lev_max.  ext (13
 * doubles, see ext_one) or NULL: the external field's acceleration and jerk
 * at the predicted position and velocity are added to the pair sums. */
int64_t orc_block_step_ext(int64_t n, const double *m, double *x, double *v,
                           double *a, double *jk, int64_t *t_tick, int32_t *lev,
                           double G, double eps, double eta, int lev_min,
                           int lev_max, int block_levels, int64_t replay_t_next,
                           int64_t replay_n_act, const int64_t *replay_act,
                           const double *ext, int64_t *t_next_out, int64_t *act_out,
                           int64_t *n_clamped) {
  const double tick = ldexp(1.0, -ORC_TICKS_LOG2);
  int64_t t_next, n_act = 0;
  if (replay_n_act >= 0) {
    t_next = replay_t_next;
    n_act = replay_n_act;
    for (int64_t k = 0; k < n_act; ++k) act_out[k] = replay_act[k];
  } else {
    t_next = INT64_MAX;
    for (int64_t i = 0; i < n; ++i) {
      int64_t te = t_tick[i] + ((int64_t)1 << (ORC_TICKS_LOG2 - lev[i]));
      if (te < t_next) t_next = te;
    }
    for (int64_t i = 0; i < n; ++i) {
      int64_t te = t_tick[i] + ((int64_t)1 << (ORC_TICKS_LOG2 - lev[i]));
      if (te == t_next) act_out[n_act++] = i;
    }
  }
  *t_next_out = t_next;

  double *xp = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  double *vp = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    double dt = (double)(t_next - t_tick[i]) * tick;
    predict_one(x + 3 * i, v + 3 * i, a + 3 * i, jk + 3 * i, dt, xp + 3 * i,
                vp + 3 * i);
  }
  double *a1 = (double *)malloc(sizeof(double) * 3 * (size_t)(n_act > 0 ? n_act : 1));
  double *j1 = (double *)malloc(sizeof(double) * 3 * (size_t)(n_act > 0 ? n_act : 1));
  orc_force_jerk(n, m, xp, vp, G, eps, n_act, act_out, a1, j1);
  if (ext) {
    for (int64_t k = 0; k < n_act; ++k) {
      const int64_t i = act_out[k];
      double ea[3], ej[3];
      ext_one(ext, xp + 3 * i, vp + 3 * i, ea, ej, NULL);
      for (int c = 0; c < 3; ++c) {
        a1[3 * k + c] += ea[c];
        j1[3 * k + c] += ej[c];
      }
    }
  }

  int64_t clamped_here = 0;
  for (int64_t k = 0; k < n_act; ++k) {
    int64_t i = act_out[k];
    double dt = (double)(t_next - t_tick[i]) * tick;
    double x1[3], v1[3], a2e[3], a3e[3];
    correct_one(dt, xp + 3 * i, vp + 3 * i, a + 3 * i, jk + 3 * i, a1 + 3 * k,
                j1 + 3 * k, x1, v1, a2e, a3e);
    for (int c = 0; c < 3; ++c) {
      x[3 * i + c] = x1[c];
      v[3 * i + c] = v1[c];
      a[3 * i + c] = a1[3 * k + c];
      jk[3 * i + c] = j1[3 * k + c];
    }
    t_tick[i] = t_next;
    if (block_levels) {
      double dtc = orc_aarseth_dt(a1 + 3 * k, j1 + 3 * k, a2e, a3e, eta);
      int cl = 0;
      int want = orc_level_from_dt(dtc, lev_min, lev_max, &cl);
      clamped_here += cl;
      lev[i] = orc_next_level(lev[i], want, t_next, lev_min);
    }
  }
  if (n_clamped) *n_clamped += clamped_here;
  free(xp);
  free(vp);
  free(a1);
  free(j1);
  return n_act;
}

int64_t orc_block_step(int64_t n, const double *m, double *x, double *v,
                       double *a, double *jk, int64_t *t_tick, int32_t *lev,
                       double G, double eps, double eta, int lev_min,
                       int lev_max, int block_levels, int64_t replay_t_next,
                       int64_t replay_n_act, const int64_t *replay_act,
                       int64_t *t_next_out, int64_t *act_out,
                       int64_t *n_clamped) {
  return orc_block_step_ext(n, m, x, v, a, jk, t_tick, lev, G, eps, eta, lev_min, lev_max,
                            block_levels, replay_t_next, replay_n_act, replay_act, NULL,
                            t_next_out, act_out, n_clamped);
}

/* Shared fixed step dt = 2^-lev for nsteps steps (every particle active). */
void orc_hermite_shared(int64_t n, const double *m, double *x, double *v,
                        double *a, double *jk, double G, double eps, int lev,
                        int64_t nsteps) {
  int64_t *t_tick = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int32_t *levs = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t *act = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) levs[i] = lev;
  int64_t tn = 0;
  for (int64_t s = 0; s < nsteps; ++s)
    orc_block_step(n, m, x, v, a, jk, t_tick, levs, G, eps, 0.0, lev, lev, 0,
                   0, -1, NULL, &tn, act, NULL);
  free(t_tick);
  free(levs);
  free(act);
}

/* ------------------------------------------------------------------------
 * Leapfrog (paper Sec. 3.1), kick-drift-kick, fixed dt, acceleration only:
 *   v += a(x) dt/2 ; x += v dt ; v += a(x) dt/2
 * ---------------------------------------------------------------------- */
void orc_acc(int64_t n, const double *m, const double *x, double G, double eps,
             double *acc) {
  orc_force_jerk(n, m, x, NULL, G, eps, n, NULL, acc, NULL);
}

void orc_leapfrog(int64_t n, const double *m, double *x, double *v, double G,
                  double eps, double dt, int64_t nsteps) {
  double *acc = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  orc_acc(n, m, x, G, eps, acc);
  for (int64_t s = 0; s < nsteps; ++s) {
    for (int64_t q = 0; q < 3 * n; ++q) v[q] += acc[q] * dt / 2.0;
    for (int64_t q = 0; q < 3 * n; ++q) x[q] += v[q] * dt;
    orc_acc(n, m, x, G, eps, acc);
    for (int64_t q = 0; q < 3 * n; ++q) v[q] += acc[q] * dt / 2.0;
  }
  free(acc);
}

/* Vector-Jacobian product of the acceleration map a = A(x, m).
 * Given g_i = dL/da_i, with d = x_j - x_k, s^2 = |d|^2 + eps^2 and the
 * softened tidal tensor T(d) = I/s^3 - 3 d d^T / s^5 (symmetric, even in d):
 *   dL/dx_k = G sum_{j != k} T(x_j - x_k) (m_k g_j - m_j g_k)
 *   dL/dm_k = G sum_{i != k} g_i . (x_k - x_i) / s_ik^3
 * gx is (n,3), gm is (n,). */
void orc_acc_vjp(int64_t n, const double *m, const double *x, double G,
                 double eps, const double *g, double *gx, double *gm) {
  const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < n; ++k) {
    double ox = 0, oy = 0, oz = 0, om = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == k) continue;
      double dx = x[3 * j + 0] - x[3 * k + 0];
      double dy = x[3 * j + 1] - x[3 * k + 1];
      double dz = x[3 * j + 2] - x[3 * k + 2];
      double s2 = dx * dx + dy * dy + dz * dz + e2;
      double sinv = 1.0 / sqrt(s2);
      double s3 = sinv / s2;
      double s5 = s3 / s2;
      double ux = m[k] * g[3 * j + 0] - m[j] * g[3 * k + 0];
      double uy = m[k] * g[3 * j + 1] - m[j] * g[3 * k + 1];
      double uz = m[k] * g[3 * j + 2] - m[j] * g[3 * k + 2];
      double du = dx * ux + dy * uy + dz * uz;
      ox += ux * s3 - 3.0 * du * s5 * dx;
      oy += uy * s3 - 3.0 * du * s5 * dy;
      oz += uz * s3 - 3.0 * du * s5 * dz;
      /* (x_k - x_i) = -d with i = j */
      om += -(g[3 * j + 0] * dx + g[3 * j + 1] * dy + g[3 * j + 2] * dz) * s3;
    }
    gx[3 * k + 0] = G * ox;
    gx[3 * k + 1] = G * oy;
    gx[3 * k + 2] = G * oz;
    gm[k] = G * om;
  }
}

/* Reverse sweep of nsteps KDK steps along a given path of positions
 * xs[s] (s = 0..nsteps, each (n,3)).  On entry lx, lv hold dL/dx(T) and
 * dL/dv(T); on exit dL/dx(0), dL/dv(0); lm receives dL/dm.
 * Reverse of one step (x, v) -> (x', v'):
 *   v_h = v + A(x) dt/2, x' = x + v_h dt, v' = v_h + A(x') dt/2
 * adjoint:  lv_h = lv' ;  (lx', lm) += vjp_A(x'; lv' dt/2)
 *           lx = lx' ; lv_h += lx' dt
 *           lv = lv_h ; (lx, lm) += vjp_A(x; lv_h dt/2) */
void orc_leapfrog_adjoint_path(int64_t n, const double *m, const double *xs,
                               double G, double eps, double dt, int64_t nsteps,
                               double *lx, double *lv, double *lm) {
  size_t n3 = 3 * (size_t)n;
  double *g = (double *)malloc(sizeof(double) * n3);
  double *tx = (double *)malloc(sizeof(double) * n3);
  double *tm = (double *)malloc(sizeof(double) * (size_t)n);
  for (int64_t k = 0; k < n; ++k) lm[k] = 0.0;
  for (int64_t s = nsteps - 1; s >= 0; --s) {
    const double *xa = xs + n3 * (size_t)s;       /* x at step start */
    const double *xb = xs + n3 * (size_t)(s + 1); /* x' */
    /* second kick */
    for (size_t q = 0; q < n3; ++q) g[q] = lv[q] * dt / 2.0;
    orc_acc_vjp(n, m, xb, G, eps, g, tx, tm);
    for (size_t q = 0; q < n3; ++q) lx[q] += tx[q];
    for (int64_t k = 0; k < n; ++k) lm[k] += tm[k];
    /* drift */
    for (size_t q = 0; q < n3; ++q) lv[q] += lx[q] * dt;
    /* first kick */
    for (size_t q = 0; q < n3; ++q) g[q] = lv[q] * dt / 2.0;
    orc_acc_vjp(n, m, xa, G, eps, g, tx, tm);
    for (size_t q = 0; q < n3; ++q) lx[q] += tx[q];
    for (int64_t k = 0; k < n; ++k) lm[k] += tm[k];
  }
  free(g); free(tx); free(tm);
}

/* Loss L = sum_i |x_i(T) - y_i|^2 after nsteps KDK steps from (x0, v0) and
 * its exact gradient with respect to x0, v0 and m: the forward pass keeps
 * every position (no checkpointing here), then the reverse sweep above
 * starts from dL/dx(T) = 2 (x(T) - y), dL/dv(T) = 0.  Returns L. */
double orc_leapfrog_loss_grad(int64_t n, const double *m, const double *x0,
                              const double *v0, const double *y, double G,
                              double eps, double dt, int64_t nsteps,
                              double *gx0, double *gv0, double *gmass) {
  size_t n3 = 3 * (size_t)n;
  double *xs = (double *)malloc(sizeof(double) * n3 * (size_t)(nsteps + 1));
  double *x = (double *)malloc(sizeof(double) * n3);
  double *v = (double *)malloc(sizeof(double) * n3);
  double *acc = (double *)malloc(sizeof(double) * n3);
  memcpy(x, x0, sizeof(double) * n3);
  memcpy(v, v0, sizeof(double) * n3);
  memcpy(xs, x, sizeof(double) * n3);
  orc_acc(n, m, x, G, eps, acc);
  for (int64_t s = 0; s < nsteps; ++s) {
    for (size_t q = 0; q < n3; ++q) v[q] += acc[q] * dt / 2.0;
    for (size_t q = 0; q < n3; ++q) x[q] += v[q] * dt;
    orc_acc(n, m, x, G, eps, acc);
    for (size_t q = 0; q < n3; ++q) v[q] += acc[q] * dt / 2.0;
    memcpy(xs + n3 * (size_t)(s + 1), x, sizeof(double) * n3);
  }
  double L = 0.0;
  for (size_t q = 0; q < n3; ++q) {
    double d = x[q] - y[q];
    L += d * d;
    gx0[q] = 2.0 * d;
    gv0[q] = 0.0;
  }
  orc_leapfrog_adjoint_path(n, m, xs, G, eps, dt, nsteps, gx0, gv0, gmass);
  free(xs); free(x); free(v); free(acc);
  return L;
}

/* External Galactic field (Allen & Santillan 1991).  p holds 13 doubles:
 *   G, centre (cx, cy, cz), bulge (M_b, b_b), disk (M_d, a_d, b_d),
 *   halo (M_h, a_h, gamma, r_cut).
 * With d = x - centre, r = |d|, R^2 = d_x^2 + d_y^2, z = d_z:
 *   bulge  Phi_b = -G M_b / sqrt(r^2 + b_b^2)
 *   disk   Phi_d = -G M_d / sqrt(R^2 + (a_d + sqrt(z^2 + b_d^2))^2)
 *   halo   mass inside r: M(r) = M_h (r/a_h)^gamma / (1 + (r/a_h)^(gamma-1)),
 *          M(r_cut) beyond r_cut; force -G M(r) / r^2 along d / r;
 *          Phi_h(r) = -G M(r)/r - G M_h / ((gamma-1) a_h) [F(q_cut) - F(q)]
 *          for r < r_cut with q = r / a_h and
 *          F(q) = -(gamma-1) / (1 + q^(gamma-1)) + ln(1 + q^(gamma-1)),
 *          and -G M(r_cut) / r beyond (so that dPhi_h/dr = G M(r) / r^2).
 * The jerk is the time derivative of the acceleration along the velocity
 * vi, d a(x + vi t)/dt at t = 0, written out per component below.
 * acc (3), jerk (3, needs vi) and phi (1) may be NULL. */
static void ext_one(const double *p, const double *xi, const double *vi, double *acc,
                    double *jerk, double *phi) {
  const double G = p[0];
  const double dx = xi[0] - p[1], dy = xi[1] - p[2], dz = xi[2] - p[3];
  const double mb = p[4], bb = p[5], md = p[6], ad = p[7], bd = p[8];
  const double mh = p[9], ah = p[10], gam = p[11], rcut = p[12];
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double r = sqrt(r2);
  const double vx = vi ? vi[0] : 0.0, vy = vi ? vi[1] : 0.0, vz = vi ? vi[2] : 0.0;
  double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
  double jx = 0.0, jy = 0.0, jz = 0.0;
  /* bulge: -grad of -G M_b (r^2 + b^2)^(-1/2) */
  {
    const double s2 = r2 + bb * bb;
    const double s = sqrt(s2);
    const double f = G * mb / (s2 * s);
    ax -= f * dx;
    ay -= f * dy;
    az -= f * dz;
    ph -= G * mb / s;
    /* d/dt of -G M d / s^3: -G M (v / s^3 - 3 (d.v) d / s^5) */
    const double c = 3.0 * (dx * vx + dy * vy + dz * vz) / s2;
    jx -= f * (vx - c * dx);
    jy -= f * (vy - c * dy);
    jz -= f * (vz - c * dz);
  }
  /* disk */
  {
    const double zeta = sqrt(dz * dz + bd * bd);
    const double w = ad + zeta;
    const double D2 = dx * dx + dy * dy + w * w;
    const double D = sqrt(D2);
    const double f = G * md / (D2 * D);
    ax -= f * dx;
    ay -= f * dy;
    az -= f * dz * w / zeta;
    ph -= G * md / D;
    /* with g = d_z w / zeta: dD/dt = (d_x v_x + d_y v_y + w d_z v_z / zeta) / D,
     * dg/dt = v_z (1 + a_d b_d^2 / zeta^3); a = -G M_d (d_x, d_y, g) / D^3 */
    const double Ddot = (dx * vx + dy * vy + w * dz * vz / zeta) / D;
    const double g = dz * w / zeta;
    const double gdot = vz * (1.0 + ad * bd * bd / (zeta * zeta * zeta));
    const double c = 3.0 * Ddot / D;
    jx -= f * (vx - c * dx);
    jy -= f * (vy - c * dy);
    jz -= f * (gdot - c * g);
  }
  /* halo */
  {
    const double rr = r < rcut ? r : rcut;
    const double q = rr / ah;
    const double u = pow(q, gam - 1.0);
    const double Mr = mh * q * u / (1.0 + u);
    if (r > 0.0) {
      const double f = G * Mr / (r2 * r);
      ax -= f * dx;
      ay -= f * dy;
      az -= f * dz;
      /* d/dt of -G M(r) d / r^3 with dr/dt = d.v / r:
       * -G [M v / r^3 + (M'(r) - 3 M / r) (d.v) d / r^4];
       * M'(r) = M_h q^(gamma-1) (gamma + u) / ((1 + u)^2 a_h) inside the cut */
      const double Mp = r < rcut ? mh * u * (gam + u) / ((1.0 + u) * (1.0 + u) * ah) : 0.0;
      const double c = (Mp - 3.0 * Mr / r) * (dx * vx + dy * vy + dz * vz) / (r2 * r2);
      jx -= f * vx + G * c * dx;
      jy -= f * vy + G * c * dy;
      jz -= f * vz + G * c * dz;
    }
    if (r < rcut) {
      const double qc = rcut / ah;
      const double uc = pow(qc, gam - 1.0);
      const double Fc = -(gam - 1.0) / (1.0 + uc) + log(1.0 + uc);
      const double Fq = -(gam - 1.0) / (1.0 + u) + log(1.0 + u);
      ph += (r > 0.0 ? -G * Mr / r : 0.0) - G * mh / ((gam - 1.0) * ah) * (Fc - Fq);
    } else {
      ph -= G * Mr / r;
    }
  }
  if (acc) {
    acc[0] = ax;
    acc[1] = ay;
    acc[2] = az;
  }
  if (jerk) {
    jerk[0] = jx;
    jerk[1] = jy;
    jerk[2] = jz;
  }
  if (phi) *phi = ph;
}

/* Acceleration (n,3), potential (n) and, with v, jerk (n,3) of the external
 * field at x; any output may be NULL. */
void orc_ext(int64_t n, const double *x, const double *v, const double *p, double *acc,
             double *jerk, double *phi) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    ext_one(p, x + 3 * i, v ? v + 3 * i : NULL, acc ? acc + 3 * i : NULL,
            (jerk && v) ? jerk + 3 * i : NULL, phi ? phi + i : NULL);
}

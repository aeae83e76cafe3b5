/*
 * sde_oracle.c -- plain, slow FP64 CPU oracle for ensemble SDE integration.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library; both sides implement the counter-based
 * generator independently from its published definition.
 *
 * Paper: Januszewski & Kostur, "Accelerating numerical solution of
 * stochastic differential equations with CUDA" (arXiv:0903.3852).
 *
 *   Eq. 1  (Sec. 3)   driven damped particle in V(x) = sin(2 pi x):
 *          x'' + gamma x' = -V'(x) + a cos(omega t) + f + sqrt(2 gamma D) xi(t)
 *   Eq. 2  (Sec. 3)   Kuramoto: gamma x_i' = omega_i + sum_j K_ij sin(x_j - x_i)
 *                                  + sqrt(2 gamma D) xi_i(t),   gamma = 1 here
 *   Alg. 2 (Sec. 4.1) SRK2 (Heun with additive noise, the same psi in both
 *          stages):  F1 = f(x0); F2 = f(x0 + dt F1 + sqrt(2 D dt) psi);
 *          x(dt) = x0 + dt/2 (F1 + F2) + sqrt(2 D dt) psi
 *   Eq. 3  (Sec. 4.2) mean-field form of the uniform coupling sum.
 *   Sec. 4.2          PROG2 advances with a first-order Euler scheme;
 *          with noise this is Euler-Maruyama: x(dt) = x0 + dt f(x0) +
 *          sqrt(2 D dt) psi (the *_euler_* functions, scheme 1).
 *   Sec. 4.1          two uniforms -> Box-Muller -> Gaussians; one RNG
 *                     stream per path.  The paper's xorshift is replaced by
 *                     Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11,
 *                     "Parallel random numbers: as easy as 1, 2, 3").
 *   Sec. 5            drive time kept modulo the period; here the drive is
 *                     evaluated directly at t_n = n dt in FP64.
 *
 * Every floating-point quantity is double.  No blocking, fusion or
 * reordering beyond the definitions above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11, Sec. 4 and Table 2).            */
/* Round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2 (full 64-bit products);  */
/* c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by  */
/* the Weyl constants between rounds.                                   */
/* ------------------------------------------------------------------ */
/* The first `rounds` rounds (Philox4x32-R); R = 10 is the generator used
 * everywhere.  Fewer rounds exist only so that tests can read the round
 * function and key schedule off known inputs. */
void oracle_philox4x32_rounds(const uint32_t ctr[4], const uint32_t key[2],
                              int rounds, uint32_t out[4]) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < rounds; ++round) {
    uint64_t p0 = M0 * (uint64_t)c[0];
    uint64_t p1 = M1 * (uint64_t)c[2];
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += W0;
    k1 += W1;
  }
  memcpy(out, c, sizeof c);
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  oracle_philox4x32_rounds(ctr, key, 10, out);
}

/* Uniform variate from one 32-bit word: the top 24 bits, shifted into
 * (0, 1]:  u = ((w >> 8) + 1) * 2^-24.  Never 0, so log(u) is finite. */
double oracle_uniform(uint32_t w) {
  return ((double)(w >> 8) + 1.0) * (1.0 / 16777216.0);
}

/* Box-Muller (Sec. 4.1: two uniforms -> two Gaussians). */
void oracle_box_muller(uint32_t w0, uint32_t w1, double *z0, double *z1) {
  double u0 = oracle_uniform(w0), u1 = oracle_uniform(w1);
  double rho = sqrt(-2.0 * log(u0));
  double th = 2.0 * OR_PI * u1;
  *z0 = rho * cos(th);
  *z1 = rho * sin(th);
}

/* Noise stream layout.  Key = (seed low word, seed high word).  The
 * Gaussian used by step n of stream (c1, c2, tag) comes from the Philox
 * block with counter (n / 4, c1, c2, tag): steps 4g, 4g+1 take the pair
 * built from words (0, 1), steps 4g+2, 4g+3 the pair from words (2, 3). */
double oracle_gaussian(uint64_t seed, uint32_t tag, uint32_t c1, uint32_t c2,
                       uint64_t n) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)(n >> 2), c1, c2, tag};
  uint32_t w[4];
  oracle_philox4x32_10(ctr, key, w);
  double z0, z1;
  if (n & 2) oracle_box_muller(w[2], w[3], &z0, &z1);
  else       oracle_box_muller(w[0], w[1], &z0, &z1);
  return (n & 1) ? z1 : z0;
}

#define TAG_JOSEPHSON 1u
#define TAG_KURAMOTO 2u

/* ------------------------------------------------------------------ */
/* Eq. 1 as a first-order system y = (x, v):                           */
/*   x' = v,   v' = -gamma v - 2 pi cos(2 pi x) + a cos(omega t) + f     */
/* plus noise sqrt(2 gamma D) xi on v only.                              */
/* ------------------------------------------------------------------ */
typedef struct {
  double gamma, a, omega, f, D;
} oracle_jj_params;

static double jj_force(double x, double v, double t, const oracle_jj_params *p) {
  return -p->gamma * v - 2.0 * OR_PI * cos(2.0 * OR_PI * x) +
         p->a * cos(p->omega * t) + p->f;
}

/* One SRK2 step (Alg. 2) of Eq. 1 from t_n = n dt to t_{n+1}, with the
 * given standard Gaussian psi.  The noise increment on v is
 * sqrt(2 gamma D dt) psi, the same psi in predictor and corrector; the
 * second stage is evaluated at t_{n+1}. */
void oracle_jj_step(double *x, double *v, uint64_t n, double dt,
                    const oracle_jj_params *p, double psi) {
  double t0 = (double)n * dt, t1 = (double)(n + 1) * dt;
  double noise = sqrt(2.0 * p->gamma * p->D * dt) * psi;
  double F1x = *v;
  double F1v = jj_force(*x, *v, t0, p);
  double xt = *x + dt * F1x;
  double vt = *v + dt * F1v + noise;
  double F2x = vt;
  double F2v = jj_force(xt, vt, t1, p);
  *x = *x + 0.5 * dt * (F1x + F2x);
  *v = *v + 0.5 * dt * (F1v + F2v) + noise;
}

/* Deterministic right-hand side of Eq. 1 (for comparison with an ODE
 * solver in the D = 0 limit). */
void oracle_jj_rhs(double t, const double y[2], const oracle_jj_params *p,
                   double dy[2]) {
  dy[0] = y[1];
  dy[1] = jj_force(y[0], y[1], t, p);
}

/* Advance an ensemble of paths of one parameter point from step n_begin
 * to n_end (Alg. 1: per path, load state, loop over steps drawing fresh
 * Gaussians, store state).  Path j of point k uses noise stream
 * (c1 = path0 + j, c2 = k, tag 1).  The time step is dt = 2 pi /
 * (omega * steps_per_period).  vsum accumulates v after every step whose
 * new state index n + 1 lies in the averaging window (S - W, S] with
 * W = floor(S / 2) and S = total_steps. */
/* One Euler-Maruyama step of Eq. 1: the first-order scheme that the
 * paper's PROG2 uses in its AdvanceSystem kernel (Sec. 4.2), here on
 * (x, v): y_{n+1} = y_n + dt F(y_n, t_n) + (0, sqrt(2 gamma D dt) psi). */
void oracle_jj_euler_step(double *x, double *v, uint64_t n, double dt,
                          const oracle_jj_params *p, double psi) {
  double t0 = (double)n * dt;
  double noise = sqrt(2.0 * p->gamma * p->D * dt) * psi;
  double Fx = *v;
  double Fv = jj_force(*x, *v, t0, p);
  *x = *x + dt * Fx;
  *v = *v + dt * Fv + noise;
}

/* oracle_jj_run with the scheme chosen: 0 = SRK2 (Alg. 2), 1 = Euler-Maruyama. */
void oracle_jj_run_scheme(int64_t npaths, double *x, double *v, double *vsum,
                          const oracle_jj_params *p, int32_t steps_per_period,
                          uint64_t n_begin, uint64_t n_end, uint64_t total_steps,
                          uint64_t seed, uint32_t point, uint32_t path0, int scheme) {
  double dt = 2.0 * OR_PI / (p->omega * (double)steps_per_period);
  uint64_t wstart = total_steps - total_steps / 2; /* first index NOT in window is <= wstart */
  for (int64_t j = 0; j < npaths; ++j) {
    double xj = x[j], vj = v[j], sj = vsum ? vsum[j] : 0.0;
    for (uint64_t n = n_begin; n < n_end; ++n) {
      double psi = oracle_gaussian(seed, TAG_JOSEPHSON, path0 + (uint32_t)j,
                                   point, n);
      if (scheme == 1)
        oracle_jj_euler_step(&xj, &vj, n, dt, p, psi);
      else
        oracle_jj_step(&xj, &vj, n, dt, p, psi);
      if (n + 1 > wstart) sj += vj;
    }
    x[j] = xj;
    v[j] = vj;
    if (vsum) vsum[j] = sj;
  }
}

void oracle_jj_run(int64_t npaths, double *x, double *v, double *vsum,
                   const oracle_jj_params *p, int32_t steps_per_period,
                   uint64_t n_begin, uint64_t n_end, uint64_t total_steps,
                   uint64_t seed, uint32_t point, uint32_t path0) {
  oracle_jj_run_scheme(npaths, x, v, vsum, p, steps_per_period, n_begin, n_end,
                       total_steps, seed, point, path0, 0);
}

/* Linear test drift for the weak-order check: x' = v,
 * v' = -gamma v - kappa x + f, noise sqrt(2 gamma D) xi on v.  Same SRK2
 * step as oracle_jj_step, with the force replaced. */
void oracle_linear_step(double *x, double *v, double dt, double gamma,
                        double kappa, double f, double D, double psi) {
  double noise = sqrt(2.0 * gamma * D * dt) * psi;
  double F1x = *v, F1v = -gamma * *v - kappa * *x + f;
  double xt = *x + dt * F1x, vt = *v + dt * F1v + noise;
  double F2x = vt, F2v = -gamma * vt - kappa * xt + f;
  *x = *x + 0.5 * dt * (F1x + F2x);
  *v = *v + 0.5 * dt * (F1v + F2v) + noise;
}

/* Euler-Maruyama step with the same linear force. */
void oracle_linear_euler_step(double *x, double *v, double dt, double gamma,
                              double kappa, double f, double D, double psi) {
  double noise = sqrt(2.0 * gamma * D * dt) * psi;
  double Fx = *v, Fv = -gamma * *v - kappa * *x + f;
  *x = *x + dt * Fx;
  *v = *v + dt * Fv + noise;
}

/* ------------------------------------------------------------------ */
/* Kuramoto (Eq. 2, gamma = 1).                                         */
/* ------------------------------------------------------------------ */

/* Direct coupling sum, the plain definition: out_i = sum_j K_ij
 * sin(phi_j - phi_i).  Kmat is N x N row-major (row i); if Kmat is NULL
 * every K_ij equals Kconst. */
void oracle_kuramoto_coupling_direct(int64_t N, const double *phi,
                                     const double *Kmat, double Kconst,
                                     double *out) {
  for (int64_t i = 0; i < N; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      double kij = Kmat ? Kmat[i * N + j] : Kconst;
      s += kij * sin(phi[j] - phi[i]);
    }
    out[i] = s;
  }
}

/* Mean-field form for uniform K_ij = Kconst (Eq. 3):
 * sum_j sin(phi_j - phi_i) = cos(phi_i) S - sin(phi_i) C,
 * S = sum_j sin(phi_j), C = sum_j cos(phi_j). */
void oracle_kuramoto_coupling_meanfield(int64_t N, const double *phi,
                                        double Kconst, double *out) {
  double S = 0.0, C = 0.0;
  for (int64_t j = 0; j < N; ++j) {
    S += sin(phi[j]);
    C += cos(phi[j]);
  }
  for (int64_t i = 0; i < N; ++i)
    out[i] = Kconst * (cos(phi[i]) * S - sin(phi[i]) * C);
}

/* Order parameter r = |N^-1 sum_j exp(i phi_j)|. */
double oracle_order_parameter(int64_t N, const double *phi) {
  double S = 0.0, C = 0.0;
  for (int64_t j = 0; j < N; ++j) {
    S += sin(phi[j]);
    C += cos(phi[j]);
  }
  return sqrt(S * S + C * C) / (double)N;
}

/* One replica of Eq. 2 advanced by SRK2 (Alg. 2) from step n_begin to
 * n_end.  phi, omega: length N.  Coupling: Kmat (N x N) or uniform
 * Kconst; use_meanfield selects Eq. 3 for the uniform case (Kmat NULL).
 * Oscillator i of replica `replica` uses noise stream
 * (c1 = i, c2 = replica, tag 2), the same psi in both stages.  If r_out
 * is not NULL, r(t_n) is written to r_out[(n - n_begin) / sample_every]
 * for every n in [n_begin, n_end) with (n - n_begin) % sample_every == 0,
 * and r at n_end to the slot after the last sample. */
void oracle_kuramoto_run_scheme(int64_t N, double *phi, const double *omega,
                                const double *Kmat, double Kconst, int use_meanfield,
                                double D, double dt, uint64_t n_begin, uint64_t n_end,
                                uint64_t seed, uint32_t replica, double *r_out,
                                int64_t sample_every, int scheme) {
  double *F1 = (double *)malloc(sizeof(double) * N);
  double *F2 = (double *)malloc(sizeof(double) * N);
  double *pt = (double *)malloc(sizeof(double) * N);
  double *psi = (double *)malloc(sizeof(double) * N);
  double amp = sqrt(2.0 * D * dt);
  for (uint64_t n = n_begin; n < n_end; ++n) {
    if (r_out && sample_every > 0 && (n - n_begin) % (uint64_t)sample_every == 0)
      r_out[(n - n_begin) / (uint64_t)sample_every] = oracle_order_parameter(N, phi);
    if (Kmat || !use_meanfield)
      oracle_kuramoto_coupling_direct(N, phi, Kmat, Kconst, F1);
    else
      oracle_kuramoto_coupling_meanfield(N, phi, Kconst, F1);
    if (scheme == 1) {
      /* Euler-Maruyama (PROG2's AdvanceSystem): phi += dt F(phi) + noise */
      for (int64_t i = 0; i < N; ++i) {
        double z = oracle_gaussian(seed, TAG_KURAMOTO, (uint32_t)i, replica, n);
        phi[i] = phi[i] + dt * (F1[i] + omega[i]) + amp * z;
      }
      continue;
    }
    for (int64_t i = 0; i < N; ++i) {
      F1[i] += omega[i];
      psi[i] = oracle_gaussian(seed, TAG_KURAMOTO, (uint32_t)i, replica, n);
      pt[i] = phi[i] + dt * F1[i] + amp * psi[i];
    }
    if (Kmat || !use_meanfield)
      oracle_kuramoto_coupling_direct(N, pt, Kmat, Kconst, F2);
    else
      oracle_kuramoto_coupling_meanfield(N, pt, Kconst, F2);
    for (int64_t i = 0; i < N; ++i) {
      F2[i] += omega[i];
      phi[i] = phi[i] + 0.5 * dt * (F1[i] + F2[i]) + amp * psi[i];
    }
  }
  if (r_out && sample_every > 0) {
    uint64_t ns = (n_end - n_begin + (uint64_t)sample_every - 1) / (uint64_t)sample_every;
    r_out[ns] = oracle_order_parameter(N, phi);
  }
  free(F1);
  free(F2);
  free(pt);
  free(psi);
}

void oracle_kuramoto_run(int64_t N, double *phi, const double *omega,
                         const double *Kmat, double Kconst, int use_meanfield,
                         double D, double dt, uint64_t n_begin, uint64_t n_end,
                         uint64_t seed, uint32_t replica, double *r_out,
                         int64_t sample_every) {
  oracle_kuramoto_run_scheme(N, phi, omega, Kmat, Kconst, use_meanfield, D, dt,
                             n_begin, n_end, seed, replica, r_out, sample_every, 0);
}

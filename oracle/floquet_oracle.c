/*
 * floquet_oracle.c -- plain FP64 CPU oracle for the Floquet evolution of an
 * open spin chain (arXiv 2111.08044, Sec. III).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg may load this file's library.  It shares no code, header,
 * table or helper with the CUDA library; the two meet only through seeded
 * inputs.
 *
 * What it computes, written as the plain definition (no blocking, no fusion,
 * no reordering):
 *   - the product state  psi_x = prod_i s_i[b_i(x)]  (a product initial
 *     state as in Eq. 9, here of single-site states; bit i of x is site i);
 *   - each gate  U_b = exp(-i tau h_b)  of a two-site Hermitian h_b (Eq. 5)
 *     by Taylor series with scaling and squaring;
 *   - one period  U_F = R * (U_second U_first)^K  applied gate by gate by
 *     explicit index pairing, all gates of one layer then all of the other
 *     (the alternation of Eq. 4, repeated K times as a Trotter sequence,
 *     Sec. III.A), then the kick R = prod_i exp(-i theta X_i); periods are
 *     applied one after another as in Eq. 3;
 *   - the energy  <psi| H0 |psi>,  H0 = sum_b h_b  (Eq. 7, Eq. 10), by
 *     applying every h_b to its four-amplitude groups;
 *   - the reverse-mode gradient of the final energy with respect to
 *     per-period kick angles and transverse fields (adjoint sweep);
 *   - the energy moments <psi|H0|psi> and <psi|H0^2|psi> = |H0 psi|^2 behind
 *     E and sigma_E (Eq. 10, Eq. 11), with H0 psi built term by term.
 *
 * Local two-site index: r = 2*b_i + b_{i+1}; site i is the high bit of r,
 * as in the contraction U_{b7 b8 alpha beta} of Eq. 2.
 * Matrices are row-major, complex entries stored as (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

int or_version(void) { return 1; }

/* Thread count of the OpenMP loops (for the timed CPU baseline: single-
 * thread and all-core runs in one process).  No arithmetic depends on it
 * beyond the order of the parallel reductions' partial sums. */
#ifdef _OPENMP
#include <omp.h>
int or_max_threads(void) { return omp_get_max_threads(); }
int or_set_threads(int n) {
  if (n < 1) return OR_EINVAL;
  omp_set_num_threads(n);
  return OR_OK;
}
#else
int or_max_threads(void) { return 1; }
int or_set_threads(int n) { return n < 1 ? OR_EINVAL : OR_OK; }
#endif

/* ---------------------------------------------------------------- matrices */

static void mat_load(int n, const double *src, cplx *dst) {
  for (int k = 0; k < n * n; ++k) dst[k] = src[2 * k] + I * src[2 * k + 1];
}

static void mat_store(int n, const cplx *src, double *dst) {
  for (int k = 0; k < n * n; ++k) {
    dst[2 * k] = creal(src[k]);
    dst[2 * k + 1] = cimag(src[k]);
  }
}

static void mat_mul(int n, const cplx *a, const cplx *b, cplx *c) {
  cplx t[16 * 16];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cplx s = 0;
      for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + j];
      t[i * n + j] = s;
    }
  memcpy(c, t, sizeof(cplx) * n * n);
}

/* exp(A) for n <= 16 by scaling and squaring of the Taylor series. */
static void mat_exp(int n, const cplx *a, cplx *e) {
  double norm = 0.0; /* max column sum */
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += cabs(a[i * n + j]);
    if (s > norm) norm = s;
  }
  int sq = 0;
  while (norm > 0.25) {
    norm *= 0.5;
    ++sq;
  }
  double scale = ldexp(1.0, -sq);
  cplx b[16 * 16], term[16 * 16], sum[16 * 16];
  for (int k = 0; k < n * n; ++k) b[k] = a[k] * scale;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) sum[i * n + j] = term[i * n + j] = (i == j);
  for (int k = 1; k <= 30; ++k) {
    mat_mul(n, term, b, term);
    for (int q = 0; q < n * n; ++q) {
      term[q] /= (double)k;
      sum[q] += term[q];
    }
  }
  for (int s = 0; s < sq; ++s) mat_mul(n, sum, sum, sum);
  memcpy(e, sum, sizeof(cplx) * n * n);
}

/* G = exp(-i tau h) for an n x n Hermitian h (n = 2 or 4). */
int or_expm_herm(int n, const double *h, double tau, double *g_out) {
  if (n < 1 || n > 16 || !h || !g_out) return OR_EINVAL;
  cplx hm[16 * 16], a[16 * 16], g[16 * 16];
  mat_load(n, h, hm);
  for (int k = 0; k < n * n; ++k) a[k] = -I * tau * hm[k];
  mat_exp(n, a, g);
  mat_store(n, g, g_out);
  return OR_OK;
}

/* ------------------------------------------------------------ state basics */

int or_product_state(int L, const double *spinors, double *psi) {
  if (L < 1 || L > 34 || !spinors || !psi) return OR_EINVAL;
  const uint64_t dim = 1ull << L;
#pragma omp parallel for schedule(static) if (L >= 14)
  for (uint64_t x = 0; x < dim; ++x) {
    cplx amp = 1.0;
    for (int i = 0; i < L; ++i) {
      int b = (int)((x >> i) & 1u);
      amp *= spinors[4 * i + 2 * b] + I * spinors[4 * i + 2 * b + 1];
    }
    psi[2 * x] = creal(amp);
    psi[2 * x + 1] = cimag(amp);
  }
  return OR_OK;
}

/* Apply a 4x4 gate to sites (i, i+1) by explicit index pairing. */
int or_apply_2q(int L, double *psi, int i, const double *g) {
  if (L < 2 || i < 0 || i + 1 >= L || !psi || !g) return OR_EINVAL;
  cplx G[16];
  mat_load(4, g, G);
  const uint64_t ngroups = 1ull << (L - 2);
  const uint64_t lomask = (1ull << i) - 1;
  const uint64_t si = 1ull << i, sj = 1ull << (i + 1);
  cplx *p = (cplx *)psi;
#pragma omp parallel for schedule(static) if (L >= 14)
  for (uint64_t q = 0; q < ngroups; ++q) {
    uint64_t x = (q & lomask) | ((q >> i) << (i + 2));
    uint64_t idx[4];
    cplx v[4], w[4];
    for (int r = 0; r < 4; ++r) {
      idx[r] = x + (uint64_t)(r >> 1) * si + (uint64_t)(r & 1) * sj;
      v[r] = p[idx[r]];
    }
    for (int r = 0; r < 4; ++r) {
      w[r] = 0;
      for (int c = 0; c < 4; ++c) w[r] += G[4 * r + c] * v[c];
    }
    for (int r = 0; r < 4; ++r) p[idx[r]] = w[r];
  }
  return OR_OK;
}

/* Apply a 2x2 gate to site i. */
int or_apply_1q(int L, double *psi, int i, const double *g) {
  if (L < 1 || i < 0 || i >= L || !psi || !g) return OR_EINVAL;
  cplx G[4];
  mat_load(2, g, G);
  const uint64_t npairs = 1ull << (L - 1);
  const uint64_t lomask = (1ull << i) - 1;
  const uint64_t si = 1ull << i;
  cplx *p = (cplx *)psi;
#pragma omp parallel for schedule(static) if (L >= 14)
  for (uint64_t q = 0; q < npairs; ++q) {
    uint64_t x = (q & lomask) | ((q >> i) << (i + 1));
    cplx v0 = p[x], v1 = p[x + si];
    p[x] = G[0] * v0 + G[1] * v1;
    p[x + si] = G[2] * v0 + G[3] * v1;
  }
  return OR_OK;
}

/* <psi| A_b |psi> for a 4x4 operator on sites (i, i+1), and the norm. */
static cplx expect_2q(int L, const double *psi, int i, const cplx *A) {
  const uint64_t ngroups = 1ull << (L - 2);
  const uint64_t lomask = (1ull << i) - 1;
  const uint64_t si = 1ull << i, sj = 1ull << (i + 1);
  const cplx *p = (const cplx *)psi;
  double acc_re = 0.0, acc_im = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc_re, acc_im) if (L >= 14)
  for (uint64_t q = 0; q < ngroups; ++q) {
    uint64_t x = (q & lomask) | ((q >> i) << (i + 2));
    cplx v[4];
    for (int r = 0; r < 4; ++r)
      v[r] = p[x + (uint64_t)(r >> 1) * si + (uint64_t)(r & 1) * sj];
    cplx s = 0;
    for (int r = 0; r < 4; ++r) {
      cplx av = 0;
      for (int c = 0; c < 4; ++c) av += A[4 * r + c] * v[c];
      s += conj(v[r]) * av;
    }
    acc_re += creal(s);
    acc_im += cimag(s);
  }
  return acc_re + I * acc_im;
}

int or_norm2(int L, const double *psi, double *norm2) {
  if (L < 1 || !psi || !norm2) return OR_EINVAL;
  const uint64_t dim = 1ull << L;
  double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc) if (L >= 14)
  for (uint64_t x = 0; x < dim; ++x)
    acc += psi[2 * x] * psi[2 * x] + psi[2 * x + 1] * psi[2 * x + 1];
  *norm2 = acc;
  return OR_OK;
}

/* E = sum_b <psi|h_b|psi> (unnormalised psi), hbond: (L-1) 4x4 matrices. */
int or_energy(int L, const double *psi, const double *hbond, double *energy,
              double *norm2) {
  if (L < 2 || !psi || !hbond) return OR_EINVAL;
  double e = 0.0;
  for (int b = 0; b < L - 1; ++b) {
    cplx h[16];
    mat_load(4, hbond + 32 * b, h);
    e += creal(expect_2q(L, psi, b, h));
  }
  if (energy) *energy = e;
  if (norm2) or_norm2(L, psi, norm2);
  return OR_OK;
}

/* ------------------------------------------------------------------ period */

/*
 * One Floquet period.  gates: (L-1) 4x4 bond gates; kick: L 2x2 site gates
 * (may be NULL for no kick).  Layer order per Trotter step: bonds with
 * b % 2 == first_layer, then the other parity; K steps; then the kick.
 */
int or_period(int L, double *psi, const double *gates, const double *kick, int K,
              int first_layer) {
  if (L < 2 || !psi || !gates || K < 1 || (first_layer != 0 && first_layer != 1))
    return OR_EINVAL;
  for (int s = 0; s < K; ++s)
    for (int layer = 0; layer < 2; ++layer) {
      int parity = layer == 0 ? first_layer : 1 - first_layer;
      for (int b = parity; b < L - 1; b += 2) or_apply_2q(L, psi, b, gates + 32 * b);
    }
  if (kick)
    for (int i = 0; i < L; ++i) or_apply_1q(L, psi, i, kick + 8 * i);
  return OR_OK;
}

/* The inverse period U_F^dagger, for echo studies: kick^dagger, then the
 * layers in reverse order, each gate replaced by its adjoint. */
int or_period_inverse(int L, double *psi, const double *gates, const double *kick,
                      int K, int first_layer) {
  if (L < 2 || !psi || !gates || K < 1 || (first_layer != 0 && first_layer != 1))
    return OR_EINVAL;
  double gd[32], kd[8];
  if (kick)
    for (int i = 0; i < L; ++i) {
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
          kd[2 * (2 * r + c)] = kick[8 * i + 2 * (2 * c + r)];
          kd[2 * (2 * r + c) + 1] = -kick[8 * i + 2 * (2 * c + r) + 1];
        }
      or_apply_1q(L, psi, i, kd);
    }
  for (int s = 0; s < K; ++s)
    for (int layer = 1; layer >= 0; --layer) {
      int parity = layer == 0 ? first_layer : 1 - first_layer;
      for (int b = parity; b < L - 1; b += 2) {
        const double *g = gates + 32 * b;
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) {
            gd[2 * (4 * r + c)] = g[2 * (4 * c + r)];
            gd[2 * (4 * r + c) + 1] = -g[2 * (4 * c + r) + 1];
          }
        or_apply_2q(L, psi, b, gd);
      }
    }
  return OR_OK;
}

static void kick_gate(double theta, double *k8) {
  /* exp(-i theta X) through the same Taylor route as the bond gates. */
  double x[8] = {0, 0, 1, 0, 1, 0, 0, 0};
  or_expm_herm(2, x, theta, k8);
}

/*
 * Evolve `periods` periods and record the energy density of the normalised
 * state, <psi|H0|psi> / (L <psi|psi>), and |psi|^2 after each one.
 *   hdrive : bond Hamiltonians that generate the gates, (L-1) 4x4 each;
 *            if per_period != 0 there are `periods` such sets back to back.
 *   theta  : kick angle, one value or one per period (per_period != 0).
 *   hobs   : bond Hamiltonians of the observable H0 = sum_b h_b.
 *   tau    : gate time, gate = exp(-i tau h_b).
 */
int or_evolve(int L, double *psi, int64_t periods, const double *hdrive,
              int per_period, double tau, const double *theta, int K,
              int first_layer, const double *hobs, double *energy_density,
              double *norm2) {
  if (L < 2 || !psi || !hdrive || !theta || periods < 0 || K < 1) return OR_EINVAL;
  double *gates = (double *)malloc(sizeof(double) * 32 * (L - 1));
  double *kick = (double *)malloc(sizeof(double) * 8 * L);
  if (!gates || !kick) {
    free(gates);
    free(kick);
    return OR_ENOMEM;
  }
  for (int64_t p = 0; p < periods; ++p) {
    if (p == 0 || per_period) {
      const double *hd = hdrive + (per_period ? (size_t)p * 32 * (L - 1) : 0);
      for (int b = 0; b < L - 1; ++b) or_expm_herm(4, hd + 32 * b, tau, gates + 32 * b);
      double th = theta[per_period ? p : 0];
      for (int i = 0; i < L; ++i) kick_gate(th, kick + 8 * i);
    }
    or_period(L, psi, gates, kick, K, first_layer);
    if (energy_density || norm2) {
      double e = 0.0, n2 = 0.0;
      if (hobs) or_energy(L, psi, hobs, &e, &n2);
      else or_norm2(L, psi, &n2);
      if (energy_density) energy_density[p] = hobs ? e / (L * n2) : 0.0;
      if (norm2) norm2[p] = n2;
    }
  }
  free(gates);
  free(kick);
  return OR_OK;
}

/* ----------------------------------------------------------------- adjoint */

/* out = A applied to sites (i, i+1) of a copy of psi. */
static void apply_2q_copy(int L, const double *psi, int i, const double *a, double *out) {
  memcpy(out, psi, sizeof(double) * 2 * (1ull << L));
  or_apply_2q(L, out, i, a);
}

static void apply_1q_copy(int L, const double *psi, int i, const double *a, double *out) {
  memcpy(out, psi, sizeof(double) * 2 * (1ull << L));
  or_apply_1q(L, out, i, a);
}

/* Re <u|v> */
static double inner_re(int L, const double *u, const double *v) {
  const uint64_t n = 2ull << L;
  double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc) if (L >= 14)
  for (uint64_t k = 0; k < n; ++k) acc += u[k] * v[k];
  return acc;
}

static void dagger(int n, const double *g, double *gd) {
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      gd[2 * (n * r + c)] = g[2 * (n * c + r)];
      gd[2 * (n * r + c) + 1] = -g[2 * (n * c + r) + 1];
    }
}

/*
 * Directional derivative of G(a) = exp(-i tau h(a)) along dh = dh/da, from
 * the block-triangular identity exp([[A, E], [0, A]]) = [[e^A, D], [0, e^A]]
 * with A = -i tau h, E = -i tau dh, D the Frechet derivative of exp at A
 * in direction E (Van Loan, IEEE TAC 23 (1978) 395).
 */
static void expm_frechet(const double *h, const double *dh, double tau, double *g,
                         double *d) {
  cplx big[64], e[64];
  memset(big, 0, sizeof(big));
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      cplx hv = h[2 * (4 * r + c)] + I * h[2 * (4 * r + c) + 1];
      cplx dv = dh[2 * (4 * r + c)] + I * dh[2 * (4 * r + c) + 1];
      big[8 * r + c] = -I * tau * hv;
      big[8 * (r + 4) + (c + 4)] = -I * tau * hv;
      big[8 * r + (c + 4)] = -I * tau * dv;
    }
  mat_exp(8, big, e);
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      g[2 * (4 * r + c)] = creal(e[8 * r + c]);
      g[2 * (4 * r + c) + 1] = cimag(e[8 * r + c]);
      d[2 * (4 * r + c)] = creal(e[8 * r + c + 4]);
      d[2 * (4 * r + c) + 1] = cimag(e[8 * r + c + 4]);
    }
}

/*
 * Gradient of the final energy density f = <psi_P| H0 |psi_P> / L with
 * respect to the per-period kick angles theta_p and fields hx_p.
 *   psi      : in, the initial state; out, psi_P.
 *   hdrive   : P sets of (L-1) bond Hamiltonians at the given parameters.
 *   dhdrive  : P sets of (L-1) matrices dh_b / dhx_p.
 * Forward pass without storing states; then a reverse sweep that un-applies
 * every gate from psi and from the costate lambda (lambda_P = H0 psi_P / L)
 * and accumulates 2 Re <lambda | dG psi_before> per gate.
 */
int or_adjoint(int L, double *psi, int64_t P, const double *hdrive,
               const double *dhdrive, double tau, const double *theta, int K,
               int first_layer, const double *hobs, double *grad_theta,
               double *grad_hx, double *energy_density) {
  if (L < 2 || L > 34 || !psi || P < 1 || !hdrive || !dhdrive || !theta || !hobs ||
      K < 1)
    return OR_EINVAL;
  const size_t nd = 2ull << L;
  double *lam = (double *)calloc(nd, sizeof(double));
  double *tmp = (double *)malloc(sizeof(double) * nd);
  double *gates = (double *)malloc(sizeof(double) * 32 * (L - 1));
  double *dgates = (double *)malloc(sizeof(double) * 32 * (L - 1));
  double kick[8], kickd[8], dkick[8];
  if (!lam || !tmp || !gates || !dgates) {
    free(lam); free(tmp); free(gates); free(dgates);
    return OR_ENOMEM;
  }
  /* forward */
  for (int64_t p = 0; p < P; ++p) {
    const double *hd = hdrive + (size_t)p * 32 * (L - 1);
    for (int b = 0; b < L - 1; ++b) or_expm_herm(4, hd + 32 * b, tau, gates + 32 * b);
    double kk[8 * 64];
    kick_gate(theta[p], kick);
    for (int i = 0; i < L; ++i) memcpy(kk + 8 * i, kick, sizeof(kick));
    or_period(L, psi, gates, kk, K, first_layer);
  }
  /* lambda = H0 psi / L */
  for (int b = 0; b < L - 1; ++b) {
    apply_2q_copy(L, psi, b, hobs + 32 * b, tmp);
    for (size_t k = 0; k < nd; ++k) lam[k] += tmp[k] / L;
  }
  if (energy_density) *energy_density = inner_re(L, psi, lam);
  /* reverse sweep */
  const double xm[8] = {0, 0, 1, 0, 1, 0, 0, 0};
  for (int64_t p = P - 1; p >= 0; --p) {
    const double *hd = hdrive + (size_t)p * 32 * (L - 1);
    const double *dhd = dhdrive + (size_t)p * 32 * (L - 1);
    for (int b = 0; b < L - 1; ++b)
      expm_frechet(hd + 32 * b, dhd + 32 * b, tau, gates + 32 * b, dgates + 32 * b);
    /* d/dtheta exp(-i theta X) = -i X exp(-i theta X) */
    kick_gate(theta[p], kick);
    dagger(2, kick, kickd);
    {
      cplx k2[4], x2[4], r2[4];
      mat_load(2, kick, k2);
      mat_load(2, xm, x2);
      mat_mul(2, x2, k2, r2);
      for (int q = 0; q < 4; ++q) r2[q] *= -I;
      mat_store(2, r2, dkick);
    }
    double gt = 0.0, gh = 0.0;
    for (int i = L - 1; i >= 0; --i) {
      or_apply_1q(L, psi, i, kickd);
      apply_1q_copy(L, psi, i, dkick, tmp);
      gt += 2.0 * inner_re(L, lam, tmp);
      or_apply_1q(L, lam, i, kickd);
    }
    for (int s = K - 1; s >= 0; --s)
      for (int layer = 1; layer >= 0; --layer) {
        int parity = layer == 0 ? first_layer : 1 - first_layer;
        int last = L - 2; /* largest bond index of this parity */
        if ((last - parity) % 2 != 0) --last;
        for (int b = last; b >= parity; b -= 2) {
          double gd[32];
          dagger(4, gates + 32 * b, gd);
          or_apply_2q(L, psi, b, gd);
          apply_2q_copy(L, psi, b, dgates + 32 * b, tmp);
          gh += 2.0 * inner_re(L, lam, tmp);
          or_apply_2q(L, lam, b, gd);
        }
      }
    if (grad_theta) grad_theta[p] = gt;
    if (grad_hx) grad_hx[p] = gh;
  }
  /* psi is back at the initial state; run forward again so that it holds
     psi_P on return, as documented. */
  for (int64_t p = 0; p < P; ++p) {
    const double *hd = hdrive + (size_t)p * 32 * (L - 1);
    for (int b = 0; b < L - 1; ++b) or_expm_herm(4, hd + 32 * b, tau, gates + 32 * b);
    double kk[8 * 64];
    kick_gate(theta[p], kick);
    for (int i = 0; i < L; ++i) memcpy(kk + 8 * i, kick, sizeof(kick));
    or_period(L, psi, gates, kk, K, first_layer);
  }
  free(lam); free(tmp); free(gates); free(dgates);
  return OR_OK;
}

/* ----------------------------------------------------------- energy moments */

/*
 * e1 = <psi|H0|psi>, e2 = <psi|H0^2|psi> = |H0 psi|^2 and norm2 = <psi|psi>
 * (unnormalised psi), H0 = sum_b h_b (Eq. 7).  H0 psi is accumulated one
 * bond term at a time, each applied to a copy of psi by index pairing, so
 * that sigma_E = sqrt(e2/norm2 - (e1/norm2)^2) follows Eq. 11 directly.
 */
int or_energy_moments(int L, const double *psi, const double *hbond, double *e1, double *e2,
                      double *norm2) {
  if (L < 2 || !psi || !hbond) return OR_EINVAL;
  const uint64_t n = 2ull << L;
  double *hpsi = (double *)calloc(n, sizeof(double));
  double *tmp = (double *)malloc(n * sizeof(double));
  if (!hpsi || !tmp) {
    free(hpsi);
    free(tmp);
    return OR_ENOMEM;
  }
  for (int b = 0; b < L - 1; ++b) {
    apply_2q_copy(L, psi, b, hbond + 32 * b, tmp);
    for (uint64_t k = 0; k < n; ++k) hpsi[k] += tmp[k];
  }
  if (e1) *e1 = inner_re(L, psi, hpsi);
  if (e2) *e2 = inner_re(L, hpsi, hpsi);
  if (norm2) or_norm2(L, psi, norm2);
  free(hpsi);
  free(tmp);
  return OR_OK;
}

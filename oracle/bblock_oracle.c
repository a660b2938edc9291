/*
 * CPU FP64 oracle for stochastic-LapH baryon blocks (arXiv:2211.16278).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct reference
 * that the CUDA path is checked against. Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load it. It shares no code, header, table or
 * helper with the CUDA library, and it never calls it.
 *
 * Every routine writes out a definition from the paper as plain loops in double
 * precision, in the order the paper states it:
 *   - oracle_phase_table        the momentum phase e^{-i p.x} of Eq. (1)/(3),
 *                               p = 2 pi n / L, with (n.x) mod L taken in integers
 *                               before the trigonometry (the paper precomputes the
 *                               phase once per momentum set, Sec. 3).
 *   - oracle_reconstruct        Eq. (2): q_{alpha a x}^{(d)} = sum_l Q_{alpha l}^{(d)} phi^{(l)}_{a x}.
 *   - oracle_contract           Eq. (1): B^{(p)}_{d1 d2 d3} = sum_s c_s sum_x e^{-i p.x}
 *                               eps_{abc} q1_{alpha_s a x} q2_{beta_s b x} q3_{gamma_s c x}.
 *   - oracle_bblock             Eq. (2) followed by Eq. (1) for one time slice.
 *   - oracle_mode_triplet       Eq. (4): T^{p}_{l1 l2 l3}.
 *   - oracle_bblock_via_triplet Eq. (3) evaluated as T contracted with the three
 *                               coefficient matrices (the paper's two-step approach).
 *   - oracle_contract_compensated  Eq. (1) with compensated (Neumaier) summation of
 *                               the site sum; used only to bound the oracle's own
 *                               rounding error.
 *
 * Conventions (the paper leaves them implicit):
 *   - site x = (x0, x1, x2) in [0, L)^3, linear index x0 + L*(x1 + L*x2), origin 0;
 *   - eps_{012} = +1, totally antisymmetric;
 *   - no complex conjugation anywhere: B is complex-trilinear in q1, q2, q3;
 *   - coefficient matrix rows are spin-major: row alpha*n_ev + l, column d;
 *   - eigenvector storage V[l][x][a] (eigenvector l, site x, colour a).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following OpenMP loops (n >= 1); a timing control, no arithmetic. */
void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* The six nonzero entries of eps_{abc}: (a, b, c, sign). */
static const int EPS_PERM[6][4] = {
    {0, 1, 2, +1}, {1, 2, 0, +1}, {2, 0, 1, +1},
    {0, 2, 1, -1}, {2, 1, 0, -1}, {1, 0, 2, -1},
};

static const double PI_D = 3.14159265358979323846;

/* e^{-i 2 pi k / L} for the integer k = (n.x) mod L. */
static cplx phase_of(int L, const int n[3], long x) {
  long x0 = x % L, x1 = (x / L) % L, x2 = x / ((long)L * L);
  long k = (long)n[0] * x0 + (long)n[1] * x1 + (long)n[2] * x2;
  k %= L;
  if (k < 0) k += L;
  double ang = 2.0 * PI_D * (double)k / (double)L;
  return cos(ang) - I * sin(ang);
}

/* ph[p][x] = e^{-i p.x} for every momentum n_p (integer triples, p = 2 pi n / L). */
void oracle_phase_table(int L, int n_mom, const int *mom, cplx *ph) {
  long X = (long)L * L * L;
  for (int p = 0; p < n_mom; ++p)
    for (long x = 0; x < X; ++x) ph[(long)p * X + x] = phase_of(L, mom + 3 * p, x);
}

/* Eq. (2) for one spin alpha of one quark line:
 *   q[x][a][d] = sum_l V[l][x][a] * phi[alpha*n_ev + l][d],   d in [0, ndil). */
void oracle_reconstruct(long X, int n_ev, const cplx *V, const cplx *phi, int ndil, int alpha,
                        cplx *q) {
#pragma omp parallel for schedule(static)
  for (long x = 0; x < X; ++x)
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < ndil; ++d) {
        cplx acc = 0.0;
        for (int l = 0; l < n_ev; ++l)
          acc += V[((long)l * X + x) * 3 + a] * phi[((long)alpha * n_ev + l) * ndil + d];
        q[(x * 3 + a) * ndil + d] = acc;
      }
}

static cplx coef_of(const cplx *coef, int coef_per_mom, int n_spin, int p, int s) {
  return coef_per_mom ? coef[(long)p * n_spin + s] : coef[s];
}

/* Eq. (1) given reconstructed fields.
 * qi has layout [4 spins][X][3 colours][ndi]; spin[s] = (alpha_s, beta_s, gamma_s);
 * coef is [n_spin] (same for every momentum) or [n_mom][n_spin] (coef_per_mom != 0).
 * B[p][d1][d2][d3]. */
void oracle_contract(int L, const cplx *q1, int nd1, const cplx *q2, int nd2, const cplx *q3,
                     int nd3, int n_mom, const int *mom, int n_spin, const int *spin,
                     const cplx *coef, int coef_per_mom, cplx *B) {
  long X = (long)L * L * L;
  for (int p = 0; p < n_mom; ++p) {
#pragma omp parallel for schedule(dynamic)
    for (int d1 = 0; d1 < nd1; ++d1)
      for (int d2 = 0; d2 < nd2; ++d2)
        for (int d3 = 0; d3 < nd3; ++d3) {
          cplx acc = 0.0;
          for (int s = 0; s < n_spin; ++s) {
            int al = spin[3 * s], be = spin[3 * s + 1], ga = spin[3 * s + 2];
            cplx cs = coef_of(coef, coef_per_mom, n_spin, p, s);
            cplx site_sum = 0.0;
            for (long x = 0; x < X; ++x) {
              cplx e = 0.0;
              for (int k = 0; k < 6; ++k) {
                int a = EPS_PERM[k][0], b = EPS_PERM[k][1], c = EPS_PERM[k][2];
                cplx t = q1[(((long)al * X + x) * 3 + a) * nd1 + d1] *
                         q2[(((long)be * X + x) * 3 + b) * nd2 + d2] *
                         q3[(((long)ga * X + x) * 3 + c) * nd3 + d3];
                e += EPS_PERM[k][3] > 0 ? t : -t;
              }
              site_sum += phase_of(L, mom + 3 * p, x) * e;
            }
            acc += cs * site_sum;
          }
          B[(((long)p * nd1 + d1) * nd2 + d2) * nd3 + d3] = acc;
        }
  }
}

/* Neumaier-compensated running sum of one real component. */
typedef struct { double s, c; } csum;
static void csum_add(csum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}

/* Eq. (1) exactly as oracle_contract, but the site sum and the spin sum are
 * accumulated with compensated summation. Only used to bound the rounding error
 * of oracle_contract. */
void oracle_contract_compensated(int L, const cplx *q1, int nd1, const cplx *q2, int nd2,
                                 const cplx *q3, int nd3, int n_mom, const int *mom, int n_spin,
                                 const int *spin, const cplx *coef, int coef_per_mom, cplx *B) {
  long X = (long)L * L * L;
  for (int p = 0; p < n_mom; ++p) {
#pragma omp parallel for schedule(dynamic)
    for (int d1 = 0; d1 < nd1; ++d1)
      for (int d2 = 0; d2 < nd2; ++d2)
        for (int d3 = 0; d3 < nd3; ++d3) {
          csum re = {0, 0}, im = {0, 0};
          for (int s = 0; s < n_spin; ++s) {
            int al = spin[3 * s], be = spin[3 * s + 1], ga = spin[3 * s + 2];
            cplx cs = coef_of(coef, coef_per_mom, n_spin, p, s);
            for (long x = 0; x < X; ++x) {
              cplx w = cs * phase_of(L, mom + 3 * p, x);
              for (int k = 0; k < 6; ++k) {
                int a = EPS_PERM[k][0], b = EPS_PERM[k][1], c = EPS_PERM[k][2];
                cplx t = q1[(((long)al * X + x) * 3 + a) * nd1 + d1] *
                         q2[(((long)be * X + x) * 3 + b) * nd2 + d2] *
                         q3[(((long)ga * X + x) * 3 + c) * nd3 + d3];
                t = (EPS_PERM[k][3] > 0 ? t : -t) * w;
                csum_add(&re, creal(t));
                csum_add(&im, cimag(t));
              }
            }
          }
          B[(((long)p * nd1 + d1) * nd2 + d2) * nd3 + d3] = (re.s + re.c) + I * (im.s + im.c);
        }
  }
}

/* Eq. (2) then Eq. (1) for one time slice.
 * V is [n_ev][X][3]; phi_i is [4*n_ev][nd_i]; B is [n_mom][nd1][nd2][nd3].
 * Returns 0, or -1 if the scratch for the reconstructed fields cannot be allocated. */
int oracle_bblock(int L, int n_ev, const cplx *V, const cplx *phi1, int nd1, const cplx *phi2,
                  int nd2, const cplx *phi3, int nd3, int n_mom, const int *mom, int n_spin,
                  const int *spin, const cplx *coef, int coef_per_mom, cplx *B) {
  long X = (long)L * L * L;
  cplx *q1 = calloc((size_t)4 * X * 3 * nd1, sizeof(cplx));
  cplx *q2 = calloc((size_t)4 * X * 3 * nd2, sizeof(cplx));
  cplx *q3 = calloc((size_t)4 * X * 3 * nd3, sizeof(cplx));
  if (!q1 || !q2 || !q3) {
    free(q1); free(q2); free(q3);
    return -1;
  }
  int used[3][4];
  memset(used, 0, sizeof(used));
  for (int s = 0; s < n_spin; ++s)
    for (int i = 0; i < 3; ++i) used[i][spin[3 * s + i]] = 1;
  for (int al = 0; al < 4; ++al) {
    if (used[0][al]) oracle_reconstruct(X, n_ev, V, phi1, nd1, al, q1 + (long)al * X * 3 * nd1);
    if (used[1][al]) oracle_reconstruct(X, n_ev, V, phi2, nd2, al, q2 + (long)al * X * 3 * nd2);
    if (used[2][al]) oracle_reconstruct(X, n_ev, V, phi3, nd3, al, q3 + (long)al * X * 3 * nd3);
  }
  oracle_contract(L, q1, nd1, q2, nd2, q3, nd3, n_mom, mom, n_spin, spin, coef, coef_per_mom, B);
  free(q1); free(q2); free(q3);
  return 0;
}

/* Eq. (4): T[p][l1][l2][l3] = sum_x e^{-i p.x} eps_abc V[l1][x][a] V[l2][x][b] V[l3][x][c]. */
void oracle_mode_triplet(int L, int n_ev, const cplx *V, int n_mom, const int *mom, cplx *T) {
  long X = (long)L * L * L;
  for (int p = 0; p < n_mom; ++p) {
#pragma omp parallel for schedule(dynamic)
    for (int l1 = 0; l1 < n_ev; ++l1)
      for (int l2 = 0; l2 < n_ev; ++l2)
        for (int l3 = 0; l3 < n_ev; ++l3) {
          cplx acc = 0.0;
          for (long x = 0; x < X; ++x) {
            cplx e = 0.0;
            for (int k = 0; k < 6; ++k) {
              int a = EPS_PERM[k][0], b = EPS_PERM[k][1], c = EPS_PERM[k][2];
              cplx t = V[((long)l1 * X + x) * 3 + a] * V[((long)l2 * X + x) * 3 + b] *
                       V[((long)l3 * X + x) * 3 + c];
              e += EPS_PERM[k][3] > 0 ? t : -t;
            }
            acc += phase_of(L, mom + 3 * p, x) * e;
          }
          T[(((long)p * n_ev + l1) * n_ev + l2) * n_ev + l3] = acc;
        }
  }
}

/* Eq. (3) through the mode triplet:
 *   B[p][d1][d2][d3] = sum_s c_s sum_{l1 l2 l3} T[p][l1][l2][l3]
 *                      phi1[alpha_s n_ev + l1][d1] phi2[beta_s n_ev + l2][d2] phi3[gamma_s n_ev + l3][d3]. */
void oracle_bblock_via_triplet(int n_ev, const cplx *T, const cplx *phi1, int nd1,
                               const cplx *phi2, int nd2, const cplx *phi3, int nd3, int n_mom,
                               int n_spin, const int *spin, const cplx *coef, int coef_per_mom,
                               cplx *B) {
  for (int p = 0; p < n_mom; ++p) {
#pragma omp parallel for schedule(dynamic)
    for (int d1 = 0; d1 < nd1; ++d1)
      for (int d2 = 0; d2 < nd2; ++d2)
        for (int d3 = 0; d3 < nd3; ++d3) {
          cplx acc = 0.0;
          for (int s = 0; s < n_spin; ++s) {
            int al = spin[3 * s], be = spin[3 * s + 1], ga = spin[3 * s + 2];
            cplx part = 0.0;
            for (int l1 = 0; l1 < n_ev; ++l1)
              for (int l2 = 0; l2 < n_ev; ++l2)
                for (int l3 = 0; l3 < n_ev; ++l3)
                  part += T[(((long)p * n_ev + l1) * n_ev + l2) * n_ev + l3] *
                          phi1[((long)al * n_ev + l1) * nd1 + d1] *
                          phi2[((long)be * n_ev + l2) * nd2 + d2] *
                          phi3[((long)ga * n_ev + l3) * nd3 + d3];
            acc += coef_of(coef, coef_per_mom, n_spin, p, s) * part;
          }
          B[(((long)p * nd1 + d1) * nd2 + d2) * nd3 + d3] = acc;
        }
  }
}

/* Brute-force FP64 oracle for the ABC model (TEST INFRASTRUCTURE ONLY: used by
 * the tests, the smoke check and the benchmark's CPU baseline, never by the
 * product path).
 *
 * The model (paper App. F, and Sec. I-C): three scalar particles A, B, C and a single
 * vertex joining one of each.  In A(p) + B(k_0) -> A(p') + B(k_1) ... B(k_k)
 * every B attaches to the one A/C line that runs from the incoming to the
 * outgoing A, and the line changes species at every attachment: after i
 * attachments it is a C for odd i and an A for even i (Fig. ab_compton).  The
 * tree-level diagrams are therefore the n! orders (n = k + 1) in which the B
 * lines attach; the outgoing line is an A only for even n, so odd n (even k)
 * has no diagram and M = 0.
 *
 * With vertex factor -ig, propagator i/(q^2 - m^2) and external factors 1,
 *   M = g^n sum_{orders} prod_{i=1}^{n-1} 1 / (Q_i^2 - m_{s(i)}^2)
 * up to an overall phase, where Q_i = p + sum of the first i attached B
 * momenta, the incoming one with sign +1 and the outgoing ones with -1, and
 * s(i) is the species after i attachments.  |M|^2 is returned.
 *
 * kappa = sum_d |A_d| / |sum_d A_d| measures the cancellation among the
 * diagrams (0 for a vanishing amplitude with no diagram).
 *
 * Momenta: [npts][k+3][4] (E, px, py, pz); slot 0 = A in, 1 = B in,
 * 2 = A out, 3.. = B out.  Written in plain C in FP64, one point per
 * OpenMP iteration, no subexpression shared between diagrams.
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>

static double mdot(const double* a, const double* b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

/* next permutation in lexicographic order; 0 after the last one */
static int next_perm(int* a, int n) {
  int i = n - 2;
  while (i >= 0 && a[i] >= a[i + 1]) --i;
  if (i < 0) return 0;
  int j = n - 1;
  while (a[j] <= a[i]) --j;
  int t = a[i]; a[i] = a[j]; a[j] = t;
  for (int l = i + 1, r = n - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
  return 1;
}

/* sum with Knuth's TwoSum compensation */
static void add_comp(double* s, double* c, double x) {
  double t = *s + x;
  double bb = t - *s;
  *c += (*s - (t - bb)) + (x - bb);
  *s = t;
}

static double one_point(int k, const double* mom, double ma, double mc, double* kappa) {
  const int n = k + 1;
  if (n % 2 == 1) { *kappa = 0.0; return 0.0; }
  int order[16];
  const double* kb[16];
  double sign[16];
  for (int j = 0; j < n; ++j) {
    order[j] = j;
    kb[j] = mom + 4 * (j == 0 ? 1 : j + 2);
    sign[j] = j == 0 ? 1.0 : -1.0;
  }
  double sum = 0.0, comp = 0.0, abs_sum = 0.0;
  do {
    double amp = 1.0;
    unsigned attached = 0;
    for (int i = 1; i < n; ++i) {
      attached |= 1u << order[i - 1];
      /* Q_i from scratch: p, then the attached B's in ascending slot order */
      double q[4] = {mom[0], mom[1], mom[2], mom[3]};
      for (int j = 0; j < n; ++j)
        if (attached & (1u << j))
          for (int c = 0; c < 4; ++c) q[c] += sign[j] * kb[j][c];
      const double m = (i % 2 == 1) ? mc : ma;
      amp /= mdot(q, q) - m * m;
    }
    add_comp(&sum, &comp, amp);
    abs_sum += fabs(amp);
  } while (next_perm(order, n));
  const double total = sum + comp;
  *kappa = total != 0.0 ? abs_sum / fabs(total) : 0.0;
  return total;
}

int abc_oracle_m2(int k, long long npts, const double* momenta, double mass_a, double mass_c,
                  double coupling, double* out_m2, double* out_kappa, int nthreads) {
  if (k < 1 || k > 9 || npts < 0 || !momenta || !out_m2) return 1;
  const int n = k + 1;
  const double gn = pow(coupling, n);
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (long long i = 0; i < npts; ++i) {
    double kap;
    const double m = gn * one_point(k, momenta + i * (k + 3) * 4, mass_a, mass_c, &kap);
    out_m2[i] = m * m;
    if (out_kappa) out_kappa[i] = kap;
  }
  return 0;
}

int abc_oracle_amplitude(int k, const double* momenta, double mass_a, double mass_c, double coupling,
                         double* out_m) {
  if (k < 1 || k > 9 || !momenta || !out_m) return 1;
  double kap;
  *out_m = pow(coupling, k + 1) * one_point(k, momenta, mass_a, mass_c, &kap);
  return 0;
}

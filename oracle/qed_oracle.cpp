// Brute-force FP64 oracle for tree-level |M|^2 of multi-photon Compton
// scattering e-(p) gamma(k0) -> e-(p') + gamma(k1) ... gamma(kK).
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
// call this file: only the tests, the smoke check and the benchmark's CPU
// baseline leg use it.  It shares no code with the CUDA path.
//
// What it computes (paper Sec. I-D, Feynman rules and Eq. 1; Sec. III-A for
// the (n+1)! diagram count):
//
//   |M|^2 = sum_{lambda} | sum_{sigma in S_n} A_sigma(lambda) |^2 ,
//   A_sigma = ubar(p',s') eps/_{sigma(n)} S(Q_{n-1}) ... S(Q_1) eps/_{sigma(1)} u(p,s)
//   S(Q)    = (Q/ + m) / (Q^2 - m^2),
//   Q_i     = p + sum_{l<=i} c_{sigma(l)} k_{sigma(l)},  c = +1 (incoming
//             photon, absorbed), -1 (outgoing photon, emitted).
//
// Every diagram is evaluated on its own with explicit 4x4 complex Dirac
// matrices; nothing is shared between diagrams or spin configurations.  The
// common factor (-ie)^n i^(n-1) has unit modulus for e = 1 and is dropped.
// Diagram sums and the spin sum are accumulated in double-double (TwoSum).
//
// Conventions (the paper names the states but prints no convention; these
// are the readings documented with the project):
//   metric (+,-,-,-); Dirac representation gamma^0 = diag(1,1,-1,-1),
//   gamma^i = [[0, sigma^i], [-sigma^i, 0]]; a/ = gamma^0 a^0 - gamma.a.
//   u(p,h) = (sqrt(E+m) chi_h, h sqrt(E-m) chi_h), helicity two-spinors
//     chi_+ = (|p|+pz, px+i py) / sqrt(2|p|(|p|+pz)),
//     chi_- = (-px+i py, |p|+pz) / sqrt(2|p|(|p|+pz)),
//     |p| = 0 -> chi_+ = (1,0), chi_- = (0,1);
//     |p| + pz = 0 -> chi_+ = (0,1), chi_- = (-1,0).
//   ubar = u^dagger gamma^0 (normalisation ubar u = 2m).
//   Photons: real linear polarisation, eps^0 = 0,
//     eps_1 = (kx kz, ky kz, -kT^2) / (|k| kT),  eps_2 = (-ky, kx, 0) / kT,
//     kT = 0 -> eps_1 = x, eps_2 = y.  Real, so eps* = eps.
//   Propagator momenta are formed from the external momenta in ascending
//   slot order for the photon set to the left of the line, and
//   D = Q0*Q0 - Qx*Qx - Qy*Qy - Qz*Qz - m*m.
//
// Input layout: momenta[N][k+3][4], slot 0 = e- in, 1 = gamma in,
// 2 = e- out, 3..k+2 = gamma out; components (E, px, py, pz).
// Spin index of slot i: electrons h = +1/-1, photons pol = 1/2.
//
// Build: g++ -O2 -fopenmp -shared -fPIC qed_oracle.cpp -o liboracle.so

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <omp.h>

namespace {

// ---------------------------------------------------------------- scalars
struct Dual {  // forward-mode dual number: v + d * epsilon
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual sqrt_(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline double sqrt_(double a) { return std::sqrt(a); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }

template <class S>
struct Cx {
  S re, im;
  Cx() : re(0.0), im(0.0) {}
  Cx(S r) : re(r), im(0.0) {}
  Cx(S r, S i) : re(r), im(i) {}
};
template <class S> inline Cx<S> operator+(Cx<S> a, Cx<S> b) { return Cx<S>(a.re + b.re, a.im + b.im); }
template <class S> inline Cx<S> operator-(Cx<S> a, Cx<S> b) { return Cx<S>(a.re - b.re, a.im - b.im); }
template <class S> inline Cx<S> operator*(Cx<S> a, Cx<S> b) {
  return Cx<S>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class S> inline Cx<S> conj(Cx<S> a) { return Cx<S>(a.re, -a.im); }
template <class S> inline Cx<S> scale(Cx<S> a, S s) { return Cx<S>(a.re * s, a.im * s); }

template <class S> struct Vec4 { Cx<S> c[4]; };
template <class S> struct Mat4 { Cx<S> m[4][4]; };

template <class S>
Vec4<S> matvec(const Mat4<S>& A, const Vec4<S>& x) {
  Vec4<S> y;
  for (int i = 0; i < 4; ++i) {
    Cx<S> acc;
    for (int j = 0; j < 4; ++j) acc = acc + A.m[i][j] * x.c[j];
    y.c[i] = acc;
  }
  return y;
}

// ------------------------------------------------------- Dirac matrices
// gamma^mu in the Dirac representation, as explicit 4x4 complex matrices.
struct Gammas {
  Mat4<double> g[4];
  Gammas() {
    for (int mu = 0; mu < 4; ++mu)
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) g[mu].m[i][j] = Cx<double>(0.0, 0.0);
    // gamma^0 = diag(1, 1, -1, -1)
    g[0].m[0][0] = Cx<double>(1, 0); g[0].m[1][1] = Cx<double>(1, 0);
    g[0].m[2][2] = Cx<double>(-1, 0); g[0].m[3][3] = Cx<double>(-1, 0);
    // Pauli matrices
    Cx<double> pauli[3][2][2];
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) pauli[a][i][j] = Cx<double>(0, 0);
    pauli[0][0][1] = Cx<double>(1, 0);  pauli[0][1][0] = Cx<double>(1, 0);
    pauli[1][0][1] = Cx<double>(0, -1); pauli[1][1][0] = Cx<double>(0, 1);
    pauli[2][0][0] = Cx<double>(1, 0);  pauli[2][1][1] = Cx<double>(-1, 0);
    // gamma^i = [[0, sigma^i], [-sigma^i, 0]]
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          g[a + 1].m[i][j + 2] = pauli[a][i][j];
          g[a + 1].m[i + 2][j] = Cx<double>(-pauli[a][i][j].re, -pauli[a][i][j].im);
        }
  }
};
const Gammas& gammas() {
  static Gammas G;
  return G;
}

// a/ = gamma^0 a^0 - gamma^1 a^1 - gamma^2 a^2 - gamma^3 a^3 (a given with
// contravariant components).
template <class S>
Mat4<S> slash(const S a[4]) {
  const Gammas& G = gammas();
  Mat4<S> r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      Cx<S> acc;
      for (int mu = 0; mu < 4; ++mu) {
        S sgn = (mu == 0) ? S(1.0) : S(-1.0);
        Cx<S> gm(S(G.g[mu].m[i][j].re), S(G.g[mu].m[i][j].im));
        acc = acc + scale(gm, sgn * a[mu]);
      }
      r.m[i][j] = acc;
    }
  return r;
}

// Electron propagator numerator over denominator: (Q/ + m) / (Q^2 - m^2).
template <class S>
Mat4<S> propagator(const S Q[4], double m) {
  Mat4<S> P = slash(Q);
  S D = Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3] - S(m * m);
  for (int i = 0; i < 4; ++i) P.m[i][i] = P.m[i][i] + Cx<S>(S(m), S(0.0));
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) P.m[i][j] = Cx<S>(P.m[i][j].re / D, P.m[i][j].im / D);
  return P;
}

// Helicity two-spinor chi_h for the direction of the 3-momentum p.
template <class S>
void two_spinor(const S p[3], int h, Cx<S> chi[2]) {
  S px = p[0], py = p[1], pz = p[2];
  S ap = sqrt_(px * px + py * py + pz * pz);
  if (val(ap) == 0.0) {
    if (h > 0) { chi[0] = Cx<S>(S(1.0)); chi[1] = Cx<S>(S(0.0)); }
    else       { chi[0] = Cx<S>(S(0.0)); chi[1] = Cx<S>(S(1.0)); }
    return;
  }
  S apz = ap + pz;
  if (val(apz) == 0.0) {
    if (h > 0) { chi[0] = Cx<S>(S(0.0)); chi[1] = Cx<S>(S(1.0)); }
    else       { chi[0] = Cx<S>(S(-1.0)); chi[1] = Cx<S>(S(0.0)); }
    return;
  }
  S nrm = sqrt_(S(2.0) * ap * apz);
  if (h > 0) {
    chi[0] = Cx<S>(apz / nrm, S(0.0));
    chi[1] = Cx<S>(px / nrm, py / nrm);
  } else {
    chi[0] = Cx<S>(-px / nrm, py / nrm);
    chi[1] = Cx<S>(apz / nrm, S(0.0));
  }
}

// Dirac spinor u(p, h) = (sqrt(E+m) chi, h sqrt(E-m) chi).  E is taken from
// the given four-momentum.
template <class S>
Vec4<S> spinor_u(const S p[4], int h, double m) {
  Cx<S> chi[2];
  S p3[3] = {p[1], p[2], p[3]};
  two_spinor(p3, h, chi);
  S a = sqrt_(p[0] + S(m));
  S bb = p[0] - S(m);
  S b = (val(bb) > 0.0) ? sqrt_(bb) : S(0.0);
  if (h < 0) b = -b;
  Vec4<S> u;
  u.c[0] = scale(chi[0], a); u.c[1] = scale(chi[1], a);
  u.c[2] = scale(chi[0], b); u.c[3] = scale(chi[1], b);
  return u;
}

// ubar = u^dagger gamma^0, returned as a row vector.
template <class S>
Vec4<S> spinor_ubar(const S p[4], int h, double m) {
  Vec4<S> u = spinor_u(p, h, m);
  Vec4<S> r;
  for (int i = 0; i < 4; ++i) {
    Cx<S> c = conj(u.c[i]);
    r.c[i] = (i < 2) ? c : Cx<S>(-c.re, -c.im);
  }
  return r;
}

// Real linear photon polarisation four-vector (eps^0 = 0).
template <class S>
void polarisation(const S k[4], int pol, S eps[4]) {
  S kx = k[1], ky = k[2], kz = k[3];
  S kt2 = kx * kx + ky * ky;
  eps[0] = S(0.0);
  if (val(kt2) == 0.0) {
    eps[1] = S(pol == 1 ? 1.0 : 0.0);
    eps[2] = S(pol == 1 ? 0.0 : 1.0);
    eps[3] = S(0.0);
    return;
  }
  S kt = sqrt_(kt2);
  if (pol == 1) {
    S ak = sqrt_(kt2 + kz * kz);
    S den = ak * kt;
    eps[1] = kx * kz / den;
    eps[2] = ky * kz / den;
    eps[3] = -kt2 / den;
  } else {
    eps[1] = -ky / kt;
    eps[2] = kx / kt;
    eps[3] = S(0.0);
  }
}

// ------------------------------------------------- compensated summation
inline void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
struct DD {  // double-double accumulator
  double hi = 0.0, lo = 0.0;
  void add(double x) {
    double s, e;
    two_sum(hi, x, s, e);
    e += lo;
    two_sum(s, e, hi, lo);
  }
  double value() const { return hi + lo; }
};
template <class S> struct Acc;
template <> struct Acc<double> {
  DD a;
  void add(double x) { a.add(x); }
  double value() const { return a.value(); }
};
template <> struct Acc<Dual> {
  DD v, d;
  void add(Dual x) { v.add(x.v); d.add(x.d); }
  Dual value() const { return Dual(v.value(), d.value()); }
};

// ------------------------------------------------------------ the process
template <class S>
struct Process {
  int k = 0;            // number of outgoing photons
  int n = 0;            // number of photons = k + 1
  double m = 1.0;
  S p_in[4], p_out[4];
  S kph[8][4];          // photon momenta, photon 0 = incoming
  int csign[8];         // +1 incoming, -1 outgoing
};

// Photon index j (0 = incoming photon in slot 1, j >= 1 -> slot j + 2).
inline int photon_slot(int j) { return j == 0 ? 1 : j + 2; }

template <class S>
void momentum_of_set(const Process<S>& P, unsigned mask, S Q[4]) {
  // Q = p_in + sum over the photons of the set, in ascending slot order.
  for (int mu = 0; mu < 4; ++mu) Q[mu] = P.p_in[mu];
  for (int slot = 0; slot < P.n + 2; ++slot) {
    int j = (slot == 1) ? 0 : (slot >= 3 ? slot - 2 : -1);
    if (j < 0 || !(mask & (1u << j))) continue;
    for (int mu = 0; mu < 4; ++mu) {
      if (P.csign[j] > 0) Q[mu] = Q[mu] + P.kph[j][mu];
      else Q[mu] = Q[mu] - P.kph[j][mu];
    }
  }
}

struct Options {
  int sum_mask = 0;     // bit i set -> sum over both states of slot i
  int hel[10] = {0};    // fixed state of each slot where not summed
  int ward_photon = -1; // >= 0: replace eps of that photon by its momentum
};

// Result for one point: |M|^2 summed over the requested states, and the
// aggregate cancellation measure
//   kappa = sqrt( sum_lambda (sum_sigma |A|)^2 / sum_lambda |sum_sigma A|^2 ).
template <class S>
struct PointResult {
  S m2;
  double kappa;
  double ward_ratio;  // max_lambda |sum A| / sum |A|
};

template <class S>
PointResult<S> evaluate_point(const Process<S>& P, const Options& opt) {
  const int n = P.n;
  const int nslots = n + 2;
  std::vector<int> perm(n);
  int summed_slots[10];
  int ns = 0;
  for (int s = 0; s < nslots; ++s)
    if (opt.sum_mask & (1 << s)) summed_slots[ns++] = s;
  Acc<S> spin_sum;
  double sum_abs2 = 0.0, sum_m2 = 0.0, ward_ratio = 0.0;
  for (int cfg = 0; cfg < (1 << ns); ++cfg) {
    int st[10];
    for (int s = 0; s < nslots; ++s) st[s] = opt.hel[s];
    for (int b = 0; b < ns; ++b) {
      int s = summed_slots[b];
      int bit = (cfg >> b) & 1;
      bool electron = (s == 0 || s == 2);
      st[s] = electron ? (bit ? -1 : +1) : (bit ? 2 : 1);
    }
    Vec4<S> u = spinor_u(P.p_in, st[0], P.m);
    Vec4<S> ubar = spinor_ubar(P.p_out, st[2], P.m);
    Mat4<S> epsl[8];
    for (int j = 0; j < n; ++j) {
      S e[4];
      if (j == opt.ward_photon) {
        for (int mu = 0; mu < 4; ++mu) e[mu] = P.kph[j][mu];
      } else {
        polarisation(P.kph[j], st[photon_slot(j)], e);
      }
      epsl[j] = slash(e);
    }
    for (int j = 0; j < n; ++j) perm[j] = j;
    Acc<S> re, im;
    double abs_sum = 0.0;
    do {
      Vec4<S> v = u;
      unsigned mask = 0;
      for (int i = 0; i < n; ++i) {
        v = matvec(epsl[perm[i]], v);
        mask |= 1u << perm[i];
        if (i + 1 < n) {
          S Q[4];
          momentum_of_set(P, mask, Q);
          Mat4<S> Sq = propagator(Q, P.m);
          v = matvec(Sq, v);
        }
      }
      Cx<S> A;
      for (int c = 0; c < 4; ++c) A = A + ubar.c[c] * v.c[c];
      re.add(A.re);
      im.add(A.im);
      abs_sum += std::sqrt(val(A.re) * val(A.re) + val(A.im) * val(A.im));
    } while (std::next_permutation(perm.begin(), perm.end()));
    S mr = re.value(), mi = im.value();
    spin_sum.add(mr * mr);
    spin_sum.add(mi * mi);
    double am = std::sqrt(val(mr) * val(mr) + val(mi) * val(mi));
    sum_abs2 += abs_sum * abs_sum;
    sum_m2 += am * am;
    if (abs_sum > 0.0) ward_ratio = std::max(ward_ratio, am / abs_sum);
  }
  PointResult<S> r;
  r.m2 = spin_sum.value();
  r.kappa = (sum_m2 > 0.0) ? std::sqrt(sum_abs2 / sum_m2) : INFINITY;
  r.ward_ratio = ward_ratio;
  return r;
}

template <class S>
void load_process(Process<S>& P, int k, const double* mom, double mass) {
  P.k = k;
  P.n = k + 1;
  P.m = mass;
  for (int mu = 0; mu < 4; ++mu) {
    P.p_in[mu] = S(mom[0 * 4 + mu]);
    P.p_out[mu] = S(mom[2 * 4 + mu]);
    P.kph[0][mu] = S(mom[1 * 4 + mu]);
  }
  P.csign[0] = +1;
  for (int j = 1; j <= k; ++j) {
    for (int mu = 0; mu < 4; ++mu) P.kph[j][mu] = S(mom[(j + 2) * 4 + mu]);
    P.csign[j] = -1;
  }
}

bool valid_options(int k, int sum_mask, const int* hel, Options& opt) {
  if (k < 1 || k > 7) return false;
  int nslots = k + 3;
  opt.sum_mask = sum_mask & ((1 << nslots) - 1);
  for (int s = 0; s < nslots; ++s) {
    if (opt.sum_mask & (1 << s)) { opt.hel[s] = 0; continue; }
    int v = hel ? hel[s] : 0;
    bool electron = (s == 0 || s == 2);
    if (electron && v != 1 && v != -1) return false;
    if (!electron && v != 1 && v != 2) return false;
    opt.hel[s] = v;
  }
  return true;
}

}  // namespace

extern "C" {

// |M|^2 at npts points.  sum_mask: bit i -> slot i summed over its two
// states; hel[k+3] gives the fixed state of the other slots (ignored for
// summed slots, may be NULL when all are summed).  out_kappa may be NULL.
// nthreads > 0 fixes the OpenMP thread count.  Returns 0, or -1 on invalid
// arguments.
int oracle_m2(int k, long long npts, const double* momenta, int sum_mask, const int* hel,
              double mass, double* out_m2, double* out_kappa, int nthreads) {
  Options opt;
  if (!valid_options(k, sum_mask, hel, opt) || npts < 0 || !momenta || !out_m2) return -1;
  const int stride = (k + 3) * 4;
  int nt = nthreads > 0 ? nthreads : 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt > 0 ? nt : omp_get_max_threads())
  for (long long i = 0; i < npts; ++i) {
    Process<double> P;
    load_process(P, k, momenta + i * stride, mass);
    PointResult<double> r = evaluate_point(P, opt);
    out_m2[i] = r.m2;
    if (out_kappa) out_kappa[i] = r.kappa;
  }
  return 0;
}

// Ward-identity probe: eps of photon `photon` (0 = incoming) replaced by its
// four-momentum; returns per point the max over spin configurations of
// |sum_sigma A| / sum_sigma |A| (zero up to rounding when the identity holds).
int oracle_ward(int k, long long npts, const double* momenta, int photon, int sum_mask,
                const int* hel, double mass, double* out_ratio) {
  Options opt;
  if (!valid_options(k, sum_mask, hel, opt) || photon < 0 || photon > k || !out_ratio) return -1;
  opt.ward_photon = photon;
  const int stride = (k + 3) * 4;
#pragma omp parallel for schedule(dynamic, 1)
  for (long long i = 0; i < npts; ++i) {
    Process<double> P;
    load_process(P, k, momenta + i * stride, mass);
    out_ratio[i] = evaluate_point(P, opt).ward_ratio;
  }
  return 0;
}

// Per-diagram amplitudes A_sigma for one point and one fully fixed spin
// configuration hel[k+3]; diagrams in lexicographic order of the photon
// permutation (photon 0 = incoming).  out_re/out_im have (k+1)! entries.
int oracle_amplitudes(int k, const double* momenta, const int* hel, double mass,
                      double* out_re, double* out_im) {
  Options opt;
  if (!valid_options(k, 0, hel, opt) || !out_re || !out_im) return -1;
  Process<double> P;
  load_process(P, k, momenta, mass);
  const int n = P.n;
  Vec4<double> u = spinor_u(P.p_in, opt.hel[0], P.m);
  Vec4<double> ubar = spinor_ubar(P.p_out, opt.hel[2], P.m);
  Mat4<double> epsl[8];
  for (int j = 0; j < n; ++j) {
    double e[4];
    polarisation(P.kph[j], opt.hel[photon_slot(j)], e);
    epsl[j] = slash(e);
  }
  std::vector<int> perm(n);
  for (int j = 0; j < n; ++j) perm[j] = j;
  long long d = 0;
  do {
    Vec4<double> v = u;
    unsigned mask = 0;
    for (int i = 0; i < n; ++i) {
      v = matvec(epsl[perm[i]], v);
      mask |= 1u << perm[i];
      if (i + 1 < n) {
        double Q[4];
        momentum_of_set(P, mask, Q);
        v = matvec(propagator(Q, P.m), v);
      }
    }
    Cx<double> A;
    for (int c = 0; c < 4; ++c) A = A + ubar.c[c] * v.c[c];
    out_re[d] = A.re;
    out_im[d] = A.im;
    ++d;
  } while (std::next_permutation(perm.begin(), perm.end()));
  return 0;
}

// Gradient of |M|^2 with respect to the 3-momenta of the k outgoing photons
// (slots 3..k+2), their energies taken on shell, E_j = |k_j|; every other
// momentum held fixed.  Forward-mode dual numbers, one direction at a time.
// out_grad[npts][k][3]; out_m2 (may be NULL) receives the value.
int oracle_grad(int k, long long npts, const double* momenta, int sum_mask, const int* hel,
                double mass, double* out_m2, double* out_grad) {
  Options opt;
  if (!valid_options(k, sum_mask, hel, opt) || !out_grad) return -1;
  const int stride = (k + 3) * 4;
  const int ndir = 3 * k;
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
  for (long long i = 0; i < npts; ++i) {
    for (int dir = 0; dir < ndir; ++dir) {
      Process<Dual> P;
      load_process(P, k, momenta + i * stride, mass);
      int j = 1 + dir / 3, comp = dir % 3;
      for (int jj = 1; jj <= k; ++jj) {
        Dual kx = P.kph[jj][1], ky = P.kph[jj][2], kz = P.kph[jj][3];
        if (jj == j) {
          if (comp == 0) kx.d = 1.0;
          if (comp == 1) ky.d = 1.0;
          if (comp == 2) kz.d = 1.0;
        }
        P.kph[jj][1] = kx; P.kph[jj][2] = ky; P.kph[jj][3] = kz;
        P.kph[jj][0] = sqrt_(kx * kx + ky * ky + kz * kz);
      }
      PointResult<Dual> r = evaluate_point(P, opt);
      out_grad[(i * k + (j - 1)) * 3 + comp] = r.m2.d;
      if (out_m2 && dir == 0) out_m2[i] = r.m2.v;
    }
  }
  return 0;
}

// External states, exposed so that tests can check them against the Dirac
// equation and the textbook completeness relations.
// out[8] = (re, im) of the 4 components.
int oracle_spinor(const double* p, int h, double mass, int bar, double* out) {
  if (h != 1 && h != -1) return -1;
  Vec4<double> u = bar ? spinor_ubar(p, h, mass) : spinor_u(p, h, mass);
  for (int c = 0; c < 4; ++c) { out[2 * c] = u.c[c].re; out[2 * c + 1] = u.c[c].im; }
  return 0;
}
int oracle_polarisation(const double* k, int pol, double* out) {
  if (pol != 1 && pol != 2) return -1;
  polarisation(k, pol, out);
  return 0;
}
// Explicit gamma^mu (mu = 0..3) as 4x4 complex, out[32] row-major (re, im).
int oracle_gamma(int mu, double* out) {
  if (mu < 0 || mu > 3) return -1;
  const Gammas& G = gammas();
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      out[2 * (4 * i + j)] = G.g[mu].m[i][j].re;
      out[2 * (4 * i + j) + 1] = G.g[mu].m[i][j].im;
    }
  return 0;
}

}  // extern "C"

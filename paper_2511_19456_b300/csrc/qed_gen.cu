// Device-side phase-space generation and Monte Carlo cross sections: the
// step before the |M|^2 path.  A Monte Carlo event generator samples points
// and integrates sum|M|^2 over phase space.
//
// Points follow the same recipe and the same counter-based random draws as
// the host generator (paper_2511_19456_b300/phasespace.py), one point per
// thread in FP64:
//   * k = 1: flat two-body phase space, uniform cos(theta*) and phi* in the CM
//     frame (draws 2i, 2i+1 of the stream);
//   * k >= 2: RAMBO (Kleiss, Stirling, Ellis 1986) with draws
//     4 (i nf + j) + c for particle j, component c: massless CM momenta,
//     rescaled for the electron mass by Newton's method;
// then boosted to the lab (e- at rest, photon along +z with energy omega), with
// final-state energies set on shell from the 3-momenta.
//
// Weights (phase-space density, (2 pi)^4 delta^4 prod d^3p / ((2 pi)^3 2E)):
// the massless RAMBO weight (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!)
// times the massive factor (sum|p|/sqrt s)^(2n-3) prod(|p|/E) sqrt s / sum(|p|^2/E),
// which for two bodies is |p*| / (4 pi sqrt s).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "qed_plan.hpp"

namespace qed {
namespace {

__device__ __forceinline__ double uniform53(unsigned long long seed, unsigned long long idx, bool open_zero) {
  unsigned long long z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  double u = (double)(z >> 11);
  if (open_zero) u += 1.0;
  return u * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void lab_boost(double beta, double g, double* p) {
  const double e = g * (p[0] + beta * p[3]);
  const double z = g * (p[3] + beta * p[0]);
  p[0] = e;
  p[3] = z;
}

template <int NF>
__device__ void rambo_point(unsigned long long seed, long long i, double rs, double mass, double* fin,
                            double* w_factor) {
  double q[NF][4];
  double Q[4] = {0, 0, 0, 0};
  for (int j = 0; j < NF; ++j) {
    const unsigned long long b = 4ull * ((unsigned long long)i * NF + j);
    const double r0 = uniform53(seed, b, true), r1 = uniform53(seed, b + 1, true);
    const double r2 = uniform53(seed, b + 2, true), r3 = uniform53(seed, b + 3, true);
    const double c = 2.0 * r0 - 1.0;
    const double phi = 2.0 * M_PI * r1;
    const double q0 = -log(r2 * r3);
    const double st = sqrt(fmax(0.0, (1.0 - c) * (1.0 + c)));
    double sp, cp;
    sincos(phi, &sp, &cp);
    q[j][0] = q0; q[j][1] = q0 * st * cp; q[j][2] = q0 * st * sp; q[j][3] = q0 * c;
    for (int m = 0; m < 4; ++m) Q[m] += q[j][m];
  }
  const double M = sqrt(Q[0] * Q[0] - (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]));
  const double b1 = -Q[1] / M, b2 = -Q[2] / M, b3 = -Q[3] / M;
  const double x = rs / M, gam = Q[0] / M, a = 1.0 / (1.0 + gam);
  double en[NF];
  for (int j = 0; j < NF; ++j) {
    const double bq = b1 * q[j][1] + b2 * q[j][2] + b3 * q[j][3];
    en[j] = x * (gam * q[j][0] + bq);
    fin[4 * j + 1] = x * (q[j][1] + b1 * q[j][0] + a * bq * b1);
    fin[4 * j + 2] = x * (q[j][2] + b2 * q[j][0] + a * bq * b2);
    fin[4 * j + 3] = x * (q[j][3] + b3 * q[j][0] + a * bq * b3);
  }
  // massive rescaling, particle 0 is the electron
  double xi = sqrt(fmax(0.0, 1.0 - (mass / rs) * (mass / rs)));
  for (int it = 0; it < 40; ++it) {
    double f = -rs, fp = 0.0;
    for (int j = 0; j < NF; ++j) {
      const double mj = j == 0 ? mass : 0.0;
      const double e = sqrt(mj * mj + (xi * en[j]) * (xi * en[j]));
      f += e;
      fp += xi * en[j] * en[j] / e;
    }
    const double step = f / fp;
    xi -= step;
    if (!(fabs(step) > 4e-16 * fabs(xi + step))) break;
  }
  double sum_p = 0.0, prod = 1.0, sum_p2e = 0.0;
  for (int j = 0; j < NF; ++j) {
    const double mj = j == 0 ? mass : 0.0;
    for (int m = 1; m < 4; ++m) fin[4 * j + m] *= xi;
    const double pa = xi * en[j];
    const double e = sqrt(mj * mj + pa * pa);
    fin[4 * j] = e;
    sum_p += pa;
    prod *= pa / e;
    sum_p2e += pa * pa / e;
  }
  *w_factor = pow(sum_p / rs, 2 * NF - 3) * prod * rs / sum_p2e;
}

template <int K>
__global__ void __launch_bounds__(128)
qed_gen_kernel(double omega, double mass, unsigned long long seed, long long offset, long long n,
               double* __restrict__ mom, double* __restrict__ weight) {
  constexpr int NF = K + 1;
  constexpr int NS = K + 3;
  const double s = mass * mass + 2.0 * mass * omega;
  const double rs = sqrt(s);
  const double beta = omega / (mass + omega);
  const double g = 1.0 / sqrt((1.0 - beta) * (1.0 + beta));
  double w0 = 1.0;  // massless RAMBO weight
  {
    double f1 = 1.0, f2 = 1.0;
    for (int i = 2; i <= NF - 1; ++i) f1 *= i;
    for (int i = 2; i <= NF - 2; ++i) f2 *= i;
    w0 = pow(2.0 * M_PI, 4 - 3 * NF) * pow(M_PI / 2.0, NF - 1) * pow(s, NF - 2) / (f1 * f2);
  }
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = offset + t;
    double fin[4 * NF];
    double wf;
    if constexpr (K == 1) {
      const double e_gam = (s - mass * mass) / (2.0 * rs);
      const double u0 = uniform53(seed, 2ull * (unsigned long long)i, false);
      const double u1 = uniform53(seed, 2ull * (unsigned long long)i + 1, false);
      const double cth = 2.0 * u0 - 1.0;
      const double phi = 2.0 * M_PI * u1;
      const double sth = sqrt(fmax(0.0, (1.0 - cth) * (1.0 + cth)));
      double sp, cp;
      sincos(phi, &sp, &cp);
      fin[4] = e_gam; fin[5] = e_gam * sth * cp; fin[6] = e_gam * sth * sp; fin[7] = e_gam * cth;
      fin[0] = sqrt(mass * mass + e_gam * e_gam);
      fin[1] = -fin[5]; fin[2] = -fin[6]; fin[3] = -fin[7];
      wf = 2.0 * e_gam / rs;  // two-body: massive factor = 2|p*|/sqrt s
    } else {
      rambo_point<NF>(seed, i, rs, mass, fin, &wf);
    }
    double* out = mom + t * (NS * 4);
    out[0] = mass; out[1] = 0.0; out[2] = 0.0; out[3] = 0.0;
    out[4] = omega; out[5] = 0.0; out[6] = 0.0; out[7] = omega;
    for (int j = 0; j < NF; ++j) {
      double p[4] = {fin[4 * j], fin[4 * j + 1], fin[4 * j + 2], fin[4 * j + 3]};
      lab_boost(beta, g, p);
      const double mj = j == 0 ? mass : 0.0;
      p[0] = sqrt(mj * mj + (p[1] * p[1] + p[2] * p[2] + p[3] * p[3]));
      double* o = out + 4 * (2 + j);
      o[0] = p[0]; o[1] = p[1]; o[2] = p[2]; o[3] = p[3];
    }
    if (weight) weight[t] = w0 * wf;
  }
}

// acc[0] += sum w m2, acc[1] += sum (w m2)^2
__global__ void __launch_bounds__(256)
qed_wsum_kernel(const double* __restrict__ w, const double* __restrict__ m2, long long n, double* acc) {
  double s1 = 0.0, s2 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = w[i] * m2[i];
    s1 += v;
    s2 += v * v;
  }
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  __shared__ double red[2][8];
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][wid] = s1; red[1][wid] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[0][i]; b += red[1][i]; }
    atomicAdd(acc, a);
    atomicAdd(acc + 1, b);
  }
}

using GenFn = void (*)(double, double, unsigned long long, long long, long long, double*, double*);

GenFn gen_fn(int k) {
  switch (k) {
    case 1: return qed_gen_kernel<1>;
    case 2: return qed_gen_kernel<2>;
    case 3: return qed_gen_kernel<3>;
    case 4: return qed_gen_kernel<4>;
    case 5: return qed_gen_kernel<5>;
    case 6: return qed_gen_kernel<6>;
    case 7: return qed_gen_kernel<7>;
    default: return nullptr;
  }
}

int grid_for(long long n, int block) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long need = (n + block - 1) / block;
  return (int)std::min<long long>(need, (long long)std::max(1, sms) * 16);
}

}  // namespace
}  // namespace qed

using namespace qed;

extern "C" {

qed_status qed_generate(int k, double omega, double mass, unsigned long long seed, long long offset,
                        long long n, double* d_momenta, double* d_weight, void* stream) {
  if (k < 1 || k > 7 || !(omega > 0.0) || !(mass > 0.0) || offset < 0 || n < 0) return QED_EINVAL;
  if (n == 0) return QED_OK;
  if (!d_momenta || ((uintptr_t)d_momenta & 7u) || ((uintptr_t)d_weight & 7u)) return QED_EINVAL;
  GenFn fn = gen_fn(k);
  fn<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(omega, mass, seed, offset, n, d_momenta, d_weight);
  return cuda_status(cudaGetLastError());
}

qed_status qed_cross_section(qed_plan_t plan, double omega, unsigned long long seed, long long offset,
                             long long n, long long chunk, double* d_momenta, double* d_weight,
                             double* d_m2, double* d_acc, void* stream, double* sigma, double* sigma_err,
                             double* sum_wm2, double* sum_wm2_sq) {
  if (!plan || !plan->summed || !(omega > 0.0) || n < 1 || chunk < 1 || offset < 0) return QED_EINVAL;
  if (!d_momenta || !d_weight || !d_m2 || !d_acc) return QED_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(d_acc, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return cuda_status(e);
  for (long long o = 0; o < n; o += chunk) {
    const long long m = std::min(chunk, n - o);
    qed_status s = qed_generate(plan->k, omega, plan->mass, seed, offset + o, m, d_momenta, d_weight, stream);
    if (s != QED_OK) return s;
    s = qed_eval(plan, d_momenta, m, d_m2, stream);
    if (s != QED_OK) return s;
    qed_wsum_kernel<<<grid_for(m, 256), 256, 0, st>>>(d_weight, d_m2, m, d_acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
  }
  double acc[2];
  e = cudaMemcpyAsync(acc, d_acc, sizeof(acc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  // spin average 1/4, identical photons 1/k!, flux 4 m omega (e- at rest)
  double kf = 1.0;
  for (int i = 2; i <= plan->k; ++i) kf *= i;
  const double norm = 1.0 / (4.0 * plan->mass * omega) / 4.0 / kf;
  const double mean = acc[0] / (double)n;
  const double var = std::max(0.0, acc[1] / (double)n - mean * mean);
  if (sigma) *sigma = norm * mean;
  if (sigma_err) *sigma_err = norm * std::sqrt(var / (double)n);
  if (sum_wm2) *sum_wm2 = acc[0];
  if (sum_wm2_sq) *sum_wm2_sq = acc[1];
  return QED_OK;
}

}  // extern "C"

// 1D factor assembly (FP64 closed forms) and dense IC/BC Gram assembly.
//
// Sec. 3.1 (Eq. linop-simplified): an interval functional int_a^b u^(alpha)
// equals U^(alpha-1)(b) - U^(alpha-1)(a), where U^(-1) is an antiderivative of
// u.  Covariances of such "atoms" under the unit-scale Matern-5/2 kernel are
//   cov(d^m u(x), d^n u(x')) = (-1)^n k^(m+n)(x - x'),
// with k^(-1) = K1 (K1' = k, K1(0) = 0) and k^(-2) = K2 (K2'' = k, K2(0) = 0).
// With s = sqrt(5)/ell and z = s|r| (closed forms derived for q = 2):
//   k    = (1 + z + z^2/3) e^-z
//   k'   = -sgn(r) s z (1 + z)/3 e^-z
//   k''  = -s^2 (1 + z - z^2)/3 e^-z
//   k''' = sgn(r) s^3 z (3 - z)/3 e^-z       (collocation of second-order operators only)
//   k''''= s^4 (3 - 5z + z^2)/3 e^-z
//   s K1 = sgn(r) [8/3 - (8/3 + 5z/3 + z^2/3) e^-z]
//   s^2 K2 = 8z/3 - 5 + (5 + 7z/3 + z^2/3) e^-z
// Evaluation rules that keep every entry accurate relative to its own size:
//   * if every atom separation of an entry has z < 1, the Taylor series of
//     s K1 / sgn(r) and s^2 K2 are summed (no 5 - 5 or 8/3 - 8/3 cancellation);
//   * otherwise the polynomial parts are summed apart from the exponential
//     parts; for K1 the polynomial part is an exact integer multiple of 8/3,
//     for K2 it cancels exactly when all separations share one sign (atom
//     weights of an interval sum to zero), so it is dropped in that case.
#include "common.cuh"
#include "kernels.cuh"

namespace gpfvm {

__device__ __forceinline__ double sgnd(double r) { return (r > 0.0) - (r < 0.0); }

// s*K1(r)/sgn(r) for small z: sum_{k>=1} (-1)^(k+1) (k-2)(k-4)/(3 k!) z^k
__device__ double k1_series(double z) {
  double t = 1.0, acc = 0.0;
  for (int k = 1; k < 24; ++k) {
    t *= z / (double)k;
    const double c = (double)((k - 2) * (k - 4)) * (1.0 / 3.0);
    acc += (k & 1) ? c * t : -c * t;
  }
  return acc;
}

// s^2*K2(r) for small z: sum_{k>=2} (-1)^k (k-3)(k-5)/(3 k!) z^k
__device__ double k2_series(double z) {
  double t = z, acc = 0.0;  // t = z^k / k! starting at k = 1
  for (int k = 2; k < 24; ++k) {
    t *= z / (double)k;
    const double c = (double)((k - 3) * (k - 5)) * (1.0 / 3.0);
    acc += (k & 1) ? -c * t : c * t;
  }
  return acc;
}

// Covariance of entry (i, j) of a 1D factor job.
__device__ double factor_entry(const FactorJob& J, int i, int j) {
  double xa[2], wa[2], xb[2], wb[2];
  int na, nb, ma, mb;
  if (J.kind_a == 0) {
    xa[0] = J.ca[i + 1]; wa[0] = 1.0; xa[1] = J.ca[i]; wa[1] = -1.0; na = 2; ma = J.ord_a - 1;
  } else {
    xa[0] = J.ca[i]; wa[0] = 1.0; na = 1; ma = (J.has2_a && i == 1) ? J.ord2_a : J.ord_a;
  }
  if (J.kind_b == 0) {
    xb[0] = J.cb[j + 1]; wb[0] = 1.0; xb[1] = J.cb[j]; wb[1] = -1.0; nb = 2; mb = J.ord_b - 1;
  } else {
    xb[0] = J.cb[j]; wb[0] = 1.0; nb = 1; mb = (J.has2_b && j == 1) ? J.ord2_b : J.ord_b;
  }
  const int order = ma + mb;
  const double sign_n = (mb & 1) ? -1.0 : 1.0;  // (-1)^n, n may be -1
  const double s = 2.2360679774997896964 / J.ell;

  if (order >= 0) {
    double acc = 0.0;
    for (int a = 0; a < na; ++a)
      for (int b = 0; b < nb; ++b) {
        const double r = xa[a] - xb[b];
        const double z = s * fabs(r);
        const double e = exp(-z);
        double kv;
        if (order == 0) kv = (1.0 + z + z * z * (1.0 / 3.0)) * e;
        else if (order == 1) kv = -sgnd(r) * s * z * (1.0 + z) * (1.0 / 3.0) * e;
        else if (order == 2) kv = -s * s * (1.0 + z - z * z) * (1.0 / 3.0) * e;
        else if (order == 3) kv = sgnd(r) * s * s * s * z * (3.0 - z) * (1.0 / 3.0) * e;
        else kv = s * s * s * s * (3.0 - 5.0 * z + z * z) * (1.0 / 3.0) * e;
        acc += wa[a] * wb[b] * sign_n * kv;
      }
    return acc;
  }
  double zmax = 0.0;
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < nb; ++b) zmax = fmax(zmax, s * fabs(xa[a] - xb[b]));
  const bool near = zmax < 1.0;
  if (order == -1) {
    double series = 0.0, ipart = 0.0, epart = 0.0;
    for (int a = 0; a < na; ++a)
      for (int b = 0; b < nb; ++b) {
        const double r = xa[a] - xb[b];
        const double z = s * fabs(r);
        const double w = wa[a] * wb[b] * sign_n * sgnd(r);
        if (near) {
          series += w * k1_series(z);
        } else {
          ipart += w;
          epart -= w * (8.0 / 3.0 + z * (5.0 / 3.0) + z * z * (1.0 / 3.0)) * exp(-z);
        }
      }
    return near ? series / s : (ipart * (8.0 / 3.0) + epart) / s;
  }
  // order == -2: integral x integral
  double series = 0.0, lin = 0.0, epart = 0.0;
  bool all_pos = true, all_neg = true;
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < nb; ++b) {
      const double r = xa[a] - xb[b];
      const double z = s * fabs(r);
      const double w = wa[a] * wb[b] * sign_n;
      all_pos = all_pos && (r >= 0.0);
      all_neg = all_neg && (r <= 0.0);
      if (near) {
        series += w * k2_series(z);
      } else {
        lin += w * (z * (8.0 / 3.0) - 5.0);
        epart += w * (5.0 + z * (7.0 / 3.0) + z * z * (1.0 / 3.0)) * exp(-z);
      }
    }
  if (near) return series / (s * s);
  return ((all_pos || all_neg) ? epart : lin + epart) / (s * s);
}

__global__ void factor_kernel(const FactorJob* __restrict__ jobs) {
  const FactorJob J = jobs[blockIdx.y];
  const i64 total = (i64)J.n_a * J.n_b;
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(e / J.n_b), j = (int)(e % J.n_b);
    J.out[e] = factor_entry(J, i, j);
  }
}

void launch_factors(const FactorJob* d_jobs, int n_jobs, i64 max_entries, cudaStream_t st) {
  if (n_jobs == 0) return;
  int gx = ceil_div(max_entries, 256);
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  dim3 grid(gx, n_jobs);
  factor_kernel<<<grid, 256, 0, st>>>(d_jobs);
  GPFVM_LAUNCH_CHECK();
}

// Dense IC/BC Gram: entry (o1, o2) of G_BB = sigma^2 prod_i D_i^{s s'}[l_i, l'_i]
// (+ noise variance on the diagonal), sets enumerated by their offsets; zero
// between sets observing different outputs of a system (Eq. multioutput-cov-def).
__global__ void gbb_kernel(GbbParams P, double* __restrict__ G) {
  const i64 M = P.M;
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < M * M; e += (i64)gridDim.x * blockDim.x) {
    const int o1 = (int)(e / M), o2 = (int)(e % M);
    int s1 = 0, s2 = 0;
    while (s1 + 1 < P.n_sets && o1 >= P.off[s1 + 1]) ++s1;
    while (s2 + 1 < P.n_sets && o2 >= P.off[s2 + 1]) ++s2;
    int l1 = o1 - P.off[s1], l2 = o2 - P.off[s2];
    double v = P.comp[s1] == P.comp[s2] ? P.outputscale : 0.0;  // outputs are a priori uncorrelated
    int i0 = 0;  // axis-0 index of point o1
    for (int ax = P.ndim - 1; ax >= 0; --ax) {
      const int n1 = P.dims[s1][ax], n2 = P.dims[s2][ax];
      const int i1 = l1 % n1, i2 = l2 % n2;
      l1 /= n1;
      l2 /= n2;
      v *= P.fac[s1][s2][ax][(i64)i1 * n2 + i2];
      i0 = i1;
    }
    if (o1 == o2) v += i0 > 0 ? P.noise2[s1] : P.noise[s1];
    G[e] = v;
  }
}

void launch_gbb(const GbbParams& P, double* G, cudaStream_t st) {
  const i64 tot = (i64)P.M * P.M;
  if (tot == 0) return;
  int g = ceil_div(tot, 256);
  if (g > 152 * 16) g = 152 * 16;
  gbb_kernel<<<g, 256, 0, st>>>(P, G);
  GPFVM_LAUNCH_CHECK();
}

}  // namespace gpfvm

// Structured IC/BC stage: the exact inverse of G_BB through the Kronecker
// structure of its largest point set.
//
// The first point set K (e.g. the initial condition on a tensor grid at
// t = 0) has the self-covariance  A = sigma^2 (D_0 (x) D_1 (x) D_2) + nu I,
// where D_i are its 1D point-point factors.  With D_i = Q_i diag(lam_i) Q_i^T,
//   A^-1 = (x)Q_i  diag(1 / (sigma^2 prod_i lam_i + nu))  (x)Q_i^T ,
// so A needs no factorisation.  The remaining sets R enter through the Schur
// complement S = G_RR - G_RK A^-1 G_KR (block elimination, exact), which is
// small (the boundary points) and factorised by the recursive Cholesky +
// inverse of chol.cu.  This file holds the kernels: a one-sided Jacobi
// eigensolver for the small symmetric factors D_i, and the eigenvalue-tensor
// scalings.
#include "kernels.cuh"

namespace gpfvm {

constexpr int JAC_MAX_N = 96;

// One-sided (Hestenes) Jacobi on a symmetric positive semidefinite n x n
// matrix: rotate column pairs of U = A V until they are orthogonal; then
// A V = U = Q diag(lam) with Q = V, lam_j = ||U_j||.  Pairs follow the
// round-robin (circle) schedule, so the n/2 rotations of a round touch
// disjoint columns (one warp per pair).  The bulk of the sweeps runs in FP32
// (the FP64 pipe of one SM is slow); V is then re-orthonormalised in FP64
// (modified Gram-Schmidt), U = A V is recomputed in FP64 and FP64 sweeps
// polish to the rounding level.  A pair counts as converged when its cosine
// is below the phase's target (about the rounding level of n-term dot
// products), or its inner product is at the rounding level of the largest
// column, |c| <= 4 eps ||A||_F (|u_p| + |u_q|), or both columns are below the
// rounding floor n eps ||A||_F of U = A V: such columns hold noise whose
// mutual angle is meaningless, and rotating them kept sweeps from converging.
// Sweeps are bounded in both phases.
// One pair per 8 lanes (4 pairs per warp): the per-pair scalar work (FP64 on
// the polish sweeps, where one SM's DFMA rate is the bound) is repeated by 8
// lanes instead of 32.  Column norms are carried in nrm[] (recomputed at
// every sweep start, updated exactly for the applied rotation), so a pair
// needs one inner product.  The angle is formed in FP32; its cosine is
// normalised in T by two Newton steps, so the applied rotation is orthogonal
// to T's rounding.  Shuffles run in warp-uniform loops.
template <typename T>
__device__ int jacobi_sweeps(T* U, T* V, T* nrm, int n, double fro, double tol_rot, double tol_abs, double noise,
                             int max_sweeps, double* maxrot, int extra = 0) {
  const int np = (n + 1) & ~1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int oct = lane >> 3, sl = lane & 7;
  const double noise2 = noise * noise * fro * fro;
  const double tol2 = tol_rot * tol_rot;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int j0 = warp * 4; j0 < n; j0 += nw * 4) {
      const int j = j0 + oct;
      T a = T(0);
      if (j < n)
        for (int i = sl; i < n; i += 8) a = fma(U[j * n + i], U[j * n + i], a);
      a += __shfl_xor_sync(0xffffffffu, a, 4);
      a += __shfl_xor_sync(0xffffffffu, a, 2);
      a += __shfl_xor_sync(0xffffffffu, a, 1);
      if (j < n && sl == 0) nrm[j] = a;
    }
    if (tid == 0) *maxrot = 0.0;
    __syncthreads();
    double local_max2 = 0.0;
    for (int r = 0; r < np - 1; ++r) {
      for (int k0 = warp * 4; k0 < np / 2; k0 += nw * 4) {
        const int k = k0 + oct;
        int p = n, q = n;
        if (k < np / 2) {
          if (k == 0) { p = r; q = np - 1; }
          else { p = (r + k) % (np - 1); q = (r - k + (np - 1)) % (np - 1); }
        }
        const bool valid = p < n && q < n;
        T c = T(0);
        if (valid)
          for (int i = sl; i < n; i += 8) c = fma(U[p * n + i], U[q * n + i], c);
        c += __shfl_xor_sync(0xffffffffu, c, 4);
        c += __shfl_xor_sync(0xffffffffu, c, 2);
        c += __shfl_xor_sync(0xffffffffu, c, 1);
        if (!valid) continue;
        const T a = nrm[p], b = nrm[q];
        const double cd = (double)c;
        if (a == T(0) || b == T(0) ||
            fabs(cd) <= tol_abs * fro * ((double)sqrtf((float)a) + (double)sqrtf((float)b)))
          continue;
        // both columns at the rounding floor of U = A V: their mutual angle is noise
        if ((double)a <= noise2 && (double)b <= noise2) continue;
        const double rot2 = cd * cd / ((double)a * (double)b);
        if (rot2 < tol2) continue;
        local_max2 = fmax(local_max2, rot2);
        const float zeta = (float)(b - a) / (2.0f * (float)c);
        const float tf = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
        const T t = (T)tf, h = T(1) + t * t;
        T cs = (T)rsqrtf((float)h);
        cs = cs * (T(1.5) - T(0.5) * h * cs * cs);
        cs = cs * (T(1.5) - T(0.5) * h * cs * cs);
        const T sn = cs * t;
        for (int i = sl; i < n; i += 8) {
          const T up = U[p * n + i], uq = U[q * n + i];
          U[p * n + i] = cs * up - sn * uq;
          U[q * n + i] = sn * up + cs * uq;
          const T vp = V[p * n + i], vq = V[q * n + i];
          V[p * n + i] = cs * vp - sn * vq;
          V[q * n + i] = sn * vp + cs * vq;
        }
        if (sl == 0) {
          const T cs2 = cs * cs, tc2 = T(2) * t * c, tt = t * t;
          nrm[p] = cs2 * (a - tc2 + tt * b);
          nrm[q] = cs2 * (b + tc2 + tt * a);
        }
      }
      __syncthreads();
    }
    double m2 = local_max2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    if (lane == 0) atomicMax((unsigned long long*)maxrot, __double_as_longlong(sqrt(m2)));
    __syncthreads();
    const bool done = *maxrot < tol_rot * 10.0;
    __syncthreads();
    if (done) {
      if (extra-- > 0) continue;  // quadratic convergence: one more sweep reaches the rounding level
      return sweep + 1;
    }
  }
  return sweep;
}

__global__ void __launch_bounds__(1024) jacobi_kernel(const JacobiJob* __restrict__ jobs) {
  extern __shared__ double sm[];
  const JacobiJob J = jobs[blockIdx.x];
  const int n = J.n;
  double* U = sm;  // FP64 column-major U[j * n + i]
  double* V = sm + n * n;
  float* Uf = (float*)(sm + 2 * n * n);
  float* Vf = Uf + n * n;
  double* nrm = sm + 3 * n * n;       // column norms of U (FP64 phase)
  float* nrmf = (float*)(nrm + n);    // ... of Uf (FP32 phase)
  __shared__ double maxrot, fro2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    const double a = 0.5 * (J.A[(i64)i * n + j] + J.A[(i64)j * n + i]);
    U[e] = a;
    Uf[e] = (float)a;
    Vf[e] = (i == j) ? 1.0f : 0.0f;
  }
  __syncthreads();
  if (tid == 0) {
    double f = 0.0;
    for (int e = 0; e < n * n; ++e) f += U[e] * U[e];
    fro2 = f;
  }
  __syncthreads();
  const double fro = sqrt(fro2);
  // phase 1: FP32 sweeps until the largest rotation of a sweep is below 1e-4
  // (FP32 dot products carry ~n * 6e-8 of rounding, so tighter targets only
  // rotate on noise); the FP64 polish converges quadratically from there
  const int sw32 = jacobi_sweeps<float>(Uf, Vf, nrmf, n, fro, 1e-5, 4e-8, n * 6e-8, 30, &maxrot);
  // re-orthonormalise V in FP64 (modified Gram-Schmidt over its columns)
  for (int e = tid; e < n * n; e += blockDim.x) V[e] = (double)Vf[e];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    // normalise column j (warp 0), then remove it from the later columns (all warps)
    if (warp == 0) {
      double s = 0.0;
      for (int i = lane; i < n; i += 32) s += V[j * n + i] * V[j * n + i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double inv = 1.0 / sqrt(s);
      for (int i = lane; i < n; i += 32) V[j * n + i] *= inv;
    }
    __syncthreads();
    for (int k = j + 1 + warp; k < n; k += nw) {
      double s = 0.0;
      for (int i = lane; i < n; i += 32) s += V[j * n + i] * V[k * n + i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      for (int i = lane; i < n; i += 32) V[k * n + i] -= s * V[j * n + i];
    }
    __syncthreads();
  }
  // U = A V in FP64 (A row-major, symmetric)
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += 0.5 * (J.A[(i64)i * n + l] + J.A[(i64)l * n + i]) * V[j * n + l];
    U[e] = s;
  }
  __syncthreads();
  // phase 2: FP64 polish: rotations down to 1e-15 are applied (eigenvectors of
  // eigenvalues near the noise term are weighted by 1/noise in G_BB^-1, so
  // their angles matter); once a sweep's largest rotation is below 1e-14
  // (reachable thanks to the noise-floor skip) one more sweep is run, which
  // takes the angles to the rounding level
  const int sw64 = jacobi_sweeps<double>(U, V, nrm, n, fro, 1e-15, 4e-16, n * 1.2e-16, 12, &maxrot, 1);
  if (J.sweeps && tid == 0) {
    J.sweeps[0] = sw32;
    J.sweeps[1] = sw64;
  }
  // eigenvalues = column norms of U, eigenvectors = columns of V
  for (int j = warp; j < n; j += nw) {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += U[j * n + i] * U[j * n + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) J.lam[j] = sqrt(s);
  }
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    J.Q[(i64)i * n + j] = V[j * n + i];  // Q row-major, column j = eigenvector j
  }
}

// U, V (FP64), Uf, Vf (FP32) and the column norms of both phases
static int jacobi_smem_bytes(int n) { return 3 * n * n * (int)sizeof(double) + n * (int)(sizeof(double) + sizeof(float)); }

void launch_jacobi(const JacobiJob* d_jobs, int n_jobs, int max_n, cudaStream_t st) {
  if (n_jobs <= 0) return;
  if (max_n > JAC_MAX_N) throw CudaError{cudaErrorInvalidValue, "jacobi: matrix too large"};
  const int smem = jacobi_smem_bytes(max_n);
  static bool attr = false;
  if (!attr) {
    GPFVM_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    jacobi_smem_bytes(JAC_MAX_N)));
    attr = true;
  }
  jacobi_kernel<<<n_jobs, 1024, smem, st>>>(d_jobs);
  GPFVM_LAUNCH_CHECK();
}

// lt[m] = sigma^2 prod_i lam_i[m_i] + nu  over the row-major multi-index m of (n0, n1, n2)
// With two stacked sets (axis 0 = two points at one coordinate, carrying the
// two sets' noise levels nu and nu_b) the noise is diag(nu, nu_b) on axis 0;
// in the eigenbasis it stays diagonal when the axis-0 factor is (the
// cross-covariance of orders 0 and 1 at one point is an odd derivative of the
// even kernel at 0, so Q0 is the identity), and its diagonal is
// sum_i Q0[i][j]^2 nu_i.
__global__ void k_lambda_tensor(const double* l0, const double* l1, const double* l2, int n0, int n1, int n2,
                                double s2, double nu, const double* __restrict__ q0, double nu_b,
                                double* __restrict__ lt) {
  const i64 tot = (i64)n0 * n1 * n2;
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (i64)gridDim.x * blockDim.x) {
    const int i2 = (int)(e % n2), i1 = (int)((e / n2) % n1), i0 = (int)(e / ((i64)n1 * n2));
    const double nz = q0 ? nu * q0[i0] * q0[i0] + nu_b * q0[n0 + i0] * q0[n0 + i0] : nu;
    lt[e] = s2 * (l0 ? l0[i0] : 1.0) * (l1 ? l1[i1] : 1.0) * (l2 ? l2[i2] : 1.0) + nz;
  }
}
void lambda_tensor(const double* l0, const double* l1, const double* l2, int n0, int n1, int n2, double s2, double nu,
                   const double* q0, double nu_b, double* lt, cudaStream_t st) {
  if (q0 && n0 != 2) throw CudaError{cudaErrorInvalidValue, "lambda_tensor: a stacked axis has two points"};
  const i64 tot = (i64)n0 * n1 * n2;
  int g = ceil_div(tot, 256);
  if (g > 2048) g = 2048;
  k_lambda_tensor<<<g, 256, 0, st>>>(l0, l1, l2, n0, n1, n2, s2, nu, q0, nu_b, lt);
  GPFVM_LAUNCH_CHECK();
}

// E~ = G_RK (x)Q Lambda~^-1 from its Kronecker structure: G_RK between set s
// and set 0 is sigma^2 (x)_i F_i(s, 0), so E~[r][m] = sigma^2 prod_i
// C_i[s](r_i, m_i) / lt[m] with C_i[s] = F_i(s, 0) Q_i (n_{s,i} x nK_i).
__global__ void k_etilde(EtildeSets S, int nk0, int nk1, int nk2, double s2, const double* __restrict__ ltinv,
                         double* __restrict__ Et, int MR) {
  const i64 MK = (i64)nk0 * nk1 * nk2;
  const i64 tot = (i64)MR * MK;
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (i64)gridDim.x * blockDim.x) {
    const int r = (int)(e / MK);
    const int m = (int)(e - (i64)r * MK);
    int s = 0;
    while (s + 1 < S.ns && S.off[s + 1] <= r) ++s;
    const int rl = r - S.off[s];
    const int r2 = rl % S.n[s][2], r01 = rl / S.n[s][2], r1 = r01 % S.n[s][1], r0 = r01 / S.n[s][1];
    const int m2 = m % nk2, m01 = m / nk2, m1 = m01 % nk1, m0 = m01 / nk1;
    double v = s2 * S.c[s][0][r0 * nk0 + m0];
    if (S.c[s][1]) v *= S.c[s][1][r1 * nk1 + m1];
    if (S.c[s][2]) v *= S.c[s][2][r2 * nk2 + m2];
    Et[e] = v * ltinv[m];
  }
}
void etilde(const EtildeSets& S, int nk0, int nk1, int nk2, double s2, const double* ltinv, double* Et, int MR,
            cudaStream_t st) {
  const i64 tot = (i64)MR * nk0 * nk1 * nk2;
  if (tot <= 0) return;
  int g = ceil_div(tot, 256);
  if (g > 8192) g = 8192;
  k_etilde<<<g, 256, 0, st>>>(S, nk0, nk1, nk2, s2, ltinv, Et, MR);
  GPFVM_LAUNCH_CHECK();
}

// D[r ldd + c] += alpha S[r lds + c] for r < rows, c < cols
__global__ void k_axpy_block(double* __restrict__ D, i64 ldd, const double* __restrict__ S, i64 lds, int rows,
                             int cols, double alpha) {
  const i64 tot = (i64)rows * cols;
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (i64)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e - (i64)r * cols);
    D[r * ldd + c] += alpha * S[r * lds + c];
  }
}
void axpy_block(double* D, i64 ldd, const double* S, i64 lds, int rows, int cols, double alpha, cudaStream_t st) {
  const i64 tot = (i64)rows * cols;
  if (tot <= 0) return;
  int g = ceil_div(tot, 256);
  if (g > 8192) g = 8192;
  k_axpy_block<<<g, 256, 0, st>>>(D, ldd, S, lds, rows, cols, alpha);
  GPFVM_LAUNCH_CHECK();
}

// out[m] = 1/lt[m] (the weight tensor of the A^-1 quadratic form)
__global__ void k_recip(const double* __restrict__ lt, double* __restrict__ out, i64 n) {
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x)
    out[e] = 1.0 / lt[e];
}
void recip(const double* lt, double* out, i64 n, cudaStream_t st) {
  if (n <= 0) return;
  int g = ceil_div(n, 256);
  if (g > 2048) g = 2048;
  k_recip<<<g, 256, 0, st>>>(lt, out, n);
  GPFVM_LAUNCH_CHECK();
}

// out[i][j] = in[i][j]^2 (squared factors for the A^-1 quadratic form on the grid)
__global__ void k_square(const double* __restrict__ in, double* __restrict__ out, i64 n) {
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x)
    out[e] = in[e] * in[e];
}
void square(const double* in, double* out, i64 n, cudaStream_t st) {
  if (n <= 0) return;
  int g = ceil_div(n, 256);
  if (g > 2048) g = 2048;
  k_square<<<g, 256, 0, st>>>(in, out, n);
  GPFVM_LAUNCH_CHECK();
}

}  // namespace gpfvm

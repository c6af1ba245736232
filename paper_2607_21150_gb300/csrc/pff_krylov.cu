// Krylov vector kernels (FP64 inner products), precision conversions and the
// assembled coarse (Q1) operator of the p-multigrid hierarchy.
#include "pff_internal.h"

namespace pff {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = kReduceBlocks;

// ---------------------------------------------------------------- reductions
// partial[j * kRedBlocks + b] = block b's share of sum_i V_j[i] w[i], j < k.
template <typename TV, typename T>
__global__ void __launch_bounds__(kRedThreads) k_mdot_partial(const TV* __restrict__ V, long long ldv, int k,
                                                              const T* __restrict__ w, long long n,
                                                              double* __restrict__ partial) {
  __shared__ double red[kRedThreads / 32];
  for (int j = 0; j < k; ++j) {
    const TV* v = V + j * ldv;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      s += (double)v[i] * (double)w[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = (threadIdx.x < kRedThreads / 32) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) partial[j * kRedBlocks + blockIdx.x] = t;
    }
    __syncthreads();
  }
}
// out[j] = sum_b partial[j * kRedBlocks + b] (one block per j, fixed order).
__global__ void k_mdot_final(const double* __restrict__ partial, int k, double* __restrict__ out) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) s += partial[j * kRedBlocks + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (int)(blockDim.x / 32)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) out[j] = t;
  }
}

template <typename TV, typename T>
cudaError_t launch_mdot(const TV* V, long long ldv, int k, const T* w, long long n, double* partial, double* out,
                        cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  k_mdot_partial<TV, T><<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, k, w, n, partial);
  k_mdot_final<<<k, 256, 0, st>>>(partial, k, out);
  return cudaGetLastError();
}
template cudaError_t launch_mdot<double, double>(const double*, long long, int, const double*, long long, double*,
                                                 double*, cudaStream_t);
template cudaError_t launch_mdot<float, float>(const float*, long long, int, const float*, long long, double*,
                                               double*, cudaStream_t);

// ---------------------------------------------------------------- vector updates
// w -= sum_j h[j] V_j   (h on the device, k <= 64)
__global__ void k_maxpy(double* __restrict__ w, const double* __restrict__ V, long long ldv, int k,
                        const double* __restrict__ h, double sign, long long n) {
  __shared__ double hs[64];
  if (threadIdx.x < k) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int j = 0; j < k; ++j) s += sign * hs[j] * V[j * ldv + i];
    w[i] = s;
  }
}
cudaError_t launch_maxpy(double* w, const double* V, long long ldv, int k, const double* h, double sign, long long n,
                         cudaStream_t st) {
  if (k <= 0 || n == 0) return cudaSuccess;
  k_maxpy<<<kRedBlocks * 2, 256, 0, st>>>(w, V, ldv, k, h, sign, n);
  return cudaGetLastError();
}

// y = a x + b y
template <typename T>
__global__ void k_axpby(T* __restrict__ y, const T* __restrict__ x, double a, double b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (T)(a * (double)x[i] + b * (double)y[i]);
}
template <typename T>
cudaError_t launch_axpby(T* y, const T* x, double a, double b, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_axpby<T><<<kRedBlocks * 2, 256, 0, st>>>(y, x, a, b, n);
  return cudaGetLastError();
}
template cudaError_t launch_axpby<double>(double*, const double*, double, double, long long, cudaStream_t);
template cudaError_t launch_axpby<float>(float*, const float*, double, double, long long, cudaStream_t);

// y = (b - y) elementwise (residual from y = A x)
template <typename T>
__global__ void k_bminus(T* __restrict__ y, const T* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = b[i] - y[i];
}
template <typename T>
cudaError_t launch_bminus(T* y, const T* b, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_bminus<T><<<kRedBlocks * 2, 256, 0, st>>>(y, b, n);
  return cudaGetLastError();
}
template cudaError_t launch_bminus<double>(double*, const double*, long long, cudaStream_t);
template cudaError_t launch_bminus<float>(float*, const float*, long long, cudaStream_t);

// y = x / d elementwise
template <typename T>
__global__ void k_dscale(T* __restrict__ y, const T* __restrict__ x, const T* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] / d[i];
}
template <typename T>
cudaError_t launch_dscale(T* y, const T* x, const T* d, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_dscale<T><<<kRedBlocks * 2, 256, 0, st>>>(y, x, d, n);
  return cudaGetLastError();
}
template cudaError_t launch_dscale<double>(double*, const double*, const double*, long long, cudaStream_t);
template cudaError_t launch_dscale<float>(float*, const float*, const float*, long long, cudaStream_t);

template <typename A, typename B>
__global__ void k_convert(B* __restrict__ y, const A* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (B)x[i];
}
cudaError_t launch_d2f(float* y, const double* x, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_convert<double, float><<<kRedBlocks * 2, 256, 0, st>>>(y, x, n);
  return cudaGetLastError();
}
cudaError_t launch_f2d(double* y, const float* x, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_convert<float, double><<<kRedBlocks * 2, 256, 0, st>>>(y, x, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Q1 coarse operator
// Assembled Q1 operator at the fine Gauss points (coarse Lagrange basis of
// order 1 evaluated at the fine points, fine stored tangent): the exact
// Galerkin operator of the p-hierarchy.  Storage: 27-point stencil with a 4x4
// block per neighbour, A[(slot*16 + f*4 + g) * nn + node], slot = neighbour
// offset (dx+1) + 3 (dy+1) + 9 (dz+1).  One thread block per element.
//
// Per point, with the 67 stored words W (already scaled by w det J and the
// parent factors) and the parent gradients dN_alpha(a) of the 8 vertex functions:
//   K[f a][g b] += sum_{alpha,beta} dN_alpha(a) W_A[f alpha][g beta] dN_beta(b)      (f, g < 3)
//   K[f a][3 b] += sum_alpha dN_alpha(a) W_P[f alpha] N(b)
//   K[3 a][g b] += N(a) sum_beta W_C[g beta] dN_beta(b)
//   K[3 a][3 b] += W_D N(a) N(b) + sum_alpha W_K[alpha] dN_alpha(a) dN_alpha(b)
constexpr int kAsmThreads = 128;

__global__ void __launch_bounds__(kAsmThreads)
k_q1_assemble(MeshDev mc, int Q, const double* __restrict__ lin, const double* __restrict__ B1,
              const double* __restrict__ D1, const uint8_t* __restrict__ maskc, double* __restrict__ A) {
  __shared__ double W[kLinWords];
  __shared__ double Nv[8], dN[3][8];
  __shared__ double T[9][3][8];  // T[f alpha][g][b] = sum_beta W_A[f alpha][g beta] dN_beta(b)
  const int e = blockIdx.x;
  const int t = threadIdx.x;
  const int EB = elems_per_block(Q);
  const int Q2 = Q * Q, Q3 = Q2 * Q;
  const long long stride = (long long)Q3 * EB;
  const long long base = (long long)(e / EB) * kLinWords * stride + (e % EB) * Q2;
  double acc[8];
  for (int s = 0; s < 8; ++s) acc[s] = 0.0;
  for (int q = 0; q < Q3; ++q) {
    const int i = q % Q, j = (q / Q) % Q, k = q / Q2;
    if (t < kLinWords) W[t] = lin[base + (long long)t * stride + (long long)k * Q2 * EB + j * Q + i];
    if (t < 8) {
      const int a0 = t & 1, a1 = (t >> 1) & 1, a2 = t >> 2;
      const double bx = B1[i * 2 + a0], by = B1[j * 2 + a1], bz = B1[k * 2 + a2];
      Nv[t] = bx * by * bz;
      dN[0][t] = D1[i * 2 + a0] * by * bz;
      dN[1][t] = bx * D1[j * 2 + a1] * bz;
      dN[2][t] = bx * by * D1[k * 2 + a2];
    }
    __syncthreads();
    for (int idx = t; idx < 9 * 3 * 8; idx += kAsmThreads) {
      const int m = idx / 24, g = (idx / 8) % 3, b = idx % 8;
      double s = 0.0;
      for (int be = 0; be < 3; ++be) {
        const int n = 3 * g + be;
        s += W[kWA + (m <= n ? sym9(m, n) : sym9(n, m))] * dN[be][b];
      }
      T[m][g][b] = s;
    }
    __syncthreads();
    for (int s = 0; s < 8; ++s) {
      const int idx = t + s * kAsmThreads;  // entry (f a, g b) of the 32 x 32 element matrix
      const int row = idx / 32, col = idx % 32;
      const int f = row / 8, a = row % 8, g = col / 8, b = col % 8;
      double v = 0.0;
      if (f < 3 && g < 3) {
        for (int al = 0; al < 3; ++al) v += dN[al][a] * T[3 * f + al][g][b];
      } else if (f < 3) {
        for (int al = 0; al < 3; ++al) v += dN[al][a] * W[kWP + 3 * f + al];
        v *= Nv[b];
      } else if (g < 3) {
        for (int be = 0; be < 3; ++be) v += W[kWC + 3 * g + be] * dN[be][b];
        v *= Nv[a];
      } else {
        v = W[kWD] * Nv[a] * Nv[b];
        for (int al = 0; al < 3; ++al) v += W[kWK + al] * dN[al][a] * dN[al][b];
      }
      acc[s] += v;
    }
    __syncthreads();
  }
  const int ex = e % mc.nx, ey = (e / mc.nx) % mc.ny, ez = e / (mc.nx * mc.ny);
  for (int s = 0; s < 8; ++s) {
    const int idx = t + s * kAsmThreads;
    const int row = idx / 32, col = idx % 32;
    const int f = row / 8, a = row % 8, g = col / 8, b = col % 8;
    const int ax = ex + (a & 1), ay = ey + ((a >> 1) & 1), az = ez + (a >> 2);
    const int bx = ex + (b & 1), by = ey + ((b >> 1) & 1), bz = ez + (b >> 2);
    const long long na = ax + (long long)mc.nnx * (ay + (long long)mc.nny * az);
    const long long nb = bx + (long long)mc.nnx * (by + (long long)mc.nny * bz);
    if (maskc && (maskc[f * mc.nn + na] || maskc[g * mc.nn + nb])) continue;
    const int slot = (bx - ax + 1) + 3 * (by - ay + 1) + 9 * (bz - az + 1);
    atomicAdd(A + (long long)(slot * 16 + f * 4 + g) * mc.nn + na, acc[s]);
  }
}

// Dirichlet rows of the coarse operator: identity (slot 13 = centre, f == g).
__global__ void k_q1_mask_identity(MeshDev mc, const uint8_t* __restrict__ maskc, double* __restrict__ A) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= mc.nn) return;
  for (int f = 0; f < 4; ++f)
    if (maskc[f * mc.nn + n]) A[(long long)(13 * 16 + f * 4 + f) * mc.nn + n] = 1.0;
}

cudaError_t launch_q1_assemble(const MeshDev& mc, int Q, const double* lin, const double* B1, const double* D1,
                               const uint8_t* maskc, double* A, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(A, 0, sizeof(double) * 27 * 16 * mc.nn, st);
  if (e != cudaSuccess) return e;
  k_q1_assemble<<<mc.nel, kAsmThreads, 0, st>>>(mc, Q, lin, B1, D1, maskc, A);
  if (maskc) k_q1_mask_identity<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, maskc, A);
  return cudaGetLastError();
}

// y = A x with the stencil storage (FP64), one thread per node; also the
// diagonal when diag != nullptr.
__global__ void k_q1_spmv(MeshDev mc, const double* __restrict__ A, const double* __restrict__ x,
                          double* __restrict__ y) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= mc.nn) return;
  const int nnz_ = (int)(mc.nn / ((long long)mc.nnx * mc.nny));
  const int I = (int)(n % mc.nnx), J = (int)((n / mc.nnx) % mc.nny), K = (int)(n / ((long long)mc.nnx * mc.nny));
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int slot = 0; slot < 27; ++slot) {
    const int dx = slot % 3 - 1, dy = (slot / 3) % 3 - 1, dz = slot / 9 - 1;
    const int I2 = I + dx, J2 = J + dy, K2 = K + dz;
    if (I2 < 0 || J2 < 0 || K2 < 0 || I2 >= mc.nnx || J2 >= mc.nny || K2 >= nnz_) continue;
    const long long m = I2 + (long long)mc.nnx * (J2 + (long long)mc.nny * K2);
    double xv[4];
    for (int g = 0; g < 4; ++g) xv[g] = x[g * mc.nn + m];
    for (int f = 0; f < 4; ++f)
      for (int g = 0; g < 4; ++g) acc[f] += A[(long long)(slot * 16 + f * 4 + g) * mc.nn + n] * xv[g];
  }
  for (int f = 0; f < 4; ++f) y[f * mc.nn + n] = acc[f];
}
// y = A^T x with the stencil storage: row (g, m) of A^T gathers the entries
// A[(f, n), (g, m)] of the nodes n = m - offset(slot).
__global__ void k_q1_spmv_t(MeshDev mc, const double* __restrict__ A, const double* __restrict__ x,
                            double* __restrict__ y) {
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= mc.nn) return;
  const int nnz_ = (int)(mc.nn / ((long long)mc.nnx * mc.nny));
  const int I = (int)(m % mc.nnx), J = (int)((m / mc.nnx) % mc.nny), K = (int)(m / ((long long)mc.nnx * mc.nny));
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int slot = 0; slot < 27; ++slot) {
    const int dx = slot % 3 - 1, dy = (slot / 3) % 3 - 1, dz = slot / 9 - 1;
    const int I2 = I - dx, J2 = J - dy, K2 = K - dz;
    if (I2 < 0 || J2 < 0 || K2 < 0 || I2 >= mc.nnx || J2 >= mc.nny || K2 >= nnz_) continue;
    const long long n = I2 + (long long)mc.nnx * (J2 + (long long)mc.nny * K2);
    double xv[4];
    for (int f = 0; f < 4; ++f) xv[f] = x[f * mc.nn + n];
    for (int f = 0; f < 4; ++f)
      for (int g = 0; g < 4; ++g) acc[g] += A[(long long)(slot * 16 + f * 4 + g) * mc.nn + n] * xv[f];
  }
  for (int g = 0; g < 4; ++g) y[g * mc.nn + m] = acc[g];
}
cudaError_t launch_q1_spmv_t(const MeshDev& mc, const double* A, const double* x, double* y, cudaStream_t st) {
  k_q1_spmv_t<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, A, x, y);
  return cudaGetLastError();
}

// y = s * sel (uint8 selector to FP64), and zeroing of Dirichlet entries.
__global__ void k_sel_scale(double* __restrict__ y, const uint8_t* __restrict__ sel, double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = sel[i] ? s : 0.0;
}
__global__ void k_zero_masked(double* __restrict__ y, const uint8_t* __restrict__ mask, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (mask[i]) y[i] = 0.0;
}
cudaError_t launch_sel_scale(double* y, const uint8_t* sel, double s, long long n, cudaStream_t st) {
  k_sel_scale<<<kRedBlocks * 2, 256, 0, st>>>(y, sel, s, n);
  return cudaGetLastError();
}
cudaError_t launch_zero_masked(double* y, const uint8_t* mask, long long n, cudaStream_t st) {
  if (!mask) return cudaSuccess;
  k_zero_masked<<<kRedBlocks * 2, 256, 0, st>>>(y, mask, n);
  return cudaGetLastError();
}

__global__ void k_q1_diag(MeshDev mc, const double* __restrict__ A, double* __restrict__ d) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= mc.nn) return;
  for (int f = 0; f < 4; ++f) d[f * mc.nn + n] = A[(long long)(13 * 16 + f * 4 + f) * mc.nn + n];
}
cudaError_t launch_q1_spmv(const MeshDev& mc, const double* A, const double* x, double* y, cudaStream_t st) {
  k_q1_spmv<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, A, x, y);
  return cudaGetLastError();
}
cudaError_t launch_q1_diag(const MeshDev& mc, const double* A, double* d, cudaStream_t st) {
  k_q1_diag<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, A, d);
  return cudaGetLastError();
}

}  // namespace pff

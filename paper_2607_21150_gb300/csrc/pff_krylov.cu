// Krylov vector kernels (FP64 inner products), precision conversions, the
// assembled coarse (Q1) operator of the p-multigrid hierarchy (element
// matrices, stencil gather, SpMV and diagonal) and the geometric h-multigrid
// below it (Galerkin coarsening, masks, prolongation and restriction).
#include "pff_df.cuh"
#include "pff_internal.h"

namespace pff {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = kReduceBlocks;

// ---------------------------------------------------------------- reductions
// partial[j * kRedBlocks + b] = block b's share of sum_i V_j[i] w[i], j < k.
// Vectors are taken in chunks of CH so that w is read once per chunk (long
// vectors: HBM traffic k + k / CH instead of 2 k vectors); short vectors live
// in L2 and take CH = 1, which keeps fewer registers and barriers per pass.
template <typename TV, typename T, int CH>
__global__ void __launch_bounds__(kRedThreads) k_mdot_partial(const TV* __restrict__ V, long long ldv, int k,
                                                              const T* __restrict__ w, long long n,
                                                              double* __restrict__ partial) {
  __shared__ double red[CH][kRedThreads / 32];
  for (int j0 = 0; j0 < k; j0 += CH) {
    double s[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) s[c] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      const double wi = (double)w[i];
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (j0 + c < k) s[c] += (double)V[(j0 + c) * ldv + i] * wi;
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      double t = s[c];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x < CH && j0 + (int)threadIdx.x < k) {
      double t = 0.0;
      for (int wp = 0; wp < kRedThreads / 32; ++wp) t += red[threadIdx.x][wp];
      partial[(j0 + threadIdx.x) * kRedBlocks + blockIdx.x] = t;
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
  if (n >= (1LL << 22))
    k_mdot_partial<TV, T, 8><<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, k, w, n, partial);
  else
    k_mdot_partial<TV, T, 1><<<kRedBlocks, kRedThreads, 0, st>>>(V, ldv, k, w, n, partial);
  note_launch();
  k_mdot_final<<<k, 256, 0, st>>>(partial, k, out); note_launch();
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
  k_maxpy<<<kRedBlocks * 2, 256, 0, st>>>(w, V, ldv, k, h, sign, n); note_launch();
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
  k_axpby<T><<<kRedBlocks * 2, 256, 0, st>>>(y, x, a, b, n); note_launch();
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
  k_bminus<T><<<kRedBlocks * 2, 256, 0, st>>>(y, b, n); note_launch();
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
  k_dscale<T><<<kRedBlocks * 2, 256, 0, st>>>(y, x, d, n); note_launch();
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
  k_convert<double, float><<<kRedBlocks * 2, 256, 0, st>>>(y, x, n); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_f2d(double* y, const float* x, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_convert<float, double><<<kRedBlocks * 2, 256, 0, st>>>(y, x, n); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Q1 coarse operator
// Assembled Q1 operator at the fine Gauss points (coarse Lagrange basis of
// order 1 evaluated at the fine points, fine stored tangent): the exact
// Galerkin operator of the p-hierarchy.  Storage: 27-point stencil with a 4x4
// block per neighbour, A[(slot*16 + f*4 + g) * nn + node], slot = neighbour
// offset (dx+1) + 3 (dy+1) + 9 (dz+1); Dirichlet rows and columns are zero
// with a unit diagonal.

// y = A x with the stencil storage (FP64), one thread per node.
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
// The same product with an FP32 copy of the stencil, FP32 arithmetic, FP64
// vectors in and out (the mixed solver's coarse level: a preconditioner, whose
// FP64 product is bound by the FP64 pipe at 432 multiply-adds per node).  x is
// taken to FP32 by truncation of its significand (integer operations: the
// conversion instructions run at the FP64 rate).
__global__ void k_q1_spmv32(MeshDev mc, const float* __restrict__ A, const double* __restrict__ x,
                            double* __restrict__ y) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= mc.nn) return;
  const int nnz_ = (int)(mc.nn / ((long long)mc.nnx * mc.nny));
  const int I = (int)(n % mc.nnx), J = (int)((n / mc.nnx) % mc.nny), K = (int)(n / ((long long)mc.nnx * mc.nny));
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int slot = 0; slot < 27; ++slot) {
    const int dx = slot % 3 - 1, dy = (slot / 3) % 3 - 1, dz = slot / 9 - 1;
    const int I2 = I + dx, J2 = J + dy, K2 = K + dz;
    if (I2 < 0 || J2 < 0 || K2 < 0 || I2 >= mc.nnx || J2 >= mc.nny || K2 >= nnz_) continue;
    const long long m = I2 + (long long)mc.nnx * (J2 + (long long)mc.nny * K2);
    float xv[4];
    for (int g = 0; g < 4; ++g) xv[g] = df_split(x[g * mc.nn + m]).hi;
    for (int f = 0; f < 4; ++f)
      for (int g = 0; g < 4; ++g) acc[f] = fmaf(A[(long long)(slot * 16 + f * 4 + g) * mc.nn + n], xv[g], acc[f]);
  }
  for (int f = 0; f < 4; ++f) y[f * mc.nn + n] = df_f2d(acc[f]);
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
  k_q1_spmv_t<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, A, x, y); note_launch();
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
  k_sel_scale<<<kRedBlocks * 2, 256, 0, st>>>(y, sel, s, n); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_zero_masked(double* y, const uint8_t* mask, long long n, cudaStream_t st) {
  if (!mask) return cudaSuccess;
  k_zero_masked<<<kRedBlocks * 2, 256, 0, st>>>(y, mask, n); note_launch();
  return cudaGetLastError();
}

__global__ void k_q1_diag(MeshDev mc, const double* __restrict__ A, double* __restrict__ d) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= mc.nn) return;
  for (int f = 0; f < 4; ++f) d[f * mc.nn + n] = A[(long long)(13 * 16 + f * 4 + f) * mc.nn + n];
}
cudaError_t launch_q1_spmv(const MeshDev& mc, const double* A, const double* x, double* y, cudaStream_t st) {
  k_q1_spmv<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, A, x, y); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_q1_spmv32(const MeshDev& mc, const float* A, const double* x, double* y, cudaStream_t st) {
  k_q1_spmv32<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, A, x, y); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_q1_diag(const MeshDev& mc, const double* A, double* d, cudaStream_t st) {
  k_q1_diag<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, A, d); note_launch();
  return cudaGetLastError();
}

// ---- sum-factorised element matrices of the order-1 level (FP64) ----------
// One block per element.  The stored words of the element's 125 (Q^3) points
// give 67 "combinations" (word, test derivative, trial derivative) on the box
// and 70 on a mapped mesh: 45 from the symmetric 9x9 block (the transposed
// block of an off-diagonal pair is placed from the same result), 9 dP/dphi,
// 9 d(s_phi L)/dF, the phi value term, the 3 diagonal phase-gradient terms and
// (mapped) the 3 off-diagonal ones.  Each combination's 8x8 block is
//   sum_{ijk} D(i,j,k) X0[i][a0 b0] X1[j][a1 b1] X2[k][a2 b2],
// Xd[q][a b] = F_r,d[q][a] F_c,d[q][b], F = B1 or its derivative D1,
// contracted one direction at a time.  Output: Ke[e][32][32].
constexpr int kQ1Combos = 70;  // 67 on the affine box (no off-diagonal phase-gradient words)
constexpr int kQ1Threads = 256;

__device__ __forceinline__ void q1_combo(int c, int& word, int& rk, int& ck) {
  // rk/ck: 0 value, 1 + alpha derivative
  if (c < 45) {
    int m = 0, rem = c;
    while (rem >= 9 - m) { rem -= 9 - m; ++m; }
    const int n = m + rem;
    word = sym9(m, n);
    rk = 1 + m % 3;
    ck = 1 + n % 3;
  } else if (c < 54) {
    const int m = c - 45;
    word = kWP + m; rk = 1 + m % 3; ck = 0;
  } else if (c < 63) {
    const int n = c - 54;
    word = kWC + n; rk = 0; ck = 1 + n % 3;
  } else if (c == 63) {
    word = kWD; rk = 0; ck = 0;
  } else if (c < 67) {
    const int al = c - 64;
    word = kWK + al; rk = 1 + al; ck = 1 + al;
  } else {  // off-diagonal phase-gradient pairs 01, 02, 12 (mapped meshes)
    const int pr = c - 67;
    word = kWKX + pr; rk = 1 + ((pr == 2) ? 1 : 0); ck = 1 + ((pr == 0) ? 1 : 2);
  }
}

// One block (8 warps) per element; warp w takes the combinations c = w, w + 8,
// ... and contracts them one direction at a time in its own shared scratch
// (D[Q^3] -> T1[4][Q^2] -> T2[16][Q] -> R[c][64]) with the 1D products
// X[(fa, fb)][i][(a, b)] = F_fa(i, a) F_fb(i, b) tabulated once per block; the
// block then sums the combinations of each (f, g) block of Ke.
// T = double: FP64 words (planar layout), FP64 arithmetic; T = float (the
// mixed solver, whose coarse level only preconditions): the FP32 words (quad
// layout) and FP32 arithmetic, about sixty times the FP64 rate on GB300.
// Ke is FP64 either way.
__device__ __forceinline__ double q1_out(double v) { return v; }
__device__ __forceinline__ double q1_out(float v) { return df_f2d(v); }
template <int Q, typename T>
__device__ __forceinline__ T q1_word(const T* lin, long long blockbase, int word, int k, int t, long long stride) {
  constexpr long long q2eb = (long long)Q * Q * elems_per_block(Q);
  if constexpr (sizeof(T) == 8) return lin[blockbase + (long long)word * stride + (long long)k * q2eb + t];
  else return lin[blockbase + lin32_word(word, k, t, stride, q2eb)];
}
template <int Q, typename T>
__global__ void __launch_bounds__(kQ1Threads)
k_q1_elem(int nel, int ncombo, const T* __restrict__ lin, const double* __restrict__ B1,
          const double* __restrict__ D1, double* __restrict__ Ke) {
  constexpr int Q2 = Q * Q, Q3 = Q2 * Q;
  constexpr int EB = elems_per_block(Q);
  constexpr int kWarps = kQ1Threads / 32;
  constexpr int kScratch = Q3 + 4 * Q2 + 16 * Q;
  extern __shared__ __align__(16) unsigned char q1_smem[];
  T* R = reinterpret_cast<T*>(q1_smem);             // [67][64]
  T* X = R + kQ1Combos * 64;                        // [4][Q][4]
  T* W = X + 16 * Q;                                // [warps][kScratch]
  int* ctab = reinterpret_cast<int*>(W + kWarps * kScratch);  // [67][3]: word, rk, ck
  const int e = blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int idx = t; idx < 16 * Q; idx += kQ1Threads) {
    const int p = idx / (4 * Q), i = (idx / 4) % Q, ab = idx % 4;
    const int fa = p >> 1, fb = p & 1, a = ab >> 1, b = ab & 1;
    const double Fa = fa ? D1[i * 2 + a] : B1[i * 2 + a];
    const double Fb = fb ? D1[i * 2 + b] : B1[i * 2 + b];
    X[idx] = (T)(Fa * Fb);
  }
  for (int c = t; c < ncombo; c += kQ1Threads) q1_combo(c, ctab[3 * c], ctab[3 * c + 1], ctab[3 * c + 2]);
  __syncthreads();
  const long long stride = (long long)Q3 * EB;
  const long long blockbase = (long long)(e / EB) * kLinWords * stride;
  const int t0 = (e % EB) * Q2;
  T* D = W + warp * kScratch;
  T* T1 = D + Q3;
  T* T2 = T1 + 4 * Q2;
  for (int c = warp; c < ncombo; c += kWarps) {
    const int word = ctab[3 * c], rk = ctab[3 * c + 1], ck = ctab[3 * c + 2];
    for (int q = lane; q < Q3; q += 32) {
      const int k = q / Q2, jq = q % Q2;
      D[q] = q1_word<Q, T>(lin, blockbase, word, k, t0 + jq, stride);
    }
    __syncwarp();
    // direction 0 (i): T1[a0 b0][j + Q k]
    const T* X0 = X + ((rk == 1) * 2 + (ck == 1)) * 4 * Q;
    for (int idx = lane; idx < 4 * Q2; idx += 32) {
      const int ab = idx / Q2, jk = idx % Q2;
      T s = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) s += X0[i * 4 + ab] * D[jk * Q + i];
      T1[idx] = s;
    }
    __syncwarp();
    // direction 1 (j): T2[(a0 b0) 4 + (a1 b1)][k]
    const T* X1 = X + ((rk == 2) * 2 + (ck == 2)) * 4 * Q;
    for (int idx = lane; idx < 16 * Q; idx += 32) {
      const int abab = idx / Q, k = idx % Q;
      const int ab0 = abab >> 2, ab1 = abab & 3;
      const T* Tc = T1 + ab0 * Q2 + k * Q;
      T s = 0;
#pragma unroll
      for (int j = 0; j < Q; ++j) s += X1[j * 4 + ab1] * Tc[j];
      T2[idx] = s;
    }
    __syncwarp();
    // direction 2 (k): R[c][a][b], a = a0 + 2 a1 + 4 a2
    const T* X2 = X + ((rk == 3) * 2 + (ck == 3)) * 4 * Q;
    for (int r = lane; r < 64; r += 32) {
      const int a = r / 8, b = r % 8;
      const int a0 = a & 1, a1 = (a >> 1) & 1, a2 = a >> 2;
      const int b0 = b & 1, b1 = (b >> 1) & 1, b2 = b >> 2;
      const T* Tc = T2 + ((a0 * 2 + b0) * 4 + (a1 * 2 + b1)) * Q;
      T s = 0;
#pragma unroll
      for (int k = 0; k < Q; ++k) s += X2[k * 4 + a2 * 2 + b2] * Tc[k];
      R[c * 64 + r] = s;
    }
    __syncwarp();
  }
  __syncthreads();
  // element matrix: sum of the combinations of each (f, g) block
  double* out = Ke + (long long)e * 1024;
  for (int idx = t; idx < 1024; idx += kQ1Threads) {
    const int row = idx / 32, col = idx % 32;
    const int f = row / 8, a = row % 8, g = col / 8, b = col % 8;
    T v = 0;
    if (f < 3 && g < 3) {
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) {
          const int m = 3 * f + al, n = 3 * g + be;
          const int mm = m <= n ? m : n, nn2 = m <= n ? n : m;
          const int c = sym9(mm, nn2);  // combos are enumerated in the sym9 order
          v += (m <= n) ? R[c * 64 + a * 8 + b] : R[c * 64 + b * 8 + a];
        }
    } else if (f < 3) {
      for (int al = 0; al < 3; ++al) v += R[(45 + 3 * f + al) * 64 + a * 8 + b];
    } else if (g < 3) {
      for (int be = 0; be < 3; ++be) v += R[(54 + 3 * g + be) * 64 + a * 8 + b];
    } else {
      for (int c = 63; c < 67; ++c) v += R[c * 64 + a * 8 + b];
      for (int c = 67; c < ncombo; ++c) v += R[c * 64 + a * 8 + b] + R[c * 64 + b * 8 + a];
    }
    out[idx] = q1_out(v);
  }
}

// Stencil entry (slot, f, g) of node n: the sum, over the elements holding both
// n and its neighbour m, of Ke[(f, a(n)), (g, b(m))]; Dirichlet rows/columns of
// the identity.  One thread per (node, f, g); deterministic order.
__global__ void k_q1_gather(MeshDev mc, const double* __restrict__ Ke, const uint8_t* __restrict__ maskc,
                            double* __restrict__ A) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= mc.nn * 16) return;
  const long long n = tid % mc.nn;
  const int fg = (int)(tid / mc.nn);
  const int f = fg / 4, g = fg % 4;
  const int nnz_ = (int)(mc.nn / ((long long)mc.nnx * mc.nny));
  const int I = (int)(n % mc.nnx), J = (int)((n / mc.nnx) % mc.nny), K = (int)(n / ((long long)mc.nnx * mc.nny));
  const bool rowmask = maskc && maskc[f * mc.nn + n];
  for (int slot = 0; slot < 27; ++slot) {
    const int dx = slot % 3 - 1, dy = (slot / 3) % 3 - 1, dz = slot / 9 - 1;
    const int I2 = I + dx, J2 = J + dy, K2 = K + dz;
    double v = 0.0;
    if (I2 >= 0 && J2 >= 0 && K2 >= 0 && I2 < mc.nnx && J2 < mc.nny && K2 < nnz_) {
      const long long m = I2 + (long long)mc.nnx * (J2 + (long long)mc.nny * K2);
      if (rowmask) {
        v = (slot == 13 && f == g) ? 1.0 : 0.0;
      } else if (!(maskc && maskc[g * mc.nn + m])) {
        // elements whose closure holds both nodes
        const int ex0 = max(max(I, I2) - 1, 0), ex1 = min(min(I, I2), mc.nx - 1);
        const int ey0 = max(max(J, J2) - 1, 0), ey1 = min(min(J, J2), mc.ny - 1);
        const int ez0 = max(max(K, K2) - 1, 0), ez1 = min(min(K, K2), mc.nz - 1);
        for (int ez = ez0; ez <= ez1; ++ez)
          for (int ey = ey0; ey <= ey1; ++ey)
            for (int ex = ex0; ex <= ex1; ++ex) {
              const long long e = ex + (long long)mc.nx * (ey + (long long)mc.ny * ez);
              const int a = (I - ex) + 2 * ((J - ey) + 2 * (K - ez));
              const int b = (I2 - ex) + 2 * ((J2 - ey) + 2 * (K2 - ez));
              v += Ke[e * 1024 + (f * 8 + a) * 32 + g * 8 + b];
            }
      }
    }
    A[(long long)(slot * 16 + f * 4 + g) * mc.nn + n] = v;
  }
}

// ---- geometric h-hierarchy on the order-1 grid ---------------------------
// Coarse element E (2x2x2 fine elements c) of a vertex-centred full coarsening
// with trilinear interpolation: the prolongation restricted to E maps the 8
// coarse vertices to the 27 fine vertices inside E, so the Galerkin operator
// is a sum of element matrices
//   Ke_c[E] = sum_c W_c^T ((I - M) Ke_f[c] (I - M)) W_c,
// W_c[(f, a), (f, A)] = prod_d w((c_d + a_d) / 2, A_d), w(x, 0) = 1 - x,
// w(x, 1) = x, M the fine Dirichlet mask (prescribed DoFs take no correction).
// One block per coarse element, the two contractions through shared memory.
// The weights are products of 0, 1/2 and 1: exact in FP32 and FP64.  T =
// float for the mixed solver (FP32 arithmetic, FP64 storage of Ke).
template <typename T> __device__ __forceinline__ T q1_weight(int c, int a, int A) {
  T w = 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int cd = (c >> d) & 1, ad = (a >> d) & 1, Ad = (A >> d) & 1;
    const T x = (T)0.5 * (T)(cd + ad);
    w *= Ad ? x : (T)1 - x;
  }
  return w;
}
__device__ __forceinline__ double q1_in(double v, double) { return v; }
__device__ __forceinline__ float q1_in(double v, float) { return df_split(v).hi; }

template <typename T>
__global__ void __launch_bounds__(256) k_q1_coarsen(MeshDev mf, MeshDev mc, const uint8_t* __restrict__ maskf,
                                                    const double* __restrict__ Kef, double* __restrict__ Kec) {
  __shared__ T Kf[1024], Y[1024], Kc[1024];
  __shared__ int fnode[8];
  const int E = blockIdx.x, t = threadIdx.x;
  const int Ex = E % mc.nx, Ey = (E / mc.nx) % mc.ny, Ez = E / (mc.nx * mc.ny);
  for (int idx = t; idx < 1024; idx += blockDim.x) Kc[idx] = 0;
  for (int c = 0; c < 8; ++c) {
    const int ex = 2 * Ex + (c & 1), ey = 2 * Ey + ((c >> 1) & 1), ez = 2 * Ez + (c >> 2);
    const long long e = ex + (long long)mf.nx * (ey + (long long)mf.ny * ez);
    __syncthreads();  // Kf, Y and fnode of the previous child are consumed
    if (t < 8)
      fnode[t] = (int)((ex + (t & 1)) + (long long)mf.nnx * ((ey + ((t >> 1) & 1)) + (long long)mf.nny * (ez + (t >> 2))));
    __syncthreads();
    for (int idx = t; idx < 1024; idx += blockDim.x) {
      const int row = idx >> 5, col = idx & 31;
      T v = q1_in(Kef[e * 1024 + idx], T(0));
      if (maskf && (maskf[(row >> 3) * mf.nn + fnode[row & 7]] || maskf[(col >> 3) * mf.nn + fnode[col & 7]])) v = 0;
      Kf[idx] = v;
    }
    __syncthreads();
    // Y[(f, a)][(g, B)] = sum_b Kf[(f, a)][(g, b)] W_c[b][B]
    for (int idx = t; idx < 1024; idx += blockDim.x) {
      const int row = idx >> 5, g = (idx >> 3) & 3, B = idx & 7;
      T acc = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) acc += Kf[row * 32 + g * 8 + b] * q1_weight<T>(c, b, B);
      Y[idx] = acc;
    }
    __syncthreads();
    // Kc[(f, A)][(g, B)] += sum_a W_c[a][A] Y[(f, a)][(g, B)]
    for (int idx = t; idx < 1024; idx += blockDim.x) {
      const int f = idx >> 8, A = (idx >> 5) & 7, col = idx & 31;
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) acc += q1_weight<T>(c, a, A) * Y[(f * 8 + a) * 32 + col];
      Kc[idx] += acc;
    }
  }
  __syncthreads();
  for (int idx = t; idx < 1024; idx += blockDim.x) Kec[(long long)E * 1024 + idx] = q1_out(Kc[idx]);
}

// Coarse Dirichlet mask: a coarse vertex is prescribed where the coincident
// fine vertex is.
__global__ void k_hmask(MeshDev mf, MeshDev mc, const uint8_t* __restrict__ maskf, uint8_t* __restrict__ maskc) {
  const long long N = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (N >= mc.nn) return;
  const int I = (int)(N % mc.nnx), J = (int)((N / mc.nnx) % mc.nny), K = (int)(N / ((long long)mc.nnx * mc.nny));
  const long long n = 2 * I + (long long)mf.nnx * (2 * J + (long long)mf.nny * 2 * K);
  for (int f = 0; f < 4; ++f) maskc[f * mc.nn + N] = maskf ? maskf[f * mf.nn + n] : 0;
}

// x_f += P x_c on unmasked fine DoFs (trilinear, one thread per fine vertex).
__global__ void k_hprolong_add(MeshDev mc, MeshDev mf, const double* __restrict__ xc, double* __restrict__ xf,
                               const uint8_t* __restrict__ maskc, const uint8_t* __restrict__ maskf) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= mf.nn) return;
  const int i = (int)(n % mf.nnx), j = (int)((n / mf.nnx) % mf.nny), k = (int)(n / ((long long)mf.nnx * mf.nny));
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int dz = 0; dz < 2; ++dz) {
    if (dz && !(k & 1)) break;
    const int K = (k >> 1) + dz;
    const double wz = (k & 1) ? 0.5 : 1.0;
    for (int dy = 0; dy < 2; ++dy) {
      if (dy && !(j & 1)) break;
      const int J = (j >> 1) + dy;
      const double wy = (j & 1) ? 0.5 : 1.0;
      for (int dx = 0; dx < 2; ++dx) {
        if (dx && !(i & 1)) break;
        const int I = (i >> 1) + dx;
        const double w = wz * wy * ((i & 1) ? 0.5 : 1.0);
        const long long N = I + (long long)mc.nnx * (J + (long long)mc.nny * K);
        for (int f = 0; f < 4; ++f)
          if (!(maskc && maskc[f * mc.nn + N])) acc[f] += w * xc[f * mc.nn + N];
      }
    }
  }
  for (int f = 0; f < 4; ++f)
    if (!(maskf && maskf[f * mf.nn + n])) xf[f * mf.nn + n] += acc[f];
}

// r_c = P^T r_f (zero on masked DoFs), one thread per coarse vertex gathering
// the fine vertices within one fine spacing.
__global__ void k_hrestrict(MeshDev mc, MeshDev mf, const double* __restrict__ rf, double* __restrict__ rc,
                            const uint8_t* __restrict__ maskc, const uint8_t* __restrict__ maskf) {
  const long long N = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (N >= mc.nn) return;
  const int I = (int)(N % mc.nnx), J = (int)((N / mc.nnx) % mc.nny), K = (int)(N / ((long long)mc.nnx * mc.nny));
  const int nnzf = (int)(mf.nn / ((long long)mf.nnx * mf.nny));
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int dz = -1; dz <= 1; ++dz) {
    const int k = 2 * K + dz;
    if (k < 0 || k >= nnzf) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int j = 2 * J + dy;
      if (j < 0 || j >= mf.nny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = 2 * I + dx;
        if (i < 0 || i >= mf.nnx) continue;
        const double w = (dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0);
        const long long n = i + (long long)mf.nnx * (j + (long long)mf.nny * k);
        for (int f = 0; f < 4; ++f)
          if (!(maskf && maskf[f * mf.nn + n])) acc[f] += w * rf[f * mf.nn + n];
      }
    }
  }
  for (int f = 0; f < 4; ++f) rc[f * mc.nn + N] = (maskc && maskc[f * mc.nn + N]) ? 0.0 : acc[f];
}

cudaError_t launch_q1_coarsen(const MeshDev& mf, const MeshDev& mc, const uint8_t* maskf, const double* Kef,
                              double* Kec, bool f32, cudaStream_t st) {
  if (mc.nel == 0) return cudaSuccess;
  if (f32) k_q1_coarsen<float><<<mc.nel, 256, 0, st>>>(mf, mc, maskf, Kef, Kec);
  else k_q1_coarsen<double><<<mc.nel, 256, 0, st>>>(mf, mc, maskf, Kef, Kec);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_q1_gather(const MeshDev& mc, const double* Ke, const uint8_t* maskc, double* A, cudaStream_t st) {
  const long long nt = mc.nn * 16;
  k_q1_gather<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(mc, Ke, maskc, A); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_hmask(const MeshDev& mf, const MeshDev& mc, const uint8_t* maskf, uint8_t* maskc, cudaStream_t st) {
  k_hmask<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mf, mc, maskf, maskc); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_hprolong_add(const MeshDev& mc, const MeshDev& mf, const double* xc, double* xf,
                                const uint8_t* maskc, const uint8_t* maskf, cudaStream_t st) {
  k_hprolong_add<<<(unsigned)((mf.nn + 255) / 256), 256, 0, st>>>(mc, mf, xc, xf, maskc, maskf); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_hrestrict(const MeshDev& mc, const MeshDev& mf, const double* rf, double* rc,
                             const uint8_t* maskc, const uint8_t* maskf, cudaStream_t st) {
  k_hrestrict<<<(unsigned)((mc.nn + 255) / 256), 256, 0, st>>>(mc, mf, rf, rc, maskc, maskf); note_launch();
  return cudaGetLastError();
}

template <int Q, typename T>
void q1_elem_launch(const MeshDev& mc, const T* lin, const double* B1, const double* D1, double* Ke, int ncombo,
                    cudaStream_t st) {
  const size_t smem = sizeof(T) * (size_t)(kQ1Combos * 64 + 16 * Q + (kQ1Threads / 32) * (Q * Q * Q + 4 * Q * Q + 16 * Q)) +
                      sizeof(int) * 3 * kQ1Combos;
  cudaFuncSetAttribute(k_q1_elem<Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_q1_elem<Q, T><<<mc.nel, kQ1Threads, smem, st>>>(mc.nel, ncombo, lin, B1, D1, Ke); note_launch();
}
template <typename T>
cudaError_t q1_elem_dispatch(const MeshDev& mc, int Q, const T* lin, const double* B1, const double* D1, double* Ke,
                             int ncombo, cudaStream_t st) {
  switch (Q) {
    case 2: q1_elem_launch<2, T>(mc, lin, B1, D1, Ke, ncombo, st); break;
    case 3: q1_elem_launch<3, T>(mc, lin, B1, D1, Ke, ncombo, st); break;
    case 4: q1_elem_launch<4, T>(mc, lin, B1, D1, Ke, ncombo, st); break;
    case 5: q1_elem_launch<5, T>(mc, lin, B1, D1, Ke, ncombo, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_q1_assemble_sf(const MeshDev& mc, int Q, const double* lin, const float* lin32, const double* B1,
                                  const double* D1, const uint8_t* maskc, double* Ke, double* A, int kx,
                                  cudaStream_t st) {
  const int ncombo = kx ? kQ1Combos : 67;
  const cudaError_t d = lin32 ? q1_elem_dispatch<float>(mc, Q, lin32, B1, D1, Ke, ncombo, st)
                              : q1_elem_dispatch<double>(mc, Q, lin, B1, D1, Ke, ncombo, st);
  if (d != cudaSuccess) return d;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long nt = mc.nn * 16;
  k_q1_gather<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(mc, Ke, maskc, A); note_launch();
  return cudaGetLastError();
}

}  // namespace pff

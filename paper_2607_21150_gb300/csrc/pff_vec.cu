// Vector kernels: Dirichlet initialisation, the FP32 (and double-float)
// planes of the stored linearisation, the p-multigrid transfer operators, the
// Chebyshev smoother updates, the export of the linearisation, reaction sums
// and the geometric factors of mapped meshes.
#include <cuda_bf16.h>

#include "pff_df.cuh"
#include "pff_internal.h"

namespace pff {

constexpr int kVecThreads = 256;

static unsigned grid_for(long long n) {
  long long b = (n + kVecThreads - 1) / kVecThreads;
  if (b > 152LL * 64) b = 152LL * 64;  // grid-stride beyond 64 blocks per SM
  return (unsigned)(b > 0 ? b : 1);
}

// mode 0: y = mask ? x : 0      (Jacobian action: identity rows of Dirichlet DoFs)
// mode 1: y = mask ? x - u : 0  (residual: z - ubar on Dirichlet DoFs)
// mode 2: y = mask ? 1 : 0      (diagonal)
template <typename T>
__global__ void k_init_masked(T* __restrict__ y, const T* __restrict__ x, const double* __restrict__ ubar,
                              const uint8_t* __restrict__ mask, long long n, int mode) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    bool m = mask && mask[i];
    T v = T(0);
    if (m) {
      if (mode == 0) v = x[i];
      else if (mode == 1) v = x[i] - (ubar ? (T)ubar[i] : T(0));
      else v = T(1);
    }
    y[i] = v;
  }
}

cudaError_t launch_init_masked(int prec, void* y, const void* x, const double* ubar, const uint8_t* mask,
                               long long n, int mode, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (prec == 0)
    k_init_masked<double><<<grid_for(n), kVecThreads, 0, st>>>((double*)y, (const double*)x, ubar, mask, n, mode);
  else
    k_init_masked<float><<<grid_for(n), kVecThreads, 0, st>>>((float*)y, (const float*)x, ubar, mask, n, mode);
  note_launch();
  return cudaGetLastError();
}

// Deterministic transpose E^T: every node sums the values its incident
// elements left in evec, always in the same order (elements ascending), so
// reruns are bitwise identical.  Node (I, J, K) lies in elements
// ex = I / p (local a = I mod p) and, on an element boundary (I mod p = 0),
// also ex - 1 (local a = p); likewise in y and z.
template <typename T>
__global__ void k_node_gather(MeshDev m, const T* __restrict__ evec, const uint8_t* __restrict__ mask, int mode,
                              const T* __restrict__ x, const double* __restrict__ ubar, T* __restrict__ y, long long n0,
                              long long n1) {
  const long long n = n0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= n1) return;
  const int p = m.p, P = p + 1, P3 = P * P * P;
  const int I = (int)(n % m.nnx), J = (int)((n / m.nnx) % m.nny), K = (int)(n / ((long long)m.nnx * m.nny));
  int ex[2], ax[2], nxc = 0, ey[2], ay[2], nyc = 0, ez[2], az[2], nzc = 0;
  if (I % p == 0 && I > 0) { ex[nxc] = I / p - 1; ax[nxc++] = p; }
  if (I / p < m.nx) { ex[nxc] = I / p; ax[nxc++] = I % p; }
  if (J % p == 0 && J > 0) { ey[nyc] = J / p - 1; ay[nyc++] = p; }
  if (J / p < m.ny) { ey[nyc] = J / p; ay[nyc++] = J % p; }
  if (K % p == 0 && K > 0) { ez[nzc] = K / p - 1; az[nzc++] = p; }
  if (K / p < m.nz) { ez[nzc] = K / p; az[nzc++] = K % p; }
  for (int f = 0; f < 4; ++f) {
    const long long g = f * m.nn + n;
    T v = T(0);
    if (mask && mask[g]) {
      v = (mode == 0) ? x[g] : (mode == 1) ? x[g] - (ubar ? (T)ubar[g] : T(0)) : (mode == 2) ? T(1) : T(0);
    } else {
      for (int cz = 0; cz < nzc; ++cz)
        for (int cy = 0; cy < nyc; ++cy)
          for (int cx = 0; cx < nxc; ++cx) {
            const long long e = ex[cx] + (long long)m.nx * (ey[cy] + (long long)m.ny * ez[cz]);
            v += evec[(e * 4 + f) * P3 + ax[cx] + P * (ay[cy] + P * az[cz])];
          }
    }
    y[g] = v;
  }
}
cudaError_t launch_node_gather(int prec, const MeshDev& m, const void* evec, const uint8_t* mask, int mode,
                               const void* x, const double* ubar, void* y, long long n0, long long n1,
                               cudaStream_t st) {
  if (n1 <= n0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n1 - n0 + 255) / 256);
  if (prec == 0)
    k_node_gather<double><<<blocks, 256, 0, st>>>(m, (const double*)evec, mask, mode, (const double*)x, ubar,
                                                  (double*)y, n0, n1);
  else
    k_node_gather<float><<<blocks, 256, 0, st>>>(m, (const float*)evec, mask, mode, (const float*)x, ubar,
                                                 (float*)y, n0, n1);
  note_launch();
  return cudaGetLastError();
}

// emask[e] = 1 if any of element e's nodes has a prescribed (masked) DoF in
// any field, else 0: the element kernels read the node mask only for flagged
// elements (on a box with Dirichlet faces, a few percent of them).
__global__ void k_elem_mask(MeshDev m, const uint8_t* __restrict__ mask, uint8_t* __restrict__ emask) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= m.nel) return;
  const int P = m.p + 1;
  const int ex = (int)(e % m.nx), t = (int)(e / m.nx), ey = t % m.ny, ez = t / m.ny;
  uint8_t any = 0;
  for (int c = 0; c < P && !any; ++c)
    for (int b = 0; b < P && !any; ++b)
      for (int a = 0; a < P; ++a) {
        const long long n = m.offsets ? (long long)m.offsets[e * P * P * P + a + P * (b + P * c)]
                                      : (long long)(m.p * ex + a) +
                                            (long long)m.nnx * ((long long)(m.p * ey + b) + (long long)m.nny * (m.p * ez + c));
        for (int f = 0; f < 4; ++f) any |= mask[f * m.nn + n];
        if (any) break;
      }
  emask[e] = any ? 1 : 0;
}
cudaError_t launch_elem_mask(const MeshDev& m, const uint8_t* mask, uint8_t* emask, cudaStream_t st) {
  if (m.nel == 0) return cudaSuccess;
  k_elem_mask<<<(unsigned)((m.nel + 255) / 256), 256, 0, st>>>(m, mask, emask); note_launch();
  return cudaGetLastError();
}

// y = mask ? x : 0 on the nodes [n0, n1) of each of the four fields (rows of
// one range of node layers; the pipelined action through host buffers).
template <typename T>
__global__ void k_init_rows(T* __restrict__ y, const T* __restrict__ x, const uint8_t* __restrict__ mask, long long nn,
                            long long n0, long long cnt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * cnt; i += (long long)gridDim.x * blockDim.x) {
    const long long g = (i / cnt) * nn + n0 + i % cnt;
    y[g] = (mask && mask[g]) ? x[g] : T(0);
  }
}
cudaError_t launch_init_rows(int prec, void* y, const void* x, const uint8_t* mask, long long nn, long long n0,
                             long long n1, cudaStream_t st) {
  const long long cnt = n1 - n0;
  if (cnt <= 0) return cudaSuccess;
  if (prec == 0) k_init_rows<double><<<grid_for(4 * cnt), kVecThreads, 0, st>>>((double*)y, (const double*)x, mask, nn, n0, cnt);
  else k_init_rows<float><<<grid_for(4 * cnt), kVecThreads, 0, st>>>((float*)y, (const float*)x, mask, nn, n0, cnt);
  note_launch();
  return cudaGetLastError();
}

// BF16 word of x, round to nearest even, by integer operations on the FP64
// bit pattern (zero and FP64 subnormals give signed zero; the rare |x| outside
// the normal FP32 range goes through the library conversion).
__device__ __forceinline__ unsigned bf16_rne(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned sgn = (hw >> 16) & 0x8000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  if (e == 0) return sgn;
  const int ef = e - 896;
  if (ef <= 0 || ef >= 255) return __bfloat16_as_ushort(__double2bfloat16(x));
  const unsigned top = ((unsigned)ef << 7) | ((hw & 0xfffffu) >> 13);  // exponent and 7 significand bits
  const unsigned r = hw & 0x1fffu;                                      // significand bits 44..32 (44: half)
  const unsigned inc = (r > 0x1000u || (r == 0x1000u && (lw != 0u || (top & 1u)))) ? 1u : 0u;
  return sgn | (top + inc);  // a carry moves into the exponent
}

// The level copies of the stored linearisation in one pass over the FP64
// words: the FP32 planes (lin32_word layout; hi = fl32(a), round to nearest
// even, and lo = a - hi to 23 bits, df_split_rn) and the BF16 words
// (lin16_word layout; words 70 and 71 zero), each optional.  All conversions
// are integer operations, so that the pass runs at HBM speed rather than at
// the FP64 rate of the conversion instructions.  One thread per octet of a
// point's words [0, 64) (eight coalesced FP64 reads; two 128-bit writes per
// FP32 plane, one for the BF16 octet), then one per tail plane of four words.
// Writing these copies from the pointwise kernel instead measured slower
// (64^3 Q4 residual 154 -> 176 ms): its scattered narrow stores cost more than
// this pass.
__global__ void k_split_words(const double* __restrict__ a, float* __restrict__ hi, float* __restrict__ lo,
                              uint16_t* __restrict__ b16, long long nblk, long long q3eb) {
  const long long bw = (long long)kLinWords * q3eb, ow = (long long)kLin16Words * q3eb;
  const long long opb = 8 * q3eb, tpb = 2 * q3eb;  // octet / tail units per block
  const long long no = nblk * opb, n = no + nblk * tpb;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
    if (u < no) {
      const long long b = u / opb, rem = u % opb;
      const long long oc = rem / q3eb, r2 = rem % q3eb;
      const double* src = a + b * bw + 8 * oc * q3eb + r2;
      double x[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = src[c * q3eb];
      if (hi) {
        float h[8], l[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const df64 v = df_split_rn(x[c]);
          h[c] = v.hi;
          l[c] = v.lo;
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const long long o = b * bw + (2 * oc + g) * 4 * q3eb + 4 * r2;
          *reinterpret_cast<float4*>(hi + o) = make_float4(h[4 * g], h[4 * g + 1], h[4 * g + 2], h[4 * g + 3]);
          if (lo) *reinterpret_cast<float4*>(lo + o) = make_float4(l[4 * g], l[4 * g + 1], l[4 * g + 2], l[4 * g + 3]);
        }
      }
      if (b16) {
        unsigned v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = bf16_rne(x[2 * c]) | (bf16_rne(x[2 * c + 1]) << 16);
        *reinterpret_cast<uint4*>(b16 + b * ow + oc * 8 * q3eb + 8 * r2) = make_uint4(v[0], v[1], v[2], v[3]);
      }
    } else {
      const long long w = u - no, b = w / tpb, rem = w % tpb;
      const long long tp = rem / q3eb, r2 = rem % q3eb;
      unsigned v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int wd = 64 + 4 * (int)tp + c;
        v[c] = 0u;
        if (wd < kLinWords) {
          const long long i = b * bw + wd * q3eb + r2;
          const double x = a[i];
          if (hi) {
            const df64 sv = df_split_rn(x);
            hi[i] = sv.hi;
            if (lo) lo[i] = sv.lo;
          }
          v[c] = bf16_rne(x);
        }
      }
      if (b16)
        *reinterpret_cast<uint2*>(b16 + b * ow + (64 + 4 * tp) * q3eb + 4 * r2) =
            make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
    }
  }
}
cudaError_t launch_split_words(const double* a, float* hi, float* lo, uint16_t* b16, long long nblk, int Q,
                               cudaStream_t st) {
  if (nblk == 0 || (!hi && !b16)) return cudaSuccess;
  const long long q3eb = (long long)Q * Q * Q * elems_per_block(Q);
  const long long n = nblk * 10 * q3eb;
  k_split_words<<<grid_for(n), kVecThreads, 0, st>>>(a, hi, lo, b16, nblk, q3eb); note_launch();
  return cudaGetLastError();
}

// Prolongation x_f = P x_c, P[f, c] = coarse Lagrange basis at the fine GLL
// node (I1[a][b], a fine, b coarse, per direction).  One thread per fine node;
// the owning element is any element whose closure holds the node (the coarse
// space is continuous, so every choice gives the same value).
template <typename T>
__global__ void k_prolong(MeshDev mc, MeshDev mf, const T* __restrict__ I1, const T* __restrict__ xc,
                          T* __restrict__ xf, const uint8_t* __restrict__ maskc, const uint8_t* __restrict__ maskf) {
  const int Pc = mc.p + 1, Pf = mf.p + 1;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= mf.nn) return;
  const int I = (int)(n % mf.nnx);
  const int J = (int)((n / mf.nnx) % mf.nny);
  const int K = (int)(n / ((long long)mf.nnx * mf.nny));
  const int idx[3] = {I, J, K};
  const int ne[3] = {mf.nx, mf.ny, mf.nz};
  int el[3], loc[3];
  for (int d = 0; d < 3; ++d) {
    int e = idx[d] / mf.p;
    if (e >= ne[d]) e = ne[d] - 1;
    el[d] = e;
    loc[d] = idx[d] - mf.p * e;
  }
  for (int f = 0; f < 4; ++f) {
    long long gf = f * mf.nn + n;
    if (maskf && maskf[gf]) { xf[gf] = T(0); continue; }
    T s = T(0);
    for (int c = 0; c < Pc; ++c) {
      T wz = I1[loc[2] * Pc + c];
      for (int b = 0; b < Pc; ++b) {
        T wyz = wz * I1[loc[1] * Pc + b];
        for (int a = 0; a < Pc; ++a) {
          long long nc = (long long)(mc.p * el[0] + a) + (long long)mc.nnx * ((long long)(mc.p * el[1] + b) + (long long)mc.nny * (mc.p * el[2] + c));
          long long gc = f * mc.nn + nc;
          if (maskc && maskc[gc]) continue;
          s += wyz * I1[loc[0] * Pc + a] * xc[gc];
        }
      }
    }
    xf[gf] = s;
  }
  (void)Pf;
}

template <typename T>
cudaError_t launch_prolong(const MeshDev& mc, const MeshDev& mf, const T* I1, const T* xc, T* xf,
                           const uint8_t* maskc, const uint8_t* maskf, cudaStream_t st) {
  if (mf.nn == 0) return cudaSuccess;
  unsigned nb = (unsigned)((mf.nn + 255) / 256);
  k_prolong<T><<<nb, 256, 0, st>>>(mc, mf, I1, xc, xf, maskc, maskf); note_launch();
  return cudaGetLastError();
}

// Restriction r_c = P^T r_f, element by element: every element adds
// I1^T-weighted fine residuals divided by the fine node's multiplicity (the
// number of elements sharing it), which sums to exactly P^T r_f.  One thread
// per (element, coarse local node).
template <typename T>
__global__ void k_restrict(MeshDev mc, MeshDev mf, const T* __restrict__ I1, const T* __restrict__ rf,
                           T* __restrict__ rc, const uint8_t* __restrict__ maskc, const uint8_t* __restrict__ maskf,
                           T* __restrict__ evec) {
  const int Pc = mc.p + 1, Pf = mf.p + 1;
  const int Pc3 = Pc * Pc * Pc;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)mc.nel * Pc3) return;
  const int e = (int)(tid / Pc3);
  const int lb = (int)(tid % Pc3);
  const int b0 = lb % Pc, b1 = (lb / Pc) % Pc, b2 = lb / (Pc * Pc);
  const int ex = e % mf.nx, ey = (e / mf.nx) % mf.ny, ez = e / (mf.nx * mf.ny);
  const long long nc = (long long)(mc.p * ex + b0) + (long long)mc.nnx * ((long long)(mc.p * ey + b1) + (long long)mc.nny * (mc.p * ez + b2));
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int c = 0; c < Pf; ++c) {
    const int K = mf.p * ez + c;
    const T mz = (c == 0 && ez > 0) || (c == mf.p && ez < mf.nz - 1) ? T(0.5) : T(1);
    const T wz = I1[c * Pc + b2] * mz;
    for (int b = 0; b < Pf; ++b) {
      const int J = mf.p * ey + b;
      const T my = (b == 0 && ey > 0) || (b == mf.p && ey < mf.ny - 1) ? T(0.5) : T(1);
      const T wyz = wz * I1[b * Pc + b1] * my;
      for (int a = 0; a < Pf; ++a) {
        const int I = mf.p * ex + a;
        const T mx = (a == 0 && ex > 0) || (a == mf.p && ex < mf.nx - 1) ? T(0.5) : T(1);
        const T w = wyz * I1[a * Pc + b0] * mx;
        const long long nf = I + (long long)mf.nnx * (J + (long long)mf.nny * K);
        for (int f = 0; f < 4; ++f) {
          long long gf = f * mf.nn + nf;
          if (maskf && maskf[gf]) continue;
          acc[f] += w * rf[gf];
        }
      }
    }
  }
  if (evec) {  // deterministic: element values, summed per coarse node by k_node_gather
    for (int f = 0; f < 4; ++f) evec[((long long)e * 4 + f) * Pc3 + lb] = acc[f];
    return;
  }
  for (int f = 0; f < 4; ++f) {
    long long gc = f * mc.nn + nc;
    if (maskc && maskc[gc]) continue;
    atomicAdd(rc + gc, acc[f]);
  }
}

template <typename T>
cudaError_t launch_restrict(const MeshDev& mc, const MeshDev& mf, const T* I1, const T* rf, T* rc,
                            const uint8_t* maskc, const uint8_t* maskf, cudaStream_t st, void* evec) {
  long long n = (long long)mc.nel * (mc.p + 1) * (mc.p + 1) * (mc.p + 1);
  if (!evec) {
    cudaError_t err = cudaMemsetAsync(rc, 0, sizeof(T) * 4 * mc.nn, st);
    if (err != cudaSuccess) return err;
  }
  if (n == 0) return cudaSuccess;
  k_restrict<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mc, mf, I1, rf, rc, maskc, maskf, (T*)evec);
  note_launch();
  if (evec) return launch_node_gather(sizeof(T) == 8 ? 0 : 1, mc, evec, maskc, 3, nullptr, nullptr, rc, 0, mc.nn, st);
  return cudaGetLastError();
}

// Chebyshev iteration (Saad, Alg. 12.1) on D^-1 A:
//   init:  r = D^-1 (b - A x),  d = r / theta
//   step:  x += d;  r -= D^-1 A d;  d = c_d d + c_r r      (c_d = rho_k+1 rho_k, c_r = 2 rho_k+1 / delta)
//   last:  x += d
template <typename T>
__global__ void k_cheb_init(long long n, const T* __restrict__ b, const T* __restrict__ Ax, const T* __restrict__ diag,
                            T* __restrict__ r, T* __restrict__ d, T inv_theta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T ri = (b[i] - Ax[i]) / diag[i];
    r[i] = ri;
    d[i] = ri * inv_theta;
  }
}
template <typename T>
__global__ void k_cheb_step(long long n, T* __restrict__ x, T* __restrict__ d, T* __restrict__ r,
                            const T* __restrict__ Ad, const T* __restrict__ diag, T c_d, T c_r, int last) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T di = d[i];
    x[i] += di;
    if (!last) {
      T ri = r[i] - Ad[i] / diag[i];
      r[i] = ri;
      d[i] = c_d * di + c_r * ri;
    }
  }
}

template <typename T>
cudaError_t launch_cheb_init(long long n, const T* b, const T* Ax, const T* diag, T* r, T* d, double inv_theta,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_cheb_init<T><<<grid_for(n), kVecThreads, 0, st>>>(n, b, Ax, diag, r, d, (T)inv_theta); note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cheb_step(long long n, T* x, T* d, T* r, const T* Ad, const T* diag, double c_d, double c_r,
                             int last, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_cheb_step<T><<<grid_for(n), kVecThreads, 0, st>>>(n, x, d, r, Ad, diag, (T)c_d, (T)c_r, last); note_launch();
  return cudaGetLastError();
}


// Stored linearisation from the tiled layout to the canonical order [67][N_q]
// (the off-diagonal phase-gradient words of mapped meshes are not exported).
__global__ void k_untile(const double* __restrict__ lin, double* __restrict__ out, long long nq, int Q) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int Q2 = Q * Q, Q3 = Q2 * Q, EB = elems_per_block(Q);
  const long long e = q / Q3;
  const int lq = (int)(q % Q3);
  const int i = lq % Q, j = (lq / Q) % Q, k = lq / Q2;
  const long long stride = (long long)Q3 * EB;
  const long long base = (e / EB) * kLinWords * stride + (long long)k * Q2 * EB + (e % EB) * Q2 + j * Q + i;
  for (int w = 0; w < kLinWordsExport; ++w) out[w * nq + q] = lin[base + w * stride];
}
cudaError_t launch_untile(const double* lin, double* out, long long nq, int Q, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  k_untile<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(lin, out, nq, Q); note_launch();
  return cudaGetLastError();
}


// z = ubar on Dirichlet DoFs (other entries untouched).
__global__ void k_apply_dirichlet(double* __restrict__ z, const double* __restrict__ ubar,
                                  const uint8_t* __restrict__ mask, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (mask[i]) z[i] = ubar ? ubar[i] : 0.0;
}
cudaError_t launch_apply_dirichlet(double* z, const double* ubar, const uint8_t* mask, long long n, cudaStream_t st) {
  if (n == 0 || !mask) return cudaSuccess;
  k_apply_dirichlet<<<grid_for(n), kVecThreads, 0, st>>>(z, ubar, mask, n); note_launch();
  return cudaGetLastError();
}

// out[f] += sum over nodes n with sel[f][n] of v[f][n] (FP64, per-block partial
// sums combined with atomics).
__global__ void k_masked_field_sums(const double* __restrict__ v, const uint8_t* __restrict__ sel, long long nn,
                                    double* __restrict__ out) {
  __shared__ double red[4][kVecThreads / 32];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
    for (int f = 0; f < 4; ++f)
      if (sel[f * nn + i]) s[f] += v[f * nn + i];
  for (int f = 0; f < 4; ++f) {
    double t = s[f];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[f][threadIdx.x >> 5] = t;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) t += red[threadIdx.x][w];
    atomicAdd(out + threadIdx.x, t);
  }
}
cudaError_t launch_masked_field_sums(const double* v, const uint8_t* sel, long long nn, double* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, 4 * sizeof(double), st);
  if (e != cudaSuccess || nn == 0) return e;
  k_masked_field_sums<<<grid_for(nn), kVecThreads, 0, st>>>(v, sel, nn, out); note_launch();
  return cudaGetLastError();
}

// State summary of a load step (the per-step log): out[0..2] = points whose
// flags have bit 0 (Prandtl yield), bit 1 (history active), bit 2 (theta >=
// 0); out[3], out[4] = largest and smallest nodal phase field; out[5] = nodes
// with phi > 0.9; out[6], out[7] = largest accumulated plastic strain and
// history field of the given history.  One block-reduced pass per quantity.
__device__ __forceinline__ void atomic_max_d(double* a, double v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
  unsigned long long old = *p;
  while (v > __longlong_as_double((long long)old)) {
    const unsigned long long prev = atomicCAS(p, old, (unsigned long long)__double_as_longlong(v));
    if (prev == old) break;
    old = prev;
  }
}
__device__ __forceinline__ void atomic_min_d(double* a, double v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
  unsigned long long old = *p;
  while (v < __longlong_as_double((long long)old)) {
    const unsigned long long prev = atomicCAS(p, old, (unsigned long long)__double_as_longlong(v));
    if (prev == old) break;
    old = prev;
  }
}
__global__ void k_state_summary(const uint8_t* __restrict__ flags, const double* __restrict__ hist, long long nq,
                                const double* __restrict__ phi, long long nn, double* __restrict__ out) {
  double cnt[3] = {0.0, 0.0, 0.0}, hi = -INFINITY, lo = INFINITY, n9 = 0.0, ep = -INFINITY, H = -INFINITY;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq; q += stride) {
    const unsigned f = flags[q];
    cnt[0] += (f & 1u) ? 1.0 : 0.0;
    cnt[1] += (f & 2u) ? 1.0 : 0.0;
    cnt[2] += (f & 4u) ? 1.0 : 0.0;
    ep = fmax(ep, hist[12 * nq + q]);
    H = fmax(H, hist[13 * nq + q]);
  }
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += stride) {
    const double v = phi[n];
    hi = fmax(hi, v);
    lo = fmin(lo, v);
    n9 += (v > 0.9) ? 1.0 : 0.0;
  }
  for (int off = 16; off > 0; off >>= 1) {
    for (int c = 0; c < 3; ++c) cnt[c] += __shfl_down_sync(0xffffffffu, cnt[c], off);
    hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, off));
    lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, off));
    n9 += __shfl_down_sync(0xffffffffu, n9, off);
    ep = fmax(ep, __shfl_down_sync(0xffffffffu, ep, off));
    H = fmax(H, __shfl_down_sync(0xffffffffu, H, off));
  }
  if ((threadIdx.x & 31) == 0) {
    for (int c = 0; c < 3; ++c) atomicAdd(out + c, cnt[c]);
    atomic_max_d(out + 3, hi);
    atomic_min_d(out + 4, lo);
    atomicAdd(out + 5, n9);
    atomic_max_d(out + 6, ep);
    atomic_max_d(out + 7, H);
  }
}
__global__ void k_state_summary_init(double* out) {
  if (threadIdx.x < 8) out[threadIdx.x] = (threadIdx.x == 3 || threadIdx.x >= 6) ? -INFINITY
                                          : (threadIdx.x == 4 ? INFINITY : 0.0);
}
cudaError_t launch_state_summary(const uint8_t* flags, const double* hist, long long nq, const double* phi,
                                 long long nn, double* out, cudaStream_t st) {
  k_state_summary_init<<<1, 32, 0, st>>>(out); note_launch();
  k_state_summary<<<grid_for(nq > nn ? nq : nn), kVecThreads, 0, st>>>(flags, hist, nq, phi, nn, out); note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_prolong<double>(const MeshDev&, const MeshDev&, const double*, const double*, double*,
                                            const uint8_t*, const uint8_t*, cudaStream_t);
template cudaError_t launch_prolong<float>(const MeshDev&, const MeshDev&, const float*, const float*, float*,
                                           const uint8_t*, const uint8_t*, cudaStream_t);
template cudaError_t launch_restrict<double>(const MeshDev&, const MeshDev&, const double*, const double*, double*,
                                             const uint8_t*, const uint8_t*, cudaStream_t, void*);
template cudaError_t launch_restrict<float>(const MeshDev&, const MeshDev&, const float*, const float*, float*,
                                            const uint8_t*, const uint8_t*, cudaStream_t, void*);
template cudaError_t launch_cheb_init<double>(long long, const double*, const double*, const double*, double*, double*,
                                              double, cudaStream_t);
template cudaError_t launch_cheb_init<float>(long long, const float*, const float*, const float*, float*, float*,
                                             double, cudaStream_t);
template cudaError_t launch_cheb_step<double>(long long, double*, double*, double*, const double*, const double*,
                                              double, double, int, cudaStream_t);
template cudaError_t launch_cheb_step<float>(long long, float*, float*, float*, const float*, const float*, double,
                                             double, int, cudaStream_t);

// Geometry of a mapped mesh at every quadrature point from the parent Jacobian
// J = dX / dxi (rows 3 f + al of an eval of the nodal coordinates):
// geo[3 al + A] = (J^-1)[al][A] = d xi_al / dX_A, geo[9] = w_q det J.
__global__ void k_geometry(const double* __restrict__ J, double* __restrict__ geo, Geom g, int Q, long long nq,
                           int* __restrict__ status) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double A[3][3];
  for (int f = 0; f < 3; ++f)
    for (int al = 0; al < 3; ++al) A[f][al] = J[(3 * f + al) * nq + q];
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (!(det > 0.0)) atomicOr(status, 2);
  const double r = 1.0 / det;
  double G[3][3];
  G[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) * r;
  G[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * r;
  G[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * r;
  G[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) * r;
  G[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * r;
  G[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * r;
  G[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) * r;
  G[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * r;
  G[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * r;
  for (int al = 0; al < 3; ++al)
    for (int B = 0; B < 3; ++B) geo[(3 * al + B) * nq + q] = G[al][B];
  const int Q2 = Q * Q;
  const int lq = (int)(q % ((long long)Q2 * Q));
  geo[9 * nq + q] = g.wq[lq % Q] * g.wq[(lq / Q) % Q] * g.wq[lq / Q2] * det;
}
cudaError_t launch_geometry(const double* J, double* geo, const Geom& g, int Q, long long nq, int* status,
                            cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  k_geometry<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(J, geo, g, Q, nq, status); note_launch();
  return cudaGetLastError();
}

}  // namespace pff

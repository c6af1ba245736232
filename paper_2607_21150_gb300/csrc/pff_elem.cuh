// Element kernels of the matrix-free operator (Sec. 4):
//   y = P^T sum_el E^T [B_I; B_xi]^T W Lambda f_hat(...) [B_I; B_xi] E P x
//
// One thread block handles EB = 256 / Q^2 consecutive elements with Q*Q threads
// per element; thread (i, j) of an element owns the column of quadrature
// points (i, j, 0..Q-1).  The tensor contractions are sum-factorised through
// shared memory one direction at a time; gradients at the Gauss points use
// the collocated derivative D_c (exact because p <= Q - 1).  The pointwise
// linearisation is read from a tiled layout so that every load of a block is
// one contiguous run: in FP64, word w of slice k of block b sits at
//   b * kLinWords * Q^3 * EB + w * Q^3 * EB + k * Q^2 * EB + threadIdx.x;
// the FP32 planes group words 0..63 of a point by four (lin32_word), so that
// one 128-bit load fetches four words.
//
// The arithmetic type T is double, float or df64 (double-float pairs on the
// FP32 pipes, FP64 vectors in and out); every multiply-add goes through
// madd/mul/add so that one source serves all three.
#pragma once
#include "pff_df.cuh"
#include "pff_internal.h"

namespace pff {

template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
// Loads of the stored linearisation: the read-only path for the FP64 and FP32
// actions, streaming loads (evict-first) for the two planes of the
// double-float action (64^3 Q4: 16.0 -> 10.3 ms; the FP32 action measured
// 2.9 ms with the read-only path, 3.0 ms with streaming loads).
template <bool STREAM> __device__ __forceinline__ float ld_lin1(const float* p) { return STREAM ? __ldcs(p) : __ldg(p); }
template <bool STREAM> __device__ __forceinline__ float4 ld_lin4(const float* p) {
  return STREAM ? __ldcs(reinterpret_cast<const float4*>(p)) : __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ double madd(double c, double a, double b) { return fma(a, b, c); }
__device__ __forceinline__ float madd(float c, float a, float b) { return fmaf(a, b, c); }
__device__ __forceinline__ df64 madd(df64 c, df64 a, df64 b) { return df_madd(c, a, b); }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ df64 mul(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ df64 add(df64 a, df64 b) { return df_add(a, b); }

template <typename T> __device__ __forceinline__ T zero() { return T(0); }
template <> __device__ __forceinline__ df64 zero<df64>() { return df_make(0.0f, 0.0f); }
// storage value (vector entry or basis matrix) -> arithmetic type; FP64 ->
// double-float by integer operations (the conversion instructions run at the
// FP64 rate on GB300)
template <typename T, typename S> __device__ __forceinline__ T from_store(S x) { return (T)x; }
template <> __device__ __forceinline__ df64 from_store<df64, double>(double x) { return df_split(x); }
// arithmetic type -> vector entry
__device__ __forceinline__ double to_vec(double v) { return v; }
__device__ __forceinline__ float to_vec(float v) { return v; }
__device__ __forceinline__ double to_vec(df64 v) { return df_join(v); }
// stored linearisation word (df64: hi plane at p, lo plane at p + lo)
template <typename T>
__device__ __forceinline__ T ld_lin(const typename ElemTypes<T>::L* p, long long lo) {
  if constexpr (sizeof(T) == sizeof(typename ElemTypes<T>::L)) {
    return ldg(p);
  } else {
    return df_make(ld_lin1<true>(p), ld_lin1<true>(p + lo));
  }
}

// four consecutive words of the FP32 quad layout (df64: hi plane at p, lo
// plane at p + lo); p is 16-byte aligned
template <typename T>
__device__ __forceinline__ void ld_quad(const float* p, long long lo, T w[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 h = ld_lin4<false>(p);
    w[0] = h.x; w[1] = h.y; w[2] = h.z; w[3] = h.w;
  } else {
    const float4 h = ld_lin4<true>(p);
    const float4 l = ld_lin4<true>(p + lo);
    w[0] = df_make(h.x, l.x); w[1] = df_make(h.y, l.y); w[2] = df_make(h.z, l.z); w[3] = df_make(h.w, l.w);
  }
}

template <int P, int Q>
__device__ __forceinline__ long long node_of(const MeshDev& m, int e, int a, int b, int c) {
  if (m.offsets) return m.offsets[(long long)e * (P * P * P) + a + P * (b + P * c)];
  int ex = e % m.nx;
  int t = e / m.nx;
  int ey = t % m.ny;
  int ez = t / m.ny;
  return (long long)(m.p * ex + a) + (long long)m.nnx * ((long long)(m.p * ey + b) + (long long)m.nny * (m.p * ez + c));
}

// Shared-memory layout per element: two ping-pong buffers of 4 fields x Q^3
// values and a slice buffer of 8 x Q^2 values (x- and y-derivative outputs of
// the four fields at one k).  The FP32 action ("split" form) instead keeps the
// x- and y-derivative outputs of all Q slices, 8 x Q^3 values starting at the
// second buffer, so that its pointwise stage runs without barriers.
template <int Q> __host__ __device__ constexpr int elem_smem_words() { return 8 * Q * Q * Q + 8 * Q * Q; }
template <typename T> __host__ __device__ constexpr bool elem_split() { return sizeof(T) == 4; }
template <int Q, typename T> __host__ __device__ constexpr int elem_smem_words_t() {
  return elem_split<T>() ? 12 * Q * Q * Q : elem_smem_words<Q>();
}

template <int P, int Q, typename T>
struct ElemSmem {
  T* bufA;  // [4][Q^3]
  T* bufB;  // [4][Q^3]
  T* slice; // [8][Q^2]
  const T* B;
  const T* Dc;
  const T* Dt;
};

// Gather x into bufA [4][c][b][a] (masked entries zero).
template <int P, int Q, typename T>
__device__ __forceinline__ void gather(const ElemArgs<T>& a, T* bufA, int e, bool valid, int ij) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q, P3 = P * P * P;
  const long long nn = a.mesh.nn;
  // the node mask is read only for elements flagged as having masked nodes
  const bool masked = a.mask && valid && (!a.emask || a.emask[e]);
  // every thread's gather loads (values and mask bytes) are independent and
  // issued together: one memory round trip instead of one per node and a
  // second one behind each mask byte
#pragma unroll
  for (int r = 0; r < (P3 + Q2 - 1) / Q2; ++r) {
    const int idx = ij + r * Q2;
    if (idx >= P3) break;
    int aa = idx % P, bb = (idx / P) % P, cc = idx / (P * P);
    long long n = valid ? node_of<P, Q>(a.mesh, e, aa, bb, cc) : 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      T v = zero<T>();
      if (valid) {
        long long g = f * nn + n;
        const auto xv = ldg(a.x + g);
        const bool fixed = masked && ldg(a.mask + g);
        if (!fixed) v = from_store<T>(xv);
      }
      bufA[f * Q3 + idx] = v;
    }
  }
}

// Forward: gather x into bufA, interpolate to Gauss points into bufB.
template <int P, int Q, typename T>
__device__ __forceinline__ void forward(const ElemArgs<T>& a, const ElemSmem<P, Q, T>& s, int e, bool valid, int ij) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  gather<P, Q, T>(a, s.bufA, e, valid, ij);
  __syncthreads();
  // x: [c][b][a] -> [c][b][i]
  for (int idx = ij; idx < P * P * Q; idx += Q2) {
    int i = idx % Q, r = idx / Q;  // r = b + P c
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T* in = s.bufA + f * Q3 + r * P;
      T acc = zero<T>();
#pragma unroll
      for (int k = 0; k < P; ++k) acc = madd(acc, s.B[i * P + k], in[k]);
      s.bufB[f * Q3 + idx] = acc;
    }
  }
  __syncthreads();
  // y: [c][b][i] -> [c][j][i]
  for (int idx = ij; idx < P * Q * Q; idx += Q2) {
    int i = idx % Q, j = (idx / Q) % Q, c = idx / Q2;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T* in = s.bufB + f * Q3 + c * (P * Q) + i;
      T acc = zero<T>();
#pragma unroll
      for (int k = 0; k < P; ++k) acc = madd(acc, s.B[j * P + k], in[k * Q]);
      s.bufA[f * Q3 + idx] = acc;
    }
  }
  __syncthreads();
  // z: [c][j][i] -> [k][j][i]
  {
    const int i = ij % Q, j = ij / Q;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      T col[P];
#pragma unroll
      for (int c = 0; c < P; ++c) col[c] = s.bufA[f * Q3 + c * Q2 + j * Q + i];
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        T acc = zero<T>();
#pragma unroll
        for (int c = 0; c < P; ++c) acc = madd(acc, s.B[k * P + c], col[c]);
        s.bufB[f * Q3 + k * Q2 + j * Q + i] = acc;
      }
    }
  }
  __syncthreads();
}

// The 1D interpolation matrix B [Q][P] as kernel parameters, read as
// constant-bank operands where the index is fixed at compile time.
__device__ __forceinline__ float basis_b(const ElemArgs<float>& a, int idx) { return a.cB[idx]; }

// Interpolation to the Gauss points as line transforms (the persistent FP32
// kernel; the double-float action measured slower with them, 9.7 -> 9.9 ms at
// 64^3 Q4, its registers being the tighter limit): each thread takes whole
// lines (P inputs in registers, Q outputs),
// with the 1D matrix as kernel-parameter operands, so that a stage costs P
// loads and Q stores of shared memory per line instead of two loads per
// multiply-add, and a line's Q outputs are independent chains.  From bufA
// [4][c][b][a] (gathered); x: -> bufB [4][c][b][i]; y: -> bufA [4][c][j][i];
// z: -> bufB [4][k][j][i].
template <int P, int Q, typename T>
__device__ __forceinline__ void fwd_lines(const ElemArgs<T>& a, T* bufA, T* bufB, int ij) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < (4 * P * P + Q2 - 1) / Q2; ++r) {  // x: lines (f, c, b)
    const int L = ij + r * Q2;
    if (L >= 4 * P * P) break;
    const int f = L / (P * P), cb = L % (P * P);
    const T* in = bufA + f * Q3 + cb * P;
    T v[P];
#pragma unroll
    for (int aa = 0; aa < P; ++aa) v[aa] = in[aa];
    T* out = bufB + f * Q3 + cb * Q;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      T acc = zero<T>();
#pragma unroll
      for (int aa = 0; aa < P; ++aa) acc = madd(acc, basis_b(a, i * P + aa), v[aa]);
      out[i] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < (4 * P * Q + Q2 - 1) / Q2; ++r) {  // y: lines (f, c, i)
    const int L = ij + r * Q2;
    if (L >= 4 * P * Q) break;
    const int f = L / (P * Q), ci = L % (P * Q), c = ci / Q, i = ci % Q;
    const T* in = bufB + f * Q3 + c * (P * Q) + i;
    T v[P];
#pragma unroll
    for (int b = 0; b < P; ++b) v[b] = in[b * Q];
    T* out = bufA + f * Q3 + c * Q2 + i;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      T acc = zero<T>();
#pragma unroll
      for (int b = 0; b < P; ++b) acc = madd(acc, basis_b(a, j * P + b), v[b]);
      out[j * Q] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int f = 0; f < 4; ++f) {  // z: the thread's own column (j, i) of every field
    T v[P];
#pragma unroll
    for (int c = 0; c < P; ++c) v[c] = bufA[f * Q3 + c * Q2 + ij];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T acc = zero<T>();
#pragma unroll
      for (int c = 0; c < P; ++c) acc = madd(acc, basis_b(a, k * P + c), v[c]);
      bufB[f * Q3 + k * Q2 + ij] = acc;
    }
  }
  __syncthreads();
}

// Transposed interpolation as line transforms, from the accumulated column
// values Y[f][k] of the thread's own column, then the scatter-add (or the
// element values of the deterministic transpose): z (registers) -> bufA
// [4][c][j][i]; y: -> bufB [4][c][b][i]; x: -> bufA [4][c][b][a].  em: the
// element has masked nodes.
template <int P, int Q, typename T>
__device__ __forceinline__ void bwd_lines(const ElemArgs<T>& a, T* bufA, T* bufB, int e, bool valid, bool em, int ij,
                                          const T Y[4][Q]) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q, P3 = P * P * P;
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int c = 0; c < P; ++c) {
      T acc = zero<T>();
#pragma unroll
      for (int k = 0; k < Q; ++k) acc = madd(acc, basis_b(a, k * P + c), Y[f][k]);
      bufA[f * Q3 + c * Q2 + ij] = acc;
    }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < (4 * P * Q + Q2 - 1) / Q2; ++r) {  // y: lines (f, c, i)
    const int L = ij + r * Q2;
    if (L >= 4 * P * Q) break;
    const int f = L / (P * Q), ci = L % (P * Q), c = ci / Q, i = ci % Q;
    const T* in = bufA + f * Q3 + c * Q2 + i;
    T v[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) v[j] = in[j * Q];
    T* out = bufB + f * Q3 + c * (P * Q) + i;
#pragma unroll
    for (int b = 0; b < P; ++b) {
      T acc = zero<T>();
#pragma unroll
      for (int j = 0; j < Q; ++j) acc = madd(acc, basis_b(a, j * P + b), v[j]);
      out[b * Q] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < (4 * P * P + Q2 - 1) / Q2; ++r) {  // x: lines (f, c, b)
    const int L = ij + r * Q2;
    if (L >= 4 * P * P) break;
    const int f = L / (P * P), cb = L % (P * P);
    const T* in = bufB + f * Q3 + cb * Q;
    T v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = in[i];
    T* out = bufA + f * Q3 + cb * P;
#pragma unroll
    for (int aa = 0; aa < P; ++aa) {
      T acc = zero<T>();
#pragma unroll
      for (int i = 0; i < Q; ++i) acc = madd(acc, basis_b(a, i * P + aa), v[i]);
      out[aa] = acc;
    }
  }
  __syncthreads();
  if (!valid) return;
  if (a.evec) {  // deterministic transpose: element-local values, summed per node by k_node_gather
    using V = typename ElemTypes<T>::V;
    V* ev = static_cast<V*>(a.evec) + (long long)e * 4 * P3;
    for (int idx = ij; idx < P3; idx += Q2)
#pragma unroll
      for (int f = 0; f < 4; ++f) ev[f * P3 + idx] = to_vec(bufA[f * Q3 + idx]);
    return;
  }
  const long long nn = a.mesh.nn;
  const bool masked = a.mask && em;
#pragma unroll
  for (int r = 0; r < (P3 + Q2 - 1) / Q2; ++r) {
    const int idx = ij + r * Q2;
    if (idx >= P3) break;
    const int aa = idx % P, bb = (idx / P) % P, cc = idx / (P * P);
    const long long n = node_of<P, Q>(a.mesh, e, aa, bb, cc);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const long long g = f * nn + n;
      if (masked && __ldg(a.mask + g)) continue;
      atomicAdd(a.y + g, to_vec(bufA[f * Q3 + idx]));
    }
  }
}

// Parent-frame gradients of the four fields at point (i, j, k) from bufB.
template <int P, int Q, typename T>
__device__ __forceinline__ void grad_at(const ElemSmem<P, Q, T>& s, int i, int j, int k, T g[4][3], T& phi) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const T* V = s.bufB + f * Q3;
    T gx = zero<T>(), gy = zero<T>(), gz = zero<T>();
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      gx = madd(gx, s.Dc[i * Q + m], V[k * Q2 + j * Q + m]);
      gy = madd(gy, s.Dc[j * Q + m], V[k * Q2 + m * Q + i]);
      gz = madd(gz, s.Dc[k * Q + m], V[m * Q2 + j * Q + i]);
    }
    g[f][0] = gx; g[f][1] = gy; g[f][2] = gz;
  }
  phi = s.bufB[3 * Q3 + k * Q2 + j * Q + i];
}

// Backward: from accumulated column values Y[f][k] (transposed derivative
// already applied) to nodal element values, then scatter-add.
template <int P, int Q, typename T>
__device__ __forceinline__ void backward(const ElemArgs<T>& a, const ElemSmem<P, Q, T>& s, int e, bool valid, int ij,
                                         T Y[4][Q]) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q, P3 = P * P * P;
  const int i = ij % Q, j = ij / Q;
  // z (registers): [k][j][i] -> [c][j][i]
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int c = 0; c < P; ++c) {
      T acc = zero<T>();
#pragma unroll
      for (int k = 0; k < Q; ++k) acc = madd(acc, s.B[k * P + c], Y[f][k]);
      s.bufA[f * Q3 + c * Q2 + j * Q + i] = acc;
    }
  __syncthreads();
  // y: [c][j][i] -> [c][b][i]
  for (int idx = ij; idx < P * P * Q; idx += Q2) {
    int ii = idx % Q, bb = (idx / Q) % P, c = idx / (P * Q);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T* in = s.bufA + f * Q3 + c * Q2 + ii;
      T acc = zero<T>();
#pragma unroll
      for (int jj = 0; jj < Q; ++jj) acc = madd(acc, s.B[jj * P + bb], in[jj * Q]);
      s.bufB[f * Q3 + idx] = acc;
    }
  }
  __syncthreads();
  // x: [c][b][i] -> [c][b][a]
  for (int idx = ij; idx < P3; idx += Q2) {
    int aa = idx % P, r = idx / P;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T* in = s.bufB + f * Q3 + r * Q;
      T acc = zero<T>();
#pragma unroll
      for (int ii = 0; ii < Q; ++ii) acc = madd(acc, s.B[ii * P + aa], in[ii]);
      s.bufA[f * Q3 + idx] = acc;
    }
  }
  __syncthreads();
  if (!valid) return;
  if (a.evec) {  // deterministic transpose: element-local values, summed per node by k_node_gather
    using V = typename ElemTypes<T>::V;
    V* ev = static_cast<V*>(a.evec) + (long long)e * 4 * P3;
    for (int idx = ij; idx < P3; idx += Q2)
#pragma unroll
      for (int f = 0; f < 4; ++f) ev[f * P3 + idx] = to_vec(s.bufA[f * Q3 + idx]);
    return;
  }
  const long long nn = a.mesh.nn;
  const bool masked = a.mask && (!a.emask || a.emask[e]);
#pragma unroll
  for (int r = 0; r < (P3 + Q2 - 1) / Q2; ++r) {
    const int idx = ij + r * Q2;
    if (idx >= P3) break;
    int aa = idx % P, bb = (idx / P) % P, cc = idx / (P * P);
    long long n = node_of<P, Q>(a.mesh, e, aa, bb, cc);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      long long g = f * nn + n;
      if (masked && ldg(a.mask + g)) continue;
      atomicAdd(a.y + g, to_vec(s.bufA[f * Q3 + idx]));
    }
  }
}

// Pointwise linear map of the Jacobian with the stored words (already scaled
// by the quadrature weight and the parent-to-reference factors).
template <typename T>
__device__ __forceinline__ void jac_point(const typename ElemTypes<T>::L* lin, const typename ElemTypes<T>::L* linP,
                                          const typename ElemTypes<T>::L* linC, long long stride, long long lo,
                                          int kx, const T g[4][3], T phi, T o[4][3], T& o0) {
  T gu[9];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int al = 0; al < 3; ++al) gu[3 * f + al] = g[f][al];
  T ou[9];
#pragma unroll
  for (int m = 0; m < 9; ++m) ou[m] = mul(ld_lin<T>(linP + m * stride, lo), phi);
  // symmetric 9x9 block
#pragma unroll
  for (int m = 0; m < 9; ++m) {
#pragma unroll
    for (int n = m; n < 9; ++n) {
      T A = ld_lin<T>(lin + (long long)sym9(m, n) * stride, lo);
      ou[m] = madd(ou[m], A, gu[n]);
      if (n != m) ou[n] = madd(ou[n], A, gu[m]);
    }
  }
  T s0 = mul(ld_lin<T>(lin + kWD * stride, lo), phi);
#pragma unroll
  for (int m = 0; m < 9; ++m) s0 = madd(s0, ld_lin<T>(linC + m * stride, lo), gu[m]);
  o0 = s0;
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int al = 0; al < 3; ++al) o[f][al] = ou[3 * f + al];
#pragma unroll
  for (int al = 0; al < 3; ++al) o[3][al] = mul(ld_lin<T>(lin + (kWK + al) * stride, lo), g[3][al]);
  if (kx) {  // mapped mesh: symmetric off-diagonal coefficients 01, 02, 12
    const T k01 = ld_lin<T>(lin + (kWKX + 0) * stride, lo);
    const T k02 = ld_lin<T>(lin + (kWKX + 1) * stride, lo);
    const T k12 = ld_lin<T>(lin + (kWKX + 2) * stride, lo);
    o[3][0] = madd(madd(o[3][0], k01, g[3][1]), k02, g[3][2]);
    o[3][1] = madd(madd(o[3][1], k01, g[3][0]), k12, g[3][2]);
    o[3][2] = madd(madd(o[3][2], k02, g[3][0]), k12, g[3][1]);
  }
}

// The same map reading the FP32 planes in the quad layout: q = the point's
// first quad (quads at stride qs), tl = its word 64 (tail words at stride ts).
// Every quad is used as it arrives, in word order: the 9x9 block, dP/dphi and
// d(s_phi L)/dF (their roles swapped for the transpose, TR), d(s_phi L)/dphi.
template <typename T, bool TR>
__device__ __forceinline__ void jac_point_q(const float* q, long long qs, const float* tl, long long ts, long long lo,
                                            int kx, const T g[4][3], T phi, T o[4][3], T& o0) {
  T gu[9];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int al = 0; al < 3; ++al) gu[3 * f + al] = g[f][al];
  T ou[9], s0 = zero<T>();
#pragma unroll
  for (int m = 0; m < 9; ++m) ou[m] = zero<T>();
  T cur[4];
#pragma unroll
  for (int m = 0; m < 9; ++m) {  // upper triangle of the symmetric 9x9 block, row-major
#pragma unroll
    for (int n = m; n < 9; ++n) {
      const int wd = sym9(m, n);
      if ((wd & 3) == 0) ld_quad<T>(q + (wd >> 2) * qs, lo, cur);
      const T w = cur[wd & 3];
      ou[m] = madd(ou[m], w, gu[n]);
      if (n != m) ou[n] = madd(ou[n], w, gu[m]);
    }
  }
#pragma unroll
  for (int wd = kWP; wd < kLinQuadWords; ++wd) {  // the quad of word 44 is loaded
    if ((wd & 3) == 0) ld_quad<T>(q + (wd >> 2) * qs, lo, cur);
    const T w = cur[wd & 3];
    if (wd < kWC) {
      if (TR) s0 = madd(s0, w, gu[wd - kWP]);
      else ou[wd - kWP] = madd(ou[wd - kWP], w, phi);
    } else if (wd < kWD) {
      if (TR) ou[wd - kWC] = madd(ou[wd - kWC], w, phi);
      else s0 = madd(s0, w, gu[wd - kWC]);
    } else {
      s0 = madd(s0, w, phi);
    }
  }
  o0 = s0;
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int al = 0; al < 3; ++al) o[f][al] = ou[3 * f + al];
#pragma unroll
  for (int al = 0; al < 3; ++al) o[3][al] = mul(ld_lin<T>(tl + al * ts, lo), g[3][al]);
  if (kx) {  // mapped mesh: symmetric off-diagonal coefficients 01, 02, 12
    const T k01 = ld_lin<T>(tl + 3 * ts, lo);
    const T k02 = ld_lin<T>(tl + 4 * ts, lo);
    const T k12 = ld_lin<T>(tl + 5 * ts, lo);
    o[3][0] = madd(madd(o[3][0], k01, g[3][1]), k02, g[3][2]);
    o[3][1] = madd(madd(o[3][1], k01, g[3][0]), k12, g[3][2]);
    o[3][2] = madd(madd(o[3][2], k02, g[3][0]), k12, g[3][1]);
  }
}

// Jacobian map at point (slice k, thread t) of this block: FP64 planar words
// or the FP32 quad layout.
template <int Q, typename T>
__device__ __forceinline__ void jac_at(const ElemArgs<T>& a, int k, int t, const T g[4][3], T phi, T o[4][3], T& o0) {
  constexpr long long EB = elems_per_block(Q);
  constexpr long long run = (long long)Q * Q * EB, stride = run * Q;
  const long long blk = (a.blk0 + blockIdx.x) * (long long)kLinWords * stride;
  if constexpr (sizeof(typename ElemTypes<T>::L) == 4) {
    const float* q = a.lin + blk + lin32_word(0, k, t, stride, run);
    const float* tl = a.lin + blk + lin32_word(kLinQuadWords, k, t, stride, run);
    if (a.transpose) jac_point_q<T, true>(q, 4 * stride, tl, stride, a.lo, a.kx, g, phi, o, o0);
    else jac_point_q<T, false>(q, 4 * stride, tl, stride, a.lo, a.kx, g, phi, o, o0);
  } else {
    const long long off = blk + (long long)k * run + t;
    jac_point<T>(a.lin + off, a.linP + off, a.linC + off, stride, a.lo, a.kx, g, phi, o, o0);
  }
}

// L2 prefetch of slice k of this block's stored linearisation (FP32 action):
// threads 0..15 request the contiguous run of one quad plane (4 Q^2 EB words),
// the next three (six on mapped meshes) the run of one tail word (Q^2 EB words),
// each with one bulk prefetch, so the next slice streams from HBM while this
// one computes (64^3 Q4: 3.76 -> 3.48 ms; two or three slices ahead measured
// slower).  The double-float action does not prefetch: with the same requests
// for both of its planes it took 14.2 ms instead of 10.4 ms.  Tail runs
// start on 8-byte boundaries; the request is widened to 16-byte boundaries and
// clipped to the plane.
constexpr int kPrefetchAhead = 1;  // slices requested ahead of the one computed
__device__ __forceinline__ void prefetch_run(uintptr_t base, long long first, long long run, long long plane) {
  const uintptr_t lo = (base + 4 * first) & ~uintptr_t(15);
  uintptr_t hi = (base + 4 * (first + run) + 15) & ~uintptr_t(15);
  const uintptr_t end = (base + 4 * plane) & ~uintptr_t(15);
  if (hi > end) hi = end;
  if (hi <= lo) return;
  asm volatile(
      "{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tcp.async.bulk.prefetch.L2.global [ga], %1;\n\t}"
      :: "l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}
template <int Q, typename T>
__device__ __forceinline__ void prefetch_slice(const ElemArgs<T>& a, int k, int t) {
  if constexpr (sizeof(T) == 4) {
    constexpr int EB = elems_per_block(Q);
    constexpr long long run = (long long)Q * Q * EB;   // words of one (word, slice) run
    constexpr int NQ = kLinQuadWords / 4;
    if (t >= NQ + (a.kx ? kLinWords - kLinQuadWords : kWKX - kLinQuadWords) || k >= Q) return;
    const long long nblk = (a.mesh.nel + EB - 1) / EB;
    const long long plane = nblk * kLinWords * Q * Q * Q * EB;
    const long long blk = (a.blk0 + blockIdx.x) * kLinWords * Q * run;
    const uintptr_t base = reinterpret_cast<uintptr_t>(a.lin);
    if (t < NQ) prefetch_run(base, blk + lin32_word(4 * t, k, 0, Q * run, run), 4 * run, plane);
    else prefetch_run(base, blk + lin32_word(kLinQuadWords + t - NQ, k, 0, Q * run, run), run, plane);
  }
}

// Entry k of a thread's column accumulators when k is not a compile-time
// constant: selects over the unrolled entries, so the column stays in
// registers.
template <int Q, typename T>
__device__ __forceinline__ T column_at(const T (&y)[Q], int k) {
  T v = y[0];
#pragma unroll
  for (int kk = 1; kk < Q; ++kk)
    if (kk == k) v = y[kk];
  return v;
}
template <int Q, typename T>
__device__ __forceinline__ void set_column_at(T (&y)[Q], int k, T v) {
#pragma unroll
  for (int kk = 0; kk < Q; ++kk)
    if (kk == k) y[kk] = v;
}

// Resident blocks per SM the register allocation is held to (Q = 5: 250
// threads per block, 97 KB of shared memory at 8-byte words): two for FP64 and
// double-float (<= 128 registers), three for FP32 (<= 85 registers).  With a
// single resident block the barriers of the slice loop leave the SM idle.
template <typename T> constexpr int elem_min_blocks() { return sizeof(T) == 4 ? 3 : 2; }

template <int P, int Q, typename T, int MODE>
__global__ void __launch_bounds__(Q * Q * elems_per_block(Q), elem_min_blocks<T>())
k_elem(const ElemArgs<T> a) {
  constexpr int EB = elems_per_block(Q);
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int t = threadIdx.x;
  const int el = t / Q2, ij = t % Q2;
  const int i = ij % Q, j = ij / Q;
  const int e = (a.blk0 + blockIdx.x) * EB + el;
  const bool valid = e < a.mesh.nel;

  T* mats = sm;
  T* Bs = mats;
  T* Dcs = Bs + Q * P;
  for (int idx = t; idx < Q * P; idx += blockDim.x) Bs[idx] = from_store<T>(a.B[idx]);
  for (int idx = t; idx < Q * Q; idx += blockDim.x) Dcs[idx] = from_store<T>(a.Dc[idx]);
  constexpr bool kSplit = elem_split<T>() && MODE == kApply;
  T* base = sm + mat_smem_words<P, Q>() + el * elem_smem_words_t<Q, T>();
  // split form: bufB first (read by every slice's gradients), then bufA which
  // extends to the 8 x Q^3 derivative outputs of the pointwise stage
  ElemSmem<P, Q, T> s = kSplit ? ElemSmem<P, Q, T>{base + 4 * Q3, base, nullptr, Bs, Dcs, nullptr}
                               : ElemSmem<P, Q, T>{base, base + 4 * Q3, base + 8 * Q3, Bs, Dcs, nullptr};
  __syncthreads();
  if constexpr (kSplit)
    for (int k = 0; k < kPrefetchAhead; ++k) prefetch_slice<Q, T>(a, k, t);

  if constexpr (MODE == kApply || MODE == kEval) forward<P, Q, T>(a, s, e, valid, ij);

  if constexpr (MODE == kEval) {
    if (valid) {
      T sd[3];  // d xi / dX of the box
#pragma unroll
      for (int al = 0; al < 3; ++al) sd[al] = from_store<T>(a.s[al]);
#pragma unroll 1
      for (int k = 0; k < Q; ++k) {
        T g[4][3], phi;
        grad_at<P, Q, T>(s, i, j, k, g, phi);
        long long q = (long long)e * Q3 + k * Q2 + j * Q + i;
        if (a.geo) {  // mapped mesh: reference gradient = parent gradient x d xi / dX
          T G[3][3];
#pragma unroll
          for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int A = 0; A < 3; ++A) G[al][A] = from_store<T>(a.geo[(3 * al + A) * a.nq + q]);
#pragma unroll
          for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int A = 0; A < 3; ++A) {
              const T v = madd(madd(mul(g[f][0], G[0][A]), g[f][1], G[1][A]), g[f][2], G[2][A]);
              a.scratch[((f < 3) ? 3 * f + A : 10 + A) * a.nq + q] = to_vec(v);
            }
        } else {
#pragma unroll
          for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int al = 0; al < 3; ++al) a.scratch[(3 * f + al) * a.nq + q] = to_vec(mul(g[f][al], sd[al]));
#pragma unroll
          for (int al = 0; al < 3; ++al) a.scratch[(10 + al) * a.nq + q] = to_vec(mul(g[3][al], sd[al]));
        }
        a.scratch[9 * a.nq + q] = to_vec(phi);
      }
    }
    return;
  }

  T Y[4][Q];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int k = 0; k < Q; ++k) Y[f][k] = zero<T>();

  if constexpr (kSplit) {
    // pointwise stage of all slices without barriers: z-derivative and value
    // terms into the registers of the own column, x- and y-derivative outputs
    // to shared memory
    T* oxy = s.bufA;  // [8][Q^3]
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      T g[4][3], phi, o[4][3], o0 = zero<T>();
      prefetch_slice<Q, T>(a, k + kPrefetchAhead, t);
      grad_at<P, Q, T>(s, i, j, k, g, phi);
      if (valid) {
        jac_at<Q, T>(a, k, t, g, phi, o, o0);
      } else {
#pragma unroll
        for (int f = 0; f < 4; ++f) o[f][0] = o[f][1] = o[f][2] = zero<T>();
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) Y[f][kk] = madd(Y[f][kk], s.Dc[k * Q + kk], o[f][2]);
        oxy[(2 * f) * Q3 + k * Q2 + ij] = o[f][0];
        oxy[(2 * f + 1) * Q3 + k * Q2 + ij] = o[f][1];
      }
      Y[3][k] = add(Y[3][k], o0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const T* ox = oxy + (2 * f) * Q3 + k * Q2;
        const T* oy = oxy + (2 * f + 1) * Q3 + k * Q2;
        T acc = Y[f][k];
#pragma unroll
        for (int m = 0; m < Q; ++m) {
          acc = madd(acc, s.Dc[m * Q + i], ox[j * Q + m]);
          acc = madd(acc, s.Dc[m * Q + j], oy[m * Q + i]);
        }
        Y[f][k] = acc;
      }
    __syncthreads();  // the derivative outputs are read; backward reuses the buffers
    backward<P, Q, T>(a, s, e, valid, ij, Y);
    return;
  }
  // The double-float action keeps this loop rolled: its pointwise map takes
  // about ten times the instructions of the FP64 one, and five unrolled
  // slices, each with both orientations of the map, overflow the instruction
  // cache.  Y[f][k] is then selected and written back by column_at /
  // set_column_at; o0 joins Y[3][k] after the barrier, in the same order of
  // operations as the FP64 loop.
  constexpr bool kRollSlices = sizeof(T) != sizeof(typename ElemTypes<T>::L);
#pragma unroll(kRollSlices ? 1 : Q)
  for (int k = 0; k < Q; ++k) {
    T o[4][3], o0 = zero<T>();
    if constexpr (MODE == kApply) {
      T g[4][3], phi;
      grad_at<P, Q, T>(s, i, j, k, g, phi);
      if (valid) {
        jac_at<Q, T>(a, k, t, g, phi, o, o0);
      } else {
#pragma unroll
        for (int f = 0; f < 4; ++f) o[f][0] = o[f][1] = o[f][2] = zero<T>();
      }
    } else {  // kBack: integrands from the pointwise kernel
      if (valid) {
        long long q = (long long)e * Q3 + k * Q2 + j * Q + i;
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
          for (int al = 0; al < 3; ++al) o[f][al] = from_store<T>(a.scratch[(3 * f + al) * a.nq + q]);
        o0 = from_store<T>(a.scratch[9 * a.nq + q]);
#pragma unroll
        for (int al = 0; al < 3; ++al) o[3][al] = from_store<T>(a.scratch[(10 + al) * a.nq + q]);
      } else {
#pragma unroll
        for (int f = 0; f < 4; ++f) o[f][0] = o[f][1] = o[f][2] = zero<T>();
      }
    }
    // transposed z-derivative (own column) and the value term
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int kk = 0; kk < Q; ++kk) Y[f][kk] = madd(Y[f][kk], s.Dc[k * Q + kk], o[f][2]);
    if constexpr (!kRollSlices) Y[3][k] = add(Y[3][k], o0);
    // x- and y-derivative outputs of this slice through shared memory
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      s.slice[(2 * f) * Q2 + ij] = o[f][0];
      s.slice[(2 * f + 1) * Q2 + ij] = o[f][1];
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      T acc;
      if constexpr (kRollSlices) {
        acc = column_at<Q>(Y[f], k);
        if (f == 3) acc = add(acc, o0);
      } else {
        acc = Y[f][k];
      }
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        acc = madd(acc, s.Dc[m * Q + i], s.slice[(2 * f) * Q2 + j * Q + m]);
        acc = madd(acc, s.Dc[m * Q + j], s.slice[(2 * f + 1) * Q2 + m * Q + i]);
      }
      if constexpr (kRollSlices) set_column_at<Q>(Y[f], k, acc);
      else Y[f][k] = acc;
    }
    __syncthreads();
  }
  backward<P, Q, T>(a, s, e, valid, ij, Y);
}

// Diagonal of the element operators: for each field f and node a,
//   sum_q sum_{alpha,beta} D_{f alpha, f beta}(q) d_alpha N_a d_beta N_a
// (+ the value term of the phase field), sum-factorised per (alpha, beta)
// pair with the 1D products B*B, B*D, D*D.
template <int P, int Q, typename T>
__global__ void __launch_bounds__(Q * Q * elems_per_block(Q))
k_diag(const ElemArgs<T> a) {
  constexpr int EB = elems_per_block(Q);
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q, P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int t = threadIdx.x;
  const int el = t / Q2, ij = t % Q2;
  const int i = ij % Q, j = ij / Q;
  const int e = (a.blk0 + blockIdx.x) * EB + el;
  const bool valid = e < a.mesh.nel;
  T* M = sm;  // [3][Q][P]: BB, BD, DD
  for (int idx = t; idx < Q * P; idx += blockDim.x) {
    T b = a.B[idx], d = a.Dt[idx];
    M[idx] = b * b;
    M[Q * P + idx] = b * d;
    M[2 * Q * P + idx] = d * d;
  }
  T* base = sm + mat_smem_words<P, Q>() + el * elem_smem_words<Q>();
  T* bufA = base;           // Q^3
  T* bufB = base + Q3;      // Q^3
  T* acc = base + 2 * Q3;   // [4][P3]
  for (int idx = ij; idx < 4 * P3; idx += Q2) acc[idx] = T(0);
  __syncthreads();
  const long long blk_words = (long long)kLinWords * Q3 * EB;
  const long long stride = (long long)Q3 * EB;
  // term list: (field, word, dim-kinds mask, weight)
  // u fields: pairs alpha <= beta; phase field: value term and 3 gradient terms
  const int nterms = a.kx ? 25 : 22;
#pragma unroll 1
  for (int term = 0; term < nterms; ++term) {
    int f, word, kx, ky, kz;
    T wgt = T(1);
    if (term < 18) {
      f = term / 6;
      int pr = term % 6;
      const int al_of[6] = {0, 1, 2, 0, 0, 1};
      const int be_of[6] = {0, 1, 2, 1, 2, 2};
      int al = al_of[pr], be = be_of[pr];
      word = sym9(3 * f + al, 3 * f + be);
      if (al != be) wgt = T(2);
      int kd[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) kd[d] = (d == al) + (d == be);  // 0: BB, 1: BD, 2: DD
      kx = kd[0]; ky = kd[1]; kz = kd[2];
    } else {
      f = 3;
      if (term == 18) { word = kWD; kx = ky = kz = 0; }
      else if (term < 22) {
        int al = term - 19;
        word = kWK + al;
        kx = (al == 0) ? 2 : 0; ky = (al == 1) ? 2 : 0; kz = (al == 2) ? 2 : 0;
      } else {  // off-diagonal phase-gradient pair (al, be): 2 K_al,be d_al N d_be N
        const int pr = term - 22;               // 01, 02, 12
        const int al = (pr == 2) ? 1 : 0, be = (pr == 0) ? 1 : 2;
        word = kWKX + pr;
        wgt = T(2);
        kx = (al == 0) + (be == 0); ky = (al == 1) + (be == 1); kz = (al == 2) + (be == 2);
      }
    }
    const T* Mx = M + kx * Q * P;
    const T* My = M + ky * Q * P;
    const T* Mz = M + kz * Q * P;
    // coefficients on the column (i, j, :) -> z contraction in registers
    T col[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const long long off = (a.blk0 + blockIdx.x) * blk_words + (sizeof(T) == 4 ? lin32_word(word, k, t, stride, Q2 * EB)
                                                                    : (long long)word * stride + (long long)k * Q2 * EB + t);
      col[k] = valid ? ldg(a.lin + off) * wgt : T(0);
    }
#pragma unroll
    for (int c = 0; c < P; ++c) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < Q; ++k) s += Mz[k * P + c] * col[k];
      bufA[c * Q2 + j * Q + i] = s;
    }
    __syncthreads();
    for (int idx = ij; idx < P * P * Q; idx += Q2) {
      int ii = idx % Q, bb = (idx / Q) % P, c = idx / (P * Q);
      T s = T(0);
#pragma unroll
      for (int jj = 0; jj < Q; ++jj) s += My[jj * P + bb] * bufA[c * Q2 + jj * Q + ii];
      bufB[idx] = s;
    }
    __syncthreads();
    for (int idx = ij; idx < P3; idx += Q2) {
      int aa = idx % P, r = idx / P;
      T s = T(0);
#pragma unroll
      for (int ii = 0; ii < Q; ++ii) s += Mx[ii * P + aa] * bufB[r * Q + ii];
      acc[f * P3 + idx] += s;
    }
    __syncthreads();
  }
  if (!valid) return;
  if (a.evec) {  // deterministic: element-local values, summed per node by k_node_gather
    T* ev = static_cast<T*>(a.evec) + (long long)e * 4 * P3;
    for (int idx = ij; idx < P3; idx += Q2)
#pragma unroll
      for (int f = 0; f < 4; ++f) ev[f * P3 + idx] = acc[f * P3 + idx];
    return;
  }
  const long long nn = a.mesh.nn;
  for (int idx = ij; idx < P3; idx += Q2) {
    int aa = idx % P, bb = (idx / P) % P, cc = idx / (P * P);
    long long n = node_of<P, Q>(a.mesh, e, aa, bb, cc);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      long long g = f * nn + n;
      if (a.mask && a.mask[g]) continue;
      atomicAdd(a.y + g, acc[f * P3 + idx]);
    }
  }
}

}  // namespace pff

#include "pff_elem_pipe.cuh"

namespace pff {

template <int P, int Q, typename T>
cudaError_t launch_elem_pq(int mode, const ElemArgs<T>& a, cudaStream_t st) {
  constexpr int EB = elems_per_block(Q);
  int nblk = a.nblk > 0 ? a.nblk : (a.mesh.nel + EB - 1) / EB;
  if (nblk == 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4 && sizeof(typename ElemTypes<T>::L) == 4) {  // FP32 arithmetic: persistent kernel
    if (a.lin16 && mode != kApply) return cudaErrorInvalidValue;
    if (mode == kApply) {
      cudaError_t err = cudaSuccess;
      if (launch_level_pipe<P, Q>(a, nblk, st, &err)) return err;
    }
  }
  size_t smem = sizeof(T) * (size_t)(mat_smem_words<P, Q>() + EB * elem_smem_words<Q>());
  dim3 block(Q * Q * EB);
  if (mode == kApply) smem = sizeof(T) * (size_t)(mat_smem_words<P, Q>() + EB * elem_smem_words_t<Q, T>());
  if constexpr (sizeof(T) != sizeof(typename ElemTypes<T>::L)) {  // double-float: the action only
    if (mode != kApply) return cudaErrorInvalidValue;
    auto k = k_elem<P, Q, T, kApply>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<nblk, block, smem, st>>>(a); note_launch();
  } else if (mode == kApply) {
    auto k = k_elem<P, Q, T, kApply>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<nblk, block, smem, st>>>(a); note_launch();
  } else if (mode == kEval) {
    auto k = k_elem<P, Q, T, kEval>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<nblk, block, smem, st>>>(a); note_launch();
  } else {
    auto k = k_elem<P, Q, T, kBack>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<nblk, block, smem, st>>>(a); note_launch();
  }
  return cudaGetLastError();
}

template <int P, int Q, typename T>
cudaError_t launch_diag_pq(const ElemArgs<T>& a, cudaStream_t st) {
  constexpr int EB = elems_per_block(Q);
  int nblk = (a.mesh.nel + EB - 1) / EB;
  if (nblk == 0) return cudaSuccess;
  size_t smem = sizeof(T) * (size_t)(mat_smem_words<P, Q>() + EB * elem_smem_words<Q>());
  auto k = k_diag<P, Q, T>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<nblk, Q * Q * EB, smem, st>>>(a); note_launch();
  return cudaGetLastError();
}

}  // namespace pff

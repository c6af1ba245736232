// Level action with 16-bit stored words (PFF_F32_BF16): the FP32 matrix-free
// Jacobian action of Sec. 4 (gather, sum-factorised interpolation and
// gradients, pointwise linear map with the stored linearisation, transposed
// contractions, scatter-add), reading the stored words as BF16.  The
// p-multigrid levels only precondition an FP64 (or double-float) outer solve,
// so 8 mantissa bits per word leave the outer iteration counts unchanged,
// while the word stream -- the bulk of the action's HBM traffic -- halves.
//
// Each block stages its words through shared memory: slice k of the block
// (Q^2 EB points, 136 bytes each, 144 on mapped meshes) arrives as ten 1D bulk
// copies (cp.async.bulk, completion counted in bytes on one mbarrier) while the
// block computes.  Slice 0 is requested before the gather and streams in
// during the gather and the forward contractions; slice k+1 is requested as
// soon as every thread has moved its slice-k words into registers, and
// streams in during slice k's pointwise work.  One copy per plane of a few KB
// keeps tens of KB in flight per SM however few warps are resident, which is
// what the register-load version of this kernel could not do (it stalled on
// the word loads at 48 % of HBM).
//
// Every wait on the mbarrier is bounded (about one second of clock cycles);
// a wait that runs out sets status bit 32 (the result is then invalid).  A
// wait that has already lasted about 2 ms (a thousand times a slice's usual
// latency) also gives up once that bit is set in global memory, so that after
// one block has given up the others follow quickly and the kernel ends; the
// block decides together (one barrier vote) to stop requesting slices, and
// thread 0 waits once more, again bounded, for a copy still in flight before
// the block exits.
#pragma once

namespace pff {

constexpr unsigned kStatusPipe = 32;             // status bit: a staging wait gave up
constexpr long long kStageWaitCycles = 1LL << 31;  // ~1 s at 2 GHz: give up
constexpr long long kStageFollowCycles = 1LL << 22;  // ~2 ms: give up if another wait already did

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false if it gave up (and
// then status bit 32 is set, when status is given).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0) {
      const long long dt = clock64() - t0;
      const bool others = status && dt > kStageFollowCycles && (*(volatile int*)status & kStatusPipe);
      if (others || dt > kStageWaitCycles) {
        if (status) atomicOr(status, (int)kStatusPipe);
        return false;
      }
    }
  }
}
// 1D bulk copy global -> shared, completion counted on bar.  Addresses and
// size are multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %1;\n\t"
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [ga], %2, [%3];\n\t}" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// The same copy with an L2 eviction-priority hint: the words are read once,
// so they go first and the x and y lines that neighbouring blocks reuse stay.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                              unsigned long long policy) {
  asm volatile(
      "{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %1;\n\t"
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [ga], %2, [%3], %4;\n\t}" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// L2 prefetch of the x rows that element block `blk` will gather (structured
// numbering): thread t < 4 P^2 takes field f and node row (b, c) and requests
// the row segment of each element row the block covers (16-byte rounded).
template <int P, int Q>
__device__ __forceinline__ void prefetch_x_rows(const MeshDev& m, const float* x, long long blk, int t) {
  constexpr int EB = elems_per_block(Q);
  if (m.offsets || t >= 4 * P * P || !x) return;
  const long long e0 = blk * EB;
  if (e0 >= m.nel) return;
  const long long e1 = (e0 + EB < (long long)m.nel ? e0 + EB : (long long)m.nel) - 1;
  const int f = t / (P * P), bb = t % P, cc = (t / P) % P;
  const uintptr_t end = reinterpret_cast<uintptr_t>(x + 4 * m.nn) & ~uintptr_t(15);
  for (long long es = e0; es <= e1;) {
    const int ex = (int)(es % m.nx);
    const long long row = es / m.nx;
    const int ey = (int)(row % m.ny), ez = (int)(row / m.ny);
    long long last = es + (m.nx - 1 - ex);
    if (last > e1) last = e1;
    const long long node0 =
        (long long)m.p * ex + (long long)m.nnx * ((long long)(m.p * ey + bb) + (long long)m.nny * (m.p * ez + cc));
    const long long cnt = (long long)m.p * (last - es) + m.p + 1;
    const uintptr_t base = reinterpret_cast<uintptr_t>(x + f * m.nn + node0);
    const uintptr_t lo = base & ~uintptr_t(15);
    uintptr_t hi = (base + cnt * sizeof(float) + 15) & ~uintptr_t(15);
    if (hi > end) hi = end;
    if (hi > lo)
      asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tcp.async.bulk.prefetch.L2.global [ga], %1;\n\t}" ::"l"(lo),
                   "r"((unsigned)(hi - lo))
                   : "memory");
    es = last + 1;
  }
}
// Orders this thread's earlier generic-proxy shared-memory accesses (and, after
// a barrier, the block's) before later async-proxy writes to the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// BF16 -> FP32 of the low / high half of a packed pair (exact).
__device__ __forceinline__ float bf_lo(unsigned r) { return __uint_as_float(r << 16); }
__device__ __forceinline__ float bf_hi(unsigned r) { return __uint_as_float(r & 0xffff0000u); }
template <int W> __device__ __forceinline__ float w16(const unsigned* wr) {
  return (W & 1) ? bf_hi(wr[W >> 1]) : bf_lo(wr[W >> 1]);
}

// Shared-memory bytes of one staged slice (octet planes, then the tail planes).
template <int Q> __host__ __device__ constexpr int w16_slot_bytes() {
  return 144 * Q * Q * elems_per_block(Q);
}

// The pointwise map of jac_point_q with the point's words in registers:
// wr[i] holds words 2i (low half) and 2i + 1 (high half); wr[32..33] the first
// tail plane (words 64..67), wr[34..35] the second (68..71, mapped meshes).
template <bool TR, bool KX>
__device__ __forceinline__ void jac_point_w16(const unsigned* wr, const float g[4][3], float phi, float o[4][3],
                                              float& o0) {
  float gu[9];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int al = 0; al < 3; ++al) gu[3 * f + al] = g[f][al];
  float ou[9], s0 = 0.0f;
#pragma unroll
  for (int m = 0; m < 9; ++m) ou[m] = 0.0f;
#pragma unroll
  for (int m = 0; m < 9; ++m) {  // upper triangle of the symmetric 9x9 block
#pragma unroll
    for (int n = m; n < 9; ++n) {
      const int wd = sym9(m, n);
      const float w = (wd & 1) ? bf_hi(wr[wd >> 1]) : bf_lo(wr[wd >> 1]);
      ou[m] = fmaf(w, gu[n], ou[m]);
      if (n != m) ou[n] = fmaf(w, gu[m], ou[n]);
    }
  }
#pragma unroll
  for (int wd = kWP; wd < kWK; ++wd) {
    const float w = (wd & 1) ? bf_hi(wr[wd >> 1]) : bf_lo(wr[wd >> 1]);
    if (wd < kWC) {
      if (TR) s0 = fmaf(w, gu[wd - kWP], s0);
      else ou[wd - kWP] = fmaf(w, phi, ou[wd - kWP]);
    } else if (wd < kWD) {
      if (TR) ou[wd - kWC] = fmaf(w, phi, ou[wd - kWC]);
      else s0 = fmaf(w, gu[wd - kWC], s0);
    } else {
      s0 = fmaf(w, phi, s0);
    }
  }
  o0 = s0;
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int al = 0; al < 3; ++al) o[f][al] = ou[3 * f + al];
  o[3][0] = w16<64>(wr) * g[3][0];
  o[3][1] = w16<65>(wr) * g[3][1];
  o[3][2] = w16<66>(wr) * g[3][2];
  if (KX) {  // mapped mesh: symmetric off-diagonal coefficients 01, 02, 12
    const float k01 = w16<67>(wr), k02 = w16<68>(wr), k12 = w16<69>(wr);
    o[3][0] = fmaf(k02, g[3][2], fmaf(k01, g[3][1], o[3][0]));
    o[3][1] = fmaf(k12, g[3][2], fmaf(k01, g[3][0], o[3][1]));
    o[3][2] = fmaf(k12, g[3][1], fmaf(k02, g[3][0], o[3][2]));
  }
}

// Requests slice k of this block's words into the slot (thread 0 only).
template <int Q>
__device__ __forceinline__ void w16_issue(const unsigned char* gblk, unsigned char* slot, uint64_t* bar, int k,
                                          bool kx) {
  constexpr unsigned q2eb = Q * Q * elems_per_block(Q);
  constexpr unsigned long long q3eb = (unsigned long long)Q * q2eb;
  const unsigned bytes = (kx ? 144u : 136u) * q2eb;
  const unsigned long long pol = l2_evict_first_policy();
  mbar_expect_tx(bar, bytes);
#pragma unroll
  for (int o = 0; o < 8; ++o)
    bulk_g2s_hint(slot + o * 16 * q2eb, gblk + o * 16 * q3eb + (unsigned long long)k * 16 * q2eb, 16 * q2eb, bar, pol);
  bulk_g2s_hint(slot + 128 * q2eb, gblk + 128 * q3eb + (unsigned long long)k * 8 * q2eb, 8 * q2eb, bar, pol);
  if (kx) bulk_g2s_hint(slot + 136 * q2eb, gblk + 136 * q3eb + (unsigned long long)k * 8 * q2eb, 8 * q2eb, bar, pol);
}

template <int P, int Q, bool KX, bool TR>
__global__ void __launch_bounds__(Q * Q * elems_per_block(Q), 2)
k_elem_w16(const ElemArgs<float> a) {
  constexpr int EB = elems_per_block(Q);
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  constexpr int q2eb = Q2 * EB;
  constexpr int kSlot = w16_slot_bytes<Q>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* slot = smem_raw;                               // staged slice
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kSlot);  // 16 bytes reserved
  float* sm = reinterpret_cast<float*>(smem_raw + kSlot + 16);
  const int t = threadIdx.x;
  const int el = t / Q2, ij = t % Q2;
  const int i = ij % Q, j = ij / Q;
  const int e = (a.blk0 + blockIdx.x) * EB + el;
  const bool valid = e < a.mesh.nel;
  const unsigned char* gblk =
      reinterpret_cast<const unsigned char*>(a.lin16) + (unsigned long long)(a.blk0 + blockIdx.x) * 2 * kLin16Words * Q3 * EB;

  float* Bs = sm;
  float* Dcs = Bs + Q * P;
  for (int idx = t; idx < Q * P; idx += blockDim.x) Bs[idx] = a.B[idx];
  for (int idx = t; idx < Q * Q; idx += blockDim.x) Dcs[idx] = a.Dc[idx];
  float* base = sm + mat_smem_words<P, Q>() + el * elem_smem_words_t<Q, float>();
  const ElemSmem<P, Q, float> s{base + 4 * Q3, base, nullptr, Bs, Dcs, nullptr};
  if (t == 0) mbar_init(bar, 1);
  __syncthreads();
  if (t == 0) w16_issue<Q>(gblk, slot, bar, 0, KX);
  // the fine-order level (P = Q) gathers most: warm L2 with the x rows of the
  // block that starts about one wave of resident blocks later (64^3 Q4:
  // 2.57 -> 2.46 ms together with the evict-first words; the p-levels gain nothing)
  if constexpr (P == Q)
    if (a.pf_ahead > 0) prefetch_x_rows<P, Q>(a.mesh, a.x, a.blk0 + blockIdx.x + a.pf_ahead, t);

  forward<P, Q, float>(a, s, e, valid, ij);

  float Y[4][Q];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int k = 0; k < Q; ++k) Y[f][k] = 0.0f;
  float* oxy = s.bufA;  // [8][Q^3] x- and y-derivative outputs of all slices
  bool staged = true;   // every wait of every thread so far succeeded (block-uniform)
  int last = -1;        // the last slice requested
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    last = k;
    const bool ok = mbar_wait(bar, k & 1, a.status);
    unsigned wr[36];
    {
      const uint4* oc = reinterpret_cast<const uint4*>(slot) + t;
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const uint4 v = oc[o * q2eb];
        wr[4 * o] = v.x; wr[4 * o + 1] = v.y; wr[4 * o + 2] = v.z; wr[4 * o + 3] = v.w;
      }
      const uint2 t1 = reinterpret_cast<const uint2*>(slot + 128 * q2eb)[t];
      wr[32] = t1.x; wr[33] = t1.y;
      if (KX) {
        const uint2 t2 = reinterpret_cast<const uint2*>(slot + 136 * q2eb)[t];
        wr[34] = t2.x; wr[35] = t2.y;
      } else {
        wr[34] = wr[35] = 0u;
      }
    }
    // every thread holds its words: the slot is free for the next slice,
    // unless some wait of the block gave up (then no further slice is requested)
    staged = __syncthreads_and(ok && staged) != 0;
    if (t == 0 && k + 1 < Q && staged) {
      fence_proxy_async_smem();
      w16_issue<Q>(gblk, slot, bar, k + 1, KX);
    }
    float g[4][3], phi, o[4][3], o0 = 0.0f;
    grad_at<P, Q, float>(s, i, j, k, g, phi);
    if (valid) {
      jac_point_w16<TR, KX>(wr, g, phi, o, o0);
    } else {
#pragma unroll
      for (int f = 0; f < 4; ++f) o[f][0] = o[f][1] = o[f][2] = 0.0f;
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
#pragma unroll
      for (int kk = 0; kk < Q; ++kk) Y[f][kk] = fmaf(s.Dc[k * Q + kk], o[f][2], Y[f][kk]);
      oxy[(2 * f) * Q3 + k * Q2 + ij] = o[f][0];
      oxy[(2 * f + 1) * Q3 + k * Q2 + ij] = o[f][1];
    }
    Y[3][k] += o0;
    if (!staged) break;  // no further slice was requested
  }
  // a copy of the slice whose wait gave up may still be in flight: wait for it
  // (bounded) before the block's shared memory is released
  if (!staged && t == 0) mbar_wait(bar, last & 1, nullptr);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < Q; ++k)
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float* ox = oxy + (2 * f) * Q3 + k * Q2;
      const float* oy = oxy + (2 * f + 1) * Q3 + k * Q2;
      float acc = Y[f][k];
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        acc = fmaf(s.Dc[m * Q + i], ox[j * Q + m], acc);
        acc = fmaf(s.Dc[m * Q + j], oy[m * Q + i], acc);
      }
      Y[f][k] = acc;
    }
  __syncthreads();
  backward<P, Q, float>(a, s, e, valid, ij, Y);
}

template <int P, int Q>
cudaError_t launch_elem_w16(const ElemArgs<float>& a, cudaStream_t st) {
  constexpr int EB = elems_per_block(Q);
  const int nblk = a.nblk > 0 ? a.nblk : (a.mesh.nel + EB - 1) / EB;
  if (nblk == 0) return cudaSuccess;
  const size_t smem = w16_slot_bytes<Q>() + 16 +
                      sizeof(float) * (size_t)(mat_smem_words<P, Q>() + EB * elem_smem_words_t<Q, float>());
  auto k = a.kx ? (a.transpose ? k_elem_w16<P, Q, true, true> : k_elem_w16<P, Q, true, false>)
                : (a.transpose ? k_elem_w16<P, Q, false, true> : k_elem_w16<P, Q, false, false>);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<nblk, Q * Q * EB, smem, st>>>(a); note_launch();
  return cudaGetLastError();
}

}  // namespace pff

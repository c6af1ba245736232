// Level actions in FP32 arithmetic (PFF_F32 and PFF_F32_BF16): the matrix-free
// Jacobian action of Sec. 4 (gather, sum-factorised interpolation and
// gradients, pointwise linear map with the stored linearisation, transposed
// contractions, scatter-add) as a persistent kernel whose stored-word stream
// never stops between element blocks.
//
// Two blocks of Q^2 EB threads run on each SM; each walks the element blocks
// blockIdx.x, blockIdx.x + gridDim.x, ... and owns a ring of two shared-memory
// slots.  The words of an element block arrive as a sequence of stages -- one
// per Gauss slice with BF16 words (136 bytes per point, 144 on mapped meshes),
// two per slice with FP32 words (quads 0..7, then quads 8..15 and the tail
// words) -- each a handful of 1D bulk copies (cp.async.bulk) completing on the
// slot's mbarrier.  Stage s + 2 is requested as soon as every thread has moved
// stage s into registers, whether it belongs to this element block or the
// next, so that the first two stages of block b + 1 stream in while block b
// runs its transposed contractions and scatter and block b + 1 its gather and
// forward contractions.  The nodal values of the next element block are
// loaded into registers while the present one runs its transposed contractions
// and scatter (an additional L2 prefetch of those x rows, one element block
// ahead, measured slower: 64^3 Q4 FP32 words 2.33 -> 2.19 ms without it).
//
// The x- and y-derivative outputs of slice k go through a double-buffered
// slice buffer and are contracted at the next slice, after the barrier that
// frees the slot; shared memory per element is then 8 Q^3 values (Q = 5), so
// that two slots and two blocks fit on an SM.  The interpolation and its
// transpose are line transforms (fwd_lines / bwd_lines, pff_elem.cuh) with the
// 1D matrices as kernel parameters; the slice loop stays rolled for P >= 3.
//
// Every wait on an mbarrier is bounded (about one second of clock cycles); a
// wait that runs out sets status bit 32 (the result is then invalid).  A wait
// that has already lasted about 2 ms (a thousand times a stage's usual
// latency) also gives up once that bit is set in global memory, so that after
// one block has given up the others follow quickly and the kernel ends; the
// block decides together (one barrier vote) to stop, and thread 0 waits once
// more, again bounded, for the copies still in flight before the block exits.
#pragma once

namespace pff {

constexpr unsigned kStatusPipe = 32;                 // status bit: a staging wait gave up
constexpr long long kStageWaitCycles = 1LL << 31;    // ~1 s at 2 GHz: give up
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
// 1D bulk copy global -> shared with an L2 eviction-priority hint, completion
// counted on bar.  Addresses and size are multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                              unsigned long long policy) {
  asm volatile(
      "{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %1;\n\t"
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [ga], %2, [%3], %4;\n\t}" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
// The words are read once: they go first from L2, so that the x and y lines
// that neighbouring blocks reuse stay.
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Orders this thread's earlier generic-proxy shared-memory accesses (and, after
// a barrier, the block's) before later async-proxy writes to the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// BF16 -> FP32 of the low / high half of a packed pair (exact).
__device__ __forceinline__ float bf_lo(unsigned r) { return __uint_as_float(r << 16); }
__device__ __forceinline__ float bf_hi(unsigned r) { return __uint_as_float(r & 0xffff0000u); }

static_assert(pipe_fits<5, 5, true, true>() && pipe_fits<5, 5, false, false>(),
              "the Q = 5 level kernels need two resident blocks per SM");

// Requests stage h of slice k of element block blk into slot (thread 0 only).
template <int Q, bool BF, bool KX>
__device__ __forceinline__ void pipe_issue(const ElemArgs<float>& a, unsigned char* slot, uint64_t* bar, long long blk,
                                           int k, int h) {
  constexpr unsigned q2eb = pipe_q2eb<Q>();
  constexpr unsigned long long q3eb = (unsigned long long)Q * q2eb;
  const unsigned long long pol = l2_evict_first_policy();
  if constexpr (BF) {
    const unsigned char* g =
        reinterpret_cast<const unsigned char*>(a.lin16) + (unsigned long long)blk * 2 * kLin16Words * q3eb;
    mbar_expect_tx(bar, (KX ? 144u : 136u) * q2eb);
#pragma unroll
    for (int o = 0; o < 8; ++o)
      bulk_g2s_hint(slot + o * 16 * q2eb, g + o * 16 * q3eb + (unsigned long long)k * 16 * q2eb, 16 * q2eb, bar, pol);
    bulk_g2s_hint(slot + 128 * q2eb, g + 128 * q3eb + (unsigned long long)k * 8 * q2eb, 8 * q2eb, bar, pol);
    if (KX) bulk_g2s_hint(slot + 136 * q2eb, g + 136 * q3eb + (unsigned long long)k * 8 * q2eb, 8 * q2eb, bar, pol);
  } else {
    const float* g = a.lin + (unsigned long long)blk * kLinWords * q3eb;
    if (h == 0) {
      mbar_expect_tx(bar, 128 * q2eb);
#pragma unroll
      for (int o = 0; o < 8; ++o)
        bulk_g2s_hint(slot + o * 16 * q2eb, g + lin32_word(4 * o, k, 0, q3eb, q2eb), 16 * q2eb, bar, pol);
    } else {
      constexpr int NT = pipe_tails<BF, KX>();
      uintptr_t lo[NT];
      unsigned nb[NT], tot = 128 * q2eb;
#pragma unroll
      for (int jt = 0; jt < NT; ++jt) {
        const uintptr_t ad = reinterpret_cast<uintptr_t>(g + lin32_word(kLinQuadWords + jt, k, 0, q3eb, q2eb));
        lo[jt] = ad & ~uintptr_t(15);
        nb[jt] = (unsigned)((ad - lo[jt] + 4 * q2eb + 15) & ~uintptr_t(15));
        tot += nb[jt];
      }
      mbar_expect_tx(bar, tot);
#pragma unroll
      for (int o = 0; o < 8; ++o)
        bulk_g2s_hint(slot + o * 16 * q2eb, g + lin32_word(32 + 4 * o, k, 0, q3eb, q2eb), 16 * q2eb, bar, pol);
#pragma unroll
      for (int jt = 0; jt < NT; ++jt)
        bulk_g2s_hint(slot + 128 * q2eb + jt * pipe_tail_bytes<Q>(), reinterpret_cast<const void*>(lo[jt]), nb[jt],
                      bar, pol);
    }
  }
}

// Thread t's words of stage h of slice k from the slot: r[i] = word LO + i
// (FP32, LO = 0 or 32) or the BF16 pair of words 2i, 2i + 1.
template <int Q, bool BF, bool KX>
__device__ __forceinline__ void pipe_read(const ElemArgs<float>& a, const unsigned char* slot, int t, long long blk,
                                          int k, int h, unsigned* r) {
  constexpr int q2eb = pipe_q2eb<Q>();
  const uint4* oc = reinterpret_cast<const uint4*>(slot) + t;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const uint4 v = oc[o * q2eb];
    r[4 * o] = v.x; r[4 * o + 1] = v.y; r[4 * o + 2] = v.z; r[4 * o + 3] = v.w;
  }
  if constexpr (BF) {
    const uint2 t1 = reinterpret_cast<const uint2*>(slot + 128 * q2eb)[t];
    r[32] = t1.x; r[33] = t1.y;
    if (KX) {
      const uint2 t2 = reinterpret_cast<const uint2*>(slot + 136 * q2eb)[t];
      r[34] = t2.x; r[35] = t2.y;
    } else {
      r[34] = r[35] = 0u;
    }
  } else if (h == 1) {
    constexpr unsigned long long q3eb = (unsigned long long)Q * q2eb;
    const float* g = a.lin + (unsigned long long)blk * kLinWords * q3eb;
#pragma unroll
    for (int jt = 0; jt < pipe_tails<BF, KX>(); ++jt) {
      const unsigned sh =
          (unsigned)(reinterpret_cast<uintptr_t>(g + lin32_word(kLinQuadWords + jt, k, 0, q3eb, q2eb)) & 15);
      r[32 + jt] = *reinterpret_cast<const unsigned*>(slot + 128 * q2eb + jt * pipe_tail_bytes<Q>() + sh + 4 * t);
    }
  }
}

template <bool BF> __device__ __forceinline__ float word_at(const unsigned* r, int w) {
  if constexpr (BF) return (w & 1) ? bf_hi(r[w >> 1]) : bf_lo(r[w >> 1]);
  else return __uint_as_float(r[w]);
}

// The pointwise linear map of the stored words [LO, HI) of a point, r as read
// by pipe_read: the 9x9 block, dP/dphi and d(s_phi L)/dF (their roles swapped
// for the transpose, TR), d(s_phi L)/dphi and the phase-gradient coefficients.
// ou, s0 accumulate over the stages of the point; o3 is set by the stage that
// holds the phase-gradient words.
template <int LO, int HI, bool BF, bool TR, bool KX>
__device__ __forceinline__ void jac_words(const unsigned* r, const float g[4][3], float phi, float ou[9], float& s0,
                                          float o3[3]) {
  float gu[9];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int al = 0; al < 3; ++al) gu[3 * f + al] = g[f][al];
#pragma unroll
  for (int m = 0; m < 9; ++m) {  // upper triangle of the symmetric 9x9 block
#pragma unroll
    for (int n = m; n < 9; ++n) {
      const int wd = sym9(m, n);
      if (wd >= LO && wd < HI) {
        const float w = word_at<BF>(r, wd - LO);
        ou[m] = fmaf(w, gu[n], ou[m]);
        if (n != m) ou[n] = fmaf(w, gu[m], ou[n]);
      }
    }
  }
#pragma unroll
  for (int wd = kWP; wd < kWK; ++wd) {
    if (wd >= LO && wd < HI) {
      const float w = word_at<BF>(r, wd - LO);
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
  }
  if (kWK >= LO && kWK + 3 <= HI) {
    o3[0] = word_at<BF>(r, kWK - LO) * g[3][0];
    o3[1] = word_at<BF>(r, kWK + 1 - LO) * g[3][1];
    o3[2] = word_at<BF>(r, kWK + 2 - LO) * g[3][2];
    if (KX) {  // mapped mesh: symmetric off-diagonal coefficients 01, 02, 12
      const float k01 = word_at<BF>(r, kWKX - LO), k02 = word_at<BF>(r, kWKX + 1 - LO),
                  k12 = word_at<BF>(r, kWKX + 2 - LO);
      o3[0] = fmaf(k02, g[3][2], fmaf(k01, g[3][1], o3[0]));
      o3[1] = fmaf(k12, g[3][2], fmaf(k01, g[3][0], o3[1]));
      o3[2] = fmaf(k12, g[3][1], fmaf(k02, g[3][0], o3[2]));
    }
  }
}

// Gather of an element's nodal values (structured map or explicit offsets),
// split so that the loads of the next element block are in flight while the
// present block runs its transposed contractions: pipe_gather_load issues the
// loads of thread ij's nodes (masked entries read as zero), pipe_gather_store
// writes them to bufA [4][c][b][a].
template <int P, int Q> __host__ __device__ constexpr int pipe_gather_rounds() {
  return (P * P * P + Q * Q - 1) / (Q * Q);
}
template <int P, int Q>
__device__ __forceinline__ void pipe_gather_load(const ElemArgs<float>& a, int e, bool valid, bool em, int ij,
                                                 float xv[pipe_gather_rounds<P, Q>()][4]) {
  constexpr int Q2 = Q * Q, P3 = P * P * P;
  const long long nn = a.mesh.nn;
  const bool masked = a.mask && valid && em;
#pragma unroll
  for (int r = 0; r < pipe_gather_rounds<P, Q>(); ++r) {
    const int idx = ij + r * Q2;
    const bool live = valid && idx < P3;
    const int aa = idx % P, bb = (idx / P) % P, cc = idx / (P * P);
    const long long n = live ? node_of<P, Q>(a.mesh, e, aa, bb, cc) : 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const long long g = f * nn + n;
      xv[r][f] = live ? __ldg(a.x + g) : 0.0f;
      if (live && masked && __ldg(a.mask + g)) xv[r][f] = 0.0f;
    }
  }
}
template <int P, int Q>
__device__ __forceinline__ void pipe_gather_store(float* bufA, int ij, const float xv[pipe_gather_rounds<P, Q>()][4]) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q, P3 = P * P * P;
#pragma unroll
  for (int r = 0; r < pipe_gather_rounds<P, Q>(); ++r) {
    const int idx = ij + r * Q2;
    if (idx < P3)
#pragma unroll
      for (int f = 0; f < 4; ++f) bufA[f * Q3 + idx] = xv[r][f];
  }
}

// Gradients of the four fields at point (i, j, k) from the Gauss-point values
// V = bufB; the z-derivative row Dc[k][.] as kernel-parameter operands (k is
// fixed at compile time), the x- and y-rows from shared memory.
template <int Q>
__device__ __forceinline__ void grad_at_c(const ElemArgs<float>& a, const float* V0, const float* Dc, int i, int j,
                                          int k, float g[4][3], float& phi) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  float di[Q], dj[Q];
#pragma unroll
  for (int m = 0; m < Q; ++m) {
    di[m] = Dc[i * Q + m];
    dj[m] = Dc[j * Q + m];
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float* V = V0 + f * Q3;
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      gx = fmaf(di[m], V[k * Q2 + j * Q + m], gx);
      gy = fmaf(dj[m], V[k * Q2 + m * Q + i], gy);
      gz = fmaf(a.cDc[k * Q + m], V[m * Q2 + j * Q + i], gz);
    }
    g[f][0] = gx; g[f][1] = gy; g[f][2] = gz;
  }
  phi = V0[3 * Q3 + k * Q2 + j * Q + i];
}

// Transposed x- and y-derivatives of slice kc: Y[f][kc] += sum_m Dc[m, i] ox(m, j)
// + Dc[m, j] oy(i, m), from the slice buffer sb = [8][Q^2] (ox, oy per field).
template <int Q>
__device__ __forceinline__ void pipe_contract_xy(const float* Dc, const float* sb, int i, int j, float Y[4][Q],
                                                 int kc) {
  constexpr int Q2 = Q * Q;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    float acc = Y[f][kc];
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      acc = fmaf(Dc[m * Q + i], sb[(2 * f) * Q2 + j * Q + m], acc);
      acc = fmaf(Dc[m * Q + j], sb[(2 * f + 1) * Q2 + m * Q + i], acc);
    }
    Y[f][kc] = acc;
  }
}

// The same contraction returned as the contribution c[f] to Y[f][kc], and its
// addition at a slice index known only at run time (the rolled slice loop).
template <int Q>
__device__ __forceinline__ void pipe_contract_c(const float* Dc, const float* sb, int i, int j, float c[4]) {
  constexpr int Q2 = Q * Q;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    float acc = 0.0f;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      acc = fmaf(Dc[m * Q + i], sb[(2 * f) * Q2 + j * Q + m], acc);
      acc = fmaf(Dc[m * Q + j], sb[(2 * f + 1) * Q2 + m * Q + i], acc);
    }
    c[f] = acc;
  }
}
template <int Q>
__device__ __forceinline__ void add_at(float Y[4][Q], int kc, const float c[4]) {
#pragma unroll
  for (int kk = 0; kk < Q; ++kk)
    if (kk == kc)
#pragma unroll
      for (int f = 0; f < 4; ++f) Y[f][kk] += c[f];
}

template <int P, int Q, bool BF, bool KX, bool TR>
__global__ void __launch_bounds__(Q * Q * elems_per_block(Q), 2)
k_level_pipe(const ElemArgs<float> a) {
  constexpr int EB = elems_per_block(Q);
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  constexpr int SPS = BF ? 1 : 2;  // stages per slice
  constexpr int NS = SPS * Q;      // stages per element block
  constexpr int kSlot = pipe_slot_bytes<Q, BF, KX>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* slots = smem_raw;                                    // [2][kSlot]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * kSlot);  // one mbarrier per slot
  float* sm = reinterpret_cast<float*>(smem_raw + 2 * kSlot + 16);
  const int t = threadIdx.x;
  const int el = t / Q2, ij = t % Q2;
  const int i = ij % Q, j = ij / Q;
  const int G = gridDim.x;
  const int nmine = (a.nblk - (int)blockIdx.x + G - 1) / G;  // element blocks of this block (grid <= nblk)
  const long long nstage = (long long)nmine * NS;
  const long long blk_first = (long long)a.blk0 + blockIdx.x;

  float* Bs = sm;  // the 1D matrices where a thread's own index selects the row
  float* Dcs = Bs + Q * P;
  for (int idx = t; idx < Q * P; idx += blockDim.x) Bs[idx] = a.cB[idx];
  for (int idx = t; idx < Q * Q; idx += blockDim.x) Dcs[idx] = a.cDc[idx];
  float* base = sm + mat_smem_words<P, Q>() + el * pipe_elem_stride<Q>();
  const ElemSmem<P, Q, float> s{base + 4 * Q3, base, nullptr, Bs, Dcs, nullptr};
  float* sbuf = s.bufA;  // [2][8][Q^2] during the slice loop
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
  }
  __syncthreads();
  if (t == 0)
    for (long long sq = 0; sq < 2 && sq < nstage; ++sq)
      pipe_issue<Q, BF, KX>(a, slots + (sq & 1) * kSlot, bar + (sq & 1), blk_first + (sq / NS) * G,
                            (int)(sq % NS) / SPS, (int)(sq % NS) % SPS);
  long long issued = nstage < 2 ? nstage : 2;  // stages requested so far (block-uniform)
  long long seq = 0;                           // the next stage to consume
  bool staged = true;                          // every wait of the block so far succeeded (block-uniform)

  // element flag (has masked nodes) and nodal values of the first element block
  int e = (int)(blk_first * EB) + el;
  bool valid = e < a.mesh.nel;
  bool em = valid && (!a.emask || a.emask[e]);
  float xv[pipe_gather_rounds<P, Q>()][4];
  pipe_gather_load<P, Q>(a, e, valid, em, ij, xv);

  for (int it = 0; it < nmine; ++it) {
    const long long blk = blk_first + (long long)it * G;
    pipe_gather_store<P, Q>(s.bufA, ij, xv);
    fwd_lines<P, Q>(a, s.bufA, s.bufB, ij);

    float Y[4][Q];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int k = 0; k < Q; ++k) Y[f][k] = 0.0f;
    float g[4][3], phi = 0.0f, ou[9], s0 = 0.0f, o3[3] = {0.0f, 0.0f, 0.0f};
    // the slice loop stays rolled (smaller code: at 64^3 Q4 1 % faster with
    // FP32 words, 3 % with BF16 words) except on the order-1 level, whose
    // short contractions leave the loop overhead exposed (5 % slower rolled)
#pragma unroll(P >= 3 ? 1 : Q)
    for (int k = 0; k < Q; ++k) {
#pragma unroll
    for (int h = 0; h < SPS; ++h) {
      const int sl = (int)(seq & 1);
      const bool ok = mbar_wait(bar + sl, (unsigned)((seq >> 1) & 1), a.status);
      unsigned r[38];
      pipe_read<Q, BF, KX>(a, slots + sl * kSlot, t, blk, k, h, r);
      // every thread holds its words and the slice buffer of slice k - 1 is
      // written: the slot takes stage seq + 2 (of this element block or the next)
      staged = __syncthreads_and(ok && staged) != 0;
      if (!staged) break;
      if (seq + 2 < nstage) {
        if (t == 0) {
          fence_proxy_async_smem();
          const long long sq = seq + 2;
          pipe_issue<Q, BF, KX>(a, slots + sl * kSlot, bar + sl, blk_first + (sq / NS) * G, (int)(sq % NS) / SPS,
                                (int)(sq % NS) % SPS);
        }
        issued = seq + 3;
      }
      ++seq;
      if (h == 0) {
        if (k > 0) {
          float c[4];
          pipe_contract_c<Q>(s.Dc, sbuf + ((k - 1) & 1) * 8 * Q2, i, j, c);
          add_at<Q>(Y, k - 1, c);
        }
        grad_at_c<Q>(a, s.bufB, s.Dc, i, j, k, g, phi);
#pragma unroll
        for (int m = 0; m < 9; ++m) ou[m] = 0.0f;
        s0 = 0.0f;
      }
      if (valid) {
        if constexpr (BF) jac_words<0, 72, true, TR, KX>(r, g, phi, ou, s0, o3);
        else if (h == 0) jac_words<0, 32, false, TR, KX>(r, g, phi, ou, s0, o3);
        else jac_words<32, kLinWords, false, TR, KX>(r, g, phi, ou, s0, o3);
      }
      if (h == SPS - 1) {
        if (!valid) {
#pragma unroll
          for (int m = 0; m < 9; ++m) ou[m] = 0.0f;
          s0 = 0.0f;
          o3[0] = o3[1] = o3[2] = 0.0f;
        }
        float* sb = sbuf + (k & 1) * 8 * Q2;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float ox = f < 3 ? ou[3 * f] : o3[0];
          const float oy = f < 3 ? ou[3 * f + 1] : o3[1];
          const float oz = f < 3 ? ou[3 * f + 2] : o3[2];
#pragma unroll
          for (int kk = 0; kk < Q; ++kk) Y[f][kk] = fmaf(a.cDc[k * Q + kk], oz, Y[f][kk]);
          sb[(2 * f) * Q2 + ij] = ox;
          sb[(2 * f + 1) * Q2 + ij] = oy;
        }
#pragma unroll
        for (int kk = 0; kk < Q; ++kk)
          if (kk == k) Y[3][kk] += s0;
      }
    }
    if (!staged) break;
    }
    if (!staged) break;
    __syncthreads();
    pipe_contract_xy<Q>(s.Dc, sbuf + ((Q - 1) & 1) * 8 * Q2, i, j, Y, Q - 1);
    // the next element block's nodal values are loaded while this one runs
    // its transposed contractions and scatter
    const int e_now = e;
    const bool valid_now = valid, em_now = em;
    if (it + 1 < nmine) {
      e = (int)((blk + G) * EB) + el;
      valid = e < a.mesh.nel;
      em = valid && (!a.emask || a.emask[e]);
      pipe_gather_load<P, Q>(a, e, valid, em, ij, xv);
    }
    __syncthreads();  // the slice buffers are read; backward reuses them
    bwd_lines<P, Q>(a, s.bufA, s.bufB, e_now, valid_now, em_now, ij, Y);
    __syncthreads();  // the scatter has read bufA; the next gather writes it
  }
  // a wait gave up: the copies still in flight (stages [seq, issued), at most
  // one per slot) land before the block's shared memory is released
  if (!staged && t == 0)
    for (long long sq = seq; sq < issued; ++sq) mbar_wait(bar + (sq & 1), (unsigned)((sq >> 1) & 1), nullptr);
}

template <int P, int Q, bool BF, bool KX>
cudaError_t launch_level_pipe_v(const ElemArgs<float>& a, int nblk, cudaStream_t st) {
  constexpr int EB = elems_per_block(Q);
  constexpr size_t smem = pipe_smem_bytes<P, Q, BF, KX>();
  ElemArgs<float> b = a;
  b.nblk = nblk;
  const int ctas = a.ctas > 0 && a.ctas < nblk ? a.ctas : nblk;
  auto k = a.transpose ? k_level_pipe<P, Q, BF, KX, true> : k_level_pipe<P, Q, BF, KX, false>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<ctas, Q * Q * EB, smem, st>>>(b); note_launch();
  return cudaGetLastError();
}

// The FP32-arithmetic action through the persistent kernel: BF16 words
// (a.lin16) always; FP32 words when two slots of them fit (every box mesh;
// mapped meshes at Q = 5 take k_elem instead).  Returns false when it does not apply.
template <int P, int Q>
bool launch_level_pipe(const ElemArgs<float>& a, int nblk, cudaStream_t st, cudaError_t* err) {
  if (a.lin16) {
    *err = a.kx ? launch_level_pipe_v<P, Q, true, true>(a, nblk, st) : launch_level_pipe_v<P, Q, true, false>(a, nblk, st);
    return true;
  }
  if constexpr (pipe_fits<P, Q, false, true>()) {
    if (a.kx) {
      *err = launch_level_pipe_v<P, Q, false, true>(a, nblk, st);
      return true;
    }
  }
  if (a.kx) return false;
  *err = launch_level_pipe_v<P, Q, false, false>(a, nblk, st);
  return true;
}

}  // namespace pff

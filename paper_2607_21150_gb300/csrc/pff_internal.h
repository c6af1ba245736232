// Internal declarations of the CUDA library (not part of the public C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pff {

constexpr int kMaxPhase = 8;
constexpr int kMaxQ = 5;          // quadrature points per direction (Q <= p_fine + 1 <= 5)
constexpr int kLinWords = 70;     // stored pointwise linearisation words per quadrature point
// word layout: [0,45) upper triangle of the 9x9 block dP/dF (row-major, m <= n,
// m = 3 i + A), [45,54) dP/dphi, [54,63) d(s_phi L)/dF, [63] d(s_phi L)/dphi,
// [64,67) diagonal coefficients of the phase-gradient term, [67,70) its
// off-diagonal coefficients (01, 02, 12), non-zero on mapped meshes only.
// All words are in the parent frame (w_q det J and d xi / dX folded in).
constexpr int kWA = 0, kWP = 45, kWC = 54, kWD = 63, kWK = 64, kWKX = 67;
constexpr int kLinWordsExport = 67;  // words returned by pff_get_linearization
// FP32 planes (level actions, double-float hi/lo): words [0, 64) interleaved by
// four, so that one 128-bit load fetches four words of one point; words
// [64, 70) as in the FP64 layout.  Offset of word w of slice k, thread t within
// a block's region (q3eb = Q^3 EB words per word plane, q2eb = Q^2 EB per slice):
constexpr int kLinQuadWords = 64;
__host__ __device__ constexpr long long lin32_word(int w, int k, int t, long long q3eb, long long q2eb) {
  return w < kLinQuadWords ? (long long)(w >> 2) * 4 * q3eb + (long long)k * 4 * q2eb + 4LL * t + (w & 3)
                           : (long long)w * q3eb + (long long)k * q2eb + t;
}
// Floats allocated past the FP32 planes: the persistent level kernel copies
// each tail-word run widened to 16-byte boundaries, up to 12 bytes past it.
constexpr long long kLin32Pad = 16;

// BF16 words of the stored linearisation (the level actions of PFF_F32_BF16):
// per block a region of kLin16Words * Q^3 EB uint16, words [0, 64) of a point
// grouped by eight (one 16-byte load), words [64, 68) and [68, 72) in two
// planes of four per point (8 bytes; the second is read on mapped meshes
// only, its words 70 and 71 are zero).  Slice k of a block is one contiguous
// run per plane: 8 Q^2 EB words of each octet plane, 4 Q^2 EB of each tail
// plane, so that a slice moves as ten 1D bulk copies.
constexpr int kLin16Words = 72;
__host__ __device__ constexpr long long lin16_word(int w, int k, int t, long long q3eb, long long q2eb) {
  return w < 64 ? (long long)(w >> 3) * 8 * q3eb + (long long)k * 8 * q2eb + 8LL * t + (w & 7)
       : w < 68 ? 64 * q3eb + (long long)k * 4 * q2eb + 4LL * t + (w - 64)
                : 68 * q3eb + (long long)k * 4 * q2eb + 4LL * t + (w - 68);
}

// Elements handled by one thread block of the element kernels: Q*Q threads per element.
__host__ __device__ constexpr int elems_per_block(int Q) { return 256 / (Q * Q); }
// 128-bit alignment of the FP32 quad planes needs an even Q^3 EB for every Q
static_assert((2 * 2 * 2 * elems_per_block(2)) % 2 == 0 && (3 * 3 * 3 * elems_per_block(3)) % 2 == 0 &&
              (4 * 4 * 4 * elems_per_block(4)) % 2 == 0 && (5 * 5 * 5 * elems_per_block(5)) % 2 == 0,
              "FP32 quad layout needs Q^3 EB even");

// Shared-memory words of the 1D matrices in an element kernel (B, D_t, and
// the collocated derivative D_c; the persistent kernel keeps B and D_c).
template <int P, int Q> __host__ __device__ constexpr int mat_smem_words() { return 3 * Q * P + Q * Q; }

// Geometry of the persistent FP32-arithmetic level kernel (pff_elem_pipe.cuh);
// here so that the host tests can check the bulk copies it issues.
// Stage geometry.  q2eb = points of one Gauss slice of an element block.
template <int Q> __host__ __device__ constexpr int pipe_q2eb() { return Q * Q * elems_per_block(Q); }
// Region of one FP32 tail-word run in a slot: the run of 4 q2eb bytes widened
// to 16-byte boundaries (it starts 0, 4, 8 or 12 bytes into the region).
template <int Q> __host__ __device__ constexpr int pipe_tail_bytes() { return (4 * pipe_q2eb<Q>() + 12 + 15) / 16 * 16; }
template <bool BF, bool KX> __host__ __device__ constexpr int pipe_tails() { return BF ? (KX ? 2 : 1) : (KX ? 6 : 3); }
template <int Q, bool BF, bool KX> __host__ __device__ constexpr int pipe_slot_bytes() {
  return BF ? (KX ? 144 : 136) * pipe_q2eb<Q>() : 128 * pipe_q2eb<Q>() + pipe_tails<BF, KX>() * pipe_tail_bytes<Q>();
}
// Per element: the values at the Gauss points (4 Q^3), then the ping-pong
// buffer of the contractions, which holds the two slice buffers (2 x 8 Q^2)
// during the slice loop.
template <int Q> __host__ __device__ constexpr int pipe_elem_words() {
  return 4 * Q * Q * Q + (4 * Q * Q * Q > 16 * Q * Q ? 4 * Q * Q * Q : 16 * Q * Q);
}
// Element stride in shared memory: the element's words, padded to Q^2 mod 32,
// so that the Q^2 threads of consecutive elements fall on consecutive banks
// (Q = 5: 1017 instead of 1000 words cuts the wavefronts of the contraction
// stages by a fifth, counted over every access pattern of the kernel).
template <int Q> __host__ __device__ constexpr int pipe_elem_stride() {
  return pipe_elem_words<Q>() + ((Q * Q - pipe_elem_words<Q>()) % 32 + 32) % 32;
}
template <int P, int Q, bool BF, bool KX> __host__ __device__ constexpr int pipe_smem_bytes() {
  return 2 * pipe_slot_bytes<Q, BF, KX>() + 16 +
         4 * (mat_smem_words<P, Q>() + elems_per_block(Q) * pipe_elem_stride<Q>());
}
// Two resident blocks per SM: 228 KB of shared memory per SM, 1 KB reserved per block.
template <int P, int Q, bool BF, bool KX> __host__ __device__ constexpr bool pipe_fits() {
  return pipe_smem_bytes<P, Q, BF, KX>() <= 113 * 1024;
}
__host__ __device__ constexpr int sym9(int m, int n) {  // m <= n
  return m * 9 - (m * (m - 1)) / 2 + (n - m);
}

// Per-phase material constants for the pointwise update (host-derived).
struct PhaseDev {
  double mu[3], kap[3];   // branch 0 Hooke, 1 Maxwell, 2 Prandtl
  int has[3];
  double cmax;            // Maxwell: mu dt / eta_d (0 when eta_d = +inf)
  double sig0;            // Prandtl initial yield stress
  double Hlin, sinf, beta;// Prandtl hardening law sigma_y = sig0 + Hlin ep + (sinf - sig0)(1 - exp(-beta ep))
  int hard;               // 0: perfect plasticity (Hlin = 0, sinf = sig0)
  double kap_tot;
  double gc_c0l0;         // Gc / (c0 l0)
  double kphi;            // s_phi * 2 Gc l0 / c0
  // raw parameters (adjoint): Hooke E, nu; Maxwell eta_d (0 = infinite); Gc, l0; c0
  double E0, nu0, eta_d, Gc, l0, c0;
};

struct GlobDev {
  int at;                 // 1 = AT1, 2 = AT2
  double eta, zeta, dt, s_phi;
};

// Geometry of the affine box elements.
struct Geom {
  double s[3];            // d xi / d X per direction = 2 / h
  double detJ;            // h_x h_y h_z / 8
  double wq[kMaxQ];       // 1D Gauss weights
};

// Mesh / restriction description shared by the element kernels.
struct MeshDev {
  int nel, nx, ny, nz;    // element grid
  int p;                  // order of this level (P = p + 1 nodes per direction)
  int nnx, nny;           // node grid sizes in x and y
  long long nn;           // nodes per field
  const int32_t* offsets; // optional explicit element -> node map [nel][P^3]
};

struct PointArgs {
  PhaseDev phase[kMaxPhase];
  GlobDev glob;
  Geom geom;
  int Q;
  int nphase;
  long long nq;
  long long nel;
  double* io;             // [13][nq] inputs in, residual integrands out
  const double* hist;     // [15][nq] committed history
  double* hist_trial;     // [15][nq]
  const uint8_t* phase_id;// [nq]
  uint8_t* flags;         // [nq]
  double* lin;            // tiled stored linearisation (FP64)
  const double* geo;      // mapped mesh: [10][nq] d xi_alpha / dX_A (word 3 alpha + A), w det J; null = box
  int* status;            // device status word (bit0 eigen sweeps, bit1 J <= 0, bit2 non-finite, bit3 phase id)
  int want_tangent;
};

// Adjoint of the pointwise update (pff_adjoint.cu).  Mode 0: qa = (dPhi/da)^T hbar
// as parent-frame pseudo-integrands [13][nq]; mode 1: hbar_out = p^T df/dh +
// hbar^T dPhi/dh [15][nq] and gtheta[phase*6 + j] += p^T df/dtheta_j +
// hbar^T dPhi/dtheta_j (theta_j = E_inf, nu_inf, sigma0, eta_d, Gc, l0).
struct AdjArgs {
  PhaseDev phase[kMaxPhase];
  GlobDev glob;
  Geom geom;
  int Q, nphase, mode;
  long long nq;
  const double* a_in;     // [13][nq] grad_X u, phi, grad_X phi
  const double* hist;     // [15][nq] committed history of the step
  const uint8_t* phase_id;
  const double* p;        // [13][nq] interpolated adjoint (reference frame), mode 1
  const double* hbar;     // [15][nq] adjoint of the trial history (may be null)
  double* qa_out;         // mode 0
  double* hbar_out;       // mode 1
  double* gtheta;         // mode 1, [nphase][6]
  const double* geo;      // mapped mesh: [10][nq] d xi / dX and w det J; null = box
  int* status;
};
cudaError_t launch_adjoint_point(const AdjArgs& a, cudaStream_t st);

// Element-kernel launches (pff_elem*.cu).  T = double, float or df64.
enum ElemMode { kApply = 0, kEval = 1, kBack = 2 };

// Double-float value hi + lo (two FP32 words, about 48 significant bits); the
// arithmetic lives in pff_df.cuh.  8-byte aligned so that shared-memory
// accesses are single 64-bit transactions.
struct __align__(8) df64 {
  float hi, lo;
};

// Storage types of an element kernel computing in T: vectors V, stored
// linearisation L, 1D basis matrices M.  The double-float kernel reads and
// writes FP64 vectors, the stored linearisation as two FP32 planes (hi, then
// lo at a fixed offset) and converts the FP64 basis matrices on entry.
template <typename T> struct ElemTypes { using V = T; using L = T; using M = T; };
template <> struct ElemTypes<df64> { using V = double; using L = float; using M = double; };

template <typename T>
struct ElemArgs {
  using V = typename ElemTypes<T>::V;
  using L = typename ElemTypes<T>::L;
  using M = typename ElemTypes<T>::M;
  MeshDev mesh;
  const V* x;             // [4][nn] input (apply) / unused
  V* y;                   // [4][nn] output (scatter-add)
  const uint8_t* mask;    // [4][nn] Dirichlet mask or nullptr
  const M* B;             // [Q][P] interpolation to Gauss points
  const M* Dc;            // [Q][Q] collocated derivative at Gauss points
  const M* Dt;            // [Q][P] derivative of the basis at Gauss points (diagonal)
  const L* lin;           // tiled stored linearisation (apply / diagonal)
  const L* linP;          // words multiplying dphi in the u rows (dP/dphi or, transposed, dL/dF)
  const L* linC;          // words multiplying grad u in the phi row
  double* scratch;        // [13][nq] (eval / back)
  double s[3];            // d xi / d X (eval, box)
  const double* geo;      // mapped mesh (eval): [10][nq] d xi / dX per point; null = box
  long long nq;
  int transpose;
  int kx;                 // 1: add the off-diagonal phase-gradient words (mapped meshes)
  long long lo;           // df64: offset (in words) from the hi plane to the lo plane
  const uint16_t* lin16;  // FP32 action only: read the BF16 words (lin16_word layout) instead of lin
  int* status;            // device status word (BF16-word action: bit 32 when a staging wait gave up)
  const uint8_t* emask;   // [nel] 1 = the element has masked nodes (null: check the mask everywhere)
  void* evec;             // deterministic transpose: element values [nel][4][P^3] (type V) instead of atomics
  int blk0;               // first element block of the launch (actions; 0 = from the first)
  int ctas;               // FP32-arithmetic actions: resident blocks of the persistent kernel (0 = one per element block)
  int nblk;               // element blocks of the launch (actions; 0 = all blocks from blk0 = 0)
  // FP32-arithmetic actions: the 1D matrices B [Q][P] and Dc [Q][Q] as kernel
  // parameters, read as constant-bank operands where the index is fixed at compile time
  float cB[kMaxQ * kMaxQ];
  float cDc[kMaxQ * kMaxQ];
};

// One translation unit per quadrature size Q (pff_elem_q<Q>.cu); each covers
// every basis size P <= Q in both precisions.
#define PFF_DECLARE_ELEM_Q(QQ)                                                                  \
  template <typename T> cudaError_t launch_elem_q##QQ(int P, int mode, const ElemArgs<T>& a, cudaStream_t st); \
  template <typename T> cudaError_t launch_diag_q##QQ(int P, const ElemArgs<T>& a, cudaStream_t st);
PFF_DECLARE_ELEM_Q(2)
PFF_DECLARE_ELEM_Q(3)
PFF_DECLARE_ELEM_Q(4)
PFF_DECLARE_ELEM_Q(5)

cudaError_t launch_pointwise(const PointArgs& a, cudaStream_t st);
// geo[10][nq] from the parent Jacobians J[3f + al][nq] (= d X_f / d xi_al, the
// first nine rows of an eval): d xi / dX = J^-1 and w_q det J; status bit 2
// where det J <= 0.
cudaError_t launch_geometry(const double* J, double* geo, const Geom& g, int Q, long long nq, int* status,
                            cudaStream_t st);

// Vector / transfer kernels (pff_vec.cu)
cudaError_t launch_init_masked(int prec, void* y, const void* x, const double* ubar,
                               const uint8_t* mask, long long n, int mode, cudaStream_t st);
// Deterministic transpose: for nodes [n0, n1) of each field, y = mask ? init :
// the sum of the element values evec[e][f][local] of the node's incident
// elements (up to eight, in ascending element order; structured numbering).
// init as launch_init_masked's mode: 0 x, 1 x - ubar, 2 one; 3 zero.  prec 0: FP64
// values and vectors, 1: FP32.
cudaError_t launch_node_gather(int prec, const MeshDev& m, const void* evec, const uint8_t* mask, int mode,
                               const void* x, const double* ubar, void* y, long long n0, long long n1,
                               cudaStream_t st);
// emask[e] = 1 where element e has a masked node (any field), 0 elsewhere.
cudaError_t launch_elem_mask(const MeshDev& m, const uint8_t* mask, uint8_t* emask, cudaStream_t st);
// y = mask ? x : 0 on nodes [n0, n1) of each field (prec 0: FP64, 1: FP32).
cudaError_t launch_init_rows(int prec, void* y, const void* x, const uint8_t* mask, long long nn, long long n0,
                             long long n1, cudaStream_t st);
// Level copies of the FP64 words a in one pass, each optional: FP32 planes hi
// (round to nearest even) and lo = a - hi (lin32_word layout), BF16 words b16
// (round to nearest even, lin16_word layout).
cudaError_t launch_split_words(const double* a, float* hi, float* lo, uint16_t* b16, long long nblk, int Q,
                               cudaStream_t st);
cudaError_t launch_apply_dirichlet(double* z, const double* ubar, const uint8_t* mask, long long n, cudaStream_t st);
cudaError_t launch_masked_field_sums(const double* v, const uint8_t* sel, long long nn, double* out, cudaStream_t st);
// out[8]: flag counts (yield, history active, theta >= 0), phi max / min, nodes
// with phi > 0.9, max eps_p and max H of hist (device memory).
cudaError_t launch_state_summary(const uint8_t* flags, const double* hist, long long nq, const double* phi,
                                 long long nn, double* out, cudaStream_t st);
cudaError_t launch_untile(const double* lin, double* out, long long nq, int Q, cudaStream_t st);
template <typename T>
cudaError_t launch_prolong(const MeshDev& mc, const MeshDev& mf, const T* I1, const T* xc, T* xf,
                           const uint8_t* maskc, const uint8_t* maskf, cudaStream_t st);
// evec (deterministic mode): element values and a node gather instead of atomics.
template <typename T>
cudaError_t launch_restrict(const MeshDev& mc, const MeshDev& mf, const T* I1, const T* rf, T* rc,
                            const uint8_t* maskc, const uint8_t* maskf, cudaStream_t st, void* evec = nullptr);
template <typename T>
cudaError_t launch_cheb_init(long long n, const T* b, const T* Ax, const T* diag, T* r, T* d,
                             double inv_theta, cudaStream_t st);
template <typename T>
cudaError_t launch_cheb_step(long long n, T* x, T* d, T* r, const T* Ad, const T* diag,
                             double c_d, double c_r, int last, cudaStream_t st);


// Krylov vectors and the assembled coarse operator (pff_krylov.cu)
constexpr int kReduceBlocks = 152 * 4;
// out[j] = V_j . w for j < k (vectors V_j at stride ldv), FP64 accumulation in a
// fixed order; partial needs k * kReduceBlocks doubles.
template <typename TV, typename T>
cudaError_t launch_mdot(const TV* V, long long ldv, int k, const T* w, long long n, double* partial, double* out,
                        cudaStream_t st);
cudaError_t launch_maxpy(double* w, const double* V, long long ldv, int k, const double* h, double sign, long long n,
                         cudaStream_t st);
template <typename T>
cudaError_t launch_axpby(T* y, const T* x, double a, double b, long long n, cudaStream_t st);
template <typename T>
cudaError_t launch_bminus(T* y, const T* b, long long n, cudaStream_t st);
template <typename T>
cudaError_t launch_dscale(T* y, const T* x, const T* d, long long n, cudaStream_t st);
cudaError_t launch_d2f(float* y, const double* x, long long n, cudaStream_t st);
cudaError_t launch_f2d(double* y, const float* x, long long n, cudaStream_t st);
cudaError_t launch_q1_spmv(const MeshDev& mc, const double* A, const double* x, double* y, cudaStream_t st);
// The same with an FP32 copy of the stencil and FP32 arithmetic (FP64 vectors).
cudaError_t launch_q1_spmv32(const MeshDev& mc, const float* A, const double* x, double* y, cudaStream_t st);
cudaError_t launch_q1_diag(const MeshDev& mc, const double* A, double* d, cudaStream_t st);
// Sum-factorised element matrices (Ke: [nel][32][32] work space) and a
// deterministic gather into the stencil storage.
// lin32 not null: from the FP32 words (quad layout) in FP32 arithmetic (the
// mixed solver's preconditioner); Ke and A stay FP64.
cudaError_t launch_q1_assemble_sf(const MeshDev& mc, int Q, const double* lin, const float* lin32, const double* B1,
                                  const double* D1, const uint8_t* maskc, double* Ke, double* A, int kx,
                                  cudaStream_t st);
cudaError_t launch_q1_spmv_t(const MeshDev& mc, const double* A, const double* x, double* y, cudaStream_t st);
// Geometric h-hierarchy on the order-1 grid (full coarsening, trilinear
// transfers): Galerkin element matrices of the coarse grid, their gather into
// the stencil storage, the coarse mask, and the transfers.
// f32: Galerkin products in FP32 arithmetic (the mixed solver), FP64 storage.
cudaError_t launch_q1_coarsen(const MeshDev& mf, const MeshDev& mc, const uint8_t* maskf, const double* Kef,
                              double* Kec, bool f32, cudaStream_t st);
cudaError_t launch_q1_gather(const MeshDev& mc, const double* Ke, const uint8_t* maskc, double* A, cudaStream_t st);
cudaError_t launch_hmask(const MeshDev& mf, const MeshDev& mc, const uint8_t* maskf, uint8_t* maskc, cudaStream_t st);
cudaError_t launch_hprolong_add(const MeshDev& mc, const MeshDev& mf, const double* xc, double* xf,
                                const uint8_t* maskc, const uint8_t* maskf, cudaStream_t st);
cudaError_t launch_hrestrict(const MeshDev& mc, const MeshDev& mf, const double* rf, double* rc,
                             const uint8_t* maskc, const uint8_t* maskf, cudaStream_t st);
cudaError_t launch_sel_scale(double* y, const uint8_t* sel, double s, long long n, cudaStream_t st);
cudaError_t launch_zero_masked(double* y, const uint8_t* mask, long long n, cudaStream_t st);

// Records the message returned by pff_last_error_message and returns code (pff_abi.cpp).
int set_last_error(int code, const char* msg);
// Counts one kernel launch of this library (read by pff_kernel_launches); every
// <<<...>>> launch site calls it right after the launch.
void note_launch();

// Host basis data (pff_basis.cpp)
void gll_nodes(int p, double* x);
void gauss_rule(int Q, double* x, double* w);
double lagrange(const double* nodes, int n, int a, double t);
double lagrange_deriv(const double* nodes, int n, int a, double t);

}  // namespace pff

// Definitions of the opaque libpff handles, shared by the ABI and solver files.
#pragma once
#include <vector>

#include "../../include/pff.h"
#include "pff_internal.h"

using pff::PhaseDev;
using pff::GlobDev;
using pff::MeshDev;
using pff::Geom;
using pff::kMaxPhase;

struct pff_ctx {
  int nphase;
  PhaseDev phase[kMaxPhase];
  GlobDev glob;
};

struct pff_basis {
  int p, q;
  std::vector<double> xg, xq, wq, B, Dc, Dt;
};

struct pff_restr {
  pff_box box;
  int p;
  const int32_t* offsets;
  int64_t nn;
};

struct Tables {  // per-level device copies of the 1D matrices, both precisions
  double *B64 = nullptr, *Dc64 = nullptr, *Dt64 = nullptr;
  float *B32 = nullptr, *Dc32 = nullptr, *Dt32 = nullptr;
  float hB32[pff::kMaxQ * pff::kMaxQ] = {}, hDc32[pff::kMaxQ * pff::kMaxQ] = {};  // host copies (kernel parameters)
};

struct pff_op {
  pff_ctx* ctx;
  int p, Q;
  pff_box box;
  MeshDev mesh;
  long long nq, nel;
  Geom geom;
  Tables tab;
  double* hist_c = nullptr;
  double* hist_t = nullptr;
  uint8_t* phase = nullptr;
  uint8_t* flags = nullptr;
  double* lin64 = nullptr;
  float* lin32 = nullptr;     // FP32 copy; with df = 1 the hi plane [0, lin_len) and lo plane [lin_len, 2 lin_len)
  long long lin_len = 0;
  double* io = nullptr;
  uint8_t* mask = nullptr;
  uint8_t* emask = nullptr;   // [nel] elements with masked nodes (fine level), from pff_set_dirichlet
  double* dvals = nullptr;
  int* status = nullptr;
  int f32 = 0;
  int df = 0;                 // maintain the double-float planes of the stored linearisation
  int lin32_planes = 0;       // FP32 planes allocated at lin32 (0, 1 or 2)
  int det = 0;                // deterministic transpose (pff_op_set_deterministic)
  void* evec = nullptr;       // its element values, [nel][4][P^3] doubles of the fine order
  uint16_t* lin16 = nullptr;  // BF16 words (lin16_word layout), written by pff_residual when bf16 = 1
  long long lin16_len = 0;    // uint16 entries at lin16
  int bf16 = 0;
  double* geo = nullptr;      // mapped mesh: [10][nq] d xi / dX and w det J (null: the affine box)
  double* fint = nullptr;     // internal force work vector of pff_reaction (allocated on first use)
  double* sums = nullptr;     // 8 doubles (reaction sums, state summary)
};

namespace pff { struct HostIO; }

struct pff_level {
  pff::HostIO* hio = nullptr;  // device staging and streams of pff_jacobian_apply_host (created on first use)
  pff_op* op;
  int p;
  MeshDev mesh;
  Tables tab;
  uint8_t* mask = nullptr;   // owned copy (coarse levels) ; fine level uses op->mask
  uint8_t* emask = nullptr;  // [nel] elements with masked nodes (coarse levels; the fine level uses op->emask)
  bool is_fine = false;
  // prolongation table towards the finer level with order I_pf
  int I_pf = -1;
  double* I64 = nullptr;
  float* I32 = nullptr;
};


namespace pff {
// Element blocks [blk0, blk0 + nblk) of a level action (nblk = 0: all), without
// the initialisation of y; prec PFF_F64, PFF_F32, PFF_DF64 or PFF_F32_BF16
// (pff_abi.cpp).
int apply_blocks(pff_level* L, int prec, const void* x, void* y, int transpose, int blk0, int nblk, cudaStream_t st);
// The Dirichlet mask of a level's rows (pff_abi.cpp).
const uint8_t* level_rows_mask(const pff_level* L);
// Releases the staging buffers, streams and events of pff_jacobian_apply_host (pff_hostio.cpp).
void free_host_io(pff_level* L);
}  // namespace pff

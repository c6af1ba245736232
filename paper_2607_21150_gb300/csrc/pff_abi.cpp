// C ABI of libpff: handles, parameter derivation, kernel launches.
#include "../../include/pff.h"

#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pff_internal.h"
#include "pff_handles.h"

using namespace pff;

namespace {

thread_local std::string g_err;
std::atomic<long long> g_launches{0};

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define PFF_CK(call)                                                                             \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail(PFF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define PFF_REQUIRE(cond, msg)                          \
  do {                                                  \
    if (!(cond)) return fail(PFF_ERR_INVALID, (msg));   \
  } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

template <typename T>
int upload(const std::vector<double>& h, T** d) {
  std::vector<T> tmp(h.begin(), h.end());
  PFF_CK(cudaMalloc((void**)d, sizeof(T) * (tmp.empty() ? 1 : tmp.size())));
  if (!tmp.empty()) PFF_CK(cudaMemcpy(*d, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice));
  return PFF_OK;
}

}  // namespace

namespace {

long long stride_of(int Q) { return (long long)Q * Q * Q * elems_per_block(Q); }

int make_tables(int p, int Q, Tables& t) {
  std::vector<double> xg(p + 1), xq(Q), wq(Q);
  gll_nodes(p, xg.data());
  gauss_rule(Q, xq.data(), wq.data());
  int P = p + 1;
  std::vector<double> B(Q * P), Dt(Q * P), Dc(Q * Q);
  for (int i = 0; i < Q; ++i)
    for (int a = 0; a < P; ++a) {
      B[i * P + a] = lagrange(xg.data(), P, a, xq[i]);
      Dt[i * P + a] = lagrange_deriv(xg.data(), P, a, xq[i]);
    }
  for (int i = 0; i < Q; ++i)
    for (int k = 0; k < Q; ++k) Dc[i * Q + k] = lagrange_deriv(xq.data(), Q, k, xq[i]);
  for (int i = 0; i < Q * P; ++i) t.hB32[i] = (float)B[i];
  for (int i = 0; i < Q * Q; ++i) t.hDc32[i] = (float)Dc[i];
  int rc;
  if ((rc = upload(B, &t.B64))) return rc;
  if ((rc = upload(B, &t.B32))) return rc;
  if ((rc = upload(Dc, &t.Dc64))) return rc;
  if ((rc = upload(Dc, &t.Dc32))) return rc;
  if ((rc = upload(Dt, &t.Dt64))) return rc;
  if ((rc = upload(Dt, &t.Dt32))) return rc;
  return PFF_OK;
}

void free_tables(Tables& t) {
  cudaFree(t.B64); cudaFree(t.Dc64); cudaFree(t.Dt64);
  cudaFree(t.B32); cudaFree(t.Dc32); cudaFree(t.Dt32);
  t = Tables();
}

MeshDev mesh_for(const pff_box& b, int p, const int32_t* offsets) {
  MeshDev m;
  m.nel = b.nx * b.ny * b.nz;
  m.nx = b.nx; m.ny = b.ny; m.nz = b.nz;
  m.p = p;
  m.nnx = p * b.nx + 1;
  m.nny = p * b.ny + 1;
  m.nn = (long long)m.nnx * m.nny * (p * b.nz + 1);
  m.offsets = offsets;
  return m;
}

template <typename T>
cudaError_t elem_dispatch(int Q, int P, int mode, const ElemArgs<T>& a, cudaStream_t st) {
  switch (Q) {
    case 2: return launch_elem_q2<T>(P, mode, a, st);
    case 3: return launch_elem_q3<T>(P, mode, a, st);
    case 4: return launch_elem_q4<T>(P, mode, a, st);
    case 5: return launch_elem_q5<T>(P, mode, a, st);
  }
  return cudaErrorInvalidValue;
}
template <typename T>
cudaError_t diag_dispatch(int Q, int P, const ElemArgs<T>& a, cudaStream_t st) {
  switch (Q) {
    case 2: return launch_diag_q2<T>(P, a, st);
    case 3: return launch_diag_q3<T>(P, a, st);
    case 4: return launch_diag_q4<T>(P, a, st);
    case 5: return launch_diag_q5<T>(P, a, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T> const T* tabB(const Tables& t);
template <> const double* tabB<double>(const Tables& t) { return t.B64; }
template <> const float* tabB<float>(const Tables& t) { return t.B32; }
template <typename T> const T* tabDc(const Tables& t);
template <> const double* tabDc<double>(const Tables& t) { return t.Dc64; }
template <> const float* tabDc<float>(const Tables& t) { return t.Dc32; }
template <typename T> const T* tabDt(const Tables& t);
template <> const double* tabDt<double>(const Tables& t) { return t.Dt64; }
template <> const float* tabDt<float>(const Tables& t) { return t.Dt32; }
template <typename T> const T* linOf(const pff_op* op);
template <> const double* linOf<double>(const pff_op* op) { return op->lin64; }
template <> const float* linOf<float>(const pff_op* op) { return op->lin32; }

// Multiprocessors of the current device (cached per device).
int sm_count() {
  static thread_local int dev_cached = -1, sms = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev != dev_cached) {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 0;
    dev_cached = dev;
  }
  return sms;
}

const uint8_t* level_mask(const pff_level* L) { return L->is_fine ? L->op->mask : L->mask; }
const uint8_t* level_emask(const pff_level* L) { return L->is_fine ? L->op->emask : L->emask; }

template <typename T>
ElemArgs<T> level_args(const pff_level* L) {
  ElemArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.mesh = L->mesh;
  a.mask = level_mask(L);
  a.emask = a.mask ? level_emask(L) : nullptr;
  a.B = tabB<T>(L->tab);
  a.Dc = tabDc<T>(L->tab);
  a.Dt = tabDt<T>(L->tab);
  a.lin = linOf<T>(L->op);
  a.nq = L->op->nq;
  a.kx = L->op->geo != nullptr;
  for (int d = 0; d < 3; ++d) a.s[d] = L->op->geom.s[d];
  std::memcpy(a.cB, L->tab.hB32, sizeof(a.cB));
  std::memcpy(a.cDc, L->tab.hDc32, sizeof(a.cDc));
  return a;
}

// w16: FP32 action reading the BF16 words (PFF_F32_BF16) instead of the FP32 copy.
// blk0, nblk: element blocks [blk0, blk0 + nblk) only (nblk = 0: all) and, with
// init = false, no initialisation of y (the caller has initialised the rows).
template <typename T>
int apply_t(pff_level* L, const T* x, T* y, int transpose, cudaStream_t st, bool w16 = false, int blk0 = 0,
            int nblk = 0, bool init = true) {
  pff_op* op = L->op;
  if (w16) PFF_REQUIRE(op->bf16 && op->lin16, "PFF_F32_BF16 apply needs pff_op_enable_bf16 before pff_residual");
  else PFF_REQUIRE(linOf<T>(op) != nullptr, "FP32 apply needs pff_op_enable_f32 before pff_residual");
  const bool det = op->det && op->evec;
  if (init && !det) PFF_CK(launch_init_masked(sizeof(T) == 8 ? 0 : 1, y, x, nullptr, level_mask(L), 4 * L->mesh.nn, 0, st));
  ElemArgs<T> a = level_args<T>(L);
  a.blk0 = blk0;
  a.nblk = nblk;
  if (det) a.evec = op->evec;
  if (w16) a.lin16 = op->lin16;
  if (sizeof(T) == 4) {  // the persistent FP32-arithmetic kernel: two resident blocks per SM
    a.status = op->status;
    a.ctas = 2 * sm_count();
  }
  a.x = x;
  a.y = y;
  long long stride = stride_of(op->Q);
  const T* lin = a.lin;
  a.linP = lin + (transpose ? kWC : kWP) * stride;
  a.linC = lin + (transpose ? kWP : kWC) * stride;
  a.transpose = transpose;
  PFF_CK(elem_dispatch<T>(op->Q, L->p + 1, kApply, a, st));
  if (det && init)
    PFF_CK(launch_node_gather(sizeof(T) == 8 ? 0 : 1, L->mesh, op->evec, level_mask(L), 0, x, nullptr, y, 0,
                              L->mesh.nn, st));
  return PFF_OK;
}

// Double-float action: FP64 vectors, contractions on the FP32 pipes with
// pairs of floats, stored linearisation read from its hi/lo planes.
int apply_df(pff_level* L, const double* x, double* y, int transpose, cudaStream_t st, int blk0 = 0, int nblk = 0,
             bool init = true) {
  pff_op* op = L->op;
  PFF_REQUIRE(op->df && op->lin32, "PFF_DF64 apply needs pff_op_enable_df before pff_residual");
  const bool det = op->det && op->evec;
  if (init && !det) PFF_CK(launch_init_masked(0, y, x, nullptr, level_mask(L), 4 * L->mesh.nn, 0, st));
  ElemArgs<df64> a;
  std::memset(&a, 0, sizeof(a));
  a.blk0 = blk0;
  a.nblk = nblk;
  if (det) a.evec = op->evec;
  a.mesh = L->mesh;
  a.mask = level_mask(L);
  a.emask = a.mask ? level_emask(L) : nullptr;
  a.B = L->tab.B64;
  a.Dc = L->tab.Dc64;
  a.Dt = L->tab.Dt64;
  a.nq = op->nq;
  a.kx = op->geo != nullptr;
  a.x = x;
  a.y = y;
  const long long stride = stride_of(op->Q);
  a.lin = op->lin32;
  a.linP = op->lin32 + (transpose ? kWC : kWP) * stride;
  a.linC = op->lin32 + (transpose ? kWP : kWC) * stride;
  a.lo = op->lin_len;
  a.transpose = transpose;
  PFF_CK(elem_dispatch<df64>(op->Q, L->p + 1, kApply, a, st));
  if (det && init)
    PFF_CK(launch_node_gather(0, L->mesh, op->evec, level_mask(L), 0, x, nullptr, y, 0, L->mesh.nn, st));
  return PFF_OK;
}

template <typename T>
int diag_t(pff_level* L, T* diag, cudaStream_t st) {
  pff_op* op = L->op;
  PFF_REQUIRE(linOf<T>(op) != nullptr, "FP32 diagonal needs pff_op_enable_f32 before pff_residual");
  const bool det = op->det && op->evec;
  if (!det)
    PFF_CK(launch_init_masked(sizeof(T) == 8 ? 0 : 1, diag, nullptr, nullptr, level_mask(L), 4 * L->mesh.nn, 2, st));
  ElemArgs<T> a = level_args<T>(L);
  a.y = diag;
  if (det) a.evec = op->evec;
  PFF_CK(diag_dispatch<T>(op->Q, L->p + 1, a, st));
  if (det)
    PFF_CK(launch_node_gather(sizeof(T) == 8 ? 0 : 1, L->mesh, op->evec, level_mask(L), 2, nullptr, nullptr, diag, 0,
                              L->mesh.nn, st));
  return PFF_OK;
}

int ensure_prolong_table(pff_level* c, pff_level* f) {
  if (c->I_pf == f->p) return PFF_OK;
  cudaFree(c->I64); cudaFree(c->I32);
  c->I64 = nullptr; c->I32 = nullptr;
  int pc = c->p, pf = f->p;
  std::vector<double> xc(pc + 1), xf(pf + 1);
  gll_nodes(pc, xc.data());
  gll_nodes(pf, xf.data());
  std::vector<double> I((pf + 1) * (pc + 1));
  for (int a = 0; a <= pf; ++a)
    for (int b = 0; b <= pc; ++b) I[a * (pc + 1) + b] = lagrange(xc.data(), pc + 1, b, xf[a]);
  int rc;
  if ((rc = upload(I, &c->I64))) return rc;
  if ((rc = upload(I, &c->I32))) return rc;
  c->I_pf = pf;
  return PFF_OK;
}

}  // namespace

template <typename T>
static int cheb_t(pff_level* L, int degree, double lmin, double lmax, const T* diag, const T* b, T* x, T* work,
                  cudaStream_t st, bool w16 = false) {
  const long long n = 4 * L->mesh.nn;
  T* r = work;
  T* d = work + n;
  T* Ad = work + 2 * n;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  int rc = apply_t<T>(L, x, Ad, 0, st, w16);
  if (rc) return rc;
  PFF_CK(launch_cheb_init<T>(n, b, Ad, diag, r, d, 1.0 / theta, st));
  for (int k = 0; k < degree; ++k) {
    if (k == degree - 1) {
      PFF_CK(launch_cheb_step<T>(n, x, d, r, Ad, diag, 0.0, 0.0, 1, st));
      break;
    }
    rc = apply_t<T>(L, d, Ad, 0, st, w16);
    if (rc) return rc;
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    PFF_CK(launch_cheb_step<T>(n, x, d, r, Ad, diag, rho_new * rho, 2.0 * rho_new / delta, 0, st));
    rho = rho_new;
  }
  return PFF_OK;
}

namespace pff {
int apply_blocks(pff_level* L, int prec, const void* x, void* y, int transpose, int blk0, int nblk, cudaStream_t st) {
  if (prec == PFF_F64) return apply_t<double>(L, (const double*)x, (double*)y, transpose, st, false, blk0, nblk, false);
  if (prec == PFF_F32 || prec == PFF_F32_BF16)
    return apply_t<float>(L, (const float*)x, (float*)y, transpose, st, prec == PFF_F32_BF16, blk0, nblk, false);
  if (prec == PFF_DF64) return apply_df(L, (const double*)x, (double*)y, transpose, st, blk0, nblk, false);
  return fail(PFF_ERR_INVALID, "unknown precision");
}
const uint8_t* level_rows_mask(const pff_level* L) { return level_mask(L); }
int set_last_error(int code, const char* msg) { return fail(code, msg); }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace pff

extern "C" {

const char* pff_last_error_message(void) { return g_err.c_str(); }
int pff_version(void) { return 1; }
int64_t pff_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int pff_create_context(pff_ctx** out, const pff_problem* pr) {
  PFF_REQUIRE(out && pr, "pff_create_context: null argument");
  PFF_REQUIRE(pr->nphase >= 1 && pr->nphase <= kMaxPhase, "pff_create_context: 1 <= nphase <= 8");
  PFF_REQUIRE(pr->at == 1 || pr->at == 2, "pff_create_context: at must be 1 (AT1) or 2 (AT2)");
  PFF_REQUIRE(pr->dt > 0.0, "pff_create_context: dt must be positive");
  PFF_REQUIRE(pr->phase_params != nullptr, "pff_create_context: phase_params is null");
  pff_ctx* c = new (std::nothrow) pff_ctx();
  if (!c) return fail(PFF_ERR_INVALID, "out of host memory");
  c->nphase = pr->nphase;
  const double c0 = (pr->at == 1) ? 8.0 / 3.0 : 2.0;
  for (int i = 0; i < pr->nphase; ++i) {
    const double* v = pr->phase_params + 12 * i;
    PhaseDev& ph = c->phase[i];
    std::memset(&ph, 0, sizeof(ph));
    const double E[3] = {v[2], v[5], v[9]};
    const double nu[3] = {v[3], v[6], v[10]};
    ph.has[0] = 1;
    ph.has[1] = v[4] != 0.0;
    ph.has[2] = v[8] != 0.0;
    ph.kap_tot = 0.0;
    for (int b = 0; b < 3; ++b) {
      if (!ph.has[b]) continue;
      if (!(E[b] > 0.0) || !(nu[b] > -1.0 && nu[b] < 0.5)) {
        delete c;
        return fail(PFF_ERR_INVALID, "pff_create_context: branch moduli must satisfy E > 0, -1 < nu < 0.5");
      }
      ph.mu[b] = E[b] / (2.0 * (1.0 + nu[b]));
      ph.kap[b] = E[b] / (3.0 * (1.0 - 2.0 * nu[b]));
      ph.kap_tot += ph.kap[b];
    }
    ph.cmax = (ph.has[1] && std::isfinite(v[7])) ? ph.mu[1] * pr->dt / v[7] : 0.0;
    ph.E0 = v[2];
    ph.nu0 = v[3];
    ph.eta_d = (ph.has[1] && std::isfinite(v[7])) ? v[7] : 0.0;
    ph.Gc = v[0];
    ph.l0 = v[1];
    ph.c0 = c0;
    ph.sig0 = v[11];
    ph.Hlin = 0.0;
    ph.sinf = v[11];
    ph.beta = 0.0;
    ph.hard = 0;
    ph.gc_c0l0 = v[0] / (c0 * v[1]);
    ph.kphi = pr->s_phi * 2.0 * v[0] * v[1] / c0;
  }
  c->glob.at = pr->at;
  c->glob.eta = pr->eta;
  c->glob.zeta = pr->zeta;
  c->glob.dt = pr->dt;
  c->glob.s_phi = pr->s_phi;
  *out = c;
  return PFF_OK;
}

int pff_destroy_context(pff_ctx* ctx) {
  delete ctx;
  return PFF_OK;
}

int pff_context_set_hardening(pff_ctx* ctx, int phase, double H_lin, double sigma_inf, double beta) {
  PFF_REQUIRE(ctx, "pff_context_set_hardening: null context");
  PFF_REQUIRE(phase >= 0 && phase < ctx->nphase, "pff_context_set_hardening: phase out of range");
  PhaseDev& ph = ctx->phase[phase];
  PFF_REQUIRE(ph.has[2], "pff_context_set_hardening: the phase has no Prandtl branch");
  PFF_REQUIRE(H_lin >= 0.0 && beta >= 0.0 && sigma_inf >= ph.sig0 && std::isfinite(H_lin) && std::isfinite(beta) &&
                  std::isfinite(sigma_inf),
              "pff_context_set_hardening: need H_lin >= 0, beta >= 0, sigma_inf >= sigma0 (non-decreasing sigma_y)");
  ph.Hlin = H_lin;
  ph.sinf = sigma_inf;
  ph.beta = beta;
  ph.hard = (H_lin != 0.0 || (sigma_inf != ph.sig0 && beta != 0.0)) ? 1 : 0;
  return PFF_OK;
}

int pff_context_set_time_step(pff_ctx* ctx, double dt) {
  PFF_REQUIRE(ctx, "pff_context_set_time_step: null context");
  PFF_REQUIRE(dt > 0.0 && std::isfinite(dt), "pff_context_set_time_step: dt must be positive and finite");
  ctx->glob.dt = dt;
  for (int i = 0; i < ctx->nphase; ++i) {
    PhaseDev& ph = ctx->phase[i];
    ph.cmax = (ph.has[1] && ph.eta_d > 0.0) ? ph.mu[1] * dt / ph.eta_d : 0.0;
  }
  return PFF_OK;
}

int pff_create_basis(pff_ctx* ctx, int p, int q, pff_basis** out) {
  PFF_REQUIRE(ctx && out, "pff_create_basis: null argument");
  PFF_REQUIRE(p >= 1 && q >= p + 1 && q <= kMaxQ, "pff_create_basis: need 1 <= p and p + 1 <= q <= 5");
  pff_basis* b = new pff_basis();
  b->p = p; b->q = q;
  int P = p + 1;
  b->xg.resize(P); b->xq.resize(q); b->wq.resize(q);
  gll_nodes(p, b->xg.data());
  gauss_rule(q, b->xq.data(), b->wq.data());
  b->B.resize(q * P); b->Dt.resize(q * P); b->Dc.resize(q * q);
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < P; ++a) {
      b->B[i * P + a] = lagrange(b->xg.data(), P, a, b->xq[i]);
      b->Dt[i * P + a] = lagrange_deriv(b->xg.data(), P, a, b->xq[i]);
    }
    for (int k = 0; k < q; ++k) b->Dc[i * q + k] = lagrange_deriv(b->xq.data(), q, k, b->xq[i]);
  }
  *out = b;
  return PFF_OK;
}

int pff_basis_get(const pff_basis* b, double* xg, double* xq, double* wq, double* B, double* Dc) {
  PFF_REQUIRE(b, "pff_basis_get: null basis");
  if (xg) std::memcpy(xg, b->xg.data(), sizeof(double) * b->xg.size());
  if (xq) std::memcpy(xq, b->xq.data(), sizeof(double) * b->xq.size());
  if (wq) std::memcpy(wq, b->wq.data(), sizeof(double) * b->wq.size());
  if (B) std::memcpy(B, b->B.data(), sizeof(double) * b->B.size());
  if (Dc) std::memcpy(Dc, b->Dc.data(), sizeof(double) * b->Dc.size());
  return PFF_OK;
}

int pff_destroy_basis(pff_basis* b) {
  delete b;
  return PFF_OK;
}

int pff_create_restriction(pff_ctx* ctx, const pff_box* box, int p, const int32_t* offsets, int64_t nnodes,
                           pff_restr** out) {
  PFF_REQUIRE(ctx && box && out, "pff_create_restriction: null argument");
  PFF_REQUIRE(box->nx >= 1 && box->ny >= 1 && box->nz >= 1, "pff_create_restriction: empty element grid");
  PFF_REQUIRE(box->hx > 0 && box->hy > 0 && box->hz > 0, "pff_create_restriction: element sizes must be positive");
  PFF_REQUIRE(p >= 1 && p + 1 <= kMaxQ, "pff_create_restriction: 1 <= p <= 4");
  long long nn_box = (long long)(p * box->nx + 1) * (p * box->ny + 1) * (p * box->nz + 1);
  PFF_REQUIRE(offsets || nnodes == nn_box, "pff_create_restriction: nnodes does not match the structured box");
  PFF_REQUIRE(nnodes > 0 && nnodes < (1LL << 40), "pff_create_restriction: nnodes out of range");
  pff_restr* r = new pff_restr();
  r->box = *box;
  r->p = p;
  r->offsets = offsets;
  r->nn = nnodes;
  *out = r;
  return PFF_OK;
}

int pff_destroy_restriction(pff_restr* r) {
  delete r;
  return PFF_OK;
}

int pff_create_operator(pff_ctx* ctx, pff_basis* fine, pff_restr* restr, pff_op** out) {
  PFF_REQUIRE(ctx && fine && restr && out, "pff_create_operator: null argument");
  PFF_REQUIRE(fine->p == restr->p, "pff_create_operator: basis and restriction orders differ");
  pff_op* op = new pff_op();
  op->ctx = ctx;
  op->p = fine->p;
  op->Q = fine->q;
  op->box = restr->box;
  op->mesh = mesh_for(restr->box, fine->p, restr->offsets);
  op->mesh.nn = restr->nn;
  op->nel = op->mesh.nel;
  op->nq = op->nel * (long long)op->Q * op->Q * op->Q;
  op->geom.s[0] = 2.0 / restr->box.hx;
  op->geom.s[1] = 2.0 / restr->box.hy;
  op->geom.s[2] = 2.0 / restr->box.hz;
  op->geom.detJ = restr->box.hx * restr->box.hy * restr->box.hz / 8.0;
  for (int i = 0; i < kMaxQ; ++i) op->geom.wq[i] = (i < op->Q) ? fine->wq[i] : 0.0;
  int EB = elems_per_block(op->Q);
  long long nblk = (op->nel + EB - 1) / EB;
  op->lin_len = nblk * kLinWords * stride_of(op->Q);
  int rc = make_tables(op->p, op->Q, op->tab);
  if (rc) { delete op; return rc; }
  cudaError_t e = cudaSuccess;
  e = cudaMalloc((void**)&op->hist_c, sizeof(double) * 15 * op->nq);
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->hist_t, sizeof(double) * 15 * op->nq);
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->phase, op->nq);
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->flags, op->nq);
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->lin64, sizeof(double) * op->lin_len);
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->io, sizeof(double) * 13 * op->nq);
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(op->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(op->phase, 0, op->nq);
  if (e == cudaSuccess) e = cudaMemset(op->lin64, 0, sizeof(double) * op->lin_len);
  if (e != cudaSuccess) {
    pff_destroy_operator(op);
    return fail(PFF_ERR_CUDA, std::string("pff_create_operator: ") + cudaGetErrorString(e));
  }
  *out = op;
  return PFF_OK;
}

int pff_destroy_operator(pff_op* op) {
  if (!op) return PFF_OK;
  cudaFree(op->hist_c); cudaFree(op->hist_t); cudaFree(op->phase); cudaFree(op->flags);
  cudaFree(op->lin64); cudaFree(op->lin32); cudaFree(op->lin16); cudaFree(op->io); cudaFree(op->mask);
  cudaFree(op->emask);
  cudaFree(op->evec);
  cudaFree(op->dvals); cudaFree(op->status);
  cudaFree(op->fint); cudaFree(op->sums); cudaFree(op->geo);
  free_tables(op->tab);
  delete op;
  return PFF_OK;
}

int pff_op_enable_f32(pff_op* op, int enable) {
  PFF_REQUIRE(op, "pff_op_enable_f32: null operator");
  if (enable && !op->lin32) {
    PFF_CK(cudaMalloc((void**)&op->lin32, sizeof(float) * (op->lin_len + kLin32Pad)));
    PFF_CK(cudaMemset(op->lin32, 0, sizeof(float) * (op->lin_len + kLin32Pad)));
    op->lin32_planes = 1;
  }
  if (!enable && op->lin32) {
    cudaFree(op->lin32);
    op->lin32 = nullptr;
    op->lin32_planes = 0;
    op->df = 0;
  }
  op->f32 = enable ? 1 : 0;
  return PFF_OK;
}

int pff_op_enable_df(pff_op* op, int enable) {
  PFF_REQUIRE(op, "pff_op_enable_df: null operator");
  if (enable && op->lin32_planes < 2) {
    float* planes = nullptr;
    PFF_CK(cudaMalloc((void**)&planes, sizeof(float) * (2 * op->lin_len + kLin32Pad)));
    const cudaError_t e = cudaMemset(planes, 0, sizeof(float) * (2 * op->lin_len + kLin32Pad));
    if (e != cudaSuccess) cudaFree(planes);  // keep the operator as it was
    PFF_CK(e);
    cudaFree(op->lin32);
    op->lin32 = planes;
    op->lin32_planes = 2;
  }
  if (enable) op->f32 = 1;
  op->df = enable ? 1 : 0;  // disabling keeps both planes allocated until pff_op_enable_f32(op, 0)
  return PFF_OK;
}

int pff_op_set_deterministic(pff_op* op, int enable) {
  PFF_REQUIRE(op, "pff_op_set_deterministic: null operator");
  if (enable) {
    PFF_REQUIRE(op->mesh.offsets == nullptr, "pff_op_set_deterministic: needs the structured element numbering");
    if (!op->evec) {
      const long long P = op->p + 1;
      const size_t bytes = sizeof(double) * 4 * (size_t)P * P * P * (size_t)(op->mesh.nel > 0 ? op->mesh.nel : 1);
      PFF_CK(cudaMalloc(&op->evec, bytes));
    }
  } else {
    cudaFree(op->evec);
    op->evec = nullptr;
  }
  op->det = enable ? 1 : 0;
  return PFF_OK;
}

int pff_op_enable_bf16(pff_op* op, int enable) {
  PFF_REQUIRE(op, "pff_op_enable_bf16: null operator");
  if (enable && !op->lin16) {
    const long long nblk = op->lin_len / (kLinWords * stride_of(op->Q));
    const long long len = nblk * kLin16Words * stride_of(op->Q);
    PFF_CK(cudaMalloc((void**)&op->lin16, sizeof(uint16_t) * len));
    const cudaError_t e = cudaMemset(op->lin16, 0, sizeof(uint16_t) * len);
    if (e != cudaSuccess) {
      cudaFree(op->lin16);
      op->lin16 = nullptr;
    }
    PFF_CK(e);
    op->lin16_len = len;
  }
  if (!enable && op->lin16) {
    cudaFree(op->lin16);
    op->lin16 = nullptr;
    op->lin16_len = 0;
  }
  op->bf16 = enable ? 1 : 0;
  return PFF_OK;
}

int64_t pff_op_num_qpoints(const pff_op* op) { return op ? op->nq : -1; }
int64_t pff_op_num_nodes(const pff_op* op) { return op ? op->mesh.nn : -1; }

int pff_set_qpoint_state(pff_op* op, const uint8_t* phase, const double* hist, void* stream) {
  PFF_REQUIRE(op && phase && hist, "pff_set_qpoint_state: null argument");
  PFF_CK(cudaMemcpyAsync(op->phase, phase, op->nq, cudaMemcpyDeviceToDevice, S(stream)));
  PFF_CK(cudaMemcpyAsync(op->hist_c, hist, sizeof(double) * 15 * op->nq, cudaMemcpyDeviceToDevice, S(stream)));
  return PFF_OK;
}

int pff_set_dirichlet(pff_op* op, const uint8_t* mask, const double* values, void* stream) {
  PFF_REQUIRE(op, "pff_set_dirichlet: null operator");
  long long n = 4 * op->mesh.nn;
  if (!mask) {
    cudaFree(op->mask); op->mask = nullptr;
    cudaFree(op->emask);
  cudaFree(op->evec); op->emask = nullptr;
    cudaFree(op->dvals); op->dvals = nullptr;
    return PFF_OK;
  }
  if (!op->mask) PFF_CK(cudaMalloc((void**)&op->mask, n));
  if (!op->emask) PFF_CK(cudaMalloc((void**)&op->emask, op->mesh.nel > 0 ? op->mesh.nel : 1));
  PFF_CK(cudaMemcpyAsync(op->mask, mask, n, cudaMemcpyDeviceToDevice, S(stream)));
  PFF_CK(launch_elem_mask(op->mesh, op->mask, op->emask, S(stream)));
  if (values) {
    if (!op->dvals) PFF_CK(cudaMalloc((void**)&op->dvals, sizeof(double) * n));
    PFF_CK(cudaMemcpyAsync(op->dvals, values, sizeof(double) * n, cudaMemcpyDeviceToDevice, S(stream)));
  } else if (op->dvals) {
    PFF_CK(cudaMemsetAsync(op->dvals, 0, sizeof(double) * n, S(stream)));
  }
  return PFF_OK;
}

int pff_op_set_geometry(pff_op* op, const double* X, void* stream) {
  PFF_REQUIRE(op, "pff_op_set_geometry: null operator");
  cudaStream_t st = S(stream);
  if (!X) {
    PFF_CK(cudaStreamSynchronize(st));
    cudaFree(op->geo);
    op->geo = nullptr;
    return PFF_OK;
  }
  const long long nn = op->mesh.nn, nq = op->nq;
  // the status word reports inverted elements here; bits still pending from
  // earlier calls are set aside and put back afterwards
  int h0 = 0;
  PFF_CK(cudaStreamSynchronize(st));
  PFF_CK(cudaMemcpy(&h0, op->status, sizeof(int), cudaMemcpyDeviceToHost));
  PFF_CK(cudaMemset(op->status, 0, sizeof(int)));
  if (!op->geo) PFF_CK(cudaMalloc((void**)&op->geo, sizeof(double) * 10 * nq));
  // parent Jacobians dX_f / dxi_al at every Gauss point: an eval of the
  // coordinates (fourth field zero) with unit parent-to-reference factors
  double* xc = nullptr;
  PFF_CK(cudaMalloc((void**)&xc, sizeof(double) * 4 * nn));
  cudaError_t e = cudaMemcpyAsync(xc, X, sizeof(double) * 3 * nn, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(xc + 3 * nn, 0, sizeof(double) * nn, st);
  ElemArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  a.mesh = op->mesh;
  a.x = xc;
  a.B = op->tab.B64;
  a.Dc = op->tab.Dc64;
  a.Dt = op->tab.Dt64;
  a.scratch = op->io;
  a.nq = nq;
  for (int d = 0; d < 3; ++d) a.s[d] = 1.0;
  if (e == cudaSuccess) e = elem_dispatch<double>(op->Q, op->p + 1, kEval, a, st);
  if (e == cudaSuccess) e = launch_geometry(op->io, op->geo, op->geom, op->Q, nq, op->status, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(xc);
  if (e != cudaSuccess) return fail(PFF_ERR_CUDA, std::string("pff_op_set_geometry: ") + cudaGetErrorString(e));
  int h = 0;
  PFF_CK(cudaMemcpy(&h, op->status, sizeof(int), cudaMemcpyDeviceToHost));
  PFF_CK(cudaMemcpy(op->status, &h0, sizeof(int), cudaMemcpyHostToDevice));
  if (h & 2) {
    cudaFree(op->geo);
    op->geo = nullptr;
    return fail(PFF_ERR_INVALID, "pff_op_set_geometry: det J <= 0 at some Gauss point (inverted element)");
  }
  return PFF_OK;
}

int pff_residual(pff_op* op, const double* z, double* r, void* stream) {
  PFF_REQUIRE(op && z && r, "pff_residual: null argument");
  cudaStream_t st = S(stream);
  const long long n = 4 * op->mesh.nn;
  const bool det = op->det && op->evec;
  if (!det) PFF_CK(launch_init_masked(0, r, z, op->dvals, op->mask, n, 1, st));
  ElemArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  a.mesh = op->mesh;
  a.x = z;
  a.mask = nullptr;
  a.B = op->tab.B64;
  a.Dc = op->tab.Dc64;
  a.Dt = op->tab.Dt64;
  a.scratch = op->io;
  a.nq = op->nq;
  a.geo = op->geo;
  for (int d = 0; d < 3; ++d) a.s[d] = op->geom.s[d];
  PFF_CK(elem_dispatch<double>(op->Q, op->p + 1, kEval, a, st));
  PointArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  for (int i = 0; i < op->ctx->nphase; ++i) pa.phase[i] = op->ctx->phase[i];
  pa.glob = op->ctx->glob;
  pa.geom = op->geom;
  pa.Q = op->Q;
  pa.nphase = op->ctx->nphase;
  pa.nq = op->nq;
  pa.nel = op->nel;
  pa.io = op->io;
  pa.hist = op->hist_c;
  pa.hist_trial = op->hist_t;
  pa.phase_id = op->phase;
  pa.flags = op->flags;
  pa.lin = op->lin64;
  pa.status = op->status;
  pa.geo = op->geo;
  pa.want_tangent = 1;
  PFF_CK(launch_pointwise(pa, st));
  a.y = r;
  a.mask = op->mask;
  a.emask = op->mask ? op->emask : nullptr;
  if (det) a.evec = op->evec;
  PFF_CK(elem_dispatch<double>(op->Q, op->p + 1, kBack, a, st));
  if (det) PFF_CK(launch_node_gather(0, op->mesh, op->evec, op->mask, 1, z, op->dvals, r, 0, op->mesh.nn, st));
  float* w32 = (op->f32 && op->lin32) ? op->lin32 : nullptr;
  PFF_CK(launch_split_words(op->lin64, w32, w32 && op->df ? op->lin32 + op->lin_len : nullptr,
                            (op->bf16 && op->lin16) ? op->lin16 : nullptr,
                            op->lin_len / (kLinWords * stride_of(op->Q)), op->Q, st));
  return PFF_OK;
}

int pff_apply_dirichlet(pff_op* op, double* z, void* stream) {
  PFF_REQUIRE(op && z, "pff_apply_dirichlet: null argument");
  PFF_CK(launch_apply_dirichlet(z, op->dvals, op->mask, 4 * op->mesh.nn, S(stream)));
  return PFF_OK;
}

int pff_reaction(pff_op* op, const uint8_t* sel, double* out4, void* stream) {
  PFF_REQUIRE(op && sel && out4, "pff_reaction: null argument");
  cudaStream_t st = S(stream);
  const long long n = 4 * op->mesh.nn;
  if (!op->fint) PFF_CK(cudaMalloc((void**)&op->fint, sizeof(double) * n));
  if (!op->sums) PFF_CK(cudaMalloc((void**)&op->sums, sizeof(double) * 8));
  PFF_CK(cudaMemsetAsync(op->fint, 0, sizeof(double) * n, st));
  ElemArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  a.mesh = op->mesh;
  a.y = op->fint;
  a.mask = nullptr;
  a.B = op->tab.B64;
  a.Dc = op->tab.Dc64;
  a.Dt = op->tab.Dt64;
  a.scratch = op->io;
  a.nq = op->nq;
  PFF_CK(elem_dispatch<double>(op->Q, op->p + 1, kBack, a, st));
  PFF_CK(launch_masked_field_sums(op->fint, sel, op->mesh.nn, op->sums, st));
  PFF_CK(cudaMemcpyAsync(out4, op->sums, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
  PFF_CK(cudaStreamSynchronize(st));
  return PFF_OK;
}

int pff_create_level(pff_op* fine, int p, pff_level** out) {
  PFF_REQUIRE(fine && out, "pff_create_level: null argument");
  PFF_REQUIRE(p >= 1 && p <= fine->p, "pff_create_level: 1 <= p_level <= fine order");
  PFF_REQUIRE(p == fine->p || fine->mesh.offsets == nullptr,
              "pff_create_level: coarse levels need the structured restriction");
  pff_level* L = new pff_level();
  L->op = fine;
  L->p = p;
  L->is_fine = (p == fine->p);
  L->mesh = L->is_fine ? fine->mesh : mesh_for(fine->box, p, nullptr);
  int rc = make_tables(p, fine->Q, L->tab);
  if (rc) { delete L; return rc; }
  *out = L;
  return PFF_OK;
}

int pff_destroy_level(pff_level* L) {
  if (!L) return PFF_OK;
  pff::free_host_io(L);
  free_tables(L->tab);
  cudaFree(L->mask);
  cudaFree(L->emask);
  cudaFree(L->I64); cudaFree(L->I32);
  delete L;
  return PFF_OK;
}

int64_t pff_level_num_nodes(const pff_level* L) { return L ? L->mesh.nn : -1; }

int pff_level_set_mask(pff_level* L, const uint8_t* mask, void* stream) {
  PFF_REQUIRE(L, "pff_level_set_mask: null level");
  PFF_REQUIRE(!L->is_fine, "pff_level_set_mask: the fine level uses pff_set_dirichlet");
  long long n = 4 * L->mesh.nn;
  if (!mask) {
    cudaFree(L->mask); L->mask = nullptr;
    cudaFree(L->emask); L->emask = nullptr;
    return PFF_OK;
  }
  if (!L->mask) PFF_CK(cudaMalloc((void**)&L->mask, n));
  if (!L->emask) PFF_CK(cudaMalloc((void**)&L->emask, L->mesh.nel > 0 ? L->mesh.nel : 1));
  PFF_CK(cudaMemcpyAsync(L->mask, mask, n, cudaMemcpyDeviceToDevice, S(stream)));
  PFF_CK(launch_elem_mask(L->mesh, L->mask, L->emask, S(stream)));
  return PFF_OK;
}

int pff_jacobian_apply(pff_level* L, pff_prec prec, const void* x, void* y, void* stream) {
  PFF_REQUIRE(L && x && y, "pff_jacobian_apply: null argument");
  if (prec == PFF_F64) return apply_t<double>(L, (const double*)x, (double*)y, 0, S(stream));
  if (prec == PFF_F32) return apply_t<float>(L, (const float*)x, (float*)y, 0, S(stream));
  if (prec == PFF_DF64) return apply_df(L, (const double*)x, (double*)y, 0, S(stream));
  if (prec == PFF_F32_BF16) return apply_t<float>(L, (const float*)x, (float*)y, 0, S(stream), true);
  return fail(PFF_ERR_INVALID, "pff_jacobian_apply: unknown precision");
}

int pff_jacobian_transpose_apply(pff_level* L, pff_prec prec, const void* x, void* y, void* stream) {
  PFF_REQUIRE(L && x && y, "pff_jacobian_transpose_apply: null argument");
  if (prec == PFF_F64) return apply_t<double>(L, (const double*)x, (double*)y, 1, S(stream));
  if (prec == PFF_F32) return apply_t<float>(L, (const float*)x, (float*)y, 1, S(stream));
  if (prec == PFF_DF64) return apply_df(L, (const double*)x, (double*)y, 1, S(stream));
  if (prec == PFF_F32_BF16) return apply_t<float>(L, (const float*)x, (float*)y, 1, S(stream), true);
  return fail(PFF_ERR_INVALID, "pff_jacobian_transpose_apply: unknown precision");
}

int pff_assemble_diagonal(pff_level* L, pff_prec prec, void* diag, void* stream) {
  PFF_REQUIRE(L && diag, "pff_assemble_diagonal: null argument");
  if (prec == PFF_F64) return diag_t<double>(L, (double*)diag, S(stream));
  if (prec == PFF_F32 || prec == PFF_F32_BF16) return diag_t<float>(L, (float*)diag, S(stream));
  return fail(PFF_ERR_INVALID, "pff_assemble_diagonal: unknown precision");
}

int pff_prolong(pff_level* c, pff_level* f, pff_prec prec, const void* xc, void* xf, void* stream) {
  PFF_REQUIRE(c && f && xc && xf, "pff_prolong: null argument");
  PFF_REQUIRE(c->op == f->op && c->p < f->p, "pff_prolong: levels must share the operator, coarse p < fine p");
  PFF_REQUIRE(f->mesh.offsets == nullptr, "pff_prolong: structured restriction required");
  int rc = ensure_prolong_table(c, f);
  if (rc) return rc;
  const uint8_t* mc = level_mask(c);
  const uint8_t* mf = level_mask(f);
  if (prec == PFF_F64) PFF_CK(launch_prolong<double>(c->mesh, f->mesh, c->I64, (const double*)xc, (double*)xf, mc, mf, S(stream)));
  else if (prec == PFF_F32 || prec == PFF_F32_BF16) PFF_CK(launch_prolong<float>(c->mesh, f->mesh, c->I32, (const float*)xc, (float*)xf, mc, mf, S(stream)));
  else return fail(PFF_ERR_INVALID, "pff_prolong: unknown precision");
  return PFF_OK;
}

int pff_restrict(pff_level* c, pff_level* f, pff_prec prec, const void* rf, void* rc_, void* stream) {
  PFF_REQUIRE(c && f && rf && rc_, "pff_restrict: null argument");
  PFF_REQUIRE(c->op == f->op && c->p < f->p, "pff_restrict: levels must share the operator, coarse p < fine p");
  PFF_REQUIRE(f->mesh.offsets == nullptr, "pff_restrict: structured restriction required");
  int rc = ensure_prolong_table(c, f);
  if (rc) return rc;
  const uint8_t* mc = level_mask(c);
  const uint8_t* mf = level_mask(f);
  void* ev = (c->op->det && c->op->evec) ? c->op->evec : nullptr;
  if (prec == PFF_F64) PFF_CK(launch_restrict<double>(c->mesh, f->mesh, c->I64, (const double*)rf, (double*)rc_, mc, mf, S(stream), ev));
  else if (prec == PFF_F32 || prec == PFF_F32_BF16) PFF_CK(launch_restrict<float>(c->mesh, f->mesh, c->I32, (const float*)rf, (float*)rc_, mc, mf, S(stream), ev));
  else return fail(PFF_ERR_INVALID, "pff_restrict: unknown precision");
  return PFF_OK;
}

int pff_chebyshev_smooth(pff_level* L, pff_prec prec, int degree, double lmin, double lmax, const void* diag,
                         const void* b, void* x, void* work, void* stream) {
  PFF_REQUIRE(L && diag && b && x && work, "pff_chebyshev_smooth: null argument");
  PFF_REQUIRE(degree >= 1 && degree <= 64, "pff_chebyshev_smooth: 1 <= degree <= 64");
  PFF_REQUIRE(lmax > lmin && lmin > 0.0, "pff_chebyshev_smooth: need 0 < lmin < lmax");
  if (prec == PFF_F64)
    return cheb_t<double>(L, degree, lmin, lmax, (const double*)diag, (const double*)b, (double*)x, (double*)work, S(stream));
  if (prec == PFF_F32 || prec == PFF_F32_BF16)
    return cheb_t<float>(L, degree, lmin, lmax, (const float*)diag, (const float*)b, (float*)x, (float*)work, S(stream),
                         prec == PFF_F32_BF16);
  return fail(PFF_ERR_INVALID, "pff_chebyshev_smooth: unknown precision");
}

int pff_commit_history(pff_op* op, void* stream) {
  PFF_REQUIRE(op, "pff_commit_history: null operator");
  PFF_CK(cudaMemcpyAsync(op->hist_c, op->hist_t, sizeof(double) * 15 * op->nq, cudaMemcpyDeviceToDevice, S(stream)));
  return PFF_OK;
}

int pff_get_history(pff_op* op, int which, double* hist, void* stream) {
  PFF_REQUIRE(op && hist && (which == 0 || which == 1), "pff_get_history: bad argument");
  PFF_CK(cudaMemcpyAsync(hist, which ? op->hist_t : op->hist_c, sizeof(double) * 15 * op->nq,
                         cudaMemcpyDeviceToDevice, S(stream)));
  return PFF_OK;
}

int pff_state_summary(pff_op* op, const double* z, double* out8, void* stream) {
  PFF_REQUIRE(op && z && out8, "pff_state_summary: null argument");
  cudaStream_t st = S(stream);
  if (!op->sums) PFF_CK(cudaMalloc((void**)&op->sums, sizeof(double) * 8));
  PFF_CK(launch_state_summary(op->flags, op->hist_c, op->nq, z + 3 * op->mesh.nn, op->mesh.nn, op->sums, st));
  PFF_CK(cudaMemcpyAsync(out8, op->sums, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
  PFF_CK(cudaStreamSynchronize(st));
  return PFF_OK;
}

int pff_get_flags(pff_op* op, uint8_t* flags, void* stream) {
  PFF_REQUIRE(op && flags, "pff_get_flags: null argument");
  PFF_CK(cudaMemcpyAsync(flags, op->flags, op->nq, cudaMemcpyDeviceToDevice, S(stream)));
  return PFF_OK;
}

int pff_get_linearization(pff_op* op, double* out, void* stream) {
  PFF_REQUIRE(op && out, "pff_get_linearization: null argument");
  PFF_CK(launch_untile(op->lin64, out, op->nq, op->Q, S(stream)));
  return PFF_OK;
}

int pff_get_status(pff_op* op, void* stream, int* status) {
  PFF_REQUIRE(op && status, "pff_get_status: null argument");
  PFF_CK(cudaStreamSynchronize(S(stream)));
  int h = 0;
  PFF_CK(cudaMemcpy(&h, op->status, sizeof(int), cudaMemcpyDeviceToHost));
  PFF_CK(cudaMemset(op->status, 0, sizeof(int)));
  *status = h;
  return PFF_OK;
}

}  // extern "C"

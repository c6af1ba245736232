// Jacobian action on host buffers with the copies overlapped (pff_jacobian_apply_host).
//
// The action of Sec. 4 needs, for the elements of one layer of the structured
// grid, only the nodes of the adjacent node layers, and the elements are
// numbered layer by layer (e = ex + nx (ey + ny ez)).  So the element blocks
// are cut into chunks in element order, and:
//   - the copy stream uploads the node layers a chunk reaches (all four
//     fields) ahead of it;
//   - the caller's stream initialises the rows of the new layers (Dirichlet
//     identity rows), runs the chunk's element blocks, and marks the node
//     layers that no later chunk touches as final;
//   - the download stream copies the final layers back while later chunks run.
// The uploads of chunk c + 1 and the downloads of chunk c - 1 then run while
// chunk c computes; only the first chunk's upload and the last chunk's
// download stay exposed.  Chunks are whole multiples of the blocks one wave of
// the element kernel holds, so that no chunk ends in a partly filled wave.
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/pff.h"
#include "pff_handles.h"
#include "pff_internal.h"

namespace pff {

struct HostIO {
  void* xd = nullptr;  // device staging of x and y, 8 bytes per entry
  void* yd = nullptr;
  size_t bytes = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_in = nullptr, ev_out = nullptr, ev_done = nullptr;
  int sms = 0;
};

void free_host_io(pff_level* L) {
  HostIO* h = L->hio;
  if (!h) return;
  cudaFree(h->xd);
  cudaFree(h->yd);
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  for (cudaEvent_t e : {h->ev_start, h->ev_in, h->ev_out, h->ev_done})
    if (e) cudaEventDestroy(e);
  delete h;
  L->hio = nullptr;
}

namespace {

int fail_cuda(const char* what, cudaError_t e) {
  return set_last_error(PFF_ERR_CUDA, (std::string("pff_jacobian_apply_host: ") + what + ": " + cudaGetErrorString(e)).c_str());
}

#define HIO_CK(call)                          \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return fail_cuda(#call, e_); \
  } while (0)

int ensure_host_io(pff_level* L, size_t bytes) {
  if (!L->hio) {
    HostIO* h = new HostIO();
    L->hio = h;
    int dev = 0;
    HIO_CK(cudaGetDevice(&dev));
    HIO_CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
    HIO_CK(cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking));
    HIO_CK(cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&h->ev_start, &h->ev_in, &h->ev_out, &h->ev_done})
      HIO_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  HostIO* h = L->hio;
  if (h->bytes < bytes) {
    cudaFree(h->xd);
    cudaFree(h->yd);
    h->xd = h->yd = nullptr;
    h->bytes = 0;
    HIO_CK(cudaMalloc(&h->xd, bytes));
    HIO_CK(cudaMalloc(&h->yd, bytes));
    h->bytes = bytes;
  }
  return PFF_OK;
}

// Copies node layers [l0, l1) of all four fields between host and device.
int copy_layers(char* dst, const char* src, long long nn, long long layer, long long l0, long long l1, size_t esz,
                cudaMemcpyKind kind, cudaStream_t s) {
  if (l1 <= l0) return PFF_OK;
  const size_t off = (size_t)(l0 * layer) * esz, len = (size_t)((l1 - l0) * layer) * esz;
  for (int f = 0; f < 4; ++f) {
    const size_t base = (size_t)f * (size_t)nn * esz + off;
    HIO_CK(cudaMemcpyAsync(dst + base, src + base, len, kind, s));
  }
  return PFF_OK;
}

}  // namespace
}  // namespace pff

extern "C" int pff_jacobian_apply_host(pff_level* L, pff_prec prec, const void* x_host, void* y_host, int nchunks,
                                       void* stream) {
  using namespace pff;
  if (!L || !x_host || !y_host)
    return set_last_error(PFF_ERR_INVALID, "pff_jacobian_apply_host: null argument");
  if (prec != PFF_F64 && prec != PFF_F32 && prec != PFF_DF64 && prec != PFF_F32_BF16)
    return set_last_error(PFF_ERR_INVALID, "pff_jacobian_apply_host: unknown precision");
  if (nchunks < 1 || nchunks > 4096)
    return set_last_error(PFF_ERR_INVALID, "pff_jacobian_apply_host: 1 <= nchunks <= 4096");
  if (L->mesh.offsets)
    return set_last_error(PFF_ERR_INVALID, "pff_jacobian_apply_host: needs the structured element numbering");
  const MeshDev& m = L->mesh;
  const size_t esz = (prec == PFF_F64 || prec == PFF_DF64) ? 8 : 4;
  const long long nn = m.nn, layer = (long long)m.nnx * m.nny, nlay = nn / layer;
  int rc = ensure_host_io(L, sizeof(double) * 4 * (size_t)nn);
  if (rc) return rc;
  HostIO* h = L->hio;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int Q = L->op->Q;
  const int EB = elems_per_block(Q);
  const long long nel = m.nel, nblk = (nel + EB - 1) / EB;
  // blocks per wave: two resident blocks per SM for the FP64, double-float and
  // BF16-word kernels, three for the FP32 one
  const long long wave = (long long)h->sms * (prec == PFF_F32 ? 3 : 2);
  long long cb = (nblk + nchunks - 1) / nchunks;
  if (nblk > wave) cb = std::max(wave, (cb + wave - 1) / wave * wave);
  char* xd = static_cast<char*>(h->xd);
  char* yd = static_cast<char*>(h->yd);
  const char* xh = static_cast<const char*>(x_host);
  char* yh = static_cast<char*>(y_host);
  const uint8_t* mask = level_rows_mask(L);
  const bool det = L->op->det && L->op->evec;  // deterministic transpose (pff_op_set_deterministic)
  const int vprec = esz == 8 ? 0 : 1;
  const long long per_layer_el = (long long)m.nx * m.ny;
  // the staging buffers are free once the caller's earlier work is done
  HIO_CK(cudaEventRecord(h->ev_start, st));
  HIO_CK(cudaStreamWaitEvent(h->s_in, h->ev_start, 0));
  HIO_CK(cudaStreamWaitEvent(h->s_out, h->ev_start, 0));
  long long have = 0, done = 0;  // node layers uploaded / downloaded so far
  for (long long b0 = 0; b0 < nblk; b0 += cb) {
    const long long b1 = std::min(nblk, b0 + cb);
    const long long e_last = std::min(b1 * EB, nel) - 1;
    const long long need = std::min(nlay, (long long)m.p * (e_last / per_layer_el) + m.p + 1);  // layers [0, need)
    rc = copy_layers(xd, xh, nn, layer, have, need, esz, cudaMemcpyHostToDevice, h->s_in);
    if (rc) return rc;
    HIO_CK(cudaEventRecord(h->ev_in, h->s_in));
    HIO_CK(cudaStreamWaitEvent(st, h->ev_in, 0));
    if (!det) HIO_CK(launch_init_rows(vprec, yd, xd, mask, nn, have * layer, need * layer, st));
    have = std::max(have, need);
    rc = apply_blocks(L, prec, xd, yd, 0, (int)b0, (int)(b1 - b0), st);
    if (rc) return rc;
    // layers below the first node layer of the next chunk's first element are final
    const long long fin = (b1 == nblk) ? nlay : (long long)m.p * ((b1 * EB) / per_layer_el);
    if (fin > done) {
      if (det)  // their rows: the fixed-order sums of the element values
        HIO_CK(launch_node_gather(vprec, m, L->op->evec, mask, 0, xd, nullptr, yd, done * layer, fin * layer, st));
      HIO_CK(cudaEventRecord(h->ev_out, st));
      HIO_CK(cudaStreamWaitEvent(h->s_out, h->ev_out, 0));
      rc = copy_layers(yh, yd, nn, layer, done, fin, esz, cudaMemcpyDeviceToHost, h->s_out);
      if (rc) return rc;
      done = fin;
    }
  }
  HIO_CK(cudaEventRecord(h->ev_done, h->s_out));
  HIO_CK(cudaStreamWaitEvent(st, h->ev_done, 0));
  return PFF_OK;
}

// Element kernels for Q = 3 Gauss points per direction, every P <= Q, FP64, FP32 and double-float (action only).
#include "pff_elem.cuh"

namespace pff {

template <typename T>
cudaError_t launch_elem_q3(int P, int mode, const ElemArgs<T>& a, cudaStream_t st) {
  switch (P) {
    case 2: return launch_elem_pq<2, 3, T>(mode, a, st);
    case 3: return launch_elem_pq<3, 3, T>(mode, a, st);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t launch_diag_q3(int P, const ElemArgs<T>& a, cudaStream_t st) {
  switch (P) {
    case 2: return launch_diag_pq<2, 3, T>(a, st);
    case 3: return launch_diag_pq<3, 3, T>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_elem_q3<double>(int, int, const ElemArgs<double>&, cudaStream_t);
template cudaError_t launch_elem_q3<float>(int, int, const ElemArgs<float>&, cudaStream_t);
template cudaError_t launch_elem_q3<df64>(int, int, const ElemArgs<df64>&, cudaStream_t);
template cudaError_t launch_diag_q3<double>(int, const ElemArgs<double>&, cudaStream_t);
template cudaError_t launch_diag_q3<float>(int, const ElemArgs<float>&, cudaStream_t);

}  // namespace pff

// Element kernels for Q = 5 Gauss points per direction, every P <= Q, FP64, FP32 and double-float (action only).
#include "pff_elem.cuh"

namespace pff {

template <typename T>
cudaError_t launch_elem_q5(int P, int mode, const ElemArgs<T>& a, cudaStream_t st) {
  switch (P) {
    case 2: return launch_elem_pq<2, 5, T>(mode, a, st);
    case 3: return launch_elem_pq<3, 5, T>(mode, a, st);
    case 4: return launch_elem_pq<4, 5, T>(mode, a, st);
    case 5: return launch_elem_pq<5, 5, T>(mode, a, st);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t launch_diag_q5(int P, const ElemArgs<T>& a, cudaStream_t st) {
  switch (P) {
    case 2: return launch_diag_pq<2, 5, T>(a, st);
    case 3: return launch_diag_pq<3, 5, T>(a, st);
    case 4: return launch_diag_pq<4, 5, T>(a, st);
    case 5: return launch_diag_pq<5, 5, T>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_elem_q5<double>(int, int, const ElemArgs<double>&, cudaStream_t);
template cudaError_t launch_elem_q5<float>(int, int, const ElemArgs<float>&, cudaStream_t);
template cudaError_t launch_elem_q5<df64>(int, int, const ElemArgs<df64>&, cudaStream_t);
template cudaError_t launch_diag_q5<double>(int, const ElemArgs<double>&, cudaStream_t);
template cudaError_t launch_diag_q5<float>(int, const ElemArgs<float>&, cudaStream_t);

}  // namespace pff

// FP64 (complex128) instantiation of the FFT passes.
#include "passes_impl.cuh"

namespace ori {
template cudaError_t run_xfwd<double>(int, bool, const XArgs&, cudaStream_t, bool);
template cudaError_t run_xinv<double>(int, const XArgs&, Scalars*, int, cudaStream_t, bool, unsigned*);
template cudaError_t run_strided<double>(int, int, bool, const SArgs&, cudaStream_t, bool);
}  // namespace ori

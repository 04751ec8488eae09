// FP32 (complex64) instantiation of the FFT passes.
#include "passes_impl.cuh"

namespace ori {
template cudaError_t run_xfwd<float>(int, bool, const XArgs&, cudaStream_t, bool);
template cudaError_t run_xinv<float>(int, const XArgs&, Scalars*, int, cudaStream_t, bool, unsigned*);
template cudaError_t run_strided<float>(int, int, bool, const SArgs&, cudaStream_t, bool);
}  // namespace ori

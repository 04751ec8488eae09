// Paired-FP32 (double-float) instantiation of the FFT passes: the arithmetic
// of the mixed solver's FP64-class refinement residual.
#include "passes_impl.cuh"

namespace ori {
template cudaError_t run_xfwd<dfl>(int, bool, const XArgs&, cudaStream_t, bool);
template cudaError_t run_xinv<dfl>(int, const XArgs&, Scalars*, int, cudaStream_t, bool, unsigned*);
template cudaError_t run_strided<dfl>(int, int, bool, const SArgs&, cudaStream_t, bool);
}  // namespace ori

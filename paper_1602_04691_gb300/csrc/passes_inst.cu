// Explicit instantiation of one part of the FFT passes in one arithmetic.
//
// The build compiles this file once per (ORI_PASS_T, ORI_PASS_PART) pair so
// that the passes' many template instances compile in parallel:
//   ORI_PASS_T    1 = float (the FP32 inner solver), 2 = double (FP64),
//                 3 = dfl (paired FP32: the mixed solver's FP64-class residual)
//   ORI_PASS_PART 1 = X forward and inverse passes, 2 = strided forward (Y),
//                 3 = strided inverse (Y), 4 = the fused Z convolution pass
#include "passes_impl.cuh"

#if ORI_PASS_T == 1
#define ORI_T float
#elif ORI_PASS_T == 2
#define ORI_T double
#elif ORI_PASS_T == 3
#define ORI_T dfl
#else
#error "ORI_PASS_T must be 1, 2 or 3"
#endif

namespace ori {
#if ORI_PASS_PART == 1
template cudaError_t run_xfwd<ORI_T>(int, bool, const XArgs&, cudaStream_t, bool);
template cudaError_t run_xinv<ORI_T>(int, const XArgs&, Scalars*, int, cudaStream_t, bool, unsigned*);
#elif ORI_PASS_PART == 2
template cudaError_t run_strided_fwd<ORI_T>(int, bool, const SArgs&, cudaStream_t, bool);
#elif ORI_PASS_PART == 3
template cudaError_t run_strided_inv<ORI_T>(int, const SArgs&, cudaStream_t, bool);
#elif ORI_PASS_PART == 4
template cudaError_t run_zconv<ORI_T>(int, const SArgs&, cudaStream_t, bool);
#else
#error "ORI_PASS_PART must be 1, 2, 3 or 4"
#endif
}  // namespace ori

// Explicit instantiation of the operator pipeline for one (precision, box
// size); the build compiles this file once per pair with -DTC_REAL=float|double
// and -DTC_N=<n> so the specialisations compile in parallel.
#include "tc_pipeline.cuh"

#ifndef TC_REAL
#error "define TC_REAL (float or double)"
#endif
#ifndef TC_N
#error "define TC_N (FFT box size)"
#endif

namespace tc {
TC_INSTANTIATE(TC_REAL, TC_N)
}

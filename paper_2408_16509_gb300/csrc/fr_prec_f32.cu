// Kernels and launch sequences of the library for FP32 values and RK registers:
// the one unit that instantiates them (the ABI calls in through kPrecF32).
#include "fr_impl.cuh"

FR_DEFINE_PREC_TABLE(kPrecF32, float, float)

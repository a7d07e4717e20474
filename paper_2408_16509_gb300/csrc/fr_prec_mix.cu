// Kernels and launch sequences of the library for FP32 values, FP64 RK registers (mixed form):
// the one unit that instantiates them (the ABI calls in through kPrecMixed).
#include "fr_impl.cuh"

FR_DEFINE_PREC_TABLE(kPrecMixed, float, double)

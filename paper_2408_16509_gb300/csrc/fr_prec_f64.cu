// Kernels and launch sequences of the library for FP64 values and RK registers:
// the one unit that instantiates them (the ABI calls in through kPrecF64).
#include "fr_impl.cuh"

FR_DEFINE_PREC_TABLE(kPrecF64, double, double)

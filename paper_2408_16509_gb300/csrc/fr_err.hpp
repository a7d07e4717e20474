// Error reporting shared by every unit of the library: the thread's last
// message (fr_last_error) and the CUDA-call check used by the entry points.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/frgb.h"

namespace frgb {

// message of the last failed call, one per thread, shared by every unit
inline thread_local std::string g_err;

inline int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess)                                              \
      return fail(FR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace frgb

// Internal host/device declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lf.h"
#include "lf_common.cuh"

namespace lf {

// Largest dynamic shared memory a block may ask for on sm_103a (227 KiB).
constexpr uint32_t LF_SMEM_MAX = 227u * 1024u;
constexpr int LF_MAX_PLANES = 8;   // lens planes of one model

// Members summed in FP32 before each fold into the float-float accumulators.
extern int g_member_chunk;

lf_status fail(lf_status st, const char* fmt, ...);

}  // namespace lf

#define LF_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return ::lf::fail(LF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

#define LF_TRY(expr)                  \
  do {                                \
    lf_status s_ = (expr);            \
    if (s_ != LF_OK) return s_;       \
  } while (0)

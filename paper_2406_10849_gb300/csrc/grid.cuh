// The 2^-10 grid that apply operands, frames and message high parts live on.
#pragma once
#include <cuda_runtime.h>

namespace treeot {
namespace {
__device__ __forceinline__ float quant(float v) { return rintf(v * 1024.f) * (1.f / 1024.f); }
}  // namespace
}  // namespace treeot

// Internal operator entry points used by the ABI and the IRLS solver.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace ashrt {

// Per-gather FP64 scalars of the solver, kScalStride doubles per gather.
constexpr int kScalStride = 80;
// Per-gather selection scratch (radix-select histograms), in 32-bit words.
constexpr int kSelStride = 2048;

size_t model_elems(const ashrt_plan* p);
size_t data_elems(const ashrt_plan* p);

// cg (optional): a CGLS update fused into the operator's first transform, on
// the input m (forward, mode 1) or d (adjoint, mode 2), which is then written.
cudaError_t op_forward(const ashrt_plan* p, const float* m, float* d, const float* ew_model,
                       const float* ew_data, const float* tmask, double* dot, int batch,
                       cudaStream_t s, const CgFuse* cg = nullptr);
cudaError_t op_adjoint(const ashrt_plan* p, const float* d, float* m, const float* ew_model,
                       const float* ew_data, const float* tmask, double* dot, int batch,
                       cudaStream_t s, const CgFuse* cg = nullptr);

}  // namespace ashrt

// Launch descriptors shared by the kernel translation units and the C ABI.
#pragma once
#include <cuda_runtime.h>
#include "lbm_device.cuh"
#include "step2d.cuh"

namespace lbmd {

struct Launch {
  KParams kp;
  const void* fin;
  void* fout;
  const double* rin;
  double* rout;
  StepAux aux;
  FieldOut fo;
  GradIn gi;
  cudaStream_t stream;
};

// launch one fused step (mode MODE_STEP), an observation pass (MODE_OBS) or a
// field dump (MODE_FIELDS); returns the number of CTAs through *nblocks
using StepFn = cudaError_t (*)(const Launch&, int mode, int* nblocks);

// precision index: 0 = FP64, 1 = FP32DEV with FP32 mu, 2 = FP32DEV with FP64 mu
StepFn step2d_fn(int scheme, int prec);
StepFn step3d_fn(int scheme, int prec);

}  // namespace lbmd

// FP32 grid kernels and FFT passes (PM_FP32).
#define NUPM_T float
#define NUPM_SFX _f32
#include "grid_impl.cuh"

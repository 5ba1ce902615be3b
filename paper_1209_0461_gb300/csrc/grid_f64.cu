// FP64 grid kernels and FFT passes (PM_FP64).
#define NUPM_T double
#define NUPM_SFX _f64
#include "grid_impl.cuh"

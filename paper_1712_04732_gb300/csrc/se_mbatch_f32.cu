// FP32 instantiation of the multi-system batch kernels and their launchers.
#define T_INST float
#include "se_mbatch_impl.cuh"

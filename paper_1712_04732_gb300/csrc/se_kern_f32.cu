// FP32 instantiation of the kernels and their launchers.
#define T_INST float
#include "se_kern_impl.cuh"

// FP64 instantiation of the kernels and their launchers.
#define T_INST double
#include "se_kern_impl.cuh"

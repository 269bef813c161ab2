// FP64 instantiation of the multi-system batch kernels and their launchers.
#define T_INST double
#include "se_mbatch_impl.cuh"

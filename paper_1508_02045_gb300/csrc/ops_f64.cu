// FP64 instantiation of the pass kernels and their launchers.
#include "ops_impl.cuh"
template struct hom::Ops<double>;

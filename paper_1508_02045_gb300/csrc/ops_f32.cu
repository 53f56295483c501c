// FP32 instantiation of the pass kernels and their launchers (inner solves of the
// FP32-with-FP64-refinement path).
#include "ops_impl.cuh"
template struct hom::Ops<float>;

// FP32 instantiation of the device kernels and their launchers.
#include "ops_impl.cuh"
namespace sigw {
template struct OpsRT<float>;
}

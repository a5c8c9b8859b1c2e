// m2l_rot_p16.cu -- instantiations of the rotation-accelerated M2L kernel for p = 16..16
#include "m2l_rot.cuh"

namespace gb3 {
template void rot_launch<16>(const RotArgs&, cudaStream_t);
}  // namespace gb3

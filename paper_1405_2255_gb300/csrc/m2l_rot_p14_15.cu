// m2l_rot_p14_15.cu -- instantiations of the rotation-accelerated M2L kernel for p = 14..15
#include "m2l_rot.cuh"

namespace gb3 {
template void rot_launch<14>(const RotArgs&, cudaStream_t);
template void rot_launch<15>(const RotArgs&, cudaStream_t);
}  // namespace gb3

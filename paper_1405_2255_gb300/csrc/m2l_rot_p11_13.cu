// m2l_rot_p11_13.cu -- instantiations of the rotation-accelerated M2L kernel for p = 11..13
#include "m2l_rot.cuh"

namespace gb3 {
template void rot_launch<11>(const RotArgs&, cudaStream_t);
template void rot_launch<12>(const RotArgs&, cudaStream_t);
template void rot_launch<13>(const RotArgs&, cudaStream_t);
}  // namespace gb3

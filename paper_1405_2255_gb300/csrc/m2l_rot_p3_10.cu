// m2l_rot_p3_10.cu -- instantiations of the rotation-accelerated M2L kernel for p = 3..10
#include "m2l_rot.cuh"

namespace gb3 {
template void rot_launch<3>(const RotArgs&, cudaStream_t);
template void rot_launch<4>(const RotArgs&, cudaStream_t);
template void rot_launch<5>(const RotArgs&, cudaStream_t);
template void rot_launch<6>(const RotArgs&, cudaStream_t);
template void rot_launch<7>(const RotArgs&, cudaStream_t);
template void rot_launch<8>(const RotArgs&, cudaStream_t);
template void rot_launch<9>(const RotArgs&, cudaStream_t);
template void rot_launch<10>(const RotArgs&, cudaStream_t);
}  // namespace gb3

// faces_f32.cu -- k_faces of the mixed path (FP32 reconstruction, face physics and HLLE).
#include "faces_impl.cuh"

GRS_DEFINE_LAUNCH_FACES(float)

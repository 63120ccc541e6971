// faces_f64.cu -- k_faces of the FP64 path.
#include "faces_impl.cuh"

GRS_DEFINE_LAUNCH_FACES(double)

// float32 instantiation of the SIMT kernels (the DNA_F32 form).
#include "simt_launch.cuh"

namespace dna {
template struct Simt<float>;
}

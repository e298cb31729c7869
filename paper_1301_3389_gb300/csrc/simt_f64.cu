// float64 instantiation of the SIMT kernels (the DNA_F64 form).
#include "simt_launch.cuh"

namespace dna {
template struct Simt<double>;
}
